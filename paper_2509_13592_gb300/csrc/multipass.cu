// Multi-pass ISTA / FISTA / ADMM solver for grids the fused on-chip kernel does not
// hold (L_i up to 1024) and for the FP64 solve path.  Same iteration as the fused
// kernel (Section III-B, eq:Rc with eq:ista / eq:fista / eq:admm):
//     u = x - IFFT2(q . FFT2(x) - Bt)   (the identity part never enters the FFT)
// but with the grid in global memory (L2-resident at 1024 x 1024 in FP32) and two
// kernels per iteration:
//   column pass: forward column DFTs, q . X - Bt, inverse column DFTs, for the
//                Fourier columns p1 < kcols only (the spectrum vanishes beyond);
//   row pass:    inverse row DFTs (columns >= kcols read as zero), the pointwise
//                update of the state, and the next iteration's forward row DFTs.
// V = float2 (complex64) or double2 (complex128); transforms are radix-4 Stockham
// stages (one radix-2 stage for odd log2 n) staged in shared memory.
#include "fft_smem.cuh"
#include "solver.h"

namespace bccb {
namespace {

template <typename V>
struct MpArgs {
  const InstDesc* desc;
  const int* ids;
  const InstParams* par;
  const FusedInst* fused;  // kcols
  V* work;
  V* s0;  // c (ISTA/FISTA) or z (ADMM)
  V* s1;  // z (FISTA) or v (ADMM)
  const typename ScalarOf<V>::T* mult;
  const V* bt;
  const V* tw;  // W_1024^e
  const typename ScalarOf<V>::T* beta;
  const V* c0;
  V* c_out;
  V* aux;
  uint2* lo;  // FP32 ISTA/FISTA: low-order parts {c_lo, z_lo} (bf16 pairs), packed like c_out
  int algo;  // 0 ISTA, 1 FISTA, 2 ADMM
  int it;
  int last;
  double rho;
};

template <typename V>
__device__ __forceinline__ V shrink(V u, typename ScalarOf<V>::T kappa) {
  using T = typename ScalarOf<V>::T;
  const T r2 = u.x * u.x + u.y * u.y;
  if (r2 > kappa * kappa) {
    const T s = (T)1 - kappa / sqrt(r2);
    return cmk<V>(u.x * s, u.y * s);
  }
  return cmk<V>((T)0, (T)0);
}

template <typename T, typename V>
__device__ __forceinline__ T shrink_scale(V u, T kappa) {
  const T r2 = u.x * u.x + u.y * u.y;
  return r2 > kappa * kappa ? (T)1 - kappa / sqrt(r2) : (T)0;
}

__device__ __forceinline__ int active_cols(int kcols, int L1) { return min(L1, (kcols + 3) & ~3); }

// state <- warm start (or zero); work row input of the first forward row pass is built there too
template <typename V>
__global__ void mp_init_kernel(MpArgs<V> a) {
  using T = typename ScalarOf<V>::T;
  const int inst = a.ids[blockIdx.x];
  const InstDesc d = a.desc[inst];
  const int L = d.L1 * d.L2;
  for (int cell = blockIdx.y * blockDim.x + threadIdx.x; cell < L; cell += gridDim.y * blockDim.x) {
    const V x = a.c0 ? a.c0[d.c_off + cell] : cmk<V>((T)0, (T)0);
    a.s0[d.g_off + cell] = x;
    a.s1[d.g_off + cell] = (a.algo == 2) ? cmk<V>((T)0, (T)0) : x;
  }
}

// MODE 0: forward row DFTs of the initial input; 1: inverse row DFTs, update, forward row
// DFTs of the next input; 2: inverse row DFTs and update (last iteration)
template <typename V, int MODE>
__global__ void mp_rows_kernel(MpArgs<V> a) {
  using T = typename ScalarOf<V>::T;
  const int inst = a.ids[blockIdx.x];
  const InstDesc d = a.desc[inst];
  const int row = blockIdx.y;
  if (row >= d.L2) return;
  const int L1 = d.L1;
  const int kc = active_cols(a.fused[inst].kcols, L1);
  extern __shared__ unsigned char mp_sm[];
  V* x = reinterpret_cast<V*>(mp_sm);
  V* y = x + L1;
  V* work = a.work + d.g_off + (int64_t)row * L1;
  V* s0 = a.s0 + d.g_off + (int64_t)row * L1;
  V* s1 = a.s1 + d.g_off + (int64_t)row * L1;
  V* res = x;
  if (MODE == 0) {
    for (int e = threadIdx.x; e < L1; e += blockDim.x)
      x[e] = (a.algo == 2) ? csub(s0[e], s1[e]) : (a.algo == 1 ? s1[e] : s0[e]);
    __syncthreads();
  } else {
    for (int e = threadIdx.x; e < L1; e += blockDim.x) x[e] = (e < kc) ? work[e] : cmk<V>((T)0, (T)0);
    __syncthreads();
    res = fft_smem<V, true>(x, y, L1, 1, a.tw);
    const InstParams p = a.par[inst];
    const T kappa = (T)(a.algo == 2 ? p.lam / a.rho : p.mu * p.lam);
    const T beta = (a.algo == 1) ? a.beta[a.it] : (T)0;
    V* aux = a.aux ? a.aux + d.c_off + (int64_t)row * L1 : nullptr;
    const bool outside_rows = d.bL1 != 0 && row >= d.bL2;
    for (int e = threadIdx.x; e < L1; e += blockDim.x) {
      const V g = res[e];
      V next;
      if (d.bL1 != 0 && (outside_rows || e >= d.bL1)) {
        // outside the unknown block of a circulant embedding: stays 0
        s0[e] = cmk<V>((T)0, (T)0);
        s1[e] = cmk<V>((T)0, (T)0);
        next = cmk<V>((T)0, (T)0);
      } else if (a.algo != 2 && a.lo) {
        if constexpr (sizeof(T) == 4) {
          // FP32: the state in compensated form, as in the fused kernel (c = s0 + c_lo, z = s1 +
          // z_lo; double-float u, soft-threshold and momentum; ISTA is FISTA with beta = 0, so s1
          // holds z = c).  The low parts are read only where the state is nonzero and are zero in
          // the first iteration (an exact warm start).
          const V c_old = s0[e];
          const V xin = s1[e];
          const bool live = (c_old.x != 0.f) | (c_old.y != 0.f) | (xin.x != 0.f) | (xin.y != 0.f);
          uint2* const lp = a.lo + d.c_off + (int64_t)row * L1 + e;
          if (!live && !(g.x * g.x + g.y * g.y > kappa * kappa)) {
            next = cmk<V>((T)0, (T)0);
          } else {
            float2 cl = make_float2(0.f, 0.f), zl = make_float2(0.f, 0.f);
            if (live && a.it > 0) {
              const uint2 w = *lp;
              cl = unpack_bf16x2(w.x);
              zl = unpack_bf16x2(w.y);
            }
            float uxh, uxl, uyh, uyl;
            dd_add(xin.x, zl.x, -g.x, 0.f, uxh, uxl);
            dd_add(xin.y, zl.y, -g.y, 0.f, uyh, uyl);
            float cxh = 0.f, cxl = 0.f, cyh = 0.f, cyl = 0.f;
            const float r2 = uxh * uxh + uyh * uyh;
            if (r2 > kappa * kappa) {
              const float kr = kappa * rsqrtf(r2);
              dd_add(uxh, uxl, -(kr * uxh), 0.f, cxh, cxl);
              dd_add(uyh, uyl, -(kr * uyh), 0.f, cyh, cyl);
            }
            float dxh, dxl, dyh, dyl;
            dd_add(cxh, cxl, -c_old.x, -cl.x, dxh, dxl);
            dd_add(cyh, cyl, -c_old.y, -cl.y, dyh, dyl);
            float zxh, zxl, zyh, zyl;
            dd_axpy(beta, dxh, dxl, cxh, cxl, zxh, zxl);
            dd_axpy(beta, dyh, dyl, cyh, cyl, zyh, zyl);
            s0[e] = cmk<V>(cxh, cyh);
            s1[e] = cmk<V>(zxh, zyh);
            if ((cxh != 0.f) | (cyh != 0.f) | (zxh != 0.f) | (zyh != 0.f))
              *lp = make_uint2(pack_bf16x2(cxl, cyl), pack_bf16x2(zxl, zyl));
            next = cmk<V>(zxh, zyh);
          }
        }
      } else if (a.algo != 2) {
        const V c_old = s0[e];
        const V xin = (a.algo == 1) ? s1[e] : c_old;
        const V un = csub(xin, g);
        const T sc = shrink_scale(un, kappa);
        const V cn = cmk<V>(un.x * sc, un.y * sc);
        s0[e] = cn;
        if (a.algo == 1) {
          // momentum difference from the unrounded product u s (see the fused kernel)
          const T dx = fma(un.x, sc, -c_old.x), dy = fma(un.y, sc, -c_old.y);
          next = cmk<V>(fma(beta, dx, cn.x), fma(beta, dy, cn.y));
          s1[e] = next;
        } else {
          next = cn;
        }
      } else {
        const V zo = s0[e], vo = s1[e];
        const V un = csub(zo, g);  // c^(t+1) + v^(t)
        const V zn = shrink(un, kappa);
        const V vn = csub(un, zn);
        s0[e] = zn;
        s1[e] = vn;
        next = csub(zn, vn);
        if (MODE == 2 && aux) aux[e] = csub(un, vo);
      }
      res[e] = next;
    }
    __syncthreads();
  }
  if (MODE != 2) {
    V* other = (res == x) ? y : x;
    V* out = fft_smem<V, false>(res, other, L1, 1, a.tw);
    for (int e = threadIdx.x; e < kc; e += blockDim.x) work[e] = out[e];
  }
}

// columns c0 .. c0 + cnt - 1 (< kcols): forward DFT over the column, q . X - Bt, inverse DFT
template <typename V>
__global__ void mp_cols_kernel(MpArgs<V> a, int cpb) {
  const int inst = a.ids[blockIdx.x];
  const InstDesc d = a.desc[inst];
  const int kc = active_cols(a.fused[inst].kcols, d.L1);
  const int c0 = blockIdx.y * cpb;
  if (c0 >= kc) return;
  const int cnt = min(cpb, kc - c0);
  extern __shared__ unsigned char mp_sm[];
  V* x = reinterpret_cast<V*>(mp_sm);
  V* y = x + d.L2 * cpb;
  V* work = a.work + d.g_off;
  for (int idx = threadIdx.x; idx < d.L2 * cnt; idx += blockDim.x) {
    const int e = idx / cnt, q = idx % cnt;
    x[idx] = work[(int64_t)e * d.L1 + c0 + q];
  }
  __syncthreads();
  V* r = fft_smem<V, false>(x, y, d.L2, cnt, a.tw);
  for (int idx = threadIdx.x; idx < d.L2 * cnt; idx += blockDim.x) {
    const int e = idx / cnt, q = idx % cnt;
    const int64_t f = d.g_off + (int64_t)e * d.L1 + c0 + q;
    const auto m = a.mult[f];
    const V b = a.bt[f];
    const V v = r[idx];
    r[idx] = cmk<V>(v.x * m - b.x, v.y * m - b.y);
  }
  __syncthreads();
  V* other = (r == x) ? y : x;
  V* out = fft_smem<V, true>(r, other, d.L2, cnt, a.tw);
  for (int idx = threadIdx.x; idx < d.L2 * cnt; idx += blockDim.x) {
    const int e = idx / cnt, q = idx % cnt;
    work[(int64_t)e * d.L1 + c0 + q] = out[idx];
  }
}

template <typename V>
__global__ void mp_output_kernel(MpArgs<V> a) {
  const int inst = a.ids[blockIdx.x];
  const InstDesc d = a.desc[inst];
  const int L = d.L1 * d.L2;
  for (int cell = blockIdx.y * blockDim.x + threadIdx.x; cell < L; cell += gridDim.y * blockDim.x)
    a.c_out[d.c_off + cell] = a.s0[d.g_off + cell];
}

constexpr int kMpThreads = 256;

int mp_cols_per_block(int max_L2, int vbytes) {
  // two L2 x cpb tiles within 96 KB
  int cpb = 16;
  while (cpb > 1 && 2 * max_L2 * cpb * vbytes > 96 * 1024) cpb >>= 1;
  return cpb;
}

template <typename V>
cudaError_t run_t(bccb_solver* s, const int* ids, int count, int iters, const void* c0, void* c_out, void* aux,
                  cudaStream_t st) {
  using T = typename ScalarOf<V>::T;
  MpArgs<V> a{};
  a.desc = s->d_desc;
  a.ids = ids;
  a.par = s->d_par;
  a.fused = s->d_fused;
  a.work = static_cast<V*>(s->d_mp_work);
  a.s0 = static_cast<V*>(s->d_mp_s0);
  a.s1 = static_cast<V*>(s->d_mp_s1);
  if constexpr (sizeof(T) == 8) {
    a.mult = s->d_mult64;
    a.bt = s->d_bt64;
    a.tw = s->d_tw64;
    a.beta = s->d_beta64;
  } else {
    a.mult = s->d_mult;
    a.bt = s->d_cterm;
    a.tw = s->d_tw32;
    a.beta = s->d_beta;
  }
  a.c0 = static_cast<const V*>(c0);
  a.c_out = static_cast<V*>(c_out);
  a.aux = static_cast<V*>(aux);
  a.algo = s->algo;
  a.rho = s->rho;
  if constexpr (sizeof(T) == 4) a.lo = (s->algo != 2) ? s->d_lo : nullptr;
  const int cells = s->max_L1 * s->max_L2;
  const dim3 gcell((unsigned)count, (unsigned)min(64, (cells + kMpThreads - 1) / kMpThreads));
  const dim3 grow((unsigned)count, (unsigned)s->max_L2);
  // a handful of instances: one column per block, so the few active columns still spread over many SMs
  const int cpb = count <= 8 ? 1 : mp_cols_per_block(s->max_L2, (int)sizeof(V));
  const dim3 gcol((unsigned)count, (unsigned)((s->max_L1 + cpb - 1) / cpb));
  const size_t sm_row = 2 * (size_t)s->max_L1 * sizeof(V);
  const size_t sm_col = 2 * (size_t)s->max_L2 * cpb * sizeof(V);
  mp_init_kernel<V><<<gcell, kMpThreads, 0, st>>>(a);
  mp_rows_kernel<V, 0><<<grow, kMpThreads, sm_row, st>>>(a);
  s->launches += 2;
  for (int it = 0; it < iters; ++it) {
    a.it = it;
    mp_cols_kernel<V><<<gcol, kMpThreads, sm_col, st>>>(a, cpb);
    if (it + 1 < iters)
      mp_rows_kernel<V, 1><<<grow, kMpThreads, sm_row, st>>>(a);
    else
      mp_rows_kernel<V, 2><<<grow, kMpThreads, sm_row, st>>>(a);
    s->launches += 2;
  }
  mp_output_kernel<V><<<gcell, kMpThreads, 0, st>>>(a);
  s->launches += 1;
  return cudaGetLastError();
}

template <typename V>
cudaError_t prepare_t(int max_L1, int max_L2) {
  const int cpb = mp_cols_per_block(max_L2, (int)sizeof(V));
  const int sm_col = 2 * max_L2 * cpb * (int)sizeof(V);
  const int sm_row = 2 * max_L1 * (int)sizeof(V);
  cudaError_t e = cudaFuncSetAttribute(mp_cols_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_col);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mp_rows_kernel<V, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_row);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mp_rows_kernel<V, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_row);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mp_rows_kernel<V, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_row);
  return e;
}

}  // namespace

cudaError_t prepare_multipass(bccb_solver* s) {
  return s->prec == 1 ? prepare_t<double2>(s->max_L1, s->max_L2) : prepare_t<float2>(s->max_L1, s->max_L2);
}

cudaError_t run_multipass(bccb_solver* s, const int* ids, int count, int iters, const void* c0, void* c_out,
                          void* aux, cudaStream_t stream) {
  if (s->prec == 1) return run_t<double2>(s, ids, count, iters, c0, c_out, aux, stream);
  return run_t<float2>(s, ids, count, iters, c0, c_out, aux, stream);
}

}  // namespace bccb
