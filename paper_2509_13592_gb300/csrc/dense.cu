// The "regular" implementation of ISTA / FISTA / ADMM: every iteration multiplies by
// the stored dense L x L Gram matrix G = D_s^H D_s (Section II-B, eq:ista, eq:fista,
// eq:admm, whose dominant term is this O(L^2) product), for the t_reg / t_fast
// comparison of Section III-C on the GPU.
//
// The identity part of each iteration matrix is applied exactly and only G is stored:
//   ISTA/FISTA:  (I - mu G) x + mu b       = x - mu (G x) + mu b
//   ADMM:        (G + rho I)^{-1}(b + rho w), with D_s D_s^H = L I (no fold: M_i <= L_i)
//                = w - (G w)/(rho + L) + b/(rho + L)        (w = z - v)
// the second line by the Woodbury identity (G + rho I)^{-1} = (I - G/(rho + L))/rho and
// G b = D^H (D D^H) y = L b.
//
// G[l, l'] = g(l - l') with g(d1, d2) = sum_n exp(+j 2 pi (d1 m1_n / L1 + d2 m2_n / L2))
// (indices mod L_i), evaluated in FP64 from that definition and stored as complex64,
// row-major, one L x L block per instance.  One launch per iteration: a warp per output
// row streams its row of G (HBM-bound GEMV) and applies the pointwise update; the
// input vector x is double-buffered because every row reads all of it.
#include <stdint.h>

#include "solver.h"

namespace bccb {
namespace {

constexpr int kDenseWarps = 8;

// first column g of G, FP64, per instance (one thread per lag d = d1 + d2 L1)
__global__ void dense_gcol_kernel(const InstDesc* __restrict__ desc, const int* __restrict__ mask_idx,
                                  const int64_t* __restrict__ gcol_off, double2* gcol) {
  const InstDesc d = desc[blockIdx.y];
  const int L = d.L1 * d.L2;
  const int* mi = mask_idx + d.mask_off;
  for (int lag = blockIdx.x * blockDim.x + threadIdx.x; lag < L; lag += gridDim.x * blockDim.x) {
    const int64_t d1 = lag % d.L1, d2 = lag / d.L1;
    double re = 0.0, im = 0.0;
    for (int m2 = 0; m2 < d.M2; ++m2)
      for (int m1 = 0; m1 < d.M1; ++m1) {
        if (mi[m1 + m2 * d.M1] < 0) continue;
        // phase 2 pi (d1 m1 / L1 + d2 m2 / L2) = 2 pi k / L with an exact integer k
        const int64_t k = ((d1 * m1) % d.L1) * d.L2 + ((d2 * m2) % d.L2) * d.L1;
        double s, c;
        sincospi(2.0 * (double)(k % L) / (double)L, &s, &c);
        re += c;
        im += s;
      }
    gcol[gcol_off[blockIdx.y] + lag] = make_double2(re, im);
  }
}

// G[l, l'] = g(l - l') as complex64, row-major
__global__ void dense_expand_kernel(const InstDesc* __restrict__ desc, const int64_t* __restrict__ gcol_off,
                                    const double2* __restrict__ gcol, const int64_t* __restrict__ gram_off,
                                    float2* gram) {
  const InstDesc d = desc[blockIdx.y];
  const int64_t L = (int64_t)d.L1 * d.L2;
  const double2* g = gcol + gcol_off[blockIdx.y];
  float2* G = gram + gram_off[blockIdx.y];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < L * L; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = e / L, lp = e % L;
    const int d1 = (int)(((l % d.L1) - (lp % d.L1) + d.L1) % d.L1);
    const int d2 = (int)(((l / d.L1) - (lp / d.L1) + d.L2) % d.L2);
    const double2 v = g[d1 + (int64_t)d2 * d.L1];
    G[e] = make_float2((float)v.x, (float)v.y);
  }
}

// per cell: the constant term (mu b, or b/(rho + L) for ADMM) and the initial state
__global__ void dense_init_kernel(const InstDesc* __restrict__ desc, const InstParams* __restrict__ par,
                                  const double2* __restrict__ b64, const float2* __restrict__ c0, int admm,
                                  double rho, float2* kterm, float2* s0, float2* s1, float2* x) {
  const InstDesc d = desc[blockIdx.y];
  const int L = d.L1 * d.L2;
  const double scale = admm ? 1.0 / (rho + (double)L) : par[blockIdx.y].mu;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < L; l += gridDim.x * blockDim.x) {
    const int64_t gi = d.c_off + l;
    const double2 b = b64[d.g_off + l];
    kterm[gi] = make_float2((float)(scale * b.x), (float)(scale * b.y));
    const float2 c = c0 ? c0[gi] : make_float2(0.f, 0.f);
    s0[gi] = c;                                   // c^(0) (ISTA/FISTA) or z^(0) (ADMM)
    s1[gi] = admm ? make_float2(0.f, 0.f) : c;   // unused (FISTA keeps c only) or v^(0) = 0
    x[gi] = c;                                    // z^(1) = c^(0), or z^(0) - v^(0)
  }
}

struct DenseArgs {
  const InstDesc* desc;
  const InstParams* par;
  const FusedInst* fused;  // kappa
  const int64_t* gram_off;
  const float2* gram;
  const float2* kterm;
  const float2* x_in;
  float2* x_out;
  float2* s0;  // c (ISTA/FISTA) or z (ADMM), updated in place
  float2* s1;  // v (ADMM), updated in place
  float2* aux_out;  // ADMM, last iteration: c^(T) (nullable)
  const float* beta;
  int it;
  int last;
  double rho;
};

__device__ __forceinline__ float2 soft_thr(float2 u, float kappa) {
  const float r2 = u.x * u.x + u.y * u.y;
  if (!(r2 > kappa * kappa)) return make_float2(0.f, 0.f);
  const float s = 1.0f - kappa * rsqrtf(r2);
  return make_float2(u.x * s, u.y * s);
}

// x is staged through shared memory in chunks of kDenseChunk entries that all eight row
// warps of the CTA use, so that L2 carries x once per CTA rather than once per row
constexpr int kDenseChunk = 4096;  // complex entries (32 KB)

template <bool ADMM>
__global__ void __launch_bounds__(32 * kDenseWarps) dense_iter_kernel(const DenseArgs a) {
  __shared__ float4 xs[kDenseChunk / 2];
  const InstDesc d = a.desc[blockIdx.y];
  const int L = d.L1 * d.L2;
  const int lane = threadIdx.x & 31;
  const int row0 = blockIdx.x * kDenseWarps;
  if (row0 >= L) return;  // uniform over the CTA
  const int row = row0 + (threadIdx.x >> 5);
  const bool live = row < L;
  const float4* G = reinterpret_cast<const float4*>(a.gram + a.gram_off[blockIdx.y] + (int64_t)(live ? row : row0) * L);
  const float4* X = reinterpret_cast<const float4*>(a.x_in + d.c_off);
  // two complex entries per 16-byte load
  float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
  const int nq = L >> 1;
  for (int base = 0; base < nq; base += kDenseChunk / 2) {
    const int cq = min(kDenseChunk / 2, nq - base);
    __syncthreads();
    for (int q = threadIdx.x; q < cq; q += 32 * kDenseWarps) xs[q] = __ldg(&X[base + q]);
    __syncthreads();
    int q = lane;
    for (; q + 7 * 32 < cq; q += 8 * 32) {
      float4 g[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) g[k] = __ldg(&G[base + q + 32 * k]);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float4 x = xs[q + 32 * k];
        acc0.x = fmaf(g[k].x, x.x, acc0.x);
        acc0.x = fmaf(-g[k].y, x.y, acc0.x);
        acc0.y = fmaf(g[k].x, x.y, acc0.y);
        acc0.y = fmaf(g[k].y, x.x, acc0.y);
        acc1.x = fmaf(g[k].z, x.z, acc1.x);
        acc1.x = fmaf(-g[k].w, x.w, acc1.x);
        acc1.y = fmaf(g[k].z, x.w, acc1.y);
        acc1.y = fmaf(g[k].w, x.z, acc1.y);
      }
    }
    for (; q < cq; q += 32) {
      const float4 g = __ldg(&G[base + q]), x = xs[q];
      acc0.x = fmaf(g.x, x.x, acc0.x);
      acc0.x = fmaf(-g.y, x.y, acc0.x);
      acc0.y = fmaf(g.x, x.y, acc0.y);
      acc0.y = fmaf(g.y, x.x, acc0.y);
      acc1.x = fmaf(g.z, x.z, acc1.x);
      acc1.x = fmaf(-g.w, x.w, acc1.x);
      acc1.y = fmaf(g.z, x.w, acc1.y);
      acc1.y = fmaf(g.w, x.z, acc1.y);
    }
  }
  if (!live) return;
  float gx = acc0.x + acc1.x, gy = acc0.y + acc1.y;
  for (int o = 16; o > 0; o >>= 1) {
    gx += __shfl_xor_sync(0xffffffffu, gx, o);
    gy += __shfl_xor_sync(0xffffffffu, gy, o);
  }
  if (lane != 0) return;
  const int64_t gi = d.c_off + row;
  const float2 xv = a.x_in[gi], k = a.kterm[gi];
  const float kappa = a.fused[blockIdx.y].kappa;
  if constexpr (!ADMM) {
    const float mu = (float)a.par[blockIdx.y].mu;
    const float2 u = make_float2(xv.x - mu * gx + k.x, xv.y - mu * gy + k.y);
    const float2 c_old = a.s0[gi];
    const float r2 = u.x * u.x + u.y * u.y;
    const float sc = r2 > kappa * kappa ? 1.0f - kappa * rsqrtf(r2) : 0.0f;
    const float2 cn = make_float2(u.x * sc, u.y * sc);
    const float beta = a.beta ? a.beta[a.it] : 0.f;
    a.s0[gi] = cn;
    // momentum difference from the unrounded product u s (one rounding)
    const float dx = fmaf(u.x, sc, -c_old.x), dy = fmaf(u.y, sc, -c_old.y);
    a.x_out[gi] = make_float2(fmaf(beta, dx, cn.x), fmaf(beta, dy, cn.y));
  } else {
    const float sc = (float)(1.0 / (a.rho + (double)L));
    const float2 c = make_float2(xv.x - sc * gx + k.x, xv.y - sc * gy + k.y);
    const float2 v = a.s1[gi];
    const float2 cv = make_float2(c.x + v.x, c.y + v.y);
    const float2 zn = soft_thr(cv, kappa);
    const float2 vn = make_float2(cv.x - zn.x, cv.y - zn.y);
    a.s0[gi] = zn;
    a.s1[gi] = vn;
    a.x_out[gi] = make_float2(zn.x - vn.x, zn.y - vn.y);
    if (a.last && a.aux_out) a.aux_out[gi] = c;
  }
}

__global__ void dense_out_kernel(const InstDesc* __restrict__ desc, const float2* __restrict__ s0, float2* c_out) {
  const InstDesc d = desc[blockIdx.y];
  const int L = d.L1 * d.L2;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < L; l += gridDim.x * blockDim.x)
    c_out[d.c_off + l] = s0[d.c_off + l];
}

}  // namespace

cudaError_t dense_prepare(bccb_solver* s) {
  cudaError_t e;
  std::vector<int64_t> gcol_off(s->n), gram_off(s->n);
  int64_t gsum = 0, msum = 0;
  for (int i = 0; i < s->n; ++i) {
    const int64_t L = (int64_t)s->h_desc[i].L1 * s->h_desc[i].L2;
    gcol_off[i] = gsum;
    gram_off[i] = msum;
    gsum += L;
    msum += L * L;
  }
  double2* d_gcol = nullptr;
  int64_t* d_gcol_off = nullptr;
  if ((e = cudaMalloc(&d_gcol, sizeof(double2) * gsum)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&d_gcol_off, sizeof(int64_t) * s->n)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&s->d_gram_off, sizeof(int64_t) * s->n)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&s->d_gram, sizeof(float2) * msum)) != cudaSuccess) return e;
  const size_t cb = sizeof(float2) * (size_t)s->total_c;
  if ((e = cudaMalloc(&s->d_dense_k, cb)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&s->d_dense_s0, cb)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&s->d_dense_s1, cb)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&s->d_dense_x[0], cb)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&s->d_dense_x[1], cb)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(d_gcol_off, gcol_off.data(), sizeof(int64_t) * s->n, cudaMemcpyHostToDevice, s->stream)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(s->d_gram_off, gram_off.data(), sizeof(int64_t) * s->n, cudaMemcpyHostToDevice,
                           s->stream)) != cudaSuccess)
    return e;
  const int maxL = s->max_L1 * s->max_L2;
  dense_gcol_kernel<<<dim3((maxL + 255) / 256, s->n), 256, 0, s->stream>>>(s->d_desc, s->d_mask_idx, d_gcol_off,
                                                                          d_gcol);
  dense_expand_kernel<<<dim3(4096, s->n), 256, 0, s->stream>>>(s->d_desc, d_gcol_off, d_gcol, s->d_gram_off,
                                                               s->d_gram);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return e;
  cudaFree(d_gcol);
  cudaFree(d_gcol_off);
  s->dense_bytes = sizeof(float2) * msum;
  return cudaSuccess;
}

cudaError_t run_dense(bccb_solver* s, int iters, const void* c0, void* c_out, void* aux) {
  const int maxL = s->max_L1 * s->max_L2;
  const bool admm = s->algo == 2;
  dense_init_kernel<<<dim3((maxL + 255) / 256, s->n), 256, 0, s->stream>>>(
      s->d_desc, s->d_par, s->d_b64, reinterpret_cast<const float2*>(c0), admm ? 1 : 0, s->rho, s->d_dense_k,
      s->d_dense_s0, s->d_dense_s1, s->d_dense_x[0]);
  s->launches += 1;
  DenseArgs a{};
  a.desc = s->d_desc;
  a.par = s->d_par;
  a.fused = s->d_fused;
  a.gram_off = s->d_gram_off;
  a.gram = s->d_gram;
  a.kterm = s->d_dense_k;
  a.s0 = s->d_dense_s0;
  a.s1 = s->d_dense_s1;
  a.aux_out = reinterpret_cast<float2*>(aux);
  a.beta = admm ? nullptr : s->d_beta;
  a.rho = s->rho;
  const dim3 grid((maxL + kDenseWarps - 1) / kDenseWarps, s->n);
  for (int it = 0; it < iters; ++it) {
    a.x_in = s->d_dense_x[it & 1];
    a.x_out = s->d_dense_x[(it + 1) & 1];
    a.it = it;
    a.last = it == iters - 1;
    if (admm)
      dense_iter_kernel<true><<<grid, 32 * kDenseWarps, 0, s->stream>>>(a);
    else
      dense_iter_kernel<false><<<grid, 32 * kDenseWarps, 0, s->stream>>>(a);
  }
  s->launches += iters;
  dense_out_kernel<<<dim3((maxL + 255) / 256, s->n), 256, 0, s->stream>>>(s->d_desc, s->d_dense_s0,
                                                                          reinterpret_cast<float2*>(c_out));
  s->launches += 1;
  return cudaGetLastError();
}

}  // namespace bccb
