// Reverse-mode pass through the unrolled FISTA network run by fused_solve_kernel
// with per-layer multipliers (FusedArgs::scale / ::thresh):
//   layer k:  u_k = z_k - a_k G'_k,  G'_k = mu (G z_k - b) = IFFT2(q . FFT2(z_k) - Bt),
//             c_k = S_{t_k kappa}(u_k),  z_{k+1} = c_k + beta_k (c_k - c_{k-1})     (eq:fista)
// The forward stored z_k and G'_k.  Going back from g_c = dLoss/dc_{K-1} (complex
// gradients g = dLoss/dRe + j dLoss/dIm), for k = K-1 .. 0:
//   g_u = s g_c + (theta/|u|^3) Re(conj(g_c) u) u with s = 1 - theta/|u|, theta = t_k kappa,
//         and 0 where |u| <= theta                                 (soft-threshold Jacobian)
//   dLoss/dt_k += -kappa Re(conj(g_c) u)/|u|  (active entries)
//   dLoss/da_k += -Re(conj(g_u) G'_k)
//   g_z = g_u - a_k mu G g_u      (G is Hermitian: the same BCCB product, without Bt)
//   g_{c_{k-1}} = (1 + beta_{k-1}) g_z + (carried -beta_k g_z of the layer above)
// For dLoss/dy (optional): every layer sees b = A^H y through u_k, with du_k/db = a_k mu, so
// grad_b collects sum_k a_k g_u (mu is applied afterwards), and grad_lam collects, per instance,
// sum_k t_k dLoss/dtheta_k with theta_k = t_k kappa (the threshold's dependence on b when lam is
// a fraction of ||b||_inf).
// The Gram product reuses the fused kernel's transform stages; one cluster per
// instance, the two gradient grids stay in shared memory for all K layers.
#pragma once

#include "fused_solve.cuh"

namespace bccb {

struct AdjArgs {
  const FusedInst* insts;
  const int* ids;
  const float* beta;      // FISTA momentum beta_k (length layers)
  const float2* twiddle;
  const float* mult;      // q of the forward pass
  const float* scale;     // a_k
  const float* thresh;    // t_k
  const float2* save;     // z_k at (2k) * save_stride, G'_k at (2k + 1) * save_stride
  int64_t save_stride;
  const float2* grad_c;   // dLoss/dc_{K-1}, packed like the solution
  double* grad_scale;     // += dLoss/da_k
  double* grad_thresh;    // += dLoss/dt_k
  float2* grad_b;         // nullable: sum_k a_k g_{u_k}, packed like the solution (overwritten)
  double* grad_lam;       // with grad_b: += sum_k t_k dLoss/dtheta_k per instance (zeroed by the caller)
  int layers;
  int pad_;
};

__device__ __forceinline__ void warp_add_to(double* dst, float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(dst, (double)v);
}

template <int L1, int L2, int TILE>
__global__ void __launch_bounds__(FusedShape<L1, L2, false, TILE>::T, FusedShape<L1, L2, false, TILE>::MIN_BLOCKS)
    adjoint_kernel(const AdjArgs a) {
  using S = FusedShape<L1, L2, false, TILE>;
  constexpr int C = S::C, E = S::E, T = S::T, P = S::P, NMAX = S::NMAX, R = S::R;

  extern __shared__ float4 smem_raw[];
  FusedCta<S> cta;
  char* sp = reinterpret_cast<char*>(smem_raw);
  cta.work = reinterpret_cast<float2*>(sp);
  sp += R * P * 8;
  cta.s0 = reinterpret_cast<float2*>(sp);  // g_c, then g_u
  sp += E * 8;
  cta.s1 = reinterpret_cast<float2*>(sp);  // carried momentum term
  sp += E * 8;
  cta.tw = reinterpret_cast<float2*>(sp);
  sp += NMAX * 8;
  cta.pmask = reinterpret_cast<uint16_t*>(sp);
  sp += ((S::SH * 2 + 15) / 16) * 16;
  cta.tw256 = reinterpret_cast<float2*>(sp);
  sp += 256 * 8;
  cta.tw16 = reinterpret_cast<float2*>(sp);
  sp += 16 * 8;
  cta.mtab = reinterpret_cast<float4*>(sp);
  sp += S::MCAP * 16;
  cta.poff = reinterpret_cast<uint16_t*>(sp);
  cta.tid = threadIdx.x;
  int crank = 0;
  if constexpr (C > 1) crank = (int)cg::this_cluster().block_rank();
  cta.crank = crank;

  const int inst_id = a.ids[blockIdx.x / C];
  const FusedInst in = a.insts[inst_id];
  const float kappa = in.kappa;
  const int kc = min(L1, (in.kcols + 15) & ~15);
  const float* mult = a.mult + in.g_off;
  uint32_t peer[C];
  {
    const uint32_t w = smem_addr(cta.work);
#pragma unroll
    for (int c = 0; c < C; ++c) peer[c] = (C > 1) ? cluster_map(w, c) : w;
  }
  cta.load_tables(a.twiddle, mult, nullptr, kc);
  for (int idx = threadIdx.x; idx < E; idx += T) {
    const int s = idx / L1, e = idx % L1;
    cta.s0[idx] = a.grad_c[in.c_off + (crank + C * s) * L1 + e];
    cta.s1[idx] = make_float2(0.f, 0.f);
  }
  __syncthreads();

  for (int k = a.layers - 1; k >= 0; --k) {
    const float ak = __ldg(&a.scale[k]);
    const float theta = __ldg(&a.thresh[k]) * kappa;
    const float2* zk = a.save + (int64_t)(2 * k) * a.save_stride + in.c_off;
    const float2* gk = a.save + (int64_t)(2 * k + 1) * a.save_stride + in.c_off;
    // soft-threshold Jacobian and the two scalar gradients
    float d_a = 0.f, d_t = 0.f;
    for (int idx = threadIdx.x; idx < E; idx += T) {
      const int s = idx / L1, e = idx % L1;
      const int gidx = (crank + C * s) * L1 + e;
      const float2 z = zk[gidx], g = gk[gidx];
      const float2 u = make_float2(z.x - ak * g.x, z.y - ak * g.y);
      const float2 gc = cta.s0[idx];
      float2 gu = make_float2(0.f, 0.f);
      const float r2 = u.x * u.x + u.y * u.y;
      if (r2 > theta * theta) {
        const float inv = rsqrtf(r2);
        const float sfac = 1.0f - theta * inv;
        const float proj = gc.x * u.x + gc.y * u.y;
        const float w = theta * inv * inv * inv * proj;
        gu = make_float2(sfac * gc.x + w * u.x, sfac * gc.y + w * u.y);
        d_t -= proj * inv;
      }
      d_a -= gu.x * g.x + gu.y * g.y;
      cta.s0[idx] = gu;
      cta.work[s * P + pad16(e)] = gu;
      if (a.grad_b) {
        float2* gb = a.grad_b + in.c_off + gidx;
        const float2 prev = (k == a.layers - 1) ? make_float2(0.f, 0.f) : *gb;
        *gb = make_float2(prev.x + ak * gu.x, prev.y + ak * gu.y);
      }
    }
    warp_add_to(&a.grad_scale[k], d_a);
    warp_add_to(&a.grad_thresh[k], d_t * kappa);
    if (a.grad_b) warp_add_to(&a.grad_lam[inst_id], d_t * __ldg(&a.thresh[k]));
    __syncthreads();
    // g_z = g_u - a_k mu G g_u, then the momentum chain
    const float bk = (k > 0) ? __ldg(&a.beta[k - 1]) : 0.f;
    cta.template row_fft_from<0, false>(
        [&](int row, int e, float2 x) {
          if (e < kc) cta.work[row * P + pad16(e)] = x;
        },
        L1);
    __syncthreads();
    cta.template col_dft<false>(kc);
    cluster_barrier<C>();
    cta.middle(peer, mult, nullptr, kc);
    cluster_barrier<C>();
    cta.template col_dft<true>(kc);
    __syncthreads();
    cta.template row_fft_from<0, true>(
        [&](int row, int e, float2 ggu) {
          const int sidx = row * L1 + e;
          const float2 gu = cta.s0[sidx];
          const float2 gz = make_float2(gu.x - ak * ggu.x, gu.y - ak * ggu.y);
          const float2 gn = cta.s1[sidx];
          cta.s0[sidx] = make_float2((1.0f + bk) * gz.x + gn.x, (1.0f + bk) * gz.y + gn.y);
          cta.s1[sidx] = make_float2(-bk * gz.x, -bk * gz.y);
        },
        kc);
  }
  if constexpr (C > 1) cg::this_cluster().sync();
}

struct AdjointEntry {
  int L1, L2, tile;
  cudaError_t (*launch)(const AdjArgs&, int n_inst, cudaStream_t);
  cudaError_t (*prepare)();
};

template <int L1, int L2, int TILE>
cudaError_t adjoint_prepare() {
  using S = FusedShape<L1, L2, false, TILE>;
  cudaError_t e = cudaFuncSetAttribute(adjoint_kernel<L1, L2, TILE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       S::SMEM);
  if (e == cudaSuccess && S::C > 8)
    e = cudaFuncSetAttribute(adjoint_kernel<L1, L2, TILE>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

template <int L1, int L2, int TILE>
cudaError_t adjoint_launch(const AdjArgs& a, int n_inst, cudaStream_t st) {
  using S = FusedShape<L1, L2, false, TILE>;
  if (n_inst <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n_inst * S::C), 1, 1);
  cfg.blockDim = dim3(S::T, 1, 1);
  cfg.dynamicSmemBytes = S::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = S::C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, adjoint_kernel<L1, L2, TILE>, a);
}

template <int L1, int L2, int TILE = kFusedTileElems>
AdjointEntry adjoint_entry() {
  return AdjointEntry{L1, L2, TILE, &adjoint_launch<L1, L2, TILE>, &adjoint_prepare<L1, L2, TILE>};
}

}  // namespace bccb
