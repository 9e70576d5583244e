// Fused on-chip ISTA / FISTA / ADMM solver for one L2 x L1 grid per thread-block
// cluster (FP32, complex64 state).
//
// Each iteration applies the BCCB Gram operator through the 2D FFT (Section
// III-B, eq:Rc).  The identity part of the iteration matrix never goes through
// the FFT: with G' = IFFT2(q . FFT2(x) - Bt) (unnormalised inverse),
//   ISTA/FISTA (eq:ista, eq:fista): q = mu Lambda/L, Bt = mu FFT2(b)/L, x = z^(t):
//       u = z^(t) - G'  ( = (I - mu G) z^(t) + mu b ),  c^(t) = S_kappa(u),
//       z^(t+1) = c^(t) + beta_t (c^(t) - c^(t-1));  ISTA has z^(t) = c^(t-1), beta = 0.
//   ADMM (eq:admm):  q = Lambda/(Lambda + rho)/L, Bt = FFT2(b)/(Lambda + rho)/L, x = z - v:
//       u = z^(t) - G'  ( = c^(t+1) + v^(t) ),  z^(t+1) = S_kappa(u),  v^(t+1) = u - z^(t+1).
// The subtraction b - G x happens in the Fourier domain, where its operands are of
// the size of the data residual, and directions the Gram does not see pass through
// exactly; both keep FP32 round-off from being amplified by FISTA's momentum.
// q and Bt vanish off the element mask (Lambda = 0), so the middle stage skips
// those frequencies.
//
// Layout.  The grid is stored L2 rows x L1 columns, row-major (the paper's
// vec(C) with C in C^{L1 x L2}, Section III-B).  A cluster of C CTAs owns one
// instance; CTA c keeps global rows c + C*s (s = 0..R-1, R = L2/C) in shared
// memory for the whole solve, so the iterations never touch HBM except for the
// nonzero Fourier-domain multiplier entries, read through L2.
//
// Transform.  Row DFTs (length L1) are local.  The column DFT of length L2 is
// split as L2 = Q * R' (decimation in time): group g = c + C*v (v < Q/C) holds
// the rows g + Q*t; every CTA runs the R'-point DFTs of its groups locally, then
// the final radix-Q stage combines one value from each group.  That stage is the
// only cross-CTA step: each CTA takes a 1/C share of the (frequency k1, column)
// pairs, gathers its Q operands from the cluster's shared memory (DSMEM), runs
// the forward radix-Q butterfly, multiplies by m, runs the inverse radix-Q
// butterfly and scatters the results back.  Two cluster barriers per iteration.
// Local DFTs are in-place Stockham stages (radix 16, last stage 2/4/8/16) with
// the operands staged in registers; shared rows are padded by one element per
// 16 to keep the strided stage writes free of bank conflicts.
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace bccb {

struct FusedInst {
  int64_t g_off;  // offset of this instance's grids in FusedArgs::mult / ::bt
  int64_t c_off;  // offset of this instance's solution in c_out / aux_out / c0
  float kappa;    // threshold mu*lam (ISTA/FISTA) or lam/rho (ADMM), set by the setup kernels
  int pad_;
};

struct FusedArgs {
  const FusedInst* insts;  // device array of instances
  const int* ids;          // instance index for cluster k = blockIdx.x / C
  const float* beta;       // FISTA momentum beta_t (length iters); nullptr for ISTA
  const float2* twiddle;   // W_1024^e, e = 0..1023 (float2)
  const float* mult;       // Fourier multiplier q (includes 1/(L1 L2)), natural order [p2][p1]
  const float2* bt;        // Fourier-domain constant term Bt, natural order [p2][p1]
  const float2* c0;        // warm start (z^(0) for ADMM) or nullptr for zeros
  float2* c_out;           // c^(T) (ISTA/FISTA) or z^(T) (ADMM)
  float2* aux_out;         // ADMM only: c^(T); nullable
  int iters;
  int pad_;
};

__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }

// Elements of the grid held by one CTA: at most 8192 (64 KB of complex64).
constexpr int kFusedTileElems = 8192;

template <int L1_, int L2_, bool ADMM_>
struct FusedShape {
  static constexpr int L1 = L1_, L2 = L2_;
  static constexpr bool ADMM = ADMM_;
  static constexpr int C = cmax(1, (L1 * L2) / kFusedTileElems);  // CTAs per cluster
  static constexpr int R = L2 / C;                                // rows per CTA
  static constexpr int E = R * L1;                                // elements per CTA
  static constexpr int T = cmax(32, E / 16);                      // threads per CTA
  static constexpr int Q = cmin(16, L2);                          // cross-group radix
  static constexpr int QV = Q / C;                                // groups per CTA
  static constexpr int RP = L2 / Q;                               // local column DFT length
  static constexpr int P = L1 + L1 / 16;                          // padded row pitch
  static constexpr int NMAX = cmax(L1, L2);
  static constexpr int SH = RP * L1 / C;                          // middle-stage pairs per CTA
  // work (padded) + two state grids + a flag byte per owned frequency + twiddles
  static constexpr int SMEM = (R * P + 2 * E) * 8 + E + NMAX * 8;
  static_assert(L1 >= 16 && L2 >= 16, "fused path needs L1, L2 >= 16");
  static_assert(C <= 8, "cluster larger than 8 CTAs");
  static_assert(QV * C == Q, "cluster size must divide the cross-group radix");
  static_assert(SH * C == RP * L1, "middle-stage pairs must split evenly");
  static_assert(E % 16 == 0, "tile");
};

__device__ __forceinline__ int pad16(int e) { return e + (e >> 4); }

__device__ __forceinline__ float2 soft_threshold(float2 u, float kappa) {
  // S_kappa(u) = u * max(1 - kappa/|u|, 0); |u| <= kappa -> exactly 0
  float r2 = u.x * u.x + u.y * u.y;
  if (r2 > kappa * kappa) {
    float s = 1.0f - kappa * rsqrtf(r2);
    return make_float2(u.x * s, u.y * s);
  }
  return make_float2(0.0f, 0.0f);
}

template <typename S>
struct FusedCta {
  static constexpr int L1 = S::L1, L2 = S::L2, C = S::C, R = S::R, E = S::E, T = S::T;
  static constexpr int Q = S::Q, QV = S::QV, RP = S::RP, P = S::P, NMAX = S::NMAX, SH = S::SH;

  float2* work;        // R x P (padded)
  float2* s0;          // E: c (ISTA/FISTA) or z (ADMM)
  float2* s1;          // E: z (FISTA) or v (ADMM)
  uint8_t* flag;       // E: 1 where this CTA's middle-stage frequency has q != 0
  float2* tw;          // NMAX twiddles W_NMAX^e
  int crank;
  int tid;

  // ---------------------------------------------------------------------------------------
  // one in-place Stockham stage over all R rows (length L1), radix RS, stride NS
  // EPI: instead of storing, hand each output (row, column, value) to the epilogue
  // ---------------------------------------------------------------------------------------
  template <int RS, int NS, bool INV, typename Epi>
  __device__ __forceinline__ void row_stage(Epi&& epi) {
    constexpr int NBR = L1 / RS;
    constexpr int NB = R * NBR;
    constexpr int NBT = (NB + T - 1) / T;
    float2 v[NBT][RS];
#pragma unroll
    for (int k = 0; k < NBT; ++k) {
      const int b = tid + k * T;
      if (NB % T == 0 || b < NB) {
        const int row = b / NBR, j = b % NBR;
#pragma unroll
        for (int i = 0; i < RS; ++i) v[k][i] = work[row * P + pad16(j + i * NBR)];
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NBT; ++k) {
      const int b = tid + k * T;
      if (NB % T == 0 || b < NB) {
        const int row = b / NBR, j = b % NBR;
        const int kk = j % NS;
        if constexpr (NS > 1) {
#pragma unroll
          for (int i = 1; i < RS; ++i) v[k][i] = twmul<INV>(v[k][i], tw[i * kk * (NMAX / (NS * RS))]);
        }
        Dft<RS, INV, float2>::run(v[k]);
        const int base = (j / NS) * NS * RS + kk;
#pragma unroll
        for (int i = 0; i < RS; ++i) epi(row, base + i * NS, v[k][i]);
      }
    }
    __syncthreads();
  }

  template <int STG, bool INV, typename Epi>
  __device__ __forceinline__ void row_fft_from(Epi&& last_epi) {
    constexpr int NST = num_stages(L1);
    constexpr int RS = radix_of(L1, STG);
    constexpr int NS = 1 << (4 * STG);
    if constexpr (STG == NST - 1) {
      row_stage<RS, NS, INV>(last_epi);
    } else {
      row_stage<RS, NS, INV>([&](int row, int e, float2 x) { work[row * P + pad16(e)] = x; });
      row_fft_from<STG + 1, INV>(last_epi);
    }
  }

  // ---------------------------------------------------------------------------------------
  // local column DFTs: QV groups x L1 columns, length RP; group v holds local rows v + QV*t
  // ---------------------------------------------------------------------------------------
  template <int RS, int NS, bool INV>
  __device__ __forceinline__ void col_stage() {
    constexpr int NBS = RP / RS;
    constexpr int NB = QV * L1 * NBS;
    constexpr int NBT = (NB + T - 1) / T;
    float2 v[NBT][RS];
#pragma unroll
    for (int k = 0; k < NBT; ++k) {
      const int b = tid + k * T;
      if (NB % T == 0 || b < NB) {
        const int col = b % L1, rest = b / L1, g = rest % QV, j = rest / QV;
#pragma unroll
        for (int i = 0; i < RS; ++i) v[k][i] = work[(g + QV * (j + i * NBS)) * P + pad16(col)];
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NBT; ++k) {
      const int b = tid + k * T;
      if (NB % T == 0 || b < NB) {
        const int col = b % L1, rest = b / L1, g = rest % QV, j = rest / QV;
        const int kk = j % NS;
        if constexpr (NS > 1) {
#pragma unroll
          for (int i = 1; i < RS; ++i) v[k][i] = twmul<INV>(v[k][i], tw[i * kk * (NMAX / (NS * RS))]);
        }
        Dft<RS, INV, float2>::run(v[k]);
        const int base = (j / NS) * NS * RS + kk;
#pragma unroll
        for (int i = 0; i < RS; ++i) work[(g + QV * (base + i * NS)) * P + pad16(col)] = v[k][i];
      }
    }
    __syncthreads();
  }

  template <int STG, bool INV>
  __device__ __forceinline__ void col_fft_from() {
    constexpr int NST = num_stages(RP);
    if constexpr (STG < NST) {
      col_stage<radix_of(RP, STG), (1 << (4 * STG)), INV>();
      col_fft_from<STG + 1, INV>();
    }
  }

  // ---------------------------------------------------------------------------------------
  // cross-group radix-Q stage, Fourier multiplier, inverse radix-Q stage (in place)
  // ---------------------------------------------------------------------------------------
  __device__ __forceinline__ void middle(float2* const* peer, const float* mult_g, const float2* bt_g) {
    constexpr int PT = (SH + T - 1) / T;
#pragma unroll
    for (int k = 0; k < PT; ++k) {
      const int pl = tid + k * T;
      if (SH % T == 0 || pl < SH) {
        const int p = crank * SH + pl;
        const int k1 = p / L1, col = p % L1;
        float2 v[Q];
#pragma unroll
        for (int g = 0; g < Q; ++g) {
          const int c = g % C, vv = g / C;
          v[g] = peer[c][(vv + QV * k1) * P + pad16(col)];
        }
#pragma unroll
        for (int g = 1; g < Q; ++g) v[g] = twmul<false>(v[g], tw[g * k1 * (NMAX / L2)]);
        Dft<Q, false, float2>::run(v);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          if (flag[q * SH + pl]) {
            const int f = (k1 + RP * q) * L1 + col;
            const float m = __ldg(&mult_g[f]);
            const float2 b = __ldg(&bt_g[f]);
            v[q] = make_float2(v[q].x * m - b.x, v[q].y * m - b.y);
          } else {
            v[q] = make_float2(0.f, 0.f);
          }
        }
        Dft<Q, true, float2>::run(v);
#pragma unroll
        for (int g = 1; g < Q; ++g) v[g] = twmul<true>(v[g], tw[g * k1 * (NMAX / L2)]);
#pragma unroll
        for (int g = 0; g < Q; ++g) {
          const int c = g % C, vv = g / C;
          peer[c][(vv + QV * k1) * P + pad16(col)] = v[g];
        }
      }
    }
  }
};

template <int L1, int L2, bool ADMM>
__global__ void __launch_bounds__(FusedShape<L1, L2, ADMM>::T, 1)
    fused_solve_kernel(const FusedArgs a) {
  using S = FusedShape<L1, L2, ADMM>;
  constexpr int C = S::C, R = S::R, E = S::E, T = S::T, P = S::P, NMAX = S::NMAX;
  constexpr int Q = S::Q, RP = S::RP, SH = S::SH;

  extern __shared__ float4 smem_raw[];
  FusedCta<S> cta;
  char* sp = reinterpret_cast<char*>(smem_raw);
  cta.work = reinterpret_cast<float2*>(sp);
  sp += R * P * 8;
  cta.s0 = reinterpret_cast<float2*>(sp);
  sp += E * 8;
  cta.s1 = reinterpret_cast<float2*>(sp);
  sp += E * 8;
  cta.tw = reinterpret_cast<float2*>(sp);
  sp += NMAX * 8;
  cta.flag = reinterpret_cast<uint8_t*>(sp);
  cta.tid = threadIdx.x;
  int crank = 0;
  if constexpr (C > 1) crank = (int)cg::this_cluster().block_rank();
  cta.crank = crank;

  const int inst_id = a.ids[blockIdx.x / C];
  const FusedInst in = a.insts[inst_id];
  const float kappa = in.kappa;
  const float* mult = a.mult + in.g_off;
  const float2* bt = a.bt + in.g_off;
  const float2* c0 = a.c0 ? a.c0 + in.c_off : nullptr;
  float2* c_out = a.c_out + in.c_off;
  float2* aux_out = a.aux_out ? a.aux_out + in.c_off : nullptr;

  float2* peer[C];
  if constexpr (C > 1) {
    cg::cluster_group cl = cg::this_cluster();
#pragma unroll
    for (int c = 0; c < C; ++c) peer[c] = cl.map_shared_rank(cta.work, c);
  } else {
    peer[0] = cta.work;
  }

  // ---- load twiddles, multiplier share, initial state
  for (int e = threadIdx.x; e < NMAX; e += T) cta.tw[e] = a.twiddle[e * (kTwiddleLen / NMAX)];
  for (int idx = threadIdx.x; idx < E; idx += T) {
    const int q = idx / SH, pl = idx % SH;
    const int p = crank * SH + pl;
    const int k1 = p / L1, col = p % L1;
    const int f = (k1 + RP * q) * L1 + col;
    cta.flag[idx] = (mult[f] != 0.f || bt[f].x != 0.f || bt[f].y != 0.f) ? 1 : 0;
  }
  for (int idx = threadIdx.x; idx < E; idx += T) {
    const int s = idx / L1, e = idx % L1;
    const int gidx = (crank + C * s) * L1 + e;
    float2 x = c0 ? c0[gidx] : make_float2(0.f, 0.f);
    cta.s0[idx] = x;                                        // c^(0) or z^(0)
    cta.s1[idx] = ADMM ? make_float2(0.f, 0.f) : x;         // z^(1) = c^(0), or v^(0) = 0
    cta.work[s * P + pad16(e)] = x;
  }
  __syncthreads();

  const bool fista = (a.beta != nullptr) && !ADMM;
  for (int it = 0; it < a.iters; ++it) {
    const float beta = fista ? __ldg(&a.beta[it]) : 0.0f;
    const bool last = (it == a.iters - 1);

    // forward row DFTs (store in place)
    cta.template row_fft_from<0, false>(
        [&](int row, int e, float2 x) { cta.work[row * P + pad16(e)] = x; });
    // forward local column DFTs
    cta.template col_fft_from<0, false>();
    if constexpr (C > 1) cg::this_cluster().sync(); else __syncthreads();
    cta.middle(peer, mult, bt);
    if constexpr (C > 1) cg::this_cluster().sync(); else __syncthreads();
    cta.template col_fft_from<0, true>();
    // inverse row DFTs with the fused epilogue
    cta.template row_fft_from<0, true>([&](int row, int e, float2 g) {
      const int sidx = row * L1 + e;
      if constexpr (!ADMM) {
        const float2 c_old = cta.s0[sidx];
        const float2 x = fista ? cta.s1[sidx] : c_old;  // z^(t)
        const float2 un = make_float2(x.x - g.x, x.y - g.y);
        const float2 cn = soft_threshold(un, kappa);
        cta.s0[sidx] = cn;
        if (fista) {
          const float2 zn = make_float2(cn.x + beta * (cn.x - c_old.x), cn.y + beta * (cn.y - c_old.y));
          cta.s1[sidx] = zn;
          cta.work[row * P + pad16(e)] = zn;
        } else {
          cta.work[row * P + pad16(e)] = cn;
        }
      } else {
        const float2 zo = cta.s0[sidx];
        const float2 vo = cta.s1[sidx];
        const float2 un = make_float2(zo.x - g.x, zo.y - g.y);  // c^(t+1) + v^(t)
        const float2 zn = soft_threshold(un, kappa);
        const float2 vn = make_float2(un.x - zn.x, un.y - zn.y);
        cta.s0[sidx] = zn;
        cta.s1[sidx] = vn;
        cta.work[row * P + pad16(e)] = make_float2(zn.x - vn.x, zn.y - vn.y);
        if (last && aux_out) aux_out[(crank + C * row) * L1 + e] = make_float2(un.x - vo.x, un.y - vo.y);
      }
    });
  }

  // ---- write the result
  for (int idx = threadIdx.x; idx < E; idx += T) {
    const int s = idx / L1, e = idx % L1;
    c_out[(crank + C * s) * L1 + e] = cta.s0[idx];
  }
  if constexpr (C > 1) cg::this_cluster().sync();
}

// ------------------------------------------------------------------------------------------
// host-side launch table
// ------------------------------------------------------------------------------------------
struct FusedEntry {
  int L1, L2, admm;
  int cluster, threads, smem;
  cudaError_t (*launch)(const FusedArgs&, int n_inst, cudaStream_t);
  cudaError_t (*prepare)();
};

template <int L1, int L2, bool ADMM>
cudaError_t fused_prepare() {
  using S = FusedShape<L1, L2, ADMM>;
  return cudaFuncSetAttribute(fused_solve_kernel<L1, L2, ADMM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              S::SMEM);
}

template <int L1, int L2, bool ADMM>
cudaError_t fused_launch(const FusedArgs& a, int n_inst, cudaStream_t st) {
  using S = FusedShape<L1, L2, ADMM>;
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
  return cudaLaunchKernelEx(&cfg, fused_solve_kernel<L1, L2, ADMM>, a);
}

template <int L1, int L2, bool ADMM>
FusedEntry fused_entry() {
  using S = FusedShape<L1, L2, ADMM>;
  return FusedEntry{L1, L2, ADMM ? 1 : 0, S::C, S::T, S::SMEM, &fused_launch<L1, L2, ADMM>,
                    &fused_prepare<L1, L2, ADMM>};
}

}  // namespace bccb
