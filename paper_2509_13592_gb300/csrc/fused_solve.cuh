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
//
// Layout.  The grid is stored L2 rows x L1 columns, row-major (the paper's
// vec(C) with C in C^{L1 x L2}, Section III-B).  A cluster of C CTAs owns one
// instance; CTA c keeps global rows c + C*s (s = 0..R-1, R = L2/C) in shared
// memory for the whole solve, so the iterations never touch HBM except for the
// nonzero Fourier-domain multiplier entries, read through L2.
//
// Transform.  Row DFTs (length L1) are local; each warp owns whole rows, so the
// row stages synchronise only the warp.  The column DFT of length L2 is split as
// L2 = Q * R' (decimation in time): group g = c + C*v (v < Q/C) holds the rows
// g + Q*t; every CTA runs the R'-point DFTs of its groups locally (one in-place
// stage), then the final radix-Q stage combines one value from each group.  That
// stage is the only cross-CTA step: each CTA takes a 1/C share of the (frequency
// k1, column) pairs, gathers its Q operands from the cluster's shared memory
// (DSMEM), runs the forward radix-Q butterfly, applies q and Bt, runs the inverse
// butterfly and scatters the results back.  q and Bt vanish off the element mask
// (Lambda = 0); a pair whose Q frequencies all vanish stores zeros without any
// load or butterfly.  Per iteration: two CTA barriers and two cluster barriers.
// Local DFTs are in-place Stockham stages (radix 16, last stage 2/4/8/16) with
// the operands staged in registers; shared rows are padded by one element per
// 16 to keep the strided stage writes free of bank conflicts.
#pragma once

#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace bccb {

struct FusedInst {
  int64_t g_off;  // offset of this instance's grids in FusedArgs::mult / ::bt
  int64_t c_off;  // offset of this instance's solution in c_out / aux_out / c0
  float kappa;    // threshold mu*lam (ISTA/FISTA) or lam/rho (ADMM), set by the setup kernels
  int kcols;      // 1 + the largest Fourier column p1 where q or Bt is nonzero (set by setup)
  int bl1 = 0;    // > 0: only the block l1 < bl1, l2 < bl2 of the grid is the unknown (the
  int bl2 = 0;    //   circulant embedding of a Toeplitz Gram); the update keeps 0 outside it
};

struct FusedArgs {
  const FusedInst* insts;  // device array of instances
  const int* ids;          // instance index for cluster k = blockIdx.x / C
  const float* beta;       // momentum beta_t (length iters); zeros or nullptr for ISTA
  const float2* twiddle;   // W_1024^e, e = 0..1023 (float2)
  const float* mult;       // Fourier multiplier q (includes 1/(L1 L2)), natural order [p2][p1]
  const float2* bt;        // Fourier-domain constant term Bt, natural order [p2][p1]
  const float2* c0;        // warm start (z^(0) for ADMM) or nullptr for zeros
  float2* c_out;           // c^(T) (ISTA/FISTA) or z^(T) (ADMM)
  float2* aux_out;         // ADMM only: c^(T); nullable
  // unrolled network (all nullable): iteration t uses u = x - scale[t] * G' and the
  // threshold thresh[t] * kappa, and stores its input z^(t) and G' into
  // save[(2t) * save_stride + c] and save[(2t + 1) * save_stride + c]
  const float* scale;
  const float* thresh;
  float2* save;
  int64_t save_stride;
  // ISTA/FISTA: low-order parts of the state, packed like c_out: {c_lo, z_lo} as bf16 pairs.
  // Read and written only where the state is nonzero (see the update in fused_solve_kernel).
  uint2* lo;
  // sparse-state variant: high parts {c_hi, z_hi} of the positions its slots cannot hold
  float4* hi;
  int iters;
  int pad_;
};

// ---- compensated (double-float) arithmetic for the ISTA/FISTA state.  A value is hi + lo
// with |lo| <= ulp(hi)/2; the sums below are Knuth's two-sum and Dekker's fast two-sum, the
// product uses the exact FMA residual.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
// (ah + al) + (bh + bl), renormalised
__device__ __forceinline__ void dd_add(float ah, float al, float bh, float bl, float& sh, float& sl) {
  float s, e;
  two_sum(ah, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(al, bl));
  fast_two_sum(s, e, sh, sl);
}
// (ch + cl) + b (dh + dl)
__device__ __forceinline__ void dd_axpy(float b, float dh, float dl, float ch, float cl, float& sh, float& sl) {
  const float p = __fmul_rn(b, dh);
  const float pl = fmaf(b, dl, fmaf(b, dh, -p));
  dd_add(ch, cl, p, pl, sh, sl);
}
__device__ __forceinline__ uint32_t pack_bf16x2(float x, float y) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ float2 unpack_bf16x2(uint32_t w) {
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }

// Elements of the grid held by one CTA: at most 8192 (64 KB of complex64); the
// 4096-element tile doubles the cluster and fits two CTAs per SM.
constexpr int kFusedTileElems = 8192;

// SPARSE: the ISTA/FISTA state is not kept as two dense grids in shared memory but only at its
// nonzero positions (per-thread slots, global memory beyond them), and each thread runs the row
// stages over two bands of rows; 8192 elements then fit in ~106 KB and two CTAs share an SM.
template <int L1_, int L2_, bool ADMM_, int TILE_ = kFusedTileElems, bool SPARSE_ = false>
struct FusedShape {
  static constexpr int L1 = L1_, L2 = L2_, TILE = TILE_;
  static constexpr bool ADMM = ADMM_, SPARSE = SPARSE_;
  static constexpr int PASSES = SPARSE ? 2 : 1;                  // row bands per thread
  static constexpr int C = cmax(1, (L1 * L2) / TILE);  // CTAs per cluster
  static constexpr int R = L2 / C;                                // rows per CTA
  static constexpr int E = R * L1;                                // elements per CTA
  static constexpr int T = cmax(32, E / (16 * PASSES));           // threads per CTA
  static constexpr int V = E / T / PASSES;                        // elements per thread per stage and band
  static constexpr int Q = cmin(16, L2);                          // cross-group radix
  static constexpr int QV = Q / C;                                // groups per CTA
  static constexpr int RP = L2 / Q;                               // local column DFT length
  static constexpr int NMAX = cmax(L1, L2);
  static constexpr int SH = RP * L1 / C;                          // middle-stage pairs per CTA
  // each warp owns 512/L1 whole rows through every row stage
  static constexpr bool ROW_WARP = (V == 16) && (L1 <= 512) && ((32 * V) % L1 == 0);
  // rows of 256 = 16 x 16: a thread reads and writes the same 16 positions in the
  // last inverse and the first forward row stage (see FusedCta::sq_*)
  static constexpr bool SQ16 = ROW_WARP && (L1 == 256);
  // padded row pitch; for rows of 256 one more element puts the two rows of a warp in
  // different banks, so that their broadcast reads of the spectrum do not conflict
  static constexpr int P = L1 + L1 / 16 + (SQ16 ? 1 : 0);
  // middle stage with each 16-point butterfly split over 4 lanes (cluster path)
  static constexpr bool SPLIT_MID = (C > 1) && (Q == 16) && (SH % L1 == 0);
  // the split middle stage keeps up to MCAP of its nonzero (q, Bt) entries in shared
  // memory (indexed through a per-pair offset); any beyond are read from global memory
  static constexpr int MCAP = SPLIT_MID ? E / 16 : 0;
  static constexpr int POFF = SPLIT_MID ? ((SH * 2 + 15) / 16) * 16 : 0;
  // work (padded) + two state grids + twiddles + a frequency bit mask per middle-stage pair
  // + W_256^{i j} (16 x 16, rows of 256) + W_16^m + the cached multipliers and offsets
  // rows per band of the SQ16 row stages: two rows per warp
  static constexpr int BAND = 2 * (T / 32);
  // ISTA/FISTA: two 8-byte slots per thread for the low-order parts of its first two
  // positions with a nonzero state (see the update in fused_solve_kernel); the sparse variant
  // keeps {c_hi, z_hi} and the low parts there (24 bytes), in two sets used alternately
  static constexpr int SLOTS = ADMM ? 0 : SPARSE ? 2 * 2 * T * 24 : 2 * T * 8;
  static constexpr int STATE = SPARSE ? 0 : 2 * E * 8;          // dense state grids
  static constexpr int SMEM = R * P * 8 + STATE + NMAX * 8 + ((SH * 2 + 15) / 16) * 16 + 256 * 8 + 16 * 8 +
                              MCAP * 16 + POFF + SLOTS;
  static_assert(!SPARSE || (SQ16 && !ADMM && PASSES * BAND == R), "sparse state: rows of 256, ISTA/FISTA");
  static_assert(SMEM <= 227 * 1024, "shared memory per CTA");
  static_assert((R * P * 8) % 16 == 0, "16-byte aligned layout after the work rows");
  // two CTAs per SM when their shared memory fits (227 KB per CTA, 228 KB per SM)
  static constexpr int MIN_BLOCKS = (2 * (SMEM + 1024) <= 228 * 1024) ? 2 : 1;
  static_assert(L1 >= 16 && L2 >= 16, "fused path needs L1, L2 >= 16");
  static_assert(C <= 16, "cluster larger than 16 CTAs");
  static_assert(QV * C == Q, "cluster size must divide the cross-group radix");
  static_assert(SH * C == RP * L1, "middle-stage pairs must split evenly");
  static_assert(num_stages(RP) <= 1, "local column DFT is a single stage");
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

// the factor s of S_kappa(u) = u s (0 at and below the threshold)
__device__ __forceinline__ float soft_scale(float2 u, float kappa) {
  const float r2 = u.x * u.x + u.y * u.y;
  return r2 > kappa * kappa ? 1.0f - kappa * rsqrtf(r2) : 0.0f;
}

// ---- distributed shared memory with 32-bit shared::cluster addresses
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t cluster_map(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ float2 ld_cluster(uint32_t a) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void st_cluster(uint32_t a, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}

// read-only global loads kept in program order (the compiler may not hoist them)
__device__ __forceinline__ float ld_ro_f32(const float* p) {
  float v;
  asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float2 ld_ro_f32x2(const float2* p) {
  float2 v;
  asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}

template <typename S>
struct FusedCta {
  static constexpr int L1 = S::L1, L2 = S::L2, C = S::C, R = S::R, E = S::E, T = S::T;
  static constexpr int Q = S::Q, QV = S::QV, RP = S::RP, P = S::P, NMAX = S::NMAX, SH = S::SH;

  float2* work;     // R x P (padded)
  float2* s0;       // E: c (ISTA/FISTA) or z (ADMM)
  float2* s1;       // E: z (FISTA) or v (ADMM)
  float2* tw;       // NMAX twiddles W_NMAX^e
  uint16_t* pmask;  // SH: bit q set when frequency (k1 + RP q, col) of pair pl has q != 0
  float2* tw256;    // 16 x 16: tw256[i * 16 + j] = W_256^{i j} (conflict-free per-lane twiddles)
  float2* tw16;     // W_16^m, m < 16
  float4* mtab;     // MCAP: {q, Bt.x, Bt.y, 0} of the active pairs' nonzero frequencies, in pair order
  uint16_t* poff;   // per active pair: index of its first entry in mtab
  int crank;
  int tid;
  int band = 0;  // SQ16 row stages: the band of S::BAND rows being processed
  // every nonzero frequency of this CTA's pairs has q < 2 (the spectrum lives in the first
  // 2 RP rows, e.g. a 32-row array on a 256-row grid): the split middle stage then forms
  // and reads only X[0] and X[1] of each 16-point butterfly
  bool q2 = false;

  // ---------------------------------------------------------------------------------------
  // one in-place Stockham stage over all R rows (length L1), radix RS, stride NS; the
  // epilogue functor receives every output (row, column, value)
  // ---------------------------------------------------------------------------------------
  // kin: columns >= kin hold zeros and are not loaded (the first inverse stage after
  // the middle stage, whose spectrum vanishes beyond the instance's active columns)
  template <int RS, int NS, bool INV, typename Epi>
  __device__ __forceinline__ void row_stage(Epi&& epi, int kin = L1) {
    constexpr int NBR = L1 / RS;
    if constexpr (S::ROW_WARP) {
      constexpr int RPW = 512 / L1;          // rows per warp
      constexpr int NBT = (RPW * NBR) / 32;  // butterflies per thread (= 16 / RS)
      const int warp = tid >> 5, lane = tid & 31;
      float2 v[NBT][RS];
#pragma unroll
      for (int k = 0; k < NBT; ++k) {
        const int bw = lane + 32 * k;
        const int row = warp * RPW + bw / NBR, j = bw % NBR;
#pragma unroll
        for (int i = 0; i < RS; ++i)
          v[k][i] = (j + i * NBR < kin) ? work[row * P + pad16(j + i * NBR)] : make_float2(0.f, 0.f);
      }
      __syncwarp();
#pragma unroll
      for (int k = 0; k < NBT; ++k) {
        const int bw = lane + 32 * k;
        const int row = warp * RPW + bw / NBR, j = bw % NBR;
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
      __syncwarp();
    } else {
      constexpr int NB = R * NBR;
      constexpr int NBT = (NB + T - 1) / T;
      float2 v[NBT][RS];
#pragma unroll
      for (int k = 0; k < NBT; ++k) {
        const int b = tid + k * T;
        if (NB % T == 0 || b < NB) {
          const int row = b / NBR, j = b % NBR;
#pragma unroll
          for (int i = 0; i < RS; ++i)
            v[k][i] = (j + i * NBR < kin) ? work[row * P + pad16(j + i * NBR)] : make_float2(0.f, 0.f);
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
  }

  template <int STG, bool INV, typename Epi>
  __device__ __forceinline__ void row_fft_from(Epi&& last_epi, int kin) {
    constexpr int NST = num_stages(L1);
    constexpr int RS = radix_of(L1, STG);
    constexpr int NS = 1 << (4 * STG);
    const int k = (STG == 0) ? kin : L1;
    if constexpr (STG == NST - 1) {
      row_stage<RS, NS, INV>(last_epi, k);
    } else {
      row_stage<RS, NS, INV>([&](int row, int e, float2 x) { work[row * P + pad16(e)] = x; }, k);
      row_fft_from<STG + 1, INV>(last_epi, kin);
    }
  }

  // ---------------------------------------------------------------------------------------
  // local column DFTs: QV groups x L1 columns, length RP, a single radix-RP stage;
  // group g holds local rows g + QV*t.  Each thread reads and writes the same RP
  // positions, so the stage needs no barrier of its own.
  // ---------------------------------------------------------------------------------------
  template <bool INV>
  __device__ __forceinline__ void col_dft(int kc) {
    // The split form only where one thread per active column would leave more than three
    // quarters of the CTA idle (the 256 x 256 grid with 32 active columns: 2 of 16 warps); where
    // that form keeps the threads busy (rows of 64 or 128 over 256 rows) the shuffles only cost
    // (13 % slower there), and the sparse-state tile, whose two CTAs per SM belong to different
    // instances, was 3 % slower with it (A/B on one box).
    if constexpr (RP == 16 && !S::SPARSE && 4 * QV * 16 < T) {  // kc >= 16 once active
      if (4 * QV * kc < T) {
        col_dft_lanes<INV>(kc);
        return;
      }
    }
    if constexpr (RP > 1) {
      constexpr int NB = QV * L1;
      constexpr int NBT = (NB + T - 1) / T;
#pragma unroll
      for (int k = 0; k < NBT; ++k) {
        const int b = tid + k * T;
        if ((NB % T == 0 || b < NB) && (b % L1) < kc) {
          const int col = b % L1, g = b / L1;
          float2 v[RP];
#pragma unroll
          for (int i = 0; i < RP; ++i) v[i] = work[(g + QV * i) * P + pad16(col)];
          Dft<RP, INV, float2>::run(v);
#pragma unroll
          for (int i = 0; i < RP; ++i) work[(g + QV * i) * P + pad16(col)] = v[i];
        }
      }
    }
  }

  // The same local column DFTs for RP = 16, each split over 4 lanes (4 x 4 with a shuffle
  // transpose, as in the middle stage): lane e of the pair (group g, column col) reads inputs
  // n = e + 4 i, runs the inner 4-point DFT over i, twiddles by W_16^{e k'}, exchanges across
  // the pair's lanes, runs the outer 4-point DFT and holds outputs e + 4 k'' -- the rows it
  // read, so the stage still needs no barrier of its own.  Four times the threads of the
  // one-thread-per-column form for the few active columns.
  template <bool INV>
  __device__ __forceinline__ void col_dft_lanes(int kc) {
    const int np = QV * kc;  // active (group, column) pairs
    const int lane = tid & 31, e = tid & 3;
    const int rounds = (4 * np + T - 1) / T;
    for (int rd = 0; rd < rounds; ++rd) {
      if (rd * T + (tid & ~31) >= 4 * np) break;  // the whole warp is past the active pairs
      const int t = rd * T + tid;
      const bool on = t < 4 * np;
      const int a = on ? (t >> 2) : 0;
      const int g = a / kc, col = a % kc;
      float2* const base = work + g * P + pad16(col);
      float2 v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] = base[(e + 4 * i) * QV * P];
      dft4<INV>(v[0], v[1], v[2], v[3]);
#pragma unroll
      for (int i = 1; i < 4; ++i) v[i] = twmul<INV>(v[i], tw16[e * i]);
      transpose4(v, e, lane);
      dft4<INV>(v[0], v[1], v[2], v[3]);  // v[k''] = X[e + 4 k'']
      if (on) {
#pragma unroll
        for (int k = 0; k < 4; ++k) base[(e + 4 * k) * QV * P] = v[k];
      }
    }
  }

  // ---------------------------------------------------------------------------------------
  // Rows of 256 = 16 x 16 (two radix-16 Stockham stages).  Thread (row, j), j < 16,
  // reads positions j + 16 i in both stages and writes 16 j + k in the first, j + 16 k
  // in the second.  Only the first nz = kc/16 Fourier column blocks are nonzero
  // after the middle stage and only they are needed after the forward transform, so
  // the forward second stage forms just its first nz outputs and the inverse first
  // stage reads just its first nz inputs.
  // ---------------------------------------------------------------------------------------
  __device__ __forceinline__ void sq_rowj(int& row, int& j) const {
    row = band * S::BAND + (tid >> 5) * 2 + ((tid & 31) >> 4);
    j = tid & 15;
  }
  // with j < 16, the padded position of j + 16 i is j + 17 i and that of 16 j + k is 17 j + k:
  // a per-thread base pointer and compile-time offsets
  __device__ __forceinline__ float2* sq_col(int row, int j) const { return work + row * P + j; }
  __device__ __forceinline__ float2* sq_blk(int row, int j) const { return work + row * P + 17 * j; }

  // forward first stage from the work rows (used once, before the first iteration)
  __device__ __forceinline__ void sq_fwd1_from_work() {
    int row, j;
    sq_rowj(row, j);
    float2* const cp = sq_col(row, j);
    float2* const bp = sq_blk(row, j);
    (void)cp;
    (void)bp;
    float2 v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = cp[17 * i];
    __syncwarp();
    Dft<16, false, float2>::run(v);
#pragma unroll
    for (int k = 0; k < 16; ++k) bp[k] = v[k];
    __syncwarp();
  }

  // forward second stage, outputs j + 16 k2 for k2 < nz only
  __device__ __forceinline__ void sq_fwd2(int nz) {
    int row, j;
    sq_rowj(row, j);
    float2* const cp = sq_col(row, j);
    float2* const bp = sq_blk(row, j);
    (void)cp;
    (void)bp;
    float2 v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = cp[17 * i];
    __syncwarp();
#pragma unroll
    for (int i = 1; i < 16; ++i) v[i] = twmul<false>(v[i], tw256[i * 16 + j]);
    if (nz == 1) {
      float2 s0 = v[0];
#pragma unroll
      for (int i = 1; i < 16; ++i) s0 = cadd(s0, v[i]);
      cp[0] = s0;
    } else if (nz == 2) {
      // outputs k2 = 0 and 1 of the 16-point DFT: sum_i v_i and sum_i v_i W_16^i
      float2 s0 = v[0], s1 = v[0];
#pragma unroll
      for (int i = 1; i < 16; ++i) {
        s0 = cadd(s0, v[i]);
        s1 = twmadd<false>(s1, v[i], tw16[i]);
      }
      cp[0] = s0;
      cp[17] = s1;
    } else {
      Dft<16, false, float2>::run(v);
#pragma unroll
      for (int k = 0; k < 16; ++k)
        if (k < nz) cp[17 * k] = v[k];
    }
    __syncwarp();
  }

  // inverse first stage, inputs j + 16 i for i < nz only
  __device__ __forceinline__ void sq_inv1(int nz) {
    int row, j;
    sq_rowj(row, j);
    float2* const cp = sq_col(row, j);
    float2* const bp = sq_blk(row, j);
    (void)cp;
    (void)bp;
    float2 v[16];
    if (nz <= 2) {
      const float2 a = cp[0];
      const float2 b = (nz == 2) ? cp[17] : make_float2(0.f, 0.f);
      __syncwarp();
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = twmadd<true>(a, b, tw16[k]);
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = (i < nz) ? cp[17 * i] : make_float2(0.f, 0.f);
      __syncwarp();
      Dft<16, true, float2>::run(v);
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) bp[k] = v[k];
    __syncwarp();
  }

  // inverse second stage, the epilogue on its 16 outputs, and (unless last) the next
  // iteration's forward first stage on the 16 new inputs, all in registers
  //
  // With nz <= 2 the first inverse stage is folded in as well: its output at position
  // j + 16 i is X[i] + W_16^{-j} X[i + 16], formed from the row's 2 x 16 nonzero inputs
  // (read by all 16 threads of the row: broadcasts); otherwise sq_inv1 has run before.
  template <typename Epi>
  __device__ __forceinline__ void sq_inv2_epi_fwd1(Epi&& epi, bool next, int nz) {
    int row, j;
    sq_rowj(row, j);
    float2* const cp = sq_col(row, j);
    float2* const bp = sq_blk(row, j);
    (void)cp;
    (void)bp;
    float2 v[16];
    const float2* xr = work + row * P;
    if (nz == 2) {
      const float2 w = tw16[j];
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = twmadd<true>(xr[pad16(i)], xr[pad16(i + 16)], w);
    } else if (nz == 1) {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = xr[pad16(i)];
    } else if (nz == 0) {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = make_float2(0.f, 0.f);
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = xr[j + 17 * i];
    }
    __syncwarp();
#pragma unroll
    for (int i = 1; i < 16; ++i) v[i] = twmul<true>(v[i], tw256[i * 16 + j]);
    Dft<16, true, float2>::run(v);
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = epi(row, j + 16 * i, v[i]);
    if (next) {
      Dft<16, false, float2>::run(v);
#pragma unroll
      for (int k = 0; k < 16; ++k) bp[k] = v[k];
    }
    __syncwarp();
  }

  // As sq_inv2_epi_fwd1, with the epilogue split in two: quick(row, e, i, g, flag) runs on all
  // 16 outputs (unrolled) and either finishes the element (flag false) or returns a value to
  // keep for the second part; ext(row, e, i, value) then runs on the flagged outputs only, in
  // ascending i, in a loop that is not unrolled (one copy of its code).  The kept values wait in
  // the positions this thread writes in the forward stage (free once the inputs are read).
  template <typename Quick, typename Ext>
  __device__ __forceinline__ void sq_inv2_split_fwd1(Quick&& quick, Ext&& ext, bool next, int nz) {
    int row, j;
    sq_rowj(row, j);
    float2* const bp = sq_blk(row, j);
    float2 v[16];
    const float2* xr = work + row * P;
    if (nz == 2) {
      const float2 w = tw16[j];
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = twmadd<true>(xr[pad16(i)], xr[pad16(i + 16)], w);
    } else if (nz == 1) {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = xr[pad16(i)];
    } else if (nz == 0) {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = make_float2(0.f, 0.f);
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = xr[j + 17 * i];
    }
    __syncwarp();
#pragma unroll
    for (int i = 1; i < 16; ++i) v[i] = twmul<true>(v[i], tw256[i * 16 + j]);
    Dft<16, true, float2>::run(v);
    uint32_t flagged = 0u;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      bool f;
      v[i] = quick(row, j + 16 * i, 16 * band + i, v[i], f);
      if (f) flagged |= 1u << i;
    }
    if (flagged) {
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (flagged & (1u << i)) bp[i] = v[i];
#pragma unroll 1
      for (uint32_t m = flagged; m; m &= m - 1u) {
        const int i = __ffs(m) - 1;
        bp[i] = ext(row, j + 16 * i, 16 * band + i, bp[i]);
      }
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (flagged & (1u << i)) v[i] = bp[i];
    }
    if (next) {
      Dft<16, false, float2>::run(v);
#pragma unroll
      for (int k = 0; k < 16; ++k) bp[k] = v[k];
    }
    __syncwarp();
  }

  // (row, position) of the o-th output a thread handles in the last stage of row_fft_from
  // (o = k RS + i for butterfly k and output i of row_stage's loops)
  __device__ __forceinline__ void last_row_output(int o, int& row, int& e) const {
    constexpr int NST = num_stages(L1);
    constexpr int RS = radix_of(L1, NST - 1);
    constexpr int NS = 1 << (4 * (NST - 1));
    constexpr int NBR = L1 / RS;
    const int k = o / RS, i = o % RS;
    int j;
    if constexpr (S::ROW_WARP) {
      constexpr int RPW = 512 / L1;
      const int bw = (tid & 31) + 32 * k;
      row = (tid >> 5) * RPW + bw / NBR;
      j = bw % NBR;
    } else {
      const int b = tid + k * T;
      row = b / NBR;
      j = b % NBR;
    }
    e = (j / NS) * NS * RS + (j % NS) + i * NS;
  }

  // twiddles and the per-pair frequency masks (bt may be null: a Gram product alone)
  __device__ __forceinline__ void load_tables(const float2* twiddle, const float* mult, const float2* bt, int kc) {
    for (int e = tid; e < NMAX; e += T) tw[e] = twiddle[e * (kTwiddleLen / NMAX)];
    for (int e = tid; e < 256; e += T) tw256[e] = twiddle[((e >> 4) * (e & 15)) * (kTwiddleLen / 256)];
    for (int e = tid; e < 16; e += T) tw16[e] = twiddle[e * (kTwiddleLen / 16)];
    uint32_t high = 0;
    for (int pl = tid; pl < SH; pl += T) {
      const int p = crank * SH + pl;
      const int k1 = p / L1, col = p % L1;
      uint32_t pm = 0;
      for (int q = 0; q < Q; ++q) {
        const int f = (k1 + RP * q) * L1 + col;
        if (mult[f] != 0.f || (bt && (bt[f].x != 0.f || bt[f].y != 0.f))) pm |= 1u << q;
      }
      pmask[pl] = (uint16_t)pm;
      high |= pm >> 2;
    }
    q2 = !__syncthreads_or(high != 0u);
    if constexpr (S::SPLIT_MID) {
      // active pair a = (k1 - crank KPO) kc + col; exclusive prefix of the flag counts by
      // one warp (each lane a contiguous chunk), then every thread copies its pairs' entries
      constexpr int KPO = SH / L1;
      const int np = KPO * kc;
      __syncthreads();
      if (tid < 32) {
        const int chunk = (np + 31) / 32, lo = min(np, tid * chunk), hi = min(np, lo + chunk);
        int sum = 0;
        for (int q = lo; q < hi; ++q) sum += __popc(pmask[(q / kc) * L1 + q % kc]);
        int incl = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int o = __shfl_up_sync(0xffffffffu, incl, d);
          if (tid >= d) incl += o;
        }
        int run = incl - sum;
        for (int q = lo; q < hi; ++q) {
          poff[q] = (uint16_t)run;
          run += __popc(pmask[(q / kc) * L1 + q % kc]);
        }
      }
      __syncthreads();
      for (int q = tid; q < np; q += T) {
        const int pl = (q / kc) * L1 + q % kc;
        const int k1 = crank * KPO + q / kc, col = q % kc;
        uint32_t pm = pmask[pl];
        int idx = poff[q];
        while (pm && idx < S::MCAP) {
          const int fq = __ffs(pm) - 1;
          pm &= pm - 1;
          const int f = (k1 + RP * fq) * L1 + col;
          const float2 b = bt ? bt[f] : make_float2(0.f, 0.f);
          mtab[idx++] = make_float4(mult[f], b.x, b.y, 0.f);
        }
      }
    }
  }


  // ---------------------------------------------------------------------------------------
  // The middle stage with each pair's 16-point butterflies split over 4 lanes (4 x 4):
  // lane e of a pair holds groups g = e + 4 i (i < 4); inner 4-point DFT over i, twiddle
  // W_16^{e k'}, a 4 x 4 transpose across the lanes (four shuffle rounds), outer 4-point DFT
  // over e, giving frequencies k' + 4 k'' on lane k'; then q . X - Bt and the mirror image
  // back to groups.  The active pairs (columns < kc) are spread over all of the CTA's warps.
  // ---------------------------------------------------------------------------------------
  // 4 x 4 transpose across the 4 lanes of a pair: lane e's a[k] goes to lane k's a[e].
  // Round r moves the entries with k - e = -r (mod 4); lane-dependent indices are resolved
  // with selects over constant indices so that the values stay in registers.
  static __device__ __forceinline__ void transpose4(float2 (&a)[4], int e, int lane) {
    float2 out[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int si = (e - r) & 3, di = (e + r) & 3;
      float2 send = a[0];
#pragma unroll
      for (int j = 1; j < 4; ++j) send = (si == j) ? a[j] : send;
      const int src = (lane & ~3) | di;
      float2 got;
      got.x = __shfl_sync(0xffffffffu, send.x, src);
      got.y = __shfl_sync(0xffffffffu, send.y, src);
#pragma unroll
      for (int j = 0; j < 4; ++j) out[j] = (di == j) ? got : out[j];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = out[i];
  }

  // Lane e of active pair a = (k1 - crank KPO) kc + col: load(i) returns group e + 4 i of the
  // pair after the local column DFT, store(i, x) takes the same group's inverse result.
  template <typename Load, typename Store>
  __device__ __forceinline__ void middle_lanes(const float* mult_g, const float2* bt_g, int kc, Load&& load,
                                               Store&& store) {
    constexpr int KPO = SH / L1;  // frequencies k1 owned by this CTA, all columns each
    const int np = KPO * kc;     // active pairs
    const int lane = tid & 31, e = tid & 3;
    const int rounds = (4 * np + T - 1) / T;
    if (q2) {
      // Only X[0] and X[1] of each 16-point butterfly, with the arithmetic of the full form
      // below in the same order (so the nonzero results are the same bits): lane e's inner
      // 4-point outputs 0 and 1 (the latter times W_16^e), summed over the quad as the outer
      // 4-point DFT sums them, (s_0 + s_2) + (s_1 + s_3) (xor 2, then xor 1; every lane gets
      // the same value).  The inverse: lane e's twiddled inverse input W_16^{-e} Y[1] and Y[0]
      // through the same inverse 4-point DFT, zeros elsewhere.
      for (int rd = 0; rd < rounds; ++rd) {
        if (rd * T + (tid & ~31) >= 4 * np) break;  // the whole warp is past the active pairs
        const int t = rd * T + tid;
        const bool on = t < 4 * np;
        const int a = on ? (t >> 2) : 0;
        const int k1 = crank * KPO + a / kc, col = a % kc;
        const int pl = (k1 - crank * KPO) * L1 + col;
        const uint32_t pm = on ? pmask[pl] : 0u;
        const int pbase = on ? (int)poff[a] : 0;
        float2 v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int g = e + 4 * i;
          v[i] = pm ? load(a, k1, col, i) : make_float2(0.f, 0.f);
          if (g) v[i] = twmul<false>(v[i], tw[g * k1 * (NMAX / L2)]);
        }
        float2 x0 = cadd(cadd(v[0], v[2]), cadd(v[1], v[3]));
        float2 x1 = twmul<false>(cadd(csub(v[0], v[2]), mul_mj<false>(csub(v[1], v[3]))), tw16[e]);
#pragma unroll
        for (int m = 2; m >= 1; m >>= 1) {
          x0.x += __shfl_xor_sync(0xffffffffu, x0.x, m);
          x0.y += __shfl_xor_sync(0xffffffffu, x0.y, m);
          x1.x += __shfl_xor_sync(0xffffffffu, x1.x, m);
          x1.y += __shfl_xor_sync(0xffffffffu, x1.y, m);
        }
        float2 y[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const float2 xq = q ? x1 : x0;
          y[q] = make_float2(0.f, 0.f);
          if (pm & (1u << q)) {
            const int idx = pbase + (q ? (int)(pm & 1u) : 0);
            float mq;
            float2 b;
            if (idx < S::MCAP) {
              const float4 t4 = mtab[idx];
              mq = t4.x;
              b = make_float2(t4.y, t4.z);
            } else {
              const int f = (k1 + RP * q) * L1 + col;
              mq = ld_ro_f32(&mult_g[f]);
              b = bt_g ? ld_ro_f32x2(&bt_g[f]) : make_float2(0.f, 0.f);
            }
            y[q] = make_float2(xq.x * mq - b.x, xq.y * mq - b.y);
          }
        }
        v[0] = y[0];
        v[1] = twmul<true>(y[1], tw16[e]);
        v[2] = v[3] = make_float2(0.f, 0.f);
        dft4<true>(v[0], v[1], v[2], v[3]);  // v[i] -> group e + 4 i
        if (on) {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int g = e + 4 * i;
            float2 o = v[i];
            if (g) o = twmul<true>(o, tw[g * k1 * (NMAX / L2)]);
            store(k1, col, i, o);
          }
        }
      }
      return;
    }
    for (int rd = 0; rd < rounds; ++rd) {
      if (rd * T + (tid & ~31) >= 4 * np) break;  // the whole warp is past the active pairs
      const int t = rd * T + tid;
      const bool on = t < 4 * np;
      const int a = on ? (t >> 2) : 0;
      const int k1 = crank * KPO + a / kc, col = a % kc;
      const int pl = (k1 - crank * KPO) * L1 + col;
      const uint32_t pm = on ? pmask[pl] : 0u;
      const int pbase = on ? (int)poff[a] : 0;
      float2 v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int g = e + 4 * i;
        v[i] = pm ? load(a, k1, col, i) : make_float2(0.f, 0.f);
        if (g) v[i] = twmul<false>(v[i], tw[g * k1 * (NMAX / L2)]);
      }
      dft4<false>(v[0], v[1], v[2], v[3]);
#pragma unroll
      for (int i = 1; i < 4; ++i) v[i] = twmul<false>(v[i], tw16[e * i]);
      transpose4(v, e, lane);
      dft4<false>(v[0], v[1], v[2], v[3]);  // v[k''] = X[e + 4 k'']
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const int q = e + 4 * kk;
        if (pm & (1u << q)) {
          const int idx = pbase + __popc(pm & ((1u << q) - 1u));
          float m;
          float2 b;
          if (idx < S::MCAP) {
            const float4 t4 = mtab[idx];
            m = t4.x;
            b = make_float2(t4.y, t4.z);
          } else {
            const int f = (k1 + RP * q) * L1 + col;
            m = ld_ro_f32(&mult_g[f]);
            b = bt_g ? ld_ro_f32x2(&bt_g[f]) : make_float2(0.f, 0.f);
          }
          v[kk] = make_float2(v[kk].x * m - b.x, v[kk].y * m - b.y);
        } else {
          v[kk] = make_float2(0.f, 0.f);
        }
      }
      dft4<true>(v[0], v[1], v[2], v[3]);  // index e' of the inverse outer DFT
      transpose4(v, e, lane);
#pragma unroll
      for (int i = 1; i < 4; ++i) v[i] = twmul<true>(v[i], tw16[e * i]);
      dft4<true>(v[0], v[1], v[2], v[3]);  // v[i] -> group e + 4 i
      if (on) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int g = e + 4 * i;
          float2 o = v[i];
          if (g) o = twmul<true>(o, tw[g * k1 * (NMAX / L2)]);
          store(k1, col, i, o);
        }
      }
    }
  }

  // pull form: every group is read from and written back to the CTA that holds it
  __device__ __forceinline__ void middle_split(const float* mult_g, const float2* bt_g, int kc) {
    const int e = tid & 3;
    // shared::cluster base of the CTA holding each of this lane's groups e + 4 i
    uint32_t base[4];
    const uint32_t w = smem_addr(work);
#pragma unroll
    for (int i = 0; i < 4; ++i) base[i] = cluster_map(w, (e + 4 * i) % C);
    middle_lanes(
        mult_g, bt_g, kc,
        [&](int, int k1, int col, int i) {
          const int g = e + 4 * i;
          return ld_cluster(base[i] + (((g / C) + QV * k1) * P + pad16(col)) * 8);
        },
        [&](int k1, int col, int i, float2 o) {
          const int g = e + 4 * i;
          st_cluster(base[i] + (((g / C) + QV * k1) * P + pad16(col)) * 8, o);
        });
  }

  // ---------------------------------------------------------------------------------------
  __device__ __forceinline__ void middle(const uint32_t* peer, const float* mult_g, const float2* bt_g, int kc) {
    if constexpr (S::SPLIT_MID) {
      middle_split(mult_g, bt_g, kc);
      return;
    }
    constexpr int PT = (SH + T - 1) / T;
#pragma unroll
    for (int k = 0; k < PT; ++k) {
      const int pl = tid + k * T;
      if ((SH % T == 0 || pl < SH) && ((crank * SH + pl) % L1) < kc) {
        const int p = crank * SH + pl;
        const int k1 = p / L1, col = p % L1;
        const uint32_t pm = pmask[pl];
        float2 v[Q];
        if (pm != 0) {
          // The first two nonzero frequencies of the pair (the common case off a
          // sparse mask) are fetched now, so their latency hides behind the gather
          // and the forward butterfly; any further ones are read when needed.
          const int q0 = __ffs(pm) - 1;
          const uint32_t rest = pm & (pm - 1);
          const int q1 = rest ? __ffs(rest) - 1 : -1;
          const int f0 = (k1 + RP * q0) * L1 + col;
          const float m0 = ld_ro_f32(&mult_g[f0]);
          const float2 b0 = bt_g ? ld_ro_f32x2(&bt_g[f0]) : make_float2(0.f, 0.f);
          float m1 = 0.f;
          float2 b1 = make_float2(0.f, 0.f);
          if (q1 >= 0) {
            const int f1 = (k1 + RP * q1) * L1 + col;
            m1 = ld_ro_f32(&mult_g[f1]);
            if (bt_g) b1 = ld_ro_f32x2(&bt_g[f1]);
          }
#pragma unroll
          for (int g = 0; g < Q; ++g) {
            const int c = g % C, vv = g / C;
            const int off = (vv + QV * k1) * P + pad16(col);
            if constexpr (C > 1) {
              v[g] = ld_cluster(peer[c] + off * 8);
            } else {
              v[g] = work[off];
            }
          }
#pragma unroll
          for (int g = 1; g < Q; ++g) v[g] = twmul<false>(v[g], tw[g * k1 * (NMAX / L2)]);
          Dft<Q, false, float2>::run(v);
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            if (pm & (1u << q)) {
              float m;
              float2 b;
              if (q == q0) {
                m = m0;
                b = b0;
              } else if (q == q1) {
                m = m1;
                b = b1;
              } else {
                const int f = (k1 + RP * q) * L1 + col;
                m = ld_ro_f32(&mult_g[f]);
                b = bt_g ? ld_ro_f32x2(&bt_g[f]) : make_float2(0.f, 0.f);
              }
              v[q] = make_float2(v[q].x * m - b.x, v[q].y * m - b.y);
            } else {
              v[q] = make_float2(0.f, 0.f);
            }
          }
          Dft<Q, true, float2>::run(v);
#pragma unroll
          for (int g = 1; g < Q; ++g) v[g] = twmul<true>(v[g], tw[g * k1 * (NMAX / L2)]);
        } else {
#pragma unroll
          for (int g = 0; g < Q; ++g) v[g] = make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int g = 0; g < Q; ++g) {
          const int c = g % C, vv = g / C;
          const int off = (vv + QV * k1) * P + pad16(col);
          if constexpr (C > 1) {
            st_cluster(peer[c] + off * 8, v[g]);
          } else {
            work[off] = v[g];
          }
        }
      }
    }
  }
};

template <int C>
__device__ __forceinline__ void cluster_barrier() {
  if constexpr (C > 1) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
}

// LEARN: honour FusedArgs::scale / ::thresh / ::save (the unrolled network's forward pass);
// plain solves are compiled without them.
// BLOCK: the grid is the circulant embedding of a Toeplitz Gram and the update keeps the
// unknown at 0 outside the instance's block (FusedInst::bl1, bl2); ordinary grids compile without it.
// SPARSE: the state outside shared memory (see FusedShape); ISTA/FISTA solves only.
template <int L1, int L2, bool ADMM, int TILE, bool LEARN = false, bool BLOCK = false, bool SPARSE = false>
__global__ void __launch_bounds__(FusedShape<L1, L2, ADMM, TILE, SPARSE>::T,
                                  FusedShape<L1, L2, ADMM, TILE, SPARSE>::MIN_BLOCKS)
    fused_solve_kernel(const FusedArgs a) {
  using S = FusedShape<L1, L2, ADMM, TILE, SPARSE>;
  constexpr int C = S::C, E = S::E, T = S::T, P = S::P, NMAX = S::NMAX, R = S::R;
  static_assert(!SPARSE || (!LEARN && !BLOCK), "the sparse-state variant serves plain solves");

  extern __shared__ float4 smem_raw[];
  FusedCta<S> cta;
  char* sp = reinterpret_cast<char*>(smem_raw);
  cta.work = reinterpret_cast<float2*>(sp);
  sp += R * P * 8;
  cta.s0 = SPARSE ? nullptr : reinterpret_cast<float2*>(sp);
  cta.s1 = SPARSE ? nullptr : reinterpret_cast<float2*>(sp + E * 8);
  sp += S::STATE;
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
  sp += S::POFF;
  uint2* const slot = reinterpret_cast<uint2*>(sp) + 2 * threadIdx.x;  // this thread's two slots
  // sparse variant: slot sets [2][2][T] of {c_hi, z_hi} (float4) and of the low parts (uint2)
  float4* const shi = reinterpret_cast<float4*>(sp);
  uint2* const slo = reinterpret_cast<uint2*>(sp + 2 * 2 * T * 16);
  cta.tid = threadIdx.x;
  int crank = 0;
  if constexpr (C > 1) crank = (int)cg::this_cluster().block_rank();
  cta.crank = crank;

  const int inst_id = a.ids[blockIdx.x / C];
  const FusedInst in = a.insts[inst_id];
  const float kappa = in.kappa;
  // active Fourier columns, rounded up to a multiple of 16 (every column when the
  // instance's multiplier reaches past that)
  const int kc = min(L1, (in.kcols + 15) & ~15);
  const float* mult = a.mult + in.g_off;
  const float2* bt = a.bt + in.g_off;
  const float2* c0 = a.c0 ? a.c0 + in.c_off : nullptr;
  float2* c_out = a.c_out + in.c_off;
  float2* aux_out = a.aux_out ? a.aux_out + in.c_off : nullptr;

  uint32_t peer[C];
  {
    const uint32_t w = smem_addr(cta.work);
#pragma unroll
    for (int c = 0; c < C; ++c) peer[c] = (C > 1) ? cluster_map(w, c) : w;
  }

  // ---- load twiddles, the frequency masks and the initial state
  cta.load_tables(a.twiddle, mult, bt, kc);
  uint2* const lo = ADMM ? nullptr : a.lo + in.c_off;
  float4* const hi = SPARSE ? a.hi + in.c_off : nullptr;
  for (int idx = threadIdx.x; idx < E; idx += T) {
    const int s = idx / L1, e = idx % L1;
    const int gidx = (crank + C * s) * L1 + e;
    float2 x = c0 ? c0[gidx] : make_float2(0.f, 0.f);
    if constexpr (!SPARSE) {
      cta.s0[idx] = x;                                 // c^(0) or z^(0)
      cta.s1[idx] = ADMM ? make_float2(0.f, 0.f) : x;  // z^(1) = c^(0), or v^(0) = 0
    }
    cta.work[s * P + pad16(e)] = x;
  }
  __syncthreads();

  // ISTA/FISTA state in compensated form (see the update below).  Every thread updates the same
  // positions, in the same order, in every iteration's epilogue; `live` has bit o set when its
  // o-th position holds a nonzero state.  The low-order parts of its first two live positions
  // sit in the thread's two shared-memory slots, those of any further ones in global memory (lo,
  // packed like c_out).  The first epilogue treats every position as live with a zero low-order
  // part (a complex64 warm start is exact), so no memory has to be cleared beforehand.
  // The sparse variant keeps the whole state of a live position, {c_hi, z_hi} and the low parts,
  // in the thread's two slots of the current set (global memory, hi and lo, for any further ones)
  // and writes the new state to the other set, so the sets alternate between iterations; the
  // first epilogue reads the warm start itself.
  uint32_t live = 0xffffffffu, live_next = 0u;
  int ord = 0, rank_old = 0, rank_new = 0, set = 0;
  uint2 slot_old0 = make_uint2(0u, 0u), slot_old1 = make_uint2(0u, 0u);
  bool first = true;
  auto epilogue_begin = [&]() {
    if constexpr (!ADMM) {
      if constexpr (!SPARSE) {
        if (!first) {
          slot_old0 = slot[0];
          slot_old1 = slot[1];
        }
      }
      ord = rank_old = rank_new = 0;
      live_next = 0u;
    }
  };
  auto epilogue_end = [&]() {
    if constexpr (!ADMM) {
      live = live_next;
      first = false;
      set ^= 1;
    }
  };

  // ISTA runs as FISTA with every momentum weight 0 (a zero table, or no table):
  // c + 0 (c - c_prev) = c exactly, so the iterates are ISTA's.

  // ISTA/FISTA.  The state is kept in compensated form: c = s0 + c_lo, z = s1 + z_lo, the high
  // parts complex64 in shared memory, the low parts bf16.  FISTA's momentum carries every
  // rounding at the scale of |z| through the rest of the solve (it has a double root at 1 along
  // directions the Gram does not see), so u = z - G', the soft-threshold and the momentum are
  // formed in double-float arithmetic; G' itself is of the size of the gradient and keeps its
  // FP32 transform.  The soft-threshold is taken as c = u - kappa u/|u|, whose rounded term is
  // of the size of kappa, not of |u|.
  //
  // quick: every output of the inverse transform (the thread's o-th).  Off the support the
  // state is exactly 0 and stays 0 while |G'| <= kappa: that element is finished here, touching
  // no memory.  Otherwise it is flagged and the (scaled) G' is kept for ext.
  auto quick = [&](int row, int e, int o, float2 g, bool& flag, float sc, float kap, float2* save_t) -> float2 {
    if constexpr (BLOCK) {
      if (e >= in.bl1 || crank + C * row >= in.bl2) {  // outside the caller's block: stays 0
        flag = false;
        return make_float2(0.f, 0.f);
      }
    }
    const bool was_live = (live >> o) & 1u;
    if constexpr (LEARN) {
      if (save_t) {
        const int gidx = (crank + C * row) * L1 + e;
        save_t[gidx] = was_live ? cta.s1[row * L1 + e] : make_float2(0.f, 0.f);
        save_t[a.save_stride + gidx] = g;
      }
      g = make_float2(sc * g.x, sc * g.y);
    } else {
      (void)sc;
      (void)save_t;
    }
    flag = was_live || (g.x * g.x + g.y * g.y > kap * kap);
    return flag ? g : make_float2(0.f, 0.f);
  };
  // ext: a flagged element, in ascending o; returns z^(t+1), the next FFT input
  auto ext = [&](int row, int e, int o, float2 g, float beta, float kap, bool last) -> float2 {
    const int sidx = row * L1 + e;
    const int gidx = (crank + C * row) * L1 + e;
    float2 c_old = make_float2(0.f, 0.f), x = make_float2(0.f, 0.f);  // c^(t-1), z^(t)
    float2 cl = make_float2(0.f, 0.f), zl = make_float2(0.f, 0.f);
    if ((live >> o) & 1u) {
      if constexpr (SPARSE) {
        if (first) {
          c_old = x = c0 ? c0[gidx] : make_float2(0.f, 0.f);  // c^(0), z^(1) = c^(0); exact
        } else {
          const int k = (set * 2 + rank_old) * T + (int)threadIdx.x;
          const float4 h = rank_old < 2 ? shi[k] : hi[gidx];
          const uint2 w = rank_old < 2 ? slo[k] : lo[gidx];
          c_old = make_float2(h.x, h.y);
          x = make_float2(h.z, h.w);
          cl = unpack_bf16x2(w.x);
          zl = unpack_bf16x2(w.y);
        }
      } else {
        c_old = cta.s0[sidx];
        x = cta.s1[sidx];
        if (!first) {
          const uint2 w = rank_old == 0 ? slot_old0 : rank_old == 1 ? slot_old1 : lo[gidx];
          cl = unpack_bf16x2(w.x);
          zl = unpack_bf16x2(w.y);
        }
      }
      ++rank_old;
    }
    float uxh, uxl, uyh, uyl;  // u = z - G'
    dd_add(x.x, zl.x, -g.x, 0.f, uxh, uxl);
    dd_add(x.y, zl.y, -g.y, 0.f, uyh, uyl);
    float cxh = 0.f, cxl = 0.f, cyh = 0.f, cyl = 0.f;
    const float r2 = uxh * uxh + uyh * uyh;
    if (r2 > kap * kap) {
      const float kr = kap * rsqrtf(r2);
      dd_add(uxh, uxl, -(kr * uxh), 0.f, cxh, cxl);
      dd_add(uyh, uyl, -(kr * uyh), 0.f, cyh, cyl);
    }
    float dxh, dxl, dyh, dyl;  // c^(t) - c^(t-1)
    dd_add(cxh, cxl, -c_old.x, -cl.x, dxh, dxl);
    dd_add(cyh, cyl, -c_old.y, -cl.y, dyh, dyl);
    float zxh, zxl, zyh, zyl;  // z^(t+1) = c^(t) + beta_t (c^(t) - c^(t-1))
    dd_axpy(beta, dxh, dxl, cxh, cxl, zxh, zxl);
    dd_axpy(beta, dyh, dyl, cyh, cyl, zyh, zyl);
    if constexpr (SPARSE) {
      if (last) c_out[gidx] = make_float2(cxh, cyh);
    } else {
      cta.s0[sidx] = make_float2(cxh, cyh);
      cta.s1[sidx] = make_float2(zxh, zyh);
      (void)last;
    }
    if ((cxh != 0.f) | (cyh != 0.f) | (zxh != 0.f) | (zyh != 0.f)) {
      const uint2 w = make_uint2(pack_bf16x2(cxl, cyl), pack_bf16x2(zxl, zyl));
      if constexpr (SPARSE) {
        const float4 h = make_float4(cxh, cyh, zxh, zyh);
        if (rank_new < 2) {
          const int k = ((set ^ 1) * 2 + rank_new) * T + (int)threadIdx.x;
          shi[k] = h;
          slo[k] = w;
        } else {
          hi[gidx] = h;
          lo[gidx] = w;
        }
      } else {
        if (rank_new < 2)
          slot[rank_new] = w;
        else
          lo[gidx] = w;
      }
      ++rank_new;
      live_next |= 1u << o;
    }
    return make_float2(zxh, zyh);
  };
  // ADMM: u = z - G' = c^(t+1) + v^(t), z^(t+1) = S(u), v^(t+1) = u - z^(t+1); returns z - v
  auto update_admm = [&](int row, int e, float2 g, bool last, float kap) -> float2 {
    const int sidx = row * L1 + e;
    const float2 zo = cta.s0[sidx];
    const float2 vo = cta.s1[sidx];
    const float2 un = make_float2(zo.x - g.x, zo.y - g.y);  // c^(t+1) + v^(t)
    const float2 zn = soft_threshold(un, kap);
    const float2 vn = make_float2(un.x - zn.x, un.y - zn.y);
    cta.s0[sidx] = zn;
    cta.s1[sidx] = vn;
    if (last && aux_out) aux_out[(crank + C * row) * L1 + e] = make_float2(un.x - vo.x, un.y - vo.y);
    return make_float2(zn.x - vn.x, zn.y - vn.y);
  };
  // per-iteration multipliers of the unrolled network (1 and kappa otherwise)
  auto layer = [&](int it, float& sc, float& kap, float2*& save_t) {
    if constexpr (LEARN) {
      sc = a.scale ? __ldg(&a.scale[it]) : 1.0f;
      kap = a.thresh ? __ldg(&a.thresh[it]) * kappa : kappa;
      save_t = a.save ? a.save + (int64_t)(2 * it) * a.save_stride + in.c_off : nullptr;
    } else {
      sc = 1.0f;
      kap = kappa;
      save_t = nullptr;
    }
  };

  if constexpr (S::SQ16) {
    const int nz = kc / 16;
    // the row stages run over S::PASSES bands of S::BAND rows (one band unless SPARSE)
    for (int b = 0; b < S::PASSES; ++b) {
      cta.band = b;
      cta.sq_fwd1_from_work();
    }
    for (int it = 0; it < a.iters; ++it) {
      const float beta = a.beta ? __ldg(&a.beta[it]) : 0.0f;
      const bool last = (it == a.iters - 1);
      for (int b = 0; b < S::PASSES; ++b) {
        cta.band = b;
        cta.sq_fwd2(nz);
      }
      __syncthreads();
      cta.template col_dft<false>(kc);
      cluster_barrier<C>();
      cta.middle(peer, mult, bt, kc);
      cluster_barrier<C>();
      cta.template col_dft<true>(kc);
      __syncthreads();
      if (nz > 2) {
        for (int b = 0; b < S::PASSES; ++b) {
          cta.band = b;
          cta.sq_inv1(nz);
        }
      }
      float sc, kap;
      float2* save_t;
      layer(it, sc, kap, save_t);
      if constexpr (ADMM) {
        cta.band = 0;
        cta.sq_inv2_epi_fwd1([&](int row, int e, float2 g) { return update_admm(row, e, g, last, kap); }, !last, nz);
      } else {
        if constexpr (SPARSE) {
          // The sparse variant writes its result from the last epilogue (no dense grid to copy
          // from): zeros at every position this thread updates there, then ext overwrites the
          // flagged ones.  After a single iteration every position is flagged (all live in the
          // first epilogue), and the warm start, read in that epilogue, stays untouched.
          if (last && !first) {
            for (int b = 0; b < S::PASSES; ++b) {
              cta.band = b;
              int row, j;
              cta.sq_rowj(row, j);
              float2* const o = c_out + (crank + C * row) * L1 + j;
#pragma unroll
              for (int i = 0; i < 16; ++i) o[16 * i] = make_float2(0.f, 0.f);
            }
          }
        }
        epilogue_begin();
        for (int b = 0; b < S::PASSES; ++b) {
          cta.band = b;
          cta.sq_inv2_split_fwd1(
              [&](int row, int e, int o, float2 g, bool& f) { return quick(row, e, o, g, f, sc, kap, save_t); },
              [&](int row, int e, int o, float2 g) { return ext(row, e, o, g, beta, kap, last); }, !last, nz);
        }
        epilogue_end();
      }
    }
  } else {
    for (int it = 0; it < a.iters; ++it) {
      const float beta = a.beta ? __ldg(&a.beta[it]) : 0.0f;
      const bool last = (it == a.iters - 1);
      cta.template row_fft_from<0, false>(
          [&](int row, int e, float2 x) {
            if (e < kc) cta.work[row * P + pad16(e)] = x;
          },
          L1);
      __syncthreads();
      cta.template col_dft<false>(kc);
      cluster_barrier<C>();
      cta.middle(peer, mult, bt, kc);
      cluster_barrier<C>();
      cta.template col_dft<true>(kc);
      __syncthreads();
      float sc, kap;
      float2* save_t;
      layer(it, sc, kap, save_t);
      if constexpr (ADMM) {
        cta.template row_fft_from<0, true>(
            [&](int row, int e, float2 g) { cta.work[row * P + pad16(e)] = update_admm(row, e, g, last, kap); },
            kc);
      } else {
        // the quick part inside the last row stage, then the flagged outputs (this thread's own
        // work positions) one by one, before the next stage reads them
        epilogue_begin();
        uint32_t flagged = 0u;
        cta.template row_fft_from<0, true>(
            [&](int row, int e, float2 g) {
              bool f;
              const int o = ord++;
              cta.work[row * P + pad16(e)] = quick(row, e, o, g, f, sc, kap, save_t);
              if (f) flagged |= 1u << o;
            },
            kc);
#pragma unroll 1
        for (uint32_t m = flagged; m; m &= m - 1u) {
          const int o = __ffs(m) - 1;
          int row, e;
          cta.last_row_output(o, row, e);
          float2* w = &cta.work[row * P + pad16(e)];
          *w = ext(row, e, o, *w, beta, kap, last);
        }
        if constexpr (S::ROW_WARP)
          __syncwarp();
        else
          __syncthreads();
        epilogue_end();
      }
    }
  }

  // ---- write the result (the sparse variant wrote it in the last epilogue)
  if constexpr (!SPARSE) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < E; idx += T) {
      const int s = idx / L1, e = idx % L1;
      c_out[(crank + C * s) * L1 + e] = cta.s0[idx];
    }
  }
  // no CTA may leave while a peer can still address its shared memory
  if constexpr (C > 1) cg::this_cluster().sync();
}

// ------------------------------------------------------------------------------------------
// host-side launch table
// ------------------------------------------------------------------------------------------
struct FusedEntry {
  int L1, L2, admm, tile, block, sparse;
  int cluster, threads, smem;
  cudaError_t (*launch)(const FusedArgs&, int n_inst, cudaStream_t);
  cudaError_t (*prepare)();
};

template <int L1, int L2, bool ADMM, int TILE, bool LEARN = false, bool BLOCK = false, bool SPARSE = false>
cudaError_t fused_prepare() {
  using S = FusedShape<L1, L2, ADMM, TILE, SPARSE>;
  cudaError_t e = cudaFuncSetAttribute(fused_solve_kernel<L1, L2, ADMM, TILE, LEARN, BLOCK, SPARSE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
  if (e == cudaSuccess && S::C > 8)
    e = cudaFuncSetAttribute(fused_solve_kernel<L1, L2, ADMM, TILE, LEARN, BLOCK, SPARSE>,
                             cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

template <int L1, int L2, bool ADMM, int TILE, bool LEARN = false, bool BLOCK = false, bool SPARSE = false>
cudaError_t fused_launch(const FusedArgs& a, int n_inst, cudaStream_t st) {
  using S = FusedShape<L1, L2, ADMM, TILE, SPARSE>;
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
  return cudaLaunchKernelEx(&cfg, fused_solve_kernel<L1, L2, ADMM, TILE, LEARN, BLOCK, SPARSE>, a);
}

template <int L1, int L2, bool ADMM, int TILE = kFusedTileElems, bool LEARN = false, bool BLOCK = false,
          bool SPARSE = false>
FusedEntry fused_entry() {
  using S = FusedShape<L1, L2, ADMM, TILE, SPARSE>;
  return FusedEntry{L1,      L2,      ADMM ? 1 : 0, TILE, BLOCK ? 1 : 0, SPARSE ? 1 : 0, S::C, S::T, S::SMEM,
                    &fused_launch<L1, L2, ADMM, TILE, LEARN, BLOCK, SPARSE>,
                    &fused_prepare<L1, L2, ADMM, TILE, LEARN, BLOCK, SPARSE>};
}

}  // namespace bccb
