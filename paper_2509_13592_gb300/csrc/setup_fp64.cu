// One-time FP64 work around the FP32 iterations:
//   * Lambda: the eigenvalues of the BCCB Gram A^H A, computed as the 2D DFT of its
//     first column (eq:lambda, property (iv)).  The first column itself,
//     g(k) = sum_n exp(+j 2 pi (k1 m1_n/L1 + k2 m2_n/L2)), is the unnormalised inverse
//     2D DFT of the element-count grid (kept elements folded modulo (L1, L2)).
//   * mu = 1 / sigma_max(A)^2 = 1 / max Lambda (eq:ista).
//   * b = A^H y: with gamma = 1/2 the dictionary entry is (-1)^(m1+m2) times a DFT
//     kernel, so b is the unnormalised inverse 2D DFT of the grid holding
//     (-1)^(m1+m2) y_n at (m1 mod L1, m2 mod L2) (eq:ista, eq:admm).
//   * the FP32 Fourier multiplier q and the Fourier-domain constant term Bt used by the
//     fused iterations: FFT2(b) is L1 L2 times the signed measurement grid, so Bt needs
//     no transform; for ADMM it carries the "precomputed" (A^H A + rho I)^{-1} A^H y of
//     eq:admm as FFT2(b)/(Lambda + rho).
//   * the final check: r = A^H (y - A c) = b - G c, the relative KKT residual of the
//     1/2-scaled LASSO, and the objective 1/2 ||y - A c||^2 + lam ||c||_1.
// The FP64 2D DFTs are radix-4 Stockham passes (rows, then columns) over global
// memory with each row / column tile staged in shared memory.
#include <math.h>

#include <algorithm>
#include <vector>

#include "fft_smem.cuh"
#include "solver.h"

namespace bccb {

namespace {

constexpr int kThreads = 256;

// In-place DFT of every row (length L1) of every instance's grid (of the instances sel lists,
// when sel is given).  The DFT of a row of zeros is zeros: such a row is left as it is.
__global__ void fft64_rows_kernel(const InstDesc* __restrict__ desc, const int* __restrict__ sel, double2* base,
                                  int inv, const double2* __restrict__ tw) {
  const InstDesc d = desc[sel ? sel[blockIdx.x] : blockIdx.x];
  if ((int)blockIdx.y >= d.L2) return;
  extern __shared__ double2 sm64[];
  double2* x = sm64;
  double2* y = sm64 + d.L1;
  double2* g = base + d.g_off + (int64_t)blockIdx.y * d.L1;
  int nz = 0;
  for (int e = threadIdx.x; e < d.L1; e += blockDim.x) {
    const double2 v = g[e];
    x[e] = v;
    nz |= (v.x != 0.0) | (v.y != 0.0);
  }
  if (!__syncthreads_or(nz)) return;
  const double2* out = inv ? fft_smem<double2, true>(x, y, d.L1, 1, tw) : fft_smem<double2, false>(x, y, d.L1, 1, tw);
  for (int e = threadIdx.x; e < d.L1; e += blockDim.x) g[e] = out[e];
}

// columns staged per block: 8, or fewer so that two L2 x cpb FP64 tiles fit in 128 KB
int cols_per_block(int max_L2) { return max_L2 <= 512 ? 8 : 4096 / max_L2; }

// In-place DFT of every column (length L2) of every instance's grid (of the instances sel
// lists, when sel is given), cpb at a time; with lim given, only columns < lim[i].kcols.
__global__ void fft64_cols_kernel(const InstDesc* __restrict__ desc, const int* __restrict__ sel, double2* base,
                                  int inv, const double2* __restrict__ tw, int cpb, const FusedInst* __restrict__ lim) {
  const int i = sel ? sel[blockIdx.x] : blockIdx.x;
  const InstDesc d = desc[i];
  const int ncols = lim ? min(d.L1, lim[i].kcols) : d.L1;
  const int c0 = blockIdx.y * cpb;
  if (c0 >= ncols) return;
  const int cnt = min(cpb, ncols - c0);
  extern __shared__ double2 sm64[];
  double2* x = sm64;
  double2* y = sm64 + d.L2 * cnt;
  double2* g = base + d.g_off;
  for (int idx = threadIdx.x; idx < d.L2 * cnt; idx += blockDim.x) {
    const int e = idx / cnt, q = idx % cnt;
    x[idx] = g[(int64_t)e * d.L1 + c0 + q];
  }
  __syncthreads();
  const double2* out =
      inv ? fft_smem<double2, true>(x, y, d.L2, cnt, tw) : fft_smem<double2, false>(x, y, d.L2, cnt, tw);
  for (int idx = threadIdx.x; idx < d.L2 * cnt; idx += blockDim.x) {
    const int e = idx / cnt, q = idx % cnt;
    g[(int64_t)e * d.L1 + c0 + q] = out[idx];
  }
}

// count grid (for Lambda) and the signed measurement grid (for b); Y = float2 or double2
template <typename Y>
__global__ void scatter_kernel(const InstDesc* __restrict__ desc, const int* __restrict__ mask_idx,
                               const Y* __restrict__ y, double2* cnt_grid, double2* meas_grid) {
  const InstDesc d = desc[blockIdx.x];
  const int L = d.L1 * d.L2;
  const int* mi = mask_idx + d.mask_off;
  const Y* yi = y ? y + d.y_off : nullptr;
  for (int cell = blockIdx.y * blockDim.x + threadIdx.x; cell < L; cell += gridDim.y * blockDim.x) {
    const int p1 = cell % d.L1, p2 = cell / d.L1;
    double cnt = 0.0;
    double2 acc = make_double2(0.0, 0.0);
    for (int m2 = p2; m2 < d.M2; m2 += d.L2) {
      for (int m1 = p1; m1 < d.M1; m1 += d.L1) {
        const int n = mi[m1 + m2 * d.M1];
        if (n >= 0) {
          cnt += 1.0;
          if (y) {  // y = NULL: the mask part alone (Lambda, mu), as if y were 0
            const double sgn = ((m1 + m2) & 1) ? -1.0 : 1.0;
            acc.x += sgn * (double)yi[n].x;
            acc.y += sgn * (double)yi[n].y;
          }
        }
      }
    }
    cnt_grid[d.g_off + cell] = make_double2(cnt, 0.0);
    meas_grid[d.g_off + cell] = acc;
  }
}

template <typename T, typename Op>
__device__ T block_reduce(T v, Op op, T* sh, T identity) {
  for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < (int)(blockDim.x >> 5)) ? sh[l] : identity;
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (l == 0) sh[0] = v;
  }
  __syncthreads();
  v = sh[0];
  __syncthreads();
  return v;
}

struct MaxOp {
  __device__ double operator()(double a, double b) const { return fmax(a, b); }
};
struct SumOp {
  __device__ double operator()(double a, double b) const { return a + b; }
};

// Lambda (real part of the FFT2 of the Gram's first column), mu = 1/max Lambda, the FP32
// Fourier multiplier q and the FP32 Fourier-domain constant term Bt (both include the
// 1/(L1 L2) of the unnormalised inverse DFT):
//   ISTA/FISTA: q = mu Lambda / L,          Bt = mu * FFT2(b) / L = mu * s
//   ADMM:       q = Lambda/(Lambda+rho)/L,  Bt = FFT2(b) / (Lambda + rho) / L = s / (Lambda + rho)
// where s is the signed, folded measurement grid (FFT2(b) = L * s because b is the
// unnormalised inverse DFT of s).  Entries of Lambda below 1e-9 max Lambda are the
// round-off of the FP64 DFTs of an exactly zero eigenvalue and are set to 0.
// With lam_src given, instance i takes Lambda from the grid of instance lam_src[i] (an instance
// with the same array and grid, whose transform ran in its place).
__global__ void eig_mult_kernel(const InstDesc* __restrict__ desc, const int* __restrict__ lam_src,
                                const double2* __restrict__ lam_grid, const double2* __restrict__ sgrid,
                                double* lam64, InstParams* par, float* mult, float2* bt, double* mult64,
                                double2* bt64, FusedInst* fused, int algo, double rho) {
  __shared__ double sh[32];
  const InstDesc d = desc[blockIdx.x];
  const int L = d.L1 * d.L2;
  const double2* lam_c = lam_grid + (lam_src ? desc[lam_src[blockIdx.x]].g_off : d.g_off);
  double top = 0.0;
  for (int cell = threadIdx.x; cell < L; cell += blockDim.x) top = fmax(top, lam_c[cell].x);
  top = block_reduce(top, MaxOp(), sh, 0.0);
  // an all-zero mask (no element kept: A has no rows) has Lambda = 0; mu = 0 then makes q,
  // Bt and kappa 0 and the iterations return c = 0, the minimiser of the data-free problem
  const double mu = top > 0.0 ? 1.0 / top : 0.0;
  const double inv_L = 1.0 / (double)L;
  // inv_L is a power of two, so mu inv_L is exact and lv (mu inv_L) rounds like (mu lv) inv_L
  const double mu_L = mu * inv_L;
  int kc = 0;  // 1 + largest Fourier column with a nonzero multiplier or constant term
  for (int cell = threadIdx.x; cell < L; cell += blockDim.x) {
    double lv = lam_c[cell].x;
    if (lv < 1e-9 * top) lv = 0.0;
    lam64[d.g_off + cell] = lv;
    const double2 sv = sgrid[d.g_off + cell];
    double m, bs;
    if (algo == 2) {
      m = lv / (lv + rho) * inv_L;
      bs = 1.0 / (lv + rho);
    } else {
      m = lv * mu_L;
      bs = mu;
    }
    const float mf = (float)m;
    const float2 bf = make_float2((float)(sv.x * bs), (float)(sv.y * bs));
    mult[d.g_off + cell] = mf;
    bt[d.g_off + cell] = bf;
    if (mult64) {
      mult64[d.g_off + cell] = m;
      bt64[d.g_off + cell] = make_double2(sv.x * bs, sv.y * bs);
    }
    if (m != 0.0 || sv.x != 0.0 || sv.y != 0.0) kc = max(kc, (cell & (d.L1 - 1)) + 1);
  }
  const double kc_all = block_reduce((double)kc, MaxOp(), sh, 0.0);
  if (threadIdx.x == 0) {
    par[blockIdx.x].mu = mu;
    par[blockIdx.x].lam_top = top;
    fused[blockIdx.x].kcols = (int)kc_all;
  }
}

// lam (absolute, or a fraction of ||A^H y||_inf) and the soft-threshold kappa
__global__ void lam_kappa_kernel(const InstDesc* __restrict__ desc, const double2* __restrict__ b64,
                                 InstParams* par, FusedInst* fused, int algo, double rho) {
  __shared__ double sh[32];
  const InstDesc d = desc[blockIdx.x];
  const int L = d.L1 * d.L2;
  // max |b| = sqrt(max |b|^2): the correctly rounded square root is monotone, so one root
  // per instance gives the same value as one per cell
  double bmax2 = 0.0;
  for (int cell = threadIdx.x; cell < L; cell += blockDim.x) {
    const double2 bv = b64[d.g_off + cell];
    bmax2 = fmax(bmax2, bv.x * bv.x + bv.y * bv.y);
  }
  const double bmax = sqrt(block_reduce(bmax2, MaxOp(), sh, 0.0));
  if (threadIdx.x == 0) {
    const double mu = par[blockIdx.x].mu;
    const double lam = d.lam_is_frac ? d.lam * bmax : d.lam;
    par[blockIdx.x].lam = lam;
    par[blockIdx.x].lmax = bmax;
    fused[blockIdx.x].kappa = (float)(algo == 2 ? lam / rho : mu * lam);
  }
}

// w <- c (solution in the solver's grid layout; C = float2 or double2)
template <typename C>
__global__ void load_solution_kernel(const InstDesc* __restrict__ desc, const C* __restrict__ c, double2* w) {
  const InstDesc d = desc[blockIdx.x];
  const int L = d.L1 * d.L2;
  for (int cell = blockIdx.y * blockDim.x + threadIdx.x; cell < L; cell += gridDim.y * blockDim.x) {
    const C v = c[d.c_off + cell];
    w[d.g_off + cell] = make_double2((double)v.x, (double)v.y);
  }
}

// sum_n |y_n - (A c)_n|^2 with (A c)_n = (-1)^(m1+m2) FFT2(c)[m2 mod L2, m1 mod L1]
template <typename Y>
__global__ void data_residual_kernel(const InstDesc* __restrict__ desc, const int* __restrict__ mask_idx,
                                     const Y* __restrict__ y, const double2* __restrict__ cf, double* red) {
  __shared__ double sh[32];
  const InstDesc d = desc[blockIdx.x];
  const int* mi = mask_idx + d.mask_off;
  const Y* yi = y + d.y_off;
  double acc = 0.0;
  for (int pos = threadIdx.x; pos < d.M1 * d.M2; pos += blockDim.x) {
    const int n = mi[pos];
    if (n < 0) continue;
    const int m1 = pos % d.M1, m2 = pos / d.M1;
    const double sgn = ((m1 + m2) & 1) ? -1.0 : 1.0;
    const double2 v = cf[d.g_off + (int64_t)(m2 % d.L2) * d.L1 + (m1 % d.L1)];
    const double ex = (double)yi[n].x - sgn * v.x, ey = (double)yi[n].y - sgn * v.y;
    acc += ex * ex + ey * ey;
  }
  acc = block_reduce(acc, SumOp(), sh, 0.0);
  if (threadIdx.x == 0) red[blockIdx.x] = acc;
}

__global__ void mul_lambda_kernel(const InstDesc* __restrict__ desc, const double* __restrict__ lam64,
                                  double2* w) {
  const InstDesc d = desc[blockIdx.x];
  const int L = d.L1 * d.L2;
  for (int cell = blockIdx.y * blockDim.x + threadIdx.x; cell < L; cell += gridDim.y * blockDim.x) {
    const double s = lam64[d.g_off + cell];
    const double2 v = w[d.g_off + cell];
    w[d.g_off + cell] = make_double2(v.x * s, v.y * s);
  }
}

// r = b - G c (G c = IFFT2(Lambda FFT2(c)), held unnormalised in w); KKT residual and objective
template <typename C>
__global__ void kkt_final_kernel(const InstDesc* __restrict__ desc, const double2* __restrict__ b64,
                                 const double2* __restrict__ gc, const C* __restrict__ c,
                                 const InstParams* __restrict__ par, const double* __restrict__ red,
                                 double* kkt, double* obj) {
  __shared__ double sh[32];
  const InstDesc d = desc[blockIdx.x];
  const int L = d.L1 * d.L2;
  const double lam = par[blockIdx.x].lam;
  const double inv_L = 1.0 / (double)L;
  // On a zero entry the violation max(|r| - lam, 0) is a monotone function of |r|^2 (each step
  // correctly rounded), so the largest |r|^2 over the zero entries gives their largest violation:
  // one square root per thread instead of one per cell.
  double worst = 0.0, l1 = 0.0, r2_zero = 0.0;
  for (int cell = threadIdx.x; cell < L; cell += blockDim.x) {
    const double2 bv = b64[d.g_off + cell];
    const double2 gv = gc[d.g_off + cell];
    const double rx = bv.x - gv.x * inv_L, ry = bv.y - gv.y * inv_L;
    const C cv = c[d.c_off + cell];
    const double cx = cv.x, cy = cv.y;
    if (cx != 0.0 || cy != 0.0) {
      const double mag = sqrt(cx * cx + cy * cy);
      l1 += mag;
      if (mag > 0.0) {
        const double ex = rx - lam * cx / mag, ey = ry - lam * cy / mag;
        worst = fmax(worst, sqrt(ex * ex + ey * ey));
        continue;
      }
    }
    r2_zero = fmax(r2_zero, rx * rx + ry * ry);
  }
  worst = fmax(worst, fmax(sqrt(r2_zero) - lam, 0.0));
  worst = block_reduce(worst, MaxOp(), sh, 0.0);
  l1 = block_reduce(l1, SumOp(), sh, 0.0);
  if (threadIdx.x == 0) {
    kkt[blockIdx.x] = lam > 0.0 ? worst / lam : worst;
    obj[blockIdx.x] = 0.5 * red[blockIdx.x] + lam * l1;
  }
}

__global__ void fista_beta_kernel(float* beta, double* beta64, int iters) {
  // alpha_1 = 1, alpha_(t+1) = (1 + sqrt(1 + 4 alpha_t^2))/2, beta_t = (alpha_t - 1)/alpha_(t+1),
  // evaluated in FP64 with explicit round-to-nearest operations (no contraction).
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 1.0;
  for (int t = 0; t < iters; ++t) {
    const double an = __dmul_rn(__dadd_rn(1.0, __dsqrt_rn(__dadd_rn(1.0, __dmul_rn(__dmul_rn(4.0, a), a)))), 0.5);
    const double b = __ddiv_rn(__dadd_rn(a, -1.0), an);
    beta[t] = (float)b;
    if (beta64) beta64[t] = b;
    a = an;
  }
}

dim3 grid_cells(const bccb_solver* s) {
  const int cells = s->max_L1 * s->max_L2;
  const int blocks = (cells + kThreads - 1) / kThreads;
  return dim3((unsigned)s->n, (unsigned)(blocks < 64 ? blocks : 64));
}

void fft64_rows(bccb_solver* s, double2* grid, int inv, int rows, const int* sel, int count) {
  const int nb = sel ? count : s->n;
  const int ry = rows > 0 ? std::min(rows, s->max_L2) : s->max_L2;
  const size_t smr = (size_t)2 * s->max_L1 * sizeof(double2);
  fft64_rows_kernel<<<dim3(nb, ry), 128, smr, s->stream>>>(s->d_desc, sel, grid, inv, s->d_tw64);
  s->launches += 1;
}

void fft64_cols(bccb_solver* s, double2* grid, int inv, const int* sel, int count, const FusedInst* lim) {
  const int nb = sel ? count : s->n;
  const int cpb = cols_per_block(s->max_L2);
  const size_t smc = (size_t)2 * s->max_L2 * cpb * sizeof(double2);
  fft64_cols_kernel<<<dim3(nb, (s->max_L1 + cpb - 1) / cpb), 128, smc, s->stream>>>(s->d_desc, sel, grid, inv,
                                                                                     s->d_tw64, cpb, lim);
  s->launches += 1;
}

// FFT2 of every instance's grid, or of the `count` instances listed in sel; rows > 0 says that
// every row from `rows` on is zero in each grid (the rows pass then launches only the others).
cudaError_t fft2_64(bccb_solver* s, double2* grid, int inv, int rows = 0, const int* sel = nullptr, int count = 0) {
  fft64_rows(s, grid, inv, rows, sel, count);
  fft64_cols(s, grid, inv, sel, count, nullptr);
  return cudaGetLastError();
}


// ------------------------------------------------------------------------------------------
// Element spacing gamma != 1/2 (Section III-A): on the grids f_{i,l} = -gamma_i + l 2 gamma_i/L_i
// (eq:uniform_grid) the Gram G = A^H A is block Toeplitz with Toeplitz blocks,
//   G[l, l'] = g(l1 - l1', l2 - l2'),  g(d1, d2) = sum_n exp(+j 2 pi (2 gamma1 d1 m1_n / L1 + 2 gamma2 d2 m2_n / L2)),
// for lags |d_i| < L_i.  Its product is the top-left L1 x L2 block of the product with the
// 2L1 x 2L2 circulant whose first column holds g at lags d (d >= 0) and d - 2L (d > L), and 0 at
// d = L (the lag no pair of block entries uses): the same FFT2 iteration then runs on the
// embedded grid with the unknown kept at 0 outside the block.  Here the descriptor's L1 x L2 is
// the embedded grid and bL1 x bL2 the block (the caller's grid).  mu = 1/lambda_max(G) =
// 1/lambda_max(A A^H) (eq:ista) comes from an FP32 power iteration on the N x N matrix A A^H,
// finished by its FP64 Rayleigh quotient (accurate to the square of the vector's error).
// ------------------------------------------------------------------------------------------

// lag of embedded index e on an axis of block length Lb (embedded 2 Lb); Lb itself is unused
__device__ __forceinline__ int toep_lag(int e, int Lb) { return e < Lb ? e : e - 2 * Lb; }

// h[e1][m2] = sum over kept m1 of exp(+j 2 pi 2 gamma1 d1 m1 / bL1), d1 = lag(e1); 0 at e1 = bL1
__global__ void toep_col1_kernel(const InstDesc* __restrict__ desc, const int* __restrict__ mask_idx, double g1,
                                 double2* h) {
  const InstDesc d = desc[blockIdx.x];
  const int* mi = mask_idx + d.mask_off;
  for (int t = blockIdx.y * blockDim.x + threadIdx.x; t < d.L1 * d.M2; t += gridDim.y * blockDim.x) {
    const int e1 = t % d.L1, m2 = t / d.L1;
    double2 acc = make_double2(0.0, 0.0);
    if (e1 != d.bL1) {
      const double w = 2.0 * g1 * (double)toep_lag(e1, d.bL1) / (double)d.bL1;
      for (int m1 = 0; m1 < d.M1; ++m1) {
        if (mi[m1 + m2 * d.M1] < 0) continue;
        double sn, cs;
        sincospi(2.0 * w * (double)m1, &sn, &cs);
        acc.x += cs;
        acc.y += sn;
      }
    }
    h[d.g_off + t] = acc;
  }
}

// first column of the embedding: sum_m2 h[e1][m2] exp(+j 2 pi 2 gamma2 d2 m2 / bL2); 0 at e2 = bL2
__global__ void toep_col2_kernel(const InstDesc* __restrict__ desc, const double2* __restrict__ h, double g2,
                                 double2* w) {
  const InstDesc d = desc[blockIdx.x];
  const int L = d.L1 * d.L2;
  for (int cell = blockIdx.y * blockDim.x + threadIdx.x; cell < L; cell += gridDim.y * blockDim.x) {
    const int e1 = cell % d.L1, e2 = cell / d.L1;
    double2 acc = make_double2(0.0, 0.0);
    if (e2 != d.bL2) {
      const double wt = 2.0 * g2 * (double)toep_lag(e2, d.bL2) / (double)d.bL2;
      for (int m2 = 0; m2 < d.M2; ++m2) {
        const double2 hv = h[d.g_off + e1 + (int64_t)m2 * d.L1];
        double sn, cs;
        sincospi(2.0 * wt * (double)m2, &sn, &cs);
        acc.x += hv.x * cs - hv.y * sn;
        acc.y += hv.x * sn + hv.y * cs;
      }
    }
    w[d.g_off + cell] = acc;
  }
}

// b = A^H y on the block, 0 elsewhere: hb[l1][m2] = sum_m1 exp(+j 2 pi f1 m1) y(m1, m2), then
// b[l2][l1] = sum_m2 exp(+j 2 pi f2 m2) hb[l1][m2], with f_i = -gamma_i + l 2 gamma_i / bL_i
template <typename Y>
__global__ void toep_b1_kernel(const InstDesc* __restrict__ desc, const int* __restrict__ mask_idx,
                               const Y* __restrict__ y, double g1, double2* h) {
  const InstDesc d = desc[blockIdx.x];
  const int* mi = mask_idx + d.mask_off;
  const Y* yi = y ? y + d.y_off : nullptr;
  for (int t = blockIdx.y * blockDim.x + threadIdx.x; t < d.bL1 * d.M2; t += gridDim.y * blockDim.x) {
    const int l1 = t % d.bL1, m2 = t / d.bL1;
    const double f1 = -g1 + (double)l1 * (2.0 * g1 / (double)d.bL1);
    double2 acc = make_double2(0.0, 0.0);
    for (int m1 = 0; m1 < d.M1 && yi; ++m1) {  // y = NULL: b = 0 (the mask part alone)
      const int n = mi[m1 + m2 * d.M1];
      if (n < 0) continue;
      double sn, cs;
      sincospi(2.0 * f1 * (double)m1, &sn, &cs);
      const double yx = (double)yi[n].x, yy = (double)yi[n].y;
      acc.x += cs * yx - sn * yy;
      acc.y += cs * yy + sn * yx;
    }
    h[d.g_off + t] = acc;
  }
}

__global__ void toep_b2_kernel(const InstDesc* __restrict__ desc, const double2* __restrict__ h, double g2,
                               double2* b) {
  const InstDesc d = desc[blockIdx.x];
  const int L = d.L1 * d.L2;
  for (int cell = blockIdx.y * blockDim.x + threadIdx.x; cell < L; cell += gridDim.y * blockDim.x) {
    const int e1 = cell % d.L1, e2 = cell / d.L1;
    double2 acc = make_double2(0.0, 0.0);
    if (e1 < d.bL1 && e2 < d.bL2) {
      const double f2 = -g2 + (double)e2 * (2.0 * g2 / (double)d.bL2);
      for (int m2 = 0; m2 < d.M2; ++m2) {
        const double2 hv = h[d.g_off + e1 + (int64_t)m2 * d.bL1];
        double sn, cs;
        sincospi(2.0 * f2 * (double)m2, &sn, &cs);
        acc.x += hv.x * cs - hv.y * sn;
        acc.y += hv.x * sn + hv.y * cs;
      }
    }
    b[d.g_off + cell] = acc;
  }
}

// lambda_max(A A^H): (A A^H)[n, n'] = S1(m1_n - m1_n') S2(m2_n - m2_n') with
// S_i(k) = sum_{l < bL_i} exp(-j 2 pi f_{i,l} k).  One CTA per instance; N <= kToepMaxN.

__device__ double2 toep_s(int k, int Lb, double g) {
  double2 acc = make_double2(0.0, 0.0);
  for (int l = 0; l < Lb; ++l) {
    const double f = -g + (double)l * (2.0 * g / (double)Lb);
    double sn, cs;
    sincospi(-2.0 * f * (double)k, &sn, &cs);
    acc.x += cs;
    acc.y += sn;
  }
  return acc;
}

__global__ void __launch_bounds__(1024) toep_mu_kernel(const InstDesc* __restrict__ desc,
                                                       const int* __restrict__ mask_idx, double g1, double g2,
                                                       InstParams* par) {
  extern __shared__ double2 tsm[];
  const InstDesc d = desc[blockIdx.x];
  const int N = d.N, M1 = d.M1, M2 = d.M2;
  double2* s1 = tsm;                        // 2 M1 - 1, index k + M1 - 1
  double2* s2 = s1 + (2 * M1 - 1);          // 2 M2 - 1
  float2* f1 = reinterpret_cast<float2*>(s2 + (2 * M2 - 1));
  float2* f2 = f1 + (2 * M1 - 1);
  float2* v = f2 + (2 * M2 - 1);            // N
  float2* w = v + N;                        // N
  int* pm1 = reinterpret_cast<int*>(w + N);  // N
  int* pm2 = pm1 + N;                        // N
  __shared__ double red[32];
  const int* mi = mask_idx + d.mask_off;
  for (int k = threadIdx.x; k < 2 * M1 - 1; k += blockDim.x) {
    s1[k] = toep_s(k - (M1 - 1), d.bL1, g1);
    f1[k] = make_float2((float)s1[k].x, (float)s1[k].y);
  }
  for (int k = threadIdx.x; k < 2 * M2 - 1; k += blockDim.x) {
    s2[k] = toep_s(k - (M2 - 1), d.bL2, g2);
    f2[k] = make_float2((float)s2[k].x, (float)s2[k].y);
  }
  for (int cell = threadIdx.x; cell < M1 * M2; cell += blockDim.x) {
    const int n = mi[cell];
    if (n >= 0) {
      pm1[n] = cell % M1;
      pm2[n] = cell / M1;
    }
  }
  for (int n = threadIdx.x; n < N; n += blockDim.x) v[n] = make_float2(1.0f + 0.25f * __sinf(0.7f * n), 0.0f);
  __syncthreads();
  double rq_prev = -1.0, rq = 0.0;
  for (int outer = 0; outer < 256; ++outer) {
    for (int it = 0; it < 64; ++it) {
      // w = B v (FP32), then v = w / ||w||
      float nrm = 0.f;
      for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const int a1 = pm1[n] + M1 - 1, a2 = pm2[n] + M2 - 1;
        float ax = 0.f, ay = 0.f;
        for (int q = 0; q < N; ++q) {
          const float2 p = f1[a1 - pm1[q]], r = f2[a2 - pm2[q]];
          const float bx = p.x * r.x - p.y * r.y, by = p.x * r.y + p.y * r.x;
          const float2 vq = v[q];
          ax += bx * vq.x - by * vq.y;
          ay += bx * vq.y + by * vq.x;
        }
        w[n] = make_float2(ax, ay);
        nrm += ax * ax + ay * ay;
      }
      const double tot = block_reduce((double)nrm, SumOp(), red, 0.0);
      const float inv = (float)(1.0 / sqrt(tot > 0.0 ? tot : 1.0));
      for (int n = threadIdx.x; n < N; n += blockDim.x) v[n] = make_float2(w[n].x * inv, w[n].y * inv);
      __syncthreads();
    }
    // FP64 Rayleigh quotient v^H B v / v^H v
    double num = 0.0, den = 0.0;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
      const int a1 = pm1[n] + M1 - 1, a2 = pm2[n] + M2 - 1;
      double ax = 0.0, ay = 0.0;
      for (int q = 0; q < N; ++q) {
        const double2 p = s1[a1 - pm1[q]], r = s2[a2 - pm2[q]];
        const double bx = p.x * r.x - p.y * r.y, by = p.x * r.y + p.y * r.x;
        const double vx = v[q].x, vy = v[q].y;
        ax += bx * vx - by * vy;
        ay += bx * vy + by * vx;
      }
      const double vx = v[n].x, vy = v[n].y;
      num += vx * ax + vy * ay;  // Re(conj(v_n) (B v)_n)
      den += vx * vx + vy * vy;
    }
    num = block_reduce(num, SumOp(), red, 0.0);
    den = block_reduce(den, SumOp(), red, 0.0);
    rq = num / den;
    if (fabs(rq - rq_prev) <= 1e-14 * rq) break;
    rq_prev = rq;
  }
  if (threadIdx.x == 0) {
    par[blockIdx.x].mu = 1.0 / rq;
    par[blockIdx.x].lam_top = rq;
  }
}

// Lambda_ext (real part of the embedding's spectrum), q = mu Lambda_ext / L and
// Bt = mu FFT2(b)/L over the embedded grid (L = its size); the whole spectrum is active
__global__ void toep_lam_kernel(const InstDesc* __restrict__ desc, const double2* __restrict__ lam_c, double* lam64) {
  const InstDesc d = desc[blockIdx.x];
  const int L = d.L1 * d.L2;
  for (int cell = blockIdx.y * blockDim.x + threadIdx.x; cell < L; cell += gridDim.y * blockDim.x)
    lam64[d.g_off + cell] = lam_c[d.g_off + cell].x;
}

__global__ void toep_mult_kernel(const InstDesc* __restrict__ desc, const double* __restrict__ lam64,
                                 const double2* __restrict__ fb, const InstParams* __restrict__ par, float* mult,
                                 float2* bt, double* mult64, double2* bt64, FusedInst* fused) {
  const InstDesc d = desc[blockIdx.x];
  const int L = d.L1 * d.L2;
  const double mu = par[blockIdx.x].mu, inv_L = 1.0 / (double)L;
  for (int cell = blockIdx.y * blockDim.x + threadIdx.x; cell < L; cell += gridDim.y * blockDim.x) {
    const double lv = lam64[d.g_off + cell];
    const double2 f = fb[d.g_off + cell];
    const double m = mu * lv * inv_L;
    mult[d.g_off + cell] = (float)m;
    bt[d.g_off + cell] = make_float2((float)(mu * f.x * inv_L), (float)(mu * f.y * inv_L));
    if (mult64) {
      mult64[d.g_off + cell] = m;
      bt64[d.g_off + cell] = make_double2(mu * f.x * inv_L, mu * f.y * inv_L);
    }
  }
  if (threadIdx.x == 0 && blockIdx.y == 0) fused[blockIdx.x].kcols = d.L1;
}

// KKT residual and objective on the block: r = b - G c with G c the block of the
// (unnormalised) embedded product in gc; objective 1/2 ||y||^2 - Re(b^H c) + 1/2 Re(c^H G c) + lam ||c||_1
template <typename C>
__global__ void toep_kkt_kernel(const InstDesc* __restrict__ desc, const double2* __restrict__ b64,
                                const double2* __restrict__ gc, const C* __restrict__ c, const C* __restrict__ y,
                                const InstParams* __restrict__ par, double* kkt, double* obj) {
  __shared__ double sh[32];
  const InstDesc d = desc[blockIdx.x];
  const double lam = par[blockIdx.x].lam;
  const double inv_L = 1.0 / (double)(d.L1 * d.L2);
  double worst = 0.0, l1 = 0.0, bc = 0.0, cgc = 0.0, yy = 0.0;
  for (int t = threadIdx.x; t < d.bL1 * d.bL2; t += blockDim.x) {
    const int cell = (t % d.bL1) + (t / d.bL1) * d.L1;
    const double2 bv = b64[d.g_off + cell];
    const double2 g = make_double2(gc[d.g_off + cell].x * inv_L, gc[d.g_off + cell].y * inv_L);
    const double rx = bv.x - g.x, ry = bv.y - g.y;
    const C cv = c[d.c_off + cell];
    const double cx = cv.x, cy = cv.y;
    const double mag = sqrt(cx * cx + cy * cy);
    double viol;
    if (mag > 0.0) {
      const double ex = rx - lam * cx / mag, ey = ry - lam * cy / mag;
      viol = sqrt(ex * ex + ey * ey);
    } else {
      viol = fmax(sqrt(rx * rx + ry * ry) - lam, 0.0);
    }
    worst = fmax(worst, viol);
    l1 += mag;
    bc += bv.x * cx + bv.y * cy;  // Re(conj(b) c)
    cgc += cx * g.x + cy * g.y;   // Re(conj(c) G c)
  }
  for (int n = threadIdx.x; n < d.N; n += blockDim.x) {
    const C v = y[d.y_off + n];
    yy += (double)v.x * v.x + (double)v.y * v.y;
  }
  worst = block_reduce(worst, MaxOp(), sh, 0.0);
  l1 = block_reduce(l1, SumOp(), sh, 0.0);
  bc = block_reduce(bc, SumOp(), sh, 0.0);
  cgc = block_reduce(cgc, SumOp(), sh, 0.0);
  yy = block_reduce(yy, SumOp(), sh, 0.0);
  if (threadIdx.x == 0) {
    kkt[blockIdx.x] = lam > 0.0 ? worst / lam : worst;
    obj[blockIdx.x] = 0.5 * yy - bc + 0.5 * cgc + lam * l1;
  }
}

// caller's packing (block grids at u_off) <-> embedded grids (at c_off, zero outside the block)
template <typename C>
__global__ void toep_pad_kernel(const InstDesc* __restrict__ desc, const C* __restrict__ cu, C* ci) {
  const InstDesc d = desc[blockIdx.x];
  const int L = d.L1 * d.L2;
  for (int cell = blockIdx.y * blockDim.x + threadIdx.x; cell < L; cell += gridDim.y * blockDim.x) {
    const int e1 = cell % d.L1, e2 = cell / d.L1;
    C v;
    v.x = 0;
    v.y = 0;
    if (cu && e1 < d.bL1 && e2 < d.bL2) v = cu[d.u_off + e1 + (int64_t)e2 * d.bL1];
    ci[d.c_off + cell] = v;
  }
}

template <typename C>
__global__ void toep_crop_kernel(const InstDesc* __restrict__ desc, const C* __restrict__ ci, C* cu) {
  const InstDesc d = desc[blockIdx.x];
  for (int t = blockIdx.y * blockDim.x + threadIdx.x; t < d.bL1 * d.bL2; t += gridDim.y * blockDim.x)
    cu[d.u_off + t] = ci[d.c_off + (t % d.bL1) + (int64_t)(t / d.bL1) * d.L1];
}


// ---- dLoss/dy of the unrolled network (bccb_unrolled_bwd): b = A^H y enters every layer, so
// with g_b = dLoss/db, g_y = A g_b, and (A v)_n = (-1)^(m1+m2) FFT2(v)[m2 mod L2][m1 mod L1]
// (the unnormalised forward DFT; A's columns are exp(-j 2 pi f.m) with f = -1/2 + l/L).

// w = mu * (sum_k a_k g_{u_k}): the layers' part of g_b
__global__ void gy_load_kernel(const InstDesc* __restrict__ desc, const InstParams* __restrict__ par,
                               const float2* __restrict__ grad_b, double2* w) {
  const InstDesc d = desc[blockIdx.x];
  const double mu = par[blockIdx.x].mu;
  for (int cell = blockIdx.y * blockDim.x + threadIdx.x; cell < d.L1 * d.L2; cell += gridDim.y * blockDim.x) {
    const float2 g = grad_b[d.c_off + cell];
    w[d.g_off + cell] = make_double2(mu * (double)g.x, mu * (double)g.y);
  }
}

// lam = frac ||b||_inf: the thresholds t_k mu lam depend on b through its largest entry i*,
// d lam / d b = frac b_i*/|b_i*| (first index among equal maxima), and dLoss/dlam = mu * gl with
// gl = sum_k t_k dLoss/dtheta_k; one block per instance
__global__ void gy_lam_kernel(const InstDesc* __restrict__ desc, const InstParams* __restrict__ par,
                              const double2* __restrict__ b64, const double* __restrict__ grad_lam, double2* w) {
  __shared__ double sv[32];
  __shared__ int si[32];
  const InstDesc d = desc[blockIdx.x];
  if (!d.lam_is_frac) return;
  const int L = d.L1 * d.L2;
  double best = -1.0;
  int bi = 0;
  for (int cell = threadIdx.x; cell < L; cell += blockDim.x) {
    const double2 v = b64[d.g_off + cell];
    const double m = v.x * v.x + v.y * v.y;
    if (m > best) {  // cells ascend per thread: the first maximum wins
      best = m;
      bi = cell;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) {
      best = ob;
      bi = oi;
    }
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sv[wid] = best;
    si[wid] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k)
      if (sv[k] > best || (sv[k] == best && si[k] < bi)) {
        best = sv[k];
        bi = si[k];
      }
    if (best > 0.0) {
      const double2 v = b64[d.g_off + bi];
      const double r = sqrt(best);
      const double f = d.lam * par[blockIdx.x].mu * grad_lam[blockIdx.x] / r;
      double2 t = w[d.g_off + bi];
      t.x += f * v.x;
      t.y += f * v.y;
      w[d.g_off + bi] = t;
    }
  }
}

// g_y[n] = (-1)^(m1 + m2) W[m2 mod L2][m1 mod L1] for every kept element n at (m1, m2)
__global__ void gy_gather_kernel(const InstDesc* __restrict__ desc, const int* __restrict__ mask_idx,
                                 const double2* __restrict__ w, float2* grad_y) {
  const InstDesc d = desc[blockIdx.x];
  const int* mi = mask_idx + d.mask_off;
  for (int p = blockIdx.y * blockDim.x + threadIdx.x; p < d.M1 * d.M2; p += gridDim.y * blockDim.x) {
    const int n = mi[p];
    if (n < 0) continue;
    const int m1 = p % d.M1, m2 = p / d.M1;
    const double2 v = w[d.g_off + (m2 % d.L2) * d.L1 + (m1 % d.L1)];
    const double sg = ((m1 + m2) & 1) ? -1.0 : 1.0;
    grad_y[d.y_off + n] = make_float2((float)(sg * v.x), (float)(sg * v.y));
  }
}

}  // namespace

cudaError_t fill_twiddles(bccb_solver* s) {
  // the column pass stages cpb columns of length L2 twice (ping-pong)
  const int col_smem = 2 * s->max_L2 * cols_per_block(s->max_L2) * (int)sizeof(double2);
  cudaError_t e0 = cudaFuncSetAttribute(fft64_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, col_smem);
  if (e0 != cudaSuccess) return e0;
  std::vector<float2> t32(kTwiddleLen);
  std::vector<double2> t64(kTwiddleLen);
  for (int e = 0; e < kTwiddleLen; ++e) {
    const double ang = -2.0 * M_PI * (double)e / (double)kTwiddleLen;
    t64[e] = make_double2(cos(ang), sin(ang));
    t32[e] = make_float2((float)cos(ang), (float)sin(ang));
  }
  cudaError_t err = cudaMemcpy(s->d_tw32, t32.data(), kTwiddleLen * sizeof(float2), cudaMemcpyHostToDevice);
  if (err != cudaSuccess) return err;
  return cudaMemcpy(s->d_tw64, t64.data(), kTwiddleLen * sizeof(double2), cudaMemcpyHostToDevice);
}

cudaError_t fista_schedule(bccb_solver* s, int iters) {
  if (iters <= 0 || s->beta_len == iters) return cudaSuccess;
  if (iters > s->beta_cap) {
    if (s->d_beta) cudaFree(s->d_beta);
    if (s->d_beta64) cudaFree(s->d_beta64);
    s->d_beta = nullptr;
    s->d_beta64 = nullptr;
    cudaError_t err = cudaMalloc(&s->d_beta, (size_t)iters * sizeof(float));
    if (err == cudaSuccess && s->prec == 1) err = cudaMalloc(&s->d_beta64, (size_t)iters * sizeof(double));
    if (err != cudaSuccess) return err;
    s->beta_cap = iters;
  }
  if (s->algo == 0) {  // ISTA: FISTA with zero momentum
    cudaError_t err = cudaMemsetAsync(s->d_beta, 0, (size_t)iters * sizeof(float), s->stream);
    if (err == cudaSuccess && s->d_beta64)
      err = cudaMemsetAsync(s->d_beta64, 0, (size_t)iters * sizeof(double), s->stream);
    if (err != cudaSuccess) return err;
  } else {
    fista_beta_kernel<<<1, 32, 0, s->stream>>>(s->d_beta, s->d_beta64, iters);
    s->launches += 1;
  }
  s->beta_len = iters;
  return cudaGetLastError();
}

cudaError_t run_setup(bccb_solver* s, const void* y_dev) {
  const dim3 gc = grid_cells(s);
  // count grid -> d_w64, signed measurement grid s -> d_b64
  if (s->prec == 1)
    scatter_kernel<double2><<<gc, kThreads, 0, s->stream>>>(s->d_desc, s->d_mask_idx,
                                                             static_cast<const double2*>(y_dev), s->d_w64, s->d_b64);
  else
    scatter_kernel<float2><<<gc, kThreads, 0, s->stream>>>(s->d_desc, s->d_mask_idx,
                                                           static_cast<const float2*>(y_dev), s->d_w64, s->d_b64);
  s->launches += 3;  // scatter, eig_mult, lam_kappa
  // Both scattered grids are zero from row min(M2, L2) on.  Lambda depends on the mask alone:
  // an instance whose array and grid repeat an earlier instance's takes that one's (lam_src),
  // and the two transforms run only over the distinct ones (lam_sel).
  cudaError_t err;
  if ((err = fft2_64(s, s->d_w64, 1, s->scat_rows, s->d_lam_sel, s->n_lam)) != cudaSuccess)
    return err;  // first column of the Gram
  if ((err = fft2_64(s, s->d_w64, 0, 0, s->d_lam_sel, s->n_lam)) != cudaSuccess) return err;  // Lambda (eq:lambda)
  eig_mult_kernel<<<s->n, kThreads, 0, s->stream>>>(s->d_desc, s->d_lam_src, s->d_w64, s->d_b64, s->d_lam64,
                                                     s->d_par, s->d_mult, s->d_cterm, s->d_mult64, s->d_bt64,
                                                     s->d_fused, s->algo, s->rho);
  if ((err = fft2_64(s, s->d_b64, 1, s->scat_rows)) != cudaSuccess) return err;  // b = A^H y
  lam_kappa_kernel<<<s->n, kThreads, 0, s->stream>>>(s->d_desc, s->d_b64, s->d_par, s->d_fused, s->algo, s->rho);
  return cudaGetLastError();
}

template <typename V>
cudaError_t run_check_t(bccb_solver* s, const V* y_dev, const V* c_dev) {
  const dim3 gc = grid_cells(s);
  load_solution_kernel<V><<<gc, kThreads, 0, s->stream>>>(s->d_desc, c_dev, s->d_w64);
  s->launches += 4;  // load_solution, data_residual, mul_lambda, kkt_final
  // Lambda vanishes on the Fourier columns from kcols on (as q does), and the data residual
  // reads FFT2(c) only at the element positions, where Lambda > 0: the forward column pass
  // transforms only the columns below kcols, and the product Lambda . FFT2(c) zeroes the rest
  // (they hold finite row-pass values).  The inverse is the plain FFT2, whose row pass skips
  // the rows that product leaves at zero.
  fft64_rows(s, s->d_w64, 0, 0, nullptr, 0);
  fft64_cols(s, s->d_w64, 0, nullptr, 0, s->d_fused);
  data_residual_kernel<V><<<s->n, kThreads, 0, s->stream>>>(s->d_desc, s->d_mask_idx, y_dev, s->d_w64, s->d_red);
  mul_lambda_kernel<<<gc, kThreads, 0, s->stream>>>(s->d_desc, s->d_lam64, s->d_w64);
  cudaError_t err;
  if ((err = fft2_64(s, s->d_w64, 1)) != cudaSuccess) return err;
  kkt_final_kernel<V><<<s->n, kThreads, 0, s->stream>>>(s->d_desc, s->d_b64, s->d_w64, c_dev, s->d_par, s->d_red,
                                                         s->d_kkt, s->d_obj);
  return cudaGetLastError();
}

cudaError_t run_check(bccb_solver* s, const void* y_dev, const void* c_dev) {
  if (s->prec == 1)
    return run_check_t<double2>(s, static_cast<const double2*>(y_dev), static_cast<const double2*>(c_dev));
  return run_check_t<float2>(s, static_cast<const float2*>(y_dev), static_cast<const float2*>(c_dev));
}

cudaError_t unrolled_grad_y(bccb_solver* s, const float2* grad_b, const double* grad_lam, void* grad_y) {
  const dim3 gc = grid_cells(s);
  gy_load_kernel<<<gc, kThreads, 0, s->stream>>>(s->d_desc, s->d_par, grad_b, s->d_w64);
  gy_lam_kernel<<<s->n, kThreads, 0, s->stream>>>(s->d_desc, s->d_par, s->d_b64, grad_lam, s->d_w64);
  cudaError_t err;
  if ((err = fft2_64(s, s->d_w64, 0)) != cudaSuccess) return err;
  gy_gather_kernel<<<gc, kThreads, 0, s->stream>>>(s->d_desc, s->d_mask_idx, s->d_w64,
                                                    static_cast<float2*>(grad_y));
  s->launches += 3;
  return cudaGetLastError();
}

cudaError_t prepare_fp64_passes(int max_L2) {
  const int col_smem = 2 * max_L2 * cols_per_block(max_L2) * (int)sizeof(double2);
  return cudaFuncSetAttribute(fft64_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, col_smem);
}


size_t toeplitz_mu_smem(int N, int M1, int M2) {
  return (size_t)(2 * M1 - 1 + 2 * M2 - 1) * sizeof(double2) + (size_t)(2 * M1 - 1 + 2 * M2 - 1) * sizeof(float2) +
         (size_t)2 * N * sizeof(float2) + (size_t)2 * N * sizeof(int);
}

cudaError_t run_setup_toeplitz(bccb_solver* s, const void* y_dev) {
  const dim3 gc = grid_cells(s);
  cudaError_t err;
  // the mask-only part (the embedding's spectrum and mu) runs once per solver; a solve
  // being captured into a graph does not count, since its kernels have not run yet
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if ((err = cudaStreamIsCapturing(s->stream, &cs)) != cudaSuccess) return err;
  const bool mask_part = !s->toep_ready;
  if (mask_part) {
    toep_col1_kernel<<<gc, kThreads, 0, s->stream>>>(s->d_desc, s->d_mask_idx, s->gamma1, s->d_toep_h);
    toep_col2_kernel<<<gc, kThreads, 0, s->stream>>>(s->d_desc, s->d_toep_h, s->gamma2, s->d_w64);
    if ((err = fft2_64(s, s->d_w64, 0)) != cudaSuccess) return err;  // spectrum of the embedding
    toep_lam_kernel<<<gc, kThreads, 0, s->stream>>>(s->d_desc, s->d_w64, s->d_lam64);
    s->launches += 3;
  }
  if (s->prec == 1)
    toep_b1_kernel<double2><<<gc, kThreads, 0, s->stream>>>(s->d_desc, s->d_mask_idx,
                                                            static_cast<const double2*>(y_dev), s->gamma1, s->d_toep_h);
  else
    toep_b1_kernel<float2><<<gc, kThreads, 0, s->stream>>>(s->d_desc, s->d_mask_idx,
                                                           static_cast<const float2*>(y_dev), s->gamma1, s->d_toep_h);
  toep_b2_kernel<<<gc, kThreads, 0, s->stream>>>(s->d_desc, s->d_toep_h, s->gamma2, s->d_b64);
  if (mask_part) {
    int maxN = 0, maxM1 = 0, maxM2 = 0;
    for (const InstDesc& d : s->h_desc) {
      maxN = std::max(maxN, d.N);
      maxM1 = std::max(maxM1, d.M1);
      maxM2 = std::max(maxM2, d.M2);
    }
    const size_t mu_smem = toeplitz_mu_smem(maxN, maxM1, maxM2);
    if ((err = cudaFuncSetAttribute(toep_mu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mu_smem)) !=
        cudaSuccess)
      return err;
    toep_mu_kernel<<<s->n, 1024, mu_smem, s->stream>>>(s->d_desc, s->d_mask_idx, s->gamma1, s->gamma2, s->d_par);
    s->launches += 1;
    if (cs == cudaStreamCaptureStatusNone) s->toep_ready = 1;
  }
  lam_kappa_kernel<<<s->n, kThreads, 0, s->stream>>>(s->d_desc, s->d_b64, s->d_par, s->d_fused, s->algo, s->rho);
  if ((err = cudaMemcpyAsync(s->d_toep_fb, s->d_b64, sizeof(double2) * (size_t)s->total_L, cudaMemcpyDeviceToDevice,
                             s->stream)) != cudaSuccess)
    return err;
  if ((err = fft2_64(s, s->d_toep_fb, 0)) != cudaSuccess) return err;
  toep_mult_kernel<<<gc, kThreads, 0, s->stream>>>(s->d_desc, s->d_lam64, s->d_toep_fb, s->d_par, s->d_mult,
                                                   s->d_cterm, s->d_mult64, s->d_bt64, s->d_fused);
  s->launches += 4;
  return cudaGetLastError();
}

template <typename V>
cudaError_t run_check_toeplitz_t(bccb_solver* s, const V* y_dev, const V* c_int) {
  const dim3 gc = grid_cells(s);
  load_solution_kernel<V><<<gc, kThreads, 0, s->stream>>>(s->d_desc, c_int, s->d_w64);
  cudaError_t err;
  if ((err = fft2_64(s, s->d_w64, 0)) != cudaSuccess) return err;
  mul_lambda_kernel<<<gc, kThreads, 0, s->stream>>>(s->d_desc, s->d_lam64, s->d_w64);
  if ((err = fft2_64(s, s->d_w64, 1)) != cudaSuccess) return err;
  toep_kkt_kernel<V><<<s->n, kThreads, 0, s->stream>>>(s->d_desc, s->d_b64, s->d_w64, c_int, y_dev, s->d_par,
                                                        s->d_kkt, s->d_obj);
  s->launches += 3;
  return cudaGetLastError();
}

cudaError_t run_check_toeplitz(bccb_solver* s, const void* y_dev, const void* c_int) {
  if (s->prec == 1)
    return run_check_toeplitz_t<double2>(s, static_cast<const double2*>(y_dev), static_cast<const double2*>(c_int));
  return run_check_toeplitz_t<float2>(s, static_cast<const float2*>(y_dev), static_cast<const float2*>(c_int));
}

cudaError_t toeplitz_pad(bccb_solver* s, const void* c_user, void* c_int) {
  const dim3 gc = grid_cells(s);
  if (s->prec == 1)
    toep_pad_kernel<double2><<<gc, kThreads, 0, s->stream>>>(s->d_desc, static_cast<const double2*>(c_user),
                                                             static_cast<double2*>(c_int));
  else
    toep_pad_kernel<float2><<<gc, kThreads, 0, s->stream>>>(s->d_desc, static_cast<const float2*>(c_user),
                                                            static_cast<float2*>(c_int));
  s->launches += 1;
  return cudaGetLastError();
}

cudaError_t toeplitz_crop(bccb_solver* s, const void* c_int, void* c_user) {
  const dim3 gc = grid_cells(s);
  if (s->prec == 1)
    toep_crop_kernel<double2><<<gc, kThreads, 0, s->stream>>>(s->d_desc, static_cast<const double2*>(c_int),
                                                              static_cast<double2*>(c_user));
  else
    toep_crop_kernel<float2><<<gc, kThreads, 0, s->stream>>>(s->d_desc, static_cast<const float2*>(c_int),
                                                             static_cast<float2*>(c_user));
  s->launches += 1;
  return cudaGetLastError();
}

}  // namespace bccb
