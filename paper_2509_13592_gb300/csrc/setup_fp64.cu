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

#include <vector>

#include "fft_smem.cuh"
#include "solver.h"

namespace bccb {

namespace {

constexpr int kThreads = 256;

// In-place DFT of every row (length L1) of every instance's grid.
__global__ void fft64_rows_kernel(const InstDesc* __restrict__ desc, double2* base, int inv,
                                  const double2* __restrict__ tw) {
  const InstDesc d = desc[blockIdx.x];
  if ((int)blockIdx.y >= d.L2) return;
  extern __shared__ double2 sm64[];
  double2* x = sm64;
  double2* y = sm64 + d.L1;
  double2* g = base + d.g_off + (int64_t)blockIdx.y * d.L1;
  for (int e = threadIdx.x; e < d.L1; e += blockDim.x) x[e] = g[e];
  __syncthreads();
  const double2* out = inv ? fft_smem<double2, true>(x, y, d.L1, 1, tw) : fft_smem<double2, false>(x, y, d.L1, 1, tw);
  for (int e = threadIdx.x; e < d.L1; e += blockDim.x) g[e] = out[e];
}

// columns staged per block: 8, or fewer so that two L2 x cpb FP64 tiles fit in 128 KB
int cols_per_block(int max_L2) { return max_L2 <= 512 ? 8 : 4096 / max_L2; }

// In-place DFT of every column (length L2) of every instance's grid, cpb at a time.
__global__ void fft64_cols_kernel(const InstDesc* __restrict__ desc, double2* base, int inv,
                                  const double2* __restrict__ tw, int cpb) {
  const InstDesc d = desc[blockIdx.x];
  const int c0 = blockIdx.y * cpb;
  if (c0 >= d.L1) return;
  const int cnt = min(cpb, d.L1 - c0);
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
  const Y* yi = y + d.y_off;
  for (int cell = blockIdx.y * blockDim.x + threadIdx.x; cell < L; cell += gridDim.y * blockDim.x) {
    const int p1 = cell % d.L1, p2 = cell / d.L1;
    double cnt = 0.0;
    double2 acc = make_double2(0.0, 0.0);
    for (int m2 = p2; m2 < d.M2; m2 += d.L2) {
      for (int m1 = p1; m1 < d.M1; m1 += d.L1) {
        const int n = mi[m1 + m2 * d.M1];
        if (n >= 0) {
          cnt += 1.0;
          const double sgn = ((m1 + m2) & 1) ? -1.0 : 1.0;
          acc.x += sgn * (double)yi[n].x;
          acc.y += sgn * (double)yi[n].y;
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
__global__ void eig_mult_kernel(const InstDesc* __restrict__ desc, const double2* __restrict__ lam_c,
                                const double2* __restrict__ sgrid, double* lam64, InstParams* par, float* mult,
                                float2* bt, double* mult64, double2* bt64, FusedInst* fused, int algo, double rho) {
  __shared__ double sh[32];
  const InstDesc d = desc[blockIdx.x];
  const int L = d.L1 * d.L2;
  double top = 0.0;
  for (int cell = threadIdx.x; cell < L; cell += blockDim.x) top = fmax(top, lam_c[d.g_off + cell].x);
  top = block_reduce(top, MaxOp(), sh, 0.0);
  const double mu = 1.0 / top;
  const double inv_L = 1.0 / (double)L;
  double kc = 0.0;  // 1 + largest Fourier column with a nonzero multiplier or constant term
  for (int cell = threadIdx.x; cell < L; cell += blockDim.x) {
    double lv = lam_c[d.g_off + cell].x;
    if (lv < 1e-9 * top) lv = 0.0;
    lam64[d.g_off + cell] = lv;
    const double2 sv = sgrid[d.g_off + cell];
    double m, bs;
    if (algo == 2) {
      m = lv / (lv + rho) * inv_L;
      bs = 1.0 / (lv + rho);
    } else {
      m = mu * lv * inv_L;
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
    if (m != 0.0 || sv.x != 0.0 || sv.y != 0.0) kc = fmax(kc, (double)(cell % d.L1 + 1));
  }
  kc = block_reduce(kc, MaxOp(), sh, 0.0);
  if (threadIdx.x == 0) {
    par[blockIdx.x].mu = mu;
    par[blockIdx.x].lam_top = top;
    fused[blockIdx.x].kcols = (int)kc;
  }
}

// lam (absolute, or a fraction of ||A^H y||_inf) and the soft-threshold kappa
__global__ void lam_kappa_kernel(const InstDesc* __restrict__ desc, const double2* __restrict__ b64,
                                 InstParams* par, FusedInst* fused, int algo, double rho) {
  __shared__ double sh[32];
  const InstDesc d = desc[blockIdx.x];
  const int L = d.L1 * d.L2;
  double bmax = 0.0;
  for (int cell = threadIdx.x; cell < L; cell += blockDim.x) {
    const double2 bv = b64[d.g_off + cell];
    bmax = fmax(bmax, sqrt(bv.x * bv.x + bv.y * bv.y));
  }
  bmax = block_reduce(bmax, MaxOp(), sh, 0.0);
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
  double worst = 0.0, l1 = 0.0;
  for (int cell = threadIdx.x; cell < L; cell += blockDim.x) {
    const double2 bv = b64[d.g_off + cell];
    const double2 gv = gc[d.g_off + cell];
    const double rx = bv.x - gv.x * inv_L, ry = bv.y - gv.y * inv_L;
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
  }
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

cudaError_t fft2_64(bccb_solver* s, double2* grid, int inv) {
  s->launches += 2;
  const size_t smr = (size_t)2 * s->max_L1 * sizeof(double2);
  fft64_rows_kernel<<<dim3(s->n, s->max_L2), 128, smr, s->stream>>>(s->d_desc, grid, inv, s->d_tw64);
  const int cpb = cols_per_block(s->max_L2);
  const size_t smc = (size_t)2 * s->max_L2 * cpb * sizeof(double2);
  fft64_cols_kernel<<<dim3(s->n, (s->max_L1 + cpb - 1) / cpb), 128, smc, s->stream>>>(s->d_desc, grid, inv,
                                                                                        s->d_tw64, cpb);
  return cudaGetLastError();
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
  cudaError_t err;
  if ((err = fft2_64(s, s->d_w64, 1)) != cudaSuccess) return err;  // first column of the Gram
  if ((err = fft2_64(s, s->d_w64, 0)) != cudaSuccess) return err;  // Lambda (eq:lambda)
  eig_mult_kernel<<<s->n, kThreads, 0, s->stream>>>(s->d_desc, s->d_w64, s->d_b64, s->d_lam64, s->d_par,
                                                     s->d_mult, s->d_cterm, s->d_mult64, s->d_bt64, s->d_fused,
                                                     s->algo, s->rho);
  if ((err = fft2_64(s, s->d_b64, 1)) != cudaSuccess) return err;  // b = A^H y
  lam_kappa_kernel<<<s->n, kThreads, 0, s->stream>>>(s->d_desc, s->d_b64, s->d_par, s->d_fused, s->algo, s->rho);
  return cudaGetLastError();
}

template <typename V>
cudaError_t run_check_t(bccb_solver* s, const V* y_dev, const V* c_dev) {
  const dim3 gc = grid_cells(s);
  load_solution_kernel<V><<<gc, kThreads, 0, s->stream>>>(s->d_desc, c_dev, s->d_w64);
  s->launches += 4;  // load_solution, data_residual, mul_lambda, kkt_final
  cudaError_t err;
  if ((err = fft2_64(s, s->d_w64, 0)) != cudaSuccess) return err;
  data_residual_kernel<V><<<s->n, kThreads, 0, s->stream>>>(s->d_desc, s->d_mask_idx, y_dev, s->d_w64, s->d_red);
  mul_lambda_kernel<<<gc, kThreads, 0, s->stream>>>(s->d_desc, s->d_lam64, s->d_w64);
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

cudaError_t prepare_fp64_passes(int max_L2) {
  const int col_smem = 2 * max_L2 * cols_per_block(max_L2) * (int)sizeof(double2);
  return cudaFuncSetAttribute(fft64_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, col_smem);
}

}  // namespace bccb
