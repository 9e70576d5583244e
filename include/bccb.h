/*
 * bccb.h -- C ABI of the GB300 BCCB sparse-recovery solver.
 *
 * Solves the single-snapshot 2D harmonic-recovery LASSO of arXiv 2509.13592,
 *     minimise_c  1/2 ||y - D_s c||_2^2 + lam ||c||_1       (eq:lasso_objective, Section II-A)
 * with ISTA (eq:ista), FISTA (eq:fista) or ADMM (eq:admm).  The sparse array's
 * elements sit on a half-wavelength grid and the harmonic grids are uniform
 * (eq:uniform_grid, gamma = 1/2), so D_s^H D_s is block-circulant with circulant
 * blocks (eq:bccb_sum) and every Gram product is IFFT2(Lambda . FFT2(x)) on the
 * L1 x L2 grid (eq:Rc, Section III-B).  All iterations run in hand-written
 * sm_103a kernels; nothing falls back to the CPU.
 *
 * Notation: lam is the paper's tau (the LASSO weight), N the number of kept array
 * elements (the paper's M), L1 x L2 the harmonic grid.
 *
 * Layouts
 *   mask   uint8, M1*M2 entries, mask[m1 + m2*M1] != 0 keeps URA element (m1, m2)
 *          (the subsampling matrix Psi, Section II-A).  Host memory.
 *   y      complex64 (interleaved float re, im), N entries: the kept elements in
 *          ascending order of m1 + m2*M1 (the rows of Psi).
 *   c      complex64, L1*L2 entries stored as an L2 x L1 row-major grid: entry
 *          l1 + l2*L1 is the amplitude at harmonics (f_{1,l1}, f_{2,l2}) with
 *          f_{i,l} = -1/2 + l/L_i (Section II-A: column l1 + l2 L1 of D).
 * Supported grids: L1, L2 powers of two in [8, 1024]; M1, M2 >= 1 (masks wider
 * than the grid fold, which the BCCB structure allows).  FP32 grids with both sides
 * in [16, 256] run on chip (one thread-block cluster per instance); other grids (a
 * side of 8, or above 256) and the FP64 path run as two passes per iteration over
 * L2-resident global memory.
 *
 * Conventions
 *   * Every call returns a status (BCCB_OK = 0).  No exception crosses the ABI and
 *     no kernel traps; bccb_last_error() gives a message for the last failure.
 *   * Device pointers are caller-owned and must stay valid until the stream work
 *     finishes; the solver owns its internal buffers (Lambda, mu*b or d,
 *     multipliers, FP64 workspace).
 *   * All device work is queued on the solver's stream (cudaStream_t passed as
 *     void*, NULL = legacy default stream).  Calls that return host values
 *     (bccb_batch_results, bccb_solve's kkt/objective, *_host) synchronise that
 *     stream.
 *   * Not thread-safe per solver; distinct solvers may be used from distinct threads.
 */
#ifndef BCCB_H
#define BCCB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bccb_solver* bccb_solver_t;

/* Algorithms (Section II-B). */
enum { BCCB_ISTA = 0, BCCB_FISTA = 1, BCCB_ADMM = 2 };

/* Arithmetic of the iterations: complex64 (y, c complex64) or complex128 (y, c complex128). */
enum { BCCB_F32 = 0, BCCB_F64 = 1 };

/* Status codes. */
enum {
  BCCB_OK = 0,
  BCCB_ERR_INVALID_ARG = 1, /* null pointer, bad size, empty mask, rho <= 0, ... */
  BCCB_ERR_UNSUPPORTED = 2, /* grid size outside the supported set */
  BCCB_ERR_CUDA = 3,        /* a CUDA call failed; see bccb_last_error() */
  BCCB_ERR_KKT = 4,         /* result returned, but its FP64 KKT check failed (bccb_batch_solve) */
  BCCB_ERR_TIMEOUT = 5      /* reserved for a bounded device wait that expired; no kernel of this library
                               waits on a flag or a peer (its waits are CTA and cluster barriers), so
                               no call returns it */
};

/* One instance of a batch.  Offsets let the caller pack many instances into one
 * mask buffer (bytes), one y buffer and one c buffer (complex elements). */
typedef struct {
  int32_t M1, M2;      /* URA size (Section II-A) */
  int32_t L1, L2;      /* harmonic grid lengths (powers of two, 16..1024) */
  int64_t mask_off;    /* byte offset of this instance's M1*M2 mask in masks_host */
  int64_t y_off;       /* complex64 offset of this instance's N measurements */
  int64_t c_off;       /* complex64 offset of this instance's L1*L2 solution */
  double lam;          /* LASSO weight, or a fraction of ||A^H y||_inf if lam_is_frac */
  int32_t lam_is_frac; /* 0: lam is absolute; 1: lam := lam * ||A^H y||_inf per solve */
  int32_t reserved;    /* must be 0 */
} bccb_inst_t;

/* Create a solver for a batch of n independent instances that share one algorithm
 * (and, for ADMM, one rho > 0; eq:admm).  Copies the masks and instance table to
 * the device; allocates all internal buffers.  Does not launch the solve.  Instances
 * with the same M1, M2, L1, L2 and mask (a fixed array observing many snapshots)
 * share one Lambda transform in every setup; results are as if each had its own.
 * Errors: INVALID_ARG (n < 1, null pointers, empty mask, bad algo/rho,
 * reserved != 0), UNSUPPORTED (grid size), CUDA. */
int bccb_batch_create(bccb_solver_t* out, const bccb_inst_t* insts, int n, const uint8_t* masks_host,
                      int algo, double rho, void* cuda_stream);
/* As bccb_batch_create, with the arithmetic: BCCB_F32 (complex64 y and c) or
 * BCCB_F64 (complex128 y and c in every call on this solver; the whole solve in
 * FP64, the check path the FP32 results are compared with). */
int bccb_batch_create2(bccb_solver_t* out, const bccb_inst_t* insts, int n, const uint8_t* masks_host,
                       int algo, double rho, int prec, void* cuda_stream);

/* bccb_batch_create2 for element spacings gamma1, gamma2 (in wavelengths, Section II-A)
 * other than 1/2.  The harmonic grids are f_{i,l} = -gamma_i + l 2 gamma_i / L_i
 * (eq:uniform_grid); the Gram A^H A is then block Toeplitz with Toeplitz blocks
 * (Section III-A), and every product with it is the L1 x L2 block of a product with
 * the 2L1 x 2L2 circulant embedding, so the same FFT2 iterations run on the embedded
 * grid with the unknown held at 0 outside the block.  mu = 1/lambda_max(A A^H) comes
 * from a power iteration (FP32, finished by an FP64 Rayleigh quotient), b = A^H y from
 * its definition in FP64.  The caller's packing is unchanged (L1 x L2 per instance).
 * Limits: ISTA or FISTA (ADMM's (G + rho I)^{-1} is not a product with the embedding:
 * UNSUPPORTED); L_i powers of two in [16, 512]; 1 <= M_i <= L_i, M_i <= 512; at most
 * 1024 elements per instance; gamma_i in (0, 2].  gamma1 = gamma2 = 1/2 is exactly
 * bccb_batch_create2.  bccb_batch_get, the dense method and the unrolled network are
 * UNSUPPORTED on such a solver. */
int bccb_batch_create_gamma(bccb_solver_t* out, const bccb_inst_t* insts, int n, const uint8_t* masks_host,
                            int algo, double rho, int prec, double gamma1, double gamma2, void* cuda_stream);

/* Run the whole hot path for every instance on the solver's stream:
 *   setup (FP64): Lambda = FFT2 of the Gram's first column (eq:lambda),
 *                 mu = 1/max Lambda (eq:ista), b = A^H y, lam, and the FP32
 *                 Fourier-domain multiplier q and constant term Bt: mu Lambda/L and
 *                 mu FFT2(b)/L (ISTA/FISTA), Lambda/(Lambda+rho)/L and
 *                 FFT2(b)/(Lambda+rho)/L (ADMM, the "precomputed" term of eq:admm);
 *   iterations (FP32): `iters` fused ISTA/FISTA/ADMM iterations, each one FFT2,
 *                 multiply, IFFT2 and the pointwise update (eq:ista/fista/admm, eq:Rc);
 *   check (FP64, if check != 0): relative KKT residual and objective per instance.
 * y_dev: packed complex64 measurements (device).  c0_dev: nullable warm start
 * (complex64, same packing as c_out_dev; ADMM: z^(0)).  c_out_dev: packed complex64
 * results: c^(T) for ISTA/FISTA, z^(T) for ADMM.  aux_out_dev: nullable; ADMM
 * writes c^(T) there.  Asynchronous unless status_out is given.
 * status_out: nullable host array of n ints.  When given, the FP64 check runs whatever
 * `check` says, the call synchronises the stream and writes, per instance, BCCB_OK or
 * BCCB_ERR_KKT: the relative KKT residual of the LASSO optimality conditions
 * (Section II-A; see bccb_batch_results) exceeds the solver's tolerance
 * (bccb_set_kkt_tol, default 1e-2), or is not a number.  The call then returns
 * BCCB_ERR_KKT if any instance failed; every result is still written.  status_out is
 * refused (INVALID_ARG) inside a stream capture, which cannot synchronise.
 * Errors: INVALID_ARG (null y/c_out, iters < 1), KKT, CUDA. */
int bccb_batch_solve(bccb_solver_t s, const void* y_dev, int iters, const void* c0_dev, void* c_out_dev,
                     void* aux_out_dev, int check, int* status_out);

/* Tolerance on the relative KKT residual behind status BCCB_ERR_KKT (tol > 0). */
int bccb_set_kkt_tol(bccb_solver_t s, double tol);

/* Per-instance status of the last solve that ran the FP64 check (bccb_batch_solve with
 * check or status_out, bccb_unrolled_fwd with check), as bccb_batch_solve's status_out:
 * BCCB_OK or BCCB_ERR_KKT per instance in the host array status_out[0..n-1]; returns
 * BCCB_ERR_KKT if any failed, INVALID_ARG if the last solve ran no check.  Synchronises. */
int bccb_batch_status(bccb_solver_t s, int* status_out);

/* Step size mu = 1/sigma_max(A)^2 of each instance (eq:ista), written to the host array
 * mu[0..n-1]: 1/max Lambda for half-wavelength spacing (eq:lambda), the power-iteration
 * value for gamma != 1/2.  mu depends on the mask alone; if no solve has been queued yet,
 * the call runs the setup on the mask (with y = 0) first.  Synchronises. */
int bccb_mu(bccb_solver_t s, double* mu);

/* bccb_batch_solve with HOST buffers: copies y to the device, solves, copies c
 * back; synchronises.  y_host / c_out_host use the same packing as above.  A batch
 * of one on-chip shape class (FP32, gamma = 1/2, FFT method) with at least 64
 * instances is solved as 8 launches of consecutive instances; each launch's
 * solutions are copied back while the later ones run, when they fill a contiguous
 * range of c_out (with pageable c_out_host the copies still follow all GPU work).
 * On an error no copy into c_out_host is still in flight when the call returns. */
int bccb_batch_solve_host(bccb_solver_t s, const void* y_host, int iters, void* c_out_host, int check);

/* Per-instance scalars of the last solve, copied to host arrays of length n (each
 * nullable): relative KKT residual max_i viol_i / lam (viol = (|r_i| - lam)_+ off
 * the support, |r_i - lam c_i/|c_i|| on it, r = A^H(y - A c)), objective
 * 1/2||y - A c||^2 + lam||c||_1, the lam used and mu.  Synchronises. */
int bccb_batch_results(bccb_solver_t s, double* kkt, double* obj, double* lam, double* mu);

/* Copy an internal per-instance grid of the last solve (device to device), packed
 * like c_out (instance i at its c_off).  what: 0 = Lambda (float64, real);
 * 1 = b = A^H y (complex128); 2 = the FP32 Fourier multiplier q (float32); 3 = the
 * FP32 Fourier-domain constant term Bt (complex64); 2 and 3 are in frequency order
 * [p2][p1] and include 1/(L1 L2).  Asynchronous. */
int bccb_batch_get(bccb_solver_t s, int what, void* dst_dev);

/* Single-instance convenience: a batch of one (c_off = y_off = 0) with the arithmetic
 * prec (BCCB_F32 or BCCB_F64, as bccb_batch_create2). */
int bccb_create(bccb_solver_t* out, int M1, int M2, const uint8_t* mask_host, int L1, int L2, int algo,
                double rho, int prec, void* cuda_stream);
/* Solve one instance with LASSO weight lam (absolute, or a fraction of
 * ||A^H y||_inf if lam_is_frac).  kkt_out / obj_out nullable; when either is
 * given the FP64 check runs and the call synchronises. */
int bccb_solve(bccb_solver_t s, const void* y_dev, double lam, int lam_is_frac, int iters, const void* c0_dev,
               void* c_out_dev, void* aux_out_dev, double* kkt_out, double* obj_out);

/* Capture the whole of bccb_batch_solve (same arguments) into a CUDA graph on the
 * solver's stream, which must not be the legacy default stream; bccb_batch_replay
 * launches it again (same buffers, same iteration count).  A later capture or
 * bccb_batch_tune replaces it.  The multi-class launch is a fork/join over one
 * stream per (L1, L2) class, so the classes of a ragged batch run concurrently. */
int bccb_batch_capture(bccb_solver_t s, const void* y_dev, int iters, const void* c0_dev, void* c_out_dev,
                       void* aux_out_dev, int check);
int bccb_batch_replay(bccb_solver_t s);

/* Autotuner: for every (L1, L2) class of the batch, time each fused-kernel variant
 * (8192 grid elements per CTA, or 4096 = twice the CTAs per cluster, two CTAs per
 * SM, both with the state in shared memory; for ISTA/FISTA on rows of 256 also 8192
 * elements per CTA with the state held only at its nonzero positions, two CTAs per
 * SM) for probe_iters iterations on the class's own instances, after one setup with
 * y_dev, and keep the fastest.  cache_path (nullable): a text file of lines
 * "gpu_name L1 L2 admm tile sparse" (a line without the last field means sparse = 0);
 * classes found there for this GPU are not measured, new choices are appended.
 * Synchronises.  bccb_batch_tile reports the tile and bccb_batch_variant the tile
 * and whether the state is sparse (0 for a multi-pass class). */
int bccb_batch_tune(bccb_solver_t s, const void* y_dev, int probe_iters, const char* cache_path);
int bccb_batch_tile(bccb_solver_t s, int L1, int L2, int* tile);
int bccb_batch_variant(bccb_solver_t s, int L1, int L2, int* tile, int* sparse_state);

/* Unrolled FISTA network (a learned extension of eq:fista; the paper has no learned
 * part).  On a FISTA solver, layer k = 0..layers-1 runs
 *     u_k = z_k - a_k mu (G z_k - b),  c_k = S_{t_k mu lam}(u_k),  z_{k+1} = c_k + beta_k (c_k - c_{k-1})
 * with z_0 = c_{-1} = 0, FISTA's beta_k, and per-layer multipliers a_k = scale_dev[k],
 * t_k = thresh_dev[k] (device float arrays; a = t = 1 is plain FISTA with `layers`
 * iterations).  batch is the number of snapshots and must equal the solver's instance
 * count (INVALID_ARG otherwise).  bccb_unrolled_fwd runs the setup and the layers, writes c_{K-1} to
 * c_out_dev, and, if saved_dev is not NULL, stores each layer's input z_k and
 * mu (G z_k - b) there (layers * 2 * (packed solution length) complex64 values) for
 * the backward pass; check != 0 runs the FP64 KKT check on c_{K-1}.
 * bccb_unrolled_bwd takes grad_c_dev = dLoss/dc_{K-1} (complex64, packed like c, as
 * dLoss/dRe + j dLoss/dIm) and ADDS dLoss/da_k and dLoss/dt_k, summed over the batch,
 * to the device float64 arrays grad_scale_dev / grad_thresh_dev (length layers).  If
 * grad_y_dev is not NULL it also WRITES dLoss/dy there (complex64, packed like y, same
 * convention): y enters every layer through b = A^H y, and, for instances whose lam is a
 * fraction of ||A^H y||_inf, every threshold through that maximum (the derivative is taken at
 * the first cell that attains it).  It needs the same solver, layers, multipliers and saved
 * buffer as the forward call, with no other solve on the solver in between.
 * Square grids (L1 = L2, up to 256) only; BCCB_ERR_UNSUPPORTED otherwise. */
int bccb_unrolled_fwd(bccb_solver_t s, const void* y_dev, int batch, int layers, const float* scale_dev,
                      const float* thresh_dev, void* c_out_dev, void* saved_dev, int check);
int bccb_unrolled_bwd(bccb_solver_t s, int batch, int layers, const float* scale_dev, const float* thresh_dev,
                      const void* saved_dev, const void* grad_c_dev, void* grad_y_dev, double* grad_scale_dev,
                      double* grad_thresh_dev);

/* Phase timing of bccb_batch_solve, for profiling.  bccb_set_timing(s, 1) makes
 * every later solve record CUDA events on the solver's stream around its three
 * phases; bccb_last_timing synchronises and returns the last solve's setup,
 * iteration and check durations in milliseconds (0 when timing is off) and the
 * number of kernels that solve launched (always counted). */
int bccb_set_timing(bccb_solver_t s, int enable);
int bccb_last_timing(bccb_solver_t s, float* setup_ms, float* iterate_ms, float* check_ms, int64_t* launches);

/* Iteration engine of a solver. */
enum { BCCB_FFT = 0, BCCB_DENSE = 1 };

/* Select how the iterations apply the Gram product.  BCCB_FFT (the default): the 2D
 * FFT identity of eq:Rc (fused cluster kernel or multi-pass).  BCCB_DENSE: the
 * paper's "regular" implementation, whose dominant term is the O(L^2) product with an
 * L x L matrix (eq:ista, eq:fista, eq:admm): the Gram G = D_s^H D_s of every instance
 * is built once from its definition (FP64, stored complex64, L^2 * 8 bytes per
 * instance) and each iteration is one dense matrix-vector product plus the pointwise
 * update, with the identity part applied exactly:
 *   ISTA/FISTA  u = x - mu (G x) + mu b;
 *   ADMM        c = w - (G w)/(rho + L) + b/(rho + L), w = z - v, from the Woodbury
 *               form of (G + rho I)^{-1} with D_s D_s^H = L I.
 * Setup (Lambda, mu, b, lam) and the FP64 check are those of the FFT engine, so the
 * two engines differ only in the iterations.  Requirements: a BCCB_F32 solver; for
 * ADMM every M_i <= L_i; at most 64 GiB of matrices in total; else UNSUPPORTED.
 * Switching to BCCB_DENSE builds the matrices and synchronises; switching back frees
 * them. */
int bccb_batch_set_method(bccb_solver_t s, int method);

/* Harmonic and angle estimates from a solution (Section II-A): the support of c
 * marks harmonic pairs (f1, f2) = (-g1 + l1 2 g1/L1, -g2 + l2 2 g2/L2), and each pair
 * gives the angles through f1 = g1 cos(phi) sin(theta), f2 = g2 sin(phi) sin(theta),
 * with the solver's element spacings g1, g2 (1/2 unless created by
 * bccb_batch_create_gamma).  The paper gives no peak-picking rule; this one:
 *   m(p) = |c(p)|^2 in c's precision (x*x and y*y rounded, then their sum);
 *   p is a peak when m(p) > 0, m(p) >= rel_thresh^2 * max m, and for each of its 8
 *   cyclic neighbours q: m(p) > m(q), or m(p) == m(q) and p < q (index l1 + l2 L1);
 *   peaks rank by m descending, then index ascending; the first K are returned.
 * c_dev: a solution packed like c_out (complex64, or complex128 for a BCCB_F64
 * solver).  Outputs (device, instance i at [i*K, (i+1)*K), caller-owned):
 *   idx_dev  int32   l1 + l2 L1, -1 past the instance's peak count;
 *   mag_dev  float64 |c| = sqrt(m) in c's precision (0 past the count);
 *   harm_dev float64 pairs (f1, f2);
 *   ang_dev  float64 pairs (phi, theta), phi = atan2(f2/g2, f1/g1) in [-pi, pi],
 *            theta = asin(sqrt((f1/g1)^2 + (f2/g2)^2)); NaN where that sum exceeds 1
 *            (outside the visible region) and past the count;
 *   count_dev int32 per instance, nullable: the number of peaks before the cut to K.
 * K in [1, 1024], rel_thresh in [0, 1], else INVALID_ARG.  Asynchronous. */
int bccb_batch_peaks(bccb_solver_t s, const void* c_dev, int K, double rel_thresh, int32_t* idx_dev,
                     double* mag_dev, double* harm_dev, double* ang_dev, int32_t* count_dev);

/* Number of instances, and the (L1, L2, N) of instance i. */
int bccb_batch_size(bccb_solver_t s, int* n);
int bccb_instance_shape(bccb_solver_t s, int i, int* L1, int* L2, int* N);

int bccb_destroy(bccb_solver_t s);

/* Solve one instance without allocating any device memory.
 *
 * For callers that cannot call cudaMalloc: code running where the device
 * allocator is off limits (a host process whose memory budget is fixed up
 * front, a plugin inside another runtime that owns all allocations, or a path
 * that must not risk an allocation failure or the implicit synchronisation an
 * allocation can bring).  The paper has no counterpart; this is a deployment
 * convenience over the same kernels as bccb_solve.
 *
 * All working memory (about 3.9 MB) is one fixed array compiled into the
 * library, which every GPU that loads the library holds until the process
 * exits.  The first call on each device looks that array up and uploads the
 * twiddle tables (make that first call before any stream capture); later calls
 * do no set-up.  Every call on a device reuses the same array: calls whose work
 * overlaps on the GPU (two streams, or two threads) race and corrupt each other,
 * so serialise them.  Each call rewrites every part of the array it reads, so
 * nothing left by an earlier call leaks into a result.
 *
 * Arguments as for bccb_create + bccb_solve, except that the mask is a DEVICE
 * pointer (uint8, M1*M2) and there is no KKT check.  The mask cannot be inspected
 * on the host, so an all-zero mask is not refused: with no element kept, A has no
 * rows and c_out receives c = 0, the minimiser of the data-free problem (mu is
 * taken as 0 instead of 1/max Lambda = 1/0).  The device address of the array is
 * looked up on every call, so the set-up runs again after cudaDeviceReset.
 * Limits: L1, L2 powers of
 * two in [16, 256] (L1*L2 <= 65536), M1*M2 <= 16384, 1 <= iters <= 8192; larger
 * sizes return BCCB_ERR_UNSUPPORTED before any work is queued.  Asynchronous on
 * cuda_stream; y_dev and c_out_dev as for bccb_solve (c_out receives c^(T), or
 * z^(T) for ADMM). */
int bccb_solve_noalloc(int M1, int M2, const uint8_t* mask_dev, int L1, int L2, int algo, double rho,
                       const void* y_dev, double lam, int lam_is_frac, int iters, void* c_out_dev,
                       void* cuda_stream);
/* Measurement helper (no counterpart in the paper): the device's FP32 fused multiply-add
 * rate in TFLOP/s, from event-timed launches on cuda_stream of a kernel whose threads run 16
 * independent multiply-add chains for `iters` steps each, at full occupancy on every SM (best
 * of three after a warm-up).  paired = 0: scalar fma.rn.f32; paired = 1: fma.rn.f32x2 (two
 * lanes per instruction, the form the fused solver's butterflies use for their sums).  It
 * confirms the FP32 peak (SMs x 128 lanes x 2 flop x clock) that the fused solver's roofline
 * fraction is reported against.  Synchronises the stream; allocates nothing.  iters of about
 * 20000 take a few milliseconds on a GB300.  Errors: INVALID_ARG (null tflops_out, iters < 1),
 * CUDA. */
int bccb_fp32_fma_rate(int paired, int iters, void* cuda_stream, double* tflops_out);
const char* bccb_status_string(int status);
/* Message for the solver's last failure ("" if none); s may be NULL for create errors. */
const char* bccb_last_error(bccb_solver_t s);

#ifdef __cplusplus
}
#endif

#endif /* BCCB_H */
