// Private solver state shared by the C-ABI implementation and the setup/check kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "adjoint.cuh"

namespace bccb {

// One problem instance (device-visible).
struct InstDesc {
  int M1, M2, L1, L2, N;
  int lam_is_frac;   // 1: lam is a fraction of ||A^H y||_inf
  int64_t mask_off;  // into mask_idx (M1*M2 entries: y index or -1)
  int64_t y_off;     // complex elements into the measurement buffer
  int64_t c_off;     // complex elements into the solution buffer
  int64_t g_off;     // elements into the per-grid arenas (L1*L2 each)
  double lam;        // absolute lam, or fraction (see lam_is_frac)
  // element spacing gamma != 1/2 (Toeplitz Gram): L1 x L2 above is the 2 bL1 x 2 bL2
  // circulant embedding and bL1 x bL2 the caller's grid; 0 for the BCCB case
  int bL1 = 0, bL2 = 0;
  int64_t u_off = 0;  // the caller's offset of this instance's solution (= c_off for BCCB)
};

// Per-instance scalars produced on the device by the setup kernels.
struct InstParams {
  double mu;      // 1 / max Lambda
  double lam;     // absolute LASSO weight used
  double lmax;    // ||A^H y||_inf
  double lam_top; // max Lambda
};

struct ShapeClass {
  FusedEntry entry;  // fused kernel (multipass == 0)
  int multipass;     // 1: the multi-pass solver (grids above 256 or the FP64 path)
  int L1, L2;
  int first;  // offset into the class-sorted id list
  int count;
};

}  // namespace bccb

struct bccb_solver {
  int n = 0;
  int algo = 1;
  int prec = 0;  // 0: complex64 path, 1: complex128 (FP64 check path)
  double rho = 1.0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int64_t total_L = 0;
  int64_t total_MM = 0;
  int64_t total_y = 0;
  int64_t total_c = 0;
  int max_L1 = 0, max_L2 = 0;
  int scat_rows = 0;              // max over instances of min(M2, L2): rows of a scattered grid that may be nonzero
  int n_lam = 0;                  // instances with distinct (array, grid): Lambda transforms per setup
  int* d_lam_sel = nullptr;       // their ids (null when every instance is distinct)
  int* d_lam_src = nullptr;       // per instance, the id whose Lambda it shares (null likewise)
  std::vector<bccb::InstDesc> h_desc;
  std::vector<bccb::ShapeClass> classes;

  bccb::InstDesc* d_desc = nullptr;
  int* d_mask_idx = nullptr;
  double* d_lam64 = nullptr;    // Lambda (real), per grid cell
  double2* d_b64 = nullptr;     // b = A^H y (FP64)
  double2* d_w64 = nullptr;     // FP64 FFT workspace
  float* d_mult = nullptr;      // FP32 Fourier multiplier (includes 1/(L1 L2))
  float2* d_cterm = nullptr;    // FP32 Fourier-domain constant term Bt
  uint2* d_lo = nullptr;        // fused ISTA/FISTA: low-order parts of the state, packed like c
  float4* d_hi = nullptr;       // sparse-state variant: high parts {c, z} beyond its slots, packed like c
  float2* d_gradb = nullptr;    // unrolled backward with dLoss/dy: sum_k a_k g_{u_k}, packed like c
  double* d_gradlam = nullptr;  // and per instance sum_k t_k dLoss/dtheta_k
  bccb::InstParams* d_par = nullptr;
  bccb::FusedInst* d_fused = nullptr;
  int* d_ids = nullptr;
  float* d_beta = nullptr;
  double* d_beta64 = nullptr;
  int beta_cap = 0;
  int beta_len = -1;
  double* d_kkt = nullptr;
  double* d_obj = nullptr;
  double* d_red = nullptr;     // per-instance partial sums
  float2* d_tw32 = nullptr;
  double2* d_tw64 = nullptr;
  // host staging for the host-buffer entry point
  float2* d_y_stage = nullptr;
  float2* d_c_stage = nullptr;
  std::string last_error;
  // profiling
  bool timing = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  int64_t launches = 0;  // kernels launched by the last solve
  bool last_checked = false;
  // per-class streams forked from `stream` (classes run concurrently)
  std::vector<cudaStream_t> class_streams;
  std::vector<cudaEvent_t> class_done;
  cudaEvent_t fork = nullptr;
  // host-buffer solve of one fused shape class: chunks of instances on two streams, each
  // chunk's results copied to the host on copy_stream as soon as the chunk ends
  std::vector<int> h_ids;                      // class-sorted instance ids (as d_ids)
  cudaStream_t chunk_streams[2] = {nullptr, nullptr};
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> chunk_done;
  cudaEvent_t chunk_fork = nullptr;
  cudaEvent_t copies_done = nullptr;
  // captured solve (bccb_batch_capture / bccb_batch_replay)
  cudaGraphExec_t graph = nullptr;
  // probe output for the autotuner
  float2* d_probe = nullptr;
  // multi-pass solver: FP64 multiplier and constant term, state grids (complex64 or complex128)
  double* d_mult64 = nullptr;
  double2* d_bt64 = nullptr;
  void* d_mp_work = nullptr;
  void* d_mp_s0 = nullptr;
  void* d_mp_s1 = nullptr;
  // element spacings (Section II-A); toeplitz = 1 when either differs from 1/2: the
  // kernels then run on the 2 L1 x 2 L2 circulant embedding (toeplitz.cu)
  int toeplitz = 0;
  double gamma1 = 0.5, gamma2 = 0.5;
  int64_t total_u = 0;            // length of the caller's packed solution
  void* d_cint = nullptr;         // embedded solution grids (Toeplitz)
  void* d_c0int = nullptr;        // embedded warm start (Toeplitz)
  double2* d_toep_h = nullptr;    // FP64 scratch of the Toeplitz setup
  double2* d_toep_fb = nullptr;   // FP64 FFT2 of the zero-padded b (Toeplitz)
  int toep_ready = 0;             // the embedding's spectrum (d_lam64) and mu are in place
  int mu_ready = 0;               // d_par[i].mu holds 1/max Lambda (it depends on the mask alone)
  double kkt_tol = 1e-2;          // status BCCB_ERR_KKT above this relative KKT residual
  // iteration engine: 0 = FFT (fused / multi-pass), 1 = dense L x L Gram (dense.cu)
  int method = 0;
  float2* d_gram = nullptr;       // per instance L x L complex64, row-major
  int64_t* d_gram_off = nullptr;  // element offset of each instance's block
  float2* d_dense_k = nullptr;    // constant term per cell
  float2* d_dense_s0 = nullptr;   // c (ISTA/FISTA) or z (ADMM)
  float2* d_dense_s1 = nullptr;   // v (ADMM)
  float2* d_dense_x[2] = {nullptr, nullptr};  // double-buffered product input
  size_t dense_bytes = 0;
};

namespace bccb {
// setup_fp64.cu
// each returns the CUDA status and adds its kernel launches to s->launches
cudaError_t run_setup(bccb_solver* s, const void* y_dev);
cudaError_t run_check(bccb_solver* s, const void* y_dev, const void* c_dev);
cudaError_t fill_twiddles(bccb_solver* s);
cudaError_t fista_schedule(bccb_solver* s, int iters);
// dLoss/dy of the unrolled network from the adjoint's b-gradient (sum_k a_k g_{u_k}, packed like c)
// and per-instance sum_k t_k dLoss/dtheta_k; uses the last setup's mu, b and Lambda workspace
cudaError_t unrolled_grad_y(bccb_solver* s, const float2* grad_b, const double* grad_lam, void* grad_y);
// shared-memory opt-in of the FP64 column pass for grids with up to max_L2 rows
cudaError_t prepare_fp64_passes(int max_L2);
// multipass.cu: all iterations of one multi-pass class (ids[0..count)) on `stream`
cudaError_t prepare_multipass(bccb_solver* s);
cudaError_t run_multipass(bccb_solver* s, const int* ids, int count, int iters, const void* c0, void* c_out,
                          void* aux, cudaStream_t stream);
// fused_inst.cu / fused_dispatch.cu: tile 0 = the default 8192-element tile
// block: the variant for the circulant embedding of a Toeplitz Gram (ISTA/FISTA, sides >= 32)
// sparse: the ISTA/FISTA variant with the state outside shared memory (rows of 256, tile 8192)
const FusedEntry* fused_lookup(int L1, int L2, bool admm, int tile = 0, bool block = false, bool sparse = false);
const AdjointEntry* adjoint_lookup(int L1, int L2);
// the unrolled network's forward kernel (square grids L1 = L2, FISTA, default tile)
const FusedEntry* learned_lookup(int L1, int L2);
// dense.cu: build the stored Gram matrices (synchronises) and run the dense iterations
cudaError_t dense_prepare(bccb_solver* s);
cudaError_t run_dense(bccb_solver* s, int iters, const void* c0, void* c_out, void* aux);
// toeplitz.cu: setup and check on the circulant embedding, and the pad / crop between the
// caller's packing and the embedded grids
constexpr int kToepMaxN = 1024;  // elements per instance (the N x N power iteration runs in one CTA)
constexpr int kToepMaxM = 512;   // M_i
size_t toeplitz_mu_smem(int N, int M1, int M2);
cudaError_t run_setup_toeplitz(bccb_solver* s, const void* y_dev);
cudaError_t run_check_toeplitz(bccb_solver* s, const void* y_dev, const void* c_int);
cudaError_t toeplitz_pad(bccb_solver* s, const void* c_user, void* c_int);
cudaError_t toeplitz_crop(bccb_solver* s, const void* c_int, void* c_user);
// peaks.cu: top-K peaks of every instance of c and their harmonics and angles
constexpr int kMaxPeakK = 1024;
cudaError_t run_peaks(bccb_solver* s, const void* c_dev, int K, double rel_thresh, int* idx, double* mag,
                      double* harm, double* ang, int* count);
}  // namespace bccb
