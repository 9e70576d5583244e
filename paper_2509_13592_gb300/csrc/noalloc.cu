// bccb_solve_noalloc: one instance, the same kernels as bccb_solve, with every
// device buffer carved from a fixed array compiled into the library instead of
// cudaMalloc'd memory.  See include/bccb.h for who needs this and the limits.
#include <math.h>
#include <mutex>

#include "bccb.h"
#include "solver.h"

namespace {

constexpr int kMaxGrid = 256 * 256;  // L1 * L2
constexpr int kMaxUra = 16384;       // M1 * M2
constexpr int kMaxIters = 8192;
constexpr size_t kAlign = 256;
constexpr size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// byte offsets of each region inside the array
constexpr size_t kOffDesc = 0;
constexpr size_t kOffFused = kOffDesc + up(sizeof(bccb::InstDesc));
constexpr size_t kOffIds = kOffFused + up(sizeof(bccb::FusedInst));
constexpr size_t kOffPar = kOffIds + up(sizeof(int));
constexpr size_t kOffMaskIdx = kOffPar + up(sizeof(bccb::InstParams));
constexpr size_t kOffLam64 = kOffMaskIdx + up(sizeof(int) * kMaxUra);
constexpr size_t kOffB64 = kOffLam64 + up(sizeof(double) * kMaxGrid);
constexpr size_t kOffW64 = kOffB64 + up(sizeof(double2) * kMaxGrid);
constexpr size_t kOffMult = kOffW64 + up(sizeof(double2) * kMaxGrid);
constexpr size_t kOffBt = kOffMult + up(sizeof(float) * kMaxGrid);
constexpr size_t kOffBeta = kOffBt + up(sizeof(float2) * kMaxGrid);
constexpr size_t kOffTw32 = kOffBeta + up(sizeof(float) * kMaxIters);
constexpr size_t kOffTw64 = kOffTw32 + up(sizeof(float2) * bccb::kTwiddleLen);
constexpr size_t kOffLo = kOffTw64 + up(sizeof(double2) * bccb::kTwiddleLen);
constexpr size_t kScratchBytes = kOffLo + up(sizeof(uint2) * kMaxGrid);

// The working memory.  In host code this name is only a stand-in for the device
// array: host code must use the address cudaGetSymbolAddress returns.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_base[kMaxDevices] = {};

// y index of each URA position (-1 if the element is not kept): exclusive count
// of the kept elements in ascending m1 + m2*M1, as the rows of Psi are ordered.
// The total goes to desc->N, so the record matches the one bccb_create builds.
__global__ void mask_index_kernel(const uint8_t* __restrict__ mask, int n, int* __restrict__ idx,
                                  bccb::InstDesc* desc) {
  __shared__ int warp_tot[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int keep = (i < n && mask[i]) ? 1 : 0;
    int v = keep;  // inclusive scan within the warp
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) >= o) v += t;
    }
    if ((threadIdx.x & 31) == 31) warp_tot[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
      int w = (threadIdx.x < (blockDim.x >> 5)) ? warp_tot[threadIdx.x] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, w, o);
        if (threadIdx.x >= o) w += t;
      }
      warp_tot[threadIdx.x] = w;  // inclusive over warps
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    const int before = carry + (warp ? warp_tot[warp - 1] : 0) + v - keep;
    if (i < n) idx[i] = keep ? before : -1;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + keep;
    __syncthreads();
  }
  if (threadIdx.x == 0) desc->N = carry;
}

// the per-call records (passed by value, written on the device)
__global__ void records_kernel(bccb::InstDesc d, bccb::InstDesc* desc, bccb::FusedInst* fused, int* ids) {
  desc[0] = d;
  bccb::FusedInst f;
  f.g_off = 0;
  f.c_off = 0;
  f.kappa = 0.f;
  f.kcols = d.L1;
  fused[0] = f;
  ids[0] = 0;
}

// Find the array on the current device and, the first time it is seen at that address,
// upload the twiddle tables.  The address is looked up on every call (a lookup allocates
// nothing): after cudaDeviceReset the module is loaded again, possibly elsewhere and
// without the tables, and the set-up then runs again.
int device_setup(int dev, unsigned char** base, const char** err) {
  std::lock_guard<std::mutex> lock(g_mu);
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess) {
    *err = cudaGetErrorString(e);
    return BCCB_ERR_CUDA;
  }
  if (g_base[dev] == p) {
    *base = g_base[dev];
    return BCCB_OK;
  }
  static float2 t32[bccb::kTwiddleLen];
  static double2 t64[bccb::kTwiddleLen];
  for (int k = 0; k < bccb::kTwiddleLen; ++k) {
    const double ang = -2.0 * M_PI * (double)k / (double)bccb::kTwiddleLen;
    t64[k] = make_double2(cos(ang), sin(ang));
    t32[k] = make_float2((float)cos(ang), (float)sin(ang));
  }
  unsigned char* b = static_cast<unsigned char*>(p);
  if ((e = cudaMemcpy(b + kOffTw32, t32, sizeof(t32), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(b + kOffTw64, t64, sizeof(t64), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = bccb::prepare_fp64_passes(256)) != cudaSuccess) {
    *err = cudaGetErrorString(e);
    return BCCB_ERR_CUDA;
  }
  g_base[dev] = b;
  *base = b;
  return BCCB_OK;
}

// The status code is the whole error report: BCCB_ERR_UNSUPPORTED for sizes above
// the limits in include/bccb.h, BCCB_ERR_INVALID_ARG for bad arguments,
// BCCB_ERR_CUDA for a failed CUDA call.
int reject(int code, const char* /*why*/) { return code; }

bool pow2_in(int x, int lo, int hi) { return x >= lo && x <= hi && (x & (x - 1)) == 0; }

}  // namespace

extern "C" int bccb_solve_noalloc(int M1, int M2, const uint8_t* mask_dev, int L1, int L2, int algo, double rho,
                                  const void* y_dev, double lam, int lam_is_frac, int iters, void* c_out_dev,
                                  void* cuda_stream) {
  if (!mask_dev || !y_dev || !c_out_dev) return reject(BCCB_ERR_INVALID_ARG, "mask, y and c_out must be device pointers");
  if (algo != BCCB_ISTA && algo != BCCB_FISTA && algo != BCCB_ADMM) return reject(BCCB_ERR_INVALID_ARG, "bad algo");
  if (algo == BCCB_ADMM && !(rho > 0.0)) return reject(BCCB_ERR_INVALID_ARG, "ADMM needs rho > 0");
  if (!(lam >= 0.0) || M1 < 1 || M2 < 1 || iters < 1) return reject(BCCB_ERR_INVALID_ARG, "bad lam, M1, M2 or iters");
  if (!pow2_in(L1, 16, 256) || !pow2_in(L2, 16, 256))
    return reject(BCCB_ERR_UNSUPPORTED, "bccb_solve_noalloc: L1, L2 must be powers of two in [16, 256]");
  if ((long)M1 * M2 > kMaxUra) return reject(BCCB_ERR_UNSUPPORTED, "bccb_solve_noalloc: M1*M2 above 16384");
  if (iters > kMaxIters) return reject(BCCB_ERR_UNSUPPORTED, "bccb_solve_noalloc: iters above 8192");
  const bccb::FusedEntry* fe = bccb::fused_lookup(L1, L2, algo == BCCB_ADMM);
  if (!fe) return reject(BCCB_ERR_UNSUPPORTED, "no fused kernel for this grid");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return reject(BCCB_ERR_CUDA, "cudaGetDevice failed");
  unsigned char* base = nullptr;
  const char* err = "";
  if (int st = device_setup(dev, &base, &err)) return reject(st, err);
  (void)err;

  // a solver view whose buffers all point into the array (no allocation)
  bccb_solver s;
  s.n = 1;
  s.algo = algo;
  s.rho = (algo == BCCB_ADMM) ? rho : 1.0;
  s.stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  s.device = dev;
  s.max_L1 = L1;
  s.max_L2 = L2;
  s.scat_rows = std::min(M2, L2);
  s.d_desc = reinterpret_cast<bccb::InstDesc*>(base + kOffDesc);
  s.d_fused = reinterpret_cast<bccb::FusedInst*>(base + kOffFused);
  s.d_ids = reinterpret_cast<int*>(base + kOffIds);
  s.d_par = reinterpret_cast<bccb::InstParams*>(base + kOffPar);
  s.d_mask_idx = reinterpret_cast<int*>(base + kOffMaskIdx);
  s.d_lam64 = reinterpret_cast<double*>(base + kOffLam64);
  s.d_b64 = reinterpret_cast<double2*>(base + kOffB64);
  s.d_w64 = reinterpret_cast<double2*>(base + kOffW64);
  s.d_mult = reinterpret_cast<float*>(base + kOffMult);
  s.d_cterm = reinterpret_cast<float2*>(base + kOffBt);
  s.d_beta = reinterpret_cast<float*>(base + kOffBeta);
  s.beta_cap = kMaxIters;  // fista_schedule then never allocates
  s.d_tw32 = reinterpret_cast<float2*>(base + kOffTw32);
  s.d_tw64 = reinterpret_cast<double2*>(base + kOffTw64);

  bccb::InstDesc d;
  d.M1 = M1;
  d.M2 = M2;
  d.L1 = L1;
  d.L2 = L2;
  d.N = 0;  // mask_index_kernel writes the kept-element count into the device record
  d.lam_is_frac = lam_is_frac ? 1 : 0;
  d.mask_off = 0;
  d.y_off = 0;
  d.c_off = 0;
  d.g_off = 0;
  d.lam = lam;

  records_kernel<<<1, 1, 0, s.stream>>>(d, s.d_desc, s.d_fused, s.d_ids);
  mask_index_kernel<<<1, 1024, 0, s.stream>>>(mask_dev, M1 * M2, s.d_mask_idx, s.d_desc);
  if ((e = cudaGetLastError()) != cudaSuccess) return reject(BCCB_ERR_CUDA, cudaGetErrorString(e));
  if (algo == BCCB_FISTA && (e = bccb::fista_schedule(&s, iters)) != cudaSuccess)
    return reject(BCCB_ERR_CUDA, cudaGetErrorString(e));
  if ((e = bccb::run_setup(&s, reinterpret_cast<const float2*>(y_dev))) != cudaSuccess)
    return reject(BCCB_ERR_CUDA, cudaGetErrorString(e));
  if ((e = fe->prepare()) != cudaSuccess) return reject(BCCB_ERR_CUDA, cudaGetErrorString(e));
  bccb::FusedArgs a{};
  a.insts = s.d_fused;
  a.ids = s.d_ids;
  a.beta = (algo == BCCB_FISTA) ? s.d_beta : nullptr;
  a.twiddle = s.d_tw32;
  a.mult = s.d_mult;
  a.bt = s.d_cterm;
  a.c0 = nullptr;
  a.c_out = reinterpret_cast<float2*>(c_out_dev);
  a.aux_out = nullptr;
  a.lo = reinterpret_cast<uint2*>(base + kOffLo);
  a.iters = iters;
  a.pad_ = 0;
  if ((e = fe->launch(a, 1, s.stream)) != cudaSuccess) return reject(BCCB_ERR_CUDA, cudaGetErrorString(e));
  return BCCB_OK;
}
