// C-ABI implementation: argument checks, device buffers, launch sequence.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <unordered_map>
#include <string>
#include <utility>
#include <vector>

#include "bccb.h"
#include "solver.h"

using bccb::FusedArgs;
using bccb::FusedEntry;
using bccb::FusedInst;
using bccb::InstDesc;
using bccb::InstParams;

namespace {

thread_local std::string g_create_error;

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }
// grids the fused on-chip kernel serves (FP32, sides 16 .. 256: its row and column stages are radix 16);
// every other supported grid runs on the multi-pass solver, whose transforms take any power of two
bool on_chip_grid(int prec, int L1, int L2) { return prec == BCCB_F32 && L1 >= 16 && L2 >= 16 && L1 <= 256 && L2 <= 256; }

constexpr size_t kDenseMaxBytes = size_t(64) << 30;

int fail(bccb_solver* s, int code, const std::string& msg) {
  if (s)
    s->last_error = msg;
  else
    g_create_error = msg;
  return code;
}

#define BCCB_CUDA(s, expr)                                                                   \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess) return fail((s), BCCB_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// A timing event: inside a stream capture it must become an external event-record node
// to be readable after a graph launch; outside a capture a plain record.
cudaError_t record_timing(bccb_solver* s, int i) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s->stream, &cs);
  if (e != cudaSuccess) return e;
  if (cs == cudaStreamCaptureStatusActive) return cudaEventRecordWithFlags(s->ev[i], s->stream, cudaEventRecordExternal);
  return cudaEventRecord(s->ev[i], s->stream);
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  if (count == 0) count = 1;
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

void release_streams(bccb_solver* s) {
  for (cudaStream_t st : s->class_streams) cudaStreamDestroy(st);
  for (cudaEvent_t ev : s->class_done) cudaEventDestroy(ev);
  if (s->fork) cudaEventDestroy(s->fork);
  if (s->graph) cudaGraphExecDestroy(s->graph);
  if (s->d_probe) cudaFree(s->d_probe);
  for (cudaStream_t st : s->chunk_streams)
    if (st) cudaStreamDestroy(st);
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  for (cudaEvent_t ev : s->chunk_done) cudaEventDestroy(ev);
  if (s->chunk_fork) cudaEventDestroy(s->chunk_fork);
  if (s->copies_done) cudaEventDestroy(s->copies_done);
  s->class_streams.clear();
  s->class_done.clear();
  s->fork = nullptr;
  s->chunk_streams[0] = s->chunk_streams[1] = s->copy_stream = nullptr;
  s->chunk_done.clear();
  s->chunk_fork = s->copies_done = nullptr;
  s->graph = nullptr;
  s->d_probe = nullptr;
}

void release_dense(bccb_solver* s) {
  void* ptrs[] = {s->d_gram, s->d_gram_off, s->d_dense_k, s->d_dense_s0, s->d_dense_s1, s->d_dense_x[0],
                  s->d_dense_x[1]};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  s->d_gram = nullptr;
  s->d_gram_off = nullptr;
  s->d_dense_k = s->d_dense_s0 = s->d_dense_s1 = nullptr;
  s->d_dense_x[0] = s->d_dense_x[1] = nullptr;
  s->dense_bytes = 0;
}

void release(bccb_solver* s) {
  release_streams(s);
  release_dense(s);
  void* ptrs[] = {s->d_desc,   s->d_mask_idx, s->d_lam64,   s->d_b64,     s->d_w64,     s->d_mult,
                  s->d_cterm,  s->d_par,      s->d_fused,   s->d_ids,     s->d_beta,    s->d_beta64,
                  s->d_kkt,    s->d_obj,      s->d_red,     s->d_tw32,    s->d_tw64,    s->d_y_stage,
                  s->d_c_stage, s->d_mult64,  s->d_bt64,    s->d_mp_work, s->d_mp_s0,   s->d_mp_s1,
                  s->d_cint,   s->d_c0int,    s->d_toep_h,  s->d_toep_fb, s->d_lam_sel, s->d_lam_src,
                  s->d_lo,     s->d_hi,       s->d_gradb,   s->d_gradlam};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

}  // namespace

extern "C" {

const char* bccb_status_string(int status) {
  switch (status) {
    case BCCB_OK: return "ok";
    case BCCB_ERR_INVALID_ARG: return "invalid argument";
    case BCCB_ERR_UNSUPPORTED: return "unsupported size";
    case BCCB_ERR_CUDA: return "CUDA error";
    case BCCB_ERR_KKT: return "KKT check failed";
    case BCCB_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

const char* bccb_last_error(bccb_solver_t s) { return s ? s->last_error.c_str() : g_create_error.c_str(); }

int bccb_batch_create(bccb_solver_t* out, const bccb_inst_t* insts, int n, const uint8_t* masks_host, int algo,
                      double rho, void* cuda_stream) {
  return bccb_batch_create2(out, insts, n, masks_host, algo, rho, BCCB_F32, cuda_stream);
}

}  // extern "C"

namespace {

// blk (2 per instance, nullable): the caller's block bL1, bL2 of a circulant embedding whose
// embedded size the instance table gives; uoff (nullable): the caller's solution offsets
int create_impl(bccb_solver_t* out, const bccb_inst_t* insts, int n, const uint8_t* masks_host, int algo,
                double rho, int prec, void* cuda_stream, const int* blk, const int64_t* uoff, double gamma1,
                double gamma2) {
  g_create_error.clear();
  if (!out) return fail(nullptr, BCCB_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!insts || !masks_host || n < 1) return fail(nullptr, BCCB_ERR_INVALID_ARG, "need n >= 1 instances and masks");
  if (algo != BCCB_ISTA && algo != BCCB_FISTA && algo != BCCB_ADMM)
    return fail(nullptr, BCCB_ERR_INVALID_ARG, "algo must be ISTA, FISTA or ADMM");
  if (algo == BCCB_ADMM && !(rho > 0.0)) return fail(nullptr, BCCB_ERR_INVALID_ARG, "ADMM needs rho > 0");
  if (prec != BCCB_F32 && prec != BCCB_F64) return fail(nullptr, BCCB_ERR_INVALID_ARG, "prec must be F32 or F64");

  bccb_solver* s = new bccb_solver;
  s->n = n;
  s->prec = prec;
  s->algo = algo;
  s->rho = (algo == BCCB_ADMM) ? rho : 1.0;
  s->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  cudaGetDevice(&s->device);

  std::vector<int> mask_idx;
  std::vector<FusedInst> fused(n);
  std::map<std::pair<int, int>, std::vector<int>> by_shape;
  int64_t mm_off = 0, g_off = 0;
  for (int i = 0; i < n; ++i) {
    const bccb_inst_t& q = insts[i];
    if (q.M1 < 1 || q.M2 < 1 || q.mask_off < 0 || q.y_off < 0 || q.c_off < 0 || q.reserved != 0) {
      delete s;
      return fail(nullptr, BCCB_ERR_INVALID_ARG, "instance " + std::to_string(i) + ": bad M1/M2/offsets");
    }
    if (!is_pow2(q.L1) || !is_pow2(q.L2) || q.L1 < 8 || q.L2 < 8 || q.L1 > 1024 || q.L2 > 1024) {
      delete s;
      return fail(nullptr, BCCB_ERR_UNSUPPORTED,
                  "instance " + std::to_string(i) + ": L1, L2 must be powers of two in [8, 1024]");
    }
    if (!(q.lam >= 0.0)) {
      delete s;
      return fail(nullptr, BCCB_ERR_INVALID_ARG, "instance " + std::to_string(i) + ": lam must be >= 0");
    }
    const bool on_chip = on_chip_grid(prec, q.L1, q.L2);
    if (on_chip && !bccb::fused_lookup(q.L1, q.L2, algo == BCCB_ADMM, 0, blk != nullptr)) {
      delete s;
      return fail(nullptr, BCCB_ERR_UNSUPPORTED, "no fused kernel for this grid");
    }
    InstDesc d;
    d.M1 = q.M1;
    d.M2 = q.M2;
    d.L1 = q.L1;
    d.L2 = q.L2;
    d.lam_is_frac = q.lam_is_frac ? 1 : 0;
    d.mask_off = mm_off;
    d.y_off = q.y_off;
    d.c_off = q.c_off;
    d.g_off = g_off;
    d.lam = q.lam;
    d.bL1 = blk ? blk[2 * i] : 0;
    d.bL2 = blk ? blk[2 * i + 1] : 0;
    d.u_off = uoff ? uoff[i] : q.c_off;
    int cnt = 0;
    const uint8_t* m = masks_host + q.mask_off;
    for (int pos = 0; pos < q.M1 * q.M2; ++pos) mask_idx.push_back(m[pos] ? cnt++ : -1);
    if (cnt == 0) {
      delete s;
      return fail(nullptr, BCCB_ERR_INVALID_ARG, "instance " + std::to_string(i) + ": empty mask");
    }
    d.N = cnt;
    s->h_desc.push_back(d);
    fused[i].g_off = g_off;
    fused[i].c_off = q.c_off;
    fused[i].kappa = 0.f;
    fused[i].kcols = q.L1;
    fused[i].bl1 = d.bL1;
    fused[i].bl2 = d.bL2;
    by_shape[{q.L1, q.L2}].push_back(i);
    mm_off += (int64_t)q.M1 * q.M2;
    g_off += (int64_t)q.L1 * q.L2;
    s->total_y = std::max<int64_t>(s->total_y, q.y_off + cnt);
    s->total_c = std::max<int64_t>(s->total_c, q.c_off + (int64_t)q.L1 * q.L2);
    s->total_u = std::max<int64_t>(s->total_u,
                                   blk ? d.u_off + (int64_t)d.bL1 * d.bL2 : q.c_off + (int64_t)q.L1 * q.L2);
    s->max_L1 = std::max(s->max_L1, q.L1);
    s->max_L2 = std::max(s->max_L2, q.L2);
    s->scat_rows = std::max(s->scat_rows, std::min(q.M2, q.L2));
  }
  s->total_L = g_off;

  // Lambda depends only on (M1, M2, L1, L2, mask): instances that repeat an earlier one's share it
  std::vector<int> lam_src(n), lam_sel;
  {
    std::unordered_map<std::string, int> first_of;
    for (int i = 0; i < n; ++i) {
      const bccb_inst_t& q = insts[i];
      std::string key(reinterpret_cast<const char*>(&q.M1), 4 * sizeof(int));
      const uint8_t* m = masks_host + q.mask_off;
      for (int pos = 0; pos < q.M1 * q.M2; ++pos) key.push_back(m[pos] ? '\1' : '\0');
      auto it = first_of.emplace(std::move(key), i).first;
      lam_src[i] = it->second;
      if (it->second == i) lam_sel.push_back(i);
    }
  }
  s->n_lam = (int)lam_sel.size();
  s->total_MM = mm_off;
  s->toeplitz = blk ? 1 : 0;
  s->gamma1 = gamma1;
  s->gamma2 = gamma2;

  // class-sorted instance ids; largest grids first so they start earliest
  std::vector<std::pair<int, std::pair<int, int>>> order;
  for (auto& kv : by_shape) order.push_back({-(kv.first.first * kv.first.second), kv.first});
  std::sort(order.begin(), order.end());
  std::vector<int> ids;
  bool any_mp = false;
  for (auto& o : order) {
    auto& v = by_shape[o.second];
    bccb::ShapeClass sc;
    sc.L1 = o.second.first;
    sc.L2 = o.second.second;
    sc.multipass = !on_chip_grid(prec, sc.L1, sc.L2);
    if (!sc.multipass)
      sc.entry = *bccb::fused_lookup(sc.L1, sc.L2, algo == BCCB_ADMM, 0, blk != nullptr);
    else
      memset(&sc.entry, 0, sizeof(sc.entry));
    any_mp = any_mp || sc.multipass;
    sc.first = (int)ids.size();
    sc.count = (int)v.size();
    ids.insert(ids.end(), v.begin(), v.end());
    s->classes.push_back(sc);
  }

#define CREATE_CUDA(expr)                                                                               \
  do {                                                                                                  \
    cudaError_t e_ = (expr);                                                                            \
    if (e_ != cudaSuccess) {                                                                            \
      std::string msg = std::string(#expr) + ": " + cudaGetErrorString(e_);                             \
      release(s);                                                                                       \
      delete s;                                                                                         \
      return fail(nullptr, BCCB_ERR_CUDA, msg);                                                         \
    }                                                                                                   \
  } while (0)

  CREATE_CUDA(dalloc(&s->d_desc, n));
  CREATE_CUDA(dalloc(&s->d_mask_idx, mask_idx.size()));
  CREATE_CUDA(dalloc(&s->d_lam64, s->total_L));
  CREATE_CUDA(dalloc(&s->d_b64, s->total_L));
  CREATE_CUDA(dalloc(&s->d_w64, s->total_L));
  CREATE_CUDA(dalloc(&s->d_mult, s->total_L));
  CREATE_CUDA(dalloc(&s->d_cterm, s->total_L));
  CREATE_CUDA(dalloc(&s->d_par, n));
  CREATE_CUDA(dalloc(&s->d_fused, n));
  CREATE_CUDA(dalloc(&s->d_ids, n));
  CREATE_CUDA(dalloc(&s->d_kkt, n));
  CREATE_CUDA(dalloc(&s->d_obj, n));
  CREATE_CUDA(dalloc(&s->d_red, n));
  CREATE_CUDA(dalloc(&s->d_tw32, bccb::kTwiddleLen));
  CREATE_CUDA(dalloc(&s->d_tw64, bccb::kTwiddleLen));
  if (s->toeplitz) {
    const size_t vb = prec == BCCB_F64 ? sizeof(double2) : sizeof(float2);
    CREATE_CUDA(cudaMalloc(&s->d_cint, vb * (size_t)s->total_c));
    CREATE_CUDA(cudaMalloc(&s->d_c0int, vb * (size_t)s->total_c));
    CREATE_CUDA(dalloc(&s->d_toep_h, s->total_L));
    CREATE_CUDA(dalloc(&s->d_toep_fb, s->total_L));
  }
  CREATE_CUDA(cudaMemcpy(s->d_desc, s->h_desc.data(), n * sizeof(InstDesc), cudaMemcpyHostToDevice));
  CREATE_CUDA(cudaMemcpy(s->d_mask_idx, mask_idx.data(), mask_idx.size() * sizeof(int), cudaMemcpyHostToDevice));
  CREATE_CUDA(cudaMemcpy(s->d_fused, fused.data(), n * sizeof(FusedInst), cudaMemcpyHostToDevice));
  CREATE_CUDA(cudaMemcpy(s->d_ids, ids.data(), n * sizeof(int), cudaMemcpyHostToDevice));
  s->h_ids = ids;
  if (s->n_lam < n) {
    CREATE_CUDA(dalloc(&s->d_lam_sel, s->n_lam));
    CREATE_CUDA(dalloc(&s->d_lam_src, n));
    CREATE_CUDA(cudaMemcpy(s->d_lam_sel, lam_sel.data(), s->n_lam * sizeof(int), cudaMemcpyHostToDevice));
    CREATE_CUDA(cudaMemcpy(s->d_lam_src, lam_src.data(), n * sizeof(int), cudaMemcpyHostToDevice));
  }
  if (prec == BCCB_F64) {
    CREATE_CUDA(dalloc(&s->d_mult64, s->total_L));
    CREATE_CUDA(dalloc(&s->d_bt64, s->total_L));
  }
  if (any_mp) {
    const size_t vb = prec == BCCB_F64 ? sizeof(double2) : sizeof(float2);
    CREATE_CUDA(cudaMalloc(&s->d_mp_work, vb * (size_t)s->total_L));
    CREATE_CUDA(cudaMalloc(&s->d_mp_s0, vb * (size_t)s->total_L));
    CREATE_CUDA(cudaMalloc(&s->d_mp_s1, vb * (size_t)s->total_L));
    CREATE_CUDA(bccb::prepare_multipass(s));
  }
  CREATE_CUDA(bccb::fill_twiddles(s));
  bool any_sparse = false;
  for (auto& c : s->classes)
    if (!c.multipass) {
      CREATE_CUDA(c.entry.prepare());
      any_sparse = any_sparse || (algo != BCCB_ADMM && !blk && bccb::fused_lookup(c.L1, c.L2, false, 0, false, true));
    }
  // the fused ISTA/FISTA kernel keeps the low-order parts of its state here (8 bytes per cell;
  // only cells where the state is nonzero are ever read or written, so no initialisation), and
  // its sparse-state variant the high parts of the positions its slots cannot hold (16 bytes)
  // (the FP32 multi-pass solver keeps its low parts here as well)
  if (prec == BCCB_F32 && algo != BCCB_ADMM) CREATE_CUDA(dalloc(&s->d_lo, s->total_c));
  if (any_sparse) CREATE_CUDA(dalloc(&s->d_hi, s->total_c));
  if (s->classes.size() > 1) {
    CREATE_CUDA(cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming));
    for (size_t k = 0; k < s->classes.size(); ++k) {
      cudaStream_t st;
      cudaEvent_t ev;
      CREATE_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      s->class_streams.push_back(st);
      CREATE_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      s->class_done.push_back(ev);
    }
  }
#undef CREATE_CUDA
  *out = s;
  return BCCB_OK;
}

// A chunk of the single fused shape class: positions [first, first + count) of its
// class-sorted ids, whose solutions fill the complex range [lo, hi) of c_out exactly.
struct Chunk {
  int first, count;
  int64_t lo, hi;
};

// Splits the batch for a streamed host-buffer solve.  Only a solver with one fused shape class
// (FFT method, gamma = 1/2) and at least 64 instances is split, into 8 chunks, and only when
// each chunk's instances tile a contiguous range of c_out; otherwise chunks stays empty.
bool plan_chunks(bccb_solver* s, std::vector<Chunk>& chunks) {
  chunks.clear();
  if (s->toeplitz || s->method != BCCB_FFT || s->classes.size() != 1 || s->classes[0].multipass) return false;
  const bccb::ShapeClass& c = s->classes[0];
  constexpr int kChunks = 8;
  if (c.count < 8 * kChunks) return false;
  for (int j = 0; j < kChunks; ++j) {
    Chunk k;
    k.first = (int)((int64_t)c.count * j / kChunks);
    k.count = (int)((int64_t)c.count * (j + 1) / kChunks) - k.first;
    k.lo = INT64_MAX;
    k.hi = 0;
    int64_t cells = 0;
    for (int q = 0; q < k.count; ++q) {
      const InstDesc& d = s->h_desc[s->h_ids[c.first + k.first + q]];
      const int64_t L = (int64_t)d.L1 * d.L2;
      k.lo = std::min(k.lo, d.c_off);
      k.hi = std::max(k.hi, d.c_off + L);
      cells += L;
    }
    if (k.hi - k.lo != cells) {
      chunks.clear();
      return false;
    }
    chunks.push_back(k);
  }
  if (!s->copy_stream) {
    for (cudaStream_t& st : s->chunk_streams)
      if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
    if (cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess) s->copy_stream = nullptr;
    cudaEventCreateWithFlags(&s->chunk_fork, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&s->copies_done, cudaEventDisableTiming);
  }
  while (s->chunk_done.size() < chunks.size()) {
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) break;
    s->chunk_done.push_back(ev);
  }
  if (!s->chunk_streams[0] || !s->chunk_streams[1] || !s->copy_stream || !s->chunk_fork || !s->copies_done ||
      s->chunk_done.size() < chunks.size()) {
    chunks.clear();
    return false;
  }
  return true;
}

// The whole solve (bccb_batch_solve); with host_out it also copies the solutions to that host
// buffer on the solver's stream (the caller synchronises).
int solve_impl(bccb_solver_t s, const void* y_dev, int iters, const void* c0_dev, void* c_out_dev,
               void* aux_out_dev, int check, void* host_out) {
  if (!s) return fail(nullptr, BCCB_ERR_INVALID_ARG, "solver is NULL");

  s->last_error.clear();
  if (!y_dev || !c_out_dev) return fail(s, BCCB_ERR_INVALID_ARG, "y and c_out must be device pointers");
  if (iters < 1) return fail(s, BCCB_ERR_INVALID_ARG, "iters must be >= 1");
  BCCB_CUDA(s, cudaSetDevice(s->device));
  s->launches = 0;
  if (s->timing) BCCB_CUDA(s, record_timing(s, 0));
  if (s->algo != BCCB_ADMM) BCCB_CUDA(s, bccb::fista_schedule(s, iters));
  const void* y = y_dev;
  // a Toeplitz solver iterates on embedded grids: warm start padded in, result cropped out
  const void* k_c0 = c0_dev;
  void* k_out = c_out_dev;
  if (s->toeplitz) {
    BCCB_CUDA(s, bccb::run_setup_toeplitz(s, y));
    if (c0_dev) {
      BCCB_CUDA(s, bccb::toeplitz_pad(s, c0_dev, s->d_c0int));
      k_c0 = s->d_c0int;
    }
    k_out = s->d_cint;
  } else {
    BCCB_CUDA(s, bccb::run_setup(s, y));
  }
  {
    // mu depends on the mask alone: once a setup has been queued outside a capture,
    // bccb_mu can read it after a synchronisation
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    BCCB_CUDA(s, cudaStreamIsCapturing(s->stream, &cs));
    if (cs == cudaStreamCaptureStatusNone) s->mu_ready = 1;
  }
  if (s->timing) BCCB_CUDA(s, record_timing(s, 1));
  FusedArgs a{};
  a.insts = s->d_fused;
  a.beta = (s->algo != BCCB_ADMM) ? s->d_beta : nullptr;
  a.twiddle = s->d_tw32;
  a.mult = s->d_mult;
  a.bt = s->d_cterm;
  a.c0 = reinterpret_cast<const float2*>(k_c0);
  a.c_out = reinterpret_cast<float2*>(k_out);
  a.aux_out = (s->algo == BCCB_ADMM) ? reinterpret_cast<float2*>(aux_out_dev) : nullptr;
  a.lo = s->d_lo;
  a.hi = s->d_hi;
  a.iters = iters;
  a.pad_ = 0;
  if (s->method == BCCB_DENSE) {
    BCCB_CUDA(s, bccb::run_dense(s, iters, c0_dev, c_out_dev, s->algo == BCCB_ADMM ? aux_out_dev : nullptr));
    if (s->timing) BCCB_CUDA(s, record_timing(s, 2));
    if (check) BCCB_CUDA(s, bccb::run_check(s, y, c_out_dev));
    if (s->timing) BCCB_CUDA(s, record_timing(s, 3));
    if (host_out) {
      const size_t vb = s->prec == BCCB_F64 ? sizeof(double2) : sizeof(float2);
      BCCB_CUDA(s, cudaMemcpyAsync(host_out, c_out_dev, s->total_u * vb, cudaMemcpyDeviceToHost, s->stream));
    }
    s->last_checked = check != 0;
    return BCCB_OK;
  }
  auto launch_class = [&](const bccb::ShapeClass& c, cudaStream_t st) -> cudaError_t {
    if (c.multipass)
      return bccb::run_multipass(s, s->d_ids + c.first, c.count, iters, k_c0, k_out,
                                 s->algo == BCCB_ADMM ? aux_out_dev : nullptr, st);
    a.ids = s->d_ids + c.first;
    s->launches += 1;
    return c.entry.launch(a, c.count, st);
  };
  std::vector<Chunk> chunks;
  if (host_out && plan_chunks(s, chunks)) {
    // chunks alternate between two streams, so that one chunk's last wave overlaps the next
    // one's first; their copies to the host are queued after the check (below)
    const bccb::ShapeClass& c = s->classes[0];
    BCCB_CUDA(s, cudaEventRecord(s->chunk_fork, s->stream));
    for (cudaStream_t st : s->chunk_streams) BCCB_CUDA(s, cudaStreamWaitEvent(st, s->chunk_fork, 0));
    for (size_t j = 0; j < chunks.size(); ++j) {
      cudaStream_t st = s->chunk_streams[j & 1];
      a.ids = s->d_ids + c.first + chunks[j].first;
      s->launches += 1;
      BCCB_CUDA(s, c.entry.launch(a, chunks[j].count, st));
      BCCB_CUDA(s, cudaEventRecord(s->chunk_done[j], st));
    }
    for (size_t j = chunks.size() - 2; j < chunks.size(); ++j)
      BCCB_CUDA(s, cudaStreamWaitEvent(s->stream, s->chunk_done[j], 0));
  } else if (s->classes.size() == 1) {
    BCCB_CUDA(s, launch_class(s->classes[0], s->stream));
  } else {
    // one stream per shape class, forked from and joined back to the solver's stream
    BCCB_CUDA(s, cudaEventRecord(s->fork, s->stream));
    for (size_t k = 0; k < s->classes.size(); ++k) {
      BCCB_CUDA(s, cudaStreamWaitEvent(s->class_streams[k], s->fork, 0));
      BCCB_CUDA(s, launch_class(s->classes[k], s->class_streams[k]));
      BCCB_CUDA(s, cudaEventRecord(s->class_done[k], s->class_streams[k]));
      BCCB_CUDA(s, cudaStreamWaitEvent(s->stream, s->class_done[k], 0));
    }
  }
  if (s->toeplitz) BCCB_CUDA(s, bccb::toeplitz_crop(s, s->d_cint, c_out_dev));
  if (s->timing) BCCB_CUDA(s, record_timing(s, 2));
  if (check) {
    if (s->toeplitz)
      BCCB_CUDA(s, bccb::run_check_toeplitz(s, y, s->d_cint));
    else
      BCCB_CUDA(s, bccb::run_check(s, y, c_out_dev));
  }
  if (s->timing) BCCB_CUDA(s, record_timing(s, 3));
  if (host_out) {
    const size_t vb = s->prec == BCCB_F64 ? sizeof(double2) : sizeof(float2);
    if (chunks.empty()) {
      BCCB_CUDA(s, cudaMemcpyAsync(host_out, c_out_dev, s->total_u * vb, cudaMemcpyDeviceToHost, s->stream));
    } else {
      // each chunk's copy waits only for that chunk: with pinned memory the copies overlap the
      // later chunks and the check (all GPU work is queued before the first copy, which with
      // pageable memory returns only when done)
      for (size_t j = 0; j < chunks.size(); ++j) {
        const Chunk& k = chunks[j];
        BCCB_CUDA(s, cudaStreamWaitEvent(s->copy_stream, s->chunk_done[j], 0));
        BCCB_CUDA(s, cudaMemcpyAsync(static_cast<char*>(host_out) + k.lo * vb,
                                     static_cast<const char*>(c_out_dev) + k.lo * vb, (size_t)(k.hi - k.lo) * vb,
                                     cudaMemcpyDeviceToHost, s->copy_stream));
      }
      BCCB_CUDA(s, cudaEventRecord(s->copies_done, s->copy_stream));
      BCCB_CUDA(s, cudaStreamWaitEvent(s->stream, s->copies_done, 0));
    }
  }
  s->last_checked = check != 0;
  return BCCB_OK;
}

}  // namespace

extern "C" {

int bccb_batch_create2(bccb_solver_t* out, const bccb_inst_t* insts, int n, const uint8_t* masks_host, int algo,
                       double rho, int prec, void* cuda_stream) {
  return create_impl(out, insts, n, masks_host, algo, rho, prec, cuda_stream, nullptr, nullptr, 0.5, 0.5);
}

int bccb_batch_create_gamma(bccb_solver_t* out, const bccb_inst_t* insts, int n, const uint8_t* masks_host,
                            int algo, double rho, int prec, double gamma1, double gamma2, void* cuda_stream) {
  g_create_error.clear();
  if (!out) return fail(nullptr, BCCB_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!(gamma1 > 0.0 && gamma1 <= 2.0 && gamma2 > 0.0 && gamma2 <= 2.0))
    return fail(nullptr, BCCB_ERR_INVALID_ARG, "gamma must lie in (0, 2]");
  if (gamma1 == 0.5 && gamma2 == 0.5)
    return bccb_batch_create2(out, insts, n, masks_host, algo, rho, prec, cuda_stream);
  if (!insts || !masks_host || n < 1) return fail(nullptr, BCCB_ERR_INVALID_ARG, "need n >= 1 instances and masks");
  if (algo == BCCB_ADMM)
    return fail(nullptr, BCCB_ERR_UNSUPPORTED,
                "ADMM with gamma != 1/2: (G + rho I)^-1 of a Toeplitz Gram is not a circulant-embedding product");
  std::vector<bccb_inst_t> emb(insts, insts + n);
  std::vector<int> blk(2 * (size_t)n);
  std::vector<int64_t> uoff(n);
  int64_t off = 0;
  for (int i = 0; i < n; ++i) {
    const bccb_inst_t& q = insts[i];
    if (!is_pow2(q.L1) || !is_pow2(q.L2) || q.L1 < 16 || q.L2 < 16 || q.L1 > 512 || q.L2 > 512)
      return fail(nullptr, BCCB_ERR_UNSUPPORTED,
                  "instance " + std::to_string(i) + ": with gamma != 1/2, L1 and L2 must be powers of two in [16, 512]");
    if (q.M1 < 1 || q.M2 < 1 || q.M1 > q.L1 || q.M2 > q.L2 || q.M1 > bccb::kToepMaxM || q.M2 > bccb::kToepMaxM)
      return fail(nullptr, BCCB_ERR_UNSUPPORTED,
                  "instance " + std::to_string(i) + ": with gamma != 1/2, 1 <= M_i <= L_i and M_i <= 512");
    int cnt = 0;
    for (int pos = 0; pos < q.M1 * q.M2; ++pos) cnt += masks_host[q.mask_off + pos] ? 1 : 0;
    if (cnt > bccb::kToepMaxN)
      return fail(nullptr, BCCB_ERR_UNSUPPORTED, "instance " + std::to_string(i) + ": more than 1024 elements");
    blk[2 * i] = q.L1;
    blk[2 * i + 1] = q.L2;
    uoff[i] = q.c_off;
    emb[i].L1 = 2 * q.L1;
    emb[i].L2 = 2 * q.L2;
    emb[i].c_off = off;
    off += (int64_t)emb[i].L1 * emb[i].L2;
  }
  return create_impl(out, emb.data(), n, masks_host, algo, rho, prec, cuda_stream, blk.data(), uoff.data(), gamma1,
                     gamma2);
}

int bccb_batch_solve(bccb_solver_t s, const void* y_dev, int iters, const void* c0_dev, void* c_out_dev,
                     void* aux_out_dev, int check, int* status_out) {
  if (s && status_out) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    BCCB_CUDA(s, cudaSetDevice(s->device));
    BCCB_CUDA(s, cudaStreamIsCapturing(s->stream, &cs));
    if (cs != cudaStreamCaptureStatusNone)
      return fail(s, BCCB_ERR_INVALID_ARG, "status_out needs a synchronisation, which a stream capture forbids");
  }
  const int st = solve_impl(s, y_dev, iters, c0_dev, c_out_dev, aux_out_dev, check || status_out, nullptr);
  if (st != BCCB_OK || !status_out) return st;
  return bccb_batch_status(s, status_out);
}

int bccb_batch_status(bccb_solver_t s, int* status_out) {
  if (!s) return fail(nullptr, BCCB_ERR_INVALID_ARG, "solver is NULL");
  if (!status_out) return fail(s, BCCB_ERR_INVALID_ARG, "status_out is NULL");
  if (!s->last_checked) return fail(s, BCCB_ERR_INVALID_ARG, "the last solve ran without the FP64 check");
  BCCB_CUDA(s, cudaSetDevice(s->device));
  std::vector<double> kkt(s->n);
  BCCB_CUDA(s, cudaStreamSynchronize(s->stream));
  BCCB_CUDA(s, cudaMemcpy(kkt.data(), s->d_kkt, s->n * sizeof(double), cudaMemcpyDeviceToHost));
  int failed = 0;
  for (int i = 0; i < s->n; ++i) {
    // a NaN residual fails too
    status_out[i] = kkt[i] <= s->kkt_tol ? BCCB_OK : BCCB_ERR_KKT;
    failed += status_out[i] != BCCB_OK;
  }
  if (failed)
    return fail(s, BCCB_ERR_KKT, std::to_string(failed) + " of " + std::to_string(s->n) +
                                     " instances above the KKT tolerance");
  return BCCB_OK;
}

int bccb_set_kkt_tol(bccb_solver_t s, double tol) {
  if (!s) return fail(nullptr, BCCB_ERR_INVALID_ARG, "solver is NULL");
  if (!(tol > 0.0)) return fail(s, BCCB_ERR_INVALID_ARG, "tol must be > 0");
  s->kkt_tol = tol;
  return BCCB_OK;
}

int bccb_mu(bccb_solver_t s, double* mu) {
  if (!s) return fail(nullptr, BCCB_ERR_INVALID_ARG, "solver is NULL");
  if (!mu) return fail(s, BCCB_ERR_INVALID_ARG, "mu is NULL");
  BCCB_CUDA(s, cudaSetDevice(s->device));
  if (!s->mu_ready) {
    // the setup's mask part with y = 0 (mu depends on the mask alone); a later solve
    // repeats the whole setup with its measurements
    if (s->toeplitz)
      BCCB_CUDA(s, bccb::run_setup_toeplitz(s, nullptr));
    else
      BCCB_CUDA(s, bccb::run_setup(s, nullptr));
  }
  std::vector<InstParams> p(s->n);
  BCCB_CUDA(s, cudaStreamSynchronize(s->stream));
  BCCB_CUDA(s, cudaMemcpy(p.data(), s->d_par, s->n * sizeof(InstParams), cudaMemcpyDeviceToHost));
  for (int i = 0; i < s->n; ++i) mu[i] = p[i].mu;
  s->mu_ready = 1;
  return BCCB_OK;
}


int bccb_batch_solve_host(bccb_solver_t s, const void* y_host, int iters, void* c_out_host, int check) {
  if (!s) return fail(nullptr, BCCB_ERR_INVALID_ARG, "solver is NULL");
  if (!y_host || !c_out_host) return fail(s, BCCB_ERR_INVALID_ARG, "y and c_out must be host pointers");
  BCCB_CUDA(s, cudaSetDevice(s->device));
  const size_t vb = s->prec == BCCB_F64 ? sizeof(double2) : sizeof(float2);
  if (!s->d_y_stage) BCCB_CUDA(s, dalloc(&s->d_y_stage, s->total_y * vb / sizeof(float2)));
  if (!s->d_c_stage) BCCB_CUDA(s, dalloc(&s->d_c_stage, s->total_u * vb / sizeof(float2)));
  BCCB_CUDA(s, cudaMemcpyAsync(s->d_y_stage, y_host, s->total_y * vb, cudaMemcpyHostToDevice, s->stream));
  int st = solve_impl(s, s->d_y_stage, iters, nullptr, s->d_c_stage, nullptr, check, c_out_host);
  if (st != BCCB_OK) {
    cudaStreamSynchronize(s->stream);  // no copy into the caller's buffer outlives the call
    if (s->copy_stream) cudaStreamSynchronize(s->copy_stream);
    return st;
  }
  BCCB_CUDA(s, cudaStreamSynchronize(s->stream));
  return BCCB_OK;
}

int bccb_batch_results(bccb_solver_t s, double* kkt, double* obj, double* lam, double* mu) {
  if (!s) return fail(nullptr, BCCB_ERR_INVALID_ARG, "solver is NULL");
  BCCB_CUDA(s, cudaSetDevice(s->device));
  BCCB_CUDA(s, cudaStreamSynchronize(s->stream));
  if (kkt) BCCB_CUDA(s, cudaMemcpy(kkt, s->d_kkt, s->n * sizeof(double), cudaMemcpyDeviceToHost));
  if (obj) BCCB_CUDA(s, cudaMemcpy(obj, s->d_obj, s->n * sizeof(double), cudaMemcpyDeviceToHost));
  if (lam || mu) {
    std::vector<InstParams> p(s->n);
    BCCB_CUDA(s, cudaMemcpy(p.data(), s->d_par, s->n * sizeof(InstParams), cudaMemcpyDeviceToHost));
    for (int i = 0; i < s->n; ++i) {
      if (lam) lam[i] = p[i].lam;
      if (mu) mu[i] = p[i].mu;
    }
  }
  return BCCB_OK;
}

int bccb_batch_get(bccb_solver_t s, int what, void* dst_dev) {
  if (!s) return fail(nullptr, BCCB_ERR_INVALID_ARG, "solver is NULL");
  if (!dst_dev || what < 0 || what > 3) return fail(s, BCCB_ERR_INVALID_ARG, "bad what / dst");
  if (s->toeplitz) return fail(s, BCCB_ERR_UNSUPPORTED, "the grids of a gamma != 1/2 solver are embedded 2L1 x 2L2");
  BCCB_CUDA(s, cudaSetDevice(s->device));
  const void* src = what == 0 ? (const void*)s->d_lam64
                  : what == 1 ? (const void*)s->d_b64
                  : what == 2 ? (const void*)s->d_mult
                              : (const void*)s->d_cterm;
  const size_t es = what == 0 ? 8 : what == 1 ? 16 : what == 2 ? 4 : 8;
  for (const InstDesc& d : s->h_desc) {
    BCCB_CUDA(s, cudaMemcpyAsync((char*)dst_dev + d.c_off * es, (const char*)src + d.g_off * es,
                                 (size_t)d.L1 * d.L2 * es, cudaMemcpyDeviceToDevice, s->stream));
  }
  return BCCB_OK;
}

int bccb_create(bccb_solver_t* out, int M1, int M2, const uint8_t* mask_host, int L1, int L2, int algo, double rho,
                int prec, void* cuda_stream) {
  bccb_inst_t q;
  memset(&q, 0, sizeof(q));
  q.M1 = M1;
  q.M2 = M2;
  q.L1 = L1;
  q.L2 = L2;
  q.lam = 0.0;
  return bccb_batch_create2(out, &q, 1, mask_host, algo, rho, prec, cuda_stream);
}

int bccb_solve(bccb_solver_t s, const void* y_dev, double lam, int lam_is_frac, int iters, const void* c0_dev,
               void* c_out_dev, void* aux_out_dev, double* kkt_out, double* obj_out) {
  if (!s) return fail(nullptr, BCCB_ERR_INVALID_ARG, "solver is NULL");
  if (s->n != 1) return fail(s, BCCB_ERR_INVALID_ARG, "bccb_solve needs a single-instance solver");
  if (!(lam >= 0.0)) return fail(s, BCCB_ERR_INVALID_ARG, "lam must be >= 0");
  BCCB_CUDA(s, cudaSetDevice(s->device));
  if (s->h_desc[0].lam != lam || s->h_desc[0].lam_is_frac != (lam_is_frac ? 1 : 0)) {
    s->h_desc[0].lam = lam;
    s->h_desc[0].lam_is_frac = lam_is_frac ? 1 : 0;
    BCCB_CUDA(s, cudaMemcpyAsync(s->d_desc, s->h_desc.data(), sizeof(InstDesc), cudaMemcpyHostToDevice, s->stream));
    BCCB_CUDA(s, cudaStreamSynchronize(s->stream));
  }
  const int check = (kkt_out || obj_out) ? 1 : 0;
  int st = bccb_batch_solve(s, y_dev, iters, c0_dev, c_out_dev, aux_out_dev, check, nullptr);
  if (st != BCCB_OK) return st;
  if (check) return bccb_batch_results(s, kkt_out, obj_out, nullptr, nullptr);
  return BCCB_OK;
}

int bccb_set_timing(bccb_solver_t s, int enable) {
  if (!s) return fail(nullptr, BCCB_ERR_INVALID_ARG, "solver is NULL");
  BCCB_CUDA(s, cudaSetDevice(s->device));
  if (enable && !s->ev[0])
    for (int i = 0; i < 4; ++i) BCCB_CUDA(s, cudaEventCreate(&s->ev[i]));
  s->timing = enable != 0;
  return BCCB_OK;
}

int bccb_last_timing(bccb_solver_t s, float* setup_ms, float* iterate_ms, float* check_ms, int64_t* launches) {
  if (!s) return fail(nullptr, BCCB_ERR_INVALID_ARG, "solver is NULL");
  float t[3] = {0.f, 0.f, 0.f};
  if (s->timing) {
    BCCB_CUDA(s, cudaSetDevice(s->device));
    BCCB_CUDA(s, cudaEventSynchronize(s->ev[3]));
    for (int i = 0; i < 3; ++i) BCCB_CUDA(s, cudaEventElapsedTime(&t[i], s->ev[i], s->ev[i + 1]));
  }
  if (setup_ms) *setup_ms = t[0];
  if (iterate_ms) *iterate_ms = t[1];
  if (check_ms) *check_ms = s->last_checked ? t[2] : 0.f;
  if (launches) *launches = s->launches;
  return BCCB_OK;
}

int bccb_batch_capture(bccb_solver_t s, const void* y_dev, int iters, const void* c0_dev, void* c_out_dev,
                       void* aux_out_dev, int check) {
  if (!s) return fail(nullptr, BCCB_ERR_INVALID_ARG, "solver is NULL");
  if (!y_dev || !c_out_dev || iters < 1) return fail(s, BCCB_ERR_INVALID_ARG, "bad y, c_out or iters");
  BCCB_CUDA(s, cudaSetDevice(s->device));
  if (s->stream == nullptr)
    return fail(s, BCCB_ERR_INVALID_ARG, "graph capture needs a non-default stream");
  // anything that may allocate happens before the capture
  if (s->algo != BCCB_ADMM) BCCB_CUDA(s, bccb::fista_schedule(s, iters));
  BCCB_CUDA(s, cudaStreamSynchronize(s->stream));
  if (s->graph) {
    cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  BCCB_CUDA(s, cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
  const int st = bccb_batch_solve(s, y_dev, iters, c0_dev, c_out_dev, aux_out_dev, check, nullptr);
  cudaError_t e = cudaStreamEndCapture(s->stream, &g);
  if (st != BCCB_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(s, BCCB_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&s->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(s, BCCB_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  return BCCB_OK;
}

int bccb_batch_replay(bccb_solver_t s) {
  if (!s) return fail(nullptr, BCCB_ERR_INVALID_ARG, "solver is NULL");
  if (!s->graph) return fail(s, BCCB_ERR_INVALID_ARG, "no captured solve (call bccb_batch_capture first)");
  BCCB_CUDA(s, cudaSetDevice(s->device));
  BCCB_CUDA(s, cudaGraphLaunch(s->graph, s->stream));
  return BCCB_OK;
}

int bccb_batch_tune(bccb_solver_t s, const void* y_dev, int probe_iters, const char* cache_path) {
  if (!s) return fail(nullptr, BCCB_ERR_INVALID_ARG, "solver is NULL");
  if (!y_dev || probe_iters < 1) return fail(s, BCCB_ERR_INVALID_ARG, "bad y or probe_iters");
  BCCB_CUDA(s, cudaSetDevice(s->device));
  cudaDeviceProp prop;
  BCCB_CUDA(s, cudaGetDeviceProperties(&prop, s->device));
  std::string gpu(prop.name);
  for (char& ch : gpu)
    if (ch == ' ') ch = '_';
  // cached choices: lines "gpu L1 L2 admm tile [sparse]" (a missing last field reads as 0)
  std::map<std::tuple<int, int, int>, std::pair<int, int>> cached;
  if (cache_path) {
    if (FILE* f = fopen(cache_path, "r")) {
      char line[512], name[256];
      while (fgets(line, sizeof line, f)) {
        int l1, l2, ad, tile, sparse = 0;
        const int got = sscanf(line, "%255s %d %d %d %d %d", name, &l1, &l2, &ad, &tile, &sparse);
        if (got >= 5 && gpu == name) cached[std::make_tuple(l1, l2, ad)] = {tile, got == 6 ? sparse : 0};
      }
      fclose(f);
    }
  }
  const int admm = s->algo == BCCB_ADMM ? 1 : 0;
  bool need_probe = false;
  for (auto& c : s->classes)
    if (!c.multipass && !cached.count(std::make_tuple(c.entry.L1, c.entry.L2, admm))) need_probe = true;
  FILE* out = nullptr;
  if (need_probe) {
    if (s->algo != BCCB_ADMM) BCCB_CUDA(s, bccb::fista_schedule(s, probe_iters));
    if (!s->d_probe) BCCB_CUDA(s, dalloc(&s->d_probe, s->total_c));
    if (s->toeplitz)
      BCCB_CUDA(s, bccb::run_setup_toeplitz(s, y_dev));
    else
      BCCB_CUDA(s, bccb::run_setup(s, y_dev));
    if (cache_path) out = fopen(cache_path, "a");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (need_probe) {
    BCCB_CUDA(s, cudaEventCreate(&e0));
    BCCB_CUDA(s, cudaEventCreate(&e1));
  }
  int status = BCCB_OK;
  for (auto& c : s->classes) {
    if (c.multipass) continue;
    const auto key = std::make_tuple(c.entry.L1, c.entry.L2, admm);
    auto it = cached.find(key);
    if (it != cached.end()) {
      const bool sp = it->second.second != 0 && s->d_hi != nullptr;
      if (const bccb::FusedEntry* fe =
              bccb::fused_lookup(c.entry.L1, c.entry.L2, admm != 0, it->second.first, s->toeplitz != 0, sp)) {
        c.entry = *fe;
        if (c.entry.prepare() != cudaSuccess) status = BCCB_ERR_CUDA;
        continue;
      }
    }
    FusedArgs a{};
    a.insts = s->d_fused;
    a.ids = s->d_ids + c.first;
    a.beta = (s->algo != BCCB_ADMM) ? s->d_beta : nullptr;
    a.twiddle = s->d_tw32;
    a.mult = s->d_mult;
    a.bt = s->d_cterm;
    a.c0 = nullptr;
    a.c_out = s->d_probe;
    a.aux_out = nullptr;
    a.lo = s->d_lo;
    a.hi = s->d_hi;
    a.iters = probe_iters;
    a.pad_ = 0;
    float best = 1e30f;
    bccb::FusedEntry best_e = c.entry;
    // candidates: the 8192- and 4096-element tiles with the state in shared memory, and the
    // 8192-element tile with the sparse state (where it exists and its arrays were allocated)
    const std::pair<int, int> cands[] = {{8192, 0}, {4096, 0}, {8192, 1}};
    for (const auto& cand : cands) {
      const int tile = cand.first;
      if (cand.second && !s->d_hi) continue;
      const bccb::FusedEntry* fe =
          bccb::fused_lookup(c.entry.L1, c.entry.L2, admm != 0, tile, s->toeplitz != 0, cand.second != 0);
      if (!fe || fe->prepare() != cudaSuccess) continue;
      float ms = 0.f;
      bool ok = fe->launch(a, c.count, s->stream) == cudaSuccess;  // warm-up
      ok = ok && cudaEventRecord(e0, s->stream) == cudaSuccess;
      ok = ok && fe->launch(a, c.count, s->stream) == cudaSuccess;
      ok = ok && cudaEventRecord(e1, s->stream) == cudaSuccess;
      ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
      ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
      if (ok && ms < best) {
        best = ms;
        best_e = *fe;
      }
    }
    c.entry = best_e;
    if (out)
      fprintf(out, "%s %d %d %d %d %d\n", gpu.c_str(), c.entry.L1, c.entry.L2, admm, c.entry.tile, c.entry.sparse);
  }
  if (out) fclose(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  BCCB_CUDA(s, cudaGetLastError());
  if (s->graph) {  // a captured solve would still launch the old kernels
    cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
  }
  if (status != BCCB_OK) return fail(s, status, "preparing a cached tile failed");
  return BCCB_OK;
}

int bccb_unrolled_fwd(bccb_solver_t s, const void* y_dev, int batch, int layers, const float* scale_dev,
                      const float* thresh_dev, void* c_out_dev, void* saved_dev, int check) {
  if (!s) return fail(nullptr, BCCB_ERR_INVALID_ARG, "solver is NULL");
  s->last_error.clear();
  if (batch != s->n) return fail(s, BCCB_ERR_INVALID_ARG, "batch differs from the solver's instance count");
  if (s->algo != BCCB_FISTA) return fail(s, BCCB_ERR_INVALID_ARG, "the unrolled network needs a FISTA solver");
  if (s->toeplitz) return fail(s, BCCB_ERR_UNSUPPORTED, "the unrolled network needs gamma = 1/2");
  for (const auto& c : s->classes)
    if (c.multipass) return fail(s, BCCB_ERR_UNSUPPORTED, "the unrolled network needs FP32 grids up to 256");
  if (!y_dev || !c_out_dev || !scale_dev || !thresh_dev || layers < 1)
    return fail(s, BCCB_ERR_INVALID_ARG, "bad y, c_out, scale, thresh or layers");
  BCCB_CUDA(s, cudaSetDevice(s->device));
  s->launches = 0;
  BCCB_CUDA(s, bccb::fista_schedule(s, layers));
  const void* y = y_dev;
  BCCB_CUDA(s, bccb::run_setup(s, y));
  FusedArgs a{};
  a.insts = s->d_fused;
  a.beta = s->d_beta;
  a.twiddle = s->d_tw32;
  a.mult = s->d_mult;
  a.bt = s->d_cterm;
  a.c_out = reinterpret_cast<float2*>(c_out_dev);
  a.scale = scale_dev;
  a.thresh = thresh_dev;
  a.save = reinterpret_cast<float2*>(saved_dev);
  a.save_stride = s->total_c;
  a.lo = s->d_lo;
  a.iters = layers;
  for (const auto& c : s->classes) {
    const bccb::FusedEntry* le = bccb::learned_lookup(c.L1, c.L2);
    if (!le) return fail(s, BCCB_ERR_UNSUPPORTED, "the unrolled network needs square grids (L1 = L2)");
    BCCB_CUDA(s, le->prepare());
    a.ids = s->d_ids + c.first;
    BCCB_CUDA(s, le->launch(a, c.count, s->stream));
    s->launches += 1;
  }
  if (check) BCCB_CUDA(s, bccb::run_check(s, y, c_out_dev));
  s->last_checked = check != 0;
  return BCCB_OK;
}

int bccb_unrolled_bwd(bccb_solver_t s, int batch, int layers, const float* scale_dev, const float* thresh_dev,
                      const void* saved_dev, const void* grad_c_dev, void* grad_y_dev, double* grad_scale_dev,
                      double* grad_thresh_dev) {
  if (!s) return fail(nullptr, BCCB_ERR_INVALID_ARG, "solver is NULL");
  s->last_error.clear();
  if (batch != s->n) return fail(s, BCCB_ERR_INVALID_ARG, "batch differs from the solver's instance count");
  if (s->algo != BCCB_FISTA) return fail(s, BCCB_ERR_INVALID_ARG, "the unrolled network needs a FISTA solver");
  if (s->toeplitz) return fail(s, BCCB_ERR_UNSUPPORTED, "the unrolled network needs gamma = 1/2");
  if (!scale_dev || !thresh_dev || !saved_dev || !grad_c_dev || !grad_scale_dev || !grad_thresh_dev || layers < 1)
    return fail(s, BCCB_ERR_INVALID_ARG, "bad pointer or layers");
  if (s->beta_len < layers) return fail(s, BCCB_ERR_INVALID_ARG, "run bccb_unrolled_fwd with these layers first");
  BCCB_CUDA(s, cudaSetDevice(s->device));
  bccb::AdjArgs a{};
  a.insts = s->d_fused;
  a.beta = s->d_beta;
  a.twiddle = s->d_tw32;
  a.mult = s->d_mult;
  a.scale = scale_dev;
  a.thresh = thresh_dev;
  a.save = reinterpret_cast<const float2*>(saved_dev);
  a.save_stride = s->total_c;
  a.grad_c = reinterpret_cast<const float2*>(grad_c_dev);
  a.grad_scale = grad_scale_dev;
  a.grad_thresh = grad_thresh_dev;
  a.layers = layers;
  if (grad_y_dev) {
    if (!s->d_gradb) BCCB_CUDA(s, dalloc(&s->d_gradb, s->total_c));
    if (!s->d_gradlam) BCCB_CUDA(s, dalloc(&s->d_gradlam, s->n));
    BCCB_CUDA(s, cudaMemsetAsync(s->d_gradlam, 0, sizeof(double) * s->n, s->stream));
    a.grad_b = s->d_gradb;
    a.grad_lam = s->d_gradlam;
  }
  for (const auto& c : s->classes) {
    const bccb::AdjointEntry* ae = bccb::adjoint_lookup(c.entry.L1, c.entry.L2);
    if (!ae) return fail(s, BCCB_ERR_UNSUPPORTED, "no adjoint kernel for this grid");
    BCCB_CUDA(s, ae->prepare());
    a.ids = s->d_ids + c.first;
    BCCB_CUDA(s, ae->launch(a, c.count, s->stream));
  }
  if (grad_y_dev) BCCB_CUDA(s, bccb::unrolled_grad_y(s, s->d_gradb, s->d_gradlam, grad_y_dev));
  return BCCB_OK;
}

int bccb_batch_set_method(bccb_solver_t s, int method) {
  if (!s) return fail(nullptr, BCCB_ERR_INVALID_ARG, "solver is NULL");
  if (method != BCCB_FFT && method != BCCB_DENSE) return fail(s, BCCB_ERR_INVALID_ARG, "unknown method");
  BCCB_CUDA(s, cudaSetDevice(s->device));
  if (method == s->method) return BCCB_OK;
  if (method == BCCB_FFT) {
    BCCB_CUDA(s, cudaStreamSynchronize(s->stream));
    release_dense(s);
    s->method = BCCB_FFT;
    return BCCB_OK;
  }
  if (s->prec != BCCB_F32) return fail(s, BCCB_ERR_UNSUPPORTED, "the dense method runs in complex64 only");
  if (s->toeplitz) return fail(s, BCCB_ERR_UNSUPPORTED, "the dense method builds the BCCB Gram (gamma = 1/2) only");
  size_t bytes = 0;
  for (const InstDesc& d : s->h_desc) {
    if (s->algo == BCCB_ADMM && (d.M1 > d.L1 || d.M2 > d.L2))
      return fail(s, BCCB_ERR_UNSUPPORTED, "dense ADMM needs M_i <= L_i (no fold: D D^H = L I)");
    bytes += sizeof(float2) * (size_t)d.L1 * d.L2 * (size_t)d.L1 * d.L2;
  }
  if (bytes > kDenseMaxBytes) return fail(s, BCCB_ERR_UNSUPPORTED, "dense Gram matrices exceed 64 GiB");
  const cudaError_t e = bccb::dense_prepare(s);
  if (e != cudaSuccess) {
    release_dense(s);
    return fail(s, BCCB_ERR_CUDA, std::string("dense_prepare: ") + cudaGetErrorString(e));
  }
  s->method = BCCB_DENSE;
  return BCCB_OK;
}

int bccb_batch_peaks(bccb_solver_t s, const void* c_dev, int K, double rel_thresh, int32_t* idx_dev,
                     double* mag_dev, double* harm_dev, double* ang_dev, int32_t* count_dev) {
  if (!s) return fail(nullptr, BCCB_ERR_INVALID_ARG, "solver is NULL");
  if (!c_dev || !idx_dev || !mag_dev || !harm_dev || !ang_dev) return fail(s, BCCB_ERR_INVALID_ARG, "NULL buffer");
  if (K < 1 || K > bccb::kMaxPeakK) return fail(s, BCCB_ERR_INVALID_ARG, "K outside [1, 1024]");
  if (!(rel_thresh >= 0.0 && rel_thresh <= 1.0)) return fail(s, BCCB_ERR_INVALID_ARG, "rel_thresh outside [0, 1]");
  BCCB_CUDA(s, cudaSetDevice(s->device));
  BCCB_CUDA(s, bccb::run_peaks(s, c_dev, K, rel_thresh, idx_dev, mag_dev, harm_dev, ang_dev, count_dev));
  return BCCB_OK;
}

int bccb_batch_tile(bccb_solver_t s, int L1, int L2, int* tile) {
  return bccb_batch_variant(s, L1, L2, tile, nullptr);
}

int bccb_batch_variant(bccb_solver_t s, int L1, int L2, int* tile, int* sparse_state) {
  if (!s || !tile) return fail(s, BCCB_ERR_INVALID_ARG, "NULL argument");
  *tile = 0;
  if (sparse_state) *sparse_state = 0;
  for (const auto& c : s->classes)
    if (c.L1 == L1 && c.L2 == L2) {
      *tile = c.multipass ? 0 : c.entry.tile;
      if (sparse_state) *sparse_state = c.multipass ? 0 : c.entry.sparse;
    }
  return BCCB_OK;
}

int bccb_batch_size(bccb_solver_t s, int* n) {
  if (!s || !n) return fail(s, BCCB_ERR_INVALID_ARG, "NULL argument");
  *n = s->n;
  return BCCB_OK;
}

int bccb_instance_shape(bccb_solver_t s, int i, int* L1, int* L2, int* N) {
  if (!s || i < 0 || i >= s->n) return fail(s, BCCB_ERR_INVALID_ARG, "bad solver or index");
  if (L1) *L1 = s->h_desc[i].L1;
  if (L2) *L2 = s->h_desc[i].L2;
  if (N) *N = s->h_desc[i].N;
  return BCCB_OK;
}

int bccb_destroy(bccb_solver_t s) {
  if (!s) return BCCB_OK;
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->stream);
  for (int i = 0; i < 4; ++i)
    if (s->ev[i]) cudaEventDestroy(s->ev[i]);
  release(s);
  delete s;
  return BCCB_OK;
}

}  // extern "C"
