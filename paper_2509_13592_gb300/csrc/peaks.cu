// Peak extraction on |c| and the harmonic-to-angle map (Section II-A).
//
// The support of the recovered c marks harmonic pairs (f1, f2) on the uniform grids
// f_{i,l} = -gamma_i + l 2 gamma_i / L_i (eq:uniform_grid; gamma_i = 1/2 for half-wavelength
// spacing), and each pair gives the angles through f1 = gamma1 cos(phi) sin(theta),
// f2 = gamma2 sin(phi) sin(theta).
// The paper states the map but no peak-picking rule; the one used:
//   m(p) = |c(p)|^2 in c's precision (products and sum rounded separately);
//   p is a peak when m(p) > 0, m(p) >= rel^2 max m and, for each of its 8 cyclic
//   neighbours q, m(p) > m(q) or (m(p) == m(q) and p < q);
//   peaks rank by m descending, then linear index ascending; the first K are kept.
//
// One CTA per instance.  The K-th largest key (the bit pattern of m, which orders
// like m for m >= 0) is found exactly by a most-significant-byte-first radix select
// over repeated scans of the grid, the keys above it are gathered in any order, the
// ties at it in index order (a block scan per chunk), and the <= K selected entries
// are sorted by a bitonic network in shared memory.
#include <stdint.h>

#include "solver.h"

namespace bccb {
namespace {

constexpr int kPeakThreads = 1024;

template <typename V>
struct PeakT;
template <>
struct PeakT<float2> {
  using M = float;
  using Key = uint32_t;
  static __device__ __forceinline__ M sq(float2 v) { return __fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y)); }
  static __device__ __forceinline__ Key bits(M m) { return __float_as_uint(m); }
  static __device__ __forceinline__ M value(Key k) { return __uint_as_float(k); }
  static __device__ __forceinline__ double root(M m) { return (double)sqrtf(m); }
};
template <>
struct PeakT<double2> {
  using M = double;
  using Key = unsigned long long;
  static __device__ __forceinline__ M sq(double2 v) {
    return __dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y));
  }
  static __device__ __forceinline__ Key bits(M m) { return (Key)__double_as_longlong(m); }
  static __device__ __forceinline__ M value(Key k) { return __longlong_as_double((long long)k); }
  static __device__ __forceinline__ double root(M m) { return sqrt(m); }
};

template <typename T>
__device__ T warp_max(T v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ unsigned warp_sum(unsigned v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// exclusive prefix sum of f over the block (in thread order) and the block total
__device__ void block_scan(unsigned f, unsigned& excl, unsigned& total, unsigned* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned incl = f;
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned o = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += o;
  }
  __syncthreads();
  if (lane == 31) sh[w] = incl;
  __syncthreads();
  if (w == 0) {
    unsigned v = lane < nw ? sh[lane] : 0u, s = v;
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned o = __shfl_up_sync(0xffffffffu, s, d);
      if (lane >= d) s += o;
    }
    if (lane < nw) sh[lane] = s - v;  // exclusive warp offsets
    if (lane == 31) sh[32] = s;
  }
  __syncthreads();
  excl = sh[w] + incl - f;
  total = sh[32];
  __syncthreads();
}

template <typename V>
__global__ void __launch_bounds__(kPeakThreads) peaks_kernel(const InstDesc* __restrict__ desc, const V* __restrict__ c,
                                                             int K, double rel2, double g1, double g2, int* idx_out,
                                                             double* mag_out, double* harm_out, double* ang_out,
                                                             int* count_out) {
  using P = PeakT<V>;
  using M = typename P::M;
  using Key = typename P::Key;
  __shared__ unsigned hist[256];
  __shared__ Key skey[kMaxPeakK];
  __shared__ int sidx[kMaxPeakK];
  __shared__ unsigned shs[33];
  __shared__ M shm[32];
  __shared__ Key s_prefix;
  __shared__ unsigned s_need, s_ngt;

  const InstDesc d = desc[blockIdx.x];
  // the caller's grid (the block of a circulant embedding when bL1 > 0)
  const int L1 = d.bL1 ? d.bL1 : d.L1, L2 = d.bL1 ? d.bL2 : d.L2, L = L1 * L2;
  const V* ci = c + d.u_off;
  const int tid = threadIdx.x, nt = blockDim.x;

  // ---- max m and the threshold
  M mx = (M)0;
  for (int p = tid; p < L; p += nt) mx = max(mx, P::sq(ci[p]));
  mx = warp_max(mx);
  if ((tid & 31) == 0) shm[tid >> 5] = mx;
  __syncthreads();
  if (tid < 32) {
    M v = tid < (nt >> 5) ? shm[tid] : (M)0;
    v = warp_max(v);
    if (tid == 0) shm[0] = v;
  }
  __syncthreads();
  const double thr = rel2 * (double)shm[0];

  // key of cell p: the bits of m(p) if p is a peak, else 0
  auto key_at = [&](int p) -> Key {
    const M m = P::sq(ci[p]);
    if (!(m > (M)0) || (double)m < thr) return (Key)0;
    const int l1 = p % L1, l2 = p / L1;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int r = (l2 + dy + L2) % L2;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        if (dy == 0 && dx == 0) continue;
        const int q = r * L1 + (l1 + dx + L1) % L1;
        const M mq = P::sq(ci[q]);
        if (mq > m || (mq == m && q < p)) return (Key)0;
      }
    }
    return P::bits(m);
  };

  // ---- number of peaks
  unsigned cnt = 0;
  for (int p = tid; p < L; p += nt) cnt += key_at(p) != (Key)0;
  cnt = warp_sum(cnt);
  __syncthreads();
  if ((tid & 31) == 0) shs[tid >> 5] = cnt;
  __syncthreads();
  if (tid < 32) {
    unsigned v = tid < (nt >> 5) ? shs[tid] : 0u;
    v = warp_sum(v);
    if (tid == 0) shs[32] = v;
  }
  __syncthreads();
  cnt = shs[32];
  __syncthreads();

  // ---- the K-th largest key kth and how many of the keys equal to it are taken
  Key kth = (Key)0;
  unsigned need = 0;
  if (cnt > (unsigned)K) {
    Key prefix = (Key)0, kmask = (Key)0;
    need = (unsigned)K;
    for (int shift = 8 * (int)sizeof(Key) - 8; shift >= 0; shift -= 8) {
      for (int i = tid; i < 256; i += nt) hist[i] = 0u;
      __syncthreads();
      for (int p = tid; p < L; p += nt) {
        const Key k = key_at(p);
        if (k != (Key)0 && (k & kmask) == prefix) atomicAdd(&hist[(unsigned)(k >> shift) & 255u], 1u);
      }
      __syncthreads();
      if (tid == 0) {
        unsigned acc = 0;
        for (int b = 255; b >= 0; --b) {
          if (acc + hist[b] >= need) {
            s_prefix = prefix | ((Key)b << shift);
            s_need = need - acc;
            break;
          }
          acc += hist[b];
        }
      }
      __syncthreads();
      prefix = s_prefix;
      need = s_need;
      kmask |= (Key)255 << shift;
      __syncthreads();
    }
    kth = prefix;
  }

  // ---- gather: every key above kth (any order), then `need` ties at kth in index order
  if (tid == 0) s_ngt = 0u;
  __syncthreads();
  for (int p = tid; p < L; p += nt) {
    const Key k = key_at(p);
    if (k > kth) {
      const unsigned pos = atomicAdd(&s_ngt, 1u);
      skey[pos] = k;
      sidx[pos] = p;
    }
  }
  __syncthreads();
  const unsigned ngt = s_ngt;
  unsigned taken = 0;
  for (int base = 0; base < L && taken < need; base += nt) {
    const int p = base + tid;
    const unsigned f = (p < L && key_at(p) == kth) ? 1u : 0u;
    unsigned excl, tot;
    block_scan(f, excl, tot, shs);
    if (f && taken + excl < need) {
      skey[ngt + taken + excl] = kth;
      sidx[ngt + taken + excl] = p;
    }
    taken += tot;
  }
  const int nsel = (int)min(cnt, (unsigned)K);

  // ---- sort the selection: key descending, then index ascending
  int np2 = 1;
  while (np2 < nsel) np2 <<= 1;
  for (int i = nsel + tid; i < np2; i += nt) {
    skey[i] = (Key)0;
    sidx[i] = 0x7fffffff;
  }
  __syncthreads();
  for (int size = 2; size <= np2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = tid; i < np2; i += nt) {
        const int j = i ^ stride;
        if (j > i) {
          const Key ki = skey[i], kj = skey[j];
          const int ii = sidx[i], ij = sidx[j];
          const bool j_first = kj > ki || (kj == ki && ij < ii);
          const bool i_first = ki > kj || (ki == kj && ii < ij);
          if (((i & size) == 0) ? j_first : i_first) {
            skey[i] = kj;
            skey[j] = ki;
            sidx[i] = ij;
            sidx[j] = ii;
          }
        }
      }
      __syncthreads();
    }
  }

  // ---- outputs
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  for (int i = tid; i < K; i += nt) {
    const int64_t o = (int64_t)blockIdx.x * K + i;
    if (i < nsel) {
      const int p = sidx[i];
      const int l1 = p % L1, l2 = p / L1;
      // product and sum rounded separately (no contraction), as the grid is defined
      const double f1 = __dadd_rn(-g1, __dmul_rn((double)l1, 2.0 * g1 / (double)L1));
      const double f2 = __dadd_rn(-g2, __dmul_rn((double)l2, 2.0 * g2 / (double)L2));
      idx_out[o] = p;
      mag_out[o] = P::root(P::value(skey[i]));
      harm_out[2 * o] = f1;
      harm_out[2 * o + 1] = f2;
      const double u1 = f1 / g1, u2 = f2 / g2;
      const double s = __dadd_rn(__dmul_rn(u1, u1), __dmul_rn(u2, u2));
      if (s <= 1.0) {
        ang_out[2 * o] = atan2(u2, u1);
        ang_out[2 * o + 1] = asin(sqrt(s));
      } else {
        ang_out[2 * o] = nan;
        ang_out[2 * o + 1] = nan;
      }
    } else {
      idx_out[o] = -1;
      mag_out[o] = 0.0;
      harm_out[2 * o] = nan;
      harm_out[2 * o + 1] = nan;
      ang_out[2 * o] = nan;
      ang_out[2 * o + 1] = nan;
    }
  }
  if (tid == 0 && count_out) count_out[blockIdx.x] = (int)cnt;
}

}  // namespace

cudaError_t run_peaks(bccb_solver* s, const void* c_dev, int K, double rel_thresh, int* idx, double* mag,
                      double* harm, double* ang, int* count) {
  const double rel2 = rel_thresh * rel_thresh;
  if (s->prec == 1)
    peaks_kernel<double2><<<s->n, kPeakThreads, 0, s->stream>>>(
        s->d_desc, reinterpret_cast<const double2*>(c_dev), K, rel2, s->gamma1, s->gamma2, idx, mag, harm, ang,
        count);
  else
    peaks_kernel<float2><<<s->n, kPeakThreads, 0, s->stream>>>(
        s->d_desc, reinterpret_cast<const float2*>(c_dev), K, rel2, s->gamma1, s->gamma2, idx, mag, harm, ang,
        count);
  s->launches += 1;
  return cudaGetLastError();
}

}  // namespace bccb
