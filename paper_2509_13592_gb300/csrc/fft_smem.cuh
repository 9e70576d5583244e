// Radix-4 (plus one radix-2 stage for odd log2 n) Stockham FFT in shared memory for
// runtime lengths n <= 1024, on float2 or double2; used by the FP64 setup/check passes
// and the multi-pass solver.
#pragma once

#include "common.cuh"

namespace bccb {

// Stockham FFT of `cnt` interleaved sequences of length n (element e of sequence q at
// x[e * cnt + q]), ping-pong between x and y; returns the buffer that holds the result.
template <typename V, bool INV>
__device__ inline V* fft_smem(V* x, V* y, int n, int cnt, const V* __restrict__ tw) {
  int Ns = 1;
  while (Ns * 4 <= n) {
    const int q4 = n >> 2;
    const int step = kTwiddleLen / (4 * Ns);
    for (int idx = threadIdx.x; idx < q4 * cnt; idx += blockDim.x) {
      const int q = idx % cnt, j = idx / cnt;
      const int kk = j % Ns;
      V v0 = x[j * cnt + q], v1 = x[(j + q4) * cnt + q], v2 = x[(j + 2 * q4) * cnt + q],
        v3 = x[(j + 3 * q4) * cnt + q];
      if (Ns > 1) {
        v1 = twmul<INV>(v1, tw[kk * step]);
        v2 = twmul<INV>(v2, tw[2 * kk * step]);
        v3 = twmul<INV>(v3, tw[3 * kk * step]);
      }
      dft4<INV>(v0, v1, v2, v3);
      const int o = (j / Ns) * 4 * Ns + kk;
      y[o * cnt + q] = v0;
      y[(o + Ns) * cnt + q] = v1;
      y[(o + 2 * Ns) * cnt + q] = v2;
      y[(o + 3 * Ns) * cnt + q] = v3;
    }
    __syncthreads();
    V* t = x;
    x = y;
    y = t;
    Ns *= 4;
  }
  if (Ns < n) {
    const int h = n >> 1;
    const int step = kTwiddleLen / (2 * Ns);
    for (int idx = threadIdx.x; idx < h * cnt; idx += blockDim.x) {
      const int q = idx % cnt, j = idx / cnt;
      const int kk = j % Ns;
      const V a = x[j * cnt + q];
      const V b = twmul<INV>(x[(j + h) * cnt + q], tw[kk * step]);
      const int o = (j / Ns) * 2 * Ns + kk;
      y[o * cnt + q] = cadd(a, b);
      y[(o + Ns) * cnt + q] = csub(a, b);
    }
    __syncthreads();
    x = y;
  }
  return x;
}


}  // namespace bccb
