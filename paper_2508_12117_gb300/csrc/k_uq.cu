// Posterior summaries from the stored samples (Sec. 3.5 uncertainty
// quantification, Sec. 4.1 calibration against synthetic truth, Sec. 5 effective
// sample size), one warp per (event, coordinate) series of the n stored samples:
//   - effective sample size n / tau, tau = 1 + 2 sum_{t >= 1} rho_t over the
//     lags while the autocorrelation rho_t stays positive (time order);
//   - median and the half-length of the [lo, hi] percentile interval, linear
//     interpolation between order statistics at rank (n - 1) p / 100 (sorted
//     in shared memory, bitonic);
//   - the fraction of samples below the true value.
// FP64 arithmetic on the FP32 stored offsets from theta_0.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"
#include "view.h"

namespace spider {
namespace {

constexpr int kUqWarps = 8;

__device__ __forceinline__ double warp_sum_d(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ double pct_sorted(const float* a, int n, double p) {
  const double pos = (double)(n - 1) * p / 100.0;
  int lo = (int)floor(pos);
  if (lo < 0) lo = 0;
  if (lo > n - 1) lo = n - 1;
  const int hi = lo + 1 < n ? lo + 1 : n - 1;
  const double f = pos - (double)lo;
  return (double)a[lo] + f * ((double)a[hi] - (double)a[lo]);
}

// samples: sample_cap slots of M float4; the n series values are slots
// (first + s) % cap, s = 0..n-1, oldest first.  n2: next power of two >= n.
__global__ void __launch_bounds__(kUqWarps * 32)
    k_uq(const float4* __restrict__ samples, int64_t M, int64_t cap, int64_t first, int n, int n2,
         const double* __restrict__ truth_off, double lo_pct, double hi_pct, double* med, double* half,
         double* calib, double* ess) {
  extern __shared__ float sbuf[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* x = sbuf + (size_t)w * n2;
  const int64_t series = (int64_t)blockIdx.x * kUqWarps + w;
  if (series >= 4 * M) return;
  const int64_t m = series >> 2;
  const int a = (int)(series & 3);
  for (int s = lane; s < n2; s += 32) {
    float val = __int_as_float(0x7F800000);   // +inf pads the sort
    if (s < n) {
      const float4 v = samples[((first + s) % cap) * M + m];
      val = a == 0 ? v.x : (a == 1 ? v.y : (a == 2 ? v.z : v.w));
    }
    x[s] = val;
  }
  __syncwarp();
  // effective sample size (time order)
  double mu = 0.0;
  for (int s = lane; s < n; s += 32) mu += (double)x[s];
  mu = warp_sum_d(mu) / n;
  double c0 = 0.0;
  for (int s = lane; s < n; s += 32) {
    const double d = (double)x[s] - mu;
    c0 += d * d;
  }
  c0 = warp_sum_d(c0);
  double tau = 1.0;
  if (c0 > 0.0) {
    for (int t = 1; t < n; ++t) {
      double ct = 0.0;
      for (int s = lane; s + t < n; s += 32) ct += ((double)x[s] - mu) * ((double)x[s + t] - mu);
      ct = warp_sum_d(ct);
      const double rho = ct / c0;
      if (!(rho > 0.0)) break;
      tau += 2.0 * rho;
    }
  }
  // calibration against the truth (offset from theta_0)
  double below = 0.0;
  if (truth_off) {
    const double tv = truth_off[4 * m + a];
    for (int s = lane; s < n; s += 32) below += (double)x[s] < tv ? 1.0 : 0.0;
    below = warp_sum_d(below);
  }
  __syncwarp();
  // bitonic sort of the series (ascending)
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < n2; i += 32) {
        const int l = i ^ j;
        if (l > i) {
          const float p = x[i], q = x[l];
          const bool up = (i & k) == 0;
          if ((p > q) == up) {
            x[i] = q;
            x[l] = p;
          }
        }
      }
      __syncwarp();
    }
  if (lane == 0) {
    const size_t o = 4 * (size_t)m + a;
    if (med) med[o] = pct_sorted(x, n, 50.0);
    if (half) half[o] = 0.5 * (pct_sorted(x, n, hi_pct) - pct_sorted(x, n, lo_pct));
    if (calib) calib[o] = below / n;
    if (ess) ess[o] = (double)n / tau;
  }
}

}  // namespace

int uq_max_samples() { return 4096; }

cudaError_t launch_uq(const StepView& v, int64_t first, int n, const double* truth_off, double lo_pct,
                      double hi_pct, double* med, double* half, double* calib, double* ess, cudaStream_t st) {
  int n2 = 1;
  while (n2 < n) n2 <<= 1;
  const size_t smem = (size_t)kUqWarps * n2 * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_uq, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t nser = 4 * v.M;
  const unsigned grid = (unsigned)((nser + kUqWarps - 1) / kUqWarps);
  k_uq<<<grid, kUqWarps * 32, smem, st>>>(v.samples, v.M, v.sample_cap, first, n, n2, truth_off, lo_pct, hi_pct,
                                          med, half, calib, ess);
  return cudaGetLastError();
}

}  // namespace spider
