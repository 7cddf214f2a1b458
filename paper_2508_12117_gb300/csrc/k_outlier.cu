// Stage-1 outlier rejection (Sec. 3.2, "residuals greater than 4 median
// absolute deviations"): per sub-problem, the median of the full-batch
// residuals, their median absolute deviation MAD = median |r - median|, and the
// keep mask |r - median| <= k MAD.  Medians are found by radix selection over
// order-preserving integer keys of the FP32 values (4 passes of 8 bits, exact
// and deterministic: integer histograms); an even count takes the mean of the
// two middle values.
#include <cuda_runtime.h>

#include <cstdint>

#include "dfloat.cuh"
#include "kernels.h"
#include "spider.h"
#include "view.h"

namespace spider {
namespace {

constexpr int kBins = 256;
constexpr int kSmemSubs = 8;           // sub-problems histogrammed in shared memory

__device__ __forceinline__ uint32_t fkey(float x) {
  const uint32_t u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// per sub-problem: observation range, two ranks (the middle pair), their
// key prefixes fixed so far, the median and the MAD
struct SelSub {
  int64_t lo, hi;
  int64_t k[2];
  uint32_t prefix[2];
  float med, mad;
};

__device__ __forceinline__ int sub_of(const SelSub* s, int n_sub, int64_t e) {
  int a = 0, b = n_sub - 1;
  while (a < b) {
    const int m = (a + b + 1) >> 1;
    if (s[m].lo <= e) a = m;
    else b = m - 1;
  }
  return a;
}

__global__ void k_sel_init(StepView v, SelSub* s, int n_sub) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_sub) return;
  const int64_t lo = v.blk_e0[v.sub_blk_off[i]], hi = v.blk_e0[v.sub_blk_off[i + 1]];
  const int64_t n = hi - lo;
  s[i].lo = lo;
  s[i].hi = hi;
  s[i].k[0] = n > 0 ? (n - 1) / 2 : 0;
  s[i].k[1] = n > 0 ? n / 2 : 0;
  s[i].prefix[0] = s[i].prefix[1] = 0;
  s[i].med = 0.f;
  s[i].mad = 0.f;
}

// histogram of the next 8 key bits of the values matching each rank's prefix;
// mode 0: keys of r, mode 1: keys of |r - median|
__global__ void k_sel_hist(const float* __restrict__ r, int64_t N, const SelSub* s, int n_sub, int mode,
                           uint32_t mask, int shift, uint32_t* hist) {
  __shared__ uint32_t sh[kSmemSubs * 2 * kBins];
  const bool use_smem = n_sub <= kSmemSubs;
  if (use_smem) {
    for (int i = threadIdx.x; i < n_sub * 2 * kBins; i += blockDim.x) sh[i] = 0;
    __syncthreads();
  }
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    const int sb = sub_of(s, n_sub, e);
    const float x = mode == 0 ? r[e] : fabsf(r[e] - s[sb].med);
    const uint32_t key = fkey(x);
    const uint32_t bin = (key >> shift) & (kBins - 1);
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      if ((key & mask) != s[sb].prefix[l]) continue;
      if (l == 1 && s[sb].k[1] == s[sb].k[0] && s[sb].prefix[1] == s[sb].prefix[0]) continue;   // same rank
      if (use_smem) atomicAdd(&sh[(sb * 2 + l) * kBins + bin], 1u);
      else atomicAdd(&hist[((size_t)sb * 2 + l) * kBins + bin], 1u);
    }
  }
  if (use_smem) {
    __syncthreads();
    for (int i = threadIdx.x; i < n_sub * 2 * kBins; i += blockDim.x)
      if (sh[i]) atomicAdd(&hist[i], sh[i]);
  }
}

// one block per sub-problem: pick the bin holding each rank, extend its prefix
__global__ void k_sel_pick(SelSub* s, int shift, uint32_t* hist) {
  __shared__ uint32_t cnt[kBins];
  const int sb = blockIdx.x;
  // both ranks on one path (odd count): rank 1 was not histogrammed, it reuses rank 0's
  const bool same = s[sb].k[1] == s[sb].k[0] && s[sb].prefix[1] == s[sb].prefix[0];
  __syncthreads();
  for (int l = 0; l < 2; ++l) {
    const int src = (l == 1 && same) ? 0 : l;
    uint32_t* h = hist + ((size_t)sb * 2 + src) * kBins;
    for (int i = threadIdx.x; i < kBins; i += blockDim.x) cnt[i] = h[i];
    __syncthreads();
    if (threadIdx.x == 0) {
      int64_t k = s[sb].k[l];
      int b = 0;
      for (; b < kBins - 1; ++b) {
        if (k < (int64_t)cnt[b]) break;
        k -= cnt[b];
      }
      s[sb].k[l] = k;
      s[sb].prefix[l] |= (uint32_t)b << shift;
    }
    __syncthreads();
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * kBins; i += blockDim.x) hist[(size_t)sb * 2 * kBins + i] = 0;
}

__global__ void k_sel_done(SelSub* s, int n_sub, int mode) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_sub) return;
  const float a = fkey_inv(s[i].prefix[0]), b = fkey_inv(s[i].prefix[1]);
  const float m = s[i].hi > s[i].lo ? 0.5f * (a + b) : 0.f;
  if (mode == 0) s[i].med = m;
  else s[i].mad = m;
  // reset the ranks for the next selection
  const int64_t n = s[i].hi - s[i].lo;
  s[i].k[0] = n > 0 ? (n - 1) / 2 : 0;
  s[i].k[1] = n > 0 ? n / 2 : 0;
  s[i].prefix[0] = s[i].prefix[1] = 0;
}

__global__ void k_keep(const float* __restrict__ r, int64_t N, const SelSub* s, int n_sub, float kmad,
                       uint8_t* keep, unsigned long long* kept) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int mine = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
    const int sb = sub_of(s, n_sub, e);
    const uint8_t k = fabsf(r[e] - s[sb].med) <= kmad * s[sb].mad ? 1 : 0;
    keep[e] = k;
    mine += k;
  }
  atomicAdd(&cnt, mine);
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(kept, (unsigned long long)cnt);
}

}  // namespace

size_t outlier_scratch_bytes(int n_sub) {
  return (size_t)n_sub * sizeof(SelSub) + (size_t)n_sub * 2 * kBins * sizeof(uint32_t) + 64;
}

// residuals r (canonical order, the full catalog) -> keep mask, per-sub median
// and MAD (host copies), kept count.  scratch: outlier_scratch_bytes(n_sub).
cudaError_t launch_outlier(const StepView& v, int n_sub, float kmad, void* scratch, uint8_t* keep,
                           int num_sms, cudaStream_t st, float* med_host, float* mad_host, int64_t* n_kept) {
  SelSub* s = reinterpret_cast<SelSub*>(scratch);
  uint32_t* hist = reinterpret_cast<uint32_t*>(s + n_sub);
  unsigned long long* kept = reinterpret_cast<unsigned long long*>(hist + (size_t)n_sub * 2 * kBins);
  cudaError_t e;
  if ((e = cudaMemsetAsync(hist, 0, (size_t)n_sub * 2 * kBins * sizeof(uint32_t) + sizeof(unsigned long long), st)))
    return e;
  const int gs = (n_sub + 127) / 128;
  k_sel_init<<<gs, 128, 0, st>>>(v, s, n_sub);
  const int grid = 2 * num_sms;
  for (int mode = 0; mode < 2; ++mode) {
    uint32_t mask = 0;
    for (int pass = 0; pass < 4; ++pass) {
      const int shift = 24 - 8 * pass;
      k_sel_hist<<<grid, 256, 0, st>>>(v.r_obs, v.N, s, n_sub, mode, mask, shift, hist);
      k_sel_pick<<<n_sub, 256, 0, st>>>(s, shift, hist);
      mask |= 0xFFu << shift;
    }
    k_sel_done<<<gs, 128, 0, st>>>(s, n_sub, mode);
  }
  k_keep<<<grid, 256, 0, st>>>(v.r_obs, v.N, s, n_sub, kmad, keep, kept);
  if ((e = cudaGetLastError())) return e;
  for (int i = 0; i < n_sub; ++i) {
    if ((e = cudaMemcpyAsync(&med_host[i], &s[i].med, sizeof(float), cudaMemcpyDeviceToHost, st))) return e;
    if ((e = cudaMemcpyAsync(&mad_host[i], &s[i].mad, sizeof(float), cudaMemcpyDeviceToHost, st))) return e;
  }
  unsigned long long kh = 0;
  if ((e = cudaMemcpyAsync(&kh, kept, sizeof(kh), cudaMemcpyDeviceToHost, st))) return e;
  if ((e = cudaStreamSynchronize(st))) return e;
  *n_kept = (int64_t)kh;
  return cudaSuccess;
}

}  // namespace spider

// ---------------------------------------------------------------------------
// Linearisation-regime filter (Proposition 1; Sec. 4 drops observations whose
// linearisation error exceeds 5 %): with T and dT/dx_s of every pair at the
// current state, observation (i, j, k) has
//   dT = T(x_j, s_k) - T(x_i, s_k),   dT_lin = grad_x T(x_i, s_k) . (x_j - x_i),
// and is kept when |dT - dT_lin| <= max_rel |dT|.
namespace spider {
namespace {

__global__ void k_linfilter(StepView v, float max_rel, uint8_t* keep, unsigned long long* kept) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  const int s = blockIdx.x;
  const int32_t b = v.sel[s];
  const int32_t q0 = v.blk_node_off[b];
  const int64_t e0 = v.blk_e0[b];
  const int ne = v.blk_e0[b + 1] - v.blk_e0[b];
  int mine = 0;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    const uint32_t lij = v.obs_l[e0 + e];
    const int32_t qi = q0 + (int)(lij & 0xFFFF), qj = q0 + (int)(lij >> 16);
    const int32_t ui = v.loc2u[qi], uj = v.loc2u[qj];
    const float2 ti = v.T2[ui], tj = v.T2[uj];
    const float4 Ji = v.J[ui];
    const int32_t mi = v.pair_ev[v.node_pair[qi]], mj = v.pair_ev[v.node_pair[qj]];
    const float4 hi_i = v.th0_hi[mi], lo_i = v.th0_lo[mi], d_i = v.dth[mi];
    const float4 hi_j = v.th0_hi[mj], lo_j = v.th0_lo[mj], d_j = v.dth[mj];
    const df32 dT = df_add(df32{tj.x, tj.y}, df32{-ti.x, -ti.y});
    const float dx = df_coord_diff(hi_j.x, lo_j.x, d_j.x - d_i.x, hi_i.x, lo_i.x).hi;
    const float dy = df_coord_diff(hi_j.y, lo_j.y, d_j.y - d_i.y, hi_i.y, lo_i.y).hi;
    const float dz = df_coord_diff(hi_j.z, lo_j.z, d_j.z - d_i.z, hi_i.z, lo_i.z).hi;
    const float lin = fmaf(Ji.x, dx, fmaf(Ji.y, dy, Ji.z * dz));
    const float err = fabsf(df_add_f(dT, -lin).hi);
    const uint8_t k = err <= max_rel * fabsf(dT.hi) ? 1 : 0;
    keep[e0 + e] = k;
    mine += k;
  }
  atomicAdd(&cnt, mine);
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(kept, (unsigned long long)cnt);
}

}  // namespace

// after a full-batch evaluation (every block selected, T and J per unique pair)
cudaError_t launch_linfilter(const StepView& v, int64_t n_b, float max_rel, uint8_t* keep,
                             unsigned long long* kept, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(kept, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  if (n_b > 0) k_linfilter<<<(unsigned)n_b, 256, 0, st>>>(v, max_rel, keep, kept);
  return cudaGetLastError();
}

}  // namespace spider
