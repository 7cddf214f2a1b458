// spider_tt_pairs_noalloc: the FP32 travel-time MLP (forward + source
// Jacobian) for callers that must not allocate device memory.
//
// Everything the kernel needs beyond the caller's inputs and outputs -- the
// network weights in the layouts the kernel reads, the per-CTA slots holding
// silu'(z) between the forward and the reverse sweep, and the (hi, lo) staging
// of T -- lives in one file-scope __device__ array of fixed size.  The array
// exists on every GPU that loads the library, from module load until exit.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "kernels.h"
#include "spider.h"

namespace spider {
namespace {

constexpr int kNaMaxH = 256;
constexpr int64_t kNaMaxPairs = int64_t(1) << 20;
constexpr int kNaCtas = 152;                 // persistent grid of the FP32 MLP kernel
constexpr int kNaTile = 64;                  // pairs per tile of that kernel
constexpr size_t kNaWeights = (size_t)kNaMaxH * 6 + kNaMaxH + 6 * (size_t)kNaMaxH * kNaMaxH +
                              3 * (size_t)kNaMaxH + kNaMaxH;
constexpr size_t kNaSlots = (size_t)kNaCtas * 3 * kNaMaxH * kNaTile;
constexpr size_t kNaStage = 2 * (size_t)kNaMaxPairs;
constexpr size_t kNaFloats = kNaWeights + kNaSlots + kNaStage;   // ~40 MB

__device__ __align__(256) float g_na_scratch[kNaFloats];

constexpr int kNaMaxDevices = 64;
float* g_na_ptr[kNaMaxDevices] = {};
std::mutex g_na_mu;

// device address of the scratch array on the current device, looked up once
// per device and kept for the life of the process (a cudaDeviceReset while the
// library is loaded would leave it stale: not supported)
cudaError_t scratch_address(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_na_mu);
  if (!g_na_ptr[dev]) {
    float* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_na_scratch);
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = p;
  }
  *out = g_na_ptr[dev];
  return cudaSuccess;
}

__global__ void k_transpose(const float* __restrict__ W, float* __restrict__ Wt, int H) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= H * H) return;
  const int o = i / H, k = i % H;
  Wt[(size_t)k * H + o] = W[i];
}

}  // namespace
}  // namespace spider

using namespace spider;

static void na_error(const char* m) { set_static_error(m); }

extern "C" int spider_tt_pairs_noalloc(const spider_net* net, int64_t P, const float* src,
                                       const float* rcv, float* T_hi, float* T_lo, float* J,
                                       void* stream) {
  if (!net || net->kind != SPIDER_TT_MLP) {
    na_error("spider_tt_pairs_noalloc serves the MLP travel-time model only");
    return SPIDER_E_UNSUPPORTED;
  }
  const int H = net->H;
  if (!tt_supported_width(H) || H > kNaMaxH) {
    na_error("spider_tt_pairs_noalloc: H must be 32, 64, 128 or 256");
    return SPIDER_E_UNSUPPORTED;
  }
  if (P < 0 || P > kNaMaxPairs) {
    na_error("spider_tt_pairs_noalloc: P must be in [0, 2^20]");
    return SPIDER_E_INVAL;
  }
  {
    const size_t wn[5] = {(size_t)H * 6, (size_t)H * H, (size_t)H * H, (size_t)H * H, (size_t)H};
    const size_t bn[5] = {(size_t)H, (size_t)H, (size_t)H, (size_t)H, 1};
    for (int l = 0; l < 5; ++l) {
      if (!net->W[l] || !net->b[l]) {
        na_error("spider_tt_pairs_noalloc: null weight or bias");
        return SPIDER_E_INVAL;
      }
      // the same rejection as spider_tt_pairs: a NaN or Inf weight would only
      // surface as NaN travel times
      for (size_t i = 0; i < wn[l]; ++i)
        if (!std::isfinite(net->W[l][i])) {
          na_error("spider_tt_pairs_noalloc: non-finite MLP weight");
          return SPIDER_E_INVAL;
        }
      for (size_t i = 0; i < bn[l]; ++i)
        if (!std::isfinite(net->b[l][i])) {
          na_error("spider_tt_pairs_noalloc: non-finite MLP bias");
          return SPIDER_E_INVAL;
        }
    }
  }
  if (P == 0) return SPIDER_OK;
  if (!src || !rcv || !T_hi) {
    na_error("spider_tt_pairs_noalloc: null src, rcv or T_hi");
    return SPIDER_E_INVAL;
  }
  float* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) {
    na_error(cudaGetErrorString(e));
    return SPIDER_E_CUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t HH = (size_t)H * H;
  float* W1 = base;
  float* b1 = W1 + (size_t)H * 6;
  float* Wn = b1 + H;          // 3 x H x H, (out, in)
  float* Wt = Wn + 3 * HH;     // 3 x H x H, (in, out)
  float* bh = Wt + 3 * HH;     // 3 x H
  float* W5 = bh + 3 * H;      // H
  float* slots = base + kNaWeights;
  float2* stage = reinterpret_cast<float2*>(slots + kNaSlots);
  e = cudaMemcpyAsync(W1, net->W[0], (size_t)H * 6 * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b1, net->b[0], H * sizeof(float), cudaMemcpyHostToDevice, st);
  for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
    e = cudaMemcpyAsync(Wn + l * HH, net->W[l + 1], HH * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(bh + l * H, net->b[l + 1], H * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
      k_transpose<<<(unsigned)((HH + 255) / 256), 256, 0, st>>>(Wn + l * HH, Wt + l * HH, H);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(W5, net->W[4], H * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    NetView nv{};
    nv.kind = SPIDER_TT_MLP;
    nv.H = H;
    nv.precision = SPIDER_FP32;
    nv.W1 = W1;
    nv.b1 = b1;
    for (int l = 0; l < 3; ++l) {
      nv.Wn[l] = Wn + l * HH;
      nv.Wt[l] = Wt + l * HH;
      nv.bh[l] = bh + l * H;
    }
    nv.W5 = W5;
    nv.b5 = net->b[4][0];
    PairSource ps{};
    ps.src = reinterpret_cast<const float4*>(src);
    ps.rcv = reinterpret_cast<const float4*>(rcv);
    ps.n_host = P;
    TTOut o{stage, reinterpret_cast<float4*>(J)};
    // launch_tt sizes the FP32 MLP grid as 2 x (its SM argument): kNaCtas CTAs,
    // one scratch slot each
    e = launch_tt(nv, ps, o, kNaCtas / 2, slots, st, 2);
  }
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(T_hi, sizeof(float), stage, sizeof(float2), sizeof(float), (size_t)P,
                          cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && T_lo)
    e = cudaMemcpy2DAsync(T_lo, sizeof(float), reinterpret_cast<float*>(stage) + 1, sizeof(float2),
                          sizeof(float), (size_t)P, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) {
    na_error(cudaGetErrorString(e));
    return SPIDER_E_CUDA;
  }
  return SPIDER_OK;
}
