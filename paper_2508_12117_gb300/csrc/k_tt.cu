// Travel times T(x; s) and source Jacobians dT/dx for a list of
// (event, station) pairs (Sec. 2.1 and the forward model of Eq. forwardmodel).
//
//  * homogeneous medium: T = r / v, dT/dx = (x - s) / (v r), with r and T in
//    double-float so that dd differences keep sub-microsecond accuracy;
//  * linear-gradient medium v = v0 + g z: T = arccosh(1 + g^2 r^2/(2 v_x v_s))/g
//    in FP32;
//  * MLP stand-in for EikoNet (Sec. 3.2): T = r * tau(x, s), tau = 6 -> 4 x H
//    SiLU -> 1, with the source Jacobian by a hand-written reverse sweep
//    (delta_L = w_out * silu'(z_L), delta_{l-1} = (W_l^T delta_l) * silu'(z_{l-1}),
//    dtau/dx = W_1[:, :3]^T delta_1) and dT/dx = tau (x - s)/r + r dtau/dx.
//    This file holds the FP32 SIMT form; the tensor-core forms live in k_mlp_tc.cu.
#include <cuda_runtime.h>

#include "dfloat.cuh"
#include "kernels.h"
#include "pairs.cuh"
#include "spider.h"

namespace spider {

namespace {

__global__ void k_tt_homogeneous(NetView net, PairSource src, TTOut out) {
  const int64_t P = pair_count(src);
  const df32 inv_v = {net.inv_v_hi, net.inv_v_lo};
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < P;
       u += (int64_t)gridDim.x * blockDim.x) {
    PairGeo g;
    load_pair(src, u, g);
    df32 d[3];
    const df32 r = geometry(g, d);
    const df32 T = df_mul(r, inv_v);
    out.T2[u] = make_float2(T.hi, T.lo);
    if (out.J) {
      const float f = net.inv_v_hi / r.hi;
      out.J[u] = make_float4(d[0].hi * f, d[1].hi * f, d[2].hi * f, 0.f);
    }
  }
}

__global__ void k_tt_gradient(NetView net, PairSource src, TTOut out) {
  const int64_t P = pair_count(src);
  const float v0 = net.v0, gg = net.g;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < P;
       u += (int64_t)gridDim.x * blockDim.x) {
    PairGeo g;
    load_pair(src, u, g);
    df32 d[3];
    const df32 r = geometry(g, d);
    const float zs = g.shi[2] + (g.slo[2] + g.soff[2]);
    const float zr = g.rhi[2] + g.rlo[2];
    const float vs = v0 + gg * zs, vr = v0 + gg * zr;
    const float X = gg * gg * r.hi * r.hi / (2.f * vs * vr);
    const float sq = sqrtf(X * (2.f + X));
    const float T = log1pf(X + sq) / gg;
    out.T2[u] = make_float2(T, 0.f);
    if (out.J) {
      const float dTdX = 1.f / (gg * sq);
      const float c = dTdX * gg * gg / (vs * vr);
      out.J[u] = make_float4(c * d[0].hi, c * d[1].hi, c * d[2].hi - dTdX * X * gg / vs, 0.f);
    }
  }
}

// ------------------------------------------------------------------ FP32 MLP
constexpr int kTP = 64;       // pairs per tile
constexpr int kKC = 16;       // weight rows staged per chunk
constexpr int kWarps = 8;

__device__ __forceinline__ void silu_fp32(float z, float& h, float& ds) {
  const float s = 1.0f / (1.0f + expf(-z));
  h = z * s;
  ds = s * (1.0f + z * (1.0f - s));
}

// acc[pp][uu] = sum_k act[k][l + 32 pp] * Bm[k][w UPT + uu]  (Bm row-major H x H)
template <int H>
__device__ __forceinline__ void gemm_tile(const float* __restrict__ Bm, const float* act, float* wbuf,
                                          float (&acc)[2][H / kWarps], int w, int l) {
  constexpr int UPT = H / kWarps;
#pragma unroll
  for (int pp = 0; pp < 2; ++pp)
#pragma unroll
    for (int uu = 0; uu < UPT; ++uu) acc[pp][uu] = 0.f;
  for (int k0 = 0; k0 < H; k0 += kKC) {
    __syncthreads();
    const float4* srcw = reinterpret_cast<const float4*>(Bm + (size_t)k0 * H);
    for (int i = threadIdx.x; i < kKC * H / 4; i += blockDim.x)
      reinterpret_cast<float4*>(wbuf)[i] = __ldg(srcw + i);
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kKC; ++kk) {
      const float a0 = act[(k0 + kk) * kTP + l];
      const float a1 = act[(k0 + kk) * kTP + l + 32];
      const float4* wr = reinterpret_cast<const float4*>(wbuf + kk * H + w * UPT);
#pragma unroll
      for (int q = 0; q < UPT / 4; ++q) {
        const float4 b = wr[q];
        acc[0][4 * q + 0] = fmaf(a0, b.x, acc[0][4 * q + 0]);
        acc[0][4 * q + 1] = fmaf(a0, b.y, acc[0][4 * q + 1]);
        acc[0][4 * q + 2] = fmaf(a0, b.z, acc[0][4 * q + 2]);
        acc[0][4 * q + 3] = fmaf(a0, b.w, acc[0][4 * q + 3]);
        acc[1][4 * q + 0] = fmaf(a1, b.x, acc[1][4 * q + 0]);
        acc[1][4 * q + 1] = fmaf(a1, b.y, acc[1][4 * q + 1]);
        acc[1][4 * q + 2] = fmaf(a1, b.z, acc[1][4 * q + 2]);
        acc[1][4 * q + 3] = fmaf(a1, b.w, acc[1][4 * q + 3]);
      }
    }
  }
  __syncthreads();   // every read of act for this layer is done
}

// Persistent FP32 SIMT MLP: tiles of 64 pairs, 8 warps; lane l owns pairs l and
// l + 32 of the tile, warp w owns hidden units [w H/8, (w+1) H/8).  silu'(z) of
// layers 1-3 goes to a per-CTA scratch slot (rewritten every tile, so it stays in L2).
template <int H>
__global__ void __launch_bounds__(256) k_tt_mlp_fp32(NetView net, PairSource src, TTOut out,
                                                     float* __restrict__ scratch) {
  constexpr int UPT = H / kWarps;
  extern __shared__ float sm[];
  float* act = sm;                         // [H][kTP]
  float* wbuf = act + H * kTP;             // [kKC][H]
  float* xin = wbuf + kKC * H;             // [6][kTP]
  float* red = xin + 6 * kTP;              // [kWarps][4][kTP]
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  float* dsg = scratch + (size_t)blockIdx.x * 3 * H * kTP;
  const int64_t P = pair_count(src);
  const int64_t ntiles = (P + kTP - 1) / kTP;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t u0 = tile * kTP;
    __syncthreads();
    if (threadIdx.x < kTP) {
      const int64_t u = u0 + threadIdx.x;
      PairGeo g;
      load_pair(src, u < P ? u : u0, g);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        xin[c * kTP + threadIdx.x] = g.shi[c] + (g.slo[c] + g.soff[c]);
        xin[(3 + c) * kTP + threadIdx.x] = g.rhi[c] + g.rlo[c];
      }
    }
    __syncthreads();
    // layer 1 (6 -> H)
#pragma unroll
    for (int pp = 0; pp < 2; ++pp) {
      const int p = l + 32 * pp;
      float x[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) x[c] = xin[c * kTP + p];
      for (int uu = 0; uu < UPT; ++uu) {
        const int n = w * UPT + uu;
        float z = __ldg(net.b1 + n);
#pragma unroll
        for (int c = 0; c < 6; ++c) z = fmaf(__ldg(net.W1 + n * 6 + c), x[c], z);
        float h, ds;
        silu_fp32(z, h, ds);
        act[n * kTP + p] = h;
        dsg[(0 * H + n) * kTP + p] = ds;
      }
    }
    float acc[2][UPT];
    float tp[2] = {0.f, 0.f};
    // layers 2..4
#pragma unroll 1
    for (int lyr = 0; lyr < 3; ++lyr) {
      gemm_tile<H>(net.Wt[lyr], act, wbuf, acc, w, l);
#pragma unroll
      for (int pp = 0; pp < 2; ++pp) {
        const int p = l + 32 * pp;
#pragma unroll
        for (int uu = 0; uu < UPT; ++uu) {
          const int n = w * UPT + uu;
          float h, ds;
          silu_fp32(acc[pp][uu] + __ldg(net.bh[lyr] + n), h, ds);
          if (lyr < 2) {
            act[n * kTP + p] = h;
            dsg[((lyr + 1) * H + n) * kTP + p] = ds;
          } else {
            const float w5 = __ldg(net.W5 + n);
            tp[pp] = fmaf(w5, h, tp[pp]);
            act[n * kTP + p] = w5 * ds;     // delta_4
          }
        }
      }
    }
    red[(w * 4 + 0) * kTP + l] = tp[0];
    red[(w * 4 + 0) * kTP + l + 32] = tp[1];
    // backward: delta_{l-1} = (W_l^T delta_l) * silu'(z_{l-1}), l = 4, 3
#pragma unroll 1
    for (int lyr = 2; lyr >= 1; --lyr) {
      gemm_tile<H>(net.Wn[lyr], act, wbuf, acc, w, l);
#pragma unroll
      for (int pp = 0; pp < 2; ++pp) {
        const int p = l + 32 * pp;
#pragma unroll
        for (int uu = 0; uu < UPT; ++uu) {
          const int n = w * UPT + uu;
          act[n * kTP + p] = acc[pp][uu] * dsg[(lyr * H + n) * kTP + p];
        }
      }
    }
    // delta_1 = (W_2^T delta_2) * silu'(z_1); dtau/dx_src = W_1[:, :3]^T delta_1
    gemm_tile<H>(net.Wn[0], act, wbuf, acc, w, l);
#pragma unroll
    for (int pp = 0; pp < 2; ++pp) {
      const int p = l + 32 * pp;
      float g3[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int uu = 0; uu < UPT; ++uu) {
        const int n = w * UPT + uu;
        const float d1 = acc[pp][uu] * dsg[(0 * H + n) * kTP + p];
#pragma unroll
        for (int c = 0; c < 3; ++c) g3[c] = fmaf(__ldg(net.W1 + n * 6 + c), d1, g3[c]);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) red[(w * 4 + 1 + c) * kTP + p] = g3[c];
    }
    __syncthreads();
    if (threadIdx.x < kTP) {
      const int64_t u = u0 + threadIdx.x;
      if (u < P) {
        float s[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ww = 0; ww < kWarps; ++ww)
#pragma unroll
          for (int c = 0; c < 4; ++c) s[c] += red[(ww * 4 + c) * kTP + threadIdx.x];
        PairGeo g;
        load_pair(src, u, g);
        df32 d[3];
        const df32 r = geometry(g, d);
        // T = r * (b5 + dtau): the bias part in double-float, the network part in FP32
        const df32 T = df_add_f(df_mul_f(r, net.b5), r.hi * s[0]);
        out.T2[u] = make_float2(T.hi, T.lo);
        if (out.J) {
          const float tau = net.b5 + s[0];
          const float f = tau / r.hi;
          out.J[u] = make_float4(f * d[0].hi + r.hi * s[1], f * d[1].hi + r.hi * s[2],
                                 f * d[2].hi + r.hi * s[3], 0.f);
        }
      }
    }
  }
}

template <int H>
size_t mlp_fp32_smem() {
  return (size_t)(H * kTP + kKC * H + 6 * kTP + kWarps * 4 * kTP) * sizeof(float);
}

template <int H>
cudaError_t launch_mlp_fp32(const NetView& net, const PairSource& src, TTOut out, int grid,
                            float* scratch, cudaStream_t st) {
  const size_t smem = mlp_fp32_smem<H>();
  cudaError_t e = cudaFuncSetAttribute(k_tt_mlp_fp32<H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_tt_mlp_fp32<H><<<grid, 256, smem, st>>>(net, src, out, scratch);
  return cudaGetLastError();
}

}  // namespace

int mlp_fp32_grid(int num_sms) { return 2 * num_sms; }

size_t tt_scratch_floats(const NetView& net, int num_sms) {
  if (net.kind != SPIDER_TT_MLP) return 0;
  const size_t fp32 = (size_t)mlp_fp32_grid(num_sms) * 3 * net.H * kTP;
  const size_t tc = (size_t)num_sms * 3 * 128 * net.H / 2; // three 128 x H BF16 slots per SM
  return fp32 > tc ? fp32 : tc;
}

bool tt_supported_width(int H) { return H == 32 || H == 64 || H == 128 || H == 256; }

cudaError_t launch_tt(const NetView& net, const PairSource& src, TTOut out, int num_sms, float* scratch,
                      cudaStream_t st, int ctas_per_sm) {
  if (net.kind == SPIDER_TT_HOMOGENEOUS) {
    k_tt_homogeneous<<<4 * num_sms, 256, 0, st>>>(net, src, out);
    return cudaGetLastError();
  }
  if (net.kind == SPIDER_TT_LINEAR_GRADIENT) {
    k_tt_gradient<<<4 * num_sms, 256, 0, st>>>(net, src, out);
    return cudaGetLastError();
  }
  if (net.precision != SPIDER_FP32) {
    cudaError_t e = launch_mlp_tc(net, src, out, num_sms, scratch, st);
    if (e != cudaErrorNotSupported) return e;
    return cudaErrorNotSupported;
  }
  const int grid = (ctas_per_sm == 1 ? 1 : 2) * num_sms;   // never above the scratch slots
  switch (net.H) {
    case 32: return launch_mlp_fp32<32>(net, src, out, grid, scratch, st);
    case 64: return launch_mlp_fp32<64>(net, src, out, grid, scratch, st);
    case 128: return launch_mlp_fp32<128>(net, src, out, grid, scratch, st);
    case 256: return launch_mlp_fp32<256>(net, src, out, grid, scratch, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace spider
