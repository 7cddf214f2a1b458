// Loading (event, station) pair geometry for the travel-time kernels.
#pragma once
#include <cuda_runtime.h>

#include "dfloat.cuh"
#include "view.h"

namespace spider {

struct PairGeo {
  float shi[3], slo[3], soff[3], rhi[3], rlo[3];
};

__device__ __forceinline__ int64_t pair_count(const PairSource& s) {
  return s.n_dev ? (int64_t)(*s.n_dev) : s.n_host;
}

__device__ __forceinline__ void load_pair(const PairSource& s, int64_t u, PairGeo& g) {
  if (s.uniq_pair) {
    const int32_t p = s.uniq_pair[u];
    const int32_t m = s.pair_ev[p], k = s.pair_st[p];
    const float4 a = s.th0_hi[m], b = s.th0_lo[m], d = s.dth[m], c = s.sta_hi[k], e = s.sta_lo[k];
    g.shi[0] = a.x; g.shi[1] = a.y; g.shi[2] = a.z;
    g.slo[0] = b.x; g.slo[1] = b.y; g.slo[2] = b.z;
    g.soff[0] = d.x; g.soff[1] = d.y; g.soff[2] = d.z;
    g.rhi[0] = c.x; g.rhi[1] = c.y; g.rhi[2] = c.z;
    g.rlo[0] = e.x; g.rlo[1] = e.y; g.rlo[2] = e.z;
  } else {
    const float4 a = s.src[u], c = s.rcv[u];
    g.shi[0] = a.x; g.shi[1] = a.y; g.shi[2] = a.z;
    g.rhi[0] = c.x; g.rhi[1] = c.y; g.rhi[2] = c.z;
#pragma unroll
    for (int i = 0; i < 3; ++i) g.slo[i] = g.soff[i] = g.rlo[i] = 0.f;
  }
}

// source - receiver per axis and the distance, in double-float
__device__ __forceinline__ df32 geometry(const PairGeo& g, df32 d[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) d[i] = df_coord_diff(g.shi[i], g.slo[i], g.soff[i], g.rhi[i], g.rlo[i]);
  df32 r2 = df_add(df_add(df_sqr(d[0]), df_sqr(d[1])), df_sqr(d[2]));
  return df_sqrt(r2);
}

}  // namespace spider
