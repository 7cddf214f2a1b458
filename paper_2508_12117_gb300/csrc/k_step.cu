// Step kernels: minibatch selection, the minibatch pair table, residuals,
// whitening (Eq. marginal_sigma through the push-through identity, solved by
// Jacobi-preconditioned CG in one cooperative launch), the deterministic
// scatter of dlogp/dT onto pairs and events, and the fused prior + SGLD update.
//
// Determinism: every reduction runs in a fixed order (per-node half-edge lists
// in observation order, per-pair occurrence lists in block order, per-CTA
// partials summed by index); no floating-point atomics anywhere.
#include <cuda_runtime.h>

#include "dfloat.cuh"
#include "kernels.h"
#include "philox.cuh"
#include "spider.h"
#include "step_util.cuh"

namespace spider {

namespace {

constexpr int kThreads = 256;

// Sum over the selected occurrences of pair p of vals[q] (block order).
__device__ __forceinline__ float merge_occ(const StepView& v, int32_t p, int tag, const float* vals) {
  float a = 0.f;
  for (int32_t t = v.inc_off[p], t1 = v.inc_off[p + 1]; t < t1; ++t)
    if (v.blk_stamp[v.inc_b[t]] == tag) a += vals[v.inc_q[t]];
  return a;
}

// ------------------------------------------------------------------ selection
__global__ void k_select(StepView v, int64_t n_b) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_b) return;
  const StepParams& pr = *v.prm;
  const int32_t* so = pr.full ? v.sub_sel_full : v.sub_sel_mb;
  int lo = 0, hi = v.n_sub;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (so[mid] <= t) lo = mid; else hi = mid;
  }
  const int s = lo;
  const int64_t i = t - so[s];
  const int64_t nbs = v.sub_blk_off[s + 1] - v.sub_blk_off[s];
  // each sub-problem draws its blocks with its own key
  const uint64_t key = pr.seed ^ (0x9E3779B97F4A7C15ull * (uint64_t)s);
  int64_t b = pr.full ? i : feistel_index(i, nbs, key);
  if (b < 0 || b >= nbs) {
    set_error(v.counters, SPIDER_E_TIMEOUT);
    b = i % nbs;
  }
  b += v.sub_blk_off[s];
  v.sel[t] = (int32_t)b;
  v.blk_stamp[b] = pr.tag;
  const int sz = v.blk_e0[b + 1] - v.blk_e0[b];
  atomicAdd(&v.counters[kCntObs], sz);
  atomicAdd(&v.sub_nsel[s], sz);
}

// owner of each local node = its occurrence in the selected block of lowest id
__global__ void k_owner(StepView v) {
  const int tag = v.prm->tag;
  __shared__ int sm[33];
  const int s = blockIdx.x;
  const int32_t b = v.sel[s];
  const int32_t q0 = v.blk_node_off[b], q1 = v.blk_node_off[b + 1];
  int cnt = 0;
  for (int32_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    const int32_t p = v.node_pair[q];
    int32_t qo = -1, bo = -1;
    int c = 0;
    for (int32_t t = v.inc_off[p], t1 = v.inc_off[p + 1]; t < t1; ++t)
      if (v.blk_stamp[v.inc_b[t]] == tag) {
        if (qo < 0) {
          qo = v.inc_q[t];
          bo = v.inc_b[t];
        }
        ++c;
      }
    v.owner_q[q] = qo;
    if (v.owner_b) v.owner_b[q] = bo;
    v.multi[q] = (uint8_t)(c > 1);
    cnt += (qo == q);
  }
  int tot = block_sum<int>(cnt, sm);
  if (threadIdx.x == 0) v.blk_owner_cnt[s] = tot;
}

__global__ void k_scan_owner(StepView v, int64_t n_b) {
  __shared__ int sm[33];
  int carry = 0;
  for (int64_t c = 0; c < n_b; c += blockDim.x) {
    int64_t s = c + threadIdx.x;
    int val = s < n_b ? v.blk_owner_cnt[s] : 0;
    int total;
    int pre = block_exscan(val, sm, &total);
    if (s < n_b) v.blk_owner_off[s] = carry + pre;
    carry += total;
  }
  if (threadIdx.x == 0) v.counters[kCntPairs] = carry;
}

__global__ void k_assign(StepView v) {
  __shared__ int sm[33];
  const int s = blockIdx.x;
  const int32_t b = v.sel[s];
  const int32_t q0 = v.blk_node_off[b], q1 = v.blk_node_off[b + 1];
  int carry = v.blk_owner_off[s];
  for (int32_t c = q0; c < q1; c += blockDim.x) {
    int32_t q = c + threadIdx.x;
    int own = (q < q1) && (v.owner_q[q] == q);
    int total;
    int pre = block_exscan(own, sm, &total);
    if (own) {
      int u = carry + pre;
      v.loc2u[q] = u;
      v.uniq_pair[u] = v.node_pair[q];
      v.uniq_q[u] = q;
      v.umulti[u] = v.multi[q];
    }
    carry += total;
  }
}

__global__ void k_link(StepView v) {
  const int32_t b = v.sel[blockIdx.x];
  const int32_t q0 = v.blk_node_off[b], q1 = v.blk_node_off[b + 1];
  for (int32_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    int32_t qo = v.owner_q[q];
    if (qo != q) v.loc2u[q] = v.loc2u[qo];
  }
}

// ------------------------------------------------------------------ residuals
// r_n = dt~_n - [(T_i - T_j) + (dt0_i - dt0_j)]  (Eq. 1; dt~ = dt - (t0_i - t0_j) of theta_0)
// and the whitening right-hand side u = B^T r (double-float), diag(lambda + B^T B) per node.
__global__ void k_resid(StepView v) {
  extern __shared__ float smf[];
  const int L_max = v.L_max;
  float* Thi = smf;
  float* Tlo = Thi + L_max;
  float* t0 = Tlo + L_max;
  float* rs = t0 + L_max;
  float* sw = rs + v.B;
  const int s = blockIdx.x;
  const int32_t b = v.sel[s];
  const int32_t q0 = v.blk_node_off[b];
  const int L = v.blk_node_off[b + 1] - q0;
  const int64_t e0 = v.blk_e0[b];
  const int ne = v.blk_e0[b + 1] - v.blk_e0[b];
  for (int l = threadIdx.x; l < L; l += blockDim.x) {
    const int32_t q = q0 + l;
    const float2 t = v.T2[v.loc2u[q]];
    Thi[l] = t.x;
    Tlo[l] = t.y;
    t0[l] = v.dth[v.pair_ev[v.node_pair[q]]].w;
  }
  for (int e = threadIdx.x; e < ne; e += blockDim.x) sw[e] = v.obs_sw[e0 + e];
  __syncthreads();
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    const uint32_t lij = v.obs_l[e0 + e];
    const int li = lij & 0xFFFF, lj = lij >> 16;
    const float dhi = Thi[li] - Thi[lj];
    const float dlo = Tlo[li] - Tlo[lj];
    const float dt0 = t0[li] - t0[lj];
    const float r = ((v.obs_dt[e0 + e] - dhi) - dt0) - dlo;
    rs[e] = r;
    v.r_obs[e0 + e] = r;
  }
  __syncthreads();
  if (!v.whiten) return;
  const uint16_t* he = v.blk_he + 2 * e0;
  for (int l = threadIdx.x; l < L; l += blockDim.x) {
    const int32_t q = q0 + l;
    const int h0 = v.node_he[q];
    const int h1 = (l + 1 < L) ? (int)v.node_he[q + 1] : 2 * ne;
    df32 a = {0.f, 0.f};
    float d = 0.f;
    for (int h = h0; h < h1; ++h) {
      const int code = he[h];
      const int e = code >> 1;
      const float w = sw[e];
      a = df_add(a, df_two_prod((code & 1) ? -w : w, rs[e]));
      d += w * w;
    }
    if (!v.multi[q]) {
      const int32_t u = v.loc2u[q];
      v.rhs[u] = a.hi;
      v.rhs_lo[u] = a.lo;
      v.diag[u] = v.lam + d;
      v.rowlen[u] = h1 - h0;
      v.occ_off[q] = 0;
    } else {
      v.part_a[q] = a.hi;
      v.part_c[q] = a.lo;
      v.part_b[q] = d;
    }
  }
}

// double-float sum over the selected occurrences of pair p (block order)
__device__ __forceinline__ df32 merge_occ_df(const StepView& v, int32_t p, int tag) {
  df32 a = {0.f, 0.f};
  for (int32_t t = v.inc_off[p], t1 = v.inc_off[p + 1]; t < t1; ++t)
    if (v.blk_stamp[v.inc_b[t]] == tag) {
      const int32_t qq = v.inc_q[t];
      a = df_add(a, df32{v.part_a[qq], v.part_c[qq]});
    }
  return a;
}

__global__ void k_merge_rhs(StepView v) {
  const int tag = v.prm->tag;
  const int32_t P_u = v.counters[kCntPairs];
  for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < P_u; u += gridDim.x * blockDim.x) {
    const int32_t q = v.uniq_q[u];
    if (!v.multi[q]) continue;
    const int32_t p = v.node_pair[q];
    const df32 a = merge_occ_df(v, p, tag);
    v.rhs[u] = a.hi;
    v.rhs_lo[u] = a.lo;
    v.diag[u] = v.lam + merge_occ(v, p, tag, v.part_b);
    int32_t run = 0;
    for (int32_t t = v.inc_off[p], t1 = v.inc_off[p + 1]; t < t1; ++t) {
      const int32_t bb = v.inc_b[t];
      if (v.blk_stamp[bb] != tag) continue;
      const int32_t qq = v.inc_q[t];
      const int32_t qb1 = v.blk_node_off[bb + 1];
      const int ne = v.blk_e0[bb + 1] - v.blk_e0[bb];
      const int h1 = (qq + 1 < qb1) ? (int)v.node_he[qq + 1] : 2 * ne;
      v.occ_off[qq] = run;
      run += h1 - (int)v.node_he[qq];
    }
    v.rowlen[u] = run;
  }
}

// ------------------------------------------------------------------ whitening
// Fixed-order sum of G partials (every CTA computes the same value).
__device__ float sum_partials(const float* part, int G, float* sm) {
  float a = 0.f;
  for (int i = threadIdx.x; i < G; i += blockDim.x) a += part[i];
  return block_sum<float>(a, sm);
}

struct BlockRange {
  int32_t q0;
  int L;
  int64_t e0;
  int ne;
};

__device__ __forceinline__ BlockRange block_range(const StepView& v, int64_t s) {
  BlockRange r;
  const int32_t b = v.sel[s];
  r.q0 = v.blk_node_off[b];
  r.L = v.blk_node_off[b + 1] - r.q0;
  r.e0 = v.blk_e0[b];
  r.ne = v.blk_e0[b + 1] - v.blk_e0[b];
  return r;
}

// ---- CSR of the merged minibatch matrix: row u = unique pair, entries in
// block order then half-edge order (so every sum below has a fixed order).
// Three-phase exclusive scan of src[0, n) into dst (dst[n] = total), n = *n_dev.
__global__ void k_scan_a(const int32_t* __restrict__ src, const int32_t* n_dev, int32_t* part,
                         const int32_t* gate) {
  __shared__ int sm[33];
  if (gate && *gate == 0) return;
  const int64_t n = *n_dev;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t a = blockIdx.x * chunk, b = a + chunk < n ? a + chunk : n;
  int acc = 0;
  for (int64_t u = a + threadIdx.x; u < b; u += blockDim.x) acc += src[u];
  acc = block_sum<int>(acc, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_scan_b(int32_t* part, int parts, const int32_t* gate) {
  __shared__ int sm[33];
  if (gate && *gate == 0) return;
  int carry = 0;
  for (int c = 0; c < parts; c += blockDim.x) {
    const int i = c + threadIdx.x;
    const int val = i < parts ? part[i] : 0;
    int total;
    const int pre = block_exscan(val, sm, &total);
    if (i < parts) part[i] = carry + pre;
    carry += total;
  }
  if (threadIdx.x == 0) part[parts] = carry;
}

__global__ void k_scan_c(const int32_t* src, const int32_t* n_dev, const int32_t* part, int32_t* dst,
                         const int32_t* gate) {
  __shared__ int sm[33];
  if (gate && *gate == 0) return;
  const int64_t n = *n_dev;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t a = blockIdx.x * chunk, b = a + chunk < n ? a + chunk : n;
  int carry = part[blockIdx.x];
  for (int64_t c = a; c < b; c += blockDim.x) {
    const int64_t u = c + threadIdx.x;
    const int val = u < b ? src[u] : 0;
    int total;
    const int pre = block_exscan(val, sm, &total);
    if (u < b) dst[u] = carry + pre;
    carry += total;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) dst[n] = part[gridDim.x];
}

// entries of every occurrence: neighbour's unique index and sqrt(w_e)
__global__ void k_fill_rows(StepView v) {
  if (gated_off(v)) return;
  const BlockRange br = block_range(v, blockIdx.x);
  const uint16_t* he = v.blk_he + 2 * br.e0;
  for (int l = threadIdx.x; l < br.L; l += blockDim.x) {
    const int32_t q = br.q0 + l;
    const int h0 = v.node_he[q];
    const int h1 = (l + 1 < br.L) ? (int)v.node_he[q + 1] : 2 * br.ne;
    const int32_t base = v.rowptr[v.loc2u[q]] + v.occ_off[q] - h0;
    for (int h = h0; h < h1; ++h) {
      const int code = he[h];
      const int e = code >> 1;
      const uint32_t lij = v.obs_l[br.e0 + e];
      const int other = (code & 1) ? (int)(lij & 0xFFFF) : (int)(lij >> 16);
      v.csr_col[base + h] = v.loc2u[br.q0 + other];
      v.csr_sw[base + h] = v.obs_sw[br.e0 + e];
    }
  }
}

// ---- connected components of the minibatch graph (rows = unique pairs,
// edges = CSR entries).  Labels converge to the smallest index of each
// component: roots are only ever hooked below smaller roots (atomicMin), so
// parent pointers strictly decrease and the fixed point is unique whatever
// the order of the atomics.  Rounds alternate hooking and full path
// compression until a round hooks nothing.
constexpr int kCcRounds = 64;
constexpr int kCompMax = 192;        // largest component solved by one warp
constexpr int kCompPad = 256;        // kCompMax rounded up to a power of two (sort padding)
constexpr int kCompEnt = 1280;       // largest CSR entry count cached by one warp
constexpr int kCtaMax = 1024;        // largest component solved by one CTA (larger: grid-wide CG)
constexpr int kCqBins = kCompMax + 1;   // work-list bins (see k_corder_scan)

__device__ __forceinline__ int32_t cc_root(const int32_t* lab, int32_t u) {
  const volatile int32_t* vl = lab;
  int32_t r = u;
  for (int k = 0; k < 1 << 20; ++k) {
    const int32_t n = vl[r];
    if (n == r) return r;
    r = n;
  }
  return r;
}

// Components inside each selected block first (its observations link its local
// nodes): min-label union-find in shared memory, one CTA per block.  Each local
// node then records its block-local root; the grid-wide rounds below only
// have to glue these stars together through pairs shared by several blocks.
__device__ __forceinline__ int lroot_find(const int* par, int x) {
  const volatile int* vp = par;
  for (int k = 0; k < 1 << 16; ++k) {
    const int p = vp[x];
    if (p == x) return x;
    x = p;
  }
  return x;
}

__global__ void k_cc_local(StepView v) {
  extern __shared__ int par[];
  __shared__ int changed;
  if (gated_off(v)) return;
  const int s = blockIdx.x;
  const int32_t b = v.sel[s];
  const int32_t q0 = v.blk_node_off[b];
  const int L = v.blk_node_off[b + 1] - q0;
  const int64_t e0 = v.blk_e0[b];
  const int ne = v.blk_e0[b + 1] - v.blk_e0[b];
  for (int l = threadIdx.x; l < L; l += blockDim.x) par[l] = l;
  __syncthreads();
  for (int round = 0; round < 64; ++round) {
    if (threadIdx.x == 0) changed = 0;
    __syncthreads();
    int mine = 0;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
      const uint32_t lij = v.obs_l[e0 + e];
      int a = lroot_find(par, (int)(lij & 0xFFFF)), c = lroot_find(par, (int)(lij >> 16));
      if (a == c) continue;
      const int lo = a < c ? a : c, hi = a < c ? c : a;
      if (atomicMin(&par[hi], lo) > lo) mine = 1;
    }
    if (mine) changed = 1;
    __syncthreads();
    // every thread takes the flag before the next round's reset can overwrite it
    const int any = changed;
    for (int l = threadIdx.x; l < L; l += blockDim.x) par[l] = lroot_find(par, l);
    __syncthreads();
    if (!any) break;
    if (round == 63 && threadIdx.x == 0) set_error(v.counters, SPIDER_E_TIMEOUT);
  }
  for (int l = threadIdx.x; l < L; l += blockDim.x) v.cc_lroot[q0 + l] = q0 + par[l];
}

__global__ void __launch_bounds__(512) k_cc(StepView v, int64_t n_b) {
  __shared__ int any;
  if (aborted_cta(v) || gated_off(v)) return;
  const int32_t P_u = v.counters[kCntPairs];
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gstride = gridDim.x * blockDim.x;
  int32_t* flags = v.scan_part;          // one flag per round
  for (int32_t u = gtid; u < P_u; u += gstride) {
    v.lab[u] = u;
    v.ccount[u] = 0;
  }
  for (int i = gtid; i < kCcRounds; i += gstride) flags[i] = 0;
  for (int i = gtid; i < kCqBins + 4; i += gstride) v.chist[i] = 0;
  if (!grid_barrier(v.counters, v.prm->wait_ns)) return;
  int round = 0;
  for (; round < kCcRounds; ++round) {
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    int changed = 0;
    // one link per local node of every selected block: (its pair, its block root's pair)
    for (int64_t sb = blockIdx.x; sb < n_b; sb += gridDim.x) {
      const int32_t b = v.sel[sb];
      const int32_t q0 = v.blk_node_off[b], L = v.blk_node_off[b + 1] - q0;
      for (int l = threadIdx.x; l < L; l += blockDim.x) {
        const int32_t q = q0 + l, rq = v.cc_lroot[q];
        if (rq == q) continue;
        const int32_t ru = cc_root(v.lab, v.loc2u[q]), rc = cc_root(v.lab, v.loc2u[rq]);
        if (rc == ru) continue;
        const int32_t lo = rc < ru ? rc : ru, hi = rc < ru ? ru : rc;
        if (atomicMin(&v.lab[hi], lo) > lo) changed = 1;
      }
    }
    if (changed) any = 1;
    __syncthreads();
    if (threadIdx.x == 0 && any) flags[round] = 1;
    if (!grid_barrier(v.counters, v.prm->wait_ns)) return;
    for (int32_t u = gtid; u < P_u; u += gstride) v.lab[u] = cc_root(v.lab, u);
    if (!grid_barrier(v.counters, v.prm->wait_ns)) return;
    if (((volatile int32_t*)flags)[round] == 0) break;
  }
  if (round == kCcRounds) {
    if (gtid == 0) set_error(v.counters, SPIDER_E_TIMEOUT);
    return;
  }
  // member counts per root; root flags for the compaction scan
  for (int32_t u = gtid; u < P_u; u += gstride) {
    const int32_t r = v.lab[u];
    atomicAdd(&v.ccount[r], 1);
    v.cslot[u] = (r == u) ? 1 : 0;
  }
}

// roots (ascending) -> component index; sizes in component order
__global__ void k_cc_roots(StepView v) {
  if (aborted(v) || gated_off(v)) return;
  const int32_t P_u = v.counters[kCntPairs];
  for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < P_u; u += gridDim.x * blockDim.x) {
    if (v.lab[u] != u) continue;
    const int32_t c = v.members[u];          // exclusive scan of root flags (held in members)
    v.comp_root[c] = u;
    v.comp_off[c] = v.ccount[u];             // size, scanned in place next
    v.centries[c] = 0;
    v.cslot[u] = c;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) v.counters[kCntComps] = v.members[P_u];
}

// member lists (arbitrary order inside a component; the solver sorts them)
__global__ void k_cc_fill(StepView v) {
  if (aborted(v) || gated_off(v)) return;
  const int32_t P_u = v.counters[kCntPairs];
  for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < P_u; u += gridDim.x * blockDim.x) {
    const int32_t r = v.lab[u];
    const int32_t c = v.cslot[r];
    const int32_t size = v.comp_off[c + 1] - v.comp_off[c];
    const int32_t pos = atomicSub(&v.ccount[r], 1) - 1;
    v.lidx[u] = v.comp_off[c] + pos;          // slot in the member array
    (void)size;
    atomicAdd(&v.centries[c], v.rowlen[u]);
  }
}

// members into place; solver tier per component: one warp (n <= kCompMax and
// entries <= kCompEnt), one CTA (n <= kCtaMax), else the grid-wide solver
__global__ void k_cc_place(StepView v) {
  if (aborted(v) || gated_off(v)) return;
  const int32_t P_u = v.counters[kCntPairs];
  for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < P_u; u += gridDim.x * blockDim.x) {
    v.members[v.lidx[u]] = u;
    const int32_t c = v.cslot[v.lab[u]];
    const int32_t n = v.comp_off[c + 1] - v.comp_off[c];
    const int tier = (n <= kCompMax && v.centries[c] <= kCompEnt) ? 0 : (n <= kCtaMax ? 1 : 2);
    v.big[u] = tier == 2 ? 1 : 0;
    v.bigpos[u] = tier == 2 ? 1 : 0;
    if (u == v.comp_root[c]) {
      v.ctier[c] = (uint8_t)tier;
      if (tier < 2) atomicAdd(&v.chist[tier == 1 ? 0 : 1 + (kCompMax - n)], 1);
    }
  }
}

// the nodes of the grid-tier components as a list in pair order (bigpos holds
// their exclusive prefix)
__global__ void k_big_list(StepView v) {
  if (aborted(v) || gated_off(v)) return;
  const int32_t P_u = v.counters[kCntPairs];
  for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < P_u; u += gridDim.x * blockDim.x)
    if (v.big[u]) v.biglist[v.bigpos[u]] = u;
}

__device__ __forceinline__ float warp_allsum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__device__ void warp_sort(int32_t* a, int n2, int lane) {
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < n2; i += 32) {
        const int l = i ^ j;
        if (l > i) {
          const int32_t x = a[i], y = a[l];
          const bool up = (i & k) == 0;
          if ((x > y) == up) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      __syncwarp();
    }
}

// Two-value block reduction with one barrier: partials go to one of two
// alternating buffers and every warp adds them up in the same order, so all
// threads get the same (deterministic) sums.
__device__ __forceinline__ float2 block_sum2(float a, float b, float2* sm /* 2 x 32 */, int& par) {
  a = warp_allsum(a);
  b = warp_allsum(b);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float2* buf = sm + 32 * par;
  if (lane == 0) buf[wid] = make_float2(a, b);
  __syncthreads();
  float2 s = make_float2(0.f, 0.f);
  for (int k = 0; k < nw; ++k) {
    const float2 t = buf[k];
    s.x += t.x;
    s.y += t.y;
  }
  par ^= 1;
  return s;
}

// Largest i with a[i] <= x for a sorted ascending, padded to n2 (a power of
// two) with INT32_MAX, and a[0] <= x.
__device__ __forceinline__ int bsearch_le(const int32_t* a, int n2, int32_t x) {
  int i = 0;
  for (int s = n2 >> 1; s > 0; s >>= 1)
    if (a[i + s] <= x) i += s;
  return i;
}

// Work list of the component solvers: the CTA tier first, then the warp tier by
// decreasing size, so that the dynamic schedule starts the longest solves
// first.  chist holds kCqBins counters (bin 0: CTA tier; bin 1 + kCompMax - n:
// warp tier of size n), then [kCqBins] CTA cursor, [+1] warp cursor, [+2] start
// of the warp tier, [+3] end of the list.
__global__ void k_corder_scan(StepView v) {
  __shared__ int sm[33];
  if (aborted_cta(v) || gated_off(v)) return;
  int carry = 0;
  for (int c = 0; c < kCqBins; c += blockDim.x) {
    const int b = c + threadIdx.x;
    const int val = b < kCqBins ? v.chist[b] : 0;
    int total;
    const int pre = block_exscan(val, sm, &total);
    __syncthreads();
    if (b < kCqBins) v.chist[b] = carry + pre;
    carry += total;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    v.chist[kCqBins] = 0;
    v.chist[kCqBins + 1] = 0;
    v.chist[kCqBins + 2] = v.chist[1];
    v.chist[kCqBins + 3] = carry;
  }
}

__global__ void k_corder_fill(StepView v) {
  if (aborted(v) || gated_off(v)) return;
  const int32_t ncomp = v.counters[kCntComps];
  for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncomp; c += gridDim.x * blockDim.x) {
    const int tier = v.ctier[c];
    if (tier > 1) continue;
    const int n = v.comp_off[c + 1] - v.comp_off[c];
    const int bin = tier == 1 ? 0 : 1 + (kCompMax - n);
    v.corder[atomicAdd(&v.chist[bin], 1)] = c;
  }
}

// One warp per component of at most kCompMax nodes and kCompEnt CSR entries,
// taken from the work list.  Members are sorted first so that every sum runs in
// a fixed order; the component's CSR is cached in shared memory with local
// column indices.  Up to kDenseMax nodes (and kDenseEnt entries) the matrix is
// factorised (dense Cholesky, FP32) and z refined with the double-float
// residual; otherwise (or when the factorisation fails) the same refinement
// takes Jacobi-CG corrections to 1e-3.
constexpr int kCompWarps = 2;
constexpr int kDenseMax = 64;
constexpr int kDenseEnt = 640;
constexpr int kDenseSlots = (kDenseMax + 31) / 32;

static_assert(kCompPad >= kCompMax && kCompPad <= 2 * kCompMax, "sort padding of the warp tier");

struct WarpSmem {
  int32_t mu[kCompPad];              // sorted members, padded to a power of two
  int32_t lrp[kCompPad + 1];         // local row pointers, padded
  uint8_t perm[kCompMax];            // iterative path: rows by decreasing length
  union {
    struct {
      float vec[8][kCompMax];        // zh, zl, diag, res, y, p, Ap, dz (row starts while loading)
      float lsw[kCompEnt];
      uint8_t lcol[kCompEnt];
    } it;
    struct {
      float L[kDenseMax * (kDenseMax + 1) / 2];   // packed lower triangle, column-major
      float zh[kDenseMax], zl[kDenseMax], rdiag[kDenseMax];
      int32_t rp0[kDenseMax];
      float lsw[kDenseEnt];
      uint8_t lcol[kDenseEnt];
    } dn;
  };
};

// Sorted members and the component's local CSR: row pointers by a warp scan of
// the row lengths, then every entry (in parallel) its neighbour's local index.
__device__ int warp_load_comp(const StepView& v, int32_t off, int n, int n2, int32_t* mu, int32_t* lrp,
                              int32_t* rp0, uint8_t* lcol, float* lsw, int lane) {
  for (int i = lane; i < n2; i += 32) mu[i] = i < n ? v.members[off + i] : 0x7FFFFFFF;
  __syncwarp();
  warp_sort(mu, n2, lane);
  int carry = 0;
  for (int base = 0; base < n; base += 32) {
    const int i = base + lane;
    int len = 0;
    if (i < n) {
      const int32_t u = mu[i];
      const int32_t r0 = v.rowptr[u];
      len = v.rowptr[u + 1] - r0;
      rp0[i] = r0;
    }
    int x = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (i < n) lrp[i] = carry + x - len;
    carry += __shfl_sync(0xffffffffu, x, 31);
  }
  for (int i = n + 1 + lane; i < n2; i += 32) lrp[i] = 0x7FFFFFFF;
  if (lane == 0) lrp[n] = carry;
  __syncwarp();
  const int E = carry;
  for (int e0 = 0; e0 < E; e0 += 4 * 32) {
    int32_t col[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = e0 + 32 * q + lane;
      col[q] = 0;
      if (e < E) {
        const int row = bsearch_le(lrp, n2, e);
        const int32_t t = rp0[row] + (e - lrp[row]);
        col[q] = v.csr_col[t];
        if (lsw) lsw[e] = v.csr_sw[t];
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = e0 + 32 * q + lane;
      if (e < E) lcol[e] = (uint8_t)bsearch_le(mu, n2, col[q]);
    }
  }
  __syncwarp();
  return E;
}

// Dense path: A = lambda I + B^T B assembled into the packed lower triangle
// (column-major: column j holds rows j..n-1 from j n - j (j - 1) / 2, so that
// lanes over rows read consecutive words), factorised A = L L^T left-looking:
// column j is A(:, j) minus the dot products of the finished columns, each lane
// one row (two interleaved partial sums), the pivot from a running sum of
// squares per row.  z is then refined: residual in double-float, correction by
// the two triangular solves (rows held in registers, the pivot broadcast by
// shuffle).  NS is the number of 32-row slots (n <= 32 NS).  Returns the
// refinement rounds, or -1 when a pivot is not positive or the refinement
// stalls (z is then unusable).
__device__ __forceinline__ int cm_off(int j, int n) { return j * n - (j * (j - 1)) / 2; }

// rows i = j + 1 + lane + 32 s (s < NA) of column j: sum over p < j of L(i, p) L(j, p)
template <int NA>
__device__ __forceinline__ void dense_col_dots(const float* L, int n, int j, int lane, float* out) {
  float a0[NA], a1[NA], a2[NA], a3[NA];
  int ro[NA];
#pragma unroll
  for (int s = 0; s < NA; ++s) {
    a0[s] = a1[s] = a2[s] = a3[s] = 0.f;
    const int i = j + 1 + lane + 32 * s;
    ro[s] = i < n ? i : j;            // rows past the end read row j (in bounds) and are dropped
  }
  int cb = 0;                         // column p starts at cb + p
  int p = 0;
  // four columns per pass (four independent partial sums)
  for (; p + 3 < j; p += 4) {
    const int cb1 = cb + n - p - 1, cb2 = cb1 + n - p - 2, cb3 = cb2 + n - p - 3;
    const float l0 = L[cb + j], l1 = L[cb1 + j], l2 = L[cb2 + j], l3 = L[cb3 + j];
#pragma unroll
    for (int s = 0; s < NA; ++s) {
      a0[s] = fmaf(L[cb + ro[s]], l0, a0[s]);
      a1[s] = fmaf(L[cb1 + ro[s]], l1, a1[s]);
      a2[s] = fmaf(L[cb2 + ro[s]], l2, a2[s]);
      a3[s] = fmaf(L[cb3 + ro[s]], l3, a3[s]);
    }
    cb = cb3 + n - p - 4;
  }
  for (; p < j; ++p) {
    const float l0 = L[cb + j];
#pragma unroll
    for (int s = 0; s < NA; ++s) a0[s] = fmaf(L[cb + ro[s]], l0, a0[s]);
    cb += n - p - 1;
  }
#pragma unroll
  for (int s = 0; s < NA; ++s) out[s] = (a0[s] + a1[s]) + (a2[s] + a3[s]);
}

template <int NS>
__device__ int warp_dense_solve(const StepView& v, WarpSmem& S, int n, float tol, int lane) {
  auto& D = S.dn;
  float* L = D.L;
  float* sq = D.zh;                   // sum of squares of each row's finished entries
  const float lam = v.lam;
  const int tot = n * (n + 1) / 2;
  for (int t = lane; t < tot; t += 32) L[t] = 0.f;
  __syncwarp();
  for (int i = lane; i < n; i += 32) {
    L[cm_off(i, n)] = v.diag[S.mu[i]];
    sq[i] = 0.f;
    for (int l = S.lrp[i], l1 = S.lrp[i + 1]; l < l1; ++l) {
      const int lc = D.lcol[l];
      if (lc < i) {
        const float sw = D.lsw[l];
        float* a = L + cm_off(lc, n) + (i - lc);
        *a = fmaf(-sw, sw, *a);
      }
    }
  }
  __syncwarp();
  for (int j = 0; j < n; ++j) {
    const int cj = cm_off(j, n);
    const float d = L[cj] - sq[j];
    if (!(d > 0.f)) return -1;
    const float ljj = sqrtf(d);
    const float inv = 1.0f / ljj;
    const int na = (n - j + 30) >> 5;   // slots holding rows j+1..n-1
    float dots[NS];
    if (NS >= 3 && na >= 3) dense_col_dots<NS >= 3 ? 3 : 1>(L, n, j, lane, dots);
    else if (NS >= 2 && na == 2) dense_col_dots<NS >= 2 ? 2 : 1>(L, n, j, lane, dots);
    else if (na == 1) dense_col_dots<1>(L, n, j, lane, dots);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const int i = j + 1 + lane + 32 * s;
      if (s < na && i < n) {
        const float lij = (L[cj + i - j] - dots[s]) * inv;
        L[cj + i - j] = lij;
        sq[i] = fmaf(lij, lij, sq[i]);
      }
    }
    if (lane == 0) {
      L[cj] = ljj;
      D.rdiag[j] = inv;
    }
    __syncwarp();
  }
  float bb = 0.f;
  for (int i = lane; i < n; i += 32) {
    const float b = v.rhs[S.mu[i]];
    bb = fmaf(b, b, bb);
    D.zh[i] = 0.f;
    D.zl[i] = 0.f;
  }
  bb = warp_allsum(bb);
  __syncwarp();
  if (!(bb > 0.f)) return 0;
  int rowb[NS];                       // L(q, i) = L[rowb + q] for i < q
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const int i = lane + 32 * s;
    rowb[s] = cm_off(i, n) - i;
  }
  float prev = 0.f;
  for (int round = 0; round < 10; ++round) {
    float rr = 0.f;
    float yr[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const int i = lane + 32 * s;
      yr[s] = 0.f;
      if (i >= n) continue;
      const int32_t u = S.mu[i];
      float r;
      if (round == 0) {
        r = v.rhs[u] + v.rhs_lo[u];
      } else {
        const df32 zu = {D.zh[i], D.zl[i]};
        df32 acc = {0.f, 0.f};
        for (int l = S.lrp[i], l1 = S.lrp[i + 1]; l < l1; ++l) {
          const int lc = D.lcol[l];
          const float sw = D.lsw[l];
          acc = df_add(acc, df_mul(df_two_prod(sw, sw), df_add(zu, df32{-D.zh[lc], -D.zl[lc]})));
        }
        df32 rd = df_add(df32{v.rhs[u], v.rhs_lo[u]}, df_mul_f(zu, -lam));
        rd = df_add(rd, df32{-acc.hi, -acc.lo});
        r = rd.hi;
      }
      yr[s] = r;
      rr = fmaf(r, r, rr);
    }
    rr = warp_allsum(rr);
    if (rr <= tol * tol * bb) return round;
    if (round > 0 && !(rr < 0.25f * prev)) return -1;
    prev = rr;
    // L w = r (column sweep: column p is contiguous)
    int cp = 0;
    for (int p = 0; p < n; ++p) {
      const int sp = p >> 5;
      float mine = yr[0];
#pragma unroll
      for (int s = 1; s < NS; ++s) mine = sp == s ? yr[s] : mine;
      const float wp = __shfl_sync(0xffffffffu, mine, p & 31) * D.rdiag[p];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const int i = lane + 32 * s;
        if (i == p) yr[s] = wp;
        else if (i > p && i < n) yr[s] = fmaf(-L[cp + i - p], wp, yr[s]);
      }
      cp += n - p;
    }
    // L^T d = w
    for (int q = n - 1; q >= 0; --q) {
      const int sq_ = q >> 5;
      float mine = yr[0];
#pragma unroll
      for (int s = 1; s < NS; ++s) mine = sq_ == s ? yr[s] : mine;
      const float dq = __shfl_sync(0xffffffffu, mine, q & 31) * D.rdiag[q];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const int i = lane + 32 * s;
        if (i == q) yr[s] = dq;
        else if (i < q) yr[s] = fmaf(-L[rowb[s] + q], dq, yr[s]);
      }
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const int i = lane + 32 * s;
      if (i < n) {
        const df32 zn = df_add_f(df32{D.zh[i], D.zl[i]}, yr[s]);
        D.zh[i] = zn.hi;
        D.zl[i] = zn.lo;
      }
    }
    __syncwarp();
  }
  return -1;
}

__global__ void __launch_bounds__(kCompWarps * 32) k_comp_solve(StepView v, int max_it, float tol) {
  extern __shared__ __align__(16) uint8_t smem_w[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpSmem& S = reinterpret_cast<WarpSmem*>(smem_w)[w];
  const float lam = v.lam;
  int32_t* mu = S.mu;
  float* zh = S.it.vec[0];
  float* zl = S.it.vec[1];
  float* dg = S.it.vec[2];
  float* rs = S.it.vec[3];
  float* yv = S.it.vec[4];
  float* pv = S.it.vec[5];
  float* ap = S.it.vec[6];
  float* dz = S.it.vec[7];
  if (aborted(v) || gated_off(v)) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    return;
  }
  const int32_t w_beg = v.chist[kCqBins + 2], w_end = v.chist[kCqBins + 3];
  int max_iters = 0;
  for (;;) {
    int32_t k = 0;
    if (lane == 0) k = atomicAdd(&v.chist[kCqBins + 1], 1);
    k = __shfl_sync(0xffffffffu, k, 0) + w_beg;
    if (k >= w_end) break;
    const int32_t c = v.corder[k];
    const int32_t off = v.comp_off[c];
    const int n = v.comp_off[c + 1] - off;
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    if (n <= kDenseMax && v.centries[c] <= kDenseEnt) {
      warp_load_comp(v, off, n, n2, mu, S.lrp, S.dn.rp0, S.dn.lcol, S.dn.lsw, lane);
      const int rounds = n <= 32   ? warp_dense_solve<1>(v, S, n, tol, lane)
                         : n <= 64 ? warp_dense_solve<2>(v, S, n, tol, lane)
                                   : warp_dense_solve<kDenseSlots>(v, S, n, tol, lane);
      __syncwarp();
      if (rounds >= 0) {
        for (int i = lane; i < n; i += 32) {
          v.z[mu[i]] = S.dn.zh[i];
          v.z_lo[mu[i]] = S.dn.zl[i];
        }
        __syncwarp();
        continue;
      }
    }
    // iterative path (row starts in dz while loading)
    warp_load_comp(v, off, n, n2, mu, S.lrp, reinterpret_cast<int32_t*>(dz), S.it.lcol, S.it.lsw, lane);
    {
      // row order by decreasing length, so that the lanes of a 32-row slot
      // run inner loops of similar trip counts
      // n2 <= kCompPad <= 2 kCompMax entries: vec[3] continues into vec[4] (unused yet)
      int32_t* key = reinterpret_cast<int32_t*>(S.it.vec[3]);
      for (int i = lane; i < n2; i += 32) key[i] = i < n ? ((S.lrp[i + 1] - S.lrp[i]) << 8 | i) : -1;
      __syncwarp();
      warp_sort(key, n2, lane);
      for (int r = lane; r < n; r += 32) S.perm[r] = (uint8_t)(key[n2 - 1 - r] & 255);
      __syncwarp();
    }
    for (int i = lane; i < n; i += 32) {
      zh[i] = 0.f;
      zl[i] = 0.f;
      dg[i] = v.diag[mu[i]];
    }
    __syncwarp();
    float bb = 0.f;
    for (int i = lane; i < n; i += 32) {
      const float b = v.rhs[mu[i]];
      bb = fmaf(b, b, bb);
    }
    bb = warp_allsum(bb);
    const float outer_thr = tol * tol * bb;
    int it = 0;
    for (int round = 0; round < 8 && bb > 0.f && it < max_it; ++round) {
      float rz = 0.f, rr0 = 0.f;
      for (int r_ = lane; r_ < n; r_ += 32) {
        const int i = S.perm[r_];
        const int32_t u = mu[i];
        float r;
        if (round == 0) {
          r = v.rhs[u] + v.rhs_lo[u];
        } else {
          const df32 zu = {zh[i], zl[i]};
          df32 acc = {0.f, 0.f};
          for (int l = S.lrp[i], l1 = S.lrp[i + 1]; l < l1; ++l) {
            const int lc = S.it.lcol[l];
            const float sw = S.it.lsw[l];
            acc = df_add(acc, df_mul(df_two_prod(sw, sw), df_add(zu, df32{-zh[lc], -zl[lc]})));
          }
          df32 rd = df_add(df32{v.rhs[u], v.rhs_lo[u]}, df_mul_f(zu, -lam));
          rd = df_add(rd, df32{-acc.hi, -acc.lo});
          r = rd.hi;
        }
        const float y = r / dg[i];
        rs[i] = r;
        yv[i] = y;
        dz[i] = 0.f;
        rz = fmaf(r, y, rz);
        rr0 = fmaf(r, r, rr0);
      }
      rz = warp_allsum(rz);
      rr0 = warp_allsum(rr0);
      __syncwarp();
      if (rr0 <= outer_thr) break;
      const float inner_thr = 1e-6f * rr0;
      float beta = 0.f;
      bool first = true;
      while (it < max_it) {
        float dot = 0.f;
        for (int r_ = lane; r_ < n; r_ += 32) {
          const int i = S.perm[r_];
          const float yu = yv[i];
          float sacc = 0.f;
          for (int l = S.lrp[i], l1 = S.lrp[i + 1]; l < l1; ++l) {
            const float sw = S.it.lsw[l];
            sacc = fmaf(sw * sw, yu - yv[S.it.lcol[l]], sacc);
          }
          const float ay = fmaf(lam, yu, sacc);
          const float pn = first ? yu : fmaf(beta, pv[i], yu);
          const float apn = first ? ay : fmaf(beta, ap[i], ay);
          pv[i] = pn;
          ap[i] = apn;
          dot = fmaf(pn, apn, dot);
        }
        const float pap = warp_allsum(dot);
        const float alpha = pap > 0.f ? rz / pap : 0.f;
        float rzn = 0.f, rr = 0.f;
        __syncwarp();
        for (int r_ = lane; r_ < n; r_ += 32) {
          const int i = S.perm[r_];
          dz[i] = fmaf(alpha, pv[i], dz[i]);
          const float r = fmaf(-alpha, ap[i], rs[i]);
          rs[i] = r;
          const float y = r / dg[i];
          yv[i] = y;
          rzn = fmaf(r, y, rzn);
          rr = fmaf(r, r, rr);
        }
        rzn = warp_allsum(rzn);
        rr = warp_allsum(rr);
        __syncwarp();
        ++it;
        if (rr <= inner_thr || !(pap > 0.f)) break;
        beta = rzn / rz;
        rz = rzn;
        first = false;
      }
      for (int i = lane; i < n; i += 32) {
        const df32 zn = df_add_f(df32{zh[i], zl[i]}, dz[i]);
        zh[i] = zn.hi;
        zl[i] = zn.lo;
      }
      __syncwarp();
    }
    for (int i = lane; i < n; i += 32) {
      v.z[mu[i]] = zh[i];
      v.z_lo[mu[i]] = zl[i];
    }
    __syncwarp();
    if (it > max_iters) max_iters = it;
  }
  if (lane == 0 && max_iters > 0) atomicMax(&v.counters[kCntCompIters], max_iters);
  // the CTA tier (launched before this kernel) is complete and visible once this returns
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// One CTA per component of more than kCompMax (or kCompEnt entries) and at most
// kCtaMax nodes, taken from the work list.  Up to kCtaSm nodes and kCtaSmEnt
// entries the component's CSR and vectors live in shared memory (local column
// indices, two-value reductions with one barrier); larger components keep
// their vectors in global memory, indexed by unique pair.
constexpr int kCtaThreads = 256;
constexpr int kCtaSm = 1024;
constexpr int kCtaSmEnt = 11264;

struct CtaSmem {
  int32_t mu[kCtaSm];
  int32_t lrp[kCtaSm + 4];
  float vec[8][kCtaSm];             // zh, zl, diag, res, y, p, Ap, dz (row starts while loading)
  float lsw[kCtaSmEnt];
  uint16_t lcol[kCtaSmEnt];
  uint16_t perm[kCtaSm];            // rows by decreasing length
};
static_assert(sizeof(CtaSmem) >= kCtaMax * sizeof(int32_t), "member sort buffer");

__device__ void cta_sort(int32_t* mu, int n2) {
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const int32_t x = mu[i], y = mu[l];
          const bool up = (i & k) == 0;
          if ((x > y) == up) {
            mu[i] = y;
            mu[l] = x;
          }
        }
      }
      __syncthreads();
    }
}

// shared-memory CTA solve; returns the inner iterations
__device__ int cta_solve_smem(const StepView& v, CtaSmem& S, int32_t off, int n, int n2, int max_it, float tol,
                              float2* red2, int* smi) {
  const float lam = v.lam;
  const int tid = threadIdx.x, nt = blockDim.x;
  int32_t* mu = S.mu;
  float* zh = S.vec[0];
  float* zl = S.vec[1];
  float* dg = S.vec[2];
  float* rs = S.vec[3];
  float* yv = S.vec[4];
  float* pv = S.vec[5];
  float* ap = S.vec[6];
  float* dz = S.vec[7];
  int32_t* rp0 = reinterpret_cast<int32_t*>(dz);
  for (int i = tid; i < n2; i += nt) mu[i] = i < n ? v.members[off + i] : 0x7FFFFFFF;
  __syncthreads();
  cta_sort(mu, n2);
  int carry = 0;
  for (int base = 0; base < n; base += nt) {
    const int i = base + tid;
    int len = 0;
    if (i < n) {
      const int32_t u = mu[i];
      const int32_t r0 = v.rowptr[u];
      len = v.rowptr[u + 1] - r0;
      rp0[i] = r0;
    }
    int total;
    const int pre = block_exscan(len, smi, &total);
    if (i < n) S.lrp[i] = carry + pre;
    carry += total;
  }
  for (int i = n + 1 + tid; i < n2; i += nt) S.lrp[i] = 0x7FFFFFFF;
  if (tid == 0) S.lrp[n] = carry;
  __syncthreads();
  const int E = carry;
  for (int e = tid; e < E; e += nt) {
    const int row = bsearch_le(S.lrp, n2, e);
    const int32_t t = rp0[row] + (e - S.lrp[row]);
    S.lsw[e] = v.csr_sw[t];
    S.lcol[e] = (uint16_t)bsearch_le(mu, n2, v.csr_col[t]);
  }
  {
    int32_t* key = reinterpret_cast<int32_t*>(rs);
    for (int i = tid; i < n2; i += nt) key[i] = i < n ? ((S.lrp[i + 1] - S.lrp[i]) << 10 | i) : -1;
    __syncthreads();
    cta_sort(key, n2);
    for (int r = tid; r < n; r += nt) S.perm[r] = (uint16_t)(key[n2 - 1 - r] & 1023);
  }
  __syncthreads();
  int par = 0;
  float bb = 0.f;
  for (int i = tid; i < n; i += nt) {
    const float b = v.rhs[mu[i]];
    bb = fmaf(b, b, bb);
    zh[i] = 0.f;
    zl[i] = 0.f;
    dg[i] = v.diag[mu[i]];
  }
  bb = block_sum2(bb, 0.f, red2, par).x;
  const float outer_thr = tol * tol * bb;
  int it = 0;
  for (int round = 0; round < 8 && bb > 0.f && it < max_it; ++round) {
    float rz = 0.f, rr0 = 0.f;
    for (int r_ = tid; r_ < n; r_ += nt) {
      const int i = S.perm[r_];
      const int32_t u = mu[i];
      float r;
      if (round == 0) {
        r = v.rhs[u] + v.rhs_lo[u];
      } else {
        const df32 zu = {zh[i], zl[i]};
        df32 acc = {0.f, 0.f};
        for (int l = S.lrp[i], l1 = S.lrp[i + 1]; l < l1; ++l) {
          const int lc = S.lcol[l];
          const float sw = S.lsw[l];
          acc = df_add(acc, df_mul(df_two_prod(sw, sw), df_add(zu, df32{-zh[lc], -zl[lc]})));
        }
        df32 rd = df_add(df32{v.rhs[u], v.rhs_lo[u]}, df_mul_f(zu, -lam));
        rd = df_add(rd, df32{-acc.hi, -acc.lo});
        r = rd.hi;
      }
      const float y = r / dg[i];
      rs[i] = r;
      yv[i] = y;
      dz[i] = 0.f;
      rz = fmaf(r, y, rz);
      rr0 = fmaf(r, r, rr0);
    }
    const float2 s0 = block_sum2(rz, rr0, red2, par);
    rz = s0.x;
    if (s0.y <= outer_thr) break;
    const float inner_thr = 1e-6f * s0.y;
    float beta = 0.f;
    bool first = true;
    while (it < max_it) {
      float dot = 0.f;
      for (int r_ = tid; r_ < n; r_ += nt) {
        const int i = S.perm[r_];
        const float yu = yv[i];
        float sacc = 0.f;
        for (int l = S.lrp[i], l1 = S.lrp[i + 1]; l < l1; ++l) {
          const float sw = S.lsw[l];
          sacc = fmaf(sw * sw, yu - yv[S.lcol[l]], sacc);
        }
        const float ay = fmaf(lam, yu, sacc);
        const float pn = first ? yu : fmaf(beta, pv[i], yu);
        const float apn = first ? ay : fmaf(beta, ap[i], ay);
        pv[i] = pn;
        ap[i] = apn;
        dot = fmaf(pn, apn, dot);
      }
      const float pap = block_sum2(dot, 0.f, red2, par).x;
      const float alpha = pap > 0.f ? rz / pap : 0.f;
      float rzn = 0.f, rr = 0.f;
      for (int r_ = tid; r_ < n; r_ += nt) {
        const int i = S.perm[r_];
        dz[i] = fmaf(alpha, pv[i], dz[i]);
        const float r = fmaf(-alpha, ap[i], rs[i]);
        rs[i] = r;
        const float y = r / dg[i];
        yv[i] = y;
        rzn = fmaf(r, y, rzn);
        rr = fmaf(r, r, rr);
      }
      const float2 s1 = block_sum2(rzn, rr, red2, par);
      ++it;
      if (s1.y <= inner_thr || !(pap > 0.f)) break;
      beta = s1.x / rz;
      rz = s1.x;
      first = false;
    }
    for (int i = tid; i < n; i += nt) {
      const df32 zn = df_add_f(df32{zh[i], zl[i]}, dz[i]);
      zh[i] = zn.hi;
      zl[i] = zn.lo;
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += nt) {
    v.z[mu[i]] = zh[i];
    v.z_lo[mu[i]] = zl[i];
  }
  return it;
}

__global__ void __launch_bounds__(kCtaThreads) k_comp_solve_cta(StepView v, int max_it, float tol) {
  extern __shared__ __align__(16) uint8_t smem_c[];
  CtaSmem& S = *reinterpret_cast<CtaSmem*>(smem_c);
  __shared__ float smr[33];
  __shared__ float2 red2[64];
  __shared__ int smi[33];
  __shared__ int32_t s_k;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (aborted_cta(v) || gated_off(v)) return;
  const float lam = v.lam;
  const int32_t c_end = v.chist[kCqBins + 2];
  int max_iters = 0;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_k = atomicAdd(&v.chist[kCqBins], 1);
    __syncthreads();
    const int32_t k = s_k;
    if (k >= c_end) break;
    const int32_t c = v.corder[k];
    const int32_t off = v.comp_off[c];
    const int n = v.comp_off[c + 1] - off;
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    if (n <= kCtaSm && v.centries[c] <= kCtaSmEnt) {
      const int it = cta_solve_smem(v, S, off, n, n2, max_it, tol, red2, smi);
      if (it > max_iters) max_iters = it;
      continue;
    }
    int32_t* mu = reinterpret_cast<int32_t*>(smem_c);
    for (int i = threadIdx.x; i < n2; i += blockDim.x) mu[i] = i < n ? v.members[off + i] : 0x7FFFFFFF;
    __syncthreads();
    cta_sort(mu, n2);
    float bb = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int32_t u = mu[i];
      const float b = v.rhs[u];
      v.z[u] = 0.f;
      v.z_lo[u] = 0.f;
      bb = fmaf(b, b, bb);
    }
    bb = block_sum<float>(bb, smr);
    const float outer_thr = tol * tol * bb;
    int it = 0;
    for (int round = 0; round < 8 && bb > 0.f && it < max_it; ++round) {
      float rz = 0.f, rr0 = 0.f;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int32_t u = mu[i];
        float r;
        if (round == 0) {
          r = v.rhs[u] + v.rhs_lo[u];
        } else {
          const df32 zu = {v.z[u], v.z_lo[u]};
          df32 acc = {0.f, 0.f};
          for (int32_t t = v.rowptr[u], t1 = v.rowptr[u + 1]; t < t1; ++t) {
            const int32_t cc = v.csr_col[t];
            const float sw = v.csr_sw[t];
            acc = df_add(acc, df_mul(df_two_prod(sw, sw), df_add(zu, df32{-v.z[cc], -v.z_lo[cc]})));
          }
          df32 rd = df_add(df32{v.rhs[u], v.rhs_lo[u]}, df_mul_f(zu, -lam));
          rd = df_add(rd, df32{-acc.hi, -acc.lo});
          r = rd.hi;
        }
        const float y = r / v.diag[u];
        v.res[u] = r;
        v.yv[u] = y;
        v.dz[u] = 0.f;
        rz = fmaf(r, y, rz);
        rr0 = fmaf(r, r, rr0);
      }
      rz = block_sum<float>(rz, smr);
      rr0 = block_sum<float>(rr0, smr);
      if (rr0 <= outer_thr) break;
      const float inner_thr = 1e-6f * rr0;
      float beta = 0.f;
      bool first = true;
      while (it < max_it) {
        float dot = 0.f;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
          const int32_t u = mu[i];
          const float yu = v.yv[u];
          float sacc = 0.f;
          for (int32_t t = v.rowptr[u], t1 = v.rowptr[u + 1]; t < t1; ++t) {
            const float sw = v.csr_sw[t];
            sacc = fmaf(sw * sw, yu - v.yv[v.csr_col[t]], sacc);
          }
          const float ay = fmaf(lam, yu, sacc);
          const float pn = first ? yu : fmaf(beta, v.pv[u], yu);
          const float apn = first ? ay : fmaf(beta, v.Ap[u], ay);
          v.pv[u] = pn;
          v.Ap[u] = apn;
          dot = fmaf(pn, apn, dot);
        }
        const float pap = block_sum<float>(dot, smr);
        const float alpha = pap > 0.f ? rz / pap : 0.f;
        float rzn = 0.f, rr = 0.f;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
          const int32_t u = mu[i];
          v.dz[u] = fmaf(alpha, v.pv[u], v.dz[u]);
          const float r = fmaf(-alpha, v.Ap[u], v.res[u]);
          v.res[u] = r;
          const float y = r / v.diag[u];
          v.yv[u] = y;
          rzn = fmaf(r, y, rzn);
          rr = fmaf(r, r, rr);
        }
        rzn = block_sum<float>(rzn, smr);
        rr = block_sum<float>(rr, smr);
        ++it;
        if (rr <= inner_thr || !(pap > 0.f)) break;
        beta = rzn / rz;
        rz = rzn;
        first = false;
      }
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int32_t u = mu[i];
        const df32 zn = df_add_f(df32{v.z[u], v.z_lo[u]}, v.dz[u]);
        v.z[u] = zn.hi;
        v.z_lo[u] = zn.lo;
      }
      __syncthreads();
    }
    if (it > max_iters) max_iters = it;
  }
  if (threadIdx.x == 0 && max_iters > 0) atomicMax(&v.counters[kCntCompIters], max_iters);
}

// Solve (lambda I + B^T B) z = u over all station groups at once (nodes of
// different groups never share an edge) by iterative refinement: the residual
// is evaluated in double-float, each correction by Jacobi-preconditioned FP32 CG
// to a relative tolerance of 1e-3; stop when |u - A z| <= tol |u| (double-float
// residual) or after max_it inner iterations in total.  The CG recurs
// A p = A y + beta A p so that its SpMV runs on y, which is complete after the
// update phase: two grid barriers per iteration.
__global__ void __launch_bounds__(512) k_pcg(StepView v, int max_it, float tol) {
  __shared__ float smr[33];
  if (aborted_cta(v) || gated_off(v)) return;
  const int G = gridDim.x;
  const int32_t P_u = v.counters[kCntPairs];
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gstride = G * blockDim.x;
  float* red = v.red;
  const float lam = v.lam;
  constexpr float kInnerTol = 1e-3f;
  constexpr int kMaxRounds = 8;
  const int32_t nbig = v.bigpos[P_u];      // nodes of the grid-tier components, in pair order
  float bb = 0.f;
  for (int32_t t = gtid; t < nbig; t += gstride) {
    const int32_t u = v.biglist[t];
    const float r = v.rhs[u];
    v.z[u] = 0.f;
    v.z_lo[u] = 0.f;
    bb += r * r;
  }
  bb = block_sum<float>(bb, smr);
  if (threadIdx.x == 0) red[5 * kMaxGrid + blockIdx.x] = bb;
  if (!grid_barrier(v.counters, v.prm->wait_ns)) return;
  bb = sum_partials(red + 5 * kMaxGrid, G, smr);
  const float outer_thr = tol * tol * bb;
  int it = 0;
  for (int round = 0; round < kMaxRounds && bb > 0.f && it < max_it; ++round) {
    // outer residual u - A z in double-float; inner start: res = y = D^-1 res
    float rz = 0.f, rr0 = 0.f;
    for (int32_t t = gtid; t < nbig; t += gstride) {
      const int32_t u = v.biglist[t];
      float r;
      if (round == 0) {
        r = v.rhs[u] + v.rhs_lo[u];
      } else {
        const df32 zu = {v.z[u], v.z_lo[u]};
        df32 acc = {0.f, 0.f};
        for (int32_t t = v.rowptr[u], t1 = v.rowptr[u + 1]; t < t1; ++t) {
          const int32_t c = v.csr_col[t];
          const float sw = v.csr_sw[t];
          acc = df_add(acc, df_mul(df_two_prod(sw, sw), df_add(zu, df32{-v.z[c], -v.z_lo[c]})));
        }
        df32 rd = df_add(df32{v.rhs[u], v.rhs_lo[u]}, df_mul_f(zu, -lam));
        rd = df_add(rd, df32{-acc.hi, -acc.lo});
        r = rd.hi;
      }
      const float y = r / v.diag[u];
      v.res[u] = r;
      v.yv[u] = y;
      v.dz[u] = 0.f;
      rz = fmaf(r, y, rz);
      rr0 = fmaf(r, r, rr0);
    }
    rz = block_sum<float>(rz, smr);
    rr0 = block_sum<float>(rr0, smr);
    if (threadIdx.x == 0) {
      red[0 * kMaxGrid + blockIdx.x] = rz;
      red[1 * kMaxGrid + blockIdx.x] = rr0;
    }
    if (!grid_barrier(v.counters, v.prm->wait_ns)) return;
    rz = sum_partials(red + 0 * kMaxGrid, G, smr);
    rr0 = sum_partials(red + 1 * kMaxGrid, G, smr);
    if (rr0 <= outer_thr) break;                 // refined solution is accurate enough
    const float inner_thr = kInnerTol * kInnerTol * rr0;
    float beta = 0.f;
    bool first = true;
    while (it < max_it) {
      // p = y + beta p;  A p = A y + beta A p;  p.Ap
      float dot = 0.f;
      for (int32_t t = gtid; t < nbig; t += gstride) {
        const int32_t u = v.biglist[t];
        const float yu = v.yv[u];
        float s = 0.f;
        for (int32_t t = v.rowptr[u], t1 = v.rowptr[u + 1]; t < t1; ++t) {
          const float sw = v.csr_sw[t];
          s = fmaf(sw * sw, yu - v.yv[v.csr_col[t]], s);
        }
        const float ay = fmaf(lam, yu, s);
        const float pn = first ? yu : fmaf(beta, v.pv[u], yu);
        const float apn = first ? ay : fmaf(beta, v.Ap[u], ay);
        v.pv[u] = pn;
        v.Ap[u] = apn;
        dot = fmaf(pn, apn, dot);
      }
      dot = block_sum<float>(dot, smr);
      if (threadIdx.x == 0) red[2 * kMaxGrid + blockIdx.x] = dot;
      if (!grid_barrier(v.counters, v.prm->wait_ns)) return;
      const float pap = sum_partials(red + 2 * kMaxGrid, G, smr);
      const float alpha = pap > 0.f ? rz / pap : 0.f;
      float rzn = 0.f, rr = 0.f;
      for (int32_t t = gtid; t < nbig; t += gstride) {
        const int32_t u = v.biglist[t];
        v.dz[u] = fmaf(alpha, v.pv[u], v.dz[u]);
        const float r = fmaf(-alpha, v.Ap[u], v.res[u]);
        v.res[u] = r;
        const float y = r / v.diag[u];
        v.yv[u] = y;
        rzn = fmaf(r, y, rzn);
        rr = fmaf(r, r, rr);
      }
      rzn = block_sum<float>(rzn, smr);
      rr = block_sum<float>(rr, smr);
      if (threadIdx.x == 0) {
        red[3 * kMaxGrid + blockIdx.x] = rzn;
        red[4 * kMaxGrid + blockIdx.x] = rr;
      }
      if (!grid_barrier(v.counters, v.prm->wait_ns)) return;
      rzn = sum_partials(red + 3 * kMaxGrid, G, smr);
      rr = sum_partials(red + 4 * kMaxGrid, G, smr);
      ++it;
      if (rr <= inner_thr || !(pap > 0.f)) break;
      beta = rzn / rz;
      rz = rzn;
      first = false;
    }
    // z += dz in double-float; the next round reads z at neighbours
    for (int32_t t = gtid; t < nbig; t += gstride) {
      const int32_t u = v.biglist[t];
      const df32 zn = df_add_f(df32{v.z[u], v.z_lo[u]}, v.dz[u]);
      v.z[u] = zn.hi;
      v.z_lo[u] = zn.lo;
    }
    if (!grid_barrier(v.counters, v.prm->wait_ns)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) v.counters[kCntIters] = it;
}

// q_e = sigma^-2 (r_e - sqrt(w_e) (z_i - z_j)) with z in double-float, the node
// sums s_p = sum_{e: p = i-end} q_e - sum_{e: p = j-end} q_e (= d loglik / d T_p),
// and r^T Sigma^-1 r = sum_e r_e q_e (FP64 per block).
__global__ void k_final(StepView v) {
  extern __shared__ float smf[];
  __shared__ double smd[33];
  if (aborted_cta(v)) return;
  float* zh = smf;
  float* zl = zh + v.L_max;
  float* qs = zl + v.L_max;
  const int s = blockIdx.x;
  const BlockRange br = block_range(v, s);
  for (int l = threadIdx.x; l < br.L; l += blockDim.x) {
    if (v.whiten) {
      const int32_t u = v.loc2u[br.q0 + l];
      zh[l] = v.z[u];
      zl[l] = v.z_lo[u];
    } else {
      zh[l] = 0.f;
      zl[l] = 0.f;
    }
  }
  __syncthreads();
  double quad = 0.0;
  for (int e = threadIdx.x; e < br.ne; e += blockDim.x) {
    const uint32_t lij = v.obs_l[br.e0 + e];
    const int li = lij & 0xFFFF, lj = lij >> 16;
    const df32 d = df_add(df32{zh[li], zl[li]}, df32{-zh[lj], -zl[lj]});
    const df32 bz = df_mul_f(d, v.obs_sw[br.e0 + e]);
    const float r = v.r_obs[br.e0 + e];
    float qe;
    if (v.loss == SPIDER_LOSS_L1) {
      // stage 1: d(-sum |r|)/dr = -sign(r); the quadratic slot carries 2|r| so
      // that the log posterior's -1/2 (quad) is -sum |r|
      qe = r > 0.f ? 1.f : (r < 0.f ? -1.f : 0.f);
      quad += 2.0 * fabs((double)r);
    } else {
      const df32 t = df_add_f(df32{-bz.hi, -bz.lo}, r);
      qe = v.inv_s2 * t.hi;
      quad += (double)r * (double)qe;
    }
    qs[e] = qe;
    v.q_obs[br.e0 + e] = qe;
  }
  quad = block_sum<double>(quad, smd);
  if (threadIdx.x == 0) v.dblk[s] = quad;
  const uint16_t* he = v.blk_he + 2 * br.e0;
  for (int l = threadIdx.x; l < br.L; l += blockDim.x) {
    const int32_t q = br.q0 + l;
    const int h0 = v.node_he[q];
    const int h1 = (l + 1 < br.L) ? (int)v.node_he[q + 1] : 2 * br.ne;
    float a = 0.f;
    for (int h = h0; h < h1; ++h) {
      const int code = he[h];
      a += (code & 1) ? -qs[code >> 1] : qs[code >> 1];
    }
    if (!v.multi[q]) v.s_u[v.loc2u[q]] = a;
    else v.part_a[q] = a;
  }
}

// s_p * (N_s/n_s) times (dT/dx_p, 1) into the global pair slots, stamped.
__global__ void k_merge_s(StepView v) {
  if (aborted(v)) return;
  const int tag = v.prm->tag;
  const int32_t P_u = v.counters[kCntPairs];
  for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < P_u; u += gridDim.x * blockDim.x) {
    const int32_t q = v.uniq_q[u];
    const int32_t p = v.node_pair[q];
    const int32_t m = v.pair_ev[p];
    const int sb = v.ev_sub[m];
    const float scale = (float)((double)v.sub_nobs[sb] / (double)v.sub_nsel[sb]);
    float sp = v.multi[q] ? merge_occ(v, p, tag, v.part_a) : v.s_u[u];
    sp *= scale;
    const float4 J = v.J[u];
    v.gp[p] = make_float4(sp * J.x, sp * J.y, sp * J.z, sp);
    v.pstamp[p] = tag;
    v.estamp[m] = tag;
  }
}

// ------------------------------------------------------------------ events
// centroid of the current state offset, per sub-problem: fixed chunks of
// events summed in a fixed tree, chunks summed in order
__global__ void k_cen_chunk(StepView v) {
  __shared__ float smr[33];
  if (aborted_cta(v)) return;
  const int c = blockIdx.x;
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int32_t m = v.chunk_ev0[c] + threadIdx.x; m < v.chunk_ev0[c + 1]; m += blockDim.x) {
    const float4 d = v.dth[m];
    a.x += d.x; a.y += d.y; a.z += d.z; a.w += d.w;
  }
  a.x = block_sum<float>(a.x, smr);
  a.y = block_sum<float>(a.y, smr);
  a.z = block_sum<float>(a.z, smr);
  a.w = block_sum<float>(a.w, smr);
  if (threadIdx.x == 0) v.cen_chunk[c] = a;
}

__global__ void k_cen_final(StepView v) {
  __shared__ float smr[33];
  if (aborted_cta(v)) return;
  const int s = blockIdx.x;
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int32_t c = v.sub_chunk_off[s] + threadIdx.x; c < v.sub_chunk_off[s + 1]; c += blockDim.x) {
    const float4 d = v.cen_chunk[c];
    a.x += d.x; a.y += d.y; a.z += d.z; a.w += d.w;
  }
  a.x = block_sum<float>(a.x, smr);
  a.y = block_sum<float>(a.y, smr);
  a.z = block_sum<float>(a.z, smr);
  a.w = block_sum<float>(a.w, smr);
  if (threadIdx.x == 0) {
    const float inv = 1.0f / (float)v.sub_nev[s];
    v.sub_cen[s] = make_float4(a.x * inv, a.y * inv, a.z * inv, a.w * inv);
  }
}

// grad_m = (N_s/n_s) sum_k s_(m,k) (dT/dx, 1) - dtheta_m / sigma_e^2
//          - mean_s(dtheta) / (M_s sigma_c^2)             (priors of Sec. 3.1)
// mode 0: write grad; mode 1: SGLD theta += eps grad + ns sqrt(2 eps) eta (Sec. 3.2)
__global__ void k_event(StepView v) {
  __shared__ double smd[33];
  if (aborted_cta(v)) return;
  const StepParams& pr = *v.prm;
  const int tag = pr.tag, mode = pr.mode;
  const float eps = pr.eps;
  const float4 ise = v.inv_sig_e2, isc = v.inv_sig_c2;
  const float sq = pr.noise_scale * sqrtf(2.0f * eps);
  const uint2 key = seed_key(pr.seed);
  double lp = 0.0;
  int bad = 0, touched = 0;
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < v.M; m += (int64_t)gridDim.x * blockDim.x) {
    const int sb = v.ev_sub[m];
    const float4 cen = v.sub_cen[sb];
    const float invM = 1.0f / (float)v.sub_nev[sb];
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    if (v.estamp[m] == tag) {
      ++touched;
      for (int32_t p = v.pair_off[m], p1 = v.pair_off[m + 1]; p < p1; ++p)
        if (v.pstamp[p] == tag) {
          const float4 c = v.gp[p];
          g.x += c.x; g.y += c.y; g.z += c.z; g.w += c.w;
        }
    }
    const float4 d = v.dth[m];
    g.x -= d.x * ise.x + cen.x * isc.x * invM;
    g.y -= d.y * ise.y + cen.y * isc.y * invM;
    g.z -= d.z * ise.z + cen.z * isc.z * invM;
    g.w -= d.w * ise.w + cen.w * isc.w * invM;
    if (mode == 0) {
      v.grad[m] = g;
      lp += (double)d.x * d.x * ise.x + (double)d.y * d.y * ise.y + (double)d.z * d.z * ise.z +
            (double)d.w * d.w * ise.w;
      if (!(isfinite(g.x) && isfinite(g.y) && isfinite(g.z) && isfinite(g.w))) bad = 1;
    } else {
      float4 nd;
      if (v.update == SPIDER_UPDATE_ADAM) {
        // stage-1 optimiser: Adam ascent on the objective, no noise
        float4 m1 = v.mom1[m], m2 = v.mom2[m];
        const float b1 = v.beta1, b2 = v.beta2;
        m1.x = fmaf(b1, m1.x, (1.f - b1) * g.x); m2.x = fmaf(b2, m2.x, (1.f - b2) * (g.x * g.x));
        m1.y = fmaf(b1, m1.y, (1.f - b1) * g.y); m2.y = fmaf(b2, m2.y, (1.f - b2) * (g.y * g.y));
        m1.z = fmaf(b1, m1.z, (1.f - b1) * g.z); m2.z = fmaf(b2, m2.z, (1.f - b2) * (g.z * g.z));
        m1.w = fmaf(b1, m1.w, (1.f - b1) * g.w); m2.w = fmaf(b2, m2.w, (1.f - b2) * (g.w * g.w));
        v.mom1[m] = m1;
        v.mom2[m] = m2;
        const float bc1 = pr.bc1, bc2 = pr.bc2, pe = v.upd_eps;
        nd.x = d.x + eps * (m1.x * bc1) / (sqrtf(m2.x * bc2) + pe);
        nd.y = d.y + eps * (m1.y * bc1) / (sqrtf(m2.y * bc2) + pe);
        nd.z = d.z + eps * (m1.z * bc1) / (sqrtf(m2.z * bc2) + pe);
        nd.w = d.w + eps * (m1.w * bc1) / (sqrtf(m2.w * bc2) + pe);
      } else {
        const uint4 w = philox4x32_10(
            make_uint4((uint32_t)v.ev_caller[m], (uint32_t)v.sub_chain[sb], (uint32_t)v.sub_catalog[sb], kTagNoise),
            key);
        const float2 n01 = box_muller(w.x, w.y), n23 = box_muller(w.z, w.w);
        if (v.update == SPIDER_UPDATE_PSGLD) {
          // Eq. pSGLD: per-coordinate preconditioner from the running second moment
          float4 m2 = v.mom2[m];
          const float b2 = v.beta2, pe = v.upd_eps, ns = pr.noise_scale;
          m2.x = fmaf(b2, m2.x, (1.f - b2) * (g.x * g.x));
          m2.y = fmaf(b2, m2.y, (1.f - b2) * (g.y * g.y));
          m2.z = fmaf(b2, m2.z, (1.f - b2) * (g.z * g.z));
          m2.w = fmaf(b2, m2.w, (1.f - b2) * (g.w * g.w));
          v.mom2[m] = m2;
          const float Vx = 1.f / (sqrtf(m2.x) + pe), Vy = 1.f / (sqrtf(m2.y) + pe);
          const float Vz = 1.f / (sqrtf(m2.z) + pe), Vw = 1.f / (sqrtf(m2.w) + pe);
          nd.x = d.x + eps * Vx * g.x + ns * sqrtf(2.f * eps * Vx) * n01.x;
          nd.y = d.y + eps * Vy * g.y + ns * sqrtf(2.f * eps * Vy) * n01.y;
          nd.z = d.z + eps * Vz * g.z + ns * sqrtf(2.f * eps * Vz) * n23.x;
          nd.w = d.w + eps * Vw * g.w + ns * sqrtf(2.f * eps * Vw) * n23.y;
        } else {
          nd.x = d.x + eps * g.x + sq * n01.x;
          nd.y = d.y + eps * g.y + sq * n01.y;
          nd.z = d.z + eps * g.z + sq * n23.x;
          nd.w = d.w + eps * g.w + sq * n23.y;
        }
      }
      if (!(isfinite(nd.x) && isfinite(nd.y) && isfinite(nd.z) && isfinite(nd.w))) bad = 1;
      v.dth[m] = nd;
      if (pr.sample_slot >= 0) v.samples[pr.sample_slot * v.M + m] = nd;
    }
  }
  if (bad) set_error(v.counters, SPIDER_E_NONFINITE);
  touched = block_sum<int>(touched, reinterpret_cast<int*>(smd));
  if (threadIdx.x == 0 && touched) atomicAdd(&v.counters[kCntEvents], touched);
  if (mode == 0) {
    lp = block_sum<double>(lp, smd);
    if (threadIdx.x == 0) v.dred[2 * kMaxGrid + blockIdx.x] = lp;
  }
}

// FP64 log posterior: sum_s -1/2 (N_s/n_s) r_s^T Sigma^-1 r_s - 1/2 |dtheta/sigma_e|^2
//                     - 1/2 sum_s |mean_s(dtheta)/sigma_c|^2   (constants dropped)
__global__ void k_logpost(StepView v, int64_t n_b) {
  __shared__ double smd[33];
  if (aborted_cta(v)) return;
  double quad = 0.0, lp = 0.0;
  for (int64_t t = threadIdx.x; t < n_b; t += blockDim.x) {
    const int sb = v.blk_sub[v.sel[t]];
    quad += v.dblk[t] * ((double)v.sub_nobs[sb] / (double)v.sub_nsel[sb]);
  }
  for (int i = threadIdx.x; i < v.cen_grid; i += blockDim.x) lp += v.dred[2 * kMaxGrid + i];
  quad = block_sum<double>(quad, smd);
  lp = block_sum<double>(lp, smd);
  double lc = 0.0;
  const float isc[4] = {v.inv_sig_c2.x, v.inv_sig_c2.y, v.inv_sig_c2.z, v.inv_sig_c2.w};
  for (int sb = threadIdx.x; sb < v.n_sub; sb += blockDim.x) {
    const float4 c = v.sub_cen[sb];
    const double cc[4] = {c.x, c.y, c.z, c.w};
    for (int a = 0; a < 4; ++a) lc += cc[a] * cc[a] * (double)isc[a];
  }
  lc = block_sum<double>(lc, smd);
  if (threadIdx.x == 0) {
    const double ll = -0.5 * quad;
    v.dout[0] = ll;
    v.dout[1] = -0.5 * lp;
    v.dout[2] = -0.5 * lc;
    v.dout[3] = ll - 0.5 * lp - 0.5 * lc;
  }
}

// FP64 diagnostics: |g_m| of the minibatch gradient and sum (g - G)^2
__global__ void k_diag(StepView v, const float4* __restrict__ g, const float4* __restrict__ G,
                       double* norms, double* part) {
  __shared__ double smd[33];
  double acc = 0.0;
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < v.M; m += (int64_t)gridDim.x * blockDim.x) {
    const float4 a = g[m], b = G[m];
    norms[m] = sqrt((double)a.x * a.x + (double)a.y * a.y + (double)a.z * a.z + (double)a.w * a.w);
    const double dx = (double)a.x - b.x, dy = (double)a.y - b.y, dz = (double)a.z - b.z, dw = (double)a.w - b.w;
    acc += dx * dx + dy * dy + dz * dz + dw * dw;
  }
  acc = block_sum<double>(acc, smd);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// theta = theta_0 + dtheta in FP64, written in the caller's event order (the
// read-back of spider_get_state / spider_samples); src is the state offset or
// one stored sample.
__global__ void k_state_out(StepView v, const float4* __restrict__ src, double* __restrict__ out) {
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < v.M; m += (int64_t)gridDim.x * blockDim.x) {
    const float4 d = src[m];
    const double* t = v.th0_d + 4 * m;
    double4 o;
    o.x = t[0] + (double)d.x;
    o.y = t[1] + (double)d.y;
    o.z = t[2] + (double)d.z;
    o.w = t[3] + (double)d.w;
    reinterpret_cast<double4*>(out)[v.ev_out[m]] = o;
  }
}

// the gradient (FP32) in the caller's event order
__global__ void k_grad_out(StepView v, float4* __restrict__ out) {
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < v.M; m += (int64_t)gridDim.x * blockDim.x)
    out[v.ev_out[m]] = v.grad[m];
}

__global__ void k_philox_words(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                               int64_t n, uint32_t* out) {
  int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  uint4 w = philox4x32_10(make_uint4(c0 + (uint32_t)m, c1, c2, c3), seed_key(seed));
  reinterpret_cast<uint4*>(out)[m] = w;
}

}  // namespace

// ------------------------------------------------------------------ launchers
#define CK_LAUNCH(call)                      \
  do {                                       \
    cudaError_t _e = (call);                 \
    if (_e != cudaSuccess) return _e;        \
  } while (0)

static inline int grid_for(int64_t n, int t = kThreads) { return (int)((n + t - 1) / t); }

cudaError_t launch_select(const StepView& v, int64_t n_b, cudaStream_t st, int bthreads) {
  k_select<<<grid_for(n_b), kThreads, 0, st>>>(v, n_b);
  k_owner<<<(unsigned)n_b, bthreads, 0, st>>>(v);
  k_scan_owner<<<1, 1024, 0, st>>>(v, n_b);
  k_assign<<<(unsigned)n_b, bthreads, 0, st>>>(v);
  k_link<<<(unsigned)n_b, bthreads, 0, st>>>(v);
  return cudaGetLastError();
}

size_t resid_smem(const StepView& v) { return (size_t)(3 * v.L_max + 2 * v.B) * sizeof(float); }
size_t final_smem(const StepView& v) { return (size_t)(2 * v.L_max + v.B) * sizeof(float); }

cudaError_t configure_step_kernels(const StepView& v) {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_resid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)resid_smem(v))))
    return e;
  if ((e = cudaFuncSetAttribute(k_final, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)final_smem(v))))
    return e;
  if ((e = cudaFuncSetAttribute(k_comp_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(kCompWarps * sizeof(WarpSmem)))))
    return e;
  if ((e = cudaFuncSetAttribute(k_comp_solve_cta, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(CtaSmem))))
    return e;
  return cudaSuccess;
}

int pcg_grid(const StepView& v, int num_sms) {
  (void)v;
  int a = 0, b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_pcg, 512, 0) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_cc, 512, 0) != cudaSuccess)
    return 0;
  int per_sm = a < b ? a : b;
  if (per_sm > 2) per_sm = 2;   // fewer barrier participants; 512 threads each
  if (per_sm < 1) return 0;
  const int g = num_sms * per_sm;
  return g > kMaxGrid ? kMaxGrid : g;
}

// ev (or null): events recorded after k_resid and after k_merge_rhs
cudaError_t launch_resid(const StepView& v, int64_t n_b, int gu, cudaStream_t st, const cudaEvent_t* ev,
                         int bthreads) {
  k_resid<<<(unsigned)n_b, bthreads, resid_smem(v), st>>>(v);
  if (ev) CK_LAUNCH(cudaEventRecord(ev[0], st));
  if (v.whiten) k_merge_rhs<<<gu, kThreads, 0, st>>>(v);
  if (ev) CK_LAUNCH(cudaEventRecord(ev[1], st));
  return cudaGetLastError();
}

cudaError_t launch_pcg(const StepView& v, int64_t n_b, int max_it, float tol, int grid, int warp_mult,
                       int cta_mult, cudaStream_t st) {
  if (!v.whiten) return cudaSuccess;
  const int32_t* Pdev = v.counters + kCntPairs;
  const int parts = grid;
  // CSR of the merged minibatch matrix
  k_scan_a<<<parts, kThreads, 0, st>>>(v.rowlen, Pdev, v.scan_part, v.gate);
  k_scan_b<<<1, 1024, 0, st>>>(v.scan_part, parts, v.gate);
  k_scan_c<<<parts, kThreads, 0, st>>>(v.rowlen, Pdev, v.scan_part, v.rowptr, v.gate);
  k_fill_rows<<<(unsigned)n_b, kThreads, 0, st>>>(v);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // connected components
  k_cc_local<<<(unsigned)n_b, kThreads, (size_t)v.L_max * sizeof(int), st>>>(v);
  {
    StepView vv = v;
    int64_t nb = n_b;
    void* args[] = {&vv, &nb};
    e = cudaLaunchCooperativeKernel((const void*)k_cc, dim3(grid), dim3(512), args, 0, st);
    if (e != cudaSuccess) return e;
  }
  CK_LAUNCH(cudaMemsetAsync(v.counters + kCntBarArrive, 0, 2 * sizeof(int32_t), st));
  k_scan_a<<<parts, kThreads, 0, st>>>(v.cslot, Pdev, v.scan_part, v.gate);
  k_scan_b<<<1, 1024, 0, st>>>(v.scan_part, parts, v.gate);
  k_scan_c<<<parts, kThreads, 0, st>>>(v.cslot, Pdev, v.scan_part, v.members, v.gate);
  k_cc_roots<<<parts, kThreads, 0, st>>>(v);
  k_scan_a<<<parts, kThreads, 0, st>>>(v.comp_off, v.counters + kCntComps, v.scan_part, v.gate);
  k_scan_b<<<1, 1024, 0, st>>>(v.scan_part, parts, v.gate);
  k_scan_c<<<parts, kThreads, 0, st>>>(v.comp_off, v.counters + kCntComps, v.scan_part, v.comp_off, v.gate);
  k_cc_fill<<<parts, kThreads, 0, st>>>(v);
  k_cc_place<<<parts, kThreads, 0, st>>>(v);
  k_scan_a<<<parts, kThreads, 0, st>>>(v.bigpos, Pdev, v.scan_part, v.gate);
  k_scan_b<<<1, 1024, 0, st>>>(v.scan_part, parts, v.gate);
  k_scan_c<<<parts, kThreads, 0, st>>>(v.bigpos, Pdev, v.scan_part, v.bigpos, v.gate);
  k_big_list<<<parts, kThreads, 0, st>>>(v);
  k_corder_scan<<<1, 512, 0, st>>>(v);
  k_corder_fill<<<parts, kThreads, 0, st>>>(v);
  // the CTA tier first; the warp tier may start as soon as every CTA of it has
  // begun (programmatic dependent launch) and waits for it before it exits
  k_comp_solve_cta<<<cta_mult * parts, kCtaThreads, sizeof(CtaSmem), st>>>(v, max_it, tol);
  {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)(warp_mult * parts * (4 / kCompWarps)));   // the same warps for any CTA size
    lc.blockDim = dim3(kCompWarps * 32);
    lc.dynamicSmemBytes = kCompWarps * sizeof(WarpSmem);
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    e = cudaLaunchKernelEx(&lc, k_comp_solve, v, max_it, tol);
    if (e != cudaSuccess) return e;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  StepView vv = v;
  int mi = max_it;
  float tl = tol;
  void* args[] = {&vv, &mi, &tl};
  return cudaLaunchCooperativeKernel((const void*)k_pcg, dim3(grid), dim3(512), args, 0, st);
}

// ev (or null): events recorded after k_final, k_merge_s, the centroid, k_event
cudaError_t launch_finish(const StepView& v, int64_t n_b, int gu, bool logpost, cudaStream_t st,
                          const cudaEvent_t* ev, int bthreads) {
  k_final<<<(unsigned)n_b, bthreads, final_smem(v), st>>>(v);
  if (ev) CK_LAUNCH(cudaEventRecord(ev[0], st));
  k_merge_s<<<gu, kThreads, 0, st>>>(v);
  if (ev) CK_LAUNCH(cudaEventRecord(ev[1], st));
  k_cen_chunk<<<v.n_chunks, kThreads, 0, st>>>(v);
  k_cen_final<<<v.n_sub, kThreads, 0, st>>>(v);
  if (ev) CK_LAUNCH(cudaEventRecord(ev[2], st));
  k_event<<<v.cen_grid, kThreads, 0, st>>>(v);
  if (ev) CK_LAUNCH(cudaEventRecord(ev[3], st));
  if (logpost) k_logpost<<<1, kThreads, 0, st>>>(v, n_b);
  return cudaGetLastError();
}

cudaError_t launch_diag(const StepView& v, const float4* g, const float4* G, double* norms, double* part,
                        int grid, cudaStream_t st) {
  k_diag<<<grid, kThreads, 0, st>>>(v, g, G, norms, part);
  return cudaGetLastError();
}

cudaError_t launch_state_out(const StepView& v, const float4* src, double* out, int grid, cudaStream_t st) {
  k_state_out<<<grid, kThreads, 0, st>>>(v, src, out);
  return cudaGetLastError();
}

cudaError_t launch_grad_out(const StepView& v, float4* out, int grid, cudaStream_t st) {
  k_grad_out<<<grid, kThreads, 0, st>>>(v, out);
  return cudaGetLastError();
}

cudaError_t launch_philox_words(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                int64_t n, uint32_t* out, cudaStream_t st) {
  k_philox_words<<<grid_for(n), kThreads, 0, st>>>(seed, c0, c1, c2, c3, n, out);
  return cudaGetLastError();
}

}  // namespace spider
