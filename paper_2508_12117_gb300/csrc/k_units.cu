// Units of the piece-inverse whitening, solved data-parallel (row a5, Eq.
// marginal_sigma): the Schur complement on the shared nodes of every unit at
// once (see k_whiten.cu for the decomposition).
//
// A unit u owns the occurrence slots [uocc_off[u], uocc_off[u + 1]): its pieces'
// members, piece by piece in ascending piece id and member order.  The same
// range indexes every other per-step list of the unit (its shared occurrences
// in slot order and sorted by pair, its shared nodes), each shorter than it.
// Set-up (once per step): sorted pieces and member counts (one warp per unit);
// occurrence tables, shared lists and shared nodes (one warp per unit); the
// pieces' (A_p[G,G])^-1 and the units' S^-1 by Gauss-Jordan (a warp per matrix
// in shared memory up to 32 nodes, a CTA per matrix in registers up to 64 (96
// for the pieces), S^-1 above 64 nodes in shared memory by one CTA per unit).
// Each refinement round: residual (one thread per occurrence, then per shared
// node), w = A_p[:, I] f_I (one thread per occurrence), the small dense Schur
// solve (one warp per unit), the update of z (one thread per occurrence).
// A unit beyond the limits below is marked invalid and raises the flag on
// which the general component solver takes the whole step.
#include <cuda_runtime.h>

#include <cstdint>

#include "dfloat.cuh"
#include "kernels.h"
#include "step_util.cuh"

namespace spider {

namespace {

constexpr int kUMaxPieces = 32;    // pieces of a unit
constexpr int kUMaxShared = 1024;  // shared occurrences of a unit
constexpr int kUMaxGamma = 192;    // shared nodes of a unit
constexpr int kUMaxGp = 96;        // shared nodes of one piece
constexpr int kUWarps = 8;         // warps per CTA of the per-unit kernels
constexpr int kUOccWarps = 4;      // warps per CTA of k_u_occ (a sort buffer of kUMaxShared keys each)
constexpr int kUTh = 256;          // threads per CTA of the per-occurrence kernels

__device__ __forceinline__ int gwarp() { return (blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ int nwarps() { return (gridDim.x * blockDim.x) >> 5; }

__device__ __forceinline__ void flag_general(const StepView& v) { atomicExch(&v.wfast[kWGeneral], 1); }

// a unit beyond this solver's limits: marked invalid (exactly once) and handed
// to the CTA unit passes of k_whiten.cu
__device__ __forceinline__ void give_up_unit(const StepView& v, int32_t u, int why) {
  if (atomicExch(&v.u_ng[u], -1) != -1) {
    v.unit_defer[atomicAdd(&v.wfast[kWDefer], 1)] = u;
    atomicAdd(&v.wfast[kWSlots + 64 + 16 + why], 1);     // why it was handed over
  }
}

// exclusive warp scan of small integers; *total = sum over the warp
__device__ __forceinline__ int warp_exscan(int x, int lane, int* total) {
  int s = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, s, o);
    if (lane >= o) s += y;
  }
  *total = __shfl_sync(0xffffffffu, s, 31);
  return s - x;
}

// warp Gauss-Jordan inverse of the SPD n x n matrix M (row-major, shared
// memory): lanes own columns; sweep k first keeps m_kj = M[k][j] / p of the
// lane's columns, updates every row (row k comes out as 0 and is then set to
// m_kj), then column k and the pivot (see k_whiten.cu for the sweep)
__device__ bool warp_gj(float* M, int n, int lane) {
  for (int k = 0; k < n; ++k) {
    const float p = M[k * n + k];
    if (!(p > 0.f)) return false;
    const float ip = 1.f / p;
    __syncwarp();
    for (int j = lane; j < n; j += 32) {
      if (j == k) continue;
      const float mkj = M[k * n + j] * ip;
      int i = 0;
      for (; i + 3 < n; i += 4) {
        const float c0 = M[i * n + k], c1 = M[(i + 1) * n + k], c2 = M[(i + 2) * n + k], c3 = M[(i + 3) * n + k];
        const float x0 = M[i * n + j], x1 = M[(i + 1) * n + j], x2 = M[(i + 2) * n + j], x3 = M[(i + 3) * n + j];
        M[i * n + j] = fmaf(-c0, mkj, x0);
        M[(i + 1) * n + j] = fmaf(-c1, mkj, x1);
        M[(i + 2) * n + j] = fmaf(-c2, mkj, x2);
        M[(i + 3) * n + j] = fmaf(-c3, mkj, x3);
      }
      for (; i < n; ++i) M[i * n + j] = fmaf(-M[i * n + k], mkj, M[i * n + j]);
      M[k * n + j] = mkj;
    }
    __syncwarp();
    for (int t = lane; t < n; t += 32)
      if (t != k) M[t * n + k] = -M[t * n + k] * ip;
    __syncwarp();
    if (lane == 0) M[k * n + k] = ip;
    __syncwarp();
  }
  return true;
}

template <int NT>
__device__ __forceinline__ void group_sync() {
  if constexpr (NT == 32) __syncwarp(); else __syncthreads();
}

// Gauss-Jordan inverse of an SPD n x n matrix (n <= NP, padded with the
// identity) held in registers by a group of NT threads: thread t owns column
// j = t % NP, rows RB (t / NP) .. RB (t / NP) + RB - 1 (NT RB = NP^2).  At pivot
// k the owners of column k and of row k publish them in shared memory (two
// alternating buffers of NP floats each, so one barrier per pivot suffices)
// and every thread updates its strip with
//   m_ij -= m_ik m_kj / p (i, j != k),  m_kj /= p,  m_ik = -m_ik / p,  m_kk = 1 / p.
// Shared-memory traffic per pivot is the two published vectors, not the matrix.
// False when a pivot is not positive (every thread of the group sees the same
// pivots, so the result is uniform).
template <int NP, int RB, int NT>
__device__ __forceinline__ bool strip_gj(float (&m)[RB], int t, float* ck2, float* rk2) {
  static_assert(NP * NP == NT * RB, "strip shape");
  const int j = t % NP, rb = t / NP;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    float* ck = ck2 + (k & 1) * NP;
    float* rk = rk2 + (k & 1) * NP;
    if (j == k) {
#pragma unroll
      for (int r = 0; r < RB; ++r) ck[rb * RB + r] = m[r];
    }
    if (rb == k / RB) rk[j] = m[k % RB];
    group_sync<NT>();
    const float p = ck[k];
    if (!(p > 0.f)) ok = false;
    const float ip = 1.f / p;
    const float mkj = rk[j] * ip;
#pragma unroll
    for (int r = 0; r < RB; ++r) m[r] = fmaf(-ck[rb * RB + r], mkj, m[r]);
    if (rb == k / RB) m[k % RB] = mkj;
    if (j == k) {
#pragma unroll
      for (int r = 0; r < RB; ++r) m[r] = -ck[rb * RB + r] * ip;
      if (rb == k / RB) m[k % RB] = ip;
    }
  }
  group_sync<NT>();
  return ok;
}

// a value every thread of the group reads the same (lane 0 / thread 0 reads it)
template <int NT>
__device__ __forceinline__ int group_read(const int32_t* p, int t, int* slot) {
  if constexpr (NT == 32) {
    int x = 0;
    if (t == 0) x = *((volatile const int32_t*)p);
    return __shfl_sync(0xffffffffu, x, 0);
  } else {
    __syncthreads();
    if (t == 0) *slot = *((volatile const int32_t*)p);
    __syncthreads();
    return *slot;
  }
}

// ------------------------------------------------------------------ set-up
// sorted pieces, member counts and per-piece bases (one warp per unit)
__global__ void k_u_prep(StepView v) {
  if (aborted(v)) return;
  const int lane = threadIdx.x & 31;
  const int32_t nu = v.wfast[kWUnits];
  for (int32_t u = gwarp(); u < nu; u += nwarps()) {
    const int32_t e0 = v.unit_off[u];
    const int k = v.unit_off[u + 1] - e0;
    if (lane == 0) v.u_ng[u] = 0;
    if (k > kUMaxPieces) {
      if (lane == 0) {
        v.u_nocc[u] = 0;
        give_up_unit(v, u, 0);
      }
      continue;
    }
    int32_t g = lane < k ? v.unit_pieces[e0 + lane] : INT32_MAX;
    int32_t b = lane < k ? v.unit_pblk[e0 + lane] : 0;
    // warp bitonic sort by piece id (ids are distinct)
    for (int kk = 2; kk <= 32; kk <<= 1)
      for (int j = kk >> 1; j > 0; j >>= 1) {
        const int32_t og = __shfl_xor_sync(0xffffffffu, g, j), ob = __shfl_xor_sync(0xffffffffu, b, j);
        const bool up = (lane & kk) == 0, lower = (lane & j) == 0;
        const bool take = lower ? (up ? og < g : og > g) : (up ? og > g : og < g);
        if (take) {
          g = og;
          b = ob;
        }
      }
    const int n = lane < k ? v.piece_node_off[g + 1] - v.piece_node_off[g] : 0;
    int tot;
    const int base = warp_exscan(n, lane, &tot);
    if (lane < k) {
      v.unit_pieces[e0 + lane] = g;
      v.unit_pblk[e0 + lane] = b;
      v.pu_base[e0 + lane] = base;
      v.pu_unit[e0 + lane] = u;
    }
    if (lane == 0) v.u_nocc[u] = tot;
  }
}

// exclusive scan of cnt[0, n) into off[0, n] (one CTA); n from the device
__global__ void k_u_scan(const int32_t* __restrict__ cnt, const int32_t* n_dev, int32_t* off, int64_t cap,
                         int32_t* wfast) {
  __shared__ int sm[33];
  const int32_t n = *n_dev;
  int carry = 0;
  for (int32_t c = 0; c < n; c += blockDim.x) {
    const int32_t i = c + threadIdx.x;
    const int val = i < n ? cnt[i] : 0;
    int total;
    const int pre = block_exscan(val, sm, &total);
    if (i < n) off[i] = carry + pre;
    carry += total;
  }
  if (threadIdx.x == 0) {
    off[n] = carry;
    if (carry > cap) atomicExch(&wfast[kWGeneral], 1);
  }
}

// occurrence tables, shared lists and shared nodes (one warp per unit)
__global__ void __launch_bounds__(kUOccWarps * 32) k_u_occ(StepView v) {
  __shared__ unsigned long long keys[kUOccWarps][kUMaxShared];
  if (aborted(v)) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int32_t nu = v.wfast[kWUnits];
  const int64_t cap = v.u_cap;
  for (int32_t u = gwarp(); u < nu; u += nwarps()) {
    const int32_t e0 = v.unit_off[u];
    const int k = v.unit_off[u + 1] - e0;
    const int32_t O = v.uocc_off[u];
    const int nocc = v.uocc_off[u + 1] - O;
    bool bad = k > kUMaxPieces || (int64_t)v.uocc_off[nu] > cap;
    int m_seen = 0, ng_seen = 0;
    if (!bad) {
      // occurrences: (piece entry, member) -> unique pair, base, shared flag
      for (int p = 0; p < k; ++p) {
        const int32_t pe = e0 + p, g = v.unit_pieces[pe];
        const int32_t q0 = v.blk_node_off[v.unit_pblk[pe]], m0 = v.piece_node_off[g];
        const int n = v.piece_node_off[g + 1] - m0, base = O + v.pu_base[pe];
        for (int i = lane; i < n; i += 32) {
          const int32_t q = q0 + v.piece_nodes[m0 + i];
          const int32_t o = base + i;
          v.o_g[o] = g;
          v.o_pe[o] = pe;
          v.o_i[o] = (uint16_t)i;
          v.o_base[o] = base;
          v.o_u[o] = v.loc2u[q];
          v.o_x[o] = v.multi[q] ? 0 : -1;
          v.o_unit[o] = u;
        }
      }
      __syncwarp();
      // shared occurrences in slot order
      int m = 0;
      for (int c = 0; c < nocc; c += 32) {
        const int o = O + c + lane;
        const bool sh = c + lane < nocc && v.o_x[o] >= 0;
        const unsigned bal = __ballot_sync(0xffffffffu, sh);
        const int t = m + __popc(bal & ((1u << lane) - 1u));
        if (sh && t < kUMaxShared) {
          v.sh_slot[O + t] = o;
          v.o_t[o] = O + t;
          keys[w][t] = ((unsigned long long)(uint32_t)v.o_u[o] << 32) | (uint32_t)t;
        }
        m += __popc(bal);
      }
      bad = m > kUMaxShared;
      m_seen = m;
      if (!bad) {
        __syncwarp();
        int m2 = 1;
        while (m2 < m) m2 <<= 1;
        for (int i = m + lane; i < m2; i += 32) keys[w][i] = ~0ull;
        __syncwarp();
        // bitonic sort of (pair, slot)
        for (int kk = 2; kk <= m2; kk <<= 1)
          for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int i = lane; i < m2; i += 32) {
              const int l = i ^ jj;
              if (l > i) {
                const unsigned long long a = keys[w][i], c = keys[w][l];
                if ((a > c) == ((i & kk) == 0)) {
                  keys[w][i] = c;
                  keys[w][l] = a;
                }
              }
            }
            __syncwarp();
          }
        // shared nodes: runs of equal pairs
        int ng = 0;
        for (int c = 0; c < m; c += 32) {
          const int i = c + lane;
          bool start = false;
          int32_t o = 0;
          if (i < m) {
            o = v.sh_slot[O + (int)(keys[w][i] & 0xFFFFFFFFu)];
            start = i == 0 || (keys[w][i] >> 32) != (keys[w][i - 1] >> 32);
          }
          const unsigned bal = __ballot_sync(0xffffffffu, start);
          const int x = ng + __popc(bal & ((1u << lane) - 1u)) + (start ? 0 : -1);
          if (i < m) {
            v.sh_sorted[O + i] = o;
            if (x < kUMaxGamma) v.o_x[o] = O + x;
            if (start && x < kUMaxGamma) {
              v.g_u[O + x] = (int32_t)(keys[w][i] >> 32);
              v.g_beg[O + x] = O + i;
            }
          }
          ng += __popc(bal);
        }
        bad = ng > kUMaxGamma;
        ng_seen = ng;
        if (!bad) {
          __syncwarp();
          for (int x = lane; x < ng; x += 32)
            v.g_cnt[O + x] = (x + 1 < ng ? v.g_beg[O + x + 1] : O + m) - v.g_beg[O + x];
          // per piece: its shared slots (slot order is piece order) and G^-1 offsets
          int gb = 0, gn = 0;
          if (lane < k) {
            const int b0 = O + v.pu_base[e0 + lane];
            const int b1 = lane + 1 < k ? O + v.pu_base[e0 + lane + 1] : O + nocc;
            int lo = 0, hi = m;                            // first slot with occurrence >= b0
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              if (v.sh_slot[O + mid] < b0) lo = mid + 1; else hi = mid;
            }
            gb = lo;
            hi = m;                                          // first slot with occurrence >= b1
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              if (v.sh_slot[O + mid] < b1) lo = mid + 1; else hi = mid;
            }
            gn = lo - gb;
          }
          bad = __any_sync(0xffffffffu, gn > kUMaxGp);
          int gtot;
          const int goff = warp_exscan(gn * gn, lane, &gtot);
          if (lane < k) {
            v.pu_gb[e0 + lane] = gb;
            v.pu_gn[e0 + lane] = gn;
            v.pu_ginv[e0 + lane] = goff;
          }
          if (lane == 0) {
            v.u_m[u] = m;
            if (!bad) v.u_ng[u] = ng;
            v.u_gsz[u] = bad ? 0 : gtot;
            v.u_ssz[u] = bad ? 0 : ng * ng;
          }
        }
      }
    }
    if (bad && lane == 0) {
      v.u_gsz[u] = 0;
      v.u_ssz[u] = 0;
      give_up_unit(v, u, k > kUMaxPieces ? 0 : (m_seen > kUMaxShared ? 1 : (ng_seen > kUMaxGamma ? 2 : 3)));
    }
  }
}

// the small classes by one warp per matrix in shared memory (many warps per
// SM; the strip form below pays for its registers in occupancy there):
// (A_p[G,G])^-1 of every piece of every valid unit (one warp per piece)
// pieces with MINN < g_p <= MAXN shared nodes (one launch per size class: the
// small ones with little shared memory per warp, hence many warps per SM)
template <int MINN, int MAXN, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_u_ginv_w(StepView v) {
  __shared__ float Ms[WARPS][MAXN * MAXN];
  __shared__ int Is[WARPS][MAXN];     // the shared members' rows in the piece inverse
  if (aborted(v)) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int32_t npe = v.unit_off[v.wfast[kWUnits]];
  for (int32_t pe = gwarp(); pe < npe; pe += nwarps()) {
    const int32_t u = v.pu_unit[pe];
    const int gn = v.pu_gn[pe];
    if (v.u_ng[u] < 0 || gn <= MINN || gn > MAXN) continue;
    const int32_t O = v.uocc_off[u];
    const int32_t g = v.unit_pieces[pe];
    const int n = v.piece_node_off[g + 1] - v.piece_node_off[g];
    const float* A = v.piece_inv + v.piece_inv_off[g];
    const int gb = v.pu_gb[pe];
    float* M = Ms[w];
    const int64_t dst_off = (int64_t)v.u_goff[u] + v.pu_ginv[pe];
    if (dst_off + (int64_t)gn * gn > v.ginv_cap) {
      if (lane == 0) give_up_unit(v, u, 6);
      continue;
    }
    int* I = Is[w];
    for (int c = lane; c < gn; c += 32) I[c] = v.o_i[v.sh_slot[O + gb + c]];
    __syncwarp();
    for (int c = lane; c < gn; c += 32) {
      const float* Ac = A + I[c];
#pragma unroll 8
      for (int a = 0; a < gn; ++a) M[a * gn + c] = __ldg(Ac + (size_t)I[a] * n);
    }
    __syncwarp();
    const bool ok = warp_gj(M, gn, lane);
    if (!ok) {
      if (lane == 0) give_up_unit(v, u, 4);
      continue;
    }
    float* dst = v.ginv_pool + dst_off;
    for (int t = lane; t < gn * gn; t += 32) dst[t] = M[t];
    __syncwarp();
  }
}

// S = sum_p R_p^T (A_p[G,G])^-1 R_p - lambda diag(c - 1), then S^-1 (one warp per unit)
template <int MINN, int MAXN, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_u_sinv_w(StepView v) {
  __shared__ float Ss[WARPS][MAXN * MAXN];
  __shared__ int Xs[WARPS][kUMaxGp];   // a piece's shared members as indices into S
  if (aborted(v)) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int32_t nu = v.wfast[kWUnits];
  const float lam = v.lam;
  for (int32_t u = gwarp(); u < nu; u += nwarps()) {
    const int ng = v.u_ng[u];
    if (ng <= MINN || ng > MAXN) continue;
    const int32_t O = v.uocc_off[u], e0 = v.unit_off[u];
    const int k = v.unit_off[u + 1] - e0;
    if ((int64_t)v.u_soff[u] + (int64_t)ng * ng > v.sinv_cap || (int64_t)v.u_goff[nu] > v.ginv_cap) {
      if (lane == 0) give_up_unit(v, u, 6);
      continue;
    }
    float* S = Ss[w];
    for (int t = lane; t < ng * ng; t += 32) S[t] = 0.f;
    __syncwarp();
    for (int p = 0; p < k; ++p) {           // pieces in order: a fixed summation order
      const int gn = v.pu_gn[e0 + p], gb = v.pu_gb[e0 + p];
      if (gn == 0) continue;
      const float* G = v.ginv_pool + v.u_goff[u] + v.pu_ginv[e0 + p];
      int* X = Xs[w];
      for (int c = lane; c < gn; c += 32) X[c] = v.o_x[v.sh_slot[O + gb + c]] - O;
      __syncwarp();
      for (int c = lane; c < gn; c += 32) {
        const int xc = X[c];
#pragma unroll 4
        for (int a = 0; a < gn; ++a) S[X[a] * ng + xc] += G[a * gn + c];
      }
      __syncwarp();
    }
    for (int x = lane; x < ng; x += 32) S[x * ng + x] -= lam * (float)(v.g_cnt[O + x] - 1);
    __syncwarp();
    if (!warp_gj(S, ng, lane)) {
      if (lane == 0) give_up_unit(v, u, 5);
      continue;
    }
    float* dst = v.sinv_pool + v.u_soff[u];
    for (int t = lane; t < ng * ng; t += 32) dst[t] = S[t];
    __syncwarp();
  }
}

// (A_p[G,G])^-1 of every piece of every valid unit whose number of shared
// members g_p lies in (MINN, MAXN]: one group of NT threads per piece (strip_gj;
// GROUPS groups per CTA), the matrix gathered straight into registers
template <int MINN, int MAXN, int NP, int RB, int NT, int GROUPS>
__global__ void __launch_bounds__(NT * GROUPS) k_u_ginv(StepView v) {
  static_assert(MAXN <= NP && (NT == 32 || GROUPS == 1), "group shape");
  __shared__ float Cs[GROUPS][2 * NP], Rs[GROUPS][2 * NP];
  __shared__ int Is[GROUPS][NP];      // the shared members' rows in the piece inverse
  __shared__ int flag[GROUPS];
  if (aborted_cta(v)) return;
  const int grp = threadIdx.x / NT, t = threadIdx.x % NT;
  const int j = t % NP, rb = t / NP;
  const int32_t npe = v.unit_off[v.wfast[kWUnits]];
  for (int32_t pe = blockIdx.x * GROUPS + grp; pe < npe; pe += gridDim.x * GROUPS) {
    const int32_t u = v.pu_unit[pe];
    const int gn = v.pu_gn[pe];
    if (gn <= MINN || gn > MAXN) continue;
    if (group_read<NT>(&v.u_ng[u], t, &flag[grp]) < 0) continue;
    const int32_t O = v.uocc_off[u];
    const int32_t g = v.unit_pieces[pe];
    const int n = v.piece_node_off[g + 1] - v.piece_node_off[g];
    const float* A = v.piece_inv + v.piece_inv_off[g];
    const int gb = v.pu_gb[pe];
    const int64_t dst_off = (int64_t)v.u_goff[u] + v.pu_ginv[pe];
    if (dst_off + (int64_t)gn * gn > v.ginv_cap) {
      if (t == 0) give_up_unit(v, u, 6);
      continue;
    }
    // the index chain (slot -> occurrence -> member) once per member
    int* I = Is[grp];
    for (int c = t; c < gn; c += NT) I[c] = v.o_i[v.sh_slot[O + gb + c]];
    group_sync<NT>();
    float m[RB];
    const int ij = j < gn ? I[j] : 0;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int i = rb * RB + r;
      m[r] = (i < gn && j < gn) ? __ldg(A + (size_t)I[i] * n + ij) : (i == j ? 1.f : 0.f);
    }
    if (!strip_gj<NP, RB, NT>(m, t, Cs[grp], Rs[grp])) {
      if (t == 0) give_up_unit(v, u, 4);
      continue;
    }
    float* dst = v.ginv_pool + dst_off;
    if (j < gn) {
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const int i = rb * RB + r;
        if (i < gn) dst[i * gn + j] = m[r];
      }
    }
  }
}

// S = sum_p R_p^T (A_p[G,G])^-1 R_p - lambda diag(c - 1) assembled in shared
// memory (pieces in order: a fixed summation order), then S^-1 by strip_gj in
// registers; units with MINN < ng <= MAXN, one group of NT threads per unit
template <int MINN, int MAXN, int NP, int RB, int NT, int GROUPS>
__global__ void __launch_bounds__(NT * GROUPS) k_u_sinv(StepView v) {
  static_assert(MAXN <= NP && (NT == 32 || GROUPS == 1), "group shape");
  __shared__ float Ss[GROUPS][MAXN * MAXN];
  __shared__ float Cs[GROUPS][2 * NP], Rs[GROUPS][2 * NP];
  __shared__ int Xs[GROUPS][kUMaxGp];   // a piece's shared members as indices into S
  __shared__ int flag[GROUPS];
  if (aborted_cta(v)) return;
  const int grp = threadIdx.x / NT, t = threadIdx.x % NT;
  const int j = t % NP, rb = t / NP;
  const int32_t nu = v.wfast[kWUnits];
  const float lam = v.lam;
  for (int32_t u = blockIdx.x * GROUPS + grp; u < nu; u += gridDim.x * GROUPS) {
    const int ng = group_read<NT>(&v.u_ng[u], t, &flag[grp]);
    if (ng <= MINN || ng > MAXN) continue;
    const int32_t O = v.uocc_off[u], e0 = v.unit_off[u];
    const int k = v.unit_off[u + 1] - e0;
    if ((int64_t)v.u_soff[u] + (int64_t)ng * ng > v.sinv_cap || (int64_t)v.u_goff[nu] > v.ginv_cap) {
      if (t == 0) give_up_unit(v, u, 6);
      continue;
    }
    float* S = Ss[grp];
    for (int q = t; q < ng * ng; q += NT) S[q] = 0.f;
    group_sync<NT>();
    int* X = Xs[grp];
    for (int p = 0; p < k; ++p) {
      const int gn = v.pu_gn[e0 + p], gb = v.pu_gb[e0 + p];
      if (gn == 0) continue;
      const float* G = v.ginv_pool + v.u_goff[u] + v.pu_ginv[e0 + p];
      for (int c = t; c < gn; c += NT) X[c] = v.o_x[v.sh_slot[O + gb + c]] - O;
      group_sync<NT>();
      // thread t adds the entries (a, c) with c = t % gn .. of its column
      for (int q = t; q < gn * gn; q += NT) {
        const int a = q / gn, c = q - a * gn;
        S[X[a] * ng + X[c]] += G[q];
      }
      group_sync<NT>();
    }
    for (int x = t; x < ng; x += NT) S[x * ng + x] -= lam * (float)(v.g_cnt[O + x] - 1);
    group_sync<NT>();
    float m[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int i = rb * RB + r;
      m[r] = (i < ng && j < ng) ? S[i * ng + j] : (i == j ? 1.f : 0.f);
    }
    if (!strip_gj<NP, RB, NT>(m, t, Cs[grp], Rs[grp])) {
      if (t == 0) give_up_unit(v, u, 5);
      continue;
    }
    float* dst = v.sinv_pool + v.u_soff[u];
    if (j < ng) {
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const int i = rb * RB + r;
        if (i < ng) dst[i * ng + j] = m[r];
      }
    }
  }
}

// the same for units with MINN < ng <= NP whose S does not fit in static shared
// memory: one CTA per unit from the work cursor wfast[CURSOR], S assembled in
// dynamic shared memory (NP x NP floats), S^-1 by strip_gj in registers
template <int MINN, int NP, int RB, int NT, int CURSOR>
__global__ void __launch_bounds__(NT) k_u_sinv_d(StepView v) {
  extern __shared__ __align__(16) float Sd[];
  __shared__ float Cs[2 * NP], Rs[2 * NP];
  __shared__ int Xs[kUMaxGp];
  __shared__ int cur;
  if (aborted_cta(v)) return;
  const int t = threadIdx.x;
  const int j = t % NP, rb = t / NP;
  const int32_t nu = v.wfast[kWUnits];
  const float lam = v.lam;
  for (;;) {
    __syncthreads();
    if (t == 0) cur = atomicAdd(&v.wfast[CURSOR], 1);
    __syncthreads();
    const int32_t u = cur;
    if (u >= nu) break;
    const int ng = v.u_ng[u];
    if (ng <= MINN || ng > NP) continue;
    const int32_t O = v.uocc_off[u], e0 = v.unit_off[u];
    const int k = v.unit_off[u + 1] - e0;
    if ((int64_t)v.u_soff[u] + (int64_t)ng * ng > v.sinv_cap || (int64_t)v.u_goff[nu] > v.ginv_cap) {
      if (t == 0) give_up_unit(v, u, 6);
      continue;
    }
    for (int q = t; q < ng * ng; q += NT) Sd[q] = 0.f;
    __syncthreads();
    for (int p = 0; p < k; ++p) {           // pieces in order: a fixed summation order
      const int gn = v.pu_gn[e0 + p], gb = v.pu_gb[e0 + p];
      if (gn == 0) continue;
      const float* G = v.ginv_pool + v.u_goff[u] + v.pu_ginv[e0 + p];
      for (int c = t; c < gn; c += NT) Xs[c] = v.o_x[v.sh_slot[O + gb + c]] - O;
      __syncthreads();
      for (int q = t; q < gn * gn; q += NT) {
        const int a = q / gn, c = q - a * gn;
        Sd[Xs[a] * ng + Xs[c]] += G[q];
      }
      __syncthreads();
    }
    for (int x = t; x < ng; x += NT) Sd[x * ng + x] -= lam * (float)(v.g_cnt[O + x] - 1);
    __syncthreads();
    float m[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const int i = rb * RB + r;
      m[r] = (i < ng && j < ng) ? Sd[i * ng + j] : (i == j ? 1.f : 0.f);
    }
    if (!strip_gj<NP, RB, NT>(m, t, Cs, Rs)) {
      if (t == 0) give_up_unit(v, u, 5);
      continue;
    }
    float* dst = v.sinv_pool + v.u_soff[u];
    if (j < ng) {
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const int i = rb * RB + r;
        if (i < ng) dst[i * ng + j] = m[r];
      }
    }
  }
}

// the same for units with more than 128 shared nodes: one CTA per
// unit (taken from a work cursor, so that no CTA solves two of the few large
// units while others idle), S in dynamic shared memory, Gauss-Jordan sweeps by
// the whole CTA (warps take rows, lanes columns)
__global__ void __launch_bounds__(256) k_u_sinv_big(StepView v) {
  extern __shared__ __align__(16) float Sb[];
  __shared__ int Xb[kUMaxGp];         // a piece's shared members as indices into S
  if (aborted_cta(v)) return;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int32_t nu = v.wfast[kWUnits];
  const float lam = v.lam;
  __shared__ int bad, cur;
  for (;;) {
    __syncthreads();
    if (tid == 0) cur = atomicAdd(&v.wfast[kWCursorS], 1);
    __syncthreads();
    const int32_t u = cur;
    if (u >= nu) break;
    const int ng = v.u_ng[u];
    if (ng <= 128) continue;
    const int32_t O = v.uocc_off[u], e0 = v.unit_off[u];
    const int k = v.unit_off[u + 1] - e0;
    if ((int64_t)v.u_soff[u] + (int64_t)ng * ng > v.sinv_cap || (int64_t)v.u_goff[nu] > v.ginv_cap) {
      if (tid == 0) give_up_unit(v, u, 6);
      continue;
    }
    for (int t = tid; t < ng * ng; t += nt) Sb[t] = 0.f;
    __syncthreads();
    for (int p = 0; p < k; ++p) {           // pieces in order: a fixed summation order
      const int gn = v.pu_gn[e0 + p], gb = v.pu_gb[e0 + p];
      const float* G = v.ginv_pool + v.u_goff[u] + v.pu_ginv[e0 + p];
      for (int c = tid; c < gn; c += nt) Xb[c] = v.o_x[v.sh_slot[O + gb + c]] - O;
      __syncthreads();
      for (int a = wid; a < gn; a += nw) {
        const int xa = Xb[a];
        for (int c = lane; c < gn; c += 32) Sb[xa * ng + Xb[c]] += G[a * gn + c];
      }
      __syncthreads();
    }
    for (int x = tid; x < ng; x += nt) Sb[x * ng + x] -= lam * (float)(v.g_cnt[O + x] - 1);
    if (tid == 0) bad = 0;
    for (int kk = 0; kk < ng; ++kk) {
      __syncthreads();
      const float pv = Sb[kk * ng + kk];
      if (!(pv > 0.f)) {
        if (tid == 0) bad = 1;
        break;
      }
      const float ip = 1.f / pv;
      for (int i = wid; i < ng; i += nw) {
        if (i == kk) continue;
        const float mik = Sb[i * ng + kk] * ip;
        for (int j = lane; j < ng; j += 32)
          if (j != kk) Sb[i * ng + j] = fmaf(-mik, Sb[kk * ng + j], Sb[i * ng + j]);
      }
      __syncthreads();
      for (int t = tid; t < ng; t += nt)
        if (t != kk) {
          Sb[t * ng + kk] = -Sb[t * ng + kk] * ip;
          Sb[kk * ng + t] = Sb[kk * ng + t] * ip;
        }
      __syncthreads();
      if (tid == 0) Sb[kk * ng + kk] = ip;
    }
    __syncthreads();
    if (bad) {
      if (tid == 0) give_up_unit(v, u, 5);
      continue;
    }
    float* dst = v.sinv_pool + v.u_soff[u];
    for (int t = tid; t < ng * ng; t += nt) dst[t] = Sb[t];
    __syncthreads();
  }
}

// ------------------------------------------------------------------ rounds
// u, z = 0, f = u for every occurrence and shared node of the valid units
__global__ void k_u_init(StepView v) {
  if (aborted(v)) return;
  const int64_t tot = v.uocc_off[v.wfast[kWUnits]];
  if (tot > v.u_cap) return;                 // over capacity: every unit is invalid
  for (int32_t o = blockIdx.x * blockDim.x + threadIdx.x; o < tot; o += gridDim.x * blockDim.x) {
    const int32_t u = v.o_unit[o];
    const int ng = v.u_ng[u];
    if (ng < 0) continue;
    if (v.o_x[o] < 0) {
      const int32_t uu = v.o_u[o];
      const float h = v.rhs[uu], l = v.rhs_lo[uu];
      v.o_uh[o] = h;
      v.o_ul[o] = l;
      v.o_zh[o] = 0.f;
      v.o_zl[o] = 0.f;
      v.o_f[o] = h + l;
    }
    const int x = o - v.uocc_off[u];          // the same slot as a shared node index
    if (x < ng) {
      const int32_t uu = v.g_u[o];
      const float h = v.rhs[uu], l = v.rhs_lo[uu];
      v.g_uh[o] = h;
      v.g_ul[o] = l;
      v.g_zh[o] = 0.f;
      v.g_zl[o] = 0.f;
      v.g_f[o] = h + l;
    }
  }
}

// w = A_p[:, I_p] f_I (shared entries count as zero), one row per thread
__global__ void __launch_bounds__(kUTh) k_u_w(StepView v) {
  if (aborted(v)) return;
  const int64_t tot = v.uocc_off[v.wfast[kWUnits]];
  if (tot > v.u_cap) return;                 // over capacity: every unit is invalid
  for (int32_t o = blockIdx.x * blockDim.x + threadIdx.x; o < tot; o += gridDim.x * blockDim.x) {
    if (v.u_ng[v.o_unit[o]] < 0) continue;
    const int32_t g = v.o_g[o];
    const int n = v.piece_node_off[g + 1] - v.piece_node_off[g];
    const int32_t base = v.o_base[o];
    const float* A = v.piece_inv + v.piece_inv_off[g] + v.o_i[o];
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    int j = 0;
    for (; j + 7 < n; j += 8) {
      float a[8], f[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        a[t] = __ldg(A + (size_t)(j + t) * n);
        f[t] = v.o_x[base + j + t] < 0 ? v.o_f[base + j + t] : 0.f;
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) acc[t & 3] = fmaf(a[t], f[t], acc[t & 3]);
    }
    for (; j < n; ++j)
      acc[0] = fmaf(__ldg(A + (size_t)j * n), v.o_x[base + j] < 0 ? v.o_f[base + j] : 0.f, acc[0]);
    v.o_w[o] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  }
}

// the Schur step of a round (one warp per unit): h_p = w[G_p],
// b = f_G + sum_p (A_p[G,G])^-1 h_p, z_G' = S^-1 b, t_p = (A_p[G,G])^-1 (z_G' - h_p)
__global__ void __launch_bounds__(kUWarps * 32) k_u_schur(StepView v) {
  __shared__ float th_s[kUWarps][kUMaxShared];
  __shared__ float b_s[kUWarps][kUMaxGamma];
  if (aborted(v)) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int32_t nu = v.wfast[kWUnits];
  float* th = th_s[w];
  float* bb = b_s[w];
  for (int32_t u = gwarp(); u < nu; u += nwarps()) {
    const int ng = v.u_ng[u];
    if (ng <= 0) continue;
    const int32_t O = v.uocc_off[u], e0 = v.unit_off[u];
    const int k = v.unit_off[u + 1] - e0, m = v.u_m[u];
    for (int t = lane; t < m; t += 32) th[t] = v.o_w[v.sh_slot[O + t]];
    __syncwarp();
    // tt = (A_p[G,G])^-1 h_p
    for (int p = 0; p < k; ++p) {
      const int gn = v.pu_gn[e0 + p], gb = v.pu_gb[e0 + p];
      const float* G = v.ginv_pool + v.u_goff[u] + v.pu_ginv[e0 + p];
      for (int a = lane; a < gn; a += 32) {
        float acc = 0.f;
        for (int c = 0; c < gn; ++c) acc = fmaf(G[c * gn + a], th[gb + c], acc);   // symmetric: column reads
        v.sh_tt[O + gb + a] = acc;
      }
    }
    __syncwarp();
    // b = f_G + the pieces' terms over each shared node's occurrences (piece order)
    for (int x = lane; x < ng; x += 32) {
      float acc = v.g_f[O + x];
      for (int i = v.g_beg[O + x], i1 = i + v.g_cnt[O + x]; i < i1; ++i) acc += v.sh_tt[v.o_t[v.sh_sorted[i]]];
      bb[x] = acc;
    }
    __syncwarp();
    // z_G' = S^-1 b
    const float* Si = v.sinv_pool + v.u_soff[u];
    for (int x = lane; x < ng; x += 32) {
      float acc = 0.f;
      for (int c = 0; c < ng; ++c) acc = fmaf(Si[c * ng + x], bb[c], acc);
      v.g_x[O + x] = acc;
    }
    __syncwarp();
    // t_p = (A_p[G,G])^-1 (z_G' - h_p)
    for (int t = lane; t < m; t += 32) th[t] = v.g_x[v.o_x[v.sh_slot[O + t]]] - th[t];
    __syncwarp();
    for (int p = 0; p < k; ++p) {
      const int gn = v.pu_gn[e0 + p], gb = v.pu_gb[e0 + p];
      const float* G = v.ginv_pool + v.u_goff[u] + v.pu_ginv[e0 + p];
      for (int a = lane; a < gn; a += 32) {
        float acc = 0.f;
        for (int c = 0; c < gn; ++c) acc = fmaf(G[c * gn + a], th[gb + c], acc);   // symmetric: column reads
        v.sh_tt[O + gb + a] = acc;
      }
    }
    __syncwarp();
  }
}

// z_I += w + A_p[I, G_p] t_p (double-float), z_G += z_G'
__global__ void __launch_bounds__(kUTh) k_u_z(StepView v) {
  if (aborted(v)) return;
  const int64_t tot = v.uocc_off[v.wfast[kWUnits]];
  if (tot > v.u_cap) return;                 // over capacity: every unit is invalid
  for (int32_t o = blockIdx.x * blockDim.x + threadIdx.x; o < tot; o += gridDim.x * blockDim.x) {
    const int32_t u = v.o_unit[o];
    const int ng = v.u_ng[u];
    if (ng < 0) continue;
    if (v.o_x[o] < 0) {
      const int32_t g = v.o_g[o], pe = v.o_pe[o];
      const int n = v.piece_node_off[g + 1] - v.piece_node_off[g];
      const float* A = v.piece_inv + v.piece_inv_off[g] + v.o_i[o];
      const int32_t O = v.uocc_off[u];
      const int t0 = O + v.pu_gb[pe], t1 = t0 + v.pu_gn[pe];
      float acc = v.o_w[o], acc2 = 0.f;
      int t = t0;
      for (; t + 3 < t1; t += 4) {
        float x[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = __ldg(A + (size_t)v.o_i[v.sh_slot[t + q]] * n);
        acc = fmaf(x[0], v.sh_tt[t], acc);
        acc2 = fmaf(x[1], v.sh_tt[t + 1], acc2);
        acc = fmaf(x[2], v.sh_tt[t + 2], acc);
        acc2 = fmaf(x[3], v.sh_tt[t + 3], acc2);
      }
      for (; t < t1; ++t) acc = fmaf(__ldg(A + (size_t)v.o_i[v.sh_slot[t]] * n), v.sh_tt[t], acc);
      const df32 z = df_add_f(df32{v.o_zh[o], v.o_zl[o]}, acc + acc2);
      v.o_zh[o] = z.hi;
      v.o_zl[o] = z.lo;
    }
    if (o - v.uocc_off[u] < ng) {
      const df32 z = df_add_f(df32{v.g_zh[o], v.g_zl[o]}, v.g_x[o]);
      v.g_zh[o] = z.hi;
      v.g_zl[o] = z.lo;
    }
  }
}

__device__ __forceinline__ df32 occ_z(const StepView& v, int32_t o) {
  const int32_t x = v.o_x[o];
  return x < 0 ? df32{v.o_zh[o], v.o_zl[o]} : df32{v.g_zh[x], v.g_zl[x]};
}

// residual u - lambda z - B^T B z of interior occurrences (into f); the edge
// partials of shared occurrences (into ph, pl)
__global__ void __launch_bounds__(kUTh) k_u_res(StepView v) {
  if (aborted(v)) return;
  const int64_t tot = v.uocc_off[v.wfast[kWUnits]];
  if (tot > v.u_cap) return;                 // over capacity: every unit is invalid
  const float lam = v.lam;
  for (int32_t o = blockIdx.x * blockDim.x + threadIdx.x; o < tot; o += gridDim.x * blockDim.x) {
    if (v.u_ng[v.o_unit[o]] < 0) continue;
    const df32 zi = occ_z(v, o);
    const int32_t m = v.piece_node_off[v.o_g[o]] + v.o_i[o];
    const int32_t base = v.o_base[o];
    df32 acc = {0.f, 0.f};
#pragma unroll 4
    for (int32_t t = v.mem_rp[m], t1 = v.mem_rp[m + 1]; t < t1; ++t) {
      const float sw = v.edge_sw[t];
      const df32 zo = occ_z(v, base + v.edge_pos[t]);
      acc = df_add(acc, df_mul(df_two_prod(sw, sw), df_add(zi, df32{-zo.hi, -zo.lo})));
    }
    if (v.o_x[o] < 0) {
      df32 rd = df_add(df32{v.o_uh[o], v.o_ul[o]}, df_mul_f(zi, -lam));
      rd = df_add(rd, df32{-acc.hi, -acc.lo});
      v.o_f[o] = rd.hi;
    } else {
      v.o_ph[o] = acc.hi;
      v.o_pl[o] = acc.lo;
    }
  }
}

// residual of the shared nodes: u - lambda z - the occurrences' partials (in order)
__global__ void __launch_bounds__(kUTh) k_u_gres(StepView v) {
  if (aborted(v)) return;
  const int64_t tot = v.uocc_off[v.wfast[kWUnits]];
  if (tot > v.u_cap) return;                 // over capacity: every unit is invalid
  const float lam = v.lam;
  for (int32_t o = blockIdx.x * blockDim.x + threadIdx.x; o < tot; o += gridDim.x * blockDim.x) {
    const int32_t u = v.o_unit[o];
    if (o - v.uocc_off[u] >= v.u_ng[u]) continue;
    df32 acc = {0.f, 0.f};
    for (int i = v.g_beg[o], i1 = i + v.g_cnt[o]; i < i1; ++i) {
      const int32_t s = v.sh_sorted[i];
      acc = df_add(acc, df32{v.o_ph[s], v.o_pl[s]});
    }
    df32 rd = df_add(df32{v.g_uh[o], v.g_ul[o]}, df_mul_f(df32{v.g_zh[o], v.g_zl[o]}, -lam));
    rd = df_add(rd, df32{-acc.hi, -acc.lo});
    v.g_f[o] = rd.hi;
  }
}

// convergence of every valid unit (one warp per unit): |r| <= tol |u|, else the
// general solver takes the step; then z (hi, lo) by unique pair
__global__ void __launch_bounds__(kUWarps * 32) k_u_out(StepView v, float tol) {
  if (aborted(v)) return;
  const int lane = threadIdx.x & 31;
  const int32_t nu = v.wfast[kWUnits];
  for (int32_t u = gwarp(); u < nu; u += nwarps()) {
    const int ng = v.u_ng[u];
    if (ng < 0) continue;
    const int32_t O = v.uocc_off[u];
    const int nocc = v.uocc_off[u + 1] - O;
    float rr = 0.f, uu = 0.f;
    for (int i = lane; i < nocc; i += 32) {
      const int32_t o = O + i;
      if (v.o_x[o] < 0) {
        rr = fmaf(v.o_f[o], v.o_f[o], rr);
        uu = fmaf(v.o_uh[o], v.o_uh[o], uu);
        v.z[v.o_u[o]] = v.o_zh[o];
        v.z_lo[v.o_u[o]] = v.o_zl[o];
      }
      if (i < ng) {
        rr = fmaf(v.g_f[o], v.g_f[o], rr);
        uu = fmaf(v.g_uh[o], v.g_uh[o], uu);
        v.z[v.g_u[o]] = v.g_zh[o];
        v.z_lo[v.g_u[o]] = v.g_zl[o];
      }
    }
    rr = warp_sum(rr);
    uu = warp_sum(uu);
    if (lane == 0) {
      if (rr > tol * tol * uu) flag_general(v);
      atomicMax(&v.wfast[kWRounds], 2);
    }
  }
}

}  // namespace

int units_grid(int num_sms) { return num_sms * 4; }

cudaError_t configure_units_kernels() {
  cudaError_t e = cudaFuncSetAttribute(k_u_sinv_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(kUMaxGamma * kUMaxGamma * sizeof(float)));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_u_sinv_d<96, 128, 32, 512, kWCursorS2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(128 * 128 * sizeof(float)));
}

cudaError_t launch_units(const StepView& v, float tol, int num_sms, cudaStream_t st, cudaEvent_t mid,
                         const Branches* br) {
  const int gw = num_sms * 4;            // CTAs of the per-unit kernels (kUWarps warps each)
  const int gt = num_sms * 8;            // CTAs of the per-occurrence kernels
  int32_t* n_units = v.wfast + kWUnits;
  cudaError_t e;
  k_u_prep<<<gw, kUWarps * 32, 0, st>>>(v);
  k_u_scan<<<1, 1024, 0, st>>>(v.u_nocc, n_units, v.uocc_off, v.u_cap, v.wfast);
  k_u_occ<<<gw * (kUWarps / kUOccWarps), kUOccWarps * 32, 0, st>>>(v);
  k_u_scan<<<1, 1024, 0, st>>>(v.u_gsz, n_units, v.u_goff, v.ginv_cap, v.wfast);
  k_u_scan<<<1, 1024, 0, st>>>(v.u_ssz, n_units, v.u_soff, v.sinv_cap, v.wfast);
  // (A_p[G,G])^-1 and S^-1 by size class: a warp per matrix in shared memory up
  // to 32 nodes, a CTA per matrix in registers above (strips of 16 and 24 rows).
  // The classes of one group take disjoint pieces (units) and write disjoint
  // parts of the pools, so with branch streams they run side by side; every
  // S^-1 waits for all the piece inverses.
  auto fork = [&](int n) -> cudaError_t {
    if (!br) return cudaSuccess;
    cudaError_t r = cudaEventRecord(br->fork, st);
    for (int i = 0; i < n && r == cudaSuccess; ++i) r = cudaStreamWaitEvent(br->s[i], br->fork, 0);
    return r;
  };
  auto join = [&](int n) -> cudaError_t {
    if (!br) return cudaSuccess;
    cudaError_t r = cudaSuccess;
    for (int i = 0; i < n && r == cudaSuccess; ++i) {
      r = cudaEventRecord(br->join[i], br->s[i]);
      if (r == cudaSuccess) r = cudaStreamWaitEvent(st, br->join[i], 0);
    }
    return r;
  };
  auto lane = [&](int i) { return br ? br->s[i] : st; };
  if ((e = fork(2)) != cudaSuccess) return e;
  k_u_ginv<32, 64, 64, 16, 256, 1><<<num_sms * 6, 256, 0, lane(0)>>>(v);
  k_u_ginv<64, 96, 96, 24, 384, 1><<<num_sms * 2, 384, 0, lane(1)>>>(v);
  k_u_ginv_w<0, 32, 8><<<num_sms * 6, 256, 0, st>>>(v);
  if ((e = join(2)) != cudaSuccess) return e;
  if ((e = fork(4)) != cudaSuccess) return e;
  k_u_sinv_big<<<num_sms, 256, kUMaxGamma * kUMaxGamma * sizeof(float), lane(0)>>>(v);
  k_u_sinv_d<96, 128, 32, 512, kWCursorS2><<<num_sms, 512, 128 * 128 * sizeof(float), lane(1)>>>(v);
  k_u_sinv<64, 96, 96, 24, 384, 1><<<num_sms * 2, 384, 0, lane(2)>>>(v);
  k_u_sinv<32, 64, 64, 16, 256, 1><<<num_sms * 6, 256, 0, lane(3)>>>(v);
  k_u_sinv_w<0, 32, 8><<<num_sms * 6, 256, 0, st>>>(v);
  if ((e = join(4)) != cudaSuccess) return e;
  if (mid && (e = cudaEventRecord(mid, st)) != cudaSuccess) return e;
  k_u_init<<<gt, kUTh, 0, st>>>(v);
  for (int r = 0; r < 2; ++r) {
    if (r > 0) {
      k_u_res<<<gt, kUTh, 0, st>>>(v);
      k_u_gres<<<gt, kUTh, 0, st>>>(v);
    }
    k_u_w<<<gt, kUTh, 0, st>>>(v);
    k_u_schur<<<gw, kUWarps * 32, 0, st>>>(v);
    k_u_z<<<gt, kUTh, 0, st>>>(v);
  }
  k_u_res<<<gt, kUTh, 0, st>>>(v);
  k_u_gres<<<gt, kUTh, 0, st>>>(v);
  k_u_out<<<gw, kUWarps * 32, 0, st>>>(v, tol);
  return cudaGetLastError();
}

}  // namespace spider
