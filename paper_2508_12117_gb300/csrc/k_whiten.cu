// Whitening of a minibatch through the precomputed piece inverses (row a5,
// Eq. marginal_sigma by the push-through identity: z = (lambda I + B^T B)^-1 u).
//
// A piece is a connected set of local nodes of one block (see pieces.h); its
// inverse A = (lambda I + B^T B)^-1 was computed once at create.  In a step:
//   * a piece none of whose nodes occurs in another selected block is a whole
//     component of the minibatch system: z = A u, refined with the residual
//     u - K z evaluated in double-float (one warp per piece);
//   * pieces that share nodes (the same (event, station) pair in several
//     selected blocks) form a unit, solved exactly by the Schur complement on
//     the shared nodes Gamma.  For each piece p with interior nodes I_p and
//     shared nodes Gamma_p, and A_p = K_p^-1 partitioned accordingly:
//        S = sum_p R_p^T (A_p[G,G])^-1 R_p - lambda diag(c - 1)
//        S z_G = f_G + sum_p R_p^T (A_p[G,G])^-1 A_p[G,I] f_I
//        z_I = A_p[I,I] f_I + A_p[I,G] (A_p[G,G])^-1 (z_G - A_p[G,I] f_I)
//     (c = the number of pieces holding a shared node; each piece's matrix
//     carries lambda once, the unit's matrix once per node), refined like the
//     single pieces: by the data-parallel unit solver (k_units.cu), and the
//     units beyond its limits here, one CTA per unit in two passes by size
//     (k_whiten_units, MODE 1 and 2).
// A unit beyond every limit, or one that does not converge, sets a flag on
// which the general component solver then runs for the whole step.
// Every sum runs in a fixed order, so the result is reproducible.
#include <cuda_runtime.h>

#include "dfloat.cuh"
#include "kernels.h"
#include "step_util.cuh"

namespace spider {

namespace {

constexpr int kPieceMaxDev = 256;   // largest piece (the host builds no larger one)
constexpr int kCleanWarps = 8;
constexpr int kRounds = 6;          // refinement rounds (the first is the plain solve)
constexpr int kUGamma = 256;        // shared nodes of a unit solved directly (last pass)
constexpr int kUGinv = 65536;       // floats for the pieces' (A_p[G,G])^-1
}  // namespace
// global scratch of one CTA of the unit solver: S^-1, then the pieces' inverses
constexpr int64_t kUScratch = (int64_t)kUGamma * kUGamma + kUGinv;
namespace {

// ------------------------------------------------------------------ labels
// labels and flags of the pieces of each selected block (one CTA per block)
__global__ void k_piece_init(StepView v) {
  const int32_t b = v.sel[blockIdx.x];
  const int32_t g0 = v.blk_piece_off[b], g1 = v.blk_piece_off[b + 1];
  for (int32_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
    v.plab[g] = g;
    v.pmulti[g] = 0;
    v.pcount[g] = 0;
  }
  __syncthreads();
  const int32_t q0 = v.blk_node_off[b], q1 = v.blk_node_off[b + 1];
  for (int32_t q = q0 + threadIdx.x; q < q1; q += blockDim.x)
    if (v.multi[q]) v.pmulti[g0 + v.node_piece[q]] = 1;   // every writer stores 1
}

__device__ __forceinline__ int32_t plab_root(const int32_t* lab, int32_t g) {
  const volatile int32_t* vl = lab;
  int32_t r = g;
  for (int k = 0; k < 1 << 20; ++k) {
    const int32_t n = vl[r];
    if (n == r) return r;
    r = n;
  }
  return r;
}

// Units: the selected pieces joined through shared pairs.  Every occurrence of
// a shared pair links its piece to the piece of the pair's owner occurrence;
// roots are hooked below smaller roots (atomicMin) and labels compressed, with
// bounded grid-wide barriers, until a round changes nothing (as k_cc does for
// nodes).  Labels end as the smallest piece id of each unit.
constexpr int kPieceRounds = 64;

__global__ void __launch_bounds__(512) k_piece_cc(StepView v, int64_t n_b) {
  __shared__ int any;
  if (aborted_cta(v)) return;
  int32_t* flags = v.wfast + kWSlots;          // one flag per round
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gstride = gridDim.x * blockDim.x;
  for (int i = gtid; i < kPieceRounds; i += gstride) flags[i] = 0;
  if (!grid_barrier(v.counters, v.prm->wait_ns)) return;
  int round = 0;
  for (; round < kPieceRounds; ++round) {
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    int changed = 0;
    for (int64_t sb = blockIdx.x; sb < n_b; sb += gridDim.x) {
      const int32_t b = v.sel[sb];
      const int32_t q0 = v.blk_node_off[b], q1 = v.blk_node_off[b + 1];
      for (int32_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        if (!v.multi[q]) continue;
        const int32_t qo = v.owner_q[q];
        if (qo == q) continue;
        const int32_t bo = v.owner_b[q];
        const int32_t ga = plab_root(v.plab, v.blk_piece_off[b] + v.node_piece[q]);
        const int32_t gb = plab_root(v.plab, v.blk_piece_off[bo] + v.node_piece[qo]);
        if (ga == gb) continue;
        const int32_t lo = ga < gb ? ga : gb, hi = ga < gb ? gb : ga;
        if (atomicMin(&v.plab[hi], lo) > lo) changed = 1;
      }
    }
    if (changed) any = 1;
    __syncthreads();
    if (threadIdx.x == 0 && any) flags[round] = 1;
    if (!grid_barrier(v.counters, v.prm->wait_ns)) return;
    for (int64_t sb = blockIdx.x; sb < n_b; sb += gridDim.x) {
      const int32_t b = v.sel[sb];
      for (int32_t g = v.blk_piece_off[b] + threadIdx.x; g < v.blk_piece_off[b + 1]; g += blockDim.x)
        v.plab[g] = plab_root(v.plab, g);
    }
    if (!grid_barrier(v.counters, v.prm->wait_ns)) return;
    if (((volatile int32_t*)flags)[round] == 0) break;
  }
  if (round == kPieceRounds) {
    if (gtid == 0) set_error(v.counters, SPIDER_E_TIMEOUT);
    return;
  }
  // pieces per unit, counted at the root
  for (int64_t sb = blockIdx.x; sb < n_b; sb += gridDim.x) {
    const int32_t b = v.sel[sb];
    for (int32_t g = v.blk_piece_off[b] + threadIdx.x; g < v.blk_piece_off[b + 1]; g += blockDim.x)
      if (v.pmulti[g]) atomicAdd(&v.pcount[v.plab[g]], 1);
  }
}

// unit ids for the roots, and the list of single pieces (arbitrary order: a
// unit's or a piece's result does not depend on it)
__global__ void k_unit_ids(StepView v) {
  if (aborted(v)) return;
  const int32_t b = v.sel[blockIdx.x];
  for (int32_t g = v.blk_piece_off[b] + threadIdx.x; g < v.blk_piece_off[b + 1]; g += blockDim.x) {
    if (v.pmulti[g] && v.plab[g] == g) {
      const int32_t u = atomicAdd(&v.wfast[kWUnits], 1);
      v.unit_of[g] = u;
      v.unit_cnt[u] = v.pcount[g];
    } else if (!v.pmulti[g]) {
      const int32_t c = atomicAdd(&v.wfast[kWClean], 1);
      v.clean_list[c] = g;
      v.clean_blk[c] = b;
    }
  }
}

// exclusive scan of the pieces per unit (one CTA)
__global__ void k_unit_scan(StepView v) {
  __shared__ int sm[33];
  if (aborted_cta(v)) return;
  const int32_t nu = v.wfast[kWUnits];
  int carry = 0;
  for (int32_t c = 0; c < nu; c += blockDim.x) {
    const int32_t u = c + threadIdx.x;
    const int val = u < nu ? v.unit_cnt[u] : 0;
    int total;
    const int pre = block_exscan(val, sm, &total);
    if (u < nu) v.unit_off[u] = carry + pre;
    carry += total;
  }
  if (threadIdx.x == 0) v.unit_off[nu] = carry;
}

__global__ void k_unit_fill(StepView v) {
  if (aborted(v)) return;
  const int32_t b = v.sel[blockIdx.x];
  for (int32_t g = v.blk_piece_off[b] + threadIdx.x; g < v.blk_piece_off[b + 1]; g += blockDim.x)
    if (v.pmulti[g]) {
      const int32_t u = v.unit_of[v.plab[g]];
      const int32_t pos = atomicSub(&v.unit_cnt[u], 1) - 1;
      v.unit_pieces[v.unit_off[u] + pos] = g;
      v.unit_pblk[v.unit_off[u] + pos] = b;
    }
}

// ------------------------------------------------------------------ single pieces
// y = A x for one piece held by a warp: A is n x n, symmetric, stored whole, so
// lane i reads A[j][i] over j (consecutive lanes, consecutive words); four
// rows of A in flight per lane.
template <int NS>
__device__ __forceinline__ void warp_matvec(const float* __restrict__ A, int n, const float* x, float* y,
                                            int lane) {
  float acc[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) acc[s] = 0.f;
  int j = 0;
  for (; j + 7 < n; j += 8) {
    const float* r0 = A + (size_t)j * n;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const int i = lane + 32 * s;
      if (i < n) {
        float a[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) a[t] = __ldg(r0 + (size_t)t * n + i);
#pragma unroll
        for (int t = 0; t < 8; ++t) acc[s] = fmaf(a[t], x[j + t], acc[s]);
      }
    }
  }
  for (; j < n; ++j) {
    const float xj = x[j];
    const float* row = A + (size_t)j * n;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const int i = lane + 32 * s;
      if (i < n) acc[s] = fmaf(__ldg(row + i), xj, acc[s]);
    }
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const int i = lane + 32 * s;
    if (i < n) y[i] = acc[s];
  }
}

__device__ __forceinline__ void warp_matvec_n(const float* A, int n, const float* x, float* y, int lane) {
  if (n <= 32) warp_matvec<1>(A, n, x, y, lane);
  else if (n <= 64) warp_matvec<2>(A, n, x, y, lane);
  else if (n <= 128) warp_matvec<4>(A, n, x, y, lane);
  else warp_matvec<8>(A, n, x, y, lane);
}

// sum over member m's edges of w_e (z_i - z_other) in double-float; zi is the
// member's own value, zoth(j) the value of the member at position j
template <typename ZF>
__device__ __forceinline__ df32 member_bz(const StepView& v, int32_t m, df32 zi, ZF zoth) {
  df32 acc = {0.f, 0.f};
#pragma unroll 4
  for (int32_t t = v.mem_rp[m], t1 = v.mem_rp[m + 1]; t < t1; ++t) {
    const float sw = v.edge_sw[t];
    const df32 zo = zoth((int)v.edge_pos[t]);
    acc = df_add(acc, df_mul(df_two_prod(sw, sw), df_add(zi, df32{-zo.hi, -zo.lo})));
  }
  return acc;
}

struct CleanWarp {
  float uh[kPieceMaxDev], ul[kPieceMaxDev];
  float zh[kPieceMaxDev], zl[kPieceMaxDev];
  float r[kPieceMaxDev], dz[kPieceMaxDev];
};

// Persistent warps over the step's single pieces (one piece at a time each).
__global__ void __launch_bounds__(kCleanWarps * 32) k_whiten_clean(StepView v, float tol) {
  __shared__ CleanWarp sw_[kCleanWarps];
  if (aborted_cta(v)) return;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  CleanWarp& S = sw_[w];
  const float lam = v.lam;
  const int32_t nclean = v.wfast[kWClean];
  int max_rounds = 0;
  for (;;) {
    int32_t c = 0;
    if (lane == 0) c = atomicAdd(&v.wfast[kWCursorC], 1);
    c = __shfl_sync(0xffffffffu, c, 0);
    if (c >= nclean) break;
    const int32_t g = v.clean_list[c];
    const int32_t q0 = v.blk_node_off[v.clean_blk[c]];
    const int32_t m0 = v.piece_node_off[g];
    const int n = v.piece_node_off[g + 1] - m0;
    const float* A = v.piece_inv + v.piece_inv_off[g];
    float uu = 0.f;
    for (int i = lane; i < n; i += 32) {
      const int32_t u = v.loc2u[q0 + v.piece_nodes[m0 + i]];
      S.uh[i] = v.rhs[u];
      S.ul[i] = v.rhs_lo[u];
      S.zh[i] = 0.f;
      S.zl[i] = 0.f;
      uu = fmaf(S.uh[i], S.uh[i], uu);
    }
    uu = warp_sum(uu);
    __syncwarp();
    int round = 0;
    bool done = false;
    for (; round < kRounds; ++round) {
      float rr = 0.f;
      for (int i = lane; i < n; i += 32) {
        float r;
        if (round == 0) {
          r = S.uh[i] + S.ul[i];
        } else {
          const df32 zi = {S.zh[i], S.zl[i]};
          const df32 bz = member_bz(v, m0 + i, zi, [&](int j) { return df32{S.zh[j], S.zl[j]}; });
          df32 rd = df_add(df32{S.uh[i], S.ul[i]}, df_mul_f(zi, -lam));
          rd = df_add(rd, df32{-bz.hi, -bz.lo});
          r = rd.hi;
        }
        S.r[i] = r;
        rr = fmaf(r, r, rr);
      }
      rr = warp_sum(rr);
      __syncwarp();
      if (rr <= tol * tol * uu) {
        done = true;
        break;
      }
      warp_matvec_n(A, n, S.r, S.dz, lane);
      __syncwarp();
      for (int i = lane; i < n; i += 32) {
        const df32 z = df_add_f(df32{S.zh[i], S.zl[i]}, S.dz[i]);
        S.zh[i] = z.hi;
        S.zl[i] = z.lo;
      }
      __syncwarp();
    }
    if (!done && lane == 0) atomicExch(&v.wfast[kWGeneral], 1);
    if (round > max_rounds) max_rounds = round;
    for (int i = lane; i < n; i += 32) {
      const int32_t u = v.loc2u[q0 + v.piece_nodes[m0 + i]];
      v.z[u] = S.zh[i];
      v.z_lo[u] = S.zl[i];
    }
    __syncwarp();
  }
  if (lane == 0 && max_rounds > 0) atomicMax(&v.wfast[kWRounds], max_rounds);
}

// ------------------------------------------------------------------ units
// Two CTA passes over the units the data-parallel unit solver (k_units.cu)
// handed over, the first deferring what exceeds its shared memory to the
// second: 256-thread CTAs, two per SM (S^-1 of up to 64 shared nodes in shared
// memory), then one CTA per SM (up to 160; beyond that the CTA's global
// scratch holds S^-1 and the pieces' small inverses).
template <int PC, int OCC, int GAM, int SMG, int SMGINV>
struct UnitSmem {
  int32_t pg[PC];                  // piece ids (ascending)
  int32_t pb[PC];                  // their blocks
  int32_t pm0[PC];                 // first member (piece_nodes numbering) of each piece
  int32_t pq0[PC];                 // first local node of the piece's block
  int32_t pbase[PC + 1];           // first occurrence slot of each piece
  int32_t pgb[PC + 1];             // first entry of each piece's shared list
  int32_t pginv[PC + 1];           // offset of each piece's (A_p[G,G])^-1
  int32_t ou[OCC];                 // occurrence -> unique pair
  int16_t og[OCC];                 // occurrence -> shared node index, -1 interior
  int16_t opc[OCC];                // occurrence -> piece
  int16_t gl[OCC];                 // shared occurrences in slot order (per piece, member order)
  float uh[OCC], ul[OCC];          // u of interior occurrences
  float zh[OCC], zl[OCC];          // z of interior occurrences
  float f[OCC];                    // right-hand side of the round (interior)
  float w[OCC];                    // A_p[:, I] f_I
  float ph[OCC], pl[OCC];          // residual partial of a shared occurrence
  float th[OCC], tt[OCC];          // h_p and (A_p[G,G])^-1 h_p, per shared occurrence
  int32_t key[2 * OCC];            // shared occurrences sorted by (pair, slot)
  int32_t gu[GAM];                 // shared node -> unique pair
  int32_t gbeg[GAM + 1];           // shared node -> its run in key
  float guh[GAM], gul[GAM], gzh[GAM], gzl[GAM], gf[GAM], gb[GAM], gx[GAM];
  float s_sm[SMG * SMG];           // S^-1 when it fits
  float ginv_sm[SMGINV];           // the pieces' small inverses when they fit
  int32_t scan[33];
  float red[32];
  int32_t flag;
  int32_t cnt;
  int32_t tot;
};

__device__ __forceinline__ float cta_sum(float x, float* red) {
  x = warp_sum(x);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = x;
  __syncthreads();
  float s = 0.f;
  for (int k = 0; k < nw; ++k) s += red[k];
  __syncthreads();
  return s;
}

// In-place inverse of the symmetric positive definite n x n matrix M
// (row-major) by Gauss-Jordan sweeps without pivoting (every pivot is a
// diagonal entry of a Schur complement of M, hence positive): sweeping pivot k
// maps M[k][k] -> 1 / p, row k -> M[k][j] / p, column k -> -M[i][k] / p and
// the rest -> M[i][j] - M[i][k] M[k][j] / p; after all n sweeps M holds M^-1.
// One warp.  Returns false on a non-positive pivot.
__device__ bool warp_spd_inverse(float* M, int n, int lane) {
  for (int k = 0; k < n; ++k) {
    const float p = M[k * n + k];
    if (!(p > 0.f)) return false;
    const float ip = 1.f / p;
    __syncwarp();
    // lane j updates its columns j != k of every row i != k (row k and column k
    // are only read here)
    for (int j = lane; j < n; j += 32) {
      if (j == k) continue;
      const float mkj = M[k * n + j] * ip;
      for (int i = 0; i < n; ++i)
        if (i != k) M[i * n + j] = fmaf(-M[i * n + k], mkj, M[i * n + j]);
    }
    __syncwarp();
    for (int t = lane; t < n; t += 32)
      if (t != k) {
        M[t * n + k] = -M[t * n + k] * ip;
        M[k * n + t] = M[k * n + t] * ip;
      }
    __syncwarp();
    if (lane == 0) M[k * n + k] = ip;
    __syncwarp();
  }
  return true;
}

// the same sweeps by the whole CTA (all threads call it; false on a bad pivot)
__device__ bool cta_spd_inverse(float* M, int n) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int k = 0; k < n; ++k) {
    __syncthreads();
    const float p = M[k * n + k];
    if (!(p > 0.f)) return false;
    const float ip = 1.f / p;
    // warps take rows i != k, lanes columns j != k (row k and column k are
    // only read here)
    for (int i = wid; i < n; i += nw) {
      if (i == k) continue;
      const float mik = M[i * n + k] * ip;
      for (int j = lane; j < n; j += 32)
        if (j != k) M[i * n + j] = fmaf(-mik, M[k * n + j], M[i * n + j]);
    }
    __syncthreads();
    for (int t = tid; t < n; t += nt)
      if (t != k) {
        M[t * n + k] = -M[t * n + k] * ip;
        M[k * n + t] = M[k * n + t] * ip;
      }
    __syncthreads();
    if (tid == 0) M[k * n + k] = ip;
  }
  __syncthreads();
  return true;
}

// exclusive prefix over flags[0, n) by the CTA in chunks; *total = sum
template <typename F>
__device__ void cta_exscan(int n, F flag_of, int* pre_out, int32_t* sm, int32_t* total) {
  int carry = 0;
  for (int c = 0; c < n; c += blockDim.x) {
    const int i = c + threadIdx.x;
    const int val = i < n ? flag_of(i) : 0;
    int t;
    const int pre = block_exscan(val, sm, &t);
    if (i < n) pre_out[i] = carry + pre;
    carry += t;
  }
  if (threadIdx.x == 0) *total = carry;
  __syncthreads();
}

// MODE 1: the units the data-parallel solver handed over; MODE 2: the units
// MODE 1 deferred (the last pass: S^-1 and the small inverses go to global
// scratch when they exceed its shared memory, and a unit beyond PC, OCC or GAM
// hands the step to the general solver).
template <int PC, int OCC, int GAM, int SMG, int SMGINV, int NT, int MODE>
__global__ void __launch_bounds__(NT) k_whiten_units(StepView v, float tol) {
  static_assert(MODE == 1 || MODE == 2, "unit pass");
  extern __shared__ __align__(16) uint8_t smu[];
  using Smem = UnitSmem<PC, OCC, GAM, SMG, SMGINV>;
  Smem& S = *reinterpret_cast<Smem*>(smu);
  if (aborted_cta(v)) return;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const float lam = v.lam;
  const int32_t nu = MODE == 1 ? v.wfast[kWDefer] : v.wfast[kWDefer2];
  // the pass's deferral: the next pass's list, or the general solver after the last
  auto defer = [&](int32_t unit) {
    if (MODE == 1) v.unit_defer2[atomicAdd(&v.wfast[kWDefer2], 1)] = unit;
    else atomicExch(&v.wfast[kWGeneral], 1);
  };
  float* const s_glob = v.wscratch + (int64_t)blockIdx.x * kUScratch;   // S^-1 when it is large
  float* const ginv_glob = s_glob + (int64_t)kUGamma * kUGamma;         // small inverses when many
  int max_rounds = 0;
  for (;;) {
    __syncthreads();
    if (tid == 0) S.cnt = atomicAdd(&v.wfast[MODE == 1 ? kWCursor : kWCursor2], 1);
    __syncthreads();
    if (S.cnt >= nu) break;
    const int32_t u = MODE == 1 ? v.unit_defer[S.cnt] : v.unit_defer2[S.cnt];
    const long long t_unit = clock64();
    int32_t* const dbg = v.wfast + kWSlots + 64 + MODE * 5;
    long long t_ph = t_unit;
    auto phase = [&](int ph) {
      if (tid == 0) {
        const long long t = clock64();
        atomicAdd(&dbg[ph], (int)((t - t_ph) >> 10));
        t_ph = t;
      }
    };
    const int32_t p0 = v.unit_off[u];
    const int k = v.unit_off[u + 1] - p0;
    if (k > PC) {
      if (tid == 0) defer(u);
      continue;
    }
    // pieces ascending (k <= 32, one thread), sizes and bases
    if (tid == 0) {
      for (int i = 0; i < k; ++i) {
        const int32_t g = v.unit_pieces[p0 + i], gbk = v.unit_pblk[p0 + i];
        int j = i;
        while (j > 0 && S.pg[j - 1] > g) {
          S.pg[j] = S.pg[j - 1];
          S.pb[j] = S.pb[j - 1];
          --j;
        }
        S.pg[j] = g;
        S.pb[j] = gbk;
      }
      int base = 0;
      for (int i = 0; i < k; ++i) {
        const int32_t g = S.pg[i];
        S.pm0[i] = v.piece_node_off[g];
        S.pq0[i] = v.blk_node_off[S.pb[i]];
        S.pbase[i] = base;
        base += v.piece_node_off[g + 1] - v.piece_node_off[g];
      }
      S.pbase[k] = base;
      S.flag = base > OCC ? 1 : 0;
    }
    __syncthreads();
    if (S.flag) {
      if (tid == 0) defer(u);
      continue;
    }
    const int nocc = S.pbase[k];
    for (int o = tid; o < nocc; o += nt) {
      int p = 0;
      while (S.pbase[p + 1] <= o) ++p;
      const int32_t q = S.pq0[p] + v.piece_nodes[S.pm0[p] + (o - S.pbase[p])];
      S.ou[o] = v.loc2u[q];
      S.opc[o] = (int16_t)p;
      S.og[o] = v.multi[q] ? 0 : -1;
    }
    __syncthreads();
    // shared occurrences in slot order: positions by a CTA scan of the flags
    cta_exscan(nocc, [&](int o) { return S.og[o] >= 0 ? 1 : 0; }, reinterpret_cast<int*>(S.w), S.scan,
               &S.tot);
    const int m = S.tot;
    for (int o = tid; o < nocc; o += nt) {
      const int pre = reinterpret_cast<int*>(S.w)[o];
      if (S.og[o] >= 0) {
        S.gl[pre] = (int16_t)o;
        S.key[pre] = o;
      }
      for (int p = 0; p <= k; ++p)
        if (S.pbase[p] == o) S.pgb[p] = pre;
    }
    if (tid == 0) {
      S.pgb[k] = m;
      for (int p = k - 1; p >= 0; --p)           // empty trailing pieces
        if (S.pbase[p] == nocc) S.pgb[p] = m;
    }
    int m2 = 1;
    while (m2 < m) m2 <<= 1;
    for (int i = m + tid; i < m2; i += nt) S.key[i] = -1;
    __syncthreads();
    // bitonic sort by (pair, slot); padding last
    for (int kk = 2; kk <= m2; kk <<= 1)
      for (int jj = kk >> 1; jj > 0; jj >>= 1) {
        for (int i = tid; i < m2; i += nt) {
          const int l = i ^ jj;
          if (l > i) {
            const int32_t a = S.key[i], c = S.key[l];
            bool gt;
            if (a < 0 || c < 0) gt = a < 0 && c >= 0;
            else gt = S.ou[a] > S.ou[c] || (S.ou[a] == S.ou[c] && a > c);
            if (gt == ((i & kk) == 0)) {
              S.key[i] = c;
              S.key[l] = a;
            }
          }
        }
        __syncthreads();
      }
    // shared nodes: runs of equal pairs (run index by a CTA scan of run starts)
    cta_exscan(m, [&](int i) { return (i == 0 || S.ou[S.key[i]] != S.ou[S.key[i - 1]]) ? 1 : 0; },
               reinterpret_cast<int*>(S.w), S.scan, &S.tot);
    const int ng = S.tot;
    if (ng > GAM) {
      if (tid == 0) defer(u);
      continue;
    }
    for (int i = tid; i < m; i += nt) {
      const int pre = reinterpret_cast<int*>(S.w)[i];
      const bool start = i == 0 || S.ou[S.key[i]] != S.ou[S.key[i - 1]];
      const int x = start ? pre : pre - 1;
      S.og[S.key[i]] = (int16_t)x;
      if (start) {
        S.gu[x] = S.ou[S.key[i]];
        S.gbeg[x] = i;
      }
    }
    if (tid == 0) S.gbeg[ng] = m;
    // offsets of the small inverses (one warp: k <= 32)
    if (wid == 0) {
      const int gp = lane < k ? S.pgb[lane + 1] - S.pgb[lane] : 0;
      int x = gp * gp;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane < k) S.pginv[lane + 1] = x;
      if (lane == 0) S.pginv[0] = 0;
      const int tot = __shfl_sync(0xffffffffu, x, 31);
      if (lane == 0) S.flag = tot > kUGinv ? 1 : 0;
    }
    __syncthreads();
    if (S.flag) {
      if (tid == 0) atomicExch(&v.wfast[kWGeneral], 1);
      continue;
    }
    if (MODE < 2 && (ng > SMG || S.pginv[k] > SMGINV)) {
      // too large for this pass's shared memory: the next pass takes it
      if (tid == 0) defer(u);
      continue;
    }
    float* const ginv = S.pginv[k] <= SMGINV ? S.ginv_sm : ginv_glob;
    float* const Sinv = ng <= SMG ? S.s_sm : s_glob;
    phase(0);
    // (A_p[G,G])^-1 per piece (one warp per piece)
    for (int p = wid; p < k; p += nw) {
      const int gp = S.pgb[p + 1] - S.pgb[p];
      if (gp == 0) continue;
      const int32_t g = S.pg[p];
      const int n = S.pbase[p + 1] - S.pbase[p];
      const float* A = v.piece_inv + v.piece_inv_off[g];
      float* Gm = ginv + S.pginv[p];
      const int gb0 = S.pgb[p], bs = S.pbase[p];
      for (int c = lane; c < gp; c += 32) {
        const int ic = S.gl[gb0 + c] - bs;
        int a = 0;
        for (; a + 3 < gp; a += 4) {
          float x[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) x[q] = __ldg(A + (size_t)(S.gl[gb0 + a + q] - bs) * n + ic);
#pragma unroll
          for (int q = 0; q < 4; ++q) Gm[(a + q) * gp + c] = x[q];
        }
        for (; a < gp; ++a) Gm[a * gp + c] = __ldg(A + (size_t)(S.gl[gb0 + a] - bs) * n + ic);
      }
      __syncwarp();
      if (!warp_spd_inverse(Gm, gp, lane) && lane == 0) S.flag = 1;
    }
    // S = sum_p R_p^T (A_p[G,G])^-1 R_p - lambda diag(c - 1), pieces in order
    for (int t = tid; t < ng * ng; t += nt) Sinv[t] = 0.f;
    __syncthreads();
    phase(1);
    if (S.flag) {
      if (tid == 0) atomicExch(&v.wfast[kWGeneral], 1);
      continue;
    }
    for (int p = 0; p < k; ++p) {
      const int gp = S.pgb[p + 1] - S.pgb[p];
      const float* Gm = ginv + S.pginv[p];
      for (int a = wid; a < gp; a += nw) {
        const int xa = S.og[S.gl[S.pgb[p] + a]];
        for (int c = lane; c < gp; c += 32) Sinv[xa * ng + S.og[S.gl[S.pgb[p] + c]]] += Gm[a * gp + c];
      }
      __syncthreads();
    }
    for (int x = tid; x < ng; x += nt) Sinv[x * ng + x] -= lam * (float)(S.gbeg[x + 1] - S.gbeg[x] - 1);
    if (!cta_spd_inverse(Sinv, ng)) {
      if (tid == 0) atomicExch(&v.wfast[kWGeneral], 1);
      continue;
    }
    phase(2);
    // u and the starting state
    float uu = 0.f;
    for (int o = tid; o < nocc; o += nt)
      if (S.og[o] < 0) {
        S.uh[o] = v.rhs[S.ou[o]];
        S.ul[o] = v.rhs_lo[S.ou[o]];
        S.zh[o] = 0.f;
        S.zl[o] = 0.f;
        uu = fmaf(S.uh[o], S.uh[o], uu);
      }
    for (int x = tid; x < ng; x += nt) {
      S.guh[x] = v.rhs[S.gu[x]];
      S.gul[x] = v.rhs_lo[S.gu[x]];
      S.gzh[x] = 0.f;
      S.gzl[x] = 0.f;
      uu = fmaf(S.guh[x], S.guh[x], uu);
    }
    uu = cta_sum(uu, S.red);
    auto zval = [&](int o) -> df32 {
      const int x = S.og[o];
      return x < 0 ? df32{S.zh[o], S.zl[o]} : df32{S.gzh[x], S.gzl[x]};
    };
    int round = 0;
    bool done = false;
    for (; round < kRounds; ++round) {
      // right-hand side: u, then the residual u - K z (double-float)
      float rr = 0.f;
      for (int o = tid; o < nocc; o += nt) {
        const int x = S.og[o];
        if (round == 0) {
          if (x < 0) {
            const float r = S.uh[o] + S.ul[o];
            S.f[o] = r;
            rr = fmaf(r, r, rr);
          }
          continue;
        }
        const int p = S.opc[o];
        const int base = S.pbase[p];
        const df32 zi = zval(o);
        const df32 bz = member_bz(v, S.pm0[p] + (o - base), zi, [&](int j) { return zval(base + j); });
        if (x < 0) {
          df32 rd = df_add(df32{S.uh[o], S.ul[o]}, df_mul_f(zi, -lam));
          rd = df_add(rd, df32{-bz.hi, -bz.lo});
          S.f[o] = rd.hi;
          rr = fmaf(rd.hi, rd.hi, rr);
        } else {
          S.ph[o] = bz.hi;
          S.pl[o] = bz.lo;
        }
      }
      __syncthreads();
      for (int x = tid; x < ng; x += nt) {
        float r;
        if (round == 0) {
          r = S.guh[x] + S.gul[x];
        } else {
          df32 acc = {0.f, 0.f};
          for (int i = S.gbeg[x]; i < S.gbeg[x + 1]; ++i) {      // occurrences in piece order
            const int o = S.key[i];
            acc = df_add(acc, df32{S.ph[o], S.pl[o]});
          }
          df32 rd = df_add(df32{S.guh[x], S.gul[x]}, df_mul_f(df32{S.gzh[x], S.gzl[x]}, -lam));
          rd = df_add(rd, df32{-acc.hi, -acc.lo});
          r = rd.hi;
        }
        S.gf[x] = r;
        rr = fmaf(r, r, rr);
      }
      rr = cta_sum(rr, S.red);
      if (rr <= tol * tol * uu) {
        done = true;
        break;
      }
      // w_p = A_p[:, I_p] f_I  (shared entries of f count as zero); two rows per
      // thread, eight columns per load batch
      for (int o0 = tid; o0 < nocc; o0 += 2 * nt) {
        const int o1 = o0 + nt < nocc ? o0 + nt : o0;
        const int b0 = S.pbase[S.opc[o0]], b1 = S.pbase[S.opc[o1]];
        const int n0 = S.pbase[S.opc[o0] + 1] - b0, n1 = o1 != o0 ? S.pbase[S.opc[o1] + 1] - b1 : 0;
        const float* A0 = v.piece_inv + v.piece_inv_off[S.pg[S.opc[o0]]] + (o0 - b0);
        const float* A1 = v.piece_inv + v.piece_inv_off[S.pg[S.opc[o1]]] + (o1 - b1);
        float c0[2] = {0.f, 0.f}, c1[2] = {0.f, 0.f};
        const int nmax = n0 > n1 ? n0 : n1;
        for (int j = 0; j < nmax; j += 8) {
          float a0[8], a1[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            a0[t] = j + t < n0 ? __ldg(A0 + (size_t)(j + t) * n0) : 0.f;
            a1[t] = j + t < n1 ? __ldg(A1 + (size_t)(j + t) * n1) : 0.f;
          }
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            if (j + t < n0 && S.og[b0 + j + t] < 0) c0[t & 1] = fmaf(a0[t], S.f[b0 + j + t], c0[t & 1]);
            if (j + t < n1 && S.og[b1 + j + t] < 0) c1[t & 1] = fmaf(a1[t], S.f[b1 + j + t], c1[t & 1]);
          }
        }
        S.w[o0] = c0[0] + c0[1];
        if (o1 != o0) S.w[o1] = c1[0] + c1[1];
      }
      __syncthreads();
      // h_p = w_p[G_p]; tt = (A_p[G,G])^-1 h_p per shared occurrence
      for (int t = tid; t < m; t += nt) S.th[t] = S.w[S.gl[t]];
      __syncthreads();
      for (int t = tid; t < m; t += nt) {
        const int p = S.opc[S.gl[t]];
        const int gp = S.pgb[p + 1] - S.pgb[p], a = t - S.pgb[p];
        const float* Gm = ginv + S.pginv[p];
        float acc = 0.f;
        for (int c = 0; c < gp; ++c) acc = fmaf(Gm[a * gp + c], S.th[S.pgb[p] + c], acc);
        S.tt[t] = acc;
      }
      __syncthreads();
      // b = f_G + the pieces' terms, over each shared node's occurrences in piece order
      for (int x = tid; x < ng; x += nt) {
        float acc = S.gf[x];
        for (int i = S.gbeg[x]; i < S.gbeg[x + 1]; ++i) {
          const int o = S.key[i];
          int t = S.pgb[S.opc[o]];
          while (S.gl[t] != o) ++t;
          acc += S.tt[t];
        }
        S.gb[x] = acc;
      }
      __syncthreads();
      // z_G correction = S^-1 b
      for (int x = tid; x < ng; x += nt) {
        float acc = 0.f;
        for (int c = 0; c < ng; ++c) acc = fmaf(Sinv[c * ng + x], S.gb[c], acc);
        S.gx[x] = acc;
      }
      __syncthreads();
      // t_p = (A_p[G,G])^-1 (z_G - h_p), per shared occurrence
      for (int t = tid; t < m; t += nt) S.th[t] = S.gx[S.og[S.gl[t]]] - S.th[t];
      __syncthreads();
      for (int t = tid; t < m; t += nt) {
        const int p = S.opc[S.gl[t]];
        const int gp = S.pgb[p + 1] - S.pgb[p], a = t - S.pgb[p];
        const float* Gm = ginv + S.pginv[p];
        float acc = 0.f;
        for (int c = 0; c < gp; ++c) acc = fmaf(Gm[a * gp + c], S.th[S.pgb[p] + c], acc);
        S.tt[t] = acc;
      }
      __syncthreads();
      // z_I += w_p[I] + A_p[I, G] t_p;  z_G += S^-1 b
      for (int o = tid; o < nocc; o += nt) {
        if (S.og[o] >= 0) continue;
        const int p = S.opc[o];
        const int base = S.pbase[p];
        const int n = S.pbase[p + 1] - base;
        const float* A = v.piece_inv + v.piece_inv_off[S.pg[p]] + (o - base);
        float acc = S.w[o], acc2 = 0.f;
        int t = S.pgb[p];
        const int t1 = S.pgb[p + 1];
        for (; t + 3 < t1; t += 4) {
          float x[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) x[q] = __ldg(A + (size_t)(S.gl[t + q] - base) * n);
          acc = fmaf(x[0], S.tt[t], acc);
          acc2 = fmaf(x[1], S.tt[t + 1], acc2);
          acc = fmaf(x[2], S.tt[t + 2], acc);
          acc2 = fmaf(x[3], S.tt[t + 3], acc2);
        }
        for (; t < t1; ++t) acc = fmaf(__ldg(A + (size_t)(S.gl[t] - base) * n), S.tt[t], acc);
        acc += acc2;
        const df32 z = df_add_f(df32{S.zh[o], S.zl[o]}, acc);
        S.zh[o] = z.hi;
        S.zl[o] = z.lo;
      }
      for (int x = tid; x < ng; x += nt) {
        const df32 z = df_add_f(df32{S.gzh[x], S.gzl[x]}, S.gx[x]);
        S.gzh[x] = z.hi;
        S.gzl[x] = z.lo;
      }
      __syncthreads();
    }
    if (!done && tid == 0) atomicExch(&v.wfast[kWGeneral], 1);
    if (round > max_rounds) max_rounds = round;
    phase(3);
    if (tid == 0) atomicAdd(&dbg[4], 1);
    if (tid == 0) {
      if (MODE == 2) atomicAdd(&v.wfast[kWBigS], 1);
      atomicAdd(&v.wfast[MODE == 1 ? kWCycSm : kWCycBig],
                (int)((clock64() - t_unit) >> 10));
    }
    for (int o = tid; o < nocc; o += nt)
      if (S.og[o] < 0) {
        v.z[S.ou[o]] = S.zh[o];
        v.z_lo[S.ou[o]] = S.zl[o];
      }
    for (int x = tid; x < ng; x += nt) {
      v.z[S.gu[x]] = S.gzh[x];
      v.z_lo[S.gu[x]] = S.gzl[x];
    }
  }
  if (tid == 0 && max_rounds > 0) atomicMax(&v.wfast[kWRounds], max_rounds);
}

// the rounds used, into the step's iteration counter
__global__ void k_whiten_stats(StepView v) {
  if (threadIdx.x == 0) atomicMax(&v.counters[kCntCompIters], v.wfast[kWRounds]);
}

}  // namespace

// the two CTA passes for the units the data-parallel solver hands over:
// <pieces, members, shared nodes, S^-1 and small inverses in shared memory, threads>
#define KW1 32, 1024, 256, 64, 4096, 256, 1
#define KW2 32, 1024, 256, 160, 8192, 256, 2
using Smem1 = UnitSmem<32, 1024, 256, 64, 4096>;
using Smem2 = UnitSmem<32, 1024, 256, 160, 8192>;

cudaError_t configure_whiten_kernels() {
  cudaError_t e = configure_units_kernels();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_whiten_units<KW1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem1));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_whiten_units<KW2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(Smem2));
}

int piece_max_nodes() { return kPieceMaxDev; }

int64_t whiten_unit_scratch_floats() { return kUScratch; }

// CTAs of the two CTA unit passes in grids[1], grids[2] (returns 0 when one of
// them cannot run on this device)
int whiten_units_grids(int num_sms, int grids[3]) {
  int b = 0, c = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_whiten_units<KW1>, 256, sizeof(Smem1)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_whiten_units<KW2>, 256, sizeof(Smem2)) != cudaSuccess ||
      b < 1 || c < 1)
    return 0;
  grids[0] = 0;
  grids[1] = num_sms * b;
  grids[2] = num_sms * c;
  return grids[1];
}

int whiten_clean_grid(int num_sms) {
  int a = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_whiten_clean, kCleanWarps * 32, 0) != cudaSuccess ||
      a < 1)
    return 0;
  return num_sms * a;
}

int piece_cc_grid(int num_sms) {
  int a = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_piece_cc, 512, 0) != cudaSuccess || a < 1) return 0;
  return num_sms * (a < 2 ? a : 2);
}

// side, fork, join: a second stream and two events; the single pieces are
// solved on the side stream while the units are solved on st
cudaError_t launch_whiten_fast(const StepView& v, int64_t n_b, float tol, int cc_grid, const int grids[4],
                               int clean_grid, cudaStream_t st, cudaStream_t side, cudaEvent_t fork,
                               cudaEvent_t join, const cudaEvent_t* ev, int clean_share, const Branches* br) {
  if (!v.whiten) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(v.wfast, 0, kWSlots * sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  k_piece_init<<<(unsigned)n_b, 256, 0, st>>>(v);
  {
    StepView vv = v;
    int64_t nb = n_b;
    void* args[] = {&vv, &nb};
    e = cudaLaunchCooperativeKernel((const void*)k_piece_cc, dim3(cc_grid), dim3(512), args, 0, st);
    if (e != cudaSuccess) return e;
  }
  e = cudaMemsetAsync(v.counters + kCntBarArrive, 0, 2 * sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  k_unit_ids<<<(unsigned)n_b, 256, 0, st>>>(v);
  k_unit_scan<<<1, 1024, 0, st>>>(v);
  k_unit_fill<<<(unsigned)n_b, 256, 0, st>>>(v);
  if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
  // the clean pieces: on the side stream with clean_share / 4 of the
  // persistent grid, concurrently with the units; clean_share 0: on st after them
  if (clean_share > 0) {
    if ((e = cudaEventRecord(fork, st)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(side, fork, 0)) != cudaSuccess) return e;
    const int g = clean_grid * clean_share / 4;
    k_whiten_clean<<<g > 0 ? g : 1, kCleanWarps * 32, 0, side>>>(v, tol);
    if ((e = cudaEventRecord(join, side)) != cudaSuccess) return e;
  }
  // units: data-parallel, then the CTA passes for the units it handed over
  e = launch_units(v, tol, grids[3], st, ev ? ev[1] : nullptr, br);
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[2], st)) != cudaSuccess) return e;
  k_whiten_units<KW1><<<grids[1], 256, sizeof(Smem1), st>>>(v, tol);
  k_whiten_units<KW2><<<grids[2], 256, sizeof(Smem2), st>>>(v, tol);
  if (ev && (e = cudaEventRecord(ev[3], st)) != cudaSuccess) return e;
  if (clean_share == 0)
    k_whiten_clean<<<clean_grid, kCleanWarps * 32, 0, st>>>(v, tol);
  else if ((e = cudaStreamWaitEvent(st, join, 0)) != cudaSuccess)
    return e;
  k_whiten_stats<<<1, 32, 0, st>>>(v);
  if (ev && (e = cudaEventRecord(ev[4], st)) != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace spider
