// Device-side views shared by the step kernels (plain pointers, passed by value).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace spider {

// counters[] slots (int32, device)
enum : int {
  kCntPairs = 0,     // P_u: unique pairs of the current minibatch
  kCntObs = 1,       // n: observations of the current minibatch
  kCntIters = 2,     // whitening iterations used
  kCntError = 3,     // first device-side error (SPIDER_E_*), sticky until read
  kCntBarArrive = 4, // grid barrier arrivals
  kCntBarGen = 5,    // grid barrier generation
  kCntComps = 6,     // connected components of the minibatch graph
  kCntCompIters = 7, // largest CG iteration count of a component solved by one warp
  kCntEvents = 8,    // events touched by the minibatch (with at least one pair)
  kCntSlots = 9
};

// Travel-time network on the device.
struct NetView {
  int kind;          // SPIDER_TT_*
  int H;
  int precision;     // SPIDER_FP32 / BF16 / FP8
  float v0, g;
  float inv_v_hi, inv_v_lo;   // 1/v0 as a double-float
  const float* W1;   // H x 6 (out, in)
  const float* b1;   // H
  const float* Wt[3];  // W2..W4 transposed: [in][out] (forward operand)
  const float* Wn[3];  // W2..W4 as given: [out][in] (backward operand)
  const float* bh[3];  // b2..b4
  const float* W5;     // H
  float b5;
  const void* tc;      // tensor-core operand images (BF16 / FP8), null in FP32
  const float* tc_scale;  // per-layer FP8 dequantisation scales (6), null otherwise
  int32_t* err;           // device error flag the tensor-core kernel reports bounded-wait timeouts to
};

// Where the pairs of a travel-time launch come from.
struct PairSource {
  // problem mode: pair u -> uniq_pair[u] -> (event, station)
  const int32_t* uniq_pair;
  const int32_t* pair_ev;
  const int32_t* pair_st;
  const float4* th0_hi;   // event theta_0 (hi)
  const float4* th0_lo;   // event theta_0 (lo)
  const float4* dth;      // event state offset theta - theta_0
  const float4* sta_hi;
  const float4* sta_lo;
  // raw mode (uniq_pair == nullptr): absolute FP32 positions per pair
  const float4* src;
  const float4* rcv;
  const int32_t* n_dev;   // device count (problem mode) or nullptr
  int64_t n_host;         // host count (raw mode) / upper bound
};

struct TTOut {
  float2* T2;   // (T_hi, T_lo)
  float4* J;    // (dT/dx, dT/dy, dT/dz, 0), may be null
};

// Per-step parameters, read by the kernels from device memory (the host
// writes them before each step, so a captured step graph can be relaunched).
struct StepParams {
  uint64_t seed;
  float eps;
  float noise_scale;
  int32_t tag;
  int32_t mode;          // 0: gradient only, 1: SGLD update
  int32_t full;          // 1: every block of every sub-problem
  int32_t pad;
  int64_t sample_slot;   // -1: no sample this step
  float bc1, bc2;        // Adam bias corrections 1 / (1 - beta^t)
  uint64_t wait_ns;      // limit of every bounded device-side wait (grid barriers)
};

// Step state and tables.
struct StepView {
  int64_t M, N, S, NB, B, P, Q;
  int L_max;
  const StepParams* prm;
  // sub-problems (catalog x chain); a single catalog is one sub-problem
  int n_sub;
  const int32_t* blk_e0;          // NB + 1 first observation of each block
  const int32_t* blk_sub;         // NB
  const int32_t* ev_sub;          // M
  const int32_t* sub_blk_off;     // n_sub + 1
  const int32_t* sub_sel_full;    // n_sub + 1 prefix of blocks selected per step, full batch
  const int32_t* sub_sel_mb;      // n_sub + 1 prefix of blocks selected per step, minibatch
  const int32_t* sub_nobs;        // n_sub observations
  const int32_t* sub_nev;         // n_sub events
  const int32_t* sub_chain;       // n_sub Philox counter word 1
  const int32_t* sub_catalog;     // n_sub Philox counter word 2
  int32_t* sub_nsel;              // n_sub observations in this step's minibatch
  float4* sub_cen;                // n_sub centroid of the current state offset
  int n_chunks;
  const int32_t* chunk_ev0;       // n_chunks + 1 event chunks for the centroid sums
  const int32_t* sub_chunk_off;   // n_sub + 1
  float4* cen_chunk;              // n_chunks
  const float4* th0_hi;
  const float4* th0_lo;
  const double* th0_d;        // M x 4 theta_0 in FP64 (read-back only)
  const int32_t* ev_out;      // M: caller's event index (global) of each internal event
  float4* dth;
  const int32_t* ev_caller;   // caller's index of each (internal) event: the noise counter
  const float4* sta_hi;
  const float4* sta_lo;
  const int32_t* pair_ev;
  const int32_t* pair_st;
  const int32_t* pair_off;
  const uint32_t* obs_l;
  const float* obs_dt;
  const float* obs_sw;
  const int32_t* blk_node_off;
  const int32_t* node_pair;
  const uint16_t* node_he;
  const uint16_t* blk_he;
  const int32_t* inc_off;
  const int32_t* inc_q;
  const int32_t* inc_b;
  // per-step scratch
  int32_t* sel;
  int32_t* blk_stamp;
  int32_t* owner_q;
  uint8_t* multi;
  int32_t* loc2u;
  int32_t* blk_owner_cnt;
  int32_t* blk_owner_off;
  int32_t* uniq_pair;
  int32_t* uniq_q;
  float2* T2;
  float4* J;
  float* r_obs;
  float* q_obs;
  float* part_a;     // per-occurrence partials (multi nodes): hi part
  float* part_b;     //   degree partials
  float* part_c;     //   lo part
  float* rhs;        // u = B^T r (hi)
  float* rhs_lo;     //           (lo)
  float* diag;       // lambda + diag(B^T B)
  float* z;          // solution (hi)
  float* z_lo;       //          (lo)
  float* rres;       // outer (double-float) residual rounded to FP32: inner right-hand side
  float* dz;         // inner correction
  float* res;
  float* pv;        // search direction (two buffers, alternating per iteration)
  float* pv2;
  float* Ap;
  float* yv;
  uint8_t* umulti;  // per unique pair: 1 if it has occurrences in several selected blocks
  // merged minibatch matrix lambda I + B^T B as CSR over unique pairs (per solve)
  int32_t* rowlen;   // [P] half-edges of the pair over all selected occurrences
  int32_t* rowptr;   // [P + 1]
  int32_t* occ_off;  // [Q] offset of an occurrence's entries inside its pair's row
  int32_t* csr_col;  // [2N] neighbour pair (unique index)
  float* csr_sw;     // [2N] sqrt(w_e) of the edge
  int32_t* scan_part;  // [kMaxGrid + 1] scan partials
  // connected components of the minibatch graph (per solve)
  int32_t* lab;      // [P] component label = smallest unique index in the component
  int32_t* cslot;    // [P] per root: component index; per member: position (scratch)
  int32_t* ccount;   // [P] member count per root
  int32_t* comp_root;  // [P] roots in ascending order
  int32_t* comp_off;   // [P + 1] member list offsets
  int32_t* members;    // [P] member lists (sorted within each component by the solver)
  int32_t* lidx;       // [P] local index of a member inside its component
  uint8_t* big;        // [P] 1: the row belongs to a component solved by the grid-wide CG
  int32_t* chist;      // [kCqBins + 4] solver work-list bins and cursors
  int32_t* bigpos;     // [P + 1] exclusive prefix of the grid-tier flags (then the count)
  int32_t* biglist;    // [P] grid-tier nodes in pair order
  int32_t* cc_lroot;   // [Q] per local node of a selected block: its block-local component root (local node id)
  int32_t* corder;     // [P] solver work list (component ids)
  int32_t* centries;   // [P] CSR entries per component
  uint8_t* ctier;      // [P] per component: 0 one warp, 1 one CTA, 2 grid-wide
  float* s_u;
  float4* gp;
  int32_t* pstamp;
  int32_t* estamp;
  float4* grad;
  int32_t* counters;
  float* red;        // float reduction partials (whitening), 8 x kMaxGrid
  double* dblk;      // FP64 sum r^2 per selected block (NB)
  double* dred;      // FP64 diagnostics partials, 4 x kMaxGrid
  double* dout;      // FP64 results: [0] loglik (scaled), [1] logprior, [2] logcen, [3] logpost
  // whitening through the precomputed piece inverses (null when not built)
  const int32_t* blk_piece_off;   // NB + 1
  const uint16_t* node_piece;     // Q: piece of a local node, numbered within its block
  const uint16_t* node_ppos;      // Q: position of a local node inside its piece
  const int32_t* piece_node_off;  // G + 1
  const uint16_t* piece_nodes;    // Q: block-local index of each piece member
  const int64_t* piece_inv_off;   // G + 1
  const float* piece_inv;         // (lambda I + B^T B)^-1 of every piece, n x n each
  const int32_t* mem_rp;          // Q + 1: edges of each member (piece_nodes order)
  const uint16_t* edge_pos;       // 2N: position of the other end inside the piece
  const float* edge_sw;           // 2N: sqrt w of the edge
  int32_t* owner_b;               // Q: block of the owner occurrence (per step)
  int32_t* plab;                  // G: piece labels of the selected pieces (per step)
  uint8_t* pmulti;                // G: the piece has a node shared with another selected block
  int32_t* pcount;                // G: pieces per unit, at the unit's root piece
  int32_t* unit_of;               // G: unit of a root piece
  int32_t* unit_cnt;              // [G]: pieces per unit (fill cursor afterwards)
  int32_t* unit_off;              // [G + 1]
  int32_t* unit_pieces;           // [G]
  int32_t* unit_pblk;             // [G]: block of each entry of unit_pieces
  int32_t* unit_defer;            // [G]: units the data-parallel solver handed to the CTA pass
  int32_t* unit_defer2;           // [G]: units deferred from the CTA pass to the last pass
  int32_t* clean_list;            // [G]: pieces of the step with no shared node
  int32_t* clean_blk;             // [G]: their blocks
  int32_t* wfast;                 // [kWSlots] unit count, unit cursor, fallback flag, rounds
  float* wscratch;                // per CTA of the unit solver: S^-1 and the pieces' small inverses
  // units solved data-parallel (k_units.cu): per unit [G (+1)], per unit piece
  // entry [G], per occurrence slot [u_cap], pools of the small inverses
  int32_t *u_nocc, *uocc_off, *u_ng, *u_m, *u_gsz, *u_goff, *u_ssz, *u_soff;
  int32_t *pu_base, *pu_unit, *pu_gb, *pu_gn, *pu_ginv;
  int32_t *o_g, *o_pe, *o_base, *o_u, *o_x, *o_unit, *o_t;
  uint16_t* o_i;
  float *o_uh, *o_ul, *o_zh, *o_zl, *o_f, *o_w, *o_ph, *o_pl;
  int32_t *sh_slot, *sh_sorted;
  float* sh_tt;
  int32_t *g_u, *g_beg, *g_cnt;
  float *g_uh, *g_ul, *g_zh, *g_zl, *g_f, *g_x;
  float *ginv_pool, *sinv_pool;
  int64_t u_cap, ginv_cap, sinv_cap;
  const int32_t* gate;            // non-null: the general solver runs only while *gate != 0
  float4* samples;
  float4* mom1;      // Adam first moment (M), null otherwise
  float4* mom2;      // pSGLD / Adam second moment (M), null for SGLD
  int64_t sample_cap;
  // constants
  float lam;        // sigma^2 / kappa^2
  float inv_s2;     // 1 / sigma^2
  int whiten;       // kappa > 0 and the whitened loss
  int loss;         // SPIDER_LOSS_*
  int update;       // SPIDER_UPDATE_*
  float beta1, beta2, upd_eps;
  float4 inv_sig_e2;   // 1 / sigma_e^2
  float4 inv_sig_c2;   // 1 / sigma_c^2
  int cen_grid;     // CTAs of the event kernel
};

constexpr int kMaxGrid = 4096;
// wfast[] slots of the piece-inverse whitening
enum : int {
  kWUnits = 0, kWCursor = 1, kWGeneral = 2, kWRounds = 3,
  kWBigS = 4,      // units solved by the second pass (large shared-node sets)
  kWCycSm = 5,     // SM cycles / 1024 spent on units of the first pass
  kWCycBig = 6,    // the same for the second pass
  kWDefer = 7,     // units deferred to the second pass
  kWCursor2 = 8,   // work cursor of the second pass
  kWClean = 9,     // single pieces of the step (no shared node)
  kWCursorC = 10,  // work cursor of the single-piece solver
  // slots 11 and 13: unused
  kWDefer2 = 12,   // units deferred from the CTA pass to the last pass
  kWCursorS = 14,  // work cursor of the CTA inverse of the largest S
  kWCursorS2 = 15, // work cursor of the register inverse of S at 97..128 shared nodes
  kWSlots = 16
};
constexpr int kCenChunk = 4096;   // events per centroid partial sum

}  // namespace spider
