// C ABI of the library: context lifetime, uploads, step orchestration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.h"
#include "pieces.h"
#include "prep.h"
#include "spider.h"

using namespace spider;

struct spider_ctx {
  std::string err;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0, num_sms = 0;
  spider_config cfg{};
  std::vector<int32_t> ev_old;     // internal event -> caller event
  std::vector<int32_t> ord;        // canonical obs -> caller obs
  std::vector<double> th0;         // M x 4 internal order
  NetView net{};
  StepView v{};
  std::vector<void*> allocs;
  float* tt_scratch = nullptr;
  int gu = 0, pgrid = 0;
  int tag = 0;
  int64_t step = 0;
  int n_sub = 1;
  int64_t nb_full = 0, nb_mb = 0;  // blocks per step: full batch / minibatch
  StepParams* prm = nullptr;       // device copy of the per-step parameters
  cudaGraph_t graph = nullptr;     // the captured SGLD step (timing off)
  cudaGraphExec_t graph_exec = nullptr;
  bool graph_ok = true;
  bool use_graph = true;
  int32_t knobs[7] = {2, 1, 2, 1, 2, 2, 1};   // see spider_set_tuning
  // whitening through precomputed piece inverses (minibatch steps)
  bool fast = false;               // tables built
  bool mb_full_sub = false;        // a sub-problem selects all its blocks in a minibatch
  int cc_grid = 0, clean_grid = 0;
  int unit_grids[4] = {0, 0, 0, 0};   // [3]: SMs (the data-parallel unit solver)
  int64_t piece_bytes = 0;
  cudaStream_t side = nullptr;     // second stream of the piece-inverse whitening
  cudaEvent_t fork = nullptr, join = nullptr;
  Branches ubr{};                  // branch streams of the units' set-up
  int64_t n_samples = 0;           // samples written so far (ring of sample_cap)
  int64_t last_nb = 0;
  bool timing = false;
  uint64_t wait_ns = 2000000000ull; // limit of the bounded device-side waits
  double* state_dev = nullptr;     // M x 4 FP64 read-back buffer (caller order)
  float4* grad_dev = nullptr;      // M gradient read-back buffer (caller order)
  int grid_ev = 1;                 // CTAs of the read-back kernels
  // stage events of a timed evaluation: start, after selection + pair table,
  // travel times, k_resid, k_merge_rhs, whitening, k_final, k_merge_s,
  // centroid, k_event, end
  static constexpr int kEv = 11;
  cudaEvent_t ev[kEv] = {};
  cudaEvent_t wev[5] = {};          // whitening phases (timed evaluations of the piece path)
  bool have_wtiming = false;
  int64_t graph_kernels = 0;        // kernel nodes of the captured step graph
  float last_ms[5] = {0, 0, 0, 0, 0};
  bool have_timing = false;
};

struct spider_netdev {
  NetView net{};
  std::vector<void*> allocs;
  float* scratch = nullptr;
  int num_sms = 0;
};

namespace {

const char* g_static_err = "";

int cuda_fail(spider_ctx* c, cudaError_t e, const char* what) {
  if (c) c->err = std::string(what) + ": " + cudaGetErrorString(e);
  g_static_err = cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? SPIDER_E_OOM : SPIDER_E_CUDA;
}

void destroy_branches(Branches& b) {
  for (int i = 0; i < 4; ++i) {
    if (b.s[i]) {
      cudaStreamSynchronize(b.s[i]);
      cudaStreamDestroy(b.s[i]);
    }
    if (b.join[i]) cudaEventDestroy(b.join[i]);
    b.s[i] = nullptr;
    b.join[i] = nullptr;
  }
  if (b.fork) cudaEventDestroy(b.fork);
  b.fork = nullptr;
}

#define CK(ctx, call)                                   \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, #call); \
  } while (0)

template <typename T>
cudaError_t dalloc(std::vector<void*>& list, T** p, size_t n) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  list.push_back(q);
  *p = reinterpret_cast<T*>(q);
  return cudaSuccess;
}

template <typename T>
cudaError_t dupload(std::vector<void*>& list, T** p, const T* src, size_t n, cudaStream_t st) {
  cudaError_t e = dalloc(list, p, n);
  if (e != cudaSuccess || n == 0) return e;
  return cudaMemcpyAsync(*p, src, n * sizeof(T), cudaMemcpyHostToDevice, st);
}

void split_df(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

bool finite_arr(const float* a, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

// Validates a network description; returns 0 or an error code with msg.
int check_net(const spider_net* net, int precision, std::string* msg) {
  if (!net) { *msg = "null network"; return SPIDER_E_INVAL; }
  if (net->kind == SPIDER_TT_HOMOGENEOUS) {
    if (!(net->v0 > 0.0)) { *msg = "homogeneous medium needs v0 > 0"; return SPIDER_E_INVAL; }
    return SPIDER_OK;
  }
  if (net->kind == SPIDER_TT_LINEAR_GRADIENT) {
    if (!(net->v0 > 0.0) || !(net->g > 0.0)) { *msg = "gradient medium needs v0 > 0, g > 0"; return SPIDER_E_INVAL; }
    return SPIDER_OK;
  }
  if (net->kind != SPIDER_TT_MLP) { *msg = "unknown travel-time kind"; return SPIDER_E_INVAL; }
  const int H = net->H;
  if (!tt_supported_width(H)) { *msg = "MLP width H must be 32, 64, 128 or 256"; return SPIDER_E_UNSUPPORTED; }
  if (precision < SPIDER_FP32 || precision > SPIDER_FP8) { *msg = "unknown precision"; return SPIDER_E_INVAL; }
  if (precision != SPIDER_FP32 && !mlp_tc_supported(H, precision)) {
    *msg = "this precision / width has no tensor-core kernel in this build";
    return SPIDER_E_UNSUPPORTED;
  }
  const size_t wn[5] = {(size_t)H * 6, (size_t)H * H, (size_t)H * H, (size_t)H * H, (size_t)H};
  const size_t bn[5] = {(size_t)H, (size_t)H, (size_t)H, (size_t)H, 1};
  for (int l = 0; l < 5; ++l) {
    if (!net->W[l] || !net->b[l]) { *msg = "null MLP weight or bias"; return SPIDER_E_INVAL; }
    if (!finite_arr(net->W[l], wn[l]) || !finite_arr(net->b[l], bn[l])) {
      *msg = "non-finite MLP weight or bias";
      return SPIDER_E_INVAL;
    }
  }
  return SPIDER_OK;
}

// Uploads weights into a NetView (allocations appended to `list`).
cudaError_t upload_net(const spider_net* in, int precision, NetView* nv, std::vector<void*>& list,
                       cudaStream_t st) {
  NetView n{};
  n.kind = in->kind;
  n.precision = precision;
  n.H = in->H;
  n.v0 = (float)in->v0;
  n.g = (float)in->g;
  if (in->v0 > 0.0) split_df(1.0 / in->v0, n.inv_v_hi, n.inv_v_lo);
  cudaError_t e = cudaSuccess;
  if (in->kind == SPIDER_TT_MLP) {
    const int H = in->H;
    float* p = nullptr;
    if ((e = dupload(list, &p, in->W[0], (size_t)H * 6, st))) return e;
    n.W1 = p;
    if ((e = dupload(list, &p, in->b[0], (size_t)H, st))) return e;
    n.b1 = p;
    std::vector<float> t((size_t)H * H);
    for (int l = 0; l < 3; ++l) {
      const float* W = in->W[l + 1];
      for (int o = 0; o < H; ++o)
        for (int i = 0; i < H; ++i) t[(size_t)i * H + o] = W[(size_t)o * H + i];
      if ((e = dupload(list, &p, t.data(), t.size(), st))) return e;
      n.Wt[l] = p;
      if ((e = dupload(list, &p, W, (size_t)H * H, st))) return e;
      n.Wn[l] = p;
      if ((e = dupload(list, &p, in->b[l + 1], (size_t)H, st))) return e;
      n.bh[l] = p;
    }
    if ((e = dupload(list, &p, in->W[4], (size_t)H, st))) return e;
    n.W5 = p;
    n.b5 = in->b[4][0];
    if (precision != SPIDER_FP32) {
      void* img = nullptr;
      float* sc = nullptr;
      const float* Wn_host[3] = {in->W[1], in->W[2], in->W[3]};
      if ((e = mlp_tc_prepare(in->W[0], Wn_host, in->W[4], H, precision, &img, &sc, st))) return e;
      if (img) list.push_back(img);
      if (sc) list.push_back(sc);
      n.tc = img;
      n.tc_scale = sc;
    }
    // the transposed copy above must outlive the async copy
    if ((e = cudaStreamSynchronize(st))) return e;
  }
  *nv = n;
  return cudaSuccess;
}

void free_all(std::vector<void*>& list) {
  for (void* p : list) cudaFree(p);
  list.clear();
}

int check_device_error(spider_ctx* c) {
  int32_t e = 0;
  cudaError_t ce = cudaMemcpyAsync(&e, c->v.counters + kCntError, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                   c->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
  if (ce != cudaSuccess) return cuda_fail(c, ce, "device error check");
  if (e != 0) {
    cudaMemsetAsync(c->v.counters + kCntError, 0, sizeof(int32_t), c->stream);
    cudaStreamSynchronize(c->stream);
    c->err = e == SPIDER_E_NONFINITE ? "non-finite value in the state or gradient"
             : e == SPIDER_E_TIMEOUT ? "a bounded device-side wait timed out"
                                     : "device-side error";
    return e;
  }
  return SPIDER_OK;
}

// The kernels of one evaluation, in stream order (everything a step does).
// fast: whiten through the piece inverses, with the general component solver
// gated on the flag that path raises for units beyond its limits.
cudaError_t step_sequence(spider_ctx* c, int64_t n_b, bool logpost, bool timed, bool fast) {
  StepView& v = c->v;
  cudaStream_t st = c->stream;
  cudaError_t e;
#define TRY(x)                       \
  do {                               \
    if ((e = (x)) != cudaSuccess) return e; \
  } while (0)
  TRY(cudaMemsetAsync(v.counters, 0, 3 * sizeof(int32_t), st));
  TRY(cudaMemsetAsync(v.counters + kCntBarArrive, 0, (kCntSlots - kCntBarArrive) * sizeof(int32_t), st));
  TRY(cudaMemsetAsync(v.sub_nsel, 0, c->n_sub * sizeof(int32_t), st));
  TRY(launch_select(v, n_b, st, 256 * c->knobs[5]));
  if (timed) TRY(cudaEventRecord(c->ev[1], st));
  PairSource src{};
  src.uniq_pair = v.uniq_pair;
  src.pair_ev = v.pair_ev;
  src.pair_st = v.pair_st;
  src.th0_hi = v.th0_hi;
  src.th0_lo = v.th0_lo;
  src.dth = v.dth;
  src.sta_hi = v.sta_hi;
  src.sta_lo = v.sta_lo;
  src.n_dev = v.counters + kCntPairs;
  src.n_host = v.P;
  TTOut out{v.T2, v.J};
  TRY(launch_tt(c->net, src, out, c->num_sms, c->tt_scratch, st, c->knobs[2]));
  if (timed) TRY(cudaEventRecord(c->ev[2], st));
  TRY(launch_resid(v, n_b, c->gu, st, timed ? &c->ev[3] : nullptr, 256 * c->knobs[5]));
  if (fast) {
    TRY(launch_whiten_fast(v, n_b, c->cfg.pcg_tol, c->cc_grid, c->unit_grids, c->clean_grid, st, c->side,
                           c->fork, c->join, timed ? c->wev : nullptr, c->knobs[4],
                           c->knobs[6] ? &c->ubr : nullptr));
    StepView vg = v;
    vg.gate = v.wfast + kWGeneral;
    TRY(launch_pcg(vg, n_b, c->cfg.pcg_max_it, c->cfg.pcg_tol, c->pgrid, c->knobs[0], c->knobs[1], st));
  } else {
    TRY(launch_pcg(v, n_b, c->cfg.pcg_max_it, c->cfg.pcg_tol, c->pgrid, c->knobs[0], c->knobs[1], st));
  }
  if (timed) TRY(cudaEventRecord(c->ev[5], st));
  TRY(launch_finish(v, n_b, c->gu, logpost, st, timed ? &c->ev[6] : nullptr, 256 * c->knobs[5]));
#undef TRY
  return cudaSuccess;
}

// One evaluation of the gradient (mode 0) or one SGLD step (mode 1).
int evaluate(spider_ctx* c, uint64_t seed, int mode, float eps) {
  const spider_config& cfg = c->cfg;
  StepView& v = c->v;
  const bool batch_full = cfg.batch_n <= 0 || cfg.batch_n >= v.N;
  const bool full = batch_full || (mode == 0 && seed == 0);
  const int64_t n_b = full ? c->nb_full : c->nb_mb;
  const bool fast = c->fast && c->knobs[3] && !full && !c->mb_full_sub && v.whiten;
  cudaStream_t st = c->stream;
  StepParams hp{};
  hp.seed = seed;
  hp.eps = eps;
  hp.noise_scale = cfg.noise_scale;
  hp.tag = ++c->tag;
  hp.mode = mode;
  hp.full = full ? 1 : 0;
  hp.sample_slot = -1;
  hp.wait_ns = c->wait_ns;
  if (mode == 1 && ((c->step + 1) % cfg.thin) == 0 && v.sample_cap > 0) hp.sample_slot = c->n_samples % v.sample_cap;
  {
    const double t = (double)(c->step + 1);
    hp.bc1 = (float)(1.0 / (1.0 - std::pow((double)cfg.beta1, t)));
    hp.bc2 = (float)(1.0 / (1.0 - std::pow((double)cfg.beta2, t)));
  }
  if (c->timing) CK(c, cudaEventRecord(c->ev[0], st));
  CK(c, cudaMemcpyAsync(c->prm, &hp, sizeof(hp), cudaMemcpyHostToDevice, st));
  const bool graphable = mode == 1 && !c->timing && c->use_graph && c->graph_ok;
  if (graphable && !c->graph_exec) {
    // capture the step once; relaunch it every step with fresh parameters
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t e1 = step_sequence(c, n_b, false, false, fast);
      cudaGraph_t g = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(st, &g);
      if (e1 == cudaSuccess && e2 == cudaSuccess && g &&
          cudaGraphInstantiate(&c->graph_exec, g, 0) == cudaSuccess) {
        c->graph = g;
        // kernel launches per graph step (what the step runs on the device)
        size_t nn = 0;
        c->graph_kernels = 0;
        if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
          std::vector<cudaGraphNode_t> nodes(nn);
          if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
            for (size_t i = 0; i < nn; ++i) {
              cudaGraphNodeType ty;
              if (cudaGraphNodeGetType(nodes[i], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel)
                ++c->graph_kernels;
            }
        }
      } else {
        if (g) cudaGraphDestroy(g);
        c->graph_exec = nullptr;
        c->graph_ok = false;
        cudaGetLastError();   // clear the capture failure; fall back to direct launches
      }
    } else {
      c->graph_ok = false;
      cudaGetLastError();
    }
  }
  if (graphable && c->graph_exec) {
    CK(c, cudaGraphLaunch(c->graph_exec, st));
  } else {
    const cudaError_t e = step_sequence(c, n_b, mode == 0, c->timing, fast);
    if (e != cudaSuccess) return cuda_fail(c, e, "step launch");
  }
  if (c->timing) CK(c, cudaEventRecord(c->ev[spider_ctx::kEv - 1], st));
  if (mode == 1) {
    c->step += 1;
    if (hp.sample_slot >= 0) c->n_samples += 1;
  }
  c->last_nb = n_b;
  c->have_timing = c->timing;
  c->have_wtiming = c->timing && fast;
  return SPIDER_OK;
}

}  // namespace

void spider::set_static_error(const char* msg) { g_static_err = msg; }

extern "C" {

void spider_config_default(spider_config* c) {
  std::memset(c, 0, sizeof(*c));
  c->sigma = 0.01;
  c->kappa = 0.03;
  c->p = 0.25;
  c->ell = 40.0;
  c->eps_w = 1e-5;
  c->sig_e[0] = c->sig_e[1] = c->sig_e[2] = 0.5;
  c->sig_e[3] = 0.1;
  for (int a = 0; a < 4; ++a) c->sig_c[a] = 0.01;
  c->batch_n = 0;
  c->block_obs = 4096;
  c->precision = SPIDER_FP32;
  c->thin = 1;
  c->reorder = 1;
  c->chain = 0;
  c->catalog = 0;
  c->noise_scale = 1.0f;
  c->pcg_max_it = 1000;
  c->pcg_tol = 1e-7f;
  c->sample_cap = 16;
  c->update = SPIDER_UPDATE_SGLD;
  c->beta1 = 0.9f;
  c->beta2 = 0.99f;
  c->upd_eps = 1e-5f;
  c->loss = SPIDER_LOSS_WHITENED;
}

}  // extern "C"

namespace {

// Pieces of every block and their inverses (pieces.h), for whitening the
// minibatch steps; skipped (the general component solver serves every step)
// when a piece is larger than the device path takes or the inverses would use
// more than half of the free device memory.  Returns an error code only for a
// failed CUDA call.
int build_fast_whitening(spider_ctx* c, const Prep& P) {
  Pieces T;
  if (!build_pieces(P, piece_max_nodes(), &T, 0)) return SPIDER_OK;
  const int64_t inv_floats = T.piece_inv_off[T.G];
  const int64_t bytes = inv_floats * 4 + P.Q * (2 + 2 + 2 + 4 + 4) + P.N * 2 * 6 + (T.G + 1) * (8 + 4 * 7) +
                        (P.NB + 1) * 4 +
                        (int64_t)c->num_sms * whiten_unit_scratch_floats() * 4;
  size_t free_b = 0, total_b = 0;
  cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemGetInfo");
  if (bytes > (int64_t)(free_b / 2)) return SPIDER_OK;
  // the shared-memory attribute first: the occupancy query depends on it
  if (configure_whiten_kernels() != cudaSuccess) {
    cudaGetLastError();            // this device cannot run the direct path: the general solver serves
    return SPIDER_OK;
  }
  c->cc_grid = piece_cc_grid(c->num_sms);
  c->clean_grid = whiten_clean_grid(c->num_sms);
  if (c->cc_grid < 1 || whiten_units_grids(c->num_sms, c->unit_grids) < 1 || c->clean_grid < 1) return SPIDER_OK;
  c->unit_grids[3] = c->num_sms;
  auto& L = c->allocs;
  StepView& v = c->v;
  cudaStream_t st = c->stream;
  const size_t G = T.G, Q = P.Q;
#define UPF(field, src, n)                                                                       \
  do {                                                                                           \
    using _T = std::remove_const_t<std::remove_pointer_t<decltype(v.field)>>;                    \
    _T* _q = nullptr;                                                                            \
    if ((e = dupload(L, &_q, (const _T*)(src), (n), st))) return cuda_fail(c, e, "upload " #field); \
    v.field = _q;                                                                                \
  } while (0)
#define ALF(field, n)                                                                \
  do {                                                                               \
    using _T = std::remove_pointer_t<decltype(v.field)>;                             \
    _T* _q = nullptr;                                                                \
    if ((e = dalloc(L, &_q, (n)))) return cuda_fail(c, e, "alloc " #field);          \
    v.field = _q;                                                                    \
  } while (0)
  UPF(blk_piece_off, T.blk_piece_off.data(), P.NB + 1);
  UPF(node_piece, T.node_piece.data(), Q);
  UPF(node_ppos, T.node_ppos.data(), Q);
  UPF(piece_node_off, T.piece_node_off.data(), G + 1);
  UPF(piece_nodes, T.piece_nodes.data(), Q);
  UPF(piece_inv_off, T.piece_inv_off.data(), G + 1);
  UPF(mem_rp, T.mem_rp.data(), Q + 1);
  UPF(edge_pos, T.edge_pos.data(), T.edge_pos.size());
  UPF(edge_sw, T.edge_sw.data(), T.edge_sw.size());
  ALF(owner_b, Q);
  ALF(plab, G);
  ALF(pmulti, G);
  ALF(pcount, G);
  ALF(unit_of, G);
  ALF(unit_cnt, G);
  ALF(unit_off, G + 1);
  ALF(unit_pieces, G);
  ALF(unit_pblk, G);
  ALF(unit_defer, G);
  ALF(unit_defer2, G);
  {
    // the data-parallel unit solver: at most L_max occurrences per selected block
    const size_t cap = (size_t)std::max<int64_t>(1, c->nb_mb) * (size_t)P.L_max;
    v.u_cap = (int64_t)cap;
    v.ginv_cap = int64_t(1) << 25;
    v.sinv_cap = int64_t(1) << 24;
    ALF(u_nocc, G); ALF(uocc_off, G + 1); ALF(u_ng, G); ALF(u_m, G);
    ALF(u_gsz, G); ALF(u_goff, G + 1); ALF(u_ssz, G); ALF(u_soff, G + 1);
    ALF(pu_base, G); ALF(pu_unit, G); ALF(pu_gb, G); ALF(pu_gn, G); ALF(pu_ginv, G);
    ALF(o_g, cap); ALF(o_pe, cap); ALF(o_base, cap); ALF(o_u, cap); ALF(o_x, cap); ALF(o_unit, cap);
    ALF(o_t, cap); ALF(o_i, cap);
    ALF(o_uh, cap); ALF(o_ul, cap); ALF(o_zh, cap); ALF(o_zl, cap); ALF(o_f, cap); ALF(o_w, cap);
    ALF(o_ph, cap); ALF(o_pl, cap);
    ALF(sh_slot, cap); ALF(sh_sorted, cap); ALF(sh_tt, cap);
    ALF(g_u, cap); ALF(g_beg, cap); ALF(g_cnt, cap);
    ALF(g_uh, cap); ALF(g_ul, cap); ALF(g_zh, cap); ALF(g_zl, cap); ALF(g_f, cap); ALF(g_x, cap);
    ALF(ginv_pool, (size_t)v.ginv_cap); ALF(sinv_pool, (size_t)v.sinv_cap);
  }
  ALF(clean_list, G);
  ALF(clean_blk, G);
  ALF(wfast, kWSlots + 64 + 32);
  ALF(wscratch, (size_t)c->unit_grids[2] * whiten_unit_scratch_floats());
#undef UPF
#undef ALF
  float* inv = nullptr;
  if ((e = dalloc(L, &inv, (size_t)inv_floats))) return cuda_fail(c, e, "alloc piece inverses");
  v.piece_inv = inv;
  // the inverses block by block in chunks of at most 64 M floats
  const double lam = (double)c->cfg.sigma * c->cfg.sigma / ((double)c->cfg.kappa * c->cfg.kappa);
  std::vector<float> buf;
  for (int64_t b0 = 0; b0 < P.NB;) {
    int64_t b1 = b0 + 1;
    const int64_t f0 = T.piece_inv_off[T.blk_piece_off[b0]];
    while (b1 < P.NB && T.piece_inv_off[T.blk_piece_off[b1 + 1]] - f0 <= (int64_t(1) << 26)) ++b1;
    const int64_t nf = T.piece_inv_off[T.blk_piece_off[b1]] - f0;
    buf.resize((size_t)std::max<int64_t>(nf, 1));
    piece_inverses(P, T, lam, b0, b1, buf.data(), 0);
    if (nf > 0) {
      if ((e = cudaMemcpyAsync(inv + f0, buf.data(), nf * sizeof(float), cudaMemcpyHostToDevice, st)))
        return cuda_fail(c, e, "upload piece inverses");
      if ((e = cudaStreamSynchronize(st))) return cuda_fail(c, e, "upload piece inverses");
    }
    b0 = b1;
  }
  if ((e = cudaStreamSynchronize(st))) return cuda_fail(c, e, "upload sync");
  if ((e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking))) return cuda_fail(c, e, "side stream");
  if ((e = cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming))) return cuda_fail(c, e, "event");
  if ((e = cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming))) return cuda_fail(c, e, "event");
  if ((e = cudaEventCreateWithFlags(&c->ubr.fork, cudaEventDisableTiming))) return cuda_fail(c, e, "event");
  for (int i = 0; i < 4; ++i) {
    if ((e = cudaStreamCreateWithFlags(&c->ubr.s[i], cudaStreamNonBlocking))) return cuda_fail(c, e, "branch stream");
    if ((e = cudaEventCreateWithFlags(&c->ubr.join[i], cudaEventDisableTiming))) return cuda_fail(c, e, "event");
  }
  c->piece_bytes = bytes;
  c->fast = true;
  return SPIDER_OK;
}

// Builds a context over a catalog made of n_sub independent sub-problems
// (a single catalog is one sub-problem); see prepare() for the splits.
int create_impl(const spider_catalog* cat, const spider_stations* sta, const spider_net* net,
                const spider_config* cfg, void* stream, spider_ctx** out,
                const std::vector<int64_t>* ev_splits, const std::vector<int64_t>* obs_splits,
                const std::vector<int32_t>& sub_chain, const std::vector<int32_t>& sub_catalog) {
  if (!out) return SPIDER_E_INVAL;
  *out = nullptr;
  spider_ctx* c = new spider_ctx();
  auto bail = [&](int code) {
    g_static_err = "spider_create failed";
    static thread_local std::string last;
    last = c->err;
    g_static_err = last.c_str();
    free_all(c->allocs);
    for (auto& ev : c->ev)
      if (ev) cudaEventDestroy(ev);
    for (auto& ev : c->wev)
      if (ev) cudaEventDestroy(ev);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->fork) cudaEventDestroy(c->fork);
    if (c->join) cudaEventDestroy(c->join);
    destroy_branches(c->ubr);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return code;
  };
  if (!cfg) { c->err = "null config"; return bail(SPIDER_E_INVAL); }
  c->cfg = *cfg;
  if (c->cfg.thin < 1 || c->cfg.pcg_max_it < 0 || !(c->cfg.pcg_tol >= 0.f) || c->cfg.sample_cap < 0 ||
      !(c->cfg.noise_scale >= 0.f)) {
    c->err = "need thin >= 1, pcg_max_it >= 0, pcg_tol >= 0, sample_cap >= 0, noise_scale >= 0";
    return bail(SPIDER_E_INVAL);
  }
  if (c->cfg.update < SPIDER_UPDATE_SGLD || c->cfg.update > SPIDER_UPDATE_ADAM ||
      c->cfg.loss < SPIDER_LOSS_WHITENED || c->cfg.loss > SPIDER_LOSS_L1 || !(c->cfg.beta1 >= 0.f) ||
      !(c->cfg.beta1 < 1.f) || !(c->cfg.beta2 >= 0.f) || !(c->cfg.beta2 < 1.f) || !(c->cfg.upd_eps > 0.f)) {
    c->err = "need update in SPIDER_UPDATE_*, loss in SPIDER_LOSS_*, beta1, beta2 in [0, 1), upd_eps > 0";
    return bail(SPIDER_E_INVAL);
  }
  int rc = check_net(net, cfg->precision, &c->err);
  if (rc) return bail(rc);
  Prep P;
  rc = prepare(cat, sta, cfg, &P, &c->err, 0, ev_splits, obs_splits);
  if (rc) return bail(rc);
  c->n_sub = P.n_sub;

  cudaError_t e;
  if ((e = cudaGetDevice(&c->device))) return bail(cuda_fail(c, e, "cudaGetDevice"));
  if ((e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device)))
    return bail(cuda_fail(c, e, "device attribute"));
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking))) return bail(cuda_fail(c, e, "stream"));
    c->own_stream = true;
  }
  cudaStream_t st = c->stream;
  auto& L = c->allocs;
  StepView& v = c->v;
  v.M = P.M; v.N = P.N; v.S = P.S; v.NB = P.NB; v.B = P.B; v.P = P.P; v.Q = P.Q; v.L_max = P.L_max;
  const size_t M = P.M, N = P.N, S = P.S, NB = P.NB, PP = P.P, Q = P.Q;

  std::vector<float4> h_hi(M), h_lo(M);
  for (size_t m = 0; m < M; ++m) {
    float hx[4], lx[4];
    for (int a = 0; a < 4; ++a) split_df(P.th0[4 * m + a], hx[a], lx[a]);
    h_hi[m] = make_float4(hx[0], hx[1], hx[2], hx[3]);
    h_lo[m] = make_float4(lx[0], lx[1], lx[2], lx[3]);
  }
  std::vector<float4> s_hi(S), s_lo(S);
  for (size_t s = 0; s < S; ++s) {
    float hx[3], lx[3];
    for (int a = 0; a < 3; ++a) split_df(sta->xyz[3 * s + a], hx[a], lx[a]);
    s_hi[s] = make_float4(hx[0], hx[1], hx[2], 0.f);
    s_lo[s] = make_float4(lx[0], lx[1], lx[2], 0.f);
  }
#define UP(field, src, n)                                                       \
  do {                                                                          \
    decltype(v.field) _p;                                                       \
    using _T = std::remove_const_t<std::remove_pointer_t<decltype(v.field)>>;   \
    _T* _q = nullptr;                                                           \
    if ((e = dupload(L, &_q, (const _T*)(src), (n), st))) return bail(cuda_fail(c, e, "upload " #field)); \
    _p = _q;                                                                    \
    v.field = _p;                                                               \
  } while (0)
#define AL(field, n)                                                            \
  do {                                                                          \
    using _T = std::remove_pointer_t<decltype(v.field)>;                        \
    _T* _q = nullptr;                                                           \
    if ((e = dalloc(L, &_q, (n)))) return bail(cuda_fail(c, e, "alloc " #field)); \
    v.field = _q;                                                               \
  } while (0)
  UP(th0_hi, h_hi.data(), M);
  UP(th0_lo, h_lo.data(), M);
  UP(th0_d, P.th0.data(), 4 * M);
  UP(ev_out, P.ev_old.data(), M);
  UP(ev_caller, P.ev_local.data(), M);
  {
    // sub-problem tables
    const int ns = P.n_sub;
    std::vector<int32_t> blk_off(ns + 1), sel_full(ns + 1, 0), sel_mb(ns + 1, 0), nobs(ns), nev(ns), ch(ns), ca(ns);
    std::vector<int32_t> chunk_ev0, sub_chunk_off(ns + 1, 0);
    const bool bfull = cfg->batch_n <= 0 || cfg->batch_n >= (int64_t)N;
    for (int s2 = 0; s2 < ns; ++s2) {
      blk_off[s2] = (int32_t)P.sub_blk_off[s2];
      const int64_t nbs = P.sub_blk_off[s2 + 1] - P.sub_blk_off[s2];
      const int64_t want = bfull ? nbs : std::min<int64_t>(nbs, (cfg->batch_n + P.B - 1) / P.B);
      sel_full[s2 + 1] = sel_full[s2] + (int32_t)nbs;
      sel_mb[s2 + 1] = sel_mb[s2] + (int32_t)want;
      if (!bfull && want == nbs && nbs > 1) c->mb_full_sub = true;
      nobs[s2] = (int32_t)(P.sub_obs_off[s2 + 1] - P.sub_obs_off[s2]);
      nev[s2] = (int32_t)(P.sub_ev_off[s2 + 1] - P.sub_ev_off[s2]);
      ch[s2] = sub_chain[s2];
      ca[s2] = sub_catalog[s2];
      sub_chunk_off[s2] = (int32_t)chunk_ev0.size();
      for (int64_t m = P.sub_ev_off[s2]; m < P.sub_ev_off[s2 + 1]; m += kCenChunk) chunk_ev0.push_back((int32_t)m);
    }
    blk_off[ns] = (int32_t)P.sub_blk_off[ns];
    sub_chunk_off[ns] = (int32_t)chunk_ev0.size();
    chunk_ev0.push_back((int32_t)M);
    v.n_sub = ns;
    v.n_chunks = (int)chunk_ev0.size() - 1;
    c->nb_full = sel_full[ns];
    c->nb_mb = sel_mb[ns];
    UP(blk_e0, P.blk_e0.data(), NB + 1);
    UP(blk_sub, P.blk_sub.data(), NB);
    UP(ev_sub, P.ev_sub.data(), M);
    UP(sub_blk_off, blk_off.data(), ns + 1);
    UP(sub_sel_full, sel_full.data(), ns + 1);
    UP(sub_sel_mb, sel_mb.data(), ns + 1);
    UP(sub_nobs, nobs.data(), ns);
    UP(sub_nev, nev.data(), ns);
    UP(sub_chain, ch.data(), ns);
    UP(sub_catalog, ca.data(), ns);
    UP(chunk_ev0, chunk_ev0.data(), chunk_ev0.size());
    UP(sub_chunk_off, sub_chunk_off.data(), ns + 1);
    AL(sub_nsel, ns);
    AL(sub_cen, ns);
    AL(cen_chunk, chunk_ev0.size());
    StepParams* pp = nullptr;
    if ((e = dalloc(L, &pp, 1))) return bail(cuda_fail(c, e, "alloc params"));
    c->prm = pp;
    v.prm = pp;
    // the host copies of the tables above must outlive the asynchronous uploads
    if ((e = cudaStreamSynchronize(st))) return bail(cuda_fail(c, e, "upload sync"));
  }
  UP(sta_hi, s_hi.data(), S);
  UP(sta_lo, s_lo.data(), S);
  UP(pair_ev, P.pair_ev.data(), PP);
  UP(pair_st, P.pair_st.data(), PP);
  UP(pair_off, P.pair_off.data(), M + 1);
  UP(obs_l, P.obs_l.data(), N);
  UP(obs_dt, P.obs_dt.data(), N);
  UP(obs_sw, P.obs_sw.data(), N);
  UP(blk_node_off, P.blk_node_off.data(), NB + 1);
  UP(node_pair, P.node_pair.data(), Q);
  UP(node_he, P.node_he.data(), Q);
  UP(blk_he, P.blk_he.data(), 2 * N);
  UP(inc_off, P.inc_off.data(), PP + 1);
  UP(inc_q, P.inc_q.data(), Q);
  UP(inc_b, P.inc_b.data(), Q);
  AL(dth, M);
  AL(sel, NB);
  AL(blk_stamp, NB);
  AL(owner_q, Q);
  AL(multi, Q);
  AL(loc2u, Q);
  AL(blk_owner_cnt, NB);
  AL(blk_owner_off, NB);
  AL(uniq_pair, PP);
  AL(uniq_q, PP);
  AL(T2, PP);
  AL(J, PP);
  AL(r_obs, N);
  AL(q_obs, N);
  AL(part_a, Q);
  AL(part_b, Q);
  AL(part_c, Q);
  AL(rhs, PP);
  AL(rhs_lo, PP);
  AL(diag, PP);
  AL(z, PP);
  AL(z_lo, PP);
  AL(rres, PP);
  AL(dz, PP);
  AL(res, PP);
  AL(pv, PP);
  AL(pv2, PP);
  AL(umulti, PP);
  AL(rowlen, PP);
  AL(rowptr, PP + 1);
  AL(occ_off, Q);
  AL(csr_col, 2 * N);
  AL(csr_sw, 2 * N);
  AL(scan_part, kMaxGrid + 1);
  AL(lab, PP);
  AL(cslot, PP);
  AL(ccount, PP);
  AL(comp_root, PP);
  AL(comp_off, PP + 1);
  AL(members, PP + 1);
  AL(lidx, PP);
  AL(big, PP);
  AL(chist, 512);
  AL(cc_lroot, Q);
  AL(bigpos, PP + 1);
  AL(biglist, PP);
  AL(corder, PP);
  AL(centries, PP);
  AL(ctier, PP);
  AL(Ap, PP);
  AL(yv, PP);
  AL(s_u, PP);
  AL(gp, PP);
  AL(pstamp, PP);
  AL(estamp, M);
  AL(grad, M);
  AL(counters, kCntSlots);
  AL(red, 8 * kMaxGrid);
  AL(dblk, NB);
  AL(dred, 4 * kMaxGrid);
  AL(dout, 8);
  {
    double* sd = nullptr;
    float4* gd = nullptr;
    if ((e = dalloc(L, &sd, 4 * M))) return bail(cuda_fail(c, e, "alloc read-back"));
    if ((e = dalloc(L, &gd, M))) return bail(cuda_fail(c, e, "alloc read-back"));
    c->state_dev = sd;
    c->grad_dev = gd;
  }
  const int64_t cap = c->cfg.sample_cap;
  AL(samples, (size_t)std::max<int64_t>(cap, 1) * M);
  if (c->cfg.update != SPIDER_UPDATE_SGLD) {
    AL(mom2, M);
    if ((e = cudaMemsetAsync(v.mom2, 0, M * sizeof(float4), st))) return bail(cuda_fail(c, e, "memset"));
  }
  if (c->cfg.update == SPIDER_UPDATE_ADAM) {
    AL(mom1, M);
    if ((e = cudaMemsetAsync(v.mom1, 0, M * sizeof(float4), st))) return bail(cuda_fail(c, e, "memset"));
  }
#undef UP
#undef AL
  v.sample_cap = cap;
  if ((e = cudaMemsetAsync(v.dth, 0, M * sizeof(float4), st))) return bail(cuda_fail(c, e, "memset"));
  if ((e = cudaMemsetAsync(v.blk_stamp, 0xFF, NB * sizeof(int32_t), st))) return bail(cuda_fail(c, e, "memset"));
  if ((e = cudaMemsetAsync(v.pstamp, 0xFF, PP * sizeof(int32_t), st))) return bail(cuda_fail(c, e, "memset"));
  if ((e = cudaMemsetAsync(v.estamp, 0xFF, M * sizeof(int32_t), st))) return bail(cuda_fail(c, e, "memset"));
  if ((e = cudaMemsetAsync(v.counters, 0, kCntSlots * sizeof(int32_t), st))) return bail(cuda_fail(c, e, "memset"));
  const double s2 = cfg->sigma * cfg->sigma;
  v.whiten = (cfg->kappa > 0.0 && cfg->loss == SPIDER_LOSS_WHITENED) ? 1 : 0;
  v.loss = cfg->loss;
  v.update = cfg->update;
  v.beta1 = cfg->beta1;
  v.beta2 = cfg->beta2;
  v.upd_eps = cfg->upd_eps;
  v.lam = v.whiten ? (float)(s2 / (cfg->kappa * cfg->kappa)) : 0.f;
  v.inv_s2 = (float)(1.0 / s2);
  v.inv_sig_e2 = make_float4((float)(1.0 / (cfg->sig_e[0] * cfg->sig_e[0])), (float)(1.0 / (cfg->sig_e[1] * cfg->sig_e[1])),
                             (float)(1.0 / (cfg->sig_e[2] * cfg->sig_e[2])), (float)(1.0 / (cfg->sig_e[3] * cfg->sig_e[3])));
  v.inv_sig_c2 = make_float4((float)(1.0 / (cfg->sig_c[0] * cfg->sig_c[0])), (float)(1.0 / (cfg->sig_c[1] * cfg->sig_c[1])),
                             (float)(1.0 / (cfg->sig_c[2] * cfg->sig_c[2])), (float)(1.0 / (cfg->sig_c[3] * cfg->sig_c[3])));
  v.cen_grid = (int)std::min<int64_t>((int64_t)(M + 255) / 256, (int64_t)std::min(kMaxGrid, 4 * c->num_sms));
  c->gu = std::min(kMaxGrid, 4 * c->num_sms);
  c->grid_ev = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)(M + 255) / 256, 8 * c->num_sms));

  if ((e = upload_net(net, cfg->precision, &c->net, L, st))) return bail(cuda_fail(c, e, "network upload"));
  c->net.err = v.counters + kCntError;
  const size_t scr = tt_scratch_floats(c->net, c->num_sms);
  if (scr) {
    if ((e = dalloc(L, &c->tt_scratch, scr))) return bail(cuda_fail(c, e, "alloc scratch"));
  }
  if ((e = configure_step_kernels(v))) return bail(cuda_fail(c, e, "kernel attributes"));
  c->pgrid = pcg_grid(v, c->num_sms);
  if (c->pgrid < 1) {
    c->err = "whitening kernel does not fit on the device (block too large)";
    return bail(SPIDER_E_UNSUPPORTED);
  }
  if (v.whiten && !(cfg->batch_n <= 0 || cfg->batch_n >= (int64_t)N)) {
    rc = build_fast_whitening(c, P);
    if (rc) return bail(rc);
  }
  c->ev_old = std::move(P.ev_old);
  c->ord = std::move(P.ord);
  c->th0 = std::move(P.th0);
  for (int i = 0; i < spider_ctx::kEv; ++i)
    if ((e = cudaEventCreate(&c->ev[i]))) return bail(cuda_fail(c, e, "event"));
  for (int i = 0; i < 5; ++i)
    if ((e = cudaEventCreate(&c->wev[i]))) return bail(cuda_fail(c, e, "event"));
  if ((e = cudaStreamSynchronize(st))) return bail(cuda_fail(c, e, "create sync"));
  *out = c;
  return SPIDER_OK;
}

}  // namespace

extern "C" {

int spider_create(const spider_catalog* cat, const spider_stations* sta, const spider_net* net,
                  const spider_config* cfg, void* stream, spider_ctx** out) {
  const std::vector<int32_t> ch{cfg ? cfg->chain : 0}, ca{cfg ? cfg->catalog : 0};
  return create_impl(cat, sta, net, cfg, stream, out, nullptr, nullptr, ch, ca);
}

int spider_create_batch(int32_t n_catalogs, const spider_catalog* cats, const spider_stations* stas,
                        const spider_net* net, const spider_config* cfg, int32_t chains, void* stream,
                        spider_ctx** out) {
  if (!out) return SPIDER_E_INVAL;
  *out = nullptr;
  if (n_catalogs < 1 || chains < 1 || !cats || !stas || !cfg) {
    g_static_err = "spider_create_batch: need n_catalogs >= 1, chains >= 1 and non-null arrays";
    return SPIDER_E_INVAL;
  }
  // concatenate catalog x chain sub-problems: events and observations copied per
  // chain, stations once per catalog
  int64_t M = 0, N = 0, S = 0;
  bool any_w = false, all_w = true;
  for (int c = 0; c < n_catalogs; ++c) {
    if (!cats[c].xyzt0 || !cats[c].i || !cats[c].j || !cats[c].k || !cats[c].dt || !stas[c].xyz ||
        cats[c].M < 2 || cats[c].N < 1 || stas[c].S < 1) {
      g_static_err = "spider_create_batch: catalog with null arrays or empty sizes";
      return SPIDER_E_INVAL;
    }
    M += cats[c].M * chains;
    N += cats[c].N * chains;
    S += stas[c].S;
    any_w |= cats[c].w != nullptr;
    all_w &= cats[c].w != nullptr;
  }
  if (any_w != all_w) {
    g_static_err = "spider_create_batch: give edge weights for every catalog or for none";
    return SPIDER_E_INVAL;
  }
  if (M > INT32_MAX || N >= (int64_t(1) << 30)) {
    g_static_err = "spider_create_batch: the batch exceeds 2^31 events or 2^30 observations";
    return SPIDER_E_INVAL;
  }
  std::vector<double> xyzt(4 * M), dt(N), sxyz(3 * S);
  std::vector<int32_t> I(N), J(N), K(N);
  std::vector<float> W(all_w ? N : 0);
  std::vector<int64_t> evs{0}, obss{0};
  std::vector<int32_t> ch, ca;
  int64_t m0 = 0, n0 = 0, s0 = 0;
  for (int c = 0; c < n_catalogs; ++c) {
    const spider_catalog& k = cats[c];
    std::copy(stas[c].xyz, stas[c].xyz + 3 * stas[c].S, sxyz.begin() + 3 * s0);
    for (int h = 0; h < chains; ++h) {
      std::copy(k.xyzt0, k.xyzt0 + 4 * k.M, xyzt.begin() + 4 * m0);
      for (int64_t n = 0; n < k.N; ++n) {
        const bool ok = k.i[n] >= 0 && k.i[n] < k.M && k.j[n] >= 0 && k.j[n] < k.M && k.k[n] >= 0 &&
                        k.k[n] < stas[c].S;
        // out-of-range indices are kept out of range so that prepare() rejects them
        I[n0 + n] = ok ? (int32_t)(k.i[n] + m0) : -1;
        J[n0 + n] = ok ? (int32_t)(k.j[n] + m0) : -1;
        K[n0 + n] = ok ? (int32_t)(k.k[n] + s0) : -1;
        dt[n0 + n] = k.dt[n];
        if (all_w) W[n0 + n] = k.w[n];
      }
      m0 += k.M;
      n0 += k.N;
      evs.push_back(m0);
      obss.push_back(n0);
      ch.push_back(h);
      ca.push_back(c);
    }
    s0 += stas[c].S;
  }
  spider_catalog all{M, N, xyzt.data(), I.data(), J.data(), K.data(), dt.data(), all_w ? W.data() : nullptr};
  spider_stations sall{(int32_t)S, sxyz.data()};
  return create_impl(&all, &sall, net, cfg, stream, out, &evs, &obss, ch, ca);
}

int spider_grad_logpost(spider_ctx* c, uint64_t batch_seed, float* grad_out, double* logpost_out) {
  if (!c) return SPIDER_E_INVAL;
  int rc = evaluate(c, batch_seed, 0, 0.f);
  if (rc) return rc;
  const size_t M = c->v.M;
  double lp = 0.0;
  if (grad_out) {
    // reordered to the caller's events on the device, then one copy
    CK(c, launch_grad_out(c->v, c->grad_dev, c->grid_ev, c->stream));
    CK(c, cudaMemcpyAsync(grad_out, c->grad_dev, M * sizeof(float4), cudaMemcpyDeviceToHost, c->stream));
  }
  if (logpost_out) CK(c, cudaMemcpyAsync(&lp, c->v.dout + 3, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  rc = check_device_error(c);
  if (rc) return rc;
  if (logpost_out) *logpost_out = lp;
  return SPIDER_OK;
}

int spider_sgld_step(spider_ctx* c, float eps, uint64_t batch_seed) {
  if (!c) return SPIDER_E_INVAL;
  if (!(eps > 0.f) || !std::isfinite(eps)) {
    c->err = "eps must be finite and > 0";
    return SPIDER_E_INVAL;
  }
  return evaluate(c, batch_seed, 1, eps);
}

int spider_samples(spider_ctx* c, double* out, int64_t cap, int64_t* n_written) {
  if (!c || !n_written || (cap > 0 && !out)) return SPIDER_E_INVAL;
  CK(c, cudaStreamSynchronize(c->stream));
  int rc = check_device_error(c);
  if (rc) return rc;
  const int64_t have = std::min<int64_t>(c->n_samples, c->v.sample_cap);
  const int64_t n = std::min<int64_t>(have, cap);
  const int64_t first = c->n_samples - have;     // oldest kept sample index
  const size_t M = c->v.M;
  for (int64_t s = 0; s < n; ++s) {
    const int64_t slot = (first + s) % c->v.sample_cap;
    CK(c, launch_state_out(c->v, c->v.samples + slot * M, c->state_dev, c->grid_ev, c->stream));
    CK(c, cudaMemcpyAsync(out + (size_t)s * 4 * M, c->state_dev, 4 * M * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
  }
  *n_written = n;
  return SPIDER_OK;
}

int spider_get_state(spider_ctx* c, double* theta_out, int64_t* step_out) {
  if (!c) return SPIDER_E_INVAL;
  const size_t M = c->v.M;
  if (theta_out) {
    // theta_0 + dtheta formed on the device in FP64 and the caller's order:
    // one device-to-host copy (a page-locked theta_out is copied by DMA)
    CK(c, launch_state_out(c->v, c->v.dth, c->state_dev, c->grid_ev, c->stream));
    CK(c, cudaMemcpyAsync(theta_out, c->state_dev, 4 * M * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  CK(c, cudaStreamSynchronize(c->stream));
  int rc = check_device_error(c);
  if (rc) return rc;
  if (step_out) *step_out = c->step;
  return SPIDER_OK;
}

int spider_set_state(spider_ctx* c, const double* theta, int64_t step) {
  if (!c || !theta || step < 0) return SPIDER_E_INVAL;
  const size_t M = c->v.M;
  std::vector<float4> buf(M);
  for (size_t m = 0; m < M; ++m) {
    const double* x = theta + 4 * (size_t)c->ev_old[m];
    const double* t = &c->th0[4 * m];
    for (int a = 0; a < 4; ++a)
      if (!std::isfinite(x[a])) {
        c->err = "non-finite state";
        return SPIDER_E_INVAL;
      }
    buf[m] = make_float4((float)(x[0] - t[0]), (float)(x[1] - t[1]), (float)(x[2] - t[2]), (float)(x[3] - t[3]));
  }
  CK(c, cudaMemcpyAsync(c->v.dth, buf.data(), M * sizeof(float4), cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->step = step;
  return SPIDER_OK;
}

static int moments_io(spider_ctx* c, double* m_out, double* v_out, const double* m_in, const double* v_in) {
  if (!c) return SPIDER_E_INVAL;
  if (c->cfg.update == SPIDER_UPDATE_SGLD) {
    c->err = "the SGLD update keeps no moments";
    return SPIDER_E_INVAL;
  }
  const size_t M = c->v.M;
  float4* dev[2] = {c->v.mom1, c->v.mom2};
  double* outs[2] = {m_out, v_out};
  const double* ins[2] = {m_in, v_in};
  std::vector<float4> buf(M);
  for (int k = 0; k < 2; ++k) {
    if (!dev[k]) continue;
    if (outs[k]) {
      CK(c, cudaMemcpyAsync(buf.data(), dev[k], M * sizeof(float4), cudaMemcpyDeviceToHost, c->stream));
      CK(c, cudaStreamSynchronize(c->stream));
      for (size_t m = 0; m < M; ++m) {
        double* x = outs[k] + 4 * (size_t)c->ev_old[m];
        x[0] = buf[m].x; x[1] = buf[m].y; x[2] = buf[m].z; x[3] = buf[m].w;
      }
    }
    if (ins[k]) {
      for (size_t m = 0; m < M; ++m) {
        const double* x = ins[k] + 4 * (size_t)c->ev_old[m];
        for (int a = 0; a < 4; ++a)
          if (!std::isfinite(x[a]) || (k == 1 && x[a] < 0.0)) {
            c->err = "moments must be finite (and the second moment non-negative)";
            return SPIDER_E_INVAL;
          }
        buf[m] = make_float4((float)x[0], (float)x[1], (float)x[2], (float)x[3]);
      }
      CK(c, cudaMemcpyAsync(dev[k], buf.data(), M * sizeof(float4), cudaMemcpyHostToDevice, c->stream));
      CK(c, cudaStreamSynchronize(c->stream));
    }
  }
  return check_device_error(c);
}

int spider_set_noise_scale(spider_ctx* c, float noise_scale) {
  if (!c || !(noise_scale >= 0.f) || !std::isfinite(noise_scale)) return SPIDER_E_INVAL;
  c->cfg.noise_scale = noise_scale;
  return SPIDER_OK;
}

int spider_get_moments(spider_ctx* c, double* m_out, double* v_out) {
  return moments_io(c, m_out, v_out, nullptr, nullptr);
}

int spider_set_moments(spider_ctx* c, const double* m, const double* v) {
  return moments_io(c, nullptr, nullptr, m, v);
}

int spider_outlier_mask(spider_ctx* c, double k_mad, uint8_t* keep_out, int64_t* n_kept_out, double* med_out,
                        double* mad_out) {
  if (!c || !(k_mad > 0.0) || !std::isfinite(k_mad)) return SPIDER_E_INVAL;
  int rc = evaluate(c, 0, 0, 0.f);          // full-batch residuals at the current state
  if (rc) return rc;
  rc = spider_sync(c);
  if (rc) return rc;
  const int ns = c->n_sub;
  const size_t N = c->v.N;
  void* scratch = nullptr;
  uint8_t* keep = nullptr;
  CK(c, cudaMallocAsync(&scratch, outlier_scratch_bytes(ns), c->stream));
  cudaError_t e = cudaMallocAsync(&keep, N > 0 ? N : 1, c->stream);
  std::vector<float> med(ns), mad(ns);
  int64_t kept = 0;
  if (e == cudaSuccess)
    e = launch_outlier(c->v, ns, (float)k_mad, scratch, keep, c->num_sms, c->stream, med.data(), mad.data(), &kept);
  std::vector<uint8_t> hk;
  if (e == cudaSuccess && keep_out) {
    hk.resize(N);
    e = cudaMemcpyAsync(hk.data(), keep, N, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  }
  if (keep) cudaFreeAsync(keep, c->stream);
  cudaFreeAsync(scratch, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "outlier mask");
  if (keep_out)
    for (size_t n = 0; n < N; ++n) keep_out[c->ord[n]] = hk[n];
  if (n_kept_out) *n_kept_out = kept;
  for (int i = 0; i < ns; ++i) {
    if (med_out) med_out[i] = med[i];
    if (mad_out) mad_out[i] = mad[i];
  }
  return check_device_error(c);
}

int spider_linearisation_mask(spider_ctx* c, double max_rel, uint8_t* keep_out, int64_t* n_kept_out) {
  if (!c || !(max_rel >= 0.0) || !std::isfinite(max_rel)) return SPIDER_E_INVAL;
  int rc = evaluate(c, 0, 0, 0.f);          // T and dT/dx of every pair at the current state
  if (rc) return rc;
  rc = spider_sync(c);
  if (rc) return rc;
  const size_t N = c->v.N;
  uint8_t* keep = nullptr;
  unsigned long long* kept = nullptr;
  CK(c, cudaMallocAsync(&kept, sizeof(unsigned long long), c->stream));
  cudaError_t e = cudaMallocAsync(&keep, N > 0 ? N : 1, c->stream);
  if (e == cudaSuccess) e = launch_linfilter(c->v, c->nb_full, (float)max_rel, keep, kept, c->stream);
  std::vector<uint8_t> hk(keep_out ? N : 0);
  unsigned long long kh = 0;
  if (e == cudaSuccess && keep_out) e = cudaMemcpyAsync(hk.data(), keep, N, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&kh, kept, sizeof(kh), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (keep) cudaFreeAsync(keep, c->stream);
  cudaFreeAsync(kept, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "linearisation mask");
  if (keep_out)
    for (size_t n = 0; n < N; ++n) keep_out[c->ord[n]] = hk[n];
  if (n_kept_out) *n_kept_out = (int64_t)kh;
  return check_device_error(c);
}

int spider_uq(spider_ctx* c, const double* truth, double lo_pct, double hi_pct, double* median_out,
              double* halfwidth_out, double* calib_out, double* ess_out) {
  if (!c || !(lo_pct >= 0.0) || !(hi_pct <= 100.0) || !(lo_pct <= hi_pct)) return SPIDER_E_INVAL;
  CK(c, cudaStreamSynchronize(c->stream));
  int rc = check_device_error(c);
  if (rc) return rc;
  const int64_t have = std::min<int64_t>(c->n_samples, c->v.sample_cap);
  if (have < 2 || have > uq_max_samples()) {
    c->err = "spider_uq needs 2..4096 stored samples";
    return SPIDER_E_INVAL;
  }
  const int64_t first = c->n_samples - have;
  const size_t M = c->v.M;
  std::vector<double> toff;
  if (truth) {
    toff.resize(4 * M);
    for (size_t m = 0; m < M; ++m)
      for (int a = 0; a < 4; ++a) toff[4 * m + a] = truth[4 * (size_t)c->ev_old[m] + a] - c->th0[4 * m + a];
  }
  double* d = nullptr;
  const size_t nb = 4 * M * sizeof(double);
  CK(c, cudaMallocAsync(&d, 5 * nb, c->stream));
  double* dt = d;
  double* outs[4] = {d + 4 * M, d + 8 * M, d + 12 * M, d + 16 * M};
  double* want[4] = {median_out, halfwidth_out, calib_out, ess_out};
  cudaError_t e = cudaSuccess;
  if (truth) e = cudaMemcpyAsync(dt, toff.data(), nb, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = launch_uq(c->v, first % c->v.sample_cap, (int)have, truth ? dt : nullptr, lo_pct, hi_pct,
                  want[0] ? outs[0] : nullptr, want[1] ? outs[1] : nullptr, truth && want[2] ? outs[2] : nullptr,
                  want[3] ? outs[3] : nullptr, c->stream);
  std::vector<double> h(4 * M);
  for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
    if (!want[k] || (k == 2 && !truth)) continue;
    e = cudaMemcpyAsync(h.data(), outs[k], nb, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) break;
    for (size_t m = 0; m < M; ++m)
      for (int a = 0; a < 4; ++a) {
        double val = h[4 * m + a];
        if (k == 0) val += c->th0[4 * m + a];          // the median back to absolute coordinates
        want[k][4 * (size_t)c->ev_old[m] + a] = val;
      }
  }
  cudaFreeAsync(d, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "posterior summaries");
  if (calib_out && !truth)
    for (size_t i = 0; i < 4 * M; ++i) calib_out[i] = std::nan("");
  return check_device_error(c);
}

int spider_sync(spider_ctx* c) {
  if (!c) return SPIDER_E_INVAL;
  CK(c, cudaStreamSynchronize(c->stream));
  return check_device_error(c);
}

int spider_set_wait_limit_ns(spider_ctx* c, uint64_t limit_ns) {
  if (!c || limit_ns > 600000000000ull) return SPIDER_E_INVAL;
  c->wait_ns = limit_ns;
  return SPIDER_OK;
}

int spider_set_timing(spider_ctx* c, int enable) {
  if (!c) return SPIDER_E_INVAL;
  c->timing = enable != 0;
  return SPIDER_OK;
}

int spider_last_timing(spider_ctx* c, float out_ms[5], int64_t* pairs, int64_t* n_obs, int32_t* pcg_iters) {
  if (!c) return SPIDER_E_INVAL;
  int32_t cnt[kCntSlots] = {0};
  CK(c, cudaMemcpyAsync(cnt, c->v.counters, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (out_ms) {
    for (int i = 0; i < 5; ++i) out_ms[i] = 0.f;
    if (c->have_timing) {
      const int a[4] = {0, 1, 2, 5}, b[4] = {1, 2, 5, spider_ctx::kEv - 1};
      for (int i = 0; i < 4; ++i) CK(c, cudaEventElapsedTime(&out_ms[i], c->ev[a[i]], c->ev[b[i]]));
      CK(c, cudaEventElapsedTime(&out_ms[4], c->ev[0], c->ev[spider_ctx::kEv - 1]));
    }
  }
  if (pairs) *pairs = cnt[kCntPairs];
  if (n_obs) *n_obs = cnt[kCntObs];
  if (pcg_iters) *pcg_iters = cnt[kCntIters] > cnt[kCntCompIters] ? cnt[kCntIters] : cnt[kCntCompIters];
  return SPIDER_OK;
}

int spider_last_kernel_timing(spider_ctx* c, float out_ms[10], int64_t* touched_events) {
  if (!c) return SPIDER_E_INVAL;
  int32_t cnt[kCntSlots] = {0};
  CK(c, cudaMemcpyAsync(cnt, c->v.counters, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (out_ms) {
    for (int i = 0; i < 10; ++i) out_ms[i] = 0.f;
    if (c->have_timing)
      for (int i = 0; i < 10; ++i) CK(c, cudaEventElapsedTime(&out_ms[i], c->ev[i], c->ev[i + 1]));
  }
  if (touched_events) *touched_events = cnt[kCntEvents];
  return SPIDER_OK;
}

int spider_last_whiten_timing(spider_ctx* c, float out_ms[6]) {
  if (!c || !out_ms) return SPIDER_E_INVAL;
  CK(c, cudaStreamSynchronize(c->stream));
  for (int i = 0; i < 6; ++i) out_ms[i] = 0.f;
  if (!c->have_wtiming) return SPIDER_OK;
  const cudaEvent_t a[6] = {c->ev[4], c->wev[0], c->wev[1], c->wev[2], c->wev[3], c->wev[4]};
  const cudaEvent_t b[6] = {c->wev[0], c->wev[1], c->wev[2], c->wev[3], c->wev[4], c->ev[5]};
  for (int i = 0; i < 6; ++i) CK(c, cudaEventElapsedTime(&out_ms[i], a[i], b[i]));
  return SPIDER_OK;
}

int spider_debug_blocks(spider_ctx* c, int64_t* out, int64_t cap, int64_t* n) {
  if (!c || !n || (cap > 0 && !out)) return SPIDER_E_INVAL;
  std::vector<int32_t> s(c->last_nb);
  if (c->last_nb)
    CK(c, cudaMemcpyAsync(s.data(), c->v.sel, c->last_nb * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  const int64_t k = std::min<int64_t>(cap, c->last_nb);
  for (int64_t i = 0; i < k; ++i) out[i] = s[i];
  *n = c->last_nb;
  return SPIDER_OK;
}

int spider_debug_obs(spider_ctx* c, int64_t* idx_out, float* r_out, float* q_out, int64_t cap, int64_t* n) {
  if (!c || !n) return SPIDER_E_INVAL;
  std::vector<int32_t> s(c->last_nb);
  if (c->last_nb)
    CK(c, cudaMemcpyAsync(s.data(), c->v.sel, c->last_nb * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  const int64_t B = c->v.B, N = c->v.N;
  int64_t w = 0;
  std::vector<float> rb(B), qb(B);
  for (int64_t i = 0; i < c->last_nb; ++i) {
    const int64_t e0 = (int64_t)s[i] * B, ne = std::min(B, N - e0);
    if (w + ne <= cap) {
      CK(c, cudaMemcpy(rb.data(), c->v.r_obs + e0, ne * sizeof(float), cudaMemcpyDeviceToHost));
      CK(c, cudaMemcpy(qb.data(), c->v.q_obs + e0, ne * sizeof(float), cudaMemcpyDeviceToHost));
      for (int64_t e = 0; e < ne; ++e) {
        if (idx_out) idx_out[w + e] = c->ord[e0 + e];
        if (r_out) r_out[w + e] = rb[e];
        if (q_out) q_out[w + e] = qb[e];
      }
    }
    w += ne;
  }
  *n = w;
  return SPIDER_OK;
}

int spider_set_tuning(spider_ctx* c, const int32_t* knobs, int32_t n) {
  if (!c || (n > 0 && !knobs)) return SPIDER_E_INVAL;
  const int32_t lo[7] = {1, 1, 1, 0, 0, 1, 0}, hi[7] = {8, 4, 2, 1, 4, 4, 1};
  for (int32_t i = 0; i < n && i < 7; ++i)
    if (knobs[i] < lo[i] || knobs[i] > hi[i]) {
      c->err = "tuning knob out of range";
      return SPIDER_E_INVAL;
    }
  CK(c, cudaStreamSynchronize(c->stream));
  for (int32_t i = 0; i < n && i < 7; ++i) {
    if (i == 5 && knobs[i] == 3) {
      c->err = "tuning knob out of range";
      return SPIDER_E_INVAL;
    }
    c->knobs[i] = knobs[i];
  }
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->graph_exec = nullptr;
  c->graph = nullptr;
  return SPIDER_OK;
}

int spider_info(spider_ctx* c, int64_t* out, int32_t n) {
  if (!c || (n > 0 && !out)) return SPIDER_E_INVAL;
  int32_t cnt[kCntSlots] = {0};
  CK(c, cudaMemcpyAsync(cnt, c->v.counters, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  int32_t wf[kWSlots + 64 + 32] = {0};
  if (c->fast) {
    CK(c, cudaMemcpyAsync(wf, c->v.wfast, sizeof(wf), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
  }
  int64_t vals[39] = {c->n_sub, c->graph_exec ? 1 : 0, c->nb_mb, c->nb_full, c->v.P, c->v.M, c->v.N,
                      cnt[kCntComps], c->v.Q, c->fast ? 1 : 0, c->fast ? (c->mb_full_sub ? 0 : 1) : 0,
                      wf[kWUnits], wf[kWGeneral], wf[kWBigS], wf[kWCycSm], wf[kWCycBig]};
  for (int i = 0; i < 15; ++i) vals[16 + i] = wf[kWSlots + 64 + i];
  for (int i = 0; i < 7; ++i) vals[31 + i] = wf[kWSlots + 64 + 16 + i];
  vals[38] = c->graph_kernels;
  for (int32_t i = 0; i < n && i < 39; ++i) out[i] = vals[i];
  return SPIDER_OK;
}

int spider_diagnostics(spider_ctx* c, uint64_t batch_seed, float eps, double* grad_norms_out, double* ratio_out) {
  if (!c || !(eps > 0.f)) return SPIDER_E_INVAL;
  const size_t M = c->v.M;
  float4* gmb = nullptr;
  double* norms = nullptr;
  double* part = nullptr;
  const int grid = std::min(kMaxGrid, 4 * c->num_sms);
  cudaError_t e = cudaMallocAsync(&gmb, M * sizeof(float4), c->stream);
  if (e == cudaSuccess) e = cudaMallocAsync(&norms, M * sizeof(double), c->stream);
  if (e == cudaSuccess) e = cudaMallocAsync(&part, grid * sizeof(double), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "diagnostics buffers");
  int rc = evaluate(c, batch_seed, 0, 0.f);                 // minibatch gradient
  if (!rc) {
    e = cudaMemcpyAsync(gmb, c->v.grad, M * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) rc = cuda_fail(c, e, "copy");
  }
  if (!rc) rc = evaluate(c, 0, 0, 0.f);                      // full-batch gradient
  std::vector<double> hn(grad_norms_out ? M : 0), hp(grid);
  if (!rc) {
    e = launch_diag(c->v, gmb, c->v.grad, norms, part, grid, c->stream);
    if (e == cudaSuccess && grad_norms_out)
      e = cudaMemcpyAsync(hn.data(), norms, M * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), part, grid * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) rc = cuda_fail(c, e, "diagnostics");
  }
  cudaFreeAsync(gmb, c->stream);
  cudaFreeAsync(norms, c->stream);
  cudaFreeAsync(part, c->stream);
  cudaStreamSynchronize(c->stream);
  if (rc) return rc;
  rc = check_device_error(c);
  if (rc) return rc;
  double ss = 0.0;
  for (double x : hp) ss += x;
  if (ratio_out) *ratio_out = (double)eps * eps * (ss / (4.0 * (double)M)) / (2.0 * (double)eps);
  if (grad_norms_out)
    for (size_t m = 0; m < M; ++m) grad_norms_out[c->ev_old[m]] = hn[m];
  return SPIDER_OK;
}

const char* spider_last_error(const spider_ctx* c) { return c ? c->err.c_str() : g_static_err; }

void spider_destroy(spider_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : c->wev)
    if (e) cudaEventDestroy(e);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaStreamDestroy(c->side);
  }
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->join) cudaEventDestroy(c->join);
  destroy_branches(c->ubr);
  free_all(c->allocs);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

int spider_net_upload(const spider_net* net, int32_t precision, spider_netdev** out) {
  if (!out) return SPIDER_E_INVAL;
  *out = nullptr;
  std::string msg;
  int rc = check_net(net, precision, &msg);
  if (rc) {
    static thread_local std::string last;
    last = msg;
    g_static_err = last.c_str();
    return rc;
  }
  spider_netdev* nd = new spider_netdev();
  cudaError_t e = upload_net(net, precision, &nd->net, nd->allocs, 0);
  int dev = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nd->num_sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t scr = e == cudaSuccess ? tt_scratch_floats(nd->net, nd->num_sms) : 0;
  if (e == cudaSuccess && scr) e = dalloc(nd->allocs, &nd->scratch, scr);
  if (e == cudaSuccess) e = dalloc(nd->allocs, &nd->net.err, 1);
  if (e == cudaSuccess) e = cudaMemset(nd->net.err, 0, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    g_static_err = cudaGetErrorString(e);
    free_all(nd->allocs);
    delete nd;
    return e == cudaErrorMemoryAllocation ? SPIDER_E_OOM : SPIDER_E_CUDA;
  }
  *out = nd;
  return SPIDER_OK;
}

void spider_net_free(spider_netdev* nd) {
  if (!nd) return;
  cudaDeviceSynchronize();
  free_all(nd->allocs);
  delete nd;
}

int spider_tt_pairs(const spider_netdev* nd, int64_t P, const float* src, const float* rcv, float* T_hi,
                    float* T_lo, float* J, void* stream) {
  if (!nd || P < 0 || (P > 0 && (!src || !rcv || !T_hi))) return SPIDER_E_INVAL;
  if (P == 0) return SPIDER_OK;
  if (P > (int64_t)INT32_MAX) return SPIDER_E_INVAL;
  cudaStream_t st = (cudaStream_t)stream;
  // T is produced as (hi, lo) pairs; split into the caller's arrays afterwards
  float2* T2 = nullptr;
  cudaError_t e = cudaMallocAsync(&T2, (size_t)P * sizeof(float2), st);
  if (e != cudaSuccess) { g_static_err = cudaGetErrorString(e); return SPIDER_E_OOM; }
  PairSource ps{};
  ps.src = reinterpret_cast<const float4*>(src);
  ps.rcv = reinterpret_cast<const float4*>(rcv);
  ps.n_host = P;
  TTOut o{T2, reinterpret_cast<float4*>(J)};
  e = launch_tt(nd->net, ps, o, nd->num_sms, nd->scratch, st, 2);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(T_hi, sizeof(float), T2, sizeof(float2), sizeof(float), (size_t)P,
                          cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && T_lo)
    e = cudaMemcpy2DAsync(T_lo, sizeof(float), reinterpret_cast<float*>(T2) + 1, sizeof(float2), sizeof(float),
                          (size_t)P, cudaMemcpyDeviceToDevice, st);
  cudaError_t e2 = cudaFreeAsync(T2, st);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    g_static_err = cudaGetErrorString(e);
    return SPIDER_E_CUDA;
  }
  return SPIDER_OK;
}

int spider_philox_words(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int64_t n,
                        uint32_t* out) {
  if (n < 0 || (n > 0 && !out) || n > (int64_t(1) << 28)) return SPIDER_E_INVAL;
  if (n == 0) return SPIDER_OK;
  uint32_t* d = nullptr;
  cudaError_t e = cudaMalloc(&d, (size_t)n * 16);
  if (e != cudaSuccess) { g_static_err = cudaGetErrorString(e); return SPIDER_E_OOM; }
  e = launch_philox_words(seed, c0, c1, c2, c3, n, d, 0);
  if (e == cudaSuccess) e = cudaMemcpy(out, d, (size_t)n * 16, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) {
    g_static_err = cudaGetErrorString(e);
    return SPIDER_E_CUDA;
  }
  return SPIDER_OK;
}

}  // extern "C"
