// Test-only harness: runs the library's host preparation (prep.cpp) without a
// GPU so that its orderings and index tables can be checked on the CPU.
#include <cstring>
#include <string>

#include "prep.h"

static spider::Prep g_prep;
static std::string g_err;

extern "C" int prep_run(const spider_catalog* cat, const spider_stations* sta, const spider_config* cfg,
                        int64_t* sizes) {
  int rc = spider::prepare(cat, sta, cfg, &g_prep, &g_err, 2);
  if (rc) return rc;
  const spider::Prep& P = g_prep;
  int64_t s[8] = {P.M, P.N, P.S, P.B, P.NB, P.P, P.Q, P.L_max};
  std::memcpy(sizes, s, sizeof(s));
  return 0;
}

extern "C" const char* prep_error() { return g_err.c_str(); }

template <typename T>
static void cp(const std::vector<T>& v, void* out) {
  std::memcpy(out, v.data(), v.size() * sizeof(T));
}

extern "C" int prep_get(const char* name, void* out) {
  const spider::Prep& P = g_prep;
  std::string n(name);
  if (n == "ev_old") cp(P.ev_old, out);
  else if (n == "ord") cp(P.ord, out);
  else if (n == "pair_off") cp(P.pair_off, out);
  else if (n == "pair_st") cp(P.pair_st, out);
  else if (n == "pair_ev") cp(P.pair_ev, out);
  else if (n == "obs_l") cp(P.obs_l, out);
  else if (n == "obs_dt") cp(P.obs_dt, out);
  else if (n == "obs_sw") cp(P.obs_sw, out);
  else if (n == "blk_node_off") cp(P.blk_node_off, out);
  else if (n == "node_pair") cp(P.node_pair, out);
  else if (n == "node_he") cp(P.node_he, out);
  else if (n == "blk_he") cp(P.blk_he, out);
  else if (n == "inc_off") cp(P.inc_off, out);
  else if (n == "inc_q") cp(P.inc_q, out);
  else if (n == "inc_b") cp(P.inc_b, out);
  else return -1;
  return 0;
}

// ---- block-local pieces and their inverses (pieces.cpp) ----
#include "pieces.h"

static spider::Pieces g_pieces;
static std::vector<float> g_inv;

extern "C" int pieces_run(int max_n, double lam, int64_t* sizes) {
  if (!spider::build_pieces(g_prep, max_n, &g_pieces, 2)) return 1;
  const spider::Pieces& T = g_pieces;
  g_inv.assign((size_t)T.piece_inv_off[T.G], 0.f);
  spider::piece_inverses(g_prep, T, lam, 0, g_prep.NB, g_inv.data(), 2);
  int64_t s[3] = {T.G, T.max_n, T.piece_inv_off[T.G]};
  std::memcpy(sizes, s, sizeof(s));
  return 0;
}

extern "C" int pieces_get(const char* name, void* out) {
  const spider::Pieces& T = g_pieces;
  std::string n(name);
  if (n == "blk_piece_off") cp(T.blk_piece_off, out);
  else if (n == "node_piece") cp(T.node_piece, out);
  else if (n == "node_ppos") cp(T.node_ppos, out);
  else if (n == "piece_node_off") cp(T.piece_node_off, out);
  else if (n == "piece_nodes") cp(T.piece_nodes, out);
  else if (n == "piece_inv_off") cp(T.piece_inv_off, out);
  else if (n == "inv") cp(g_inv, out);
  else if (n == "mem_rp") cp(T.mem_rp, out);
  else if (n == "edge_pos") cp(T.edge_pos, out);
  else if (n == "edge_sw") cp(T.edge_sw, out);
  else return -1;
  return 0;
}
