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
