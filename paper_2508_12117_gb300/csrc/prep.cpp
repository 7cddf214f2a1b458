// Host-side preparation of a catalog (spider_create): validation, Morton
// renumbering, canonical observation order, (event, station) pair table,
// minibatch blocks with their local half-edge lists, pair -> block incidence,
// edge weights (Eq. correlation_decay) and reduced dd times.
#include "prep.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>
#include <thread>

namespace spider {

namespace {

void parallel_for(int64_t n, int threads, const std::function<void(int64_t, int64_t)>& f) {
  if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());
  if (n < 4096 || threads == 1) {
    f(0, n);
    return;
  }
  threads = (int)std::min<int64_t>(threads, (n + 4095) / 4096);
  std::vector<std::thread> pool;
  int64_t chunk = (n + threads - 1) / threads;
  for (int t = 0; t < threads; ++t) {
    int64_t a = t * chunk, b = std::min(n, a + chunk);
    if (a >= b) break;
    pool.emplace_back([=, &f] { f(a, b); });
  }
  for (auto& th : pool) th.join();
}

bool finite(double x) { return std::isfinite(x); }

}  // namespace

// Morton key: per-axis minimum lo_c, ext = largest per-axis extent,
// q_c = floor((c - lo_c) * (2097151 / ext)) clamped to [0, 2097151], bit b of
// (q_x, q_y, q_z) at key bits (3b, 3b+1, 3b+2); ties keep the input order.
std::vector<int32_t> morton_order(const double* xyzt, int64_t M) {
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t m = 0; m < M; ++m)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], xyzt[4 * m + a]);
      hi[a] = std::max(hi[a], xyzt[4 * m + a]);
    }
  double ext = 0.0;
  for (int a = 0; a < 3; ++a) ext = std::max(ext, hi[a] - lo[a]);
  double scale = ext > 0.0 ? 2097151.0 / ext : 0.0;
  std::vector<uint64_t> key(M);
  for (int64_t m = 0; m < M; ++m) {
    uint64_t k = 0;
    for (int a = 0; a < 3; ++a) {
      volatile double d = xyzt[4 * m + a] - lo[a];   // keep (c - lo) * scale unfused
      double f = std::floor(d * scale);
      int64_t q = f < 0 ? 0 : (f > 2097151.0 ? 2097151 : (int64_t)f);
      for (int b = 0; b < 21; ++b) k |= (uint64_t)((q >> b) & 1) << (3 * b + a);
    }
    key[m] = k;
  }
  std::vector<int32_t> perm(M);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
  return perm;
}

int prepare(const spider_catalog* cat, const spider_stations* sta, const spider_config* cfg,
            Prep* out, std::string* err, int threads, const std::vector<int64_t>* ev_splits,
            const std::vector<int64_t>* obs_splits) {
  auto fail = [&](const std::string& m) {
    *err = m;
    return SPIDER_E_INVAL;
  };
  if (!cat || !sta || !cfg) return fail("null catalog, stations or config");
  const int64_t M = cat->M, N = cat->N, S = sta->S;
  if (M < 2 || M > (int64_t)INT32_MAX) return fail("M must be in [2, 2^31)");
  if (N < 1 || N >= (int64_t(1) << 30)) return fail("N must be in [1, 2^30)");
  if (S < 1) return fail("S must be >= 1");
  if (!cat->xyzt0 || !cat->i || !cat->j || !cat->k || !cat->dt || !sta->xyz)
    return fail("null catalog or station array");
  const int64_t B = cfg->block_obs;
  if (B < 1 || B > 4096) return fail("block_obs must be in [1, 4096]");
  if (!(cfg->sigma > 0.0) || !(cfg->kappa >= 0.0) || !(cfg->ell > 0.0) || !(cfg->p > 0.0) ||
      !(cfg->eps_w > 0.0))
    return fail("need sigma > 0, kappa >= 0, ell > 0, p > 0, eps_w > 0");
  for (int a = 0; a < 4; ++a)
    if (!(cfg->sig_e[a] > 0.0) || !(cfg->sig_c[a] > 0.0)) return fail("prior sigmas must be > 0");
  for (int64_t m = 0; m < 4 * M; ++m)
    if (!finite(cat->xyzt0[m])) return fail("non-finite theta_0");
  for (int64_t s = 0; s < 3 * S; ++s)
    if (!finite(sta->xyz[s])) return fail("non-finite station position");
  std::vector<int64_t> evs = ev_splits ? *ev_splits : std::vector<int64_t>{0, M};
  std::vector<int64_t> obss = obs_splits ? *obs_splits : std::vector<int64_t>{0, N};
  const int n_sub = (int)evs.size() - 1;
  if (n_sub < 1 || (int)obss.size() != n_sub + 1 || evs.front() != 0 || evs.back() != M ||
      obss.front() != 0 || obss.back() != N)
    return fail("inconsistent sub-problem splits");
  for (int s = 0; s < n_sub; ++s)
    if (evs[s + 1] - evs[s] < 2 || obss[s + 1] < obss[s]) return fail("every sub-problem needs >= 2 events");
  std::vector<int32_t> obs_sub_of(n_sub > 1 ? N : 0);
  for (int s = 0; s < n_sub && n_sub > 1; ++s)
    for (int64_t n = obss[s]; n < obss[s + 1]; ++n) obs_sub_of[n] = s;
  {
    std::atomic<int64_t> bad(-1);
    parallel_for(N, threads, [&](int64_t a, int64_t b) {
      for (int64_t n = a; n < b; ++n) {
        int32_t i = cat->i[n], j = cat->j[n], k = cat->k[n];
        bool ok = i >= 0 && i < M && j >= 0 && j < M && i != j && k >= 0 && k < S &&
                  finite(cat->dt[n]) && (!cat->w || (finite(cat->w[n]) && cat->w[n] > 0.f));
        if (ok && n_sub > 1) {
          const int s = obs_sub_of[n];
          ok = i >= evs[s] && i < evs[s + 1] && j >= evs[s] && j < evs[s + 1];
        }
        if (!ok) {
          int64_t e = -1;
          bad.compare_exchange_strong(e, n);
          return;
        }
      }
    });
    if (bad.load() >= 0)
      return fail("observation " + std::to_string(bad.load()) +
                  ": index out of range, i == j, non-finite dt or non-positive weight");
  }

  Prep& P = *out;
  P = Prep();
  P.M = M; P.N = N; P.S = S; P.B = B;
  P.n_sub = n_sub;
  P.sub_ev_off = evs;
  P.sub_obs_off = obss;

  // ---- event renumbering (Morton order inside each sub-problem) ----
  P.ev_old.resize(M);
  P.ev_sub.resize(M);
  P.ev_local.resize(M);
  for (int s = 0; s < n_sub; ++s) {
    const int64_t e0 = evs[s], ne = evs[s + 1] - evs[s];
    std::vector<int32_t> o;
    if (cfg->reorder) {
      o = morton_order(cat->xyzt0 + 4 * e0, ne);
    } else {
      o.resize(ne);
      std::iota(o.begin(), o.end(), 0);
    }
    for (int64_t m = 0; m < ne; ++m) {
      P.ev_old[e0 + m] = (int32_t)(e0 + o[m]);
      P.ev_sub[e0 + m] = s;
      P.ev_local[e0 + m] = o[m];
    }
  }
  std::vector<int32_t> rank(M);
  for (int64_t m = 0; m < M; ++m) rank[P.ev_old[m]] = (int32_t)m;
  P.th0.resize(4 * M);
  for (int64_t m = 0; m < M; ++m)
    for (int a = 0; a < 4; ++a) P.th0[4 * m + a] = cat->xyzt0[4 * P.ev_old[m] + a];

  // ---- canonical order: (rank i, rank j, k), stable ----
  P.ord.resize(N);
  {
    std::atomic<bool> sorted(true);
    parallel_for(N - 1, threads, [&](int64_t a, int64_t b) {
      for (int64_t n = a; n < b && sorted.load(std::memory_order_relaxed); ++n) {
        int32_t a0 = rank[cat->i[n]], a1 = rank[cat->i[n + 1]];
        if (a0 != a1) {
          if (a0 > a1) sorted = false;
          continue;
        }
        int32_t b0 = rank[cat->j[n]], b1 = rank[cat->j[n + 1]];
        if (b0 != b1) {
          if (b0 > b1) sorted = false;
          continue;
        }
        if (cat->k[n] > cat->k[n + 1]) sorted = false;
      }
    });
    if (sorted) {
      std::iota(P.ord.begin(), P.ord.end(), 0);
    } else {
      std::vector<int64_t> cnt(M + 1, 0);
      for (int64_t n = 0; n < N; ++n) cnt[rank[cat->i[n]] + 1]++;
      for (int64_t m = 0; m < M; ++m) cnt[m + 1] += cnt[m];
      std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
      for (int64_t n = 0; n < N; ++n) P.ord[pos[rank[cat->i[n]]]++] = (int32_t)n;
      parallel_for(M, threads, [&](int64_t a, int64_t b) {
        for (int64_t m = a; m < b; ++m)
          std::stable_sort(P.ord.begin() + cnt[m], P.ord.begin() + cnt[m + 1],
                           [&](int32_t x, int32_t y) {
                             int32_t bx = rank[cat->j[x]], by = rank[cat->j[y]];
                             if (bx != by) return bx < by;
                             return cat->k[x] < cat->k[y];
                           });
      });
    }
  }

  // ---- pair table: stations met by each event (as i or j end) ----
  std::vector<int32_t> ia(N), ja(N), ka(N);
  parallel_for(N, threads, [&](int64_t a, int64_t b) {
    for (int64_t n = a; n < b; ++n) {
      int32_t o = P.ord[n];
      ia[n] = rank[cat->i[o]];
      ja[n] = rank[cat->j[o]];
      ka[n] = cat->k[o];
    }
  });
  {
    std::vector<int64_t> cnt(M + 1, 0);
    for (int64_t n = 0; n < N; ++n) {
      cnt[ia[n] + 1]++;
      cnt[ja[n] + 1]++;
    }
    for (int64_t m = 0; m < M; ++m) cnt[m + 1] += cnt[m];
    std::vector<int32_t> st(2 * N);
    std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
    for (int64_t n = 0; n < N; ++n) {
      st[pos[ia[n]]++] = ka[n];
      st[pos[ja[n]]++] = ka[n];
    }
    std::vector<int32_t> ucnt(M, 0);
    parallel_for(M, threads, [&](int64_t a, int64_t b) {
      for (int64_t m = a; m < b; ++m) {
        auto s0 = st.begin() + cnt[m], s1 = st.begin() + cnt[m + 1];
        std::sort(s0, s1);
        ucnt[m] = (int32_t)(std::unique(s0, s1) - s0);
      }
    });
    P.pair_off.assign(M + 1, 0);
    for (int64_t m = 0; m < M; ++m) P.pair_off[m + 1] = P.pair_off[m] + ucnt[m];
    P.P = P.pair_off[M];
    P.pair_st.resize(P.P);
    P.pair_ev.resize(P.P);
    parallel_for(M, threads, [&](int64_t a, int64_t b) {
      for (int64_t m = a; m < b; ++m)
        for (int32_t t = 0; t < ucnt[m]; ++t) {
          P.pair_st[P.pair_off[m] + t] = st[cnt[m] + t];
          P.pair_ev[P.pair_off[m] + t] = (int32_t)m;
        }
    });
  }
  auto pair_of = [&](int32_t m, int32_t k) -> int32_t {
    const int32_t* b = P.pair_st.data() + P.pair_off[m];
    const int32_t* e = P.pair_st.data() + P.pair_off[m + 1];
    return (int32_t)(std::lower_bound(b, e, k) - P.pair_st.data());
  };

  // ---- edge weights (Eq. correlation_decay), reduced dd times ----
  P.obs_dt.resize(N);
  P.obs_sw.resize(N);
  {
    std::vector<double> w(N);
    parallel_for(N, threads, [&](int64_t a, int64_t b) {
      for (int64_t n = a; n < b; ++n) {
        const double* xi = &P.th0[4 * ia[n]];
        const double* xj = &P.th0[4 * ja[n]];
        if (cat->w) {
          w[n] = cat->w[P.ord[n]];
        } else {
          double dx = xi[0] - xj[0], dy = xi[1] - xj[1], dz = xi[2] - xj[2];
          double d = std::sqrt(dx * dx + dy * dy + dz * dz);
          w[n] = std::pow(d / cfg->ell, cfg->p) + cfg->eps_w;
        }
        P.obs_dt[n] = (float)(cat->dt[P.ord[n]] - (xi[3] - xj[3]));
      }
    });
    if (!cat->w) {
      std::vector<double> tot(S, 0.0);
      std::vector<int64_t> cnt(S, 0);
      for (int64_t n = 0; n < N; ++n) {
        tot[ka[n]] += w[n];
        cnt[ka[n]]++;
      }
      for (int64_t s = 0; s < S; ++s) tot[s] = cnt[s] ? tot[s] / (double)cnt[s] : 1.0;
      parallel_for(N, threads, [&](int64_t a, int64_t b) {
        for (int64_t n = a; n < b; ++n) w[n] /= tot[ka[n]];
      });
    }
    parallel_for(N, threads, [&](int64_t a, int64_t b) {
      for (int64_t n = a; n < b; ++n) P.obs_sw[n] = (float)std::sqrt(w[n]);
    });
  }

  // ---- blocks: cut per sub-problem, then local nodes, local indices, half-edge lists ----
  P.sub_blk_off.assign(n_sub + 1, 0);
  P.blk_e0.clear();
  P.blk_sub.clear();
  for (int s = 0; s < n_sub; ++s) {
    P.sub_blk_off[s] = (int64_t)P.blk_sub.size();
    for (int64_t e = obss[s]; e < obss[s + 1]; e += B) {
      P.blk_e0.push_back((int32_t)e);
      P.blk_sub.push_back(s);
    }
  }
  P.sub_blk_off[n_sub] = (int64_t)P.blk_sub.size();
  P.blk_e0.push_back((int32_t)N);
  P.NB = (int64_t)P.blk_sub.size();
  const int64_t NB = P.NB;
  std::vector<std::vector<int32_t>> bnodes(NB);
  std::vector<std::vector<uint16_t>> bhe_beg(NB);
  P.obs_l.resize(N);
  P.blk_he.resize(2 * N);
  parallel_for(NB, threads, [&](int64_t a, int64_t b) {
    std::vector<int32_t> tmp;
    std::vector<int32_t> pi, pj;
    std::vector<uint16_t> deg, fill;
    for (int64_t blk = a; blk < b; ++blk) {
      int64_t e0 = P.blk_e0[blk], ne = P.blk_e0[blk + 1] - e0;
      pi.resize(ne); pj.resize(ne);
      tmp.clear();
      for (int64_t e = 0; e < ne; ++e) {
        pi[e] = pair_of(ia[e0 + e], ka[e0 + e]);
        pj[e] = pair_of(ja[e0 + e], ka[e0 + e]);
        tmp.push_back(pi[e]);
        tmp.push_back(pj[e]);
      }
      std::sort(tmp.begin(), tmp.end());
      tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
      const int64_t L = (int64_t)tmp.size();
      deg.assign(L + 1, 0);
      for (int64_t e = 0; e < ne; ++e) {
        uint32_t li = (uint32_t)(std::lower_bound(tmp.begin(), tmp.end(), pi[e]) - tmp.begin());
        uint32_t lj = (uint32_t)(std::lower_bound(tmp.begin(), tmp.end(), pj[e]) - tmp.begin());
        P.obs_l[e0 + e] = li | (lj << 16);
        deg[li + 1]++;
        deg[lj + 1]++;
      }
      for (int64_t l = 0; l < L; ++l) deg[l + 1] += deg[l];
      fill.assign(deg.begin(), deg.end() - 1);
      uint16_t* he = P.blk_he.data() + 2 * e0;
      for (int64_t e = 0; e < ne; ++e) {
        uint32_t l = P.obs_l[e0 + e];
        he[fill[l & 0xFFFF]++] = (uint16_t)(2 * e);
        he[fill[l >> 16]++] = (uint16_t)(2 * e + 1);
      }
      bnodes[blk] = tmp;
      bhe_beg[blk].assign(deg.begin(), deg.end() - 1);
    }
  });
  P.blk_node_off.assign(NB + 1, 0);
  for (int64_t blk = 0; blk < NB; ++blk) {
    P.blk_node_off[blk + 1] = P.blk_node_off[blk] + (int32_t)bnodes[blk].size();
    P.L_max = std::max<int32_t>(P.L_max, (int32_t)bnodes[blk].size());
  }
  P.Q = P.blk_node_off[NB];
  P.node_pair.resize(P.Q);
  P.node_he.resize(P.Q);
  parallel_for(NB, threads, [&](int64_t a, int64_t b) {
    for (int64_t blk = a; blk < b; ++blk) {
      std::copy(bnodes[blk].begin(), bnodes[blk].end(), P.node_pair.begin() + P.blk_node_off[blk]);
      std::copy(bhe_beg[blk].begin(), bhe_beg[blk].end(), P.node_he.begin() + P.blk_node_off[blk]);
      std::vector<int32_t>().swap(bnodes[blk]);
      std::vector<uint16_t>().swap(bhe_beg[blk]);
    }
  });

  // ---- pair -> occurrences (block-ascending) ----
  P.inc_off.assign(P.P + 1, 0);
  for (int64_t q = 0; q < P.Q; ++q) P.inc_off[P.node_pair[q] + 1]++;
  for (int64_t p = 0; p < P.P; ++p) P.inc_off[p + 1] += P.inc_off[p];
  P.inc_q.resize(P.Q);
  P.inc_b.resize(P.Q);
  {
    std::vector<int32_t> pos(P.inc_off.begin(), P.inc_off.end() - 1);
    for (int64_t blk = 0; blk < NB; ++blk)
      for (int32_t q = P.blk_node_off[blk]; q < P.blk_node_off[blk + 1]; ++q) {
        int32_t t = pos[P.node_pair[q]]++;
        P.inc_q[t] = q;
        P.inc_b[t] = (int32_t)blk;
      }
  }
  return SPIDER_OK;
}

}  // namespace spider
