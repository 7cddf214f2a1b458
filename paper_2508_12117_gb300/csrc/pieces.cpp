// Block-local components of the whitening system and their inverses (host).
#include "pieces.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <functional>
#include <thread>

namespace spider {

namespace {

void for_blocks(int64_t n, int threads, const std::function<void(int64_t, int64_t)>& f) {
  if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());
  threads = (int)std::min<int64_t>(threads, std::max<int64_t>(1, n / 16));
  if (threads <= 1) {
    f(0, n);
    return;
  }
  // dynamic chunks: piece sizes (and so the work per block) vary
  std::atomic<int64_t> next(0);
  const int64_t chunk = 16;
  std::vector<std::thread> pool;
  for (int t = 0; t < threads; ++t)
    pool.emplace_back([&] {
      for (;;) {
        const int64_t a = next.fetch_add(chunk);
        if (a >= n) break;
        f(a, std::min(n, a + chunk));
      }
    });
  for (auto& th : pool) th.join();
}

int find_root(std::vector<int32_t>& par, int32_t x) {
  while (par[x] != x) {
    par[x] = par[par[x]];
    x = par[x];
  }
  return x;
}

}  // namespace

bool build_pieces(const Prep& P, int max_n, Pieces* out, int threads) {
  Pieces& T = *out;
  T = Pieces();
  const int64_t NB = P.NB, Q = P.Q;
  T.node_piece.assign(Q, 0);
  T.node_ppos.assign(Q, 0);
  T.piece_nodes.assign(Q, 0);
  std::vector<int32_t> npieces(NB, 0);
  std::vector<int32_t> bmax(NB, 0);
  // pass 1: per block, the piece of every local node and its position
  for_blocks(NB, threads, [&](int64_t a, int64_t b) {
    std::vector<int32_t> par, id, cnt;
    for (int64_t blk = a; blk < b; ++blk) {
      const int32_t q0 = P.blk_node_off[blk];
      const int L = P.blk_node_off[blk + 1] - q0;
      const int64_t e0 = P.blk_e0[blk], ne = P.blk_e0[blk + 1] - e0;
      par.resize(L);
      for (int l = 0; l < L; ++l) par[l] = l;
      for (int64_t e = 0; e < ne; ++e) {
        const uint32_t lij = P.obs_l[e0 + e];
        int x = find_root(par, (int32_t)(lij & 0xFFFF)), y = find_root(par, (int32_t)(lij >> 16));
        if (x != y) par[std::max(x, y)] = std::min(x, y);
      }
      // pieces numbered by their smallest local node; members ascending
      id.assign(L, -1);
      cnt.clear();
      for (int l = 0; l < L; ++l) {
        const int r = find_root(par, l);
        if (id[r] < 0) {
          id[r] = (int32_t)cnt.size();
          cnt.push_back(0);
        }
        T.node_piece[q0 + l] = (uint16_t)id[r];
        T.node_ppos[q0 + l] = (uint16_t)std::min<int32_t>(cnt[id[r]], 0xFFFF);
        cnt[id[r]]++;
      }
      npieces[blk] = (int32_t)cnt.size();
      int mx = 0;
      for (int32_t c : cnt) mx = std::max(mx, c);
      bmax[blk] = mx;
    }
  });
  T.blk_piece_off.assign(NB + 1, 0);
  for (int64_t blk = 0; blk < NB; ++blk) {
    T.blk_piece_off[blk + 1] = T.blk_piece_off[blk] + npieces[blk];
    T.max_n = std::max(T.max_n, bmax[blk]);
  }
  T.G = T.blk_piece_off[NB];
  if (T.max_n > max_n) return false;
  // pass 2: member lists and the offsets of the inverses
  T.piece_node_off.assign(T.G + 1, 0);
  std::vector<int32_t> psize(T.G, 0);
  for (int64_t blk = 0; blk < NB; ++blk)
    for (int32_t q = P.blk_node_off[blk]; q < P.blk_node_off[blk + 1]; ++q)
      psize[T.blk_piece_off[blk] + T.node_piece[q]]++;
  T.piece_inv_off.assign(T.G + 1, 0);
  for (int64_t g = 0; g < T.G; ++g) {
    T.piece_node_off[g + 1] = T.piece_node_off[g] + psize[g];
    const int64_t n = psize[g];
    T.piece_inv_off[g + 1] = T.piece_inv_off[g] + n * n;
  }
  for_blocks(NB, threads, [&](int64_t a, int64_t b) {
    for (int64_t blk = a; blk < b; ++blk) {
      const int32_t q0 = P.blk_node_off[blk];
      for (int32_t q = q0; q < P.blk_node_off[blk + 1]; ++q) {
        const int64_t g = T.blk_piece_off[blk] + T.node_piece[q];
        T.piece_nodes[T.piece_node_off[g] + T.node_ppos[q]] = (uint16_t)(q - q0);
      }
    }
  });
  // member edge lists: the degree of member m is the half-edge count of its
  // local node; entries follow the node's half-edges (observation order)
  T.mem_rp.assign(Q + 1, 0);
  for (int64_t blk = 0; blk < NB; ++blk) {
    const int32_t q0 = P.blk_node_off[blk];
    const int L = P.blk_node_off[blk + 1] - q0;
    const int ne = P.blk_e0[blk + 1] - P.blk_e0[blk];
    for (int l = 0; l < L; ++l) {
      const int32_t q = q0 + l;
      const int h1 = (l + 1 < L) ? (int)P.node_he[q + 1] : 2 * ne;
      const int64_t g = T.blk_piece_off[blk] + T.node_piece[q];
      T.mem_rp[T.piece_node_off[g] + T.node_ppos[q] + 1] = h1 - (int)P.node_he[q];
    }
  }
  for (int64_t m = 0; m < Q; ++m) T.mem_rp[m + 1] += T.mem_rp[m];
  T.edge_pos.assign((size_t)T.mem_rp[Q], 0);
  T.edge_sw.assign((size_t)T.mem_rp[Q], 0.f);
  for_blocks(NB, threads, [&](int64_t a, int64_t b) {
    for (int64_t blk = a; blk < b; ++blk) {
      const int32_t q0 = P.blk_node_off[blk];
      const int L = P.blk_node_off[blk + 1] - q0;
      const int64_t e0 = P.blk_e0[blk];
      const int ne = P.blk_e0[blk + 1] - (int)e0;
      const uint16_t* he = P.blk_he.data() + 2 * e0;
      for (int l = 0; l < L; ++l) {
        const int32_t q = q0 + l;
        const int h0 = P.node_he[q], h1 = (l + 1 < L) ? (int)P.node_he[q + 1] : 2 * ne;
        const int64_t g = T.blk_piece_off[blk] + T.node_piece[q];
        int32_t t = T.mem_rp[T.piece_node_off[g] + T.node_ppos[q]];
        for (int h = h0; h < h1; ++h, ++t) {
          const int code = he[h];
          const int e = code >> 1;
          const uint32_t lij = P.obs_l[e0 + e];
          const int other = (code & 1) ? (int)(lij & 0xFFFF) : (int)(lij >> 16);
          T.edge_pos[t] = T.node_ppos[q0 + other];
          T.edge_sw[t] = P.obs_sw[e0 + e];
        }
      }
    }
  });
  return true;
}

void piece_inverses(const Prep& P, const Pieces& T, double lam, int64_t b0, int64_t b1, float* out,
                    int threads) {
  const int64_t base = T.piece_inv_off[T.blk_piece_off[b0]];
  for_blocks(b1 - b0, threads, [&](int64_t a, int64_t b) {
    std::vector<double> K;
    std::vector<std::vector<double>> Ks;
    for (int64_t blk = b0 + a; blk < b0 + b; ++blk) {
      const int32_t q0 = P.blk_node_off[blk];
      const int64_t g0 = T.blk_piece_off[blk], np = T.blk_piece_off[blk + 1] - g0;
      Ks.resize(std::max<size_t>(Ks.size(), (size_t)np));
      for (int64_t c = 0; c < np; ++c) {
        const int n = T.piece_node_off[g0 + c + 1] - T.piece_node_off[g0 + c];
        Ks[c].assign((size_t)n * n, 0.0);
        for (int i = 0; i < n; ++i) Ks[c][(size_t)i * n + i] = lam;
      }
      // lambda I + B^T B: every observation adds w to both ends and -w between them
      const int64_t e0 = P.blk_e0[blk], ne = P.blk_e0[blk + 1] - e0;
      for (int64_t e = 0; e < ne; ++e) {
        const uint32_t lij = P.obs_l[e0 + e];
        const int32_t qi = q0 + (int32_t)(lij & 0xFFFF), qj = q0 + (int32_t)(lij >> 16);
        const int c = T.node_piece[qi];
        const int n = T.piece_node_off[g0 + c + 1] - T.piece_node_off[g0 + c];
        const int i = T.node_ppos[qi], j = T.node_ppos[qj];
        const double sw = (double)P.obs_sw[e0 + e];
        const double w = sw * sw;
        double* A = Ks[c].data();
        A[(size_t)i * n + i] += w;
        A[(size_t)j * n + j] += w;
        A[(size_t)i * n + j] -= w;
        A[(size_t)j * n + i] -= w;
      }
      for (int64_t c = 0; c < np; ++c) {
        const int n = T.piece_node_off[g0 + c + 1] - T.piece_node_off[g0 + c];
        double* A = Ks[c].data();
        // Cholesky A = L L^T (lower triangle in place)
        for (int j = 0; j < n; ++j) {
          double d = A[(size_t)j * n + j];
          for (int k = 0; k < j; ++k) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
          const double ljj = std::sqrt(d);
          A[(size_t)j * n + j] = ljj;
          for (int i = j + 1; i < n; ++i) {
            double s = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) s -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
            A[(size_t)i * n + j] = s / ljj;
          }
        }
        // column j of the inverse: solve L y = e_j, then L^T x = y (rows i >= j, mirrored)
        K.assign((size_t)n, 0.0);
        float* dst = out + (T.piece_inv_off[g0 + c] - base);
        for (int j = 0; j < n; ++j) {
          for (int i = 0; i < n; ++i) {
            double s = (i == j) ? 1.0 : 0.0;
            for (int k = j; k < i; ++k) s -= A[(size_t)i * n + k] * K[k];
            K[i] = i < j ? 0.0 : s / A[(size_t)i * n + i];
          }
          for (int i = n - 1; i >= j; --i) {
            double s = K[i];
            for (int k = i + 1; k < n; ++k) s -= A[(size_t)k * n + i] * K[k];
            K[i] = s / A[(size_t)i * n + i];
          }
          for (int i = j; i < n; ++i) {
            dst[(int64_t)j * n + i] = (float)K[i];    // symmetric: row j = column j
            dst[(int64_t)i * n + j] = (float)K[i];
          }
        }
      }
    }
  });
}

}  // namespace spider
