// Host-side preparation of a catalog for the device step (spider_create).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "spider.h"

namespace spider {

// Everything the device path needs, laid out on the host before upload.
//
// Numbering: events are renumbered along a Morton curve of theta_0 (when
// cfg->reorder), observations sorted by (i, j, k) in that numbering (stable),
// then cut into blocks of B consecutive observations (the minibatch unit; the
// last block of each sub-problem may be shorter).
//
// A "pair" is an (event, station) combination met by some observation: the
// node of the latent field b of Sec. 3.1 and the unit of travel-time work.
// Inside block b the pairs it touches are its "local nodes" (sorted by pair
// id); the global index of local node l of block b is q = blk_node_off[b] + l.
struct Prep {
  int64_t M = 0, N = 0, S = 0, B = 0, NB = 0, P = 0, Q = 0;
  int32_t L_max = 0;                 // largest local-node count of a block
  std::vector<int32_t> ev_old;       // new event -> caller event
  std::vector<int32_t> ord;          // canonical obs position -> caller obs index
  std::vector<double> th0;           // M x 4, new numbering
  std::vector<int32_t> pair_off;     // M + 1, pairs of event m: [pair_off[m], pair_off[m+1])
  std::vector<int32_t> pair_st;      // P station of each pair (ascending within an event)
  std::vector<int32_t> pair_ev;      // P event of each pair
  std::vector<uint32_t> obs_l;       // N: local node of the i-end | local node of the j-end << 16
  std::vector<float> obs_dt;         // N: dt - (t0_i - t0_j) of theta_0, rounded to FP32
  std::vector<float> obs_sw;         // N: sqrt(w_e)
  std::vector<int32_t> blk_node_off; // NB + 1
  std::vector<int32_t> node_pair;    // Q: pair id of each local node
  std::vector<uint16_t> node_he;     // Q: first half-edge of the node in its block's list
  std::vector<uint16_t> blk_he;      // 2 N: block b's half-edges at [2 b B, 2 b B + 2 n_b):
                                     //   code = 2 e + side, e the obs within the block,
                                     //   side 0: the node is the i-end, 1: the j-end
  std::vector<int32_t> inc_off;      // P + 1: occurrences of a pair in blocks
  std::vector<int32_t> inc_q;        // Q: local node q of each occurrence (block-ascending)
  std::vector<int32_t> inc_b;        // Q: its block
  // independent sub-problems (catalog x chain) sharing one device layout:
  // disjoint event ranges, blocks never straddle two sub-problems
  int32_t n_sub = 1;
  std::vector<int32_t> blk_e0;       // NB + 1: first observation of each block
  std::vector<int32_t> blk_sub;      // NB: sub-problem of each block
  std::vector<int64_t> sub_ev_off;   // n_sub + 1 (events, new numbering = caller ranges)
  std::vector<int64_t> sub_blk_off;  // n_sub + 1
  std::vector<int64_t> sub_obs_off;  // n_sub + 1
  std::vector<int32_t> ev_sub;       // M: sub-problem of each event
  std::vector<int32_t> ev_local;     // M: caller index of the event inside its sub-problem
};

// Validates the inputs (returns SPIDER_E_INVAL with a message on failure) and
// fills `out`.  threads: worker threads for the O(N) passes (0 = hardware).
// With ev_splits / obs_splits (n_sub + 1 prefix offsets each) the catalog is
// the concatenation of n_sub independent sub-problems: the observations of
// sub-problem s lie in [obs_splits[s], obs_splits[s+1]) and reference only
// events in [ev_splits[s], ev_splits[s+1]).
int prepare(const spider_catalog* cat, const spider_stations* sta, const spider_config* cfg,
            Prep* out, std::string* err, int threads = 0,
            const std::vector<int64_t>* ev_splits = nullptr,
            const std::vector<int64_t>* obs_splits = nullptr);

// The Morton order of the library (events new -> old); see prepare().
std::vector<int32_t> morton_order(const double* xyzt, int64_t M);

}  // namespace spider
