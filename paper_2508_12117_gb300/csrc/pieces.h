// Block-local components ("pieces") of the whitening system and their dense
// inverses, built once at spider_create (host).
//
// Within one minibatch block the latent nodes (its (event, station) pairs) are
// linked by the block's observations; a connected set of them is a piece.  The
// matrix of a piece, K = lambda I + B^T B over the piece's edges (B^T B has
// w_e on both ends' diagonals and -w_e between them, w_e = sw_e^2 with the
// stored FP32 sqrt-weights), depends on nothing that changes during sampling
// (the edge weights are frozen), so its inverse is computed once, in FP64, and
// kept rounded to FP32.  A piece none of whose nodes occurs in another
// selected block is a whole connected component of the minibatch system and
// is solved with that inverse alone.
#pragma once
#include <cstdint>
#include <vector>

#include "prep.h"

namespace spider {

struct Pieces {
  int32_t max_n = 0;                    // nodes of the largest piece
  int64_t G = 0;                        // pieces in total
  std::vector<int32_t> blk_piece_off;   // NB + 1: pieces of block b are [off[b], off[b + 1])
  std::vector<uint16_t> node_piece;     // Q: piece of local node q, numbered within its block
  std::vector<uint16_t> node_ppos;      // Q: position of local node q inside its piece
  std::vector<int32_t> piece_node_off;  // G + 1: members of piece g, in the Q numbering
  std::vector<uint16_t> piece_nodes;    // Q: block-local index of each member, grouped by piece,
                                        //    ascending within a piece
  std::vector<int64_t> piece_inv_off;   // G + 1: inverse of piece g (n x n floats)
  // the edges of every member, grouped like piece_nodes: member m (in the
  // piece_nodes order) has entries [mem_rp[m], mem_rp[m + 1]), each the position
  // of the other end inside the same piece and the edge's sqrt-weight, in the
  // block's observation order
  std::vector<int32_t> mem_rp;          // Q + 1
  std::vector<uint16_t> edge_pos;       // 2 N
  std::vector<float> edge_sw;           // 2 N
};

// Finds the pieces of every block (union-find over the block's observations);
// pieces are numbered by their smallest local node.  Returns false when a
// piece has more than max_n nodes (the tables are then incomplete).
bool build_pieces(const Prep& P, int max_n, Pieces* out, int threads);

// (lambda I + B^T B)^-1 of every piece of blocks [b0, b1), computed in FP64 by
// Cholesky and rounded to FP32, stored whole (n x n, symmetric, so row j is
// column j: a warp reading row j of a matrix-vector product reads consecutive
// words).  out receives the floats from piece_inv_off[blk_piece_off[b0]] on.
void piece_inverses(const Prep& P, const Pieces& T, double lam, int64_t b0, int64_t b1, float* out,
                    int threads);

}  // namespace spider
