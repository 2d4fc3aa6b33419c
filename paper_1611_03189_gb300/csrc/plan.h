// Symbolic planner: block structure and elimination waves of the hierarchical
// factorization, from the sparsity pattern alone.
//
// Sec. 3 (Algorithm 1): 2^L leaf red nodes are merged pairwise into super nodes,
// level by level.  Sec. 3.1: two nodes are neighbours when their leaf sets are
// joined by an edge of the ORIGINAL graph; a block between non-neighbours is a
// well-separated interaction.  Eliminating a super node s (Sec. 3.2) creates
// blocks between every pair of its neighbours N(s) (Schur complement) and, if s
// has a well-separated block, a red node r with blocks to N(s) and W(s)
// (extension, eq. extended).  A super node without well-separated blocks is
// eliminated exactly and leaves no red node.  A red node keeps the leaf set of
// its super node.
//
// Elimination order: canonical waves -- within a level, repeatedly take, in
// ascending super-node index, a maximal set of super nodes no two of which
// share a block, and eliminate it.  Members of a wave touch disjoint data apart
// from additive updates of shared neighbour blocks.
#pragma once

#include <stdint.h>

#include "../../include/hs.h"

#include <vector>

namespace hs {

struct PlanSuper {
  int wave = -1;            // wave index, -1 if the super node does not exist
  std::vector<int> N;       // neighbour keys, ascending
  std::vector<int> W;       // well-separated keys, ascending
};

struct PlanLevel {
  int level = 0;                       // L .. 2
  int nsup = 0;                        // 2^(level-1)
  std::vector<char> exists;            // super node exists
  std::vector<std::vector<int>> waves; // super indices per wave
  std::vector<PlanSuper> sup;          // by super index
  std::vector<char> red_made;          // by super index: a red node was created
};

struct Plan {
  int64_t n = 0, nnz = 0;
  int L = 0, nleaf = 0;
  std::vector<int32_t> perm, iperm, leaf_ptr;
  // permuted CSR pattern (cluster order) and, per permuted entry, the index of
  // the original entry
  std::vector<int32_t> prow, pcol, psrc;
  std::vector<PlanLevel> levels;       // levels[0] is level L
  std::vector<char> red1;              // red nodes of level 1 (root children) that exist
  int total_waves = 0;
};

// nbr_dist: 0 or 1, neighbours are joined by an edge of the original graph
// (Sec. 3.1); 2, also the nodes of a level that share a neighbour.
// order_mode: HS_ORDER_WAVES (canonical waves) or HS_ORDER_SEQUENTIAL (one
// super node per step, in ascending index).
// Throws hs::fail(HS_ERR_INVALID, ...) on bad input.
void build_plan(int64_t n, const int32_t *rowptr, const int32_t *col, const int32_t *perm,
                const int32_t *leaf_ptr, int32_t nleaf, Plan &out, int nbr_dist = 1,
                int order_mode = HS_ORDER_WAVES);

}  // namespace hs
