// Symbolic planner (see plan.h).
#include "plan.h"

#include <algorithm>
#include <set>
#include <string>

#include "hs_internal.h"

namespace hs {

namespace {

void check(bool ok, const std::string &msg) {
  if (!ok) fail(HS_ERR_INVALID, msg);
}

}  // namespace

void build_plan(int64_t n, const int32_t *rowptr, const int32_t *col, const int32_t *perm,
                const int32_t *leaf_ptr, int32_t nleaf, Plan &P, int nbr_dist, int order_mode) {
  check(order_mode == HS_ORDER_WAVES || order_mode == HS_ORDER_SEQUENTIAL, "order_mode must be 0 or 1");
  check(n > 0, "n must be positive");
  check(nbr_dist >= 0 && nbr_dist <= 2, "nbr_dist must be 0, 1 or 2");
  check(n < (int64_t)1 << 31, "n must fit in int32");
  check(nleaf >= 1 && (nleaf & (nleaf - 1)) == 0, "nleaf must be a power of two");
  int L = 0;
  while ((1 << L) < nleaf) ++L;
  P.n = n;
  P.L = L;
  P.nleaf = nleaf;
  check(rowptr[0] == 0, "rowptr[0] must be 0");
  for (int64_t i = 0; i < n; ++i) check(rowptr[i + 1] >= rowptr[i], "rowptr must be non-decreasing");
  P.nnz = rowptr[n];
  P.perm.assign(perm, perm + n);
  P.iperm.assign(n, -1);
  for (int64_t p = 0; p < n; ++p) {
    check(perm[p] >= 0 && perm[p] < n && P.iperm[perm[p]] < 0, "perm is not a permutation");
    P.iperm[perm[p]] = (int32_t)p;
  }
  P.leaf_ptr.assign(leaf_ptr, leaf_ptr + nleaf + 1);
  check(leaf_ptr[0] == 0 && leaf_ptr[nleaf] == n, "leaf_ptr must run from 0 to n");
  for (int i = 0; i < nleaf; ++i) check(leaf_ptr[i + 1] > leaf_ptr[i], "leaves must be non-empty");
  std::vector<int32_t> leaf_of(n);
  for (int i = 0; i < nleaf; ++i)
    for (int32_t p = leaf_ptr[i]; p < leaf_ptr[i + 1]; ++p) leaf_of[p] = i;

  // permuted CSR (rows in cluster order, columns sorted)
  P.prow.assign(n + 1, 0);
  for (int64_t p = 0; p < n; ++p) {
    const int32_t i = perm[p];
    P.prow[p + 1] = P.prow[p] + (rowptr[i + 1] - rowptr[i]);
  }
  P.pcol.resize(P.nnz);
  P.psrc.resize(P.nnz);
  std::vector<std::pair<int32_t, int32_t>> tmp;
  bool has_diag_all = true;
  for (int64_t p = 0; p < n; ++p) {
    const int32_t i = perm[p];
    tmp.clear();
    bool diag = false;
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      check(col[e] >= 0 && col[e] < n, "column index out of range");
      const int32_t c = P.iperm[col[e]];
      if (c == p) diag = true;
      tmp.emplace_back(c, e);
    }
    has_diag_all = has_diag_all && diag;
    std::sort(tmp.begin(), tmp.end());
    for (size_t q = 0; q < tmp.size(); ++q) {
      check(q == 0 || tmp[q].first != tmp[q - 1].first, "duplicate column in a row");
      P.pcol[P.prow[p] + q] = tmp[q].first;
      P.psrc[P.prow[p] + q] = tmp[q].second;
    }
  }
  check(has_diag_all, "every row needs a diagonal entry");

  // leaf adjacency (Sec. 3.1: edges of the original graph between leaf sets)
  std::vector<std::vector<int>> leaf_adj(nleaf);
  for (int64_t p = 0; p < n; ++p)
    for (int32_t e = P.prow[p]; e < P.prow[p + 1]; ++e) {
      const int a = leaf_of[p], b = leaf_of[P.pcol[e]];
      if (a != b) leaf_adj[a].push_back(b);
    }
  for (int a = 0; a < nleaf; ++a) {
    auto &v = leaf_adj[a];
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
  }
  // structural symmetry
  for (int a = 0; a < nleaf; ++a)
    for (int b : leaf_adj[a])
      check(std::binary_search(leaf_adj[b].begin(), leaf_adj[b].end(), a),
            "pattern is not structurally symmetric");

  // red nodes of the current level: existence, leaf sets, and red-red blocks
  int nred = nleaf;
  std::vector<char> red_exists(nred, 1);
  std::vector<std::vector<int>> red_leaves(nred);
  for (int i = 0; i < nred; ++i) red_leaves[i] = {i};
  std::vector<std::pair<int, int>> red_blocks;  // a < b
  for (int a = 0; a < nleaf; ++a)
    for (int b : leaf_adj[a])
      if (a < b) red_blocks.emplace_back(a, b);

  P.levels.clear();
  P.total_waves = 0;
  for (int lev = L; lev >= 2; --lev) {
    PlanLevel lv;
    lv.level = lev;
    const int nsup = 1 << (lev - 1);
    lv.nsup = nsup;
    lv.exists.assign(nsup, 0);
    lv.sup.assign(nsup, PlanSuper());
    lv.red_made.assign(nsup, 0);
    std::vector<std::vector<int>> sup_leaves(nsup);
    std::vector<int> owner(nleaf, -1);
    for (int i = 0; i < nsup; ++i)
      for (int c = 2 * i; c <= 2 * i + 1; ++c)
        if (red_exists[c]) {
          lv.exists[i] = 1;
          for (int a : red_leaves[c]) {
            sup_leaves[i].push_back(a);
            owner[a] = i;
          }
        }
    // adjacency of super nodes (red node nsup+i has the leaf set of super i)
    std::vector<std::vector<int>> sadj(nsup);
    for (int i = 0; i < nsup; ++i) {
      for (int a : sup_leaves[i])
        for (int b : leaf_adj[a])
          if (owner[b] >= 0 && owner[b] != i) sadj[i].push_back(owner[b]);
      auto &v = sadj[i];
      std::sort(v.begin(), v.end());
      v.erase(std::unique(v.begin(), v.end()), v.end());
    }
    if (nbr_dist == 2) {
      // also the super nodes that share a neighbour at this level (cluster-graph
      // distance 2)
      std::vector<std::vector<int>> s2(nsup);
      for (int i = 0; i < nsup; ++i) {
        auto &v = s2[i];
        v = sadj[i];
        for (int z : sadj[i])
          for (int y : sadj[z])
            if (y != i) v.push_back(y);
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
      }
      sadj.swap(s2);
    }
    auto base = [nsup](int key) { return key >= nsup ? key - nsup : key; };
    auto adjacent = [&](int x, int y) {
      const auto &v = sadj[base(x)];
      return std::binary_search(v.begin(), v.end(), base(y));
    };
    // live blocks, keyed by node (keys 0..2 nsup-1)
    std::vector<std::set<int>> nb(2 * nsup);
    for (auto &ab : red_blocks) {
      const int I = ab.first / 2, J = ab.second / 2;
      if (I != J) {
        nb[I].insert(J);
        nb[J].insert(I);
      }
    }
    std::vector<int> remaining;
    for (int i = 0; i < nsup; ++i)
      if (lv.exists[i]) remaining.push_back(i);
    int widx = 0;
    // wave members so far (a node conflicts with the wave when one of its
    // blocks leads to a member): O(blocks) per candidate
    std::vector<char> inwave(2 * nsup, 0);
    while (!remaining.empty()) {
      std::vector<int> wave;
      for (int s : remaining) {
        bool ok = true;
        for (int x : nb[s])
          if (inwave[x]) {
            ok = false;
            break;
          }
        if (ok) {
          wave.push_back(s);
          inwave[s] = 1;
          if (order_mode == HS_ORDER_SEQUENTIAL) break;   // one super node per step, ascending
        }
      }
      for (int s : wave) {
        PlanSuper &ps = lv.sup[s];
        ps.wave = widx;
        for (int x : nb[s]) (adjacent(s, x) ? ps.N : ps.W).push_back(x);
        for (int x : nb[s]) nb[x].erase(s);
        nb[s].clear();
        for (size_t i = 0; i < ps.N.size(); ++i)
          for (size_t j = i + 1; j < ps.N.size(); ++j) {
            nb[ps.N[i]].insert(ps.N[j]);
            nb[ps.N[j]].insert(ps.N[i]);
          }
        if (!ps.W.empty()) {
          const int r = nsup + s;
          lv.red_made[s] = 1;
          for (int x : ps.N) {
            nb[r].insert(x);
            nb[x].insert(r);
          }
          for (int x : ps.W) {
            nb[r].insert(x);
            nb[x].insert(r);
          }
        }
      }
      std::vector<int> rest;
      for (int s : remaining)
        if (!inwave[s]) rest.push_back(s);
      for (int s : wave) inwave[s] = 0;
      remaining.swap(rest);
      lv.waves.push_back(wave);
      ++widx;
    }
    P.total_waves += widx;
    // the parent level: red node nsup+i becomes red node i
    std::vector<std::pair<int, int>> nxt;
    for (int x = nsup; x < 2 * nsup; ++x)
      for (int y : nb[x]) {
        if (y < nsup) fail(HS_ERR_INVALID, "internal: super node left uneliminated");
        if (x < y) nxt.emplace_back(x - nsup, y - nsup);
      }
    for (int x = 0; x < nsup; ++x)
      if (!nb[x].empty()) fail(HS_ERR_INVALID, "internal: super node left with blocks");
    red_blocks.swap(nxt);
    nred = nsup;
    std::vector<char> nexists(nred, 0);
    std::vector<std::vector<int>> nleaves(nred);
    for (int i = 0; i < nsup; ++i)
      if (lv.red_made[i]) {
        nexists[i] = 1;
        nleaves[i] = sup_leaves[i];
      }
    red_exists.swap(nexists);
    red_leaves.swap(nleaves);
    P.levels.push_back(std::move(lv));
  }
  // root children: the red nodes of level 1 (or the single leaf when L == 0)
  P.red1.assign(red_exists.begin(), red_exists.end());
}

}  // namespace hs
