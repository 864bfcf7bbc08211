// Host-side structural setup: graph of A through shared row supports,
// cleanup of unaggregated nodes (Section 3.3), overlapping subdomains
// Omega_i = omega_i u Gamma_i (Section 2.2), touched aggregates and the row
// multiplicity M of the Lemma (Section 3.1), and standard aggregation of the
// coarse block graph (Section 2.1 passes; the coarse-level rule of
// Algorithm 1 is left open by the paper and is read as aggregating whole
// blocks of coarse dofs).
#include "structure.h"

#include <algorithm>

namespace amgdd {

void node_groups(const Supports& S, int64_t n, std::vector<int64_t>& nptr, std::vector<int32_t>& ngrp) {
  nptr.assign(n + 1, 0);
  for (int32_t v : S.idx) nptr[v + 1]++;
  for (int64_t i = 0; i < n; ++i) nptr[i + 1] += nptr[i];
  ngrp.assign(S.idx.size(), 0);
  std::vector<int64_t> fill(nptr.begin(), nptr.end() - 1);
  const int64_t ng = S.size();
  for (int64_t g = 0; g < ng; ++g)
    for (int64_t p = S.ptr[g]; p < S.ptr[g + 1]; ++p) ngrp[fill[S.idx[p]]++] = (int32_t)g;
}

bool cleanup_aggregates(const int32_t* agg_in, int64_t n, const Supports& S, const std::vector<int64_t>& nptr,
                        const std::vector<int32_t>& ngrp, std::vector<int32_t>& agg, int& nagg) {
  std::vector<int64_t> a(agg_in, agg_in + n);
  for (int64_t j = 0; j < n; ++j)
    if (a[j] < -1) return false;
  for (;;) {
    std::vector<int64_t> todo;
    for (int64_t j = 0; j < n; ++j)
      if (a[j] < 0) todo.push_back(j);
    if (todo.empty()) break;
    bool progress = false;
    for (int64_t j : todo) {
      int64_t best = -1;
      for (int64_t q = nptr[j]; q < nptr[j + 1]; ++q) {
        const int32_t g = ngrp[q];
        for (int64_t p = S.ptr[g]; p < S.ptr[g + 1]; ++p) {
          const int64_t id = a[S.idx[p]];
          if (id >= 0 && (best < 0 || id < best)) best = id;
        }
      }
      if (best >= 0) {
        a[j] = best;
        progress = true;
      }
    }
    if (!progress) {
      int64_t nxt = 0;
      for (int64_t j = 0; j < n; ++j) nxt = std::max(nxt, a[j] + 1);
      for (int64_t j = 0; j < n; ++j)
        if (a[j] < 0) a[j] = nxt++;
    }
  }
  std::vector<int64_t> ids(a);
  std::sort(ids.begin(), ids.end());
  ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
  agg.resize(n);
  for (int64_t j = 0; j < n; ++j) agg[j] = (int32_t)(std::lower_bound(ids.begin(), ids.end(), a[j]) - ids.begin());
  nagg = (int)ids.size();
  return true;
}

void overlap_sets(const std::vector<int32_t>& agg, int nagg, const Supports& S, const std::vector<int64_t>& nptr,
                  const std::vector<int32_t>& ngrp, int overlap, std::vector<int64_t>& om_ptr,
                  std::vector<int32_t>& om_idx, std::vector<int32_t>& nomega) {
  const int64_t n = (int64_t)agg.size();
  std::vector<int64_t> aptr(nagg + 1, 0);
  for (int32_t v : agg) aptr[v + 1]++;
  for (int i = 0; i < nagg; ++i) aptr[i + 1] += aptr[i];
  std::vector<int32_t> members(n);
  {
    std::vector<int64_t> fill(aptr.begin(), aptr.end() - 1);
    for (int64_t j = 0; j < n; ++j) members[fill[agg[j]]++] = (int32_t)j;  // ascending within aggregate
  }
  std::vector<int32_t> mark(n, -1);
  om_ptr.assign(nagg + 1, 0);
  om_idx.clear();
  nomega.assign(nagg, 0);
  std::vector<int32_t> cur, nxt, all, gam;
  for (int i = 0; i < nagg; ++i) {
    cur.assign(members.begin() + aptr[i], members.begin() + aptr[i + 1]);
    all = cur;
    for (int32_t v : cur) mark[v] = i;
    for (int hop = 0; hop < overlap; ++hop) {
      nxt.clear();
      for (int32_t u : cur)
        for (int64_t q = nptr[u]; q < nptr[u + 1]; ++q) {
          const int32_t g = ngrp[q];
          for (int64_t p = S.ptr[g]; p < S.ptr[g + 1]; ++p) {
            const int32_t v = S.idx[p];
            if (mark[v] != i) {
              mark[v] = i;
              nxt.push_back(v);
            }
          }
        }
      all.insert(all.end(), nxt.begin(), nxt.end());
      cur.swap(nxt);
    }
    gam.clear();
    for (int32_t v : all)
      if (agg[v] != i) gam.push_back(v);
    std::sort(gam.begin(), gam.end());
    nomega[i] = (int32_t)(aptr[i + 1] - aptr[i]);
    om_idx.insert(om_idx.end(), members.begin() + aptr[i], members.begin() + aptr[i + 1]);
    om_idx.insert(om_idx.end(), gam.begin(), gam.end());
    om_ptr[i + 1] = (int64_t)om_idx.size();
  }
}

void touched_aggregates(const Supports& S, const std::vector<int32_t>& agg, std::vector<int64_t>& tptr,
                        std::vector<int32_t>& tids, std::vector<int32_t>& M) {
  const int64_t ng = S.size();
  tptr.assign(ng + 1, 0);
  tids.clear();
  M.assign(ng, 0);
  std::vector<int32_t> t;
  for (int64_t g = 0; g < ng; ++g) {
    t.clear();
    for (int64_t p = S.ptr[g]; p < S.ptr[g + 1]; ++p) t.push_back(agg[S.idx[p]]);
    std::sort(t.begin(), t.end());
    t.erase(std::unique(t.begin(), t.end()), t.end());
    tids.insert(tids.end(), t.begin(), t.end());
    tptr[g + 1] = (int64_t)tids.size();
    M[g] = (int32_t)t.size();
  }
}

void block_aggregation(int nb, const std::vector<int64_t>& tptr, const std::vector<int32_t>& tids,
                       std::vector<int32_t>& bagg, int& nagg) {
  std::vector<std::vector<int32_t>> nbr(nb);
  const int64_t ng = (int64_t)tptr.size() - 1;
  for (int64_t g = 0; g < ng; ++g)
    for (int64_t p = tptr[g]; p < tptr[g + 1]; ++p)
      for (int64_t q = tptr[g]; q < tptr[g + 1]; ++q)
        if (tids[p] != tids[q]) nbr[tids[p]].push_back(tids[q]);
  for (auto& v : nbr) {
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
  }
  bagg.assign(nb, -1);
  int nxt = 0;
  // pass 1: roots whose neighbours are all unaggregated
  for (int j = 0; j < nb; ++j) {
    if (bagg[j] >= 0) continue;
    bool free_all = true;
    for (int32_t u : nbr[j])
      if (bagg[u] >= 0) {
        free_all = false;
        break;
      }
    if (free_all) {
      bagg[j] = nxt;
      for (int32_t u : nbr[j]) bagg[u] = nxt;
      ++nxt;
    }
  }
  // pass 2: join the lowest-index neighbour aggregated in pass 1
  const std::vector<int32_t> after1(bagg);
  for (int j = 0; j < nb; ++j) {
    if (bagg[j] >= 0) continue;
    for (int32_t u : nbr[j])
      if (after1[u] >= 0) {
        bagg[j] = after1[u];
        break;
      }
  }
  // pass 3: leftovers start aggregates with their unaggregated neighbours
  for (int j = 0; j < nb; ++j) {
    if (bagg[j] >= 0) continue;
    bagg[j] = nxt;
    for (int32_t u : nbr[j])
      if (bagg[u] < 0) bagg[u] = nxt;
    ++nxt;
  }
  nagg = nxt;
}

}  // namespace amgdd
