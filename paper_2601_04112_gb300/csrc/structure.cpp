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

// Standard aggregation (Section 2.1 passes, every edge strong) on a graph
// given by hyperedges: two vertices are adjacent when an edge holds both.
void hyper_aggregation(int64_t nv, const std::vector<int64_t>& eptr, const std::vector<int32_t>& eidx,
                       std::vector<int32_t>& agg, int64_t& nagg) {
  // neighbour lists (sorted, no self) through vertex -> edge incidence
  std::vector<int64_t> vptr(nv + 1, 0);
  const int64_t ne = (int64_t)eptr.size() - 1;
  for (int64_t e = 0; e < ne; ++e)
    for (int64_t q = eptr[e]; q < eptr[e + 1]; ++q) vptr[eidx[q] + 1]++;
  for (int64_t v = 0; v < nv; ++v) vptr[v + 1] += vptr[v];
  std::vector<int64_t> ve(vptr[nv]);
  {
    std::vector<int64_t> fill(vptr.begin(), vptr.end() - 1);
    for (int64_t e = 0; e < ne; ++e)
      for (int64_t q = eptr[e]; q < eptr[e + 1]; ++q) ve[fill[eidx[q]]++] = e;
  }
  std::vector<int64_t> nptr(nv + 1, 0);
  std::vector<int32_t> nbr;
  std::vector<int64_t> stamp(nv, -1);
  for (int64_t v = 0; v < nv; ++v) {
    stamp[v] = v;
    const size_t s0 = nbr.size();
    for (int64_t k = vptr[v]; k < vptr[v + 1]; ++k) {
      const int64_t e = ve[k];
      for (int64_t q = eptr[e]; q < eptr[e + 1]; ++q) {
        const int32_t u = eidx[q];
        if (stamp[u] != v) {
          stamp[u] = v;
          nbr.push_back(u);
        }
      }
    }
    std::sort(nbr.begin() + s0, nbr.end());
    nptr[v + 1] = (int64_t)nbr.size();
  }
  agg.assign(nv, -1);
  int64_t nxt = 0;
  // pass 1: roots whose neighbours are all unaggregated
  for (int64_t j = 0; j < nv; ++j) {
    if (agg[j] >= 0) continue;
    bool free_all = true;
    for (int64_t k = nptr[j]; k < nptr[j + 1]; ++k)
      if (agg[nbr[k]] >= 0) {
        free_all = false;
        break;
      }
    if (free_all) {
      agg[j] = (int32_t)nxt;
      for (int64_t k = nptr[j]; k < nptr[j + 1]; ++k) agg[nbr[k]] = (int32_t)nxt;
      ++nxt;
    }
  }
  // pass 2: join the lowest-index neighbour aggregated in pass 1
  const std::vector<int32_t> after1(agg);
  for (int64_t j = 0; j < nv; ++j) {
    if (agg[j] >= 0) continue;
    for (int64_t k = nptr[j]; k < nptr[j + 1]; ++k)
      if (after1[nbr[k]] >= 0) {
        agg[j] = after1[nbr[k]];
        break;
      }
  }
  // pass 3: leftovers start aggregates with their unaggregated neighbours
  for (int64_t j = 0; j < nv; ++j) {
    if (agg[j] >= 0) continue;
    agg[j] = (int32_t)nxt;
    for (int64_t k = nptr[j]; k < nptr[j + 1]; ++k)
      if (agg[nbr[k]] < 0) agg[nbr[k]] = (int32_t)nxt;
    ++nxt;
  }
  nagg = nxt;
}

void block_aggregation(int nb, const std::vector<int64_t>& tptr, const std::vector<int32_t>& tids,
                       std::vector<int32_t>& bagg, int& nagg) {
  int64_t na = 0;
  hyper_aggregation(nb, tptr, tids, bagg, na);
  nagg = (int)na;
}

void standard_aggregation(int64_t n, const Supports& S, int passes, std::vector<int32_t>& agg, int64_t& nagg) {
  hyper_aggregation(n, S.ptr, S.idx, agg, nagg);
  std::vector<int64_t> tptr;
  std::vector<int32_t> tids, bagg, seen;
  for (int p = 1; p < passes; ++p) {
    // hyperedges of the graph of T^T A T: the distinct aggregates each row touches
    tptr.assign(1, 0);
    tids.clear();
    seen.assign(nagg, -1);
    const int64_t ng = S.size();
    for (int64_t g = 0; g < ng; ++g) {
      for (int64_t q = S.ptr[g]; q < S.ptr[g + 1]; ++q) {
        const int32_t a = agg[S.idx[q]];
        if (seen[a] != (int32_t)g) {
          seen[a] = (int32_t)g;
          tids.push_back(a);
        }
      }
      tptr.push_back((int64_t)tids.size());
    }
    int64_t nb = 0;
    hyper_aggregation(nagg, tptr, tids, bagg, nb);
    for (auto& a : agg) a = bagg[a];
    nagg = nb;
  }
}

int colour_subdomains(const std::vector<int64_t>& om_ptr, const std::vector<int32_t>& om_idx, int64_t n,
                      const Supports& S, const std::vector<int64_t>& nptr, const std::vector<int32_t>& ngrp) {
  const int64_t nagg = (int64_t)om_ptr.size() - 1;
  if (nagg <= 0) return 0;
  // node -> subdomains holding it
  std::vector<int64_t> sptr(n + 1, 0);
  for (int32_t v : om_idx) sptr[v + 1]++;
  for (int64_t v = 0; v < n; ++v) sptr[v + 1] += sptr[v];
  std::vector<int32_t> sidx(om_idx.size());
  {
    std::vector<int64_t> fill(sptr.begin(), sptr.end() - 1);
    for (int64_t i = 0; i < nagg; ++i)
      for (int64_t q = om_ptr[i]; q < om_ptr[i + 1]; ++q) sidx[fill[om_idx[q]]++] = (int32_t)i;
  }
  std::vector<int32_t> colour(nagg, -1);
  std::vector<int64_t> vstamp(n, -1), cstamp;
  int ncol = 0;
  for (int64_t i = 0; i < nagg; ++i) {
    auto visit = [&](int32_t v) {
      if (vstamp[v] == i) return;
      vstamp[v] = i;
      for (int64_t e = sptr[v]; e < sptr[v + 1]; ++e) {
        const int32_t j = sidx[e];
        if (j < i) cstamp[colour[j]] = i;
      }
    };
    cstamp.resize((size_t)ncol + 1, -1);
    for (int64_t q = om_ptr[i]; q < om_ptr[i + 1]; ++q) {
      const int32_t u = om_idx[q];
      visit(u);
      for (int64_t e = nptr[u]; e < nptr[u + 1]; ++e) {
        const int32_t g = ngrp[e];
        for (int64_t k = S.ptr[g]; k < S.ptr[g + 1]; ++k) visit(S.idx[k]);
      }
    }
    int c = 0;
    while (cstamp[c] == i) ++c;
    colour[i] = c;
    ncol = std::max(ncol, c + 1);
  }
  return ncol;
}

double kappa_threshold(double kappa, int n_color, int n_mult) {
  return std::max(0.1, (kappa - n_color) / ((double)n_color * n_mult));
}

}  // namespace amgdd
