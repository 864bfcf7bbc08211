// Host-side structural setup: graph of A through shared row supports,
// cleanup of unaggregated nodes (Section 3.3), overlapping subdomains
// Omega_i = omega_i u Gamma_i (Section 2.2), touched aggregates and the row
// multiplicity M of the Lemma (Section 3.1), the subdomain colouring of
// Section 3.4.  Standard aggregation itself (level 0, and the coarse block
// graph) runs on the device (aggregate_kernels.cu).
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
