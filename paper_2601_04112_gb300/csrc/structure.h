// Host-side structural setup (integer work) of the hierarchy.
#pragma once

#include <cstdint>
#include <vector>

namespace amgdd {

// Supports of the row groups of G_l: group g covers g_idx[g_ptr[g] .. g_ptr[g+1]).
struct Supports {
  std::vector<int64_t> ptr;
  std::vector<int32_t> idx;
  int64_t size() const { return (int64_t)ptr.size() - 1; }
  int len(int64_t g) const { return (int)(ptr[g + 1] - ptr[g]); }
};

// node -> groups containing it (CSR, groups ascending)
void node_groups(const Supports& S, int64_t n, std::vector<int64_t>& nptr, std::vector<int32_t>& ngrp);

// Attach -1 nodes (smallest aggregated neighbour id, ascending sweeps;
// isolated leftovers become new aggregates) and relabel ids 0..nagg-1.
// Returns false if an id is < -1.
bool cleanup_aggregates(const int32_t* agg_in, int64_t n, const Supports& S, const std::vector<int64_t>& nptr,
                        const std::vector<int32_t>& ngrp, std::vector<int32_t>& agg, int& nagg);

// Omega_i (omega_i ascending, then Gamma_i ascending) within `overlap` hops.
void overlap_sets(const std::vector<int32_t>& agg, int nagg, const Supports& S, const std::vector<int64_t>& nptr,
                  const std::vector<int32_t>& ngrp, int overlap, std::vector<int64_t>& om_ptr,
                  std::vector<int32_t>& om_idx, std::vector<int32_t>& nomega);

// Per group: sorted touched aggregate ids (touched_ptr/touched) and the
// multiplicity M = number of touched aggregates (Lemma).
void touched_aggregates(const Supports& S, const std::vector<int32_t>& agg, std::vector<int64_t>& tptr,
                        std::vector<int32_t>& tids, std::vector<int32_t>& M);

// Greedy colouring of the overlapping subdomains (Section 3.4, n_color):
// Omega_i and Omega_j take distinct colours when A couples them (a node of
// one shares a row group of G with, or is, a node of the other); subdomains
// are coloured in ascending index with the smallest colour no earlier coupled
// subdomain holds.  Returns the number of colours.
int colour_subdomains(const std::vector<int64_t>& om_ptr, const std::vector<int32_t>& om_idx, int64_t n,
                      const Supports& S, const std::vector<int64_t>& nptr, const std::vector<int32_t>& ngrp);

// Local eigenvalue threshold from a target condition number kappa (Section
// 3.4): max{0.1, (kappa - n_color) / (n_color n_multiplicity)}.
double kappa_threshold(double kappa, int n_color, int n_mult);

// Standard aggregation (Section 2.1 passes, every edge strong) on the graph
// whose vertices are adjacent when a hyperedge (eptr/eidx lists) holds both;
// ids in creation order.
void hyper_aggregation(int64_t nv, const std::vector<int64_t>& eptr, const std::vector<int32_t>& eidx,
                       std::vector<int32_t>& agg, int64_t& nagg);

// Level-0 aggregates on the graph of A = D1 + G^T G (rows of G as
// hyperedges), with `passes` passes of aggregating aggregates: pass p + 1
// aggregates the graph of T_p^T A T_p (Section 3.3).
void standard_aggregation(int64_t n, const Supports& S, int passes, std::vector<int32_t>& agg, int64_t& nagg);

// Standard aggregation with all edges strong on the graph of aggregates
// that share a row (block graph); returns block -> coarse aggregate.
void block_aggregation(int nblocks, const std::vector<int64_t>& tptr, const std::vector<int32_t>& tids,
                       std::vector<int32_t>& bagg, int& nagg);

}  // namespace amgdd
