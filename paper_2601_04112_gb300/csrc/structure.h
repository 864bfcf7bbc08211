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

}  // namespace amgdd
