// Host bookkeeping of accord_path's subsamples (plain C++, no CUDA).
//
// The objective sees the data only through S = X^T X / n (Eq. 3.2), so a
// subsample of n_s row indices with repeats (a bootstrap sample, Sec 3.4)
// can run on the K x p matrix of its K distinct rows, row j scaled by
// sqrt(K c_j / n_s) with c_j its multiplicity: that matrix, divided by K,
// gives the same S as the n_s rows divided by n_s.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "accord.h"

namespace accord {

// Distinct rows of every subsample, ascending, with their scales.
struct Subsamples {
  std::vector<int32_t> rows;   // distinct rows of subsample 0, then 1, ...
  std::vector<double> scale;   // sqrt(K c_j / n_s) of each row
  std::vector<int64_t> off;    // n_sub + 1 offsets into rows
  std::vector<double> n_obs;   // n_s of each subsample
  int64_t kmax = 0;            // largest K
};

// Fills S from the caller's index lists: rows[row_offsets[s] .. row_offsets[s+1])
// are subsample s.  ACCORD_EINVAL for an empty subsample or an index outside
// [0, n).  Multiplicities come from a sorted copy of each subsample, so the
// host memory grows with the subsample, never with n.
inline int compress_subsamples(const int32_t* rows, const int64_t* row_offsets, int64_t n_sub, int64_t n,
                               Subsamples& S) {
  S = Subsamples();
  S.off.assign(1, 0);
  std::vector<int32_t> sorted;
  std::vector<int64_t> count;
  for (int64_t s = 0; s < n_sub; ++s) {
    const int64_t a = row_offsets[s], b = row_offsets[s + 1];
    if (b <= a) return ACCORD_EINVAL;
    sorted.assign(rows + a, rows + b);
    for (int32_t r : sorted)
      if (r < 0 || r >= n) return ACCORD_EINVAL;
    std::sort(sorted.begin(), sorted.end());
    const int64_t first = (int64_t)S.rows.size();
    count.clear();
    for (size_t i = 0; i < sorted.size();) {
      size_t j = i + 1;
      while (j < sorted.size() && sorted[j] == sorted[i]) ++j;
      S.rows.push_back(sorted[i]);
      count.push_back((int64_t)(j - i));
      i = j;
    }
    const double ns = (double)(b - a), K = (double)count.size();
    for (int64_t c : count) S.scale.push_back(std::sqrt(K * (double)c / ns));
    S.off.push_back((int64_t)S.rows.size());
    S.n_obs.push_back(ns);
    S.kmax = std::max<int64_t>(S.kmax, (int64_t)S.rows.size() - first);
  }
  return ACCORD_OK;
}

}  // namespace accord
