// cbs_bands.h -- line matrices whose rows repeat with a short period: the
// flattened form of block-tridiagonal systems with b x b block entries
// (Sec. 1: block entries, as in compact shock capturing).
//
// A line of N points with b unknowns each, point-major (unknown c of point m
// is row m b + c), with the blocks L, D, U of a block-tridiagonal matrix
// (point m couples to points m - 1, m, m + 1), is a banded matrix of half
// bandwidth 2 b - 1 whose row m b + c holds
//     L[c][j] at offset j - c - b,  D[c][j] at j - c,  U[c][j] at b + j - c
// (j = 0 .. b - 1): its bands depend on the row only through c = row mod b.
// The partition method applies unchanged when every partition starts on a
// point (its size is a multiple of b): then every partition sees the same
// rows, and the per-partition tables stay shared.
#pragma once
#include <string>

#include "cbs_internal.h"

namespace cbs {

constexpr int kMaxPeriod = 2;  // 2 x 2 blocks: half bandwidth 3 = kMaxR

struct PBands {
  int r = 1;
  int period = 1;
  double v[kMaxPeriod][2 * kMaxR + 1] = {};  // v[row % period][t + r]
  double at(int row, int t) const { return (t < -r || t > r) ? 0.0 : v[row % period][t + r]; }
  double max_abs() const {
    double m = 0.0;
    for (int c = 0; c < period; c++)
      for (int t = 0; t < 2 * r + 1; t++) m = m > (v[c][t] < 0 ? -v[c][t] : v[c][t]) ? m : (v[c][t] < 0 ? -v[c][t] : v[c][t]);
    return m;
  }
};

// Bands of the block-tridiagonal matrix with b x b blocks L, D, U (row-major
// b*b doubles each, b <= kMaxPeriod): half bandwidth 2 b - 1, period b.
PBands block_bands(int b, const double* L, const double* D, const double* U);

// build_line_tables for periodic rows; every partition size (the `sizes`
// triple, or n / p) must be a multiple of A.period.
std::string build_line_tables_periodic(LineTables& T, int n, const PBands& A, int p, bool cyclic, bool* singular,
                                       int max_lanes, const int* sizes = nullptr);

}  // namespace cbs
