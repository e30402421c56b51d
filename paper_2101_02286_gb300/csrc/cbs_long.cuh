// cbs_long.cuh -- arguments of the long-line kernels (see cbs_long.cu).
#pragma once
#include <stdint.h>

#include "cbs_internal.h"

namespace cbs {

struct LongArgs {
  const void* in;     // b, lines x n (line-contiguous)
  void* out;          // x, same layout, FP64 (or FP32 for FP32 mode)
  double* yb;         // [line][seg][2r]: y_i first r, then last r rows
  double* xt;         // [line][seg][r]: interface solution x~
  double* cc;         // [line][seg][2r]: RHS corrections of the first r / last r bulk rows
  const double* G;    // [q][K]: leading entries of rows q < r of D^{-1}
  int K;              // kept entries per row
  int64_t lines;
  int n, p, m, r;     // line length, segments, rows of the first cbig segments, half bandwidth
  int cbig, msmall;   // segments cbig.. have msmall rows
  int sweeps;
  double band[2 * kMaxR + 1];
};

}  // namespace cbs
