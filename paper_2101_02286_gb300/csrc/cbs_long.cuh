// cbs_long.cuh -- arguments of the long-line kernels (see cbs_long.cu).
#pragma once
#include <stdint.h>

#include "cbs_internal.h"

namespace cbs {

// Lines per CTA of the ends and segment kernels for y/z lines: a tile of
// adjacent lines, so that every row of the tile is one contiguous run.
constexpr int kLongLines = 8;

struct LongArgs {
  const void* in;     // b: the field (x-lines: lines x n, line-contiguous; see LongGeom)
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

// Geometry of the lines, passed to the kernels after their other arguments:
// lines along dir (0 = x, 1 = y, 2 = z) of an (nx, ny, nz) field; es = row
// stride in elements (1, nx or nx ny).  y-lines are numbered x + nx z and
// z-lines x + nx y, so consecutive lines are adjacent in x.
struct LongGeom {
  int64_t nx, ny, es;
  int dir;
};

}  // namespace cbs
