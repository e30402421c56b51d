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

// First row and row count of segment s (the first cbig segments have m rows,
// the rest msmall).
__host__ __device__ __forceinline__ int64_t seg_start(const LongArgs& a, int s) {
  return s < a.cbig ? (int64_t)s * a.m : (int64_t)a.cbig * a.m + (int64_t)(s - a.cbig) * a.msmall;
}
__host__ __device__ __forceinline__ int seg_rows(const LongArgs& a, int s) { return s < a.cbig ? a.m : a.msmall; }

// Geometry of the lines, passed to the kernels after their other arguments:
// lines along dir (0 = x, 1 = y, 2 = z) of an (nx, ny, nz) field; es = row
// stride in elements (1, nx or nx ny).  y-lines are numbered x + nx z and
// z-lines x + nx y, so consecutive lines are adjacent in x.
struct LongGeom {
  int64_t nx, ny, es;
  int dir;
};

// Element offset of row 0 of a line (row k at + k * es); line < 2^31.
__device__ __forceinline__ int64_t long_base(const LongArgs& a, const LongGeom& gm, int64_t line) {
  if (gm.dir == 0) return line * a.n;
  if (gm.dir == 1) {
    const unsigned L = (unsigned)line, NX = (unsigned)gm.nx;
    return (int64_t)(L % NX) + gm.nx * gm.ny * (int64_t)(L / NX);
  }
  return line;
}

// The warp-per-segment path (cbs_long_warp.cu): segments of 32 x 16 + r rows
// (or 31 x 16 + r), whose outer interface system is decoupled to FP64
// rounding.  Launch for segments seg0 .. seg0 + nseg - 1 (all of one size);
// x-lines: kLongWarps consecutive segments of one line per CTA; y/z lines:
// one segment of kLongWarps adjacent lines per CTA.
constexpr int kLongWarps = 4;
// Register budget of the kernel as CTAs per SM (65536 / (CTAs x 128 threads)
// registers per thread): 8 (64 registers) for the FP64 / FP32 modes and the
// one-sweep refinement, 5 (96) for more sweeps, which keep x0 as a float pair.
constexpr int long_ctas_per_sm(bool light) { return light ? 8 : 5; }
// The inner (segment-level) acyclic interface system of one segment size in
// compact form: the stages that act, in order.  Entry e has flags bit 0 (a
// message stage: x~ -= KM x~_{i-s} + KP x~_{i+s}, from the values before the
// stage), bit 1 (x~ <- C x~; consecutive stages without messages are
// multiplied into one), stride s, and its per-lane blocks at tab + 32 off:
// [C (bit 1)] [KM, KP (bit 0)], each r x r entries x 32 lanes, lane
// fastest, in the interface precision.
constexpr int kLwMaxEnt = 8;
struct LwIface {
  const void* tab;
  int ne;
  int s[kLwMaxEnt], flags[kLwMaxEnt], off[kLwMaxEnt];
};
struct LongWarpArgs {
  double Dinv[kMaxR * kMaxR];            // inverse of the outer diagonal block D-hat (r x r)
  double Lt[kMaxR * kMaxR], Ut[kMaxR * kMaxR];  // b-hat assembly (Eq. 21)
  const float* Gh;                       // [r][K] leading entries of D^{-1}'s first rows as
  const float* Gl;                       //   float pairs (G = Gh + Gl)
  LwIface ifc;                           // inner system of this launch's segment size
  LongGeom gm;                           // line geometry (y/z lines: a CTA per group of adjacent lines)
  int ngroups;                           // y/z lines: groups of kLongWarps adjacent lines
  int seg0, nseg, nchunks;               // nchunks = ceil(nseg / kLongWarps)
  int* status;                           // device status word
};

}  // namespace cbs
