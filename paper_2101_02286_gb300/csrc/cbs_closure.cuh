// cbs_closure.cuh -- one-sided boundary closures of an acyclic derivative.
//
// The line kernels solve the acyclic Toeplitz system T y = S f, with S the
// central stencil whose rows near the ends read the end values in place of
// the rows beyond them (f_{-q} = f_0, f_{n-1+q} = f_{n-1}: the right-hand side
// then stays of the size of f' for smooth f, where a periodic wrap would put
// jumps of size f / h into it and amplify the FP32 solves' rounding).  The
// closure system A_c x = B_c f differs from it only in
// the c first and c last rows (the 2c "boundary rows" u_0..u_{2c-1}):
//   A_c = T + U E^T,   B_c f = S f + U d,
// with U = [e_{u_0} .. e_{u_{2c-1}}], E^T the differences of the LHS rows and
// d the differences of the RHS rows at the boundary rows.  Woodbury gives
//   x = y + Z M^{-1} (d - E^T y),   Z = T^{-1} U,   M = I + E^T Z,
// a correction that only touches the rows where the columns of Z exceed
// 2^-60 of their largest entry (they decay geometrically away from the ends).
// The plan precomputes, in FP64 on the host: the window rows that d and E^T y
// read, their coefficients, M^{-1} and the kept rows of Z.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "cbs_internal.h"

namespace cbs {

constexpr int kMaxClosureRows = 4;   // c: boundary rows at each end
constexpr int kMaxClosureWidth = 16; // columns of a closure row

struct ClosureArgs {
  const void* f;      // the field (input of the solve)
  void* x;            // the solve's output: y on entry, x on exit
  int64_t lines, nx, ny;
  int dir, n;
  int c2;             // 2c boundary rows
  int nw, nu;         // window rows (d and E^T y), updated rows
  const int* wrow;    // [nw] window rows
  const int* urow;    // [nu] updated rows
  const double* Df;   // [c2][nw]: d = Df f (row coefficients on f, 1/h included)
  const double* Ey;   // [c2][nw]: E^T y = Ey y
  const double* Minv; // [c2][c2]
  const double* Zt;   // [nu][c2]: the kept rows of Z
};

// Host tables of a closure plan: built by closure_build, uploaded by the plan.
struct ClosureTables {
  int c2 = 0;
  std::vector<int> wrow, urow;
  std::vector<double> Df, Ey, Minv, Zt;
};

// Build the tables for lines of n points: Toeplitz bands `band` (2r+1 values,
// t = -r..r), central stencil weights w[q-1] = c_q / (2 q h) for q = 1..K,
// c closure rows of width W from `closure` (as in cbs_desc), spacing h.
// Returns "" or an error; *singular is set when M is singular.
std::string closure_build(ClosureTables& C, int n, int r, const double* band, int K, const double* w, int c, int W,
                          const double* closure, double h, bool* singular);

// Launch the correction over every line (after the line kernel, same stream).
cudaError_t launch_closure(const ClosureArgs& a, bool in64, bool out64, cudaStream_t s);

}  // namespace cbs
