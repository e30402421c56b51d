// cbs_line_launch.cuh -- template dispatch for the on-chip line kernel.
#pragma once
#include "cbs_line.cuh"

namespace cbs {

constexpr int kLineThreads = 256;

// Launch grid of the tile kernels: x-lines are tiled along the line index;
// y/z lines along x (grid.x) and the remaining coordinate (grid.y).
inline dim3 tile_grid(int64_t nx, int64_t ny, int64_t nz, int64_t nlines, int dir, int lines_per_cta) {
  if (dir == 0) return dim3((unsigned)((nlines + lines_per_cta - 1) / lines_per_cta), 1, 1);
  return dim3((unsigned)((nx + lines_per_cta - 1) / lines_per_cta), (unsigned)(dir == 1 ? nz : ny), 1);
}

template <int R, int M, int MODE, int KS, typename TIn, typename TOut>
cudaError_t launch_one(const LineArgs& a, const DevLineTables& t, cudaStream_t s) {
  using TT = typename std::conditional<(sizeof(TIn) == 8 || sizeof(TOut) == 8), double, float>::type;
  const int threads = kLineThreads;
  const int lines_per_cta = threads / t.pw;
  if (a.nlines <= 0) return cudaSuccess;
  const dim3 grid = tile_grid(a.nx, a.ny, a.nz, a.nlines, a.dir, lines_per_cta);
  const size_t smem = (size_t)lines_per_cta * t.lsz * sizeof(TT);
  static size_t configured = 0;  // per instantiation
  if (smem > 48 * 1024 && smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(line_kernel<R, M, MODE, KS, TIn, TOut>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  line_kernel<R, M, MODE, KS, TIn, TOut><<<grid, threads, smem, s>>>(a, t);
  return cudaGetLastError();
}

template <int R, int M, int MODE, typename TIn, typename TOut>
cudaError_t launch_ks(int KS, const LineArgs& a, const DevLineTables& t, cudaStream_t s) {
  switch (KS) {
    case 0: return launch_one<R, M, MODE, 0, TIn, TOut>(a, t, s);
    case 2: return launch_one<R, M, MODE, 2, TIn, TOut>(a, t, s);
    case 3: return launch_one<R, M, MODE, 3, TIn, TOut>(a, t, s);
  }
  return cudaErrorInvalidValue;
}

template <int R, int MODE, typename TIn, typename TOut>
cudaError_t launch_m(int M, int KS, const LineArgs& a, const DevLineTables& t, cudaStream_t s) {
  switch (M) {
    case 8: return launch_ks<R, 8, MODE, TIn, TOut>(KS, a, t, s);
    case 16: return launch_ks<R, 16, MODE, TIn, TOut>(KS, a, t, s);
    case 32:
      if (MODE != kModeRefine) return launch_ks<R, (MODE != kModeRefine ? 32 : 16), MODE, TIn, TOut>(KS, a, t, s);
      break;
  }
  return cudaErrorInvalidValue;
}

// Defined once per (MODE, R) in its own translation unit.
template <int MODE, int R>
cudaError_t launch_line_mode_r(int M, int KS, int tin, int tout, const LineArgs& a,
                               const DevLineTables& t, cudaStream_t s);

#define CBS_DEFINE_LINE_LAUNCH(MODE, R)                                                      \
  template <>                                                                                \
  cudaError_t launch_line_mode_r<MODE, R>(int M, int KS, int tin, int tout, const LineArgs& a, \
                                          const DevLineTables& t, cudaStream_t s) {          \
    const bool i64 = tin == CBS_DTYPE_F64, o64 = tout == CBS_DTYPE_F64;                     \
    if (MODE != kModeF32 && !o64) return cudaErrorInvalidValue;                              \
    if (i64 && o64) return launch_m<R, MODE, double, double>(M, KS, a, t, s);                \
    if (!i64 && o64) return launch_m<R, MODE, float, double>(M, KS, a, t, s);                \
    if (MODE == kModeF32) {                                                                  \
      if (i64) return launch_m<R, MODE, double, float>(M, KS, a, t, s);                      \
      return launch_m<R, MODE, float, float>(M, KS, a, t, s);                                \
    }                                                                                        \
    return cudaErrorInvalidValue;                                                            \
  }

}  // namespace cbs
