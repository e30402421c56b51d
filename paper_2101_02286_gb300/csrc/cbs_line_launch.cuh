// cbs_line_launch.cuh -- template dispatch for the on-chip line kernel.
#pragma once
#include <mutex>

#include "cbs_line.cuh"

namespace cbs {

constexpr int kLineThreads = 256;

// Streaming multiprocessors of the current device (cached per process).
inline int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      n = v;
    else
      return 152;
  }
  return n;
}

// Launch grid of the tile kernels: x-lines are tiled along the line index;
// y/z lines along x (grid.x) and the remaining coordinate (grid.y).
inline dim3 tile_grid(int64_t nx, int64_t ny, int64_t nz, int64_t nlines, int dir, int lines_per_cta) {
  if (dir == 0) return dim3((unsigned)((nlines + lines_per_cta - 1) / lines_per_cta), 1, 1);
  return dim3((unsigned)((nx + lines_per_cta - 1) / lines_per_cta), (unsigned)(dir == 1 ? nz : ny), 1);
}

template <int R, int M, int MODE, int KS, typename TIn, typename TOut, bool FULL = false, int LAYOUT = kStaged,
          int ST = 0>
cudaError_t launch_one(const LineArgs& a, const DevLineTables& t, cudaStream_t s) {
  using TT = typename std::conditional<(sizeof(TIn) == 8 || sizeof(TOut) == 8), double, float>::type;
  if (a.nlines <= 0) return cudaSuccess;
  // 256 threads per CTA; small problems shrink the CTA (down to 64 threads)
  // until the grid covers every SM at least twice
  int threads = LAYOUT == kDirectStrided ? kStridedLines * t.pw : kLineThreads;
  dim3 grid = tile_grid(a.nx, a.ny, a.nz, a.nlines, a.dir, threads / t.pw);
  const int64_t want = 2 * (int64_t)sm_count();
  while (LAYOUT != kDirectStrided && threads > 64 && threads > t.pw && (int64_t)grid.x * grid.y < want) {
    threads /= 2;
    grid = tile_grid(a.nx, a.ny, a.nz, a.nlines, a.dir, threads / t.pw);
  }
  const int lines_per_cta = threads / t.pw;
  // staged: the tile; direct strided: the message buffer
  const size_t smem = LAYOUT == kStaged ? (size_t)lines_per_cta * t.lsz * sizeof(TT)
                      : LAYOUT == kDirectStrided ? (size_t)kCtaXchgSlots * threads * sizeof(unsigned long long) : 0;
  static size_t configured = 0;  // per instantiation
  if (smem > 48 * 1024 && smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(line_kernel<R, M, MODE, KS, TIn, TOut, FULL, LAYOUT, ST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  line_kernel<R, M, MODE, KS, TIn, TOut, FULL, LAYOUT, ST><<<grid, threads, smem, s>>>(a, t);
  return cudaGetLastError();
}

// Persistent pipelined launch (whole-size partitions, direct layouts): one
// CTA per resident slot (occupancy x SMs), each walking tiles with the next
// tile's rows in flight while it computes the current one.
template <int R, int M, int MODE, int KS, typename TIn, typename TOut, int LAYOUT, int ST = 0>
cudaError_t launch_pipe(const LineArgs& a, const DevLineTables& t, cudaStream_t s) {
  if (a.nlines <= 0) return cudaSuccess;
  constexpr int NS = M + 2 * KS;
  const int threads = strided_layout(LAYOUT) ? kStridedLines * t.pw : kLineThreads;
  const dim3 grid = tile_grid(a.nx, a.ny, a.nz, a.nlines, a.dir, threads / t.pw);
  const int64_t ntiles = (int64_t)grid.x * grid.y;
  if (ntiles > 0x7fffffff) return cudaErrorInvalidValue;
  const size_t smem = (LAYOUT == kDirectStrided ? (size_t)kCtaXchgSlots * threads * sizeof(unsigned long long) : 0) +
                      2 * (size_t)pipe_buf_elems<M, KS, TIn, LAYOUT>(threads, t.pw, t.p) * sizeof(TIn);
  (void)NS;
  auto kern = line_kernel_pipe<R, M, MODE, KS, TIn, TOut, LAYOUT, ST>;
  // per instantiation: the largest dynamic shared memory configured so far
  // and the occupancy of the last (threads, smem) launched (both depend on
  // the plan's lanes per line, not only on the instantiation)
  static std::mutex mu;
  static size_t attr_smem = 0, occ_smem = 0;
  static int occ_threads = 0, per_sm = 0;
  int blocks_per_sm = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    cudaError_t e = cudaSuccess;
    if (smem > 48 * 1024 && smem > attr_smem) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr_smem = smem;
    }
    if (occ_smem != smem || occ_threads != threads) {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
      if (e != cudaSuccess) return e;
      occ_smem = smem;
      occ_threads = threads;
    }
    blocks_per_sm = per_sm;
  }
  if (blocks_per_sm < 1) return cudaErrorInvalidConfiguration;
  const int per_sm_now = blocks_per_sm;
  const int64_t want = (int64_t)per_sm_now * sm_count();
  const unsigned blocks = (unsigned)(ntiles < want ? ntiles : want);
  kern<<<blocks, threads, smem, s>>>(a, t, (int)grid.x, (int)ntiles);
  return cudaGetLastError();
}

// Whole-size partitions (n = p M): sizes are compile-time constants and the
// direct and pipelined layouts apply.  Compiled for FP64 input and output
// only; x-lines whose arrays are not 16-byte aligned take the staged path.
inline bool tile_full(const DevLineTables& t, int M) { return t.count_big == t.p && t.rows_big == M; }
// The x-line layouts move rows in 16-byte units: both arrays must start on a
// 16-byte boundary (rows of a line then do too, n being a multiple of M).
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <int R, int M, int MODE, int KSV, typename TIn, typename TOut, int ST = 0>
cudaError_t launch_variant(const LineArgs& a, const DevLineTables& t, cudaStream_t s) {
  if constexpr (sizeof(TIn) == 8 && sizeof(TOut) == 8) {
    // acyclic lines with a stencil (boundary closures) extend the end values
    // in the stencil halo, which only the staged layout does
    if (tile_full(t, M) && (a.dir != 0 || (aligned16(a.in) && aligned16(a.out))) && (KSV == 0 || t.cyclic)) {
      // the refinement kernel holds 2 CTAs per SM (registers), too few to
      // hide HBM latency without the pipelined prefetch; the FP64 / FP32
      // kernels keep 3 CTAs per SM and load directly
      if constexpr (refine_mode(MODE)) {
        // y/z lines: with 32 partitions per line a warp can hold a line
        // (messages by shuffles, rows and results through the slots)
        if (a.dir == 0) return launch_pipe<R, M, MODE, KSV, TIn, TOut, kTileX, ST>(a, t, s);
        if (t.pw == 32) return launch_pipe<R, M, MODE, KSV, TIn, TOut, kStridedWarp, ST>(a, t, s);
        return launch_pipe<R, M, MODE, KSV, TIn, TOut, kDirectStrided, ST>(a, t, s);
      } else {
        if (a.dir == 0) return launch_one<R, M, MODE, KSV, TIn, TOut, true, kDirectX, ST>(a, t, s);
        return launch_one<R, M, MODE, KSV, TIn, TOut, true, kDirectStrided, ST>(a, t, s);
      }
    }
  }
  return launch_one<R, M, MODE, KSV, TIn, TOut, false, kStaged, ST>(a, t, s);
}

// KS: stencil terms compiled in; the staggered stencils (LineArgs::stag_*
// in use, a.K <= 2) have their own kernels with two terms.
template <int R, int M, int MODE, typename TIn, typename TOut>
cudaError_t launch_ks(int KS, bool staggered, const LineArgs& a, const DevLineTables& t, cudaStream_t s) {
  if (staggered) {  // staggered stencils: tri- and pentadiagonal bands
    if constexpr (R <= 2) return KS == 2 ? launch_variant<R, M, MODE, 2, TIn, TOut, 1>(a, t, s) : cudaErrorNotSupported;
    return cudaErrorNotSupported;
  }
  switch (KS) {
    case 0: return launch_variant<R, M, MODE, 0, TIn, TOut>(a, t, s);
    case 2: return launch_variant<R, M, MODE, 2, TIn, TOut>(a, t, s);
    case 3: return launch_variant<R, M, MODE, 3, TIn, TOut>(a, t, s);
  }
  return cudaErrorInvalidValue;
}

// Defined once per (MODE, R, M) in its own translation unit (parallel build).
template <int MODE, int R, int M>
cudaError_t launch_line_mrm(int KS, bool staggered, int tin, int tout, const LineArgs& a, const DevLineTables& t,
                            cudaStream_t s);

// Supported element types: FP64 -> FP64 for every mode; FP32 -> FP32 for the
// FP32 mode; FP32 input -> FP64 output without a stencil for the FP64 and
// refinement modes.
#define CBS_DEFINE_LINE_LAUNCH(MODE, R, M)                                                        \
  template <>                                                                                     \
  cudaError_t launch_line_mrm<MODE, R, M>(int KS, bool stag, int tin, int tout, const LineArgs& a, \
                                          const DevLineTables& t, cudaStream_t s) {               \
    const bool i64 = tin == CBS_DTYPE_F64, o64 = tout == CBS_DTYPE_F64;                          \
    if (i64 && o64) return launch_ks<R, M, MODE, double, double>(KS, stag, a, t, s);              \
    if constexpr (MODE == kModeF32) {                                                             \
      if (!i64 && !o64) return launch_ks<R, M, MODE, float, float>(KS, stag, a, t, s);            \
    } else {                                                                                      \
      if (!i64 && o64 && KS == 0 && !stag) return launch_one<R, M, MODE, 0, float, double>(a, t, s); \
    }                                                                                             \
    return cudaErrorNotSupported;                                                                 \
  }

// Dispatch over M (declared specialisations live in the per-M units).
template <int MODE, int R>
inline cudaError_t launch_line_mode_r(int M, int KS, bool stag, int tin, int tout, const LineArgs& a,
                                      const DevLineTables& t, cudaStream_t s) {
  switch (M) {
    case 8:  // heptadiagonal plans take M >= 16
      if constexpr (R <= 2) return launch_line_mrm<MODE, R, 8>(KS, stag, tin, tout, a, t, s);
      break;
    case 16: return launch_line_mrm<MODE, R, 16>(KS, stag, tin, tout, a, t, s);
    case 32:
      if constexpr (!refine_mode(MODE)) return launch_line_mrm<MODE, R, 32>(KS, stag, tin, tout, a, t, s);
      break;
  }
  return cudaErrorNotSupported;
}

}  // namespace cbs
