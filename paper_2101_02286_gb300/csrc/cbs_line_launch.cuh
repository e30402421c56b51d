// cbs_line_launch.cuh -- template dispatch for the on-chip line kernel.
#pragma once
#include <mutex>

#include "cbs_line.cuh"

namespace cbs {

constexpr int kLineThreads = 256;

constexpr int kMaxDevices = 64;

// Streaming multiprocessors of the current device (cached per device).
inline int sm_count() {
  static int n[kMaxDevices] = {};
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 152;
  if (n[dev] == 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 152;
    n[dev] = v;
  }
  return n[dev];
}

// Opt-in to more than 48 KB of dynamic shared memory for one kernel: the
// attribute belongs to the device, so the largest size set so far is kept
// per device (one instance per kernel, a static at the call site).
struct SmemOptIn {
  std::mutex mu;
  size_t done[kMaxDevices] = {};
  template <typename K>
  cudaError_t ensure(K kern, size_t smem) {
    if (smem <= 48 * 1024) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (smem <= done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) done[dev] = smem;
    return e;
  }
};

// Resident blocks per SM of one kernel at the last (device, threads, shared
// memory) it was launched with (one instance per kernel, a static at the
// call site).
struct OccupancyCache {
  std::mutex mu;
  size_t smem = 0;
  int threads = 0, dev = -1, per_sm = 0;
  template <typename K>
  cudaError_t get(K kern, int nthreads, size_t nsmem, int* out) {
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (dev != d || smem != nsmem || threads != nthreads) {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nthreads, nsmem);
      if (e != cudaSuccess) {
        dev = -1;
        return e;
      }
      dev = d;
      smem = nsmem;
      threads = nthreads;
    }
    *out = per_sm;
    return cudaSuccess;
  }
};

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
  static SmemOptIn opt;  // per instantiation
  cudaError_t e = opt.ensure(line_kernel<R, M, MODE, KS, TIn, TOut, FULL, LAYOUT, ST>, smem);
  if (e != cudaSuccess) return e;
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
  // per instantiation: the shared-memory opt-in and the occupancy (both
  // depend on the plan's lanes per line, not only on the instantiation)
  static SmemOptIn opt;
  cudaError_t e = opt.ensure(kern, smem);
  if (e != cudaSuccess) return e;
  static OccupancyCache occ;
  int blocks_per_sm = 0;
  e = occ.get(kern, threads, smem, &blocks_per_sm);
  if (e != cudaSuccess) return e;
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
