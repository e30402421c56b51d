// cbs_batch.cu -- ragged batches: many independent problems (own sizes,
// direction, bandwidth, precision) solved by one persistent launch.
//
// Every problem is a pre-factorised plan (its DevLineTables and LineArgs live
// in a device array); the host builds a work table with one entry per tile
// of lines (problem, tile x, tile y).  The persistent kernel walks the work
// table with a static stride of gridDim.x, dispatching each tile to the
// line_tile instantiation of its problem.  Input and output pointers travel
// by value in the kernel parameters, so a solve is exactly one launch with
// no allocation, copy or host synchronisation, and can be captured in a CUDA
// graph.
#include <cstring>

#include "cbs_line_launch.cuh"
#include "cbs_long_warp.cuh"

namespace cbs {

// One entry of the batch: an on-chip problem (line tiles: args, tab) or one
// segment size of a long-line problem (warp per segment: largs, lwa, tab =
// the inner tables of that size).  `user` indexes the caller's in/out arrays.
struct alignas(16) BatchProblem {
  LineArgs args;
  DevLineTables tab;
  LongArgs largs;
  LongWarpArgs lwa;
  int variant;
  int user;
};

constexpr int kMaxBatch = 256;

struct BatchParams {
  const BatchProblem* probs;
  const int4* items;  // (problem, tile x, tile y, 0)
  int nitems;
  const void* in[kMaxBatch];
  void* out[kMaxBatch];
};

// The tile variants compiled into the persistent kernel: (R, KS) in
// {(1,2), (2,3), (1,0), (2,0)} x M in {8, 16} x {FP64, FP32 + refinement},
// plus whole-size 16-row partitions (FULL: compile-time sizes) of the same
// (R, KS, mode), FP64 input and output; the same (R, KS) x M in the FP32
// mode with FP32 input and output.
__host__ __device__ constexpr int batch_variant(int R, int KS, int M, int MODE, bool FULL = false) {
  const int rk = (R == 1 && KS == 2) ? 0 : (R == 2 && KS == 3) ? 1 : (R == 1 && KS == 0) ? 2 : (R == 2 && KS == 0) ? 3 : -1;
  const int mi = FULL ? (M == 16 ? 2 : -1) : (M == 8) ? 0 : (M == 16) ? 1 : -1;
  const int mo = (MODE == kModeF64) ? 0 : (MODE == kModeRefine) ? 1 : -1;
  return (rk < 0 || mi < 0 || mo < 0) ? -1 : (rk * 3 + mi) * 2 + mo;
}
// Long-line entries (x-lines, a warp per segment; FP64 in and out): after
// the tile variants.
constexpr int kBatchLong = 24;
__host__ __device__ constexpr int batch_long_variant(int R, int MODE) {
  return (R < 1 || R > 2 || (MODE != kModeF64 && MODE != kModeRefine)) ? -1
                                                                       : kBatchLong + (R - 1) * 2 + (MODE == kModeRefine);
}

// FP32 problems (FP32 in and out, the FP32 mode): after the long-line entries.
constexpr int kBatchF32 = 28;
__host__ __device__ constexpr int batch_f32_variant(int R, int KS, int M) {
  const int rk = (R == 1 && KS == 2) ? 0 : (R == 2 && KS == 3) ? 1 : (R == 1 && KS == 0) ? 2 : (R == 2 && KS == 0) ? 3 : -1;
  const int mi = (M == 8) ? 0 : (M == 16) ? 1 : -1;
  return (rk < 0 || mi < 0) ? -1 : kBatchF32 + rk * 2 + mi;
}

// One tile of an on-chip problem.  A separate function per variant (not
// inlined), so that each variant's register allocation stays its own instead
// of the largest one's pressure spilling in all of them.
template <int R, int M, int MODE, int KS, typename T, bool FULL>
__device__ __noinline__ void batch_tile_item(const BatchProblem& P, const void* in, void* out, int tx, int ty,
                                             unsigned char* smem) {
  line_tile<R, M, MODE, KS, T, T, FULL>(P.args, P.tab, in, out, tx, ty, smem);
}

#define CBS_BV32(R, KS, M)                                                                        \
  case batch_f32_variant(R, KS, M):                                                               \
    batch_tile_item<R, M, kModeF32, KS, float, false>(P, bp.in[P.user], bp.out[P.user], w.y, w.z, \
                                                      tile_smem);                                 \
    break;

#define CBS_BV(R, KS, M, MODE)                                                                  \
  case batch_variant(R, KS, M, MODE):                                                           \
    batch_tile_item<R, M, MODE, KS, double, false>(P, bp.in[P.user], bp.out[P.user], w.y, w.z, \
                                                   tile_smem);                                  \
    break;
#define CBS_BVF(R, KS, MODE)                                                                   \
  case batch_variant(R, KS, 16, MODE, true):                                                   \
    batch_tile_item<R, 16, MODE, KS, double, true>(P, bp.in[P.user], bp.out[P.user], w.y, w.z, \
                                                   tile_smem);                                 \
    break;

// Long-line entry: item (entry, chunk, line); the chunk's kLongWarps
// segments of the line, in the tile's shared memory.  A separate function
// (not inlined), so that its register allocation stays its own.
template <int R, int MODE>
__device__ __noinline__ void batch_long_item(const BatchProblem& P, const void* in, void* out, int chunk, int line,
                                             unsigned char* smem) {
  LongArgs la = P.largs;
  la.in = in;
  la.out = out;
  long_warp_item<R, MODE, double, double>(la, P.tab, P.lwa, chunk, (int64_t)line, smem);
}
#define CBS_BL(R, MODE)                                                                          \
  case batch_long_variant(R, MODE):                                                              \
    batch_long_item<R, MODE>(P, bp.in[P.user], bp.out[P.user], w.y, w.z, tile_smem);             \
    break;

// Shared memory: the current problem's BatchProblem (its tables are read by
// every row operation, so they live on chip instead of in global memory),
// then the tile.
static_assert(sizeof(BatchProblem) % sizeof(int4) == 0, "copied in 16-byte units");
constexpr size_t kBatchProblemBytes = (sizeof(BatchProblem) + 127) / 128 * 128;

__global__ void __launch_bounds__(256, 2) batch_kernel(const __grid_constant__ BatchParams bp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BatchProblem& P = *reinterpret_cast<BatchProblem*>(smem_raw);
  unsigned char* tile_smem = smem_raw + kBatchProblemBytes;
  int loaded = -1;
  for (int it = blockIdx.x; it < bp.nitems; it += gridDim.x) {
    const int4 w = bp.items[it];
    if (w.x != loaded) {  // uniform over the CTA
      const int4* src = reinterpret_cast<const int4*>(bp.probs + w.x);
      int4* dst = reinterpret_cast<int4*>(smem_raw);
      for (int k = threadIdx.x; k < (int)(sizeof(BatchProblem) / sizeof(int4)); k += blockDim.x) dst[k] = src[k];
      __syncthreads();
      loaded = w.x;
    }
    switch (P.variant) {
      CBS_BV(1, 2, 8, kModeF64)
      CBS_BV(1, 2, 8, kModeRefine)
      CBS_BV(1, 2, 16, kModeF64)
      CBS_BV(1, 2, 16, kModeRefine)
      CBS_BV(2, 3, 8, kModeF64)
      CBS_BV(2, 3, 8, kModeRefine)
      CBS_BV(2, 3, 16, kModeF64)
      CBS_BV(2, 3, 16, kModeRefine)
      CBS_BV(1, 0, 8, kModeF64)
      CBS_BV(1, 0, 8, kModeRefine)
      CBS_BV(1, 0, 16, kModeF64)
      CBS_BV(1, 0, 16, kModeRefine)
      CBS_BV(2, 0, 8, kModeF64)
      CBS_BV(2, 0, 8, kModeRefine)
      CBS_BV(2, 0, 16, kModeF64)
      CBS_BV(2, 0, 16, kModeRefine)
      CBS_BVF(1, 2, kModeF64)
      CBS_BVF(1, 2, kModeRefine)
      CBS_BVF(2, 3, kModeF64)
      CBS_BVF(2, 3, kModeRefine)
      CBS_BVF(1, 0, kModeF64)
      CBS_BVF(1, 0, kModeRefine)
      CBS_BVF(2, 0, kModeF64)
      CBS_BVF(2, 0, kModeRefine)
      CBS_BL(1, kModeF64)
      CBS_BL(1, kModeRefine)
      CBS_BL(2, kModeF64)
      CBS_BL(2, kModeRefine)
      CBS_BV32(1, 2, 8)
      CBS_BV32(1, 2, 16)
      CBS_BV32(2, 3, 8)
      CBS_BV32(2, 3, 16)
      CBS_BV32(1, 0, 8)
      CBS_BV32(1, 0, 16)
      CBS_BV32(2, 0, 8)
      CBS_BV32(2, 0, 16)
      default:
        break;
    }
    __syncthreads();  // the next tile reuses the shared memory
  }
}
#undef CBS_BV
#undef CBS_BVF
#undef CBS_BL
#undef CBS_BV32

int batch_variant_host(int R, int KS, int M, int MODE, bool full) { return batch_variant(R, KS, M, MODE, full); }

size_t batch_smem(size_t tile_bytes) { return kBatchProblemBytes + tile_bytes; }

cudaError_t batch_configure(size_t smem) {
  static SmemOptIn opt;
  return opt.ensure(batch_kernel, smem);
}

cudaError_t batch_launch(const BatchProblem* probs, const int4* items, int nitems, const void* const* ins,
                         void* const* outs, int count, int grid, size_t smem, cudaStream_t s) {
  BatchParams bp;
  bp.probs = probs;
  bp.items = items;
  bp.nitems = nitems;
  for (int k = 0; k < kMaxBatch; k++) {
    bp.in[k] = k < count ? ins[k] : nullptr;
    bp.out[k] = k < count ? outs[k] : nullptr;
  }
  batch_kernel<<<grid, kLineThreads, smem, s>>>(bp);
  return cudaGetLastError();
}

size_t batch_problem_bytes() { return sizeof(BatchProblem); }

void batch_fill_problem(void* dst, const LineArgs& a, const DevLineTables& t, int variant, int user) {
  BatchProblem* p = static_cast<BatchProblem*>(dst);
  std::memset(p, 0, sizeof(*p));
  p->args = a;
  p->tab = t;
  p->variant = variant;
  p->user = user;
}

void batch_fill_long(void* dst, const LongArgs& la, const DevLineTables& inner, const LongWarpArgs& wa, int R,
                     int MODE, int user) {
  BatchProblem* p = static_cast<BatchProblem*>(dst);
  std::memset(p, 0, sizeof(*p));
  p->largs = la;
  p->tab = inner;
  p->lwa = wa;
  p->variant = batch_long_variant(R, MODE);
  p->user = user;
}

int batch_long_variant_host(int R, int MODE) { return batch_long_variant(R, MODE); }
int batch_f32_variant_host(int R, int KS, int M) { return batch_f32_variant(R, KS, M); }

// Shared memory of a long-line entry (truncation length K, FP64 input).
size_t batch_long_bytes(int R, int K) { return R == 1 ? lw_bytes<1>(K, 8) : lw_bytes<2>(K, 8); }

}  // namespace cbs
