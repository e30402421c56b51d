// cbs_long.cu -- lines too long for one warp: p segments per line, one CTA
// per segment (the paper's distributed level across thread blocks).
//
// A solve is three launches on one stream (four when the segments come in
// two sizes: the segment kernel then runs once per size):
//   1. ends:  for every segment only the first r and last r rows of
//             y_i = D_i^{-1} b_i are needed (Sec. 4: only those rows cross
//             partitions).  They are dot products of the segment's right-hand
//             side with rows of D_i^{-1} (Toeplitz, symmetric and
//             persymmetric, so one table of r rows serves both ends).  The
//             rows decay geometrically away from the diagonal; the plan keeps
//             the K leading entries whose tail is below 2^-60 of the row's
//             l1 norm, so only the segment ends are read.  FP64.
//   2. iface: per line, b-hat (Eq. 21) and the cyclic interface system by
//             the pre-factorised block PCR with detach/reattach
//             (Algorithms 1-4), messages through shared memory.  FP64.
//   3. seg:   per segment, D_i x_i = b_i - L_i x~_i - U_i x~_{i+1} (Eq. 9),
//             solved by the same partition method one level down: the
//             CTA's threads are acyclic sub-partitions exchanging through
//             shared memory; FP64, FP32, or FP32 + refinement with an
//             FP64-accurate residual.  Writes every row of x, interface rows
//             included.  When every segment's bulk is a whole number of
//             16-row inner partitions, the partition sizes are compile-time
//             constants and the refinement residual runs two rows per
//             instruction.
// Scratch: yb and cc (2r doubles per segment) and xt (r doubles per segment).
#include <mutex>
#include <string>

#include "cbs_line_launch.cuh"
#include "cbs_long.cuh"
#include "cbs_plan_struct.h"

namespace cbs {




// ---------------------------------------------------------------- 1. ends
// One CTA per (segment, LG lines): x-lines LG = 1; y/z lines LG = kLongLines
// adjacent lines, thread = (j, line) with the line fastest, so each row of
// the tile is read as one contiguous run.
template <typename TIn, int LG>
__global__ void __launch_bounds__(128) long_ends_kernel(const LongArgs a, const LongGeom gm) {
  constexpr int J = 128 / LG;           // threads per line
  const int seg = blockIdx.y;           // grid (line tiles, segments): lines may exceed 65535
  const int g = LG == 1 ? 0 : threadIdx.x % LG, jj = LG == 1 ? threadIdx.x : threadIdx.x / LG;
  const int64_t line = (int64_t)blockIdx.x * LG + g;
  const bool line_ok = LG == 1 || line < a.lines;
  const int r = a.r, N = seg_rows(a, seg) - r;
  const int64_t es = LG == 1 ? 1 : gm.es;
  const TIn* b = (const TIn*)a.in + (LG == 1 ? line * a.n : long_base(a, gm, line)) + (seg_start(a, seg) + r) * es;
  double accF[kMaxR], accL[kMaxR];
#pragma unroll
  for (int q = 0; q < kMaxR; q++) accF[q] = accL[q] = 0.0;
  for (int j = jj; line_ok && j < a.K; j += J) {
    const double bf = (double)__ldg(b + j * es), bl = (double)__ldg(b + (N - 1 - j) * es);
#pragma unroll
    for (int q = 0; q < kMaxR; q++)
      if (q < r) {
        accF[q] += __ldg(a.G + q * a.K + j) * bf;
        accL[q] += __ldg(a.G + (r - 1 - q) * a.K + j) * bl;  // persymmetry of D^{-1}
      }
  }
  __shared__ double red[2 * kMaxR][4][LG];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 2 * kMaxR; q++) {
    double v = (q < kMaxR) ? accF[q] : accL[q - kMaxR];
#pragma unroll
    for (int o = 16; o >= LG; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    if (lane < LG) red[q][wid][lane] = v;  // lane = the line for lane < LG
  }
  __syncthreads();
  if (threadIdx.x < 2 * r * LG) {
    const int q = threadIdx.x / LG, gg = threadIdx.x % LG;  // q: 0..r-1 first rows, r..2r-1 last rows
    const int64_t ln = (int64_t)blockIdx.x * LG + gg;
    if (LG == 1 || ln < a.lines) {
      const int slot = (q < r) ? q : kMaxR + (q - r);
      double v = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) v += red[slot][w][gg];
      a.yb[(ln * a.p + seg) * 2 * r + q] = v;
    }
  }
}

// x-lines: one warp per (line, segment) item, 8 items per CTA; lane j reads
// rows j, j + 32, ... of both ends (contiguous) and the sums are reduced with
// shuffles.  A CTA per item spent more time launching and reducing than
// reading (K ~ 50 rows per end).
template <typename TIn>
__global__ void __launch_bounds__(256) long_ends_warp_kernel(const LongArgs a, const int64_t items) {
  const int64_t item = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (item >= items) return;  // whole warps: no barrier below
  const int lane = threadIdx.x & 31;
  const int64_t line = item / a.p;
  const int seg = (int)(item - line * a.p);
  const int r = a.r, N = seg_rows(a, seg) - r;
  const TIn* b = (const TIn*)a.in + line * a.n + seg_start(a, seg) + r;  // first bulk row
  double accF[kMaxR], accL[kMaxR];
#pragma unroll
  for (int q = 0; q < kMaxR; q++) accF[q] = accL[q] = 0.0;
  for (int j = lane; j < a.K; j += 32) {
    const double bf = (double)__ldg(b + j), bl = (double)__ldg(b + N - 1 - j);
#pragma unroll
    for (int q = 0; q < kMaxR; q++)
      if (q < r) {
        accF[q] += __ldg(a.G + q * a.K + j) * bf;
        accL[q] += __ldg(a.G + (r - 1 - q) * a.K + j) * bl;  // persymmetry of D^{-1}
      }
  }
#pragma unroll
  for (int q = 0; q < kMaxR; q++) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      accF[q] += __shfl_xor_sync(kFull, accF[q], o);
      accL[q] += __shfl_xor_sync(kFull, accL[q], o);
    }
  }
  double* yb = a.yb + item * 2 * r;  // item = line * p + seg
#pragma unroll
  for (int q = 0; q < kMaxR; q++)
    if (q < r && lane == 0) {
      yb[q] = accF[q];
      yb[r + q] = accL[q];
    }
}

// ---------------------------------------------------------------- 2. interface
template <typename TIn, bool STR>
__global__ void __launch_bounds__(1024) long_iface_kernel(const LongArgs a, const DevLineTables t, const LongGeom gm) {
  extern __shared__ __align__(16) double xs[];  // 2 buffers of p*r
  const int64_t line = blockIdx.x;
  const int p = a.p, r = a.r, rr = r * r;
  const double* yb = a.yb + line * p * 2 * r;
  const TIn* bl = (const TIn*)a.in + (STR ? long_base(a, gm, line) : line * a.n);
  const int64_t es = STR ? gm.es : 1;
  double* X0 = xs;
  double* X1 = xs + p * r;
  // b-hat_i = b~_i - L~ y_{i-1}[last] - U~ y_i[first]   (Eq. 21)
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    const int im = (i == 0) ? p - 1 : i - 1;
    for (int q = 0; q < r; q++) {
      double v = STR ? (double)__ldg(bl + (seg_start(a, i) + q) * es) : (double)__ldg(bl + seg_start(a, i) + q);
      for (int e = 0; e < r; e++) {
        v -= t.Lt[q][e] * yb[im * 2 * r + r + e];
        v -= t.Ut[q][e] * yb[i * 2 * r + e];
      }
      X0[i * r + q] = v;
    }
  }
  __syncthreads();
  for (int st = 0; st < t.nstage; st++) {
    // flags exist for the first kMaxStages stages; later ones run in full
    const bool known = st < kMaxStages;
    const bool msg = !known || (t.stage_msg[st] & 1) != 0;  // couplings above FP64 rounding
    if (!msg && known && !t.stage_has_c[st]) continue;
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
      const int sm = __ldg(t.src + (st * 2 + 0) * p + i), sp = __ldg(t.src + (st * 2 + 1) * p + i);
      for (int q = 0; q < r; q++) {
        double acc = 0.0;
        for (int e = 0; e < r; e++) {
          acc += __ldg(t.coef + ((st * 3 + 0) * rr + q * r + e) * p + i) * X0[i * r + e];
          if (msg) {
            acc -= __ldg(t.coef + ((st * 3 + 1) * rr + q * r + e) * p + i) * X0[sm * r + e];
            acc -= __ldg(t.coef + ((st * 3 + 2) * rr + q * r + e) * p + i) * X0[sp * r + e];
          }
        }
        X1[i * r + q] = acc;
      }
    }
    __syncthreads();
    double* tmp = X0;
    X0 = X1;
    X1 = tmp;
  }
  for (int k = threadIdx.x; k < p * r; k += blockDim.x) a.xt[line * p * r + k] = X0[k];
  // Eq. 9 right-hand-side terms for every segment: bulk row j < r couples to
  // x~_i[q] at offset q - r - j; bulk row N - r + e couples to x~_{i+1}[q]
  // at offset q + r - e.
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    const int ip = (i + 1 == p) ? 0 : i + 1;
    for (int j = 0; j < r; j++) {
      double c = 0.0, d = 0.0;
      for (int q = 0; q < r; q++) {
        const int o1 = q - r - j, o2 = q + r - j;
        if (o1 >= -r) c += a.band[o1 + r] * X0[i * r + q];
        if (o2 <= r) d += a.band[o2 + r] * X0[ip * r + q];
      }
      a.cc[(line * p + i) * 2 * r + j] = c;
      a.cc[(line * p + i) * 2 * r + r + j] = d;
    }
  }
}

// ---------------------------------------------------------------- 3. segments
// One CTA per (segment, line); thread i = inner partition i of the segment's
// bulk rows (acyclic, tables `tin`).  Grid (lines, segments): line blockIdx.x,
// segment seg0 + blockIdx.y.  FULL: every
// inner partition has exactly M rows (whole-16-row layout): sizes are
// compile-time and the refinement uses the paired residual.
// One (segment, line) item, solved by the whole CTA.
// LG: lines per CTA (1: x-lines, thread i = inner partition i; 2, 4 or 8:
// y/z lines, thread = (inner partition i, line g) with g fastest).
// PIPE: the bulk rows were copied ahead into shared-memory slots (this
// thread's row k at pslot[k * pstride]) by the persistent kernel below.
template <int R, int M, int MODE, typename TIn, typename TOut, bool FULL, int LG, typename X, bool PIPE = false>
__device__ __forceinline__ void seg_item(const LongArgs& a, const DevLineTables& tin, const LongGeom& gm,
                                         const int seg, const int64_t line, X& xch, const TIn* pslot = nullptr,
                                         const int pstride = 0) {
  using T = typename std::conditional<MODE == kModeF64, double, float>::type;
  const int i = LG == 1 ? threadIdx.x : threadIdx.x / LG, P = tin.p;
  const bool line_ok = LG == 1 || line < a.lines;
  const bool lane_ok = i < P && line_ok;
  int start = 0, size = FULL ? M : 2 * R;
  if (FULL) start = i * M;
  else if (lane_ok) partition_of(tin, i, start, size);
  const int64_t es = LG == 1 ? 1 : gm.es;
  // the segment's first row, then this partition's first bulk row
  const int64_t row0 = LG == 1 ? line * a.n + seg_start(a, seg) : long_base(a, gm, line) + seg_start(a, seg) * es;
  const TIn* b = LG == 1 ? (const TIn*)a.in + row0 + R + start : (const TIn*)a.in + row0 + (R + start) * es;
  TOut* x = LG == 1 ? (TOut*)a.out + row0 + R + start : (TOut*)a.out + row0 + (R + start) * es;
  const double* xt_here = a.xt + (line * a.p + seg) * R;
  const double* cc = a.cc + (line * a.p + seg) * 2 * R;  // [first R rows | last R rows]
  // Eq. 9 couplings to the known interface values, moved to the RHS; only the
  // first partition (bulk rows 0..R-1) and the last (rows size-R..size-1)
  double cF[R], cL[R];
#pragma unroll
  for (int e = 0; e < R; e++) {
    cF[e] = (lane_ok && i == 0) ? cc[e] : 0.0;
    cL[e] = (lane_ok && i == P - 1) ? cc[R + e] : 0.0;
  }
  using TIR = typename std::conditional<MODE == kModeRefineI64, double, float>::type;  // interface of the FP32 solves
  if constexpr (!refine_mode(MODE)) {
    T v[M];
#pragma unroll
    for (int k = 0; k < M; k++) {
      T val = T(0);
      if (lane_ok && (FULL || k < size)) val = conv<T>(PIPE ? pslot[k * pstride] : __ldg(b + k * es));
      if (k < R) val -= conv<T>(cF[k]);
#pragma unroll
      for (int e = 0; e < R; e++) {
        if (FULL) {
          if (k == M - R + e) val -= conv<T>(cL[e]);
        } else {
          val -= sel(k == size - R + e, conv<T>(cL[e]), T(0));
        }
      }
      v[k] = val;
    }
    solve_partition<T, R, M, T, FULL>(v, size, i, lane_ok, tin, xch);
    if (lane_ok) {
#pragma unroll
      for (int k = 0; k < M; k++)
        if (FULL || k < size) x[k * es] = conv<TOut>(v[k]);
    }
  } else {
    float bh[M], bl[M], xh[M], xl[M], v[M];
    f2 sF[R], sL[R];
#pragma unroll
    for (int e = 0; e < R; e++) {
      sF[e] = split_f64(cF[e]);
      sL[e] = split_f64(cL[e]);
    }
#pragma unroll
    for (int k = 0; k < M; k++) {
      f2 s = {0.f, 0.f};
      if (lane_ok && (FULL || k < size)) s = split_in(PIPE ? pslot[k * pstride] : __ldg(b + k * es));
      // subtract the correction (zero on all but the edge rows) exactly
      f2 c = {0.f, 0.f};
      if (k < R) c = sF[k];
#pragma unroll
      for (int e = 0; e < R; e++) {
        if (FULL) {
          if (k == M - R + e) c = sL[e];
        } else {
          c.hi = sel(k == size - R + e, sL[e].hi, c.hi);
          c.lo = sel(k == size - R + e, sL[e].lo, c.lo);
        }
      }
      const f2 d = two_sum(s.hi, -c.hi);
      bh[k] = d.hi;
      bl[k] = d.lo + (s.lo - c.lo);
      v[k] = d.hi;
    }
    solve_partition<float, R, M, TIR, FULL>(v, size, i, lane_ok, tin, xch);
#pragma unroll
    for (int k = 0; k < M; k++) {
      xh[k] = v[k];
      xl[k] = 0.f;
    }
    for (int sw = 0; sw < a.sweeps; sw++) {
      if constexpr (FULL && (M % 2) == 0) {
        if (sw == 0) residual_sym2<R, M, false>(bh, bl, xh, xl, v, i, tin, xch);
        else residual_sym2<R, M, true>(bh, bl, xh, xl, v, i, tin, xch);
      } else {
        if (sw == 0) residual_df<R, M, false, false>(bh, bl, xh, xl, v, size, i, tin, xch);
        else residual_df<R, M, true, false>(bh, bl, xh, xl, v, size, i, tin, xch);
      }
      solve_partition<float, R, M, TIR, FULL>(v, size, i, lane_ok, tin, xch);
#pragma unroll
      for (int k = 0; k < M; k++) {
        const f2 s = two_sum(xh[k], v[k]);
        xh[k] = s.hi;
        xl[k] = xl[k] + s.lo;
      }
    }
    if (lane_ok) {
#pragma unroll
      for (int k = 0; k < M; k++)
        if (FULL || k < size) x[k * es] = (TOut)(f32_to_f64(xh[k]) + f32_to_f64(xl[k]));
    }
  }
  // the segment's interface rows
  if (LG == 1) {
    if (threadIdx.x < R) ((TOut*)a.out)[row0 + threadIdx.x] = (TOut)xt_here[threadIdx.x];
  } else if (i < R && line_ok) {
    ((TOut*)a.out)[row0 + i * es] = (TOut)xt_here[i];
  }
}

template <int R, int M, int MODE, typename TIn, typename TOut, bool FULL, int LG>
__global__ void __launch_bounds__(512, 1) long_seg_kernel(const LongArgs a, const DevLineTables tin, const int seg0,
                                                         const LongGeom gm) {
  extern __shared__ __align__(16) unsigned long long xbuf[];  // kCtaXchgSlots * blockDim slots
  const int g = LG == 1 ? 0 : threadIdx.x % LG;
  CtaXchgT<LG == 1 ? 0 : LG> xch{xbuf, 0, 1, g};
  seg_item<R, M, MODE, TIn, TOut, FULL, LG>(a, tin, gm, seg0 + blockIdx.y, (int64_t)blockIdx.x * LG + g, xch);
}

// Persistent, software-pipelined segment kernel for y/z tiles: each CTA
// walks the items (tile, segment) = it % tiles, seg0 + it / tiles for it =
// blockIdx.x, + gridDim.x, ..., and issues the asynchronous copies of the next
// item's bulk rows into the other half of a double buffer of thread-private
// shared-memory slots before solving the current one, so that the strided
// HBM reads overlap the arithmetic (the plain kernel is bound by load
// latency: 16 warps per SM at 128 registers).  Shared memory: the message
// buffer (kCtaXchgSlots slots per thread), then 2 x M slots of TIn per thread.
// Slots of one buffer: thread t's row k at sbuf[k * blockDim + t]; each thread
// copies its own rows (a tile row is one contiguous run of LG elements).
template <int R, int M, int MODE, typename TIn, typename TOut, bool FULL, int LG>
__device__ __forceinline__ void seg_prefetch(const LongArgs& a, const DevLineTables& tin, const LongGeom& gm,
                                             const int it, const int tiles, const int seg0, TIn* sbuf) {
  const int seg = seg0 + it / tiles;
  const int i = threadIdx.x / LG, g = threadIdx.x % LG;
  const int64_t line = (int64_t)(it % tiles) * LG + g;
  if (i < tin.p && line < a.lines) {
    int start = i * M, size = M;
    if (!FULL) partition_of(tin, i, start, size);
    const int64_t es = gm.es;
    const TIn* b = (const TIn*)a.in + long_base(a, gm, line) + (seg_start(a, seg) + R + start) * es;
#pragma unroll
    for (int k = 0; k < M; k++)
      if (FULL || k < size) cp_async<sizeof(TIn)>(sbuf + k * blockDim.x + threadIdx.x, b + k * es);
  }
  cp_async_commit();
}

template <int R, int M, int MODE, typename TIn, typename TOut, bool FULL, int LG>
__global__ void __launch_bounds__(256, 2) long_seg_pipe_kernel(const LongArgs a, const DevLineTables tin,
                                                               const int seg0, const LongGeom gm, const int tiles,
                                                               const int items) {
  extern __shared__ __align__(16) unsigned long long xbuf[];
  const int bd = blockDim.x, g = threadIdx.x % LG;
  TIn* slots = reinterpret_cast<TIn*>(xbuf + (size_t)kCtaXchgSlots * bd);
  CtaXchgT<LG> xch{xbuf, 0, 1, g};  // one exchanger for every item: the buffers keep alternating
  int it = blockIdx.x, buf = 0;
  if (it < items) seg_prefetch<R, M, MODE, TIn, TOut, FULL, LG>(a, tin, gm, it, tiles, seg0, slots);
  for (; it < items; it += gridDim.x, buf ^= 1) {
    const int next = it + gridDim.x;
    if (next < items) {
      seg_prefetch<R, M, MODE, TIn, TOut, FULL, LG>(a, tin, gm, next, tiles, seg0, slots + (size_t)(buf ^ 1) * M * bd);
      cp_async_wait<1>();  // this item's copies are done, the next item's stay in flight
    } else {
      cp_async_wait<0>();
    }
    seg_item<R, M, MODE, TIn, TOut, FULL, LG, CtaXchgT<LG>, true>(a, tin, gm, seg0 + it / tiles,
                                                                  (int64_t)(it % tiles) * LG + g, xch,
                                                                  slots + (size_t)buf * M * bd + threadIdx.x, bd);
  }
}

// ---------------------------------------------------------------- launchers
// Persistent launch of long_seg_pipe_kernel: one CTA per resident slot
// (occupancy x SMs) over the tiles x nseg items of segments seg0..
template <int R, int MODE, typename TIn, typename TOut, bool FULL, int LG>
cudaError_t launch_seg_pipe(const LongArgs& a, const DevLineTables& tin, int seg0, int nseg, const LongGeom& gm,
                            int threads, cudaStream_t s) {
  constexpr int M = 16;
  const int64_t tiles = (a.lines + LG - 1) / LG, items = tiles * nseg;
  if (items > 0x7fffffff || threads > 256) return cudaErrorInvalidValue;
  const size_t smem = (size_t)kCtaXchgSlots * threads * sizeof(unsigned long long) + 2 * (size_t)M * threads * sizeof(TIn);
  auto kern = long_seg_pipe_kernel<R, M, MODE, TIn, TOut, FULL, LG>;
  // per instantiation: the shared-memory opt-in and the occupancy
  static SmemOptIn opt;
  cudaError_t e = opt.ensure(kern, smem);
  if (e != cudaSuccess) return e;
  static OccupancyCache occ;
  int blocks_per_sm = 0;
  e = occ.get(kern, threads, smem, &blocks_per_sm);
  if (e != cudaSuccess) return e;
  if (blocks_per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t want = (int64_t)blocks_per_sm * sm_count();
  const unsigned blocks = (unsigned)(items < want ? items : want);
  kern<<<blocks, threads, smem, s>>>(a, tin, seg0, gm, (int)tiles, (int)items);
  return cudaGetLastError();
}

// y/z tiles: the pipelined kernel for the FP32 modes (load-latency bound
// otherwise); FP64 is bound by its FP64 pipe and runs the plain kernel (the
// pipelined one measured a few per cent slower there).
template <int R, int MODE, typename TIn, typename TOut, bool FULL, int LG>
cudaError_t launch_seg_tiled(const LongArgs& a, const DevLineTables& tin, int seg0, int nseg, const LongGeom& gm,
                             int threads, cudaStream_t s) {
  if constexpr (MODE == kModeF64) {
    const dim3 g((unsigned)((a.lines + LG - 1) / LG), (unsigned)nseg);
    const size_t smem = (size_t)kCtaXchgSlots * threads * sizeof(unsigned long long);
    long_seg_kernel<R, 16, MODE, TIn, TOut, FULL, LG><<<g, threads, smem, s>>>(a, tin, seg0, gm);
    return cudaGetLastError();
  } else {
    return launch_seg_pipe<R, MODE, TIn, TOut, FULL, LG>(a, tin, seg0, nseg, gm, threads, s);
  }
}

cudaError_t launch_long(int mode, int R, bool in64, bool out64, const LongArgs& a, const LongGeom& gm,
                        const DevLineTables& outer,
                        const DevLineTables& inner, const DevLineTables* inner_small, bool full, cudaStream_t s,
                        int* launches) {
  *launches = 0;
  if (a.p > 65535 || a.lines > 0x7fffffff) return cudaErrorInvalidValue;
  const bool tiled = gm.dir != 0;  // y/z lines: kLongLines adjacent lines per CTA
  const int LG = tiled ? kLongLines : 1;
  const unsigned tiles = (unsigned)((a.lines + LG - 1) / LG);
  const dim3 gs(tiles, (unsigned)a.p);
  if (tiled) {
    if (in64) long_ends_kernel<double, kLongLines><<<gs, 128, 0, s>>>(a, gm);
    else long_ends_kernel<float, kLongLines><<<gs, 128, 0, s>>>(a, gm);
  } else {
    const int64_t items = a.lines * a.p;
    if ((items + 7) / 8 > 0x7fffffff) return cudaErrorInvalidValue;
    const unsigned blocks = (unsigned)((items + 7) / 8);
    if (in64) long_ends_warp_kernel<double><<<blocks, 256, 0, s>>>(a, items);
    else long_ends_warp_kernel<float><<<blocks, 256, 0, s>>>(a, items);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int ithreads = a.p < 1024 ? ((a.p + 31) / 32) * 32 : 1024;
  const size_t ismem = 2 * (size_t)a.p * a.r * sizeof(double);
  {
    static SmemOptIn opt[4];  // one per interface kernel
    const void* ks[4] = {(const void*)long_iface_kernel<double, false>, (const void*)long_iface_kernel<float, false>,
                         (const void*)long_iface_kernel<double, true>, (const void*)long_iface_kernel<float, true>};
    for (int k = 0; k < 4 && e == cudaSuccess; k++) e = opt[k].ensure(ks[k], ismem);
    if (e != cudaSuccess) return e;
  }
  const unsigned nl = (unsigned)a.lines;
  if (tiled) {
    if (in64) long_iface_kernel<double, true><<<nl, ithreads, ismem, s>>>(a, outer, gm);
    else long_iface_kernel<float, true><<<nl, ithreads, ismem, s>>>(a, outer, gm);
  } else {
    if (in64) long_iface_kernel<double, false><<<nl, ithreads, ismem, s>>>(a, outer, gm);
    else long_iface_kernel<float, false><<<nl, ithreads, ismem, s>>>(a, outer, gm);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  *launches = 2;
  // segment launches: the first cbig segments with `inner`, the rest with
  // `inner_small` (segments of two sizes)
  const int nbig = inner_small ? a.cbig : a.p;
  for (int part = 0; part < (inner_small ? 2 : 1); part++) {
    const DevLineTables& tin = part == 0 ? inner : *inner_small;
    const int seg0 = part == 0 ? 0 : nbig, nseg = part == 0 ? nbig : a.p - nbig;
    if (nseg <= 0) continue;
    // x: one warp-multiple of inner partitions; y/z: a tile of lg lines x
    // (inner partitions rounded up), a multiple of 32 threads as well, with
    // lg the widest of 8, 4, 2 lines that keeps the CTA at <= 256 threads
    // (two CTAs per SM at 128 registers: one loads while the other computes)
    int lg = 1;
    if (tiled) {
      lg = kLongLines;
      while (lg > 2 && lg * (((tin.p + 32 / lg - 1) / (32 / lg)) * (32 / lg)) > 256) lg /= 2;
    }
    const int rnd = 32 / lg;
    const int threads = lg > 1 ? lg * (((tin.p + rnd - 1) / rnd) * rnd) : ((tin.p + 31) / 32) * 32;
    if (threads > 512) return cudaErrorInvalidConfiguration;
    const dim3 g((unsigned)((a.lines + lg - 1) / lg), (unsigned)nseg);
    const size_t smem = (size_t)kCtaXchgSlots * threads * sizeof(unsigned long long);
#define CBS_SEGP(MO, RR, TI, TO, LGV)                                                                  \
  (full ? launch_seg_tiled<RR, MO, TI, TO, true, LGV>(a, tin, seg0, nseg, gm, threads, s)              \
        : launch_seg_tiled<RR, MO, TI, TO, false, LGV>(a, tin, seg0, nseg, gm, threads, s))
#define CBS_SEG(MO, RR, TI, TO)                                                                        \
  do {                                                                                                 \
    if (lg == 8) e = CBS_SEGP(MO, RR, TI, TO, 8);                                                      \
    else if (lg == 4) e = CBS_SEGP(MO, RR, TI, TO, 4);                                                 \
    else if (lg == 2) e = CBS_SEGP(MO, RR, TI, TO, 2);                                                 \
    else if (full) long_seg_kernel<RR, 16, MO, TI, TO, true, 1><<<g, threads, smem, s>>>(a, tin, seg0, gm); \
    else long_seg_kernel<RR, 16, MO, TI, TO, false, 1><<<g, threads, smem, s>>>(a, tin, seg0, gm);        \
  } while (0)
    if (mode == kModeRefine) {
      if (R == 1) { if (in64) CBS_SEG(kModeRefine, 1, double, double); else CBS_SEG(kModeRefine, 1, float, double); }
      else { if (in64) CBS_SEG(kModeRefine, 2, double, double); else CBS_SEG(kModeRefine, 2, float, double); }
    } else if (mode == kModeRefineI64) {
      if (R == 1) { if (in64) CBS_SEG(kModeRefineI64, 1, double, double); else CBS_SEG(kModeRefineI64, 1, float, double); }
      else { if (in64) CBS_SEG(kModeRefineI64, 2, double, double); else CBS_SEG(kModeRefineI64, 2, float, double); }
    } else if (mode == kModeF64) {
      if (R == 1) { if (in64) CBS_SEG(kModeF64, 1, double, double); else CBS_SEG(kModeF64, 1, float, double); }
      else { if (in64) CBS_SEG(kModeF64, 2, double, double); else CBS_SEG(kModeF64, 2, float, double); }
    } else {
      if (R == 1) { if (in64) CBS_SEG(kModeF32, 1, double, float); else CBS_SEG(kModeF32, 1, float, float); }
      else { if (in64) CBS_SEG(kModeF32, 2, double, float); else CBS_SEG(kModeF32, 2, float, float); }
    }
#undef CBS_SEG
#undef CBS_SEGP
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ++*launches;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------- no-alloc entry
// Long-line solve whose per-solve scratch (yb, cc, xt) is one library-wide
// array in the device image instead of the plan's own buffer.  It exists for
// callers that must not call cudaMalloc when they solve: applications that
// hand all device memory to their own allocator at start-up, and loops with a
// fixed memory footprint where a late allocation could fail.  Plans that run
// a warp per segment need no scratch at all.
//
// The array is a host-side stand-in in host code: the device address comes
// from cudaGetSymbolAddress in the current context, on every call.  Every
// call shares the array and the previous call's contents stay in it; nothing
// needs to start at zero because every slot is written before it is read
// within a solve.  Calls whose launches overlap on the GPU (different
// streams, or the same plan from several host threads without ordering) race
// on the array.
}  // namespace cbs

namespace {

constexpr size_t kNoAllocScratchDoubles = (size_t)1 << 19;  // 4 MiB

}  // namespace

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

namespace {

// Device address of the array in the current context.  Looked up on every
// call rather than cached: after a device reset the new context maps the
// array at a new address.
cbs_status noalloc_scratch(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess)
    return cbs::set_error(CBS_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
  *out = static_cast<double*>(p);
  return CBS_OK;
}

}  // namespace

extern "C" cbs_status cbs_solve_noalloc(cbs_plan* P, const void* in, void* out, void* stream) {
  using namespace cbs;
  set_launch_count(0);
  if (!P || !in || !out) return set_error(CBS_ERR_INVALID_ARG, "null argument");
  if (in == out) return set_error(CBS_ERR_INVALID_ARG, "out must not alias in");
  if (P->kind != 1) return set_error(CBS_ERR_UNSUPPORTED, "cbs_solve_noalloc runs long-line plans (segments per CTA)");
  const LongArgs& pa = P->largs;
  const cbs_desc& d = P->desc;
  const int mode = d.precision == CBS_FP64 ? kModeF64
                   : d.precision == CBS_FP32 ? kModeF32
                   : d.precision == CBS_FP32_REFINE ? kModeRefine
                                                    : kModeRefineI64;
  if (P->long_warp && P->variant == 0) {  // a warp per segment: no per-solve scratch at all
    LongArgs a = pa;
    a.in = in;
    a.out = out;
    int launches = 0;
    const cudaError_t e = launch_long_warp(mode, P->r, d.in_dtype == CBS_DTYPE_F64, d.out_dtype == CBS_DTYPE_F64, a,
                                           P->dev_inner, a.cbig < a.p ? &P->dev_inner_small : nullptr, P->lwargs,
                                           P->lwifc, (cudaStream_t)stream, &launches);
    if (e != cudaSuccess)
      return set_error(CBS_ERR_CUDA, std::string("long-line kernel launch: ") + cudaGetErrorString(e));
    set_launch_count(launches);
    return CBS_OK;
  }
  const size_t nseg = (size_t)pa.lines * pa.p;
  const size_t need = nseg * 5 * pa.r;
  if (need > kNoAllocScratchDoubles)
    return set_error(CBS_ERR_INVALID_ARG, "cbs_solve_noalloc: lines x segments x 5r = " + std::to_string(need) +
                                              " doubles exceeds the fixed scratch of 524288 (4 MiB)");
  double* scratch = nullptr;
  cbs_status st = noalloc_scratch(&scratch);
  if (st) return st;
  LongArgs a = pa;
  a.in = in;
  a.out = out;
  a.yb = scratch;
  a.cc = scratch + nseg * 2 * a.r;
  a.xt = scratch + nseg * 4 * a.r;
  int launches = 0;
  cudaError_t e = launch_long(mode, P->r, d.in_dtype == CBS_DTYPE_F64, d.out_dtype == CBS_DTYPE_F64, a, P->lgeom,
                              P->dev,
                              P->dev_inner, a.cbig < a.p ? &P->dev_inner_small : nullptr,
                              P->inner_full, (cudaStream_t)stream, &launches);
  if (e != cudaSuccess) return set_error(CBS_ERR_CUDA, std::string("long-line kernel launch: ") + cudaGetErrorString(e));
  set_launch_count(launches);
  return CBS_OK;
}
