// cbs_tma.cuh -- FP32 + refinement line kernel fed by the tensor memory
// accelerator (TMA): one warp per line of 32 partitions, tiles of TL adjacent
// lines moved between HBM and shared memory by cp.async.bulk.tensor.
//
// Same method as the on-chip line kernel (cbs_line.cuh), per line:
//   a1  b = S f (Eq. 1) in double-float from the FP64 field,
//   a2-a4  x0 = A^{-1} b by the partition method in FP32 (Eq. 17, 21, 22;
//       Algorithms 1-4 on the interface system, pre-factorised),
//   a5  one refinement sweep x = x0 + A^{-1}(b - A x0) with the residual
//       evaluated to FP64 accuracy, result written in FP64.
// What differs is how the work is arranged for this GPU:
//   * TMA tiles.  A tile is TL lines x n rows of FP64.  x-lines: a 2-D view
//     (M rows, partitions) of the field, one box per tile.  y/z lines: a 4-D
//     view (x, partition i, row k within the partition, remaining axis) of
//     the strided field, so the box lands in shared memory as [k][i][x] and
//     the lanes of a warp (one line, lane = partition) read distinct banks
//     under the 64-byte (32-byte for 4 lines) swizzle.  Results go back into
//     the same slots and leave by a TMA store of the whole tile.  Two tile
//     buffers per CTA: the next tile's load is in flight while the current
//     one is computed.  No per-thread global loads or stores.
//   * Quantised first solution.  After the first FP32 solve, x0 is rounded
//     to a per-line grid Q = 2^(E - 21) (2^E <= max|x0| < 2^(E+1)), 22 bits
//     relative to the line's largest value.  Sums of two neighbours are then
//     exact in FP32, and the residual b - x0 - alpha (x0_{i-1} + x0_{i+1})
//     needs one error-free two-sum instead of three.  The rounding of x0
//     (<= 2^-22 of the line's largest value) is one more error the
//     refinement removes.
//   * Output without FP64 conversions.  x = x0q + delta is formed as the sum
//     of two doubles built with integer operations in the binade of
//     C = 1.5 2^(E+2): (x0q + C) and (delta - C); one FP64 add per element.
//   * Stencil halo by shuffles of the split values; right-hand side pairs
//     (b_hi, b_lo) parked in the tile's slots during the first solve (fewer
//     live registers, three CTAs of 256 threads per SM).
// Bounded waits only: a TMA load that has not arrived after about one second
// sets CBS_ERR_TIMEOUT in the status word and the CTA returns.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "cbs_line.cuh"

namespace cbs {

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of barrier `bar`; false after `limit_ns` without it.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (int spin = 0; spin < (1 << 26); spin++) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((spin & 255) == 255 && global_ns() - t0 > limit_ns) return false;
  }
  return false;
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap* map, unsigned bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(map), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_4d(unsigned dst, const CUtensorMap* map, unsigned bar, int c0, int c1, int c2,
                                            int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(dst),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, unsigned src, int c0, int c1) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map), "r"(c0), "r"(c1),
               "r"(src)
               : "memory");
}
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, unsigned src, int c0, int c1, int c2, int c3) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(map),
               "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(src)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
template <int N>
__device__ __forceinline__ void bulk_wait() {
  asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

// Byte offset inside a tile buffer after the TMA swizzle of span SW bytes
// (32, 64 or 128): 16-byte unit bits [4, 4 + log2(SW/16)) are XORed with
// address bits [7, 7 + log2(SW/16)).  The buffer is 1024-byte aligned.
template <int SW>
__host__ __device__ constexpr unsigned swz(unsigned off) {
  return off ^ (((off >> 7) & (unsigned)(SW / 16 - 1)) << 4);
}

// Swizzle span of a tile: x-lines have rows of M doubles per partition;
// y/z lines rows of TL doubles (one per line of the tile).
template <int M, bool STRIDED, int TL>
__host__ __device__ constexpr int tma_swizzle() {
  return STRIDED ? TL * 8 : M * 8;
}

constexpr int kTmaMaxLines = 8;  // lines per tile (one warp each)
constexpr int kTmaMaxMsg = 6;    // interface stages with messages (p = 32: at most 5 PCR steps)

// The interface solve of a line of 32 partitions with uniform tridiagonal
// blocks (Toeplitz bands, p a power of two), pre-factorised (Algorithms 1-4,
// Sec. 4): the stages whose couplings exceed rounding in the solve's
// precision, each x~ <- C x~ - KM x~_{i-s} - KP x~_{i+s}, in order; every
// other stage is a uniform scaling x~ <- C x~, and since all lanes scale
// alike these commute with the message stages and are applied at the end as
// one product (folded into the last message stage's blocks when there is
// one).
struct TmaIface {
  int nmsg;
  int s[kTmaMaxMsg];
  float cf[kTmaMaxMsg][3];   // C, KM, KP in FP32
  double cd[kTmaMaxMsg][3];  // in FP64 (interface of the _I64 mode)
  float scalef;
  double scaled;
  // limit of a tile wait (1 s), and the fault injected for tests of the
  // timeout path: 1 = CTA 0 does not issue its first tile load, so its wait
  // for that tile expires (cbs_plan_inject_fault)
  unsigned long long wait_ns;
  int fault;
  // Integer bands: alpha = 1/D with D in 2..6.  The launch then solves
  // A' = D A = (1, D, 1) with right-hand side D b (host-side: stencil
  // weights times D; bulk pivot reciprocals divided by D; the b-hat blocks
  // L~, U~ times D and the interface's final scaling divided by D, so the
  // interface rows need no division), and the residual D b - A' x0q is
  // formed with D x0q + (x0q_{k-1} + x0q_{k+1}) exact in one FMA on a 21-bit
  // grid.
  int ib;
  float dband, invdf;
  double invdd;
};

// ---------------------------------------------------------------- shared memory
// 32-bit shared-space addresses with compile-time offsets.
template <int OFF = 0>
__device__ __forceinline__ double lds_f64(unsigned a) {
  double v;
  asm volatile("ld.shared.f64 %0, [%1+%2];" : "=d"(v) : "r"(a), "n"(OFF));
  return v;
}
template <int OFF = 0>
__device__ __forceinline__ void lds_v2f64(unsigned a, double& x, double& y) {
  asm volatile("ld.shared.v2.f64 {%0, %1}, [%2+%3];" : "=d"(x), "=d"(y) : "r"(a), "n"(OFF));
}
template <int OFF = 0>
__device__ __forceinline__ f32x2 lds_b64(unsigned a) {
  f32x2 v;
  asm volatile("ld.shared.b64 %0, [%1+%2];" : "=l"(v) : "r"(a), "n"(OFF));
  return v;
}
template <int OFF = 0>
__device__ __forceinline__ void lds_v2b64(unsigned a, f32x2& x, f32x2& y) {
  asm volatile("ld.shared.v2.b64 {%0, %1}, [%2+%3];" : "=l"(x), "=l"(y) : "r"(a), "n"(OFF));
}
template <int OFF = 0>
__device__ __forceinline__ void sts_b64(unsigned a, unsigned long long v) {
  asm volatile("st.shared.b64 [%0+%1], %2;" ::"r"(a), "n"(OFF), "l"(v) : "memory");
}
template <int OFF = 0>
__device__ __forceinline__ void sts_v2b64(unsigned a, unsigned long long x, unsigned long long y) {
  asm volatile("st.shared.v2.b64 [%0+%1], {%2, %3};" ::"r"(a), "n"(OFF), "l"(x), "l"(y) : "memory");
}
__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }

// ---------------------------------------------------------------- arithmetic
// FP64 -> FP32 pair (hi = x truncated to 24 bits, lo = the next 23 bits) by
// integer operations, valid for 2^-103 <= |x| < 2^128; `bad` is set for
// values outside 2^-60 <= |x| < 2^100 (zeros included), which send the line
// to the general path.
__device__ __forceinline__ f2 split_tma(double x, unsigned& bad) {
  const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
  bad |= ((hw & 0x7fffffffu) - (963u << 20)) >= (160u << 20) ? 1u : 0u;
  const unsigned F = __funnelshift_l(lw, hw, 3);                                   // (hw << 3) | (lw >> 29)
  const unsigned hb = ((F - 0x40000000u) & 0x7fffffffu) | (hw & 0x80000000u);     // exponent e - 896
  const unsigned SE = (hb & 0xff800000u) - (23u << 23);                            // sign | (e - 919) << 23
  f2 r;
  r.hi = __uint_as_float(hb);
  r.lo = __fsub_rn(__uint_as_float(SE | ((lw >> 6) & 0x7fffffu)), __uint_as_float(SE));
  return r;
}

// a2-a4 for one partition of M rows (lane i of a line of 32 partitions,
// whole-size partitions, tridiagonal Toeplitz bands): on entry v holds b_i,
// on exit x_i.  FP32 bulk; interface system in TI.
template <int M, typename TI>
__device__ __forceinline__ void tma_solve(float (&v)[M], const int i, const DevLineTables& t, const TmaIface& f) {
  constexpr int NB = M - 1;  // bulk rows 1 .. M - 1
  // a2: y = D_i^{-1} b (pre-factorised LU of the bulk block, Eq. 17)
#pragma unroll
  for (int j = 1; j < NB; j++) v[1 + j] -= t.facF[j * 3] * v[j];
#pragma unroll
  for (int j = NB - 1; j >= 0; j--) {
    float s = t.facF[j * 3 + 1] * v[1 + j];
    if (j + 1 < NB) s -= t.facF[j * 3 + 2] * v[2 + j];
    v[1 + j] = s;
  }
  // a3: b-hat_i = b~_i - L~_i y_{i-1}[last] - U~_i y_i[first] (Eq. 21); an
  // FP64 interface widens its inputs with integer operations (the FP64
  // pipe, which also runs conversions, is the bound of that mode)
  const float yp = __shfl_sync(kFull, v[M - 1], (i + 31) & 31);
  auto widen = [](float x) -> TI {
    if constexpr (sizeof(TI) == 8) return f32_to_f64(x);
    else return x;
  };
  TI xt = widen(v[0]);
  xt -= ITab<TI>::Lt(t, 0, 0) * widen(yp);
  xt -= ITab<TI>::Ut(t, 0, 0) * widen(v[1]);
  // a3: interface system (message stages, then the product of the others)
#pragma unroll
  for (int st = 0; st < kTmaMaxMsg; st++) {
    if (st < f.nmsg) {
      const int s = f.s[st];
      const TI xm = __shfl_sync(kFull, xt, (i - s) & 31), xp = __shfl_sync(kFull, xt, (i + s) & 31);
      if constexpr (sizeof(TI) == 8) {
        TI acc = f.cd[st][0] * xt;
        acc -= f.cd[st][1] * xm + f.cd[st][2] * xp;
        xt = acc;
      } else {
        TI acc = f.cf[st][0] * xt;
        acc -= f.cf[st][1] * xm + f.cf[st][2] * xp;
        xt = acc;
      }
    }
  }
  if (f.nmsg == 0) {  // otherwise folded into the last message stage
    if constexpr (sizeof(TI) == 8) xt *= f.scaled;
    else xt *= f.scalef;
  }
  // a4: x_i = y_i - S_i x~_i - R_i x~_{i+1} (Eq. 22)
  const TI xn = __shfl_sync(kFull, xt, (i + 1) & 31);
  float xa, xb;
  if constexpr (sizeof(TI) == 8) {  // narrowed with integer operations (hi + lo of the FP32 split)
    const f2 sa = split_f64(xt), sb = split_f64(xn);
    xa = __fadd_rn(sa.hi, sa.lo);
    xb = __fadd_rn(sb.hi, sb.lo);
  } else {
    xa = xt;
    xb = xn;
  }
#pragma unroll
  for (int j = 0; j < NB; j++) {
    float s = v[1 + j];
    s -= t.srBF[j * 2] * xa;
    s -= t.srBF[j * 2 + 1] * xb;
    v[1 + j] = s;
  }
  v[0] = xa;
}

// ---------------------------------------------------------------- one line
// Warp `g` of the CTA solves line g of the tile in buffer `tb` (shared
// address); lane i owns partition i (rows i M .. i M + M - 1).  On exit the
// line's FP64 results are in the slots its rows came from.  `flag` collects
// CBS_ERR_* conditions of this thread.
//
// Slots.  y/z lines: row k of the thread's partition at tb + k RS + o0 (one
// double).  x-lines: 16-byte unit c (rows 2c, 2c + 1) at (xa ^ (c << 4)).
// While the first solve runs, the slot pairs hold the right-hand side as the
// row pairs (k, k + M/2) the paired arithmetic uses: slot k (x: unit k/2 for
// k even, both pairs k and k + 1) (b_hi[k], b_hi[k + M/2]), slot k + M/2
// (b_lo[k], b_lo[k + M/2]).
template <int M, int KS, typename TIR, bool STRIDED, int TL>
__device__ __forceinline__ void tma_line(const LineArgs& a, const DevLineTables& t, const TmaIface& f,
                                         const unsigned tb, const int g, const int i, int& flag) {
  constexpr int H = M / 2;
  constexpr int KA = KS > 0 ? KS : 1;
  constexpr int SW = tma_swizzle<M, STRIDED, TL>();
  static_assert(M == 8 || M == 16, "8 or 16 rows per partition");
  static_assert(SW == 32 || SW == 64 || SW == 128, "swizzle span");
  static_assert(H % 2 == 0, "rows k, k + 1 share a 16-byte unit");
  const int prev = (i + 31) & 31, next = (i + 1) & 31;
  constexpr unsigned RS = 32u * TL * 8u;  // y/z: bytes between rows k and k + 1 of a partition
  const unsigned ys = tb + (STRIDED ? swz<SW>((unsigned)i * TL * 8u + (unsigned)g * 8u) : 0u);
  const unsigned xrow = (unsigned)(g * 32 + i) * M * 8u;
  const unsigned xa = tb + (STRIDED ? 0u : (xrow | (swz<SW>(xrow) ^ xrow)));
  auto ux = [&](int c) -> unsigned { return xa ^ ((unsigned)c << 4); };  // x-lines: unit c

  // ---- a1: own rows -> FP32 pairs; halo rows from the neighbouring lanes
  float fh[M + KS], fl[M + KS], hhh[KA], hhl[KA];
  auto row = [&](int k) -> double {  // own row k (FP64) from the tile
    if constexpr (STRIDED) return lds_f64(ys + k * RS);
    else {
      double x0, x1;
      lds_v2f64(ux(k / 2), x0, x1);
      return (k & 1) ? x1 : x0;
    }
  };
  // Lines whose values leave [2^-60, 2^100) (zeros included) take a
  // warp-uniform slow path: the line is scaled by a power of two 2^sx that
  // brings its largest |f| to [1, 2) when that largest value is outside the
  // range (exact; the system is linear, so x is scaled back by 2^-sx), and
  // every element is split the general way.  Inside the range the double-
  // float arithmetic keeps its low parts above the FP32 subnormals.
  int sx = 0;
  {
    unsigned bad = 0u;
#pragma unroll
    for (int c = 0; c < H; c++) {  // rows 2c, 2c + 1
      double f0, f1;
      if constexpr (STRIDED) {
        f0 = lds_f64(ys + 2 * c * RS);
        f1 = lds_f64(ys + (2 * c + 1) * RS);
      } else {
        lds_v2f64(ux(c), f0, f1);
      }
      const f2 s0 = split_tma(f0, bad), s1 = split_tma(f1, bad);
      fh[KS + 2 * c] = s0.hi;
      fl[KS + 2 * c] = s0.lo;
      fh[KS + 2 * c + 1] = s1.hi;
      fl[KS + 2 * c + 1] = s1.lo;
    }
    if (__any_sync(kFull, bad)) {
      unsigned mx = 0u;  // largest |f| of the line, as the high word of its bit pattern
#pragma unroll 1
      for (int k = 0; k < M; k++) mx = max(mx, (unsigned)__double2hiint(row(k)) & 0x7fffffffu);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
      const int el = (int)(mx >> 20);  // its biased exponent (0: zero line)
      if (mx != 0u && el != 0x7ff && (el < 963 || el >= 1123)) sx = max(-1022, min(1022, 1023 - el));
      const double sc = __longlong_as_double((long long)(1023 + sx) << 52);  // 2^sx
#pragma unroll
      for (int k = 0; k < M; k++) {
        const f2 s = split_f64(sx ? row(k) * sc : row(k));
        fh[KS + k] = s.hi;
        fl[KS + k] = s.lo;
        if (!(fabsf(s.hi) <= 3.402823466e38f)) flag = CBS_ERR_RANGE;  // inf or nan in the input
      }
    }
  }
#pragma unroll
  for (int q = 0; q < KS; q++) {
    fh[q] = __shfl_sync(kFull, fh[KS + M - KS + q], prev);
    fl[q] = __shfl_sync(kFull, fl[KS + M - KS + q], prev);
    hhh[q] = __shfl_sync(kFull, fh[KS + q], next);
    hhl[q] = __shfl_sync(kFull, fl[KS + q], next);
  }

  // b = sum_q w_q (f_{k+q} - f_{k-q}) in double-float, rows k and k + H per
  // instruction; b_hi also stays in v for the first solve
  float v[M];
  auto win = [&](const float (&w)[M + KS], const float (&hh)[KA], int r) -> float {
    return r < M ? w[KS + (r < M ? r : 0)] : hh[r >= M ? r - M : 0];
  };
  auto b_pair = [&](int k, f32x2& dh, f32x2& dl) {
    if constexpr (KS == 0) {
      dh = pk(fh[k], fh[k + H]);
      dl = pk(fl[k], fl[k + H]);
    } else {
#pragma unroll
      for (int q = 1; q <= KS; q++) {
        const f32x2 uh = pk(win(fh, hhh, k + q), win(fh, hhh, k + H + q));
        const f32x2 ul = pk(win(fl, hhl, k + q), win(fl, hhl, k + H + q));
        f32x2 ds, de;
        two_diff2(uh, pk(fh[KS + k - q], fh[KS + k + H - q]), ds, de);
        const f32x2 dlo = add2(de, sub2(ul, pk(fl[KS + k - q], fl[KS + k + H - q])));
        const f32x2 W = a.wP[q - 1][0], NW = a.wP[q - 1][1], WL = a.wP[q - 1][2];
        const f32x2 pr = mul2(W, ds);
        const f32x2 pen = fma2(NW, ds, pr);  // -(error of pr)
        const f32x2 plo = sub2(fma2(W, dlo, mul2(WL, ds)), pen);
        if (q == 1) {
          dh = pr;
          dl = plo;
        } else {
          f32x2 sh, se;
          two_sum2(dh, pr, sh, se);
          dh = sh;
          dl = add2(dl, add2(se, plo));
        }
      }
    }
  };
  if constexpr (STRIDED) {
#pragma unroll
    for (int k = 0; k < H; k++) {
      f32x2 dh, dl;
      b_pair(k, dh, dl);
      unpk(dh, v[k], v[k + H]);
      sts_b64(ys + k * RS, dh);
      sts_b64(ys + (k + H) * RS, dl);
    }
  } else {
#pragma unroll
    for (int k = 0; k < H; k += 2) {
      f32x2 dh0, dl0, dh1, dl1;
      b_pair(k, dh0, dl0);
      b_pair(k + 1, dh1, dl1);
      unpk(dh0, v[k], v[k + H]);
      unpk(dh1, v[k + 1], v[k + 1 + H]);
      sts_v2b64(ux(k / 2), dh0, dh1);
      sts_v2b64(ux((k + H) / 2), dl0, dl1);
    }
  }

  // ---- a2-a4: x0 = A^{-1} b_hi in FP32
  tma_solve<M, TIR>(v, i, t, f);

  // ---- quantise x0 on the line's grid Q = ulp of C = 1.5 2^(E+2)
  float m = 0.f;
#pragma unroll
  for (int k = 0; k < M; k++) m = fmaxf(m, fabsf(v[k]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
  const unsigned mb = __float_as_uint(m) & 0x7f800000u;  // biased exponent e_b << 23
  const unsigned eb = mb >> 23;
  if (eb > 251u) flag = CBS_ERR_RANGE;  // |x0| >= 2^125 or non-finite
  // grid: 22 bits below 2^(E+1) (integer bands: 21 bits, room for D x + sum)
  const float C = __uint_as_float((mb + ((f.ib ? 3u : 2u) << 23)) | 0x00400000u);
  float xq[M];
  {
    const f32x2 C2 = pk(C, C);
#pragma unroll
    for (int k = 0; k < H; k++) unpk(sub2(add2(pk(v[k], v[k + H]), C2), C2), xq[k], xq[k + H]);
  }

  // ---- a5: residual r = b - x0q - alpha (x0q_{k-1} + x0q_{k+1}), rows k and
  // k + H per instruction
  {
    const float xlo = __shfl_sync(kFull, xq[M - 1], prev), xhi = __shfl_sync(kFull, xq[0], next);
    const float aH = t.bandHi[2], aL = t.bandLo[2];
    const f32x2 AH = pk(aH, aH), NAH = pk(-aH, -aH), NAL = pk(-aL, -aL);
    auto xr = [&](int r) -> float { return r < 0 ? xlo : r >= M ? xhi : xq[r < 0 ? 0 : r >= M ? M - 1 : r]; };
    auto pair = [&](int k, f32x2 bh, f32x2 bl) {
      const f32x2 sg = add2(pk(xr(k - 1), xr(k + H - 1)), pk(xr(k + 1), xr(k + H + 1)));  // exact
      const f32x2 P = mul2(AH, sg);
      const f32x2 NE = fma2(NAH, sg, P);  // P - aH sg = -(error of P)
      f32x2 s, se;
      two_diff2(bh, P, s, se);
      const f32x2 rh = sub2(s, pk(xq[k], xq[k + H]));
      const f32x2 lo = fma2(NAL, sg, add2(add2(se, NE), bl));
      unpk(add2(rh, lo), v[k], v[k + H]);
    };
    // integer bands: r' = (b'_hi - (D x0q + sum)) + b'_lo, the bracket exact
    const f32x2 DB = pk(f.dband, f.dband);
    auto pair_ib = [&](int k, f32x2 bh, f32x2 bl) {
      const f32x2 sg = add2(pk(xr(k - 1), xr(k + H - 1)), pk(xr(k + 1), xr(k + H + 1)));  // exact
      const f32x2 tq = fma2(DB, pk(xq[k], xq[k + H]), sg);                                 // exact
      unpk(add2(sub2(bh, tq), bl), v[k], v[k + H]);
    };
    if (f.ib) {
      if constexpr (STRIDED) {
#pragma unroll
        for (int k = 0; k < H; k++) pair_ib(k, lds_b64(ys + k * RS), lds_b64(ys + (k + H) * RS));
      } else {
#pragma unroll
        for (int k = 0; k < H; k += 2) {
          f32x2 bh0, bh1, bl0, bl1;
          lds_v2b64(ux(k / 2), bh0, bh1);
          lds_v2b64(ux((k + H) / 2), bl0, bl1);
          pair_ib(k, bh0, bl0);
          pair_ib(k + 1, bh1, bl1);
        }
      }
    } else {
      if constexpr (STRIDED) {
#pragma unroll
        for (int k = 0; k < H; k++) pair(k, lds_b64(ys + k * RS), lds_b64(ys + (k + H) * RS));
      } else {
#pragma unroll
        for (int k = 0; k < H; k += 2) {
          f32x2 bh0, bh1, bl0, bl1;
          lds_v2b64(ux(k / 2), bh0, bh1);
          lds_v2b64(ux((k + H) / 2), bl0, bl1);
          pair(k, bh0, bl0);
          pair(k + 1, bh1, bl1);
        }
      }
    }
  }
  tma_solve<M, TIR>(v, i, t, f);

  // ---- x = x0q + delta in FP64, one FP64 add per element (integer
  // widening: exact for normal values; a zero gives below 2^-126, under
  // 2^-50 of the line's largest value when eb >= 51).  Lines below that
  // (zero lines included) widen exactly.
  if (eb >= 51u) {
    if constexpr (STRIDED) {
#pragma unroll
      for (int k = 0; k < M; k++) sts_b64(ys + k * RS, dbits(f32_to_f64_nz(xq[k]) + f32_to_f64_nz(v[k])));
    } else {
#pragma unroll
      for (int c = 0; c < H; c++)
        sts_v2b64(ux(c), dbits(f32_to_f64_nz(xq[2 * c]) + f32_to_f64_nz(v[2 * c])),
                  dbits(f32_to_f64_nz(xq[2 * c + 1]) + f32_to_f64_nz(v[2 * c + 1])));
    }
  } else {
    if constexpr (STRIDED) {
#pragma unroll
      for (int k = 0; k < M; k++) sts_b64(ys + k * RS, dbits(f32_to_f64(xq[k]) + f32_to_f64(v[k])));
    } else {
#pragma unroll
      for (int c = 0; c < H; c++)
        sts_v2b64(ux(c), dbits(f32_to_f64(xq[2 * c]) + f32_to_f64(v[2 * c])),
                  dbits(f32_to_f64(xq[2 * c + 1]) + f32_to_f64(v[2 * c + 1])));
    }
  }
  if (sx) {  // rescaled line: x = x' 2^-sx (a loop, so it is never predicated into the common path)
    const double us = __longlong_as_double((long long)(1023 - sx) << 52);
#pragma unroll 1
    for (int k = 0; k < M; k++) {
      const unsigned adr = STRIDED ? ys + k * RS : (ux(k / 2) + (k & 1) * 8u);
      sts_b64(adr, dbits(lds_f64(adr) * us));
    }
  }
}

// ---------------------------------------------------------------- kernel
// Tile shapes: TL lines per tile (4, 8 or 16), solved by W warps of which
// each takes TL / W lines; NBUF tile buffers per CTA (2: the next tile's load
// is in flight while the current tile is computed; 1: overlap across the
// CTAs of an SM instead).
template <int M, int TL, int W, int NBUF>
__host__ __device__ constexpr int tma_ctas_per_sm() {
  // shared memory: NBUF buffers of TL lines x 32 partitions x M rows x 8 bytes;
  // registers: up to 80 per thread
  return (int)((200u * 1024u) / (NBUF * (unsigned)TL * 32u * M * 8u + 1040u)) <
                 (int)(65536u / (80u * 32u * (unsigned)W))
             ? (int)((200u * 1024u) / (NBUF * (unsigned)TL * 32u * M * 8u + 1040u))
             : (int)(65536u / (80u * 32u * (unsigned)W));
}

// Persistent: CTA b walks tiles b, b + gridDim.x, ...  x-lines: tile j =
// lines j TL .. j TL + TL - 1 (map coordinates (0, j TL 32)).  y/z lines:
// tile j = x positions (j % gx) TL .. + TL - 1 at the remaining coordinate
// j / gx (map coordinates (x0, 0, 0, j / gx)).  Shared memory: NBUF tile
// buffers of TL n doubles (1024-byte aligned) and NBUF mbarriers.
template <int M, int KS, typename TIR, bool STRIDED, int TL, int W, int NBUF>
__global__ void __launch_bounds__(W * 32, tma_ctas_per_sm<M, TL, W, NBUF>())
    refine_tma_kernel(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout,
                      const LineArgs a, const DevLineTables t, const TmaIface f, const int gx, const int ntiles) {
  static_assert(NBUF == 1 || NBUF == 2, "one or two tile buffers");
  static_assert(TL % W == 0, "whole lines per warp");
  constexpr int LPW = TL / W;
  extern __shared__ unsigned char smem_raw[];
  constexpr unsigned TB = (unsigned)TL * 32u * M * 8u;  // bytes per tile buffer
  unsigned char* base = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  const unsigned bar0 = smem_addr(base + NBUF * TB), bar1 = bar0 + 8;
  const int w = threadIdx.x >> 5, i = threadIdx.x & 31;
  const bool leader = threadIdx.x == 0;

  auto load = [&](int tile, int b) {
    const unsigned bar = b ? bar1 : bar0;
    mbar_expect_tx(bar, TB);
    const unsigned dst = smem_addr(base) + (unsigned)b * TB;
    if constexpr (STRIDED) tma_load_4d(dst, &tin, bar, (tile % gx) * TL, 0, 0, tile / gx);
    else tma_load_2d(dst, &tin, bar, 0, tile * TL * 32);
  };
  if (leader) {
    mbar_init(bar0, 1);
    if (NBUF == 2) mbar_init(bar1, 1);
    mbar_fence_init();
  }
  __syncthreads();
  int tile = blockIdx.x;
  if (leader) {
    if (tile < ntiles && !(f.fault == 1 && blockIdx.x == 0)) load(tile, 0);
    if (NBUF == 2 && tile + (int)gridDim.x < ntiles) load(tile + gridDim.x, 1);
  }
  int flag = 0;
  for (int it = 0; tile < ntiles; it++, tile += gridDim.x) {
    const int b = NBUF == 2 ? (it & 1) : 0;
    const unsigned parity = (unsigned)(NBUF == 2 ? (it >> 1) : it) & 1u;
    const bool arrived = mbar_wait_bounded(b ? bar1 : bar0, parity, f.wait_ns);
    const int nl = STRIDED ? (int)min((int64_t)TL, a.nx - (int64_t)(tile % gx) * TL)
                           : (int)min((int64_t)TL, a.nlines - (int64_t)tile * TL);
#pragma unroll 1
    for (int l = 0; l < LPW; l++) {
      const int g = w + l * W;
      if (arrived && g < nl) tma_line<M, KS, TIR, STRIDED, TL>(a, t, f, smem_addr(base) + b * TB, g, i, flag);
    }
    fence_proxy_async();  // this thread's slot writes -> visible to the TMA store
    if (__syncthreads_or(!arrived)) {
      if (leader) {
        atomicExch(a.status, CBS_ERR_TIMEOUT);
        // give the overdue load (and the next one, if issued) another bounded
        // wait to land before the CTA's shared memory is released
        if (!(f.fault == 1 && blockIdx.x == 0 && it == 0)) mbar_wait_bounded(b ? bar1 : bar0, parity, f.wait_ns);
        if (NBUF == 2 && tile + (int)gridDim.x < ntiles)
          mbar_wait_bounded(b ? bar0 : bar1, (unsigned)((it + 1) >> 1) & 1u, f.wait_ns);
      }
      break;
    }
    if (leader) {
      const unsigned src = smem_addr(base) + (unsigned)b * TB;
      if constexpr (STRIDED) tma_store_4d(&tout, src, (tile % gx) * TL, 0, 0, tile / gx);
      else tma_store_2d(&tout, src, 0, tile * TL * 32);
      bulk_commit();
      const int nt = tile + NBUF * (int)gridDim.x;
      if (nt < ntiles) {
        bulk_wait_read<0>();  // the store has read this buffer
        load(nt, b);
      }
    }
  }
  if (flag) atomicExch(a.status, flag);
  if (leader) bulk_wait<0>();  // every store of this CTA has completed
}

}  // namespace cbs
