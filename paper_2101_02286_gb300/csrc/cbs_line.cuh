// cbs_line.cuh -- on-chip line kernel: one warp lane per partition.
//
// Each line (one independent cyclic system) is handled by a group of `pw`
// lanes of one warp; lane i owns partition i (rows start_i .. start_i+m_i-1,
// Sec. 3, Fig. 3): its first r rows are the interface unknowns x~_i, the rest
// the bulk block D_i.  Per line the kernel performs, without leaving the SM:
//   a1  the periodic central stencil b = S f (Eq. 1), from a register window;
//   a2  y_i = D_i^{-1} b_i by banded forward/backward elimination with the
//       plan's pre-factorised LU of D_i (Eq. 17), in registers;
//   a3  b-hat_i = b~_i - L~_i y_{i-1} - U~_i y_i (Eq. 21) and the cyclic
//       block-PCR with detach/reattach on the interface system
//       (Algorithms 1-4) using warp shuffles (or shared memory when the
//       partitions of a line span several warps), with the W^{-1} products
//       precomputed per stage (Sec. 4), in the precision of the solve;
//   a4  x_i = y_i - S_i x~_i - R_i x~_{i+1} (Eq. 22).
// The FP32 + refinement mode runs a2-a4 in FP32 twice (or three times) and
// evaluates the residual b - A x to FP64 accuracy with error-free FP32
// transformations (two-sum / two-product), because the FP64 pipe of this
// GPU issues ~1/69 as many operations per clock as the FP32 pipe.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "cbs_internal.h"

namespace cbs {

constexpr unsigned kFull = 0xffffffffu;

// kModeRefineI64: the refinement with the interface system of every FP32
// solve in FP64.
enum Mode { kModeF64 = 0, kModeF32 = 1, kModeRefine = 2, kModeRefineI64 = 3 };
__host__ __device__ constexpr bool refine_mode(int m) { return m == kModeRefine || m == kModeRefineI64; }

struct LineArgs {
  const void* in;
  void* out;
  int64_t nx, ny, nz;
  int64_t nlines;
  int dir;
  int K;                 // stencil terms actually used (<= template KS)
  int sweeps;            // refinement sweeps (refinement modes)
  // staggered stencils (kernels compiled with ST = 1): stag_shift = s moves the
  // window up by s rows; stag_sum = 1 adds the two points of a term
  // (interpolation), 0 subtracts them (derivative).  Two shorts fill the
  // alignment gap before w, so the argument block keeps its layout.
  short stag_shift, stag_sum;
  double w[kMaxRhsTerms];              // c_q / (2 q h)
  float wHi[kMaxRhsTerms], wLo[kMaxRhsTerms];
  // the same split weights as pairs for the two-rows-per-instruction
  // arithmetic: [q][0] = (wHi, wHi), [q][1] = (-wHi, -wHi), [q][2] = (wLo, wLo)
  unsigned long long wP[kMaxRhsTerms][3];
  int* status;
};

// Host: refresh the paired weights after wHi / wLo changed.
inline void pack_weights(LineArgs& a) {
  for (int q = 0; q < kMaxRhsTerms; q++) {
    const float v[3] = {a.wHi[q], -a.wHi[q], a.wLo[q]};
    for (int m = 0; m < 3; m++) {
      unsigned u;
      static_assert(sizeof(u) == sizeof(float), "float size");
      __builtin_memcpy(&u, &v[m], sizeof(u));
      a.wP[q][m] = ((unsigned long long)u << 32) | u;
    }
  }
}

// Field geometry: (nx, ny, nz) with x contiguous, lines along `dir`.
struct Geom {
  int64_t nx, ny;
  int dir;
};

// ---------------------------------------------------------------- helpers
template <typename A>
__device__ __forceinline__ int64_t line_base(const A& a, int64_t L, int64_t& es) {
  if (a.dir == 0) {
    es = 1;
    return L * a.nx;
  }
  const int64_t x = L % a.nx, o = L / a.nx;
  if (a.dir == 1) {
    es = a.nx;
    return x + a.nx * a.ny * o;
  }
  es = a.nx * a.ny;
  return x + a.nx * o;
}

template <typename T> __device__ __forceinline__ T ld_in(const T* p) { return __ldg(p); }

template <typename T> struct Tab;
template <> struct Tab<double> {
  static __device__ __forceinline__ double fac(const DevLineTables& t, int k) { return t.fac[k]; }
  static __device__ __forceinline__ double sr(const DevLineTables& t, bool big, int k) {
    return big ? t.srB[k] : t.srS[k];
  }
};
template <> struct Tab<float> {
  static __device__ __forceinline__ float fac(const DevLineTables& t, int k) { return t.facF[k]; }
  static __device__ __forceinline__ float sr(const DevLineTables& t, bool big, int k) {
    return big ? t.srBF[k] : t.srSF[k];
  }
};

template <typename TI> struct ITab;
template <> struct ITab<double> {
  static __device__ __forceinline__ double coef(const DevLineTables& t, int k) { return __ldg(t.coef + k); }
  static __device__ __forceinline__ double ucoef(const DevLineTables& t, int st, int k) { return t.ucoef[st][k]; }
  static __device__ __forceinline__ double Lt(const DevLineTables& t, int q, int e) { return t.Lt[q][e]; }
  static __device__ __forceinline__ double Ut(const DevLineTables& t, int q, int e) { return t.Ut[q][e]; }
};
template <> struct ITab<float> {
  static __device__ __forceinline__ float coef(const DevLineTables& t, int k) { return __ldg(t.coefF + k); }
  static __device__ __forceinline__ float ucoef(const DevLineTables& t, int st, int k) { return t.ucoefF[st][k]; }
  static __device__ __forceinline__ float Lt(const DevLineTables& t, int q, int e) { return t.LtF[q][e]; }
  static __device__ __forceinline__ float Ut(const DevLineTables& t, int q, int e) { return t.UtF[q][e]; }
};

// Error-free transformations on FP32 (Knuth two-sum, FMA two-product).
struct f2 {
  float hi, lo;
};
__device__ __forceinline__ f2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ f2 two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ f2 fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// ---------------------------------------------------------------- paired FP32
// Two FP32 lanes per instruction (add/sub/mul/fma .f32x2, round to nearest,
// no contraction): the error-free transformations of two rows at once, bit
// for bit the same results as the scalar forms above.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk(float a, float b) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void unpk(f32x2 v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
// s + e = a + b exactly (two-sum) and a - b exactly (two-sum of a and -b)
__device__ __forceinline__ void two_sum2(f32x2 a, f32x2 b, f32x2& s, f32x2& e) {
  s = add2(a, b);
  const f32x2 bb = sub2(s, a);
  e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
__device__ __forceinline__ void two_diff2(f32x2 a, f32x2 b, f32x2& s, f32x2& e) {
  s = sub2(a, b);
  const f32x2 bb = sub2(s, a);
  e = sub2(sub2(a, sub2(s, bb)), add2(b, bb));
}
// FP64 <-> FP32-pair conversions with integer operations.  On this GPU the
// f32<->f64 conversion instructions and every FP64 add issue on the FP64
// pipe (~1/69 of the FP32 rate), so the FP32 paths build the bit patterns
// themselves and keep the FP64 pipe for nothing but the rare special values.
//
// No FP64 instruction is issued by these helpers, not even for special
// values: a rarely taken FP64 slow path gets if-converted into predicated
// FP64 instructions that are issued for every element.  The FP32 modes work
// in the FP32 range: magnitudes below 2^-126 are flushed to zero (below
// 2^-103 the low part is dropped), magnitudes of 2^128 and more become inf.
//
// split_f64: hi = x truncated to 24 significant bits, lo = the next 23 bits
// (|x - hi - lo| <= 2^-46 |x| for 2^-103 <= |x| < 2^128).
__device__ __forceinline__ f2 split_f64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const unsigned e = (hw >> 20) & 0x7ffu;
  const unsigned sign = hw & 0x80000000u;
  const unsigned m23 = ((hw & 0xfffffu) << 3) | (lw >> 29);
  if (e - 920u < 231u) {
    const float hi = __uint_as_float(sign | ((e - 896u) << 23) | m23);
    const unsigned E = (e - 919u) << 23;
    const float lo = __fsub_rn(__uint_as_float(sign | E | ((lw & 0x1fffffffu) >> 6)), __uint_as_float(sign | E));
    return {hi, lo};
  }
  unsigned hb;
  if (e - 897u < 23u) hb = sign | ((e - 896u) << 23) | m23;          // 2^-126 <= |x| < 2^-103
  else if (e < 897u) hb = sign;                                        // flushed to +-0
  else if (e == 0x7ffu && ((hw & 0xfffffu) | lw)) hb = 0x7fc00000u;    // nan
  else hb = sign | 0x7f800000u;                                        // inf / overflow
  return {__uint_as_float(hb), 0.f};
}
// Fast path of split_f64 alone, for 2^-103 <= |x| < 2^128: the same pair in
// fewer integer operations (the float's exponent field is the double's low 8
// exponent bits minus 128, taken from a funnel shift of the two words).
// Returns nonzero when x is outside that range (zero, tiny, huge, inf, nan);
// the pair is then meaningless and split_f64 must be used instead.
__device__ __forceinline__ unsigned split_fast(double x, f2& r) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const unsigned e = (hw >> 20) & 0x7ffu;
  const unsigned F = __funnelshift_l(lw, hw, 3);  // (hw << 3) | (lw >> 29)
  const unsigned sign = hw & 0x80000000u;
  r.hi = __uint_as_float(((F - 0x40000000u) & 0x7fffffffu) | sign);
  const unsigned SE = sign | ((e - 919u) << 23);
  r.lo = __fsub_rn(__uint_as_float(SE | ((lw >> 6) & 0x7fffffu)), __uint_as_float(SE));
  return (e - 920u) >= 231u ? 1u : 0u;
}

// FP32 -> FP64 bit pattern (exact for every float).
__device__ __forceinline__ double f32_to_f64(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu, sign = u & 0x80000000u;
  unsigned hw, lw;
  if (e - 1u < 254u) {
    hw = sign | ((e + 896u) << 20) | (m >> 3);
    lw = m << 29;
  } else if (e == 0u) {
    if (m == 0u) {
      hw = sign;
      lw = 0u;
    } else {  // subnormal: m * 2^-149 with its top bit at position k
      const unsigned k = 31u - (unsigned)__clz(m);
      const unsigned f = (m << (23u - k)) & 0x7fffffu;
      hw = sign | ((k + 874u) << 20) | (f >> 3);
      lw = f << 29;
    }
  } else {  // inf / nan
    hw = sign | 0x7ff00000u | (m >> 3);
    lw = m << 29;
  }
  return __hiloint2double((int)hw, (int)lw);
}
// FP32 -> FP64 for normal numbers and zero only (5 integer operations plus
// a zero test); subnormal FP32 inputs become zero, inf/nan are not handled.
// Used for the refinement's output, whose values are normal or zero.
__device__ __forceinline__ double f32_to_f64_normal(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned mag = u & 0x7fffffffu;
  unsigned hw = ((mag >> 3) + 0x38000000u) | (u & 0x80000000u);
  unsigned lw = u << 29;
  if (mag < 0x00800000u) {  // zero (or subnormal): signed zero
    hw = u & 0x80000000u;
    lw = 0u;
  }
  return __hiloint2double((int)hw, (int)lw);
}

// FP64 value of a float by integer operations: exact for normal values; a
// zero or subnormal input gives a value of magnitude below 2^-126.
__device__ __forceinline__ double f32_to_f64_nz(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned hw = (((u >> 3) & 0x0fffffffu) + 0x38000000u) | (u & 0x80000000u);
  return __hiloint2double((int)hw, (int)(u << 29));
}

// The double at or toward zero from hi + lo (exact when the pair spans <= 53
// bits) for |lo| <= ulp(hi) as produced by two_sum; integer arithmetic on the
// 53-bit significand.  Outside the normal FP32 range the result is hi alone.
__device__ __forceinline__ double df_to_double(float hi, float lo) {
  const unsigned uh = __float_as_uint(hi), ul = __float_as_uint(lo);
  const unsigned eh = (uh >> 23) & 0xffu, el = (ul >> 23) & 0xffu;
  if ((ul << 1) != 0u && eh - 1u < 253u && el - 1u < 253u && eh >= el + 24u) {
    long long M = (long long)((uh & 0x7fffffu) | 0x800000u) << 29;  // bit 52 = leading one
    const long long Ml = (long long)((ul & 0x7fffffu) | 0x800000u);
    const unsigned d = eh - el;                                        // >= 24
    const long long add = (d <= 29u) ? (Ml << (29u - d)) : (Ml >> (d - 29u));
    M += ((uh ^ ul) & 0x80000000u) ? -add : add;
    long long E = (long long)eh + 896;
    if (M < (1ll << 52)) {  // hi was a power of two and lo pulled it below
      M <<= 1;
      E -= 1;
    }
    const unsigned long long bits = ((unsigned long long)(uh & 0x80000000u) << 32) |
                                    ((unsigned long long)E << 52) | ((unsigned long long)M & ((1ull << 52) - 1));
    return __longlong_as_double((long long)bits);
  }
  return f32_to_f64(hi);
}

// Element conversions used by the staging and the kernels (no FP64-pipe
// conversion instructions on the FP32 paths).
template <typename To, typename From> struct Conv {
  static __device__ __forceinline__ To f(From x) { return (To)x; }
};
template <> struct Conv<double, float> {
  static __device__ __forceinline__ double f(float x) { return f32_to_f64(x); }
};
template <> struct Conv<float, double> {
  static __device__ __forceinline__ float f(double x) {
    const f2 s = split_f64(x);
    return __fadd_rn(s.hi, s.lo);
  }
};
template <typename To, typename From> __device__ __forceinline__ To conv(From x) { return Conv<To, From>::f(x); }

// c ? a : b through an explicit PTX select, so that choosing one register
// out of an unrolled array by a runtime index never becomes an indexed
// (local-memory) access.
__device__ __forceinline__ double sel(bool c, double a, double b) {
  double r;
  asm("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %3, 0;\n\tselp.f64 %0, %1, %2, p;\n\t}"
      : "=d"(r) : "d"(a), "d"(b), "r"((int)c));
  return r;
}
__device__ __forceinline__ float sel(bool c, float a, float b) {
  float r;
  asm("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %3, 0;\n\tselp.f32 %0, %1, %2, p;\n\t}"
      : "=f"(r) : "f"(a), "f"(b), "r"((int)c));
  return r;
}

// sel with a compile-time switch: PLAIN (partition sizes known at compile
// time, so conditions fold away) uses the C++ conditional.
template <bool PLAIN, typename T>
__device__ __forceinline__ T sel2(bool c, T a, T b) {
  if constexpr (PLAIN) return c ? a : b;
  else return sel(c, a, b);
}

// Partition of lane i (first count_big partitions have rows_big rows).
__device__ __forceinline__ void partition_of(const DevLineTables& t, int i, int& start, int& size) {
  if (i < t.count_big) {
    start = i * t.rows_big;
    size = t.rows_big;
  } else {
    start = t.count_big * t.rows_big + (i - t.count_big) * t.rows_small;
    size = t.rows_small;
  }
}

// Residual r = b - A x for whole-size partitions of a symmetric band with
// unit diagonal (the Toeplitz plans): r_k = b_k - x_k - sum_q a_q (x_{k-q} +
// x_{k+q}); each x-pair sum and band product is formed exactly (two-sum,
// two-product), the unit diagonal needs no product.  Same accuracy as
// residual_df with fewer operations.
template <int R, int M, bool XLO, typename X>
__device__ __forceinline__ void residual_sym(const float (&bh)[M], const float (&bl)[M], const float (&xh)[M],
                                             const float (&xl)[M], float (&res)[M], const int i,
                                             const DevLineTables& t, X& xch) {
  const int p = t.p;
  const int prev = (i == 0) ? p - 1 : i - 1;
  const int next = (i + 1 >= p) ? 0 : i + 1;
  float ph[R], pl[R], nh[R], nl[R];  // last R rows of the previous partition, first R of the next
#pragma unroll
  for (int e = 0; e < R; e++) {
    xch.get_two(xh[M - R + e], prev, xh[e], next, ph[e], nh[e]);
    pl[e] = nl[e] = 0.f;
    if (XLO) xch.get_two(xl[M - R + e], prev, xl[e], next, pl[e], nl[e]);
    if (!t.cyclic) {
      if (i == 0) ph[e] = pl[e] = 0.f;
      if (i + 1 >= p) nh[e] = nl[e] = 0.f;
    }
  }
#pragma unroll
  for (int k = 0; k < M; k++) {
    const f2 s0 = two_sum(bh[k], -xh[k]);
    float ah = s0.hi;
    float al = bl[k] + s0.lo;
    if (XLO) al -= xl[k];
#pragma unroll
    for (int q = 1; q <= R; q++) {
      const float mh = (k - q >= 0) ? xh[(k - q >= 0) ? k - q : 0] : ph[(k - q >= 0) ? 0 : R + k - q];
      const float uh = (k + q < M) ? xh[(k + q < M) ? k + q : 0] : nh[(k + q < M) ? 0 : k + q - M];
      const f2 sx = two_sum(mh, uh);
      const float aH = t.bandHi[R + q], aL = t.bandLo[R + q];
      const f2 pr = two_prod(aH, sx.hi);
      const f2 s1 = two_sum(ah, -pr.hi);
      ah = s1.hi;
      float lo = s1.lo - pr.lo - __fmaf_rn(aH, sx.lo, aL * sx.hi);
      if (XLO) {
        const float ml = (k - q >= 0) ? xl[(k - q >= 0) ? k - q : 0] : pl[(k - q >= 0) ? 0 : R + k - q];
        const float ul = (k + q < M) ? xl[(k + q < M) ? k + q : 0] : nl[(k + q < M) ? 0 : k + q - M];
        lo -= aH * (ml + ul);
      }
      al += lo;
    }
    res[k] = ah + al;
  }
}

// Window row r in [-KS, M + KS) of a partition: rows below M from the window
// w (w[KS + r]), the rest from the upper halo hh (r compile-time).
template <int M, int KS, int KA>
__device__ __forceinline__ float win_row(const float (&w)[M + KS], const float (&hh)[KA], int r) {
  return (r < M) ? w[(r < M) ? KS + r : 0] : hh[(r >= M) ? r - M : 0];
}

// x at row offset r in [-R, M + R) of a partition: its own rows, the last R
// rows of the previous partition (lo) or the first R of the next (hi); r is a
// compile-time constant after unrolling.
template <int R, int M>
__device__ __forceinline__ float row_at(const float (&x)[M], const float (&lo)[R], const float (&hi)[R], int r) {
  return (r < 0) ? lo[(r < 0) ? R + r : 0] : (r >= M) ? hi[(r >= M) ? r - M : 0] : x[(r >= 0 && r < M) ? r : 0];
}

// residual_sym with two rows per instruction (M even); same results.
template <int R, int M, bool XLO, typename X>
__device__ __forceinline__ void residual_sym2(const float (&bh)[M], const float (&bl)[M], const float (&xh)[M],
                                              const float (&xl)[M], float (&res)[M], const int i,
                                              const DevLineTables& t, X& xch) {
  static_assert(M % 2 == 0, "paired rows");
  const int p = t.p;
  const int prev = (i == 0) ? p - 1 : i - 1;
  const int next = (i + 1 >= p) ? 0 : i + 1;
  float ph[R], pl[R], nh[R], nl[R];
#pragma unroll
  for (int e = 0; e < R; e++) {
    xch.get_two(xh[M - R + e], prev, xh[e], next, ph[e], nh[e]);
    pl[e] = nl[e] = 0.f;
    if (XLO) xch.get_two(xl[M - R + e], prev, xl[e], next, pl[e], nl[e]);
    if (!t.cyclic) {
      if (i == 0) ph[e] = pl[e] = 0.f;
      if (i + 1 >= p) nh[e] = nl[e] = 0.f;
    }
  }
  // rows j and j + M/2 share an instruction, so a neighbour pair (j +- q,
  // j + M/2 +- q) is again a pair of the same layout except at the ends
  constexpr int H = M / 2;
#pragma unroll
  for (int k = 0; k < H; k++) {
    f32x2 ah, ae;
    two_diff2(pk(bh[k], bh[k + H]), pk(xh[k], xh[k + H]), ah, ae);
    f32x2 al = add2(pk(bl[k], bl[k + H]), ae);
    if (XLO) al = sub2(al, pk(xl[k], xl[k + H]));
#pragma unroll
    for (int q = 1; q <= R; q++) {
      const f32x2 mh = pk(row_at<R, M>(xh, ph, nh, k - q), row_at<R, M>(xh, ph, nh, k + H - q));
      const f32x2 uh = pk(row_at<R, M>(xh, ph, nh, k + q), row_at<R, M>(xh, ph, nh, k + H + q));
      f32x2 sxh, sxe;
      two_sum2(mh, uh, sxh, sxe);
      const float aH = t.bandHi[R + q], aL = t.bandLo[R + q];
      const f32x2 AH = pk(aH, aH), NAH = pk(-aH, -aH), AL = pk(aL, aL);
      const f32x2 P = mul2(AH, sxh);
      const f32x2 Pen = fma2(NAH, sxh, P);  // -(error of P)
      f32x2 e1;
      two_diff2(ah, P, ah, e1);
      f32x2 lo = sub2(add2(e1, Pen), fma2(AH, sxe, mul2(AL, sxh)));
      if (XLO) {
        const f32x2 ml = pk(row_at<R, M>(xl, pl, nl, k - q), row_at<R, M>(xl, pl, nl, k + H - q));
        const f32x2 ul = pk(row_at<R, M>(xl, pl, nl, k + q), row_at<R, M>(xl, pl, nl, k + H + q));
        lo = sub2(lo, mul2(AH, add2(ml, ul)));
      }
      al = add2(al, lo);
    }
    unpk(add2(ah, al), res[k], res[k + H]);
  }
}

// ------------------------------------------------- interface messages
// The paper's sendToPartition / getFromPartition (Algorithms 1-4): value of
// `v` held by partition `src`.  Within a line group of a warp the message is
// a shuffle; when the partitions of one system span a whole CTA it goes
// through a double-buffered shared-memory slot (one barrier per message; all
// threads of the CTA must exchange in lock step).
// get2: the value v of partitions a and b (one message round);
// get_two: va of partition a and vb of partition b (one message round).
struct WarpXchg {
  int pw;
  template <typename V>
  __device__ __forceinline__ V get(V v, int src) {
    return __shfl_sync(kFull, v, src, pw);
  }
  template <typename V>
  __device__ __forceinline__ void get2(V v, int a, int b, V& ra, V& rb) {
    ra = __shfl_sync(kFull, v, a, pw);
    rb = __shfl_sync(kFull, v, b, pw);
  }
  template <typename V>
  __device__ __forceinline__ void get_two(V va, int a, V vb, int b, V& ra, V& rb) {
    ra = __shfl_sync(kFull, va, a, pw);
    rb = __shfl_sync(kFull, vb, b, pw);
  }
};
constexpr int kCtaXchgSlots = 4;  // 64-bit slots per thread: 2 buffers x 2 values
// STRIDE > 0: compile-time stride (the `stride` member is then unused).
template <int STRIDE = 0>
struct CtaXchgT {
  unsigned long long* buf;  // kCtaXchgSlots * blockDim.x slots
  int flip;
  int stride = 1, offset = 0;  // partition src lives in thread src * stride + offset
  __device__ __forceinline__ int thread_of(int src) const { return (STRIDE > 0 ? src * STRIDE : src * stride) + offset; }
  template <typename V>
  static __device__ __forceinline__ unsigned long long bits(V v) {
    if constexpr (sizeof(V) == 8) return (unsigned long long)__double_as_longlong((double)v);
    else return (unsigned long long)__float_as_uint((float)v);
  }
  template <typename V>
  static __device__ __forceinline__ V value(unsigned long long u) {
    if constexpr (sizeof(V) == 8) return (V)__longlong_as_double((long long)u);
    else return (V)__uint_as_float((unsigned)u);
  }
  // the buffer of this round (alternating, so one barrier per round suffices)
  __device__ __forceinline__ unsigned long long* round() {
    unsigned long long* b = buf + flip * 2 * blockDim.x;
    flip ^= 1;
    return b;
  }
  template <typename V>
  __device__ __forceinline__ V get(V v, int src) {
    unsigned long long* b = round();
    b[threadIdx.x] = bits(v);
    __syncthreads();
    return value<V>(b[thread_of(src)]);
  }
  template <typename V>
  __device__ __forceinline__ void get2(V v, int a, int b_, V& ra, V& rb) {
    unsigned long long* b = round();
    b[threadIdx.x] = bits(v);
    __syncthreads();
    ra = value<V>(b[thread_of(a)]);
    rb = value<V>(b[thread_of(b_)]);
  }
  template <typename V>
  __device__ __forceinline__ void get_two(V va, int a, V vb, int b_, V& ra, V& rb) {
    unsigned long long* b = round();
    const unsigned n = blockDim.x;
    b[threadIdx.x] = bits(va);
    b[n + threadIdx.x] = bits(vb);
    __syncthreads();
    ra = value<V>(b[thread_of(a)]);
    rb = value<V>(b[n + thread_of(b_)]);
  }
};
using CtaXchg = CtaXchgT<0>;

// ------------------------------------------------- per-partition solve (a2-a4)
// v[0..size) holds b of this partition on entry and x on exit.  Must be
// called by all 32 lanes of the warp (it shuffles).  `lane_ok` marks lanes
// that own a partition (i < p).
template <typename T, int R, int M, typename TI, bool FULL = false, typename X = WarpXchg>
__device__ __forceinline__ void solve_partition(T (&v)[M], const int size_rt, const int i,
                                                const bool lane_ok, const DevLineTables& t, X& xch) {
  const int size = FULL ? M : size_rt;
  constexpr int F = 2 * R + 1;
  constexpr int NB = M - R;  // max bulk rows
  const int N = size - R;
  const bool big = FULL || i < t.count_big;  // whole-size partitions are all "big"
  const int pw = t.pw, p = t.p;

  // a2: forward elimination of the bulk block
#pragma unroll
  for (int j = 0; j < NB; j++) {
    if (j < N) {
      T s = v[R + j];
#pragma unroll
      for (int q = 1; q <= R; q++)
        if (j - q >= 0) s -= Tab<T>::fac(t, j * F + q - 1) * v[R + j - q];
      v[R + j] = s;
    }
  }
  // a2: backward substitution -> y_i
#pragma unroll
  for (int j = NB - 1; j >= 0; j--) {
    if (j < N) {
      T s = Tab<T>::fac(t, j * F + R) * v[R + j];
#pragma unroll
      for (int q = 1; q <= R; q++)
        if (R + j + q < M) {
          if (j + q < N) s -= Tab<T>::fac(t, j * F + R + q) * v[R + j + q];
        }
      v[R + j] = s;
    }
  }

  // a3: b-hat_i = b~_i - L~_i y_{i-1}[last r] - U~_i y_i[first r]   (Eq. 21)
  T ylast[R];
#pragma unroll
  for (int e = 0; e < R; e++) {
    T val = T(0);
#pragma unroll
    for (int u = R; u < M; u++) val = sel2<FULL>(u == N + e, v[u], val);
    ylast[e] = val;
  }
  const int prev = (i == 0) ? p - 1 : i - 1;
  const int next = (i + 1 >= p) ? 0 : i + 1;
  const bool has_prev = t.cyclic || i > 0;
  const bool has_next = t.cyclic || i + 1 < p;
  TI xt[R];
#pragma unroll
  for (int e = 0; e < R; e++) {
    const T yp = xch.get(ylast[e], prev);
    ylast[e] = yp;  // now y_{i-1}[N_{i-1} - r + e]
  }
#pragma unroll
  for (int q = 0; q < R; q++) {
    TI b = (TI)v[q];
#pragma unroll
    for (int e = 0; e < R; e++) {
      if (has_prev) b -= ITab<TI>::Lt(t, q, e) * (TI)ylast[e];
      b -= ITab<TI>::Ut(t, q, e) * (TI)v[R + e];
    }
    xt[q] = b;
  }

  // a3: interface system by block PCR with detach / reattach (Alg. 1-4),
  // with the W^{-1} products of every stage precomputed in the plan
  constexpr int rr = R * R;
  for (int st = 0; st < t.nstage; st++) {
    const bool hc = t.stage_has_c[st] != 0;
    const bool msg = (t.stage_msg[st] & (sizeof(TI) == 8 ? 1 : 2)) != 0;  // uniform over the CTA
    if (!msg && !hc) continue;  // coupling below rounding and C = I: nothing to do
    int sm = i, sp = i;
    TI C[rr], KM[rr], KP[rr];
    if (t.uniform) {
      const int s = t.ustage_s[st];
      sp = (i + s) & (p - 1);
      sm = (i - s) & (p - 1);
#pragma unroll
      for (int e = 0; e < rr; e++) {
        C[e] = ITab<TI>::ucoef(t, st, e);
        KM[e] = ITab<TI>::ucoef(t, st, rr + e);
        KP[e] = ITab<TI>::ucoef(t, st, 2 * rr + e);
      }
    } else if (lane_ok) {
      sm = __ldg(t.src + (st * 2 + 0) * p + i);
      sp = __ldg(t.src + (st * 2 + 1) * p + i);
#pragma unroll
      for (int e = 0; e < rr; e++) {
        C[e] = ITab<TI>::coef(t, ((st * 3 + 0) * rr + e) * p + i);
        KM[e] = ITab<TI>::coef(t, ((st * 3 + 1) * rr + e) * p + i);
        KP[e] = ITab<TI>::coef(t, ((st * 3 + 2) * rr + e) * p + i);
      }
    } else {
#pragma unroll
      for (int e = 0; e < rr; e++) C[e] = KM[e] = KP[e] = TI(0);
    }
    TI xm[R], xp[R];
    if (msg) {
#pragma unroll
      for (int q = 0; q < R; q++) xch.get2(xt[q], sm, sp, xm[q], xp[q]);
    }
    TI nxt[R];
#pragma unroll
    for (int q = 0; q < R; q++) {
      TI acc;
      if (hc) {
        acc = TI(0);
#pragma unroll
        for (int e = 0; e < R; e++) acc += C[q * R + e] * xt[e];
      } else {
        acc = xt[q];
      }
      if (msg) {
#pragma unroll
        for (int e = 0; e < R; e++) acc -= KM[q * R + e] * xm[e] + KP[q * R + e] * xp[e];
      }
      nxt[q] = acc;
    }
#pragma unroll
    for (int q = 0; q < R; q++) xt[q] = nxt[q];
  }

  // a4: back-substitution x_i = y_i - S_i x~_i - R_i x~_{i+1}   (Eq. 22)
  T xa[R], xb[R];
#pragma unroll
  for (int q = 0; q < R; q++) {
    const TI xn = xch.get(xt[q], next);
    xa[q] = (T)xt[q];
    xb[q] = has_next ? (T)xn : T(0);
  }
#pragma unroll
  for (int j = 0; j < NB; j++) {
    if (j < N) {
      T s = v[R + j];
#pragma unroll
      for (int q = 0; q < R; q++) {
        s -= Tab<T>::sr(t, big, j * 2 * R + q) * xa[q];
        s -= Tab<T>::sr(t, big, j * 2 * R + R + q) * xb[q];
      }
      v[R + j] = s;
    }
  }
#pragma unroll
  for (int q = 0; q < R; q++) v[q] = xa[q];
}

// Residual r = b - A x for this partition's rows, to FP64 accuracy, with x
// given as an unevaluated sum xh + xl of floats and b as bh + bl.  Neighbour
// rows of x come from the adjacent lanes.  Result rounded to FP32.
template <int R, int M, bool XLO, bool FULL = false, typename X = WarpXchg>
__device__ __forceinline__ void residual_df(const float (&bh)[M], const float (&bl)[M],
                                            const float (&xh)[M], const float (&xl)[M],
                                            float (&res)[M], const int size_rt, const int i,
                                            const DevLineTables& t, X& xch) {
  const int size = FULL ? M : size_rt;
  const int p = t.p, pw = t.pw;
  const int prev = (i == 0) ? p - 1 : i - 1;
  const int next = (i + 1 >= p) ? 0 : i + 1;
  // halo: last R rows of the previous partition, first R rows of the next
  float hh_prev[R], hl_prev[R], hh_next[R], hl_next[R];
#pragma unroll
  for (int e = 0; e < R; e++) {
    float lh = 0.f, ll = 0.f;
#pragma unroll
    for (int u = 0; u < M; u++) {
      lh = sel2<FULL>(u == size - R + e, xh[u], lh);
      ll = sel2<FULL>(u == size - R + e, xl[u], ll);
    }
    xch.get_two(lh, prev, xh[e], next, hh_prev[e], hh_next[e]);
    if (XLO) {
      xch.get_two(ll, prev, xl[e], next, hl_prev[e], hl_next[e]);
    } else {
      hl_prev[e] = 0.f;
      hl_next[e] = 0.f;
    }
    if (!t.cyclic) {  // acyclic system: nothing beyond its first and last rows
      if (i == 0) hh_prev[e] = hl_prev[e] = 0.f;
      if (i + 1 >= p) hh_next[e] = hl_next[e] = 0.f;
    }
  }
#pragma unroll
  for (int k = 0; k < M; k++) {
    if (k < size) {
      float ah = bh[k], al = bl[k];
#pragma unroll
      for (int tt = -R; tt <= R; tt++) {
        float vh = 0.f, vl = 0.f;
        const int kk = k + tt;
        if (kk < 0) {
          vh = hh_prev[R + kk];
          vl = hl_prev[R + kk];
        } else {
          if (kk < M) {
            vh = xh[kk];
            vl = XLO ? xl[kk] : 0.f;
          }
          // rows past the end of this partition belong to the next one
#pragma unroll
          for (int e = 0; e < R; e++) {
            vh = sel2<FULL>(kk == size + e, hh_next[e], vh);
            vl = sel2<FULL>(kk == size + e, hl_next[e], vl);
          }
        }
        const float bH = t.bandHi[tt + R], bL = t.bandLo[tt + R];
        const f2 pr = two_prod(bH, vh);
        const f2 s = two_sum(ah, -pr.hi);
        ah = s.hi;
        float lo = s.lo - pr.lo - bL * vh;
        if (XLO) lo -= bH * vl;
        al += lo;
      }
      res[k] = ah + al;
    }
  }
}

// ---------------------------------------------------------------- staging
// Shared-memory tile: line l of the tile owns S[l*lsz ...]; row k of
// partition i sits at k*sp + i (sp = pw + 1).  Lanes of a line read
// consecutive words for the same k (conflict-free sweeps) and the cooperative
// copies write consecutive rows of one partition at stride sp (odd), which is
// conflict-free too.
__device__ __forceinline__ int fdiv(int x, int d, unsigned mag) {
  return d == 1 ? x : (int)__umulhi((unsigned)x, mag);
}
__device__ __forceinline__ unsigned magic_of(int d) {
  return d <= 1 ? 0u : (unsigned)(((1ull << 32) + (unsigned)d - 1) / (unsigned)d);
}
__device__ __forceinline__ int slot_of(const DevLineTables& t, int row) {
  if (t.rows_lg >= 0) return (row & ((1 << t.rows_lg) - 1)) * t.sp + (row >> t.rows_lg);
  if (row < t.bound) {
    const int i = fdiv(row, t.rows_big, t.mag_b);
    return (row - i * t.rows_big) * t.sp + i;
  }
  const int r2 = row - t.bound;
  const int j = fdiv(r2, t.rows_small, t.mag_s);
  return (r2 - j * t.rows_small) * t.sp + t.count_big + j;
}

template <typename T, int V> struct V16;
template <> struct V16<double, 2> {
  static __device__ __forceinline__ void ld(const double* p, double (&v)[2]) {
    const double2 x = __ldg(reinterpret_cast<const double2*>(p));
    v[0] = x.x; v[1] = x.y;
  }
  static __device__ __forceinline__ void st(double* p, const double (&v)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
};
template <> struct V16<float, 4> {
  static __device__ __forceinline__ void ld(const float* p, float (&v)[4]) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  }
  static __device__ __forceinline__ void st(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};

// A tile of nl lines: dir 0 -> nl consecutive x-lines starting at `base`
// (line l at base + l*n, contiguous); dir 1/2 -> nl consecutive x positions,
// row `row` of line l at base + l + row*es.
struct TileRef {
  int64_t base, es;
  int nl, dir;
};

// Tile of the CTA.  dir 0: tile tx covers lines tx*TL ...; dir 1/2: tile
// (tx, to) covers x = tx*TL ... at z = to (dir 1) or y = to (dir 2).  No
// integer division: the launch grid is 2-D for y/z lines.
template <typename A>
__device__ __forceinline__ TileRef tile_of(const A& a, int n, int TL, int tx, int to) {
  TileRef r;
  r.dir = a.dir;
  if (a.dir == 0) {
    const int64_t L0 = (int64_t)tx * TL;
    r.base = L0 * n;
    r.es = 1;
    r.nl = (int)((a.nlines - L0) < TL ? (a.nlines - L0) : TL);
  } else {
    const int64_t x0 = (int64_t)tx * TL;
    r.base = x0 + (int64_t)to * (a.dir == 1 ? a.nx * a.ny : a.nx);
    r.es = (a.dir == 1) ? a.nx : a.nx * a.ny;
    r.nl = (int)((a.nx - x0) < TL ? (a.nx - x0) : TL);
  }
  return r;
}

// Global <-> shared copy of a tile (LOAD: global -> S, else S -> global).
template <bool LOAD, typename TG, typename TT>
__device__ __forceinline__ void tile_copy(const TileRef& tr, const DevLineTables& t, TT* S, TG* g0) {
  using TB = typename std::remove_const<TG>::type;
  constexpr int V = 16 / sizeof(TB);
  const int n = t.n, tid = threadIdx.x, nth = blockDim.x, nl = tr.nl;
  TG* g = g0 + tr.base;
  if (tr.dir == 0) {
    const int total = nl * n;
    if ((n % V) == 0 && (reinterpret_cast<uintptr_t>(g) & 15) == 0) {
      for (int c = tid; c < total / V; c += nth) {
        const int e = c * V, l = fdiv(e, n, t.mag_n), row = e - l * n;
        TB v[V];
        if constexpr (LOAD) {
          V16<TB, V>::ld(g + e, v);
#pragma unroll
          for (int u = 0; u < V; u++) S[l * t.lsz + slot_of(t, row + u)] = conv<TT>(v[u]);
        } else {
#pragma unroll
          for (int u = 0; u < V; u++) v[u] = conv<TB>(S[l * t.lsz + slot_of(t, row + u)]);
          V16<TB, V>::st(g + e, v);
        }
      }
    } else {
      for (int e = tid; e < total; e += nth) {
        const int l = fdiv(e, n, t.mag_n), row = e - l * n;
        if constexpr (LOAD) S[l * t.lsz + slot_of(t, row)] = conv<TT>(__ldg(g + e));
        else g[e] = conv<TB>(S[l * t.lsz + slot_of(t, row)]);
      }
    }
    return;
  }
  const int64_t es = tr.es;
  if ((nl % V) == 0 && (es % V) == 0 && (reinterpret_cast<uintptr_t>(g) & 15) == 0 && ((nl / V) & (nl / V - 1)) == 0) {
    const int cpr = nl / V;  // 16-byte chunks per row, a power of two
    const int lg = __ffs(cpr) - 1;
    for (int c = tid; c < n * cpr; c += nth) {
      const int row = c >> lg, ch = c & (cpr - 1);
      const int so = slot_of(t, row);
      TB v[V];
      if constexpr (LOAD) {
        V16<TB, V>::ld(g + row * es + ch * V, v);
#pragma unroll
        for (int u = 0; u < V; u++) S[(ch * V + u) * t.lsz + so] = conv<TT>(v[u]);
      } else {
#pragma unroll
        for (int u = 0; u < V; u++) v[u] = conv<TB>(S[(ch * V + u) * t.lsz + so]);
        V16<TB, V>::st(g + row * es + ch * V, v);
      }
    }
  } else {
    for (int e = tid; e < n * nl; e += nth) {
      const int row = e / nl, l = e - row * nl;
      if constexpr (LOAD) S[l * t.lsz + slot_of(t, row)] = conv<TT>(__ldg(g + row * es + l));
      else g[row * es + l] = conv<TB>(S[l * t.lsz + slot_of(t, row)]);
    }
  }
}

// h[idx] for a small register array and a runtime idx in [0, K), written as a
// select chain so the array stays in registers.
template <typename T, int K, bool PLAIN = false>
__device__ __forceinline__ T pick(const T (&h)[K], int idx) {
  T r = h[0];
#pragma unroll
  for (int e = 1; e < K; e++) r = sel2<PLAIN>(idx == e, h[e], r);
  return r;
}

// ---------------------------------------------------------------- kernel
// Window value at row offset k + q of a lane's partition: its own rows, or
// the upper halo once k + q runs past the partition (k, q compile-time).
template <typename TW, int M, int KS, int KA, bool FULL>
__device__ __forceinline__ TW window_up(const TW (&w)[M + KS], const TW (&hh)[KA], int k, int q, int size) {
  const int kq = (k + q < M) ? k + q : M - 1;  // compile-time clamp
  if (k + q < M) return sel2<FULL>(k + q < size, w[KS + kq], pick<TW, KA, FULL>(hh, k + q - size));
  return pick<TW, KA, FULL>(hh, k + q - size);
}

// Staggered stencils (App. A.2; Eq. 2): when s is set, move the window up by
// one row, so that window row r holds partition row r + 1 for r in
// [-KS, M + KS - 2] (the top halo row is then never read).  Ascending order
// reads every source before it is overwritten.
template <typename X, int M, int KS, int KA, bool FULL>
__device__ __forceinline__ void shift_window(X (&w)[M + KS], X (&hh)[KA], int size, bool s) {
  if (!s) return;
#pragma unroll
  for (int j = 0; j < KS; j++) w[j] = w[j + 1];
#pragma unroll
  for (int k = 0; k < M; k++) w[KS + k] = window_up<X, M, KS, KA, FULL>(w, hh, k, 1, size);
#pragma unroll
  for (int q = 0; q + 1 < KA; q++) hh[q] = hh[q + 1];
}

// a1 with a staggered stencil on the (shifted) window:
// b_k = sum_q w_q (f_{k+q-1} + SG f_{k-q}), SG = +1 interpolation, -1 derivative.
template <int SG, typename T, typename TW, int M, int KS, int KA, bool FULL>
__device__ __forceinline__ void staggered_rhs(const double* wq, const TW (&w)[M + KS], const TW (&hh)[KA], int size,
                                              T (&v)[M]) {
#pragma unroll
  for (int k = 0; k < M; k++) {
    T s = T(0);
#pragma unroll
    for (int q = 1; q <= KS; q++) {
      const T up = conv<T>(window_up<TW, M, KS, KA, FULL>(w, hh, k, q - 1, size));
      const T dn = conv<T>(w[KS + k - q]);
      s += (T)wq[q - 1] * (SG > 0 ? up + dn : up - dn);
    }
    v[k] = s;
  }
}

// Split of an input element into an unevaluated FP32 pair.
template <typename X>
__device__ __forceinline__ f2 split_in(X x) {
  if constexpr (sizeof(X) == 8) return split_f64((double)x);
  else return f2{(float)x, 0.f};
}

// a1 in double-float on the refinement path: b_k = sum_q w_q (f_{k+q+DU} +
// SG f_{k-q}) from the split window (fh, fl; upper halo hhh, hhl), as an
// unevaluated pair (bh carries the leading bits, bl the rest).  DU = 0, SG =
// -1: the central stencil of Eq. 1; DU = -1: the staggered stencils of App.
// A.2 / Eq. 2 on a shifted window.  Whole-size partitions with M even take
// rows k and k + M/2 in one instruction (same results as the scalar form).
template <int DU, int SG, int M, int KS, int KA, bool FULL>
__device__ __forceinline__ void rhs_df(const LineArgs& a, const float (&fh)[M + KS], const float (&fl)[M + KS],
                                       const float (&hhh)[KA], const float (&hhl)[KA], int size, float (&bh)[M],
                                       float (&bl)[M]) {
  if constexpr (FULL && (M % 2) == 0) {
    constexpr int H = M / 2;
#pragma unroll
    for (int k = 0; k < H; k++) {
      f32x2 dh = 0ull, dl = 0ull;
#pragma unroll
      for (int q = 1; q <= KS; q++) {
        const f32x2 uh = pk(win_row<M, KS, KA>(fh, hhh, k + q + DU), win_row<M, KS, KA>(fh, hhh, k + H + q + DU));
        const f32x2 ul = pk(win_row<M, KS, KA>(fl, hhl, k + q + DU), win_row<M, KS, KA>(fl, hhl, k + H + q + DU));
        f32x2 ds, de, dlo;
        if constexpr (SG > 0) {
          two_sum2(uh, pk(fh[KS + k - q], fh[KS + k + H - q]), ds, de);
          dlo = add2(de, add2(ul, pk(fl[KS + k - q], fl[KS + k + H - q])));
        } else {
          two_diff2(uh, pk(fh[KS + k - q], fh[KS + k + H - q]), ds, de);
          dlo = add2(de, sub2(ul, pk(fl[KS + k - q], fl[KS + k + H - q])));
        }
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
      unpk(dh, bh[k], bh[k + H]);
      unpk(dl, bl[k], bl[k + H]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < M; k++) {
      float dh = 0.f, dl = 0.f;
#pragma unroll
      for (int q = 1; q <= KS; q++) {
        const int u = k + q + DU;  // row of the upper point
        const int kq = (u < M) ? u : M - 1;
        float uh, ul;
        if (u < M) {
          uh = sel2<FULL>(u < size, fh[KS + kq], pick<float, KA, FULL>(hhh, u - size));
          ul = sel2<FULL>(u < size, fl[KS + kq], pick<float, KA, FULL>(hhl, u - size));
        } else {
          uh = pick<float, KA, FULL>(hhh, u - size);
          ul = pick<float, KA, FULL>(hhl, u - size);
        }
        const float dnh = fh[KS + k - q], dnl = fl[KS + k - q];
        const f2 df = two_sum(uh, SG > 0 ? dnh : -dnh);
        const float dlo = df.lo + (SG > 0 ? ul + dnl : ul - dnl);
        const f2 pr = two_prod(a.wHi[q - 1], df.hi);
        const float plo = pr.lo + __fmaf_rn(a.wHi[q - 1], dlo, a.wLo[q - 1] * df.hi);
        if (q == 1) {
          dh = pr.hi;
          dl = plo;
        } else {
          const f2 sm = two_sum(dh, pr.hi);
          dh = sm.hi;
          dl += sm.lo + plo;
        }
      }
      bh[k] = dh;
      bl[k] = dl;
    }
  }
}

// ---------------------------------------------------------------- async copies
// Global -> shared copies that hold no registers while in flight (the
// pipelined kernel prefetches the next tile's rows while it computes).
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
template <int B>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_addr(dst)), "l"(src), "n"(B) : "memory");
}
// 16-byte copy that bypasses L1 (streamed tiles)
__device__ __forceinline__ void cp_async_cg16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// How a tile reaches its threads.
//  kStaged: a warp holds one line (lane = partition); the tile is staged
//    through shared memory with 16-byte coalesced global accesses.
//  kDirectX: x-lines, a warp holds one line and each lane reads and writes
//    its own contiguous rows with 16-byte vector accesses (no staging).
//  kDirectStrided: y/z lines, thread = (partition i, line g) with g fastest,
//    so one warp-wide access of a row covers kStridedLines consecutive x
//    positions of 32 / kStridedLines partitions (full 32-byte sectors, no
//    staging); the interface messages between partitions then cross warps
//    through shared memory.  The CTA has kStridedLines x pw threads.
//  kStridedWarp: y/z lines of 32 partitions in the pipelined kernel.  The
//    rows are copied with the line-fastest mapping of kDirectStrided (same
//    global access pattern) but into the shared-memory slots of the thread
//    that solves them, where a warp holds one line (lane = partition), so the
//    interface messages are warp shuffles as for x-lines; the results go back
//    through the same slots and leave with the line-fastest mapping.
//  kTileX: x-lines in the pipelined kernel.  A warp holds one line (lane =
//    partition; or 32 / pw lines), which is contiguous in HBM: the warp copies
//    it with 16-byte copies of consecutive pieces (coalesced) into shared
//    memory, one chunk of M rows per partition, each chunk padded by 16 bytes
//    so that the lanes' reads of their own chunks fall on distinct banks; the
//    stencil halo comes from the neighbouring chunks.
constexpr int kStaged = 0, kDirectX = 1, kDirectStrided = 2, kStridedWarp = 3, kTileX = 4;
constexpr int kStridedLines = 8;
constexpr int kStridedWarpThreads = kStridedLines * 32;  // kStridedWarp: 8 lines of 32 lanes
__host__ __device__ constexpr bool strided_layout(int layout) {
  return layout == kDirectStrided || layout == kStridedWarp;
}

// Column of solving thread c in the pipelined kernel's slot rows.  In
// kStridedWarp (32 lanes per line, c = 32 g + i) the lanes of line g are
// permuted (i ^ 2g): the copies of one warp (8 lines x 4 partitions) and the
// reads of one line then fall on distinct banks in each half-warp.
// Elements of one half of the pipelined kernel's double buffer: kTileX holds
// (bd / pw) lines of p padded chunks, kStridedWarp M slot rows of bd threads
// (the halo rows are read from the neighbouring lanes' slots), the others
// NS = M + 2 KS slot rows of bd threads.
template <int M, int KS, typename TIn, int LAYOUT>
__host__ __device__ constexpr int pipe_buf_elems(int bd, int pw, int p) {
  return LAYOUT == kTileX ? (bd / pw) * p * (M + 16 / (int)sizeof(TIn))
         : LAYOUT == kStridedWarp ? M * bd : (M + 2 * KS) * bd;
}

template <int LAYOUT>
__device__ __forceinline__ int slot_col(int c) {
  if constexpr (LAYOUT == kStridedWarp) return c ^ (((c >> 5) & 7) << 1);
  else return c;
}

// Exchanger of the interface messages for a layout: warp shuffles when a
// warp holds a whole line, shared memory otherwise (strided layout: partition
// src of line g is thread src * kStridedLines + g).
template <bool CTA>
__device__ __forceinline__ auto make_xchg(int pw, unsigned char* smem, int offset) {
  if constexpr (CTA) return CtaXchgT<kStridedLines>{reinterpret_cast<unsigned long long*>(smem), 0, 1, offset};
  else return WarpXchg{pw};
}

// This thread's own rows from the prefetch slots (layout of prefetch_rows;
// VEC: 16-byte units read back with 16-byte shared loads).
template <int M, typename TIn, bool VEC, int BD = 0>
__device__ __forceinline__ void pipe_rows(const TIn* slots, TIn (&v)[M], const int col) {
  const int bd = BD ? BD : blockDim.x;  // BD: block size known at compile time
  if constexpr (VEC && (M % (16 / sizeof(TIn))) == 0) {
    constexpr int V = 16 / sizeof(TIn);
#pragma unroll
    for (int u = 0; u < M / V; u++) {
      const float4 q = *reinterpret_cast<const float4*>(slots + ((size_t)u * bd + col) * V);
      const TIn* e = reinterpret_cast<const TIn*>(&q);
#pragma unroll
      for (int j = 0; j < V; j++) v[u * V + j] = e[j];
    }
  } else {
#pragma unroll
    for (int k = 0; k < M; k++) v[k] = slots[(size_t)k * bd + col];
  }
}

// Partition and line of this thread within a tile (see the layouts above).
struct ThreadPart {
  int g, i, start, size;
  bool lane_ok;
};
template <int M, bool FULL, int LAYOUT>
__device__ __forceinline__ ThreadPart thread_part(const DevLineTables& t) {
  ThreadPart r;
  const int pw = t.pw;
  r.g = LAYOUT == kDirectStrided ? threadIdx.x % kStridedLines : threadIdx.x / pw;
  r.i = LAYOUT == kDirectStrided ? threadIdx.x / kStridedLines : threadIdx.x % pw;
  r.lane_ok = r.i < t.p;
  r.start = 0;
  r.size = 2 * t.r;
  if (FULL) {
    r.start = r.i * M;
    r.size = M;
  } else if (r.lane_ok) {
    partition_of(t, r.i, r.start, r.size);
  }
  return r;
}

// Prefetch slots of the pipelined kernel: thread-private, slot j of thread
// tid at slots[j * blockDim + tid] (conflict-free); j < M: own row j,
// M + q: row start - KS + q, M + KS + q: row start + size + q (periodic).
// VEC (contiguous rows, M a multiple of the 16-byte vector width V): own
// rows are copied in 16-byte units, unit u of thread tid at element offset
// (u * bd + tid) * V, conflict-free for 16-byte shared loads.
template <int M, int KS, bool FULL, typename TIn, bool VEC = false, int BD = 0>
__device__ __forceinline__ void prefetch_rows(TIn* slot0, const TIn* gline, int64_t es, int start, int size,
                                              int n) {
  const int bd = BD ? BD : blockDim.x;  // BD: block size known at compile time
  if constexpr (VEC) {
    constexpr int V = 16 / sizeof(TIn);
    TIn* base = slot0 - threadIdx.x;  // thread 0's slot 0
#pragma unroll
    for (int u = 0; u < M / V; u++) cp_async<16>(base + ((size_t)u * bd + threadIdx.x) * V, gline + start + u * V);
  } else {
#pragma unroll
    for (int k = 0; k < M; k++)
      if (FULL || k < size) cp_async<sizeof(TIn)>(slot0 + k * bd, gline + (start + k) * es);
  }
#pragma unroll
  for (int q = 0; q < KS; q++) {
    int rlo = start - KS + q;
    rlo += (rlo < 0) ? n : 0;
    cp_async<sizeof(TIn)>(slot0 + (M + q) * bd, gline + rlo * es);
    int rhi = start + size + q;
    rhi -= (rhi >= n) ? n : 0;
    cp_async<sizeof(TIn)>(slot0 + (M + KS + q) * bd, gline + rhi * es);
  }
}

// kTileX: rows of this lane's chunk (chunk g p + i of the half-buffer
// `buf`, M rows padded to CS = M + 16 / sizeof(TIn) elements) and the KS
// halo rows on each side from the neighbouring chunks of the same line
// (periodic).  Lanes without a partition read chunk g p (values unused).
template <int M, int KS, int KA, typename TIn>
__device__ __forceinline__ void tilex_rows(const TIn* buf, const DevLineTables& t, const int g, const int i,
                                           const bool lane_ok, TIn (&own)[M], TIn (&lo_h)[KA], TIn (&hi_h)[KA]) {
  constexpr int CS = M + 16 / (int)sizeof(TIn);
  const int c0 = g * t.p, c = c0 + (lane_ok ? i : 0);
  const TIn* chunk = buf + (size_t)c * CS;
  const TIn* cprev = buf + (size_t)(i == 0 || !lane_ok ? c0 + t.p - 1 : c - 1) * CS;
  const TIn* cnext = buf + (size_t)(i >= t.p - 1 || !lane_ok ? c0 : c + 1) * CS;
  static_assert((M * sizeof(TIn)) % 16 == 0, "whole 16-byte units per chunk");
#pragma unroll
  for (int u = 0; u < (int)(M * sizeof(TIn) / 16); u++) {
    const float4 q = *reinterpret_cast<const float4*>(chunk + u * (16 / sizeof(TIn)));
    const TIn* e = reinterpret_cast<const TIn*>(&q);
#pragma unroll
    for (int j = 0; j < (int)(16 / sizeof(TIn)); j++) own[u * (16 / sizeof(TIn)) + j] = e[j];
  }
#pragma unroll
  for (int q = 0; q < KS; q++) {
    lo_h[q] = cprev[M - KS + q];
    hi_h[q] = cnext[q];
  }
}

// kStridedWarp: rows of lane i of line g (slot column slot_col(32 g + i) of
// the half-buffer `buf`, M slot rows of kStridedWarpThreads) and the KS halo
// rows on each side from the slots of lanes i - 1 and i + 1 of the same line
// (periodic over the line's p partitions; lanes i >= p read in-range slots
// whose values are unused).
template <int M, int KS, int KA, typename TIn>
__device__ __forceinline__ void swarp_rows(const TIn* buf, const int p, const int g, const int i, TIn (&own)[M],
                                           TIn (&lo_h)[KA], TIn (&hi_h)[KA]) {
  constexpr int BD = kStridedWarpThreads;
  const int prev = i == 0 ? p - 1 : i - 1, next = i + 1 >= p ? 0 : i + 1;
  pipe_rows<M, TIn, false, BD>(buf, own, slot_col<kStridedWarp>(32 * g + i));
  const TIn* bp = buf + slot_col<kStridedWarp>(32 * g + prev);
  const TIn* bn = buf + slot_col<kStridedWarp>(32 * g + next);
#pragma unroll
  for (int q = 0; q < KS; q++) {
    lo_h[q] = bp[(M - KS + q) * BD];
    hi_h[q] = bn[q * BD];
  }
}

// One tile = blockDim / pw consecutive lines, processed by the whole CTA:
// gather the rows (+ stencil halo) of every partition, stencil + solve per
// thread, write back.  KS: stencil terms compiled in (0 = the input already
// is b).  FULL: every partition has exactly M rows (sizes known at compile
// time).  LAYOUT: see kStaged / kDirectX / kDirectStrided.  Used by the
// per-plan kernel (one tile per CTA) and by the persistent batch kernel (many
// tiles per CTA).
template <int R, int M, int MODE, int KS, typename TIn, typename TOut, bool FULL = false, int LAYOUT = kStaged,
          bool PIPE = false, int ST = 0>
__device__ __forceinline__ void line_tile(const LineArgs& a, const DevLineTables& t, const void* in_ptr,
                                          void* out_ptr, const int tx, const int to, unsigned char* smem_raw,
                                          const TIn* pslots = nullptr, int* xflip = nullptr) {
  using T = typename std::conditional<MODE == kModeF64, double, float>::type;
  using TT = typename std::conditional<(sizeof(TIn) == 8 || sizeof(TOut) == 8), double, float>::type;
  constexpr bool DIRECT = LAYOUT == kDirectX, DSTR = LAYOUT == kDirectStrided, SWARP = LAYOUT == kStridedWarp;
  constexpr bool TILEX = LAYOUT == kTileX;
  static_assert(!(SWARP || TILEX) || (PIPE && FULL), "pipelined whole-size partitions only");
  static_assert(!TILEX || (sizeof(TIn) == 8 && refine_mode(MODE)), "kTileX: FP64 input, refinement");
  using TW = typename std::conditional<DIRECT || DSTR || SWARP || TILEX, TIn, TT>::type;  // element type of the gathered window
  constexpr int KA = KS > 0 ? KS : 1;  // halo array size (KS = 0 compiles no stencil)
  TT* S = reinterpret_cast<TT*>(smem_raw);
  const int pw = t.pw;
  const int TL = strided_layout(LAYOUT) ? kStridedLines : blockDim.x / pw;
  const TileRef tr = tile_of(a, t.n, TL, tx, to);
  const int nl = tr.nl;
  const ThreadPart tp = thread_part<M, FULL, LAYOUT>(t);
  const int g = tp.g, i = tp.i, start = tp.start, size = tp.size;
  const bool lane_ok = tp.lane_ok;
  const bool ok = lane_ok && g < nl;
  const int n = t.n;
  TT* SL = S + g * t.lsz;
  // direct layouts: row 0 of this thread's line; row r at gin[r * es]
  const int64_t es = strided_layout(LAYOUT) ? tr.es : 1;
  const TIn* gin = (const TIn*)in_ptr + tr.base + (strided_layout(LAYOUT) ? (int64_t)g : (int64_t)g * n);
  TOut* gout = (TOut*)out_ptr + tr.base + (strided_layout(LAYOUT) ? (int64_t)g : (int64_t)g * n);
  const int col = slot_col<LAYOUT>(threadIdx.x);  // this thread's column of the prefetch slots

  // ---- gather: w[KS + k] = row start + k, w[q] = row start - KS + q, hh[q] = row start + size + q
  // (the refinement mode gathers straight into FP32 pairs below)
  TW w[M + KS], hh[KA];
  if constexpr (refine_mode(MODE)) {
    if constexpr (LAYOUT == kStaged) {
      tile_copy<true, const TIn, TT>(tr, t, S, (const TIn*)in_ptr);
      __syncthreads();
    }
  } else if constexpr (PIPE) {
    const TIn* s0 = pslots + col;
    const int bd = blockDim.x;
    TIn own[M];
    pipe_rows<M, TIn, DIRECT>(pslots, own, col);
#pragma unroll
    for (int k = 0; k < M; k++) w[KS + k] = (ok && (FULL || k < size)) ? own[k] : TIn(0);
#pragma unroll
    for (int q = 0; q < KS; q++) {
      w[q] = ok ? s0[(M + q) * bd] : TIn(0);
      hh[q] = ok ? s0[(M + KS + q) * bd] : TIn(0);
    }
  } else if constexpr (DSTR) {
#pragma unroll
    for (int k = 0; k < M; k++) w[KS + k] = (ok && (FULL || k < size)) ? __ldg(gin + (start + k) * es) : TIn(0);
#pragma unroll
    for (int q = 0; q < KS; q++) {
      int rlo = start - KS + q;
      rlo += (rlo < 0) ? n : 0;
      w[q] = ok ? __ldg(gin + rlo * es) : TIn(0);
      int rhi = start + size + q;
      rhi -= (rhi >= n) ? n : 0;
      hh[q] = ok ? __ldg(gin + rhi * es) : TIn(0);
    }
  } else if constexpr (DIRECT) {
    constexpr int V = 16 / sizeof(TIn);
    if (FULL && (M % V) == 0) {
#pragma unroll
      for (int k = 0; k < M; k += V) {
        TIn tmp[V];
        if (ok) V16<TIn, V>::ld(gin + start + k, tmp);
        else {
#pragma unroll
          for (int u = 0; u < V; u++) tmp[u] = TIn(0);
        }
#pragma unroll
        for (int u = 0; u < V; u++) w[KS + k + u] = tmp[u];
      }
    } else {
#pragma unroll
      for (int k = 0; k < M; k++) w[KS + k] = (ok && k < size) ? __ldg(gin + start + k) : TIn(0);
    }
#pragma unroll
    for (int q = 0; q < KS; q++) {
      int rlo = start - KS + q;
      rlo += (rlo < 0) ? n : 0;
      w[q] = ok ? __ldg(gin + rlo) : TIn(0);
      int rhi = start + size + q;
      rhi -= (rhi >= n) ? n : 0;
      hh[q] = ok ? __ldg(gin + rhi) : TIn(0);
    }
  } else {
    tile_copy<true, const TIn, TT>(tr, t, S, (const TIn*)in_ptr);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < M; k++) w[KS + k] = (ok && (FULL || k < size)) ? SL[k * t.sp + i] : TT(0);
#pragma unroll
    for (int q = 0; q < KS; q++) {  // acyclic lines (boundary closures): the end values extended
      int rlo = start - KS + q;
      rlo = rlo >= 0 ? rlo : t.cyclic ? rlo + n : 0;
      w[q] = ok ? SL[slot_of(t, rlo)] : TT(0);
      int rhi = start + size + q;
      rhi = rhi < n ? rhi : t.cyclic ? rhi - n : n - 1;
      hh[q] = ok ? SL[slot_of(t, rhi)] : TT(0);
    }
  }

  TOut xo[M];
  auto xch = make_xchg<DSTR>(pw, smem_raw, g);
  // a CTA walking several tiles continues the exchange buffers' alternation
  // across tiles: the first round of a tile then never writes the buffer the
  // previous tile's last round is still being read from
  if constexpr (DSTR) {
    if (xflip) xch.flip = *xflip;
  }
  using TIR = typename std::conditional<MODE == kModeRefineI64, double, float>::type;  // interface of the FP32 solves
  if constexpr (!refine_mode(MODE)) {
    T v[M];
    if constexpr (KS > 0 && ST != 0) {
      shift_window<TW, M, KS, KA, FULL>(w, hh, size, a.stag_shift != 0);
      if (a.stag_sum) staggered_rhs<1, T, TW, M, KS, KA, FULL>(a.w, w, hh, size, v);
      else staggered_rhs<-1, T, TW, M, KS, KA, FULL>(a.w, w, hh, size, v);
    } else {
#pragma unroll
      for (int k = 0; k < M; k++) {
        if (KS == 0) {
          v[k] = conv<T>(w[KS + k]);
        } else {
          // a1: b_k = sum_q w_q (f_{k+q} - f_{k-q})
          T s = T(0);
#pragma unroll
          for (int q = 1; q <= KS; q++)
            s += (T)a.w[q - 1] *
                 (conv<T>(window_up<TW, M, KS, KA, FULL>(w, hh, k, q, size)) - conv<T>(w[KS + k - q]));
          v[k] = s;
        }
      }
    }
    solve_partition<T, R, M, T, FULL>(v, size, i, lane_ok, t, xch);
#pragma unroll
    for (int k = 0; k < M; k++) xo[k] = conv<TOut>(v[k]);
  } else {
    // FP32 bulk + FP64-accurate residual refinement.  Every element is split
    // into an FP32 pair as soon as it is loaded.
    float bh[M], bl[M];
    float fh[M + KS], fl[M + KS], hhh[KA], hhl[KA];
    if constexpr (PIPE && sizeof(TIn) == 8) {
      // whole-size partitions only (PIPE implies FULL)
      const TIn* s0 = pslots + col;
      const int bd = blockDim.x;
      TIn own[M], lo_h[KA], hi_h[KA];
      if constexpr (TILEX) {
        tilex_rows<M, KS, KA>(pslots, t, g, i, lane_ok, own, lo_h, hi_h);
      } else if constexpr (SWARP) {
        swarp_rows<M, KS, KA>(pslots, t.p, g, i, own, lo_h, hi_h);
      } else {
        pipe_rows<M, TIn, DIRECT>(pslots, own, col);
#pragma unroll
        for (int q = 0; q < KS; q++) {
          lo_h[q] = s0[(M + q) * bd];
          hi_h[q] = s0[(M + KS + q) * bd];
        }
      }
      if (ok) {
        unsigned bad = 0u;
        f2 sv;
#pragma unroll
        for (int k = 0; k < M; k++) {
          bad |= split_fast((double)own[k], sv);
          fh[KS + k] = sv.hi;
          fl[KS + k] = sv.lo;
        }
#pragma unroll
        for (int q = 0; q < KS; q++) {
          bad |= split_fast((double)lo_h[q], sv);
          fh[q] = sv.hi;
          fl[q] = sv.lo;
          bad |= split_fast((double)hi_h[q], sv);
          hhh[q] = sv.hi;
          hhl[q] = sv.lo;
        }
        if (bad) {  // a zero or a value outside [2^-103, 2^128) in this thread's rows:
                    // split them again (re-read from the slots) the general way
          if constexpr (TILEX || SWARP) {
            TIn again[M], lo_a[KA], hi_a[KA];
            if constexpr (TILEX) tilex_rows<M, KS, KA>(pslots, t, g, i, lane_ok, again, lo_a, hi_a);
            else swarp_rows<M, KS, KA>(pslots, t.p, g, i, again, lo_a, hi_a);
#pragma unroll
            for (int k = 0; k < M; k++) {
              sv = split_f64((double)again[k]);
              fh[KS + k] = sv.hi;
              fl[KS + k] = sv.lo;
            }
#pragma unroll
            for (int q = 0; q < KS; q++) {
              sv = split_f64((double)lo_a[q]);
              fh[q] = sv.hi;
              fl[q] = sv.lo;
              sv = split_f64((double)hi_a[q]);
              hhh[q] = sv.hi;
              hhl[q] = sv.lo;
            }
          } else {
            TIn again[M];
            pipe_rows<M, TIn, DIRECT>(pslots, again, col);
#pragma unroll
            for (int k = 0; k < M; k++) {
              sv = split_f64((double)again[k]);
              fh[KS + k] = sv.hi;
              fl[KS + k] = sv.lo;
            }
#pragma unroll
            for (int q = 0; q < KS; q++) {
              sv = split_f64((double)s0[(M + q) * bd]);
              fh[q] = sv.hi;
              fl[q] = sv.lo;
              sv = split_f64((double)s0[(M + KS + q) * bd]);
              hhh[q] = sv.hi;
              hhl[q] = sv.lo;
            }
          }
        }
      } else {
#pragma unroll
        for (int k = 0; k < M + KS; k++) fh[k] = fl[k] = 0.f;
#pragma unroll
        for (int q = 0; q < KA; q++) hhh[q] = hhl[q] = 0.f;
      }
    } else if constexpr (PIPE) {
      const TIn* s0 = pslots + col;
      const int bd = blockDim.x;
      TIn own[M];
      pipe_rows<M, TIn, DIRECT>(pslots, own, col);
#pragma unroll
      for (int k = 0; k < M; k++) {
        const f2 sv = split_in((ok && (FULL || k < size)) ? own[k] : TIn(0));
        fh[KS + k] = sv.hi;
        fl[KS + k] = sv.lo;
      }
#pragma unroll
      for (int q = 0; q < KS; q++) {
        const f2 a0 = split_in(ok ? s0[(M + q) * bd] : TIn(0));
        fh[q] = a0.hi;
        fl[q] = a0.lo;
        const f2 a1 = split_in(ok ? s0[(M + KS + q) * bd] : TIn(0));
        hhh[q] = a1.hi;
        hhl[q] = a1.lo;
      }
    } else if constexpr (DSTR) {
#pragma unroll
      for (int k = 0; k < M; k++) {
        const f2 sv = split_in((ok && (FULL || k < size)) ? __ldg(gin + (start + k) * es) : TIn(0));
        fh[KS + k] = sv.hi;
        fl[KS + k] = sv.lo;
      }
#pragma unroll
      for (int q = 0; q < KS; q++) {
        int rlo = start - KS + q;
        rlo += (rlo < 0) ? n : 0;
        const f2 a0 = split_in(ok ? __ldg(gin + rlo * es) : TIn(0));
        fh[q] = a0.hi;
        fl[q] = a0.lo;
        int rhi = start + size + q;
        rhi -= (rhi >= n) ? n : 0;
        const f2 a1 = split_in(ok ? __ldg(gin + rhi * es) : TIn(0));
        hhh[q] = a1.hi;
        hhl[q] = a1.lo;
      }
    } else if constexpr (DIRECT) {
      constexpr int V = 16 / sizeof(TIn);
      if (FULL && (M % V) == 0) {
#pragma unroll
        for (int k = 0; k < M; k += V) {
          TIn tmp[V];
          if (ok) V16<TIn, V>::ld(gin + start + k, tmp);
          else {
#pragma unroll
            for (int u = 0; u < V; u++) tmp[u] = TIn(0);
          }
#pragma unroll
          for (int u = 0; u < V; u++) {
            const f2 sv = split_in(tmp[u]);
            fh[KS + k + u] = sv.hi;
            fl[KS + k + u] = sv.lo;
          }
        }
      } else {
#pragma unroll
        for (int k = 0; k < M; k++) {
          const f2 sv = split_in((ok && k < size) ? __ldg(gin + start + k) : TIn(0));
          fh[KS + k] = sv.hi;
          fl[KS + k] = sv.lo;
        }
      }
#pragma unroll
      for (int q = 0; q < KS; q++) {
        int rlo = start - KS + q;
        rlo += (rlo < 0) ? n : 0;
        const f2 a0 = split_in(ok ? __ldg(gin + rlo) : TIn(0));
        fh[q] = a0.hi;
        fl[q] = a0.lo;
        int rhi = start + size + q;
        rhi -= (rhi >= n) ? n : 0;
        const f2 a1 = split_in(ok ? __ldg(gin + rhi) : TIn(0));
        hhh[q] = a1.hi;
        hhl[q] = a1.lo;
      }
    } else {
#pragma unroll
      for (int k = 0; k < M; k++) {
        const f2 sv = split_in((ok && (FULL || k < size)) ? SL[k * t.sp + i] : TT(0));
        fh[KS + k] = sv.hi;
        fl[KS + k] = sv.lo;
      }
#pragma unroll
      for (int q = 0; q < KS; q++) {  // acyclic lines (boundary closures): the end values extended
        int rlo = start - KS + q;
        rlo = rlo >= 0 ? rlo : t.cyclic ? rlo + n : 0;
        const f2 a0 = split_in(ok ? SL[slot_of(t, rlo)] : TT(0));
        fh[q] = a0.hi;
        fl[q] = a0.lo;
        int rhi = start + size + q;
        rhi = rhi < n ? rhi : t.cyclic ? rhi - n : n - 1;
        const f2 a1 = split_in(ok ? SL[slot_of(t, rhi)] : TT(0));
        hhh[q] = a1.hi;
        hhl[q] = a1.lo;
      }
    }
    if (KS == 0) {
#pragma unroll
      for (int k = 0; k < M; k++) {
        bh[k] = fh[KS + k];
        bl[k] = fl[KS + k];
      }
    } else if constexpr (ST != 0) {
      shift_window<float, M, KS, KA, FULL>(fh, hhh, size, a.stag_shift != 0);
      shift_window<float, M, KS, KA, FULL>(fl, hhl, size, a.stag_shift != 0);
      if (a.stag_sum) rhs_df<-1, 1, M, KS, KA, FULL>(a, fh, fl, hhh, hhl, size, bh, bl);
      else rhs_df<-1, -1, M, KS, KA, FULL>(a, fh, fl, hhh, hhl, size, bh, bl);
    } else {
      // a1: b = sum_q w_q (f_{k+q} - f_{k-q}) in double-float
      rhs_df<0, -1, M, KS, KA, FULL>(a, fh, fl, hhh, hhl, size, bh, bl);
    }
    // sweep 0: x0 = A^{-1} bh
    float xh[M], v[M];
#pragma unroll
    for (int k = 0; k < M; k++) v[k] = bh[k];
    solve_partition<float, R, M, TIR, FULL>(v, size, i, lane_ok, t, xch);
#pragma unroll
    for (int k = 0; k < M; k++) xh[k] = v[k];
    // refinement sweep 1: x <- x0 + A^{-1}(b - A x0), residual to FP64 accuracy
    if constexpr (FULL && (M % 2) == 0) residual_sym2<R, M, false>(bh, bl, xh, xh, v, i, t, xch);
    else if constexpr (FULL) residual_sym<R, M, false>(bh, bl, xh, xh, v, i, t, xch);
    else residual_df<R, M, false, FULL>(bh, bl, xh, xh, v, size, i, t, xch);
    solve_partition<float, R, M, TIR, FULL>(v, size, i, lane_ok, t, xch);
    // an input of 2^128 or more (inf after the split), or a non-finite one,
    // leaves x0 or the correction non-finite: CBS_ERR_RANGE (integer tests)
    unsigned nonfin = 0u;
#pragma unroll
    for (int k = 0; k < M; k++)
      nonfin |= ((__float_as_uint(xh[k]) & 0x7f800000u) == 0x7f800000u) ||
                ((__float_as_uint(v[k]) & 0x7f800000u) == 0x7f800000u) ? 1u : 0u;
    if (nonfin && ok) atomicExch(a.status, CBS_ERR_RANGE);
    if (a.sweeps < 2) {
      // x = x0 + delta: one FP64 add (the FP64 pipe is idle otherwise on this
      // path); x0 is widened with integer operations, delta too in the
      // x-line layout, and by the FP64 pipe in the strided layout, whose
      // integer work is heavier (measured: each choice is faster where used)
#pragma unroll
      for (int k = 0; k < M; k++) {
        double dv;
        if constexpr (DSTR) dv = (double)v[k];
        else dv = f32_to_f64_normal(v[k]);
        const double xd = f32_to_f64_normal(xh[k]) + dv;
        if constexpr (sizeof(TOut) == 8) xo[k] = (TOut)xd;
        else xo[k] = (TOut)(xh[k] + v[k]);
      }
    } else {
      // sweep 2 on the unevaluated pair x = xh + xl
      float xl[M];
#pragma unroll
      for (int k = 0; k < M; k++) {
        const f2 sm = two_sum(xh[k], v[k]);
        xh[k] = sm.hi;
        xl[k] = sm.lo;
      }
      if constexpr (FULL && (M % 2) == 0) residual_sym2<R, M, true>(bh, bl, xh, xl, v, i, t, xch);
      else if constexpr (FULL) residual_sym<R, M, true>(bh, bl, xh, xl, v, i, t, xch);
      else residual_df<R, M, true, FULL>(bh, bl, xh, xl, v, size, i, t, xch);
      solve_partition<float, R, M, TIR, FULL>(v, size, i, lane_ok, t, xch);
#pragma unroll
      for (int k = 0; k < M; k++) {
        const double xd = f32_to_f64_normal(xh[k]) + f32_to_f64_normal(xl[k] + v[k]);
        if constexpr (sizeof(TOut) == 8) xo[k] = (TOut)xd;
        else xo[k] = (TOut)(xh[k] + (xl[k] + v[k]));
      }
    }
  }

  if constexpr (DSTR) {
    if (xflip) *xflip = xch.flip;
  }
  // ---- write back
  if constexpr (SWARP) {
    // into this thread's own slots (its rows are consumed), then out with
    // the line-fastest mapping of the copies: one warp-wide store covers
    // kStridedLines consecutive x positions of 32 / kStridedLines rows
    static_assert(sizeof(TOut) == sizeof(TIn), "kStridedWarp: the slots hold the results");
    TOut* so = reinterpret_cast<TOut*>(const_cast<TIn*>(pslots));
    constexpr int bd = kStridedWarpThreads;
#pragma unroll
    for (int k = 0; k < M; k++) so[(size_t)k * bd + col] = xo[k];
    __syncthreads();
    const int gp = threadIdx.x % kStridedLines, ip = threadIdx.x / kStridedLines;
    if (gp < nl && ip < t.p) {
      const int cs = slot_col<LAYOUT>(gp * pw + ip);
      TOut* go = (TOut*)out_ptr + tr.base + gp + (int64_t)ip * M * tr.es;
#pragma unroll
      for (int k = 0; k < M; k++) go[(int64_t)k * tr.es] = so[(size_t)k * bd + cs];
    }
  } else if constexpr (DSTR) {
    if (ok) {
#pragma unroll
      for (int k = 0; k < M; k++)
        if (FULL || k < size) gout[(start + k) * es] = xo[k];
    }
  } else if constexpr (DIRECT || TILEX) {
    constexpr int V = 16 / sizeof(TOut);
    if (ok) {
      if (FULL && (M % V) == 0) {
#pragma unroll
        for (int k = 0; k < M; k += V) {
          TOut tmp[V];
#pragma unroll
          for (int u = 0; u < V; u++) tmp[u] = xo[k + u];
          V16<TOut, V>::st(gout + start + k, tmp);
        }
      } else {
#pragma unroll
        for (int k = 0; k < M; k++)
          if (k < size) gout[start + k] = xo[k];
      }
    }
  } else {
    __syncwarp();
    if (ok) {
#pragma unroll
      for (int k = 0; k < M; k++)
        if (FULL || k < size) SL[k * t.sp + i] = conv<TT>(xo[k]);
    }
    __syncthreads();
    tile_copy<false, TOut, TT>(tr, t, S, (TOut*)out_ptr);
  }
}

template <int R, int M, int MODE, int KS, typename TIn, typename TOut, bool FULL, int LAYOUT, int ST = 0>
__global__ void __launch_bounds__(256, (refine_mode(MODE) || M == 32) ? 2 : 3) line_kernel(const LineArgs a, const DevLineTables t) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  line_tile<R, M, MODE, KS, TIn, TOut, FULL, LAYOUT, false, ST>(a, t, a.in, a.out, blockIdx.x, blockIdx.y, smem_raw);
}

// Issue (and commit) the copies of this thread's rows of tile `tile` into
// half `buf` of the double buffer (whole-size partitions).
template <int M, int KS, typename TIn, int LAYOUT>
__device__ __forceinline__ void prefetch_tile(const LineArgs& a, const DevLineTables& t, const ThreadPart& tp,
                                              const int gx, const int tile, TIn* slots, const int buf) {
  constexpr int NS = M + 2 * KS;
  constexpr bool STR = strided_layout(LAYOUT);
  const int bd = blockDim.x, TL = STR ? kStridedLines : bd / t.pw;
  const int tx = STR ? tile % gx : tile, to = STR ? tile / gx : 0;
  const TileRef tr = tile_of(a, t.n, TL, tx, to);
  if constexpr (LAYOUT == kTileX) {
    // each warp copies its own 32 / pw lines, nl' n consecutive elements, in
    // 16-byte pieces taken in order (512 contiguous bytes per warp-wide copy);
    // element e (from the warp's first line l0) goes to chunk l0 p + e / M
    // (a chunk holds M rows, M % V == 0)
    constexpr int V = 16 / sizeof(TIn), CS = M + V;
    static_assert(M % V == 0, "kTileX: whole 16-byte pieces per chunk");
    const int lpw = 32 / t.pw, l0 = (threadIdx.x >> 5) * lpw;
    const int lines = tr.nl - l0 < lpw ? tr.nl - l0 : lpw;
    if (lines > 0) {
      TIn* dst = slots + (size_t)buf * pipe_buf_elems<M, KS, TIn, LAYOUT>(bd, t.pw, t.p) + (size_t)l0 * t.p * CS;
      const TIn* gsrc = (const TIn*)a.in + tr.base + (int64_t)l0 * t.n;
      const int pieces = lines * t.n / V;
      for (int j = threadIdx.x & 31; j < pieces; j += 32) {
        const int e = j * V;
        cp_async_cg16(dst + (e / M) * CS + (e % M), gsrc + e);
      }
    }
    (void)NS;
  } else if constexpr (LAYOUT == kStridedWarp) {
    // line-fastest copy mapping (line gp, partition ip) into the slots of
    // the thread gp * pw + ip that solves that partition
    const int gp = threadIdx.x % kStridedLines, ip = threadIdx.x / kStridedLines;
    if (gp < tr.nl && ip < t.p) {
      const TIn* gline = (const TIn*)a.in + tr.base + gp;
      // own rows only: the halo rows are read from the neighbouring lanes' slots
      prefetch_rows<M, 0, true, TIn, false, kStridedWarpThreads>(
          slots + (size_t)buf * M * kStridedWarpThreads + slot_col<LAYOUT>(gp * t.pw + ip), gline, tr.es, ip * M, M,
          t.n);
    }
  } else if (tp.lane_ok && tp.g < tr.nl) {
    const TIn* gline = (const TIn*)a.in + tr.base + (LAYOUT == kDirectStrided ? (int64_t)tp.g : (int64_t)tp.g * t.n);
    constexpr bool VEC = LAYOUT == kDirectX && (M % (16 / sizeof(TIn))) == 0;
    prefetch_rows<M, KS, true, TIn, VEC>(slots + (size_t)buf * NS * bd + threadIdx.x, gline,
                                         LAYOUT == kDirectStrided ? tr.es : 1, tp.start, tp.size, t.n);
  }
  cp_async_commit();
}

// Persistent, software-pipelined variant of the direct layouts: each CTA
// walks the tiles tile = blockIdx.x, + gridDim.x, ... (tile -> (tx, to) with
// gx tiles along the first grid axis) and, before computing a tile, issues
// the asynchronous copies of the next tile's rows into the other half of a
// double buffer of thread-private shared-memory slots, so HBM traffic
// overlaps the arithmetic.  Shared memory: the message buffer (strided
// layout only, kCtaXchgSlots 64-bit slots per thread) followed by the two
// halves of the double buffer (pipe_buf_elems elements of TIn each).
template <int R, int M, int MODE, int KS, typename TIn, typename TOut, int LAYOUT, int ST = 0>
__global__ void __launch_bounds__(256, (refine_mode(MODE) || M == 32) ? 2 : 3)
    line_kernel_pipe(const LineArgs a, const DevLineTables t, const int gx, const int ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NS = M + 2 * KS;
  const int bd = blockDim.x;
  const size_t xbytes = LAYOUT == kDirectStrided ? (size_t)kCtaXchgSlots * bd * sizeof(unsigned long long) : 0;
  TIn* slots = reinterpret_cast<TIn*>(smem_raw + xbytes);
  const ThreadPart tp = thread_part<M, true, LAYOUT>(t);
  int tile = blockIdx.x, buf = 0, xflip = 0;
  if (tile < ntiles) prefetch_tile<M, KS, TIn, LAYOUT>(a, t, tp, gx, tile, slots, 0);
  if constexpr (LAYOUT == kStridedWarp) {
    // the copies land in other threads' slots: wait for this tile's, then a
    // barrier, which also shows that every thread is done with the previous
    // tile in the other half before the next copies go there
    for (; tile < ntiles; tile += gridDim.x, buf ^= 1) {
      cp_async_wait<0>();
      __syncthreads();
      const int next = tile + gridDim.x;
      if (next < ntiles) prefetch_tile<M, KS, TIn, LAYOUT>(a, t, tp, gx, next, slots, buf ^ 1);
      line_tile<R, M, MODE, KS, TIn, TOut, true, LAYOUT, true, ST>(a, t, a.in, a.out, tile % gx, tile / gx, smem_raw,
                                                                 slots + (size_t)buf * M * kStridedWarpThreads);
    }
    return;
  }
  // kTileX: a warp reads only the lines it copied, so warp barriers order
  // its lanes' copies and reads
  for (; tile < ntiles; tile += gridDim.x, buf ^= 1) {
    const int next = tile + gridDim.x;
    if (next < ntiles) {
      if constexpr (LAYOUT == kTileX) __syncwarp();  // the warp is done reading the other half
      prefetch_tile<M, KS, TIn, LAYOUT>(a, t, tp, gx, next, slots, buf ^ 1);
      cp_async_wait<1>();  // this tile's copies are done, the next tile's stay in flight
    } else {
      cp_async_wait<0>();
    }
    if constexpr (LAYOUT == kTileX) __syncwarp();  // every lane's copies of this tile have landed
    const int tx = LAYOUT == kDirectStrided ? tile % gx : tile, to = LAYOUT == kDirectStrided ? tile / gx : 0;
    line_tile<R, M, MODE, KS, TIn, TOut, true, LAYOUT, true, ST>(
        a, t, a.in, a.out, tx, to, smem_raw,
        slots + (size_t)buf * pipe_buf_elems<M, KS, TIn, LAYOUT>(bd, t.pw, t.p), &xflip);
  }
}

}  // namespace cbs
