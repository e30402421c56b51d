// cbs_long_warp.cuh -- long x-lines with one warp per segment and one launch
// per segment size (no separate end-row and interface passes).
//
// Segments have r interface rows and a bulk of 32 (or 31) inner partitions
// of 16 rows, one per lane.  The path applies when the outer interface
// system is decoupled to FP64 rounding: its coupling blocks L-hat, U-hat are
// below 2^-60 of the diagonal blocks D-hat (they shrink like the corner
// entries of D_i^{-1}, i.e. geometrically in the 512 bulk rows), so every
// PCR stage reduces to a local product and x~_i = D-hat^{-1} b-hat_i.  b-hat_i
// (Eq. 21) needs the last r rows of y_{i-1} and the first r rows of y_i, each
// a truncated dot product of K input rows with rows of D^{-1} (the long-line
// reading of Sec. 4: only those rows cross segments).
//
// A CTA takes kLongWarps consecutive segments of one line.  Each warp stages
// its bulk rows in shared memory (lane i's row k at slot k * 33 + i), forms
// the end rows of its own y_i from them, and the CTA's first and last warps
// also those of the neighbouring segments outside the CTA (halo rows read
// from global memory).  One barrier shares the ends; each warp then forms
// x~_i and x~_{i+1}, moves their couplings to the right-hand side of its bulk
// rows (Eq. 9) and runs the inner partition solve (FP32 + refinement with an
// FP64-accurate residual, or FP64 / FP32) in registers with shuffled
// messages.  The results leave through the same slots, one row per lane per
// store instruction.
#pragma once
#include "cbs_line.cuh"
#include "cbs_long.cuh"

namespace cbs {

namespace {

constexpr int kWarpM = 16;         // rows per lane
constexpr int kSlot = 33;          // padded row stride of a warp's slots
constexpr int kSlotsPerWarp = kWarpM * kSlot;

// Dot products of one CTA: a left and a right end (R rows each) for each of
// the kLongWarps + 1 segment boundaries, each spread over kTpd<R> threads.
template <int R> constexpr int kNdot = (kLongWarps + 1) * 2 * R;
template <int R> constexpr int kTpd = kLongWarps * 32 / kNdot<R>;

// acc += g b in double-float, g = gh + gl and b an input element (exact FP32,
// or an FP64 value split into two floats).
template <typename TIn>
__device__ __forceinline__ void df_madd(float& ah, float& al, float gh, float gl, TIn b) {
  const f2 bs = split_in(b);
  const float p = __fmul_rn(gh, bs.hi);
  const float pe = __fmaf_rn(gh, bs.hi, -p);
  const f2 s = two_sum(ah, p);
  ah = s.hi;
  al += (s.lo + pe) + (gl * bs.hi + gh * bs.lo);
}

// a2-a4 for the lane's inner partition of 16 rows (whole-size, acyclic inner
// system of P <= 32 partitions; lanes >= P hold zeros and zero blocks): on
// entry v holds the partition's right-hand side, on exit its solution.  Bulk
// in T, interface in TI through the compact stage list `f`.
template <typename T, int R, typename TI>
__device__ __forceinline__ void lw_solve(T (&v)[kWarpM], const int lane, const int P, const DevLineTables& t,
                                         const LwIface& f) {
  constexpr int M = kWarpM, NB = M - R, F = 2 * R + 1, rr = R * R;
  // a2: y = D_i^{-1} b (pre-factorised LU of the bulk block, Eq. 17)
#pragma unroll
  for (int j = 0; j < NB; j++) {
    T s = v[R + j];
#pragma unroll
    for (int q = 1; q <= R; q++)
      if (j - q >= 0) s -= Tab<T>::fac(t, j * F + q - 1) * v[R + j - q];
    v[R + j] = s;
  }
#pragma unroll
  for (int j = NB - 1; j >= 0; j--) {
    T s = Tab<T>::fac(t, j * F + R) * v[R + j];
#pragma unroll
    for (int q = 1; q <= R; q++)
      if (j + q < NB) s -= Tab<T>::fac(t, j * F + R + q) * v[R + j + q];
    v[R + j] = s;
  }
  // a3: b-hat_i = b~_i - L~ y_{i-1}[last r] - U~ y_i[first r]   (Eq. 21)
  TI xt[R];
#pragma unroll
  for (int q = 0; q < R; q++) xt[q] = (TI)v[q];
#pragma unroll
  for (int e = 0; e < R; e++) {
    const T yp = __shfl_sync(kFull, v[M - R + e], lane > 0 ? lane - 1 : 0);
#pragma unroll
    for (int q = 0; q < R; q++) {
      if (lane > 0) xt[q] -= ITab<TI>::Lt(t, q, e) * (TI)yp;
      xt[q] -= ITab<TI>::Ut(t, q, e) * (TI)v[R + e];
    }
  }
  // a3: the acting stages of block PCR (acyclic, Sec. 4), per-lane blocks;
  // a stage's messages carry the values from before the stage
  const TI* tab = static_cast<const TI*>(f.tab) + lane;
#pragma unroll 1
  for (int en = 0; en < f.ne; en++) {
    const TI* b = tab + f.off[en] * 32;
    const int fl = f.flags[en];
    TI xm[R], xp[R], nx[R];
    if (fl & 1) {
      const int s = f.s[en];
#pragma unroll
      for (int q = 0; q < R; q++) {  // out-of-range partners carry zero blocks
        xm[q] = __shfl_sync(kFull, xt[q], lane >= s ? lane - s : lane);
        xp[q] = __shfl_sync(kFull, xt[q], lane + s < 32 ? lane + s : lane);
      }
    }
    int o = 0;
    if (fl & 2) {
#pragma unroll
      for (int q = 0; q < R; q++) {
        TI acc = TI(0);
#pragma unroll
        for (int e = 0; e < R; e++) acc += __ldg(b + (q * R + e) * 32) * xt[e];
        nx[q] = acc;
      }
      o = rr;
    } else {
#pragma unroll
      for (int q = 0; q < R; q++) nx[q] = xt[q];
    }
    if (fl & 1) {
#pragma unroll
      for (int q = 0; q < R; q++)
#pragma unroll
        for (int e = 0; e < R; e++)
          nx[q] -= __ldg(b + (o + q * R + e) * 32) * xm[e] + __ldg(b + (o + rr + q * R + e) * 32) * xp[e];
    }
#pragma unroll
    for (int q = 0; q < R; q++) xt[q] = nx[q];
  }
  // a4: back-substitution x_i = y_i - S x~_i - R x~_{i+1} (Eq. 22); the last
  // partition has no next interface
  T xa[R], xb[R];
#pragma unroll
  for (int q = 0; q < R; q++) {
    const TI xn = __shfl_sync(kFull, xt[q], lane + 1 < 32 ? lane + 1 : lane);
    xa[q] = (T)xt[q];
    xb[q] = lane + 1 < P ? (T)xn : T(0);
  }
#pragma unroll
  for (int j = 0; j < NB; j++) {
    T s = v[R + j];
#pragma unroll
    for (int q = 0; q < R; q++) {
      s -= Tab<T>::sr(t, true, j * 2 * R + q) * xa[q];
      s -= Tab<T>::sr(t, true, j * 2 * R + R + q) * xb[q];
    }
    v[R + j] = s;
  }
#pragma unroll
  for (int q = 0; q < R; q++) v[q] = xa[q];
}

}  // namespace

// Shared memory of one CTA for truncation length K and input element size.
__host__ __device__ constexpr size_t lw_off_halo() { return (size_t)kLongWarps * kSlotsPerWarp * 8; }
template <int R>
__host__ __device__ constexpr size_t lw_bytes(int K, int in_size) {
  return lw_off_halo() + (size_t)(2 * K * in_size + 15) / 16 * 16 + (size_t)kNdot<R> * kTpd<R> * 8 +
         (size_t)(kLongWarps + 1) * R * 8 * 4;
}

// Phase D of a segment, for one warp: D_i x_i = b_i - couplings (Eq. 9) by
// the inner partition method in registers (a lane per partition), the rows
// read from the warp's slots S (lane i's row k at k * 33 + i) and the results
// written back to them as TOut.  cF0 / cL0: the coupling terms of the first
// and last R bulk rows (FP64).  Returns whether this lane's result left the
// FP32 range (refinement modes).
template <int R, int MODE, typename TIn, typename TOut, bool SW1>
__device__ __forceinline__ bool lw_segment_solve(TIn* S, const double* cF0, const double* cL0, const int lane,
                                                 const LongArgs& a, const DevLineTables& tin, const LongWarpArgs& wa) {
  const int P = tin.p;  // 32 or 31 inner partitions
  const bool lane_ok = lane < P;
  double cF[R], cL[R];
#pragma unroll
  for (int j = 0; j < R; j++) {
    cF[j] = lane == 0 ? cF0[j] : 0.0;
    cL[j] = lane == P - 1 ? cL0[j] : 0.0;
  }
  TOut* O = reinterpret_cast<TOut*>(S);
  WarpXchg xch{32};
  using TIR = typename std::conditional<MODE == kModeRefineI64, double, float>::type;
  bool bad = false;
  if constexpr (!refine_mode(MODE)) {
    using T = typename std::conditional<MODE == kModeF64, double, float>::type;
    T v[kWarpM];
#pragma unroll
    for (int k = 0; k < kWarpM; k++) {
      T val = lane_ok ? conv<T>(S[k * kSlot + lane]) : T(0);
      if (k < R) val -= conv<T>(cF[k]);
      if (k >= kWarpM - R) val -= conv<T>(cL[k - (kWarpM - R)]);
      v[k] = val;
    }
    lw_solve<T, R, T>(v, lane, P, tin, wa.ifc);
    __syncwarp();  // every lane has read its input slots
#pragma unroll
    for (int k = 0; k < kWarpM; k++) O[k * kSlot + lane] = conv<TOut>(v[k]);
  } else {
    float bh[kWarpM], blo[kWarpM], xh[kWarpM], xlo[kWarpM], v[kWarpM];
    f2 sF[R], sL[R];
#pragma unroll
    for (int e = 0; e < R; e++) {
      sF[e] = split_f64(cF[e]);
      sL[e] = split_f64(cL[e]);
    }
#pragma unroll
    for (int k = 0; k < kWarpM; k++) {
      const f2 sv = lane_ok ? split_in(S[k * kSlot + lane]) : f2{0.f, 0.f};
      if (k < R || k >= kWarpM - R) {  // the rows that carry a coupling term
        const f2 c = k < R ? sF[k] : sL[k - (kWarpM - R)];
        const f2 dd = two_sum(sv.hi, -c.hi);  // subtract the coupling exactly
        bh[k] = dd.hi;
        blo[k] = dd.lo + (sv.lo - c.lo);
      } else {  // FP32 input: the low part is the constant zero
        bh[k] = sv.hi;
        blo[k] = sv.lo;
      }
      v[k] = bh[k];
    }
    lw_solve<float, R, TIR>(v, lane, P, tin, wa.ifc);
#pragma unroll
    for (int k = 0; k < kWarpM; k++) {
      xh[k] = v[k];
      xlo[k] = 0.f;
    }
    if constexpr (SW1) {  // one sweep: x = x0 + delta, added in FP64 at the output
      residual_sym2<R, kWarpM, false>(bh, blo, xh, xlo, v, lane, tin, xch);
      lw_solve<float, R, TIR>(v, lane, P, tin, wa.ifc);
      __syncwarp();  // every lane has read its input slots
#pragma unroll
      for (int k = 0; k < kWarpM; k++) {  // values in the FP32 range: normal or zero (below 2^-126: flushed)
        bad |= !(fabsf(xh[k]) <= 3.4e38f);  // inf or nan (the FP32 range was left)
        O[k * kSlot + lane] = (TOut)(f32_to_f64_nz(xh[k]) + f32_to_f64_nz(v[k]));
      }
    }
    for (int sw = 0; sw < (SW1 ? 0 : a.sweeps); sw++) {
      if (sw == 0) residual_sym2<R, kWarpM, false>(bh, blo, xh, xlo, v, lane, tin, xch);
      else residual_sym2<R, kWarpM, true>(bh, blo, xh, xlo, v, lane, tin, xch);
      lw_solve<float, R, TIR>(v, lane, P, tin, wa.ifc);
#pragma unroll
      for (int k = 0; k < kWarpM; k++) {
        const f2 t = two_sum(xh[k], v[k]);
        xh[k] = t.hi;
        xlo[k] = xlo[k] + t.lo;
      }
    }
    if constexpr (!SW1) {
      __syncwarp();  // every lane has read its input slots
#pragma unroll
      for (int k = 0; k < kWarpM; k++) {  // values in the FP32 range: normal or zero (below 2^-126: flushed)
        bad |= !(fabsf(xh[k]) <= 3.4e38f);  // inf or nan (the FP32 range was left)
        O[k * kSlot + lane] = (TOut)(f32_to_f64_nz(xh[k]) + f32_to_f64_nz(xlo[k]));
      }
    }
  }
  return bad && lane_ok;
}

// One CTA's work: segments seg0 + chunk * kLongWarps .. of `line`, shared
// memory at smem (lw_bytes<R>(K, sizeof(TIn)) bytes, 16-byte aligned).  All
// threads of the CTA (kLongWarps warps) call it; it ends without a barrier.
// SW1: the plan runs one refinement sweep (compiled apart: the sum x0 +
// delta then needs no extra registers across the second solve).
template <int R, int MODE, typename TIn, typename TOut, bool SW1 = false>
__device__ __forceinline__ void long_warp_item(const LongArgs& a, const DevLineTables& tin, const LongWarpArgs& wa,
                                               const int chunk, const int64_t line, unsigned char* smem) {
  constexpr int W = kLongWarps, ND = kNdot<R>, TPD = kTpd<R>;
  // [W][kSlotsPerWarp] 8-byte slots (a warp's input rows as TIn, then its
  // results as TOut) | halo rows: K before the chunk, K after | dot-product
  // partials [ND][TPD] (float pairs) | per boundary k = 0..W: b~_k, x~_k, the
  // coupling terms of segment k's first bulk rows and of segment k-1's last
  // (R doubles each)
  const int K = a.K;
  TIn* Hp = reinterpret_cast<TIn*>(smem + lw_off_halo());
  TIn* Hn = Hp + K;
  float2* Pp = reinterpret_cast<float2*>(smem + lw_off_halo() + (size_t)(2 * K * sizeof(TIn) + 15) / 16 * 16);
  double* Bt = reinterpret_cast<double*>(Pp + ND * TPD);
  double* Xt = Bt + (W + 1) * R;
  double* CF = Xt + (W + 1) * R;
  double* CL = CF + (W + 1) * R;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto slots = [&](int k) { return reinterpret_cast<TIn*>(smem + (size_t)k * kSlotsPerWarp * 8); };

  const int sfirst = wa.seg0 + chunk * W;
  const int nv = min(W, wa.seg0 + wa.nseg - sfirst);  // segments of this CTA
  const bool valid = w < nv;
  const int N = seg_rows(a, sfirst) - R;  // bulk rows, the same for every segment of a launch
  const TIn* bl = (const TIn*)a.in + line * a.n;
  TOut* xl = (TOut*)a.out + line * a.n;
  const int64_t S0 = seg_start(a, sfirst);
  const int64_t s0 = S0 + (int64_t)w * (N + R);

  // A: every warp stages its segment's bulk rows and b~; warp 0 the last K
  // bulk rows of the segment before the CTA, warp W - 1 the interface rows
  // and first K bulk rows of the segment after it (both cyclic)
  // lane l moves bulk rows l + 32 t (coalesced): slot (l & 15) * 33 + (l >> 4) + 2 t
  const int sb = (lane & 15) * kSlot + (lane >> 4);
  if (valid) {
    TIn* S = slots(w) + sb;
    const TIn* bb = bl + s0 + R + lane;
#pragma unroll
    for (int t = 0; t < kWarpM; t++)
      if (lane + 32 * t < N) S[2 * t] = __ldg(bb + 32 * t);
    if (lane < R) Bt[w * R + lane] = (double)__ldg(bl + s0 + lane);
  }
  if (w == 0) {
    const int64_t e = (S0 == 0 ? a.n : S0) - 1;  // last bulk row of the segment before
    for (int j = lane; j < K; j += 32) Hp[j] = __ldg(bl + e - j);
  } else if (w == W - 1) {
    const int sn = sfirst + nv;
    const int64_t s1 = sn == a.p ? 0 : S0 + (int64_t)nv * (N + R);  // the segment after
    for (int j = lane; j < K; j += 32) Hn[j] = __ldg(bl + s1 + R + j);
    if (lane < R) Bt[nv * R + lane] = (double)__ldg(bl + s1 + lane);
  }
  __syncthreads();

  // B: the end rows of y for every boundary k = 0..nv (Sec. 4: only these
  // cross segments): left end y_{k-1}[N - R + e] and right end y_k[e], each
  // a truncated dot product of K rows with a row of D^{-1} (persymmetric:
  // row R - 1 - e serves the last rows), in double-float
  {
    const int d = threadIdx.x / TPD, part = threadIdx.x % TPD;
    const int k = d / (2 * R), e = d % (2 * R);
    if (d < ND && k <= nv) {
      float ah = 0.f, al = 0.f;
      const bool left = e < R;
      const int g = left ? R - 1 - e : e - R;
      const float* Gh = wa.Gh + g * K;
      const float* Gl = wa.Gl + g * K;
      if (left) {
        const TIn* S = k > 0 ? slots(k - 1) : nullptr;
        for (int j = part; j < K; j += TPD) {
          const int row = N - 1 - j;
          const TIn b = k > 0 ? S[(row & 15) * kSlot + (row >> 4)] : Hp[j];
          df_madd(ah, al, __ldg(Gh + j), __ldg(Gl + j), b);
        }
      } else {
        const TIn* S = k < nv ? slots(k) : nullptr;
        for (int j = part; j < K; j += TPD) {
          const TIn b = k < nv ? S[(j & 15) * kSlot + (j >> 4)] : Hn[j];
          df_madd(ah, al, __ldg(Gh + j), __ldg(Gl + j), b);
        }
      }
      Pp[d * TPD + part] = make_float2(ah, al);
    }
  }
  __syncthreads();

  // C: one lane per boundary: x~_k = D-hat^{-1} (b~_k - L~ y_{k-1}[last] -
  // U~ y_k[first]) (Eq. 21, the decoupled outer system) and the Eq. 9
  // couplings of the bulk rows next to it
  if (w == 0 && lane <= nv) {
    const int k = lane;
    double y[2 * R];
#pragma unroll
    for (int e = 0; e < 2 * R; e++) {
      float h = 0.f, l = 0.f;
      for (int q = 0; q < TPD; q++) {
        const float2 v = Pp[(k * 2 * R + e) * TPD + q];
        const f2 s = two_sum(h, v.x);
        h = s.hi;
        l += s.lo + v.y;
      }
      y[e] = f32_to_f64(h) + f32_to_f64(l);
    }
    double bh[R], xt[R];
#pragma unroll
    for (int q = 0; q < R; q++) {
      double v = Bt[k * R + q];
#pragma unroll
      for (int e = 0; e < R; e++) v -= wa.Lt[q * R + e] * y[e] + wa.Ut[q * R + e] * y[R + e];
      bh[q] = v;
    }
#pragma unroll
    for (int q = 0; q < R; q++) {
      double v = 0.0;
#pragma unroll
      for (int e = 0; e < R; e++) v += wa.Dinv[q * R + e] * bh[e];
      xt[q] = v;
      Xt[k * R + q] = v;
    }
    // bulk row j < R of segment k couples to x~_k[q] at band offset q - R - j;
    // bulk row N - R + j of segment k - 1 at offset q + R - j
#pragma unroll
    for (int j = 0; j < R; j++) {
      double c = 0.0, dd = 0.0;
#pragma unroll
      for (int q = 0; q < R; q++) {
        if (q >= j) c += a.band[q - j] * xt[q];
        if (q <= j) dd += a.band[q - j + 2 * R] * xt[q];
      }
      CF[k * R + j] = c;
      CL[k * R + j] = dd;
    }
  }
  __syncthreads();
  if (valid) {  // no barrier below

  // D: the segment's bulk: D_i x_i = b_i - (couplings) (Eq. 9), the inner
  // partition method in registers, a lane per partition
  const bool bad = lw_segment_solve<R, MODE, TIn, TOut, SW1>(slots(w), CF + w * R, CL + (w + 1) * R, lane, a, tin, wa);
  TOut* O = reinterpret_cast<TOut*>(slots(w));
  if (__any_sync(kFull, bad) && lane == 0 && wa.status) atomicExch(wa.status, (int)CBS_ERR_RANGE);
  __syncwarp();
  TOut* xb0 = xl + s0 + R + lane;
#pragma unroll
  for (int t = 0; t < kWarpM; t++)  // lane l: bulk rows l + 32 t (coalesced)
    if (lane + 32 * t < N) xb0[32 * t] = O[sb + 2 * t];
  if (lane < R) xl[s0 + lane] = (TOut)Xt[w * R + lane];  // the segment's interface rows
  }
}

// ---------------------------------------------------------------- y/z lines
// Dot products of one y/z CTA: per line, the left and right ends of its two
// boundaries (b~_s side: y_{s-1}[last], y_s[first]; b~_{s+1} side: y_s[last],
// y_{s+1}[first]), R rows each.
template <int R> constexpr int kNdotYZ = kLongWarps * 4 * R;
template <int R> constexpr int kTpdYZ = kLongWarps * 32 / kNdotYZ<R>;

// Shared memory of a y/z CTA: slots, halos [2][W][K] TIn, partials, and per
// line b~ and x~ of both boundaries and the coupling terms (R doubles each).
template <int R>
__host__ __device__ constexpr size_t lwyz_off_part(int K, int in_size) {
  return lw_off_halo() + (size_t)(2 * kLongWarps * K * in_size + 15) / 16 * 16;
}
template <int R>
__host__ __device__ constexpr size_t lwyz_bytes(int K, int in_size) {
  return lwyz_off_part<R>(K, in_size) + (size_t)kNdotYZ<R> * kTpdYZ<R> * 8 + (size_t)kLongWarps * R * 8 * 6;
}

// One y/z CTA: segment s of the lines line0 .. line0 + kLongWarps - 1
// (consecutive line indices: adjacent in x), a warp per line.  Rows of the
// group are moved cooperatively, thread t taking line t % kLongWarps of rows
// t / kLongWarps + 32 m, so that a warp's access covers 8 rows of 4 adjacent
// lines (32-byte runs for FP64); the halo rows of the neighbouring segments
// are read the same way.  Then as for x-lines: double-float end rows spread
// over the CTA, x~ of every (line, boundary) by one lane, each warp's
// segment solve, results out through the slots.
template <int R, int MODE, typename TIn, typename TOut, bool SW1 = false>
__device__ __forceinline__ void long_warp_item_yz(const LongArgs& a, const DevLineTables& tin, const LongWarpArgs& wa,
                                                  const int s, const int64_t line0, unsigned char* smem) {
  constexpr int W = kLongWarps, ND = kNdotYZ<R>, TPD = kTpdYZ<R>;
  static_assert(W == 4, "cooperative moves: 8 rows x 4 lines per warp access");
  const int K = a.K;
  TIn* Hp = reinterpret_cast<TIn*>(smem + lw_off_halo());  // [W][K]
  TIn* Hn = Hp + W * K;
  float2* Pp = reinterpret_cast<float2*>(smem + lwyz_off_part<R>(K, (int)sizeof(TIn)));
  double* Bt = reinterpret_cast<double*>(Pp + ND * TPD);  // [W][2][R]
  double* Xt = Bt + W * 2 * R;                            // [W][2][R]
  double* CF = Xt + W * 2 * R;                            // [W][R]
  double* CL = CF + W * R;                                // [W][R]
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  auto slots = [&](int k) { return reinterpret_cast<TIn*>(smem + (size_t)k * kSlotsPerWarp * 8); };
  const LongGeom& gm = wa.gm;
  const int64_t es = gm.es;

  const int N = seg_rows(a, s) - R;
  const int64_t s0 = seg_start(a, s);
  const int64_t s1 = s + 1 == a.p ? 0 : s0 + N + R;  // the next segment (cyclic)
  const int64_t pe = (s0 == 0 ? a.n : s0) - 1;       // last bulk row of the previous one
  // A: this thread's line of the group and its rows
  {
    const int g = t & (W - 1), r0 = t >> 2;
    const int64_t line = line0 + g;
    if (line < a.lines) {
      const TIn* b = (const TIn*)a.in + long_base(a, gm, line);
      TIn* S = slots(g);
#pragma unroll 4
      for (int m = 0; m < kWarpM; m++) {
        const int j = r0 + 32 * m;
        if (j < N) S[(j & 15) * kSlot + (j >> 4)] = __ldg(b + (s0 + R + j) * es);
      }
      for (int j = r0; j < K; j += 32) {
        Hp[g * K + j] = __ldg(b + (pe - j) * es);
        Hn[g * K + j] = __ldg(b + (s1 + R + j) * es);
      }
      if (r0 < R) {
        Bt[(g * 2 + 0) * R + r0] = (double)__ldg(b + (s0 + r0) * es);
        Bt[(g * 2 + 1) * R + r0] = (double)__ldg(b + (s1 + r0) * es);
      }
    }
  }
  __syncthreads();

  // B: the four end rows of y of every line (double-float dot products)
  {
    const int d = t / TPD, part = t % TPD;
    const int g = d / (4 * R), e = d % (4 * R);
    if (d < ND && line0 + g < a.lines) {
      const int kind = e / R, q = e % R;  // 0: y_{s-1} last, 1: y_s first, 2: y_s last, 3: y_{s+1} first
      const bool last = kind == 0 || kind == 2;
      const int grow = last ? R - 1 - q : q;
      const float* Gh = wa.Gh + grow * K;
      const float* Gl = wa.Gl + grow * K;
      const TIn* S = slots(g);
      float ah = 0.f, al = 0.f;
      for (int j = part; j < K; j += TPD) {
        TIn b;
        if (kind == 0) b = Hp[g * K + j];
        else if (kind == 3) b = Hn[g * K + j];
        else {
          const int row = kind == 1 ? j : N - 1 - j;
          b = S[(row & 15) * kSlot + (row >> 4)];
        }
        df_madd(ah, al, __ldg(Gh + j), __ldg(Gl + j), b);
      }
      Pp[d * TPD + part] = make_float2(ah, al);
    }
  }
  __syncthreads();

  // C: one lane per (line, boundary): x~ = D-hat^{-1} (b~ - L~ y_left - U~
  // y_right) (Eq. 21, the decoupled outer system) and the Eq. 9 couplings
  if (w == 0 && lane < 2 * W && line0 + (lane >> 1) < a.lines) {
    const int g = lane >> 1, bd = lane & 1;
    double y[2 * R];
#pragma unroll
    for (int e = 0; e < 2 * R; e++) {
      float h = 0.f, l = 0.f;
      const int d = g * 4 * R + bd * 2 * R + e;
      for (int q = 0; q < TPD; q++) {
        const float2 v = Pp[d * TPD + q];
        const f2 u = two_sum(h, v.x);
        h = u.hi;
        l += u.lo + v.y;
      }
      y[e] = f32_to_f64(h) + f32_to_f64(l);
    }
    double bh[R], xt[R];
#pragma unroll
    for (int q = 0; q < R; q++) {
      double v = Bt[(g * 2 + bd) * R + q];
#pragma unroll
      for (int e = 0; e < R; e++) v -= wa.Lt[q * R + e] * y[e] + wa.Ut[q * R + e] * y[R + e];
      bh[q] = v;
    }
#pragma unroll
    for (int q = 0; q < R; q++) {
      double v = 0.0;
#pragma unroll
      for (int e = 0; e < R; e++) v += wa.Dinv[q * R + e] * bh[e];
      xt[q] = v;
      Xt[(g * 2 + bd) * R + q] = v;
    }
    // boundary s: the segment's first bulk rows (offset q - R - j); boundary
    // s + 1: its last bulk rows (offset q + R - j)
#pragma unroll
    for (int j = 0; j < R; j++) {
      double c = 0.0;
#pragma unroll
      for (int q = 0; q < R; q++) {
        if (bd == 0 && q >= j) c += a.band[q - j] * xt[q];
        if (bd == 1 && q <= j) c += a.band[q - j + 2 * R] * xt[q];
      }
      (bd == 0 ? CF : CL)[g * R + j] = c;
    }
  }
  __syncthreads();

  // D: each warp's segment
  bool bad = false;
  if (line0 + w < a.lines) bad = lw_segment_solve<R, MODE, TIn, TOut, SW1>(slots(w), CF + w * R, CL + w * R, lane, a, tin, wa);
  if (__any_sync(kFull, bad) && lane == 0 && wa.status) atomicExch(wa.status, (int)CBS_ERR_RANGE);
  __syncthreads();  // the results of every warp, out cooperatively
  {
    const int g = t & (W - 1), r0 = t >> 2;
    const int64_t line = line0 + g;
    if (line < a.lines) {
      TOut* x = (TOut*)a.out + long_base(a, gm, line);
      const TOut* O = reinterpret_cast<const TOut*>(slots(g));
#pragma unroll 4
      for (int m = 0; m < kWarpM; m++) {
        const int j = r0 + 32 * m;
        if (j < N) x[(s0 + R + j) * es] = O[(j & 15) * kSlot + (j >> 4)];
      }
      if (r0 < R) x[(s0 + r0) * es] = (TOut)Xt[(g * 2 + 0) * R + r0];  // the segment's interface rows
    }
  }
}

}  // namespace cbs
