// cbs_var.cuh -- variable-coefficient cyclic tridiagonal lines (row-wise
// alpha_i read from a device field) and the adjoint of the compact
// derivative.
//
// With per-point bands nothing is RHS-independent across lines, so the kernel
// runs the paper's whole algorithm per line on the fly:
//   - Thomas factorisation of each bulk block D_i together with the three
//     right-hand sides of Eq. 15-17 (S_i, R_i, y_i), in registers;
//   - the reduced blocks of Eq. 18-21 from the neighbours' boundary values;
//   - block PCR with detach / reattach on (W, L-hat, U-hat, x~) exactly as in
//     Algorithms 1-4, one lane per partition, warp shuffles as the messages;
//   - back-substitution Eq. 22.
// Forward:  x = A(alpha)^{-1} S f.
// Adjoint:  lambda = A^{-T} g (A^T has sub-diagonal alpha_{i-1} and
//           super-diagonal alpha_{i+1}), grad_f = S^T lambda and
//           grad_alpha_i = -lambda_i (x_{i-1} + x_{i+1}).
#pragma once
#include "cbs_line.cuh"

namespace cbs {

struct VarArgs {
  const void* f;      // forward: field f (or b when KS == 0); adjoint: g
  const void* alpha;  // per-point alpha_i
  const void* x;      // adjoint: the forward solution (for grad_alpha), may be null
  void* out;          // forward: x; adjoint: grad_f (S^T lambda) or lambda when KS == 0
  void* lam;          // adjoint: optional lambda output
  void* grad_alpha;   // adjoint: optional grad_alpha output
  int64_t nx, ny, nz, nlines;
  int dir;
  double w[kMaxRhsTerms];
  int stage_type[kMaxStages], stage_s[kMaxStages], stage_na[kMaxStages];
  int* status;
};

// Pivot reciprocals of the per-line factorisation.  The FP64 pipe bounds
// this kernel, and an IEEE division costs several FP64 instructions more
// than Newton-Raphson on the hardware's approximate reciprocal: r <- r + r e
// with e = 1 - v r squares the relative error at every step, so two steps
// from the approximation reach FP64 rounding (within an ulp or two; not
// correctly rounded).  The pivots are normal numbers (|1 - alpha^2 ...| of a
// diagonally dominant band), where the flush-to-zero variant is exact.
__device__ __forceinline__ double rcp_(double v) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(v));
  double e = fma(-v, r, 1.0);
  r = fma(r, e, r);
  e = fma(-v, r, 1.0);
  return fma(r, e, r);
}
// FP32: the hardware reciprocal (about one ulp) is accurate enough for the
// FP32 solve.
__device__ __forceinline__ float rcp_(float v) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}

// Variable-band line kernel.  ADJ = false: forward solve; ADJ = true:
// transposed solve + S^T + band gradient.  T: arithmetic type, TG: element
// type of the fields.
template <int M, int KS, bool ADJ, typename T, typename TG>
__global__ void __launch_bounds__(256, 1) var_kernel(const VarArgs a, const DevLineTables t) {
  constexpr int KA = KS > 0 ? KS : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TG* Sf = reinterpret_cast<TG*>(smem_raw);
  const int pw = t.pw;
  const int TL = blockDim.x / pw;
  TG* Sa = Sf + (size_t)TL * t.lsz;
  TG* Sx = Sa + (size_t)TL * t.lsz;
  const TileRef tr = tile_of(a, t.n, TL, blockIdx.x, blockIdx.y);
  const int nl = tr.nl;
  const int g = threadIdx.x / pw, i = threadIdx.x % pw;
  const int p = t.p;
  const bool lane_ok = i < p;
  const bool ok = lane_ok && g < nl;
  int start = 0, size = 2;
  if (lane_ok) partition_of(t, i, start, size);
  const int n = t.n;
  const int N = size - 1;  // bulk rows
  const bool want_ga = ADJ && a.x != nullptr && a.grad_alpha != nullptr;

  tile_copy<true, const TG, TG>(tr, t, Sf, (const TG*)a.f);
  tile_copy<true, const TG, TG>(tr, t, Sa, (const TG*)a.alpha);
  if (want_ga) tile_copy<true, const TG, TG>(tr, t, Sx, (const TG*)a.x);
  __syncthreads();
  TG* SfL = Sf + g * t.lsz;
  TG* SaL = Sa + g * t.lsz;
  TG* SxL = Sx + g * t.lsz;
  auto rowval = [&](TG* base, int row) -> T {  // periodic row of this line
    row += (row < 0) ? n : 0;
    row -= (row >= n) ? n : 0;
    return ok ? (T)base[slot_of(t, row)] : T(0);
  };

  // right-hand side b (rows start .. start+size-1)
  T b[M];
  if (KS == 0 || ADJ) {
#pragma unroll
    for (int k = 0; k < M; k++) b[k] = (ok && k < size) ? (T)SfL[k * t.sp + i] : T(0);
  } else {
    T fw[M + KS], hh[KA];
#pragma unroll
    for (int q = 0; q < KS; q++) {
      fw[q] = rowval(SfL, start - KS + q);
      hh[q] = rowval(SfL, start + size + q);
    }
#pragma unroll
    for (int k = 0; k < M; k++) fw[KS + k] = (ok && k < size) ? (T)SfL[k * t.sp + i] : T(0);
#pragma unroll
    for (int k = 0; k < M; k++) {
      T s = T(0);
#pragma unroll
      for (int q = 1; q <= KS; q++) {
        const int kq = (k + q < M) ? k + q : M - 1;
        T up;
        if (k + q < M) up = sel(k + q < size, fw[KS + kq], pick<T, KA>(hh, k + q - size));
        else up = pick<T, KA>(hh, k + q - size);
        s += (T)a.w[q - 1] * (up - fw[KS + k - q]);
      }
      b[k] = s;
    }
  }
  // bands of this partition's rows: lo[k] = A[row, row-1], up[k] = A[row, row+1]
  T lo[M], upb[M];
  {
    T am = rowval(SaL, start - 1), ap;
#pragma unroll
    for (int k = 0; k < M; k++) {
      const T ak = (ok && k < size) ? (T)SaL[k * t.sp + i] : T(0);
      if (!ADJ) {
        lo[k] = ak;
        upb[k] = ak;
      } else {
        lo[k] = am;  // A^T[row, row-1] = alpha_{row-1}
        am = ak;
      }
    }
    if (ADJ) {
      // A^T[row, row+1] = alpha_{row+1}
      ap = rowval(SaL, start + size);
#pragma unroll
      for (int k = 0; k < M; k++) {
        const T nxt = (k + 1 < M) ? sel(k + 1 < size, (T)((ok && k + 1 < size) ? SaL[(k + 1 < M ? k + 1 : 0) * t.sp + i] : TG(0)), ap) : ap;
        upb[k] = nxt;
      }
    }
  }

  // ---- Thomas on D_i (rows 1..size-1) with right-hand sides b, L_i e, U_i e ----
  // forward: z = y-part, zs = S column, zr = R column
  T ipiv[M], c[M], y[M], sc[M], rc[M];
#pragma unroll
  for (int k = 0; k < M; k++) {
    ipiv[k] = T(0);
    c[k] = T(0);
    y[k] = T(0);
    sc[k] = T(0);
    rc[k] = T(0);
  }
  {
    T cprev = T(0), yprev = T(0), sprev = T(0);
#pragma unroll
    for (int j = 1; j < M; j++) {
      if (j < size) {
        const T l = (j == 1) ? T(0) : lo[j];
        const T piv = T(1) - l * cprev;
        const T ip = rcp_(piv);
        ipiv[j] = ip;
        c[j] = upb[j] * ip;   // scaled super-diagonal (last one unused)
        const T yj = (b[j] - l * yprev) * ip;
        const T sj = ((j == 1) ? lo[1] : -l * sprev) * ip;  // RHS of S: lo of bulk row 1
        y[j] = yj;
        sc[j] = sj;
        cprev = c[j];
        yprev = yj;
        sprev = sj;
      }
    }
    // R column RHS: up of the last bulk row; after forward elimination it is
    // upb[N] / piv[N] at row N = size-1 (selected without indexing)
    T rN = T(0);
#pragma unroll
    for (int k = 1; k < M; k++) rN = sel(k == size - 1, upb[k] * ipiv[k], rN);
    T rprev = T(0);
#pragma unroll
    for (int j = M - 1; j >= 1; j--) {
      if (j < size) {
        const bool last = (j == size - 1);
        const int jn = (j + 1 < M) ? j + 1 : j;  // compile-time clamp
        // backward substitution v_j = fwd_j - c_j v_{j+1} (none on the last row)
        y[j] = sel(last, y[j], y[j] - c[j] * y[jn]);
        sc[j] = sel(last, sc[j], sc[j] - c[j] * sc[jn]);
        const T rnew = sel(last, rN, -c[j] * rprev);
        rc[j] = rnew;
        rprev = rnew;
      }
    }
  }
  // boundary values: first bulk row (k = 1) and last bulk row (k = size-1)
  T y_last = T(0), s_last = T(0), r_last = T(0);
#pragma unroll
  for (int k = 1; k < M; k++) {
    const bool is = (k == size - 1);
    y_last = sel(is, y[k], y_last);
    s_last = sel(is, sc[k], s_last);
    r_last = sel(is, rc[k], r_last);
  }
  const int prev = (i == 0) ? p - 1 : i - 1;
  const int next = (i + 1 >= p) ? 0 : i + 1;
  const T yp = __shfl_sync(kFull, y_last, prev, pw);
  const T sp_ = __shfl_sync(kFull, s_last, prev, pw);
  const T rp = __shfl_sync(kFull, r_last, prev, pw);
  // interface row `start`: lo couples to the previous partition's last bulk
  // row (L~_i), up to this partition's first bulk row (U~_i)
  const T Lt = lo[0], Ut = upb[0];
  T W = T(1) - Lt * rp - Ut * sc[1];
  T Lh = -Lt * sp_;
  T Uh = -Ut * rc[1];
  T xt = b[0] - Lt * yp - Ut * y[1];

  // ---- Algorithms 1-4 on (L-hat, W, U-hat, x~), in the solve's precision ----
  // Once every coupling block of every line in the warp is below 2^-60
  // (FP64) / 2^-30 (FP32) of its diagonal block, the remaining steps change
  // nothing above rounding: PCR and detach steps are skipped and reattach /
  // final steps keep only their diagonal division.  The blocks shrink
  // geometrically with the partition size (diagonal dominance) and square at
  // every PCR step, so this usually ends the loop after a few steps.
  const T tiny = sizeof(T) == 8 ? T(8.673617379884035e-19) : T(9.313225746154785e-10);  // 2^-60, 2^-30
  // Singular (or numerically singular) interface system: a block divided by
  // that is zero, non-finite, or below 2^-40 (FP64) / 2^-16 (FP32) of the
  // magnitude of its row -- e.g. alpha = 1/2 on a cyclic line of even length,
  // whose symbol 1 + cos(theta) vanishes.  Reported as CBS_ERR_SINGULAR.
  const T sthr = sizeof(T) == 8 ? T(9.094947017729282e-13) : T(1.52587890625e-05);  // 2^-40, 2^-16
  bool sing = false;
  auto check = [&](T den, T scale) {
    if (!(fabs(den) > sthr * scale)) sing = true;  // also true for nan
  };
  bool decoupled = false;
  for (int st = 0; st < t.nstage; st++) {
    if (!decoupled)
      decoupled = __all_sync(kFull, !lane_ok || (fabs(Lh) <= tiny * fabs(W) && fabs(Uh) <= tiny * fabs(W)));
    if (decoupled) {
      const int type = a.stage_type[st], s = a.stage_s[st], na = a.stage_na[st];
      if (!lane_ok) continue;
      if (type == kFinal) {
        if (i < na) {
          const T den = t.cyclic ? (W + Lh + Uh) : W;
          check(den, fabs(W) + fabs(Lh) + fabs(Uh));
          xt = xt * rcp_(den);
        }
      } else if (type == kReattach) {
        if (i >= na && i < na + s) {
          check(W, fabs(W) + fabs(Lh) + fabs(Uh));
          xt = xt * rcp_(W);
        }
      }
      continue;
    }
    const int type = a.stage_type[st], s = a.stage_s[st], na = a.stage_na[st];
    int src1 = i, src2 = i;
    if (type == kDetach) {
      src1 = (i >= na - s && i < na) ? i + s : i;   // receives from the detached row i+s
      src2 = (i < s) ? i + na : i;                  // receives from the detached row i+na
    } else if (type == kPcr) {
      src1 = (i < na) ? (i + s) % na : i;
      src2 = (i < na) ? (i - s + na) % na : i;
    } else if (type == kReattach) {
      src1 = (i >= na && i < na + s) ? i - s : i;   // x~_{i-s}
      src2 = (i >= na && i < na + s) ? i - na : i;  // x~_{i+s} lives at i - na
    }
    if (!lane_ok) src1 = src2 = i;
    const T L1 = __shfl_sync(kFull, Lh, src1, pw), W1 = __shfl_sync(kFull, W, src1, pw);
    const T U1 = __shfl_sync(kFull, Uh, src1, pw), X1 = __shfl_sync(kFull, xt, src1, pw);
    const T L2 = __shfl_sync(kFull, Lh, src2, pw), W2 = __shfl_sync(kFull, W, src2, pw);
    const T U2 = __shfl_sync(kFull, Uh, src2, pw), X2 = __shfl_sync(kFull, xt, src2, pw);
    if (!lane_ok) continue;
    if (type == kDetach) {
      if (i >= na - s && i < na) {
        check(W1, fabs(W1) + fabs(L1) + fabs(U1));
        const T k = Uh * rcp_(W1);
        W -= k * L1;
        xt -= k * X1;
        Uh = -k * U1;
      }
      if (i < s) {
        check(W2, fabs(W2) + fabs(L2) + fabs(U2));
        const T k = Lh * rcp_(W2);
        W -= k * U2;
        xt -= k * X2;
        Lh = -k * L2;
      }
    } else if (type == kPcr) {
      if (i < na) {
        check(W1, fabs(W1) + fabs(L1) + fabs(U1));
        check(W2, fabs(W2) + fabs(L2) + fabs(U2));
        const T kp = Uh * rcp_(W1), km = Lh * rcp_(W2);
        const T Wn = W - kp * L1 - km * U2;
        const T xn = xt - kp * X1 - km * X2;
        const T Ln = -km * L2, Un = -kp * U1;
        W = Wn;
        xt = xn;
        Lh = Ln;
        Uh = Un;
      }
    } else if (type == kFinal) {
      if (i < na) {
        const T den = t.cyclic ? (W + Lh + Uh) : W;
        check(den, fabs(W) + fabs(Lh) + fabs(Uh));
        xt = xt * rcp_(den);
      }
    } else {
      if (i >= na && i < na + s) {
        check(W, fabs(W) + fabs(Lh) + fabs(Uh));
        xt = (xt - Lh * X1 - Uh * X2) * rcp_(W);
      }
    }
  }
  const T xn = __shfl_sync(kFull, xt, next, pw);
  const T xa = xt, xb = xn;
  // back-substitution (Eq. 22); row 0 is the interface unknown
  T x[M];
  x[0] = xa;
#pragma unroll
  for (int k = 1; k < M; k++) x[k] = y[k] - sc[k] * xa - rc[k] * xb;
  // a zero or non-finite bulk pivot shows as a non-finite result (integer
  // tests: no FP64-pipe work)
  if (ok) {
    unsigned nf = 0u;
#pragma unroll
    for (int k = 0; k < M; k++) {
      if (k < size) {
        if constexpr (sizeof(T) == 8) nf |= (((unsigned)__double2hiint((double)x[k]) & 0x7ff00000u) == 0x7ff00000u) ? 1u : 0u;
        else nf |= ((__float_as_uint((float)x[k]) & 0x7f800000u) == 0x7f800000u) ? 1u : 0u;
      }
    }
    if (nf || (lane_ok && sing)) atomicExch(a.status, CBS_ERR_SINGULAR);
  }

  if (!ADJ) {
    __syncwarp();
    if (ok) {
#pragma unroll
      for (int k = 0; k < M; k++)
        if (k < size) SfL[k * t.sp + i] = (TG)x[k];
    }
    __syncthreads();
    tile_copy<false, TG, TG>(tr, t, Sf, (TG*)a.out);
    return;
  }
  // ---- adjoint epilogue: lambda = x here ----
  // grad_alpha_i = -lambda_i (x_{i-1} + x_{i+1}) with the forward solution x
  T ga[M];
  if (want_ga) {
#pragma unroll
    for (int k = 0; k < M; k++) {
      const int row = start + k;
      const T xm = rowval(SxL, row - 1), xp = rowval(SxL, row + 1);
      ga[k] = -x[k] * (xm + xp);
    }
  }
  __syncwarp();
  // lambda into the f tile (g no longer needed) for the S^T stencil halo
  if (ok) {
#pragma unroll
    for (int k = 0; k < M; k++)
      if (k < size) SfL[k * t.sp + i] = (TG)x[k];
  }
  __syncwarp();
  T gf[M];
  if (KS > 0) {
    // (S^T lambda)_j = sum_q w_q (lambda_{j-q} - lambda_{j+q})
#pragma unroll
    for (int k = 0; k < M; k++) {
      T s = T(0);
      const int row = start + k;
#pragma unroll
      for (int q = 1; q <= KS; q++) s += (T)a.w[q - 1] * (rowval(SfL, row - q) - rowval(SfL, row + q));
      gf[k] = s;
    }
  }
  __syncthreads();
  if (a.lam) tile_copy<false, TG, TG>(tr, t, Sf, (TG*)a.lam);
  if (KS > 0 && a.out) {
    __syncthreads();
    if (ok) {
#pragma unroll
      for (int k = 0; k < M; k++)
        if (k < size) SfL[k * t.sp + i] = (TG)gf[k];
    }
    __syncthreads();
    tile_copy<false, TG, TG>(tr, t, Sf, (TG*)a.out);
  }
  if (want_ga) {
    __syncthreads();
    if (ok) {
#pragma unroll
      for (int k = 0; k < M; k++)
        if (k < size) SaL[k * t.sp + i] = (TG)ga[k];
    }
    __syncthreads();
    tile_copy<false, TG, TG>(tr, t, Sa, (TG*)a.grad_alpha);
  }
}

}  // namespace cbs
