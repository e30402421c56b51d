// cbs_plan.cpp -- host-side pre-factorisation of the partitioned system.
//
// For a Toeplitz line matrix A (half bandwidth r, cyclic or not), or one
// whose rows repeat with a short period (block entries, cbs_bands.h), split
// into p partitions this computes, in FP64, everything the per-solve kernels need
// that does not depend on the right-hand side (paper Sec. 4, last paragraph):
//   - the banded LU factors of the bulk blocks D_i (Sec. 3, Fig. 3);
//   - S_i = D_i^{-1} L_i and R_i = D_i^{-1} U_i (Eq. 15-16);
//   - the reduced blocks D-hat, L-hat, U-hat of the interface system (Eq. 18-20);
//   - the interface schedule (Algorithm 1) and, for every stage, the
//     coefficient blocks acting on x~ (Algorithms 2-4 with the W^{-1}
//     products precomputed), so a solve only updates x~.
#include <cmath>
#include <cstring>
#include <utility>

#include "cbs_bands.h"
#include "cbs_internal.h"

namespace cbs {

std::vector<Stage> build_schedule(int p, bool cyclic) {
  std::vector<Stage> st;
  if (p < 1) return st;
  if (!cyclic) {
    // Classic block PCR on an acyclic system: ceil(log2 p) steps (Sec. 4).
    int s = 1;
    while (s < p) {
      st.push_back({kPcr, s, p});
      s *= 2;
    }
    st.push_back({kFinal, s, p});
    return st;
  }
  // Algorithm 1: detach the last row of each sub-system whenever the
  // sub-system dimension is odd, then one block PCR step.
  int s = 1, n0 = p, na = p;
  std::vector<int> stack;
  while (n0 > 1) {
    int odd = n0 % 2;
    stack.push_back(odd);
    if (odd) {
      n0 -= 1;
      na -= s;
      st.push_back({kDetach, s, na});
    }
    st.push_back({kPcr, s, na});
    s *= 2;
    n0 /= 2;
  }
  st.push_back({kFinal, s, na});
  while (!stack.empty()) {
    n0 *= 2;
    s /= 2;
    int odd = stack.back();
    stack.pop_back();
    if (odd) {
      st.push_back({kReattach, s, na});
      na += s;
      n0 += 1;
    }
  }
  return st;
}

namespace {

// r x r row-major blocks, r <= kMaxR.
struct Blk {
  int r;
  double a[kMaxR * kMaxR];
  explicit Blk(int r_ = 1) : r(r_) { std::memset(a, 0, sizeof(a)); }
  double& operator()(int i, int j) { return a[i * r + j]; }
  double operator()(int i, int j) const { return a[i * r + j]; }
  static Blk eye(int r) {
    Blk b(r);
    for (int i = 0; i < r; i++) b(i, i) = 1.0;
    return b;
  }
};
Blk operator*(const Blk& x, const Blk& y) {
  Blk z(x.r);
  for (int i = 0; i < x.r; i++)
    for (int j = 0; j < x.r; j++) {
      double s = 0;
      for (int k = 0; k < x.r; k++) s += x(i, k) * y(k, j);
      z(i, j) = s;
    }
  return z;
}
Blk operator+(const Blk& x, const Blk& y) {
  Blk z(x.r);
  for (int i = 0; i < x.r * x.r; i++) z.a[i] = x.a[i] + y.a[i];
  return z;
}
Blk operator-(const Blk& x, const Blk& y) {
  Blk z(x.r);
  for (int i = 0; i < x.r * x.r; i++) z.a[i] = x.a[i] - y.a[i];
  return z;
}
Blk neg(const Blk& x) {
  Blk z(x.r);
  for (int i = 0; i < x.r * x.r; i++) z.a[i] = -x.a[i];
  return z;
}
double maxabs(const Blk& x) {
  double m = 0.0;
  for (int i = 0; i < x.r * x.r; i++) m = std::fmax(m, std::fabs(x.a[i]));
  return m;
}
// Inverse; returns false when non-finite or numerically singular, i.e. when
// |det| <= 1e-12 * scale^r with `scale` the magnitude of the blocks that were
// combined into x (so rounding residue of an exactly singular block counts).
// Closed forms for r = 1, 2; Gauss-Jordan elimination with partial pivoting
// above (det = the product of the pivots, up to sign).
bool inv(const Blk& x, Blk& out, double scale = 0.0) {
  const int r = x.r;
  scale = std::fmax(scale, maxabs(x));
  if (r == 1) {
    out = Blk(1);
    if (!std::isfinite(x.a[0]) || !(std::fabs(x.a[0]) > 1e-12 * scale)) return false;
    out.a[0] = 1.0 / x.a[0];
    return true;
  }
  if (r == 2) {
    out = Blk(2);
    const double det = x(0, 0) * x(1, 1) - x(0, 1) * x(1, 0);
    if (!std::isfinite(det) || !(std::fabs(det) > 1e-12 * scale * scale)) return false;
    out(0, 0) = x(1, 1) / det;
    out(1, 1) = x(0, 0) / det;
    out(0, 1) = -x(0, 1) / det;
    out(1, 0) = -x(1, 0) / det;
    return true;
  }
  out = Blk::eye(r);
  Blk w = x;
  double det = 1.0;
  for (int c = 0; c < r; c++) {
    int piv = c;
    for (int i = c + 1; i < r; i++)
      if (std::fabs(w(i, c)) > std::fabs(w(piv, c))) piv = i;
    if (piv != c)
      for (int j = 0; j < r; j++) {
        std::swap(w(c, j), w(piv, j));
        std::swap(out(c, j), out(piv, j));
      }
    const double d = w(c, c);
    det *= d;
    if (!std::isfinite(d) || d == 0.0) return false;
    for (int j = 0; j < r; j++) {
      w(c, j) /= d;
      out(c, j) /= d;
    }
    for (int i = 0; i < r; i++) {
      if (i == c) continue;
      const double f = w(i, c);
      if (f == 0.0) continue;
      for (int j = 0; j < r; j++) {
        w(i, j) -= f * w(c, j);
        out(i, j) -= f * out(c, j);
      }
    }
  }
  double tol = 1e-12;
  for (int k = 0; k < r; k++) tol *= scale;
  if (!std::isfinite(det) || !(std::fabs(det) > tol)) return false;
  for (int k = 0; k < r * r; k++)
    if (!std::isfinite(out.a[k])) return false;
  return true;
}

}  // namespace

PBands block_bands(int b, const double* L, const double* D, const double* U) {
  PBands A;
  A.r = 2 * b - 1;
  A.period = b;
  for (int c = 0; c < b; c++)
    for (int j = 0; j < b; j++) {
      A.v[c][j - c - b + A.r] = L[c * b + j];
      A.v[c][j - c + A.r] = D[c * b + j];
      A.v[c][b + j - c + A.r] = U[c * b + j];
    }
  return A;
}

std::string build_line_tables(LineTables& T, int n, const Bands& A, int p, bool cyclic,
                              bool* singular, int max_lanes, const int* sizes) {
  PBands B;
  B.r = A.r;
  B.period = 1;
  for (int t = 0; t < 2 * A.r + 1; t++) B.v[0][t] = A.v[t];
  return build_line_tables_periodic(T, n, B, p, cyclic, singular, max_lanes, sizes);
}

// Row indices below are relative to a partition's first row, which is a
// multiple of the period: interface row q is row q, bulk row j is row r + j.
std::string build_line_tables_periodic(LineTables& T, int n, const PBands& A, int p, bool cyclic, bool* singular,
                                       int max_lanes, const int* sizes) {
  *singular = false;
  const int r = A.r;
  T = LineTables();
  T.n = n;
  T.r = r;
  T.p = p;
  T.cyclic = cyclic;
  if (p < 1 || p > max_lanes) return "segments out of range";
  if (sizes) {
    T.count_big = sizes[0];
    T.rows_big = sizes[1];
    T.rows_small = sizes[2];
    if (T.count_big < 1 || T.count_big > p || T.rows_small > T.rows_big ||
        (int64_t)T.count_big * T.rows_big + (int64_t)(p - T.count_big) * T.rows_small != n)
      return "inconsistent partition sizes";
    if (T.count_big == p) T.rows_small = T.rows_big;
  } else {
    T.rows_small = n / p;
    T.count_big = n % p;
    T.rows_big = T.rows_small + (T.count_big ? 1 : 0);
    if (T.count_big == 0) T.count_big = p;  // all partitions equal
  }
  if (T.rows_small < 2 * r) return "partitions need at least 2r rows (n >= 2 r p)";
  if (A.period > 1 && (n % A.period || T.rows_big % A.period || T.rows_small % A.period))
    return "block entries: every partition must hold whole points (sizes multiples of the block size)";
  T.start.resize(p);
  T.size.resize(p);
  int acc = 0;
  for (int i = 0; i < p; i++) {
    T.size[i] = (i < T.count_big) ? T.rows_big : T.rows_small;
    T.start[i] = acc;
    acc += T.size[i];
  }
  const int nmax = T.rows_big - r;
  T.nmax = nmax;

  // ---- banded LU of the bulk block (rows from the top; Toeplitz rows) ----
  // Work arrays Ub[j][t] = U[j][j+t] (t = 0..r), Lb[j][q] = L[j][j-q].
  std::vector<double> Ub((size_t)nmax * (r + 1)), Lb((size_t)nmax * (r + 1), 0.0);
  // start from D's rows
  std::vector<double> work((size_t)nmax * (2 * r + 1));
  for (int j = 0; j < nmax; j++)
    for (int t = -r; t <= r; t++) work[(size_t)j * (2 * r + 1) + t + r] = A.at(r + j, t);
  const double bscale = A.max_abs();
  for (int j = 0; j < nmax; j++) {
    double piv = work[(size_t)j * (2 * r + 1) + r];
    if (!(std::fabs(piv) > 1e-12 * bscale) || !std::isfinite(piv)) {
      *singular = true;
      return "zero pivot in a bulk block D_i";
    }
    for (int t = 0; t <= r; t++) Ub[(size_t)j * (r + 1) + t] = (j + t < nmax) ? work[(size_t)j * (2 * r + 1) + r + t] : 0.0;
    for (int q = 1; q <= r && j + q < nmax; q++) {
      // row j+q, column j: offset -q
      double l = work[(size_t)(j + q) * (2 * r + 1) + r - q] / piv;
      Lb[(size_t)(j + q) * (r + 1) + q] = l;
      work[(size_t)(j + q) * (2 * r + 1) + r - q] = 0.0;
      for (int t = 1; t <= r; t++) {
        int off = t - q;  // column j+t seen from row j+q
        if (off > r) continue;
        work[(size_t)(j + q) * (2 * r + 1) + r + off] -= l * work[(size_t)j * (2 * r + 1) + r + t];
      }
    }
  }
  const int F = 2 * r + 1;
  T.fac.assign((size_t)nmax * F, 0.0);
  for (int j = 0; j < nmax; j++) {
    double ip = 1.0 / Ub[(size_t)j * (r + 1)];
    for (int q = 1; q <= r; q++) T.fac[(size_t)j * F + q - 1] = Lb[(size_t)j * (r + 1) + q];
    T.fac[(size_t)j * F + r] = ip;
    for (int q = 1; q <= r; q++) T.fac[(size_t)j * F + r + q] = Ub[(size_t)j * (r + 1) + q] * ip;
  }
  auto solveD = [&](int N, const double* b, double* y) {
    for (int j = 0; j < N; j++) {
      double s = b[j];
      for (int q = 1; q <= r && j - q >= 0; q++) s -= T.fac[(size_t)j * F + q - 1] * y[j - q];
      y[j] = s;
    }
    for (int j = N - 1; j >= 0; j--) {
      double s = T.fac[(size_t)j * F + r] * y[j];
      for (int q = 1; q <= r && j + q < N; q++) s -= T.fac[(size_t)j * F + r + q] * y[j + q];
      y[j] = s;
    }
  };

  // ---- S_i, R_i (Eq. 15-16): they depend only on the partition size ----
  // class 0 = rows_big, class 1 = rows_small; [j*r + q]
  std::vector<double> Scl[2], Rcl[2];
  std::vector<double> col(nmax), sol(nmax);
  for (int c = 0; c < 2; c++) {
    const int m = c == 0 ? T.rows_big : T.rows_small, N = m - r;
    Scl[c].assign((size_t)N * r, 0.0);
    Rcl[c].assign((size_t)N * r, 0.0);
    for (int q = 0; q < r; q++) {
      // L_i[:, q]: bulk row j couples to own interface column q at offset q - r - j
      for (int j = 0; j < N; j++) col[j] = A.at(r + j, q - r - j);
      solveD(N, col.data(), sol.data());
      for (int j = 0; j < N; j++) Scl[c][(size_t)j * r + q] = sol[j];
      // U_i[:, q]: bulk row j couples to next interface column q at offset m + q - r - j
      for (int j = 0; j < N; j++) col[j] = A.at(r + j, m + q - r - j);
      solveD(N, col.data(), sol.data());
      for (int j = 0; j < N; j++) Rcl[c][(size_t)j * r + q] = sol[j];
    }
  }
  T.srB.assign((size_t)(T.rows_big - r) * 2 * r, 0.0);
  T.srS.assign((size_t)(T.rows_small - r) * 2 * r, 0.0);
  for (int c = 0; c < 2; c++) {
    std::vector<double>& dst = c == 0 ? T.srB : T.srS;
    const int N = (c == 0 ? T.rows_big : T.rows_small) - r;
    for (int j = 0; j < N; j++)
      for (int q = 0; q < r; q++) {
        dst[(size_t)j * 2 * r + q] = Scl[c][(size_t)j * r + q];
        dst[(size_t)j * 2 * r + r + q] = Rcl[c][(size_t)j * r + q];
      }
  }
  auto cls = [&](int i) { return i < T.count_big ? 0 : 1; };
  // acyclic: the last partition has no next interface, so its R is zero
  auto S_at = [&](int i, int j, int q) { return Scl[cls(i)][(size_t)j * r + q]; };
  auto R_at = [&](int i, int j, int q) {
    return (!cyclic && i == p - 1) ? 0.0 : Rcl[cls(i)][(size_t)j * r + q];
  };

  // ---- b-hat assembly blocks (Eq. 21) ----
  for (int q = 0; q < r; q++)
    for (int e = 0; e < r; e++) {
      T.Lt[q][e] = (e >= q) ? A.at(q, e - r - q) : 0.0;
      T.Ut[q][e] = (e <= q) ? A.at(q, r + e - q) : 0.0;
    }

  // ---- reduced blocks (Eq. 18-20) ----
  std::vector<Blk> W(p, Blk(r)), Lh(p, Blk(r)), Uh(p, Blk(r));
  for (int i = 0; i < p; i++) {
    const int im = (i + p - 1) % p;
    const bool has_prev = cyclic || i > 0;
    const int Nm = T.size[im] - r, N = T.size[i] - r;
    Blk Dt(r), LRm(r), USi(r), LSm(r), URi(r);
    for (int q = 0; q < r; q++)
      for (int qq = 0; qq < r; qq++) Dt(q, qq) = A.at(q, qq - q);
    for (int q = 0; q < r; q++)
      for (int qq = 0; qq < r; qq++) {
        double a1 = 0, a2 = 0, a3 = 0, a4 = 0;
        for (int e = 0; e < r; e++) {
          if (has_prev) {
            a1 += T.Lt[q][e] * R_at(im, Nm - r + e, qq);
            a3 += T.Lt[q][e] * S_at(im, Nm - r + e, qq);
          }
          a2 += T.Ut[q][e] * S_at(i, e, qq);
          a4 += T.Ut[q][e] * R_at(i, e, qq);
        }
        (void)N;
        LRm(q, qq) = a1;
        USi(q, qq) = a2;
        LSm(q, qq) = a3;
        URi(q, qq) = a4;
      }
    W[i] = Dt - LRm - USi;
    Lh[i] = neg(LSm);
    Uh[i] = neg(URi);
  }
  T.Dhat.resize((size_t)p * r * r);
  T.Lhat.resize((size_t)p * r * r);
  T.Uhat.resize((size_t)p * r * r);
  for (int i = 0; i < p; i++)
    for (int e = 0; e < r * r; e++) {
      T.Dhat[(size_t)i * r * r + e] = W[i].a[e];
      T.Lhat[(size_t)i * r * r + e] = Lh[i].a[e];
      T.Uhat[(size_t)i * r * r + e] = Uh[i].a[e];
    }

  // ---- interface schedule and per-stage coefficients (Algorithms 1-4) ----
  T.stages = build_schedule(p, cyclic);
  const int ns = (int)T.stages.size();
  if (ns > kMaxStages && max_lanes <= kMaxLanes) return "interface schedule too long";
  const int rr = r * r;
  T.coef.assign((size_t)ns * 3 * rr * p, 0.0);
  T.src.assign((size_t)ns * 2 * p, 0);
  T.stage_has_c.assign(ns, 0);
  auto put = [&](int st, int mat, int i, const Blk& b) {
    for (int e = 0; e < rr; e++) T.coef[((size_t)(st * 3 + mat) * rr + e) * p + i] = b.a[e];
  };
  for (int st = 0; st < ns; st++)
    for (int i = 0; i < p; i++) {
      put(st, 0, i, Blk::eye(r));
      T.src[(size_t)(st * 2 + 0) * p + i] = i;
      T.src[(size_t)(st * 2 + 1) * p + i] = i;
    }
  for (int st = 0; st < ns; st++) {
    const Stage S_ = T.stages[st];
    const int s = S_.s, na = S_.na;
    Blk Wi(r);
    if (S_.type == kDetach) {
      T.detach_steps++;
      T.detached_rows += s;
      std::vector<Blk> W2 = W, L2 = Lh, U2 = Uh;
      for (int i = na - s; i < na; i++) {  // receives from detached row i + s
        const int j = i + s;
        if (!inv(W[j], Wi)) { *singular = true; return "singular interface block (detach)"; }
        Blk KP = Uh[i] * Wi;
        W2[i] = W[i] - KP * Lh[j];
        U2[i] = neg(KP * Uh[j]);
        put(st, 2, i, KP);
        T.src[(size_t)(st * 2 + 1) * p + i] = j;
      }
      for (int i = 0; i < s; i++) {  // receives from detached row i + na
        const int j = i + na;
        if (!inv(W[j], Wi)) { *singular = true; return "singular interface block (detach)"; }
        Blk KM = Lh[i] * Wi;
        W2[i] = W2[i] - KM * Uh[j];
        L2[i] = neg(KM * Lh[j]);
        put(st, 1, i, KM);
        T.src[(size_t)(st * 2 + 0) * p + i] = j;
      }
      W = W2;
      Lh = L2;
      Uh = U2;
    } else if (S_.type == kPcr) {
      T.pcr_steps++;
      std::vector<Blk> W2 = W, L2 = Lh, U2 = Uh;
      for (int i = 0; i < na; i++) {
        int jp, jm;
        bool hp = true, hm = true;
        if (cyclic) {
          jp = (i + s) % na;
          jm = (i - s + na) % na;
        } else {
          jp = i + s;
          jm = i - s;
          hp = jp < na;
          hm = jm >= 0;
        }
        Blk KP(r), KM(r);
        Blk acc = W[i];
        if (hp) {
          if (!inv(W[jp], Wi)) { *singular = true; return "singular interface block (PCR)"; }
          KP = Uh[i] * Wi;
          acc = acc - KP * Lh[jp];
          U2[i] = neg(KP * Uh[jp]);
          T.src[(size_t)(st * 2 + 1) * p + i] = jp;
        } else {
          U2[i] = Blk(r);
        }
        if (hm) {
          if (!inv(W[jm], Wi)) { *singular = true; return "singular interface block (PCR)"; }
          KM = Lh[i] * Wi;
          acc = acc - KM * Uh[jm];
          L2[i] = neg(KM * Lh[jm]);
          T.src[(size_t)(st * 2 + 0) * p + i] = jm;
        } else {
          L2[i] = Blk(r);
        }
        W2[i] = acc;
        put(st, 1, i, KM);
        put(st, 2, i, KP);
      }
      W = W2;
      Lh = L2;
      Uh = U2;
    } else if (S_.type == kFinal) {
      T.stage_has_c[st] = 1;
      for (int i = 0; i < na; i++) {
        // Cyclic: after the last PCR step every sub-system is one row whose
        // L-hat and U-hat couple the row to itself, so the block to invert is
        // W + L-hat + U-hat (this also covers p = 1 and p = 2).
        Blk M = cyclic ? (W[i] + Lh[i] + Uh[i]) : W[i];
        const double sc = std::fmax(maxabs(W[i]), std::fmax(maxabs(Lh[i]), maxabs(Uh[i])));
        if (!inv(M, Wi, sc)) { *singular = true; return "singular interface block (final)"; }
        put(st, 0, i, Wi);
      }
    } else {  // kReattach: rows na .. na+s-1, neighbours j - s and j - na
      T.stage_has_c[st] = 1;
      for (int j = na; j < na + s; j++) {
        if (!inv(W[j], Wi)) { *singular = true; return "singular interface block (reattach)"; }
        put(st, 0, j, Wi);
        put(st, 1, j, Wi * Lh[j]);
        put(st, 2, j, Wi * Uh[j]);
        T.src[(size_t)(st * 2 + 0) * p + j] = j - s;
        T.src[(size_t)(st * 2 + 1) * p + j] = j - na;
      }
    }
  }
  for (double v : T.coef)
    if (!std::isfinite(v)) {
      *singular = true;
      return "non-finite interface coefficient";
    }
  for (double v : T.srB)
    if (!std::isfinite(v)) {
      *singular = true;
      return "non-finite S/R entry";
    }
  // Coupling blocks below rounding.  The interface blocks L-hat, U-hat shrink
  // geometrically with the partition size for a diagonally dominant A, and
  // every PCR step squares their ratio to W, so after a few steps KM and KP
  // are far below one unit in the last place of C x~.  Dropping a term
  // |K| <= 2^-60 max|C| changes the stage's result by less than 2^-60 of
  // ||x~||, below FP64 rounding (2^-30 for the FP32 copy, below FP32
  // rounding); such a stage needs no messages.
  T.stage_msg.assign(ns, 0);
  for (int st = 0; st < ns; st++) {
    double cmax = 0.0, kmax = 0.0;
    for (int e = 0; e < rr; e++)
      for (int i = 0; i < p; i++) {
        cmax = std::fmax(cmax, std::fabs(T.coef[((size_t)(st * 3 + 0) * rr + e) * p + i]));
        kmax = std::fmax(kmax, std::fabs(T.coef[((size_t)(st * 3 + 1) * rr + e) * p + i]));
        kmax = std::fmax(kmax, std::fabs(T.coef[((size_t)(st * 3 + 2) * rr + e) * p + i]));
      }
    if (kmax > std::ldexp(cmax, -60)) T.stage_msg[st] |= 1;
    if (kmax > std::ldexp(cmax, -30)) T.stage_msg[st] |= 2;
  }
  return "";
}

std::vector<double> bulk_inverse_rows(const LineTables& T, int N, int nrows) {
  const int r = T.r, F = 2 * r + 1;
  std::vector<double> out((size_t)nrows * N), y(N);
  for (int q = 0; q < nrows; q++) {
    for (int j = 0; j < N; j++) y[j] = (j == q) ? 1.0 : 0.0;
    for (int j = 0; j < N; j++) {
      double s = y[j];
      for (int k = 1; k <= r && j - k >= 0; k++) s -= T.fac[(size_t)j * F + k - 1] * y[j - k];
      y[j] = s;
    }
    for (int j = N - 1; j >= 0; j--) {
      double s = T.fac[(size_t)j * F + r] * y[j];
      for (int k = 1; k <= r && j + k < N; k++) s -= T.fac[(size_t)j * F + r + k] * y[j + k];
      y[j] = s;
    }
    // D is symmetric, so column q of D^{-1} is row q
    for (int j = 0; j < N; j++) out[(size_t)q * N + j] = y[j];
  }
  return out;
}

}  // namespace cbs
