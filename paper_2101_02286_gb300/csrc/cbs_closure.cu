// cbs_closure.cu -- one-sided boundary closures (see cbs_closure.cuh): the
// host tables of the Woodbury correction and the kernel that applies it.
#include <algorithm>
#include <cmath>
#include <utility>

#include "cbs_closure.cuh"

namespace cbs {

namespace {

// Banded LU without pivoting of the acyclic n x n matrix with half bandwidth
// r (T is symmetric positive definite for the schemes in use: its symbol is
// positive).  F[i * (2r+1) + (j - i + r)] holds entry (i, j).
bool band_factor(std::vector<double>& F, int n, int r) {
  const int w = 2 * r + 1;
  for (int k = 0; k < n; k++) {
    const double piv = F[(size_t)k * w + r];
    if (!std::isfinite(piv) || piv == 0.0) return false;
    for (int i = k + 1; i <= std::min(n - 1, k + r); i++) {
      const double l = F[(size_t)i * w + (k - i + r)] / piv;
      F[(size_t)i * w + (k - i + r)] = l;
      for (int j = k + 1; j <= std::min(n - 1, k + r); j++) F[(size_t)i * w + (j - i + r)] -= l * F[(size_t)k * w + (j - k + r)];
    }
  }
  return true;
}

void band_solve(const std::vector<double>& F, int n, int r, std::vector<double>& b) {
  const int w = 2 * r + 1;
  for (int i = 0; i < n; i++)
    for (int j = std::max(0, i - r); j < i; j++) b[i] -= F[(size_t)i * w + (j - i + r)] * b[j];
  for (int i = n - 1; i >= 0; i--) {
    for (int j = i + 1; j <= std::min(n - 1, i + r); j++) b[i] -= F[(size_t)i * w + (j - i + r)] * b[j];
    b[i] /= F[(size_t)i * w + r];
  }
}

// Gauss-Jordan inverse with partial pivoting of the m x m matrix A (row
// major); false when a pivot is non-finite or below 1e-13 of the largest
// entry of A.
bool dense_inverse(std::vector<double> A, int m, std::vector<double>& inv) {
  double scale = 0.0;
  for (double v : A) scale = std::fmax(scale, std::fabs(v));
  inv.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; i++) inv[(size_t)i * m + i] = 1.0;
  for (int c = 0; c < m; c++) {
    int piv = c;
    for (int i = c + 1; i < m; i++)
      if (std::fabs(A[(size_t)i * m + c]) > std::fabs(A[(size_t)piv * m + c])) piv = i;
    for (int j = 0; j < m && piv != c; j++) {
      std::swap(A[(size_t)c * m + j], A[(size_t)piv * m + j]);
      std::swap(inv[(size_t)c * m + j], inv[(size_t)piv * m + j]);
    }
    const double d = A[(size_t)c * m + c];
    if (!std::isfinite(d) || !(std::fabs(d) > 1e-13 * scale)) return false;
    for (int j = 0; j < m; j++) {
      A[(size_t)c * m + j] /= d;
      inv[(size_t)c * m + j] /= d;
    }
    for (int i = 0; i < m; i++) {
      const double f = A[(size_t)i * m + c];
      if (i == c || f == 0.0) continue;
      for (int j = 0; j < m; j++) {
        A[(size_t)i * m + j] -= f * A[(size_t)c * m + j];
        inv[(size_t)i * m + j] -= f * inv[(size_t)c * m + j];
      }
    }
  }
  return true;
}

}  // namespace

std::string closure_build(ClosureTables& C, int n, int r, const double* band, int K, const double* w, int c, int W,
                          const double* cl, double h, bool* singular) {
  *singular = false;
  C = ClosureTables();
  if (c < 1 || c > kMaxClosureRows) return "closure_rows must be 1..4";
  if (W < 1 || W > kMaxClosureWidth) return "closure_width must be 1..16";
  if (!cl) return "closure rows need the host array";
  if (c < r || c < K) return "closure_rows must be >= max(r, rhs_terms): interior rows reach c - max(r, K)";
  if (n < 2 * W || n < 4 * c) return "line too short for its closure rows (n >= 2 closure_width, n >= 4 closure_rows)";
  for (int k = 0; k < 2 * c * W; k++)
    if (!std::isfinite(cl[k])) return "non-finite closure coefficients";
  const int c2 = 2 * c;
  std::vector<int> u(c2);
  for (int k = 0; k < c; k++) {
    u[k] = k;
    u[c + k] = n - 1 - k;
  }
  // E^T and d as dense rows (n is at most a few thousand)
  std::vector<double> E((size_t)c2 * n, 0.0), D((size_t)c2 * n, 0.0);
  for (int k = 0; k < c; k++)
    for (int j = 0; j < W; j++) {
      const double L = cl[(size_t)k * 2 * W + j], R = cl[(size_t)k * 2 * W + W + j];
      E[(size_t)k * n + j] += L;
      D[(size_t)k * n + j] += R / h;
      E[(size_t)(c + k) * n + (n - 1 - j)] += L;   // mirror image
      D[(size_t)(c + k) * n + (n - 1 - j)] -= R / h;  // odd under reflection
    }
  for (int b = 0; b < c2; b++) {
    const int i = u[b];
    for (int t = -r; t <= r; t++)
      if (i + t >= 0 && i + t < n) E[(size_t)b * n + i + t] -= band[t + r];  // T's row (acyclic)
    for (int q = 1; q <= K; q++) {  // the kernels' stencil row, end values extended
      D[(size_t)b * n + std::min(i + q, n - 1)] -= w[q - 1];
      D[(size_t)b * n + std::max(i - q, 0)] += w[q - 1];
    }
  }
  // Z = T^{-1} U
  const int bw = 2 * r + 1;
  std::vector<double> F((size_t)n * bw, 0.0);
  for (int i = 0; i < n; i++)
    for (int t = -r; t <= r; t++)
      if (i + t >= 0 && i + t < n) F[(size_t)i * bw + t + r] = band[t + r];
  if (!band_factor(F, n, r)) {
    *singular = true;
    return "closure: zero pivot in the acyclic Toeplitz factorisation";
  }
  std::vector<double> Z((size_t)c2 * n);  // column b at Z[b * n + i]
  for (int b = 0; b < c2; b++) {
    std::vector<double> col(n, 0.0);
    col[u[b]] = 1.0;
    band_solve(F, n, r, col);
    for (int i = 0; i < n; i++) Z[(size_t)b * n + i] = col[i];
  }
  // M = I + E^T Z
  std::vector<double> M((size_t)c2 * c2, 0.0);
  for (int a = 0; a < c2; a++)
    for (int b = 0; b < c2; b++) {
      double s = a == b ? 1.0 : 0.0;
      for (int i = 0; i < n; i++) s += E[(size_t)a * n + i] * Z[(size_t)b * n + i];
      M[(size_t)a * c2 + b] = s;
    }
  if (!dense_inverse(M, c2, C.Minv)) {
    *singular = true;
    return "closure: the boundary system I + E^T T^{-1} U is singular";
  }
  // window rows: where E^T or d has an entry
  for (int i = 0; i < n; i++) {
    bool any = false;
    for (int b = 0; b < c2 && !any; b++) any = E[(size_t)b * n + i] != 0.0 || D[(size_t)b * n + i] != 0.0;
    if (any) C.wrow.push_back(i);
  }
  const int nw = (int)C.wrow.size();
  C.Df.assign((size_t)c2 * nw, 0.0);
  C.Ey.assign((size_t)c2 * nw, 0.0);
  for (int b = 0; b < c2; b++)
    for (int k = 0; k < nw; k++) {
      C.Df[(size_t)b * nw + k] = D[(size_t)b * n + C.wrow[k]];
      C.Ey[(size_t)b * nw + k] = E[(size_t)b * n + C.wrow[k]];
    }
  // updated rows: where a column of Z is above 2^-60 of its largest entry
  std::vector<double> cmax(c2, 0.0);
  for (int b = 0; b < c2; b++)
    for (int i = 0; i < n; i++) cmax[b] = std::fmax(cmax[b], std::fabs(Z[(size_t)b * n + i]));
  for (int i = 0; i < n; i++) {
    bool keep = false;
    for (int b = 0; b < c2 && !keep; b++) keep = std::fabs(Z[(size_t)b * n + i]) > std::ldexp(cmax[b], -60);
    if (keep) C.urow.push_back(i);
  }
  for (int i : C.urow)
    for (int b = 0; b < c2; b++) C.Zt.push_back(Z[(size_t)b * n + i]);
  C.c2 = c2;
  return "";
}

// ---------------------------------------------------------------- kernel
// One thread per line; consecutive y/z lines are adjacent in x, so a warp's
// accesses to one row are one contiguous run.  Every read of a line happens
// before that thread's first write to it.
template <typename TIn, typename TOut>
__global__ void __launch_bounds__(128) closure_kernel(const ClosureArgs a) {
  const int64_t line = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= a.lines) return;
  int64_t base, es;
  if (a.dir == 0) {
    base = line * a.n;
    es = 1;
  } else if (a.dir == 1) {  // lines x + nx z
    base = line % a.nx + a.nx * a.ny * (line / a.nx);
    es = a.nx;
  } else {                  // lines x + nx y
    base = line;
    es = a.nx * a.ny;
  }
  const TIn* f = (const TIn*)a.f + base;
  TOut* x = (TOut*)a.x + base;
  constexpr int C2 = 2 * kMaxClosureRows;
  double s[C2];
#pragma unroll
  for (int b = 0; b < C2; b++) s[b] = 0.0;
  for (int k = 0; k < a.nw; k++) {  // s = d - E^T y
    const int64_t o = (int64_t)__ldg(a.wrow + k) * es;
    const double fv = (double)f[o], yv = (double)x[o];
#pragma unroll
    for (int b = 0; b < C2; b++)
      if (b < a.c2) s[b] += __ldg(a.Df + b * a.nw + k) * fv - __ldg(a.Ey + b * a.nw + k) * yv;
  }
  double g[C2];  // g = M^{-1} s
#pragma unroll
  for (int b = 0; b < C2; b++) {
    double v = 0.0;
#pragma unroll
    for (int e = 0; e < C2; e++)
      if (b < a.c2 && e < a.c2) v += __ldg(a.Minv + b * a.c2 + e) * s[e];
    g[b] = v;
  }
  for (int k = 0; k < a.nu; k++) {  // x = y + Z g on the kept rows
    const int64_t o = (int64_t)__ldg(a.urow + k) * es;
    double v = (double)x[o];
#pragma unroll
    for (int b = 0; b < C2; b++)
      if (b < a.c2) v += __ldg(a.Zt + (int64_t)k * a.c2 + b) * g[b];
    x[o] = (TOut)v;
  }
}

cudaError_t launch_closure(const ClosureArgs& a, bool in64, bool out64, cudaStream_t s) {
  if (a.lines <= 0) return cudaSuccess;
  const int64_t blocks = (a.lines + 127) / 128;
  if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
  if (in64 && out64) closure_kernel<double, double><<<(unsigned)blocks, 128, 0, s>>>(a);
  else if (!in64 && !out64) closure_kernel<float, float><<<(unsigned)blocks, 128, 0, s>>>(a);
  else if (!in64 && out64) closure_kernel<float, double><<<(unsigned)blocks, 128, 0, s>>>(a);
  else return cudaErrorNotSupported;
  return cudaGetLastError();
}

}  // namespace cbs
