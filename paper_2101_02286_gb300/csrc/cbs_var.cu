// cbs_var.cu -- launchers for the variable-coefficient kernels and the band
// gradient.
#include "cbs_line_launch.cuh"
#include "cbs_var.cuh"

namespace cbs {

template <int M, int KS, bool ADJ, typename T, typename TG>
static cudaError_t launch_var_one(const VarArgs& a, const DevLineTables& t, cudaStream_t s) {
  const int threads = 256;
  const int lines_per_cta = threads / t.pw;
  if (a.nlines <= 0) return cudaSuccess;
  const dim3 grid = tile_grid(a.nx, a.ny, a.nz, a.nlines, a.dir, lines_per_cta);
  const size_t smem = 3 * (size_t)lines_per_cta * t.lsz * sizeof(TG);
  static SmemOptIn opt;  // per instantiation
  cudaError_t e = opt.ensure(var_kernel<M, KS, ADJ, T, TG>, smem);
  if (e != cudaSuccess) return e;
  var_kernel<M, KS, ADJ, T, TG><<<grid, threads, smem, s>>>(a, t);
  return cudaGetLastError();
}

template <int M, bool ADJ, typename T>
static cudaError_t launch_var_ks(int KS, const VarArgs& a, const DevLineTables& t, cudaStream_t s) {
  switch (KS) {
    case 0: return launch_var_one<M, 0, ADJ, T, T>(a, t, s);
    case 2: return launch_var_one<M, 2, ADJ, T, T>(a, t, s);
    case 3: return launch_var_one<M, 3, ADJ, T, T>(a, t, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_var(int M, int KS, bool adj, bool f64, const VarArgs& a, const DevLineTables& t,
                       cudaStream_t s) {
#define CBS_V(MM, AD)                                                                  \
  return f64 ? launch_var_ks<MM, AD, double>(KS, a, t, s) : launch_var_ks<MM, AD, float>(KS, a, t, s)
  if (M == 8) {
    if (adj) { CBS_V(8, true); } else { CBS_V(8, false); }
  }
  if (M == 16) {
    if (adj) { CBS_V(16, true); } else { CBS_V(16, false); }
  }
#undef CBS_V
  return cudaErrorInvalidValue;
}

// grad_alpha_i = -lambda_i (x_{i-1} + x_{i+1}) along lines (periodic).
template <typename TG>
__global__ void band_grad_kernel(const TG* __restrict__ lam, const TG* __restrict__ x, TG* __restrict__ ga,
                                 int64_t nx, int64_t ny, int64_t nz, int dir, int64_t total) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int64_t ix = idx % nx, iy = (idx / nx) % ny, iz = idx / (nx * ny);
  int64_t es, n, c;
  if (dir == 0) { es = 1; n = nx; c = ix; }
  else if (dir == 1) { es = nx; n = ny; c = iy; }
  else { es = nx * ny; n = nz; c = iz; }
  const int64_t im = (c == 0) ? idx + (n - 1) * es : idx - es;
  const int64_t ip = (c == n - 1) ? idx - (n - 1) * es : idx + es;
  ga[idx] = -lam[idx] * (x[im] + x[ip]);
}

cudaError_t launch_band_grad(bool f64, const void* lam, const void* x, void* ga, int64_t nx, int64_t ny,
                             int64_t nz, int dir, cudaStream_t s) {
  const int64_t total = nx * ny * nz;
  const int threads = 256;
  const int64_t blocks = (total + threads - 1) / threads;
  if (f64)
    band_grad_kernel<double><<<(unsigned)blocks, threads, 0, s>>>((const double*)lam, (const double*)x,
                                                                   (double*)ga, nx, ny, nz, dir, total);
  else
    band_grad_kernel<float><<<(unsigned)blocks, threads, 0, s>>>((const float*)lam, (const float*)x,
                                                                  (float*)ga, nx, ny, nz, dir, total);
  return cudaGetLastError();
}

}  // namespace cbs
