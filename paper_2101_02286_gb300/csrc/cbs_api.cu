// cbs_api.cu -- the C-ABI: plan creation (validation, partition choice,
// host pre-factorisation, upload) and the solve entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "cbs_bands.h"
#include "cbs_line_launch.cuh"
#include "cbs_plan_struct.h"

using namespace cbs;

namespace cbs {
cudaError_t launch_var(int M, int KS, bool adj, bool f64, const VarArgs& a, const DevLineTables& t,
                       cudaStream_t s);
cudaError_t launch_band_grad(bool f64, const void* lam, const void* x, void* ga, int64_t nx, int64_t ny,
                             int64_t nz, int dir, cudaStream_t s);
struct BatchProblem;
int batch_variant_host(int R, int KS, int M, int MODE, bool full);
cudaError_t batch_configure(size_t smem);
size_t batch_smem(size_t tile_bytes);
cudaError_t batch_launch(const BatchProblem* probs, const int4* items, int nitems, const void* const* ins,
                         void* const* outs, int count, int grid, size_t smem, cudaStream_t s);
size_t batch_problem_bytes();
void batch_fill_problem(void* dst, const LineArgs& a, const DevLineTables& t, int variant, int user);
void batch_fill_long(void* dst, const LongArgs& la, const DevLineTables& inner, const LongWarpArgs& wa, int R,
                     int MODE, int user);
int batch_long_variant_host(int R, int MODE);
int batch_f32_variant_host(int R, int KS, int M);
size_t batch_long_bytes(int R, int K);
constexpr int kBatchMax = 256;
// automatic batch mode: per-problem launches from this many unknowns per
// problem on average (a launch then carries tens of microseconds of work)
constexpr int64_t kBatchPerProblemUnknowns = (int64_t)1 << 20;
bool tma_eligible(int mode, int KS, bool staggered, bool in64, bool out64, const LineArgs& a, const DevLineTables& t);
cudaError_t launch_tma(int mode, int KS, const LineArgs& a, const DevLineTables& t, int tile_lines, int fault,
                       cudaStream_t s);
}  // namespace cbs

namespace {

// autotuner cache: descriptor key -> (partitions per line, kernel variant)
using TuneKey = std::tuple<int64_t, int64_t, int64_t, int, int, int, int, int, int, int, int>;
struct TuneChoice {
  int segments = 0, variant = 0, tile_lines = 0;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune_cache;
TuneKey tune_key(const cbs_desc* d) {
  return TuneKey(d->dims[0], d->dims[1], d->dims[2], d->direction, d->bandwidth, d->precision, d->in_dtype,
                 d->out_dtype, d->rhs_kind, d->rhs_terms, d->lhs_kind);
}
TuneChoice tuned_choice(const cbs_desc* d) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune_cache.find(tune_key(d));
  return it == g_tune_cache.end() ? TuneChoice() : it->second;
}

thread_local std::string g_err;
thread_local int g_launches = 0;

cbs_status fail(cbs_status s, const std::string& msg) {
  g_err = msg;
  return s;
}
cbs_status cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return CBS_ERR_CUDA;
}

// Autotuner input: values in [lo, lo + span) from a hash of the element
// index (varying, so the kernels take their usual paths; a constant field
// would make every derivative zero).
template <typename T>
__global__ void tune_fill_kernel(T* p, int64_t n, double lo, double span) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)i * 0x9E3779B9u ^ (uint32_t)(i >> 32);
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    p[i] = (T)(lo + span * (double)(h >> 8) * (1.0 / 16777216.0));
  }
}

cudaError_t tune_fill(void* p, int64_t n, bool f64, double lo, double span) {
  const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
  if (f64) tune_fill_kernel<double><<<blocks, 256>>>((double*)p, n, lo, span);
  else tune_fill_kernel<float><<<blocks, 256>>>((float*)p, n, lo, span);
  return cudaGetLastError();
}

int next_pow2(int p) {
  int w = 1;
  while (w < p) w *= 2;
  return w;
}

}  // namespace



namespace {

bool is_refine(int precision) { return precision == CBS_FP32_REFINE || precision == CBS_FP32_REFINE_I64; }
int mode_of(int precision) {
  return precision == CBS_FP64 ? kModeF64
         : precision == CBS_FP32 ? kModeF32
         : precision == CBS_FP32_REFINE ? kModeRefine
                                        : kModeRefineI64;
}

// Symmetric Toeplitz bands of half width r with unit diagonal: a_{+-1} =
// alpha, a_{+-2} = d->beta, a_{+-3} = d->gamma.
Bands desc_bands(const cbs_desc* d, int r, double alpha) {
  Bands A;
  A.r = r;
  for (int k = 0; k < 2 * kMaxR + 1; k++) A.v[k] = 0.0;
  A.v[r] = 1.0;
  A.v[r - 1] = A.v[r + 1] = alpha;
  if (r >= 2) A.v[r - 2] = A.v[r + 2] = d->beta;
  if (r >= 3) A.v[r - 3] = A.v[r + 3] = d->gamma;
  return A;
}

// Block-entry plans (CBS_LHS_BLOCK): the periodic bands of the flattened
// block-tridiagonal matrix, and partition sizes in whole points (the n / b
// points split as evenly as possible over p partitions).  false when p
// exceeds the points.
PBands desc_block_bands(const cbs_desc* d) {
  const int b = d->block_size;
  return block_bands(b, d->blocks, d->blocks + b * b, d->blocks + 2 * b * b);
}
bool block_sizes(int n, int b, int p, int sizes[3]) {
  const int npts = n / b;
  if (p < 1 || p > npts) return false;
  const int small = npts / p, extra = npts % p;
  sizes[0] = extra ? extra : p;
  sizes[1] = (small + (extra ? 1 : 0)) * b;
  sizes[2] = small * b;
  return true;
}

bool is_staggered(const cbs_desc* d) { return d->rhs_kind == CBS_RHS_STAGGERED || d->rhs_kind == CBS_RHS_MIDPOINT; }

cbs_status validate(const cbs_desc* d) {
  if (!d) return fail(CBS_ERR_INVALID_ARG, "null descriptor");
  for (int k = 0; k < 3; k++)
    if (d->dims[k] < 1) return fail(CBS_ERR_INVALID_ARG, "dims must be >= 1");
  if (d->direction < 0 || d->direction > 2) return fail(CBS_ERR_INVALID_ARG, "direction must be 0, 1 or 2");
  if (d->bandwidth != 3 && d->bandwidth != 5 && d->bandwidth != 7)
    return fail(CBS_ERR_INVALID_ARG, "bandwidth must be 3, 5 or 7");
  if (d->cyclic != 0 && d->cyclic != 1) return fail(CBS_ERR_INVALID_ARG, "cyclic must be 0 or 1");
  if (d->lhs_kind != CBS_LHS_TOEPLITZ && d->lhs_kind != CBS_LHS_VARIABLE && d->lhs_kind != CBS_LHS_BLOCK)
    return fail(CBS_ERR_INVALID_ARG, "bad lhs_kind");
  if (d->lhs_kind == CBS_LHS_BLOCK) {
    if (d->block_size != 2) return fail(CBS_ERR_UNSUPPORTED, "block entries: block_size 2");
    if (d->bandwidth != 7) return fail(CBS_ERR_INVALID_ARG, "block entries of size 2: bandwidth 7 (half bandwidth 3)");
    if (!d->blocks) return fail(CBS_ERR_INVALID_ARG, "block entries need the host array of L, D, U");
    for (int k = 0; k < 3 * d->block_size * d->block_size; k++)
      if (!std::isfinite(d->blocks[k])) return fail(CBS_ERR_INVALID_ARG, "non-finite block entries");
    if (d->dims[d->direction] % d->block_size != 0)
      return fail(CBS_ERR_INVALID_ARG, "block entries: the line length must be a multiple of block_size");
    if (d->rhs_kind != CBS_RHS_NONE) return fail(CBS_ERR_UNSUPPORTED, "block entries: right-hand side given (no stencil)");
    if (d->precision != CBS_FP64 && d->precision != CBS_FP32)
      return fail(CBS_ERR_UNSUPPORTED, "block entries: FP64 or FP32 (the refinement residual is for Toeplitz bands)");
  }
  if (d->rhs_kind < CBS_RHS_NONE || d->rhs_kind > CBS_RHS_MIDPOINT) return fail(CBS_ERR_INVALID_ARG, "bad rhs_kind");
  if (d->rhs_kind == CBS_RHS_CENTRAL) {
    if (d->rhs_terms < 1 || d->rhs_terms > 3) return fail(CBS_ERR_INVALID_ARG, "rhs_terms must be 1..3");
    if (!(d->h > 0.0) || !std::isfinite(d->h)) return fail(CBS_ERR_INVALID_ARG, "h must be positive");
    if (!d->cyclic && d->closure_rows == 0)
      return fail(CBS_ERR_UNSUPPORTED, "an acyclic derivative needs boundary closures (closure_rows)");
  }
  if (is_staggered(d)) {
    if (d->rhs_terms < 1 || d->rhs_terms > 2) return fail(CBS_ERR_INVALID_ARG, "staggered stencils: rhs_terms 1..2");
    if (d->rhs_shift != 0 && d->rhs_shift != 1) return fail(CBS_ERR_INVALID_ARG, "rhs_shift must be 0 or 1");
    if (d->rhs_kind == CBS_RHS_STAGGERED && (!(d->h > 0.0) || !std::isfinite(d->h)))
      return fail(CBS_ERR_INVALID_ARG, "h must be positive");
    if (!d->cyclic) return fail(CBS_ERR_UNSUPPORTED, "the staggered stencils are periodic: needs cyclic = 1");
    if (d->lhs_kind != CBS_LHS_TOEPLITZ) return fail(CBS_ERR_UNSUPPORTED, "staggered stencils: Toeplitz bands only");
    if (d->bandwidth > 5) return fail(CBS_ERR_UNSUPPORTED, "staggered stencils: bandwidth 3 or 5");
  }
  if (d->closure_rows < 0) return fail(CBS_ERR_INVALID_ARG, "closure_rows must be >= 0");
  if (d->closure_rows > 0) {
    if (d->cyclic || d->rhs_kind != CBS_RHS_CENTRAL || d->lhs_kind != CBS_LHS_TOEPLITZ)
      return fail(CBS_ERR_UNSUPPORTED, "boundary closures: acyclic lines, central stencil, Toeplitz bands");
    if (!d->closure) return fail(CBS_ERR_INVALID_ARG, "boundary closures need the host array");
    if (d->closure_rows > cbs::kMaxClosureRows || d->closure_width < 1 || d->closure_width > cbs::kMaxClosureWidth)
      return fail(CBS_ERR_INVALID_ARG, "closure_rows 1..4, closure_width 1..16");
  }
  if (d->precision < CBS_FP64 || d->precision > CBS_FP32_REFINE_I64) return fail(CBS_ERR_INVALID_ARG, "bad precision");
  if (is_refine(d->precision) && (d->refine_sweeps < 1 || d->refine_sweeps > 2))
    return fail(CBS_ERR_INVALID_ARG, "refine_sweeps must be 1 or 2");
  if (d->in_dtype != CBS_DTYPE_F64 && d->in_dtype != CBS_DTYPE_F32) return fail(CBS_ERR_INVALID_ARG, "bad in_dtype");
  if (d->out_dtype != CBS_DTYPE_F64 && d->out_dtype != CBS_DTYPE_F32) return fail(CBS_ERR_INVALID_ARG, "bad out_dtype");
  if (d->precision != CBS_FP32 && d->out_dtype != CBS_DTYPE_F64)
    return fail(CBS_ERR_INVALID_ARG, "FP64 and FP32_REFINE write FP64 output");
  if (!std::isfinite(d->alpha) || !std::isfinite(d->beta) || !std::isfinite(d->gamma))
    return fail(CBS_ERR_INVALID_ARG, "non-finite bands");
  if (d->precision == CBS_FP32 && d->in_dtype != d->out_dtype)
    return fail(CBS_ERR_UNSUPPORTED, "FP32 mode: input and output share the element type");
  if (d->precision != CBS_FP32 && d->in_dtype == CBS_DTYPE_F32 && d->rhs_kind != CBS_RHS_NONE)
    return fail(CBS_ERR_UNSUPPORTED, "FP32 input with an FP64 output: right-hand side given (no stencil)");
  if (d->segments < 0) return fail(CBS_ERR_INVALID_ARG, "segments must be >= 0");
  if ((d->direction == 1 && d->dims[2] > 65535) || (d->direction == 2 && d->dims[1] > 65535))
    return fail(CBS_ERR_UNSUPPORTED, "y/z lines: the remaining grid extent must be <= 65535");
  if (d->dims[0] * d->dims[1] * d->dims[2] >= (int64_t)1 << 40) return fail(CBS_ERR_UNSUPPORTED, "field too large");
  if (d->lhs_kind == CBS_LHS_VARIABLE) {
    if (d->bandwidth != 3) return fail(CBS_ERR_UNSUPPORTED, "variable bands: tridiagonal only");
    if (!d->cyclic) return fail(CBS_ERR_UNSUPPORTED, "variable bands: cyclic only");
    if (!d->bands) return fail(CBS_ERR_INVALID_ARG, "variable bands need the alpha field pointer");
    if (is_refine(d->precision)) return fail(CBS_ERR_UNSUPPORTED, "variable bands: FP64 or FP32");
    const int want = d->precision == CBS_FP64 ? CBS_DTYPE_F64 : CBS_DTYPE_F32;
    if (d->in_dtype != want || d->out_dtype != want)
      return fail(CBS_ERR_INVALID_ARG, "variable bands: input, output and alpha share the precision's dtype");
  }
  return CBS_OK;
}

// Default partition count for the on-chip kernel: the fewest partitions
// (<= 32 lanes) whose size fits the register budget of the mode.
int default_segments(int n, int r, int precision) {
  const int target = 16;
  (void)precision;
  // whole 16-row partitions (compile-time partition sizes in the kernels)
  if (n % 16 == 0 && n / 16 <= kMaxLanes && 16 >= 2 * r) return n / 16;
  for (int p = 1; p <= kMaxLanes; p *= 2)
    if ((n + p - 1) / p <= target && n / p >= 2 * r) return p;
  for (int p = kMaxLanes; p >= 1; p /= 2)
    if (n / p >= 2 * r && (n + p - 1) / p <= 32) return p;
  return 0;
}

}  // namespace

namespace cbs {
cbs_status set_error(cbs_status s, const std::string& msg) { return fail(s, msg); }
void set_launch_count(int n) { g_launches = n; }
}  // namespace cbs

namespace {
// Fill the kernel-side tables of plan tables T (fac, S/R, b-hat blocks,
// bands, interface coefficients, shared-memory tile geometry) and upload the
// per-lane interface coefficients to a new device buffer *dbuf.
cbs_status fill_dev_tables(DevLineTables& D, const LineTables& T, const Bands& A, const cbs_desc* d, int pw_override,
                           void** dbuf, bool with_bulk = true) {
  const int r = T.r, F = 2 * r + 1, p = T.p;
  std::memset(&D, 0, sizeof(D));
  if (with_bulk && T.nmax > kMaxBulk) return fail(CBS_ERR_UNSUPPORTED, "partitions too long");
  for (int j = 0; j < T.nmax && with_bulk; j++)
    for (int c = 0; c < F; c++) {
      D.fac[j * F + c] = T.fac[(size_t)j * F + c];
      D.facF[j * F + c] = (float)T.fac[(size_t)j * F + c];
    }
  for (int j = 0; j < T.rows_big - r && with_bulk; j++)
    for (int c = 0; c < 2 * r; c++) {
      D.srB[j * 2 * r + c] = T.srB[(size_t)j * 2 * r + c];
      D.srBF[j * 2 * r + c] = (float)D.srB[j * 2 * r + c];
    }
  for (int j = 0; j < T.rows_small - r && with_bulk; j++)
    for (int c = 0; c < 2 * r; c++) {
      D.srS[j * 2 * r + c] = T.srS[(size_t)j * 2 * r + c];
      D.srSF[j * 2 * r + c] = (float)D.srS[j * 2 * r + c];
    }
  for (int q = 0; q < r; q++)
    for (int e = 0; e < r; e++) {
      D.Lt[q][e] = T.Lt[q][e];
      D.Ut[q][e] = T.Ut[q][e];
      D.LtF[q][e] = (float)T.Lt[q][e];
      D.UtF[q][e] = (float)T.Ut[q][e];
    }
  const int ns = (int)T.stages.size();
  // uniform interface: p a power of two, cyclic, only PCR / final stages and
  // identical blocks on every lane (then sources are (i -+ s) mod p)
  {
    const int rr = r * r;
    bool uni = T.cyclic && (p & (p - 1)) == 0 && ns <= kMaxStages;
    for (int st = 0; st < ns && uni; st++) {
      const Stage& S_ = T.stages[st];
      if (S_.type != kPcr && S_.type != kFinal) uni = false;
      for (int i = 0; i < p && uni; i++) {
        for (int m = 0; m < 3 * rr; m++)
          if (T.coef[((size_t)st * 3 * rr + m) * p + i] != T.coef[((size_t)st * 3 * rr + m) * p]) uni = false;
        if (S_.type == kPcr) {
          if (T.src[(size_t)(st * 2 + 0) * p + i] != ((i - S_.s) & (p - 1)) ||
              T.src[(size_t)(st * 2 + 1) * p + i] != ((i + S_.s) & (p - 1)))
            uni = false;
        }
      }
    }
    D.uniform = uni ? 1 : 0;
    if (uni)
      for (int st = 0; st < ns; st++) {
        D.ustage_s[st] = (T.stages[st].type == kPcr) ? T.stages[st].s : 0;
        for (int m = 0; m < 3 * rr; m++) {
          D.ucoef[st][m] = T.coef[((size_t)st * 3 * rr + m) * p];
          D.ucoefF[st][m] = (float)D.ucoef[st][m];
        }
      }
  }
  for (int k = 0; k < F; k++) {
    D.band[k] = A.v[k];
    D.bandHi[k] = (float)A.v[k];
    D.bandLo[k] = (float)(A.v[k] - (double)D.bandHi[k]);
  }
  D.n = T.n;
  D.r = r;
  D.p = p;
  D.pw = pw_override ? pw_override : next_pow2(p);
  D.rows_big = T.rows_big;
  D.rows_small = T.rows_small;
  D.count_big = T.count_big;
  D.nstage = ns;
  D.cyclic = T.cyclic ? 1 : 0;
  for (int st = 0; st < ns && st < kMaxStages; st++) {
    D.stage_has_c[st] = T.stage_has_c[st];
    D.stage_msg[st] = T.stage_msg[st];
  }
  // shared-memory tile geometry (see tile_copy): sp odd, lsz chosen so the
  // lanes of different lines in one wavefront hit different banks
  {
    const bool wide = (d->in_dtype == CBS_DTYPE_F64 || d->out_dtype == CBS_DTYPE_F64);
    const int mod = wide ? 16 : 32;
    const int pw = D.pw;
    D.sp = pw + 1;
    const int target = (pw < mod) ? pw : 1;
    int lsz = T.rows_big * D.sp;
    while (lsz % mod != target % mod) lsz++;
    D.lsz = lsz;
    D.bound = T.count_big * T.rows_big;
    auto mag = [](int dd) -> unsigned {
      return dd <= 1 ? 0u : (unsigned)((((unsigned long long)1 << 32) + (unsigned)dd - 1) / (unsigned)dd);
    };
    D.mag_b = mag(T.rows_big);
    D.mag_s = mag(T.rows_small);
    D.mag_n = mag(T.n);
    D.rows_lg = -1;
    if (T.count_big == p && (T.rows_big & (T.rows_big - 1)) == 0) {
      int lg = 0;
      while ((1 << lg) < T.rows_big) lg++;
      D.rows_lg = lg;
    }
  }
  const size_t ncoef = T.coef.size(), nsrc = T.src.size();
  const size_t bytes = ncoef * sizeof(double) + ncoef * sizeof(float) + nsrc * sizeof(int) + 256;
  std::vector<float> coefF(T.coef.begin(), T.coef.end());
  cudaError_t e = cudaMalloc(dbuf, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(plan tables)");
  char* base = (char*)*dbuf;
  e = cudaMemcpy(base, T.coef.data(), ncoef * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(base + ncoef * sizeof(double), coefF.data(), ncoef * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(base + ncoef * (sizeof(double) + sizeof(float)), T.src.data(), nsrc * sizeof(int),
                   cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(*dbuf);
    *dbuf = nullptr;
    return cuda_fail(e, "uploading plan tables");
  }
  D.coef = (const double*)base;
  D.coefF = (const float*)(base + ncoef * sizeof(double));
  D.src = (const int*)(base + ncoef * (sizeof(double) + sizeof(float)));
  return CBS_OK;
}

// Leading entries of the first r rows of D^{-1} for a bulk block of N rows:
// keeps K entries per row with a tail below 2^-60 of the row's l1 norm (K = N
// when the rows do not decay).  G is [q][K].
static int truncated_inverse_rows(const LineTables& T, int N, int r, std::vector<double>& G) {
  std::vector<double> Gfull = bulk_inverse_rows(T, N, r);
  int K = 1;
  for (int q = 0; q < r; q++) {
    double tot = 0.0;
    for (int j = 0; j < N; j++) tot += std::fabs(Gfull[(size_t)q * N + j]);
    double tail = 0.0;
    int kq = N;
    for (int j = N - 1; j >= 0; j--) {
      tail += std::fabs(Gfull[(size_t)q * N + j]);
      if (tail > std::ldexp(tot, -60)) {
        kq = j + 1;
        break;
      }
    }
    K = std::max(K, kq);
  }
  G.assign((size_t)r * K, 0.0);
  for (int q = 0; q < r; q++)
    for (int j = 0; j < K; j++) G[(size_t)q * K + j] = Gfull[(size_t)q * N + j];
  return K;
}

// Segment count of the warp-per-segment layout for x-lines of n rows: the
// smallest p with n - p r a multiple of 16 whose segments get 32 x 16 + r or
// 31 x 16 + r rows; 0 when there is none (n below two such segments).
int warp_layout_segments(int n, int r) {
  for (int64_t p = std::max<int64_t>(2, (n + 16 * 32 + r - 1) / (16 * 32 + r)); p <= n / (16 * 31 + r); p++) {
    if ((n - p * r) % 16 != 0) continue;
    const int64_t T16 = (n - p * r) / 16, K16 = (T16 + p - 1) / p;
    if (K16 == 32) return (int)p;
    if (K16 < 32) break;
  }
  return 0;
}

// The outer interface system of a long-line plan decoupled to FP64 rounding:
// every coupling block below 2^-60 of the diagonal blocks, which agree to
// 2^-50.  Then x~_i = D-hat^{-1} b-hat_i; Dinv gets D-hat^{-1} (r x r).
bool outer_decoupled(const LineTables& T, int r, double* Dinv) {
  const int p = T.p, rr = r * r;
  if ((int)T.Dhat.size() < p * rr || (int)T.Lhat.size() < p * rr || (int)T.Uhat.size() < p * rr) return false;
  double dmax = 0.0, cmax = 0.0, ddiff = 0.0;
  for (int e = 0; e < rr; e++) dmax = std::fmax(dmax, std::fabs(T.Dhat[e]));
  for (int i = 0; i < p; i++)
    for (int e = 0; e < rr; e++) {
      ddiff = std::fmax(ddiff, std::fabs(T.Dhat[(size_t)i * rr + e] - T.Dhat[e]));
      cmax = std::fmax(cmax, std::fmax(std::fabs(T.Lhat[(size_t)i * rr + e]), std::fabs(T.Uhat[(size_t)i * rr + e])));
    }
  if (!(dmax > 0.0) || !(cmax <= std::ldexp(dmax, -60)) || !(ddiff <= std::ldexp(dmax, -50))) return false;
  const double* D = T.Dhat.data();
  if (r == 1) {
    if (!(std::fabs(D[0]) > 0.0)) return false;
    Dinv[0] = 1.0 / D[0];
    return std::isfinite(Dinv[0]);
  }
  if (r != 2) return false;
  const double det = D[0] * D[3] - D[1] * D[2];
  if (!(std::fabs(det) > 1e-12 * dmax * dmax)) return false;
  Dinv[0] = D[3] / det;
  Dinv[1] = -D[1] / det;
  Dinv[2] = -D[2] / det;
  Dinv[3] = D[0] / det;
  return std::isfinite(Dinv[0]) && std::isfinite(Dinv[1]) && std::isfinite(Dinv[2]) && std::isfinite(Dinv[3]);
}

// Compact stage list (LwIface) of an inner acyclic system T of P <= 32
// partitions for the interface precision `bit` (1: FP64, 2: FP32): the
// stages whose couplings exceed rounding keep their messages; the others
// with C != I are local products, folded into the next message stage (its
// KM and KP then act on the neighbours' values from before the fold: KM
// P_{i-s}, KP P_{i+s}) or into one final product.  Blocks of lanes >= P are
// zero.  False when a message stage is not a PCR step with partners i -+ s.
bool lw_compact(const LineTables& T, int r, int bit, LwIface& f, std::vector<double>& tab) {
  f = LwIface{};
  tab.clear();
  const int P = T.p, rr = r * r, ns = (int)T.stages.size();
  if (P > 32 || ns > kMaxStages) return false;
  auto cf = [&](int st, int m, int i, int e) { return T.coef[((size_t)(st * 3 + m) * rr + e) * P + i]; };
  auto mul = [&](const double* A, const double* B, double* C) {  // C = A B (r x r)
    for (int q = 0; q < r; q++)
      for (int e = 0; e < r; e++) {
        double v = 0.0;
        for (int k = 0; k < r; k++) v += A[q * r + k] * B[k * r + e];
        C[q * r + e] = v;
      }
  };
  std::vector<double> pend((size_t)P * rr, 0.0);  // pending local product per lane
  auto reset = [&] {
    std::fill(pend.begin(), pend.end(), 0.0);
    for (int i = 0; i < P; i++)
      for (int q = 0; q < r; q++) pend[(size_t)i * rr + q * r + q] = 1.0;
  };
  reset();
  bool has_pend = false;
  auto push = [&](const std::vector<double>& blk) {  // blk[i * rr + e], lanes < P
    for (int e = 0; e < rr; e++)
      for (int i = 0; i < 32; i++) tab.push_back(i < P ? blk[(size_t)i * rr + e] : 0.0);
  };
  for (int st = 0; st < ns; st++) {
    const bool msg = (T.stage_msg[st] & bit) != 0, hc = T.stage_has_c[st] != 0;
    if (!msg && !hc) continue;
    std::vector<double> C((size_t)P * rr);
    for (int i = 0; i < P; i++) {
      double Ci[kMaxR * kMaxR];
      for (int e = 0; e < rr; e++) Ci[e] = cf(st, 0, i, e);
      mul(Ci, &pend[(size_t)i * rr], &C[(size_t)i * rr]);
    }
    if (!msg) {
      pend = C;
      has_pend = true;
      continue;
    }
    if (T.stages[st].type != kPcr || f.ne == kLwMaxEnt) return false;
    const int s = T.stages[st].s;
    std::vector<double> KM((size_t)P * rr, 0.0), KP((size_t)P * rr, 0.0);
    for (int i = 0; i < P; i++) {
      const int jm = i - s, jp = i + s;
      double K[kMaxR * kMaxR];
      for (int e = 0; e < rr; e++) K[e] = cf(st, 1, i, e);
      if (jm >= 0) {
        if (T.src[(size_t)(st * 2 + 0) * P + i] != jm) return false;
        mul(K, &pend[(size_t)jm * rr], &KM[(size_t)i * rr]);
      } else {
        for (int e = 0; e < rr; e++)
          if (K[e] != 0.0) return false;
      }
      for (int e = 0; e < rr; e++) K[e] = cf(st, 2, i, e);
      if (jp < P) {
        if (T.src[(size_t)(st * 2 + 1) * P + i] != jp) return false;
        mul(K, &pend[(size_t)jp * rr], &KP[(size_t)i * rr]);
      } else {
        for (int e = 0; e < rr; e++)
          if (K[e] != 0.0) return false;
      }
    }
    const bool withc = hc || has_pend;
    f.s[f.ne] = s;
    f.flags[f.ne] = 1 | (withc ? 2 : 0);
    f.off[f.ne] = (int)(tab.size() / 32);
    if (withc) push(C);
    push(KM);
    push(KP);
    f.ne++;
    reset();
    has_pend = false;
  }
  if (has_pend) {
    if (f.ne == kLwMaxEnt) return false;
    f.s[f.ne] = 0;
    f.flags[f.ne] = 2;
    f.off[f.ne] = (int)(tab.size() / 32);
    push(pend);
    f.ne++;
  }
  return true;
}

// Long lines: p segments per line, one CTA per segment (cbs_long.cu).
//
// Segment layout.  When n - p r is a multiple of 16, the segments get
// 16 K + r rows (the first cbig of them) or 16 (K - 1) + r rows, so every
// segment's bulk is a whole number of 16-row inner partitions and the segment
// kernel runs with compile-time partition sizes; a segment's end rows are
// computed from the same truncated rows of D^{-1} when both sizes agree on
// them to 2^-60.  Otherwise p must divide n and the segments are equal, with
// ragged inner partitions.
cbs_status create_long(cbs_plan* P, const cbs_desc* d) {
  if (d->rhs_kind != CBS_RHS_NONE || !d->cyclic || d->lhs_kind != CBS_LHS_TOEPLITZ)
    return fail(CBS_ERR_UNSUPPORTED, "long lines: right-hand side given, cyclic Toeplitz bands");
  const int n = P->n, r = P->r;
  if (r > 2) return fail(CBS_ERR_UNSUPPORTED, "long lines: bandwidth 3 or 5");
  if (d->closure_rows > 0) return fail(CBS_ERR_UNSUPPORTED, "long lines: no boundary closures");
  // y/z lines run a tile of adjacent lines per CTA (kLongLines, or half as
  // many above 512 / kLongLines inner partitions): at most 1024 / kLongLines
  // inner partitions (segments of about 2048 rows)
  const bool tiled = d->direction != 0;
  const int max_inner = tiled ? 1024 / kLongLines : 512;
  int p = d->segments;
  if (!p) p = warp_layout_segments(n, r);  // a warp per segment where it applies
  if (!p) {  // segments of about 512 rows (y/z: tiles of 8 lines x 32 inner partitions), 1024 (x, n <= 2^16),
             // 4096 (longer x-lines)
    p = tiled ? (n + 511) / 512 : n <= 65536 ? (n + 1023) / 1024 : (n + 4095) / 4096;
    if ((n - (int64_t)p * r) % 16 != 0)
      while (p < n && n % p) p++;
  }
  const Bands A = desc_bands(d, r, d->alpha);
  bool singular = false;
  std::string msg;
  std::vector<double> G;
  int K = 0;
  bool full = false;
  int sizes[3] = {p, 0, 0};
  // whole 16-row inner partitions
  if (p >= 1 && (n - (int64_t)p * r) % 16 == 0 && n - (int64_t)p * r >= 32 * (int64_t)p) {
    const int64_t T16 = (n - (int64_t)p * r) / 16;        // 16-row blocks of all bulks
    const int64_t K16 = (T16 + p - 1) / p;                 // blocks of a big segment
    const int64_t cbig = T16 - (int64_t)p * (K16 - 1);     // in [1, p]
    if (K16 <= max_inner && K16 - 1 >= 2 * r) {
      sizes[0] = (int)cbig;
      sizes[1] = (int)(16 * K16 + r);
      sizes[2] = (int)(16 * (K16 - 1) + r);
      msg = build_line_tables(P->host, n, A, p, true, &singular, 1 << 30, sizes);
      if (msg.empty())
        msg = build_line_tables(P->inner, (int)(16 * K16), A, (int)K16, false, &singular, 1 << 30);
      if (msg.empty() && cbig < p)
        msg = build_line_tables(P->inner_small, (int)(16 * (K16 - 1)), A, (int)(K16 - 1), false, &singular,
                                1 << 30);
      if (!msg.empty()) return fail(singular ? CBS_ERR_SINGULAR : CBS_ERR_UNSUPPORTED, msg);
      K = truncated_inverse_rows(P->host, (int)(16 * K16), r, G);
      full = true;
      if (cbig < p) {  // the small segments must share the truncated rows
        std::vector<double> G2;
        const int K2 = truncated_inverse_rows(P->host, (int)(16 * (K16 - 1)), r, G2);
        double tot = 0.0, diff = 0.0;
        for (size_t k = 0; k < G.size(); k++) tot += std::fabs(G[k]);
        if (K2 != K || K >= 16 * (K16 - 1)) full = false;
        for (size_t k = 0; full && k < G.size(); k++) diff = std::fmax(diff, std::fabs(G[k] - G2[k]));
        if (diff > std::ldexp(tot, -60)) full = false;
      }
    }
  }
  if (!full) {  // the first n mod p segments get ceil(n / p) rows, the rest floor
    if (p < 1 || p > n) return fail(CBS_ERR_INVALID_ARG, "long lines: bad segment count");
    sizes[0] = n % p ? n % p : p;
    sizes[1] = (n + p - 1) / p;
    sizes[2] = n / p;
  }
  if (p > 65535) return fail(CBS_ERR_UNSUPPORTED, "long lines: at most 65535 segments per line");
  const int m = sizes[1], N = m - r;
  const int pin = full ? N / 16 : (N + 15) / 16;
  const int Ns = sizes[2] - r, pin_s = full ? Ns / 16 : (Ns + 15) / 16;
  if (pin > max_inner)
    return fail(CBS_ERR_UNSUPPORTED, tiled ? "long y/z lines: segments above 2048 rows (raise segments)"
                                           : "long lines: segments above 8192 rows (raise segments)");
  if (N < 2 * r * pin || Ns < 2 * r * pin_s || sizes[2] < 4 * r)
    return fail(CBS_ERR_INVALID_ARG, "long lines: segments too short");
  if (!full) {
    msg = build_line_tables(P->host, n, A, p, true, &singular, 1 << 30, sizes);
    if (msg.empty()) msg = build_line_tables(P->inner, N, A, pin, false, &singular, 1 << 30);
    if (msg.empty() && sizes[0] < p) msg = build_line_tables(P->inner_small, Ns, A, pin_s, false, &singular, 1 << 30);
    if (!msg.empty()) return fail(singular ? CBS_ERR_SINGULAR : CBS_ERR_UNSUPPORTED, msg);
    K = truncated_inverse_rows(P->host, N, r, G);
    if (sizes[0] < p) {  // the smaller segments must share the truncated rows
      std::vector<double> G2;
      const int K2 = truncated_inverse_rows(P->host, Ns, r, G2);
      double tot = 0.0, diff = 0.0;
      for (size_t k = 0; k < G.size(); k++) tot += std::fabs(G[k]);
      bool same = K2 == K && K < Ns;
      for (size_t k = 0; same && k < G.size(); k++) diff = std::fmax(diff, std::fabs(G[k] - G2[k]));
      if (!same || diff > std::ldexp(tot, -60))
        return fail(CBS_ERR_UNSUPPORTED, "long lines: segments too short for this band (choose p dividing n)");
    }
  }
  // x-lines whose segments have 32 (31) whole 16-row inner partitions and
  // whose outer system is decoupled: a warp per segment (cbs_long_warp.cu)
  double Dinv[kMaxR * kMaxR] = {};
  P->long_warp = full && m == 16 * 32 + r && (sizes[0] == p || sizes[2] == 16 * 31 + r) && p >= 2 &&
                 long_warp_fits(r, K, d->in_dtype == CBS_DTYPE_F64 ? 8 : 4, tiled) &&
                 outer_decoupled(P->host, r, Dinv);
  if (!P->long_warp && 2 * (size_t)p * r * sizeof(double) > 227 * 1024)
    return fail(CBS_ERR_UNSUPPORTED, "long lines: more than 14528 interface unknowns per line (raise the segment size)");
  cbs_status st = fill_dev_tables(P->dev, P->host, A, d, 0, &P->dbuf, false);
  if (st) return st;
  const int threads = ((pin + 31) / 32) * 32;
  st = fill_dev_tables(P->dev_inner, P->inner, A, d, threads, &P->lbuf, true);
  if (st) return st;
  if (sizes[0] < p) {
    const int threads_s = ((P->inner_small.p + 31) / 32) * 32;
    st = fill_dev_tables(P->dev_inner_small, P->inner_small, A, d, threads_s, &P->lbuf_small, true);
    if (st) return st;
  }
  P->inner_full = full;
  // scratch: yb, cc (2r per segment), xt (r per segment), then G
  const size_t nseg = (size_t)P->nlines * p;
  // G as float pairs for the warp-per-segment path (double-float dot products)
  std::vector<float> Gf(2 * G.size());
  for (size_t k = 0; k < G.size(); k++) {
    Gf[k] = (float)G[k];
    Gf[G.size() + k] = (float)(G[k] - (double)Gf[k]);
  }
  const size_t bytes = (nseg * (5 * r) + G.size()) * sizeof(double) + Gf.size() * sizeof(float);
  cudaError_t e = cudaMalloc(&P->sbuf, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&P->dstatus, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(P->dstatus, 0, sizeof(int));
  double* sb = (double*)P->sbuf;
  if (e == cudaSuccess)
    e = cudaMemcpy(sb + nseg * 5 * r, G.data(), G.size() * sizeof(double), cudaMemcpyHostToDevice);
  float* gf = reinterpret_cast<float*>(sb + nseg * 5 * r + G.size());
  if (e == cudaSuccess) e = cudaMemcpy(gf, Gf.data(), Gf.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "long-line scratch");
  LongArgs& a = P->largs;
  std::memset(&a, 0, sizeof(a));
  a.yb = sb;
  a.cc = sb + nseg * 2 * r;
  a.xt = sb + nseg * 4 * r;
  a.G = sb + nseg * 5 * r;
  a.K = K;
  a.lines = P->nlines;
  a.n = n;
  a.p = p;
  a.m = m;
  a.r = r;
  a.cbig = sizes[0];
  a.msmall = sizes[2];
  a.sweeps = d->refine_sweeps;
  for (int k = 0; k < 2 * kMaxR + 1; k++) a.band[k] = A.v[k];
  LongGeom& gm = P->lgeom;
  gm.nx = d->dims[0];
  gm.ny = d->dims[1];
  gm.dir = d->direction;
  gm.es = d->direction == 0 ? 1 : d->direction == 1 ? d->dims[0] : d->dims[0] * d->dims[1];
  P->kind = 1;
  P->M = 16;
  P->inner_threads = threads;
  if (P->long_warp) {
    // compact inner systems in the interface precision of the mode's solves
    const int mode = mode_of(d->precision);
    const bool i64 = mode == kModeF64 || mode == kModeRefineI64;
    std::vector<double> tb[2];
    const bool two = sizes[0] < p;
    bool okc = lw_compact(P->inner, r, i64 ? 1 : 2, P->lwifc[0], tb[0]);
    if (okc && two) okc = lw_compact(P->inner_small, r, i64 ? 1 : 2, P->lwifc[1], tb[1]);
    if (!okc) {
      P->long_warp = false;
      if (2 * (size_t)p * r * sizeof(double) > 227 * 1024)
        return fail(CBS_ERR_UNSUPPORTED, "long lines: more than 14528 interface unknowns per line (raise the segment size)");
    } else {
      const size_t es = i64 ? 8 : 4;
      const size_t n0 = tb[0].size(), n1 = two ? tb[1].size() : 0;
      std::vector<unsigned char> hb((n0 + n1) * es);
      for (size_t k = 0; k < n0 + n1; k++) {
        const double v = k < n0 ? tb[0][k] : tb[1][k - n0];
        if (i64) {
          std::memcpy(hb.data() + k * es, &v, 8);
        } else {
          const float fv = (float)v;
          std::memcpy(hb.data() + k * es, &fv, 4);
        }
      }
      e = cudaMalloc(&P->lwbuf, hb.size());
      if (e == cudaSuccess) e = cudaMemcpy(P->lwbuf, hb.data(), hb.size(), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return cuda_fail(e, "long-line interface tables");
      P->lwifc[0].tab = P->lwbuf;
      if (two) P->lwifc[1].tab = static_cast<unsigned char*>(P->lwbuf) + n0 * es;
    }
  }
  if (P->long_warp) {
    LongWarpArgs& w = P->lwargs;
    std::memset(&w, 0, sizeof(w));
    for (int q = 0; q < r; q++)
      for (int e = 0; e < r; e++) {
        w.Dinv[q * r + e] = Dinv[q * r + e];
        w.Lt[q * r + e] = P->host.Lt[q][e];
        w.Ut[q * r + e] = P->host.Ut[q][e];
      }
    w.status = P->dstatus;
    w.gm = P->lgeom;
    w.ngroups = (int)((P->nlines + kLongWarps - 1) / kLongWarps);
    w.Gh = gf;
    w.Gl = gf + G.size();
  }
  return CBS_OK;
}

// The on-chip line kernel of plan P with arguments a: `ks` stencil terms
// compiled in, staggered stencil or not, element types tin -> tout.  Variant
// 0 takes the TMA-fed refinement kernel when the plan and arrays qualify.
cudaError_t launch_line_plan(const cbs_plan* P, const LineArgs& a, int ks, bool stag, int tin, int tout,
                             cudaStream_t s) {
  const int mode = mode_of(P->desc.precision);
  if (P->variant == 0 && tma_eligible(mode, ks, stag, tin == CBS_DTYPE_F64, tout == CBS_DTYPE_F64, a, P->dev)) {
    const cudaError_t e = launch_tma(mode, ks, a, P->dev, P->tile_lines, P->fault, s);
    if (e != cudaErrorNotSupported) return e;  // NotSupported: a tensor map was refused
  }
  const int R = P->r;
#define CBS_L(MO, RR) launch_line_mode_r<MO, RR>(P->M, ks, stag, tin, tout, a, P->dev, s)
  if (mode == kModeF64) return (R == 1) ? CBS_L(0, 1) : (R == 2) ? CBS_L(0, 2) : CBS_L(0, 3);
  if (mode == kModeF32) return (R == 1) ? CBS_L(1, 1) : (R == 2) ? CBS_L(1, 2) : CBS_L(1, 3);
  if (mode == kModeRefine) return (R == 1) ? CBS_L(2, 1) : (R == 2) ? CBS_L(2, 2) : CBS_L(2, 3);
  return (R == 1) ? CBS_L(3, 1) : (R == 2) ? CBS_L(3, 2) : CBS_L(3, 3);
#undef CBS_L
}

}  // namespace

extern "C" {

const char* cbs_last_error_string(void) { return g_err.c_str(); }
int32_t cbs_version(void) { return 100; }
int32_t cbs_last_launch_count(void) { return g_launches; }

cbs_status cbs_schedule(int32_t p, int32_t cyclic, int32_t* stages, int32_t cap, int32_t* count) {
  if (p < 1 || !count || (cap > 0 && !stages)) return fail(CBS_ERR_INVALID_ARG, "bad schedule arguments");
  std::vector<Stage> st = build_schedule(p, cyclic != 0);
  *count = (int32_t)st.size();
  for (int k = 0; k < (int)st.size() && k < cap; k++) {
    stages[3 * k + 0] = st[k].type;
    stages[3 * k + 1] = st[k].s;
    stages[3 * k + 2] = st[k].na;
  }
  return CBS_OK;
}

cbs_status cbs_interface_model(const cbs_desc* d, int32_t p, double* dhat, double* lhat, double* uhat,
                               const double* bhat, double* xt) {
  cbs_status st = validate(d);
  if (st) return st;
  if (d->lhs_kind == CBS_LHS_VARIABLE) return fail(CBS_ERR_UNSUPPORTED, "Toeplitz or block-entry LHS only");
  const int r = (d->bandwidth - 1) / 2, n = (int)d->dims[d->direction];
  if (p < 1 || n < 2 * r * p) return fail(CBS_ERR_INVALID_ARG, "need 1 <= p and n >= 2 r p");
  LineTables T;
  bool singular = false;
  std::string msg;
  if (d->lhs_kind == CBS_LHS_BLOCK) {
    int sizes[3];
    if (!block_sizes(n, d->block_size, p, sizes)) return fail(CBS_ERR_INVALID_ARG, "more partitions than points");
    msg = build_line_tables_periodic(T, n, desc_block_bands(d), p, d->cyclic != 0, &singular, 1 << 30, sizes);
  } else {
    msg = build_line_tables(T, n, desc_bands(d, r, d->alpha), p, d->cyclic != 0, &singular, /*max_lanes=*/1 << 30);
  }
  if (!msg.empty()) return fail(singular ? CBS_ERR_SINGULAR : CBS_ERR_UNSUPPORTED, msg);
  const size_t nb = (size_t)p * r * r;
  if (dhat) std::memcpy(dhat, T.Dhat.data(), nb * sizeof(double));
  if (lhat) std::memcpy(lhat, T.Lhat.data(), nb * sizeof(double));
  if (uhat) std::memcpy(uhat, T.Uhat.data(), nb * sizeof(double));
  if (bhat && xt) {
    std::vector<double> x(bhat, bhat + (size_t)p * r), y((size_t)p * r);
    const int rr = r * r;
    for (int s = 0; s < (int)T.stages.size(); s++) {
      const bool msg = (T.stage_msg[s] & 1) != 0;  // FP64 kernels skip the rest
      for (int i = 0; i < p; i++) {
        const int sm = T.src[(size_t)(s * 2 + 0) * p + i], sp = T.src[(size_t)(s * 2 + 1) * p + i];
        for (int q = 0; q < r; q++) {
          double acc = 0.0;
          for (int e = 0; e < r; e++) {
            const double C = T.coef[((size_t)(s * 3 + 0) * rr + q * r + e) * p + i];
            const double KM = T.coef[((size_t)(s * 3 + 1) * rr + q * r + e) * p + i];
            const double KP = T.coef[((size_t)(s * 3 + 2) * rr + q * r + e) * p + i];
            acc += C * x[(size_t)i * r + e];
            if (msg) acc -= KM * x[(size_t)sm * r + e] + KP * x[(size_t)sp * r + e];
          }
          y[(size_t)i * r + q] = acc;
        }
      }
      x.swap(y);
    }
    std::memcpy(xt, x.data(), (size_t)p * r * sizeof(double));
  }
  return CBS_OK;
}

// Closure tables of plan P (cbs_closure.cuh), uploaded to one device buffer.
static cbs_status setup_closure(cbs_plan* P, const cbs_desc* d) {
  ClosureTables C;
  bool singular = false;
  const LineArgs& a = P->args;
  const std::string msg = closure_build(C, P->n, P->r, P->dev.band, a.K, a.w, d->closure_rows, d->closure_width,
                                        d->closure, d->h, &singular);
  if (!msg.empty()) return fail(singular ? CBS_ERR_SINGULAR : CBS_ERR_INVALID_ARG, msg);
  const size_t ints = C.wrow.size() + C.urow.size();
  const size_t ioff = (ints * sizeof(int) + 15) / 16 * 16;
  const size_t dbl = C.Df.size() + C.Ey.size() + C.Minv.size() + C.Zt.size();
  std::vector<unsigned char> host(ioff + dbl * sizeof(double));
  int* ip = reinterpret_cast<int*>(host.data());
  std::copy(C.wrow.begin(), C.wrow.end(), ip);
  std::copy(C.urow.begin(), C.urow.end(), ip + C.wrow.size());
  double* dp = reinterpret_cast<double*>(host.data() + ioff);
  size_t o = 0;
  for (const std::vector<double>* v : {&C.Df, &C.Ey, &C.Minv, &C.Zt}) {
    std::copy(v->begin(), v->end(), dp + o);
    o += v->size();
  }
  cudaError_t e = cudaMalloc(&P->cbuf, host.size());
  if (e == cudaSuccess) e = cudaMemcpy(P->cbuf, host.data(), host.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "closure tables");
  ClosureArgs& c = P->cargs;
  std::memset(&c, 0, sizeof(c));
  c.lines = P->nlines;
  c.nx = d->dims[0];
  c.ny = d->dims[1];
  c.dir = d->direction;
  c.n = P->n;
  c.c2 = C.c2;
  c.nw = (int)C.wrow.size();
  c.nu = (int)C.urow.size();
  const int* di = static_cast<const int*>(P->cbuf);
  c.wrow = di;
  c.urow = di + C.wrow.size();
  const double* dd = reinterpret_cast<const double*>(static_cast<const unsigned char*>(P->cbuf) + ioff);
  c.Df = dd;
  c.Ey = dd + C.Df.size();
  c.Minv = dd + C.Df.size() + C.Ey.size();
  c.Zt = dd + C.Df.size() + C.Ey.size() + C.Minv.size();
  P->closure = true;
  return CBS_OK;
}

cbs_status cbs_plan_create(cbs_plan** out, const cbs_desc* d) {
  if (!out) return fail(CBS_ERR_INVALID_ARG, "null plan pointer");
  *out = nullptr;
  cbs_status st = validate(d);
  if (st) return st;
  cbs_plan* P = new (std::nothrow) cbs_plan();
  if (!P) return fail(CBS_ERR_NO_MEMORY, "host allocation failed");
  P->desc = *d;
  P->r = (d->bandwidth - 1) / 2;
  P->n = (int)d->dims[d->direction];
  if ((int64_t)P->n != d->dims[d->direction]) {
    delete P;
    return fail(CBS_ERR_INVALID_ARG, "line length too large");
  }
  P->nlines = d->dims[0] * d->dims[1] * d->dims[2] / P->n;
  P->var = d->lhs_kind == CBS_LHS_VARIABLE;
  const TuneChoice tuned = tuned_choice(d);
  int p = d->segments ? d->segments : tuned.segments;
  if (!d->segments && tuned.segments) {
    P->variant = tuned.variant;
    P->tile_lines = tuned.tile_lines;
  }
  if (p) {
    cbs_desc dd = *d;
    dd.segments = p;
    P->desc = dd;
    d = &P->desc;
  }
  if (!p) {
    if (P->var) {
      // registers hold ~5 arrays of rows per lane: keep partitions <= 8 rows
      p = 1;
      while (p < kMaxLanes && (P->n + p - 1) / p > 8) p *= 2;
      while (p > 1 && P->n / p < 2) p /= 2;
    } else {
      p = default_segments(P->n, P->r, d->precision);
    }
  }
  {
    const int maxM0 = (is_refine(d->precision) || P->var) ? 16 : 32;
    // a line whose partitions do not fit one lane's registers goes to the
    // segment-per-CTA path
    const bool use_long = !P->var && (d->segments > kMaxLanes || p < 1 || (P->n + p - 1) / p > maxM0);
    if (use_long && d->lhs_kind == CBS_LHS_BLOCK) {
      delete P;
      return fail(CBS_ERR_UNSUPPORTED, "block entries: on-chip lines only (at most 32 partitions of at most 32 rows)");
    }
    if (use_long) {
      st = create_long(P, d);
      if (st) {
        if (P->dbuf) cudaFree(P->dbuf);
        if (P->lbuf) cudaFree(P->lbuf);
        if (P->lbuf_small) cudaFree(P->lbuf_small);
        if (P->sbuf) cudaFree(P->sbuf);
        if (P->lwbuf) cudaFree(P->lwbuf);
        if (P->dstatus) cudaFree(P->dstatus);
        delete P;
        return st;
      }
      *out = P;
      return CBS_OK;
    }
  }
  if (p < 1) {
    delete P;
    return fail(CBS_ERR_UNSUPPORTED, "line too long for the on-chip kernel");
  }
  if (P->n < 2 * P->r * p) {
    delete P;
    return fail(CBS_ERR_INVALID_ARG, "need n >= 2 r p (every partition holds at least 2r rows)");
  }
  if (p > kMaxLanes) {
    delete P;
    return fail(CBS_ERR_UNSUPPORTED, "more than 32 partitions per line needs the long-line kernel");
  }
  const Bands A = desc_bands(d, P->r, P->var ? 0.25 : d->alpha);  // variable: geometry only
  bool singular = false;
  std::string msg;
  if (d->lhs_kind == CBS_LHS_BLOCK) {
    int sizes[3];
    if (!block_sizes(P->n, d->block_size, p, sizes)) {
      delete P;
      return fail(CBS_ERR_INVALID_ARG, "block entries: more partitions than points");
    }
    msg = build_line_tables_periodic(P->host, P->n, desc_block_bands(d), p, d->cyclic != 0, &singular, kMaxLanes,
                                     sizes);
  } else {
    msg = build_line_tables(P->host, P->n, A, p, d->cyclic != 0, &singular, kMaxLanes);
  }
  if (!msg.empty()) {
    delete P;
    return fail(singular ? CBS_ERR_SINGULAR : CBS_ERR_UNSUPPORTED, msg);
  }
  const LineTables& T = P->host;
  const int maxM = (is_refine(d->precision) || P->var) ? 16 : 32;
  int M = P->r == 3 ? 16 : 8;  // heptadiagonal bands are compiled for 16 and 32 rows per lane
  while (M < T.rows_big) M *= 2;
  if (M > maxM || T.nmax > kMaxBulk) {
    delete P;
    return fail(CBS_ERR_UNSUPPORTED, "partitions too long for the on-chip kernel (raise segments)");
  }
  P->M = M;
  P->ks = 0;
  if (d->rhs_kind != CBS_RHS_NONE) P->ks = d->rhs_terms <= 2 ? 2 : 3;

  // ---- device tables ----
  st = fill_dev_tables(P->dev, T, A, d, 0, &P->dbuf);
  if (st) {
    delete P;
    return st;
  }
  if (cudaMalloc(&P->dstatus, sizeof(int)) != cudaSuccess || cudaMemset(P->dstatus, 0, sizeof(int)) != cudaSuccess) {
    cudaFree(P->dbuf);
    if (P->dstatus) cudaFree(P->dstatus);
    delete P;
    return fail(CBS_ERR_CUDA, "status word allocation");
  }

  // ---- kernel arguments that do not change between solves ----
  LineArgs& a = P->args;
  std::memset(&a, 0, sizeof(a));
  a.nx = d->dims[0];
  a.ny = d->dims[1];
  a.nz = d->dims[2];
  a.nlines = P->nlines;
  a.dir = d->direction;
  a.K = (d->rhs_kind != CBS_RHS_NONE) ? d->rhs_terms : 0;
  a.sweeps = d->refine_sweeps;
  a.stag_shift = is_staggered(d) ? d->rhs_shift : 0;
  a.stag_sum = d->rhs_kind == CBS_RHS_MIDPOINT;
  for (int q = 0; q < kMaxRhsTerms; q++) {
    // term weights: c_q / (2 q h) (Eq. 1), c_q / ((2q - 1) h) (staggered
    // derivative), c_q / 2 (midpoint interpolation)
    const double den = d->rhs_kind == CBS_RHS_CENTRAL     ? 2.0 * (q + 1) * d->h
                       : d->rhs_kind == CBS_RHS_STAGGERED ? (2.0 * q + 1.0) * d->h
                                                          : 2.0;
    const double w = (q < a.K) ? d->rhs_coef[q] / den : 0.0;
    a.w[q] = w;
    a.wHi[q] = (float)w;
    a.wLo[q] = (float)(w - (double)a.wHi[q]);
  }
  pack_weights(a);
  a.status = P->dstatus;
  P->kind = 0;
  if (P->var) {
    VarArgs& v = P->vargs;
    std::memset(&v, 0, sizeof(v));
    v.alpha = d->bands;
    v.nx = a.nx;
    v.ny = a.ny;
    v.nz = a.nz;
    v.nlines = a.nlines;
    v.dir = a.dir;
    for (int q = 0; q < kMaxRhsTerms; q++) v.w[q] = a.w[q];
    for (int k = 0; k < (int)T.stages.size(); k++) {
      v.stage_type[k] = T.stages[k].type;
      v.stage_s[k] = T.stages[k].s;
      v.stage_na[k] = T.stages[k].na;
    }
    v.status = P->dstatus;
  }
  if (d->closure_rows > 0) {
    st = setup_closure(P, d);
    if (st) {
      cbs_plan_destroy(P);
      return st;
    }
  }
  P->desc.closure = nullptr;  // the caller's host arrays are not kept
  P->desc.blocks = nullptr;
  *out = P;
  return CBS_OK;
}

cbs_status cbs_plan_set_bands(cbs_plan* P, const void* bands) {
  if (!P || !bands) return fail(CBS_ERR_INVALID_ARG, "null argument");
  if (!P->var) return fail(CBS_ERR_INVALID_ARG, "plan has Toeplitz bands");
  P->desc.bands = bands;
  P->vargs.alpha = bands;
  return CBS_OK;
}

cbs_status cbs_plan_destroy(cbs_plan* P) {
  if (!P) return fail(CBS_ERR_INVALID_ARG, "null plan");
  cudaDeviceSynchronize();
  if (P->dbuf) cudaFree(P->dbuf);
  if (P->lbuf) cudaFree(P->lbuf);
  if (P->lbuf_small) cudaFree(P->lbuf_small);
  if (P->sbuf) cudaFree(P->sbuf);
  if (P->dstatus) cudaFree(P->dstatus);
  if (P->cbuf) cudaFree(P->cbuf);
  if (P->lwbuf) cudaFree(P->lwbuf);
  delete P;
  return CBS_OK;
}

cbs_status cbs_plan_info_get(const cbs_plan* P, cbs_plan_info* info) {
  if (!P || !info) return fail(CBS_ERR_INVALID_ARG, "null argument");
  std::memset(info, 0, sizeof(*info));
  info->n = P->n;
  info->bandwidth = P->desc.bandwidth;
  info->segments = P->host.p;
  info->rows_big = P->host.rows_big;
  info->rows_small = P->host.rows_small;
  info->count_big = P->host.count_big;
  info->pcr_steps = P->host.pcr_steps;
  info->detach_steps = P->host.detach_steps;
  info->detached_rows = P->host.detached_rows;
  info->stage_count = (int32_t)P->host.stages.size();
  info->kernel = P->kind;
  info->threads_per_line = P->kind == 1 ? P->inner_threads : P->dev.pw;
  info->segment_warp = P->kind == 1 && P->long_warp && P->variant == 0;
  info->lines = P->nlines;
  auto count = [](const LineTables& T, int bit) {
    int c = 0;
    for (int m : T.stage_msg) c += (m & bit) ? 1 : 0;
    return c;
  };
  info->message_stages = count(P->host, 1);
  info->message_stages_f32 = count(P->host, 2);
  if (P->kind == 1) {
    info->inner_message_stages = count(P->inner, 1);
    info->inner_message_stages_f32 = count(P->inner, 2);
  }
  info->variant = P->variant;
  info->tile_lines = P->tile_lines;
  if (P->kind == 0 && !P->var) {
    static const double aligned[2] = {0.0, 0.0};  // any 16-byte aligned address stands in for the arrays
    LineArgs a = P->args;
    void* al = reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(aligned) + 15) & ~(uintptr_t)15);
    a.in = al;
    a.out = al;
    info->tma = tma_eligible(mode_of(P->desc.precision), P->ks, is_staggered(&P->desc),
                             P->desc.in_dtype == CBS_DTYPE_F64, P->desc.out_dtype == CBS_DTYPE_F64, a, P->dev)
                    ? 1 : 0;
  }
  return CBS_OK;
}

cbs_status cbs_plan_inject_fault(cbs_plan* P, int32_t kind) {
  if (!P) return fail(CBS_ERR_INVALID_ARG, "null plan");
  if (kind != 0 && kind != 1) return fail(CBS_ERR_INVALID_ARG, "fault kind must be 0 or 1");
  P->fault = kind;
  return CBS_OK;
}

cbs_status cbs_plan_set_variant(cbs_plan* P, int32_t variant, int32_t tile_lines) {
  if (!P) return fail(CBS_ERR_INVALID_ARG, "null plan");
  if (variant != 0 && variant != 1) return fail(CBS_ERR_INVALID_ARG, "variant must be 0 or 1");
  if (tile_lines != 0 && tile_lines != 4 && tile_lines != 8 && tile_lines != 16 && tile_lines != 32)
    return fail(CBS_ERR_INVALID_ARG, "tile_lines must be 0, 4, 8, 16 or 32");
  P->variant = variant;
  P->tile_lines = tile_lines;
  return CBS_OK;
}

cbs_status cbs_solve(cbs_plan* P, const void* in, void* out, void* stream) {
  g_launches = 0;
  if (!P || !in || !out) return fail(CBS_ERR_INVALID_ARG, "null argument");
  if (in == out) return fail(CBS_ERR_INVALID_ARG, "out must not alias in");
  const cbs_desc& d = P->desc;
  if (P->var) {
    VarArgs v = P->vargs;
    v.f = in;
    v.out = out;
    v.alpha = d.bands;
    cudaError_t e = launch_var(P->M, P->ks, false, d.precision == CBS_FP64, v, P->dev, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "variable-band kernel launch");
    g_launches = 1;
    return CBS_OK;
  }
  const int mode = mode_of(d.precision);
  if (P->kind == 1) {
    LongArgs la = P->largs;
    la.in = in;
    la.out = out;
    int launches = 0;
    cudaError_t e =
        P->long_warp && P->variant == 0
            ? launch_long_warp(mode, P->r, d.in_dtype == CBS_DTYPE_F64, d.out_dtype == CBS_DTYPE_F64, la, P->dev_inner,
                               la.cbig < la.p ? &P->dev_inner_small : nullptr, P->lwargs, P->lwifc,
                               (cudaStream_t)stream, &launches)
            : launch_long(mode, P->r, d.in_dtype == CBS_DTYPE_F64, d.out_dtype == CBS_DTYPE_F64, la, P->lgeom, P->dev,
                          P->dev_inner, la.cbig < la.p ? &P->dev_inner_small : nullptr, P->inner_full,
                          (cudaStream_t)stream, &launches);
    if (e != cudaSuccess) return cuda_fail(e, "long-line kernel launch");
    g_launches = launches;
    return CBS_OK;
  }
  LineArgs a = P->args;
  a.in = in;
  a.out = out;
  const cudaError_t e =
      launch_line_plan(P, a, P->ks, is_staggered(&d), d.in_dtype, d.out_dtype, (cudaStream_t)stream);
  if (e == cudaErrorNotSupported) return fail(CBS_ERR_UNSUPPORTED, "no kernel variant for these element types");
  if (e != cudaSuccess) return cuda_fail(e, "line kernel launch");
  g_launches = 1;
  if (P->closure) {  // boundary rows: the Woodbury correction on the rows near both ends
    ClosureArgs c = P->cargs;
    c.f = in;
    c.x = out;
    const cudaError_t ec =
        launch_closure(c, d.in_dtype == CBS_DTYPE_F64, d.out_dtype == CBS_DTYPE_F64, (cudaStream_t)stream);
    if (ec != cudaSuccess) return cuda_fail(ec, "closure kernel launch");
    g_launches = 2;
  }
  return CBS_OK;
}

cbs_status cbs_solve_transpose(cbs_plan* P, const void* g, const void* x, void* lambda, void* grad_in,
                               void* grad_bands, void* stream) {
  g_launches = 0;
  if (!P || !g) return fail(CBS_ERR_INVALID_ARG, "null argument");
  const cbs_desc& d = P->desc;
  cudaStream_t s = (cudaStream_t)stream;
  if (P->var) {
    if (!lambda && !grad_in && !(x && grad_bands)) return CBS_OK;
    VarArgs v = P->vargs;
    v.f = g;
    v.alpha = d.bands;
    v.x = (x && grad_bands) ? x : nullptr;
    v.grad_alpha = (x && grad_bands) ? grad_bands : nullptr;
    v.lam = lambda;
    v.out = (P->ks > 0) ? grad_in : nullptr;
    cudaError_t e = launch_var(P->M, P->ks, true, d.precision == CBS_FP64, v, P->dev, s);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint kernel launch");
    g_launches = 1;
    return CBS_OK;
  }
  if (P->kind != 0) return fail(CBS_ERR_UNSUPPORTED, "transpose solve of long-line plans");
  if (d.lhs_kind == CBS_LHS_BLOCK) return fail(CBS_ERR_UNSUPPORTED, "transpose solve of block-entry plans");
  // Toeplitz: A is symmetric, and on a periodic grid A^{-1} and the stencil S
  // are both circulant, so S^T A^{-T} g = A^{-1} (S^T g), with S^T = -S for the
  // central stencil: the same line kernel with transposed stencil weights.
  if (d.in_dtype != d.out_dtype) return fail(CBS_ERR_UNSUPPORTED, "transpose needs in_dtype == out_dtype");
  if (!d.cyclic) return fail(CBS_ERR_UNSUPPORTED, "transpose of acyclic plans");
  if (grad_bands) return fail(CBS_ERR_INVALID_ARG, "Toeplitz plans have no band field");
  int launches = 0;
  auto run = [&](const LineArgs& a, int ks) -> cudaError_t {
    return launch_line_plan(P, a, ks, ks > 0 && is_staggered(&d), d.out_dtype, d.in_dtype, s);
  };
  if (lambda) {
    LineArgs a = P->args;
    a.in = g;
    a.out = lambda;
    a.K = 0;
    cudaError_t e = run(a, 0);
    if (e != cudaSuccess) return cuda_fail(e, "transpose solve launch");
    launches++;
  }
  if (grad_in && P->ks > 0) {
    LineArgs a = P->args;
    a.in = g;
    a.out = grad_in;
    // staggered stencils: S^T is the stencil of the other shift (the input
    // and output grids swap), negated for the derivative, as is the central one
    if (is_staggered(&d)) a.stag_shift = 1 - a.stag_shift;
    if (d.rhs_kind != CBS_RHS_MIDPOINT) {
      for (int q = 0; q < kMaxRhsTerms; q++) {
        a.w[q] = -a.w[q];
        a.wHi[q] = -a.wHi[q];
        a.wLo[q] = -a.wLo[q];
      }
    }
    pack_weights(a);
    cudaError_t e = run(a, P->ks);
    if (e != cudaSuccess) return cuda_fail(e, "transpose solve launch");
    launches++;
  } else if (grad_in) {
    return fail(CBS_ERR_INVALID_ARG, "grad_in needs a plan with a stencil (use lambda)");
  }
  g_launches = launches;
  return CBS_OK;
}

cbs_status cbs_band_grad(cbs_plan* P, const void* lambda, const void* x, void* grad_bands, void* stream) {
  g_launches = 0;
  if (!P || !lambda || !x || !grad_bands) return fail(CBS_ERR_INVALID_ARG, "null argument");
  if (P->desc.lhs_kind == CBS_LHS_BLOCK) return fail(CBS_ERR_UNSUPPORTED, "band gradient of block-entry plans");
  const cbs_desc& d = P->desc;
  cudaError_t e = launch_band_grad(d.in_dtype == CBS_DTYPE_F64, lambda, x, grad_bands, d.dims[0], d.dims[1],
                                   d.dims[2], d.direction, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "band gradient launch");
  g_launches = 1;
  return CBS_OK;
}

cbs_status cbs_status_poll(cbs_plan* P, int32_t* device_status) {
  if (!P || !device_status) return fail(CBS_ERR_INVALID_ARG, "null argument");
  int v = 0;
  cudaError_t e = cudaMemcpy(&v, P->dstatus, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "reading the status word");
  e = cudaMemset(P->dstatus, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "clearing the status word");
  *device_status = v;
  return CBS_OK;
}

cbs_status cbs_batch_create(cbs_batch** out, const cbs_desc* descs, int32_t count) {
  if (!out || !descs) return fail(CBS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (count < 1 || count > kBatchMax) return fail(CBS_ERR_INVALID_ARG, "batch count must be 1..256");
  cbs_batch* B = new (std::nothrow) cbs_batch();
  if (!B) return fail(CBS_ERR_NO_MEMORY, "host allocation failed");
  const size_t pb = batch_problem_bytes();
  std::vector<unsigned char> probs;  // one entry per on-chip problem, one per segment size of a long line
  int nent = 0;
  std::vector<int4> items;
  std::vector<double> cost;
  // every problem gets its plan (any problem a plan takes can be batched);
  // the persistent launch takes the kinds below, and a batch holding any
  // other problem runs per problem
  auto not_persistent = [&](int k, const char* why) {
    if (B->persistent) B->why = "batch problem " + std::to_string(k) + ": " + why;
    B->persistent = false;
  };
  for (int k = 0; k < count; k++) {
    const cbs_desc& d = descs[k];
    cbs_plan* P = nullptr;
    cbs_status st = cbs_plan_create(&P, &d);
    if (st) {
      const std::string msg = "batch problem " + std::to_string(k) + ": " + g_err;
      cbs_batch_destroy(B);
      return fail(st, msg);
    }
    B->plans.push_back(P);
    B->unknowns += d.dims[0] * d.dims[1] * d.dims[2];
    const bool f32 = d.precision == CBS_FP32 && d.in_dtype == CBS_DTYPE_F32 && d.out_dtype == CBS_DTYPE_F32;
    const bool f64io = d.in_dtype == CBS_DTYPE_F64 && d.out_dtype == CBS_DTYPE_F64 &&
                       (d.precision == CBS_FP64 || d.precision == CBS_FP32_REFINE);
    if (d.lhs_kind != CBS_LHS_TOEPLITZ || !(f32 || f64io) || is_staggered(&d) || d.closure_rows || d.bandwidth > 5) {
      not_persistent(k, "the persistent launch takes Toeplitz bands of width 3 or 5; FP64 or FP32_REFINE with "
                        "FP64 in/out, or FP32 with FP32 in/out; no staggered stencil or closures");
      continue;
    }
    const int mode = d.precision == CBS_FP64 ? kModeF64 : d.precision == CBS_FP32 ? kModeF32 : kModeRefine;
    if (P->kind != 0) {
      // long lines: the x-lines of a warp-per-segment plan, an entry per
      // segment size, an item per (chunk of kLongWarps segments, line)
      if (!(P->long_warp && P->variant == 0) || P->lgeom.dir != 0 || batch_long_variant_host(P->r, mode) < 0) {
        not_persistent(k, "the persistent launch takes long lines as x-lines of a warp per segment (segments of "
                          "32 x 16 + r rows, decoupled interface system)");
        continue;
      }
      const LongArgs& la = P->largs;
      for (int part = 0; part < 2; part++) {
        LongWarpArgs wa = P->lwargs;
        wa.ifc = P->lwifc[part];
        wa.seg0 = part == 0 ? 0 : la.cbig;
        wa.nseg = part == 0 ? la.cbig : la.p - la.cbig;
        if (wa.nseg <= 0) continue;
        wa.nchunks = (wa.nseg + kLongWarps - 1) / kLongWarps;
        probs.resize(pb * (nent + 1));
        batch_fill_long(probs.data() + pb * nent, la, part == 0 ? P->dev_inner : P->dev_inner_small, wa, P->r, mode,
                        k);
        B->smem = std::max(B->smem, batch_long_bytes(P->r, la.K));
        const double c = (double)kLongWarps * la.m * (mode == kModeRefine ? 2.0 : 1.0);
        for (int64_t line = 0; line < la.lines; line++)
          for (int ch = 0; ch < wa.nchunks; ch++) {
            items.push_back(make_int4(nent, ch, (int)line, 0));
            cost.push_back(c);
          }
        nent++;
      }
      continue;
    }
    const bool full = P->dev.count_big == P->dev.p && P->dev.rows_big == 16 && P->M == 16;
    int variant = -1;
    if (mode == kModeF32) {
      variant = batch_f32_variant_host(P->r, P->ks, P->M);
    } else {
      variant = full ? batch_variant_host(P->r, P->ks, P->M, mode, true) : -1;
      if (variant < 0) variant = batch_variant_host(P->r, P->ks, P->M, mode, false);
    }
    if (variant < 0) {
      not_persistent(k, "tile variant of the persistent launch not compiled");
      continue;
    }
    probs.resize(pb * (nent + 1));
    batch_fill_problem(probs.data() + pb * nent, P->args, P->dev, variant, k);
    const int TL = kLineThreads / P->dev.pw;
    B->smem = std::max(B->smem, (size_t)TL * P->dev.lsz * sizeof(double));
    const dim3 g = tile_grid(d.dims[0], d.dims[1], d.dims[2], P->nlines, d.direction, TL);
    const double c = (double)TL * P->n * (mode == kModeRefine ? 2.0 : 1.0);
    for (unsigned ty = 0; ty < g.y; ty++)
      for (unsigned tx = 0; tx < g.x; tx++) {
        items.push_back(make_int4(nent, (int)tx, (int)ty, 0));
        cost.push_back(c);
      }
    nent++;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    cbs_batch_destroy(B);
    return cuda_fail(e, "batch setup");
  }
  const int grid = (int)std::min<size_t>(items.size(), 2 * (size_t)sms);
  // most expensive tiles first, so the static stride (CTA b takes positions
  // b, b + grid, ...) ends with small tiles; FP64 and other tiles stay mixed
  // on every SM (FP64 tiles on CTAs of their own measured 6.38 against 4.54
  // ms on the 48-grid batch: the FP64 pipe then idles on half of the SMs)
  std::vector<size_t> order(items.size());
  for (size_t q = 0; q < order.size(); q++) order[q] = q;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
  std::vector<int4> sorted(items.size());
  for (size_t q = 0; q < order.size(); q++) sorted[q] = items[order[q]];
  B->nitems = (int)sorted.size();
  B->count = count;
  B->smem = batch_smem(B->smem);  // + the current problem's tables
  if (B->persistent) {  // the work table of the persistent launch
    e = batch_configure(B->smem);
    if (e == cudaSuccess) e = cudaMalloc(&B->dprobs, probs.size());
    if (e == cudaSuccess) e = cudaMalloc(&B->ditems, sorted.size() * sizeof(int4));
    if (e == cudaSuccess) e = cudaMemcpy(B->dprobs, probs.data(), probs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(B->ditems, sorted.data(), sorted.size() * sizeof(int4), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    cbs_batch_destroy(B);
    return cuda_fail(e, "batch setup");
  }
  B->grid = grid;
  B->device = dev;
  // per-problem launches: FP64 problems (bound by the FP64 pipe) on a stream
  // of their own, beside the others, each list largest first
  std::vector<int> byk(count);
  for (int k = 0; k < count; k++) byk[k] = k;
  auto size_of = [&](int k) { return descs[k].dims[0] * descs[k].dims[1] * descs[k].dims[2]; };
  std::stable_sort(byk.begin(), byk.end(), [&](int a, int b) { return size_of(a) > size_of(b); });
  for (int k : byk) (descs[k].precision == CBS_FP64 ? B->order_fp64 : B->order_other).push_back(k);
  e = cudaStreamCreateWithFlags(&B->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->join, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cbs_batch_destroy(B);
    return cuda_fail(e, "batch setup");
  }
  *out = B;
  return CBS_OK;
}

cbs_status cbs_batch_destroy(cbs_batch* B) {
  if (!B) return fail(CBS_ERR_INVALID_ARG, "null batch");
  if (B->side) cudaStreamSynchronize(B->side);
  for (cbs_plan* P : B->plans) cbs_plan_destroy(P);
  if (B->dprobs) cudaFree(B->dprobs);
  if (B->ditems) cudaFree(B->ditems);
  if (B->fork) cudaEventDestroy(B->fork);
  if (B->join) cudaEventDestroy(B->join);
  if (B->side) cudaStreamDestroy(B->side);
  delete B;
  return CBS_OK;
}

cbs_status cbs_batch_set_mode(cbs_batch* B, int32_t mode) {
  if (!B) return fail(CBS_ERR_INVALID_ARG, "null batch");
  if (mode < CBS_BATCH_AUTO || mode > CBS_BATCH_PER_PROBLEM) return fail(CBS_ERR_INVALID_ARG, "batch mode must be 0, 1 or 2");
  if (mode == CBS_BATCH_PERSISTENT && !B->persistent) return fail(CBS_ERR_UNSUPPORTED, B->why);
  B->mode = mode;
  return CBS_OK;
}

// Per-problem launches: every problem's own plan (the kernels cbs_solve runs
// for it).  The FP64 problems go to the batch's side stream, forked from the
// caller's stream by an event and joined back into it by another, so they
// share the SMs with the FP32-pipe work of the others (48-grid ragged batch:
// 3.60 ms against 3.99 ms on one stream and 4.52 ms for the persistent
// launch).  Only stream-ordered calls: capturable like a single launch.
static cbs_status batch_solve_per_problem(cbs_batch* B, const void* const* ins, void* const* outs, cudaStream_t s) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != B->device)
    return fail(CBS_ERR_INVALID_ARG, "batch: solve with the device it was created on current");
  int launches = 0;
  const bool fork = !B->order_fp64.empty() && !B->order_other.empty();
  cudaError_t e = cudaSuccess;
  if (fork) {
    e = cudaEventRecord(B->fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(B->side, B->fork, 0);
    if (e != cudaSuccess) return cuda_fail(e, "batch fork");
  }
  cbs_status r = CBS_OK;
  std::string msg;
  for (int pass = 0; pass < 2 && !r; pass++) {
    const std::vector<int>& ks = pass == 0 ? B->order_fp64 : B->order_other;
    const cudaStream_t st = (pass == 0 && fork) ? B->side : s;
    for (size_t q = 0; q < ks.size() && !r; q++) {
      r = cbs_solve(B->plans[ks[q]], ins[ks[q]], outs[ks[q]], st);
      if (r) msg = "batch problem " + std::to_string(ks[q]) + ": " + g_err;
      launches += g_launches;
    }
  }
  if (fork) {  // joined also after a failed launch, so the caller's stream never leaves work behind
    e = cudaEventRecord(B->join, B->side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, B->join, 0);
  }
  if (r) return fail(r, msg);
  if (e != cudaSuccess) return cuda_fail(e, "batch join");
  g_launches = launches;
  return CBS_OK;
}

cbs_status cbs_batch_solve(cbs_batch* B, const void* const* ins, void* const* outs, void* stream) {
  g_launches = 0;
  if (!B || !ins || !outs) return fail(CBS_ERR_INVALID_ARG, "null argument");
  for (int k = 0; k < B->count; k++)
    if (!ins[k] || !outs[k] || ins[k] == outs[k]) return fail(CBS_ERR_INVALID_ARG, "bad pointer for problem " + std::to_string(k));
  const bool per_problem = !B->persistent || B->mode == CBS_BATCH_PER_PROBLEM ||
                           (B->mode == CBS_BATCH_AUTO && B->unknowns >= (int64_t)B->count * kBatchPerProblemUnknowns);
  if (per_problem) return batch_solve_per_problem(B, ins, outs, (cudaStream_t)stream);
  cudaError_t e = batch_launch((const BatchProblem*)B->dprobs, (const int4*)B->ditems, B->nitems, ins, outs, B->count,
                               B->grid, B->smem, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch kernel launch");
  g_launches = 1;
  return CBS_OK;
}

cbs_status cbs_batch_status_poll(cbs_batch* B, int32_t* st) {
  if (!B || !st) return fail(CBS_ERR_INVALID_ARG, "null argument");
  *st = CBS_OK;
  for (cbs_plan* P : B->plans) {  // each problem's kernels report to its plan's status word
    int32_t v = CBS_OK;
    const cbs_status r = cbs_status_poll(P, &v);
    if (r) return r;
    if (v && !*st) *st = v;
  }
  return CBS_OK;
}

cbs_status cbs_autotune(const cbs_desc* d, int32_t reps, int32_t* best_segments, double* best_ms) {
  cbs_status st = validate(d);
  if (st) return st;
  if (reps < 1) reps = 1;
  const int n = (int)d->dims[d->direction], r = (d->bandwidth - 1) / 2;
  // candidates
  std::vector<int> cand;
  for (int p = 1; p <= kMaxLanes; p++)
    if (n >= 2 * r * p) cand.push_back(p);
  for (int p = kMaxLanes + 1; p <= n / 64 && (int)cand.size() < 256; p++)
    if ((n % p == 0 || (n - p * r) % 16 == 0) && n / p <= 8192 + r) cand.push_back(p);
  const int64_t elems = d->dims[0] * d->dims[1] * d->dims[2];
  const size_t isz = d->in_dtype == CBS_DTYPE_F64 ? 8 : 4, osz = d->out_dtype == CBS_DTYPE_F64 ? 8 : 4;
  void *in = nullptr, *out = nullptr, *bands = nullptr;
  cudaError_t e = cudaMalloc(&in, elems * isz);
  if (e == cudaSuccess) e = cudaMalloc(&out, elems * osz);
  if (e == cudaSuccess && d->lhs_kind == CBS_LHS_VARIABLE) e = cudaMalloc(&bands, elems * isz);
  // inputs: varying values in [-1, 1); variable bands in [0.1, 0.4)
  // (diagonally dominant), as the kernels' fast paths see real data
  if (e == cudaSuccess) e = tune_fill(in, elems, d->in_dtype == CBS_DTYPE_F64, -1.0, 2.0);
  if (e == cudaSuccess && bands) e = tune_fill(bands, elems, d->in_dtype == CBS_DTYPE_F64, 0.1, 0.3);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaFree(in); cudaFree(out); cudaFree(bands);
    if (e0) cudaEventDestroy(e0);
    return cuda_fail(e, "autotune buffers");
  }
  TuneChoice best;
  double bms = 1e300;
  for (int p : cand) {
    cbs_desc dd = *d;
    dd.segments = p;
    if (bands) dd.bands = bands;
    cbs_plan* P = nullptr;
    if (cbs_plan_create(&P, &dd) != CBS_OK) continue;  // not admissible for this kernel
    cbs_plan_info info;
    cbs_plan_info_get(P, &info);
    // (variant, tile shape) pairs: the line kernels, and for plans the TMA
    // kernel takes, its tile shapes for the direction
    std::vector<std::pair<int, int>> kinds = {{0, 0}};
    if (info.tma) {
      kinds = {{1, 0}, {0, 4}, {0, 8}};
      if (d->direction != 0) {
        kinds.push_back({0, 16});
        kinds.push_back({0, 32});
      }
    }
    for (const auto& kind : kinds) {
      P->variant = kind.first;
      P->tile_lines = kind.second;
      bool ok = true;
      for (int w = 0; w < 2 && ok; w++) ok = cbs_solve(P, in, out, nullptr) == CBS_OK;
      float ms = 0.f;
      if (ok) {
        cudaEventRecord(e0, nullptr);
        for (int k = 0; k < reps && ok; k++) ok = cbs_solve(P, in, out, nullptr) == CBS_OK;
        cudaEventRecord(e1, nullptr);
        ok = ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
      }
      if (ok && ms / reps < bms) {
        bms = ms / reps;
        best.segments = p;
        best.variant = kind.first;
        best.tile_lines = kind.second;
      }
    }
    cbs_plan_destroy(P);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(in);
  cudaFree(out);
  if (bands) cudaFree(bands);
  if (!best.segments) return fail(CBS_ERR_UNSUPPORTED, "no admissible partition count for this descriptor");
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[tune_key(d)] = best;
  }
  if (best_segments) *best_segments = best.segments;
  if (best_ms) *best_ms = bms;
  return CBS_OK;
}

}  // extern "C"
