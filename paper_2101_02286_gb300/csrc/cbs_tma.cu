// cbs_tma.cu -- host side of the TMA-fed refinement line kernel
// (cbs_tma.cuh): eligibility, the tensor-map encoder, the interface tables
// and the dispatch over rows per partition and interface precision.
#include <cmath>

#include "cbs_tma_launch.cuh"

namespace cbs {

namespace {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// dependency on libcuda); looked up once per process.
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

bool tma_encode_impl(CUtensorMap* map, const void* ptr, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
            const cuuint32_t* box, CUtensorMapSwizzle sw) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, (cuuint32_t)rank, const_cast<void*>(ptr), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool tma_encode(CUtensorMap* map, const void* ptr, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
                const cuuint32_t* box, CUtensorMapSwizzle sw) {
  return tma_encode_impl(map, ptr, rank, dims, strides, box, sw);
}

// Interface stages of a uniform 32-partition plan for the kernel: the stages
// whose couplings exceed rounding in the interface precision (bit 0 of
// stage_msg: FP64, bit 1: FP32), in order, and the product of the scalings
// of all the others.  False when the plan is not uniform or has more
// message stages than the kernel unrolls.
bool make_iface(const DevLineTables& D, bool fp64, TmaIface& f) {
  f = TmaIface{};
  if (!D.uniform || D.r != 1) return false;
  double scale = 1.0;
  for (int st = 0; st < D.nstage && st < kMaxStages; st++) {
    const double C = D.ucoef[st][0], KM = D.ucoef[st][1], KP = D.ucoef[st][2];
    if (D.stage_msg[st] & (fp64 ? 1 : 2)) {
      if (f.nmsg == kTmaMaxMsg) return false;
      const int k = f.nmsg++;
      f.s[k] = D.ustage_s[st];
      f.cd[k][0] = C;
      f.cd[k][1] = KM;
      f.cd[k][2] = KP;
      f.cf[k][0] = D.ucoefF[st][0];
      f.cf[k][1] = D.ucoefF[st][1];
      f.cf[k][2] = D.ucoefF[st][2];
    } else if (D.stage_has_c[st]) {
      scale *= C;
    }
  }
  // the scaling commutes with the message stages: fold it into the last one
  if (f.nmsg > 0) {
    const int k = f.nmsg - 1;
    for (int m = 0; m < 3; m++) {
      f.cd[k][m] *= scale;
      f.cf[k][m] = (float)((double)f.cf[k][m] * scale);
    }
    scale = 1.0;
  }
  f.scaled = scale;
  f.scalef = (float)scale;
  f.wait_ns = 1000000000ull;  // 1 s
  f.fault = 0;
  return true;
}

bool tma_integer_bands(const LineArgs& a, const DevLineTables& t, LineArgs& a2, DevLineTables& t2, TmaIface& f) {
  f.ib = 0;
  f.dband = 1.f;
  f.invdf = 1.f;
  f.invdd = 1.0;
  const double alpha = t.band[0];
  // a stencil is needed to form D b exactly (the weights take D)
  if (a.K < 1 || !(alpha > 0.0) || t.band[1] != 1.0 || t.band[2] != alpha) return false;
  const double D = std::nearbyint(1.0 / alpha);
  if (D < 2.0 || D > 6.0 || std::fabs(alpha * D - 1.0) > std::ldexp(1.0, -48)) return false;
  a2 = a;
  for (int q = 0; q < kMaxRhsTerms; q++) {  // stencil weights of D b
    const double w = a.w[q] * D;
    a2.w[q] = w;
    a2.wHi[q] = (float)w;
    a2.wLo[q] = (float)(w - (double)a2.wHi[q]);
  }
  pack_weights(a2);
  t2 = t;
  for (int j = 0; j < kMaxBulk; j++) {  // bulk pivot reciprocals of A' = D A: y' = y / D
    t2.fac[j * 3 + 1] = t.fac[j * 3 + 1] / D;
    t2.facF[j * 3 + 1] = (float)t2.fac[j * 3 + 1];
  }
  // b-hat' = b~' - D L~ y'_{i-1} - D U~ y'_i = D b-hat: the interface then
  // returns D x~, undone by the final scaling (or the last message stage)
  t2.Lt[0][0] = t.Lt[0][0] * D;
  t2.Ut[0][0] = t.Ut[0][0] * D;
  t2.LtF[0][0] = (float)t2.Lt[0][0];
  t2.UtF[0][0] = (float)t2.Ut[0][0];
  if (f.nmsg > 0) {
    for (int m = 0; m < 3; m++) {
      f.cd[f.nmsg - 1][m] /= D;
      f.cf[f.nmsg - 1][m] = (float)f.cd[f.nmsg - 1][m];
    }
  } else {
    f.scaled /= D;
    f.scalef = (float)f.scaled;
  }
  f.ib = 1;
  f.dband = (float)D;
  f.invdd = 1.0 / D;
  f.invdf = (float)f.invdd;
  return true;
}

// The TMA kernel takes: FP32 + refinement with one sweep, cyclic symmetric
// tridiagonal Toeplitz bands (unit diagonal), 32 whole partitions of 8 or 16
// rows per line (n = 256 or 512), the central stencil of at most two terms
// or none, FP64 in and out on 16-byte boundaries, and for y/z lines an even
// nx (the tensor map's strides are multiples of 16 bytes).
bool tma_eligible(int mode, int KS, bool staggered, bool in64, bool out64, const LineArgs& a, const DevLineTables& t) {
  if (!refine_mode(mode) || a.sweeps != 1 || staggered || !in64 || !out64) return false;
  if (t.r != 1 || !t.cyclic || !t.uniform || t.p != 32 || t.pw != 32 || t.count_big != 32) return false;
  TmaIface f;
  if (!make_iface(t, mode == kModeRefineI64, f)) return false;
  if (t.rows_big != 8 && t.rows_big != 16) return false;
  if (KS != 0 && KS != 2) return false;
  if (KS == 2 && a.K > 2) return false;
  if ((reinterpret_cast<uintptr_t>(a.in) & 15u) || (reinterpret_cast<uintptr_t>(a.out) & 15u)) return false;
  if (a.dir != 0 && (a.nx & 1)) return false;
  return true;
}

// cudaErrorNotSupported: the driver refused a tensor map (the caller then
// runs the pipelined line kernel instead).
cudaError_t launch_tma(int mode, int KS, const LineArgs& a, const DevLineTables& t, int tile_lines, int fault,
                       cudaStream_t s) {
  if (mode == kModeRefineI64)
    return t.rows_big == 16 ? launch_tma_m<16, double>(KS, a, t, tile_lines, fault, s)
                            : launch_tma_m<8, double>(KS, a, t, tile_lines, fault, s);
  return t.rows_big == 16 ? launch_tma_m<16, float>(KS, a, t, tile_lines, fault, s)
                          : launch_tma_m<8, float>(KS, a, t, tile_lines, fault, s);
}

}  // namespace cbs
