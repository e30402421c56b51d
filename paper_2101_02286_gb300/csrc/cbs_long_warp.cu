// cbs_long_warp.cu -- launch of the warp-per-segment long-line item
// (cbs_long_warp.cuh): one CTA per chunk of kLongWarps segments of a line.
#include "cbs_long_warp.cuh"

namespace cbs {

template <int R, int MODE, typename TIn, typename TOut, bool SW1, bool YZ>
__global__ void __launch_bounds__(kLongWarps * 32, long_ctas_per_sm(SW1 || !refine_mode(MODE)))
    long_warp_kernel(const LongArgs a, const DevLineTables tin, const LongWarpArgs wa) {
  extern __shared__ __align__(16) unsigned char smem[];
  if constexpr (YZ)  // groups fastest: CTAs in flight read the same rows (z-planes) of adjacent groups
    long_warp_item_yz<R, MODE, TIn, TOut, SW1>(a, tin, wa, wa.seg0 + (int)(blockIdx.x / (unsigned)wa.ngroups),
                                               (int64_t)(blockIdx.x % (unsigned)wa.ngroups) * kLongWarps, smem);
  else
    long_warp_item<R, MODE, TIn, TOut, SW1>(a, tin, wa, (int)(blockIdx.x % (unsigned)wa.nchunks),
                                            (int64_t)(blockIdx.x / (unsigned)wa.nchunks), smem);
}

// The launch of one segment size.
template <int R, int MODE, typename TIn, typename TOut>
cudaError_t launch_long_warp_t(const LongArgs& a, const DevLineTables& tin, const LongWarpArgs& wa, cudaStream_t s) {
  const bool yz = wa.gm.dir != 0;
  const size_t smem = yz ? lwyz_bytes<R>(a.K, (int)sizeof(TIn)) : lw_bytes<R>(a.K, (int)sizeof(TIn));
  if (a.K > 16 * 31 || smem > 48 * 1024) return cudaErrorInvalidValue;  // no opt-in above 48 KB
  const bool sw1 = refine_mode(MODE) && a.sweeps == 1;
  auto kern = yz ? (sw1 ? long_warp_kernel<R, MODE, TIn, TOut, refine_mode(MODE), true>
                        : long_warp_kernel<R, MODE, TIn, TOut, false, true>)
                 : (sw1 ? long_warp_kernel<R, MODE, TIn, TOut, refine_mode(MODE), false>
                        : long_warp_kernel<R, MODE, TIn, TOut, false, false>);
  const int64_t blocks = yz ? (int64_t)wa.ngroups * wa.nseg : a.lines * wa.nchunks;
  if (blocks > 0x7fffffff || blocks < 1) return cudaErrorInvalidValue;
  kern<<<(unsigned)blocks, kLongWarps * 32, smem, s>>>(a, tin, wa);
  return cudaGetLastError();
}

// Whether the shared memory of one CTA stays within 48 KB (no opt-in).
bool long_warp_fits(int R, int K, int in_size, bool yz) {
  if (K < 1 || K > 16 * 31) return false;
  const size_t b = yz ? (R == 1 ? lwyz_bytes<1>(K, in_size) : lwyz_bytes<2>(K, in_size))
                      : (R == 1 ? lw_bytes<1>(K, in_size) : lw_bytes<2>(K, in_size));
  return b <= 48 * 1024;
}

// Element types per mode: FP64 in and out for every mode; FP32 in and out
// for the FP32 mode; FP32 in, FP64 out for the others.
template <int R, int MODE>
cudaError_t launch_long_warp_types(bool in64, bool out64, const LongArgs& a, const DevLineTables& t,
                                   const LongWarpArgs& wa, cudaStream_t s) {
  if (in64 && out64) return launch_long_warp_t<R, MODE, double, double>(a, t, wa, s);
  if constexpr (MODE == kModeF32) {
    if (!in64 && !out64) return launch_long_warp_t<R, MODE, float, float>(a, t, wa, s);
  } else {
    if (!in64 && out64) return launch_long_warp_t<R, MODE, float, double>(a, t, wa, s);
  }
  return cudaErrorNotSupported;
}

template <int R>
cudaError_t launch_long_warp_r(int mode, bool in64, bool out64, const LongArgs& a, const DevLineTables& t,
                               const LongWarpArgs& wa, cudaStream_t s) {
  switch (mode) {
    case kModeRefine: return launch_long_warp_types<R, kModeRefine>(in64, out64, a, t, wa, s);
    case kModeRefineI64: return launch_long_warp_types<R, kModeRefineI64>(in64, out64, a, t, wa, s);
    case kModeF64: return launch_long_warp_types<R, kModeF64>(in64, out64, a, t, wa, s);
    default: return launch_long_warp_types<R, kModeF32>(in64, out64, a, t, wa, s);
  }
}

// Both segment sizes: segments [0, cbig) with `inner` (32 inner partitions),
// [cbig, p) with `inner_small` (31).
cudaError_t launch_long_warp(int mode, int R, bool in64, bool out64, const LongArgs& a, const DevLineTables& inner,
                             const DevLineTables* inner_small, const LongWarpArgs& wa0, const LwIface* ifc,
                             cudaStream_t s, int* launches) {
  *launches = 0;
  for (int part = 0; part < 2; part++) {
    LongWarpArgs wa = wa0;
    wa.ifc = ifc[part];
    wa.seg0 = part == 0 ? 0 : a.cbig;
    wa.nseg = part == 0 ? a.cbig : a.p - a.cbig;
    if (wa.nseg <= 0) continue;
    if (part == 1 && !inner_small) return cudaErrorInvalidValue;
    wa.nchunks = (wa.nseg + kLongWarps - 1) / kLongWarps;
    const DevLineTables& t = part == 0 ? inner : *inner_small;
    const cudaError_t e = R == 1 ? launch_long_warp_r<1>(mode, in64, out64, a, t, wa, s)
                                 : launch_long_warp_r<2>(mode, in64, out64, a, t, wa, s);
    if (e != cudaSuccess) return e;
    ++*launches;
  }
  return cudaSuccess;
}

}  // namespace cbs
