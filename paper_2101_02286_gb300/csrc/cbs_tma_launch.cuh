// cbs_tma_launch.cuh -- host side of the TMA-fed refinement line kernel:
// tensor maps over the caller's arrays, the interface tables and the launch
// of one tile shape.  Instantiated per (rows per partition, interface
// precision) in the cbs_tma_m*.cu units.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "cbs_line_launch.cuh"
#include "cbs_tma.cuh"

namespace cbs {

bool make_iface(const DevLineTables& D, bool fp64, TmaIface& f);
bool tma_encode(CUtensorMap* map, const void* ptr, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
                const cuuint32_t* box, CUtensorMapSwizzle sw);

inline CUtensorMapSwizzle tma_swizzle_mode(int bytes) {
  return bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
}

// Tensor map of the caller's array `ptr` as the kernel tiles it (see the
// kernel's comment); false when the driver refuses it.
template <int M, bool STRIDED, int TL>
bool tile_map(CUtensorMap* map, const void* ptr, const LineArgs& a) {
  const CUtensorMapSwizzle sw = tma_swizzle_mode(tma_swizzle<M, STRIDED, TL>());
  if constexpr (!STRIDED) {
    const cuuint64_t dims[2] = {(cuuint64_t)M, (cuuint64_t)a.nlines * 32};
    const cuuint64_t strides[1] = {(cuuint64_t)M * 8};
    const cuuint32_t box[2] = {(cuuint32_t)M, (cuuint32_t)TL * 32};
    return tma_encode(map, ptr, 2, dims, strides, box, sw);
  } else {
    // (x, partition i, row k in the partition, remaining axis)
    const cuuint64_t nx = (cuuint64_t)a.nx, ny = (cuuint64_t)a.ny, nz = (cuuint64_t)a.nz;
    const cuuint64_t es = a.dir == 1 ? nx : nx * ny;       // row stride of a line (elements)
    const cuuint64_t other = a.dir == 1 ? nz : ny;         // extent of the remaining axis
    const cuuint64_t ostride = a.dir == 1 ? nx * ny : nx;  // its stride
    const cuuint64_t dims[4] = {nx, 32, (cuuint64_t)M, other};
    const cuuint64_t strides[3] = {es * M * 8, es * 8, ostride * 8};
    const cuuint32_t box[4] = {(cuuint32_t)TL, 32, (cuuint32_t)M, 1};
    return tma_encode(map, ptr, 4, dims, strides, box, sw);
  }
}

constexpr int kTmaMaxDevices = 64;

// Integer bands (alpha = 1/D, D in 2..6, to 2^-48): the launch arguments of
// the scaled system A' = D A (stencil weights times D, bulk pivot
// reciprocals divided by D); false otherwise.
bool tma_integer_bands(const LineArgs& a, const DevLineTables& t, LineArgs& a2, DevLineTables& t2, TmaIface& f);

template <int M, int KS, typename TIR, bool STRIDED, int TL, int W, int NBUF>
cudaError_t launch_tma_t(const LineArgs& a0, const DevLineTables& t0, int fault, cudaStream_t s) {
  alignas(64) CUtensorMap tin, tout;
  TmaIface f;
  if (!make_iface(t0, sizeof(TIR) == 8, f)) return cudaErrorNotSupported;
  LineArgs a = a0;
  DevLineTables t = t0;
  tma_integer_bands(a0, t0, a, t, f);
  if (fault == 1) {  // test of the timeout path: a 1 ms limit on the wait that CTA 0 cannot satisfy
    f.fault = 1;
    f.wait_ns = 1000000ull;
  }
  if (!tile_map<M, STRIDED, TL>(&tin, a.in, a) || !tile_map<M, STRIDED, TL>(&tout, a.out, a))
    return cudaErrorNotSupported;
  int gx = 1;
  int64_t ntiles;
  if constexpr (STRIDED) {
    gx = (int)((a.nx + TL - 1) / TL);
    ntiles = (int64_t)gx * (a.dir == 1 ? a.nz : a.ny);
  } else {
    ntiles = (a.nlines + TL - 1) / TL;
  }
  if (ntiles > 0x7fffffff / (32 * TL)) return cudaErrorNotSupported;
  if (ntiles == 0) return cudaSuccess;
  const size_t smem = NBUF * (size_t)TL * 32 * M * 8 + 16 + 1024;
  auto kern = refine_tma_kernel<M, KS, TIR, STRIDED, TL, W, NBUF>;
  // the dynamic shared-memory limit and the occupancy are per device
  static std::mutex mu;
  static int per_sm[kTmaMaxDevices] = {};
  int dev = 0, blocks_per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kTmaMaxDevices) return cudaErrorNotSupported;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (per_sm[dev] == 0) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[dev], kern, W * 32, smem);
      if (e != cudaSuccess) {
        per_sm[dev] = 0;
        return e;
      }
      if (per_sm[dev] < 1) return cudaErrorInvalidConfiguration;
    }
    blocks_per_sm = per_sm[dev];
  }
  const int64_t want = (int64_t)blocks_per_sm * sm_count();
  const unsigned blocks = (unsigned)(ntiles < want ? ntiles : want);
  kern<<<blocks, W * 32, smem, s>>>(tin, tout, a, t, f, gx, (int)ntiles);
  return cudaGetLastError();
}

// Tile shapes (tile_lines): x-lines 4 or 8 lines per tile (two buffers, a warp
// per line); y/z lines 4 or 8 (two buffers, a warp per line), 16 (one buffer,
// 8 warps of two lines each) or, for 32, 16 lines with 16 warps and two
// buffers.  0 = the default of the direction.
template <int M, typename TIR>
cudaError_t launch_tma_m(int KS, const LineArgs& a, const DevLineTables& t, int tile_lines, int fault, cudaStream_t s);

#define CBS_DEFINE_TMA_LAUNCH(M, TIR)                                                                        \
  template <>                                                                                                \
  cudaError_t launch_tma_m<M, TIR>(int KS, const LineArgs& a, const DevLineTables& t, int tl, int fault, cudaStream_t s) { \
    if (a.dir == 0) {                                                                                        \
      if (tl == 8) return KS == 2 ? launch_tma_t<M, 2, TIR, false, 8, 8, 2>(a, t, fault, s)                         \
                                  : launch_tma_t<M, 0, TIR, false, 8, 8, 2>(a, t, fault, s);                        \
      return KS == 2 ? launch_tma_t<M, 2, TIR, false, 4, 4, 2>(a, t, fault, s)                                      \
                     : launch_tma_t<M, 0, TIR, false, 4, 4, 2>(a, t, fault, s);                                     \
    }                                                                                                        \
    if (tl == 0) tl = a.dir == 1 ? 4 : 16;                                                                   \
    if (tl == 16) return KS == 2 ? launch_tma_t<M, 2, TIR, true, 16, 8, 1>(a, t, fault, s)                          \
                                 : launch_tma_t<M, 0, TIR, true, 16, 8, 1>(a, t, fault, s);                         \
    if (tl == 32) return KS == 2 ? launch_tma_t<M, 2, TIR, true, 16, 16, 2>(a, t, fault, s)                         \
                                 : launch_tma_t<M, 0, TIR, true, 16, 16, 2>(a, t, fault, s);                        \
    if (tl == 8) return KS == 2 ? launch_tma_t<M, 2, TIR, true, 8, 8, 2>(a, t, fault, s)                            \
                                : launch_tma_t<M, 0, TIR, true, 8, 8, 2>(a, t, fault, s);                           \
    return KS == 2 ? launch_tma_t<M, 2, TIR, true, 4, 4, 2>(a, t, fault, s) : launch_tma_t<M, 0, TIR, true, 4, 4, 2>(a, t, fault, s); \
  }

}  // namespace cbs
