// Instantiations of the TMA-fed refinement kernel: 8 rows per partition, interface in FP32.
#include "cbs_tma_launch.cuh"
namespace cbs {
CBS_DEFINE_TMA_LAUNCH(8, float)
}  // namespace cbs
