// Instantiations of the TMA-fed refinement kernel: 16 rows per partition, interface in FP64.
#include "cbs_tma_launch.cuh"
namespace cbs {
CBS_DEFINE_TMA_LAUNCH(16, double)
}  // namespace cbs
