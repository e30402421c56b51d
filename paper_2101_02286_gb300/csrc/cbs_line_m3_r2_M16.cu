// Instantiations of the on-chip line kernel: mode 3 (refinement, FP64 interface), half bandwidth 2, 16 rows per lane.
#include "cbs_line_launch.cuh"
namespace cbs {
CBS_DEFINE_LINE_LAUNCH(3, 2, 16)
}  // namespace cbs
