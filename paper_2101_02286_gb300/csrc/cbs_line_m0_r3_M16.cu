// Instantiations of the on-chip line kernel: mode 0, half bandwidth 3, 16 rows per lane.
#include "cbs_line_launch.cuh"
namespace cbs {
CBS_DEFINE_LINE_LAUNCH(0, 3, 16)
}  // namespace cbs
