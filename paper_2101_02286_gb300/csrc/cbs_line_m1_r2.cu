// Instantiations of the on-chip line kernel for mode 1, half bandwidth 2.
#include "cbs_line_launch.cuh"
namespace cbs {
CBS_DEFINE_LINE_LAUNCH(1, 2)
}  // namespace cbs
