// Traversal kernels for row widths: 1 2 4 (32-bit words per bitset row).
#include "mce_trav_inst.cuh"
namespace mce {
MCE_INSTANTIATE_WP(1)
MCE_INSTANTIATE_WP(2)
MCE_INSTANTIATE_WP(4)
}  // namespace mce
