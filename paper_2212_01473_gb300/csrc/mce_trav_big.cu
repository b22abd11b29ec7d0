// Traversal kernels for row widths: 28 36 (32-bit words per bitset row).
#include "mce_trav_inst.cuh"
namespace mce {
MCE_INSTANTIATE_WP(28)
MCE_INSTANTIATE_WP(36)
}  // namespace mce
