// Traversal kernels for row widths: 12 20 (32-bit words per bitset row).
#include "mce_trav_inst.cuh"
namespace mce {
MCE_INSTANTIATE_WP(12)
MCE_INSTANTIATE_WP(20)
}  // namespace mce
