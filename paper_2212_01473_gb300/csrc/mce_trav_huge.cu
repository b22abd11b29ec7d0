// Traversal kernels for row widths: 68 132 (32-bit words per bitset row).
#include "mce_trav_inst.cuh"
namespace mce {
MCE_INSTANTIATE_WP(68)
MCE_INSTANTIATE_WP(132)
}  // namespace mce
