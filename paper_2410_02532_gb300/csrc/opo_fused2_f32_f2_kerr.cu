// Instantiates the size-specialised fused kernel with the Kerr terms for
// float fields, 2 fields.
#include "opo_fused2.cuh"

namespace opo {
namespace f2 {
OPO_F2_DISPATCH_KERR_DEF(dispatch_f32_f2, float, 2)
} // namespace f2
} // namespace opo
