// Instantiates the size-specialised fused kernel for float fields, 2 fields.
#include "opo_fused2.cuh"

namespace opo {
namespace f2 {
OPO_F2_DISPATCH_DEF_NODK(dispatch_f32_f2, float, 2)
} // namespace f2
} // namespace opo
