// Instantiates the size-specialised fused kernel for float fields, 3 fields,
// for instances whose crystals all have dk = 0 (no phase-factor products).
#include "opo_fused2.cuh"

namespace opo {
namespace f2 {
OPO_F2_DISPATCH_NODK_DEF(dispatch_f32_f3, float, 3)
} // namespace f2
} // namespace opo
