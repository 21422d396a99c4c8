// Instantiates the size-specialised fused kernel for float fields, 2 fields,
// for instances whose crystals all have dk = 0 (no phase-factor products).
#include "opo_fused2.cuh"

namespace opo {
namespace f2 {
OPO_F2_DISPATCH_NODK_DEF(dispatch_f32_f2, float, 2)
} // namespace f2
} // namespace opo
