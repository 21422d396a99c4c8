// Instantiates the size-specialised fused kernel with the Kerr terms for
// double fields, 3 fields.
#include "opo_fused2.cuh"

namespace opo {
namespace f2 {
OPO_F2_DISPATCH_KERR_DEF(dispatch_f64_f3, double, 3)
} // namespace f2
} // namespace opo
