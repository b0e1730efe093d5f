// Instantiation of the cRKFR kernels for one (system, precision, volume flux); N = 1..5.
#include "cr_variant.cuh"
namespace crk {
bool ops_euler2_fp64_central(int N, VariantOps* o) { return fill_ops<Euler<2, VOL_CENTRAL>, double>(N, o); }
}  // namespace crk
