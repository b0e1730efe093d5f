// Instantiation of the cRKFR kernels for one (system, precision, volume flux); N = 1..5.
#include "cr_variant.cuh"
namespace crk {
bool ops_euler3_fp64_ec(int N, VariantOps* o) { return fill_ops<Euler<3, VOL_EC>, double>(N, o); }
}  // namespace crk
