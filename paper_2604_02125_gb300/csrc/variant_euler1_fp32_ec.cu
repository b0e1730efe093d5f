// Instantiation of the cRKFR kernels for one (system, precision, volume flux); N = 1..5.
#include "cr_variant.cuh"
namespace crk {
bool ops_euler1_fp32_ec(int N, VariantOps* o) { return fill_ops<Euler<1, VOL_EC>, float>(N, o); }
}  // namespace crk
