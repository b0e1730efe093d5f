// Instantiation of the cRKFR kernels for one (system, precision); N = 1..5.
#include "cr_variant.cuh"
namespace crk {
bool ops_euler1_fp32(int N, VariantOps* o) { return fill_ops<Euler<1>, float>(N, o); }
}  // namespace crk
