// Instantiation of the cRKFR kernels for one (system, precision); N = 1..5.
#include "cr_variant.cuh"
namespace crk {
bool ops_euler1_fp64(int N, VariantOps* o) { return fill_ops<Euler<1>, double>(N, o); }
}  // namespace crk
