// Instantiation of the cRKFR kernels for one (system, precision); N = 1..5.
#include "cr_variant.cuh"
namespace crk {
bool ops_euler3_fp64(int N, VariantOps* o) { return fill_ops<Euler<3>, double>(N, o); }
}  // namespace crk
