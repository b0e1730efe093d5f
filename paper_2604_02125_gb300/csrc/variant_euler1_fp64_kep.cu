// Instantiation of the cRKFR kernels for one (system, precision, volume flux); N = 1..5.
#include "cr_variant.cuh"
namespace crk {
bool ops_euler1_fp64_kep(int N, VariantOps* o) { return fill_ops<Euler<1, VOL_KEP>, double>(N, o); }
}  // namespace crk
