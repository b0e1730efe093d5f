// Instantiation of the cRKFR kernels for one (system, precision, volume flux); N = 1..5.
#include "cr_variant.cuh"
namespace crk {
bool ops_mhd2_fp32_central(int N, VariantOps* o) { return fill_ops<GlmMhd<VOL_CENTRAL>, float>(N, o); }
}  // namespace crk
