// Instantiation of the cRKFR kernels for one (system, precision, volume flux); N = 1..5.
// GLM-MHD with the stage-wise non-conservative numerical flux (eq. bad.numflux.non.cons).
#include "cr_variant.cuh"
namespace crk {
bool ops_mhd2s_fp32_ec(int N, VariantOps* o) { return fill_ops<GlmMhdStages<VOL_EC>, float>(N, o); }
}  // namespace crk
