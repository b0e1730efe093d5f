// cr_batched.cu -- batched persistent form (not yet available: rejects).
#include "cr_batched.h"
namespace crk {
struct BatchedCtx {};
int batched_init(BatchedCtx** out, const cr_mesh_desc*, int, cudaStream_t) { *out = nullptr; return CR_EINVAL; }
int batched_state_size(const BatchedCtx*, int, int*, long long*) { return CR_EINVAL; }
int batched_set_state(BatchedCtx*, int, const double*, int) { return CR_EINVAL; }
int batched_step(BatchedCtx*, int) { return CR_EINVAL; }
int batched_sync(BatchedCtx*) { return CR_EINVAL; }
int batched_get_state(BatchedCtx*, int, double*, int) { return CR_EINVAL; }
int batched_get_info(BatchedCtx*, int, double*, double*, long long*, double*) { return CR_EINVAL; }
int batched_time_kernels(BatchedCtx*, int, void*, size_t, double*) { return CR_EINVAL; }
void batched_destroy(BatchedCtx*) {}
}  // namespace crk
