// cr_batched.h -- batched form: many independent 2D Euler solves advanced by one
// persistent kernel per step (implemented in cr_batched.cu).
#pragma once
#include "../../include/cr.h"
#include <cuda_runtime.h>

namespace crk {
struct BatchedCtx;
int batched_init(BatchedCtx** out, const cr_mesh_desc* desc, int n, cudaStream_t s);
int batched_state_size(const BatchedCtx* b, int solve, int* n_vars, long long* n_nodes);
int batched_set_state(BatchedCtx* b, int solve, const double* u, int on_device);
int batched_set_state_async(BatchedCtx* b, int solve, const double* u, int on_device);
int batched_get_state_async(BatchedCtx* b, int solve, double* u, int on_device);
int batched_step(BatchedCtx* b, int nsteps);
int batched_sync(BatchedCtx* b);
int batched_get_state(BatchedCtx* b, int solve, double* u, int on_device);
int batched_get_info(BatchedCtx* b, int solve, double* t, double* dt, long long* steps, double* totals);
int batched_time_kernels(BatchedCtx* b, int nsteps, void* flush, size_t bytes, double* ms);
const char* batched_tuning(const BatchedCtx* b);
void batched_destroy(BatchedCtx* b);
}  // namespace crk
