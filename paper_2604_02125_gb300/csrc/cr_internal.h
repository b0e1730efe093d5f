// cr_internal.h -- host-side declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include "crkfr_kernels.cuh"

namespace crk {

// Everything a launch needs; R-typed buffers are passed as void*.
struct LaunchCtx {
  double* u;
  void* rbar;
  void* trace;
  DevState* st;
  double* partials;
  double* totals_part;
  MeshArgs ma;
  PhysParams<double> pp64;
  PhysParams<float> pp32;
  RefTab<double> tb64;
  RefTab<float> tb32;
  int epb;            // elements per CTA of the volume kernel
};

struct VariantOps {
  int M, NP, NF, C, dim;
  size_t vol_bytes_per_elem;   // shared memory per element of the volume kernel
  size_t real_bytes;           // sizeof(R)
  cudaError_t (*volume)(const LaunchCtx&, cudaStream_t);
  cudaError_t (*face_update)(const LaunchCtx&, cudaStream_t);
  cudaError_t (*lambda)(const LaunchCtx&, cudaStream_t);
  cudaError_t (*totals)(const LaunchCtx&, cudaStream_t);
  cudaError_t (*set_smem)(size_t bytes);
};

// one getter per (system, dim, precision); N = 1..5; returns false if absent
bool ops_euler1_fp64(int N, VariantOps* o);
bool ops_euler2_fp64(int N, VariantOps* o);
bool ops_euler3_fp64(int N, VariantOps* o);
bool ops_mhd2_fp64(int N, VariantOps* o);
bool ops_euler1_fp32(int N, VariantOps* o);
bool ops_euler2_fp32(int N, VariantOps* o);
bool ops_euler3_fp32(int N, VariantOps* o);
bool ops_mhd2_fp32(int N, VariantOps* o);

// reference-element tables on [0,1] computed on the host (Newton on P_N', barycentric D)
void ref_tables(int N, double* xi, double* w, double D[6][6]);

// launchers of a (system, dim, precision, degree) variant; false if none
bool get_ops(int eq, int dim, int prec, int N, VariantOps* o);

// elements per CTA of the volume kernel used by every context of a variant
int default_epb(const VariantOps& o);

}  // namespace crk
