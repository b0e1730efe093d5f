// cr_internal.h -- host-side declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include "../../include/cr.h"
#include "crkfr_fused.cuh"
#include "crkfr_limiter.cuh"
#include "crkfr_volume_lanes.cuh"

namespace crk {

// Everything a launch needs; R-typed buffers are passed as void*.
struct LaunchCtx {
  double* u;
  void* rbar;
  void* trace;
  DevState* st;
  double* totals_part;
  MeshArgs ma;
  PhysParams<double> pp64;
  PhysParams<float> pp32;
  RefTab<double> tb64;
  RefTab<float> tb32;
  int epb;            // elements per CTA of the volume kernel (tile form)
  int sms;            // multiprocessors of the device (persistent grids)
  int slot;           // step parity: CFL-reduction slot of the state the next step starts from
  // multi-stage RKFR scratch: stage state u^(j) (FP64, like u) and the
  // increments K_0..K_{s-2} ([stage][var][elem][node], R)
  double* ustage;
  void* kbuf;
  // subcell blending limiter: the state buffer the step writes (u holds u^n),
  // the coefficients before smoothing (one per element) and the tables
  double* u_next;
  double* araw;
  double* alpha;      // smoothed coefficients
  unsigned char* touched;   // 1 where the limited step changes the element's update
  unsigned* tlist;          // the touched elements, in no particular order
  unsigned* tcount;         // their number (reset by the coefficient kernel)
  LimTab lt;
  // fused single-launch step: per-tile readiness values
  unsigned* flags;
};

// One launch of a batched persistent kernel (all solves of one degree).
struct BatchLaunch {
  const BatchSolve* solves;
  const BatchTile* tiles;
  unsigned ntiles;
  int grid;
  PhysParams<double> pp64;
  PhysParams<float> pp32;
  RefTab<double> tb64;
  RefTab<float> tb32;
  int slot;           // step parity (as LaunchCtx::slot)
  int shape;          // volume kernel shape (0: default, 1: alternative; chosen by the autotuner)
};

struct VariantOps {
  int M, NP, NF, C, dim;       // C: components of a face record
  size_t ncs_per_elem;         // stage-wise non-conservative flux: stage-trace values per element after the records
  size_t vol_bytes_per_elem;   // shared memory per element of the tile volume kernel
  bool lanes;                  // the lane-form volume kernel is used (32 elements per CTA)
  size_t (*vol_smem)(int epb); // dynamic shared memory of one volume CTA
  size_t real_bytes;           // sizeof(R)
  cudaError_t (*volume)(const LaunchCtx&, cudaStream_t);
  cudaError_t (*face_update)(const LaunchCtx&, cudaStream_t);
  // one stage of the multi-stage RKFR step: volume part on u_in (first: the
  // step's first launch, which derives and records dt), face / update part of
  // stage j of s (intermediate stage states go to ustage, the last to u)
  cudaError_t (*volume_stage)(const LaunchCtx&, cudaStream_t, const double* u_in, int first);
  cudaError_t (*face_stage)(const LaunchCtx&, cudaStream_t, int j, int s);
  // subcell blending limiter (Euler; null elsewhere): coefficients of u, then
  // the limited face / update kernel from u into u_next
  cudaError_t (*alpha)(const LaunchCtx&, cudaStream_t);
  cudaError_t (*face_limited)(const LaunchCtx&, cudaStream_t);
  // FP32 lane form: the volume kernel that also evaluates the raw
  // coefficients of u, then the smoothing pass alone (null elsewhere)
  cudaError_t (*volume_ind)(const LaunchCtx&, cudaStream_t);
  cudaError_t (*alpha_smooth)(const LaunchCtx&, cudaStream_t);
  // the whole step in one cooperative persistent launch (lane forms of the
  // single-stage scheme; null where the layouts do not allow it); phase 0..2
  cudaError_t (*step_fused)(const LaunchCtx&, cudaStream_t, int phase);
  cudaError_t (*lambda)(const LaunchCtx&, cudaStream_t);
  cudaError_t (*totals)(const LaunchCtx&, cudaStream_t);
  cudaError_t (*set_smem)(size_t bytes);
  // batched persistent kernels (2D Euler only; null elsewhere)
  cudaError_t (*vol_batched)(const BatchLaunch&, cudaStream_t);
  cudaError_t (*face_batched)(const BatchLaunch&, cudaStream_t);
  int (*occupancy)(int which, int shape);   // resident CTAs per SM: 0 = volume, 1 = face
  int vol_shapes;               // volume kernel shapes of the batched form
  int threads_vol, threads_face;
};

// one getter per (system, dim, precision, volume flux); N = 1..5; false if absent
bool ops_euler1_fp64_ec(int N, VariantOps* o);
bool ops_euler1_fp64_kep(int N, VariantOps* o);
bool ops_euler1_fp64_central(int N, VariantOps* o);
bool ops_euler1_fp32_ec(int N, VariantOps* o);
bool ops_euler1_fp32_kep(int N, VariantOps* o);
bool ops_euler1_fp32_central(int N, VariantOps* o);
bool ops_euler2_fp64_ec(int N, VariantOps* o);
bool ops_euler2_fp64_kep(int N, VariantOps* o);
bool ops_euler2_fp64_central(int N, VariantOps* o);
bool ops_euler2_fp32_ec(int N, VariantOps* o);
bool ops_euler2_fp32_kep(int N, VariantOps* o);
bool ops_euler2_fp32_central(int N, VariantOps* o);
bool ops_euler3_fp64_ec(int N, VariantOps* o);
bool ops_euler3_fp64_kep(int N, VariantOps* o);
bool ops_euler3_fp64_central(int N, VariantOps* o);
bool ops_euler3_fp32_ec(int N, VariantOps* o);
bool ops_euler3_fp32_kep(int N, VariantOps* o);
bool ops_euler3_fp32_central(int N, VariantOps* o);
bool ops_mhd2_fp64_ec(int N, VariantOps* o);
bool ops_mhd2_fp64_central(int N, VariantOps* o);
bool ops_mhd2_fp32_ec(int N, VariantOps* o);
bool ops_mhd2_fp32_central(int N, VariantOps* o);
bool ops_mhd2s_fp64_ec(int N, VariantOps* o);
bool ops_mhd2s_fp64_central(int N, VariantOps* o);
bool ops_mhd2s_fp32_ec(int N, VariantOps* o);
bool ops_mhd2s_fp32_central(int N, VariantOps* o);

// reference-element tables on [0,1] computed on the host (Newton on P_N', barycentric D)
void ref_tables(int N, double* xi, double* w, double D[6][6]);

// reference-element and tableau tables of degree N in both precisions
void fill_ref_tables(int N, const MeshArgs& ma, RefTab<double>* t64, RefTab<float>* t32);

// launchers of a (system, dim, precision, degree) variant; false if none;
// ncflux = CR_NCFLUX_STAGES selects the GLM-MHD kernels with the stage-wise
// non-conservative flux
bool get_ops(int eq, int dim, int prec, int vol, int N, VariantOps* o, int ncflux = 0);

// limiter tables of degree N (orthonormal Legendre modes from GLL values,
// subcell widths, logistic threshold and sharpness)
void fill_lim_tab(int N, double alpha_max, LimTab* lt);

// elements per CTA of the volume kernel used by every context of a variant
int default_epb(const VariantOps& o);

// mesh arguments, physics parameters and tables of one descriptor (no allocation)
void fill_launch_ctx(const cr_mesh_desc& d, const VariantOps& o, LaunchCtx* lc);

// 1 if whole tiles of a state at u (E elements of NP nodes) can be bulk-copied
int tma_ok_for(const double* u, long long E, int NP);

}  // namespace crk
