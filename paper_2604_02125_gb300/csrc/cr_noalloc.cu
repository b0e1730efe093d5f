// cr_noalloc.cu -- cr_step_noalloc: one cRKFR step that allocates no memory.
//
// Some callers cannot allocate device memory when they advance a solve: an
// application whose memory pool (for example a framework's caching allocator)
// has already reserved the device, or a host loop that must not stall other
// streams, which cudaMalloc/cudaFree can do by synchronising the device.  For
// them this entry point runs the same volume and face/update kernels as
// cr_step, with every scratch buffer (stage residual sums, face traces and
// the step record with its CFL reduction) carved out of one file-scope
// __device__ array of CR_NOALLOC_SCRATCH_BYTES.  The caller passes the input
// and output states; nothing is allocated or freed.
//
// The array exists once per device that loads the library and lives until the
// process exits.  All calls on a device share it and it keeps the last call's
// contents, so calls that overlap on the GPU (on different streams, or from
// several threads) race; the step record is cleared at the start of every
// call.  The array's device address is looked up on the first call on each
// device and kept for the life of the process; cudaDeviceReset destroys the
// context that address belongs to, so a process that resets a device must
// not call this entry point on that device afterwards.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/cr.h"
#include "cr_internal.h"

namespace crk {

static __device__ __align__(256) unsigned char g_noalloc_scratch[CR_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device address of the scratch array on the current device; looked up once
// per device (the host-side symbol is only a stand-in, never a device address).
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

int to_status(cudaError_t e) {
  if (e == cudaSuccess) return CR_OK;
  if (e == cudaErrorNoKernelImageForDevice || e == cudaErrorInvalidDevice || e == cudaErrorNoDevice)
    return CR_ENODEV;
  return CR_ECUDA;
}

bool desc_ok(const cr_mesh_desc& d) {
  if (d.eq != CR_EULER && d.eq != CR_GLM_MHD) return false;
  if (d.dim < 1 || d.dim > 3 || d.degree_N < 1 || d.degree_N > 5) return false;
  if (d.eq == CR_GLM_MHD && (d.dim != 2 || d.vol == CR_VOL_KEP)) return false;
  if (d.vol < 0 || d.vol > 2 || d.surf != CR_SURF_RUSANOV) return false;
  if (d.prec != CR_FP64 && d.prec != CR_FP32_PAIRFLUX) return false;
  if (d.scheme != CR_SCHEME_CRKFR || d.ncflux != CR_NCFLUX_REDUCED || d.limiter != CR_LIMITER_NONE) return false;
  if (!(d.gamma > 1.0) || !(d.cfl > 0.0) || !(d.dt_fixed >= 0.0) || !(d.c_h >= 0.0)) return false;   // NaN fails
  for (int k = 0; k < d.dim; ++k)
    if (d.cells[k] < 1 || !(d.hi[k] > d.lo[k])) return false;
  return true;
}

}  // namespace
}  // namespace crk

using namespace crk;

extern "C" int cr_step_noalloc(const cr_mesh_desc* desc, const double* u_in, double* u_out, double* dt_out,
                               void* cuda_stream) {
  if (!desc || !u_in || !u_out || !desc_ok(*desc)) return CR_EINVAL;
  const cr_mesh_desc& d = *desc;
  VariantOps o;
  if (!get_ops(d.eq, d.dim, d.prec, d.vol, d.degree_N, &o)) return CR_EINVAL;
  long long E = 1;
  for (int k = 0; k < d.dim; ++k) E *= d.cells[k];
  const long long nodes = E * o.NP;
  // scratch layout: step record | rbar | face traces
  const size_t off_rbar = align256(sizeof(DevState));
  const size_t off_trace = off_rbar + align256(o.real_bytes * (size_t)o.M * nodes);
  const size_t need = off_trace + align256(o.real_bytes * (size_t)o.dim * 2 * o.C * (E * o.NF));
  if (need > (size_t)CR_NOALLOC_SCRATCH_BYTES) return CR_ETOOLARGE;

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return to_status(e);
  unsigned char* base = nullptr;
  e = scratch_address(dev, (void**)&base);
  if (e != cudaSuccess) return to_status(e);
  cudaStream_t s = (cudaStream_t)cuda_stream;

  LaunchCtx lc;
  memset(&lc, 0, sizeof(lc));
  lc.u = u_out;
  lc.st = (DevState*)base;
  lc.rbar = base + off_rbar;
  lc.trace = base + off_trace;
  lc.totals_part = nullptr;
  lc.ma.E = E;
  for (int k = 0; k < 3; ++k) {
    lc.ma.cells[k] = k < d.dim ? d.cells[k] : 1;
    lc.ma.cdiv[k] = make_fastdiv((unsigned)lc.ma.cells[k]);
    lc.ma.inv_dx[k] = k < d.dim ? d.cells[k] / (d.hi[k] - d.lo[k]) : 0.0;
  }
  for (int k = 0; k < 3; ++k) lc.ma.inv_dx_f[k] = (float)lc.ma.inv_dx[k];
  lc.ma.gamma_f = (float)d.gamma;
  lc.ma.c_h_f = (float)d.c_h;
  lc.ma.cfl = d.cfl;
  lc.ma.dt_fixed = d.dt_fixed;
  lc.ma.gamma = d.gamma;
  lc.ma.c_h = d.c_h;
  lc.pp64 = PhysParams<double>{d.gamma, 1.0 / (d.gamma - 1.0), d.c_h, d.vol};
  lc.pp32 = PhysParams<float>{(float)d.gamma, (float)(1.0 / (d.gamma - 1.0)), (float)d.c_h, d.vol};
  fill_ref_tables(d.degree_N, lc.ma, &lc.tb64, &lc.tb32);
  lc.epb = default_epb(o);
  lc.sms = 1;
  if ((e = cudaDeviceGetAttribute(&lc.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return to_status(e);
  lc.ma.tma_ok = tma_ok_for(u_out, E, o.NP);

  if ((e = o.set_smem(o.vol_smem(lc.epb))) != cudaSuccess) return to_status(e);
  if (u_out != u_in &&
      (e = cudaMemcpyAsync(u_out, u_in, sizeof(double) * (size_t)o.M * nodes, cudaMemcpyDeviceToDevice, s)) !=
          cudaSuccess)
    return to_status(e);
  // the shared step record starts clean: t, steps, status, CFL slots (slot 0: u^n)
  if ((e = cudaMemsetAsync(lc.st, 0, sizeof(DevState), s)) != cudaSuccess) return to_status(e);
  lc.slot = 0;
  if ((e = o.lambda(lc, s)) != cudaSuccess) return to_status(e);
  if ((e = o.volume(lc, s)) != cudaSuccess) return to_status(e);
  if ((e = o.face_update(lc, s)) != cudaSuccess) return to_status(e);
  if (dt_out && (e = cudaMemcpyAsync(dt_out, &lc.st->dt, sizeof(double), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return to_status(e);
  return CR_OK;
}
