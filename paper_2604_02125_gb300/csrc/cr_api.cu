// cr_api.cu -- C ABI of the cRKFR library (declared in include/cr.h).
//
// One solve (n_solves == 1): per step the volume kernel and the fused
// face-flux/update kernel run on the caller's stream, replayed from CUDA graphs
// captured at set-up (1-step and 16-step graphs); the multi-stage RKFR scheme
// runs the pair once per RK stage.  The batched form (n_solves > 1) lives in
// cr_batched.cu.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/cr.h"
#include "cr_internal.h"
#include "cr_batched.h"

namespace crk {

// ---------------------------------------------------------------------------
// Reference element on [0,1]: GLL points by Newton's method on
// (1 - x^2) P_N'(x) (whose derivative is -N(N+1) P_N by Legendre's equation)
// from Chebyshev-Lobatto guesses; weights 1/(N(N+1) P_N(x)^2); differentiation
// matrix by barycentric weights with the negative-sum diagonal.
// ---------------------------------------------------------------------------
static void legendre_pd(int N, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x;
  for (int k = 1; k < N; ++k) {
    double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    p0 = p1;
    p1 = p2;
  }
  *P = (N == 0) ? 1.0 : p1;
  // P_N' = N (P_{N-1} - x P_N) / (1 - x^2) away from the end points
  *dP = (N == 0) ? 0.0 : N * (p0 - x * p1) / (1.0 - x * x);
}

void ref_tables(int N, double* xi, double* w, double D[6][6]) {
  const double pi = 3.14159265358979323846;
  double x[6];
  for (int k = 0; k <= N; ++k) {
    double xk = -std::cos(pi * k / N);
    if (k > 0 && k < N) {
      for (int it = 0; it < 100; ++it) {
        double P, dP;
        legendre_pd(N, xk, &P, &dP);
        double dx = (1.0 - xk * xk) * dP / (N * (N + 1.0) * P);
        xk += dx;
        if (std::fabs(dx) < 1e-16) break;
      }
    }
    x[k] = xk;
  }
  x[0] = -1.0;
  x[N] = 1.0;
  for (int k = 0; k <= N; ++k) {
    double P, dP;
    legendre_pd(N, x[k], &P, &dP);
    if (k == 0) P = (N % 2 == 0) ? 1.0 : -1.0;   // P_N(-1) = (-1)^N
    if (k == N) P = 1.0;
    xi[k] = 0.5 * (x[k] + 1.0);
    w[k] = 1.0 / (N * (N + 1.0) * P * P);
  }
  double lam[6];
  for (int j = 0; j <= N; ++j) {
    double prod = 1.0;
    for (int k = 0; k <= N; ++k)
      if (k != j) prod *= (xi[j] - xi[k]);
    lam[j] = 1.0 / prod;
  }
  for (int i = 0; i <= N; ++i) {
    double diag = 0.0;
    for (int j = 0; j <= N; ++j) {
      if (i == j) continue;
      D[i][j] = (lam[j] / lam[i]) / (xi[i] - xi[j]);
      diag -= D[i][j];
    }
    D[i][i] = diag;
  }
}

bool get_ops(int eq, int dim, int prec, int vol, int N, VariantOps* o, int ncflux) {
  if (ncflux == CR_NCFLUX_STAGES) {
    if (eq != CR_GLM_MHD || dim != 2) return false;
    if (prec == CR_FP64) return vol == 0 ? ops_mhd2s_fp64_ec(N, o) : vol == 2 ? ops_mhd2s_fp64_central(N, o) : false;
    return vol == 0 ? ops_mhd2s_fp32_ec(N, o) : vol == 2 ? ops_mhd2s_fp32_central(N, o) : false;
  }
  if (ncflux != CR_NCFLUX_REDUCED) return false;
  struct Entry {
    int eq, dim, prec, vol;
    bool (*fn)(int, VariantOps*);
  };
  static const Entry table[] = {
    {0, 1, 0, 0, &ops_euler1_fp64_ec},
    {0, 1, 0, 1, &ops_euler1_fp64_kep},
    {0, 1, 0, 2, &ops_euler1_fp64_central},
    {0, 1, 1, 0, &ops_euler1_fp32_ec},
    {0, 1, 1, 1, &ops_euler1_fp32_kep},
    {0, 1, 1, 2, &ops_euler1_fp32_central},
    {0, 2, 0, 0, &ops_euler2_fp64_ec},
    {0, 2, 0, 1, &ops_euler2_fp64_kep},
    {0, 2, 0, 2, &ops_euler2_fp64_central},
    {0, 2, 1, 0, &ops_euler2_fp32_ec},
    {0, 2, 1, 1, &ops_euler2_fp32_kep},
    {0, 2, 1, 2, &ops_euler2_fp32_central},
    {0, 3, 0, 0, &ops_euler3_fp64_ec},
    {0, 3, 0, 1, &ops_euler3_fp64_kep},
    {0, 3, 0, 2, &ops_euler3_fp64_central},
    {0, 3, 1, 0, &ops_euler3_fp32_ec},
    {0, 3, 1, 1, &ops_euler3_fp32_kep},
    {0, 3, 1, 2, &ops_euler3_fp32_central},
    {1, 2, 0, 0, &ops_mhd2_fp64_ec},
    {1, 2, 0, 2, &ops_mhd2_fp64_central},
    {1, 2, 1, 0, &ops_mhd2_fp32_ec},
    {1, 2, 1, 2, &ops_mhd2_fp32_central},
  };
  for (const Entry& e : table)
    if (e.eq == eq && e.dim == dim && e.prec == prec && e.vol == vol) return e.fn(N, o);
  return false;
}

void fill_ref_tables(int N, const MeshArgs& ma, RefTab<double>* t64, RefTab<float>* t32) {
  double xi[6], w[6], D[6][6];
  ref_tables(N, xi, w, D);
  std::memset(t64, 0, sizeof(*t64));
  std::memset(t32, 0, sizeof(*t32));
  for (int p = 0; p < 6; ++p) {
    for (int q = 0; q < 6; ++q) {
      t64->D[p][q] = (p <= N && q <= N) ? D[p][q] : 0.0;
      t32->D[p][q] = (float)t64->D[p][q];
      t32->D2f[p][q] = t64->D2f[p][q] = make_float2(2.0f * t32->D[p][q], 2.0f * t32->D[p][q]);
      t32->D2s[p][q] = t64->D2s[p][q] =
          make_float2(2.0f * t32->D[p][q] * ma.inv_dx_f[0], 2.0f * t32->D[p][q] * ma.inv_dx_f[1]);
    }
    t64->w[p] = t32->w[p] = p <= N ? w[p] : 0.0;
  }
  t64->iw0 = 1.0 / w[0];
  t64->iwN = 1.0 / w[N];
  t32->iw0 = (float)t64->iw0;
  t32->iwN = (float)t64->iwN;
  const int S = rk_stages(N);
  int slot = 0;
  for (int i = 0; i < 7; ++i) {
    t64->b[i] = i < S ? rk_b(N, i) : 0.0;
    t32->b[i] = (float)t64->b[i];
    for (int j = 0; j < 7; ++j) {
      t64->a[i][j] = (i < S && j < i) ? rk_a(N, i, j) : 0.0;
      t32->a[i][j] = (float)t64->a[i][j];
    }
    // a residual is kept in a slot if a stage beyond the next one uses it
    bool saved = false;
    for (int k = i + 2; k < S; ++k) saved = saved || rk_a(N, k, i) != 0.0;
    t64->slot[i] = t32->slot[i] = saved ? (signed char)slot++ : (signed char)-1;
  }
}

// Limiter tables.  Modal coefficients of the orthonormal Legendre basis
// phi_j = sqrt((2j+1)/2) P_j on [-1,1] from GLL node values: GLL quadrature is
// exact to degree 2N-1, so the discrete Gram matrix sum_p W_p phi_i phi_j is
// diagonal, with 1 for j < N and (2N+1)/N for j = N (the discrete norm of P_N
// is 2/N against 2/(2N+1)); hence m_j = sum_p W_p phi_j(x_p) v_p / G_jj,
// W_p = 2 w_p the weights on [-1,1].
void fill_lim_tab(int N, double alpha_max, LimTab* lt) {
  std::memset(lt, 0, sizeof(*lt));
  double xi[6], w[6], D[6][6];
  ref_tables(N, xi, w, D);
  for (int p = 0; p <= N; ++p) {
    const double x = 2.0 * xi[p] - 1.0;
    double pm1 = 1.0, pk = x;   // P_0, P_1
    for (int j = 0; j <= N; ++j) {
      double Pj;
      if (j == 0) Pj = 1.0;
      else if (j == 1) Pj = x;
      else {
        const double pn = ((2.0 * j - 1.0) * x * pk - (j - 1.0) * pm1) / j;
        pm1 = pk;
        pk = pn;
        Pj = pn;
      }
      const double phi = std::sqrt((2.0 * j + 1.0) / 2.0) * Pj;
      const double g = j < N ? 1.0 : (2.0 * N + 1.0) / N;
      lt->vinv[j][p] = 2.0 * w[p] * phi / g;
    }
    lt->w01[p] = w[p];
  }
  lt->tau = 0.5 * std::pow(10.0, -1.8 * std::pow(N + 1.0, 0.25));
  lt->sharp = std::log(9999.0);
  lt->alpha_max = alpha_max;
  for (int j = 0; j < 6; ++j)
    for (int p = 0; p < 6; ++p) lt->vinv_f[j][p] = (float)lt->vinv[j][p];
  lt->tau_f = (float)lt->tau;
  lt->sharp_f = (float)lt->sharp;
  lt->alpha_max_f = (float)alpha_max;
  // the energy fractions where 1/(1 + exp(-(sharp/tau)(E - tau))) = 0.001 and 0.999
  lt->e_lo_f = (float)(lt->tau * (1.0 + std::log(0.001 / 0.999) / lt->sharp));
  lt->e_hi_f = (float)(lt->tau * (1.0 + std::log(0.999 / 0.001) / lt->sharp));
}

void fill_launch_ctx(const cr_mesh_desc& d, const VariantOps& o, LaunchCtx* plc) {
  LaunchCtx& lc = *plc;
  std::memset(&lc, 0, sizeof(lc));
  long long E = 1;
  for (int k = 0; k < d.dim; ++k) E *= d.cells[k];
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
  int dev = 0;
  cudaGetDevice(&dev);
  lc.sms = 1;
  cudaDeviceGetAttribute(&lc.sms, cudaDevAttrMultiProcessorCount, dev);
}

// whole 32-element tiles of the state can be fetched with 16-byte bulk copies
int tma_ok_for(const double* u, long long E, int NP) {
  return ((reinterpret_cast<size_t>(u) & 15) == 0 && ((E * NP) % 2) == 0) ? 1 : 0;
}

int default_epb(const VariantOps& o) {
  int epb = 256 / o.NF;
  if (epb < 1) epb = 1;
  const size_t cap = 160 * 1024;
  while (epb > 1 && (size_t)epb * o.vol_bytes_per_elem > cap) --epb;
  // prefer a whole number of warps
  for (int e = epb; e >= 1; --e)
    if ((e * o.NF) % 32 == 0) return e;
  return epb;
}

}  // namespace crk

using namespace crk;

// NVTX range over an entry point (visible to Nsight tools; a push and a pop
// when no tool is attached)
namespace {
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

struct cr_ctx {
  int n_solves = 0;
  std::vector<cr_mesh_desc> desc;
  cudaStream_t stream = nullptr;
  int device = 0;
  // single-solve form
  VariantOps ops{};
  LaunchCtx lc{};
  long long E = 0, NP = 0;
  int M = 0;
  size_t totals_blocks = 0;
  bool has_state = false;
  int parity = 0;     // slot of the CFL reduction of the current state (the fused step: its phase, 0..2)
  // state buffers: ubuf[0] only, or with the limiter two, the state of parity p
  // in ubuf[p] (the limited step reads one and writes the other)
  double* ubuf[2] = {nullptr, nullptr};
  bool limited = false;
  // limiter, FP32 form: the indicator kernels run on a second stream beside
  // the volume kernel (both only read u^n; the indicator uses the FP64 pipe,
  // the volume kernel the FP32 one), joined before the face kernels
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // device buffers carved out of a caller's workspace (cr_init_mesh_ws): not freed here
  bool borrowed = false;
  cudaStream_t cap_stream = nullptr;
  // the whole step in one cooperative launch (crkfr_fused.cuh), phases mod 3
  bool fused = false;
  int nphase = 2;     // 2, or 3 for the fused step
  // graphs of 1 and 16 steps, one per starting parity / phase
  cudaGraphExec_t g1[3] = {nullptr, nullptr, nullptr}, g16[3] = {nullptr, nullptr, nullptr};
  // batched form
  BatchedCtx* batched = nullptr;
};

static int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return CR_OK;
  if (e == cudaErrorMemoryAllocation) return CR_ENOMEM;
  if (e == cudaErrorNoKernelImageForDevice || e == cudaErrorInvalidDevice || e == cudaErrorNoDevice ||
      e == cudaErrorInsufficientDriver)
    return CR_ENODEV;
  return CR_ECUDA;
}

#define CR_TRY(call)                       \
  do {                                     \
    cudaError_t _e = (call);               \
    if (_e != cudaSuccess) return cuda_status(_e); \
  } while (0)

static bool desc_valid(const cr_mesh_desc& d) {
  // node indices are 32-bit: at most 2^31 - 1 nodes per solve
  long long nodes = 1;
  for (int k = 0; k < d.dim && k < 3; ++k) nodes *= (long long)(d.cells[k] > 0 ? d.cells[k] : 1) * (d.degree_N + 1);
  if (nodes >= (1LL << 31)) return false;
  if (d.eq != CR_EULER && d.eq != CR_GLM_MHD) return false;
  if (d.dim < 1 || d.dim > 3) return false;
  if (d.eq == CR_GLM_MHD && (d.dim != 2 || d.vol == CR_VOL_KEP)) return false;
  if (d.degree_N < 1 || d.degree_N > 5) return false;
  if (d.vol < 0 || d.vol > 2 || d.surf != CR_SURF_RUSANOV) return false;
  if (d.prec != CR_FP64 && d.prec != CR_FP32_PAIRFLUX) return false;
  if (d.scheme != CR_SCHEME_CRKFR && d.scheme != CR_SCHEME_RKFR) return false;
  // the stage-wise non-conservative flux: GLM-MHD, single-stage scheme
  if (d.ncflux != CR_NCFLUX_REDUCED &&
      (d.ncflux != CR_NCFLUX_STAGES || d.eq != CR_GLM_MHD || d.scheme != CR_SCHEME_CRKFR))
    return false;
  if (!(d.gamma > 1.0) || !(d.cfl > 0.0) || !(d.dt_fixed >= 0.0) || !(d.c_h >= 0.0)) return false;   // NaN fails
  for (int k = 0; k < d.dim; ++k) {
    if (d.cells[k] < 1) return false;
    if (!(d.hi[k] > d.lo[k])) return false;
  }
  // the subcell blending limiter: Euler, single-stage scheme, 0 <= alpha_max <= 1
  if (d.limiter != CR_LIMITER_NONE &&
      (d.limiter != CR_LIMITER_BLENDING || d.eq != CR_EULER || d.scheme != CR_SCHEME_CRKFR ||
       !(d.alpha_max >= 0.0 && d.alpha_max <= 1.0)))
    return false;
  return true;
}

static void free_single(cr_ctx* c) {
  for (int p = 0; p < 3; ++p) {
    if (c->g1[p]) cudaGraphExecDestroy(c->g1[p]);
    if (c->g16[p]) cudaGraphExecDestroy(c->g16[p]);
    c->g1[p] = c->g16[p] = nullptr;
  }
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  c->side = nullptr;
  c->ev_fork = c->ev_join = nullptr;
  if (!c->borrowed) {
    cudaFree(c->ubuf[0]);
    cudaFree(c->ubuf[1]);
    cudaFree(c->lc.araw);
    cudaFree(c->lc.alpha);
    cudaFree(c->lc.touched);
    cudaFree(c->lc.tlist);
    cudaFree(c->lc.tcount);
    cudaFree(c->lc.flags);
    cudaFree(c->lc.rbar);
    cudaFree(c->lc.trace);
    cudaFree(c->lc.st);
    cudaFree(c->lc.totals_part);
    cudaFree(c->lc.ustage);
    cudaFree(c->lc.kbuf);
  }
  c->ubuf[0] = c->ubuf[1] = nullptr;
  c->lc.u = nullptr;
  c->lc.araw = c->lc.alpha = nullptr;
  c->lc.touched = nullptr;
  c->lc.tlist = c->lc.tcount = nullptr;
  c->lc.flags = nullptr;
  c->lc.rbar = c->lc.trace = nullptr;
  c->lc.st = nullptr;
  c->lc.totals_part = nullptr;
  c->lc.ustage = nullptr;
  c->lc.kbuf = nullptr;
  c->cap_stream = nullptr;
}

// one step from the state whose CFL reduction sits in slot `parity`
// state buffer of the given parity (the only one without the limiter)
static double* state_buf(const cr_ctx* c, int parity) { return c->ubuf[c->limited ? (parity & 1) : 0]; }

// phase / parity after one step
static int next_phase(const cr_ctx* c, int p) { return c->fused ? (p + 1) % 3 : p ^ 1; }

static int launch_step(cr_ctx* c, cudaStream_t s, int parity) {
  c->lc.slot = parity;
  if (c->fused) {
    CR_TRY(c->ops.step_fused(c->lc, s, parity));
    return CR_OK;
  }
  if (c->limited) {
    // coefficients of u^n, the cRKFR volume work, then the limited face /
    // update kernel from the parity's buffer into the other one
    c->lc.u = state_buf(c, parity);
    c->lc.u_next = state_buf(c, parity ^ 1);
    if (c->ops.volume_ind) {
      // FP32 lane form: the volume kernel evaluates the raw coefficients of
      // the tiles it has finished, then the smoothing pass
      CR_TRY(c->ops.volume_ind(c->lc, s));
      CR_TRY(c->ops.alpha_smooth(c->lc, s));
    } else if (c->desc[0].prec == CR_FP32_PAIRFLUX) {
      // FP32 form: the FP64 indicator beside the FP32 volume kernel
      // (measured 0.164 -> 0.155 ms per step at 256^2, N = 3)
      CR_TRY(cudaEventRecord(c->ev_fork, s));
      CR_TRY(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
      CR_TRY(c->ops.alpha(c->lc, c->side));
      CR_TRY(cudaEventRecord(c->ev_join, c->side));
      CR_TRY(c->ops.volume(c->lc, s));
      CR_TRY(cudaStreamWaitEvent(s, c->ev_join, 0));
    } else {
      // FP64 form: both would compete for the FP64 pipe (measured slower side by side)
      CR_TRY(c->ops.alpha(c->lc, s));
      CR_TRY(c->ops.volume(c->lc, s));
    }
    CR_TRY(c->ops.face_limited(c->lc, s));
    c->lc.u = state_buf(c, c->parity);
    return CR_OK;
  }
  if (c->desc[0].scheme == CR_SCHEME_RKFR) {
    // stage j: volume part on u^(j) (u^n for j = 0), face / update part
    // forming u^(j+1) (the state itself after the last stage)
    const int S = rk_stages(c->desc[0].degree_N);
    for (int j = 0; j < S; ++j) {
      CR_TRY(c->ops.volume_stage(c->lc, s, j == 0 ? c->lc.u : c->lc.ustage, j == 0));
      CR_TRY(c->ops.face_stage(c->lc, s, j, S));
    }
    return CR_OK;
  }
  CR_TRY(c->ops.volume(c->lc, s));
  CR_TRY(c->ops.face_update(c->lc, s));
  return CR_OK;
}

static int capture(cr_ctx* c, int steps, int parity, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  CR_TRY(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = CR_OK;
  int p = parity;
  for (int k = 0; k < steps && rc == CR_OK; ++k, p = next_phase(c, p)) rc = launch_step(c, c->cap_stream, p);
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
  if (rc != CR_OK) { if (g) cudaGraphDestroy(g); return rc; }
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  return cuda_status(e);
}

// The device buffers of a single-solve context, in carving order: where each
// pointer goes and its size.  Sets c->limited, c->fused and the sizes the
// context keeps; no CUDA call.
struct BufSpec {
  void** p;
  size_t bytes;
};
static int plan_single(cr_ctx* c, std::vector<BufSpec>* plan) {
  const cr_mesh_desc& d = c->desc[0];
  if (!get_ops(d.eq, d.dim, d.prec, d.vol, d.degree_N, &c->ops, d.ncflux)) return CR_EINVAL;
  const VariantOps& o = c->ops;
  c->M = o.M;
  c->NP = o.NP;
  long long E = 1;
  for (int k = 0; k < d.dim; ++k) E *= d.cells[k];
  c->E = E;
  LaunchCtx& lc = c->lc;
  const long long nodes = E * o.NP;
  const long long NFt = E * o.NF;
  // one partial sum per CTA of the totals kernel (256 nodes per CTA)
  c->totals_blocks = (size_t)((nodes + 255) / 256);
  c->limited = d.limiter == CR_LIMITER_BLENDING;
  if (c->limited && (!o.alpha || !o.face_limited)) return CR_EINVAL;
  // the single-launch step (crkfr_fused.cuh) on request only:
  // CRKFR_STEP_KERNELS=fused in the environment, for variants that have one.
  // Measured slower than the two kernels on every workload (the face / update
  // work, latency-bound, runs at the volume kernel's occupancy there), so the
  // two-kernel step is the default.
  const char* sk = std::getenv("CRKFR_STEP_KERNELS");
  c->fused = o.step_fused && d.scheme == CR_SCHEME_CRKFR && d.ncflux == CR_NCFLUX_REDUCED && !c->limited && sk &&
             std::strcmp(sk, "fused") == 0;
  c->nphase = c->fused ? 3 : 2;
  plan->clear();
  plan->push_back({(void**)&c->ubuf[0], sizeof(double) * (size_t)o.M * nodes});
  if (c->limited) {
    plan->push_back({(void**)&c->ubuf[1], sizeof(double) * (size_t)o.M * nodes});
    plan->push_back({(void**)&lc.araw, sizeof(double) * (size_t)E});
    plan->push_back({(void**)&lc.alpha, sizeof(double) * (size_t)E});
    plan->push_back({(void**)&lc.touched, (size_t)E});
    plan->push_back({(void**)&lc.tlist, sizeof(unsigned) * (size_t)E});
    plan->push_back({(void**)&lc.tcount, sizeof(unsigned)});
  }
  plan->push_back({&lc.rbar, o.real_bytes * (size_t)o.M * nodes});
  plan->push_back({&lc.trace, o.real_bytes * ((size_t)o.dim * 2 * o.C * NFt + o.ncs_per_elem * (size_t)E)});
  plan->push_back({(void**)&lc.st, sizeof(DevState)});
  plan->push_back({(void**)&lc.totals_part, sizeof(double) * c->totals_blocks * (o.M + 2)});
  if (d.scheme == CR_SCHEME_RKFR) {
    plan->push_back({(void**)&lc.ustage, sizeof(double) * (size_t)o.M * nodes});
    plan->push_back({&lc.kbuf, o.real_bytes * (size_t)(rk_stages(d.degree_N) - 1) * o.M * nodes});
  }
  if (c->fused) plan->push_back({(void**)&lc.flags, sizeof(unsigned) * (size_t)((E + 31) / 32)});
  return CR_OK;
}

static size_t align_ws(size_t b) { return (b + 255) & ~(size_t)255; }

static size_t plan_bytes(const std::vector<BufSpec>& plan) {
  size_t total = 0;
  for (const BufSpec& b : plan) total += align_ws(b.bytes);
  return total;
}

// workspace: nullptr = allocate every buffer; else carve them out of it
// (ws_bytes checked against the plan by the caller)
static int init_single(cr_ctx* c, void* workspace = nullptr) {
  const cr_mesh_desc& d = c->desc[0];
  std::vector<BufSpec> plan;
  int rc = plan_single(c, &plan);
  if (rc != CR_OK) return rc;
  const VariantOps& o = c->ops;
  const long long E = c->E;
  LaunchCtx& lc = c->lc;
  fill_launch_ctx(d, o, &lc);
  if (c->limited) fill_lim_tab(d.degree_N, d.alpha_max, &lc.lt);
  c->borrowed = workspace != nullptr;
  size_t off = 0;
  for (const BufSpec& b : plan) {
    if (workspace) {
      *b.p = static_cast<unsigned char*>(workspace) + off;
      off += align_ws(b.bytes);
    } else {
      cudaError_t e = cudaMalloc(b.p, b.bytes);
      if (e != cudaSuccess) { rc = cuda_status(e); break; }
    }
  }
  lc.u = c->ubuf[0];
  if (rc != CR_OK) { free_single(c); return rc; }
  lc.ma.tma_ok = tma_ok_for(lc.u, E, o.NP);
  cudaError_t e = o.set_smem(o.vol_smem(lc.epb));
  if (e != cudaSuccess) { free_single(c); return cuda_status(e); }
  e = cudaMemsetAsync(lc.st, 0, sizeof(DevState), c->stream);
  if (e == cudaSuccess && c->limited) e = cudaMemsetAsync(lc.alpha, 0, sizeof(double) * (size_t)E, c->stream);
  if (e == cudaSuccess && c->limited) e = cudaMemsetAsync(lc.tcount, 0, sizeof(unsigned), c->stream);
  if (e == cudaSuccess && c->fused) e = cudaMemsetAsync(lc.flags, 0, sizeof(unsigned) * (size_t)((E + 31) / 32), c->stream);
  if (e != cudaSuccess) { free_single(c); return cuda_status(e); }
  e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess && c->limited) e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
  if (e == cudaSuccess && c->limited) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess && c->limited) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
  if (e != cudaSuccess) { free_single(c); return cuda_status(e); }
  for (int p = 0; p < c->nphase && rc == CR_OK; ++p) {
    rc = capture(c, 1, p, &c->g1[p]);
    if (rc == CR_OK) rc = capture(c, 16, p, &c->g16[p]);
  }
  if (rc != CR_OK) { free_single(c); return rc; }
  return CR_OK;
}

extern "C" {

int cr_init_mesh(cr_ctx** out, const cr_mesh_desc* desc, int n_solves, void* cuda_stream) {
  NvtxRange range("cr_init_mesh");
  if (!out) return CR_EINVAL;
  *out = nullptr;
  if (!desc || n_solves < 1) return CR_EINVAL;
  for (int k = 0; k < n_solves; ++k)
    if (!desc_valid(desc[k])) return CR_EINVAL;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (prop.major != 10 || prop.minor != 3) return CR_ENODEV;   // built for sm_103a only
  cr_ctx* c = new (std::nothrow) cr_ctx();
  if (!c) return CR_ENOMEM;
  c->n_solves = n_solves;
  c->desc.assign(desc, desc + n_solves);
  c->stream = (cudaStream_t)cuda_stream;
  c->device = dev;
  int rc;
  if (n_solves == 1) {
    rc = init_single(c);
  } else {
    rc = batched_init(&c->batched, c->desc.data(), n_solves, c->stream);
  }
  if (rc != CR_OK) { delete c; return rc; }
  *out = c;
  return CR_OK;
}

int cr_workspace_bytes(const cr_mesh_desc* desc, size_t* bytes) {
  if (!desc || !bytes || !desc_valid(*desc)) return CR_EINVAL;
  cr_ctx tmp;
  tmp.n_solves = 1;
  tmp.desc.assign(desc, desc + 1);
  std::vector<BufSpec> plan;
  const int rc = plan_single(&tmp, &plan);
  if (rc != CR_OK) return rc;
  *bytes = plan_bytes(plan);
  return CR_OK;
}

int cr_init_mesh_ws(cr_ctx** out, const cr_mesh_desc* desc, void* workspace, size_t bytes, void* cuda_stream) {
  NvtxRange range("cr_init_mesh_ws");
  if (!out) return CR_EINVAL;
  *out = nullptr;
  if (!desc || !workspace || (reinterpret_cast<size_t>(workspace) & 255) != 0 || !desc_valid(*desc)) return CR_EINVAL;
  size_t need = 0;
  int rc = cr_workspace_bytes(desc, &need);
  if (rc != CR_OK) return rc;
  if (bytes < need) return CR_EINVAL;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  cudaPointerAttributes attr;
  e = cudaPointerGetAttributes(&attr, workspace);
  if (e != cudaSuccess || attr.type != cudaMemoryTypeDevice || attr.device != dev) return CR_EINVAL;
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (prop.major != 10 || prop.minor != 3) return CR_ENODEV;
  cr_ctx* c = new (std::nothrow) cr_ctx();
  if (!c) return CR_ENOMEM;
  c->n_solves = 1;
  c->desc.assign(desc, desc + 1);
  c->stream = (cudaStream_t)cuda_stream;
  c->device = dev;
  rc = init_single(c, workspace);
  if (rc != CR_OK) { delete c; return rc; }
  *out = c;
  return CR_OK;
}

int cr_state_size(const cr_ctx* c, int solve, int* n_vars, long long* n_nodes) {
  if (!c || solve < 0 || solve >= c->n_solves) return CR_EINVAL;
  if (c->batched) return batched_state_size(c->batched, solve, n_vars, n_nodes);
  if (n_vars) *n_vars = c->M;
  if (n_nodes) *n_nodes = c->E * c->NP;
  return CR_OK;
}

static int read_status(cr_ctx* c) {
  DevState h;
  CR_TRY(cudaMemcpyAsync(&h, c->lc.st, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CR_TRY(cudaStreamSynchronize(c->stream));
  if (h.status & ST_TIMEOUT) return CR_ETIMEOUT;
  if (h.status & ST_NONPHYS) return CR_ENONPHYSICAL;
  return CR_OK;
}

int cr_set_state(cr_ctx* c, int solve, const double* u, int u_on_device) {
  NvtxRange range("cr_set_state");
  if (!c || !u || solve < 0 || solve >= c->n_solves) return CR_EINVAL;
  if (c->batched) return batched_set_state(c->batched, solve, u, u_on_device);
  const size_t bytes = sizeof(double) * (size_t)c->M * c->E * c->NP;
  c->lc.u = state_buf(c, 0);
  CR_TRY(cudaMemcpyAsync(c->lc.u, u, bytes, u_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                         c->stream));
  CR_TRY(cudaMemsetAsync(c->lc.st, 0, sizeof(DevState), c->stream));
  if (c->fused) CR_TRY(cudaMemsetAsync(c->lc.flags, 0, sizeof(unsigned) * (size_t)((c->E + 31) / 32), c->stream));
  c->parity = 0;
  c->lc.slot = 0;
  CR_TRY(c->ops.lambda(c->lc, c->stream));
  int rc = read_status(c);
  c->has_state = (rc == CR_OK);
  return rc;
}

int cr_set_state_async(cr_ctx* c, int solve, const double* u, int u_on_device) {
  if (!c || !u || solve < 0 || solve >= c->n_solves) return CR_EINVAL;
  if (c->batched) return batched_set_state_async(c->batched, solve, u, u_on_device);
  const size_t bytes = sizeof(double) * (size_t)c->M * c->E * c->NP;
  c->lc.u = state_buf(c, 0);
  CR_TRY(cudaMemcpyAsync(c->lc.u, u, bytes, u_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                         c->stream));
  CR_TRY(cudaMemsetAsync(c->lc.st, 0, sizeof(DevState), c->stream));
  if (c->fused) CR_TRY(cudaMemsetAsync(c->lc.flags, 0, sizeof(unsigned) * (size_t)((c->E + 31) / 32), c->stream));
  c->parity = 0;
  c->lc.slot = 0;
  CR_TRY(c->ops.lambda(c->lc, c->stream));
  c->has_state = true;
  return CR_OK;
}

int cr_get_state_async(cr_ctx* c, int solve, double* u, int u_on_device) {
  if (!c || !u || solve < 0 || solve >= c->n_solves) return CR_EINVAL;
  if (c->batched) return batched_get_state_async(c->batched, solve, u, u_on_device);
  const size_t bytes = sizeof(double) * (size_t)c->M * c->E * c->NP;
  CR_TRY(cudaMemcpyAsync(u, state_buf(c, c->parity), bytes,
                         u_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  return CR_OK;
}

int cr_step(cr_ctx* c, int nsteps) {
  NvtxRange range("cr_step");
  if (!c || nsteps < 0) return CR_EINVAL;
  if (c->batched) return batched_step(c->batched, nsteps);
  if (!c->has_state) return CR_EINVAL;
  int k = 0;
  for (; k + 16 <= nsteps; k += 16) {
    CR_TRY(cudaGraphLaunch(c->g16[c->parity], c->stream));
    if (c->fused) c->parity = (c->parity + 16) % 3;   // the two-kernel parity is unchanged
  }
  for (; k < nsteps; ++k) {
    CR_TRY(cudaGraphLaunch(c->g1[c->parity], c->stream));
    c->parity = next_phase(c, c->parity);
    c->lc.u = state_buf(c, c->parity);
  }
  return CR_OK;
}

int cr_sync(cr_ctx* c) {
  if (!c) return CR_EINVAL;
  if (c->batched) return batched_sync(c->batched);
  return read_status(c);
}

int cr_get_state(cr_ctx* c, int solve, double* u, int u_on_device) {
  NvtxRange range("cr_get_state");
  if (!c || !u || solve < 0 || solve >= c->n_solves) return CR_EINVAL;
  if (c->batched) return batched_get_state(c->batched, solve, u, u_on_device);
  const size_t bytes = sizeof(double) * (size_t)c->M * c->E * c->NP;
  CR_TRY(cudaMemcpyAsync(u, state_buf(c, c->parity), bytes,
                         u_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  return read_status(c);
}

int cr_get_info(cr_ctx* c, int solve, double* t, double* dt, long long* steps, double* totals) {
  if (!c || solve < 0 || solve >= c->n_solves) return CR_EINVAL;
  if (c->batched) return batched_get_info(c->batched, solve, t, dt, steps, totals);
  DevState h;
  CR_TRY(cudaMemcpyAsync(&h, c->lc.st, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  std::vector<double> part;
  if (totals) {
    CR_TRY(c->ops.totals(c->lc, c->stream));
    part.resize(c->totals_blocks * (c->M + 2));
    CR_TRY(cudaMemcpyAsync(part.data(), c->lc.totals_part, sizeof(double) * part.size(), cudaMemcpyDeviceToHost,
                           c->stream));
  }
  CR_TRY(cudaStreamSynchronize(c->stream));
  if (t) *t = h.t;
  if (dt) *dt = h.dt;
  if (steps) *steps = h.steps;
  if (totals) {
    const int K = c->M + 2;
    for (int k = 0; k < K; ++k) totals[k] = 0.0;
    for (size_t b = 0; b < c->totals_blocks; ++b)
      for (int k = 0; k < K; ++k) totals[k] += part[b * K + k];
  }
  if (h.status & ST_TIMEOUT) return CR_ETIMEOUT;
  if (h.status & ST_NONPHYS) return CR_ENONPHYSICAL;
  return CR_OK;
}

int cr_time_kernels(cr_ctx* c, int nsteps, void* flush_buf, size_t flush_bytes, double* ms) {
  NvtxRange range("cr_time_kernels");
  if (!c || nsteps < 1 || !ms) return CR_EINVAL;
  if (c->batched) return batched_time_kernels(c->batched, nsteps, flush_buf, flush_bytes, ms);
  if (!c->has_state) return CR_EINVAL;
  // launches per step of each kind: 1, or one per RK stage (multi-stage RKFR)
  const bool rk = c->desc[0].scheme == CR_SCHEME_RKFR;
  const int S = rk ? rk_stages(c->desc[0].degree_N) : 1;
  std::vector<cudaEvent_t> ev(4 * (size_t)nsteps * S, nullptr);
  int rc = CR_OK;
  for (auto& e : ev)
    if (rc == CR_OK && cudaEventCreate(&e) != cudaSuccess) rc = CR_ECUDA;
  for (int k = 0; k < nsteps && rc == CR_OK; ++k) {
    if (flush_buf && flush_bytes && cudaMemsetAsync(flush_buf, k & 0xff, flush_bytes, c->stream) != cudaSuccess) {
      rc = CR_ECUDA;
      break;
    }
    c->lc.slot = c->parity;
    c->lc.u = state_buf(c, c->parity);
    c->lc.u_next = state_buf(c, c->parity ^ 1);
    if (c->fused) {
      // the single-launch step: ms[0] is the whole step, ms[1] = 0
      cudaEvent_t* e4 = &ev[4 * (size_t)k];
      cudaEventRecord(e4[0], c->stream);
      if (c->ops.step_fused(c->lc, c->stream, c->parity) != cudaSuccess) rc = CR_ECUDA;
      cudaEventRecord(e4[1], c->stream);
      cudaEventRecord(e4[2], c->stream);
      cudaEventRecord(e4[3], c->stream);
      if (rc == CR_OK) c->parity = next_phase(c, c->parity);
      continue;
    }
    for (int j = 0; j < S && rc == CR_OK; ++j) {
      cudaEvent_t* e4 = &ev[4 * ((size_t)k * S + j)];
      cudaEventRecord(e4[0], c->stream);
      // limiter: the coefficient kernels count with the volume kernel
      cudaError_t e = cudaSuccess;
      if (c->limited && c->ops.volume_ind) {
        e = c->ops.volume_ind(c->lc, c->stream);
        if (e == cudaSuccess) e = c->ops.alpha_smooth(c->lc, c->stream);
      } else {
        if (c->limited) e = c->ops.alpha(c->lc, c->stream);
        if (e == cudaSuccess)
          e = rk ? c->ops.volume_stage(c->lc, c->stream, j == 0 ? c->lc.u : c->lc.ustage, j == 0)
                 : c->ops.volume(c->lc, c->stream);
      }
      if (e != cudaSuccess) rc = CR_ECUDA;
      cudaEventRecord(e4[1], c->stream);
      cudaEventRecord(e4[2], c->stream);
      if (rc == CR_OK) {
        e = rk ? c->ops.face_stage(c->lc, c->stream, j, S)
               : (c->limited ? c->ops.face_limited(c->lc, c->stream) : c->ops.face_update(c->lc, c->stream));
        if (e != cudaSuccess) rc = CR_ECUDA;
      }
      cudaEventRecord(e4[3], c->stream);
    }
    if (rc == CR_OK) c->parity = next_phase(c, c->parity);
    c->lc.u = state_buf(c, c->parity);
  }
  if (rc == CR_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = CR_ECUDA;
  double tv = 0.0, tf = 0.0;
  for (size_t k = 0; k < (size_t)nsteps * S && rc == CR_OK; ++k) {
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, ev[4 * k + 0], ev[4 * k + 1]);
    cudaEventElapsedTime(&b, ev[4 * k + 2], ev[4 * k + 3]);
    tv += a;
    tf += b;
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  if (rc != CR_OK) return rc;
  ms[0] = tv / nsteps;
  ms[1] = c->fused ? 0.0 : tf / nsteps;
  return read_status(c);
}

int cr_get_blend_alpha(cr_ctx* c, double* alpha, int on_device) {
  if (!c || !alpha || c->batched || !c->limited) return CR_EINVAL;
  CR_TRY(cudaMemcpyAsync(alpha, c->lc.alpha, sizeof(double) * (size_t)c->E,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  CR_TRY(cudaStreamSynchronize(c->stream));
  return CR_OK;
}

int cr_destroy(cr_ctx* c) {
  if (!c) return CR_EINVAL;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  if (c->batched) batched_destroy(c->batched);
  else free_single(c);
  delete c;
  return CR_OK;
}

int cr_tuning_info(cr_ctx* c, char* buf, size_t len) {
  if (!c || !buf || len == 0) return CR_EINVAL;
  std::string info;
  if (c->batched) {
    info = batched_tuning(c->batched);
  } else {
    char tmp[256];
    std::snprintf(tmp, sizeof(tmp),
                  "{\"scheme\": \"%s\", \"step\": \"%s\", \"volume\": \"%s\", \"elements_per_cta\": %d, "
                  "\"face\": \"%s\"}",
                  c->desc[0].scheme == CR_SCHEME_RKFR ? "rkfr" : "crkfr", c->fused ? "fused" : "split",
                  c->ops.lanes ? "lanes" : "tile",
                  c->ops.lanes ? 32 : c->lc.epb,
                  c->limited ? "limited per-node" : (c->ops.threads_face > 0 ? "lanes" : "per-node"));
    info = tmp;
  }
  std::snprintf(buf, len, "%s", info.c_str());
  return info.size() < len ? CR_OK : CR_EINVAL;
}

const char* cr_status_string(int s) {
  switch (s) {
    case CR_OK: return "ok";
    case CR_EINVAL: return "invalid argument or mesh descriptor";
    case CR_ENOMEM: return "device allocation failed";
    case CR_ECUDA: return "CUDA runtime error";
    case CR_ENONPHYSICAL: return "non-physical state (rho <= 0, p <= 0 or non-finite)";
    case CR_ETIMEOUT: return "bounded device wait expired";
    case CR_ENODEV: return "no usable sm_103 CUDA device";
    case CR_ETOOLARGE: return "mesh exceeds the static scratch of cr_step_noalloc";
  }
  return "unknown status";
}

}  // extern "C"
