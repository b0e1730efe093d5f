// cr_batched.cu -- batched form: many independent solves advanced together.
//
// Solves of uneven mesh size and degree share one state buffer (and one
// scratch buffer each for Rbar and the face traces), sliced per solve, and one
// step record (dt, t, CFL reduction) per solve.  Per step, for every degree N
// present, one persistent volume kernel and then one persistent face/update
// kernel walk a work list of 32-element tiles spanning all solves of that
// degree.  Register allocation is per kernel, so a kernel per degree keeps the
// small degrees from running at the register count of N = 5.  The whole step
// (all degrees) is captured in CUDA graphs (1 and 8 steps) and replayed.
//
// Autotuning: before the first step, every candidate persistent grid
// (1 .. max resident CTAs per SM, times the SM count, and one CTA per tile) of
// every kernel is timed with CUDA events on the actual batch; the fastest is
// kept.  The state and step records are saved before and restored after the
// trials, so tuning does not advance the solution.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "cr_batched.h"
#include "cr_internal.h"

namespace crk {

struct BatchGroup {
  int N = 0;
  VariantOps ops{};
  std::vector<int> solves;
  BatchTile* d_tiles = nullptr;
  unsigned ntiles = 0;
  BatchLaunch vol{}, face{};
};

struct BatchedCtx {
  int n = 0, dev = 0, sms = 0;
  cudaStream_t stream = nullptr, cap = nullptr;
  std::vector<cr_mesh_desc> desc;
  std::vector<VariantOps> ops;
  std::vector<LaunchCtx> lc;
  std::vector<size_t> off_u;          // doubles
  std::vector<size_t> nvals;          // M * nodes per solve
  std::vector<bool> has_state;
  size_t total_u = 0, bytes_r = 0, bytes_t = 0;
  double* u = nullptr;
  char* rbar = nullptr;
  char* trace = nullptr;
  DevState* st = nullptr;
  double* totals_part = nullptr;
  size_t totals_blocks = 0;
  BatchSolve* d_solves = nullptr;
  std::vector<BatchGroup> groups;
  bool tuned = false;
  int parity = 0;     // slot of the CFL reductions of the current states (all solves step together)
  // graphs of 1 and 8 steps, one per starting parity
  cudaGraphExec_t g1[2] = {nullptr, nullptr}, g8[2] = {nullptr, nullptr};
  std::string tuning;
};

static int st_of(cudaError_t e) {
  if (e == cudaSuccess) return CR_OK;
  if (e == cudaErrorMemoryAllocation) return CR_ENOMEM;
  return CR_ECUDA;
}
#define BT(call)                          \
  do {                                    \
    cudaError_t _e = (call);              \
    if (_e != cudaSuccess) return st_of(_e); \
  } while (0)

static size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

static void free_all(BatchedCtx* b) {
  for (int p = 0; p < 2; ++p) {
    if (b->g1[p]) cudaGraphExecDestroy(b->g1[p]);
    if (b->g8[p]) cudaGraphExecDestroy(b->g8[p]);
  }
  if (b->cap) cudaStreamDestroy(b->cap);
  for (auto& g : b->groups) cudaFree(g.d_tiles);
  cudaFree(b->u);
  cudaFree(b->rbar);
  cudaFree(b->trace);
  cudaFree(b->st);
  cudaFree(b->totals_part);
  cudaFree(b->d_solves);
}

int batched_init(BatchedCtx** out, const cr_mesh_desc* desc, int n, cudaStream_t s) {
  *out = nullptr;
  // all solves take the single-stage scheme and share the system, dimension,
  // precision and volume flux
  for (int k = 0; k < n; ++k)
    if (desc[k].scheme != CR_SCHEME_CRKFR || desc[k].ncflux != CR_NCFLUX_REDUCED ||
        desc[k].limiter != CR_LIMITER_NONE)
      return CR_EINVAL;
  for (int k = 1; k < n; ++k)
    if (desc[k].eq != desc[0].eq || desc[k].dim != desc[0].dim || desc[k].prec != desc[0].prec ||
        desc[k].vol != desc[0].vol)
      return CR_EINVAL;
  BatchedCtx* b = new (std::nothrow) BatchedCtx();
  if (!b) return CR_ENOMEM;
  b->n = n;
  b->stream = s;
  b->desc.assign(desc, desc + n);
  cudaGetDevice(&b->dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->dev);
  b->ops.resize(n);
  b->lc.resize(n);
  b->off_u.resize(n);
  b->nvals.resize(n);
  b->has_state.assign(n, false);
  std::vector<size_t> off_r(n), off_t(n);
  for (int k = 0; k < n; ++k) {
    const cr_mesh_desc& d = desc[k];
    if (!get_ops(d.eq, d.dim, d.prec, d.vol, d.degree_N, &b->ops[k]) || !b->ops[k].vol_batched) {
      delete b;
      return CR_EINVAL;
    }
    const VariantOps& o = b->ops[k];
    fill_launch_ctx(d, o, &b->lc[k]);
    const long long E = b->lc[k].ma.E, nodes = E * o.NP;
    b->nvals[k] = (size_t)o.M * nodes;
    b->off_u[k] = b->total_u;
    b->total_u += (b->nvals[k] + 31) & ~(size_t)31;
    off_r[k] = b->bytes_r;
    b->bytes_r += a256(o.real_bytes * b->nvals[k]);
    off_t[k] = b->bytes_t;
    b->bytes_t += a256(o.real_bytes * (size_t)o.dim * 2 * o.C * (size_t)(E * o.NF));
    b->totals_blocks = std::max(b->totals_blocks, (size_t)((nodes + 255) / 256));
  }
  int rc = CR_OK;
  auto al = [&](void** p, size_t bytes) {
    if (rc == CR_OK && cudaMalloc(p, bytes) != cudaSuccess) rc = CR_ENOMEM;
  };
  al((void**)&b->u, sizeof(double) * b->total_u);
  al((void**)&b->rbar, b->bytes_r);
  al((void**)&b->trace, b->bytes_t);
  al((void**)&b->st, sizeof(DevState) * n);
  al((void**)&b->totals_part, sizeof(double) * b->totals_blocks * 11);
  al((void**)&b->d_solves, sizeof(BatchSolve) * n);
  if (rc != CR_OK) { free_all(b); delete b; return rc; }
  std::vector<BatchSolve> hs(n);
  for (int k = 0; k < n; ++k) {
    LaunchCtx& lc = b->lc[k];
    lc.u = b->u + b->off_u[k];
    lc.rbar = b->rbar + off_r[k];
    lc.trace = b->trace + off_t[k];
    lc.st = b->st + k;
    lc.totals_part = b->totals_part;
    lc.ma.tma_ok = tma_ok_for(lc.u, lc.ma.E, b->ops[k].NP);
    std::memset(&hs[k], 0, sizeof(BatchSolve));
    hs[k].ma = lc.ma;
    hs[k].u = lc.u;
    hs[k].rbar = lc.rbar;
    hs[k].trace = lc.trace;
    hs[k].st = lc.st;
    hs[k].ntiles = (unsigned)((lc.ma.E + 31) / 32);
    cudaError_t e = b->ops[k].set_smem(b->ops[k].vol_smem(lc.epb));
    if (e != cudaSuccess) { free_all(b); delete b; return st_of(e); }
  }
  // work lists per degree: tiles of all solves of that degree, largest solves first
  std::map<int, std::vector<int>> by_n;
  for (int k = 0; k < n; ++k) by_n[desc[k].degree_N].push_back(k);
  for (auto& kv : by_n) {
    BatchGroup g;
    g.N = kv.first;
    g.ops = b->ops[kv.second[0]];
    g.solves = kv.second;
    std::sort(g.solves.begin(), g.solves.end(), [&](int a, int c) { return b->lc[a].ma.E > b->lc[c].ma.E; });
    std::vector<BatchTile> tiles;
    for (int sidx : g.solves)
      for (unsigned t = 0; t < hs[sidx].ntiles; ++t) tiles.push_back(BatchTile{(unsigned)sidx, t * 32u});
    g.ntiles = (unsigned)tiles.size();
    if (cudaMalloc((void**)&g.d_tiles, sizeof(BatchTile) * tiles.size()) != cudaSuccess) rc = CR_ENOMEM;
    if (rc == CR_OK && cudaMemcpy(g.d_tiles, tiles.data(), sizeof(BatchTile) * tiles.size(), cudaMemcpyHostToDevice) !=
                           cudaSuccess)
      rc = CR_ECUDA;
    const LaunchCtx& l0 = b->lc[g.solves[0]];
    for (BatchLaunch* bl : {&g.vol, &g.face}) {
      bl->solves = b->d_solves;
      bl->tiles = g.d_tiles;
      bl->ntiles = g.ntiles;
      bl->pp64 = l0.pp64;
      bl->pp32 = l0.pp32;
      bl->tb64 = l0.tb64;
      bl->tb32 = l0.tb32;
    }
    // untuned default: one CTA per tile
    g.vol.grid = g.face.grid = (int)g.ntiles;
    g.vol.shape = g.face.shape = 0;
    b->groups.push_back(g);
    if (rc != CR_OK) break;
  }
  // physics parameters must agree within a degree group (gamma, c_h)
  for (auto& g : b->groups)
    for (int sidx : g.solves)
      if (b->desc[sidx].gamma != b->desc[g.solves[0]].gamma || b->desc[sidx].c_h != b->desc[g.solves[0]].c_h)
        rc = CR_EINVAL;
  if (rc == CR_OK && cudaMemcpy(b->d_solves, hs.data(), sizeof(BatchSolve) * n, cudaMemcpyHostToDevice) != cudaSuccess)
    rc = CR_ECUDA;
  if (rc == CR_OK && cudaMemset(b->st, 0, sizeof(DevState) * n) != cudaSuccess) rc = CR_ECUDA;
  if (rc == CR_OK && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) rc = CR_ECUDA;
  if (rc != CR_OK) { free_all(b); delete b; return rc; }
  *out = b;
  return CR_OK;
}

int batched_state_size(const BatchedCtx* b, int solve, int* n_vars, long long* n_nodes) {
  if (n_vars) *n_vars = b->ops[solve].M;
  if (n_nodes) *n_nodes = b->lc[solve].ma.E * b->ops[solve].NP;
  return CR_OK;
}

static int status_of(const DevState& h) {
  if (h.status & ST_TIMEOUT) return CR_ETIMEOUT;
  if (h.status & ST_NONPHYS) return CR_ENONPHYSICAL;
  return CR_OK;
}

int batched_set_state_async(BatchedCtx* b, int solve, const double* u, int on_device) {
  LaunchCtx& lc = b->lc[solve];
  BT(cudaMemcpyAsync(lc.u, u, sizeof(double) * b->nvals[solve],
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->stream));
  BT(cudaMemsetAsync(lc.st, 0, sizeof(DevState), b->stream));
  lc.slot = b->parity;
  BT(b->ops[solve].lambda(lc, b->stream));
  b->has_state[solve] = true;
  return CR_OK;
}

int batched_get_state_async(BatchedCtx* b, int solve, double* u, int on_device) {
  BT(cudaMemcpyAsync(u, b->lc[solve].u, sizeof(double) * b->nvals[solve],
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
  return CR_OK;
}

int batched_set_state(BatchedCtx* b, int solve, const double* u, int on_device) {
  LaunchCtx& lc = b->lc[solve];
  const int rc0 = batched_set_state_async(b, solve, u, on_device);
  if (rc0 != CR_OK) return rc0;
  DevState h;
  BT(cudaMemcpyAsync(&h, lc.st, sizeof(h), cudaMemcpyDeviceToHost, b->stream));
  BT(cudaStreamSynchronize(b->stream));
  const int rc = status_of(h);
  b->has_state[solve] = rc == CR_OK;
  return rc;
}

static void set_slot(BatchedCtx* b, int parity) {
  for (auto& g : b->groups) g.vol.slot = g.face.slot = parity;
}

// one step of every solve from the states whose CFL reductions sit in slot `parity`
static int launch_step(BatchedCtx* b, cudaStream_t s, int parity) {
  set_slot(b, parity);
  for (auto& g : b->groups) BT(g.ops.vol_batched(g.vol, s));
  for (auto& g : b->groups) BT(g.ops.face_batched(g.face, s));
  return CR_OK;
}

static int capture(BatchedCtx* b, int steps, int parity, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  BT(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  int rc = CR_OK;
  for (int k = 0; k < steps && rc == CR_OK; ++k) rc = launch_step(b, b->cap, (parity + k) & 1);
  cudaError_t e = cudaStreamEndCapture(b->cap, &g);
  if (rc != CR_OK) { if (g) cudaGraphDestroy(g); return rc; }
  if (e != cudaSuccess) return st_of(e);
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  return st_of(e);
}

// time one launch (ms) of a batched kernel on the context stream
static float time_launch(BatchedCtx* b, cudaError_t (*fn)(const BatchLaunch&, cudaStream_t), const BatchLaunch& bl,
                         cudaEvent_t t0, cudaEvent_t t1) {
  cudaEventRecord(t0, b->stream);
  if (fn(bl, b->stream) != cudaSuccess) return 1e30f;
  cudaEventRecord(t1, b->stream);
  if (cudaEventSynchronize(t1) != cudaSuccess) return 1e30f;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, t0, t1);
  return ms;
}

static int autotune(BatchedCtx* b) {
  // snapshot state and step records: the face trials advance them
  double* u_save = nullptr;
  DevState* st_save = nullptr;
  BT(cudaMalloc((void**)&u_save, sizeof(double) * b->total_u));
  if (cudaMalloc((void**)&st_save, sizeof(DevState) * b->n) != cudaSuccess) { cudaFree(u_save); return CR_ENOMEM; }
  cudaMemcpyAsync(u_save, b->u, sizeof(double) * b->total_u, cudaMemcpyDeviceToDevice, b->stream);
  cudaMemcpyAsync(st_save, b->st, sizeof(DevState) * b->n, cudaMemcpyDeviceToDevice, b->stream);
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  set_slot(b, b->parity);   // trials run as the next step; the snapshot is restored afterwards
  char buf[256];
  b->tuning = "{";
  int rc = CR_OK;
  for (size_t gi = 0; gi < b->groups.size() && rc == CR_OK; ++gi) {
    BatchGroup& g = b->groups[gi];
    for (int which = 0; which < 2; ++which) {
      BatchLaunch& bl = which == 0 ? g.vol : g.face;
      auto fn = which == 0 ? g.ops.vol_batched : g.ops.face_batched;
      // candidates: every kernel shape (volume) x every persistent grid of
      // 1 .. resident CTAs per SM times the SM count, and one CTA per tile
      const int shapes = which == 0 ? std::max(1, g.ops.vol_shapes) : 1;
      int best = (int)g.ntiles, best_shape = 0;
      float best_ms = 1e30f;
      for (int shape = 0; shape < shapes; ++shape) {
        bl.shape = shape;
        const int occ = std::max(1, g.ops.occupancy(which, shape));
        std::vector<int> cands;
        for (int c = 1; c <= occ; ++c) cands.push_back(std::min((int)g.ntiles, c * b->sms));
        cands.push_back((int)g.ntiles);
        std::sort(cands.begin(), cands.end());
        cands.erase(std::unique(cands.begin(), cands.end()), cands.end());
        for (int grid : cands) {
          bl.grid = grid;
          float ms = 1e30f;
          for (int rep = 0; rep < 3; ++rep) {   // first run warms up
            float t = time_launch(b, fn, bl, t0, t1);
            if (rep > 0) ms = std::min(ms, t);
            if (which == 1) {   // undo the update of the face trial
              cudaMemcpyAsync(b->u, u_save, sizeof(double) * b->total_u, cudaMemcpyDeviceToDevice, b->stream);
              cudaMemcpyAsync(b->st, st_save, sizeof(DevState) * b->n, cudaMemcpyDeviceToDevice, b->stream);
            }
          }
          if (ms < best_ms) { best_ms = ms; best = grid; best_shape = shape; }
        }
      }
      bl.grid = best;
      bl.shape = best_shape;
      std::snprintf(buf, sizeof(buf),
                    "%s\"N%d_%s\": {\"grid\": %d, \"ctas_per_sm\": %.2f, \"shape\": %d, \"ms\": %.4f, \"tiles\": %u}",
                    b->tuning.size() > 1 ? ", " : "", g.N, which == 0 ? "volume" : "face", best,
                    (double)best / b->sms, best_shape, best_ms, g.ntiles);
      b->tuning += buf;
    }
  }
  b->tuning += "}";
  cudaMemcpyAsync(b->u, u_save, sizeof(double) * b->total_u, cudaMemcpyDeviceToDevice, b->stream);
  cudaMemcpyAsync(b->st, st_save, sizeof(DevState) * b->n, cudaMemcpyDeviceToDevice, b->stream);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) rc = CR_ECUDA;
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaFree(u_save);
  cudaFree(st_save);
  if (cudaGetLastError() != cudaSuccess && rc == CR_OK) rc = CR_ECUDA;
  return rc;
}

static int ensure_ready(BatchedCtx* b) {
  for (int k = 0; k < b->n; ++k)
    if (!b->has_state[k]) return CR_EINVAL;
  if (b->tuned) return CR_OK;
  int rc = autotune(b);
  for (int p = 0; p < 2 && rc == CR_OK; ++p) {
    rc = capture(b, 1, p, &b->g1[p]);
    if (rc == CR_OK) rc = capture(b, 8, p, &b->g8[p]);
  }
  if (rc == CR_OK) b->tuned = true;
  return rc;
}

int batched_step(BatchedCtx* b, int nsteps) {
  int rc = ensure_ready(b);
  if (rc != CR_OK) return rc;
  int k = 0;
  for (; k + 8 <= nsteps; k += 8) BT(cudaGraphLaunch(b->g8[b->parity], b->stream));   // parity unchanged
  for (; k < nsteps; ++k) {
    BT(cudaGraphLaunch(b->g1[b->parity], b->stream));
    b->parity ^= 1;
  }
  return CR_OK;
}

int batched_sync(BatchedCtx* b) {
  std::vector<DevState> h(b->n);
  BT(cudaMemcpyAsync(h.data(), b->st, sizeof(DevState) * b->n, cudaMemcpyDeviceToHost, b->stream));
  BT(cudaStreamSynchronize(b->stream));
  int rc = CR_OK;
  for (auto& x : h) {
    const int r = status_of(x);
    if (r != CR_OK) rc = r;
  }
  return rc;
}

int batched_get_state(BatchedCtx* b, int solve, double* u, int on_device) {
  BT(cudaMemcpyAsync(u, b->lc[solve].u, sizeof(double) * b->nvals[solve],
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
  DevState h;
  BT(cudaMemcpyAsync(&h, b->lc[solve].st, sizeof(h), cudaMemcpyDeviceToHost, b->stream));
  BT(cudaStreamSynchronize(b->stream));
  return status_of(h);
}

int batched_get_info(BatchedCtx* b, int solve, double* t, double* dt, long long* steps, double* totals) {
  LaunchCtx& lc = b->lc[solve];
  DevState h;
  BT(cudaMemcpyAsync(&h, lc.st, sizeof(h), cudaMemcpyDeviceToHost, b->stream));
  const int M = b->ops[solve].M, K = M + 2;
  const size_t blocks = (size_t)((lc.ma.E * b->ops[solve].NP + 255) / 256);
  std::vector<double> part;
  if (totals) {
    BT(b->ops[solve].totals(lc, b->stream));
    part.resize(blocks * K);
    BT(cudaMemcpyAsync(part.data(), lc.totals_part, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, b->stream));
  }
  BT(cudaStreamSynchronize(b->stream));
  if (t) *t = h.t;
  if (dt) *dt = h.dt;
  if (steps) *steps = h.steps;
  if (totals) {
    for (int k = 0; k < K; ++k) totals[k] = 0.0;
    for (size_t blk = 0; blk < blocks; ++blk)
      for (int k = 0; k < K; ++k) totals[k] += part[blk * K + k];
  }
  return status_of(h);
}

int batched_time_kernels(BatchedCtx* b, int nsteps, void* flush, size_t bytes, double* ms) {
  int rc = ensure_ready(b);
  if (rc != CR_OK) return rc;
  cudaEvent_t e[3];
  for (auto& x : e) cudaEventCreate(&x);
  double tv = 0.0, tf = 0.0;
  for (int k = 0; k < nsteps && rc == CR_OK; ++k) {
    if (flush && bytes) cudaMemsetAsync(flush, k & 0xff, bytes, b->stream);
    set_slot(b, b->parity);
    cudaEventRecord(e[0], b->stream);
    for (auto& g : b->groups)
      if (g.ops.vol_batched(g.vol, b->stream) != cudaSuccess) rc = CR_ECUDA;
    cudaEventRecord(e[1], b->stream);
    for (auto& g : b->groups)
      if (g.ops.face_batched(g.face, b->stream) != cudaSuccess) rc = CR_ECUDA;
    cudaEventRecord(e[2], b->stream);
    if (cudaEventSynchronize(e[2]) != cudaSuccess) rc = CR_ECUDA;
    float a = 0.f, c = 0.f;
    cudaEventElapsedTime(&a, e[0], e[1]);
    cudaEventElapsedTime(&c, e[1], e[2]);
    tv += a;
    tf += c;
    if (rc == CR_OK) b->parity ^= 1;
  }
  for (auto& x : e) cudaEventDestroy(x);
  if (rc != CR_OK) return rc;
  ms[0] = tv / nsteps;
  ms[1] = tf / nsteps;
  return batched_sync(b);
}

const char* batched_tuning(const BatchedCtx* b) { return b->tuning.c_str(); }

void batched_destroy(BatchedCtx* b) {
  if (!b) return;
  free_all(b);
  delete b;
}

}  // namespace crk
