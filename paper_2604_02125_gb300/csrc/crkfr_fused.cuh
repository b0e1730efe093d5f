// crkfr_fused.cuh -- the whole cRKFR step of one solve in one persistent,
// cooperative launch (sm_103a): the element-volume work of every tile (eqs.
// crkfr.inner, entropy.cons.flux.dev, disc.avg.flux) and the single
// inter-element step with the final update (eqs. numflux.cons,
// crkfr.non.cons.final) of every tile, so that the memory- and FP64-bound
// update of finished tiles overlaps the FP32- (or FP64-) bound volume work of
// others on the same SM.
//
// Schedule.  CTA b computes the volume tiles b, b + G, ... (G = grid, every
// CTA resident: cooperative launch) exactly as the persistent volume kernel
// does, TMA prefetch included.  After each tile it publishes the tile's
// readiness value (release), and then runs the face / update work of any of
// its own earlier tiles whose records are complete: the tile's own and those
// of every tile holding a face neighbour of one of its elements (acquire; a
// single non-blocking check).  Only after its last volume tile does a CTA wait
// (bounded) for the tiles still pending, so no CTA waits while it still owes
// volume work to others: with all CTAs resident every wait ends.  A wait that
// expires sets CR_ETIMEOUT's status bit and skips that tile.
//
// In-place update: a tile's face work writes u^{n+1} over its own u^n after
// its own volume work has read u^n, and the volume work of a tile reads only
// its own u^n, so no tile reads a state another tile has already advanced.
//
// The CFL reduction: the wave-speed maximum of u^{n+1} goes to lam_bits[w]
// while the step reads lam_bits[r] and its lead CTA clears lam_bits[c],
// (r, w, c) = (phase, phase + 1, phase + 2) mod 3: a clear and reductions of
// the same slot never share a launch.  The readiness value of a step is
// epoch[r] + 1, recorded by the lead in epoch[w] for the next step; cr_set_state
// clears the records, the slots and the flags together.
#pragma once
#include "crkfr_volume_lanes.cuh"

namespace crk {

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// polls of a bounded readiness wait (each after a short sleep): well beyond
// any legitimate wait, which is a fraction of one step
constexpr unsigned kFusedWaitPolls = 1u << 22;

// Whether the face / update work of tile t may start: the readiness value of
// t and of the tiles of all face neighbours of its elements has reached
// epoch.  Warp 0 checks (one lane per element), the CTA gets the verdict.
// block: wait (bounded) instead of a single check; on expiry the timeout bit
// is set and false returned.  Called by every thread of the CTA.
template <int DIM>
__device__ __forceinline__ bool tile_ready(const unsigned* flags, unsigned t, unsigned epoch, const MeshArgs& ma,
                                           DevState* st, bool block, int* s_flag) {
  if (threadIdx.x < 32) {
    const long long e = (long long)t * 32 + threadIdx.x;
    unsigned need[2 * DIM + 1];
    int nn = 0;
    need[nn++] = t;
    if (e < ma.E) {
      unsigned c[3] = {0, 0, 0};
      elem_coords<DIM>((unsigned)e, ma, c);
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        need[nn++] = neighbour_of((unsigned)e, c, d, +1, ma) >> 5;
        need[nn++] = neighbour_of((unsigned)e, c, d, -1, ma) >> 5;
      }
    }
    bool ok = true;
    for (int k = 0; k < nn; ++k) ok = ok && ld_acquire_u32(flags + need[k]) >= epoch;
    bool all = __all_sync(0xffffffffu, ok);
    bool expired = false;
    if (block && !all) {
      for (unsigned it = 0; it < kFusedWaitPolls && !all; ++it) {
        __nanosleep(64);
        ok = true;
        for (int k = 0; k < nn; ++k) ok = ok && ld_acquire_u32(flags + need[k]) >= epoch;
        all = __all_sync(0xffffffffu, ok);
      }
      expired = !all;
    }
    if (threadIdx.x == 0) {
      *s_flag = all ? 1 : 0;
      if (expired) atomicOr(&st->status, ST_TIMEOUT);
    }
  }
  __syncthreads();
  const bool r = *s_flag != 0;
  __syncthreads();   // s_flag is reused by the next check
  return r;
}

template <class EQ, int N, typename R>
struct FusedLayout {
  using L = LaneLayout<EQ, N, R>;
  using PL = PersistLayout<EQ, N, R>;
  using FL = FaceLaneLayout<EQ, N, R>;
  // the face work of a tile uses the lane layout's region for its jumps
  static constexpr bool fits() { return PL::fits() && FL::fits() && FL::bytes() <= L::bytes() && FL::THREADS == L::THREADS; }
  static constexpr size_t bytes() { return PL::bytes(); }
};

template <class EQ, int N, typename R>
__global__ void __launch_bounds__(LaneLayout<EQ, N, R>::THREADS, LaneLayout<EQ, N, R>::MINB)
k_step_fused(double* u, R* rbar, R* trace, DevState* st, unsigned* flags, const MeshArgs ma, const PhysParams<R> pp,
             const RefTab<R> tb, int phase) {
  using PL = PersistLayout<EQ, N, R>;
  constexpr int M = EQ::M, NP = LaneLayout<EQ, N, R>::NP, DIM = EQ::DIM;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);
  double* staging = reinterpret_cast<double*>(smem_raw + PL::O_STAGE);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw + PL::O_BAR);
  const int rs = phase, ws = (phase + 1) % 3, cs = (phase + 2) % 3;
  const long long E = ma.E;
  const unsigned ntiles = (unsigned)((E + 31) / 32);
  auto whole = [&](unsigned t) { return PL::STAGE && ma.tma_ok && (long long)(t + 1) * 32 <= E; };
  auto pf_of = [&](unsigned t) {
    return Prefetch{u + (size_t)t * 32 * NP, E * NP, (unsigned)(32 * NP * sizeof(double)), staging, bar};
  };
  __shared__ double s_dt;
  __shared__ unsigned s_epoch;
  __shared__ int s_flag;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    const bool lead = blockIdx.x == 0;
    s_dt = step_begin_slots(st, rs, cs, ma.cfl, ma.dt_fixed, lead);
    s_epoch = st->epoch[rs] + 1u;
    if (lead) st->epoch[ws] = s_epoch;
  }
  __syncthreads();
  const R dtR = dt_as<R>(s_dt);
  const unsigned epoch = s_epoch;
  const unsigned G = gridDim.x;
  // this CTA's tiles: t_k = blockIdx.x + k G; face work done for k < 64 in `done`
  const unsigned K = blockIdx.x < ntiles ? (ntiles - blockIdx.x + G - 1) / G : 0;
  unsigned long long done = 0ull;
  auto face = [&](unsigned t) {
    face_lanes_tile<EQ, N, R, false, true>(u, rbar, trace, st, ma, pp, tb, t * 32u, ws, sm,
                                           RkStage<R>{nullptr, nullptr, 0, 1}, dtR);
    __syncthreads();   // the jump buffer is the volume tile's region
  };

  unsigned phase_bar = 0;
  unsigned t = blockIdx.x;
  if (t < ntiles && whole(t) && threadIdx.x == 0) issue_prefetch<M>(pf_of(t));
  for (unsigned k = 0; k < K; ++k, t += G) {
    const bool staged = whole(t);
    if (staged) {
      const bool ok = mbar_wait_bounded(bar, phase_bar);
      if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
          atomicOr(&st->status, ST_TIMEOUT);
          mbar_wait_bounded(bar, phase_bar);
        }
        return;
      }
      phase_bar ^= 1u;
    }
    const unsigned tn = t + G;
    const Prefetch pf = (tn < ntiles && whole(tn)) ? pf_of(tn) : Prefetch{nullptr, 0, 0, nullptr, nullptr};
    volume_lanes_tile<EQ, N, R, 0, 0, true>(u, rbar, trace, st, ma, pp, tb, (long long)t * 32, dtR, sm,
                                      staged ? staging : nullptr, pf);
    // publish: every thread's records and R-bar are visible device-wide
    // before the readiness value
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) st_release_u32(flags + t, epoch);
    // face / update work of earlier own tiles whose neighbours are complete
    for (unsigned j = 0; j < k && j < 64; ++j) {
      if (done >> j & 1ull) continue;
      const unsigned tj = blockIdx.x + j * G;
      if (tile_ready<DIM>(flags, tj, epoch, ma, st, false, &s_flag)) {
        face(tj);
        done |= 1ull << j;
      }
    }
  }
  // the rest, in order, waiting (bounded) for the neighbours
  for (unsigned j = 0; j < K; ++j) {
    if (j < 64 && (done >> j & 1ull)) continue;
    const unsigned tj = blockIdx.x + j * G;
    if (tile_ready<DIM>(flags, tj, epoch, ma, st, true, &s_flag)) face(tj);
  }
}

}  // namespace crk
