// crkfr_kernels.cuh -- shared pieces of the cRKFR step kernels on sm_103a,
// and the general (tile-form) kernels that serve the variants whose lane form
// (crkfr_volume_lanes.cuh) does not fit in shared memory.
//
//  k_volume_tile  element-local cRK stages (eq. crkfr.inner) with the
//                 flux-differencing local residual (Sec. 3, eqs.
//                 entropy.cons.flux.dev, entropy.cons.noncons.dev), the
//                 b-weighted volume residual of the final update (Sec. 3,
//                 time-averaged flux differencing), and the face traces of the
//                 time averages U, F (eq. disc.avg.flux), F^nc (Sec. 2.3) and
//                 of lambda(u^n).  One CTA holds `epb` elements in shared
//                 memory; one thread per line (N+1 nodes along a direction).
//  k_face_update  the single inter-element step, one thread per node: per face
//                 node one time-averaged Rusanov flux (eq. numflux.cons) and
//                 the reduced-communication non-conservative flux
//                 B(u^{n,+-}) g^avg(U) (Sec. 2.3), applied through the g2
//                 correction derivatives g_R'(1) = 1/w_N, g_L'(0) = -1/w_0
//                 (GLL + g2) in the FP64 update (eq. crkfr.non.cons.final);
//                 then the CFL reduction of the new state and the
//                 physicality flag.
//  k_lambda       CFL reduction of a state (first step after set_state).
//  k_totals       FP64 quadrature-weighted totals (diagnostics).
// Shared: the mesh and reference-element parameters, the step record and its
// fence-free CFL protocol (reduce_lambda / step_begin), element coordinates
// and periodic neighbours, the face-record layout and the Rusanov jump.
//
// Layouts in HBM:
//   u     [M][E][NP] FP64        state, updated in place by k_face_update
//   rbar  [M][E][NP] R           sum_i b_i R(u^(i))
//   trace [DIM][2][NF][C][E] R   face data; side 0 = xi_d = 0 face, side 1 = xi_d = 1;
//         per face node C components, each contiguous over the elements
//         (a warp's 32 consecutive elements load one 128-byte line):
//         U (M), F^d (M), lambda_d(u^n) (1) [+ GLM-MHD: F^nc,d (M), u^n (M)]
#pragma once
#include "crkfr_async.cuh"
#include "crkfr_physics.cuh"

namespace crk {

// Division of n < 2^31 by an invariant d >= 1 with one wide multiply:
// q = (n * m) >> (32 + l), l = ceil(log2 d), m = ceil(2^(32+l) / d) < 2^33.
// With m = 2^(32+l)/d + eps, 0 <= eps < 1, the quotient is n/d + n eps / 2^(32+l)
// and n eps / 2^(32+l) < 2^31 / 2^(32+l) <= 1/(2d), too small to change floor(n/d).
struct FastDiv {
  unsigned long long m;
  unsigned shift;   // 32 + l
  unsigned d;
};
__host__ __device__ inline FastDiv make_fastdiv(unsigned d) {
  unsigned l = 0;
  while ((1ull << l) < d) ++l;
  FastDiv f;
  f.d = d;
  f.shift = 32 + l;
  f.m = (((1ull << (32 + l)) + d - 1) / d);
  return f;
}
__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv& f) {
  return (unsigned)(((unsigned long long)n * f.m) >> f.shift);
}

struct MeshArgs {
  long long E;          // elements; E * (N+1)^dim < 2^31 nodes per solve
  int cells[3];
  FastDiv cdiv[3];      // division by cells[k]
  double inv_dx[3];
  double cfl, dt_fixed;
  double gamma, c_h;
  float inv_dx_f[3], gamma_f, c_h_f;   // FP32 copies (no conversions on the FP64 pipe)
  int tma_ok;           // state base 16-byte aligned and E * NP even: whole tiles can be bulk-copied
};
template <typename R> __device__ __forceinline__ R inv_dx_of(const MeshArgs& ma, int d);
template <> __device__ __forceinline__ double inv_dx_of<double>(const MeshArgs& ma, int d) { return ma.inv_dx[d]; }
template <> __device__ __forceinline__ float inv_dx_of<float>(const MeshArgs& ma, int d) { return ma.inv_dx_f[d]; }

template <typename R>
struct RefTab {
  R D[6][6];       // D_pq = l_q'(xi_p) on [0,1]
  R iw0, iwN;      // 1/w_0, 1/w_N
  double w[6];     // quadrature weights (FP64, diagnostics)
  R a[7][7], b[7]; // Butcher tableau of the degree (same values as rk_a / rk_b)
  signed char slot[7];   // register slot of a stage residual needed beyond the next stage, else -1
  // (2 D_pq, 2 D_pq) in FP32: the coefficients of the packed FP32x2 pair loop
  // as ready register pairs (measured 53.8 -> 52.5 us per volume launch, 2D
  // Euler 256^2, N = 3, against forming them from D_pq in the loop)
  float2 D2f[6][6];
  // (2 D_pq / dx, 2 D_pq / dy) of one solve: a single solve's packed pair loop
  // folds the 1/dx scaling of its two lines into the coefficients (measured
  // 52.7 -> 51.4 us per volume launch, 2D Euler 256^2, N = 3); the batched
  // kernels, which share one table among solves of different sizes, scale
  float2 D2s[6][6];
};

// Step record of one solve.  The CFL reduction needs no fence and no
// ticket: the wave-speed maximum of a state is accumulated by fire-and-forget
// atomics into lam_bits[slot], where slot alternates with the step parity
// (the host passes it to every kernel); the volume kernel of the step that
// starts from that state reads it (kernel boundaries order the two), derives
// dt, records the step and clears the other slot for the new state.
// The fused single-launch step (crkfr_fused.cuh) reduces into a third slot: it
// rotates read / write / clear slots modulo 3, because its clear and its
// reductions happen within one launch.  epoch[] carries its per-step tile
// readiness value the same way.
// Each slot is spread over kLamSpread words: warp w of CTA b reduces into word
// (b NW + w) mod kLamSpread, and the step start takes the maximum of the
// words -- thousands of warps' atomics on a single word would serialise.
constexpr int kLamSpread = 32;
struct DevState {
  unsigned long long lam_bits[3][kLamSpread];   // max over nodes of sum_d lambda_d / dx_d (bits of a non-negative double)
  unsigned epoch[3];   // fused step: readiness value of the step that starts from a slot
  unsigned pad0;
  double dt;           // dt of the last step (set when the step starts)
  double t;            // time after the last step
  double lam_max;      // wave-speed maximum the last step's dt came from
  long long steps;
  unsigned status;     // bit 0: non-physical state, bit 1: barrier timeout
  unsigned pad;
};

constexpr unsigned ST_NONPHYS = 1u, ST_TIMEOUT = 2u;

// One stage of the multi-stage RKFR step (eq. rkfr.non.cons), for the face /
// update kernels in stage mode.  Stage j (0-based) of s forms the increment
// K_j = -dt R_FR(u^(j)) at every node and combines it with the earlier ones:
// u^(j+1) = u^n + sum_{q<=j} a_{j+1,q} K_q into uout, or, at the last stage,
// u^{n+1} = u^n + sum_q b_q K_q into the state (followed by the CFL
// reduction).  k holds K_0..K_{s-2}, [stage][var][elem][node].
template <typename R>
struct RkStage {
  R* k;
  double* uout;
  int j, s;
};

// ---------------------------------------------------------------------------
// CFL reduction: every warp takes its maximum with shuffles and folds it into
// its word of lam_bits[slot] with one 64-bit atomicMax (non-negative doubles order like
// their bit patterns; the result is not waited for).  Must be reached by every
// lane of the warp.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void reduce_lambda(T lam, bool bad, DevState* st, int slot) {
  for (int o = 16; o > 0; o >>= 1) lam = fmax(lam, __shfl_xor_sync(0xffffffffu, lam, o));
  const unsigned anybad = __ballot_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    if (anybad) atomicOr(&st->status, ST_NONPHYS);
    // a warp whose lanes did no work (maximum 0) leaves the slot alone: the
    // atomics of thousands of idle warps on one word would serialise
    if (lam > T(0)) {
      const unsigned word = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) % kLamSpread;
      atomicMax(&st->lam_bits[slot][word], (unsigned long long)__double_as_longlong((double)lam));
    }
  }
}

// dt of the step that starts now, from the wave-speed maximum of its initial
// state: cfl / max_nodes sum_d lambda_d/dx_d, or the fixed dt.  Every caller
// computes the same value; the one with lead set (one per solve and launch)
// records the step and clears the other slot for the new state's reduction.
__device__ __forceinline__ double step_begin_slots(DevState* st, int slot, int clear_slot, double cfl, double dt_fixed,
                                                   bool lead) {
  // all words loaded at once (one round trip), then reduced
  unsigned long long w[kLamSpread];
#pragma unroll
  for (int k = 0; k < kLamSpread; ++k) w[k] = st->lam_bits[slot][k];
  unsigned long long bits = 0ull;
#pragma unroll
  for (int k = 0; k < kLamSpread; ++k) bits = max(bits, w[k]);
  const double lam = __longlong_as_double((long long)bits);
  const double dt = dt_fixed > 0.0 ? dt_fixed : cfl / lam;
  if (lead) {
#pragma unroll 8
    for (int k = 0; k < kLamSpread; ++k) st->lam_bits[clear_slot][k] = 0ull;
    st->dt = dt;
    st->t += dt;
    st->steps += 1;
    st->lam_max = lam;
    if (!(lam > 0.0) || !isfinite(lam)) atomicOr(&st->status, ST_NONPHYS);
  }
  return dt;
}
__device__ __forceinline__ double step_begin(DevState* st, int slot, double cfl, double dt_fixed, bool lead) {
  return step_begin_slots(st, slot, slot ^ 1, cfl, dt_fixed, lead);
}


// Loads of data another CTA wrote earlier in the same launch (fused step):
// through L2 (ld.global.cg), never the non-coherent path or a stale L1 line.
template <bool COH, typename T>
__device__ __forceinline__ T ldx(const T* p) {
  if constexpr (COH) return __ldcg(p);
  else return *p;
}

// the current step's dt in the path's arithmetic (face kernels, after the
// volume kernel of the same step has recorded it)
template <typename R>
__device__ __forceinline__ R dt_as(double dt) {
  if constexpr (sizeof(R) == 4) return d2f_int(dt);
  else return dt;
}
template <typename R>
__device__ __forceinline__ R step_dt(const DevState* st) {
  return dt_as<R>(st->dt);
}


template <class EQ>
__host__ __device__ constexpr int trace_comps() { return EQ::NC ? 4 * EQ::M + 1 : 2 * EQ::M + 1; }
// component c of the record of face node f of face (d, side) of element e
template <class EQ, int NF>
__host__ __device__ __forceinline__ size_t trace_index(int d, int side, int f, int c, long long E, long long e) {
  return ((((size_t)(d * 2 + side) * NF + f) * trace_comps<EQ>() + c) * (size_t)E) + (size_t)e;
}
// Stage-wise non-conservative flux (EQ::NCS): after the records, the seven
// primitives of every stage's face trace, [DIM][2][NF][stage][7][E].
template <class EQ, int N>
__host__ __device__ constexpr size_t ncs_values_per_elem() {
  return (size_t)EQ::DIM * 2 * (ipow(N + 1, EQ::DIM) / (N + 1)) * rk_stages(N) * 7;
}
template <class EQ, int N>
__host__ __device__ __forceinline__ size_t ncs_index(int d, int side, int f, int j, int c, long long E, long long e) {
  constexpr int NF = ipow(N + 1, EQ::DIM) / (N + 1), S = rk_stages(N);
  const size_t base = (size_t)EQ::DIM * 2 * NF * trace_comps<EQ>() * (size_t)E;
  return base + (((((size_t)(d * 2 + side) * NF + f) * S + j) * 7 + c) * (size_t)E) + (size_t)e;
}
// the primitives of stage j at face node f of face (d, side) of element e
template <class EQ, int N, typename R>
__device__ __forceinline__ void write_stage_prims(R* __restrict__ trace, int d, int side, int f, int j, long long E,
                                                  long long e, const R* q) {
  if constexpr (EQ::NCS) {
    R w[7];
    EQ::stage_prims(q, w);
#pragma unroll
    for (int c = 0; c < 7; ++c) trace[ncs_index<EQ, N>(d, side, f, j, c, E, e)] = w[c];
  }
}

template <class EQ, int N, typename R>
struct VolLayout {
  static constexpr int DIM = EQ::DIM, M = EQ::M, P = EQ::P, n = N + 1;
  static constexpr int NP = ipow(n, DIM), NF = NP / n, S = rk_stages(N);
  static constexpr int O_U0 = 0;
  static constexpr int O_Q = O_U0 + M * NP;
  static constexpr int O_RS = O_Q + P * NP;
  static constexpr int O_UB = O_RS + S * M * NP;
  static constexpr int O_FB = O_UB + M * NP;
  static constexpr int O_FN = O_FB + DIM * M * NP;
  static constexpr int O_LAM = O_FN + (EQ::NC ? DIM * M * NP : 0);
  static constexpr int SZ = O_LAM + DIM * NP;    // elements of R per mesh element
  static constexpr size_t bytes_per_elem() { return sizeof(R) * (size_t)SZ; }
};

// node index of the first node of line l in direction d, and its stride
template <int n>
__device__ __forceinline__ int line_base(int l, int stride) { return (l % stride) + (l / stride) * stride * n; }

// element coordinates (x fastest) of element e
template <int DIM>
__device__ __forceinline__ void elem_coords(unsigned e, const MeshArgs& ma, unsigned (&c)[3]) {
  unsigned r = e;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    const unsigned q = (k == DIM - 1) ? 0u : fdiv(r, ma.cdiv[k]);
    c[k] = (k == DIM - 1) ? r : r - q * (unsigned)ma.cells[k];
    r = q;
  }
}
// periodic neighbour of element e (coordinates c) in direction d, offset +-1
__device__ __forceinline__ unsigned neighbour_of(unsigned e, const unsigned (&c)[3], int d, int off,
                                                 const MeshArgs& ma) {
  unsigned stride = 1;
  for (int k = 0; k < d; ++k) stride *= (unsigned)ma.cells[k];
  const unsigned nd = (unsigned)ma.cells[d];
  if (off > 0) return c[d] + 1 == nd ? e - (nd - 1) * stride : e + stride;
  return c[d] == 0 ? e + (nd - 1) * stride : e - stride;
}

// ---------------------------------------------------------------------------
// Volume kernel, tile form: one CTA holds epb elements; one thread per line.
// Used where the lane form below does not fit in shared memory.
// ---------------------------------------------------------------------------
// S1 = 1: a single stage with b = 1 (R-bar = R(u), face records of u), the
// volume part of one stage of the multi-stage RKFR step; first = false takes
// the dt the step's first launch recorded.
template <class EQ, int N, typename R, int S1>
__device__ __forceinline__ void volume_tile_body(const double* __restrict__ u, R* __restrict__ rbar,
                                                 R* __restrict__ trace, DevState* __restrict__ st, const MeshArgs& ma,
                                                 const PhysParams<R>& pp, const RefTab<R>& tb, int slot, bool first) {
  using L = VolLayout<EQ, N, R>;
  constexpr int DIM = L::DIM, M = L::M, P = L::P, n = L::n, NP = L::NP, NF = L::NF, S = S1 ? S1 : L::S;
  constexpr int C = trace_comps<EQ>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);

  const int NT = blockDim.x;
  const int epb = NT / NF;
  const int tid = threadIdx.x;
  const long long E = ma.E;
  const long long e0 = (long long)blockIdx.x * epb;
  const int nel = (int)min((long long)epb, E - e0);
  const int el = tid / NF, l = tid % NF;
  const bool active = el < nel;
  R* my = sm + (size_t)el * L::SZ;

  __shared__ double s_dt;
  if (tid == 0) s_dt = first ? step_begin(st, slot, ma.cfl, ma.dt_fixed, blockIdx.x == 0) : st->dt;
  __syncthreads();
  const R dtR = dt_as<R>(s_dt);

  // u^n -> shared memory (coalesced over [v][e0..e0+nel)[p])
#pragma unroll 1
  for (int v = 0; v < M; ++v)
    for (int r = tid; r < nel * NP; r += NT) {
      const int ee = r / NP, p = r % NP;
      sm[(size_t)ee * L::SZ + L::O_U0 + v * NP + p] = (R)u[((size_t)v * E + e0) * NP + r];
    }
  __syncthreads();

#pragma unroll
  for (int i = 0; i < S; ++i) {
    // ---- node phase: stage state u^(i), pair data, time-average face sums
    if (active) {
#pragma unroll
      for (int k = 0; k < n; ++k) {
        const int p = l * n + k;
        R uu[M];
#pragma unroll
        for (int v = 0; v < M; ++v) {
          R acc = R(0);
#pragma unroll
          for (int j = 0; j < i; ++j)
            if (rk_a(N, i, j) != 0.0) acc += R(rk_a(N, i, j)) * my[L::O_RS + (j * M + v) * NP + p];
          uu[v] = my[L::O_U0 + v * NP + p] - dtR * acc;
        }
        R q[P];
        EQ::pair_data(uu, q, pp);
#pragma unroll
        for (int c = 0; c < P; ++c) my[L::O_Q + c * NP + p] = q[c];
        if constexpr (EQ::NCS) {
          // face traces of this stage (stage-wise non-conservative flux)
          int rq = p;
#pragma unroll
          for (int d = 0; d < DIM; ++d) {
            const int cq = rq % n;
            rq /= n;
            const int stride = ipow(n, d);
            if (cq == 0 || cq == N)
              write_stage_prims<EQ, N, R>(trace, d, cq == N ? 1 : 0, (p % stride) + (p / (stride * n)) * stride, i, E,
                                          e0 + el, q);
          }
        }
#pragma unroll
        for (int v = 0; v < M; ++v) my[L::O_RS + (i * M + v) * NP + p] = R(0);
        // which faces this node lies on
        int rem = p;
        bool onface = false;
        int cd[3] = {0, 0, 0};
#pragma unroll
        for (int d = 0; d < DIM; ++d) { cd[d] = rem % n; rem /= n; onface = onface || cd[d] == 0 || cd[d] == N; }
        if (i == 0) {
#pragma unroll
          for (int d = 0; d < DIM; ++d)
            if (cd[d] == 0 || cd[d] == N) my[L::O_LAM + d * NP + p] = EQ::wave_speed(d, q, pp);
        }
        const double bi = S1 ? 1.0 : rk_b(N, i);
        if (bi != 0.0 && onface) {
          const R b = R(bi);
#pragma unroll
          for (int v = 0; v < M; ++v) {
            R* ub = &my[L::O_UB + v * NP + p];
            *ub = (i == 0 ? R(0) : *ub) + b * uu[v];
          }
#pragma unroll
          for (int d = 0; d < DIM; ++d) {
            if (cd[d] == 0 || cd[d] == N) {
              R f[M];
              EQ::flux(d, q, f, pp);
#pragma unroll
              for (int v = 0; v < M; ++v) {
                R* fb = &my[L::O_FB + (d * M + v) * NP + p];
                *fb = (i == 0 ? R(0) : *fb) + b * f[v];
              }
              if constexpr (EQ::NC) {
                R g[2], nc[M];
#pragma unroll
                for (int v = 0; v < M; ++v) nc[v] = R(0);
                EQ::ncg(d, q, g);
                EQ::nc_apply(d, q, g, nc);
#pragma unroll
                for (int v = 0; v < M; ++v) {
                  R* fn = &my[L::O_FN + (d * M + v) * NP + p];
                  *fn = (i == 0 ? R(0) : *fn) + b * nc[v];
                }
              }
            }
          }
        }
      }
    }
    __syncthreads();

    // ---- line phase: flux differencing along each direction
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      if (active) {
        constexpr int dummy = 0;
        (void)dummy;
        const int stride = ipow(n, d);
        const int base = line_base<n>(l, stride);
        R q[n][P];
#pragma unroll
        for (int k = 0; k < n; ++k)
#pragma unroll
          for (int c = 0; c < P; ++c) q[k][c] = my[L::O_Q + c * NP + base + k * stride];
        R acc[n][M];
#pragma unroll
        for (int k = 0; k < n; ++k)
#pragma unroll
          for (int v = 0; v < M; ++v) acc[k][v] = R(0);
        // D_pp f(u_p): non-zero only at the two end points of a GLL line
        {
          R f[M];
          EQ::flux(d, q[0], f, pp);
#pragma unroll
          for (int v = 0; v < M; ++v) acc[0][v] += R(2) * tb.D[0][0] * f[v];
          EQ::flux(d, q[N], f, pp);
#pragma unroll
          for (int v = 0; v < M; ++v) acc[N][v] += R(2) * tb.D[N][N] * f[v];
        }
        // every pair once: f_S is symmetric
#pragma unroll
        for (int a = 0; a < n; ++a)
#pragma unroll
          for (int b = a + 1; b < n; ++b) {
            R f[M];
            EQ::two_point(d, q[a], q[b], f, pp);
            const R dab = R(2) * tb.D[a][b], dba = R(2) * tb.D[b][a];
#pragma unroll
            for (int v = 0; v < M; ++v) { acc[a][v] += dab * f[v]; acc[b][v] += dba * f[v]; }
          }
        if constexpr (EQ::NC) {
          // sum_q D_pq B(u_p) g(u_q) = B(u_p) (D g)_p (no factor 2)
#pragma unroll
          for (int a = 0; a < n; ++a) {
            R dg[2] = {R(0), R(0)};
#pragma unroll
            for (int b = 0; b < n; ++b) {
              R g[2];
              EQ::ncg(d, q[b], g);
              dg[0] += tb.D[a][b] * g[0];
              dg[1] += tb.D[a][b] * g[1];
            }
            EQ::nc_apply(d, q[a], dg, acc[a]);
          }
        }
        const R idx_d = inv_dx_of<R>(ma, d);
#pragma unroll
        for (int k = 0; k < n; ++k)
#pragma unroll
          for (int v = 0; v < M; ++v) my[L::O_RS + (i * M + v) * NP + base + k * stride] += acc[k][v] * idx_d;
      }
      __syncthreads();
    }
  }

  // ---- outputs: Rbar = sum_i b_i R_i (coalesced over [v][elements][p])
#pragma unroll 1
  for (int v = 0; v < M; ++v)
    for (int r = tid; r < nel * NP; r += NT) {
      const int ee = r / NP, p = r % NP;
      const R* mm = sm + (size_t)ee * L::SZ;
      R s = R(0);
#pragma unroll
      for (int i = 0; i < S; ++i)
        if ((S1 ? 1.0 : rk_b(N, i)) != 0.0) s += R(S1 ? 1.0 : rk_b(N, i)) * mm[L::O_RS + (i * M + v) * NP + p];
      rbar[((size_t)v * E + e0) * NP + r] = s;
    }
  // face traces: per face node C components (coalesced over the elements)
#pragma unroll 1
  for (int ds = 0; ds < DIM * 2; ++ds)
    for (int idx = tid; idx < nel * NF * C; idx += NT) {
    const int ee = idx % nel;
    const int c = (idx / nel) % C;
    const int f = idx / (nel * C);
    const int side = ds & 1;
    const int d = ds >> 1;
    const int stride = ipow(n, d);
    const int p = line_base<n>(f, stride) + side * N * stride;
    const R* mm = sm + (size_t)ee * L::SZ;
    R val;
    if (c < M) val = mm[L::O_UB + c * NP + p];
    else if (c < 2 * M) val = mm[L::O_FB + (d * M + (c - M)) * NP + p];
    else if (c == 2 * M) val = mm[L::O_LAM + d * NP + p];
    else if (c < 3 * M + 1) val = mm[L::O_FN + (d * M + (c - 2 * M - 1)) * NP + p];
    else val = mm[L::O_U0 + (c - 3 * M - 1) * NP + p];
    trace[trace_index<EQ, NF>(d, side, f, c, E, e0 + ee)] = val;
  }
}

template <class EQ, int N, typename R>
__global__ void __launch_bounds__(256)
k_volume_tile(const double* __restrict__ u, R* __restrict__ rbar, R* __restrict__ trace,
         DevState* __restrict__ st, const MeshArgs ma, const PhysParams<R> pp, const RefTab<R> tb, int slot) {
  volume_tile_body<EQ, N, R, 0>(u, rbar, trace, st, ma, pp, tb, slot, true);
}

// volume part of one RKFR stage (input: the stage state)
template <class EQ, int N, typename R>
__global__ void __launch_bounds__(256)
k_volume_tile_stage(const double* __restrict__ u, R* __restrict__ rbar, R* __restrict__ trace,
                    DevState* __restrict__ st, const MeshArgs ma, const PhysParams<R> pp, const RefTab<R> tb,
                    int slot, int first) {
  volume_tile_body<EQ, N, R, 1>(u, rbar, trace, st, ma, pp, tb, slot, first != 0);
}

// physicality and sum_d lambda_d/dx_d of an updated state; the FP32 form
// evaluates the wave speeds in FP32 (the dt reduction is a max)
template <class EQ, typename R>
__device__ __forceinline__ bool physical_state(const double* uu, const MeshArgs& ma, R& lam) {
  if constexpr (sizeof(R) == 8) {
    if constexpr (EQ::NC) return EQ::physical(uu, ma.gamma, ma.c_h, lam, ma.inv_dx);
    else return EQ::physical(uu, ma.gamma, lam, ma.inv_dx);
  } else {
    float uf[EQ::M];
#pragma unroll
    for (int v = 0; v < EQ::M; ++v) uf[v] = d2f_rz(uu[v]);
    if constexpr (EQ::NC) return EQ::physical(uf, ma.gamma_f, ma.c_h_f, lam, ma.inv_dx_f);
    else return EQ::physical(uf, ma.gamma_f, lam, ma.inv_dx_f);
  }
}

// ---------------------------------------------------------------------------
// Face + update kernel: one thread per node
// ---------------------------------------------------------------------------
// the C components of the record of face node f of face (d, side) of element e
template <class EQ, int N, typename R, bool COH = false>
__device__ __forceinline__ void load_face_record(const R* __restrict__ trace, long long E, int d, int side, int f,
                                                 long long e, R (&rec)[trace_comps<EQ>()]) {
  constexpr int NF = ipow(N + 1, EQ::DIM) / (N + 1), C = trace_comps<EQ>();
  const R* p = trace + trace_index<EQ, NF>(d, side, f, 0, E, e);
#pragma unroll
  for (int c = 0; c < C; ++c) rec[c] = ldx<COH>(p + (size_t)c * E);
}

// Jump J = F^num - F_own [+ B(u^n_own) g^avg(U) - F^nc_own] at one face node
// from the own record o and the other side's record x (eq. numflux.cons and
// the reduced-communication non-conservative flux of Sec. 2.3).
template <class EQ, typename R>
__device__ __forceinline__ void jump_of(const R* o, const R* x, int d, int side_own, R* J, const PhysParams<R>& pp) {
  constexpr int M = EQ::M;
  const R lam = fmax(o[2 * M], x[2 * M]);
  // own is the '-' state when it is the xi = 1 side: U+ - U- = sgn (Ux - Uo)
  const R sgn = side_own == 1 ? R(1) : R(-1);
#pragma unroll
  for (int v = 0; v < M; ++v) J[v] = R(0.5) * (o[M + v] + x[M + v]) - R(0.5) * lam * sgn * (x[v] - o[v]) - o[M + v];
  if constexpr (EQ::NC) {
    // + B(u^n_own) g^avg(U) - F^nc_own (the stage-wise flux adds its own sum
    // in face_jump instead of the first term)
    if constexpr (!EQ::NCS) {
      R un[M], q[EQ::P];
#pragma unroll
      for (int v = 0; v < M; ++v) un[v] = o[3 * M + 1 + v];
      EQ::pair_data(un, q, pp);
      R g[2];
      g[0] = R(0.5) * (o[5 + d] + x[5 + d]);
      g[1] = R(0.5) * (o[8] + x[8]);
      EQ::nc_apply(d, q, g, J);
    }
#pragma unroll
    for (int v = 0; v < M; ++v) J[v] -= o[2 * M + 1 + v];
  }
}

template <class EQ, int N, typename R, bool COH = false>
__device__ __forceinline__ void face_jump(const R* __restrict__ trace, long long E, int d, int side_own, long long e_own,
                                          long long e_oth, int f, R* J, const PhysParams<R>& pp, const RefTab<R>& tb) {
  constexpr int C = trace_comps<EQ>();
  R o[C], x[C];
  load_face_record<EQ, N, R, COH>(trace, E, d, side_own, f, e_own, o);
  load_face_record<EQ, N, R, COH>(trace, E, d, 1 - side_own, f, e_oth, x);
  jump_of<EQ, R>(o, x, d, side_own, J, pp);
  if constexpr (EQ::NCS) {
    // + sum_j b_j B(u^(j)_own) g^avg(u^(j)) (eq. bad.numflux.non.cons)
#pragma unroll 1
    for (int j = 0; j < rk_stages(N); ++j) {
      R wo[7], wx[7];
#pragma unroll
      for (int c = 0; c < 7; ++c) {
        wo[c] = trace[ncs_index<EQ, N>(d, side_own, f, j, c, E, e_own)];
        wx[c] = trace[ncs_index<EQ, N>(d, 1 - side_own, f, j, c, E, e_oth)];
      }
      R go[2], gx[2], g[2], nc[EQ::M];
      EQ::ncg_prims(d, wo, go);
      EQ::ncg_prims(d, wx, gx);
      g[0] = R(0.5) * (go[0] + gx[0]);
      g[1] = R(0.5) * (go[1] + gx[1]);
#pragma unroll
      for (int v = 0; v < EQ::M; ++v) nc[v] = R(0);
      EQ::nc_apply_prims(d, wo, g, nc);
#pragma unroll
      for (int v = 0; v < EQ::M; ++v) J[v] += tb.b[j] * nc[v];
    }
  }
}

// RK = true: stage mode of the multi-stage RKFR step (RkStage)
template <class EQ, int N, typename R, bool RK>
__device__ __forceinline__ void face_update_body(double* __restrict__ u, const R* __restrict__ rbar,
                                                 const R* __restrict__ trace, DevState* __restrict__ st,
                                                 const MeshArgs& ma, const PhysParams<R>& pp, const RefTab<R>& tb,
                                                 int slot, const RkStage<R>& rk) {
  constexpr int DIM = EQ::DIM, M = EQ::M, n = N + 1, NP = ipow(n, DIM);
  constexpr bool F32 = sizeof(R) == 4;
  const long long E = ma.E;
  // a volume CTA that timed out left its records unwritten: leave u^n as it is
  if (st->status & ST_TIMEOUT) return;
  const unsigned gid = blockIdx.x * blockDim.x + threadIdx.x;
  R lam = R(0);
  bool bad = false;
  if (gid < (unsigned)(E * NP)) {
    const unsigned e = gid / NP;
    const int p = (int)(gid % NP);
    unsigned ec[3] = {0, 0, 0};
    elem_coords<DIM>(e, ma, ec);
    const R dtR = step_dt<R>(st);
    // increment of the final update (eq. crkfr.non.cons.final) in the path's
    // arithmetic: -dt Rbar - dt J^- g_R'(1)/dx + dt J^+ (-g_L'(0))/dx
    R du[M];
#pragma unroll
    for (int v = 0; v < M; ++v) du[v] = -dtR * rbar[((size_t)v * E + e) * NP + p];
    int rem = p;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const int cd = rem % n;
      rem /= n;
      const int stride = ipow(n, d);
      const int f = (p % stride) + (p / (stride * n)) * stride;
      if (cd == N) {   // face xi_d = 1: element is the '-' state
        const unsigned nb = neighbour_of(e, ec, d, +1, ma);
        R J[M];
        face_jump<EQ, N, R>(trace, E, d, 1, e, nb, f, J, pp, tb);
        const R s = dtR * tb.iwN * inv_dx_of<R>(ma, d);
#pragma unroll
        for (int v = 0; v < M; ++v) du[v] -= s * J[v];
      }
      if (cd == 0) {   // face xi_d = 0: element is the '+' state
        const unsigned nb = neighbour_of(e, ec, d, -1, ma);
        R J[M];
        face_jump<EQ, N, R>(trace, E, d, 0, e, nb, f, J, pp, tb);
        const R s = dtR * tb.iw0 * inv_dx_of<R>(ma, d);
#pragma unroll
        for (int v = 0; v < M; ++v) du[v] += s * J[v];
      }
    }
    bool last = true;
    double* dst = u;
    if constexpr (RK) {
      // du is this stage's K_j; combine it with the earlier stages' (eq. rkfr1
      // for the next stage state, eq. rkfr2 at the last stage)
      last = rk.j == rk.s - 1;
      const size_t nodes = (size_t)E * NP;
#pragma unroll
      for (int v = 0; v < M; ++v) {
        const size_t g = ((size_t)v * E + e) * NP + p;
        const R kj = du[v];
        if (!last) rk.k[(size_t)rk.j * M * nodes + g] = kj;
        R acc = (last ? tb.b[rk.j] : tb.a[rk.j + 1][rk.j]) * kj;
        for (int q = 0; q < rk.j; ++q) {
          const R c = last ? tb.b[q] : tb.a[rk.j + 1][q];
          if (c != R(0)) acc += c * rk.k[(size_t)q * M * nodes + g];
        }
        du[v] = acc;
      }
      if (!last) dst = rk.uout;
    }
    // u^{n+1} = u^n + du in FP64 (one FP64 add per variable)
    double uu[M];
#pragma unroll
    for (int v = 0; v < M; ++v) {
      const size_t g = ((size_t)v * E + e) * NP + p;
      if constexpr (F32) uu[v] = u[g] + f2d_int(du[v]);
      else uu[v] = u[g] + du[v];
      dst[g] = uu[v];
    }
    if (last) bad = !physical_state<EQ, R>(uu, ma, lam);
  }
  // the CFL reduction of the new state (RKFR: after the last stage only; the
  // stage index is uniform over the grid)
  if (!RK || rk.j == rk.s - 1) reduce_lambda<R>(lam, bad, st, slot ^ 1);
}

template <class EQ, int N, typename R>
__global__ void __launch_bounds__(256)
k_face_update(double* __restrict__ u, const R* __restrict__ rbar, const R* __restrict__ trace,
              DevState* __restrict__ st, const MeshArgs ma, const PhysParams<R> pp, const RefTab<R> tb,
              int slot) {
  face_update_body<EQ, N, R, false>(u, rbar, trace, st, ma, pp, tb, slot, RkStage<R>{nullptr, nullptr, 0, 1});
}

// face / update part of stage rk.j of the multi-stage RKFR step
template <class EQ, int N, typename R>
__global__ void __launch_bounds__(256)
k_face_stage(double* __restrict__ u, const R* __restrict__ rbar, const R* __restrict__ trace,
             DevState* __restrict__ st, const MeshArgs ma, const PhysParams<R> pp, const RefTab<R> tb,
             int slot, const RkStage<R> rk) {
  face_update_body<EQ, N, R, true>(u, rbar, trace, st, ma, pp, tb, slot, rk);
}

// CFL reduction of the current state (used after set_state); wave speeds in
// the path's arithmetic R, like the reduction inside k_face_update
template <class EQ, int N, typename R>
__global__ void __launch_bounds__(256)
k_lambda(const double* __restrict__ u, DevState* __restrict__ st, const MeshArgs ma, int slot) {
  constexpr int M = EQ::M, NP = ipow(N + 1, EQ::DIM);
  const long long E = ma.E;
  const unsigned gid = blockIdx.x * blockDim.x + threadIdx.x;
  R lam = R(0);
  bool bad = false;
  if (gid < (unsigned)(E * NP)) {
    const unsigned e = gid / NP;
    const int p = (int)(gid % NP);
    double uu[M];
#pragma unroll
    for (int v = 0; v < M; ++v) uu[v] = u[((size_t)v * E + e) * NP + p];
    bad = !physical_state<EQ, R>(uu, ma, lam);
  }
  reduce_lambda<R>(lam, bad, st, slot);
}

// FP64 quadrature-weighted totals: per block partial sums, fixed order
template <class EQ, int N>
__global__ void __launch_bounds__(256)
k_totals(const double* __restrict__ u, double* __restrict__ part, const MeshArgs ma, const RefTab<double> tb) {
  constexpr int DIM = EQ::DIM, M = EQ::M, n = N + 1, NP = ipow(n, DIM), K = M + 2;
  const long long E = ma.E;
  const unsigned gid = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  if (gid < (unsigned)(E * NP)) {
    const unsigned e = gid / NP;
    const int p = (int)(gid % NP);
    double wq = 1.0;
    int rem = p;
#pragma unroll
    for (int d = 0; d < DIM; ++d) { wq *= tb.w[rem % n] / ma.inv_dx[d]; rem /= n; }
    double uu[M];
#pragma unroll
    for (int v = 0; v < M; ++v) { uu[v] = u[((size_t)v * E + e) * NP + p]; acc[v] = wq * uu[v]; }
    double rho = uu[0], ke = 0.0, p_;
    if constexpr (EQ::NC) {
      double vv = (uu[1] * uu[1] + uu[2] * uu[2] + uu[3] * uu[3]) / rho;
      ke = 0.5 * vv;
      p_ = (ma.gamma - 1.0) * (uu[4] - ke - 0.5 * (uu[5] * uu[5] + uu[6] * uu[6] + uu[7] * uu[7]) - 0.5 * uu[8] * uu[8]);
    } else {
      double mm = 0.0;
#pragma unroll
      for (int k = 0; k < DIM; ++k) mm += uu[1 + k] * uu[1 + k];
      ke = 0.5 * mm / rho;
      p_ = (ma.gamma - 1.0) * (uu[DIM + 1] - ke);
    }
    acc[M] = wq * ke;
    acc[M + 1] = wq * (-rho * (log(p_) - ma.gamma * log(rho)) / (ma.gamma - 1.0));
  }
  __shared__ double s[K][256];
#pragma unroll
  for (int k = 0; k < K; ++k) s[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
#pragma unroll
      for (int k = 0; k < K; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) part[(size_t)blockIdx.x * K + k] = s[k][0];
}

}  // namespace crk
