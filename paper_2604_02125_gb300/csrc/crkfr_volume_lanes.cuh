// crkfr_volume_lanes.cuh -- the lane-form kernels of the cRKFR step (sm_103a):
// the persistent volume kernel (single solve and batched), the face/update
// kernel (single solve and batched) and their shared-memory layouts.
//
// Same computation as k_volume_tile (element-local cRK stages with the
// flux-differencing residual, the b-weighted volume residual and the face
// traces of the time averages; eqs. crkfr.inner, entropy.cons.flux.dev,
// entropy.cons.noncons.dev, disc.avg.flux), mapped for throughput:
//
//  * a CTA holds 32 elements; warp w handles line index w of every element
//    and lane l handles element l, so every shared-memory access of a warp
//    touches 32 different elements at the same offset: with an odd element
//    stride there are no bank conflicts, and whether a line lies on a face is
//    uniform across the warp;
//  * each thread owns one x-line (N+1 nodes): u^n, the stage combination, the
//    pair data and the whole x-direction flux differencing stay in
//    registers; only the y (and z) lines go through shared memory;
//  * residuals of earlier stages that later stages still need (dense
//    tableaux, N >= 4) stay with the owner thread;
//  * 2D Euler in FP32 (N <= 3): the thread's x-line and y-line are
//    flux-differenced together, one in each half of packed FP32x2
//    instructions (crkfr_f2.cuh), which halves the instructions of the pair
//    fluxes;
//  * the next tile's u^n arrives by TMA bulk copy while the current tile
//    computes (persistent CTAs, one mbarrier, bounded waits);
//  * the register budget (resident CTAs per SM) is set per variant from
//    measurements; the batched form compiles a second shape and lets its
//    autotuner choose.
#pragma once
#include <type_traits>

#include "crkfr_f2.cuh"
#include "crkfr_kernels.cuh"
#include "crkfr_limiter.cuh"

namespace crk {

// stage j's residual is needed by a stage later than j+1
__host__ __device__ constexpr bool rk_saved(int N, int j) {
  bool need = false;
  for (int i = j + 2; i < rk_stages(N); ++i) need = need || (rk_a(N, i, j) != 0.0);
  return need;
}
__host__ __device__ constexpr int rk_slot(int N, int j) {
  int s = 0;
  for (int k = 0; k < j; ++k) s += rk_saved(N, k) ? 1 : 0;
  return s;
}
__host__ __device__ constexpr int rk_nsaved(int N) { return rk_slot(N, rk_stages(N)); }

// Flux differencing along one line of n = N+1 nodes in direction D from the
// pair data q: acc_p = inv_dx (sum_q 2 D_pq f_S(q_p, q_q) [+ B(q_p) sum_q D_pq g(q_q)]).
// Every pair is evaluated once (f_S is symmetric); D_pp f(q_p) only at the two
// end points of a GLL line, where D_pp is non-zero.
template <class EQ, int N, typename R, int D>
__device__ __forceinline__ void line_residual(const R (&q)[N + 1][EQ::P], R (&acc)[N + 1][EQ::M],
                                              R (&fend)[2][EQ::M], const PhysParams<R>& pp, const RefTab<R>& tb,
                                              R inv_dx) {
  constexpr int n = N + 1, M = EQ::M;
#pragma unroll
  for (int k = 0; k < n; ++k)
#pragma unroll
    for (int v = 0; v < M; ++v) acc[k][v] = R(0);
  // physical fluxes at the two end points: the D_pp terms here, and the face
  // sums of the time-averaged flux (eq. disc.avg.flux) in the caller
  EQ::flux(D, q[0], fend[0], pp);
  EQ::flux(D, q[N], fend[1], pp);
#pragma unroll
  for (int v = 0; v < M; ++v) {
    acc[0][v] = R(2) * tb.D[0][0] * fend[0][v];
    acc[N][v] = R(2) * tb.D[N][N] * fend[1][v];
  }
#pragma unroll
  for (int a = 0; a < n; ++a)
#pragma unroll
    for (int b = a + 1; b < n; ++b) {
      R f[M];
      EQ::two_point(D, q[a], q[b], f, pp);
      const R dab = R(2) * tb.D[a][b], dba = R(2) * tb.D[b][a];
#pragma unroll
      for (int v = 0; v < M; ++v) { acc[a][v] += dab * f[v]; acc[b][v] += dba * f[v]; }
    }
  if constexpr (EQ::NC) {
#pragma unroll
    for (int a = 0; a < n; ++a) {
      R dg[2] = {R(0), R(0)};
#pragma unroll
      for (int b = 0; b < n; ++b) {
        R g[2];
        EQ::ncg(D, q[b], g);
        dg[0] += tb.D[a][b] * g[0];
        dg[1] += tb.D[a][b] * g[1];
      }
      EQ::nc_apply(D, q[a], dg, acc[a]);
    }
  }
#pragma unroll
  for (int k = 0; k < n; ++k)
#pragma unroll
    for (int v = 0; v < M; ++v) acc[k][v] *= inv_dx;
}

// The x-line and the y-line of one thread in the two halves of packed FP32
// pairs (2D Euler, FP32 form).  Both lines are flux-differenced in a frame
// rotated to the line: the y half holds (rho, v_y, v_x, p, aux), so the
// normal direction is the first velocity component in both halves, and the
// momentum results of the y half come out in (normal, tangential) order.
template <class EQ>
struct PackXY {
  static constexpr bool value = EQ::DIM == 2 && !EQ::NC;
  // pair-data / residual component of the x line -> of the y half
  __host__ __device__ static constexpr int rot(int c) { return c == 1 ? 2 : (c == 2 ? 1 : c); }
};

// Component of the pair data or residual of a line in direction y, seen in a
// frame reflected across the diagonal so that y becomes the first direction:
// swap of the x and y vector components (velocity / momentum, and the
// magnetic field for GLM-MHD).  The systems and their two-point fluxes are
// invariant under this relabelling, and it is its own inverse.
template <class EQ>
__host__ __device__ constexpr int swap_xy(int c) {
  return c == 1 ? 2 : c == 2 ? 1 : (EQ::NC && c == 5) ? 6 : (EQ::NC && c == 6) ? 5 : c;
}

// PRE: the coefficients carry 1/dx of each line (RefTab::D2s), else the
// residual is scaled at the end
template <class EQ, int N, bool PRE>
__device__ __forceinline__ void line_residual_xy(const f2 (&q)[N + 1][EQ::P], f2 (&acc)[N + 1][EQ::M],
                                                 f2 (&fend)[2][EQ::M], const PhysParams<f2>& pp,
                                                 const RefTab<float>& tb, f2 inv_dx) {
  constexpr int n = N + 1, M = EQ::M;
#pragma unroll
  for (int k = 0; k < n; ++k)
#pragma unroll
    for (int v = 0; v < M; ++v) acc[k][v] = f2(0.0f);
#pragma unroll
  for (int a = 0; a < n; ++a)
#pragma unroll
    for (int b = a + 1; b < n; ++b) {
      f2 f[M];
      EQ::two_point(0, q[a], q[b], f, pp);
      const f2 dab(PRE ? tb.D2s[a][b] : tb.D2f[a][b]), dba(PRE ? tb.D2s[b][a] : tb.D2f[b][a]);
#pragma unroll
      for (int v = 0; v < M; ++v) { acc[a][v] += dab * f[v]; acc[b][v] += dba * f[v]; }
    }
  // end points last: the fluxes there stay live only until the face sums
  EQ::flux(0, q[0], fend[0], pp);
  EQ::flux(0, q[N], fend[1], pp);
#pragma unroll
  for (int v = 0; v < M; ++v) {
    acc[0][v] += f2(PRE ? tb.D2s[0][0] : tb.D2f[0][0]) * fend[0][v];
    acc[N][v] += f2(PRE ? tb.D2s[N][N] : tb.D2f[N][N]) * fend[1][v];
  }
  if constexpr (!PRE) {
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int v = 0; v < M; ++v) acc[k][v] *= inv_dx;
  }
}


// Flux differencing of one line of the element at `my`, rolled over the pairs
// so that the two-point flux is compiled once: pair data read from shared
// memory (Q, component c at Q[c * NP + node]) in the frame of swap_xy when
// sw is set, the residual (times inv_dx) added into shared memory (RY, in the
// element's own frame); the end nodes' pair data and fluxes are returned for
// the face sums.  Every node of the line belongs to the calling thread.
template <class EQ, int N, typename R>
__device__ __forceinline__ void line_residual_rolled(const R* __restrict__ Q, R* __restrict__ RY, int NPv, int base,
                                                     int stride, bool sw, R (&qe)[N + 1][EQ::P], R (&fend)[2][EQ::M],
                                                     const PhysParams<R>& pp, const RefTab<R>& tb, R inv_dx) {
  constexpr int n = N + 1, M = EQ::M, P = EQ::P;
  auto load = [&](int node, R* q) {
#pragma unroll
    for (int c = 0; c < P; ++c) q[c] = Q[(sw ? swap_xy<EQ>(c) : c) * NPv + node];
  };
  load(base, qe[0]);
  load(base + N * stride, qe[N]);
  EQ::flux(0, qe[0], fend[0], pp);
  EQ::flux(0, qe[N], fend[1], pp);
#pragma unroll 1
  for (int a = 0; a < n; ++a) {
    const int na = base + a * stride;
    R qa[P], acc[M];
    load(na, qa);
    // D_aa f(q_a): non-zero only at the two end points of a GLL line
    const R caa = R(2) * tb.D[a][a] * inv_dx;
#pragma unroll
    for (int v = 0; v < M; ++v) acc[v] = a == 0 ? caa * fend[0][v] : (a == N ? caa * fend[1][v] : R(0));
#pragma unroll 1
    for (int b = a + 1; b < n; ++b) {
      const int nb = base + b * stride;
      R qb[P], f[M];
      load(nb, qb);
      EQ::two_point(0, qa, qb, f, pp);
      const R cab = R(2) * tb.D[a][b] * inv_dx, cba = R(2) * tb.D[b][a] * inv_dx;
#pragma unroll
      for (int v = 0; v < M; ++v) {
        acc[v] += cab * f[v];
        RY[(sw ? swap_xy<EQ>(v) : v) * NPv + nb] += cba * f[v];
      }
    }
    if constexpr (EQ::NC) {
      // sum_b D_ab B(u_a) g(u_b) = B(u_a) (D g)_a (no factor 2)
      R dg[2] = {R(0), R(0)};
#pragma unroll 1
      for (int b = 0; b < n; ++b) {
        const int nb = base + b * stride;
        const R dab = tb.D[a][b] * inv_dx;
        dg[0] += dab * Q[(sw ? swap_xy<EQ>(EQ::IB) : EQ::IB) * NPv + nb];
        dg[1] += dab * Q[EQ::IPSI * NPv + nb];
      }
      EQ::nc_apply(0, qa, dg, acc);
    }
#pragma unroll
    for (int v = 0; v < M; ++v) RY[(sw ? swap_xy<EQ>(v) : v) * NPv + na] += acc[v];
  }
}

// Time averages at the two end points of one line in direction D (the face
// nodes of the two faces normal to D): U = sum_i b_i u^(i), F^D = sum_i b_i
// f^D(u^(i)) (eq. disc.avg.flux), lambda_D(u^n), and for the non-conservative
// system F^nc,D = sum_i b_i B^D g^D (Sec. 2.3).  One record per end.
template <class EQ, typename R, bool NC = EQ::NC>
struct FaceAccNc {
  R Nc[2][EQ::M];
};
template <class EQ, typename R>
struct FaceAccNc<EQ, R, false> {};

template <class EQ, typename R>
struct FaceAcc : FaceAccNc<EQ, R> {
  static constexpr int M = EQ::M;
  R U[2][M], F[2][M], lam[2];
};

// Register budget of the 2D Euler lane kernels of degree 4 and 5 (resident
// CTAs per SM; measured: more CTAs outweigh the spills up to the shared-memory
// limit) and the highest degree that takes the packed x/y form.  Degree 4
// packed runs at 2 CTAs per SM (168 registers, 108 B of spills): 99 against
// 117 us per volume launch of the scalar form at 3 CTAs (2D Euler 128^2, FP32);
// at 3 CTAs the packed form spilled 488 B (140 us).  At degree 5 both lines'
// pair data no longer fit: packed 99 (2 CTAs) or 109 us (1 CTA) against 83 us
// for the scalar form (96^2).
constexpr int kMinB4 = 3, kMinB4Pack = 2, kMinB5 = 2, kPackMaxN = 4;
// degree 2, FP32: short lines, little per-thread state; 8 CTAs per SM (measured
// 0.50 -> 0.42 ms per batched volume launch against 3)
constexpr int kMinB2 = 8;
// GLM-MHD (9 variables, 13 pair data): 2 CTAs per SM where the layout allows
// it, which needs the shared memory of the next tile's staging buffer
// (measured: 0.58 against 0.73 ms per volume launch at 128^2, N = 4, FP32)
constexpr int kMinBNc = 2;
constexpr bool kStageNc = false;

// Kernel shapes: SH = 0 is the measured default of each variant; SH = 1 is the
// alternative the batched form's autotuner also times: the scalar form (no
// x/y packing) at one resident CTA per SM more than the packed default, or,
// for a scalar default, one fewer (fewer spills, fewer warps).
template <class EQ, int N, typename R, int SH = 0>
struct LaneLayout;

template <class EQ, int N, typename R>
struct LaneLayout<EQ, N, R, 0> {
  static constexpr int DIM = EQ::DIM, M = EQ::M, P = EQ::P, n = N + 1;
  static constexpr int NP = ipow(n, DIM), NF = NP / n, S = rk_stages(N);
  static constexpr int O_Q = 0;                                // [P][NP] pair data (also staging)
  static constexpr int O_RY = O_Q + P * NP;                    // [M][NP] y (+z) residual
  static constexpr int O_U0 = O_RY + (DIM > 1 ? M * NP : 0);   // [M][NP] u^n
  static constexpr int SZ0 = O_U0 + M * NP;
  static constexpr int SZ = SZ0 | 1;                           // odd element stride: no bank conflicts
  static constexpr int EPB = 32;
  static constexpr int THREADS = 32 * NF;
  static constexpr size_t bytes() { return sizeof(R) * (size_t)SZ * EPB; }
  // packed x/y form (2D Euler, FP32 pair fluxes)
  static constexpr bool PACK = PackXY<EQ>::value && sizeof(R) == 4 && N <= kPackMaxN;
  // CTAs per SM the register allocation aims at (the packed form holds both
  // lines' pair data at once)
  static constexpr int MINB = EQ::NC ? (2 * (bytes() + 1024) <= 228 * 1024 ? kMinBNc : 1)
                            : (THREADS <= 128) ? ((N == 2 && sizeof(R) == 4) ? kMinB2 : PACK ? 3 : 4)
                            : (DIM == 2) ? (N == 4 ? (PACK ? kMinB4Pack : kMinB4) : N == 5 ? kMinB5 : 1) : 1;
  static constexpr bool fits() { return bytes() <= 227 * 1024 && THREADS <= 1024; }
};

template <class EQ, int N, typename R>
struct LaneLayout<EQ, N, R, 1> : LaneLayout<EQ, N, R, 0> {
  using B = LaneLayout<EQ, N, R, 0>;
  static constexpr bool PACK = false;
  static constexpr int MINB = B::PACK ? B::MINB + 1 : (B::MINB > 1 ? B::MINB - 1 : 1);
};

// face_accumulate for both lines of the packed form at once (x-line ends in
// the low halves, y-line ends in the high halves, the latter in the frame of
// the y-line); the wave speeds are taken separately
template <class EQ, int N>
__device__ __forceinline__ void face_accumulate_xy(FaceAcc<EQ, f2>& fa, const f2 (&q)[N + 1][EQ::P],
                                                   const f2 (&fend)[2][EQ::M], f2 b, bool first,
                                                   const PhysParams<f2>& pp) {
  constexpr int M = EQ::M;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    f2 uu[M];
    EQ::cons_from_pair(q[side ? N : 0], uu, pp);
    if (first) {
#pragma unroll
      for (int v = 0; v < M; ++v) {
        fa.U[side][v] = f2(0.0f);
        fa.F[side][v] = f2(0.0f);
      }
    }
#pragma unroll
    for (int v = 0; v < M; ++v) {
      fa.U[side][v] += b * uu[v];
      fa.F[side][v] += b * fend[side][v];
    }
  }
}

template <class EQ, int N, typename R, int D>
__device__ __forceinline__ void face_accumulate(FaceAcc<EQ, R>& fa, const R (&q)[N + 1][EQ::P],
                                                const R (&fend)[2][EQ::M], R b, bool first,
                                                const PhysParams<R>& pp) {
  constexpr int M = EQ::M;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const R* qs = q[side ? N : 0];
    R uu[M];
    EQ::cons_from_pair(qs, uu, pp);
    if (first) {
      fa.lam[side] = EQ::wave_speed(D, qs, pp);
#pragma unroll
      for (int v = 0; v < M; ++v) {
        fa.U[side][v] = R(0);
        fa.F[side][v] = R(0);
      }
      if constexpr (EQ::NC) {
#pragma unroll
        for (int v = 0; v < M; ++v) fa.Nc[side][v] = R(0);
      }
    }
#pragma unroll
    for (int v = 0; v < M; ++v) {
      fa.U[side][v] += b * uu[v];
      fa.F[side][v] += b * fend[side][v];
    }
    if constexpr (EQ::NC) {
      R g[2], nc[M];
#pragma unroll
      for (int v = 0; v < M; ++v) nc[v] = R(0);
      EQ::ncg(D, qs, g);
      EQ::nc_apply(D, qs, g, nc);
#pragma unroll
      for (int v = 0; v < M; ++v) fa.Nc[side][v] += b * nc[v];
    }
  }
}

// Record of one face node: U, F, lambda [, F^nc, u^n] (C components, each
// store coalesced over the warp's elements).  u^n of the two end nodes
// (non-conservative system) is read from shared memory: un0 / unN point at
// variable 0 of the end nodes, variables NP apart.
template <class EQ, typename R, int NF>
__device__ __forceinline__ void write_records(R* __restrict__ trace, const FaceAcc<EQ, R>& fa, int d, long long E,
                                              long long e, int f, const R* un0, const R* unN, int NPv) {
  constexpr int M = EQ::M;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    R* dst = trace + trace_index<EQ, NF>(d, side, f, 0, E, e);
#pragma unroll
    for (int v = 0; v < M; ++v) {
      dst[(size_t)v * E] = fa.U[side][v];
      dst[(size_t)(M + v) * E] = fa.F[side][v];
    }
    dst[(size_t)(2 * M) * E] = fa.lam[side];
    if constexpr (EQ::NC) {
#pragma unroll
      for (int v = 0; v < M; ++v) {
        dst[(size_t)(2 * M + 1 + v) * E] = fa.Nc[side][v];
        dst[(size_t)(3 * M + 1 + v) * E] = (side ? unN : un0)[v * NPv];
      }
    }
  }
}

// Prefetch of the next tile's u^n into the staging buffer (TMA bulk copies,
// one per variable), issued by thread 0 once the current tile's staging data
// has been consumed.  src == nullptr: nothing to prefetch.
struct Prefetch {
  const double* src;        // u^n of variable 0 of the next tile
  long long var_stride;     // doubles between variables (E * NP of the next tile's solve)
  unsigned bytes;           // bytes per variable (32 * NP * 8)
  double* staging;
  unsigned long long* bar;
};

template <int M>
__device__ __forceinline__ void issue_prefetch(const Prefetch& pf) {
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(pf.bar, M * pf.bytes);
#pragma unroll
  for (int v = 0; v < M; ++v)
    bulk_copy_g2s(pf.staging + (size_t)v * (pf.bytes / 8), pf.src + (size_t)v * pf.var_stride, pf.bytes, pf.bar);
}

// One tile of 32 elements starting at e0 (the CTA's whole shared memory sm).
// staged != nullptr: u^n of the tile already sits in shared memory as FP64,
// [var][32][NP] (the tile's slice of the global layout).  S1 = 1: a single
// stage with b = 1 (R-bar = R(u), face records of u), the volume part of one
// stage of the multi-stage RKFR step.
// PRE: a single solve's reference table (the packed pair loop's coefficients
// carry 1/dx, RefTab::D2s); false for the batched kernels
template <class EQ, int N, typename R, int SH = 0, int S1 = 0, bool PRE = false>
__device__ __forceinline__ void volume_lanes_tile(const double* __restrict__ u, R* __restrict__ rbar,
                                                  R* __restrict__ trace, const DevState* __restrict__ st,
                                                  const MeshArgs& ma, const PhysParams<R>& pp, const RefTab<R>& tb,
                                                  long long e0, R dtR, R* sm, const double* staged = nullptr,
                                                  Prefetch pf = Prefetch{nullptr, 0, 0, nullptr, nullptr}) {
  using L = LaneLayout<EQ, N, R, SH>;
  constexpr int DIM = L::DIM, M = L::M, P = L::P, n = L::n, NP = L::NP, NF = L::NF, S = S1 ? S1 : L::S;
  // 2D scalar form, degree 5 and GLM-MHD in FP64: the x-line and the y-line go
  // through one copy of the pair loop (a rolled loop over the two directions,
  // the y-line in the frame of swap_xy), with the pair data read back from
  // shared memory: half the code of two inlined copies, and no pair data held
  // across the barrier.  Measured: degree 5 (FP32) 244 against 254 us and the
  // GLM-MHD vortex at degree 4 (FP64) 4.71 against 4.86 ms per launch, but
  // degree 4 (FP32) 211 against 194 us; elsewhere no gain.
  constexpr bool ROLL = !L::PACK && DIM == 2 && (N >= 5 || (EQ::NC && sizeof(R) == 8)) && !(EQ::NC && sizeof(R) == 4 && N >= 4);
  // 2D GLM-MHD in FP32 at degree 4 and 5: the pair loop itself rolled
  // (line_residual_rolled), both directions' residuals added in place into the
  // shared buffer RY (cleared by the node phase), so the x-line residual is not
  // held in registers either.  Measured per launch: degree 5 (96^2) 520 against
  // 600 us, degree 4 (128^2) 542 against 569 us; degree 3 slower (110 against
  // 87 us), so it keeps the form below.
  constexpr bool ROLLP = !L::PACK && DIM == 2 && EQ::NC && sizeof(R) == 4 && N >= 4;
  constexpr bool ONEQ = ROLL || ROLLP;   // the node phase keeps no pair data
  constexpr int NS = rk_nsaved(N) > 0 ? rk_nsaved(N) : 1;

  const int tid = threadIdx.x;
  const int l = tid >> 5;              // line index (warp-uniform)
  const int el = tid & 31;             // element within the CTA
  const long long E = ma.E;
  const int nel = (int)min(32LL, E - e0);
  const bool active = el < nel;
  R* my = sm + (size_t)el * L::SZ;
  constexpr bool PACK = L::PACK;
  const PhysParams<f2> pp2{f2(float(pp.gamma)), f2(float(pp.inv_gm1)), f2(float(pp.c_h)), pp.vol};

  // ---- u^n: coalesced into shared memory (staging in the Q region), then own x-line to registers
  // (index arithmetic with compile-time divisors only).  FP32 form: the hardware conversion, one
  // issue slot on the FP64 pipe, which this kernel leaves otherwise idle (the integer d2f_int is
  // about twenty ALU instructions; measured 59.5 -> 56.6 us per launch, 2D Euler 256^2, N = 3)
  // each variable's 32 NP values are n rounds of the CTA's 32 NF threads:
  // the node offsets of the rounds are computed once, the variable loop only
  // adds its stride
  static_assert(32 * NP == n * L::THREADS, "a tile's values per variable are n rounds of the CTA");
  int tofs[n];
  bool tok[n];
#pragma unroll
  for (int j = 0; j < n; ++j) {
    const int r = tid + j * L::THREADS, ee = r / NP;
    tofs[j] = ee * L::SZ + L::O_U0 + r % NP;
    tok[j] = ee < nel;
  }
  {
    const double* src = staged ? staged + tid : u + (size_t)e0 * NP + tid;
    const size_t vstride = staged ? (size_t)32 * NP : (size_t)E * NP;
#pragma unroll 1
    for (int v = 0; v < M; ++v, src += vstride) {
#pragma unroll
      for (int j = 0; j < n; ++j)
        if (tok[j]) {
          const double x = src[j * L::THREADS];
          if constexpr (sizeof(R) == 4) sm[tofs[j] + v * NP] = __double2float_rn(x);
          else sm[tofs[j] + v * NP] = x;
        }
    }
  }
  __syncthreads();
  // the staging buffer is free: start the next tile's copy, overlapped with this tile's work
  if (pf.src && tid == 0) issue_prefetch<M>(pf);

  R rb[n][M], ax[n][M], rs[NS][n][M];
#pragma unroll
  for (int k = 0; k < n; ++k)
#pragma unroll
    for (int v = 0; v < M; ++v) { rb[k][v] = R(0); ax[k][v] = R(0); }
  // face sums of the ends of this thread's x-line (faces normal to x), y-line and z-line
  FaceAcc<EQ, R> fx, fy, fz;
  FaceAcc<EQ, f2> fxy;   // packed form: both lines' face sums

  // the stage loop stays rolled: one stage's code is large, and S copies of it
  // would overflow the instruction cache; the tableau comes from the parameters
#pragma unroll 1
  for (int i = 0; i < S; ++i) {
    const R bi = S1 ? R(1) : tb.b[i];
    // ---------------- node phase (own x-line): stage state and pair data
    R q[ONEQ ? 1 : n][P];
    if (active) {
#pragma unroll
      for (int k = 0; k < n; ++k) {
        const int p = l * n + k;
        R uu[M];
#pragma unroll
        for (int v = 0; v < M; ++v) {
          R acc = R(0);
          if (i > 0) {
            // complete R_{i-1} = x part (registers) + y/z part (shared); the
            // rolled-pair form keeps both in shared memory
            R r = (ROLLP ? R(0) : ax[k][v]) + (DIM > 1 ? my[L::O_RY + v * NP + p] : R(0));
            rb[k][v] += tb.b[i - 1] * r;
            acc = tb.a[i][i - 1] * r;
            if constexpr (rk_nsaved(N) > 0) {
              if (tb.slot[i - 1] >= 0) rs[tb.slot[i - 1]][k][v] = r;
              for (int j = 0; j < i - 1; ++j)
                if (tb.slot[j] >= 0) acc += tb.a[i][j] * rs[tb.slot[j]][k][v];
            }
          }
          uu[v] = my[L::O_U0 + v * NP + p] - dtR * acc;
          if constexpr (ROLLP) my[L::O_RY + v * NP + p] = R(0);
        }
        R* qk = q[ONEQ ? 0 : k];
        EQ::pair_data(uu, qk, pp);
        if (DIM > 1) {
#pragma unroll
          for (int c = 0; c < P; ++c) my[L::O_Q + c * NP + p] = qk[c];
        }
        if constexpr (ONEQ && EQ::NCS) {
          // face traces of this stage: the ends of the x-line, and the whole
          // x-line where it lies on a face normal to y
          if (k == 0) write_stage_prims<EQ, N, R>(trace, 0, 0, l, i, E, e0 + el, qk);
          if (k == N) write_stage_prims<EQ, N, R>(trace, 0, 1, l, i, E, e0 + el, qk);
          if (l == 0) write_stage_prims<EQ, N, R>(trace, 1, 0, k, i, E, e0 + el, qk);
          if (l == N) write_stage_prims<EQ, N, R>(trace, 1, 1, k, i, E, e0 + el, qk);
        }
      }
      if constexpr (EQ::NCS && !ONEQ) {
        // face traces of this stage at the ends of the x-line (stage-wise
        // non-conservative flux)
        write_stage_prims<EQ, N, R>(trace, 0, 0, l, i, E, e0 + el, q[0]);
        write_stage_prims<EQ, N, R>(trace, 0, 1, l, i, E, e0 + el, q[N]);
      }
      // ---------------- x-direction flux differencing, all in registers
      // (packed form: together with the y-line below)
      if constexpr (!PACK && !ONEQ) {
        R fend[2][M];
        line_residual<EQ, N, R, 0>(q, ax, fend, pp, tb, inv_dx_of<R>(ma, 0));
        face_accumulate<EQ, N, R, 0>(fx, q, fend, bi, i == 0, pp);
      }
    }
    if constexpr (PACK) {
      __syncthreads();   // Q of this stage visible; RY of the last stage consumed
      if (active) {
        // y-line l: nodes (i = l, j = 0..N); x-line in the low halves, y-line in the high halves
        R qy[n][P];
        f2 q2[n][P], acc2[n][M], fe2[2][M];
#pragma unroll
        for (int k = 0; k < n; ++k)
#pragma unroll
          for (int c = 0; c < P; ++c) qy[k][c] = my[L::O_Q + c * NP + l + k * n];
#pragma unroll
        for (int k = 0; k < n; ++k)
#pragma unroll
          for (int c = 0; c < P; ++c) q2[k][c] = f2(q[k][c], qy[k][PackXY<EQ>::rot(c)]);
        line_residual_xy<EQ, N, PRE>(q2, acc2, fe2, pp2, tb, f2(inv_dx_of<float>(ma, 0), inv_dx_of<float>(ma, 1)));
#pragma unroll
        for (int k = 0; k < n; ++k)
#pragma unroll
          for (int v = 0; v < M; ++v) {
            ax[k][v] = acc2[k][v].v.x;
            my[L::O_RY + v * NP + l + k * n] = acc2[k][PackXY<EQ>::rot(v)].v.y;
          }
        if (i == 0) {
#pragma unroll
          for (int sd = 0; sd < 2; ++sd) {
            fx.lam[sd] = EQ::wave_speed(0, q[sd ? N : 0], pp);
            fy.lam[sd] = EQ::wave_speed(1, qy[sd ? N : 0], pp);
          }
        }
        face_accumulate_xy<EQ, N>(fxy, q2, fe2, f2(bi), i == 0, pp2);
      }
      __syncthreads();   // RY complete
    } else if constexpr (ROLLP) {
      __syncthreads();   // Q of this stage visible; RY of the last stage consumed and cleared
#pragma unroll 1
      for (int dir = 0; dir < 2; ++dir) {
        if (active) {
          R qe[n][P], fe[2][M];
          line_residual_rolled<EQ, N, R>(my + L::O_Q, my + L::O_RY, NP, dir ? l : l * n, dir ? n : 1, dir != 0, qe,
                                         fe, pp, tb, dir ? inv_dx_of<R>(ma, 1) : inv_dx_of<R>(ma, 0));
          if (dir == 0) face_accumulate<EQ, N, R, 0>(fx, qe, fe, bi, i == 0, pp);
          else face_accumulate<EQ, N, R, 0>(fy, qe, fe, bi, i == 0, pp);   // swapped frame
        }
        // the x pass is complete before the y pass adds into the same nodes;
        // after the y pass RY holds the whole residual
        __syncthreads();
      }
    } else if constexpr (ROLL) {
      __syncthreads();   // Q of this stage visible; RY of the last stage consumed
      if (active) {
#pragma unroll 1
        for (int dir = 0; dir < 2; ++dir) {
          // x-line l: nodes l n + k; y-line l: nodes l + k n (2D)
          const int base = dir ? l : l * n, stride = dir ? n : 1;
          R qd[n][P], ad[n][M], fe[2][M];
#pragma unroll
          for (int k = 0; k < n; ++k)
#pragma unroll
            for (int c = 0; c < P; ++c) qd[k][c] = my[L::O_Q + (dir ? swap_xy<EQ>(c) : c) * NP + base + k * stride];
          line_residual<EQ, N, R, 0>(qd, ad, fe, pp, tb, dir ? inv_dx_of<R>(ma, 1) : inv_dx_of<R>(ma, 0));
          if (dir == 0) {
#pragma unroll
            for (int k = 0; k < n; ++k)
#pragma unroll
              for (int v = 0; v < M; ++v) ax[k][v] = ad[k][v];
            face_accumulate<EQ, N, R, 0>(fx, qd, fe, bi, i == 0, pp);
          } else {
#pragma unroll
            for (int k = 0; k < n; ++k)
#pragma unroll
              for (int v = 0; v < M; ++v) my[L::O_RY + swap_xy<EQ>(v) * NP + base + k * n] = ad[k][v];
            // accumulated in the swapped frame; swapped back when written
            face_accumulate<EQ, N, R, 0>(fy, qd, fe, bi, i == 0, pp);
          }
        }
      }
      __syncthreads();   // RY complete
    } else if (DIM > 1) {
      __syncthreads();   // Q of this stage visible; RY of the last stage consumed
      if (active) {
        // y-line l: nodes (i = l % n, j = 0..N, k = l / n)
        const int base = (l % n) + (l / n) * n * n;
        R qy[n][P], ay[n][M], fend[2][M];
#pragma unroll
        for (int k = 0; k < n; ++k)
#pragma unroll
          for (int c = 0; c < P; ++c) qy[k][c] = my[L::O_Q + c * NP + base + k * n];
        if constexpr (EQ::NCS) {
          static_assert(DIM == 2, "stage-wise non-conservative flux: 2D only");
          write_stage_prims<EQ, N, R>(trace, 1, 0, l, i, E, e0 + el, qy[0]);
          write_stage_prims<EQ, N, R>(trace, 1, 1, l, i, E, e0 + el, qy[N]);
        }
        line_residual<EQ, N, R, (DIM > 1 ? 1 : 0)>(qy, ay, fend, pp, tb, inv_dx_of<R>(ma, 1));
        face_accumulate<EQ, N, R, (DIM > 1 ? 1 : 0)>(fy, qy, fend, bi, i == 0, pp);
#pragma unroll
        for (int k = 0; k < n; ++k)
#pragma unroll
          for (int v = 0; v < M; ++v) my[L::O_RY + v * NP + base + k * n] = ay[k][v];
      }
      if (DIM == 3) {
        __syncthreads();
        if (active) {
          // z-line l: nodes (i, j) = (l % n, l / n), k = 0..N
          const int base = l;
          R qz[n][P], az[n][M], fend[2][M];
#pragma unroll
          for (int k = 0; k < n; ++k)
#pragma unroll
            for (int c = 0; c < P; ++c) qz[k][c] = my[L::O_Q + c * NP + base + k * n * n];
          line_residual<EQ, N, R, DIM - 1>(qz, az, fend, pp, tb, inv_dx_of<R>(ma, DIM - 1));
          face_accumulate<EQ, N, R, DIM - 1>(fz, qz, fend, bi, i == 0, pp);
#pragma unroll
          for (int k = 0; k < n; ++k)
#pragma unroll
            for (int v = 0; v < M; ++v) my[L::O_RY + v * NP + base + k * n * n] += az[k][v];
        }
      }
      __syncthreads();   // RY complete
    }
  }

  // ---- last stage's residual, Rbar to shared (Q region) then coalesced store
  if (active) {
#pragma unroll
    for (int k = 0; k < n; ++k) {
      const int p = l * n + k;
#pragma unroll
      for (int v = 0; v < M; ++v) {
        R r = (ROLLP ? R(0) : ax[k][v]) + (DIM > 1 ? my[L::O_RY + v * NP + p] : R(0));
        my[L::O_Q + v * NP + p] = rb[k][v] + (S1 ? R(1) : tb.b[S - 1]) * r;
      }
    }
  }
  __syncthreads();
  {
    int qofs[n];
    bool qok[n];
#pragma unroll
    for (int j = 0; j < n; ++j) {
      const int r = tid + j * L::THREADS, ee = r / NP;
      qofs[j] = ee * L::SZ + L::O_Q + r % NP;
      qok[j] = ee < nel;
    }
    R* dst = rbar + (size_t)e0 * NP + tid;
#pragma unroll 1
    for (int v = 0; v < M; ++v, dst += (size_t)E * NP) {
#pragma unroll
      for (int j = 0; j < n; ++j)
        if (qok[j]) dst[j * L::THREADS] = sm[qofs[j] + v * NP];
    }
  }
  // ---- face records [DIM][2][NF][C][E]: this thread owns the two ends of its
  // x-, y- and z-line, i.e. face node f = l of every face; consecutive lanes
  // write consecutive records
  if (active) {
    const R* u0 = my + L::O_U0;
    // end nodes: x-line l (l n, l n + N), y-line l (by, by + N n), z-line l (l, l + N n^2)
    const int by = (l % n) + (l / n) * n * n;
    if constexpr (PACK) {
#pragma unroll
      for (int sd = 0; sd < 2; ++sd)
#pragma unroll
        for (int v = 0; v < M; ++v) {
          fx.U[sd][v] = fxy.U[sd][v].v.x;
          fx.F[sd][v] = fxy.F[sd][v].v.x;
          fy.U[sd][v] = fxy.U[sd][PackXY<EQ>::rot(v)].v.y;
          fy.F[sd][v] = fxy.F[sd][PackXY<EQ>::rot(v)].v.y;
        }
    }
    write_records<EQ, R, NF>(trace, fx, 0, E, e0 + el, l, u0 + l * n, u0 + l * n + N, NP);
    if constexpr (ONEQ) {
      FaceAcc<EQ, R> fyo;
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        fyo.lam[sd] = fy.lam[sd];
#pragma unroll
        for (int v = 0; v < M; ++v) {
          fyo.U[sd][swap_xy<EQ>(v)] = fy.U[sd][v];
          fyo.F[sd][swap_xy<EQ>(v)] = fy.F[sd][v];
          if constexpr (EQ::NC) fyo.Nc[sd][swap_xy<EQ>(v)] = fy.Nc[sd][v];
        }
      }
      write_records<EQ, R, NF>(trace, fyo, 1, E, e0 + el, l, u0 + by, u0 + by + N * n, NP);
    } else if (DIM > 1) {
      write_records<EQ, R, NF>(trace, fy, 1, E, e0 + el, l, u0 + by, u0 + by + N * n, NP);
    }
    if (DIM > 2) write_records<EQ, R, NF>(trace, fz, 2, E, e0 + el, l, u0 + l, u0 + l + N * n * n, NP);
  }
}

// shared memory of the persistent lane kernels: lane layout, then the FP64
// staging buffer of one tile, then the mbarrier
template <class EQ, int N, typename R>
struct PersistLayout {
  using L = LaneLayout<EQ, N, R>;
  static constexpr bool STAGE = !EQ::NC || kStageNc;
  static constexpr size_t O_STAGE = (L::bytes() + 15) & ~(size_t)15;
  static constexpr size_t STAGE_BYTES = STAGE ? sizeof(double) * (size_t)EQ::M * 32 * L::NP : 0;
  static constexpr size_t O_BAR = O_STAGE + STAGE_BYTES;
  static constexpr size_t bytes() { return O_BAR + 16; }
  static constexpr bool fits() { return L::fits() && bytes() <= 227 * 1024; }
};

// Persistent volume kernel for one solve: CTA b handles tiles b, b + grid, ...;
// u^n of whole tiles arrives by TMA bulk copy one tile ahead.  first = false
// (later stages of a multi-stage RKFR step) takes the dt the step's first
// launch recorded.
struct NoTileWork {
  __device__ void operator()(long long, const float*) const {}
};

// after_tile(e0, sm): more work on a finished tile whose u^n is still in the
// lane layout's u^n region of sm (the rest of the layout is free)
template <class EQ, int N, typename R, int S1, class After = NoTileWork>
__device__ __forceinline__ void volume_lanes_persistent(const double* __restrict__ u, R* __restrict__ rbar,
                                                        R* __restrict__ trace, DevState* __restrict__ st,
                                                        const MeshArgs& ma, const PhysParams<R>& pp,
                                                        const RefTab<R>& tb, int slot, bool first,
                                                        After after_tile = After{}) {
  using PL = PersistLayout<EQ, N, R>;
  constexpr int M = EQ::M, NP = LaneLayout<EQ, N, R>::NP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);
  double* staging = reinterpret_cast<double*>(smem_raw + PL::O_STAGE);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw + PL::O_BAR);
  const long long E = ma.E;
  const unsigned ntiles = (unsigned)((E + 31) / 32);
  auto whole = [&](unsigned t) { return PL::STAGE && ma.tma_ok && (long long)(t + 1) * 32 <= E; };
  auto pf_of = [&](unsigned t) {
    return Prefetch{u + (size_t)t * 32 * NP, E * NP, (unsigned)(32 * NP * sizeof(double)), staging, bar};
  };
  __shared__ double s_dt;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    s_dt = first ? step_begin(st, slot, ma.cfl, ma.dt_fixed, blockIdx.x == 0) : st->dt;
  }
  __syncthreads();
  const R dtR = dt_as<R>(s_dt);
  unsigned phase = 0;
  unsigned t = blockIdx.x;
  if (t < ntiles && whole(t) && threadIdx.x == 0) issue_prefetch<M>(pf_of(t));
  for (; t < ntiles; t += gridDim.x) {
    const bool staged = whole(t);
    if (staged) {
      const bool ok = mbar_wait_bounded(bar, phase);
      if (__syncthreads_or(!ok)) {
        // the copy may still be in flight: thread 0 waits for it once more
        // (bounded) before the CTA's shared memory is released
        if (threadIdx.x == 0) {
          atomicOr(&st->status, ST_TIMEOUT);
          mbar_wait_bounded(bar, phase);
        }
        return;
      }
      phase ^= 1u;
    }
    const unsigned tn = t + gridDim.x;
    const Prefetch pf = (tn < ntiles && whole(tn)) ? pf_of(tn) : Prefetch{nullptr, 0, 0, nullptr, nullptr};
    volume_lanes_tile<EQ, N, R, 0, S1, true>(u, rbar, trace, st, ma, pp, tb, (long long)t * 32, dtR, sm,
                                       staged ? staging : nullptr, pf);
    __syncthreads();   // shared memory is reused by the next tile
    if constexpr (!std::is_same<After, NoTileWork>::value) {
      after_tile((long long)t * 32, reinterpret_cast<const float*>(sm));
      __syncthreads();
    }
  }
}

template <class EQ, int N, typename R>
__global__ void __launch_bounds__(LaneLayout<EQ, N, R>::THREADS, LaneLayout<EQ, N, R>::MINB)
k_volume_lanes(const double* __restrict__ u, R* __restrict__ rbar, R* __restrict__ trace,
               DevState* __restrict__ st, const MeshArgs ma, const PhysParams<R> pp, const RefTab<R> tb,
               int slot) {
  volume_lanes_persistent<EQ, N, R, 0>(u, rbar, trace, st, ma, pp, tb, slot, true);
}

// The volume kernel of the limited FP32 step, which also evaluates the
// limiter's raw coefficients of every tile it has finished: rho p at the nodes
// from the tile's FP32 u^n (the same values k_alpha_raw converts), staged in
// the pair-data region, then one lane per element takes the energy fraction
// and the coefficient; near a clip threshold it leaves -1 for k_alpha_fix's
// FP64 evaluation (measured: the FP64 evaluation here stalled the tile on
// fronts, 110.2 against 108.5 us per step).  It also empties the touched list
// for k_alpha_smooth.
template <class EQ, int N, typename R>
__global__ void __launch_bounds__(LaneLayout<EQ, N, R>::THREADS, LaneLayout<EQ, N, R>::MINB)
k_volume_lanes_ind(const double* __restrict__ u, R* __restrict__ rbar, R* __restrict__ trace,
                   DevState* __restrict__ st, const MeshArgs ma, const PhysParams<R> pp, const RefTab<R> tb,
                   int slot, double* __restrict__ araw, unsigned* __restrict__ tcount, const LimTab lt) {
  static_assert(sizeof(R) == 4 && !EQ::NC, "the FP32 Euler form");
  using L = LaneLayout<EQ, N, R>;
  constexpr int DIM = EQ::DIM, n = N + 1, NP = L::NP;
  if (blockIdx.x == 0 && threadIdx.x == 0) *tcount = 0u;
  auto indicator = [&](long long e0, const float* sm) {
    float* smw = const_cast<float*>(sm);
    const int tid = threadIdx.x, l = tid >> 5, el = tid & 31;
    const int nel = (int)min(32LL, ma.E - e0);
    float* my = smw + (size_t)el * L::SZ;
    if (el < nel) {
      const float gm1 = ma.gamma_f - 1.0f;
#pragma unroll
      for (int k = 0; k < n; ++k) {
        const int p = l * n + k;
        const float rho = my[L::O_U0 + p], Et = my[L::O_U0 + (DIM + 1) * NP + p];
        float mm = 0.0f;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          const float mk = my[L::O_U0 + (1 + d) * NP + p];
          mm += mk * mk;
        }
        my[L::O_Q + p] = gm1 * (rho * Et - 0.5f * mm);
      }
    }
    __syncthreads();
    if (tid < 32 && el < nel) {
      const float En = indicator_of_values<EQ, N, float>([&](int p) { return my[L::O_Q + p]; }, lt);
      const float a = alpha_of_energy_f32(En, lt);
      araw[e0 + el] = a >= 0.0f ? f2d_int(a) : -1.0;   // k_alpha_fix takes it in FP64
    }
  };
  volume_lanes_persistent<EQ, N, R, 0>(u, rbar, trace, st, ma, pp, tb, slot, true, indicator);
}

// volume part of one RKFR stage (input: the stage state)
template <class EQ, int N, typename R>
__global__ void __launch_bounds__(LaneLayout<EQ, N, R>::THREADS, LaneLayout<EQ, N, R>::MINB)
k_volume_lanes_stage(const double* __restrict__ u, R* __restrict__ rbar, R* __restrict__ trace,
                     DevState* __restrict__ st, const MeshArgs ma, const PhysParams<R> pp, const RefTab<R> tb,
                     int slot, int first) {
  volume_lanes_persistent<EQ, N, R, 1>(u, rbar, trace, st, ma, pp, tb, slot, first != 0);
}

}  // namespace crk

namespace crk {

// ---------------------------------------------------------------------------
// Face + update kernel, lane form: 32 elements per CTA, warp = x-line index,
// lane = element.  Every face record a warp loads (own and neighbour) is a run
// of 32 consecutive elements of the [DIM][2][NF][C][E] trace array, and face
// membership is uniform across the warp.  u^n (FP64) and Rbar are staged
// through shared memory with coalesced loads; u^{n+1} leaves the same way.
// ---------------------------------------------------------------------------
template <class EQ, int N, typename R>
struct FaceLaneLayout {
  static constexpr int DIM = EQ::DIM, M = EQ::M, n = N + 1;
  static constexpr int NP = ipow(n, DIM), NF = NP / n;
  static constexpr int THREADS = 32 * NF;
  // jumps of the faces normal to y (and z): [DIM-1][side][face node][M][32 elements]
  static constexpr int NJ = (DIM - 1) * 2 * NF;
  static constexpr size_t bytes() { return sizeof(R) * (size_t)NJ * M * 32; }
  static constexpr bool fits() { return THREADS <= 1024 && bytes() <= 227 * 1024; }
};

// n contiguous values starting at src (vector loads where the alignment
// allows; COH: through L2, for data written earlier in the same launch)
template <int n, typename T, bool COH = false>
__device__ __forceinline__ void load_line(const T* __restrict__ src, T (&out)[n]) {
  if constexpr (sizeof(T) == 4 && n % 4 == 0) {
#pragma unroll
    for (int k = 0; k < n / 4; ++k) {
      const float4 t = ldx<COH>(reinterpret_cast<const float4*>(src) + k);
      out[4 * k] = t.x; out[4 * k + 1] = t.y; out[4 * k + 2] = t.z; out[4 * k + 3] = t.w;
    }
  } else if constexpr (sizeof(T) == 8 && n % 2 == 0) {
#pragma unroll
    for (int k = 0; k < n / 2; ++k) {
      const double2 t = ldx<COH>(reinterpret_cast<const double2*>(src) + k);
      out[2 * k] = t.x; out[2 * k + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < n; ++k) out[k] = ldx<COH>(src + k);
  }
}
template <int n>
__device__ __forceinline__ void store_line(float* __restrict__ dst, const float (&in)[n]) {
  if constexpr (n % 4 == 0) {
#pragma unroll
    for (int k = 0; k < n / 4; ++k)
      reinterpret_cast<float4*>(dst)[k] = make_float4(in[4 * k], in[4 * k + 1], in[4 * k + 2], in[4 * k + 3]);
  } else {
#pragma unroll
    for (int k = 0; k < n; ++k) dst[k] = in[k];
  }
}
template <int n>
__device__ __forceinline__ void store_line(double* __restrict__ dst, const double (&in)[n]) {
  if constexpr (n % 2 == 0) {
#pragma unroll
    for (int k = 0; k < n / 2; ++k) reinterpret_cast<double2*>(dst)[k] = make_double2(in[2 * k], in[2 * k + 1]);
  } else {
#pragma unroll
    for (int k = 0; k < n; ++k) dst[k] = in[k];
  }
}

// One tile of 32 elements starting at e0 (sj: the CTA's shared memory; slot:
// step parity of the CFL reduction).
//
// Phase A: every warp computes the Rusanov jumps of 2 DIM face nodes of each
// of its 32 elements: the two x-face nodes at the ends of its own x-line, and
// face node f = l of both faces normal to y (and z), whatever x-line they lie
// on, into shared memory -- the same record loads for every warp.
// Phase B: each thread forms the increment of its x-line (eq.
// crkfr.non.cons.final), the CFL reduction runs, and u^{n+1} is stored last,
// after the reduction's atomics.
// RK = true: stage mode of the multi-stage RKFR step (RkStage): the increment
// is the stage's K_j, combined with the earlier stages' into the next stage
// state (eq. rkfr1) or, at the last stage, into u^{n+1} (eq. rkfr2).
// FUSED: a tile of the fused single-launch step (crkfr_fused.cuh): dt comes
// from the caller (dt_fused), slot is the CFL reduction's write slot itself,
// and R-bar and the face records, written by other CTAs in the same launch,
// are read through L2.
// touched != nullptr (subcell blending limiter): the elements the limiter
// touches (blending coefficient of the element or of a face neighbour above
// zero, flagged by k_alpha_smooth) are left out -- k_face_update_limited takes
// them -- and u^{n+1} of the others goes to uout (the limited step keeps u^n
// intact).
template <class EQ, int N, typename R, bool RK = false, bool FUSED = false>
__device__ __forceinline__ void face_lanes_tile(double* __restrict__ u, const R* __restrict__ rbar,
                                                const R* __restrict__ trace, DevState* __restrict__ st,
                                                const MeshArgs& ma, const PhysParams<R>& pp, const RefTab<R>& tb,
                                                unsigned e0, int slot, R* __restrict__ sj,
                                                const RkStage<R>& rk = RkStage<R>{nullptr, nullptr, 0, 1},
                                                R dt_fused = R(0), const unsigned char* __restrict__ touched = nullptr,
                                                double* __restrict__ uout = nullptr) {
  using L = FaceLaneLayout<EQ, N, R>;
  constexpr int DIM = L::DIM, M = L::M, n = L::n, NP = L::NP, NF = L::NF;
  constexpr bool F32 = sizeof(R) == 4;
  const int tid = threadIdx.x;
  const int l = tid >> 5, el = tid & 31;
  const long long E = ma.E;
  // a volume CTA that timed out left its records unwritten: leave u^n as it is
  if constexpr (!FUSED) {
    if (st->status & ST_TIMEOUT) return;
  }
  const unsigned e = e0 + el;
  const bool active = (long long)e0 + el < E && !(touched && touched[e]);
  const R dtR = FUSED ? dt_fused : step_dt<R>(st);

  // own x-line: Rbar and u^n (N+1 contiguous values per variable), loads issued first
  R rb[M][n];
  double un[M][n];
  unsigned ec[3] = {0, 0, 0};
  R Jm[M], Jp[M];
  if (active) {
#pragma unroll
    for (int v = 0; v < M; ++v) {
      const size_t g = ((size_t)v * E + e) * NP + l * n;
      load_line<n, R, FUSED>(rbar + g, rb[v]);
      load_line<n>(u + g, un[v]);
    }
    elem_coords<DIM>(e, ma, ec);
    // ---- phase A: x faces at the own line's ends, face node l of the y / z faces
    face_jump<EQ, N, R, FUSED>(trace, E, 0, 1, e, neighbour_of(e, ec, 0, +1, ma), l, Jm, pp, tb);
    face_jump<EQ, N, R, FUSED>(trace, E, 0, 0, e, neighbour_of(e, ec, 0, -1, ma), l, Jp, pp, tb);
#pragma unroll
    for (int d = 1; d < DIM; ++d)
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        R J[M];
        face_jump<EQ, N, R, FUSED>(trace, E, d, side, e, neighbour_of(e, ec, d, side ? +1 : -1, ma), l, J, pp, tb);
        const R sc = side ? -(dtR * tb.iwN * inv_dx_of<R>(ma, d)) : dtR * tb.iw0 * inv_dx_of<R>(ma, d);
        R* dst = sj + ((size_t)(((d - 1) * 2 + side) * NF + l) * M) * 32 + el;
#pragma unroll
        for (int v = 0; v < M; ++v) dst[v * 32] = sc * J[v];
      }
  }
  if (DIM > 1) __syncthreads();

  // ---- phase B: increment of the own x-line, new state, CFL reduction, store
  R lam = R(0);
  bool bad = false;
  if (active) {
    const int cy = DIM >= 2 ? l % n : 0;
    const int cz = DIM == 3 ? l / n : 0;
    R du[n][M];
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int v = 0; v < M; ++v) du[k][v] = -dtR * rb[v][k];
    {
      // - dt J^- g_R'(1)/dx + dt J^+ (-g_L'(0))/dx at the x faces
      const R sR = dtR * tb.iwN * inv_dx_of<R>(ma, 0), sL = dtR * tb.iw0 * inv_dx_of<R>(ma, 0);
#pragma unroll
      for (int v = 0; v < M; ++v) { du[N][v] -= sR * Jm[v]; du[0][v] += sL * Jp[v]; }
    }
    // y / z faces: whole lines on the face (warp-uniform), scaled jumps from phase A
#pragma unroll
    for (int d = 1; d < DIM; ++d) {
      const int cd = d == 1 ? cy : cz;
      if (cd == 0 || cd == N) {
        const int side = cd == N ? 1 : 0;
#pragma unroll
        for (int k = 0; k < n; ++k) {
          const int f = d == 1 ? (k + n * cz) : (k + n * cy);
          const R* src = sj + ((size_t)(((d - 1) * 2 + side) * NF + f) * M) * 32 + el;
#pragma unroll
          for (int v = 0; v < M; ++v) du[k][v] += src[v * 32];
        }
      }
    }
    if constexpr (RK) {
      // du is this stage's K_j: keep it for the later stages and combine it
      // with the earlier ones (a_{j+1,q}, or b_q at the last stage)
      const bool last = rk.j == rk.s - 1;
      const size_t nodes = (size_t)E * NP;
#pragma unroll
      for (int v = 0; v < M; ++v) {
        const size_t g = ((size_t)v * E + e) * NP + l * n;
        R kj[n], acc[n];
        const R cj = last ? tb.b[rk.j] : tb.a[rk.j + 1][rk.j];
#pragma unroll
        for (int k = 0; k < n; ++k) { kj[k] = du[k][v]; acc[k] = cj * kj[k]; }
        if (!last) store_line<n>(rk.k + (size_t)rk.j * M * nodes + g, kj);
#pragma unroll 1
        for (int q = 0; q < rk.j; ++q) {
          const R c = last ? tb.b[q] : tb.a[rk.j + 1][q];
          if (c != R(0)) {
            R kq[n];
            load_line<n>(rk.k + (size_t)q * M * nodes + g, kq);
#pragma unroll
            for (int k = 0; k < n; ++k) acc[k] += c * kq[k];
          }
        }
#pragma unroll
        for (int k = 0; k < n; ++k) du[k][v] = acc[k];
      }
    }
    // u^{n+1} = u^n + du in FP64
#pragma unroll
    for (int k = 0; k < n; ++k) {
      double uu[M];
#pragma unroll
      for (int v = 0; v < M; ++v) {
        if constexpr (F32) uu[v] = un[v][k] + f2d_int(du[k][v]);
        else uu[v] = un[v][k] + du[k][v];
        un[v][k] = uu[v];
      }
      if (!RK || rk.j == rk.s - 1) {
        R lk;
        bad = bad || !physical_state<EQ, R>(uu, ma, lk);
        lam = fmax(lam, lk);
      }
    }
  }
  // the CFL reduction of the new state (RKFR: after the last stage only; the
  // stage index is uniform over the grid); intermediate stage states go to
  // rk.uout
  double* dst = uout ? uout : u;
  if (RK && rk.j != rk.s - 1) dst = rk.uout;
  else reduce_lambda<R>(lam, bad, st, FUSED ? slot : slot ^ 1);
  if (active) {
#pragma unroll
    for (int v = 0; v < M; ++v) store_line<n>(dst + ((size_t)v * E + e) * NP + l * n, un[v]);
  }
}

template <class EQ, int N, typename R>
__global__ void __launch_bounds__(FaceLaneLayout<EQ, N, R>::THREADS)
k_face_update_lanes(double* __restrict__ u, const R* __restrict__ rbar, const R* __restrict__ trace,
                    DevState* __restrict__ st, const MeshArgs ma, const PhysParams<R> pp, const RefTab<R> tb,
                    int slot) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  face_lanes_tile<EQ, N, R>(u, rbar, trace, st, ma, pp, tb, blockIdx.x * 32u, slot, reinterpret_cast<R*>(smem_raw));
}

// the limited step's elements that the limiter does not touch: the plain
// update from u^n (uin) into uout (touched: the flags of k_alpha_smooth)
template <class EQ, int N, typename R>
__global__ void __launch_bounds__(FaceLaneLayout<EQ, N, R>::THREADS)
k_face_update_lanes_clean(double* __restrict__ uin, double* __restrict__ uout, const R* __restrict__ rbar,
                          const R* __restrict__ trace, const unsigned char* __restrict__ touched,
                          DevState* __restrict__ st, const MeshArgs ma, const PhysParams<R> pp, const RefTab<R> tb,
                          int slot) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  face_lanes_tile<EQ, N, R>(uin, rbar, trace, st, ma, pp, tb, blockIdx.x * 32u, slot, reinterpret_cast<R*>(smem_raw),
                            RkStage<R>{nullptr, nullptr, 0, 1}, R(0), touched, uout);
}

// face / update part of stage rk.j of the multi-stage RKFR step
template <class EQ, int N, typename R>
__global__ void __launch_bounds__(FaceLaneLayout<EQ, N, R>::THREADS)
k_face_stage_lanes(double* __restrict__ u, const R* __restrict__ rbar, const R* __restrict__ trace,
                   DevState* __restrict__ st, const MeshArgs ma, const PhysParams<R> pp, const RefTab<R> tb,
                   int slot, const RkStage<R> rk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  face_lanes_tile<EQ, N, R, true>(u, rbar, trace, st, ma, pp, tb, blockIdx.x * 32u, slot,
                                  reinterpret_cast<R*>(smem_raw), rk);
}

// ---------------------------------------------------------------------------
// Batched persistent form: many independent solves of one degree.  Each
// persistent CTA walks a work list of 32-element tiles spanning all solves
// (grid-stride); the solve's mesh, buffers and step record come from a
// device table.
// ---------------------------------------------------------------------------
struct BatchSolve {
  MeshArgs ma;
  double* u;
  void* rbar;
  void* trace;
  DevState* st;
  unsigned ntiles;     // tiles of this solve
  unsigned pad;
};
struct BatchTile {
  unsigned solve;
  unsigned e0;
};

template <class EQ, int N, typename R, int SH = 0>
__global__ void __launch_bounds__(LaneLayout<EQ, N, R, SH>::THREADS, LaneLayout<EQ, N, R, SH>::MINB)
k_volume_batched(const BatchSolve* __restrict__ solves, const BatchTile* __restrict__ tiles, unsigned ntiles,
                 const PhysParams<R> pp, const RefTab<R> tb, int slot) {
  using PL = PersistLayout<EQ, N, R>;
  constexpr int M = EQ::M, NP = LaneLayout<EQ, N, R>::NP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);
  double* staging = reinterpret_cast<double*>(smem_raw + PL::O_STAGE);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw + PL::O_BAR);
  auto whole = [&](const BatchTile& t) {
    const BatchSolve& bs = solves[t.solve];
    return bs.ma.tma_ok && (long long)t.e0 + 32 <= bs.ma.E;
  };
  auto pf_of = [&](const BatchTile& t) {
    const BatchSolve& bs = solves[t.solve];
    return Prefetch{bs.u + (size_t)t.e0 * NP, bs.ma.E * NP, (unsigned)(32 * NP * sizeof(double)), staging, bar};
  };
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  unsigned phase = 0;
  unsigned it = blockIdx.x;
  if (it < ntiles && threadIdx.x == 0) {
    const BatchTile t0 = tiles[it];
    if (whole(t0)) issue_prefetch<M>(pf_of(t0));
  }
  for (; it < ntiles; it += gridDim.x) {
    const BatchTile t = tiles[it];
    const BatchSolve& bs = solves[t.solve];
    const bool staged = whole(t);
    if (staged) {
      const bool ok = mbar_wait_bounded(bar, phase);
      if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
          atomicOr(&bs.st->status, ST_TIMEOUT);
          mbar_wait_bounded(bar, phase);
        }
        return;
      }
      phase ^= 1u;
    }
    Prefetch pf{nullptr, 0, 0, nullptr, nullptr};
    if (it + gridDim.x < ntiles) {
      const BatchTile tn = tiles[it + gridDim.x];
      if (whole(tn)) pf = pf_of(tn);
    }
    const MeshArgs ma = bs.ma;
    // dt of this solve's step; its first tile records the step
    __shared__ double s_dt;
    if (threadIdx.x == 0) s_dt = step_begin(bs.st, slot, ma.cfl, ma.dt_fixed, t.e0 == 0);
    __syncthreads();
    volume_lanes_tile<EQ, N, R, SH>(bs.u, (R*)bs.rbar, (R*)bs.trace, bs.st, ma, pp, tb, (long long)t.e0,
                                dt_as<R>(s_dt), sm, staged ? staging : nullptr, pf);
    __syncthreads();   // shared memory is reused by the next tile
  }
}

template <class EQ, int N, typename R>
__global__ void __launch_bounds__(FaceLaneLayout<EQ, N, R>::THREADS)
k_face_batched(const BatchSolve* __restrict__ solves, const BatchTile* __restrict__ tiles, unsigned ntiles,
               const PhysParams<R> pp, const RefTab<R> tb, int slot) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (unsigned it = blockIdx.x; it < ntiles; it += gridDim.x) {
    const BatchTile t = tiles[it];
    const MeshArgs ma = solves[t.solve].ma;
    face_lanes_tile<EQ, N, R>(solves[t.solve].u, (const R*)solves[t.solve].rbar, (const R*)solves[t.solve].trace,
                              solves[t.solve].st, ma, pp, tb, t.e0, slot, reinterpret_cast<R*>(smem_raw));
    if (EQ::DIM > 1) __syncthreads();   // the jump buffer is reused by the next tile
  }
}

}  // namespace crk
