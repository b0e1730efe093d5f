// crkfr_volume_lanes.cuh -- volume kernel, lane form (sm_103a).
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
//    tableaux, N >= 4) stay in the owner's registers.
#pragma once
#include "crkfr_kernels.cuh"

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
                                              const PhysParams<R>& pp, const RefTab<R>& tb, R inv_dx) {
  constexpr int n = N + 1, M = EQ::M;
#pragma unroll
  for (int k = 0; k < n; ++k)
#pragma unroll
    for (int v = 0; v < M; ++v) acc[k][v] = R(0);
  {
    R f[M];
    EQ::flux(D, q[0], f, pp);
#pragma unroll
    for (int v = 0; v < M; ++v) acc[0][v] = R(2) * tb.D[0][0] * f[v];
    EQ::flux(D, q[N], f, pp);
#pragma unroll
    for (int v = 0; v < M; ++v) acc[N][v] = R(2) * tb.D[N][N] * f[v];
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

template <class EQ, int N, typename R>
struct LaneLayout {
  static constexpr int DIM = EQ::DIM, M = EQ::M, P = EQ::P, n = N + 1;
  static constexpr int NP = ipow(n, DIM), NF = NP / n, S = rk_stages(N);
  static constexpr int FACE = DIM * M * 2 * NF;            // [DIM][M][2][NF]
  static constexpr int O_Q = 0;                            // [P][NP] pair data (also staging)
  static constexpr int O_RY = O_Q + P * NP;                // [M][NP] y (+z) residual
  static constexpr int O_UB = O_RY + (DIM > 1 ? M * NP : 0);   // [M][NP] time-averaged U (face nodes)
  static constexpr int O_FB = O_UB + M * NP;               // time-averaged F^d at d-faces
  static constexpr int O_FN = O_FB + FACE;                 // GLM-MHD: time-averaged F^nc,d
  static constexpr int O_UN = O_FN + (EQ::NC ? FACE : 0);  // GLM-MHD: u^n at d-faces
  static constexpr int O_LAM = O_UN + (EQ::NC ? FACE : 0); // [DIM][2][NF] lambda_d(u^n)
  static constexpr int SZ0 = O_LAM + DIM * 2 * NF;
  static constexpr int SZ = SZ0 | 1;                       // odd element stride: no bank conflicts
  static constexpr int EPB = 32;
  static constexpr int THREADS = 32 * NF;
  static constexpr size_t bytes() { return sizeof(R) * (size_t)SZ * EPB; }
  // CTAs per SM the register allocation aims at (Euler with small lines:
  // 5 x 128 threads = 20 warps; larger variants are limited by registers anyway)
  static constexpr int MINB = (!EQ::NC && THREADS <= 128) ? 5 : 1;
  static constexpr bool fits() { return bytes() <= 227 * 1024 && THREADS <= 1024; }
};

// One tile of 32 elements starting at e0 (the CTA's whole shared memory sm).
template <class EQ, int N, typename R>
__device__ __forceinline__ void volume_lanes_tile(const double* __restrict__ u, R* __restrict__ rbar,
                                                  R* __restrict__ trace, const DevState* __restrict__ st,
                                                  const MeshArgs& ma, const PhysParams<R>& pp, const RefTab<R>& tb,
                                                  long long e0, R* sm) {
  using L = LaneLayout<EQ, N, R>;
  constexpr int DIM = L::DIM, M = L::M, P = L::P, n = L::n, NP = L::NP, NF = L::NF, S = L::S;
  constexpr int C = trace_comps<EQ>();
  constexpr int NS = rk_nsaved(N) > 0 ? rk_nsaved(N) : 1;

  const int tid = threadIdx.x;
  const int l = tid >> 5;              // line index (warp-uniform)
  const int el = tid & 31;             // element within the CTA
  const long long E = ma.E;
  const int nel = (int)min(32LL, E - e0);
  const bool active = el < nel;
  R* my = sm + (size_t)el * L::SZ;

  R dtR;
  if constexpr (sizeof(R) == 4) dtR = st->dt_next_f;
  else dtR = st->dt_next;

  // coordinates of this thread's x-line in the other directions (warp-uniform)
  int cy = 0, cz = 0;
  if (DIM >= 2) cy = l % n;
  if (DIM == 3) cz = l / n;
  const bool yface = DIM >= 2 && (cy == 0 || cy == N);
  const bool zface = DIM == 3 && (cz == 0 || cz == N);

  // ---- u^n: coalesced into shared memory (staging in the Q region), then own x-line to registers
  // (index arithmetic with compile-time divisors only)
#pragma unroll 4
  for (int it = 0; it < (M * 32 * NP + L::THREADS - 1) / L::THREADS; ++it) {
    const int idx = tid + it * L::THREADS;
    const int v = idx / (32 * NP), r = idx % (32 * NP);
    const int ee = r / NP, p = r % NP;
    if (v < M && ee < nel) {
      const double x = u[((size_t)v * E + e0) * NP + r];
      if constexpr (sizeof(R) == 4) sm[(size_t)ee * L::SZ + L::O_Q + v * NP + p] = d2f_int(x);
      else sm[(size_t)ee * L::SZ + L::O_Q + v * NP + p] = x;
    }
  }
  __syncthreads();
  R u0[n][M];
#pragma unroll
  for (int k = 0; k < n; ++k)
#pragma unroll
    for (int v = 0; v < M; ++v) u0[k][v] = active ? my[L::O_Q + v * NP + l * n + k] : R(1);
  __syncthreads();

  R rb[n][M], ax[n][M], rs[NS][n][M];
#pragma unroll
  for (int k = 0; k < n; ++k)
#pragma unroll
    for (int v = 0; v < M; ++v) { rb[k][v] = R(0); ax[k][v] = R(0); }

  // the stage loop stays rolled: one stage's code is large, and S copies of it
  // would overflow the instruction cache; the tableau comes from the parameters
#pragma unroll 1
  for (int i = 0; i < S; ++i) {
    // ---------------- node phase (own x-line)
    R q[n][P];
    if (active) {
#pragma unroll
      for (int k = 0; k < n; ++k) {
        const int p = l * n + k;
        R uu[M];
#pragma unroll
        for (int v = 0; v < M; ++v) {
          R acc = R(0);
          if (i > 0) {
            // complete R_{i-1} = x part (registers) + y/z part (shared)
            R r = ax[k][v] + (DIM > 1 ? my[L::O_RY + v * NP + p] : R(0));
            rb[k][v] += tb.b[i - 1] * r;
            acc = tb.a[i][i - 1] * r;
            if constexpr (rk_nsaved(N) > 0) {
              if (tb.slot[i - 1] >= 0) rs[tb.slot[i - 1]][k][v] = r;
              for (int j = 0; j < i - 1; ++j)
                if (tb.slot[j] >= 0) acc += tb.a[i][j] * rs[tb.slot[j]][k][v];
            }
          }
          uu[v] = u0[k][v] - dtR * acc;
        }
        EQ::pair_data(uu, q[k], pp);
        if (DIM > 1) {
#pragma unroll
          for (int c = 0; c < P; ++c) my[L::O_Q + c * NP + p] = q[k][c];
        }
        // face sums of the time averages: x faces at k = 0, N; y/z faces per line
        const bool xf = (k == 0 || k == N);
        const bool onface = xf || yface || zface;
        if (i == 0 && onface) {
          if (xf) my[L::O_LAM + (0 * 2 + (k == N)) * NF + l] = EQ::wave_speed(0, q[k], pp);
          if (yface) my[L::O_LAM + (1 * 2 + (cy == N)) * NF + (k + n * cz)] = EQ::wave_speed(1, q[k], pp);
          if (zface) my[L::O_LAM + (2 * 2 + (cz == N)) * NF + (k + n * cy)] = EQ::wave_speed(DIM - 1, q[k], pp);
          if constexpr (EQ::NC) {
#pragma unroll
            for (int v = 0; v < M; ++v) {
              if (xf) my[L::O_UN + ((0 * M + v) * 2 + (k == N)) * NF + l] = uu[v];
              if (yface) my[L::O_UN + ((1 * M + v) * 2 + (cy == N)) * NF + k] = uu[v];
            }
          }
        }
        const R b = tb.b[i];
        if (b != R(0) && onface) {
#pragma unroll
          for (int v = 0; v < M; ++v) {
            R* ub = &my[L::O_UB + v * NP + p];
            *ub = (i == 0 ? R(0) : *ub) + b * uu[v];
          }
#pragma unroll
          for (int d = 0; d < DIM; ++d) {
            bool on = d == 0 ? xf : d == 1 ? yface : zface;
            if (!on) continue;
            const int side = d == 0 ? (k == N) : d == 1 ? (cy == N) : (cz == N);
            const int f = d == 0 ? l : d == 1 ? (k + n * cz) : (k + n * cy);
            R fl[M];
            EQ::flux(d, q[k], fl, pp);
#pragma unroll
            for (int v = 0; v < M; ++v) {
              R* fb = &my[L::O_FB + ((d * M + v) * 2 + side) * NF + f];
              *fb = (i == 0 ? R(0) : *fb) + b * fl[v];
            }
            if constexpr (EQ::NC) {
              R g[2], nc[M];
#pragma unroll
              for (int v = 0; v < M; ++v) nc[v] = R(0);
              EQ::ncg(d, q[k], g);
              EQ::nc_apply(d, q[k], g, nc);
#pragma unroll
              for (int v = 0; v < M; ++v) {
                R* fn = &my[L::O_FN + ((d * M + v) * 2 + side) * NF + f];
                *fn = (i == 0 ? R(0) : *fn) + b * nc[v];
              }
            }
          }
        }
      }
      // ---------------- x-direction flux differencing, all in registers
      line_residual<EQ, N, R, 0>(q, ax, pp, tb, inv_dx_of<R>(ma, 0));
    }
    if (DIM > 1) {
      __syncthreads();   // Q of this stage visible; RY of the last stage consumed
      if (active) {
        // y-line l: nodes (i = l % n, j = 0..N, k = l / n)
        const int base = (l % n) + (l / n) * n * n;
        R qy[n][P], ay[n][M];
#pragma unroll
        for (int k = 0; k < n; ++k)
#pragma unroll
          for (int c = 0; c < P; ++c) qy[k][c] = my[L::O_Q + c * NP + base + k * n];
        line_residual<EQ, N, R, (DIM > 1 ? 1 : 0)>(qy, ay, pp, tb, inv_dx_of<R>(ma, 1));
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
          R qz[n][P], az[n][M];
#pragma unroll
          for (int k = 0; k < n; ++k)
#pragma unroll
            for (int c = 0; c < P; ++c) qz[k][c] = my[L::O_Q + c * NP + base + k * n * n];
          line_residual<EQ, N, R, DIM - 1>(qz, az, pp, tb, inv_dx_of<R>(ma, DIM - 1));
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
        R r = ax[k][v] + (DIM > 1 ? my[L::O_RY + v * NP + p] : R(0));
        my[L::O_Q + v * NP + p] = rb[k][v] + tb.b[S - 1] * r;
      }
    }
  }
  __syncthreads();
#pragma unroll 4
  for (int it = 0; it < (M * 32 * NP + L::THREADS - 1) / L::THREADS; ++it) {
    const int idx = tid + it * L::THREADS;
    const int v = idx / (32 * NP), r = idx % (32 * NP);
    const int ee = r / NP, p = r % NP;
    if (v < M && ee < nel) rbar[((size_t)v * E + e0) * NP + r] = sm[(size_t)ee * L::SZ + L::O_Q + v * NP + p];
  }
  // ---- face traces [DIM][2][NF][E][CP]: thread (warp l, lane el) writes the
  // record of face node f = l of element el, CP values with 16-byte stores;
  // consecutive lanes write consecutive records
  constexpr int CP = trace_stride<EQ, R>();
  if (active) {
    const int f = l;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const int stride = ipow(n, d);
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int p = line_base<n>(f, stride) + side * N * stride;
        R rec[CP];
#pragma unroll
        for (int v = 0; v < M; ++v) {
          rec[v] = my[L::O_UB + v * NP + p];
          rec[M + v] = my[L::O_FB + ((d * M + v) * 2 + side) * NF + f];
        }
        rec[2 * M] = my[L::O_LAM + (d * 2 + side) * NF + f];
        if constexpr (EQ::NC) {
#pragma unroll
          for (int v = 0; v < M; ++v) {
            rec[2 * M + 1 + v] = my[L::O_FN + ((d * M + v) * 2 + side) * NF + f];
            rec[3 * M + 1 + v] = my[L::O_UN + ((d * M + v) * 2 + side) * NF + f];
          }
        }
#pragma unroll
        for (int c = C; c < CP; ++c) rec[c] = R(0);
        store_record<R, CP>(trace + ((((size_t)(d * 2 + side) * NF + f) * E) + e0 + el) * CP, rec);
      }
    }
  }
}

template <class EQ, int N, typename R>
__global__ void __launch_bounds__(LaneLayout<EQ, N, R>::THREADS, LaneLayout<EQ, N, R>::MINB)
k_volume_lanes(const double* __restrict__ u, R* __restrict__ rbar, R* __restrict__ trace,
               DevState* __restrict__ st, const MeshArgs ma, const PhysParams<R> pp, const RefTab<R> tb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  volume_lanes_tile<EQ, N, R>(u, rbar, trace, st, ma, pp, tb, (long long)blockIdx.x * 32,
                              reinterpret_cast<R*>(smem_raw));
}

}  // namespace crk

namespace crk {

// ---------------------------------------------------------------------------
// Face + update kernel, lane form: 32 elements per CTA, warp = x-line index,
// lane = element.  Every face record a warp loads (own and neighbour) is a run
// of 32 consecutive records of the [DIM][2][NF][E][CP] trace array, and face
// membership is uniform across the warp.  u^n (FP64) and Rbar are staged
// through shared memory with coalesced loads; u^{n+1} leaves the same way.
// ---------------------------------------------------------------------------
template <class EQ, int N, typename R>
struct FaceLaneLayout {
  static constexpr int DIM = EQ::DIM, M = EQ::M, n = N + 1;
  static constexpr int NP = ipow(n, DIM), NF = NP / n;
  static constexpr int THREADS = 32 * NF;
  static constexpr size_t bytes() { return 0; }
  static constexpr bool fits() { return THREADS <= 1024; }
};

// n contiguous values starting at src (vector loads where the alignment allows)
template <int n, typename T>
__device__ __forceinline__ void load_line(const T* __restrict__ src, T (&out)[n]) {
  if constexpr (sizeof(T) == 4 && n % 4 == 0) {
#pragma unroll
    for (int k = 0; k < n / 4; ++k) {
      const float4 t = reinterpret_cast<const float4*>(src)[k];
      out[4 * k] = t.x; out[4 * k + 1] = t.y; out[4 * k + 2] = t.z; out[4 * k + 3] = t.w;
    }
  } else if constexpr (sizeof(T) == 8 && n % 2 == 0) {
#pragma unroll
    for (int k = 0; k < n / 2; ++k) {
      const double2 t = reinterpret_cast<const double2*>(src)[k];
      out[2 * k] = t.x; out[2 * k + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < n; ++k) out[k] = src[k];
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

// One tile of 32 elements starting at e0; total_warps = warps of all tiles of
// this solve in the launch (for the barrier-free CFL reduction).
template <class EQ, int N, typename R>
__device__ __forceinline__ void face_lanes_tile(double* __restrict__ u, const R* __restrict__ rbar,
                                                const R* __restrict__ trace, DevState* __restrict__ st,
                                                const MeshArgs& ma, const PhysParams<R>& pp, const RefTab<R>& tb,
                                                unsigned e0, unsigned total_warps) {
  using L = FaceLaneLayout<EQ, N, R>;
  constexpr int DIM = L::DIM, M = L::M, n = L::n, NP = L::NP;
  constexpr bool F32 = sizeof(R) == 4;
  const int tid = threadIdx.x;
  const int l = tid >> 5, el = tid & 31;
  const long long E = ma.E;
  const bool active = (long long)e0 + el < E;

  R lam = R(0);
  bool bad = false;
  if (active) {
    const unsigned e = e0 + el;
    R dtR;
    if constexpr (F32) dtR = st->dt_next_f;
    else dtR = st->dt_next;
    // own x-line: Rbar and u^n (N+1 contiguous values per variable)
    R rb[M][n];
    double un[M][n];
#pragma unroll
    for (int v = 0; v < M; ++v) {
      const size_t g = ((size_t)v * E + e) * NP + l * n;
      load_line<n>(rbar + g, rb[v]);
      load_line<n>(u + g, un[v]);
    }
    unsigned ec[3] = {0, 0, 0};
    elem_coords<DIM>(e, ma, ec);
    const int cy = DIM >= 2 ? l % n : 0;
    const int cz = DIM == 3 ? l / n : 0;
    R du[n][M];
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int v = 0; v < M; ++v) du[k][v] = -dtR * rb[v][k];
    // x faces at the line ends (eq. crkfr.non.cons.final: - dt J^- g_R'(1)/dx + dt J^+ (-g_L'(0))/dx)
    {
      R Jm[M], Jp[M];
      face_jump<EQ, N, R>(trace, E, 0, 1, e, neighbour_of(e, ec, 0, +1, ma), l, Jm, pp);
      face_jump<EQ, N, R>(trace, E, 0, 0, e, neighbour_of(e, ec, 0, -1, ma), l, Jp, pp);
      const R sR = dtR * tb.iwN * inv_dx_of<R>(ma, 0), sL = dtR * tb.iw0 * inv_dx_of<R>(ma, 0);
#pragma unroll
      for (int v = 0; v < M; ++v) { du[N][v] -= sR * Jm[v]; du[0][v] += sL * Jp[v]; }
    }
    // y / z faces: whole lines on the face (warp-uniform)
#pragma unroll
    for (int d = 1; d < DIM; ++d) {
      const int cd = d == 1 ? cy : cz;
      if (cd == 0 || cd == N) {
        const int side = cd == N ? 1 : 0;
        const unsigned nb = neighbour_of(e, ec, d, side ? +1 : -1, ma);
        const R s = side ? -(dtR * tb.iwN * inv_dx_of<R>(ma, d)) : dtR * tb.iw0 * inv_dx_of<R>(ma, d);
#pragma unroll
        for (int k = 0; k < n; ++k) {
          const int f = d == 1 ? (k + n * cz) : (k + n * cy);
          R J[M];
          face_jump<EQ, N, R>(trace, E, d, side, e, nb, f, J, pp);
#pragma unroll
          for (int v = 0; v < M; ++v) du[k][v] += s * J[v];
        }
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
      R lk;
      bad = bad || !physical_state<EQ, R>(uu, ma, lk);
      lam = fmax(lam, lk);
    }
#pragma unroll
    for (int v = 0; v < M; ++v) store_line<n>(u + ((size_t)v * E + e) * NP + l * n, un[v]);
  }
  finalize_warps<R>(lam, bad, st, total_warps, true, ma.cfl, ma.dt_fixed);
}

template <class EQ, int N, typename R>
__global__ void __launch_bounds__(FaceLaneLayout<EQ, N, R>::THREADS)
k_face_update_lanes(double* __restrict__ u, const R* __restrict__ rbar, const R* __restrict__ trace,
                    DevState* __restrict__ st, double* __restrict__ partials, const MeshArgs ma,
                    const PhysParams<R> pp, const RefTab<R> tb) {
  face_lanes_tile<EQ, N, R>(u, rbar, trace, st, ma, pp, tb, blockIdx.x * 32u,
                            gridDim.x * (FaceLaneLayout<EQ, N, R>::THREADS / 32));
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

template <class EQ, int N, typename R>
__global__ void __launch_bounds__(LaneLayout<EQ, N, R>::THREADS, LaneLayout<EQ, N, R>::MINB)
k_volume_batched(const BatchSolve* __restrict__ solves, const BatchTile* __restrict__ tiles, unsigned ntiles,
                 const PhysParams<R> pp, const RefTab<R> tb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (unsigned it = blockIdx.x; it < ntiles; it += gridDim.x) {
    const BatchTile t = tiles[it];
    const MeshArgs ma = solves[t.solve].ma;
    volume_lanes_tile<EQ, N, R>(solves[t.solve].u, (R*)solves[t.solve].rbar, (R*)solves[t.solve].trace,
                                solves[t.solve].st, ma, pp, tb, (long long)t.e0, reinterpret_cast<R*>(smem_raw));
    __syncthreads();   // shared memory is reused by the next tile
  }
}

template <class EQ, int N, typename R>
__global__ void __launch_bounds__(FaceLaneLayout<EQ, N, R>::THREADS)
k_face_batched(const BatchSolve* __restrict__ solves, const BatchTile* __restrict__ tiles, unsigned ntiles,
               const PhysParams<R> pp, const RefTab<R> tb) {
  constexpr unsigned WPT = FaceLaneLayout<EQ, N, R>::THREADS / 32;   // warps per tile
  for (unsigned it = blockIdx.x; it < ntiles; it += gridDim.x) {
    const BatchTile t = tiles[it];
    const MeshArgs ma = solves[t.solve].ma;
    face_lanes_tile<EQ, N, R>(solves[t.solve].u, (const R*)solves[t.solve].rbar, (const R*)solves[t.solve].trace,
                              solves[t.solve].st, ma, pp, tb, t.e0, solves[t.solve].ntiles * WPT);
  }
}

}  // namespace crk
