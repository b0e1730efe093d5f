// crkfr_limiter.cuh -- the subcell blending limiter of the cRKFR step (the
// paper's Sec. 4 runs blend the update with a first-order subcell finite-volume
// update, the blending coefficient capped by alpha_max; compressible Euler).
//
//  k_alpha_raw           per element: the modal smoothness indicator of rho p
//                        (energy fraction of the highest orthonormal Legendre
//                        modes), the logistic map, its clips and the cap
//                        alpha_max; FP64, or in the FP32 form FP32 with the
//                        FP64 evaluation near the clip thresholds.  One thread
//                        per element.
//  k_alpha_smooth        per element: a_e = max(raw_e, raw_nb / 2 over the
//                        face neighbours), and whether the limiter touches
//                        the element (a_e or a face neighbour's a above zero,
//                        i.e. a raw value above zero within two face steps).
//  k_face_update_limited per node: the cRKFR update u^H with the limited face
//                        flux at element faces, the first-order subcell update
//                        u^L with the same face flux, the blend
//                        (1 - a_e) u^H + a_e u^L into the other state buffer,
//                        and the CFL reduction of the result.  Where the lane
//                        face kernel exists it takes the elements the limiter
//                        does not touch (a = 0 there and at every face
//                        neighbour: the plain update, k_face_update_lanes_clean)
//                        and this kernel only the others.
//
// The limited face flux at a face node between elements '-' and '+':
//   F_blend = (1 - a_f) F^num + a_f f_lo   (f_lo alone where a_f = 1),
//   a_f = (a_- + a_+)/2, F^num the time-averaged Rusanov flux of eq.
//   numflux.cons (records of the volume kernel), f_lo the Rusanov flux of the
//   two u^n traces; where a_f > 0, F = f_lo + theta (F_blend - f_lo) with the
//   largest theta in [0,1] that keeps rho and p of both adjacent end
//   subcells' one-direction low-order states at or above a tenth of their
//   values with f_lo.  Both elements evaluate it from the same '-'/'+' data
//   in the same order, so they get the same bits and the step conserves.
//
// u^n is read from one state buffer and u^{n+1} written to the other (the
// first-order fluxes read neighbouring nodes of other elements), so a limited
// context ping-pongs between two buffers.
#pragma once
#include <type_traits>

#include "crkfr_kernels.cuh"

namespace crk {

// Host-filled tables of the limiter.
struct LimTab {
  double vinv[6][6];   // orthonormal Legendre modes from GLL node values: m_j = sum_p vinv[j][p] v_p
  double w01[6];       // GLL weights on [0,1] (subcell widths / dx)
  double tau, sharp;   // logistic threshold 0.5 10^(-1.8 (N+1)^(1/4)) and sharpness ln 9999
  double alpha_max;
  // FP32 form: the same tables in FP32, and the energy fractions at which the
  // logistic map crosses the clips (alpha = 0.001: tau (1 + ln(0.001/0.999)/sharp),
  // alpha = 0.999: tau (1 + ln(0.999/0.001)/sharp))
  float vinv_f[6][6];
  float tau_f, sharp_f, alpha_max_f, e_lo_f, e_hi_f;
};


// The energy fraction of one element from its rho p node values, load(p) for
// node p (the values stay in this function's registers).
template <class EQ, int N, typename T, class Load>
__device__ __forceinline__ T indicator_of_values(Load load, const LimTab& lt) {
  constexpr int DIM = EQ::DIM, n = N + 1, NP = ipow(n, DIM);
  constexpr bool F32 = sizeof(T) == 4;
  T m[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) m[p] = load(p);
  // modal coefficients: the 1D transform along every direction in turn (fully
  // unrolled: compile-time indices keep the element's values in registers)
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int stride = ipow(n, d);
#pragma unroll
    for (int l = 0; l < NP / n; ++l) {
      const int base = line_base<n>(l, stride);
      T t[n];
#pragma unroll
      for (int j = 0; j < n; ++j) {
        T acc = T(0);
#pragma unroll
        for (int p = 0; p < n; ++p) acc += (F32 ? T(lt.vinv_f[j][p]) : T(lt.vinv[j][p])) * m[base + p * stride];
        t[j] = acc;
      }
#pragma unroll
      for (int j = 0; j < n; ++j) m[base + j * stride] = t[j];
    }
  }
  // energy of all modes, of those of degree <= N-1 and <= N-2 in every direction
  // (FP32: of those of degree N and N-1 at most, summed directly)
  T tot = T(0), a1 = T(0), a2 = T(0);
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    int rem = p, top = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      const int j = rem % n;
      rem /= n;
      top = j > top ? j : top;
    }
    const T e2 = m[p] * m[p];
    tot += e2;
    if constexpr (F32) {
      if (top == N) a1 += e2;
      if (top == N - 1) a2 += e2;
    } else {
      if (top <= N - 1) a1 += e2;
      if (top <= N - 2) a2 += e2;
    }
  }
  T En;
  if constexpr (F32) {
    En = a1 / tot;
    if (N >= 2) En = fmax(En, a2 / (tot - a1));
  } else {
    En = (tot - a1) / tot;
    if (N >= 2) En = fmax(En, (a1 - a2) / a1);
  }
  return En;
}

// Energy fraction of the highest modes of one element's rho p (see
// k_alpha_raw).  FP64: E = max((T - T1)/T, (T1 - T2)/T1) from the three sums;
// FP32: the top and second-top energies summed directly (sums of squares, no
// cancellation), E = max(Ttop/T, Tsec/(T - Ttop)).
template <class EQ, int N, typename T>
__device__ __forceinline__ T indicator_energy(const double* __restrict__ u, long long E, long long e,
                                              const MeshArgs& ma, const LimTab& lt) {
  constexpr int DIM = EQ::DIM, NP = ipow(N + 1, DIM);
  constexpr bool F32 = sizeof(T) == 4;
  return indicator_of_values<EQ, N, T>([&](int p) {
    T rho, Et, mm = T(0);
    if constexpr (F32) {
      rho = d2f_int(u[(size_t)e * NP + p]);
      Et = d2f_int(u[((size_t)(DIM + 1) * E + e) * NP + p]);
    } else {
      rho = u[(size_t)e * NP + p];
      Et = u[((size_t)(DIM + 1) * E + e) * NP + p];
    }
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      T mk;
      if constexpr (F32) mk = d2f_int(u[((size_t)(1 + k) * E + e) * NP + p]);
      else mk = u[((size_t)(1 + k) * E + e) * NP + p];
      mm += mk * mk;
    }
    // rho p = (gamma - 1)(rho E - |m|^2 / 2)
    const T gm1 = F32 ? T(ma.gamma_f - 1.0f) : T(ma.gamma - 1.0);
    return gm1 * (rho * Et - T(0.5) * mm);
  }, lt);
}

// FP32 form: the raw coefficient of an FP32 energy fraction, or -1 where it
// lies within 2% of a clip threshold (the FP64 evaluation decides there).
__device__ __forceinline__ float alpha_of_energy_f32(float En, const LimTab& lt) {
  const bool near = fabsf(En - lt.e_lo_f) <= 0.02f * lt.e_lo_f || fabsf(En - lt.e_hi_f) <= 0.02f * lt.e_hi_f;
  if (near) return -1.0f;
  const float a = En < lt.e_lo_f ? 0.0f : En > lt.e_hi_f ? 1.0f
                                  : 1.0f / (1.0f + expf(-(lt.sharp_f / lt.tau_f) * (En - lt.tau_f)));
  return fminf(a, lt.alpha_max_f);
}

// The raw coefficient in FP64 from u^n in global memory (the FP32 form's
// elements near a clip threshold).
template <class EQ, int N>
__device__ __forceinline__ double alpha_raw_fp64(const double* __restrict__ u, long long E, long long e,
                                              const MeshArgs& ma, const LimTab& lt) {
  const double En = indicator_energy<EQ, N, double>(u, E, e, ma, lt);
  double a = 1.0 / (1.0 + exp(-(lt.sharp / lt.tau) * (En - lt.tau)));
  if (a < 0.001) a = 0.0;
  if (a > 0.999) a = 1.0;
  return fmin(a, lt.alpha_max);
}

// The FP64 evaluation of the raw coefficients the FP32 volume kernel left
// at -1 (near a clip threshold).
template <class EQ, int N>
__global__ void __launch_bounds__(128)
k_alpha_fix(const double* __restrict__ u, double* __restrict__ araw, const MeshArgs ma, const LimTab lt) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < ma.E && araw[e] < 0.0) araw[e] = alpha_raw_fp64<EQ, N>(u, ma.E, e, ma, lt);
}

// Elements per block of k_alpha_raw (one thread each) when their rho p values
// fit the static shared memory (48 KB), else 0: every thread reads its own
// element's values from global memory.
template <class EQ, int N, typename R>
struct AlphaRawLayout {
  using T = typename std::conditional<sizeof(R) == 4, float, double>::type;
  static constexpr int NP = ipow(N + 1, EQ::DIM);
  static constexpr int FIT = 49152 / (int)((NP + 1) * sizeof(T)) / 32 * 32;
  static constexpr int EB = FIT >= 128 ? 128 : FIT >= 32 ? FIT : 0;
  static constexpr int THREADS = EB > 0 ? EB : 128;
};

// ---------------------------------------------------------------------------
// Blending coefficient per element before smoothing.  The FP64 form evaluates
// it in FP64 throughout.  The FP32 form evaluates the energy fraction in FP32
// and takes the FP64 evaluation for the elements whose FP32 value lies within
// 2% of a clip threshold, so every clip decision is the FP64 one (the FP32
// value's relative error is below 1e-4 there); elsewhere the logistic map in
// FP32 differs from the FP64 one by about 1e-6.
// ---------------------------------------------------------------------------
template <class EQ, int N, typename R>
__global__ void __launch_bounds__(AlphaRawLayout<EQ, N, R>::THREADS)
k_alpha_raw(const double* __restrict__ u, double* __restrict__ araw, unsigned* __restrict__ tcount, const MeshArgs ma,
            const LimTab lt) {
  constexpr int DIM = EQ::DIM, NP = ipow(N + 1, DIM), EB = AlphaRawLayout<EQ, N, R>::EB;
  using T = typename AlphaRawLayout<EQ, N, R>::T;
  const long long E = ma.E;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  // the touched list of this step starts empty (k_alpha_smooth fills it after
  // this kernel; the last step's limited kernel has read it before)
  if (e == 0) *tcount = 0u;
  const T* row = nullptr;
  if constexpr (EB > 0) {
    // rho p of the block's EB elements through shared memory: coalesced loads
    // of the block's contiguous slice of every variable, one row of NP + 1
    // values per element (no bank conflicts when each thread reads its row)
    __shared__ T s_m[EB > 0 ? EB * (NP + 1) : 1];
    const long long e0 = (long long)blockIdx.x * EB;
    const int nel = (int)min((long long)EB, E - e0);
    const size_t vs = (size_t)E * NP;
    const T gm1 = sizeof(T) == 4 ? T(ma.gamma_f - 1.0f) : T(ma.gamma - 1.0);
    for (int r = threadIdx.x; r < nel * NP; r += EB) {
      const size_t g = (size_t)e0 * NP + r;
      T rho, Et, mm = T(0);
      if constexpr (sizeof(T) == 4) {
        rho = d2f_int(u[g]);
        Et = d2f_int(u[(DIM + 1) * vs + g]);
      } else {
        rho = u[g];
        Et = u[(DIM + 1) * vs + g];
      }
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        T mk;
        if constexpr (sizeof(T) == 4) mk = d2f_int(u[(1 + k) * vs + g]);
        else mk = u[(1 + k) * vs + g];
        mm += mk * mk;
      }
      s_m[(r / NP) * (NP + 1) + r % NP] = gm1 * (rho * Et - T(0.5) * mm);
    }
    __syncthreads();
    row = s_m + threadIdx.x * (NP + 1);
  }
  auto from_row = [&](int p) { return row[p]; };
  if (e >= E) return;
  if constexpr (sizeof(R) == 4) {
    float En;
    if constexpr (EB > 0) En = indicator_of_values<EQ, N, float>(from_row, lt);
    else En = indicator_energy<EQ, N, float>(u, E, e, ma, lt);
    const float a = alpha_of_energy_f32(En, lt);
    if (a >= 0.0f) {
      araw[e] = f2d_int(a);
      return;
    }
  }
  double En;
  if constexpr (sizeof(R) == 8 && EB > 0) En = indicator_of_values<EQ, N, double>(from_row, lt);
  else En = indicator_energy<EQ, N, double>(u, E, e, ma, lt);
  double a = 1.0 / (1.0 + exp(-(lt.sharp / lt.tau) * (En - lt.tau)));
  if (a < 0.001) a = 0.0;
  if (a > 0.999) a = 1.0;
  araw[e] = fmin(a, lt.alpha_max);
}

// one element of k_alpha_smooth; returns whether the limiter touches it
template <int DIM>
__device__ __forceinline__ bool alpha_smooth_one(const double* __restrict__ araw, double* __restrict__ alpha,
                                                      unsigned char* __restrict__ touched, const MeshArgs& ma,
                                                      unsigned e) {
  const unsigned long long* rb = reinterpret_cast<const unsigned long long*>(araw);
  unsigned c[3] = {0, 0, 0};
  elem_coords<DIM>((unsigned)e, ma, c);
  double a = araw[e];
  unsigned long long any = rb[e];
#pragma unroll
  for (int d = 0; d < DIM; ++d)
#pragma unroll
    for (int off = -1; off <= 1; off += 2) {
      const unsigned nb = neighbour_of((unsigned)e, c, d, off, ma);
      a = fmax(a, 0.5 * araw[nb]);
      unsigned cn[3] = {0, 0, 0};
      elem_coords<DIM>(nb, ma, cn);
      any |= rb[nb];
#pragma unroll
      for (int d2 = 0; d2 < DIM; ++d2) {
        any |= rb[neighbour_of(nb, cn, d2, +1, ma)];
        any |= rb[neighbour_of(nb, cn, d2, -1, ma)];
      }
    }
  alpha[e] = a;
  touched[e] = any != 0ull ? 1 : 0;
  return any != 0ull;
}

// smoothed coefficient per element: max(raw_e, raw_nb / 2 over the face
// neighbours); touched[e] = 1 where the limited step changes the element's
// update: a raw coefficient above zero on the element, a face neighbour or a
// face neighbour's face neighbour (the raw values are non-negative, so "above
// zero" is "bits not all zero", tested with integer ORs).  The touched
// elements are also appended to tlist (one atomic per warp), so that the
// per-node limited kernel runs over them alone.
template <int DIM>
__global__ void __launch_bounds__(256)
k_alpha_smooth(const double* __restrict__ araw, double* __restrict__ alpha, unsigned char* __restrict__ touched,
               unsigned* __restrict__ tlist, unsigned* __restrict__ tcount, const MeshArgs ma) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool t = e < ma.E && alpha_smooth_one<DIM>(araw, alpha, touched, ma, (unsigned)e);
  // warp-aggregated append (every lane of the warp takes part)
  const unsigned mask = __ballot_sync(0xffffffffu, t);
  if (mask) {
    const int lane = threadIdx.x & 31, lead = __ffs(mask) - 1;
    unsigned base = 0;
    if (lane == lead) base = atomicAdd(tcount, (unsigned)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, lead);
    if (t) tlist[base + __popc(mask & ((1u << lane) - 1u))] = (unsigned)e;
  }
}

// u^n of node p of element e in the path's arithmetic
template <int M, typename R>
__device__ __forceinline__ void load_node(const double* __restrict__ u, long long E, unsigned e, int NP, int p, R* out) {
#pragma unroll
  for (int v = 0; v < M; ++v) {
    const double x = u[((size_t)v * E + e) * NP + p];
    if constexpr (sizeof(R) == 4) out[v] = d2f_int(x);
    else out[v] = x;
  }
}

// first-order Rusanov flux in direction d: (f(a) + f(b))/2 - lam/2 (b - a)
template <class EQ, typename R>
__device__ __forceinline__ void rusanov_lo(int d, const R* a, const R* b, R* F, const PhysParams<R>& pp) {
  constexpr int M = EQ::M;
  R qa[EQ::P], qb[EQ::P], fa[M], fb[M];
  EQ::pair_data(a, qa, pp);
  EQ::pair_data(b, qb, pp);
  EQ::flux(d, qa, fa, pp);
  EQ::flux(d, qb, fb, pp);
  const R lam = fmax(EQ::wave_speed(d, qa, pp), EQ::wave_speed(d, qb, pp));
#pragma unroll
  for (int v = 0; v < M; ++v) F[v] = R(0.5) * (fa[v] + fb[v]) - R(0.5) * lam * (b[v] - a[v]);
}

template <class EQ, typename R>
__device__ __forceinline__ void rho_p_of(const R* u, R& rho, R& p, const PhysParams<R>& pp) {
  constexpr int DIM = EQ::DIM;
  rho = u[0];
  R mm = R(0);
#pragma unroll
  for (int k = 0; k < DIM; ++k) mm += u[1 + k] * u[1 + k];
  p = (pp.gamma - R(1)) * (u[DIM + 1] - R(0.5) * mm / rho);
}

// Largest theta in [0,1] keeping rho and p of u0 + theta du at or above a
// tenth of those of u0 (0 if u0 is not admissible).
template <class EQ, typename R>
__device__ __forceinline__ R admissible_theta(const R* u0, const R* du, const PhysParams<R>& pp) {
  constexpr int M = EQ::M;
  R r0, p0;
  rho_p_of<EQ, R>(u0, r0, p0, pp);
  if (!(r0 > R(0)) || !(p0 > R(0))) return R(0);
  R u1[M];
#pragma unroll
  for (int v = 0; v < M; ++v) u1[v] = u0[v] + du[v];
  R r1, p1;
  rho_p_of<EQ, R>(u1, r1, p1, pp);
  R theta = R(1);
  const R er = R(0.1) * r0;
  if (r1 < er) theta = (r0 - er) / (r0 - r1);
#pragma unroll
  for (int v = 0; v < M; ++v) u1[v] = u0[v] + theta * du[v];
  R rt, pt;
  rho_p_of<EQ, R>(u1, rt, pt, pp);
  const R ep = R(0.1) * p0;
  if (pt < ep) theta = theta * (p0 - ep) / (p0 - pt);
  return theta;
}

// Limited flux at face node f of the face normal to d between element em
// ('-', its xi_d = 1 side) and ep ('+', its xi_d = 0 side).
template <class EQ, int N, typename R>
__device__ __forceinline__ void limited_face_flux(const double* __restrict__ uin, const R* __restrict__ trace,
                                                  const double* __restrict__ alpha, const MeshArgs& ma,
                                                  const PhysParams<R>& pp, const LimTab& lt, int d, unsigned em,
                                                  unsigned ep, int f, R dtR, R* F) {
  constexpr int DIM = EQ::DIM, M = EQ::M, n = N + 1, NP = ipow(n, DIM), C = trace_comps<EQ>();
  const long long E = ma.E;
  // time-averaged Rusanov flux from the two records (eq. numflux.cons)
  R rm[C], rp[C];
  load_face_record<EQ, N, R>(trace, E, d, 1, f, em, rm);
  load_face_record<EQ, N, R>(trace, E, d, 0, f, ep, rp);
  const R lam = fmax(rm[2 * M], rp[2 * M]);
  R Fho[M];
#pragma unroll
  for (int v = 0; v < M; ++v) Fho[v] = R(0.5) * (rm[M + v] + rp[M + v]) - R(0.5) * lam * (rp[v] - rm[v]);
  // u^n traces and the neighbouring interior nodes
  const int stride = ipow(n, d);
  const int fb = line_base<n>(f, stride);
  R um[M], up[M], umi[M], upi[M];
  load_node<M, R>(uin, E, em, NP, fb + N * stride, um);
  load_node<M, R>(uin, E, ep, NP, fb, up);
  load_node<M, R>(uin, E, em, NP, fb + (N - 1) * stride, umi);
  load_node<M, R>(uin, E, ep, NP, fb + stride, upi);
  R flo[M];
  rusanov_lo<EQ, R>(d, um, up, flo, pp);
  const double af64 = 0.5 * (alpha[em] + alpha[ep]);
  const R af = dt_as<R>(af64);
  R Fb[M];
#pragma unroll
  for (int v = 0; v < M; ++v) Fb[v] = af64 >= 1.0 ? flo[v] : (R(1) - af) * Fho[v] + af * flo[v];
  if (!(af64 > 0.0)) {
#pragma unroll
    for (int v = 0; v < M; ++v) F[v] = Fb[v];
    return;
  }
  // one-direction low-order states of the two end subcells with f_lo and the
  // change the blend would make to them
  R fmi[M], fpi[M];
  rusanov_lo<EQ, R>(d, umi, um, fmi, pp);
  rusanov_lo<EQ, R>(d, up, upi, fpi, pp);
  const R idx = inv_dx_of<R>(ma, d);
  const R cm = R(DIM) * dtR * idx / R(lt.w01[N]), cp = R(DIM) * dtR * idx / R(lt.w01[0]);
  R lm[M], dm[M], lp[M], dp[M];
#pragma unroll
  for (int v = 0; v < M; ++v) {
    lm[v] = um[v] - cm * (flo[v] - fmi[v]);
    dm[v] = -cm * (Fb[v] - flo[v]);
    lp[v] = up[v] - cp * (fpi[v] - flo[v]);
    dp[v] = cp * (Fb[v] - flo[v]);
  }
  const R theta = fmin(admissible_theta<EQ, R>(lm, dm, pp), admissible_theta<EQ, R>(lp, dp, pp));
#pragma unroll
  for (int v = 0; v < M; ++v) F[v] = flo[v] + theta * (Fb[v] - flo[v]);
}

// ---------------------------------------------------------------------------
// Limited face / update kernel: one thread per node (alpha: the smoothed
// coefficients; only_touched: leave the elements the limiter does not touch
// to the lane kernel)
// ---------------------------------------------------------------------------
template <class EQ, int N, typename R>
__global__ void __launch_bounds__(256)
k_face_update_limited(const double* __restrict__ uin, double* __restrict__ uout, const R* __restrict__ rbar,
                      const R* __restrict__ trace, const double* __restrict__ alpha,
                      const unsigned* __restrict__ tlist, const unsigned* __restrict__ tcount,
                      DevState* __restrict__ st, const MeshArgs ma, const PhysParams<R> pp, const RefTab<R> tb,
                      const LimTab lt, int slot, int only_touched) {
  constexpr int DIM = EQ::DIM, M = EQ::M, n = N + 1, NP = ipow(n, DIM), NF = NP / n;
  constexpr bool F32 = sizeof(R) == 4;
  const long long E = ma.E;
  if (st->status & ST_TIMEOUT) return;
  R lam = R(0);
  bool bad = false;
  // nodes of the touched elements (only_touched), else of every element
  const unsigned total = (only_touched ? *tcount : (unsigned)E) * (unsigned)NP;
  for (unsigned gid = blockIdx.x * blockDim.x + threadIdx.x; gid < total; gid += gridDim.x * blockDim.x) {
    const unsigned e = only_touched ? tlist[gid / NP] : gid / NP;
    const int p = (int)(gid % NP);
    unsigned ec[3] = {0, 0, 0};
    elem_coords<DIM>(e, ma, ec);
    const R dtR = step_dt<R>(st);
    const double ae = alpha[e];
    R uc[M];
    load_node<M, R>(uin, E, e, NP, p, uc);
    // high-order increment (eq. crkfr.non.cons.final) and first-order subcell increment
    R dh[M], dl[M];
#pragma unroll
    for (int v = 0; v < M; ++v) {
      dh[v] = -dtR * rbar[((size_t)v * E + e) * NP + p];
      dl[v] = R(0);
    }
    int rem = p;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const int cd = rem % n;
      rem /= n;
      const int stride = ipow(n, d);
      const int f = (p % stride) + (p / (stride * n)) * stride;
      const R idx = inv_dx_of<R>(ma, d);
      R fl[M], fr[M];
      if (cd > 0) {
        R un[M];
        load_node<M, R>(uin, E, e, NP, p - stride, un);
        rusanov_lo<EQ, R>(d, un, uc, fl, pp);
      }
      if (cd < N) {
        R un[M];
        load_node<M, R>(uin, E, e, NP, p + stride, un);
        rusanov_lo<EQ, R>(d, uc, un, fr, pp);
      }
      if (cd == N) {   // face xi_d = 1: this element is '-'
        R F[M];
        limited_face_flux<EQ, N, R>(uin, trace, alpha, ma, pp, lt, d, e, neighbour_of(e, ec, d, +1, ma), f, dtR, F);
        const R s = dtR * tb.iwN * idx;
#pragma unroll
        for (int v = 0; v < M; ++v) {
          dh[v] -= s * (F[v] - trace[trace_index<EQ, NF>(d, 1, f, M + v, E, e)]);
          fr[v] = F[v];
        }
      }
      if (cd == 0) {   // face xi_d = 0: this element is '+'
        R F[M];
        limited_face_flux<EQ, N, R>(uin, trace, alpha, ma, pp, lt, d, neighbour_of(e, ec, d, -1, ma), e, f, dtR, F);
        const R s = dtR * tb.iw0 * idx;
#pragma unroll
        for (int v = 0; v < M; ++v) {
          dh[v] += s * (F[v] - trace[trace_index<EQ, NF>(d, 0, f, M + v, E, e)]);
          fl[v] = F[v];
        }
      }
      const R c = dtR * idx / R(lt.w01[cd]);
#pragma unroll
      for (int v = 0; v < M; ++v) dl[v] -= c * (fr[v] - fl[v]);
    }
    // blend of the increments (the low-order one alone where a_e = 1), then
    // u^{n+1} = u^n + du in FP64
    const R a = dt_as<R>(ae);
    double uu[M];
#pragma unroll
    for (int v = 0; v < M; ++v) {
      const R du = ae >= 1.0 ? dl[v] : (R(1) - a) * dh[v] + a * dl[v];
      const size_t g = ((size_t)v * E + e) * NP + p;
      if constexpr (F32) uu[v] = uin[g] + f2d_int(du);
      else uu[v] = uin[g] + du;
      uout[g] = uu[v];
    }
    R lamn = R(0);
    bad = !physical_state<EQ, R>(uu, ma, lamn) || bad;
    lam = fmax(lam, lamn);
  }
  reduce_lambda<R>(lam, bad, st, slot ^ 1);
}

}  // namespace crk
