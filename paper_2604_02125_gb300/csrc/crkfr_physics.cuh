// crkfr_physics.cuh -- device physics of the cRKFR hot path (sm_103a).
//
// System u_t + f(u)_x + B(u) g(u)_x = 0 (paper: eq. flux.and.non.cons).
// Point-wise physical flux, spectral radius of f' + B g' (eqs.
// rusanov.wave.speed / combined.wave.speed), two-point volume fluxes f_S of
// the flux-differencing form (Sec. 3, eq. entropy.cons.flux.dev) and the
// non-conservative product of eq. entropy.cons.noncons.dev.
//
// Every routine works on "pair data" q[P]: primitive values of one node that
// the two-point fluxes need, computed once per node and stage.  Templated on
// the arithmetic type R (double for the FP64 path, float for the FP32
// pair-flux form).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace crk {

constexpr int VOL_EC = 0, VOL_KEP = 1, VOL_CENTRAL = 2;

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

template <typename R>
struct PhysParams {
  R gamma, inv_gm1, c_h;
  int vol;
};

// ---------------------------------------------------------------------------
// Logarithmic mean L(a,b) = (a-b)/(ln a - ln b) and its inverse.
// For a ~ b both use the series in u = ((a-b)/(a+b))^2:
//   L = (a+b) / (2 F(u)),  F(u) = 1 + u/3 + u^2/5 + u^3/7 + ...
// FP64: 4 terms below u = 1e-4 (truncation u^4/9 < 1.2e-17).
// FP32: 5 terms below u = 0.05 (truncation below u^5 / (11 (1 - u)) < 3e-8,
// half an FP32 ulp of F ~ 1); above it the ratio a/b exceeds 1.57 and
// log(a/b) is well conditioned.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double series_F(double u) {
  return 1.0 + u * (1.0 / 3.0 + u * (1.0 / 5.0 + u * (1.0 / 7.0)));
}
__device__ __forceinline__ float series_F(float u) {
  return 1.0f + u * (1.0f / 3.0f + u * (1.0f / 5.0f + u * (1.0f / 7.0f + u * (1.0f / 9.0f))));
}
template <typename R> struct LogMeanEps;
template <> struct LogMeanEps<double> { static constexpr double v = 1e-4; };
template <> struct LogMeanEps<float> { static constexpr float v = 0.05f; };

// FP64: IEEE division.  FP32: the MUFU reciprocal (rcp.approx, about 1 ulp),
// no slow-path branch.
__device__ __forceinline__ double fast_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float fast_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double plain_log(double x) { return log(x); }
__device__ __forceinline__ float plain_log(float x) { return logf(x); }

template <typename R>
__device__ __forceinline__ R logmean(R a, R b) {
  R s = a + b, d = a - b;
  R rs = fast_rcp(s);
  R f = d * rs;
  R u = f * f;
  if (u < LogMeanEps<R>::v) return R(0.5) * s * fast_rcp(series_F(u));
  return d * fast_rcp(plain_log(a * fast_rcp(b)));
}

template <typename R>
__device__ __forceinline__ R inv_logmean(R a, R b) {
  R s = a + b, d = a - b;
  R rs = fast_rcp(s);
  R f = d * rs;
  R u = f * f;
  if (u < LogMeanEps<R>::v) return R(2) * series_F(u) * rs;
  return plain_log(a * fast_rcp(b)) * fast_rcp(d);
}

// Out of line so that the compiler cannot if-convert it into the common path
// (a predicated copy would be executed by every pair).
template <typename R>
__device__ __noinline__ void logmean_pair_general(R a1, R b1, R a2, R b2, R& L1, R& iL2) {
  L1 = logmean(a1, b1);
  iL2 = inv_logmean(a2, b2);
}

// L(a1,b1) and 1/L(a2,b2) together: one branch decides for both whether the
// series applies (the common case on resolved data), otherwise each takes its
// own branch above.
template <typename R>
__device__ __forceinline__ void logmean_pair(R a1, R b1, R a2, R b2, R& L1, R& iL2) {
  R s1 = a1 + b1, d1 = a1 - b1, s2 = a2 + b2, d2 = a2 - b2;
  R rs1 = fast_rcp(s1), rs2 = fast_rcp(s2);
  R f1 = d1 * rs1, f2 = d2 * rs2;
  R u1 = f1 * f1, u2 = f2 * f2;
  if (fmax(u1, u2) < LogMeanEps<R>::v) {
    L1 = R(0.5) * s1 * fast_rcp(series_F(u1));
    iL2 = R(2) * series_F(u2) * rs2;
  } else {
    logmean_pair_general(a1, b1, a2, b2, L1, iL2);
  }
}

// FP32: 1/F(u) = sqrt(u)/artanh(sqrt(u)) by its own series (five terms; the
// truncation is below 7e-9 relative for u < 0.05), so that the series branch
// needs a single reciprocal: 1/(s1 s2) gives both 1/s1 and 1/s2.
__device__ __forceinline__ float series_invF(float u) {
  return 1.0f + u * (-1.0f / 3.0f + u * (-4.0f / 45.0f + u * (-44.0f / 945.0f + u * (-428.0f / 14175.0f))));
}
__device__ __forceinline__ void logmean_pair(float a1, float b1, float a2, float b2, float& L1, float& iL2) {
  const float s1 = a1 + b1, d1 = a1 - b1, s2 = a2 + b2, d2 = a2 - b2;
  const float r = fast_rcp(s1 * s2);
  const float rs1 = s2 * r, rs2 = s1 * r;
  const float f1 = d1 * rs1, f2 = d2 * rs2;
  const float u1 = f1 * f1, u2 = f2 * f2;
  if (fmaxf(u1, u2) < LogMeanEps<float>::v) {
    L1 = 0.5f * s1 * series_invF(u1);
    iL2 = 2.0f * series_F(u2) * rs2;
  } else {
    logmean_pair_general(a1, b1, a2, b2, L1, iL2);
  }
}

// FP64: the same single-reciprocal form (each FP64 division is a dozen
// instructions on the narrow FP64 pipe): 1/F(u) by its own series, five terms
// (truncation below 1e-21 for u < 1e-4), and 1/s1, 1/s2 from 1/(s1 s2).
__device__ __forceinline__ double series_invF(double u) {
  return 1.0 + u * (-1.0 / 3.0 + u * (-4.0 / 45.0 + u * (-44.0 / 945.0 + u * (-428.0 / 14175.0))));
}
__device__ __forceinline__ void logmean_pair(double a1, double b1, double a2, double b2, double& L1, double& iL2) {
  const double s1 = a1 + b1, d1 = a1 - b1, s2 = a2 + b2, d2 = a2 - b2;
  const double r = 1.0 / (s1 * s2);
  const double rs1 = s2 * r, rs2 = s1 * r;
  const double f1 = d1 * rs1, f2 = d2 * rs2;
  const double u1 = f1 * f1, u2 = f2 * f2;
  if (fmax(u1, u2) < LogMeanEps<double>::v) {
    L1 = 0.5 * s1 * series_invF(u1);
    iL2 = 2.0 * series_F(u2) * rs2;
  } else {
    logmean_pair_general(a1, b1, a2, b2, L1, iL2);
  }
}

// Exact float <-> double conversions with integer instructions only (the FP64
// pipe of this GPU is narrow and also executes the hardware conversions, and a
// predicated hardware fallback would still occupy it).  Values below the
// normal FP32 range become signed zero; overflow gives a signed infinity,
// NaN stays NaN.
__device__ __forceinline__ float d2f_int(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7FFu;
  const unsigned sign = hi & 0x80000000u;
  const unsigned mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const unsigned rest = lo & 0x1FFFFFFFu;
  unsigned bits = sign | ((e - 896u) << 23) | mant;
  bits += (rest > 0x10000000u) | ((rest == 0x10000000u) & (mant & 1u));   // round to nearest even
  const bool nan = e == 0x7FFu && ((hi & 0xFFFFFu) | lo) != 0u;
  bits = e < 897u ? sign : bits;
  bits = e > 1150u ? (sign | 0x7F800000u | (nan ? 0x400000u : 0u)) : bits;
  return __uint_as_float(bits);
}
__device__ __forceinline__ double f2d_int(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xFFu;
  const unsigned ed = e == 255u ? 0x7FFu : e + 896u;
  unsigned hi = (b & 0x80000000u) | (ed << 20) | ((b & 0x7FFFFFu) >> 3);
  unsigned lo = b << 29;
  hi = e == 0u ? (b & 0x80000000u) : hi;
  lo = e == 0u ? 0u : lo;
  return __hiloint2double((int)hi, (int)lo);
}

// Double -> float rounded toward zero, for the FP32 physicality and wave-speed
// check of an updated state (a sign test and a maximum: the rounding
// direction does not matter there).  Values below the normal FP32 range give
// signed zero; values beyond it, infinities and NaNs give NaN, which fails the
// check.  About ten integer instructions against twenty-five for d2f_int.
__device__ __forceinline__ float d2f_rz(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7FFu;
  const unsigned mant = __funnelshift_r(lo, hi, 29) & 0x7FFFFFu;
  const unsigned sign = hi & 0x80000000u;
  unsigned bits = sign | ((e - 896u) << 23) | mant;
  bits = e - 897u < 254u ? bits : (e < 897u ? sign : 0x7FC00000u);
  return __uint_as_float(bits);
}

// Reciprocal and square root of the CFL wave speeds: IEEE in FP64, the MUFU
// approximations (about 1 ulp) in FP32, where the result only enters the
// maximum that sets dt.
__device__ __forceinline__ double speed_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float speed_rcp(float x) { return fast_rcp(x); }
__device__ __forceinline__ double speed_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float speed_sqrt(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// ---------------------------------------------------------------------------
// Compressible Euler in DIM dimensions: u = (rho, rho v_1..rho v_DIM, E).
// Pair data q = (rho, v_1..v_DIM, p, aux); aux = rho/p for the EC flux,
// e = E/rho for the KEP and central fluxes.
// ---------------------------------------------------------------------------
template <int DIM_, int VOL_ = VOL_EC>
struct Euler {
  static constexpr int DIM = DIM_;
  static constexpr int VOL = VOL_;
  static constexpr int M = DIM_ + 2;
  static constexpr int P = DIM_ + 3;
  static constexpr bool NC = false;
  static constexpr bool NCS = false;   // stage-wise non-conservative flux (GLM-MHD only)
  static constexpr int IRHO = 0, IP = DIM_ + 1, IAUX = DIM_ + 2;

  template <typename R>
  __device__ __forceinline__ static void pair_data(const R* u, R* q, const PhysParams<R>& pp) {
    R rho = u[0];
    R E = u[DIM + 1];
    if constexpr (sizeof(R) == 8 && VOL == VOL_EC) {
      // one FP64 division for 1/rho and rho/p: p needs |m|^2 / rho, so
      // p rho = (gamma-1)(E rho - |m|^2/2) and 1/(rho p rho) gives both
      R mm = R(0);
#pragma unroll
      for (int k = 0; k < DIM; ++k) mm += u[1 + k] * u[1 + k];
      const R prho = (pp.gamma - R(1)) * (E * rho - R(0.5) * mm);   // p rho
      const R r = R(1) / (prho * rho);
      const R ir = prho * r;                                         // 1 / rho
#pragma unroll
      for (int k = 0; k < DIM; ++k) q[1 + k] = u[1 + k] * ir;
      q[0] = rho;
      q[IP] = prho * ir;
      q[IAUX] = rho * rho * rho * r;                                 // rho / p
      return;
    }
    R ir = fast_rcp(rho);
    R ke = R(0);
    q[0] = rho;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      R v = u[1 + k] * ir;
      q[1 + k] = v;
      ke += v * u[1 + k];
    }
    R p = (pp.gamma - R(1)) * (E - R(0.5) * ke);
    q[IP] = p;
    if constexpr (VOL == VOL_EC) q[IAUX] = rho * fast_rcp(p);
    else q[IAUX] = E * ir;
  }

  template <typename R>
  __device__ __forceinline__ static R total_energy(const R* q, const PhysParams<R>& pp) {
    if constexpr (VOL == VOL_EC) {
      R ke = R(0);
#pragma unroll
      for (int k = 0; k < DIM; ++k) ke += q[1 + k] * q[1 + k];
      return q[IP] * pp.inv_gm1 + R(0.5) * q[0] * ke;
    }
    return q[0] * q[IAUX];
  }

  // conserved variables from pair data
  template <typename R>
  __device__ __forceinline__ static void cons_from_pair(const R* q, R* u, const PhysParams<R>& pp) {
    u[0] = q[0];
#pragma unroll
    for (int k = 0; k < DIM; ++k) u[1 + k] = q[0] * q[1 + k];
    u[DIM + 1] = total_energy(q, pp);
  }

  // physical flux in direction d from pair data
  template <typename R>
  __device__ __forceinline__ static void flux(int d, const R* q, R* f, const PhysParams<R>& pp) {
    R mflux = q[0] * q[1 + d];
    f[0] = mflux;
#pragma unroll
    for (int k = 0; k < DIM; ++k) f[1 + k] = mflux * q[1 + k] + (k == d ? q[IP] : R(0));
    f[DIM + 1] = q[1 + d] * (total_energy(q, pp) + q[IP]);
  }

  // symmetric two-point flux f_S(q_a, q_b) in direction d
  template <typename R>
  __device__ __forceinline__ static void two_point(int d, const R* a, const R* b, R* f, const PhysParams<R>& pp) {
    R vavg[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) vavg[k] = R(0.5) * (a[1 + k] + b[1 + k]);
    R pavg = R(0.5) * (a[IP] + b[IP]);
    if constexpr (VOL == VOL_EC) {
      // Ranocha: rho^ln {{v}}, momentum f_rho {{v}} + {{p}} n, energy with
      // 1/ln-mean(rho/p) and the product p_a v_b + p_b v_a
      R rho_ln, irp_ln;
      logmean_pair(a[0], b[0], a[IAUX], b[IAUX], rho_ln, irp_ln);
      R f0 = rho_ln * vavg[d];
      R vv = R(0);
#pragma unroll
      for (int k = 0; k < DIM; ++k) vv += a[1 + k] * b[1 + k];
      f[0] = f0;
#pragma unroll
      for (int k = 0; k < DIM; ++k) f[1 + k] = f0 * vavg[k] + (k == d ? pavg : R(0));
      f[DIM + 1] = f0 * (R(0.5) * vv + pp.inv_gm1 * irp_ln)
                 + R(0.5) * (a[IP] * b[1 + d] + b[IP] * a[1 + d]);
    } else if constexpr (VOL == VOL_KEP) {
      // Kennedy-Gruber: arithmetic means of rho, v, p and e = E/rho
      R ravg = R(0.5) * (a[0] + b[0]);
      R eavg = R(0.5) * (a[IAUX] + b[IAUX]);
      R f0 = ravg * vavg[d];
      f[0] = f0;
#pragma unroll
      for (int k = 0; k < DIM; ++k) f[1 + k] = f0 * vavg[k] + (k == d ? pavg : R(0));
      f[DIM + 1] = (ravg * eavg + pavg) * vavg[d];
    } else {
      R fa[M], fb[M];
      flux(d, a, fa, pp);
      flux(d, b, fb, pp);
#pragma unroll
      for (int m = 0; m < M; ++m) f[m] = R(0.5) * (fa[m] + fb[m]);
    }
  }

  template <typename R>
  __device__ __forceinline__ static R wave_speed(int d, const R* q, const PhysParams<R>& pp) {
    return fabs(q[1 + d]) + sqrt(pp.gamma * q[IP] / q[0]);
  }

  // g^d(u) for the non-conservative product: none for Euler
  template <typename R>
  __device__ __forceinline__ static void ncg(int, const R*, R*) {}
  template <typename R>
  __device__ __forceinline__ static void nc_apply(int, const R*, const R*, R*) {}

  // physicality of a conserved state (rho > 0, p > 0, finite) and sum_d lambda_d / dx_d
  template <typename T>
  __device__ __forceinline__ static bool physical(const T* u, T gamma, T& lam_sum, const T* inv_dx) {
    T rho = u[0];
    T ke = T(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) ke += u[1 + k] * u[1 + k];
    T ir = speed_rcp(rho);
    T p = (gamma - T(1)) * (u[DIM + 1] - T(0.5) * ke * ir);
    T c = speed_sqrt(gamma * p * ir);
    T s = T(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) s += (fabs(u[1 + k] * ir) + c) * inv_dx[k];
    lam_sum = s;
    return rho > T(0) && p > T(0) && isfinite(s);
  }
};

// ---------------------------------------------------------------------------
// Ideal GLM-MHD (2D): u = (rho, rho v1..3, E, B1..3, psi),
// E = p/(gamma-1) + rho|v|^2/2 + |B|^2/2 + psi^2/2.
// Non-conservative term along d: phi_Powell(u) dB_d/dx_d + phi_GLM^d(u) dpsi/dx_d,
// phi_Powell = (0, B, v.B, v, 0), phi_GLM^d = (0, 0,0,0, v_d psi, 0,0,0, v_d),
// so g^d(u) = (B_d, psi).
// Pair data q = (rho, v1, v2, v3, p, B1, B2, B3, psi, beta = rho/(2p), |v|^2, |B|^2, v.B).
// ---------------------------------------------------------------------------
template <int VOL_ = VOL_EC>
struct GlmMhd {
  static constexpr int DIM = 2;
  static constexpr int VOL = VOL_;
  static constexpr int M = 9;
  static constexpr int P = 13;
  static constexpr bool NC = true;
  static constexpr bool NCS = false;
  static constexpr int IRHO = 0, IP = 4, IB = 5, IPSI = 8, IBETA = 9, IV2 = 10, IB2 = 11, IVB = 12;

  template <typename R>
  __device__ __forceinline__ static void pair_data(const R* u, R* q, const PhysParams<R>& pp) {
    R rho = u[0];
    R B1 = u[5], B2 = u[6], B3 = u[7], psi = u[8];
    R BB = B1 * B1 + B2 * B2 + B3 * B3;
    R ir, p, irp;   // 1/rho, p, rho/p
    if constexpr (sizeof(R) == 8) {
      // one FP64 division: p rho = (gamma-1)(rho (E - |B|^2/2 - psi^2/2) - |m|^2/2)
      const R mm = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
      const R prho = (pp.gamma - R(1)) * (rho * (u[4] - R(0.5) * BB - R(0.5) * psi * psi) - R(0.5) * mm);
      const R r = R(1) / (prho * rho);
      ir = prho * r;
      p = prho * ir;
      irp = rho * rho * rho * r;
    } else {
      ir = fast_rcp(rho);
      const R w1 = u[1] * ir, w2 = u[2] * ir, w3 = u[3] * ir;
      const R vv0 = w1 * w1 + w2 * w2 + w3 * w3;
      p = (pp.gamma - R(1)) * (u[4] - R(0.5) * rho * vv0 - R(0.5) * BB - R(0.5) * psi * psi);
      irp = rho * fast_rcp(p);
    }
    R v1 = u[1] * ir, v2 = u[2] * ir, v3 = u[3] * ir;
    R vv = v1 * v1 + v2 * v2 + v3 * v3;
    q[0] = rho; q[1] = v1; q[2] = v2; q[3] = v3; q[4] = p;
    q[5] = B1; q[6] = B2; q[7] = B3; q[8] = psi;
    q[IBETA] = R(0.5) * irp;
    q[IV2] = vv; q[IB2] = BB; q[IVB] = v1 * B1 + v2 * B2 + v3 * B3;
  }

  // conserved variables from pair data
  template <typename R>
  __device__ __forceinline__ static void cons_from_pair(const R* q, R* u, const PhysParams<R>& pp) {
    const R rho = q[0];
    u[0] = rho;
    u[1] = rho * q[1]; u[2] = rho * q[2]; u[3] = rho * q[3];
    u[4] = q[IP] * pp.inv_gm1 + R(0.5) * (rho * q[IV2] + q[IB2] + q[IPSI] * q[IPSI]);
    u[5] = q[5]; u[6] = q[6]; u[7] = q[7]; u[8] = q[8];
  }

  template <typename R>
  __device__ __forceinline__ static void flux(int d, const R* q, R* f, const PhysParams<R>& pp) {
    R rho = q[0], p = q[IP], psi = q[IPSI];
    R vd = q[1 + d], Bd = q[IB + d];
    R mflux = rho * vd;
    f[0] = mflux;
#pragma unroll
    for (int k = 0; k < 3; ++k) f[1 + k] = mflux * q[1 + k] - Bd * q[IB + k] + (k == d ? p + R(0.5) * q[IB2] : R(0));
    f[4] = vd * (R(0.5) * rho * q[IV2] + pp.gamma * pp.inv_gm1 * p + q[IB2]) - Bd * q[IVB] + pp.c_h * psi * Bd;
#pragma unroll
    for (int k = 0; k < 3; ++k) f[5 + k] = (k == d) ? pp.c_h * psi : vd * q[IB + k] - q[1 + k] * Bd;
    f[8] = pp.c_h * Bd;
  }

  // entropy-conservative flux: satisfies [[w]].f = [[psi_d]] + {{theta}} [[B_d]]
  // with theta = w.phi_Powell = rho (v.B)/p (derived from the entropy
  // variables of S = -rho s/(gamma-1)); central flux for CR_VOL_CENTRAL.
  template <typename R>
  __device__ __forceinline__ static void two_point(int d, const R* a, const R* b, R* f, const PhysParams<R>& pp) {
    if constexpr (VOL != VOL_EC) {
      R fa[M], fb[M];
      flux(d, a, fa, pp);
      flux(d, b, fb, pp);
#pragma unroll
      for (int m = 0; m < M; ++m) f[m] = R(0.5) * (fa[m] + fb[m]);
      return;
    }
    R v[3], B[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) { v[k] = R(0.5) * (a[1 + k] + b[1 + k]); B[k] = R(0.5) * (a[IB + k] + b[IB + k]); }
    R psi = R(0.5) * (a[IPSI] + b[IPSI]);
    R rho_ln, ibeta_ln;
    logmean_pair(a[0], b[0], a[IBETA], b[IBETA], rho_ln, ibeta_ln);
    R ptil = (a[0] + b[0]) * fast_rcp(R(2) * (a[IBETA] + b[IBETA]));     // {{rho}} / (2 {{beta}})
    R v2avg = R(0.5) * (a[IV2] + b[IV2]);
    R B2avg = R(0.5) * (a[IB2] + b[IB2]);
    R vB2avg = R(0.5) * (a[1 + d] * a[IB2] + b[1 + d] * b[IB2]);
    R psiBavg = R(0.5) * (a[IPSI] * a[IB + d] + b[IPSI] * b[IB + d]);
    R vBavg = R(0.5) * (a[IVB] + b[IVB]);
    R Bd = B[d];
    R ch = pp.c_h;
    R f0 = rho_ln * v[d];
    f[0] = f0;
#pragma unroll
    for (int k = 0; k < 3; ++k) f[1 + k] = f0 * v[k] - Bd * B[k] + (k == d ? ptil + R(0.5) * B2avg : R(0));
#pragma unroll
    for (int k = 0; k < 3; ++k) f[5 + k] = (k == d) ? ch * psi : v[d] * B[k] - v[k] * Bd;
    f[8] = ch * Bd;
    f[4] = f0 * R(0.5) * (pp.inv_gm1 * ibeta_ln - v2avg)
         + f[1] * v[0] + f[2] * v[1] + f[3] * v[2]
         + f[5] * B[0] + f[6] * B[1] + f[7] * B[2] + f[8] * psi
         - R(0.5) * vB2avg - ch * psiBavg + Bd * vBavg;
  }

  // |v_d| + max(c_f, c_h): the GLM pair travels at v_d -+ c_h
  template <typename R>
  __device__ __forceinline__ static R wave_speed(int d, const R* q, const PhysParams<R>& pp) {
    R ir = R(1) / q[0];
    R a2 = pp.gamma * q[IP] * ir;
    R b2 = q[IB2] * ir;
    R bd2 = q[IB + d] * q[IB + d] * ir;
    R s = a2 + b2;
    R cf = sqrt(R(0.5) * (s + sqrt(fmax(s * s - R(4) * a2 * bd2, R(0)))));
    return fabs(q[1 + d]) + fmax(cf, pp.c_h);
  }

  // g^d(u) = (B_d, psi)
  template <typename R>
  __device__ __forceinline__ static void ncg(int d, const R* q, R* g) { g[0] = q[IB + d]; g[1] = q[IPSI]; }

  // out += phi_Powell(q) g0 + phi_GLM^d(q) g1
  template <typename R>
  __device__ __forceinline__ static void nc_apply(int d, const R* q, const R* g, R* out) {
    R g0 = g[0], g1 = g[1];
    out[1] += q[IB + 0] * g0;
    out[2] += q[IB + 1] * g0;
    out[3] += q[IB + 2] * g0;
    out[4] += q[IVB] * g0 + q[1 + d] * q[IPSI] * g1;
    out[5] += q[1] * g0;
    out[6] += q[2] * g0;
    out[7] += q[3] * g0;
    out[8] += q[1 + d] * g1;
  }

  template <typename T>
  __device__ __forceinline__ static bool physical(const T* u, T gamma, T c_h, T& lam_sum, const T* inv_dx) {
    T rho = u[0];
    T ir = speed_rcp(rho);
    T v1 = u[1] * ir, v2 = u[2] * ir, v3 = u[3] * ir;
    T BB = u[5] * u[5] + u[6] * u[6] + u[7] * u[7];
    T p = (gamma - T(1)) * (u[4] - T(0.5) * rho * (v1 * v1 + v2 * v2 + v3 * v3) - T(0.5) * BB - T(0.5) * u[8] * u[8]);
    T a2 = gamma * p * ir, b2 = BB * ir, s = a2 + b2;
    T vv[2] = {v1, v2};
    T tot = T(0);
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      T bd2 = u[5 + d] * u[5 + d] * ir;
      T cf = speed_sqrt(T(0.5) * (s + speed_sqrt(fmax(s * s - T(4) * a2 * bd2, T(0)))));
      tot += (fabs(vv[d]) + fmax(cf, c_h)) * inv_dx[d];
    }
    lam_sum = tot;
    return rho > T(0) && p > T(0) && isfinite(tot);
  }
};

// GLM-MHD with the stage-wise non-conservative numerical flux of eq.
// bad.numflux.non.cons: sum_j b_j B(u^{(j),+-}) g^avg(u^(j)).  B(u) and g(u)
// depend on u through v, B and psi only, so each stage leaves these seven
// values of both face traces for the face kernel (stage_prims), which applies
// B(own) to the averaged g of both sides (nc_apply_prims).
template <int VOL_ = VOL_EC>
struct GlmMhdStages : GlmMhd<VOL_> {
  using Base = GlmMhd<VOL_>;
  static constexpr bool NCS = true;
  static constexpr int NPRIM = 7;   // v1, v2, v3, B1, B2, B3, psi
  template <typename R>
  __device__ __forceinline__ static void stage_prims(const R* q, R* o) {
    o[0] = q[1]; o[1] = q[2]; o[2] = q[3];
    o[3] = q[Base::IB]; o[4] = q[Base::IB + 1]; o[5] = q[Base::IB + 2]; o[6] = q[Base::IPSI];
  }
  // g^d of a primitive record: (B_d, psi)
  template <typename R>
  __device__ __forceinline__ static void ncg_prims(int d, const R* w, R* g) { g[0] = w[3 + d]; g[1] = w[6]; }
  // out += phi_Powell(w) g0 + phi_GLM^d(w) g1 (as nc_apply, from the primitives)
  template <typename R>
  __device__ __forceinline__ static void nc_apply_prims(int d, const R* w, const R* g, R* out) {
    const R g0 = g[0], g1 = g[1];
    out[1] += w[3] * g0;
    out[2] += w[4] * g0;
    out[3] += w[5] * g0;
    out[4] += (w[0] * w[3] + w[1] * w[4] + w[2] * w[5]) * g0 + w[d] * w[6] * g1;
    out[5] += w[0] * g0;
    out[6] += w[1] * g0;
    out[7] += w[2] * g0;
    out[8] += w[d] * g1;
  }
};

// ---------------------------------------------------------------------------
// Butcher tableaux per degree N (explicit RK of order N+1), as constexpr
// functions so that fully unrolled stage loops fold zero coefficients.
//  N=1 Heun RK2, N=2 Heun RK3, N=3 classical RK4, N=4 Butcher's 6-stage
//  order 5, N=5 Butcher's 7-stage order 6.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int rk_stages(int N) { return N == 1 ? 2 : N == 2 ? 3 : N == 3 ? 4 : N == 4 ? 6 : 7; }

__host__ __device__ constexpr double rk_a(int N, int i, int j) {
  // i, j zero-based stage indices, a_ij for j < i
  return N == 1 ? (i == 1 && j == 0 ? 1.0 : 0.0)
       : N == 2 ? ((i == 1 && j == 0) ? 1.0 / 3.0 : (i == 2 && j == 1) ? 2.0 / 3.0 : 0.0)
       : N == 3 ? ((i == 1 && j == 0) ? 0.5 : (i == 2 && j == 1) ? 0.5 : (i == 3 && j == 2) ? 1.0 : 0.0)
       : N == 4 ? (i == 1 ? (j == 0 ? 0.25 : 0.0)
                 : i == 2 ? (j == 0 ? 0.125 : j == 1 ? 0.125 : 0.0)
                 : i == 3 ? (j == 1 ? -0.5 : j == 2 ? 1.0 : 0.0)
                 : i == 4 ? (j == 0 ? 3.0 / 16.0 : j == 3 ? 9.0 / 16.0 : 0.0)
                 : i == 5 ? (j == 0 ? -3.0 / 7.0 : j == 1 ? 2.0 / 7.0 : j == 2 ? 12.0 / 7.0 : j == 3 ? -12.0 / 7.0 : j == 4 ? 8.0 / 7.0 : 0.0)
                 : 0.0)
       : (i == 1 ? (j == 0 ? 1.0 / 3.0 : 0.0)
        : i == 2 ? (j == 1 ? 2.0 / 3.0 : 0.0)
        : i == 3 ? (j == 0 ? 1.0 / 12.0 : j == 1 ? 1.0 / 3.0 : j == 2 ? -1.0 / 12.0 : 0.0)
        : i == 4 ? (j == 0 ? -1.0 / 16.0 : j == 1 ? 9.0 / 8.0 : j == 2 ? -3.0 / 16.0 : j == 3 ? -3.0 / 8.0 : 0.0)
        : i == 5 ? (j == 1 ? 9.0 / 8.0 : j == 2 ? -3.0 / 8.0 : j == 3 ? -3.0 / 4.0 : j == 4 ? 0.5 : 0.0)
        : i == 6 ? (j == 0 ? 9.0 / 44.0 : j == 1 ? -9.0 / 11.0 : j == 2 ? 63.0 / 44.0 : j == 3 ? 18.0 / 11.0 : j == 5 ? -16.0 / 11.0 : 0.0)
        : 0.0);
}

__host__ __device__ constexpr double rk_b(int N, int i) {
  return N == 1 ? 0.5
       : N == 2 ? (i == 0 ? 0.25 : i == 1 ? 0.0 : 0.75)
       : N == 3 ? (i == 0 || i == 3 ? 1.0 / 6.0 : 1.0 / 3.0)
       : N == 4 ? (i == 0 || i == 5 ? 7.0 / 90.0 : i == 1 ? 0.0 : i == 2 || i == 4 ? 32.0 / 90.0 : 12.0 / 90.0)
       : (i == 0 || i == 6 ? 11.0 / 120.0 : i == 1 ? 0.0 : i == 2 || i == 3 ? 27.0 / 40.0 : -4.0 / 15.0);
}

// true if R_j is needed by a later stage's combination
__host__ __device__ constexpr bool rk_needed_later(int N, int j) {
  bool need = false;
  for (int i = j + 1; i < rk_stages(N); ++i) need = need || (rk_a(N, i, j) != 0.0);
  return need;
}

}  // namespace crk
