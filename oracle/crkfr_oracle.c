/*
 * crkfr_oracle.c -- plain, slow FP64 CPU oracle for one step of the compact
 * Runge-Kutta flux reconstruction (cRKFR) method with entropy-conservative /
 * kinetic-energy-preserving flux differencing (Babbar, Chen, Ranocha,
 * arXiv 2604.02125).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares no
 * code, header, table or helper with the CUDA library in
 * paper_2604_02125_gb300/csrc; neither includes or links the other.
 *
 * Every routine follows the paper literally, element by element, with no
 * symmetry tricks and no fusion:
 *   - reference element [0,1], GLL solution points, Lagrange basis (Sec. 2),
 *   - differentiation matrix D_pq = l_q'(xi_p) (eq. diff.matrix),
 *   - Huynh's g2 correction functions evaluated from Legendre polynomials
 *     (Sec. 2.1, used throughout the paper),
 *   - cRK inner stages (eq. crkfr.inner) with the flux-differencing local
 *     derivative (eq. entropy.cons.flux.dev) and the non-symmetric
 *     non-conservative product (eq. entropy.cons.noncons.dev),
 *   - time averages of flux, solution and non-conservative extrapolations
 *     (eqs. disc.avg.flux, local.time.avg.non.cons, Sec. 2.3),
 *   - time-averaged Rusanov flux (eq. numflux.cons) and the reduced-
 *     communication non-conservative numerical flux B(u^{n,+-}) g^avg(U)
 *     (Sec. 2.3, the variant used for all of the paper's results), or the
 *     stage-wise one of eq. bad.numflux.non.cons (or_desc.ncflux = 1),
 *   - final update (eqs. crkfr.non.cons.final, total.F.non.cons) with the
 *     flux-differencing time-averaged volume term (Sec. 3);
 *   - the multi-stage RKFR step the cRKFR method is derived from (eq.
 *     rkfr.non.cons): the same RK tableau on the semi-discrete FR system,
 *     one face exchange per stage (or_rkfr_step).
 *
 * Readings of points the paper leaves open:
 *   - multi-D: tensor product, sum of per-direction 1D operators on a
 *     uniform periodic Cartesian grid;
 *   - Butcher tableaux per degree N (order N+1), see or_butcher();
 *   - face wave speed from the u^n traces: lambda = max(sigma(u^{n-}), sigma(u^{n+}));
 *   - dt = CFL / max_p sum_d sigma_d(u_p) / dx_d;
 *   - two-point fluxes: Ranocha (EC+KEP) and Kennedy-Gruber (KEP) for Euler,
 *     an EC flux for ideal GLM-MHD derived from the discrete entropy
 *     condition [[w]].f = [[psi]] + {{theta}} [[B_d]] (theta = w . phi_Powell),
 *     GLM cleaning speed c_h fixed per run;
 *   - logarithmic mean: series in u = ((a-b)/(a+b))^2 below 1e-4, else
 *     (a-b)/log1p((a-b)/b).
 *
 * Data layout of every state array: [var][elem][node] (structure of arrays),
 * node index i fastest, then j, then k; element index x fastest.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXN 5
#define OR_MAXNP 6      /* N+1 */
#define OR_MAXS 7
#define OR_MAXM 9

typedef struct {
  int eq;          /* 0 = compressible Euler, 1 = ideal GLM-MHD (2D only)      */
  int dim;         /* 1, 2, 3                                                  */
  int N;           /* polynomial degree 1..5                                   */
  int cells[3];    /* elements per direction                                   */
  double lo[3], hi[3];
  double gamma, cfl, c_h;
  int vol;         /* 0 = EC (Ranocha / GLM-MHD EC), 1 = KEP Kennedy-Gruber, 2 = central */
  int surf;        /* 0 = Rusanov, 1 = EC two-point surface flux (semi-discrete tests) */
  int ncflux;      /* non-conservative numerical flux of the cRKFR step (Sec. 2.3):
                      0 = B(u^{n,+-}) g^avg(U) (reduced communication, all of the paper's results),
                      1 = sum_j b_j B(u^{(j),+-}) g^avg(u^(j)) (eq. bad.numflux.non.cons)      */
  int tab_s;       /* > 0: use this explicit RK tableau instead of the degree's (tests)   */
  const double *tab_A, *tab_b;   /* [7][7] row-major, [7]                            */
  int limiter;     /* 1: subcell blending limiter (Sec. 4; Euler, cRKFR step only)       */
  double alpha_max;    /* cap of the blending coefficient                             */
  double alpha_fixed;  /* >= 0: this blending coefficient in every element (pins);
                          < 0: the smoothness indicator decides                        */
} or_desc;

/* ------------------------------------------------------------------------- */
/* Reference element: GLL points and weights on [0,1] (Sec. 2)               */
/* ------------------------------------------------------------------------- */

/* Legendre polynomial P_k(x) and derivative on [-1,1] by the three-term
 * recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}. */
static void legendre(int k, double x, double *P, double *dP) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (k == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int m = 1; m < k; ++m) {
    double p2 = ((2.0 * m + 1.0) * x * p1 - m * p0) / (m + 1.0);
    double d2 = d0 + (2.0 * m + 1.0) * p1;   /* P'_{m+1} = P'_{m-1} + (2m+1) P_m */
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *P = p1; *dP = d1;
}

/* GLL points on [-1,1] in closed form for N = 1..5 (roots of (1-x^2) P_N'). */
static int gll_ref_points(int N, double *x) {
  switch (N) {
    case 1: x[0] = -1; x[1] = 1; return 0;
    case 2: x[0] = -1; x[1] = 0; x[2] = 1; return 0;
    case 3: x[0] = -1; x[1] = -1.0 / sqrt(5.0); x[2] = 1.0 / sqrt(5.0); x[3] = 1; return 0;
    case 4: x[0] = -1; x[1] = -sqrt(3.0 / 7.0); x[2] = 0; x[3] = sqrt(3.0 / 7.0); x[4] = 1; return 0;
    case 5: {
      double a = sqrt(1.0 / 3.0 - 2.0 * sqrt(7.0) / 21.0);
      double b = sqrt(1.0 / 3.0 + 2.0 * sqrt(7.0) / 21.0);
      x[0] = -1; x[1] = -b; x[2] = -a; x[3] = a; x[4] = b; x[5] = 1; return 0;
    }
  }
  return -1;
}

/* Points xi_p and weights w_p on [0,1]: xi = (x+1)/2, w = 1/(N(N+1) P_N(x)^2)
 * (the [-1,1] weight 2/(N(N+1)P_N^2) halved), so that sum_p w_p = 1. */
static int gll01(int N, double *xi, double *w) {
  double x[OR_MAXNP];
  if (gll_ref_points(N, x)) return -1;
  for (int p = 0; p <= N; ++p) {
    double P, dP;
    legendre(N, x[p], &P, &dP);
    xi[p] = 0.5 * (x[p] + 1.0);
    w[p] = 1.0 / (N * (N + 1.0) * P * P);
  }
  xi[0] = 0.0; xi[N] = 1.0;
  return 0;
}

/* Lagrange basis l_q(s) = prod_{m != q} (s - xi_m) / (xi_q - xi_m). */
static double lagrange(int N, const double *xi, int q, double s) {
  double v = 1.0;
  for (int m = 0; m <= N; ++m)
    if (m != q) v *= (s - xi[m]) / (xi[q] - xi[m]);
  return v;
}

/* l_q'(s) by the product rule: sum_{k != q} 1/(xi_q - xi_k) prod_{m != q,k} (s - xi_m)/(xi_q - xi_m). */
static double lagrange_deriv(int N, const double *xi, int q, double s) {
  double sum = 0.0;
  for (int k = 0; k <= N; ++k) {
    if (k == q) continue;
    double t = 1.0 / (xi[q] - xi[k]);
    for (int m = 0; m <= N; ++m)
      if (m != q && m != k) t *= (s - xi[m]) / (xi[q] - xi[m]);
    sum += t;
  }
  return sum;
}

/* Huynh's g2 left correction function on [-1,1]:
 *   g_L = N/(2N+1) R_{N+1} + (N+1)/(2N+1) R_N,  R_k = (-1)^k/2 (P_k - P_{k-1}),
 * so g_L(-1) = 1, g_L(1) = 0.  Returns its derivative at x. */
static double g2_left_deriv_ref(int N, double x) {
  double Pn1, dPn1, Pn, dPn, Pnm1, dPnm1;
  legendre(N + 1, x, &Pn1, &dPn1);
  legendre(N, x, &Pn, &dPn);
  legendre(N - 1, x, &Pnm1, &dPnm1);
  double sN1 = ((N + 1) % 2 == 0) ? 0.5 : -0.5;   /* (-1)^(N+1)/2 */
  double sN = (N % 2 == 0) ? 0.5 : -0.5;          /* (-1)^N/2     */
  double dR_N1 = sN1 * (dPn1 - dPn);
  double dR_N = sN * (dPn - dPnm1);
  return (N * dR_N1 + (N + 1.0) * dR_N) / (2.0 * N + 1.0);
}

/* On [0,1]: g_L(xi) = gref(2 xi - 1) so g_L'(xi) = 2 gref'(2xi - 1);
 * g_R(xi) = g_L(1 - xi) so g_R'(xi) = -g_L'(1 - xi). */
static double gL_deriv01(int N, double xi) { return 2.0 * g2_left_deriv_ref(N, 2.0 * xi - 1.0); }
static double gR_deriv01(int N, double xi) { return -gL_deriv01(N, 1.0 - xi); }

/* Exported: reference-element tables (for pins). D is row-major D[p*(N+1)+q]. */
int or_tables(int N, double *xi, double *w, double *D, double *dgL, double *dgR) {
  if (N < 1 || N > OR_MAXN) return -1;
  if (gll01(N, xi, w)) return -1;
  for (int p = 0; p <= N; ++p) {
    for (int q = 0; q <= N; ++q) D[p * (N + 1) + q] = lagrange_deriv(N, xi, q, xi[p]);
    dgL[p] = gL_deriv01(N, xi[p]);
    dgR[p] = gR_deriv01(N, xi[p]);
  }
  return 0;
}

/* Exported: Lagrange basis value l_q(s), for pins. */
double or_lagrange(int N, int q, double s) {
  double xi[OR_MAXNP], w[OR_MAXNP];
  if (gll01(N, xi, w)) return NAN;
  return lagrange(N, xi, q, s);
}

/* ------------------------------------------------------------------------- */
/* Butcher tableaux (eq. butcher).  The paper fixes only the form; the        */
/* tableau per degree N is a reading: explicit RK of order N+1.               */
/*  N=1 Heun RK2, N=2 Heun RK3, N=3 classical RK4, N=4 Butcher's 6-stage      */
/*  order-5 method, N=5 Butcher's 7-stage order-6 method.                     */
/* ------------------------------------------------------------------------- */
int or_butcher(int N, int *s_out, double *A /* [7][7] */, double *b /* [7] */) {
  for (int i = 0; i < OR_MAXS * OR_MAXS; ++i) A[i] = 0.0;
  for (int i = 0; i < OR_MAXS; ++i) b[i] = 0.0;
#define a(i, j) A[((i) - 1) * OR_MAXS + ((j) - 1)]
  switch (N) {
    case 1:
      *s_out = 2; a(2, 1) = 1.0; b[0] = 0.5; b[1] = 0.5; return 0;
    case 2:
      *s_out = 3; a(2, 1) = 1.0 / 3.0; a(3, 2) = 2.0 / 3.0;
      b[0] = 0.25; b[1] = 0.0; b[2] = 0.75; return 0;
    case 3:
      *s_out = 4; a(2, 1) = 0.5; a(3, 2) = 0.5; a(4, 3) = 1.0;
      b[0] = 1.0 / 6.0; b[1] = 1.0 / 3.0; b[2] = 1.0 / 3.0; b[3] = 1.0 / 6.0; return 0;
    case 4:
      *s_out = 6;
      a(2, 1) = 0.25;
      a(3, 1) = 0.125; a(3, 2) = 0.125;
      a(4, 2) = -0.5; a(4, 3) = 1.0;
      a(5, 1) = 3.0 / 16.0; a(5, 4) = 9.0 / 16.0;
      a(6, 1) = -3.0 / 7.0; a(6, 2) = 2.0 / 7.0; a(6, 3) = 12.0 / 7.0; a(6, 4) = -12.0 / 7.0; a(6, 5) = 8.0 / 7.0;
      b[0] = 7.0 / 90.0; b[2] = 32.0 / 90.0; b[3] = 12.0 / 90.0; b[4] = 32.0 / 90.0; b[5] = 7.0 / 90.0;
      return 0;
    case 5:
      *s_out = 7;
      a(2, 1) = 1.0 / 3.0;
      a(3, 2) = 2.0 / 3.0;
      a(4, 1) = 1.0 / 12.0; a(4, 2) = 1.0 / 3.0; a(4, 3) = -1.0 / 12.0;
      a(5, 1) = -1.0 / 16.0; a(5, 2) = 9.0 / 8.0; a(5, 3) = -3.0 / 16.0; a(5, 4) = -3.0 / 8.0;
      a(6, 2) = 9.0 / 8.0; a(6, 3) = -3.0 / 8.0; a(6, 4) = -3.0 / 4.0; a(6, 5) = 0.5;
      a(7, 1) = 9.0 / 44.0; a(7, 2) = -9.0 / 11.0; a(7, 3) = 63.0 / 44.0; a(7, 4) = 18.0 / 11.0; a(7, 6) = -16.0 / 11.0;
      b[0] = 11.0 / 120.0; b[2] = 27.0 / 40.0; b[3] = 27.0 / 40.0; b[4] = -4.0 / 15.0; b[5] = -4.0 / 15.0; b[6] = 11.0 / 120.0;
      return 0;
  }
#undef a
  return -1;
}

/* ------------------------------------------------------------------------- */
/* Physics: u_t + f(u)_x + B(u) g(u)_x = 0 (eq. flux.and.non.cons)             */
/* ------------------------------------------------------------------------- */

static int nvars(const or_desc *d) { return d->eq == 0 ? d->dim + 2 : 9; }

/* Euler: u = (rho, rho v_1..rho v_dim, E), p = (gamma-1)(E - rho|v|^2/2). */
static void euler_prim(const or_desc *d, const double *u, double *rho, double *v, double *p) {
  *rho = u[0];
  double ke = 0.0;
  for (int k = 0; k < d->dim; ++k) { v[k] = u[1 + k] / u[0]; ke += 0.5 * u[0] * v[k] * v[k]; }
  *p = (d->gamma - 1.0) * (u[d->dim + 1] - ke);
}

/* GLM-MHD: u = (rho, rho v1, rho v2, rho v3, E, B1, B2, B3, psi),
 * E = p/(gamma-1) + rho|v|^2/2 + |B|^2/2 + psi^2/2. */
static void mhd_prim(const or_desc *d, const double *u, double *rho, double *v, double *p, double *B, double *psi) {
  *rho = u[0];
  double ke = 0.0, me = 0.0;
  for (int k = 0; k < 3; ++k) { v[k] = u[1 + k] / u[0]; ke += 0.5 * u[0] * v[k] * v[k]; B[k] = u[5 + k]; me += 0.5 * B[k] * B[k]; }
  *psi = u[8];
  *p = (d->gamma - 1.0) * (u[4] - ke - me - 0.5 * u[8] * u[8]);
}

/* Physical flux f^dir(u). */
static void phys_flux(const or_desc *d, int dir, const double *u, double *f) {
  double g = d->gamma;
  if (d->eq == 0) {
    double rho, v[3], p;
    euler_prim(d, u, &rho, v, &p);
    f[0] = rho * v[dir];
    for (int k = 0; k < d->dim; ++k) f[1 + k] = rho * v[dir] * v[k] + (k == dir ? p : 0.0);
    f[d->dim + 1] = v[dir] * (u[d->dim + 1] + p);
  } else {
    double rho, v[3], p, B[3], psi;
    mhd_prim(d, u, &rho, v, &p, B, &psi);
    double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    double B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    double vB = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
    double ch = d->c_h;
    f[0] = rho * v[dir];
    for (int k = 0; k < 3; ++k) f[1 + k] = rho * v[dir] * v[k] - B[dir] * B[k] + (k == dir ? p + 0.5 * B2 : 0.0);
    f[4] = v[dir] * (0.5 * rho * v2 + g * p / (g - 1.0) + B2) - B[dir] * vB + ch * psi * B[dir];
    for (int k = 0; k < 3; ++k) f[5 + k] = (k == dir) ? ch * psi : v[dir] * B[k] - v[k] * B[dir];
    f[8] = ch * B[dir];
  }
}

/* Non-conservative product B^dir(ua) g^dir(ub), g^dir = (B_dir, psi):
 *   phi_Powell(ua) * B_dir(ub) + phi_GLM^dir(ua) * psi(ub),
 *   phi_Powell = (0, B, v.B, v, 0), phi_GLM^dir = (0, 0,0,0, v_dir psi, 0,0,0, v_dir).
 * Zero for Euler (B = 0). */
static void nc_product(const or_desc *d, int dir, const double *ua, const double *ub, double *out) {
  int M = nvars(d);
  for (int m = 0; m < M; ++m) out[m] = 0.0;
  if (d->eq == 0) return;
  double rho, v[3], p, B[3], psi;
  mhd_prim(d, ua, &rho, v, &p, B, &psi);
  double gB = ub[5 + dir], gpsi = ub[8];
  double vB = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
  out[1] = B[0] * gB; out[2] = B[1] * gB; out[3] = B[2] * gB;
  out[4] = vB * gB + v[dir] * psi * gpsi;
  out[5] = v[0] * gB; out[6] = v[1] * gB; out[7] = v[2] * gB;
  out[8] = v[dir] * gpsi;
}

/* Spectral radius of f'(u) + B(u) g'(u) in direction dir (eqs. rusanov.wave.speed,
 * combined.wave.speed).  Euler: |v_dir| + c.  GLM-MHD: |v_dir| + max(c_f, c_h). */
static double wave_speed(const or_desc *d, int dir, const double *u) {
  double g = d->gamma;
  if (d->eq == 0) {
    double rho, v[3], p;
    euler_prim(d, u, &rho, v, &p);
    return fabs(v[dir]) + sqrt(g * p / rho);
  } else {
    double rho, v[3], p, B[3], psi;
    mhd_prim(d, u, &rho, v, &p, B, &psi);
    double a2 = g * p / rho;
    double b2 = (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]) / rho;
    double bd2 = B[dir] * B[dir] / rho;
    double cf2 = 0.5 * (a2 + b2 + sqrt((a2 + b2) * (a2 + b2) - 4.0 * a2 * bd2));
    /* the GLM pair travels at v_dir -+ c_h because of the non-conservative terms */
    double c = sqrt(cf2) > d->c_h ? sqrt(cf2) : d->c_h;
    return fabs(v[dir]) + c;
  }
}

/* Logarithmic mean (a-b)/(ln a - ln b).  For a close to b it uses the series
 * (a+b) / (2 (1 + u/3 + u^2/5 + u^3/7)), u = ((a-b)/(a+b))^2, whose
 * truncation error u^4/9 is below FP64 round-off for u < 1e-4; otherwise
 * ln a - ln b is evaluated as log1p((a-b)/b), which keeps its relative
 * accuracy when a/b is close to 1. */
double or_logmean(double a, double b) {
  double f = (a - b) / (a + b);
  double u = f * f;
  if (u < 1e-4) return (a + b) / (2.0 * (1.0 + u / 3.0 + u * u / 5.0 + u * u * u / 7.0));
  return (a - b) / log1p((a - b) / b);
}

/* Symmetric two-point volume flux f_S^dir(uL, uR) (eq. entropy.cons.flux.dev). */
static void two_point_flux(const or_desc *d, int dir, const double *uL, const double *uR, double *f) {
  int M = nvars(d);
  double g = d->gamma;
  if (d->vol == 2) {                       /* central: (f(uL) + f(uR))/2, reduces to D f (Sec. 3) */
    double fL[OR_MAXM], fR[OR_MAXM];
    phys_flux(d, dir, uL, fL);
    phys_flux(d, dir, uR, fR);
    for (int m = 0; m < M; ++m) f[m] = 0.5 * (fL[m] + fR[m]);
    return;
  }
  if (d->eq == 0) {
    double rL, vL[3], pL, rR, vR[3], pR;
    euler_prim(d, uL, &rL, vL, &pL);
    euler_prim(d, uR, &rR, vR, &pR);
    double vavg[3];
    for (int k = 0; k < d->dim; ++k) vavg[k] = 0.5 * (vL[k] + vR[k]);
    double pavg = 0.5 * (pL + pR);
    if (d->vol == 0) {                     /* Ranocha: entropy conservative and kinetic energy preserving */
      double rho_ln = or_logmean(rL, rR);
      double rp_ln = or_logmean(rL / pL, rR / pR);
      double vv = 0.0;
      for (int k = 0; k < d->dim; ++k) vv += 0.5 * vL[k] * vR[k];
      f[0] = rho_ln * vavg[dir];
      for (int k = 0; k < d->dim; ++k) f[1 + k] = f[0] * vavg[k] + (k == dir ? pavg : 0.0);
      f[d->dim + 1] = f[0] * (vv + 1.0 / ((g - 1.0) * rp_ln)) + 0.5 * (pL * vR[dir] + pR * vL[dir]);
    } else {                               /* Kennedy-Gruber: kinetic energy preserving, arithmetic means */
      double ravg = 0.5 * (rL + rR);
      double eavg = 0.5 * (uL[d->dim + 1] / rL + uR[d->dim + 1] / rR);
      f[0] = ravg * vavg[dir];
      for (int k = 0; k < d->dim; ++k) f[1 + k] = ravg * vavg[dir] * vavg[k] + (k == dir ? pavg : 0.0);
      f[d->dim + 1] = (ravg * eavg + pavg) * vavg[dir];
    }
    return;
  }
  /* GLM-MHD entropy-conservative flux, derived from [[w]].f = [[psi]] + {{theta}}[[B_dir]]
   * with w the entropy variables of S = -rho s/(gamma-1) and theta = w.phi_Powell. */
  double rL, vL[3], pL, BL[3], psL, rR, vR[3], pR, BR[3], psR;
  mhd_prim(d, uL, &rL, vL, &pL, BL, &psL);
  mhd_prim(d, uR, &rR, vR, &pR, BR, &psR);
  double betaL = 0.5 * rL / pL, betaR = 0.5 * rR / pR;
  double rho_ln = or_logmean(rL, rR);
  double beta_ln = or_logmean(betaL, betaR);
  double ravg = 0.5 * (rL + rR), betaavg = 0.5 * (betaL + betaR);
  double v[3], B[3];
  for (int k = 0; k < 3; ++k) { v[k] = 0.5 * (vL[k] + vR[k]); B[k] = 0.5 * (BL[k] + BR[k]); }
  double psi = 0.5 * (psL + psR);
  double v2avg = 0.5 * ((vL[0] * vL[0] + vL[1] * vL[1] + vL[2] * vL[2]) + (vR[0] * vR[0] + vR[1] * vR[1] + vR[2] * vR[2]));
  double B2L = BL[0] * BL[0] + BL[1] * BL[1] + BL[2] * BL[2];
  double B2R = BR[0] * BR[0] + BR[1] * BR[1] + BR[2] * BR[2];
  double B2avg = 0.5 * (B2L + B2R);
  double vB2avg = 0.5 * (vL[dir] * B2L + vR[dir] * B2R);
  double psiBavg = 0.5 * (psL * BL[dir] + psR * BR[dir]);
  double vBavg = 0.5 * ((vL[0] * BL[0] + vL[1] * BL[1] + vL[2] * BL[2]) + (vR[0] * BR[0] + vR[1] * BR[1] + vR[2] * BR[2]));
  double ptilde = ravg / (2.0 * betaavg);
  double ch = d->c_h;
  f[0] = rho_ln * v[dir];
  for (int k = 0; k < 3; ++k) f[1 + k] = f[0] * v[k] - B[dir] * B[k] + (k == dir ? ptilde + 0.5 * B2avg : 0.0);
  for (int k = 0; k < 3; ++k) f[5 + k] = (k == dir) ? ch * psi : v[dir] * B[k] - v[k] * B[dir];
  f[8] = ch * B[dir];
  f[4] = f[0] * 0.5 * (1.0 / ((g - 1.0) * beta_ln) - v2avg)
       + f[1] * v[0] + f[2] * v[1] + f[3] * v[2]
       + f[5] * B[0] + f[6] * B[1] + f[7] * B[2] + f[8] * psi
       - 0.5 * vB2avg - ch * psiBavg + B[dir] * vBavg;
}

/* Exported point-wise physics, for pins. */
int or_phys_flux(const or_desc *d, int dir, const double *u, double *f) { phys_flux(d, dir, u, f); return 0; }
int or_two_point_flux(const or_desc *d, int dir, const double *uL, const double *uR, double *f) { two_point_flux(d, dir, uL, uR, f); return 0; }
int or_nc_product(const or_desc *d, int dir, const double *ua, const double *ub, double *out) { nc_product(d, dir, ua, ub, out); return 0; }
double or_wave_speed(const or_desc *d, int dir, const double *u) { return wave_speed(d, dir, u); }

/* ------------------------------------------------------------------------- */
/* Mesh helpers                                                              */
/* ------------------------------------------------------------------------- */

typedef struct {
  int M, n, np, E, S;
  double xi[OR_MAXNP], w[OR_MAXNP], D[OR_MAXNP][OR_MAXNP];
  double dgL[OR_MAXNP], dgR[OR_MAXNP];
  double lend0[OR_MAXNP], lend1[OR_MAXNP];   /* l_p(0), l_p(1) */
  double A[OR_MAXS][OR_MAXS], b[OR_MAXS];
  double dx[3];
} or_mesh;

static int mesh_setup(const or_desc *d, or_mesh *m) {
  if (d->dim < 1 || d->dim > 3 || d->N < 1 || d->N > OR_MAXN) return -1;
  if (d->eq == 1 && d->dim != 2) return -1;
  m->M = nvars(d);
  m->n = d->N + 1;
  m->np = 1; m->E = 1;
  for (int k = 0; k < d->dim; ++k) {
    if (d->cells[k] < 1) return -1;
    m->np *= m->n; m->E *= d->cells[k];
    m->dx[k] = (d->hi[k] - d->lo[k]) / d->cells[k];
  }
  double D[OR_MAXNP * OR_MAXNP];
  if (or_tables(d->N, m->xi, m->w, D, m->dgL, m->dgR)) return -1;
  for (int p = 0; p < m->n; ++p) {
    for (int q = 0; q < m->n; ++q) m->D[p][q] = D[p * m->n + q];
    m->lend0[p] = lagrange(d->N, m->xi, p, 0.0);
    m->lend1[p] = lagrange(d->N, m->xi, p, 1.0);
  }
  double A[OR_MAXS * OR_MAXS], b[OR_MAXS];
  if (or_butcher(d->N, &m->S, A, b)) return -1;
  if (d->tab_s > 0) {
    if (d->tab_s > OR_MAXS || !d->tab_A || !d->tab_b) return -1;
    m->S = d->tab_s;
    for (int k = 0; k < OR_MAXS * OR_MAXS; ++k) A[k] = d->tab_A[k];
    for (int k = 0; k < OR_MAXS; ++k) b[k] = d->tab_b[k];
  }
  for (int i = 0; i < OR_MAXS; ++i) { m->b[i] = b[i]; for (int j = 0; j < OR_MAXS; ++j) m->A[i][j] = A[i * OR_MAXS + j]; }
  return 0;
}

/* node index (i,j,k) -> flat, i fastest */
static int node_id(const or_mesh *m, const int *ijk, int dim) {
  int id = 0, mul = 1;
  for (int k = 0; k < dim; ++k) { id += ijk[k] * mul; mul *= m->n; }
  return id;
}
static void node_ijk(const or_mesh *m, int id, int dim, int *ijk) {
  for (int k = 0; k < 3; ++k) ijk[k] = 0;
  for (int k = 0; k < dim; ++k) { ijk[k] = id % m->n; id /= m->n; }
}
static void elem_ijk(const or_desc *d, int e, int *c) {
  c[0] = c[1] = c[2] = 0;
  for (int k = 0; k < d->dim; ++k) { c[k] = e % d->cells[k]; e /= d->cells[k]; }
}
static int elem_id(const or_desc *d, const int *c) {
  int id = 0, mul = 1;
  for (int k = 0; k < d->dim; ++k) { id += c[k] * mul; mul *= d->cells[k]; }
  return id;
}
/* periodic neighbour of element e in direction dir, offset +-1 */
static int neighbour(const or_desc *d, int e, int dir, int off) {
  int c[3];
  elem_ijk(d, e, c);
  c[dir] = (c[dir] + off + d->cells[dir]) % d->cells[dir];
  return elem_id(d, c);
}

/* ------------------------------------------------------------------------- */
/* Local residual (inner-stage operator, Sec. 3):                            */
/*  R(u)_p = sum_dir 1/dx_dir [ sum_q 2 D_pq f_S(u_p,u_q)                     */
/*                              + sum_q D_pq (B g)_NS(u_p,u_q) ]              */
/* with (B g)_NS(u_p,u_q) = B(u_p) g(u_q); q runs along p's line in dir.      */
/* u and R are one element, [node][var].                                      */
/* ------------------------------------------------------------------------- */
static void local_residual(const or_desc *d, const or_mesh *m, const double *u, double *R) {
  int M = m->M;
  for (int i = 0; i < m->np * M; ++i) R[i] = 0.0;
  for (int p = 0; p < m->np; ++p) {
    int ijk[3];
    node_ijk(m, p, d->dim, ijk);
    for (int dir = 0; dir < d->dim; ++dir) {
      int pd = ijk[dir];
      for (int qd = 0; qd < m->n; ++qd) {
        int qijk[3] = {ijk[0], ijk[1], ijk[2]};
        qijk[dir] = qd;
        int q = node_id(m, qijk, d->dim);
        double fs[OR_MAXM], nc[OR_MAXM];
        two_point_flux(d, dir, &u[p * M], &u[q * M], fs);
        nc_product(d, dir, &u[p * M], &u[q * M], nc);
        for (int v = 0; v < M; ++v)
          R[p * M + v] += (2.0 * m->D[pd][qd] * fs[v] + m->D[pd][qd] * nc[v]) / m->dx[dir];
      }
    }
  }
}

static void gather_elem(const or_mesh *m, const double *U, int e, double *ue) {
  for (int v = 0; v < m->M; ++v)
    for (int p = 0; p < m->np; ++p) ue[p * m->M + v] = U[((size_t)v * m->E + e) * m->np + p];
}

/* ------------------------------------------------------------------------- */
/* dt from the CFL condition (reading: dt = CFL / max_p sum_d sigma_d/dx_d).  */
/* ------------------------------------------------------------------------- */
double or_cfl_dt(const or_desc *d, const double *U) {
  or_mesh m;
  if (mesh_setup(d, &m)) return -1.0;
  double mx = 0.0;
  double ue[OR_MAXNP * OR_MAXNP * OR_MAXNP * OR_MAXM];
  for (int e = 0; e < m.E; ++e) {
    gather_elem(&m, U, e, ue);
    for (int p = 0; p < m.np; ++p) {
      double s = 0.0;
      for (int dir = 0; dir < d->dim; ++dir) s += wave_speed(d, dir, &ue[p * m.M]) / m.dx[dir];
      if (s > mx) mx = s;
    }
  }
  return d->cfl / mx;
}

/* ------------------------------------------------------------------------- */
/* Face traces and numerical fluxes.                                         */
/* Extrapolation of a nodal field to face side 0 (xi_dir = 0) or 1 (xi_dir = 1)
 * of element e for the face node indexed by the other coordinates:
 * sum_p field_p l_p(0 or 1) along the line (Sec. 2.1).                       */
/* ------------------------------------------------------------------------- */
static void extrapolate(const or_desc *d, const or_mesh *m, const double *field /*[node][var] of the element*/,
                        int dir, int side, const int *fijk, double *out) {
  for (int v = 0; v < m->M; ++v) out[v] = 0.0;
  for (int p = 0; p < m->n; ++p) {
    int ijk[3] = {fijk[0], fijk[1], fijk[2]};
    ijk[dir] = p;
    int id = node_id(m, ijk, d->dim);
    double l = side ? m->lend1[p] : m->lend0[p];
    for (int v = 0; v < m->M; ++v) out[v] += field[id * m->M + v] * l;
  }
}

/* Per-element time-averaged data of one cRKFR step. */
typedef struct {
  double *Rbar;      /* [E][np][M]           sum_i b_i R(u^(i))                 */
  double *Ubar;      /* [E][np][M]           sum_i b_i u^(i)                    */
  double *Fbar;      /* [dim][E][np][M]      sum_i b_i f^dir(u^(i))             */
  double *Fnc;       /* [dim][E][np][M]      sum_i b_i B^dir(u^(i)) g^dir(u^(i)) */
  double *un;        /* [E][np][M]           u^n per element                    */
  double *Us;        /* [E][S][np][M]        stage states u^(i) (ncflux 1 only) */
} or_work;

/* The cRK inner stages of one element (eq. crkfr.inner) and its time averages
 * (eqs. disc.avg.flux, local.time.avg.non.cons and the flux-differencing final
 * volume term of Sec. 3). */
static void element_stages(const or_desc *d, const or_mesh *m, const double *une, double dt,
                           double *Rbar, double *Ubar, double *Fbar /*[dim][np][M] stride np*M*/, double *Fnc,
                           double *Ust /* [S][np][M] stage states, or NULL */) {
  int M = m->M, np = m->np, S = m->S;
  size_t sz = (size_t)np * M;
  double *us = malloc(sizeof(double) * sz * S);
  double *R = malloc(sizeof(double) * sz * S);
  for (size_t k = 0; k < sz; ++k) { Rbar[k] = 0.0; Ubar[k] = 0.0; }
  for (int dir = 0; dir < d->dim; ++dir)
    for (size_t k = 0; k < sz; ++k) { Fbar[dir * sz + k] = 0.0; Fnc[dir * sz + k] = 0.0; }
  for (int i = 0; i < S; ++i) {
    /* u^(i) = u^n - dt sum_{j<i} a_ij R(u^(j)) */
    for (size_t k = 0; k < sz; ++k) {
      double acc = 0.0;
      for (int j = 0; j < i; ++j) acc += m->A[i][j] * R[j * sz + k];
      us[i * sz + k] = une[k] - dt * acc;
    }
    local_residual(d, m, &us[i * sz], &R[i * sz]);
    if (Ust)
      for (size_t k = 0; k < sz; ++k) Ust[i * sz + k] = us[i * sz + k];
    double bi = m->b[i];
    for (size_t k = 0; k < sz; ++k) { Rbar[k] += bi * R[i * sz + k]; Ubar[k] += bi * us[i * sz + k]; }
    for (int p = 0; p < np; ++p)
      for (int dir = 0; dir < d->dim; ++dir) {
        double f[OR_MAXM], nc[OR_MAXM];
        phys_flux(d, dir, &us[i * sz + p * M], f);
        nc_product(d, dir, &us[i * sz + p * M], &us[i * sz + p * M], nc);
        for (int v = 0; v < M; ++v) {
          Fbar[dir * sz + p * M + v] += bi * f[v];
          Fnc[dir * sz + p * M + v] += bi * nc[v];
        }
      }
  }
  free(us);
  free(R);
}

/* g^dir(u) = (B_dir, psi) enters the non-conservative numerical flux through
 * g^avg = (g(U-) + g(U+))/2; B^dir(u^{n+-}) g^avg is nc_product with the
 * "g" argument replaced by the average of the two U states. */
static void nc_with_gavg(const or_desc *d, int dir, const double *un_side, const double *Um, const double *Up, double *out) {
  double gavg_state[OR_MAXM];
  int M = nvars(d);
  for (int v = 0; v < M; ++v) gavg_state[v] = 0.5 * (Um[v] + Up[v]);
  nc_product(d, dir, un_side, gavg_state, out);
}

/* ------------------------------------------------------------------------- */
/* Subcell blending limiter (Sec. 4: the paper's Kelvin-Helmholtz and         */
/* Richtmyer-Meshkov runs blend the cRKFR update with a first-order subcell   */
/* finite-volume update, the coefficient capped by alpha_max; the paper cites */
/* the method without printing it).  Readings, compressible Euler only:       */
/*  - subcells: the element line of N+1 GLL points is cut into N+1 subcells   */
/*    of widths w_p dx (the quadrature weights); subcell p holds node p;      */
/*  - low-order update: first-order finite volumes with the Rusanov flux of   */
/*    the two u^n node values at every interior subcell face, forward Euler   */
/*    in time, per direction summed (tensor product);                        */
/*  - at an element face both updates take one flux: the blend                */
/*    (1 - a_f) F^num + a_f f_lo, a_f the mean of the two elements'           */
/*    coefficients, F^num the time-averaged Rusanov flux of eq. numflux.cons, */
/*    f_lo the Rusanov flux of the u^n traces; where a_f > 0 it is pulled     */
/*    toward f_lo (F = f_lo + theta (blend - f_lo)) by the largest theta in   */
/*    [0,1] for which both adjacent end subcells' one-direction low-order     */
/*    states keep rho and p above a tenth of their values with f_lo (density  */
/*    linear, pressure concave in theta);                                    */
/*  - u^{n+1} = (1 - a_e) u^H + a_e u^L per element (u^L alone where a_e = 1, */
/*    f_lo alone where a_f = 1);                                             */
/*  - a_e from the modal smoothness indicator of rho p: energy fraction of    */
/*    the highest modes in the orthonormal Legendre basis, mapped through a   */
/*    logistic function with threshold 0.5 10^(-1.8 (N+1)^(1/4)) and         */
/*    sharpness ln(9999), set to 0 below 0.001 and 1 above 0.999, capped by   */
/*    alpha_max, then raised to half of the largest face neighbour's value.   */
/* ------------------------------------------------------------------------- */

/* orthonormal Legendre polynomial sqrt((2j+1)/2) P_j(x) on [-1,1] */
static double legendre_orthonormal(int j, double x) {
  double P, dP;
  legendre(j, x, &P, &dP);
  return sqrt((2.0 * j + 1.0) / 2.0) * P;
}

/* Solve A x = b (n <= OR_MAXNP) by Gaussian elimination with partial pivoting;
 * A (row-major) and b are overwritten, x returned in b. */
static void solve_dense(int n, double *A, double *b) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[i * n + k]) > fabs(A[piv * n + k])) piv = i;
    if (piv != k) {
      for (int j = 0; j < n; ++j) { double t = A[k * n + j]; A[k * n + j] = A[piv * n + j]; A[piv * n + j] = t; }
      double t = b[k]; b[k] = b[piv]; b[piv] = t;
    }
    for (int i = k + 1; i < n; ++i) {
      double f = A[i * n + k] / A[k * n + k];
      for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double acc = b[k];
    for (int j = k + 1; j < n; ++j) acc -= A[k * n + j] * b[j];
    b[k] = acc / A[k * n + k];
  }
}

/* Highest-mode energy fraction E of one element's rho p ([node][var] in ue):
 * modal coefficients m of the tensor-product orthonormal Legendre expansion
 * interpolating rho p at the nodes (a 1D Vandermonde solve along every
 * direction), then E = max((T - T1)/T, (T1 - T2)/T1) with T the sum of all
 * m^2, T1 over the modes of degree <= N-1 in every direction, T2 <= N-2
 * (the second fraction only for N >= 2). */
double or_indicator_energy(const or_desc *d, const double *ue) {
  int n = d->N + 1, dim = d->dim, M = nvars(d);
  double x[OR_MAXNP];
  gll_ref_points(d->N, x);
  int np = 1;
  for (int k = 0; k < dim; ++k) np *= n;
  double m[OR_MAXNP * OR_MAXNP * OR_MAXNP];
  for (int p = 0; p < np; ++p) {
    double rho, v[3], pr;
    euler_prim(d, &ue[p * M], &rho, v, &pr);
    m[p] = rho * pr;
  }
  /* along direction k: for every line, solve V c = values (V_pj = phi_j(x_p)) */
  for (int k = 0; k < dim; ++k) {
    int stride = 1;
    for (int j = 0; j < k; ++j) stride *= n;
    for (int base = 0; base < np; ++base) {
      if ((base / stride) % n != 0) continue;           /* first node of a line in direction k */
      double V[OR_MAXNP * OR_MAXNP], b[OR_MAXNP];
      for (int p = 0; p < n; ++p) {
        b[p] = m[base + p * stride];
        for (int j = 0; j < n; ++j) V[p * n + j] = legendre_orthonormal(j, x[p]);
      }
      solve_dense(n, V, b);
      for (int p = 0; p < n; ++p) m[base + p * stride] = b[p];
    }
  }
  double T = 0.0, T1 = 0.0, T2 = 0.0;
  for (int p = 0; p < np; ++p) {
    int rem = p, top = 0;
    for (int k = 0; k < dim; ++k) { int j = rem % n; rem /= n; if (j > top) top = j; }
    double e2 = m[p] * m[p];
    T += e2;
    if (top <= d->N - 1) T1 += e2;
    if (top <= d->N - 2) T2 += e2;
  }
  double E = (T - T1) / T;
  if (d->N >= 2) {
    double E2 = (T1 - T2) / T1;
    if (E2 > E) E = E2;
  }
  return E;
}

/* Blending coefficient of one element before the neighbour smoothing. */
static double alpha_raw(const or_desc *d, const double *ue) {
  double E = or_indicator_energy(d, ue);
  double T = 0.5 * pow(10.0, -1.8 * pow(d->N + 1.0, 0.25));
  double s = log(9999.0);
  double a = 1.0 / (1.0 + exp(-(s / T) * (E - T)));
  if (a < 0.001) a = 0.0;
  if (a > 0.999) a = 1.0;
  if (a > d->alpha_max) a = d->alpha_max;
  return a;
}

/* Exported: per element the coefficient before (raw, may be NULL) and after
 * the smoothing a_e = max(raw_e, raw_nb / 2 over the 2 dim face neighbours);
 * alpha_fixed >= 0 gives that value everywhere. */
int or_blend_alpha(const or_desc *d, const double *U, double *raw, double *alpha) {
  or_mesh m;
  if (mesh_setup(d, &m) || d->eq != 0) return -1;
  double *r = malloc(sizeof(double) * m.E);
  double ue[OR_MAXNP * OR_MAXNP * OR_MAXNP * OR_MAXM];
  for (int e = 0; e < m.E; ++e) {
    if (d->alpha_fixed >= 0.0) { r[e] = d->alpha_fixed; continue; }
    gather_elem(&m, U, e, ue);
    r[e] = alpha_raw(d, ue);
  }
  for (int e = 0; e < m.E; ++e) {
    double a = r[e];
    if (d->alpha_fixed < 0.0)
      for (int dir = 0; dir < d->dim; ++dir)
        for (int off = -1; off <= 1; off += 2) {
          double h = 0.5 * r[neighbour(d, e, dir, off)];
          if (h > a) a = h;
        }
    if (raw) raw[e] = r[e];
    alpha[e] = a;
  }
  free(r);
  return 0;
}

/* First-order Rusanov flux of two states: (f(uL) + f(uR))/2 - lam/2 (uR - uL),
 * lam = max(sigma(uL), sigma(uR)). */
static void rusanov_flux(const or_desc *d, int dir, const double *uL, const double *uR, double *F) {
  int M = nvars(d);
  double fL[OR_MAXM], fR[OR_MAXM];
  phys_flux(d, dir, uL, fL);
  phys_flux(d, dir, uR, fR);
  double lL = wave_speed(d, dir, uL), lR = wave_speed(d, dir, uR);
  double lam = lL > lR ? lL : lR;
  for (int v = 0; v < M; ++v) F[v] = 0.5 * (fL[v] + fR[v]) - 0.5 * lam * (uR[v] - uL[v]);
}

static void euler_rho_p(const or_desc *d, const double *u, double *rho, double *p) {
  double v[3];
  euler_prim(d, u, rho, v, p);
}

/* Largest theta in [0,1] with rho(u(theta)) >= rho(u(0))/10 and
 * p(u(theta)) >= p(u(0))/10 along u(theta) = u0 + theta du (density linear in
 * theta; pressure concave, so its chord bound is safe). 0 if u0 itself is not
 * admissible. */
static double admissible_theta(const or_desc *d, const double *u0, const double *du) {
  int M = nvars(d);
  double r0, p0;
  euler_rho_p(d, u0, &r0, &p0);
  if (!(r0 > 0.0) || !(p0 > 0.0)) return 0.0;
  double u1[OR_MAXM];
  for (int v = 0; v < M; ++v) u1[v] = u0[v] + du[v];
  double r1, p1;
  euler_rho_p(d, u1, &r1, &p1);
  double theta = 1.0;
  double er = 0.1 * r0;
  if (r1 < er) theta = (r0 - er) / (r0 - r1);
  double ut[OR_MAXM];
  for (int v = 0; v < M; ++v) ut[v] = u0[v] + theta * du[v];
  double rt, pt;
  euler_rho_p(d, ut, &rt, &pt);
  double ep = 0.1 * p0;
  if (pt < ep) theta = theta * (p0 - ep) / (p0 - pt);
  return theta;
}

/* The element-face flux of the limited step (readings above).  um, up: u^n
 * traces of the '-' and '+' element; umi, upi: u^n at the neighbouring
 * interior node of each (index N-1 of '-', 1 of '+'); Fho: time-averaged
 * Rusanov flux; wN, w0: end subcell widths; a_f: face coefficient. */
static void limited_face_flux(const or_desc *d, int dir, const double *um, const double *up, const double *umi,
                              const double *upi, const double *Fho, double a_f, double dt, double dx, double wN,
                              double w0, double *F) {
  int M = nvars(d);
  double flo[OR_MAXM], Fb[OR_MAXM];
  rusanov_flux(d, dir, um, up, flo);
  /* a_f = 1 takes f_lo alone (so a high-order flux that is not finite on
   * data the first-order scheme still handles does not enter) */
  for (int v = 0; v < M; ++v) Fb[v] = a_f >= 1.0 ? flo[v] : (1.0 - a_f) * Fho[v] + a_f * flo[v];
  if (!(a_f > 0.0)) {
    for (int v = 0; v < M; ++v) F[v] = Fb[v];
    return;
  }
  /* one-direction low-order states of the two end subcells, with the face
   * flux f_lo (theta = 0) and with the blend (theta = 1):
   *   '-' end: u_N - (dim dt/(w_N dx)) (F - f_{N-1/2}),  '+' end: u_0 - (dim dt/(w_0 dx)) (f_{1/2} - F) */
  double fmi[OR_MAXM], fpi[OR_MAXM];
  rusanov_flux(d, dir, umi, um, fmi);
  rusanov_flux(d, dir, up, upi, fpi);
  double cm = d->dim * dt / (wN * dx), cp = d->dim * dt / (w0 * dx);
  double lm[OR_MAXM], dm[OR_MAXM], lp[OR_MAXM], dpl[OR_MAXM];
  for (int v = 0; v < M; ++v) {
    lm[v] = um[v] - cm * (flo[v] - fmi[v]);
    dm[v] = -cm * (Fb[v] - flo[v]);
    lp[v] = up[v] - cp * (fpi[v] - flo[v]);
    dpl[v] = cp * (Fb[v] - flo[v]);
  }
  double tm = admissible_theta(d, lm, dm), tp = admissible_theta(d, lp, dpl);
  double theta = tm < tp ? tm : tp;
  for (int v = 0; v < M; ++v) F[v] = flo[v] + theta * (Fb[v] - flo[v]);
}

/* Exported for pins: the limited element-face flux (arguments as above). */
int or_limited_face_flux(const or_desc *d, int dir, const double *um, const double *up, const double *umi,
                         const double *upi, const double *Fho, double a_f, double dt, double dx, double wN,
                         double w0, double *F) {
  if (d->eq != 0 || dir < 0 || dir >= d->dim) return -1;
  limited_face_flux(d, dir, um, up, umi, upi, Fho, a_f, dt, dx, wN, w0, F);
  return 0;
}

/* Time-averaged data of a set of elements: element e sits at local index
 * loc[e] of the W arrays (Fbar, Fnc: [dir][nloc][np][M]). */
typedef struct {
  or_work W;
  int *loc;     /* [E] local index or -1 */
  int nloc;
} or_set;

static void set_alloc(or_set *S, int E, int nloc, size_t sz, int dim, int stages) {
  S->nloc = nloc;
  S->loc = malloc(sizeof(int) * E);
  for (int e = 0; e < E; ++e) S->loc[e] = -1;
  S->W.Rbar = malloc(sizeof(double) * sz * nloc);
  S->W.Ubar = malloc(sizeof(double) * sz * nloc);
  S->W.Fbar = malloc(sizeof(double) * sz * nloc * dim);
  S->W.Fnc = malloc(sizeof(double) * sz * nloc * dim);
  S->W.un = malloc(sizeof(double) * sz * nloc);
  S->W.Us = stages > 0 ? malloc(sizeof(double) * sz * nloc * stages) : NULL;
}
static void set_free(or_set *S) {
  free(S->loc); free(S->W.Rbar); free(S->W.Ubar); free(S->W.Fbar); free(S->W.Fnc); free(S->W.un); free(S->W.Us);
}

/* 1. element-local stages and time averages of element e into local slot k */
static void set_stages(const or_desc *d, const or_mesh *m, const double *Un, double dt, or_set *S, int e, int k) {
  size_t sz = (size_t)m->np * m->M;
  int dim = d->dim;
  double *fb = malloc(sizeof(double) * sz * dim), *fn = malloc(sizeof(double) * sz * dim);
  S->loc[e] = k;
  gather_elem(m, Un, e, &S->W.un[k * sz]);
  element_stages(d, m, &S->W.un[k * sz], dt, &S->W.Rbar[k * sz], &S->W.Ubar[k * sz], fb, fn,
                 S->W.Us ? &S->W.Us[(size_t)k * m->S * sz] : NULL);
  for (int dir = 0; dir < dim; ++dir)
    for (size_t q = 0; q < sz; ++q) {
      S->W.Fbar[((size_t)dir * S->nloc + k) * sz + q] = fb[dir * sz + q];
      S->W.Fnc[((size_t)dir * S->nloc + k) * sz + q] = fn[dir * sz + q];
    }
  free(fb);
  free(fn);
}

/* 2. final update of element e ([node][var] into unew), with the face terms of
 *    eq. crkfr.non.cons.final evaluated at both faces of every direction; the
 *    element and its neighbours must be in the set. */
/*    alpha != NULL: the limited step (subcell blending, readings above): the
 *    face fluxes of both updates are the limited face fluxes, and the result
 *    is (1 - a_e) u^H + a_e u^L. */
static void set_update(const or_desc *d, const or_mesh *m, const or_set *S, int e, double dt, double *unew,
                       const double *alpha) {
  int M = m->M, np = m->np, dim = d->dim;
  size_t sz = (size_t)np * M;
  const or_work *W = &S->W;
  const int ke = S->loc[e];
  /* limited step: face flux per direction, side and face node */
  double *Fface = alpha ? malloc(sizeof(double) * 3 * 2 * np * M) : NULL;
  for (size_t k = 0; k < sz; ++k) unew[k] = W->un[ke * sz + k] - dt * W->Rbar[ke * sz + k];
  for (int dir = 0; dir < dim; ++dir) {
    for (int side = 0; side < 2; ++side) {
      /* side 1: interface e+1/2 (element e is the '-' state); side 0: e-1/2 (e is '+') */
      int nb = neighbour(d, e, dir, side ? +1 : -1);
      const int kn = S->loc[nb];
      const double *Fe = &W->Fbar[((size_t)dir * S->nloc + ke) * sz], *Fn = &W->Fbar[((size_t)dir * S->nloc + kn) * sz];
      const double *Ne = &W->Fnc[((size_t)dir * S->nloc + ke) * sz], *Nn = &W->Fnc[((size_t)dir * S->nloc + kn) * sz];
      for (int fnode = 0; fnode < np; ++fnode) {
        int fijk[3];
        node_ijk(m, fnode, dim, fijk);
        if (fijk[dir] != 0) continue;            /* enumerate face nodes once */
        double um[OR_MAXM], up[OR_MAXM], Um[OR_MAXM], Up[OR_MAXM], Fm[OR_MAXM], Fp[OR_MAXM], Nm[OR_MAXM], Np_[OR_MAXM];
        const double *uel = &W->un[ke * sz], *unb = &W->un[kn * sz];
        const double *Uel = &W->Ubar[ke * sz], *Unb = &W->Ubar[kn * sz];
        if (side) {   /* e is '-', nb is '+' */
          extrapolate(d, m, uel, dir, 1, fijk, um); extrapolate(d, m, unb, dir, 0, fijk, up);
          extrapolate(d, m, Uel, dir, 1, fijk, Um); extrapolate(d, m, Unb, dir, 0, fijk, Up);
          extrapolate(d, m, Fe, dir, 1, fijk, Fm);  extrapolate(d, m, Fn, dir, 0, fijk, Fp);
          extrapolate(d, m, Ne, dir, 1, fijk, Nm);  extrapolate(d, m, Nn, dir, 0, fijk, Np_);
        } else {      /* nb is '-', e is '+' */
          extrapolate(d, m, unb, dir, 1, fijk, um); extrapolate(d, m, uel, dir, 0, fijk, up);
          extrapolate(d, m, Unb, dir, 1, fijk, Um); extrapolate(d, m, Uel, dir, 0, fijk, Up);
          extrapolate(d, m, Fn, dir, 1, fijk, Fm);  extrapolate(d, m, Fe, dir, 0, fijk, Fp);
          extrapolate(d, m, Nn, dir, 1, fijk, Nm);  extrapolate(d, m, Ne, dir, 0, fijk, Np_);
        }
        /* eq. numflux.cons: F^num = (F- + F+)/2 - lambda/2 (U+ - U-) */
        double lm = wave_speed(d, dir, um), lp = wave_speed(d, dir, up);
        double lam = lm > lp ? lm : lp;
        double Fnum[OR_MAXM], ncs[OR_MAXM];
        for (int v = 0; v < M; ++v) Fnum[v] = 0.5 * (Fm[v] + Fp[v]) - 0.5 * lam * (Up[v] - Um[v]);
        if (alpha) {
          /* limited face flux from the '-' and '+' elements' u^n (traces and
           * the neighbouring interior nodes) and their coefficients */
          int emi = side ? e : nb, epl = side ? nb : e;
          const double *unm = &W->un[(size_t)S->loc[emi] * sz], *unp = &W->un[(size_t)S->loc[epl] * sz];
          int im[3] = {fijk[0], fijk[1], fijk[2]}, ip[3] = {fijk[0], fijk[1], fijk[2]};
          im[dir] = d->N - 1;
          ip[dir] = 1;
          double a_f = 0.5 * (alpha[emi] + alpha[epl]);
          double Fl[OR_MAXM];
          limited_face_flux(d, dir, um, up, &unm[node_id(m, im, dim) * M], &unp[node_id(m, ip, dim) * M], Fnum, a_f,
                            dt, m->dx[dir], m->w[d->N], m->w[0], Fl);
          for (int v = 0; v < M; ++v) {
            Fnum[v] = Fl[v];
            Fface[((size_t)(dir * 2 + side) * np + fnode) * M + v] = Fl[v];
          }
        }
        /* F^{num,+-}_nc = B(u^{n,+-}) g^avg(U), or with ncflux 1 (eq. bad.numflux.non.cons)
         * sum_j b_j B(u^{(j),+-}) g^avg(u^(j)) from the stage traces of both sides;
         * then the jump F^num_{+-} - F^tot_{+-} */
        double J[OR_MAXM];
        if (d->ncflux == 1) {
          for (int v = 0; v < M; ++v) ncs[v] = 0.0;
          for (int j = 0; j < m->S; ++j) {
            const double *sel = &W->Us[((size_t)ke * m->S + j) * sz], *snb = &W->Us[((size_t)kn * m->S + j) * sz];
            double sm[OR_MAXM], sp[OR_MAXM], nj[OR_MAXM];
            if (side) { extrapolate(d, m, sel, dir, 1, fijk, sm); extrapolate(d, m, snb, dir, 0, fijk, sp); }
            else      { extrapolate(d, m, snb, dir, 1, fijk, sm); extrapolate(d, m, sel, dir, 0, fijk, sp); }
            nc_with_gavg(d, dir, side ? sm : sp, sm, sp, nj);
            for (int v = 0; v < M; ++v) ncs[v] += m->b[j] * nj[v];
          }
        } else {
          nc_with_gavg(d, dir, side ? um : up, Um, Up, ncs);
        }
        if (side) {
          for (int v = 0; v < M; ++v) J[v] = Fnum[v] + ncs[v] - (Fm[v] + Nm[v]);
        } else {
          for (int v = 0; v < M; ++v) J[v] = Fnum[v] + ncs[v] - (Fp[v] + Np_[v]);
        }
        /* - dt J d_x g_R (side 1) or - dt J d_x g_L (side 0), at every node of the line */
        for (int p = 0; p < m->n; ++p) {
          int ijk[3] = {fijk[0], fijk[1], fijk[2]};
          ijk[dir] = p;
          int id = node_id(m, ijk, dim);
          double dg = (side ? m->dgR[p] : m->dgL[p]) / m->dx[dir];
          for (int v = 0; v < M; ++v) unew[id * M + v] -= dt * J[v] * dg;
        }
      }
    }
  }
  if (alpha) {
    /* low-order update: first-order finite volumes on the subcells of every
     * line, the limited face fluxes at the element faces; then the blend */
    const double *ue = &W->un[ke * sz];
    double *ul = malloc(sizeof(double) * sz);
    for (size_t k = 0; k < sz; ++k) ul[k] = ue[k];
    for (int p = 0; p < np; ++p) {
      int ijk[3];
      node_ijk(m, p, dim, ijk);
      for (int dir = 0; dir < dim; ++dir) {
        int pd = ijk[dir];
        int fi[3] = {ijk[0], ijk[1], ijk[2]};
        fi[dir] = 0;
        int fnode = node_id(m, fi, dim);
        double fL[OR_MAXM], fR[OR_MAXM];
        int q[3] = {ijk[0], ijk[1], ijk[2]};
        if (pd == 0) {
          for (int v = 0; v < M; ++v) fL[v] = Fface[((size_t)(dir * 2 + 0) * np + fnode) * M + v];
        } else {
          q[dir] = pd - 1;
          rusanov_flux(d, dir, &ue[node_id(m, q, dim) * M], &ue[p * M], fL);
        }
        if (pd == d->N) {
          for (int v = 0; v < M; ++v) fR[v] = Fface[((size_t)(dir * 2 + 1) * np + fnode) * M + v];
        } else {
          q[dir] = pd + 1;
          rusanov_flux(d, dir, &ue[p * M], &ue[node_id(m, q, dim) * M], fR);
        }
        for (int v = 0; v < M; ++v) ul[p * M + v] -= dt * (fR[v] - fL[v]) / (m->w[pd] * m->dx[dir]);
      }
    }
    /* a_e = 1 takes u^L alone (u^H may not be finite where the
     * first-order update still is) */
    double a = alpha[e];
    for (size_t k = 0; k < sz; ++k) unew[k] = a >= 1.0 ? ul[k] : (1.0 - a) * unew[k] + a * ul[k];
    free(ul);
    free(Fface);
  }
}

/* validity of the limiter options: Euler, reduced non-conservative flux,
 * 0 <= alpha_max <= 1 */
static int limiter_ok(const or_desc *d) {
  if (!d->limiter) return 1;
  return d->eq == 0 && d->ncflux == 0 && d->alpha_max >= 0.0 && d->alpha_max <= 1.0 && d->alpha_fixed <= 1.0;
}

/* Exported: one cRKFR step u^n -> u^{n+1} with the given dt. */
int or_step(const or_desc *d, const double *Un, double dt, double *Unew) {
  or_mesh m;
  if (mesh_setup(d, &m) || !limiter_ok(d)) return -1;
  int M = m.M, np = m.np, E = m.E;
  size_t sz = (size_t)np * M;
  double *alpha = NULL;
  if (d->limiter) {
    alpha = malloc(sizeof(double) * E);
    or_blend_alpha(d, Un, NULL, alpha);
  }
  or_set S;
  set_alloc(&S, E, E, sz, d->dim, d->ncflux == 1 ? m.S : 0);
  for (int e = 0; e < E; ++e) set_stages(d, &m, Un, dt, &S, e, e);
  for (int e = 0; e < E; ++e) {
    double unew[OR_MAXNP * OR_MAXNP * OR_MAXNP * OR_MAXM];
    set_update(d, &m, &S, e, dt, unew, alpha);
    for (int v = 0; v < M; ++v)
      for (int p = 0; p < np; ++p) Unew[((size_t)v * E + e) * np + p] = unew[p * M + v];
  }
  set_free(&S);
  free(alpha);
  return 0;
}

/* Exported: the same step for nsel selected elements only (for checks of
 * large meshes): the stages of every selected element and of its 2 dim
 * neighbours, then the update of the selected elements.  Unew_sel receives
 * [var][k][node] for sel[k]. */
int or_step_elements(const or_desc *d, const double *Un, double dt, int nsel, const int *sel, double *Unew_sel) {
  or_mesh m;
  if (mesh_setup(d, &m) || !limiter_ok(d)) return -1;
  int M = m.M, np = m.np, E = m.E, dim = d->dim;
  size_t sz = (size_t)np * M;
  for (int k = 0; k < nsel; ++k)
    if (sel[k] < 0 || sel[k] >= E) return -1;
  double *alpha = NULL;
  if (d->limiter) {
    alpha = malloc(sizeof(double) * E);
    or_blend_alpha(d, Un, NULL, alpha);
  }
  or_set S;
  set_alloc(&S, E, nsel * (1 + 2 * dim), sz, dim, d->ncflux == 1 ? m.S : 0);
  int nloc = 0;
  for (int k = 0; k < nsel; ++k) {
    int need[7];
    int nn = 0;
    need[nn++] = sel[k];
    for (int dir = 0; dir < dim; ++dir) {
      need[nn++] = neighbour(d, sel[k], dir, +1);
      need[nn++] = neighbour(d, sel[k], dir, -1);
    }
    for (int j = 0; j < nn; ++j)
      if (S.loc[need[j]] < 0) { set_stages(d, &m, Un, dt, &S, need[j], nloc); ++nloc; }
  }
  for (int k = 0; k < nsel; ++k) {
    double unew[OR_MAXNP * OR_MAXNP * OR_MAXNP * OR_MAXM];
    set_update(d, &m, &S, sel[k], dt, unew, alpha);
    for (int v = 0; v < M; ++v)
      for (int p = 0; p < np; ++p) Unew_sel[((size_t)v * nsel + k) * np + p] = unew[p * M + v];
  }
  set_free(&S);
  free(alpha);
  return 0;
}

/* Exported: the time-averaged data of one element (for pins of the stage
 * structure): Rbar, Ubar, Fbar[dim], Fnc[dim], each [node][var]. */
int or_element_stages(const or_desc *d, const double *une, double dt, double *Rbar, double *Ubar, double *Fbar, double *Fnc) {
  or_mesh m;
  if (mesh_setup(d, &m)) return -1;
  element_stages(d, &m, une, dt, Rbar, Ubar, Fbar, Fnc, NULL);
  return 0;
}

/* Exported: local residual R(u) of one element ([node][var]), for pins. */
int or_local_residual(const or_desc *d, const double *ue, double *R) {
  or_mesh m;
  if (mesh_setup(d, &m)) return -1;
  local_residual(d, &m, ue, R);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Semi-discrete standard FR right-hand side (eq. general.non.conservative.fr.one
 * in flux-differencing form), used only to pin the volume fluxes: with an EC
 * surface flux (d->surf == 1) it conserves the total entropy exactly.        */
/* ------------------------------------------------------------------------- */
int or_fr_rhs(const or_desc *d, const double *Un, double *RHS) {
  or_mesh m;
  if (mesh_setup(d, &m)) return -1;
  int M = m.M, np = m.np, E = m.E, dim = d->dim;
  size_t sz = (size_t)np * M;
  double *un = malloc(sizeof(double) * sz * E);
  for (int e = 0; e < E; ++e) gather_elem(&m, Un, e, &un[e * sz]);
  for (int e = 0; e < E; ++e) {
    double R[OR_MAXNP * OR_MAXNP * OR_MAXNP * OR_MAXM];
    local_residual(d, &m, &un[e * sz], R);
    for (size_t k = 0; k < sz; ++k) R[k] = -R[k];
    for (int dir = 0; dir < dim; ++dir)
      for (int side = 0; side < 2; ++side) {
        int nb = neighbour(d, e, dir, side ? +1 : -1);
        for (int fnode = 0; fnode < np; ++fnode) {
          int fijk[3];
          node_ijk(&m, fnode, dim, fijk);
          if (fijk[dir] != 0) continue;
          double um[OR_MAXM], up[OR_MAXM];
          if (side) { extrapolate(d, &m, &un[e * sz], dir, 1, fijk, um); extrapolate(d, &m, &un[nb * sz], dir, 0, fijk, up); }
          else      { extrapolate(d, &m, &un[nb * sz], dir, 1, fijk, um); extrapolate(d, &m, &un[e * sz], dir, 0, fijk, up); }
          double Fnum[OR_MAXM], fm[OR_MAXM], fp[OR_MAXM], nm[OR_MAXM], npl[OR_MAXM], ncs[OR_MAXM], J[OR_MAXM];
          phys_flux(d, dir, um, fm); phys_flux(d, dir, up, fp);
          nc_product(d, dir, um, um, nm); nc_product(d, dir, up, up, npl);
          if (d->surf == 1) {
            two_point_flux(d, dir, um, up, Fnum);
          } else {
            double lm = wave_speed(d, dir, um), lp = wave_speed(d, dir, up);
            double lam = lm > lp ? lm : lp;
            for (int v = 0; v < M; ++v) Fnum[v] = 0.5 * (fm[v] + fp[v]) - 0.5 * lam * (up[v] - um[v]);
          }
          if (side) { nc_with_gavg(d, dir, um, um, up, ncs); for (int v = 0; v < M; ++v) J[v] = Fnum[v] + ncs[v] - (fm[v] + nm[v]); }
          else      { nc_with_gavg(d, dir, up, um, up, ncs); for (int v = 0; v < M; ++v) J[v] = Fnum[v] + ncs[v] - (fp[v] + npl[v]); }
          for (int p = 0; p < m.n; ++p) {
            int ijk[3] = {fijk[0], fijk[1], fijk[2]};
            ijk[dir] = p;
            int id = node_id(&m, ijk, dim);
            double dg = (side ? m.dgR[p] : m.dgL[p]) / m.dx[dir];
            for (int v = 0; v < M; ++v) R[id * M + v] -= J[v] * dg;
          }
        }
      }
    for (int v = 0; v < M; ++v)
      for (int p = 0; p < np; ++p) RHS[((size_t)v * E + e) * np + p] = R[p * M + v];
  }
  free(un);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Multi-stage RKFR step (eqs. rkfr1, rkfr2): the degree's explicit RK method
 * (or_butcher) applied to the semi-discrete FR system (eq.
 * general.non.conservative.fr.one) with the Rusanov surface flux.  With
 * L(u) = -(local derivative + face corrections) = or_fr_rhs(u):
 *   u^(i)   = u^n + dt sum_{j<i} a_ij L(u^(j)),  i = 1..s,
 *   u^{n+1} = u^n + dt sum_j   b_j  L(u^(j)).
 * Every stage evaluates the numerical fluxes of its own face traces u^(j,+-)
 * (s inter-element exchanges per step, against one for cRKFR).              */
/* ------------------------------------------------------------------------- */
int or_rkfr_step(const or_desc *d, const double *Un, double dt, double *Unew) {
  or_mesh m;
  if (d->surf != 0 || d->limiter || mesh_setup(d, &m)) return -1;
  size_t tot = (size_t)m.M * m.E * m.np;
  double *K = malloc(sizeof(double) * tot * m.S);
  double *us = malloc(sizeof(double) * tot);
  int rc = 0;
  for (int i = 0; i < m.S && rc == 0; ++i) {
    for (size_t k = 0; k < tot; ++k) {
      double acc = 0.0;
      for (int j = 0; j < i; ++j) acc += m.A[i][j] * K[j * tot + k];
      us[k] = Un[k] + dt * acc;
    }
    rc = or_fr_rhs(d, us, &K[i * tot]);
  }
  if (rc == 0)
    for (size_t k = 0; k < tot; ++k) {
      double acc = 0.0;
      for (int j = 0; j < m.S; ++j) acc += m.b[j] * K[j * tot + k];
      Unew[k] = Un[k] + dt * acc;
    }
  free(K);
  free(us);
  return rc;
}

/* ------------------------------------------------------------------------- */
/* Diagnostics: quadrature-weighted domain totals of every conserved variable,
 * kinetic energy and entropy S = -rho s/(gamma-1), s = ln p - gamma ln rho.  */
/* ------------------------------------------------------------------------- */
int or_totals(const or_desc *d, const double *U, double *tot /* [M+2] */) {
  or_mesh m;
  if (mesh_setup(d, &m)) return -1;
  int M = m.M;
  double vol = 1.0;
  for (int k = 0; k < d->dim; ++k) vol *= m.dx[k];
  for (int v = 0; v < M + 2; ++v) tot[v] = 0.0;
  double ue[OR_MAXNP * OR_MAXNP * OR_MAXNP * OR_MAXM];
  for (int e = 0; e < m.E; ++e) {
    gather_elem(&m, U, e, ue);
    for (int p = 0; p < m.np; ++p) {
      int ijk[3];
      node_ijk(&m, p, d->dim, ijk);
      double wq = vol;
      for (int k = 0; k < d->dim; ++k) wq *= m.w[ijk[k]];
      const double *u = &ue[p * M];
      for (int v = 0; v < M; ++v) tot[v] += wq * u[v];
      double rho, vel[3] = {0, 0, 0}, pr, B[3], psi;
      if (d->eq == 0) euler_prim(d, u, &rho, vel, &pr); else mhd_prim(d, u, &rho, vel, &pr, B, &psi);
      double ke = 0.5 * rho * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]);
      double s = log(pr) - d->gamma * log(rho);
      tot[M] += wq * ke;
      tot[M + 1] += wq * (-rho * s / (d->gamma - 1.0));
    }
  }
  return 0;
}
