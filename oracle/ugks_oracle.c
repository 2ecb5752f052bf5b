/*
 * ugks_oracle.c -- plain FP64 CPU oracle of one UGKS time step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA path is checked against.  It shares no code, header, table or helper
 * with the CUDA library; only tests/, the package's smoke() check and the
 * CPU-baseline leg of bench.py may load it.  The product path never calls it.
 *
 * It follows the paper (arXiv 2606.15720, "A GPGPU-Oriented Full Phase-Space
 * Parallel UGKS with Velocity-Block Pipelining") Sec. 2.1 and Algorithm 5 step
 * by step, with every velocity loop written out over all k (B_v = N_v) unless
 * a blocked summation order is requested (Sec. 2.2.6, Eq. 63-64), and no
 * fusion.  Where the paper is silent the following readings are used (they
 * bind the CUDA path too):
 *   R1 limiter: Venkatakrishnan with eps^2 = (K_v h)^3 m^2, h = |Omega|^(1/D),
 *      m = the largest |value| over the cell and its stencil (the limited
 *      quantity's own scale; f spans many decades, so an absolute eps never
 *      limits it), phi clipped to [0,1]; per cell, per velocity, per reduced
 *      function; also per component of W for the macroscopic reconstruction.
 *   R2 gradient: unweighted least squares over face neighbours, M^-1 sum d df.
 *   R3 stencil: far-field / outflow ghosts included (ghost centroid mirrored
 *      across the face, ghost distribution = Maxwellian of the ghost state);
 *      a wall contributes a mirrored ghost that carries the cell's own value
 *      (zero gradient): its offset enters the least-squares matrix, nothing
 *      enters the right-hand side or the limiter's max/min; the wall face is
 *      one of the faces the limiter checks.  (With walls left out of the
 *      matrix, wall cells with two interior neighbours extrapolate: some
 *      outflow face values then weigh the cell's own value negatively, the
 *      transport of that velocity amplifies instead of damping, and the
 *      limiter alone bounds it, so steady states depended on the start.)
 *   R4 time step: dt = CFL min_i |Omega_i| / max_k sum_f S_f max(u_k.n_f, 0).
 *   R5 tau = mu/p with mu = mu_ref T^omega.
 *   R6 W0 = half-range moments of the two reconstructed Maxwellians.
 *   R7 q0 = (q_l + q_r)/2, ghost q = 0.
 *   R8 grad W0 = (phi grad W_l + phi grad W_r)/2, ghost gradient = 0.
 *   R9 wall free transport is f(x - u t): integral = dt f_in - dt^2/2 u.grad f.
 *   R11 optional tau0 += dt |p_l - p_r| / (p_l + p_r).
 *   R12 stage 2 uses the lagged heat flux q^n.
 *   R13 residual R_m = sqrt(mean_i (dW_im)^2).
 *   R17/18 stage 1 uses q^n; the initial f is the discrete Maxwellian.
 *   R20 surface quantities of a wall face from the moments F of its
 *      time-integrated flux (n out of the gas, P = F_momentum / dt):
 *      p_w = P.n, tau_w = P - p_w n, q_w = (F_energy - U_w.F_momentum) / dt;
 *      coefficients against a free stream (rho, U, T): C_p = (p_w - rho T/2)
 *      / (rho|U|^2/2), C_t = |tau_w| / (rho|U|^2/2), C_h = q_w / (rho|U|^3/2).
 *   R21 thirteen-moment fields of a cell: rho, U, T = 1/lambda of W, the
 *      deviatoric stress sigma_ij = sum_k w c_i c_j h - p delta_ij (p = rho /
 *      (2 lambda)) and q (Eq. 13), c = u - U of W; their Chapman-Enskog
 *      (Grad 13-moment) distribution, reduced over xi:
 *        h = H [1 + 2 lam^2/rho sigma_ij c_i c_j - lam tr(sigma)/rho
 *               + 4 lam^2/((K+5) rho) (q.c)(2 lam c^2 - (D+2))]
 *        b = kappa H [1 + 2 lam^2/rho sigma_ij c_i c_j - lam (K_xi+2) tr(sigma)/(K_xi rho)
 *               + 4 lam^2/((K+5) rho) (q.c)(2 lam c^2 - D)]
 *      (K + 5 = N + 2 for N = D + K_xi degrees of freedom; at K = 0 the
 *      heat-flux term has the form of the Shakhov term of Eq. 18-19).  The
 *      trace terms: the full stress over all D + K_xi degrees of freedom is
 *      trace-free, so the K_xi components of xi share -tr(sigma) equally
 *      (for D = 2, K = 0 this is sigma_zz = -(sigma_xx + sigma_yy)); reducing
 *      that xi-stress term over xi gives the two constants, with which the
 *      moments of (h, b) return rho, E and sigma for any in-plane trace.
 *      At K_xi = 0 sigma must be trace-free.
 * Parity: every function below is pinned by tests/test_oracle_pins.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXD 3
#define NW 5 /* at most D + 2 conservative variables */
#define MAXF 32 /* at most this many faces per cell */

typedef struct {
  int32_t type; /* 1 wall, 2 far field, 3 outflow */
  double rho, u[3], T;
} orc_bc;

typedef struct {
  int32_t dim;
  int64_t n_cells, n_faces;
  const double *vol, *xc;           /* [Nc], [Nc][dim] */
  const int64_t *own, *nei;         /* [Nf] */
  const double *area, *nrm, *xf;    /* [Nf], [Nf][dim], [Nf][dim] */
  const double *shift;              /* [Nf][dim] */
  int32_t n_bc;
  const orc_bc *bc;
} orc_mesh;

typedef struct {
  int32_t K;            /* internal degrees of freedom */
  int32_t model;        /* 0 BGK, 1 Shakhov */
  double Pr, omega, mu_ref;
  double cfl, dt_override;
  int32_t limiter;      /* 0 none, 1 Venkatakrishnan, 2 Barth-Jespersen */
  double venkat_K;
  int32_t shock_tau_fix;
  int32_t block_v, p_v; /* velocity summation order (Eq. 63-64); 0 = plain */
} orc_params;

/* ------------------------------------------------------------------------ */
/* Primitive variables, Maxwellian, Shakhov correction (Sec. 2.1)            */
/* ------------------------------------------------------------------------ */

typedef struct { double rho, U[MAXD], lam; } prim_t;

/* lambda = (K+3) rho / (4 (rho E - rho |U|^2 / 2)): rho E carries (K+3)/2 RT per
 * unit mass with R = 1/2, lambda = 1/(2RT) (Eq. 6, 10).  Returns 0 if invalid. */
static int prim_from_W(int D, int K, const double *W, prim_t *p) {
  p->rho = W[0];
  if (!(p->rho > 0.0)) return 0;
  double u2 = 0.0;
  for (int d = 0; d < D; ++d) { p->U[d] = W[1 + d] / W[0]; u2 += p->U[d] * p->U[d]; }
  double ein = W[D + 1] - 0.5 * W[0] * u2;
  if (!(ein > 0.0)) return 0;
  p->lam = (K + 3) * W[0] / (4.0 * ein);
  return 1;
}

static void W_from_prim(int D, int K, const prim_t *p, double *W) {
  W[0] = p->rho;
  double u2 = 0.0;
  for (int d = 0; d < D; ++d) { W[1 + d] = p->rho * p->U[d]; u2 += p->U[d] * p->U[d]; }
  W[D + 1] = 0.5 * p->rho * u2 + (K + 3) * p->rho / (4.0 * p->lam);
}

/* Reduced Maxwellian H (Eq. 16) and B = K_xi/(2 lambda) H (Eq. 17). */
static double maxwell_H(int D, const prim_t *p, const double *u) {
  double c2 = 0.0;
  for (int d = 0; d < D; ++d) { double c = u[d] - p->U[d]; c2 += c * c; }
  return p->rho * pow(p->lam / M_PI, 0.5 * D) * exp(-p->lam * c2);
}

/* Reduced Shakhov corrections H+ (Eq. 18) and B+ (Eq. 19), K = 0. */
static void shakhov_plus(int D, int Kxi, double Pr, const prim_t *p, const double *q,
                         const double *u, double H, double *Hp, double *Bp) {
  double c2 = 0.0, cq = 0.0;
  for (int d = 0; d < D; ++d) { double c = u[d] - p->U[d]; c2 += c * c; cq += c * q[d]; }
  double pref = 4.0 * (1.0 - Pr) * p->lam * p->lam / (5.0 * p->rho) * cq;
  *Hp = pref * (2.0 * p->lam * c2 - 2.0 - D) * H;
  *Bp = pref * ((2.0 * p->lam * c2 - D) * Kxi) / (2.0 * p->lam) * H;
}

/* Reduced equilibrium h+ = H + H+, b+ = B + B+ (Eq. 15). */
static void equilibrium_hb(int D, int Kxi, int shakhov, double Pr, const prim_t *p,
                           const double *q, const double *u, double *hp, double *bp) {
  double H = maxwell_H(D, p, u);
  double B = Kxi / (2.0 * p->lam) * H;
  double Hs = 0.0, Bs = 0.0;
  if (shakhov) shakhov_plus(D, Kxi, Pr, p, q, u, H, &Hs, &Bs);
  *hp = H + Hs;
  *bp = B + Bs;
}

/* ------------------------------------------------------------------------ */
/* Time-integration coefficients: integrals over [0, dt] of c1..c5 (Eq. 34-35) */
/* ------------------------------------------------------------------------ */

/* G[0] = int c1, G[1] = int c2, G[2] = int c3, G[3] = int c4, G[4] = int c5.
 * Closed forms with expm1 for x = dt/tau >= 0.5; power series below. */
void orc_time_coefficients(double dt, double tau, double *G) {
  double x = dt / tau;
  if (x >= 0.5) {
    double em = -expm1(-x); /* 1 - E */
    double E = exp(-x);
    G[0] = tau * em;
    G[1] = tau * (dt * E - tau * em);
    G[2] = dt - tau * em;
    G[3] = tau * (2.0 * tau * em - dt * (1.0 + E));
    G[4] = 0.5 * dt * dt - tau * dt + tau * tau * em;
    return;
  }
  /* series in x:  G0/dt = sum_n (-x)^n/(n+1)!,  G2 = dt - G0,
   * G1/dt^2 = sum_m (-1)^(m+1) (m+1)/(m+2)! x^m,
   * G3/dt^2 = sum_j>=1 (-1)^j j x^j/(j+2)!,  G4/dt^2 = sum_j>=1 (-1)^(j+1) x^j/(j+2)! */
  double s0 = 0.0, s2 = 0.0, s1 = 0.0, s3 = 0.0, s4 = 0.0;
  double xp = 1.0;      /* x^n */
  double fact1 = 1.0;   /* (n+1)! */
  double fact2 = 2.0;   /* (n+2)! */
  for (int n = 0; n < 40; ++n) {
    double sg = (n % 2 == 0) ? 1.0 : -1.0; /* (-1)^n */
    s0 += sg * xp / fact1;
    if (n >= 1) s2 += -sg * xp / fact1;
    s1 += -sg * (n + 1) * xp / fact2;
    if (n >= 1) {
      s3 += sg * n * xp / fact2;
      s4 += -sg * xp / fact2;
    }
    xp *= x;
    fact1 *= (n + 2);
    fact2 *= (n + 3);
  }
  G[0] = dt * s0;
  G[2] = dt * s2;
  G[1] = dt * dt * s1;
  G[3] = dt * dt * s3;
  G[4] = dt * dt * s4;
}

/* ------------------------------------------------------------------------ */
/* Gaussian moments via polynomials in (u_1..u_D, s = xi^2)                   */
/* ------------------------------------------------------------------------ */

#define PMAX 256
typedef struct { int n; double c[PMAX]; int e[PMAX][MAXD + 1]; } poly_t;

static void poly_zero(poly_t *p) { p->n = 0; }
static void poly_add_term(poly_t *p, double c, const int *e) {
  for (int i = 0; i < p->n; ++i) {
    if (memcmp(p->e[i], e, sizeof(int) * (MAXD + 1)) == 0) { p->c[i] += c; return; }
  }
  p->c[p->n] = c;
  memcpy(p->e[p->n], e, sizeof(int) * (MAXD + 1));
  p->n++;
}
static void poly_mul(const poly_t *a, const poly_t *b, poly_t *out) {
  poly_zero(out);
  for (int i = 0; i < a->n; ++i)
    for (int j = 0; j < b->n; ++j) {
      int e[MAXD + 1];
      for (int t = 0; t <= MAXD; ++t) e[t] = a->e[i][t] + b->e[j][t];
      poly_add_term(out, a->c[i] * b->c[j], e);
    }
}
/* collision invariant psi_alpha (Eq. 8) as a polynomial */
static void poly_psi(int D, int alpha, poly_t *p) {
  int e[MAXD + 1] = {0, 0, 0, 0};
  poly_zero(p);
  if (alpha == 0) { poly_add_term(p, 1.0, e); return; }
  if (alpha <= D) { e[alpha - 1] = 1; poly_add_term(p, 1.0, e); return; }
  for (int d = 0; d < D; ++d) { int f[MAXD + 1] = {0, 0, 0, 0}; f[d] = 2; poly_add_term(p, 0.5, f); }
  e[MAXD] = 1;
  poly_add_term(p, 0.5, e);
}
/* <u^n> of the 1-D Gaussian N(U, 1/(2 lambda)) */
static double gauss_moment1(double U, double lam, int n) {
  double m0 = 1.0, m1 = U;
  if (n == 0) return m0;
  for (int k = 1; k < n; ++k) { double m2 = U * m1 + k / (2.0 * lam) * m0; m0 = m1; m1 = m2; }
  return m1;
}
/* <(xi^2)^e> of the K_xi-dimensional isotropic Gaussian, variance 1/(2 lambda) */
static double xi_moment(int Kxi, double lam, int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= (Kxi + 2.0 * i) / (2.0 * lam);
  return r;
}
static double poly_expect(int D, int Kxi, const prim_t *pr, const poly_t *p) {
  double s = 0.0;
  for (int i = 0; i < p->n; ++i) {
    double t = p->c[i];
    for (int d = 0; d < D; ++d) t *= gauss_moment1(pr->U[d], pr->lam, p->e[i][d]);
    t *= xi_moment(Kxi, pr->lam, p->e[i][MAXD]);
    s += t;
  }
  return s;
}

/* Dense solve by Gaussian elimination with partial pivoting (n <= 5). */
static int solve_dense(int n, double *A, double *b, double *x) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r) if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return 0;
    if (piv != c) {
      for (int t = 0; t < n; ++t) { double tmp = A[c * n + t]; A[c * n + t] = A[piv * n + t]; A[piv * n + t] = tmp; }
      double tmp = b[c]; b[c] = b[piv]; b[piv] = tmp;
    }
    for (int r = c + 1; r < n; ++r) {
      double f = A[r * n + c] / A[c * n + c];
      for (int t = c; t < n; ++t) A[r * n + t] -= f * A[c * n + t];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int t = r + 1; t < n; ++t) s -= A[r * n + t] * x[t];
    x[r] = s / A[r * n + r];
  }
  return 1;
}


/* Inverse of the least-squares matrix M = sum d d^T (reading R2).  M is
 * treated as singular (zero gradient) when det M <= 1e-12 (tr M / D)^D. */
static int lsq_inverse(int D, const double *M, double *Minv) {
  double det, tr = 0.0;
  for (int d = 0; d < D; ++d) tr += M[d * D + d];
  tr /= D;
  if (D == 1) {
    det = M[0];
    if (!(det > 1e-12 * tr) || !(tr > 0.0)) return 0;
    Minv[0] = 1.0 / det;
    return 1;
  }
  if (D == 2) {
    det = M[0] * M[3] - M[1] * M[2];
    if (!(tr > 0.0) || !(det > 1e-12 * tr * tr)) return 0;
    Minv[0] = M[3] / det; Minv[1] = -M[1] / det; Minv[2] = -M[2] / det; Minv[3] = M[0] / det;
    return 1;
  }
  double c00 = M[4] * M[8] - M[5] * M[7], c01 = M[5] * M[6] - M[3] * M[8], c02 = M[3] * M[7] - M[4] * M[6];
  det = M[0] * c00 + M[1] * c01 + M[2] * c02;
  if (!(tr > 0.0) || !(det > 1e-12 * tr * tr * tr)) return 0;
  Minv[0] = c00 / det;
  Minv[1] = (M[2] * M[7] - M[1] * M[8]) / det;
  Minv[2] = (M[1] * M[5] - M[2] * M[4]) / det;
  Minv[3] = c01 / det;
  Minv[4] = (M[0] * M[8] - M[2] * M[6]) / det;
  Minv[5] = (M[2] * M[3] - M[0] * M[5]) / det;
  Minv[6] = c02 / det;
  Minv[7] = (M[1] * M[6] - M[0] * M[7]) / det;
  Minv[8] = (M[0] * M[4] - M[1] * M[3]) / det;
  return 1;
}

/* Spatial slope of the interface Maxwellian: grad g0 = g0 (a . psi), so
 * rho0 <psi psi^T> a = dW0 for each direction (Eq. 32). */
void orc_micro_slope(int D, int K, const double *W0, const double *dW, double *a) {
  prim_t p;
  int nw = D + 2, Kxi = K + 3 - D;
  prim_from_W(D, K, W0, &p);
  double M[NW * NW], rhs[NW];
  poly_t pa, pb, pab;
  for (int al = 0; al < nw; ++al) {
    poly_psi(D, al, &pa);
    for (int be = 0; be < nw; ++be) {
      poly_psi(D, be, &pb);
      poly_mul(&pa, &pb, &pab);
      M[al * nw + be] = p.rho * poly_expect(D, Kxi, &p, &pab);
    }
    rhs[al] = dW[al];
  }
  if (!solve_dense(nw, M, rhs, a)) for (int t = 0; t < nw; ++t) a[t] = 0.0;
}

/* Time slope A from compatibility: int psi (u . grad g0 + d_t g0) = 0, i.e.
 * rho0 <psi psi^T> A = -sum_d rho0 <psi u_d (a_d . psi)> (Eq. 32, Eq. 7). */
void orc_time_slope(int D, int K, const double *W0, const double *a /*[D][nw]*/, double *A) {
  prim_t p;
  int nw = D + 2, Kxi = K + 3 - D;
  prim_from_W(D, K, W0, &p);
  double M[NW * NW], rhs[NW];
  poly_t pa, pb, pab, tmp, ad, ud;
  for (int al = 0; al < nw; ++al) {
    poly_psi(D, al, &pa);
    for (int be = 0; be < nw; ++be) {
      poly_psi(D, be, &pb);
      poly_mul(&pa, &pb, &pab);
      M[al * nw + be] = p.rho * poly_expect(D, Kxi, &p, &pab);
    }
    double r = 0.0;
    for (int d = 0; d < D; ++d) {
      /* a_d . psi */
      poly_zero(&ad);
      for (int be = 0; be < nw; ++be) {
        poly_psi(D, be, &pb);
        for (int i = 0; i < pb.n; ++i) poly_add_term(&ad, a[d * nw + be] * pb.c[i], pb.e[i]);
      }
      int e[MAXD + 1] = {0, 0, 0, 0};
      e[d] = 1;
      poly_zero(&ud);
      poly_add_term(&ud, 1.0, e);
      poly_mul(&ud, &ad, &tmp);
      poly_mul(&pa, &tmp, &pab);
      r -= p.rho * poly_expect(D, Kxi, &p, &pab);
    }
    rhs[al] = r;
  }
  if (!solve_dense(nw, M, rhs, A)) for (int t = 0; t < nw; ++t) A[t] = 0.0;
}

/* rho <psi> over the half space sign * (u . n) > 0 (reading R6). */
static void half_moments(int D, int K, const prim_t *p, const double *n, int sign, double *out) {
  int Kxi = K + 3 - D;
  double Un = 0.0;
  for (int d = 0; d < D; ++d) Un += p->U[d] * n[d];
  double sl = sqrt(p->lam);
  double ex = exp(-p->lam * Un * Un) / (2.0 * sqrt(M_PI * p->lam));
  double a0, a1;
  if (sign > 0) { a0 = 0.5 * erfc(-sl * Un); a1 = Un * a0 + ex; }
  else          { a0 = 0.5 * erfc(sl * Un);  a1 = Un * a0 - ex; }
  double a2 = Un * a1 + a0 / (2.0 * p->lam);
  double Ut2 = 0.0;
  out[0] = p->rho * a0;
  for (int d = 0; d < D; ++d) {
    double Ut = p->U[d] - Un * n[d];
    Ut2 += Ut * Ut;
    out[1 + d] = p->rho * (a1 * n[d] + a0 * Ut);
  }
  out[D + 1] = 0.5 * p->rho * (a2 + a0 * (Ut2 + (D - 1 + Kxi) / (2.0 * p->lam)));
}

void orc_interface_W0(int D, int K, const double *Wl, const double *Wr, const double *n, double *W0) {
  prim_t pl, pr;
  prim_from_W(D, K, Wl, &pl);
  prim_from_W(D, K, Wr, &pr);
  double a[NW], b[NW];
  half_moments(D, K, &pl, n, +1, a);
  half_moments(D, K, &pr, n, -1, b);
  for (int t = 0; t < D + 2; ++t) W0[t] = a[t] + b[t];
}

/* ------------------------------------------------------------------------ */
/* Limiters (reading R1)                                                      */
/* ------------------------------------------------------------------------ */

static double limiter_phi(int kind, double d2, double dmax, double dmin, double eps2) {
  if (kind == 0) return 1.0;
  if (d2 == 0.0) return 1.0;
  double dp = d2 > 0.0 ? dmax : dmin;
  if (kind == 2) {
    double r = dp / d2;
    return r < 1.0 ? r : 1.0;
  }
  double num = dp * dp + eps2 + 2.0 * d2 * dp;
  double den = dp * dp + 2.0 * d2 * d2 + dp * d2 + eps2;
  if (den == 0.0) return 1.0;
  return num / den;
}

/* The limiter of one face increment d2 of a cell whose stencil spans
 * [dmin, dmax] around the cell value, exported for the pin tests. */
double orc_limiter_phi(int kind, double d2, double dmax, double dmin, double eps2) {
  return limiter_phi(kind, d2, dmax, dmin, eps2);
}

/* ------------------------------------------------------------------------ */
/* Blocked velocity summation (Sec. 2.2.2, Eq. 48-49; Sec. 2.2.6, Eq. 63-64)   */
/* ------------------------------------------------------------------------ */

static double vsum(const double *x, int64_t nv, int32_t bv, int32_t pv) {
  if (bv <= 0 || bv >= nv) {
    double s = 0.0;
    for (int64_t k = 0; k < nv; ++k) s += x[k];
    if (pv <= 1) return s;
  }
  if (bv <= 0) bv = (int32_t)nv;
  if (pv <= 0) pv = 1;
  int64_t M = (nv + bv - 1) / bv; /* padded velocities carry omega = 0 */
  double total = 0.0;
  int64_t m = 0;
  for (int32_t q = 0; q < pv; ++q) {
    int64_t Mq = M / pv + (q < M % pv ? 1 : 0);
    double part = 0.0;
    for (int64_t j = 0; j < Mq; ++j, ++m) {
      double blk = 0.0;
      for (int64_t k = m * bv; k < (m + 1) * bv; ++k) blk += (k < nv) ? x[k] : 0.0;
      part += blk;
    }
    total += part;
  }
  return total;
}

/* ------------------------------------------------------------------------ */
/* Mesh helpers                                                               */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t *off, *face; /* CSR: faces of each cell */
} adj_t;

static void build_adj(const orc_mesh *m, adj_t *a) {
  int64_t Nc = m->n_cells, Nf = m->n_faces;
  a->off = (int64_t *)calloc(Nc + 1, sizeof(int64_t));
  a->face = (int64_t *)malloc(sizeof(int64_t) * 2 * Nf + 1);
  for (int64_t f = 0; f < Nf; ++f) {
    a->off[m->own[f] + 1]++;
    if (m->nei[f] >= 0) a->off[m->nei[f] + 1]++;
  }
  for (int64_t i = 0; i < Nc; ++i) a->off[i + 1] += a->off[i];
  int64_t *fill = (int64_t *)calloc(Nc, sizeof(int64_t));
  for (int64_t f = 0; f < Nf; ++f) {
    int64_t o = m->own[f];
    a->face[a->off[o] + fill[o]++] = f;
    if (m->nei[f] >= 0) { int64_t j = m->nei[f]; a->face[a->off[j] + fill[j]++] = f; }
  }
  free(fill);
}

/* Geometry of face f seen from cell c: outward normal, face centroid in c's
 * frame, and the neighbour (or ghost) centroid.  Returns the neighbour index,
 * or -(bc+1) for a boundary face. */
static int64_t face_view(const orc_mesh *m, int64_t f, int64_t c, double *nout, double *xfc, double *xo) {
  int D = m->dim;
  const double *n = m->nrm + f * D, *xf = m->xf + f * D, *sh = m->shift + f * D;
  const double *xcc = m->xc + c * D;
  if (m->own[f] == c) {
    for (int d = 0; d < D; ++d) { nout[d] = n[d]; xfc[d] = xf[d]; }
    int64_t j = m->nei[f];
    if (j >= 0) {
      for (int d = 0; d < D; ++d) xo[d] = m->xc[j * D + d] + sh[d];
    } else {
      double dn = 0.0;
      for (int d = 0; d < D; ++d) dn += (xf[d] - xcc[d]) * n[d];
      for (int d = 0; d < D; ++d) xo[d] = xcc[d] + 2.0 * dn * n[d];
    }
    return j;
  }
  for (int d = 0; d < D; ++d) { nout[d] = -n[d]; xfc[d] = xf[d] - sh[d]; xo[d] = m->xc[m->own[f] * D + d] - sh[d]; }
  return m->own[f];
}

static double mu_of_T(const orc_params *p, double T) { return p->mu_ref * pow(T, p->omega); }
static double tau_of(const orc_params *p, const prim_t *pr) {
  double T = 1.0 / pr->lam, pres = pr->rho / (2.0 * pr->lam);
  return mu_of_T(p, T) / pres;
}

/* Time step (reading R4), padded / zero-weight velocities excluded. */
double orc_time_step(const orc_mesh *m, int64_t nv, const double *u, const double *w, double cfl) {
  adj_t a;
  build_adj(m, &a);
  int D = m->dim;
  double best = INFINITY;
  for (int64_t i = 0; i < m->n_cells; ++i) {
    double worst = 0.0;
    for (int64_t k = 0; k < nv; ++k) {
      if (w[k] == 0.0) continue;
      double s = 0.0;
      for (int64_t t = a.off[i]; t < a.off[i + 1]; ++t) {
        int64_t f = a.face[t];
        double nout[MAXD], xfc[MAXD], xo[MAXD];
        face_view(m, f, i, nout, xfc, xo);
        double un = 0.0;
        for (int d = 0; d < D; ++d) un += u[k * D + d] * nout[d];
        if (un > 0.0) s += m->area[f] * un;
      }
      if (s > worst) worst = s;
    }
    if (worst > 0.0 && m->vol[i] / worst < best) best = m->vol[i] / worst;
  }
  free(a.off);
  free(a.face);
  return cfl * best;
}

/* Heat flux q = 1/2 sum_k omega_k c_k (|c_k|^2 h_k + b_k), Eq. 13. */
static void heat_flux(int D, int64_t nv, const double *u, const double *w, const double *h,
                      const double *b, const double *U, const orc_params *p, double *q, double *scratch) {
  for (int d = 0; d < D; ++d) {
    for (int64_t k = 0; k < nv; ++k) {
      double c2 = 0.0;
      for (int e = 0; e < D; ++e) { double c = u[k * D + e] - U[e]; c2 += c * c; }
      double c = u[k * D + d] - U[d];
      scratch[k] = 0.5 * w[k] * c * (c2 * h[k] + (b ? b[k] : 0.0));
    }
    q[d] = vsum(scratch, nv, p->block_v, p->p_v);
  }
}

void orc_heat_flux(int D, int K, int64_t nv, const double *u, const double *w, const double *h,
                   const double *b, const double *W, double *q) {
  prim_t pr;
  prim_from_W(D, K, W, &pr);
  orc_params p;
  memset(&p, 0, sizeof(p));
  double *s = (double *)malloc(sizeof(double) * nv);
  heat_flux(D, nv, u, w, h, b, pr.U, &p, q, s);
  free(s);
}

/* Reduced equilibria at one velocity, for the pins. out = {H, B, H+, B+}. */
void orc_reduced_equilibrium(int D, int K, double Pr, const double *prim /*rho,U,lam*/, const double *q,
                             const double *u, double *out) {
  prim_t p;
  p.rho = prim[0];
  for (int d = 0; d < D; ++d) p.U[d] = prim[1 + d];
  p.lam = prim[D + 1];
  int Kxi = K + 3 - D;
  double H = maxwell_H(D, &p, u);
  out[0] = H;
  out[1] = Kxi / (2.0 * p.lam) * H;
  shakhov_plus(D, Kxi, Pr, &p, q, u, H, &out[2], &out[3]);
}

/* Thirteen-moment fields of every cell (reading R21): out[cell] = (rho,
 * U[D], T, sigma[D(D+1)/2] in the order xx, xy, (xz), yy, (yz), zz, q[D]). */
void orc_moments13(int D, int K, int64_t nc, int64_t nv, const double *u, const double *w, const double *W,
                   const double *f, double *out) {
  const int Kxi = K + 3 - D, nr = Kxi > 0 ? 2 : 1, ns = D * (D + 1) / 2, n13 = 2 * D + 2 + ns;
  for (int64_t i = 0; i < nc; ++i) {
    prim_t p;
    prim_from_W(D, K, W + i * (D + 2), &p);
    const double *h = f + i * nv, *b = nr == 2 ? f + (nc + i) * nv : NULL;
    double P[MAXD][MAXD], q[MAXD];
    for (int a = 0; a < D; ++a) {
      q[a] = 0.0;
      for (int c = 0; c < D; ++c) P[a][c] = 0.0;
    }
    for (int64_t k = 0; k < nv; ++k) {
      double c[MAXD], c2 = 0.0;
      for (int d = 0; d < D; ++d) {
        c[d] = u[k * D + d] - p.U[d];
        c2 += c[d] * c[d];
      }
      for (int a = 0; a < D; ++a) {
        q[a] += 0.5 * w[k] * c[a] * (c2 * h[k] + (b ? b[k] : 0.0));
        for (int e = 0; e < D; ++e) P[a][e] += w[k] * c[a] * c[e] * h[k];
      }
    }
    double *o = out + i * n13;
    const double pr = p.rho / (2.0 * p.lam);
    o[0] = p.rho;
    for (int d = 0; d < D; ++d) o[1 + d] = p.U[d];
    o[D + 1] = 1.0 / p.lam;
    int s = 0;
    for (int a = 0; a < D; ++a)
      for (int e = a; e < D; ++e) o[D + 2 + s++] = P[a][e] - (a == e ? pr : 0.0);
    for (int d = 0; d < D; ++d) o[D + 2 + ns + d] = q[d];
  }
}

/* Chapman-Enskog distribution of given thirteen-moment fields (reading R21):
 * fields[cell] as written by orc_moments13; f[r][cell][k]. */
void orc_chapman_enskog(int D, int K, int64_t nc, int64_t nv, const double *u, const double *fields, double *f) {
  const int Kxi = K + 3 - D, nr = Kxi > 0 ? 2 : 1, ns = D * (D + 1) / 2, n13 = 2 * D + 2 + ns;
  for (int64_t i = 0; i < nc; ++i) {
    const double *x = fields + i * n13;
    prim_t p;
    p.rho = x[0];
    for (int d = 0; d < D; ++d) p.U[d] = x[1 + d];
    p.lam = 1.0 / x[D + 1];
    const double *sig = x + D + 2, *q = x + D + 2 + ns;
    const double a2 = 2.0 * p.lam * p.lam / p.rho, a3 = 4.0 * p.lam * p.lam / ((K + 5.0) * p.rho);
    double tr = 0.0;
    for (int a = 0, s = 0; a < D; ++a)
      for (int e = a; e < D; ++e, ++s)
        if (a == e) tr += sig[s];
    const double th = -p.lam * tr / p.rho, tb = Kxi > 0 ? -p.lam * (Kxi + 2.0) * tr / (Kxi * p.rho) : 0.0;
    for (int64_t k = 0; k < nv; ++k) {
      double c[MAXD], c2 = 0.0, qc = 0.0, scc = 0.0;
      for (int d = 0; d < D; ++d) {
        c[d] = u[k * D + d] - p.U[d];
        c2 += c[d] * c[d];
        qc += q[d] * c[d];
      }
      int s = 0;
      for (int a = 0; a < D; ++a)
        for (int e = a; e < D; ++e) scc += (a == e ? 1.0 : 2.0) * sig[s++] * c[a] * c[e];
      const double H = maxwell_H(D, &p, u + k * D);
      f[i * nv + k] = H * (1.0 + a2 * scc + th + a3 * qc * (2.0 * p.lam * c2 - (D + 2)));
      if (nr == 2)
        f[(nc + i) * nv + k] = Kxi / (2.0 * p.lam) * H * (1.0 + a2 * scc + tb + a3 * qc * (2.0 * p.lam * c2 - D));
    }
  }
}

/* Initial distribution: discrete reduced Maxwellian of W (reading R18). */
void orc_initial_f(int D, int K, int64_t nc, int64_t nv, const double *u, const double *W, double *f) {
  int Kxi = K + 3 - D, nr = Kxi > 0 ? 2 : 1;
  for (int64_t i = 0; i < nc; ++i) {
    prim_t p;
    prim_from_W(D, K, W + i * (D + 2), &p);
    for (int64_t k = 0; k < nv; ++k) {
      double H = maxwell_H(D, &p, u + k * D);
      f[i * nv + k] = H;
      if (nr == 2) f[(nc + i) * nv + k] = Kxi / (2.0 * p.lam) * H;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* One time step (Algorithm 5)                                                */
/* ------------------------------------------------------------------------ */

typedef struct {
  prim_t p0;          /* interface Maxwellian */
  double a[MAXD][NW]; /* spatial slopes per direction */
  double A[NW];       /* time slope */
  double q0[MAXD];
  double G[5];
  double xi4;         /* <xi^4> of g0 */
} face_coef_t;

/* Velocity-independent part of the equilibrium flux terms at velocity u:
 * returns h0 = H0 + H0+, b0 = B0 + B0+, ugH = u.grad H0, ugB, dtH, dtB. */
static void eq_terms(int D, int Kxi, int shakhov, double Pr, const face_coef_t *fc, const double *u,
                     double *h0, double *b0, double *ugH, double *ugB, double *dtH, double *dtB) {
  const prim_t *p = &fc->p0;
  double H = maxwell_H(D, p, u);
  double B = Kxi / (2.0 * p->lam) * H;
  double Hs = 0.0, Bs = 0.0;
  if (shakhov) shakhov_plus(D, Kxi, Pr, p, fc->q0, u, H, &Hs, &Bs);
  *h0 = H + Hs;
  *b0 = B + Bs;
  double u2 = 0.0;
  for (int d = 0; d < D; ++d) u2 += u[d] * u[d];
  double gH = 0.0, gB = 0.0;
  for (int d = 0; d < D; ++d) {
    const double *a = fc->a[d];
    double poly = a[0] + 0.5 * a[D + 1] * u2;
    for (int e = 0; e < D; ++e) poly += a[1 + e] * u[e];
    gH += u[d] * (poly * H + 0.5 * a[D + 1] * B);
    gB += u[d] * (poly * B + 0.5 * a[D + 1] * fc->xi4 * H);
  }
  *ugH = gH;
  *ugB = gB;
  double poly = fc->A[0] + 0.5 * fc->A[D + 1] * u2;
  for (int e = 0; e < D; ++e) poly += fc->A[1 + e] * u[e];
  *dtH = poly * H + 0.5 * fc->A[D + 1] * B;
  *dtB = poly * B + 0.5 * fc->A[D + 1] * fc->xi4 * H;
}

/* Ghost conservative state of boundary condition bc for interior cell state Wi. */
static void ghost_W(int D, int K, const orc_bc *bc, const double *Wi, double *Wg) {
  if (bc->type == 3) { for (int t = 0; t < D + 2; ++t) Wg[t] = Wi[t]; return; }
  prim_t p;
  p.rho = bc->rho;
  for (int d = 0; d < D; ++d) p.U[d] = bc->u[d];
  p.lam = 1.0 / bc->T;
  W_from_prim(D, K, &p, Wg);
}

int orc_step(const orc_mesh *m, int64_t nv, const double *u, const double *w, const orc_params *p,
             double dt, double *W, double *f, double *diag, double *F_out) {
  const int D = m->dim, K = p->K, nw = D + 2;
  const int Kxi = K + 3 - D, nr = Kxi > 0 ? 2 : 1;
  const int shakhov = p->model == 1;
  const int64_t Nc = m->n_cells, Nf = m->n_faces;
  adj_t adj;
  build_adj(m, &adj);

  prim_t *pc = (prim_t *)malloc(sizeof(prim_t) * Nc);
  double *tau = (double *)malloc(sizeof(double) * Nc);
  double *q = (double *)calloc(Nc * MAXD, sizeof(double));
  double *gW = (double *)calloc(Nc * MAXD * NW, sizeof(double));    /* limited macro gradients */
  double *gf = (double *)calloc((size_t)nr * Nc * nv * D, sizeof(double)); /* limited micro gradients */
  double *Hf = (double *)calloc((size_t)nr * Nf * nv, sizeof(double));     /* time-integrated micro fluxes */
  double *F = (double *)calloc(Nf * NW, sizeof(double));
  double *Wnew = (double *)malloc(sizeof(double) * Nc * nw);
  face_coef_t *fcs = (face_coef_t *)calloc(Nf, sizeof(face_coef_t));
  int bad = 0;
  for (int64_t i = 0; i < Nc; ++i)
    if (adj.off[i + 1] - adj.off[i] > MAXF) bad = 1;
  for (int64_t fidx = 0; fidx < Nf; ++fidx)
    if (m->own[fidx] == m->nei[fidx]) bad = 1; /* a face must join two distinct cells */
  if (bad) goto fail;

  /* 1. cell primitives, relaxation time, heat flux (Algorithm 5, first step; Eq. 13) */
#pragma omp parallel
  {
    double *scr = (double *)malloc(sizeof(double) * nv);
#pragma omp for schedule(static)
    for (int64_t i = 0; i < Nc; ++i) {
      if (!prim_from_W(D, K, W + i * nw, &pc[i])) { bad = 1; continue; }
      tau[i] = tau_of(p, &pc[i]);
      if (shakhov) heat_flux(D, nv, u, w, f + i * nv, nr == 2 ? f + (Nc + i) * nv : NULL, pc[i].U, p, q + i * MAXD, scr);
    }
    free(scr);
  }
  if (bad) goto fail;

  /* 2-3. ghost states and limited least-squares gradient of W (Algorithm 5, macro reconstruction) */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < Nc; ++i) {
    double Mm[MAXD * MAXD] = {0}, rhs[NW][MAXD];
    memset(rhs, 0, sizeof(rhs));
    double wmax[NW], wmin[NW];
    const double *Wi = W + i * nw;
    for (int t = 0; t < nw; ++t) { wmax[t] = Wi[t]; wmin[t] = Wi[t]; }
    int nst = 0;
    for (int64_t s = adj.off[i]; s < adj.off[i + 1]; ++s) {
      int64_t fidx = adj.face[s];
      double nout[MAXD], xfc[MAXD], xo[MAXD], Wo[NW];
      int64_t j = face_view(m, fidx, i, nout, xfc, xo);
      if (j < 0) {
        const orc_bc *bc = &m->bc[-j - 1];
        if (bc->type == 1) {
          /* wall: zero-gradient ghost, offset in the matrix only (reading R3) */
          for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b)
              Mm[a * D + b] += (xo[a] - m->xc[i * D + a]) * (xo[b] - m->xc[i * D + b]);
          continue;
        }
        ghost_W(D, K, bc, Wi, Wo);
      } else {
        for (int t = 0; t < nw; ++t) Wo[t] = W[j * nw + t];
      }
      double dx[MAXD];
      for (int d = 0; d < D; ++d) dx[d] = xo[d] - m->xc[i * D + d];
      for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) Mm[a * D + b] += dx[a] * dx[b];
      for (int t = 0; t < nw; ++t) {
        for (int d = 0; d < D; ++d) rhs[t][d] += dx[d] * (Wo[t] - Wi[t]);
        if (Wo[t] > wmax[t]) wmax[t] = Wo[t];
        if (Wo[t] < wmin[t]) wmin[t] = Wo[t];
      }
      nst++;
    }
    double g[NW][MAXD];
    memset(g, 0, sizeof(g));
    double Minv[MAXD * MAXD];
    if (nst > 0 && lsq_inverse(D, Mm, Minv)) {
      for (int t = 0; t < nw; ++t)
        for (int a = 0; a < D; ++a)
          for (int b = 0; b < D; ++b) g[t][a] += Minv[a * D + b] * rhs[t][b];
    }
    double hcell = pow(m->vol[i], 1.0 / D), eps2 = pow(p->venkat_K * hcell, 3.0);
    for (int t = 0; t < nw; ++t) {
      double phi = 1.0;
      for (int64_t s = adj.off[i]; s < adj.off[i + 1]; ++s) {
        double nout[MAXD], xfc[MAXD], xo[MAXD];
        face_view(m, adj.face[s], i, nout, xfc, xo);
        double d2 = 0.0;
        for (int d = 0; d < D; ++d) d2 += g[t][d] * (xfc[d] - m->xc[i * D + d]);
        double mag = fabs(wmax[t]) > fabs(wmin[t]) ? fabs(wmax[t]) : fabs(wmin[t]);
        double ph = limiter_phi(p->limiter, d2, wmax[t] - Wi[t], wmin[t] - Wi[t], eps2 * mag * mag);
        if (ph < phi) phi = ph;
      }
      if (phi < 0.0) phi = 0.0;
      for (int d = 0; d < D; ++d) gW[(i * NW + t) * MAXD + d] = phi * g[t][d];
    }
  }

  /* 4. interface equilibrium state and coefficients (Algorithm 5; Eq. 32-35) */
#pragma omp parallel for schedule(static)
  for (int64_t fidx = 0; fidx < Nf; ++fidx) {
    int64_t i = m->own[fidx], j = m->nei[fidx];
    face_coef_t *fc = &fcs[fidx];
    if (j < 0 && m->bc[-j - 1].type == 1) continue; /* walls: step 7 */
    const double *n = m->nrm + fidx * D, *xf = m->xf + fidx * D, *sh = m->shift + fidx * D;
    double Wl[NW], Wr[NW], dW0[MAXD][NW];
    const double *Wi = W + i * nw;
    for (int t = 0; t < nw; ++t) {
      double s = 0.0;
      for (int d = 0; d < D; ++d) s += gW[(i * NW + t) * MAXD + d] * (xf[d] - m->xc[i * D + d]);
      Wl[t] = Wi[t] + s;
    }
    prim_t tp;
    if (!prim_from_W(D, K, Wl, &tp)) for (int t = 0; t < nw; ++t) Wl[t] = Wi[t];
    double qr[MAXD] = {0, 0, 0};
    if (j >= 0) {
      const double *Wj = W + j * nw;
      for (int t = 0; t < nw; ++t) {
        double s = 0.0;
        for (int d = 0; d < D; ++d) s += gW[(j * NW + t) * MAXD + d] * (xf[d] - sh[d] - m->xc[j * D + d]);
        Wr[t] = Wj[t] + s;
      }
      if (!prim_from_W(D, K, Wr, &tp)) for (int t = 0; t < nw; ++t) Wr[t] = Wj[t];
      for (int t = 0; t < nw; ++t)
        for (int d = 0; d < D; ++d)
          dW0[d][t] = 0.5 * (gW[(i * NW + t) * MAXD + d] + gW[(j * NW + t) * MAXD + d]);
      for (int d = 0; d < D; ++d) qr[d] = q[j * MAXD + d];
    } else {
      ghost_W(D, K, &m->bc[-j - 1], Wi, Wr);
      for (int t = 0; t < nw; ++t)
        for (int d = 0; d < D; ++d) dW0[d][t] = 0.5 * gW[(i * NW + t) * MAXD + d];
    }
    double W0[NW];
    orc_interface_W0(D, K, Wl, Wr, n, W0);
    prim_from_W(D, K, W0, &fc->p0);
    for (int d = 0; d < D; ++d) fc->q0[d] = 0.5 * (q[i * MAXD + d] + qr[d]);
    for (int d = 0; d < D; ++d) orc_micro_slope(D, K, W0, dW0[d], fc->a[d]);
    {
      /* orc_time_slope takes the D slope vectors packed with stride D + 2 */
      double apack[MAXD * NW];
      for (int d = 0; d < D; ++d)
        for (int t = 0; t < nw; ++t) apack[d * nw + t] = fc->a[d][t];
      orc_time_slope(D, K, W0, apack, fc->A);
    }
    double tau0 = tau_of(p, &fc->p0);
    if (p->shock_tau_fix) {
      prim_t pl, pr;
      prim_from_W(D, K, Wl, &pl);
      prim_from_W(D, K, Wr, &pr);
      double PL = pl.rho / (2.0 * pl.lam), PR = pr.rho / (2.0 * pr.lam);
      tau0 += dt * fabs(PL - PR) / (PL + PR);
    }
    orc_time_coefficients(dt, tau0, fc->G);
    fc->xi4 = Kxi * (Kxi + 2.0) / (4.0 * fc->p0.lam * fc->p0.lam);
  }

  /* 5. limited least-squares gradients of h and b (reconstruction, Eq. 31) */
#pragma omp parallel
  {
#pragma omp for schedule(static)
    for (int64_t i = 0; i < Nc; ++i) {
      const double *xi = m->xc + i * D;
      double Mm[MAXD * MAXD] = {0};
      int64_t sidx[MAXF];
      double dxs[MAXF][MAXD];
      int nst = 0;
      for (int64_t s = adj.off[i]; s < adj.off[i + 1]; ++s) {
        double nout[MAXD], xfc[MAXD], xo[MAXD];
        int64_t j = face_view(m, adj.face[s], i, nout, xfc, xo);
        if (j < 0 && m->bc[-j - 1].type == 1) {
          /* wall: zero-gradient ghost, offset in the matrix only (reading R3) */
          for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b) Mm[a * D + b] += (xo[a] - xi[a]) * (xo[b] - xi[b]);
          continue;
        }
        sidx[nst] = s;
        for (int d = 0; d < D; ++d) dxs[nst][d] = xo[d] - xi[d];
        for (int a = 0; a < D; ++a)
          for (int b = 0; b < D; ++b) Mm[a * D + b] += dxs[nst][a] * dxs[nst][b];
        nst++;
      }
      double Minv[MAXD * MAXD];
      int ok = nst > 0 && lsq_inverse(D, Mm, Minv);
      double hcell = pow(m->vol[i], 1.0 / D), eps2 = pow(p->venkat_K * hcell, 3.0);
      for (int r = 0; r < nr; ++r) {
        const double *fi = f + ((size_t)r * Nc + i) * nv;
        for (int64_t k = 0; k < nv; ++k) {
          double g[MAXD] = {0, 0, 0}, rhs[MAXD] = {0, 0, 0};
          double fmax = fi[k], fmin = fi[k];
          for (int t = 0; t < nst; ++t) {
            int64_t fidx = adj.face[sidx[t]];
            double nout[MAXD], xfc[MAXD], xo[MAXD], fo_v;
            int64_t j = face_view(m, fidx, i, nout, xfc, xo);
            if (j >= 0) {
              fo_v = f[((size_t)r * Nc + j) * nv + k];
            } else {
              double Wg[NW];
              prim_t pg;
              ghost_W(D, K, &m->bc[-j - 1], W + i * nw, Wg);
              prim_from_W(D, K, Wg, &pg);
              double H = maxwell_H(D, &pg, u + k * D);
              fo_v = (r == 0) ? H : Kxi / (2.0 * pg.lam) * H;
            }
            for (int d = 0; d < D; ++d) rhs[d] += dxs[t][d] * (fo_v - fi[k]);
            if (fo_v > fmax) fmax = fo_v;
            if (fo_v < fmin) fmin = fo_v;
          }
          if (ok)
            for (int a = 0; a < D; ++a)
              for (int b = 0; b < D; ++b) g[a] += Minv[a * D + b] * rhs[b];
          double phi = 1.0;
          for (int64_t s = adj.off[i]; s < adj.off[i + 1]; ++s) {
            double nout[MAXD], xfc[MAXD], xo[MAXD];
            face_view(m, adj.face[s], i, nout, xfc, xo);
            double d2 = 0.0;
            for (int d = 0; d < D; ++d) d2 += g[d] * (xfc[d] - xi[d]);
            double mag = fabs(fmax) > fabs(fmin) ? fabs(fmax) : fabs(fmin);
            double ph = limiter_phi(p->limiter, d2, fmax - fi[k], fmin - fi[k], eps2 * mag * mag);
            if (ph < phi) phi = ph;
          }
          if (phi < 0.0) phi = 0.0;
          for (int d = 0; d < D; ++d) gf[(((size_t)r * Nc + i) * nv + k) * D + d] = phi * g[d];
        }
      }
    }
  }

  /* 6-7. time-integrated micro fluxes and macro fluxes per face (Eq. 25, 28-29, 33-38) */
  double wall_mass_max = 0.0;
#pragma omp parallel
  {
    double *cH = (double *)malloc(sizeof(double) * nv * NW);
    double *tmp = (double *)malloc(sizeof(double) * nv);
    double local_wall = 0.0;
#pragma omp for schedule(dynamic, 16)
    for (int64_t fidx = 0; fidx < Nf; ++fidx) {
      int64_t i = m->own[fidx], j = m->nei[fidx];
      const double *n = m->nrm + fidx * D, *xf = m->xf + fidx * D, *sh = m->shift + fidx * D;
      const double *xi = m->xc + i * D;
      double *Hout = Hf + (size_t)fidx * nv, *Bout = nr == 2 ? Hf + ((size_t)Nf + fidx) * nv : NULL;
      if (j < 0 && m->bc[-j - 1].type == 1) {
        /* diffuse wall: Eq. 36-38 with reading R9 */
        const orc_bc *bc = &m->bc[-j - 1];
        prim_t pw;
        pw.rho = 1.0;
        for (int d = 0; d < D; ++d) pw.U[d] = bc->u[d];
        pw.lam = 1.0 / bc->T;
        for (int64_t k = 0; k < nv; ++k) {
          const double *uk = u + k * D;
          double un = 0.0;
          for (int d = 0; d < D; ++d) un += uk[d] * n[d];
          double in = 0.0, out = 0.0;
          if (un > 0.0) {
            const double *g = gf + ((size_t)i * nv + k) * D;
            double fin = f[i * nv + k], ug = 0.0;
            for (int d = 0; d < D; ++d) { fin += g[d] * (xf[d] - xi[d]); ug += uk[d] * g[d]; }
            in = w[k] * un * (dt * fin - 0.5 * dt * dt * ug);
          } else if (un < 0.0) {
            out = w[k] * un * dt * maxwell_H(D, &pw, uk);
          }
          cH[k] = in;
          tmp[k] = out;
        }
        double sin = vsum(cH, nv, p->block_v, p->p_v), sout = vsum(tmp, nv, p->block_v, p->p_v);
        double rho_w = (sout != 0.0) ? -sin / sout : 0.0;
        for (int64_t k = 0; k < nv; ++k) {
          const double *uk = u + k * D;
          double un = 0.0;
          for (int d = 0; d < D; ++d) un += uk[d] * n[d];
          double ih = 0.0, ib = 0.0;
          if (un > 0.0) {
            for (int r = 0; r < nr; ++r) {
              const double *g = gf + (((size_t)r * Nc + i) * nv + k) * D;
              double fin = f[((size_t)r * Nc + i) * nv + k], ug = 0.0;
              for (int d = 0; d < D; ++d) { fin += g[d] * (xf[d] - xi[d]); ug += uk[d] * g[d]; }
              double v = dt * fin - 0.5 * dt * dt * ug;
              if (r == 0) ih = v; else ib = v;
            }
          } else if (un < 0.0) {
            double H = maxwell_H(D, &pw, uk);
            ih = dt * rho_w * H;
            ib = dt * rho_w * Kxi / (2.0 * pw.lam) * H;
          }
          Hout[k] = un * ih;
          if (Bout) Bout[k] = un * ib;
        }
      } else {
        const face_coef_t *fc = &fcs[fidx];
        double Wg[NW];
        prim_t pg;
        if (j < 0) {
          ghost_W(D, K, &m->bc[-j - 1], W + i * nw, Wg);
          prim_from_W(D, K, Wg, &pg);
        }
        for (int64_t k = 0; k < nv; ++k) {
          const double *uk = u + k * D;
          double un = 0.0;
          for (int d = 0; d < D; ++d) un += uk[d] * n[d];
          if (un == 0.0) { Hout[k] = 0.0; if (Bout) Bout[k] = 0.0; continue; }
          double h0, b0, ugH, ugB, dtH, dtB;
          eq_terms(D, Kxi, shakhov, p->Pr, fc, uk, &h0, &b0, &ugH, &ugB, &dtH, &dtB);
          for (int r = 0; r < nr; ++r) {
            double fface, ug = 0.0;
            if (un > 0.0) {
              const double *g = gf + (((size_t)r * Nc + i) * nv + k) * D;
              fface = f[((size_t)r * Nc + i) * nv + k];
              for (int d = 0; d < D; ++d) { fface += g[d] * (xf[d] - xi[d]); ug += uk[d] * g[d]; }
            } else if (j >= 0) {
              const double *g = gf + (((size_t)r * Nc + j) * nv + k) * D;
              const double *xj = m->xc + j * D;
              fface = f[((size_t)r * Nc + j) * nv + k];
              for (int d = 0; d < D; ++d) { fface += g[d] * (xf[d] - sh[d] - xj[d]); ug += uk[d] * g[d]; }
            } else {
              double H = maxwell_H(D, &pg, uk);
              fface = (r == 0) ? H : Kxi / (2.0 * pg.lam) * H;
            }
            double eq = (r == 0) ? fc->G[2] * h0 + fc->G[3] * ugH + fc->G[4] * dtH
                                 : fc->G[2] * b0 + fc->G[3] * ugB + fc->G[4] * dtB;
            double val = un * (fc->G[0] * fface + fc->G[1] * ug + eq);
            if (r == 0) Hout[k] = val; else Bout[k] = val;
          }
        }
      }
      /* macro flux F = sum_k omega_k (H, u H, (|u|^2 H + B)/2), Eq. 28 */
      for (int t = 0; t < nw; ++t) {
        for (int64_t k = 0; k < nv; ++k) {
          const double *uk = u + k * D;
          double v;
          if (t == 0) v = Hout[k];
          else if (t <= D) v = uk[t - 1] * Hout[k];
          else {
            double u2 = 0.0;
            for (int d = 0; d < D; ++d) u2 += uk[d] * uk[d];
            v = 0.5 * (u2 * Hout[k] + (Bout ? Bout[k] : 0.0));
          }
          tmp[k] = w[k] * v;
        }
        F[fidx * NW + t] = vsum(tmp, nv, p->block_v, p->p_v);
      }
      if (j < 0 && m->bc[-j - 1].type == 1) {
        double s = fabs(F[fidx * NW]);
        if (s > local_wall) local_wall = s;
      }
    }
#pragma omp critical
    { if (local_wall > wall_mass_max) wall_mass_max = local_wall; }
    free(cH);
    free(tmp);
  }

  /* 8. stage 1 (Eq. 41): transport and the old-time half of the collision term */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < Nc; ++i) {
    double beta0 = dt / (2.0 * tau[i]);
    for (int64_t k = 0; k < nv; ++k) {
      const double *uk = u + k * D;
      double fp0[2];
      equilibrium_hb(D, Kxi, shakhov, p->Pr, &pc[i], q + i * MAXD, uk, &fp0[0], &fp0[1]);
      for (int r = 0; r < nr; ++r) {
        double *fik = f + ((size_t)r * Nc + i) * nv + k;
        double flux = 0.0;
        for (int64_t s = adj.off[i]; s < adj.off[i + 1]; ++s) {
          int64_t fidx = adj.face[s];
          double sg = (m->own[fidx] == i) ? 1.0 : -1.0;
          flux += sg * m->area[fidx] * Hf[((size_t)r * Nf + fidx) * nv + k];
        }
        *fik = *fik - flux / m->vol[i] + beta0 * (fp0[r] - *fik);
      }
    }
  }

  /* 9. conservative update (Eq. 27) */
  double res[NW] = {0, 0, 0, 0, 0};
  for (int64_t i = 0; i < Nc; ++i) {
    double acc[NW] = {0, 0, 0, 0, 0};
    for (int64_t s = adj.off[i]; s < adj.off[i + 1]; ++s) {
      int64_t fidx = adj.face[s];
      double sg = (m->own[fidx] == i) ? 1.0 : -1.0;
      for (int t = 0; t < nw; ++t) acc[t] += sg * m->area[fidx] * F[fidx * NW + t];
    }
    for (int t = 0; t < nw; ++t) {
      Wnew[i * nw + t] = W[i * nw + t] - acc[t] / m->vol[i];
      double dw = Wnew[i * nw + t] - W[i * nw + t];
      res[t] += dw * dw;
    }
  }

  /* 10. stage 2 (Eq. 42) from W^{n+1}, lagged heat flux (reading R12) */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < Nc; ++i) {
    prim_t pn;
    if (!prim_from_W(D, K, Wnew + i * nw, &pn)) { bad = 1; continue; }
    double beta1 = dt / (2.0 * tau_of(p, &pn));
    for (int64_t k = 0; k < nv; ++k) {
      double fp1[2];
      equilibrium_hb(D, Kxi, shakhov, p->Pr, &pn, q + i * MAXD, u + k * D, &fp1[0], &fp1[1]);
      for (int r = 0; r < nr; ++r) {
        double *fik = f + ((size_t)r * Nc + i) * nv + k;
        *fik = (*fik + beta1 * fp1[r]) / (1.0 + beta1);
      }
    }
  }
  if (bad) goto fail;
  memcpy(W, Wnew, sizeof(double) * Nc * nw);
  if (F_out) memcpy(F_out, F, sizeof(double) * Nf * NW);
  if (diag) {
    for (int t = 0; t < nw; ++t) diag[t] = sqrt(res[t] / Nc);
    diag[nw] = wall_mass_max;
  }
  free(pc); free(tau); free(q); free(gW); free(gf); free(Hf); free(F); free(Wnew); free(fcs);
  free(adj.off); free(adj.face);
  return 0;
fail:
  free(pc); free(tau); free(q); free(gW); free(gf); free(Hf); free(F); free(Wnew); free(fcs);
  free(adj.off); free(adj.face);
  return 1;
}

/* Runs n steps; dt from reading R4 unless p->dt_override > 0.  diag receives
 * nsteps rows of (residual[nw], max |wall mass flux|); F_out (if not NULL)
 * the macro fluxes F[face][5] of the last step. */
int orc_run(const orc_mesh *m, int64_t nv, const double *u, const double *w, const orc_params *p,
            double *W, double *f, int32_t nsteps, double *dt_out, double *diag, double *F_out) {
  double dt = p->dt_override > 0.0 ? p->dt_override : orc_time_step(m, nv, u, w, p->cfl);
  if (dt_out) *dt_out = dt;
  for (int32_t s = 0; s < nsteps; ++s) {
    if (orc_step(m, nv, u, w, p, dt, W, f, diag ? diag + (size_t)s * (m->dim + 3) : NULL,
                 s == nsteps - 1 ? F_out : NULL)) return 1;
  }
  return 0;
}

/* Surface quantities of every diffuse-wall face (reading R20), wall faces in
 * ascending face order: faces[i], vals[i] = (p_w, tau_w[0..D-1], q_w) and, if
 * freestream = (rho, U[0..D-1], T) is given, coef[i] = (C_p, C_t, C_h).
 * Returns the number of wall faces. */
int64_t orc_surface(const orc_mesh *m, const double *F, double dt, const double *freestream, int64_t *faces,
                    double *vals, double *coef) {
  const int D = m->dim;
  int64_t nw_ = 0;
  for (int64_t fidx = 0; fidx < m->n_faces; ++fidx) {
    int64_t j = m->nei[fidx];
    if (j >= 0 || m->bc[-j - 1].type != 1) continue;
    const orc_bc *bc = &m->bc[-j - 1];
    const double *n = m->nrm + fidx * D, *Ff = F + fidx * NW;
    double P[MAXD], pn = 0.0, work = 0.0;
    for (int d = 0; d < D; ++d) {
      P[d] = Ff[1 + d] / dt;
      pn += P[d] * n[d];
      work += bc->u[d] * Ff[1 + d];
    }
    double *v = vals + nw_ * (D + 2);
    v[0] = pn;
    double t2 = 0.0;
    for (int d = 0; d < D; ++d) {
      v[1 + d] = P[d] - pn * n[d];
      t2 += v[1 + d] * v[1 + d];
    }
    v[D + 1] = (Ff[D + 1] - work) / dt;
    if (freestream && coef) {
      double rho = freestream[0], U2 = 0.0, T = freestream[D + 1];
      for (int d = 0; d < D; ++d) U2 += freestream[1 + d] * freestream[1 + d];
      double qdyn = 0.5 * rho * U2;
      coef[nw_ * 3 + 0] = (pn - 0.5 * rho * T) / qdyn;
      coef[nw_ * 3 + 1] = sqrt(t2) / qdyn;
      coef[nw_ * 3 + 2] = v[D + 1] / (qdyn * sqrt(U2));
    }
    faces[nw_] = fidx;
    ++nw_;
  }
  return nw_;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the following calls (n >= 1); returns the previous count. */
int orc_set_threads(int n) {
  const int old = orc_num_threads();
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
  return old;
}
