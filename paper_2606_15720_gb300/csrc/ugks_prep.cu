// Per-cell and per-face FP64 kernels of one UGKS step (Algorithm 5, the
// stages before the velocity-block sweep), plus set-up and data-movement
// kernels.  GB300 executes FP64 at a small fraction of its FP32 rate, so FP64
// is confined to O(N_cells + N_faces) work here: primitive variables, the
// limited least-squares gradient of W, and the interface coefficients whose
// exp(-dt/tau) terms cancel at small dt/tau (Eq. 34-35).
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "ugks_device.cuh"
#include "ugks_internal.cuh"
#include "ugks_kernels.cuh"

namespace ugks {

namespace {

// Small fixed-size vectors passed by value, so that with D a template
// parameter every loop unrolls and all of them live in registers.
struct Vec5 {
  double v[NWP];
};

struct Prim {
  double rho, U[3], lam;
};

// lambda = (K+3) rho / (4 (rho E - rho |U|^2 / 2)), R = 1/2 (Eq. 6, 10).
template <int D>
__device__ __forceinline__ Prim prim_of(const Vec5& W, int K, bool& ok) {
  Prim p;
  p.rho = W.v[0];
  double u2 = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) p.U[d] = d < D ? W.v[1 + (d < D ? d : 0)] / W.v[0] : 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) u2 += p.U[d] * p.U[d];
  const double ein = W.v[D + 1] - 0.5 * W.v[0] * u2;
  p.lam = (K + 3) * W.v[0] / (4.0 * ein);
  ok = (p.rho > 0.0) && (ein > 0.0) && isfinite(p.lam) && isfinite(u2);
  return p;
}

template <int D>
__device__ __forceinline__ Vec5 cons_of(const Prim& p, int K) {
  Vec5 W;
  double u2 = 0.0;
#pragma unroll
  for (int t = 0; t < NWP; ++t) W.v[t] = 0.0;
  W.v[0] = p.rho;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    W.v[1 + d] = p.rho * p.U[d];
    u2 += p.U[d] * p.U[d];
  }
  W.v[D + 1] = 0.5 * p.rho * u2 + (K + 3) * p.rho / (4.0 * p.lam);
  return W;
}

template <int D>
__device__ __forceinline__ Vec5 load5(const double* W) {
  Vec5 r;
#pragma unroll
  for (int t = 0; t < NWP; ++t) r.v[t] = t < D + 2 ? W[t] : 0.0;
  return r;
}

// tau = mu / p with mu = mu_ref T^omega and p = rho / (2 lambda).
__device__ __forceinline__ double tau_of(const Prim& p, const Gas& g) {
  const double T = 1.0 / p.lam;
  return g.mu_ref * pow(T, g.omega) * 2.0 * p.lam / p.rho;
}

// Ghost conservative state of an artificial boundary (Sec. 2.1).
template <int D>
__device__ __forceinline__ Vec5 ghost_state(const BCDev& bc, const Vec5& Wi, int K) {
  if (bc.type == 3) return Wi;
  Prim p;
  p.rho = bc.rho;
#pragma unroll
  for (int d = 0; d < 3; ++d) p.U[d] = bc.u[d];
  p.lam = 1.0 / bc.T;
  return cons_of<D>(p, K);
}

// Venkatakrishnan / Barth-Jespersen limiter value for one face; eps2 is the
// Venkatakrishnan constant (K_v h)^3 already scaled by the squared magnitude
// of the limited quantity on the stencil.
__device__ __forceinline__ double limiter_fn(int kind, double d2, double dmax, double dmin, double eps2) {
  if (kind == 0 || d2 == 0.0) return 1.0;
  const double dp = d2 > 0.0 ? dmax : dmin;
  if (kind == 2) return fmin(1.0, dp / d2);
  const double num = dp * dp + eps2 + 2.0 * d2 * dp;
  const double den = dp * dp + 2.0 * d2 * d2 + dp * d2 + eps2;
  return den != 0.0 ? num / den : 1.0;
}

// Solves rho <psi psi^T> x = rhs for a Maxwellian with N = K + 3 degrees of
// freedom, in closed form through the peculiar velocity: with a.psi written
// as b0 + b.c + aE (c^2 + xi^2)/2, the mass, momentum and energy moments give
//   b0 + aE N/(4 lam) = dr,  b = 2 lam (dm - U dr),
//   b0 N/(4 lam) + aE N(N+2)/(16 lam^2) = dE - |U|^2 dr/2 - U.b/(2 lam).
template <int D>
__device__ __forceinline__ Vec5 maxwell_solve(const Prim& p, int K, const Vec5& rhs) {
  const double N = K + 3.0, lam = p.lam;
  const double dr = rhs.v[0] / p.rho, dE = rhs.v[D + 1] / p.rho;
  double b[3] = {0.0, 0.0, 0.0}, u2 = 0.0, ub = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    b[d] = 2.0 * lam * (rhs.v[1 + d] / p.rho - p.U[d] * dr);
    u2 += p.U[d] * p.U[d];
    ub += p.U[d] * b[d];
  }
  const double R = dE - 0.5 * u2 * dr - ub / (2.0 * lam);
  const double aE = (R - dr * N / (4.0 * lam)) * 8.0 * lam * lam / N;
  const double b0 = dr - aE * N / (4.0 * lam);
  Vec5 x;
#pragma unroll
  for (int t = 0; t < NWP; ++t) x.v[t] = 0.0;
  double a0 = b0 - 0.5 * aE * u2;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const double au = b[d] - aE * p.U[d];
    x.v[1 + d] = au;
    a0 -= au * p.U[d];
  }
  x.v[0] = a0;
  x.v[D + 1] = aE;
  return x;
}

// Directional derivative of the Euler flux F_dir(W) along dW; equal to the
// moment rho <psi u_dir (a.psi)> of the slope a with rho <psi psi^T> a = dW.
template <int D>
__device__ __forceinline__ Vec5 euler_flux_derivative(const Prim& p, int K, int dir, const Vec5& W, const Vec5& dW) {
  const double N = K + 3.0;
  double u2 = 0.0, Udm = 0.0, dU[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int d = 0; d < D; ++d) {
    u2 += p.U[d] * p.U[d];
    Udm += p.U[d] * dW.v[1 + d];
    dU[d] = (dW.v[1 + d] - p.U[d] * dW.v[0]) / p.rho;
  }
  const double pres = p.rho / (2.0 * p.lam);
  const double dp = (2.0 / N) * (dW.v[D + 1] - Udm + 0.5 * u2 * dW.v[0]);
  double Udir = 0.0, dUdir = 0.0, mdir = 0.0, dmdir = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d)
    if (d == dir) {
      Udir = p.U[d];
      dUdir = dU[d];
      mdir = W.v[1 + d];
      dmdir = dW.v[1 + d];
    }
  Vec5 out;
#pragma unroll
  for (int t = 0; t < NWP; ++t) out.v[t] = 0.0;
  out.v[0] = dmdir;
#pragma unroll
  for (int e = 0; e < D; ++e) out.v[1 + e] = dmdir * p.U[e] + mdir * dU[e] + (e == dir ? dp : 0.0);
  out.v[D + 1] = dUdir * (W.v[D + 1] + pres) + Udir * (dW.v[D + 1] + dp);
  return out;
}

// rho <psi> over the half space s (u.n) > 0 of a Maxwellian.
template <int D>
__device__ __forceinline__ Vec5 half_space_moments(const Prim& p, int K, const double* n, double s) {
  const int Kxi = K + 3 - D;
  double Un = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) Un += p.U[d] * n[d];
  const double sl = sqrt(p.lam);
  const double e = exp(-p.lam * Un * Un) / (2.0 * sqrt(M_PI * p.lam));
  const double m0 = 0.5 * erfc(-s * sl * Un);
  const double m1 = Un * m0 + s * e;
  const double m2 = Un * m1 + m0 / (2.0 * p.lam);
  double ut2 = 0.0;
  Vec5 out;
#pragma unroll
  for (int t = 0; t < NWP; ++t) out.v[t] = 0.0;
  out.v[0] = p.rho * m0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const double ut = p.U[d] - Un * n[d];
    ut2 += ut * ut;
    out.v[1 + d] = p.rho * (m1 * n[d] + m0 * ut);
  }
  out.v[D + 1] = 0.5 * p.rho * (m2 + m0 * (ut2 + (D - 1 + Kxi) / (2.0 * p.lam)));
  return out;
}

struct G5 {
  double g[5];
};

// Integrals over [0, dt] of c1..c5 (Eq. 34-35).  Closed forms for x = dt/tau
// >= 0.5; below, power series in x (evaluated by Horner), because the closed
// forms cancel:
//   G0 = dt sum_n (-x)^n/(n+1)!            G2 = dt x sum_j (-x)^j/(j+2)!
//   G1 = dt^2 sum_m (-1)^(m+1)(m+1) x^m/(m+2)!
//   G3 = dt^2 x sum_j>=0 (-1)^(j+1)(j+1) x^j/(j+3)!
//   G4 = dt^2 x sum_j>=0 (-1)^j x^j/(j+3)!
__device__ __forceinline__ G5 time_integrals(double dt, double tau) {
  G5 r;
  const double x = dt / tau;
  if (x >= 0.5) {
    const double em = -expm1(-x);
    const double E = exp(-x);
    r.g[0] = tau * em;
    r.g[1] = tau * (dt * E - tau * em);
    r.g[2] = dt - tau * em;
    r.g[3] = tau * (2.0 * tau * em - dt * (1.0 + E));
    r.g[4] = 0.5 * dt * dt - tau * dt + tau * tau * em;
    return r;
  }
  constexpr int NT = 24;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0;
  // 1/(n+1)!, 1/(n+2)!, 1/(n+3)! for n = NT-1 down to 0, built from 1/(NT+2)!
  double f1 = 1.0, f2 = 1.0, f3 = 1.0;
#pragma unroll
  for (int i = 2; i <= NT; ++i) f1 /= i;        // 1/NT!
  f2 = f1 / (NT + 1);                            // 1/(NT+1)!
  f3 = f2 / (NT + 2);                            // 1/(NT+2)!
#pragma unroll
  for (int n = NT - 1; n >= 0; --n) {
    const double sg = (n & 1) ? -1.0 : 1.0;
    s0 = s0 * x + sg * f1;
    s2 = s2 * x + sg * f2;
    s1 = s1 * x - sg * (n + 1) * f2;
    s3 = s3 * x - sg * (n + 1) * f3;
    s4 = s4 * x + sg * f3;
    f3 = f2;
    f2 = f1;
    f1 = f1 * (n + 1 > 1 ? n + 1 : 1);
  }
  r.g[0] = dt * s0;
  r.g[1] = dt * dt * s1;
  r.g[2] = dt * x * s2;
  r.g[3] = dt * dt * x * s3;
  r.g[4] = dt * dt * x * s4;
  return r;
}

}  // namespace

// ---------------------------------------------------------------------------
// Time step: one warp per cell, lanes over velocities.  The positive double
// dt_i is min-reduced through its bit pattern (positive doubles order like
// their unsigned 64-bit images).
// ---------------------------------------------------------------------------
// The largest outflow sum_f S_f max(u_k . n_f, 0) of a cell over the
// velocities, in two passes: FP32 sums find the maximum M32; the velocities
// whose FP32 sum is within 1e-4 of M32 (a bound far above the FP32 error of
// these sums of non-negative terms, so they include the FP64 maximiser) are
// summed again in FP64 in the face order of the reference definition.  This
// keeps the 3e9 (cell, velocity) pairs of the sphere workload off GB300's
// narrow FP64 pipe and gives the FP64 result.  One warp per cell, its faces
// (at most 32) staged in shared memory.
template <int D>
__global__ void __launch_bounds__(256) k_time_step(int64_t Nc, const int64_t* cf_off, const CellFace* cf,
                                                    const double* fnormal, const double* vol, const double* u,
                                                    const double* w, int64_t nv, unsigned long long* out_bits) {
  __shared__ double sn[8][32][3], sa[8][32];
  __shared__ float fn[8][32][3], fa[8][32];
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (i >= Nc) return;
  const int64_t e0 = cf_off[i];
  const int nf = int(cf_off[i + 1] - e0);
  if (lane < nf) {
    const CellFace& c = cf[e0 + lane];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      sn[wi][lane][d] = fnormal[c.face * 3 + d] * c.sign;
      fn[wi][lane][d] = float(sn[wi][lane][d]);
    }
    sa[wi][lane] = c.area;
    fa[wi][lane] = float(c.area);
  }
  __syncwarp();
  auto sum32 = [&](int64_t k) {
    float uk[3];
#pragma unroll
    for (int d = 0; d < D; ++d) uk[d] = float(u[k * D + d]);
    float s = 0.f;
    for (int e = 0; e < nf; ++e) {
      float un = 0.f;
#pragma unroll
      for (int d = 0; d < D; ++d) un = fmaf(uk[d], fn[wi][e][d], un);
      s = fmaf(fa[wi][e], fmaxf(un, 0.f), s);
    }
    return s;
  };
  float m32 = 0.f;
  for (int64_t k = lane; k < nv; k += 32)
    if (w[k] != 0.0) m32 = fmaxf(m32, sum32(k));
  for (int o = 16; o > 0; o >>= 1) m32 = fmaxf(m32, __shfl_xor_sync(0xffffffffu, m32, o));
  const float cut = m32 * (1.f - 1e-4f);
  double worst = 0.0;
  for (int64_t k = lane; k < nv; k += 32) {
    if (w[k] == 0.0 || sum32(k) < cut) continue;
    double s = 0.0;
    for (int e = 0; e < nf; ++e) {
      double un = 0.0;
#pragma unroll
      for (int d = 0; d < D; ++d) un += u[k * D + d] * sn[wi][e][d];
      if (un > 0.0) s += sa[wi][e] * un;
    }
    worst = fmax(worst, s);
  }
  for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  if (lane == 0 && worst > 0.0) {
    double v = vol[i] / worst;
    atomicMin(out_bits, (unsigned long long)__double_as_longlong(v));
  }
}

// ---------------------------------------------------------------------------
// Initial distribution: discrete reduced Maxwellians of W (h = H, b = K_xi/(2 lam) H);
// padded velocities (k >= nv) hold zero.  The per-cell factors (rho
// (lam/pi)^(D/2), lam, U, kappa) are formed once per cell in FP64; per value
// only the exponential remains (FP64 for FP64 storage, FP32 for FP32), so the
// 3e9-value initialisation of the sphere workload stays off GB300's narrow
// FP64 pipe.
// ---------------------------------------------------------------------------
struct InitRec {
  double pref, lam, U[3], kap;
};

template <int D>
__global__ void k_init_rec(int64_t Nc, Gas g, const double* W, InitRec* rec) {
  const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= Nc) return;
  bool ok;
  const Prim p = prim_of<D>(load5<D>(W + c * NWP), g.K, ok);
  InitRec r;
  r.pref = p.rho * pow(p.lam / M_PI, 0.5 * D);
  r.lam = p.lam;
#pragma unroll
  for (int d = 0; d < 3; ++d) r.U[d] = p.U[d];
  r.kap = g.Kxi / (2.0 * p.lam);
  rec[c] = r;
}

// grid: x over cells (one warp each), y over velocity blocks
template <int D, typename T>
__global__ void k_init_f(int64_t Nc, int64_t M, int64_t nv, int NR, const InitRec* rec, const double* ux,
                         const double* uy, const double* uz, T* f) {
  const int64_t c = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= Nc) return;
  const InitRec r = rec[c];
  for (int64_t m = blockIdx.y; m < M; m += gridDim.y) {
  const int64_t k = m * BV + lane;
  T h = T(0), b = T(0);
  if (k < nv) {
    const double uu[3] = {ux[k], uy[k], uz[k]};
    double c2 = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) c2 += (uu[d] - r.U[d]) * (uu[d] - r.U[d]);
    if constexpr (sizeof(T) == 8) {
      h = T(r.pref * exp(-r.lam * c2));
      b = T(r.kap * double(h));
    } else {
      const float H = float(r.pref) * expf(float(-r.lam * c2));
      h = T(H);
      b = T(float(r.kap) * H);
    }
  }
  const size_t plane = size_t(M) * Nc * BV, at = size_t(m) * Nc * BV + size_t(c) * BV + lane;
  f[at] = h;
  if (NR == 2) f[plane + at] = b;
  }
}

// ---------------------------------------------------------------------------
// Cell stage (Algorithm 5: primitive variables, relaxation time, and the
// limited least-squares gradient of W), one thread per cell, FP64.
// ---------------------------------------------------------------------------
template <int D>
__global__ void k_cell(int64_t Nc, Gas g, const double* W, const double* q, const int64_t* cf_off,
                       const CellFace* cf, const double* vol, const BCDev* bcs, CellPrim* cp, double* gW,
                       int* status) {
  constexpr int nw = D + 2;
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= Nc) return;
  const Vec5 Wi = load5<D>(W + i * NWP);
  bool ok;
  Prim p = prim_of<D>(Wi, g.K, ok);
  if (!ok) {
    atomicOr(status, 1);
    p.rho = 1.0;
    p.lam = 1.0;
  }
  CellPrim c;
  c.rho = p.rho;
#pragma unroll
  for (int d = 0; d < 3; ++d) c.U[d] = p.U[d];
  c.lam = p.lam;
  c.tau = tau_of(p, g);
#pragma unroll
  for (int d = 0; d < 3; ++d) c.q[d] = (d < D && g.shakhov) ? q[i * 3 + d] : 0.0;
  c.pad = 0.0;
  cp[i] = c;

  double grad[nw][D], wmax[nw], wmin[nw];
#pragma unroll
  for (int t = 0; t < nw; ++t) {
    wmax[t] = wmin[t] = Wi.v[t];
#pragma unroll
    for (int d = 0; d < D; ++d) grad[t][d] = 0.0;
  }
  const int64_t e0 = cf_off[i], e1 = cf_off[i + 1];
  for (int64_t e = e0; e < e1; ++e) {
    const CellFace& s = cf[e];
    if (s.bc_type == 1) continue;  // walls are not in the least-squares stencil
    const Vec5 Wo = s.other >= 0 ? load5<D>(W + s.other * NWP) : ghost_state<D>(bcs[-s.other - 1], Wi, g.K);
#pragma unroll
    for (int t = 0; t < nw; ++t) {
      const double dw = Wo.v[t] - Wi.v[t];
#pragma unroll
      for (int d = 0; d < D; ++d) grad[t][d] += s.w[d] * dw;
      wmax[t] = fmax(wmax[t], Wo.v[t]);
      wmin[t] = fmin(wmin[t], Wo.v[t]);
    }
  }
  const double h = pow(vol[i], 1.0 / D), eps2 = pow(g.venkat_K * h, 3.0);
  double phi[nw];
#pragma unroll
  for (int t = 0; t < nw; ++t) phi[t] = 1.0;
  for (int64_t e = e0; e < e1; ++e) {
    const CellFace& s = cf[e];
#pragma unroll
    for (int t = 0; t < nw; ++t) {
      double d2 = 0.0;
#pragma unroll
      for (int d = 0; d < D; ++d) d2 += grad[t][d] * s.r[d];
      const double mag = fmax(fabs(wmax[t]), fabs(wmin[t]));
      phi[t] = fmin(phi[t], limiter_fn(g.limiter, d2, wmax[t] - Wi.v[t], wmin[t] - Wi.v[t], eps2 * mag * mag));
    }
  }
#pragma unroll
  for (int t = 0; t < nw; ++t)
#pragma unroll
    for (int d = 0; d < 3; ++d) gW[(i * NWP + t) * 3 + d] = d < D ? fmax(phi[t], 0.0) * grad[t][d < D ? d : 0] : 0.0;
}

// ---------------------------------------------------------------------------
// Face stage (Algorithm 5: interface equilibrium, slopes, time integrals),
// one thread per face, FP64 arithmetic, record stored in the sweep precision.
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ Vec5 slope_column(const double* gW, int64_t c, int d) {
  Vec5 r;
#pragma unroll
  for (int t = 0; t < NWP; ++t) r.v[t] = t < D + 2 ? gW[(c * NWP + t) * 3 + d] : 0.0;
  return r;
}

// Coefficients of the equilibrium bracket of one reduced distribution as a
// cubic in c = u - U0 (FacePoly): with u = c + U0,
//   G2 mu (1 + s (c.q)(2 lambda |c|^2 - delta))
// + G3 [mu (sum_d u_d a_d0 + sum_de a_de u_d u_e) + (mu |u|^2 + nu)/2 sum_d a_d,D+1 u_d]
// + G4 [mu (A_0 + sum_e A_e u_e + A_D+1 |u|^2 / 2) + A_D+1 nu / 2]
// (h: mu = 1, nu = kappa, delta = D + 2; b: mu = kappa, nu = <xi^4>, delta = D),
// i.e. G2 (g0 + g0+) + G3 u.grad g0 + G4 d_t g0 divided by g0 (Eq. 32-33,
// 18-19).  Expanded in FP64.
template <int D>
__device__ __forceinline__ void cub_add(double (&p)[NPoly<D>::value], int e0, int e1, int e2, double v) {
  p[mono_index<D>(e0, e1, e2)] += v;
}

template <int D>
__device__ __forceinline__ void bracket_cubic(double (&p)[NPoly<D>::value], const G5& G, const Vec5 (&a)[D],
                                              const Vec5& A, const Prim& p0, double s, const double (&qf)[3],
                                              double mu, double nu, double delta) {
  constexpr int NP = NPoly<D>::value;
#pragma unroll
  for (int t = 0; t < NP; ++t) p[t] = 0.0;
  const double G2 = G.g[2], G3 = G.g[3], G4 = G.g[4], lam = p0.lam;
  double U2 = 0.0, aU = 0.0, quadU = 0.0, alpha = 0.0, AU = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    U2 += p0.U[d] * p0.U[d];
    aU += a[d].v[0] * p0.U[d];
    alpha += a[d].v[D + 1] * p0.U[d];
    AU += A.v[1 + d] * p0.U[d];
#pragma unroll
    for (int e = 0; e < D; ++e) quadU += a[d].v[1 + e] * p0.U[d] * p0.U[e];
  }
  // G2 term (with the Shakhov correction)
  cub_add<D>(p, 0, 0, 0, G2 * mu);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    cub_add<D>(p, d == 0, d == 1, d == 2, -delta * G2 * mu * s * qf[d]);
#pragma unroll
    for (int e = 0; e < D; ++e)
      cub_add<D>(p, (d == 0) + 2 * (e == 0), (d == 1) + 2 * (e == 1), (d == 2) + 2 * (e == 2),
                 2.0 * lam * G2 * mu * s * qf[d]);
  }
  // G3 term: sum_d u_d a_d0 + sum_de a_de u_d u_e
  cub_add<D>(p, 0, 0, 0, G3 * mu * (aU + quadU));
#pragma unroll
  for (int k = 0; k < D; ++k) {
    double lin = a[k].v[0];
#pragma unroll
    for (int e = 0; e < D; ++e) lin += a[k].v[1 + e] * p0.U[e] + a[e].v[1 + k] * p0.U[e];
    cub_add<D>(p, k == 0, k == 1, k == 2, G3 * mu * lin);
  }
#pragma unroll
  for (int d = 0; d < D; ++d)
#pragma unroll
    for (int e = 0; e < D; ++e)
      cub_add<D>(p, (d == 0) + (e == 0), (d == 1) + (e == 1), (d == 2) + (e == 2), G3 * mu * a[d].v[1 + e]);
  // G3 term: (mu |u|^2 + nu) / 2 sum_d a_d,D+1 u_d
  cub_add<D>(p, 0, 0, 0, 0.5 * G3 * (mu * U2 + nu) * alpha);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const double b = a[d].v[D + 1];
    cub_add<D>(p, d == 0, d == 1, d == 2, 0.5 * G3 * (mu * U2 + nu) * b + G3 * mu * alpha * p0.U[d]);
    cub_add<D>(p, 2 * (d == 0), 2 * (d == 1), 2 * (d == 2), 0.5 * G3 * mu * alpha);
#pragma unroll
    for (int e = 0; e < D; ++e) {
      cub_add<D>(p, (d == 0) + 2 * (e == 0), (d == 1) + 2 * (e == 1), (d == 2) + 2 * (e == 2), 0.5 * G3 * mu * b);
      cub_add<D>(p, (d == 0) + (e == 0), (d == 1) + (e == 1), (d == 2) + (e == 2), G3 * mu * p0.U[e] * b);
    }
  }
  // G4 term
  const double A0 = A.v[0], A4 = A.v[D + 1];
  cub_add<D>(p, 0, 0, 0, G4 * (mu * (A0 + AU + 0.5 * A4 * U2) + 0.5 * A4 * nu));
#pragma unroll
  for (int e = 0; e < D; ++e) {
    cub_add<D>(p, e == 0, e == 1, e == 2, G4 * mu * (A.v[1 + e] + A4 * p0.U[e]));
    cub_add<D>(p, 2 * (e == 0), 2 * (e == 1), 2 * (e == 2), 0.5 * G4 * mu * A4);
  }
}

template <int D, int NR, typename T>
__device__ __forceinline__ void store_face_poly(void* out, int64_t f, const Prim& p0, double rho_pref, double kappa,
                                                double G0, double G1, const double (&ph)[NPoly<D>::value],
                                                const double (&pb)[NPoly<D>::value]) {
  FacePoly<D, NR, T> P;
#pragma unroll
  for (int d = 0; d < 3; ++d) P.U[d] = T(p0.U[d]);
  P.lam = T(p0.lam);
  P.rho_pref = T(rho_pref);
  P.kappa = T(kappa);
  P.G0 = T(G0);
  P.G1 = T(G1);
#pragma unroll
  for (int t = 0; t < NPoly<D>::value; ++t) {
    P.P[0][t] = T(ph[t]);
    if (NR == 2) P.P[NR - 1][t] = T(pb[t]);
  }
  static_cast<FacePoly<D, NR, T>*>(out)[f] = P;
}

template <int D, typename T>
__global__ void k_face(int64_t Nf, Gas g, const double* W, const double* gW, const double* q,
                       const int64_t* fown, const int64_t* fnei, const double* fnormal, const double* fcent,
                       const double* fshift, const double* xc, const BCDev* bcs, FaceRec<T>* rec, void* poly) {
  constexpr int nw = D + 2;
  const int64_t f = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (f >= Nf) return;
  const int K = g.K;
  const int64_t o = fown[f], j = fnei[f];
  FaceRec<T> R;
#pragma unroll
  for (int t = 0; t < 5; ++t) {
    R.G[t] = T(0);
    R.A[t] = T(0);
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    R.U[d] = T(0);
    R.q[d] = T(0);
#pragma unroll
    for (int t = 0; t < 5; ++t) R.a[d][t] = T(0);
  }
  R.pad[0] = R.pad[1] = T(0);
  R.sq = T(0);
  R.xi4 = T(0);
  if (j < 0 && bcs[-j - 1].type == 1) {
    // diffuse wall: unit-density wall Maxwellian (Eq. 37)
    const BCDev& bc = bcs[-j - 1];
    const double lam = 1.0 / bc.T;
    R.rho_pref = T(pow(lam / M_PI, 0.5 * D));
    R.lam = T(lam);
#pragma unroll
    for (int d = 0; d < 3; ++d) R.U[d] = T(bc.u[d]);
    R.kappa = T(g.Kxi / (2.0 * lam));
    if (rec) rec[f] = R;
    if (poly) {
      constexpr int NP = NPoly<D>::value;
      double zero[NP];
#pragma unroll
      for (int t = 0; t < NP; ++t) zero[t] = 0.0;
      Prim pw;
      pw.rho = 1.0;
      pw.lam = lam;
#pragma unroll
      for (int d = 0; d < 3; ++d) pw.U[d] = bc.u[d];
      const double rp = pow(lam / M_PI, 0.5 * D), kp = g.Kxi / (2.0 * lam);
      if (g.NR == 2) store_face_poly<D, 2, T>(poly, f, pw, rp, kp, 0.0, 0.0, zero, zero);
      else store_face_poly<D, 1, T>(poly, f, pw, rp, kp, 0.0, 0.0, zero, zero);
    }
    return;
  }
  double n[3], rl[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    n[d] = fnormal[f * 3 + d];
    rl[d] = fcent[f * 3 + d] - xc[o * 3 + d];
  }
  const Vec5 Wo = load5<D>(W + o * NWP);
  bool ok;
  // reconstructed conservative states on both sides (Eq. 31 for W, reading R8)
  Vec5 Wl = Wo;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const Vec5 s = slope_column<D>(gW, o, d);
#pragma unroll
    for (int t = 0; t < nw; ++t) Wl.v[t] += s.v[t] * rl[d];
  }
  Prim pl = prim_of<D>(Wl, K, ok);
  if (!ok) {
    Wl = Wo;
    pl = prim_of<D>(Wl, K, ok);
  }
  Vec5 Wr;
  Vec5 dW0[D];
  double qr[3] = {0.0, 0.0, 0.0};
  if (j >= 0) {
    const Vec5 Wj = load5<D>(W + j * NWP);
    Wr = Wj;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const double rr = fcent[f * 3 + d] - fshift[f * 3 + d] - xc[j * 3 + d];
      const Vec5 s = slope_column<D>(gW, j, d);
#pragma unroll
      for (int t = 0; t < nw; ++t) Wr.v[t] += s.v[t] * rr;
    }
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const Vec5 so = slope_column<D>(gW, o, d), sj = slope_column<D>(gW, j, d);
#pragma unroll
      for (int t = 0; t < NWP; ++t) dW0[d].v[t] = 0.5 * (so.v[t] + sj.v[t]);
    }
#pragma unroll
    for (int d = 0; d < D; ++d) qr[d] = q[j * 3 + d];
  } else {
    Wr = ghost_state<D>(bcs[-j - 1], Wo, K);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const Vec5 so = slope_column<D>(gW, o, d);
#pragma unroll
      for (int t = 0; t < NWP; ++t) dW0[d].v[t] = 0.5 * so.v[t];
    }
  }
  Prim pr = prim_of<D>(Wr, K, ok);
  if (!ok && j >= 0) {
    Wr = load5<D>(W + j * NWP);
    pr = prim_of<D>(Wr, K, ok);
  }
  // interface state from the two half-range moments (reading R6)
  const Vec5 hl = half_space_moments<D>(pl, K, n, +1.0);
  const Vec5 hr = half_space_moments<D>(pr, K, n, -1.0);
  Vec5 W0;
#pragma unroll
  for (int t = 0; t < NWP; ++t) W0.v[t] = hl.v[t] + hr.v[t];
  const Prim p0 = prim_of<D>(W0, K, ok);
  // spatial slopes a_d and the time slope A from compatibility (Eq. 7, 32)
  Vec5 rhsA;
#pragma unroll
  for (int t = 0; t < NWP; ++t) rhsA.v[t] = 0.0;
  Vec5 av[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const Vec5 a = maxwell_solve<D>(p0, K, dW0[d]);
    av[d] = a;
#pragma unroll
    for (int t = 0; t < nw; ++t) R.a[d][t] = T(a.v[t]);
    const Vec5 dF = euler_flux_derivative<D>(p0, K, d, W0, dW0[d]);
#pragma unroll
    for (int t = 0; t < NWP; ++t) rhsA.v[t] -= dF.v[t];
  }
  const Vec5 A = maxwell_solve<D>(p0, K, rhsA);
#pragma unroll
  for (int t = 0; t < nw; ++t) R.A[t] = T(A.v[t]);
  double tau0 = tau_of(p0, g);
  if (g.shock_fix) {
    const double PL = pl.rho / (2.0 * pl.lam), PR = pr.rho / (2.0 * pr.lam);
    tau0 += g.dt * fabs(PL - PR) / (PL + PR);
  }
  const G5 G = time_integrals(g.dt, tau0);
#pragma unroll
  for (int t = 0; t < 5; ++t) R.G[t] = T(G.g[t]);
  R.rho_pref = T(p0.rho * pow(p0.lam / M_PI, 0.5 * D));
  R.lam = T(p0.lam);
#pragma unroll
  for (int d = 0; d < D; ++d) R.U[d] = T(p0.U[d]);
  if (g.shakhov) {
    R.sq = T(4.0 * (1.0 - g.Pr) * p0.lam * p0.lam / (5.0 * p0.rho));
#pragma unroll
    for (int d = 0; d < D; ++d) R.q[d] = T(0.5 * (q[o * 3 + d] + qr[d]));
  }
  R.kappa = T(g.Kxi / (2.0 * p0.lam));
  R.xi4 = T(g.Kxi * (g.Kxi + 2.0) / (4.0 * p0.lam * p0.lam));
  if (rec) rec[f] = R;
  if (poly) {
    constexpr int NP = NPoly<D>::value;
    const double s = g.shakhov ? 4.0 * (1.0 - g.Pr) * p0.lam * p0.lam / (5.0 * p0.rho) : 0.0;
    double qf[3] = {0.0, 0.0, 0.0};
    if (g.shakhov)
#pragma unroll
      for (int d = 0; d < D; ++d) qf[d] = 0.5 * (q[o * 3 + d] + qr[d]);
    const double kappa = g.Kxi / (2.0 * p0.lam);
    const double xi4 = g.Kxi * (g.Kxi + 2.0) / (4.0 * p0.lam * p0.lam);
    double ph[NP], pb[NP];
    bracket_cubic<D>(ph, G, av, A, p0, s, qf, 1.0, kappa, double(D + 2));
    const double rp = p0.rho * pow(p0.lam / M_PI, 0.5 * D);
    if (g.NR == 2) {
      bracket_cubic<D>(pb, G, av, A, p0, s, qf, kappa, xi4, double(D));
      store_face_poly<D, 2, T>(poly, f, p0, rp, kappa, G.g[0], G.g[1], ph, pb);
    } else {
      store_face_poly<D, 1, T>(poly, f, p0, rp, kappa, G.g[0], G.g[1], ph, ph);
    }
  }
}

// ---------------------------------------------------------------------------
// Surface quantities of the diffuse-wall faces from the moments of their
// time-integrated flux F (FP64; Sec. 2.1: the macroscopic surface quantities
// follow from the moments of the wall flux).  With n the face normal out of
// the gas and P = F_momentum / dt: p_w = P.n, tau_w = P - p_w n,
// q_w = (F_energy - U_w.F_momentum) / dt; optionally the coefficients against
// a free stream (rho, U, T): C_p = (p_w - rho T/2) / (rho|U|^2/2),
// C_t = |tau_w| / (rho|U|^2/2), C_h = q_w / (rho|U|^3/2).  One thread per wall face.
// ---------------------------------------------------------------------------
__global__ void k_surface(int64_t nwall, int D, double dt, const int64_t* walls, const double* Facc, int facc_stride,
                          const double* fnormal, const int64_t* fnei, const BCDev* bcs, const double* freestream,
                          double* vals, double* coef) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= nwall) return;
  const int64_t f = walls[i];
  const double* F = Facc + f * facc_stride;
  const BCDev& bc = bcs[-fnei[f] - 1];
  double P[3] = {0.0, 0.0, 0.0}, pn = 0.0, work = 0.0;
  for (int d = 0; d < D; ++d) {
    P[d] = F[1 + d] / dt;
    pn += P[d] * fnormal[f * 3 + d];
    work += bc.u[d] * F[1 + d];
  }
  double* v = vals + i * (D + 2);
  v[0] = pn;
  double t2 = 0.0;
  for (int d = 0; d < D; ++d) {
    v[1 + d] = P[d] - pn * fnormal[f * 3 + d];
    t2 += v[1 + d] * v[1 + d];
  }
  v[D + 1] = (F[D + 1] - work) / dt;
  if (freestream) {
    double U2 = 0.0;
    for (int d = 0; d < D; ++d) U2 += freestream[1 + d] * freestream[1 + d];
    const double rho = freestream[0], T = freestream[D + 1], qdyn = 0.5 * rho * U2;
    coef[i * 3 + 0] = (pn - 0.5 * rho * T) / qdyn;
    coef[i * 3 + 1] = sqrt(t2) / qdyn;
    coef[i * 3 + 2] = v[D + 1] / (qdyn * sqrt(U2));
  }
}

void launch_surface(cudaStream_t s, int64_t nwall, int D, double dt, const int64_t* walls, const double* Facc,
                    int facc_stride, const double* fnormal, const int64_t* fnei, const BCDev* bcs,
                    const double* freestream, double* vals, double* coef) {
  if (nwall <= 0) return;
  k_surface<<<unsigned((nwall + 127) / 128), 128, 0, s>>>(nwall, D, dt, walls, Facc, facc_stride, fnormal, fnei, bcs,
                                                   freestream, vals, coef);
}

// ---------------------------------------------------------------------------
// Moments of the stored distribution: heat flux (Eq. 13) about U of W, and
// the discrete conservative moments (Eq. 10, 21).  One warp per cell.
// ---------------------------------------------------------------------------
template <int D, typename T>
__global__ void k_moments(int64_t Nc, int64_t M, Gas g, const T* f, const double* W, const double* ux,
                          const double* uy, const double* uz, const double* w, const Vel4<float>* v4,
                          double* q_out, double* Wf_out) {
  const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= Nc) return;
  bool ok;
  const Prim p = prim_of<D>(load5<D>(W + i * NWP), g.K, ok);
  if constexpr (sizeof(T) == 4) {
    if (v4) {
      // FP32 values: FP32 terms summed as float pairs, one FP64 reduction per cell
      float U[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) U[d] = float(p.U[d]);
      const float2 z = make_float2(0.f, 0.f);
      float2 qa[3] = {z, z, z}, ma[3] = {z, z, z}, m0 = z, mE = z;
      const size_t plane = size_t(M) * Nc * BV;
      for (int64_t m = 0; m < M; ++m) {
        const Vel4<float> vq = v4[m * BV + lane];
        const size_t at = size_t(m) * Nc * BV + size_t(i) * BV + lane;
        const float h = float(f[at]);
        const float b = g.NR == 2 ? float(f[plane + at]) : 0.f;
        const float uu[3] = {vq.x, vq.y, vq.z};
        float c[3], c2 = 0.f, u2 = 0.f;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          c[d] = uu[d] - U[d];
          c2 = fmaf(c[d], c[d], c2);
          u2 = fmaf(uu[d], uu[d], u2);
        }
        const float e = 0.5f * vq.w * fmaf(c2, h, b);
#pragma unroll
        for (int d = 0; d < D; ++d) qa[d] = pair_add(qa[d], c[d] * e);
        if (Wf_out) {
          const float wh = vq.w * h;
          m0 = pair_add(m0, wh);
#pragma unroll
          for (int d = 0; d < D; ++d) ma[d] = pair_add(ma[d], wh * uu[d]);
          mE = pair_add(mE, 0.5f * vq.w * fmaf(u2, h, b));
        }
      }
      double qd[3], md[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        qd[d] = d < D ? warp_sum(double(qa[d].x) + double(qa[d].y)) : 0.0;
        md[d] = (Wf_out && d < D) ? warp_sum(double(ma[d].x) + double(ma[d].y)) : 0.0;
      }
      const double m0d = Wf_out ? warp_sum(double(m0.x) + double(m0.y)) : 0.0;
      const double mEd = Wf_out ? warp_sum(double(mE.x) + double(mE.y)) : 0.0;
      if (lane == 0) {
#pragma unroll
        for (int d = 0; d < 3; ++d) q_out[i * 3 + d] = qd[d];
        if (Wf_out) {
          Wf_out[i * NWP + 0] = m0d;
#pragma unroll
          for (int d = 0; d < D; ++d) Wf_out[i * NWP + 1 + d] = md[d];
          Wf_out[i * NWP + D + 1] = mEd;
        }
      }
      return;
    }
  }
  double qa[3] = {0.0, 0.0, 0.0}, ma[3] = {0.0, 0.0, 0.0}, m0 = 0.0, mE = 0.0;
  const size_t plane = size_t(M) * Nc * BV;
  for (int64_t m = 0; m < M; ++m) {
    const int64_t k = m * BV + lane;
    const double h = double(f[size_t(m) * Nc * BV + size_t(i) * BV + lane]);
    const double b = g.NR == 2 ? double(f[plane + size_t(m) * Nc * BV + size_t(i) * BV + lane]) : 0.0;
    const double uu[3] = {ux[k], uy[k], uz[k]}, wk = w[k];
    double c2 = 0.0, u2 = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      c2 += (uu[d] - p.U[d]) * (uu[d] - p.U[d]);
      u2 += uu[d] * uu[d];
    }
#pragma unroll
    for (int d = 0; d < D; ++d) {
      qa[d] += 0.5 * wk * (uu[d] - p.U[d]) * (c2 * h + b);
      ma[d] += wk * uu[d] * h;
    }
    m0 += wk * h;
    mE += 0.5 * wk * (u2 * h + b);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m0 += __shfl_xor_sync(0xffffffffu, m0, o);
    mE += __shfl_xor_sync(0xffffffffu, mE, o);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      qa[d] += __shfl_xor_sync(0xffffffffu, qa[d], o);
      ma[d] += __shfl_xor_sync(0xffffffffu, ma[d], o);
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int d = 0; d < 3; ++d) q_out[i * 3 + d] = d < D ? qa[d] : 0.0;
    if (Wf_out) {
      Wf_out[i * NWP + 0] = m0;
#pragma unroll
      for (int d = 0; d < D; ++d) Wf_out[i * NWP + 1 + d] = ma[d];
      Wf_out[i * NWP + D + 1] = mE;
    }
  }
}

// Gather of selected rows as FP64: out[n][NR][nv] for cells sel[] (renumbered).
template <typename T>
__global__ void k_gather_f(int64_t Nc, int64_t M, int NR, int64_t nv, const T* f, const int64_t* sel, int64_t n,
                           double* out) {
  int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= n * NR * nv) return;
  int64_t k = idx % nv, r = (idx / nv) % NR, s = idx / (nv * NR);
  int64_t c = sel[s], m = k / BV, lane = k % BV;
  out[idx] = double(f[(size_t(r) * M + m) * Nc * BV + size_t(c) * BV + lane]);
}

// ---------------------------------------------------------------------------
// Thirteen-moment fields of each cell: rho, U, T of W, the deviatoric stress
// sigma_ij = sum_k w c_i c_j h - p delta_ij (p = rho/(2 lambda)) in the order
// xx, xy, (xz), yy, (yz), zz, and the heat flux (Eq. 13), about U of W.
// One warp per cell, FP64 sums.
// ---------------------------------------------------------------------------
template <int D, typename T>
__global__ void k_moments13(int64_t Nc, int64_t M, Gas g, const T* f, const double* W, const double* ux,
                            const double* uy, const double* uz, const double* w, double* out) {
  constexpr int NS = D * (D + 1) / 2, N13 = 2 * D + 2 + NS;
  const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= Nc) return;
  bool ok;
  const Prim p = prim_of<D>(load5<D>(W + i * NWP), g.K, ok);
  double P[NS], q[D];
#pragma unroll
  for (int s = 0; s < NS; ++s) P[s] = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) q[d] = 0.0;
  const size_t plane = size_t(M) * Nc * BV;
  for (int64_t m = 0; m < M; ++m) {
    const int64_t k = m * BV + lane;
    const double h = double(f[size_t(m) * Nc * BV + size_t(i) * BV + lane]);
    const double b = g.NR == 2 ? double(f[plane + size_t(m) * Nc * BV + size_t(i) * BV + lane]) : 0.0;
    const double uu[3] = {ux[k], uy[k], uz[k]}, wk = w[k];
    double c[3] = {0.0, 0.0, 0.0}, c2 = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      c[d] = uu[d] - p.U[d];
      c2 += c[d] * c[d];
    }
    int s = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      q[a] += 0.5 * wk * c[a] * (c2 * h + b);
#pragma unroll
      for (int e = a; e < D; ++e) P[s++] += wk * c[a] * c[e] * h;
    }
  }
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) P[s] += __shfl_xor_sync(0xffffffffu, P[s], o);
#pragma unroll
  for (int d = 0; d < D; ++d)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q[d] += __shfl_xor_sync(0xffffffffu, q[d], o);
  if (lane == 0) {
    double* o = out + i * N13;
    const double pr = p.rho / (2.0 * p.lam);
    o[0] = p.rho;
#pragma unroll
    for (int d = 0; d < D; ++d) o[1 + d] = p.U[d];
    o[D + 1] = 1.0 / p.lam;
    int s = 0;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int e = a; e < D; ++e) {
        o[D + 2 + s] = P[s] - (a == e ? pr : 0.0);
        ++s;
      }
#pragma unroll
    for (int d = 0; d < D; ++d) o[D + 2 + NS + d] = q[d];
  }
}

// Chapman-Enskog (Grad 13-moment) distribution of given fields, reduced over
// xi (N = D + K_xi = K + 3 degrees of freedom):
//   h = H [1 + 2 lam^2/rho sigma_ij c_i c_j + 4 lam^2/((N+2) rho) (q.c)(2 lam |c|^2 - (D+2))]
//   b = kappa H [1 + 2 lam^2/rho sigma_ij c_i c_j + 4 lam^2/((N+2) rho) (q.c)(2 lam |c|^2 - D)]
// with H the Maxwellian of (rho, U, lam = 1/T); FP64, one thread per value.
template <int D, typename T>
__global__ void k_init_ce(int64_t Nc, int64_t M, int64_t nv, Gas g, const double* fields, const double* ux,
                          const double* uy, const double* uz, T* f) {
  // grid: x over cells (one warp each), y over velocity blocks; the per-cell
  // factors are formed once per thread
  constexpr int NS = D * (D + 1) / 2, N13 = 2 * D + 2 + NS;
  const int64_t c = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= Nc) return;
  const double* x = fields + c * N13;
  const double rho = x[0], lam = 1.0 / x[D + 1];
  const double pref = rho * pow(lam / M_PI, 0.5 * D);
  // the K_xi components of xi carry -tr(sigma) / K_xi each (trace-free
  // stress over all degrees of freedom); reduced over xi that gives the
  // constants th (in h) and tb (in b)
  double tr = 0.0;
#pragma unroll
  for (int a = 0, s2 = 0; a < D; ++a)
#pragma unroll
    for (int e = a; e < D; ++e, ++s2)
      if (a == e) tr += x[D + 2 + s2];
  const double a2 = 2.0 * lam * lam / rho, a3 = 4.0 * lam * lam / ((g.K + 5.0) * rho);
  const double th = -lam * tr / rho, tb = g.Kxi > 0 ? -lam * (g.Kxi + 2.0) * tr / (g.Kxi * rho) : 0.0;
  const double kap = g.Kxi / (2.0 * lam);
  const size_t plane = size_t(M) * Nc * BV;
  for (int64_t m = blockIdx.y; m < M; m += gridDim.y) {
    const int64_t k = m * BV + lane;
    double h = 0.0, b = 0.0;
    if (k < nv) {
      const double uu[3] = {ux[k], uy[k], uz[k]};
      double cc[3] = {0.0, 0.0, 0.0}, c2 = 0.0, qc = 0.0, scc = 0.0;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        cc[d] = uu[d] - x[1 + d];
        c2 += cc[d] * cc[d];
        qc += x[D + 2 + NS + d] * cc[d];
      }
      int s = 0;
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int e = a; e < D; ++e) scc += (a == e ? 1.0 : 2.0) * x[D + 2 + s++] * cc[a] * cc[e];
      const double H = pref * exp(-lam * c2);
      h = H * (1.0 + a2 * scc + th + a3 * qc * (2.0 * lam * c2 - (D + 2)));
      b = kap * H * (1.0 + a2 * scc + tb + a3 * qc * (2.0 * lam * c2 - D));
    }
    const size_t at = size_t(m) * Nc * BV + size_t(c) * BV + lane;
    f[at] = T(h);
    if (g.NR == 2) f[plane + at] = T(b);
  }
}

// Scatter of a full FP64 state in[NR][Nc_orig][nv] (original order) into f.
template <typename T>
__global__ void k_scatter_f(int64_t Nc, int64_t M, int NR, int64_t nv, const double* in, const int64_t* old_of_new,
                            T* f) {
  int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= int64_t(NR) * M * Nc * BV) return;
  int lane = int(idx & 31);
  int64_t row = idx >> 5;
  int64_t c = row % Nc, m = (row / Nc) % M, r = row / (Nc * M);
  int64_t k = m * BV + lane;
  double v = k < nv ? in[(size_t(r) * Nc + old_of_new[c]) * nv + k] : 0.0;
  f[idx] = T(v);
}

__global__ void k_residual_finalize(int nw, int64_t Nc, const double* acc, double* res) {
  int t = threadIdx.x;
  if (t < nw) res[t] = sqrt(acc[t] / double(Nc));
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
static inline unsigned blocks_for(int64_t n, int threads) { return unsigned((n + threads - 1) / threads); }

void launch_time_step(cudaStream_t s, int64_t Nc, int D, const int64_t* cf_off, const CellFace* cf,
                      const double* fnormal, const double* vol, const double* u, const double* w, int64_t nv,
                      unsigned long long* out_bits) {
  const unsigned nb = blocks_for(Nc * 32, 256);
  if (D == 1) k_time_step<1><<<nb, 256, 0, s>>>(Nc, cf_off, cf, fnormal, vol, u, w, nv, out_bits);
  if (D == 2) k_time_step<2><<<nb, 256, 0, s>>>(Nc, cf_off, cf, fnormal, vol, u, w, nv, out_bits);
  if (D == 3) k_time_step<3><<<nb, 256, 0, s>>>(Nc, cf_off, cf, fnormal, vol, u, w, nv, out_bits);
}

template <typename T>
cudaError_t launch_init_f(cudaStream_t s, int64_t Nc, int64_t M, int64_t nv, const Gas& g, const double* W,
                          const double* ux, const double* uy, const double* uz, T* f) {
  InitRec* rec = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&rec), size_t(Nc) * sizeof(InitRec), s);
  if (e != cudaSuccess) return e;
  const unsigned nc = blocks_for(Nc, 128);
  if (g.D == 1) k_init_rec<1><<<nc, 128, 0, s>>>(Nc, g, W, rec);
  if (g.D == 2) k_init_rec<2><<<nc, 128, 0, s>>>(Nc, g, W, rec);
  if (g.D == 3) k_init_rec<3><<<nc, 128, 0, s>>>(Nc, g, W, rec);
  const dim3 grid(blocks_for(Nc * 32, 256), unsigned(std::min<int64_t>(M, 65535)));
  if (g.D == 1) k_init_f<1, T><<<grid, 256, 0, s>>>(Nc, M, nv, g.NR, rec, ux, uy, uz, f);
  if (g.D == 2) k_init_f<2, T><<<grid, 256, 0, s>>>(Nc, M, nv, g.NR, rec, ux, uy, uz, f);
  if (g.D == 3) k_init_f<3, T><<<grid, 256, 0, s>>>(Nc, M, nv, g.NR, rec, ux, uy, uz, f);
  e = cudaGetLastError();
  const cudaError_t e2 = cudaFreeAsync(rec, s);
  return e != cudaSuccess ? e : e2;
}

void launch_cell(cudaStream_t s, int64_t Nc, const Gas& g, const double* W, const double* q, const int64_t* cf_off,
                 const CellFace* cf, const double* vol, const BCDev* bcs, CellPrim* cp, double* gW, int* status) {
  const unsigned nb = blocks_for(Nc, 128);
  if (g.D == 1) k_cell<1><<<nb, 128, 0, s>>>(Nc, g, W, q, cf_off, cf, vol, bcs, cp, gW, status);
  if (g.D == 2) k_cell<2><<<nb, 128, 0, s>>>(Nc, g, W, q, cf_off, cf, vol, bcs, cp, gW, status);
  if (g.D == 3) k_cell<3><<<nb, 128, 0, s>>>(Nc, g, W, q, cf_off, cf, vol, bcs, cp, gW, status);
}

template <typename T>
void launch_face(cudaStream_t s, int64_t Nf, const Gas& g, const double* W, const double* gW, const double* q,
                 const int64_t* fown, const int64_t* fnei, const double* fnormal, const double* fcent,
                 const double* fshift, const double* xc, const BCDev* bcs, FaceRec<T>* rec, void* poly) {
  const unsigned nb = blocks_for(Nf, 128);
  if (g.D == 1) k_face<1, T><<<nb, 128, 0, s>>>(Nf, g, W, gW, q, fown, fnei, fnormal, fcent, fshift, xc, bcs, rec, poly);
  if (g.D == 2) k_face<2, T><<<nb, 128, 0, s>>>(Nf, g, W, gW, q, fown, fnei, fnormal, fcent, fshift, xc, bcs, rec, poly);
  if (g.D == 3) k_face<3, T><<<nb, 128, 0, s>>>(Nf, g, W, gW, q, fown, fnei, fnormal, fcent, fshift, xc, bcs, rec, poly);
}

template <typename T>
void launch_moments(cudaStream_t s, int64_t Nc, int64_t M, const Gas& g, const T* f, const double* W,
                    const double* ux, const double* uy, const double* uz, const double* w, double* q_out,
                    double* Wf_out, const void* vel4) {
  const unsigned nb = blocks_for(Nc * 32, 256);
  const Vel4<float>* v4 = sizeof(T) == 4 ? static_cast<const Vel4<float>*>(vel4) : nullptr;
  if (g.D == 1) k_moments<1, T><<<nb, 256, 0, s>>>(Nc, M, g, f, W, ux, uy, uz, w, v4, q_out, Wf_out);
  if (g.D == 2) k_moments<2, T><<<nb, 256, 0, s>>>(Nc, M, g, f, W, ux, uy, uz, w, v4, q_out, Wf_out);
  if (g.D == 3) k_moments<3, T><<<nb, 256, 0, s>>>(Nc, M, g, f, W, ux, uy, uz, w, v4, q_out, Wf_out);
}

template <typename T>
void launch_gather_f(cudaStream_t s, int64_t Nc, int64_t M, int NR, int64_t nv, const T* f, const int64_t* sel,
                     int64_t n, double* out) {
  if (n * NR * nv == 0) return;
  k_gather_f<T><<<blocks_for(n * NR * nv, 256), 256, 0, s>>>(Nc, M, NR, nv, f, sel, n, out);
}

template <typename T>
void launch_scatter_f(cudaStream_t s, int64_t Nc, int64_t M, int NR, int64_t nv, const double* in,
                      const int64_t* old_of_new, T* f) {
  k_scatter_f<T><<<blocks_for(int64_t(NR) * M * Nc * BV, 256), 256, 0, s>>>(Nc, M, NR, nv, in, old_of_new, f);
}

template <typename T>
void launch_moments13(cudaStream_t s, int64_t Nc, int64_t M, const Gas& g, const T* f, const double* W,
                      const double* ux, const double* uy, const double* uz, const double* w, double* out) {
  const unsigned nb = blocks_for(Nc * 32, 256);
  if (g.D == 1) k_moments13<1, T><<<nb, 256, 0, s>>>(Nc, M, g, f, W, ux, uy, uz, w, out);
  if (g.D == 2) k_moments13<2, T><<<nb, 256, 0, s>>>(Nc, M, g, f, W, ux, uy, uz, w, out);
  if (g.D == 3) k_moments13<3, T><<<nb, 256, 0, s>>>(Nc, M, g, f, W, ux, uy, uz, w, out);
}

template <typename T>
void launch_init_ce(cudaStream_t s, int64_t Nc, int64_t M, int64_t nv, const Gas& g, const double* fields,
                    const double* ux, const double* uy, const double* uz, T* f) {
  const dim3 grid(blocks_for(Nc * 32, 256), unsigned(std::min<int64_t>(M, 65535)));
  if (g.D == 1) k_init_ce<1, T><<<grid, 256, 0, s>>>(Nc, M, nv, g, fields, ux, uy, uz, f);
  if (g.D == 2) k_init_ce<2, T><<<grid, 256, 0, s>>>(Nc, M, nv, g, fields, ux, uy, uz, f);
  if (g.D == 3) k_init_ce<3, T><<<grid, 256, 0, s>>>(Nc, M, nv, g, fields, ux, uy, uz, f);
}

void launch_residual_finalize(cudaStream_t s, int nw, int64_t Nc, const double* acc, double* res) {
  k_residual_finalize<<<1, 32, 0, s>>>(nw, Nc, acc, res);
}

#define UGKS_INSTANTIATE(T)                                                                                      \
  template void launch_moments13<T>(cudaStream_t, int64_t, int64_t, const Gas&, const T*, const double*,         \
                                    const double*, const double*, const double*, const double*, double*);         \
  template void launch_init_ce<T>(cudaStream_t, int64_t, int64_t, int64_t, const Gas&, const double*,             \
                                  const double*, const double*, const double*, T*);                               \
  template cudaError_t launch_init_f<T>(cudaStream_t, int64_t, int64_t, int64_t, const Gas&, const double*,      \
                                        const double*, const double*, const double*, T*);                       \
  template void launch_face<T>(cudaStream_t, int64_t, const Gas&, const double*, const double*, const double*,   \
                               const int64_t*, const int64_t*, const double*, const double*, const double*,      \
                               const double*, const BCDev*, FaceRec<T>*, void*);                                 \
  template void launch_moments<T>(cudaStream_t, int64_t, int64_t, const Gas&, const T*, const double*,           \
                                  const double*, const double*, const double*, const double*, double*, double*,  \
                                  const void*);                                                                 \
  template void launch_gather_f<T>(cudaStream_t, int64_t, int64_t, int, int64_t, const T*, const int64_t*,       \
                                   int64_t, double*);                                                            \
  template void launch_scatter_f<T>(cudaStream_t, int64_t, int64_t, int, int64_t, const double*, const int64_t*, \
                                    T*);
UGKS_INSTANTIATE(float)
UGKS_INSTANTIATE(double)

}  // namespace ugks
