// Block-parallel velocity sweep of one UGKS time step (kernel templates;
// instantiated per precision in ugks_blocked_f32.cu / ugks_blocked_f64.cu).
//
// The velocity set is swept in blocks (Sec. 2.2.2, Eq. 48) of VB x 32
// points: lane L of a warp owns the velocities k = (m0 + j) * 32 + L,
// j = 0 .. VB-1.  For each block the three stages of Table B.1 run as three
// grid-wide kernels over the whole mesh, in stream order:
//   k_brecon   one warp per cell: limited least-squares gradient of h, b
//              (Eq. 31), then, for every face of the cell and every velocity
//              for which the cell is upwind, the free-transport part of the
//              interface distribution, c0 f(x_f) + c1 u.grad f (Eq. 33:
//              c0, c1 = the time integrals of c1, c2; at a wall the free
//              transport dt f - dt^2/2 u.grad f of Eq. 36)          [K2]
//   k_bflux    one warp per face: adds the equilibrium part (Eq. 32-35),
//              forms the micro flux u.n (...) in place, and adds its weighted
//              moments in FP64 to the face accumulator (Eq. 52, Algorithm 4)
//                                                                  [K1]
//   k_bstage1  one warp per cell: first-stage update (Eq. 41; Algorithm 1)
//                                                                  [K3]
// The only intermediate is one per-face buffer X [face][NR][VB][32]: each
// velocity's upwind cell writes its lane (the two cells of a face write
// complementary lanes), the flux kernel overwrites it with the flux.  It is
// rewritten by every block and stays mostly in L2.  After the last block:
//   k_bwall    wall density from non-penetration (Eq. 38)
//   k_bW       conservative update (Eq. 27) and the primitive record of W^{n+1}
//   k_bstage2  second stage (Eq. 42), in velocity chunks, and partial sums of
//              the heat flux of f^{n+1} (Eq. 13); k_bqsum adds the chunks.
// No kernel waits on another CTA and every face is evaluated once per block,
// so W is exactly conservative; no atomics are needed (each face belongs to
// one warp, the block kernels are stream-ordered, partial sums are added in
// a fixed order), so every result is bitwise reproducible.
#pragma once
#include <cmath>
#include <cstdint>

#include "ugks_device.cuh"
#include "ugks_internal.cuh"
#include "ugks_kernels.cuh"

namespace ugks {

constexpr int kBlockedThreads = 256;  // 8 warps per CTA in every blocked kernel
constexpr int kIncChunk = 4;          // incidences whose loads are issued together

template <int D, int NR, int VB, typename T>
struct BlockVel {
  T u[VB][3];
  T w[VB];   // quadrature weight, 0 for padding
  T u2[VB];
  bool real[VB];

  __device__ __forceinline__ void load(const BlockedArgs<T>& a, int64_t m0, int lane) {
#pragma unroll
    for (int j = 0; j < VB; ++j) {
      const int64_t k = (m0 + j) * BV + lane;
      const Vel4<T> q = a.vel[k];
      u[j][0] = q.x;
      u[j][1] = D > 1 ? q.y : T(0);
      u[j][2] = D > 2 ? q.z : T(0);
      real[j] = k < a.nv;
      w[j] = q.w;  // zero on padding
      T s = T(0);
#pragma unroll
      for (int d = 0; d < D; ++d) s += u[j][d] * u[j][d];
      u2[j] = s;
    }
  }
};

// Maxwellian (h, b) of a ghost state for an artificial boundary (far field:
// the prescribed state; outflow: the interior cell's own state).
template <int D, int NR, typename T>
__device__ __forceinline__ void ghost_state(const BlockedArgs<T>& a, int bc_index, int cell, T& rho, T& lam,
                                            T (&U)[3]) {
  const BCDev& bc = a.bcs[bc_index];
  if (bc.type == 3) {
    const CellPrim& p = a.cp[cell];
    rho = T(p.rho);
    lam = T(p.lam);
    U[0] = T(p.U[0]);
    U[1] = T(p.U[1]);
    U[2] = T(p.U[2]);
  } else {
    rho = T(bc.rho);
    lam = T(1.0 / bc.T);
    U[0] = T(bc.u[0]);
    U[1] = T(bc.u[1]);
    U[2] = T(bc.u[2]);
  }
}

// ---------------------------------------------------------------------------
// K2: limited least-squares gradient (Eq. 31) and the upwind free-transport
// part of every face of the cell.
// ---------------------------------------------------------------------------
template <int D, int NR, int VB, typename T>
__global__ void __launch_bounds__(kBlockedThreads) k_brecon(const BlockedArgs<T> a, const int64_t m0) {
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * (kBlockedThreads / 32) + (threadIdx.x >> 5);
  if (c >= a.Nc) return;
  const size_t sj = size_t(a.Nc) * BV, sr = size_t(a.M) * sj;
  const T* fb = a.f_cur + size_t(m0) * sj + lane;
  BlockVel<D, NR, VB, T> v;
  v.load(a, m0, lane);
  const int Kxi = a.g.Kxi;

  T fc[NR][VB], g[NR][VB][D], fmx[NR][VB], fmn[NR][VB];
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int j = 0; j < VB; ++j) {
      fc[r][j] = fb[r * sr + j * sj + size_t(c) * BV];
      fmx[r][j] = fmn[r][j] = fc[r][j];
#pragma unroll
      for (int d = 0; d < D; ++d) g[r][j][d] = T(0);
    }
  const int e0 = a.cf_off[c], e1 = a.cf_off[c + 1];
  // incidences in chunks of kIncChunk: all neighbour rows of a chunk are
  // requested before the first is used
  for (int eb = e0; eb < e1; eb += kIncChunk) {
    int other[kIncChunk], flags[kIncChunk], bcx[kIncChunk];
    T wd[kIncChunk][D], fo[kIncChunk][NR][VB];
#pragma unroll
    for (int i = 0; i < kIncChunk; ++i) {
      const bool on = eb + i < e1;
      const IncT<T>& in = a.inc[on ? eb + i : e0];
      other[i] = in.other;
      flags[i] = on ? in.flags : 1;  // past the end: skipped like a wall
      bcx[i] = in.bc;
#pragma unroll
      for (int d = 0; d < D; ++d) wd[i][d] = in.w[d];
    }
#pragma unroll
    for (int i = 0; i < kIncChunk; ++i)
      if (!(flags[i] & 1) && other[i] >= 0) {
        const size_t oc = size_t(other[i]) * BV;
#pragma unroll
        for (int r = 0; r < NR; ++r)
#pragma unroll
          for (int j = 0; j < VB; ++j) fo[i][r][j] = fb[r * sr + j * sj + oc];
      }
#pragma unroll
    for (int i = 0; i < kIncChunk; ++i) {
      if (flags[i] & 1) continue;  // walls: one-sided stencil
      if (other[i] < 0) {
        T rho, lam, U[3];
        ghost_state<D, NR, T>(a, bcx[i], c, rho, lam, U);
        const T pref = rho * maxwell_pref<D>(lam);
#pragma unroll
        for (int j = 0; j < VB; ++j) {
          T c2 = T(0);
#pragma unroll
          for (int d = 0; d < D; ++d) c2 += (v.u[j][d] - U[d]) * (v.u[j][d] - U[d]);
          const T H = v.real[j] ? pref * t_exp(-lam * c2) : T(0);
          fo[i][0][j] = H;
          if (NR == 2) fo[i][NR - 1][j] = T(Kxi) / (T(2) * lam) * H;
        }
      }
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int j = 0; j < VB; ++j) {
          const T df = fo[i][r][j] - fc[r][j];
#pragma unroll
          for (int d = 0; d < D; ++d) g[r][j][d] += wd[i][d] * df;
          fmx[r][j] = fmax(fmx[r][j], fo[i][r][j]);
          fmn[r][j] = fmin(fmn[r][j], fo[i][r][j]);
        }
    }
  }
  T phi[NR][VB];
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int j = 0; j < VB; ++j) phi[r][j] = T(1);
  const int limiter = a.g.limiter;
  if (limiter != 0) {
    const T eps2c = a.eps2[c];
    T eps2[NR][VB], dmx[NR][VB], dmn[NR][VB];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int j = 0; j < VB; ++j) {
        const T mag = fmax(fabs(fmx[r][j]), fabs(fmn[r][j]));
        eps2[r][j] = eps2c * mag * mag;  // Venkatakrishnan constant in the units of f
        dmx[r][j] = fmx[r][j] - fc[r][j];
        dmn[r][j] = fmn[r][j] - fc[r][j];
      }
    for (int e = e0; e < e1; ++e) {
      T rr[D];
#pragma unroll
      for (int d = 0; d < D; ++d) rr[d] = a.inc[e].r[d];
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int j = 0; j < VB; ++j) {
          T d2 = T(0);
#pragma unroll
          for (int d = 0; d < D; ++d) d2 += g[r][j][d] * rr[d];
          const T dp = d2 > T(0) ? dmx[r][j] : dmn[r][j];
          T ph;
          if (limiter == 2) {
            ph = d2 != T(0) ? fast_div(dp, d2) : T(1);
          } else {
            // (dp^2 + eps + 2 d2 dp) / (dp^2 + 2 d2^2 + dp d2 + eps); equals 1 at d2 = 0
            const T num = fma(dp, dp + T(2) * d2, eps2[r][j]);
            const T den = fma(dp + d2, dp, fma(T(2) * d2, d2, eps2[r][j]));
            ph = fast_div(num, den);
          }
          phi[r][j] = fmin(phi[r][j], ph);  // fmin ignores a NaN from 0/0 (then d2 = 0, phi stays)
        }
    }
  }
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int j = 0; j < VB; ++j) {
      const T p = fmin(fmax(phi[r][j], T(0)), T(1));
#pragma unroll
      for (int d = 0; d < D; ++d) g[r][j][d] *= p;
    }
  // free-transport part on every face for which this cell is upwind
  const T dt = T(a.g.dt);
  const T hdt2 = T(0.5 * a.g.dt * a.g.dt);
  for (int eb = e0; eb < e1; eb += kIncChunk) {
    int face[kIncChunk];
    bool wall[kIncChunk];
    T c0[kIncChunk], c1[kIncChunk];
#pragma unroll
    for (int i = 0; i < kIncChunk; ++i) {
      const IncT<T>& in = a.inc[eb + i < e1 ? eb + i : e0];
      face[i] = in.face;
      wall[i] = in.flags & 1;
    }
#pragma unroll
    for (int i = 0; i < kIncChunk; ++i) {
      if (wall[i]) {
        c0[i] = dt;
        c1[i] = -hdt2;
      } else {
        c0[i] = a.fr[face[i]].G[0];
        c1[i] = a.fr[face[i]].G[1];
      }
    }
#pragma unroll
    for (int i = 0; i < kIncChunk; ++i) {
      if (eb + i >= e1) break;
      const IncT<T>& in = a.inc[eb + i];
      T n[D], rr[D];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        n[d] = in.n[d];
        rr[d] = in.r[d];
      }
      T* Xf = a.X + size_t(face[i]) * (NR * VB * BV) + lane;
#pragma unroll
      for (int j = 0; j < VB; ++j) {
        T un = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) un += v.u[j][d] * n[d];
        if (un > T(0)) {
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            T ff = fc[r][j], ug = T(0);
#pragma unroll
            for (int d = 0; d < D; ++d) {
              ff += g[r][j][d] * rr[d];
              ug += v.u[j][d] * g[r][j][d];
            }
            Xf[(r * VB + j) * BV] = c0[i] * ff + c1[i] * ug;
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// K1: micro fluxes of one velocity block and their FP64 moments (Eq. 29,
// 32-38, 52).  X holds the upwind free-transport part on entry and the flux
// on exit.
// ---------------------------------------------------------------------------
template <int D, int NR, int VB, typename T>
__global__ void __launch_bounds__(kBlockedThreads) k_bflux(const BlockedArgs<T> a, const int64_t m0,
                                                           const int first) {
  constexpr int NW = D + 2;
  const int lane = threadIdx.x & 31;
  const int f = blockIdx.x * (kBlockedThreads / 32) + (threadIdx.x >> 5);
  if (f >= a.Nf) return;
  const int idx8 = sum8_index(lane);
  const bool writer = (lane & 3) == 0 && idx8 < NW;
  double* Fa = a.Facc + size_t(f) * FACC_W;
  const double fold = (writer && !first) ? Fa[idx8] : 0.0;  // issued early, used at the end
  const T dt = T(a.g.dt);
  BlockVel<D, NR, VB, T> v;
  v.load(a, m0, lane);
  const FaceGeom<T> fg = a.fg[f];
  const FaceRec<T> R = a.fr[f];
  T* Xf = a.X + size_t(f) * (NR * VB * BV) + lane;
  T m_in[NWP], m_out[NWP];  // moments of the block, conservative variable order (energy at D + 1)
#pragma unroll
  for (int t = 0; t < NWP; ++t) m_in[t] = m_out[t] = T(0);

  if (fg.bc_type == 1) {
    // diffuse wall (Eq. 36-38): free transport on the incoming side; the
    // re-emitted half is the unit-density wall Maxwellian, scaled by rho_w
    // once all blocks are summed.
    const double fold_out = (writer && !first) ? Fa[5 + idx8] : 0.0;
#pragma unroll
    for (int j = 0; j < VB; ++j) {
      T un = T(0);
#pragma unroll
      for (int d = 0; d < D; ++d) un += v.u[j][d] * fg.n[d];
      T phi_h = T(0), phi_b = T(0), out_h = T(0);
      if (un > T(0)) {
        phi_h = un * Xf[(0 * VB + j) * BV];
        if (NR == 2) phi_b = un * Xf[((NR - 1) * VB + j) * BV];
      } else if (un < T(0)) {
        T c2 = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) c2 += (v.u[j][d] - R.U[d]) * (v.u[j][d] - R.U[d]);
        out_h = un * dt * R.rho_pref * t_exp(-R.lam * c2);
      }
      Xf[(0 * VB + j) * BV] = phi_h;
      if (NR == 2) Xf[((NR - 1) * VB + j) * BV] = phi_b;
      const T wph = v.w[j] * phi_h, wpo = v.w[j] * out_h;
      m_in[0] += wph;
      m_out[0] += wpo;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        m_in[1 + d] += wph * v.u[j][d];
        m_out[1 + d] += wpo * v.u[j][d];
      }
      m_in[D + 1] += T(0.5) * v.w[j] * (v.u2[j] * phi_h + phi_b);
      m_out[D + 1] += T(0.5) * v.w[j] * (v.u2[j] * out_h + R.kappa * out_h);
    }
    const T sin = warp_sum8<T>(m_in[0], m_in[1], m_in[2], m_in[3], m_in[4], T(0), T(0), T(0), lane);
    const T sout = warp_sum8<T>(m_out[0], m_out[1], m_out[2], m_out[3], m_out[4], T(0), T(0), T(0), lane);
    if (writer) {
      Fa[idx8] = fold + double(sin);
      Fa[5 + idx8] = fold_out + double(sout);
    }
    return;
  }

  const bool ghost = fg.nei < 0;
  T gr = T(0), gl = T(0), gU[3] = {T(0), T(0), T(0)}, gk = T(0);
  if (ghost) {
    // ghost side of an artificial boundary: Maxwellian of the ghost state, no slope
    T rho, lam;
    ghost_state<D, NR, T>(a, int(-fg.nei - 1), int(fg.own), rho, lam, gU);
    gr = rho * maxwell_pref<D>(lam);
    gl = lam;
    gk = T(a.g.Kxi) / (T(2) * lam);
  }
#pragma unroll
  for (int j = 0; j < VB; ++j) {
    T un = T(0);
#pragma unroll
    for (int d = 0; d < D; ++d) un += v.u[j][d] * fg.n[d];
    T phi_h = T(0), phi_b = T(0);
    if (un != T(0)) {
      T tr[NR];
      if (un > T(0) || !ghost) {
#pragma unroll
        for (int r = 0; r < NR; ++r) tr[r] = Xf[(r * VB + j) * BV];
      } else {
        T c2 = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) c2 += (v.u[j][d] - gU[d]) * (v.u[j][d] - gU[d]);
        const T H = gr * t_exp(-gl * c2);
        tr[0] = R.G[0] * H;
        if (NR == 2) tr[NR - 1] = R.G[0] * (gk * H);
      }
      // equilibrium part: G2 (g0 + g0+) + G3 u.grad g0 + G4 d_t g0 (Eq. 32-33)
      T c2 = T(0), cq = T(0);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const T cd = v.u[j][d] - R.U[d];
        c2 += cd * cd;
        cq += cd * R.q[d];
      }
      const T H0 = R.rho_pref * t_exp(-R.lam * c2);
      const T sq = R.sq * cq;
      const T twolc2 = T(2) * R.lam * c2;
      const T h0 = H0 * (T(1) + sq * (twolc2 - T(2 + D)));
      T ugH = T(0), ugB = T(0);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        T poly = R.a[d][0] + T(0.5) * R.a[d][D + 1] * v.u2[j];
#pragma unroll
        for (int e = 0; e < D; ++e) poly += R.a[d][1 + e] * v.u[j][e];
        ugH += v.u[j][d] * (poly + T(0.5) * R.a[d][D + 1] * R.kappa);
        if (NR == 2) ugB += v.u[j][d] * (poly * R.kappa + T(0.5) * R.a[d][D + 1] * R.xi4);
      }
      T pA = R.A[0] + T(0.5) * R.A[D + 1] * v.u2[j];
#pragma unroll
      for (int e = 0; e < D; ++e) pA += R.A[1 + e] * v.u[j][e];
      const T dtH = pA + T(0.5) * R.A[D + 1] * R.kappa;
      phi_h = un * (tr[0] + R.G[2] * h0 + H0 * (R.G[3] * ugH + R.G[4] * dtH));
      if (NR == 2) {
        const T b0 = H0 * R.kappa * (T(1) + sq * (twolc2 - T(D)));
        const T dtB = pA * R.kappa + T(0.5) * R.A[D + 1] * R.xi4;
        phi_b = un * (tr[NR - 1] + R.G[2] * b0 + H0 * (R.G[3] * ugB + R.G[4] * dtB));
      }
    }
    Xf[(0 * VB + j) * BV] = phi_h;
    if (NR == 2) Xf[((NR - 1) * VB + j) * BV] = phi_b;
    const T wph = v.w[j] * phi_h;
    m_in[0] += wph;
#pragma unroll
    for (int d = 0; d < D; ++d) m_in[1 + d] += wph * v.u[j][d];
    m_in[D + 1] += T(0.5) * v.w[j] * (v.u2[j] * phi_h + phi_b);
  }
  // value index t of the reduction is conservative variable t (energy at D + 1)
  const T sm = warp_sum8<T>(m_in[0], m_in[1], m_in[2], m_in[3], m_in[4], T(0), T(0), T(0), lane);
  if (writer) Fa[idx8] = fold + double(sm);
}

// ---------------------------------------------------------------------------
// K3: first-stage update of one velocity block (Eq. 41; Algorithm 1).
// ---------------------------------------------------------------------------
template <int D, int NR, int VB, typename T>
__global__ void __launch_bounds__(kBlockedThreads) k_bstage1(const BlockedArgs<T> a, const int64_t m0) {
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * (kBlockedThreads / 32) + (threadIdx.x >> 5);
  if (c >= a.Nc) return;
  const size_t sj = size_t(a.Nc) * BV, sr = size_t(a.M) * sj;
  const size_t base = size_t(m0) * sj + size_t(c) * BV + lane;
  BlockVel<D, NR, VB, T> v;
  v.load(a, m0, lane);
  const T dt = T(a.g.dt);
  const CellPrim& p = a.cp[c];
  const T rho = T(p.rho), lam = T(p.lam), beta0 = dt / (T(2) * T(p.tau));
  const T pref = rho * maxwell_pref<D>(lam);
  const T s0 = a.g.shakhov ? T(4.0 * (1.0 - a.g.Pr)) * lam * lam / (T(5) * rho) : T(0);
  const T kap = T(a.g.Kxi) / (T(2) * lam);
  T Uc[3], qc[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    Uc[d] = T(p.U[d]);
    qc[d] = T(p.q[d]);
  }
  T flux[NR][VB];
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int j = 0; j < VB; ++j) flux[r][j] = T(0);
  const int e0 = a.cf_off[c], e1 = a.cf_off[c + 1];
  for (int eb = e0; eb < e1; eb += kIncChunk) {
    int face[kIncChunk];
    T sa[kIncChunk], P[kIncChunk][NR][VB];
#pragma unroll
    for (int i = 0; i < kIncChunk; ++i) {
      const bool on = eb + i < e1;
      const IncT<T>& in = a.inc[on ? eb + i : e0];
      face[i] = in.face;
      sa[i] = on ? in.sarea : T(0);
    }
#pragma unroll
    for (int i = 0; i < kIncChunk; ++i) {
      const T* Xf = a.X + size_t(face[i]) * (NR * VB * BV) + lane;
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int j = 0; j < VB; ++j) P[i][r][j] = Xf[(r * VB + j) * BV];
    }
#pragma unroll
    for (int i = 0; i < kIncChunk; ++i)
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int j = 0; j < VB; ++j) flux[r][j] += sa[i] * P[i][r][j];
  }
  const T inv_vol = T(1.0 / a.vol[c]);
#pragma unroll
  for (int j = 0; j < VB; ++j) {
    T c2 = T(0), cq = T(0);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const T cd = v.u[j][d] - Uc[d];
      c2 += cd * cd;
      cq += cd * qc[d];
    }
    const T H = pref * t_exp(-lam * c2);
    const T s = s0 * cq;
    T fp[NR];
    fp[0] = H * (T(1) + s * (T(2) * lam * c2 - T(2 + D)));
    if (NR == 2) fp[NR - 1] = kap * H * (T(1) + s * (T(2) * lam * c2 - T(D)));
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const size_t idx = base + r * sr + j * sj;
      const T f = a.f_cur[idx];
      const T ft = f - flux[r][j] * inv_vol + beta0 * (fp[r] - f);
      a.f_next[idx] = v.real[j] ? ft : T(0);
    }
  }
}

// ---------------------------------------------------------------------------
// Wall density from non-penetration (Eq. 38) and the completed wall moments.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_bwall(const BlockedArgs<T> a) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= a.Nf || a.fg[f].bc_type != 1) return;
  double* F = a.Facc + size_t(f) * FACC_W;
  const int NW = a.g.D + 2;
  const double rw = F[5] != 0.0 ? -F[0] / F[5] : 0.0;
  for (int t = 0; t < NW; ++t) F[t] += rw * F[5 + t];
  F[10] = rw;
}

// ---------------------------------------------------------------------------
// Conservative update (Eq. 27), residual sums and the primitive record of
// W^{n+1} (with the lagged heat flux of f^n for the second stage).
// ---------------------------------------------------------------------------
template <int D, typename T>
__global__ void __launch_bounds__(kBlockedThreads) k_bW(const BlockedArgs<T> a) {
  constexpr int NW = D + 2;
  __shared__ double s_res[kBlockedThreads / 32][NWP];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double res[NWP] = {0, 0, 0, 0, 0};
  if (c < a.Nc) {
    double acc[NWP] = {0, 0, 0, 0, 0};
    for (int e = a.cf_off[c]; e < a.cf_off[c + 1]; ++e) {
      const double sa = double(a.inc[e].sarea);
      const double* F = a.Facc + size_t(a.inc[e].face) * FACC_W;
#pragma unroll
      for (int t = 0; t < NW; ++t) acc[t] += sa * F[t];
    }
    const double iv = 1.0 / a.vol[c];
    double Wn[NWP];
#pragma unroll
    for (int t = 0; t < NW; ++t) {
      const double w0 = a.W_cur[size_t(c) * NWP + t];
      Wn[t] = w0 - acc[t] * iv;
      a.W_next[size_t(c) * NWP + t] = Wn[t];
      res[t] = (Wn[t] - w0) * (Wn[t] - w0);
    }
    CellPrim pn;
    double u2 = 0.0;
    pn.rho = Wn[0];
#pragma unroll
    for (int d = 0; d < 3; ++d) pn.U[d] = d < D ? Wn[1 + (d < D ? d : 0)] / Wn[0] : 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) u2 += pn.U[d] * pn.U[d];
    const double ein = Wn[D + 1] - 0.5 * Wn[0] * u2;
    pn.lam = (a.g.K + 3) * Wn[0] / (4.0 * ein);
    const bool ok = (pn.rho > 0.0) && (ein > 0.0) && isfinite(pn.lam) && isfinite(u2);
    if (!ok) {
      atomicOr(a.status, 1);
      pn.rho = 1.0;
      pn.lam = 1.0;
    }
    pn.tau = a.g.mu_ref * pow(1.0 / pn.lam, a.g.omega) * 2.0 * pn.lam / pn.rho;
#pragma unroll
    for (int d = 0; d < 3; ++d) pn.q[d] = a.cp[c].q[d];  // lagged heat flux in stage 2
    pn.pad = 0.0;
    a.cp_next[c] = pn;
  }
#pragma unroll
  for (int t = 0; t < NW; ++t) res[t] = warp_sum(res[t]);
  if (lane == 0)
#pragma unroll
    for (int t = 0; t < NW; ++t) s_res[warp][t] = res[t];
  __syncthreads();
  if (threadIdx.x < NW) {
    double sum = 0.0;
    for (int w_ = 0; w_ < kBlockedThreads / 32; ++w_) sum += s_res[w_][threadIdx.x];
    atomicAdd(a.res_acc + threadIdx.x, sum);
  }
}

// ---------------------------------------------------------------------------
// Second stage (Eq. 42) of one cell over one chunk of velocity blocks, with
// the outgoing wall flux rho_w g_w (known only after the sweep), and the
// chunk's partial sums of the heat flux of f^{n+1} (Eq. 13).  Four blocks are
// loaded before any is updated (memory-level parallelism); per-lane FP32
// partial sums of q are flushed to FP64 every 32 blocks and reduced over the
// warp once.
// ---------------------------------------------------------------------------
template <int D, int NR, typename T>
__device__ __forceinline__ void stage2_block(const BlockedArgs<T>& a, int c, int e0, int e1, bool has_wall, int64_t m,
                                             int lane, const Vel4<T>& vq, T (&ft)[NR], const T (&Uc)[3], const T (&qc)[3], T pref, T lam,
                                             T s0, T kap, T beta1, T inv1, T iv, T* fc, size_t sr, size_t sj,
                                             T (&qp)[3]) {
  const T dt = T(a.g.dt);
  const int64_t k = m * BV + lane;
  T u[3];
  u[0] = vq.x;
  u[1] = D > 1 ? vq.y : T(0);
  u[2] = D > 2 ? vq.z : T(0);
  const bool real_v = k < a.nv;
  if (has_wall) {
    for (int e = e0; e < e1; ++e) {
      if (!(a.inc[e].flags & 1)) continue;
      const int fidx = a.inc[e].face;
      const FaceGeom<T>& fg = a.fg[fidx];
      const FaceRec<T>& R = a.fr[fidx];
      T un = T(0), c2 = T(0);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        un += u[d] * fg.n[d];
        c2 += (u[d] - R.U[d]) * (u[d] - R.U[d]);
      }
      if (un < T(0)) {
        const T rw = T(a.Facc[size_t(fidx) * FACC_W + 10]);
        const T out = un * dt * rw * R.rho_pref * t_exp(-R.lam * c2);
        const T area = a.inc[e].sarea;  // walls have owner cells only: +area
        ft[0] -= area * iv * out;
        if (NR == 2) ft[NR - 1] -= area * iv * R.kappa * out;
      }
    }
  }
  T cc[3], c2 = T(0), cq = T(0);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    cc[d] = u[d] - Uc[d];
    c2 += cc[d] * cc[d];
    cq += cc[d] * qc[d];
  }
  const T H = pref * t_exp(-lam * c2);
  const T s = s0 * cq;
  T f1[NR];
  f1[0] = (ft[0] + beta1 * H * (T(1) + s * (T(2) * lam * c2 - T(2 + D)))) * inv1;
  if (NR == 2) f1[NR - 1] = (ft[NR - 1] + beta1 * kap * H * (T(1) + s * (T(2) * lam * c2 - T(D)))) * inv1;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    if (!real_v) f1[r] = T(0);
    fc[r * sr + m * sj] = f1[r];
  }
  const T wq = T(0.5) * vq.w;  // zero on padding
  const T e_ = wq * (c2 * f1[0] + (NR == 2 ? f1[NR - 1] : T(0)));
#pragma unroll
  for (int d = 0; d < D; ++d) qp[d] += cc[d] * e_;
}

template <int D, int NR, typename T>
__global__ void __launch_bounds__(kBlockedThreads) k_bstage2(const BlockedArgs<T> a) {
  constexpr int UNR = 8;
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * (kBlockedThreads / 32) + (threadIdx.x >> 5);
  if (c >= a.Nc) return;
  const int chunk = blockIdx.y;
  const int64_t per = (a.M + a.nchunk - 1) / a.nchunk;
  const int64_t mb = int64_t(chunk) * per;
  const int64_t me = mb + per < a.M ? mb + per : a.M;
  const size_t sj = size_t(a.Nc) * BV, sr = size_t(a.M) * sj;
  T* fc = a.f_next + size_t(c) * BV + lane;
  const T dt = T(a.g.dt);
  const CellPrim& p = a.cp_next[c];
  const T rho = T(p.rho), lam = T(p.lam), beta1 = dt / (T(2) * T(p.tau));
  const T inv1 = T(1) / (T(1) + beta1);
  const T pref = rho * maxwell_pref<D>(lam);
  const T s0 = a.g.shakhov ? T(4.0 * (1.0 - a.g.Pr)) * lam * lam / (T(5) * rho) : T(0);
  const T kap = T(a.g.Kxi) / (T(2) * lam);
  const T iv = T(1.0 / a.vol[c]);
  T Uc[3], qc[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    Uc[d] = T(p.U[d]);
    qc[d] = T(p.q[d]);
  }
  const int e0 = a.cf_off[c], e1 = a.cf_off[c + 1];
  bool has_wall = false;
  for (int e = e0; e < e1; ++e) has_wall |= (a.inc[e].flags & 1) != 0;
  double qd[3] = {0.0, 0.0, 0.0};
  T qp[3] = {T(0), T(0), T(0)};
  int since_flush = 0;
  int64_t m = mb;
  for (; m + UNR <= me; m += UNR) {
    T ft[UNR][NR];
    Vel4<T> vq[UNR];
#pragma unroll
    for (int i = 0; i < UNR; ++i) {
#pragma unroll
      for (int r = 0; r < NR; ++r) ft[i][r] = fc[r * sr + (m + i) * sj];
      vq[i] = a.vel[(m + i) * BV + lane];
    }
#pragma unroll
    for (int i = 0; i < UNR; ++i)
      stage2_block<D, NR, T>(a, c, e0, e1, has_wall, m + i, lane, vq[i], ft[i], Uc, qc, pref, lam, s0, kap, beta1,
                             inv1, iv, fc, sr, sj, qp);
    since_flush += UNR;
    if (since_flush >= 32) {
#pragma unroll
      for (int d = 0; d < D; ++d) {
        qd[d] += double(qp[d]);
        qp[d] = T(0);
      }
      since_flush = 0;
    }
  }
  for (; m < me; ++m) {
    T ft[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) ft[r] = fc[r * sr + m * sj];
    const Vel4<T> vq = a.vel[m * BV + lane];
    stage2_block<D, NR, T>(a, c, e0, e1, has_wall, m, lane, vq, ft, Uc, qc, pref, lam, s0, kap, beta1, inv1, iv, fc,
                           sr, sj, qp);
  }
#pragma unroll
  for (int d = 0; d < D; ++d) qd[d] = warp_sum(qd[d] + double(qp[d]));
  double* qo = a.qpart + (size_t(chunk) * a.Nc + c) * 3;
  if (lane < 3) qo[lane] = lane < D ? (lane == 0 ? qd[0] : lane == 1 ? qd[D > 1 ? 1 : 0] : qd[D > 2 ? 2 : 0]) : 0.0;
}

// Heat flux of f^{n+1}: the chunks' partial sums added in chunk order.
template <typename T>
__global__ void k_bqsum(const BlockedArgs<T> a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.Nc * 3) return;
  double q = 0.0;
  for (int ch = 0; ch < a.nchunk; ++ch) q += a.qpart[size_t(ch) * a.Nc * 3 + i];
  a.q_next[i] = q;
}

// ---------------------------------------------------------------------------
// Launchers (dispatch on dimension, reduced distributions and VB).
// ---------------------------------------------------------------------------
inline unsigned blocked_warp_grid(int64_t n) {
  return unsigned((n + kBlockedThreads / 32 - 1) / (kBlockedThreads / 32));
}

#define UGKS_BLOCKED_DISPATCH(KERNEL, GRID, ...)                                                         \
  do {                                                                                                   \
    const int D_ = a.g.D, NR_ = a.g.NR;                                                                  \
    if (D_ == 1 && NR_ == 2 && vb == 1) KERNEL<1, 2, 1, T><<<GRID, kBlockedThreads, 0, s>>>(__VA_ARGS__); \
    else if (D_ == 1 && NR_ == 2 && vb == 2) KERNEL<1, 2, 2, T><<<GRID, kBlockedThreads, 0, s>>>(__VA_ARGS__); \
    else if (D_ == 1 && NR_ == 2 && vb == 4) KERNEL<1, 2, 4, T><<<GRID, kBlockedThreads, 0, s>>>(__VA_ARGS__); \
    else if (D_ == 2 && NR_ == 2 && vb == 1) KERNEL<2, 2, 1, T><<<GRID, kBlockedThreads, 0, s>>>(__VA_ARGS__); \
    else if (D_ == 2 && NR_ == 2 && vb == 2) KERNEL<2, 2, 2, T><<<GRID, kBlockedThreads, 0, s>>>(__VA_ARGS__); \
    else if (D_ == 2 && NR_ == 2 && vb == 4) KERNEL<2, 2, 4, T><<<GRID, kBlockedThreads, 0, s>>>(__VA_ARGS__); \
    else if (D_ == 3 && NR_ == 1 && vb == 1) KERNEL<3, 1, 1, T><<<GRID, kBlockedThreads, 0, s>>>(__VA_ARGS__); \
    else if (D_ == 3 && NR_ == 1 && vb == 2) KERNEL<3, 1, 2, T><<<GRID, kBlockedThreads, 0, s>>>(__VA_ARGS__); \
    else if (D_ == 3 && NR_ == 1 && vb == 4) KERNEL<3, 1, 4, T><<<GRID, kBlockedThreads, 0, s>>>(__VA_ARGS__); \
    else if (D_ == 3 && NR_ == 2 && vb == 1) KERNEL<3, 2, 1, T><<<GRID, kBlockedThreads, 0, s>>>(__VA_ARGS__); \
    else if (D_ == 3 && NR_ == 2 && vb == 2) KERNEL<3, 2, 2, T><<<GRID, kBlockedThreads, 0, s>>>(__VA_ARGS__); \
    else if (D_ == 3 && NR_ == 2 && vb == 4) KERNEL<3, 2, 4, T><<<GRID, kBlockedThreads, 0, s>>>(__VA_ARGS__); \
    else return cudaErrorInvalidValue;                                                                   \
  } while (0)

template <typename T>
cudaError_t launch_brecon(cudaStream_t s, const BlockedArgs<T>& a, int64_t m0, int vb) {
  UGKS_BLOCKED_DISPATCH(k_brecon, blocked_warp_grid(a.Nc), a, m0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bflux(cudaStream_t s, const BlockedArgs<T>& a, int64_t m0, int vb, int first) {
  UGKS_BLOCKED_DISPATCH(k_bflux, blocked_warp_grid(a.Nf), a, m0, first);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bstage1(cudaStream_t s, const BlockedArgs<T>& a, int64_t m0, int vb) {
  UGKS_BLOCKED_DISPATCH(k_bstage1, blocked_warp_grid(a.Nc), a, m0);
  return cudaGetLastError();
}

#undef UGKS_BLOCKED_DISPATCH

template <typename T>
cudaError_t launch_bconserve(cudaStream_t s, const BlockedArgs<T>& a) {
  k_bwall<T><<<unsigned((a.Nf + 255) / 256), 256, 0, s>>>(a);
  const unsigned nb = unsigned((a.Nc + kBlockedThreads - 1) / kBlockedThreads);
  if (a.g.D == 1) k_bW<1, T><<<nb, kBlockedThreads, 0, s>>>(a);
  else if (a.g.D == 2) k_bW<2, T><<<nb, kBlockedThreads, 0, s>>>(a);
  else if (a.g.D == 3) k_bW<3, T><<<nb, kBlockedThreads, 0, s>>>(a);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bstage2(cudaStream_t s, const BlockedArgs<T>& a) {
  const dim3 grid(blocked_warp_grid(a.Nc), unsigned(a.nchunk));
  const int D = a.g.D, NR = a.g.NR;
  if (D == 1 && NR == 2) k_bstage2<1, 2, T><<<grid, kBlockedThreads, 0, s>>>(a);
  else if (D == 2 && NR == 2) k_bstage2<2, 2, T><<<grid, kBlockedThreads, 0, s>>>(a);
  else if (D == 3 && NR == 1) k_bstage2<3, 1, T><<<grid, kBlockedThreads, 0, s>>>(a);
  else if (D == 3 && NR == 2) k_bstage2<3, 2, T><<<grid, kBlockedThreads, 0, s>>>(a);
  else return cudaErrorInvalidValue;
  k_bqsum<T><<<unsigned((int64_t(a.Nc) * 3 + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

#define UGKS_INSTANTIATE_BLOCKED(T)                                                                  \
  template cudaError_t launch_brecon<T>(cudaStream_t, const BlockedArgs<T>&, int64_t, int);          \
  template cudaError_t launch_bflux<T>(cudaStream_t, const BlockedArgs<T>&, int64_t, int, int);     \
  template cudaError_t launch_bstage1<T>(cudaStream_t, const BlockedArgs<T>&, int64_t, int);        \
  template cudaError_t launch_bconserve<T>(cudaStream_t, const BlockedArgs<T>&);                     \
  template cudaError_t launch_bstage2<T>(cudaStream_t, const BlockedArgs<T>&);

}  // namespace ugks
