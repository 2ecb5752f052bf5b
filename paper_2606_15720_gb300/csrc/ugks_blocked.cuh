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
// complementary lanes; the owner also writes the lanes with u.n = 0, so every
// lane of an interior face is written once per block), the flux kernel
// overwrites it with the flux.  It is
// rewritten by every block and stays mostly in L2.  After the last block:
//   k_bwall    face accumulators to FP64 (FP32 sweeps: float pairs) and the
//              wall density from non-penetration (Eq. 38)
//   k_bW       conservative update (Eq. 27) and the primitive record of W^{n+1}
//   k_bstage2  second stage (Eq. 42), in velocity chunks, and partial sums of
//              the heat flux of f^{n+1} (Eq. 13); k_bqsum adds the chunks.
// No kernel waits on another CTA and every face is evaluated once per block,
// so W is exactly conservative; no atomics are needed (each face belongs to
// one warp, the block kernels are stream-ordered, partial sums are added in
// a fixed order), so every result is bitwise reproducible.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <type_traits>

#include "ugks_bulk.cuh"
#include "ugks_device.cuh"
#include "ugks_internal.cuh"
#include "ugks_kernels.cuh"
#include "ugks_store.cuh"

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

// Cubic in c (coefficients in mono_index order) by nested Horner: 3, 9 or 19 FMA.
template <int D, typename T>
__device__ __forceinline__ T horner_cubic(const T (&p)[NPoly<D>::value], T c0, T c1, T c2) {
  if constexpr (D == 1) {
    return fma(c0, fma(c0, fma(c0, p[3], p[2]), p[1]), p[0]);
  } else if constexpr (D == 2) {
    const T x0 = fma(c1, p[7], fma(c0, p[6], p[3]));
    const T x1 = fma(c1, p[8], p[4]);
    const T y0 = fma(c1, x1, fma(c0, x0, p[1]));
    const T y1 = fma(c1, fma(c1, p[9], p[5]), p[2]);
    return fma(c1, y1, fma(c0, y0, p[0]));
  } else {
    const T x0 = fma(c2, p[12], fma(c1, p[11], fma(c0, p[10], p[4])));
    const T x1 = fma(c2, p[14], fma(c1, p[13], p[5]));
    const T x2 = fma(c2, p[15], p[6]);
    const T y0 = fma(c2, x2, fma(c1, x1, fma(c0, x0, p[1])));
    const T z0 = fma(c2, p[17], fma(c1, p[16], p[7]));
    const T z1 = fma(c2, p[18], p[8]);
    const T y1 = fma(c2, z1, fma(c1, z0, p[2]));
    const T y2 = fma(c2, fma(c2, p[19], p[9]), p[3]);
    return fma(c2, y2, fma(c1, y1, fma(c0, y0, p[0])));
  }
}

// Equilibrium record of one cell from its FP64 primitive record.
template <int D, typename T>
__device__ __forceinline__ CellEq<T> make_cell_eq(const Gas& g, const CellPrim& p, double vol) {
  CellEq<T> e;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    e.U[d] = T(p.U[d]);
    e.q[d] = T(p.q[d]);
  }
  e.lam = T(p.lam);
  e.pref = T(p.rho * pow(p.lam / M_PI, 0.5 * D));
  e.s0 = g.shakhov ? T(4.0 * (1.0 - g.Pr) * p.lam * p.lam / (5.0 * p.rho)) : T(0);
  e.kap = T(g.Kxi / (2.0 * p.lam));
  e.beta = T(g.dt / (2.0 * p.tau));
  e.inv_vol = T(1.0 / vol);
  return e;
}

template <int D, typename T>
__global__ void k_bcelleq(const BlockedArgs<T> a) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.Nc) return;
  a.ceq0[c] = make_cell_eq<D, T>(a.g, a.cp[c], a.vol[c]);
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
  T ug[NR][VB];  // u . (limited gradient), the same on every face
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int j = 0; j < VB; ++j) {
      const T p = fmin(fmax(phi[r][j], T(0)), T(1));
      ug[r][j] = T(0);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        g[r][j][d] *= p;
        ug[r][j] += v.u[j][d] * g[r][j][d];
      }
    }
  const FacePoly<D, NR, T>* FP = static_cast<const FacePoly<D, NR, T>*>(a.fpoly);
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
        c0[i] = FP[face[i]].G0;
        c1[i] = FP[face[i]].G1;
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
      const bool owner = in.sarea > T(0);
#pragma unroll
      for (int j = 0; j < VB; ++j) {
        T un = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) un += v.u[j][d] * n[d];
        // upwind side; u.n = 0 (padding included) written by the owner, so
        // that every lane of an interior face is written once per block
        if (un > T(0) || (un == T(0) && owner)) {
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            T ff = fc[r][j];
#pragma unroll
            for (int d = 0; d < D; ++d) ff += g[r][j][d] * rr[d];
            Xf[(r * VB + j) * BV] = c0[i] * ff + c1[i] * ug[r][j];
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// K1: micro fluxes of one velocity block and their FP64 moments (Eq. 29,
// 32-38, 52).  X holds the upwind free-transport part on entry and the flux
// on exit.  The kernel is persistent: each warp walks faces f, f + stride,
// ... and stages the next face's records (FacePoly, FaceGeom), its X rows and
// its accumulators into shared memory with cp.async while it computes the
// current face, so the loads of one face overlap the arithmetic of the
// previous one.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = unsigned(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Tensor grids (a row of 32 velocities is one line along the fastest axis,
// the lane axis): with c = u - U0 split into its lane component c0 and its
// row components, the equilibrium part of a face factors as
//   g0(u) P_r(c) = [rho_pref exp(-lam |c_row|^2)] exp(-lam c0^2) sum_a c0^a Q_{r,a}(c_row),
// Q_{r,a} the polynomial of the coefficients of c0^a (degree <= 3 - a in the
// row components).  Per face, one lane per row evaluates that row's factors
// and publishes them in shared memory; every lane then needs one exponential
// per face and three FMA per velocity for the cubic.  The flux moments
// factor the same way: sums over the lane's rows with the row weight, times
// the lane's weight and velocity once per face.
template <int NR, typename T>
struct __align__(16) RowFac {
  T Q[NR][4];     // row polynomials times rho_pref exp(-lam |c_row|^2)
  T un;           // row part of u . n
  T w;            // row weight factor
  T wu1, wu2;     // w u_1, w u_2 (row components of u)
  T wusq;         // w |u_row|^2
  T pad[(4 - (4 * NR + 5) % 4) % 4];
};

// Q_a(c1, c2) of one face polynomial (coefficients in mono_index order).
template <int D, typename T>
__device__ __forceinline__ void row_polys(const T (&p)[NPoly<D>::value], T c1, T c2, T (&Q)[4]) {
#pragma unroll
  for (int a = 0; a <= 3; ++a) {
    if constexpr (D == 1) {
      Q[a] = p[a];
    } else if constexpr (D == 2) {
      T q = p[mono_index<2>(a, 3 - a, 0)];
#pragma unroll
      for (int e1 = 2 - a; e1 >= 0; --e1) q = fma(q, c1, p[mono_index<2>(a, e1, 0)]);
      Q[a] = q;
    } else {
      T q = T(0);
#pragma unroll
      for (int e1 = 3 - a; e1 >= 0; --e1) {
        T in = p[mono_index<3>(a, e1, 3 - a - e1)];
#pragma unroll
        for (int e2 = 2 - a - e1; e2 >= 0; --e2) in = fma(in, c2, p[mono_index<3>(a, e1, e2)]);
        q = e1 == 3 - a ? in : fma(q, c1, in);
      }
      Q[a] = q;
    }
  }
}

// Shared-memory stage of one face: [FacePoly][FaceGeom][X rows][accumulators].
template <int D, int NR, int VB, typename T>
struct FluxStage {
  static constexpr int SP = int(sizeof(FacePoly<D, NR, T>));
  static constexpr int SG = int(sizeof(FaceGeom<T>));
  static constexpr int SX = NR * VB * BV * int(sizeof(T));
  static constexpr int SF = FACC_W * int(sizeof(double));
  static constexpr int BYTES = SP + SG + SX + SF;
  static_assert(SP % 16 == 0 && SG % 16 == 0 && SX % 16 == 0 && SF % 16 == 0, "16-byte stage pieces");
};

template <int D, int NR, int VB, typename T>
__device__ __forceinline__ void flux_prefetch(const BlockedArgs<T>& a, int f, unsigned char* st, int lane) {
  using S = FluxStage<D, NR, VB, T>;
  const unsigned char* srcP = static_cast<const unsigned char*>(a.fpoly) + size_t(f) * S::SP;
  const unsigned char* srcG = reinterpret_cast<const unsigned char*>(a.fg) + size_t(f) * S::SG;
  const unsigned char* srcX = reinterpret_cast<const unsigned char*>(a.X) + size_t(f) * S::SX;
  const unsigned char* srcF = reinterpret_cast<const unsigned char*>(a.Facc) + size_t(f) * S::SF;
  for (int q = lane; q < S::BYTES / 16; q += 32) {
    const int b = q * 16;
    const unsigned char* src = b < S::SP                   ? srcP + b
                               : b < S::SP + S::SG         ? srcG + (b - S::SP)
                               : b < S::SP + S::SG + S::SX ? srcX + (b - S::SP - S::SG)
                                                           : srcF + (b - S::SP - S::SG - S::SX);
    cp_async16(st + b, src);
  }
}

// Running sum of a face moment over the velocity blocks.  FP32 sweeps keep it
// as an unevaluated pair of floats hi + lo (Knuth's two-sum, then a fast
// renormalisation), which carries the sum of the block sums to ~2^-44
// relative without FP64 instructions: GB300's FP64 pipe runs at a small
// fraction of its FP32 rate (with a convert and an add in FP64 per face and
// block the flux kernel kept that pipe 21 % busy, and ran 4 % slower).
// k_bwall turns the pairs into doubles after the last block.  FP64 sweeps
// add in double.
template <typename T>
__device__ __forceinline__ void facc_add(double* dst, const double* prev, bool first, T v) {
  if constexpr (sizeof(T) == 4) {
    const float2 p = first ? make_float2(0.f, 0.f) : *reinterpret_cast<const float2*>(prev);
    *reinterpret_cast<float2*>(dst) = pair_add(p, v);
  } else {
    *dst = (first ? 0.0 : *prev) + double(v);
  }
}

// Micro fluxes of one face for this lane's velocities of the block (Eq. 28-29,
// 32-38), time-integrated and without the face area, in the face's
// orientation (u.n with the normal from owner to neighbour): Phi[r][j] for
// velocity (m0 + j) 32 + lane.  Xs: this lane's column of the face's rows of
// upwind free-transport parts (written by the reconstruction).  Every caller
// runs the same code on the same inputs, so both cells of a face obtain
// bitwise the same fluxes.  With `moments` the block's weighted moments of
// the flux are added to m_in (conservative-variable order, energy at D + 1)
// and, at a diffuse wall, those of the unit-density re-emitted half to m_out.
template <int D, int NR, int VB, typename T>
__device__ __forceinline__ void face_fluxes(const BlockedArgs<T>& a, const FacePoly<D, NR, T>& R,
                                            const FaceGeom<T>& fg, const T* Xs, const BlockVel<D, NR, VB, T>& v,
                                            const int lane, const int64_t m0, RowFac<NR, T>* rowbuf, const T ul,
                                            const T wl, const bool moments, T (&Phi)[NR][VB], T (&m_in)[NWP],
                                            T (&m_out)[NWP]) {
  const T dt = T(a.g.dt);
  T n[D];
#pragma unroll
  for (int d = 0; d < D; ++d) n[d] = fg.n[d];

  if (fg.bc_type == 1) {
    // diffuse wall (Eq. 36-38): free transport on the incoming side; the
    // re-emitted half is the unit-density wall Maxwellian, scaled by rho_w
    // once all blocks are summed (added in the second stage).
#pragma unroll
    for (int j = 0; j < VB; ++j) {
      T un = T(0);
#pragma unroll
      for (int d = 0; d < D; ++d) un += v.u[j][d] * n[d];
      T phi_h = T(0), phi_b = T(0), out_h = T(0);
      if (un > T(0)) {
        phi_h = un * Xs[(0 * VB + j) * BV];
        if (NR == 2) phi_b = un * Xs[((NR - 1) * VB + j) * BV];
      } else if (un < T(0) && moments) {
        T c2 = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) c2 += (v.u[j][d] - R.U[d]) * (v.u[j][d] - R.U[d]);
        out_h = un * dt * R.rho_pref * t_exp(-R.lam * c2);
      }
      Phi[0][j] = phi_h;
      if (NR == 2) Phi[NR - 1][j] = phi_b;
      if (moments) {
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
    }
    return;
  }

  const bool ghost = fg.nei < 0;
  if (!ghost && a.tensor) {
    // interior face on a tensor grid: lanes 0 .. VB-1 publish the row factors
    // (row polynomials times the row's Maxwellian factor, u.n and weight parts)
    __syncwarp();   // earlier readers of rowbuf are done
    if (lane < VB) {
      const Vel4<T> rv = a.rowv[m0 + lane];
      const T c1 = D > 1 ? rv.y - R.U[D > 1 ? 1 : 0] : T(0), c2 = D > 2 ? rv.z - R.U[D > 2 ? 2 : 0] : T(0);
      RowFac<NR, T> rf;
      const T E = R.rho_pref * t_exp(-R.lam * (c1 * c1 + c2 * c2));
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        row_polys<D, T>(R.P[r], c1, c2, rf.Q[r]);
#pragma unroll
        for (int q = 0; q < 4; ++q) rf.Q[r][q] *= E;
      }
      rf.un = (D > 1 ? n[D > 1 ? 1 : 0] * rv.y : T(0)) + (D > 2 ? n[D > 2 ? 2 : 0] * rv.z : T(0));
      rf.w = rv.w;
      rf.wu1 = rv.w * rv.y;
      rf.wu2 = rv.w * rv.z;
      rf.wusq = rv.w * (rv.y * rv.y + rv.z * rv.z);
#pragma unroll
      for (int q = 0; q < int(sizeof(rf.pad) / sizeof(T)); ++q) rf.pad[q] = T(0);
      rowbuf[lane] = rf;
    }
    __syncwarp();
    const T c0 = ul - R.U[0];
    const T El = t_exp(-R.lam * c0 * c0);
    const T un0 = n[0] * ul;
    T A0 = T(0), A1 = T(0), A2 = T(0), A4 = T(0);   // sums over the lane's rows, lane weight factored out
#pragma unroll
    for (int j = 0; j < VB; ++j) {
      const RowFac<NR, T> rf = rowbuf[j];
      const T un = un0 + rf.un;
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const T P = fma(c0, fma(c0, fma(c0, rf.Q[r][3], rf.Q[r][2]), rf.Q[r][1]), rf.Q[r][0]);
        Phi[r][j] = un * fma(El, P, Xs[(r * VB + j) * BV]);
      }
      if (moments) {
        A0 = fma(rf.w, Phi[0][j], A0);
        if (D > 1) A1 = fma(rf.wu1, Phi[0][j], A1);
        if (D > 2) A2 = fma(rf.wu2, Phi[0][j], A2);
        A4 = fma(rf.wusq, Phi[0][j], A4);
        if (NR == 2) A4 = fma(rf.w, Phi[NR - 1][j], A4);
      }
    }
    if (moments) {
      m_in[0] += wl * A0;
      m_in[1] += wl * ul * A0;
      if (D > 1) m_in[2] += wl * A1;
      if (D > 2) m_in[3] += wl * A2;
      m_in[D + 1] += T(0.5) * wl * fma(ul * ul, A0, A4);
    }
    return;
  }
  if (!ghost) {
    // interior face: straight-line code (u.n = 0 gives a zero flux by itself)
#pragma unroll
    for (int j = 0; j < VB; ++j) {
      T un = T(0);
#pragma unroll
      for (int d = 0; d < D; ++d) un += v.u[j][d] * n[d];
      T c[3] = {T(0), T(0), T(0)}, c2 = T(0);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        c[d] = v.u[j][d] - R.U[d];
        c2 += c[d] * c[d];
      }
      const T H0 = R.rho_pref * t_exp(-R.lam * c2);
#pragma unroll
      for (int r = 0; r < NR; ++r)
        Phi[r][j] = un * fma(H0, horner_cubic<D, T>(R.P[r], c[0], c[1], c[2]), Xs[(r * VB + j) * BV]);
      if (moments) {
        const T wph = v.w[j] * Phi[0][j];
        m_in[0] += wph;
#pragma unroll
        for (int d = 0; d < D; ++d) m_in[1 + d] += wph * v.u[j][d];
        m_in[D + 1] += T(0.5) * v.w[j] * (v.u2[j] * Phi[0][j] + (NR == 2 ? Phi[NR - 1][j] : T(0)));
      }
    }
    return;
  }
  T gr = T(0), gl = T(0), gU[3] = {T(0), T(0), T(0)}, gk = T(0);
  {
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
    for (int d = 0; d < D; ++d) un += v.u[j][d] * n[d];
    T phi_h = T(0), phi_b = T(0);
    if (un != T(0)) {
      T tr[NR];
      if (un > T(0)) {
#pragma unroll
        for (int r = 0; r < NR; ++r) tr[r] = Xs[(r * VB + j) * BV];
      } else {
        T c2 = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) c2 += (v.u[j][d] - gU[d]) * (v.u[j][d] - gU[d]);
        const T H = gr * t_exp(-gl * c2);
        tr[0] = R.G0 * H;
        if (NR == 2) tr[NR - 1] = R.G0 * (gk * H);
      }
      // equilibrium part G2 (g0 + g0+) + G3 u.grad g0 + G4 d_t g0 = g0(u) P(c) (Eq. 32-33)
      T c[3] = {T(0), T(0), T(0)}, c2 = T(0);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        c[d] = v.u[j][d] - R.U[d];
        c2 += c[d] * c[d];
      }
      const T H0 = R.rho_pref * t_exp(-R.lam * c2);
      phi_h = un * fma(H0, horner_cubic<D, T>(R.P[0], c[0], c[1], c[2]), tr[0]);
      if (NR == 2) phi_b = un * fma(H0, horner_cubic<D, T>(R.P[NR - 1], c[0], c[1], c[2]), tr[NR - 1]);
    }
    Phi[0][j] = phi_h;
    if (NR == 2) Phi[NR - 1][j] = phi_b;
    if (moments) {
      const T wph = v.w[j] * phi_h;
      m_in[0] += wph;
#pragma unroll
      for (int d = 0; d < D; ++d) m_in[1 + d] += wph * v.u[j][d];
      m_in[D + 1] += T(0.5) * v.w[j] * (v.u2[j] * phi_h + phi_b);
    }
  }
}

// Adds the block's moments of one face (per-lane partials, reduced over the
// warp) to its accumulator: slots [0, D+2) the flux, [5, 5+D+2) at a wall the
// unit re-emitted half.  Fs: the accumulator as it was before this block
// (ignored on the first block).
template <int D, typename T>
__device__ __forceinline__ void face_moments_add(double* Fa, const double* Fs, bool wall, int first,
                                                 const T (&m_in)[NWP], const T (&m_out)[NWP], int lane) {
  constexpr int NW = D + 2;
  const int idx8 = sum8_index(lane);
  const bool writer = (lane & 3) == 0 && idx8 < NW;
  const T sin = warp_sum8<T>(m_in[0], m_in[1], m_in[2], m_in[3], m_in[4], T(0), T(0), T(0), lane);
  if (writer) facc_add<T>(Fa + idx8, Fs + idx8, first, sin);
  if (wall) {
    const T sout = warp_sum8<T>(m_out[0], m_out[1], m_out[2], m_out[3], m_out[4], T(0), T(0), T(0), lane);
    if (writer) facc_add<T>(Fa + 5 + idx8, Fs + 5 + idx8, first, sout);
  }
}

// Flux kernel step for one face: its fluxes overwrite the face's rows of X,
// its moments go to the face accumulator.
template <int D, int NR, int VB, typename T>
__device__ __forceinline__ void flux_face(const BlockedArgs<T>& a, const int f, const unsigned char* st,
                                          const BlockVel<D, NR, VB, T>& v, const int first, const int lane,
                                          const int64_t m0, RowFac<NR, T>* rowbuf, const T ul, const T wl) {
  using S = FluxStage<D, NR, VB, T>;
  const FacePoly<D, NR, T>& R = *reinterpret_cast<const FacePoly<D, NR, T>*>(st);
  const FaceGeom<T>& fg = *reinterpret_cast<const FaceGeom<T>*>(st + S::SP);
  const T* Xs = reinterpret_cast<const T*>(st + S::SP + S::SG) + lane;
  const double* Fs = reinterpret_cast<const double*>(st + S::SP + S::SG + S::SX);
  T Phi[NR][VB], m_in[NWP], m_out[NWP];
#pragma unroll
  for (int t = 0; t < NWP; ++t) m_in[t] = m_out[t] = T(0);
  face_fluxes<D, NR, VB, T>(a, R, fg, Xs, v, lane, m0, rowbuf, ul, wl, true, Phi, m_in, m_out);
  T* Xf = a.X + size_t(f) * (NR * VB * BV) + lane;
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int j = 0; j < VB; ++j) Xf[(r * VB + j) * BV] = Phi[r][j];
  face_moments_add<D, T>(a.Facc + size_t(f) * FACC_W, Fs, fg.bc_type == 1, first, m_in, m_out, lane);
}

template <int D, int NR, int VB, typename T>
__global__ void __launch_bounds__(kBlockedThreads, VB == 8 ? 3 : 1) k_bflux(const BlockedArgs<T> a, const int64_t m0,
                                                           const int first) {
  using S = FluxStage<D, NR, VB, T>;
  extern __shared__ __align__(16) unsigned char flux_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* const st = flux_smem + warp * (2 * S::BYTES);
  RowFac<NR, T>* const rowbuf =
      reinterpret_cast<RowFac<NR, T>*>(flux_smem + (kBlockedThreads / 32) * 2 * S::BYTES) + warp * VB;
  BlockVel<D, NR, VB, T> v;
  v.load(a, m0, lane);
  const T ul = a.tensor ? a.lanev[lane] : T(0), wl = a.tensor ? a.lanev[BV + lane] : T(0);
  const int stride = gridDim.x * (kBlockedThreads / 32);
  int f = blockIdx.x * (kBlockedThreads / 32) + warp;
  if (f < a.Nf) flux_prefetch<D, NR, VB, T>(a, f, st, lane);
  cp_async_commit();
  for (int it = 0; f < a.Nf; f += stride, ++it) {
    const int fn = f + stride;
    if (fn < a.Nf) flux_prefetch<D, NR, VB, T>(a, fn, st + ((it + 1) & 1) * S::BYTES, lane);
    cp_async_commit();
    cp_async_wait<1>();  // this face's stage has landed
    __syncwarp();
    flux_face<D, NR, VB, T>(a, f, st + (it & 1) * S::BYTES, v, first, lane, m0, rowbuf, ul, wl);
    __syncwarp();        // all lanes done with the stage before it is refilled
  }
  cp_async_wait<0>();
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
  const CellEq<T> E = a.ceq0[c];
  const T lam = E.lam, beta0 = E.beta, pref = E.pref, s0 = E.s0, kap = E.kap;
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
  const T inv_vol = E.inv_vol;
#pragma unroll
  for (int j = 0; j < VB; ++j) {
    T c2 = T(0), cq = T(0);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const T cd = v.u[j][d] - E.U[d];
      c2 += cd * cd;
      cq += cd * E.q[d];
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
// Pipelined per-cell kernels (K2 and K3 on meshes with at most kEllMax faces
// per cell).  Each warp walks cells c, c + stride, ...; per cell it needs
// the cell's incidence records (an ELL table: W slots per cell, padding
// flagged) and then rows addressed through them (neighbour or flux rows).
// Both are staged into shared memory with cp.async: the records two cells
// ahead, the rows one cell ahead, so the dependent loads of the next cells
// overlap the arithmetic of the current one.
// ---------------------------------------------------------------------------
constexpr int kEllMax = 8;

// cp.async of one 4- or 8-byte value.
template <int N>
__device__ __forceinline__ void cp_async_small(void* smem, const void* gmem) {
  static_assert(N == 4 || N == 8, "cp.async.ca copies 4, 8 or 16 bytes");
  const unsigned s = unsigned(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(N) : "memory");
}

// Contiguous bytes (a multiple of 16) by all lanes of the warp.
__device__ __forceinline__ void stage_bytes(unsigned char* dst, const void* src, int bytes, int lane) {
  const unsigned char* s = static_cast<const unsigned char*>(src);
  for (int q = lane; q < bytes / 16; q += 32) cp_async16(dst + q * 16, s + q * 16);
}

template <int NR, int VB, typename T>
struct CellStage {
  static constexpr int ROW = NR * VB * BV * int(sizeof(T));  // rows of one face (flux buffer X)
  static constexpr int INC = int(sizeof(IncT<T>));
};

// One cell's stored rows in shared memory: the NR x VB rows in the storage
// type S, then (scaled storage) their FP32 scales and the cell's reference
// Maxwellian.
template <int NR, int VB, typename S>
struct CellSlot {
  static constexpr bool SCALED = StoreTraits<S>::scaled;
  static constexpr int ROWS = NR * VB * BV * int(sizeof(S));
  static constexpr int SCL = SCALED ? ((NR * VB * 4 + 15) / 16) * 16 : 0;
  static constexpr int REF = SCALED ? int(sizeof(RefMaxwell)) : 0;
  static constexpr int BYTES = ROWS + SCL + REF;
};

// Stages cell c's slot of f^n for block m0.
template <int NR, int VB, typename T, typename S>
__device__ __forceinline__ void stage_cell(unsigned char* dst, const BlockedArgs<T>& a, int64_t m0, int c, int lane) {
  using CS = CellSlot<NR, VB, S>;
  constexpr int CH = BV * int(sizeof(S)) / 16;  // 16-byte chunks per row
  const size_t sj = size_t(a.Nc) * BV, sr = size_t(a.M) * sj;
  const S* f = reinterpret_cast<const S*>(a.f_cur);
  for (int q = lane; q < NR * VB * CH; q += 32) {
    const int row = q / CH, part = q % CH, r = row / VB, j = row % VB;
    const S* src = f + r * sr + (size_t(m0) + j) * sj + size_t(c) * BV;
    cp_async16(dst + q * 16, reinterpret_cast<const unsigned char*>(src) + part * 16);
  }
  if constexpr (CS::SCALED) {
    for (int q = lane; q < NR * VB; q += 32) {
      const int r = q / VB, j = q % VB;
      cp_async_small<4>(dst + CS::ROWS + q * 4, a.sc_cur + (size_t(r) * a.M + m0 + j) * a.Nc + c);
    }
    if (lane < 2)
      cp_async16(dst + CS::ROWS + CS::SCL + lane * 16, reinterpret_cast<const unsigned char*>(a.ref_cur + c) + lane * 16);
  }
}

// Values of a staged cell slot: f of reduced distribution r at sub-block j for
// this lane (decoded for scaled storage; g0[j] = the slot's reference
// Maxwellian at the lane's velocity, computed by slot_refs).
template <int D, int NR, int VB, typename T, typename S>
__device__ __forceinline__ void slot_refs(const unsigned char* slot, const BlockVel<D, NR, VB, T>& v, T (&g0)[VB]) {
  using CS = CellSlot<NR, VB, S>;
  if constexpr (CS::SCALED) {
    const RefMaxwell& R = *reinterpret_cast<const RefMaxwell*>(slot + CS::ROWS + CS::SCL);
#pragma unroll
    for (int j = 0; j < VB; ++j) g0[j] = ref_value<D>(R, 0, v.u[j], v.real[j]);
  }
}
template <int NR, int VB, typename T, typename S>
__device__ __forceinline__ T slot_value(const unsigned char* slot, int r, int j, int lane, const T (&g0)[VB]) {
  using CS = CellSlot<NR, VB, S>;
  const S d = reinterpret_cast<const S*>(slot)[(r * VB + j) * BV + lane];
  if constexpr (CS::SCALED) {
    const RefMaxwell& R = *reinterpret_cast<const RefMaxwell*>(slot + CS::ROWS + CS::SCL);
    const float sc = reinterpret_cast<const float*>(slot + CS::ROWS)[r * VB + j];
    return decode_value(d, sc, r == 0 ? g0[j] : R.kap * g0[j]);
  } else {
    return T(d);
  }
}

// Shared-memory bytes per warp of the pipelined kernels (3 record slots, 2 row slots).
template <int NR, int VB, typename T, typename S>
__host__ __device__ constexpr int recon_warp_bytes(int W) {
  return 3 * (W * CellStage<NR, VB, T>::INC + 16) + 2 * ((W + 1) * CellSlot<NR, VB, S>::BYTES + W * 16);
}
template <int NR, int VB, typename T, typename S>
__host__ __device__ constexpr int stage1_warp_bytes(int W) {
  return 3 * (W * CellStage<NR, VB, T>::INC + int(sizeof(CellEq<T>))) +
         2 * (W * CellStage<NR, VB, T>::ROW + CellSlot<NR, VB, S>::BYTES) + 16;   // + two mbarriers
}

// byte offset of the 16-byte chunk of a FacePoly that holds G0 and G1
template <int D, int NR, typename T>
__host__ __device__ constexpr int g01_chunk() {
  using FP = FacePoly<D, NR, T>;
  return (int(offsetof(FP, G0)) / 16) * 16;
}

template <int D, int NR, int VB, int WT, typename T, typename S>
__global__ void __launch_bounds__(kBlockedThreads) k_brecon_p(const BlockedArgs<T> a, const int64_t m0) {
  using CS = CellStage<NR, VB, T>;
  using SL = CellSlot<NR, VB, S>;
  using FP = FacePoly<D, NR, T>;
  static_assert(offsetof(FP, G1) + sizeof(T) <= size_t(g01_chunk<D, NR, T>() + 16),
                "G0 and G1 share one 16-byte chunk");
  extern __shared__ __align__(16) unsigned char cell_smem[];
  constexpr int W = WT;  // ELL slots per cell (the table is padded to WT)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int AB = W * CS::INC + 16, BB = (W + 1) * SL::BYTES + W * 16;
  unsigned char* const As = cell_smem + warp * recon_warp_bytes<NR, VB, T, S>(W);
  unsigned char* const Bs = As + 3 * AB;
  BlockVel<D, NR, VB, T> v;
  v.load(a, m0, lane);
  const int Kxi = a.g.Kxi, limiter = a.g.limiter;
  const T dt = T(a.g.dt);
  const T hdt2 = T(0.5 * a.g.dt * a.g.dt);
  const int stride = gridDim.x * nwarps;
  const int cbeg = blockIdx.x * nwarps + warp;

  auto issueA = [&](int c, unsigned char* dst) {
    stage_bytes(dst, a.ell + size_t(c) * W, W * CS::INC, lane);
    if (lane == 0) cp_async_small<int(sizeof(T))>(dst + W * CS::INC, a.eps2 + c);
  };
  auto issueB = [&](int c, const unsigned char* A, unsigned char* dst) {
    const IncT<T>* inc = reinterpret_cast<const IncT<T>*>(A);
    for (int i = 0; i < W; ++i) {
      const int fl = inc[i].flags;
      if (fl & 3) continue;  // wall or padding: no neighbour row, no G0/G1
      const int o = inc[i].other;
      if (o >= 0) stage_cell<NR, VB, T, S>(dst + i * SL::BYTES, a, m0, o, lane);
      if (lane == 0)
        cp_async16(dst + (W + 1) * SL::BYTES + i * 16,
                   static_cast<const unsigned char*>(a.fpoly) + size_t(inc[i].face) * sizeof(FacePoly<D, NR, T>) +
                       g01_chunk<D, NR, T>());
    }
    stage_cell<NR, VB, T, S>(dst + W * SL::BYTES, a, m0, c, lane);
  };

  if (cbeg < a.Nc) issueA(cbeg, As);
  cp_async_commit();
  cp_async_wait<0>();
  __syncwarp();
  if (cbeg < a.Nc) issueB(cbeg, As, Bs);
  if (cbeg + stride < a.Nc) issueA(cbeg + stride, As + AB);
  cp_async_commit();
  int it = 0;
  for (int c = cbeg; c < a.Nc; c += stride, ++it) {
    cp_async_wait<0>();  // rows of c and records of c + stride have landed
    __syncwarp();
    const int cn = c + stride, cnn = c + 2 * stride;
    if (cn < a.Nc) issueB(cn, As + ((it + 1) % 3) * AB, Bs + ((it + 1) & 1) * BB);
    if (cnn < a.Nc) issueA(cnn, As + ((it + 2) % 3) * AB);
    cp_async_commit();

    const unsigned char* A = As + (it % 3) * AB;
    const unsigned char* B = Bs + (it & 1) * BB;
    const IncT<T>* inc = reinterpret_cast<const IncT<T>*>(A);
    const unsigned char* own = B + W * SL::BYTES;  // slots [W+1]: the neighbours, then this cell
    T g0[VB];
    slot_refs<D, NR, VB, T, S>(own, v, g0);
    T fc[NR][VB], g[NR][VB][D], fmx[NR][VB], fmn[NR][VB];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int j = 0; j < VB; ++j) {
        fc[r][j] = slot_value<NR, VB, T, S>(own, r, j, lane, g0);
        fmx[r][j] = fmn[r][j] = fc[r][j];
#pragma unroll
        for (int d = 0; d < D; ++d) g[r][j][d] = T(0);
      }
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const int fl = inc[i].flags;
      if (fl & 3) continue;  // walls: one-sided stencil; padding
      T wd[D];
#pragma unroll
      for (int d = 0; d < D; ++d) wd[d] = inc[i].w[d];
      T fo[NR][VB];
      if (inc[i].other >= 0) {
        const unsigned char* nb = B + i * SL::BYTES;
        T gn[VB];
        slot_refs<D, NR, VB, T, S>(nb, v, gn);
#pragma unroll
        for (int r = 0; r < NR; ++r)
#pragma unroll
          for (int j = 0; j < VB; ++j) fo[r][j] = slot_value<NR, VB, T, S>(nb, r, j, lane, gn);
      } else {
        T rho, lam, U[3];
        ghost_state<D, NR, T>(a, inc[i].bc, c, rho, lam, U);
        const T pref = rho * maxwell_pref<D>(lam);
#pragma unroll
        for (int j = 0; j < VB; ++j) {
          T c2 = T(0);
#pragma unroll
          for (int d = 0; d < D; ++d) c2 += (v.u[j][d] - U[d]) * (v.u[j][d] - U[d]);
          const T H = v.real[j] ? pref * t_exp(-lam * c2) : T(0);
          fo[0][j] = H;
          if (NR == 2) fo[NR - 1][j] = T(Kxi) / (T(2) * lam) * H;
        }
      }
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int j = 0; j < VB; ++j) {
          const T df = fo[r][j] - fc[r][j];
#pragma unroll
          for (int d = 0; d < D; ++d) g[r][j][d] += wd[d] * df;
          fmx[r][j] = fmax(fmx[r][j], fo[r][j]);
          fmn[r][j] = fmin(fmn[r][j], fo[r][j]);
        }
    }
    T phi[NR][VB];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int j = 0; j < VB; ++j) phi[r][j] = T(1);
    if (limiter != 0) {
      const T eps2c = *reinterpret_cast<const T*>(A + W * CS::INC);
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
      // Both limiters are non-increasing in |d2| on each side (Venkatakrishnan's
      // psi(dp, d2) is >= 1 for d2/dp <= 1/2 and decreasing beyond), so the
      // minimum over faces is taken at the largest positive and the most
      // negative face increment: two evaluations instead of one per face.
      T d2p[NR][VB], d2n[NR][VB];
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int j = 0; j < VB; ++j) d2p[r][j] = d2n[r][j] = T(0);
#pragma unroll
      for (int i = 0; i < W; ++i) {
        if (inc[i].flags & 2) continue;  // padding
        T rr[D];
#pragma unroll
        for (int d = 0; d < D; ++d) rr[d] = inc[i].r[d];
#pragma unroll
        for (int r = 0; r < NR; ++r)
#pragma unroll
          for (int j = 0; j < VB; ++j) {
            T d2 = T(0);
#pragma unroll
            for (int d = 0; d < D; ++d) d2 += g[r][j][d] * rr[d];
            d2p[r][j] = fmax(d2p[r][j], d2);
            d2n[r][j] = fmin(d2n[r][j], d2);
          }
      }
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int j = 0; j < VB; ++j)
#pragma unroll
          for (int side = 0; side < 2; ++side) {
            const T d2 = side == 0 ? d2p[r][j] : d2n[r][j];
            const T dp = side == 0 ? dmx[r][j] : dmn[r][j];
            if (d2 == T(0)) continue;
            T ph;
            if (limiter == 2) {
              ph = fast_div(dp, d2);
            } else {
              // (dp^2 + eps + 2 d2 dp) / (dp^2 + 2 d2^2 + dp d2 + eps)
              const T num = fma(dp, dp + T(2) * d2, eps2[r][j]);
              const T den = fma(dp + d2, dp, fma(T(2) * d2, d2, eps2[r][j]));
              ph = fast_div(num, den);
            }
            phi[r][j] = fmin(phi[r][j], ph);
          }
    }
    T ug[NR][VB];  // u . (limited gradient), the same on every face
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int j = 0; j < VB; ++j) {
        const T p = fmin(fmax(phi[r][j], T(0)), T(1));
        ug[r][j] = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) {
          g[r][j][d] *= p;
          ug[r][j] += v.u[j][d] * g[r][j][d];
        }
      }
    // free-transport part on every face for which this cell is upwind
    const T* G01 = reinterpret_cast<const T*>(B + (W + 1) * SL::BYTES);
    constexpr int g0i = (int(offsetof(FP, G0)) - g01_chunk<D, NR, T>()) / int(sizeof(T));
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const int fl = inc[i].flags;
      if (fl & 2) continue;
      T c0, c1;
      if (fl & 1) {
        c0 = dt;
        c1 = -hdt2;
      } else {
        c0 = G01[i * (16 / int(sizeof(T))) + g0i];
        c1 = G01[i * (16 / int(sizeof(T))) + g0i + 1];
      }
      T n[D], rr[D];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        n[d] = inc[i].n[d];
        rr[d] = inc[i].r[d];
      }
      T* Xf = a.X + size_t(inc[i].face) * (NR * VB * BV) + lane;
      const bool owner = inc[i].sarea > T(0);
#pragma unroll
      for (int j = 0; j < VB; ++j) {
        T un = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) un += v.u[j][d] * n[d];
        // upwind side; u.n = 0 (padding included) written by the owner, so
        // that every lane of an interior face is written once per block
        if (un > T(0) || (un == T(0) && owner)) {
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            T ff = fc[r][j];
#pragma unroll
            for (int d = 0; d < D; ++d) ff += g[r][j][d] * rr[d];
            Xf[(r * VB + j) * BV] = c0 * ff + c1 * ug[r][j];
          }
        }
      }
    }
    __syncwarp();  // all lanes done with the slots before they are refilled
  }
  cp_async_wait<0>();
}

template <int D, int NR, int VB, int WT, typename T, typename S>
__global__ void __launch_bounds__(kBlockedThreads) k_bstage1_p(const BlockedArgs<T> a, const int64_t m0) {
  using CS = CellStage<NR, VB, T>;
  using SL = CellSlot<NR, VB, S>;
  extern __shared__ __align__(16) unsigned char cell_smem[];
  constexpr int W = WT;  // ELL slots per cell (the table is padded to WT)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int AB = W * CS::INC + int(sizeof(CellEq<T>)), BB = W * CS::ROW + SL::BYTES;
  unsigned char* const As = cell_smem + warp * stage1_warp_bytes<NR, VB, T, S>(W);
  unsigned char* const Bs = As + 3 * AB;
  BlockVel<D, NR, VB, T> v;
  v.load(a, m0, lane);
  const size_t sj = size_t(a.Nc) * BV, sr = size_t(a.M) * sj;
  const int stride = gridDim.x * nwarps;
  const int cbeg = blockIdx.x * nwarps + warp;
  // Cells are visited from the last to the first (item i is cell Nc - 1 - i):
  // the flux kernel writes the per-face buffer in increasing face order, so
  // the rows it wrote last, still in L2, are read first.
  auto cell_of = [&](int i) { return a.Nc - 1 - i; };

  auto issueA = [&](int item, unsigned char* dst) {
    const int c = cell_of(item);
    stage_bytes(dst, a.ell + size_t(c) * W, W * CS::INC, lane);
    stage_bytes(dst + W * CS::INC, a.ceq0 + c, int(sizeof(CellEq<T>)), lane);
  };
  // The rows of a cell's slot arrive by 1-D bulk copies, one per lane: the
  // block of each face in X (one contiguous CS::ROW segment) and each of the
  // cell's NR x VB rows of f^n (one 32-velocity segment each), completing in
  // bytes on the slot's mbarrier; records and the scaled-storage extras come
  // by cp.async.
  uint64_t* const bars = reinterpret_cast<uint64_t*>(Bs + 2 * BB);
  if (lane == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init_fence();
  }
  __syncwarp();
  const S* const fs = reinterpret_cast<const S*>(a.f_cur);
  constexpr unsigned kRowBytes = BV * unsigned(sizeof(S));
  static_assert(CS::ROW % 16 == 0 && kRowBytes % 16 == 0, "bulk copies move multiples of 16 bytes");
  static_assert((WT * CS::INC + sizeof(CellEq<T>)) % 16 == 0 && (WT * CS::ROW + SL::BYTES) % 16 == 0,
                "16-byte aligned slots");
  static_assert(WT + NR * VB <= 32, "one copy per lane");
  auto issueB = [&](int item, const unsigned char* A, unsigned char* dst, uint64_t* bar) {
    const int c = cell_of(item);
    const IncT<T>* inc = reinterpret_cast<const IncT<T>*>(A);
    unsigned bytes = NR * VB * kRowBytes;
#pragma unroll
    for (int i = 0; i < W; ++i)
      if (!(inc[i].flags & 2)) bytes += CS::ROW;
    // this lane's reads of the slot (two items ago) before the copies' writes;
    // the slot's bytes announced before any copy is issued
    fence_proxy_async_smem();
    if (lane == 0) mbar_arrive_expect_tx(bar, bytes);
    __syncwarp();
    if (lane < W) {
      if (!(inc[lane].flags & 2))
        bulk_load(dst + lane * CS::ROW, a.X + size_t(inc[lane].face) * (NR * VB * BV), CS::ROW, bar);
    } else if (lane < W + NR * VB) {
      const int q = lane - W, r = q / VB, j = q % VB;
      bulk_load(dst + W * CS::ROW + q * kRowBytes, fs + r * sr + (size_t(m0) + j) * sj + size_t(c) * BV,
                kRowBytes, bar);
    }
    if constexpr (SL::SCALED) {
      unsigned char* cs = dst + W * CS::ROW;
      for (int q = lane; q < NR * VB; q += 32) {
        const int r = q / VB, j = q % VB;
        cp_async_small<4>(cs + SL::ROWS + q * 4, a.sc_cur + (size_t(r) * a.M + m0 + j) * a.Nc + c);
      }
      if (lane < 2)
        cp_async16(cs + SL::ROWS + SL::SCL + lane * 16, reinterpret_cast<const unsigned char*>(a.ref_cur + c) + lane * 16);
    }
  };

  if (cbeg < a.Nc) issueA(cbeg, As);
  cp_async_commit();
  cp_async_wait<0>();
  __syncwarp();
  if (cbeg < a.Nc) issueB(cbeg, As, Bs, &bars[0]);
  if (cbeg + stride < a.Nc) issueA(cbeg + stride, As + AB);
  cp_async_commit();
  int it = 0;
  for (int ci = cbeg; ci < a.Nc; ci += stride, ++it) {
    cp_async_wait<0>();
    // slot it & 1 is used for the (it >> 1)-th time: that phase of its barrier
    if (!mbar_wait(&bars[it & 1], unsigned(it >> 1) & 1u, a.status)) {
      mbar_wait(&bars[it & 1], unsigned(it >> 1) & 1u, a.status);   // its copies may still be in flight
      break;
    }
    __syncwarp();
    const int cn = ci + stride, cnn = ci + 2 * stride;
    if (cn < a.Nc) issueB(cn, As + ((it + 1) % 3) * AB, Bs + ((it + 1) & 1) * BB, &bars[(it + 1) & 1]);
    if (cnn < a.Nc) issueA(cnn, As + ((it + 2) % 3) * AB);
    cp_async_commit();
    const int c = cell_of(ci);

    const unsigned char* A = As + (it % 3) * AB;
    const unsigned char* B = Bs + (it & 1) * BB;
    const IncT<T>* inc = reinterpret_cast<const IncT<T>*>(A);
    const CellEq<T>& E = *reinterpret_cast<const CellEq<T>*>(A + W * CS::INC);
    const T* rows = reinterpret_cast<const T*>(B) + lane;
    T flux[NR][VB];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int j = 0; j < VB; ++j) flux[r][j] = T(0);
#pragma unroll
    for (int i = 0; i < W; ++i) {
      if (inc[i].flags & 2) continue;
      const T sa = inc[i].sarea;
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int j = 0; j < VB; ++j) flux[r][j] += sa * rows[(i * NR * VB + r * VB + j) * BV];
    }
    const unsigned char* own = B + W * CS::ROW;
    T g0[VB];
    slot_refs<D, NR, VB, T, S>(own, v, g0);
    const T lam = E.lam, beta0 = E.beta, pref = E.pref, s0 = E.s0, kap = E.kap, inv_vol = E.inv_vol;
    const size_t base = size_t(m0) * sj + size_t(c) * BV + lane;
#pragma unroll
    for (int j = 0; j < VB; ++j) {
      T c2 = T(0), cq = T(0);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const T cd = v.u[j][d] - E.U[d];
        c2 += cd * cd;
        cq += cd * E.q[d];
      }
      const T H = pref * t_exp(-lam * c2);
      const T s = s0 * cq;
      T fp[NR];
      fp[0] = H * (T(1) + s * (T(2) * lam * c2 - T(2 + D)));
      if (NR == 2) fp[NR - 1] = kap * H * (T(1) + s * (T(2) * lam * c2 - T(D)));
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const T f = slot_value<NR, VB, T, S>(own, r, j, lane, g0);
        const T ft = v.real[j] ? f - flux[r][j] * inv_vol + beta0 * (fp[r] - f) : T(0);
        if constexpr (SL::SCALED) {
          // f~ is stored against the same reference as f^n
          const RefMaxwell& R = *reinterpret_cast<const RefMaxwell*>(own + SL::ROWS + SL::SCL);
          float scale;
          const S d = encode_value<S>(ft, r == 0 ? g0[j] : R.kap * g0[j], scale);
          reinterpret_cast<S*>(a.f_next)[base + r * sr + j * sj] = d;
          if (lane == 0) a.sc_next[(size_t(r) * a.M + m0 + j) * a.Nc + c] = scale;
        } else {
          a.f_next[base + r * sr + j * sj] = ft;
        }
      }
    }
    __syncwarp();
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// K1 + K3 fused: the micro fluxes of every face of the cell and the first
// stage (Eq. 28-29, 32-38, 41; Algorithms 1 and 4).  Each cell evaluates the
// fluxes of its faces itself (an interior face is evaluated by both of its
// cells, with the same code on the same inputs, so both use bitwise the same
// fluxes); the owner cell alone adds the face's moments to the face
// accumulator.  This replaces the per-face flux kernel, whose write and
// re-read of the face buffer X cost two DRAM passes over X per block.  The
// pipeline is that of k_bstage1_p: per incidence the face's X rows, interface
// polynomial, geometry and accumulator are staged one cell ahead.
// ---------------------------------------------------------------------------
template <int D, int NR, int VB, typename T>
struct FaceSlot {
  static constexpr int ROW = NR * VB * BV * int(sizeof(T));   // the face's rows of X
  static constexpr int SP = int(sizeof(FacePoly<D, NR, T>));
  static constexpr int SG = int(sizeof(FaceGeom<T>));
  static constexpr int SF = FACC_W * int(sizeof(double));
  static constexpr int BYTES = ROW + SP + SG + SF;
  static_assert(ROW % 16 == 0 && SP % 16 == 0 && SG % 16 == 0 && SF % 16 == 0, "16-byte slot pieces");
};

template <int D, int NR, int VB, typename T, typename S>
__host__ __device__ constexpr int stage1f_warp_bytes(int W) {
  return 3 * (W * CellStage<NR, VB, T>::INC + int(sizeof(CellEq<T>))) +
         2 * (W * FaceSlot<D, NR, VB, T>::BYTES + CellSlot<NR, VB, S>::BYTES) + VB * int(sizeof(RowFac<NR, T>));
}

template <int D, int NR, int VB, int WT, typename T, typename S>
__global__ void __launch_bounds__(kBlockedThreads) k_bstage1f(const BlockedArgs<T> a, const int64_t m0,
                                                              const int first) {
  using CS = CellStage<NR, VB, T>;
  using SL = CellSlot<NR, VB, S>;
  using FS = FaceSlot<D, NR, VB, T>;
  extern __shared__ __align__(16) unsigned char cell_smem[];
  constexpr int W = WT;  // ELL slots per cell (the table is padded to WT)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int AB = W * CS::INC + int(sizeof(CellEq<T>)), BB = W * FS::BYTES + SL::BYTES;
  unsigned char* const As = cell_smem + warp * stage1f_warp_bytes<D, NR, VB, T, S>(W);
  unsigned char* const Bs = As + 3 * AB;
  RowFac<NR, T>* const rowbuf = reinterpret_cast<RowFac<NR, T>*>(Bs + 2 * BB);
  BlockVel<D, NR, VB, T> v;
  v.load(a, m0, lane);
  const T ul = a.tensor ? a.lanev[lane] : T(0), wl = a.tensor ? a.lanev[BV + lane] : T(0);
  const size_t sj = size_t(a.Nc) * BV, sr = size_t(a.M) * sj;
  const int stride = gridDim.x * nwarps;
  const int cbeg = blockIdx.x * nwarps + warp;

  auto issueA = [&](int c, unsigned char* dst) {
    stage_bytes(dst, a.ell + size_t(c) * W, W * CS::INC, lane);
    stage_bytes(dst + W * CS::INC, a.ceq0 + c, int(sizeof(CellEq<T>)), lane);
  };
  auto issueB = [&](int c, const unsigned char* A, unsigned char* dst) {
    const IncT<T>* inc = reinterpret_cast<const IncT<T>*>(A);
    for (int i = 0; i < W; ++i) {
      if (inc[i].flags & 2) continue;
      const size_t f = size_t(inc[i].face);
      unsigned char* d = dst + i * FS::BYTES;
      stage_bytes(d, a.X + f * (NR * VB * BV), FS::ROW, lane);
      stage_bytes(d + FS::ROW, static_cast<const unsigned char*>(a.fpoly) + f * FS::SP, FS::SP, lane);
      stage_bytes(d + FS::ROW + FS::SP, a.fg + f, FS::SG, lane);
      if (!first && inc[i].sarea > T(0)) stage_bytes(d + FS::ROW + FS::SP + FS::SG, a.Facc + f * FACC_W, FS::SF, lane);
    }
    stage_cell<NR, VB, T, S>(dst + W * FS::BYTES, a, m0, c, lane);
  };

  if (cbeg < a.Nc) issueA(cbeg, As);
  cp_async_commit();
  cp_async_wait<0>();
  __syncwarp();
  if (cbeg < a.Nc) issueB(cbeg, As, Bs);
  if (cbeg + stride < a.Nc) issueA(cbeg + stride, As + AB);
  cp_async_commit();
  int it = 0;
  for (int c = cbeg; c < a.Nc; c += stride, ++it) {
    cp_async_wait<0>();
    __syncwarp();
    const int cn = c + stride, cnn = c + 2 * stride;
    if (cn < a.Nc) issueB(cn, As + ((it + 1) % 3) * AB, Bs + ((it + 1) & 1) * BB);
    if (cnn < a.Nc) issueA(cnn, As + ((it + 2) % 3) * AB);
    cp_async_commit();

    const unsigned char* A = As + (it % 3) * AB;
    const unsigned char* B = Bs + (it & 1) * BB;
    const IncT<T>* inc = reinterpret_cast<const IncT<T>*>(A);
    const CellEq<T>& E = *reinterpret_cast<const CellEq<T>*>(A + W * CS::INC);
    T flux[NR][VB];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int j = 0; j < VB; ++j) flux[r][j] = T(0);
#pragma unroll 1
    for (int i = 0; i < W; ++i) {
      if (inc[i].flags & 2) continue;
      const unsigned char* fsl = B + i * FS::BYTES;
      const FacePoly<D, NR, T>& R = *reinterpret_cast<const FacePoly<D, NR, T>*>(fsl + FS::ROW);
      const FaceGeom<T>& fg = *reinterpret_cast<const FaceGeom<T>*>(fsl + FS::ROW + FS::SP);
      const T* Xs = reinterpret_cast<const T*>(fsl) + lane;
      const T sa = inc[i].sarea;
      const bool owner = sa > T(0);   // walls and artificial boundaries have owner cells only
      T Phi[NR][VB], m_in[NWP], m_out[NWP];
#pragma unroll
      for (int t = 0; t < NWP; ++t) m_in[t] = m_out[t] = T(0);
      face_fluxes<D, NR, VB, T>(a, R, fg, Xs, v, lane, m0, rowbuf, ul, wl, owner, Phi, m_in, m_out);
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int j = 0; j < VB; ++j) flux[r][j] = fma(sa, Phi[r][j], flux[r][j]);
      if (owner)
        face_moments_add<D, T>(a.Facc + size_t(inc[i].face) * FACC_W,
                               reinterpret_cast<const double*>(fsl + FS::ROW + FS::SP + FS::SG), fg.bc_type == 1,
                               first, m_in, m_out, lane);
    }
    const unsigned char* own = B + W * FS::BYTES;
    T g0[VB];
    slot_refs<D, NR, VB, T, S>(own, v, g0);
    const T lam = E.lam, beta0 = E.beta, pref = E.pref, s0 = E.s0, kap = E.kap, inv_vol = E.inv_vol;
    const size_t base = size_t(m0) * sj + size_t(c) * BV + lane;
#pragma unroll
    for (int j = 0; j < VB; ++j) {
      T c2 = T(0), cq = T(0);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const T cd = v.u[j][d] - E.U[d];
        c2 += cd * cd;
        cq += cd * E.q[d];
      }
      const T H = pref * t_exp(-lam * c2);
      const T s = s0 * cq;
      T fp[NR];
      fp[0] = H * (T(1) + s * (T(2) * lam * c2 - T(2 + D)));
      if (NR == 2) fp[NR - 1] = kap * H * (T(1) + s * (T(2) * lam * c2 - T(D)));
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const T f = slot_value<NR, VB, T, S>(own, r, j, lane, g0);
        const T ft = v.real[j] ? f - flux[r][j] * inv_vol + beta0 * (fp[r] - f) : T(0);
        if constexpr (SL::SCALED) {
          // f~ is stored against the same reference as f^n
          const RefMaxwell& Rf = *reinterpret_cast<const RefMaxwell*>(own + SL::ROWS + SL::SCL);
          float scale;
          const S d = encode_value<S>(ft, r == 0 ? g0[j] : Rf.kap * g0[j], scale);
          reinterpret_cast<S*>(a.f_next)[base + r * sr + j * sj] = d;
          if (lane == 0) a.sc_next[(size_t(r) * a.M + m0 + j) * a.Nc + c] = scale;
        } else {
          a.f_next[base + r * sr + j * sj] = ft;
        }
      }
    }
    __syncwarp();
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Wall density from non-penetration (Eq. 38) and the completed wall moments.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_bwall(const BlockedArgs<T> a) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= a.Nf) return;
  double* F = a.Facc + size_t(f) * FACC_W;
  if constexpr (sizeof(T) == 4) {
    // float pairs of the FP32 sweep (facc_add) -> doubles
    const bool wall = a.fg[f].bc_type == 1;
    for (int t = 0; t < 10; ++t)
      if (t < a.g.D + 2 || (wall && t >= 5 && t < 5 + a.g.D + 2)) {
        const float2 p = *reinterpret_cast<const float2*>(F + t);
        F[t] = double(p.x) + double(p.y);
      }
  }
  if (a.fg[f].bc_type != 1) return;
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
    a.ceq1[c] = make_cell_eq<D, T>(a.g, pn, a.vol[c]);
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
// Second stage (Eq. 42) over one chunk of velocity rows, with the outgoing
// wall flux rho_w g_w (known only after the sweep), and the chunk's partial
// sums of the heat flux of f^{n+1} (Eq. 13).  A streaming pass over f~: a CTA
// owns 32 consecutive cells, whose rows of one velocity block are one
// contiguous segment (4 KB in FP32).  A producer warp stages the chunk's rows
// into a ring of shared-memory stages with 1-D bulk asynchronous copies
// (completion counted in bytes on an mbarrier per stage); 8 consumer warps
// (8 threads per cell, 4 consecutive velocities each) read their values,
// release the stage, update and write f^{n+1} in place.  On tensor grids
// whose fastest axis has 32 points (a row is one line along that axis) the
// Maxwellians factor into a per-row part (one exponential per row and thread)
// and the thread's four lane parts (computed once), and the heat-flux sums
// factor the same way.
// ---------------------------------------------------------------------------
constexpr int kS2Consumers = 256;                    // 8 warps: 32 cells x 8 threads
constexpr int kS2Threads = kS2Consumers + 32;        // and one producer warp
constexpr int kS2Cells = kS2Consumers / 8;           // cells per CTA
constexpr int kS2Flush = 8;                          // rows between flushes of the FP32 heat-flux partials

template <int NR, typename S>
struct S2Ring {
  static constexpr int ROW = kS2Cells * BV * int(sizeof(S));   // one row (r, m) of the CTA's cells
  static constexpr int STAGE = NR * ROW;
  static constexpr int NST = (32 * 1024 / STAGE) < 2 ? 2 : (32 * 1024 / STAGE) > 8 ? 8 : (32 * 1024 / STAGE);
  static constexpr int BYTES = NST * STAGE + 2 * NST * 8;        // stages, then full and empty barriers
};

// Four consecutive stored values of one row (the thread's velocities).
template <typename S>
struct Quad {
  S v[4];
};
template <typename S>
__device__ __forceinline__ Quad<S> quad_lds(const unsigned char* p) {
  Quad<S> q;
  if constexpr (sizeof(S) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    q.v[0] = t.x, q.v[1] = t.y, q.v[2] = t.z, q.v[3] = t.w;
  } else if constexpr (sizeof(S) == 8) {
    const double2 t0 = reinterpret_cast<const double2*>(p)[0];
    const double2 t1 = reinterpret_cast<const double2*>(p)[1];
    q.v[0] = t0.x, q.v[1] = t0.y, q.v[2] = t1.x, q.v[3] = t1.y;
  } else {
    const uint2 t = *reinterpret_cast<const uint2*>(p);
    const S* h = reinterpret_cast<const S*>(&t);
    q.v[0] = h[0], q.v[1] = h[1], q.v[2] = h[2], q.v[3] = h[3];
  }
  return q;
}
template <typename S>
__device__ __forceinline__ void quad_store(S* p, const Quad<S>& q) {
  if constexpr (sizeof(S) == 4) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(q.v[0], q.v[1], q.v[2], q.v[3]));
  } else if constexpr (sizeof(S) == 8) {
    __stcs(reinterpret_cast<double2*>(p), make_double2(q.v[0], q.v[1]));
    __stcs(reinterpret_cast<double2*>(p) + 1, make_double2(q.v[2], q.v[3]));
  } else {
    uint2 t;
    S* h = reinterpret_cast<S*>(&t);
    h[0] = q.v[0], h[1] = q.v[1], h[2] = q.v[2], h[3] = q.v[3];
    __stcs(reinterpret_cast<uint2*>(p), t);
  }
}

// Maximum over the 8 threads of one cell (lanes 8k .. 8k+7 of the warp).
__device__ __forceinline__ float max8(float v) {
  v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 1));
  v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 2));
  return fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 4));
}

// The first diffuse-wall face of a cell, held in registers by the second
// stage: its re-emitted flux at velocity u is coef (u.n) exp(-lam |u - U|^2)
// for u.n < 0 (and kappa times that for b), coef = area/|Omega| dt rho_w
// rho_pref (Eq. 36-38).
template <typename T>
struct WallEmit {
  T coef, lam, kap;
  T n[3], U[3];
};

// Launched twice per step: WALL = false handles the CTAs without a wall cell,
// WALL = true the CTAs holding one (threads of their other cells carry
// coef = 0); each launch returns at once for the other kind, so the common
// kind keeps the registers of the wall terms free.
template <int D, int NR, bool TENSOR, bool WALL, typename T, typename S>
__global__ void __launch_bounds__(kS2Threads, sizeof(T) == 4 && NR == 1 && !WALL ? 3 : 2) k_bstage2(const BlockedArgs<T> a) {
  constexpr bool SCALED = StoreTraits<S>::scaled;
  using RG = S2Ring<NR, S>;
  extern __shared__ __align__(128) unsigned char s2_smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(s2_smem + RG::NST * RG::STAGE);
  uint64_t* empty = full + RG::NST;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool producer = warp == kS2Consumers / 32;
  const int qd_ = threadIdx.x & 7;                     // velocities 4 qd_ .. 4 qd_ + 3 of every row
  const int cl0 = (threadIdx.x >> 3) & (kS2Cells - 1); // the thread's cell within the CTA
  const int c0 = blockIdx.x * kS2Cells;
  const int ncta = a.Nc - c0 < kS2Cells ? a.Nc - c0 : kS2Cells;
  const int c = c0 + cl0;
  const bool valid = !producer && cl0 < ncta;
  const int cc = valid ? c : c0;
  const int chunk = blockIdx.y;
  const int64_t per = (a.M + a.nchunk - 1) / a.nchunk;
  const int64_t mb = int64_t(chunk) * per;
  const int64_t me = mb + per < a.M ? mb + per : a.M;
  const int nrow = me > mb ? int(me - mb) : 0;
  const size_t sj = size_t(a.Nc) * BV, sr = size_t(a.M) * sj;

  // diffuse-wall faces of the cell: the first in registers, further ones
  // (rare) re-read per row
  const int e0 = a.cf_off[cc], e1 = a.cf_off[cc + 1];
  int nwall = 0, ewall = -1;
  if (valid)
    for (int e = e0; e < e1; ++e)
      if (a.inc[e].flags & 1) {
        if (nwall == 0) ewall = e;
        ++nwall;
      }
  if ((__syncthreads_or(nwall > 0) != 0) != WALL) return;   // CTA-uniform
  if (threadIdx.x == 0) {
    for (int st = 0; st < RG::NST; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], kS2Consumers / 32);
    }
    mbar_init_fence();
  }
  __syncthreads();

  if (producer) {
    if (lane != 0) return;
    const S* src = reinterpret_cast<const S*>(a.f_next) + size_t(c0) * BV;
    const unsigned bytes = unsigned(ncta) * BV * unsigned(sizeof(S));   // a multiple of 16
    int issued = 0;
    for (int i = 0; i < nrow; ++i) {
      const int st = i % RG::NST;
      if (i >= RG::NST && !mbar_wait(&empty[st], unsigned((i / RG::NST) - 1) & 1u, a.status)) break;
      mbar_arrive_expect_tx(&full[st], NR * bytes);
#pragma unroll
      for (int r = 0; r < NR; ++r)
        bulk_load(s2_smem + st * RG::STAGE + r * RG::ROW, src + r * sr + (mb + i) * sj, bytes, &full[st]);
      issued = i + 1;
    }
    // the CTA's shared memory must outlive every copy issued into it
    for (int i = issued > RG::NST ? issued - RG::NST : 0; i < issued; ++i)
      if (!mbar_wait(&full[i % RG::NST], unsigned(i / RG::NST) & 1u, a.status)) break;
    return;
  }

  S* fc = reinterpret_cast<S*>(a.f_next) + size_t(cc) * BV + 4 * qd_;
  const CellEq<T> E = a.ceq1[cc];
  RefMaxwell Rc{};  // reference of f~ (scaled storage)
  if constexpr (SCALED) {
    Rc = a.ref_cur[cc];
    if (valid && chunk == 0 && qd_ == 0) {
      // f^{n+1} is stored against the Maxwellian of W^{n+1}
      RefMaxwell Rn;
      Rn.pref = E.pref;
      Rn.lam = E.lam;
      Rn.U[0] = E.U[0];
      Rn.U[1] = E.U[1];
      Rn.U[2] = E.U[2];
      Rn.kap = E.kap;
      Rn.pad[0] = Rn.pad[1] = 0.f;
      a.ref_next[c] = Rn;
    }
  }
  const T lam = E.lam, beta1 = E.beta, pref = E.pref, s0 = E.s0, kap = E.kap, iv = E.inv_vol;
  const T inv1 = T(1) / (T(1) + beta1);
  const T tl = T(2) * lam;
  WallEmit<T> wf{};
  if (WALL && nwall > 0) {
    const int fidx = a.inc[ewall].face;
    const FaceGeom<T>& fg = a.fg[fidx];
    const FacePoly<D, NR, T>& R = static_cast<const FacePoly<D, NR, T>*>(a.fpoly)[fidx];
    wf.coef = a.inc[ewall].sarea * iv * T(a.g.dt) * T(a.Facc[size_t(fidx) * FACC_W + 10]) * R.rho_pref;
    wf.lam = R.lam;
    wf.kap = R.kappa;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      wf.n[d] = d < D ? fg.n[d] : T(0);
      wf.U[d] = d < D ? R.U[d] : T(0);
    }
  }

  // lane parts (tensor grids): c along the lane axis, its Maxwellian factors
  // (the cell's, that of the reference of f~, the wall's), the lane weight
  T cl[4], El[4], wl[4], Er[4], Ew[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    cl[i] = El[i] = wl[i] = Er[i] = Ew[i] = T(0);
    if constexpr (TENSOR) {
      const T ul = a.lanev[4 * qd_ + i];
      wl[i] = a.lanev[BV + 4 * qd_ + i];
      cl[i] = ul - E.U[0];
      El[i] = t_exp(-lam * cl[i] * cl[i]);
      if constexpr (SCALED) Er[i] = t_exp(-T(Rc.lam) * (ul - T(Rc.U[0])) * (ul - T(Rc.U[0])));
      if constexpr (WALL) Ew[i] = t_exp(-wf.lam * (ul - wf.U[0]) * (ul - wf.U[0]));
    }
  }
  // heat-flux partial sums: FP32 for kS2Flush rows, then into float pairs
  // (FP32 sweeps) or doubles (FP64 sweep)
  T qp[3] = {T(0), T(0), T(0)};
  float2 qf[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  double qdd[3] = {0.0, 0.0, 0.0};
  int since_flush = 0;
  const unsigned char* mine = s2_smem + (cl0 * BV + 4 * qd_) * int(sizeof(S));

  for (int i = 0; i < nrow; ++i) {
    const int64_t m = mb + i;
    const int st = i % RG::NST;
    if (!mbar_wait(&full[st], unsigned(i / RG::NST) & 1u, a.status)) break;
    Quad<S> x[NR];
    float sc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      x[r] = quad_lds<S>(mine + st * RG::STAGE + r * RG::ROW);
      if constexpr (SCALED) sc[r] = a.sc_next[(size_t(r) * a.M + m) * a.Nc + cc];
    }

    // row part of the velocities (tensor grids)
    T crow[3] = {T(0), T(0), T(0)}, c2row = T(0), cqrow = T(0), Hrow = pref, Grow = T(0), wrow = T(0);
    T unrow = T(0), Wrow = T(0);
    Vel4<T> rv{};
    if constexpr (TENSOR) {
      rv = a.rowv[m];
      const T ur[3] = {T(0), rv.y, rv.z};
#pragma unroll
      for (int d = 1; d < D; ++d) {
        crow[d] = ur[d] - E.U[d];
        c2row += crow[d] * crow[d];
        cqrow += crow[d] * E.q[d];
      }
      Hrow = pref * t_exp(-lam * c2row);
      wrow = T(0.5) * rv.w;
      if constexpr (SCALED) {
        T g2 = T(0);
#pragma unroll
        for (int d = 1; d < D; ++d) g2 += (ur[d] - T(Rc.U[d])) * (ur[d] - T(Rc.U[d]));
        Grow = T(Rc.pref) * t_exp(-T(Rc.lam) * g2);
      }
      if constexpr (WALL) {
        // u.n = n0 (c_lane + U0) + n1 u1 + n2 u2, and the wall Maxwellian's row factor
        T w2 = T(0);
        unrow = wf.n[0] * E.U[0];
#pragma unroll
        for (int d = 1; d < D; ++d) {
          unrow = fma(wf.n[d], ur[d], unrow);
          w2 += (ur[d] - wf.U[d]) * (ur[d] - wf.U[d]);
        }
        Wrow = wf.coef * t_exp(-wf.lam * w2);
      }
    }
    T Se = T(0), Sl = T(0);   // tensor: sum of e and of c_lane e over the thread's 4 velocities
    // per velocity: the cell's Maxwellian H of W^{n+1}, |c|^2, c.q, the
    // weight; f~ decoded; then the wall's re-emitted flux subtracted
    T ft[4][NR], c2v[4], cqv[4], Hv[4], wv[4], uv[4][3];
    bool real_v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t k = m * BV + 4 * qd_ + j;
      T g = T(0);
      real_v[j] = true;
      uv[j][0] = uv[j][1] = uv[j][2] = T(0);
      if constexpr (TENSOR) {
        c2v[j] = fma(cl[j], cl[j], c2row);
        cqv[j] = fma(cl[j], E.q[0], cqrow);
        Hv[j] = Hrow * El[j];
        wv[j] = wl[j];
        if constexpr (SCALED) g = Grow * Er[j];
      } else {
        const Vel4<T> vq = a.vel[k];
        uv[j][0] = vq.x;
        uv[j][1] = D > 1 ? vq.y : T(0);
        uv[j][2] = D > 2 ? vq.z : T(0);
        real_v[j] = k < a.nv;
        T c2 = T(0), cq = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const T cd = uv[j][d] - E.U[d];
          c2 += cd * cd;
          cq += cd * E.q[d];
        }
        c2v[j] = c2;
        cqv[j] = cq;
        Hv[j] = real_v[j] ? pref * t_exp(-lam * c2) : T(0);
        wv[j] = T(0.5) * vq.w;   // zero on padding
        if constexpr (SCALED) {
          const float uf[3] = {float(uv[j][0]), float(uv[j][1]), float(uv[j][2])};
          g = ref_value<D>(Rc, 0, uf, real_v[j]);
        }
      }
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if constexpr (SCALED)
          ft[j][r] = decode_value(x[r].v[j], sc[r], r == 0 ? g : T(Rc.kap) * g);
        else
          ft[j][r] = T(x[r].v[j]);
      }
      if constexpr (WALL) {
        T un, ew;
        if constexpr (TENSOR) {
          un = fma(wf.n[0], cl[j], unrow);
          ew = Wrow * Ew[j];
        } else {
          T w2 = T(0);
          un = T(0);
#pragma unroll
          for (int d = 0; d < D; ++d) {
            un = fma(wf.n[d], uv[j][d], un);
            w2 += (uv[j][d] - wf.U[d]) * (uv[j][d] - wf.U[d]);
          }
          ew = wf.coef * t_exp(-wf.lam * w2);
        }
        const T out = un < T(0) ? un * ew : T(0);
        ft[j][0] -= out;
        if (NR == 2) ft[j][NR - 1] -= wf.kap * out;
      }
    }
    // The stage is released for refilling only after the decode above has
    // consumed the values read from it, behind a proxy fence: a release issued
    // right after the shared-memory loads let the bulk copy of row i + NST
    // overwrite the stage before those loads had returned.
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
    if constexpr (WALL) {
      // further wall faces of the cell (rare): records re-read per row
      if (nwall > 1) {
        if constexpr (TENSOR) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            uv[j][0] = a.lanev[4 * qd_ + j];
            uv[j][1] = rv.y;
            uv[j][2] = rv.z;
          }
        }
        const T dt = T(a.g.dt);
        for (int e = e0; e < e1; ++e) {
          if (e == ewall || !(a.inc[e].flags & 1)) continue;
          const int fidx = a.inc[e].face;
          const FaceGeom<T>& fg = a.fg[fidx];
          const FacePoly<D, NR, T>& R = static_cast<const FacePoly<D, NR, T>*>(a.fpoly)[fidx];
          const T coef = a.inc[e].sarea * iv * dt * T(a.Facc[size_t(fidx) * FACC_W + 10]) * R.rho_pref;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            T un = T(0), w2 = T(0);
#pragma unroll
            for (int d = 0; d < D; ++d) {
              un = fma(fg.n[d], uv[j][d], un);
              w2 += (uv[j][d] - R.U[d]) * (uv[j][d] - R.U[d]);
            }
            const T out = un < T(0) ? coef * un * t_exp(-R.lam * w2) : T(0);
            ft[j][0] -= out;
            if (NR == 2) ft[j][NR - 1] -= R.kappa * out;
          }
        }
      }
    }
    T f1[4][NR];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const T s = s0 * cqv[j];
      const T bh = beta1 * Hv[j];
      f1[j][0] = (ft[j][0] + bh * fma(s, fma(tl, c2v[j], -T(2 + D)), T(1))) * inv1;
      if (NR == 2) f1[j][NR - 1] = (ft[j][NR - 1] + kap * bh * fma(s, fma(tl, c2v[j], -T(D)), T(1))) * inv1;
#pragma unroll
      for (int r = 0; r < NR; ++r) f1[j][r] = real_v[j] ? f1[j][r] : T(0);
      const T e_ = wv[j] * fma(c2v[j], f1[j][0], NR == 2 ? f1[j][NR - 1] : T(0));
      if constexpr (TENSOR) {
        Se += e_;
        Sl = fma(cl[j], e_, Sl);
      } else {
#pragma unroll
        for (int d = 0; d < D; ++d) qp[d] = fma(uv[j][d] - E.U[d], e_, qp[d]);
      }
    }
    if constexpr (TENSOR) {
      qp[0] = fma(Sl, wrow, qp[0]);
      const T sw = Se * wrow;
#pragma unroll
      for (int d = 1; d < D; ++d) qp[d] = fma(crow[d], sw, qp[d]);
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      Quad<S> y;
      if constexpr (SCALED) {
        float dev[4], mx = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          dev[j] = f1[j][r] - (r == 0 ? Hv[j] : kap * Hv[j]);
          mx = fmaxf(mx, fabsf(dev[j]));
        }
        float scale = max8(mx);
        if (scale < kScaleFloor) scale = 0.f;
        const float inv = scale > 0.f ? 1.f / scale : 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) y.v[j] = StoreTraits<S>::from_f(dev[j] * inv);
        if (qd_ == 0 && valid) a.sc_next[(size_t(r) * a.M + m) * a.Nc + cc] = scale;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) y.v[j] = S(f1[j][r]);
      }
      if (valid) quad_store(fc + r * sr + m * sj, y);
    }
    if (++since_flush == kS2Flush) {
      since_flush = 0;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        if constexpr (sizeof(T) == 4)
          qf[d] = pair_add(qf[d], float(qp[d]));
        else
          qdd[d] += double(qp[d]);
        qp[d] = T(0);
      }
    }
  }

  // sum over the cell's 8 threads
#pragma unroll
  for (int d = 0; d < D; ++d) {
    if constexpr (sizeof(T) == 4) {
      float2 v = pair_add(qf[d], float(qp[d]));
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        const float2 w = make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
        v = pair_add(v, w);
      }
      qdd[d] = double(v.x) + double(v.y);
    } else {
      double v = qdd[d] + double(qp[d]);
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      qdd[d] = v;
    }
  }
  if (!valid || qd_ != 0) return;
  double* qo = a.qpart + (size_t(chunk) * a.Nc + c) * 3;
  qo[0] = qdd[0];
  qo[1] = D > 1 ? qdd[D > 1 ? 1 : 0] : 0.0;
  qo[2] = D > 2 ? qdd[D > 2 ? 2 : 0] : 0.0;
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

// Persistent launch of a pipelined per-cell kernel with `bytes` of shared
// memory per warp: warps per CTA chosen so that a CTA needs at most 100 KB.
template <typename K>
cudaError_t launch_cell_pipelined(K kernel, int nsm, int bytes, int& warps_out, unsigned& grid_out) {
  int warps = kBlockedThreads / 32;
  while (warps > 1 && warps * bytes > 100 * 1024) warps /= 2;
  const int smem = warps * bytes;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, warps * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  warps_out = warps;
  grid_out = unsigned(int64_t(per_sm) * nsm);  // CTAs resident on the whole GPU
  return cudaSuccess;
}

// Per-warp shared memory above which the pipelined kernels are not used.
constexpr int kPipelineWarpBytes = 24 * 1024;

// Launch of a pipelined per-cell kernel: warps per CTA and the persistent grid
// are worked out once per instantiation and per-warp size.
template <typename T, typename K>
cudaError_t launch_cell_cached(K kernel, cudaStream_t s, const BlockedArgs<T>& a, int64_t m0, int bytes,
                               int& cached_bytes, int& cached_warps, unsigned& cached_grid) {
  if (cached_bytes != bytes) {
    cudaError_t e = launch_cell_pipelined(kernel, a.nsm, bytes, cached_warps, cached_grid);
    if (e != cudaSuccess) return e;
    cached_bytes = bytes;
  }
  const unsigned grid = std::min<unsigned>(cached_grid, unsigned((a.Nc + cached_warps - 1) / cached_warps));
  kernel<<<grid, cached_warps * 32, cached_warps * bytes, s>>>(a, m0);
  return cudaGetLastError();
}

// The pipelined kernels are compiled for ELL widths 4 and 8 (the host pads
// the table to one of them); other widths and oversize stages use the plain
// kernels.
template <int D, int NR, int VB, typename T, typename S>
cudaError_t launch_brecon_tpl(cudaStream_t s, const BlockedArgs<T>& a, int64_t m0) {
  const int bytes = recon_warp_bytes<NR, VB, T, S>(a.W);
  if ((a.W != 4 && a.W != 8) || bytes > kPipelineWarpBytes) {
    if constexpr (StoreTraits<S>::scaled) {
      return cudaErrorNotSupported;  // scaled storage runs only in the pipelined kernels
    } else {
      k_brecon<D, NR, VB, T><<<blocked_warp_grid(a.Nc), kBlockedThreads, 0, s>>>(a, m0);
      return cudaGetLastError();
    }
  }
  static int cb4 = -1, cw4 = 0, cb8 = -1, cw8 = 0;
  static unsigned cg4 = 0, cg8 = 0;
  if (a.W == 4) return launch_cell_cached<T>(k_brecon_p<D, NR, VB, 4, T, S>, s, a, m0, bytes, cb4, cw4, cg4);
  return launch_cell_cached<T>(k_brecon_p<D, NR, VB, 8, T, S>, s, a, m0, bytes, cb8, cw8, cg8);
}

template <int D, int NR, int VB, typename T, typename S>
cudaError_t launch_bstage1_tpl(cudaStream_t s, const BlockedArgs<T>& a, int64_t m0) {
  const int bytes = stage1_warp_bytes<NR, VB, T, S>(a.W);
  if ((a.W != 4 && a.W != 8) || bytes > kPipelineWarpBytes) {
    if constexpr (StoreTraits<S>::scaled) {
      return cudaErrorNotSupported;
    } else {
      k_bstage1<D, NR, VB, T><<<blocked_warp_grid(a.Nc), kBlockedThreads, 0, s>>>(a, m0);
      return cudaGetLastError();
    }
  }
  static int cb4 = -1, cw4 = 0, cb8 = -1, cw8 = 0;
  static unsigned cg4 = 0, cg8 = 0;
  if (a.W == 4) return launch_cell_cached<T>(k_bstage1_p<D, NR, VB, 4, T, S>, s, a, m0, bytes, cb4, cw4, cg4);
  return launch_cell_cached<T>(k_bstage1_p<D, NR, VB, 8, T, S>, s, a, m0, bytes, cb8, cw8, cg8);
}

// The fused flux and first-stage kernel; cudaErrorNotSupported where it does
// not apply (ELL widths other than 4 and 8, or stages beyond the per-warp
// shared-memory bound): the caller then runs the flux and first-stage kernels.
// Per-warp shared memory above which the fused kernel is not used.
constexpr int kFusedWarpBytes = 48 * 1024;

template <int D, int NR, int VB, typename T, typename S>
bool bstage1f_fits(const BlockedArgs<T>& a) {
  return (a.W == 4 || a.W == 8) && stage1f_warp_bytes<D, NR, VB, T, S>(a.W) <= kFusedWarpBytes;
}

template <int D, int NR, int VB, typename T, typename S>
cudaError_t launch_bstage1f_tpl(cudaStream_t s, const BlockedArgs<T>& a, int64_t m0, int first) {
  const int bytes = stage1f_warp_bytes<D, NR, VB, T, S>(a.W);
  if (!bstage1f_fits<D, NR, VB, T, S>(a)) return cudaErrorNotSupported;
  static int cb4 = -1, cw4 = 0, cb8 = -1, cw8 = 0;
  static unsigned cg4 = 0, cg8 = 0;
  auto run = [&](auto kernel, int& cb, int& cw, unsigned& cg) -> cudaError_t {
    if (cb != bytes) {
      cudaError_t e = launch_cell_pipelined(kernel, a.nsm, bytes, cw, cg);
      if (e != cudaSuccess) return e;
      cb = bytes;
    }
    const unsigned grid = std::min<unsigned>(cg, unsigned((a.Nc + cw - 1) / cw));
    kernel<<<grid, cw * 32, cw * bytes, s>>>(a, m0, first);
    return cudaGetLastError();
  };
  if (a.W == 4) return run(k_bstage1f<D, NR, VB, 4, T, S>, cb4, cw4, cg4);
  return run(k_bstage1f<D, NR, VB, 8, T, S>, cb8, cw8, cg8);
}

#define UGKS_CELL_CASES(FN)                                                                               \
  FN(1, 2, 1) FN(1, 2, 2) FN(1, 2, 4) FN(2, 2, 1) FN(2, 2, 2) FN(2, 2, 4) FN(3, 1, 1) FN(3, 1, 2) FN(3, 1, 4) \
  FN(3, 1, 8) \
  FN(3, 2, 1) FN(3, 2, 2) FN(3, 2, 4)

template <typename T, typename S>
cudaError_t launch_brecon(cudaStream_t s, const BlockedArgs<T>& a, int64_t m0, int vb) {
  const int D = a.g.D, NR = a.g.NR;
#define UGKS_RECON_CASE(d, nr, b) \
  if (D == d && NR == nr && vb == b) return launch_brecon_tpl<d, nr, b, T, S>(s, a, m0);
  UGKS_CELL_CASES(UGKS_RECON_CASE)
#undef UGKS_RECON_CASE
  return cudaErrorInvalidValue;
}

// Persistent launch of the flux kernel: as many CTAs as fit on the GPU
// (occupancy with the kernel's shared-memory stages), at most one warp per face.
template <int D, int NR, int VB, typename T>
cudaError_t launch_bflux_tpl(cudaStream_t s, const BlockedArgs<T>& a, int64_t m0, int first) {
  constexpr int smem = (kBlockedThreads / 32) * (2 * FluxStage<D, NR, VB, T>::BYTES + VB * int(sizeof(RowFac<NR, T>)));
  static int per_sm = 0;  // per instantiation, computed on first use
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(k_bflux<D, NR, VB, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bflux<D, NR, VB, T>, kBlockedThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
  }
  const unsigned grid = unsigned(std::min<int64_t>(int64_t(per_sm) * a.nsm, blocked_warp_grid(a.Nf)));
  k_bflux<D, NR, VB, T><<<grid, kBlockedThreads, smem, s>>>(a, m0, first);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bflux(cudaStream_t s, const BlockedArgs<T>& a, int64_t m0, int vb, int first) {
  const int D = a.g.D, NR = a.g.NR;
#define UGKS_FLUX_CASE(d, nr, b) \
  if (D == d && NR == nr && vb == b) return launch_bflux_tpl<d, nr, b, T>(s, a, m0, first);
  UGKS_FLUX_CASE(1, 2, 1) UGKS_FLUX_CASE(1, 2, 2) UGKS_FLUX_CASE(1, 2, 4)
  UGKS_FLUX_CASE(2, 2, 1) UGKS_FLUX_CASE(2, 2, 2) UGKS_FLUX_CASE(2, 2, 4)
  UGKS_FLUX_CASE(3, 1, 1) UGKS_FLUX_CASE(3, 1, 2) UGKS_FLUX_CASE(3, 1, 4) UGKS_FLUX_CASE(3, 1, 8)
  UGKS_FLUX_CASE(3, 2, 1) UGKS_FLUX_CASE(3, 2, 2) UGKS_FLUX_CASE(3, 2, 4)
#undef UGKS_FLUX_CASE
  return cudaErrorInvalidValue;
}

template <typename T, typename S>
cudaError_t launch_bstage1(cudaStream_t s, const BlockedArgs<T>& a, int64_t m0, int vb) {
  const int D = a.g.D, NR = a.g.NR;
#define UGKS_STAGE1_CASE(d, nr, b) \
  if (D == d && NR == nr && vb == b) return launch_bstage1_tpl<d, nr, b, T, S>(s, a, m0);
  UGKS_CELL_CASES(UGKS_STAGE1_CASE)
#undef UGKS_STAGE1_CASE
  return cudaErrorInvalidValue;
}

template <typename T, typename S>
bool bstage1f_supported(const BlockedArgs<T>& a, int vb) {
  const int D = a.g.D, NR = a.g.NR;
#define UGKS_STAGE1F_Q(d, nr, b) \
  if (D == d && NR == nr && vb == b) return bstage1f_fits<d, nr, b, T, S>(a);
  UGKS_CELL_CASES(UGKS_STAGE1F_Q)
#undef UGKS_STAGE1F_Q
  return false;
}

template <typename T, typename S>
cudaError_t launch_bstage1f(cudaStream_t s, const BlockedArgs<T>& a, int64_t m0, int vb, int first) {
  const int D = a.g.D, NR = a.g.NR;
#define UGKS_STAGE1F_CASE(d, nr, b) \
  if (D == d && NR == nr && vb == b) return launch_bstage1f_tpl<d, nr, b, T, S>(s, a, m0, first);
  UGKS_CELL_CASES(UGKS_STAGE1F_CASE)
#undef UGKS_STAGE1F_CASE
  return cudaErrorInvalidValue;
}

#undef UGKS_BLOCKED_DISPATCH

template <typename T>
cudaError_t launch_bcelleq(cudaStream_t s, const BlockedArgs<T>& a) {
  const unsigned nb = unsigned((a.Nc + 255) / 256);
  if (a.g.D == 1) k_bcelleq<1, T><<<nb, 256, 0, s>>>(a);
  else if (a.g.D == 2) k_bcelleq<2, T><<<nb, 256, 0, s>>>(a);
  else if (a.g.D == 3) k_bcelleq<3, T><<<nb, 256, 0, s>>>(a);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

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

template <int D, int NR, bool TENSOR, typename T, typename S>
cudaError_t launch_bstage2_tpl(cudaStream_t s, const BlockedArgs<T>& a) {
  constexpr int smem = S2Ring<NR, S>::BYTES;
  static bool attr = false;   // per instantiation
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_bstage2<D, NR, TENSOR, false, T, S>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_bstage2<D, NR, TENSOR, true, T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const dim3 grid(unsigned((a.Nc + kS2Cells - 1) / kS2Cells), unsigned(a.nchunk));
  k_bstage2<D, NR, TENSOR, false, T, S><<<grid, kS2Threads, smem, s>>>(a);
  k_bstage2<D, NR, TENSOR, true, T, S><<<grid, kS2Threads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, typename S>
cudaError_t launch_bstage2(cudaStream_t s, const BlockedArgs<T>& a) {
  const int D = a.g.D, NR = a.g.NR;
  const bool ten = a.tensor != 0;
  cudaError_t e = cudaErrorInvalidValue;
#define UGKS_S2(d, nr)                                                                     \
  if (D == d && NR == nr)                                                                  \
    e = ten ? launch_bstage2_tpl<d, nr, true, T, S>(s, a) : launch_bstage2_tpl<d, nr, false, T, S>(s, a);
  UGKS_S2(1, 2) UGKS_S2(2, 2) UGKS_S2(3, 1) UGKS_S2(3, 2)
#undef UGKS_S2
  if (e != cudaSuccess) return e;
  k_bqsum<T><<<unsigned((int64_t(a.Nc) * 3 + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

#define UGKS_INSTANTIATE_BLOCKED(T)                                                                  \
  template cudaError_t launch_brecon<T, T>(cudaStream_t, const BlockedArgs<T>&, int64_t, int);       \
  template cudaError_t launch_bflux<T>(cudaStream_t, const BlockedArgs<T>&, int64_t, int, int);     \
  template cudaError_t launch_bstage1<T, T>(cudaStream_t, const BlockedArgs<T>&, int64_t, int);     \
  template cudaError_t launch_bstage1f<T, T>(cudaStream_t, const BlockedArgs<T>&, int64_t, int, int); \
  template bool bstage1f_supported<T, T>(const BlockedArgs<T>&, int);                                \
  template cudaError_t launch_bcelleq<T>(cudaStream_t, const BlockedArgs<T>&);                       \
  template cudaError_t launch_bconserve<T>(cudaStream_t, const BlockedArgs<T>&);                     \
  template cudaError_t launch_bstage2<T, T>(cudaStream_t, const BlockedArgs<T>&);

// FP32 arithmetic with FP16 / BF16 scaled storage: the kernels that read or
// write f (the flux kernel reads only the per-face buffer).
#define UGKS_INSTANTIATE_SCALED(S)                                                                   \
  template cudaError_t launch_brecon<float, S>(cudaStream_t, const BlockedArgs<float>&, int64_t, int);   \
  template cudaError_t launch_bstage1<float, S>(cudaStream_t, const BlockedArgs<float>&, int64_t, int);  \
  template cudaError_t launch_bstage1f<float, S>(cudaStream_t, const BlockedArgs<float>&, int64_t, int, int); \
  template bool bstage1f_supported<float, S>(const BlockedArgs<float>&, int);                           \
  template cudaError_t launch_bstage2<float, S>(cudaStream_t, const BlockedArgs<float>&);

}  // namespace ugks
