// Internal device data layout of the GB300 UGKS library.
//
// Distribution storage (Sec. 2.2.2, Eq. 47-48): the padded velocity set is
// split into blocks of BV = 32 points, one warp lane per velocity, and each
// reduced distribution r (h, then b) is stored block-major with the velocity
// innermost:  f[r][m][cell][lane], so that one (r, m, cell) row is a single
// contiguous 32-element segment (128 B in FP32, 256 B in FP64).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ugks {

constexpr int BV = 32;      // velocity block = warp width
constexpr int NWP = 5;      // stride of conservative vectors (dim + 2 <= 5)
constexpr int MAXF = 32;    // faces per cell
constexpr int FACC_W = 12;  // per-face accumulator: [0,5) flux, [5,10) wall unit-outflow moments, 10 rho_w

// Per-cell primitive record, FP64 (computed each step from W).
struct CellPrim {
  double rho, U[3], lam, tau;
  double q[3];
  double pad;
};

// Per-cell incidence entry (CSR over cells): one per face of the cell.
struct CellFace {
  int64_t face;    // global face index
  int64_t other;   // neighbour cell (renumbered) or -(bc+1)
  double w[3];     // least-squares weight M^-1 d (zero for walls)
  double r[3];     // face centroid minus cell centroid (cell's frame)
  double area;
  int32_t sign;    // +1 owner, -1 neighbour
  int32_t bc_type; // 0 interior, else UGKS_BC_*
};

// Same entry in the storage/compute precision of the sweep kernel (16-byte
// aligned so that a copy to registers is a few vector loads).
template <typename T>
struct __align__(16) CellFaceT {
  T w[3];
  T r[3];
  T area;
  int64_t other;
  int32_t bc;      // -1 interior, else bc index
  int32_t flags;   // bit 0: wall
};

// Constant per-face geometry in the sweep precision.
template <typename T>
struct __align__(16) FaceGeom {
  T n[3];          // unit normal owner -> neighbour
  T rl[3];         // face centroid - owner centroid
  T rr[3];         // face centroid - neighbour centroid (neighbour's frame), or 0
  T area;
  int64_t own, nei;   // renumbered cells; nei < 0: -(bc+1)
  int32_t bc_type;    // 0 interior
  int32_t pad;
};

// Per-step interface coefficients in the sweep precision (Eq. 32-35).
// Interior / far-field / outflow faces: interface Maxwellian g0 and its
// slopes.  Wall faces: the unit-density wall Maxwellian (rho_pref, U, lam,
// kappa) and zero elsewhere.
template <typename T>
struct __align__(16) FaceRec {
  T G[5];          // integrals of c1..c5 over [0, dt]
  T rho_pref;      // rho0 (lambda0/pi)^(D/2)
  T lam;           // lambda0
  T U[3];
  T sq;            // Shakhov prefactor 4 (1-Pr) lambda0^2 / (5 rho0), 0 for BGK
  T q[3];          // interface heat flux
  T a[3][5];       // spatial slopes per direction
  T A[5];          // time slope
  T kappa;         // K_xi / (2 lambda0)
  T xi4;           // <xi^4> = K_xi (K_xi + 2) / (4 lambda0^2)
  T pad[2];
};

// One velocity of the padded grid and its quadrature weight, loaded by one
// vector access in the blocked sweep.
template <typename T>
struct __align__(16) Vel4 {
  T x, y, z, w;
};

// Per-cell incidence entry of the blocked sweep, in the sweep precision.
template <typename T>
struct __align__(16) IncT {
  T w[3];          // least-squares weight M^-1 d (zero for walls)
  T r[3];          // face centroid minus cell centroid (the cell's frame)
  T n[3];          // unit normal pointing out of the cell
  T sarea;         // +area on the owner side, -area on the neighbour side
  int32_t face;    // global face index
  int32_t other;   // neighbour cell, or -(bc+1)
  int32_t bc;      // -1 interior, else bc index
  int32_t flags;   // bit 0: wall
};

// Number of monomials of degree <= 3 in D variables.
template <int D>
struct NPoly {
  static constexpr int value = D == 1 ? 4 : D == 2 ? 10 : 20;
};

// Position of the monomial c0^e0 c1^e1 c2^e2 in the coefficient arrays of
// FacePoly (degree by degree; within a degree by descending e0, then e1),
// the order in which the nested Horner evaluation of the blocked sweep
// reads them.
template <int D>
__host__ __device__ constexpr int mono_index(int e0, int e1, int e2) {
  return D == 1 ? e0
       : D == 2 ? ((e0 + e1) == 0 ? 0 : (e0 + e1) == 1 ? 1 : (e0 + e1) == 2 ? 3 : 6) + e1
                : ((e0 + e1 + e2) == 0 ? 0 : (e0 + e1 + e2) == 1 ? 1 : (e0 + e1 + e2) == 2 ? 4 : 10) +
                      (e1 + e2) * (e1 + e2 + 1) / 2 + e2;
}

// Per-step interface record of the blocked sweep (Eq. 32-35).  The
// equilibrium part of the interface distribution, G2 (g0 + g0+) + G3 u.grad
// g0 + G4 d_t g0, equals g0(u) * P_r(c) with c = u - U0 and P_r a cubic
// polynomial whose coefficients are built in FP64 per face.  Wall faces: the
// unit-density wall Maxwellian (rho_pref, U, lam, kappa), zero elsewhere.
template <int D, int NR, typename T>
struct __align__(16) FacePoly {
  T U[3];          // U0
  T lam;           // lambda0
  T rho_pref;      // rho0 (lambda0/pi)^(D/2)
  T kappa;         // K_xi / (2 lambda0)
  T G0, G1;        // integrals of c1, c2 over [0, dt] (Eq. 34)
  T P[NR][NPoly<D>::value];
};

// Per-cell equilibrium record of the blocked sweep in the sweep precision,
// built from the FP64 primitive record: the (Shakhov) Maxwellian of the cell
// and the relaxation factor of a stage update (Eq. 41-42).
template <typename T>
struct __align__(16) CellEq {
  T U[3];
  T lam;
  T pref;          // rho (lambda/pi)^(D/2)
  T s0;            // Shakhov prefactor 4 (1-Pr) lambda^2 / (5 rho), 0 for BGK
  T kap;           // K_xi / (2 lambda)
  T beta;          // dt / (2 tau)
  T q[3];          // heat flux entering the Shakhov term
  T inv_vol;
};

// Reference Maxwellian of one cell for scaled (FP16 / BF16) storage of f:
// g_ref = pref exp(-lam |u - U|^2) for h and kap g_ref for b.  Each stored
// row of 32 values holds (f - g_ref) / s in the storage type, s = the row's
// largest |f - g_ref| in FP32.
struct __align__(16) RefMaxwell {
  float pref, lam, U[3], kap, pad[2];
};

struct BCDev {
  int32_t type;
  int32_t pad;
  double rho, u[3], T;
};

// Tile face entry: global face index and the local gradient-set indices of
// the two sides (-1 for a ghost side).
struct TileFace {
  int64_t face;
  int32_t lo, ln;
};

struct Gas {
  int D, K, Kxi, NR, shakhov, limiter, shock_fix;
  double Pr, omega, mu_ref, venkat_K, dt;
};

}  // namespace ugks
