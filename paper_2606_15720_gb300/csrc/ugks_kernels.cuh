// Host-side launchers of the UGKS kernels (implemented in ugks_prep.cu,
// ugks_sweep.cu and ugks_blocked_*.cu), called by the C ABI in ugks_capi.cu.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "ugks_internal.cuh"

namespace ugks {

void launch_time_step(cudaStream_t s, int64_t Nc, int D, const int64_t* cf_off, const CellFace* cf,
                      const double* fnormal, const double* vol, const double* u, const double* w, int64_t nv,
                      unsigned long long* out_bits);

template <typename T>
cudaError_t launch_init_f(cudaStream_t s, int64_t Nc, int64_t M, int64_t nv, const Gas& g, const double* W,
                          const double* ux, const double* uy, const double* uz, T* f);

void launch_cell(cudaStream_t s, int64_t Nc, const Gas& g, const double* W, const double* q, const int64_t* cf_off,
                 const CellFace* cf, const double* vol, const BCDev* bcs, CellPrim* cp, double* gW, int* status);

template <typename T>
void launch_face(cudaStream_t s, int64_t Nf, const Gas& g, const double* W, const double* gW, const double* q,
                 const int64_t* fown, const int64_t* fnei, const double* fnormal, const double* fcent,
                 const double* fshift, const double* xc, const BCDev* bcs, FaceRec<T>* rec, void* poly);

template <typename T>
// vel4: the context's FP32 velocity records (x, y, z, weight) for FP32
// values (then the sums run in FP32 pairs), or NULL (FP64 sums)
void launch_moments(cudaStream_t s, int64_t Nc, int64_t M, const Gas& g, const T* f, const double* W,
                    const double* ux, const double* uy, const double* uz, const double* w, double* q_out,
                    double* Wf_out, const void* vel4 = nullptr);

template <typename T>
void launch_gather_f(cudaStream_t s, int64_t Nc, int64_t M, int NR, int64_t nv, const T* f, const int64_t* sel,
                     int64_t n, double* out);

template <typename T>
void launch_scatter_f(cudaStream_t s, int64_t Nc, int64_t M, int NR, int64_t nv, const double* in,
                      const int64_t* old_of_new, T* f);

void launch_residual_finalize(cudaStream_t s, int nw, int64_t Nc, const double* acc, double* res);

template <typename T>
void launch_moments13(cudaStream_t s, int64_t Nc, int64_t M, const Gas& g, const T* f, const double* W,
                      const double* ux, const double* uy, const double* uz, const double* w, double* out);
template <typename T>
void launch_init_ce(cudaStream_t s, int64_t Nc, int64_t M, int64_t nv, const Gas& g, const double* fields,
                    const double* ux, const double* uy, const double* uz, T* f);

void launch_surface(cudaStream_t s, int64_t nwall, int D, double dt, const int64_t* walls, const double* Facc,
                    int facc_stride, const double* fnormal, const int64_t* fnei, const BCDev* bcs,
                    const double* freestream, double* vals, double* coef);

// Arguments of the persistent velocity-block sweep (ugks_sweep.cu).
template <typename T>
struct SweepArgs {
  Gas g;
  int64_t Nc, M, nv;
  const T* f_cur;        // f^n        [NR][M][Nc][BV]
  T* f_next;             // f~ then f^{n+1}
  const double* W_cur;   // [Nc][NWP]
  double* W_next;
  const CellPrim* cp;    // primitive record of W^n (with q^n)
  CellPrim* cp_next;     // primitive record of W^{n+1} (written for tile cells)
  double* q_next;        // [Nc][3] heat flux of f^{n+1}
  const T* ux;           // [M*BV] velocity components and weights (padded)
  const T* uy;
  const T* uz;
  const T* w;
  const double* vol;
  const T* eps2;                 // limiter constant (K_v |Omega|^(1/D))^3 per cell
  const int64_t* cf_off;         // per cell incidence CSR
  const CellFaceT<T>* cf;
  const FaceGeom<T>* fg;
  const FaceRec<T>* fr;
  const BCDev* bcs;
  const int64_t* tile_begin;     // [ntiles+1] cell ranges
  const int64_t* gset_off;       // [ntiles+1]
  const int64_t* gset;           // gradient-set cells per tile (tile cells first)
  const int64_t* tf_off;         // [ntiles+1]
  const TileFace* tf;            // tile faces
  const int32_t* tcf;            // per cell incidence as local tile-face index << 1 | (sign < 0)
  int ntiles;                    // tiles; CTA b sweeps tiles b, b + gridDim.x, ...
  int64_t smem_g_elems;          // shared memory: gradients [gmax][NR][D][BV]
  int64_t smem_phi_elems;        // shared memory: micro fluxes [fmax][NR][BV]
  double* Facc;                  // per-tile scratch: face accumulators [fmax][FACC_W]
  int64_t Facc_stride;
  double* res_acc;               // [NWP] sum of squared W increments
  int* status;
};

template <typename T>
cudaError_t launch_sweep(cudaStream_t s, const SweepArgs<T>& a, int grid, int threads, size_t smem_bytes);

template <typename T>
int sweep_occupancy(int D, int NR, int threads, size_t smem_bytes);

// Arguments of the block-parallel sweep (ugks_blocked.cuh).  Cell and face
// indices are 32-bit inside these kernels (checked at create time).
template <typename T>
struct BlockedArgs {
  Gas g;
  int32_t Nc, Nf;
  int64_t M, nv;
  const T* f_cur;                // f^n        [NR][M][Nc][BV]
  T* f_next;                     // f~ then f^{n+1}
  const double* W_cur;           // [Nc][NWP]
  double* W_next;
  const CellPrim* cp;            // primitive record of W^n (with q^n)
  CellPrim* cp_next;             // primitive record of W^{n+1}
  double* q_next;                // [Nc][3] heat flux of f^{n+1}
  const Vel4<T>* vel;            // [M*BV] velocities and weights (padded: zero)
  // tensor grids whose fastest axis has BV points (no padding): every row of
  // BV velocities is one line along that axis, u = (lanev[l], rowv[m].y,
  // rowv[m].z) and weight = lanev[BV + l] * rowv[m].w
  int tensor;
  const Vel4<T>* rowv;           // [M] row components (y, z) and row weight factor (w)
  const T* lanev;                // [2][BV] lane-axis values, lane weight factors
  const double* vol;
  const T* eps2;                 // limiter constant (K_v |Omega|^(1/D))^3 per cell
  const int32_t* cf_off;         // per cell incidence CSR
  const IncT<T>* inc;
  const IncT<T>* ell;            // the same records as a padded table [Nc][W] (flags bit 1: padding)
  int W;                         // ELL width: the largest number of faces of a cell
  const FaceGeom<T>* fg;
  const void* fpoly;             // FacePoly<D, NR, T> [Nf] of this step
  CellEq<T>* ceq0;               // equilibrium record of W^n (first stage)
  CellEq<T>* ceq1;               // equilibrium record of W^{n+1} (second stage)
  const BCDev* bcs;
  T* X;                          // per face, one block [Nf][NR][VB][BV]: the upwind
                                 // reconstruction, then the micro flux
  double* Facc;                  // face accumulators [Nf][FACC_W]
  // scaled storage only (FP16 / BF16 rows): f_cur / f_next then point to the
  // stored deviations, and
  const float* sc_cur;           // per-row scales of f^n [NR][M][Nc]
  float* sc_next;                // per-row scales of f~, then of f^{n+1}
  const RefMaxwell* ref_cur;     // reference Maxwellian of f^n and f~ per cell
  RefMaxwell* ref_next;          // reference Maxwellian of f^{n+1}
  double* qpart;                 // heat-flux partial sums [nchunk][Nc][3]
  int nchunk;                    // velocity chunks of the second stage
  int nsm;                       // multiprocessors of the device (persistent grids)
  double* res_acc;               // [NWP] sum of squared W increments
  int* status;
};

template <typename T, typename S>
cudaError_t launch_brecon(cudaStream_t s, const BlockedArgs<T>& a, int64_t m0, int vb);
template <typename T>
cudaError_t launch_bflux(cudaStream_t s, const BlockedArgs<T>& a, int64_t m0, int vb, int first);
template <typename T, typename S>
cudaError_t launch_bstage1(cudaStream_t s, const BlockedArgs<T>& a, int64_t m0, int vb);
template <typename T, typename S>
cudaError_t launch_bstage1f(cudaStream_t s, const BlockedArgs<T>& a, int64_t m0, int vb, int first);
template <typename T, typename S>
bool bstage1f_supported(const BlockedArgs<T>& a, int vb);
template <typename T>
cudaError_t launch_bcelleq(cudaStream_t s, const BlockedArgs<T>& a);
template <typename T>
cudaError_t launch_bconserve(cudaStream_t s, const BlockedArgs<T>& a);
template <typename T, typename S>
cudaError_t launch_bstage2(cudaStream_t s, const BlockedArgs<T>& a);

// Scaled (FP16 / BF16) storage of f, ugks_store_util.cu.
void launch_sref(cudaStream_t s, int64_t Nc, const Gas& g, const double* W, RefMaxwell* ref);
template <typename S>
void launch_smoments(cudaStream_t s, int64_t Nc, int64_t M, int64_t nv, const Gas& g, const S* f, const float* sc,
                     const RefMaxwell* ref, const double* W, const double* ux, const double* uy, const double* uz,
                     const double* w, double* q_out, double* Wf_out);
template <typename S>
void launch_sgather(cudaStream_t s, int64_t Nc, int64_t M, int D, int NR, int64_t nv, const S* f, const float* sc,
                    const RefMaxwell* ref, const double* ux, const double* uy, const double* uz, const int64_t* sel,
                    int64_t n, double* out);
template <typename S>
void launch_sscatter(cudaStream_t s, int64_t Nc, int64_t M, int D, int NR, int64_t nv, const double* in,
                     const int64_t* old_of_new, const RefMaxwell* ref, const double* ux, const double* uy,
                     const double* uz, S* f, float* sc);

// Size of the file-scope device scratch used by ugks_step_static_scratch.
constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB

// Device address of that scratch on the current device (looked up once per
// device with cudaGetSymbolAddress).
cudaError_t static_scratch_address(void** ptr);

}  // namespace ugks
