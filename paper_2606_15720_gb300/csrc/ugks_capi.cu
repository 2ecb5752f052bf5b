// C ABI of the GB300 UGKS library (declared in include/ugks.h): validation,
// locality renumbering of cells, least-squares geometry, tiling of the
// velocity-block sweep, device memory, and the per-step launch sequence of
// Algorithm 5 (cell stage -> face stage -> persistent sweep).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <string>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "ugks.h"
#include "ugks_internal.cuh"
#include "ugks_kernels.cuh"
#include "ugks_store.cuh"

using namespace ugks;

namespace {

thread_local std::string g_thread_err;

struct KernelTiming {
  int id;
  cudaEvent_t start, stop;
};

// Timed regions of ugks_stats.  velocity_block_sweep is the whole sweep (the
// persistent kernel of the tiled sweep; every block kernel plus the
// conservative update and the second stage of the blocked sweep); the
// block_* entries and the two after them split the blocked sweep by kernel.
const char* const kKernelNames[] = {"cell_stage",   "face_stage",   "velocity_block_sweep",
                                    "residual",     "block_reconstruction", "block_fluxes",
                                    "block_stage1", "conserve",     "stage2", "block_flux_stage1"};
constexpr int kNumKernels = 10;
enum { kTCell = 0, kTFace, kTSweep, kTRes, kTGrad, kTFlux, kTStage1, kTConserve, kTStage2, kTFused };

}  // namespace

struct ugks_ctx {
  int D = 0, K = 0, NR = 1, storage = UGKS_STORAGE_F32;
  int64_t Nc = 0, Nf = 0, nv = 0, M = 0;
  double dt = 0.0;
  Gas gas{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<int64_t> new_of_old, old_of_new;   // cells
  std::vector<int64_t> face_old_of_new;            // faces
  std::vector<void*> allocs;
  // cells
  double *d_vol = nullptr, *d_xc = nullptr, *d_W[2] = {nullptr, nullptr}, *d_q[2] = {nullptr, nullptr};
  double *d_gW = nullptr, *d_res_acc = nullptr, *d_res = nullptr;
  int* d_status = nullptr;
  CellPrim *d_cp[2] = {nullptr, nullptr};
  int64_t* d_cf_off = nullptr;
  CellFace* d_cf = nullptr;
  void* d_cfT = nullptr;
  void* d_eps2 = nullptr;
  // faces
  int64_t *d_fown = nullptr, *d_fnei = nullptr;
  double *d_fnormal = nullptr, *d_fcent = nullptr, *d_fshift = nullptr;
  void* d_fg = nullptr;
  void* d_fr = nullptr;
  BCDev* d_bcs = nullptr;
  // velocities
  double *d_u = nullptr, *d_wgt = nullptr, *d_ux = nullptr, *d_uy = nullptr, *d_uz = nullptr, *d_wp = nullptr;
  void *d_uxT = nullptr, *d_uyT = nullptr, *d_uzT = nullptr, *d_wT = nullptr, *d_velT = nullptr;
  // tensor grid whose fastest axis has BV points: per-row and per-lane tables
  int tensor = 0;
  void *d_rowv = nullptr, *d_lanev = nullptr;
  // distributions
  void* d_f[2] = {nullptr, nullptr};
  // scaled (FP16 / BF16) storage: per-row scales and per-cell reference Maxwellians
  float* d_sc[2] = {nullptr, nullptr};
  RefMaxwell* d_ref[2] = {nullptr, nullptr};
  // sweep organisation: 1 tiled, 2 blocked; velocities per lane of the blocked sweep
  int variant = 2, vb = 1, vb_max = 1;  // vb_max: the block size the per-face buffer was sized for
  bool fused = false;                    // blocked sweep: fluxes and first stage in one kernel per block
  bool fused_used = false;               // the last blocked step ran the fused kernel (its stages fit)
  // blocked sweep: 32-bit incidence records, per-block scratch
  int32_t* d_cf_off32 = nullptr;
  void* d_inc = nullptr;
  void* d_ell = nullptr;
  int W = 0;
  void* d_X = nullptr;
  void* d_fpoly = nullptr;
  void *d_ceq0 = nullptr, *d_ceq1 = nullptr;
  double *d_Facc_b = nullptr, *d_qpart = nullptr;
  // surface quantities: diffuse-wall faces (ascending), output buffers, the
  // face accumulators of the last step
  std::vector<int64_t> walls;
  int64_t* d_walls = nullptr;
  double *d_surf = nullptr, *d_freestream = nullptr;
  const double* last_facc = nullptr;
  int nchunk = 1;
  int nsm = 1;
  // tiles and scratch of the tiled sweep
  int ntiles = 0, grid = 0, threads = 1024;
  size_t smem_bytes = 0;
  int64_t *d_tile_begin = nullptr, *d_gset_off = nullptr, *d_gset = nullptr, *d_tf_off = nullptr;
  TileFace* d_tf = nullptr;
  int32_t* d_tcf = nullptr;
  double* d_Facc = nullptr;
  int64_t smem_g_elems = 0, smem_phi_elems = 0, Facc_stride = 0;
  int cur = 0;
  int64_t step = 0;
  bool stats_on = false;
  std::vector<KernelTiming> timings;
  std::vector<cudaEvent_t> event_pool;
  double stat_ms[kNumKernels] = {};
  int64_t stat_count[kNumKernels] = {};
  std::string err;
};

namespace {

ugks_status fail(ugks_ctx* ctx, ugks_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  g_thread_err = buf;
  return st;
}

#define CUDA_TRY(ctx, call)                                                                       \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) {                                                                      \
      if (e_ == cudaErrorMemoryAllocation)                                                        \
        return fail(ctx, UGKS_ERR_OUT_OF_MEMORY, "%s: %s", #call, cudaGetErrorString(e_));        \
      return fail(ctx, UGKS_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));            \
    }                                                                                             \
  } while (0)

// Calls CALL(T, S) with the arithmetic type T and the storage type S of the context.
#define UGKS_BY_STORAGE(ctx, CALL)                                          \
  ((ctx)->storage == UGKS_STORAGE_F64    ? CALL(double, double)             \
   : (ctx)->storage == UGKS_STORAGE_F16  ? CALL(float, __half)              \
   : (ctx)->storage == UGKS_STORAGE_BF16 ? CALL(float, __nv_bfloat16)       \
                                         : CALL(float, float))

template <typename P>
cudaError_t dalloc(ugks_ctx* ctx, P** ptr, size_t bytes) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
  if (e != cudaSuccess) return e;
  ctx->allocs.push_back(p);
  *ptr = static_cast<P*>(p);
  return cudaSuccess;
}

template <typename P>
cudaError_t upload(ugks_ctx* ctx, P** ptr, const void* host, size_t bytes) {
  cudaError_t e = dalloc(ctx, ptr, bytes);
  if (e != cudaSuccess) return e;
  if (bytes) e = cudaMemcpyAsync(*ptr, host, bytes, cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(ctx->stream);
}

void release(ugks_ctx* ctx) {
  for (auto& t : ctx->timings) {
    cudaEventDestroy(t.start);
    cudaEventDestroy(t.stop);
  }
  ctx->timings.clear();
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  ctx->event_pool.clear();
  for (void* p : ctx->allocs) cudaFree(p);
  ctx->allocs.clear();
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  ctx->stream = nullptr;
}

// Spread the low 21 bits of x so that two zero bits follow each bit.
uint64_t spread3(uint64_t x) {
  x &= 0x1fffff;
  x = (x | x << 32) & 0x1f00000000ffffULL;
  x = (x | x << 16) & 0x1f0000ff0000ffULL;
  x = (x | x << 8) & 0x100f00f00f00f00fULL;
  x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
  x = (x | x << 2) & 0x1249249249249249ULL;
  return x;
}

// Least-squares weights M^-1 d (M = sum d d^T); M is singular (zero gradient)
// when det M <= 1e-12 (tr M / D)^D.
bool lsq_inverse(int D, const double* M, double* Minv) {
  double tr = 0.0;
  for (int d = 0; d < D; ++d) tr += M[d * D + d];
  tr /= D;
  if (!(tr > 0.0)) return false;
  if (D == 1) {
    if (!(M[0] > 1e-12 * tr)) return false;
    Minv[0] = 1.0 / M[0];
    return true;
  }
  if (D == 2) {
    double det = M[0] * M[3] - M[1] * M[2];
    if (!(det > 1e-12 * tr * tr)) return false;
    Minv[0] = M[3] / det;
    Minv[1] = -M[1] / det;
    Minv[2] = -M[2] / det;
    Minv[3] = M[0] / det;
    return true;
  }
  double c00 = M[4] * M[8] - M[5] * M[7], c01 = M[5] * M[6] - M[3] * M[8], c02 = M[3] * M[7] - M[4] * M[6];
  double det = M[0] * c00 + M[1] * c01 + M[2] * c02;
  if (!(det > 1e-12 * tr * tr * tr)) return false;
  double inv[9] = {c00, M[2] * M[7] - M[1] * M[8], M[1] * M[5] - M[2] * M[4],
                   c01, M[0] * M[8] - M[2] * M[6], M[2] * M[3] - M[0] * M[5],
                   c02, M[1] * M[6] - M[0] * M[7], M[0] * M[4] - M[1] * M[3]};
  for (int t = 0; t < 9; ++t) Minv[t] = inv[t] / det;
  return true;
}

ugks_status validate(const ugks_mesh* m, const ugks_vgrid* v, const ugks_params* p) {
  if (!m || !v || !p) return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "mesh, vgrid and params must not be NULL");
  if (m->dim < 1 || m->dim > 3) return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "dim must be 1, 2 or 3");
  if (m->n_cells <= 0 || m->n_faces <= 0) return fail(nullptr, UGKS_ERR_MESH, "mesh needs cells and faces");
  if (!m->cell_volume || !m->cell_centroid || !m->face_owner || !m->face_neighbor || !m->face_area ||
      !m->face_normal || !m->face_centroid)
    return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "mesh arrays must not be NULL");
  if (m->n_bc < 0 || (m->n_bc > 0 && !m->bc)) return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "bad bc list");
  const int D = m->dim;
  for (int b = 0; b < m->n_bc; ++b) {
    const ugks_bc& bc = m->bc[b];
    if (bc.type < UGKS_BC_WALL || bc.type > UGKS_BC_OUTFLOW)
      return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "bc %d has unknown type %d", b, bc.type);
    if (!(bc.T > 0.0) || !std::isfinite(bc.T)) return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "bc %d: T <= 0", b);
    if (bc.type == UGKS_BC_FARFIELD && !(bc.rho > 0.0))
      return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "bc %d: rho <= 0", b);
  }
  for (int64_t i = 0; i < m->n_cells; ++i)
    if (!(m->cell_volume[i] > 0.0) || !std::isfinite(m->cell_volume[i]))
      return fail(nullptr, UGKS_ERR_MESH, "cell %lld has non-positive volume", (long long)i);
  std::vector<int> nfaces(m->n_cells, 0);
  for (int64_t f = 0; f < m->n_faces; ++f) {
    int64_t o = m->face_owner[f], n = m->face_neighbor[f];
    if (o < 0 || o >= m->n_cells) return fail(nullptr, UGKS_ERR_MESH, "face %lld: owner out of range", (long long)f);
    if (n >= m->n_cells || n == o || (n < 0 && -n - 1 >= m->n_bc))
      return fail(nullptr, UGKS_ERR_MESH, "face %lld: bad neighbour %lld", (long long)f, (long long)n);
    if (!(m->face_area[f] > 0.0)) return fail(nullptr, UGKS_ERR_MESH, "face %lld: non-positive area", (long long)f);
    double nn = 0.0;
    for (int d = 0; d < D; ++d) nn += m->face_normal[f * D + d] * m->face_normal[f * D + d];
    if (std::fabs(nn - 1.0) > 1e-8) return fail(nullptr, UGKS_ERR_MESH, "face %lld: normal not unit", (long long)f);
    if (++nfaces[o] > MAXF || (n >= 0 && ++nfaces[n] > MAXF))
      return fail(nullptr, UGKS_ERR_MESH, "more than %d faces on a cell", MAXF);
  }
  if (v->n_v <= 0 || !v->u || !v->weight) return fail(nullptr, UGKS_ERR_VGRID, "empty velocity grid");
  for (int64_t k = 0; k < v->n_v; ++k) {
    if (!(v->weight[k] >= 0.0) || !std::isfinite(v->weight[k]))
      return fail(nullptr, UGKS_ERR_VGRID, "velocity %lld: bad weight", (long long)k);
    for (int d = 0; d < D; ++d)
      if (!std::isfinite(v->u[k * D + d])) return fail(nullptr, UGKS_ERR_VGRID, "velocity %lld: non-finite", (long long)k);
  }
  if (v->tensor_n[0] != 0 || v->tensor_n[1] != 0 || v->tensor_n[2] != 0) {
    // declared tensor product: the axes must reproduce u, first axis fastest
    int64_t prod = 1;
    for (int d = 0; d < D; ++d) {
      if (v->tensor_n[d] <= 0 || !v->axis[d])
        return fail(nullptr, UGKS_ERR_VGRID, "tensor grid: tensor_n[%d] and axis[%d] needed", d, d);
      prod *= v->tensor_n[d];
    }
    for (int d = D; d < 3; ++d)
      if (v->tensor_n[d] != 0) return fail(nullptr, UGKS_ERR_VGRID, "tensor grid: tensor_n[%d] beyond dim", d);
    if (prod != v->n_v) return fail(nullptr, UGKS_ERR_VGRID, "tensor grid: product of tensor_n != n_v");
    for (int64_t k = 0; k < v->n_v; ++k) {
      int64_t rem = k;
      for (int d = 0; d < D; ++d) {
        const int64_t i = rem % v->tensor_n[d];
        rem /= v->tensor_n[d];
        if (v->u[k * D + d] != v->axis[d][i])
          return fail(nullptr, UGKS_ERR_VGRID, "tensor grid: velocity %lld does not match the axes", (long long)k);
      }
    }
  }
  if (p->model != UGKS_MODEL_BGK && p->model != UGKS_MODEL_SHAKHOV)
    return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "unknown model");
  if (p->K < 0) return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "K must be >= 0");
  if (p->model == UGKS_MODEL_SHAKHOV && p->K != 0)
    return fail(nullptr, UGKS_ERR_UNSUPPORTED, "the reduced Shakhov terms (Eq. 18-19) hold for K = 0 only");
  if (p->model == UGKS_MODEL_BGK && p->Pr != 1.0)
    return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "BGK has Pr = 1");
  if (!(p->Pr > 0.0) || !(p->mu_ref > 0.0)) return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "Pr, mu_ref must be > 0");
  if (!(p->dt_override > 0.0) && !(p->cfl > 0.0))
    return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "need cfl > 0 or dt_override > 0");
  if (p->limiter < 0 || p->limiter > 2) return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "unknown limiter");
  if (p->storage < UGKS_STORAGE_F64 || p->storage > UGKS_STORAGE_BF16)
    return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "unknown storage precision %d", p->storage);
  if ((p->storage == UGKS_STORAGE_F16 || p->storage == UGKS_STORAGE_BF16) && p->sweep == UGKS_SWEEP_TILED)
    return fail(nullptr, UGKS_ERR_UNSUPPORTED, "FP16 / BF16 storage runs in the blocked sweep only");
  if (p->tile_cells < 0) return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "tile_cells must be >= 0");
  if (p->sweep < UGKS_SWEEP_AUTO || p->sweep > UGKS_SWEEP_BLOCKED_FUSED)
    return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "unknown sweep %d", p->sweep);
  if (p->block_velocities != 0 && p->block_velocities != 32 && p->block_velocities != 64 &&
      p->block_velocities != 128 && p->block_velocities != 256)
    return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "block_velocities must be 0, 32, 64, 128 or 256");
  if (p->block_velocities == 256 && !(m->dim == 3 && p->K == 0))
    return fail(nullptr, UGKS_ERR_UNSUPPORTED, "256 velocities per block: dim 3 with K_xi = 0 only");
  return UGKS_OK;
}

template <typename T>
size_t tsize() {
  return sizeof(T);
}

cudaEvent_t pooled_event(ugks_ctx* ctx) {
  cudaEvent_t e = nullptr;
  if (!ctx->event_pool.empty()) {
    e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    e = nullptr;
  }
  return e;
}

void record_start(ugks_ctx* ctx, int id, cudaEvent_t* ev) {
  *ev = nullptr;
  if (!ctx->stats_on) return;
  *ev = pooled_event(ctx);
  if (*ev) cudaEventRecord(*ev, ctx->stream);
  (void)id;
}

void record_stop(ugks_ctx* ctx, int id, cudaEvent_t start) {
  if (!ctx->stats_on || !start) return;
  cudaEvent_t stop = pooled_event(ctx);
  if (!stop) {
    ctx->event_pool.push_back(start);
    return;
  }
  cudaEventRecord(stop, ctx->stream);
  ctx->timings.push_back({id, start, stop});
}

// Scratch of the blocked sweep: the per-face buffer of one block, the face
// accumulators, the heat-flux partial sums of the second stage.
template <typename T>
size_t blocked_X_bytes(const ugks_ctx* ctx) {
  return size_t(ctx->Nf) * ctx->NR * ctx->vb * BV * sizeof(T);
}
size_t blocked_Facc_bytes(const ugks_ctx* ctx) { return size_t(ctx->Nf) * FACC_W * sizeof(double); }
size_t blocked_qpart_bytes(const ugks_ctx* ctx) { return size_t(ctx->nchunk) * ctx->Nc * 3 * sizeof(double); }

// Tensor grids whose fastest axis has BV points and no padding: every row of
// BV velocities is one line along that axis.  Splits the velocities into the
// lane component (the same in every row) and the row components (the same
// along a row), and the weights into lane and row factors (w = lane_w[l] *
// row_w[m], checked to 1e-13 relative).  Returns false for other grids.
bool split_tensor_rows(int64_t nv, int64_t M, const double* ux, const double* uy, const double* uz,
                       const double* wp, std::vector<double>& lane, std::vector<double>& rows) {
  if (nv != M * BV || !(wp[0] > 0.0)) return false;
  lane.assign(2 * BV, 0.0);
  rows.assign(size_t(M) * 4, 0.0);
  for (int l = 0; l < BV; ++l) {
    lane[l] = ux[l];
    lane[BV + l] = wp[l];
  }
  for (int64_t m = 0; m < M; ++m) {
    const int64_t k0 = m * BV;
    rows[m * 4 + 1] = uy[k0];
    rows[m * 4 + 2] = uz[k0];
    rows[m * 4 + 3] = wp[k0] / wp[0];
    for (int l = 0; l < BV; ++l) {
      const int64_t k = k0 + l;
      if (ux[k] != ux[l] || uy[k] != uy[k0] || uz[k] != uz[k0]) return false;
      const double w = lane[BV + l] * rows[m * 4 + 3];
      if (!(std::fabs(w - wp[k]) <= 1e-13 * std::fabs(wp[k]))) return false;
    }
  }
  return true;
}

template <typename T, typename S>
ugks_status build_typed(ugks_ctx* ctx, const std::vector<int64_t>& cf_off, const std::vector<CellFace>& cf,
                        const std::vector<double>& eps2,
                        const std::vector<FaceGeom<double>>& fg64, const double* ux, const double* uy,
                        const double* uz, const double* wp) {
  std::vector<CellFaceT<T>> cft(cf.size());
  for (size_t e = 0; e < cf.size(); ++e) {
    for (int d = 0; d < 3; ++d) {
      cft[e].w[d] = T(cf[e].w[d]);
      cft[e].r[d] = T(cf[e].r[d]);
    }
    cft[e].area = T(cf[e].area);
    cft[e].other = cf[e].other;
    cft[e].bc = cf[e].other < 0 ? int32_t(-cf[e].other - 1) : -1;
    cft[e].flags = cf[e].bc_type == UGKS_BC_WALL ? 1 : 0;
  }
  std::vector<T> e2(eps2.begin(), eps2.end());
  std::vector<FaceGeom<T>> fg(fg64.size());
  for (size_t f = 0; f < fg64.size(); ++f) {
    for (int d = 0; d < 3; ++d) {
      fg[f].n[d] = T(fg64[f].n[d]);
      fg[f].rl[d] = T(fg64[f].rl[d]);
      fg[f].rr[d] = T(fg64[f].rr[d]);
    }
    fg[f].area = T(fg64[f].area);
    fg[f].own = fg64[f].own;
    fg[f].nei = fg64[f].nei;
    fg[f].bc_type = fg64[f].bc_type;
    fg[f].pad = 0;
  }
  const size_t Mp = size_t(ctx->M) * BV;
  std::vector<T> tux(Mp), tuy(Mp), tuz(Mp), tw(Mp);
  for (size_t k = 0; k < Mp; ++k) {
    tux[k] = T(ux[k]);
    tuy[k] = T(uy[k]);
    tuz[k] = T(uz[k]);
    tw[k] = T(wp[k]);
  }
  T *cfT, *ep, *fgp, *a, *b, *c, *w;
  CUDA_TRY(ctx, upload(ctx, reinterpret_cast<CellFaceT<T>**>(&cfT), cft.data(), cft.size() * sizeof(CellFaceT<T>)));
  ctx->d_cfT = cfT;
  CUDA_TRY(ctx, upload(ctx, &ep, e2.data(), e2.size() * sizeof(T)));
  ctx->d_eps2 = ep;
  CUDA_TRY(ctx, upload(ctx, reinterpret_cast<FaceGeom<T>**>(&fgp), fg.data(), fg.size() * sizeof(FaceGeom<T>)));
  ctx->d_fg = fgp;
  CUDA_TRY(ctx, upload(ctx, &a, tux.data(), Mp * sizeof(T)));
  CUDA_TRY(ctx, upload(ctx, &b, tuy.data(), Mp * sizeof(T)));
  CUDA_TRY(ctx, upload(ctx, &c, tuz.data(), Mp * sizeof(T)));
  CUDA_TRY(ctx, upload(ctx, &w, tw.data(), Mp * sizeof(T)));
  ctx->d_uxT = a;
  ctx->d_uyT = b;
  ctx->d_uzT = c;
  ctx->d_wT = w;
  {
    std::vector<Vel4<T>> vel(Mp);
    for (size_t k = 0; k < Mp; ++k) vel[k] = Vel4<T>{tux[k], tuy[k], tuz[k], tw[k]};
    Vel4<T>* dv;
    CUDA_TRY(ctx, upload(ctx, &dv, vel.data(), Mp * sizeof(Vel4<T>)));
    ctx->d_velT = dv;
    std::vector<double> lane, rows;
    ctx->tensor = split_tensor_rows(ctx->nv, ctx->M, ux, uy, uz, wp, lane, rows) ? 1 : 0;
    if (ctx->tensor) {
      std::vector<T> laneT(lane.begin(), lane.end());
      std::vector<Vel4<T>> rowT(ctx->M);
      for (int64_t m = 0; m < ctx->M; ++m)
        rowT[m] = Vel4<T>{T(0), T(rows[m * 4 + 1]), T(rows[m * 4 + 2]), T(rows[m * 4 + 3])};
      Vel4<T>* dr;
      T* dl;
      CUDA_TRY(ctx, upload(ctx, &dr, rowT.data(), rowT.size() * sizeof(Vel4<T>)));
      CUDA_TRY(ctx, upload(ctx, &dl, laneT.data(), laneT.size() * sizeof(T)));
      ctx->d_rowv = dr;
      ctx->d_lanev = dl;
    }
  }
  if (ctx->variant == 1) {
    FaceRec<T>* fr;
    CUDA_TRY(ctx, dalloc(ctx, &fr, size_t(ctx->Nf) * sizeof(FaceRec<T>)));
    ctx->d_fr = fr;
  }
  if (ctx->variant == 2) {
    const int D = ctx->D, NR = ctx->NR;
    const size_t poly_bytes = D == 1   ? sizeof(FacePoly<1, 2, T>)
                              : D == 2 ? sizeof(FacePoly<2, 2, T>)
                              : NR == 1 ? sizeof(FacePoly<3, 1, T>)
                                        : sizeof(FacePoly<3, 2, T>);
    CUDA_TRY(ctx, dalloc(ctx, &ctx->d_fpoly, size_t(ctx->Nf) * poly_bytes));
    CellEq<T>* ce;
    CUDA_TRY(ctx, dalloc(ctx, &ce, size_t(ctx->Nc) * sizeof(CellEq<T>)));
    ctx->d_ceq0 = ce;
    CUDA_TRY(ctx, dalloc(ctx, &ce, size_t(ctx->Nc) * sizeof(CellEq<T>)));
    ctx->d_ceq1 = ce;
    std::vector<IncT<T>> inc(cf.size());
    for (size_t e = 0; e < cf.size(); ++e) {
      const CellFace& c = cf[e];
      IncT<T>& r = inc[e];
      for (int d = 0; d < 3; ++d) {
        r.w[d] = T(c.w[d]);
        r.r[d] = T(c.r[d]);
        r.n[d] = c.sign > 0 ? T(fg64[c.face].n[d]) : -T(fg64[c.face].n[d]);
      }
      r.sarea = c.sign > 0 ? T(c.area) : -T(c.area);
      r.face = int32_t(c.face);
      r.other = int32_t(c.other);
      r.bc = c.other < 0 ? int32_t(-c.other - 1) : -1;
      r.flags = c.bc_type == UGKS_BC_WALL ? 1 : 0;
    }
    IncT<T>* di;
    CUDA_TRY(ctx, upload(ctx, &di, inc.data(), inc.size() * sizeof(IncT<T>)));
    ctx->d_inc = di;
    // the same records as a padded table [Nc][W]: W = the most faces of a
    // cell, rounded up to 4 or 8 (the widths the pipelined kernels are
    // compiled for; padding slots are flagged)
    int W = 1;
    for (int64_t c = 0; c < ctx->Nc; ++c) W = std::max<int>(W, int(cf_off[c + 1] - cf_off[c]));
    W = W <= 4 ? 4 : W <= 8 ? 8 : W;
    ctx->W = W;
    IncT<T> pad{};
    pad.face = 0;
    pad.other = -1;
    pad.bc = -1;
    pad.flags = 2;
    std::vector<IncT<T>> ell(size_t(ctx->Nc) * W, pad);
    for (int64_t c = 0; c < ctx->Nc; ++c)
      for (int64_t e = cf_off[c]; e < cf_off[c + 1]; ++e) ell[size_t(c) * W + (e - cf_off[c])] = inc[e];
    IncT<T>* de;
    CUDA_TRY(ctx, upload(ctx, &de, ell.data(), ell.size() * sizeof(IncT<T>)));
    ctx->d_ell = de;
    T* X;
    CUDA_TRY(ctx, dalloc(ctx, &X, blocked_X_bytes<T>(ctx)));
    CUDA_TRY(ctx, cudaMemsetAsync(X, 0, blocked_X_bytes<T>(ctx), ctx->stream));
    ctx->d_X = X;
    CUDA_TRY(ctx, dalloc(ctx, &ctx->d_Facc_b, blocked_Facc_bytes(ctx)));
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_Facc_b, 0, blocked_Facc_bytes(ctx), ctx->stream));
    ctx->last_facc = ctx->d_Facc_b;
    CUDA_TRY(ctx, dalloc(ctx, &ctx->d_qpart, blocked_qpart_bytes(ctx)));
  }
  const size_t fsz = size_t(ctx->NR) * ctx->M * ctx->Nc * BV * sizeof(S);
  for (int s = 0; s < 2; ++s) {
    S* f;
    CUDA_TRY(ctx, dalloc(ctx, &f, fsz));
    ctx->d_f[s] = f;
  }
  if (StoreTraits<S>::scaled) {
    if (ctx->W > 8)
      return fail(ctx, UGKS_ERR_UNSUPPORTED, "FP16 / BF16 storage needs at most 8 faces per cell (this mesh has %d)",
                  ctx->W);
    for (int s = 0; s < 2; ++s) {
      CUDA_TRY(ctx, dalloc(ctx, &ctx->d_sc[s], size_t(ctx->NR) * ctx->M * ctx->Nc * sizeof(float)));
      CUDA_TRY(ctx, dalloc(ctx, &ctx->d_ref[s], size_t(ctx->Nc) * sizeof(RefMaxwell)));
    }
  }
  return UGKS_OK;
}

template <typename T, typename S>
ugks_status init_state_typed(ugks_ctx* ctx) {
  if constexpr (StoreTraits<S>::scaled) {
    // f^0 = the discrete Maxwellian of W_init = its reference: zero deviations and scales
    launch_sref(ctx->stream, ctx->Nc, ctx->gas, ctx->d_W[0], ctx->d_ref[0]);
    CUDA_TRY(ctx, cudaGetLastError());
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_f[0], 0, size_t(ctx->NR) * ctx->M * ctx->Nc * BV * sizeof(S), ctx->stream));
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_sc[0], 0, size_t(ctx->NR) * ctx->M * ctx->Nc * sizeof(float), ctx->stream));
    launch_smoments<S>(ctx->stream, ctx->Nc, ctx->M, ctx->nv, ctx->gas, static_cast<const S*>(ctx->d_f[0]),
                       ctx->d_sc[0], ctx->d_ref[0], ctx->d_W[0], ctx->d_ux, ctx->d_uy, ctx->d_uz, ctx->d_wp,
                       ctx->d_q[0], nullptr);
    CUDA_TRY(ctx, cudaGetLastError());
    return UGKS_OK;
  }
  CUDA_TRY(ctx, launch_init_f<T>(ctx->stream, ctx->Nc, ctx->M, ctx->nv, ctx->gas, ctx->d_W[0], ctx->d_ux,
                                 ctx->d_uy, ctx->d_uz, static_cast<T*>(ctx->d_f[0])));
  // q of f^0 (FP32 values: FP32 terms in float-pair sums over the context's velocity records)
  launch_moments<T>(ctx->stream, ctx->Nc, ctx->M, ctx->gas, static_cast<const T*>(ctx->d_f[0]), ctx->d_W[0],
                    ctx->d_ux, ctx->d_uy, ctx->d_uz, ctx->d_wp, ctx->d_q[0], nullptr,
                    sizeof(T) == 4 ? ctx->d_velT : nullptr);
  CUDA_TRY(ctx, cudaGetLastError());
  return UGKS_OK;
}

#define LAUNCH_TRY(ctx, call)                                                                     \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return fail(ctx, UGKS_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// The velocity-block sweep of Algorithm 5 as block kernels: for every block
// of vb x 32 velocities gradients -> fluxes -> first stage, then the
// conservative update and the second stage.  The last M mod vb blocks run
// with one velocity per lane.
template <typename T, typename S>
ugks_status sweep_blocked(ugks_ctx* ctx, int cur, void* X, double* Facc, double* qpart) {
  const int nxt = 1 - cur;
  BlockedArgs<T> a;
  a.g = ctx->gas;
  a.Nc = int32_t(ctx->Nc);
  a.Nf = int32_t(ctx->Nf);
  a.M = ctx->M;
  a.nv = ctx->nv;
  a.f_cur = static_cast<const T*>(ctx->d_f[cur]);
  a.f_next = static_cast<T*>(ctx->d_f[nxt]);
  a.W_cur = ctx->d_W[cur];
  a.W_next = ctx->d_W[nxt];
  a.cp = ctx->d_cp[0];
  a.cp_next = ctx->d_cp[1];
  a.q_next = ctx->d_q[nxt];
  a.vel = static_cast<const Vel4<T>*>(ctx->d_velT);
  a.tensor = ctx->tensor;
  a.rowv = static_cast<const Vel4<T>*>(ctx->d_rowv);
  a.lanev = static_cast<const T*>(ctx->d_lanev);
  a.vol = ctx->d_vol;
  a.eps2 = static_cast<const T*>(ctx->d_eps2);
  a.cf_off = ctx->d_cf_off32;
  a.inc = static_cast<const IncT<T>*>(ctx->d_inc);
  a.ell = static_cast<const IncT<T>*>(ctx->d_ell);
  a.W = ctx->W;
  a.fg = static_cast<const FaceGeom<T>*>(ctx->d_fg);
  a.fpoly = ctx->d_fpoly;
  a.ceq0 = static_cast<CellEq<T>*>(ctx->d_ceq0);
  a.ceq1 = static_cast<CellEq<T>*>(ctx->d_ceq1);
  a.bcs = ctx->d_bcs;
  a.X = static_cast<T*>(X);
  a.Facc = Facc;
  a.qpart = qpart;
  a.nchunk = ctx->nchunk;
  a.nsm = ctx->nsm;
  a.sc_cur = ctx->d_sc[cur];
  a.sc_next = ctx->d_sc[nxt];
  a.ref_cur = ctx->d_ref[cur];
  a.ref_next = ctx->d_ref[nxt];
  a.res_acc = ctx->d_res_acc;
  a.status = ctx->d_status;
  cudaStream_t s = ctx->stream;
  cudaEvent_t ev_all, ev;
  record_start(ctx, kTSweep, &ev_all);
  LAUNCH_TRY(ctx, launch_bcelleq<T>(s, a));
  const int64_t M = ctx->M;
  int64_t m0 = 0;
  for (int pass = 0; pass < 2; ++pass) {
    const int vb = pass == 0 ? ctx->vb : 1;
    // the fused flux + first-stage kernel where requested and its stages
    // fit, else the flux kernel (fluxes into X) and the first stage
    const bool fused = ctx->fused && bstage1f_supported<T, S>(a, vb);
    if (pass == 0) ctx->fused_used = fused;
    for (; m0 + vb <= M; m0 += vb) {
      record_start(ctx, kTGrad, &ev);
      LAUNCH_TRY(ctx, (launch_brecon<T, S>(s, a, m0, vb)));
      record_stop(ctx, kTGrad, ev);
      if (fused) {
        record_start(ctx, kTFused, &ev);
        LAUNCH_TRY(ctx, (launch_bstage1f<T, S>(s, a, m0, vb, m0 == 0 ? 1 : 0)));
        record_stop(ctx, kTFused, ev);
        continue;
      }
      record_start(ctx, kTFlux, &ev);
      LAUNCH_TRY(ctx, launch_bflux<T>(s, a, m0, vb, m0 == 0 ? 1 : 0));
      record_stop(ctx, kTFlux, ev);
      record_start(ctx, kTStage1, &ev);
      LAUNCH_TRY(ctx, (launch_bstage1<T, S>(s, a, m0, vb)));
      record_stop(ctx, kTStage1, ev);
    }
  }
  record_start(ctx, kTConserve, &ev);
  LAUNCH_TRY(ctx, launch_bconserve<T>(s, a));
  record_stop(ctx, kTConserve, ev);
  record_start(ctx, kTStage2, &ev);
  LAUNCH_TRY(ctx, (launch_bstage2<T, S>(s, a)));
  record_stop(ctx, kTStage2, ev);
  record_stop(ctx, kTSweep, ev_all);
  return UGKS_OK;
}

template <typename T, typename S>
ugks_status step_typed(ugks_ctx* ctx) {
  const int cur = ctx->cur, nxt = 1 - cur;
  cudaEvent_t ev;
  CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_res_acc, 0, NWP * sizeof(double), ctx->stream));
  record_start(ctx, 0, &ev);
  launch_cell(ctx->stream, ctx->Nc, ctx->gas, ctx->d_W[cur], ctx->d_q[cur], ctx->d_cf_off, ctx->d_cf, ctx->d_vol,
              ctx->d_bcs, ctx->d_cp[0], ctx->d_gW, ctx->d_status);
  CUDA_TRY(ctx, cudaGetLastError());
  record_stop(ctx, 0, ev);
  record_start(ctx, 1, &ev);
  launch_face<T>(ctx->stream, ctx->Nf, ctx->gas, ctx->d_W[cur], ctx->d_gW, ctx->d_q[cur], ctx->d_fown, ctx->d_fnei,
                 ctx->d_fnormal, ctx->d_fcent, ctx->d_fshift, ctx->d_xc, ctx->d_bcs,
                 static_cast<FaceRec<T>*>(ctx->d_fr), ctx->d_fpoly);
  CUDA_TRY(ctx, cudaGetLastError());
  record_stop(ctx, 1, ev);
  if (ctx->variant == 2) {
    ugks_status st = sweep_blocked<T, S>(ctx, cur, ctx->d_X, ctx->d_Facc_b, ctx->d_qpart);
    if (st != UGKS_OK) return st;
    ctx->last_facc = ctx->d_Facc_b;
    record_start(ctx, kTRes, &ev);
    launch_residual_finalize(ctx->stream, ctx->D + 2, ctx->Nc, ctx->d_res_acc, ctx->d_res);
    CUDA_TRY(ctx, cudaGetLastError());
    record_stop(ctx, kTRes, ev);
    ctx->cur = nxt;
    ctx->step++;
    return UGKS_OK;
  }
  SweepArgs<T> a;
  a.g = ctx->gas;
  a.Nc = ctx->Nc;
  a.M = ctx->M;
  a.nv = ctx->nv;
  a.f_cur = static_cast<const T*>(ctx->d_f[cur]);
  a.f_next = static_cast<T*>(ctx->d_f[nxt]);
  a.W_cur = ctx->d_W[cur];
  a.W_next = ctx->d_W[nxt];
  a.cp = ctx->d_cp[0];
  a.cp_next = ctx->d_cp[1];
  a.q_next = ctx->d_q[nxt];
  a.ux = static_cast<const T*>(ctx->d_uxT);
  a.uy = static_cast<const T*>(ctx->d_uyT);
  a.uz = static_cast<const T*>(ctx->d_uzT);
  a.w = static_cast<const T*>(ctx->d_wT);
  a.vol = ctx->d_vol;
  a.eps2 = static_cast<const T*>(ctx->d_eps2);
  a.cf_off = ctx->d_cf_off;
  a.cf = static_cast<const CellFaceT<T>*>(ctx->d_cfT);
  a.fg = static_cast<const FaceGeom<T>*>(ctx->d_fg);
  a.fr = static_cast<const FaceRec<T>*>(ctx->d_fr);
  a.bcs = ctx->d_bcs;
  a.tile_begin = ctx->d_tile_begin;
  a.gset_off = ctx->d_gset_off;
  a.gset = ctx->d_gset;
  a.tf_off = ctx->d_tf_off;
  a.tf = ctx->d_tf;
  a.tcf = ctx->d_tcf;
  a.ntiles = ctx->ntiles;
  a.smem_g_elems = ctx->smem_g_elems;
  a.smem_phi_elems = ctx->smem_phi_elems;
  a.Facc = ctx->d_Facc;
  a.Facc_stride = ctx->Facc_stride;
  a.res_acc = ctx->d_res_acc;
  a.status = ctx->d_status;
  record_start(ctx, 2, &ev);
  CUDA_TRY(ctx, launch_sweep<T>(ctx->stream, a, ctx->grid, ctx->threads, ctx->smem_bytes));
  record_stop(ctx, 2, ev);
  record_start(ctx, 3, &ev);
  launch_residual_finalize(ctx->stream, ctx->D + 2, ctx->Nc, ctx->d_res_acc, ctx->d_res);
  CUDA_TRY(ctx, cudaGetLastError());
  record_stop(ctx, 3, ev);
  ctx->cur = nxt;
  ctx->step++;
  return UGKS_OK;
}


// Variant of step_typed whose sweep takes its scratch (blocked sweep:
// gradients, micro fluxes and face accumulators; tiled sweep: face
// accumulators) from the file-scope device array of ugks_sweep.cu instead of
// the context's own buffers; it records no timing events.
size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

template <typename T>
size_t static_scratch_need(const ugks_ctx* ctx) {
  if (ctx->variant == 2)
    return align256(blocked_X_bytes<T>(ctx)) + align256(blocked_Facc_bytes(ctx)) + align256(blocked_qpart_bytes(ctx));
  return align256(size_t(ctx->ntiles) * ctx->Facc_stride * sizeof(double));
}

template <typename T, typename S>
ugks_status step_typed_static(ugks_ctx* ctx, unsigned char* base) {
  const int cur = ctx->cur, nxt = 1 - cur;
  CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_res_acc, 0, NWP * sizeof(double), ctx->stream));
  launch_cell(ctx->stream, ctx->Nc, ctx->gas, ctx->d_W[cur], ctx->d_q[cur], ctx->d_cf_off, ctx->d_cf, ctx->d_vol,
              ctx->d_bcs, ctx->d_cp[0], ctx->d_gW, ctx->d_status);
  CUDA_TRY(ctx, cudaGetLastError());
  launch_face<T>(ctx->stream, ctx->Nf, ctx->gas, ctx->d_W[cur], ctx->d_gW, ctx->d_q[cur], ctx->d_fown, ctx->d_fnei,
                 ctx->d_fnormal, ctx->d_fcent, ctx->d_fshift, ctx->d_xc, ctx->d_bcs,
                 static_cast<FaceRec<T>*>(ctx->d_fr), ctx->d_fpoly);
  CUDA_TRY(ctx, cudaGetLastError());
  if (ctx->variant == 2) {
    unsigned char* X = base;
    unsigned char* Facc = X + align256(blocked_X_bytes<T>(ctx));
    unsigned char* qpart = Facc + align256(blocked_Facc_bytes(ctx));
    const bool was_on = ctx->stats_on;
    ctx->stats_on = false;
    ugks_status st = sweep_blocked<T, S>(ctx, cur, X, reinterpret_cast<double*>(Facc), reinterpret_cast<double*>(qpart));
    ctx->stats_on = was_on;
    if (st != UGKS_OK) return st;
    // The shared array is overwritten by the next static step of any context:
    // keep this step's face accumulators (wall fluxes for ugks_surface) in the
    // context's own buffer, allocated at create.
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->d_Facc_b, Facc, blocked_Facc_bytes(ctx), cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->last_facc = ctx->d_Facc_b;
    launch_residual_finalize(ctx->stream, ctx->D + 2, ctx->Nc, ctx->d_res_acc, ctx->d_res);
    CUDA_TRY(ctx, cudaGetLastError());
    ctx->cur = nxt;
    ctx->step++;
    return UGKS_OK;
  }
  SweepArgs<T> a;
  a.g = ctx->gas;
  a.Nc = ctx->Nc;
  a.M = ctx->M;
  a.nv = ctx->nv;
  a.f_cur = static_cast<const T*>(ctx->d_f[cur]);
  a.f_next = static_cast<T*>(ctx->d_f[nxt]);
  a.W_cur = ctx->d_W[cur];
  a.W_next = ctx->d_W[nxt];
  a.cp = ctx->d_cp[0];
  a.cp_next = ctx->d_cp[1];
  a.q_next = ctx->d_q[nxt];
  a.ux = static_cast<const T*>(ctx->d_uxT);
  a.uy = static_cast<const T*>(ctx->d_uyT);
  a.uz = static_cast<const T*>(ctx->d_uzT);
  a.w = static_cast<const T*>(ctx->d_wT);
  a.vol = ctx->d_vol;
  a.eps2 = static_cast<const T*>(ctx->d_eps2);
  a.cf_off = ctx->d_cf_off;
  a.cf = static_cast<const CellFaceT<T>*>(ctx->d_cfT);
  a.fg = static_cast<const FaceGeom<T>*>(ctx->d_fg);
  a.fr = static_cast<const FaceRec<T>*>(ctx->d_fr);
  a.bcs = ctx->d_bcs;
  a.tile_begin = ctx->d_tile_begin;
  a.gset_off = ctx->d_gset_off;
  a.gset = ctx->d_gset;
  a.tf_off = ctx->d_tf_off;
  a.tf = ctx->d_tf;
  a.tcf = ctx->d_tcf;
  a.ntiles = ctx->ntiles;
  a.smem_g_elems = ctx->smem_g_elems;
  a.smem_phi_elems = ctx->smem_phi_elems;
  a.Facc = reinterpret_cast<double*>(base);
  a.Facc_stride = ctx->Facc_stride;
  a.res_acc = ctx->d_res_acc;
  a.status = ctx->d_status;
  CUDA_TRY(ctx, launch_sweep<T>(ctx->stream, a, ctx->grid, ctx->threads, ctx->smem_bytes));
  launch_residual_finalize(ctx->stream, ctx->D + 2, ctx->Nc, ctx->d_res_acc, ctx->d_res);
  CUDA_TRY(ctx, cudaGetLastError());
  ctx->cur = nxt;
  ctx->step++;
  return UGKS_OK;
}

ugks_status check_status(ugks_ctx* ctx) {
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  int st = 0;
  CUDA_TRY(ctx, cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st & 2)
    return fail(ctx, UGKS_ERR_TIMEOUT, "a bounded device wait (shared-memory staging) gave up; results are invalid");
  if (st) return fail(ctx, UGKS_ERR_NONFINITE, "non-physical state (rho <= 0, T <= 0 or NaN) was produced");
  return UGKS_OK;
}

ugks_status create_impl(const ugks_mesh* m, const ugks_vgrid* v, const ugks_params* p, const double* W_init,
                        void* stream, ugks_ctx* ctx) {
  const int D = m->dim;
  ctx->D = D;
  ctx->K = p->K;
  const int Kxi = p->K + 3 - D;
  ctx->NR = Kxi > 0 ? 2 : 1;
  ctx->storage = p->storage;
  ctx->Nc = m->n_cells;
  ctx->Nf = m->n_faces;
  ctx->nv = v->n_v;
  ctx->M = (v->n_v + BV - 1) / BV;
  if (stream) {
    ctx->stream = static_cast<cudaStream_t>(stream);
  } else {
    CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
    ctx->own_stream = true;
  }
  const int64_t Nc = ctx->Nc, Nf = ctx->Nf;

  // ---- locality renumbering: Morton order of the cell centroids ----
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t i = 0; i < Nc; ++i)
    for (int d = 0; d < D; ++d) {
      lo[d] = std::min(lo[d], m->cell_centroid[i * D + d]);
      hi[d] = std::max(hi[d], m->cell_centroid[i * D + d]);
    }
  std::vector<uint64_t> key(Nc);
  for (int64_t i = 0; i < Nc; ++i) {
    uint64_t kk = 0;
    for (int d = 0; d < D; ++d) {
      double span = hi[d] > lo[d] ? hi[d] - lo[d] : 1.0;
      uint64_t q = uint64_t(std::min(2097151.0, std::max(0.0, (m->cell_centroid[i * D + d] - lo[d]) / span * 2097151.0)));
      kk |= spread3(q) << d;
    }
    key[i] = kk;
  }
  ctx->old_of_new.resize(Nc);
  std::iota(ctx->old_of_new.begin(), ctx->old_of_new.end(), 0);
  std::stable_sort(ctx->old_of_new.begin(), ctx->old_of_new.end(),
                   [&](int64_t a, int64_t b) { return key[a] < key[b]; });
  ctx->new_of_old.resize(Nc);
  for (int64_t i = 0; i < Nc; ++i) ctx->new_of_old[ctx->old_of_new[i]] = i;
  const auto& n_of_o = ctx->new_of_old;
  const auto& o_of_n = ctx->old_of_new;

  // ---- cell geometry in the new order ----
  std::vector<double> vol(Nc), xc(Nc * 3, 0.0);
  for (int64_t i = 0; i < Nc; ++i) {
    int64_t o = o_of_n[i];
    vol[i] = m->cell_volume[o];
    for (int d = 0; d < D; ++d) xc[i * 3 + d] = m->cell_centroid[o * D + d];
  }
  // ---- face renumbering: faces in the order of their lower-numbered cell,
  // so that the kernels that walk faces and those that walk cells touch the
  // per-face rows (interface records, the block's face buffer) in the same
  // spatial order ----
  std::vector<int64_t>& f_old = ctx->face_old_of_new;
  f_old.resize(Nf);
  std::iota(f_old.begin(), f_old.end(), 0);
  {
    std::vector<int64_t> fkey(Nf);
    for (int64_t f = 0; f < Nf; ++f) {
      const int64_t a = n_of_o[m->face_owner[f]], nb = m->face_neighbor[f];
      fkey[f] = nb >= 0 ? std::min(a, n_of_o[nb]) : a;
    }
    std::stable_sort(f_old.begin(), f_old.end(), [&](int64_t x, int64_t y) { return fkey[x] < fkey[y]; });
  }
  // ---- face geometry (new face order) ----
  std::vector<int64_t> fown(Nf), fnei(Nf);
  std::vector<double> fnormal(Nf * 3, 0.0), fcent(Nf * 3, 0.0), fshift(Nf * 3, 0.0);
  std::vector<FaceGeom<double>> fg(Nf);
  for (int64_t f = 0; f < Nf; ++f) {
    const int64_t fo = f_old[f];
    fown[f] = n_of_o[m->face_owner[fo]];
    int64_t nb = m->face_neighbor[fo];
    fnei[f] = nb >= 0 ? n_of_o[nb] : nb;
    for (int d = 0; d < D; ++d) {
      fnormal[f * 3 + d] = m->face_normal[fo * D + d];
      fcent[f * 3 + d] = m->face_centroid[fo * D + d];
      fshift[f * 3 + d] = m->face_shift ? m->face_shift[fo * D + d] : 0.0;
    }
    FaceGeom<double>& g = fg[f];
    for (int d = 0; d < 3; ++d) {
      g.n[d] = fnormal[f * 3 + d];
      g.rl[d] = d < D ? fcent[f * 3 + d] - xc[fown[f] * 3 + d] : 0.0;
      g.rr[d] = (d < D && fnei[f] >= 0) ? fcent[f * 3 + d] - fshift[f * 3 + d] - xc[fnei[f] * 3 + d] : 0.0;
    }
    g.area = m->face_area[fo];
    g.own = fown[f];
    g.nei = fnei[f];
    g.bc_type = nb >= 0 ? 0 : m->bc[-nb - 1].type;
    g.pad = 0;
  }
  // ---- diffuse-wall faces (surface quantities), in ascending original index ----
  for (int64_t f = 0; f < Nf; ++f)
    if (fg[f].bc_type == UGKS_BC_WALL) ctx->walls.push_back(f);
  std::sort(ctx->walls.begin(), ctx->walls.end(), [&](int64_t x, int64_t y) { return f_old[x] < f_old[y]; });

  // ---- incidence CSR with least-squares weights ----
  std::vector<int64_t> cf_off(Nc + 1, 0);
  for (int64_t f = 0; f < Nf; ++f) {
    cf_off[fown[f] + 1]++;
    if (fnei[f] >= 0) cf_off[fnei[f] + 1]++;
  }
  for (int64_t i = 0; i < Nc; ++i) cf_off[i + 1] += cf_off[i];
  std::vector<CellFace> cf(cf_off[Nc]);
  {
    std::vector<int64_t> fill(cf_off.begin(), cf_off.end() - 1);
    for (int64_t f = 0; f < Nf; ++f) {
      for (int side = 0; side < 2; ++side) {
        int64_t c = side == 0 ? fown[f] : fnei[f];
        if (c < 0) continue;
        CellFace e{};
        e.face = f;
        e.sign = side == 0 ? 1 : -1;
        e.other = side == 0 ? fnei[f] : fown[f];
        e.bc_type = fnei[f] >= 0 ? 0 : m->bc[-fnei[f] - 1].type;
        e.area = m->face_area[f_old[f]];
        for (int d = 0; d < D; ++d) e.r[d] = fcent[f * 3 + d] - (side == 0 ? 0.0 : fshift[f * 3 + d]) - xc[c * 3 + d];
        cf[fill[c]++] = e;
      }
    }
  }
  std::vector<double> eps2(Nc);
  for (int64_t i = 0; i < Nc; ++i) {
    double M3[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    double dx[MAXF][3];
    for (int64_t e = cf_off[i]; e < cf_off[i + 1]; ++e) {
      CellFace& s = cf[e];
      double* d_ = dx[e - cf_off[i]];
      for (int d = 0; d < 3; ++d) d_[d] = 0.0;
      // A wall is a mirrored ghost holding the cell's own value (zero
      // gradient): its offset enters M, its weight stays 0 (nothing enters the
      // right-hand side).  Left out of M, wall cells with two interior
      // neighbours extrapolate and some outflow face values weigh the cell's
      // own value negatively (transport then amplifies that velocity).
      const double* n = &fnormal[s.face * 3];
      if (s.other >= 0) {
        double sh = s.sign > 0 ? 1.0 : -1.0;
        for (int d = 0; d < D; ++d) d_[d] = xc[s.other * 3 + d] + sh * fshift[s.face * 3 + d] - xc[i * 3 + d];
      } else {
        double dn = 0.0;
        for (int d = 0; d < D; ++d) dn += s.r[d] * n[d];
        for (int d = 0; d < D; ++d) d_[d] = 2.0 * dn * n[d];
      }
      for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) M3[a * D + b] += d_[a] * d_[b];
    }
    double Minv[9];
    bool ok = lsq_inverse(D, M3, Minv);
    for (int64_t e = cf_off[i]; e < cf_off[i + 1]; ++e) {
      CellFace& s = cf[e];
      const double* d_ = dx[e - cf_off[i]];
      for (int a = 0; a < 3; ++a) {
        double w = 0.0;
        if (ok && a < D && s.bc_type != UGKS_BC_WALL)
          for (int b = 0; b < D; ++b) w += Minv[a * D + b] * d_[b];
        s.w[a] = w;
      }
    }
    eps2[i] = std::pow(p->venkat_K * std::pow(vol[i], 1.0 / D), 3.0);
  }

  // ---- padded velocity grid (zero weight, zero velocity beyond n_v) ----
  const int64_t Mp = ctx->M * BV;
  std::vector<double> ux(Mp, 0.0), uy(Mp, 0.0), uz(Mp, 0.0), wp(Mp, 0.0);
  for (int64_t k = 0; k < v->n_v; ++k) {
    ux[k] = v->u[k * D];
    if (D > 1) uy[k] = v->u[k * D + 1];
    if (D > 2) uz[k] = v->u[k * D + 2];
    wp[k] = v->weight[k];
  }

  // ---- organisation of the sweep ----
  // The blocked sweep indexes cells, faces and incidences with 32 bits.
  const bool fits32 = Nc < INT32_MAX && Nf < INT32_MAX && int64_t(cf.size()) < INT32_MAX;
  ctx->variant = p->sweep == UGKS_SWEEP_TILED ? 1 : 2;
  ctx->fused = p->sweep == UGKS_SWEEP_BLOCKED_FUSED;
  if (ctx->variant == 2 && !fits32) {
    if (p->sweep == UGKS_SWEEP_BLOCKED || p->sweep == UGKS_SWEEP_BLOCKED_FUSED)
      return fail(ctx, UGKS_ERR_UNSUPPORTED, "the blocked sweep needs fewer than 2^31 cells, faces and incidences");
    ctx->variant = 1;
  }
  // default: 256 velocities per block where compiled (3-D, one reduced
  // distribution), else 128; fewer velocities than that: the largest power
  // of two that fits
  const bool vb8 = ctx->D == 3 && ctx->NR == 1;
  ctx->vb = p->block_velocities > 0 ? p->block_velocities / BV : (vb8 ? 8 : 4);
  while (ctx->vb > ctx->M) ctx->vb /= 2;
  ctx->vb_max = ctx->vb;

  // ---- tiles of the tiled sweep ----
  // One CTA of 1024 threads per SM sweeps tiles b, b + grid, ...; a tile's
  // gradients and micro fluxes for one velocity block must fit in shared
  // memory, which fixes the smallest tile count.
  ctx->threads = 1024;
  int dev = 0, nsm = 1;
  CUDA_TRY(ctx, cudaGetDevice(&dev));
  CUDA_TRY(ctx, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  ctx->nsm = nsm;
  // Velocity chunks of the second stage (grid: 32 cells per CTA x chunks):
  // enough chunks for about 8 waves of 4 CTAs per SM, so that the last wave
  // is a small part of the pass, and no more (each CTA's set-up and
  // heat-flux reduction are per chunk).
  {
    const int64_t cell_ctas = (Nc + 31) / 32;
    int64_t chunks = 1;
    while (chunks < 16 && cell_ctas * chunks < int64_t(32) * nsm) chunks *= 2;
    ctx->nchunk = int(std::min<int64_t>(ctx->M, chunks));
  }
  int smem_optin = 0;
  CUDA_TRY(ctx, cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t elem = ctx->storage == UGKS_STORAGE_F64 ? sizeof(double) : sizeof(float);
  const size_t smem_budget = size_t(std::max(0, smem_optin - 8 * 1024));
  std::vector<int64_t> tile_begin, gset_off, gset, tf_off;
  std::vector<TileFace> tfl;
  std::vector<int32_t> tcf(cf.size(), 0);
  std::vector<int64_t> cell_mark(Nc, -1), cell_local(Nc, -1), face_mark(Nf, -1), face_local(Nf, -1);
  int64_t max_ng = 1, max_nf = 1, ntiles = 0;
  auto build_tiles = [&](int64_t nt_) {
    tile_begin.assign(nt_ + 1, 0);
    for (int64_t t = 0; t <= nt_; ++t) tile_begin[t] = (Nc * t) / nt_;
    gset_off.assign(nt_ + 1, 0);
    tf_off.assign(nt_ + 1, 0);
    gset.clear();
    tfl.clear();
    std::fill(cell_mark.begin(), cell_mark.end(), -1);
    std::fill(face_mark.begin(), face_mark.end(), -1);
    max_ng = 1;
    max_nf = 1;
    for (int64_t t = 0; t < nt_; ++t) {
      int64_t ng = 0;
      for (int64_t c = tile_begin[t]; c < tile_begin[t + 1]; ++c) {
        cell_mark[c] = t;
        cell_local[c] = ng++;
        gset.push_back(c);
      }
      for (int64_t c = tile_begin[t]; c < tile_begin[t + 1]; ++c)
        for (int64_t e = cf_off[c]; e < cf_off[c + 1]; ++e) {
          int64_t o = cf[e].other;
          if (o >= 0 && cell_mark[o] != t) {
            cell_mark[o] = t;
            cell_local[o] = ng++;
            gset.push_back(o);
          }
        }
      int64_t nfl = 0;
      for (int64_t c = tile_begin[t]; c < tile_begin[t + 1]; ++c)
        for (int64_t e = cf_off[c]; e < cf_off[c + 1]; ++e) {
          int64_t f = cf[e].face;
          if (face_mark[f] != t) {
            face_mark[f] = t;
            face_local[f] = nfl++;
            TileFace tfe;
            tfe.face = f;
            tfe.lo = int32_t(cell_local[fown[f]]);
            tfe.ln = fnei[f] >= 0 ? int32_t(cell_local[fnei[f]]) : -1;
            tfl.push_back(tfe);
          }
          tcf[e] = int32_t(face_local[f] << 1) | (cf[e].sign < 0 ? 1 : 0);
        }
      gset_off[t + 1] = gset_off[t] + ng;
      tf_off[t + 1] = tf_off[t] + nfl;
      max_ng = std::max(max_ng, ng);
      max_nf = std::max(max_nf, nfl);
    }
  };
  auto smem_need = [&]() {
    return size_t(max_ng) * ctx->NR * D * BV * elem + size_t(max_nf) * ctx->NR * BV * elem;
  };
  if (ctx->variant != 1) {
    // no tiles
  } else if (p->tile_cells > 0) {
    ntiles = std::max<int64_t>(1, (Nc + p->tile_cells - 1) / p->tile_cells);
    build_tiles(ntiles);
    if (smem_need() > smem_budget)
      return fail(ctx, UGKS_ERR_INVALID_ARGUMENT, "tile_cells=%d needs %zu bytes of shared memory per tile (limit %zu)",
                  p->tile_cells, smem_need(), smem_budget);
  } else {
    for (int64_t k = 1;; ++k) {
      ntiles = std::min<int64_t>(int64_t(nsm) * k, Nc);
      build_tiles(ntiles);
      if (smem_need() <= smem_budget) break;
      if (ntiles == Nc) return fail(ctx, UGKS_ERR_UNSUPPORTED, "cell stencil too large for shared memory");
    }
  }
  if (ctx->variant == 1) {
    ctx->ntiles = int(ntiles);
    ctx->smem_g_elems = max_ng * ctx->NR * D * BV;
    ctx->smem_phi_elems = max_nf * ctx->NR * BV;
    ctx->smem_bytes = smem_need();
    ctx->Facc_stride = max_nf * FACC_W;
    int occ = ctx->storage == UGKS_STORAGE_F64
                  ? sweep_occupancy<double>(D, ctx->NR, ctx->threads, ctx->smem_bytes)
                  : sweep_occupancy<float>(D, ctx->NR, ctx->threads, ctx->smem_bytes);
    CUDA_TRY(ctx, cudaGetLastError());
    if (occ < 1)
      return fail(ctx, UGKS_ERR_UNSUPPORTED, "the sweep kernel cannot be resident with %zu bytes of shared memory",
                  ctx->smem_bytes);
    ctx->grid = int(std::min<int64_t>(ntiles, int64_t(nsm) * occ));
  }

  // ---- gas ----
  Gas& g = ctx->gas;
  g.D = D;
  g.K = p->K;
  g.Kxi = Kxi;
  g.NR = ctx->NR;
  g.shakhov = p->model == UGKS_MODEL_SHAKHOV;
  g.limiter = p->limiter;
  g.shock_fix = p->shock_tau_fix;
  g.Pr = p->Pr;
  g.omega = p->omega;
  g.mu_ref = p->mu_ref;
  g.venkat_K = p->venkat_K;

  // ---- device uploads ----
  std::vector<BCDev> bcs(std::max(1, m->n_bc));
  for (int b = 0; b < m->n_bc; ++b) {
    bcs[b].type = m->bc[b].type;
    bcs[b].pad = 0;
    bcs[b].rho = m->bc[b].rho;
    for (int d = 0; d < 3; ++d) bcs[b].u[d] = m->bc[b].u[d];
    bcs[b].T = m->bc[b].T;
  }
  std::vector<double> W0(Nc * NWP, 0.0);
  for (int64_t i = 0; i < Nc; ++i) {
    int64_t o = o_of_n[i];
    if (W_init) {
      for (int t = 0; t < D + 2; ++t) W0[i * NWP + t] = W_init[o * (D + 2) + t];
    } else {
      if (m->n_bc < 1) return fail(ctx, UGKS_ERR_INVALID_ARGUMENT, "W_init is NULL and the mesh has no bc");
      const ugks_bc& b = m->bc[0];
      double u2 = 0.0;
      W0[i * NWP] = b.rho;
      for (int d = 0; d < D; ++d) {
        W0[i * NWP + 1 + d] = b.rho * b.u[d];
        u2 += b.u[d] * b.u[d];
      }
      W0[i * NWP + D + 1] = 0.5 * b.rho * u2 + (p->K + 3) * b.rho * b.T / 4.0;
    }
  }
  for (int64_t i = 0; i < Nc; ++i) {
    const double* Wi = &W0[i * NWP];
    double u2 = 0.0;
    for (int d = 0; d < D; ++d) u2 += (Wi[1 + d] / Wi[0]) * (Wi[1 + d] / Wi[0]);
    if (!(Wi[0] > 0.0) || !(Wi[D + 1] - 0.5 * Wi[0] * u2 > 0.0) || !std::isfinite(Wi[D + 1]))
      return fail(ctx, UGKS_ERR_NONFINITE, "W_init of cell %lld is not a physical state", (long long)o_of_n[i]);
  }
  std::vector<double> uflat(v->n_v * D);
  std::copy(v->u, v->u + v->n_v * D, uflat.begin());
  CUDA_TRY(ctx, upload(ctx, &ctx->d_vol, vol.data(), Nc * sizeof(double)));
  CUDA_TRY(ctx, upload(ctx, &ctx->d_xc, xc.data(), Nc * 3 * sizeof(double)));
  for (int s = 0; s < 2; ++s) {
    CUDA_TRY(ctx, dalloc(ctx, &ctx->d_W[s], Nc * NWP * sizeof(double)));
    CUDA_TRY(ctx, dalloc(ctx, &ctx->d_q[s], Nc * 3 * sizeof(double)));
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_q[s], 0, Nc * 3 * sizeof(double), ctx->stream));
    CUDA_TRY(ctx, dalloc(ctx, &ctx->d_cp[s], Nc * sizeof(CellPrim)));
  }
  CUDA_TRY(ctx, cudaMemcpyAsync(ctx->d_W[0], W0.data(), Nc * NWP * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CUDA_TRY(ctx, dalloc(ctx, &ctx->d_gW, Nc * NWP * 3 * sizeof(double)));
  CUDA_TRY(ctx, dalloc(ctx, &ctx->d_res_acc, NWP * sizeof(double)));
  CUDA_TRY(ctx, dalloc(ctx, &ctx->d_res, NWP * sizeof(double)));
  CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_res, 0, NWP * sizeof(double), ctx->stream));
  CUDA_TRY(ctx, dalloc(ctx, &ctx->d_status, sizeof(int)));
  CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
  CUDA_TRY(ctx, upload(ctx, &ctx->d_cf_off, cf_off.data(), cf_off.size() * sizeof(int64_t)));
  CUDA_TRY(ctx, upload(ctx, &ctx->d_cf, cf.data(), cf.size() * sizeof(CellFace)));
  CUDA_TRY(ctx, upload(ctx, &ctx->d_fown, fown.data(), Nf * sizeof(int64_t)));
  CUDA_TRY(ctx, upload(ctx, &ctx->d_fnei, fnei.data(), Nf * sizeof(int64_t)));
  CUDA_TRY(ctx, upload(ctx, &ctx->d_fnormal, fnormal.data(), Nf * 3 * sizeof(double)));
  CUDA_TRY(ctx, upload(ctx, &ctx->d_fcent, fcent.data(), Nf * 3 * sizeof(double)));
  CUDA_TRY(ctx, upload(ctx, &ctx->d_fshift, fshift.data(), Nf * 3 * sizeof(double)));
  CUDA_TRY(ctx, upload(ctx, &ctx->d_bcs, bcs.data(), bcs.size() * sizeof(BCDev)));
  {
    const size_t nwall = ctx->walls.size();
    CUDA_TRY(ctx, upload(ctx, &ctx->d_walls, ctx->walls.data(), nwall * sizeof(int64_t)));
    CUDA_TRY(ctx, dalloc(ctx, &ctx->d_surf, nwall * (D + 2 + 3) * sizeof(double)));
    CUDA_TRY(ctx, dalloc(ctx, &ctx->d_freestream, 5 * sizeof(double)));
  }
  CUDA_TRY(ctx, upload(ctx, &ctx->d_u, uflat.data(), uflat.size() * sizeof(double)));
  CUDA_TRY(ctx, upload(ctx, &ctx->d_wgt, v->weight, v->n_v * sizeof(double)));
  CUDA_TRY(ctx, upload(ctx, &ctx->d_ux, ux.data(), Mp * sizeof(double)));
  CUDA_TRY(ctx, upload(ctx, &ctx->d_uy, uy.data(), Mp * sizeof(double)));
  CUDA_TRY(ctx, upload(ctx, &ctx->d_uz, uz.data(), Mp * sizeof(double)));
  CUDA_TRY(ctx, upload(ctx, &ctx->d_wp, wp.data(), Mp * sizeof(double)));
  if (ctx->variant == 1) {
    CUDA_TRY(ctx, upload(ctx, &ctx->d_tile_begin, tile_begin.data(), tile_begin.size() * sizeof(int64_t)));
    CUDA_TRY(ctx, upload(ctx, &ctx->d_gset_off, gset_off.data(), gset_off.size() * sizeof(int64_t)));
    CUDA_TRY(ctx, upload(ctx, &ctx->d_gset, gset.data(), gset.size() * sizeof(int64_t)));
    CUDA_TRY(ctx, upload(ctx, &ctx->d_tf_off, tf_off.data(), tf_off.size() * sizeof(int64_t)));
    CUDA_TRY(ctx, upload(ctx, &ctx->d_tf, tfl.data(), tfl.size() * sizeof(TileFace)));
    CUDA_TRY(ctx, upload(ctx, &ctx->d_tcf, tcf.data(), tcf.size() * sizeof(int32_t)));
    CUDA_TRY(ctx, dalloc(ctx, &ctx->d_Facc, size_t(ntiles) * ctx->Facc_stride * sizeof(double)));
  } else {
    std::vector<int32_t> off32(cf_off.begin(), cf_off.end());
    CUDA_TRY(ctx, upload(ctx, &ctx->d_cf_off32, off32.data(), off32.size() * sizeof(int32_t)));
  }

  // ---- time step ----
  if (p->dt_override > 0.0) {
    ctx->dt = p->dt_override;
  } else {
    unsigned long long* bits;
    CUDA_TRY(ctx, dalloc(ctx, &bits, sizeof(unsigned long long)));
    unsigned long long init = 0x7ff0000000000000ULL;  // +inf
    CUDA_TRY(ctx, cudaMemcpyAsync(bits, &init, sizeof(init), cudaMemcpyHostToDevice, ctx->stream));
    launch_time_step(ctx->stream, Nc, D, ctx->d_cf_off, ctx->d_cf, ctx->d_fnormal, ctx->d_vol, ctx->d_u, ctx->d_wgt,
                     v->n_v, bits);
    CUDA_TRY(ctx, cudaGetLastError());
    unsigned long long out = 0;
    CUDA_TRY(ctx, cudaMemcpyAsync(&out, bits, sizeof(out), cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    double dmin;
    std::memcpy(&dmin, &out, sizeof(dmin));
    if (!std::isfinite(dmin)) return fail(ctx, UGKS_ERR_VGRID, "no velocity with positive weight moves");
    ctx->dt = p->cfl * dmin;
  }
  g.dt = ctx->dt;

#define UGKS_BUILD(T, S) build_typed<T, S>(ctx, cf_off, cf, eps2, fg, ux.data(), uy.data(), uz.data(), wp.data())
  ugks_status st = UGKS_BY_STORAGE(ctx, UGKS_BUILD);
#undef UGKS_BUILD
  if (st != UGKS_OK) return st;
#define UGKS_INIT(T, S) init_state_typed<T, S>(ctx)
  st = UGKS_BY_STORAGE(ctx, UGKS_INIT);
#undef UGKS_INIT
  if (st != UGKS_OK) return st;
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return UGKS_OK;
}

}  // namespace

extern "C" {

ugks_status ugks_create(const ugks_mesh* mesh, const ugks_vgrid* vgrid, const ugks_params* params,
                        const double* W_init, void* cuda_stream, ugks_ctx** out) {
  if (!out) return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "out must not be NULL");
  *out = nullptr;
  ugks_status st = validate(mesh, vgrid, params);
  if (st != UGKS_OK) return st;
  if (vgrid->n_v > 0 && mesh->n_cells > 0) {
    // (NR * M * Nc * BV) elements must be addressable
    double elems = 2.0 * double((vgrid->n_v + BV - 1) / BV) * BV * double(mesh->n_cells);
    if (elems > 9.0e18) return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "problem too large");
  }
  ugks_ctx* ctx = new (std::nothrow) ugks_ctx();
  if (!ctx) return fail(nullptr, UGKS_ERR_OUT_OF_MEMORY, "host allocation failed");
  st = create_impl(mesh, vgrid, params, W_init, cuda_stream, ctx);
  if (st != UGKS_OK) {
    g_thread_err = ctx->err;
    release(ctx);
    delete ctx;
    return st;
  }
  *out = ctx;
  return UGKS_OK;
}

ugks_status ugks_step(ugks_ctx* ctx, int32_t n_steps) {
  if (!ctx) return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "NULL context");
  if (n_steps < 0) return fail(ctx, UGKS_ERR_INVALID_ARGUMENT, "n_steps must be >= 0");
  for (int32_t s = 0; s < n_steps; ++s) {
#define UGKS_STEP(T, S) step_typed<T, S>(ctx)
    ugks_status st = UGKS_BY_STORAGE(ctx, UGKS_STEP);
#undef UGKS_STEP
    if (st != UGKS_OK) return st;
  }
  return UGKS_OK;
}


ugks_status ugks_step_static_scratch(ugks_ctx* ctx, int32_t n_steps) {
  if (!ctx) return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "NULL context");
  if (n_steps < 0) return fail(ctx, UGKS_ERR_INVALID_ARGUMENT, "n_steps must be >= 0");
  const size_t need = ctx->storage == UGKS_STORAGE_F64 ? static_scratch_need<double>(ctx)
                                                       : static_scratch_need<float>(ctx);  // FP32 arithmetic otherwise
  if (need > kStaticScratchBytes)
    return fail(ctx, UGKS_ERR_INVALID_ARGUMENT,
                "ugks_step_static_scratch: this context needs %zu bytes of sweep scratch, more than the static "
                "limit of %zu bytes; use ugks_step", need, kStaticScratchBytes);
  void* base = nullptr;
  CUDA_TRY(ctx, static_scratch_address(&base));
  for (int32_t s = 0; s < n_steps; ++s) {
#define UGKS_STEP_STATIC(T, S) step_typed_static<T, S>(ctx, static_cast<unsigned char*>(base))
    ugks_status st = UGKS_BY_STORAGE(ctx, UGKS_STEP_STATIC);
#undef UGKS_STEP_STATIC
    if (st != UGKS_OK) return st;
  }
  return UGKS_OK;
}

ugks_status ugks_moments(ugks_ctx* ctx, double* W_out, double* q_out) {
  if (!ctx || !W_out) return fail(ctx, UGKS_ERR_INVALID_ARGUMENT, "NULL argument");
  ugks_status st = check_status(ctx);
  if (st != UGKS_OK) return st;
  const int D = ctx->D;
  std::vector<double> W(ctx->Nc * NWP), q(ctx->Nc * 3);
  CUDA_TRY(ctx, cudaMemcpy(W.data(), ctx->d_W[ctx->cur], W.size() * sizeof(double), cudaMemcpyDeviceToHost));
  if (q_out) CUDA_TRY(ctx, cudaMemcpy(q.data(), ctx->d_q[ctx->cur], q.size() * sizeof(double), cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < ctx->Nc; ++i) {
    int64_t o = ctx->old_of_new[i];
    for (int t = 0; t < D + 2; ++t) W_out[o * (D + 2) + t] = W[i * NWP + t];
    if (q_out)
      for (int d = 0; d < D; ++d) q_out[o * D + d] = q[i * 3 + d];
  }
  return UGKS_OK;
}

ugks_status ugks_residual(ugks_ctx* ctx, double* res_out) {
  if (!ctx || !res_out) return fail(ctx, UGKS_ERR_INVALID_ARGUMENT, "NULL argument");
  ugks_status st = check_status(ctx);
  if (st != UGKS_OK) return st;
  CUDA_TRY(ctx, cudaMemcpy(res_out, ctx->d_res, (ctx->D + 2) * sizeof(double), cudaMemcpyDeviceToHost));
  return UGKS_OK;
}

ugks_status ugks_surface(ugks_ctx* ctx, const double* freestream, int64_t cap, int64_t* n_wall, int64_t* faces,
                         double* vals, double* coef) {
  if (!ctx || !n_wall) return fail(ctx, UGKS_ERR_INVALID_ARGUMENT, "NULL argument");
  const int64_t nwall = int64_t(ctx->walls.size());
  *n_wall = nwall;
  if (ctx->variant != 2)
    return fail(ctx, UGKS_ERR_UNSUPPORTED, "ugks_surface needs the blocked sweep (sweep = UGKS_SWEEP_BLOCKED or AUTO)");
  if (nwall == 0) return UGKS_OK;
  if (cap < nwall || !faces || !vals || (freestream && !coef))
    return fail(ctx, UGKS_ERR_INVALID_ARGUMENT, "ugks_surface: %lld wall faces need arrays of that capacity",
                (long long)nwall);
  const int D = ctx->D;
  if (freestream) {
    double U2 = 0.0;
    for (int d = 0; d < D; ++d) U2 += freestream[1 + d] * freestream[1 + d];
    if (!(freestream[0] > 0.0) || !(U2 > 0.0))
      return fail(ctx, UGKS_ERR_INVALID_ARGUMENT, "ugks_surface: the free stream needs rho > 0 and |U| > 0");
  }
  ugks_status st = check_status(ctx);
  if (st != UGKS_OK) return st;
  double fs[5] = {0, 0, 0, 0, 0};
  if (freestream)
    for (int t = 0; t < D + 2; ++t) fs[t] = freestream[t];
  CUDA_TRY(ctx, cudaMemcpyAsync(ctx->d_freestream, fs, sizeof(fs), cudaMemcpyHostToDevice, ctx->stream));
  double* d_vals = ctx->d_surf;
  double* d_coef = ctx->d_surf + nwall * (D + 2);
  launch_surface(ctx->stream, nwall, D, ctx->dt, ctx->d_walls, ctx->last_facc, FACC_W, ctx->d_fnormal, ctx->d_fnei,
                 ctx->d_bcs, freestream ? ctx->d_freestream : nullptr, d_vals, d_coef);
  CUDA_TRY(ctx, cudaGetLastError());
  CUDA_TRY(ctx, cudaMemcpyAsync(vals, d_vals, nwall * (D + 2) * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  if (freestream)
    CUDA_TRY(ctx, cudaMemcpyAsync(coef, d_coef, nwall * 3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  for (int64_t i = 0; i < nwall; ++i) faces[i] = ctx->face_old_of_new[ctx->walls[i]];
  return UGKS_OK;
}

ugks_status ugks_moments13(ugks_ctx* ctx, double* out) {
  if (!ctx || !out) return fail(ctx, UGKS_ERR_INVALID_ARGUMENT, "NULL argument");
  if (ctx->storage != UGKS_STORAGE_F64 && ctx->storage != UGKS_STORAGE_F32)
    return fail(ctx, UGKS_ERR_UNSUPPORTED, "ugks_moments13 needs FP64 or FP32 storage");
  ugks_status st = check_status(ctx);
  if (st != UGKS_OK) return st;
  const int D = ctx->D, n13 = 2 * D + 2 + D * (D + 1) / 2;
  double* d_out = nullptr;
  CUDA_TRY(ctx, cudaMalloc(&d_out, size_t(ctx->Nc) * n13 * sizeof(double)));
  const int c = ctx->cur;
  if (ctx->storage == UGKS_STORAGE_F64)
    launch_moments13<double>(ctx->stream, ctx->Nc, ctx->M, ctx->gas, static_cast<const double*>(ctx->d_f[c]),
                             ctx->d_W[c], ctx->d_ux, ctx->d_uy, ctx->d_uz, ctx->d_wp, d_out);
  else
    launch_moments13<float>(ctx->stream, ctx->Nc, ctx->M, ctx->gas, static_cast<const float*>(ctx->d_f[c]),
                            ctx->d_W[c], ctx->d_ux, ctx->d_uy, ctx->d_uz, ctx->d_wp, d_out);
  cudaError_t e = cudaGetLastError();
  std::vector<double> tmp(size_t(ctx->Nc) * n13);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tmp.data(), d_out, tmp.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                            ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(d_out);
  if (e != cudaSuccess) return fail(ctx, UGKS_ERR_CUDA, "ugks_moments13: %s", cudaGetErrorString(e));
  for (int64_t i = 0; i < ctx->Nc; ++i)
    std::memcpy(out + size_t(ctx->old_of_new[i]) * n13, &tmp[size_t(i) * n13], n13 * sizeof(double));
  return UGKS_OK;
}

ugks_status ugks_init_moments13(ugks_ctx* ctx, const double* fields) {
  if (!ctx || !fields) return fail(ctx, UGKS_ERR_INVALID_ARGUMENT, "NULL argument");
  if (ctx->storage != UGKS_STORAGE_F64 && ctx->storage != UGKS_STORAGE_F32)
    return fail(ctx, UGKS_ERR_UNSUPPORTED, "ugks_init_moments13 needs FP64 or FP32 storage");
  const int D = ctx->D, n13 = 2 * D + 2 + D * (D + 1) / 2;
  std::vector<double> fl(size_t(ctx->Nc) * n13), Wn(size_t(ctx->Nc) * NWP, 0.0);
  for (int64_t i = 0; i < ctx->Nc; ++i) {
    const double* x = fields + size_t(ctx->old_of_new[i]) * n13;
    for (int t = 0; t < n13; ++t)
      if (!std::isfinite(x[t]))
        return fail(ctx, UGKS_ERR_INVALID_ARGUMENT, "cell %lld: non-finite field", (long long)ctx->old_of_new[i]);
    if (!(x[0] > 0.0) || !(x[D + 1] > 0.0))
      return fail(ctx, UGKS_ERR_INVALID_ARGUMENT, "cell %lld: rho and T must be > 0", (long long)ctx->old_of_new[i]);
    std::memcpy(&fl[size_t(i) * n13], x, n13 * sizeof(double));
    double u2 = 0.0;
    Wn[size_t(i) * NWP] = x[0];
    for (int d = 0; d < D; ++d) {
      Wn[size_t(i) * NWP + 1 + d] = x[0] * x[1 + d];
      u2 += x[1 + d] * x[1 + d];
    }
    Wn[size_t(i) * NWP + D + 1] = 0.5 * x[0] * u2 + (ctx->K + 3) * x[0] * x[D + 1] / 4.0;
  }
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  const int c = ctx->cur;
  double* d_fields = nullptr;
  CUDA_TRY(ctx, cudaMalloc(&d_fields, fl.size() * sizeof(double)));
  cudaError_t e = cudaMemcpyAsync(d_fields, fl.data(), fl.size() * sizeof(double), cudaMemcpyHostToDevice,
                                  ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->d_W[c], Wn.data(), Wn.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) {
    if (ctx->storage == UGKS_STORAGE_F64) {
      launch_init_ce<double>(ctx->stream, ctx->Nc, ctx->M, ctx->nv, ctx->gas, d_fields, ctx->d_ux, ctx->d_uy,
                             ctx->d_uz, static_cast<double*>(ctx->d_f[c]));
      launch_moments<double>(ctx->stream, ctx->Nc, ctx->M, ctx->gas, static_cast<const double*>(ctx->d_f[c]),
                             ctx->d_W[c], ctx->d_ux, ctx->d_uy, ctx->d_uz, ctx->d_wp, ctx->d_q[c], nullptr);
    } else {
      launch_init_ce<float>(ctx->stream, ctx->Nc, ctx->M, ctx->nv, ctx->gas, d_fields, ctx->d_ux, ctx->d_uy,
                            ctx->d_uz, static_cast<float*>(ctx->d_f[c]));
      launch_moments<float>(ctx->stream, ctx->Nc, ctx->M, ctx->gas, static_cast<const float*>(ctx->d_f[c]),
                            ctx->d_W[c], ctx->d_ux, ctx->d_uy, ctx->d_uz, ctx->d_wp, ctx->d_q[c], nullptr);
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_res, 0, NWP * sizeof(double), ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(d_fields);
  if (e != cudaSuccess) return fail(ctx, UGKS_ERR_CUDA, "ugks_init_moments13: %s", cudaGetErrorString(e));
  ctx->step = 0;
  return UGKS_OK;
}

ugks_status ugks_dt(const ugks_ctx* ctx, double* dt_out) {
  if (!ctx || !dt_out) return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "NULL argument");
  *dt_out = ctx->dt;
  return UGKS_OK;
}

ugks_status ugks_sizes(const ugks_ctx* ctx, int32_t* n_reduced, int64_t* n_v_padded) {
  if (!ctx) return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "NULL context");
  if (n_reduced) *n_reduced = ctx->NR;
  if (n_v_padded) *n_v_padded = ctx->M * BV;
  return UGKS_OK;
}

ugks_status ugks_mesh_sizes(const ugks_ctx* ctx, int32_t* dim, int64_t* n_cells, int64_t* n_faces) {
  if (!ctx) return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "NULL context");
  if (dim) *dim = ctx->D;
  if (n_cells) *n_cells = ctx->Nc;
  if (n_faces) *n_faces = ctx->Nf;
  return UGKS_OK;
}

ugks_status ugks_get_f(ugks_ctx* ctx, const int64_t* cells, int64_t n, double* out) {
  if (!ctx || (n > 0 && (!cells || !out)) || n < 0) return fail(ctx, UGKS_ERR_INVALID_ARGUMENT, "bad arguments");
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (n == 0) return UGKS_OK;
  std::vector<int64_t> sel(n);
  for (int64_t s = 0; s < n; ++s) {
    if (cells[s] < 0 || cells[s] >= ctx->Nc) return fail(ctx, UGKS_ERR_INVALID_ARGUMENT, "cell index out of range");
    sel[s] = ctx->new_of_old[cells[s]];
  }
  int64_t *d_sel = nullptr;
  double* d_out = nullptr;
  const size_t nout = size_t(n) * ctx->NR * ctx->nv;
  CUDA_TRY(ctx, cudaMalloc(&d_sel, n * sizeof(int64_t)));
  cudaError_t e = cudaMalloc(&d_out, nout * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_sel, sel.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) {
    const int c = ctx->cur;
    if (ctx->storage == UGKS_STORAGE_F64)
      launch_gather_f<double>(ctx->stream, ctx->Nc, ctx->M, ctx->NR, ctx->nv,
                              static_cast<const double*>(ctx->d_f[ctx->cur]), d_sel, n, d_out);
    else if (ctx->storage == UGKS_STORAGE_F16)
      launch_sgather<__half>(ctx->stream, ctx->Nc, ctx->M, ctx->D, ctx->NR, ctx->nv,
                             static_cast<const __half*>(ctx->d_f[c]), ctx->d_sc[c], ctx->d_ref[c], ctx->d_ux,
                             ctx->d_uy, ctx->d_uz, d_sel, n, d_out);
    else if (ctx->storage == UGKS_STORAGE_BF16)
      launch_sgather<__nv_bfloat16>(ctx->stream, ctx->Nc, ctx->M, ctx->D, ctx->NR, ctx->nv,
                                    static_cast<const __nv_bfloat16*>(ctx->d_f[c]), ctx->d_sc[c], ctx->d_ref[c],
                                    ctx->d_ux, ctx->d_uy, ctx->d_uz, d_sel, n, d_out);
    else
      launch_gather_f<float>(ctx->stream, ctx->Nc, ctx->M, ctx->NR, ctx->nv,
                             static_cast<const float*>(ctx->d_f[ctx->cur]), d_sel, n, d_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, nout * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(d_sel);
  if (d_out) cudaFree(d_out);
  if (e != cudaSuccess) return fail(ctx, UGKS_ERR_CUDA, "ugks_get_f: %s", cudaGetErrorString(e));
  return UGKS_OK;
}

ugks_status ugks_get_state(ugks_ctx* ctx, double* W, double* f, int64_t* step) {
  if (!ctx || !W) return fail(ctx, UGKS_ERR_INVALID_ARGUMENT, "NULL argument");
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  {
    const int D = ctx->D;
    std::vector<double> Wd(ctx->Nc * NWP);
    CUDA_TRY(ctx, cudaMemcpy(Wd.data(), ctx->d_W[ctx->cur], Wd.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < ctx->Nc; ++i)
      for (int t = 0; t < D + 2; ++t) W[ctx->old_of_new[i] * (D + 2) + t] = Wd[i * NWP + t];
  }
  ugks_status st = UGKS_OK;
  if (step) *step = ctx->step;
  if (!f) return UGKS_OK;
  std::vector<int64_t> all(ctx->Nc);
  std::iota(all.begin(), all.end(), 0);
  // gather in original order: out[cell][r][k] -> f[r][cell][k]
  std::vector<double> tmp(size_t(ctx->Nc) * ctx->NR * ctx->nv);
  st = ugks_get_f(ctx, all.data(), ctx->Nc, tmp.data());
  if (st != UGKS_OK) return st;
  for (int64_t c = 0; c < ctx->Nc; ++c)
    for (int r = 0; r < ctx->NR; ++r)
      std::memcpy(f + (size_t(r) * ctx->Nc + c) * ctx->nv, &tmp[(size_t(c) * ctx->NR + r) * ctx->nv],
                  ctx->nv * sizeof(double));
  return UGKS_OK;
}

ugks_status ugks_set_state(ugks_ctx* ctx, const double* W, const double* f, int64_t step) {
  if (!ctx || !W || !f) return fail(ctx, UGKS_ERR_INVALID_ARGUMENT, "NULL argument");
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  const int D = ctx->D;
  std::vector<double> Wn(ctx->Nc * NWP, 0.0);
  for (int64_t i = 0; i < ctx->Nc; ++i)
    for (int t = 0; t < D + 2; ++t) Wn[i * NWP + t] = W[ctx->old_of_new[i] * (D + 2) + t];
  const int c = ctx->cur;
  CUDA_TRY(ctx, cudaMemcpy(ctx->d_W[c], Wn.data(), Wn.size() * sizeof(double), cudaMemcpyHostToDevice));
  double* d_in = nullptr;
  int64_t* d_map = nullptr;
  const size_t nin = size_t(ctx->NR) * ctx->Nc * ctx->nv;
  CUDA_TRY(ctx, cudaMalloc(&d_in, nin * sizeof(double)));
  cudaError_t e = cudaMalloc(&d_map, ctx->Nc * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMemcpy(d_in, f, nin * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_map, ctx->old_of_new.data(), ctx->Nc * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    if (ctx->storage == UGKS_STORAGE_F64) {
      launch_scatter_f<double>(ctx->stream, ctx->Nc, ctx->M, ctx->NR, ctx->nv, d_in, d_map,
                               static_cast<double*>(ctx->d_f[c]));
    } else if (ctx->storage == UGKS_STORAGE_F16 || ctx->storage == UGKS_STORAGE_BF16) {
      // references from the given W, then deviations against them
      launch_sref(ctx->stream, ctx->Nc, ctx->gas, ctx->d_W[c], ctx->d_ref[c]);
      if (ctx->storage == UGKS_STORAGE_F16)
        launch_sscatter<__half>(ctx->stream, ctx->Nc, ctx->M, ctx->D, ctx->NR, ctx->nv, d_in, d_map, ctx->d_ref[c],
                                ctx->d_ux, ctx->d_uy, ctx->d_uz, static_cast<__half*>(ctx->d_f[c]), ctx->d_sc[c]);
      else
        launch_sscatter<__nv_bfloat16>(ctx->stream, ctx->Nc, ctx->M, ctx->D, ctx->NR, ctx->nv, d_in, d_map,
                                       ctx->d_ref[c], ctx->d_ux, ctx->d_uy, ctx->d_uz,
                                       static_cast<__nv_bfloat16*>(ctx->d_f[c]), ctx->d_sc[c]);
    } else
      launch_scatter_f<float>(ctx->stream, ctx->Nc, ctx->M, ctx->NR, ctx->nv, d_in, d_map,
                              static_cast<float*>(ctx->d_f[c]));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    if (ctx->storage == UGKS_STORAGE_F64)
      launch_moments<double>(ctx->stream, ctx->Nc, ctx->M, ctx->gas, static_cast<const double*>(ctx->d_f[c]),
                             ctx->d_W[c], ctx->d_ux, ctx->d_uy, ctx->d_uz, ctx->d_wp, ctx->d_q[c], nullptr);
    else if (ctx->storage == UGKS_STORAGE_F16)
      launch_smoments<__half>(ctx->stream, ctx->Nc, ctx->M, ctx->nv, ctx->gas, static_cast<const __half*>(ctx->d_f[c]),
                              ctx->d_sc[c], ctx->d_ref[c], ctx->d_W[c], ctx->d_ux, ctx->d_uy, ctx->d_uz, ctx->d_wp,
                              ctx->d_q[c], nullptr);
    else if (ctx->storage == UGKS_STORAGE_BF16)
      launch_smoments<__nv_bfloat16>(ctx->stream, ctx->Nc, ctx->M, ctx->nv, ctx->gas,
                                     static_cast<const __nv_bfloat16*>(ctx->d_f[c]), ctx->d_sc[c], ctx->d_ref[c],
                                     ctx->d_W[c], ctx->d_ux, ctx->d_uy, ctx->d_uz, ctx->d_wp, ctx->d_q[c], nullptr);
    else
      launch_moments<float>(ctx->stream, ctx->Nc, ctx->M, ctx->gas, static_cast<const float*>(ctx->d_f[c]),
                            ctx->d_W[c], ctx->d_ux, ctx->d_uy, ctx->d_uz, ctx->d_wp, ctx->d_q[c], nullptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(d_in);
  if (d_map) cudaFree(d_map);
  if (e != cudaSuccess) return fail(ctx, UGKS_ERR_CUDA, "ugks_set_state: %s", cudaGetErrorString(e));
  ctx->step = step;
  return UGKS_OK;
}

ugks_status ugks_stats_enable(ugks_ctx* ctx, int32_t on) {
  if (!ctx) return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "NULL context");
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  for (auto& t : ctx->timings) {
    ctx->event_pool.push_back(t.start);
    ctx->event_pool.push_back(t.stop);
  }
  ctx->timings.clear();
  for (int i = 0; i < kNumKernels; ++i) {
    ctx->stat_ms[i] = 0.0;
    ctx->stat_count[i] = 0;
  }
  ctx->stats_on = on != 0;
  return UGKS_OK;
}

ugks_status ugks_stats(ugks_ctx* ctx, int32_t cap, const char** names, double* ms, int64_t* count, int32_t* n) {
  if (!ctx) return fail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "NULL context");
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  for (auto& t : ctx->timings) {
    float e = 0.0f;
    CUDA_TRY(ctx, cudaEventElapsedTime(&e, t.start, t.stop));
    ctx->stat_ms[t.id] += e;
    ctx->stat_count[t.id]++;
    ctx->event_pool.push_back(t.start);
    ctx->event_pool.push_back(t.stop);
  }
  ctx->timings.clear();
  for (int i = 0; i < kNumKernels && i < cap; ++i) {
    if (names) names[i] = kKernelNames[i];
    if (ms) ms[i] = ctx->stat_ms[i];
    if (count) count[i] = ctx->stat_count[i];
  }
  if (n) *n = kNumKernels;
  return UGKS_OK;
}

ugks_status ugks_solve(const ugks_mesh* mesh, const ugks_vgrid* vgrid, const ugks_params* params,
                       const double* W_init, int32_t n_steps, double* W_out, double* res_out) {
  ugks_ctx* ctx = nullptr;
  ugks_status st = ugks_create(mesh, vgrid, params, W_init, nullptr, &ctx);
  if (st != UGKS_OK) return st;
  st = ugks_step(ctx, n_steps);
  if (st == UGKS_OK && W_out) st = ugks_moments(ctx, W_out, nullptr);
  if (st == UGKS_OK && res_out) st = ugks_residual(ctx, res_out);
  if (st != UGKS_OK) g_thread_err = ctx->err;
  ugks_destroy(ctx);
  return st;
}

ugks_status ugks_destroy(ugks_ctx* ctx) {
  if (!ctx) return UGKS_OK;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  release(ctx);
  delete ctx;
  return UGKS_OK;
}

const char* ugks_last_error(const ugks_ctx* ctx) {
  if (ctx) return ctx->err.c_str();
  return g_thread_err.c_str();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches of cases: one CUDA-graph launch advances every case by two steps
// (the graph holds two steps of each case, so the double buffers return to
// their starting parity), each case on its own forked stream so that small
// cases run concurrently; a block-size autotuner per case.
// ---------------------------------------------------------------------------
struct ugks_batch {
  std::vector<ugks_ctx*> cases;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaEvent_t fork = nullptr, done = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<int> tuned_bv;                 // velocities per block chosen by the autotuner (0: not tuned)
  std::vector<std::vector<double>> tune_ms;  // ms per step of each block-size candidate (32, 64, 128, 256)
  std::vector<int> tuned_fused, tuned_chunks;  // organisation and second-stage chunks chosen with it
  std::vector<double> tuned_best_ms;           // ms per step of the chosen shape
  std::vector<int> tune_trials;                // shapes timed for the case (0: from the cache)
  std::string err;
};

namespace {

using TuneKey = std::tuple<int64_t, int64_t, int, int, int>;  // cells, velocities, dim, reduced, storage
struct TuneShape {
  int vb;        // velocities per block lane (1, 2, 4 or 8)
  int fused;     // fluxes evaluated per cell in the first-stage kernel
  int nchunk;    // velocity chunks of the second stage
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneShape> g_tune_cache;

ugks_status bfail(ugks_batch* b, ugks_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (b) b->err = buf;
  g_thread_err = buf;
  return st;
}

void batch_release(ugks_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  b->join.clear();
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->done) cudaEventDestroy(b->done);
  for (ugks_ctx* c : b->cases) ugks_destroy(c);
  b->cases.clear();
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

ugks_status ctx_step(ugks_ctx* ctx) {
#define UGKS_STEP(T, S) step_typed<T, S>(ctx)
  return UGKS_BY_STORAGE(ctx, UGKS_STEP);
#undef UGKS_STEP
}

// The batch stream waits for the work queued on every case stream, or the
// case streams wait for the batch stream.
cudaError_t batch_join_cases(ugks_batch* b) {
  for (size_t i = 0; i < b->cases.size(); ++i) {
    cudaError_t e = cudaEventRecord(b->join[i], b->cases[i]->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join[i], 0);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
cudaError_t batch_release_cases(ugks_batch* b) {
  cudaError_t e = cudaEventRecord(b->done, b->stream);
  for (size_t i = 0; e == cudaSuccess && i < b->cases.size(); ++i) e = cudaStreamWaitEvent(b->cases[i]->stream, b->done, 0);
  return e;
}

ugks_status batch_capture(ugks_batch* b) {
  const size_t n = b->cases.size();
  std::vector<int> cur(n);
  std::vector<int64_t> step(n);
  std::vector<bool> stats(n);
  for (size_t i = 0; i < n; ++i) {
    cur[i] = b->cases[i]->cur;
    step[i] = b->cases[i]->step;
    stats[i] = b->cases[i]->stats_on;
    b->cases[i]->stats_on = false;
  }
  ugks_status st = UGKS_OK;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->stream);
  for (size_t i = 0; e == cudaSuccess && st == UGKS_OK && i < n; ++i) {
    ugks_ctx* c = b->cases[i];
    e = cudaStreamWaitEvent(c->stream, b->fork, 0);
    for (int k = 0; e == cudaSuccess && st == UGKS_OK && k < 2; ++k) st = ctx_step(c);
    if (e == cudaSuccess && st == UGKS_OK) e = cudaEventRecord(b->join[i], c->stream);
    if (e == cudaSuccess && st == UGKS_OK) e = cudaStreamWaitEvent(b->stream, b->join[i], 0);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e_end = cudaStreamEndCapture(b->stream, &g);
  for (size_t i = 0; i < n; ++i) {  // the capture recorded the steps; none ran
    b->cases[i]->cur = cur[i];
    b->cases[i]->step = step[i];
    b->cases[i]->stats_on = stats[i];
  }
  if (st != UGKS_OK) {
    if (g) cudaGraphDestroy(g);
    return bfail(b, st, "capturing the batch step failed: %s", ugks_last_error(nullptr));
  }
  if (e == cudaSuccess) e = e_end;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    b->exec = nullptr;
    return bfail(b, UGKS_ERR_CUDA, "capturing the batch step failed: %s", cudaGetErrorString(e));
  }
  b->graph = g;
  return UGKS_OK;
}

}  // namespace

extern "C" {

ugks_status ugks_batch_create(int32_t n, const ugks_mesh* const* meshes, const ugks_vgrid* const* vgrids,
                              const ugks_params* params, const double* const* W_init, void* cuda_stream,
                              ugks_batch** out) {
  if (!out) return bfail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "out must not be NULL");
  *out = nullptr;
  if (n < 1 || !meshes || !vgrids || !params)
    return bfail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "a batch needs n >= 1 meshes, grids and parameter sets");
  for (int32_t i = 0; i < n; ++i)
    if (params[i].sweep == UGKS_SWEEP_TILED)
      return bfail(nullptr, UGKS_ERR_UNSUPPORTED, "case %d: batches run the blocked sweep", i);
  ugks_batch* b = new (std::nothrow) ugks_batch();
  if (!b) return bfail(nullptr, UGKS_ERR_OUT_OF_MEMORY, "host allocation failed");
  cudaError_t e = cudaSuccess;
  if (cuda_stream) {
    b->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    b->own_stream = e == cudaSuccess;
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    batch_release(b);
    delete b;
    return bfail(nullptr, UGKS_ERR_CUDA, "batch set-up: %s", cudaGetErrorString(e));
  }
  for (int32_t i = 0; i < n; ++i) {
    ugks_ctx* c = nullptr;
    ugks_status st = ugks_create(meshes[i], vgrids[i], &params[i], W_init ? W_init[i] : nullptr, nullptr, &c);
    if (st != UGKS_OK) {
      std::string msg = g_thread_err;
      batch_release(b);
      delete b;
      return bfail(nullptr, st, "case %d: %s", i, msg.c_str());
    }
    b->cases.push_back(c);
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      batch_release(b);
      delete b;
      return bfail(nullptr, UGKS_ERR_CUDA, "batch set-up: %s", cudaGetErrorString(e));
    }
    b->join.push_back(ev);
    // a shape tuned earlier in this process needs no tuning steps
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(TuneKey(c->Nc, c->nv, c->D, c->NR, c->storage));
    b->tuned_bv.push_back(0);
    b->tune_ms.push_back(std::vector<double>(4, 0.0));
    b->tuned_fused.push_back(c->fused ? 1 : 0);
    b->tuned_chunks.push_back(c->nchunk);
    b->tuned_best_ms.push_back(0.0);
    b->tune_trials.push_back(0);
    if (it != g_tune_cache.end() && it->second.vb <= c->vb_max && it->second.nchunk <= c->nchunk) {
      c->vb = it->second.vb;
      c->fused = it->second.fused != 0;
      c->nchunk = it->second.nchunk;
      b->tuned_bv.back() = it->second.vb * BV;
      b->tuned_fused.back() = it->second.fused;
      b->tuned_chunks.back() = it->second.nchunk;
    }
  }
  *out = b;
  return UGKS_OK;
}

ugks_status ugks_batch_autotune(ugks_batch* b) {
  if (!b) return bfail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "NULL batch");
  if (b->exec) {  // a new block size changes the kernels: recapture on the next step
    cudaGraphExecDestroy(b->exec);
    cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
  }
  if (batch_release_cases(b) != cudaSuccess) return bfail(b, UGKS_ERR_CUDA, "autotune: stream ordering failed");
  cudaEvent_t t0, t1;
  if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess)
    return bfail(b, UGKS_ERR_CUDA, "autotune: event creation failed");
  ugks_status st = UGKS_OK;
  // ms of the second of two steps at the case's current shape (the first
  // takes any set-up outside the timing)
  auto time_shape = [&](ugks_ctx* c, double& ms_out) -> ugks_status {
    ugks_status s2 = ctx_step(c);
    if (s2 != UGKS_OK) return s2;
    cudaEventRecord(t0, c->stream);
    s2 = ctx_step(c);
    cudaEventRecord(t1, c->stream);
    if (s2 != UGKS_OK) return s2;
    float ms = 0.f;
    if (cudaEventSynchronize(t1) != cudaSuccess || cudaEventElapsedTime(&ms, t0, t1) != cudaSuccess)
      return bfail(b, UGKS_ERR_CUDA, "autotune: timing failed");
    ms_out = ms;
    return UGKS_OK;
  };
  for (size_t i = 0; st == UGKS_OK && i < b->cases.size(); ++i) {
    ugks_ctx* c = b->cases[i];
    if (b->tuned_bv[i]) continue;
    // coordinate search: block size (split form, all chunks), then the
    // organisation (split / fused), then the second stage's chunk count
    const int chunks_max = c->nchunk;
    int trials = 0;
    TuneShape best{c->vb, 0, chunks_max};
    double best_ms = 1e300;
    c->fused = false;
    for (int v = 1, slot = 0; v <= c->vb_max && st == UGKS_OK; v *= 2, ++slot) {
      c->vb = v;
      double ms = 0.0;
      st = time_shape(c, ms);
      if (st != UGKS_OK) break;
      ++trials;
      b->tune_ms[i][slot] = ms;
      if (ms < best_ms) {
        best_ms = ms;
        best.vb = v;
      }
    }
    if (st != UGKS_OK) break;
    c->vb = best.vb;
    c->fused = true;
    {
      double ms = 0.0;
      st = time_shape(c, ms);
      if (st != UGKS_OK) break;
      ++trials;
      if (ms < best_ms && c->fused_used) {   // only where the fused kernel's stages fit
        best_ms = ms;
        best.fused = 1;
      }
    }
    c->fused = best.fused != 0;
    for (int ch = chunks_max / 2; ch >= 1 && ch >= chunks_max / 8; ch /= 2) {
      c->nchunk = ch;
      double ms = 0.0;
      st = time_shape(c, ms);
      if (st != UGKS_OK) break;
      ++trials;
      if (ms < best_ms) {
        best_ms = ms;
        best.nchunk = ch;
      }
    }
    if (st != UGKS_OK) break;
    c->vb = best.vb;
    c->fused = best.fused != 0;
    c->nchunk = best.nchunk;
    b->tuned_bv[i] = best.vb * BV;
    b->tuned_fused[i] = best.fused;
    b->tuned_chunks[i] = best.nchunk;
    b->tuned_best_ms[i] = best_ms;
    b->tune_trials[i] = trials;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[TuneKey(c->Nc, c->nv, c->D, c->NR, c->storage)] = best;
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (st != UGKS_OK && b->err.empty()) b->err = g_thread_err;
  return st;
}

ugks_status ugks_batch_step(ugks_batch* b, int32_t n_steps) {
  if (!b) return bfail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "NULL batch");
  if (n_steps < 0) return bfail(b, UGKS_ERR_INVALID_ARGUMENT, "n_steps must be >= 0");
  if (n_steps >= 2 && !b->exec) {
    ugks_status st = batch_capture(b);
    if (st != UGKS_OK) return st;
  }
  cudaError_t e = batch_join_cases(b);
  for (int32_t k = 0; e == cudaSuccess && k + 1 < n_steps; k += 2) {
    e = cudaGraphLaunch(b->exec, b->stream);
    for (ugks_ctx* c : b->cases) c->step += 2;
  }
  if (e == cudaSuccess) e = batch_release_cases(b);
  if (e != cudaSuccess) return bfail(b, UGKS_ERR_CUDA, "batch step: %s", cudaGetErrorString(e));
  if (n_steps % 2) {
    for (ugks_ctx* c : b->cases) {
      ugks_status st = ctx_step(c);
      if (st != UGKS_OK) return bfail(b, st, "batch step: %s", c->err.c_str());
    }
  }
  return UGKS_OK;
}

ugks_status ugks_batch_context(ugks_batch* b, int32_t i, ugks_ctx** ctx_out) {
  if (!b || !ctx_out || i < 0 || i >= int32_t(b->cases.size()))
    return bfail(b, UGKS_ERR_INVALID_ARGUMENT, "no case %d in this batch", i);
  *ctx_out = b->cases[i];
  return UGKS_OK;
}

ugks_status ugks_batch_tuning(ugks_batch* b, int32_t i, int32_t* block_velocities, double* ms_per_step) {
  if (!b || i < 0 || i >= int32_t(b->cases.size()))
    return bfail(b, UGKS_ERR_INVALID_ARGUMENT, "no case %d in this batch", i);
  if (block_velocities) *block_velocities = b->tuned_bv[i] ? b->tuned_bv[i] : b->cases[i]->vb * BV;
  if (ms_per_step)
    for (int k = 0; k < 4; ++k) ms_per_step[k] = b->tune_ms[i][k];
  return UGKS_OK;
}

ugks_status ugks_batch_shape(ugks_batch* b, int32_t i, int32_t* block_velocities, int32_t* fused,
                             int32_t* stage2_chunks, double* ms_per_step, int32_t* trials) {
  if (!b || i < 0 || i >= int32_t(b->cases.size()))
    return bfail(b, UGKS_ERR_INVALID_ARGUMENT, "no case %d in this batch", i);
  const ugks_ctx* c = b->cases[i];
  if (block_velocities) *block_velocities = c->vb * BV;
  if (fused) *fused = c->fused ? 1 : 0;
  if (stage2_chunks) *stage2_chunks = c->nchunk;
  if (ms_per_step) *ms_per_step = b->tuned_best_ms[i];
  if (trials) *trials = b->tune_trials[i];
  return UGKS_OK;
}

ugks_status ugks_create_batch(int32_t n, const ugks_mesh* const* meshes, const ugks_vgrid* const* vgrids,
                              const ugks_params* params, const double* const* W_init, void* cuda_stream,
                              ugks_batch** out) {
  return ugks_batch_create(n, meshes, vgrids, params, W_init, cuda_stream, out);
}

ugks_status ugks_step_batch(ugks_batch* b, int32_t n_steps) { return ugks_batch_step(b, n_steps); }

ugks_status ugks_batch_destroy(ugks_batch* b) {
  if (!b) return UGKS_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_release(b);
  delete b;
  return UGKS_OK;
}

}  // extern "C"
