// FP16 / BF16 scaled storage of f (ugks_store.cuh): initialisation, velocity
// moments and the host gather / scatter of the checkpoint calls.  The sweep
// kernels decode and encode rows themselves (ugks_blocked.cuh).
#include <cmath>
#include <cstdint>

#include "ugks_device.cuh"
#include "ugks_internal.cuh"
#include "ugks_kernels.cuh"
#include "ugks_store.cuh"

namespace ugks {

namespace {

// Primitive record (rho, U, lambda) of a conservative state, R = 1/2.
template <int D>
__device__ __forceinline__ CellPrim prim_from_W(const double* W, int K) {
  CellPrim p{};
  p.rho = W[0];
  double u2 = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    p.U[d] = W[1 + d] / W[0];
    u2 += p.U[d] * p.U[d];
  }
  p.lam = (K + 3) * W[0] / (4.0 * (W[D + 1] - 0.5 * W[0] * u2));
  return p;
}

template <int D>
__device__ __forceinline__ void vel3(const double* ux, const double* uy, const double* uz, int64_t k, float (&u)[3]) {
  u[0] = float(ux[k]);
  u[1] = D > 1 ? float(uy[k]) : 0.f;
  u[2] = D > 2 ? float(uz[k]) : 0.f;
}

// Reference Maxwellian of every cell from W (its discrete Maxwellian is then
// the stored f with zero deviations).
template <int D>
__global__ void k_sref(int64_t Nc, int K, int Kxi, const double* W, RefMaxwell* ref) {
  const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= Nc) return;
  ref[c] = make_ref<D>(prim_from_W<D>(W + c * NWP, K), Kxi);
}

// Heat flux about U of W (Eq. 13) and, optionally, the discrete conservative
// moments of the decoded f.  One warp per cell.
template <int D, typename S>
__global__ void k_smoments(int64_t Nc, int64_t M, int NR, int64_t nv, int K, const S* f, const float* sc,
                           const RefMaxwell* ref, const double* W, const double* ux, const double* uy,
                           const double* uz, const double* w, double* q_out, double* Wf_out) {
  const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= Nc) return;
  const CellPrim p = prim_from_W<D>(W + i * NWP, K);
  const RefMaxwell R = ref[i];
  double qa[3] = {0.0, 0.0, 0.0}, ma[3] = {0.0, 0.0, 0.0}, m0 = 0.0, mE = 0.0;
  for (int64_t m = 0; m < M; ++m) {
    const int64_t k = m * BV + lane;
    float u[3];
    vel3<D>(ux, uy, uz, k, u);
    const bool real = k < nv;
    const float g = ref_value<D>(R, 0, u, real);
    const size_t row0 = size_t(m) * Nc + size_t(i);
    const double h = decode_value(f[row0 * BV + lane], sc[row0], g);
    double b = 0.0;
    if (NR == 2) {
      const size_t row1 = (size_t(M) + m) * Nc + size_t(i);
      b = decode_value(f[row1 * BV + lane], sc[row1], R.kap * g);
    }
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
  for (int d = 0; d < D; ++d) {
    qa[d] = warp_sum(qa[d]);
    ma[d] = warp_sum(ma[d]);
  }
  m0 = warp_sum(m0);
  mE = warp_sum(mE);
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

// Decoded f of selected cells: out[s][r][k], FP64.
template <int D, typename S>
__global__ void k_sgather(int64_t Nc, int64_t M, int NR, int64_t nv, const S* f, const float* sc,
                          const RefMaxwell* ref, const double* ux, const double* uy, const double* uz,
                          const int64_t* sel, int64_t n, double* out) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= n * NR * nv) return;
  const int64_t k = idx % nv, r = (idx / nv) % NR, s = idx / (nv * NR);
  const int64_t c = sel[s], m = k / BV, lane = k % BV;
  float u[3];
  vel3<D>(ux, uy, uz, k, u);
  const size_t row = (size_t(r) * M + m) * Nc + size_t(c);
  out[idx] = decode_value(f[row * BV + lane], sc[row], ref_value<D>(ref[c], int(r), u, true));
}

// Encodes a full FP64 state in[NR][Nc_orig][nv] (original cell order): one
// warp per stored row.
template <int D, typename S>
__global__ void k_sscatter(int64_t Nc, int64_t M, int NR, int64_t nv, const double* in, const int64_t* old_of_new,
                           const RefMaxwell* ref, const double* ux, const double* uy, const double* uz, S* f,
                           float* sc) {
  const int64_t row = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= int64_t(NR) * M * Nc) return;
  const int64_t c = row % Nc, m = (row / Nc) % M, r = row / (Nc * M);
  const int64_t k = m * BV + lane;
  const bool real = k < nv;
  float u[3];
  vel3<D>(ux, uy, uz, k, u);
  const float v = real ? float(in[(size_t(r) * Nc + old_of_new[c]) * nv + k]) : 0.f;
  float scale;
  const S d = encode_value<S>(v, ref_value<D>(ref[c], int(r), u, real), scale);
  f[size_t(row) * BV + lane] = d;
  if (lane == 0) sc[row] = scale;
}

inline unsigned nblocks(int64_t n, int threads) { return unsigned((n + threads - 1) / threads); }

}  // namespace

void launch_sref(cudaStream_t s, int64_t Nc, const Gas& g, const double* W, RefMaxwell* ref) {
  const unsigned nb = nblocks(Nc, 128);
  if (g.D == 1) k_sref<1><<<nb, 128, 0, s>>>(Nc, g.K, g.Kxi, W, ref);
  if (g.D == 2) k_sref<2><<<nb, 128, 0, s>>>(Nc, g.K, g.Kxi, W, ref);
  if (g.D == 3) k_sref<3><<<nb, 128, 0, s>>>(Nc, g.K, g.Kxi, W, ref);
}

template <typename S>
void launch_smoments(cudaStream_t s, int64_t Nc, int64_t M, int64_t nv, const Gas& g, const S* f, const float* sc,
                     const RefMaxwell* ref, const double* W, const double* ux, const double* uy, const double* uz,
                     const double* w, double* q_out, double* Wf_out) {
  const unsigned nb = nblocks(Nc * 32, 256);
  if (g.D == 1) k_smoments<1, S><<<nb, 256, 0, s>>>(Nc, M, g.NR, nv, g.K, f, sc, ref, W, ux, uy, uz, w, q_out, Wf_out);
  if (g.D == 2) k_smoments<2, S><<<nb, 256, 0, s>>>(Nc, M, g.NR, nv, g.K, f, sc, ref, W, ux, uy, uz, w, q_out, Wf_out);
  if (g.D == 3) k_smoments<3, S><<<nb, 256, 0, s>>>(Nc, M, g.NR, nv, g.K, f, sc, ref, W, ux, uy, uz, w, q_out, Wf_out);
}

template <typename S>
void launch_sgather(cudaStream_t s, int64_t Nc, int64_t M, int D, int NR, int64_t nv, const S* f, const float* sc,
                    const RefMaxwell* ref, const double* ux, const double* uy, const double* uz, const int64_t* sel,
                    int64_t n, double* out) {
  if (n * NR * nv == 0) return;
  const unsigned nb = nblocks(n * NR * nv, 256);
  if (D == 1) k_sgather<1, S><<<nb, 256, 0, s>>>(Nc, M, NR, nv, f, sc, ref, ux, uy, uz, sel, n, out);
  if (D == 2) k_sgather<2, S><<<nb, 256, 0, s>>>(Nc, M, NR, nv, f, sc, ref, ux, uy, uz, sel, n, out);
  if (D == 3) k_sgather<3, S><<<nb, 256, 0, s>>>(Nc, M, NR, nv, f, sc, ref, ux, uy, uz, sel, n, out);
}

template <typename S>
void launch_sscatter(cudaStream_t s, int64_t Nc, int64_t M, int D, int NR, int64_t nv, const double* in,
                     const int64_t* old_of_new, const RefMaxwell* ref, const double* ux, const double* uy,
                     const double* uz, S* f, float* sc) {
  const unsigned nb = nblocks(int64_t(NR) * M * Nc * 32, 256);
  if (D == 1) k_sscatter<1, S><<<nb, 256, 0, s>>>(Nc, M, NR, nv, in, old_of_new, ref, ux, uy, uz, f, sc);
  if (D == 2) k_sscatter<2, S><<<nb, 256, 0, s>>>(Nc, M, NR, nv, in, old_of_new, ref, ux, uy, uz, f, sc);
  if (D == 3) k_sscatter<3, S><<<nb, 256, 0, s>>>(Nc, M, NR, nv, in, old_of_new, ref, ux, uy, uz, f, sc);
}

#define UGKS_INSTANTIATE_STORE(S)                                                                               \
  template void launch_smoments<S>(cudaStream_t, int64_t, int64_t, int64_t, const Gas&, const S*, const float*,   \
                                   const RefMaxwell*, const double*, const double*, const double*, const double*, \
                                   const double*, double*, double*);                                              \
  template void launch_sgather<S>(cudaStream_t, int64_t, int64_t, int, int, int64_t, const S*, const float*,      \
                                  const RefMaxwell*, const double*, const double*, const double*, const int64_t*,  \
                                  int64_t, double*);                                                              \
  template void launch_sscatter<S>(cudaStream_t, int64_t, int64_t, int, int, int64_t, const double*,              \
                                   const int64_t*, const RefMaxwell*, const double*, const double*, const double*, \
                                   S*, float*);
UGKS_INSTANTIATE_STORE(__half)
UGKS_INSTANTIATE_STORE(__nv_bfloat16)

}  // namespace ugks
