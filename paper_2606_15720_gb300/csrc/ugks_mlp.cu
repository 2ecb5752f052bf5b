// Warm-start network: a multilayer perceptron (tanh hidden layers, linear
// output) trained and evaluated by this library's own kernels.
//
// Maps per-cell features (Mach, log10 Kn, centroid x, y, z, wall distance)
// to the thirteen-moment fields of a converged steady state (rho, U, T,
// deviatoric stress, heat flux), whose Chapman-Enskog distribution starts a
// steady solve (ugks_init_moments13).  Weights and activations are BF16,
// products accumulate in FP32 on the tensor cores (mma.sync m16n8k16),
// master weights and Adam moments are FP32.  Layer widths are padded to
// multiples of 16 with zero weights, which the gradients keep at zero.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "ugks.h"

namespace {

using bf16 = __nv_bfloat16;

inline int pad16(int n) { return (n + 15) / 16 * 16; }

// ---------------------------------------------------------------------------
// C[M][N] = A[M][K] B[K][N]: BF16 operands with arbitrary strides, FP32
// accumulation on the tensor cores.  Four warps (2 x 2) per CTA, each WM x WN
// mma tiles of 16 x 8 x 16: CTA tiles of 64 x 64 (WM 2, WN 4) or, when that
// leaves the GPU mostly idle, 32 x 32 (WM 1, WN 2); K in steps of 32.  Both
// operand tiles are kept K-contiguous in shared memory, the layout the mma
// fragments read.
// ---------------------------------------------------------------------------
constexpr int kTK = 32, kSK = kTK + 8;  // kSK: padded row (bank spread)

struct GemmArgs {
  int M, N, K;
  const bf16* A;
  int64_t a_m, a_k;  // A(i, k) = A[i a_m + k a_k]
  const bf16* B;
  int64_t b_k, b_n;  // B(k, j) = B[k b_k + j b_n]
  int a_mode, b_mode;// operand tile loads (load_tile), set by gemm()
  int mode;          // 0: + bias, activation; 1: times (1 - aprev^2); 2: plain
  const float* bias; // mode 0, [N]
  int act;           // mode 0: 1 = tanh
  const float* aprev;// mode 1, [M][ldc]
  int valid_n;       // columns >= valid_n are stored as 0 (padding)
  float* C;
  int64_t ldc;
  bf16* Cb;          // optional BF16 copy, same leading dimension
};

__device__ __forceinline__ uint32_t ld_pair(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One operand tile S[r][k] = P(r0 + r, k0 + k) (rows x kTK, zero outside
// rows_total x K) with element (r, k) at P[r s_r + k s_k].  mode 1: 16-byte
// vectors along k (s_k == 1); mode 2: 16-byte vectors along r (s_r == 1);
// mode 0: single elements.
template <int ROWS>
__device__ __forceinline__ void load_tile(const bf16* __restrict__ P, int64_t s_r, int64_t s_k, int rows_total,
                                          int K, int r0, int k0, int mode, bf16 (*S)[kSK], int tid) {
  const bf16 zero = __float2bfloat16_rn(0.f);
  if (mode == 1) {
    for (int v = tid; v < ROWS * kTK / 8; v += 128) {
      const int r = v / (kTK / 8), k = (v % (kTK / 8)) * 8;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (r0 + r < rows_total && k0 + k < K) val = *reinterpret_cast<const uint4*>(P + (r0 + r) * s_r + (k0 + k));
      *reinterpret_cast<uint4*>(&S[r][k]) = val;
    }
  } else if (mode == 2) {
    for (int v = tid; v < ROWS * kTK / 8; v += 128) {
      const int k = v / (ROWS / 8), r = (v % (ROWS / 8)) * 8;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (r0 + r < rows_total && k0 + k < K) val = *reinterpret_cast<const uint4*>(P + (k0 + k) * s_k + (r0 + r));
      const bf16* e = reinterpret_cast<const bf16*>(&val);
#pragma unroll
      for (int j = 0; j < 8; ++j) S[r + j][k] = e[j];
    }
  } else {
    for (int idx = tid; idx < ROWS * kTK; idx += 128) {
      const int r = idx / kTK, k = idx % kTK;
      S[r][k] = (r0 + r < rows_total && k0 + k < K) ? P[(r0 + r) * s_r + (k0 + k) * s_k] : zero;
    }
  }
}

// vector mode of an operand: rows_total and K must be multiples of 8 so that a
// vector never straddles the valid range, and the base 16-byte aligned
__host__ int tile_mode(const bf16* P, int64_t s_r, int64_t s_k, int rows_total, int K) {
  if (reinterpret_cast<uintptr_t>(P) % 16 != 0 || rows_total % 8 != 0 || K % 8 != 0) return 0;
  if (s_k == 1 && s_r % 8 == 0) return 1;
  if (s_r == 1 && s_k % 8 == 0) return 2;
  return 0;
}

template <int WM, int WN>
__global__ void __launch_bounds__(128) k_gemm(const GemmArgs g) {
  constexpr int TM = 32 * WM, TN = 16 * WN;  // CTA tile
  __shared__ __align__(16) bf16 As[TM][kSK];
  __shared__ __align__(16) bf16 Bs[TN][kSK];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;
  const int gid = lane >> 2, tig = lane & 3;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  float acc[WM][WN][4];
#pragma unroll
  for (int i = 0; i < WM; ++i)
#pragma unroll
    for (int j = 0; j < WN; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
  for (int k0 = 0; k0 < g.K; k0 += kTK) {
    load_tile<TM>(g.A, g.a_m, g.a_k, g.M, g.K, m0, k0, g.a_mode, As, tid);
    load_tile<TN>(g.B, g.b_n, g.b_k, g.N, g.K, n0, k0, g.b_mode, Bs, tid);
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kTK; ks += 16) {
      uint32_t af[WM][4], bfr[WN][2];
#pragma unroll
      for (int mi = 0; mi < WM; ++mi) {
        const int r = wm * 16 * WM + mi * 16 + gid;
        af[mi][0] = ld_pair(&As[r][ks + 2 * tig]);
        af[mi][1] = ld_pair(&As[r + 8][ks + 2 * tig]);
        af[mi][2] = ld_pair(&As[r][ks + 2 * tig + 8]);
        af[mi][3] = ld_pair(&As[r + 8][ks + 2 * tig + 8]);
      }
#pragma unroll
      for (int ni = 0; ni < WN; ++ni) {
        const int c = wn * 8 * WN + ni * 8 + gid;
        bfr[ni][0] = ld_pair(&Bs[c][ks + 2 * tig]);
        bfr[ni][1] = ld_pair(&Bs[c][ks + 2 * tig + 8]);
      }
#pragma unroll
      for (int mi = 0; mi < WM; ++mi)
#pragma unroll
        for (int ni = 0; ni < WN; ++ni) mma_bf16(acc[mi][ni], af[mi], bfr[ni]);
    }
    __syncthreads();
  }
  // epilogue: accumulator r of tile (mi, ni) is row gid (+8 for r >= 2), column 2 tig + (r & 1)
#pragma unroll
  for (int mi = 0; mi < WM; ++mi)
#pragma unroll
    for (int ni = 0; ni < WN; ++ni)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = m0 + wm * 16 * WM + mi * 16 + gid + (r >= 2 ? 8 : 0);
        const int col = n0 + wn * 8 * WN + ni * 8 + 2 * tig + (r & 1);
        if (row >= g.M || col >= g.N) continue;
        float v = acc[mi][ni][r];
        const int64_t o = row * g.ldc + col;
        if (g.mode == 0) {
          v += g.bias[col];
          if (g.act) v = tanhf(v);
        } else if (g.mode == 1) {
          const float a = g.aprev[o];
          v *= 1.f - a * a;
        }
        if (col >= g.valid_n) v = 0.f;
        g.C[o] = v;
        if (g.Cb) g.Cb[o] = __float2bfloat16_rn(v);
      }
}

// bias gradient db[j] = sum_s dz[s][j]: a CTA of 32 columns x 8 row groups,
// reduced in shared memory in a fixed order (reproducible).
__global__ void __launch_bounds__(256) k_colsum(int rows, int cols, const float* dz, int64_t ld, float* out) {
  __shared__ float part[8][33];
  const int jj = threadIdx.x & 31, rg = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + jj;
  float s = 0.f;
  if (j < cols)
    for (int r = rg; r < rows; r += 8) s += dz[r * ld + j];
  part[rg][jj] = s;
  __syncthreads();
  if (rg == 0 && j < cols) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += part[k][jj];
    out[j] = t;
  }
}

// Distance from every cell centroid to the nearest centroid of a wall face
// (brute force over the wall faces, FP64).
__global__ void k_wall_distance(int64_t Nc, int dim, const double* xc, int64_t nw, const double* xw, double* d) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= Nc) return;
  double best = nw > 0 ? 1e300 : 0.0;
  for (int64_t w = 0; w < nw; ++w) {
    double r2 = 0.0;
    for (int k = 0; k < dim; ++k) {
      const double t = xc[i * dim + k] - xw[w * dim + k];
      r2 += t * t;
    }
    best = fmin(best, r2);
  }
  d[i] = sqrt(best);
}

// Batch input and targets from the data set by index, normalised:
// x0 = (x - shift) / scale as BF16 (zero padding), t = (y - shift) / scale.
__global__ void k_gather(int nb, int nvalid, const int64_t* idx, const int64_t* cursor, const float* X, int n_in,
                         int in_pad, const float* Y, int n_out, const float* in_shift, const float* in_scale,
                         const float* out_shift, const float* out_scale, bf16* x0, float* t) {
  const int s = blockIdx.x;
  if (s >= nb) return;
  if (cursor) idx += *cursor;  // training: the batch's offset in the shuffled order
  for (int j = threadIdx.x; j < in_pad; j += blockDim.x) {
    float v = 0.f;
    if (s < nvalid && j < n_in) v = (X[idx[s] * n_in + j] - in_shift[j]) / in_scale[j];
    x0[int64_t(s) * in_pad + j] = __float2bfloat16_rn(v);
  }
  if (t)
    for (int j = threadIdx.x; j < n_out; j += blockDim.x)
      t[int64_t(s) * n_out + j] = s < nvalid ? (Y[idx[s] * n_out + j] - out_shift[j]) / out_scale[j] : 0.f;
}

// Mean-squared error on the valid samples and outputs and its gradient:
// dy = 2 (y - t) / (nvalid n_out); padding rows and columns get 0.
__global__ void k_mse(int nb, int nvalid, int n_out, int out_pad, const float* y, const float* t, float* dy,
                      bf16* dyb, double* loss) {
  __shared__ double part[256];
  double acc = 0.0;
  const int total = nb * out_pad;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int s = i / out_pad, j = i % out_pad;
    float g = 0.f;
    if (s < nvalid && j < n_out) {
      const float d = y[i] - t[int64_t(s) * n_out + j];
      acc += double(d) * d;
      g = 2.f * d / float(double(nvalid) * n_out);
    }
    dy[i] = g;
    dyb[i] = __float2bfloat16_rn(g);
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, part[0] / (double(nvalid) * n_out));
}

// Adam on FP32 master parameters (bias-corrected, step t = *step + 1);
// refreshes the BF16 weights.
__global__ void k_adam(int64_t n, float* p, const float* gr, float* m, float* v, bf16* pb, float lr, const int* step) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float t = float(*step + 1);
  const float c1 = 1.f - powf(0.9f, t), c2 = 1.f - powf(0.999f, t);
  const float g = gr[i];
  const float mm = 0.9f * m[i] + 0.1f * g;
  const float vv = 0.999f * v[i] + 0.001f * g * g;
  m[i] = mm;
  v[i] = vv;
  const float w = p[i] - lr * (mm / c1) / (sqrtf(vv / c2) + 1e-8f);
  p[i] = w;
  if (pb) pb[i] = __float2bfloat16_rn(w);
}

// after a training step: next batch, next Adam step
__global__ void k_train_advance(int64_t* cursor, int64_t batch, int* step) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *cursor += batch;
    *step += 1;
  }
}

__global__ void k_to_bf16(int64_t n, const float* a, bf16* b) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

// output de-normalisation: y = y_net scale + shift on the valid outputs
__global__ void k_denorm(int nb, int n_out, int out_pad, const float* y, const float* shift, const float* scale,
                         float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb * n_out) return;
  const int s = i / n_out, j = i % n_out;
  out[i] = y[int64_t(s) * out_pad + j] * scale[j] + shift[j];
}

thread_local std::string g_mlp_err;

}  // namespace

struct ugks_mlp {
  int n_in = 0, n_out = 0, width = 0, hidden = 0, L = 0;
  std::vector<int> din, dout, rin, rout;       // padded and real in / out widths per layer
  std::vector<int64_t> woff, boff;             // offsets of W_l and b_l in the parameter arrays
  int64_t nW = 0, nb = 0;
  float *W = nullptr, *b = nullptr, *mW = nullptr, *vW = nullptr, *mb = nullptr, *vb = nullptr;
  float *gW = nullptr, *gb = nullptr;
  bf16* Wb = nullptr;
  float *norm = nullptr;                       // in_shift, in_scale, out_shift, out_scale (device)
  std::vector<float> hnorm;
  int max_batch = 4096;
  std::vector<float*> actf;                    // [L+1] FP32 layer outputs (actf[0] unused)
  std::vector<bf16*> actb;                     // [L+1] BF16 layer outputs (actb[0] = input)
  std::vector<float*> dzf;                     // [L] FP32 gradients at layer outputs
  std::vector<bf16*> dzb;
  float* tgt = nullptr;
  double* dloss = nullptr;
  int64_t* didx = nullptr;
  float *dX = nullptr, *dY = nullptr;
  int64_t data_cap = 0;
  int* d_step = nullptr;          // Adam steps taken (device)
  int64_t* d_cursor = nullptr;    // offset of the next training batch in the shuffled order (device)
  cudaGraph_t train_graph = nullptr;
  cudaGraphExec_t train_exec = nullptr;  // one full training step (gather .. Adam), replayed per batch
  int train_batch = 0;
  float train_lr = 0.f;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<void*> allocs;
  std::string err;
};

namespace {

ugks_status mfail(ugks_mlp* n, ugks_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (n) n->err = buf;
  g_mlp_err = buf;
  return st;
}

#define MLP_TRY(n, call)                                                                            \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      return mfail(n, e_ == cudaErrorMemoryAllocation ? UGKS_ERR_OUT_OF_MEMORY : UGKS_ERR_CUDA,     \
                   "%s: %s", #call, cudaGetErrorString(e_));                                        \
  } while (0)

template <typename P>
cudaError_t malloc_n(ugks_mlp* n, P** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(P));
  if (e != cudaSuccess) return e;
  n->allocs.push_back(q);
  *p = static_cast<P*>(q);
  return cudaMemsetAsync(q, 0, std::max<size_t>(count, 1) * sizeof(P), n->stream);
}

// splitmix64: deterministic initial weights
uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

void gemm(cudaStream_t s, GemmArgs g) {
  g.a_mode = tile_mode(g.A, g.a_m, g.a_k, g.M, g.K);
  g.b_mode = tile_mode(g.B, g.b_n, g.b_k, g.N, g.K);
  const int64_t big = int64_t((g.N + 63) / 64) * ((g.M + 63) / 64);
  if (big >= 304) {  // two 64 x 64 tiles per SM or more
    dim3 grid(unsigned((g.N + 63) / 64), unsigned((g.M + 63) / 64));
    k_gemm<2, 4><<<grid, 128, 0, s>>>(g);
  } else {
    dim3 grid(unsigned((g.N + 31) / 32), unsigned((g.M + 31) / 32));
    k_gemm<1, 2><<<grid, 128, 0, s>>>(g);
  }
}

// Forward pass of nbatch rows of actb[0] (BF16 input, padded).
void forward(ugks_mlp* n, int nbatch) {
  for (int l = 0; l < n->L; ++l) {
    GemmArgs g{};
    g.M = nbatch;
    g.N = n->dout[l];
    g.K = n->din[l];
    g.A = n->actb[l];
    g.a_m = n->din[l];
    g.a_k = 1;
    g.B = n->Wb + n->woff[l];
    g.b_k = 1;
    g.b_n = n->din[l];
    g.mode = 0;
    g.bias = n->b + n->boff[l];
    g.act = l + 1 < n->L ? 1 : 0;
    g.valid_n = n->rout[l];
    g.C = n->actf[l + 1];
    g.ldc = n->dout[l];
    g.Cb = n->actb[l + 1];
    gemm(n->stream, g);
  }
}

// Backward pass from dzf[L-1] / dzb[L-1] (set by the loss): gW, gb.
void backward(ugks_mlp* n, int nbatch) {
  for (int l = n->L - 1; l >= 0; --l) {
    GemmArgs g{};
    // dW_l = dz_l^T a_l
    g.M = n->dout[l];
    g.N = n->din[l];
    g.K = nbatch;
    g.A = n->dzb[l];
    g.a_m = 1;
    g.a_k = n->dout[l];
    g.B = n->actb[l];
    g.b_k = n->din[l];
    g.b_n = 1;
    g.mode = 2;
    g.valid_n = n->din[l];
    g.C = n->gW + n->woff[l];
    g.ldc = n->din[l];
    g.Cb = nullptr;
    gemm(n->stream, g);
    k_colsum<<<unsigned((n->dout[l] + 31) / 32), 256, 0, n->stream>>>(nbatch, n->dout[l], n->dzf[l], n->dout[l],
                                                                     n->gb + n->boff[l]);
    if (l > 0) {
      // dz_{l-1} = (dz_l W_l) (1 - a_{l}^2), a_l = tanh output of layer l-1
      GemmArgs h{};
      h.M = nbatch;
      h.N = n->din[l];
      h.K = n->dout[l];
      h.A = n->dzb[l];
      h.a_m = n->dout[l];
      h.a_k = 1;
      h.B = n->Wb + n->woff[l];
      h.b_k = n->din[l];
      h.b_n = 1;
      h.mode = 1;
      h.aprev = n->actf[l];
      h.valid_n = n->rin[l];
      h.C = n->dzf[l - 1];
      h.ldc = n->din[l];
      h.Cb = n->dzb[l - 1];
      gemm(n->stream, h);
    }
  }
}

void drop_train_graph(ugks_mlp* n) {
  if (n->train_exec) cudaGraphExecDestroy(n->train_exec);
  if (n->train_graph) cudaGraphDestroy(n->train_graph);
  n->train_exec = nullptr;
  n->train_graph = nullptr;
  n->train_batch = 0;
}

void release(ugks_mlp* n, void* p) {
  if (!p) return;
  cudaStreamSynchronize(n->stream);
  cudaFree(p);
  n->allocs.erase(std::remove(n->allocs.begin(), n->allocs.end(), p), n->allocs.end());
}

ugks_status upload_data(ugks_mlp* n, const float* X, const float* Y, int64_t count) {
  if (count > n->data_cap) {
    drop_train_graph(n);  // it holds the old data pointers
    // grow the device copy of the data set
    release(n, n->dX);
    release(n, n->dY);
    release(n, n->didx);
    n->dX = n->dY = nullptr;
    n->didx = nullptr;
    n->data_cap = 0;
    MLP_TRY(n, malloc_n(n, &n->dX, size_t(count) * n->n_in));
    MLP_TRY(n, malloc_n(n, &n->dY, size_t(count) * n->n_out));
    MLP_TRY(n, malloc_n(n, &n->didx, size_t(std::max<int64_t>(count, n->max_batch))));
    n->data_cap = count;
  }
  MLP_TRY(n, cudaMemcpyAsync(n->dX, X, size_t(count) * n->n_in * sizeof(float), cudaMemcpyHostToDevice, n->stream));
  if (Y)
    MLP_TRY(n, cudaMemcpyAsync(n->dY, Y, size_t(count) * n->n_out * sizeof(float), cudaMemcpyHostToDevice,
                               n->stream));
  return UGKS_OK;
}

void gather(ugks_mlp* n, int nb, int nvalid, const int64_t* idx, bool targets, const int64_t* cursor = nullptr) {
  const float* nm = n->norm;
  k_gather<<<unsigned(nb), 64, 0, n->stream>>>(nb, nvalid, idx, cursor, n->dX, n->n_in, n->din[0], n->dY, n->n_out, nm,
                                                nm + n->n_in, nm + 2 * n->n_in, nm + 2 * n->n_in + n->n_out,
                                                n->actb[0], targets ? n->tgt : nullptr);
}

void loss_grad(ugks_mlp* n, int nb, int nvalid) {
  const int L = n->L;
  k_mse<<<120, 256, 0, n->stream>>>(nb, nvalid, n->n_out, n->dout[L - 1], n->actf[L], n->tgt, n->dzf[L - 1],
                                     n->dzb[L - 1], n->dloss);
}

}  // namespace

extern "C" {

ugks_status ugks_mlp_create(int32_t n_in, int32_t n_out, int32_t width, int32_t hidden_layers, uint64_t seed,
                            void* cuda_stream, ugks_mlp** out) {
  if (!out) return mfail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "out must not be NULL");
  *out = nullptr;
  if (n_in < 1 || n_out < 1 || width < 1 || hidden_layers < 1 || n_in > 4096 || n_out > 4096 || width > 4096)
    return mfail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "bad network shape");
  ugks_mlp* n = new (std::nothrow) ugks_mlp();
  if (!n) return mfail(nullptr, UGKS_ERR_OUT_OF_MEMORY, "host allocation failed");
  n->n_in = n_in;
  n->n_out = n_out;
  n->width = width;
  n->hidden = hidden_layers;
  n->L = hidden_layers + 1;
  if (cuda_stream) {
    n->stream = static_cast<cudaStream_t>(cuda_stream);
  } else if (cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking) == cudaSuccess) {
    n->own_stream = true;
  } else {
    delete n;
    return mfail(nullptr, UGKS_ERR_CUDA, "stream creation failed");
  }
  for (int l = 0; l < n->L; ++l) {
    const int ri = l == 0 ? n_in : width, ro = l + 1 == n->L ? n_out : width;
    n->rin.push_back(ri);
    n->rout.push_back(ro);
    n->din.push_back(pad16(ri));
    n->dout.push_back(pad16(ro));
    n->woff.push_back(n->nW);
    n->boff.push_back(n->nb);
    n->nW += int64_t(pad16(ro)) * pad16(ri);
    n->nb += pad16(ro);
  }
  auto fail_here = [&](ugks_status st) {
    ugks_mlp_destroy(n);
    return st;
  };
#define CREATE_TRY(call)                                                                        \
  do {                                                                                          \
    if ((call) != cudaSuccess) return fail_here(mfail(nullptr, UGKS_ERR_OUT_OF_MEMORY, "%s", #call)); \
  } while (0)
  CREATE_TRY(malloc_n(n, &n->W, n->nW));
  CREATE_TRY(malloc_n(n, &n->mW, n->nW));
  CREATE_TRY(malloc_n(n, &n->vW, n->nW));
  CREATE_TRY(malloc_n(n, &n->gW, n->nW));
  CREATE_TRY(malloc_n(n, &n->Wb, n->nW));
  CREATE_TRY(malloc_n(n, &n->b, n->nb));
  CREATE_TRY(malloc_n(n, &n->mb, n->nb));
  CREATE_TRY(malloc_n(n, &n->vb, n->nb));
  CREATE_TRY(malloc_n(n, &n->gb, n->nb));
  CREATE_TRY(malloc_n(n, &n->norm, size_t(2 * n_in + 2 * n_out)));
  CREATE_TRY(malloc_n(n, &n->tgt, size_t(n->max_batch) * n_out));
  CREATE_TRY(malloc_n(n, &n->dloss, 1));
  CREATE_TRY(malloc_n(n, &n->d_step, 1));
  CREATE_TRY(malloc_n(n, &n->d_cursor, 1));
  n->actf.assign(n->L + 1, nullptr);
  n->actb.assign(n->L + 1, nullptr);
  n->dzf.assign(n->L, nullptr);
  n->dzb.assign(n->L, nullptr);
  CREATE_TRY(malloc_n(n, &n->actb[0], size_t(n->max_batch) * n->din[0]));
  for (int l = 0; l < n->L; ++l) {
    CREATE_TRY(malloc_n(n, &n->actf[l + 1], size_t(n->max_batch) * n->dout[l]));
    CREATE_TRY(malloc_n(n, &n->actb[l + 1], size_t(n->max_batch) * n->dout[l]));
    CREATE_TRY(malloc_n(n, &n->dzf[l], size_t(n->max_batch) * n->dout[l]));
    CREATE_TRY(malloc_n(n, &n->dzb[l], size_t(n->max_batch) * n->dout[l]));
  }
#undef CREATE_TRY
  // Glorot-uniform weights from a counter-based generator, zero biases
  std::vector<float> hW(n->nW, 0.f);
  uint64_t st = seed;
  for (int l = 0; l < n->L; ++l) {
    const double a = std::sqrt(6.0 / (n->rin[l] + n->rout[l]));
    for (int o = 0; o < n->rout[l]; ++o)
      for (int i = 0; i < n->rin[l]; ++i) {
        const double u = double(splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
        hW[n->woff[l] + int64_t(o) * n->din[l] + i] = float((2.0 * u - 1.0) * a);
      }
  }
  n->hnorm.assign(2 * n_in + 2 * n_out, 0.f);
  for (int j = 0; j < n_in; ++j) n->hnorm[n_in + j] = 1.f;
  for (int j = 0; j < n_out; ++j) n->hnorm[2 * n_in + n_out + j] = 1.f;
  if (cudaMemcpyAsync(n->W, hW.data(), hW.size() * sizeof(float), cudaMemcpyHostToDevice, n->stream) != cudaSuccess ||
      cudaMemcpyAsync(n->norm, n->hnorm.data(), n->hnorm.size() * sizeof(float), cudaMemcpyHostToDevice,
                      n->stream) != cudaSuccess)
    return fail_here(mfail(nullptr, UGKS_ERR_CUDA, "upload of the initial weights failed"));
  k_to_bf16<<<unsigned((n->nW + 255) / 256), 256, 0, n->stream>>>(n->nW, n->W, n->Wb);
  if (cudaStreamSynchronize(n->stream) != cudaSuccess)
    return fail_here(mfail(nullptr, UGKS_ERR_CUDA, "network set-up failed"));
  *out = n;
  return UGKS_OK;
}

ugks_status ugks_mlp_set_scaling(ugks_mlp* n, const float* in_shift, const float* in_scale, const float* out_shift,
                                 const float* out_scale) {
  if (!n || !in_shift || !in_scale || !out_shift || !out_scale)
    return mfail(n, UGKS_ERR_INVALID_ARGUMENT, "NULL argument");
  for (int j = 0; j < n->n_in; ++j)
    if (!(in_scale[j] > 0.f)) return mfail(n, UGKS_ERR_INVALID_ARGUMENT, "input scale %d must be > 0", j);
  for (int j = 0; j < n->n_out; ++j)
    if (!(out_scale[j] > 0.f)) return mfail(n, UGKS_ERR_INVALID_ARGUMENT, "output scale %d must be > 0", j);
  std::copy(in_shift, in_shift + n->n_in, n->hnorm.begin());
  std::copy(in_scale, in_scale + n->n_in, n->hnorm.begin() + n->n_in);
  std::copy(out_shift, out_shift + n->n_out, n->hnorm.begin() + 2 * n->n_in);
  std::copy(out_scale, out_scale + n->n_out, n->hnorm.begin() + 2 * n->n_in + n->n_out);
  MLP_TRY(n, cudaMemcpyAsync(n->norm, n->hnorm.data(), n->hnorm.size() * sizeof(float), cudaMemcpyHostToDevice,
                             n->stream));
  MLP_TRY(n, cudaStreamSynchronize(n->stream));
  return UGKS_OK;
}

ugks_status ugks_mlp_param_count(const ugks_mlp* n, int64_t* count) {
  if (!n || !count) return mfail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "NULL argument");
  int64_t c = 0;
  for (int l = 0; l < n->L; ++l) c += int64_t(n->rout[l]) * n->rin[l] + n->rout[l];
  *count = c;
  return UGKS_OK;
}

// Parameters (or their gradients) layer by layer: W_l [out][in], then b_l.
static ugks_status copy_params(ugks_mlp* n, const float* dW, const float* db, float* out) {
  std::vector<float> hW(n->nW), hb(n->nb);
  MLP_TRY(n, cudaMemcpyAsync(hW.data(), dW, hW.size() * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
  MLP_TRY(n, cudaMemcpyAsync(hb.data(), db, hb.size() * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
  MLP_TRY(n, cudaStreamSynchronize(n->stream));
  int64_t o = 0;
  for (int l = 0; l < n->L; ++l) {
    for (int r = 0; r < n->rout[l]; ++r)
      for (int i = 0; i < n->rin[l]; ++i) out[o++] = hW[n->woff[l] + int64_t(r) * n->din[l] + i];
    for (int r = 0; r < n->rout[l]; ++r) out[o++] = hb[n->boff[l] + r];
  }
  return UGKS_OK;
}

ugks_status ugks_mlp_get_params(ugks_mlp* n, float* params) {
  if (!n || !params) return mfail(n, UGKS_ERR_INVALID_ARGUMENT, "NULL argument");
  return copy_params(n, n->W, n->b, params);
}

ugks_status ugks_mlp_set_params(ugks_mlp* n, const float* params) {
  if (!n || !params) return mfail(n, UGKS_ERR_INVALID_ARGUMENT, "NULL argument");
  std::vector<float> hW(n->nW, 0.f), hb(n->nb, 0.f);
  int64_t o = 0;
  for (int l = 0; l < n->L; ++l) {
    for (int r = 0; r < n->rout[l]; ++r)
      for (int i = 0; i < n->rin[l]; ++i) hW[n->woff[l] + int64_t(r) * n->din[l] + i] = params[o++];
    for (int r = 0; r < n->rout[l]; ++r) hb[n->boff[l] + r] = params[o++];
  }
  MLP_TRY(n, cudaMemcpyAsync(n->W, hW.data(), hW.size() * sizeof(float), cudaMemcpyHostToDevice, n->stream));
  MLP_TRY(n, cudaMemcpyAsync(n->b, hb.data(), hb.size() * sizeof(float), cudaMemcpyHostToDevice, n->stream));
  k_to_bf16<<<unsigned((n->nW + 255) / 256), 256, 0, n->stream>>>(n->nW, n->W, n->Wb);
  MLP_TRY(n, cudaMemsetAsync(n->mW, 0, n->nW * sizeof(float), n->stream));
  MLP_TRY(n, cudaMemsetAsync(n->vW, 0, n->nW * sizeof(float), n->stream));
  MLP_TRY(n, cudaMemsetAsync(n->mb, 0, n->nb * sizeof(float), n->stream));
  MLP_TRY(n, cudaMemsetAsync(n->vb, 0, n->nb * sizeof(float), n->stream));
  MLP_TRY(n, cudaMemsetAsync(n->d_step, 0, sizeof(int), n->stream));
  MLP_TRY(n, cudaStreamSynchronize(n->stream));
  return UGKS_OK;
}

ugks_status ugks_mlp_gradients(ugks_mlp* n, const float* X, const float* Y, int64_t count, float* grads,
                               double* loss) {
  if (!n || !X || !Y || !grads) return mfail(n, UGKS_ERR_INVALID_ARGUMENT, "NULL argument");
  if (count < 1 || count > n->max_batch)
    return mfail(n, UGKS_ERR_INVALID_ARGUMENT, "1 <= n <= %d samples per gradient", n->max_batch);
  ugks_status st = upload_data(n, X, Y, count);
  if (st != UGKS_OK) return st;
  std::vector<int64_t> idx(count);
  std::iota(idx.begin(), idx.end(), 0);
  MLP_TRY(n, cudaMemcpyAsync(n->didx, idx.data(), count * sizeof(int64_t), cudaMemcpyHostToDevice, n->stream));
  const int nb = int((count + 63) / 64 * 64);
  gather(n, nb, int(count), n->didx, true);
  MLP_TRY(n, cudaMemsetAsync(n->dloss, 0, sizeof(double), n->stream));
  forward(n, nb);
  loss_grad(n, nb, int(count));
  backward(n, nb);
  MLP_TRY(n, cudaGetLastError());
  if (loss) MLP_TRY(n, cudaMemcpyAsync(loss, n->dloss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
  return copy_params(n, n->gW, n->gb, grads);
}

ugks_status ugks_mlp_train(ugks_mlp* n, const float* X, const float* Y, int64_t count, int32_t epochs,
                           int32_t batch, float lr, uint64_t seed, double* loss_out) {
  if (!n || !X || !Y) return mfail(n, UGKS_ERR_INVALID_ARGUMENT, "NULL argument");
  if (count < 1 || epochs < 0 || batch < 1 || batch > n->max_batch || !(lr > 0.f))
    return mfail(n, UGKS_ERR_INVALID_ARGUMENT, "need n >= 1, epochs >= 0, 1 <= batch <= %d, lr > 0", n->max_batch);
  ugks_status st = upload_data(n, X, Y, count);
  if (st != UGKS_OK) return st;
  // one training step: batch at *d_cursor of the shuffled order, forward,
  // loss, backward, Adam at step *d_step + 1, then both advance
  auto train_step = [&](int nvalid) {
    const int nb = (nvalid + 63) / 64 * 64;
    gather(n, nb, nvalid, n->didx, true, n->d_cursor);
    forward(n, nb);
    loss_grad(n, nb, nvalid);
    backward(n, nb);
    k_adam<<<unsigned((n->nW + 255) / 256), 256, 0, n->stream>>>(n->nW, n->W, n->gW, n->mW, n->vW, n->Wb, lr,
                                                                 n->d_step);
    k_adam<<<unsigned((n->nb + 255) / 256), 256, 0, n->stream>>>(n->nb, n->b, n->gb, n->mb, n->vb, nullptr, lr,
                                                                 n->d_step);
    k_train_advance<<<1, 32, 0, n->stream>>>(n->d_cursor, nvalid, n->d_step);
  };
  // full batches replay one captured CUDA graph of the step (~30 launches)
  if (n->train_exec && (n->train_batch != batch || n->train_lr != lr)) drop_train_graph(n);
  if (!n->train_exec && count >= batch) {
    MLP_TRY(n, cudaStreamBeginCapture(n->stream, cudaStreamCaptureModeThreadLocal));
    train_step(batch);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(n->stream, &g);
    if (ce != cudaSuccess) return mfail(n, UGKS_ERR_CUDA, "training graph capture: %s", cudaGetErrorString(ce));
    n->train_graph = g;
    MLP_TRY(n, cudaGraphInstantiate(&n->train_exec, g, 0));
    n->train_batch = batch;
    n->train_lr = lr;
  }
  std::vector<int64_t> perm(count);
  uint64_t rs = seed;
  double last = 0.0;
  for (int ep = 0; ep < epochs; ++ep) {
    std::iota(perm.begin(), perm.end(), 0);
    for (int64_t i = count - 1; i > 0; --i) std::swap(perm[i], perm[int64_t(splitmix(rs) % uint64_t(i + 1))]);
    MLP_TRY(n, cudaMemcpyAsync(n->didx, perm.data(), count * sizeof(int64_t), cudaMemcpyHostToDevice, n->stream));
    MLP_TRY(n, cudaMemsetAsync(n->dloss, 0, sizeof(double), n->stream));
    MLP_TRY(n, cudaMemsetAsync(n->d_cursor, 0, sizeof(int64_t), n->stream));
    int64_t nbatches = 0;
    for (int64_t s0 = 0; s0 < count; s0 += batch, ++nbatches) {
      const int nvalid = int(std::min<int64_t>(batch, count - s0));
      if (nvalid == batch)
        MLP_TRY(n, cudaGraphLaunch(n->train_exec, n->stream));
      else
        train_step(nvalid);
    }
    MLP_TRY(n, cudaGetLastError());
    double acc = 0.0;
    MLP_TRY(n, cudaMemcpyAsync(&acc, n->dloss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    MLP_TRY(n, cudaStreamSynchronize(n->stream));  // perm is rewritten next epoch
    last = acc / double(nbatches);  // mean over the epoch's batches
    if (!std::isfinite(last)) return mfail(n, UGKS_ERR_NONFINITE, "training diverged at epoch %d", ep);
  }
  if (loss_out) *loss_out = last;
  return UGKS_OK;
}

ugks_status ugks_mlp_predict(ugks_mlp* n, const float* X, int64_t count, float* Y) {
  if (!n || !X || !Y) return mfail(n, UGKS_ERR_INVALID_ARGUMENT, "NULL argument");
  if (count < 1) return mfail(n, UGKS_ERR_INVALID_ARGUMENT, "n must be >= 1");
  ugks_status st = upload_data(n, X, nullptr, count);
  if (st != UGKS_OK) return st;
  std::vector<int64_t> idx(count);
  std::iota(idx.begin(), idx.end(), 0);
  MLP_TRY(n, cudaMemcpyAsync(n->didx, idx.data(), count * sizeof(int64_t), cudaMemcpyHostToDevice, n->stream));
  float* dout = nullptr;
  MLP_TRY(n, cudaMalloc(&dout, size_t(n->max_batch) * n->n_out * sizeof(float)));
  cudaError_t e = cudaSuccess;
  for (int64_t s0 = 0; s0 < count && e == cudaSuccess; s0 += n->max_batch) {
    const int nvalid = int(std::min<int64_t>(n->max_batch, count - s0));
    const int nb = (nvalid + 63) / 64 * 64;
    gather(n, nb, nvalid, n->didx + s0, false);
    forward(n, nb);
    const float* nm = n->norm + 2 * n->n_in;
    k_denorm<<<unsigned((nvalid * n->n_out + 255) / 256), 256, 0, n->stream>>>(nvalid, n->n_out, n->dout[n->L - 1],
                                                                              n->actf[n->L], nm, nm + n->n_out, dout);
    e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(Y + s0 * n->n_out, dout, size_t(nvalid) * n->n_out * sizeof(float), cudaMemcpyDeviceToHost,
                          n->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  cudaFree(dout);
  if (e != cudaSuccess) return mfail(n, UGKS_ERR_CUDA, "ugks_mlp_predict: %s", cudaGetErrorString(e));
  return UGKS_OK;
}

ugks_status ugks_mlp_get_scaling(const ugks_mlp* n, float* in_shift, float* in_scale, float* out_shift,
                                 float* out_scale) {
  if (!n || !in_shift || !in_scale || !out_shift || !out_scale)
    return mfail(nullptr, UGKS_ERR_INVALID_ARGUMENT, "NULL argument");
  const float* h = n->hnorm.data();
  std::copy(h, h + n->n_in, in_shift);
  std::copy(h + n->n_in, h + 2 * n->n_in, in_scale);
  std::copy(h + 2 * n->n_in, h + 2 * n->n_in + n->n_out, out_shift);
  std::copy(h + 2 * n->n_in + n->n_out, h + 2 * n->n_in + 2 * n->n_out, out_scale);
  return UGKS_OK;
}

ugks_status ugks_mlp_fit_scaling(ugks_mlp* n, const float* X, const float* Y, int64_t count) {
  if (!n || !X || !Y || count < 1) return mfail(n, UGKS_ERR_INVALID_ARGUMENT, "bad arguments");
  auto stats = [count](const float* A, int cols, std::vector<float>& shift, std::vector<float>& scale) {
    shift.assign(cols, 0.f);
    scale.assign(cols, 1.f);
    for (int j = 0; j < cols; ++j) {
      double s = 0.0, mx = 0.0;
      for (int64_t i = 0; i < count; ++i) s += A[i * cols + j];
      const double mean = s / double(count);
      double v = 0.0;
      for (int64_t i = 0; i < count; ++i) {
        const double t = A[i * cols + j] - mean;
        v += t * t;
        mx = std::max(mx, std::fabs(double(A[i * cols + j])));
      }
      const double sd = std::sqrt(v / double(count));
      shift[j] = float(mean);
      scale[j] = float(sd > 1e-6 * mx && sd > 0.0 ? sd : 1.0);
    }
  };
  std::vector<float> is, ic, os, oc;
  stats(X, n->n_in, is, ic);
  stats(Y, n->n_out, os, oc);
  return ugks_mlp_set_scaling(n, is.data(), ic.data(), os.data(), oc.data());
}

ugks_status ugks_mlp_features(ugks_mlp* n, const ugks_mesh* mesh, double mach, double kn, float* out) {
  if (!n || !mesh || !out) return mfail(n, UGKS_ERR_INVALID_ARGUMENT, "NULL argument");
  if (mesh->dim < 1 || mesh->dim > 3 || mesh->n_cells < 1 || !mesh->cell_centroid ||
      (mesh->n_faces > 0 && (!mesh->face_neighbor || !mesh->face_centroid)) || !(kn > 0.0))
    return mfail(n, UGKS_ERR_INVALID_ARGUMENT, "bad mesh or kn <= 0");
  const int D = mesh->dim;
  const int64_t Nc = mesh->n_cells;
  std::vector<double> xw;
  for (int64_t f = 0; f < mesh->n_faces; ++f) {
    const int64_t nb = mesh->face_neighbor[f];
    if (nb >= 0) continue;
    const int64_t b = -nb - 1;
    if (b >= mesh->n_bc || !mesh->bc) return mfail(n, UGKS_ERR_MESH, "face %lld: no boundary condition", (long long)f);
    if (mesh->bc[b].type == UGKS_BC_WALL)
      for (int k = 0; k < D; ++k) xw.push_back(mesh->face_centroid[f * D + k]);
  }
  const int64_t nw = int64_t(xw.size()) / D;
  double *dxc = nullptr, *dxw = nullptr, *dd = nullptr;
  cudaError_t e = cudaMalloc(&dxc, size_t(Nc) * D * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&dxw, std::max<size_t>(xw.size(), 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&dd, size_t(Nc) * sizeof(double));
  std::vector<double> d(Nc);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dxc, mesh->cell_centroid, size_t(Nc) * D * sizeof(double), cudaMemcpyHostToDevice, n->stream);
  if (e == cudaSuccess && nw > 0)
    e = cudaMemcpyAsync(dxw, xw.data(), xw.size() * sizeof(double), cudaMemcpyHostToDevice, n->stream);
  if (e == cudaSuccess) {
    k_wall_distance<<<unsigned((Nc + 127) / 128), 128, 0, n->stream>>>(Nc, D, dxc, nw, dxw, dd);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(d.data(), dd, size_t(Nc) * sizeof(double), cudaMemcpyDeviceToHost, n->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  cudaFree(dxc);
  cudaFree(dxw);
  cudaFree(dd);
  if (e != cudaSuccess) return mfail(n, UGKS_ERR_CUDA, "ugks_mlp_features: %s", cudaGetErrorString(e));
  for (int64_t i = 0; i < Nc; ++i) {
    float* o = out + i * 6;
    o[0] = float(mach);
    o[1] = float(std::log10(kn));
    for (int k = 0; k < 3; ++k) o[2 + k] = k < D ? float(mesh->cell_centroid[i * D + k]) : 0.f;
    o[5] = float(d[i]);
  }
  return UGKS_OK;
}

ugks_status ugks_mlp_warm_start(ugks_mlp* n, ugks_ctx* ctx, const ugks_mesh* mesh, double mach, double kn,
                                const double* freestream, int64_t* n_fallback) {
  if (!n || !ctx || !mesh || !freestream) return mfail(n, UGKS_ERR_INVALID_ARGUMENT, "NULL argument");
  int32_t D = 0;
  int64_t Nc = 0;
  ugks_status st = ugks_mesh_sizes(ctx, &D, &Nc, nullptr);
  if (st != UGKS_OK) return mfail(n, st, "%s", ugks_last_error(ctx));
  const int n13 = 2 * D + 2 + D * (D + 1) / 2;
  if (mesh->dim != D || mesh->n_cells != Nc) return mfail(n, UGKS_ERR_INVALID_ARGUMENT, "mesh does not match the context");
  if (n->n_in != 6 || n->n_out != n13)
    return mfail(n, UGKS_ERR_INVALID_ARGUMENT, "network shape (%d -> %d) is not (6 -> %d)", n->n_in, n->n_out, n13);
  if (!(freestream[0] > 0.0) || !(freestream[D + 1] > 0.0))
    return mfail(n, UGKS_ERR_INVALID_ARGUMENT, "freestream rho and T must be > 0");
  std::vector<float> X(size_t(Nc) * 6), Y(size_t(Nc) * n13);
  st = ugks_mlp_features(n, mesh, mach, kn, X.data());
  if (st != UGKS_OK) return st;
  st = ugks_mlp_predict(n, X.data(), Nc, Y.data());
  if (st != UGKS_OK) return st;
  std::vector<double> fields(size_t(Nc) * n13);
  int64_t nf = 0;
  for (int64_t i = 0; i < Nc; ++i) {
    const float* y = Y.data() + i * n13;
    bool ok = y[0] > 0.f && y[D + 1] > 0.f;
    for (int j = 0; j < n13; ++j) ok = ok && std::isfinite(y[j]);
    double* o = fields.data() + i * n13;
    if (ok) {
      for (int j = 0; j < n13; ++j) o[j] = y[j];
      // bounded non-equilibrium: stress and heat flux scaled by one factor so
      // that |sigma_ij| <= p/2 and |q| <= p sqrt(T)/2 (p = rho T / 2), where the
      // Grad correction stays above -1/2 at thermal speeds and f stays positive
      const double p = 0.5 * o[0] * o[D + 1];
      double smax = 0.0, q2 = 0.0;
      for (int j = D + 2; j < D + 2 + D * (D + 1) / 2; ++j) smax = std::max(smax, std::fabs(o[j]));
      for (int j = D + 2 + D * (D + 1) / 2; j < n13; ++j) q2 += o[j] * o[j];
      double alpha = 1.0;
      if (smax > 0.5 * p) alpha = std::min(alpha, 0.5 * p / smax);
      const double qb = 0.5 * p * std::sqrt(o[D + 1]);
      if (q2 > qb * qb) alpha = std::min(alpha, qb / std::sqrt(q2));
      for (int j = D + 2; j < n13; ++j) o[j] *= alpha;
    } else {
      ++nf;
      for (int j = 0; j < n13; ++j) o[j] = j < D + 2 ? freestream[j] : 0.0;
    }
  }
  st = ugks_init_moments13(ctx, fields.data());
  if (st != UGKS_OK) return mfail(n, st, "%s", ugks_last_error(ctx));
  if (n_fallback) *n_fallback = nf;
  return UGKS_OK;
}

ugks_status ugks_mlp_destroy(ugks_mlp* n) {
  if (!n) return UGKS_OK;
  if (n->stream) cudaStreamSynchronize(n->stream);
  drop_train_graph(n);
  for (void* p : n->allocs) cudaFree(p);
  if (n->own_stream && n->stream) cudaStreamDestroy(n->stream);
  delete n;
  return UGKS_OK;
}

const char* ugks_mlp_last_error(const ugks_mlp* n) { return n ? n->err.c_str() : g_mlp_err.c_str(); }

}  // extern "C"
