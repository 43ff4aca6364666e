// Learned surrogate of the lookup table for graded lattices (strut width w per tile).
//
// Factorisation: T(w) ~ U V(w)^T with U (n_nz x r, orthonormal columns, shared) and V(w)
// (9 n_pi x r) predicted by a small MLP, so that a tile block is K_t = U (V(w_t)^T A_t):
// the eq. 58 product becomes Z_t = V(w_t)^T A_t (r x 9 per tile) and one product with K = r.
//
// U is the dominant left singular subspace of the training tables applied to coefficient
// blocks of the workload, [T(w_k) A_s], found by a randomized range finder with power
// iterations (Halko, Martinsson & Tropp 2011); the MLP targets are V_k = T(w_k)^T U, the
// best factor for that U.  The MLP is 1 -> H -> H -> n_out, tanh hidden layers, FP16
// weights (FP32 master copy for Adam), FP32 accumulation; all its kernels are below.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <memory>
#include <random>
#include <vector>

#include "common.h"
#include "store.h"

namespace msasm {

template <typename T>
msasm_status gemm_simt(const T* A, int64_t lda, const T* B, int64_t ldb, int64_t N, int M, int K, T* C, int64_t ldc,
                       cudaStream_t stream);
int tc_kpad(int K, int kind);
size_t tc_slice_bytes(int64_t rows, int K, int kind);
msasm_status tc_split_f32_gpu(const float* x, int64_t rows, int K, int kind, void* hi, void* lo, float* row_scale,
                              cudaStream_t s);
msasm_status contract_tc_gpu(int kind, const void* a_hi, const void* a_lo, const float* a_scale, int M,
                             const void* b_hi, const void* b_lo, const float* b_scale, int64_t N, int K, float* out,
                             int ld, bool blocks, unsigned* d_err, cudaStream_t s);
constexpr int kLowRankSplit = 0;   // split FP16 (hi + 2^-11 lo, three products): about 6e-7 relative
template <typename T>
msasm_status transpose_table_gpu(const double* d_T, int n_nz, int K, T* d_Tt, cudaStream_t s);
bool cholesky_upper_inverse(const std::vector<double>& A, int n, std::vector<double>& Rinv);
void symmetric_eigen(std::vector<double> A, int n, std::vector<double>& w, std::vector<double>& V);
msasm_status pullback_gpu(const msasm_plan* plan, const double* d_ctrl, double lam, double mu, int64_t t0,
                          int64_t n_tiles, double* d_coef, cudaStream_t stream);
template <typename T>
msasm_status scatter_pass_gpu(const msasm_plan* plan, const T* d_nz, int ld_nz, int64_t t0, int64_t n_tiles,
                              T* d_values, cudaStream_t stream);

// ------------------------------------------------------------------ MLP layout
// params (FP32 master and FP16 copy): W1[H], b1[H], W2[H][H], b2[H], W3[n_out][H], b3[n_out]
struct MlpLayout {
  int H, n_out;
  size_t W1, b1, W2, b2, W3, b3, total;
  MlpLayout(int h, int n) : H(h), n_out(n) {
    W1 = 0;
    b1 = W1 + H;
    W2 = b1 + H;
    b2 = W2 + size_t(H) * H;
    W3 = b2 + H;
    b3 = W3 + size_t(n_out) * H;
    total = b3 + n_out;
  }
};

__global__ void mlp_hidden_kernel(const __half* __restrict__ p, const float* __restrict__ x, int B, int H, size_t oW1,
                                  size_t ob1, size_t oW2, size_t ob2, float* __restrict__ h1, float* __restrict__ h2) {
  extern __shared__ float sh[];
  for (int b = blockIdx.x; b < B; b += gridDim.x) {
    for (int j = threadIdx.x; j < H; j += blockDim.x) {
      const float v = tanhf(fmaf(__half2float(p[oW1 + j]), x[b], __half2float(p[ob1 + j])));
      sh[j] = v;
      h1[size_t(b) * H + j] = v;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < H; j += blockDim.x) {
      float s = __half2float(p[ob2 + j]);
      for (int i = 0; i < H; ++i) s = fmaf(__half2float(p[oW2 + size_t(j) * H + i]), sh[i], s);
      h2[size_t(b) * H + j] = tanhf(s);
    }
    __syncthreads();
  }
}

__global__ void widen_half_kernel(const __half* __restrict__ x, int64_t n, float* __restrict__ y) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = __half2float(x[i]);
}

__global__ void add_bias_kernel(float* __restrict__ y, int64_t n, int n_out, const __half* __restrict__ b) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] += __half2float(b[i % n_out]);
}

// dy = 2 (y - t) / (B n_out) and the mean squared error (block partial sums into loss)
__global__ void mlp_loss_kernel(const float* __restrict__ y, const float* __restrict__ t, int64_t n, float inv,
                                float* __restrict__ dy, float* __restrict__ loss) {
  float acc = 0.0f;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float d = y[i] - t[i];
    dy[i] = 2.0f * d * inv;
    acc = fmaf(d * d, inv, acc);
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

// gradient of the output layer: dW3[o][i] = sum_b dy[b][o] h2[b][i], db3[o] = sum_b dy[b][o]
__global__ void mlp_grad_out_kernel(const float* __restrict__ dy, const float* __restrict__ h2, int B, int H, int n_out,
                                    float* __restrict__ gW3, float* __restrict__ gb3) {
  const int64_t total = int64_t(n_out) * (H + 1);
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int o = int(idx / (H + 1)), i = int(idx % (H + 1));
    float s = 0.0f;
    if (i < H)
      for (int b = 0; b < B; ++b) s = fmaf(dy[size_t(b) * n_out + o], h2[size_t(b) * H + i], s);
    else
      for (int b = 0; b < B; ++b) s += dy[size_t(b) * n_out + o];
    if (i < H) gW3[size_t(o) * H + i] = s; else gb3[o] = s;
  }
}

// back through the output layer and the hidden layers, one block per sample:
// dz2 = (W3^T dy) (1 - h2^2), dz1 = (W2^T dz2) (1 - h1^2)
__global__ void mlp_back_hidden_kernel(const __half* __restrict__ p, const float* __restrict__ dy,
                                       const float* __restrict__ h1, const float* __restrict__ h2, int B, int H,
                                       int n_out, size_t oW2, size_t oW3, float* __restrict__ dz1,
                                       float* __restrict__ dz2) {
  extern __shared__ float sh[];
  const int b = blockIdx.x;
  const float* dyb = dy + size_t(b) * n_out;
  for (int i = threadIdx.x; i < H; i += blockDim.x) {
    float s = 0.0f;
    for (int o = 0; o < n_out; ++o) s = fmaf(dyb[o], __half2float(p[oW3 + size_t(o) * H + i]), s);
    const float hv = h2[size_t(b) * H + i];
    const float d = s * (1.0f - hv * hv);
    sh[i] = d;
    dz2[size_t(b) * H + i] = d;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < H; i += blockDim.x) {
    float s = 0.0f;
    for (int j = 0; j < H; ++j) s = fmaf(sh[j], __half2float(p[oW2 + size_t(j) * H + i]), s);
    const float hv = h1[size_t(b) * H + i];
    dz1[size_t(b) * H + i] = s * (1.0f - hv * hv);
  }
}

// dW2[j][i] = sum_b dz2[b][j] h1[b][i]; db2 = sum dz2; dW1[j] = sum_b dz1[b][j] x[b]; db1 = sum dz1
__global__ void mlp_grad_hidden_kernel(const float* __restrict__ dz1, const float* __restrict__ dz2,
                                       const float* __restrict__ h1, const float* __restrict__ x, int B, int H,
                                       float* __restrict__ g, size_t oW1, size_t ob1, size_t oW2, size_t ob2) {
  const int64_t total = int64_t(H) * H + 3 * H;
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += int64_t(gridDim.x) * blockDim.x) {
    float s = 0.0f;
    if (idx < int64_t(H) * H) {
      const int j = int(idx / H), i = int(idx % H);
      for (int b = 0; b < B; ++b) s = fmaf(dz2[size_t(b) * H + j], h1[size_t(b) * H + i], s);
      g[oW2 + idx] = s;
    } else {
      const int r = int(idx - int64_t(H) * H), j = r % H, which = r / H;
      for (int b = 0; b < B; ++b) {
        if (which == 0) s += dz2[size_t(b) * H + j];
        else if (which == 1) s = fmaf(dz1[size_t(b) * H + j], x[b], s);
        else s += dz1[size_t(b) * H + j];
      }
      g[(which == 0 ? ob2 : which == 1 ? oW1 : ob1) + j] = s;
    }
  }
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, __half* __restrict__ w16, size_t n, float lr,
                            const int* __restrict__ step) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const int t = *step + 1;
  const float c1 = 1.0f - powf(b1, float(t)), c2 = 1.0f - powf(b2, float(t));
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    w16[i] = __float2half_rn(wi);
  }
}

__global__ void step_kernel(int* step) { *step += 1; }

__global__ void to_half_kernel(const float* __restrict__ w, size_t n, __half* __restrict__ w16) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    w16[i] = __float2half_rn(w[i]);
}

// ------------------------------------------------------------------ surrogate helpers
// Qt[r][i] = sum_l S[r][l] Y[l][i]   (S small, r x l row-major, on the device)
__global__ void small_left_kernel(const double* __restrict__ S, int R, int L, const double* __restrict__ Y, int64_t n,
                                  double* __restrict__ Q) {
  const int64_t total = int64_t(R) * n;
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int r = int(idx / n);
    const int64_t i = idx % n;
    double s = 0.0;
    for (int l = 0; l < L; ++l) s = fma(S[r * L + l], Y[l * n + i], s);
    Q[idx] = s;
  }
}

// targets: y[k][o] = (Vt_k[o] - mean[o]) / scale, with mean over the k samples
__global__ void normalise_targets_kernel(float* __restrict__ y, const double* __restrict__ v, int K, int n_out,
                                         float* __restrict__ mean, double inv_scale) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n_out; o += gridDim.x * blockDim.x) {
    double mu = 0.0;
    for (int k = 0; k < K; ++k) mu += v[size_t(k) * n_out + o];
    mu /= K;
    mean[o] = float(mu);
    for (int k = 0; k < K; ++k) y[size_t(k) * n_out + o] = float((v[size_t(k) * n_out + o] - mu) * inv_scale);
  }
}

// V = mean + scale * y, in place on y
__global__ void denormalise_kernel(float* __restrict__ y, int64_t B, int n_out, const float* __restrict__ mean,
                                   float scale) {
  const int64_t total = B * n_out;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = fmaf(y[i], scale, mean[i % n_out]);
}

__global__ void normalise_inputs_kernel(const double* __restrict__ w, int64_t n, double w0, double ws,
                                        float* __restrict__ x) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i] = float((w[i] - w0) / ws);
}

// Z[9t + ab][r] = sum_k Vt_t[r][k] coef[9t + ab][k]  (FP32 result; V FP32, coefficients FP64)
// Z[9t + ab][r] = sum_k Vt_t[r][k] coef[9t + ab][k]: one CTA per tile, the tile's 9 coefficient rows
// in shared memory (FP32), one warp per r at a time with the lanes splitting k (coalesced rows of Vt)
__global__ void lowrank_z_kernel(const float* __restrict__ Vt, const double* __restrict__ coef, int64_t n_tiles,
                                 int rank, int K, float* __restrict__ Z) {
  extern __shared__ float cs[];                 // [9][K]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    for (int i = threadIdx.x; i < 9 * K; i += blockDim.x) cs[i] = float(coef[9 * t * K + i]);
    __syncthreads();
    for (int r = warp; r < rank; r += warps) {
      const float* v = Vt + (t * rank + r) * K;
      float acc[9];
#pragma unroll
      for (int ab = 0; ab < 9; ++ab) acc[ab] = 0.0f;
      for (int k = lane; k < K; k += 32) {
        const float vk = v[k];
#pragma unroll
        for (int ab = 0; ab < 9; ++ab) acc[ab] = fmaf(vk, cs[ab * K + k], acc[ab]);
      }
#pragma unroll
      for (int ab = 0; ab < 9; ++ab) {
        float x = acc[ab];
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) Z[(9 * t + ab) * rank + r] = x;
      }
    }
    __syncthreads();
  }
}

}  // namespace msasm

using namespace msasm;

struct msasm_mlp {
  MlpLayout lay;
  float* d_w = nullptr;      // FP32 master
  __half* d_w16 = nullptr;   // FP16 compute copy
  float* d_w3f = nullptr;    // the output layer's FP16 weights widened to FP32 (exact) for the GEMM
  // tensor-core output layer (inference): split-FP16 slices of W3 (exact: W3 is FP16) made once per
  // set of weights, and of the batch's last hidden layer
  void *d_w3hi = nullptr, *d_w3lo = nullptr, *d_ahi = nullptr, *d_alo = nullptr;
  float *d_w3scale = nullptr, *d_ascale = nullptr;
  unsigned* d_tc_err = nullptr;
  bool w3_split_ok = false;
  int act_cap = 0;
  float* d_g = nullptr;
  float* d_m = nullptr;
  float* d_v = nullptr;
  int* d_step = nullptr;
  float* d_loss = nullptr;
  // batch work buffers (capacity)
  int cap = 0;
  float *d_h1 = nullptr, *d_h2 = nullptr, *d_y = nullptr, *d_dy = nullptr, *d_dz1 = nullptr, *d_dz2 = nullptr;
  cudaGraphExec_t graph = nullptr;
  const float* graph_x = nullptr;
  const float* graph_t = nullptr;
  int graph_B = 0;
  float graph_lr = 0.0f;
  msasm_mlp(int H, int n_out) : lay(H, n_out) {}
  ~msasm_mlp() {
    if (graph) cudaGraphExecDestroy(graph);
    cudaFree(d_w);
    cudaFree(d_w16);
    cudaFree(d_w3f);
    cudaFree(d_w3hi);
    cudaFree(d_w3lo);
    cudaFree(d_w3scale);
    cudaFree(d_ahi);
    cudaFree(d_alo);
    cudaFree(d_ascale);
    cudaFree(d_tc_err);
    cudaFree(d_g);
    cudaFree(d_m);
    cudaFree(d_v);
    cudaFree(d_step);
    cudaFree(d_loss);
    cudaFree(d_h1);
    cudaFree(d_h2);
    cudaFree(d_y);
    cudaFree(d_dy);
    cudaFree(d_dz1);
    cudaFree(d_dz2);
  }
};

struct msasm_surrogate {
  int rank = 0, K = 0, n_nz = 0, n_train = 0;
  int qd[3] = {0, 0, 0};           // the tables' projection degrees
  double w0 = 0.275, ws = 0.125;   // input normalisation of the width
  float scale = 1.0f;              // target scale
  float* d_U = nullptr;            // n_nz x rank (FP32), row-major
  void* d_Uhi = nullptr;           // split-FP16 slices of U for the tensor-core low-rank product
  void* d_Ulo = nullptr;
  float* d_Uscale = nullptr;
  unsigned* d_err = nullptr;
  float* d_mean = nullptr;         // n_out
  float* d_x = nullptr;            // normalised training widths
  float* d_targets = nullptr;      // n_train x n_out (normalised)
  msasm_mlp* mlp = nullptr;
  ~msasm_surrogate() {
    delete mlp;
    cudaFree(d_U);
    cudaFree(d_Uhi);
    cudaFree(d_Ulo);
    cudaFree(d_Uscale);
    cudaFree(d_err);
    cudaFree(d_mean);
    cudaFree(d_x);
    cudaFree(d_targets);
  }
};

namespace msasm {

static msasm_status mlp_ensure_batch(msasm_mlp* n, int B) {
  if (n->cap >= B) return MSASM_OK;
  const int H = n->lay.H, O = n->lay.n_out;
  if (n->graph) {                      // the captured training step refers to the old buffers
    MSASM_CUDA(cudaDeviceSynchronize());
    cudaGraphExecDestroy(n->graph);
    n->graph = nullptr;
  }
  cudaFree(n->d_h1);
  cudaFree(n->d_h2);
  cudaFree(n->d_y);
  cudaFree(n->d_dy);
  cudaFree(n->d_dz1);
  cudaFree(n->d_dz2);
  MSASM_CUDA(cudaMalloc(&n->d_h1, size_t(B) * H * 4));
  MSASM_CUDA(cudaMalloc(&n->d_h2, size_t(B) * H * 4));
  MSASM_CUDA(cudaMalloc(&n->d_y, size_t(B) * O * 4));
  MSASM_CUDA(cudaMalloc(&n->d_dy, size_t(B) * O * 4));
  MSASM_CUDA(cudaMalloc(&n->d_dz1, size_t(B) * H * 4));
  MSASM_CUDA(cudaMalloc(&n->d_dz2, size_t(B) * H * 4));
  n->cap = B;
  return MSASM_OK;
}

static msasm_status mlp_forward(msasm_mlp* n, const float* d_x, int B, float* d_y, cudaStream_t s) {
  const MlpLayout& L = n->lay;
  mlp_hidden_kernel<<<std::min(B, 1024), 128, L.H * sizeof(float), s>>>(n->d_w16, d_x, B, L.H, L.W1, L.b1, L.W2, L.b2,
                                                                        n->d_h1, n->d_h2);
  MSASM_CUDA(cudaGetLastError());
  // output layer as one CUDA-core GEMM over the batch: y = h2 W3^T + b3
  const int64_t nw3 = int64_t(L.n_out) * L.H;
  widen_half_kernel<<<unsigned(std::min<int64_t>((nw3 + 255) / 256, 152 * 8)), 256, 0, s>>>(n->d_w16 + L.W3, nw3,
                                                                                             n->d_w3f);
  MSASM_CUDA(cudaGetLastError());
  MSASM_TRY(gemm_simt<float>(n->d_h2, L.H, n->d_w3f, L.H, B, L.n_out, L.H, d_y, L.n_out, s));
  const int64_t ny = int64_t(B) * L.n_out;
  add_bias_kernel<<<unsigned(std::min<int64_t>((ny + 255) / 256, 152 * 8)), 256, 0, s>>>(d_y, ny, L.n_out,
                                                                                         n->d_w16 + L.b3);
  MSASM_CUDA(cudaGetLastError());
  return MSASM_OK;
}

// The same forward pass with the output layer y = h2 W3^T + b3 on the tensor cores: split FP16
// (h2 = hi + 2^-11 lo per row-scaled slice, three products, FP32 accumulation; W3 is FP16, so its
// slices are exact), about 1e-7 relative to the CUDA-core product.
static msasm_status mlp_forward_tc(msasm_mlp* n, const float* d_x, int B, float* d_y, cudaStream_t s) {
  const MlpLayout& L = n->lay;
  constexpr int kind = kLowRankSplit;
  mlp_hidden_kernel<<<std::min(B, 1024), 128, L.H * sizeof(float), s>>>(n->d_w16, d_x, B, L.H, L.W1, L.b1, L.W2, L.b2,
                                                                        n->d_h1, n->d_h2);
  MSASM_CUDA(cudaGetLastError());
  if (!n->w3_split_ok) {
    const int64_t nw3 = int64_t(L.n_out) * L.H;
    widen_half_kernel<<<unsigned(std::min<int64_t>((nw3 + 255) / 256, 152 * 8)), 256, 0, s>>>(n->d_w16 + L.W3, nw3,
                                                                                               n->d_w3f);
    MSASM_CUDA(cudaGetLastError());
    if (!n->d_w3hi) {
      const size_t wb = tc_slice_bytes(L.n_out, L.H, kind);
      MSASM_CUDA(cudaMalloc(&n->d_w3hi, wb));
      MSASM_CUDA(cudaMalloc(&n->d_w3lo, wb));
      MSASM_CUDA(cudaMalloc(&n->d_w3scale, size_t(L.n_out) * 4));
      MSASM_CUDA(cudaMalloc(&n->d_tc_err, sizeof(unsigned)));
      MSASM_CUDA(cudaMemsetAsync(n->d_tc_err, 0, sizeof(unsigned), s));
    }
    MSASM_TRY(tc_split_f32_gpu(n->d_w3f, L.n_out, L.H, kind, n->d_w3hi, n->d_w3lo, n->d_w3scale, s));
    n->w3_split_ok = true;
  }
  if (n->act_cap < B) {
    cudaFree(n->d_ahi);
    cudaFree(n->d_alo);
    cudaFree(n->d_ascale);
    n->d_ahi = n->d_alo = nullptr;
    n->d_ascale = nullptr;
    n->act_cap = 0;
    const size_t ab = tc_slice_bytes(B, L.H, kind);
    MSASM_CUDA(cudaMalloc(&n->d_ahi, ab));
    MSASM_CUDA(cudaMalloc(&n->d_alo, ab));
    MSASM_CUDA(cudaMalloc(&n->d_ascale, size_t(B) * 4));
    n->act_cap = B;
  }
  MSASM_TRY(tc_split_f32_gpu(n->d_h2, B, L.H, kind, n->d_ahi, n->d_alo, n->d_ascale, s));
  MSASM_TRY(contract_tc_gpu(kind, n->d_w3hi, n->d_w3lo, n->d_w3scale, L.n_out, n->d_ahi, n->d_alo, n->d_ascale, B,
                            L.H, d_y, L.n_out, false, n->d_tc_err, s));
  const int64_t ny = int64_t(B) * L.n_out;
  add_bias_kernel<<<unsigned(std::min<int64_t>((ny + 255) / 256, 152 * 8)), 256, 0, s>>>(d_y, ny, L.n_out,
                                                                                         n->d_w16 + L.b3);
  MSASM_CUDA(cudaGetLastError());
  return MSASM_OK;
}

// loss (into n->d_loss, accumulated) and the full gradient (into n->d_g) for targets d_t
static msasm_status mlp_loss_grad(msasm_mlp* n, const float* d_x, const float* d_t, int B, cudaStream_t s) {
  const MlpLayout& L = n->lay;
  MSASM_TRY(mlp_forward(n, d_x, B, n->d_y, s));
  const int64_t ny = int64_t(B) * L.n_out;
  mlp_loss_kernel<<<152 * 4, 256, 0, s>>>(n->d_y, d_t, ny, 1.0f / float(ny), n->d_dy, n->d_loss);
  MSASM_CUDA(cudaGetLastError());
  mlp_grad_out_kernel<<<152 * 8, 256, 0, s>>>(n->d_dy, n->d_h2, B, L.H, L.n_out, n->d_g + L.W3, n->d_g + L.b3);
  MSASM_CUDA(cudaGetLastError());
  mlp_back_hidden_kernel<<<B, 128, L.H * sizeof(float), s>>>(n->d_w16, n->d_dy, n->d_h1, n->d_h2, B, L.H, L.n_out,
                                                             L.W2, L.W3, n->d_dz1, n->d_dz2);
  MSASM_CUDA(cudaGetLastError());
  mlp_grad_hidden_kernel<<<152, 256, 0, s>>>(n->d_dz1, n->d_dz2, n->d_h1, d_x, B, L.H, n->d_g, L.W1, L.b1, L.W2, L.b2);
  MSASM_CUDA(cudaGetLastError());
  return MSASM_OK;
}

static msasm_status mlp_train_step(msasm_mlp* n, const float* d_x, const float* d_t, int B, float lr, cudaStream_t s) {
  n->w3_split_ok = false;                        // the weights change
  MSASM_TRY(mlp_loss_grad(n, d_x, d_t, B, s));
  adam_kernel<<<152 * 4, 256, 0, s>>>(n->d_w, n->d_g, n->d_m, n->d_v, n->d_w16, n->lay.total, lr, n->d_step);
  MSASM_CUDA(cudaGetLastError());
  step_kernel<<<1, 1, 0, s>>>(n->d_step);
  MSASM_CUDA(cudaGetLastError());
  return MSASM_OK;
}

}  // namespace msasm

extern "C" {

msasm_status msasm_mlp_create(int32_t n_out, int32_t hidden, uint64_t seed, msasm_mlp** out) {
  if (!out) return fail(MSASM_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_out <= 0 || hidden <= 0 || hidden > 1024 || (hidden % 2)) return fail(MSASM_EINVAL, "bad MLP shape");
  msasm_mlp* n = new msasm_mlp(hidden, n_out);
  const size_t P = n->lay.total;
  // Glorot-uniform weights, zero biases (host generator, then copied)
  std::vector<float> w(P, 0.0f);
  std::mt19937_64 g(seed);
  auto fill = [&](size_t off, size_t count, int fan_in, int fan_out) {
    const double a = std::sqrt(6.0 / (fan_in + fan_out));
    std::uniform_real_distribution<double> U(-a, a);
    for (size_t i = 0; i < count; ++i) w[off + i] = float(U(g));
  };
  fill(n->lay.W1, hidden, 1, hidden);
  fill(n->lay.W2, size_t(hidden) * hidden, hidden, hidden);
  fill(n->lay.W3, size_t(n_out) * hidden, hidden, n_out);
  cudaError_t e = cudaMalloc(&n->d_w, P * 4);
  if (e == cudaSuccess) e = cudaMalloc(&n->d_w16, P * 2);
  if (e == cudaSuccess) e = cudaMalloc(&n->d_w3f, size_t(n_out) * hidden * 4);
  if (e == cudaSuccess) e = cudaMalloc(&n->d_g, P * 4);
  if (e == cudaSuccess) e = cudaMalloc(&n->d_m, P * 4);
  if (e == cudaSuccess) e = cudaMalloc(&n->d_v, P * 4);
  if (e == cudaSuccess) e = cudaMalloc(&n->d_step, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&n->d_loss, sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(n->d_w, w.data(), P * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(n->d_m, 0, P * 4);
  if (e == cudaSuccess) e = cudaMemset(n->d_v, 0, P * 4);
  if (e == cudaSuccess) e = cudaMemset(n->d_step, 0, sizeof(int));
  if (e != cudaSuccess) {
    delete n;
    return cuda_fail(e, "msasm_mlp_create");
  }
  to_half_kernel<<<152 * 4, 256>>>(n->d_w, P, n->d_w16);
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    delete n;
    return cuda_fail(e, "msasm_mlp_create");
  }
  *out = n;
  return MSASM_OK;
}

msasm_status msasm_mlp_info(const msasm_mlp* n, int64_t* n_params, int32_t* n_out, int32_t* hidden) {
  if (!n) return fail(MSASM_EINVAL, "mlp is NULL");
  if (n_params) *n_params = int64_t(n->lay.total);
  if (n_out) *n_out = n->lay.n_out;
  if (hidden) *hidden = n->lay.H;
  return MSASM_OK;
}

msasm_status msasm_mlp_set_params(msasm_mlp* n, const float* d_params, void* stream) {
  if (!n || !d_params) return fail(MSASM_EINVAL, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  n->w3_split_ok = false;
  MSASM_CUDA(cudaMemcpyAsync(n->d_w, d_params, n->lay.total * 4, cudaMemcpyDeviceToDevice, s));
  to_half_kernel<<<152 * 4, 256, 0, s>>>(n->d_w, n->lay.total, n->d_w16);
  MSASM_CUDA(cudaGetLastError());
  return MSASM_OK;
}

// FP32 master parameters and/or their FP16 compute copy (as float values)
msasm_status msasm_mlp_get_params(const msasm_mlp* n, float* d_master, void* d_half, void* stream) {
  if (!n) return fail(MSASM_EINVAL, "mlp is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (d_master) MSASM_CUDA(cudaMemcpyAsync(d_master, n->d_w, n->lay.total * 4, cudaMemcpyDeviceToDevice, s));
  if (d_half) MSASM_CUDA(cudaMemcpyAsync(d_half, n->d_w16, n->lay.total * 2, cudaMemcpyDeviceToDevice, s));
  return MSASM_OK;
}

msasm_status msasm_mlp_forward(msasm_mlp* n, const float* d_x, int32_t B, float* d_y, void* stream) {
  if (!n || !d_x || !d_y || B <= 0) return fail(MSASM_EINVAL, "bad MLP forward arguments");
  MSASM_TRY(mlp_ensure_batch(n, B));
  return mlp_forward(n, d_x, B, d_y, static_cast<cudaStream_t>(stream));
}

msasm_status msasm_mlp_forward_tc(msasm_mlp* n, const float* d_x, int32_t B, float* d_y, void* stream) {
  if (!n || !d_x || !d_y || B <= 0) return fail(MSASM_EINVAL, "bad MLP forward arguments");
  MSASM_TRY(mlp_ensure_batch(n, B));
  return mlp_forward_tc(n, d_x, B, d_y, static_cast<cudaStream_t>(stream));
}

// mean squared error over B samples and its gradient w.r.t. the (FP16) parameters; synchronises
msasm_status msasm_mlp_loss_grad(msasm_mlp* n, const float* d_x, const float* d_t, int32_t B, float* h_loss,
                                 float* d_grad, void* stream) {
  if (!n || !d_x || !d_t || B <= 0) return fail(MSASM_EINVAL, "bad MLP arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MSASM_TRY(mlp_ensure_batch(n, B));
  MSASM_CUDA(cudaMemsetAsync(n->d_loss, 0, sizeof(float), s));
  MSASM_TRY(mlp_loss_grad(n, d_x, d_t, B, s));
  if (d_grad) MSASM_CUDA(cudaMemcpyAsync(d_grad, n->d_g, n->lay.total * 4, cudaMemcpyDeviceToDevice, s));
  float l = 0.0f;
  MSASM_CUDA(cudaMemcpyAsync(&l, n->d_loss, sizeof(float), cudaMemcpyDeviceToHost, s));
  MSASM_CUDA(cudaStreamSynchronize(s));
  if (h_loss) *h_loss = l;
  return MSASM_OK;
}

// `steps` Adam steps on the whole batch; one step is captured in a CUDA graph and replayed.
// h_loss (optional, `steps` floats) receives the loss before each step.  Synchronises.
msasm_status msasm_mlp_train(msasm_mlp* n, const float* d_x, const float* d_t, int32_t B, int32_t steps, float lr,
                             float* h_loss, void* stream) {
  if (!n || !d_x || !d_t || B <= 0 || steps < 0) return fail(MSASM_EINVAL, "bad MLP training arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (steps > 0) n->w3_split_ok = false;         // the weights change
  MSASM_TRY(mlp_ensure_batch(n, B));
  float* d_hist = nullptr;
  if (h_loss && steps > 0) MSASM_CUDA(cudaMallocAsync(&d_hist, size_t(steps) * 4, s));
  if (!n->graph || n->graph_x != d_x || n->graph_t != d_t || n->graph_B != B || n->graph_lr != lr) {
    if (n->graph) cudaGraphExecDestroy(n->graph);
    n->graph = nullptr;
    cudaStream_t cs;
    MSASM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g;
    msasm_status st = MSASM_OK;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaMemsetAsync(n->d_loss, 0, sizeof(float), cs);
      st = mlp_train_step(n, d_x, d_t, B, lr, cs);
      e = cudaStreamEndCapture(cs, &g);
    }
    if (e == cudaSuccess && st == MSASM_OK) e = cudaGraphInstantiate(&n->graph, g, 0);
    if (e == cudaSuccess) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (st != MSASM_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "MLP training graph");
    n->graph_x = d_x;
    n->graph_t = d_t;
    n->graph_B = B;
    n->graph_lr = lr;
  }
  for (int i = 0; i < steps; ++i) {
    MSASM_CUDA(cudaGraphLaunch(n->graph, s));
    if (d_hist) MSASM_CUDA(cudaMemcpyAsync(d_hist + i, n->d_loss, sizeof(float), cudaMemcpyDeviceToDevice, s));
  }
  if (d_hist) {
    MSASM_CUDA(cudaMemcpyAsync(h_loss, d_hist, size_t(steps) * 4, cudaMemcpyDeviceToHost, s));
    MSASM_CUDA(cudaFreeAsync(d_hist, s));
  }
  MSASM_CUDA(cudaStreamSynchronize(s));
  return MSASM_OK;
}

void msasm_mlp_destroy(msasm_mlp* n) { delete n; }

// ------------------------------------------------------------------ surrogate
static msasm_status surrogate_create_impl(const msasm_tables* const* tables, const double* widths,
                                          int32_t n_tables, const double* d_coef_samples, int64_t n_sample_rows,
                                          int32_t rank, int32_t hidden, int32_t power_iters, uint64_t seed,
                                          void* stream, msasm_surrogate** out) {
  if (!tables || !widths || n_tables < 2 || !d_coef_samples || n_sample_rows <= 0 || rank <= 0 || rank > 64)
    return fail(MSASM_EINVAL, "surrogate: need >= 2 tables, coefficient samples and 1 <= rank <= 64");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n_nz = tables[0]->n_nz, K = 9 * tables[0]->n_pi;
  for (int k = 0; k < n_tables; ++k)
    if (!tables[k] || tables[k]->n_nz != n_nz || tables[k]->qd[0] != tables[0]->qd[0] ||
        tables[k]->qd[1] != tables[0]->qd[1] || tables[k]->qd[2] != tables[0]->qd[2])
      return fail(MSASM_EINVAL, "surrogate: all tables must share topology and q");
  const int over = 8, r_s = rank + over;                  // sketch width
  const int64_t J = int64_t(n_tables) * n_sample_rows;     // columns of M = [T_k C^T]
  std::unique_ptr<msasm_surrogate> guard(new msasm_surrogate());   // freed on an error or an exception
  msasm_surrogate* sur = guard.get();
  sur->rank = rank;
  for (int d = 0; d < 3; ++d) sur->qd[d] = tables[0]->qd[d];
  sur->K = K;
  sur->n_nz = n_nz;
  sur->n_train = n_tables;
  auto bail = [&](msasm_status st) { return st; };
  double *Mt = nullptr, *M = nullptr, *Om = nullptr, *Yt = nullptr, *Qt = nullptr, *Zt = nullptr, *Gd = nullptr,
         *Sd = nullptr, *Ud = nullptr, *Tt = nullptr, *Vk = nullptr;
  auto release = [&]() {
    cudaFree(Mt); cudaFree(M); cudaFree(Om); cudaFree(Yt); cudaFree(Qt); cudaFree(Zt); cudaFree(Gd); cudaFree(Sd);
    cudaFree(Ud); cudaFree(Tt); cudaFree(Vk);
  };
  cudaError_t e = cudaMalloc(&Mt, size_t(J) * n_nz * 8);
  if (e == cudaSuccess) e = cudaMalloc(&M, size_t(J) * n_nz * 8);
  if (e == cudaSuccess) e = cudaMalloc(&Om, size_t(r_s) * J * 8);
  if (e == cudaSuccess) e = cudaMalloc(&Yt, size_t(r_s) * n_nz * 8);
  if (e == cudaSuccess) e = cudaMalloc(&Qt, size_t(r_s) * n_nz * 8);
  if (e == cudaSuccess) e = cudaMalloc(&Zt, size_t(r_s) * J * 8);
  if (e == cudaSuccess) e = cudaMalloc(&Gd, size_t(r_s) * r_s * 8);
  if (e == cudaSuccess) e = cudaMalloc(&Sd, size_t(r_s) * r_s * 8);
  if (e == cudaSuccess) e = cudaMalloc(&Ud, size_t(rank) * n_nz * 8);
  if (e == cudaSuccess) e = cudaMalloc(&Tt, size_t(K) * n_nz * 8);
  if (e == cudaSuccess) e = cudaMalloc(&Vk, size_t(n_tables) * rank * K * 8);
  if (e != cudaSuccess) {
    release();
    return bail(cuda_fail(e, "surrogate work buffers"));
  }
  msasm_status st = MSASM_OK;
  // M^T rows: block k holds (T_k C^T)^T = C T_k^T  (n_sample_rows x n_nz)
  for (int k = 0; k < n_tables && st == MSASM_OK; ++k)
    st = gemm_simt<double>(d_coef_samples, K, tables[k]->d_T, K, n_sample_rows, n_nz, K,
                           Mt + size_t(k) * n_sample_rows * n_nz, n_nz, s);
  // M = (M^T)^T  (n_nz x J) through the generic transpose (rows J, columns n_nz)
  if (st == MSASM_OK) st = transpose_table_gpu<double>(Mt, int(J), n_nz, M, s);
  // Gaussian sketch Omega^T (r_s x J)
  std::vector<double> om(size_t(r_s) * J);
  {
    std::mt19937_64 g(seed ^ 0x9E3779B97F4A7C15ull);
    std::normal_distribution<double> N(0.0, 1.0);
    for (auto& v : om) v = N(g);
  }
  if (st == MSASM_OK) {
    e = cudaMemcpyAsync(Om, om.data(), om.size() * 8, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) st = cuda_fail(e, "sketch");
  }
  auto orthonormalise = [&]() -> msasm_status {  // rows of Yt -> orthonormal rows of Qt (Cholesky QR, twice)
    for (int pass = 0; pass < 2; ++pass) {
      double* src = pass == 0 ? Yt : Qt;
      MSASM_TRY(gemm_simt<double>(src, n_nz, src, n_nz, r_s, r_s, n_nz, Gd, r_s, s));
      std::vector<double> G(size_t(r_s) * r_s), Rinv;
      MSASM_CUDA(cudaMemcpyAsync(G.data(), Gd, G.size() * 8, cudaMemcpyDeviceToHost, s));
      MSASM_CUDA(cudaStreamSynchronize(s));
      if (!cholesky_upper_inverse(G, r_s, Rinv)) return fail(MSASM_EUNSUPPORTED, "surrogate: rank-deficient sketch");
      std::vector<double> S(size_t(r_s) * r_s);   // S = Rinv^T
      for (int i = 0; i < r_s; ++i)
        for (int j = 0; j < r_s; ++j) S[size_t(i) * r_s + j] = Rinv[size_t(j) * r_s + i];
      MSASM_CUDA(cudaMemcpyAsync(Sd, S.data(), S.size() * 8, cudaMemcpyHostToDevice, s));
      double* dst = pass == 0 ? Qt : Yt;
      small_left_kernel<<<152 * 8, 256, 0, s>>>(Sd, r_s, r_s, src, n_nz, dst);
      MSASM_CUDA(cudaGetLastError());
      MSASM_CUDA(cudaStreamSynchronize(s));   // S (host) reused next pass
      if (pass == 1) MSASM_CUDA(cudaMemcpyAsync(Qt, Yt, size_t(r_s) * n_nz * 8, cudaMemcpyDeviceToDevice, s));
    }
    return MSASM_OK;
  };
  // Y^T = Omega^T M^T ... as rows: Yt[r][i] = sum_j Om[r][j] M[i][j]
  if (st == MSASM_OK) st = gemm_simt<double>(Om, J, M, J, r_s, n_nz, int(J), Yt, n_nz, s);
  if (st == MSASM_OK) st = orthonormalise();
  for (int it = 0; it < power_iters && st == MSASM_OK; ++it) {
    st = gemm_simt<double>(Qt, n_nz, Mt, n_nz, r_s, int(J), n_nz, Zt, J, s);      // Zt = Q^T M
    if (st == MSASM_OK) st = gemm_simt<double>(Zt, J, M, J, r_s, n_nz, int(J), Yt, n_nz, s);   // Y = M Z
    if (st == MSASM_OK) st = orthonormalise();
  }
  // small SVD: eig of (Q^T M)(Q^T M)^T, U = Q E[:, :rank]
  if (st == MSASM_OK) st = gemm_simt<double>(Qt, n_nz, Mt, n_nz, r_s, int(J), n_nz, Zt, J, s);
  if (st == MSASM_OK) st = gemm_simt<double>(Zt, J, Zt, J, r_s, r_s, int(J), Gd, r_s, s);
  if (st == MSASM_OK) {
    std::vector<double> G(size_t(r_s) * r_s), w, E;
    e = cudaMemcpyAsync(G.data(), Gd, G.size() * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "surrogate basis");
    if (st == MSASM_OK) {
      symmetric_eigen(G, r_s, w, E);
      std::vector<double> S(size_t(rank) * r_s);   // S[k][l] = E[l][k]
      for (int k = 0; k < rank; ++k)
        for (int l = 0; l < r_s; ++l) S[size_t(k) * r_s + l] = E[size_t(l) * r_s + k];
      e = cudaMemcpyAsync(Sd, S.data(), S.size() * 8, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) {
        small_left_kernel<<<152 * 8, 256, 0, s>>>(Sd, rank, r_s, Qt, n_nz, Ud);   // Ut (rank x n_nz)
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) st = cuda_fail(e, "surrogate basis");
    }
  }
  // targets V_k^T = U^T T_k  (rank x K): rows of Ut against the transposed table
  for (int k = 0; k < n_tables && st == MSASM_OK; ++k) {
    st = transpose_table_gpu<double>(tables[k]->d_T, n_nz, K, Tt, s);
    if (st == MSASM_OK) st = gemm_simt<double>(Ud, n_nz, Tt, n_nz, rank, K, n_nz, Vk + size_t(k) * rank * K, K, s);
  }
  // U (FP32, n_nz x rank row-major) = transpose of Ut
  if (st == MSASM_OK) {
    e = cudaMalloc(&sur->d_U, size_t(n_nz) * rank * 4);
    if (e != cudaSuccess) st = cuda_fail(e, "surrogate U");
  }
  if (st == MSASM_OK) st = transpose_table_gpu<float>(Ud, rank, n_nz, sur->d_U, s);
  // targets, normalised: scale = RMS of the centred targets
  const int n_out = rank * K;
  if (st == MSASM_OK) {
    std::vector<double> V(size_t(n_tables) * n_out);
    e = cudaMemcpyAsync(V.data(), Vk, V.size() * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "surrogate targets");
    double ss = 0.0;
    for (int o = 0; o < n_out && st == MSASM_OK; ++o) {
      double mu = 0.0;
      for (int k = 0; k < n_tables; ++k) mu += V[size_t(k) * n_out + o];
      mu /= n_tables;
      for (int k = 0; k < n_tables; ++k) ss += (V[size_t(k) * n_out + o] - mu) * (V[size_t(k) * n_out + o] - mu);
    }
    sur->scale = float(std::sqrt(ss / (double(n_tables) * n_out)) + 1e-30);
    e = cudaMalloc(&sur->d_mean, size_t(n_out) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&sur->d_targets, size_t(n_tables) * n_out * 4);
    if (e == cudaSuccess) e = cudaMalloc(&sur->d_x, size_t(n_tables) * 4);
    if (e != cudaSuccess) st = cuda_fail(e, "surrogate targets");
  }
  if (st == MSASM_OK) {
    normalise_targets_kernel<<<152 * 4, 256, 0, s>>>(sur->d_targets, Vk, n_tables, n_out, sur->d_mean,
                                                    1.0 / double(sur->scale));
    std::vector<float> x(n_tables);
    for (int k = 0; k < n_tables; ++k) x[k] = float((widths[k] - sur->w0) / sur->ws);
    e = cudaMemcpyAsync(sur->d_x, x.data(), x.size() * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "surrogate targets");
  }
  release();
  if (st != MSASM_OK) return bail(st);
  st = msasm_mlp_create(n_out, hidden, seed, &sur->mlp);
  if (st != MSASM_OK) return bail(st);
  *out = guard.release();
  return MSASM_OK;
}

msasm_status msasm_surrogate_create(const msasm_tables* const* tables, const double* widths, int32_t n_tables,
                                    const double* d_coef_samples, int64_t n_sample_rows, int32_t rank, int32_t hidden,
                                    int32_t power_iters, uint64_t seed, void* stream, msasm_surrogate** out) {
  if (!out) return fail(MSASM_EINVAL, "out is NULL");
  *out = nullptr;
  try {
    return surrogate_create_impl(tables, widths, n_tables, d_coef_samples, n_sample_rows, rank, hidden, power_iters,
                                 seed, stream, out);
  } catch (const std::bad_alloc&) {
    return fail(MSASM_ENOMEM, "host allocation failed while fitting the surrogate");
  }
}

msasm_status msasm_surrogate_train(msasm_surrogate* sur, int32_t steps, float lr, float* h_loss, void* stream) {
  if (!sur) return fail(MSASM_EINVAL, "surrogate is NULL");
  return msasm_mlp_train(sur->mlp, sur->d_x, sur->d_targets, sur->n_train, steps, lr, h_loss, stream);
}

msasm_status msasm_surrogate_mlp(msasm_surrogate* sur, msasm_mlp** mlp) {
  if (!sur || !mlp) return fail(MSASM_EINVAL, "NULL argument");
  *mlp = sur->mlp;
  return MSASM_OK;
}

msasm_status msasm_surrogate_info(const msasm_surrogate* sur, int32_t* rank, int32_t* K, int32_t* n_nz) {
  if (!sur) return fail(MSASM_EINVAL, "surrogate is NULL");
  if (rank) *rank = sur->rank;
  if (K) *K = sur->K;
  if (n_nz) *n_nz = sur->n_nz;
  return MSASM_OK;
}

msasm_status msasm_surrogate_basis(const msasm_surrogate* sur, float* d_U, void* stream) {
  if (!sur || !d_U) return fail(MSASM_EINVAL, "NULL argument");
  MSASM_CUDA(cudaMemcpyAsync(d_U, sur->d_U, size_t(sur->n_nz) * sur->rank * 4, cudaMemcpyDeviceToDevice,
                             static_cast<cudaStream_t>(stream)));
  return MSASM_OK;
}

// V(w)^T for n widths: d_Vt (n x rank x K) FP32
msasm_status msasm_surrogate_predict(msasm_surrogate* sur, const double* d_widths, int64_t n, float* d_Vt,
                                     void* stream) {
  if (!sur || !d_widths || !d_Vt || n <= 0 || n > (1 << 30)) return fail(MSASM_EINVAL, "bad predict arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* x = nullptr;
  MSASM_CUDA(cudaMallocAsync(&x, size_t(n) * 4, s));
  normalise_inputs_kernel<<<152, 256, 0, s>>>(d_widths, n, sur->w0, sur->ws, x);
  MSASM_TRY(mlp_ensure_batch(sur->mlp, int(n)));
  msasm_status st = mlp_forward_tc(sur->mlp, x, int(n), d_Vt, s);
  if (st == MSASM_OK) {
    denormalise_kernel<<<152 * 4, 256, 0, s>>>(d_Vt, n, sur->mlp->lay.n_out, sur->d_mean, sur->scale);
    if (cudaGetLastError() != cudaSuccess) st = fail(MSASM_ECUDA, "denormalise");
  }
  cudaFreeAsync(x, s);
  return st;
}

// nzdata of n_tiles tiles from the low-rank factors: nz[t][m][ab] = sum_r Z[9t + ab][r] U[m][r],
// Z[9t + ab][r] = sum_k Vt_t[r][k] coef[9t + ab][k] (FP32), the second product on the tensor cores
// in split FP16 (U given as its slices; d_nz in the tile-block layout with m stride ld).  d_work holds the slices of Z:
// lowrank_work_bytes(n_tiles, rank).
static size_t lowrank_work_bytes(int64_t n_tiles, int rank) {
  return 2 * ((tc_slice_bytes(9 * n_tiles, rank, kLowRankSplit) + 255) & ~size_t(255)) + size_t(9 * n_tiles) * 4;
}
static msasm_status lowrank_contract_gpu(const void* U_hi, const void* U_lo, const float* U_scale, int n_nz, int rank,
                                         int K, const float* d_Vt, const double* d_coef, int64_t n_tiles, float* d_Z,
                                         void* d_work, float* d_nz, int ld, unsigned* d_err, cudaStream_t s) {
  const size_t zsm = size_t(9) * K * sizeof(float);
  if (zsm > 200 * 1024) return fail(MSASM_EUNSUPPORTED, "K too large for the low-rank kernel");
  MSASM_CUDA(cudaFuncSetAttribute(lowrank_z_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(zsm)));
  lowrank_z_kernel<<<unsigned(std::min<int64_t>(n_tiles, 152 * 8)), 256, zsm, s>>>(d_Vt, d_coef, n_tiles, rank, K, d_Z);
  MSASM_CUDA(cudaGetLastError());
  const size_t sb = (tc_slice_bytes(9 * n_tiles, rank, kLowRankSplit) + 255) & ~size_t(255);
  uint8_t* w = static_cast<uint8_t*>(d_work);
  float* z_scale = reinterpret_cast<float*>(w + 2 * sb);
  MSASM_TRY(tc_split_f32_gpu(d_Z, 9 * n_tiles, rank, kLowRankSplit, w, w + sb, z_scale, s));
  return contract_tc_gpu(kLowRankSplit, U_hi, U_lo, U_scale, n_nz, w, w + sb, z_scale, 9 * n_tiles, rank, d_nz, ld,
                         true, d_err, s);
}

// split-FP16 slices of U, made once per surrogate
static msasm_status ensure_u_split(msasm_surrogate* sur, cudaStream_t s) {
  if (sur->d_Uhi) return MSASM_OK;
  const size_t ub = tc_slice_bytes(sur->n_nz, sur->rank, kLowRankSplit);
  MSASM_CUDA(cudaMalloc(&sur->d_Uhi, ub));
  MSASM_CUDA(cudaMalloc(&sur->d_Ulo, ub));
  MSASM_CUDA(cudaMalloc(&sur->d_Uscale, size_t(sur->n_nz) * 4));
  MSASM_CUDA(cudaMalloc(&sur->d_err, sizeof(unsigned)));
  MSASM_CUDA(cudaMemsetAsync(sur->d_err, 0, sizeof(unsigned), s));
  return tc_split_f32_gpu(sur->d_U, sur->n_nz, sur->rank, kLowRankSplit, sur->d_Uhi, sur->d_Ulo, sur->d_Uscale, s);
}

msasm_status msasm_lowrank_contract(const float* d_U, int32_t n_nz, int32_t rank, int32_t K, const float* d_Vt,
                                    const double* d_coef, int64_t n_tiles, float* d_nz, void* stream) {
  if (!d_U || !d_Vt || !d_coef || !d_nz || n_tiles <= 0 || n_nz <= 0 || rank <= 0 || K <= 0)
    return fail(MSASM_EINVAL, "bad low-rank contraction arguments");
  if (rank > 64) return fail(MSASM_EUNSUPPORTED, "rank above 64");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t ub = (tc_slice_bytes(n_nz, rank, kLowRankSplit) + 255) & ~size_t(255);
  const size_t zb = (size_t(9 * n_tiles) * rank * 4 + 255) & ~size_t(255);
  const size_t bytes = 2 * ub + ((size_t(n_nz) * 4 + 255) & ~size_t(255)) + zb + lowrank_work_bytes(n_tiles, rank) + 256;
  void* buf = nullptr;
  MSASM_CUDA(cudaMallocAsync(&buf, bytes, s));
  uint8_t* b = static_cast<uint8_t*>(buf);
  float* u_scale = reinterpret_cast<float*>(b + 2 * ub);
  float* Z = reinterpret_cast<float*>(b + 2 * ub + ((size_t(n_nz) * 4 + 255) & ~size_t(255)));
  void* work = reinterpret_cast<uint8_t*>(Z) + zb;
  unsigned* err = reinterpret_cast<unsigned*>(static_cast<uint8_t*>(work) + lowrank_work_bytes(n_tiles, rank));
  msasm_status st = MSASM_OK;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) st = cuda_fail(e, "cudaMemsetAsync");
  if (st == MSASM_OK) st = tc_split_f32_gpu(d_U, n_nz, rank, kLowRankSplit, b, b + ub, u_scale, s);
  if (st == MSASM_OK)
    st = lowrank_contract_gpu(b, b + ub, u_scale, n_nz, rank, K, d_Vt, d_coef, n_tiles, Z, work, d_nz, n_nz, err, s);
  unsigned h_err = 0;
  if (st == MSASM_OK) {
    e = cudaMemcpyAsync(&h_err, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "low-rank contraction");
  }
  cudaFreeAsync(buf, s);
  if (st == MSASM_OK && h_err) st = fail(MSASM_ECUDA, "a tensor-core pipeline wait timed out (results invalid)");
  return st;
}

// K from per-tile widths: pullback, MLP, low-rank contraction, scatter (FP32 values)
msasm_status msasm_surrogate_assemble(msasm_plan* plan, msasm_surrogate* sur, const double* d_ctrl, double E,
                                      double nu, const double* d_widths, float* d_values, void* stream) {
  if (!plan || !sur || !d_ctrl || !d_widths || !d_values) return fail(MSASM_EINVAL, "NULL argument");
  if (plan->tab->n_nz != sur->n_nz || 9 * plan->tab->n_pi != sur->K || plan->tab->qd[0] != sur->qd[0] ||
      plan->tab->qd[1] != sur->qd[1] || plan->tab->qd[2] != sur->qd[2])
    return fail(MSASM_EINVAL, "surrogate and plan disagree on the table shape");
  if (!(E > 0.0) || !(nu > -1.0 && nu < 0.5)) return fail(MSASM_EINVAL, "material: need E > 0 and -1 < nu < 0.5");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = E / (2.0 * (1.0 + nu));
  const int64_t P = plan->tiles_per_pass;
  const int ld = (sur->n_nz + 7) & ~7;
  if (sur->rank > 64) return fail(MSASM_EUNSUPPORTED, "rank above 64");
  MSASM_TRY(ensure_u_split(sur, s));
  float *Vt = nullptr, *Z = nullptr;
  void* work = nullptr;
  MSASM_CUDA(cudaMallocAsync(&Vt, size_t(P) * sur->rank * sur->K * 4, s));
  MSASM_CUDA(cudaMallocAsync(&Z, size_t(9 * P) * sur->rank * 4, s));
  MSASM_CUDA(cudaMallocAsync(&work, lowrank_work_bytes(P, sur->rank), s));
  msasm_status st = MSASM_OK;
  for (int64_t t0 = 0; t0 < plan->n_tiles && st == MSASM_OK; t0 += P) {
    const int64_t nt = std::min(P, plan->n_tiles - t0);
    st = pullback_gpu(plan, d_ctrl, lam, mu, t0, nt, plan->d_coef, s);
    if (st == MSASM_OK) st = msasm_surrogate_predict(sur, d_widths + t0, nt, Vt, stream);
    if (st == MSASM_OK)
      st = lowrank_contract_gpu(sur->d_Uhi, sur->d_Ulo, sur->d_Uscale, sur->n_nz, sur->rank, sur->K, Vt, plan->d_coef,
                                nt, Z, work, static_cast<float*>(plan->d_nz), ld, sur->d_err, s);
    if (st == MSASM_OK) st = scatter_pass_gpu<float>(plan, static_cast<const float*>(plan->d_nz), ld, t0, nt, d_values, s);
  }
  cudaFreeAsync(Vt, s);
  cudaFreeAsync(Z, s);
  cudaFreeAsync(work, s);
  return st;
}

void msasm_surrogate_destroy(msasm_surrogate* sur) { delete sur; }

// Surrogate file payload (kind tag "MSASMSUR"): rank, K, n_nz, n_train, q3 (int32), the width
// normalisation w0, ws (double) and target scale (float), the MLP shape H, n_out (int32), its
// parameter count (int64) and Adam step (int32); then the FP32 arrays U (n_nz x rank), target mean
// (n_out), training inputs (n_train), normalised targets (n_train x n_out), and the MLP's master
// weights, Adam first and second moments (each n_params).  A loaded surrogate predicts, assembles
// and continues training exactly as the saved one.
static const char kSurrogateTag[8] = {'M', 'S', 'A', 'S', 'M', 'S', 'U', 'R'};

static msasm_status surrogate_save_impl(const msasm_surrogate* sur, const char* path, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const msasm_mlp* n = sur->mlp;
  const int32_t head[7] = {sur->rank, sur->K, sur->n_nz, sur->n_train, sur->qd[0], sur->qd[1], sur->qd[2]};
  StoreWriter w;
  w.put_array(head, 7);
  w.put(sur->w0);
  w.put(sur->ws);
  w.put(sur->scale);
  const int32_t shape[2] = {n->lay.H, n->lay.n_out};
  w.put_array(shape, 2);
  const int64_t P = int64_t(n->lay.total);
  w.put(P);
  int32_t* step = w.reserve_array<int32_t>(1);
  const size_t n_out = size_t(n->lay.n_out);
  const size_t nU = size_t(sur->n_nz) * sur->rank, nX = size_t(sur->n_train), nTg = nX * n_out;
  const size_t step_off = reinterpret_cast<unsigned char*>(step) - w.at(0);
  const size_t arr_off = w.size();
  w.reserve_array<float>(nU + n_out + nX + nTg + 3 * size_t(P));
  // pointers into the buffer only after its last growth
  int32_t* hstep = reinterpret_cast<int32_t*>(w.at(step_off));
  float* h = reinterpret_cast<float*>(w.at(arr_off));
  MSASM_CUDA(cudaMemcpyAsync(hstep, n->d_step, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  MSASM_CUDA(cudaMemcpyAsync(h, sur->d_U, nU * 4, cudaMemcpyDeviceToHost, s));
  MSASM_CUDA(cudaMemcpyAsync(h + nU, sur->d_mean, n_out * 4, cudaMemcpyDeviceToHost, s));
  MSASM_CUDA(cudaMemcpyAsync(h + nU + n_out, sur->d_x, nX * 4, cudaMemcpyDeviceToHost, s));
  MSASM_CUDA(cudaMemcpyAsync(h + nU + n_out + nX, sur->d_targets, nTg * 4, cudaMemcpyDeviceToHost, s));
  float* hw = h + nU + n_out + nX + nTg;
  MSASM_CUDA(cudaMemcpyAsync(hw, n->d_w, size_t(P) * 4, cudaMemcpyDeviceToHost, s));
  MSASM_CUDA(cudaMemcpyAsync(hw + P, n->d_m, size_t(P) * 4, cudaMemcpyDeviceToHost, s));
  MSASM_CUDA(cudaMemcpyAsync(hw + 2 * P, n->d_v, size_t(P) * 4, cudaMemcpyDeviceToHost, s));
  MSASM_CUDA(cudaStreamSynchronize(s));
  return w.write(path, kSurrogateTag);
}

msasm_status msasm_surrogate_save(const msasm_surrogate* sur, const char* path, void* stream) {
  if (!sur || !path || !sur->mlp) return fail(MSASM_EINVAL, "surrogate or path is NULL");
  try {
    return surrogate_save_impl(sur, path, stream);
  } catch (const std::bad_alloc&) {
    return fail(MSASM_ENOMEM, "no host memory to stage the surrogate");
  }
}

msasm_status msasm_surrogate_load(const char* path, void* stream, msasm_surrogate** out) {
  if (!out || !path) return fail(MSASM_EINVAL, "out or path is NULL");
  *out = nullptr;
  StoreReader r;
  MSASM_TRY(r.open(path, kSurrogateTag));
  auto bad = [&](const char* what) { return fail(MSASM_EIO, std::string("surrogate file: ") + what + ": " + path); };
  int32_t head[7], shape[2], step = 0;
  double w0 = 0.0, ws = 0.0;
  float scale = 0.0f;
  int64_t P = 0;
  bool ok = true;
  for (int i = 0; i < 7; ++i) ok = ok && r.get(head[i]);
  ok = ok && r.get(w0) && r.get(ws) && r.get(scale) && r.get(shape[0]) && r.get(shape[1]) && r.get(P) && r.get(step);
  if (!ok) return bad("header");
  const int rank = head[0], K = head[1], n_nz = head[2], n_train = head[3];
  if (rank < 1 || rank > 64 || K < 1 || K > 9 * 216 || n_nz < 1 || n_train < 2 || shape[1] != rank * K)
    return bad("sizes");
  for (int d = 0; d < 3; ++d)
    if (head[4 + d] < 0 || head[4 + d] > 5) return bad("degrees");
  if (shape[0] <= 0 || shape[0] > 1024 || (shape[0] % 2) || int64_t(MlpLayout(shape[0], shape[1]).total) != P)
    return bad("MLP shape");
  const size_t n_out = size_t(shape[1]);
  const size_t nU = size_t(n_nz) * rank, nX = size_t(n_train), nTg = nX * n_out;
  const unsigned char* src = r.get_array<float>(nU + n_out + nX + nTg + 3 * size_t(P));
  if (!src || !r.at_end()) return bad("arrays");
  msasm_surrogate* sur = new msasm_surrogate();
  auto bail = [&](msasm_status st) {
    delete sur;
    return st;
  };
  sur->rank = rank;
  sur->K = K;
  sur->n_nz = n_nz;
  sur->n_train = n_train;
  for (int d = 0; d < 3; ++d) sur->qd[d] = head[4 + d];
  sur->w0 = w0;
  sur->ws = ws;
  sur->scale = scale;
  msasm_status st = msasm_mlp_create(int32_t(n_out), shape[0], 0, &sur->mlp);
  if (st != MSASM_OK) return bail(st);
  msasm_mlp* n = sur->mlp;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMalloc(&sur->d_U, nU * 4);
  if (e == cudaSuccess) e = cudaMalloc(&sur->d_mean, n_out * 4);
  if (e == cudaSuccess) e = cudaMalloc(&sur->d_x, nX * 4);
  if (e == cudaSuccess) e = cudaMalloc(&sur->d_targets, nTg * 4);
  size_t off = 0;
  auto up = [&](void* dst, size_t count) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src + off, count * 4, cudaMemcpyHostToDevice, s);
    off += count * 4;
  };
  up(sur->d_U, nU);
  up(sur->d_mean, n_out);
  up(sur->d_x, nX);
  up(sur->d_targets, nTg);
  up(n->d_w, size_t(P));
  up(n->d_m, size_t(P));
  up(n->d_v, size_t(P));
  if (e == cudaSuccess) e = cudaMemcpyAsync(n->d_step, &step, sizeof(int32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    to_half_kernel<<<152 * 4, 256, 0, s>>>(n->d_w, n->lay.total, n->d_w16);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the reader's buffer and `step` must outlive the copies
  if (e != cudaSuccess) return bail(cuda_fail(e, "msasm_surrogate_load"));
  n->w3_split_ok = false;
  *out = sur;
  return MSASM_OK;
}

}  // extern "C"
