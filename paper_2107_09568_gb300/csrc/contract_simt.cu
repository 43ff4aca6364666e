// K3: the contraction of eq. 58 on the CUDA cores (FP64 DFMA or FP32 FFMA).
//
//   nz[t][m][3a + b] = sum_k coef[n][k] * T[m][k],   n = 9t + 3a + b,  k = 9C + 3i + j,
//
// i.e. the tile blocks of nzdata = mat[K] mat[<A>] (the same GEMM serves the adjoint and the
// surrogate with a plain row-major output C[n][m]).  A 128 x 128 output tile per CTA, 256
// threads with an 8 x 8 register tile each (two 4-wide groups per direction, so
// that in the row layout the stores of a warp are contiguous), operands staged through shared
// memory k-major with a register prefetch of the next k-slab.  On GB300 the FP64
// form is bound by the DFMA rate (about 1.2 TFLOP/s for the whole GPU), the FP32
// form by the FFMA rate.
#include "common.h"

namespace msasm {

// C[n][m] = sum_k A[n][k] B[m][k] with row strides lda, ldb, ldc (the adjoint uses A = G, B = the
// transposed table, C = W); with BLOCKS the contraction's tile blocks C[n/9][m][n%9] with m stride
// ld_nz (A = coef, B = table).
template <typename T, int BK, bool BLOCKS>
__global__ void __launch_bounds__(256) contract_simt_kernel(const T* __restrict__ coef, int64_t lda,
                                                            const T* __restrict__ tab, int64_t ldb, int64_t N, int M,
                                                            int K, int64_t ld_nz, T* __restrict__ nz) {
  constexpr int BN = 128, BM = 128;
  constexpr int LOADS = BN * BK / 256;          // elements per thread per operand per slab
  __shared__ T As[2][BK][BN + 4];
  __shared__ T Bs[2][BK][BM + 4];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t n0 = int64_t(blockIdx.y) * BN;
  const int m0 = blockIdx.x * BM;
  T acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = T(0);
  T ra[LOADS], rb[LOADS];
  auto load = [&](int k0) {
#pragma unroll
    for (int l = 0; l < LOADS; ++l) {
      int e = tid + l * 256;
      int r = e / BK, kk = e % BK;
      int64_t n = n0 + r;
      int m = m0 + r, k = k0 + kk;
      ra[l] = (n < N && k < K) ? coef[n * lda + k] : T(0);
      rb[l] = (m < M && k < K) ? tab[int64_t(m) * ldb + k] : T(0);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int l = 0; l < LOADS; ++l) {
      int e = tid + l * 256;
      int r = e / BK, kk = e % BK;
      As[buf][kk][r] = ra[l];
      Bs[buf][kk][r] = rb[l];
    }
  };
  const int n_slabs = (K + BK - 1) / BK;
  load(0);
  store(0);
  __syncthreads();
  for (int s = 0; s < n_slabs; ++s) {
    const int buf = s & 1;
    if (s + 1 < n_slabs) load((s + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[8], b[8];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[buf][kk][ty * 4 + i];
        a[i + 4] = As[buf][kk][64 + ty * 4 + i];
        b[i] = Bs[buf][kk][tx * 4 + i];
        b[i + 4] = Bs[buf][kk][64 + tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (s + 1 < n_slabs) store(buf ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int64_t n = n0 + ((i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (n >= N) continue;
    if constexpr (BLOCKS) {
      T* blk = nz + (n / 9) * 9 * ld_nz + (n % 9);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        int m = m0 + ((j < 4) ? tx * 4 + j : 64 + tx * 4 + (j - 4));
        if (m < M) blk[int64_t(m) * 9] = acc[i][j];
      }
    } else {
      T* row = nz + n * ld_nz;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        int m = m0 + ((j < 4) ? tx * 4 + j : 64 + tx * 4 + (j - 4));
        if (m < M) row[m] = acc[i][j];
      }
    }
  }
}

template <typename T, bool BLOCKS>
static msasm_status gemm_simt_any(const T* A, int64_t lda, const T* B, int64_t ldb, int64_t N, int M, int K, T* C,
                                  int64_t ldc, cudaStream_t stream) {
  dim3 grid(unsigned((M + 127) / 128), unsigned((N + 127) / 128));
  if (grid.y > 65535) return fail(MSASM_EUNSUPPORTED, "too many rows for one CUDA-core contraction");
  constexpr int BK = sizeof(T) == 8 ? 8 : 16;
  contract_simt_kernel<T, BK, BLOCKS><<<grid, 256, 0, stream>>>(A, lda, B, ldb, N, M, K, ldc, C);
  MSASM_CUDA(cudaGetLastError());
  return MSASM_OK;
}

template <typename T>
msasm_status gemm_simt(const T* A, int64_t lda, const T* B, int64_t ldb, int64_t N, int M, int K, T* C, int64_t ldc,
                       cudaStream_t stream) {
  return gemm_simt_any<T, false>(A, lda, B, ldb, N, M, K, C, ldc, stream);
}
template msasm_status gemm_simt<double>(const double*, int64_t, const double*, int64_t, int64_t, int, int, double*,
                                        int64_t, cudaStream_t);
template msasm_status gemm_simt<float>(const float*, int64_t, const float*, int64_t, int64_t, int, int, float*,
                                       int64_t, cudaStream_t);

msasm_status contract_simt_f64(const double* d_coef, const double* d_T, int64_t n_tiles, int n_nz, int K, int ld_nz,
                               double* d_nz, cudaStream_t stream) {
  return gemm_simt_any<double, true>(d_coef, K, d_T, K, 9 * n_tiles, n_nz, K, d_nz, ld_nz, stream);
}

msasm_status contract_simt_f32(const float* d_coef, const float* d_T, int64_t n_tiles, int n_nz, int K, int ld_nz,
                               float* d_nz, cudaStream_t stream) {
  return gemm_simt_any<float, true>(d_coef, K, d_T, K, 9 * n_tiles, n_nz, K, d_nz, ld_nz, stream);
}

// FP64 -> FP32 conversion of an operand (round to nearest).
__global__ void to_f32_kernel(const double* __restrict__ x, int64_t n, float* __restrict__ y) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = __double2float_rn(x[i]);
}

msasm_status to_f32_gpu(const double* x, int64_t n, float* y, cudaStream_t stream) {
  to_f32_kernel<<<152 * 8, 256, 0, stream>>>(x, n, y);
  MSASM_CUDA(cudaGetLastError());
  return MSASM_OK;
}

}  // namespace msasm
