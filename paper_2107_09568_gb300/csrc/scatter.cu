// K5: step 4 of Sec. 3.2.4 -- add the tile blocks of nzdata into the global CSR values.
//
// Pair m = (A, B) of tile t owns the 3x3 block at rows 3 g(A) + a, columns
// 3 g(B) + b, and (A != B) its transpose at rows 3 g(B) + b, columns 3 g(A) + a.
// With the rank word r_u | r_l << 16 of the plan, the upper entry (a, b) lives at
// rowptr[3 g(A) + a] + 3 r_u + b and the lower one at rowptr[3 g(B) + b] + 3 r_l + a.
// Entries shared by two tiles (both points on a glued face) get the lower-indexed
// tile's value by a plain store here; the second tile adds its value in
// scatter_second_kernel, launched after this one on the same stream, so every
// entry is written without atomics and the two-term sum is order independent.
#include "common.h"

namespace msasm {

// One CTA per (tile, chunk of kScatterChunk pairs), chunks of a tile adjacent in launch
// order: the whole GPU works on a few tiles at a time, so the rows being written (about
// 1.6 MB of FP32 values per 725-point tile) stay in L2 until every sector of them is
// complete, and no partially written sector is evicted (which would cost a DRAM read).
// The row starts of the tile's points (rowptr[3 g(A)] and the row length 3 deg(g(A))) are
// staged in shared memory, so a pair needs only its rank word, its nine values and two
// shared-memory reads before its stores; every thread keeps kScatterUnroll pairs in flight.
constexpr int kScatterThreads = 256;
constexpr int kScatterUnroll = 4;
constexpr int kScatterChunk = 2048;

template <typename T>
__global__ void __launch_bounds__(kScatterThreads) scatter_tile_kernel(
    const T* __restrict__ nz, int ld_nz, int n_nz, int64_t t0, const int32_t* __restrict__ pairs,
    const int32_t* __restrict__ gmap, int n_T, const uint32_t* __restrict__ rank, const int64_t* __restrict__ rowptr,
    T* __restrict__ values) {
  extern __shared__ int64_t rowbase[];               // [n_T] row start, then [n_T] int32 row lengths
  int32_t* rowlen = reinterpret_cast<int32_t*>(rowbase + n_T);
  const int chunks = (n_nz + kScatterChunk - 1) / kScatterChunk;
  const int64_t tl = blockIdx.x / chunks, t = t0 + tl;
  const int c_begin = (blockIdx.x % chunks) * kScatterChunk;
  const int c_end = min(n_nz, c_begin + kScatterChunk);
  for (int A = threadIdx.x; A < n_T; A += blockDim.x) {
    const int64_t g = gmap[t * n_T + A];
    const int64_t b = rowptr[3 * g];
    rowbase[A] = b;
    rowlen[A] = int32_t(rowptr[3 * g + 1] - b);
  }
  __syncthreads();
  const T* nzt = nz + 9 * tl * ld_nz;
  const uint32_t* rk = rank + t * n_nz;
  for (int m0 = c_begin + threadIdx.x; m0 < c_end; m0 += kScatterThreads * kScatterUnroll) {
    uint32_t w[kScatterUnroll];
    int2 ab[kScatterUnroll];
    T v[kScatterUnroll][9];
#pragma unroll
    for (int u = 0; u < kScatterUnroll; ++u) {
      const int m = m0 + u * kScatterThreads;
      if (m < c_end) {
        w[u] = rk[m];
        ab[u] = reinterpret_cast<const int2*>(pairs)[m];
#pragma unroll
        for (int k = 0; k < 9; ++k) v[u][k] = nzt[size_t(k) * ld_nz + m];
      } else {
        w[u] = 1u << 31;
      }
    }
#pragma unroll
    for (int u = 0; u < kScatterUnroll; ++u) {
      if (w[u] >> 31) continue;
      const int A = ab[u].x, B = ab[u].y;
      const int ru = int(w[u] & 0xffffu), rl = int((w[u] >> 16) & 0x7fffu);
      const int64_t ba = rowbase[A] + 3 * ru;
      const int64_t la = rowlen[A];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        T* dst = values + ba + a * la;
        dst[0] = v[u][3 * a + 0];
        dst[1] = v[u][3 * a + 1];
        dst[2] = v[u][3 * a + 2];
      }
      if (A != B) {
        const int64_t bb = rowbase[B] + 3 * rl;
        const int64_t lb = rowlen[B];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          T* dst = values + bb + b * lb;
          dst[0] = v[u][b];
          dst[1] = v[u][3 + b];
          dst[2] = v[u][6 + b];
        }
      }
    }
  }
}

template <typename T>
__global__ void scatter_second_kernel(const T* __restrict__ nz, int ld_nz, int n_nz, int64_t t0,
                                      const int64_t* __restrict__ list, int64_t n_list,
                                      const int32_t* __restrict__ pairs, const int32_t* __restrict__ gmap, int n_T,
                                      const uint32_t* __restrict__ rank, const int64_t* __restrict__ rowptr,
                                      T* __restrict__ values) {
  for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < n_list; s += int64_t(gridDim.x) * blockDim.x) {
    const int64_t code = list[s];
    const int64_t t = code / n_nz;
    const int m = int(code % n_nz);
    const int64_t tl = t - t0;
    const uint32_t w = rank[code];
    const int A = pairs[2 * m], B = pairs[2 * m + 1];
    const int64_t gA = gmap[t * n_T + A], gB = gmap[t * n_T + B];
    const int ru = int(w & 0xffffu), rl = int((w >> 16) & 0x7fffu);
    T v[9];
#pragma unroll
    for (int ab = 0; ab < 9; ++ab) v[ab] = nz[(9 * tl + ab) * ld_nz + m];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T* dst = values + rowptr[3 * gA + a] + 3 * ru;
      dst[0] += v[3 * a + 0];
      dst[1] += v[3 * a + 1];
      dst[2] += v[3 * a + 2];
    }
    if (A != B) {
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        T* dst = values + rowptr[3 * gB + b] + 3 * rl;
        dst[0] += v[b];
        dst[1] += v[3 + b];
        dst[2] += v[6 + b];
      }
    }
  }
}

template <typename T>
msasm_status scatter_gpu(const msasm_plan* plan, const T* d_nz, int ld_nz, int64_t t0, int64_t n_tiles,
                         const int64_t* d_list, int64_t n_list, T* d_values, cudaStream_t stream) {
  const msasm_tables* tab = plan->tab;
  if (n_tiles > 0) {
    const size_t smem = size_t(tab->topo.n_T) * (sizeof(int64_t) + sizeof(int32_t));
    if (smem > 200 * 1024) return fail(MSASM_EUNSUPPORTED, "reference tile too large for the scatter kernel");
    MSASM_CUDA(cudaFuncSetAttribute(scatter_tile_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    const int64_t chunks = (tab->n_nz + kScatterChunk - 1) / kScatterChunk;
    scatter_tile_kernel<T><<<unsigned(n_tiles * chunks), kScatterThreads, smem, stream>>>(
        d_nz, ld_nz, tab->n_nz, t0, tab->d_pairs, plan->d_gmap, tab->topo.n_T, plan->d_rank, plan->d_rowptr,
        d_values);
    MSASM_CUDA(cudaGetLastError());
  }
  if (n_list > 0) {
    int64_t b2 = (n_list + 255) / 256;
    if (b2 > 152 * 8) b2 = 152 * 8;
    scatter_second_kernel<T><<<unsigned(b2), 256, 0, stream>>>(d_nz, ld_nz, tab->n_nz, t0, d_list, n_list,
                                                               tab->d_pairs, plan->d_gmap, tab->topo.n_T,
                                                               plan->d_rank, plan->d_rowptr, d_values);
    MSASM_CUDA(cudaGetLastError());
  }
  return MSASM_OK;
}

template msasm_status scatter_gpu<double>(const msasm_plan*, const double*, int, int64_t, int64_t, const int64_t*,
                                          int64_t, double*, cudaStream_t);
template msasm_status scatter_gpu<float>(const msasm_plan*, const float*, int, int64_t, int64_t, const int64_t*,
                                         int64_t, float*, cudaStream_t);

}  // namespace msasm
