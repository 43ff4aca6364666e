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

template <typename T>
__global__ void scatter_kernel(const T* __restrict__ nz, int ld_nz, int n_nz, int64_t t0, int64_t n_tiles,
                               const int32_t* __restrict__ pairs, const int32_t* __restrict__ gmap, int n_T,
                               const uint32_t* __restrict__ rank, const int64_t* __restrict__ rowptr,
                               T* __restrict__ values) {
  const int64_t total = n_tiles * n_nz;
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int64_t tl = idx / n_nz;
    const int m = int(idx % n_nz);
    const int64_t t = t0 + tl;
    const uint32_t w = rank[t * n_nz + m];
    if (w >> 31) continue;
    const int A = pairs[2 * m], B = pairs[2 * m + 1];
    const int64_t gA = gmap[t * n_T + A], gB = gmap[t * n_T + B];
    const int ru = int(w & 0xffffu), rl = int((w >> 16) & 0x7fffu);
    T v[9];
#pragma unroll
    for (int ab = 0; ab < 9; ++ab) v[ab] = nz[(9 * tl + ab) * ld_nz + m];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T* dst = values + rowptr[3 * gA + a] + 3 * ru;
      dst[0] = v[3 * a + 0];
      dst[1] = v[3 * a + 1];
      dst[2] = v[3 * a + 2];
    }
    if (A != B) {
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        T* dst = values + rowptr[3 * gB + b] + 3 * rl;
        dst[0] = v[b];
        dst[1] = v[3 + b];
        dst[2] = v[6 + b];
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
  int64_t total = n_tiles * tab->n_nz;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks > 0) {
    scatter_kernel<T><<<unsigned(blocks), 256, 0, stream>>>(d_nz, ld_nz, tab->n_nz, t0, n_tiles, tab->d_pairs,
                                                            plan->d_gmap, tab->topo.n_T, plan->d_rank,
                                                            plan->d_rowptr, d_values);
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
