// K5: step 4 of Sec. 3.2.4 -- the tile blocks of nzdata into the global CSR values.
//
// Pair m = (A, B) of tile t owns the 3x3 block at rows 3 g(A) + a, columns 3 g(B) + b, and
// (A != B) its transpose at rows 3 g(B) + b, columns 3 g(A) + a.  With the rank word
// r_u | r_l << 16 of the plan the upper entry (a, b) lives at rowptr[3 g(A) + a] + 3 r_u + b and
// the lower one at rowptr[3 g(B) + b] + 3 r_l + a.
//
// Staged pass: the rows of the points a tile owns are one contiguous range of values (tile-major
// numbering).  One CTA per chunk of that range builds the chunk in shared memory from the chunk's
// program (the pairs whose upper or lower block lands there, in increasing m, so the nzdata
// loads of neighbouring threads are mostly contiguous), entries no pair of the tile reaches
// staying zero, and streams it out with coalesced 16-byte stores.  Every CSR value is written
// exactly once by the staged pass.
//
// Secondary pass: blocks of tile t landing in rows owned by a lower tile (points on a glued lower
// face) are added to the values the owner wrote; it runs after the staged pass on the same
// stream and each position has at most one such contributor, so no atomics are needed and the
// two-term sums are order independent.
#include <algorithm>
#include <cstdint>

#include "common.h"

namespace msasm {

constexpr int kStagedThreads = 128;
constexpr int kStagedUnroll = 4;

// One CTA per work item (tile, chunk).  The chunk's layout (each point's row offset and length)
// is the same for every tile of the type and its first value index is precomputed per item, so
// a CTA starts gathering after two dependent loads.
template <typename T>
__global__ void __launch_bounds__(kStagedThreads) scatter_staged_kernel(
    const T* __restrict__ nz, int ld_nz, int n_nz, int64_t t0, const int32_t* __restrict__ work,
    const int64_t* __restrict__ work_base, const int32_t* __restrict__ chunk_info,
    const int32_t* __restrict__ chunk_points, const uint32_t* __restrict__ prog, const int32_t* __restrict__ pairs,
    int n_T, const uint32_t* __restrict__ rank, T* __restrict__ values) {
  extern __shared__ __align__(16) uint8_t sm_raw[];
  T* buf = reinterpret_cast<T*>(sm_raw);
  int32_t* off = reinterpret_cast<int32_t*>(sm_raw + kChunkValues * sizeof(T));   // [n_T]
  int32_t* len = off + n_T;                                                        // [n_T]
  const int64_t t = work[2 * blockIdx.x];
  const int c = work[2 * blockIdx.x + 1];
  const int64_t base = work_base[blockIdx.x];
  const int64_t tl = t - t0;
  const int p_begin = chunk_info[4 * c], p_count = chunk_info[4 * c + 1];
  const int q_begin = chunk_info[4 * c + 2], q_count = chunk_info[4 * c + 3];
  const int32_t* cp = chunk_points + 3 * p_begin;
  const int n_vals = cp[3 * (p_count - 1) + 1] + 3 * cp[3 * (p_count - 1) + 2];
  for (int i = threadIdx.x; i < p_count; i += blockDim.x) {
    const int A = cp[3 * i];
    off[A] = cp[3 * i + 1];
    len[A] = cp[3 * i + 2];
  }
  for (int i = threadIdx.x; i < n_vals; i += blockDim.x) buf[i] = T(0);
  __syncthreads();
  const T* nzt = nz + 9 * tl * ld_nz;
  const uint32_t* rk = rank + t * n_nz;
  for (int j0 = threadIdx.x; j0 < q_count; j0 += blockDim.x * kStagedUnroll) {
    uint32_t e[kStagedUnroll], w[kStagedUnroll];
    int2 ab[kStagedUnroll];
    T v[kStagedUnroll][9];
#pragma unroll
    for (int u = 0; u < kStagedUnroll; ++u) {      // issue every load of UNROLL entries first
      const int j = j0 + u * blockDim.x;
      e[u] = (j < q_count) ? prog[q_begin + j] : 0xffffffffu;
      if (e[u] != 0xffffffffu) {
        const int m = int(e[u] & 0x7fffffffu);
        w[u] = rk[m];
        ab[u] = reinterpret_cast<const int2*>(pairs)[m];
#pragma unroll
        for (int k = 0; k < 9; ++k) v[u][k] = nzt[size_t(k) * ld_nz + m];
      }
    }
#pragma unroll
    for (int u = 0; u < kStagedUnroll; ++u) {
      if (e[u] == 0xffffffffu) continue;
      if (!(e[u] >> 31)) {                       // upper block: rows of A
        const int o = off[ab[u].x] + 3 * int(w[u] & 0xffffu), L = len[ab[u].x];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) buf[o + a * L + b] = v[u][3 * a + b];
      } else {                                   // lower block: rows of B
        const int o = off[ab[u].y] + 3 * int((w[u] >> 16) & 0x7fffu), L = len[ab[u].y];
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
          for (int a = 0; a < 3; ++a) buf[o + b * L + a] = v[u][3 * a + b];
      }
    }
  }
  __syncthreads();
  // stream out: head up to 16-byte alignment, 16-byte body, tail
  T* dst = values + base;
  constexpr int VEC = 16 / sizeof(T);
  const int head = int((VEC - (base % VEC)) % VEC);
  const int h = head < n_vals ? head : n_vals;
  for (int i = threadIdx.x; i < h; i += blockDim.x) dst[i] = buf[i];
  const int body = (n_vals - h) / VEC;
  for (int i = threadIdx.x; i < body; i += blockDim.x) {
    float4 v;
    T* pv = reinterpret_cast<T*>(&v);
#pragma unroll
    for (int k = 0; k < VEC; ++k) pv[k] = buf[h + i * VEC + k];
    reinterpret_cast<float4*>(dst + h)[i] = v;
  }
  for (int i = h + body * VEC + threadIdx.x; i < n_vals; i += blockDim.x) dst[i] = buf[i];
}

template <typename T>
__global__ void scatter_secondary_kernel(const T* __restrict__ nz, int ld_nz, int n_nz, int64_t t0,
                                         const int32_t* __restrict__ tile_type, const int64_t* __restrict__ tmpl_ptr,
                                         const uint32_t* __restrict__ tmpl, const int32_t* __restrict__ pairs,
                                         const int32_t* __restrict__ gmap, int n_T, const uint32_t* __restrict__ rank,
                                         const int64_t* __restrict__ rowptr, T* __restrict__ values) {
  const int64_t tl = blockIdx.y, t = t0 + tl;
  const int ty = tile_type[t];
  const int64_t b0 = tmpl_ptr[ty], cnt = tmpl_ptr[ty + 1] - b0;
  const T* nzt = nz + 9 * tl * ld_nz;
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < cnt; j += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t e = tmpl[b0 + j];
    const int m = int(e & 0x3fffffffu);
    const int A = pairs[2 * m], B = pairs[2 * m + 1];
    const int64_t gA = gmap[t * n_T + A], gB = gmap[t * n_T + B];
    const uint32_t w = rank[t * n_nz + m];
    const int ru = int(w & 0xffffu), rl = int((w >> 16) & 0x7fffu);
    T v[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = nzt[size_t(k) * ld_nz + m];
    if (e & (1u << 30)) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        T* dst = values + rowptr[3 * gA + a] + 3 * ru;
        dst[0] += v[3 * a + 0];
        dst[1] += v[3 * a + 1];
        dst[2] += v[3 * a + 2];
      }
    }
    if (e & (1u << 31)) {
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

// steps 4 for tiles [t0, t0 + n_tiles) of the plan, nzdata of those tiles in d_nz
template <typename T>
msasm_status scatter_pass_gpu(const msasm_plan* plan, const T* d_nz, int ld_nz, int64_t t0, int64_t n_tiles,
                              T* d_values, cudaStream_t stream) {
  const msasm_tables* tab = plan->tab;
  const int n_T = tab->topo.n_T;
  if (reinterpret_cast<uintptr_t>(d_values) % 16 != 0)
    return fail(MSASM_EINVAL, "the CSR values buffer must be 16-byte aligned");
  const int64_t w0 = plan->work_ptr[size_t(t0)], w1 = plan->work_ptr[size_t(t0 + n_tiles)];
  if (w1 > w0) {
    const size_t smem = kChunkValues * sizeof(T) + 2 * size_t(n_T) * sizeof(int32_t);
    if (smem > 48 * 1024) return fail(MSASM_EUNSUPPORTED, "reference tile too large for the staged scatter");
    MSASM_CUDA(cudaFuncSetAttribute(scatter_staged_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    scatter_staged_kernel<T><<<unsigned(w1 - w0), kStagedThreads, smem, stream>>>(
        d_nz, ld_nz, tab->n_nz, t0, plan->d_work + 2 * w0, plan->d_work_base + w0, plan->d_chunk_info,
        plan->d_chunk_points, plan->d_prog, tab->d_pairs, n_T, plan->d_rank, d_values);
    MSASM_CUDA(cudaGetLastError());
  }
  if (plan->max_tmpl > 0 && n_tiles > 0) {
    dim3 grid(unsigned(std::max<int64_t>(1, std::min<int64_t>((plan->max_tmpl + 255) / 256, 8))), unsigned(n_tiles));
    scatter_secondary_kernel<T><<<grid, 256, 0, stream>>>(d_nz, ld_nz, tab->n_nz, t0, plan->d_tile_type,
                                                          plan->d_tmpl_ptr, plan->d_tmpl, tab->d_pairs, plan->d_gmap,
                                                          n_T, plan->d_rank, plan->d_rowptr, d_values);
    MSASM_CUDA(cudaGetLastError());
  }
  return MSASM_OK;
}

template msasm_status scatter_pass_gpu<double>(const msasm_plan*, const double*, int, int64_t, int64_t, double*,
                                               cudaStream_t);
template msasm_status scatter_pass_gpu<float>(const msasm_plan*, const float*, int, int64_t, int64_t, float*,
                                              cudaStream_t);

}  // namespace msasm
