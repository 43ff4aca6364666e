// K6: integer structure of the global stiffness (once per mesh; bit-exact).
//
// The host numbers the global control points and builds the point-level pattern
// (pptr, pcol).  On the GPU the pattern is expanded to the 3x3-block DOF pattern
// (row 3g+alpha holds columns 3h+beta for every neighbour h of g, ascending), and
// every (tile, pair) gets its rank word: the position of g(B) among the
// neighbours of g(A) (upper block), the position of g(A) among those of g(B)
// (lower block), and whether the tile is the second contributor of an entry it
// shares with a lower-indexed tile.
#include "common.h"

namespace msasm {

__global__ void csr_rowptr_kernel(const int64_t* __restrict__ pptr, int64_t n_points, int64_t* __restrict__ rowptr) {
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r <= 3 * n_points;
       r += int64_t(gridDim.x) * blockDim.x) {
    if (r == 3 * n_points) {
      rowptr[r] = 9 * pptr[n_points];
    } else {
      int64_t g = r / 3, a = r % 3;
      int64_t deg = pptr[g + 1] - pptr[g];
      rowptr[r] = 9 * pptr[g] + 3 * a * deg;
    }
  }
}

// One warp per point: row 3g+alpha, entry 3k+beta holds column 3*pcol[pptr[g]+k] + beta.
__global__ void csr_col_kernel(const int64_t* __restrict__ pptr, const int32_t* __restrict__ pcol,
                               int64_t n_points, int32_t* __restrict__ col) {
  const int lane = threadIdx.x & 31;
  for (int64_t g = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; g < n_points;
       g += (int64_t(gridDim.x) * blockDim.x) >> 5) {
    int64_t p0 = pptr[g], deg = pptr[g + 1] - p0;
    int64_t base = 9 * p0;
    for (int64_t e = lane; e < 3 * deg; e += 32) {
      int64_t k = e / 3, b = e % 3;
      int32_t c = 3 * pcol[p0 + k] + int32_t(b);
      col[base + e] = c;
      col[base + 3 * deg + e] = c;
      col[base + 6 * deg + e] = c;
    }
  }
}

__device__ inline int lower_bound_i32(const int32_t* __restrict__ a, int n, int32_t key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void rank_map_kernel(const int32_t* __restrict__ gmap, const int32_t* __restrict__ pairs,
                                const uint8_t* __restrict__ pair_face, const int64_t* __restrict__ pptr,
                                const int32_t* __restrict__ pcol, int64_t n_tiles, int n_T, int n_nz,
                                int nx, int ny, uint32_t* __restrict__ rank, unsigned long long* __restrict__ bad) {
  const int64_t total = n_tiles * n_nz;
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += int64_t(gridDim.x) * blockDim.x) {
    int64_t t = idx / n_nz;
    int m = int(idx % n_nz);
    int A = pairs[2 * m], B = pairs[2 * m + 1];
    int32_t gA = gmap[t * n_T + A], gB = gmap[t * n_T + B];
    int64_t pa = pptr[gA], pb = pptr[gB];
    int da = int(pptr[gA + 1] - pa), db = int(pptr[gB + 1] - pb);
    int ru = lower_bound_i32(pcol + pa, da, gB);
    int rl = lower_bound_i32(pcol + pb, db, gA);
    if (ru >= da || pcol[pa + ru] != gB || rl >= db || pcol[pb + rl] != gA) atomicAdd(bad, 1ull);
    int ix = int(t % nx), iy = int((t / nx) % ny), iz = int(t / (int64_t(nx) * ny));
    uint32_t lower = (ix > 0 ? 1u : 0u) | (iy > 0 ? 2u : 0u) | (iz > 0 ? 4u : 0u);
    uint32_t second = (pair_face[m] & lower) ? 1u : 0u;
    rank[idx] = uint32_t(ru) | (uint32_t(rl) << 16) | (second << 31);
  }
}

msasm_status structure_expand_gpu(int64_t n_points, const int64_t* d_pptr, const int32_t* d_pcol,
                                  int64_t* d_rowptr, int32_t* d_col, cudaStream_t stream) {
  csr_rowptr_kernel<<<152 * 4, 256, 0, stream>>>(d_pptr, n_points, d_rowptr);
  MSASM_CUDA(cudaGetLastError());
  csr_col_kernel<<<152 * 8, 256, 0, stream>>>(d_pptr, d_pcol, n_points, d_col);
  MSASM_CUDA(cudaGetLastError());
  return MSASM_OK;
}

msasm_status rank_map_gpu(const int32_t* d_gmap, const int32_t* d_pairs, const uint8_t* d_pair_face,
                          const int64_t* d_pptr, const int32_t* d_pcol, int64_t n_tiles, int n_T, int n_nz,
                          int nx, int ny, uint32_t* d_rank, unsigned long long* d_bad, cudaStream_t stream) {
  rank_map_kernel<<<152 * 8, 256, 0, stream>>>(d_gmap, d_pairs, d_pair_face, d_pptr, d_pcol, n_tiles, n_T, n_nz,
                                               nx, ny, d_rank, d_bad);
  MSASM_CUDA(cudaGetLastError());
  return MSASM_OK;
}

}  // namespace msasm
