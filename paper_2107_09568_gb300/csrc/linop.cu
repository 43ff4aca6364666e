// Matrix-free product y = K u (Sec. 4.2, eq. 74): the tile matrices are formed on the fly from the
// lookup table and the projection coefficients (the contraction of eq. 58, in any precision form)
// and applied to u without storing the global CSR values.
//
// Direct part: the rows a tile owns are laid out the same way for every tile of its type (the
// layout of the CSR pattern); per type, the value map gives each entry's source in the tile's nzdata
// and the column map its column point and component.  One warp per owned row sums
// nz[source] u[3 g(column point) + beta] over the row and writes y once.
// Glued faces: the blocks of tile t landing in rows owned by a lower tile (the secondary entries of
// the scatter) are applied afterwards and added with FP64 atomics (several per face row, so the last
// bits of those rows depend on the order of the additions).
#include <algorithm>

#include "common.h"

namespace msasm {

// column maps of all types from their representatives (layout of the value maps, preset to -1)
__global__ void type_colmaps_kernel(const int64_t* __restrict__ type_rep, int n_types,
                                    const int64_t* __restrict__ map_off, const int32_t* __restrict__ type_nvals,
                                    const int32_t* __restrict__ pairs, const int32_t* __restrict__ gmap, int n_T,
                                    int n_nz, const uint32_t* __restrict__ rank, const int64_t* __restrict__ rowptr,
                                    const int64_t* __restrict__ tile_vbase, int32_t* __restrict__ colmaps) {
  const int64_t total = int64_t(n_types) * n_nz;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int ty = int(i / n_nz), m = int(i % n_nz);
    const int64_t t = type_rep[ty];
    const int64_t vb = tile_vbase[t], nv = type_nvals[ty];
    int32_t* cm = colmaps + map_off[ty];
    const int A = pairs[2 * m], B = pairs[2 * m + 1];
    const int64_t gA = gmap[t * n_T + A], gB = gmap[t * n_T + B];
    const uint32_t w = rank[t * n_nz + m];
    const int64_t rA = rowptr[3 * gA] - vb, rB = rowptr[3 * gB] - vb;
    if (rA >= 0 && rA < nv) {                      // upper block in the rows of A: columns (B, b)
      const int64_t L = rowptr[3 * gA + 1] - rowptr[3 * gA];
      const int64_t o = rA + 3 * int64_t(w & 0xffffu);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) cm[o + a * L + b] = (B << 2) | b;
    }
    if (A != B && rB >= 0 && rB < nv) {            // lower block in the rows of B: columns (A, a)
      const int64_t L = rowptr[3 * gB + 1] - rowptr[3 * gB];
      const int64_t o = rB + 3 * int64_t((w >> 16) & 0x7fffu);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) cm[o + b * L + a] = (A << 2) | a;
    }
  }
}

constexpr int kLinopWarps = 8;

template <typename T>
__global__ void __launch_bounds__(32 * kLinopWarps) linop_direct_kernel(
    const T* __restrict__ nz, int ld_nz, int64_t t0, int64_t n_tiles, const int32_t* __restrict__ tile_type,
    const int64_t* __restrict__ type_map_off, const int32_t* __restrict__ maps, const int32_t* __restrict__ colmaps,
    const int64_t* __restrict__ type_row_off, const int32_t* __restrict__ type_rows, const int32_t* __restrict__ gmap,
    int n_T, const double* __restrict__ u, double* __restrict__ y, int64_t row_blocks) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // the row blocks of one tile are consecutive blocks: the CTAs in flight share a few tiles'
  // nzdata in L2 (tile-fastest order would touch every tile's nzdata at once and re-read it)
  const int64_t tl = int64_t(blockIdx.x) / row_blocks;
  if (tl >= n_tiles) return;
  const int64_t t = t0 + tl;
  const int ty = tile_type[t];
  const int64_t r0 = type_row_off[ty], nr = type_row_off[ty + 1] - r0;
  const int64_t r = (int64_t(blockIdx.x) - tl * row_blocks) * kLinopWarps + warp;
  if (r >= nr) return;
  const int32_t* row = type_rows + 3 * (r0 + r);
  const int off = row[0], len = row[1], code = row[2];
  const int32_t* map = maps + type_map_off[ty] + off;
  const int32_t* cm = colmaps + type_map_off[ty] + off;
  const T* nzt = nz + 9 * tl * ld_nz;
  const int32_t* gt = gmap + t * n_T;
  double s = 0.0;
  for (int i = lane; i < len; i += 32) {
    const int k = map[i];
    if (k >= 0) {
      const int c = cm[i];
      s = fma(double(nzt[k]), u[3 * int64_t(gt[c >> 2]) + (c & 3)], s);
    }
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[3 * int64_t(gt[code >> 2]) + (code & 3)] = s;
}

template <typename T>
__global__ void linop_secondary_kernel(const T* __restrict__ nz, int ld_nz, int64_t t0, int64_t e0, int64_t e1,
                                       const SecondaryEntry* __restrict__ sec, const int32_t* __restrict__ pairs,
                                       const int32_t* __restrict__ gmap, int n_T, const double* __restrict__ u,
                                       double* __restrict__ y) {
  for (int64_t i = e0 + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < e1; i += int64_t(gridDim.x) * blockDim.x) {
    const SecondaryEntry r = sec[i];
    const int m = int(r.m_flags & 0x3fffffffu);
    const int64_t t = r.tile;
    const T* src = nz + 9 * ((t - t0) * ld_nz + m);     // the tile block of pair m (9 values)
    double v[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = double(src[k]);
    const int64_t gA = gmap[t * n_T + pairs[2 * m]], gB = gmap[t * n_T + pairs[2 * m + 1]];
    if (r.m_flags & (1u << 30)) {                  // rows of A: sum_b blk[a][b] u_B,b
      const double u0 = u[3 * gB], u1 = u[3 * gB + 1], u2 = u[3 * gB + 2];
#pragma unroll
      for (int a = 0; a < 3; ++a) atomicAdd(y + 3 * gA + a, v[3 * a] * u0 + v[3 * a + 1] * u1 + v[3 * a + 2] * u2);
    }
    if (r.m_flags & (1u << 31)) {                  // rows of B: sum_a blk[a][b] u_A,a
      const double u0 = u[3 * gA], u1 = u[3 * gA + 1], u2 = u[3 * gA + 2];
#pragma unroll
      for (int b = 0; b < 3; ++b) atomicAdd(y + 3 * gB + b, v[b] * u0 + v[3 + b] * u1 + v[6 + b] * u2);
    }
  }
}

msasm_status linop_prepare_gpu(msasm_plan* plan, cudaStream_t s) {
  if (plan->d_colmaps) return MSASM_OK;
  const msasm_tables* tab = plan->tab;
  const int n_types = int(plan->type_rep_host.size());
  const size_t nmap = size_t(plan->type_map_off_host.back());
  int64_t* d_rep = nullptr;
  MSASM_CUDA(cudaMalloc(&plan->d_colmaps, std::max<size_t>(nmap, 1) * sizeof(int32_t)));
  MSASM_CUDA(cudaMalloc(&plan->d_type_rows, std::max<size_t>(plan->type_rows_host.size(), 1) * sizeof(int32_t)));
  MSASM_CUDA(cudaMalloc(&plan->d_type_row_off, plan->type_row_off_host.size() * sizeof(int64_t)));
  MSASM_CUDA(cudaMallocAsync(&d_rep, size_t(n_types) * sizeof(int64_t), s));
  MSASM_CUDA(cudaMemcpyAsync(plan->d_type_rows, plan->type_rows_host.data(),
                             plan->type_rows_host.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  MSASM_CUDA(cudaMemcpyAsync(plan->d_type_row_off, plan->type_row_off_host.data(),
                             plan->type_row_off_host.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  MSASM_CUDA(cudaMemcpyAsync(d_rep, plan->type_rep_host.data(), size_t(n_types) * sizeof(int64_t),
                             cudaMemcpyHostToDevice, s));
  MSASM_CUDA(cudaMemsetAsync(plan->d_colmaps, 0xff, nmap * sizeof(int32_t), s));
  type_colmaps_kernel<<<152 * 4, 256, 0, s>>>(d_rep, n_types, plan->d_type_map_off, plan->d_type_nvals, tab->d_pairs,
                                              plan->d_gmap, tab->topo.n_T, tab->n_nz, plan->d_rank, plan->d_rowptr,
                                              plan->d_tile_vbase, plan->d_colmaps);
  MSASM_CUDA(cudaGetLastError());
  MSASM_CUDA(cudaFreeAsync(d_rep, s));
  MSASM_CUDA(cudaStreamSynchronize(s));          // the host vectors outlive the copies
  return MSASM_OK;
}

// y (+)= K u for tiles [t0, t0 + n_tiles): direct rows of those tiles, then their face blocks
template <typename T>
msasm_status linop_pass_gpu(const msasm_plan* plan, const T* d_nz, int ld_nz, int64_t t0, int64_t n_tiles,
                            const double* d_u, double* d_y, cudaStream_t s) {
  if (n_tiles <= 0) return MSASM_OK;
  const int64_t ry = (plan->max_type_rows + kLinopWarps - 1) / kLinopWarps;
  if (ry < 1 || n_tiles * ry > 2147483647LL) return fail(MSASM_EUNSUPPORTED, "too many tiles or rows per tile");
  linop_direct_kernel<T><<<static_cast<unsigned>(n_tiles * ry), 32 * kLinopWarps, 0, s>>>(
      d_nz, ld_nz, t0, n_tiles, plan->d_tile_type, plan->d_type_map_off, plan->d_maps, plan->d_colmaps,
      plan->d_type_row_off, plan->d_type_rows, plan->d_gmap, plan->tab->topo.n_T, d_u, d_y, ry);
  MSASM_CUDA(cudaGetLastError());
  const int64_t e0 = plan->sec_off_host[size_t(t0)], e1 = plan->sec_off_host[size_t(t0 + n_tiles)];
  if (e1 > e0) {
    const int64_t blocks = std::min<int64_t>((e1 - e0 + 255) / 256, 152 * 16);
    linop_secondary_kernel<T><<<unsigned(blocks), 256, 0, s>>>(d_nz, ld_nz, t0, e0, e1, plan->d_sec,
                                                              plan->tab->d_pairs, plan->d_gmap, plan->tab->topo.n_T,
                                                              d_u, d_y);
    MSASM_CUDA(cudaGetLastError());
  }
  return MSASM_OK;
}
template msasm_status linop_pass_gpu<double>(const msasm_plan*, const double*, int, int64_t, int64_t, const double*,
                                             double*, cudaStream_t);
template msasm_status linop_pass_gpu<float>(const msasm_plan*, const float*, int, int64_t, int64_t, const double*,
                                            double*, cudaStream_t);

}  // namespace msasm
