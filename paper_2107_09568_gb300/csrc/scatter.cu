// K5: step 4 of Sec. 3.2.4 -- the tile blocks of nzdata into the global CSR values.
//
// Pair m = (A, B) of tile t owns the 3x3 block at rows 3 g(A) + a, columns 3 g(B) + b, and
// (A != B) its transpose at rows 3 g(B) + b, columns 3 g(A) + a.  With the rank word
// r_u | r_l << 16 of the plan the upper entry (a, b) lives at rowptr[3 g(A) + a] + 3 r_u + b and
// the lower one at rowptr[3 g(B) + b] + 3 r_l + a.
//
// nzdata holds the tile blocks of eq. 58 block by block: nz[t][m][3a + b], so the nine values of
// pair m of tile t are one contiguous 9-value run at 9 (t ld + m).
//
// Direct pass: the rows of the points a tile owns are one contiguous range of values, laid out
// the same way for every tile of its type.  The type's value map (built once per plan from its
// representative tile) holds for every value of the range its source in the tile's nzdata,
// 9 m + 3a + b, or -1 where no block of the tile lands; each thread writes consecutive values
// of the range (coalesced stores) from gathers that the tile's nzdata, read by the CTAs working
// on the tile at the same time, serves mostly from L2.  Every CSR value is written exactly once.
//
// Secondary pass: blocks of tile t landing in rows owned by a lower tile (points on a glued lower
// face) are added to the values the owner wrote; it runs after the direct pass on the same
// stream and each position has at most one such contributor, so no atomics are needed and the
// two-term sums are order independent.
//
// Both passes write into a window [v_lo, v_hi) of the global values (values[0] is value v_lo):
// the whole array for a full assembly, or the rows owned by a range of tiles when one mesh is
// split across GPUs (the direct pass then covers the range's tiles and the secondary pass also
// the halo tiles above it, whose blocks land partly in the window).
#include <algorithm>
#include <cstdint>

#include "common.h"

namespace msasm {

constexpr int kDirectThreads = 256;
constexpr int kDirectPerThread = kScatterSegment / kDirectThreads;   // 16
constexpr int kDirectRun64 = 2, kDirectRun32 = 4;                    // tiles per CTA (FP64, FP32 values)

// A CTA takes chunk s (values [4096 s, 4096 s + 4096) of a tile's owned range) of R consecutive
// tiles, tile order first: the CTAs the hardware keeps resident work on a few consecutive tiles,
// whose nzdata stays in L2 for the gathers of both the upper and the lower blocks.  Tiles of one
// type share the chunk's value map, so the map entries stay in registers from one tile to the
// next (reloaded only where the type changes): the map loads, one per value for one tile, are
// one per R values.  Each thread owns values i = u * 256 + threadIdx.x of the chunk (a warp's
// loads and stores cover 32 consecutive values); every gather of a tile is issued before its
// first store.
template <typename T, int R>
__global__ void __launch_bounds__(kDirectThreads, sizeof(T) == 8 ? (R > 1 ? 4 : 5) : 8) scatter_direct_kernel(
    const T* __restrict__ nz, int ld_nz, int64_t t0, int64_t ta, int64_t tb, int n_chunks,
    const int32_t* __restrict__ tile_type, const int64_t* __restrict__ tile_vbase,
    const int64_t* __restrict__ type_map_off, const int32_t* __restrict__ type_nvals,
    const int32_t* __restrict__ maps, T* __restrict__ values, int64_t v_lo) {
  const int tid = int(threadIdx.x);
  const int64_t t_first = ta + int64_t(blockIdx.x / unsigned(n_chunks)) * R;
  const int s0 = int(blockIdx.x % unsigned(n_chunks)) * kScatterSegment;
  int k[kDirectPerThread];
  int loaded = -1;                                // the type whose map chunk k holds (CTA-uniform)
#pragma unroll 1
  for (int r = 0; r < R; ++r) {
    const int64_t t = t_first + r;
    if (t >= tb) break;
    const int ty = tile_type[t];
    const int count = type_nvals[ty] - s0;        // values of this chunk (<= 0: none for this type)
    if (count <= 0) continue;
    if (ty != loaded) {
      const int32_t* map = maps + type_map_off[ty] + s0;
#pragma unroll
      for (int u = 0; u < kDirectPerThread; ++u) {
        const int i = u * kDirectThreads + tid;
        k[u] = (i < count) ? map[i] : -2;         // -1: no block of the tile lands here (value 0)
      }
      loaded = ty;
    }
    const T* nzt = nz + 9 * (t - t0) * ld_nz;
    T v[kDirectPerThread];
#pragma unroll
    for (int u = 0; u < kDirectPerThread; ++u) v[u] = (k[u] >= 0) ? __ldg(nzt + k[u]) : T(0);
    asm volatile("" ::: "memory");                // every gather is issued before the first store
    T* out = values + (tile_vbase[t] + s0 - v_lo);
    // streaming stores: the values are not read again here, so they should not push the tile's
    // nzdata (gathered twice) and the type maps out of L2
#pragma unroll
    for (int u = 0; u < kDirectPerThread; ++u)
      if (k[u] != -2) __stcs(out + u * kDirectThreads + tid, v[u]);
  }
}

// Value maps of all types from their representative tiles (maps preset to -1).
__global__ void type_maps_kernel(const int64_t* __restrict__ type_rep, int n_types, const int64_t* __restrict__ map_off,
                                 const int32_t* __restrict__ type_nvals, const int32_t* __restrict__ pairs,
                                 const int32_t* __restrict__ gmap, int n_T, int n_nz, int ld_nz,
                                 const uint32_t* __restrict__ rank, const int64_t* __restrict__ rowptr,
                                 const int64_t* __restrict__ tile_vbase, int32_t* __restrict__ maps) {
  const int64_t total = int64_t(n_types) * n_nz;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int ty = int(i / n_nz), m = int(i % n_nz);
    const int64_t t = type_rep[ty];
    const int64_t vb = tile_vbase[t], nv = type_nvals[ty];
    int32_t* map = maps + map_off[ty];
    const int A = pairs[2 * m], B = pairs[2 * m + 1];
    const int64_t gA = gmap[t * n_T + A], gB = gmap[t * n_T + B];
    const uint32_t w = rank[t * n_nz + m];
    const int64_t rA = rowptr[3 * gA] - vb, rB = rowptr[3 * gB] - vb;
    if (rA >= 0 && rA < nv) {                      // A owned: upper block in the rows of A
      const int64_t L = rowptr[3 * gA + 1] - rowptr[3 * gA];
      const int64_t o = rA + 3 * int64_t(w & 0xffffu);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) map[o + a * L + b] = int32_t(9 * m + 3 * a + b);
    }
    if (A != B && rB >= 0 && rB < nv) {            // B owned: lower block in the rows of B
      const int64_t L = rowptr[3 * gB + 1] - rowptr[3 * gB];
      const int64_t o = rB + 3 * int64_t((w >> 16) & 0x7fffu);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) map[o + b * L + a] = int32_t(9 * m + 3 * a + b);
    }
  }
}

// Every tile of a type places its blocks where the representative does (same column ranks).
__global__ void rank_invariance_kernel(const int32_t* __restrict__ tile_type, const int64_t* __restrict__ type_rep,
                                       int64_t n_tiles, int n_nz, const uint32_t* __restrict__ rank,
                                       unsigned long long* __restrict__ bad) {
  const int64_t total = n_tiles * n_nz;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t t = i / n_nz;
    const int m = int(i % n_nz);
    const int64_t r = type_rep[tile_type[t]];
    if ((rank[i] & 0x7fffffffu) != (rank[r * n_nz + m] & 0x7fffffffu)) atomicAdd(bad, 1ull);
  }
}

msasm_status scatter_maps_gpu(msasm_plan* plan, const int64_t* d_type_rep, int n_types, unsigned long long* d_bad,
                              cudaStream_t stream) {
  const msasm_tables* tab = plan->tab;
  const int ld = ld_nz_of(tab->n_nz);
  if (int64_t(9) * ld >= (int64_t(1) << 31)) return fail(MSASM_EUNSUPPORTED, "table too large for the value maps");
  type_maps_kernel<<<152 * 4, 256, 0, stream>>>(d_type_rep, n_types, plan->d_type_map_off, plan->d_type_nvals,
                                                tab->d_pairs, plan->d_gmap, tab->topo.n_T, tab->n_nz, ld, plan->d_rank,
                                                plan->d_rowptr, plan->d_tile_vbase, plan->d_maps);
  MSASM_CUDA(cudaGetLastError());
  rank_invariance_kernel<<<152 * 8, 256, 0, stream>>>(plan->d_tile_type, d_type_rep, plan->n_tiles, tab->n_nz,
                                                      plan->d_rank, d_bad);
  MSASM_CUDA(cudaGetLastError());
  return MSASM_OK;
}

// Secondary entries of all tiles, built once per plan: entry i of tile t (template entry j of
// its type) gets its nzdata column m, flags and the first value index and row length of each
// block it adds (upper: rows of A, lower: rows of B).
__global__ void secondary_entries_kernel(const int32_t* __restrict__ tile_type, const int64_t* __restrict__ sec_off,
                                         int64_t n_tiles, const int64_t* __restrict__ tmpl_ptr,
                                         const uint32_t* __restrict__ tmpl, const int32_t* __restrict__ pairs,
                                         const int32_t* __restrict__ gmap, int n_T, int n_nz,
                                         const uint32_t* __restrict__ rank, const int64_t* __restrict__ rowptr,
                                         SecondaryEntry* __restrict__ out) {
  const int64_t total = sec_off[n_tiles];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    int64_t lo = 0, hi = n_tiles;                  // tile t with sec_off[t] <= i < sec_off[t + 1]
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) / 2;
      if (sec_off[mid] <= i) lo = mid; else hi = mid;
    }
    const int64_t t = lo;
    const uint32_t e = tmpl[tmpl_ptr[tile_type[t]] + (i - sec_off[t])];
    const int m = int(e & 0x3fffffffu);
    const int A = pairs[2 * m], B = pairs[2 * m + 1];
    const int64_t gA = gmap[t * n_T + A], gB = gmap[t * n_T + B];
    const uint32_t w = rank[t * n_nz + m];
    SecondaryEntry r;
    r.dst_u = rowptr[3 * gA] + 3 * int64_t(w & 0xffffu);
    r.dst_l = rowptr[3 * gB] + 3 * int64_t((w >> 16) & 0x7fffu);
    r.len_u = int32_t(rowptr[3 * gA + 1] - rowptr[3 * gA]);
    r.len_l = int32_t(rowptr[3 * gB + 1] - rowptr[3 * gB]);
    r.tile = int32_t(t);
    r.m_flags = e;
    out[i] = r;
  }
}

msasm_status secondary_entries_gpu(msasm_plan* plan, cudaStream_t stream) {
  const int64_t total = plan->sec_off_host.back();
  if (total == 0) return MSASM_OK;
  secondary_entries_kernel<<<152 * 8, 256, 0, stream>>>(plan->d_tile_type, plan->d_sec_off, plan->n_tiles,
                                                        plan->d_tmpl_ptr, plan->d_tmpl, plan->tab->d_pairs,
                                                        plan->d_gmap, plan->tab->topo.n_T, plan->tab->n_nz,
                                                        plan->d_rank, plan->d_rowptr, plan->d_sec);
  MSASM_CUDA(cudaGetLastError());
  return MSASM_OK;
}

// Secondary pass over the entries of tiles [t0, t0 + n_tiles): add each block to the values the
// owner of its rows wrote.  The (up to) 18 destinations of an entry are distinct values (three rows
// of A and three of B), and no other entry adds to them, so all their loads are issued before the
// first store: one round trip for the read-modify-write instead of one per value.
template <typename T>
__global__ void scatter_secondary_kernel(const T* __restrict__ nz, int ld_nz, int64_t t0, int64_t e0, int64_t e1,
                                         const SecondaryEntry* __restrict__ sec, T* __restrict__ values, int64_t v_lo,
                                         int64_t v_hi) {
  for (int64_t i = e0 + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < e1; i += int64_t(gridDim.x) * blockDim.x) {
    const SecondaryEntry r = sec[i];
    const int m = int(r.m_flags & 0x3fffffffu);
    const T* src = nz + 9 * ((int64_t(r.tile) - t0) * ld_nz + m);   // the block's contiguous run
    // the three rows of a point belong to one owner: the first row decides whether a block is in the window
    const bool up = (r.m_flags & (1u << 30)) && r.dst_u >= v_lo && r.dst_u < v_hi;
    const bool lo = (r.m_flags & (1u << 31)) && r.dst_l >= v_lo && r.dst_l < v_hi;
    T* du = values + (r.dst_u - v_lo);
    T* dl = values + (r.dst_l - v_lo);
    T v[9], wu[9], wl[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = __ldg(src + k);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        wu[3 * a + c] = up ? du[int64_t(a) * r.len_u + c] : T(0);
        wl[3 * a + c] = lo ? dl[int64_t(a) * r.len_l + c] : T(0);
      }
    asm volatile("" ::: "memory");                // every load is issued before the first store
    if (up) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) du[int64_t(a) * r.len_u + c] = wu[3 * a + c] + v[3 * a + c];   // block (a, c)
    }
    if (lo) {
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) dl[int64_t(b) * r.len_l + c] = wl[3 * b + c] + v[3 * c + b];   // transpose
    }
  }
}

// step 4 for tiles [t0, t0 + n_tiles) of the plan, nzdata of those tiles in d_nz: the direct pass
// for the tiles below direct_end, the secondary pass for all of them, into the value window
// [v_lo, v_hi) (d_values holds value v_lo first)
template <typename T>
msasm_status scatter_pass_gpu(const msasm_plan* plan, const T* d_nz, int ld_nz, int64_t t0, int64_t n_tiles,
                              T* d_values, int64_t direct_end, int64_t v_lo, int64_t v_hi, cudaStream_t stream) {
  const int64_t td = std::max(t0, std::min(t0 + n_tiles, direct_end));
  // chunks of the largest type: CTAs of chunks a tile's type does not have return at once
  int n_chunks = 1;
  for (size_t ty = 0; ty + 1 < plan->type_map_off_host.size(); ++ty) {
    const int64_t nv = plan->type_map_off_host[ty + 1] - plan->type_map_off_host[ty];
    n_chunks = std::max<int>(n_chunks, int((nv + kScatterSegment - 1) / kScatterSegment));
  }
  auto direct = [&](int64_t ta, int64_t tb) -> msasm_status {
    if (tb <= ta) return MSASM_OK;
    constexpr int R = sizeof(T) == 8 ? kDirectRun64 : kDirectRun32;
    const int64_t grid = (tb - ta + R - 1) / R * n_chunks;
    if (grid > 2147483647LL) return fail(MSASM_EUNSUPPORTED, "too many scatter chunks for one launch");
    scatter_direct_kernel<T, R><<<unsigned(grid), kDirectThreads, 0, stream>>>(
        d_nz, ld_nz, t0, ta, tb, n_chunks, plan->d_tile_type, plan->d_tile_vbase, plan->d_type_map_off,
        plan->d_type_nvals, plan->d_maps, d_values, v_lo);
    MSASM_CUDA(cudaGetLastError());
    return MSASM_OK;
  };
  auto secondary = [&](int64_t ta, int64_t tb, cudaStream_t s) -> msasm_status {
    const int64_t e0 = plan->sec_off_host[size_t(ta)], e1 = plan->sec_off_host[size_t(tb)];
    if (e1 <= e0) return MSASM_OK;
    const int64_t blocks = std::min<int64_t>((e1 - e0 + 255) / 256, 152 * 16);
    scatter_secondary_kernel<T><<<unsigned(blocks), 256, 0, s>>>(d_nz, ld_nz, t0, e0, e1, plan->d_sec, d_values, v_lo,
                                                                 v_hi);
    MSASM_CUDA(cudaGetLastError());
    return MSASM_OK;
  };
  const bool overlap = plan->scatter_side != nullptr && td - t0 >= int64_t(kScatterPieces) * 64 &&
                       plan->sec_off_host[size_t(t0 + n_tiles)] > plan->sec_off_host[size_t(t0)];
  if (!overlap) {
    MSASM_TRY(direct(t0, td));
    return secondary(t0, t0 + n_tiles, stream);
  }
  // The direct pass in pieces of consecutive tiles on the caller's stream; the secondary entries of a
  // piece's tiles add to rows of those or lower tiles, all written once the piece is done, while the
  // next pieces write rows of higher tiles only: so each piece's secondary pass runs on a second
  // stream beside the next piece's direct pass (each value has at most one secondary contribution,
  // so the secondary launches never touch the same value).
  int64_t prev = t0;
  for (int k = 0; k < kScatterPieces; ++k) {
    const int64_t b = t0 + (td - t0) * (k + 1) / kScatterPieces;
    MSASM_TRY(direct(prev, b));
    MSASM_CUDA(cudaEventRecord(plan->scatter_ev[k], stream));
    MSASM_CUDA(cudaStreamWaitEvent(plan->scatter_side, plan->scatter_ev[k], 0));
    MSASM_TRY(secondary(prev, b, plan->scatter_side));
    prev = b;
  }
  MSASM_TRY(secondary(td, t0 + n_tiles, plan->scatter_side));   // halo tiles above a range
  MSASM_CUDA(cudaEventRecord(plan->scatter_ev[kScatterPieces], plan->scatter_side));
  MSASM_CUDA(cudaStreamWaitEvent(stream, plan->scatter_ev[kScatterPieces], 0));   // joined before return
  return MSASM_OK;
}

template <typename T>
msasm_status scatter_pass_gpu(const msasm_plan* plan, const T* d_nz, int ld_nz, int64_t t0, int64_t n_tiles,
                              T* d_values, cudaStream_t stream) {
  return scatter_pass_gpu<T>(plan, d_nz, ld_nz, t0, n_tiles, d_values, t0 + n_tiles, 0, plan->nnz, stream);
}

template msasm_status scatter_pass_gpu<double>(const msasm_plan*, const double*, int, int64_t, int64_t, double*,
                                               cudaStream_t);
template msasm_status scatter_pass_gpu<float>(const msasm_plan*, const float*, int, int64_t, int64_t, float*,
                                              cudaStream_t);
template msasm_status scatter_pass_gpu<double>(const msasm_plan*, const double*, int, int64_t, int64_t, double*,
                                               int64_t, int64_t, int64_t, cudaStream_t);
template msasm_status scatter_pass_gpu<float>(const msasm_plan*, const float*, int, int64_t, int64_t, float*, int64_t,
                                              int64_t, int64_t, cudaStream_t);

}  // namespace msasm
