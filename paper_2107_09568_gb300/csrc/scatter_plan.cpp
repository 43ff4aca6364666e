// Host part of the staged scatter: chunk programs per tile type.
//
// A tile's type is the pair (lower mask, upper mask) of glued faces; it fixes which of its
// points it owns (those not on a glued lower face) and the row lengths of those points.  The
// owned points of a tile have consecutive global ids, so their CSR rows form one contiguous
// range; it is cut into chunks of at most kChunkValues values.  A chunk's program lists, in
// increasing pair index m, the pairs whose upper block (A owned and in the chunk) or lower block
// (B owned and in the chunk, A != B) lands in the chunk's rows.  Blocks landing in rows owned by
// a lower tile form the type's secondary template, added after the owner has written its rows.
#include <algorithm>
#include <map>
#include <utility>
#include <vector>

#include "common.h"

namespace msasm {

msasm_status build_scatter_plan(msasm_plan* plan, const std::vector<int32_t>& gmap, const std::vector<int64_t>& pptr,
                                ScatterPlanHost& out) {
  const TileTopology& topo = plan->tab->topo;
  const int n_T = topo.n_T, n_nz = plan->tab->n_nz;
  const int64_t nx = plan->n_elem[0], ny = plan->n_elem[1], nz = plan->n_elem[2];
  std::map<std::pair<int, int>, int> type_of_mask;
  out.tile_type.assign(size_t(plan->n_tiles), 0);
  std::vector<int64_t> rep;
  for (int64_t t = 0; t < plan->n_tiles; ++t) {
    const int64_t idx[3] = {t % nx, (t / nx) % ny, t / (nx * ny)};
    const int64_t n[3] = {nx, ny, nz};
    int L = 0, U = 0;
    for (int d = 0; d < 3; ++d) {
      if (idx[d] > 0) L |= 1 << d;
      if (idx[d] + 1 < n[d]) U |= 1 << d;
    }
    auto key = std::make_pair(L, U);
    auto it = type_of_mask.find(key);
    if (it == type_of_mask.end()) {
      it = type_of_mask.emplace(key, int(rep.size())).first;
      rep.push_back(t);
    }
    out.tile_type[size_t(t)] = it->second;
  }
  const int n_types = int(rep.size());
  out.type_chunk_begin.assign(size_t(n_types) + 1, 0);
  out.tmpl_ptr.assign(size_t(n_types) + 1, 0);
  out.chunk_info.clear();
  out.chunk_points.clear();
  out.prog.clear();
  out.tmpl.clear();
  for (int ty = 0; ty < n_types; ++ty) {
    const int64_t t = rep[size_t(ty)];
    const int64_t idx[3] = {t % nx, (t / nx) % ny, t / (nx * ny)};
    std::vector<char> owned(n_T, 1);
    for (int d = 0; d < 3; ++d)
      if (idx[d] > 0)
        for (int A : topo.faces[2 * d]) owned[A] = 0;
    const int32_t* g = &gmap[size_t(t) * n_T];
    std::vector<int> chunk_of(n_T, -1);
    int64_t cur = 0;
    int n_chunks = 0;
    const int base_chunk = int(out.chunk_info.size() / 4);
    std::vector<std::vector<int>> pts;
    for (int A = 0; A < n_T; ++A) {
      if (!owned[A]) continue;
      const int64_t deg = pptr[size_t(g[A]) + 1] - pptr[size_t(g[A])];
      const int64_t vals = 9 * deg;
      if (vals > kChunkValues) return fail(MSASM_EUNSUPPORTED, "a point's rows exceed the scatter chunk size");
      if (n_chunks == 0 || cur + vals > kChunkValues) {
        pts.emplace_back();
        ++n_chunks;
        cur = 0;
      }
      pts.back().push_back(A);
      chunk_of[A] = n_chunks - 1;
      cur += vals;
    }
    std::vector<std::vector<uint32_t>> progs(n_chunks);
    for (int m = 0; m < n_nz; ++m) {
      const int A = topo.pair_A[m], B = topo.pair_B[m];
      if (owned[A]) progs[chunk_of[A]].push_back(uint32_t(m));
      if (A != B && owned[B]) progs[chunk_of[B]].push_back(uint32_t(m) | 0x80000000u);
      uint32_t flags = 0;
      if (!owned[A]) flags |= 1u;                  // upper block into a row owned by a lower tile
      if (A != B && !owned[B]) flags |= 2u;        // lower block likewise
      if (flags) out.tmpl.push_back(uint32_t(m) | (flags << 30));
    }
    for (int c = 0; c < n_chunks; ++c) {
      out.chunk_info.push_back(int32_t(out.chunk_points.size() / 3));
      out.chunk_info.push_back(int32_t(pts[c].size()));
      out.chunk_info.push_back(int32_t(out.prog.size()));
      out.chunk_info.push_back(int32_t(progs[c].size()));
      int32_t off = 0;
      for (int A : pts[c]) {                       // the owned points' rows follow each other
        const int32_t row_len = int32_t(3 * (pptr[size_t(g[A]) + 1] - pptr[size_t(g[A])]));
        out.chunk_points.push_back(A);
        out.chunk_points.push_back(off);
        out.chunk_points.push_back(row_len);
        off += 3 * row_len;
      }
      out.prog.insert(out.prog.end(), progs[c].begin(), progs[c].end());
    }
    out.type_chunk_begin[size_t(ty) + 1] = base_chunk + n_chunks;
    out.tmpl_ptr[size_t(ty) + 1] = int64_t(out.tmpl.size());
  }
  // work items (tile, global chunk id), grouped by tile
  out.work.clear();
  out.work_ptr.assign(size_t(plan->n_tiles) + 1, 0);
  out.max_tmpl = 0;
  for (int ty = 0; ty < n_types; ++ty)
    out.max_tmpl = std::max<int64_t>(out.max_tmpl, out.tmpl_ptr[size_t(ty) + 1] - out.tmpl_ptr[size_t(ty)]);
  out.work_base.clear();
  for (int64_t t = 0; t < plan->n_tiles; ++t) {
    const int ty = out.tile_type[size_t(t)];
    const int32_t* g = &gmap[size_t(t) * n_T];
    for (int c = out.type_chunk_begin[size_t(ty)]; c < out.type_chunk_begin[size_t(ty) + 1]; ++c) {
      // the chunk layout of the type holds for this tile: consecutive global ids, same row lengths
      const int p0 = out.chunk_info[size_t(4 * c)], np = out.chunk_info[size_t(4 * c + 1)];
      const int64_t g0 = g[out.chunk_points[size_t(3 * p0)]];
      for (int i = 0; i < np; ++i) {
        const int32_t* cp = &out.chunk_points[size_t(3 * (p0 + i))];
        const int64_t gi = g[cp[0]];
        if (gi != g0 + i || 3 * (pptr[size_t(gi) + 1] - pptr[size_t(gi)]) != cp[2] ||
            9 * (pptr[size_t(gi)] - pptr[size_t(g0)]) != cp[1])
          return fail(MSASM_EUNSUPPORTED, "tile numbering is not translation invariant within a tile type");
      }
      out.work.push_back(int32_t(t));
      out.work.push_back(int32_t(c));
      out.work_base.push_back(9 * pptr[size_t(g0)]);        // rows 3 g0 .. start at 9 x (entries before g0)
    }
    out.work_ptr[size_t(t) + 1] = int64_t(out.work.size() / 2);
  }
  return MSASM_OK;
}

}  // namespace msasm
