// Host part of the scatter plan.
//
// A tile's type is the pair (lower mask, upper mask) of glued faces; it fixes which of its
// points it owns (those not on a glued lower face) and the row lengths of those points.  The
// owned points of a tile have consecutive global ids (tile-major numbering), so their CSR rows
// form one contiguous range of values, laid out the same way for every tile of the type: one
// value map per type (built on the GPU from the type's representative tile) gives the source
// of every value of the range.  The direct pass cuts the range into chunks of kScatterSegment
// values; a chunk's map serves every tile of the type.
// Blocks landing in rows owned by a lower tile form the type's secondary template, added after
// the owner has written its rows; per tile, its entries are numbered from sec_off[t].
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
  out.type_rep.clear();
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
      it = type_of_mask.emplace(key, int(out.type_rep.size())).first;
      out.type_rep.push_back(t);
    }
    out.tile_type[size_t(t)] = it->second;
  }
  const int n_types = int(out.type_rep.size());
  out.type_nvals.assign(size_t(n_types), 0);
  out.type_map_off.assign(size_t(n_types) + 1, 0);
  out.tmpl_ptr.assign(size_t(n_types) + 1, 0);
  out.tmpl.clear();
  out.type_rows.clear();
  out.type_row_off.assign(1, 0);
  std::vector<std::vector<char>> owned_of(static_cast<size_t>(n_types));
  std::vector<std::vector<int64_t>> deg_of(static_cast<size_t>(n_types));
  for (int ty = 0; ty < n_types; ++ty) {
    const int64_t t = out.type_rep[size_t(ty)];
    const int64_t idx[3] = {t % nx, (t / nx) % ny, t / (nx * ny)};
    std::vector<char>& owned = owned_of[size_t(ty)];
    owned.assign(size_t(n_T), 1);
    for (int d = 0; d < 3; ++d)
      if (idx[d] > 0)
        for (int A : topo.faces[2 * d]) owned[size_t(A)] = 0;
    const int32_t* g = &gmap[size_t(t) * n_T];
    int64_t vals = 0;
    deg_of[size_t(ty)].assign(size_t(n_T), 0);
    for (int A = 0; A < n_T; ++A) {
      const int64_t deg = pptr[size_t(g[A]) + 1] - pptr[size_t(g[A])];
      deg_of[size_t(ty)][size_t(A)] = deg;
      if (owned[size_t(A)]) vals += 9 * deg;
    }
    if (vals >= (int64_t(1) << 31)) return fail(MSASM_EUNSUPPORTED, "a tile owns more than 2^31 values");
    out.type_nvals[size_t(ty)] = int32_t(vals);
    out.type_map_off[size_t(ty) + 1] = out.type_map_off[size_t(ty)] + vals;
    {
      int32_t off = 0;
      for (int A = 0; A < n_T; ++A) {
        if (!owned[size_t(A)]) continue;
        const int32_t L = int32_t(3 * deg_of[size_t(ty)][size_t(A)]);
        for (int a = 0; a < 3; ++a) {
          out.type_rows.push_back(off + a * L);
          out.type_rows.push_back(L);
          out.type_rows.push_back((A << 2) | a);
        }
        off += 3 * L;
      }
      out.type_row_off.push_back(int64_t(out.type_rows.size() / 3));
    }
    for (int m = 0; m < n_nz; ++m) {
      const int A = topo.pair_A[m], B = topo.pair_B[m];
      uint32_t flags = 0;
      if (!owned[size_t(A)]) flags |= 1u;          // upper block into a row owned by a lower tile
      if (A != B && !owned[size_t(B)]) flags |= 2u;  // lower block likewise
      if (flags) out.tmpl.push_back(uint32_t(m) | (flags << 30));
    }
    out.tmpl_ptr[size_t(ty) + 1] = int64_t(out.tmpl.size());
  }
  // every tile has its type's layout: owned points with consecutive ids in local order and the
  // same row lengths
  out.sec_off.assign(size_t(plan->n_tiles) + 1, 0);
  for (int64_t t = 0; t < plan->n_tiles; ++t) {
    const int ty = out.tile_type[size_t(t)];
    const int32_t* g = &gmap[size_t(t) * n_T];
    const std::vector<char>& owned = owned_of[size_t(ty)];
    int64_t expect = -1;
    for (int A = 0; A < n_T; ++A) {
      if (!owned[size_t(A)]) continue;
      if (expect >= 0 && g[A] != expect)
        return fail(MSASM_EUNSUPPORTED, "owned points of a tile are not numbered consecutively");
      expect = int64_t(g[A]) + 1;
      if (pptr[size_t(g[A]) + 1] - pptr[size_t(g[A])] != deg_of[size_t(ty)][size_t(A)])
        return fail(MSASM_EUNSUPPORTED, "tile numbering is not translation invariant within a tile type");
    }
    out.sec_off[size_t(t) + 1] = out.sec_off[size_t(t)] + (out.tmpl_ptr[size_t(ty) + 1] - out.tmpl_ptr[size_t(ty)]);
  }
  return MSASM_OK;
}

}  // namespace msasm
