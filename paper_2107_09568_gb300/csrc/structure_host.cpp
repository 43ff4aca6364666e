// Host part of K6: global numbering of the control points of the tiled structure
// and the point-level sparsity pattern (union over tiles of the pairs of eq. 56).
//
// Numbering convention: a control point on the xi_d = 0 face of tile t with a
// neighbour t - e_d is the matching point of the xi_d = 1 face of t - e_d; the
// owner of a point is the lowest tile index holding it, and ids are assigned in
// (owner tile, local id) order.  Row g of the pattern lists the ids of all points
// sharing a micro element with g in any tile, ascending.
#include <algorithm>
#include <thread>

#include "common.h"

namespace msasm {

void number_points(const TileTopology& topo, const int n_elem[3], std::vector<int32_t>& gmap, int64_t& n_points) {
  const int64_t nx = n_elem[0], ny = n_elem[1], nz = n_elem[2];
  const int64_t m = nx * ny * nz;
  const int n_T = topo.n_T;
  gmap.assign(size_t(m) * n_T, -1);
  const int64_t stride[3] = {1, nx, nx * ny};
  int64_t next = 0;
  for (int64_t t = 0; t < m; ++t) {
    const int64_t idx[3] = {t % nx, (t / nx) % ny, t / (nx * ny)};
    int32_t* g = &gmap[size_t(t) * n_T];
    for (int A = 0; A < n_T; ++A) {
      int32_t shared = -1;
      for (int d = 0; d < 3 && shared < 0; ++d) {
        int pos = topo.face_pos[2 * d][A];
        if (idx[d] > 0 && pos >= 0) shared = gmap[size_t(t - stride[d]) * n_T + topo.faces[2 * d + 1][pos]];
      }
      g[A] = shared >= 0 ? shared : int32_t(next++);
    }
  }
  n_points = next;
}

void point_pattern(const TileTopology& topo, const int n_elem[3], const std::vector<int32_t>& gmap, int64_t n_points,
                   std::vector<int64_t>& pptr, std::vector<int32_t>& pcol) {
  const int64_t nx = n_elem[0], ny = n_elem[1], nz = n_elem[2];
  const int64_t m = nx * ny * nz;
  const int n_T = topo.n_T;
  const int64_t stride[3] = {1, nx, nx * ny};
  unsigned n_thr = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  if (m < 64) n_thr = 1;
  std::vector<std::vector<int32_t>> cols(n_thr), degs(n_thr);
  auto work = [&](unsigned w) {
    int64_t t_begin = m * w / n_thr, t_end = m * (w + 1) / n_thr;
    std::vector<int32_t> buf;
    for (int64_t t = t_begin; t < t_end; ++t) {
      const int64_t idx[3] = {t % nx, (t / nx) % ny, t / (nx * ny)};
      const int32_t* g = &gmap[size_t(t) * n_T];
      for (int A = 0; A < n_T; ++A) {
        bool owned = true;
        for (int d = 0; d < 3; ++d)
          if (idx[d] > 0 && topo.face_pos[2 * d][A] >= 0) owned = false;
        if (!owned) continue;
        buf.clear();
        for (int64_t k = topo.nb_ptr[A]; k < topo.nb_ptr[A + 1]; ++k) buf.push_back(g[topo.nb_idx[k]]);
        for (int d = 0; d < 3; ++d) {
          int pos = topo.face_pos[2 * d + 1][A];
          if (pos >= 0 && idx[d] + 1 < n_elem[d]) {
            const int32_t* g2 = &gmap[size_t(t + stride[d]) * n_T];
            int A2 = topo.faces[2 * d][pos];
            for (int64_t k = topo.nb_ptr[A2]; k < topo.nb_ptr[A2 + 1]; ++k) buf.push_back(g2[topo.nb_idx[k]]);
          }
        }
        std::sort(buf.begin(), buf.end());
        buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
        degs[w].push_back(int32_t(buf.size()));
        cols[w].insert(cols[w].end(), buf.begin(), buf.end());
      }
    }
  };
  std::vector<std::thread> pool;
  for (unsigned w = 1; w < n_thr; ++w) pool.emplace_back(work, w);
  work(0);
  for (auto& th : pool) th.join();
  pptr.assign(size_t(n_points) + 1, 0);
  int64_t g = 0, total = 0;
  for (unsigned w = 0; w < n_thr; ++w)
    for (int32_t d : degs[w]) {
      total += d;
      pptr[size_t(++g)] = total;
    }
  pcol.clear();
  pcol.reserve(size_t(total));
  for (unsigned w = 0; w < n_thr; ++w) pcol.insert(pcol.end(), cols[w].begin(), cols[w].end());
}

}  // namespace msasm
