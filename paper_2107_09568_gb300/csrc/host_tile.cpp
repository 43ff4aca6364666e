// Reference-tile topology on the host (eq. 3, 56): unique control points of the
// glued box patches, micro elements, the pair set I_coo, local adjacency and
// the six faces of [0,1]^3 used to glue neighbouring tiles.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <set>

#include "common.h"

namespace msasm {

static const double kPosTol = 1e-10;

msasm_status build_topology(const msasm_micro_desc* micro, TileTopology& topo) {
  if (!micro || micro->n_patches <= 0 || micro->n_patches > 16 || !micro->degree || !micro->n_elem ||
      !micro->box_lo || !micro->box_hi)
    return fail(MSASM_EINVAL, "micro descriptor: null array or n_patches outside 1..16");
  topo = TileTopology();
  for (int p = 0; p < micro->n_patches; ++p) {
    Patch P;
    for (int d = 0; d < 3; ++d) {
      P.degree[d] = micro->degree[3 * p + d];
      P.n_elem[d] = micro->n_elem[3 * p + d];
      P.lo[d] = micro->box_lo[3 * p + d];
      P.hi[d] = micro->box_hi[3 * p + d];
      if (P.degree[d] < 1 || P.degree[d] > 4 || P.n_elem[d] < 1 || P.n_elem[d] > 32)
        return fail(MSASM_EINVAL, "micro patch degree must be 1..4 and elements 1..32");
      if (!(P.lo[d] >= 0.0 && P.hi[d] <= 1.0 && P.hi[d] > P.lo[d]))
        return fail(MSASM_EINVAL, "micro patch box must lie in [0,1]^3 with hi > lo (Sec. 2.2.2)");
      P.n_fun[d] = P.n_elem[d] + P.degree[d];
      if (P.n_fun[d] > 127) return fail(MSASM_EINVAL, "too many functions per patch direction");
    }
    // Greville abscissae of the open uniform knot vector, then the affine box map
    std::vector<double> grev[3];
    for (int d = 0; d < 3; ++d) {
      int p_ = P.degree[d], n = P.n_elem[d];
      for (int i = 0; i < P.n_fun[d]; ++i) {
        double s = 0.0;
        for (int k = i + 1; k <= i + p_; ++k) {
          double knot = std::min(std::max(double(k - p_) / n, 0.0), 1.0);
          s += knot;
        }
        grev[d].push_back(s / p_);
      }
    }
    int nf = P.n_fun[0] * P.n_fun[1] * P.n_fun[2];
    P.ids.resize(nf);
    for (int a3 = 0; a3 < P.n_fun[2]; ++a3)
      for (int a2 = 0; a2 < P.n_fun[1]; ++a2)
        for (int a1 = 0; a1 < P.n_fun[0]; ++a1) {
          double x[3] = {P.lo[0] + (P.hi[0] - P.lo[0]) * grev[0][a1],
                         P.lo[1] + (P.hi[1] - P.lo[1]) * grev[1][a2],
                         P.lo[2] + (P.hi[2] - P.lo[2]) * grev[2][a3]};
          int found = -1;
          for (int A = 0; A < topo.n_T && found < 0; ++A) {
            const double* y = &topo.pos[3 * A];
            if (std::fabs(x[0] - y[0]) < kPosTol && std::fabs(x[1] - y[1]) < kPosTol &&
                std::fabs(x[2] - y[2]) < kPosTol)
              found = A;
          }
          if (found < 0) {
            found = topo.n_T++;
            topo.pos.insert(topo.pos.end(), x, x + 3);
          }
          P.ids[a1 + P.n_fun[0] * (a2 + P.n_fun[1] * a3)] = found;
        }
    topo.patches.push_back(std::move(P));
  }
  // pairs sharing a micro element (eq. 56)
  std::vector<std::vector<int>> nb(topo.n_T);
  std::set<std::pair<int, int>> pairs;
  for (const Patch& P : topo.patches) {
    for (int e3 = 0; e3 < P.n_elem[2]; ++e3)
      for (int e2 = 0; e2 < P.n_elem[1]; ++e2)
        for (int e1 = 0; e1 < P.n_elem[0]; ++e1) {
          std::vector<int> act;
          for (int a3 = e3; a3 <= e3 + P.degree[2]; ++a3)
            for (int a2 = e2; a2 <= e2 + P.degree[1]; ++a2)
              for (int a1 = e1; a1 <= e1 + P.degree[0]; ++a1)
                act.push_back(P.ids[a1 + P.n_fun[0] * (a2 + P.n_fun[1] * a3)]);
          for (int A : act)
            for (int B : act)
              if (A <= B) pairs.insert({A, B});
        }
  }
  for (const auto& pr : pairs) {
    topo.pair_A.push_back(pr.first);
    topo.pair_B.push_back(pr.second);
    nb[pr.first].push_back(pr.second);
    if (pr.first != pr.second) nb[pr.second].push_back(pr.first);
  }
  topo.nb_ptr.assign(topo.n_T + 1, 0);
  for (int A = 0; A < topo.n_T; ++A) {
    std::sort(nb[A].begin(), nb[A].end());
    topo.nb_ptr[A + 1] = topo.nb_ptr[A] + int64_t(nb[A].size());
    topo.nb_idx.insert(topo.nb_idx.end(), nb[A].begin(), nb[A].end());
  }
  // faces xi_d = 0 / 1, ordered by (second, first) in-face coordinate so opposite faces match
  for (int d = 0; d < 3; ++d) {
    int o0 = (d == 0) ? 1 : 0, o1 = (d == 2) ? 1 : 2;
    for (int s = 0; s < 2; ++s) {
      std::vector<int>& F = topo.faces[2 * d + s];
      for (int A = 0; A < topo.n_T; ++A)
        if (std::fabs(topo.pos[3 * A + d] - double(s)) < kPosTol) F.push_back(A);
      std::sort(F.begin(), F.end(), [&](int a, int b) {
        double ya = topo.pos[3 * a + o1], yb = topo.pos[3 * b + o1];
        if (std::fabs(ya - yb) > kPosTol) return ya < yb;
        return topo.pos[3 * a + o0] < topo.pos[3 * b + o0] - kPosTol;
      });
      topo.face_pos[2 * d + s].assign(topo.n_T, -1);
      for (size_t k = 0; k < F.size(); ++k) topo.face_pos[2 * d + s][F[k]] = int(k);
    }
    const std::vector<int>& F0 = topo.faces[2 * d];
    const std::vector<int>& F1 = topo.faces[2 * d + 1];
    if (F0.size() != F1.size())
      return fail(MSASM_EINVAL, "opposite faces of the reference tile hold different point counts");
    for (size_t k = 0; k < F0.size(); ++k)
      for (int e = 0; e < 3; ++e)
        if (e != d && std::fabs(topo.pos[3 * F0[k] + e] - topo.pos[3 * F1[k] + e]) > kPosTol)
          return fail(MSASM_EINVAL, "opposite faces of the reference tile do not match point for point");
  }
  // Gluing matches tiles face by face: a point owned across one face has exactly one other tile
  // holding it, so the numbering, the pattern (face neighbours only) and the two-contributor
  // scatter hold only when no control point lies on faces of two directions (an edge or a corner
  // of the tile, where three or more tiles would meet).
  for (int A = 0; A < topo.n_T; ++A) {
    int dirs = 0;
    for (int d = 0; d < 3; ++d)
      if (topo.face_pos[2 * d][A] >= 0 || topo.face_pos[2 * d + 1][A] >= 0) ++dirs;
    if (dirs > 1)
      return fail(MSASM_EUNSUPPORTED,
                  "a control point of the reference tile lies on an edge or corner of [0,1]^3 (on faces of two "
                  "directions); only tiles glued through face-interior points are supported");
  }
  size_t n_nz = topo.pair_A.size();
  topo.pair_face.assign(n_nz, 0);
  for (size_t m = 0; m < n_nz; ++m)
    for (int d = 0; d < 3; ++d)
      if (topo.face_pos[2 * d][topo.pair_A[m]] >= 0 && topo.face_pos[2 * d][topo.pair_B[m]] >= 0)
        topo.pair_face[m] |= uint8_t(1u << d);
  return MSASM_OK;
}

}  // namespace msasm
