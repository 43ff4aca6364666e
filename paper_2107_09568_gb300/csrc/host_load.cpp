// Boundary data on a macro face of the tiled structure (host side, set-up only):
// the global points lying on the face (for Dirichlet conditions) and the load vector of a
// uniform traction on it, f_A = int_Gamma R_A t dGamma (eq. 29, 33), by Gauss quadrature
// on the micro patch faces that lie on the tile face.
#include <algorithm>
#include <cmath>
#include <set>
#include <vector>

#include "common.h"

namespace msasm {

// macro map x(xi) of tile t and its Jacobian dx/dxi (3x3, [p][i]) from the control net
static void macro_eval(const msasm_plan* plan, const double* ctrl, const int e[3], const double xi[3], double x[3],
                       double J[9]) {
  double vals[3][8], ders[3][8];
  int first[3];
  for (int d = 0; d < 3; ++d) {
    const std::vector<double>& t = plan->knots_host[d];
    const int p = plan->degree[d];
    int span = plan->span_host[d][e[d]];
    const double u0 = t[span], h = t[span + 1] - t[span];
    bspline_span_basis(t.data(), p, span, u0 + h * xi[d], vals[d], ders[d]);
    for (int a = 0; a <= p; ++a) ders[d][a] *= h;
    first[d] = span - p;
  }
  for (int k = 0; k < 3; ++k) x[k] = 0.0;
  for (int k = 0; k < 9; ++k) J[k] = 0.0;
  for (int a3 = 0; a3 <= plan->degree[2]; ++a3)
    for (int a2 = 0; a2 <= plan->degree[1]; ++a2)
      for (int a1 = 0; a1 <= plan->degree[0]; ++a1) {
        const int64_t gi = (first[0] + a1) + int64_t(plan->n_ctrl_dir[0]) *
                                                 ((first[1] + a2) + int64_t(plan->n_ctrl_dir[1]) * (first[2] + a3));
        const double b = vals[0][a1] * vals[1][a2] * vals[2][a3];
        const double d1 = ders[0][a1] * vals[1][a2] * vals[2][a3];
        const double d2 = vals[0][a1] * ders[1][a2] * vals[2][a3];
        const double d3 = vals[0][a1] * vals[1][a2] * ders[2][a3];
        for (int p = 0; p < 3; ++p) {
          const double c = ctrl[gi * 3 + p];
          x[p] += b * c;
          J[p * 3 + 0] += d1 * c;
          J[p * 3 + 1] += d2 * c;
          J[p * 3 + 2] += d3 * c;
        }
      }
}

// open uniform knot vector values of degree p with n elements: all p+1 functions alive on element e
static void uniform_basis(int p, int n, int e, double s, double* N) {
  std::vector<double> t(size_t(n + 2 * p + 1));
  for (size_t k = 0; k < t.size(); ++k) t[k] = std::min(std::max(double(int(k) - p) / n, 0.0), 1.0);
  double dummy[16];
  bspline_span_basis(t.data(), p, e + p, s, N, dummy);
}

static bool tile_on_face(const msasm_plan* plan, int64_t t, int face, int e[3]) {
  e[0] = int(t % plan->n_elem[0]);
  e[1] = int((t / plan->n_elem[0]) % plan->n_elem[1]);
  e[2] = int(t / (int64_t(plan->n_elem[0]) * plan->n_elem[1]));
  const int d = face / 2, s = face % 2;
  return e[d] == (s == 0 ? 0 : plan->n_elem[d] - 1);
}

}  // namespace msasm

using namespace msasm;

extern "C" msasm_status msasm_face_points(const msasm_plan* plan, int32_t face, int32_t* h_points, int64_t* count) {
  if (!plan || !count) return fail(MSASM_EINVAL, "plan or count is NULL");
  if (face < 0 || face > 5) return fail(MSASM_EINVAL, "face must be 0..5 (2 d + s for xi_d = s)");
  const TileTopology& topo = plan->tab->topo;
  std::set<int32_t> pts;
  for (int64_t t = 0; t < plan->n_tiles; ++t) {
    int e[3];
    if (!tile_on_face(plan, t, face, e)) continue;
    for (int A : topo.faces[face]) pts.insert(plan->gmap_host[size_t(t) * topo.n_T + A]);
  }
  if (h_points) {
    if (*count < int64_t(pts.size())) return fail(MSASM_EINVAL, "h_points too small (pass its length in *count)");
    int64_t k = 0;
    for (int32_t g : pts) h_points[k++] = g;
  }
  *count = int64_t(pts.size());
  return MSASM_OK;
}

extern "C" msasm_status msasm_traction_load(const msasm_plan* plan, int32_t face, const double* traction,
                                            const double* h_ctrl, double* h_f) {
  if (!plan || !traction || !h_ctrl || !h_f) return fail(MSASM_EINVAL, "NULL argument");
  if (face < 0 || face > 5) return fail(MSASM_EINVAL, "face must be 0..5 (2 d + s for xi_d = s)");
  const TileTopology& topo = plan->tab->topo;
  const int d = face / 2, s = face % 2;
  const int ia = (d == 0) ? 1 : 0, ib = (d == 2) ? 1 : 2;   // in-face directions
  std::vector<double> gx, gw;
  gauss_legendre01(6, gx, gw);
  std::fill(h_f, h_f + plan->n_rows, 0.0);
  for (int64_t t = 0; t < plan->n_tiles; ++t) {
    int e[3];
    if (!tile_on_face(plan, t, face, e)) continue;
    const int32_t* g = &plan->gmap_host[size_t(t) * topo.n_T];
    for (const Patch& P : topo.patches) {
      if (!((s == 0 && P.lo[d] == 0.0) || (s == 1 && P.hi[d] == 1.0))) continue;
      const int ad = (s == 0) ? 0 : P.n_fun[d] - 1;       // the only function not vanishing on the face
      const double ha = P.hi[ia] - P.lo[ia], hb = P.hi[ib] - P.lo[ib];
      for (int eb = 0; eb < P.n_elem[ib]; ++eb)
        for (int ea = 0; ea < P.n_elem[ia]; ++ea)
          for (int qb = 0; qb < 6; ++qb)
            for (int qa = 0; qa < 6; ++qa) {
              const double sa = (ea + gx[qa]) / P.n_elem[ia], sb = (eb + gx[qb]) / P.n_elem[ib];
              const double w = gw[qa] * gw[qb] / (P.n_elem[ia] * P.n_elem[ib]);
              double xi[3];
              xi[d] = double(s);
              xi[ia] = P.lo[ia] + ha * sa;
              xi[ib] = P.lo[ib] + hb * sb;
              double x[3], J[9];
              macro_eval(plan, h_ctrl, e, xi, x, J);
              double ta[3], tb[3];
              for (int p = 0; p < 3; ++p) {
                ta[p] = J[p * 3 + ia] * ha;
                tb[p] = J[p * 3 + ib] * hb;
              }
              const double cx = ta[1] * tb[2] - ta[2] * tb[1], cy = ta[2] * tb[0] - ta[0] * tb[2],
                           cz = ta[0] * tb[1] - ta[1] * tb[0];
              const double dA = std::sqrt(cx * cx + cy * cy + cz * cz) * w;
              double Na[8], Nb[8];
              uniform_basis(P.degree[ia], P.n_elem[ia], ea, sa, Na);
              uniform_basis(P.degree[ib], P.n_elem[ib], eb, sb, Nb);
              for (int kb = 0; kb <= P.degree[ib]; ++kb)
                for (int ka = 0; ka <= P.degree[ia]; ++ka) {
                  int a[3];
                  a[d] = ad;
                  a[ia] = ea + ka;
                  a[ib] = eb + kb;
                  const int A = P.ids[a[0] + P.n_fun[0] * (a[1] + P.n_fun[1] * a[2])];
                  const double r = Na[ka] * Nb[kb] * dA;
                  for (int c = 0; c < 3; ++c) h_f[3 * int64_t(g[A]) + c] += r * traction[c];
                }
            }
    }
  }
  return MSASM_OK;
}
