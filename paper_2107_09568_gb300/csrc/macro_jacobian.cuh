// Jacobian of a macro tile map at the interpolation nodes, by sum factorisation (one warp).
//
//   J[c][p][i] = d M^(t)_p / d xi_i (xi_c) = sum_a P_a,p  dB_a/dxi_i (xi_c),
//   B_a(xi) = B1_a1(xi_1) B2_a2(xi_2) B3_a3(xi_3)  (the span's B-spline basis, eq. 4 and 8),
//
// contracting one direction at a time: S = B1 . P, U = B2 . S, J = B3 . U, all FP64.
#pragma once

#include <cstdint>

namespace msasm {

struct MacroTileArgs {
  const double* ctrl;        // (n_ctrl, 3)
  const double* basis[3];    // per direction [e][c][a][value, d/dxi]
  const int32_t* first[3];   // per direction [e]: first control index of the span
  int n_elem[3];
  int n_ctrl_dir[3];
  int np[3];                 // degree + 1
  int nq[3];                 // points per direction (q_d + 1 at the interpolation nodes)
};

__host__ __device__ inline void jac_scratch_sizes(const int np[3], const int nq[3], int& nP, int& nS, int& nU,
                                                  int& nJ) {
  nP = np[0] * np[1] * np[2] * 3;
  nS = 2 * nq[0] * np[1] * np[2] * 3;
  nU = 3 * nq[0] * nq[1] * np[2] * 3;
  nJ = nq[0] * nq[1] * nq[2] * 9;
}

__device__ inline void tile_coords(const MacroTileArgs& a, int64_t t, int& e1, int& e2, int& e3) {
  e1 = int(t % a.n_elem[0]);
  e2 = int((t / a.n_elem[0]) % a.n_elem[1]);
  e3 = int(t / (int64_t(a.n_elem[0]) * a.n_elem[1]));
}

// Whole warp; P, S, U, Jn are this warp's shared-memory scratch; on return Jn[c*9 + p*3 + i].
__device__ inline void tile_node_jacobians(const MacroTileArgs& a, int64_t t, double* P, double* S, double* U,
                                           double* Jn, int lane) {
  const int np1 = a.np[0], np2 = a.np[1], np3 = a.np[2], nq1 = a.nq[0], nq2 = a.nq[1], nq3 = a.nq[2];
  int nP, nS, nU, nJ;
  jac_scratch_sizes(a.np, a.nq, nP, nS, nU, nJ);
  int e1, e2, e3;
  tile_coords(a, t, e1, e2, e3);
  const int f1 = a.first[0][e1], f2 = a.first[1][e2], f3 = a.first[2][e3];
  const double* B1 = a.basis[0] + size_t(e1) * nq1 * np1 * 2;
  const double* B2 = a.basis[1] + size_t(e2) * nq2 * np2 * 2;
  const double* B3 = a.basis[2] + size_t(e3) * nq3 * np3 * 2;
  for (int o = lane; o < nP; o += 32) {
    int p = o % 3, c = o / 3;
    int a1 = c % np1, a2 = (c / np1) % np2, a3 = c / (np1 * np2);
    int64_t gi = (f1 + a1) + int64_t(a.n_ctrl_dir[0]) * ((f2 + a2) + int64_t(a.n_ctrl_dir[1]) * (f3 + a3));
    P[o] = a.ctrl[gi * 3 + p];
  }
  __syncwarp();
  for (int o = lane; o < nS; o += 32) {        // S[v][c1][a2][a3][p] = sum_a1 B1[c1][a1][v] P[a1][a2][a3][p]
    int p = o % 3, r = o / 3;
    int a3 = r % np3; r /= np3;
    int a2 = r % np2; r /= np2;
    int c1 = r % nq1;
    int v = r / nq1;
    double s = 0.0;
    for (int a1 = 0; a1 < np1; ++a1) s = fma(B1[(c1 * np1 + a1) * 2 + v], P[((a1 + np1 * (a2 + np2 * a3)) * 3) + p], s);
    S[o] = s;
  }
  __syncwarp();
  for (int o = lane; o < nU; o += 32) {        // U[w][c1][c2][a3][p], w = (v1, v2) in {(0,0), (1,0), (0,1)}
    int p = o % 3, r = o / 3;
    int a3 = r % np3; r /= np3;
    int c2 = r % nq2; r /= nq2;
    int c1 = r % nq1;
    int w = r / nq1;
    int v1 = (w == 1), v2 = (w == 2);
    double s = 0.0;
    for (int a2 = 0; a2 < np2; ++a2)
      s = fma(B2[(c2 * np2 + a2) * 2 + v2], S[((((v1 * nq1 + c1) * np2 + a2) * np3 + a3) * 3) + p], s);
    U[o] = s;
  }
  __syncwarp();
  for (int o = lane; o < nJ; o += 32) {        // J[c][p][i], c = c1 + nq1 (c2 + nq2 c3)
    int i = o % 3, p = (o / 3) % 3, c = o / 9;
    int c1 = c % nq1, c2 = (c / nq1) % nq2, c3 = c / (nq1 * nq2);
    int w = (i == 0) ? 1 : (i == 1) ? 2 : 0;
    int v3 = (i == 2);
    double s = 0.0;
    for (int a3 = 0; a3 < np3; ++a3)
      s = fma(B3[(c3 * np3 + a3) * 2 + v3], U[((((w * nq1 + c1) * nq2 + c2) * np3 + a3) * 3) + p], s);
    Jn[o] = s;
  }
  __syncwarp();
}

__device__ inline double det3(const double J[9]) {
  return J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) + J[2] * (J[3] * J[7] - J[4] * J[6]);
}

// G = J^-1 by the adjugate; G[i*3 + p] (rows: xi_i, columns: physical p).
__device__ inline void inverse3(const double J[9], double inv_det, double G[9]) {
  G[0] = (J[4] * J[8] - J[5] * J[7]) * inv_det;
  G[1] = (J[2] * J[7] - J[1] * J[8]) * inv_det;
  G[2] = (J[1] * J[5] - J[2] * J[4]) * inv_det;
  G[3] = (J[5] * J[6] - J[3] * J[8]) * inv_det;
  G[4] = (J[0] * J[8] - J[2] * J[6]) * inv_det;
  G[5] = (J[2] * J[3] - J[0] * J[5]) * inv_det;
  G[6] = (J[3] * J[7] - J[4] * J[6]) * inv_det;
  G[7] = (J[1] * J[6] - J[0] * J[7]) * inv_det;
  G[8] = (J[0] * J[4] - J[1] * J[3]) * inv_det;
}

}  // namespace msasm
