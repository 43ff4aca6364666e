// K2: pullback of the elasticity tensor through each macro element and its
// interpolation at the (q+1)^3 nodes (eq. 37, 42; appendix A).
//
// One warp per tile.  The tile's (p1+1)(p2+1)(p3+1) control points are staged in
// shared memory and the Jacobian J[p][i] = d M^(t)_p / d xi_i at all nodes is
// obtained by sum factorisation (contract direction 1, then 2, then 3), all in
// FP64.  Each lane then takes nodes c = lane, lane+32, ...: determinant and
// inverse G = J^-1 in FP64 and
//
//   A_ij[a][b] = |det J| (lam G[i][a] G[j][b] + mu delta_ab (G G^T)[i][j] + mu G[i][b] G[j][a]),
//
// the Cartesian form of G_i C G_j^T |det J| (eq. 37, 84, 91-97), written as the
// transposed coefficient matrix coef[9t + 3a + b][9C + 3i + j].
#include <cmath>

#include "common.h"

namespace msasm {

struct PullbackArgs {
  const double* ctrl;
  const double* basis[3];   // [e][c][a][2]: value, d/dxi
  const int32_t* first[3];  // [e]: first control index of the span
  int n_elem[3];
  int n_ctrl_dir[3];
  int np[3];                // degree + 1 per direction
  int nq;                   // q + 1
  int64_t t0, n_tiles;      // tiles [t0, t0 + n_tiles) of this pass
  double lam, mu;
  double* coef;             // (9 n_tiles) x (9 nq^3)
  unsigned long long* degenerate;
};

__device__ inline double det3(const double J[9]) {
  return J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
         J[2] * (J[3] * J[7] - J[4] * J[6]);
}

__global__ void pullback_kernel(PullbackArgs a) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
  const int np1 = a.np[0], np2 = a.np[1], np3 = a.np[2], nq = a.nq;
  const int nP = np1 * np2 * np3 * 3, nS = 2 * nq * np2 * np3 * 3, nU = 3 * nq * nq * np3 * 3,
            n_pi = nq * nq * nq, nJ = n_pi * 9;
  double* P = smem + size_t(warp) * (nP + nS + nU + nJ);
  double* S = P + nP;
  double* U = S + nS;
  double* Jn = U + nU;
  const int K = 9 * n_pi;
  for (int64_t tl = int64_t(blockIdx.x) * warps + warp; tl < a.n_tiles; tl += int64_t(gridDim.x) * warps) {
    const int64_t t = a.t0 + tl;
    const int e1 = int(t % a.n_elem[0]), e2 = int((t / a.n_elem[0]) % a.n_elem[1]),
              e3 = int(t / (int64_t(a.n_elem[0]) * a.n_elem[1]));
    const int f1 = a.first[0][e1], f2 = a.first[1][e2], f3 = a.first[2][e3];
    const double* B1 = a.basis[0] + size_t(e1) * nq * np1 * 2;
    const double* B2 = a.basis[1] + size_t(e2) * nq * np2 * 2;
    const double* B3 = a.basis[2] + size_t(e3) * nq * np3 * 2;
    // stage 0: control points of the span
    for (int o = lane; o < nP; o += 32) {
      int p = o % 3, c = o / 3;
      int a1 = c % np1, a2 = (c / np1) % np2, a3 = c / (np1 * np2);
      int64_t gi = (f1 + a1) + int64_t(a.n_ctrl_dir[0]) * ((f2 + a2) + int64_t(a.n_ctrl_dir[1]) * (f3 + a3));
      P[o] = a.ctrl[gi * 3 + p];
    }
    __syncwarp();
    // stage 1: S[v][c1][a2][a3][p] = sum_a1 B1[c1][a1][v] P[a1][a2][a3][p]
    for (int o = lane; o < nS; o += 32) {
      int p = o % 3, r = o / 3;
      int a3 = r % np3; r /= np3;
      int a2 = r % np2; r /= np2;
      int c1 = r % nq;
      int v = r / nq;
      double s = 0.0;
      for (int a1 = 0; a1 < np1; ++a1)
        s = fma(B1[(c1 * np1 + a1) * 2 + v], P[((a1 + np1 * (a2 + np2 * a3)) * 3) + p], s);
      S[o] = s;
    }
    __syncwarp();
    // stage 2: U[w][c1][c2][a3][p], w = (v1, v2) in {(0,0), (1,0), (0,1)}
    for (int o = lane; o < nU; o += 32) {
      int p = o % 3, r = o / 3;
      int a3 = r % np3; r /= np3;
      int c2 = r % nq; r /= nq;
      int c1 = r % nq;
      int w = r / nq;
      int v1 = (w == 1), v2 = (w == 2);
      double s = 0.0;
      for (int a2 = 0; a2 < np2; ++a2)
        s = fma(B2[(c2 * np2 + a2) * 2 + v2], S[((((v1 * nq + c1) * np2 + a2) * np3 + a3) * 3) + p], s);
      U[o] = s;
    }
    __syncwarp();
    // stage 3: J[c][p][i], c = c1 + nq (c2 + nq c3)
    for (int o = lane; o < nJ; o += 32) {
      int i = o % 3, p = (o / 3) % 3, c = o / 9;
      int c1 = c % nq, c2 = (c / nq) % nq, c3 = c / (nq * nq);
      int w = (i == 0) ? 1 : (i == 1) ? 2 : 0;
      int v3 = (i == 2);
      double s = 0.0;
      for (int a3 = 0; a3 < np3; ++a3)
        s = fma(B3[(c3 * np3 + a3) * 2 + v3], U[((((w * nq + c1) * nq + c2) * np3 + a3) * 3) + p], s);
      Jn[o] = s;
    }
    __syncwarp();
    // per node: det, inverse, macro field
    double* out = a.coef + size_t(tl) * 9 * K;
    for (int c = lane; c < n_pi; c += 32) {
      double J[9];
      for (int k = 0; k < 9; ++k) J[k] = Jn[c * 9 + k];   // J[p*3 + i]
      double det = det3(J);
      double fro2 = 0.0;
      for (int k = 0; k < 9; ++k) fro2 += J[k] * J[k];
      double ref = fro2 / 3.0;
      if (!(fabs(det) > 1e-12 * ref * sqrt(ref))) atomicAdd(a.degenerate, 1ull);
      double inv = 1.0 / det;
      // G = J^-1, G[i][p] (rows: xi_i, columns: physical p)
      double G[9];
      G[0] = (J[4] * J[8] - J[5] * J[7]) * inv;
      G[1] = (J[2] * J[7] - J[1] * J[8]) * inv;
      G[2] = (J[1] * J[5] - J[2] * J[4]) * inv;
      G[3] = (J[5] * J[6] - J[3] * J[8]) * inv;
      G[4] = (J[0] * J[8] - J[2] * J[6]) * inv;
      G[5] = (J[2] * J[3] - J[0] * J[5]) * inv;
      G[6] = (J[3] * J[7] - J[4] * J[6]) * inv;
      G[7] = (J[1] * J[6] - J[0] * J[7]) * inv;
      G[8] = (J[0] * J[4] - J[1] * J[3]) * inv;
      double adet = fabs(det);
      double GG[9];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          GG[i * 3 + j] = G[i * 3 + 0] * G[j * 3 + 0] + G[i * 3 + 1] * G[j * 3 + 1] + G[i * 3 + 2] * G[j * 3 + 2];
      const double l = a.lam * adet, m = a.mu * adet;
#pragma unroll
      for (int al = 0; al < 3; ++al)
#pragma unroll
        for (int be = 0; be < 3; ++be) {
          double* row = out + size_t(3 * al + be) * K + 9 * c;
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
              double v = l * G[i * 3 + al] * G[j * 3 + be] + m * G[i * 3 + be] * G[j * 3 + al];
              if (al == be) v += m * GG[i * 3 + j];
              row[3 * i + j] = v;
            }
        }
    }
    __syncwarp();
  }
}

size_t pullback_smem_per_warp(const int np[3], int nq) {
  size_t nP = size_t(np[0]) * np[1] * np[2] * 3, nS = size_t(2) * nq * np[1] * np[2] * 3,
         nU = size_t(3) * nq * nq * np[2] * 3, nJ = size_t(nq) * nq * nq * 9;
  return (nP + nS + nU + nJ) * sizeof(double);
}

msasm_status pullback_gpu(const msasm_plan* plan, const double* d_ctrl, double lam, double mu, int64_t t0,
                          int64_t n_tiles, double* d_coef, cudaStream_t stream) {
  PullbackArgs a;
  a.ctrl = d_ctrl;
  for (int d = 0; d < 3; ++d) {
    a.basis[d] = plan->d_basis[d];
    a.first[d] = plan->d_first[d];
    a.n_elem[d] = plan->n_elem[d];
    a.n_ctrl_dir[d] = plan->n_ctrl_dir[d];
    a.np[d] = plan->degree[d] + 1;
  }
  a.nq = plan->tab->q + 1;
  a.t0 = t0;
  a.n_tiles = n_tiles;
  a.lam = lam;
  a.mu = mu;
  a.coef = d_coef;
  a.degenerate = plan->d_degenerate;
  const int warps = 4;
  size_t smem = warps * pullback_smem_per_warp(a.np, a.nq);
  if (smem > 200 * 1024) return fail(MSASM_EUNSUPPORTED, "macro degree / q too large for the pullback kernel");
  MSASM_CUDA(cudaFuncSetAttribute(pullback_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  int64_t blocks = (n_tiles + warps - 1) / warps;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  pullback_kernel<<<unsigned(blocks), 32 * warps, smem, stream>>>(a);
  MSASM_CUDA(cudaGetLastError());
  return MSASM_OK;
}

}  // namespace msasm
