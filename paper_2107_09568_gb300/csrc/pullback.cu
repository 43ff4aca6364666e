// K2: pullback of the elasticity tensor through each macro element and its
// interpolation at the (q1+1)(q2+1)(q3+1) nodes (eq. 37, 42; appendix A).
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
#include <algorithm>
#include <cmath>

#include "common.h"
#include "macro_jacobian.cuh"

namespace msasm {

struct PullbackArgs {
  MacroTileArgs geo;
  int64_t t0, n_tiles;      // tiles [t0, t0 + n_tiles) of this pass
  double lam, mu;
  double* coef;             // (9 n_tiles) x (9 n_pi)
  unsigned long long* degenerate;
};

__global__ void pullback_kernel(PullbackArgs a) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
  const int n_pi = a.geo.nq[0] * a.geo.nq[1] * a.geo.nq[2], K = 9 * n_pi;
  int nP, nS, nU, nJ;
  jac_scratch_sizes(a.geo.np, a.geo.nq, nP, nS, nU, nJ);
  double* P = smem + size_t(warp) * (nP + nS + nU + nJ);
  double* S = P + nP;
  double* U = S + nS;
  double* Jn = U + nU;
  for (int64_t tl = int64_t(blockIdx.x) * warps + warp; tl < a.n_tiles; tl += int64_t(gridDim.x) * warps) {
    tile_node_jacobians(a.geo, a.t0 + tl, P, S, U, Jn, lane);
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
      double G[9];
      inverse3(J, 1.0 / det, G);
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

size_t pullback_smem_per_warp(const int np[3], const int nq[3]) {
  int nP, nS, nU, nJ;
  jac_scratch_sizes(np, nq, nP, nS, nU, nJ);
  return size_t(nP + nS + nU + nJ) * sizeof(double);
}

MacroTileArgs macro_tile_args(const msasm_plan* plan, const double* d_ctrl) {
  MacroTileArgs g;
  g.ctrl = d_ctrl;
  for (int d = 0; d < 3; ++d) {
    g.basis[d] = plan->d_basis[d];
    g.first[d] = plan->d_first[d];
    g.n_elem[d] = plan->n_elem[d];
    g.n_ctrl_dir[d] = plan->n_ctrl_dir[d];
    g.np[d] = plan->degree[d] + 1;
  }
  for (int d = 0; d < 3; ++d) g.nq[d] = plan->tab->qd[d] + 1;
  return g;
}

msasm_status pullback_gpu(const msasm_plan* plan, const double* d_ctrl, double lam, double mu, int64_t t0,
                          int64_t n_tiles, double* d_coef, cudaStream_t stream) {
  PullbackArgs a;
  a.geo = macro_tile_args(plan, d_ctrl);
  a.t0 = t0;
  a.n_tiles = n_tiles;
  a.lam = lam;
  a.mu = mu;
  a.coef = d_coef;
  a.degenerate = plan->d_degenerate;
  const int warps = 4;
  size_t smem = warps * pullback_smem_per_warp(a.geo.np, a.geo.nq);
  if (smem > 200 * 1024) return fail(MSASM_EUNSUPPORTED, "macro degree / q too large for the pullback kernel");
  MSASM_CUDA(cudaFuncSetAttribute(pullback_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  int64_t blocks = (n_tiles + warps - 1) / warps;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  pullback_kernel<<<unsigned(blocks), 32 * warps, smem, stream>>>(a);
  MSASM_CUDA(cudaGetLastError());
  return MSASM_OK;
}

// The pullback at another set of nodes (the macro basis tables of geo), for tiles [0, n_tiles).
msasm_status pullback_geo_gpu(const MacroTileArgs& geo, int64_t n_tiles, double lam, double mu, double* d_coef,
                              unsigned long long* d_degenerate, cudaStream_t stream) {
  PullbackArgs a;
  a.geo = geo;
  a.t0 = 0;
  a.n_tiles = n_tiles;
  a.lam = lam;
  a.mu = mu;
  a.coef = d_coef;
  a.degenerate = d_degenerate;
  const int warps = 2;
  const size_t smem = warps * pullback_smem_per_warp(a.geo.np, a.geo.nq);
  if (smem > 200 * 1024) return fail(MSASM_EUNSUPPORTED, "macro degree / q too large for the pullback kernel");
  MSASM_CUDA(cudaFuncSetAttribute(pullback_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n_tiles + warps - 1) / warps, 152 * 16));
  pullback_kernel<<<unsigned(blocks), 32 * warps, smem, stream>>>(a);
  MSASM_CUDA(cudaGetLastError());
  return MSASM_OK;
}

}  // namespace msasm
