// Volume (Sec. 3.1, eq. 14-19) and the body-force load vector (eq. 39-40, 53-55) through lookup
// tables, for every tile at once.  Both need only the macro-Jacobian determinant at the
// interpolation nodes, d_C^(t) = |det J^(t)(xi_C)| (the interpolated |det J| of eq. 15 and of the
// body-force coefficients b |det J| of eq. 40):
//
//   V^(t) = t^h . d^(t)                   (eq. 17, t^h the volume table of eq. 18)
//   f_A^(t) = b sum_C F[A][C] d_C^(t)      (eq. 53, F = 0 term, F the load table of eq. 55)
//
// One warp per tile: the node Jacobians by the same sum factorisation as the pullback, then the
// determinants, the tile's volume (warp reduction) and its control points' loads.  A point shared by
// two tiles (a glued face) receives two additions; with exactly two addends the sum does not depend
// on their order, so the result is deterministic.  The total volume is a fixed-order reduction of
// the tile volumes.
#include <cmath>

#include "common.h"
#include "macro_jacobian.cuh"

namespace msasm {

MacroTileArgs macro_tile_args(const msasm_plan* plan, const double* d_ctrl);

struct VolumeArgs {
  MacroTileArgs geo;
  int64_t n_tiles;
  const double* vol;       // t^h (n_pi)
  const double* F;         // load table (n_T x n_pi)
  int n_T;
  const int32_t* gmap;
  double* tile_vol;        // per tile (or null)
  double* f;               // load vector (n_rows, accumulated; or null)
  double b0, b1, b2;
};

__global__ void volume_load_kernel(VolumeArgs a) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
  const int nq = a.geo.nq, n_pi = nq * nq * nq;
  int nP, nS, nU, nJ;
  jac_scratch_sizes(a.geo.np, nq, nP, nS, nU, nJ);
  double* P = smem + size_t(warp) * (nP + nS + nU + nJ + n_pi);
  double* S = P + nP;
  double* U = S + nS;
  double* Jn = U + nU;
  double* d = Jn + nJ;
  for (int64_t t = int64_t(blockIdx.x) * warps + warp; t < a.n_tiles; t += int64_t(gridDim.x) * warps) {
    tile_node_jacobians(a.geo, t, P, S, U, Jn, lane);
    for (int c = lane; c < n_pi; c += 32) d[c] = fabs(det3(Jn + 9 * c));
    __syncwarp();
    if (a.tile_vol) {
      double s = 0.0;
      for (int c = lane; c < n_pi; c += 32) s = fma(a.vol[c], d[c], s);
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) a.tile_vol[t] = s;
    }
    if (a.f) {
      for (int A = lane; A < a.n_T; A += 32) {
        const double* Fa = a.F + size_t(A) * n_pi;
        double s = 0.0;
        for (int c = 0; c < n_pi; ++c) s = fma(Fa[c], d[c], s);
        const int64_t g = a.gmap[t * a.n_T + A];
        atomicAdd(a.f + 3 * g + 0, a.b0 * s);
        atomicAdd(a.f + 3 * g + 1, a.b1 * s);
        atomicAdd(a.f + 3 * g + 2, a.b2 * s);
      }
    }
    __syncwarp();
  }
}

// sum of n values in a fixed order: one block, a strided partial sum per thread, then a tree
__global__ void ordered_sum_kernel(const double* __restrict__ x, int64_t n, double* __restrict__ out) {
  __shared__ double part[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (int(threadIdx.x) < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = part[0];
}

static size_t volume_smem_per_warp(const MacroTileArgs& g) {
  int nP, nS, nU, nJ;
  jac_scratch_sizes(g.np, g.nq, nP, nS, nU, nJ);
  return size_t(nP + nS + nU + nJ + g.nq * g.nq * g.nq) * sizeof(double);
}

msasm_status volume_load_gpu(const msasm_plan* plan, const double* d_ctrl, double* d_tile_vol, double* d_total,
                             double* d_f, const double b[3], cudaStream_t s) {
  VolumeArgs a;
  a.geo = macro_tile_args(plan, d_ctrl);
  a.n_tiles = plan->n_tiles;
  a.vol = plan->tab->d_vol;
  a.F = plan->tab->d_F;
  a.n_T = plan->tab->topo.n_T;
  a.gmap = plan->d_gmap;
  a.tile_vol = d_tile_vol;
  a.f = d_f;
  a.b0 = b ? b[0] : 0.0;
  a.b1 = b ? b[1] : 0.0;
  a.b2 = b ? b[2] : 0.0;
  const int warps = 4;
  const size_t smem = warps * volume_smem_per_warp(a.geo);
  if (smem > 200 * 1024) return fail(MSASM_EUNSUPPORTED, "macro degree / q too large for the volume kernel");
  MSASM_CUDA(cudaFuncSetAttribute(volume_load_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((a.n_tiles + warps - 1) / warps, 152 * 16));
  volume_load_kernel<<<unsigned(blocks), 32 * warps, smem, s>>>(a);
  MSASM_CUDA(cudaGetLastError());
  if (d_total && d_tile_vol) {
    ordered_sum_kernel<<<1, 256, 0, s>>>(d_tile_vol, plan->n_tiles, d_total);
    MSASM_CUDA(cudaGetLastError());
  }
  return MSASM_OK;
}

}  // namespace msasm
