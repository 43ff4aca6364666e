// Volume (Sec. 3.1, eq. 14-19) and the body-force and traction load vectors (eq. 39-41, 53-55,
// 85-88) through lookup tables, for every tile at once.  Both need only the macro-Jacobian determinant at the
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
#include <algorithm>
#include <cmath>
#include <vector>

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
  const int n_pi = a.geo.nq[0] * a.geo.nq[1] * a.geo.nq[2];
  int nP, nS, nU, nJ;
  jac_scratch_sizes(a.geo.np, a.geo.nq, nP, nS, nU, nJ);
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

// Traction load through the face tables (eq. 53, F >= 1 terms; eq. 87-88): on the macro face
// xi_d = s, per tile on it, the macro traction t |det I_M| at the face's (q_ia+1)(q_ib+1) nodes,
// where on that face det I_M = (n x g_ia) . g_ib = |g_ia x g_ib| (g_k = dM/dxi_k, n the unit normal
// along g^d), then f_A = t sum_C2 Ff[A][C2] |g_ia x g_ib|(node C2).  The node Jacobians come from
// the pullback's sum factorisation with a single point, xi_d = s, in the normal direction.  One
// warp per tile on the face.
struct TractionArgs {
  MacroTileArgs geo;
  int d, ia, ib, s;
  const double* Ff;        // face table of this face (n_T x nq[ia] nq[ib])
  int n_T;
  const int32_t* gmap;
  double t0, t1, t2;
  double* f;               // load vector (n_rows, accumulated)
};

__global__ void traction_load_kernel(TractionArgs a) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
  const int n2 = a.geo.nq[a.ia] * a.geo.nq[a.ib];
  int nP, nS, nU, nJ;
  jac_scratch_sizes(a.geo.np, a.geo.nq, nP, nS, nU, nJ);
  double* P = smem + size_t(warp) * (nP + nS + nU + nJ + n2);
  double* S = P + nP;
  double* U = S + nS;
  double* Jn = U + nU;
  double* area = Jn + nJ;
  const int ne[3] = {a.geo.n_elem[0], a.geo.n_elem[1], a.geo.n_elem[2]};
  const int64_t n_face = int64_t(ne[a.ia]) * ne[a.ib];
  for (int64_t k = int64_t(blockIdx.x) * warps + warp; k < n_face; k += int64_t(gridDim.x) * warps) {
    int e[3];
    e[a.d] = a.s ? ne[a.d] - 1 : 0;
    e[a.ia] = int(k % ne[a.ia]);
    e[a.ib] = int(k / ne[a.ia]);
    const int64_t t = e[0] + int64_t(ne[0]) * (e[1] + int64_t(ne[1]) * e[2]);
    tile_node_jacobians(a.geo, t, P, S, U, Jn, lane);
    for (int C2 = lane; C2 < n2; C2 += 32) {
      int c[3];
      c[a.d] = 0;
      c[a.ia] = C2 % a.geo.nq[a.ia];
      c[a.ib] = C2 / a.geo.nq[a.ia];
      const double* J = Jn + 9 * (c[0] + a.geo.nq[0] * (c[1] + a.geo.nq[1] * c[2]));   // J[p * 3 + i] = dM_p / dxi_i
      const double ga[3] = {J[a.ia], J[3 + a.ia], J[6 + a.ia]};
      const double gb[3] = {J[a.ib], J[3 + a.ib], J[6 + a.ib]};
      const double x = ga[1] * gb[2] - ga[2] * gb[1], y = ga[2] * gb[0] - ga[0] * gb[2],
                   z = ga[0] * gb[1] - ga[1] * gb[0];
      area[C2] = sqrt(x * x + y * y + z * z);
    }
    __syncwarp();
    for (int A = lane; A < a.n_T; A += 32) {
      const double* Fa = a.Ff + size_t(A) * n2;
      double v = 0.0;
      for (int C2 = 0; C2 < n2; ++C2) v = fma(Fa[C2], area[C2], v);
      if (v != 0.0) {
        const int64_t g = a.gmap[t * a.n_T + A];
        atomicAdd(a.f + 3 * g + 0, a.t0 * v);
        atomicAdd(a.f + 3 * g + 1, a.t1 * v);
        atomicAdd(a.f + 3 * g + 2, a.t2 * v);
      }
    }
    __syncwarp();
  }
}

void bspline_span_basis(const double* t, int p, int span, double u, double* vals, double* ders);

msasm_status traction_load_gpu(const msasm_plan* plan, const double* d_ctrl, int face, const double tr[3], double* d_f,
                               cudaStream_t st) {
  const int d = face / 2, sd = face % 2;
  TractionArgs a;
  a.geo = macro_tile_args(plan, d_ctrl);
  a.d = d;
  a.ia = d == 0 ? 1 : 0;
  a.ib = d == 2 ? 1 : 2;
  a.s = sd;
  a.n_T = plan->tab->topo.n_T;
  a.Ff = plan->tab->d_Fface + plan->tab->face_off[face];
  a.gmap = plan->d_gmap;
  a.t0 = tr[0];
  a.t1 = tr[1];
  a.t2 = tr[2];
  a.f = d_f;
  // the normal direction's macro basis at its single point xi_d = s
  const std::vector<double>& t = plan->knots_host[d];
  const int p = plan->degree[d];
  std::vector<double> nb;
  for (int k : plan->span_host[d]) {
    const double u0 = t[size_t(k)], h = t[size_t(k) + 1] - t[size_t(k)];
    double vals[8], ders[8];
    bspline_span_basis(t.data(), p, k, u0 + h * sd, vals, ders);
    for (int j = 0; j <= p; ++j) {
      nb.push_back(vals[j]);
      nb.push_back(ders[j] * h);
    }
  }
  double* d_nb = nullptr;
  MSASM_CUDA(cudaMallocAsync(&d_nb, nb.size() * sizeof(double), st));
  MSASM_CUDA(cudaMemcpyAsync(d_nb, nb.data(), nb.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  a.geo.basis[d] = d_nb;
  a.geo.nq[d] = 1;
  int nP, nS, nU, nJ;
  jac_scratch_sizes(a.geo.np, a.geo.nq, nP, nS, nU, nJ);
  const int warps = 4;
  const size_t smem = warps * size_t(nP + nS + nU + nJ + a.geo.nq[a.ia] * a.geo.nq[a.ib]) * sizeof(double);
  msasm_status status = MSASM_OK;
  if (smem > 200 * 1024) status = fail(MSASM_EUNSUPPORTED, "macro degree / q too large for the traction kernel");
  cudaError_t e = cudaSuccess;
  if (status == MSASM_OK)
    e = cudaFuncSetAttribute(traction_load_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (status == MSASM_OK && e == cudaSuccess) {
    const int64_t n_face = int64_t(plan->n_elem[a.ia]) * plan->n_elem[a.ib];
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n_face + warps - 1) / warps, 152 * 16));
    traction_load_kernel<<<unsigned(blocks), 32 * warps, smem, st>>>(a);
    e = cudaGetLastError();
  }
  if (status == MSASM_OK && e != cudaSuccess) status = cuda_fail(e, "traction load kernel");
  cudaStreamSynchronize(st);                     // the host table outlives its copy
  cudaFreeAsync(d_nb, st);
  return status;
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
  return size_t(nP + nS + nU + nJ + g.nq[0] * g.nq[1] * g.nq[2]) * sizeof(double);
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
