// Adjoint of the assembly (Sec. 4.1.2, eq. 69-73): gradient of L(values) with respect to the
// macro control points, for L = u^T K u (d_u given) or a general L (dL/dvalues given).
//
//   1. G_t[m][a][b] = dL/dK_t[m][a][b]: for u, w_m v_{A,a} v_{B,b} with w_m = 2 for A != B
//      (the block and its transpose) and 1 for A = B, where v = u - u_ref(t) is u minus its value
//      at one reference point of the tile: K_t(P) annihilates translations for every P (the
//      rows of the table sum to zero, eq. 56-57 with sum_B R_B = 1), so u^T dK_t u = v^T dK_t v
//      exactly, while v avoids the cancellation of large rigid-body displacements in reduced
//      precision; for dL/dvalues, the sum of the two CSR entries the block is scattered to (the
//      adjoint of step 4).
//   2. W_t = mat[K]^T G_t (eq. 73 as a product of the lookup table and the state): the adjoint
//      field at the nodes, W_t[C][i][j][a][b] = sum_m T[m][C][i][j] G_t[m][a][b] (CUDA cores).
//   The same chain gives the volume gradient (Sec. 4.1.1, eq. 66-67) with W : A_bar replaced by
//   t_C |det J| (t the volume table): the adjoint field of the volume.
//   3. Per node: S = d(W : A_bar)/dJ through |det J| and G = J^-1 (FP64), and per control point
//      dL/dP_a,p = sum_C sum_q S_C[p][q] dB_a/dxi_q (xi_C), a transposed sum factorisation; tiles
//      sharing a control point add with FP64 atomics.
#include <cmath>

#include "common.h"
#include "macro_jacobian.cuh"

namespace msasm {

MacroTileArgs macro_tile_args(const msasm_plan* plan, const double* d_ctrl);
size_t pullback_smem_per_warp(const int np[3], const int nq[3]);

// ------------------------------------------------------------------ step 1: G from u or from dL/dvalues
template <typename T>
__global__ void grad_blocks_from_u_kernel(const T* __restrict__ u, int64_t t0, int64_t n_tiles, int n_nz, int ld,
                                          const int32_t* __restrict__ pairs, const int32_t* __restrict__ gmap,
                                          int n_T, int ref_point, T* __restrict__ Gm) {
  const int64_t total = n_tiles * n_nz;
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int64_t tl = idx / n_nz;
    const int m = int(idx % n_nz);
    const int A = pairs[2 * m], B = pairs[2 * m + 1];
    const int64_t gA = gmap[(t0 + tl) * n_T + A], gB = gmap[(t0 + tl) * n_T + B];
    const int64_t gR = gmap[(t0 + tl) * n_T + ref_point];
    const T w = (A == B) ? T(1) : T(2);
    T ua[3], ub[3];
    for (int k = 0; k < 3; ++k) {
      const T ur = u[3 * gR + k];
      ua[k] = u[3 * gA + k] - ur;
      ub[k] = u[3 * gB + k] - ur;
    }
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Gm[(9 * tl + 3 * a + b) * ld + m] = w * ua[a] * ub[b];
  }
}

template <typename T>
__global__ void grad_blocks_from_values_kernel(const T* __restrict__ gv, int64_t t0, int64_t n_tiles, int n_nz, int ld,
                                               const int32_t* __restrict__ pairs, const int32_t* __restrict__ gmap,
                                               int n_T, const uint32_t* __restrict__ rank,
                                               const int64_t* __restrict__ rowptr, T* __restrict__ Gm) {
  const int64_t total = n_tiles * n_nz;
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int64_t tl = idx / n_nz;
    const int m = int(idx % n_nz);
    const int64_t t = t0 + tl;
    const int A = pairs[2 * m], B = pairs[2 * m + 1];
    const int64_t gA = gmap[t * n_T + A], gB = gmap[t * n_T + B];
    const uint32_t w = rank[t * n_nz + m];
    const int ru = int(w & 0xffffu), rl = int((w >> 16) & 0x7fffu);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        T g = gv[rowptr[3 * gA + a] + 3 * ru + b];
        if (A != B) g += gv[rowptr[3 * gB + b] + 3 * rl + a];
        Gm[(9 * tl + 3 * a + b) * ld + m] = g;
      }
  }
}

// ------------------------------------------------------------------ transposed table copy
template <typename T>
__global__ void transpose_table_kernel(const double* __restrict__ Tm, int n_nz, int K, T* __restrict__ Tt) {
  __shared__ double tile[32][33];
  for (int by = blockIdx.y; by * 32 < n_nz; by += gridDim.y)
    for (int bx = blockIdx.x; bx * 32 < K; bx += gridDim.x) {
      const int m0 = by * 32, k0 = bx * 32;
      for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int m = m0 + r, k = k0 + threadIdx.x;
        tile[r][threadIdx.x] = (m < n_nz && k < K) ? Tm[size_t(m) * K + k] : 0.0;
      }
      __syncthreads();
      for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int k = k0 + r, m = m0 + threadIdx.x;
        if (k < K && m < n_nz) Tt[size_t(k) * n_nz + m] = T(tile[threadIdx.x][r]);
      }
      __syncthreads();
    }
}

// ------------------------------------------------------------------ step 3: chain rule to the control net
struct AdjointArgs {
  MacroTileArgs geo;
  int64_t t0, n_tiles;
  double lam, mu;
  const void* W;            // [9 tl + 3a + b][9C + 3i + j]
  int w_f32;
  const double* vol_w;      // volume mode (W unused): psi = t_C, the volume table (eq. 66-67)
  double* dP;               // (n_ctrl, 3), accumulated
};

__global__ void adjoint_pullback_kernel(AdjointArgs a) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
  const int nq1 = a.geo.nq[0], nq2 = a.geo.nq[1], nq3 = a.geo.nq[2], n_pi = nq1 * nq2 * nq3, K = 9 * n_pi;
  const int np1 = a.geo.np[0], np2 = a.geo.np[1], np3 = a.geo.np[2];
  int nP, nS, nU, nJ;
  jac_scratch_sizes(a.geo.np, a.geo.nq, nP, nS, nU, nJ);
  double* P = smem + size_t(warp) * (nP + nS + nU + nJ);
  double* S = P + nP;
  double* U = S + nS;
  double* Jn = U + nU;
  const double lam = a.lam, mu = a.mu;
  for (int64_t tl = int64_t(blockIdx.x) * warps + warp; tl < a.n_tiles; tl += int64_t(gridDim.x) * warps) {
    const int64_t t = a.t0 + tl;
    tile_node_jacobians(a.geo, t, P, S, U, Jn, lane);
    // per node: S_C[p][q] = d(W : A_bar)/dJ[p][q], written over Jn
    for (int c = lane; c < n_pi; c += 32) {
      double J[9], G[9];
      for (int k = 0; k < 9; ++k) J[k] = Jn[c * 9 + k];
      const double det = det3(J);
      inverse3(J, 1.0 / det, G);
      const double adet = fabs(det);
      auto Wv = [&](int i, int j, int al, int be) -> double {
        if (a.vol_w) return 0.0;
        const size_t off = size_t(9 * tl + 3 * al + be) * K + 9 * c + 3 * i + j;
        return a.w_f32 ? double(static_cast<const float*>(a.W)[off]) : static_cast<const double*>(a.W)[off];
      };
      double Wd[9];   // Wd[i][j] = sum_a W[i][j][a][a]
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Wd[i * 3 + j] = Wv(i, j, 0, 0) + Wv(i, j, 1, 1) + Wv(i, j, 2, 2);
      double GG[9];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          GG[i * 3 + j] = G[i * 3] * G[j * 3] + G[i * 3 + 1] * G[j * 3 + 1] + G[i * 3 + 2] * G[j * 3 + 2];
      double psi = 0.0, H[9];
      for (int k = 0; k < 9; ++k) H[k] = 0.0;
      if (a.vol_w) psi = a.vol_w[c];      // d(t_C |det J|)/dJ = t_C |det J| G^T: psi = t_C, H = 0
      for (int i = 0; i < 3 && !a.vol_w; ++i)
        for (int j = 0; j < 3; ++j) {
          psi += mu * Wd[i * 3 + j] * GG[i * 3 + j];
          for (int g = 0; g < 3; ++g) {      // d/dG[i][g] and d/dG[j][g] of mu Wd[i][j] (G G^T)[i][j]
            H[i * 3 + g] += mu * Wd[i * 3 + j] * G[j * 3 + g];
            H[j * 3 + g] += mu * Wd[i * 3 + j] * G[i * 3 + g];
          }
          for (int al = 0; al < 3; ++al)
            for (int be = 0; be < 3; ++be) {
              const double w = Wv(i, j, al, be);
              if (w == 0.0) continue;
              psi += w * (lam * G[i * 3 + al] * G[j * 3 + be] + mu * G[i * 3 + be] * G[j * 3 + al]);
              H[i * 3 + al] += w * lam * G[j * 3 + be];
              H[j * 3 + be] += w * lam * G[i * 3 + al];
              H[i * 3 + be] += w * mu * G[j * 3 + al];
              H[j * 3 + al] += w * mu * G[i * 3 + be];
            }
        }
      // S[p][q] = |det J| (psi G[q][p] - (G^T H G^T)[p][q])
      double GtH[9];
      for (int p = 0; p < 3; ++p)
        for (int g = 0; g < 3; ++g) GtH[p * 3 + g] = G[p] * H[g] + G[3 + p] * H[3 + g] + G[6 + p] * H[6 + g];
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) {
          const double ghg = GtH[p * 3] * G[q * 3] + GtH[p * 3 + 1] * G[q * 3 + 1] + GtH[p * 3 + 2] * G[q * 3 + 2];
          Jn[c * 9 + p * 3 + q] = adet * (psi * G[q * 3 + p] - ghg);
        }
    }
    __syncwarp();
    int e1, e2, e3;
    tile_coords(a.geo, t, e1, e2, e3);
    const double* B1 = a.geo.basis[0] + size_t(e1) * nq1 * np1 * 2;
    const double* B2 = a.geo.basis[1] + size_t(e2) * nq2 * np2 * 2;
    const double* B3 = a.geo.basis[2] + size_t(e3) * nq3 * np3 * 2;
    double* X = U;   // [q][c1][c2][a3][p]  (nU doubles)
    double* Y = S;   // [v][c1][a2][a3][p]  (nS doubles)
    for (int o = lane; o < nU; o += 32) {     // contract c3
      int p = o % 3, r = o / 3;
      int a3 = r % np3; r /= np3;
      int c2 = r % nq2; r /= nq2;
      int c1 = r % nq1;
      int q = r / nq1;
      const int v3 = (q == 2);
      double s = 0.0;
      for (int c3 = 0; c3 < nq3; ++c3)
        s = fma(Jn[(c1 + nq1 * (c2 + nq2 * c3)) * 9 + p * 3 + q], B3[(c3 * np3 + a3) * 2 + v3], s);
      X[o] = s;
    }
    __syncwarp();
    for (int o = lane; o < nS; o += 32) {     // contract c2: Y0 (d/dxi_1 branch), Y12 (value in xi_1)
      int p = o % 3, r = o / 3;
      int a3 = r % np3; r /= np3;
      int a2 = r % np2; r /= np2;
      int c1 = r % nq1;
      int v = r / nq1;
      double s = 0.0;
      for (int c2 = 0; c2 < nq2; ++c2) {
        const double x0 = X[(((0 * nq1 + c1) * nq2 + c2) * np3 + a3) * 3 + p];
        const double x1 = X[(((1 * nq1 + c1) * nq2 + c2) * np3 + a3) * 3 + p];
        const double x2 = X[(((2 * nq1 + c1) * nq2 + c2) * np3 + a3) * 3 + p];
        if (v == 0) s = fma(x0, B2[(c2 * np2 + a2) * 2], s);
        else s += x1 * B2[(c2 * np2 + a2) * 2 + 1] + x2 * B2[(c2 * np2 + a2) * 2];
      }
      Y[o] = s;
    }
    __syncwarp();
    const int f1 = a.geo.first[0][e1], f2 = a.geo.first[1][e2], f3 = a.geo.first[2][e3];
    for (int o = lane; o < nP; o += 32) {     // contract c1 and add into the global gradient
      int p = o % 3, c = o / 3;
      int a1 = c % np1, a2 = (c / np1) % np2, a3 = c / (np1 * np2);
      double s = 0.0;
      for (int c1 = 0; c1 < nq1; ++c1) {
        const double y0 = Y[(((0 * nq1 + c1) * np2 + a2) * np3 + a3) * 3 + p];
        const double y12 = Y[(((1 * nq1 + c1) * np2 + a2) * np3 + a3) * 3 + p];
        s += y0 * B1[(c1 * np1 + a1) * 2 + 1] + y12 * B1[(c1 * np1 + a1) * 2];
      }
      const int64_t gi = (f1 + a1) + int64_t(a.geo.n_ctrl_dir[0]) * ((f2 + a2) + int64_t(a.geo.n_ctrl_dir[1]) * (f3 + a3));
      atomicAdd(&a.dP[gi * 3 + p], s);
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------ launchers
template <typename T>
msasm_status grad_blocks_gpu(const msasm_plan* plan, const T* d_u, const T* d_gv, int64_t t0, int64_t nt, int ld,
                             T* d_G, cudaStream_t s) {
  const msasm_tables* tab = plan->tab;
  int64_t total = nt * tab->n_nz;
  int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 16);
  if (d_u)
    grad_blocks_from_u_kernel<T><<<unsigned(blocks), 256, 0, s>>>(d_u, t0, nt, tab->n_nz, ld, tab->d_pairs,
                                                                  plan->d_gmap, tab->topo.n_T, tab->ref_point, d_G);
  else
    grad_blocks_from_values_kernel<T><<<unsigned(blocks), 256, 0, s>>>(d_gv, t0, nt, tab->n_nz, ld, tab->d_pairs,
                                                                       plan->d_gmap, tab->topo.n_T, plan->d_rank,
                                                                       plan->d_rowptr, d_G);
  MSASM_CUDA(cudaGetLastError());
  return MSASM_OK;
}
template msasm_status grad_blocks_gpu<double>(const msasm_plan*, const double*, const double*, int64_t, int64_t, int,
                                              double*, cudaStream_t);
template msasm_status grad_blocks_gpu<float>(const msasm_plan*, const float*, const float*, int64_t, int64_t, int,
                                             float*, cudaStream_t);

template <typename T>
msasm_status transpose_table_gpu(const double* d_T, int n_nz, int K, T* d_Tt, cudaStream_t s) {
  dim3 block(32, 8), grid(unsigned((K + 31) / 32), unsigned(std::min((n_nz + 31) / 32, 4096)));
  transpose_table_kernel<T><<<grid, block, 0, s>>>(d_T, n_nz, K, d_Tt);
  MSASM_CUDA(cudaGetLastError());
  return MSASM_OK;
}
template msasm_status transpose_table_gpu<double>(const double*, int, int, double*, cudaStream_t);
template msasm_status transpose_table_gpu<float>(const double*, int, int, float*, cudaStream_t);

msasm_status adjoint_pullback_gpu(const msasm_plan* plan, const double* d_ctrl, double lam, double mu, int64_t t0,
                                  int64_t nt, const void* d_W, bool w_f32, double* d_dP, cudaStream_t s,
                                  const double* vol_w) {
  AdjointArgs a;
  a.geo = macro_tile_args(plan, d_ctrl);
  a.t0 = t0;
  a.n_tiles = nt;
  a.lam = lam;
  a.mu = mu;
  a.W = d_W;
  a.w_f32 = w_f32 ? 1 : 0;
  a.vol_w = vol_w;
  a.dP = d_dP;
  const int warps = 4;
  const size_t smem = warps * pullback_smem_per_warp(a.geo.np, a.geo.nq);
  if (smem > 200 * 1024) return fail(MSASM_EUNSUPPORTED, "macro degree / q too large for the adjoint kernel");
  MSASM_CUDA(cudaFuncSetAttribute(adjoint_pullback_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((nt + warps - 1) / warps, 152 * 16));
  adjoint_pullback_kernel<<<unsigned(blocks), 32 * warps, smem, s>>>(a);
  MSASM_CUDA(cudaGetLastError());
  return MSASM_OK;
}

}  // namespace msasm
