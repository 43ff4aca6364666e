// Projection error of the macro field (Sec. 3.2.2, eq. 47-48; Sec. 3.3, eq. 59): for every tile,
// max over sample points xi_s of ||A_bar(xi_s) - Pi A_bar(xi_s)||_F / ||A_bar(xi_s)||_F over the 81
// components, Pi the interpolant at the (q1+1)(q2+1)(q3+1) nodes of given degrees (q1, q2, q3)
// (the reading of the projection used throughout; one degree per direction for the anisotropic
// space of Sec. 3.3.4) or the L2 projection onto that space of eq. 20-24 (l2_coef_gpu).  Samples:
// the uniform interior grid (s + 1/2)/n_s per direction.
// The exact field at the samples comes from the node Jacobians of the same sum factorisation
// with the macro basis tabulated at the samples; the interpolant from the pullback coefficients at
// the q nodes (computed with the macro basis tabulated at those nodes).  One warp per tile.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.h"
#include "macro_jacobian.cuh"

namespace msasm {

MacroTileArgs macro_tile_args(const msasm_plan* plan, const double* d_ctrl);
msasm_status pullback_geo_gpu(const MacroTileArgs& geo, int64_t n_tiles, double lam, double mu, double* d_coef,
                              unsigned long long* d_degenerate, cudaStream_t stream);
int bspline_find_span(const double* t, int n_knots, int p, double u);
void bspline_span_basis(const double* t, int p, int span, double u, double* vals, double* ders);
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w);

struct ProjErrArgs {
  MacroTileArgs geo;         // macro basis at the samples (n_s per direction)
  int64_t n_tiles;
  double lam, mu;
  const double* coef;        // pullback at the q nodes: [9t + 3a + b][9C + 3i + j]
  int nq[3];                 // q_d + 1
  const double* lag[3];      // per direction [s][c]: l_c(x_s), the 1-D Lagrange basis of its nodes at the samples
  double* err;               // per tile
};

__global__ void projection_error_kernel(ProjErrArgs a) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
  const int ns = a.geo.nq[0], n_s = ns * ns * ns;
  const int nq1 = a.nq[0], nq2 = a.nq[1], nq3 = a.nq[2], n_pi = nq1 * nq2 * nq3, K = 9 * n_pi;
  int nP, nS, nU, nJ;
  jac_scratch_sizes(a.geo.np, a.geo.nq, nP, nS, nU, nJ);
  double* P = smem + size_t(warp) * (nP + nS + nU + nJ);
  double* S = P + nP;
  double* U = S + nS;
  double* Js = U + nU;
  for (int64_t t = int64_t(blockIdx.x) * warps + warp; t < a.n_tiles; t += int64_t(gridDim.x) * warps) {
    tile_node_jacobians(a.geo, t, P, S, U, Js, lane);
    const double* ct = a.coef + size_t(9 * t) * K;
    double worst = 0.0;
    for (int sp = lane; sp < n_s; sp += 32) {
      const int s1 = sp % ns, s2 = (sp / ns) % ns, s3 = sp / (ns * ns);
      const double* J = Js + 9 * sp;
      const double det = det3(J);
      double G[9];
      inverse3(J, 1.0 / det, G);
      const double adet = fabs(det);
      double GG[9];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          GG[i * 3 + j] = G[i * 3] * G[j * 3] + G[i * 3 + 1] * G[j * 3 + 1] + G[i * 3 + 2] * G[j * 3 + 2];
      double d2 = 0.0, e2 = 0.0;
      for (int al = 0; al < 3; ++al)
        for (int be = 0; be < 3; ++be) {
          const double* row = ct + size_t(3 * al + be) * K;
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
              double ex = adet * (a.lam * G[i * 3 + al] * G[j * 3 + be] + a.mu * G[i * 3 + be] * G[j * 3 + al]);
              if (al == be) ex += adet * a.mu * GG[i * 3 + j];
              double ip = 0.0;
              for (int C = 0; C < n_pi; ++C) {
                const int c1 = C % nq1, c2 = (C / nq1) % nq2, c3 = C / (nq1 * nq2);
                const double l = a.lag[0][s1 * nq1 + c1] * a.lag[1][s2 * nq2 + c2] * a.lag[2][s3 * nq3 + c3];
                ip = fma(l, row[9 * C + 3 * i + j], ip);
              }
              d2 = fma(ex - ip, ex - ip, d2);
              e2 = fma(ex, ex, e2);
            }
        }
      worst = fmax(worst, sqrt(d2 / e2));
    }
    for (int o = 16; o; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    if (lane == 0) a.err[t] = worst;
    __syncwarp();
  }
}

// L2 projection onto Q_(q1,q2,q3) (eq. 20-24) in the Lagrange basis of the q_d+1 Gauss-Legendre
// nodes of each direction: the mass matrix int N_C N_D is diagonal there (each direction's node
// rule integrates its degree-2q_d integrand exactly, and N_C vanishes at the other nodes),
// M = diag(w_c1 w_c2 w_c3), so the coefficients of the projection with the load integrated by an
// n_g-point rule are
//   a_C = sum_g P1[c1][g1] P2[c2][g2] P3[c3][g3] A_bar(x_g),   Pd[c][g] = W_g l_c(x_g) / w_c,
// evaluated by sum factorisation (direction 1, then 2, then 3) in shared memory, one CTA per
// coefficient row (9 per tile: alpha, beta), the 9 components (i, j) side by side.
__global__ void l2_project_kernel(const double* __restrict__ vals, int64_t n_rows, int ng, int nq1, int nq2, int nq3,
                                  const double* __restrict__ Pall, double* __restrict__ coef) {
  extern __shared__ double sm[];
  const int Kg = 9 * ng * ng * ng, K = 9 * nq1 * nq2 * nq3;
  double* V = sm;                                // [(g1 + ng (g2 + ng g3)) 9 + k]
  double* T1 = V + Kg;                           // [(c1 + nq1 (g2 + ng g3)) 9 + k]
  double* T2 = T1 + 9 * nq1 * ng * ng;           // [(c1 + nq1 (c2 + nq2 g3)) 9 + k]
  double* P = T2 + 9 * nq1 * nq2 * ng;           // P1 [c][g], then P2, then P3
  const double* P1 = P;
  const double* P2 = P + nq1 * ng;
  const double* P3 = P2 + nq2 * ng;
  for (int i = threadIdx.x; i < (nq1 + nq2 + nq3) * ng; i += blockDim.x) P[i] = Pall[i];
  for (int64_t r = blockIdx.x; r < n_rows; r += gridDim.x) {
    __syncthreads();
    for (int i = threadIdx.x; i < Kg; i += blockDim.x) V[i] = vals[r * Kg + i];
    __syncthreads();
    for (int i = threadIdx.x; i < 9 * nq1 * ng * ng; i += blockDim.x) {
      const int k = i % 9, rest = i / 9, c1 = rest % nq1, g23 = rest / nq1;
      double acc = 0.0;
      for (int g1 = 0; g1 < ng; ++g1) acc = fma(P1[c1 * ng + g1], V[(g1 + ng * g23) * 9 + k], acc);
      T1[i] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 9 * nq1 * nq2 * ng; i += blockDim.x) {
      const int k = i % 9, rest = i / 9, c1 = rest % nq1, rest2 = rest / nq1, c2 = rest2 % nq2, g3 = rest2 / nq2;
      double acc = 0.0;
      for (int g2 = 0; g2 < ng; ++g2) acc = fma(P2[c2 * ng + g2], T1[(c1 + nq1 * (g2 + ng * g3)) * 9 + k], acc);
      T2[i] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
      const int k = i % 9, rest = i / 9, c12 = rest % (nq1 * nq2), c3 = rest / (nq1 * nq2);
      double acc = 0.0;
      for (int g3 = 0; g3 < ng; ++g3) acc = fma(P3[c3 * ng + g3], T2[(c12 + nq1 * nq2 * g3) * 9 + k], acc);
      coef[r * K + i] = acc;
    }
  }
}

__global__ void max_kernel(const double* __restrict__ x, int64_t n, double* __restrict__ out) {
  __shared__ double part[256];
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, x[i]);
  part[threadIdx.x] = m;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (int(threadIdx.x) < w) part[threadIdx.x] = fmax(part[threadIdx.x], part[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = part[0];
}

// macro basis tables of the plan's spans at the points x[d] of each direction (per direction
// [e][point][a][value, d/dxi])
static void basis_tables(const msasm_plan* plan, const std::vector<double> (&x)[3], std::vector<double> (&basis)[3]) {
  for (int d = 0; d < 3; ++d) {
    const std::vector<double>& t = plan->knots_host[d];
    const int p = plan->degree[d];
    basis[d].clear();
    for (int k : plan->span_host[d]) {
      const double u0 = t[size_t(k)], h = t[size_t(k) + 1] - t[size_t(k)];
      for (double xc : x[d]) {
        double vals[8], ders[8];
        bspline_span_basis(t.data(), p, k, u0 + h * xc, vals, ders);
        for (int a = 0; a <= p; ++a) {
          basis[d].push_back(vals[a]);
          basis[d].push_back(ders[a] * h);
        }
      }
    }
  }
}

// 1-D Lagrange basis of the n_c Gauss-Legendre nodes at the points x: [point][c]
static std::vector<double> lagrange_at(int n_c, const std::vector<double>& x) {
  std::vector<double> xn, wn, L(x.size() * size_t(n_c));
  gauss_legendre01(n_c, xn, wn);
  for (size_t i = 0; i < x.size(); ++i)
    for (int c = 0; c < n_c; ++c) {
      double l = 1.0;
      for (int k = 0; k < n_c; ++k)
        if (k != c) l *= (x[i] - xn[size_t(k)]) / (xn[size_t(c)] - xn[size_t(k)]);
      L[i * n_c + c] = l;
    }
  return L;
}

// The L2-projection coefficients of degrees q3 (layout of the pullback: [9t + 3a + b][9C + 3i + j])
// of all tiles, the load integrated by the n_g-point Gauss rule per direction.
msasm_status l2_coef_gpu(const msasm_plan* plan, const double* d_ctrl, const int q3[3], int n_g, double lam, double mu,
                         double* d_coef, cudaStream_t s) {
  for (int d = 0; d < 3; ++d)
    if (q3[d] < 0 || q3[d] > 7) return fail(MSASM_EINVAL, "need 0 <= q <= 7");
  if (n_g < 1 || n_g > 9) return fail(MSASM_EINVAL, "need 1 <= n_gauss <= 9");
  const int nq[3] = {q3[0] + 1, q3[1] + 1, q3[2] + 1};
  std::vector<double> xg, wg;
  gauss_legendre01(n_g, xg, wg);
  std::vector<double> xs[3] = {xg, xg, xg}, bg[3];
  basis_tables(plan, xs, bg);
  std::vector<double> Pall;                       // P1, P2, P3: [c][g] = W_g l_c(x_g) / w_c
  for (int d = 0; d < 3; ++d) {
    std::vector<double> xn, wn;
    gauss_legendre01(nq[d], xn, wn);
    const std::vector<double> L = lagrange_at(nq[d], xg);
    for (int c = 0; c < nq[d]; ++c)
      for (int g = 0; g < n_g; ++g) Pall.push_back(wg[size_t(g)] * L[size_t(g) * nq[d] + c] / wn[size_t(c)]);
  }
  const size_t n_rows = size_t(9 * plan->n_tiles), Kg = size_t(9) * n_g * n_g * n_g;
  size_t nb = Pall.size();
  for (int d = 0; d < 3; ++d) nb += bg[d].size();
  double* buf = nullptr;
  MSASM_CUDA(cudaMallocAsync(&buf, (nb + n_rows * Kg) * sizeof(double), s));
  double* cur = buf;
  auto put = [&](const std::vector<double>& v) -> double* {
    double* p = cur;
    cudaMemcpyAsync(p, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    cur += v.size();
    return p;
  };
  MacroTileArgs gg = macro_tile_args(plan, d_ctrl);
  for (int d = 0; d < 3; ++d) {
    gg.nq[d] = n_g;
    gg.basis[d] = put(bg[d]);
  }
  const double* d_P = put(Pall);
  double* vals = cur;                              // the field at the n_g^3 points of every tile
  msasm_status st = pullback_geo_gpu(gg, plan->n_tiles, lam, mu, vals, plan->d_degenerate, s);
  if (st == MSASM_OK) {
    const size_t smem = (Kg + size_t(9) * nq[0] * n_g * n_g + size_t(9) * nq[0] * nq[1] * n_g + Pall.size()) *
                        sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(l2_project_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e == cudaSuccess) {
      const unsigned blocks = unsigned(std::max<size_t>(1, std::min<size_t>(n_rows, 152 * 8)));
      l2_project_kernel<<<blocks, 256, smem, s>>>(vals, int64_t(n_rows), n_g, nq[0], nq[1], nq[2], d_P, d_coef);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) st = cuda_fail(e, "L2 projection kernel");
  }
  cudaStreamSynchronize(s);                      // the host tables outlive the copies
  cudaFreeAsync(buf, s);
  return st;
}

msasm_status projection_error_gpu(const msasm_plan* plan, const double* d_ctrl, const int q3[3], int n_s, double lam,
                                  double mu, double* d_err_tiles, double* d_err_max, cudaStream_t s, int n_gauss) {
  for (int d = 0; d < 3; ++d)
    if (q3[d] < 0 || q3[d] > 7) return fail(MSASM_EINVAL, "need 0 <= q <= 7 and 1 <= n_samples <= 8");
  if (n_s < 1 || n_s > 8) return fail(MSASM_EINVAL, "need 0 <= q <= 7 and 1 <= n_samples <= 8");
  if (n_gauss < 0 || n_gauss > 9) return fail(MSASM_EINVAL, "need 0 <= n_gauss <= 9");
  const int nq[3] = {q3[0] + 1, q3[1] + 1, q3[2] + 1}, K = 9 * nq[0] * nq[1] * nq[2];
  std::vector<double> xn[3], xs1(static_cast<size_t>(n_s));
  for (int d = 0; d < 3; ++d) {
    std::vector<double> wn;
    gauss_legendre01(nq[d], xn[d], wn);
  }
  for (int i = 0; i < n_s; ++i) xs1[size_t(i)] = (i + 0.5) / n_s;
  std::vector<double> xs[3] = {xs1, xs1, xs1}, bn[3], bs[3], lag[3];
  basis_tables(plan, xn, bn);
  basis_tables(plan, xs, bs);
  for (int d = 0; d < 3; ++d) lag[d] = lagrange_at(nq[d], xs1);
  size_t nb = 0;
  for (int d = 0; d < 3; ++d) nb += bn[d].size() + bs[d].size() + lag[d].size();
  const size_t coef_n = size_t(9 * plan->n_tiles) * K;
  double* buf = nullptr;
  MSASM_CUDA(cudaMallocAsync(&buf, (nb + coef_n + plan->n_tiles + 2) * sizeof(double), s));
  double* cur = buf;
  auto put = [&](const std::vector<double>& v) -> double* {
    double* p = cur;
    cudaMemcpyAsync(p, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    cur += v.size();
    return p;
  };
  MacroTileArgs gn = macro_tile_args(plan, d_ctrl), gs = gn;
  const double* d_lag[3];
  for (int d = 0; d < 3; ++d) {
    gn.nq[d] = nq[d];
    gs.nq[d] = n_s;
    gn.basis[d] = put(bn[d]);
    gs.basis[d] = put(bs[d]);
    d_lag[d] = put(lag[d]);
  }
  double* coef = cur;
  cur += coef_n;
  double* err = d_err_tiles ? d_err_tiles : cur;
  msasm_status st = n_gauss > 0 ? l2_coef_gpu(plan, d_ctrl, q3, n_gauss, lam, mu, coef, s)
                                 : pullback_geo_gpu(gn, plan->n_tiles, lam, mu, coef, plan->d_degenerate, s);
  if (st == MSASM_OK) {
    ProjErrArgs a;
    a.geo = gs;
    a.n_tiles = plan->n_tiles;
    a.lam = lam;
    a.mu = mu;
    a.coef = coef;
    for (int d = 0; d < 3; ++d) {
      a.nq[d] = nq[d];
      a.lag[d] = d_lag[d];
    }
    a.err = err;
    int nP, nS, nU, nJ;
    jac_scratch_sizes(gs.np, gs.nq, nP, nS, nU, nJ);
    const int warps = 2;
    const size_t smem = warps * size_t(nP + nS + nU + nJ) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(projection_error_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) st = cuda_fail(e, "projection error kernel");
    if (st == MSASM_OK) {
      const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((plan->n_tiles + warps - 1) / warps, 152 * 16));
      projection_error_kernel<<<unsigned(blocks), 32 * warps, smem, s>>>(a);
      if ((e = cudaGetLastError()) != cudaSuccess) st = cuda_fail(e, "projection error kernel");
    }
    if (st == MSASM_OK && d_err_max) {
      max_kernel<<<1, 256, 0, s>>>(err, plan->n_tiles, d_err_max);
      if ((e = cudaGetLastError()) != cudaSuccess) st = cuda_fail(e, "max");
    }
  }
  cudaStreamSynchronize(s);                      // the host tables outlive the copies
  cudaFreeAsync(buf, s);
  return st;
}

}  // namespace msasm
