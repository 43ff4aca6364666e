// K1: the stiffness lookup table mat[K] (eq. 51-52, 57) in FP64 on the GPU, and the load (body and
// face terms) and volume tables of eq. 54-55 and 18 from the same 1-D integrals.
//
// Every micro patch is an axis-aligned box with an affine map and a tensor-product
// basis, and the projection basis N_C is a tensor product too, so the 3-D
// integral of eq. 52 over one patch factorises into three 1-D integrals:
//
//   int_patch d_i phi_A d_j phi_B N_C dxi = prod_d I_p,d[i==d, j==d][a_d, b_d, c_d],
//   I_p,d[da, db][a, b, c] = int_{lo_d}^{hi_d} f_a^(da) f_b^(db) l_c dxi_d.
//
// Stage 1 computes the small 1-D tables by Gauss quadrature per element (exact:
// the integrand is a polynomial of degree <= 2 p_T + q on each element); stage 2
// writes every table entry as a sum over the patches holding both functions of
// the pair (up to four: a point on a corner of the centre cube is in four patches).  Both stages are FP64.
#include <cstdio>
#include <vector>

#include "common.h"

namespace msasm {

struct Table1DParams {
  int n_patches, nf_max, n_gauss;
  int nq[3];                 // interpolation nodes per direction (q_d + 1)
  int nq_max;                // stride of the node index in the 1-D tables
  int degree[16][3];
  int n_elem[16][3];
  double lo[16][3], hi[16][3];
  double gx[16], gw[16];     // Gauss rule on [0,1]
  double nodes[3][8];        // interpolation nodes on [0,1], per direction
};

// node index of table column C, C = c1 + nq1 (c2 + nq2 c3)
__device__ inline void node_index(int C, const int nq[3], int cc[3]) {
  cc[0] = C % nq[0];
  cc[1] = (C / nq[0]) % nq[1];
  cc[2] = C / (nq[0] * nq[1]);
}

// Nonzero basis functions (values and d/ds) of the open uniform knot vector with n
// elements and degree p on element e (span e + p); knot k = clamp((k - p)/n, 0, 1).
__device__ inline void uniform_span_basis(int p, int n, int e, double s, double* N, double* dN) {
  auto knot = [&](int k) { return fmin(fmax(double(k - p) / n, 0.0), 1.0); };
  int span = e + p;
  double left[8], right[8], low[8];
  // degree p - 1 values first (for derivatives), then degree p
  for (int deg = (p > 0 ? p - 1 : 0); deg <= p; ++deg) {
    double* out = (deg == p) ? N : low;
    out[0] = 1.0;
    for (int j = 1; j <= deg; ++j) {
      left[j] = s - knot(span + 1 - j);
      right[j] = knot(span + j) - s;
      double carry = 0.0;
      for (int r = 0; r < j; ++r) {
        double f = out[r] / (right[r + 1] + left[j - r]);
        out[r] = carry + right[r + 1] * f;
        carry = left[j - r] * f;
      }
      out[j] = carry;
    }
    if (p == 0) break;
  }
  for (int k = 0; k <= p; ++k) {
    if (p == 0) { dN[k] = 0.0; continue; }
    int i = span - p + k;
    double a = (k >= 1) ? low[k - 1] : 0.0;
    double b = (k <= p - 1) ? low[k] : 0.0;
    double da = knot(i + p) - knot(i), db = knot(i + p + 1) - knot(i + 1);
    dN[k] = (da > 0 ? p * a / da : 0.0) - (db > 0 ? p * b / db : 0.0);
  }
}

__global__ void table_1d_kernel(Table1DParams prm, double* __restrict__ I1) {
  const int nq = prm.nq_max, nf = prm.nf_max;
  const int64_t total = int64_t(prm.n_patches) * 3 * 4 * nf * nf * nq;
  int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int c = int(idx % nq);
  int64_t r = idx / nq;
  int b = int(r % nf); r /= nf;
  int a = int(r % nf); r /= nf;
  int flag = int(r % 4); r /= 4;
  int d = int(r % 3);
  int p = int(r / 3);
  int deg = prm.degree[p][d], ne = prm.n_elem[p][d];
  int nfun = ne + deg;
  double acc = 0.0;
  if (a < nfun && b < nfun && c < prm.nq[d]) {
    double lo = prm.lo[p][d], h = prm.hi[p][d] - prm.lo[p][d];
    int da = flag >> 1, db = flag & 1;
    for (int e = 0; e < ne; ++e) {
      if (a < e || a > e + deg || b < e || b > e + deg) continue;
      for (int g = 0; g < prm.n_gauss; ++g) {
        double s = (e + prm.gx[g]) / ne;
        double N[8], dN[8];
        uniform_span_basis(deg, ne, e, s, N, dN);
        double fa = da ? dN[a - e] / h : N[a - e];   // d/dxi = (1/h) d/ds
        double fb = db ? dN[b - e] / h : N[b - e];
        double xi = lo + h * s;
        double lc = 1.0;
        for (int k = 0; k < prm.nq[d]; ++k)
          if (k != c) lc *= (xi - prm.nodes[d][k]) / (prm.nodes[d][c] - prm.nodes[d][k]);
        acc += prm.gw[g] / ne * h * fa * fb * lc;    // dxi = h ds, element length 1/ne in s
      }
    }
  }
  I1[idx] = acc;
}

__global__ void table_assemble_kernel(const PairDesc* __restrict__ desc, const double* __restrict__ I1,
                                      int n_nz, Table1DParams prm, double* __restrict__ T) {
  const int nq = prm.nq_max, nf = prm.nf_max, n_pi = prm.nq[0] * prm.nq[1] * prm.nq[2], row = 9 * n_pi;
  const int64_t total = int64_t(n_nz) * row;
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += int64_t(gridDim.x) * blockDim.x) {
    int m = int(idx / row);
    int k = int(idx % row);
    int C = k / 9, i = (k % 9) / 3, j = k % 3;
    int cc[3];
    node_index(C, prm.nq, cc);
    PairDesc pd = desc[m];
    double v = 0.0;
    for (int s = 0; s < kMaxPairPatches; ++s) {
      int p = pd.patch[s];
      if (p < 0) continue;
      double prod = 1.0;
      for (int d = 0; d < 3; ++d) {
        int flag = (i == d ? 2 : 0) + (j == d ? 1 : 0);
        int64_t off = ((((int64_t(p) * 3 + d) * 4 + flag) * nf + pd.a[s][d]) * nf + pd.b[s][d]) * nq + cc[d];
        prod *= I1[off];
      }
      v += prod;
    }
    T[idx] = v;
  }
}

// The load table of eq. 54-55 (F = 0): F[A][C] = int R_A N_C over the tile.  The basis of a patch
// sums to one in each direction, so the 1-D factor int f_a l_c is the sum over b of the value-value
// table int f_a f_b l_c; the patches holding A are those of the diagonal pair (A, A).
__global__ void load_table_kernel(const PairDesc* __restrict__ diag, const double* __restrict__ I1, int n_T,
                                  Table1DParams prm, double* __restrict__ F) {
  const int nq = prm.nq_max, nf = prm.nf_max, n_pi = prm.nq[0] * prm.nq[1] * prm.nq[2];
  const int64_t total = int64_t(n_T) * n_pi;
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int A = int(idx / n_pi), C = int(idx % n_pi);
    int cc[3];
    node_index(C, prm.nq, cc);
    const PairDesc pd = diag[A];
    double v = 0.0;
    for (int s = 0; s < kMaxPairPatches; ++s) {
      const int p = pd.patch[s];
      if (p < 0) continue;
      double prod = 1.0;
      for (int d = 0; d < 3; ++d) {
        double f1 = 0.0;
        for (int b = 0; b < nf; ++b)
          f1 += I1[((((int64_t(p) * 3 + d) * 4 + 0) * nf + pd.a[s][d]) * nf + b) * nq + cc[d]];
        prod *= f1;
      }
      v += prod;
    }
    F[idx] = v;
  }
}

// The face load tables of eq. 54-55 (F >= 1): for the cube face xi_d = s (face 2 d + s),
// Ff[A][C2] = int over the tile boundary lying on that face of R_A N_C2, N_C2 = l_ca(xi_ia) l_cb(xi_ib)
// the Lagrange basis of the face's (q_ia+1)(q_ib+1) nodes (ia < ib the in-face directions), face f
// at offset face_off[f] (n_T rows of its node count each).  A patch whose
// box reaches the face contributes when A's index in the normal direction is the end one there
// (open knots: that function is 1 on the face, the others 0); the in-face factors are the 1-D
// integrals int f_a l_c of the load table (sums over b of the value-value table).
__global__ void face_table_kernel(Table1DParams prm, const PairDesc* __restrict__ diag, const double* __restrict__ I1,
                                  int n_T, double* __restrict__ Ff) {
  const int nq = prm.nq_max, nf = prm.nf_max;
  int64_t face_off[7];
  face_off[0] = 0;
  for (int f = 0; f < 6; ++f) {
    const int d = f / 2, ia = d == 0 ? 1 : 0, ib = d == 2 ? 1 : 2;
    face_off[f + 1] = face_off[f] + int64_t(n_T) * prm.nq[ia] * prm.nq[ib];
  }
  const int64_t total = face_off[6];
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += int64_t(gridDim.x) * blockDim.x) {
    int face = 0;
    while (idx >= face_off[face + 1]) ++face;
    const int d = face / 2, sd = face % 2;
    const int ia = d == 0 ? 1 : 0, ib = d == 2 ? 1 : 2;
    const int n2 = prm.nq[ia] * prm.nq[ib];
    const int rest = int(idx - face_off[face]);
    const int A = rest / n2, C2 = rest % n2;
    const int ca = C2 % prm.nq[ia], cb = C2 / prm.nq[ia];
    const PairDesc pd = diag[A];
    double v = 0.0;
    for (int sl = 0; sl < kMaxPairPatches; ++sl) {
      const int p = pd.patch[sl];
      if (p < 0) continue;
      const bool reaches = sd == 0 ? prm.lo[p][d] == 0.0 : prm.hi[p][d] == 1.0;
      const int end = sd == 0 ? 0 : prm.n_elem[p][d] + prm.degree[p][d] - 1;
      if (!reaches || pd.a[sl][d] != end) continue;
      double fa = 0.0, fb = 0.0;
      for (int b = 0; b < nf; ++b) {
        fa += I1[((((int64_t(p) * 3 + ia) * 4 + 0) * nf + pd.a[sl][ia]) * nf + b) * nq + ca];
        fb += I1[((((int64_t(p) * 3 + ib) * 4 + 0) * nf + pd.a[sl][ib]) * nf + b) * nq + cb];
      }
      v += fa * fb;
    }
    Ff[idx] = v;
  }
}

// The volume table of eq. 18: t_C = int N_C over the tile = sum_A F[A][C] (the basis sums to one).
__global__ void volume_table_kernel(const double* __restrict__ F, int n_T, int n_pi, double* __restrict__ vol) {
  for (int C = blockIdx.x * blockDim.x + threadIdx.x; C < n_pi; C += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int A = 0; A < n_T; ++A) s += F[int64_t(A) * n_pi + C];
    vol[C] = s;
  }
}

msasm_status build_table_gpu(msasm_tables* tab, cudaStream_t stream) {
  const TileTopology& topo = tab->topo;
  const int q = tab->q, nq = q + 1;             // q: the largest of the per-direction degrees
  Table1DParams prm{};
  prm.n_patches = int(topo.patches.size());
  prm.nq_max = nq;
  for (int d = 0; d < 3; ++d) prm.nq[d] = tab->qd[d] + 1;
  int p_T = 0, nf_max = 0;
  for (int p = 0; p < prm.n_patches; ++p)
    for (int d = 0; d < 3; ++d) {
      const Patch& P = topo.patches[p];
      prm.degree[p][d] = P.degree[d];
      prm.n_elem[p][d] = P.n_elem[d];
      prm.lo[p][d] = P.lo[d];
      prm.hi[p][d] = P.hi[d];
      p_T = std::max(p_T, P.degree[d]);
      nf_max = std::max(nf_max, P.n_fun[d]);
    }
  prm.nf_max = nf_max;
  int ng = tab->n_gauss > 0 ? tab->n_gauss : (2 * p_T + q + 2) / 2;
  if (ng > 16) return fail(MSASM_EINVAL, "n_gauss must be <= 16");
  tab->n_gauss = ng;
  std::vector<double> gx, gw;
  gauss_legendre01(ng, gx, gw);
  for (int g = 0; g < ng; ++g) { prm.gx[g] = gx[g]; prm.gw[g] = gw[g]; }
  prm.n_gauss = ng;
  for (int d = 0; d < 3; ++d) {
    std::vector<double> nx, nw;
    gauss_legendre01(prm.nq[d], nx, nw);
    for (int c = 0; c < prm.nq[d]; ++c) prm.nodes[d][c] = nx[c];
  }

  // pair descriptors: patches holding both functions of the pair, with local indices
  std::vector<std::vector<std::pair<int, int>>> where(topo.n_T);   // (patch, local function)
  for (int p = 0; p < prm.n_patches; ++p)
    for (size_t f = 0; f < topo.patches[p].ids.size(); ++f) where[topo.patches[p].ids[f]].push_back({p, int(f)});
  std::vector<PairDesc> desc(tab->n_nz);
  for (int m = 0; m < tab->n_nz; ++m) {
    PairDesc pd;
    for (int s = 0; s < kMaxPairPatches; ++s) {
      pd.patch[s] = -1;
      for (int d = 0; d < 3; ++d) pd.a[s][d] = pd.b[s][d] = 0;
    }
    for (int k = 0; k < 4; ++k) pd.pad[k] = 0;
    int s = 0;
    for (auto& wa : where[topo.pair_A[m]])
      for (auto& wb : where[topo.pair_B[m]]) {
        if (wa.first != wb.first) continue;
        if (s >= kMaxPairPatches) return fail(MSASM_EUNSUPPORTED, "a pair lies in more than four patches");
        const Patch& P = topo.patches[wa.first];
        pd.patch[s] = int8_t(wa.first);
        int fa = wa.second, fb = wb.second;
        pd.a[s][0] = int8_t(fa % P.n_fun[0]);
        pd.a[s][1] = int8_t((fa / P.n_fun[0]) % P.n_fun[1]);
        pd.a[s][2] = int8_t(fa / (P.n_fun[0] * P.n_fun[1]));
        pd.b[s][0] = int8_t(fb % P.n_fun[0]);
        pd.b[s][1] = int8_t((fb / P.n_fun[0]) % P.n_fun[1]);
        pd.b[s][2] = int8_t(fb / (P.n_fun[0] * P.n_fun[1]));
        ++s;
      }
    desc[m] = pd;
  }
  int64_t n1 = int64_t(prm.n_patches) * 3 * 4 * nf_max * nf_max * nq;
  double* d_I1 = nullptr;
  PairDesc* d_desc = nullptr;
  MSASM_CUDA(cudaMallocAsync(&d_I1, n1 * sizeof(double), stream));
  MSASM_CUDA(cudaMallocAsync(&d_desc, desc.size() * sizeof(PairDesc), stream));
  MSASM_CUDA(cudaMemcpyAsync(d_desc, desc.data(), desc.size() * sizeof(PairDesc), cudaMemcpyHostToDevice, stream));
  table_1d_kernel<<<unsigned((n1 + 127) / 128), 128, 0, stream>>>(prm, d_I1);
  MSASM_CUDA(cudaGetLastError());
  table_assemble_kernel<<<152 * 8, 256, 0, stream>>>(d_desc, d_I1, tab->n_nz, prm, tab->d_T);
  MSASM_CUDA(cudaGetLastError());
  // load and volume tables from the same 1-D integrals
  std::vector<PairDesc> diag(topo.n_T);
  for (int m = 0; m < tab->n_nz; ++m)
    if (topo.pair_A[m] == topo.pair_B[m]) diag[topo.pair_A[m]] = desc[m];
  const int n_pi = tab->n_pi;
  PairDesc* d_diag = nullptr;
  MSASM_CUDA(cudaMallocAsync(&d_diag, diag.size() * sizeof(PairDesc), stream));
  MSASM_CUDA(cudaMemcpyAsync(d_diag, diag.data(), diag.size() * sizeof(PairDesc), cudaMemcpyHostToDevice, stream));
  MSASM_CUDA(cudaMalloc(&tab->d_F, size_t(topo.n_T) * n_pi * sizeof(double)));
  MSASM_CUDA(cudaMalloc(&tab->d_vol, size_t(n_pi) * sizeof(double)));
  load_table_kernel<<<152 * 2, 256, 0, stream>>>(d_diag, d_I1, topo.n_T, prm, tab->d_F);
  MSASM_CUDA(cudaGetLastError());
  volume_table_kernel<<<(n_pi + 127) / 128, 128, 0, stream>>>(tab->d_F, topo.n_T, n_pi, tab->d_vol);
  MSASM_CUDA(cudaGetLastError());
  MSASM_CUDA(cudaMalloc(&tab->d_Fface, size_t(tab->face_off[6]) * sizeof(double)));
  face_table_kernel<<<152 * 2, 256, 0, stream>>>(prm, d_diag, d_I1, topo.n_T, tab->d_Fface);
  MSASM_CUDA(cudaGetLastError());
  MSASM_CUDA(cudaFreeAsync(d_I1, stream));
  MSASM_CUDA(cudaFreeAsync(d_desc, stream));
  MSASM_CUDA(cudaFreeAsync(d_diag, stream));
  MSASM_CUDA(cudaStreamSynchronize(stream));   // `desc` and `diag` (host) must outlive the copies
  return MSASM_OK;
}

}  // namespace msasm
