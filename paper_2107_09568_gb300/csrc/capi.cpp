// The C ABI of include/msasm.h: argument checking, handle lifetime, and the
// sequencing of the kernels of one assembly (pullback -> contraction -> scatter).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "common.h"

namespace msasm {

static thread_local std::string g_error;

void set_error(const std::string& msg) { g_error = msg; }
msasm_status fail(msasm_status st, const std::string& msg) {
  g_error = msg;
  return st;
}
msasm_status cuda_fail(cudaError_t err, const char* what) {
  g_error = std::string(what) + ": " + cudaGetErrorName(err) + " (" + cudaGetErrorString(err) + ")";
  return err == cudaErrorMemoryAllocation ? MSASM_ENOMEM : MSASM_ECUDA;
}

// kernels (other translation units)
msasm_status build_table_gpu(msasm_tables* tab, cudaStream_t stream);
void number_points(const TileTopology& topo, const int n_elem[3], std::vector<int32_t>& gmap, int64_t& n_points);
void point_pattern(const TileTopology& topo, const int n_elem[3], const std::vector<int32_t>& gmap,
                   int64_t n_points, std::vector<int64_t>& pptr, std::vector<int32_t>& pcol);
msasm_status structure_expand_gpu(int64_t n_points, const int64_t* d_pptr, const int32_t* d_pcol,
                                  int64_t* d_rowptr, int32_t* d_col, cudaStream_t stream);
msasm_status secondary_entries_gpu(msasm_plan* plan, cudaStream_t stream);
msasm_status scatter_maps_gpu(msasm_plan* plan, const int64_t* d_type_rep, int n_types, unsigned long long* d_bad,
                              cudaStream_t stream);
msasm_status rank_map_gpu(const int32_t* d_gmap, const int32_t* d_pairs, const uint8_t* d_pair_face,
                          const int64_t* d_pptr, const int32_t* d_pcol, int64_t n_tiles, int n_T, int n_nz,
                          int nx, int ny, uint32_t* d_rank, unsigned long long* d_bad, cudaStream_t stream);
msasm_status pullback_gpu(const msasm_plan* plan, const double* d_ctrl, double lam, double mu, int64_t t0,
                          int64_t n_tiles, double* d_coef, cudaStream_t stream);
msasm_status contract_simt_f64(const double* d_coef, const double* d_T, int64_t n_tiles, int n_nz, int K,
                               int ld_nz, double* d_nz, cudaStream_t stream);
msasm_status contract_simt_f32(const float* d_coef, const float* d_T, int64_t n_tiles, int n_nz, int K,
                               int ld_nz, float* d_nz, cudaStream_t stream);
msasm_status to_f32_gpu(const double* x, int64_t n, float* y, cudaStream_t stream);
template <typename T>
msasm_status scatter_pass_gpu(const msasm_plan* plan, const T* d_nz, int ld_nz, int64_t t0, int64_t n_tiles,
                              T* d_values, cudaStream_t stream);
template <typename T>
msasm_status scatter_pass_gpu(const msasm_plan* plan, const T* d_nz, int ld_nz, int64_t t0, int64_t n_tiles,
                              T* d_values, int64_t direct_end, int64_t v_lo, int64_t v_hi, cudaStream_t stream);
msasm_status build_scatter_plan(msasm_plan* plan, const std::vector<int32_t>& gmap, const std::vector<int64_t>& pptr,
                                ScatterPlanHost& out);
template <typename T>
msasm_status gemm_simt(const T* A, int64_t lda, const T* B, int64_t ldb, int64_t N, int M, int K, T* C, int64_t ldc,
                       cudaStream_t stream);
template <typename T>
msasm_status grad_blocks_gpu(const msasm_plan* plan, const T* d_u, const T* d_gv, int64_t t0, int64_t nt, int ld,
                             T* d_G, cudaStream_t s);
template <typename T>
msasm_status transpose_table_gpu(const double* d_T, int n_nz, int K, T* d_Tt, cudaStream_t s);
msasm_status adjoint_pullback_gpu(const msasm_plan* plan, const double* d_ctrl, double lam, double mu, int64_t t0,
                                  int64_t nt, const void* d_W, bool w_f32, double* d_dP, cudaStream_t s,
                                  const double* vol_w = nullptr);
msasm_status linop_prepare_gpu(msasm_plan* plan, cudaStream_t s);
msasm_status projection_error_gpu(const msasm_plan* plan, const double* d_ctrl, const int q3[3], int n_s, double lam,
                                  double mu, double* d_err_tiles, double* d_err_max, cudaStream_t s, int n_gauss = 0);
msasm_status l2_coef_gpu(const msasm_plan* plan, const double* d_ctrl, const int q3[3], int n_g, double lam, double mu,
                         double* d_coef, cudaStream_t s);
template <typename T>
msasm_status linop_pass_gpu(const msasm_plan* plan, const T* d_nz, int ld_nz, int64_t t0, int64_t n_tiles,
                            const double* d_u, double* d_y, cudaStream_t s);
msasm_status volume_load_gpu(const msasm_plan* plan, const double* d_ctrl, double* d_tile_vol, double* d_total,
                             double* d_f, const double b[3], cudaStream_t s);
msasm_status traction_load_gpu(const msasm_plan* plan, const double* d_ctrl, int face, const double t[3], double* d_f,
                               cudaStream_t s);
int tc_kind_of(msasm_precision prec);
int emu_kpad(int K);
size_t emu_slice_bytes(int64_t rows, int K, int n_slices = 7);
msasm_status emu_slice_gpu(const double* x, int64_t rows, int64_t ldx, int K, void* slices, int* scale_exp,
                           cudaStream_t s, int n_slices = 7);
msasm_status contract_emu_gpu(const void* a_slices, const int* a_exp, int M, const void* b_slices, const int* b_exp,
                              int64_t N, int K, void* out, int ld, bool accumulate, bool blocks, unsigned* d_err,
                              cudaStream_t s, int n_slices = 7);
msasm_status contract_tc_linop_gpu(int kind, const void* a_hi, const void* a_lo, const float* a_scale, int M,
                                   const void* b_hi, const void* b_lo, const float* b_scale, int64_t N, int K,
                                   const double* u, double* y, const int32_t* gmap, const int32_t* pairs, int n_T,
                                   int64_t t0, unsigned* d_err, cudaStream_t s);
msasm_status contract_emu_linop_gpu(const void* a_slices, const int* a_exp, int M, const void* b_slices,
                                    const int* b_exp, int64_t N, int K, const double* u, double* y,
                                    const int32_t* gmap, const int32_t* pairs, int n_T, int64_t t0, unsigned* d_err,
                                    cudaStream_t s);
int tc_kpad(int K, int kind);
size_t tc_slice_bytes(int64_t rows, int K, int kind);
msasm_status tc_split_gpu(const double* x, int64_t rows, int K, int kind, void* hi, void* lo, float* row_scale,
                          cudaStream_t s);
msasm_status contract_tc_gpu(int kind, const void* a_hi, const void* a_lo, const float* a_scale, int M,
                             const void* b_hi, const void* b_lo, const float* b_scale, int64_t N, int K, float* out,
                             int ld, bool blocks, unsigned* d_err, cudaStream_t s);


static bool is_f64_precision(msasm_precision p) { return p == MSASM_F64 || p == MSASM_F64_EMU; }

}  // namespace msasm

using namespace msasm;

msasm_tables::~msasm_tables() {
  cudaFree(d_T);
  cudaFree(d_F);
  cudaFree(d_vol);
  cudaFree(d_Fface);
  cudaFree(d_pairs);
  cudaFree(d_T32);
  cudaFree(d_Thi);
  cudaFree(d_Tlo);
  cudaFree(d_Tscale);
  cudaFree(d_Tt);
  cudaFree(d_Tt32);
  cudaFree(d_Tslices);
  cudaFree(d_Tslice_scale);
  cudaFree(d_Tslices4);
  cudaFree(d_Tslice_scale4);
}

msasm_plan::~msasm_plan() {
  for (int d = 0; d < 3; ++d) {
    cudaFree(d_basis[d]);
    cudaFree(d_first[d]);
  }
  cudaFree(d_gmap);
  cudaFree(d_rowptr);
  cudaFree(d_col);
  cudaFree(d_rank);
  cudaFree(d_tile_type);
  cudaFree(d_type_nvals);
  cudaFree(d_type_map_off);
  cudaFree(d_maps);
  cudaFree(d_tile_vbase);
  cudaFree(d_tmpl);
  cudaFree(d_tmpl_ptr);
  cudaFree(d_sec_off);
  cudaFree(d_colmaps);
  cudaFree(d_type_rows);
  cudaFree(d_type_row_off);
  cudaFree(d_sec);
  cudaFree(d_coef);
  cudaFree(d_nz);
  cudaFree(d_coef_lp);
  cudaFree(d_adj_lp);
  cudaFree(d_degenerate);
  cudaFree(d_tc_err);
  cudaFree(d_ctrl_stage);
  cudaFree(d_values_stage);
  for (cudaEvent_t e : events) cudaEventDestroy(e);
  for (cudaEvent_t e : copy_events) cudaEventDestroy(e);
  for (cudaEvent_t e : scatter_ev)
    if (e) cudaEventDestroy(e);
  if (scatter_side) cudaStreamDestroy(scatter_side);
  for (int k = 0; k < 2; ++k)
    if (copy_stream[k]) cudaStreamDestroy(copy_stream[k]);
}

namespace msasm {

// Everything of a table object but the tables themselves: the tile topology, degrees and sizes,
// the device table d_T (allocated, not filled) and the pair list (filled).  Synchronises `s`.
msasm_status tables_init(const msasm_micro_desc* micro, const int32_t q3[3], int n_gauss, cudaStream_t s,
                         msasm_tables* tab) {
  for (int d = 0; d < 3; ++d)
    if (q3[d] < 0 || q3[d] > 5) return fail(MSASM_EINVAL, "interpolation degrees must be in 0..5");
  MSASM_TRY(build_topology(micro, tab->topo));
  for (int d = 0; d < 3; ++d) tab->qd[d] = q3[d];
  tab->q = std::max({q3[0], q3[1], q3[2]});
  tab->n_pi = (q3[0] + 1) * (q3[1] + 1) * (q3[2] + 1);
  tab->face_off[0] = 0;
  for (int f = 0; f < 6; ++f) {
    const int d = f / 2, ia = d == 0 ? 1 : 0, ib = d == 2 ? 1 : 2;
    tab->face_off[f + 1] = tab->face_off[f] + int64_t(tab->topo.n_T) * (q3[ia] + 1) * (q3[ib] + 1);
  }
  double best = 1e300;
  for (int A = 0; A < tab->topo.n_T; ++A) {
    double d2 = 0.0;
    for (int k = 0; k < 3; ++k) d2 += (tab->topo.pos[3 * A + k] - 0.5) * (tab->topo.pos[3 * A + k] - 0.5);
    if (d2 < best) {
      best = d2;
      tab->ref_point = A;
    }
  }
  tab->n_nz = int(tab->topo.pair_A.size());
  tab->n_gauss = n_gauss;
  MSASM_CUDA(cudaMalloc(&tab->d_T, size_t(tab->n_nz) * 9 * tab->n_pi * sizeof(double)));
  MSASM_CUDA(cudaMalloc(&tab->d_pairs, size_t(tab->n_nz) * 2 * sizeof(int32_t)));
  std::vector<int32_t> pairs(size_t(tab->n_nz) * 2);
  for (int m = 0; m < tab->n_nz; ++m) {
    pairs[2 * m] = tab->topo.pair_A[m];
    pairs[2 * m + 1] = tab->topo.pair_B[m];
  }
  MSASM_CUDA(cudaMemcpyAsync(tab->d_pairs, pairs.data(), pairs.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  MSASM_CUDA(cudaStreamSynchronize(s));   // `pairs` (host) must outlive the copy
  return MSASM_OK;
}

}  // namespace msasm

extern "C" {

const char* msasm_last_error(void) { return g_error.c_str(); }
const char* msasm_version(void) { return "msasm 0.1 (sm_103a)"; }

msasm_status msasm_build_tables(const msasm_micro_desc* micro, int32_t q, int32_t n_gauss, void* stream,
                                msasm_tables** out) {
  const int32_t q3[3] = {q, q, q};
  return msasm_build_tables_q3(micro, q3, n_gauss, stream, out);
}

msasm_status msasm_tables_degrees(const msasm_tables* tab, int32_t* q3) {
  if (!tab || !q3) return fail(MSASM_EINVAL, "tables or q3 is NULL");
  for (int d = 0; d < 3; ++d) q3[d] = tab->qd[d];
  return MSASM_OK;
}

msasm_status msasm_build_tables_q3(const msasm_micro_desc* micro, const int32_t* q3, int32_t n_gauss, void* stream,
                                   msasm_tables** out) {
  if (!out || !q3) return fail(MSASM_EINVAL, "out or q3 is NULL");
  *out = nullptr;
  if (n_gauss > 16) return fail(MSASM_EINVAL, "n_gauss must be <= 16");
  try {
    std::unique_ptr<msasm_tables> tab(new msasm_tables());   // freed on an error or an exception
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MSASM_TRY(tables_init(micro, q3, n_gauss, s, tab.get()));
    MSASM_TRY(build_table_gpu(tab.get(), s));                // synchronises `s`
    *out = tab.release();
    return MSASM_OK;
  } catch (const std::bad_alloc&) {
    return fail(MSASM_ENOMEM, "host allocation failed while building the tables");
  }
}

msasm_status msasm_tables_info(const msasm_tables* tab, int32_t* n_T, int32_t* n_nz, int32_t* n_pi) {
  if (!tab) return fail(MSASM_EINVAL, "tables is NULL");
  if (n_T) *n_T = tab->topo.n_T;
  if (n_nz) *n_nz = tab->n_nz;
  if (n_pi) *n_pi = tab->n_pi;
  return MSASM_OK;
}

msasm_status msasm_tables_copy(const msasm_tables* tab, double* d_table, int32_t* h_pairs, void* stream) {
  if (!tab) return fail(MSASM_EINVAL, "tables is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (d_table)
    MSASM_CUDA(cudaMemcpyAsync(d_table, tab->d_T, size_t(tab->n_nz) * 9 * tab->n_pi * sizeof(double),
                               cudaMemcpyDeviceToDevice, s));
  if (h_pairs)
    for (int m = 0; m < tab->n_nz; ++m) {
      h_pairs[2 * m] = tab->topo.pair_A[m];
      h_pairs[2 * m + 1] = tab->topo.pair_B[m];
    }
  return MSASM_OK;
}

void msasm_tables_destroy(msasm_tables* tab) { delete tab; }

static msasm_status plan_create_impl(const msasm_tables* tab, const msasm_macro_desc* macro,
                                     int32_t max_tiles_per_pass, void* stream, msasm_plan** out, int64_t* n_rows,
                                     int64_t* nnz) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::unique_ptr<msasm_plan> guard(new msasm_plan());   // freed on every early return or exception
  msasm_plan* plan = guard.get();
  plan->tab = tab;
  auto bail = [&](msasm_status st) { return st; };
  std::vector<double> basis[3];
  std::vector<int32_t> first[3];
  for (int d = 0; d < 3; ++d) {
    const int nq = tab->qd[d] + 1;                 // the nodes of this direction's projection degree
    std::vector<double> xn, wn;
    gauss_legendre01(nq, xn, wn);
    int p = macro->degree[d], nk = macro->n_knots[d];
    const double* t = macro->knots[d];
    if (p < 1 || p > 5) return bail(fail(MSASM_EINVAL, "macro degree must be in 1..5"));
    if (!t || nk < 2 * (p + 1)) return bail(fail(MSASM_EINVAL, "macro knot vector too short or NULL"));
    for (int k = 0; k + 1 < nk; ++k)
      if (!(t[k + 1] >= t[k])) return bail(fail(MSASM_EINVAL, "macro knots must be non-decreasing"));
    for (int k = 0; k <= p; ++k)
      if (t[k] != t[0] || t[nk - 1 - k] != t[nk - 1])
        return bail(fail(MSASM_EINVAL, "macro knot vector must be open (end knots repeated degree+1 times)"));
    plan->degree[d] = p;
    plan->n_ctrl_dir[d] = nk - p - 1;
    int ne = 0;
    plan->knots_host[d].assign(t, t + nk);
    for (int k = p; k < nk - p - 1; ++k) {
      if (!(t[k + 1] > t[k])) continue;
      ++ne;
      plan->span_host[d].push_back(k);
      first[d].push_back(k - p);
      double u0 = t[k], h = t[k + 1] - t[k];
      for (int c = 0; c < nq; ++c) {
        double vals[8], ders[8];
        bspline_span_basis(t, p, k, u0 + h * xn[c], vals, ders);
        for (int a = 0; a <= p; ++a) {
          basis[d].push_back(vals[a]);
          basis[d].push_back(ders[a] * h);   // d/dxi of the tile map
        }
      }
    }
    if (ne == 0) return bail(fail(MSASM_EINVAL, "macro knot vector has no non-empty span"));
    plan->n_elem[d] = ne;
  }
  plan->n_tiles = int64_t(plan->n_elem[0]) * plan->n_elem[1] * plan->n_elem[2];
  plan->n_ctrl = int64_t(plan->n_ctrl_dir[0]) * plan->n_ctrl_dir[1] * plan->n_ctrl_dir[2];
  plan->tiles_per_pass = (max_tiles_per_pass <= 0) ? plan->n_tiles : std::min<int64_t>(max_tiles_per_pass, plan->n_tiles);
  if (9 * plan->tiles_per_pass > 65535LL * 128) plan->tiles_per_pass = 65535LL * 128 / 9;

  // numbering and the point pattern on the host
  std::vector<int32_t> gmap;
  number_points(tab->topo, plan->n_elem, gmap, plan->n_points);
  if (plan->n_points >= (int64_t(1) << 31) / 3) return bail(fail(MSASM_EUNSUPPORTED, "more than 715M points"));
  std::vector<int64_t> pptr;
  std::vector<int32_t> pcol;
  point_pattern(tab->topo, plan->n_elem, gmap, plan->n_points, pptr, pcol);
  int64_t max_deg = 0;
  for (int64_t g = 0; g < plan->n_points; ++g) max_deg = std::max(max_deg, pptr[g + 1] - pptr[g]);
  if (max_deg >= 32768) return bail(fail(MSASM_EUNSUPPORTED, "a point has more than 32767 neighbours"));
  plan->n_rows = 3 * plan->n_points;
  plan->nnz = 9 * pptr[plan->n_points];
  // value range of each tile's owned rows: owned points of tile t are the ids assigned while
  // numbering t, so the ranges are consecutive in tile order
  plan->tile_vbase.assign(size_t(plan->n_tiles) + 1, plan->nnz);
  plan->tile_pbase.assign(size_t(plan->n_tiles) + 1, plan->n_points);
  {
    int64_t next_id = 0;
    const int n_T = tab->topo.n_T;
    for (int64_t t = 0; t < plan->n_tiles; ++t) {
      plan->tile_vbase[size_t(t)] = 9 * pptr[size_t(next_id)];
      plan->tile_pbase[size_t(t)] = next_id;
      int32_t mx = -1;
      for (int A = 0; A < n_T; ++A) mx = std::max(mx, gmap[size_t(t) * n_T + A]);
      if (mx + 1 > next_id) next_id = mx + 1;
    }
  }

  // scatter plan: tile types, value maps, secondary templates
  ScatterPlanHost sp;
  {
    msasm_status st0 = build_scatter_plan(plan, gmap, pptr, sp);
    if (st0 != MSASM_OK) return bail(st0);
  }
  plan->sec_off_host = sp.sec_off;
  plan->type_rep_host = sp.type_rep;
  plan->type_map_off_host = sp.type_map_off;
  plan->type_row_off_host = sp.type_row_off;
  plan->type_rows_host = sp.type_rows;
  for (size_t ty = 0; ty + 1 < sp.type_row_off.size(); ++ty)
    plan->max_type_rows = std::max<int>(plan->max_type_rows, int(sp.type_row_off[ty + 1] - sp.type_row_off[ty]));
  const int n_types = int(sp.type_rep.size());
  const int n_nz = tab->n_nz;

  // device allocations
  const size_t n_pi = size_t(tab->n_pi);
  const int ld = ld_nz_of(n_nz);
  int64_t* d_pptr = nullptr;
  int32_t* d_pcol = nullptr;
  uint8_t* d_pair_face = nullptr;
  unsigned long long* d_bad = nullptr;
  int64_t* d_type_rep = nullptr;
  auto dev = [&](void** p, size_t bytes) { return cudaMalloc(p, std::max<size_t>(bytes, 16)); };
  cudaError_t err = cudaSuccess;
  for (int d = 0; d < 3 && err == cudaSuccess; ++d) {
    err = dev((void**)&plan->d_basis[d], basis[d].size() * sizeof(double));
    if (err == cudaSuccess) err = dev((void**)&plan->d_first[d], first[d].size() * sizeof(int32_t));
  }
  if (err == cudaSuccess) err = dev((void**)&plan->d_gmap, gmap.size() * sizeof(int32_t));
  if (err == cudaSuccess) err = dev((void**)&plan->d_rowptr, size_t(plan->n_rows + 1) * sizeof(int64_t));
  if (err == cudaSuccess) err = dev((void**)&plan->d_col, size_t(plan->nnz) * sizeof(int32_t));
  if (err == cudaSuccess) err = dev((void**)&plan->d_rank, size_t(plan->n_tiles) * n_nz * sizeof(uint32_t));
  if (err == cudaSuccess) err = dev((void**)&plan->d_tile_type, sp.tile_type.size() * sizeof(int32_t));
  if (err == cudaSuccess) err = dev((void**)&plan->d_type_nvals, sp.type_nvals.size() * sizeof(int32_t));
  if (err == cudaSuccess) err = dev((void**)&plan->d_type_map_off, sp.type_map_off.size() * sizeof(int64_t));
  if (err == cudaSuccess) err = dev((void**)&plan->d_maps, size_t(sp.type_map_off.back()) * sizeof(int32_t));
  if (err == cudaSuccess) err = dev((void**)&plan->d_tile_vbase, plan->tile_vbase.size() * sizeof(int64_t));
  if (err == cudaSuccess) err = dev((void**)&plan->d_tmpl, sp.tmpl.size() * sizeof(uint32_t));
  if (err == cudaSuccess) err = dev((void**)&plan->d_tmpl_ptr, sp.tmpl_ptr.size() * sizeof(int64_t));
  if (err == cudaSuccess) err = dev((void**)&d_type_rep, sp.type_rep.size() * sizeof(int64_t));
  if (err == cudaSuccess) err = dev((void**)&plan->d_sec_off, sp.sec_off.size() * sizeof(int64_t));
  if (err == cudaSuccess) err = dev((void**)&plan->d_sec, size_t(sp.sec_off.back()) * sizeof(SecondaryEntry));
  if (err == cudaSuccess) err = dev((void**)&plan->d_coef, size_t(9 * plan->tiles_per_pass) * 9 * n_pi * sizeof(double));
  if (err == cudaSuccess) err = dev((void**)&plan->d_nz, size_t(9 * plan->tiles_per_pass) * ld * sizeof(double));
  if (err == cudaSuccess) err = dev((void**)&plan->d_degenerate, sizeof(unsigned long long));
  if (err == cudaSuccess) err = dev((void**)&plan->d_tc_err, sizeof(unsigned));
  if (err == cudaSuccess) err = dev((void**)&d_pptr, pptr.size() * sizeof(int64_t));
  if (err == cudaSuccess) err = dev((void**)&d_pcol, pcol.size() * sizeof(int32_t));
  if (err == cudaSuccess) err = dev((void**)&d_pair_face, size_t(n_nz));
  if (err == cudaSuccess) err = dev((void**)&d_bad, sizeof(unsigned long long));
  auto cleanup_tmp = [&]() {
    cudaFree(d_pptr);
    cudaFree(d_pcol);
    cudaFree(d_pair_face);
    cudaFree(d_bad);
    cudaFree(d_type_rep);
  };
  if (err != cudaSuccess) {
    cleanup_tmp();
    return bail(cuda_fail(err, "cudaMalloc(plan)"));
  }
  auto h2d = [&](void* dst, const void* src, size_t bytes) {
    return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
  };
  for (int d = 0; d < 3 && err == cudaSuccess; ++d) {
    err = h2d(plan->d_basis[d], basis[d].data(), basis[d].size() * sizeof(double));
    if (err == cudaSuccess) err = h2d(plan->d_first[d], first[d].data(), first[d].size() * sizeof(int32_t));
  }
  if (err == cudaSuccess) err = h2d(plan->d_gmap, gmap.data(), gmap.size() * sizeof(int32_t));
  if (err == cudaSuccess) err = h2d(plan->d_tile_type, sp.tile_type.data(), sp.tile_type.size() * sizeof(int32_t));
  if (err == cudaSuccess) err = h2d(plan->d_type_nvals, sp.type_nvals.data(), sp.type_nvals.size() * sizeof(int32_t));
  if (err == cudaSuccess)
    err = h2d(plan->d_type_map_off, sp.type_map_off.data(), sp.type_map_off.size() * sizeof(int64_t));
  if (err == cudaSuccess)
    err = cudaMemsetAsync(plan->d_maps, 0xff, size_t(sp.type_map_off.back()) * sizeof(int32_t), s);   // -1
  if (err == cudaSuccess)
    err = h2d(plan->d_tile_vbase, plan->tile_vbase.data(), plan->tile_vbase.size() * sizeof(int64_t));
  if (err == cudaSuccess) err = h2d(plan->d_tmpl, sp.tmpl.data(), sp.tmpl.size() * sizeof(uint32_t));
  if (err == cudaSuccess) err = h2d(plan->d_tmpl_ptr, sp.tmpl_ptr.data(), sp.tmpl_ptr.size() * sizeof(int64_t));
  if (err == cudaSuccess) err = h2d(d_type_rep, sp.type_rep.data(), sp.type_rep.size() * sizeof(int64_t));
  if (err == cudaSuccess) err = h2d(plan->d_sec_off, sp.sec_off.data(), sp.sec_off.size() * sizeof(int64_t));
  if (err == cudaSuccess) err = h2d(d_pptr, pptr.data(), pptr.size() * sizeof(int64_t));
  if (err == cudaSuccess) err = h2d(d_pcol, pcol.data(), pcol.size() * sizeof(int32_t));
  if (err == cudaSuccess) err = h2d(d_pair_face, tab->topo.pair_face.data(), size_t(n_nz));
  if (err == cudaSuccess) err = cudaMemsetAsync(d_bad, 0, sizeof(unsigned long long), s);
  if (err == cudaSuccess) err = cudaMemsetAsync(plan->d_degenerate, 0, sizeof(unsigned long long), s);
  if (err == cudaSuccess) err = cudaMemsetAsync(plan->d_tc_err, 0, sizeof(unsigned), s);
  if (err != cudaSuccess) {
    cudaStreamSynchronize(s);
    cleanup_tmp();
    return bail(cuda_fail(err, "cudaMemcpyAsync(plan)"));
  }
  msasm_status st = structure_expand_gpu(plan->n_points, d_pptr, d_pcol, plan->d_rowptr, plan->d_col, s);
  if (st == MSASM_OK)
    st = rank_map_gpu(plan->d_gmap, tab->d_pairs, d_pair_face, d_pptr, d_pcol, plan->n_tiles, tab->topo.n_T, n_nz,
                      plan->n_elem[0], plan->n_elem[1], plan->d_rank, d_bad, s);
  if (st == MSASM_OK) st = scatter_maps_gpu(plan, d_type_rep, n_types, d_bad, s);
  if (st == MSASM_OK) st = secondary_entries_gpu(plan, s);
  unsigned long long bad = 0;
  if (st == MSASM_OK) {
    err = cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) st = cuda_fail(err, "plan structure kernels");
  } else {
    cudaStreamSynchronize(s);
  }
  cleanup_tmp();
  if (st != MSASM_OK) return bail(st);
  if (bad)
    return bail(fail(MSASM_ECUDA, "index map: a tile pair is missing from the CSR pattern, or a tile places its "
                                  "blocks differently from its type"));
  MSASM_CUDA(cudaStreamCreateWithFlags(&plan->scatter_side, cudaStreamNonBlocking));
  for (cudaEvent_t& e : plan->scatter_ev) MSASM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  plan->gmap_host = std::move(gmap);
  if (n_rows) *n_rows = plan->n_rows;
  if (nnz) *nnz = plan->nnz;
  *out = guard.release();
  return MSASM_OK;
}

msasm_status msasm_plan_create(const msasm_tables* tab, const msasm_macro_desc* macro, int32_t max_tiles_per_pass,
                               void* stream, msasm_plan** out, int64_t* n_rows, int64_t* nnz) {
  if (!out) return fail(MSASM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!tab || !macro) return fail(MSASM_EINVAL, "tables or macro descriptor is NULL");
  try {
    return plan_create_impl(tab, macro, max_tiles_per_pass, stream, out, n_rows, nnz);
  } catch (const std::bad_alloc&) {
    return fail(MSASM_ENOMEM, "host allocation failed while building the plan");
  }
}

msasm_status msasm_plan_info(const msasm_plan* plan, int64_t* n_tiles, int64_t* n_points, int64_t* n_rows,
                             int64_t* nnz, int64_t* n_ctrl) {
  if (!plan) return fail(MSASM_EINVAL, "plan is NULL");
  if (n_tiles) *n_tiles = plan->n_tiles;
  if (n_points) *n_points = plan->n_points;
  if (n_rows) *n_rows = plan->n_rows;
  if (nnz) *nnz = plan->nnz;
  if (n_ctrl) *n_ctrl = plan->n_ctrl;
  return MSASM_OK;
}

msasm_status msasm_plan_csr(const msasm_plan* plan, int64_t* d_rowptr, int32_t* d_col, void* stream) {
  if (!plan || !d_rowptr || !d_col) return fail(MSASM_EINVAL, "plan, d_rowptr or d_col is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MSASM_CUDA(cudaMemcpyAsync(d_rowptr, plan->d_rowptr, size_t(plan->n_rows + 1) * sizeof(int64_t),
                             cudaMemcpyDeviceToDevice, s));
  MSASM_CUDA(cudaMemcpyAsync(d_col, plan->d_col, size_t(plan->nnz) * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  return MSASM_OK;
}

msasm_status msasm_plan_numbering(const msasm_plan* plan, int32_t* d_gmap, void* stream) {
  if (!plan || !d_gmap) return fail(MSASM_EINVAL, "plan or d_gmap is NULL");
  MSASM_CUDA(cudaMemcpyAsync(d_gmap, plan->d_gmap, size_t(plan->n_tiles) * plan->tab->topo.n_T * sizeof(int32_t),
                             cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)));
  return MSASM_OK;
}

void msasm_plan_destroy(msasm_plan* plan) { delete plan; }

static msasm_status check_material(double E, double nu) {
  if (!(E > 0.0) || !(nu > -1.0 && nu < 0.5) || !std::isfinite(E))
    return fail(MSASM_EINVAL, "material: need E > 0 and -1 < nu < 0.5");
  return MSASM_OK;
}

static void lame(double E, double nu, double& lam, double& mu) {
  lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  mu = E / (2.0 * (1.0 + nu));
}

// contraction of `n_tiles` tiles of FP64 coefficients into nzdata of the precision family
// table slices for a tensor-core form, built once per table and precision
static msasm_status ensure_table_slices(msasm_tables* tab, int kind, cudaStream_t s) {
  if (tab->split_kind == kind) return MSASM_OK;
  cudaFree(tab->d_Thi);
  cudaFree(tab->d_Tlo);
  cudaFree(tab->d_Tscale);
  tab->d_Thi = tab->d_Tlo = nullptr;
  tab->d_Tscale = nullptr;
  tab->split_kind = -1;
  const int K = 9 * tab->n_pi;
  const size_t bytes = tc_slice_bytes(tab->n_nz, K, kind);
  MSASM_CUDA(cudaMalloc(&tab->d_Thi, bytes));
  MSASM_CUDA(cudaMalloc(&tab->d_Tlo, bytes));
  MSASM_CUDA(cudaMalloc(&tab->d_Tscale, size_t(tab->n_nz) * sizeof(float)));
  MSASM_TRY(tc_split_gpu(tab->d_T, tab->n_nz, K, kind, tab->d_Thi, tab->d_Tlo, tab->d_Tscale, s));
  tab->split_kind = kind;
  return MSASM_OK;
}

// bytes of coefficient slices (hi, lo, row scales; or the 7 FP64-emulation slices and scales) for n_tiles tiles
static size_t coef_lp_bytes_for(int64_t n_tiles, int n_pi) {
  const int K = 9 * n_pi;
  const size_t split = 2 * size_t(9 * n_tiles) * size_t(K + 64) * 4 + size_t(9 * n_tiles) * 4;
  // the emulated forms slice rows of K values (assembly) or of 576-pair chunks (adjoint)
  const size_t emu = emu_slice_bytes(9 * n_tiles, std::max(K, 576)) + size_t(9 * n_tiles) * 8;
  return std::max(split, emu) + 512;
}

// FP32 on the CUDA cores (FFMA): for tables wider than the exact slice accumulation allows (9 n_pi > 576)
static msasm_status contract_f32_simt(msasm_tables* tab, const double* d_coef, int64_t n_tiles, void* d_nz,
                                      void* scratch_lp, cudaStream_t s) {
  const int K = 9 * tab->n_pi, n_nz = tab->n_nz, ld = ld_nz_of(n_nz);
  if (!tab->d_T32) {
    MSASM_CUDA(cudaMalloc(&tab->d_T32, size_t(n_nz) * K * sizeof(float)));
    MSASM_TRY(to_f32_gpu(tab->d_T, int64_t(n_nz) * K, tab->d_T32, s));
  }
  float* c32 = static_cast<float*>(scratch_lp);
  MSASM_TRY(to_f32_gpu(d_coef, 9 * n_tiles * K, c32, s));
  return contract_simt_f32(c32, tab->d_T32, n_tiles, n_nz, K, ld, static_cast<float*>(d_nz), s);
}

static msasm_status contract_dispatch(const msasm_tables* ctab, msasm_precision prec, const double* d_coef,
                                      int64_t n_tiles, void* d_nz, void* scratch_lp, cudaStream_t s,
                                      unsigned* d_err) {
  msasm_tables* tab = const_cast<msasm_tables*>(ctab);
  const int K = 9 * tab->n_pi, n_nz = tab->n_nz, ld = ld_nz_of(n_nz);
  switch (prec) {
    case MSASM_F64:
      return contract_simt_f64(d_coef, tab->d_T, n_tiles, n_nz, K, ld, static_cast<double*>(d_nz), s);
    case MSASM_F32: {
      // FP32 values from the tensor cores: 4 exact BF16 slices (28 bits) of each operand row, the 10
      // slice products with i + j <= 3 accumulated exactly, the result rounded once to FP32
      if (K > 576) return contract_f32_simt(tab, d_coef, n_tiles, d_nz, scratch_lp, s);   // beyond exactness
      if (!tab->d_Tslices4) {
        MSASM_CUDA(cudaMalloc(&tab->d_Tslices4, emu_slice_bytes(n_nz, K, 4)));
        MSASM_CUDA(cudaMalloc(&tab->d_Tslice_scale4, size_t(n_nz) * sizeof(int)));
        MSASM_TRY(emu_slice_gpu(tab->d_T, n_nz, K, K, tab->d_Tslices4, tab->d_Tslice_scale4, s, 4));
      }
      uint8_t* sl = static_cast<uint8_t*>(scratch_lp);
      int* sc = reinterpret_cast<int*>(sl + ((emu_slice_bytes(9 * n_tiles, K, 4) + 255) & ~size_t(255)));
      MSASM_TRY(emu_slice_gpu(d_coef, 9 * n_tiles, K, K, sl, sc, s, 4));
      return contract_emu_gpu(tab->d_Tslices4, tab->d_Tslice_scale4, n_nz, sl, sc, 9 * n_tiles, K, d_nz, ld, false,
                              true, d_err, s, 4);
    }
    case MSASM_SPLIT_F16:
    case MSASM_SPLIT_BF16:
    case MSASM_TF32:
    case MSASM_TF32X3: {
      const int kind = tc_kind_of(prec);
      MSASM_TRY(ensure_table_slices(tab, kind, s));
      const size_t sb = tc_slice_bytes(9 * n_tiles, K, kind);
      uint8_t* hi = static_cast<uint8_t*>(scratch_lp);
      uint8_t* lo = hi + sb;
      float* sc = reinterpret_cast<float*>(lo + sb);
      MSASM_TRY(tc_split_gpu(d_coef, 9 * n_tiles, K, kind, hi, lo, sc, s));
      return contract_tc_gpu(kind, tab->d_Thi, tab->d_Tlo, tab->d_Tscale, n_nz, hi, lo, sc, 9 * n_tiles, K,
                             static_cast<float*>(d_nz), ld, true, d_err, s);
    }
    case MSASM_F64_EMU: {
      if (!tab->d_Tslices) {
        MSASM_CUDA(cudaMalloc(&tab->d_Tslices, emu_slice_bytes(n_nz, K)));
        MSASM_CUDA(cudaMalloc(&tab->d_Tslice_scale, size_t(n_nz) * sizeof(int)));
        MSASM_TRY(emu_slice_gpu(tab->d_T, n_nz, K, K, tab->d_Tslices, tab->d_Tslice_scale, s));
        tab->n_slices = 7;
      }
      uint8_t* sl = static_cast<uint8_t*>(scratch_lp);
      int* sc = reinterpret_cast<int*>(sl + ((emu_slice_bytes(9 * n_tiles, K) + 255) & ~size_t(255)));
      MSASM_TRY(emu_slice_gpu(d_coef, 9 * n_tiles, K, K, sl, sc, s));
      return contract_emu_gpu(tab->d_Tslices, tab->d_Tslice_scale, n_nz, sl, sc, 9 * n_tiles, K,
                              static_cast<double*>(d_nz), ld, false, true, d_err, s);
    }
    default:
      return fail(MSASM_EUNSUPPORTED, "precision not available in this build");
  }
}

static int contract_launches(msasm_precision prec) { return prec == MSASM_F64 ? 1 : 2; }   // slicing + product

static msasm_status ensure_lp_scratch(msasm_plan* plan, msasm_precision prec) {
  if (prec == MSASM_F64) return MSASM_OK;
  size_t need = coef_lp_bytes_for(plan->tiles_per_pass, plan->tab->n_pi);
  if (plan->coef_lp_bytes >= need) return MSASM_OK;
  cudaFree(plan->d_coef_lp);
  plan->d_coef_lp = nullptr;
  plan->coef_lp_bytes = 0;
  MSASM_CUDA(cudaMalloc(&plan->d_coef_lp, need));
  plan->coef_lp_bytes = need;
  return MSASM_OK;
}

// step 4 of tiles [t0, t0 + nt): direct pass for the tiles below direct_end, secondary pass for all,
// into the value window [v_lo, v_hi) held by d_values
static msasm_status scatter_dispatch(msasm_plan* plan, msasm_precision prec, const void* d_nz, int64_t t0,
                                     int64_t nt, void* d_values, cudaStream_t s, int64_t direct_end = -1,
                                     int64_t v_lo = 0, int64_t v_hi = -1) {
  const int ld = ld_nz_of(plan->tab->n_nz);
  if (direct_end < 0) direct_end = t0 + nt;
  if (v_hi < 0) v_hi = plan->nnz;
  if (is_f64_precision(prec))
    return scatter_pass_gpu<double>(plan, static_cast<const double*>(d_nz), ld, t0, nt,
                                    static_cast<double*>(d_values), direct_end, v_lo, v_hi, s);
  return scatter_pass_gpu<float>(plan, static_cast<const float*>(d_nz), ld, t0, nt, static_cast<float*>(d_values),
                                 direct_end, v_lo, v_hi, s);
}

// the tiles whose blocks reach the rows owned by tiles [t0, t1): the range itself and the tiles
// of the next layer above it (a tile's lower faces are glued to t - 1, t - nx and t - nx ny)
static int64_t halo_end_of(const msasm_plan* plan, int64_t t1) {
  const int64_t layer = int64_t(plan->n_elem[0]) * plan->n_elem[1];
  return std::min(plan->n_tiles, t1 + layer);
}

// steps 1, 3, 4 for the rows owned by tiles [t0, t1) (all rows for [0, n_tiles)), into d_values
// holding the window [tile_vbase[t0], tile_vbase[t1])
static msasm_status assemble_range_impl(msasm_plan* plan, const double* d_ctrl, double E, double nu,
                                        msasm_precision prec, int64_t t0, int64_t t1, void* d_values, uint32_t flags,
                                        cudaStream_t s) {
  MSASM_TRY(check_material(E, nu));
  if (prec < MSASM_F64 || prec > MSASM_F64_EMU) return fail(MSASM_EINVAL, "unknown precision");
  double lam, mu;
  lame(E, nu, lam, mu);
  MSASM_TRY(ensure_lp_scratch(plan, prec));
  MSASM_CUDA(cudaMemsetAsync(plan->d_degenerate, 0, sizeof(unsigned long long), s));
  const int64_t P = plan->tiles_per_pass;
  const int64_t t_end = halo_end_of(plan, t1);
  const int64_t v_lo = plan->tile_vbase[size_t(t0)], v_hi = plan->tile_vbase[size_t(t1)];
  const bool timed = (flags & MSASM_FLAG_STAGE_TIMES) != 0;
  const int n_pass = int((t_end - t0 + P - 1) / P);
  plan->timed_passes = 0;
  if (timed) {
    while (plan->events.size() < size_t(4 * n_pass)) {
      cudaEvent_t e;
      MSASM_CUDA(cudaEventCreate(&e));
      plan->events.push_back(e);
    }
    for (int k = 0; k < 3; ++k) plan->stage_launches[k] = 0;
  }
  int pass = 0;
  for (int64_t ta = t0; ta < t_end; ta += P, ++pass) {
    const int64_t nt = std::min(P, t_end - ta);
    if (timed) MSASM_CUDA(cudaEventRecord(plan->events[4 * pass + 0], s));
    MSASM_TRY(pullback_gpu(plan, d_ctrl, lam, mu, ta, nt, plan->d_coef, s));
    if (timed) MSASM_CUDA(cudaEventRecord(plan->events[4 * pass + 1], s));
    MSASM_TRY(contract_dispatch(plan->tab, prec, plan->d_coef, nt, plan->d_nz, plan->d_coef_lp, s, plan->d_tc_err));
    if (timed) MSASM_CUDA(cudaEventRecord(plan->events[4 * pass + 2], s));
    MSASM_TRY(scatter_dispatch(plan, prec, plan->d_nz, ta, nt, d_values, s, t1, v_lo, v_hi));
    if (timed) {
      MSASM_CUDA(cudaEventRecord(plan->events[4 * pass + 3], s));
      plan->stage_launches[0] += 1;
      plan->stage_launches[1] += contract_launches(prec);
      plan->stage_launches[2] += (ta < t1 ? 1 : 0) + (plan->sec_off_host[size_t(ta + nt)] > plan->sec_off_host[size_t(ta)] ? 1 : 0);
    }
  }
  if (timed) plan->timed_passes = n_pass;
  if (flags & MSASM_FLAG_CHECK_DEGENERATE) {
    unsigned long long cnt = 0;
    unsigned tc_err = 0;
    MSASM_CUDA(cudaMemcpyAsync(&cnt, plan->d_degenerate, sizeof(cnt), cudaMemcpyDeviceToHost, s));
    MSASM_CUDA(cudaMemcpyAsync(&tc_err, plan->d_tc_err, sizeof(tc_err), cudaMemcpyDeviceToHost, s));
    MSASM_CUDA(cudaStreamSynchronize(s));
    if (tc_err) return fail(MSASM_ECUDA, "a tensor-core pipeline wait timed out (results invalid)");
    if (cnt)
      return fail(MSASM_EDEGENERATE,
                  "degenerate macro element: |det J| <= tol at " + std::to_string(cnt) + " interpolation nodes");
  }
  return MSASM_OK;
}

msasm_status msasm_assemble(msasm_plan* plan, const double* d_ctrl, double E, double nu, msasm_precision prec,
                            void* d_values, uint32_t flags, void* stream) {
  if (!plan || !d_ctrl || !d_values) return fail(MSASM_EINVAL, "plan, d_ctrl or d_values is NULL");
  return assemble_range_impl(plan, d_ctrl, E, nu, prec, 0, plan->n_tiles, d_values, flags,
                             static_cast<cudaStream_t>(stream));
}

msasm_status msasm_plan_range(const msasm_plan* plan, int64_t t0, int64_t t1, int64_t* row0, int64_t* row1,
                              int64_t* v0, int64_t* v1, int64_t* halo_end) {
  if (!plan) return fail(MSASM_EINVAL, "plan is NULL");
  if (t0 < 0 || t1 < t0 || t1 > plan->n_tiles) return fail(MSASM_EINVAL, "tile range outside [0, n_tiles]");
  if (row0) *row0 = 3 * plan->tile_pbase[size_t(t0)];
  if (row1) *row1 = 3 * plan->tile_pbase[size_t(t1)];
  if (v0) *v0 = plan->tile_vbase[size_t(t0)];
  if (v1) *v1 = plan->tile_vbase[size_t(t1)];
  if (halo_end) *halo_end = (t1 > t0) ? halo_end_of(plan, t1) : t1;
  return MSASM_OK;
}

msasm_status msasm_assemble_range(msasm_plan* plan, const double* d_ctrl, double E, double nu, msasm_precision prec,
                                  int64_t t0, int64_t t1, void* d_values, uint32_t flags, void* stream) {
  if (!plan || !d_ctrl || !d_values) return fail(MSASM_EINVAL, "plan, d_ctrl or d_values is NULL");
  if (t0 < 0 || t1 < t0 || t1 > plan->n_tiles) return fail(MSASM_EINVAL, "tile range outside [0, n_tiles]");
  if (t1 == t0) return MSASM_OK;
  return assemble_range_impl(plan, d_ctrl, E, nu, prec, t0, t1, d_values, flags, static_cast<cudaStream_t>(stream));
}

constexpr int kAdjChunk = 576;   // pairs per exactly accumulated chunk of the emulated adjoint product

static size_t value_bytes(msasm_precision prec) { return is_f64_precision(prec) ? 8 : 4; }

msasm_status msasm_stage_times(const msasm_plan* plan, double* ms, int32_t* launches) {
  if (!plan || !ms) return fail(MSASM_EINVAL, "plan or ms is NULL");
  if (plan->timed_passes <= 0) return fail(MSASM_EINVAL, "the last assemble did not record stage times");
  for (int k = 0; k < 3; ++k) ms[k] = 0.0;
  for (int p = 0; p < plan->timed_passes; ++p) {
    MSASM_CUDA(cudaEventSynchronize(plan->events[4 * p + 3]));
    for (int k = 0; k < 3; ++k) {
      float t = 0.0f;
      MSASM_CUDA(cudaEventElapsedTime(&t, plan->events[4 * p + k], plan->events[4 * p + k + 1]));
      ms[k] += t;
    }
  }
  if (launches)
    for (int k = 0; k < 3; ++k) launches[k] = plan->stage_launches[k];
  return MSASM_OK;
}

msasm_status msasm_assemble_host(msasm_plan* plan, const double* h_ctrl, double E, double nu, msasm_precision prec,
                                 void* h_values, uint32_t flags, void* stream) {
  if (!plan || !h_ctrl || !h_values) return fail(MSASM_EINVAL, "plan, h_ctrl or h_values is NULL");
  if (prec < MSASM_F64 || prec > MSASM_F64_EMU) return fail(MSASM_EINVAL, "unknown precision");
  MSASM_TRY(check_material(E, nu));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t cbytes = size_t(plan->n_ctrl) * 3 * sizeof(double);
  const size_t vb = value_bytes(prec);
  const size_t vbytes = size_t(plan->nnz) * vb;
  if (!plan->d_ctrl_stage) MSASM_CUDA(cudaMalloc(&plan->d_ctrl_stage, cbytes));
  if (plan->values_stage_bytes < vbytes) {
    cudaFree(plan->d_values_stage);
    plan->d_values_stage = nullptr;
    plan->values_stage_bytes = 0;
    MSASM_CUDA(cudaMalloc(&plan->d_values_stage, vbytes));
    plan->values_stage_bytes = vbytes;
  }
  for (int k = 0; k < 2; ++k)
    if (!plan->copy_stream[k]) MSASM_CUDA(cudaStreamCreateWithFlags(&plan->copy_stream[k], cudaStreamNonBlocking));
  double lam, mu;
  lame(E, nu, lam, mu);
  MSASM_TRY(ensure_lp_scratch(plan, prec));
  MSASM_CUDA(cudaMemcpyAsync(plan->d_ctrl_stage, h_ctrl, cbytes, cudaMemcpyHostToDevice, s));
  MSASM_CUDA(cudaMemsetAsync(plan->d_degenerate, 0, sizeof(unsigned long long), s));
  // Passes of about 1/8 of the tiles: after a pass ending at tile t1, the rows owned by tiles
  // below t1 - nx*ny can receive no further contribution (their upper neighbours are done), so
  // that prefix of the values is copied to the host on a side stream while the next pass runs.
  const int64_t P = std::max<int64_t>(1, std::min<int64_t>(plan->tiles_per_pass, (plan->n_tiles + 7) / 8));
  const int64_t lag = int64_t(plan->n_elem[0]) * plan->n_elem[1];
  int64_t copied = 0;
  int which = 0, ev = 0;
  auto copy_upto = [&](int64_t upto) -> msasm_status {
    if (upto <= copied) return MSASM_OK;
    if (plan->copy_events.size() <= size_t(ev)) {
      cudaEvent_t e;
      MSASM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      plan->copy_events.push_back(e);
    }
    cudaEvent_t e = plan->copy_events[size_t(ev++)];
    MSASM_CUDA(cudaEventRecord(e, s));
    cudaStream_t cs = plan->copy_stream[which];
    which ^= 1;
    MSASM_CUDA(cudaStreamWaitEvent(cs, e, 0));
    MSASM_CUDA(cudaMemcpyAsync(static_cast<uint8_t*>(h_values) + size_t(copied) * vb,
                               static_cast<uint8_t*>(plan->d_values_stage) + size_t(copied) * vb,
                               size_t(upto - copied) * vb, cudaMemcpyDeviceToHost, cs));
    copied = upto;
    return MSASM_OK;
  };
  for (int64_t t0 = 0; t0 < plan->n_tiles; t0 += P) {
    const int64_t nt = std::min(P, plan->n_tiles - t0);
    MSASM_TRY(pullback_gpu(plan, plan->d_ctrl_stage, lam, mu, t0, nt, plan->d_coef, s));
    MSASM_TRY(contract_dispatch(plan->tab, prec, plan->d_coef, nt, plan->d_nz, plan->d_coef_lp, s, plan->d_tc_err));
    MSASM_TRY(scatter_dispatch(plan, prec, plan->d_nz, t0, nt, plan->d_values_stage, s));
    const int64_t t_final = t0 + nt - lag;
    if (t0 + nt < plan->n_tiles && t_final > 0) MSASM_TRY(copy_upto(plan->tile_vbase[size_t(t_final)]));
  }
  MSASM_TRY(copy_upto(plan->nnz));
  for (int k = 0; k < 2; ++k) MSASM_CUDA(cudaStreamSynchronize(plan->copy_stream[k]));
  MSASM_CUDA(cudaStreamSynchronize(s));
  if (flags & MSASM_FLAG_CHECK_DEGENERATE) {
    unsigned long long cnt = 0;
    unsigned tc_err = 0;
    MSASM_CUDA(cudaMemcpy(&cnt, plan->d_degenerate, sizeof(cnt), cudaMemcpyDeviceToHost));
    MSASM_CUDA(cudaMemcpy(&tc_err, plan->d_tc_err, sizeof(tc_err), cudaMemcpyDeviceToHost));
    if (tc_err) return fail(MSASM_ECUDA, "a tensor-core pipeline wait timed out (results invalid)");
    if (cnt) return fail(MSASM_EDEGENERATE, "degenerate macro element in msasm_assemble_host");
  }
  return MSASM_OK;
}

// dL/dP of the tiles [t0, t1) into d_grad_ctrl (overwritten): the whole gradient for [0, n_tiles)
static msasm_status grad_range_impl(msasm_plan* plan, const double* d_ctrl, double E, double nu, msasm_precision prec,
                                    int64_t t0, int64_t t1, const void* d_u, const void* d_grad_values,
                                    double* d_grad_ctrl, cudaStream_t s) {
  if (!plan || !d_ctrl || !d_grad_ctrl) return fail(MSASM_EINVAL, "plan, d_ctrl or d_grad_ctrl is NULL");
  if ((d_u == nullptr) == (d_grad_values == nullptr))
    return fail(MSASM_EINVAL, "give exactly one of d_u and d_grad_values");
  if (t0 < 0 || t1 < t0 || t1 > plan->n_tiles) return fail(MSASM_EINVAL, "tile range outside [0, n_tiles]");
  MSASM_TRY(check_material(E, nu));
  if (prec < MSASM_F64 || prec > MSASM_F64_EMU) return fail(MSASM_EINVAL, "unknown precision");
  msasm_tables* tab = const_cast<msasm_tables*>(plan->tab);
  double lam, mu;
  lame(E, nu, lam, mu);
  const bool f64 = is_f64_precision(prec);
  const int n_nz = tab->n_nz, K = 9 * tab->n_pi, ld = ld_nz_of(n_nz);
  if (f64 && !tab->d_Tt) {
    MSASM_CUDA(cudaMalloc(&tab->d_Tt, size_t(K) * n_nz * sizeof(double)));
    MSASM_TRY(transpose_table_gpu<double>(tab->d_T, n_nz, K, tab->d_Tt, s));
  }
  if (!f64 && !tab->d_Tt32) {
    MSASM_CUDA(cudaMalloc(&tab->d_Tt32, size_t(K) * n_nz * sizeof(float)));
    MSASM_TRY(transpose_table_gpu<float>(tab->d_T, n_nz, K, tab->d_Tt32, s));
  }
  if (prec == MSASM_F64_EMU) {
    if (K > 576) return fail(MSASM_EUNSUPPORTED, "FP64 emulation is exact for K <= 576 (q <= 3)");
    MSASM_TRY(ensure_lp_scratch(plan, MSASM_F64_EMU));       // slices of G (rows 9 nt, chunk of k)
    if (!plan->d_adj_lp) {
      const size_t bytes = ((emu_slice_bytes(K, kAdjChunk) + 255) & ~size_t(255)) + size_t(K) * sizeof(int);
      MSASM_CUDA(cudaMalloc(&plan->d_adj_lp, bytes));
    }
    MSASM_CUDA(cudaMemsetAsync(plan->d_tc_err, 0, sizeof(unsigned), s));
  }
  MSASM_CUDA(cudaMemsetAsync(d_grad_ctrl, 0, size_t(plan->n_ctrl) * 3 * sizeof(double), s));
  const int64_t P = plan->tiles_per_pass;
  const int64_t t_lo = t0, t_hi = t1;
  for (int64_t t0 = t_lo; t0 < t_hi; t0 += P) {
    const int64_t nt = std::min(P, t_hi - t0);
    if (prec == MSASM_F64_EMU) {
      // W = G Tt^T on the tensor cores to FP64 accuracy: the contraction over the n_nz pairs is cut
      // into chunks of at most 576 (the exactness bound of the slice accumulators); each chunk's
      // exactly rounded product is added to W in FP64
      double* G = static_cast<double*>(plan->d_nz);
      MSASM_TRY(grad_blocks_gpu<double>(plan, static_cast<const double*>(d_u), static_cast<const double*>(d_grad_values),
                                        t0, nt, ld, G, s));
      uint8_t* gl = static_cast<uint8_t*>(plan->d_coef_lp);
      int* g_exp = reinterpret_cast<int*>(gl + ((emu_slice_bytes(9 * nt, kAdjChunk) + 255) & ~size_t(255)));
      uint8_t* tl = static_cast<uint8_t*>(plan->d_adj_lp);
      int* t_exp = reinterpret_cast<int*>(tl + ((emu_slice_bytes(K, kAdjChunk) + 255) & ~size_t(255)));
      for (int m0 = 0; m0 < n_nz; m0 += kAdjChunk) {
        const int kc = std::min(kAdjChunk, n_nz - m0);
        MSASM_TRY(emu_slice_gpu(tab->d_Tt + m0, K, n_nz, kc, tl, t_exp, s));
        MSASM_TRY(emu_slice_gpu(G + m0, 9 * nt, ld, kc, gl, g_exp, s));
        MSASM_TRY(contract_emu_gpu(tl, t_exp, K, gl, g_exp, 9 * nt, kc, plan->d_coef, K, m0 > 0, false,
                                   plan->d_tc_err, s));
      }
    } else if (f64) {
      double* G = static_cast<double*>(plan->d_nz);
      MSASM_TRY(grad_blocks_gpu<double>(plan, static_cast<const double*>(d_u), static_cast<const double*>(d_grad_values),
                                        t0, nt, ld, G, s));
      MSASM_TRY(gemm_simt<double>(G, ld, tab->d_Tt, n_nz, 9 * nt, K, n_nz, plan->d_coef, K, s));
    } else {
      float* G = static_cast<float*>(plan->d_nz);
      float* W = reinterpret_cast<float*>(plan->d_coef);
      MSASM_TRY(grad_blocks_gpu<float>(plan, static_cast<const float*>(d_u), static_cast<const float*>(d_grad_values),
                                       t0, nt, ld, G, s));
      MSASM_TRY(gemm_simt<float>(G, ld, tab->d_Tt32, n_nz, 9 * nt, K, n_nz, W, K, s));
    }
    MSASM_TRY(adjoint_pullback_gpu(plan, d_ctrl, lam, mu, t0, nt, plan->d_coef, !f64, d_grad_ctrl, s));
  }
  return MSASM_OK;
}

msasm_status msasm_assemble_grad(msasm_plan* plan, const double* d_ctrl, double E, double nu, msasm_precision prec,
                                 const void* d_u, const void* d_grad_values, double* d_grad_ctrl, void* stream) {
  if (!plan) return fail(MSASM_EINVAL, "plan is NULL");
  return grad_range_impl(plan, d_ctrl, E, nu, prec, 0, plan->n_tiles, d_u, d_grad_values, d_grad_ctrl,
                         static_cast<cudaStream_t>(stream));
}

msasm_status msasm_assemble_grad_range(msasm_plan* plan, const double* d_ctrl, double E, double nu,
                                       msasm_precision prec, int64_t t0, int64_t t1, const void* d_u,
                                       const void* d_grad_values, double* d_grad_ctrl, void* stream) {
  if (!plan) return fail(MSASM_EINVAL, "plan is NULL");
  return grad_range_impl(plan, d_ctrl, E, nu, prec, t0, t1, d_u, d_grad_values, d_grad_ctrl,
                         static_cast<cudaStream_t>(stream));
}

msasm_status msasm_linop_apply(msasm_plan* plan, const double* d_coef, msasm_precision prec, const double* d_u,
                               double* d_y, void* stream) {
  if (!plan || !d_coef || !d_u || !d_y) return fail(MSASM_EINVAL, "plan, d_coef, d_u or d_y is NULL");
  if (prec < MSASM_F64 || prec > MSASM_F64_EMU) return fail(MSASM_EINVAL, "unknown precision");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MSASM_TRY(ensure_lp_scratch(plan, prec));
  const int K = 9 * plan->tab->n_pi, ld = ld_nz_of(plan->tab->n_nz);
  const int64_t P = plan->tiles_per_pass;
  const int kind = tc_kind_of(prec);
  if (kind >= 0) {
    // split tensor-core forms: the contraction's epilogue applies every tile block to u and adds it
    // into y (Sec. 4.2: the local matrices are never stored; no nzdata scratch)
    msasm_tables* tab = const_cast<msasm_tables*>(plan->tab);
    MSASM_TRY(ensure_table_slices(tab, kind, s));
    MSASM_CUDA(cudaMemsetAsync(d_y, 0, size_t(plan->n_rows) * sizeof(double), s));
    for (int64_t t0 = 0; t0 < plan->n_tiles; t0 += P) {
      const int64_t nt = std::min(P, plan->n_tiles - t0);
      const size_t sb = tc_slice_bytes(9 * nt, K, kind);
      uint8_t* hi = static_cast<uint8_t*>(plan->d_coef_lp);
      uint8_t* lo = hi + sb;
      float* sc = reinterpret_cast<float*>(lo + sb);
      MSASM_TRY(tc_split_gpu(d_coef + size_t(9 * t0) * K, 9 * nt, K, kind, hi, lo, sc, s));
      MSASM_TRY(contract_tc_linop_gpu(kind, tab->d_Thi, tab->d_Tlo, tab->d_Tscale, tab->n_nz, hi, lo, sc, 9 * nt, K,
                                      d_u, d_y, plan->d_gmap, tab->d_pairs, tab->topo.n_T, t0, plan->d_tc_err, s));
    }
    return MSASM_OK;
  }
  if (prec == MSASM_F64_EMU && K <= 576) {
    // FP64-accurate form: the same in the 7-slice contraction's epilogue (FP64 products)
    msasm_tables* tab = const_cast<msasm_tables*>(plan->tab);
    const int n_nz = tab->n_nz;
    if (!tab->d_Tslices) {
      MSASM_CUDA(cudaMalloc(&tab->d_Tslices, emu_slice_bytes(n_nz, K)));
      MSASM_CUDA(cudaMalloc(&tab->d_Tslice_scale, size_t(n_nz) * sizeof(int)));
      MSASM_TRY(emu_slice_gpu(tab->d_T, n_nz, K, K, tab->d_Tslices, tab->d_Tslice_scale, s));
      tab->n_slices = 7;
    }
    MSASM_CUDA(cudaMemsetAsync(d_y, 0, size_t(plan->n_rows) * sizeof(double), s));
    for (int64_t t0 = 0; t0 < plan->n_tiles; t0 += P) {
      const int64_t nt = std::min(P, plan->n_tiles - t0);
      uint8_t* sl = static_cast<uint8_t*>(plan->d_coef_lp);
      int* sc = reinterpret_cast<int*>(sl + ((emu_slice_bytes(9 * nt, K) + 255) & ~size_t(255)));
      MSASM_TRY(emu_slice_gpu(d_coef + size_t(9 * t0) * K, 9 * nt, K, K, sl, sc, s));
      MSASM_TRY(contract_emu_linop_gpu(tab->d_Tslices, tab->d_Tslice_scale, n_nz, sl, sc, 9 * nt, K, d_u, d_y,
                                       plan->d_gmap, tab->d_pairs, tab->topo.n_T, t0, plan->d_tc_err, s));
    }
    return MSASM_OK;
  }
  MSASM_TRY(linop_prepare_gpu(plan, s));
  for (int64_t t0 = 0; t0 < plan->n_tiles; t0 += P) {
    const int64_t nt = std::min(P, plan->n_tiles - t0);
    MSASM_TRY(contract_dispatch(plan->tab, prec, d_coef + size_t(9 * t0) * K, nt, plan->d_nz, plan->d_coef_lp, s,
                                plan->d_tc_err));
    if (is_f64_precision(prec))
      MSASM_TRY(linop_pass_gpu<double>(plan, static_cast<const double*>(plan->d_nz), ld, t0, nt, d_u, d_y, s));
    else
      MSASM_TRY(linop_pass_gpu<float>(plan, reinterpret_cast<const float*>(plan->d_nz), ld, t0, nt, d_u, d_y, s));
  }
  return MSASM_OK;
}

msasm_status msasm_projection_error(const msasm_plan* plan, const double* d_ctrl, int32_t q, int32_t n_samples,
                                    double E, double nu, double* d_err_tiles, double* d_err_max, void* stream) {
  if (!plan || !d_ctrl || (!d_err_tiles && !d_err_max)) return fail(MSASM_EINVAL, "NULL argument or no output");
  MSASM_TRY(check_material(E, nu));
  double lam, mu;
  lame(E, nu, lam, mu);
  const int q3[3] = {q, q, q};
  return projection_error_gpu(plan, d_ctrl, q3, n_samples, lam, mu, d_err_tiles, d_err_max,
                              static_cast<cudaStream_t>(stream));
}

msasm_status msasm_projection_error_q3(const msasm_plan* plan, const double* d_ctrl, const int32_t* q3,
                                       int32_t n_samples, double E, double nu, double* d_err_tiles, double* d_err_max,
                                       void* stream) {
  if (!plan || !d_ctrl || !q3 || (!d_err_tiles && !d_err_max)) return fail(MSASM_EINVAL, "NULL argument or no output");
  MSASM_TRY(check_material(E, nu));
  double lam, mu;
  lame(E, nu, lam, mu);
  const int q[3] = {q3[0], q3[1], q3[2]};
  return projection_error_gpu(plan, d_ctrl, q, n_samples, lam, mu, d_err_tiles, d_err_max,
                              static_cast<cudaStream_t>(stream));
}

msasm_status msasm_projection_error_l2(const msasm_plan* plan, const double* d_ctrl, int32_t q, int32_t n_gauss,
                                       int32_t n_samples, double E, double nu, double* d_err_tiles, double* d_err_max,
                                       void* stream) {
  if (!plan || !d_ctrl || (!d_err_tiles && !d_err_max)) return fail(MSASM_EINVAL, "NULL argument or no output");
  if (n_gauss < 1) return fail(MSASM_EINVAL, "n_gauss must be at least 1");
  MSASM_TRY(check_material(E, nu));
  double lam, mu;
  lame(E, nu, lam, mu);
  const int q3[3] = {q, q, q};
  return projection_error_gpu(plan, d_ctrl, q3, n_samples, lam, mu, d_err_tiles, d_err_max,
                              static_cast<cudaStream_t>(stream), n_gauss);
}

// ---------------------------------------------------------------- degree selection (eq. 65, Sec. 3.3.4)
// Errors within a relative kDegreeBand count as equal, both when two candidates are compared and
// when an error is compared with the tolerance, so that rounding differences between
// implementations of E_proj cannot change the selected degrees.
constexpr double kDegreeBand = 1e-9;

namespace {
struct DegreeSearch {
  const msasm_plan* plan;
  const double* d_ctrl;
  int n_s;
  double lam, mu;
  cudaStream_t s;
  double* d_tmp = nullptr;
  std::vector<std::pair<std::array<int, 3>, double>> cache;
  // E_proj of eq. 59 (largest over the tiles) for the degrees q3, computed once per q3
  msasm_status err(const std::array<int, 3>& q3, double* out) {
    for (const auto& c : cache)
      if (c.first == q3) {
        *out = c.second;
        return MSASM_OK;
      }
    const int q[3] = {q3[0], q3[1], q3[2]};
    MSASM_TRY(projection_error_gpu(plan, d_ctrl, q, n_s, lam, mu, nullptr, d_tmp, s));
    double h = 0.0;
    MSASM_CUDA(cudaMemcpyAsync(&h, d_tmp, sizeof(double), cudaMemcpyDeviceToHost, s));
    MSASM_CUDA(cudaStreamSynchronize(s));
    cache.push_back({q3, h});
    *out = h;
    return MSASM_OK;
  }
};
}  // namespace

static bool meets(double e, double tol) { return e <= tol * (1.0 + kDegreeBand); }

msasm_status msasm_select_degree(const msasm_plan* plan, const double* d_ctrl, double tol, int32_t q0, int32_t q_max,
                                 int32_t n_samples, double E, double nu, int32_t* q_out, double* err_out,
                                 void* stream) {
  if (!plan || !d_ctrl || !q_out) return fail(MSASM_EINVAL, "plan, d_ctrl or q_out is NULL");
  if (!(tol > 0.0) || !std::isfinite(tol)) return fail(MSASM_EINVAL, "tol must be positive and finite");
  if (q0 < 0 || q_max > 7 || q0 > q_max) return fail(MSASM_EINVAL, "need 0 <= q0 <= q_max <= 7");
  MSASM_TRY(check_material(E, nu));
  DegreeSearch ds{plan, d_ctrl, n_samples, 0.0, 0.0, static_cast<cudaStream_t>(stream), nullptr, {}};
  lame(E, nu, ds.lam, ds.mu);
  MSASM_CUDA(cudaMallocAsync(&ds.d_tmp, sizeof(double), ds.s));
  msasm_status st = MSASM_OK;
  int q = q_max;
  double e = 0.0;
  for (int c = q0; c <= q_max && st == MSASM_OK; ++c) {
    st = ds.err({c, c, c}, &e);
    if (st == MSASM_OK && meets(e, tol)) {
      q = c;
      break;
    }
  }
  cudaFreeAsync(ds.d_tmp, ds.s);
  if (st != MSASM_OK) return st;
  *q_out = q;
  if (err_out) *err_out = e;
  return MSASM_OK;
}

msasm_status msasm_select_degrees(const msasm_plan* plan, const double* d_ctrl, double tol, const int32_t* q_init,
                                  int32_t q_max, int32_t n_samples, double E, double nu, int32_t* q_out,
                                  double* err_out, void* stream) {
  if (!plan || !d_ctrl || !q_init || !q_out) return fail(MSASM_EINVAL, "plan, d_ctrl, q_init or q_out is NULL");
  if (!(tol > 0.0) || !std::isfinite(tol)) return fail(MSASM_EINVAL, "tol must be positive and finite");
  if (q_max < 0 || q_max > 7) return fail(MSASM_EINVAL, "q_max must be in 0..7");
  for (int d = 0; d < 3; ++d)
    if (q_init[d] < 0 || q_init[d] > q_max) return fail(MSASM_EINVAL, "q_init must be in 0..q_max");
  MSASM_TRY(check_material(E, nu));
  DegreeSearch ds{plan, d_ctrl, n_samples, 0.0, 0.0, static_cast<cudaStream_t>(stream), nullptr, {}};
  lame(E, nu, ds.lam, ds.mu);
  MSASM_CUDA(cudaMallocAsync(&ds.d_tmp, sizeof(double), ds.s));
  std::array<int, 3> q = {q_init[0], q_init[1], q_init[2]};
  double err = 0.0;
  msasm_status st = ds.err(q, &err);
  // enrich: while the tolerance is not met, raise the direction whose increase lowers E_proj most
  while (st == MSASM_OK && !meets(err, tol)) {
    bool found = false;
    double best_e = 0.0;
    std::array<int, 3> best_q = q;
    for (int d = 0; d < 3 && st == MSASM_OK; ++d) {
      if (q[d] >= q_max) continue;
      std::array<int, 3> c = q;
      ++c[d];
      double e = 0.0;
      st = ds.err(c, &e);
      if (st == MSASM_OK && (!found || e < best_e * (1.0 - kDegreeBand))) {   // a tie keeps the lower direction
        found = true;
        best_e = e;
        best_q = c;
      }
    }
    if (!found) break;
    err = best_e;
    q = best_q;
  }
  // coarsen: while possible, lower the direction whose decrease keeps E_proj lowest and within tol
  while (st == MSASM_OK) {
    bool found = false;
    double best_e = 0.0;
    std::array<int, 3> best_q = q;
    for (int d = 0; d < 3 && st == MSASM_OK; ++d) {
      if (q[d] == 0) continue;
      std::array<int, 3> c = q;
      --c[d];
      double e = 0.0;
      st = ds.err(c, &e);
      if (st == MSASM_OK && meets(e, tol) && (!found || e < best_e * (1.0 - kDegreeBand))) {
        found = true;
        best_e = e;
        best_q = c;
      }
    }
    if (!found) break;
    err = best_e;
    q = best_q;
  }
  cudaFreeAsync(ds.d_tmp, ds.s);
  if (st != MSASM_OK) return st;
  for (int d = 0; d < 3; ++d) q_out[d] = q[d];
  if (err_out) *err_out = err;
  return MSASM_OK;
}

msasm_status msasm_pullback_l2(msasm_plan* plan, const double* d_ctrl, double E, double nu, int32_t n_gauss,
                               double* d_coef, void* stream) {
  if (!plan || !d_ctrl || !d_coef) return fail(MSASM_EINVAL, "plan, d_ctrl or d_coef is NULL");
  MSASM_TRY(check_material(E, nu));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double lam, mu;
  lame(E, nu, lam, mu);
  MSASM_CUDA(cudaMemsetAsync(plan->d_degenerate, 0, sizeof(unsigned long long), s));
  return l2_coef_gpu(plan, d_ctrl, plan->tab->qd, n_gauss, lam, mu, d_coef, s);
}

msasm_status msasm_load_table_copy(const msasm_tables* tab, double* d_F, double* d_vol, void* stream) {
  if (!tab || (!d_F && !d_vol)) return fail(MSASM_EINVAL, "tables is NULL or no output given");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t n_pi = size_t(tab->n_pi);
  if (d_F)
    MSASM_CUDA(cudaMemcpyAsync(d_F, tab->d_F, size_t(tab->topo.n_T) * n_pi * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (d_vol) MSASM_CUDA(cudaMemcpyAsync(d_vol, tab->d_vol, n_pi * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return MSASM_OK;
}

msasm_status msasm_volume(const msasm_plan* plan, const double* d_ctrl, double* d_tile_volume, double* d_total,
                          void* stream) {
  if (!plan || !d_ctrl || (!d_tile_volume && !d_total)) return fail(MSASM_EINVAL, "NULL argument or no output");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* tv = d_tile_volume;
  if (!tv) MSASM_CUDA(cudaMallocAsync(&tv, size_t(plan->n_tiles) * sizeof(double), s));
  msasm_status st = volume_load_gpu(plan, d_ctrl, tv, d_total, nullptr, nullptr, s);
  if (!d_tile_volume) cudaFreeAsync(tv, s);
  return st;
}

msasm_status msasm_volume_grad(const msasm_plan* plan, const double* d_ctrl, double* d_grad_ctrl, void* stream) {
  if (!plan || !d_ctrl || !d_grad_ctrl) return fail(MSASM_EINVAL, "plan, d_ctrl or d_grad_ctrl is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MSASM_CUDA(cudaMemsetAsync(d_grad_ctrl, 0, size_t(plan->n_ctrl) * 3 * sizeof(double), s));
  return adjoint_pullback_gpu(plan, d_ctrl, 0.0, 0.0, 0, plan->n_tiles, nullptr, false, d_grad_ctrl, s,
                              plan->tab->d_vol);
}

msasm_status msasm_body_load(const msasm_plan* plan, const double* d_ctrl, double bx, double by, double bz,
                             double* d_f, void* stream) {
  if (!plan || !d_ctrl || !d_f) return fail(MSASM_EINVAL, "plan, d_ctrl or d_f is NULL");
  if (!std::isfinite(bx) || !std::isfinite(by) || !std::isfinite(bz)) return fail(MSASM_EINVAL, "body force not finite");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MSASM_CUDA(cudaMemsetAsync(d_f, 0, size_t(plan->n_rows) * sizeof(double), s));
  const double b[3] = {bx, by, bz};
  return volume_load_gpu(plan, d_ctrl, nullptr, nullptr, d_f, b, s);
}

msasm_status msasm_traction_load_lookup(const msasm_plan* plan, const double* d_ctrl, int32_t face, double tx,
                                        double ty, double tz, double* d_f, void* stream) {
  if (!plan || !d_ctrl || !d_f) return fail(MSASM_EINVAL, "plan, d_ctrl or d_f is NULL");
  if (face < 0 || face > 5) return fail(MSASM_EINVAL, "face must be 0..5");
  if (!std::isfinite(tx) || !std::isfinite(ty) || !std::isfinite(tz)) return fail(MSASM_EINVAL, "traction not finite");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MSASM_CUDA(cudaMemsetAsync(d_f, 0, size_t(plan->n_rows) * sizeof(double), s));
  const double t[3] = {tx, ty, tz};
  return traction_load_gpu(plan, d_ctrl, face, t, d_f, s);
}

msasm_status msasm_face_table_copy(const msasm_tables* tab, int32_t face, double* d_Ff, void* stream) {
  if (!tab || !d_Ff) return fail(MSASM_EINVAL, "tables or d_Ff is NULL");
  if (face < 0 || face > 5) return fail(MSASM_EINVAL, "face must be 0..5");
  const size_t n = size_t(tab->face_off[face + 1] - tab->face_off[face]);
  MSASM_CUDA(cudaMemcpyAsync(d_Ff, tab->d_Fface + tab->face_off[face], n * sizeof(double), cudaMemcpyDeviceToDevice,
                             static_cast<cudaStream_t>(stream)));
  return MSASM_OK;
}

msasm_status msasm_degenerate_count(const msasm_plan* plan, int64_t* count, void* stream) {
  if (!plan || !count) return fail(MSASM_EINVAL, "plan or count is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long cnt = 0;
  MSASM_CUDA(cudaMemcpyAsync(&cnt, plan->d_degenerate, sizeof(cnt), cudaMemcpyDeviceToHost, s));
  MSASM_CUDA(cudaStreamSynchronize(s));
  *count = int64_t(cnt);
  return MSASM_OK;
}

msasm_status msasm_pullback(msasm_plan* plan, const double* d_ctrl, double E, double nu, double* d_coef,
                            void* stream) {
  if (!plan || !d_ctrl || !d_coef) return fail(MSASM_EINVAL, "plan, d_ctrl or d_coef is NULL");
  MSASM_TRY(check_material(E, nu));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double lam, mu;
  lame(E, nu, lam, mu);
  MSASM_CUDA(cudaMemsetAsync(plan->d_degenerate, 0, sizeof(unsigned long long), s));
  const int64_t P = plan->tiles_per_pass, K = 9 * plan->tab->n_pi;
  for (int64_t t0 = 0; t0 < plan->n_tiles; t0 += P) {
    const int64_t nt = std::min(P, plan->n_tiles - t0);
    MSASM_TRY(pullback_gpu(plan, d_ctrl, lam, mu, t0, nt, d_coef + size_t(9 * t0) * K, s));
  }
  return MSASM_OK;
}

msasm_status msasm_contract(const msasm_tables* tab, msasm_precision prec, const double* d_coef, int64_t n_tiles,
                            void* d_nz, void* stream) {
  if (!tab || !d_coef || !d_nz) return fail(MSASM_EINVAL, "tables, d_coef or d_nz is NULL");
  if (n_tiles <= 0) return fail(MSASM_EINVAL, "n_tiles must be positive");
  if (9 * n_tiles > 65535LL * 128) return fail(MSASM_EINVAL, "n_tiles too large for one contraction call");
  if (prec < MSASM_F64 || prec > MSASM_F64_EMU) return fail(MSASM_EINVAL, "unknown precision");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n_nz = tab->n_nz, K = 9 * tab->n_pi, ld = ld_nz_of(n_nz);
  // the public layout is dense (tile blocks n_nz x 9 values apart); contract into the kernels'
  // padded layout (ld x 9 per tile) and copy each tile's run
  void* scratch = nullptr;
  void* lp = nullptr;
  unsigned* d_err = nullptr;
  const size_t vb = value_bytes(prec);
  (void)K;
  MSASM_CUDA(cudaMallocAsync(&scratch, size_t(n_tiles) * 9 * ld * vb, s));
  MSASM_CUDA(cudaMallocAsync(&d_err, sizeof(unsigned), s));
  MSASM_CUDA(cudaMemsetAsync(d_err, 0, sizeof(unsigned), s));
  if (prec != MSASM_F64) MSASM_CUDA(cudaMallocAsync(&lp, coef_lp_bytes_for(n_tiles, tab->n_pi), s));
  msasm_status st = contract_dispatch(tab, prec, d_coef, n_tiles, scratch, lp, s, d_err);
  if (st == MSASM_OK) {
    cudaError_t e = cudaMemcpy2DAsync(d_nz, size_t(9) * n_nz * vb, scratch, size_t(9) * ld * vb,
                                      size_t(9) * n_nz * vb, size_t(n_tiles), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaMemcpy2DAsync(nz)");
  }
  unsigned h_err = 0;
  if (st == MSASM_OK) {
    cudaError_t e = cudaMemcpyAsync(&h_err, d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "msasm_contract");
  }
  cudaFreeAsync(scratch, s);
  cudaFreeAsync(d_err, s);
  if (lp) cudaFreeAsync(lp, s);
  if (st == MSASM_OK && h_err) st = fail(MSASM_ECUDA, "a tensor-core pipeline wait timed out (results invalid)");
  return st;
}

msasm_status msasm_scatter(msasm_plan* plan, msasm_precision prec, const void* d_nz, void* d_values, void* stream) {
  if (!plan || !d_nz || !d_values) return fail(MSASM_EINVAL, "plan, d_nz or d_values is NULL");
  if (prec < MSASM_F64 || prec > MSASM_F64_EMU) return fail(MSASM_EINVAL, "unknown precision");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n_nz = plan->tab->n_nz, ld = ld_nz_of(n_nz);
  const size_t vb = value_bytes(prec);
  // re-pad the dense public layout to the kernels' (ld x 9 values per tile)
  void* padded = nullptr;
  MSASM_CUDA(cudaMallocAsync(&padded, size_t(plan->n_tiles) * 9 * ld * vb, s));
  cudaError_t e = cudaMemcpy2DAsync(padded, size_t(9) * ld * vb, d_nz, size_t(9) * n_nz * vb, size_t(9) * n_nz * vb,
                                    size_t(plan->n_tiles), cudaMemcpyDeviceToDevice, s);
  msasm_status st = (e == cudaSuccess) ? scatter_dispatch(plan, prec, padded, 0, plan->n_tiles, d_values, s)
                                       : cuda_fail(e, "cudaMemcpy2DAsync(nz)");
  cudaFreeAsync(padded, s);
  return st;
}

}  // extern "C"
