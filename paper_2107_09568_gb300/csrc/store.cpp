// Persistence of the lookup tables of a reference tile (Sec. 3.1.1, 3.2.3: the tables of a
// microstructure are computed once, offline, and stored; an assembly only reads them).
//
// Table file payload (kind tag "MSASMTAB"): the micro descriptor (n_patches; per patch degree[3],
// n_elem[3] as int32, box_lo[3], box_hi[3] as double), the projection degrees q3 (int32[3]),
// n_gauss, n_T, n_nz, n_pi (int32), face_off[7] (int64), then the FP64 arrays T (n_nz x 9 n_pi),
// F (n_T x n_pi), vol (n_pi) and the face tables (face_off[6] values).  Loading rebuilds the tile
// topology from the stored descriptor and checks that it reproduces the stored sizes, so the
// pair order of T always matches the topology it is used with.
#include <algorithm>

#include "common.h"
#include "store.h"

using namespace msasm;

static const char kTableTag[8] = {'M', 'S', 'A', 'S', 'M', 'T', 'A', 'B'};

static msasm_status tables_save_impl(const msasm_tables* tab, const char* path, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StoreWriter w;
  const int32_t n_patches = int32_t(tab->topo.patches.size());
  w.put(n_patches);
  for (const Patch& P : tab->topo.patches) {
    w.put_array(P.degree, 3);
    w.put_array(P.n_elem, 3);
    w.put_array(P.lo, 3);
    w.put_array(P.hi, 3);
  }
  const int32_t sizes[7] = {tab->qd[0], tab->qd[1], tab->qd[2], tab->n_gauss, tab->topo.n_T, tab->n_nz, tab->n_pi};
  w.put_array(sizes, 7);
  w.put_array(tab->face_off, 7);
  const size_t nT = size_t(tab->n_nz) * 9 * tab->n_pi, nF = size_t(tab->topo.n_T) * tab->n_pi;
  const size_t nV = size_t(tab->n_pi), nFf = size_t(tab->face_off[6]);
  double* hT = w.reserve_array<double>(nT + nF + nV + nFf);
  MSASM_CUDA(cudaMemcpyAsync(hT, tab->d_T, nT * 8, cudaMemcpyDeviceToHost, s));
  MSASM_CUDA(cudaMemcpyAsync(hT + nT, tab->d_F, nF * 8, cudaMemcpyDeviceToHost, s));
  MSASM_CUDA(cudaMemcpyAsync(hT + nT + nF, tab->d_vol, nV * 8, cudaMemcpyDeviceToHost, s));
  if (nFf) MSASM_CUDA(cudaMemcpyAsync(hT + nT + nF + nV, tab->d_Fface, nFf * 8, cudaMemcpyDeviceToHost, s));
  MSASM_CUDA(cudaStreamSynchronize(s));
  return w.write(path, kTableTag);
}

extern "C" {

msasm_status msasm_tables_save(const msasm_tables* tab, const char* path, void* stream) {
  if (!tab || !path) return fail(MSASM_EINVAL, "tables or path is NULL");
  try {
    return tables_save_impl(tab, path, stream);
  } catch (const std::bad_alloc&) {
    return fail(MSASM_ENOMEM, "no host memory to stage the tables");
  }
}

msasm_status msasm_tables_load(const char* path, void* stream, msasm_tables** out) {
  if (!out || !path) return fail(MSASM_EINVAL, "out or path is NULL");
  *out = nullptr;
  StoreReader r;
  MSASM_TRY(r.open(path, kTableTag));
  auto bad = [&](const char* what) { return fail(MSASM_EIO, std::string("table file: ") + what + ": " + path); };
  int32_t n_patches = 0;
  if (!r.get(n_patches) || n_patches <= 0 || n_patches > 16) return bad("patch count");
  std::vector<int32_t> degree(size_t(3) * n_patches), n_elem(size_t(3) * n_patches);
  std::vector<double> lo(size_t(3) * n_patches), hi(size_t(3) * n_patches);
  for (int p = 0; p < n_patches; ++p) {
    bool ok = true;
    for (int d = 0; d < 3; ++d) ok = ok && r.get(degree[size_t(3) * p + d]);
    for (int d = 0; d < 3; ++d) ok = ok && r.get(n_elem[size_t(3) * p + d]);
    for (int d = 0; d < 3; ++d) ok = ok && r.get(lo[size_t(3) * p + d]);
    for (int d = 0; d < 3; ++d) ok = ok && r.get(hi[size_t(3) * p + d]);
    if (!ok) return bad("patch descriptor");
  }
  int32_t sizes[7];
  int64_t face_off[7];
  for (int i = 0; i < 7; ++i)
    if (!r.get(sizes[i])) return bad("sizes");
  for (int i = 0; i < 7; ++i)
    if (!r.get(face_off[i])) return bad("face offsets");
  for (int d = 0; d < 3; ++d)
    if (sizes[d] < 0 || sizes[d] > 5) return bad("projection degrees outside 0..5");
  msasm_micro_desc micro;
  micro.n_patches = n_patches;
  micro.degree = degree.data();
  micro.n_elem = n_elem.data();
  micro.box_lo = lo.data();
  micro.box_hi = hi.data();
  msasm_tables* tab = new msasm_tables();
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto bail = [&](msasm_status st) {
    delete tab;
    return st;
  };
  // the topology is rebuilt from the descriptor before any table value is trusted
  TileTopology probe;
  msasm_status st = build_topology(&micro, probe);
  if (st != MSASM_OK) return bail(st);
  const int32_t n_pi = (sizes[0] + 1) * (sizes[1] + 1) * (sizes[2] + 1);
  if (probe.n_T != sizes[4] || int32_t(probe.pair_A.size()) != sizes[5] || n_pi != sizes[6])
    return bail(bad("the stored sizes do not match the tile the descriptor builds"));
  const size_t nT = size_t(sizes[5]) * 9 * n_pi, nF = size_t(sizes[4]) * n_pi, nV = size_t(n_pi);
  const size_t nFf = face_off[6] >= 0 ? size_t(face_off[6]) : 0;
  const unsigned char* src = r.get_array<double>(nT + nF + nV + nFf);
  if (!src || !r.at_end()) return bail(bad("table arrays"));
  st = tables_init(&micro, sizes, sizes[3], s, tab);
  if (st != MSASM_OK) return bail(st);
  for (int i = 0; i < 7; ++i)
    if (tab->face_off[i] != face_off[i]) return bail(bad("face table offsets"));
  cudaError_t e = cudaMalloc(&tab->d_F, nF * 8);
  if (e == cudaSuccess) e = cudaMalloc(&tab->d_vol, nV * 8);
  if (e == cudaSuccess) e = cudaMalloc(&tab->d_Fface, std::max<size_t>(nFf, 1) * 8);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tab->d_T, src, nT * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tab->d_F, src + nT * 8, nF * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tab->d_vol, src + (nT + nF) * 8, nV * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nFf)
    e = cudaMemcpyAsync(tab->d_Fface, src + (nT + nF + nV) * 8, nFf * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the reader's buffer must outlive the copies
  if (e != cudaSuccess) return bail(cuda_fail(e, "msasm_tables_load"));
  *out = tab;
  return MSASM_OK;
}

}  // extern "C"
