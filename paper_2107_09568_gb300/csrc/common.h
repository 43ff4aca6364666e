// Internal declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/msasm.h"

namespace msasm {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
msasm_status fail(msasm_status st, const std::string& msg);
msasm_status cuda_fail(cudaError_t err, const char* what);

#define MSASM_CUDA(call)                                          \
  do {                                                            \
    cudaError_t err__ = (call);                                   \
    if (err__ != cudaSuccess) return ::msasm::cuda_fail(err__, #call); \
  } while (0)

#define MSASM_TRY(call)                                           \
  do {                                                            \
    msasm_status st__ = (call);                                   \
    if (st__ != MSASM_OK) return st__;                            \
  } while (0)

// ------------------------------------------------------------------ host math (host_math.cpp)
// Gauss-Legendre rule with n points on [0,1] (Newton on the Legendre recurrence).
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w);
// Nonzero B-spline basis functions of degree p on the knot span `span` at u, and
// their first derivatives: vals[0..p], ders[0..p] belong to functions span-p .. span.
void bspline_span_basis(const double* knots, int p, int span, double u, double* vals, double* ders);
// Index of the knot span [t_k, t_{k+1}) holding u (the last non-empty span for u = end).
int bspline_find_span(const double* knots, int n_knots, int p, double u);

// ------------------------------------------------------------------ reference tile topology (host_tile.cpp)
struct Patch {
  int degree[3];
  int n_elem[3];
  int n_fun[3];
  double lo[3], hi[3];
  std::vector<int> ids;   // local id of patch function a1 + n1*(a2 + n2*a3)
};

struct TileTopology {
  std::vector<Patch> patches;
  int n_T = 0;
  std::vector<double> pos;              // 3*n_T control point positions in [0,1]^3
  std::vector<int> pair_A, pair_B;      // I_coo (eq. 56), lexicographic, A <= B
  std::vector<int64_t> nb_ptr;          // local adjacency incl. self (both orders)
  std::vector<int> nb_idx;
  std::vector<int> faces[6];            // local ids on xi_d = s (index 2d+s), matched order
  std::vector<int> face_pos[6];         // position of a local id in faces[f], -1 if absent
  std::vector<uint8_t> pair_face;       // bit d: A and B both on the xi_d = 0 face
};

msasm_status build_topology(const msasm_micro_desc* micro, TileTopology& topo);

// ------------------------------------------------------------------ handles
constexpr int kMaxPairPatches = 4;   // a point on a corner of the centre cube lies in 4 patches
struct PairDesc {       // the patch contributions to one table row
  int8_t patch[kMaxPairPatches];      // -1 = none
  int8_t a[kMaxPairPatches][3];
  int8_t b[kMaxPairPatches][3];
  int8_t pad[4];
};
static_assert(sizeof(PairDesc) == 32, "PairDesc is two 16-byte words");

// one block a tile adds to rows owned by a lower tile (secondary scatter pass)
struct SecondaryEntry {
  int64_t dst_u, dst_l;      // first value index of the upper block (rows of A) / lower block (rows of B)
  int32_t len_u, len_l;      // their row lengths
  int32_t tile;
  uint32_t m_flags;          // m | upper << 30 | lower << 31
};
static_assert(sizeof(SecondaryEntry) == 32, "SecondaryEntry is 32 bytes");

// scatter plan (scatter_plan.cpp): a tile's owned rows are one contiguous range of values whose
// layout depends only on the tile's type (which faces are glued), so one value map per type
// tells, for every value of the range, where it comes from in the tile's nzdata
constexpr int kScatterSegment = 4096;     // values of one chunk of a tile's owned range (one CTA)
constexpr int kScatterPieces = 8;         // direct-pass pieces whose secondary pass runs on a second stream
inline int ld_nz_of(int n_nz) { return (n_nz + 7) & ~7; }   // leading dimension of nzdata rows
struct ScatterPlanHost {
  std::vector<int32_t> tile_type;          // per tile
  std::vector<int64_t> type_rep;           // per type: representative tile
  std::vector<int32_t> type_nvals;         // per type: values in the owned rows of a tile
  std::vector<int64_t> type_map_off;       // per type: offset of its value map (n_types + 1)
  std::vector<uint32_t> tmpl;              // secondary template per type: m | upper << 30 | lower << 31
  std::vector<int64_t> tmpl_ptr;
  std::vector<int64_t> sec_off;            // per tile: first secondary entry (n_tiles + 1)
  std::vector<int32_t> type_rows;          // per type, per owned row: offset in the range, length, A << 2 | a
  std::vector<int64_t> type_row_off;       // per type: first row in type_rows (n_types + 1)
};

}  // namespace msasm

struct msasm_tables {
  msasm::TileTopology topo;
  int q = 0;                        // the largest of the per-direction projection degrees
  int qd[3] = {0, 0, 0};            // projection degree per direction (q1, q2, q3)
  int64_t face_off[7] = {0, 0, 0, 0, 0, 0, 0};   // face table f at d_Fface + face_off[f]
  int n_pi = 0;                     // (q1+1)(q2+1)(q3+1)
  int n_nz = 0;
  int n_gauss = 0;
  int ref_point = 0;                // local point nearest the tile centre
  double* d_T = nullptr;            // n_nz x 9 n_pi, FP64
  double* d_F = nullptr;            // load table n_T x n_pi (eq. 55, body term), FP64
  double* d_vol = nullptr;          // volume table n_pi (eq. 18), FP64
  double* d_Fface = nullptr;        // face load tables, face f: n_T x (q_a+1)(q_b+1) (eq. 55, F >= 1), FP64
  int32_t* d_pairs = nullptr;       // 2 n_nz (A, B)
  // operand copies for the reduced-precision contractions (created on first use)
  float* d_T32 = nullptr;           // FP32 copy
  void* d_Thi = nullptr;            // hi/lo 16-bit or tf32 operand slices
  void* d_Tlo = nullptr;
  float* d_Tscale = nullptr;        // per-row 2^-e of the split-FP16 slices
  double* d_Tt = nullptr;           // transposed table [9 n_pi][n_nz] for the adjoint (FP64)
  float* d_Tt32 = nullptr;          // the same in FP32
  int split_kind = -1;              // which precision the slices hold
  void* d_Tslices = nullptr;        // FP64-emulation slices
  int n_slices = 0;
  int* d_Tslice_scale = nullptr;    // power-of-two exponent per table row of the emulation slices
  void* d_Tslices4 = nullptr;       // the 4 slices of the FP32 form (28 bits)
  int* d_Tslice_scale4 = nullptr;
  ~msasm_tables();
};

namespace msasm {
msasm_status tables_init(const msasm_micro_desc* micro, const int32_t q3[3], int n_gauss, cudaStream_t s,
                         msasm_tables* tab);
}  // namespace msasm

struct msasm_mlp;
struct msasm_surrogate;

struct msasm_plan {
  const msasm_tables* tab = nullptr;
  int degree[3] = {0, 0, 0};
  int n_elem[3] = {0, 0, 0};
  int n_ctrl_dir[3] = {0, 0, 0};
  int64_t n_tiles = 0, n_points = 0, n_rows = 0, nnz = 0, n_ctrl = 0;
  int64_t tiles_per_pass = 0;
  // macro basis at the interpolation nodes: per direction d, element e, node c, local function a:
  // value and d/dxi (already scaled by the span length), and the first control index of the span.
  double* d_basis[3] = {nullptr, nullptr, nullptr};   // [e][c][a][2]
  int32_t* d_first[3] = {nullptr, nullptr, nullptr};  // [e]
  // structure
  int32_t* d_gmap = nullptr;        // n_tiles x n_T
  int64_t* d_rowptr = nullptr;      // n_rows + 1
  int32_t* d_col = nullptr;         // nnz
  uint32_t* d_rank = nullptr;       // n_tiles x n_nz: rank_u | rank_l << 16, bit 31 = second contributor
  // scatter (device copies of ScatterPlanHost)
  int32_t* d_tile_type = nullptr;
  int32_t* d_type_nvals = nullptr;
  int64_t* d_type_map_off = nullptr;
  int32_t* d_maps = nullptr;                 // value maps of all types: 9 m + 3a + b, or -1
  int64_t* d_tile_vbase = nullptr;
  uint32_t* d_tmpl = nullptr;
  int64_t* d_tmpl_ptr = nullptr;
  int64_t* d_sec_off = nullptr;              // secondary entries of tile t: [sec_off[t], sec_off[t+1])
  msasm::SecondaryEntry* d_sec = nullptr;
  std::vector<int64_t> sec_off_host;
  // matrix-free operator (built at its first use): per-type column maps and row tables
  std::vector<int64_t> type_rep_host, type_map_off_host, type_row_off_host;
  std::vector<int32_t> type_rows_host;
  int max_type_rows = 0;
  int32_t* d_colmaps = nullptr;              // per value: column point << 2 | beta (same offsets as d_maps)
  int32_t* d_type_rows = nullptr;
  int64_t* d_type_row_off = nullptr;
  std::vector<double> knots_host[3];  // host copies for boundary data
  std::vector<int> span_host[3];      // knot index of each element's span
  std::vector<int32_t> gmap_host;
  std::vector<int64_t> tile_vbase;    // host: first value index of the rows owned by tile t (n_tiles + 1)
  std::vector<int64_t> tile_pbase;    // host: first global point id owned by tile t (n_tiles + 1)
  cudaStream_t copy_stream[2] = {nullptr, nullptr};   // device->host copies of msasm_assemble_host
  // second stream of the scatter: the secondary pass of each finished piece of the direct pass
  cudaStream_t scatter_side = nullptr;
  cudaEvent_t scatter_ev[msasm::kScatterPieces + 1] = {};
  std::vector<cudaEvent_t> copy_events;
  // scratch
  double* d_coef = nullptr;         // 9 tiles_per_pass x 9 n_pi, FP64
  void* d_nz = nullptr;             // 9 tiles_per_pass x n_nz, FP64-sized
  void* d_coef_lp = nullptr;        // reduced-precision coefficient operands
  void* d_adj_lp = nullptr;         // slices of one chunk of the transposed table (emulated FP64 adjoint)
  size_t coef_lp_bytes = 0;
  unsigned long long* d_degenerate = nullptr;
  unsigned* d_tc_err = nullptr;     // set by a tensor-core kernel whose pipeline wait timed out
  double* d_ctrl_stage = nullptr;   // device copy of the control net for msasm_assemble_host
  void* d_values_stage = nullptr;
  size_t values_stage_bytes = 0;
  // stage timing (MSASM_FLAG_STAGE_TIMES): events per pass, 4 per pass (before pullback,
  // contraction, scatter, after scatter), and the launches each stage issued
  std::vector<cudaEvent_t> events;
  int timed_passes = 0;
  int stage_launches[3] = {0, 0, 0};
  ~msasm_plan();
};
