// K4: the contraction of eq. 58 on the 5th-generation tensor cores (tcgen05, TMEM, TMA).
//
//   D[m][n] = sum_k T[m][k] coef[n][k],  written as nz[n][m]  (m: table row / pair, n = 9t + 3a + b)
//
// Operands are split into 16-bit (or TF32) slices so that the products reach FP32 accuracy
// (x = hi + lo):
//   split FP16 : x' = 2^e_row x, hi = fp16(x'), lo' = fp16(2^11 (x' - hi)); two TMEM accumulators
//                D0 = hi.hi and D1 = hi.lo' + lo'.hi, result (D0 + 2^-11 D1) 2^-(e_m + e_n)
//                (a power-of-two scale per row keeps every row inside FP16's range)
//   split BF16 : hi = bf16(x), lo = bf16(x - hi); D0 = hi.hi, D1 = hi.lo + lo.hi, result D0 + D1
//   TF32       : one product of the rounded operands
//   TF32x3     : hi = tf32(x), lo = tf32(x - hi); D0 = hi.hi, D1 = hi.lo + lo.hi, result D0 + D1
// Keeping the small cross terms in their own accumulator keeps their FP32 accumulation error
// relative to the small terms instead of to the whole sum.
//
// Persistent kernel, one CTA per SM looping over 128 (m) x BN (n) output tiles; 10 warps: warp 0
// issues TMA loads (128-byte swizzled K-major boxes) into a shared-memory ring that runs on across
// tiles, warp 1 owns the TMEM allocation and one elected lane issues tcgen05.mma (M=128, N=BN,
// K=16 for f16/bf16, K=8 for tf32), warps 2-9 (two per 32-lane TMEM quarter, BN/2 columns each)
// drain the accumulators into registers, release TMEM so that the next tile's MMAs start, then
// scale and store.  Two output layouts:
//   rows   (BN = 256, 2 stages): out[n][m], the rows of a warp contiguous in m (the MLP's output
//          layer uses it);
//   blocks (BN = 144 = lcm(16, 9), 3 stages): the tile blocks of eq. 58, out[t][m][3a + b] for
//          n = 9t + 3a + b, which the scatter reads block by block.  Each epilogue warp holds whole
//          tile blocks (72 columns = 8 tiles) for its 32 rows m; per tile it passes the 32 x 9 values
//          through a small shared-memory buffer so that each store instruction writes 32
//          consecutive floats of the tile's contiguous 32 x 9 run.
// Every mbarrier wait is bounded; on a timeout (or another thread's) the CTA records the error
// flag, drains what it issued and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>

#include "common.h"
#include "tc_ptx.cuh"

namespace msasm {

enum SplitKind { kSplitF16 = 0, kSplitBF16 = 1, kTF32 = 2, kTF32x3 = 3 };

constexpr int TC_BM = 128;          // rows of a CTA tile (TMEM lanes), table rows m
constexpr int TC_ROW_BYTES = 128;   // one swizzle row: 64 x 16-bit or 32 x 32-bit elements of k
constexpr int TC_A_BYTES = TC_BM * TC_ROW_BYTES;   // 16 KB

// shape of the kernel for an n tile of BN columns (256: row layout; 144: block layout)
template <int BN>
struct TcShape {
  static constexpr bool kBlocks = (BN % 9 == 0);
  static constexpr int kStages = kBlocks ? 3 : 2;
  static constexpr int kBBytes = BN * TC_ROW_BYTES;                          // 18 KB / 32 KB
  static constexpr int kStageBytes = 2 * TC_A_BYTES + 2 * kBBytes;
  static constexpr int kStagingFloats = 32 * 9;                              // one tile run of a warp
  static constexpr int kStagingBytes = kBlocks ? 8 * kStagingFloats * 4 : 0;
  static constexpr int kSmemBytes = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/ + kStagingBytes;
  static_assert(BN % 16 == 0 && BN <= 256, "tcgen05 M=128 needs N a multiple of 16, at most 256");
  static_assert(kSmemBytes <= 227 * 1024, "shared memory per CTA");
};

struct TcParams {
  int M, N, K;             // logical sizes: m rows, n rows, k
  int kblocks;             // k blocks of 128 bytes of operand
  int kind;                // SplitKind
  const float* scale_m;    // per-row 2^-e for split FP16 (else null)
  const float* scale_n;
  float* out;              // rows: out[n][m], leading dimension ld; blocks: out[n/9][m][n%9], m stride ld
  int ld;
  unsigned* err;           // set to 1 on a timed-out wait
  // matrix-free mode (y += K u, nothing stored): tile t0 + n/9 of the mesh, pair m = (A, B)
  const double* u;
  double* y;
  const int32_t* gmap;     // [t][A] global point ids
  const int32_t* pairs;    // [m][2] local (A, B), sorted by A
  int n_T;
  int64_t t0;
};

// ------------------------------------------------------------------ the kernel
constexpr int TC_EPI_WARPS = 8;                          // two per TMEM lane quarter
constexpr int TC_THREADS = 64 + 32 * TC_EPI_WARPS;       // producer warp, MMA warp, epilogue warps

template <int BN, bool LINOP>
__global__ void __launch_bounds__(TC_THREADS, 1)
    contract_tc_kernel(const __grid_constant__ CUtensorMap tmA_hi, const __grid_constant__ CUtensorMap tmA_lo,
                       const __grid_constant__ CUtensorMap tmB_hi, const __grid_constant__ CUtensorMap tmB_lo,
                       TcParams p) {
  using S = TcShape<BN>;
  constexpr int STAGES = S::kStages, STAGE_BYTES = S::kStageBytes, B_BYTES = S::kBBytes;
  constexpr int EPI_COLS = BN / 2;                             // columns of one epilogue warp
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;               // 1024-B alignment for the swizzle atoms
  uint8_t* gen_base = smem_raw + (base - raw);
  const uint32_t bar0 = base + STAGES * STAGE_BYTES;          // barriers after the stages
  // barrier layout: full[S], empty[S], accum_full, tmem_empty, then the TMEM address slot
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
  const uint32_t accum_full = bar0 + 8u * (2 * STAGES);
  const uint32_t tmem_empty = bar0 + 8u * (2 * STAGES + 1);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gen_base + STAGES * STAGE_BYTES + 8 * (2 * STAGES + 2));
  // block layout: one 32 x 9 staging run per epilogue warp after the barrier area
  float* staging = reinterpret_cast<float*>(gen_base + STAGES * STAGE_BYTES + 256);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_mt = (p.M + TC_BM - 1) / TC_BM, n_nt = (p.N + BN - 1) / BN;
  // tile t: m tile t % n_mt, n tile t / n_mt (CTAs running together share the coefficient tile and
  // sweep the table, the smaller operand, which stays in L2)
  const long long total = (long long)n_mt * n_nt;
  const bool two_acc = (p.kind != kTF32);
  const bool with_lo = (p.kind != kTF32);
  const float lo_weight = (p.kind == kSplitF16) ? 1.0f / 2048.0f : 1.0f;
  const uint32_t tmem_cols = two_acc ? 512u : 256u;
  const uint32_t stage_tx = with_lo ? STAGE_BYTES : (TC_A_BYTES + B_BYTES);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    mbar_init(accum_full, 1);
    mbar_init(tmem_empty, TC_EPI_WARPS);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA_hi)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB_hi)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer: the stage ring runs on across tiles
    uint32_t g = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < total && ok; t += gridDim.x) {
      const int m0 = int(t % n_mt) * TC_BM, n0 = int(t / n_mt) * BN;
      for (int kb = 0; kb < p.kblocks; ++kb, ++g) {
        const int s = int(g % STAGES);
        const uint32_t it = g / STAGES;
        if (it > 0 && !mbar_wait_or_abort(empty_bar(s), (it - 1) & 1, p.err)) {
          ok = false;
          break;
        }
        const uint32_t st = base + s * STAGE_BYTES;
        const int kx = kb * (p.kind >= kTF32 ? 32 : 64);       // element coordinate of the block
        mbar_expect_tx(full_bar(s), stage_tx);
        tma_load_2d(st, &tmA_hi, kx, m0, full_bar(s));
        tma_load_2d(st + 2 * TC_A_BYTES, &tmB_hi, kx, n0, full_bar(s));
        if (with_lo) {
          tma_load_2d(st + TC_A_BYTES, &tmA_lo, kx, m0, full_bar(s));
          tma_load_2d(st + 2 * TC_A_BYTES + B_BYTES, &tmB_lo, kx, n0, full_bar(s));
        }
      }
    }
    // every issued copy has landed before the CTA can exit (bounded)
    for (uint32_t q = (g > uint32_t(STAGES) ? g - STAGES : 0u); q < g; ++q)
      mbar_wait(full_bar(int(q % STAGES)), (q / STAGES) & 1, p.err);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    const bool tf = p.kind >= kTF32;
    const uint32_t idesc = instr_desc(p.kind == kSplitF16 ? 0u : (tf ? 2u : 1u), TC_BM, BN);
    const int ksteps = 4;                                       // 4 x 32 B of k per 128-B row
    const uint32_t acc0 = tmem, acc1 = tmem + (two_acc ? 256u : 0u);
    uint32_t g = 0, i_tile = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < total && ok; t += gridDim.x, ++i_tile) {
      if (i_tile > 0) {                                         // the previous tile is drained
        if (!mbar_wait_or_abort(tmem_empty, (i_tile - 1) & 1, p.err)) break;
        tc_fence_after();
      }
      for (int kb = 0; kb < p.kblocks; ++kb, ++g) {
        const int s = int(g % STAGES);
        const uint32_t it = g / STAGES;
        if (!mbar_wait_or_abort(full_bar(s), it & 1, p.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t st = base + s * STAGE_BYTES;
        const uint64_t a_hi = sw128_desc(st), a_lo = sw128_desc(st + TC_A_BYTES);
        const uint64_t b_hi = sw128_desc(st + 2 * TC_A_BYTES), b_lo = sw128_desc(st + 2 * TC_A_BYTES + B_BYTES);
#pragma unroll
        for (int j = 0; j < ksteps; ++j) {
          const uint64_t dk = uint64_t(2 * j);                    // +32 bytes of k, in 16-byte units
          const uint32_t first = (kb == 0 && j == 0) ? 0u : 1u;
          // hi.hi and hi.lo share the A tile: it stays in the collector buffer for the second
          if (tf) {
            if (with_lo) {
              mma_tf32_collect<CollectorA::FILL>(acc0, a_hi + dk, b_hi + dk, idesc, first);
              mma_tf32_collect<CollectorA::LASTUSE>(acc1, a_hi + dk, b_lo + dk, idesc, first);
              mma_tf32(acc1, a_lo + dk, b_hi + dk, idesc, 1u);
            } else {
              mma_tf32(acc0, a_hi + dk, b_hi + dk, idesc, first);
            }
          } else {
            mma_f16_collect<CollectorA::FILL>(acc0, a_hi + dk, b_hi + dk, idesc, first);
            mma_f16_collect<CollectorA::LASTUSE>(acc1, a_hi + dk, b_lo + dk, idesc, first);
            mma_f16(acc1, a_lo + dk, b_hi + dk, idesc, 1u);
          }
        }
        mma_commit(empty_bar(s));                                  // stage reusable when these MMAs finish
      }
      mma_commit(accum_full);                                      // this tile's accumulators are final
    }
    if (i_tile > 0) mbar_wait(accum_full, (i_tile - 1) & 1, p.err);   // nothing in flight at exit
  } else if (warp >= 2) {
    // ---------------- epilogue: drain TMEM into registers, release it, scale and store
    const int q = warp & 3;                                      // TMEM lane quarter of this warp
    const int h = (warp - 2) >> 2;                               // column half
    const uint32_t lane_off = uint32_t(32 * q) << 16;
    float* stg = staging + (warp - 2) * S::kStagingFloats;
    uint32_t i_tile = 0;
    for (long long t = blockIdx.x; t < total; t += gridDim.x, ++i_tile) {
      if (!mbar_wait_or_abort(accum_full, i_tile & 1, p.err)) break;
      tc_fence_after();
      const int m0 = int(t % n_mt) * TC_BM, n0 = int(t / n_mt) * BN + h * EPI_COLS;
      float R[EPI_COLS];
#pragma unroll
      for (int c = 0; c < EPI_COLS / 8; ++c) {
        uint32_t v[8], w[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        tmem_ld8_nowait(tmem + lane_off + uint32_t(h * EPI_COLS + 8 * c), v);
        if (two_acc) tmem_ld8_nowait(tmem + 256u + lane_off + uint32_t(h * EPI_COLS + 8 * c), w);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          asm volatile("" : "+r"(v[j]), "+r"(w[j]));             // uses stay after the wait
          R[8 * c + j] = two_acc ? fmaf(__uint_as_float(w[j]), lo_weight, __uint_as_float(v[j]))
                                 : __uint_as_float(v[j]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tmem_empty);                    // the MMAs of the next tile may start
      const int m = m0 + 32 * q + lane;
      const float sm = (p.scale_m && m < p.M) ? p.scale_m[m] : 1.0f;
      if constexpr (LINOP) {
        // y += K_t u block by block (Sec. 4.2: the tile matrices are applied, never stored): lane m
        // holds K_t[m] = block (A, B); rows of A get K u_B, summed over the run of lanes that share A
        // (the pairs are sorted by A) before one atomic add per run, rows of B get K^T u_A
        static_assert(S::kBlocks, "the matrix-free mode takes whole tile blocks");
        const bool mv = m < p.M;
        const int A = mv ? p.pairs[2 * m] : 0, B = mv ? p.pairs[2 * m + 1] : 0;
#pragma unroll
        for (int b = 0; b < EPI_COLS / 9; ++b) {
          const int nb = n0 + 9 * b;
          if (nb >= p.N) break;
          const int64_t tt = p.t0 + nb / 9;
          int gA = -1;
          float rA[3] = {0.f, 0.f, 0.f}, rB[3] = {0.f, 0.f, 0.f};
          int gB = -1;
          if (mv) {
            const int32_t* gt = p.gmap + tt * p.n_T;
            gA = gt[A];
            gB = gt[B];
            float kv[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) kv[k] = p.scale_m ? R[9 * b + k] * sm * p.scale_n[nb + k] : R[9 * b + k];
            const double* ua = p.u + 3 * int64_t(gA);
            const double* ub = p.u + 3 * int64_t(gB);
            const float a0 = float(ua[0]), a1 = float(ua[1]), a2 = float(ua[2]);
            const float b0 = float(ub[0]), b1 = float(ub[1]), b2 = float(ub[2]);
#pragma unroll
            for (int a = 0; a < 3; ++a) rA[a] = fmaf(kv[3 * a], b0, fmaf(kv[3 * a + 1], b1, kv[3 * a + 2] * b2));
            if (A != B) {
#pragma unroll
              for (int c = 0; c < 3; ++c) rB[c] = fmaf(kv[c], a0, fmaf(kv[3 + c], a1, kv[6 + c] * a2));
            }
          }
          const int prev = __shfl_up_sync(0xffffffffu, gA, 1);
          const bool head = (lane == 0) || (prev != gA);
          const unsigned heads = __ballot_sync(0xffffffffu, head);
          const int seg = __popc(heads & ((2u << lane) - 1u));   // runs of equal gA, numbered from 1
#pragma unroll
          for (int d = 1; d < 32; d *= 2) {                       // segmented suffix sums: the head gets its run's
            const int so = __shfl_down_sync(0xffffffffu, seg, d);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              const float o = __shfl_down_sync(0xffffffffu, rA[a], d);
              if (lane + d < 32 && so == seg) rA[a] += o;
            }
          }
          if (mv && head) {
#pragma unroll
            for (int a = 0; a < 3; ++a) atomicAdd(p.y + 3 * int64_t(gA) + a, double(rA[a]));
          }
          if (mv && A != B) {
#pragma unroll
            for (int c = 0; c < 3; ++c) atomicAdd(p.y + 3 * int64_t(gB) + c, double(rB[c]));
          }
        }
      } else if constexpr (S::kBlocks) {
        // n0 is a multiple of 9: the warp holds EPI_COLS / 9 whole tile blocks of its 32 rows
        const int mr0 = m0 + 32 * q;
#pragma unroll
        for (int b = 0; b < EPI_COLS / 9; ++b) {
          const int nb = n0 + 9 * b;
          if (nb >= p.N) break;                                  // N = 9 n_tiles: whole blocks only
#pragma unroll
          for (int k = 0; k < 9; ++k) {
            float val = R[9 * b + k];
            if (p.scale_m) val *= sm * p.scale_n[nb + k];
            stg[lane * 9 + k] = val;                              // stride 9: no bank conflicts
          }
          __syncwarp();
          float* dst = p.out + (size_t(nb / 9) * size_t(p.ld) + size_t(mr0)) * 9;
#pragma unroll
          for (int j = 0; j < 9; ++j) {
            const int e = 32 * j + lane;                          // element of the 32 x 9 run
            if (mr0 + e / 9 < p.M) __stcs(dst + e, stg[e]);     // evict-first: read by the next kernel
          }
          __syncwarp();
        }
      } else if (m < p.M) {
#pragma unroll
        for (int j = 0; j < EPI_COLS; ++j) {
          const int n = n0 + j;
          if (n < p.N) {
            float val = R[j];
            if (p.scale_m) val *= sm * p.scale_n[n];
            p.out[size_t(n) * p.ld + m] = val;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
  }
}

// ------------------------------------------------------------------ operand slicing
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// One warp per row: hi/lo slices of x[row][0..K) into [row][0..Kpad) (zero padded).
template <typename Tin>
__global__ void split_rows_kernel(const Tin* __restrict__ x, int64_t rows, int K, int Kpad, int kind,
                                  void* __restrict__ hi, void* __restrict__ lo, float* __restrict__ row_scale) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; r < rows;
       r += (int64_t(gridDim.x) * blockDim.x) >> 5) {
    const Tin* xr = x + r * K;
    double scale = 1.0;
    if (kind == kSplitF16) {
      double mx = 0.0;
      for (int k = lane; k < K; k += 32) mx = fmax(mx, fabs(double(xr[k])));
      for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      int e = 0;
      if (mx > 0.0) {
        frexp(mx, &e);                         // mx = f 2^e, f in [0.5, 1)
        scale = ldexp(1.0, 15 - e);            // scaled max in [2^14, 2^15)
      }
      if (lane == 0) row_scale[r] = float(1.0 / scale);
    }
    for (int k = lane; k < Kpad; k += 32) {
      const double v = (k < K) ? double(xr[k]) * scale : 0.0;
      if (kind == kSplitF16) {
        const __half h = __double2half(v);
        const __half l = __double2half((v - double(__half2float(h))) * 2048.0);
        static_cast<__half*>(hi)[r * Kpad + k] = h;
        static_cast<__half*>(lo)[r * Kpad + k] = l;
      } else if (kind == kSplitBF16) {
        const __nv_bfloat16 h = __double2bfloat16(v);
        const __nv_bfloat16 l = __double2bfloat16(v - double(__bfloat162float(h)));
        static_cast<__nv_bfloat16*>(hi)[r * Kpad + k] = h;
        static_cast<__nv_bfloat16*>(lo)[r * Kpad + k] = l;
      } else {
        const float h = tf32_round(float(v));
        static_cast<float*>(hi)[r * Kpad + k] = h;
        if (kind == kTF32x3) static_cast<float*>(lo)[r * Kpad + k] = tf32_round(float(v - double(h)));
      }
    }
  }
}

// ------------------------------------------------------------------ host side
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::mutex g_encode_mutex;

static msasm_status get_encoder() {
  std::lock_guard<std::mutex> lock(g_encode_mutex);
  if (g_encode) return MSASM_OK;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  MSASM_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
  if (q != cudaDriverEntryPointSuccess || !fn) return fail(MSASM_ECUDA, "cuTensorMapEncodeTiled is not available");
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return MSASM_OK;
}

// 2-D tensor map over a row-major [rows][Kpad] operand; box = 128 bytes of k x box_rows rows.
static msasm_status make_map(CUtensorMap* map, const void* ptr, int kind, int64_t rows, int K, int Kpad,
                             int box_rows) {
  const bool tf = kind >= kTF32;
  const int esz = tf ? 4 : 2;
  CUtensorMapDataType dt = tf ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                              : (kind == kSplitF16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
  cuuint64_t dims[2] = {cuuint64_t(K), cuuint64_t(rows)};
  cuuint64_t strides[1] = {cuuint64_t(Kpad) * esz};
  cuuint32_t box[2] = {cuuint32_t(TC_ROW_BYTES / esz), cuuint32_t(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(map, dt, 2, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(MSASM_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(int(r)) + ")");
  return MSASM_OK;
}

int tc_kind_of(msasm_precision prec) {
  switch (prec) {
    case MSASM_SPLIT_F16: return kSplitF16;
    case MSASM_SPLIT_BF16: return kSplitBF16;
    case MSASM_TF32: return kTF32;
    case MSASM_TF32X3: return kTF32x3;
    default: return -1;
  }
}

int tc_kpad(int K, int kind) {
  const int per_row = (kind >= kTF32) ? 32 : 64;          // elements per 128-byte box row
  return (K + per_row - 1) / per_row * per_row;
}

size_t tc_slice_bytes(int64_t rows, int K, int kind) {
  const int esz = kind >= kTF32 ? 4 : 2;
  return size_t(rows) * tc_kpad(K, kind) * esz;
}

template <typename Tin>
static msasm_status tc_split_any(const Tin* x, int64_t rows, int K, int kind, void* hi, void* lo, float* row_scale,
                                 cudaStream_t s) {
  int64_t blocks = (rows * 32 + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  split_rows_kernel<Tin><<<unsigned(blocks), 256, 0, s>>>(x, rows, K, tc_kpad(K, kind), kind, hi, lo, row_scale);
  MSASM_CUDA(cudaGetLastError());
  return MSASM_OK;
}
msasm_status tc_split_gpu(const double* x, int64_t rows, int K, int kind, void* hi, void* lo, float* row_scale,
                          cudaStream_t s) {
  return tc_split_any<double>(x, rows, K, kind, hi, lo, row_scale, s);
}
msasm_status tc_split_f32_gpu(const float* x, int64_t rows, int K, int kind, void* hi, void* lo, float* row_scale,
                              cudaStream_t s) {
  return tc_split_any<float>(x, rows, K, kind, hi, lo, row_scale, s);
}

template <int BN, bool LINOP = false>
static msasm_status launch_tc(const CUtensorMap& ma_hi, const CUtensorMap& ma_lo, const CUtensorMap& mb_hi,
                              const CUtensorMap& mb_lo, const TcParams& p, cudaStream_t s) {
  constexpr int smem = TcShape<BN>::kSmemBytes;
  MSASM_CUDA(cudaFuncSetAttribute(contract_tc_kernel<BN, LINOP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const long long tiles = ((p.M + TC_BM - 1) / TC_BM) * (long long)((p.N + BN - 1) / BN);
  if (tiles == 0) return MSASM_OK;
  int dev = 0, n_sm = 0;
  MSASM_CUDA(cudaGetDevice(&dev));
  MSASM_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  const unsigned grid = unsigned(std::min<long long>(tiles, std::max(n_sm, 1)));   // one CTA per SM
  contract_tc_kernel<BN, LINOP><<<grid, TC_THREADS, smem, s>>>(ma_hi, ma_lo, mb_hi, mb_lo, p);
  MSASM_CUDA(cudaGetLastError());
  return MSASM_OK;
}

// D[m][n] = sum_k A[m][k] B[n][k] (FP32) from sliced operands A (table, M rows) and B (coef, N
// rows), stored as out[n][m] with leading dimension ld (blocks = false), or as the tile blocks of
// eq. 58, out[n/9][m][n%9] with m stride ld (blocks = true; N a multiple of 9).
struct TcLinop {                // the matrix-free mode's arguments (null y: store the product)
  const double* u = nullptr;
  double* y = nullptr;
  const int32_t* gmap = nullptr;
  const int32_t* pairs = nullptr;
  int n_T = 0;
  int64_t t0 = 0;
};

static msasm_status contract_tc_any(int kind, const void* a_hi, const void* a_lo, const float* a_scale, int M,
                                    const void* b_hi, const void* b_lo, const float* b_scale, int64_t N, int K,
                                    float* out, int ld, bool blocks, const TcLinop& lin, unsigned* d_err,
                                    cudaStream_t s) {
  MSASM_TRY(get_encoder());
  if (N > int64_t(2147483647)) return fail(MSASM_EUNSUPPORTED, "too many coefficient rows for one launch");
  if (blocks && N % 9 != 0) return fail(MSASM_EINVAL, "the block layout needs whole tiles (N a multiple of 9)");
  const int Kpad = tc_kpad(K, kind);
  const int bn = blocks ? 144 : 256;
  CUtensorMap ma_hi, ma_lo, mb_hi, mb_lo;
  MSASM_TRY(make_map(&ma_hi, a_hi, kind, M, K, Kpad, TC_BM));
  MSASM_TRY(make_map(&mb_hi, b_hi, kind, N, K, Kpad, bn));
  if (kind != kTF32) {
    MSASM_TRY(make_map(&ma_lo, a_lo, kind, M, K, Kpad, TC_BM));
    MSASM_TRY(make_map(&mb_lo, b_lo, kind, N, K, Kpad, bn));
  } else {
    ma_lo = ma_hi;
    mb_lo = mb_hi;
  }
  TcParams p;
  p.M = M;
  p.N = int(N);
  p.K = K;
  p.kblocks = Kpad / ((kind >= kTF32) ? 32 : 64);
  p.kind = kind;
  p.scale_m = (kind == kSplitF16) ? a_scale : nullptr;
  p.scale_n = (kind == kSplitF16) ? b_scale : nullptr;
  p.out = out;
  p.ld = ld;
  p.err = d_err;
  p.u = lin.u;
  p.y = lin.y;
  p.gmap = lin.gmap;
  p.pairs = lin.pairs;
  p.n_T = lin.n_T;
  p.t0 = lin.t0;
  if (lin.y) return launch_tc<144, true>(ma_hi, ma_lo, mb_hi, mb_lo, p, s);
  return blocks ? launch_tc<144>(ma_hi, ma_lo, mb_hi, mb_lo, p, s) : launch_tc<256>(ma_hi, ma_lo, mb_hi, mb_lo, p, s);
}

msasm_status contract_tc_gpu(int kind, const void* a_hi, const void* a_lo, const float* a_scale, int M,
                             const void* b_hi, const void* b_lo, const float* b_scale, int64_t N, int K, float* out,
                             int ld, bool blocks, unsigned* d_err, cudaStream_t s) {
  return contract_tc_any(kind, a_hi, a_lo, a_scale, M, b_hi, b_lo, b_scale, N, K, out, ld, blocks, TcLinop(), d_err, s);
}

// y += K u for the N / 9 tiles t0 .. of the coefficient slices B, without storing the tile matrices:
// the split-form contraction whose epilogue applies each block to u (FP32 products of the FP32
// block values and u, FP64 atomic additions into y; y must hold the sum so far)
msasm_status contract_tc_linop_gpu(int kind, const void* a_hi, const void* a_lo, const float* a_scale, int M,
                                   const void* b_hi, const void* b_lo, const float* b_scale, int64_t N, int K,
                                   const double* u, double* y, const int32_t* gmap, const int32_t* pairs, int n_T,
                                   int64_t t0, unsigned* d_err, cudaStream_t s) {
  if (N % 9 != 0) return fail(MSASM_EINVAL, "the matrix-free contraction takes whole tiles");
  TcLinop lin;
  lin.u = u;
  lin.y = y;
  lin.gmap = gmap;
  lin.pairs = pairs;
  lin.n_T = n_T;
  lin.t0 = t0;
  return contract_tc_any(kind, a_hi, a_lo, a_scale, M, b_hi, b_lo, b_scale, N, K, nullptr, 0, true, lin, d_err, s);
}

}  // namespace msasm
