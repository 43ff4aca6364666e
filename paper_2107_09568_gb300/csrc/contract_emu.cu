// K4 (FP64 and FP32 forms): the contraction of eq. 58 to FP64 (or FP32) accuracy on the BF16
// tensor cores.
//
// GB300 executes FP64 at about 1.2 TFLOP/s, so the exact-accumulation slicing scheme of Ozaki,
// Ogita, Oishi and Rump (2012) is used instead: every row x of either operand is scaled by a
// power of two sigma >= max|x| and cut into S slices of 7 bits (S = 7 for FP64, S = 4 for FP32),
//
//   x / sigma = sum_{i=0..S-1} a_i 2^-7(i+1),  a_0 in [-128, 128], a_i in [-64, 64] (i > 0),
//
// each stored exactly in BF16 as s_i = a_i 2^-7i.  Then
//   D[m][n] = sigma_m tau_n 2^-14 sum_{i+j <= S-1} sum_k s_i[m][k] t_j[n][k]
// (the terms with i + j > S - 1 are below 2^-7S of the result).  Grouping the products by
// d = i + j, acc_d for d = 0..3 holds a sum of integer multiples of 2^-7d whose magnitude stays
// below 2^24 for K <= 576 (per k: |a_0 b_0| <= 2^14, 2 * 2^13, 2 * 2^13 + 2^12, 2 * 2^13 + 2 * 2^12
// in units of the diagonal), so the tensor cores' FP32 accumulation is exact in them whatever its
// internal rounding; for S = 7, acc4 collects d = 4..6, at most 2^-28 of acc0, where that rounding
// is harmless.  (Merging d = 3 into the last accumulator, with its mixed scales, measurably loses
// accuracy: the accumulation truncates relative to the largest term.)  The epilogue forms the
// exact fixed-point sum X = sum_d acc_d 2^(7 n_acc) in int64 (acc4 rounded at 2^-35, by integer
// operations) and writes X 2^(e_m + e_n - 14 - 7 n_acc) rounded to nearest even: one conversion of X
// to FP64 (or FP32), then the exponent field moved by integer addition.  No FP64 arithmetic (about
// 1/64 of the FP32 rate per SM on GB300) is used; float-to-int64 conversions, which measured slow
// on this chip (20.9 against 16.1 ms for the kernel), are not used either.  The FP32 form keeps 28
// bits of each operand row (10 products, 4 accumulators, all exact): its error is the truncation of
// the operands, the same whatever the accumulation order.
//
// Persistent kernel, one CTA per SM looping over 128 (m) x 96 (n) output tiles.  Per 16-element
// k block, one 3-D TMA box brings all S slices of each operand (32-byte swizzle) into a ring that
// runs on across tiles; one lane issues the S(S+1)/2 MMAs (M=128, N=96, K=16, the A slice kept in
// the collector buffer across its products) into min(S, 5) TMEM accumulators of 96 columns (at
// most 480 of the 512).  Eight epilogue warps (two per TMEM lane quarter, 48 columns each) drain
// the accumulators into exact int64 sums in registers (the last accumulator as raw values, folded
// in afterwards) and release TMEM at once, so the MMAs of the next tile run while they round and
// store the previous one.  In the tile-block layout of nzdata a warp rounds 12 (FP64-accurate
// form) or 24 columns at a time into shared memory and writes each tile block's 32 rows as one run.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "common.h"
#include "tc_ptx.cuh"

namespace msasm {

constexpr int EMU_BM = 128, EMU_BN = 96, EMU_KB = 16;    // k block: 16 BF16 = one 32-byte swizzle row
constexpr int EMU_A_SLICE = EMU_BM * 32;                 // one slice tile of A: 128 rows x 32 bytes
constexpr int EMU_B_SLICE = EMU_BN * 32;                 // one slice tile of B: 96 rows x 32 bytes
// block layout: each epilogue warp rounds 24 columns of its 32 rows into a shared-memory buffer (odd
// row stride: few bank conflicts either way) and writes them back tile block by tile block; the
// FP64-accurate form stages 12 columns at a time, which leaves room for a fourth pipeline stage (its
// matrix-free mode keeps 24 columns and 3 stages: it applies whole blocks per round)

// the kernel's shape for S slices per operand (OutT the output type, BLOCKS the nzdata layout,
// LINOP the matrix-free mode)
template <int S, typename OutT, bool BLOCKS, bool LINOP>
struct EmuShape {
  static constexpr int kAcc = S < 5 ? S : 5;             // accumulators: d = 0..3 alone, d >= 4 together
  static constexpr int kABytes = S * EMU_A_SLICE;        // 28 KB (S = 7)
  static constexpr int kBBytes = S * EMU_B_SLICE;        // 21 KB (S = 7)
  static constexpr int kStageBytes = kABytes + kBBytes;
  static constexpr bool kNarrow = S == 7 && !LINOP;             // 12 staged columns, 4 stages
  static constexpr int kStages = S == 7 ? (kNarrow ? 4 : 3) : 6; // ring depth
  static constexpr int kStgCols = kNarrow ? 12 : 24;             // staged columns per round
  static constexpr int kStgLd = kStgCols + 1;
  static constexpr int kStgElems = 32 * kStgLd;
  static constexpr int kStagingBytes = BLOCKS ? 8 * kStgElems * int(sizeof(OutT)) : 0;
  static constexpr int kSmemBytes = kStages * kStageBytes + 1024 + 256 + kStagingBytes;
  static_assert(kSmemBytes <= 227 * 1024, "shared memory per CTA");
  static_assert(S >= 1 && S <= 7 && 5 * EMU_BN <= 512, "slices and TMEM columns");
};

struct EmuParams {
  int M, N, kblocks;
  const int* exp_m;        // sigma_m = 2^exp_m
  const int* exp_n;        // tau_n = 2^exp_n
  void* out;               // rows: out[n][m], leading dimension ld; blocks: out[n/9][m][n%9], m stride ld
  int ld;
  unsigned* err;
  // matrix-free mode (y += K u, nothing stored): tile t0 + n/9 of the mesh, pair m = (A, B)
  const double* u;
  double* y;
  const int32_t* gmap;     // [t][A] global point ids
  const int32_t* pairs;    // [m][2] local (A, B), sorted by A
  int n_T;
  int64_t t0;
};

// x 2^e as the nearest FP64 (ties to even): the conversion of x rounds to nearest (even), and
// scaling by 2^e is exact, so it only moves the exponent field; results below the normal range
// give a signed zero and above it a signed infinity.
__device__ __forceinline__ double round_out(long long x, int e, double*) {
  const double d = __ll2double_rn(x);
  const long long b = __double_as_longlong(d);
  const int be = int((b >> 52) & 0x7ff);
  if (be == 0) return d;                                          // x == 0
  const int nb = be + e;
  const long long sign = b & (long long)0x8000000000000000ull;
  if (nb <= 0) return __longlong_as_double(sign);
  if (nb >= 2047) return __longlong_as_double(sign | 0x7FF0000000000000ll);
  return __longlong_as_double((long long)((unsigned long long)b + ((unsigned long long)(long long)e << 52)));
}
// the same to FP32
__device__ __forceinline__ float round_out(long long x, int e, float*) {
  const float f = __ll2float_rn(x);
  const uint32_t b = __float_as_uint(f);
  const int be = int((b >> 23) & 0xff);
  if (be == 0) return f;
  const int nb = be + e;
  if (nb <= 0) return __uint_as_float(b & 0x80000000u);
  if (nb >= 255) return __uint_as_float((b & 0x80000000u) | 0x7F800000u);
  return __uint_as_float(b + (uint32_t(e) << 23));
}

constexpr int EMU_BAND = 32;                              // m tiles per band of the tile order
constexpr int EMU_EPI_WARPS = 8;                          // two per TMEM lane quarter
constexpr int EMU_THREADS = 64 + 32 * EMU_EPI_WARPS;      // producer warp, MMA warp, epilogue warps
constexpr int EMU_EPI_COLS = EMU_BN / 2;                  // columns of one epilogue warp

// Nearest int64 to a float (ties to even) by integer operations on its bits (|y| < 2^62).
__device__ __forceinline__ long long f32_to_i64_rn(float y) {
  const uint32_t b = __float_as_uint(y);
  const uint32_t mag = b & 0x7fffffffu;
  if (mag < 0x3f000000u) return 0;                         // |y| < 0.5 (and zeros, subnormals)
  const int ex = int(mag >> 23) - 150;                     // |y| = m 2^ex, m = 24-bit significand
  const unsigned long long m = (mag & 0x7fffffu) | 0x800000u;
  unsigned long long r;
  if (ex >= 0) {
    r = m << ex;
  } else {
    const int sh = -ex;                                    // 1..24
    r = m >> sh;
    const unsigned long long rem = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (r & 1ull))) ++r;
  }
  return (b >> 31) ? -(long long)r : (long long)r;
}

template <int S, typename OutT, bool ACCUMULATE, bool BLOCKS, bool LINOP = false>
__global__ void __launch_bounds__(EMU_THREADS, 1)
    contract_emu_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, EmuParams p) {
  using Sh = EmuShape<S, OutT, BLOCKS, LINOP>;
  constexpr int EMU_STAGES = Sh::kStages, EMU_STAGE_BYTES = Sh::kStageBytes, EMU_A_BYTES = Sh::kABytes;
  constexpr int EMU_ACC = Sh::kAcc;
  constexpr int EMU_STG_COLS = Sh::kStgCols, EMU_STG_LD = Sh::kStgLd, EMU_STG_ELEMS = Sh::kStgElems;
  OutT* const out = static_cast<OutT*>(p.out);
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gen_base = smem_raw + (base - raw);
  const uint32_t bar0 = base + EMU_STAGES * EMU_STAGE_BYTES;
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (EMU_STAGES + s); };
  const uint32_t accum_full = bar0 + 8u * (2 * EMU_STAGES);      // MMAs of a tile done
  const uint32_t tmem_empty = bar0 + 8u * (2 * EMU_STAGES + 1);  // accumulators drained
  uint32_t* tmem_slot =
      reinterpret_cast<uint32_t*>(gen_base + EMU_STAGES * EMU_STAGE_BYTES + 8 * (2 * EMU_STAGES + 2));
  OutT* staging = reinterpret_cast<OutT*>(gen_base + EMU_STAGES * EMU_STAGE_BYTES + 256);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_nt = (p.N + EMU_BN - 1) / EMU_BN, n_mt = (p.M + EMU_BM - 1) / EMU_BM;
  const long long total = (long long)n_nt * n_mt;
  // tile t -> (m tile, n tile) in bands of EMU_BAND m tiles: within a band the n tiles advance
  // and the band's m tiles run together, so the CTAs in flight share a few operand tiles of
  // each side and the band's table slices (EMU_BAND x 1 MB) stay in L2 while the coefficient
  // slices stream past once per band
  auto tile_mn = [&](long long t, int& m0, int& n0) {
    const long long band = t / ((long long)EMU_BAND * n_nt);
    const int rows = min(EMU_BAND, n_mt - int(band) * EMU_BAND);
    const long long r = t - band * EMU_BAND * n_nt;
    m0 = (int(band) * EMU_BAND + int(r % rows)) * EMU_BM;
    n0 = int(r / rows) * EMU_BN;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < EMU_STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    mbar_init(accum_full, 1);
    mbar_init(tmem_empty, EMU_EPI_WARPS);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer: both operands' S slices per k block, ring across tiles
    uint32_t g = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < total && ok; t += gridDim.x) {
      int m0, n0;
      tile_mn(t, m0, n0);
      for (int kb = 0; kb < p.kblocks; ++kb, ++g) {
        const int s = int(g % EMU_STAGES);
        const uint32_t it = g / EMU_STAGES;
        if (it > 0 && !mbar_wait_or_abort(empty_bar(s), (it - 1) & 1, p.err)) {
          ok = false;
          break;
        }
        const uint32_t st = base + s * EMU_STAGE_BYTES;
        mbar_expect_tx(full_bar(s), EMU_STAGE_BYTES);
        tma_load_3d(st, &tmA, kb * EMU_KB, m0, 0, full_bar(s));
        tma_load_3d(st + EMU_A_BYTES, &tmB, kb * EMU_KB, n0, 0, full_bar(s));
      }
    }
    // every issued copy has landed before the CTA can exit (bounded)
    for (uint32_t q = (g > uint32_t(EMU_STAGES) ? g - EMU_STAGES : 0u); q < g; ++q)
      mbar_wait(full_bar(int(q % EMU_STAGES)), (q / EMU_STAGES) & 1, p.err);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer: S(S+1)/2 products per k block, grouped by i + j
    const uint32_t idesc = instr_desc(1u, EMU_BM, EMU_BN);        // BF16 x BF16 -> F32
    uint32_t g = 0, i_tile = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < total && ok; t += gridDim.x, ++i_tile) {
      if (i_tile > 0) {                                           // the previous tile is drained
        if (!mbar_wait_or_abort(tmem_empty, (i_tile - 1) & 1, p.err)) break;
        tc_fence_after();
      }
      uint32_t started = 0;                                       // accumulators already written
      for (int kb = 0; kb < p.kblocks; ++kb, ++g) {
        const int s = int(g % EMU_STAGES);
        const uint32_t it = g / EMU_STAGES;
        if (!mbar_wait_or_abort(full_bar(s), it & 1, p.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t st = base + s * EMU_STAGE_BYTES;
#pragma unroll
        for (int i = 0; i < S; ++i) {
          // slice i of A stays in the collector buffer for its S - i products
          const uint64_t a = sw32_desc(st + i * EMU_A_SLICE);
#pragma unroll
          for (int j = 0; j + i < S; ++j) {
            const int acc = (i + j < EMU_ACC - 1) ? i + j : EMU_ACC - 1;
            const uint64_t b = sw32_desc(st + EMU_A_BYTES + j * EMU_B_SLICE);
            const uint32_t accumulate = (started >> acc) & 1u;
            const uint32_t d = tmem + uint32_t(acc * EMU_BN);
            if (i + j == S - 1 && j == 0)
              mma_f16(d, a, b, idesc, accumulate);                                   // a single product
            else if (j == 0)
              mma_f16_collect<CollectorA::FILL>(d, a, b, idesc, accumulate);
            else if (i + j == S - 1)
              mma_f16_collect<CollectorA::LASTUSE>(d, a, b, idesc, accumulate);
            else
              mma_f16_collect<CollectorA::USE>(d, a, b, idesc, accumulate);
            started |= 1u << acc;
          }
        }
        mma_commit(empty_bar(s));                                 // stage reusable when these finish
      }
      mma_commit(accum_full);                                     // this tile's accumulators are final
    }
    if (i_tile > 0) mbar_wait(accum_full, (i_tile - 1) & 1, p.err);   // nothing in flight at exit
  } else if (warp >= 2) {
    // ---------------- epilogue: drain the accumulators into exact int64 sums, release, round, store
    const int q = warp & 3;                                       // TMEM lane quarter of this warp
    const int h = (warp - 2) >> 2;                                // column half
    const uint32_t lane_off = uint32_t(32 * q) << 16;
    uint32_t i_tile = 0;
    for (long long t = blockIdx.x; t < total; t += gridDim.x, ++i_tile) {
      if (!mbar_wait_or_abort(accum_full, i_tile & 1, p.err)) break;
      tc_fence_after();
      int m0, n0;
      tile_mn(t, m0, n0);
      n0 += h * EMU_EPI_COLS;
      long long X[EMU_EPI_COLS];
      uint32_t R4[EMU_ACC == 5 ? EMU_EPI_COLS : 1];               // acc4 raw: converted after the release
#pragma unroll
      for (int c = 0; c < EMU_EPI_COLS / 8; ++c) {
        uint32_t v[EMU_ACC][8];
#pragma unroll
        for (int a = 0; a < EMU_ACC; ++a)
          tmem_ld8_nowait(tmem + lane_off + uint32_t(a * EMU_BN + h * EMU_EPI_COLS + 8 * c), v[a]);
        tmem_wait_ld();
#pragma unroll
        for (int a = 0; a < EMU_ACC; ++a)
#pragma unroll
          for (int j = 0; j < 8; ++j) asm volatile("" : "+r"(v[a][j]));   // uses stay after the wait
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          // exact integers acc_d 2^7d for d <= 3 (all below 2^24 in magnitude) at weight 2^7(n_acc - d);
          // for S = 7, acc4 (d >= 4) rounded at 2^-35
          long long x = 0;
#pragma unroll
          for (int a = 0; a < (EMU_ACC < 4 ? EMU_ACC : 4); ++a)
            x += (long long)__float2int_rn(__uint_as_float(v[a][j]) * __int_as_float((127 + 7 * a) << 23))
                 << (7 * (EMU_ACC - a));
          if constexpr (EMU_ACC == 5) R4[8 * c + j] = v[4][j];
          X[8 * c + j] = x;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tmem_empty);                     // the MMAs of the next tile may start
      if constexpr (EMU_ACC == 5) {
#pragma unroll
        for (int j = 0; j < EMU_EPI_COLS; ++j) X[j] += f32_to_i64_rn(__uint_as_float(R4[j]) * 34359738368.0f);
      }
      const int m = m0 + 32 * q + lane;
      const int em = (m < p.M) ? p.exp_m[m] - 14 - 7 * EMU_ACC : 0;   // D = X 2^(e_m + e_n - 14 - 7 n_acc)
      if constexpr (BLOCKS) {
        // the tile blocks of eq. 58, nz[t][m][3a + b] for n = 9t + 3a + b: the 32 rows of a block
        // are one run of 32 x 9 values, written with consecutive lanes on consecutive addresses
        OutT* stg = staging + (warp - 2) * EMU_STG_ELEMS;
        const int mr0 = m0 + 32 * q;
#pragma unroll
        for (int half = 0; half < EMU_EPI_COLS / EMU_STG_COLS; ++half) {
          const int c0 = n0 + half * EMU_STG_COLS;
#pragma unroll
          for (int j = 0; j < EMU_STG_COLS; ++j) {
            const int n = c0 + j;
            stg[lane * EMU_STG_LD + j] =
                (m < p.M && n < p.N) ? round_out(X[half * EMU_STG_COLS + j], em + p.exp_n[n], stg) : OutT(0);
          }
          __syncwarp();
          const int cend = min(c0 + EMU_STG_COLS, p.N);
          if constexpr (LINOP) {
            // y += K_t u (Sec. 4.2: applied, never stored): lane m's columns of block tb in this chunk
            // (a block split across chunks or n tiles contributes in parts), the rows of A summed over
            // the run of lanes sharing A before one atomic add per run, the rows of B per lane
            const bool mv = m < p.M;
            const int A = mv ? p.pairs[2 * m] : 0, B = mv ? p.pairs[2 * m + 1] : 0;
            for (int tb = c0 / 9; 9 * tb < cend; ++tb) {
              const int ka = max(9 * tb, c0), kb = min(9 * tb + 9, cend);
              int gA = -1, gB = -1;
              double rA[3] = {0.0, 0.0, 0.0}, rB[3] = {0.0, 0.0, 0.0};
              if (mv) {
                const int32_t* gt = p.gmap + (p.t0 + tb) * p.n_T;
                gA = gt[A];
                gB = gt[B];
                const double* ua = p.u + 3 * int64_t(gA);
                const double* ub = p.u + 3 * int64_t(gB);
                const double a3[3] = {ua[0], ua[1], ua[2]}, b3[3] = {ub[0], ub[1], ub[2]};
#pragma unroll
                for (int ab = 0; ab < 9; ++ab) {
                  const int k = 9 * tb + ab;
                  if (k >= ka && k < kb) {
                    const double v = double(stg[lane * EMU_STG_LD + (k - c0)]);
                    rA[ab / 3] = fma(v, b3[ab % 3], rA[ab / 3]);
                    if (A != B) rB[ab % 3] = fma(v, a3[ab / 3], rB[ab % 3]);
                  }
                }
              }
              const int prev = __shfl_up_sync(0xffffffffu, gA, 1);
              const bool head = (lane == 0) || (prev != gA);
              const unsigned heads = __ballot_sync(0xffffffffu, head);
              const int seg = __popc(heads & ((2u << lane) - 1u));
#pragma unroll
              for (int d = 1; d < 32; d *= 2) {
                const int so = __shfl_down_sync(0xffffffffu, seg, d);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                  const double o = __shfl_down_sync(0xffffffffu, rA[a], d);
                  if (lane + d < 32 && so == seg) rA[a] += o;
                }
              }
              if (mv && head) {
#pragma unroll
                for (int a = 0; a < 3; ++a) atomicAdd(p.y + 3 * int64_t(gA) + a, rA[a]);
              }
              if (mv && A != B) {
#pragma unroll
                for (int c = 0; c < 3; ++c) atomicAdd(p.y + 3 * int64_t(gB) + c, rB[c]);
              }
            }
          } else {
            for (int tb = c0 / 9; 9 * tb < cend; ++tb) {
              const int ka = max(9 * tb, c0), kc = min(9 * tb + 9, cend) - ka;   // columns of block tb here
              OutT* dst = out + (size_t(tb) * size_t(p.ld) + size_t(mr0)) * 9 + (ka - 9 * tb);
              const OutT* src = stg + (ka - c0);
              // e / kc as (e inv) >> 32 with inv = ceil(2^32 / kc): exact for e < 2^16, one division per block
              const unsigned long long inv = (unsigned long long)(0xFFFFFFFFu / unsigned(kc)) + 1ull;
              for (int e = lane; e < 32 * kc; e += 32) {
                const int r = int(((unsigned long long)e * inv) >> 32), kk = e - r * kc;
                if (mr0 + r < p.M) __stcs(dst + r * 9 + kk, src[r * EMU_STG_LD + kk]);   // evict-first: read by the next kernel
              }
            }
          }
          __syncwarp();
        }
      } else if (m < p.M) {
#pragma unroll
        for (int j = 0; j < EMU_EPI_COLS; ++j) {
          const int n = n0 + j;
          if (n < p.N) {
            OutT* o = out + size_t(n) * p.ld + m;
            const OutT v = round_out(X[j], em + p.exp_n[n], o);
            if constexpr (ACCUMULATE) *o += v;
            else *o = v;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
  }
}

// x 2^(bits - e) rounded to the nearest integer (ties to even), for |x| < 2^e, from the FP64 bit
// pattern by integer shifts: the fixed-point value whose base-128 digits are the slices.
__device__ __forceinline__ long long fixed_point(double x, int e, int bits) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = int((b >> 52) & 0x7ffu);
  unsigned long long M = b & ((1ull << 52) - 1);
  if (E == 0 && M == 0) return 0;
  int Eeff = 1;
  if (E != 0) {
    M |= 1ull << 52;
    Eeff = E;
  }
  // |x| = M 2^(Eeff - 1075), so X = M 2^-s with s = 1075 - bits + e - Eeff (s >= 4 for a normal x < 2^e
  // and bits <= 49)
  const int sh = 1075 - bits + e - Eeff;
  unsigned long long X;
  if (sh <= 0) {
    X = M << (-sh);
  } else if (sh >= 64) {
    X = 0;
  } else {
    X = M >> sh;
    const unsigned long long rem = M & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (X & 1ull))) ++X;
  }
  return (b >> 63) ? -(long long)X : (long long)X;
}

// One warp per row: sigma = 2^e >= max|x| and the S BF16 slices s_i = a_i 2^-7i, [i][row][Kpad],
// where X = x 2^(7S-e) = sum_i a_i 128^(S-1-i) with balanced digits a_i in [-64, 63] (i > 0) and
// |a_0| <= 128.  Integer instructions only (the FP64 pipe runs at 1/64 of the FP32 rate).
template <int S>
__global__ void emu_slice_kernel(const double* __restrict__ x, int64_t rows, int64_t ldx, int K, int Kpad,
                                 __nv_bfloat16* __restrict__ slices, int* __restrict__ scale_exp) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; r < rows;
       r += (int64_t(gridDim.x) * blockDim.x) >> 5) {
    const double* xr = x + r * ldx;
    unsigned long long mb = 0;                 // max |x| as a bit pattern (monotone for x >= 0)
    for (int k = lane; k < K; k += 32) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(xr[k]) & 0x7fffffffffffffffull;
      mb = b > mb ? b : mb;
    }
    for (int o = 16; o; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(0xffffffffu, mb, o);
      mb = y > mb ? y : mb;
    }
    int e = 0;
    if (mb != 0) frexp(__longlong_as_double((long long)mb), &e);   // max = f 2^e, f in [0.5, 1)
    if (lane == 0) scale_exp[r] = e;
    for (int k = 2 * lane; k < Kpad; k += 64) {
      long long X[2];
      X[0] = (k < K) ? fixed_point(xr[k], e, 7 * S) : 0;
      X[1] = (k + 1 < K) ? fixed_point(xr[k + 1], e, 7 * S) : 0;
      int a[2][S];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int i = S - 1; i >= 1; --i) {
          const long long d = ((X[h] + 64) & 127) - 64;
          a[h][i] = int(d);
          X[h] = (X[h] - d) / 128;             // exact
        }
        a[h][0] = int(X[h]);
      }
#pragma unroll
      for (int i = 0; i < S; ++i) {
        const float p = __int_as_float((127 - 7 * i) << 23);      // 2^-7i
        __nv_bfloat162 v;
        v.x = __float2bfloat16_rn(float(a[0][i]) * p);            // exact: |a| <= 128
        v.y = __float2bfloat16_rn(float(a[1][i]) * p);
        *reinterpret_cast<__nv_bfloat162*>(slices + (size_t(i) * rows + r) * Kpad + k) = v;
      }
    }
  }
}

int emu_kpad(int K) { return (K + EMU_KB - 1) / EMU_KB * EMU_KB; }

size_t emu_slice_bytes(int64_t rows, int K, int n_slices) {
  return size_t(n_slices) * rows * emu_kpad(K) * sizeof(__nv_bfloat16);
}

// rows of x with leading dimension ldx (elements), K of them each, into n_slices (7 or 4) slices
msasm_status emu_slice_gpu(const double* x, int64_t rows, int64_t ldx, int K, void* slices, int* scale_exp,
                           cudaStream_t s, int n_slices) {
  if (K > 576 + 15) return fail(MSASM_EUNSUPPORTED, "FP64 emulation is exact for K <= 576 (q <= 3)");
  if (n_slices != 7 && n_slices != 4) return fail(MSASM_EINVAL, "emulation slices must be 7 (FP64) or 4 (FP32)");
  int64_t blocks = std::min<int64_t>((rows * 32 + 255) / 256, 152 * 16);
  if (n_slices == 7)
    emu_slice_kernel<7><<<unsigned(blocks), 256, 0, s>>>(x, rows, ldx, K, emu_kpad(K),
                                                         static_cast<__nv_bfloat16*>(slices), scale_exp);
  else
    emu_slice_kernel<4><<<unsigned(blocks), 256, 0, s>>>(x, rows, ldx, K, emu_kpad(K),
                                                         static_cast<__nv_bfloat16*>(slices), scale_exp);
  MSASM_CUDA(cudaGetLastError());
  return MSASM_OK;
}

static PFN_cuTensorMapEncodeTiled_v12000 g_encode3 = nullptr;
static std::mutex g_encode3_mutex;

static msasm_status make_map_3d(CUtensorMap* map, const void* ptr, int64_t rows, int K, int box_rows, int n_slices) {
  {
    std::lock_guard<std::mutex> lock(g_encode3_mutex);
    if (!g_encode3) {
      void* fn = nullptr;
      cudaDriverEntryPointQueryResult q;
      MSASM_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
      if (q != cudaDriverEntryPointSuccess || !fn) return fail(MSASM_ECUDA, "cuTensorMapEncodeTiled unavailable");
      g_encode3 = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
  }
  const int Kpad = emu_kpad(K);
  cuuint64_t dims[3] = {cuuint64_t(K), cuuint64_t(rows), cuuint64_t(n_slices)};
  cuuint64_t strides[2] = {cuuint64_t(Kpad) * 2, cuuint64_t(rows) * Kpad * 2};
  cuuint32_t box[3] = {cuuint32_t(EMU_KB), cuuint32_t(box_rows), cuuint32_t(n_slices)};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode3(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(ptr), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(MSASM_ECUDA, "cuTensorMapEncodeTiled (3-D) failed (" + std::to_string(int(r)) + ")");
  return MSASM_OK;
}

template <int S, typename OutT, bool ACCUMULATE, bool BLOCKS, bool LINOP = false>
static msasm_status launch_emu(const CUtensorMap& ma, const CUtensorMap& mb, const EmuParams& p, cudaStream_t s) {
  constexpr int smem = EmuShape<S, OutT, BLOCKS, LINOP>::kSmemBytes;
  auto kernel = contract_emu_kernel<S, OutT, ACCUMULATE, BLOCKS, LINOP>;
  MSASM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const long long tiles = ((p.N + EMU_BN - 1) / EMU_BN) * (long long)((p.M + EMU_BM - 1) / EMU_BM);
  if (tiles == 0) return MSASM_OK;
  int dev = 0, n_sm = 0;
  MSASM_CUDA(cudaGetDevice(&dev));
  MSASM_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  const unsigned grid = unsigned(std::min<long long>(tiles, std::max(n_sm, 1)));   // one CTA per SM
  kernel<<<grid, EMU_THREADS, smem, s>>>(ma, mb, p);
  MSASM_CUDA(cudaGetLastError());
  return MSASM_OK;
}

// D[m][n] = sum_k A[m][k] B[n][k] from the slices of A (M rows) and B (N rows), n_slices of each:
// 7 slices give FP64 results (out double*), 4 give FP32 results (out float*, block layout only).
// Stored as out[n][m] with leading dimension ld (blocks = false; accumulate adds to out), or as the
// tile blocks of eq. 58, out[n/9][m][n%9] with m stride ld (blocks = true; N a multiple of 9).
msasm_status contract_emu_gpu(const void* a_slices, const int* a_exp, int M, const void* b_slices,
                              const int* b_exp, int64_t N, int K, void* out, int ld, bool accumulate, bool blocks,
                              unsigned* d_err, cudaStream_t s, int n_slices) {
  if (N > int64_t(2147483647) * EMU_BN) return fail(MSASM_EUNSUPPORTED, "too many rows for one launch");
  if (blocks && (accumulate || N % 9 != 0))
    return fail(MSASM_EINVAL, "the block layout takes whole tiles (N a multiple of 9) and no accumulation");
  if (n_slices != 7 && !(n_slices == 4 && blocks))
    return fail(MSASM_EINVAL, "the 4-slice (FP32) contraction writes the block layout only");
  CUtensorMap ma, mb;
  MSASM_TRY(make_map_3d(&ma, a_slices, M, K, EMU_BM, n_slices));
  MSASM_TRY(make_map_3d(&mb, b_slices, N, K, EMU_BN, n_slices));
  EmuParams p;
  p.M = M;
  p.N = int(N);
  p.kblocks = emu_kpad(K) / EMU_KB;
  p.exp_m = a_exp;
  p.exp_n = b_exp;
  p.out = out;
  p.ld = ld;
  p.err = d_err;
  p.u = nullptr;
  p.y = nullptr;
  p.gmap = nullptr;
  p.pairs = nullptr;
  p.n_T = 0;
  p.t0 = 0;
  if (n_slices == 4) return launch_emu<4, float, false, true>(ma, mb, p, s);
  if (blocks) return launch_emu<7, double, false, true>(ma, mb, p, s);
  return accumulate ? launch_emu<7, double, true, false>(ma, mb, p, s) : launch_emu<7, double, false, false>(ma, mb, p, s);
}

// y += K u for the N / 9 tiles t0 .. of the coefficient slices B (FP64-accurate, 7 slices), without
// storing the tile matrices: the epilogue applies each rounded block value to u (FP64 products, FP64
// atomic additions into y; y must hold the sum so far)
msasm_status contract_emu_linop_gpu(const void* a_slices, const int* a_exp, int M, const void* b_slices,
                                    const int* b_exp, int64_t N, int K, const double* u, double* y,
                                    const int32_t* gmap, const int32_t* pairs, int n_T, int64_t t0, unsigned* d_err,
                                    cudaStream_t s) {
  if (N > int64_t(2147483647) * EMU_BN) return fail(MSASM_EUNSUPPORTED, "too many rows for one launch");
  if (N % 9 != 0) return fail(MSASM_EINVAL, "the matrix-free contraction takes whole tiles");
  CUtensorMap ma, mb;
  MSASM_TRY(make_map_3d(&ma, a_slices, M, K, EMU_BM, 7));
  MSASM_TRY(make_map_3d(&mb, b_slices, N, K, EMU_BN, 7));
  EmuParams p;
  p.M = M;
  p.N = int(N);
  p.kblocks = emu_kpad(K) / EMU_KB;
  p.exp_m = a_exp;
  p.exp_n = b_exp;
  p.out = nullptr;
  p.ld = 0;
  p.err = d_err;
  p.u = u;
  p.y = y;
  p.gmap = gmap;
  p.pairs = pairs;
  p.n_T = n_T;
  p.t0 = t0;
  return launch_emu<7, double, false, true, true>(ma, mb, p, s);
}

}  // namespace msasm
