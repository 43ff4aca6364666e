// msasm_contract_noalloc: the FP64 contraction stage (eq. 58) without any device
// allocation, for callers that cannot let the library call cudaMalloc/cudaFree.
//
// Some callers own all of the device memory: a host application that reserves
// the GPU's memory up front for its own pool leaves nothing for cudaMalloc, and
// a latency-bound service that only allocates at start-up cannot accept the
// device-wide synchronisation that cudaFree implies in the middle of its work.
// msasm_contract allocates a padded output buffer on every call; this variant
// uses a fixed file-scope device array instead.
//
// Contract:
//  * The scratch is kNoAllocScratchBytes (32 MiB) in a static __device__ array.
//    Every GPU on which this part of the library is loaded holds it until the
//    process exits.
//  * The scratch must hold n_tiles padded tile runs of 9 * ld FP64 values (ld = n_nz
//    rounded up to 8); larger requests fail with EINVAL and a message naming the
//    limit.  No cudaMalloc, cudaFree or allocating library
//    routine is called.
//  * The device address of the array is looked up once per device with
//    cudaGetSymbolAddress, during the first call made while that device is
//    current; that first call should come before any stream capture is begun.
//  * All calls share the one array and it keeps the last call's contents.  Every
//    value a call reads from it was written earlier by the same call (the
//    contraction kernel writes every value of the n_nz blocks of each tile and the
//    copy reads only those), so nothing needs clearing.  Calls whose work overlaps on
//    the GPU (different streams, or different host threads) race on the array and
//    must be serialised by the caller.
#include <mutex>

#include "common.h"

namespace msasm {

msasm_status contract_simt_f64(const double* d_coef, const double* d_T, int64_t n_tiles, int n_nz, int K,
                               int ld_nz, double* d_nz, cudaStream_t stream);

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
constexpr size_t kNoAllocScratchDoubles = kNoAllocScratchBytes / sizeof(double);

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
static double* g_scratch_addr[kMaxDevices] = {};
static std::mutex g_scratch_mutex;

// Device address of the scratch array on the current device (looked up once per device).
static msasm_status scratch_address(double** out) {
  int dev = 0;
  MSASM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(MSASM_EUNSUPPORTED, "device ordinal above 63");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (err != cudaSuccess) return cuda_fail(err, "cudaGetSymbolAddress(no-alloc scratch)");
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return MSASM_OK;
}

}  // namespace msasm

using namespace msasm;

extern "C" msasm_status msasm_contract_noalloc(const msasm_tables* tab, const double* d_coef, int64_t n_tiles,
                                               double* d_nz, void* stream) {
  if (!tab || !d_coef || !d_nz) return fail(MSASM_EINVAL, "tables, d_coef or d_nz is NULL");
  if (n_tiles <= 0) return fail(MSASM_EINVAL, "n_tiles must be positive");
  const int n_nz = tab->n_nz, K = 9 * tab->n_pi, ld = (n_nz + 7) & ~7;
  // compare tile counts first, so that no product can wrap around for a huge n_tiles
  const int64_t max_tiles = int64_t(kNoAllocScratchDoubles / (size_t(9) * size_t(ld)));
  if (n_tiles > max_tiles) {
    return fail(MSASM_EINVAL, "msasm_contract_noalloc: " + std::to_string(n_tiles) + " tiles need more than the " +
                                  std::to_string(kNoAllocScratchBytes) + " bytes of the fixed scratch (at most " +
                                  std::to_string(max_tiles) + " tiles of this table per call)");
  }
  double* scratch = nullptr;
  MSASM_TRY(scratch_address(&scratch));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MSASM_TRY(contract_simt_f64(d_coef, tab->d_T, n_tiles, n_nz, K, ld, scratch, s));
  MSASM_CUDA(cudaMemcpy2DAsync(d_nz, size_t(9) * n_nz * sizeof(double), scratch, size_t(9) * ld * sizeof(double),
                               size_t(9) * n_nz * sizeof(double), size_t(n_tiles), cudaMemcpyDeviceToDevice, s));
  return MSASM_OK;
}
