// rp_spmv_noalloc: y = A x and x.y for callers that cannot allocate device
// memory. Same arithmetic per row as rp_spmv; the reduction scratch (one
// partial sum per block and the last-block ticket) lives in a file-scope
// static device array instead of handle-owned memory.
//
// The array is g_noalloc_scratch below: 256 bytes for the ticket, then
// kNaMaxBlocks doubles (64 KiB). Every GPU that loads the library holds it
// until the process exits. Each block covers kNaRowsPerBlock rows, so one
// call accepts at most kNaMaxBlocks * kNaRowsPerBlock = 16,777,216 rows.
#include <mutex>

#include "rp_common.cuh"

namespace rp {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaRowsPerThread = 8;
constexpr int64_t kNaRowsPerBlock = (int64_t)kNaThreads * kNaRowsPerThread;  // 2048
constexpr int kNaMaxBlocks = 8192;
constexpr size_t kNaTicketBytes = 256;
constexpr size_t kNaScratchBytes = kNaTicketBytes + sizeof(double) * kNaMaxBlocks;
constexpr int kNaMaxDevices = 64;

// Shared by every call on a device; keeps the previous call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

// Device address of g_noalloc_scratch per device (host code must not use the
// symbol itself: on the host it is only a stand-in, not a device address).
void* g_scratch_addr[kNaMaxDevices] = {};
std::mutex g_scratch_mu;

__global__ void __launch_bounds__(kNaThreads)
    k_spmv_noalloc(int64_t n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                   const double* __restrict__ vals, const double* __restrict__ x, double* __restrict__ y,
                   double* xy, unsigned char* scratch) {
  const int64_t base = (int64_t)blockIdx.x * kNaRowsPerBlock;
  double acc = 0.0;
#pragma unroll 1
  for (int k = 0; k < kNaRowsPerThread; ++k) {
    const int64_t i = base + (int64_t)k * kNaThreads + threadIdx.x;
    if (i < n) {
      const int s = __ldg(row_ptr + i), e = __ldg(row_ptr + i + 1);
      double sum = 0.0;
      for (int j = s; j < e; ++j) {
        const int c = __ldg(col + j);
        if (RP_IN(c, 0, n, kChkGather)) sum = fma(__ldg(vals + j), __ldg(x + c), sum);
      }
      y[i] = sum;
      acc += x[i] * sum;
    }
  }
  if (xy == nullptr) return;
  unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch);
  double* partials = reinterpret_cast<double*>(scratch + kNaTicketBytes);
  double v[1] = {acc}, tot[1];
  if (reduce_last_block<1>(v, partials, ticket, tot) && threadIdx.x == 0) *xy = tot[0];
}

// Once per device, with that device current: look up the array's device address.
rp_status scratch_for_current_device(unsigned char** out) {
  int dev = -1;
  RP_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNaMaxDevices) return fail(RP_EUNSUPPORTED, "device ordinal %d above %d", dev, kNaMaxDevices);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(RP_ECUDA, "cudaGetSymbolAddress of the static scratch failed on device %d: %s", dev,
                  cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return RP_OK;
}

}  // namespace

RP_CHECK_TU(noalloc)

}  // namespace rp

using namespace rp;

extern "C" rp_status rp_spmv_noalloc(int64_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* vals,
                                     const double* x, double* y, double* xy, void* stream) {
  if (n < 0) return fail(RP_EINVAL, "n must be >= 0");
  if (n > (int64_t)kNaMaxBlocks * kNaRowsPerBlock)
    return fail(RP_ERANGE, "rp_spmv_noalloc: n = %lld rows exceeds the static scratch limit of %lld rows",
                (long long)n, (long long)kNaMaxBlocks * kNaRowsPerBlock);
  if (n > 0 && (!row_ptr || !col_idx || !vals || !x || !y)) return fail(RP_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* scratch = nullptr;
  RP_TRY(scratch_for_current_device(&scratch));
  if (n == 0) {
    if (xy) RP_TRY_CUDA(cudaMemsetAsync(xy, 0, sizeof(double), s));
    return RP_OK;
  }
  const unsigned blocks = (unsigned)((n + kNaRowsPerBlock - 1) / kNaRowsPerBlock);
  // the ticket must start at zero; the partial sums are written before they are read
  if (xy) RP_TRY_CUDA(cudaMemsetAsync(scratch, 0, sizeof(unsigned int), s));
  k_spmv_noalloc<<<blocks, kNaThreads, 0, s>>>(n, row_ptr, col_idx, vals, x, y, xy, scratch);
  RP_TRY_CUDA(cudaGetLastError());
  return RP_OK;
}
