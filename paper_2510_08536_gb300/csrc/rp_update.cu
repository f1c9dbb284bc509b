// Value update (Sec. 3, update procedure): the continuous buffer, ordered by
// rank and LDU order, is reordered into the row-major device matrix by the
// permutation P (src_of). The sparsity is never rebuilt. When the iteration
// runs on the sliced layout, a second gather refills its values from the
// CSR values (k_slice_vals: 4 + 8 bytes read, 8 + 4 written per padded entry).
//
// Roofline: HBM bound. Per stored entry one 4-byte index read, one 8-byte
// gathered read and one 8-byte write (+4 bytes for the FP32 copy); the
// gather is nearly sequential (a handful of monotone streams per rank), so
// it moves close to the algorithmic bytes.
#include "rp_common.cuh"

namespace rp {

// buffer value at slot s (bounds-checked build: slots outside [0, len) read 0)
__device__ __forceinline__ double slot_value(const double* __restrict__ buf, int32_t s, int64_t len) {
  return RP_IN(s, 0, len, kChkPermute) ? __ldg(buf + s) : 0.0;
}

template <bool FP32>
__global__ void __launch_bounds__(kThreads)
    k_permute(const double* __restrict__ buf, const int32_t* __restrict__ src_of, double* __restrict__ vals,
              float* __restrict__ vals32, int64_t nnz, int64_t buf_len) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool vec = ((reinterpret_cast<uintptr_t>(src_of) | reinterpret_cast<uintptr_t>(vals)) & 15) == 0 &&
                   (!FP32 || (reinterpret_cast<uintptr_t>(vals32) & 15) == 0);
  int64_t done = 0;
  if (vec) {
    const int64_t nv = nnz >> 2;
    const int4* s4 = reinterpret_cast<const int4*>(src_of);
    double2* v2 = reinterpret_cast<double2*>(vals);
    float4* f4 = reinterpret_cast<float4*>(vals32);
    for (int64_t i = tid; i < nv; i += stride) {
      int4 s = __ldcs(s4 + i);
      double a = slot_value(buf, s.x, buf_len), b = slot_value(buf, s.y, buf_len), c = slot_value(buf, s.z, buf_len),
             d = slot_value(buf, s.w, buf_len);
      __stcs(v2 + 2 * i, make_double2(a, b));
      __stcs(v2 + 2 * i + 1, make_double2(c, d));
      if (FP32) __stcs(f4 + i, make_float4((float)a, (float)b, (float)c, (float)d));
    }
    done = nv << 2;
  }
  for (int64_t i = done + tid; i < nnz; i += stride) {
    double a = slot_value(buf, src_of[i], buf_len);
    vals[i] = a;
    if (FP32) vals32[i] = (float)a;
  }
}

// Jacobi diagonal straight from the diagonal block of each rank (contiguous
// in the buffer): dinv[i] = 1 / a_ii, and 1/(float)a_ii for the FP32 copy.
template <bool FP32>
__global__ void __launch_bounds__(kThreads)
    k_dinv(const double* __restrict__ buf, const int64_t* __restrict__ row_off,
           const int64_t* __restrict__ slot_off, int k, int64_t n, double* __restrict__ dinv,
           float* __restrict__ dinv32) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int r = find_rank(row_off, k, i);
    double d = __ldg(buf + slot_off[r] + (i - row_off[r]));
    dinv[i] = 1.0 / d;
    if (FP32) dinv32[i] = 1.0f / (float)d;
  }
}

static rp_status permute_all(rp_handle* h, const double* buf, cudaStream_t s) {
  for (int p = 0; p < h->n_parts; ++p) {
    const double* base = buf + h->part_buf_off[p];
    const int64_t blen = h->part_buf_off[p + 1] - h->part_buf_off[p];
    int64_t o = h->part_nnz_off[p], cnt = h->part_nnz_off[p + 1] - o;
    int g = grid_for(h, (cnt + 3) / 4);
    if (cnt > 0) {
      if (h->want_fp32)
        k_permute<true><<<g, kThreads, 0, s>>>(base, h->src_of + o, h->vals + o, h->vals32 + o, cnt, blen);
      else
        k_permute<false><<<g, kThreads, 0, s>>>(base, h->src_of + o, h->vals + o, nullptr, cnt, blen);
    }
    int64_t no = h->part_nl_off[p], ncnt = h->part_nl_off[p + 1] - no;
    if (ncnt > 0) {
      if (h->want_fp32)
        k_permute<true><<<grid_for(h, (ncnt + 3) / 4), kThreads, 0, s>>>(base, h->nl_src_of + no, h->nl_vals + no,
                                                                         h->nl_vals32 + no, ncnt, blen);
      else
        k_permute<false><<<grid_for(h, (ncnt + 3) / 4), kThreads, 0, s>>>(base, h->nl_src_of + no,
                                                                          h->nl_vals + no, nullptr, ncnt, blen);
    }
  }
  if (h->n > 0) {
    if (h->want_fp32)
      k_dinv<true><<<grid_for(h, h->n), kThreads, 0, s>>>(buf, h->d_row_off, h->d_slot_off, h->k, h->n, h->dinv,
                                                          h->dinv32);
    else
      k_dinv<false><<<grid_for(h, h->n), kThreads, 0, s>>>(buf, h->d_row_off, h->d_slot_off, h->k, h->n, h->dinv,
                                                           nullptr);
  }
  RP_TRY_CUDA(cudaGetLastError());
  RP_TRY(line_factors(h, s));
  return fill_sliced(h, s);
}

// Buffers, copy stream and events of RP_MEM_HOST_ASYNC, made on first use.
static rp_status ensure_async_stage(rp_handle* h) {
  if (h->copy_stream) return RP_OK;
  for (int i = 0; i < 2; ++i) {
    cudaError_t e = cudaMalloc((void**)&h->stage_async[i], sizeof(double) * (size_t)(h->n_slots > 0 ? h->n_slots : 1));
    if (e != cudaSuccess) {
      cudaGetLastError();
      h->stage_async[i] = nullptr;
      free_async_stage(h);
      return fail(RP_ENOMEM, "cudaMalloc of the asynchronous staging buffers failed");
    }
    RP_TRY_CUDA(cudaEventCreateWithFlags(&h->stage_copied[i], cudaEventDisableTiming));
    RP_TRY_CUDA(cudaEventCreateWithFlags(&h->stage_consumed[i], cudaEventDisableTiming));
  }
  RP_TRY_CUDA(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
  h->stage_next = 0;
  return RP_OK;
}

void free_async_stage(rp_handle* h) {
  for (int i = 0; i < 2; ++i) {
    if (h->stage_async[i]) cudaFree(h->stage_async[i]);
    if (h->stage_copied[i]) cudaEventDestroy(h->stage_copied[i]);
    if (h->stage_consumed[i]) cudaEventDestroy(h->stage_consumed[i]);
    h->stage_async[i] = nullptr;
    h->stage_copied[i] = h->stage_consumed[i] = nullptr;
  }
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  h->copy_stream = nullptr;
}

// Upload on the copy stream into the staging buffer whose last permutation has
// finished, then permute from it on `s` once the upload has landed. The copy
// does not wait for earlier work on `s`: it overlaps a solve still running.
static rp_status update_host_async(rp_handle* h, const double* buffer, cudaStream_t s) {
  RP_TRY(ensure_async_stage(h));
  const int i = h->stage_next;
  h->stage_next ^= 1;
  RP_TRY_CUDA(cudaStreamWaitEvent(h->copy_stream, h->stage_consumed[i], 0));
  if (h->n_slots > 0)
    RP_TRY_CUDA(cudaMemcpyAsync(h->stage_async[i], buffer, sizeof(double) * h->n_slots, cudaMemcpyHostToDevice,
                                h->copy_stream));
  RP_TRY_CUDA(cudaEventRecord(h->stage_copied[i], h->copy_stream));
  RP_TRY_CUDA(cudaStreamWaitEvent(s, h->stage_copied[i], 0));
  RP_TRY(permute_all(h, h->stage_async[i], s));
  RP_TRY_CUDA(cudaEventRecord(h->stage_consumed[i], s));
  return RP_OK;
}

}  // namespace rp

using namespace rp;

namespace rp {
RP_CHECK_TU(update)
}

// Can the current device read this host pointer in place?
static rp_status check_host_direct(const void* p) {
  cudaPointerAttributes attr{};
  cudaError_t e = cudaPointerGetAttributes(&attr, p);
  if (e != cudaSuccess) cudaGetLastError();
  if (e == cudaSuccess && (attr.type == cudaMemoryTypeHost || attr.type == cudaMemoryTypeManaged ||
                           attr.type == cudaMemoryTypeDevice))
    return RP_OK;
  int dev = 0, pageable = 0;
  RP_TRY_CUDA(cudaGetDevice(&dev));
  RP_TRY_CUDA(cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev));
  if (!pageable)
    return fail(RP_EUNSUPPORTED, "RP_MEM_HOST_DIRECT needs pinned host memory on a device without pageable-memory access");
  return RP_OK;
}

extern "C" rp_status rp_update_values_packed(rp_handle* h, const double* buffer, int32_t where, void* stream) {
  if (!h || (!buffer && h->n_slots > 0)) return fail(RP_EINVAL, "null argument");
  if (where != RP_MEM_DEVICE && where != RP_MEM_HOST && where != RP_MEM_HOST_DIRECT && where != RP_MEM_HOST_ASYNC)
    return fail(RP_EINVAL, "where must be RP_MEM_DEVICE, RP_MEM_HOST, RP_MEM_HOST_DIRECT or RP_MEM_HOST_ASYNC");
  cudaStream_t s = (cudaStream_t)stream;
  if (where == RP_MEM_HOST_ASYNC) return update_host_async(h, buffer, s);
  const double* src = buffer;
  if (where == RP_MEM_HOST_DIRECT && h->n_slots > 0) RP_TRY(check_host_direct(buffer));
  if (where == RP_MEM_HOST) {
    if (h->n_slots > 0)
      RP_TRY_CUDA(cudaMemcpyAsync(h->staging, buffer, sizeof(double) * h->n_slots, cudaMemcpyHostToDevice, s));
    src = h->staging;
  }
  return permute_all(h, src, s);
}

extern "C" rp_status rp_update_values(rp_handle* h, const double* const* diag, const double* const* upper,
                                      const double* const* lower, const double* const* iface, int32_t where,
                                      void* stream) {
  if (!h || !diag || !upper || !iface || (!h->symmetric && !lower)) return fail(RP_EINVAL, "null argument");
  if (where != RP_MEM_DEVICE && where != RP_MEM_HOST) return fail(RP_EINVAL, "where must be RP_MEM_DEVICE or RP_MEM_HOST");
  cudaStream_t s = (cudaStream_t)stream;
  const cudaMemcpyKind kind = where == RP_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  for (int r = 0; r < h->k; ++r) {
    const int64_t n = h->n_cells[r], F = h->n_faces[r], E = h->n_iface[r];
    double* dst = h->staging + h->slot_off[r];
    if ((n && !diag[r]) || (F && !upper[r]) || (F && !h->symmetric && !lower[r]) || (E && !iface[r]))
      return fail(RP_EINVAL, "rank %d: null coefficient array", r);
    if (n) RP_TRY_CUDA(cudaMemcpyAsync(dst, diag[r], 8 * n, kind, s));
    if (F) RP_TRY_CUDA(cudaMemcpyAsync(dst + n, upper[r], 8 * F, kind, s));
    int64_t at = n + F;
    if (!h->symmetric) {
      if (F) RP_TRY_CUDA(cudaMemcpyAsync(dst + at, lower[r], 8 * F, kind, s));
      at += F;
    }
    if (E) RP_TRY_CUDA(cudaMemcpyAsync(dst + at, iface[r], 8 * E, kind, s));
  }
  return permute_all(h, h->staging, s);
}

extern "C" rp_status rp_get_values(const rp_handle* h, const double** vals, const float** vals32,
                                   const double** dinv) {
  if (!h) return fail(RP_EINVAL, "null handle");
  if (vals) *vals = h->vals;
  if (vals32) *vals32 = h->vals32;
  if (dinv) *dinv = h->dinv;
  return RP_OK;
}
