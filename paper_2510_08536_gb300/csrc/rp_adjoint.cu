// Adjoint solve and gradients of the merged system.
//
// With A x = b and a loss L(x), the adjoint lambda solves A^T lambda = dL/dx;
// then dL/db = lambda and dL/da_ij = -lambda_i x_j for every stored entry.
// A^T reuses A's pattern: valsT[p] = vals[tpos[p]] (one gather pass), and the
// Jacobi diagonal is unchanged by transposition; the sliced layout of A then
// serves A^T with its values gathered from valsT. Symmetric storage needs no
// transpose at all.
#include "rp_common.cuh"

namespace rp {

rp_status solve_common(rp_handle* h, int mode, const double* vals, const double* dinv, cudaGraphExec_t* slot,
                        const double* b, double* x, double tol, int32_t x_is_guess, int32_t where,
                        rp_solve_info* info, cudaStream_t s);

__global__ void __launch_bounds__(kThreads)
    k_transpose_vals(int64_t nnz, const int32_t* __restrict__ tpos, const double* __restrict__ vals,
                     double* __restrict__ valsT) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t t = __ldg(tpos + p);
    valsT[p] = RP_IN(t, 0, nnz, kChkTranspose) ? __ldg(vals + t) : 0.0;
  }
}

// per stored entry (i, j): -lambda_i x_j, accumulated into the entry's slot
template <bool SHARED_SLOTS>
__global__ void __launch_bounds__(kThreads)
    k_entry_grad(int64_t n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                 const int32_t* __restrict__ src_of, const double* __restrict__ lam, const double* __restrict__ x,
                 double* __restrict__ g, int64_t n_slots) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double li = lam[i];
    for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
      if (!RP_IN(col[p], 0, n, kChkGather) || !RP_IN(src_of[p], 0, n_slots, kChkPermute)) continue;
      const double v = -li * __ldg(x + col[p]);
      if (SHARED_SLOTS) atomicAdd(g + src_of[p], v);  // two addends per shared slot: order-free
      else g[src_of[p]] = v;
    }
  }
}

// -(lambda_l - lambda_u)(x_l - x_u) per face, then per interface entry, rank by rank
__global__ void __launch_bounds__(kThreads)
    k_face_grad(int k, int64_t total, const int64_t* __restrict__ out_off, const int64_t* __restrict__ row_off,
                const int64_t* __restrict__ face_off, const int64_t* __restrict__ iface_off,
                const int32_t* __restrict__ lower, const int32_t* __restrict__ upper,
                const int32_t* __restrict__ iface_row, const int32_t* __restrict__ iface_gcol,
                const double* __restrict__ lam, const double* __restrict__ x, double* __restrict__ g) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int r = find_rank(out_off, k, t);
    int64_t u = t - out_off[r];
    int64_t F = face_off[r + 1] - face_off[r];
    int64_t a, b;
    if (u < F) {
      a = row_off[r] + lower[face_off[r] + u];
      b = row_off[r] + upper[face_off[r] + u];
    } else {
      int64_t e = iface_off[r] + (u - F);
      a = row_off[r] + iface_row[e];
      b = iface_gcol[e];
    }
    if (!RP_IN(a, 0, row_off[k], kChkGather) || !RP_IN(b, 0, row_off[k], kChkGather)) continue;
    g[t] = -(lam[a] - lam[b]) * (x[a] - x[b]);
  }
}

RP_CHECK_TU(adjoint)

}  // namespace rp

using namespace rp;

extern "C" rp_status rp_solve_adjoint(rp_handle* h, const double* g, double* lambda, double tol,
                                      rp_solve_info* info, void* stream) {
  if (!h || (!g && h->n) || (!lambda && h->n)) return fail(RP_EINVAL, "null argument");
  if (!(tol >= 0.0)) return fail(RP_EINVAL, "tol must be >= 0");
  if (h->n_parts != 1) return fail(RP_EUNSUPPORTED, "adjoint solve needs n_parts == 1");
  if (h->n == 0) {
    if (info) *info = rp_solve_info{RP_OK, 0, 0, 0, 0, 0.0};
    return RP_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (h->symmetric)
    return solve_common(h, false, h->vals, h->dinv, &h->graphs.fp64, g, lambda, tol, 0, RP_MEM_DEVICE, info, s);
  if (!h->tpos) return fail(RP_EINVAL, "adjoint of general storage needs want_transpose");
  if (!h->valsT) {
    cudaError_t e = cudaMalloc((void**)&h->valsT, sizeof(double) * (h->nnz + 64));
    if (e != cudaSuccess) {
      h->valsT = nullptr;
      cudaGetLastError();
      return fail(RP_ENOMEM, "cudaMalloc of transposed values failed");
    }
  }
  k_transpose_vals<<<grid_for(h, h->nnz), kThreads, 0, s>>>(h->nnz, h->tpos, h->vals, h->valsT);
  RP_TRY_CUDA(cudaGetLastError());
  RP_TRY(fill_sliced_transposed(h, s));  // the iteration multiplies with the sliced layout of A^T
  return solve_common(h, false, h->valsT, h->dinv, &h->graphs.adjoint, g, lambda, tol, 0, RP_MEM_DEVICE, info, s);
}

extern "C" rp_status rp_entry_grad(rp_handle* h, const double* lambda, const double* x, double* g_buffer,
                                   void* stream) {
  if (!h || (!lambda && h->n) || (!x && h->n) || (!g_buffer && h->n_slots)) return fail(RP_EINVAL, "null argument");
  if (h->n_parts != 1) return fail(RP_EUNSUPPORTED, "entry gradients need n_parts == 1");
  if (h->n == 0) return RP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (h->symmetric) {
    RP_TRY_CUDA(cudaMemsetAsync(g_buffer, 0, sizeof(double) * h->n_slots, s));
    k_entry_grad<true><<<h->grid, kThreads, 0, s>>>(h->n, h->row_ptr, h->col_idx, h->src_of, lambda, x, g_buffer,
                                                     h->n_slots);
  } else {
    k_entry_grad<false><<<h->grid, kThreads, 0, s>>>(h->n, h->row_ptr, h->col_idx, h->src_of, lambda, x, g_buffer,
                                                      h->n_slots);
  }
  RP_TRY_CUDA(cudaGetLastError());
  return RP_OK;
}

extern "C" rp_status rp_face_grad(rp_handle* h, const double* lambda, const double* x, double* g_face,
                                  void* stream) {
  if (!h || (!lambda && h->n) || (!x && h->n) || (!g_face && h->n_face_out)) return fail(RP_EINVAL, "null argument");
  if (h->n_face_out == 0) return RP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  static_assert(sizeof(int64_t) == 8, "");
  // per-rank output offsets F_r + E_r, kept on the device after the first call
  if (!h->d_out_off) {
    std::vector<int64_t> off(h->k + 1, 0);
    for (int r = 0; r < h->k; ++r) off[r + 1] = off[r] + h->n_faces[r] + h->n_iface[r];
    cudaError_t e = cudaMalloc((void**)&h->d_out_off, sizeof(int64_t) * (h->k + 1));
    if (e != cudaSuccess) {
      h->d_out_off = nullptr;
      cudaGetLastError();
      return fail(RP_ENOMEM, "cudaMalloc failed");
    }
    RP_TRY_CUDA(cudaMemcpy(h->d_out_off, off.data(), sizeof(int64_t) * (h->k + 1), cudaMemcpyHostToDevice));
  }
  k_face_grad<<<grid_for(h, h->n_face_out), kThreads, 0, s>>>(h->k, h->n_face_out, h->d_out_off, h->d_row_off,
                                                               h->d_face_off, h->d_iface_off, h->d_lower, h->d_upper,
                                                               h->d_iface_row, h->d_iface_gcol, lambda, x, g_face);
  RP_TRY_CUDA(cudaGetLastError());
  return RP_OK;
}
