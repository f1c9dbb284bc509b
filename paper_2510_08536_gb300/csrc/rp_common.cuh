// Internal declarations shared by the translation units of librepart.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/repart.h"

namespace rp {

// ---------------------------------------------------------------- errors

void set_error(const char* fmt, ...);
rp_status fail(rp_status s, const char* fmt, ...);

#define RP_TRY_CUDA(call)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return ::rp::fail(RP_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                               \
  } while (0)

#define RP_TRY(call)                 \
  do {                               \
    rp_status s_ = (call);           \
    if (s_ != RP_OK) return s_;      \
  } while (0)

// ---------------------------------------------------------------- bounds-checked build
//
// Compiled with -DRP_CHECK (librepart_check.so, next to the library), device
// code range-checks every gather index and every offset it derives from the
// map or the sliced layout before using it. An index outside its array skips
// the access (a load reads zero, a store or copy is dropped) and is counted in
// a device error word, with the site and index of the first one; nothing
// traps, and rp_check_violations() reads the words. The normal build compiles
// every check to nothing.
enum : int {
  kChkPermute = 1,  // buffer slot src_of[p] of the value update
  kChkSliceValues,  // CSR position pos[q] of a padded sliced entry
  kChkSliceDesc,    // a slice descriptor (x_s, y_s) and its row length
  kChkSliceCopy,    // the source range of a staged copy
  kChkSliceIndex,   // an offset index against its table's length
  kChkGather,       // a gathered vector row (row + offset, or a CSR column)
  kChkNonlocal,     // a non-local column or its halo row
  kChkTranspose,    // a transpose position tpos[p]
  kChkMap,          // a position written by the map build
  kChkRowRange,     // a row pointer range
};

struct CheckWord {
  unsigned long long count;  // accesses skipped
  long long index, limit;    // the first one: its index and the end of its range
  int site, pad;
};

#ifdef RP_CHECK
// one error word per translation unit (no relocatable device code): each
// unit's reader is registered in rp_check_violations
static __device__ CheckWord g_check;

static __device__ __noinline__ bool check_fail(long long i, long long hi, int site) {
  if (atomicAdd(&g_check.count, 1ull) == 0ull) {
    g_check.index = i;
    g_check.limit = hi;
    g_check.site = site;
  }
  return false;
}
#define RP_IN(i, lo, hi, site)                                                        \
  (((long long)(i) >= (long long)(lo) && (long long)(i) < (long long)(hi))            \
       ? true                                                                          \
       : ::rp::check_fail((long long)(i), (long long)(hi), (site)))
// host reader of this unit's word (copies it out; reset: clears it)
#define RP_CHECK_TU(name)                                                              \
  rp_status check_read_##name(CheckWord* out, int reset) {                             \
    RP_TRY_CUDA(cudaMemcpyFromSymbol(out, g_check, sizeof(CheckWord)));                \
    if (reset) {                                                                       \
      const CheckWord z{};                                                             \
      RP_TRY_CUDA(cudaMemcpyToSymbol(g_check, &z, sizeof(CheckWord)));                 \
    }                                                                                  \
    return RP_OK;                                                                      \
  }
#else
#define RP_IN(i, lo, hi, site) true
#define RP_CHECK_TU(name)
#endif
// a helper's "no index" answer (-1) is only possible in the bounds-checked build
#ifdef RP_CHECK
#define RP_IDX_OK(g) ((g) >= 0)
#else
#define RP_IDX_OK(g) true
#endif

// ---------------------------------------------------------------- constants

constexpr int kThreads = 256;        // block size of the streaming kernels
constexpr int kBlocksPerSm = 8;      // 8 x 256 threads = full residency on sm_103
constexpr int kMaxPartials = 8;      // doubles reduced per block at most

// ---------------------------------------------------------------- solver control

// Device-resident scalars of one PCG / refinement run. All values are
// written by the last block of a kernel and read by later kernels: no host
// round trip inside the iteration.
struct Ctl {
  double bb;            // ||b||^2
  double thresh;        // tol^2 ||b||^2
  double rz;            // (r, z) of the current iterate
  double rr;            // (r, r): recursive in the loop, true after a residual pass
  double pq;            // (p, A p)
  double alpha, beta;
  double inner_thresh;  // mixed: inner_tol^2 ||fl32(r)||^2
  double tol, inner_tol;
  int32_t iter;         // iterations of the current inner run
  int32_t iter_total;   // all inner iterations of the solve
  int32_t max_iter;     // cap: total (FP64) or per inner run (mixed)
  int32_t stop;         // inner loop exit requested
  int32_t skip_x;       // this iteration broke down before its x update
  int32_t status;       // -1 running, then RP_OK / RP_NOT_CONVERGED / RP_BREAKDOWN
  int32_t pass;         // residual passes done
  int32_t restarts;
  int32_t max_restarts;
  int32_t outer;        // refinement steps started (mixed)
  int32_t max_outer;
  int32_t x_zero;       // first pass starts from x = 0
  int32_t skip_correct; // mixed: no correction to add this pass
  unsigned int ticket;  // last-block election counter (reset by the last block)
  int32_t ru_apply;     // continued refinement: p = z + beta_ru p before the next run
  double beta_ru;
  double ru_delta;      // continued refinement: residual reduction per refinement
};

// Pointers that change between calls (user buffers); the captured graphs
// read them from device memory so they never need re-instantiation.
struct SolveIO {
  const double* b;
  double* x;
};

struct Graphs {
  cudaGraphExec_t fp64 = nullptr;
  cudaGraphExec_t mixed = nullptr;
  cudaGraphExec_t mixed_ru = nullptr;
  cudaGraphExec_t adjoint = nullptr;
};

// The matrix split into GPU parts (Sec. 3): per part a local CSR over the
// part's own rows and columns and a non-local CSR whose compressed columns
// map to global rows through nl_cols (the halo). n == 1: merged matrix, the
// other fields are unused.
template <typename T>
struct Parts {
  int32_t n;
  const int64_t* row_off;    // [n+1] first global row of each part
  const int64_t* nnz_off;    // [n+1] local entries
  const int64_t* nl_off;     // [n+1] non-local entries
  const int64_t* nlcol_off;  // [n+1] compressed non-local columns
  const int32_t* nl_row_ptr; // per-part segments (row_off[p] + p)
  const int32_t* nl_col;     // compressed column of each non-local entry
  const int32_t* nl_cols;    // global row behind each compressed column
  const T* nl_vals;
};

// Sliced layout of the merged matrix (one part): rows in slices of 32, one
// row per lane. Slice s keeps its values column-major at vals[x_s + 32 k +
// lane] (k < L_s, the longest row of the slice; shorter rows are padded with
// zeros) and, instead of column indices, per entry a 4- or 8-bit index into a
// table of the slice's distinct column offsets col - row. Distinct tables are
// stored once in tabs ([D, offset_0 .. offset_{D-1}] each, 32 spare words at
// the end); tinfo[s] = t_s | w4 << 31 names the slice's table (tabs[t_s - 1]
// = D_s) and its index width: w4 = 1 (D_s <= 16) packs 8 indices a word
// (entry 8 g + e in bits 4e..4e+3 of word g), else 4 (entry 4 g + e in byte
// e). The index words of lane j are at ibuf[y_s + 32 g + j]. desc[s] =
// (x_s, y_s), desc[n_slices] closes the last slice, so L_s = (x_{s+1} - x_s)
// / 32. Entries keep the CSR order of their row, so a row's products are
// summed exactly as over the CSR arrays.
constexpr int kSliceRows = 32;
constexpr int kSliceMaxDict = 256;   // 8-bit indices
constexpr int kSliceMaxWidth = 32;   // longest row the layout takes
constexpr uint32_t kSliceW4 = 0x80000000u;  // tinfo flag: 4-bit indices

template <typename T>
struct Sliced {
  int64_t n_slices;  // 0: not built (CSR only)
  const uint2* desc; // n_slices + 1 entries, then kSliceDescPad zero entries
  const uint32_t* tinfo;  // n_slices entries, then kSliceDescPad
  const int32_t* tabs;
  const int32_t* ibuf;
  const T* vals;
  int64_t spin;      // iteration limit of every shared-memory barrier wait
  // several parts: per slice (first global row, part << 6 | rows of the part in
  // it); the non-local entries of those rows follow in the part's CSR. nullptr:
  // one part, slice s holds rows 32 s ..
  const int2* srow = nullptr;
  int64_t n_entries = 0, ibuf_len = 0, tabs_len = 0;  // array lengths (bounds-checked build)
  int u4 = 0;  // every slice has 4-bit indices and rows of at most 8 entries (every chunk is staged)
};
constexpr int kSliceDescPad = 8;  // bulk copies of descriptor runs may read past the end
// Probe bound of the wait for a block's own bulk copies after another wait
// ran out: copies land within microseconds, so it is met unless the GPU
// itself stalls, and it keeps the drain bounded whatever spin_limit is.
constexpr int64_t kDrainProbes = int64_t(1) << 22;

// Grids of the three PCG iteration kernels of one precision: blocks that
// fit on the SMs at once (by each kernel's register use), capped by the rows.
struct IterGrid {
  int k1 = 1, k1s = 1, k2 = 1, k3 = 1;  // K1 on CSR, K1 on the sliced layout, K2, K3
  int k1sm = 1;                         // K1 on the sliced layout of several parts
  int k2l = 1, k3l = 1;                 // K2, K3 with the line preconditioner
  int k2s = 1, k3s = 1;                 // K2, K3 of the scaled inner system
};

struct BsState;  // BiCGStab work space and graph (rp_bicgstab.cu)

// Line (block-tridiagonal) preconditioner over 32-row blocks: per row the LU
// factors of its block's tridiagonal part, l = a_i / u_{i-1}, w = 1 / u_i,
// g = c_i / u_i (a, c: couplings to rows i-1, i+1 inside the block), and the
// buffer z that receives M^-1 r. l == nullptr: Jacobi.
template <typename T>
struct Line {
  const T* l;
  const T* w;
  const T* g;
  T* z;
};

// Per-call pointers of the batched solve (read by the captured kernel).
struct BatchIO {
  const double* buf;
  const double* b;
  double* x;
  double tol;
};

// Arguments of the persistent batched kernel (fixed per handle).
struct BatchArgs {
  int32_t n_sys;
  const int32_t* order;    // systems, largest first
  const int64_t* row_off;  // [n_sys+1] first merged row of each system
  const int64_t* nnz_off;  // [n_sys+1]
  const int64_t* buf_off;  // [n_sys+1]
  const int32_t* row_ptr;  // per-part segments (row_off[s] + s)
  const int32_t* col;
  const int32_t* src_of;
  double* vals;
  float* vals32;
  double* dinv;
  float* dinv32;
  double *r, *p, *q;
  float *r32, *p32, *q32, *d32;
  unsigned int* queue;
  rp_solve_info* info;  // [n_sys]
  const BatchIO* io;
  int32_t max_iter, max_restarts, max_outer;
  double inner_tol;
  double ru_delta;
  // sliced layout of every system (sl_desc null: the SpMV runs on CSR); the
  // kernel writes each system's sliced values from the buffer
  const int64_t* sl_soff;  // [n_sys+1] first slice of each system
  const uint2* sl_desc;
  const uint32_t* sl_tinfo;
  const int32_t* sl_tabs;
  const uint32_t* sl_ibuf;
  const int32_t* sl_pos;
  double* sl_vals;
  float* sl_vals32;
  int64_t sl_entries, sl_ibuf_len, sl_tabs_len;  // array lengths (bounds-checked build)
  // mixed forms on the sliced layout: the inner FP32 iteration runs on S A S,
  // s_i = 1/sqrt(a_ii) (FP64), written by the kernel's update
  double* s64;
};

}  // namespace rp

// ---------------------------------------------------------------- handle

struct rp_handle {
  int device = 0;
  int num_sms = 0;
  int32_t k = 0, n_parts = 0;
  int64_t n = 0;        // merged rows (all parts)
  int64_t nnz = 0;      // stored local entries (all parts)
  int64_t nl_nnz = 0;   // stored non-local entries (all parts)
  int64_t n_slots = 0;  // continuous buffer length
  int64_t n_face_out = 0;  // sum over ranks of F_r + E_r
  bool symmetric = false, want_fp32 = false, want_transpose = false;
  rp_options opts{};

  // per rank (host)
  std::vector<int64_t> row_off, slot_off, face_off, iface_off;
  std::vector<int32_t> n_cells, n_faces, n_iface;
  // per part (host)
  std::vector<int64_t> part_row_off, part_nnz_off, part_nl_off, part_buf_off, part_nlcol_off;

  // device map (per part segments, see rp_map_view)
  int32_t* row_ptr = nullptr;     // n + n_parts
  int32_t* col_idx = nullptr;     // nnz
  int32_t* src_of = nullptr;      // nnz
  int32_t* diag_pos = nullptr;    // n
  int32_t* tpos = nullptr;        // nnz (optional)
  int32_t* nl_row_ptr = nullptr;  // n + n_parts
  int32_t* nl_col_idx = nullptr;
  int32_t* nl_src_of = nullptr;
  int32_t* nl_cols = nullptr;
  // rank tables on the device (k + 1 entries)
  int64_t* d_row_off = nullptr;
  int64_t* d_slot_off = nullptr;
  int64_t* d_face_off = nullptr;
  int64_t* d_iface_off = nullptr;
  int32_t* d_lower = nullptr;  // concatenated addressing, kept for face gradients
  int32_t* d_upper = nullptr;
  int32_t* d_iface_row = nullptr;
  int32_t* d_iface_gcol = nullptr;  // global column of each interface entry
  int64_t* d_out_off = nullptr;     // per-rank offsets of the face-gradient output

  // values
  double* staging = nullptr;  // n_slots
  // RP_MEM_HOST_ASYNC uploads: two staging buffers that the handle's own copy
  // stream fills while earlier work runs; copied[i] is recorded when upload i
  // has landed, consumed[i] when the permutation that read buffer i is done
  double* stage_async[2] = {nullptr, nullptr};
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t stage_copied[2] = {nullptr, nullptr}, stage_consumed[2] = {nullptr, nullptr};
  int stage_next = 0;
  double* vals = nullptr;     // nnz (+pad)
  float* vals32 = nullptr;    // nnz (+pad)
  double* nl_vals = nullptr;
  float* nl_vals32 = nullptr;
  int64_t *d_part_row_off = nullptr, *d_part_nnz_off = nullptr;  // part tables on the device
  int64_t *d_part_nl_off = nullptr, *d_part_nlcol_off = nullptr;
  double* valsT = nullptr;    // transposed values (adjoint, on demand)
  double* dinv = nullptr;     // n
  float* dinv32 = nullptr;    // n
  double* dinvT = nullptr;

  // sliced layout (every part's rows cut into their own slices; built when
  // every slice fits; see Sliced)
  int64_t sl_slices = 0;     // 0: the iteration runs on the CSR arrays
  int64_t sl_entries = 0;    // padded entries (32 per slice and width unit)
  int64_t sl_ibuf_len = 0;   // index words
  int64_t sl_tabs_len = 0;   // int32 words of the distinct tables
  int sl_u4 = 0;             // every slice 4-bit with rows of at most 8 entries
  int64_t* sl_part_soff = nullptr;  // [n_parts + 1] first slice of each part (device)
  int2* sl_srow = nullptr;           // [sl_slices] first row, part << 6 | rows (n_parts > 1)
  uint2* sl_desc = nullptr;  // [sl_slices + 1]
  uint32_t* sl_tinfo = nullptr;  // [sl_slices]
  int32_t* sl_tabs = nullptr;
  int32_t* sl_ibuf = nullptr;
  int32_t* sl_pos = nullptr;  // CSR position of each padded entry, -1 = padding
  double* sl_vals = nullptr;
  double* sl_valsT = nullptr;  // sliced transposed values (adjoint of general storage, on demand)
  float* sl_vals32 = nullptr;
  // FP32 values of the symmetrically scaled matrix S A S (s_i = 1/sqrt(a_ii)),
  // the inner system of the mixed PCG solves (one part, Jacobi); allocated by
  // the first such solve, refilled by every value update afterwards
  float* sl_vals32s = nullptr;
  double* s64 = nullptr;  // n: s_i = 1/sqrt(a_ii)

  // solver work space
  double *r = nullptr, *p = nullptr, *q = nullptr;
  float *r32 = nullptr, *p32 = nullptr, *q32 = nullptr, *d32 = nullptr;
  double* b_host_stage = nullptr;  // device copies for host-side callers
  double* x_host_stage = nullptr;
  double* partials = nullptr;      // grid * kMaxPartials
  rp::Ctl* ctl = nullptr;          // device
  rp::Ctl* ctl_spmv = nullptr;     // device, rp_iter_spmv's own
  rp::SolveIO* io = nullptr;       // device
  unsigned int* ticket = nullptr;  // spare ticket for rp_spmv
  int grid = 0;                    // blocks of every streaming kernel
  rp::IterGrid igrid64, igrid32;   // blocks of the PCG iteration kernels
  rp::Graphs graphs;
  cudaStream_t capture_stream = nullptr;
  bool solve_ran = false;          // an rp_solve has filled the control block

  // line preconditioner (precond == RP_PRECOND_LINE)
  int precond = RP_PRECOND_JACOBI;
  double *ln_l = nullptr, *ln_w = nullptr, *ln_g = nullptr, *ln_z = nullptr;
  float *ln_l32 = nullptr, *ln_w32 = nullptr, *ln_g32 = nullptr, *ln_z32 = nullptr;

  // BiCGStab (non-symmetric systems), allocated on first use
  rp::BsState* bs = nullptr;

  // batched form (one system per part)
  bool batch_ready = false;
  int batch_cluster = 5, batch_threads = 512;  // autotuned by rp_batch_autotune
  int32_t* batch_order = nullptr;
  int64_t *batch_row_off = nullptr, *batch_nnz_off = nullptr, *batch_buf_off = nullptr;
  unsigned int* batch_queue = nullptr;
  rp_solve_info* batch_info = nullptr;
  rp::BatchIO* batch_io = nullptr;
  rp::BatchArgs batch_args{};
  double* batch_s64 = nullptr;  // s_i = 1/sqrt(a_ii) of the batched mixed forms
  cudaGraphExec_t batch_graphs[3] = {nullptr, nullptr, nullptr};
};

namespace rp {

// streaming-grid size for n rows
inline int grid_for(const rp_handle* h, int64_t n) {
  int64_t want = (n + kThreads - 1) / kThreads;
  int64_t cap = (int64_t)h->num_sms * kBlocksPerSm;
  if (want < 1) want = 1;
  return (int)(want < cap ? want : cap);
}

rp_status ensure_solver_buffers(rp_handle* h);
rp_status build_sliced(rp_handle* h, cudaStream_t s);  // after the CSR map
rp_status fill_sliced_transposed(rp_handle* h, cudaStream_t s);  // sl_valsT from valsT
rp_status fill_sliced(rp_handle* h, cudaStream_t s);   // after every value update
// the scaled inner system of the mixed PCG solves: allocated and filled from the
// current values on first use (then refilled by fill_sliced); false when the
// handle does not take it (several parts, CSR layout, no FP32 copy)
rp_status ensure_scaled(rp_handle* h, cudaStream_t s, bool* ok);
void free_sliced(rp_handle* h);
void free_async_stage(rp_handle* h);  // RP_MEM_HOST_ASYNC buffers, stream, events
void free_bicgstab(rp_handle* h);
void drop_bicgstab_graph(rp_handle* h);  // after a change of captured arguments
rp_status line_factors(rp_handle* h, cudaStream_t s);  // after every value update (precond LINE)
void free_line(rp_handle* h);
rp_status build_graphs(rp_handle* h);
void free_solver(rp_handle* h);
void free_batch(rp_handle* h);

}  // namespace rp

// ---------------------------------------------------------------- device helpers

namespace rp {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide partial sums of NV values, written to partials[blockIdx.x*NV+i];
// returns true in every thread of the one block that arrives last, with the
// grid totals in tot[] (summed in block order: deterministic for a fixed
// grid). The ticket is reset by that block.
template <int NV>
__device__ __forceinline__ bool reduce_last_block(double (&v)[NV], double* partials,
                                                  unsigned int* ticket, double (&tot)[NV]) {
  __shared__ double sm[NV][32];
  __shared__ int last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double s = warp_sum(v[i]);
    if (lane == 0) sm[i][wid] = s;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double s = lane < nw ? sm[i][lane] : 0.0;
      s = warp_sum(s);
      if (lane == 0) partials[(size_t)blockIdx.x * NV + i] = s;
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double s = 0.0;
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x)
      s += __ldcg(partials + (size_t)b * NV + i);
    s = warp_sum(s);
    __syncthreads();
    if (lane == 0) sm[i][wid] = s;
    __syncthreads();
    double t = lane < nw ? sm[i][lane] : 0.0;
    tot[i] = warp_sum(t);  // every warp computes the same total
  }
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// index of the rank owning position t in an offset table off[0..k]
__device__ __forceinline__ int find_rank(const int64_t* __restrict__ off, int k, int64_t t) {
  int lo = 0, hi = k;  // off[lo] <= t < off[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= t) lo = mid; else hi = mid;
  }
  return lo;
}

}  // namespace rp
