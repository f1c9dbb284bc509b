/*
 * repart.h -- C ABI of the GB300 repartitioning library (librepart.so).
 *
 * Method: matrix repartitioning of Olenik, Koch and Anzt, "Investigating
 * Matrix Repartitioning to Address the Over- and Undersubscription Challenge
 * for a GPU-based CFD Solver" (arXiv 2510.08536). Many CPU ranks each hold an
 * OpenFOAM LDU matrix (diagonal, upper and lower face coefficients over
 * owner/neighbour addressing, plus processor-interface coefficients). The
 * library fuses their sparsity into one device matrix per GPU part once
 * (Sec. 3, steps 1-3), updates the values in place every time step through a
 * permutation of one continuous buffer (Sec. 3, update procedure), and solves
 * the merged pressure system with Jacobi-preconditioned CG (the paper's
 * pressure solve is CG, Sec. 4).
 *
 * Conventions for every call:
 *   - Every call returns rp_status; no exception crosses the ABI. On failure
 *     rp_last_error() gives a message for the calling thread.
 *   - Host-side validation runs before any device work.
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). All device work is ordered on that stream; a call only blocks
 *     the host where its comment says so.
 *   - A handle owns all of its device memory and frees it in rp_destroy. The
 *     caller owns every pointer it passes; the library keeps none of them
 *     after the call returns.
 *   - A handle must not be used by two host threads, or on two streams whose
 *     work overlaps, at the same time.
 *   - Merged row order: the rows of a part are its CPU ranks' local rows,
 *     rank after rank (blockwise ownership, Sec. 3). Vectors b, x, lambda, g
 *     use this order.
 */
#ifndef REPART_H
#define REPART_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rp_status {
  RP_OK = 0,
  RP_EINVAL = 1,         /* malformed argument or descriptor                  */
  RP_EDUP = 2,           /* two stored coefficients share one (row, col)      */
  RP_ERANGE = 3,         /* an index is out of its range                      */
  RP_EOVERFLOW = 4,      /* a size does not fit the 32-bit index types        */
  RP_ENOMEM = 5,         /* device or host allocation failed                  */
  RP_ECUDA = 6,          /* a CUDA call failed                                */
  RP_NOT_CONVERGED = 7,  /* iteration limit reached before the tolerance      */
  RP_BREAKDOWN = 8,      /* p.Ap <= 0 (matrix not SPD) or a NaN appeared      */
  RP_DEVICE_TIMEOUT = 9, /* a bounded device wait ran out                     */
  RP_EUNSUPPORTED = 10   /* valid request this build does not serve           */
} rp_status;

/* Where a buffer lives. RP_MEM_HOST_DIRECT (value updates only): host memory
 * the GPU reads in place over the CPU-GPU link (pinned memory, or any host
 * memory on systems with pageable-memory access such as Grace), with no copy
 * into the staging buffer -- the analogue of sending the coefficients
 * straight into the device buffer (Sec. 3, update procedure).
 * RP_MEM_HOST_ASYNC (rp_update_values_packed only): host memory copied into
 * one of two device staging buffers on the handle's own copy stream. The
 * copy starts at the call -- it does not wait for work queued earlier on the
 * caller's stream, so it overlaps a solve still running there -- and the
 * permutation, queued on the caller's stream, waits for it; the next such
 * upload goes to the other buffer, once the permutation that last read it
 * is done. The caller keeps the host buffer unchanged until its stream has
 * passed the update (pinned memory makes the copy asynchronous). The
 * single-GPU analogue of sending the next time step's coefficients while the
 * GPU still solves (Sec. 3, update procedure; the GPU-aware communication of
 * Sec. 4). Allocates the two buffers, a stream and four events on first use. */
enum { RP_MEM_DEVICE = 0, RP_MEM_HOST = 1, RP_MEM_HOST_DIRECT = 2, RP_MEM_HOST_ASYNC = 3 };
/* Solve precision. RP_MIXED: FP64 iterative refinement around an FP32 PCG
 * that is restarted (p = z) at every refinement and solved to inner_tol
 * relative to its right-hand side, or to half the outer target tol ||b||
 * when that is reached first (the last refinement stops near the target).
 * RP_MIXED_RU: the same FP32 values, iterations and FP64 residual / update /
 * convergence test, but the FP32 PCG is not restarted: when its recursive
 * residual has fallen by ru_delta (or below half the outer target) its
 * iterate is added to x in FP64, the FP64 residual replaces the FP32 one and
 * the search direction continues (p = z + beta p). */
enum { RP_FP64 = 0, RP_MIXED = 1, RP_MIXED_RU = 2 };
/* Matrix layout of the PCG iteration (rp_options.layout). RP_LAYOUT_AUTO:
 * the sliced layout (see rp_get_sliced_view; every part, or every system of
 * a batched handle, in slices of its own) when no row has more than 32
 * entries and no 32-row slice more than 256 distinct column offsets; else
 * CSR. RP_LAYOUT_CSR: always CSR. Both give the same products row by row
 * (same entries, same order; with several parts the non-local entries of a
 * row follow its local ones, as in the CSR iteration). */
enum { RP_LAYOUT_AUTO = 0, RP_LAYOUT_CSR = 1 };
/* Preconditioner of the PCG solves (rp_options.precond). RP_PRECOND_JACOBI:
 * z = D^-1 r. RP_PRECOND_LINE: block-Jacobi over blocks of 32 consecutive
 * rows (blocks start at multiples of 32) with each block's tridiagonal part:
 * the diagonal and the couplings (i, i-1), (i, i+1) inside the block, solved
 * exactly (LU factors built at every value update). On a line-ordered mesh
 * (rows x-fastest, x-lines of 32 cells per rank) this is line-Jacobi along x.
 * Needs n_parts = 1; the adjoint solve and BiCGStab keep Jacobi. */
enum { RP_PRECOND_JACOBI = 0, RP_PRECOND_LINE = 1 };

typedef struct rp_handle rp_handle;

/* One CPU rank's LDU sparsity (Sec. 3, step 1: the pattern including the
 * coupling to non-local entries). Host pointers, caller-owned, read only
 * during rp_build_repartition.
 *   lower_addr[f] < upper_addr[f] < n_cells: face f couples owner l and
 *     neighbour u; upper[f] is entry (l, u), lower[f] is entry (u, l).
 *   Interface entry e: entry (iface_row[e], iface_nbr_col[e] of rank
 *     iface_nbr_rank[e]), with iface_nbr_rank[e] != this rank. Interfaces
 *     must be paired: rank q holds the transposed entry.                   */
typedef struct rp_ldu_desc {
  int32_t n_cells;
  int32_t n_faces;
  const int32_t* lower_addr;
  const int32_t* upper_addr;
  int32_t n_iface;
  const int32_t* iface_row;
  const int32_t* iface_nbr_rank;
  const int32_t* iface_nbr_col;
} rp_ldu_desc;

typedef struct rp_options {
  int32_t n_parts;        /* GPU parts n_GPU = k / alpha; must divide k (Sec. 3) */
  int32_t symmetric;      /* 1: ranks pass no lower[]; (u,l) reads upper[f]       */
  int32_t want_fp32;      /* keep an FP32 copy of the values (mixed solves)       */
  int32_t want_transpose; /* build tpos[] (transpose permutation, adjoint)        */
  int32_t max_iter;       /* PCG iteration cap (FP64; inner cap when mixed)       */
  int32_t max_outer;      /* refinement steps cap of the mixed solve              */
  int32_t max_restarts;   /* residual-replacement restarts allowed per solve      */
  int32_t device;         /* CUDA device ordinal (-1: current device)             */
  double inner_tol;       /* relative tolerance of the FP32 inner solve           */
  int64_t spin_limit;     /* probe limit of every device-side wait; a wait that
                             runs out ends the solve with RP_DEVICE_TIMEOUT after
                             its block's own copies have landed (0: every wait
                             gives up at once -- tests the timeout path)         */
  int32_t host_loop;      /* 1: rp_solve launches the same kernels from the host,
                             reading the control block after every iteration
                             (slow; for profilers that cannot look inside
                             graphs with conditional nodes)                       */
  int32_t layout;         /* RP_LAYOUT_AUTO or RP_LAYOUT_CSR                      */
  double ru_delta;        /* RP_MIXED_RU: residual reduction between two FP64
                             refinements (default 0.1; 0: use inner_tol)          */
  int32_t precond;        /* RP_PRECOND_JACOBI or RP_PRECOND_LINE                 */
  int32_t spare;          /* must be 0                                            */
} rp_options;

/* Replace the solver settings of a handle (max_iter, max_outer, max_restarts,
 * inner_tol, ru_delta, host_loop, precond, spin_limit); structural fields are ignored.
 * Takes effect at the next solve. Switching to RP_PRECOND_LINE builds its
 * factors from the current values (blocks the host); RP_EUNSUPPORTED for
 * n_parts > 1. */
rp_status rp_set_solver_options(rp_handle* h, const rp_options* opts);

/* Defaults: n_parts 1, general (non-symmetric) storage, FP32 copy on,
 * transpose off, max_iter 20000, max_outer 30, max_restarts 8, current
 * device, inner_tol 1e-5, spin_limit 1<<26, host_loop 0, layout
 * RP_LAYOUT_AUTO, ru_delta 0.1, precond RP_PRECOND_JACOBI. */
void rp_default_options(rp_options* opts);

/* Sec. 3 steps 1-3 and the three outputs (sparsity pattern, update pattern,
 * permutation P): validates the k descriptors on the host, uploads them,
 * and builds on the device, per part, the CSR pattern (columns ascending in
 * each row), src_of[p] (the buffer slot feeding CSR position p, i.e. P),
 * diag_pos, tpos (optional) and the non-local pattern for n_parts > 1.
 * Errors: RP_EINVAL (bad counts, null arrays, owner >= neighbour, self or
 * unpaired interface, n_parts not dividing k), RP_ERANGE (index outside its
 * rank), RP_EOVERFLOW (rows, entries or slots >= 2^31), RP_EDUP (repeated
 * (row, col)), RP_ENOMEM, RP_ECUDA. Blocks the host until done. */
rp_status rp_build_repartition(const rp_ldu_desc* ranks, int32_t k, const rp_options* opts,
                               rp_handle** out);

/* Device views of part `part`'s map, owned by the handle.
 * row_ptr[n_rows+1] counts from 0; col_idx is part-local; src_of indexes the
 * part's slice [buf_off, buf_off+buf_len) of the continuous buffer;
 * nl_cols[n_nl_cols] holds the global column of each compressed non-local
 * column. tpos is NULL unless want_transpose. */
typedef struct rp_map_view {
  int64_t n_rows, nnz, nl_nnz, n_nl_cols, row_off, buf_off, buf_len;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const int32_t* src_of;
  const int32_t* diag_pos;
  const int32_t* tpos;
  const int32_t* nl_row_ptr;
  const int32_t* nl_col_idx;
  const int32_t* nl_src_of;
  const int32_t* nl_cols;
} rp_map_view;
rp_status rp_get_part_map(const rp_handle* h, int32_t part, rp_map_view* out);

/* Total merged rows, stored local entries, buffer slots and parts. */
rp_status rp_get_sizes(const rp_handle* h, int64_t* n_rows, int64_t* nnz, int64_t* n_slots,
                       int32_t* n_parts);

/* Sec. 3, update procedure. `buffer` is the continuous coefficient buffer:
 * rank after rank, [diag n_r | upper F_r | lower F_r | iface E_r] (no lower
 * block in symmetric mode), n_slots doubles. where = RP_MEM_HOST copies it
 * into the handle's device staging buffer first (pinned memory makes that
 * copy asynchronous); RP_MEM_DEVICE reads it in place. Then one permutation
 * pass writes vals[p] = buffer[src_of[p]] (and the FP32 copy, round to
 * nearest even) and the Jacobi diagonal 1/a_ii. Asynchronous. */
rp_status rp_update_values_packed(rp_handle* h, const double* buffer, int32_t where, void* stream);
/* (where = RP_MEM_HOST_ASYNC: see the RP_MEM_ enum above.) */

/* Same, from per-rank arrays (k pointers each; lower may be NULL in
 * symmetric mode). The arrays are copied into the staging buffer at their
 * rank's offsets, then permuted. */
rp_status rp_update_values(rp_handle* h, const double* const* diag, const double* const* upper,
                           const double* const* lower, const double* const* iface, int32_t where,
                           void* stream);

/* Device views of the current values (vals32 NULL without want_fp32). */
rp_status rp_get_values(const rp_handle* h, const double** vals, const float** vals32,
                        const double** dinv);

/* y = A x with the FP64 values (local + non-local for n_parts > 1); if xy is not NULL the
 * device double *xy receives x.y. x, y, xy are device pointers. Uses the
 * handle's reduction scratch. Asynchronous. */
rp_status rp_spmv(rp_handle* h, const double* x, double* y, double* xy, void* stream);

/* Allocation-free SpMV: y = A x and, if xy is not NULL, *xy = x.y, for a
 * caller-owned CSR matrix (row_ptr[n+1] from 0, col_idx, vals, all device
 * pointers, like the views of rp_get_part_map / rp_get_values). The paper
 * has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- code whose device memory is owned by a host framework's
 * pool, code running while a stream is being captured, and code that must
 * not allocate after start-up -- and who therefore cannot create a handle.
 * It allocates nothing (no cudaMalloc/cudaFree, no allocating library
 * call): its reduction scratch is a static device array of 64 KiB + 256 B,
 * which every GPU that loads the library holds until the process exits.
 * Limit: n <= 16,777,216 rows (n above it returns RP_ERANGE, no device
 * work). The first call on a device looks up the array's device address
 * with that device current; make that first call before any stream
 * capture. The address stays cached for the life of the process: a reset of
 * the device (cudaDeviceReset, or of its primary context) invalidates it, so
 * after one this entry point must not be called again on that device in the
 * same process. All calls on a device share the array: calls whose work overlaps
 * on the GPU (different streams, no ordering) race and give wrong x.y. y is
 * the same per row as rp_spmv's; x.y agrees to rounding. Asynchronous. */
rp_status rp_spmv_noalloc(int64_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* vals,
                          const double* x, double* y, double* xy, void* stream);

/* The sliced layout the PCG iteration multiplies with (the paper has no
 * counterpart: it is this library's device format of the merged matrix, built
 * once next to the CSR map by rp_build_repartition and refilled from the CSR
 * values by every value update). Rows in slices of 32 (n_slices = ceil(n/32)
 * for one part, the sum of ceil(n_p/32) over parts; 0 when the layout is not
 * in use), one row per lane. Slice s: desc[2s] = x_s,
 * desc[2s+1] = y_s (uint32 pairs; desc[2 n_slices], desc[2 n_slices + 1]
 * close the last slice); L_s = (x_{s+1} - x_s) / 32 entries per row, the
 * longest row of the slice, shorter rows padded with zero values; values of
 * entry k of lane j at vals[x_s + 32 k + j] (vals32 alike, NULL without
 * want_fp32). tinfo[s] = t | w4 << 31: the slice's table of distinct column
 * offsets (col - row, first-appearance order over entry k, then lane) is
 * tabs[t .. t + D), D = tabs[t - 1] (equal tables are stored once); w4 = 1
 * (D <= 16): 4-bit offset indices, entry 8 g + e of lane j in bits 4e..4e+3
 * of ibuf[y_s + 32 g + j]; w4 = 0: 8-bit indices, entry 4 g + e in byte e of
 * ibuf[y_s + 32 g + j]. pos[x_s + 32 k + j] is the CSR position of that entry,
 * -1 for padding. Entry k of a row is its k-th CSR entry. With several parts
 * (n_parts > 1, and every batched handle: one part per system) the slices of
 * every part follow one another, part p's ceil(n_p / 32) slices after those
 * of parts < p; rows and column offsets are those of the part's local CSR
 * matrix (rp_get_part_map), pos holds positions in the handle's value array
 * (rp_get_values), and srow[2s] = the first merged row of slice s,
 * srow[2s+1] = p << 6 | (rows of the part in the slice, at most 32); srow is
 * NULL for one part (slice s holds rows 32 s ..). The non-local entries of a
 * part stay in its non-local CSR. The batched kernel writes the sliced values
 * itself; every value update refills them. Device views, owned by the handle;
 * n_entries counts padded entries, ibuf_len index words, tabs_len table
 * words. */
typedef struct rp_sliced_view {
  int64_t n_slices, n_entries, ibuf_len, tabs_len;
  const uint32_t* desc;
  const uint32_t* tinfo;
  const int32_t* tabs;
  const int32_t* ibuf;
  const int32_t* pos;
  const double* vals;
  const float* vals32;
  const int32_t* srow;
  /* The FP32 inner iteration of the mixed PCG solves (one part, Jacobi) runs
   * on the symmetrically scaled matrix S A S, S = diag(scale): scale[i] =
   * 1 / sqrt(a_ii) in FP64 (correctly rounded square root and division),
   * vals32s[q] = fl32(a_ij (scale_i scale_j)) with the products in FP64 (the
   * diagonal is exactly 1), 0 for padding -- Jacobi preconditioning made
   * explicit (CG on S A S from fl32(S r) is PCG with the preconditioner
   * S^2 = D^-1). Both NULL until the first mixed solve on a handle that takes
   * it; then refilled by every value update. */
  const float* vals32s;
  const double* scale;
  /* 1 if every slice has 4-bit indices and rows of at most 8 entries: the
   * iteration then multiplies with a kernel instance that skips the checks of
   * the general case (k_it_spmv_sl<T, true>; one part only, and not in the
   * bounds-checked build, which checks every slice). */
  int32_t uniform4;
} rp_sliced_view;
rp_status rp_get_sliced_view(const rp_handle* h, rp_sliced_view* out);

/* The SpMV of the PCG iteration, y = A x, in its working precision and
 * layout (Sec. 4: the pressure solve's matrix product): precision RP_FP64
 * reads double x, writes double y from the FP64 values; RP_MIXED or
 * RP_MIXED_RU reads float x, writes float y from the FP32 values, summing
 * each row in FP32. Same kernel the solve launches (sliced or CSR, n_parts
 * parts); a row's products are accumulated with fused multiply-adds in the
 * row's CSR order. x, y device pointers of n elements. Uses the handle's
 * reduction scratch and a control block of its own. Asynchronous. */
rp_status rp_iter_spmv(rp_handle* h, const void* x, void* y, int32_t precision, void* stream);

typedef struct rp_solve_info {
  int32_t status;           /* RP_OK, RP_NOT_CONVERGED or RP_BREAKDOWN       */
  int32_t iterations;       /* PCG iterations (FP32 inner ones when mixed)   */
  int32_t outer_iterations; /* refinement steps (mixed)                      */
  int32_t restarts;         /* residual replacements                         */
  int32_t passes;           /* FP64 residual passes (b - A x) of the solve   */
  double rel_residual;      /* ||b - A x|| / ||b|| recomputed in FP64 at exit */
} rp_solve_info;

/* Solve A x = b to ||b - A x||_2 <= tol ||b||_2 (true residual, FP64).
 * With n_parts > 1 every product runs over each part's local matrix plus
 * its non-local matrix, whose halo values are gathered from x on the device
 * (the distributed layout of Sec. 3 on one GPU); the result is the same
 * system's solution.
 * precision RP_FP64: Jacobi-PCG in FP64. RP_MIXED: iterative refinement with
 * the residual, the update x += d and the convergence test in FP64 and the
 * inner Jacobi-PCG on the FP32 values to inner_tol, or to half the outer
 * target when that comes first (needs want_fp32). RP_MIXED_RU: see above.
 * x_is_guess: start from x (else x = 0). where: b and x are host or device.
 * The whole iteration runs on the device (CUDA graph with conditional
 * nodes), with no host synchronisation. If info is not NULL the call waits
 * for the stream and fills it; the return value is then info->status. */
rp_status rp_solve(rp_handle* h, const double* b, double* x, double tol, int32_t precision,
                   int32_t x_is_guess, int32_t where, rp_solve_info* info, void* stream);

/* Outcome of the latest rp_solve on this handle that was launched with
 * info = NULL: waits for `stream` and fills info (the return value is then
 * info->status). Lets a caller queue the next time step's value update
 * (e.g. RP_MEM_HOST_ASYNC) behind a solve before it waits for the solve.
 * Value updates in between leave the outcome intact; another solve, adjoint
 * solve or rp_profile_iteration on the handle replaces it. RP_EINVAL if no
 * solve has run on the handle. */
rp_status rp_get_solve_info(rp_handle* h, rp_solve_info* info, void* stream);

/* Solve a non-symmetric system A x = b (the momentum equation, which the paper
 * solves with BiCGStab; Sec. 4) to ||b - A x||_2 <= tol ||b||_2 (true
 * residual, FP64) with Jacobi-preconditioned BiCGStab (van der Vorst, 1992;
 * D^-1 applied to the search directions) in FP64 on the handle's current
 * values (general storage: lower and upper coefficients differ). One
 * iteration = two products with A. A recursive residual at the target is
 * confirmed with b - A x; if that fails the iteration restarts from the true
 * residual with a new shadow residual (at most max_restarts times).
 * (rhat, v) = 0, (rhat, r) = 0 or omega = 0 end with RP_BREAKDOWN; max_iter
 * caps the iterations (RP_NOT_CONVERGED). Parts, x_is_guess, where, info and
 * the return value as in rp_solve; info->outer_iterations is 0. Allocates
 * five n-vectors on first use. */
rp_status rp_solve_bicgstab(rp_handle* h, const double* b, double* x, double tol, int32_t x_is_guess,
                            int32_t where, rp_solve_info* info, void* stream);

/* The same system by FP32-inner / FP64-outer iterative refinement (needs
 * want_fp32): repeat { r = b - A x with the FP64 values (true residual); stop
 * when ||r|| <= tol ||b||; solve A32 d = fl32(r) by Jacobi-preconditioned
 * BiCGStab on the FP32 values, vectors and products (dot products combined in
 * FP64; alpha, omega, beta rounded to FP32), from d = 0 with the shadow
 * residual fl32(r), to ||r_inner|| <= inner_tol ||fl32(r)|| (a half step counts
 * with ||s||); x += d in FP64 }. max_outer caps the refinements, max_iter the
 * inner iterations of all refinements together (RP_NOT_CONVERGED); a
 * breakdown of an inner solve ends with RP_BREAKDOWN. info->iterations =
 * inner iterations, info->outer_iterations = refinements, rel_residual = the
 * last FP64 residual. Other arguments as in rp_solve_bicgstab. Allocates five
 * FP32 n-vectors on first use. */
rp_status rp_solve_bicgstab_mixed(rp_handle* h, const double* b, double* x, double tol, int32_t x_is_guess,
                                  int32_t where, rp_solve_info* info, void* stream);

/* ---- Batched form: many independent systems in one persistent launch ----
 * The paper has no counterpart: it merges the LDU matrices of one problem.
 * This form applies the same repartition, update and Jacobi-PCG (Sec. 3-4)
 * to many uneven independent problems at once; it is this library's
 * extension of the method, defined by those same steps per system.
 * Each system is one LDU matrix without interfaces (n_iface = 0); system s
 * becomes GPU part s (n_parts = count, alpha = 1, Sec. 3). Rows, buffers and
 * vectors of the systems follow each other in system order.
 * rp_batch_build: as rp_build_repartition with n_parts = count. Errors as
 * there, plus RP_EINVAL if a system has interface entries. Blocks the host. */
rp_status rp_batch_build(const rp_ldu_desc* systems, int32_t count, const rp_options* opts, rp_handle** out);

/* One batched time step: the value update of every system from `buffer`
 * (all systems' continuous buffers concatenated; where = host or device)
 * and the solve of every system to its own ||b_s - A_s x_s|| <= tol ||b_s||
 * from x_s = 0 (precision RP_FP64, RP_MIXED or RP_MIXED_RU; on the sliced
 * layout the mixed forms' FP32 iteration runs on the symmetrically scaled
 * system S A S, s_i = 1/sqrt(a_ii) in FP64, FP32 values fl32(a_ij (s_i s_j)),
 * which the kernel writes into the sliced view's vals32), all in ONE
 * persistent kernel
 * launched from a CUDA graph (instantiated on first use per precision).
 * b and x are device pointers (n_rows doubles, system order). Thread-block
 * clusters act as teams that take systems largest first from a device work
 * queue; a team's CTAs synchronise with cluster barriers only. If info is not
 * NULL (host array of count entries) the call waits and fills it, returning
 * the first non-OK system status. */
rp_status rp_batch_update_solve(rp_handle* h, const double* buffer, int32_t where, const double* b, double* x,
                                double tol, int32_t precision, rp_solve_info* info, void* stream);

/* Launch shape of the batched kernel: cluster size (1 to 16 CTAs per team;
 * above 8 a non-portable cluster size) and threads per CTA (multiple of 32,
 * <= 512). RP_EINVAL outside those ranges, RP_EUNSUPPORTED if the shape
 * cannot be scheduled. Default 5 x 512. */
rp_status rp_batch_set_config(rp_handle* h, int32_t cluster, int32_t threads);

/* Autotuner: times rp_batch_update_solve (device buffer, precision) for every
 * cluster size in {2, 3, 4, 5, 6, 8, 16} and CTA size in {256, 512}, keeps
 * the fastest shape in the handle and reports it. Overwrites x. Blocks. */
rp_status rp_batch_autotune(rp_handle* h, const double* buffer, const double* b, double* x, double tol,
                            int32_t precision, int32_t* best_cluster, int32_t* best_threads, float* best_ms,
                            void* stream);

/* Kernel timing: starts a CG run from x = 0 on right-hand side b (device)
 * with the current values and launches `iters` iterations of the three
 * iteration kernels of `precision` on the stream (outside any graph, with no
 * stopping test), each bracketed by CUDA events. ms_out[0..2] receives the
 * average duration of the SpMV kernel, the residual-update kernel and the
 * x/p-update kernel. The kernels are the ones rp_solve's graph runs. Uses the
 * handle's work vectors; blocks the host. */
rp_status rp_profile_iteration(rp_handle* h, const double* b, int32_t precision, int32_t iters,
                               float* ms_out, void* stream);

/* ---- Differentiation: the paper has no counterpart ----
 * The adjoint of the pressure solve, this library's extension of the method
 * on the same merged matrix and map, defined by the plain calculus of a
 * linear solve: for A x = b and a loss L(x), A^T lambda = dL/dx gives
 * dL/db = lambda and dL/da_ij = -lambda_i x_j for every stored entry.
 *
 * Adjoint solve A^T lambda = g (FP64 Jacobi-PCG on the transposed values,
 * built through tpos; needs want_transpose unless symmetric storage).
 * Device pointers; info as in rp_solve. */
rp_status rp_solve_adjoint(rp_handle* h, const double* g, double* lambda, double tol,
                           rp_solve_info* info, void* stream);

/* Gradients of a loss L(x) with A x = b and A^T lambda = dL/dx:
 * dL/da_ij = -lambda_i x_j for every stored entry, summed per buffer slot
 * into g_buffer[n_slots] (the layout of rp_update_values_packed).
 * Device pointers. Asynchronous. */
rp_status rp_entry_grad(rp_handle* h, const double* lambda, const double* x, double* g_buffer,
                        void* stream);

/* Gradient w.r.t. face coefficients a_f that enter as +a_f on both
 * diagonals and -a_f on both off-diagonals: -(lambda_l - lambda_u)(x_l - x_u),
 * written rank after rank as [faces F_r | interface entries E_r].
 * Device pointers. Asynchronous. */
rp_status rp_face_grad(rp_handle* h, const double* lambda, const double* x, double* g_face,
                       void* stream);

/* Bounds-checked build only (librepart_check.so, compiled with RP_CHECK;
 * the paper has no counterpart: it is this library's stand-in for a memory
 * checker). Its kernels range-check every gather index and every offset they
 * derive from the map or the sliced layout -- buffer slots src_of, CSR
 * columns and positions, non-local columns and halo rows, slice descriptors,
 * table references and offset indices, the source ranges of staged copies,
 * the map build's placements -- and skip an access that would leave its
 * array (a load reads zero, a store is dropped) instead of trapping. Waits
 * for the device, then returns in *count the accesses skipped since the last
 * reset (in every kernel of the library), with the site (a small integer
 * naming the kind of index, 1-10) and the index of the first one; reset = 1
 * clears the counters. The normal build returns RP_EUNSUPPORTED with
 * *count = 0. */
rp_status rp_check_violations(uint64_t* count, int32_t* first_site, int64_t* first_index, int32_t reset);

void rp_destroy(rp_handle* h);
const char* rp_status_str(rp_status s);
const char* rp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* REPART_H */
