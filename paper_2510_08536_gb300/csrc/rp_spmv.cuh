// SpMV building blocks shared by the solvers: row products over CSR (and
// over the local + non-local CSR of GPU parts), the sliced-layout decoders,
// the TMA / mbarrier helpers and the two SpMV bodies, y = A x over CSR and
// over the sliced layout, each followed by a solver-specific epilogue.
#pragma once

#include <type_traits>

#include "rp_common.cuh"

namespace rp {

// Row i of a CSR matrix with ncols columns (ncols bounds the gathers in the
// bounds-checked build).
template <typename T>
__device__ __forceinline__ T row_dot(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                     const T* __restrict__ vals, const T* __restrict__ x, int64_t i, int64_t ncols) {
  const int s = __ldg(row_ptr + i), e = __ldg(row_ptr + i + 1);
  T sum = T(0);
  for (int j = s; j < e; ++j) {
    const int c = __ldg(col + j);
    if (RP_IN(c, 0, ncols, kChkGather)) sum = fma(__ldg(vals + j), __ldg(x + c), sum);
  }
  return sum;
}

// Global row behind non-local entry j of part p (entry and compressed-column
// offsets nlo, nco): the halo row the entry gathers. Bounds-checked build: -1
// when the compressed column or its row is out of range.
template <typename T>
__device__ __forceinline__ int nl_row_of(const Parts<T>& P, int p, int64_t nlo, int64_t nco, int j) {
  const int cc = __ldg(P.nl_col + nlo + j);
  if (!RP_IN(cc, 0, __ldg(P.nlcol_off + p + 1) - nco, kChkNonlocal)) return -1;
  const int g = __ldg(P.nl_cols + nco + cc);
  return RP_IN(g, 0, __ldg(P.row_off + P.n), kChkNonlocal) ? g : -1;
}

// The non-local entries of row i (part p) added to sum in their CSR order:
// the part's non-local CSR, whose compressed columns name the halo rows -- on
// one GPU the halo exchange is this gather from x (global vector).
template <typename T>
__device__ __forceinline__ T nonlocal_add(const Parts<T>& P, int p, int64_t i, const T* __restrict__ x, T sum) {
  const int64_t r0 = __ldg(P.row_off + p), li = i - r0;
  const int32_t* nrp = P.nl_row_ptr + r0 + p;
  const int64_t nlo = __ldg(P.nl_off + p), nco = __ldg(P.nlcol_off + p);
  for (int j = __ldg(nrp + li); j < __ldg(nrp + li + 1); ++j) {
    const int g = nl_row_of<T>(P, p, nlo, nco, j);
    if (RP_IDX_OK(g)) sum = fma(__ldg(P.nl_vals + nlo + j), __ldg(x + g), sum);
  }
  return sum;
}

// The same in two steps, so that the row's non-local range is loaded before
// its local sum: nonlocal_range, then nonlocal_sum (the part's offsets are
// read again there, from L1, to keep few registers live across the sum).
struct NlRange {
  int j0, j1;
};
template <typename T>
__device__ __forceinline__ NlRange nonlocal_range(const Parts<T>& P, int p, int64_t i) {
  const int64_t r0 = __ldg(P.row_off + p), li = i - r0;
  const int32_t* nrp = P.nl_row_ptr + r0 + p;
  return NlRange{__ldg(nrp + li), __ldg(nrp + li + 1)};
}
template <typename T>
__device__ __forceinline__ T nonlocal_sum(const Parts<T>& P, int p, const NlRange& r, const T* __restrict__ x,
                                          T sum) {
  if (r.j0 == r.j1) return sum;
  const int64_t nlo = __ldg(P.nl_off + p), nco = __ldg(P.nlcol_off + p);
  for (int j = r.j0; j < r.j1; ++j) {
    const int g = nl_row_of<T>(P, p, nlo, nco, j);
    if (RP_IDX_OK(g)) sum = fma(__ldg(P.nl_vals + nlo + j), __ldg(x + g), sum);
  }
  return sum;
}

// Row i of the matrix split into parts (Sec. 3): the part's local CSR (part-
// local columns), then its non-local entries.
template <typename T>
__device__ __forceinline__ T row_dot_parts(const Parts<T>& P, const int32_t* __restrict__ row_ptr,
                                           const int32_t* __restrict__ col, const T* __restrict__ vals,
                                           const T* __restrict__ x, int64_t i) {
  const int p = find_rank(P.row_off, P.n, i);
  const int64_t r0 = __ldg(P.row_off + p), li = i - r0;
  const int32_t* rp = row_ptr + r0 + p;
  const int64_t no = __ldg(P.nnz_off + p);
  T sum = T(0);
  for (int j = __ldg(rp + li); j < __ldg(rp + li + 1); ++j) {
    const int c = __ldg(col + no + j);
    if (RP_IN(c, 0, __ldg(P.row_off + p + 1) - r0, kChkGather)) sum = fma(__ldg(vals + no + j), __ldg(x + r0 + c), sum);
  }
  return nonlocal_add<T>(P, p, i, x, sum);
}

inline Parts<double> parts64(const rp_handle* h) {
  return Parts<double>{h->n_parts, h->d_part_row_off, h->d_part_nnz_off, h->d_part_nl_off, h->d_part_nlcol_off,
                       h->nl_row_ptr, h->nl_col_idx, h->nl_cols, h->nl_vals};
}
inline Parts<float> parts32(const rp_handle* h) {
  return Parts<float>{h->n_parts, h->d_part_row_off, h->d_part_nnz_off, h->d_part_nl_off, h->d_part_nlcol_off,
                      h->nl_row_ptr, h->nl_col_idx, h->nl_cols, h->nl_vals32};
}

// Row i of the merged matrix (n rows), one part or several.
template <typename T>
__device__ __forceinline__ T row_dot_any(const Parts<T>& P, const int32_t* __restrict__ row_ptr,
                                         const int32_t* __restrict__ col, const T* __restrict__ vals,
                                         const T* __restrict__ x, int64_t i, int64_t n) {
  return P.n > 1 ? row_dot_parts<T>(P, row_ptr, col, vals, x, i) : row_dot<T>(row_ptr, col, vals, x, i, n);
}

// The sliced layout of the iteration (with per-slice row records when the
// matrix has several parts).
inline Sliced<double> sliced64(const rp_handle* h, const double* vals) {
  const double* v = vals == h->vals ? h->sl_vals : vals == h->valsT ? h->sl_valsT : nullptr;
  if (h->sl_slices == 0 || !v) return Sliced<double>{};
  return Sliced<double>{h->sl_slices, h->sl_desc, h->sl_tinfo, h->sl_tabs, h->sl_ibuf, v, h->opts.spin_limit,
                        h->sl_srow, h->sl_entries, h->sl_ibuf_len, h->sl_tabs_len, h->sl_u4};
}
inline Sliced<float> sliced32(const rp_handle* h) {
  if (h->sl_slices == 0 || !h->sl_vals32) return Sliced<float>{};
  return Sliced<float>{h->sl_slices, h->sl_desc, h->sl_tinfo, h->sl_tabs, h->sl_ibuf, h->sl_vals32,
                       h->opts.spin_limit, h->sl_srow, h->sl_entries, h->sl_ibuf_len, h->sl_tabs_len, h->sl_u4};
}

// Rows of slice s: the first (global) row, how many of its 32 lanes hold a
// row (a part's last slice may be short) and the part.
struct SliceRows {
  int row0, rows, part;
};
template <typename T>
__device__ __forceinline__ SliceRows slice_rows(const Sliced<T>& sl, int s, int n) {
  if (sl.srow) {
    const int2 r = __ldg(sl.srow + s);
    return SliceRows{r.x, r.y & 63, r.y >> 6};
  }
  return SliceRows{s * kSliceRows, min(kSliceRows, n - s * kSliceRows), 0};
}

// 16-byte vectors of the streaming kernels
template <typename T>
struct Vec;
template <>
struct Vec<float> {
  using type = float4;
  static constexpr int N = 4;
};
template <>
struct Vec<double> {
  using type = double2;
  static constexpr int N = 2;
};

template <int E>
__device__ __forceinline__ float& comp(float4& v) {
  return E == 0 ? v.x : E == 1 ? v.y : E == 2 ? v.z : v.w;
}
template <int E>
__device__ __forceinline__ double& comp(double2& v) {
  return E == 0 ? v.x : v.y;
}

// apply f(element index e, element references...) to every component
template <int W, typename F, int E = 0>
__device__ __forceinline__ void for_each_comp(F&& f) {
  if constexpr (E < W) {
    f(std::integral_constant<int, E>{});
    for_each_comp<W, F, E + 1>(static_cast<F&&>(f));
  }
}

// ---- SpMV over the sliced layout, staged through shared memory by TMA bulk copies.
//
// A block is kChunk consumer warps plus one producer warp. The block owns
// chunks of kChunk consecutive slices (consumer warp w takes slice w of the
// chunk: rows 256 c + 32 w + lane, as the CSR body's thread 32 w + lane of
// block c maps rows). The producer keeps up to kStages chunks in flight:
// once consumers have released a stage (its "empty" mbarrier), it posts the
// byte count on the stage's "full" mbarrier and issues four cp.async.bulk
// copies -- the chunk's values, its index words, its run of slice
// descriptors and its table references. Bytes in flight cost no registers,
// and consumer warps wait only on their own chunk's data, not on each other;
// a slice then waits on one memory round trip, its gathers of p. The offset
// tables (few, shared by many slices) are read through L1 and looked up with
// warp shuffles (slice_offset); rows of up to 8 entries run a body unrolled
// for their exact width. A chunk larger than a stage (long rows) is read
// straight from global memory by the same warps. Every barrier wait is bounded: after
// spin iterations the block waits (bounded) for its own copies and calls the
// epilogue's timeout (which records RP_DEVICE_TIMEOUT and stops the solve).
//
// Epilogue (Epi): row(i, y_i) per computed row (per-thread accumulation),
// timeout() by one thread of a block whose wait ran out, finish() by every
// thread at the end (block reduction, last-block scalars).

constexpr int kChunk = kThreads / 32;  // slices per chunk, one per consumer warp
constexpr int kSlThreads = kThreads + 32;
constexpr int kStageIdx = 3072;        // index word bytes a stage holds
constexpr int kStageDesc = 128;        // descriptor run (kChunk + 1 entries, padded)
constexpr int kStageInfo = 32;         // table references of the chunk's kChunk slices

// Two stages per block (FP32 23 KB, FP64 39 KB): warps beat depth -- at
// 256^3 the FP32 SpMV takes 0.138 ms with 2 stages (7 blocks of 9 warps an
// SM, register-limited), 0.145 ms with 3 (6 blocks, shared-memory-limited),
// 0.171 ms with 4.
template <typename T>
struct SlStage {
  static constexpr int kStages = 2;
  static constexpr int kVals = kChunk * kSliceRows * 8 * (int)sizeof(T);  // rows of <= 8 entries
  static constexpr int kBytes = kVals + kStageIdx + kStageDesc + kStageInfo;
  static constexpr int kSmem = kStages * kBytes;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int64_t limit) {
  for (int64_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// global -> shared bulk copy completing on bar (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// the same with an L2 cache policy (createpolicy) for the copied lines
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
               : "memory");
}

// Asynchronous prefetch of [src, src + bytes) into L2 (no completion to wait
// for); src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// How a slice's offset indices are read: 4-bit indices into a table of at
// most 16 offsets held in tv by both half-warps (lane & 15), looked up by a
// shuffle of width 16 (the source lane is taken modulo 16, so a shifted word
// needs no mask); 8-bit indices into a table of at most 32 offsets held in tv,
// shuffle of width 32; 8-bit indices into a longer table, read from global
// memory (tables are few and stay in L1). All lanes call the shuffles.
enum : int { kIdx4 = 0, kIdx8Shfl = 1, kIdx8Glob = 2 };

template <int MODE>
__device__ __forceinline__ int slice_offset(uint32_t wd, int e, int32_t tv, const int32_t* tab, int D) {
  if (MODE == kIdx4) return __shfl_sync(0xffffffffu, tv, (int)(wd >> (4 * e)), 16);
  if (MODE == kIdx8Shfl) return __shfl_sync(0xffffffffu, tv, (int)(wd >> (8 * e)));
#ifdef RP_CHECK
  return __ldg(tab + min((int)((wd >> (8 * e)) & 255u), D - 1));  // in the table; the index is checked apart
#else
  (void)D;
  return __ldg(tab + ((wd >> (8 * e)) & 255u));
#endif
}

// Bounds of one lane's gathers in the bounds-checked build: admissible
// offsets col - row of the lane's row, [lo, hi), and the lengths of the
// arrays the slice's descriptor and table reference index.
struct SliceCk {
  int lo, hi;
  int64_t entries, ibuf, tabs;
};

// Bounds-checked build: is index e of word wd inside the slice's table of D
// offsets, and the offset it names inside the lane's admissible range?
template <int MODE>
__device__ __forceinline__ bool slice_ok(uint32_t wd, int e, int off, int D, const SliceCk& ck) {
#ifdef RP_CHECK
  const int id = MODE == kIdx4 ? (int)((wd >> (4 * e)) & 15u) : (int)((wd >> (8 * e)) & 255u);
  return RP_IN(id, 0, D, kChkSliceIndex) && RP_IN(off, ck.lo, ck.hi, kChkGather);
#else
  (void)wd, (void)e, (void)off, (void)D, (void)ck;
  return true;
#endif
}

// A gather from x: read-only path, or (COH) a plain load for a vector that the
// same kernel writes.
template <bool COH, typename T>
__device__ __forceinline__ T xload(const T* p) {
  if (COH) return *p;
  return __ldg(p);
}

// Sum of one row of a slice, L entries: values at v[32 k] (lane applied),
// index words at iw[32 g] (lane applied); the same fused multiply-adds in the
// same order as row_dot over the row's CSR entries. Lanes without a row
// (valid false) run the shuffles but load nothing.
template <typename T, int MODE, int L, bool COH = false>
__device__ __forceinline__ T slice_row_exact(const T* v, const uint32_t* iw, int32_t tv, const int32_t* tab,
                                             const T* x, bool valid, int D, const SliceCk& ck) {
  constexpr int PER = MODE == kIdx4 ? 8 : 4;
  const uint32_t w0 = iw[0], w1 = L > PER ? iw[kSliceRows] : 0u;
  T vv[L];
#pragma unroll
  for (int k = 0; k < L; ++k) vv[k] = v[k * kSliceRows];
  T sum = T(0);
#pragma unroll
  for (int k = 0; k < L; ++k) {
    const uint32_t wd = k < PER ? w0 : w1;
    const int off = slice_offset<MODE>(wd, k % PER, tv, tab, D);
    if (valid && slice_ok<MODE>(wd, k % PER, off, D, ck)) sum = fma(vv[k], xload<COH>(x + off), sum);
  }
  return sum;
}

template <typename T, int MODE, bool COH = false>
__device__ __forceinline__ T slice_row(const T* v, const uint32_t* iw, int32_t tv, const int32_t* tab, const T* x,
                                       bool valid, int L, int D, const SliceCk& ck) {
  switch (L) {
    case 1: return slice_row_exact<T, MODE, 1, COH>(v, iw, tv, tab, x, valid, D, ck);
    case 2: return slice_row_exact<T, MODE, 2, COH>(v, iw, tv, tab, x, valid, D, ck);
    case 3: return slice_row_exact<T, MODE, 3, COH>(v, iw, tv, tab, x, valid, D, ck);
    case 4: return slice_row_exact<T, MODE, 4, COH>(v, iw, tv, tab, x, valid, D, ck);
    case 5: return slice_row_exact<T, MODE, 5, COH>(v, iw, tv, tab, x, valid, D, ck);
    case 6: return slice_row_exact<T, MODE, 6, COH>(v, iw, tv, tab, x, valid, D, ck);
    case 7: return slice_row_exact<T, MODE, 7, COH>(v, iw, tv, tab, x, valid, D, ck);
    case 8: return slice_row_exact<T, MODE, 8, COH>(v, iw, tv, tab, x, valid, D, ck);
    default: break;
  }
  constexpr int PER = MODE == kIdx4 ? 8 : 4;
  T sum = T(0);
  for (int g = 0; g < (L + PER - 1) / PER; ++g) {
    const uint32_t wd = iw[g * kSliceRows];
#pragma unroll
    for (int e = 0; e < PER; ++e)
      if (PER * g + e < L) {
        const int off = slice_offset<MODE>(wd, e, tv, tab, D);
        if (valid && slice_ok<MODE>(wd, e, off, D, ck))
          sum = fma(v[(PER * g + e) * kSliceRows], xload<COH>(x + off), sum);
      }
  }
  return sum;
}

// Bounds-checked build: the slice's descriptor pair, row length, index words
// and table reference inside their arrays (warp-uniform: the whole warp
// skips a bad slice); D receives the table's length.
__device__ __forceinline__ bool slice_desc_ok(uint2 d0, uint2 d1, uint32_t info, const int32_t* __restrict__ tabs,
                                              const SliceCk& ck, int& D) {
#ifdef RP_CHECK
  const int64_t t = info & ~kSliceW4;
  if (!RP_IN(d0.x, 0, ck.entries + 1, kChkSliceDesc) || !RP_IN(d1.x, d0.x, ck.entries + 1, kChkSliceDesc) ||
      !RP_IN(d1.x - d0.x, 0, kSliceRows * kSliceMaxWidth + 1, kChkSliceDesc) || ((d1.x - d0.x) & 31u) != 0u ||
      !RP_IN(d0.y, 0, ck.ibuf + 1, kChkSliceDesc) || !RP_IN(d1.y, d0.y, ck.ibuf + 1, kChkSliceDesc) ||
      !RP_IN(t, 1, ck.tabs, kChkSliceDesc))
    return false;
  D = __ldg(tabs + t - 1);
  const int L = (int)((d1.x - d0.x) >> 5), per = (info & kSliceW4) ? 8 : 4;
  return RP_IN(D, 1, (info & kSliceW4) ? 17 : kSliceMaxDict + 1, kChkSliceDesc) &&
         RP_IN(t + D, t, ck.tabs - 32 + 1, kChkSliceDesc) &&  // the 32 spare words stay past every table
         RP_IN(d1.y - d0.y, (int64_t)kSliceRows * ((L + per - 1) / per), (int64_t)kSliceRows * ((L + per - 1) / per) + 1,
               kChkSliceDesc);
#else
  (void)d0, (void)d1, (void)info, (void)tabs, (void)ck, (void)D;
  return true;
#endif
}

// One slice: descriptor pair (d0, d1), table reference info, values v and
// index words iw (shared memory or global, lane applied), tables tabs (global),
// gathers from x relative to the lane's row (COH: plain loads, see xload);
// ck: the bounds the checked build tests.
template <typename T, bool COH = false>
__device__ __forceinline__ T slice_sum(uint2 d0, uint2 d1, uint32_t info, const T* v, const uint32_t* iw,
                                       const int32_t* __restrict__ tabs, const T* x, bool valid, int lane,
                                       const SliceCk& ck) {
  int D = 0;
  if (!slice_desc_ok(d0, d1, info, tabs, ck, D)) return T(0);
  const int L = (int)((d1.x - d0.x) >> 5);
  const int32_t* tab = tabs + (info & ~kSliceW4);
  if (info & kSliceW4) return slice_row<T, kIdx4, COH>(v, iw, __ldg(tab + (lane & 15)), tab, x, valid, L, D, ck);
  if (__ldg(tab - 1) <= 32) return slice_row<T, kIdx8Shfl, COH>(v, iw, __ldg(tab + lane), tab, x, valid, L, D, ck);
  return slice_row<T, kIdx8Glob, COH>(v, iw, 0, tab, x, valid, L, D, ck);
}

// The table entry a lane holds for a slice: entry lane & 15 of a 4-bit table,
// entry lane of an 8-bit one (the tables area keeps 32 spare words past its
// last table, so the read stays inside it). For callers that load it a slice
// ahead; in the bounds-checked build a reference outside the area loads
// nothing (slice_desc_ok reports it when the slice is summed).
__device__ __forceinline__ int32_t slice_tab_entry(uint32_t info, const int32_t* __restrict__ tabs, int lane,
                                                   int64_t tabs_len) {
  const int64_t t = info & ~kSliceW4;
#ifdef RP_CHECK
  if (t < 1 || t + 32 > tabs_len) return 0;
#else
  (void)tabs_len;
#endif
  return __ldg(tabs + t + ((info & kSliceW4) ? (lane & 15) : lane));
}

// slice_sum with the lane's table entry tv already loaded (slice_tab_entry).
template <typename T, bool COH = false>
__device__ __forceinline__ T slice_sum_tv(uint2 d0, uint2 d1, uint32_t info, int32_t tv, const T* v,
                                          const uint32_t* iw, const int32_t* __restrict__ tabs, const T* x,
                                          bool valid, const SliceCk& ck) {
  int D = 0;
  if (!slice_desc_ok(d0, d1, info, tabs, ck, D)) return T(0);
  const int L = (int)((d1.x - d0.x) >> 5);
  const int32_t* tab = tabs + (info & ~kSliceW4);
  if (info & kSliceW4) return slice_row<T, kIdx4, COH>(v, iw, tv, tab, x, valid, L, D, ck);
  if (__ldg(tab - 1) <= 32) return slice_row<T, kIdx8Shfl, COH>(v, iw, tv, tab, x, valid, L, D, ck);
  return slice_row<T, kIdx8Glob, COH>(v, iw, 0, tab, x, valid, L, D, ck);
}

// The gather bounds of a lane's row in the bounds-checked build: the rows of
// its part (several parts, MP) or of the matrix.
template <typename T, bool MP>
__device__ __forceinline__ SliceCk slice_ck(const Sliced<T>& sl, const Parts<T>& P, int part, int row, int n) {
#ifdef RP_CHECK
  int64_t lo = 0, hi = n;
  if (MP) {
    lo = __ldg(P.row_off + part);
    hi = __ldg(P.row_off + part + 1);
  }
  return SliceCk{(int)(lo - row), (int)(hi - row), sl.n_entries, sl.ibuf_len, sl.tabs_len};
#else
  (void)sl, (void)P, (void)part, (void)row, (void)n;
  return SliceCk{};
#endif
}

// Bounds-checked build: the source ranges of a chunk's four staged copies
// inside their arrays (values, index words, descriptor run, table references).
template <typename T>
__device__ __forceinline__ bool chunk_copy_ok(const Sliced<T>& sl, uint2 d0, uint2 d1, int ch, uint32_t db) {
#ifdef RP_CHECK
  return RP_IN(d0.x, 0, sl.n_entries + 1, kChkSliceCopy) && RP_IN(d1.x, d0.x, sl.n_entries + 1, kChkSliceCopy) &&
         RP_IN(d0.y, 0, sl.ibuf_len + 1, kChkSliceCopy) && RP_IN(d1.y, d0.y, sl.ibuf_len + 1, kChkSliceCopy) &&
         RP_IN((int64_t)ch * kChunk + db / 8, 0, sl.n_slices + 1 + kSliceDescPad + 1, kChkSliceCopy) &&
         RP_IN((int64_t)ch * kChunk + kStageInfo / 4, 0, sl.n_slices + kSliceDescPad + 1, kChkSliceCopy);
#else
  (void)sl, (void)d0, (void)d1, (void)ch, (void)db;
  return true;
#endif
}

// MP: several parts (slice rows from the per-slice records, non-local sums);
// instantiated separately so that the one-part body keeps its registers.
template <typename T, bool MP, class Epi>
__device__ __forceinline__ void spmv_sl_body(const Sliced<T> sl, const Parts<T>& parts, int64_t n64, const T* xin,
                                             T* yout, Epi& epi) {
  using St = SlStage<T>;
  constexpr int kStages = St::kStages;
  extern __shared__ __align__(128) unsigned char sbuf[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
  __shared__ uint32_t chunk_x[kStages], chunk_y[kStages];
  __shared__ int staged[kStages];
  __shared__ int timed_out, issued;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int S = (int)sl.n_slices, n = (int)n64;
  const int NC = (S + kChunk - 1) / kChunk, G = gridDim.x;
  const uint2* desc = sl.desc;

  if (tid == 0) {
    for (int st = 0; st < kStages; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], kChunk);
    }
    timed_out = 0;
    issued = 0;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  if (w == kChunk) {
    // producer warp: one lane posts every chunk of this block
    if (lane == 0) {
      uint2 nd0 = make_uint2(0u, 0u), nd1 = nd0;
      if ((int)blockIdx.x < NC) {
        nd0 = __ldg(desc + blockIdx.x * kChunk);
        nd1 = __ldg(desc + min((int)blockIdx.x * kChunk + kChunk, S));
      }
      int i = 0;
      for (int ch = blockIdx.x; ch < NC; ch += G, ++i) {
        const int st = i % kStages;
        if (i >= kStages && !mbar_wait(&empty[st], (uint32_t)((i / kStages - 1) & 1), sl.spin)) {
          atomicExch(&timed_out, 1);
          break;
        }
        const uint2 d0 = nd0, d1 = nd1;
        if (ch + G < NC) {  // bounds of the next chunk, loaded while this one is posted
          nd0 = __ldg(desc + (ch + G) * kChunk);
          nd1 = __ldg(desc + min((ch + G) * kChunk + kChunk, S));
        }
        unsigned char* base = sbuf + st * St::kBytes;
        const uint32_t vb = (d1.x - d0.x) * (uint32_t)sizeof(T), ib = (d1.y - d0.y) * 4u;
        const uint32_t db = 16u * (uint32_t)((kChunk + 2) / 2);  // kChunk + 1 descriptors, 16-byte multiple
        const bool fit = vb <= (uint32_t)St::kVals && ib <= (uint32_t)kStageIdx && chunk_copy_ok(sl, d0, d1, ch, db);
        chunk_x[st] = d0.x;
        chunk_y[st] = d0.y;
        staged[st] = fit;
        // consumers' generic-proxy reads of this stage (released through
        // empty[st]) before the async-proxy writes of the copy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (fit) {
          mbar_expect_tx(&full[st], vb + ib + db + kStageInfo);
          bulk_g2s(base, sl.vals + d0.x, vb, &full[st]);
          bulk_g2s(base + St::kVals, sl.ibuf + d0.y, ib, &full[st]);
          bulk_g2s(base + St::kVals + kStageIdx, desc + (int64_t)ch * kChunk, db, &full[st]);
          bulk_g2s(base + St::kVals + kStageIdx + kStageDesc, sl.tinfo + (int64_t)ch * kChunk, kStageInfo, &full[st]);
        } else {
          mbar_arrive(&full[st]);
        }
      }
      issued = i;
    }
  } else {
    int i = 0;
    for (int ch = blockIdx.x; ch < NC; ch += G, ++i) {
      const int st = i % kStages;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&full[st], (uint32_t)((i / kStages) & 1), sl.spin));
      if (!ok) {
        if (lane == 0) atomicExch(&timed_out, 1);
        break;
      }
      const int s = ch * kChunk + w;
      if (s < S) {
        SliceRows sr{s * kSliceRows, 0, 0};
        if constexpr (MP) sr = slice_rows(sl, s, n);
        const int row = sr.row0 + lane;
        const bool valid = MP ? lane < sr.rows : row < n;
        NlRange nl{0, 0};
        if constexpr (MP)
          if (valid) nl = nonlocal_range<T>(parts, sr.part, row);
        const T* x = xin + row;
        const SliceCk ck = slice_ck<T, MP>(sl, parts, sr.part, row, n);
        const unsigned char* base = sbuf + st * St::kBytes;
        T sum;
        if (staged[st]) {
          const uint2* sd = reinterpret_cast<const uint2*>(base + St::kVals + kStageIdx);
          const uint32_t* si = reinterpret_cast<const uint32_t*>(base + St::kVals + kStageIdx + kStageDesc);
          const uint2 d0 = sd[w], d1 = sd[w + 1];
          sum = slice_sum<T>(d0, d1, si[w], reinterpret_cast<const T*>(base) + (d0.x - chunk_x[st]) + lane,
                             reinterpret_cast<const uint32_t*>(base + St::kVals) + (d0.y - chunk_y[st]) + lane,
                             sl.tabs, x, valid, lane, ck);
        } else {
          const uint2 d0 = __ldg(desc + s), d1 = __ldg(desc + s + 1);
          sum = slice_sum<T>(d0, d1, __ldg(sl.tinfo + s), sl.vals + d0.x + lane,
                             reinterpret_cast<const uint32_t*>(sl.ibuf + d0.y) + lane, sl.tabs, x, valid, lane, ck);
        }
        if constexpr (MP) sum = nonlocal_sum<T>(parts, sr.part, nl, xin, sum);
        if (valid) {
          yout[row] = sum;
          epi.row(row, sum);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    }
  }
  __syncthreads();
  if (timed_out) {
    // wait (bounded) for the copies this block may still have in flight, then report
    if (tid == kChunk * 32) {
      for (int j = issued - kStages; j < issued; ++j)
        if (j >= 0) mbar_wait(&full[j % kStages], (uint32_t)((j / kStages) & 1), kDrainProbes);
      epi.timeout();
    }
    __syncthreads();
  }
  epi.finish();
}


// y = A x over CSR (any number of parts), grid-stride over rows; rows map
// to threads as in spmv_sl_body.
template <typename T, class Epi>
__device__ __forceinline__ void spmv_csr_body(int64_t n, const Parts<T>& parts, const int32_t* __restrict__ row_ptr,
                                              const int32_t* __restrict__ col, const T* __restrict__ vals,
                                              const T* xin, T* yout, Epi& epi) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T s = row_dot_any<T>(parts, row_ptr, col, vals, xin, i, n);
    yout[i] = s;
    epi.row(i, s);
  }
  epi.finish();
}

}  // namespace rp
