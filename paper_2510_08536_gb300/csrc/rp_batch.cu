// Batched form: many independent systems (each one CPU rank's LDU matrix,
// its own GPU part) updated and solved in ONE persistent launch.
//
// The grid is launched as thread-block clusters of T CTAs. A cluster is a
// team: its leader takes the next system from a work queue ordered by size
// (largest first), the team runs the value update and the whole Jacobi-PCG
// (FP64, or FP32-inner / FP64-outer refinement) of that system, writes the
// system's status, and takes the next one. Teams never wait on each other.
//
// Inside a team the rows of the system are split into T contiguous blocks
// (whole 32-row slices when the sliced layout is built: each CTA then writes
// its own slices' values in the update and its SpMV runs one warp per slice).
// The two reductions of each CG iteration go through distributed shared
// memory: every CTA publishes its partial sums in its own shared memory and,
// after a hardware cluster barrier, every CTA reads all T partials in rank
// order, so all CTAs hold bit-identical scalars and take identical control
// decisions (loop trip counts match, every barrier is reached by all).
// Three cluster barriers per iteration: after the p update (the SpMV reads
// neighbour rows of other CTAs) and one per reduction. Vectors written inside
// the kernel are read with plain (coherent) loads; the barriers carry
// release/acquire semantics at cluster scope. Every loop is capped by the
// iteration limits; there is no spin wait.
#include <cooperative_groups.h>

#include <algorithm>
#include <numeric>

#include "rp_common.cuh"
#include "rp_spmv.cuh"

namespace cg = cooperative_groups;

namespace rp {



namespace {

// Built for two CTAs of 512 threads an SM: 64 registers a thread (the kernel
// spills some). A build with 80 registers (two CTAs of 384, fewer spills, 24
// warps an SM) measured slower in every launch shape (continued refinement,
// 256 systems: 219-417 ms against 201 ms): warps in flight matter more here.
constexpr int kBatchMaxThreads = 512;

// Block-wide sum of NV values, then cluster-wide through DSMEM; every thread
// of every CTA returns the same totals.
template <int NV>
__device__ __forceinline__ void team_sum(double (&v)[NV], double (&tot)[NV], cg::cluster_group& cl,
                                         double (*spart)[kMaxPartials], double (*swarp)[32], int& parity) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double s = warp_sum(v[i]);
    if (lane == 0) swarp[i][wid] = s;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double s = lane < nw ? swarp[i][lane] : 0.0;
      s = warp_sum(s);
      if (lane == 0) spart[parity][i] = s;
    }
  }
  cl.sync();
  // lane r reads CTA r's partials (all T remote loads in flight at once), then
  // an xor butterfly over the warp: every step adds the same two operands in
  // both lanes of a pair (addition commutes exactly), so every thread of every
  // CTA ends with the same bits
  const unsigned T = cl.num_blocks();
#pragma unroll
  for (int i = 0; i < NV; ++i)
    tot[i] = warp_sum((unsigned)lane < T ? *cl.map_shared_rank(&spart[parity][i], (unsigned)lane) : 0.0);
  parity ^= 1;
}

// Index arrays are never written in the kernel (read-only path); values and
// vectors are written inside it and are read with coherent loads.
template <typename T>
__device__ __forceinline__ T row_dot_coherent(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                              const T* vals, const T* x, int64_t i, int64_t n) {
  const int s = __ldg(rp + i), e = __ldg(rp + i + 1);
  T sum = T(0);
  for (int j = s; j < e; ++j) {
    const int c = __ldg(col + j);
    if (RP_IN(c, 0, n, kChkGather)) sum = fma(vals[j], x[c], sum);
  }
  return sum;
}

// y_i = (A x)_i for rows [i0, i1) of this CTA, two independent rows per thread
// in flight (rows i and i + blockDim, so each warp stays coalesced); f(i, y_i,
// pre_i) consumes every result (pre: a vector the consumer reads at row i).
template <typename T, typename F>
__device__ __forceinline__ void spmv_rows(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                          const T* vals, const T* x, const T* pre, int64_t i0, int64_t i1,
                                          int64_t n, F&& f) {
  const int64_t nth = blockDim.x;
  int64_t i = i0 + threadIdx.x;
  for (; i + nth < i1; i += 2 * nth) {
    const int64_t k = i + nth;
    const int s0 = __ldg(rp + i), e0 = __ldg(rp + i + 1);
    const int s1 = __ldg(rp + k), e1 = __ldg(rp + k + 1);
    T a0 = T(0), a1 = T(0);
    const int m = max(e0 - s0, e1 - s1);
    for (int t = 0; t < m; ++t) {
      if (s0 + t < e0 && RP_IN(__ldg(col + s0 + t), 0, n, kChkGather))
        a0 = fma(vals[s0 + t], x[__ldg(col + s0 + t)], a0);
      if (s1 + t < e1 && RP_IN(__ldg(col + s1 + t), 0, n, kChkGather))
        a1 = fma(vals[s1 + t], x[__ldg(col + s1 + t)], a1);
    }
    f(i, a0, pre[i]);
    f(k, a1, pre[k]);
  }
  for (; i < i1; i += nth) f(i, row_dot_coherent<T>(rp, col, vals, x, i, n), pre[i]);
}

// Per-warp staging of one slice's values and index words (slices of up to
// kStageL entries per row): two buffers per warp in dynamic shared memory.
constexpr int kStageL = 8;
constexpr int kStageValBytes = kStageL * 32 * 8;      // FP64 values
constexpr int kStageIdxBytes = 2 * 32 * 4;            // 8-bit indices: 2 words per row
constexpr int kStageBuf = kStageValBytes + kStageIdxBytes;
constexpr int kWarpStage = 2 * kStageBuf;

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// The warp copies slice (d0, d1) into buf: values (a multiple of 32 entries,
// 128-byte aligned) at buf, index words (a multiple of 32) at buf + kStageValBytes.
// The slices of a team's matrix are read once an iteration and are too many to
// stay in L2 across the teams; copying them with an evict-first hint leaves L2 to
// the vectors, which every pass reads again (4.6% of the continued-refinement
// batch, 2.3% of FP64; the same hint in the single-system SpMV, whose vectors
// fit in L2 anyway, made it slower).
__device__ __forceinline__ void cp_async16_ef(void* dst, const void* src, uint64_t pol) {
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "l"(pol)
               : "memory");
}
template <typename T>
__device__ __forceinline__ void stage_slice(unsigned char* buf, const T* vals, const uint32_t* ibuf, uint2 d0,
                                            uint2 d1, int lane) {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  const uint32_t vb = (d1.x - d0.x) * (uint32_t)sizeof(T), ib = (d1.y - d0.y) * 4u;
  const unsigned char* vs = reinterpret_cast<const unsigned char*>(vals + d0.x);
  const unsigned char* is = reinterpret_cast<const unsigned char*>(ibuf + d0.y);
  for (uint32_t o = 16u * lane; o < vb; o += 512u) cp_async16_ef(buf + o, vs + o, pol);
  for (uint32_t o = 16u * lane; o < ib; o += 512u) cp_async16_ef(buf + kStageValBytes + o, is + o, pol);
}

// Slices of up to kStageL entries a row are staged; in the bounds-checked
// build also only when the copy's source ranges lie inside their arrays (an
// unstaged slice is read from global memory, where slice_sum checks it).
__device__ __forceinline__ bool stageable(uint2 d0, uint2 d1, const BatchArgs& a) {
#ifdef RP_CHECK
  if (!RP_IN(d1.x, d0.x, a.sl_entries + 1, kChkSliceCopy) || !RP_IN(d1.y, d0.y, a.sl_ibuf_len + 1, kChkSliceCopy) ||
      d1.y - d0.y > (uint32_t)(kStageIdxBytes / 4))
    return false;
#else
  (void)a;
#endif
  return d1.x - d0.x <= 32u * kStageL;
}

// y_i = (A x)_i for rows [i0, i1) (i0 a multiple of 32) on the sliced layout:
// one warp per slice, lanes on rows, the same fused multiply-adds in the same
// order as the CSR row sums. The warp's next slice is copied (cp.async, L2
// only) into its other staging buffer while the current one is summed, so the
// value and index loads of one slice overlap the gathers of the previous one;
// descriptors are loaded two slices ahead and, for FP32 values, the lane's
// table entry one slice ahead (it is on the path of every gather: 5% of the
// FP32 solves; the FP64 solve measured 1.3% slower with it). f(i, y_i, pre_i) consumes every
// result; pre_i (a vector the consumer reads at row i) is loaded before the
// slice's gathers, so its latency hides behind theirs. Values and x are written
// inside the kernel (the values before a block barrier, read back through L2;
// x and pre with plain loads); descriptors, tables and index words are read-only.
// U4: every slice has 4-bit indices and rows of at most kStageL entries (the
// layout's uniform flag): every slice is staged and summed by the 4-bit row
// sum directly, without the per-slice tests of the general case.
template <typename T, bool U4 = false, typename F>
__device__ __forceinline__ void spmv_slices(const BatchArgs& a, const T* vals, int64_t s0, const T* x, const T* pre,
                                            int64_t i0, int64_t i1, int64_t n, unsigned char* stage, F&& f) {
  if (i0 >= i1) return;  // i0 = n need not be a multiple of 32
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t nw = blockDim.x >> 5, end = (i1 + 31) >> 5;
  int64_t ls = (i0 >> 5) + wid;
  if (ls >= end) return;
  unsigned char* wbuf = stage + wid * kWarpStage;
  const uint2* desc = a.sl_desc + s0;
  const uint32_t* tinfo = a.sl_tinfo + s0;
  uint2 d0 = __ldg(desc + ls), d1 = __ldg(desc + ls + 1);
  uint32_t info = __ldg(tinfo + ls);
  uint2 n0 = d1, n1 = d1;
  uint32_t ninfo = 0u;
  if (ls + nw < end) {
    n0 = __ldg(desc + ls + nw);
    n1 = __ldg(desc + ls + nw + 1);
    ninfo = __ldg(tinfo + ls + nw);
  }
  if (U4 || stageable(d0, d1, a)) stage_slice<T>(wbuf, vals, a.sl_ibuf, d0, d1, lane);
  cp_async_commit();
  constexpr bool kTabAhead = sizeof(T) == 4;
  int32_t tv = kTabAhead ? slice_tab_entry(info, a.sl_tabs, lane, a.sl_tabs_len) : 0;  // this slice's table entry
  int b = 0;
  for (;;) {
    const bool more = ls + nw < end;
    // the next slice's copy goes out before this one is summed
    if (more && (U4 || stageable(n0, n1, a))) stage_slice<T>(wbuf + (b ^ 1) * kStageBuf, vals, a.sl_ibuf, n0, n1, lane);
    cp_async_commit();
    const int64_t lm = ls + 2 * nw;
    uint2 m0 = n1, m1 = n1;
    uint32_t minfo = 0u;
    if (lm < end) {
      m0 = __ldg(desc + lm);
      m1 = __ldg(desc + lm + 1);
      minfo = __ldg(tinfo + lm);
    }
    // the next slice's table entry, loaded while this slice is summed
    const int32_t ntv = kTabAhead && more ? slice_tab_entry(ninfo, a.sl_tabs, lane, a.sl_tabs_len) : 0;
    cp_async_wait<1>();  // this slice's copies (all but the group just issued)
    __syncwarp();
    const int64_t row = (ls << 5) + lane;
    const bool valid = row < i1;
    const T prow = valid ? pre[row] : T(0);
#ifdef RP_CHECK
    const SliceCk ck{(int)(-row), (int)(n - row), a.sl_entries, a.sl_ibuf_len, a.sl_tabs_len};
#else
    const SliceCk ck{};
    (void)n;
#endif
    // (two calls, not one with selected pointers: the staged call must read
    // through shared-memory pointers, a generic pointer made the solves slower)
    auto sum_of = [&](const T* sv, const uint32_t* si) {
      if constexpr (kTabAhead) return slice_sum_tv<T, true>(d0, d1, info, tv, sv, si, a.sl_tabs, x + row, valid, ck);
      else return slice_sum<T, true>(d0, d1, info, sv, si, a.sl_tabs, x + row, valid, lane, ck);
    };
    T sum;
    if constexpr (U4) {
      const unsigned char* cur = wbuf + b * kStageBuf;
      const int32_t* tab = a.sl_tabs + (info & ~kSliceW4);
      sum = slice_row<T, kIdx4, true>(reinterpret_cast<const T*>(cur) + lane,
                                      reinterpret_cast<const uint32_t*>(cur + kStageValBytes) + lane,
                                      kTabAhead ? tv : __ldg(tab + (lane & 15)), tab, x + row, valid,
                                      (int)((d1.x - d0.x) >> 5), 0, ck);
    } else if (stageable(d0, d1, a)) {
      const unsigned char* cur = wbuf + b * kStageBuf;
      sum = sum_of(reinterpret_cast<const T*>(cur) + lane, reinterpret_cast<const uint32_t*>(cur + kStageValBytes) + lane);
    } else {
      sum = sum_of(vals + d0.x + lane, a.sl_ibuf + d0.y + lane);
    }
    if (valid) f(row, sum, prow);
    __syncwarp();  // buffer b is read by every lane before it is refilled
    if (!more) break;
    ls += nw;
    b ^= 1;
    tv = ntv;
    d0 = n0;
    d1 = n1;
    info = ninfo;
    n0 = m0;
    n1 = m1;
    ninfo = minfo;
  }
  cp_async_wait<0>();
}

// Base pointers of the NOP operand vectors of a vector pass, as 16-byte vectors.
template <int NOP>
struct VecOps {
  const uint4* p[NOP];
  unsigned first = 0;  // bit j: operand j is not read again soon (L2 evict-first), else evict-last
};
__device__ __forceinline__ const uint4* vec16(const void* p) { return reinterpret_cast<const uint4*>(p); }
__device__ __forceinline__ float4 as_f4(uint4 u) {
  return make_float4(__uint_as_float(u.x), __uint_as_float(u.y), __uint_as_float(u.z), __uint_as_float(u.w));
}
__device__ __forceinline__ double2 as_d2(uint4 u) {
  return make_double2(__hiloint2double((int)u.y, (int)u.x), __hiloint2double((int)u.w, (int)u.z));
}

// Visit rows [i0, i1) of a system whose first row has global index ro: for
// every W-wide vector v (global vector index, 16-byte aligned) inside the range
// st(v, s, k) with operand j of v at s[j k] (NOP operands from ops), fs(i) for the
// ragged rows at either end. STAGED (the sliced layout's per-warp staging area,
// free between SpMVs): every lane copies the operands of its next vector into
// its own slots with cp.async (L2, coherent after the cluster barriers) while
// it computes the current one from shared memory, so two vectors' loads are in
// flight without holding either in registers (each lane reads only what it
// copied: no warp barrier). Otherwise the operands are loaded straight into
// registers, one vector a trip.
template <int W, int NOP, bool STAGED, typename FS, typename FT>
__device__ __forceinline__ void rows_vec(int64_t ro, int64_t i0, int64_t i1, const VecOps<NOP>& ops,
                                         unsigned char* stage, FS&& fs, FT&& st) {
  static_assert(2 * NOP * 32 * 16 <= kWarpStage, "operand slots exceed the warp's staging area");
  const int64_t nth = blockDim.x, tid = threadIdx.x;
  const int64_t g0 = ro + i0, g1 = ro + i1;
  const int64_t v0 = (g0 + W - 1) / W, v1 = g1 / W;
  if (v0 >= v1) {
    for (int64_t i = i0 + tid; i < i1; i += nth) fs(i);
    return;
  }
  for (int64_t g = g0 + tid; g < v0 * W; g += nth) fs(g - ro);
  if constexpr (STAGED) {
    // D vectors in flight a lane: three where the slots fit, else two
    constexpr int D = 3 * NOP * 32 * 16 <= kWarpStage ? 3 : 2;
    uint4* slot = reinterpret_cast<uint4*>(stage + (tid >> 5) * kWarpStage) + (tid & 31);  // [buffer][operand][lane]
    uint64_t pol_last, pol_first;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol_last));
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol_first));
    auto issue = [&](int64_t v, int b) {
#pragma unroll
      for (int j = 0; j < NOP; ++j)
        cp_async16_ef(slot + (b * NOP + j) * 32, ops.p[j] + v, (ops.first >> j) & 1u ? pol_first : pol_last);
    };
    int64_t v = v0 + tid;
#pragma unroll
    for (int j = 0; j < D - 1; ++j) {
      if (v + j * nth < v1) issue(v + j * nth, j);
      cp_async_commit();
    }
    int b = 0;
    for (; v < v1; v += nth) {
      // into the buffer the previous trip read (its values are already used)
      if (v + (D - 1) * nth < v1) issue(v + (D - 1) * nth, b == 0 ? D - 1 : b - 1);
      cp_async_commit();
      cp_async_wait<D - 1>();  // this vector's copies
      st(v, slot + b * NOP * 32, 32);
      b = b + 1 == D ? 0 : b + 1;
    }
    cp_async_wait<0>();
  } else {
    (void)stage;
    for (int64_t v = v0 + tid; v < v1; v += nth) {
      uint4 o[NOP];
#pragma unroll
      for (int j = 0; j < NOP; ++j) o[j] = ops.p[j][v];
      st(v, o, 1);
    }
  }
  for (int64_t g = v1 * W + tid; g < g1; g += nth) fs(g - ro);
}

}  // namespace

// MODE: 0 FP64 PCG, 1 mixed (restarted inner PCG), 2 mixed with continued inner PCG;
// SL: the SpMV and residual passes run on the sliced layout
template <int MODE, bool SL, bool U4 = false>
__global__ void __launch_bounds__(kBatchMaxThreads, 2) k_batch(BatchArgs a) {
  constexpr bool MIXED = MODE != 0;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned T = cl.num_blocks();
  const unsigned me = cl.block_rank();
  __shared__ double spart[2][kMaxPartials];
  __shared__ double swarp[kMaxPartials][32];
  __shared__ int s_next;
  extern __shared__ __align__(128) unsigned char stage[];  // SL: kWarpStage per warp
  int parity = 0;
  const double tol = a.io->tol;
  const double* __restrict__ bufall = a.io->buf;
  const double* __restrict__ ball = a.io->b;
  double* __restrict__ xall = a.io->x;
  const bool xvec = (reinterpret_cast<uintptr_t>(xall) & 15) == 0;  // caller's x: vectorise only if aligned

  for (;;) {
    if (me == 0 && threadIdx.x == 0) s_next = (int)atomicAdd(a.queue, 1u);
    cl.sync();
    const int k = *cl.map_shared_rank(&s_next, 0);
    cl.sync();
    if (k >= a.n_sys) break;
    const int s = a.order[k];
    const int64_t ro = a.row_off[s];
    const int64_t n = a.row_off[s + 1] - ro;
    const int32_t* __restrict__ rp = a.row_ptr + ro + s;
    const int64_t no = a.nnz_off[s];
    const int32_t* __restrict__ col = a.col + no;
    const int32_t* __restrict__ src = a.src_of + no;
    const double* __restrict__ buf = bufall + a.buf_off[s];
    double* vals = a.vals + no;
    float* vals32 = MIXED ? a.vals32 + no : nullptr;
    double* dinv = a.dinv + ro;
    float* dinv32 = MIXED ? a.dinv32 + ro : nullptr;
    // mixed on the sliced layout: the inner iteration runs on S A S (Jacobi made
    // explicit, unit diagonal: no diagonal reads in the FP32 vector passes)
    constexpr bool SCALED = MIXED && SL;
    double* s64 = SCALED ? a.s64 + ro : nullptr;
    const double* b = ball + ro;
    double* x = xall + ro;
    constexpr bool sl = SL;
    const int64_t s0 = sl ? a.sl_soff[s] : 0;
    int64_t chunk = (n + T - 1) / T;
    if (sl) chunk = (chunk + 31) & ~int64_t(31);
    const int64_t i0 = min((int64_t)me * chunk, n), i1 = min(i0 + chunk, n);
    const int tid = threadIdx.x, nth = blockDim.x;
    // A x for rows [i0, i1) of this CTA, f(i, (A x)_i) for each
    auto spmv64 = [&](const double* xv, const double* pre, auto&& f) {
      if (sl) spmv_slices<double, U4>(a, a.sl_vals, s0, xv, pre, i0, i1, n, stage, f);
      else
        for (int64_t i = i0 + tid; i < i1; i += nth) f(i, row_dot_coherent<double>(rp, col, vals, xv, i, n), pre[i]);
    };

    // value update of this CTA's rows (Sec. 3 update procedure) and the Jacobi diagonal
    const int64_t blen = a.buf_off[s + 1] - a.buf_off[s];
    (void)blen;  // bounds of the update's slots (bounds-checked build)
    for (int64_t pp = rp[i0] + tid; pp < rp[i1]; pp += nth) {
      const double v = RP_IN(src[pp], 0, blen, kChkPermute) ? buf[src[pp]] : 0.0;
      vals[pp] = v;
      if (MIXED) vals32[pp] = (float)v;
    }
    for (int64_t i = i0 + tid; i < i1; i += nth) {
      const double d = buf[i];  // diagonal block leads the system's buffer
      dinv[i] = 1.0 / d;
      if (MIXED) dinv32[i] = 1.0f / (float)d;
      if (SCALED) s64[i] = 1.0 / sqrt(d);
    }
    if constexpr (SCALED) {
      cl.sync();  // s of every row of the system before the scaled values use it
      // this CTA's slices, one warp per slice: FP64 values from the buffer and the
      // FP32 values of S A S, fl32(a_ij (s_i s_j)) (products in FP64); padding 0
      const int lane = tid & 31;
      const int64_t nw = nth >> 5, ls1 = (i1 + 31) >> 5;
      for (int64_t ls = (i0 >> 5) + (tid >> 5); i0 < i1 && ls < ls1; ls += nw) {
        const uint2 d0 = __ldg(a.sl_desc + s0 + ls), d1 = __ldg(a.sl_desc + s0 + ls + 1);
        const int64_t i = (ls << 5) + lane;
        const double si = i < n ? s64[i] : 0.0;
        for (uint32_t e = d0.x + lane; e < d1.x; e += 32) {
          const int32_t pp = __ldg(a.sl_pos + e);
          double v = 0.0;
          float v32 = 0.0f;
          if (pp >= 0 && RP_IN(pp, 0, a.nnz_off[a.n_sys], kChkSliceValues) &&
              RP_IN(__ldg(a.src_of + pp), 0, blen, kChkPermute)) {
            v = buf[__ldg(a.src_of + pp)];
            const int32_t j = __ldg(a.col + pp);
            if (RP_IN(j, 0, n, kChkGather)) v32 = (float)(v * (si * s64[j]));
          }
          a.sl_vals[e] = v;
          a.sl_vals32[e] = v32;
        }
      }
    } else if (sl && i0 < i1) {
      // this CTA's slices, padding included (zero values)
      const int64_t e0 = __ldg(a.sl_desc + s0 + (i0 >> 5)).x, e1 = __ldg(a.sl_desc + s0 + ((i1 + 31) >> 5)).x;
      for (int64_t e = e0 + tid; e < e1; e += nth) {
        const int32_t pp = __ldg(a.sl_pos + e);
        const bool in = pp >= 0 && RP_IN(pp, 0, a.nnz_off[a.n_sys], kChkSliceValues) &&
                        RP_IN(__ldg(a.src_of + pp), 0, blen, kChkPermute);
        const double v = in ? buf[__ldg(a.src_of + pp)] : 0.0;
        a.sl_vals[e] = v;
        if (MIXED) a.sl_vals32[e] = (float)v;
      }
    }
    __syncthreads();

    int status = -1, iters = 0, passes = 0, restarts = 0, outer = 0;
    double bb = 0.0, thresh = 0.0, rr = 0.0;

    if (!MIXED) {
      double* r = a.r + ro;
      double* p = a.p + ro;
      double* q = a.q + ro;
      double rz = 0.0;
      for (;;) {
        // residual pass: r = b - A x (x = 0 on the first pass), p = z = D^-1 r
        double v3[3] = {0.0, 0.0, 0.0}, t3[3];
        auto res_row = [&](int64_t i, double ri) {
          r[i] = ri;
          const double zi = dinv[i] * ri;
          p[i] = zi;
          v3[0] = fma(ri, zi, v3[0]);
          v3[1] = fma(ri, ri, v3[1]);
        };
        if (passes == 0) {
          for (int64_t i = i0 + tid; i < i1; i += nth) {
            const double ri = b[i];
            x[i] = 0.0;
            v3[2] = fma(ri, ri, v3[2]);
            res_row(i, ri);
          }
        } else {
          spmv64(x, b, [&](int64_t i, double axi, double bi) { res_row(i, bi - axi); });
        }
        team_sum<3>(v3, t3, cl, spart, swarp, parity);
        if (passes == 0) {
          bb = t3[2];
          thresh = tol * tol * bb;
        }
        rz = t3[0];
        rr = t3[1];
        const bool first = passes == 0;
        ++passes;
        if (rr <= thresh) { status = RP_OK; break; }
        if (status == RP_BREAKDOWN) break;
        if (!isfinite(rr)) { status = RP_BREAKDOWN; break; }
        if (iters >= a.max_iter || (!first && restarts >= a.max_restarts)) { status = RP_NOT_CONVERGED; break; }
        if (!first) ++restarts;
        // CG iterations
        for (;;) {
          cl.sync();  // p of every row visible to the team
          double v1[1] = {0.0}, t1[1];
          auto qrow = [&](int64_t i, double qi, double pi) {
            q[i] = qi;
            v1[0] = fma(pi, qi, v1[0]);
          };
          if (sl) spmv_slices<double, U4>(a, a.sl_vals, s0, p, p, i0, i1, n, stage, qrow);
          else spmv_rows<double>(rp, col, vals, p, p, i0, i1, n, qrow);
          team_sum<1>(v1, t1, cl, spart, swarp, parity);
          if (!(t1[0] > 0.0) || !isfinite(t1[0])) { status = RP_BREAKDOWN; break; }
          const double alpha = rz / t1[0];
          double v2[2] = {0.0, 0.0}, t2[2];
          rows_vec<2, 3, SL>(
              ro, i0, i1, VecOps<3>{{vec16(a.q), vec16(a.r), vec16(a.dinv)}}, stage,
              [&](int64_t i) {
                const double ri = fma(-alpha, q[i], r[i]);
                r[i] = ri;
                v2[0] = fma(ri, dinv[i] * ri, v2[0]);
                v2[1] = fma(ri, ri, v2[1]);
              },
              [&](int64_t v, const uint4* o, int k) {
                const double2 qv = as_d2(o[0]), dv = as_d2(o[2 * k]);
                double2 rv = as_d2(o[k]);
                rv.x = fma(-alpha, qv.x, rv.x);
                rv.y = fma(-alpha, qv.y, rv.y);
                reinterpret_cast<double2*>(a.r)[v] = rv;
                v2[0] = fma(rv.x, dv.x * rv.x, v2[0]);
                v2[0] = fma(rv.y, dv.y * rv.y, v2[0]);
                v2[1] = fma(rv.x, rv.x, v2[1]);
                v2[1] = fma(rv.y, rv.y, v2[1]);
              });
          team_sum<2>(v2, t2, cl, spart, swarp, parity);
          ++iters;
          rr = t2[1];
          bool stop = false;
          double beta = 0.0;
          if (t2[1] <= thresh || iters >= a.max_iter) stop = true;
          else if (!(t2[0] > 0.0) || !isfinite(t2[0])) { stop = true; status = RP_BREAKDOWN; }
          else { beta = t2[0] / rz; rz = t2[0]; }
          auto upd = [&](int64_t i) {
            const double pi = p[i];
            x[i] = fma(alpha, pi, x[i]);
            if (!stop) p[i] = fma(beta, pi, dinv[i] * r[i]);
          };
          if (xvec) {
            rows_vec<2, 4, SL>(
                ro, i0, i1, VecOps<4>{{vec16(a.p), vec16(xall), vec16(a.r), vec16(a.dinv)}}, stage, upd,
                [&](int64_t v, const uint4* o, int k) {
                  double2 pv = as_d2(o[0]), xv = as_d2(o[k]);
                  xv.x = fma(alpha, pv.x, xv.x);
                  xv.y = fma(alpha, pv.y, xv.y);
                  reinterpret_cast<double2*>(xall)[v] = xv;
                  if (!stop) {
                    const double2 rv = as_d2(o[2 * k]), dv = as_d2(o[3 * k]);
                    pv.x = fma(beta, pv.x, dv.x * rv.x);
                    pv.y = fma(beta, pv.y, dv.y * rv.y);
                    reinterpret_cast<double2*>(a.p)[v] = pv;
                  }
                });
          } else {
            for (int64_t i = i0 + tid; i < i1; i += nth) upd(i);
          }
          if (stop) break;
        }
        cl.sync();  // x of every row visible before the residual pass
      }
    } else {
      float* r = a.r32 + ro;
      float* p = a.p32 + ro;
      float* q = a.q32 + ro;
      float* d = a.d32 + ro;
      constexpr bool RU = MODE == 2;
      double rz = 0.0;  // continued refinement carries (r, z) across passes
      for (;;) {
        // FP64 residual pass with FP64 values; FP32 copy starts the inner solve
        double v4[4] = {0.0, 0.0, 0.0, 0.0}, t4[4];
        float rzf = 0.f, rr32f = 0.f;
        auto res_row = [&](int64_t i, double ri) {
          const float r32 = SCALED ? (float)(s64[i] * ri) : (float)ri;
          r[i] = r32;
          d[i] = 0.f;
          const float z32 = SCALED ? r32 : dinv32[i] * r32;
          if (!RU || passes == 0) p[i] = z32;
          rzf = fmaf(r32, z32, rzf);
          rr32f = fmaf(r32, r32, rr32f);
          v4[1] = fma(ri, ri, v4[1]);
        };
        if (passes == 0) {
          for (int64_t i = i0 + tid; i < i1; i += nth) {
            const double ri = b[i];
            x[i] = 0.0;
            v4[2] = fma(ri, ri, v4[2]);
            res_row(i, ri);
          }
        } else {
          spmv64(x, b, [&](int64_t i, double axi, double bi) { res_row(i, bi - axi); });
        }
        v4[0] = rzf;
        v4[3] = rr32f;
        team_sum<4>(v4, t4, cl, spart, swarp, parity);
        if (passes == 0) {
          bb = t4[2];
          thresh = tol * tol * bb;
        }
        rr = t4[1];
        const bool first = passes == 0;
        ++passes;
        if (rr <= thresh) { status = RP_OK; break; }
        if (status == RP_BREAKDOWN) break;
        if (!isfinite(rr)) { status = RP_BREAKDOWN; break; }
        if (outer >= a.max_outer || (RU && iters >= a.max_iter)) { status = RP_NOT_CONVERGED; break; }
        ++outer;
        if (RU && !first) {
          // the FP64 residual replaced the FP32 one: continue the search direction
          const float beta = (float)(t4[0] / rz);
          for (int64_t i = i0 + tid; i < i1; i += nth) p[i] = fmaf(beta, p[i], SCALED ? r[i] : dinv32[i] * r[i]);
        }
        rz = t4[0];
        // a reduction by ru_delta (inner_tol), or half the outer target in the inner
        // residual's norm (scaled: carried over by the ratio of the two residuals)
        const double ithresh = fmax((RU ? a.ru_delta * a.ru_delta : a.inner_tol * a.inner_tol) * t4[3],
                                    0.25 * thresh * (SCALED ? t4[3] / t4[1] : 1.0));
        int it = 0;
        bool broke = false;
        for (;;) {
          cl.sync();
          float acc = 0.f;
          auto qrow = [&](int64_t i, float qi, float pi) {
            q[i] = qi;
            acc = fmaf(pi, qi, acc);
          };
          if (sl) spmv_slices<float, U4>(a, a.sl_vals32, s0, p, p, i0, i1, n, stage, qrow);
          else spmv_rows<float>(rp, col, vals32, p, p, i0, i1, n, qrow);
          double v1[1] = {(double)acc}, t1[1];
          team_sum<1>(v1, t1, cl, spart, swarp, parity);
          if (!(t1[0] > 0.0) || !isfinite(t1[0])) { status = RP_BREAKDOWN; broke = true; break; }
          const float alpha = (float)(rz / t1[0]);
          float a0 = 0.f, a1 = 0.f;
          auto rstep = [&](float& rv, float qv, float dv) {
            rv = fmaf(-alpha, qv, rv);
            if (!SCALED) a0 = fmaf(rv, dv * rv, a0);
            a1 = fmaf(rv, rv, a1);
          };
          VecOps<SCALED ? 2 : 3> rops;
          rops.p[0] = vec16(a.q32);
          rops.p[1] = vec16(a.r32);
          rops.first = 1u;  // q
          if constexpr (!SCALED) rops.p[2] = vec16(a.dinv32);
          rows_vec<4, SCALED ? 2 : 3, SL>(
              ro, i0, i1, rops, stage,
              [&](int64_t i) {
                float ri = r[i];
                rstep(ri, q[i], SCALED ? 1.0f : dinv32[i]);
                r[i] = ri;
              },
              [&](int64_t v, const uint4* o, int k) {
                const float4 qv = as_f4(o[0]);
                const float4 dv = SCALED ? make_float4(1.f, 1.f, 1.f, 1.f) : as_f4(o[(SCALED ? 0 : 2) * k]);
                float4 rv = as_f4(o[k]);
                rstep(rv.x, qv.x, dv.x);
                rstep(rv.y, qv.y, dv.y);
                rstep(rv.z, qv.z, dv.z);
                rstep(rv.w, qv.w, dv.w);
                reinterpret_cast<float4*>(a.r32)[v] = rv;
              });
          if (SCALED) a0 = a1;  // z = r: (r, z) = (r, r)
          double v2[2] = {(double)a0, (double)a1}, t2[2];
          team_sum<2>(v2, t2, cl, spart, swarp, parity);
          ++it;
          ++iters;
          bool stop = false;
          float beta = 0.f;
          if (t2[1] <= ithresh || (RU ? iters : it) >= a.max_iter) stop = true;
          else if (!(t2[0] > 0.0) || !isfinite(t2[0])) { stop = true; status = RP_BREAKDOWN; broke = true; }
          else { beta = (float)(t2[0] / rz); rz = t2[0]; }
          VecOps<SCALED ? 3 : 4> xops;
          xops.p[0] = vec16(a.p32);
          xops.p[1] = vec16(a.d32);
          xops.p[2] = vec16(a.r32);
          xops.first = 2u | 4u;  // d, r
          if constexpr (!SCALED) xops.p[3] = vec16(a.dinv32);
          rows_vec<4, SCALED ? 3 : 4, SL>(
              ro, i0, i1, xops, stage,
              [&](int64_t i) {
                const float pi = p[i];
                d[i] = fmaf(alpha, pi, d[i]);
                if (!stop) p[i] = fmaf(beta, pi, SCALED ? r[i] : dinv32[i] * r[i]);
              },
              [&](int64_t v, const uint4* o, int k) {
                float4 pv = as_f4(o[0]);
                float4 dd = as_f4(o[k]);
                dd.x = fmaf(alpha, pv.x, dd.x);
                dd.y = fmaf(alpha, pv.y, dd.y);
                dd.z = fmaf(alpha, pv.z, dd.z);
                dd.w = fmaf(alpha, pv.w, dd.w);
                reinterpret_cast<float4*>(a.d32)[v] = dd;
                if (!stop) {
                  const float4 rv = as_f4(o[2 * k]);
                  const float4 iv = SCALED ? make_float4(1.f, 1.f, 1.f, 1.f) : as_f4(o[(SCALED ? 0 : 3) * k]);
                  pv.x = fmaf(beta, pv.x, iv.x * rv.x);
                  pv.y = fmaf(beta, pv.y, iv.y * rv.y);
                  pv.z = fmaf(beta, pv.z, iv.z * rv.z);
                  pv.w = fmaf(beta, pv.w, iv.w * rv.w);
                  reinterpret_cast<float4*>(a.p32)[v] = pv;
                }
              });
          if (stop) break;
        }
        // d was written with the vector mapping of rows_vec; the correction reads it
        // row by row, so every thread of the CTA must have finished its writes
        __syncthreads();
        if (!broke) {
          for (int64_t i = i0 + tid; i < i1; i += nth) x[i] += SCALED ? s64[i] * (double)d[i] : (double)d[i];
        }
        cl.sync();  // x visible before the next residual pass
      }
    }
    if (me == 0 && threadIdx.x == 0) {
      rp_solve_info inf;
      inf.status = status < 0 ? RP_NOT_CONVERGED : status;
      inf.iterations = iters;
      inf.outer_iterations = outer;
      inf.restarts = restarts;
      inf.passes = passes;
      inf.rel_residual = bb > 0.0 ? sqrt(rr / bb) : 0.0;
      a.info[s] = inf;
    }
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

__global__ void k_batch_setup(BatchIO* io, const double* buf, const double* b, double* x, double tol) {
  io->buf = buf;
  io->b = b;
  io->x = x;
  io->tol = tol;
}

namespace {

template <typename T>
rp_status balloc(T** p, int64_t count) {
  if (*p) return RP_OK;
  if (count <= 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, (size_t)count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(RP_ENOMEM, "cudaMalloc of %lld bytes failed", (long long)(count * sizeof(T)));
  }
  return RP_OK;
}

// the uniform-slice instances (never in the bounds-checked build, which checks every slice)
#ifdef RP_CHECK
constexpr bool kBatchU4 = false;
#else
constexpr bool kBatchU4 = true;
#endif
void* batch_kernel(int mode, bool sl, bool u4) {
  if (sl && u4 && kBatchU4)
    return mode == 2 ? (void*)k_batch<2, true, true> : mode == 1 ? (void*)k_batch<1, true, true>
                                                                 : (void*)k_batch<0, true, true>;
  if (sl) return mode == 2 ? (void*)k_batch<2, true> : mode == 1 ? (void*)k_batch<1, true> : (void*)k_batch<0, true>;
  return mode == 2 ? (void*)k_batch<2, false> : mode == 1 ? (void*)k_batch<1, false> : (void*)k_batch<0, false>;
}

rp_status launch_config(rp_handle* h, int mode, int cluster, int threads, cudaLaunchConfig_t* cfg,
                        cudaLaunchAttribute* attr, int* n_clusters) {
  const bool sl = h->batch_args.sl_desc != nullptr;
  void* fn = batch_kernel(mode, sl, h->sl_u4 != 0);
  if (cluster > 8) RP_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  const int smem = sl ? (threads / 32) * kWarpStage : 0;
  RP_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  *cfg = cudaLaunchConfig_t{};
  cfg->blockDim = dim3((unsigned)threads);
  cfg->gridDim = dim3((unsigned)cluster);
  cfg->dynamicSmemBytes = (size_t)smem;
  attr->id = cudaLaunchAttributeClusterDimension;
  attr->val.clusterDim.x = (unsigned)cluster;
  attr->val.clusterDim.y = 1;
  attr->val.clusterDim.z = 1;
  cfg->attrs = attr;
  cfg->numAttrs = 1;
  int nc = 0;
  RP_TRY_CUDA(cudaOccupancyMaxActiveClusters(&nc, fn, cfg));
  if (nc < 1) return fail(RP_EUNSUPPORTED, "cluster size %d with %d threads cannot be scheduled", cluster, threads);
  *n_clusters = nc;
  cfg->gridDim = dim3((unsigned)(nc * cluster));
  return RP_OK;
}

rp_status build_batch_graph(rp_handle* h, int mode, int cluster, int threads, cudaGraphExec_t* exec) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr;
  int nc = 0;
  RP_TRY(launch_config(h, mode, cluster, threads, &cfg, &attr, &nc));
  cudaStream_t cs;
  RP_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cfg.stream = cs;
  BatchArgs ba = h->batch_args;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaMemsetAsync(h->batch_queue, 0, sizeof(unsigned int), cs);
    void* args[] = {&ba};
    cudaLaunchKernelExC(&cfg, batch_kernel(mode, ba.sl_desc != nullptr, h->sl_u4 != 0), args);
    e = cudaStreamEndCapture(cs, &g);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(RP_ECUDA, "building the batch graph failed: %s", cudaGetErrorString(e));
  }
  return RP_OK;
}

}  // namespace

rp_status batch_prepare(rp_handle* h) {
  if (h->batch_ready) return RP_OK;
  if (h->n_parts != h->k) return fail(RP_EINVAL, "batched solves need one system per part (n_parts == k)");
  if (h->nl_nnz != 0) return fail(RP_EINVAL, "batched systems must be independent (no processor interfaces)");
  const int ns = h->n_parts;
  if (h->sl_slices == 0) RP_TRY(build_sliced(h, 0));  // every system sliced (when all fit)
  std::vector<int32_t> order(ns);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return h->part_nnz_off[a + 1] - h->part_nnz_off[a] > h->part_nnz_off[b + 1] - h->part_nnz_off[b];
  });
  int32_t* d_order = nullptr;
  int64_t *d_ro = nullptr, *d_no = nullptr, *d_bo = nullptr;
  RP_TRY(balloc(&d_order, ns));
  RP_TRY(balloc(&d_ro, ns + 1));
  RP_TRY(balloc(&d_no, ns + 1));
  RP_TRY(balloc(&d_bo, ns + 1));
  h->batch_order = d_order;
  h->batch_row_off = d_ro;
  h->batch_nnz_off = d_no;
  h->batch_buf_off = d_bo;
  RP_TRY_CUDA(cudaMemcpy(d_order, order.data(), 4 * ns, cudaMemcpyHostToDevice));
  RP_TRY_CUDA(cudaMemcpy(d_ro, h->part_row_off.data(), 8 * (ns + 1), cudaMemcpyHostToDevice));
  RP_TRY_CUDA(cudaMemcpy(d_no, h->part_nnz_off.data(), 8 * (ns + 1), cudaMemcpyHostToDevice));
  RP_TRY_CUDA(cudaMemcpy(d_bo, h->part_buf_off.data(), 8 * (ns + 1), cudaMemcpyHostToDevice));
  RP_TRY(balloc(&h->batch_queue, 4));
  RP_TRY(balloc(&h->batch_info, ns));
  RP_TRY(balloc(&h->batch_io, 1));
  BatchArgs& a = h->batch_args;
  a.n_sys = ns;
  a.order = d_order;
  a.row_off = d_ro;
  a.nnz_off = d_no;
  a.buf_off = d_bo;
  a.row_ptr = h->row_ptr;
  a.col = h->col_idx;
  a.src_of = h->src_of;
  a.vals = h->vals;
  a.vals32 = h->vals32;
  a.dinv = h->dinv;
  a.dinv32 = h->dinv32;
  a.r = h->r;
  a.p = h->p;
  a.q = h->q;
  a.r32 = h->r32;
  a.p32 = h->p32;
  a.q32 = h->q32;
  a.d32 = h->d32;
  a.queue = h->batch_queue;
  a.info = h->batch_info;
  a.io = h->batch_io;
  a.max_iter = h->opts.max_iter;
  a.max_restarts = h->opts.max_restarts;
  a.max_outer = h->opts.max_outer;
  a.inner_tol = h->opts.inner_tol;
  a.ru_delta = h->opts.ru_delta > 0.0 ? h->opts.ru_delta : h->opts.inner_tol;
  const bool sl = h->sl_slices > 0;
  a.sl_soff = sl ? h->sl_part_soff : nullptr;
  a.sl_desc = sl ? h->sl_desc : nullptr;
  a.sl_tinfo = sl ? h->sl_tinfo : nullptr;
  a.sl_tabs = sl ? h->sl_tabs : nullptr;
  a.sl_ibuf = sl ? reinterpret_cast<const uint32_t*>(h->sl_ibuf) : nullptr;
  a.sl_pos = sl ? h->sl_pos : nullptr;
  a.sl_vals = sl ? h->sl_vals : nullptr;
  a.sl_vals32 = sl ? h->sl_vals32 : nullptr;
  if (sl && h->want_fp32) RP_TRY(balloc(&h->batch_s64, h->n + 64));
  a.s64 = h->batch_s64;
  a.sl_entries = h->sl_entries;
  a.sl_ibuf_len = h->sl_ibuf_len;
  a.sl_tabs_len = h->sl_tabs_len;
  h->batch_ready = true;
  return RP_OK;
}

RP_CHECK_TU(batch)

void free_batch(rp_handle* h) {
  void* ptrs[] = {h->batch_order, h->batch_row_off, h->batch_nnz_off, h->batch_buf_off, h->batch_queue,
                  h->batch_info, h->batch_io, h->batch_s64};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (auto& g : h->batch_graphs)
    if (g) cudaGraphExecDestroy(g);
}

static rp_status batch_run(rp_handle* h, const double* buffer, int32_t where, const double* b, double* x,
                           double tol, int32_t precision, rp_solve_info* info, cudaStream_t s) {
  const int mode = precision == RP_MIXED_RU ? 2 : precision == RP_MIXED ? 1 : 0;
  RP_TRY(batch_prepare(h));
  cudaGraphExec_t& ex = h->batch_graphs[mode];
  if (!ex) RP_TRY(build_batch_graph(h, mode, h->batch_cluster, h->batch_threads, &ex));
  const double* src = buffer;
  if (where == RP_MEM_HOST) {
    RP_TRY_CUDA(cudaMemcpyAsync(h->staging, buffer, sizeof(double) * h->n_slots, cudaMemcpyHostToDevice, s));
    src = h->staging;
  }
  k_batch_setup<<<1, 1, 0, s>>>(h->batch_io, src, b, x, tol);
  RP_TRY_CUDA(cudaGetLastError());
  RP_TRY_CUDA(cudaGraphLaunch(ex, s));
  if (info) {
    RP_TRY_CUDA(cudaMemcpyAsync(info, h->batch_info, sizeof(rp_solve_info) * h->n_parts, cudaMemcpyDeviceToHost, s));
    RP_TRY_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < h->n_parts; ++i)
      if (info[i].status != RP_OK) return (rp_status)info[i].status;
  }
  return RP_OK;
}

}  // namespace rp

using namespace rp;

extern "C" rp_status rp_batch_build(const rp_ldu_desc* systems, int32_t count, const rp_options* opts,
                                    rp_handle** out) {
  if (!systems || count < 1 || !out) return fail(RP_EINVAL, "invalid argument");
  for (int i = 0; i < count; ++i)
    if (systems[i].n_iface != 0) return fail(RP_EINVAL, "system %d has interface entries; batched systems are independent", i);
  rp_options o;
  if (opts) o = *opts; else rp_default_options(&o);
  o.n_parts = count;
  RP_TRY(rp_build_repartition(systems, count, &o, out));
  rp_status s = batch_prepare(*out);
  if (s != RP_OK) {
    rp_destroy(*out);
    *out = nullptr;
  }
  return s;
}

extern "C" rp_status rp_batch_update_solve(rp_handle* h, const double* buffer, int32_t where, const double* b,
                                           double* x, double tol, int32_t precision, rp_solve_info* info,
                                           void* stream) {
  if (!h || !buffer || !b || !x) return fail(RP_EINVAL, "null argument");
  if (!(tol >= 0.0)) return fail(RP_EINVAL, "tol must be >= 0");
  if (where != RP_MEM_DEVICE && where != RP_MEM_HOST) return fail(RP_EINVAL, "where must be RP_MEM_DEVICE or RP_MEM_HOST");
  if (precision != RP_FP64 && precision != RP_MIXED && precision != RP_MIXED_RU)
    return fail(RP_EINVAL, "precision must be RP_FP64, RP_MIXED or RP_MIXED_RU");
  if (precision != RP_FP64 && !h->want_fp32) return fail(RP_EINVAL, "mixed precision needs want_fp32");
  return batch_run(h, buffer, where, b, x, tol, precision, info, (cudaStream_t)stream);
}

extern "C" rp_status rp_batch_set_config(rp_handle* h, int32_t cluster, int32_t threads) {
  if (!h) return fail(RP_EINVAL, "null handle");
  if (cluster < 1 || cluster > 16) return fail(RP_EINVAL, "cluster size must be in [1, 16]");
  if (threads < 64 || threads > kBatchMaxThreads || threads % 32)
    return fail(RP_EINVAL, "threads must be a multiple of 32 in [64, %d]", kBatchMaxThreads);
  RP_TRY(batch_prepare(h));
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr;
  int nc = 0;
  RP_TRY(launch_config(h, 0, cluster, threads, &cfg, &attr, &nc));
  if (h->want_fp32) RP_TRY(launch_config(h, 1, cluster, threads, &cfg, &attr, &nc));
  for (auto& g : h->batch_graphs)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  h->batch_cluster = cluster;
  h->batch_threads = threads;
  return RP_OK;
}

extern "C" rp_status rp_batch_autotune(rp_handle* h, const double* buffer, const double* b, double* x, double tol,
                                       int32_t precision, int32_t* best_cluster, int32_t* best_threads,
                                       float* best_ms, void* stream) {
  if (!h || !buffer || !b || !x) return fail(RP_EINVAL, "null argument");
  RP_TRY(batch_prepare(h));
  cudaStream_t s = (cudaStream_t)stream;
  // team counts between these shapes matter: with the largest systems first,
  // too many small teams leave the largest system's team running alone at
  // the end, too few large teams pay more barrier latency per iteration
  const int clusters[] = {2, 3, 4, 5, 6, 8, 16};
  const int threads[] = {256, 512};
  cudaEvent_t e0, e1;
  RP_TRY_CUDA(cudaEventCreate(&e0));
  RP_TRY_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int bc = h->batch_cluster, bt = h->batch_threads;
  for (int c : clusters)
    for (int t : threads) {
      if (rp_batch_set_config(h, c, t) != RP_OK) continue;
      // one untimed run (graph build, warm caches), then one timed run
      if (batch_run(h, buffer, RP_MEM_DEVICE, b, x, tol, precision, nullptr, s) != RP_OK) continue;
      cudaEventRecord(e0, s);
      if (batch_run(h, buffer, RP_MEM_DEVICE, b, x, tol, precision, nullptr, s) != RP_OK) continue;
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) continue;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        bc = c;
        bt = t;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  RP_TRY(rp_batch_set_config(h, bc, bt));
  if (best_cluster) *best_cluster = bc;
  if (best_threads) *best_threads = bt;
  if (best_ms) *best_ms = best;
  return RP_OK;
}
