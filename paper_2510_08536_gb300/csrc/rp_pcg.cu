// Jacobi-preconditioned CG on the merged device matrix, FP64 and
// FP32-inner / FP64-outer iterative refinement.
//
// One iteration is three HBM-streaming kernels with the two reductions of
// CG fused into them; every scalar stays on the device:
//   K1  q = A p,                    partial (p, q)   -> alpha = (r,z)/(p,q)
//   K2  r -= alpha q, z = D^-1 r,   partial (r,z), (r,r) -> beta, stop test
//   K3  x += alpha p, p = z + beta p
// Bytes per row and iteration (FP64, 7 entries per row): K1 12*nnz/n + 4
// (+8 p gather, +8 q write), K2 32, K3 48.
//
// Control: the solve is one CUDA graph. An outer while-node runs a residual
// pass (r = b - A x, the true residual, and the start of a CG run) and then
// an inner while-node over K1-K3; the inner condition is cleared by K2 when
// the recursive residual passes or the iteration cap is hit, the outer one
// by the residual pass when the true residual passes (or a cap is hit).
// Every loop is bounded by device-side counters.
#include <algorithm>
#include <type_traits>

#include "rp_common.cuh"
#include "rp_spmv.cuh"

namespace rp {

template <typename T>
struct IterArgs {
  int64_t n;
  const int32_t* row_ptr;
  const int32_t* col;
  const T* vals;
  const T* dinv;
  T* r;
  T* p;
  T* q;
  T* xd;  // iterate updated by K3: the correction d (mixed); nullptr = io->x
  Ctl* ctl;
  SolveIO* io;
  double* partials;
  cudaGraphConditionalHandle inner;
  int in_graph;  // 0: launched on a stream (kernel timing), no condition to set
  Parts<T> parts;
  Sliced<T> sl;  // K1 runs k_it_spmv_sl when built (n_slices > 0)
  Line<T> line;  // line preconditioner (K2 writes z, K3 reads it); l == nullptr: Jacobi
};

struct ResArgs {
  int64_t n;
  const int32_t* row_ptr;
  const int32_t* col;
  const double* vals;
  const double* dinv;  // FP64 path
  double* r;
  double* p;
  const float* dinv32;  // mixed path
  float* r32;
  float* p32;
  float* d32;
  Ctl* ctl;
  SolveIO* io;
  double* partials;
  cudaGraphConditionalHandle inner;
  cudaGraphConditionalHandle outer;
  int in_graph;
  int ru;  // mixed: continued (not restarted) inner PCG across refinements
  Parts<double> parts;
  Line<double> line;   // FP64 path, line preconditioner
  Line<float> line32;  // mixed path, line preconditioner
  const double* s64;   // mixed path, scaled inner system: s = 1/sqrt(a_ii)
};

// z = M^-1 r for the 32-row block this warp holds (lane j: row 32 s + j) of
// the line preconditioner: forward substitution y_j = r_j - l_j y_{j-1}, then
// back substitution z_j = w_j y_j - g_j z_{j+1}, each as a 5-step parallel
// scan of affine maps over the warp (l = 0 at the block start, g = 0 at its
// end). All 32 lanes must call it; lanes without a row pass zeros.
template <typename T>
__device__ __forceinline__ T line_solve(T r, T l, T w, T g, int lane) {
  T m = -l, k = r;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T mp = __shfl_up_sync(0xffffffffu, m, d), kp = __shfl_up_sync(0xffffffffu, k, d);
    if (lane >= d) {
      k = fma(m, kp, k);
      m *= mp;
    }
  }
  T M = -g, K = w * k;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T Mn = __shfl_down_sync(0xffffffffu, M, d), Kn = __shfl_down_sync(0xffffffffu, K, d);
    if (lane + d < 32) {
      K = fma(M, Kn, K);
      M *= Mn;
    }
  }
  return K;
}

// LU factors of the line preconditioner, one thread per 32-row block
// (Thomas algorithm in FP64 from the FP64 values; FP32 copies rounded to
// nearest). Columns are sorted, so a row's in-block neighbours i-1 and i+1,
// if stored, sit right before and after its diagonal entry.
__global__ void __launch_bounds__(kThreads)
    k_line_factors(int64_t n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                   const double* __restrict__ vals, const int32_t* __restrict__ diag_pos, double* __restrict__ l,
                   double* __restrict__ w, double* __restrict__ g, float* __restrict__ l32, float* __restrict__ w32,
                   float* __restrict__ g32) {
  const int64_t nb = (n + 31) / 32;
  for (int64_t blk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; blk < nb; blk += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = blk * 32, i1 = i0 + 32 < n ? i0 + 32 : n;
    double w_prev = 0.0, c_prev = 0.0;
    for (int64_t i = i0; i < i1; ++i) {
      const int dp = diag_pos[i], rs = row_ptr[i], re = row_ptr[i + 1];
      const double a = (i > i0 && dp > rs && col[dp - 1] == i - 1) ? vals[dp - 1] : 0.0;
      const double c = (i + 1 < i1 && dp + 1 < re && col[dp + 1] == i + 1) ? vals[dp + 1] : 0.0;
      const double li = a * w_prev;             // a_i / u_{i-1}
      const double wi = 1.0 / (vals[dp] - li * c_prev);  // 1 / u_i
      const double gi = wi * c;
      l[i] = li;
      w[i] = wi;
      g[i] = gi;
      if (l32) {
        l32[i] = (float)li;
        w32[i] = (float)wi;
        g32[i] = (float)gi;
      }
      w_prev = wi;
      c_prev = c;
    }
  }
}

// K1: q = A p and (p, q); the last block forms alpha.
// Per-thread partial sums are kept in T: the FP32 path does no per-element
// FP64 work (GB300 runs FP64 and float<->double conversions ~70x slower
// than FP32); one conversion per thread feeds the FP64 block reduction.
template <typename T>
__device__ __forceinline__ void pcg_k1_finish(Ctl* c, double* partials, T acc) {
  double v[1] = {(double)acc}, tot[1];
  if (reduce_last_block<1>(v, partials, &c->ticket, tot) && threadIdx.x == 0) {
    const double pq = tot[0];
    c->pq = pq;
    if (c->status == RP_DEVICE_TIMEOUT) {
      c->stop = 1;
    } else if (!(pq > 0.0) || !isfinite(pq)) {
      c->status = RP_BREAKDOWN;
      c->stop = 1;
      c->skip_x = 1;
    } else {
      c->alpha = c->rz / pq;
    }
  }
}

template <typename T>
struct PcgK1Epi {
  const T* p;
  Ctl* c;
  double* partials;
  T acc = T(0);
  __device__ __forceinline__ void row(int64_t i, T y) { acc = fma(p[i], y, acc); }
  __device__ __forceinline__ void timeout() {
    c->status = RP_DEVICE_TIMEOUT;
    c->stop = 1;
    c->skip_x = 1;
  }
  __device__ __forceinline__ void finish() { pcg_k1_finish<T>(c, partials, acc); }
};

template <typename T>
__global__ void __launch_bounds__(kThreads) k_it_spmv(IterArgs<T> a) {
  if (a.ctl->stop) return;
  PcgK1Epi<T> e{a.p, a.ctl, a.partials};
  spmv_csr_body<T>(a.n, a.parts, a.row_ptr, a.col, a.vals, a.p, a.q, e);
}

// K1 over the sliced layout: the body of spmv_sl_body written out for the
// PCG iteration. An instance of spmv_sl_body with PcgK1Epi computes the same
// but measured 5-7% slower for FP32 on GB300 (0.152-0.154 ms against 0.144 ms
// per launch at 256^3, same registers), so the hot kernel keeps its own copy.
// MP: several parts (k_it_spmv_sl_mp below). U4: every slice has 4-bit
// indices and rows of at most 8 entries (Sliced::u4), so every chunk fits its
// stage and the consumers skip the per-slice checks of the general case (9% fewer
// instructions, 1.4% of the mixed step at 256^3).
template <typename T, bool MP, bool U4 = false>
__device__ __forceinline__ void it_spmv_sl(const IterArgs<T>& a) {
  Ctl* c = a.ctl;
  if (c->stop) return;
  using St = SlStage<T>;
  constexpr int kStages = St::kStages;
  extern __shared__ __align__(128) unsigned char sbuf[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
  __shared__ uint32_t chunk_x[kStages], chunk_y[kStages];
  __shared__ int staged[kStages];
  __shared__ int timed_out, issued;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int S = (int)a.sl.n_slices, n = (int)a.n;
  const int NC = (S + kChunk - 1) / kChunk, G = gridDim.x;
  const uint2* desc = a.sl.desc;

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

  T acc = T(0);
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
        if (i >= kStages && !mbar_wait(&empty[st], (uint32_t)((i / kStages - 1) & 1), a.sl.spin)) {
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
        const bool fit = vb <= (uint32_t)St::kVals && ib <= (uint32_t)kStageIdx && chunk_copy_ok(a.sl, d0, d1, ch, db);
        chunk_x[st] = d0.x;
        chunk_y[st] = d0.y;
        staged[st] = fit;
        // consumers' generic-proxy reads of this stage (released through
        // empty[st]) before the async-proxy writes of the copy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (fit) {
          mbar_expect_tx(&full[st], vb + ib + db + kStageInfo);
          // values and index words are read once a product: evict them first, so that
          // the vectors the next kernels read stay in L2 (K1 2% faster, the step 0.15%)
          uint64_t pol;
          asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
          bulk_g2s_hint(base, a.sl.vals + d0.x, vb, &full[st], pol);
          bulk_g2s_hint(base + St::kVals, a.sl.ibuf + d0.y, ib, &full[st], pol);
          bulk_g2s(base + St::kVals + kStageIdx, desc + (int64_t)ch * kChunk, db, &full[st]);
          bulk_g2s(base + St::kVals + kStageIdx + kStageDesc, a.sl.tinfo + (int64_t)ch * kChunk, kStageInfo, &full[st]);
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
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&full[st], (uint32_t)((i / kStages) & 1), a.sl.spin));
      if (!ok) {
        if (lane == 0) atomicExch(&timed_out, 1);
        break;
      }
      const int s = ch * kChunk + w;
      if (s < S) {
        SliceRows sr{s * kSliceRows, 0, 0};
        if constexpr (MP) sr = slice_rows(a.sl, s, n);  // several parts: per-slice records
        const int row = sr.row0 + lane;
        const bool valid = MP ? lane < sr.rows : row < n;
        NlRange nl{0, 0};
        if constexpr (MP)
          if (valid) nl = nonlocal_range<T>(a.parts, sr.part, row);
        const T* x = a.p + row;
        const SliceCk ck = slice_ck<T, MP>(a.sl, a.parts, sr.part, row, n);
        const unsigned char* base = sbuf + st * St::kBytes;
        T sum;
        if constexpr (U4) {
          const uint2* sd = reinterpret_cast<const uint2*>(base + St::kVals + kStageIdx);
          const uint32_t* si = reinterpret_cast<const uint32_t*>(base + St::kVals + kStageIdx + kStageDesc);
          const uint2 d0 = sd[w], d1 = sd[w + 1];
          const int32_t* tab = a.sl.tabs + (si[w] & ~kSliceW4);
          sum = slice_row<T, kIdx4>(reinterpret_cast<const T*>(base) + (d0.x - chunk_x[st]) + lane,
                                    reinterpret_cast<const uint32_t*>(base + St::kVals) + (d0.y - chunk_y[st]) + lane,
                                    __ldg(tab + (lane & 15)), tab, x, valid, (int)((d1.x - d0.x) >> 5), 0, ck);
        } else if (staged[st]) {
          const uint2* sd = reinterpret_cast<const uint2*>(base + St::kVals + kStageIdx);
          const uint32_t* si = reinterpret_cast<const uint32_t*>(base + St::kVals + kStageIdx + kStageDesc);
          const uint2 d0 = sd[w], d1 = sd[w + 1];
          sum = slice_sum<T>(d0, d1, si[w], reinterpret_cast<const T*>(base) + (d0.x - chunk_x[st]) + lane,
                             reinterpret_cast<const uint32_t*>(base + St::kVals) + (d0.y - chunk_y[st]) + lane,
                             a.sl.tabs, x, valid, lane, ck);
        } else {
          const uint2 d0 = __ldg(desc + s), d1 = __ldg(desc + s + 1);
          sum = slice_sum<T>(d0, d1, __ldg(a.sl.tinfo + s), a.sl.vals + d0.x + lane,
                             reinterpret_cast<const uint32_t*>(a.sl.ibuf + d0.y) + lane, a.sl.tabs, x, valid, lane,
                             ck);
        }
        if constexpr (MP) sum = nonlocal_sum<T>(a.parts, sr.part, nl, a.p, sum);
        if (valid) {
          a.q[row] = sum;
          acc = fma(a.p[row], sum, acc);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    }
  }
  __syncthreads();
  if (timed_out) {
    // wait (bounded) for the copies this block may still have in flight, then stop the solve
    if (tid == kChunk * 32) {
      for (int j = issued - kStages; j < issued; ++j)
        if (j >= 0) mbar_wait(&full[j % kStages], (uint32_t)((j / kStages) & 1), kDrainProbes);
      c->status = RP_DEVICE_TIMEOUT;
      c->stop = 1;
      c->skip_x = 1;
    }
    __syncthreads();
  }
  pcg_k1_finish<T>(a.ctl, a.partials, acc);
}

template <typename T, bool U4 = false>
__global__ void __launch_bounds__(kSlThreads) k_it_spmv_sl(IterArgs<T> a) {
  it_spmv_sl<T, false, U4>(a);
}
// the uniform-slice instance (never in the bounds-checked build, which checks
// every slice's descriptors and indices)
#ifdef RP_CHECK
constexpr bool kUseU4 = false;
#else
constexpr bool kUseU4 = true;
#endif
template <typename T>
bool k1_u4(const IterArgs<T>& a) {
  return kUseU4 && a.sl.u4 && !a.sl.srow;
}
// Several parts: the FP32 instance is held to the registers of seven blocks an
// SM, which the one-part FP32 kernel reaches without a bound (FP64: five, its
// shared-memory limit).
template <typename T>
__global__ void __launch_bounds__(kSlThreads, sizeof(T) == 4 ? 7 : 5) k_it_spmv_sl_mp(IterArgs<T> a) {
  it_spmv_sl<T, true>(a);
}

template <typename T>
void* k1_kernel(const IterArgs<T>& a) {
  if (a.sl.n_slices == 0) return (void*)k_it_spmv<T>;
  return a.sl.srow ? (void*)k_it_spmv_sl_mp<T> : k1_u4(a) ? (void*)k_it_spmv_sl<T, true> : (void*)k_it_spmv_sl<T>;
}
template <typename T>
int k1_grid(const IterArgs<T>& a, const IterGrid& g) {
  return a.sl.n_slices == 0 ? g.k1 : a.sl.srow ? g.k1sm : g.k1s;
}
template <typename T>
int k1_smem(const IterArgs<T>& a) {
  return a.sl.n_slices > 0 ? SlStage<T>::kSmem : 0;
}
template <typename T>
int k1_threads(const IterArgs<T>& a) {
  return a.sl.n_slices > 0 ? kSlThreads : kThreads;
}
template <typename T>
void launch_k1(const IterArgs<T>& a, int grid, cudaStream_t s) {
  if (a.sl.n_slices > 0 && a.sl.srow) k_it_spmv_sl_mp<T><<<grid, kSlThreads, SlStage<T>::kSmem, s>>>(a);
  else if (a.sl.n_slices > 0 && k1_u4(a)) k_it_spmv_sl<T, true><<<grid, kSlThreads, SlStage<T>::kSmem, s>>>(a);
  else if (a.sl.n_slices > 0) k_it_spmv_sl<T><<<grid, kSlThreads, SlStage<T>::kSmem, s>>>(a);
  else k_it_spmv<T><<<grid, kThreads, 0, s>>>(a);
}

// K2: r -= alpha q; z = D^-1 r (LINE: z = M^-1 r, stored; SCALED: the system
// is scaled to a unit diagonal and z = r); (r, z), (r, r); stop test; beta.
// FP32 vector loads / stores with an L2 evict-first policy, for vectors whose next
// use is far: q after the residual kernel has read it, the correction d (read and
// written once an iteration), r when K3 has read it (K2 reads it next, after a whole
// SpMV). With the matrix copies of K1 also evict-first, the vector the SpMV gathers
// seven times (p) stays in L2: the headline step 257.4 -> 252.3 ms with the first two,
// -> 245.0 ms with r (K1 0.1289 -> 0.1256 ms, K3 0.0551 -> 0.0501 ms).
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ float4 ld_ef(const float4* p, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_ef(float4* p, float4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w), "l"(pol)
               : "memory");
}

template <typename T, bool LINE, bool SCALED = false>
__global__ void __launch_bounds__(kThreads) k_it_resid(IterArgs<T> a) {
  Ctl* c = a.ctl;
  if (c->stop) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.in_graph) cudaGraphSetConditional(a.inner, 0);
    return;
  }
  const T alpha = (T)c->alpha;
  using V = typename Vec<T>::type;
  constexpr int W = Vec<T>::N;
  T rz = T(0), rr = T(0);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nv = a.n / W;
  auto step = [&](V& rv, V qv, V dv) {
    for_each_comp<W>([&](auto e) {
      constexpr int E = decltype(e)::value;
      T ri = fma(-alpha, comp<E>(qv), comp<E>(rv));
      comp<E>(rv) = ri;
      rz = fma(ri, comp<E>(dv) * ri, rz);
      rr = fma(ri, ri, rr);
    });
  };
  int64_t k = tid;
  if constexpr (LINE) {
    // one 32-row block per warp per step (rows as in the Jacobi loop)
    const int lane = threadIdx.x & 31;
    for (int64_t base = tid - lane; base < a.n; base += stride) {
      const int64_t i = base + lane;
      const bool valid = i < a.n;
      T ri = T(0), li = T(0), wi = T(0), gi = T(0);
      if (valid) {
        ri = fma(-alpha, a.q[i], a.r[i]);
        li = a.line.l[i];
        wi = a.line.w[i];
        gi = a.line.g[i];
      }
      const T zi = line_solve<T>(ri, li, wi, gi, lane);
      if (valid) {
        a.r[i] = ri;
        a.line.z[i] = zi;
      }
      rz = fma(ri, zi, rz);
      rr = fma(ri, ri, rr);
    }
  }
  if constexpr (SCALED) {
    // unit diagonal: z = r, so (r, z) = (r, r) and no diagonal is read
    auto sstep = [&](V& rv, V qv) {
      for_each_comp<W>([&](auto e) {
        constexpr int E = decltype(e)::value;
        T ri = fma(-alpha, comp<E>(qv), comp<E>(rv));
        comp<E>(rv) = ri;
        rr = fma(ri, ri, rr);
      });
    };
    for (; k + stride < nv; k += 2 * stride) {
      V q0, q1;
      if constexpr (sizeof(T) == 4) {
        const uint64_t pol = l2_evict_first();  // q is not read again
        q0 = ld_ef(reinterpret_cast<const float4*>(a.q) + k, pol);
        q1 = ld_ef(reinterpret_cast<const float4*>(a.q) + k + stride, pol);
      } else {
        q0 = reinterpret_cast<const V*>(a.q)[k];
        q1 = reinterpret_cast<const V*>(a.q)[k + stride];
      }
      V r0 = reinterpret_cast<const V*>(a.r)[k], r1 = reinterpret_cast<const V*>(a.r)[k + stride];
      sstep(r0, q0);
      sstep(r1, q1);
      reinterpret_cast<V*>(a.r)[k] = r0;
      reinterpret_cast<V*>(a.r)[k + stride] = r1;
    }
    for (; k < nv; k += stride) {
      V qv = reinterpret_cast<const V*>(a.q)[k];
      V rv = reinterpret_cast<const V*>(a.r)[k];
      sstep(rv, qv);
      reinterpret_cast<V*>(a.r)[k] = rv;
    }
    for (int64_t i = nv * W + tid; i < a.n; i += stride) {
      T ri = fma(-alpha, a.q[i], a.r[i]);
      a.r[i] = ri;
      rr = fma(ri, ri, rr);
    }
    rz = rr;
  }
  if constexpr (!LINE && !SCALED) {
    // two vectors of each stream in flight per thread
    for (; k + stride < nv; k += 2 * stride) {
      V q0 = reinterpret_cast<const V*>(a.q)[k], q1 = reinterpret_cast<const V*>(a.q)[k + stride];
      V r0 = reinterpret_cast<const V*>(a.r)[k], r1 = reinterpret_cast<const V*>(a.r)[k + stride];
      V d0 = reinterpret_cast<const V*>(a.dinv)[k], d1 = reinterpret_cast<const V*>(a.dinv)[k + stride];
      step(r0, q0, d0);
      step(r1, q1, d1);
      reinterpret_cast<V*>(a.r)[k] = r0;
      reinterpret_cast<V*>(a.r)[k + stride] = r1;
    }
    for (; k < nv; k += stride) {
      V qv = reinterpret_cast<const V*>(a.q)[k];
      V rv = reinterpret_cast<const V*>(a.r)[k];
      V dv = reinterpret_cast<const V*>(a.dinv)[k];
      step(rv, qv, dv);
      reinterpret_cast<V*>(a.r)[k] = rv;
    }
    for (int64_t i = nv * W + tid; i < a.n; i += stride) {
      T ri = fma(-alpha, a.q[i], a.r[i]);
      a.r[i] = ri;
      rz = fma(ri, a.dinv[i] * ri, rz);
      rr = fma(ri, ri, rr);
    }
  }
  double v[2] = {(double)rz, (double)rr}, tot[2];
  if (reduce_last_block<2>(v, a.partials, &c->ticket, tot) && threadIdx.x == 0) {
    c->iter += 1;
    c->iter_total += 1;
    c->rr = tot[1];
    const double thresh = a.xd ? c->inner_thresh : c->thresh;
    if (tot[1] <= thresh) {
      c->stop = 1;
    } else if (c->iter >= c->max_iter) {
      c->stop = 1;
    } else if (!(tot[0] > 0.0) || !isfinite(tot[0])) {
      c->stop = 1;
      c->status = RP_BREAKDOWN;
    } else {
      c->beta = tot[0] / c->rz;
      c->rz = tot[0];
    }
    if (a.in_graph) cudaGraphSetConditional(a.inner, c->stop ? 0u : 1u);
  }
}

// K3: x += alpha p; p = z + beta p (the latter only while iterating; z = D^-1 r,
// LINE: the z K2 stored, SCALED: z = r).
template <typename T, bool LINE, bool SCALED = false>
__global__ void __launch_bounds__(kThreads) k_it_xp(IterArgs<T> a) {
  Ctl* c = a.ctl;
  if (c->skip_x) return;
  const T alpha = (T)c->alpha, beta = (T)c->beta;
  const bool upd_p = !c->stop;
  T* x = a.xd;
  if (x == nullptr) x = reinterpret_cast<T*>(a.io->x);
  using V = typename Vec<T>::type;
  constexpr int W = Vec<T>::N;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // the caller's x may not be 16-byte aligned: vectorise only when it is
  const int64_t nv = (reinterpret_cast<uintptr_t>(x) & 15) ? 0 : a.n / W;
  for (int64_t k = tid; k < nv; k += stride) {
    V pv = reinterpret_cast<const V*>(a.p)[k];
    V xv;
    if constexpr (sizeof(T) == 4 && SCALED) xv = ld_ef(reinterpret_cast<const float4*>(x) + k, l2_evict_first());
    else xv = reinterpret_cast<const V*>(x)[k];
    for_each_comp<W>([&](auto e) {
      constexpr int E = decltype(e)::value;
      comp<E>(xv) = fma(alpha, comp<E>(pv), comp<E>(xv));
    });
    if constexpr (sizeof(T) == 4 && SCALED) st_ef(reinterpret_cast<float4*>(x) + k, xv, l2_evict_first());
    else reinterpret_cast<V*>(x)[k] = xv;
    if (upd_p) {
      if constexpr (LINE) {
        V zv = reinterpret_cast<const V*>(a.line.z)[k];
        for_each_comp<W>([&](auto e) {
          constexpr int E = decltype(e)::value;
          comp<E>(pv) = fma(beta, comp<E>(pv), comp<E>(zv));
        });
      } else if constexpr (SCALED) {
        V rv;
        if constexpr (sizeof(T) == 4) rv = ld_ef(reinterpret_cast<const float4*>(a.r) + k, l2_evict_first());
        else rv = reinterpret_cast<const V*>(a.r)[k];
        for_each_comp<W>([&](auto e) {
          constexpr int E = decltype(e)::value;
          comp<E>(pv) = fma(beta, comp<E>(pv), comp<E>(rv));
        });
      } else {
        V rv = reinterpret_cast<const V*>(a.r)[k];
        V dv = reinterpret_cast<const V*>(a.dinv)[k];
        for_each_comp<W>([&](auto e) {
          constexpr int E = decltype(e)::value;
          comp<E>(pv) = fma(beta, comp<E>(pv), comp<E>(dv) * comp<E>(rv));
        });
      }
      reinterpret_cast<V*>(a.p)[k] = pv;
    }
  }
  for (int64_t i = nv * W + tid; i < a.n; i += stride) {
    T pi = a.p[i];
    x[i] = fma(alpha, pi, x[i]);
    if (upd_p) a.p[i] = fma(beta, pi, LINE ? a.line.z[i] : SCALED ? a.r[i] : a.dinv[i] * a.r[i]);
  }
}

// Residual pass of the FP64 solve: r = b - A x (or r = b, x = 0 on a cold
// start), p = z = D^-1 r (LINE: M^-1 r), (r, z), (r, r) [, (b, b)]; decides the next step.
template <bool LINE>
__global__ void __launch_bounds__(kThreads) k_res64(ResArgs a) {
  Ctl* c = a.ctl;
  const bool cold = c->pass == 0 && c->x_zero;
  const bool first = c->pass == 0;
  const double* __restrict__ b = a.io->b;
  double* __restrict__ x = a.io->x;
  double rz = 0.0, rr = 0.0, bb = 0.0;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // warp-uniform loop over 32-row blocks (the line solve needs the whole warp)
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; base < a.n; base += stride) {
    const int64_t i = base + lane;
    const bool valid = i < a.n;
    double bi = 0.0, ri = 0.0;
    if (valid) {
      bi = b[i];
      if (cold) {
        ri = bi;
        x[i] = 0.0;
      } else {
        ri = bi - row_dot_any<double>(a.parts, a.row_ptr, a.col, a.vals, x, i, a.n);
      }
      a.r[i] = ri;
    }
    double zi;
    if constexpr (LINE) {
      zi = line_solve<double>(ri, valid ? a.line.l[i] : 0.0, valid ? a.line.w[i] : 0.0, valid ? a.line.g[i] : 0.0,
                              lane);
    } else {
      zi = valid ? a.dinv[i] * ri : 0.0;
    }
    if (valid) a.p[i] = zi;
    rz += ri * zi;
    rr += ri * ri;
    bb += bi * bi;
  }
  double v[3] = {rz, rr, bb}, tot[3];
  if (reduce_last_block<3>(v, a.partials, &c->ticket, tot) && threadIdx.x == 0) {
    if (first) {
      c->bb = tot[2];
      c->thresh = c->tol * c->tol * tot[2];
    }
    c->rr = tot[1];
    c->rz = tot[0];
    c->pass += 1;
    bool go = false;
    if (tot[1] <= c->thresh) {
      c->status = RP_OK;
    } else if (c->status == RP_BREAKDOWN || c->status == RP_DEVICE_TIMEOUT) {
    } else if (!isfinite(tot[1])) {
      c->status = RP_BREAKDOWN;
    } else if (c->iter_total >= c->max_iter || (!first && c->restarts >= c->max_restarts)) {
      c->status = RP_NOT_CONVERGED;
    } else {
      if (!first) c->restarts += 1;
      go = true;
    }
    c->stop = go ? 0 : 1;
    c->skip_x = 0;
    if (a.in_graph) {
      cudaGraphSetConditional(a.inner, go ? 1u : 0u);
      cudaGraphSetConditional(a.outer, go ? 1u : 0u);
    }
  }
}

// Residual pass of the mixed solve: r = b - A x in FP64 with FP64 values,
// its FP32 copy as the inner right-hand side, d = 0, p = z = D32^-1 r32
// (LINE: z = M32^-1 r32, also stored for the continued refinement; SCALED:
// the inner system is S A S, its right-hand side r32 = fl32(S r) and z = r32).
template <bool LINE, bool SCALED = false>
__global__ void __launch_bounds__(kThreads) k_res_mixed(ResArgs a) {
  Ctl* c = a.ctl;
  const bool cold = c->pass == 0 && c->x_zero;
  const bool first = c->pass == 0;
  const double* __restrict__ b = a.io->b;
  double* __restrict__ x = a.io->x;
  double rz = 0.0, rr = 0.0, bb = 0.0, rr32 = 0.0;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // warp-uniform loop over 32-row blocks (the line solve needs the whole warp)
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; base < a.n; base += stride) {
    const int64_t i = base + lane;
    const bool valid = i < a.n;
    double bi = 0.0, ri = 0.0;
    if (valid) {
      bi = b[i];
      if (cold) {
        ri = bi;
        x[i] = 0.0;
      } else {
        ri = bi - row_dot_any<double>(a.parts, a.row_ptr, a.col, a.vals, x, i, a.n);
      }
    }
    float r32, z32;
    if constexpr (SCALED) {
      r32 = valid ? (float)(a.s64[i] * ri) : 0.0f;
      z32 = r32;
    } else if constexpr (LINE) {
      r32 = (float)ri;
      z32 = line_solve<float>(r32, valid ? a.line32.l[i] : 0.0f, valid ? a.line32.w[i] : 0.0f,
                              valid ? a.line32.g[i] : 0.0f, lane);
      if (valid) a.line32.z[i] = z32;
    } else {
      r32 = (float)ri;
      z32 = valid ? a.dinv32[i] * r32 : 0.0f;
    }
    if (valid) {
      a.r32[i] = r32;
      a.d32[i] = 0.0f;
      if (!a.ru || first) a.p32[i] = z32;  // continued refinement keeps p after the first pass
    }
    rz += (double)r32 * (double)z32;
    rr32 += (double)r32 * (double)r32;
    rr += ri * ri;
    bb += bi * bi;
  }
  double v[4] = {rz, rr, bb, rr32}, tot[4];
  if (reduce_last_block<4>(v, a.partials, &c->ticket, tot) && threadIdx.x == 0) {
    if (first) {
      c->bb = tot[2];
      c->thresh = c->tol * c->tol * tot[2];
    }
    c->rr = tot[1];
    c->pass += 1;
    bool go = false;
    if (tot[1] <= c->thresh) {
      c->status = RP_OK;
    } else if (c->status == RP_BREAKDOWN || c->status == RP_DEVICE_TIMEOUT) {
    } else if (!isfinite(tot[1])) {
      c->status = RP_BREAKDOWN;
    } else if (c->outer >= c->max_outer) {
      c->status = RP_NOT_CONVERGED;
    } else if (a.ru && c->iter_total >= c->max_iter) {
      c->status = RP_NOT_CONVERGED;
    } else {
      go = true;
      c->outer += 1;
      // half the outer target, in the inner residual's norm (scaled: carried
      // over by the ratio of the scaled to the unscaled residual)
      const double floor = 0.25 * c->thresh * (SCALED ? tot[3] / tot[1] : 1.0);
      if (a.ru) {
        // the FP64 residual replaces the FP32 one; the search direction continues
        c->ru_apply = first ? 0 : 1;
        c->beta_ru = first ? 0.0 : tot[0] / c->rz;
        // inner tolerance, or half the outer target (a residual just above the
        // target must still make progress: no endless one-step phases)
        c->inner_thresh = fmax(c->ru_delta * c->ru_delta * tot[3], floor);
      } else {
        // a reduction by inner_tol, but no further than half the outer target:
        // the last refinement stops near the target instead of far below it
        c->inner_thresh = fmax(c->inner_tol * c->inner_tol * tot[3], floor);
        c->iter = 0;
      }
      c->rz = tot[0];
    }
    if (!go) c->ru_apply = 0;
    c->stop = go ? 0 : 1;
    c->skip_x = 0;
    c->skip_correct = go ? 0 : 1;
    if (a.in_graph) {
      cudaGraphSetConditional(a.inner, go ? 1u : 0u);
      cudaGraphSetConditional(a.outer, go ? 1u : 0u);
    }
  }
}

struct CorrectArgs {
  int64_t n;
  const float* d;
  Ctl* c;
  SolveIO* io;
  const double* s64;  // scaled inner system: x += S d
};

struct RuArgs {
  int64_t n;
  const float* dinv32;
  const float* r32;
  float* p32;
  Ctl* c;
  const float* z32;  // LINE: M32^-1 r32 stored by the residual pass
};

// continued refinement: p = D32^-1 r32 + beta p (LINE: z32 + beta p, SCALED:
// r32 + beta p) after the residual was replaced
template <bool LINE, bool SCALED = false>
__global__ void __launch_bounds__(kThreads) k_ru_p(RuArgs a) {
  if (!a.c->ru_apply) return;
  const float beta = (float)a.c->beta_ru;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x)
    a.p32[i] = fmaf(beta, a.p32[i], LINE ? a.z32[i] : SCALED ? a.r32[i] : a.dinv32[i] * a.r32[i]);
}

// x += d (FP64) after an inner FP32 solve (scaled inner system: x += S d).
__global__ void __launch_bounds__(kThreads) k_correct(CorrectArgs a) {
  if (a.c->skip_correct || a.c->status == RP_BREAKDOWN || a.c->status == RP_DEVICE_TIMEOUT) return;
  double* __restrict__ x = a.io->x;
  const double* __restrict__ s = a.s64;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += s ? s[i] * (double)a.d[i] : (double)a.d[i];
}

__global__ void k_setup(Ctl* c, SolveIO* io, const double* b, double* x, double tol, double inner_tol, int x_zero,
                        int max_iter, int max_restarts, int max_outer, double ru_delta = 0.0) {
  io->b = b;
  io->x = x;
  c->tol = tol;
  c->inner_tol = inner_tol;
  c->ru_delta = ru_delta > 0.0 ? ru_delta : inner_tol;
  c->x_zero = x_zero;
  c->max_iter = max_iter;
  c->max_restarts = max_restarts;
  c->max_outer = max_outer;
  c->iter = 0;
  c->iter_total = 0;
  c->pass = 0;
  c->restarts = 0;
  c->outer = 0;
  c->status = -1;
  c->stop = 0;
  c->skip_x = 0;
  c->skip_correct = 1;
  c->alpha = c->beta = 0.0;
  c->ticket = 0u;
}

// y = A x and, optionally, x.y
__global__ void __launch_bounds__(kThreads)
    k_spmv_plain(int64_t n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                 const double* __restrict__ vals, const double* __restrict__ x, double* __restrict__ y,
                 double* xy, double* partials, unsigned int* ticket, Parts<double> parts) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = row_dot_any<double>(parts, row_ptr, col, vals, x, i, n);
    y[i] = s;
    acc += x[i] * s;
  }
  if (xy == nullptr) return;
  double v[1] = {acc}, tot[1];
  if (reduce_last_block<1>(v, partials, ticket, tot) && threadIdx.x == 0) *xy = tot[0];
}

// ------------------------------------------------------------------ graphs

namespace {

rp_status add_kernel(cudaGraph_t g, cudaGraphNode_t* node, const cudaGraphNode_t* dep, void* fn, int grid,
                     void* argp, int smem = 0, int threads = kThreads) {
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeKernel;
  np.kernel.func = fn;
  np.kernel.gridDim = dim3((unsigned)grid);
  np.kernel.blockDim = dim3((unsigned)threads);
  np.kernel.sharedMemBytes = (unsigned)smem;
  void* args[1] = {argp};
  np.kernel.kernelParams = args;
  RP_TRY_CUDA(cudaGraphAddNode(node, g, dep, nullptr, dep ? 1 : 0, &np));
  return RP_OK;
}

rp_status add_while(cudaGraph_t g, cudaGraphNode_t* node, const cudaGraphNode_t* dep,
                    cudaGraphConditionalHandle hnd, cudaGraph_t* body) {
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = hnd;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  RP_TRY_CUDA(cudaGraphAddNode(node, g, dep, nullptr, dep ? 1 : 0, &np));
  *body = np.conditional.phGraph_out[0];
  return RP_OK;
}

struct GraphGuard {
  cudaGraph_t g = nullptr;
  ~GraphGuard() {
    if (g) cudaGraphDestroy(g);
  }
};

// Arguments and kernels of one solve (graph, host loop and kernel timing use
// the same set): residual pass, continued-refinement step, iteration kernels
// of both precisions and the correction, with the Jacobi or line variants.
struct SolveSet {
  bool line;
  bool scaled;  // mixed: the inner FP32 iteration runs on S A S
  ResArgs ra;
  RuArgs ru;
  IterArgs<double> a64;
  IterArgs<float> a32;
  CorrectArgs ca;
  void *res, *rup, *k2_64, *k3_64, *k2_32, *k3_32;
  int g2_64, g3_64, g2_32, g3_32;
};

SolveSet solve_set(rp_handle* h, int mode, const double* vals, const double* dinv, cudaGraphConditionalHandle hin,
                   cudaGraphConditionalHandle hout, int in_graph) {
  SolveSet k{};
  const bool mixed = mode != 0;
  k.line = h->precond == RP_PRECOND_LINE && vals == h->vals && h->ln_l != nullptr;
  k.scaled = mixed && !k.line && vals == h->vals && h->sl_vals32s != nullptr;
  const Line<double> l64 = k.line ? Line<double>{h->ln_l, h->ln_w, h->ln_g, h->ln_z} : Line<double>{};
  const Line<float> l32 = k.line ? Line<float>{h->ln_l32, h->ln_w32, h->ln_g32, h->ln_z32} : Line<float>{};
  ResArgs& ra = k.ra;
  ra.n = h->n;
  ra.row_ptr = h->row_ptr;
  ra.col = h->col_idx;
  ra.vals = vals;
  ra.dinv = dinv;
  ra.r = h->r;
  ra.p = h->p;
  ra.dinv32 = h->dinv32;
  ra.r32 = h->r32;
  ra.p32 = h->p32;
  ra.d32 = h->d32;
  ra.ctl = h->ctl;
  ra.io = h->io;
  ra.partials = h->partials;
  ra.inner = hin;
  ra.outer = hout;
  ra.in_graph = in_graph;
  ra.ru = mode == 2;
  ra.parts = parts64(h);
  ra.line = l64;
  ra.line32 = l32;
  ra.s64 = k.scaled ? h->s64 : nullptr;
  k.ru = RuArgs{h->n, h->dinv32, h->r32, h->p32, h->ctl, h->ln_z32};
  k.a64 = IterArgs<double>{h->n, h->row_ptr, h->col_idx, vals, dinv, h->r, h->p, h->q, nullptr,
                           h->ctl, h->io, h->partials, hin, in_graph, parts64(h), sliced64(h, vals), l64};
  k.a32 = IterArgs<float>{h->n, h->row_ptr, h->col_idx, h->vals32, h->dinv32, h->r32, h->p32, h->q32, h->d32,
                          h->ctl, h->io, h->partials, hin, in_graph, parts32(h), sliced32(h), l32};
  k.ca = CorrectArgs{h->n, h->d32, h->ctl, h->io, k.scaled ? h->s64 : nullptr};
  if (k.scaled) k.a32.sl.vals = h->sl_vals32s;  // same slices, the values of S A S
  if (k.scaled) {
    k.res = (void*)k_res_mixed<false, true>;
    k.rup = (void*)k_ru_p<false, true>;
    k.k2_64 = (void*)k_it_resid<double, false>;
    k.k3_64 = (void*)k_it_xp<double, false>;
    k.k2_32 = (void*)k_it_resid<float, false, true>;
    k.k3_32 = (void*)k_it_xp<float, false, true>;
    k.g2_64 = h->igrid64.k2;
    k.g3_64 = h->igrid64.k3;
    k.g2_32 = h->igrid32.k2s;
    k.g3_32 = h->igrid32.k3s;
  } else if (k.line) {
    k.res = mixed ? (void*)k_res_mixed<true> : (void*)k_res64<true>;
    k.rup = (void*)k_ru_p<true>;
    k.k2_64 = (void*)k_it_resid<double, true>;
    k.k3_64 = (void*)k_it_xp<double, true>;
    k.k2_32 = (void*)k_it_resid<float, true>;
    k.k3_32 = (void*)k_it_xp<float, true>;
    k.g2_64 = h->igrid64.k2l;
    k.g3_64 = h->igrid64.k3l;
    k.g2_32 = h->igrid32.k2l;
    k.g3_32 = h->igrid32.k3l;
  } else {
    k.res = mixed ? (void*)k_res_mixed<false> : (void*)k_res64<false>;
    k.rup = (void*)k_ru_p<false>;
    k.k2_64 = (void*)k_it_resid<double, false>;
    k.k3_64 = (void*)k_it_xp<double, false>;
    k.k2_32 = (void*)k_it_resid<float, false>;
    k.k3_32 = (void*)k_it_xp<float, false>;
    k.g2_64 = h->igrid64.k2;
    k.g3_64 = h->igrid64.k3;
    k.g2_32 = h->igrid32.k2;
    k.g3_32 = h->igrid32.k3;
  }
  return k;
}

rp_status launch1(void* fn, int grid, int threads, int smem, void* argp, cudaStream_t s) {
  void* args[1] = {argp};
  RP_TRY_CUDA(cudaLaunchKernel(fn, dim3((unsigned)grid), dim3((unsigned)threads), args, (size_t)smem, s));
  return RP_OK;
}

// while (outer) { residual pass; [p = z + beta p]; while (inner) { K1; K2; K3 }; [x += d] }
// mode: 0 FP64, 1 mixed (restarted inner PCG), 2 mixed with continued inner PCG
rp_status build_solve_graph(rp_handle* h, int mode, const double* vals, const double* dinv,
                            cudaGraphExec_t* exec) {
  const bool mixed = mode != 0;
  GraphGuard top;
  RP_TRY_CUDA(cudaGraphCreate(&top.g, 0));
  cudaGraphConditionalHandle hout, hin;
  RP_TRY_CUDA(cudaGraphConditionalHandleCreate(&hout, top.g, 1, cudaGraphCondAssignDefault));
  cudaGraphNode_t wout, nres, win, n1, n2, n3, ncor;
  cudaGraph_t obody = nullptr, ibody = nullptr;
  RP_TRY(add_while(top.g, &wout, nullptr, hout, &obody));
  RP_TRY_CUDA(cudaGraphConditionalHandleCreate(&hin, obody, 0, 0));

  SolveSet k = solve_set(h, mode, vals, dinv, hin, hout, 1);
  RP_TRY(add_kernel(obody, &nres, nullptr, k.res, h->grid, &k.ra));
  cudaGraphNode_t before_inner = nres, nru;
  if (mode == 2) {
    RP_TRY(add_kernel(obody, &nru, &nres, k.rup, h->grid, &k.ru));
    before_inner = nru;
  }
  RP_TRY(add_while(obody, &win, &before_inner, hin, &ibody));
  if (mixed) {
    IterArgs<float>& ia = k.a32;
    RP_TRY(add_kernel(ibody, &n1, nullptr, k1_kernel(ia), k1_grid(ia, h->igrid32), &ia, k1_smem(ia), k1_threads(ia)));
    RP_TRY(add_kernel(ibody, &n2, &n1, k.k2_32, k.g2_32, &ia));
    RP_TRY(add_kernel(ibody, &n3, &n2, k.k3_32, k.g3_32, &ia));
    RP_TRY(add_kernel(obody, &ncor, &win, (void*)k_correct, h->grid, &k.ca));
  } else {
    IterArgs<double>& ia = k.a64;
    RP_TRY(add_kernel(ibody, &n1, nullptr, k1_kernel(ia), k1_grid(ia, h->igrid64), &ia, k1_smem(ia), k1_threads(ia)));
    RP_TRY(add_kernel(ibody, &n2, &n1, k.k2_64, k.g2_64, &ia));
    RP_TRY(add_kernel(ibody, &n3, &n2, k.k3_64, k.g3_64, &ia));
  }
  RP_TRY_CUDA(cudaGraphInstantiate(exec, top.g, 0));
  return RP_OK;
}

template <typename T>
rp_status dalloc(T** p, int64_t count) {
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

}  // namespace

namespace {

// Blocks of one kernel that fit on an SM at once (at most kBlocksPerSm).
int resident(const void* fn, int smem = 0, int threads = kThreads) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess || nb < 1) {
    cudaGetLastError();
    nb = 1;
  }
  return nb < kBlocksPerSm ? nb : kBlocksPerSm;
}

template <typename T>
IterGrid iter_grid(const rp_handle* h) {
  const int64_t want = (h->n + kThreads - 1) / kThreads;
  auto g = [&](int per_sm) {
    int64_t cap = (int64_t)h->num_sms * per_sm;
    return (int)(want < 1 ? 1 : want < cap ? want : cap);
  };
  const void* sl = (const void*)k_it_spmv_sl<T>;
  for (const void* f : {sl, (const void*)k_it_spmv_sl<T, true>, (const void*)k_it_spmv_sl_mp<T>})
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, SlStage<T>::kSmem) != cudaSuccess)
      cudaGetLastError();  // the launch reports it
  IterGrid gr;
  gr.k1 = g(resident((const void*)k_it_spmv<T>));
  gr.k1s = g(resident(kUseU4 && h->sl_u4 ? (const void*)k_it_spmv_sl<T, true> : sl, SlStage<T>::kSmem, kSlThreads));
  gr.k1sm = g(resident((const void*)k_it_spmv_sl_mp<T>, SlStage<T>::kSmem, kSlThreads));
  gr.k2 = g(resident((const void*)k_it_resid<T, false>));
  gr.k3 = g(resident((const void*)k_it_xp<T, false>));
  gr.k2l = g(resident((const void*)k_it_resid<T, true>));
  gr.k3l = g(resident((const void*)k_it_xp<T, true>));
  gr.k2s = g(resident((const void*)k_it_resid<T, false, true>));
  gr.k3s = g(resident((const void*)k_it_xp<T, false, true>));
  return gr;
}

}  // namespace

rp_status ensure_line_buffers(rp_handle* h) {
  const int64_t n = h->n + 64;
  RP_TRY(dalloc(&h->ln_l, n));
  RP_TRY(dalloc(&h->ln_w, n));
  RP_TRY(dalloc(&h->ln_g, n));
  RP_TRY(dalloc(&h->ln_z, n));
  if (h->want_fp32) {
    RP_TRY(dalloc(&h->ln_l32, n));
    RP_TRY(dalloc(&h->ln_w32, n));
    RP_TRY(dalloc(&h->ln_g32, n));
    RP_TRY(dalloc(&h->ln_z32, n));
  }
  return RP_OK;
}

rp_status line_factors(rp_handle* h, cudaStream_t s) {
  if (h->precond != RP_PRECOND_LINE || h->n == 0) return RP_OK;
  RP_TRY(ensure_line_buffers(h));
  const int g = grid_for(h, (h->n + 31) / 32);
  k_line_factors<<<g, kThreads, 0, s>>>(h->n, h->row_ptr, h->col_idx, h->vals, h->diag_pos, h->ln_l, h->ln_w,
                                        h->ln_g, h->ln_l32, h->ln_w32, h->ln_g32);
  RP_TRY_CUDA(cudaGetLastError());
  return RP_OK;
}

void free_line(rp_handle* h) {
  void* ptrs[] = {h->ln_l, h->ln_w, h->ln_g, h->ln_z, h->ln_l32, h->ln_w32, h->ln_g32, h->ln_z32};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  h->ln_l = h->ln_w = h->ln_g = h->ln_z = nullptr;
  h->ln_l32 = h->ln_w32 = h->ln_g32 = h->ln_z32 = nullptr;
}

rp_status ensure_solver_buffers(rp_handle* h) {
  h->igrid64 = iter_grid<double>(h);
  h->igrid32 = iter_grid<float>(h);
  if (h->precond == RP_PRECOND_LINE) RP_TRY(ensure_line_buffers(h));
  const int64_t n = h->n + 64;
  RP_TRY(dalloc(&h->r, n));
  RP_TRY(dalloc(&h->p, n));
  RP_TRY(dalloc(&h->q, n));
  if (h->want_fp32) {
    RP_TRY(dalloc(&h->r32, n));
    RP_TRY(dalloc(&h->p32, n));
    RP_TRY(dalloc(&h->q32, n));
    RP_TRY(dalloc(&h->d32, n));
  }
  RP_TRY(dalloc(&h->partials, (int64_t)h->num_sms * kBlocksPerSm * kMaxPartials));
  RP_TRY(dalloc(&h->ctl, 1));
  RP_TRY(dalloc(&h->io, 1));
  RP_TRY(dalloc(&h->ticket, 4));
  RP_TRY_CUDA(cudaMemset(h->ctl, 0, sizeof(Ctl)));
  RP_TRY_CUDA(cudaMemset(h->ticket, 0, 4 * sizeof(unsigned int)));
  return RP_OK;
}

void free_solver(rp_handle* h) {
  void* ptrs[] = {h->r, h->p, h->q, h->r32, h->p32, h->q32, h->d32, h->b_host_stage, h->x_host_stage,
                  h->partials, h->ctl, h->io, h->ticket, h->ctl_spmv};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  h->r = h->p = h->q = nullptr;
  h->r32 = h->p32 = h->q32 = h->d32 = nullptr;
  h->b_host_stage = h->x_host_stage = nullptr;
  h->partials = nullptr;
  h->ctl = nullptr;
  h->io = nullptr;
  h->ticket = nullptr;
  h->ctl_spmv = nullptr;
  if (h->graphs.fp64) cudaGraphExecDestroy(h->graphs.fp64);
  if (h->graphs.mixed) cudaGraphExecDestroy(h->graphs.mixed);
  if (h->graphs.mixed_ru) cudaGraphExecDestroy(h->graphs.mixed_ru);
  if (h->graphs.adjoint) cudaGraphExecDestroy(h->graphs.adjoint);
  h->graphs = Graphs{};
}

rp_status launch_solve(rp_handle* h, cudaGraphExec_t exec, const double* b, double* x, double tol, bool x_zero,
                       int max_iter, rp_solve_info* info, cudaStream_t s) {
  k_setup<<<1, 1, 0, s>>>(h->ctl, h->io, b, x, tol, h->opts.inner_tol, x_zero ? 1 : 0, max_iter,
                          h->opts.max_restarts, h->opts.max_outer, h->opts.ru_delta);
  RP_TRY_CUDA(cudaGetLastError());
  RP_TRY_CUDA(cudaGraphLaunch(exec, s));
  (void)info;
  return RP_OK;
}

rp_status read_info(rp_handle* h, rp_solve_info* info, cudaStream_t s) {
  Ctl c;
  RP_TRY_CUDA(cudaMemcpyAsync(&c, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  RP_TRY_CUDA(cudaStreamSynchronize(s));
  info->status = c.status < 0 ? RP_NOT_CONVERGED : c.status;
  info->iterations = c.iter_total;
  info->outer_iterations = c.outer;
  info->restarts = c.restarts;
  info->passes = c.pass;
  info->rel_residual = c.bb > 0.0 ? sqrt(c.rr / c.bb) : 0.0;
  return RP_OK;
}

// The kernel sequence of the solve graph, launched from the host: the
// control block is read back after every residual pass and every iteration.
rp_status host_loop_solve(rp_handle* h, int mode, const double* vals, const double* dinv, cudaStream_t s) {
  const bool mixed = mode != 0;
  SolveSet k = solve_set(h, mode, vals, dinv, 0, 0, 0);
  Ctl c;
  auto read = [&]() -> rp_status {
    RP_TRY_CUDA(cudaMemcpyAsync(&c, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    RP_TRY_CUDA(cudaStreamSynchronize(s));
    return RP_OK;
  };
  // same bounds as the graph: passes and iterations are capped on the device
  for (;;) {
    RP_TRY(launch1(k.res, h->grid, kThreads, 0, &k.ra, s));
    if (mode == 2) RP_TRY(launch1(k.rup, h->grid, kThreads, 0, &k.ru, s));
    RP_TRY(read());
    const bool go = !c.stop;
    while (!c.stop) {
      if (mixed) {
        launch_k1(k.a32, k1_grid(k.a32, h->igrid32), s);
        RP_TRY(launch1(k.k2_32, k.g2_32, kThreads, 0, &k.a32, s));
        RP_TRY(launch1(k.k3_32, k.g3_32, kThreads, 0, &k.a32, s));
      } else {
        launch_k1(k.a64, k1_grid(k.a64, h->igrid64), s);
        RP_TRY(launch1(k.k2_64, k.g2_64, kThreads, 0, &k.a64, s));
        RP_TRY(launch1(k.k3_64, k.g3_64, kThreads, 0, &k.a64, s));
      }
      RP_TRY_CUDA(cudaGetLastError());
      RP_TRY(read());
    }
    if (mixed) RP_TRY(launch1((void*)k_correct, h->grid, kThreads, 0, &k.ca, s));
    if (!go) break;
  }
  RP_TRY_CUDA(cudaGetLastError());
  return RP_OK;
}

rp_status solve_common(rp_handle* h, int mode, const double* vals, const double* dinv, cudaGraphExec_t* slot,
                       const double* b, double* x, double tol, int32_t x_is_guess, int32_t where,
                       rp_solve_info* info, cudaStream_t s) {
  if (!*slot && !h->opts.host_loop) RP_TRY(build_solve_graph(h, mode, vals, dinv, slot));
  const double* bd = b;
  double* xd = x;
  if (where == RP_MEM_HOST) {
    RP_TRY(dalloc(&h->b_host_stage, h->n + 64));
    RP_TRY(dalloc(&h->x_host_stage, h->n + 64));
    RP_TRY_CUDA(cudaMemcpyAsync(h->b_host_stage, b, 8 * h->n, cudaMemcpyHostToDevice, s));
    if (x_is_guess) RP_TRY_CUDA(cudaMemcpyAsync(h->x_host_stage, x, 8 * h->n, cudaMemcpyHostToDevice, s));
    bd = h->b_host_stage;
    xd = h->x_host_stage;
  }
  if (h->opts.host_loop) {
    k_setup<<<1, 1, 0, s>>>(h->ctl, h->io, bd, xd, tol, h->opts.inner_tol, x_is_guess ? 0 : 1, h->opts.max_iter,
                            h->opts.max_restarts, h->opts.max_outer, h->opts.ru_delta);
    RP_TRY(host_loop_solve(h, mode, vals, dinv, s));
  } else {
    RP_TRY(launch_solve(h, *slot, bd, xd, tol, !x_is_guess, h->opts.max_iter, info, s));
  }
  if (where == RP_MEM_HOST) RP_TRY_CUDA(cudaMemcpyAsync(x, h->x_host_stage, 8 * h->n, cudaMemcpyDeviceToHost, s));
  h->solve_ran = true;
  if (info) {
    RP_TRY(read_info(h, info, s));
    return (rp_status)info->status;
  }
  return RP_OK;
}

RP_CHECK_TU(pcg)

}  // namespace rp

using namespace rp;

extern "C" rp_status rp_solve(rp_handle* h, const double* b, double* x, double tol, int32_t precision,
                              int32_t x_is_guess, int32_t where, rp_solve_info* info, void* stream) {
  if (!h || (!b && h->n) || (!x && h->n)) return fail(RP_EINVAL, "null argument");
  if (!(tol >= 0.0)) return fail(RP_EINVAL, "tol must be >= 0");
  if (where != RP_MEM_DEVICE && where != RP_MEM_HOST) return fail(RP_EINVAL, "where must be RP_MEM_DEVICE or RP_MEM_HOST");
  if (precision != RP_FP64 && precision != RP_MIXED && precision != RP_MIXED_RU)
    return fail(RP_EINVAL, "precision must be RP_FP64, RP_MIXED or RP_MIXED_RU");
  if (precision != RP_FP64 && !h->want_fp32) return fail(RP_EINVAL, "mixed precision needs want_fp32");
  if (h->n == 0) {
    if (info) *info = rp_solve_info{RP_OK, 0, 0, 0, 0, 0.0};
    return RP_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (precision != RP_FP64 && h->precond == RP_PRECOND_JACOBI) {
    bool ok = false;
    RP_TRY(ensure_scaled(h, s, &ok));  // the inner FP32 iteration on S A S (sliced, one part)
  }
  if (precision == RP_MIXED)
    return solve_common(h, 1, h->vals, h->dinv, &h->graphs.mixed, b, x, tol, x_is_guess, where, info, s);
  if (precision == RP_MIXED_RU)
    return solve_common(h, 2, h->vals, h->dinv, &h->graphs.mixed_ru, b, x, tol, x_is_guess, where, info, s);
  return solve_common(h, 0, h->vals, h->dinv, &h->graphs.fp64, b, x, tol, x_is_guess, where, info, s);
}

extern "C" rp_status rp_get_solve_info(rp_handle* h, rp_solve_info* info, void* stream) {
  if (!h || !info) return fail(RP_EINVAL, "null argument");
  if (h->n == 0) {
    *info = rp_solve_info{RP_OK, 0, 0, 0, 0, 0.0};
    return RP_OK;
  }
  if (!h->solve_ran) return fail(RP_EINVAL, "no solve has run on this handle");
  RP_TRY(read_info(h, info, (cudaStream_t)stream));
  return (rp_status)info->status;
}

extern "C" rp_status rp_set_solver_options(rp_handle* h, const rp_options* o) {
  if (!h || !o) return fail(RP_EINVAL, "null argument");
  if (o->max_iter < 0 || o->max_outer < 0 || o->max_restarts < 0 || !(o->inner_tol > 0.0) ||
      !(o->ru_delta >= 0.0 && o->ru_delta < 1.0) || o->spin_limit < 0)
    return fail(RP_EINVAL, "invalid solver options");
  if (o->precond != RP_PRECOND_JACOBI && o->precond != RP_PRECOND_LINE)
    return fail(RP_EINVAL, "precond must be RP_PRECOND_JACOBI or RP_PRECOND_LINE");
  if (o->precond == RP_PRECOND_LINE && h->n_parts != 1)
    return fail(RP_EUNSUPPORTED, "the line preconditioner needs n_parts = 1");
  h->opts.max_iter = o->max_iter;
  h->opts.max_outer = o->max_outer;
  h->opts.max_restarts = o->max_restarts;
  h->opts.inner_tol = o->inner_tol;
  h->opts.ru_delta = o->ru_delta;
  h->opts.host_loop = o->host_loop;
  const bool new_precond = o->precond != h->precond, new_spin = o->spin_limit != h->opts.spin_limit;
  if (new_precond || new_spin) {  // both are part of the captured kernel arguments
    h->precond = o->precond;
    h->opts.precond = o->precond;
    h->opts.spin_limit = o->spin_limit;
    for (cudaGraphExec_t* g : {&h->graphs.fp64, &h->graphs.mixed, &h->graphs.mixed_ru, &h->graphs.adjoint})
      if (*g) {
        cudaGraphExecDestroy(*g);
        *g = nullptr;
      }
    drop_bicgstab_graph(h);
    if (new_precond) {
      RP_TRY(line_factors(h, 0));  // from the current values
      RP_TRY_CUDA(cudaStreamSynchronize(0));
    }
  }
  if (h->batch_ready) {  // the batched kernel's arguments are part of its graphs
    h->batch_args.max_iter = o->max_iter;
    h->batch_args.max_outer = o->max_outer;
    h->batch_args.max_restarts = o->max_restarts;
    h->batch_args.inner_tol = o->inner_tol;
    h->batch_args.ru_delta = o->ru_delta > 0.0 ? o->ru_delta : o->inner_tol;
    for (auto& g : h->batch_graphs)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
  }
  return RP_OK;
}

extern "C" rp_status rp_spmv(rp_handle* h, const double* x, double* y, double* xy, void* stream) {
  if (!h || (!x && h->n) || (!y && h->n)) return fail(RP_EINVAL, "null argument");
  if (h->n == 0) return RP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  k_spmv_plain<<<h->grid, kThreads, 0, s>>>(h->n, h->row_ptr, h->col_idx, h->vals, x, y, xy, h->partials, h->ticket,
                                            parts64(h));
  RP_TRY_CUDA(cudaGetLastError());
  return RP_OK;
}

extern "C" rp_status rp_iter_spmv(rp_handle* h, const void* x, void* y, int32_t precision, void* stream) {
  if (!h || (!x && h->n) || (!y && h->n)) return fail(RP_EINVAL, "null argument");
  if (precision != RP_FP64 && precision != RP_MIXED && precision != RP_MIXED_RU)
    return fail(RP_EINVAL, "precision must be RP_FP64, RP_MIXED or RP_MIXED_RU");
  if (precision != RP_FP64 && !h->want_fp32) return fail(RP_EINVAL, "mixed precision needs want_fp32");
  if (h->n == 0) return RP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  RP_TRY(dalloc(&h->ctl_spmv, 1));
  RP_TRY_CUDA(cudaMemsetAsync(h->ctl_spmv, 0, sizeof(Ctl), s));  // stop = 0, rz = 0
  if (precision == RP_FP64) {
    IterArgs<double> a{h->n, h->row_ptr, h->col_idx, h->vals, h->dinv, nullptr,
                       const_cast<double*>(static_cast<const double*>(x)), static_cast<double*>(y), nullptr,
                       h->ctl_spmv, h->io, h->partials, 0, 0, parts64(h), sliced64(h, h->vals)};
    launch_k1(a, k1_grid(a, h->igrid64), s);
  } else {
    IterArgs<float> a{h->n, h->row_ptr, h->col_idx, h->vals32, h->dinv32, nullptr,
                      const_cast<float*>(static_cast<const float*>(x)), static_cast<float*>(y), nullptr,
                      h->ctl_spmv, h->io, h->partials, 0, 0, parts32(h), sliced32(h)};
    launch_k1(a, k1_grid(a, h->igrid32), s);
  }
  RP_TRY_CUDA(cudaGetLastError());
  return RP_OK;
}

extern "C" rp_status rp_profile_iteration(rp_handle* h, const double* b, int32_t precision, int32_t iters,
                                          float* ms_out, void* stream) {
  if (!h || !b || !ms_out || iters < 1) return fail(RP_EINVAL, "invalid argument");
  if (precision != RP_FP64 && precision != RP_MIXED && precision != RP_MIXED_RU)
    return fail(RP_EINVAL, "precision must be RP_FP64, RP_MIXED or RP_MIXED_RU");
  if (precision != RP_FP64 && !h->want_fp32) return fail(RP_EINVAL, "mixed precision needs want_fp32");
  if (h->n == 0) return fail(RP_EINVAL, "empty system");
  cudaStream_t s = (cudaStream_t)stream;
  const bool mixed = precision != RP_FP64;  // both mixed modes run the same FP32 iteration kernels
  if (mixed && h->precond == RP_PRECOND_JACOBI) {
    bool ok = false;
    RP_TRY(ensure_scaled(h, s, &ok));  // the kernels the mixed solves run
  }
  RP_TRY(dalloc(&h->x_host_stage, h->n + 64));
  // a fresh CG run from x = 0 that never meets its tolerance (tol = 0)
  k_setup<<<1, 1, 0, s>>>(h->ctl, h->io, b, h->x_host_stage, 0.0, 0.0, 1, iters + 2, 0, 1);
  SolveSet k = solve_set(h, mixed ? 1 : 0, h->vals, h->dinv, 0, 0, 0);
  RP_TRY(launch1(k.res, h->grid, kThreads, 0, &k.ra, s));
  std::vector<cudaEvent_t> ev(3 * iters + 1, nullptr);
  struct EvFree {
    std::vector<cudaEvent_t>& v;
    ~EvFree() {
      for (auto e : v)
        if (e) cudaEventDestroy(e);
    }
  } evfree{ev};
  for (auto& e : ev) RP_TRY_CUDA(cudaEventCreate(&e));
  RP_TRY_CUDA(cudaEventRecord(ev[0], s));
  for (int it = 0; it < iters; ++it) {
    if (mixed) launch_k1(k.a32, k1_grid(k.a32, h->igrid32), s);
    else launch_k1(k.a64, k1_grid(k.a64, h->igrid64), s);
    RP_TRY_CUDA(cudaEventRecord(ev[3 * it + 1], s));
    if (mixed) RP_TRY(launch1(k.k2_32, k.g2_32, kThreads, 0, &k.a32, s));
    else RP_TRY(launch1(k.k2_64, k.g2_64, kThreads, 0, &k.a64, s));
    RP_TRY_CUDA(cudaEventRecord(ev[3 * it + 2], s));
    if (mixed) RP_TRY(launch1(k.k3_32, k.g3_32, kThreads, 0, &k.a32, s));
    else RP_TRY(launch1(k.k3_64, k.g3_64, kThreads, 0, &k.a64, s));
    RP_TRY_CUDA(cudaEventRecord(ev[3 * it + 3], s));
  }
  RP_TRY_CUDA(cudaGetLastError());
  RP_TRY_CUDA(cudaStreamSynchronize(s));
  double acc[3] = {0, 0, 0};
  for (int it = 0; it < iters; ++it)
    for (int kk = 0; kk < 3; ++kk) {
      float ms = 0.f;
      RP_TRY_CUDA(cudaEventElapsedTime(&ms, ev[3 * it + kk], ev[3 * it + kk + 1]));
      acc[kk] += ms;
    }
  for (int kk = 0; kk < 3; ++kk) ms_out[kk] = (float)(acc[kk] / iters);
  Ctl c;
  RP_TRY_CUDA(cudaMemcpy(&c, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  if (c.status == RP_BREAKDOWN) return fail(RP_BREAKDOWN, "iteration broke down while being timed");
  return RP_OK;
}
