// Jacobi-preconditioned BiCGStab (van der Vorst, 1992) on the merged matrix:
// the solver of the non-symmetric momentum system (the paper solves momentum
// with BiCGStab, pressure with CG; Sec. 4). FP64 throughout, or (mixed) an
// FP32 BiCGStab on the FP32 values inside FP64 iterative refinement.
//
// One CUDA graph per handle: while (outer) { residual pass; while (inner) {
// B1; B2; B3; B4; B5 } }, every loop bounded by device counters.
//   residual pass  r = b - A x, rhat = r, p = v = 0, (r, r) [, (b, b)]; decides
//   B1             beta = (rho / rho_old)(alpha / omega); p = r + beta (p - omega v); phat = D^-1 p
//   B2 (SpMV)      v = A phat, (rhat, v) -> alpha = rho / (rhat, v)
//   B3             s = r - alpha v; shat = D^-1 s; (s, s) -> half step when ||s|| <= tol ||b||
//   B4 (SpMV)      t = A shat, (t, s), (t, t) -> omega
//   B5             x += alpha phat + omega shat; r = s - omega t; (r, r), (rhat, r) -> rho, stop
//                  (half step: x += alpha phat, r = s, stop)
// A recursive residual at the target ends the inner loop; the residual pass
// then confirms it with b - A x or restarts from the true residual with a
// new shadow residual (bounded by max_restarts). Scalars live in device
// memory and are written only by the last block of a kernel. The SpMVs run
// over the sliced layout when the handle has it (spmv_sl_body), else CSR.
//
// Mixed: while (outer) { FP64 residual pass r = b - A x, r32 = fl(r), d = 0;
// while (inner) { B1..B5 in FP32 on d } ; x += d }, the inner loop stopping
// at inner_tol relative to its start (a new shadow residual every pass).
//
// Roofline: FP64-FMA bound on GB300 (one FMA per stored entry per product,
// two products per iteration, ~14 FP64 instructions per row in B1/B3/B5); the
// FP32 inner loop is bound by HBM and the products' gathers instead.
#include "rp_common.cuh"
#include "rp_spmv.cuh"

namespace rp {

struct BsCtl {
  double bb, thresh, tol, rr, ss;
  double rho, rho_old, alpha, omega;
  double ithresh, inner_tol;  // the inner loop's target: thresh (FP64); inner_tol^2 (r32, r32) (mixed)
  int32_t iter, max_iter, stop, status, pass, restarts, max_restarts, half, x_zero;
  int32_t outer, max_outer;
  unsigned int ticket;
};

// the vectors and the matrix of one working precision
template <typename T>
struct BsVecs {
  const T* vals;
  const T* dinv;
  Parts<T> parts;
  Sliced<T> sl;
  T *r, *rhat, *p, *v, *s, *t, *phat, *shat;
  T* x;  // FP32: the correction d; FP64: unused (the caller's x, through SolveIO)
};

struct BsArgs {
  int64_t n;
  const int32_t* row_ptr;
  const int32_t* col;
  BsVecs<double> d;  // FP64 solve; its matrix also serves the residual passes
  BsVecs<float> f;   // FP32 inner solve (mixed)
  BsCtl* c;
  SolveIO* io;
  double* partials;
  cudaGraphConditionalHandle inner, outer;
  int in_graph;
};

struct BsState {
  double *rhat = nullptr, *s = nullptr, *t = nullptr, *phat = nullptr, *shat = nullptr;
  float *rhat32 = nullptr, *s32 = nullptr, *t32 = nullptr, *phat32 = nullptr, *shat32 = nullptr;
  BsCtl* ctl = nullptr;
  SolveIO* io = nullptr;
  cudaGraphExec_t graph = nullptr, graph_mixed = nullptr;
  int grid_vec = 1, grid_sl = 1, grid_sl32 = 1;
};

namespace {

template <typename T>
__device__ __forceinline__ const BsVecs<T>& vecs(const BsArgs& a);
template <>
__device__ __forceinline__ const BsVecs<double>& vecs<double>(const BsArgs& a) {
  return a.d;
}
template <>
__device__ __forceinline__ const BsVecs<float>& vecs<float>(const BsArgs& a) {
  return a.f;
}

__global__ void k_bs_setup(BsCtl* c, SolveIO* io, const double* b, double* x, double tol, int x_zero, int max_iter,
                           int max_restarts, int max_outer, double inner_tol) {
  io->b = b;
  io->x = x;
  c->tol = tol;
  c->x_zero = x_zero;
  c->max_iter = max_iter;
  c->max_restarts = max_restarts;
  c->max_outer = max_outer;
  c->inner_tol = inner_tol;
  c->outer = 0;
  c->iter = 0;
  c->pass = 0;
  c->restarts = 0;
  c->status = -1;
  c->stop = 0;
  c->half = 0;
  c->ticket = 0u;
}

// residual pass: r = b - A x (cold start: r = b, x = 0), rhat = r, p = v = 0
__global__ void __launch_bounds__(kThreads) k_bs_res(BsArgs a) {
  BsCtl* c = a.c;
  const bool first = c->pass == 0;
  const bool cold = first && c->x_zero;
  const double* __restrict__ b = a.io->b;
  double* __restrict__ x = a.io->x;
  double rr = 0.0, bb = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = b[i];
    double ri;
    if (cold) {
      ri = bi;
      x[i] = 0.0;
    } else {
      ri = bi - row_dot_any<double>(a.d.parts, a.row_ptr, a.col, a.d.vals, x, i, a.n);
    }
    a.d.r[i] = ri;
    a.d.rhat[i] = ri;
    a.d.p[i] = 0.0;
    a.d.v[i] = 0.0;
    rr += ri * ri;
    bb += bi * bi;
  }
  double v[2] = {rr, bb}, tot[2];
  if (reduce_last_block<2>(v, a.partials, &c->ticket, tot) && threadIdx.x == 0) {
    if (first) {
      c->bb = tot[1];
      c->thresh = c->tol * c->tol * tot[1];
    }
    c->rr = tot[0];
    c->pass += 1;
    bool go = false;
    if (tot[0] <= c->thresh) {
      c->status = RP_OK;
    } else if (c->status == RP_BREAKDOWN || c->status == RP_DEVICE_TIMEOUT) {
    } else if (!isfinite(tot[0])) {
      c->status = RP_BREAKDOWN;
    } else if (c->iter >= c->max_iter || (!first && c->restarts >= c->max_restarts)) {
      c->status = RP_NOT_CONVERGED;
    } else {
      if (!first) c->restarts += 1;
      c->rho = tot[0];  // (rhat, r) with rhat = r
      c->rho_old = c->alpha = c->omega = 1.0;
      c->half = 0;
      c->ithresh = c->thresh;
      go = true;
    }
    c->stop = go ? 0 : 1;
    if (a.in_graph) {
      cudaGraphSetConditional(a.inner, go ? 1u : 0u);
      cudaGraphSetConditional(a.outer, go ? 1u : 0u);
    }
  }
}

// mixed residual pass: r = b - A x in FP64 (cold start: r = b, x = 0); the FP32
// inner solve starts from r32 = fl(r), rhat = r32, p = v = d = 0; decides
__global__ void __launch_bounds__(kThreads) k_bs_res_mixed(BsArgs a) {
  BsCtl* c = a.c;
  const bool first = c->pass == 0;
  const bool cold = first && c->x_zero;
  const double* __restrict__ b = a.io->b;
  double* __restrict__ x = a.io->x;
  const BsVecs<float>& F = a.f;
  double rr = 0.0, bb = 0.0;
  float ff = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = b[i];
    double ri;
    if (cold) {
      ri = bi;
      x[i] = 0.0;
    } else {
      ri = bi - row_dot_any<double>(a.d.parts, a.row_ptr, a.col, a.d.vals, x, i, a.n);
    }
    const float r32 = (float)ri;
    F.r[i] = r32;
    F.rhat[i] = r32;
    F.p[i] = 0.f;
    F.v[i] = 0.f;
    F.x[i] = 0.f;
    rr += ri * ri;
    bb += bi * bi;
    ff = fmaf(r32, r32, ff);
  }
  double v[3] = {rr, bb, (double)ff}, tot[3];
  if (reduce_last_block<3>(v, a.partials, &c->ticket, tot) && threadIdx.x == 0) {
    if (first) {
      c->bb = tot[1];
      c->thresh = c->tol * c->tol * tot[1];
    }
    c->rr = tot[0];
    c->pass += 1;
    bool go = false;
    if (tot[0] <= c->thresh) {
      c->status = RP_OK;
    } else if (c->status == RP_BREAKDOWN || c->status == RP_DEVICE_TIMEOUT) {
    } else if (!isfinite(tot[0])) {
      c->status = RP_BREAKDOWN;
    } else if (c->iter >= c->max_iter || c->outer >= c->max_outer) {
      c->status = RP_NOT_CONVERGED;
    } else {
      c->outer += 1;
      c->rho = tot[2];  // (rhat, r) with rhat = r32
      c->rho_old = c->alpha = c->omega = 1.0;
      c->half = 0;
      c->ithresh = c->inner_tol * c->inner_tol * tot[2];
      go = true;
    }
    c->stop = go ? 0 : 1;
    if (a.in_graph) {
      cudaGraphSetConditional(a.inner, go ? 1u : 0u);
      cudaGraphSetConditional(a.outer, go ? 1u : 0u);
    }
  }
}

// x += d in FP64 after an inner solve (not after a breakdown or a timeout, nor
// when the residual pass has ended the solve)
__global__ void __launch_bounds__(kThreads) k_bs_correct(BsArgs a) {
  if (a.c->status >= 0) return;
  double* __restrict__ x = a.io->x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += (double)a.f.x[i];
}

// B1: p = r + beta (p - omega v); phat = D^-1 p
template <typename T>
__global__ void __launch_bounds__(kThreads) k_bs_p(BsArgs a) {
  const BsCtl* c = a.c;
  if (c->stop) return;
  const BsVecs<T>& V = vecs<T>(a);
  const T beta = (T)((c->rho / c->rho_old) * (c->alpha / c->omega)), omega = (T)c->omega;
  int64_t i0 = 0;
  if constexpr (sizeof(T) == 4) {
    // FP32: 16-byte vectors, two of each stream in flight per thread
    const float4* __restrict__ R = reinterpret_cast<const float4*>(V.r);
    const float4* __restrict__ Vv = reinterpret_cast<const float4*>(V.v);
    const float4* __restrict__ D = reinterpret_cast<const float4*>(V.dinv);
    float4* __restrict__ P = reinterpret_cast<float4*>(V.p);
    float4* __restrict__ H = reinterpret_cast<float4*>(V.phat);
    auto step = [&](float4& p, const float4& r, const float4& v, const float4& d, float4& h) {
      p.x = fmaf(beta, fmaf(-omega, v.x, p.x), r.x);
      p.y = fmaf(beta, fmaf(-omega, v.y, p.y), r.y);
      p.z = fmaf(beta, fmaf(-omega, v.z, p.z), r.z);
      p.w = fmaf(beta, fmaf(-omega, v.w, p.w), r.w);
      h = make_float4(d.x * p.x, d.y * p.y, d.z * p.z, d.w * p.w);
    };
    const int64_t stride = (int64_t)gridDim.x * blockDim.x, nv = a.n / 4;
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; k + stride < nv; k += 2 * stride) {
      float4 p0 = P[k], p1 = P[k + stride], h0, h1;
      const float4 r0 = R[k], r1 = R[k + stride], v0 = Vv[k], v1 = Vv[k + stride], d0 = D[k], d1 = D[k + stride];
      step(p0, r0, v0, d0, h0);
      step(p1, r1, v1, d1, h1);
      P[k] = p0;
      P[k + stride] = p1;
      H[k] = h0;
      H[k + stride] = h1;
    }
    for (; k < nv; k += stride) {
      float4 p0 = P[k], h0;
      step(p0, R[k], Vv[k], D[k], h0);
      P[k] = p0;
      H[k] = h0;
    }
    i0 = nv * 4;
  }
  for (int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T pi = fma(beta, fma(-omega, V.v[i], V.p[i]), V.r[i]);
    V.p[i] = pi;
    V.phat[i] = V.dinv[i] * pi;
  }
}

// B2 epilogue: (rhat, v) -> alpha
template <typename T>
struct BsEpiV {
  const T* rhat;
  BsCtl* c;
  double* partials;
  T acc = T(0);
  __device__ __forceinline__ void row(int64_t i, T y) { acc = fma(rhat[i], y, acc); }
  __device__ __forceinline__ void timeout() {
    c->status = RP_DEVICE_TIMEOUT;
    c->stop = 1;
  }
  __device__ __forceinline__ void finish() {
    double v[1] = {(double)acc}, tot[1];
    if (reduce_last_block<1>(v, partials, &c->ticket, tot) && threadIdx.x == 0) {
      if (c->status == RP_DEVICE_TIMEOUT) {
        c->stop = 1;
      } else if (tot[0] == 0.0 || !isfinite(tot[0])) {
        c->status = RP_BREAKDOWN;
        c->stop = 1;
      } else {
        c->alpha = c->rho / tot[0];
      }
    }
  }
};

// B4 epilogue: (t, s), (t, t) -> omega
template <typename T>
struct BsEpiT {
  const T* s;
  BsCtl* c;
  double* partials;
  T ts = T(0), tt = T(0);
  __device__ __forceinline__ void row(int64_t i, T y) {
    ts = fma(y, s[i], ts);
    tt = fma(y, y, tt);
  }
  __device__ __forceinline__ void timeout() {
    c->status = RP_DEVICE_TIMEOUT;
    c->stop = 1;
  }
  __device__ __forceinline__ void finish() {
    double v[2] = {(double)ts, (double)tt}, tot[2];
    if (reduce_last_block<2>(v, partials, &c->ticket, tot) && threadIdx.x == 0) {
      const double omega = tot[0] / tot[1];
      if (c->status == RP_DEVICE_TIMEOUT) {
        c->stop = 1;
      } else if (!(tot[1] > 0.0) || !isfinite(omega)) {
        c->status = RP_BREAKDOWN;
        c->stop = 1;
      } else {
        c->omega = omega;
      }
    }
  }
};

// B2 / B4 over CSR (any number of parts) or the sliced layout
template <int WHICH, typename T>
__global__ void __launch_bounds__(kThreads) k_bs_spmv(BsArgs a) {
  BsCtl* c = a.c;
  if (c->stop || (WHICH == 2 && c->half)) return;
  const BsVecs<T>& V = vecs<T>(a);
  if constexpr (WHICH == 1) {
    BsEpiV<T> e{V.rhat, c, a.partials};
    spmv_csr_body<T>(a.n, V.parts, a.row_ptr, a.col, V.vals, V.phat, V.v, e);
  } else {
    BsEpiT<T> e{V.s, c, a.partials};
    spmv_csr_body<T>(a.n, V.parts, a.row_ptr, a.col, V.vals, V.shat, V.t, e);
  }
}
template <int WHICH, bool MP, typename T>
__global__ void __launch_bounds__(kSlThreads, sizeof(T) == 4 ? 7 : 5) k_bs_spmv_sl(BsArgs a) {
  BsCtl* c = a.c;
  if (c->stop || (WHICH == 2 && c->half)) return;
  const BsVecs<T>& V = vecs<T>(a);
  if constexpr (WHICH == 1) {
    BsEpiV<T> e{V.rhat, c, a.partials};
    spmv_sl_body<T, MP>(V.sl, V.parts, a.n, V.phat, V.v, e);
  } else {
    BsEpiT<T> e{V.s, c, a.partials};
    spmv_sl_body<T, MP>(V.sl, V.parts, a.n, V.shat, V.t, e);
  }
}

// B3: s = r - alpha v; shat = D^-1 s; (s, s)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_bs_s(BsArgs a) {
  BsCtl* c = a.c;
  if (c->stop) return;
  const BsVecs<T>& V = vecs<T>(a);
  const T alpha = (T)c->alpha;
  T ss = T(0);
  int64_t i0 = 0;
  if constexpr (sizeof(T) == 4) {
    const float4* __restrict__ R = reinterpret_cast<const float4*>(V.r);
    const float4* __restrict__ Vv = reinterpret_cast<const float4*>(V.v);
    const float4* __restrict__ D = reinterpret_cast<const float4*>(V.dinv);
    float4* __restrict__ Sv = reinterpret_cast<float4*>(V.s);
    float4* __restrict__ H = reinterpret_cast<float4*>(V.shat);
    auto step = [&](const float4& r, const float4& v, const float4& d, float4& s, float4& h) {
      s = make_float4(fmaf(-alpha, v.x, r.x), fmaf(-alpha, v.y, r.y), fmaf(-alpha, v.z, r.z), fmaf(-alpha, v.w, r.w));
      h = make_float4(d.x * s.x, d.y * s.y, d.z * s.z, d.w * s.w);
      ss = fmaf(s.x, s.x, ss);
      ss = fmaf(s.y, s.y, ss);
      ss = fmaf(s.z, s.z, ss);
      ss = fmaf(s.w, s.w, ss);
    };
    const int64_t stride = (int64_t)gridDim.x * blockDim.x, nv = a.n / 4;
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; k + stride < nv; k += 2 * stride) {
      const float4 r0 = R[k], r1 = R[k + stride], v0 = Vv[k], v1 = Vv[k + stride], d0 = D[k], d1 = D[k + stride];
      float4 s0, s1, h0, h1;
      step(r0, v0, d0, s0, h0);
      step(r1, v1, d1, s1, h1);
      Sv[k] = s0;
      Sv[k + stride] = s1;
      H[k] = h0;
      H[k + stride] = h1;
    }
    for (; k < nv; k += stride) {
      float4 s0, h0;
      step(R[k], Vv[k], D[k], s0, h0);
      Sv[k] = s0;
      H[k] = h0;
    }
    i0 = nv * 4;
  }
  for (int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T si = fma(-alpha, V.v[i], V.r[i]);
    V.s[i] = si;
    V.shat[i] = V.dinv[i] * si;
    ss = fma(si, si, ss);
  }
  double v[1] = {(double)ss}, tot[1];
  if (reduce_last_block<1>(v, a.partials, &c->ticket, tot) && threadIdx.x == 0) {
    c->ss = tot[0];
    c->half = tot[0] <= c->ithresh ? 1 : 0;
  }
}

// B5: x += alpha phat + omega shat; r = s - omega t; (r, r), (rhat, r)
// (half step: x += alpha phat; r = s); decides the next iteration
template <typename T>
__global__ void __launch_bounds__(kThreads) k_bs_xr(BsArgs a) {
  BsCtl* c = a.c;
  if (c->stop) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.in_graph) cudaGraphSetConditional(a.inner, 0);
    return;
  }
  const BsVecs<T>& V = vecs<T>(a);
  const bool half = c->half;
  const T alpha = (T)c->alpha, omega = (T)c->omega;
  T* __restrict__ x;
  if constexpr (sizeof(T) == 8) x = a.io->x;
  else x = V.x;
  T rr = T(0), rhr = T(0);
  int64_t i0 = 0;
  if constexpr (sizeof(T) == 4) {
    const float4* __restrict__ PH = reinterpret_cast<const float4*>(V.phat);
    const float4* __restrict__ SH = reinterpret_cast<const float4*>(V.shat);
    const float4* __restrict__ Tt = reinterpret_cast<const float4*>(V.t);
    const float4* __restrict__ Sv = reinterpret_cast<const float4*>(V.s);
    const float4* __restrict__ RH = reinterpret_cast<const float4*>(V.rhat);
    float4* __restrict__ X = reinterpret_cast<float4*>(x);
    float4* __restrict__ R = reinterpret_cast<float4*>(V.r);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x, nv = a.n / 4;
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (half) {
      for (; k < nv; k += stride) {
        const float4 ph = PH[k];
        float4 xv = X[k];
        xv = make_float4(fmaf(alpha, ph.x, xv.x), fmaf(alpha, ph.y, xv.y), fmaf(alpha, ph.z, xv.z),
                         fmaf(alpha, ph.w, xv.w));
        X[k] = xv;
        R[k] = Sv[k];
      }
    } else {
      auto step = [&](float4& xv, const float4& ph, const float4& sh, const float4& t, const float4& s,
                      const float4& rh, float4& r) {
        xv = make_float4(fmaf(omega, sh.x, fmaf(alpha, ph.x, xv.x)), fmaf(omega, sh.y, fmaf(alpha, ph.y, xv.y)),
                         fmaf(omega, sh.z, fmaf(alpha, ph.z, xv.z)), fmaf(omega, sh.w, fmaf(alpha, ph.w, xv.w)));
        r = make_float4(fmaf(-omega, t.x, s.x), fmaf(-omega, t.y, s.y), fmaf(-omega, t.z, s.z),
                        fmaf(-omega, t.w, s.w));
        rr = fmaf(r.x, r.x, rr);
        rr = fmaf(r.y, r.y, rr);
        rr = fmaf(r.z, r.z, rr);
        rr = fmaf(r.w, r.w, rr);
        rhr = fmaf(rh.x, r.x, rhr);
        rhr = fmaf(rh.y, r.y, rhr);
        rhr = fmaf(rh.z, r.z, rhr);
        rhr = fmaf(rh.w, r.w, rhr);
      };
      for (; k + stride < nv; k += 2 * stride) {
        float4 x0 = X[k], x1 = X[k + stride], r0, r1;
        const float4 ph0 = PH[k], ph1 = PH[k + stride], sh0 = SH[k], sh1 = SH[k + stride];
        const float4 t0 = Tt[k], t1 = Tt[k + stride], s0 = Sv[k], s1 = Sv[k + stride];
        const float4 rh0 = RH[k], rh1 = RH[k + stride];
        step(x0, ph0, sh0, t0, s0, rh0, r0);
        step(x1, ph1, sh1, t1, s1, rh1, r1);
        X[k] = x0;
        X[k + stride] = x1;
        R[k] = r0;
        R[k + stride] = r1;
      }
      for (; k < nv; k += stride) {
        float4 x0 = X[k], r0;
        step(x0, PH[k], SH[k], Tt[k], Sv[k], RH[k], r0);
        X[k] = x0;
        R[k] = r0;
      }
    }
    i0 = nv * 4;
  }
  for (int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (half) {
      x[i] = fma(alpha, V.phat[i], x[i]);
      V.r[i] = V.s[i];
    } else {
      x[i] = fma(omega, V.shat[i], fma(alpha, V.phat[i], x[i]));
      const T ri = fma(-omega, V.t[i], V.s[i]);
      V.r[i] = ri;
      rr = fma(ri, ri, rr);
      rhr = fma(V.rhat[i], ri, rhr);
    }
  }
  double v[2] = {(double)rr, (double)rhr}, tot[2];
  if (reduce_last_block<2>(v, a.partials, &c->ticket, tot) && threadIdx.x == 0) {
    c->iter += 1;
    if (half) {
      c->rr = c->ss;
      c->stop = 1;  // the residual pass confirms with b - A x
    } else {
      c->rr = tot[0];
      if (tot[0] <= c->ithresh) {
        c->stop = 1;
      } else if (c->iter >= c->max_iter) {
        c->stop = 1;
      } else if (c->omega == 0.0 || tot[1] == 0.0 || !isfinite(tot[1])) {
        c->status = RP_BREAKDOWN;
        c->stop = 1;
      } else {
        c->rho_old = c->rho;
        c->rho = tot[1];
      }
    }
    if (a.in_graph) cudaGraphSetConditional(a.inner, c->stop ? 0u : 1u);
  }
}

int resident_blocks(const void* fn, int threads, int smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess || nb < 1) {
    cudaGetLastError();
    nb = 1;
  }
  return nb < kBlocksPerSm ? nb : kBlocksPerSm;
}

template <typename T>
rp_status balloc(T** p, int64_t count) {
  if (*p) return RP_OK;
  if (count <= 0) count = 1;
  if (cudaMalloc((void**)p, (size_t)count * sizeof(T)) != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(RP_ENOMEM, "cudaMalloc of %lld bytes failed", (long long)(count * sizeof(T)));
  }
  return RP_OK;
}

rp_status ensure_bs(rp_handle* h) {
  if (!h->bs) h->bs = new BsState();
  BsState* b = h->bs;
  const int64_t n = h->n + 64;
  RP_TRY(balloc(&b->rhat, n));
  RP_TRY(balloc(&b->s, n));
  RP_TRY(balloc(&b->t, n));
  RP_TRY(balloc(&b->phat, n));
  RP_TRY(balloc(&b->shat, n));
  RP_TRY(balloc(&b->ctl, 1));
  RP_TRY(balloc(&b->io, 1));
  if (h->want_fp32) {
    RP_TRY(balloc(&b->rhat32, n));
    RP_TRY(balloc(&b->s32, n));
    RP_TRY(balloc(&b->t32, n));
    RP_TRY(balloc(&b->phat32, n));
    RP_TRY(balloc(&b->shat32, n));
  }
  const int64_t want = (h->n + kThreads - 1) / kThreads;
  auto grid = [&](int per_sm) {
    const int64_t cap = (int64_t)h->num_sms * per_sm;
    return (int)(want < 1 ? 1 : want < cap ? want : cap);
  };
  b->grid_vec = grid(resident_blocks((const void*)k_bs_xr<double>, kThreads, 0));
  b->grid_sl = grid(resident_blocks((const void*)k_bs_spmv_sl<2, false, double>, kSlThreads, SlStage<double>::kSmem));
  b->grid_sl32 = grid(resident_blocks((const void*)k_bs_spmv_sl<2, false, float>, kSlThreads, SlStage<float>::kSmem));
  return RP_OK;
}

BsArgs bs_args(rp_handle* h, cudaGraphConditionalHandle inner, cudaGraphConditionalHandle outer, int in_graph) {
  BsState* b = h->bs;
  BsArgs a{};
  a.n = h->n;
  a.row_ptr = h->row_ptr;
  a.col = h->col_idx;
  a.d.vals = h->vals;
  a.d.dinv = h->dinv;
  a.d.parts = parts64(h);
  a.d.sl = sliced64(h, h->vals);
  a.d.r = h->r;
  a.d.rhat = b->rhat;
  a.d.p = h->p;
  a.d.v = h->q;
  a.d.s = b->s;
  a.d.t = b->t;
  a.d.phat = b->phat;
  a.d.shat = b->shat;
  a.d.x = nullptr;
  if (h->want_fp32) {
    a.f.vals = h->vals32;
    a.f.dinv = h->dinv32;
    a.f.parts = parts32(h);
    a.f.sl = sliced32(h);
    a.f.r = h->r32;
    a.f.rhat = b->rhat32;
    a.f.p = h->p32;
    a.f.v = h->q32;
    a.f.s = b->s32;
    a.f.t = b->t32;
    a.f.phat = b->phat32;
    a.f.shat = b->shat32;
    a.f.x = h->d32;
  }
  a.c = b->ctl;
  a.io = b->io;
  a.partials = h->partials;
  a.inner = inner;
  a.outer = outer;
  a.in_graph = in_graph;
  return a;
}

rp_status node(cudaGraph_t g, cudaGraphNode_t* out, const cudaGraphNode_t* dep, void* fn, int grid, int threads,
               int smem, void* argp) {
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeKernel;
  np.kernel.func = fn;
  np.kernel.gridDim = dim3((unsigned)grid);
  np.kernel.blockDim = dim3((unsigned)threads);
  np.kernel.sharedMemBytes = (unsigned)smem;
  void* args[1] = {argp};
  np.kernel.kernelParams = args;
  RP_TRY_CUDA(cudaGraphAddNode(out, g, dep, nullptr, dep ? 1 : 0, &np));
  return RP_OK;
}

rp_status while_node(cudaGraph_t g, cudaGraphNode_t* out, const cudaGraphNode_t* dep, cudaGraphConditionalHandle hnd,
                     cudaGraph_t* body) {
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = hnd;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  RP_TRY_CUDA(cudaGraphAddNode(out, g, dep, nullptr, dep ? 1 : 0, &np));
  *body = np.conditional.phGraph_out[0];
  return RP_OK;
}

// the five inner kernels with their launch shapes
struct BsLaunch {
  void* fn;
  int grid, threads, smem;
};
template <typename T>
void bs_inner(const rp_handle* h, BsLaunch (&k)[5]) {
  const BsState* b = h->bs;
  const bool sl = h->sl_slices > 0 && (sizeof(T) == 8 || h->sl_vals32);  // as sliced64 / sliced32
  const int gs = sl ? (sizeof(T) == 8 ? b->grid_sl : b->grid_sl32) : h->grid, ts = sl ? kSlThreads : kThreads;
  const int ms = sl ? SlStage<T>::kSmem : 0;
  const bool mp = h->sl_srow != nullptr;
  k[0] = {(void*)k_bs_p<T>, b->grid_vec, kThreads, 0};
  k[1] = {sl ? (mp ? (void*)k_bs_spmv_sl<1, true, T> : (void*)k_bs_spmv_sl<1, false, T>) : (void*)k_bs_spmv<1, T>, gs,
          ts, ms};
  k[2] = {(void*)k_bs_s<T>, b->grid_vec, kThreads, 0};
  k[3] = {sl ? (mp ? (void*)k_bs_spmv_sl<2, true, T> : (void*)k_bs_spmv_sl<2, false, T>) : (void*)k_bs_spmv<2, T>, gs,
          ts, ms};
  k[4] = {(void*)k_bs_xr<T>, b->grid_vec, kThreads, 0};
}

// mixed: the FP64 residual pass, the FP32 inner loop, then the correction
rp_status build_bs_graph(rp_handle* h, bool mixed, cudaGraphExec_t* exec) {
  cudaGraph_t top = nullptr;
  RP_TRY_CUDA(cudaGraphCreate(&top, 0));
  struct Guard {
    cudaGraph_t g;
    ~Guard() { cudaGraphDestroy(g); }
  } guard{top};
  cudaGraphConditionalHandle hout, hin;
  RP_TRY_CUDA(cudaGraphConditionalHandleCreate(&hout, top, 1, cudaGraphCondAssignDefault));
  cudaGraphNode_t wout, nres, win, nk[5];
  cudaGraph_t obody = nullptr, ibody = nullptr;
  RP_TRY(while_node(top, &wout, nullptr, hout, &obody));
  RP_TRY_CUDA(cudaGraphConditionalHandleCreate(&hin, obody, 0, 0));
  BsArgs a = bs_args(h, hin, hout, 1);
  RP_TRY(node(obody, &nres, nullptr, mixed ? (void*)k_bs_res_mixed : (void*)k_bs_res, h->grid, kThreads, 0, &a));
  RP_TRY(while_node(obody, &win, &nres, hin, &ibody));
  BsLaunch k[5];
  if (mixed) bs_inner<float>(h, k);
  else bs_inner<double>(h, k);
  for (int j = 0; j < 5; ++j)
    RP_TRY(node(ibody, &nk[j], j ? &nk[j - 1] : nullptr, k[j].fn, k[j].grid, k[j].threads, k[j].smem, &a));
  if (mixed) {
    cudaGraphNode_t ncor;
    RP_TRY(node(obody, &ncor, &win, (void*)k_bs_correct, h->bs->grid_vec, kThreads, 0, &a));
  }
  RP_TRY_CUDA(cudaGraphInstantiate(exec, top, 0));
  return RP_OK;
}

// the same kernel sequence launched from the host (profilers that cannot see
// inside conditional graphs); the control block is read after every kernel group
rp_status bs_host_loop(rp_handle* h, bool mixed, cudaStream_t s) {
  BsArgs a = bs_args(h, 0, 0, 0);
  BsLaunch k[5];
  if (mixed) bs_inner<float>(h, k);
  else bs_inner<double>(h, k);
  BsCtl c;
  for (;;) {
    if (mixed) k_bs_res_mixed<<<h->grid, kThreads, 0, s>>>(a);
    else k_bs_res<<<h->grid, kThreads, 0, s>>>(a);
    RP_TRY_CUDA(cudaGetLastError());
    RP_TRY_CUDA(cudaMemcpyAsync(&c, h->bs->ctl, sizeof(BsCtl), cudaMemcpyDeviceToHost, s));
    RP_TRY_CUDA(cudaStreamSynchronize(s));
    if (c.stop) break;
    while (!c.stop) {
      void* args[1] = {&a};
      for (auto& kk : k)
        RP_TRY_CUDA(cudaLaunchKernel(kk.fn, dim3((unsigned)kk.grid), dim3((unsigned)kk.threads), args,
                                     (size_t)kk.smem, s));
      RP_TRY_CUDA(cudaMemcpyAsync(&c, h->bs->ctl, sizeof(BsCtl), cudaMemcpyDeviceToHost, s));
      RP_TRY_CUDA(cudaStreamSynchronize(s));
    }
    if (mixed) {
      k_bs_correct<<<h->bs->grid_vec, kThreads, 0, s>>>(a);
      RP_TRY_CUDA(cudaGetLastError());
    }
  }
  return RP_OK;
}

}  // namespace

void drop_bicgstab_graph(rp_handle* h) {
  if (!h->bs) return;
  for (cudaGraphExec_t* g : {&h->bs->graph, &h->bs->graph_mixed})
    if (*g) {
      cudaGraphExecDestroy(*g);
      *g = nullptr;
    }
}

void free_bicgstab(rp_handle* h) {
  BsState* b = h->bs;
  if (!b) return;
  void* ptrs[] = {b->rhat, b->s, b->t, b->phat, b->shat, b->rhat32, b->s32, b->t32, b->phat32, b->shat32, b->ctl, b->io};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  drop_bicgstab_graph(h);
  delete b;
  h->bs = nullptr;
}

RP_CHECK_TU(bicgstab)

}  // namespace rp

using namespace rp;

namespace rp {
namespace {

rp_status bicgstab_run(rp_handle* h, bool mixed, const double* b, double* x, double tol, int32_t x_is_guess,
                       int32_t where, rp_solve_info* info, void* stream) {
  if (!h || (!b && h->n) || (!x && h->n)) return fail(RP_EINVAL, "null argument");
  if (!(tol >= 0.0)) return fail(RP_EINVAL, "tol must be >= 0");
  if (where != RP_MEM_DEVICE && where != RP_MEM_HOST) return fail(RP_EINVAL, "where must be RP_MEM_DEVICE or RP_MEM_HOST");
  if (mixed && !h->want_fp32) return fail(RP_EINVAL, "mixed precision needs want_fp32");
  if (h->n == 0) {
    if (info) *info = rp_solve_info{RP_OK, 0, 0, 0, 0, 0.0};
    return RP_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  RP_TRY(ensure_bs(h));
  BsState* bs = h->bs;
  cudaGraphExec_t& graph = mixed ? bs->graph_mixed : bs->graph;
  if (!graph && !h->opts.host_loop) RP_TRY(build_bs_graph(h, mixed, &graph));
  const double* bd = b;
  double* xd = x;
  if (where == RP_MEM_HOST) {
    if (!h->b_host_stage && cudaMalloc((void**)&h->b_host_stage, 8 * (h->n + 64)) != cudaSuccess)
      return fail(RP_ENOMEM, "cudaMalloc failed");
    if (!h->x_host_stage && cudaMalloc((void**)&h->x_host_stage, 8 * (h->n + 64)) != cudaSuccess)
      return fail(RP_ENOMEM, "cudaMalloc failed");
    RP_TRY_CUDA(cudaMemcpyAsync(h->b_host_stage, b, 8 * h->n, cudaMemcpyHostToDevice, s));
    if (x_is_guess) RP_TRY_CUDA(cudaMemcpyAsync(h->x_host_stage, x, 8 * h->n, cudaMemcpyHostToDevice, s));
    bd = h->b_host_stage;
    xd = h->x_host_stage;
  }
  k_bs_setup<<<1, 1, 0, s>>>(bs->ctl, bs->io, bd, xd, tol, x_is_guess ? 0 : 1, h->opts.max_iter,
                             h->opts.max_restarts, h->opts.max_outer, h->opts.inner_tol);
  RP_TRY_CUDA(cudaGetLastError());
  if (h->opts.host_loop) RP_TRY(bs_host_loop(h, mixed, s));
  else RP_TRY_CUDA(cudaGraphLaunch(graph, s));
  if (where == RP_MEM_HOST) RP_TRY_CUDA(cudaMemcpyAsync(x, h->x_host_stage, 8 * h->n, cudaMemcpyDeviceToHost, s));
  if (!info) return RP_OK;
  BsCtl c;
  RP_TRY_CUDA(cudaMemcpyAsync(&c, bs->ctl, sizeof(BsCtl), cudaMemcpyDeviceToHost, s));
  RP_TRY_CUDA(cudaStreamSynchronize(s));
  info->status = c.status < 0 ? RP_NOT_CONVERGED : c.status;
  info->iterations = c.iter;
  info->outer_iterations = mixed ? c.outer : 0;
  info->restarts = c.restarts;
  info->passes = c.pass;
  info->rel_residual = c.bb > 0.0 ? sqrt(c.rr / c.bb) : 0.0;
  return (rp_status)info->status;
}

}  // namespace
}  // namespace rp

extern "C" rp_status rp_solve_bicgstab(rp_handle* h, const double* b, double* x, double tol, int32_t x_is_guess,
                                       int32_t where, rp_solve_info* info, void* stream) {
  return bicgstab_run(h, false, b, x, tol, x_is_guess, where, info, stream);
}

extern "C" rp_status rp_solve_bicgstab_mixed(rp_handle* h, const double* b, double* x, double tol,
                                             int32_t x_is_guess, int32_t where, rp_solve_info* info, void* stream) {
  return bicgstab_run(h, true, b, x, tol, x_is_guess, where, info, stream);
}
