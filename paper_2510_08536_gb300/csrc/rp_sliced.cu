// Sliced layout of the merged matrix: the device format the iteration
// multiplies with (every part's rows cut into slices of their own).
//
// The CSR arrays of the map stay the reference layout (the map, the value
// update, residual passes, adjoint and gradients use them). For the
// iteration the same entries are re-laid in slices of 32 rows, one row per
// lane, values column-major inside the slice, and every column index is
// replaced by a 4- or 8-bit index into a table of the slice's distinct
// column offsets col - row. Finite-volume rows touch a handful of
// neighbours at a few distinct offsets (9-13 per slice on a decomposed box
// mesh), and slices repeat the same few tables, so distinct tables are kept
// once and a slice with at most 16 offsets packs 8 indices a word: an entry
// costs 4 + 1/2 bytes in FP32 (8 + 1/2 in FP64) instead of 4 + 4 (8 + 4)
// plus the row pointer -- the SpMV, which bounds every PCG iteration, moves
// ~40% fewer bytes in FP32.
//
// Built once, next to the CSR map: one warp per slice finds the distinct
// offsets of its rows in first-appearance order (entry k, then lane) and its
// longest row; a second warp pass writes the tables to a scratch array; the
// host removes duplicate tables and sizes the slices; a third warp pass
// writes index words and the CSR position of every padded entry. The layout
// is not built (the iteration keeps the CSR kernels) when a row has more than
// 32 entries or a slice more than 256 distinct offsets. With several parts
// every part's local entries get slices of their own (part-local rows and
// offsets, a record per slice with its first row, part and row count); the
// non-local entries stay in the part's non-local CSR.
#include <algorithm>
#include <cstring>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

#include "rp_common.cuh"

namespace rp {
namespace {

constexpr int kWarpsPerBlock = kThreads / 32;

// The parts whose rows are sliced (one part: the merged matrix; a batch
// handle: every system): slices, rows and CSR entries of part p start at
// soff[p], roff[p], noff[p]; its CSR rows at row_ptr + roff[p] + p count from
// 0 and its columns are part-local.
struct SlParts {
  int32_t P;
  const int64_t* soff;
  const int64_t* roff;
  const int64_t* noff;
  const int32_t* row_ptr;
  const int32_t* col;
};

// Slice s seen from its part: that part's CSR arrays, rows and local slice index.
struct SlSlice {
  const int32_t* rp;
  const int32_t* col;
  int64_t n, s, nnz0;
};
__device__ __forceinline__ SlSlice slice_of(const SlParts& q, int64_t s) {
  const int p = q.P > 1 ? find_rank(q.soff, q.P, s) : 0;
  const int64_t r0 = q.roff[p], n0 = q.noff[p];
  return SlSlice{q.row_ptr + r0 + p, q.col + n0, q.roff[p + 1] - r0, s - q.soff[p], n0};
}

int slice_grid(const rp_handle* h, int64_t slices) {
  int64_t want = (slices + kWarpsPerBlock - 1) / kWarpsPerBlock;
  int64_t cap = (int64_t)h->num_sms * kBlocksPerSm;
  if (want < 1) want = 1;
  return (int)(want < cap ? want : cap);
}

// The distinct column offsets of slice s in first-appearance order, kept in
// the warp's shared table dict. emit(k, has, id, cnt) runs in every lane for
// every entry position k < L: has = the lane's row has an entry k, id = its
// table index, cnt = table length so far. Returns the table length, or -1
// once it would exceed kSliceMaxDict. All control flow is warp-uniform.
template <class Emit>
__device__ int slice_table(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int64_t n,
                           int64_t s, int L, int32_t* dict, Emit&& emit) {
  const int lane = threadIdx.x & 31;
  const int64_t row = s * kSliceRows + lane;
  int64_t rs = 0;
  int len = 0;
  if (row < n) {
    rs = row_ptr[row];
    len = (int)(row_ptr[row + 1] - rs);
  }
  __syncwarp();  // the previous slice's readers of dict are done
  int cnt = 0;
  for (int k = 0; k < L; ++k) {
    const bool has = k < len;
    const int32_t off = has ? (int32_t)((int64_t)col[rs + k] - row) : 0;
    int id = -1;
    if (has)
      for (int j = 0; j < cnt; ++j)
        if (dict[j] == off) {
          id = j;
          break;
        }
    unsigned need = __ballot_sync(0xffffffffu, has && id < 0);
    while (need) {
      const int32_t noff = __shfl_sync(0xffffffffu, off, __ffs(need) - 1);
      if (cnt == kSliceMaxDict) return -1;
      if (lane == 0) dict[cnt] = noff;
      __syncwarp();
      if (has && id < 0 && off == noff) id = cnt;
      ++cnt;
      need = __ballot_sync(0xffffffffu, has && id < 0);
    }
    emit(k, has, id, cnt);
  }
  return cnt;
}

// pass 1: width L_s and table length D_s of every slice; err bit 1: a
// row longer than kSliceMaxWidth, bit 2: a table longer than kSliceMaxDict
__global__ void __launch_bounds__(kThreads)
    k_slice_count(SlParts q, int64_t S, uint8_t* __restrict__ width, uint16_t* __restrict__ tlen, int32_t* err) {
  __shared__ int32_t sdict[kWarpsPerBlock][kSliceMaxDict];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + w; s < S; s += (int64_t)gridDim.x * kWarpsPerBlock) {
    const SlSlice v = slice_of(q, s);
    const int64_t row = v.s * kSliceRows + lane;
    const int len = row < v.n ? (int)(v.rp[row + 1] - v.rp[row]) : 0;
    const int L = __reduce_max_sync(0xffffffffu, len);
    if (L > kSliceMaxWidth) {
      if (lane == 0) atomicOr(err, 1);
      continue;
    }
    const int D = slice_table(v.rp, v.col, v.n, v.s, L, sdict[w], [](int, bool, int, int) {});
    if (D < 0) {
      if (lane == 0) atomicOr(err, 2);
      continue;
    }
    if (lane == 0) {
      width[s] = (uint8_t)L;
      tlen[s] = (uint16_t)D;
    }
  }
}

// pass 2: every slice's table into the scratch array at toff[s]
__global__ void __launch_bounds__(kThreads)
    k_slice_tables(SlParts q, int64_t S, const uint8_t* __restrict__ width, const int64_t* __restrict__ toff,
                   int32_t* __restrict__ tab) {
  __shared__ int32_t sdict[kWarpsPerBlock][kSliceMaxDict];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + w; s < S; s += (int64_t)gridDim.x * kWarpsPerBlock) {
    const SlSlice v = slice_of(q, s);
    const int D = slice_table(v.rp, v.col, v.n, v.s, width[s], sdict[w], [](int, bool, int, int) {});
    __syncwarp();
    for (int j = lane; j < D; j += 32) tab[toff[s] + j] = sdict[w][j];
  }
}

// pass 3: index words (4- or 8-bit as tinfo says) and CSR positions; err
// bit 4: a slice's size differs from the earlier passes (cannot happen: all
// passes are deterministic)
__global__ void __launch_bounds__(kThreads)
    k_slice_fill(SlParts q, int64_t S, const uint2* __restrict__ desc, const uint32_t* __restrict__ tinfo,
                 int32_t* __restrict__ ibuf, int32_t* __restrict__ pos, int32_t* err) {
  __shared__ int32_t sdict[kWarpsPerBlock][kSliceMaxDict];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t* dict = sdict[w];
  for (int64_t s = (int64_t)blockIdx.x * kWarpsPerBlock + w; s < S; s += (int64_t)gridDim.x * kWarpsPerBlock) {
    const uint2 d0 = desc[s], d1 = desc[s + 1];
    const int L = (int)((d1.x - d0.x) >> 5);
    const bool w4 = (tinfo[s] & kSliceW4) != 0;
    const int per = w4 ? 8 : 4, bits = w4 ? 4 : 8;
    const int nw = (L + per - 1) / per;
    if ((int64_t)(d1.y - d0.y) != (int64_t)kSliceRows * nw) {
      if (lane == 0) atomicOr(err, 4);
      continue;
    }
    const SlSlice v = slice_of(q, s);
    const int64_t row = v.s * kSliceRows + lane;
    const int64_t rs = row < v.n ? v.rp[row] : 0;
    uint32_t* iw = reinterpret_cast<uint32_t*>(ibuf + d0.y);
    int32_t* ps = pos + d0.x;
    uint32_t word = 0;
    const int D = slice_table(v.rp, v.col, v.n, v.s, L, dict, [&](int k, bool has, int id, int cnt) {
      if (!has) {
        // padding: the diagonal's index (a row < n stored its diagonal at an
        // earlier k, so offset 0 is in the table); zero value, in-range column
        id = 0;
        if (row < v.n)
          for (int j = 0; j < cnt; ++j)
            if (dict[j] == 0) {
              id = j;
              break;
            }
      }
      word |= (uint32_t)id << (bits * (k % per));
      if (k % per == per - 1 || k == L - 1) {
        iw[(k / per) * kSliceRows + lane] = word;
        word = 0;
      }
      ps[k * kSliceRows + lane] = has ? (int32_t)(v.nnz0 + rs + k) : -1;
    });
    if ((D <= 16) != w4 && lane == 0) atomicOr(err, 4);
  }
}

// sliced values from the CSR values: v[q] = vals[pos[q]], 0 for padding
template <bool FP32>
__global__ void __launch_bounds__(kThreads)
    k_slice_vals(int64_t nq4, const int4* __restrict__ pos, const double* __restrict__ vals,
                 double2* __restrict__ out, float4* __restrict__ out32, int64_t nnz) {
  // a CSR position, or -1 for padding (bounds-checked build: anything else reads 0)
  auto at = [&](int32_t q) { return q >= 0 && RP_IN(q, 0, nnz, kChkSliceValues) ? __ldg(vals + q) : 0.0; };
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq4; i += (int64_t)gridDim.x * blockDim.x) {
    const int4 p = __ldcs(pos + i);
    const double a = at(p.x), b = at(p.y), c = at(p.z), d = at(p.w);
    __stcs(out + 2 * i, make_double2(a, b));
    __stcs(out + 2 * i + 1, make_double2(c, d));
    if (FP32) __stcs(out32 + i, make_float4((float)a, (float)b, (float)c, (float)d));
  }
}

template <typename T>
rp_status salloc(T** p, int64_t count) {
  if (count <= 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, (size_t)count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(RP_ENOMEM, "cudaMalloc of %lld bytes failed", (long long)(count * sizeof(T)));
  }
  return RP_OK;
}

struct Tmp {
  std::vector<void*> v;
  ~Tmp() {
    for (void* p : v) cudaFree(p);
  }
  template <typename T>
  rp_status alloc(T** p, int64_t count) {
    RP_TRY(salloc(p, count));
    v.push_back(*p);
    return RP_OK;
  }
};

}  // namespace

void free_sliced(rp_handle* h) {
  void* ptrs[] = {h->sl_part_soff, h->sl_srow, h->sl_desc, h->sl_tinfo, h->sl_tabs, h->sl_ibuf, h->sl_pos,
                  h->sl_vals, h->sl_vals32, h->sl_valsT, h->sl_vals32s, h->s64};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  h->sl_vals32s = nullptr;
  h->s64 = nullptr;
  h->sl_part_soff = nullptr;
  h->sl_srow = nullptr;
  h->sl_desc = nullptr;
  h->sl_tinfo = nullptr;
  h->sl_tabs = nullptr;
  h->sl_ibuf = nullptr;
  h->sl_pos = nullptr;
  h->sl_vals = nullptr;
  h->sl_vals32 = nullptr;
  h->sl_valsT = nullptr;
  h->sl_slices = h->sl_entries = h->sl_ibuf_len = h->sl_tabs_len = 0;
  h->sl_u4 = 0;
}

rp_status build_sliced(rp_handle* h, cudaStream_t st) {
  if (h->n == 0 || h->opts.layout == RP_LAYOUT_CSR) return RP_OK;
  const int P = h->n_parts;
  std::vector<int64_t> soff(P + 1, 0);
  for (int p = 0; p < P; ++p)
    soff[p + 1] = soff[p] + (h->part_row_off[p + 1] - h->part_row_off[p] + kSliceRows - 1) / kSliceRows;
  const int64_t S = soff[P];
  if (S == 0) return RP_OK;
  Tmp tmp;
  int64_t* dsoff;
  RP_TRY(tmp.alloc(&dsoff, P + 1));
  RP_TRY_CUDA(cudaMemcpyAsync(dsoff, soff.data(), 8 * (P + 1), cudaMemcpyHostToDevice, st));
  const SlParts q{P, dsoff, h->d_part_row_off, h->d_part_nnz_off, h->row_ptr, h->col_idx};
  uint8_t* width;
  uint16_t* tlen;
  int32_t* err;
  RP_TRY(tmp.alloc(&width, S));
  RP_TRY(tmp.alloc(&tlen, S));
  RP_TRY(tmp.alloc(&err, 1));
  RP_TRY_CUDA(cudaMemsetAsync(err, 0, 4, st));
  const int g = slice_grid(h, S);
  k_slice_count<<<g, kThreads, 0, st>>>(q, S, width, tlen, err);
  RP_TRY_CUDA(cudaGetLastError());
  std::vector<uint8_t> hw(S);
  std::vector<uint16_t> ht(S);
  int32_t herr = 0;
  RP_TRY_CUDA(cudaMemcpyAsync(hw.data(), width, S, cudaMemcpyDeviceToHost, st));
  RP_TRY_CUDA(cudaMemcpyAsync(ht.data(), tlen, 2 * S, cudaMemcpyDeviceToHost, st));
  RP_TRY_CUDA(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st));
  RP_TRY_CUDA(cudaStreamSynchronize(st));
  if (herr) return RP_OK;  // a row or a slice does not fit: CSR iteration

  // every slice's table into one scratch array, then distinct tables kept once
  std::vector<int64_t> toff(S + 1, 0);
  for (int64_t s = 0; s < S; ++s) toff[s + 1] = toff[s] + ht[s];
  int64_t* dtoff;
  int32_t* dtab;
  RP_TRY(tmp.alloc(&dtoff, S + 1));
  RP_TRY(tmp.alloc(&dtab, toff[S] + 1));
  RP_TRY_CUDA(cudaMemcpyAsync(dtoff, toff.data(), 8 * (S + 1), cudaMemcpyHostToDevice, st));
  k_slice_tables<<<g, kThreads, 0, st>>>(q, S, width, dtoff, dtab);
  RP_TRY_CUDA(cudaGetLastError());
  std::vector<int32_t> htab(toff[S]);
  RP_TRY_CUDA(cudaMemcpyAsync(htab.data(), dtab, 4 * toff[S], cudaMemcpyDeviceToHost, st));
  RP_TRY_CUDA(cudaStreamSynchronize(st));
  std::vector<int32_t> tabs;
  std::vector<uint32_t> tinfo(S + kSliceDescPad, 0u);
  std::unordered_map<std::string, uint32_t> seen;
  std::vector<uint2> desc(S + 1 + kSliceDescPad, make_uint2(0u, 0u));
  uint64_t x = 0, y = 0;
  bool u4 = true;
  for (int64_t s = 0; s < S; ++s) {
    const int D = ht[s];
    std::string key(reinterpret_cast<const char*>(htab.data() + toff[s]), 4 * (size_t)D);
    auto it = seen.find(key);
    uint32_t t;
    if (it == seen.end()) {
      tabs.push_back(D);
      t = (uint32_t)tabs.size();
      tabs.insert(tabs.end(), htab.begin() + toff[s], htab.begin() + toff[s + 1]);
      seen.emplace(std::move(key), t);
    } else {
      t = it->second;
    }
    const bool w4 = D <= 16;
    u4 = u4 && w4 && hw[s] <= 8;
    tinfo[s] = t | (w4 ? kSliceW4 : 0u);
    desc[s] = make_uint2((uint32_t)x, (uint32_t)y);
    const int per = w4 ? 8 : 4;
    x += (uint64_t)kSliceRows * hw[s];
    y += (uint64_t)kSliceRows * ((hw[s] + per - 1) / per);
    if (x > 0xffffff00ull || y > 0xffffff00ull || tabs.size() > 0x7fffff00ull) return RP_OK;  // CSR iteration
  }
  desc[S] = make_uint2((uint32_t)x, (uint32_t)y);
  tabs.insert(tabs.end(), 32, 0);  // lanes past a table read these
  free_sliced(h);
  auto undo = [&](rp_status s) {
    free_sliced(h);
    return s;
  };
#define SL_TRY(call)                 \
  do {                               \
    rp_status s_ = (call);           \
    if (s_ != RP_OK) return undo(s_); \
  } while (0)
  SL_TRY(salloc(&h->sl_part_soff, P + 1));
  std::vector<int2> srow;
  if (P > 1) {
    srow.resize(S);
    for (int p = 0; p < P; ++p) {
      const int64_t r0 = h->part_row_off[p], np = h->part_row_off[p + 1] - r0;
      for (int64_t j = 0; j < soff[p + 1] - soff[p]; ++j)
        srow[soff[p] + j] = make_int2((int)(r0 + kSliceRows * j),
                                      (int)(((int64_t)p << 6) | std::min<int64_t>(kSliceRows, np - kSliceRows * j)));
    }
    SL_TRY(salloc(&h->sl_srow, S));
  }
  SL_TRY(salloc(&h->sl_desc, S + 1 + kSliceDescPad));
  SL_TRY(salloc(&h->sl_tinfo, S + kSliceDescPad));
  SL_TRY(salloc(&h->sl_tabs, (int64_t)tabs.size()));
  SL_TRY(salloc(&h->sl_ibuf, (int64_t)y));
  SL_TRY(salloc(&h->sl_pos, (int64_t)x));
  SL_TRY(salloc(&h->sl_vals, (int64_t)x));
  if (h->want_fp32) SL_TRY(salloc(&h->sl_vals32, (int64_t)x));
#undef SL_TRY
  auto cu = [&](cudaError_t e, const char* what) {
    if (e == cudaSuccess) return RP_OK;
    return undo(fail(RP_ECUDA, "%s failed: %s", what, cudaGetErrorString(e)));
  };
  RP_TRY(cu(cudaMemcpyAsync(h->sl_desc, desc.data(), sizeof(uint2) * desc.size(), cudaMemcpyHostToDevice, st),
            "sliced descriptor upload"));
  RP_TRY(cu(cudaMemcpyAsync(h->sl_part_soff, soff.data(), 8 * (P + 1), cudaMemcpyHostToDevice, st),
            "sliced part offsets upload"));
  if (P > 1)
    RP_TRY(cu(cudaMemcpyAsync(h->sl_srow, srow.data(), sizeof(int2) * S, cudaMemcpyHostToDevice, st),
              "sliced row records upload"));
  RP_TRY(cu(cudaMemcpyAsync(h->sl_tinfo, tinfo.data(), 4 * tinfo.size(), cudaMemcpyHostToDevice, st),
            "sliced table reference upload"));
  RP_TRY(cu(cudaMemcpyAsync(h->sl_tabs, tabs.data(), 4 * tabs.size(), cudaMemcpyHostToDevice, st),
            "sliced table upload"));
  RP_TRY(cu(cudaMemsetAsync(h->sl_vals, 0, 8 * x, st), "sliced value clear"));
  if (h->sl_vals32) RP_TRY(cu(cudaMemsetAsync(h->sl_vals32, 0, 4 * x, st), "sliced value clear"));
  k_slice_fill<<<g, kThreads, 0, st>>>(q, S, h->sl_desc, h->sl_tinfo, h->sl_ibuf, h->sl_pos, err);
  RP_TRY(cu(cudaGetLastError(), "k_slice_fill"));
  RP_TRY(cu(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st), "error readback"));
  RP_TRY(cu(cudaStreamSynchronize(st), "sliced layout build"));
  if (herr) return undo(fail(RP_ECUDA, "sliced layout: slice sizes differ between passes"));
  h->sl_slices = S;
  h->sl_u4 = u4 ? 1 : 0;
  h->sl_entries = (int64_t)x;
  h->sl_ibuf_len = (int64_t)y;
  h->sl_tabs_len = (int64_t)tabs.size();
  return RP_OK;
}

// s_i = 1 / sqrt(a_ii): FP64 square root and division (both correctly rounded)
__global__ void __launch_bounds__(kThreads)
    k_scaling(int64_t n, const int32_t* __restrict__ diag_pos, const double* __restrict__ vals, int64_t nnz,
              double* __restrict__ s64) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = diag_pos[i];
    s64[i] = RP_IN(d, 0, nnz, kChkSliceValues) ? 1.0 / sqrt(__ldg(vals + d)) : 0.0;
  }
}

// FP32 sliced values of S A S (one part: slice s holds rows 32 s ..) from the
// FP64 sliced values: entry k of lane j of slice s is v = fl32(sv (s_i s_i')),
// i = 32 s + j, with the column i' = i + its offset decoded from the slice's
// table and index words as the iteration reads them, products in FP64, s_i s_i'
// first (the diagonal comes out as exactly 1). Padding (value 0, offset 0)
// stays 0. One warp per slice; reads the FP64 values and index words once,
// coalesced, and s at the gathered rows.
__global__ void __launch_bounds__(kThreads)
    k_slice_vals_scaled(int64_t S, const uint2* __restrict__ desc, const uint32_t* __restrict__ tinfo,
                        const int32_t* __restrict__ tabs, const uint32_t* __restrict__ ibuf,
                        const double* __restrict__ sv, const double* __restrict__ s64, int64_t n,
                        float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < S; s += nw) {
    const uint2 d0 = __ldg(desc + s), d1 = __ldg(desc + s + 1);
    const uint32_t info = __ldg(tinfo + s);
    const int32_t* tab = tabs + (info & ~kSliceW4);
    const bool w4 = (info & kSliceW4) != 0;
    const int per = w4 ? 8 : 4, bits = w4 ? 4 : 8;
    const uint32_t mask = w4 ? 15u : 255u;
    const int L = (int)((d1.x - d0.x) >> 5);
    const int64_t i = s * kSliceRows + lane;
    const bool valid = i < n;
    const double si = valid ? __ldg(s64 + i) : 0.0;
    uint32_t wd = 0;
    for (int k = 0; k < L; ++k) {
      if (k % per == 0) wd = __ldg(ibuf + d0.y + (uint32_t)(kSliceRows * (k / per)) + lane);
      const int64_t q = d0.x + (int64_t)kSliceRows * k + lane;
      const int64_t j = i + __ldg(tab + ((wd >> (bits * (k % per))) & mask));
      float v = 0.0f;
      if (valid && RP_IN(j, 0, n, kChkGather)) v = (float)(__ldcs(sv + q) * (si * __ldg(s64 + j)));
      __stcs(out + q, v);
    }
  }
}

static rp_status fill_scaled(rp_handle* h, cudaStream_t s) {
  k_scaling<<<grid_for(h, h->n), kThreads, 0, s>>>(h->n, h->diag_pos, h->vals, h->nnz, h->s64);
  k_slice_vals_scaled<<<grid_for(h, h->sl_slices * kSliceRows), kThreads, 0, s>>>(
      h->sl_slices, h->sl_desc, h->sl_tinfo, h->sl_tabs, reinterpret_cast<const uint32_t*>(h->sl_ibuf), h->sl_vals,
      h->s64, h->n, h->sl_vals32s);
  RP_TRY_CUDA(cudaGetLastError());
  return RP_OK;
}

rp_status ensure_scaled(rp_handle* h, cudaStream_t s, bool* ok) {
  *ok = h->n_parts == 1 && h->sl_slices > 0 && h->sl_vals32 != nullptr && h->n > 0;
  if (!*ok || h->sl_vals32s) return RP_OK;
  RP_TRY(salloc(&h->s64, h->n + 64));
  rp_status st = salloc(&h->sl_vals32s, h->sl_entries);
  if (st != RP_OK) {
    cudaFree(h->s64);
    h->s64 = nullptr;
    return st;
  }
  return fill_scaled(h, s);
}

RP_CHECK_TU(sliced)

rp_status fill_sliced(rp_handle* h, cudaStream_t s) {
  if (h->sl_slices == 0) return RP_OK;
  const int64_t nq4 = h->sl_entries / 4;  // a multiple of 32 entries
  const int g = grid_for(h, nq4);
  const int4* pos = reinterpret_cast<const int4*>(h->sl_pos);
  double2* out = reinterpret_cast<double2*>(h->sl_vals);
  if (h->sl_vals32)
    k_slice_vals<true><<<g, kThreads, 0, s>>>(nq4, pos, h->vals, out, reinterpret_cast<float4*>(h->sl_vals32),
                                              h->nnz);
  else
    k_slice_vals<false><<<g, kThreads, 0, s>>>(nq4, pos, h->vals, out, nullptr, h->nnz);
  RP_TRY_CUDA(cudaGetLastError());
  if (h->sl_vals32s) RP_TRY(fill_scaled(h, s));
  return RP_OK;
}

// The transposed matrix of a structurally symmetric pattern (every entry has
// its transposed position) has the same slices: entry q of the layout takes
// valsT at the same CSR position.
rp_status fill_sliced_transposed(rp_handle* h, cudaStream_t s) {
  if (h->sl_slices == 0 || !h->valsT) return RP_OK;
  if (!h->sl_valsT) RP_TRY(salloc(&h->sl_valsT, h->sl_entries));
  const int64_t nq4 = h->sl_entries / 4;
  k_slice_vals<false><<<grid_for(h, nq4), kThreads, 0, s>>>(nq4, reinterpret_cast<const int4*>(h->sl_pos), h->valsT,
                                                            reinterpret_cast<double2*>(h->sl_valsT), nullptr, h->nnz);
  RP_TRY_CUDA(cudaGetLastError());
  return RP_OK;
}

}  // namespace rp

using namespace rp;

extern "C" rp_status rp_get_sliced_view(const rp_handle* h, rp_sliced_view* out) {
  if (!h || !out) return fail(RP_EINVAL, "null argument");
  out->n_slices = h->sl_slices;
  out->n_entries = h->sl_entries;
  out->ibuf_len = h->sl_ibuf_len;
  out->tabs_len = h->sl_tabs_len;
  out->desc = reinterpret_cast<const uint32_t*>(h->sl_desc);
  out->tinfo = h->sl_tinfo;
  out->tabs = h->sl_tabs;
  out->ibuf = h->sl_ibuf;
  out->pos = h->sl_pos;
  out->vals = h->sl_vals;
  out->vals32 = h->sl_vals32;
  out->vals32s = h->sl_vals32s;
  out->scale = h->s64;
  out->srow = reinterpret_cast<const int32_t*>(h->sl_srow);
  out->uniform4 = h->sl_u4 && !h->sl_srow ? 1 : 0;
  return RP_OK;
}
