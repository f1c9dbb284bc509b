// Repartitioning map (Sec. 3, steps 1-3): fuse the LDU sparsity of k CPU
// ranks into one CSR pattern per GPU part, with the permutation from the
// LDU-ordered continuous buffer to row-major order.
//
// Device algorithm (integer only, deterministic):
//   1. count: every stored entry adds 1 to its row's local or non-local degree
//   2. exclusive scan of the degrees -> row offsets
//   3. place: every entry takes a slot of its row (atomic cursor)
//   4. sort each row by column (rows are short), detect duplicates, record
//      the diagonal position; the sorted order is unique, so the result does
//      not depend on the order the atomics were served in
//   5. transpose positions by binary search in the partner row
//   6. non-local columns compressed per part by mark + scan
#include <algorithm>
#include <atomic>
#include <cstring>
#include <memory>
#include <thread>
#include <vector>

#include "rp_common.cuh"

namespace rp {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

rp_status fail(rp_status s, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

// ------------------------------------------------------------------ scan

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void k_scan_reduce(const int32_t* __restrict__ in, int64_t n, int32_t* __restrict__ bsum) {
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  int s = 0;
  for (int j = threadIdx.x; j < kScanTile; j += kScanThreads) {
    int64_t i = base + j;
    if (i < n) s += in[i];
  }
  __shared__ int sm[kScanThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    int t = threadIdx.x < kScanThreads / 32 ? sm[threadIdx.x] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) bsum[blockIdx.x] = t;
  }
}

// exclusive scan of one value per thread across the block; returns the block total
__device__ int block_exclusive(int v, int* total) {
  __shared__ int wsum[33];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int w = lane < nw ? wsum[lane] : 0;
    int winc = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, winc, o);
      if (lane >= o) winc += t;
    }
    if (lane < nw) wsum[lane] = winc - w;
    if (lane == nw - 1) wsum[32] = winc;
  }
  __syncthreads();
  int r = wsum[wid] + inc - v;
  if (total) *total = wsum[32];
  __syncthreads();
  return r;
}

__global__ void k_scan_spine(int32_t* __restrict__ bsum, int64_t nb, int32_t* __restrict__ total_out) {
  int carry = 0;
  for (int64_t base = 0; base < nb; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    int v = i < nb ? bsum[i] : 0;
    int tot;
    int ex = block_exclusive(v, &tot);
    if (i < nb) bsum[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_scan_down(const int32_t* __restrict__ in, int64_t n, const int32_t* __restrict__ boff,
                            int32_t* __restrict__ out) {
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int v[kScanItems];
  int s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    v[j] = base + j < n ? in[base + j] : 0;
    s += v[j];
  }
  int ex = block_exclusive(s, nullptr) + boff[blockIdx.x];
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    if (base + j < n) out[base + j] = ex;
    ex += v[j];
  }
}

// out[0..n] = exclusive scan of in[0..n), out[n] = total (caller guarantees < 2^31)
static rp_status scan_exclusive(const int32_t* in, int32_t* out, int64_t n, int32_t* bsum,
                                cudaStream_t st) {
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 0) {
    RP_TRY_CUDA(cudaMemsetAsync(out, 0, sizeof(int32_t), st));
    return RP_OK;
  }
  k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, bsum);
  k_scan_spine<<<1, 1024, 0, st>>>(bsum, nb, out + n);
  k_scan_down<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, bsum, out);
  RP_TRY_CUDA(cudaGetLastError());
  return RP_OK;
}

// ------------------------------------------------------------------ map kernels

struct MapIn {
  int32_t k, n_parts, alpha, symmetric;
  const int64_t* ent_off;    // [k+1] entries per rank: n + 2F + E
  const int64_t* row_off;    // [k+1]
  const int64_t* slot_off;   // [k+1]
  const int64_t* face_off;   // [k+1]
  const int64_t* iface_off;  // [k+1]
  const int64_t* part_row_off;  // [n_parts+1]
  const int64_t* part_buf_off;  // [n_parts+1]
  const int32_t* lower;
  const int32_t* upper;
  const int32_t* iface_row;
  const int32_t* iface_gcol;
  int64_t n_entries;
  int64_t n_rows, nnz, nl_nnz;  // bounds of the placement (bounds-checked build)
};

// global (row, col, slot) of entry t and its rank's part
__device__ __forceinline__ void entry_coords(const MapIn& m, int64_t t, int64_t& row, int64_t& col,
                                             int64_t& slot, int& part) {
  int r = find_rank(m.ent_off, m.k, t);
  int64_t u = t - m.ent_off[r];
  int64_t n = m.row_off[r + 1] - m.row_off[r];
  int64_t F = m.face_off[r + 1] - m.face_off[r];
  int64_t ro = m.row_off[r], so = m.slot_off[r];
  part = r / m.alpha;
  if (u < n) {
    row = col = ro + u;
    slot = so + u;
  } else if (u < n + F) {
    int64_t f = u - n;
    row = ro + m.lower[m.face_off[r] + f];
    col = ro + m.upper[m.face_off[r] + f];
    slot = so + n + f;
  } else if (u < n + 2 * F) {
    int64_t f = u - n - F;
    row = ro + m.upper[m.face_off[r] + f];
    col = ro + m.lower[m.face_off[r] + f];
    slot = so + n + (m.symmetric ? f : F + f);
  } else {
    int64_t e = u - n - 2 * F;
    row = ro + m.iface_row[m.iface_off[r] + e];
    col = m.iface_gcol[m.iface_off[r] + e];
    slot = so + n + (m.symmetric ? 1 : 2) * F + e;
  }
}

__device__ __forceinline__ bool col_in_part(const MapIn& m, int part, int64_t col) {
  return col >= m.part_row_off[part] && col < m.part_row_off[part + 1];
}

__global__ void k_count(MapIn m, int32_t* __restrict__ deg, int32_t* __restrict__ nl_deg) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m.n_entries;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t row, col, slot;
    int part;
    entry_coords(m, t, row, col, slot, part);
    if (!RP_IN(row, 0, m.n_rows, kChkMap) || !RP_IN(col, 0, m.n_rows, kChkMap)) continue;
    if (col_in_part(m, part, col)) atomicAdd(deg + row, 1);
    else atomicAdd(nl_deg + row, 1);
  }
}

__global__ void k_place(MapIn m, int32_t* __restrict__ cur, int32_t* __restrict__ nl_cur,
                        int32_t* __restrict__ col_idx, int32_t* __restrict__ src_of,
                        int32_t* __restrict__ nl_gcol, int32_t* __restrict__ nl_src_of) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m.n_entries;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t row, col, slot;
    int part;
    entry_coords(m, t, row, col, slot, part);
    int64_t sl = slot - m.part_buf_off[part];
    if (!RP_IN(row, 0, m.n_rows, kChkMap) || !RP_IN(col, 0, m.n_rows, kChkMap)) continue;
    if (col_in_part(m, part, col)) {
      int q = atomicAdd(cur + row, 1);
      if (!RP_IN(q, 0, m.nnz, kChkMap)) continue;
      col_idx[q] = (int32_t)(col - m.part_row_off[part]);
      src_of[q] = (int32_t)sl;
    } else {
      int q = atomicAdd(nl_cur + row, 1);
      if (!RP_IN(q, 0, m.nl_nnz, kChkMap)) continue;
      nl_gcol[q] = (int32_t)col;
      nl_src_of[q] = (int32_t)sl;
    }
  }
}

// per row: insertion sort by column (carrying the slot), duplicates, diagonal
__global__ void k_sort_rows(int64_t n, const int32_t* __restrict__ pos, int32_t* __restrict__ col,
                            int32_t* __restrict__ src, const int64_t* __restrict__ part_row_off,
                            int n_parts, const int32_t* __restrict__ part_pos0,
                            int32_t* __restrict__ diag_pos, int32_t* __restrict__ err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int s = pos[i], e = pos[i + 1];
    for (int a = s + 1; a < e; ++a) {
      int c = col[a], v = src[a];
      int b = a - 1;
      while (b >= s && col[b] > c) {
        col[b + 1] = col[b];
        src[b + 1] = src[b];
        --b;
      }
      col[b + 1] = c;
      src[b + 1] = v;
    }
    for (int a = s + 1; a < e; ++a)
      if (col[a] == col[a - 1]) atomicOr(err, 1);
    if (diag_pos) {
      int p = find_rank(part_row_off, n_parts, i);
      int32_t li = (int32_t)(i - part_row_off[p]);
      int d = -1;
      for (int a = s; a < e; ++a)
        if (col[a] == li) d = a - part_pos0[p];
      diag_pos[i] = d;
      if (d < 0) atomicOr(err, 4);
    }
  }
}

// tpos: for entry (i, j) of part p, the part-relative position of (j, i)
__global__ void k_tpos(int64_t n, const int32_t* __restrict__ pos, const int32_t* __restrict__ col,
                       const int64_t* __restrict__ part_row_off, int n_parts,
                       const int32_t* __restrict__ part_pos0, int32_t* __restrict__ tpos,
                       int32_t* __restrict__ err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int p = find_rank(part_row_off, n_parts, i);
    int64_t r0 = part_row_off[p];
    int32_t li = (int32_t)(i - r0);
    for (int a = pos[i]; a < pos[i + 1]; ++a) {
      int64_t jg = r0 + col[a];
      if (!RP_IN(jg, 0, n, kChkMap)) continue;
      int lo = pos[jg], hi = pos[jg + 1];
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (col[mid] < li) lo = mid + 1; else hi = mid;
      }
      if (lo < pos[jg + 1] && col[lo] == li) {
        tpos[a] = lo - part_pos0[p];
      } else {
        tpos[a] = -1;
        atomicOr(err, 2);
      }
    }
  }
}

__global__ void k_part_rowptr(const int32_t* __restrict__ pos, int64_t r0, int64_t nrows,
                              int32_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= nrows;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = pos[r0 + i] - pos[r0];
}

__global__ void k_mark(int64_t r0, int64_t r1, const int32_t* __restrict__ pos,
                       const int32_t* __restrict__ gcol, int32_t* __restrict__ mark, int64_t n) {
  int64_t s = pos[r0], e = pos[r1];
  for (int64_t q = s + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < e;
       q += (int64_t)gridDim.x * blockDim.x)
    if (RP_IN(gcol[q], 0, n, kChkMap)) mark[gcol[q]] = 1;
}

__global__ void k_compact_cols(int64_t n, const int32_t* __restrict__ mark, const int32_t* __restrict__ idx,
                               int32_t* __restrict__ cols) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n;
       g += (int64_t)gridDim.x * blockDim.x)
    if (mark[g]) cols[idx[g]] = (int32_t)g;
}

__global__ void k_renumber(int64_t r0, int64_t r1, const int32_t* __restrict__ pos,
                           const int32_t* __restrict__ gcol, const int32_t* __restrict__ idx,
                           int32_t* __restrict__ out) {
  int64_t s = pos[r0], e = pos[r1];
  for (int64_t q = s + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < e;
       q += (int64_t)gridDim.x * blockDim.x)
    out[q] = idx[gcol[q]];
}

// ------------------------------------------------------------------ host side

namespace {

template <typename T>
rp_status dalloc(T** p, int64_t count) {
  *p = nullptr;
  if (count <= 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, (size_t)count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(RP_ENOMEM, "cudaMalloc of %lld bytes failed: %s", (long long)(count * sizeof(T)),
                cudaGetErrorString(e));
  }
  return RP_OK;
}

struct DevFree {
  std::vector<void*> ptrs;
  ~DevFree() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  rp_status alloc(T** p, int64_t count) {
    rp_status s = dalloc(p, count);
    if (s == RP_OK) ptrs.push_back(*p);
    return s;
  }
};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (dev >= 0 && dev != prev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// f(i) for i in [0, n) on up to 16 host threads (dynamic schedule); on one
// thread when threads cannot be started.
template <class F>
void parallel_for(int64_t n, F&& f) {
  const unsigned hw = std::thread::hardware_concurrency();
  const int64_t T = std::min<int64_t>(n, std::min<unsigned>(hw ? hw : 1u, 16u));
  std::atomic<int64_t> next{0};
  auto work = [&]() {
    for (int64_t i; (i = next.fetch_add(1)) < n;) f(i);
  };
  std::vector<std::thread> th;
  try {
    for (int64_t t = 1; t < T; ++t) th.emplace_back(work);
  } catch (...) {  // no more threads: the ones started and this one finish the work
  }
  work();
  for (auto& t : th) t.join();
}

// Ascending sort of 64-bit keys: LSD radix, 8-bit digits, skipping digits
// that are equal in every key.
void radix_sort_u64(std::vector<uint64_t>& v) {
  std::vector<uint64_t> tmp(v.size());
  uint64_t any = 0, all = ~0ull;
  for (uint64_t x : v) {
    any |= x;
    all &= x;
  }
  for (int sh = 0; sh < 64; sh += 8) {
    if ((((any ^ all) >> sh) & 0xffu) == 0) continue;
    uint32_t cnt[256] = {0};
    for (uint64_t x : v) ++cnt[(x >> sh) & 0xffu];
    uint32_t run = 0;
    for (uint32_t& c : cnt) {
      const uint32_t t = c;
      c = run;
      run += t;
    }
    for (uint64_t x : v) tmp[cnt[(x >> sh) & 0xffu]++] = x;
    v.swap(tmp);
  }
}

rp_status validate(const rp_ldu_desc* ranks, int32_t k, const rp_options& o) {
  if (!ranks || k < 1) return fail(RP_EINVAL, "need k >= 1 rank descriptors");
  if (o.n_parts < 1 || k % o.n_parts) return fail(RP_EINVAL, "n_parts=%d must divide k=%d", o.n_parts, k);
  if (o.max_iter < 0 || o.max_outer < 0 || o.max_restarts < 0 || !(o.inner_tol > 0.0) ||
      o.spin_limit < 0 || !(o.ru_delta >= 0.0 && o.ru_delta < 1.0))
    return fail(RP_EINVAL, "invalid solver options");
  if (o.layout != RP_LAYOUT_AUTO && o.layout != RP_LAYOUT_CSR)
    return fail(RP_EINVAL, "layout must be RP_LAYOUT_AUTO or RP_LAYOUT_CSR");
  if (o.precond != RP_PRECOND_JACOBI && o.precond != RP_PRECOND_LINE)
    return fail(RP_EINVAL, "precond must be RP_PRECOND_JACOBI or RP_PRECOND_LINE");
  if (o.spare != 0) return fail(RP_EINVAL, "spare must be 0");
  if (o.precond == RP_PRECOND_LINE && o.n_parts != 1)
    return fail(RP_EUNSUPPORTED, "the line preconditioner needs n_parts = 1");
  int64_t n = 0, nnz = 0, slots = 0;
  std::vector<int64_t> off(k + 1, 0), eoff(k + 1, 0);
  for (int r = 0; r < k; ++r) {
    const rp_ldu_desc& d = ranks[r];
    if (d.n_cells < 0 || d.n_faces < 0 || d.n_iface < 0)
      return fail(RP_EINVAL, "rank %d: negative count", r);
    if ((d.n_faces > 0 && (!d.lower_addr || !d.upper_addr)) ||
        (d.n_iface > 0 && (!d.iface_row || !d.iface_nbr_rank || !d.iface_nbr_col)))
      return fail(RP_EINVAL, "rank %d: null array with a positive count", r);
    n += d.n_cells;
    nnz += (int64_t)d.n_cells + 2 * (int64_t)d.n_faces + d.n_iface;
    slots += (int64_t)d.n_cells + (o.symmetric ? 1 : 2) * (int64_t)d.n_faces + d.n_iface;
    off[r + 1] = off[r] + d.n_cells;
    eoff[r + 1] = eoff[r] + d.n_iface;
  }
  const int64_t lim = 2147483647LL - 1024;
  if (n > lim || nnz > lim || slots > lim)
    return fail(RP_EOVERFLOW, "rows=%lld entries=%lld slots=%lld exceed the 32-bit index range",
                (long long)n, (long long)nnz, (long long)slots);
  // every rank at once, without branches; a rank that fails is scanned again to name the entry
  std::vector<char> bad(k, 0);
  parallel_for(k, [&](int64_t r) {
    const rp_ldu_desc& d = ranks[r];
    const int32_t nc = d.n_cells;
    int b = 0;
    for (int32_t f = 0; f < d.n_faces; ++f) {
      const int32_t l = d.lower_addr[f], u = d.upper_addr[f];
      b |= (l < 0) | (u >= nc) | (l >= u);  // with l < u these bound both addresses
    }
    for (int32_t e = 0; e < d.n_iface; ++e) {
      const int32_t row = d.iface_row[e], q = d.iface_nbr_rank[e], c = d.iface_nbr_col[e];
      b |= (row < 0) | (row >= nc) | (q < 0) | (q >= k) | (q == (int32_t)r);
      if (q >= 0 && q < k) b |= (c < 0) | (c >= ranks[q].n_cells);
    }
    bad[r] = (char)b;
  });
  for (int r = 0; r < k; ++r) {
    if (!bad[r]) continue;
    const rp_ldu_desc& d = ranks[r];
    for (int32_t f = 0; f < d.n_faces; ++f) {
      int32_t l = d.lower_addr[f], u = d.upper_addr[f];
      if (l < 0 || u < 0 || l >= d.n_cells || u >= d.n_cells)
        return fail(RP_ERANGE, "rank %d face %d: address (%d,%d) outside [0,%d)", r, f, l, u, d.n_cells);
      if (l >= u) return fail(RP_EINVAL, "rank %d face %d: owner %d must be below neighbour %d", r, f, l, u);
    }
    for (int32_t e = 0; e < d.n_iface; ++e) {
      int32_t row = d.iface_row[e], q = d.iface_nbr_rank[e], c = d.iface_nbr_col[e];
      if (row < 0 || row >= d.n_cells) return fail(RP_ERANGE, "rank %d iface %d: row %d out of range", r, e, row);
      if (q < 0 || q >= k) return fail(RP_ERANGE, "rank %d iface %d: neighbour rank %d out of range", r, e, q);
      if (q == r) return fail(RP_EINVAL, "rank %d iface %d: interface to itself", r, e);
      if (c < 0 || c >= ranks[q].n_cells)
        return fail(RP_ERANGE, "rank %d iface %d: column %d outside rank %d", r, e, c, q);
    }
  }
  // interfaces must come in transposed pairs: the merged (row, col) of every
  // interface entry, as a multiset, equals that of the transposed entries
  std::vector<uint64_t> a(eoff[k]), b(eoff[k]);
  parallel_for(k, [&](int64_t r) {
    const rp_ldu_desc& d = ranks[r];
    for (int32_t e = 0; e < d.n_iface; ++e) {
      const uint64_t gr = (uint64_t)(off[r] + d.iface_row[e]);
      const uint64_t gc = (uint64_t)(off[d.iface_nbr_rank[e]] + d.iface_nbr_col[e]);
      a[eoff[r] + e] = gr << 32 | gc;
      b[eoff[r] + e] = gc << 32 | gr;
    }
  });
  parallel_for(2, [&](int64_t i) { radix_sort_u64(i ? b : a); });
  if (a != b) return fail(RP_EINVAL, "processor interfaces are not paired (rank q must hold the transposed entry)");
  return RP_OK;
}

}  // namespace

RP_CHECK_TU(map)

}  // namespace rp

using namespace rp;

extern "C" void rp_default_options(rp_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->n_parts = 1;
  o->symmetric = 0;
  o->want_fp32 = 1;
  o->want_transpose = 0;
  o->max_iter = 20000;
  o->max_outer = 30;
  o->max_restarts = 8;
  o->device = -1;
  o->inner_tol = 1e-5;
  o->spin_limit = 1LL << 26;
  o->layout = RP_LAYOUT_AUTO;
  o->ru_delta = 0.1;
}

extern "C" const char* rp_last_error(void) { return rp::g_last_error.c_str(); }

extern "C" const char* rp_status_str(rp_status s) {
  switch (s) {
    case RP_OK: return "RP_OK";
    case RP_EINVAL: return "RP_EINVAL";
    case RP_EDUP: return "RP_EDUP";
    case RP_ERANGE: return "RP_ERANGE";
    case RP_EOVERFLOW: return "RP_EOVERFLOW";
    case RP_ENOMEM: return "RP_ENOMEM";
    case RP_ECUDA: return "RP_ECUDA";
    case RP_NOT_CONVERGED: return "RP_NOT_CONVERGED";
    case RP_BREAKDOWN: return "RP_BREAKDOWN";
    case RP_DEVICE_TIMEOUT: return "RP_DEVICE_TIMEOUT";
    case RP_EUNSUPPORTED: return "RP_EUNSUPPORTED";
  }
  return "RP_UNKNOWN";
}

static void free_handle_memory(rp_handle* h) {
  void* ptrs[] = {h->row_ptr, h->col_idx, h->src_of, h->diag_pos, h->tpos, h->nl_row_ptr, h->nl_col_idx,
                  h->nl_src_of, h->nl_cols, h->d_row_off, h->d_slot_off, h->d_face_off, h->d_iface_off,
                  h->d_lower, h->d_upper, h->d_iface_row, h->d_iface_gcol, h->d_out_off, h->staging, h->vals,
                  h->vals32, h->nl_vals, h->valsT, h->dinv, h->dinv32, h->dinvT, h->nl_vals32,
                  h->d_part_row_off, h->d_part_nnz_off, h->d_part_nl_off, h->d_part_nlcol_off};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  free_solver(h);
  free_batch(h);
  free_sliced(h);
  free_bicgstab(h);
  free_line(h);
  free_async_stage(h);
}

extern "C" void rp_destroy(rp_handle* h) {
  if (!h) return;
  DeviceGuard g(h->device);
  cudaDeviceSynchronize();
  free_handle_memory(h);
  delete h;
}

extern "C" rp_status rp_build_repartition(const rp_ldu_desc* ranks, int32_t k, const rp_options* opts,
                                          rp_handle** out) {
  if (!out) return fail(RP_EINVAL, "out is NULL");
  *out = nullptr;
  rp_options o;
  if (opts) o = *opts; else rp_default_options(&o);
  RP_TRY(validate(ranks, k, o));

  DeviceGuard guard(o.device);
  std::unique_ptr<rp_handle> h(new rp_handle());
  RP_TRY_CUDA(cudaGetDevice(&h->device));
  RP_TRY_CUDA(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
  h->opts = o;
  h->k = k;
  h->n_parts = o.n_parts;
  h->symmetric = o.symmetric != 0;
  h->want_fp32 = o.want_fp32 != 0;
  h->want_transpose = o.want_transpose != 0;
  h->precond = o.precond;
  const int alpha = k / o.n_parts;

  // rank tables
  h->row_off.assign(k + 1, 0);
  h->slot_off.assign(k + 1, 0);
  h->face_off.assign(k + 1, 0);
  h->iface_off.assign(k + 1, 0);
  std::vector<int64_t> ent_off(k + 1, 0);
  for (int r = 0; r < k; ++r) {
    const rp_ldu_desc& d = ranks[r];
    h->n_cells.push_back(d.n_cells);
    h->n_faces.push_back(d.n_faces);
    h->n_iface.push_back(d.n_iface);
    h->row_off[r + 1] = h->row_off[r] + d.n_cells;
    h->slot_off[r + 1] = h->slot_off[r] + d.n_cells + (h->symmetric ? 1 : 2) * (int64_t)d.n_faces + d.n_iface;
    h->face_off[r + 1] = h->face_off[r] + d.n_faces;
    h->iface_off[r + 1] = h->iface_off[r] + d.n_iface;
    ent_off[r + 1] = ent_off[r] + d.n_cells + 2 * (int64_t)d.n_faces + d.n_iface;
  }
  h->n = h->row_off[k];
  h->n_slots = h->slot_off[k];
  h->n_face_out = h->face_off[k] + h->iface_off[k];
  const int64_t n = h->n, n_entries = ent_off[k];
  const int64_t F = h->face_off[k], E = h->iface_off[k];
  h->part_row_off.assign(o.n_parts + 1, 0);
  h->part_buf_off.assign(o.n_parts + 1, 0);
  for (int p = 0; p <= o.n_parts; ++p) {
    h->part_row_off[p] = h->row_off[p * alpha];
    h->part_buf_off[p] = h->slot_off[p * alpha];
  }

  // upload addressing
  std::vector<int32_t> lower(F), upper(F), irow(E), igcol(E);
  for (int r = 0; r < k; ++r) {
    const rp_ldu_desc& d = ranks[r];
    if (d.n_faces) {
      std::memcpy(lower.data() + h->face_off[r], d.lower_addr, sizeof(int32_t) * d.n_faces);
      std::memcpy(upper.data() + h->face_off[r], d.upper_addr, sizeof(int32_t) * d.n_faces);
    }
    for (int32_t e = 0; e < d.n_iface; ++e) {
      irow[h->iface_off[r] + e] = d.iface_row[e];
      igcol[h->iface_off[r] + e] = (int32_t)(h->row_off[d.iface_nbr_rank[e]] + d.iface_nbr_col[e]);
    }
  }
  cudaStream_t st;
  RP_TRY_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  struct StreamFree {
    cudaStream_t s;
    ~StreamFree() { cudaStreamDestroy(s); }
  } sfree{st};

  rp_handle* H = h.get();
  auto fail_free = [&](rp_status s) {
    free_handle_memory(H);
    H->row_ptr = nullptr;
    return s;
  };
#define ALLOC(ptr, cnt)                                \
  do {                                                 \
    rp_status s_ = dalloc(&(ptr), (cnt));              \
    if (s_ != RP_OK) return fail_free(s_);             \
  } while (0)
#define CU(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail_free(fail(RP_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),      \
                            __FILE__, __LINE__));                                                  \
  } while (0)

  ALLOC(H->d_row_off, k + 1);
  ALLOC(H->d_slot_off, k + 1);
  ALLOC(H->d_face_off, k + 1);
  ALLOC(H->d_iface_off, k + 1);
  ALLOC(H->d_lower, F);
  ALLOC(H->d_upper, F);
  ALLOC(H->d_iface_row, E);
  ALLOC(H->d_iface_gcol, E);
  CU(cudaMemcpyAsync(H->d_row_off, H->row_off.data(), 8 * (k + 1), cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(H->d_slot_off, H->slot_off.data(), 8 * (k + 1), cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(H->d_face_off, H->face_off.data(), 8 * (k + 1), cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(H->d_iface_off, H->iface_off.data(), 8 * (k + 1), cudaMemcpyHostToDevice, st));
  if (F) {
    CU(cudaMemcpyAsync(H->d_lower, lower.data(), 4 * F, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(H->d_upper, upper.data(), 4 * F, cudaMemcpyHostToDevice, st));
  }
  if (E) {
    CU(cudaMemcpyAsync(H->d_iface_row, irow.data(), 4 * E, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(H->d_iface_gcol, igcol.data(), 4 * E, cudaMemcpyHostToDevice, st));
  }

  // temporaries
  DevFree tmp;
  int64_t *d_ent_off, *d_part_row_off, *d_part_buf_off;
  int32_t *deg, *nl_deg, *pos, *nl_pos, *bsum, *err, *nl_gcol, *part_pos0;
  const int64_t nb = (n + kScanTile) / kScanTile + 1;
#define TALLOC(ptr, cnt)                             \
  do {                                               \
    rp_status s_ = tmp.alloc(&(ptr), (cnt));         \
    if (s_ != RP_OK) return fail_free(s_);           \
  } while (0)
  TALLOC(d_ent_off, k + 1);
  TALLOC(d_part_row_off, o.n_parts + 1);
  TALLOC(d_part_buf_off, o.n_parts + 1);
  TALLOC(deg, n + 1);
  TALLOC(nl_deg, n + 1);
  TALLOC(pos, n + 1);
  TALLOC(nl_pos, n + 1);
  TALLOC(bsum, nb);
  TALLOC(err, 1);
  TALLOC(part_pos0, 2 * (o.n_parts + 1));
  CU(cudaMemcpyAsync(d_ent_off, ent_off.data(), 8 * (k + 1), cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(d_part_row_off, H->part_row_off.data(), 8 * (o.n_parts + 1), cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(d_part_buf_off, H->part_buf_off.data(), 8 * (o.n_parts + 1), cudaMemcpyHostToDevice, st));
  CU(cudaMemsetAsync(deg, 0, 4 * (n + 1), st));
  CU(cudaMemsetAsync(nl_deg, 0, 4 * (n + 1), st));
  CU(cudaMemsetAsync(err, 0, 4, st));

  MapIn m;
  m.k = k;
  m.n_parts = o.n_parts;
  m.alpha = alpha;
  m.symmetric = H->symmetric;
  m.ent_off = d_ent_off;
  m.row_off = H->d_row_off;
  m.slot_off = H->d_slot_off;
  m.face_off = H->d_face_off;
  m.iface_off = H->d_iface_off;
  m.part_row_off = d_part_row_off;
  m.part_buf_off = d_part_buf_off;
  m.lower = H->d_lower;
  m.upper = H->d_upper;
  m.iface_row = H->d_iface_row;
  m.iface_gcol = H->d_iface_gcol;
  m.n_entries = n_entries;
  m.n_rows = n;
  m.nnz = m.nl_nnz = 0;
  const int g = grid_for(H, n_entries > n ? n_entries : n);

  // 1-2: degrees and their scans
  k_count<<<g, kThreads, 0, st>>>(m, deg, nl_deg);
  CU(cudaGetLastError());
  {
    rp_status s = scan_exclusive(deg, pos, n, bsum, st);
    if (s != RP_OK) return fail_free(s);
    s = scan_exclusive(nl_deg, nl_pos, n, bsum, st);
    if (s != RP_OK) return fail_free(s);
  }
  // totals and per-part starting positions
  std::vector<int32_t> pos_at(o.n_parts + 1), nl_pos_at(o.n_parts + 1);
  for (int p = 0; p <= o.n_parts; ++p) {
    CU(cudaMemcpyAsync(&pos_at[p], pos + H->part_row_off[p], 4, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(&nl_pos_at[p], nl_pos + H->part_row_off[p], 4, cudaMemcpyDeviceToHost, st));
  }
  CU(cudaStreamSynchronize(st));
  H->nnz = pos_at[o.n_parts];
  H->nl_nnz = nl_pos_at[o.n_parts];
  H->part_nnz_off.assign(pos_at.begin(), pos_at.end());
  H->part_nl_off.assign(nl_pos_at.begin(), nl_pos_at.end());
  if (H->nnz + H->nl_nnz != n_entries)
    return fail_free(fail(RP_ECUDA, "entry count mismatch after scan (%lld + %lld != %lld)",
                          (long long)H->nnz, (long long)H->nl_nnz, (long long)n_entries));
  CU(cudaMemcpyAsync(part_pos0, pos_at.data(), 4 * (o.n_parts + 1), cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(part_pos0 + o.n_parts + 1, nl_pos_at.data(), 4 * (o.n_parts + 1), cudaMemcpyHostToDevice, st));

  // 3: placement (cursors start at the row offsets)
  const int64_t pad = 64;
  ALLOC(H->col_idx, H->nnz + pad);
  ALLOC(H->src_of, H->nnz + pad);
  ALLOC(H->diag_pos, n);
  ALLOC(H->nl_col_idx, H->nl_nnz + pad);
  ALLOC(H->nl_src_of, H->nl_nnz + pad);
  CU(cudaMemsetAsync(H->col_idx, 0, 4 * (H->nnz + pad), st));
  CU(cudaMemsetAsync(H->src_of, 0, 4 * (H->nnz + pad), st));
  TALLOC(nl_gcol, H->nl_nnz + 1);
  CU(cudaMemcpyAsync(deg, pos, 4 * (n + 1), cudaMemcpyDeviceToDevice, st));
  CU(cudaMemcpyAsync(nl_deg, nl_pos, 4 * (n + 1), cudaMemcpyDeviceToDevice, st));
  m.nnz = H->nnz;
  m.nl_nnz = H->nl_nnz;
  k_place<<<g, kThreads, 0, st>>>(m, deg, nl_deg, H->col_idx, H->src_of, nl_gcol, H->nl_src_of);
  CU(cudaGetLastError());

  // 4: sort rows, duplicates, diagonal
  const int gr = grid_for(H, n);
  k_sort_rows<<<gr, kThreads, 0, st>>>(n, pos, H->col_idx, H->src_of, d_part_row_off, o.n_parts, part_pos0,
                                       H->diag_pos, err);
  CU(cudaGetLastError());

  // 5: transpose positions
  if (H->want_transpose) {
    ALLOC(H->tpos, H->nnz + pad);
    k_tpos<<<gr, kThreads, 0, st>>>(n, pos, H->col_idx, d_part_row_off, o.n_parts, part_pos0, H->tpos, err);
    CU(cudaGetLastError());
  }

  // part-relative row pointers
  ALLOC(H->row_ptr, n + o.n_parts);
  ALLOC(H->nl_row_ptr, n + o.n_parts);
  for (int p = 0; p < o.n_parts; ++p) {
    int64_t r0 = H->part_row_off[p], nr = H->part_row_off[p + 1] - r0;
    int gp = grid_for(H, nr + 1);
    k_part_rowptr<<<gp, kThreads, 0, st>>>(pos, r0, nr, H->row_ptr + r0 + p);
    k_part_rowptr<<<gp, kThreads, 0, st>>>(nl_pos, r0, nr, H->nl_row_ptr + r0 + p);
  }
  CU(cudaGetLastError());

  // 6: non-local column compression, part by part
  H->part_nlcol_off.assign(o.n_parts + 1, 0);
  if (H->nl_nnz > 0) {
    int32_t *mark, *idx;
    TALLOC(mark, n + 1);
    TALLOC(idx, n + 1);
    std::vector<int32_t> counts(o.n_parts);
    std::vector<int32_t*> part_cols(o.n_parts, nullptr);
    DevFree colbufs;
    for (int p = 0; p < o.n_parts; ++p) {
      int64_t r0 = H->part_row_off[p], r1 = H->part_row_off[p + 1];
      CU(cudaMemsetAsync(mark, 0, 4 * (n + 1), st));
      k_mark<<<gr, kThreads, 0, st>>>(r0, r1, nl_pos, nl_gcol, mark, n);
      rp_status s = scan_exclusive(mark, idx, n, bsum, st);
      if (s != RP_OK) return fail_free(s);
      CU(cudaMemcpyAsync(&counts[p], idx + n, 4, cudaMemcpyDeviceToHost, st));
      CU(cudaStreamSynchronize(st));
      {
        rp_status s2 = colbufs.alloc(&part_cols[p], counts[p] + 1);
        if (s2 != RP_OK) return fail_free(s2);
      }
      k_compact_cols<<<gr, kThreads, 0, st>>>(n, mark, idx, part_cols[p]);
      k_renumber<<<gr, kThreads, 0, st>>>(r0, r1, nl_pos, nl_gcol, idx, H->nl_col_idx);
      CU(cudaGetLastError());
      H->part_nlcol_off[p + 1] = H->part_nlcol_off[p] + counts[p];
    }
    ALLOC(H->nl_cols, H->part_nlcol_off[o.n_parts] + 1);
    for (int p = 0; p < o.n_parts; ++p)
      if (counts[p])
        CU(cudaMemcpyAsync(H->nl_cols + H->part_nlcol_off[p], part_cols[p], 4 * (int64_t)counts[p],
                           cudaMemcpyDeviceToDevice, st));
    k_sort_rows<<<gr, kThreads, 0, st>>>(n, nl_pos, H->nl_col_idx, H->nl_src_of, d_part_row_off, o.n_parts,
                                         part_pos0 + o.n_parts + 1, nullptr, err);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(st));
  } else {
    ALLOC(H->nl_cols, 1);
  }

  int32_t herr = 0;
  CU(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (herr & 1) return fail_free(fail(RP_EDUP, "two stored coefficients share one (row, col)"));
  if (herr & 4) return fail_free(fail(RP_ECUDA, "a row lost its diagonal entry"));
  if ((herr & 2) && H->want_transpose)
    return fail_free(fail(RP_EINVAL, "pattern is not structurally symmetric: no transpose position"));

  // values and solver work space
  ALLOC(H->staging, H->n_slots + pad);
  ALLOC(H->vals, H->nnz + pad);
  ALLOC(H->nl_vals, H->nl_nnz + pad);
  ALLOC(H->dinv, n + pad);
  CU(cudaMemsetAsync(H->vals, 0, 8 * (H->nnz + pad), st));
  CU(cudaMemsetAsync(H->staging, 0, 8 * (H->n_slots + pad), st));
  if (H->want_fp32) {
    ALLOC(H->vals32, H->nnz + pad);
    ALLOC(H->nl_vals32, H->nl_nnz + pad);
    ALLOC(H->dinv32, n + pad);
    CU(cudaMemsetAsync(H->vals32, 0, 4 * (H->nnz + pad), st));
  }
  // part tables for solves over the local + non-local matrices
  {
    const int np1 = o.n_parts + 1;
    std::vector<int64_t> nlcol(H->part_nlcol_off.begin(), H->part_nlcol_off.end());
    ALLOC(H->d_part_row_off, np1);
    ALLOC(H->d_part_nnz_off, np1);
    ALLOC(H->d_part_nl_off, np1);
    ALLOC(H->d_part_nlcol_off, np1);
    CU(cudaMemcpyAsync(H->d_part_row_off, H->part_row_off.data(), 8 * np1, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(H->d_part_nnz_off, H->part_nnz_off.data(), 8 * np1, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(H->d_part_nl_off, H->part_nl_off.data(), 8 * np1, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(H->d_part_nlcol_off, nlcol.data(), 8 * np1, cudaMemcpyHostToDevice, st));
  }
  CU(cudaStreamSynchronize(st));
  H->grid = grid_for(H, n);
  {
    rp_status s = build_sliced(H, st);
    if (s != RP_OK) return fail_free(s);
    s = ensure_solver_buffers(H);
    if (s != RP_OK) return fail_free(s);
  }
#undef ALLOC
#undef CU
#undef TALLOC
  *out = h.release();
  return RP_OK;
}

extern "C" rp_status rp_get_part_map(const rp_handle* h, int32_t part, rp_map_view* out) {
  if (!h || !out) return fail(RP_EINVAL, "null argument");
  if (part < 0 || part >= h->n_parts) return fail(RP_ERANGE, "part %d outside [0,%d)", part, h->n_parts);
  int64_t r0 = h->part_row_off[part];
  out->n_rows = h->part_row_off[part + 1] - r0;
  out->nnz = h->part_nnz_off[part + 1] - h->part_nnz_off[part];
  out->nl_nnz = h->part_nl_off[part + 1] - h->part_nl_off[part];
  out->n_nl_cols = h->part_nlcol_off[part + 1] - h->part_nlcol_off[part];
  out->row_off = r0;
  out->buf_off = h->part_buf_off[part];
  out->buf_len = h->part_buf_off[part + 1] - h->part_buf_off[part];
  out->row_ptr = h->row_ptr + r0 + part;
  out->col_idx = h->col_idx + h->part_nnz_off[part];
  out->src_of = h->src_of + h->part_nnz_off[part];
  out->diag_pos = h->diag_pos + r0;
  out->tpos = h->tpos ? h->tpos + h->part_nnz_off[part] : nullptr;
  out->nl_row_ptr = h->nl_row_ptr + r0 + part;
  out->nl_col_idx = h->nl_col_idx + h->part_nl_off[part];
  out->nl_src_of = h->nl_src_of + h->part_nl_off[part];
  out->nl_cols = h->nl_cols + h->part_nlcol_off[part];
  return RP_OK;
}

extern "C" rp_status rp_get_sizes(const rp_handle* h, int64_t* n_rows, int64_t* nnz, int64_t* n_slots,
                                  int32_t* n_parts) {
  if (!h) return fail(RP_EINVAL, "null handle");
  if (n_rows) *n_rows = h->n;
  if (nnz) *nnz = h->nnz;
  if (n_slots) *n_slots = h->n_slots;
  if (n_parts) *n_parts = h->n_parts;
  return RP_OK;
}

#ifdef RP_CHECK
namespace rp {
rp_status check_read_update(CheckWord*, int);
rp_status check_read_sliced(CheckWord*, int);
rp_status check_read_pcg(CheckWord*, int);
rp_status check_read_batch(CheckWord*, int);
rp_status check_read_bicgstab(CheckWord*, int);
rp_status check_read_adjoint(CheckWord*, int);
rp_status check_read_noalloc(CheckWord*, int);
}  // namespace rp
#endif

extern "C" rp_status rp_check_violations(uint64_t* count, int32_t* first_site, int64_t* first_index,
                                         int32_t reset) {
  if (!count) return fail(RP_EINVAL, "null argument");
  *count = 0;
  if (first_site) *first_site = 0;
  if (first_index) *first_index = -1;
#ifdef RP_CHECK
  using Reader = rp_status (*)(CheckWord*, int);
  const Reader readers[] = {check_read_map,   check_read_update,   check_read_sliced, check_read_pcg,
                            check_read_batch, check_read_bicgstab, check_read_adjoint, check_read_noalloc};
  RP_TRY_CUDA(cudaDeviceSynchronize());
  for (Reader r : readers) {
    CheckWord w{};
    RP_TRY(r(&w, reset));
    if (w.count && *count == 0) {
      if (first_site) *first_site = w.site;
      if (first_index) *first_index = w.index;
    }
    *count += w.count;
  }
  return RP_OK;
#else
  (void)reset;
  return fail(RP_EUNSUPPORTED, "this library was built without RP_CHECK (the bounds-checked build is "
                               "librepart_check.so)");
#endif
}
