// Global assembly support: the CSR sparsity of the global matrix and the position of
// every element-matrix entry in it.
//
// Local assembly produces each cell's contribution to the global linear system
// (section 2); the host framework of the paper then adds the element matrices into a
// global sparse matrix through each cell's local-to-global dof map, executing the
// kernels over all cells of the mesh (section 4). Here that consumer runs on the GPU:
//   1. incidence lists (dof -> cells) by count, scan and fill;
//   2. one warp per global row gathers the dofs of the row's incident cells into
//      shared memory, sorts them (bitonic network) and keeps the distinct ones: first
//      only their number (row lengths -> rowptr by a scan), then the columns themselves;
//   3. the position map: for each cell and local entry (i, j), a binary search of
//      l2g[j] in the sorted columns of row l2g[i].
// The fused assembly kernels (tensor-core and FP64) then add each element-matrix entry
// at map[e][i*nloc + j] of the CSR value array.
#include <cuda_runtime.h>
#include <climits>
#include <cstdint>
#include "coffee_internal.h"

namespace coffee {
namespace {

constexpr int SCAN_THREADS = 256, SCAN_PER_THREAD = 8, SCAN_CHUNK = SCAN_THREADS * SCAN_PER_THREAD;
constexpr int ROW_WARPS = 2;  // warps (rows in flight) per block of the row kernels (32 KB of shared memory)

// ---------------------------------------------------------------- scan
// Exclusive scan of int32 counts into int64 offsets (off[n] = total), three passes:
// per-chunk sums, a scan of the chunk sums, then per-chunk scans with their base.
__global__ void __launch_bounds__(SCAN_THREADS) k_chunk_sums(const int32_t* cnt, int64_t n, int64_t* bsum) {
  __shared__ int64_t red[SCAN_THREADS / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
  int64_t s = 0;
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    const int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
    if (i < n) s += cnt[i];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < SCAN_THREADS / 32; ++w) t += red[w];
    bsum[blockIdx.x] = t;
  }
}

// One block: exclusive scan of the chunk sums in place; the grand total goes to *total.
__global__ void __launch_bounds__(1024) k_scan_sums(int64_t* bsum, int64_t nb, int64_t* total) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x;
  const int64_t per = (nb + blockDim.x - 1) / blockDim.x;
  const int64_t lo = t * per, hi = lo + per < nb ? lo + per : nb;
  int64_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += bsum[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int64_t acc = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      const int64_t v = part[i];
      part[i] = acc;
      acc += v;
    }
    *total = acc;
  }
  __syncthreads();
  int64_t acc = part[t];
  for (int64_t i = lo; i < hi; ++i) {
    const int64_t v = bsum[i];
    bsum[i] = acc;
    acc += v;
  }
}

__global__ void __launch_bounds__(SCAN_THREADS) k_chunk_scan(const int32_t* cnt, int64_t n, const int64_t* bsum,
                                                             int64_t* off) {
  __shared__ int64_t wsum[SCAN_THREADS / 32];
  const int64_t i0 = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_PER_THREAD;
  int32_t v[SCAN_PER_THREAD];
  int64_t mine = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    v[k] = (i0 + k < n) ? cnt[i0 + k] : 0;
    mine += v[k];
  }
  // exclusive scan of the per-thread totals across the block
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t inc = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  int64_t before = bsum[blockIdx.x];
  for (int k = 0; k < w; ++k) before += wsum[k];
  int64_t acc = before + inc - mine;
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k)
    if (i0 + k < n) {
      off[i0 + k] = acc;
      acc += v[k];
    }
}

cudaError_t scan_counts(const int32_t* cnt, int64_t n, int64_t* off, int64_t* bsum, cudaStream_t s) {
  const int64_t nb = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
  if (nb == 0) return cudaMemsetAsync(off, 0, sizeof(int64_t), s);
  k_chunk_sums<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(cnt, n, bsum);
  k_scan_sums<<<1, 1024, 0, s>>>(bsum, nb, off + n);
  k_chunk_scan<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(cnt, n, bsum, off);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- incidence
__global__ void k_inc_count(const int32_t* l2g, int64_t n, int64_t nrows, int32_t* cnt, unsigned* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g = l2g[i];
    if (g < 0 || g >= nrows) {
      atomicOr(flag, ERR_INDEX);
      continue;
    }
    atomicAdd(cnt + g, 1);
  }
}

__global__ void k_inc_fill(const int32_t* l2g, int64_t n, int nloc, int64_t nrows, const int64_t* off,
                           int32_t* cursor, int32_t* inc) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g = l2g[i];
    if (g < 0 || g >= nrows) continue;
    const int32_t k = atomicAdd(cursor + g, 1);
    inc[off[g] + k] = (int32_t)(i / nloc);
  }
}

// ---------------------------------------------------------------- rows
// One warp per row: gather, sort, keep distinct columns. COUNT writes the row length;
// otherwise the columns go to colidx[rowptr[row] ..] (at most the row's allotted length).
template <bool COUNT>
__global__ void __launch_bounds__(ROW_WARPS * 32) k_rows(const int32_t* l2g, int nloc, int64_t nrows,
                                                        const int64_t* incoff, const int32_t* inc,
                                                        int32_t* rowlen, const int64_t* rowptr,
                                                        int32_t* colidx, unsigned* flag) {
  __shared__ int32_t sbuf[ROW_WARPS][CSR_ROW_CAP];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* buf = sbuf[w];
  const uint32_t lt = (1u << lane) - 1u;
  for (int64_t row = (int64_t)blockIdx.x * ROW_WARPS + w; row < nrows; row += (int64_t)gridDim.x * ROW_WARPS) {
    const int64_t b = incoff[row], ncell = incoff[row + 1] - b;
    const int64_t m = ncell * nloc;
    if (m > CSR_ROW_CAP) {
      if (lane == 0) {
        atomicOr(flag, ERR_CAPACITY);
        if (COUNT) rowlen[row] = 0;
      }
      continue;
    }
    int P = 1;
    while (P < m) P <<= 1;
    for (int t = lane; t < P; t += 32) {
      int32_t v = INT_MAX;  // padding sorts last
      if (t < m) {
        const int32_t cell = inc[b + t / nloc];
        v = l2g[(int64_t)cell * nloc + t % nloc];
      }
      buf[t] = v;
    }
    __syncwarp();
    // bitonic sorting network over P (a power of two) entries, ascending
    for (int k = 2; k <= P; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = lane; t < (P >> 1); t += 32) {
          const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
          const int l = i + j;
          const int32_t x = buf[i], y = buf[l];
          const bool up = (i & k) == 0;
          if ((x > y) == up) {
            buf[i] = y;
            buf[l] = x;
          }
        }
        __syncwarp();
      }
    // distinct entries: the first of each run of equal values
    int64_t run = 0;
    const int64_t cap = COUNT ? 0 : rowptr[row + 1] - rowptr[row];
    int32_t* out = COUNT ? nullptr : colidx + rowptr[row];
    for (int c0 = 0; c0 < m; c0 += 32) {
      const int t = c0 + lane;
      const bool keep = t < m && (t == 0 || buf[t] != buf[t - 1]);
      const uint32_t mask = __ballot_sync(0xffffffffu, keep);
      if (!COUNT && keep) {
        const int64_t at = run + __popc(mask & lt);
        if (at < cap) out[at] = buf[t];
      }
      run += __popc(mask);
    }
    if (lane == 0) {
      if (COUNT) rowlen[row] = (int32_t)run;
      else if (run != cap) atomicOr(flag, ERR_INDEX);
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------- position map
// The map is stored in blocks that match the fused kernel's epilogue chunks: cells in groups of
// 32 (padded), entries in groups of 32 (the last group npad - 32*ob wide, npad = nloc^2 rounded up
// to 4); block (cb, ob) holds [32 cells][width] entries contiguously at 32*(cb*npad + 32*ob).
// Padding entries (cells >= ncells, entries >= nloc^2) are 0xffffffff.
__global__ void k_map(const int32_t* l2g, int64_t ncells, int nloc, const int64_t* rowptr,
                      const int32_t* colidx, int64_t nrows, uint32_t* map, unsigned* err) {
  const int n2 = nloc * nloc, np = (n2 + 3) & ~3, nob = (np + 31) / 32;
  const int64_t per_cb = 32 * (int64_t)np, total = ((ncells + 31) / 32) * per_cb;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cb = x / per_cb;
    const int r = (int)(x - cb * per_cb);
    const int ob = r / 1024 < nob - 1 ? r / 1024 : nob - 1;
    const int within = r - ob * 1024, bw = np - ob * 32 < 32 ? np - ob * 32 : 32;
    const int64_t e = cb * 32 + within / bw;
    const int idx = ob * 32 + within % bw;
    if (e >= ncells || idx >= n2) {
      map[x] = 0xffffffffu;
      continue;
    }
    const int i = idx / nloc, j = idx - (idx / nloc) * nloc;
    const int32_t gi = l2g[e * nloc + i], gj = l2g[e * nloc + j];
    uint32_t pos = 0xffffffffu;
    if (gi >= 0 && gi < nrows && gj >= 0 && gj < nrows) {
      int64_t lo = rowptr[gi], hi = rowptr[gi + 1];
      while (lo < hi) {  // first column >= gj
        const int64_t mid = (lo + hi) >> 1;
        if (colidx[mid] < gj) lo = mid + 1;
        else hi = mid;
      }
      if (lo < rowptr[gi + 1] && colidx[lo] == gj) pos = (uint32_t)lo;
    }
    if (pos == 0xffffffffu) atomicOr(err, ERR_INDEX);
    map[x] = pos;
  }
}

unsigned grid_for(int64_t n, int threads, int num_sms) {
  const int64_t b = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms * 16;
  return (unsigned)(b < 1 ? 1 : (b < cap ? b : cap));
}

}  // namespace

size_t sparsity_scratch_bytes(int64_t ncells, int nloc, int64_t nrows) {
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const int64_t nb = (nrows + SCAN_CHUNK - 1) / SCAN_CHUNK + 1;
  return al(sizeof(unsigned)) + 2 * al(sizeof(int32_t) * (size_t)nrows) + al(sizeof(int64_t) * (size_t)(nrows + 1)) +
         al(sizeof(int32_t) * (size_t)(ncells * nloc)) + al(sizeof(int64_t) * (size_t)nb);
}

int launch_sparsity(const int32_t* l2g, int64_t ncells, int nloc, int64_t nrows, int64_t* rowptr, int32_t* colidx,
                    uint8_t* ws, unsigned** flag_out, int num_sms, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  uint8_t* p = ws;
  unsigned* flag = reinterpret_cast<unsigned*>(p);
  p += al(sizeof(unsigned));
  int32_t* cnt = reinterpret_cast<int32_t*>(p);
  p += al(sizeof(int32_t) * (size_t)nrows);
  int32_t* cur = reinterpret_cast<int32_t*>(p);
  p += al(sizeof(int32_t) * (size_t)nrows);
  int64_t* incoff = reinterpret_cast<int64_t*>(p);
  p += al(sizeof(int64_t) * (size_t)(nrows + 1));
  int32_t* inc = reinterpret_cast<int32_t*>(p);
  p += al(sizeof(int32_t) * (size_t)(ncells * nloc));
  int64_t* bsum = reinterpret_cast<int64_t*>(p);
  *flag_out = flag;

  const int64_t n = ncells * nloc;
  cudaError_t e;
  if ((e = cudaMemsetAsync(flag, 0, sizeof(unsigned), s)) != cudaSuccess) return (int)e;
  if ((e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)nrows, s)) != cudaSuccess) return (int)e;
  if ((e = cudaMemsetAsync(cur, 0, sizeof(int32_t) * (size_t)nrows, s)) != cudaSuccess) return (int)e;
  k_inc_count<<<grid_for(n, 256, num_sms), 256, 0, s>>>(l2g, n, nrows, cnt, flag);
  if ((e = scan_counts(cnt, nrows, incoff, bsum, s)) != cudaSuccess) return (int)e;
  k_inc_fill<<<grid_for(n, 256, num_sms), 256, 0, s>>>(l2g, n, nloc, nrows, incoff, cur, inc);
  const unsigned rg = grid_for(nrows, ROW_WARPS, num_sms * 8);
  if (!colidx) {
    // row lengths into cnt (free again), then rowptr
    k_rows<true><<<rg, ROW_WARPS * 32, 0, s>>>(l2g, nloc, nrows, incoff, inc, cnt, nullptr, nullptr, flag);
    if ((e = scan_counts(cnt, nrows, rowptr, bsum, s)) != cudaSuccess) return (int)e;
  } else {
    k_rows<false><<<rg, ROW_WARPS * 32, 0, s>>>(l2g, nloc, nrows, incoff, inc, nullptr, rowptr, colidx, flag);
  }
  return (int)cudaGetLastError();
}

int launch_csr_map(const int32_t* l2g, int64_t ncells, int nloc, const int64_t* rowptr, const int32_t* colidx,
                   int64_t nrows, uint32_t* map, unsigned* err, int num_sms, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t total = csr_map_len(ncells, nloc);
  if (total == 0) return (int)cudaSuccess;
  k_map<<<grid_for(total, 256, num_sms), 256, 0, s>>>(l2g, ncells, nloc, rowptr, colidx, nrows, map, err);
  return (int)cudaGetLastError();
}

}  // namespace coffee
