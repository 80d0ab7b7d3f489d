// CUDA-core local assembly of small element matrices (MASS, HELMHOLTZ, ADVDIFF on triangles
// P1-P3 and tetrahedra P1-P2): A_e = sum_k G_e[k] T[k], the contraction of section 4 (the
// reference tensor T against the per-cell geometry and coefficient factors G_e) in FP32, one
// thread per cell.
//
// Why not the tensor cores here: with K = 1 to 36 factors and 9 to 100 entries per cell the
// contraction is a few hundred FMAs per cell against 36 to 400 bytes written, so the work is
// bound by HBM and by the per-cell gather and geometry, not by multiply-adds. The tensor-core
// kernel (k_tc_kernel.cuh) runs that per-cell work on 8 producer warps per SM; this kernel runs
// it on every warp the SM holds, which hides the gather latency, and the FMAs (T is read from
// constant memory, uniform across the warp, as an FMA operand) cost less than the MMA hand-offs.
//
// Per warp and 32 consecutive cells: each lane gathers its cell, forms G_e (the producers'
// cell_factors_ids: FP32 geometry with the FP64 fallback for badly conditioned cells, the
// vertex differences from (hi, lo) float pairs split by integer operations, so no FP64
// instruction runs for regular cells), computes its N entries and writes them to a
// shared-memory staging block (row stride N rounded up to odd: conflict-free); the warp then
// writes the 32 rows, contiguous in the output, with coalesced 16-byte stores.
// Accuracy: T is rounded to FP32 once (2^-24) and the K-term sums accumulate in FP32, which
// meets every tensor-core precision's bound (TF32X3/BF16X3 1e-5, TF32/BF16 1e-2).
#include <cuda_runtime.h>
#include <cstdint>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <vector>
#include "coffee_internal.h"
#include "tc_common.cuh"

namespace coffee {
namespace {
using namespace tc;

constexpr int SIMT_THREADS = 256;
constexpr int SIMT_WARPS = SIMT_THREADS / 32;

__host__ __device__ constexpr int s_ns(int d, int k) { return d == 2 ? (k + 1) * (k + 2) / 2 : (k + 1) * (k + 2) * (k + 3) / 6; }
// rows of T: MASS 1, HELMHOLTZ 1 + P (edge factors), ADVDIFF (d+1) P + (d+1) d; the Burgers
// Jacobian's [T1 | T2 | T3]: 2 ns d + P (of one d x d component block's ns^2 entries)
__host__ __device__ constexpr int s_K(int form, int d, int k = 1) {
  return form == FORM_MASS ? 1 : form == FORM_HELMHOLTZ ? 1 + d * (d + 1) / 2
       : form == FORM_ADVDIFF ? (d + 1) * (d * (d + 1) / 2) + (d + 1) * d
       : 2 * s_ns(d, k) * d + d * (d + 1) / 2;
}
// instances: MASS, HELMHOLTZ, ADVDIFF on triangles P1-P3 and tetrahedra P1-P2; the Burgers
// Jacobian on triangles P1-P2 and tetrahedra P1
__host__ __device__ constexpr int s_maxdeg(int form, int d) { return form == FORM_BURGERS ? (d == 2 ? 2 : 1) : d == 2 ? 3 : 2; }
__host__ __device__ constexpr int s_size(int form, int d, int k) { return s_K(form, d, k) * s_ns(d, k) * s_ns(d, k); }
// offset of each instance's table in the constant bank
__host__ __device__ constexpr int s_off(int form, int d, int k) {
  int off = 0;
  for (int f = 0; f <= FORM_BURGERS; ++f)
    for (int dd = 2; dd <= 3; ++dd)
      for (int kk = 1; kk <= s_maxdeg(f, dd); ++kk) {
        if (f == form && dd == d && kk == k) return off;
        off += s_size(f, dd, kk);
      }
  return off;  // one past the last: the total
}
constexpr int S_TOTAL = s_off(FORM_BURGERS + 1, 0, 0);
static_assert(S_TOTAL * 4 <= 60 * 1024, "reference tensors exceed the constant bank");

// T [K][N] in FP32 of every instance (edge-basis form of the stiffness tensors, as the
// tensor-core images), written once per device before the first launch that reads it
__constant__ float c_T[S_TOTAL];

// index rows of cell e; tetrahedra with 16-byte aligned index arrays read each row with one
// 16-byte load (v4, uniform)
template <int FORM, int D>
__device__ __forceinline__ void simt_ids(const TcParams& p, int64_t e, bool v4, CellIds<FORM, D>& ids) {
  if constexpr (D == 3) {
    if (v4) {
      const int4 a = __ldg(reinterpret_cast<const int4*>(p.c2v) + e);
      ids.vid[0] = a.x, ids.vid[1] = a.y, ids.vid[2] = a.z, ids.vid[3] = a.w;
      if constexpr (FORM == FORM_ADVDIFF) {
        const int4 b = __ldg(reinterpret_cast<const int4*>(p.c2d) + e);
        ids.cid[0] = b.x, ids.cid[1] = b.y, ids.cid[2] = b.z, ids.cid[3] = b.w;
      }
      return;
    }
  }
  load_ids<FORM, D>(p, e, ids);
}

// One warp tile: the 32 cells from 32 t on, staged in st (32 rows of SR = N | 1 floats).
template <int FORM, int D, int DEG>
__device__ __forceinline__ void simt_tile(const TcParams& p, int64_t t, int lane, float* st) {
  constexpr int NS = s_ns(D, DEG), N = NS * NS, K = s_K(FORM, D), OFF = s_off(FORM, D, DEG);
  constexpr int SR = N | 1;  // staging row stride
  const bool vec = (reinterpret_cast<uintptr_t>(p.out) & 15) == 0;
  const bool v4 = (reinterpret_cast<uintptr_t>(p.c2v) & 15) == 0 &&
                  (FORM != FORM_ADVDIFF || (reinterpret_cast<uintptr_t>(p.c2d) & 15) == 0);
  const int64_t c0 = t * 32, e = c0 + lane;
  float G[K];
  bool bad = false;
  if (e < p.ncells) {
    CellIds<FORM, D> ids;
    simt_ids<FORM, D>(p, e, v4, ids);
    cell_factors_ids<FORM, D, K, true>(p, ids, G, bad);
    if (bad) atomicOr(p.err, ERR_INDEX);
  }
  if (e >= p.ncells || bad) {
#pragma unroll
    for (int k = 0; k < K; ++k) G[k] = 0.f;
  }
  if constexpr (FORM == FORM_ADVDIFF) {
#pragma unroll
    for (int o = 0; o < N; ++o) {
      float a = 0.f;
#pragma unroll
      for (int k = 0; k < K; ++k) a = fmaf(G[k], c_T[OFF + k * N + o], a);
      st[lane * SR + o] = a;
    }
  } else {
    // MASS and HELMHOLTZ are symmetric: the upper triangle is formed and mirrored
#pragma unroll
    for (int i = 0; i < NS; ++i)
#pragma unroll
      for (int j = i; j < NS; ++j) {
        float a = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) a = fmaf(G[k], c_T[OFF + k * N + i * NS + j], a);
        st[lane * SR + i * NS + j] = a;
        if (j != i) st[lane * SR + j * NS + i] = a;
      }
  }
  __syncwarp();
  // contiguous rows (the default layout): the 32 rows are 32 N floats from c0 N on (16-byte
  // aligned when the output is, since 32 N floats are a multiple of 16 bytes); padded rows
  // (a row stride above N): each row's N floats with coalesced scalar stores
  const int rows = (int)(p.ncells - c0 < 32 ? p.ncells - c0 : 32);
  float* dst = p.out + c0 * p.ostride;
  if (p.ostride != N) {
    for (int i = lane; i < rows * N; i += 32) __stcs(dst + (int64_t)(i / N) * p.ostride + i % N, st[(i / N) * SR + i % N]);
  } else if (rows == 32 && vec) {
#pragma unroll 4
    for (int i = lane; i < 8 * N; i += 32) {  // 8 N float4 per warp tile
      float4 v;
      const int j = 4 * i;
      v.x = st[((j + 0) / N) * SR + (j + 0) % N];
      v.y = st[((j + 1) / N) * SR + (j + 1) % N];
      v.z = st[((j + 2) / N) * SR + (j + 2) % N];
      v.w = st[((j + 3) / N) * SR + (j + 3) % N];
      __stcs(reinterpret_cast<float4*>(dst) + i, v);
    }
  } else {
    for (int i = lane; i < rows * N; i += 32) __stcs(dst + i, st[(i / N) * SR + i % N]);
  }
  __syncwarp();
}

// The Burgers Jacobian on triangles P1-P2 and tetrahedra P1 (vector Pk: d ns entries per row), one
// cell per thread, in the factored form of its d x d component blocks of ns^2 entries:
//   block(ci, cj) = sum_a P[a][cj] V_a^ci + [ci == cj] C,   V_a^ci = sum_r u[r][ci] T1[r d + a],
//   C = sum_{r,a} Q[r][a] T2[r d + a] + sum_p nu H_p T3[p],   Q[r][a] = sum_c u[r][c] P[a][c],
// with P = |det J| K and T = [T1 | T2 | T3] the Burgers reference tensors (rows r d + a of T1 and
// T2, then the P pair rows of T3) in constant memory. Each block row ci of the cell's matrix (its
// ns rows, contiguous in the output) goes to the staging block and out with the warp's coalesced
// 16-byte stores before the next is formed, so a warp stages ns d ns floats per cell instead of
// the whole matrix (tetrahedra: 49 instead of 145; shared memory had limited a multiprocessor to
// 12 warps); rows whose block row is not a multiple of 4 floats (triangles P1) stage the matrix.
constexpr int SIMT_BTHREADS = 128;
template <int D, int DEG, bool RES>
__host__ __device__ constexpr int sb_stride(int ns) {  // staging floats per cell (odd)
  return RES ? ((D * ns) | 1) : ((ns * D * ns) % 4 == 0 ? ((ns * D * ns) | 1) : ((D * ns * D * ns) | 1));
}
// RES: the residual instead (element vectors, R[(c, i)] = sum_s C[i][s] u[s][c]; C as above).
template <int D, int DEG, bool RES = false>
__device__ __forceinline__ void simt_tile_burgers(const TcParams& p, int64_t t, int lane, float* st) {
  constexpr int NS = s_ns(D, DEG), NV = D + 1, NDOF = D * NS, N = RES ? NDOF : NDOF * NDOF, NB = NS * NS;
  constexpr int K1 = NS * D, P = D * (D + 1) / 2, OFF = s_off(FORM_BURGERS, D, DEG);
  constexpr int BR = NS * NDOF;                     // floats of one block row of a cell
  constexpr bool BYROW = !RES && BR % 4 == 0;        // stage and write one block row at a time
  constexpr int SR = sb_stride<D, DEG, RES>(NS);
  const int64_t c0 = t * 32, e = c0 + lane;
  float u[NS][D], Pm[D][D], H[P];
#pragma unroll
  for (int r = 0; r < NS; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) u[r][c] = 0.f;
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int c = 0; c < D; ++c) Pm[a][c] = 0.f;
#pragma unroll
  for (int q = 0; q < P; ++q) H[q] = 0.f;
  if (e < p.ncells) {
    int vid[NV], did[NS];
    bool bad = false;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      vid[v] = __ldg(p.c2v + e * NV + v);
      if (p.validate && (vid[v] < 0 || vid[v] >= p.nverts)) bad = true;
    }
#pragma unroll
    for (int r = 0; r < NS; ++r) {
      did[r] = __ldg(p.c2d + e * NS + r);
      if (p.validate && (did[r] < 0 || did[r] >= p.ncoefnodes)) bad = true;
    }
    if (bad) {
      atomicOr(p.err, ERR_INDEX);
    } else {
      // u's loads first, so that they and the coordinates' share one round trip to memory
      coef_rows<NS, D>(p, did, u);
      float adj[D][D], Dm, sg;
      cell_geometry_ids<D, true>(p, vid, adj, Dm, sg);
      const float inv = 1.0f / Dm, nu = (float)p.nu;
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int c = 0; c < D; ++c) Pm[a][c] = sg * adj[a][c];
      int q = 0;
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a; b < D; ++b) {
          float s = 0.f;
#pragma unroll
          for (int r = 0; r < D; ++r) s = fmaf(adj[a][r], adj[b][r], s);
          H[q++] = nu * s * inv;
        }
    }
  }
  // C, shared by the diagonal blocks
  float Q[NS][D];  // Q[r][a] = sum_c u[r][c] P[a][c]
#pragma unroll
  for (int r = 0; r < NS; ++r)
#pragma unroll
    for (int a = 0; a < D; ++a) {
      float q = 0.f;
#pragma unroll
      for (int c = 0; c < D; ++c) q = fmaf(u[r][c], Pm[a][c], q);
      Q[r][a] = q;
    }
  float C[NB];
#pragma unroll
  for (int o = 0; o < NB; ++o) {
    float v = 0.f;
#pragma unroll
    for (int r = 0; r < NS; ++r)
#pragma unroll
      for (int a = 0; a < D; ++a) v = fmaf(Q[r][a], c_T[OFF + (K1 + r * D + a) * NB + o], v);
#pragma unroll
    for (int q = 0; q < P; ++q) v = fmaf(H[q], c_T[OFF + (2 * K1 + q) * NB + o], v);
    C[o] = v;
  }
  float* row = st + lane * SR;
  const int rows = (int)(p.ncells - c0 < 32 ? p.ncells - c0 : 32);
  if constexpr (RES) {
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        float v = 0.f;
#pragma unroll
        for (int s = 0; s < NS; ++s) v = fmaf(C[i * NS + s], u[s][c], v);
        row[c * NS + i] = v;
      }
  }
  if constexpr (BYROW) {
    // one block row per pass, the loop kept rolled (unrolled, the compiler interleaved the passes
    // and needed 255 registers): the component's u column selected without indexing by ci
#pragma unroll 1
    for (int ci = 0; ci < D; ++ci) {
      float uc[NS];
#pragma unroll
      for (int r = 0; r < NS; ++r) uc[r] = ci == 0 ? u[r][0] : (D > 2 && ci == 2) ? u[r][D - 1] : u[r][1 % D];
#pragma unroll
      for (int o = 0; o < NB; ++o) {
        float V[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          float v = 0.f;
#pragma unroll
          for (int r = 0; r < NS; ++r) v = fmaf(uc[r], c_T[OFF + (r * D + a) * NB + o], v);
          V[a] = v;
        }
        const int i = o / NS, j = o % NS;
#pragma unroll
        for (int cj = 0; cj < D; ++cj) {
          float v = ci == cj ? C[o] : 0.f;
#pragma unroll
          for (int a = 0; a < D; ++a) v = fmaf(Pm[a][cj], V[a], v);
          row[i * NDOF + cj * NS + j] = v;
        }
      }
      // block row ci of the warp's cells: BR contiguous floats per cell, N apart
      __syncwarp();
      float* dst = p.out + c0 * N + ci * BR;
      if (rows == 32 && (reinterpret_cast<uintptr_t>(p.out) & 15) == 0) {
#pragma unroll 1
        for (int v4 = lane; v4 < 8 * BR; v4 += 32) {
          const int cell = v4 / (BR / 4), off = 4 * (v4 - cell * (BR / 4));
          const float* sr = st + cell * SR + off;
          __stcs(reinterpret_cast<float4*>(dst + (int64_t)cell * N + off), make_float4(sr[0], sr[1], sr[2], sr[3]));
        }
      } else {
#pragma unroll 1
        for (int x = lane; x < rows * BR; x += 32) {
          const int cell = x / BR, off = x - cell * BR;
          __stcs(dst + (int64_t)cell * N + off, st[cell * SR + off]);
        }
      }
      __syncwarp();
    }
    return;
  }
#pragma unroll
  for (int ci = 0; ci < (RES ? 0 : D); ++ci) {
#pragma unroll
    for (int o = 0; o < NB; ++o) {
      float V[D];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        float v = 0.f;
#pragma unroll
        for (int r = 0; r < NS; ++r) v = fmaf(u[r][ci], c_T[OFF + (r * D + a) * NB + o], v);
        V[a] = v;
      }
      const int i = o / NS, j = o % NS;
#pragma unroll
      for (int cj = 0; cj < D; ++cj) {
        float v = ci == cj ? C[o] : 0.f;
#pragma unroll
        for (int a = 0; a < D; ++a) v = fmaf(Pm[a][cj], V[a], v);
        row[(ci * NS + i) * NDOF + cj * NS + j] = v;
      }
    }
  }
  __syncwarp();
  float* dst = p.out + c0 * N;
  if (rows == 32 && (reinterpret_cast<uintptr_t>(p.out) & 15) == 0) {
#pragma unroll 4
    for (int i = lane; i < 8 * N; i += 32) {
      float4 v;
      const int j = 4 * i;
      v.x = st[((j + 0) / N) * SR + (j + 0) % N];
      v.y = st[((j + 1) / N) * SR + (j + 1) % N];
      v.z = st[((j + 2) / N) * SR + (j + 2) % N];
      v.w = st[((j + 3) / N) * SR + (j + 3) % N];
      __stcs(reinterpret_cast<float4*>(dst) + i, v);
    }
  } else {
    for (int i = lane; i < rows * N; i += 32) __stcs(dst + i, st[(i / N) * SR + i % N]);
  }
  __syncwarp();
}

template <int D, int DEG, bool RES>
__global__ void __launch_bounds__(SIMT_BTHREADS) k_assemble_simt_burgers(const TcParams p) {
  extern __shared__ float stage[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* st = stage + warp * 32 * sb_stride<D, DEG, RES>(s_ns(D, DEG));
  const int64_t ntiles = (p.ncells + 31) / 32;
  for (int64_t t = (int64_t)blockIdx.x * (SIMT_BTHREADS / 32) + warp; t < ntiles;
       t += (int64_t)gridDim.x * (SIMT_BTHREADS / 32))
    simt_tile_burgers<D, DEG, RES>(p, t, lane, st);
}

// Resident blocks asked of the compiler (so registers): triangles hold 6 blocks (48 warps) at 40
// registers, which measured faster on P1 triangles (0.0304 -> 0.0289 ms on 2^21 cells) than the
// compiler's own choice; tetrahedra 4, advection-diffusion 3 (what the compiler chose unasked).
template <int FORM, int D, int DEG>
__global__ void __launch_bounds__(SIMT_THREADS, FORM == FORM_ADVDIFF ? 3 : D == 2 ? 6 : 4) k_assemble_simt(const TcParams p) {
  constexpr int NS = s_ns(D, DEG), N = NS * NS;
  extern __shared__ float stage[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* st = stage + warp * 32 * (N | 1);
  const int64_t ntiles = (p.ncells + 31) / 32;
  for (int64_t t = (int64_t)blockIdx.x * SIMT_WARPS + warp; t < ntiles; t += (int64_t)gridDim.x * SIMT_WARPS)
    simt_tile<FORM, D, DEG>(p, t, lane, st);
}

// Several groups in one launch (the CUDA-core share of a mixed batch): warp tiles are numbered
// across the groups (group g owns tiles tile0 .. of its cells), each warp finds the group of its
// tile and runs that shape's tile. The shapes are those the CUDA cores take by default.
constexpr int SB_SR = 37;  // staging stride of the largest of them (triangles P2: 36 entries)
template <int FORM, int D, int DEG>
__device__ __forceinline__ void simt_tile_b(const TcParams& p, int64_t t, int lane, float* st) {
  static_assert((s_ns(D, DEG) * s_ns(D, DEG) | 1) <= SB_SR, "batch staging stride");
  simt_tile<FORM, D, DEG>(p, t, lane, st);
}
__global__ void __launch_bounds__(SIMT_THREADS) k_simt_batch(const SimtGroup* __restrict__ groups, int ngroups,
                                                           int64_t ntiles) {
  extern __shared__ float stage[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* st = stage + warp * 32 * SB_SR;
  for (int64_t t = (int64_t)blockIdx.x * SIMT_WARPS + warp; t < ntiles; t += (int64_t)gridDim.x * SIMT_WARPS) {
    int g = 0;
    while (g + 1 < ngroups && groups[g + 1].tile0 <= t) ++g;
    const SimtGroup& G = groups[g];
    const int64_t lt = t - G.tile0;
    switch (G.kind) {
      case FORM_MASS * 8 + CELL_TRI * 4 + 1: simt_tile_b<FORM_MASS, 2, 1>(G.p, lt, lane, st); break;
      case FORM_MASS * 8 + CELL_TRI * 4 + 2: simt_tile_b<FORM_MASS, 2, 2>(G.p, lt, lane, st); break;
      case FORM_MASS * 8 + CELL_TET * 4 + 1: simt_tile_b<FORM_MASS, 3, 1>(G.p, lt, lane, st); break;
      case FORM_HELMHOLTZ * 8 + CELL_TRI * 4 + 1: simt_tile_b<FORM_HELMHOLTZ, 2, 1>(G.p, lt, lane, st); break;
      case FORM_HELMHOLTZ * 8 + CELL_TRI * 4 + 2: simt_tile_b<FORM_HELMHOLTZ, 2, 2>(G.p, lt, lane, st); break;
      case FORM_HELMHOLTZ * 8 + CELL_TET * 4 + 1: simt_tile_b<FORM_HELMHOLTZ, 3, 1>(G.p, lt, lane, st); break;
      case FORM_ADVDIFF * 8 + CELL_TRI * 4 + 1: simt_tile_b<FORM_ADVDIFF, 2, 1>(G.p, lt, lane, st); break;
      case FORM_ADVDIFF * 8 + CELL_TRI * 4 + 2: simt_tile_b<FORM_ADVDIFF, 2, 2>(G.p, lt, lane, st); break;
      case FORM_ADVDIFF * 8 + CELL_TET * 4 + 1: simt_tile_b<FORM_ADVDIFF, 3, 1>(G.p, lt, lane, st); break;
      default: break;  // the planner assigns only these shapes
    }
  }
}

using SimtKernel = void (*)(const TcParams);

template <int FORM, int D>
SimtKernel pick_deg(int degree) {
  switch (degree) {
    case 1: return k_assemble_simt<FORM, D, 1>;
    case 2: return k_assemble_simt<FORM, D, 2>;
    case 3: if constexpr (D == 2) return k_assemble_simt<FORM, D, 3>;
  }
  return nullptr;
}

SimtKernel pick(int form, int degree, int cell) {
  if (form == FORM_BURGERS || form == FORM_BURGERS_RES) {
    const bool res = form == FORM_BURGERS_RES;
    if (cell == CELL_TRI && degree == 1) return res ? k_assemble_simt_burgers<2, 1, true> : k_assemble_simt_burgers<2, 1, false>;
    if (cell == CELL_TRI && degree == 2) return res ? k_assemble_simt_burgers<2, 2, true> : k_assemble_simt_burgers<2, 2, false>;
    if (cell == CELL_TET && degree == 1) return res ? k_assemble_simt_burgers<3, 1, true> : k_assemble_simt_burgers<3, 1, false>;
    return nullptr;
  }
  if (cell == CELL_TRI) {
    switch (form) {
      case FORM_MASS: return pick_deg<FORM_MASS, 2>(degree);
      case FORM_HELMHOLTZ: return pick_deg<FORM_HELMHOLTZ, 2>(degree);
      case FORM_ADVDIFF: return pick_deg<FORM_ADVDIFF, 2>(degree);
    }
  } else if (cell == CELL_TET) {
    switch (form) {
      case FORM_MASS: return pick_deg<FORM_MASS, 3>(degree);
      case FORM_HELMHOLTZ: return pick_deg<FORM_HELMHOLTZ, 3>(degree);
      case FORM_ADVDIFF: return pick_deg<FORM_ADVDIFF, 3>(degree);
    }
  }
  return nullptr;
}

std::mutex g_simt_mu;
std::set<std::tuple<int, int, int, int>> g_simt_loaded;  // (device, form, degree, cell)

}  // namespace

int simt_supported(int form, int degree, int cell) {
  if (!(form == FORM_MASS || form == FORM_HELMHOLTZ || form == FORM_ADVDIFF || burgers_like(form))) return 0;
  if (!(cell == CELL_TRI || cell == CELL_TET)) return 0;
  const int d = cell == CELL_TRI ? 2 : 3;
  return degree >= 1 && degree <= s_maxdeg(burgers_like(form) ? FORM_BURGERS : form, d) ? 1 : 0;
}

// where the CUDA-core kernel is the faster one (measured, TF32X3 tensor-core kernel with its
// tuned knobs against this one, 1,572,864 tets and 2,097,152 triangles, every form): P1 on both
// cells (tets 1.3-2.2x, triangles 2.5-3.0x) and triangles P2 (1.35-1.8x); tets P2 and
// triangles P3 stay on the tensor cores (their 100-entry matrices cost the CUDA cores more FMAs
// than the tensor-core kernel's hand-offs)
int simt_default(int form, int degree, int cell) {
  // the Burgers forms: P1 (2^20 tets: Jacobian 0.221 vs 0.662 ms, residual 0.049 vs 0.078) and
  // triangles P2 (2^21 cells: 0.444 vs 0.520 ms, residual 0.137 vs 0.160)
  if (burgers_like(form)) return degree == 1 || (cell == CELL_TRI && degree == 2) ? 1 : 0;
  return degree == 1 || (cell == CELL_TRI && degree == 2) ? 1 : 0;
}

// T of (form, degree, cell) in the constant bank of the current device, written once
int simt_upload(int form, int degree, int cell) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  const int d = cell == CELL_TRI ? 2 : 3;
  std::lock_guard<std::mutex> lock(g_simt_mu);
  if (g_simt_loaded.count({dev, form, degree, cell})) return (int)cudaSuccess;
  std::vector<double> T;
  tc_reference_tensor(form, degree, cell, T);
  std::vector<float> f(T.size());
  for (size_t i = 0; i < T.size(); ++i) f[i] = (float)T[i];
  if ((int)f.size() != s_size(form, d, degree)) return (int)cudaErrorInvalidValue;
  e = cudaMemcpyToSymbol(c_T, f.data(), f.size() * sizeof(float), (size_t)s_off(form, d, degree) * sizeof(float),
                         cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return (int)e;
  g_simt_loaded.insert({dev, form, degree, cell});
  return (int)cudaSuccess;
}

int simt_kind(int form, int degree, int cell) { return form * 8 + cell * 4 + degree; }

int launch_simt_batch(const SimtGroup* groups, int ngroups, int64_t ntiles, int num_sms, void* stream) {
  if (ntiles == 0) return (int)cudaSuccess;
  const int smem = SIMT_WARPS * 32 * SB_SR * (int)sizeof(float);
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_simt_batch, SIMT_THREADS, smem);
  if (e != cudaSuccess) return (int)e;
  if (per_sm < 1) per_sm = 1;
  const int64_t blocks_needed = (ntiles + SIMT_WARPS - 1) / SIMT_WARPS;
  const int64_t full = (int64_t)num_sms * per_sm;
  const int grid = (int)(blocks_needed < full ? blocks_needed : full);
  k_simt_batch<<<grid, SIMT_THREADS, smem, static_cast<cudaStream_t>(stream)>>>(groups, ngroups, ntiles);
  return (int)cudaGetLastError();
}

int launch_simt(int form, int degree, int cell, const TcParams& p, int num_sms, void* stream, std::string& why) {
  SimtKernel kern = simt_supported(form, degree, cell) ? pick(form, degree, cell) : nullptr;
  if (!kern) {
    why = "no CUDA-core kernel for this form/degree/cell";
    return (int)cudaErrorInvalidValue;
  }
  if (p.ncells == 0) return (int)cudaSuccess;
  cudaError_t e = cudaSuccess;
  const int d = cell == CELL_TRI ? 2 : 3, ns = s_ns(d, degree);
  const int nd = burgers_like(form) ? d * ns : ns, N = form == FORM_BURGERS_RES ? nd : nd * nd;
  // the residual contracts the Jacobian's tensors: one table for both
  if ((e = (cudaError_t)simt_upload(burgers_like(form) ? FORM_BURGERS : form, degree, cell)) != cudaSuccess) {
    why = "reference tensor upload";
    return (int)e;
  }
  const int threads = burgers_like(form) ? SIMT_BTHREADS : SIMT_THREADS, warps = threads / 32;
  // staging floats per cell: the element matrix (or vector), or one Burgers block row
  const int sr = !burgers_like(form) ? (N | 1)
                 : form == FORM_BURGERS_RES ? (nd | 1)
                 : (ns * nd) % 4 == 0 ? ((ns * nd) | 1) : (N | 1);
  const int smem = warps * 32 * sr * (int)sizeof(float);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return (int)e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (e != cudaSuccess) return (int)e;
  if (per_sm < 1) per_sm = 1;
  const int64_t warps_needed = (p.ncells + 31) / 32;
  const int64_t blocks_needed = (warps_needed + warps - 1) / warps;
  const int64_t full = (int64_t)num_sms * per_sm;
  const int grid = (int)(blocks_needed < full ? blocks_needed : full);
  kern<<<grid, threads, smem, static_cast<cudaStream_t>(stream)>>>(p);
  return (int)cudaGetLastError();
}

}  // namespace coffee
