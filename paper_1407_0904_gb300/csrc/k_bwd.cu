// Adjoint of local assembly: dL/dA_e -> dL/d(vertex coordinates), dL/d(coefficients).
//
// The paper has no backward pass; this is its reverse mode. With A_e = sum_k G_e[k] T[k]
// (the pre-summed quadrature of section 2's loop nest), the per-cell factor gradient is
//   Gbar_e[k] = sum_o T[k][o] dA_e[o],
// followed by the chain rule through the geometry, recomputed here rather than stored:
//   D = |det J|, K = J^{-1}, dD = D tr(K dJ), dK = -K dJ K,
//   G0 = D                    -> Jbar += Gbar0 D K^T
//   H  = D K K^T (pairs a<=b) -> Jbar += (D tr(Hbar K K^T) K - 2 D K K^T Hbar K)^T
//   P  = D K (advection)      -> Jbar += (D tr(Pbar^T K) K - D K Pbar^T K)^T
// and J[r][c] = x_{c+1}[r] - x_0[r] maps Jbar to the cell's vertices. Coefficient
// gradients: eps_v -> sum_p Gbar[v,p] H_p, b_{v,r} -> sum_a Gbar[v,a] P[a][r].
// One thread per cell; dA is staged through shared memory in chunks of 32 outputs so
// that its loads are coalesced. Cell contributions are either added with atomics or,
// in deterministic mode, written per cell and summed later in a fixed order.
#include <cuda_runtime.h>
#include <cstdint>
#include "coffee_internal.h"

namespace coffee {
namespace {

constexpr int BT = 128;  // cells (threads) per block
constexpr int CH = 32;   // outputs per staged chunk

template <int FORM, int D>
struct BForm {
  static constexpr int P = D * (D + 1) / 2;
  static constexpr int NV = D + 1;
  static constexpr int K = FORM == FORM_MASS ? 1 : FORM == FORM_HELMHOLTZ ? 1 + P : NV * P + NV * D;
  static constexpr int NCF = FORM == FORM_ADVDIFF ? NV * (1 + D) : 0;  // local coefficient values
  static constexpr int NL = NV * D + NCF;                              // local gradient length
};

template <typename T, int D>
__device__ __forceinline__ void adjugate(const T (&J)[D][D], T (&adj)[D][D], T& det) {
  if constexpr (D == 2) {
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    adj[0][0] = J[1][1]; adj[0][1] = -J[0][1];
    adj[1][0] = -J[1][0]; adj[1][1] = J[0][0];
  } else {
    adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
  }
}

// Local gradient L[0 .. NL): vertex coordinates (v*D + r), then the cell's coefficient values
// (eps_v for every vertex v, then b_{v,r}).
// The arithmetic runs in the type of dL/dA (CT = TA): FP64 for FP64 dL/dA, FP32 for FP32
// dL/dA (vertex differences are still taken in FP64 and rounded). Gradients are accumulated
// into FP64 arrays.
template <int FORM, int D, typename TA>
__global__ void __launch_bounds__(BT) k_backward(const BwdParams p) {
  using F = BForm<FORM, D>;
  using CT = TA;
  constexpr int NV = F::NV, P = F::P, K = F::K;
  __shared__ TA sA[BT][CH + 1];
  __shared__ CT sT[K][CH];

  const int t = threadIdx.x;
  const int64_t c0 = (int64_t)blockIdx.x * BT;
  const int64_t e = c0 + t;
  const bool live = e < p.ncells;
  const int nrows = (int)((p.ncells - c0) < BT ? (p.ncells - c0) : BT);
  const TA* dA = static_cast<const TA*>(p.dout);
  const int N = p.N;

  // ---- Gbar = T . vec(dA_e) ----
  CT Gb[K];
#pragma unroll
  for (int k = 0; k < K; ++k) Gb[k] = CT(0);
  for (int o0 = 0; o0 < N; o0 += CH) {
    const int w = (N - o0) < CH ? (N - o0) : CH;
    __syncthreads();
    for (int i = t; i < nrows * CH; i += BT) {
      const int r = i / CH, o = i - r * CH;
      sA[r][o] = o < w ? dA[(c0 + r) * N + o0 + o] : TA(0);
    }
    for (int i = t; i < K * CH; i += BT) {
      const int k = i / CH, o = i - k * CH;
      sT[k][o] = o < w ? (CT)p.T[(int64_t)k * N + o0 + o] : CT(0);
    }
    __syncthreads();
    if (live) {
      for (int o = 0; o < w; ++o) {
        const CT a = sA[t][o];
#pragma unroll
        for (int k = 0; k < K; ++k) Gb[k] = fma(sT[k][o], a, Gb[k]);
      }
    }
  }
  if (!live) return;

  // ---- geometry, recomputed ----
  int vid[NV];
  bool bad = false;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    vid[v] = __ldg(p.c2v + e * NV + v);
    if (p.validate && (vid[v] < 0 || vid[v] >= p.nverts)) bad = true;
  }
  int cid[NV];
  if constexpr (FORM == FORM_ADVDIFF) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      cid[v] = __ldg(p.c2d + e * NV + v);
      if (p.validate && (cid[v] < 0 || cid[v] >= p.ncoefnodes)) bad = true;
    }
  }
  if (bad) {
    atomicOr(p.err, ERR_INDEX);
    if (p.local)
      for (int i = 0; i < F::NL; ++i) p.local[e * F::NL + i] = 0.0;
    return;
  }
  double X[NV][D];
  CT J[D][D], adj[D][D], det;
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int r = 0; r < D; ++r) X[v][r] = __ldg(p.coords + (int64_t)vid[v] * D + r);
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) J[r][c] = (CT)(X[c + 1][r] - X[0][r]);
  adjugate<CT, D>(J, adj, det);
  const CT Dm = fabs(det), inv = CT(1) / det;
  CT Kx[D][D], KKt[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int r = 0; r < D; ++r) Kx[a][r] = adj[a][r] * inv;
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) {
      CT s = CT(0);
#pragma unroll
      for (int r = 0; r < D; ++r) s += Kx[a][r] * Kx[b][r];
      KKt[a][b] = s;
    }

  CT Jb[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) Jb[r][c] = CT(0);
  CT L[F::NL > 0 ? F::NL : 1];

  // mass term: G0 = |det|
  if constexpr (FORM == FORM_MASS || FORM == FORM_HELMHOLTZ) {
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) Jb[r][c] += Gb[0] * Dm * Kx[c][r];
  }
  // stiffness term: H = |det| K K^T with pair gradients Hbar
  if constexpr (FORM == FORM_HELMHOLTZ || FORM == FORM_ADVDIFF) {
    CT Hb[D][D];
    int q = 0;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = a; b < D; ++b) {
        CT g;
        if constexpr (FORM == FORM_HELMHOLTZ) {
          g = Gb[1 + q];
        } else {
          g = CT(0);
#pragma unroll
          for (int v = 0; v < NV; ++v) g += (CT)__ldg(p.coef + (int64_t)cid[v] * (D + 1)) * Gb[v * P + q];
        }
        if (a == b) {
          Hb[a][a] = g;
        } else {
          Hb[a][b] = CT(0.5) * g;
          Hb[b][a] = CT(0.5) * g;
        }
        ++q;
      }
    CT tr = CT(0);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) tr += Hb[a][b] * KKt[b][a];
    CT HK[D][D];  // Hbar K
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int r = 0; r < D; ++r) {
        CT s = CT(0);
#pragma unroll
        for (int b = 0; b < D; ++b) s += Hb[a][b] * Kx[b][r];
        HK[a][r] = s;
      }
    // M = D tr K - 2 D KKt HK ; Jbar += M^T
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int r = 0; r < D; ++r) {
        CT s = CT(0);
#pragma unroll
        for (int b = 0; b < D; ++b) s += KKt[a][b] * HK[b][r];
        Jb[r][a] += Dm * tr * Kx[a][r] - CT(2) * Dm * s;
      }
  }
  if constexpr (FORM == FORM_ADVDIFF) {
    // eps_v gradient: sum_p Gbar[v,p] H_p with H_p = D KKt[a][b]
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      CT s = CT(0);
      int q = 0;
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a; b < D; ++b) s += Gb[v * P + q++] * Dm * KKt[a][b];
      L[NV * D + v] = s;
    }
    // advection: G[v,a] = sum_r P[a][r] b_{v,r}, P = D K
    CT Pb[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int r = 0; r < D; ++r) Pb[a][r] = CT(0);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double* cv = p.coef + (int64_t)cid[v] * (D + 1);
#pragma unroll
      for (int r = 0; r < D; ++r) {
        const CT bvr = (CT)__ldg(cv + 1 + r);
        CT s = CT(0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
          Pb[a][r] += Gb[NV * P + v * D + a] * bvr;
          s += Gb[NV * P + v * D + a] * Dm * Kx[a][r];
        }
        L[NV * D + NV + v * D + r] = s;
      }
    }
    CT tr2 = CT(0);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int r = 0; r < D; ++r) tr2 += Pb[a][r] * Kx[a][r];
    CT PtK[D][D];  // Pbar^T K
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        CT s = CT(0);
#pragma unroll
        for (int a = 0; a < D; ++a) s += Pb[a][r] * Kx[a][c];
        PtK[r][c] = s;
      }
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        CT s = CT(0);
#pragma unroll
        for (int r = 0; r < D; ++r) s += Kx[a][r] * PtK[r][c];
        Jb[c][a] += Dm * tr2 * Kx[a][c] - Dm * s;
      }
  }
  // vertices: x_{c+1} += Jbar[:, c], x_0 -= sum_c Jbar[:, c]
#pragma unroll
  for (int r = 0; r < D; ++r) {
    CT s = CT(0);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      L[(c + 1) * D + r] = Jb[r][c];
      s += Jb[r][c];
    }
    L[r] = -s;
  }

  if (p.local) {  // deterministic mode: per-cell contributions, summed later in cell order
    double* dst = p.local + e * F::NL;
#pragma unroll
    for (int i = 0; i < F::NL; ++i) dst[i] = (double)L[i];
    return;
  }
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int r = 0; r < D; ++r) atomicAdd(p.d_coords + (int64_t)vid[v] * D + r, (double)L[v * D + r]);
  if constexpr (FORM == FORM_ADVDIFF) {
    if (p.d_coef) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        double* dc = p.d_coef + (int64_t)cid[v] * (D + 1);
        atomicAdd(dc, (double)L[NV * D + v]);
#pragma unroll
        for (int r = 0; r < D; ++r) atomicAdd(dc + 1 + r, (double)L[NV * D + NV + v * D + r]);
      }
    }
  }
}

// ---- deterministic reduction: per-node sums over incident cells in cell order ----
// count incidences of every node (integer atomics: the result is order independent)
// (out-of-range node ids are skipped and flagged, never dereferenced)
__global__ void k_count(const int32_t* idx, int64_t n, int64_t nnodes, int32_t* cnt, unsigned* err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t node = idx[i];
    if (node < 0 || node >= nnodes) {
      atomicOr(err, ERR_INDEX);
      continue;
    }
    atomicAdd(cnt + node, 1);
  }
}
// exclusive scan of cnt[0..n) into off[0..n] by one block (nodes are few: ~ncells/5)
__global__ void k_scan(const int32_t* cnt, int64_t n, int64_t* off) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x;
  const int64_t per = (n + blockDim.x - 1) / blockDim.x;
  const int64_t lo = t * per, hi = lo + per < n ? lo + per : n;
  int64_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += cnt[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int64_t acc = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      const int64_t v = part[i];
      part[i] = acc;
      acc += v;
    }
    off[n] = acc;
  }
  __syncthreads();
  int64_t acc = part[t];
  for (int64_t i = lo; i < hi; ++i) {
    off[i] = acc;
    acc += cnt[i];
  }
}
// slot list: entry i of idx (cell i / width, local position i % width) into its node's segment
__global__ void k_fill(const int32_t* idx, int64_t n, int64_t nnodes, const int64_t* off, int32_t* cursor,
                       int64_t* slots) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t node = idx[i];
    if (node < 0 || node >= nnodes) continue;
    const int32_t pos = atomicAdd(cursor + node, 1);
    slots[off[node] + pos] = i;
  }
}
// per node: sort its (short) segment by entry index, then sum contributions in that order
__global__ void k_gather(int64_t nnodes, const int64_t* off, int64_t* slots, const double* local, int nl,
                         int width, int base, int comps, int comp_stride_entry, double* grad,
                         int grad_stride, int grad_off) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nnodes; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = off[v], b = off[v + 1];
    for (int64_t i = a + 1; i < b; ++i) {  // insertion sort: segments hold ~24 entries
      const int64_t key = slots[i];
      int64_t j = i - 1;
      while (j >= a && slots[j] > key) {
        slots[j + 1] = slots[j];
        --j;
      }
      slots[j + 1] = key;
    }
    for (int c = 0; c < comps; ++c) {
      double s = 0.0;
      for (int64_t i = a; i < b; ++i) {
        const int64_t ent = slots[i];
        const int64_t cell = ent / width, pos = ent - cell * width;
        s += local[cell * nl + base + pos * comp_stride_entry + c];
      }
      grad[v * grad_stride + grad_off + c] += s;
    }
  }
}

template <int FORM, int D>
cudaError_t launch_bwd_t(const BwdParams& p, cudaStream_t s) {
  const int64_t blocks = (p.ncells + BT - 1) / BT;
  if (p.dout_fp32)
    k_backward<FORM, D, float><<<(unsigned)blocks, BT, 0, s>>>(p);
  else
    k_backward<FORM, D, double><<<(unsigned)blocks, BT, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

int bwd_local_len(int form, int cell) {
  const int d = cell == CELL_TRI ? 2 : 3;
  return (d + 1) * d + (form == FORM_ADVDIFF ? (d + 1) * (1 + d) : 0);
}

int launch_backward(int form, int cell, const BwdParams& p, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p.ncells == 0) return (int)cudaSuccess;
  const bool tri = cell == CELL_TRI;
  switch (form) {
    case FORM_MASS: return (int)(tri ? launch_bwd_t<FORM_MASS, 2>(p, s) : launch_bwd_t<FORM_MASS, 3>(p, s));
    case FORM_HELMHOLTZ:
      return (int)(tri ? launch_bwd_t<FORM_HELMHOLTZ, 2>(p, s) : launch_bwd_t<FORM_HELMHOLTZ, 3>(p, s));
    case FORM_ADVDIFF:
      return (int)(tri ? launch_bwd_t<FORM_ADVDIFF, 2>(p, s) : launch_bwd_t<FORM_ADVDIFF, 3>(p, s));
  }
  return (int)cudaErrorInvalidValue;
}

// Deterministic sum of per-cell contributions `local` [ncells][nl] into grad for the nodes
// referenced by idx [ncells][width] (entries idx[e*width + j] own `comps` consecutive values
// at local[e*nl + base + j*comps ..]); grad row v gets them at grad[v*grad_stride + grad_off].
// Scratch: cnt/cursor [nnodes] int32, off [nnodes+1] int64, slots [ncells*width] int64.
int launch_ordered_sum(const int32_t* idx, int64_t ncells, int width, int64_t nnodes, const double* local,
                       int nl, int base, int comps, double* grad, int grad_stride, int grad_off,
                       int32_t* cnt, int32_t* cursor, int64_t* off, int64_t* slots, unsigned* err,
                       void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t n = ncells * width;
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * nnodes, s);
  if (e != cudaSuccess) return (int)e;
  e = cudaMemsetAsync(cursor, 0, sizeof(int32_t) * nnodes, s);
  if (e != cudaSuccess) return (int)e;
  const unsigned g = (unsigned)((n + 255) / 256 < 152 * 16 ? (n + 255) / 256 : 152 * 16);
  k_count<<<g ? g : 1, 256, 0, s>>>(idx, n, nnodes, cnt, err);
  k_scan<<<1, 1024, 0, s>>>(cnt, nnodes, off);
  k_fill<<<g ? g : 1, 256, 0, s>>>(idx, n, nnodes, off, cursor, slots);
  const unsigned gv = (unsigned)((nnodes + 127) / 128 < 152 * 32 ? (nnodes + 127) / 128 : 152 * 32);
  k_gather<<<gv ? gv : 1, 128, 0, s>>>(nnodes, off, slots, local, nl, width, base, comps, comps, grad,
                                       grad_stride, grad_off);
  return (int)cudaGetLastError();
}

}  // namespace coffee
