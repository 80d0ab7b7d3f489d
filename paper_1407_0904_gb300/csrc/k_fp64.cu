// Plain FP64 local-assembly kernel: one thread per cell.
//
// This is the GPU counterpart of vectorising across elements (the paper's
// section 4, "inter-kernel vectorisation" when a kernel has no iteration space to
// vectorise): every thread runs the whole local-assembly kernel of section 2 for
// its own cell, in FP64:
//   1. gather the cell's vertex coordinates through cell2vert (and coefficient
//      values through cell2dof);
//   2. Jacobian J[r][c] = x_{c+1}[r] - x_0[r], det J and the adjugate (K = adj/det,
//      the "Compute Jacobian" step of Listings 1-2);
//   3. per-cell factors G[k] (the hoisted, loop-invariant quantities of
//      section 3.2: |det| K K^T, |det| K b, ...);
//   4. the element matrix as A[o] = sum_k G[k] T[k][o] against the reference
//      tensors T (the quadrature loop pre-summed on the host).
#include <cuda_runtime.h>
#include "coffee_internal.h"

namespace coffee {
namespace {

template <int D>
struct Geo {
  double adj[D][D];  // adjugate: K = adj / det
  double det;
};

template <int D>
__device__ __forceinline__ void geometry64(const double (&X)[D + 1][D], Geo<D>& g) {
  double J[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) J[r][c] = X[c + 1][r] - X[0][r];
  if constexpr (D == 2) {
    g.det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    g.adj[0][0] = J[1][1];
    g.adj[0][1] = -J[0][1];
    g.adj[1][0] = -J[1][0];
    g.adj[1][1] = J[0][0];
  } else {
    // cofactors C[r][c]; adj[a][r] = C[r][a]
    double C00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    double C01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    double C02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    double C10 = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    double C11 = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    double C12 = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    double C20 = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    double C21 = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    double C22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    g.det = J[0][0] * C00 + J[0][1] * C01 + J[0][2] * C02;
    g.adj[0][0] = C00; g.adj[0][1] = C10; g.adj[0][2] = C20;
    g.adj[1][0] = C01; g.adj[1][1] = C11; g.adj[1][2] = C21;
    g.adj[2][0] = C02; g.adj[2][1] = C12; g.adj[2][2] = C22;
  }
}

template <int FORM, int D>
struct FormK {
  static constexpr int P = D * (D + 1) / 2;
  static constexpr int value = FORM == FORM_MASS ? 1
                               : FORM == FORM_HELMHOLTZ ? 1 + P
                               : FORM == FORM_ADVDIFF ? (D + 1) * P + (D + 1) * D
                                                      : 1;
};

// CSR: global assembly -- every entry is added into the CSR value array p.out at the
// position p.map[cell][entry] instead of being stored.
template <int FORM, int D, bool CSR>
__global__ void __launch_bounds__(128) k_assemble_fp64(const Fp64Params p) {
  constexpr int NV = D + 1;
  constexpr int P = D * (D + 1) / 2;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p.ncells) return;

  // ---- 1. gather ----
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
  if constexpr (FORM == FORM_BURGERS || FORM == FORM_BURGERS_RES) {
    if (p.validate)
      for (int r = 0; r < p.ns; ++r) {
        int id = __ldg(p.c2d + e * p.ns + r);
        if (id < 0 || id >= p.ncoefnodes) bad = true;
      }
  }
  if (bad) {
    atomicOr(p.err, ERR_INDEX);
    return;
  }
  double X[NV][D];
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int r = 0; r < D; ++r) X[v][r] = __ldg(p.coords + (int64_t)vid[v] * D + r);

  // ---- 2. geometry ----
  Geo<D> g;
  geometry64<D>(X, g);
  const double Dm = fabs(g.det);
  const double sg = g.det < 0.0 ? -1.0 : 1.0;
  double H[P];  // |det| (K K^T)_{ab} = (adj adj^T)_{ab} / |det|, pairs a <= b
  {
    int q = 0;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = a; b < D; ++b) {
        double s = 0.0;
#pragma unroll
        for (int r = 0; r < D; ++r) s += g.adj[a][r] * g.adj[b][r];
        H[q++] = s / Dm;
      }
  }
  double Pm[D][D];  // |det| K = sign(det) adj
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int r = 0; r < D; ++r) Pm[a][r] = sg * g.adj[a][r];

  double* out = static_cast<double*>(p.out) + (CSR ? 0 : e * p.ostride);
  const int npad = (p.ndof * p.ndof + 3) & ~3;
  auto put = [&](int64_t idx, double v) {
    if constexpr (CSR) {
      const uint32_t pos = __ldg(p.map + csr_map_index(e, (int)idx, npad));
      if (pos < (uint64_t)p.nnz) atomicAdd(out + pos, v);
      else atomicOr(p.err, ERR_INDEX);
    } else {
      out[idx] = v;
    }
  };
  const double* __restrict__ T = p.T;
  const int N = p.N;

  if constexpr (FORM == FORM_BURGERS_RES) {
    // Burgers residual (element vector, component-blocked rows (c, i)). R is C(u) u with
    //   C[i][s] = sum_{r,a} Q[r][a] T2[r,a][i,s] + nu sum_p H_p T3[p][i,s],
    // the advective-viscous part of the Jacobian's diagonal block: for the quadratic
    // residual, (u.grad u) = sum_s u_s (u.grad phi_s) and grad u = sum_s u_s grad phi_s.
    const int ns = p.ns, nb = ns * ns;
    double u[35 * D];
    double Q[35 * D];
    for (int r = 0; r < ns; ++r) {
      const int id = __ldg(p.c2d + e * ns + r);
#pragma unroll
      for (int c = 0; c < D; ++c) u[r * D + c] = __ldg(p.coef + (int64_t)id * D + c);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < D; ++c) s += u[r * D + c] * Pm[a][c];
        Q[r * D + a] = s;
      }
    }
    const double* T2 = T + (int64_t)ns * D * nb;
    const double* T3 = T + (int64_t)2 * ns * D * nb;
    double* outv = static_cast<double*>(p.out) + e * p.ostride;
    for (int i = 0; i < ns; ++i) {
      double R[D];
#pragma unroll
      for (int c = 0; c < D; ++c) R[c] = 0.0;
      for (int s = 0; s < ns; ++s) {
        const int ob = i * ns + s;
        double cis = 0.0;
        for (int k = 0; k < ns * D; ++k) cis = fma(Q[k], __ldg(T2 + (int64_t)k * nb + ob), cis);
#pragma unroll
        for (int q = 0; q < P; ++q) cis = fma(p.nu * H[q], __ldg(T3 + (int64_t)q * nb + ob), cis);
#pragma unroll
        for (int c = 0; c < D; ++c) R[c] = fma(cis, u[s * D + c], R[c]);
      }
#pragma unroll
      for (int c = 0; c < D; ++c) outv[c * ns + i] = R[c];
    }
  } else if constexpr (FORM != FORM_BURGERS) {
    // ---- 3. per-cell factors ----
    constexpr int K = FormK<FORM, D>::value;
    double G[K];
    if constexpr (FORM == FORM_MASS) {
      G[0] = Dm;
    } else if constexpr (FORM == FORM_HELMHOLTZ) {
      G[0] = Dm;
#pragma unroll
      for (int q = 0; q < P; ++q) G[1 + q] = H[q];
    } else {  // ADVDIFF
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double* cv = p.coef + (int64_t)cid[v] * (D + 1);  // (eps, b) row of the node
        const double eps = __ldg(cv);
        double bv[D];
#pragma unroll
        for (int r = 0; r < D; ++r) bv[r] = __ldg(cv + 1 + r);
#pragma unroll
        for (int q = 0; q < P; ++q) G[v * P + q] = eps * H[q];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          double s = 0.0;
#pragma unroll
          for (int r = 0; r < D; ++r) s += Pm[a][r] * bv[r];
          G[NV * P + v * D + a] = s;
        }
      }
    }
    // ---- 4. contraction with the reference tensors ----
    for (int o = 0; o < N; ++o) {
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < K; ++k) acc = fma(G[k], __ldg(T + (int64_t)k * N + o), acc);
      put(o, acc);
    }
  } else {
    // Burgers Jacobian, block (ci, cj) of size ns x ns:
    //  sum_{r,a} u[r][ci] P[a][cj] T1[r,a] + [ci==cj] (sum_{r,a} Q[r][a] T2[r,a] + nu sum_p H[p] T3[p])
    // with Q[r][a] = sum_c u[r][c] P[a][c].
    const int ns = p.ns, nb = ns * ns, ndof = p.ndof;
    double u[35 * D];
    double Q[35 * D];
    for (int r = 0; r < ns; ++r) {
      const int id = __ldg(p.c2d + e * ns + r);
#pragma unroll
      for (int c = 0; c < D; ++c) u[r * D + c] = __ldg(p.coef + (int64_t)id * D + c);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < D; ++c) s += u[r * D + c] * Pm[a][c];
        Q[r * D + a] = s;
      }
    }
    const double* T1 = T;
    const double* T2 = T + (int64_t)ns * D * nb;
    const double* T3 = T + (int64_t)2 * ns * D * nb;
#pragma unroll
    for (int ci = 0; ci < D; ++ci)
      for (int i = 0; i < ns; ++i)
#pragma unroll
        for (int cj = 0; cj < D; ++cj)
          for (int j = 0; j < ns; ++j) {
            const int ob = i * ns + j;
            double acc = 0.0;
            for (int r = 0; r < ns; ++r) {
              double t = 0.0;
#pragma unroll
              for (int a = 0; a < D; ++a) t = fma(Pm[a][cj], __ldg(T1 + (int64_t)(r * D + a) * nb + ob), t);
              acc = fma(u[r * D + ci], t, acc);
            }
            if (ci == cj) {
              for (int r = 0; r < ns; ++r)
#pragma unroll
                for (int a = 0; a < D; ++a)
                  acc = fma(Q[r * D + a], __ldg(T2 + (int64_t)(r * D + a) * nb + ob), acc);
#pragma unroll
              for (int q = 0; q < P; ++q) acc = fma(p.nu * H[q], __ldg(T3 + (int64_t)q * nb + ob), acc);
            }
            put((int64_t)(ci * ns + i) * ndof + cj * ns + j, acc);
          }
  }
}

template <int FORM, int D>
cudaError_t launch_one(const Fp64Params& p, cudaStream_t s) {
  const int threads = 128;
  const int64_t blocks = (p.ncells + threads - 1) / threads;
  if (p.map) k_assemble_fp64<FORM, D, true><<<(unsigned)blocks, threads, 0, s>>>(p);
  else k_assemble_fp64<FORM, D, false><<<(unsigned)blocks, threads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

int launch_fp64(int form, int cell, const Fp64Params& p, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p.ncells == 0) return (int)cudaSuccess;
  const bool tri = cell == CELL_TRI;
  switch (form) {
    case FORM_MASS: return (int)(tri ? launch_one<FORM_MASS, 2>(p, s) : launch_one<FORM_MASS, 3>(p, s));
    case FORM_HELMHOLTZ:
      return (int)(tri ? launch_one<FORM_HELMHOLTZ, 2>(p, s) : launch_one<FORM_HELMHOLTZ, 3>(p, s));
    case FORM_ADVDIFF:
      return (int)(tri ? launch_one<FORM_ADVDIFF, 2>(p, s) : launch_one<FORM_ADVDIFF, 3>(p, s));
    case FORM_BURGERS:
      return (int)(tri ? launch_one<FORM_BURGERS, 2>(p, s) : launch_one<FORM_BURGERS, 3>(p, s));
    case FORM_BURGERS_RES:
      if (p.map) return (int)cudaErrorInvalidValue;  // element vectors have no matrix entry map
      return (int)(tri ? launch_one<FORM_BURGERS_RES, 2>(p, s) : launch_one<FORM_BURGERS_RES, 3>(p, s));
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace coffee
