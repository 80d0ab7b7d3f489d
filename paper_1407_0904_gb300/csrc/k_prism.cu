// FP64 local assembly on prisms (the paper's third element shape, section 5.2): one warp per
// cell.
//
// A prism's map x(xi) = sum_v N_v(xi) X_v (degree-1 prism functions) is not affine, so the
// Jacobian, its determinant and inverse are evaluated at every quadrature point (the
// "Compute Jacobian" step of Listings 1-2 moves inside the quadrature loop) and the element
// matrix stays a quadrature sum:
//   A_e[o] = sum_q sum_kq G_e[q][kq] T[q*KQ + kq][o],
//   G_e[q] = w_q |det J_q| (1, (K_q K_q^T)_ab for a <= b)      (KQ = 1 mass, 7 Helmholtz),
//   G_e[q] = w_q |det J_q| (eps_q (K_q K_q^T)_ab, (K_q b_q)_a)  (KQ = 9 advection-diffusion,
//            eps and b degree-1 prism fields given at the six vertices),
// with per-point reference tensors T (tabulated on the host). The warp's lanes first compute
// the per-point factors G_e (one lane per point) into shared memory, then the outputs (one
// lane per entry, consecutive entries on consecutive lanes, so the reads of T and the stores
// of A_e are coalesced).
#include <cuda_runtime.h>
#include "coffee_internal.h"

namespace coffee {
namespace {

constexpr int PW = 4;  // warps (cells in flight) per block

template <int FORM, bool CSR>
__global__ void __launch_bounds__(PW * 32) k_assemble_prism(const PrismParams p) {
  extern __shared__ double psm[];
  constexpr int KQ = FORM == FORM_HELMHOLTZ ? 7 : FORM == FORM_ADVDIFF ? 9 : 1;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int K = p.Q * KQ, N = p.N;
  double* G = psm + (size_t)w * (K + 42);
  double* X = G + K;   // [6][3] vertices
  double* CF = X + 18;  // [6][4] (eps, b) at the vertices
  const double* __restrict__ T = p.T;
  const double* __restrict__ qp = p.T + (size_t)K * N;  // points [Q][3]
  const double* __restrict__ qw = qp + (size_t)p.Q * 3;  // weights [Q]
  for (int64_t e = (int64_t)blockIdx.x * PW + w; e < p.ncells; e += (int64_t)gridDim.x * PW) {
    bool bad = false;
    if (lane < 18) {
      const int v = lane / 3, r = lane % 3;
      const int vid = __ldg(p.c2v + e * 6 + v);
      if (p.validate && (vid < 0 || vid >= p.nverts)) bad = true;
      X[lane] = bad ? 0.0 : __ldg(p.coords + (int64_t)vid * 3 + r);
    }
    if constexpr (FORM == FORM_ADVDIFF) {
      if (lane < 24) {
        const int v = lane / 4, r = lane % 4;
        const int cid = __ldg(p.c2d + e * 6 + v);
        const bool badc = p.validate && (cid < 0 || cid >= p.ncoefnodes);
        if (badc) bad = true;
        CF[lane] = badc ? 0.0 : __ldg(p.coef + (int64_t)cid * 4 + r);
      }
    }
    if (__ballot_sync(0xffffffffu, bad)) {
      if (lane == 0) atomicOr(p.err, ERR_INDEX);
      __syncwarp();
      continue;
    }
    __syncwarp();
    // per-point geometry and factors
    for (int q = lane; q < p.Q; q += 32) {
      const double s = qp[q * 3], t = qp[q * 3 + 1], z = qp[q * 3 + 2];
      const double lam[3] = {1.0 - s - t, s, t};
      const double dls[3] = {-1.0, 1.0, 0.0}, dlt[3] = {-1.0, 0.0, 1.0};
      double J[3][3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        double js = 0.0, jt = 0.0, jz = 0.0;
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          const double lo = X[v * 3 + r], hi = X[(v + 3) * 3 + r];
          const double mid = (1.0 - z) * lo + z * hi;
          js += dls[v] * mid;
          jt += dlt[v] * mid;
          jz += lam[v] * (hi - lo);
        }
        J[r][0] = js;
        J[r][1] = jt;
        J[r][2] = jz;
      }
      // adjugate: adj[a][r] = cofactor C[r][a]; K = adj / det
      const double C00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
      const double C01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
      const double C02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
      const double det = J[0][0] * C00 + J[0][1] * C01 + J[0][2] * C02;
      const double adet = fabs(det);
      if constexpr (KQ != 9) G[q * KQ] = qw[q] * adet;
      if constexpr (KQ == 9) {
        const double adj[3][3] = {{C00, J[0][2] * J[2][1] - J[0][1] * J[2][2], J[0][1] * J[1][2] - J[0][2] * J[1][1]},
                                  {C01, J[0][0] * J[2][2] - J[0][2] * J[2][0], J[0][2] * J[1][0] - J[0][0] * J[1][2]},
                                  {C02, J[0][1] * J[2][0] - J[0][0] * J[2][1], J[0][0] * J[1][1] - J[0][1] * J[1][0]}};
        double eps = 0.0, bq[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int v = 0; v < 6; ++v) {
          const double Nv = v < 3 ? lam[v] * (1.0 - z) : lam[v - 3] * z;
          eps += Nv * CF[v * 4];
#pragma unroll
          for (int r = 0; r < 3; ++r) bq[r] += Nv * CF[v * 4 + 1 + r];
        }
        // eps |det| K K^T = eps adj adj^T / |det|;  |det| K b = sign(det) adj b
        int pp = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = a; b < 3; ++b) {
            double acc = 0.0;
#pragma unroll
            for (int r = 0; r < 3; ++r) acc += adj[a][r] * adj[b][r];
            G[q * KQ + pp++] = qw[q] * eps * acc / adet;
          }
        const double sg = det < 0.0 ? -1.0 : 1.0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
          G[q * KQ + 6 + a] = qw[q] * sg * (adj[a][0] * bq[0] + adj[a][1] * bq[1] + adj[a][2] * bq[2]);
      }
      if constexpr (KQ == 7) {
        const double adj[3][3] = {{C00, J[0][2] * J[2][1] - J[0][1] * J[2][2], J[0][1] * J[1][2] - J[0][2] * J[1][1]},
                                  {C01, J[0][0] * J[2][2] - J[0][2] * J[2][0], J[0][2] * J[1][0] - J[0][0] * J[1][2]},
                                  {C02, J[0][1] * J[2][0] - J[0][0] * J[2][1], J[0][0] * J[1][1] - J[0][1] * J[1][0]}};
        // |det| K K^T = adj adj^T / |det|
        int pp = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = a; b < 3; ++b) {
            double acc = 0.0;
#pragma unroll
            for (int r = 0; r < 3; ++r) acc += adj[a][r] * adj[b][r];
            G[q * KQ + 1 + pp++] = qw[q] * acc / adet;
          }
      }
    }
    __syncwarp();
    // contraction with the per-point reference tensors
    for (int o = lane; o < N; o += 32) {
      double acc = 0.0;
      for (int k = 0; k < K; ++k) acc = fma(G[k], __ldg(T + (size_t)k * N + o), acc);
      if constexpr (CSR) {
        const uint32_t pos = __ldg(p.map + csr_map_index(e, o, (N + 3) & ~3));
        if (pos < (uint64_t)p.nnz) atomicAdd(static_cast<double*>(p.out) + pos, acc);
        else atomicOr(p.err, ERR_INDEX);
      } else {
        static_cast<double*>(p.out)[e * (int64_t)N + o] = acc;
      }
    }
    __syncwarp();
  }
}

template <int FORM>
cudaError_t launch_form(const PrismParams& p, int num_sms, cudaStream_t s) {
  const int K = p.Q * (FORM == FORM_HELMHOLTZ ? 7 : FORM == FORM_ADVDIFF ? 9 : 1);
  const size_t smem = (size_t)PW * (K + 42) * sizeof(double);
  const int64_t blocks = (p.ncells + PW - 1) / PW;
  const unsigned grid = (unsigned)(blocks < (int64_t)num_sms * 16 ? blocks : (int64_t)num_sms * 16);
  if (p.map) {
    auto kern = k_assemble_prism<FORM, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, PW * 32, smem, s>>>(p);
  } else {
    auto kern = k_assemble_prism<FORM, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, PW * 32, smem, s>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace

int launch_prism(int form, const PrismParams& p, int num_sms, void* stream) {
  if (p.ncells == 0) return (int)cudaSuccess;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (form == FORM_MASS) return (int)launch_form<FORM_MASS>(p, num_sms, s);
  if (form == FORM_HELMHOLTZ) return (int)launch_form<FORM_HELMHOLTZ>(p, num_sms, s);
  if (form == FORM_ADVDIFF) return (int)launch_form<FORM_ADVDIFF>(p, num_sms, s);
  return (int)cudaErrorInvalidValue;
}

}  // namespace coffee
