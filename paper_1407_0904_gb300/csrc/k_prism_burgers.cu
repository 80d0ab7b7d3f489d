// FP64 assembly of vector Burgers on prisms (section 5.2 runs Burgers on the third element shape
// as well; Listing 2's problem): the Jacobian of
//   R[(c,i)] = int (u.grad u_c) phi_i + nu grad u_c . grad phi_i,
// or R itself, one warp per cell.
//
// The prism map is not affine, so the element matrix is the quadrature sum itself. It is
// evaluated directly from the basis at the points (per-point reference tensors, as the scalar
// prism kernel contracts, would take Q x 10 x n^2 doubles: 230 MB at P4). At each point q the
// warp first forms the cell's factors, one lane per point, into shared memory:
//   M[ci][cj] = w|det| d_cj u_ci,  beta_a = w|det| (K u)_a,  V_ab = w|det| nu (K K^T)_ab,
// with K = J^{-1} and d_m u_c = sum_a K[a][m] sum_r u[r][c] d_a phi_r; then each lane takes
// scalar pairs (i, j) and sums over the points
//   block(ci, cj)[i][j] = sum_q M[ci][cj] phi_i phi_j
//                       + [ci == cj] sum_q (phi_i beta . dphi_j + dphi_i^T V dphi_j),
// writing its nine entries (rows and columns blocked by component, as on simplices). The
// residual takes a_c = w|det| u.grad u_c and gamma_ca = w|det| nu (K grad u_c)_a and sums
// a_c phi_i + gamma_c . dphi_i per node i. The rule, the basis and its reference derivatives at
// the points come from the host's table (prism_burgers_table: (3k+3)/2 points per direction).
// Global assembly (CSR, the Jacobian): each entry is added into the CSR values at its map
// position (csr_map_index over the (3n)^2 entries of the cell) instead of being stored.
#include <cuda_runtime.h>
#include "coffee_internal.h"

namespace coffee {
namespace {

constexpr int PBW = 2;  // warps (cells in flight) per block

__host__ __device__ constexpr int pb_nodes(int k) { return (k + 1) * (k + 2) / 2 * (k + 1); }
__host__ __device__ constexpr int pb_factors(bool res) { return res ? 12 : 18; }
// doubles of shared memory per warp: the factors of every point, the vertices, u at the nodes
__host__ __device__ constexpr int pb_warp_doubles(int k, bool res, int Q) {
  return Q * pb_factors(res) + 18 + 3 * pb_nodes(k);
}

template <int DEG, bool RES, bool CSR>
__global__ void __launch_bounds__(PBW * 32) k_prism_burgers(const PrismParams p) {
  constexpr int n = pb_nodes(DEG), N = 3 * n, NF = pb_factors(RES);
  extern __shared__ double pbs[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int Q = p.Q;
  double* F = pbs + (size_t)w * pb_warp_doubles(DEG, RES, Q);
  double* X = F + (size_t)Q * NF;  // [6][3] vertices
  double* U = X + 18;              // [n][3] u at the cell's nodes
  const double* __restrict__ tab = p.T;                      // [Q][n][4]: phi, d_s, d_t, d_z
  const double* __restrict__ qp = p.T + (size_t)Q * n * 4;   // points [Q][3]
  const double* __restrict__ qw = qp + (size_t)Q * 3;        // weights [Q]
  const double nu = p.nu;
  for (int64_t e = (int64_t)blockIdx.x * PBW + w; e < p.ncells; e += (int64_t)gridDim.x * PBW) {
    bool bad = false;
    if (lane < 18) {
      const int v = lane / 3, r = lane % 3;
      const int vid = __ldg(p.c2v + e * 6 + v);
      if (p.validate && (vid < 0 || vid >= p.nverts)) bad = true;
      X[lane] = bad ? 0.0 : __ldg(p.coords + (int64_t)vid * 3 + r);
    }
    for (int r = lane; r < n; r += 32) {
      const int did = __ldg(p.c2d + e * n + r);
      const bool badc = p.validate && (did < 0 || did >= p.ncoefnodes);
      if (badc) bad = true;
#pragma unroll
      for (int c = 0; c < 3; ++c) U[r * 3 + c] = badc ? 0.0 : __ldg(p.coef + (int64_t)did * 3 + c);
    }
    if (__ballot_sync(0xffffffffu, bad)) {
      if (lane == 0) atomicOr(p.err, ERR_INDEX);
      __syncwarp();
      continue;
    }
    __syncwarp();
    // the cell's factors at every point
    for (int q = lane; q < Q; q += 32) {
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
      // adj[a][m] = cofactor (m, a); K = adj / det
      const double adj[3][3] = {{J[1][1] * J[2][2] - J[1][2] * J[2][1], J[0][2] * J[2][1] - J[0][1] * J[2][2],
                                 J[0][1] * J[1][2] - J[0][2] * J[1][1]},
                                {J[1][2] * J[2][0] - J[1][0] * J[2][2], J[0][0] * J[2][2] - J[0][2] * J[2][0],
                                 J[0][2] * J[1][0] - J[0][0] * J[1][2]},
                                {J[1][0] * J[2][1] - J[1][1] * J[2][0], J[0][1] * J[2][0] - J[0][0] * J[2][1],
                                 J[0][0] * J[1][1] - J[0][1] * J[1][0]}};
      const double det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
      double K[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int m = 0; m < 3; ++m) K[a][m] = adj[a][m] / det;
      // u and its reference gradients at the point, then the physical gradients
      double uq[3] = {0.0, 0.0, 0.0}, gr[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
      const double* tq = tab + (size_t)q * n * 4;
      for (int r = 0; r < n; ++r) {
        const double ph = __ldg(tq + r * 4), d0 = __ldg(tq + r * 4 + 1), d1 = __ldg(tq + r * 4 + 2),
                     d2 = __ldg(tq + r * 4 + 3);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double ur = U[r * 3 + c];
          uq[c] += ur * ph;
          gr[c][0] += ur * d0;
          gr[c][1] += ur * d1;
          gr[c][2] += ur * d2;
        }
      }
      double gu[3][3];  // d_m u_c
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int m = 0; m < 3; ++m) gu[c][m] = K[0][m] * gr[c][0] + K[1][m] * gr[c][1] + K[2][m] * gr[c][2];
      const double Dw = qw[q] * fabs(det);
      double* f = F + (size_t)q * NF;
      if constexpr (!RES) {
#pragma unroll
        for (int ci = 0; ci < 3; ++ci)
#pragma unroll
          for (int cj = 0; cj < 3; ++cj) f[ci * 3 + cj] = Dw * gu[ci][cj];
#pragma unroll
        for (int a = 0; a < 3; ++a) f[9 + a] = Dw * (K[a][0] * uq[0] + K[a][1] * uq[1] + K[a][2] * uq[2]);
        int pp = 12;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = a; b < 3; ++b) f[pp++] = Dw * nu * (K[a][0] * K[b][0] + K[a][1] * K[b][1] + K[a][2] * K[b][2]);
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          f[c] = Dw * (uq[0] * gu[c][0] + uq[1] * gu[c][1] + uq[2] * gu[c][2]);
#pragma unroll
          for (int a = 0; a < 3; ++a)
            f[3 + c * 3 + a] = Dw * nu * (gu[c][0] * K[a][0] + gu[c][1] * K[a][1] + gu[c][2] * K[a][2]);
        }
      }
    }
    __syncwarp();
    if constexpr (!RES) {
      double* out = CSR ? nullptr : static_cast<double*>(p.out) + e * (int64_t)N * N;
      for (int o = lane; o < n * n; o += 32) {
        const int i = o / n, j = o - (o / n) * n;
        double acc[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, dg = 0.0;
        for (int q = 0; q < Q; ++q) {
          const double* ti = tab + ((size_t)q * n + i) * 4;
          const double* tj = tab + ((size_t)q * n + j) * 4;
          const double pi = __ldg(ti), a0 = __ldg(ti + 1), a1 = __ldg(ti + 2), a2 = __ldg(ti + 3);
          const double pj = __ldg(tj), b0 = __ldg(tj + 1), b1 = __ldg(tj + 2), b2 = __ldg(tj + 3);
          const double* f = F + (size_t)q * NF;
          const double pm = pi * pj;
#pragma unroll
          for (int x = 0; x < 9; ++x) acc[x] += f[x] * pm;
          dg += pi * (f[9] * b0 + f[10] * b1 + f[11] * b2);
          dg += f[12] * a0 * b0 + f[13] * (a0 * b1 + a1 * b0) + f[14] * (a0 * b2 + a2 * b0) + f[15] * a1 * b1 +
                f[16] * (a1 * b2 + a2 * b1) + f[17] * a2 * b2;
        }
#pragma unroll
        for (int ci = 0; ci < 3; ++ci)
#pragma unroll
          for (int cj = 0; cj < 3; ++cj) {
            const int loc = (ci * n + i) * N + cj * n + j;
            const double v = acc[ci * 3 + cj] + (ci == cj ? dg : 0.0);
            if constexpr (CSR) {
              const uint32_t pos = __ldg(p.map + csr_map_index(e, loc, (N * N + 3) & ~3));
              if (pos < (uint64_t)p.nnz) atomicAdd(static_cast<double*>(p.out) + pos, v);
              else atomicOr(p.err, ERR_INDEX);
            } else {
              out[loc] = v;
            }
          }
      }
    } else {
      double* out = static_cast<double*>(p.out) + e * (int64_t)N;
      for (int i = lane; i < n; i += 32) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int q = 0; q < Q; ++q) {
          const double* ti = tab + ((size_t)q * n + i) * 4;
          const double pi = __ldg(ti), a0 = __ldg(ti + 1), a1 = __ldg(ti + 2), a2 = __ldg(ti + 3);
          const double* f = F + (size_t)q * NF;
#pragma unroll
          for (int c = 0; c < 3; ++c)
            acc[c] += f[c] * pi + f[3 + c * 3] * a0 + f[3 + c * 3 + 1] * a1 + f[3 + c * 3 + 2] * a2;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) out[c * n + i] = acc[c];
      }
    }
    __syncwarp();
  }
}

template <int DEG, bool RES>
cudaError_t launch_pb(const PrismParams& p, int num_sms, cudaStream_t s) {
  auto kern = (!RES && p.map) ? k_prism_burgers<DEG, RES, true> : k_prism_burgers<DEG, RES, false>;
  const size_t smem = (size_t)PBW * pb_warp_doubles(DEG, RES, p.Q) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (p.ncells + PBW - 1) / PBW;
  const unsigned grid = (unsigned)(blocks < (int64_t)num_sms * 8 ? blocks : (int64_t)num_sms * 8);
  kern<<<grid, PBW * 32, smem, s>>>(p);
  return cudaGetLastError();
}

template <bool RES>
cudaError_t launch_pb_deg(int degree, const PrismParams& p, int num_sms, cudaStream_t s) {
  switch (degree) {
    case 1: return launch_pb<1, RES>(p, num_sms, s);
    case 2: return launch_pb<2, RES>(p, num_sms, s);
    case 3: return launch_pb<3, RES>(p, num_sms, s);
    case 4: return launch_pb<4, RES>(p, num_sms, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

int launch_prism_burgers(int form, int degree, const PrismParams& p, int num_sms, void* stream) {
  if (p.ncells == 0) return (int)cudaSuccess;
  if (p.Q != prism_burgers_points(degree) * prism_burgers_points(degree) * prism_burgers_points(degree) ||
      p.N != pb_nodes(degree))
    return (int)cudaErrorInvalidValue;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return (int)(form == FORM_BURGERS_RES ? launch_pb_deg<true>(degree, p, num_sms, s)
                                        : launch_pb_deg<false>(degree, p, num_sms, s));
}

}  // namespace coffee
