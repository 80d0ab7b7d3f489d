// tcgen05 tensor-core local assembly for sm_103a.
//
// The quadrature loop nest of section 2 (Listings 1-2) is pre-summed into fixed
// reference tensors T[k][o] (o = i*ns + j), so that every element matrix is
//   A_e[o] = sum_k G_e[k] T[k][o]
// with per-cell factors G_e (|det J|, |det J| K K^T, coefficient-weighted terms) --
// section 3.3's outer-product view applied across cells: one dense contraction of
// shape (outputs x K) . (K x cells) per tile of 128 cells, on the 5th-generation
// tensor cores.
//
// Work decomposition (one persistent CTA per SM, cells tiled by 128):
//   producer warps 4..11  (two groups on alternate tiles) gather each cell's vertices (and coefficient dofs),
//                         compute J, det, adj in FP32 (FP64 when the cell is badly
//                         conditioned) and the factors G_e (stiffness in the edge basis
//                         c_ij = |det J| grad(lambda_i).grad(lambda_j)), split them into
//                         tensor-core operands (tf32 or bf16, one to three parts per
//                         precision) and store them as the B operand (cells x K,
//                         K-major) of a shared-memory stage;
//   MMA warp 12           one thread issues tcgen05.mma: D[o][cell] += T^T[o][k] G[cell][k]
//                         for every 128-row slice of the outputs into TMEM accumulators,
//                         one MMA per product of parts the precision keeps (Passes);
//   epilogue warps 0..3   tcgen05.ld the accumulator and store it: 128-byte warp stores
//                         of 32 outputs of one cell (outputs on the TMEM lanes), or
//                         16-byte stores of a thread's own row (cells on the lanes, for
//                         element matrices of at most 128 entries).
// T^T (the A operand) stays resident in shared memory for the whole launch.
// Every mbarrier wait is bounded (about 2 s of SM cycles); on expiry the
// kernel sets the error word and unwinds, freeing its TMEM.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstring>
#include <cmath>
#include "coffee_internal.h"
#include "tc_common.cuh"
#include "k_tc_kernel.cuh"

namespace coffee {
namespace {

using namespace tc;

template <int FORM, int D, int PREC>
cudaError_t launch_typed(const TcParams& p, int num_sms, cudaStream_t s, int nstages, int smem, bool lanes) {
  const int64_t ntiles = (p.ncells + BN - 1) / BN;
  const int grid = (int)std::min<int64_t>(ntiles, num_sms);
  if (lanes) {
    auto kern = k_assemble_tc<FORM, D, PREC, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, NTHREADS, smem, s>>>(p, nstages);
  } else {
    auto kern = k_assemble_tc<FORM, D, PREC, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, NTHREADS, smem, s>>>(p, nstages);
  }
  return cudaGetLastError();
}

template <int FORM, int D>
cudaError_t launch_prec(int prec, const TcParams& p, int num_sms, cudaStream_t s, int nst, int smem, bool lanes) {
  switch (prec) {
    case PREC_TF32: return launch_typed<FORM, D, PREC_TF32>(p, num_sms, s, nst, smem, lanes);
    case PREC_TF32X3: return launch_typed<FORM, D, PREC_TF32X3>(p, num_sms, s, nst, smem, lanes);
    case PREC_BF16: return launch_typed<FORM, D, PREC_BF16>(p, num_sms, s, nst, smem, lanes);
    case PREC_BF16X3: return launch_typed<FORM, D, PREC_BF16X3>(p, num_sms, s, nst, smem, lanes);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

int tc_supported(int form, int degree, int cell, int precision) {
  if (form == FORM_BURGERS) return burgers_tc_supported(degree, cell, precision);
  if (form == FORM_BURGERS_RES) return burgers_res_tc_supported(degree, cell, precision);
  Geom g;
  if (degree < 1 || degree > 4 || !geom_of(form, degree, cell, precision, g)) return 0;
  if (stages_for(g) > 0) return 1;
  return stream_one_supported(form, g.kbytes, precision);
}

// The stiffness reference tensors re-expressed for the edge factors of cell_factors: rows
// r0 .. r0+P-1 of T hold the pairs (a <= b) of reference directions and become the edges
// (i < j) of the simplex. With H_ab = c_{a+1,b+1} (a != b) and H_aa = -sum_{j != a+1} c_{a+1,j},
// sum_{a<=b} H_ab T_ab = sum_a c_{0,a+1} (-T_aa) + sum_{a<b} c_{a+1,b+1} (T_ab - T_aa - T_bb).
void to_edge_basis(std::vector<double>& T, int N, int r0, int d) {
  const int P = npairs(d);
  auto pr = [&](int a, int b) {  // row of the pair (a, b), a <= b
    for (int p = 0; p < P; ++p) {
      int x, y;
      pair_index(d, p, x, y);
      if (x == a && y == b) return r0 + p;
    }
    return -1;
  };
  std::vector<double> E((size_t)P * N);
  int e = 0;
  for (int i = 0; i <= d; ++i)
    for (int j = i + 1; j <= d; ++j, ++e)
      for (int o = 0; o < N; ++o) {
        double v;
        if (i == 0) v = -T[(size_t)pr(j - 1, j - 1) * N + o];
        else
          v = T[(size_t)pr(i - 1, j - 1) * N + o] - T[(size_t)pr(i - 1, i - 1) * N + o] -
              T[(size_t)pr(j - 1, j - 1) * N + o];
        E[(size_t)e * N + o] = v;
      }
  std::copy(E.begin(), E.end(), T.begin() + (size_t)r0 * N);
}

void tc_reference_tensor(int form, int degree, int cell, std::vector<double>& T) {
  reference_tensor(form, degree, cell, T);
  const int d = cell == CELL_TRI ? 2 : 3, P = npairs(d), ns = nnodes(cell, degree), N = ns * ns;
  if (form == FORM_HELMHOLTZ) to_edge_basis(T, N, 1, d);
  if (form == FORM_ADVDIFF)
    for (int v = 0; v <= d; ++v) to_edge_basis(T, N, v * P, d);
}

void build_tc_image(int form, int degree, int cell, int prec, std::vector<uint8_t>& img, TcTable& meta) {
  if (cell == CELL_PRISM) {
    build_prism_tc_image(form, degree, prec, img, meta);
    return;
  }
  if (form == FORM_BURGERS_RES) {  // the T2 and T3 columns only
    build_burgers_res_image(degree, cell, prec, img, meta);
    return;
  }
  if (form == FORM_BURGERS) {  // the Jacobian takes the exact integer form of A where it exists
    build_burgers_image(degree, cell, prec, true, img, meta);
    return;
  }
  Geom g{};
  geom_of(form, degree, cell, prec, g);
  std::vector<double> T;
  tc_reference_tensor(form, degree, cell, T);
  const bool tf32 = prec == PREC_TF32 || prec == PREC_TF32X3;
  const int elem = tf32 ? 4 : 2;
  const int64_t tile = (int64_t)BM * g.kbytes;
  img.assign((size_t)(g.mtiles * g.tparts * tile), 0);
  for (int m = 0; m < g.mtiles; ++m)
    for (int r = 0; r < BM; ++r) {
      const int o = m * BM + r;
      for (int k = 0; k < g.kelems; ++k) {
        const double x = (o < g.N && k < g.K) ? T[(size_t)k * g.N + o] : 0.0;
        host_store_parts(img.data() + (size_t)(m * g.tparts) * tile, (size_t)tile, canon_off(r, k * elem, g.kbytes), x,
                         tf32, g.tparts);
      }
    }
  meta = TcTable{};
  meta.mtiles = g.mtiles;
  meta.kbytes = g.kbytes;
  meta.kelems = g.kelems;
  meta.K = g.K;
  meta.tparts = g.tparts;
  meta.tile_bytes = tile;
}

int launch_tc(int form, int cell, const TcParams& p, int num_sms, void* stream, std::string& why) {
  if (p.ncells == 0) return (int)cudaSuccess;
  if (form == FORM_BURGERS) return launch_burgers_tc(cell, p, num_sms, stream, why);
  if (form == FORM_BURGERS_RES) return launch_burgers_res_tc(cell, p, num_sms, stream, why);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Geom g{};
  g.kbytes = p.kbytes;
  g.tparts = p.tparts;
  g.gparts = prec_gparts(p.precision);
  g.mtiles = p.mtiles;
  g.N = p.N;
  // cells on the lanes only pays for tiny element matrices (measured: P1 tets gain, P2 loses)
  const bool lanes = !(p.tune & TUNE_OUTPUT_LANES) && lanes_ok(p.mtiles) &&
                     (p.N <= 32 || (p.tune & TUNE_CELL_LANES));
  // cells per accumulator (outputs on lanes): narrower sub-tiles finish whole rows sooner,
  // which keeps the open rows of large element matrices within L2
  TcParams q = p;
  q.subw = (p.tune & TUNE_SUB32) ? 32 : (p.tune & TUNE_SUB64) ? 64 : (p.tune & TUNE_SUB128) ? 128
                                                                                             : (p.mtiles > 4 ? 64 : 128);
  int nst = stages_for(g);
  if (nst > 2 && (p.tune & TUNE_TWO_STAGES)) nst = 2;
  if (nst == 0) {
    // T^T does not fit beside the operand stages: stream it per M-tile instead
    BatchGroup bg;
    std::memset(&bg, 0, sizeof(bg));
    bg.p = p;
    bg.form = form;
    bg.cell = cell;
    if (!stream_one_supported(form, p.kbytes, p.precision)) {
      why = "operands do not fit in shared memory";
      return (int)cudaErrorInvalidValue;
    }
    return launch_stream_one(bg, num_sms, stream);
  }
  // staged epilogue (a tuning knob): rows of consecutive cells through shared memory and bulk
  // copies; direct warp stores otherwise
  if (!lanes && (p.tune & TUNE_STAGED_STORE)) {
    int w = 0, ch = 0, buf = 0;
    if (staged_plan(p, w, ch, buf)) {
      // as many row buffers as fit beside two operand stages (up to four), then the stages
      const int pad = round_up((int)sizeof(Barriers), 128) - (int)sizeof(Barriers);
      int nb = STAGE_BUFS;
      while (nb > 2 && stages_for(g, nb * buf + pad) < 2) --nb;
      const int extra = nb * buf + pad;
      int nss = stages_for(g, extra);
      if (nss > 2 && (p.tune & TUNE_TWO_STAGES)) nss = 2;
      if (nss > 0) {
        TcParams r = q;
        r.subw = w;
        r.stage_cells = ch;
        r.stage_bufs = nb;
        int smem = g.mtiles * g.tparts * BM * g.kbytes + nss * g.gparts * BN * g.kbytes + (int)sizeof(Barriers) +
                   extra + 1024 + 64;
        if (smem < SMEM_ONE_CTA) smem = SMEM_ONE_CTA;
        return launch_tc_staged(form, cell, r, num_sms, stream, nss, smem);
      }
    }
  }
  int smem = g.mtiles * g.tparts * BM * g.kbytes + nst * g.gparts * BN * g.kbytes +
             (int)sizeof(Barriers) + 1024 + 64;
  if (smem < SMEM_ONE_CTA) smem = SMEM_ONE_CTA;
  const bool tri = cell == CELL_TRI;
  cudaError_t e = cudaErrorInvalidValue;
  switch (form) {
    case FORM_MASS:
      e = tri ? launch_prec<FORM_MASS, 2>(q.precision, q, num_sms, s, nst, smem, lanes)
              : launch_prec<FORM_MASS, 3>(q.precision, q, num_sms, s, nst, smem, lanes);
      break;
    case FORM_HELMHOLTZ:
      e = tri ? launch_prec<FORM_HELMHOLTZ, 2>(q.precision, q, num_sms, s, nst, smem, lanes)
              : launch_prec<FORM_HELMHOLTZ, 3>(q.precision, q, num_sms, s, nst, smem, lanes);
      break;
    case FORM_ADVDIFF:
      e = tri ? launch_prec<FORM_ADVDIFF, 2>(q.precision, q, num_sms, s, nst, smem, lanes)
              : launch_prec<FORM_ADVDIFF, 3>(q.precision, q, num_sms, s, nst, smem, lanes);
      break;
  }
  return (int)e;
}

}  // namespace coffee
