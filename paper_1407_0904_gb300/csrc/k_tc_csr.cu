// Fused global assembly on the tensor cores: the local-assembly kernel of k_tc_kernel.cuh
// with its epilogue adding every element-matrix entry into the CSR value array of the
// global matrix (at the position given by the per-cell map) instead of storing it.
// The element matrices leave TMEM straight into L2 reductions; they are never written
// to memory. Orientation: outputs on the TMEM lanes (a warp's 32 lanes hold 32 entries
// of one cell, so its map reads are 128-byte rows).
#include <cuda_runtime.h>
#include <algorithm>
#include <cstring>
#include "coffee_internal.h"
#include "tc_common.cuh"
#include "k_tc_kernel.cuh"

namespace coffee {
namespace {

template <int FORM, int D, int PREC>
cudaError_t launch_csr_typed(const TcParams& p, int num_sms, cudaStream_t s, int nstages, int smem) {
  const int64_t ntiles = (p.ncells + BN - 1) / BN;
  const int grid = (int)std::min<int64_t>(ntiles, num_sms);
  auto kern = k_assemble_tc<FORM, D, PREC, false, true>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, NTHREADS, smem, s>>>(p, nstages);
  return cudaGetLastError();
}

template <int FORM, int D>
cudaError_t launch_csr_prec(const TcParams& p, int num_sms, cudaStream_t s, int nst, int smem) {
  switch (p.precision) {
    case PREC_TF32: return launch_csr_typed<FORM, D, PREC_TF32>(p, num_sms, s, nst, smem);
    case PREC_TF32X3: return launch_csr_typed<FORM, D, PREC_TF32X3>(p, num_sms, s, nst, smem);
    case PREC_BF16: return launch_csr_typed<FORM, D, PREC_BF16>(p, num_sms, s, nst, smem);
    case PREC_BF16X3: return launch_csr_typed<FORM, D, PREC_BF16X3>(p, num_sms, s, nst, smem);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

// The fused kernel keeps T^T resident in shared memory (no streamed variant) and covers
// the scalar forms.
int tc_csr_supported(int form, int degree, int cell, int precision) {
  if (form == FORM_BURGERS || degree < 1 || degree > 4) return 0;
  Geom g;
  if (!geom_of(form, degree, cell, precision, g)) return 0;
  return stages_for(g, CSR_SMEM) > 0 ? 1 : 0;
}

int launch_tc_csr(int form, int cell, const TcParams& p, int num_sms, void* stream, std::string& why) {
  if (p.ncells == 0) return (int)cudaSuccess;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Geom g{};
  g.kbytes = p.kbytes;
  g.tparts = p.tparts;
  g.gparts = prec_gparts(p.precision);
  g.mtiles = p.mtiles;
  g.N = p.N;
  int nst = stages_for(g, CSR_SMEM);
  if (nst == 0) {
    why = "operands do not fit in shared memory";
    return (int)cudaErrorInvalidValue;
  }
  if (nst > 2 && (p.tune & TUNE_TWO_STAGES)) nst = 2;
  TcParams q = p;
  q.subw = (p.tune & TUNE_SUB32) ? 32 : (p.tune & TUNE_SUB64) ? 64 : (p.tune & TUNE_SUB128) ? 128
                                                                                             : (p.mtiles > 4 ? 64 : 128);
  int smem = g.mtiles * g.tparts * BM * g.kbytes + nst * g.gparts * BN * g.kbytes + (int)sizeof(Barriers) + 1024 + 64 +
             CSR_SMEM;
  if (smem < SMEM_ONE_CTA) smem = SMEM_ONE_CTA;
  const bool tri = cell == CELL_TRI;
  cudaError_t e = cudaErrorInvalidValue;
  switch (form) {
    case FORM_MASS:
      e = tri ? launch_csr_prec<FORM_MASS, 2>(q, num_sms, s, nst, smem)
              : launch_csr_prec<FORM_MASS, 3>(q, num_sms, s, nst, smem);
      break;
    case FORM_HELMHOLTZ:
      e = tri ? launch_csr_prec<FORM_HELMHOLTZ, 2>(q, num_sms, s, nst, smem)
              : launch_csr_prec<FORM_HELMHOLTZ, 3>(q, num_sms, s, nst, smem);
      break;
    case FORM_ADVDIFF:
      e = tri ? launch_csr_prec<FORM_ADVDIFF, 2>(q, num_sms, s, nst, smem)
              : launch_csr_prec<FORM_ADVDIFF, 3>(q, num_sms, s, nst, smem);
      break;
  }
  return (int)e;
}

}  // namespace coffee
