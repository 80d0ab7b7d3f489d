// The tcgen05 local-assembly kernel with the staged epilogue (k_tc_kernel.cuh, SCH > 0): rows of
// consecutive cells gathered in shared memory and written by bulk copies. A translation unit of
// its own so that its instances compile in parallel with k_tc.cu's.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include "coffee_internal.h"
#include "tc_common.cuh"
#include "k_tc_kernel.cuh"

namespace coffee {
namespace {

using namespace tc;

template <int FORM, int D, int PREC>
cudaError_t launch_staged_typed(const TcParams& p, int num_sms, cudaStream_t s, int nstages, int smem) {
  const int64_t ntiles = (p.ncells + BN - 1) / BN;
  const int grid = (int)(ntiles < num_sms ? ntiles : num_sms);
  auto kern = p.stage_cells == 32 ? k_assemble_tc<FORM, D, PREC, false, false, 32>
                                  : k_assemble_tc<FORM, D, PREC, false, false, 8>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, NTHREADS, smem, s>>>(p, nstages);
  return cudaGetLastError();
}

template <int FORM, int D>
cudaError_t launch_staged_prec(const TcParams& p, int num_sms, cudaStream_t s, int nst, int smem) {
  switch (p.precision) {
    case PREC_TF32: return launch_staged_typed<FORM, D, PREC_TF32>(p, num_sms, s, nst, smem);
    case PREC_TF32X3: return launch_staged_typed<FORM, D, PREC_TF32X3>(p, num_sms, s, nst, smem);
    case PREC_BF16: return launch_staged_typed<FORM, D, PREC_BF16>(p, num_sms, s, nst, smem);
    case PREC_BF16X3: return launch_staged_typed<FORM, D, PREC_BF16X3>(p, num_sms, s, nst, smem);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

int staged_plan(const TcParams& p, int& subw, int& cells, int& buf_bytes) {
  // rows gathered for one bulk copy must be contiguous in the output
  if (p.mtiles > STAGE_MAXM || (reinterpret_cast<uintptr_t>(p.out) & 15) != 0 || p.ostride != p.N) return 0;
  // cells per accumulator: the explicit knob if every slice of a sub-tile fits the 512 TMEM
  // columns, else the widest that leaves room for two sub-tiles, else for one
  int w = (p.tune & TUNE_SUB32) ? 32 : (p.tune & TUNE_SUB64) ? 64 : (p.tune & TUNE_SUB128) ? 128 : 0;
  if (w == 0 || w * p.mtiles > 512) {
    w = 0;
    for (int c : {128, 64, 32})
      if (2 * c * p.mtiles <= 512) { w = c; break; }
    if (w == 0)
      for (int c : {128, 64, 32})
        if (c * p.mtiles <= 512) { w = c; break; }
  }
  if (w == 0) return 0;
  // rows per chunk (one TMEM load width, one bulk copy): 32 where two buffers of them stay
  // within about 80 KB of shared memory (up to 312 outputs), else 8
  const int ch = (w >= 32 && 2 * 32 * p.N * 4 <= 80 * 1024) ? 32 : 8;
  if (ch > w) return 0;
  subw = w;
  cells = ch;
  buf_bytes = ch * p.N * 4;
  return 1;
}

int launch_tc_staged(int form, int cell, const TcParams& q, int num_sms, void* stream, int nst, int smem) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool tri = cell == CELL_TRI;
  cudaError_t e = cudaErrorInvalidValue;
  switch (form) {
    case FORM_MASS:
      e = tri ? launch_staged_prec<FORM_MASS, 2>(q, num_sms, s, nst, smem)
              : launch_staged_prec<FORM_MASS, 3>(q, num_sms, s, nst, smem);
      break;
    case FORM_HELMHOLTZ:
      e = tri ? launch_staged_prec<FORM_HELMHOLTZ, 2>(q, num_sms, s, nst, smem)
              : launch_staged_prec<FORM_HELMHOLTZ, 3>(q, num_sms, s, nst, smem);
      break;
    case FORM_ADVDIFF:
      e = tri ? launch_staged_prec<FORM_ADVDIFF, 2>(q, num_sms, s, nst, smem)
              : launch_staged_prec<FORM_ADVDIFF, 3>(q, num_sms, s, nst, smem);
      break;
  }
  return (int)e;
}

}  // namespace coffee
