// Shared pieces of the Burgers tensor-core kernels (Jacobian: k_tc_burgers.cu; residual:
// k_tc_burgers_res.cu): the operand shape, the row store that forms factors as it stores,
// and the host-side geometry of the shared-memory operands.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <utility>
#include <type_traits>
#include "coffee_internal.h"
#include "tc_common.cuh"

namespace coffee {
namespace {
using namespace tc;

// Calls f(std::integral_constant<int, 0>), f(..1), .. up to N-1 while f returns true;
// true when every call did.
template <class F, int... I>
__device__ __forceinline__ bool static_for_impl(F&& f, std::integer_sequence<int, I...>) {
  return (f(std::integral_constant<int, I>{}) && ...);
}
template <int N, class F>
__device__ __forceinline__ bool static_for(F&& f) {
  return static_for_impl(f, std::make_integer_sequence<int, N>{});
}

template <int D, int NS, int PREC>
struct BurgersShape {
  using PT = PrecTraits<PREC>;
  static constexpr int KSTEP = PT::tf32 ? 8 : 16;
  static constexpr int ELEM = PT::tf32 ? 4 : 2;
  static constexpr int P = D * (D + 1) / 2;
  static constexpr int K1 = NS * D;                          // columns of T1 (and of T2)
  static constexpr int KA1 = round_up(K1, KSTEP);            // T1 padded: off-diagonal K
  static constexpr int KD = round_up(KA1 + K1 + P, KSTEP);   // diagonal K
  static constexpr int NBLK = NS * NS;
  static constexpr int MT = (NBLK + BM - 1) / BM;
  static constexpr int GPARTS = PT::GPARTS;                  // parts of the factor operand
  // Jacobian kernel: the B operand of a block is staged in K-chunks of CWB bytes per row. A
  // chunk is the whole block row: splitting it (more, smaller stages) was measured slower,
  // every extra hand-off between producers and the MMA costing more than it overlaps.
  static constexpr int CWB = KD * ELEM;
  static constexpr int CW = KD;                            // columns per chunk
  static constexpr int NCH_O = (KA1 + CW - 1) / CW;        // chunks of an off-diagonal block
  static constexpr int NCH_D = (KD + CW - 1) / CW;         // chunks of a diagonal block
  static constexpr int NCHT = D * NCH_D + (D * D - D) * NCH_O;  // chunks per tile
};

// One operand row (one cell): columns C0..NCOLS-1 whose k-th value is f(k), split into the
// precision's factor parts (part q at base + q * part_bytes) and stored 16 bytes at a time like
// store_operand_row; the values are formed as they are stored, so no K-long array is held in
// registers. C0 is a multiple of 8 elements.
template <int PREC, int NCOLS, class F, int C0 = 0>
__device__ __forceinline__ void store_operand_fn(uint8_t* base, int part_bytes, int r, int kbytes, F f) {
  using PT = PrecTraits<PREC>;
  constexpr int PER = PT::tf32 ? 4 : 8;  // columns per 16-byte unit
#pragma unroll
  for (int c = C0 / PER; c < NCOLS / PER; ++c) {
    float x[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) x[q] = f(c * PER + q);
    store_unit<PT::tf32, PT::GPARTS>(base + canon_off(r, c * 16, kbytes), part_bytes, x);
  }
}

// One K-chunk of an operand row: columns 0..CW-1 of the chunk take f(l) for l < ncols (a
// multiple of 4 tf32 / 8 bf16 columns; constant after unrolling) and are stored 16 bytes at a
// time in the canonical layout of a CWB-byte row; columns past ncols are not written.
template <int PREC, int CW, int CWB, class F>
__device__ __forceinline__ void store_chunk_fn(uint8_t* base, int part_bytes, int r, int ncols, F f) {
  using PT = PrecTraits<PREC>;
  constexpr int PER = PT::tf32 ? 4 : 8;  // columns per 16-byte unit
#pragma unroll
  for (int c = 0; c < CW / PER; ++c) {
    if (c * PER >= ncols) break;
    float x[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) x[q] = f(c * PER + q);
    store_unit<PT::tf32, PT::GPARTS>(base + canon_off(r, c * 16, CWB), part_bytes, x);
  }
}

constexpr int SMEM_LIMIT = 227 * 1024;
constexpr int SMEM_ONE_CTA = 120 * 1024;

struct BGeom {
  int ns, K1, KA1, KD, kstep, elem, mtiles, kbytes;
  int gparts;  // parts of the factor operand
  int aparts;  // parts of the resident A operand (1 when A is held exactly)
  int sbytes;  // shared-memory bytes of the A column scales (0 unless A is exact)
};
constexpr int SCALE_BYTES = 512;  // room for the column scales of any compiled shape

bool bgeom(int degree, int cell, int prec, BGeom& g) {
  if (prec == PREC_FP64 || prec < 0 || prec > PREC_BF16X3) return false;
  // compiled instances: triangles P1-P4, tetrahedra P1-P2
  if (cell == CELL_TRI ? (degree < 1 || degree > 4) : (degree < 1 || degree > 2)) return false;
  const int d = cell == CELL_TRI ? 2 : 3, P = d * (d + 1) / 2;
  const bool tf32 = prec == PREC_TF32 || prec == PREC_TF32X3;
  g.ns = nnodes(cell, degree);
  g.kstep = tf32 ? 8 : 16;
  g.elem = tf32 ? 4 : 2;
  g.K1 = g.ns * d;
  g.KA1 = (g.K1 + g.kstep - 1) / g.kstep * g.kstep;
  g.KD = (g.KA1 + g.K1 + P + g.kstep - 1) / g.kstep * g.kstep;
  g.gparts = prec_gparts(prec);
  g.mtiles = (g.ns * g.ns + BM - 1) / BM;
  g.kbytes = g.KD * g.elem;
  g.aparts = prec_tparts(prec);
  g.sbytes = 0;
  return true;
}

int bstages(const BGeom& g) {
  const int a = g.mtiles * g.aparts * BM * g.kbytes;
  const int b = g.gparts * BN * g.kbytes;
  const int fixed = a + (int)sizeof(Barriers) + g.sbytes + 1024 + 64;
  int s = MAX_STAGES;  // even: the stages are split between the two producer groups
  while (s >= 2 && fixed + s * b > SMEM_LIMIT) s -= 2;
  return s >= 2 ? s : 0;
}

// Stages of the Jacobian kernel: GPARTS x BN x CWB bytes each (CWB = kbytes), an even count.
int cstages(const BGeom& g) {
  const int a = g.mtiles * g.aparts * BM * g.kbytes;
  const int b = g.gparts * BN * g.kbytes;
  const int fixed = a + (int)sizeof(Barriers) + g.sbytes + 1024 + 64;
  int s = MAX_STAGES;
  while (s >= 2 && fixed + s * b > SMEM_LIMIT) s -= 2;
  return s >= 2 ? s : 0;
}

}  // namespace
}  // namespace coffee
