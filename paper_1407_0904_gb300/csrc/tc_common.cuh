// Shared building blocks of the tcgen05 kernels: PTX wrappers (mbarrier, tcgen05,
// descriptors), operand splitting into tf32/bf16 parts, the canonical no-swizzle
// K-major shared-memory layout, and the FP32 cell geometry with its FP64 fallback.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstring>
#include "coffee_internal.h"

namespace coffee {
namespace tc {

constexpr int BN = 128;             // cells per tile = MMA N
constexpr int BM = 128;             // output rows per MMA = MMA M
constexpr int NTHREADS = 13 * 32;   // 4 epilogue, 8 producer (two groups), 1 MMA warp
constexpr int EPI_WARPS = 4;        // warps 0..3, one per TMEM lane quadrant
constexpr int PROD_WARP0 = 4;       // warps 4..11: producer groups 0 and 1 take alternate tiles
constexpr int PROD_GROUPS = 2;
constexpr int MMA_WARP = 12;

// Operand stages are split between the producer groups (stages g, g+2, ..): a group only
// ever waits for the release of its own previous use of a stage, one phase back, which
// is what parity-based mbarrier waits can tell apart. li is the item's index among its
// group's items; spg = stages per group.
__host__ __device__ __forceinline__ void stage_of(int64_t li, int grp, int spg, int& s, uint32_t& use) {
  s = grp + PROD_GROUPS * (int)(li % spg);
  use = (uint32_t)(li / spg);
}
constexpr int RING = 4;             // TMEM accumulator slots of BN columns
constexpr int TMEM_COLS = RING * BN;
constexpr int MAX_SLOTS = 16;       // accumulator slots of 32 columns (narrowest sub-tile)
constexpr int MAX_STAGES = 4;
constexpr long long WAIT_CYCLES = 4000000000ll;  // about 2 s at 2 GHz
constexpr float KAPPA_FP64 = 32.0f;  // Frobenius condition number above which geometry is FP64

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: true when the phase completed, false (and the error word set) on expiry.
// The bound is counted on the SM's own cycle counter: reading the global nanosecond timer
// costs a long-latency round trip, which a wait that is polled often (a pipeline hand-off that
// is not yet complete) would add to every hand-off.
static __device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned* err) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try(bar, parity)) return true;
    if (clock64() - t0 > WAIT_CYCLES) {
      atomicOr(err, ERR_TIMEOUT);
      return false;
    }
  }
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
// Shared-memory matrix descriptor, no swizzle, K-major canonical layout:
// core matrices of 8 rows x 16 bytes (128 contiguous bytes); LBO = distance between
// core matrices adjacent in K (128 B here), SBO = distance between 8-row groups.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;  // descriptor version of tcgen05
  return d;
}
// Instruction descriptor: D = f32, A/B = tf32 (2) or bf16 (1), both K-major, N, M.
__host__ __device__ constexpr uint32_t make_idesc(int ab_fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)ab_fmt << 7) | ((uint32_t)ab_fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
template <bool TF32>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  if constexpr (TF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
  }
}
// 32 lanes x 32 consecutive columns of 32-bit data -> 32 registers per thread
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
        "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
        "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
        "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 1-D bulk store of `bytes` (multiple of 16) from shared to global memory (bulk group).
__device__ __forceinline__ void bulk_s2g(void* dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// wait until at most one bulk group of this thread still reads its shared-memory source
__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// 32 lanes x 4 consecutive columns of 32-bit data -> 4 registers per thread
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&v)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
               : "r"(taddr));
}
// wait until at most N bulk groups of this thread still read their shared-memory source
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
// 32 lanes x 16 consecutive columns of 32-bit data -> 16 registers per thread
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

// ------------------------------------------------------- operand splitting
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// How each precision represents the two operands of the contraction A_e = sum_k G_e[k] T[k]:
// the reference tensor T in TPARTS parts and the per-cell factors G in GPARTS parts of the
// operand type (tf32 or bf16), every part the round-to-nearest of what the previous parts left.
//   TF32    T 1, G 1: one pass.
//   TF32X3  T 2, G 2 (hi + lo, 22 bits each): the three products of order <= 1.
//   BF16    T 2, G 1: T held to 16 bits, so only G's single rounding (2^-8) remains.
//   BF16X3  T 3, G 3 (24 bits each, the full float): the six products of order <= 2.
template <int PREC>
struct PrecTraits {
  static constexpr bool tf32 = PREC == PREC_TF32 || PREC == PREC_TF32X3;
  static constexpr int TPARTS = prec_tparts(PREC), GPARTS = prec_gparts(PREC);
};

// The MMA passes of a precision, (part of T, part of G), smallest products first so that the
// accumulator is small while they are added. TEXACT: T is held exactly in one part (integer
// columns), so only G's parts are passed.
template <int PREC, bool TEXACT = false>
struct Passes {
  static constexpr int N = TEXACT ? prec_gparts(PREC)
                                  : (PREC == PREC_TF32 ? 1 : PREC == PREC_TF32X3 ? 3 : PREC == PREC_BF16 ? 2 : 6);
  __host__ __device__ static constexpr int t(int i) {
    if (TEXACT) return 0;
    if (PREC == PREC_TF32X3) return i == 1 ? 1 : 0;                      // (0,1) (1,0) (0,0)
    if (PREC == PREC_BF16) return i == 0 ? 1 : 0;                        // (1,0) (0,0)
    if (PREC == PREC_BF16X3) return i == 0 ? 1 : i == 2 ? 2 : i == 4 ? 1 : 0;  // (1,1) (0,2) (2,0) (0,1) (1,0) (0,0)
    return 0;
  }
  __host__ __device__ static constexpr int g(int i) {
    if (TEXACT) return N - 1 - i;
    if (PREC == PREC_TF32X3) return i == 0 ? 1 : 0;
    if (PREC == PREC_BF16X3) return i == 0 ? 1 : i == 1 ? 2 : i == 3 ? 1 : 0;
    return 0;
  }
};

// x as NP parts of the operand type (tf32: 32-bit patterns with the low 13 bits clear; bf16:
// 16-bit patterns), each the round-to-nearest of the remainder the previous parts left; the
// remainders are exact in FP32.
template <bool TF32, int NP>
__device__ __forceinline__ void split_bits(float x, uint32_t (&b)[NP]) {
  float r = x;
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    if constexpr (TF32) {
      b[q] = tf32_rna(r);
      r -= __uint_as_float(b[q]);
    } else {
      const __nv_bfloat16 h = __float2bfloat16_rn(r);
      b[q] = (uint32_t)__bfloat16_as_ushort(h);
      r -= __bfloat162float(h);
    }
  }
}

// One 16-byte unit of each of the NP parts of an operand row from its values x[0..3] (tf32) or
// x[0..7] (bf16), stored at dst + q * part_bytes.
template <bool TF32, int NP>
__device__ __forceinline__ void store_unit(uint8_t* dst, int part_bytes, const float* x) {
  uint32_t w[NP][4];
  if constexpr (TF32) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      uint32_t b[NP];
      split_bits<true, NP>(x[c], b);
#pragma unroll
      for (int q = 0; q < NP; ++q) w[q][c] = b[q];
    }
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      uint32_t b0[NP], b1[NP];
      split_bits<false, NP>(x[2 * c], b0);
      split_bits<false, NP>(x[2 * c + 1], b1);
#pragma unroll
      for (int q = 0; q < NP; ++q) w[q][c] = b0[q] | (b1[q] << 16);
    }
  }
#pragma unroll
  for (int q = 0; q < NP; ++q)
    *reinterpret_cast<uint4*>(dst + (size_t)q * part_bytes) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
}

// Byte offset of (row r, byte kb) in a canonical K-major operand with kbytes per row.
__host__ __device__ __forceinline__ uint32_t canon_off(int r, int kb, int kbytes) {
  return (uint32_t)((r >> 3) * (8 * kbytes) + (kb >> 4) * 128 + (r & 7) * 16 + (kb & 15));
}

// Store the row of factors G[0..KP) for cell row r into the GPARTS parts of the B operand
// (part q at base + q * part_bytes). Only the first NCOLS columns (a multiple of the 16-byte
// unit) are written.
template <int PREC, int KP, int NCOLS = KP>
__device__ __forceinline__ void store_operand_row(uint8_t* base, int part_bytes, int r, const float (&G)[KP],
                                                  int kbytes) {
  using PT = PrecTraits<PREC>;
  constexpr int PER = PT::tf32 ? 4 : 8;  // columns per 16-byte unit
#pragma unroll
  for (int c = 0; c < NCOLS / PER; ++c)
    store_unit<PT::tf32, PT::GPARTS>(base + canon_off(r, c * 16, kbytes), part_bytes, &G[c * PER]);
}

__host__ __device__ constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }

// 2x2 minor a*d - b*c with one rounding error on the larger product term
__device__ __forceinline__ float minor2(float a, float d, float b, float c) {
  const float w = b * c;
  const float e = fmaf(-b, c, w);  // exact error of w
  const float f = fmaf(a, d, -w);
  return f + e;
}

// Adjugate (K = adj/det) and determinant in FP32 from the FP32 Jacobian; false when the cell is
// badly conditioned (Frobenius condition number above KAPPA_FP64).
template <int D>
__device__ __forceinline__ bool geometry_f32(const float (&J)[D][D], float (&adj)[D][D], float& det) {
  if constexpr (D == 2) {
    det = minor2(J[0][0], J[1][1], J[0][1], J[1][0]);
    adj[0][0] = J[1][1]; adj[0][1] = -J[0][1];
    adj[1][0] = -J[1][0]; adj[1][1] = J[0][0];
  } else {
    // adj[a][r] = cofactor[r][a]
    adj[0][0] = minor2(J[1][1], J[2][2], J[1][2], J[2][1]);
    adj[1][0] = minor2(J[1][2], J[2][0], J[1][0], J[2][2]);
    adj[2][0] = minor2(J[1][0], J[2][1], J[1][1], J[2][0]);
    adj[0][1] = minor2(J[0][2], J[2][1], J[0][1], J[2][2]);
    adj[1][1] = minor2(J[0][0], J[2][2], J[0][2], J[2][0]);
    adj[2][1] = minor2(J[0][1], J[2][0], J[0][0], J[2][1]);
    adj[0][2] = minor2(J[0][1], J[1][2], J[0][2], J[1][1]);
    adj[1][2] = minor2(J[0][2], J[1][0], J[0][0], J[1][2]);
    adj[2][2] = minor2(J[0][0], J[1][1], J[0][1], J[1][0]);
    det = fmaf(J[0][0], adj[0][0], fmaf(J[0][1], adj[1][0], J[0][2] * adj[2][0]));
  }
  float nj = 0.f, na = 0.f;
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      nj = fmaf(J[r][c], J[r][c], nj);
      na = fmaf(adj[r][c], adj[r][c], na);
    }
  // kappa_F^2 = |J|_F^2 |adj|_F^2 / det^2
  return nj * na <= KAPPA_FP64 * KAPPA_FP64 * det * det;
}

// The same in FP64 from the FP64 vertex coordinates, rounded to FP32 at the end.
template <int D>
__device__ __forceinline__ void geometry_f64(const double (&X)[D + 1][D], float (&adj)[D][D], float& det) {
  double Jd[D][D], A[D][D], dd;
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) Jd[r][c] = X[c + 1][r] - X[0][r];
  if constexpr (D == 2) {
    dd = Jd[0][0] * Jd[1][1] - Jd[0][1] * Jd[1][0];
    A[0][0] = Jd[1][1]; A[0][1] = -Jd[0][1]; A[1][0] = -Jd[1][0]; A[1][1] = Jd[0][0];
  } else {
    A[0][0] = Jd[1][1] * Jd[2][2] - Jd[1][2] * Jd[2][1];
    A[1][0] = Jd[1][2] * Jd[2][0] - Jd[1][0] * Jd[2][2];
    A[2][0] = Jd[1][0] * Jd[2][1] - Jd[1][1] * Jd[2][0];
    A[0][1] = Jd[0][2] * Jd[2][1] - Jd[0][1] * Jd[2][2];
    A[1][1] = Jd[0][0] * Jd[2][2] - Jd[0][2] * Jd[2][0];
    A[2][1] = Jd[0][1] * Jd[2][0] - Jd[0][0] * Jd[2][1];
    A[0][2] = Jd[0][1] * Jd[1][2] - Jd[0][2] * Jd[1][1];
    A[1][2] = Jd[0][2] * Jd[1][0] - Jd[0][0] * Jd[1][2];
    A[2][2] = Jd[0][0] * Jd[1][1] - Jd[0][1] * Jd[1][0];
    dd = Jd[0][0] * A[0][0] + Jd[0][1] * A[1][0] + Jd[0][2] * A[2][0];
  }
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int r = 0; r < D; ++r) adj[a][r] = (float)A[a][r];
  det = (float)dd;
}

// Rows of coefficients as the floats the kernels compute with, v[r][c] = coef[ids[r] * W + c]
// (0 for rows with ok[r] false when ok is given): read from the caller's float copy when given,
// else converted from the FP64 array (the same rounding). The copy is chosen once for all the
// rows, so the loads of every row issue back to back; a test per value would hold each load
// behind the previous one.
template <int R, int W>
__device__ __forceinline__ void coef_rows(const TcParams& p, const int (&ids)[R], float (&v)[R][W],
                                          const bool* ok = nullptr) {
  if (p.cf != nullptr) {
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < W; ++c) v[r][c] = (ok == nullptr || ok[r]) ? __ldg(p.cf + (int64_t)ids[r] * W + c) : 0.f;
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < W; ++c)
        v[r][c] = (ok == nullptr || ok[r]) ? (float)__ldg(p.coef + (int64_t)ids[r] * W + c) : 0.f;
  }
}

// x = hi + lo by integer operations, with no FP64 instruction: hi is x truncated to the 24
// significant bits of a float, lo the 29 fraction bits below them as an integer r, converted to
// float (rounded to nearest) and scaled exactly by the weight of the double's last bit,
// 2^(e - 1075) for the biased exponent e. So hi + lo holds x to 2^-48 of |x|, like the
// (hi, lo) pairs of coffee_split_coords. False for |x| outside [2^-70, 2^100) other than zero
// (hi = lo = 0 then), where the caller falls back to FP64.
__device__ __forceinline__ bool split_exact(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t h = (uint32_t)(b >> 32), l = (uint32_t)b;
  const uint32_t sign = h & 0x80000000u;
  const uint32_t ef = h & 0x7FF00000u;  // biased exponent e, in place
  // e == 0: zero (a binary64 subnormal, below 2^-1022, is taken as zero too)
  const bool zero = ef == 0u;
  const bool ok = zero || (ef - ((1023u - 70u) << 20)) < (170u << 20);
  // hi: the exponent field rebiased in place (e - 896 stays within 8 bits in range, so the
  // field's top three bits are clear), then the 20 + 3 fraction bits shifted into place
  const uint32_t hb = __funnelshift_l(l, h - (896u << 20), 3) | sign;
  // lo: the 29 bits below, times 2^(e - 1075) (float exponent field e - 948)
  const float unit = __uint_as_float((ef << 3) - (948u << 23));
  const float lm = __uint2float_rn(l & 0x1FFFFFFFu) * unit;
  hi = (ok && !zero) ? __uint_as_float(hb) : 0.f;
  lo = (ok && !zero) ? __uint_as_float(__float_as_uint(lm) | sign) : 0.f;
  return ok;
}

// Geometry of the cell with vertex ids vid: adj (K = adj/det), |det| and sign(det). The Jacobian
// J[r][c] = x_{c+1}[r] - x_0[r] is taken in FP32 from (hi, lo) float pairs of the coordinates,
// (hi1 - hi0) + (lo1 - lo0) (the hi difference is exact or rounded once, the lo one is 2^-24
// smaller, so J carries about two FP32 roundings), when the caller passed the pairs or, with
// ISPLIT, from pairs split here by integer operations (split_exact); else as the FP64 difference
// rounded to FP32. Badly conditioned cells are recomputed in FP64 from the FP64 coordinates.
template <int D, bool ISPLIT = false>
__device__ __forceinline__ void cell_geometry_ids(const TcParams& p, const int (&vid)[D + 1], float (&adj)[D][D],
                                                  float& Dm, float& sg) {
  float J[D][D], det;
  bool good;
  if (p.xs != nullptr) {
    const float2* xs = reinterpret_cast<const float2*>(p.xs);
    float2 x[D + 1][D];
#pragma unroll
    for (int v = 0; v < D + 1; ++v)
#pragma unroll
      for (int r = 0; r < D; ++r) x[v][r] = __ldg(xs + (int64_t)vid[v] * D + r);
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) J[r][c] = (x[c + 1][r].x - x[0][r].x) + (x[c + 1][r].y - x[0][r].y);
    good = geometry_f32<D>(J, adj, det);
    if (!good) {
      double X[D + 1][D];
#pragma unroll
      for (int v = 0; v < D + 1; ++v)
#pragma unroll
        for (int r = 0; r < D; ++r) X[v][r] = __ldg(p.coords + (int64_t)vid[v] * D + r);
      geometry_f64<D>(X, adj, det);
    }
  } else if constexpr (ISPLIT) {
    double X[D + 1][D];
#pragma unroll
    for (int v = 0; v < D + 1; ++v)
#pragma unroll
      for (int r = 0; r < D; ++r) X[v][r] = __ldg(p.coords + (int64_t)vid[v] * D + r);
    float2 x[D + 1][D];
    bool ok = true;
#pragma unroll
    for (int v = 0; v < D + 1; ++v)
#pragma unroll
      for (int r = 0; r < D; ++r) ok = split_exact(X[v][r], x[v][r].x, x[v][r].y) && ok;
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) J[r][c] = (x[c + 1][r].x - x[0][r].x) + (x[c + 1][r].y - x[0][r].y);
    good = geometry_f32<D>(J, adj, det) && ok;
    if (!good) geometry_f64<D>(X, adj, det);
  } else {
    double X[D + 1][D];
#pragma unroll
    for (int v = 0; v < D + 1; ++v)
#pragma unroll
      for (int r = 0; r < D; ++r) X[v][r] = __ldg(p.coords + (int64_t)vid[v] * D + r);
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) J[r][c] = (float)(X[c + 1][r] - X[0][r]);
    good = geometry_f32<D>(J, adj, det);
    if (!good) geometry_f64<D>(X, adj, det);
  }
  Dm = fabsf(det);
  sg = det < 0.f ? -1.f : 1.f;
}


// ----------------------------------------------------------- per-cell factors
template <int FORM, int D>
struct Form {
  static constexpr int P = D * (D + 1) / 2;
  static constexpr int K = FORM == FORM_MASS ? 1 : FORM == FORM_HELMHOLTZ ? 1 + P : (D + 1) * P + (D + 1) * D;
};

// Stiffness factors in the edge basis: c_ij = |det J| grad(lambda_i).grad(lambda_j) for the
// vertex pairs i < j of the simplex, ordered (0,1), (0,2), .., (0,d), (1,2), .., (d-1,d).
// With grad(lambda_{a+1}) = row a of K = adj / det and grad(lambda_0) = -sum_a grad(lambda_{a+1}),
// c_ij = g_i.g_j / |det| for g_{a+1} = adj[a], g_0 = -sum_a adj[a]. Because the barycentric
// gradients sum to zero these d(d+1)/2 numbers carry exactly the information of |det| K K^T
// (the host re-expresses the stiffness reference tensors for them), and on shape-regular cells
// they share one sign (no obtuse dihedral angle), so sum_k G_k T_k cancels far less than in the
// pairs of reference directions: the rounding of the factors to the operand type costs less.
template <int D>
__device__ __forceinline__ void edge_factors(const float (&adj)[D][D], float inv, float (&c)[D * (D + 1) / 2]) {
  float g[D + 1][D];
#pragma unroll
  for (int r = 0; r < D; ++r) {
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      g[a + 1][r] = adj[a][r];
      s += adj[a][r];
    }
    g[0][r] = -s;
  }
  int q = 0;
#pragma unroll
  for (int i = 0; i < D + 1; ++i)
#pragma unroll
    for (int j = i + 1; j < D + 1; ++j) {
      float s = 0.f;
#pragma unroll
      for (int r = 0; r < D; ++r) s = fmaf(g[i][r], g[j][r], s);
      c[q++] = s * inv;
    }
}

// Per-cell factors G[0..KP) (zero padded) for MASS / HELMHOLTZ / ADVDIFF.
// The cell's index rows (cell2vert, and cell2dof for ADVDIFF); loaded one tile ahead by
// the producers so that their DRAM latency overlaps the previous cell's work.
template <int FORM, int D>
struct CellIds {
  int vid[D + 1];
  int cid[FORM == FORM_ADVDIFF ? D + 1 : 1];
};

template <int FORM, int D>
__device__ __forceinline__ void load_ids(const TcParams& p, int64_t e, CellIds<FORM, D>& ids) {
  constexpr int NV = D + 1;
#pragma unroll
  for (int v = 0; v < NV; ++v) ids.vid[v] = __ldg(p.c2v + e * NV + v);
  if constexpr (FORM == FORM_ADVDIFF) {
#pragma unroll
    for (int v = 0; v < NV; ++v) ids.cid[v] = __ldg(p.c2d + e * NV + v);
  }
}

template <int FORM, int D, int KP, bool ISPLIT = false>
__device__ __forceinline__ void cell_factors_ids(const TcParams& p, const CellIds<FORM, D>& ids, float (&G)[KP],
                                                 bool& bad) {
  constexpr int NV = D + 1, P = D * (D + 1) / 2;
#pragma unroll
  for (int k = 0; k < KP; ++k) G[k] = 0.f;
  int vid[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    vid[v] = ids.vid[v];
    if (p.validate && (vid[v] < 0 || vid[v] >= p.nverts)) bad = true;
  }
  int cid[NV];
  if constexpr (FORM == FORM_ADVDIFF) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      cid[v] = ids.cid[v];
      if (p.validate && (cid[v] < 0 || cid[v] >= p.ncoefnodes)) bad = true;
    }
  }
  if (bad) return;
  float eb[FORM == FORM_ADVDIFF ? NV : 1][D + 1];  // (eps, b) row of each vertex's node
  if constexpr (FORM == FORM_ADVDIFF) coef_rows<NV, D + 1>(p, cid, eb);  // issued before the coordinates'
  float adj[D][D], Dm, sg;
  cell_geometry_ids<D, ISPLIT>(p, vid, adj, Dm, sg);
  float C[P];  // edge factors
  if constexpr (FORM != FORM_MASS) edge_factors<D>(adj, 1.0f / Dm, C);
  if constexpr (FORM == FORM_MASS) {
    G[0] = Dm;
  } else if constexpr (FORM == FORM_HELMHOLTZ) {
    G[0] = Dm;
#pragma unroll
    for (int q = 0; q < P; ++q) G[1 + q] = C[q];
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
#pragma unroll
      for (int q = 0; q < P; ++q) G[v * P + q] = eb[v][0] * C[q];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        float s = 0.f;
#pragma unroll
        for (int r = 0; r < D; ++r) s = fmaf(adj[a][r], eb[v][1 + r], s);
        G[NV * P + v * D + a] = sg * s;
      }
    }
  }
}

template <int FORM, int D, int KP>
__device__ __forceinline__ void cell_factors(const TcParams& p, int64_t e, float (&G)[KP], bool& bad) {
  CellIds<FORM, D> ids;
  load_ids<FORM, D>(p, e, ids);
  cell_factors_ids<FORM, D, KP>(p, ids, G, bad);
}

struct alignas(8) Barriers {
  uint64_t full[MAX_STAGES];
  uint64_t empty[MAX_STAGES];
  uint64_t tfull[MAX_SLOTS];
  uint64_t tempty[MAX_SLOTS];
  uint64_t aux[MAX_SLOTS];  // Burgers residual: the u buffer of each accumulator slot written
  uint64_t done;
  uint64_t epi;  // staged epilogue: the epilogue warps' own barrier (one phase per bulk copy)
  uint32_t tmem_base;
};

// host-side operand rounding (same rounding as the device conversions)
inline uint32_t host_tf32_rna(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7F800000u) != 0x7F800000u) u = (u + 0x1000u) & 0xFFFFE000u;
  return u;
}
inline float host_f(uint32_t u) {
  float x;
  std::memcpy(&x, &u, 4);
  return x;
}
inline uint16_t host_bf16_rn(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
inline float host_bf16_f(uint16_t h) { return host_f((uint32_t)h << 16); }
// x as np parts of the operand type (tf32 patterns, or bf16 patterns in the low 16 bits), each
// the round-to-nearest of the remainder left by the previous parts (remainders in FP64).
inline void host_split(double x, bool tf32, int np, uint32_t* b) {
  double r = x;
  for (int q = 0; q < np; ++q) {
    if (tf32) {
      b[q] = host_tf32_rna((float)r);
      r -= (double)host_f(b[q]);
    } else {
      b[q] = host_bf16_rn((float)r);
      r -= (double)host_bf16_f((uint16_t)b[q]);
    }
  }
}
// Store the np parts of x at byte offset off of parts base, base + part_bytes, ..
inline void host_store_parts(uint8_t* base, size_t part_bytes, uint32_t off, double x, bool tf32, int np) {
  uint32_t b[4];
  host_split(x, tf32, np, b);
  for (int q = 0; q < np; ++q) {
    if (tf32) std::memcpy(base + q * part_bytes + off, &b[q], 4);
    else {
      const uint16_t h = (uint16_t)b[q];
      std::memcpy(base + q * part_bytes + off, &h, 2);
    }
  }
}


}  // namespace tc
}  // namespace coffee
