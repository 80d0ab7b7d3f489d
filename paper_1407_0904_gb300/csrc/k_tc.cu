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
//   producer warps 8..11  gather each cell's vertices (and coefficient dofs),
//                         compute J, det, adj in FP32 (FP64 when the cell is badly
//                         conditioned) and the factors G_e, split them into
//                         tensor-core operands (tf32 or bf16, hi/lo for the split
//                         precisions) and store them as the B operand (cells x K,
//                         K-major) of a shared-memory stage;
//   MMA warp 12           one thread issues tcgen05.mma: D[o][cell] += T^T[o][k] G[cell][k]
//                         for every 128-row slice of the outputs, into a ring of
//                         four 128-column TMEM accumulators;
//   epilogue warps 0..7   tcgen05.ld a slice (lanes = outputs, columns = cells) and
//                         store it: a warp writes 32 consecutive outputs of one cell
//                         per instruction (128 contiguous bytes).
// T^T (the A operand) stays resident in shared memory for the whole launch.
// Every mbarrier wait is bounded (about 2 s of %globaltimer); on expiry the
// kernel sets the error word and unwinds, freeing its TMEM.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstring>
#include <cmath>
#include "coffee_internal.h"

namespace coffee {
namespace {

constexpr int BN = 128;             // cells per tile = MMA N
constexpr int BM = 128;             // output rows per MMA = MMA M
constexpr int NTHREADS = 13 * 32;   // 8 epilogue, 4 producer, 1 MMA warp
constexpr int PROD_WARP0 = 8;
constexpr int MMA_WARP = 12;
constexpr int RING = 4;             // TMEM accumulator slots of BN columns
constexpr int TMEM_COLS = RING * BN;
constexpr int MAX_STAGES = 4;
constexpr uint64_t WAIT_NS = 2000000000ull;
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
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: true when the phase completed, false (and the error word set) on expiry.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned* err) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try(bar, parity)) return true;
    if (global_ns() - t0 > WAIT_NS) {
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

// ------------------------------------------------------- operand splitting
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

template <int PREC>
struct PrecTraits;
template <>
struct PrecTraits<PREC_TF32> { static constexpr bool tf32 = true, split = false; };
template <>
struct PrecTraits<PREC_TF32X3> { static constexpr bool tf32 = true, split = true; };
template <>
struct PrecTraits<PREC_BF16> { static constexpr bool tf32 = false, split = false; };
template <>
struct PrecTraits<PREC_BF16X3> { static constexpr bool tf32 = false, split = true; };

// Byte offset of (row r, byte kb) in a canonical K-major operand with kbytes per row.
__host__ __device__ __forceinline__ uint32_t canon_off(int r, int kb, int kbytes) {
  return (uint32_t)((r >> 3) * (8 * kbytes) + (kb >> 4) * 128 + (r & 7) * 16 + (kb & 15));
}

// Store the row of factors G[0..KP) for cell row r into the hi (and lo) B operand parts.
template <int PREC, int KP>
__device__ __forceinline__ void store_operand_row(uint8_t* hi, uint8_t* lo, int r, const float (&G)[KP],
                                                  int kbytes) {
  using PT = PrecTraits<PREC>;
  if constexpr (PT::tf32) {
#pragma unroll
    for (int c = 0; c < KP / 4; ++c) {
      uint32_t h[4], l[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float x = G[c * 4 + q];
        h[q] = tf32_rna(x);
        l[q] = tf32_rna(x - __uint_as_float(h[q]));
      }
      const uint32_t off = canon_off(r, c * 16, kbytes);
      *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
      if constexpr (PT::split) *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
  } else {
#pragma unroll
    for (int c = 0; c < KP / 8; ++c) {
      uint32_t h[4], l[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float x0 = G[c * 8 + 2 * q], x1 = G[c * 8 + 2 * q + 1];
        __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
        __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
        __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
        h[q] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
        l[q] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
      }
      const uint32_t off = canon_off(r, c * 16, kbytes);
      *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
      if constexpr (PT::split) *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
  }
}

// ----------------------------------------------------------- per-cell factors
template <int FORM, int D>
struct Form {
  static constexpr int P = D * (D + 1) / 2;
  static constexpr int K = FORM == FORM_MASS ? 1 : FORM == FORM_HELMHOLTZ ? 1 + P : (D + 1) * P + (D + 1) * D;
};
__host__ __device__ constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }

// 2x2 minor a*d - b*c with one rounding error on the larger product term
__device__ __forceinline__ float minor2(float a, float d, float b, float c) {
  const float w = b * c;
  const float e = fmaf(-b, c, w);  // exact error of w
  const float f = fmaf(a, d, -w);
  return f + e;
}

// Geometry in FP32 from FP64 vertex differences; falls back to FP64 for badly
// conditioned cells. Produces adj (K = adj/det), |det| and sign(det).
template <int D>
__device__ __forceinline__ void cell_geometry(const double (&X)[D + 1][D], float (&adj)[D][D], float& Dm,
                                              float& sg) {
  float J[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) J[r][c] = (float)(X[c + 1][r] - X[0][r]);
  float det;
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
  const bool bad = !(nj * na <= KAPPA_FP64 * KAPPA_FP64 * det * det);
  if (bad) {
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
  Dm = fabsf(det);
  sg = det < 0.f ? -1.f : 1.f;
}

// Per-cell factors G[0..KP) (zero padded) for MASS / HELMHOLTZ / ADVDIFF.
template <int FORM, int D, int KP>
__device__ __forceinline__ void cell_factors(const TcParams& p, int64_t e, float (&G)[KP], bool& bad) {
  constexpr int NV = D + 1, P = D * (D + 1) / 2;
#pragma unroll
  for (int k = 0; k < KP; ++k) G[k] = 0.f;
  int vid[NV];
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
  if (bad) return;
  double X[NV][D];
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int r = 0; r < D; ++r) X[v][r] = __ldg(p.coords + (int64_t)vid[v] * D + r);
  float adj[D][D], Dm, sg;
  cell_geometry<D>(X, adj, Dm, sg);
  const float inv = 1.0f / Dm;
  float H[P];
  {
    int q = 0;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = a; b < D; ++b) {
        float s = 0.f;
#pragma unroll
        for (int r = 0; r < D; ++r) s = fmaf(adj[a][r], adj[b][r], s);
        H[q++] = s * inv;
      }
  }
  if constexpr (FORM == FORM_MASS) {
    G[0] = Dm;
  } else if constexpr (FORM == FORM_HELMHOLTZ) {
    G[0] = Dm;
#pragma unroll
    for (int q = 0; q < P; ++q) G[1 + q] = H[q];
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double* cv = p.coef + (int64_t)cid[v] * (D + 1);  // (eps, b) row of the node
      const float eps = (float)__ldg(cv);
      float bv[D];
#pragma unroll
      for (int r = 0; r < D; ++r) bv[r] = (float)__ldg(cv + 1 + r);
#pragma unroll
      for (int q = 0; q < P; ++q) G[v * P + q] = eps * H[q];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        float s = 0.f;
#pragma unroll
        for (int r = 0; r < D; ++r) s = fmaf(adj[a][r], bv[r], s);
        G[NV * P + v * D + a] = sg * s;
      }
    }
  }
}

// ------------------------------------------------------------------- kernel
struct alignas(8) Barriers {
  uint64_t full[MAX_STAGES];
  uint64_t empty[MAX_STAGES];
  uint64_t tfull[RING];
  uint64_t tempty[RING];
  uint64_t done;
  uint32_t tmem_base;
};

template <int FORM, int D, int PREC>
__global__ void __launch_bounds__(NTHREADS, 1) k_assemble_tc(const TcParams p, int nstages) {
  using PT = PrecTraits<PREC>;
  constexpr int KSTEP = PT::tf32 ? 8 : 16;  // K elements per MMA (32 bytes)
  constexpr int KP = round_up(Form<FORM, D>::K, KSTEP);
  constexpr int PARTS = PT::split ? 2 : 1;
  constexpr uint32_t IDESC = make_idesc(PT::tf32 ? 2 : 1, BM, BN);

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int kbytes = p.kbytes;
  const int tile_bytes = BM * kbytes;  // one part of one operand tile (A: 128 outputs, B: 128 cells)
  const int a_bytes = p.mtiles * PARTS * tile_bytes;
  uint8_t* sA = smem;
  uint8_t* sB = smem + a_bytes;
  Barriers* bars = reinterpret_cast<Barriers*>(sB + nstages * PARTS * tile_bytes);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (p.ncells + BN - 1) / BN;

  // ---- set-up: barriers, TMEM, resident A operand ----
  if (threadIdx.x == 0) {
    for (int s = 0; s < nstages; ++s) {
      mbar_init(smem_u32(&bars->full[s]), 128);
      mbar_init(smem_u32(&bars->empty[s]), 1);
    }
    for (int r = 0; r < RING; ++r) {
      mbar_init(smem_u32(&bars->tfull[r]), 1);
      mbar_init(smem_u32(&bars->tempty[r]), 8);
    }
    mbar_init(smem_u32(&bars->done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&bars->tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  {
    const uint4* src = reinterpret_cast<const uint4*>(p.image);
    uint4* dst = reinterpret_cast<uint4*>(sA);
    for (int i = threadIdx.x; i < a_bytes / 16; i += NTHREADS) dst[i] = __ldg(src + i);
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;

  if (warp >= PROD_WARP0 && warp < MMA_WARP) {
    // ---------------- producers: one cell per thread ----------------
    const int row = threadIdx.x - PROD_WARP0 * 32;
    int it = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const int s = it % nstages;
      const uint32_t use = (uint32_t)(it / nstages);
      if (!mbar_wait(smem_u32(&bars->empty[s]), (use & 1u) ^ 1u, p.err)) break;
      const int64_t e = t * BN + row;
      float G[KP];
      bool bad = false;
      if (e < p.ncells) {
        cell_factors<FORM, D, KP>(p, e, G, bad);
        if (bad) atomicOr(p.err, ERR_INDEX);
      }
      if (e >= p.ncells || bad) {
#pragma unroll
        for (int k = 0; k < KP; ++k) G[k] = 0.f;
      }
      uint8_t* hi = sB + (size_t)s * PARTS * tile_bytes;
      store_operand_row<PREC, KP>(hi, hi + tile_bytes, row, G, kbytes);
      fence_proxy_async();
      mbar_arrive(smem_u32(&bars->full[s]));
    }
  } else if (warp == MMA_WARP) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const int ksteps = kbytes / 32;
      const uint32_t sbo = 8u * (uint32_t)kbytes;
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      uint32_t rc = 0;  // TMEM ring counter
      int it = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++it) {
        const int s = it % nstages;
        const uint32_t use = (uint32_t)(it / nstages);
        if (!mbar_wait(smem_u32(&bars->full[s]), use & 1u, p.err)) break;
        tc_fence_after();
        const uint32_t bstage = b0 + (uint32_t)(s * PARTS * tile_bytes);
        for (int m = 0; m < p.mtiles; ++m, ++rc) {
          const uint32_t slot = rc % RING, round = rc / RING;
          if (!mbar_wait(smem_u32(&bars->tempty[slot]), (round & 1u) ^ 1u, p.err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t d = tmem + slot * BN;
          const uint32_t atile = a0 + (uint32_t)(m * PARTS * tile_bytes);
          uint32_t acc = 0;
          for (int ks = 0; ks < ksteps; ++ks) {
            const uint32_t ko = (uint32_t)ks * 256u;
            if constexpr (PT::split) {
              // small terms first: T_hi G_lo, T_lo G_hi, then T_hi G_hi
              mma<PT::tf32>(d, make_desc(atile + ko, sbo), make_desc(bstage + tile_bytes + ko, sbo), IDESC, acc);
              acc = 1;
              mma<PT::tf32>(d, make_desc(atile + tile_bytes + ko, sbo), make_desc(bstage + ko, sbo), IDESC, 1);
            }
            mma<PT::tf32>(d, make_desc(atile + ko, sbo), make_desc(bstage + ko, sbo), IDESC, acc);
            acc = 1;
          }
          tc_commit(smem_u32(&bars->tfull[slot]));
        }
        tc_commit(smem_u32(&bars->empty[s]));
      }
      // all issued MMAs complete before TMEM is released
      tc_commit(smem_u32(&bars->done));
      mbar_wait(smem_u32(&bars->done), 0, p.err);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: TMEM -> registers -> global ----------------
    const int q = warp & 3, half = warp >> 2;
    uint32_t rc = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const int64_t cbase = t * BN + half * 64;
      const int64_t rem = p.ncells - cbase;
      const int ncol = rem < 64 ? (int)rem : 64;
      for (int m = 0; m < p.mtiles; ++m, ++rc) {
        const uint32_t slot = rc % RING, round = rc / RING;
        if (!mbar_wait(smem_u32(&bars->tfull[slot]), round & 1u, p.err)) { ok = false; break; }
        tc_fence_after();
        const int o = m * BM + q * 32 + lane;
        if (m * BM + q * 32 < p.N && ncol > 0) {
          const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + slot * BN + half * 64;
          uint32_t v0[32], v1[32];
          tmem_ld32(taddr, v0);
          tmem_ld32(taddr + 32, v1);
          tmem_wait_ld();
          if (o < p.N) {
            float* dst = p.out + cbase * p.N + o;
            const int64_t stride = p.N;
            if (ncol == 64) {
#pragma unroll
              for (int j = 0; j < 32; ++j) __stcs(dst + j * stride, __uint_as_float(v0[j]));
#pragma unroll
              for (int j = 0; j < 32; ++j) __stcs(dst + (32 + j) * stride, __uint_as_float(v1[j]));
            } else {
#pragma unroll
              for (int j = 0; j < 32; ++j)
                if (j < ncol) __stcs(dst + j * stride, __uint_as_float(v0[j]));
#pragma unroll
              for (int j = 0; j < 32; ++j)
                if (32 + j < ncol) __stcs(dst + (32 + j) * stride, __uint_as_float(v1[j]));
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bars->tempty[slot]));
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == MMA_WARP) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                 : "memory");
  }
}

// ------------------------------------------------------------ host helpers
constexpr int SMEM_LIMIT = 227 * 1024;
constexpr int SMEM_ONE_CTA = 120 * 1024;  // requesting more keeps one CTA (and one TMEM owner) per SM

struct Geom {
  int K, kelems, kbytes, parts, mtiles, N;
};

bool geom_of(int form, int degree, int cell, int prec, Geom& g) {
  if (form == FORM_BURGERS) return false;
  if (prec == PREC_FP64) return false;
  const bool tf32 = prec == PREC_TF32 || prec == PREC_TF32X3;
  const int elem = tf32 ? 4 : 2, kstep = tf32 ? 8 : 16;
  g.K = form_K(form, degree, cell);
  g.kelems = (g.K + kstep - 1) / kstep * kstep;
  g.kbytes = g.kelems * elem;
  g.parts = (prec == PREC_TF32X3 || prec == PREC_BF16X3) ? 2 : 1;
  const int ns = nnodes(cell, degree);
  g.N = ns * ns;
  g.mtiles = (g.N + BM - 1) / BM;
  return true;
}

int stages_for(const Geom& g) {
  const int a = g.mtiles * g.parts * BM * g.kbytes;
  const int b = g.parts * BN * g.kbytes;
  const int fixed = a + (int)sizeof(Barriers) + 1024 + 64;
  int s = MAX_STAGES;
  while (s >= 2 && fixed + s * b > SMEM_LIMIT) --s;
  return s >= 2 ? s : 0;
}

uint32_t host_tf32_rna(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7F800000u) != 0x7F800000u) u = (u + 0x1000u) & 0xFFFFE000u;
  return u;
}
float host_f(uint32_t u) {
  float x;
  std::memcpy(&x, &u, 4);
  return x;
}
uint16_t host_bf16_rn(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
float host_bf16_f(uint16_t h) { return host_f((uint32_t)h << 16); }

template <int FORM, int D, int PREC>
cudaError_t launch_typed(const TcParams& p, int num_sms, cudaStream_t s, int nstages, int smem) {
  auto kern = k_assemble_tc<FORM, D, PREC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (p.ncells + BN - 1) / BN;
  const int grid = (int)std::min<int64_t>(ntiles, num_sms);
  kern<<<grid, NTHREADS, smem, s>>>(p, nstages);
  return cudaGetLastError();
}

template <int FORM, int D>
cudaError_t launch_prec(int prec, const TcParams& p, int num_sms, cudaStream_t s, int nst, int smem) {
  switch (prec) {
    case PREC_TF32: return launch_typed<FORM, D, PREC_TF32>(p, num_sms, s, nst, smem);
    case PREC_TF32X3: return launch_typed<FORM, D, PREC_TF32X3>(p, num_sms, s, nst, smem);
    case PREC_BF16: return launch_typed<FORM, D, PREC_BF16>(p, num_sms, s, nst, smem);
    case PREC_BF16X3: return launch_typed<FORM, D, PREC_BF16X3>(p, num_sms, s, nst, smem);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

int tc_supported(int form, int degree, int cell, int precision) {
  Geom g;
  if (degree < 1 || degree > 4 || !geom_of(form, degree, cell, precision, g)) return 0;
  return stages_for(g) > 0 ? 1 : 0;
}

void build_tc_image(int form, int degree, int cell, int prec, std::vector<uint8_t>& img, TcTable& meta) {
  Geom g;
  geom_of(form, degree, cell, prec, g);
  std::vector<double> T;
  reference_tensor(form, degree, cell, T);
  const bool tf32 = prec == PREC_TF32 || prec == PREC_TF32X3;
  const int elem = tf32 ? 4 : 2;
  const int64_t tile = (int64_t)BM * g.kbytes;
  img.assign((size_t)(g.mtiles * g.parts * tile), 0);
  for (int m = 0; m < g.mtiles; ++m)
    for (int r = 0; r < BM; ++r) {
      const int o = m * BM + r;
      for (int k = 0; k < g.kelems; ++k) {
        const double x = (o < g.N && k < g.K) ? T[(size_t)k * g.N + o] : 0.0;
        const float xf = (float)x;
        const uint32_t off = canon_off(r, k * elem, g.kbytes);
        uint8_t* hi = img.data() + (size_t)(m * g.parts) * tile;
        uint8_t* lo = hi + tile;
        if (tf32) {
          const uint32_t h = host_tf32_rna(xf);
          const uint32_t l = host_tf32_rna((float)(x - (double)host_f(h)));
          std::memcpy(hi + off, &h, 4);
          if (g.parts == 2) std::memcpy(lo + off, &l, 4);
        } else {
          const uint16_t h = host_bf16_rn(xf);
          const uint16_t l = host_bf16_rn((float)(x - (double)host_bf16_f(h)));
          std::memcpy(hi + off, &h, 2);
          if (g.parts == 2) std::memcpy(lo + off, &l, 2);
        }
      }
    }
  meta = TcTable{};
  meta.mtiles = g.mtiles;
  meta.kbytes = g.kbytes;
  meta.kelems = g.kelems;
  meta.K = g.K;
  meta.parts = g.parts;
  meta.tile_bytes = tile;
}

int launch_tc(int form, int cell, const TcParams& p, int num_sms, void* stream, std::string& why) {
  if (p.ncells == 0) return (int)cudaSuccess;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Geom g{};
  g.kbytes = p.kbytes;
  g.parts = p.parts;
  g.mtiles = p.mtiles;
  const int nst = stages_for(g);
  if (nst == 0) {
    why = "operands do not fit in shared memory";
    return (int)cudaErrorInvalidValue;
  }
  int smem = g.mtiles * g.parts * BM * g.kbytes + nst * g.parts * BN * g.kbytes + (int)sizeof(Barriers) + 1024 + 64;
  if (smem < SMEM_ONE_CTA) smem = SMEM_ONE_CTA;
  const bool tri = cell == CELL_TRI;
  cudaError_t e = cudaErrorInvalidValue;
  switch (form) {
    case FORM_MASS:
      e = tri ? launch_prec<FORM_MASS, 2>(p.precision, p, num_sms, s, nst, smem)
              : launch_prec<FORM_MASS, 3>(p.precision, p, num_sms, s, nst, smem);
      break;
    case FORM_HELMHOLTZ:
      e = tri ? launch_prec<FORM_HELMHOLTZ, 2>(p.precision, p, num_sms, s, nst, smem)
              : launch_prec<FORM_HELMHOLTZ, 3>(p.precision, p, num_sms, s, nst, smem);
      break;
    case FORM_ADVDIFF:
      e = tri ? launch_prec<FORM_ADVDIFF, 2>(p.precision, p, num_sms, s, nst, smem)
              : launch_prec<FORM_ADVDIFF, 3>(p.precision, p, num_sms, s, nst, smem);
      break;
  }
  return (int)e;
}

}  // namespace coffee
