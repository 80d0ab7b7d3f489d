// tcgen05 local assembly on prisms (the paper's third element shape, section 5.2).
//
// A prism's map is not affine, so the Jacobian is evaluated at every quadrature point and the
// element matrix is a quadrature sum: A_e[o] = sum_{q,f} G_e[q][f] T[q*KQ+f][o] with
// G_e[q] = w_q g(x_q), g = |det J| (1, (K K^T)_ab), KQ = 1 (mass) or 7 (Helmholtz), or
// g = |det J| (eps (K K^T)_ab, (K b)_a), KQ = 9 (advection-diffusion with degree-1 prism fields
// eps, b given at the six vertices). The contraction over K = Q*KQ (189 at P1, 875 at P3)
// accumulates hundreds of MMAs into one FP32 accumulator, and every addition into it is
// rounded relative to the running sum. So the sum is split about the cell's factors at the
// centre of the reference prism, g_c = g(1/3, 1/3, 1/2):
//   A_e = sum_{q,f} w_q (g_f(x_q) - g_c,f) T[q*KQ+f] + sum_f g_c,f Tbar[f],  Tbar[f] = sum_q w_q T[q*KQ+f],
// the per-point chunks first (deviations only: the running sum stays small; zero for an affine
// cell) and the centre chunk (KQ columns against the weight-summed tensors) last. Both
// operands are streamed through shared memory in K-chunks of 64 bytes per row (16 tf32 / 32
// bf16 columns):
//   loader warp 13      one bulk copy per chunk of T^T (all 128-output slices, all parts),
//                       completion counted on the stage's mbarrier (transaction bytes);
//   producer warps 4-11 two threads per cell, each forming half of the chunk's columns of G_e
//                       (geometry per point in FP32, J from per-cell bilinear coefficients),
//                       split into the B operand;
//   MMA warp 12         per chunk and slice, tcgen05.mma accumulating in TMEM (D[o][cell]);
//   epilogue warps 0-3  one 128-output slice at a time: TMEM -> 128-byte warp stores.
// Every wait is bounded; on expiry the kernel sets the error word and unwinds.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstring>
#include <cmath>
#include "coffee_internal.h"
#include "tc_common.cuh"

namespace coffee {
namespace {
using namespace tc;

constexpr int PCB = 64;          // bytes per operand row in one K-chunk (two MMA K-steps)
constexpr int PROD0 = 4;         // producer warps 4..11
constexpr int NPROD = 256;       // producer threads: two per cell
constexpr int LOADER = 13;       // loader warp
constexpr int PTHREADS = 14 * 32;
constexpr int PMAX_STAGES = 6;
constexpr int PSG = 3;           // slices per group (accumulators live together in TMEM)

struct alignas(8) PBars {
  uint64_t full[PMAX_STAGES];
  uint64_t empty[PMAX_STAGES];
  uint64_t tfull[RING];
  uint64_t tempty[RING];
  uint64_t done;
  uint32_t tmem_base;
};
static_assert(sizeof(PBars) <= 256, "the point table follows the barriers at +256 bytes");

__device__ __forceinline__ void prism_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void prism_bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Factors of one quadrature point pq = (s, t, z, w) of a prism (see the kernel comment): J from
// the per-cell bilinear coefficients (d/ds = A + z B, d/dt = C + z D, d/dz = E + s F + t G), and
// for advection-diffusion eps and b from the six vertex values CF. Every factor is linear in w.
template <int KQ>
__device__ __forceinline__ void prism_point_factors(const float4 pq, const float (&JA)[3], const float (&JB)[3],
                                                    const float (&JC)[3], const float (&JD)[3], const float (&JE)[3],
                                                    const float (&JF)[3], const float (&JG)[3],
                                                    const float (&CF)[6][4], float (&gf)[9]) {
  float J[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    J[r][0] = fmaf(pq.z, JB[r], JA[r]);
    J[r][1] = fmaf(pq.z, JD[r], JC[r]);
    J[r][2] = fmaf(pq.x, JF[r], fmaf(pq.y, JG[r], JE[r]));
  }
  const float adj[3][3] = {{J[1][1] * J[2][2] - J[1][2] * J[2][1], J[0][2] * J[2][1] - J[0][1] * J[2][2],
                            J[0][1] * J[1][2] - J[0][2] * J[1][1]},
                           {J[1][2] * J[2][0] - J[1][0] * J[2][2], J[0][0] * J[2][2] - J[0][2] * J[2][0],
                            J[0][2] * J[1][0] - J[0][0] * J[1][2]},
                           {J[1][0] * J[2][1] - J[1][1] * J[2][0], J[0][1] * J[2][0] - J[0][0] * J[2][1],
                            J[0][0] * J[1][1] - J[0][1] * J[1][0]}};
  const float det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
  const float adet = fabsf(det);
  float wi = pq.w / adet;
  constexpr int P0 = KQ == 9 ? 0 : 1;  // first pair factor
  if constexpr (KQ == 9) {
    // eps and b at the point from the vertex values (degree-1 prism functions)
    const float lam[3] = {1.f - pq.x - pq.y, pq.x, pq.y};
    float eps = 0.f, bq[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int v = 0; v < 6; ++v) {
      const float Nv = v < 3 ? lam[v] * (1.f - pq.z) : lam[v - 3] * pq.z;
      eps = fmaf(Nv, CF[v][0], eps);
#pragma unroll
      for (int r = 0; r < 3; ++r) bq[r] = fmaf(Nv, CF[v][1 + r], bq[r]);
    }
    const float sw = det < 0.f ? -pq.w : pq.w;
#pragma unroll
    for (int a = 0; a < 3; ++a) gf[6 + a] = sw * (adj[a][0] * bq[0] + adj[a][1] * bq[1] + adj[a][2] * bq[2]);
    wi *= eps;
  } else {
    gf[0] = pq.w * adet;
  }
  if constexpr (KQ > 1) {
#pragma unroll
    for (int a = 0, pp = P0; a < 3; ++a)
#pragma unroll
      for (int b = a; b < 3; ++b, ++pp) {
        float acc = 0.f;
#pragma unroll
        for (int r = 0; r < 3; ++r) acc = fmaf(adj[a][r], adj[b][r], acc);
        gf[pp] = wi * acc;
      }
  }
}

// p.N outputs, p.mtiles slices, p.nkc chunks, p.ksteps_off = KQ, p.ns = Q; the image holds the
// chunks of T^T ([chunk][slice][part][128 rows x 64 B]) followed by the points (s,t,z,w) [Q][4].
// A tile's slices are contracted in groups of at most PSG (their accumulators share the 512
// TMEM columns): a tile with more slices (P3: 13) runs the chunk loop once per group, the
// producers forming the factors again from the tile's geometry (computed once per tile) and
// the loader bringing only the group's slices of each chunk (contiguous in the image).
template <int PREC, int KQ, bool CSR>
__global__ void __launch_bounds__(PTHREADS, 1) k_assemble_prism_tc(const TcParams p, int nstages) {
  using PT = PrecTraits<PREC>;
  constexpr int TPARTS = PT::TPARTS, GPARTS = PT::GPARTS;
  using PS = Passes<PREC>;
  constexpr int KC = PT::tf32 ? 16 : 32;  // K columns per chunk
  constexpr int TB = BM * PCB;            // bytes of one 128-row part of one chunk
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int MT = p.mtiles, NKC = p.nkc, Q = p.ns, N = p.N;
  const int SG = MT < PSG ? MT : PSG, NG = (MT + SG - 1) / SG;  // slices per group, groups
  const int a_full = MT * TPARTS * TB;            // T^T chunk in the image (all slices)
  const int a_chunk = SG * TPARTS * TB;           // T^T part of a stage (one group)
  const int stage_bytes = a_chunk + GPARTS * TB;  // + the G parts
  PBars* bars = reinterpret_cast<PBars*>(smem + nstages * stage_bytes);
  float4* qsm = reinterpret_cast<float4*>(reinterpret_cast<uint8_t*>(bars) + 256);  // points (s,t,z,w) [Q]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (p.ncells + BN - 1) / BN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < nstages; ++s) {
      mbar_init(smem_u32(&bars->full[s]), NPROD + 1);  // producers + the loader's arrival
      mbar_init(smem_u32(&bars->empty[s]), 1);
    }
    for (int r = 0; r < RING; ++r) {
      mbar_init(smem_u32(&bars->tfull[r]), 1);
      mbar_init(smem_u32(&bars->tempty[r]), EPI_WARPS);
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
    const float4* qg = reinterpret_cast<const float4*>(p.image + (size_t)NKC * a_full);
    for (int i = threadIdx.x; i < Q; i += PTHREADS) qsm[i] = __ldg(qg + i);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;

  if (warp >= PROD0 && warp < MMA_WARP) {
    // ---------------- producers: the G columns of every chunk, two threads per cell ----------------
    const int pt_id = threadIdx.x - PROD0 * 32;
    const int row = pt_id & (BN - 1), half = pt_id >> 7;  // cell of the tile, half of the chunk
    uint32_t c = 0;  // chunk counter (all items)
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const int64_t e = t * BN + row;
      bool live = e < p.ncells;
      // J(s,t,z) is bilinear: columns d/ds = A + z B, d/dt = C + z D, d/dz = E + s F + t G with
      // vertex differences taken in FP64 before rounding to FP32
      float JA[3], JB[3], JC[3], JD[3], JE[3], JF[3], JG[3];
      float CF[6][4] = {};  // advection-diffusion: (eps, b) at the six vertices
      if (live) {
        bool bad = false;
        double Xd[6][3];
#pragma unroll
        for (int v = 0; v < 6; ++v) {
          int vid = __ldg(p.c2v + e * 6 + v);
          if (p.validate && (vid < 0 || vid >= p.nverts)) {
            bad = true;
            vid = 0;
          }
#pragma unroll
          for (int r = 0; r < 3; ++r) Xd[v][r] = __ldg(p.coords + (int64_t)vid * 3 + r);
        }
        if constexpr (KQ == 9) {
          int cid[6];
#pragma unroll
          for (int v = 0; v < 6; ++v) {
            cid[v] = __ldg(p.c2d + e * 6 + v);
            if (p.validate && (cid[v] < 0 || cid[v] >= p.ncoefnodes)) {
              bad = true;
              cid[v] = 0;
            }
          }
          coef_rows<6, 4>(p, cid, CF);
        }
        if (bad) {
          if (half == 0) atomicOr(p.err, ERR_INDEX);
          live = false;
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const double b1 = Xd[1][r] - Xd[0][r], b2 = Xd[2][r] - Xd[0][r];  // bottom edges
          const double t1 = Xd[4][r] - Xd[3][r], t2 = Xd[5][r] - Xd[3][r];  // top edges
          const double h0 = Xd[3][r] - Xd[0][r], h1 = Xd[4][r] - Xd[1][r], h2 = Xd[5][r] - Xd[2][r];
          JA[r] = (float)b1;
          JB[r] = (float)(t1 - b1);
          JC[r] = (float)b2;
          JD[r] = (float)(t2 - b2);
          JE[r] = (float)h0;
          JF[r] = (float)(h1 - h0);
          JG[r] = (float)(h2 - h0);
        }
      }
      // the cell's factors at the centre of the reference prism (weight 1): the per-point chunks
      // carry only the deviations w_q (g(x_q) - g(centre)), the last chunk the centre factors
      // against the weight-summed tensors
      float gbar[9] = {};
      if (live) prism_point_factors<KQ>(make_float4(1.f / 3.f, 1.f / 3.f, 0.5f, 1.f), JA, JB, JC, JD, JE, JF, JG, CF, gbar);
      for (int gi = 0; gi < NG && ok; ++gi) {
      int gq = -1;       // point whose factors are cached
      float gf[9] = {};  // the point's factors (see the kernel comment)
      float wq = 0.f;    // and its weight
      for (int kc = 0; kc < NKC; ++kc, ++c) {
        const int s = (int)(c % nstages);
        if (!mbar_wait(smem_u32(&bars->empty[s]), ((c / nstages) & 1u) ^ 1u, p.err)) { ok = false; break; }
        const bool centre = kc == NKC - 1;
        auto factor = [&](int kcol) -> float {
          if (!live) return 0.f;
          if (centre) {
            float v = 0.f;
#pragma unroll
            for (int i = 0; i < KQ; ++i)
              if (kcol == i) v = gbar[i];
            return v;
          }
          const int k = kc * KC + kcol;
          const int q = k / KQ, f = k - (k / KQ) * KQ;
          if (q >= Q) return 0.f;
          if (q != gq) {
            gq = q;
            const float4 pq = qsm[q];  // (s, t, z, w)
            wq = pq.w;
            prism_point_factors<KQ>(pq, JA, JB, JC, JD, JE, JF, JG, CF, gf);
          }
          float v = gf[0], r = gbar[0];
#pragma unroll
          for (int i = 1; i < KQ; ++i)
            if (f == i) {
              v = gf[i];
              r = gbar[i];
            }
          return fmaf(-wq, r, v);
        };
        uint8_t* b = smem + (size_t)s * stage_bytes + a_chunk;  // G parts of the stage
        // this thread's half of the chunk: 32 bytes of the row (two 16-byte units per part)
        constexpr int PER = PT::tf32 ? 4 : 8;  // columns per 16-byte unit
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const int c16 = half * 2 + cc;  // 16-byte unit of the 64-byte row
          float x[PER];
#pragma unroll
          for (int qq = 0; qq < PER; ++qq) x[qq] = factor(c16 * PER + qq);
          store_unit<PT::tf32, GPARTS>(b + canon_off(row, c16 * 16, PCB), TB, x);
        }
        fence_proxy_async();
        mbar_arrive(smem_u32(&bars->full[s]));
      }
      }
    }
  } else if (warp == LOADER) {
    if (lane == 0) {
      // ---------------- loader: one bulk copy of T^T per chunk ----------------
      uint32_t c = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x)
      for (int gi = 0; gi < NG && ok; ++gi) {
        const int m0 = gi * SG, mt = MT - m0 < SG ? MT - m0 : SG;  // the group's slices
        const uint32_t bytes = (uint32_t)(mt * TPARTS * TB);
        for (int kc = 0; kc < NKC; ++kc, ++c) {
          const int s = (int)(c % nstages);
          if (!mbar_wait(smem_u32(&bars->empty[s]), ((c / nstages) & 1u) ^ 1u, p.err)) { ok = false; break; }
          const uint32_t bar = smem_u32(&bars->full[s]);
          prism_expect_tx(bar, bytes);
          prism_bulk_g2s(smem_u32(smem + (size_t)s * stage_bytes),
                         p.image + (size_t)kc * a_full + (size_t)m0 * TPARTS * TB, bytes, bar);
        }
      }
      // every issued copy is consumed by the MMA thread's wait on its stage (or the kernel timed out)
    }
    __syncwarp();
  } else if (warp == MMA_WARP) {
    // ---------------- MMA issuer: D[o][cell] += T^T[o][k] G[cell][k], chunk by chunk ----------------
    if (lane == 0) {
      const uint32_t sbo = 8u * PCB;
      const uint32_t idesc = make_idesc(PT::tf32 ? 2 : 1, BM, BN);
      const uint32_t s0 = smem_u32(smem);
      uint32_t c = 0, rc = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x)
      for (int gi = 0; gi < NG && ok; ++gi) {
        const int m0 = gi * SG, mt = MT - m0 < SG ? MT - m0 : SG;
        for (int m = 0; m < mt && ok; ++m) {
          const uint32_t r = rc + m;
          if (!mbar_wait(smem_u32(&bars->tempty[r % RING]), ((r / RING) & 1u) ^ 1u, p.err)) ok = false;
        }
        if (!ok) break;
        tc_fence_after();
        for (int kc = 0; kc < NKC; ++kc, ++c) {
          const int s = (int)(c % nstages);
          if (!mbar_wait(smem_u32(&bars->full[s]), (c / nstages) & 1u, p.err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t st = s0 + (uint32_t)(s * stage_bytes);
          const uint32_t g = st + (uint32_t)a_chunk;
          for (int m = 0; m < mt; ++m) {
            const uint32_t d = tmem + ((rc + m) % RING) * BN;
            const uint32_t a = st + (uint32_t)(m * TPARTS * TB);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              const uint32_t ko = (uint32_t)ks * 256u;
              uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
#pragma unroll
              for (int i = 0; i < PS::N; ++i) {  // products of parts, smallest first
                mma<PT::tf32>(d, make_desc(a + (uint32_t)(PS::t(i) * TB) + ko, sbo),
                              make_desc(g + (uint32_t)(PS::g(i) * TB) + ko, sbo), idesc, acc);
                acc = 1;
              }
            }
          }
          tc_commit(smem_u32(&bars->empty[s]));
        }
        if (!ok) break;
        for (int m = 0; m < mt; ++m) tc_commit(smem_u32(&bars->tfull[(rc + m) % RING]));
        rc += mt;
      }
      tc_commit(smem_u32(&bars->done));
      mbar_wait(smem_u32(&bars->done), 0, p.err);
    }
    __syncwarp();
  } else if (warp < EPI_WARPS) {
    // ---------------- epilogue: 128-byte warp stores of 32 outputs of one cell ----------------
    // (global assembly, p.map set: one reduction per entry at its CSR position instead)
    const int q = warp;
    uint32_t rc = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x)
    for (int gi = 0; gi < NG && ok; ++gi) {
      const int m0 = gi * SG, mt = MT - m0 < SG ? MT - m0 : SG;
      for (int mm = 0; mm < mt; ++mm, ++rc) {
        const int m = m0 + mm;  // slice of the element matrix
        const uint32_t slot = rc % RING;
        if (!mbar_wait(smem_u32(&bars->tfull[slot]), (rc / RING) & 1u, p.err)) { ok = false; break; }
        tc_fence_after();
        const int o = m * BM + q * 32 + lane;
        for (int cc = 0; cc < BN; cc += 64) {
          const int64_t cbase = t * BN + cc;
          const int64_t rem = p.ncells - cbase;
          const int ncol = rem <= 0 ? 0 : (rem < 64 ? (int)rem : 64);
          if (m * BM + q * 32 < N && ncol > 0) {  // warp-uniform
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + slot * BN + cc;
            if constexpr (CSR) {
              // global assembly, 32 cells per TMEM wait: a warp reads each cell's 32 map entries
              // (contiguous in the blocked layout) and adds the values at their CSR positions
              const int npad = (N + 3) & ~3;
              const int bw = npad - (o & ~31) < 32 ? npad - (o & ~31) : 32;  // width of this 32-output block
              for (int h = 0; h < 2; ++h) {
                uint32_t v[32], pos[32];
                tmem_ld32(taddr + 32 * h, v);
                // cells cbase + 32h + jj (cbase is a multiple of 32): csr_map_index = row + jj * bw
                const uint32_t* row = p.map + csr_map_index(cbase + 32 * h, o, npad);
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) pos[jj] = (o < N && h * 32 + jj < ncol) ? __ldg(row + jj * bw) : 0u;
                tmem_wait_ld();
                if (o < N) {
#pragma unroll
                  for (int jj = 0; jj < 32; ++jj)
                    if (h * 32 + jj < ncol) {
                      if (pos[jj] < (uint64_t)p.nnz) atomicAdd(p.out + pos[jj], __uint_as_float(v[jj]));
                      else atomicOr(p.err, ERR_INDEX);
                    }
                }
              }
              continue;
            }
            uint32_t v0[32], v1[32];
            tmem_ld32(taddr, v0);
            tmem_ld32(taddr + 32, v1);
            tmem_wait_ld();
            if (o < N) {
              float* dst = p.out + cbase * N + o;
#pragma unroll
              for (int jj = 0; jj < 32; ++jj)
                if (jj < ncol) __stcs(dst + (int64_t)jj * N, __uint_as_float(v0[jj]));
#pragma unroll
              for (int jj = 0; jj < 32; ++jj)
                if (32 + jj < ncol) __stcs(dst + (int64_t)(32 + jj) * N, __uint_as_float(v1[jj]));
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

struct PGeom {
  int n, N, mtiles, KQ, Q, K, nkc, tparts, gparts, kc, elem;
  int a_chunk;  // bytes of one chunk of T^T in the image (all slices)
  int stage;    // bytes of one shared-memory stage (one slice group of T^T + the G part)
};

bool pgeom(int form, int degree, int prec, PGeom& g) {
  if (!(form == FORM_MASS || form == FORM_HELMHOLTZ || form == FORM_ADVDIFF) || degree < 1 || degree > 4) return false;
  if (prec == PREC_FP64 || prec < 0 || prec > PREC_BF16X3) return false;
  const bool tf32 = prec == PREC_TF32 || prec == PREC_TF32X3;
  g.n = prism_nnodes(degree);
  g.N = g.n * g.n;
  g.mtiles = (g.N + BM - 1) / BM;
  g.KQ = form == FORM_HELMHOLTZ ? 7 : form == FORM_ADVDIFF ? 9 : 1;
  g.Q = (degree + 2) * (degree + 2) * (degree + 2);
  g.K = g.Q * g.KQ;
  g.elem = tf32 ? 4 : 2;
  g.kc = PCB / g.elem;
  g.nkc = (g.K + g.kc - 1) / g.kc + 1;  // the per-point chunks and the centre chunk
  g.tparts = prec_tparts(prec);
  g.gparts = prec_gparts(prec);
  g.a_chunk = g.mtiles * g.tparts * BM * PCB;
  const int sg = g.mtiles < PSG ? g.mtiles : PSG;
  g.stage = (sg * g.tparts + g.gparts) * BM * PCB;
  return true;
}

constexpr int P_SMEM_LIMIT = 227 * 1024;

int pstages(const PGeom& g) {
  const int fixed = 256 + g.Q * 16 + 1024 + 64;  // barriers (256 B), point table
  int s = PMAX_STAGES;
  while (s >= 2 && fixed + s * g.stage > P_SMEM_LIMIT) --s;
  return s >= 2 ? s : 0;
}

template <int PREC, int KQ>
cudaError_t launch_p(const TcParams& p, int num_sms, cudaStream_t s, int nst, int smem) {
  auto kern = p.map ? k_assemble_prism_tc<PREC, KQ, true> : k_assemble_prism_tc<PREC, KQ, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (p.ncells + BN - 1) / BN;
  const int grid = (int)(ntiles < num_sms ? ntiles : num_sms);
  kern<<<grid, PTHREADS, smem, s>>>(p, nst);
  return cudaGetLastError();
}

template <int KQ>
cudaError_t launch_prec(const TcParams& q, int num_sms, cudaStream_t s, int nst, int smem) {
  switch (q.precision) {
    case PREC_TF32: return launch_p<PREC_TF32, KQ>(q, num_sms, s, nst, smem);
    case PREC_TF32X3: return launch_p<PREC_TF32X3, KQ>(q, num_sms, s, nst, smem);
    case PREC_BF16: return launch_p<PREC_BF16, KQ>(q, num_sms, s, nst, smem);
    case PREC_BF16X3: return launch_p<PREC_BF16X3, KQ>(q, num_sms, s, nst, smem);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_kq(int KQ, const TcParams& q, int num_sms, cudaStream_t s, int nst, int smem) {
  switch (KQ) {
    case 1: return launch_prec<1>(q, num_sms, s, nst, smem);
    case 7: return launch_prec<7>(q, num_sms, s, nst, smem);
    case 9: return launch_prec<9>(q, num_sms, s, nst, smem);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

int prism_tc_supported(int form, int degree, int precision) {
  PGeom g;
  return pgeom(form, degree, precision, g) && pstages(g) > 0 ? 1 : 0;
}

// T^T chunks [chunk][slice][part][128 rows x 64 B canonical], then the points (s,t,z,w) [Q].
// The last chunk holds the weight-summed tensors sum_q w_q T[q*KQ+f] in its first KQ columns.
void build_prism_tc_image(int form, int degree, int prec, std::vector<uint8_t>& img, TcTable& meta) {
  PGeom g{};
  pgeom(form, degree, prec, g);
  std::vector<double> T, pts, wts;
  prism_tensor(form, degree, T, pts, wts);
  std::vector<double> Tbar((size_t)g.KQ * g.N, 0.0);
  for (int q = 0; q < g.Q; ++q)
    for (int f = 0; f < g.KQ; ++f)
      for (int o = 0; o < g.N; ++o) Tbar[(size_t)f * g.N + o] += wts[q] * T[((size_t)q * g.KQ + f) * g.N + o];
  const bool tf32 = g.elem == 4;
  const size_t tb = (size_t)BM * PCB;
  img.assign((size_t)g.nkc * g.a_chunk + (size_t)g.Q * 16, 0);
  for (int kc = 0; kc < g.nkc; ++kc)
    for (int m = 0; m < g.mtiles; ++m)
      for (int r = 0; r < BM; ++r) {
        const int o = m * BM + r;
        for (int j = 0; j < g.kc; ++j) {
          const int k = kc * g.kc + j;
          double x = 0.0;
          if (o < g.N) {
            if (kc == g.nkc - 1) x = j < g.KQ ? Tbar[(size_t)j * g.N + o] : 0.0;
            else if (k < g.K) x = T[(size_t)k * g.N + o];
          }
          host_store_parts(img.data() + (size_t)kc * g.a_chunk + (size_t)(m * g.tparts) * tb, tb,
                           canon_off(r, j * g.elem, PCB), x, tf32, g.tparts);
        }
      }
  float* qp = reinterpret_cast<float*>(img.data() + (size_t)g.nkc * g.a_chunk);
  for (int q = 0; q < g.Q; ++q) {
    qp[q * 4 + 0] = (float)pts[(size_t)q * 3 + 0];
    qp[q * 4 + 1] = (float)pts[(size_t)q * 3 + 1];
    qp[q * 4 + 2] = (float)pts[(size_t)q * 3 + 2];
    qp[q * 4 + 3] = (float)wts[q];
  }
  meta = TcTable{};
  meta.mtiles = g.mtiles;
  meta.kbytes = PCB;
  meta.kelems = g.nkc * g.kc;
  meta.K = g.K;
  meta.tparts = g.tparts;
  meta.ksteps_off = g.KQ;
  meta.tile_bytes = (int64_t)tb;
}

int launch_prism_tc(int form, int degree, const TcParams& p, int num_sms, void* stream, std::string& why) {
  if (p.ncells == 0) return (int)cudaSuccess;
  PGeom g;
  if (!pgeom(form, degree, p.precision, g)) {
    why = "no tensor-core prism kernel for this form/degree";
    return (int)cudaErrorInvalidValue;
  }
  const int nst = pstages(g);
  if (nst == 0) {
    why = "operands do not fit in shared memory";
    return (int)cudaErrorInvalidValue;
  }
  TcParams q = p;
  q.mtiles = g.mtiles;
  q.nkc = g.nkc;
  q.ksteps_off = g.KQ;
  q.ns = g.Q;
  q.N = g.N;
  int smem = nst * g.stage + 256 + g.Q * 16 + 1024 + 64;
  if (smem < 120 * 1024) smem = 120 * 1024;  // one CTA (one TMEM owner) per SM
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return (int)launch_kq(g.KQ, q, num_sms, s, nst, smem);
}

}  // namespace coffee
