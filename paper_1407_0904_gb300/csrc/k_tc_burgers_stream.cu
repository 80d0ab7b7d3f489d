// tcgen05 Burgers Jacobian for shapes whose operands do not fit in shared memory: tetrahedra
// P3-P4 (block matrices of 400 and 1225 entries, K up to 224) and triangles P4 in the split
// precisions. Same contraction as k_tc_burgers.cu,
//   block(ci,cj) = sum_{r,a} u[r][ci] P[a][cj] T1[r,a] + [ci==cj] (sum_{r,a} Q[r][a] T2[r,a] + nu sum_p H_p T3[p]),
// with both operands streamed through shared memory in K-chunks of 64 bytes per row (16 tf32 /
// 32 bf16 columns), as for prisms:
//   loader warp 13      one bulk copy per chunk of [T1 | T2 | T3]^T for one 128-row slice of the
//                       block entries (all its parts), counted on the stage's mbarrier;
//   producer warps 4-11 two threads per cell (adjacent lanes, so they share their cell's u through
//                       shared memory with a warp barrier): the chunk's columns of the factors of
//                       the d blocks of a block row, split into the precision's parts;
//   MMA warp 12         per chunk, one MMA group per block of the row that uses the chunk (the
//                       off-diagonal blocks contract the T1 chunks only): the chunk of T^T is
//                       loaded once for the d blocks;
//   epilogue warps 0-3  the d accumulators of a (block row, slice): 128-byte warp stores.
// Work order per 128-cell tile: block row ci, slice m, K-chunk. The factors do not depend on the
// slice, so they are formed again per slice (MT times); u is gathered once per tile.
// Every wait is bounded; on expiry the kernel sets the error word and unwinds.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstring>
#include <cmath>
#include "coffee_internal.h"
#include "tc_common.cuh"
#include "k_tc_burgers.cuh"

namespace coffee {
namespace {
using namespace tc;

constexpr int SCB = 64;            // bytes per operand row in one K-chunk (two MMA K-steps)
constexpr int S_PROD0 = 4;         // producer warps 4..11
constexpr int S_NPROD = 256;       // producer threads: two per cell
constexpr int S_LOADER = 13;
constexpr int S_THREADS = 14 * 32;
constexpr int S_MAX_STAGES = 4;
constexpr int S_TB = BM * SCB;     // one 128-row part of one chunk: 8 KB

struct alignas(8) SBars {
  uint64_t full[S_MAX_STAGES];
  uint64_t empty[S_MAX_STAGES];
  uint64_t tfull[RING];
  uint64_t tempty[RING];
  uint64_t done;
  uint32_t tmem_base;
};
static_assert(sizeof(SBars) <= 256, "u follows the barriers at +256 bytes");

__device__ __forceinline__ void s_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void s_bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

template <int D, int NS, int PREC>
struct SShape {
  using PT = PrecTraits<PREC>;
  static constexpr int CK = PT::tf32 ? 16 : 32;       // K columns per chunk
  static constexpr int P = D * (D + 1) / 2;
  static constexpr int K1 = NS * D;                    // columns of T1 (and of T2)
  static constexpr int KA1 = round_up(K1, CK);         // off-diagonal K: the T1 chunks
  static constexpr int KD = round_up(KA1 + K1 + P, CK);
  static constexpr int NCA = KA1 / CK, NCD = KD / CK;  // chunks of off-diagonal / diagonal blocks
  static constexpr int NBLK = NS * NS;
  static constexpr int MT = (NBLK + BM - 1) / BM;      // 128-entry slices of a block
  static constexpr int ASTAGE = PT::TPARTS * S_TB;     // one chunk of T^T (one slice, all parts)
  static constexpr int GSTAGE = PT::GPARTS * S_TB;     // one chunk of one block's factors
  static constexpr int STAGE = ASTAGE + D * GSTAGE;
};

template <int D, int NS, int PREC>
__global__ void __launch_bounds__(S_THREADS, 1) k_burgers_stream_tc(const TcParams p, int nstages) {
  using S = SShape<D, NS, PREC>;
  using PT = PrecTraits<PREC>;
  using PS = Passes<PREC>;
  constexpr int NV = D + 1, P = S::P, CK = S::CK, K1 = S::K1, KA1 = S::KA1, MT = S::MT;
  constexpr int NCA = S::NCA, NCD = S::NCD;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  SBars* bars = reinterpret_cast<SBars*>(smem + nstages * S::STAGE);
  float* us = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(bars) + 256);  // [cell][NS*D]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (p.ncells + BN - 1) / BN;
  const int ndof = D * NS;

  if (threadIdx.x == 0) {
    for (int s = 0; s < nstages; ++s) {
      mbar_init(smem_u32(&bars->full[s]), S_NPROD + 1);  // producers + the loader's arrival
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
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;

  if (warp >= S_PROD0 && warp < MMA_WARP) {
    // ---------------- producers: two adjacent lanes per cell ----------------
    const int pt = threadIdx.x - S_PROD0 * 32;
    const int row = pt >> 1, half = pt & 1;  // cell of the tile, half of each chunk
    float* ucell = us + row * (NS * D);
    uint32_t c = 0;  // chunk counter
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const int64_t e = t * BN + row;
      bool live = e < p.ncells;
      float Pm[D][D], H[P];
      if (live) {
        int vid[NV];
        bool bad = false;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          vid[v] = __ldg(p.c2v + e * NV + v);
          if (p.validate && (vid[v] < 0 || vid[v] >= p.nverts)) bad = true;
        }
        // u of the cell: this thread gathers nodes r = half, half + 2, ..
        constexpr int NH = (NS + 1) / 2;
        int did[NH];
        bool okr[NH];
#pragma unroll
        for (int j = 0; j < NH; ++j) {
          const int r = half + 2 * j;
          did[j] = r < NS ? __ldg(p.c2d + e * NS + r) : 0;
          okr[j] = r < NS;
          if (okr[j] && p.validate && (did[j] < 0 || did[j] >= p.ncoefnodes)) {
            bad = true;
            okr[j] = false;
          }
        }
        float uh[NH][D];
        coef_rows<NH, D>(p, did, uh, okr);
#pragma unroll
        for (int j = 0; j < NH; ++j)
          if (okr[j]) {
#pragma unroll
            for (int cc = 0; cc < D; ++cc) ucell[(half + 2 * j) * D + cc] = uh[j][cc];
          }
        if (bad) {
          atomicOr(p.err, ERR_INDEX);
          live = false;
        } else {
          float adj[D][D], Dm, sg;
          cell_geometry_ids<D>(p, vid, adj, Dm, sg);
          const float inv = 1.0f / Dm;
#pragma unroll
          for (int a = 0; a < D; ++a)
#pragma unroll
            for (int cc = 0; cc < D; ++cc) Pm[a][cc] = sg * adj[a][cc];
          int q = 0;
#pragma unroll
          for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = a; b < D; ++b) {
              float s = 0.f;
#pragma unroll
              for (int r = 0; r < D; ++r) s = fmaf(adj[a][r], adj[b][r], s);
              H[q++] = (float)p.nu * s * inv;
            }
        }
      }
      // the pair's validity and u: both lanes of a cell agree before any factor is formed
      {
        const int l0 = __shfl_sync(0xffffffffu, live ? 1 : 0, lane & ~1);
        const int l1 = __shfl_sync(0xffffffffu, live ? 1 : 0, lane | 1);
        live = l0 != 0 && l1 != 0;
      }
      __syncwarp();
      for (int ci = 0; ci < D && ok; ++ci)
        for (int m = 0; m < MT && ok; ++m)
          for (int kc = 0; kc < NCD; ++kc, ++c) {
            const int s = (int)(c % nstages);
            if (!mbar_wait(smem_u32(&bars->empty[s]), ((c / nstages) & 1u) ^ 1u, p.err)) { ok = false; break; }
            uint8_t* gbase = smem + (size_t)s * S::STAGE + S::ASTAGE;
            static_for<D>([&](auto CJ) -> bool {
              constexpr int cj = decltype(CJ)::value;
              if (cj != ci && kc >= NCA) return true;  // off-diagonal blocks: T1 chunks only
              const bool diag = cj == ci;
              // factor of column k of block (ci, cj): see the file comment
              auto factor = [&](int k) -> float {
                if (!live) return 0.f;
                if (k < K1) {
                  const int r = k / D, a = k - (k / D) * D;
                  float pa = Pm[0][cj];
#pragma unroll
                  for (int x = 1; x < D; ++x)
                    if (a == x) pa = Pm[x][cj];
                  return ucell[r * D + ci] * pa;
                }
                if (!diag || k < KA1) return 0.f;
                if (k < KA1 + K1) {
                  const int r = (k - KA1) / D, a = (k - KA1) - ((k - KA1) / D) * D;
                  float q = 0.f;
#pragma unroll
                  for (int cc = 0; cc < D; ++cc) {
                    float pa = Pm[0][cc];
#pragma unroll
                    for (int x = 1; x < D; ++x)
                      if (a == x) pa = Pm[x][cc];
                    q = fmaf(ucell[r * D + cc], pa, q);
                  }
                  return q;
                }
                if (k < KA1 + K1 + P) {
                  const int pp = k - KA1 - K1;
                  float h = H[0];
#pragma unroll
                  for (int x = 1; x < P; ++x)
                    if (pp == x) h = H[x];
                  return h;
                }
                return 0.f;
              };
              // this thread's half of the chunk: two 16-byte units of the 64-byte row per part
              constexpr int PER = PT::tf32 ? 4 : 8;
              uint8_t* g = gbase + (size_t)cj * S::GSTAGE;
#pragma unroll
              for (int cu = 0; cu < 2; ++cu) {
                const int c16 = half * 2 + cu;
                float x[PER];
#pragma unroll
                for (int l = 0; l < PER; ++l) x[l] = factor(kc * CK + c16 * PER + l);
                store_unit<PT::tf32, PT::GPARTS>(g + canon_off(row, c16 * 16, SCB), S_TB, x);
              }
              return true;
            });
            fence_proxy_async();
            mbar_arrive(smem_u32(&bars->full[s]));
          }
      __syncwarp();  // both lanes of every cell are done with u before the next tile overwrites it
    }
  } else if (warp == S_LOADER) {
    if (lane == 0) {
      // ---------------- loader: one bulk copy of T^T per chunk ----------------
      uint32_t c = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x)
        for (int ci = 0; ci < D && ok; ++ci)
          for (int m = 0; m < MT && ok; ++m)
            for (int kc = 0; kc < NCD; ++kc, ++c) {
              const int s = (int)(c % nstages);
              if (!mbar_wait(smem_u32(&bars->empty[s]), ((c / nstages) & 1u) ^ 1u, p.err)) { ok = false; break; }
              const uint32_t bar = smem_u32(&bars->full[s]);
              s_expect_tx(bar, (uint32_t)S::ASTAGE);
              s_bulk_g2s(smem_u32(smem + (size_t)s * S::STAGE), p.image + ((size_t)m * NCD + kc) * S::ASTAGE,
                         (uint32_t)S::ASTAGE, bar);
            }
      // every issued copy is consumed by the MMA thread's wait on its stage (or the kernel timed out)
    }
    __syncwarp();
  } else if (warp == MMA_WARP) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t sbo = 8u * SCB;
      const uint32_t idesc = make_idesc(PT::tf32 ? 2 : 1, BM, BN);
      const uint32_t s0 = smem_u32(smem);
      uint32_t c = 0, rc = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x)
        for (int ci = 0; ci < D && ok; ++ci)
          for (int m = 0; m < MT && ok; ++m, rc += D) {
            for (int cj = 0; cj < D && ok; ++cj) {
              const uint32_t r = rc + cj;
              if (!mbar_wait(smem_u32(&bars->tempty[r % RING]), ((r / RING) & 1u) ^ 1u, p.err)) ok = false;
            }
            if (!ok) break;
            tc_fence_after();
            for (int kc = 0; kc < NCD; ++kc, ++c) {
              const int s = (int)(c % nstages);
              if (!mbar_wait(smem_u32(&bars->full[s]), (c / nstages) & 1u, p.err)) { ok = false; break; }
              tc_fence_after();
              const uint32_t a = s0 + (uint32_t)(s * S::STAGE);
              for (int cj = 0; cj < D; ++cj) {
                if (cj != ci && kc >= NCA) continue;
                const uint32_t d = tmem + ((rc + cj) % RING) * BN;
                const uint32_t g = a + (uint32_t)(S::ASTAGE + cj * S::GSTAGE);
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                  const uint32_t ko = (uint32_t)ks * 256u;
#pragma unroll
                  for (int i = 0; i < PS::N; ++i) {  // products of parts, smallest first
                    const uint32_t acc = (kc > 0 || ks > 0 || i > 0) ? 1u : 0u;
                    mma<PT::tf32>(d, make_desc(a + (uint32_t)(PS::t(i) * S_TB) + ko, sbo),
                                  make_desc(g + (uint32_t)(PS::g(i) * S_TB) + ko, sbo), idesc, acc);
                  }
                }
              }
              tc_commit(smem_u32(&bars->empty[s]));
            }
            if (!ok) break;
            for (int cj = 0; cj < D; ++cj) tc_commit(smem_u32(&bars->tfull[(rc + cj) % RING]));
          }
      tc_commit(smem_u32(&bars->done));
      mbar_wait(smem_u32(&bars->done), 0, p.err);
    }
    __syncwarp();
  } else if (warp < EPI_WARPS) {
    // ---------------- epilogue: the d accumulators of a (block row, slice) ----------------
    const int q = warp;
    uint32_t rc = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x)
      for (int ci = 0; ci < D && ok; ++ci)
        for (int m = 0; m < MT && ok; ++m)
          for (int cj = 0; cj < D; ++cj, ++rc) {
            const uint32_t slot = rc % RING;
            if (!mbar_wait(smem_u32(&bars->tfull[slot]), (rc / RING) & 1u, p.err)) { ok = false; break; }
            tc_fence_after();
            const int o = m * BM + q * 32 + lane;  // entry (i, j) of the block
            for (int hc = 0; hc < 2; ++hc) {
              const int64_t cbase = t * BN + hc * 64;
              const int64_t rem = p.ncells - cbase;
              const int ncol = rem <= 0 ? 0 : (rem < 64 ? (int)rem : 64);
              if (m * BM + q * 32 < S::NBLK && ncol > 0) {  // warp-uniform
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + slot * BN + hc * 64;
                uint32_t v0[32], v1[32];
                tmem_ld32(taddr, v0);
                tmem_ld32(taddr + 32, v1);
                tmem_wait_ld();
                if (o < S::NBLK) {
                  const int i = o / NS, j = o - (o / NS) * NS;
                  float* dst = p.out + cbase * p.N + (int64_t)(ci * NS + i) * ndof + cj * NS + j;
#pragma unroll
                  for (int jj = 0; jj < 32; ++jj, dst += p.N)
                    if (jj < ncol) __stcs(dst, __uint_as_float(v0[jj]));
#pragma unroll
                  for (int jj = 0; jj < 32; ++jj, dst += p.N)
                    if (32 + jj < ncol) __stcs(dst, __uint_as_float(v1[jj]));
                }
              }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bars->tempty[slot]));
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

constexpr int S_SMEM_LIMIT = 227 * 1024;

struct SGeom {
  int d, ns, ck, elem, K1, KA1, KD, nca, ncd, mtiles, astage, gstage, stage, ubytes;
};

bool sgeom(int degree, int cell, int prec, SGeom& g) {
  if (prec == PREC_FP64 || prec < PREC_TF32 || prec > PREC_BF16X3) return false;
  if (cell != CELL_TRI && cell != CELL_TET) return false;
  // compiled instances: triangles P4, tetrahedra P3-P4
  if (cell == CELL_TRI ? degree != 4 : (degree < 3 || degree > 4)) return false;
  const bool tf32 = prec == PREC_TF32 || prec == PREC_TF32X3;
  g.d = cell == CELL_TRI ? 2 : 3;
  const int P = g.d * (g.d + 1) / 2;
  g.ns = nnodes(cell, degree);
  g.ck = tf32 ? 16 : 32;
  g.elem = tf32 ? 4 : 2;
  g.K1 = g.ns * g.d;
  g.KA1 = round_up(g.K1, g.ck);
  g.KD = round_up(g.KA1 + g.K1 + P, g.ck);
  g.nca = g.KA1 / g.ck;
  g.ncd = g.KD / g.ck;
  g.mtiles = (g.ns * g.ns + BM - 1) / BM;
  g.astage = prec_tparts(prec) * S_TB;
  g.gstage = prec_gparts(prec) * S_TB;
  g.stage = g.astage + g.d * g.gstage;
  g.ubytes = BN * g.ns * g.d * 4;
  return true;
}

int s_stages(const SGeom& g) {
  const int fixed = 256 + g.ubytes + 1024 + 64;  // barriers, u, alignment
  int s = S_MAX_STAGES;
  while (s >= 2 && fixed + s * g.stage > S_SMEM_LIMIT) --s;
  return s >= 2 ? s : 0;
}

template <int D, int NS, int PREC>
cudaError_t launch_s(const TcParams& p, int num_sms, cudaStream_t s, int nst, int smem) {
  auto kern = k_burgers_stream_tc<D, NS, PREC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (p.ncells + BN - 1) / BN;
  const int grid = (int)(ntiles < num_sms ? ntiles : num_sms);
  kern<<<grid, S_THREADS, smem, s>>>(p, nst);
  return cudaGetLastError();
}

template <int D, int NS>
cudaError_t launch_sp(const TcParams& p, int num_sms, cudaStream_t s, int nst, int smem) {
  switch (p.precision) {
    case PREC_TF32: return launch_s<D, NS, PREC_TF32>(p, num_sms, s, nst, smem);
    case PREC_TF32X3: return launch_s<D, NS, PREC_TF32X3>(p, num_sms, s, nst, smem);
    case PREC_BF16: return launch_s<D, NS, PREC_BF16>(p, num_sms, s, nst, smem);
    case PREC_BF16X3: return launch_s<D, NS, PREC_BF16X3>(p, num_sms, s, nst, smem);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

int burgers_stream_supported(int degree, int cell, int precision) {
  SGeom g;
  return sgeom(degree, cell, precision, g) && s_stages(g) > 0 ? 1 : 0;
}

// T^T chunks [slice][chunk][part][128 rows x 64 B canonical]: column k of a chunk row holds the
// reference-tensor row of K-column kc*CK + k (T1, then T2 after KA1, then T3), zero padding
void build_burgers_stream_image(int degree, int cell, int prec, std::vector<uint8_t>& img, TcTable& meta) {
  SGeom g{};
  sgeom(degree, cell, prec, g);
  std::vector<double> T;
  reference_tensor(FORM_BURGERS, degree, cell, T);
  const int P = g.d * (g.d + 1) / 2, nb = g.ns * g.ns, tparts = prec_tparts(prec);
  const bool tf32 = g.elem == 4;
  auto trow_of = [&](int k) {
    if (k < g.K1) return k;
    if (k >= g.KA1 && k < g.KA1 + g.K1) return g.ns * g.d + (k - g.KA1);
    if (k >= g.KA1 + g.K1 && k < g.KA1 + g.K1 + P) return 2 * g.ns * g.d + (k - g.KA1 - g.K1);
    return -1;
  };
  img.assign((size_t)g.mtiles * g.ncd * g.astage, 0);
  for (int m = 0; m < g.mtiles; ++m)
    for (int kc = 0; kc < g.ncd; ++kc)
      for (int r = 0; r < BM; ++r) {
        const int o = m * BM + r;
        for (int j = 0; j < g.ck; ++j) {
          const int tr = trow_of(kc * g.ck + j);
          const double x = (o < nb && tr >= 0) ? T[(size_t)tr * nb + o] : 0.0;
          host_store_parts(img.data() + ((size_t)m * g.ncd + kc) * g.astage, (size_t)S_TB,
                           canon_off(r, j * g.elem, SCB), x, tf32, tparts);
        }
      }
  meta = TcTable{};
  meta.mtiles = g.mtiles;
  meta.kbytes = SCB;
  meta.kelems = g.KD;
  meta.K = g.KA1 + g.K1 + P;
  meta.tparts = tparts;
  meta.ksteps_off = g.nca;  // chunks of the off-diagonal blocks
  meta.tile_bytes = (int64_t)S_TB;
}

int launch_burgers_stream_tc(int cell, int degree, const TcParams& p, int num_sms, void* stream, std::string& why) {
  if (p.ncells == 0) return (int)cudaSuccess;
  SGeom g{};
  if (!sgeom(degree, cell, p.precision, g)) {
    why = "no streamed Burgers instance for this degree";
    return (int)cudaErrorInvalidValue;
  }
  const int nst = s_stages(g);
  if (nst == 0) {
    why = "operands do not fit in shared memory";
    return (int)cudaErrorInvalidValue;
  }
  int smem = nst * g.stage + 256 + g.ubytes + 1024 + 64;
  if (smem < 120 * 1024) smem = 120 * 1024;  // one CTA (one TMEM owner) per SM
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cell == CELL_TRI) return (int)launch_sp<2, 15>(p, num_sms, s, nst, smem);
  if (degree == 3) return (int)launch_sp<3, 20>(p, num_sms, s, nst, smem);
  return (int)launch_sp<3, 35>(p, num_sms, s, nst, smem);
}

}  // namespace coffee
