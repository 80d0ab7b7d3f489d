// The tcgen05 local-assembly kernel template, shared by the element-matrix launcher
// (k_tc.cu) and the fused global-assembly launcher (k_tc_csr.cu).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include "coffee_internal.h"
#include "tc_common.cuh"

namespace coffee {
namespace {

using namespace tc;

// Global-assembly (CSR) epilogue: each epilogue warp streams the entry-map blocks of its 32
// outputs for one accumulator's cells (up to 128 cells, one 16 KB stage) from global memory into
// shared memory with bulk asynchronous copies, one accumulator ahead of the one it adds. The
// hand-off (an mbarrier with a transaction count) is paid once per accumulator, not per 32 cells.
constexpr int CSR_STAGES = 2;
constexpr int CSR_STAGE_BYTES = BN * 32 * 4;
constexpr int CSR_BAR_BYTES = 128;
constexpr int CSR_SMEM = CSR_BAR_BYTES + EPI_WARPS * CSR_STAGES * CSR_STAGE_BYTES + 128;  // barriers, ring, slack
// Staged epilogue: at most STAGE_BUFS buffers of SCH rows (p.stage_bufs, as many as shared
// memory holds: several bulk copies in flight); the most 128-output slices of one element matrix
constexpr int STAGE_BUFS = 4;
constexpr int STAGE_MAXM = 10;  // P4 tetrahedra: 1225 outputs
template <int SCH>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, uint32_t (&v)[SCH]) {
  static_assert(SCH == 8 || SCH == 32, "staged epilogue: 8 or 32 cells per chunk");
  if constexpr (SCH == 32) {
    tmem_ld32(taddr, v);
  } else {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
  }
}

__device__ __forceinline__ void csr_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void csr_bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// ------------------------------------------------------------------- kernel
// Two orientations of the per-tile contraction.
//  outputs on lanes (any N): D[o][cell] = T^T G^T, one 128-column TMEM accumulator per
//         128-output slice (ring of four); each epilogue warp store writes 32 consecutive
//         outputs of one cell (128 bytes).
//  cells on lanes (N <= 128, LANES): D[cell][o] = G T, M = 128 cells, N = outputs rounded
//         up to 16; an epilogue thread holds consecutive outputs of its own cell and writes
//         its row with 16-byte stores, so every output row is written by one thread in
//         order. The operands are the same shared-memory images with their roles swapped.
// CSR (outputs on lanes only): global assembly. Instead of being stored, every entry is
//         added into the CSR value array p.out at the position p.map[cell][o]; the element
//         matrices never reach memory.
// SCH > 0, staged (outputs on lanes only): the rows of SCH consecutive cells are gathered from
//         all of a sub-tile's accumulators into a shared-memory buffer in the output layout and
//         written with one bulk copy (16-byte aligned: 4 rows of N floats are a multiple of 16
//         bytes). Used where rows do not start on 32-byte sectors (P4 tetrahedra: 4900-byte
//         rows), which direct warp stores split. A TMEM load round trip costs hundreds of
//         cycles, so each wait covers SCH columns of up to STAGE_SG slices (about 40 registers),
//         and the loop is kept compact (rolled over slice groups): unrolling it over every
//         slice was measured to thrash the instruction cache. Two buffers alternate.
template <int FORM, int D, int PREC, bool LANES, bool CSR = false, int SCH = 0>
__global__ void __launch_bounds__(NTHREADS, 1) k_assemble_tc(const TcParams p, int nstages) {
  using PT = PrecTraits<PREC>;
  constexpr int KSTEP = PT::tf32 ? 8 : 16;  // K elements per MMA (32 bytes)
  constexpr int KP = round_up(Form<FORM, D>::K, KSTEP);
  constexpr int TPARTS = PT::TPARTS, GPARTS = PT::GPARTS;
  using PS = Passes<PREC>;

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int kbytes = p.kbytes;
  const int tile_bytes = BM * kbytes;  // one part of one operand tile (A: 128 outputs, B: 128 cells)
  const int a_bytes = p.mtiles * TPARTS * tile_bytes;
  const int N = p.N;
  uint8_t* sA = smem;
  uint8_t* sB = smem + a_bytes;
  Barriers* bars = reinterpret_cast<Barriers*>(sB + nstages * GPARTS * tile_bytes);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (p.ncells + BN - 1) / BN;
  const int NP = (N + 15) & ~15;  // LANES: MMA N (outputs, multiple of 16)

  // ---- set-up: barriers, TMEM, resident A operand ----
  if (threadIdx.x == 0) {
    for (int s = 0; s < nstages; ++s) {
      mbar_init(smem_u32(&bars->full[s]), 128);
      mbar_init(smem_u32(&bars->empty[s]), 1);
    }
    for (int r = 0; r < MAX_SLOTS; ++r) {
      mbar_init(smem_u32(&bars->tfull[r]), 1);
      mbar_init(smem_u32(&bars->tempty[r]), EPI_WARPS);
    }
    mbar_init(smem_u32(&bars->done), 1);
    if constexpr (SCH > 0) mbar_init(smem_u32(&bars->epi), EPI_WARPS);
    if constexpr (CSR) {
      uint64_t* ring = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(bars) + round_up((int)sizeof(Barriers), 128));
      for (int i = 0; i < EPI_WARPS * CSR_STAGES; ++i) mbar_init(smem_u32(ring + i), 1);
    }
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
    // ---------------- producers: one cell per thread, two groups on alternate tiles ----------------
    const int pw = warp - PROD_WARP0;
    const int grp = pw >> 2, row = ((pw & 3) << 5) + lane;
    const int spg = nstages / PROD_GROUPS;
    const int64_t tstep = (int64_t)PROD_GROUPS * gridDim.x;
    int64_t li = 0;
    CellIds<FORM, D> ids{}, nids{};  // this tile's and (prefetched) the next tile's index rows
    {
      const int64_t e0 = (blockIdx.x + (int64_t)grp * gridDim.x) * BN + row;
      if (e0 < p.ncells) load_ids<FORM, D>(p, e0, nids);
    }
    for (int64_t t = blockIdx.x + (int64_t)grp * gridDim.x; t < ntiles; t += tstep, ++li) {
      const int64_t e = t * BN + row;
      ids = nids;
      if (e + tstep * BN < p.ncells) load_ids<FORM, D>(p, e + tstep * BN, nids);
      int s;
      uint32_t use;
      stage_of(li, grp, spg, s, use);
      if (!mbar_wait(smem_u32(&bars->empty[s]), (use & 1u) ^ 1u, p.err)) break;
      float G[KP];
      bool bad = false;
      if (e < p.ncells) {
        cell_factors_ids<FORM, D, KP>(p, ids, G, bad);
        if (bad) atomicOr(p.err, ERR_INDEX);
      }
      if (e >= p.ncells || bad) {
#pragma unroll
        for (int k = 0; k < KP; ++k) G[k] = 0.f;
      }
      store_operand_row<PREC, KP>(sB + (size_t)s * GPARTS * tile_bytes, tile_bytes, row, G, kbytes);
      fence_proxy_async();
      mbar_arrive(smem_u32(&bars->full[s]));
    }
  } else if (warp == MMA_WARP) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const int ksteps = kbytes / 32;
      const uint32_t sbo = 8u * (uint32_t)kbytes;
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      const int W = LANES ? BN : p.subw;       // cells per accumulator
      const int nslot = LANES ? RING : 512 / W;
      const uint32_t idesc = make_idesc(PT::tf32 ? 2 : 1, BM, LANES ? NP : W);
      uint32_t rc = 0;  // accumulator ring counter
      const int spg = nstages / PROD_GROUPS;
      int64_t tl = 0;  // local tile number
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tl) {
        int s;
        uint32_t use;
        stage_of(tl / PROD_GROUPS, (int)(tl % PROD_GROUPS), spg, s, use);
        if (!mbar_wait(smem_u32(&bars->full[s]), use & 1u, p.err)) break;
        tc_fence_after();
        const uint32_t bstage = b0 + (uint32_t)(s * GPARTS * tile_bytes);
        for (int j = 0; j < BN / W && ok; ++j)
        for (int m = 0; m < p.mtiles; ++m, ++rc) {
          const uint32_t slot = rc % nslot, round = rc / nslot;
          if (!mbar_wait(smem_u32(&bars->tempty[slot]), (round & 1u) ^ 1u, p.err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t d = tmem + slot * W;
          const uint32_t atile = a0 + (uint32_t)(m * TPARTS * tile_bytes);
          const uint32_t bsub = bstage + (uint32_t)(j * W * kbytes);  // cells j*W.. of the stage
          uint32_t acc = 0;
          for (int ks = 0; ks < ksteps; ++ks) {
            const uint32_t ko = (uint32_t)ks * 256u;
#pragma unroll
            for (int i = 0; i < PS::N; ++i) {
              // part t of T^T and part g of G; outputs on lanes: A = T^T slice, B = G stage;
              // cells on lanes: A = G, B = T^T
              const uint32_t tt = atile + (uint32_t)(PS::t(i) * tile_bytes) + ko;
              const uint32_t gg = (LANES ? bstage : bsub) + (uint32_t)(PS::g(i) * tile_bytes) + ko;
              mma<PT::tf32>(d, make_desc(LANES ? gg : tt, sbo), make_desc(LANES ? tt : gg, sbo), idesc, acc);
              acc = 1;
            }
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
  } else if constexpr (LANES) {
    // ---------------- epilogue, cells on lanes: each thread writes its cell's row ----------------
    const int q = warp;  // lanes 32q..32q+31 = cells of the tile
    const bool vec = (p.ostride & 3) == 0 && (reinterpret_cast<uintptr_t>(p.out) & 15) == 0;
    uint32_t rc = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++rc) {
      const uint32_t slot = rc % RING, round = rc / RING;
      if (!mbar_wait(smem_u32(&bars->tfull[slot]), round & 1u, p.err)) { ok = false; break; }
      tc_fence_after();
      const int64_t cell = t * BN + q * 32 + lane;
      float* row = p.out + cell * p.ostride;
      if (t * BN + q * 32 < p.ncells) {  // warp-uniform
        for (int c0 = 0; c0 < NP; c0 += 32) {
          uint32_t v[32];
          if (NP - c0 >= 32) {
            tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + slot * BN + c0, v);
          } else {
            tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + slot * BN + c0,
                      *reinterpret_cast<uint32_t(*)[16]>(v));
          }
          tmem_wait_ld();
          if (cell < p.ncells) {
            const int w = (N - c0) < 32 ? N - c0 : 32;
            if (vec) {
#pragma unroll
              for (int k = 0; k < 8; ++k)
                if (4 * k < w)
                  __stcs(reinterpret_cast<float4*>(row + c0 + 4 * k),
                         make_float4(__uint_as_float(v[4 * k]), __uint_as_float(v[4 * k + 1]),
                                     __uint_as_float(v[4 * k + 2]), __uint_as_float(v[4 * k + 3])));
            } else {
#pragma unroll
              for (int k = 0; k < 32; ++k)
                if (k < w) __stcs(row + c0 + k, __uint_as_float(v[k]));
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars->tempty[slot]));
    }
  } else if constexpr (SCH > 0) {
    // ---------------- epilogue, rows staged in shared memory and bulk-copied ----------------
    constexpr int SG = SCH >= 32 ? 1 : 5;  // slices per TMEM wait
    const int q = warp;  // TMEM lane quadrant
    const int W = p.subw, nslot = 512 / W, MT = p.mtiles;
    float* stage0 = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(bars) + round_up((int)sizeof(Barriers), 128));
    uint32_t rc = 0, chunk = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      for (int j = 0; j < BN / W && ok; ++j, rc += MT) {
        // every slice of the sub-tile (MT consecutive slots) before any row is staged
        for (int m = 0; m < MT && ok; ++m)
          if (!mbar_wait(smem_u32(&bars->tfull[(rc + m) % nslot]), ((rc + m) / nslot) & 1u, p.err)) ok = false;
        if (!ok) break;
        tc_fence_after();
        for (int c0 = 0; c0 < W; c0 += SCH) {
          const int64_t cbase = t * BN + j * W + c0;
          const int64_t rem = p.ncells - cbase;
          const int ncol = rem <= 0 ? 0 : (rem < SCH ? (int)rem : SCH);
          if (ncol == 0) break;  // uniform over the epilogue warps
          float* sbuf = stage0 + (size_t)(chunk % (uint32_t)p.stage_bufs) * SCH * N;
#pragma unroll 1
          for (int m0 = 0; m0 < MT; m0 += SG) {
            uint32_t v[SG][SCH];
#pragma unroll
            for (int g = 0; g < SG; ++g)
              if (m0 + g < MT && (m0 + g) * BM + q * 32 < N)  // warp-uniform
                tmem_ld_cols<SCH>(tmem + ((uint32_t)(q * 32) << 16) + ((rc + m0 + g) % nslot) * W + c0, v[g]);
            tmem_wait_ld();
#pragma unroll
            for (int g = 0; g < SG; ++g) {
              const int o = (m0 + g) * BM + q * 32 + lane;
              if (m0 + g < MT && o < N) {
                float* dst = sbuf + o;
#pragma unroll
                for (int cc = 0; cc < SCH; ++cc)
                  if (cc < ncol) dst[cc * N] = __uint_as_float(v[g][cc]);
              }
            }
          }
          fence_proxy_async();  // the rows reach the bulk copy's (async) view of shared memory
          __syncwarp();
          // the buffer written next was last read by the copy of chunk + 1 - stage_bufs
          if (threadIdx.x == 0) {
            if (p.stage_bufs >= 4) bulk_wait_read<2>();
            else if (p.stage_bufs == 3) bulk_wait_read<1>();
            else bulk_wait_read<0>();
          }
          // every warp's rows are in the buffer (a bounded wait, unlike bar.sync, so that a warp
          // leaving on a timeout cannot strand the others)
          if (lane == 0) mbar_arrive(smem_u32(&bars->epi));
          if (!mbar_wait(smem_u32(&bars->epi), chunk & 1u, p.err)) { ok = false; break; }
          const int full = ncol & ~3;  // whole groups of 4 rows: a multiple of 16 bytes
          if (threadIdx.x == 0 && full > 0) {
            bulk_s2g(p.out + cbase * N, smem_u32(sbuf), (uint32_t)(full * N * 4));
            bulk_commit();
          }
          for (int i = threadIdx.x; i < (ncol - full) * N; i += EPI_WARPS * 32)  // ragged last rows
            p.out[(cbase + full) * N + i] = sbuf[full * N + i];
          ++chunk;
        }
        if (!ok) break;
        tc_fence_before();
        __syncwarp();
        if (lane == 0)
          for (int m = 0; m < MT; ++m) mbar_arrive(smem_u32(&bars->tempty[(rc + m) % nslot]));
      }
    }
    if (threadIdx.x == 0) bulk_wait_all();  // shared memory stays valid until every copy has read it
  } else if constexpr (!CSR) {
    // ---------------- epilogue, direct 128-byte stores ----------------
    const int q = warp;  // TMEM lane quadrant
    const int W = p.subw, nslot = 512 / W;
    uint32_t rc = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      for (int j = 0; j < BN / W && ok; ++j)
      for (int m = 0; m < p.mtiles; ++m, ++rc) {
        const uint32_t slot = rc % nslot, round = rc / nslot;
        if (!mbar_wait(smem_u32(&bars->tfull[slot]), round & 1u, p.err)) { ok = false; break; }
        tc_fence_after();
        const int o = m * BM + q * 32 + lane;
        for (int cc = 0; cc < W; cc += 64) {
          const int cw = W - cc < 64 ? W - cc : 64;  // 64 or 32 columns
          const int64_t cbase = t * BN + j * W + cc;
          const int64_t rem = p.ncells - cbase;
          const int ncol = rem <= 0 ? 0 : (rem < cw ? (int)rem : cw);
          if (m * BM + q * 32 < N && ncol > 0) {
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + slot * W + cc;
            uint32_t v0[32], v1[32];
            tmem_ld32(taddr, v0);
            if (cw == 64) tmem_ld32(taddr + 32, v1);
            tmem_wait_ld();
            if (o < N) {
              float* dst = p.out + cbase * p.ostride + o;
              const int64_t stride = p.ostride;
              if (ncol == 64) {
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) __stcs(dst + jj * stride, __uint_as_float(v0[jj]));
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) __stcs(dst + (32 + jj) * stride, __uint_as_float(v1[jj]));
              } else {
#pragma unroll
                for (int jj = 0; jj < 32; ++jj)
                  if (jj < ncol) __stcs(dst + jj * stride, __uint_as_float(v0[jj]));
#pragma unroll
                for (int jj = 0; jj < 32; ++jj)
                  if (32 + jj < ncol) __stcs(dst + (32 + jj) * stride, __uint_as_float(v1[jj]));
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bars->tempty[slot]));
      }
    }
  } else {
    // ---------------- epilogue, global assembly: entries added into the CSR values ----------------
    const int q = warp;  // TMEM lane quadrant
    const int W = p.subw, nslot = 512 / W;
    const int Np = (N + 3) & ~3;  // entries per cell in the map (padded to 16 bytes)
    uint8_t* ring_base = reinterpret_cast<uint8_t*>(bars) + round_up((int)sizeof(Barriers), 128);
    uint64_t* rbar = reinterpret_cast<uint64_t*>(ring_base) + q * CSR_STAGES;
    uint8_t* rbuf = ring_base + CSR_BAR_BYTES + q * CSR_STAGES * CSR_STAGE_BYTES;
    // accumulator = (tile, sub-tile, M-tile): the consumer's order
    struct Acc {
      int64_t t;
      int j, m;
    };
    auto advance = [&](Acc& k) {
      if (++k.m >= p.mtiles) {
        k.m = 0;
        if (++k.j >= BN / W) {
          k.j = 0;
          k.t += gridDim.x;
        }
      }
    };
    // the map blocks ([32 cells][width] each, stored contiguously) of this warp's 32 outputs for
    // the accumulator's cells -> stage: one bulk copy per 32-cell block, one transaction count
    auto issue = [&](const Acc& k, int stage) {
      if (lane != 0) return;
      const uint32_t bar = smem_u32(rbar + stage);
      const int64_t c0 = k.t * BN + k.j * W;  // first cell, a multiple of 32
      const int ob = k.m * 4 + q;
      const int bw = Np - ob * 32 < 32 ? Np - ob * 32 : 32;
      const int64_t rem = k.t < ntiles ? p.ncells - c0 : 0;
      const int nblk = rem <= 0 || bw <= 0 ? 0 : (int)((rem < W ? rem : W) + 31) / 32;
      if (nblk == 0) {
        mbar_arrive(bar);
        return;
      }
      const uint32_t bytes = (uint32_t)(32 * bw * 4);
      csr_expect_tx(bar, bytes * nblk);
      for (int b = 0; b < nblk; ++b)
        csr_bulk_g2s(smem_u32(rbuf + stage * CSR_STAGE_BYTES + b * bytes),
                     p.map + 32 * (((c0 >> 5) + b) * (int64_t)Np + 32 * ob), bytes, bar);
    };
    Acc prod{(int64_t)blockIdx.x, 0, 0};
    issue(prod, 0);
    advance(prod);
    uint32_t issued = 1, n = 0;  // accumulators whose map blocks were requested / consumed
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      for (int j = 0; j < BN / W && ok; ++j)
      for (int m = 0; m < p.mtiles && ok; ++m, ++n) {
        const uint32_t slot = n % nslot, round = n / nslot;
        const int stage = (int)(n % CSR_STAGES);
        issue(prod, (int)((n + 1) % CSR_STAGES));  // refills the stage consumed last
        advance(prod);
        ++issued;
        if (!mbar_wait(smem_u32(&bars->tfull[slot]), round & 1u, p.err)) { ok = false; break; }
        if (!mbar_wait(smem_u32(rbar + stage), (n / CSR_STAGES) & 1u, p.err)) { ok = false; ++n; break; }
        tc_fence_after();
        const int o = m * BM + q * 32 + lane;
        const int ob = m * 4 + q, bw = Np - ob * 32 < 32 ? Np - ob * 32 : 32;
        const uint32_t* sp0 = reinterpret_cast<const uint32_t*>(rbuf + stage * CSR_STAGE_BYTES) + (lane < bw ? lane : 0);
        for (int c = 0; c < W; c += 32) {
          const int64_t cbase = t * BN + j * W + c;
          const int64_t rem = p.ncells - cbase;
          const int ncol = rem <= 0 ? 0 : (rem < 32 ? (int)rem : 32);
          if (m * BM + q * 32 < N && ncol > 0) {  // warp-uniform
            uint32_t v[32], pos[32];
            tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + slot * W + c, v);
            const uint32_t* sp = sp0 + (c >> 5) * 32 * bw;
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) pos[jj] = sp[jj * bw];
            tmem_wait_ld();
            if (o < N) {
#pragma unroll
              for (int jj = 0; jj < 32; ++jj)
                if (jj < ncol) {
                  if (pos[jj] < (uint64_t)p.nnz) atomicAdd(p.out + pos[jj], __uint_as_float(v[jj]));
                  else atomicOr(p.err, ERR_INDEX);
                }
            }
          }
        }
        fence_proxy_async();  // this stage's reads precede its next asynchronous refill
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bars->tempty[slot]));
      }
    }
    // copies requested but not consumed (bounded waits)
    for (; n < issued; ++n) mbar_wait(smem_u32(rbar + n % CSR_STAGES), (n / CSR_STAGES) & 1u, p.err);
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
  int K, kelems, kbytes, tparts, gparts, mtiles, N;
};

// Cells-on-lanes orientation: the element matrix fits one 128-output slice
bool lanes_ok(int mtiles) { return mtiles == 1; }

bool geom_of(int form, int degree, int cell, int prec, Geom& g) {
  if (form == FORM_BURGERS) return false;
  if (prec == PREC_FP64) return false;
  const bool tf32 = prec == PREC_TF32 || prec == PREC_TF32X3;
  const int elem = tf32 ? 4 : 2, kstep = tf32 ? 8 : 16;
  g.K = form_K(form, degree, cell);
  g.kelems = (g.K + kstep - 1) / kstep * kstep;
  g.kbytes = g.kelems * elem;
  g.tparts = prec_tparts(prec);
  g.gparts = prec_gparts(prec);
  const int ns = nnodes(cell, degree);
  g.N = ns * ns;
  g.mtiles = (g.N + BM - 1) / BM;
  return true;
}

int stages_for(const Geom& g, int extra = 0) {
  const int a = g.mtiles * g.tparts * BM * g.kbytes;
  const int b = g.gparts * BN * g.kbytes;
  const int fixed = a + (int)sizeof(Barriers) + 1024 + 64;
  int s = MAX_STAGES;  // even: the stages are split between the two producer groups
  while (s >= 2 && fixed + extra + s * b > SMEM_LIMIT) s -= 2;
  return s >= 2 ? s : 0;
}

}  // namespace
}  // namespace coffee
