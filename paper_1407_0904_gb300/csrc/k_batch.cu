// Mixed-batch local assembly: many (form, degree, cell) groups in ONE persistent
// tcgen05 launch.
//
// The paper's code generator specialises one kernel per (form, degree, cell shape) and
// PyOP2 runs them one after another (sections 4-5); its cost model picks per-kernel
// parameters (section 4's cost-model figure). Here every group's cells are cut into
// 128-cell tiles, the tiles of all groups form one work list, and each CTA takes a
// contiguous, cost-balanced range of it (host plan). Per work item:
//   producer warps 4..11  compute the group's factors G_e (runtime switch over form and
//                         cell shape) into a B-operand stage laid out with that group's K;
//   loader warp 13        streams the group's T^T operand, one 128-output M-tile at a
//                         time, from global memory (L2-resident) into a two-slot ring with
//                         cp.async.bulk, completion tracked by transaction-count mbarriers;
//   MMA warp 12           issues tcgen05.mma per M-tile into the TMEM ring;
//   epilogue warps 0..3   store the element matrices into the group's output.
// Groups of at most 32 entries put the cells on the TMEM lanes (D[cell][o] = G T, operands
// swapped, N = outputs rounded up to 16), so all four epilogue warps write whole rows; the
// others keep the outputs on the lanes (D[o][cell], 128-byte warp stores per cell).
// Groups therefore need not share K, N or tables, and no group's table has to fit in
// shared memory beside the others. All waits are bounded as in k_tc.cu.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstring>
#include <vector>
#include "coffee_internal.h"
#include "tc_common.cuh"

namespace coffee {
namespace {
using namespace tc;

constexpr int BATCH_THREADS = 14 * 32;  // + one loader warp
constexpr int LOADER_WARP = 13;
constexpr int ASLOTS = 2;

struct alignas(8) BatchBars {
  uint64_t full[MAX_STAGES];
  uint64_t empty[MAX_STAGES];
  uint64_t tfull[RING];
  uint64_t tempty[RING];
  uint64_t afull[ASLOTS];
  uint64_t aempty[ASLOTS];
  uint64_t done;
  uint32_t tmem_base;
};

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Group of the work items a role visits in increasing order: found once by a scan, then moved
// forward as the items pass the next group's first item (kept in a register), so a work item
// costs one compare instead of a chain of loads over the group table.
struct GroupCursor {
  const BatchGroup* gs;
  int ngroups, g;
  int64_t next0;  // first item of group g + 1
  __device__ GroupCursor(const BatchGroup* gs_, int n, int64_t it) : gs(gs_), ngroups(n), g(0) {
    while (g + 1 < ngroups && gs[g + 1].item0 <= it) ++g;
    next0 = g + 1 < ngroups ? gs[g + 1].item0 : INT64_MAX;
  }
  __device__ __forceinline__ int at(int64_t it) {
    while (it >= next0) {
      ++g;
      next0 = g + 1 < ngroups ? gs[g + 1].item0 : INT64_MAX;
    }
    return g;
  }
};

template <int PREC, int FORM, int D>
__device__ __forceinline__ void produce_row(const BatchGroup& g, int64_t e, bool live, uint8_t* base, int row) {
  using PT = PrecTraits<PREC>;
  constexpr int KSTEP = PT::tf32 ? 8 : 16;
  constexpr int KP = round_up(Form<FORM, D>::K, KSTEP);
  float G[KP];
  bool bad = false;
  if (live) {
    cell_factors<FORM, D, KP>(g.p, e, G, bad);
    if (bad) atomicOr(g.p.err, ERR_INDEX);
  }
  if (!live || bad) {
#pragma unroll
    for (int k = 0; k < KP; ++k) G[k] = 0.f;
  }
  store_operand_row<PREC, KP>(base, BM * g.p.kbytes, row, G, g.p.kbytes);
}

template <int PREC>
__device__ __forceinline__ void batch_body(const BatchGroup* __restrict__ groups, int ngroups, int64_t it0,
                                           int64_t it1, int nstages, int kbytes_max, unsigned* err) {
  using PT = PrecTraits<PREC>;
  constexpr int TPARTS = PT::TPARTS, GPARTS = PT::GPARTS;
  using PS = Passes<PREC>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int slot_bytes = TPARTS * BM * kbytes_max;   // one A slot (T^T parts of one M-tile)
  const int stage_bytes = GPARTS * BN * kbytes_max;  // one B stage (factor parts of one tile)
  uint8_t* sA = smem;
  uint8_t* sB = smem + ASLOTS * slot_bytes;
  BatchBars* bars = reinterpret_cast<BatchBars*>(sB + nstages * stage_bytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < nstages; ++s) {
      mbar_init(smem_u32(&bars->full[s]), 128);
      mbar_init(smem_u32(&bars->empty[s]), 1);
    }
    for (int r = 0; r < RING; ++r) {
      mbar_init(smem_u32(&bars->tfull[r]), 1);
      mbar_init(smem_u32(&bars->tempty[r]), EPI_WARPS);
    }
    for (int j = 0; j < ASLOTS; ++j) {
      mbar_init(smem_u32(&bars->afull[j]), 1);
      mbar_init(smem_u32(&bars->aempty[j]), 1);
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
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;

  if (warp >= PROD_WARP0 && warp < MMA_WARP) {
    // ---------------- producers ----------------
    const int pw = warp - PROD_WARP0;
    const int grp = pw >> 2, row = ((pw & 3) << 5) + lane;
    const int spg = nstages / PROD_GROUPS;
    GroupCursor cur(groups, ngroups, it0);
    for (int64_t it = it0 + grp; it < it1; it += PROD_GROUPS) {
      const int64_t k = it - it0;
      const int gi = cur.at(it);
      const BatchGroup& g = groups[gi];
      int s;
      uint32_t use;
      stage_of(k / PROD_GROUPS, grp, spg, s, use);
      if (!mbar_wait(smem_u32(&bars->empty[s]), (use & 1u) ^ 1u, err)) break;
      const int64_t e = (it - g.item0) * BN + row;
      const bool live = e < g.p.ncells;
      uint8_t* b = sB + (size_t)s * stage_bytes;
      switch (g.form * 2 + g.cell) {
        case FORM_MASS * 2 + CELL_TRI: produce_row<PREC, FORM_MASS, 2>(g, e, live, b, row); break;
        case FORM_MASS * 2 + CELL_TET: produce_row<PREC, FORM_MASS, 3>(g, e, live, b, row); break;
        case FORM_HELMHOLTZ * 2 + CELL_TRI: produce_row<PREC, FORM_HELMHOLTZ, 2>(g, e, live, b, row); break;
        case FORM_HELMHOLTZ * 2 + CELL_TET: produce_row<PREC, FORM_HELMHOLTZ, 3>(g, e, live, b, row); break;
        case FORM_ADVDIFF * 2 + CELL_TRI: produce_row<PREC, FORM_ADVDIFF, 2>(g, e, live, b, row); break;
        default: produce_row<PREC, FORM_ADVDIFF, 3>(g, e, live, b, row); break;
      }
      fence_proxy_async();
      mbar_arrive(smem_u32(&bars->full[s]));
    }
  } else if (warp == LOADER_WARP) {
    // ---------------- T^T operand loader ----------------
    if (lane == 0) {
      uint32_t la = 0, last_round[ASLOTS] = {0, 0};
      bool used[ASLOTS] = {false, false};
      int tag[ASLOTS] = {-1, -1};  // (group, slice) held by each slot: consecutive items of a
                                   // group find their slices already resident
      bool ok = true;
      GroupCursor cur(groups, ngroups, it0);
      for (int64_t it = it0; it < it1 && ok; ++it) {
        const int gi = cur.at(it);
        const BatchGroup& g = groups[gi];
        const uint32_t part_bytes = (uint32_t)(BM * g.p.kbytes);
        for (int m = 0; m < g.p.mtiles; ++m, ++la) {
          const uint32_t j = la % ASLOTS, round = la / ASLOTS;
          if (!mbar_wait(smem_u32(&bars->aempty[j]), (round & 1u) ^ 1u, err)) { ok = false; break; }
          const uint32_t bar = smem_u32(&bars->afull[j]);
          used[j] = true;
          last_round[j] = round;  // the slot's latest phase, whether it copies or not
          if (tag[j] == gi * 64 + m) {  // already resident: complete the phase without a copy
            mbar_arrive(bar);
            continue;
          }
          tag[j] = gi * 64 + m;
          mbar_arrive_expect_tx(bar, part_bytes * TPARTS);
          const uint8_t* src = g.p.image + (size_t)m * TPARTS * part_bytes;
          const uint32_t dst = smem_u32(sA + (size_t)j * slot_bytes);
#pragma unroll
          for (int q = 0; q < TPARTS; ++q) bulk_g2s(dst + q * part_bytes, src + (size_t)q * part_bytes, part_bytes, bar);
        }
      }
      // every copy this thread started has landed before shared memory is released (phases
      // of a slot complete in order, so waiting for its latest phase covers all of them)
      for (int j = 0; j < ASLOTS; ++j)
        if (used[j]) mbar_wait(smem_u32(&bars->afull[j]), last_round[j] & 1u, err);
    }
    __syncwarp();
  } else if (warp == MMA_WARP) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      uint32_t rc = 0, ma = 0;
      int k = 0;
      bool ok = true;
      GroupCursor cur(groups, ngroups, it0);
      for (int64_t it = it0; it < it1 && ok; ++it, ++k) {
        const BatchGroup& g = groups[cur.at(it)];
        const int kb = g.p.kbytes, ksteps = kb / 32;
        const uint32_t sbo = 8u * (uint32_t)kb, part = (uint32_t)(BM * kb);
        const bool lanes = g.lanes != 0;
        const uint32_t idesc = make_idesc(PT::tf32 ? 2 : 1, BM, lanes ? ((g.p.N + 15) & ~15) : BN);
        int s;
        uint32_t use;
        stage_of(k / PROD_GROUPS, k % PROD_GROUPS, nstages / PROD_GROUPS, s, use);
        if (!mbar_wait(smem_u32(&bars->full[s]), use & 1u, err)) break;
        tc_fence_after();
        const uint32_t bstage = b0 + (uint32_t)(s * stage_bytes);
        for (int m = 0; m < g.p.mtiles; ++m, ++rc, ++ma) {
          const uint32_t j = ma % ASLOTS, around = ma / ASLOTS;
          if (!mbar_wait(smem_u32(&bars->afull[j]), around & 1u, err)) { ok = false; break; }
          const uint32_t slot = rc % RING, round = rc / RING;
          if (!mbar_wait(smem_u32(&bars->tempty[slot]), (round & 1u) ^ 1u, err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t d = tmem + slot * BN;
          const uint32_t atile = a0 + j * (uint32_t)slot_bytes;
          uint32_t acc = 0;
          for (int ks = 0; ks < ksteps; ++ks) {
            const uint32_t ko = (uint32_t)ks * 256u;
#pragma unroll
            for (int i = 0; i < PS::N; ++i) {
              // part t of T^T and part g of G, smallest products first; outputs on lanes:
              // A = T^T slice, B = G stage; cells on lanes: A = G, B = T^T
              const uint32_t tt = atile + (uint32_t)PS::t(i) * part + ko;
              const uint32_t gg = bstage + (uint32_t)PS::g(i) * part + ko;
              mma<PT::tf32>(d, make_desc(lanes ? gg : tt, sbo), make_desc(lanes ? tt : gg, sbo), idesc, acc);
              acc = 1;
            }
          }
          tc_commit(smem_u32(&bars->tfull[slot]));
          tc_commit(smem_u32(&bars->aempty[j]));
        }
        tc_commit(smem_u32(&bars->empty[s]));
      }
      tc_commit(smem_u32(&bars->done));
      mbar_wait(smem_u32(&bars->done), 0, err);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue ----------------
    const int q = warp;  // TMEM lane quadrant
    uint32_t rc = 0;
    bool ok = true;
    GroupCursor cur(groups, ngroups, it0);
    for (int64_t it = it0; it < it1 && ok; ++it) {
      const BatchGroup& g = groups[cur.at(it)];
      const int N = g.p.N;
      const int64_t RS = g.p.ostride;  // row stride of the output (N unless padded)
      if (g.lanes) {
        // cells on lanes: thread = cell, its row of N <= 32 outputs from one TMEM load
        const uint32_t slot = rc % RING, round = rc / RING;
        ++rc;
        if (!mbar_wait(smem_u32(&bars->tfull[slot]), round & 1u, err)) { ok = false; break; }
        tc_fence_after();
        const int64_t c0 = (it - g.item0) * BN + q * 32;
        if (c0 < g.p.ncells) {  // warp-uniform
          uint32_t v[32];
          const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + slot * BN;
          if (N > 16) tmem_ld32(taddr, v);
          else tmem_ld16(taddr, *reinterpret_cast<uint32_t(*)[16]>(v));
          tmem_wait_ld();
          if (c0 + lane < g.p.ncells) {
            float* row = g.p.out + (c0 + lane) * RS;
            if ((RS & 3) == 0 && (reinterpret_cast<uintptr_t>(g.p.out) & 15) == 0) {
#pragma unroll
              for (int k4 = 0; k4 < 8; ++k4)
                if (4 * k4 < N)
                  __stcs(reinterpret_cast<float4*>(row + 4 * k4),
                         make_float4(__uint_as_float(v[4 * k4]), __uint_as_float(v[4 * k4 + 1]),
                                     __uint_as_float(v[4 * k4 + 2]), __uint_as_float(v[4 * k4 + 3])));
            } else {
#pragma unroll
              for (int k = 0; k < 32; ++k)
                if (k < N) __stcs(row + k, __uint_as_float(v[k]));
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bars->tempty[slot]));
        continue;
      }
      for (int m = 0; m < g.p.mtiles; ++m, ++rc) {
        const uint32_t slot = rc % RING, round = rc / RING;
        if (!mbar_wait(smem_u32(&bars->tfull[slot]), round & 1u, err)) { ok = false; break; }
        tc_fence_after();
        const int o = m * BM + q * 32 + lane;
        for (int half = 0; half < 2; ++half) {
        const int64_t cbase = (it - g.item0) * BN + half * 64;
        const int64_t rem = g.p.ncells - cbase;
        const int ncol = rem <= 0 ? 0 : (rem < 64 ? (int)rem : 64);
        if (m * BM + q * 32 < N && ncol > 0) {
          const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + slot * BN + half * 64;
          uint32_t v0[32], v1[32];
          tmem_ld32(taddr, v0);
          tmem_ld32(taddr + 32, v1);
          tmem_wait_ld();
          if (o < N) {
            float* dst = g.p.out + cbase * RS + o;
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (j < ncol) __stcs(dst + (int64_t)j * RS, __uint_as_float(v0[j]));
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (32 + j < ncol) __stcs(dst + (int64_t)(32 + j) * RS, __uint_as_float(v1[j]));
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

// Several groups: work items of CTA b are [ranges[b], ranges[b+1]) (cost-balanced on the host).
template <int PREC>
__global__ void __launch_bounds__(BATCH_THREADS, 1)
    k_batch_tc(const BatchGroup* __restrict__ groups, int ngroups, const int64_t* __restrict__ ranges,
               int nstages, int kbytes_max, unsigned* err) {
  batch_body<PREC>(groups, ngroups, ranges[blockIdx.x], ranges[blockIdx.x + 1], nstages, kbytes_max, err);
}

// One group passed by value (no device allocation): equal split of its tiles over the grid.
template <int PREC>
__global__ void __launch_bounds__(BATCH_THREADS, 1)
    k_stream_one_tc(const __grid_constant__ BatchGroup g, int64_t items, int nstages, int kbytes_max) {
  const int64_t it0 = items * blockIdx.x / gridDim.x, it1 = items * (blockIdx.x + 1) / gridDim.x;
  batch_body<PREC>(&g, 1, it0, it1, nstages, kbytes_max, g.p.err);
}

constexpr int SMEM_LIMIT = 227 * 1024;
constexpr int SMEM_ONE_CTA = 120 * 1024;

template <int PREC>
cudaError_t prepare_t(int smem) {
  cudaError_t e = cudaFuncSetAttribute(k_batch_tc<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_stream_one_tc<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}
template <int PREC>
cudaError_t launch_one_t(const BatchGroup& g, int64_t items, int grid, int smem, int nstages, int kbytes_max,
                         cudaStream_t s) {
  k_stream_one_tc<PREC><<<grid, BATCH_THREADS, smem, s>>>(g, items, nstages, kbytes_max);
  return cudaGetLastError();
}
template <int PREC>
cudaError_t launch_t(const BatchLaunch& L, cudaStream_t s) {
  k_batch_tc<PREC><<<L.grid, BATCH_THREADS, L.smem, s>>>(L.groups, L.ngroups, L.ranges, L.nstages, L.kbytes_max,
                                                         L.err);
  return cudaGetLastError();
}

}  // namespace

int batch_smem(int kbytes_max, int precision, int* nstages) {
  const int slot = prec_tparts(precision) * BM * kbytes_max, stage = prec_gparts(precision) * BN * kbytes_max;
  const int fixed = ASLOTS * slot + (int)sizeof(BatchBars) + 1024 + 64;
  int s = MAX_STAGES;  // even: the stages are split between the two producer groups
  while (s >= 2 && fixed + s * stage > SMEM_LIMIT) s -= 2;
  if (s < 2) return 0;
  *nstages = s;
  const int smem = fixed + s * stage;
  return smem < SMEM_ONE_CTA ? SMEM_ONE_CTA : smem;
}

int batch_prepare(int precision, int smem) {
  switch (precision) {
    case PREC_TF32: return (int)prepare_t<PREC_TF32>(smem);
    case PREC_TF32X3: return (int)prepare_t<PREC_TF32X3>(smem);
    case PREC_BF16: return (int)prepare_t<PREC_BF16>(smem);
    case PREC_BF16X3: return (int)prepare_t<PREC_BF16X3>(smem);
  }
  return (int)cudaErrorInvalidValue;
}

// Single group with its T^T operand streamed per M-tile (used when it does not fit in
// shared memory for the resident-operand kernel).
int stream_one_supported(int form, int kbytes, int precision) {
  int nst = 0;
  return form != FORM_BURGERS && batch_smem(kbytes, precision, &nst) > 0;
}

int launch_stream_one(const BatchGroup& g, int num_sms, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int nstages = 0;
  const int smem = batch_smem(g.p.kbytes, g.p.precision, &nstages);
  if (smem == 0) return (int)cudaErrorInvalidValue;
  cudaError_t e = (cudaError_t)batch_prepare(g.p.precision, smem);
  if (e != cudaSuccess) return (int)e;
  const int64_t items = (g.p.ncells + BN - 1) / BN;
  const int grid = (int)(items < num_sms ? items : num_sms);
  switch (g.p.precision) {
    case PREC_TF32: return (int)launch_one_t<PREC_TF32>(g, items, grid, smem, nstages, g.p.kbytes, s);
    case PREC_TF32X3: return (int)launch_one_t<PREC_TF32X3>(g, items, grid, smem, nstages, g.p.kbytes, s);
    case PREC_BF16: return (int)launch_one_t<PREC_BF16>(g, items, grid, smem, nstages, g.p.kbytes, s);
    case PREC_BF16X3: return (int)launch_one_t<PREC_BF16X3>(g, items, grid, smem, nstages, g.p.kbytes, s);
  }
  return (int)cudaErrorInvalidValue;
}

int batch_launch(const BatchLaunch& L, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (L.precision) {
    case PREC_TF32: return (int)launch_t<PREC_TF32>(L, s);
    case PREC_TF32X3: return (int)launch_t<PREC_TF32X3>(L, s);
    case PREC_BF16: return (int)launch_t<PREC_BF16>(L, s);
    case PREC_BF16X3: return (int)launch_t<PREC_BF16X3>(L, s);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace coffee
