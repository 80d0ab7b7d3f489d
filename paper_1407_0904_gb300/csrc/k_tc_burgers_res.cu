// tcgen05 assembly of the Burgers residual, an element vector (section 2 names element
// vectors beside element matrices; Listing 2's problem, degree k).
//
// The residual is quadratic in u: with (u.grad u)_c = sum_s u[s][c] (u.grad phi_s) and
// grad u_c = sum_s u[s][c] grad phi_s, each component block of R is
//   R[(c, i)] = sum_s C[i][s] u[s][c],
//   C[i][s]   = sum_{r,a} Q[r][a] T2[r,a][i,s] + nu sum_p H_p T3[p][i,s],
// where C is the advective-viscous part of the Jacobian's diagonal block
// (Q[r][a] = sum_c u[r][c] P[a][c], P = |det J| K). C is one contraction against the T2 and T3
// tensors of the Jacobian (their columns only: the operand image holds [T2 | T3]^T, K = d ns
// + d(d+1)/2 rounded up to the MMA step), computed on the tensor cores with the CELLS on the
// TMEM lanes (M = 128 cells, N = ns*ns outputs rounded up to 16, up to 256); each epilogue
// thread then holds its own cell's C, multiplies it by the cell's u and writes its
// component-blocked row of d*ns values.
// The producers gather u for the factors Q anyway; they also leave it, as floats, in a ring of
// shared-memory buffers beside the TMEM accumulators (one per accumulator slot, [d ns][128
// cells], so producer and epilogue threads touch consecutive words), with a full barrier per
// slot: the epilogue reads its cell's u there instead of gathering it from global memory a
// second time. (Measured with per-role cycle counters before this change: the epilogue spent a
// third of its time on that gather and waited on the MMA only 4% of the time, so it set the
// rate.) A slot's buffer is rewritten after the epilogue has released the slot's accumulator,
// which it does after its last read of u.
// Each epilogue warp stages its 32 cells' rows (contiguous in the output) in shared memory and
// writes them with coalesced 16-byte stores: written by each thread as its own 4 d ns-byte row,
// every store instruction of the warp touched 32 sectors for 256 bytes (measured: without the
// output stores the kernel ran 20% faster).
// Pipeline roles and bounded waits are those of k_tc_burgers.cu.
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

// residual operand geometry: K columns [T2 | T3] (K1 = d ns, then P), padded to the MMA step
template <int D, int NS, int PREC>
struct ResShape {
  using PT = PrecTraits<PREC>;
  static constexpr int KSTEP = PT::tf32 ? 8 : 16;
  static constexpr int P = D * (D + 1) / 2;
  static constexpr int K1 = NS * D;
  static constexpr int KR = round_up(K1 + P, KSTEP);
  static constexpr int NBLK = NS * NS;
  static constexpr int MT = (NBLK + BM - 1) / BM;    // 128-row tiles of the T operand
  static constexpr int NPAD = round_up(NBLK, 16);   // MMA N (outputs), <= 256
  static constexpr int SLOTW = NPAD <= 128 ? 128 : 256;
  static constexpr int NSLOT = 512 / SLOTW;
  static constexpr int UBYTES = NSLOT * K1 * BM * 4;  // the u ring
  static constexpr int OSTRIDE = NS * D + 1;            // staged output row (odd: conflict-free)
  static constexpr int OBYTES = EPI_WARPS * 32 * OSTRIDE * 4;
};

template <int D, int NS, int PREC>
__global__ void __launch_bounds__(NTHREADS, 1) k_burgers_res_tc(const TcParams p, int nstages) {
  using S = ResShape<D, NS, PREC>;
  using PT = PrecTraits<PREC>;
  constexpr int NV = D + 1, P = S::P, K1 = S::K1, KR = S::KR, KSTEP = S::KSTEP;
  constexpr int TPARTS = PT::TPARTS, GPARTS = PT::GPARTS;
  using PS = Passes<PREC>;
  constexpr int NPAD = S::NPAD, SLOTW = S::SLOTW, NSLOT = S::NSLOT;
  static_assert(NPAD <= 256, "residual kernel: at most 256 outputs per cell");
  constexpr int NDOF = D * NS;

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int kbytes = p.kbytes;  // = KR * ELEM
  const int tile_bytes = BM * kbytes;
  const int a_bytes = S::MT * TPARTS * tile_bytes;
  uint8_t* sA = smem;
  uint8_t* sB = smem + a_bytes;
  float* ring = reinterpret_cast<float*>(sB + nstages * GPARTS * tile_bytes);  // [NSLOT][K1][BM]
  float* ostage = ring + S::UBYTES / 4;  // [EPI_WARPS][32][OSTRIDE]
  Barriers* bars = reinterpret_cast<Barriers*>(reinterpret_cast<uint8_t*>(ostage) + S::OBYTES);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (p.ncells + BN - 1) / BN;
  const float nu = (float)p.nu;

  if (threadIdx.x == 0) {
    for (int s = 0; s < nstages; ++s) {
      mbar_init(smem_u32(&bars->full[s]), 128);
      mbar_init(smem_u32(&bars->empty[s]), 1);
    }
    for (int r = 0; r < NSLOT; ++r) {
      mbar_init(smem_u32(&bars->tfull[r]), 1);
      mbar_init(smem_u32(&bars->tempty[r]), EPI_WARPS);
      mbar_init(smem_u32(&bars->aux[r]), 128);  // u of the slot's tile written
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
    // ---------------- producers: one cell per thread, one tile per stage ----------------
    const int pw = warp - PROD_WARP0;
    const int grp = pw >> 2, row = ((pw & 3) << 5) + lane;
    const int spg = nstages / PROD_GROUPS;
    const int64_t tstep = (int64_t)PROD_GROUPS * gridDim.x;
    // index rows one tile ahead (the next tile of this group): the coordinate and u gathers of
    // a tile then wait on one level of loads instead of two
    int nvid[NV], ndid[NS];
    {
      const int64_t e0 = (blockIdx.x + (int64_t)grp * gridDim.x) * BN + row;
#pragma unroll
      for (int v = 0; v < NV; ++v) nvid[v] = e0 < p.ncells ? __ldg(p.c2v + e0 * NV + v) : 0;
#pragma unroll
      for (int r = 0; r < NS; ++r) ndid[r] = e0 < p.ncells ? __ldg(p.c2d + e0 * NS + r) : 0;
    }
    int64_t li = 0;
    for (int64_t t = blockIdx.x + (int64_t)grp * gridDim.x; t < ntiles; t += tstep, ++li) {
      const int64_t e = t * BN + row;
      const int64_t tl = li * PROD_GROUPS + grp;  // the CTA's tile number: its accumulator slot
      const uint32_t slot = (uint32_t)(tl % NSLOT), round = (uint32_t)(tl / NSLOT);
      int vid[NV], did[NS];
#pragma unroll
      for (int v = 0; v < NV; ++v) vid[v] = nvid[v];
#pragma unroll
      for (int r = 0; r < NS; ++r) did[r] = ndid[r];
      {
        const int64_t en = e + tstep * BN;
#pragma unroll
        for (int v = 0; v < NV; ++v) nvid[v] = en < p.ncells ? __ldg(p.c2v + en * NV + v) : 0;
#pragma unroll
        for (int r = 0; r < NS; ++r) ndid[r] = en < p.ncells ? __ldg(p.c2d + en * NS + r) : 0;
      }
      int s;
      uint32_t use;
      stage_of(li, grp, spg, s, use);
      if (!mbar_wait(smem_u32(&bars->empty[s]), (use & 1u) ^ 1u, p.err)) break;
      float u[NS][D], Pm[D][D], H[P];
      bool live = e < p.ncells;
      if (live) {
        bool bad = false;
#pragma unroll
        for (int v = 0; v < NV; ++v)
          if (p.validate && (vid[v] < 0 || vid[v] >= p.nverts)) bad = true;
#pragma unroll
        for (int r = 0; r < NS; ++r)
          if (p.validate && (did[r] < 0 || did[r] >= p.ncoefnodes)) bad = true;
        if (bad) {
          atomicOr(p.err, ERR_INDEX);
          live = false;
        } else {
          // u's loads first: issued before the coordinates' and the geometry, both gathers share
          // one round trip to memory instead of the second waiting for the geometry
          coef_rows<NS, D>(p, did, u);
          float adj[D][D], Dm, sg;
          cell_geometry_ids<D>(p, vid, adj, Dm, sg);
          const float inv = 1.0f / Dm;
#pragma unroll
          for (int a = 0; a < D; ++a)
#pragma unroll
            for (int c = 0; c < D; ++c) Pm[a][c] = sg * adj[a][c];
          int q = 0;
#pragma unroll
          for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = a; b < D; ++b) {
              float acc = 0.f;
#pragma unroll
              for (int r = 0; r < D; ++r) acc = fmaf(adj[a][r], adj[b][r], acc);
              H[q++] = nu * acc * inv;
            }
        }
      }
      // u for the epilogue, once the slot's previous tile has left it
      if (!mbar_wait(smem_u32(&bars->tempty[slot]), (round & 1u) ^ 1u, p.err)) break;
      float* us = ring + (size_t)slot * K1 * BM;
#pragma unroll
      for (int r = 0; r < NS; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) us[(r * D + c) * BM + row] = live ? u[r][c] : 0.f;
      mbar_arrive(smem_u32(&bars->aux[slot]));
      // factors of C: Q[r][a] (T2 columns), nu H (T3 columns)
      auto factor = [&](int k) -> float {
        if (!live) return 0.f;
        if (k < K1) {
          const int r = k / D, a = k % D;
          float q = 0.f;
#pragma unroll
          for (int c = 0; c < D; ++c) q = fmaf(u[r][c], Pm[a][c], q);
          return q;
        }
        if (k < K1 + P) return H[k - K1];
        return 0.f;
      };
      store_operand_fn<PREC, KR, decltype(factor)>(sB + (size_t)s * GPARTS * tile_bytes, tile_bytes, row, kbytes, factor);
      fence_proxy_async();
      mbar_arrive(smem_u32(&bars->full[s]));
    }
  } else if (warp == MMA_WARP) {
    // ---------------- MMA issuer: D[cell][o] = G[cell][k] T^T[o][k], k over T2|T3 ----------------
    if (lane == 0) {
      const uint32_t sbo = 8u * (uint32_t)kbytes;
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      const int spg = nstages / PROD_GROUPS;
      uint32_t rc = 0;
      int64_t tl = 0;
      for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++tl, ++rc) {
        int s;
        uint32_t use;
        stage_of(tl / PROD_GROUPS, (int)(tl % PROD_GROUPS), spg, s, use);
        if (!mbar_wait(smem_u32(&bars->full[s]), use & 1u, p.err)) break;
        const uint32_t slot = rc % NSLOT, round = rc / NSLOT;
        if (!mbar_wait(smem_u32(&bars->tempty[slot]), (round & 1u) ^ 1u, p.err)) break;
        tc_fence_after();
        const uint32_t g = b0 + (uint32_t)(s * GPARTS * tile_bytes);  // A: cells x K
#pragma unroll
        for (int m = 0; m < S::MT; ++m) {  // B: 128-output tiles of T^T
          const int nm = (NPAD - m * 128) < 128 ? NPAD - m * 128 : 128;
          const uint32_t idesc = make_idesc(PT::tf32 ? 2 : 1, BM, nm);
          const uint32_t tt = a0 + (uint32_t)(m * TPARTS * tile_bytes);
          const uint32_t d = tmem + slot * SLOTW + m * 128;
          uint32_t acc = 0;
          for (int ks = 0; ks < KR / KSTEP; ++ks) {
            const uint32_t ko = (uint32_t)ks * 256u;
#pragma unroll
            for (int i = 0; i < PS::N; ++i) {  // products of parts, smallest first
              mma<PT::tf32>(d, make_desc(g + (uint32_t)(PS::g(i) * tile_bytes) + ko, sbo),
                            make_desc(tt + (uint32_t)(PS::t(i) * tile_bytes) + ko, sbo), idesc, acc);
              acc = 1;
            }
          }
        }
        tc_commit(smem_u32(&bars->tfull[slot]));
        tc_commit(smem_u32(&bars->empty[s]));
      }
      tc_commit(smem_u32(&bars->done));
      mbar_wait(smem_u32(&bars->done), 0, p.err);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: each thread forms and writes its cell's residual ----------------
    const int q = warp;  // lanes 32q..32q+31 = cells of the tile
    const int row = q * 32 + lane;
    float* ost = ostage + q * 32 * S::OSTRIDE;
    const bool vec = (reinterpret_cast<uintptr_t>(p.out) & 15u) == 0;
    uint32_t rc = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++rc) {
      const uint32_t slot = rc % NSLOT, round = rc / NSLOT;
      const int64_t cell = t * BN + row;
      const bool live = cell < p.ncells;
      if (!mbar_wait(smem_u32(&bars->tfull[slot]), round & 1u, p.err)) break;
      if (!mbar_wait(smem_u32(&bars->aux[slot]), round & 1u, p.err)) break;
      tc_fence_after();
      const float* us = ring + (size_t)slot * K1 * BM + row;
      float R[D][NS];
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int i = 0; i < NS; ++i) R[c][i] = 0.f;
      if (t * BN + q * 32 < p.ncells) {  // warp-uniform
        // 32 accumulator columns per TMEM wait (two 16-column loads)
#pragma unroll
        for (int o0 = 0; o0 < NPAD; o0 += 32) {
          uint32_t v[2][16];
          tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + slot * SLOTW + o0, v[0]);
          if (o0 + 16 < NPAD) tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + slot * SLOTW + o0 + 16, v[1]);
          tmem_wait_ld();
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
              const int o = o0 + 16 * h + jj;
              if (o < S::NBLK) {
                const int i = o / NS, s = o % NS;
#pragma unroll
                for (int c = 0; c < D; ++c) R[c][i] = fmaf(__uint_as_float(v[h][jj]), us[(s * D + c) * BM], R[c][i]);
              }
            }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars->tempty[slot]));  // accumulator and u buffer free
      // the warp's rows, contiguous in the output, through shared memory
      const int64_t c0 = t * BN + q * 32;
      if (c0 < p.ncells) {  // warp-uniform
#pragma unroll
        for (int x = 0; x < NDOF; ++x) ost[lane * S::OSTRIDE + x] = R[x / NS][x % NS];
        __syncwarp();
        const int nlive = (int)((p.ncells - c0) < 32 ? (p.ncells - c0) : 32);
        const int nel = nlive * NDOF;
        float* out = p.out + c0 * NDOF;
        const int n4 = vec ? nel / 4 : 0;  // rows of 32 cells start 128 d ns bytes apart
        for (int f = lane; f < n4; f += 32) {
          float v[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int e = 4 * f + j;
            v[j] = ost[(e / NDOF) * S::OSTRIDE + e % NDOF];
          }
          __stcs(reinterpret_cast<float4*>(out) + f, make_float4(v[0], v[1], v[2], v[3]));
        }
        for (int e = 4 * n4 + lane; e < nel; e += 32) __stcs(out + e, ost[(e / NDOF) * S::OSTRIDE + e % NDOF]);
        __syncwarp();
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

// shared-memory bytes of one launch with nst operand stages
int res_smem(int ns, int d, int prec, int nst) {
  const bool tf32 = prec == PREC_TF32 || prec == PREC_TF32X3;
  const int kstep = tf32 ? 8 : 16, elem = tf32 ? 4 : 2, P = d * (d + 1) / 2, K1 = ns * d;
  const int kbytes = round_up(K1 + P, kstep) * elem;
  const int npad = round_up(ns * ns, 16), nslot = npad <= 128 ? 4 : 2, mt = (ns * ns + BM - 1) / BM;
  const int obytes = EPI_WARPS * 32 * (ns * d + 1) * 4;  // ResShape::OBYTES
  return mt * prec_tparts(prec) * BM * kbytes + nst * prec_gparts(prec) * BN * kbytes + nslot * K1 * BM * 4 +
         obytes + (int)sizeof(Barriers) + 1024 + 64;
}

// operand stages (even, one set per producer group) that fit, 0 if none
int res_stages(int ns, int d, int prec) {
  int s = MAX_STAGES;
  while (s >= 2 && res_smem(ns, d, prec, s) > 227 * 1024) s -= 2;
  return s >= 2 ? s : 0;
}

bool res_shape(int degree, int cell, int prec, int& ns, int& d) {
  if (prec == PREC_FP64 || prec < 0 || prec > PREC_BF16X3) return false;
  if (cell == CELL_TRI ? (degree < 1 || degree > 4) : (cell != CELL_TET || degree < 1 || degree > 2)) return false;
  ns = nnodes(cell, degree);
  d = cell == CELL_TRI ? 2 : 3;
  return ns * ns <= 256;
}

template <int D, int NS, int PREC>
cudaError_t launch_r(const TcParams& p, int num_sms, cudaStream_t s, int nst, int smem) {
  auto kern = k_burgers_res_tc<D, NS, PREC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (p.ncells + BN - 1) / BN;
  const int grid = (int)(ntiles < num_sms ? ntiles : num_sms);
  kern<<<grid, NTHREADS, smem, s>>>(p, nst);
  return cudaGetLastError();
}

template <int D, int NS>
cudaError_t launch_rp(const TcParams& p, int num_sms, cudaStream_t s, int nst, int smem) {
  switch (p.precision) {
    case PREC_TF32: return launch_r<D, NS, PREC_TF32>(p, num_sms, s, nst, smem);
    case PREC_TF32X3: return launch_r<D, NS, PREC_TF32X3>(p, num_sms, s, nst, smem);
    case PREC_BF16: return launch_r<D, NS, PREC_BF16>(p, num_sms, s, nst, smem);
    case PREC_BF16X3: return launch_r<D, NS, PREC_BF16X3>(p, num_sms, s, nst, smem);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

int burgers_res_tc_supported(int degree, int cell, int precision) {
  int ns = 0, d = 0;
  if (!res_shape(degree, cell, precision, ns, d)) return 0;
  return res_stages(ns, d, precision) > 0 ? 1 : 0;
}

// The residual's operand image: [T2 | T3]^T of the Burgers reference tensors (rows = the ns*ns
// entries of a component block in 128-row tiles, columns = the K1 = d ns T2 rows then the P T3
// rows, zero padding to the MMA step), split into the precision's parts of T, in the canonical
// layout, [tile][part][128 x kbytes].
void build_burgers_res_image(int degree, int cell, int prec, std::vector<uint8_t>& img, TcTable& meta) {
  int ns = 0, d = 0;
  res_shape(degree, cell, prec, ns, d);
  std::vector<double> T;
  reference_tensor(FORM_BURGERS, degree, cell, T);  // rows: T1 (d ns), T2 (d ns), T3 (P)
  const bool tf32 = prec == PREC_TF32 || prec == PREC_TF32X3;
  const int kstep = tf32 ? 8 : 16, elem = tf32 ? 4 : 2, P = d * (d + 1) / 2, K1 = ns * d, nb = ns * ns;
  const int KR = round_up(K1 + P, kstep), kbytes = KR * elem, parts = prec_tparts(prec);
  const int mtiles = (nb + BM - 1) / BM;
  const int64_t tile = (int64_t)BM * kbytes;
  img.assign((size_t)(mtiles * parts * tile), 0);
  for (int m = 0; m < mtiles; ++m)
    for (int r = 0; r < BM; ++r) {
      const int o = m * BM + r;
      for (int k = 0; k < KR; ++k) {
        const int tr = k < K1 + P ? K1 + k : -1;  // T2 rows follow the K1 rows of T1, then T3
        const double x = (o >= nb || tr < 0) ? 0.0 : T[(size_t)tr * nb + o];
        host_store_parts(img.data() + (size_t)(m * parts) * tile, (size_t)tile, canon_off(r, k * elem, kbytes), x,
                         tf32, parts);
      }
    }
  meta = TcTable{};
  meta.mtiles = mtiles;
  meta.kbytes = kbytes;
  meta.kelems = KR;
  meta.K = K1 + P;
  meta.tparts = parts;
  meta.ksteps_off = 0;
  meta.tile_bytes = tile;
}

int launch_burgers_res_tc(int cell, const TcParams& p, int num_sms, void* stream, std::string& why) {
  if (p.ncells == 0) return (int)cudaSuccess;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int d = cell == CELL_TRI ? 2 : 3;
  const int nst = res_stages(p.ns, d, p.precision);
  if (nst == 0) {
    why = "operands do not fit in shared memory";
    return (int)cudaErrorInvalidValue;
  }
  int use = nst;
  if (use > 2 && (p.tune & TUNE_TWO_STAGES)) use = 2;
  int smem = res_smem(p.ns, d, p.precision, use);
  if (smem < SMEM_ONE_CTA) smem = SMEM_ONE_CTA;
  if (cell == CELL_TRI) {
    switch (p.ns) {
      case 3: return (int)launch_rp<2, 3>(p, num_sms, s, use, smem);
      case 6: return (int)launch_rp<2, 6>(p, num_sms, s, use, smem);
      case 10: return (int)launch_rp<2, 10>(p, num_sms, s, use, smem);
      case 15: return (int)launch_rp<2, 15>(p, num_sms, s, use, smem);
    }
  } else {
    switch (p.ns) {
      case 4: return (int)launch_rp<3, 4>(p, num_sms, s, use, smem);
      case 10: return (int)launch_rp<3, 10>(p, num_sms, s, use, smem);
    }
  }
  why = "no compiled Burgers-residual instance for this degree";
  return (int)cudaErrorInvalidValue;
}

}  // namespace coffee
