// tcgen05 local assembly of the Burgers Jacobian (vector degree-k Lagrange, Listing 2's
// problem generalised to degree k).
//
// The element matrix has d x d component blocks (ci, cj) of ns x ns entries. With
// P = |det J| K = sign(det) adj and Q[r][a] = sum_c u[r][c] P[a][c], every block is a
// contraction against fixed reference tensors:
//   block(ci,cj) = sum_{r,a} u[r][ci] P[a][cj] T1[r,a]
//                + [ci==cj] ( sum_{r,a} Q[r][a] T2[r,a] + nu sum_p H_p T3[p] )
// where T1 = int d_a phi_r phi_i phi_j, T2 = int phi_r phi_i d_a phi_j and T3 the
// stiffness pair tensors. One shared-memory A operand [T1 | T2 | T3]^T (rows = block
// entries) serves every block: off-diagonal blocks contract over its T1 columns only,
// diagonal blocks over all of them. Producers build one block's factors per operand
// stage (the per-block B operand), so the operand stages stay the size of one block.
// Pipeline roles, TMEM ring and bounded waits are those of k_tc.cu.
//
// Exact A (AX): where every column k of A is an integer vector n_k times a scale c_k with
// integers the operand type holds exactly (tf32: odd part < 2^11, bf16: < 2^8), A is stored
// once as the integers and the producers multiply factor k by c_k. The split precisions then
// need one pass per part of the factors (Passes<PREC, true>) instead of one per product of
// parts, and A takes one part of shared memory.
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

template <int D, int NS, int PREC, bool AX>
__global__ void __launch_bounds__(NTHREADS, 1) k_burgers_tc(const TcParams p, int nstages) {
  using S = BurgersShape<D, NS, PREC>;
  using PT = PrecTraits<PREC>;
  constexpr int NV = D + 1, P = S::P, KA1 = S::KA1, KD = S::KD, GPARTS = S::GPARTS;
  constexpr int APARTS = AX ? 1 : PT::TPARTS;  // parts of the resident A operand
  using PS = Passes<PREC, AX>;
  static_assert(KD * 4 <= SCALE_BYTES, "column scales exceed their shared-memory slot");
  constexpr int NB = D * D;
  constexpr uint32_t IDESC = make_idesc(PT::tf32 ? 2 : 1, BM, BN);

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int kbytes = p.kbytes;  // = KD * ELEM
  const int tile_bytes = BM * kbytes;
  const int a_bytes = S::MT * APARTS * tile_bytes;
  constexpr int SPART = BN * S::CWB;  // bytes of one part of a chunk stage
  uint8_t* sA = smem;
  uint8_t* sB = smem + a_bytes;
  Barriers* bars = reinterpret_cast<Barriers*>(sB + nstages * GPARTS * SPART);
  float* sc = reinterpret_cast<float*>(bars + 1);  // AX: scale of every A column

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (p.ncells + BN - 1) / BN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < nstages; ++s) {
      mbar_init(smem_u32(&bars->full[s]), 128);
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
    const uint4* src = reinterpret_cast<const uint4*>(p.image);
    uint4* dst = reinterpret_cast<uint4*>(sA);
    for (int i = threadIdx.x; i < a_bytes / 16; i += NTHREADS) dst[i] = __ldg(src + i);
    if constexpr (AX) {
      const float* scg = reinterpret_cast<const float*>(p.image + p.scale_off);
      for (int i = threadIdx.x; i < KD; i += NTHREADS) sc[i] = __ldg(scg + i);
    }
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;

  if (warp >= PROD_WARP0 && warp < MMA_WARP) {
    // ---------------- producers: one cell per thread, one K-chunk of a block per stage ----------------
    const int pw = warp - PROD_WARP0;
    const int grp = pw >> 2, row = ((pw & 3) << 5) + lane;
    const int spg = nstages / PROD_GROUPS;
    bool ok = true;
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
    for (int64_t tl = grp; ok; tl += PROD_GROUPS) {  // local tile number; groups alternate
      const int64_t t = blockIdx.x + tl * gridDim.x;
      if (t >= ntiles) break;
      int64_t li = (tl / PROD_GROUPS) * S::NCHT;  // index among this group's chunks
      const int64_t e = t * BN + row;
      int vid[NV], did[NS];
#pragma unroll
      for (int v = 0; v < NV; ++v) vid[v] = nvid[v];
#pragma unroll
      for (int r = 0; r < NS; ++r) did[r] = ndid[r];
      {
        const int64_t en = e + (int64_t)PROD_GROUPS * gridDim.x * BN;
#pragma unroll
        for (int v = 0; v < NV; ++v) nvid[v] = en < p.ncells ? __ldg(p.c2v + en * NV + v) : 0;
#pragma unroll
        for (int r = 0; r < NS; ++r) ndid[r] = en < p.ncells ? __ldg(p.c2d + en * NS + r) : 0;
      }
      float u[NS][D], Pm[D][D], H[P];
      bool live = e < p.ncells, bad = false;
      if (live) {
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
          // u's loads first, so that they and the coordinates' share one round trip to memory
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
              float s = 0.f;
#pragma unroll
              for (int r = 0; r < D; ++r) s = fmaf(adj[a][r], adj[b][r], s);
              H[q++] = (float)p.nu * s * inv;
            }
        }
      }
      // blocks and chunks as compile-time indices, so u[.][ci] and P[.][cj] stay in registers
      static_for<NB>([&](auto BLK) -> bool {
        constexpr int blk = decltype(BLK)::value;
        constexpr int ci = blk / D, cj = blk % D;
        constexpr int kblk = ci == cj ? KD : KA1;
        // factors of block (ci, cj): u[r][ci] P[a][cj] (T1 columns); on the diagonal also
        // Q[r][a] = sum_c u[r][c] P[a][c] (T2 columns) and nu H (T3 columns); zero padding
        auto factor = [&](int k) -> float {
          float v = 0.f;
          if (!live) return v;
          if (k < S::K1) v = u[k / D][ci] * Pm[k % D][cj];
          else if (k < KA1) v = 0.f;
          else if (k < KA1 + S::K1) {
            const int r = (k - KA1) / D, a = (k - KA1) % D;
#pragma unroll
            for (int c = 0; c < D; ++c) v = fmaf(u[r][c], Pm[a][c], v);
          } else if (k < KA1 + S::K1 + P) v = H[k - KA1 - S::K1];
          if constexpr (AX) v *= sc[k];
          return v;
        };
        return static_for<(kblk + S::CW - 1) / S::CW>([&](auto CH) -> bool {
          constexpr int ch = decltype(CH)::value;
          int s;
          uint32_t use;
          stage_of(li++, grp, spg, s, use);
          if (!mbar_wait(smem_u32(&bars->empty[s]), (use & 1u) ^ 1u, p.err)) return ok = false;
          store_chunk_fn<PREC, S::CW, S::CWB>(sB + (size_t)s * GPARTS * SPART, SPART, row, kblk - ch * S::CW,
                                      [&](int l) { return factor(ch * S::CW + l); });
          fence_proxy_async();
          mbar_arrive(smem_u32(&bars->full[s]));
          return true;
        });
      });
    }
  } else if (warp == MMA_WARP) {
    // ---------------- MMA issuer ----------------
    // Per block: the MT accumulator slots are taken, every K-chunk of the block is
    // contracted into them as its stage fills, then the slots are handed to the epilogue.
    if (lane == 0) {
      const uint32_t sbo_a = 8u * (uint32_t)kbytes, sbo_b = 8u * S::CWB;
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      uint32_t rc = 0;
      const int spg = nstages / PROD_GROUPS;
      int64_t tl = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tl) {
        const int grp = (int)(tl % PROD_GROUPS);
        int64_t li = (tl / PROD_GROUPS) * S::NCHT;
        for (int blk = 0; blk < NB && ok; ++blk, rc += S::MT) {
          const int kblk = (blk / D) == (blk % D) ? KD : KA1;
          for (int m = 0; m < S::MT && ok; ++m) {
            const uint32_t r = rc + m;
            if (!mbar_wait(smem_u32(&bars->tempty[r % RING]), ((r / RING) & 1u) ^ 1u, p.err)) ok = false;
          }
          if (!ok) break;
          tc_fence_after();
          for (int ch = 0; ch * S::CW < kblk; ++ch, ++li) {
            int s;
            uint32_t use;
            stage_of(li, grp, spg, s, use);
            if (!mbar_wait(smem_u32(&bars->full[s]), use & 1u, p.err)) { ok = false; break; }
            tc_fence_after();
            const int ksteps = (kblk - ch * S::CW < S::CW ? kblk - ch * S::CW : S::CW) / S::KSTEP;
            const uint32_t bstage = b0 + (uint32_t)(s * GPARTS * SPART);
            for (int m = 0; m < S::MT; ++m) {
              const uint32_t d = tmem + ((rc + m) % RING) * BN;
              // K-chunk ch of A: byte column ch * CWB of the row, core matrices 128 bytes apart
              const uint32_t atile = a0 + (uint32_t)(m * APARTS * tile_bytes) + (uint32_t)ch * (S::CWB * 8u);
              uint32_t acc = ch > 0 ? 1u : 0u;
              for (int ks = 0; ks < ksteps; ++ks) {
                const uint32_t ko = (uint32_t)ks * 256u;
#pragma unroll
                for (int i = 0; i < PS::N; ++i) {  // products of parts, smallest first
                  mma<PT::tf32>(d, make_desc(atile + (uint32_t)(PS::t(i) * tile_bytes) + ko, sbo_a),
                                make_desc(bstage + (uint32_t)(PS::g(i) * SPART) + ko, sbo_b), IDESC, acc);
                  acc = 1;
                }
              }
            }
            tc_commit(smem_u32(&bars->empty[s]));
          }
          if (!ok) break;
          for (int m = 0; m < S::MT; ++m) tc_commit(smem_u32(&bars->tfull[(rc + m) % RING]));
        }
      }
      tc_commit(smem_u32(&bars->done));
      mbar_wait(smem_u32(&bars->done), 0, p.err);
    }
    __syncwarp();
  } else if constexpr (S::MT == 1) {
    // ---------------- epilogue: the D blocks of a block-row together ----------------
    // Blocks (ci, 0..D-1) occupy consecutive accumulator slots; writing them together means
    // each output row (ci, i) -- all D*NS columns -- is completed by D back-to-back stores.
    const int q = warp;  // TMEM lane quadrant
    const int ndof = D * NS;
    const int o = q * 32 + lane;  // entry (i, j) of a block
    const int i = o / NS, j = o - (o / NS) * NS;
    uint32_t rc = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      for (int ci = 0; ci < D && ok; ++ci, rc += D) {
        uint32_t slot[D];
#pragma unroll
        for (int cj = 0; cj < D; ++cj) {
          slot[cj] = (rc + cj) % RING;
          if (ok && !mbar_wait(smem_u32(&bars->tfull[slot[cj]]), ((rc + cj) / RING) & 1u, p.err)) ok = false;
        }
        if (!ok) break;
        tc_fence_after();
        if (q * 32 < S::NBLK) {  // warp-uniform
          for (int c0 = 0; c0 < BN; c0 += 16) {
            const int64_t cbase = t * BN + c0;
            if (cbase >= p.ncells) break;
            const int64_t rem = p.ncells - cbase;
            const int ncol = rem < 16 ? (int)rem : 16;
            uint32_t v[D][16];
#pragma unroll
            for (int cj = 0; cj < D; ++cj) tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + slot[cj] * BN + c0, v[cj]);
            tmem_wait_ld();
            if (o < S::NBLK) {
              float* row = p.out + cbase * p.N + (int64_t)(ci * NS + i) * ndof + j;
#pragma unroll
              for (int jj = 0; jj < 16; ++jj, row += p.N)
                if (jj < ncol) {
#pragma unroll
                  for (int cj = 0; cj < D; ++cj) __stcs(row + cj * NS, __uint_as_float(v[cj][jj]));
                }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
#pragma unroll
          for (int cj = 0; cj < D; ++cj) mbar_arrive(smem_u32(&bars->tempty[slot[cj]]));
        }
      }
    }
  } else {
    // ---------------- epilogue ----------------
    const int q = warp;  // TMEM lane quadrant
    const int ndof = D * NS;
    uint32_t rc = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      for (int blk = 0; blk < NB && ok; ++blk) {
        const int ci = blk / D, cj = blk % D;
        for (int m = 0; m < S::MT; ++m, ++rc) {
          const uint32_t slot = rc % RING, round = rc / RING;
          if (!mbar_wait(smem_u32(&bars->tfull[slot]), round & 1u, p.err)) { ok = false; break; }
          tc_fence_after();
          const int o = m * BM + q * 32 + lane;  // entry (i, j) of the block
          for (int half = 0; half < 2; ++half) {
          const int64_t cbase = t * BN + half * 64;
          const int64_t rem = p.ncells - cbase;
          const int ncol = rem <= 0 ? 0 : (rem < 64 ? (int)rem : 64);
          if (m * BM + q * 32 < S::NBLK && ncol > 0) {
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + slot * BN + half * 64;
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

template <int D, int NS, int PREC>
cudaError_t launch_b(const TcParams& p, int num_sms, cudaStream_t s, int nst, int smem) {
  auto kern = p.aexact ? k_burgers_tc<D, NS, PREC, true> : k_burgers_tc<D, NS, PREC, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (p.ncells + BN - 1) / BN;
  const int grid = (int)(ntiles < num_sms ? ntiles : num_sms);
  kern<<<grid, NTHREADS, smem, s>>>(p, nst);
  return cudaGetLastError();
}

template <int D, int NS>
cudaError_t launch_bp(const TcParams& p, int num_sms, cudaStream_t s, int nst, int smem) {
  switch (p.precision) {
    case PREC_TF32: return launch_b<D, NS, PREC_TF32>(p, num_sms, s, nst, smem);
    case PREC_TF32X3: return launch_b<D, NS, PREC_TF32X3>(p, num_sms, s, nst, smem);
    case PREC_BF16: return launch_b<D, NS, PREC_BF16>(p, num_sms, s, nst, smem);
    case PREC_BF16X3: return launch_b<D, NS, PREC_BF16X3>(p, num_sms, s, nst, smem);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

namespace {
// The resident-operand kernel takes the shape (A in the precision's parts: the larger of its two
// layouts); otherwise the streamed kernel (k_tc_burgers_stream.cu) does.
bool burgers_resident(int degree, int cell, int precision) {
  BGeom g;
  return bgeom(degree, cell, precision, g) && cstages(g) > 0;
}
int degree_of(int cell, int ns) {
  for (int k = 1; k <= 4; ++k)
    if (nnodes(cell, k) == ns) return k;
  return 0;
}
}  // namespace

int burgers_tc_supported(int degree, int cell, int precision) {
  if (burgers_resident(degree, cell, precision)) return 1;
  return burgers_stream_supported(degree, cell, precision);
}

// Integer form of one A column: x[o] = n[o] * scale for all o, with integers the operand type
// holds exactly (odd part below 2^11 for tf32, 2^8 for bf16). The smallest multiplier N of
// x / max|x| that lands every entry on an integer (to 1e-9) is taken; the reconstruction
// must then agree with x to 1e-13 of max|x|. False when no such N <= 2^11 exists.
bool integer_column(const std::vector<double>& x, bool tf32, double& scale, std::vector<double>& n) {
  double m = 0.0;
  for (double v : x) m = std::max(m, std::fabs(v));
  n.assign(x.size(), 0.0);
  scale = 1.0;
  if (m == 0.0) return true;
  const int odd_limit = tf32 ? 2048 : 256;
  for (int N = 1; N <= 2048; ++N) {
    bool ok = true;
    for (size_t o = 0; o < x.size() && ok; ++o) {
      const double y = x[o] / m * N;
      const double r = std::nearbyint(y);
      if (std::fabs(y - r) > 1e-9) ok = false;
      long long q = std::llabs((long long)r);
      while (q && !(q & 1)) q >>= 1;
      if (q >= odd_limit) ok = false;
      n[o] = r;
    }
    if (!ok) continue;
    scale = m / N;
    for (size_t o = 0; o < x.size(); ++o)
      if (std::fabs(n[o] * scale - x[o]) > 1e-13 * m) return false;
    return true;
  }
  return false;
}

void build_burgers_image(int degree, int cell, int prec, bool exact_ok, std::vector<uint8_t>& img, TcTable& meta) {
  if (exact_ok && !burgers_resident(degree, cell, prec)) {  // the Jacobian on the streamed kernel
    build_burgers_stream_image(degree, cell, prec, img, meta);
    return;
  }
  BGeom g;
  bgeom(degree, cell, prec, g);
  std::vector<double> T;
  reference_tensor(FORM_BURGERS, degree, cell, T);
  const int d = cell == CELL_TRI ? 2 : 3, P = d * (d + 1) / 2;
  const int nb = g.ns * g.ns;
  const bool tf32 = g.elem == 4;
  const int64_t tile = (int64_t)BM * g.kbytes;
  // column k of A: the reference-tensor row feeding it, or -1 for zero padding
  auto trow_of = [&](int k) {
    if (k < g.K1) return k;
    if (k >= g.KA1 && k < g.KA1 + g.K1) return g.ns * d + (k - g.KA1);
    if (k >= g.KA1 + g.K1 && k < g.KA1 + g.K1 + P) return 2 * g.ns * d + (k - g.KA1 - g.K1);
    return -1;
  };
  // exact form: every column an integer vector times a scale
  std::vector<std::vector<double>> ints(g.KD);
  std::vector<float> scales(g.KD, 1.0f);
  bool exact = exact_ok && g.KD * 4 <= SCALE_BYTES;
  for (int k = 0; k < g.KD && exact; ++k) {
    const int tr = trow_of(k);
    std::vector<double> col(nb, 0.0);
    if (tr >= 0)
      for (int o = 0; o < nb; ++o) col[o] = T[(size_t)tr * nb + o];
    double sc = 1.0;
    exact = integer_column(col, tf32, sc, ints[k]);
    scales[k] = (float)sc;
  }
  const int aparts = exact ? 1 : g.aparts;
  const int64_t a_bytes = (int64_t)g.mtiles * aparts * tile;
  img.assign((size_t)(a_bytes + (exact ? g.KD * 4 : 0)), 0);
  for (int m = 0; m < g.mtiles; ++m)
    for (int r = 0; r < BM; ++r) {
      const int o = m * BM + r;
      for (int k = 0; k < g.KD; ++k) {
        const int tr = trow_of(k);
        const double x = (o >= nb || tr < 0) ? 0.0 : exact ? ints[k][o] : T[(size_t)tr * nb + o];
        const uint32_t off = canon_off(r, k * g.elem, g.kbytes);
        host_store_parts(img.data() + (size_t)(m * aparts) * tile, (size_t)tile, off, x, tf32, aparts);
      }
    }
  if (exact) std::memcpy(img.data() + a_bytes, scales.data(), (size_t)g.KD * 4);
  meta = TcTable{};
  meta.mtiles = g.mtiles;
  meta.kbytes = g.kbytes;
  meta.kelems = g.KD;
  meta.K = g.KA1 + g.K1 + P;
  meta.tparts = aparts;
  meta.ksteps_off = g.KA1 / g.kstep;
  meta.tile_bytes = tile;
  meta.aexact = exact ? 1 : 0;
  meta.scale_off = exact ? a_bytes : 0;
  // the factored-form kernel's operands follow, 1024-byte aligned, where that kernel applies
  if (exact_ok && burgers_fact_supported(degree, cell, prec)) {
    std::vector<uint8_t> aux;
    int vparts = 0, cparts = 0;
    build_burgers_fact_image(degree, cell, prec, aux, vparts, cparts);
    const size_t off = (img.size() + 1023) & ~(size_t)1023;
    img.resize(off + aux.size(), 0);
    std::memcpy(img.data() + off, aux.data(), aux.size());
    meta.aux_off = (int64_t)off;
    meta.aux_vparts = vparts;
    meta.aux_cparts = cparts;
  }
}

int launch_burgers_tc(int cell, const TcParams& p, int num_sms, void* stream, std::string& why) {
  if (p.ncells == 0) return (int)cudaSuccess;
  const int degree = degree_of(cell, p.ns);
  // the factored form where it is the faster one, or where it is asked for
  if (p.aux_off != 0 && !(p.tune & TUNE_BURGERS_BLOCKS) &&
      (burgers_fact_default(degree, cell) || (p.tune & TUNE_BURGERS_FACTORED)))
    return launch_burgers_fact_tc(cell, p, num_sms, stream, why);
  if (!burgers_resident(degree, cell, p.precision)) return launch_burgers_stream_tc(cell, degree, p, num_sms, stream, why);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  BGeom g{};
  g.mtiles = p.mtiles;
  g.gparts = prec_gparts(p.precision);
  g.aparts = p.tparts;
  g.sbytes = p.aexact ? SCALE_BYTES : 0;
  g.kbytes = p.kbytes;
  const int nst = cstages(g);
  if (nst == 0) {
    why = "operands do not fit in shared memory";
    return (int)cudaErrorInvalidValue;
  }
  int smem = g.mtiles * g.aparts * BM * g.kbytes + nst * g.gparts * BN * g.kbytes + (int)sizeof(Barriers) + g.sbytes +
             1024 + 64;
  if (smem < SMEM_ONE_CTA) smem = SMEM_ONE_CTA;
  if (cell == CELL_TRI) {
    switch (p.ns) {
      case 3: return (int)launch_bp<2, 3>(p, num_sms, s, nst, smem);
      case 6: return (int)launch_bp<2, 6>(p, num_sms, s, nst, smem);
      case 10: return (int)launch_bp<2, 10>(p, num_sms, s, nst, smem);
      case 15: return (int)launch_bp<2, 15>(p, num_sms, s, nst, smem);
    }
  } else {
    switch (p.ns) {
      case 4: return (int)launch_bp<3, 4>(p, num_sms, s, nst, smem);
      case 10: return (int)launch_bp<3, 10>(p, num_sms, s, nst, smem);
    }
  }
  why = "no compiled Burgers instance for this degree";
  return (int)cudaErrorInvalidValue;
}

}  // namespace coffee
