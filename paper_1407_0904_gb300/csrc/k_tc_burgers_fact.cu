// tcgen05 assembly of the Burgers Jacobian in factored form (Listing 2's problem, degree k),
// for component blocks of at most 128 entries (triangles P1-P3, tetrahedra P1-P2).
//
// The d x d component blocks of the element matrix (k_tc_burgers.cu) are
//   block(ci, cj) = sum_{r,a} u[r][ci] P[a][cj] T1[r,a] + [ci == cj] C,
//   C = sum_{r,a} Q[r][a] T2[r,a] + nu sum_p H_p T3[p],   Q[r][a] = sum_c u[r][c] P[a][c],
// with P = |det J| K. The first sum factors through the direction a:
//   block(ci, cj) = sum_a P[a][cj] V_a^ci + [ci == cj] C,   V_a^ci = sum_r u[r][ci] T1[r,a],
// so the tensor cores contract T1 against u alone (K = ns per direction and component: d*d
// small contractions sharing d operands) and C once per cell, and the epilogue applies P (d
// FMAs per entry). Against contracting every block over [T1 | T2 | T3] this forms about a
// quarter of the factor columns per cell and issues a third fewer MMAs.
//
// Tiles of 64 cells (MMA N = 64, outputs on the TMEM lanes). One tile occupies one of two TMEM
// regions of 256 columns: C at column 0, V_a^ci at 64 (1 + a) for the component ci of the current
// round. A tile takes d rounds (one per block row ci); C is formed in round 0 and kept. The MMA
// interleaves the rounds of two consecutive tiles (regions 0 and 1), and each region has its own
// group of four epilogue warps (warps 0-3 and 8-11), so one region's epilogue overlaps the
// other's MMAs. Producers: warps 4-7, two groups of two warps on alternate tiles, one cell per
// thread; a stage holds a tile's u operand (the d components at a 16-byte aligned column stride,
// so one descriptor per component), its C operand (Q, H) and P (for the epilogue), and is freed
// by the epilogue after the tile's last round.
// Exact forms: where every T1 entry of a direction is an integer times one scale s_a, the V
// operand is held exactly in one part and s_a is folded into P; where every column of [T2 | T3]
// is an integer vector times a scale, that operand is one part and the producers scale Q and H.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstring>
#include <cmath>
#include <vector>
#include "coffee_internal.h"
#include "tc_common.cuh"
#include "k_tc_burgers.cuh"

namespace coffee {
namespace {
using namespace tc;

constexpr int FBN = 64;                    // cells per tile
constexpr int FREGION = 256;               // TMEM columns per region
constexpr int FEPI1 = 8;                   // first warp of the second epilogue group
constexpr int FPROD0 = 4, FPROD_WARPS = 4; // producer warps 4-7, two groups of two

__host__ __device__ constexpr int f_kstep(int prec) { return prec == PREC_TF32 || prec == PREC_TF32X3 ? 8 : 16; }
__host__ __device__ constexpr int f_elem(int prec) { return prec == PREC_TF32 || prec == PREC_TF32X3 ? 4 : 2; }

template <int D, int NS, int PREC>
struct FactShape {
  static constexpr int KSTEP = f_kstep(PREC), ELEM = f_elem(PREC);
  static constexpr int P = D * (D + 1) / 2;
  static constexpr int K1 = NS * D;
  static constexpr int NBLK = NS * NS;
  static constexpr int KV = round_up(NS, KSTEP);                  // V contraction: over the nodes r
  static constexpr int CS = round_up(NS, 16 / ELEM);              // column stride of the u components
  static constexpr int KU = round_up((D - 1) * CS + KV, KSTEP);   // u operand columns
  static constexpr int KC = round_up(K1 + P, KSTEP);              // C contraction: T2 | T3
  static constexpr int VB = KV * ELEM, UB = KU * ELEM, CB = KC * ELEM;  // row bytes
  static constexpr int GP = PrecTraits<PREC>::GPARTS;
  // parts of u: as the factors, except that plain BF16 keeps u in two parts (its V contraction
  // then carries only T1's rounding, as the block form's T operand does)
  static constexpr int GU = PREC == PREC_BF16 ? 2 : GP;
  static constexpr int PW = round_up(D * D, 4);  // P floats per cell (16-byte rows)
  static constexpr int USTAGE = GU * FBN * UB, CSTAGE = GP * FBN * CB, PSTAGE = PW * FBN * 4;
  static constexpr int STAGE = USTAGE + CSTAGE + PSTAGE;
  static_assert(NBLK <= 128, "factored Burgers kernel: blocks of at most 128 entries");
  static_assert((CS * ELEM) % 16 == 0 && STAGE % 128 == 0, "operand alignment");
};

// Products (part of T, part of u) of the V contraction, smallest first: with T1 exact (one part)
// every part of u; otherwise the products of order <= 1 (two-part operands) or <= 2 (BF16X3).
template <int PREC>
struct VPasses {
  static constexpr int GU = PREC == PREC_BF16 ? 2 : prec_gparts(PREC);
  __host__ __device__ static constexpr int n(bool vx) {
    return vx ? GU : (PREC == PREC_TF32 ? 1 : PREC == PREC_BF16X3 ? 6 : 3);
  }
  __host__ __device__ static constexpr int t(bool vx, int i) {
    return vx ? 0 : PREC == PREC_BF16X3 ? Passes<PREC>::t(i) : (i == 1 ? 1 : 0);
  }
  __host__ __device__ static constexpr int g(bool vx, int i) {
    return vx ? GU - 1 - i : PREC == PREC_BF16X3 ? Passes<PREC>::g(i) : (PREC == PREC_TF32 ? 0 : (i == 0 ? 1 : 0));
  }
};

// One operand row of NCOLS columns whose k-th value is f(k), in NP parts of the operand type
// (part q at base + q * part_bytes), stored 16 bytes at a time in the canonical layout.
template <bool TF32, int NP, int NCOLS, class F>
__device__ __forceinline__ void store_row_parts(uint8_t* base, int part_bytes, int r, int kbytes, F f) {
  constexpr int PER = TF32 ? 4 : 8;
#pragma unroll
  for (int c = 0; c < NCOLS / PER; ++c) {
    float x[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) x[q] = f(c * PER + q);
    store_unit<TF32, NP>(base + canon_off(r, c * 16, kbytes), part_bytes, x);
  }
}

// image bytes (V, C, scales) for vparts / cparts parts
template <int D, int NS, int PREC>
__host__ __device__ constexpr int f_image_bytes(int vparts, int cparts) {
  using S = FactShape<D, NS, PREC>;
  return D * vparts * BM * S::VB + cparts * BM * S::CB + round_up(4 * (4 + S::KC), 16);
}

template <int D, int NS, int PREC>
__global__ void __launch_bounds__(NTHREADS, 1) k_burgers_fact_tc(const TcParams p, int nstages) {
  using S = FactShape<D, NS, PREC>;
  using PT = PrecTraits<PREC>;
  using PN = Passes<PREC, false>;
  using PX = Passes<PREC, true>;
  using VP = VPasses<PREC>;
  constexpr int NV = D + 1, P = S::P, K1 = S::K1, NDOF = D * NS;
  constexpr uint32_t IDESC = make_idesc(PT::tf32 ? 2 : 1, BM, FBN);

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int vparts = p.aux_vparts, cparts = p.aux_cparts;
  const int img_bytes = f_image_bytes<D, NS, PREC>(vparts, cparts);
  uint8_t* sV = smem;                                    // [a][part][128 x VB]
  uint8_t* sC = sV + D * vparts * BM * S::VB;            // [part][128 x CB]
  const float* scl = reinterpret_cast<const float*>(sC + cparts * BM * S::CB);  // s_a [4], column scales [KC]
  uint8_t* stages = smem + round_up(img_bytes, 1024);
  Barriers* bars = reinterpret_cast<Barriers*>(stages + nstages * S::STAGE);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (p.ncells + FBN - 1) / FBN;
  const float nu = (float)p.nu;

  if (threadIdx.x == 0) {
    for (int s = 0; s < nstages; ++s) {
      mbar_init(smem_u32(&bars->full[s]), 64);         // the 64 producer threads of a group
      mbar_init(smem_u32(&bars->empty[s]), EPI_WARPS); // the tile's epilogue group, after its last round
    }
    for (int r = 0; r < 2; ++r) {
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
    const uint4* src = reinterpret_cast<const uint4*>(p.image + p.aux_off);
    uint4* dst = reinterpret_cast<uint4*>(sV);
    for (int i = threadIdx.x; i < img_bytes / 16; i += NTHREADS) dst[i] = __ldg(src + i);
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;
  const int spg = nstages / 2;  // stages per producer group

  if (warp >= FPROD0 && warp < FPROD0 + FPROD_WARPS) {
    // ---------------- producers: one cell per thread; group g takes the CTA's tiles g, g + 2, .. ----------------
    const int pw = warp - FPROD0;
    const int grp = pw >> 1, row = ((pw & 1) << 5) + lane;
    const int64_t tstep = 2 * (int64_t)gridDim.x;
    int nvid[NV], ndid[NS];  // index rows one tile ahead
    {
      const int64_t e0 = (blockIdx.x + (int64_t)grp * gridDim.x) * FBN + row;
#pragma unroll
      for (int v = 0; v < NV; ++v) nvid[v] = e0 < p.ncells ? __ldg(p.c2v + e0 * NV + v) : 0;
#pragma unroll
      for (int r = 0; r < NS; ++r) ndid[r] = e0 < p.ncells ? __ldg(p.c2d + e0 * NS + r) : 0;
    }
    int64_t li = 0;
    for (int64_t t = blockIdx.x + (int64_t)grp * gridDim.x; t < ntiles; t += tstep, ++li) {
      const int64_t e = t * FBN + row;
      int vid[NV], did[NS];
#pragma unroll
      for (int v = 0; v < NV; ++v) vid[v] = nvid[v];
#pragma unroll
      for (int r = 0; r < NS; ++r) did[r] = ndid[r];
      {
        const int64_t en = e + tstep * FBN;
#pragma unroll
        for (int v = 0; v < NV; ++v) nvid[v] = en < p.ncells ? __ldg(p.c2v + en * NV + v) : 0;
#pragma unroll
        for (int r = 0; r < NS; ++r) ndid[r] = en < p.ncells ? __ldg(p.c2d + en * NS + r) : 0;
      }
      const int s = grp + 2 * (int)(li % spg);
      const uint32_t use = (uint32_t)(li / spg);
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
              float acc = 0.f;
#pragma unroll
              for (int r = 0; r < D; ++r) acc = fmaf(adj[a][r], adj[b][r], acc);
              H[q++] = nu * acc * inv;
            }
        }
      }
      uint8_t* st = stages + (size_t)s * S::STAGE;
      // u operand: component c at columns c*CS .. c*CS + NS - 1
      auto fu = [&](int k) -> float {
        const int c = k / S::CS, r = k - c * S::CS;
        return (live && c < D && r < NS) ? u[r][c] : 0.f;
      };
      store_row_parts<PT::tf32, S::GU, S::KU>(st, FBN * S::UB, row, S::UB, fu);
      // C operand: Q[r][a] (k = r D + a), then nu H, times the column scales of an exact image
      auto fc = [&](int k) -> float {
        if (!live) return 0.f;
        float v = 0.f;
        if (k < K1) {
          const int r = k / D, a = k % D;
#pragma unroll
          for (int c = 0; c < D; ++c) v = fmaf(u[r][c], Pm[a][c], v);
        } else if (k < K1 + P) {
          v = H[k - K1];
        }
        return v * scl[4 + k];
      };
      store_operand_fn<PREC, S::KC, decltype(fc)>(st + S::USTAGE, FBN * S::CB, row, S::CB, fc);
      // P for the epilogue, with the direction scales of an exact T1 folded in: one 16-byte
      // aligned row of PW floats per cell, read by the epilogue with vector loads
      {
        float4* pp = reinterpret_cast<float4*>(st + S::USTAGE + S::CSTAGE) + row * (S::PW / 4);
        float pr[S::PW];
#pragma unroll
        for (int x = 0; x < S::PW; ++x) pr[x] = 0.f;
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int c = 0; c < D; ++c) pr[a * D + c] = live ? Pm[a][c] * scl[a] : 0.f;
#pragma unroll
        for (int x = 0; x < S::PW / 4; ++x) pp[x] = make_float4(pr[4 * x], pr[4 * x + 1], pr[4 * x + 2], pr[4 * x + 3]);
      }
      fence_proxy_async();
      mbar_arrive(smem_u32(&bars->full[s]));
    }
  } else if (warp == MMA_WARP) {
    // ---------------- MMA issuer: the rounds of two consecutive tiles interleaved ----------------
    if (lane == 0) {
      const uint32_t sv = smem_u32(sV), sc = smem_u32(sC), s0 = smem_u32(stages);
      const uint32_t sbo_v = 8u * S::VB, sbo_c = 8u * S::CB, sbo_u = 8u * S::UB;
      const bool vx = vparts == 1, cx = cparts == 1;
      const int nv = VP::n(vx), nc = cx ? PX::N : PN::N;
      uint32_t rr[2] = {0, 0};  // rounds issued per region
      bool ok = true;
      for (int64_t tl0 = 0; ok; tl0 += 2) {
        const int64_t t0 = blockIdx.x + tl0 * gridDim.x;
        if (t0 >= ntiles) break;
        const int npair = (t0 + gridDim.x < ntiles) ? 2 : 1;
        int st[2];
        for (int e = 0; e < npair && ok; ++e) {
          const int64_t li = tl0 / 2;  // the tile's index in its producer group
          st[e] = e + 2 * (int)(li % spg);
          if (!mbar_wait(smem_u32(&bars->full[st[e]]), (uint32_t)(li / spg) & 1u, p.err)) ok = false;
        }
        if (!ok) break;
        for (int ci = 0; ci < D && ok; ++ci)
          for (int e = 0; e < npair && ok; ++e) {
            if (!mbar_wait(smem_u32(&bars->tempty[e]), (rr[e] & 1u) ^ 1u, p.err)) { ok = false; break; }
            tc_fence_after();
            const uint32_t dbase = tmem + (uint32_t)(e * FREGION);
            const uint32_t bst = s0 + (uint32_t)(st[e] * S::STAGE);
            if (ci == 0) {  // C, kept in the region for the tile's other rounds
              uint32_t acc = 0;
              for (int ks = 0; ks < S::KC / S::KSTEP; ++ks) {
                const uint32_t ko = (uint32_t)ks * 256u;
                for (int i = 0; i < nc; ++i) {
                  const int tp = cx ? PX::t(i) : PN::t(i), gp = cx ? PX::g(i) : PN::g(i);
                  mma<PT::tf32>(dbase, make_desc(sc + (uint32_t)(tp * BM * S::CB) + ko, sbo_c),
                                make_desc(bst + S::USTAGE + (uint32_t)(gp * FBN * S::CB) + ko, sbo_c), IDESC, acc);
                  acc = 1;
                }
              }
            }
            for (int a = 0; a < D; ++a) {  // V_a of component ci
              uint32_t acc = 0;
              for (int ks = 0; ks < S::KV / S::KSTEP; ++ks) {
                const uint32_t ko = (uint32_t)ks * 256u;
                const uint32_t uoff = (uint32_t)(ci * S::CS * S::ELEM / 16) * 128u + ko;
                for (int i = 0; i < nv; ++i) {
                  const int tp = VP::t(vx, i), gp = VP::g(vx, i);
                  mma<PT::tf32>(dbase + (uint32_t)(64 * (1 + a)),
                                make_desc(sv + (uint32_t)((a * vparts + tp) * BM * S::VB) + ko, sbo_v),
                                make_desc(bst + (uint32_t)(gp * FBN * S::UB) + uoff, sbo_u), IDESC, acc);
                  acc = 1;
                }
              }
            }
            tc_commit(smem_u32(&bars->tfull[e]));
            ++rr[e];
          }
      }
      tc_commit(smem_u32(&bars->done));
      mbar_wait(smem_u32(&bars->done), 0, p.err);
    }
    __syncwarp();
  } else if (warp < EPI_WARPS || (warp >= FEPI1 && warp < FEPI1 + EPI_WARPS)) {
    // ---------------- epilogue group e: the CTA's tiles e, e + 2, ..; block row ci per round ----------------
    const int eg = warp < EPI_WARPS ? 0 : 1;
    const int q = warp & 3;  // TMEM lane quadrant
    const int o = q * 32 + lane;  // entry (i, j) of a block
    const int i = o / NS, j = o - (o / NS) * NS;
    uint32_t rr = 0;
    bool ok = true;
    int64_t li = 0;
    for (int64_t t = blockIdx.x + (int64_t)eg * gridDim.x; t < ntiles && ok; t += 2 * (int64_t)gridDim.x, ++li) {
      const int s = eg + 2 * (int)(li % spg);
      const float4* pp = reinterpret_cast<const float4*>(stages + (size_t)s * S::STAGE + S::USTAGE + S::CSTAGE);
      for (int ci = 0; ci < D && ok; ++ci, ++rr) {
        if (!mbar_wait(smem_u32(&bars->tfull[eg]), rr & 1u, p.err)) { ok = false; break; }
        tc_fence_after();
        if (q * 32 < S::NBLK) {  // warp-uniform
          for (int c0 = 0; c0 < FBN; c0 += 16) {
            const int64_t cbase = t * FBN + c0;
            if (cbase >= p.ncells) break;
            const int64_t rem = p.ncells - cbase;
            const int ncol = rem < 16 ? (int)rem : 16;
            const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(eg * FREGION) + c0;
            uint32_t vc[16], vv[D][16];
            tmem_ld16(ta, vc);
#pragma unroll
            for (int a = 0; a < D; ++a) tmem_ld16(ta + (uint32_t)(64 * (1 + a)), vv[a]);
            tmem_wait_ld();
            if (o < S::NBLK) {
              float* rowp = p.out + cbase * p.N + (int64_t)(ci * NS + i) * NDOF + j;
#pragma unroll
              for (int jj = 0; jj < 16; ++jj, rowp += p.N)
                if (jj < ncol) {
                  float pc[S::PW];  // P of the cell (a broadcast read: every lane reads the same row)
#pragma unroll
                  for (int x = 0; x < S::PW / 4; ++x) {
                    const float4 w = pp[(c0 + jj) * (S::PW / 4) + x];
                    pc[4 * x] = w.x, pc[4 * x + 1] = w.y, pc[4 * x + 2] = w.z, pc[4 * x + 3] = w.w;
                  }
#pragma unroll
                  for (int cj = 0; cj < D; ++cj) {
                    float v = cj == ci ? __uint_as_float(vc[jj]) : 0.f;
#pragma unroll
                    for (int a = 0; a < D; ++a) v = fmaf(pc[a * D + cj], __uint_as_float(vv[a][jj]), v);
                    __stcs(rowp + cj * NS, v);
                  }
                }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bars->tempty[eg]));
      }
      // the tile's stage (its operands and P) is free once its last round is read
      __syncwarp();
      if (ok && lane == 0) mbar_arrive(smem_u32(&bars->empty[s]));
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

// shape parameters without the template (host)
struct FGeom {
  int d, ns, kstep, elem, KV, CS, KU, KC, gp, tp, stage, vb, cb;
};
bool fgeom(int degree, int cell, int prec, FGeom& g) {
  if (prec == PREC_FP64 || prec < 0 || prec > PREC_BF16X3) return false;
  if (cell == CELL_TRI ? (degree < 1 || degree > 3) : (cell != CELL_TET || degree < 1 || degree > 2)) return false;
  g.d = cell == CELL_TRI ? 2 : 3;
  g.ns = nnodes(cell, degree);
  g.kstep = f_kstep(prec);
  g.elem = f_elem(prec);
  const int P = g.d * (g.d + 1) / 2;
  g.KV = round_up(g.ns, g.kstep);
  g.CS = round_up(g.ns, 16 / g.elem);
  g.KU = round_up((g.d - 1) * g.CS + g.KV, g.kstep);
  g.KC = round_up(g.ns * g.d + P, g.kstep);
  g.gp = prec_gparts(prec);
  g.tp = prec_tparts(prec);
  g.vb = g.KV * g.elem;
  g.cb = g.KC * g.elem;
  const int gu = prec == PREC_BF16 ? 2 : g.gp;
  g.stage = gu * 64 * g.KU * g.elem + g.gp * 64 * g.cb + round_up(g.d * g.d, 4) * 64 * 4;
  return g.ns * g.ns <= 128;
}
int f_img_bytes(const FGeom& g, int vparts, int cparts) {
  return g.d * vparts * BM * g.vb + cparts * BM * g.cb + round_up(4 * (4 + g.KC), 16);
}
int f_smem(const FGeom& g, int vparts, int cparts, int nst) {
  return round_up(f_img_bytes(g, vparts, cparts), 1024) + nst * g.stage + (int)sizeof(Barriers) + 1024 + 64;
}
int f_stages(const FGeom& g, int vparts, int cparts) {
  for (int s : {4, 2})
    if (f_smem(g, vparts, cparts, s) <= 227 * 1024) return s;
  return 0;
}

template <int D, int NS, int PREC>
cudaError_t launch_f(const TcParams& p, int num_sms, cudaStream_t s, int nst, int smem) {
  auto kern = k_burgers_fact_tc<D, NS, PREC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (p.ncells + FBN - 1) / FBN;
  const int64_t pairs = (ntiles + 1) / 2;
  const int grid = (int)(pairs < num_sms ? pairs : num_sms);
  kern<<<grid, NTHREADS, smem, s>>>(p, nst);
  return cudaGetLastError();
}

template <int D, int NS>
cudaError_t launch_fp(const TcParams& p, int num_sms, cudaStream_t s, int nst, int smem) {
  switch (p.precision) {
    case PREC_TF32: return launch_f<D, NS, PREC_TF32>(p, num_sms, s, nst, smem);
    case PREC_TF32X3: return launch_f<D, NS, PREC_TF32X3>(p, num_sms, s, nst, smem);
    case PREC_BF16: return launch_f<D, NS, PREC_BF16>(p, num_sms, s, nst, smem);
    case PREC_BF16X3: return launch_f<D, NS, PREC_BF16X3>(p, num_sms, s, nst, smem);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

int burgers_fact_supported(int degree, int cell, int precision) {
  FGeom g;
  if (!fgeom(degree, cell, precision, g)) return 0;
  return f_stages(g, g.tp, g.tp) > 0 ? 1 : 0;  // the split (non-exact) images, the larger ones
}

// Where the factored form is the default (measured against the block form on 2^20 P2 tets,
// 1,572,864 P1 tets, 2^21 P2 and 2^20 P3 triangles): tetrahedra P2 (TF32X3 0.958 vs 0.984 ms,
// BF16X3 0.966 vs 1.136). Smaller blocks leave most epilogue lanes idle while each cell still
// costs the epilogue its P loads and FMAs: P1 tets 1.12 vs 0.98 ms, triangles P2 0.67 vs 0.52,
// P3 0.44 vs 0.33 (TF32X3), so they keep the block form unless it is asked for.
int burgers_fact_default(int degree, int cell) { return cell == CELL_TET && degree == 2 ? 1 : 0; }

// The factored-form image, [V: a][part][128 x VB], [C: part][128 x CB], then float scales
// s_a [4] and the C column scales [KC]. V column r of direction a is the T1 row r d + a of the
// Burgers reference tensor; C column k is its T2 row (k < d ns) or T3 row (the next P).
void build_burgers_fact_image(int degree, int cell, int prec, std::vector<uint8_t>& img, int& vparts, int& cparts) {
  FGeom g;
  fgeom(degree, cell, prec, g);
  std::vector<double> T;
  reference_tensor(FORM_BURGERS, degree, cell, T);
  const bool tf32 = g.elem == 4;
  const int nb = g.ns * g.ns, K1 = g.ns * g.d, P = g.d * (g.d + 1) / 2;
  // V: one scale per direction over all its columns
  std::vector<double> vscale(4, 1.0);
  std::vector<std::vector<double>> vint(g.d);
  bool vx = true;
  for (int a = 0; a < g.d && vx; ++a) {
    std::vector<double> all((size_t)g.ns * nb);
    for (int r = 0; r < g.ns; ++r)
      for (int o = 0; o < nb; ++o) all[(size_t)r * nb + o] = T[(size_t)(r * g.d + a) * nb + o];
    vx = integer_column(all, tf32, vscale[a], vint[a]);
  }
  if (!vx) std::fill(vscale.begin(), vscale.end(), 1.0);
  // C: a scale per column
  std::vector<double> cscale(g.KC, 1.0);
  std::vector<std::vector<double>> cint(g.KC);
  bool cx = true;
  for (int k = 0; k < g.KC && cx; ++k) {
    std::vector<double> col(nb, 0.0);
    if (k < K1 + P)
      for (int o = 0; o < nb; ++o) col[o] = T[(size_t)(K1 + k) * nb + o];
    cx = integer_column(col, tf32, cscale[k], cint[k]);
  }
  if (!cx) std::fill(cscale.begin(), cscale.end(), 1.0);
  vparts = vx ? 1 : g.tp;
  cparts = cx ? 1 : g.tp;
  img.assign((size_t)f_img_bytes(g, vparts, cparts), 0);
  const int64_t vtile = (int64_t)BM * g.vb, ctile = (int64_t)BM * g.cb;
  for (int a = 0; a < g.d; ++a)
    for (int r = 0; r < BM; ++r)
      for (int k = 0; k < g.KV; ++k) {
        double x = 0.0;
        if (r < nb && k < g.ns) x = vx ? vint[a][(size_t)k * nb + r] : T[(size_t)(k * g.d + a) * nb + r];
        host_store_parts(img.data() + (size_t)(a * vparts) * vtile, (size_t)vtile, canon_off(r, k * g.elem, g.vb), x,
                         tf32, vparts);
      }
  uint8_t* cbase = img.data() + (size_t)g.d * vparts * vtile;
  for (int r = 0; r < BM; ++r)
    for (int k = 0; k < g.KC; ++k) {
      double x = 0.0;
      if (r < nb && k < K1 + P) x = cx ? cint[k][r] : T[(size_t)(K1 + k) * nb + r];
      host_store_parts(cbase, (size_t)ctile, canon_off(r, k * g.elem, g.cb), x, tf32, cparts);
    }
  float* sc = reinterpret_cast<float*>(cbase + cparts * ctile);
  for (int a = 0; a < 4; ++a) sc[a] = (float)vscale[a];
  for (int k = 0; k < g.KC; ++k) sc[4 + k] = (float)cscale[k];
}

int launch_burgers_fact_tc(int cell, const TcParams& p, int num_sms, void* stream, std::string& why) {
  if (p.ncells == 0) return (int)cudaSuccess;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int degree = 0;
  for (int k = 1; k <= 4; ++k)
    if (nnodes(cell, k) == p.ns) degree = k;
  FGeom g;
  if (p.aux_off == 0 || !fgeom(degree, cell, p.precision, g)) {
    why = "no factored-form image for this shape";
    return (int)cudaErrorInvalidValue;
  }
  int nst = f_stages(g, p.aux_vparts, p.aux_cparts);
  if (nst == 0) {
    why = "operands do not fit in shared memory";
    return (int)cudaErrorInvalidValue;
  }
  if (nst > 2 && (p.tune & TUNE_TWO_STAGES)) nst = 2;
  int smem = f_smem(g, p.aux_vparts, p.aux_cparts, nst);
  if (smem < SMEM_ONE_CTA) smem = SMEM_ONE_CTA;
  if (cell == CELL_TRI) {
    switch (p.ns) {
      case 3: return (int)launch_fp<2, 3>(p, num_sms, s, nst, smem);
      case 6: return (int)launch_fp<2, 6>(p, num_sms, s, nst, smem);
      case 10: return (int)launch_fp<2, 10>(p, num_sms, s, nst, smem);
    }
  } else {
    switch (p.ns) {
      case 4: return (int)launch_fp<3, 4>(p, num_sms, s, nst, smem);
      case 10: return (int)launch_fp<3, 10>(p, num_sms, s, nst, smem);
    }
  }
  why = "no compiled factored Burgers instance for this degree";
  return (int)cudaErrorInvalidValue;
}

}  // namespace coffee
