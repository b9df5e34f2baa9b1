// tc_perm.cu -- K6: permutation exceedance counts on the tcgen05 tensor cores.
//
// The permutation test motivated in Section IV-A: for permutations pi_k of
// the l samples, r_k(i,j) = z_i . (z_j o pi_k), (z_j o pi_k)[s] =
// z_j[pi_k[s]] (only the second row of a pair is permuted), and
//   counts[J(i,j)] += #{k : |r_k(i,j)| >= |r(i,j)|}       for i < j.
//
// perm_test dispatches to one of three forms with the same counts: the
// transposed form (tc_perm_mn.cu, the default), the shared-memory form
// (tc_perm_smem.cu) and the workspace form here, which also serves where
// the other two do not apply (single CTAs, rows over 256 padded samples).
//
// The workspace form runs two kernels per batch of permutations:
//   k_perm_gather  writes the permuted halves ZP[k][j][s] = Z[j][pi_k[s]]
//                  of every row for the batch into a workspace (checking each
//                  index: an index outside [0, l) is recorded as
//                  PCC_ERR_INVALID_ARG and read as sample 0, never out of
//                  bounds).
//   k_perm_tc      a persistent kernel over work items (chunk of ~192
//                  permutations, 128 x 128 tile of the triangle), chunk-major
//                  and column by column so that concurrent CTAs reuse the
//                  same permuted column panels from L2.  Per item: the A
//                  rows (z_i, hi and lo) are loaded once into shared memory
//                  and stay resident; the unpermuted B rows give r_obs, and
//                  then the B rows of two permutations at a time (from the
//                  workspace, a 3-D TMA map), stacked into one 256-row
//                  operand, give r_k and r_k+1 with one N = 256 MMA per
//                  K step and product (the 3-product split contraction,
//                  into a double-buffered 128 x 256 TMEM accumulator).  At
//                  N = 128 the same work took twice the instructions and
//                  was bound by the MMA issue, not by the operand stream.
//                  The epilogue keeps |r_obs| and 16-bit counts in
//                  registers (thread = row i, 64 columns j, both
//                  permutations of a pass against the same |r_obs|) and
//                  adds the counts to the packed output with one atomic per
//                  pair and item.
// Same roles and bounded waits as the pair kernel (tc_pairs.cu).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdlib.h>

#include "pcc_internal.h"
#include "pcc_ptx.cuh"
#include "pcc_sched.h"
#include "tc_common.cuh"
#include "tc_perm_common.cuh"

namespace pcc {
namespace {

constexpr int kPThreads = 320;
constexpr int64_t kPermChunk = 192;          // permutations per work item

// column-major numbering of the upper triangle of tiles (diagonal in):
// column x holds tiles (0..x, x), F(x) = x(x+1)/2 tiles before it; the
// closed-form root is corrected by exact integer tests as in pcc_sched.h
__device__ __forceinline__ void col_tri_coords(int64_t t, int64_t* y,
                                               int64_t* x) {
  int64_t xx = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  if (xx < 0) xx = 0;
  while (xx > 0 && xx * (xx + 1) / 2 > t) --xx;
  while ((xx + 1) * (xx + 2) / 2 <= t) ++xx;
  *x = xx;
  *y = t - xx * (xx + 1) / 2;
}

struct PermParams {
  int64_t n;
  int64_t m;          // 128-wide tiles per side
  int64_t items;      // tiles (PAIR: tile pairs) * nchunks
  int nchunks;        // permutation chunks per tile
  int chunk;          // permutations per chunk
  int kbatch;         // permutations in this batch (workspace depth)
  int nkb;            // K blocks of 32
  int lolo;           // 1: the fourth product lo.lo (BF16X4)
  const uint8_t* flags;
  uint32_t* counts;
  int* status;
  uint64_t wait_ns;
};

// KP = K per stage: 32 (64-byte swizzle rows) or, in the pair form, 64
// (128-byte rows: half as many copies and stage hand-offs).  PAIR: a CTA
// pair runs one 2-SM MMA (M = 256: the two CTAs' tiles); each CTA holds the
// 128 B rows of one permutation, so its B stages are half as large.
template <bool RESA, bool PAIR, int KP>
struct PCfg {
  static constexpr int kPTile = kPT * KP * 2;  // 128 rows x KP (16-bit)
  // resident A: nkb blocks x (hi + lo) tiles, up to kPMaxResidentK samples
  static constexpr int kABytes =
      RESA ? (kPMaxResidentK / KP) * 2 * kPTile : 0;
  // B hi (or lo) rows of a stage: 256 (two permutations), PAIR: 128 (one)
  static constexpr int kBHalf = PAIR ? kPTile : 2 * kPTile;
  // stage: [B hi | B lo], streamed A in front of them
  static constexpr int kStageBytes =
      RESA ? 2 * kBHalf : 2 * kPTile + 2 * kBHalf;
  static constexpr int kBarBytes = 512;
  static constexpr int kStages =
      (kPSmemBudget - 1024 - kABytes - kBarBytes) / kStageBytes > 8
          ? 8
          : (kPSmemBudget - 1024 - kABytes - kBarBytes) / kStageBytes;
  static constexpr int kSmemBytes =
      1024 + kABytes + kStages * kStageBytes + kBarBytes;
  static_assert(kStages >= 2, "ring too small");
};

// One block per (permutation, group of rows).  The permutation is checked
// and staged in shared memory; with NG > 0 each lane then keeps the indices
// of its NG groups of 8 outputs in registers for all the block's rows (rows
// up to 256 * NG samples).  Each warp takes RR rows at a time and stages
// them in shared memory with hi and lo interleaved (word s = hi[s] |
// lo[s] << 16),
// so one 4-byte read fetches both halves of a sample; every lane then
// writes 8 permuted elements of each half with one 16-byte store per half
// (lpad is a multiple of 64, so rows split into whole 8-element groups).
// Shared memory: 4 * lpad bytes of indices and 4 * lpad per row a warp
// stages (two rows at a time for rows up to 1,024 samples, else one).
constexpr int kGatherWarps = 8;

template <int NG, int RR>
__global__ void __launch_bounds__(kGatherWarps * 32)
    k_perm_gather(const uint16_t* __restrict__ hi,
                  const uint16_t* __restrict__ lo,
                  const int32_t* __restrict__ perms, int64_t n, int64_t l,
                  int64_t lpad, int64_t k_lo, int64_t rows_per_block,
                  uint16_t* __restrict__ ohi, uint16_t* __restrict__ olo,
                  int* __restrict__ status) {
  extern __shared__ uint8_t gsm[];
  int32_t* pi = reinterpret_cast<int32_t*>(gsm);              // lpad
  uint32_t* rows = reinterpret_cast<uint32_t*>(pi + lpad);    // per warp
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t kk = blockIdx.y;
  const int64_t ngroups = lpad / 8;
  const int32_t* src = perms + (k_lo + kk) * l;
  bool bad = false;
  for (int64_t s = threadIdx.x; s < lpad; s += blockDim.x) {
    int32_t v = s < l ? src[s] : -1;
    if (s < l && (v < 0 || v >= l)) {
      bad = true;
      v = 0;
    }
    pi[s] = v;
  }
  if (bad) atomicCAS(status, 0, (int)PCC_ERR_INVALID_ARG);
  __syncthreads();
  // this lane's indices: groups v = lane + 32 g
  int32_t idx[NG > 0 ? 8 * NG : 1];
  if constexpr (NG > 0) {
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const int64_t v = lane + 32 * g;
#pragma unroll
      for (int t = 0; t < 8; ++t)
        idx[8 * g + t] = v < ngroups ? pi[v * 8 + t] : -1;
    }
  }
  // RR rows per warp and iteration (rows j, j + W, ...), staged together so
  // that their loads are in flight at once
  uint32_t* wrow = rows + (size_t)warp * RR * lpad;  // hi | lo << 16
  const int64_t j0 = blockIdx.x * rows_per_block;
  const int64_t j1 = j0 + rows_per_block < n ? j0 + rows_per_block : n;
  for (int64_t j = j0 + warp; j < j1; j += RR * kGatherWarps) {
    for (int64_t v = lane; v < ngroups; v += 32) {
#pragma unroll
      for (int r = 0; r < RR; ++r) {
        const int64_t jr = j + r * kGatherWarps;
        if (jr >= j1) break;
        const uint4 a = reinterpret_cast<const uint4*>(hi + jr * lpad)[v];
        const uint4 b = reinterpret_cast<const uint4*>(lo + jr * lpad)[v];
        uint4 w0, w1;  // samples 8v .. 8v+7, interleaved
        w0.x = (a.x & 0xFFFFu) | (b.x << 16);
        w0.y = (a.x >> 16) | (b.x & 0xFFFF0000u);
        w0.z = (a.y & 0xFFFFu) | (b.y << 16);
        w0.w = (a.y >> 16) | (b.y & 0xFFFF0000u);
        w1.x = (a.z & 0xFFFFu) | (b.z << 16);
        w1.y = (a.z >> 16) | (b.z & 0xFFFF0000u);
        w1.z = (a.w & 0xFFFFu) | (b.w << 16);
        w1.w = (a.w >> 16) | (b.w & 0xFFFF0000u);
        uint4* sw = reinterpret_cast<uint4*>(wrow + r * lpad);
        sw[2 * v] = w0;
        sw[2 * v + 1] = w1;
      }
    }
    __syncwarp();
    auto emit = [&](int64_t v, const int32_t* q) {
#pragma unroll
      for (int r = 0; r < RR; ++r) {
        const int64_t jr = j + r * kGatherWarps;
        if (jr >= j1) break;
        const uint32_t* w = wrow + r * lpad;
        uint32_t wv[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) wv[t] = q[t] >= 0 ? w[q[t]] : 0u;
        uint4 ua, ub;  // hi: low halves, lo: high halves
        ua.x = (wv[0] & 0xFFFFu) | (wv[1] << 16);
        ua.y = (wv[2] & 0xFFFFu) | (wv[3] << 16);
        ua.z = (wv[4] & 0xFFFFu) | (wv[5] << 16);
        ua.w = (wv[6] & 0xFFFFu) | (wv[7] << 16);
        ub.x = (wv[0] >> 16) | (wv[1] & 0xFFFF0000u);
        ub.y = (wv[2] >> 16) | (wv[3] & 0xFFFF0000u);
        ub.z = (wv[4] >> 16) | (wv[5] & 0xFFFF0000u);
        ub.w = (wv[6] >> 16) | (wv[7] & 0xFFFF0000u);
        reinterpret_cast<uint4*>(ohi + (kk * n + jr) * lpad)[v] = ua;
        reinterpret_cast<uint4*>(olo + (kk * n + jr) * lpad)[v] = ub;
      }
    };
    if constexpr (NG > 0) {
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        const int64_t v = lane + 32 * g;
        if (v < ngroups) emit(v, idx + 8 * g);
      }
    } else {
      for (int64_t v = lane; v < ngroups; v += 32) emit(v, pi + v * 8);
    }
    __syncwarp();
  }
}

// the gather for rows of lpad samples: indices in registers up to 1024
cudaError_t launch_gather(dim3 g, size_t gsmem, cudaStream_t s,
                          const uint16_t* hi, const uint16_t* lo,
                          const int32_t* perms, int64_t n, int64_t l,
                          int64_t lpad, int64_t k_lo, int64_t rpb,
                          uint16_t* ohi, uint16_t* olo, int* status) {
  const int64_t need = (lpad / 8 + 31) / 32;
  auto go = [&](auto fn) {
    if (gsmem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(
          fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsmem);
      if (e != cudaSuccess) return e;
    }
    fn<<<g, kGatherWarps * 32, gsmem, s>>>(hi, lo, perms, n, l, lpad, k_lo,
                                            rpb, ohi, olo, status);
    return cudaGetLastError();
  };
  // two rows per warp while their staging stays small (rows up to 1,024)
  if (need <= 1) return go(k_perm_gather<1, 2>);
  if (need <= 2) return go(k_perm_gather<2, 2>);
  if (need <= 4) return go(k_perm_gather<4, 2>);
  return go(k_perm_gather<0, 1>);
}

template <bool BF16, bool RESA, bool PAIR, int KP>
__global__ void __launch_bounds__(kPThreads, 1)
    k_perm_tc(const __grid_constant__ CUtensorMap tz_hi,
              const __grid_constant__ CUtensorMap tz_lo,
              const __grid_constant__ CUtensorMap tp_hi,
              const __grid_constant__ CUtensorMap tp_lo, const PermParams p) {
  using C = PCfg<RESA, PAIR, KP>;
  constexpr int S = C::kStages;
  constexpr int kPTile = C::kPTile;
  // N = 128: r_obs and a lone last permutation; N = 256: two permutations.
  // PAIR: always M = 256 (both CTAs' tiles) and N = 256 (one permutation's
  // 128 B rows from each CTA; r_obs and a lone permutation repeat theirs)
  constexpr uint32_t kIdesc1 =
      PAIR ? make_idesc_f16(BF16, 2 * kPT, 2 * kPT)
           : make_idesc_f16(BF16, kPT, kPT);
  constexpr uint32_t kIdesc2 = make_idesc_f16(BF16, PAIR ? 2 * kPT : kPT,
                                              2 * kPT);

  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned base, kept as an offset from the shared array so
  // that accesses through it compile to shared-memory instructions
  uint8_t* smem =
      smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t* aregion = smem;                 // resident A (RESA)
  uint8_t* ring = smem + C::kABytes;
  uint64_t* bars =
      reinterpret_cast<uint64_t*>(ring + S * C::kStageBytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + S;
  uint64_t* tfull = bars + 2 * S;
  uint64_t* tempty = tfull + 2;
  uint64_t* afull = tempty + 2;
  uint64_t* aempty = afull + 1;
  uint64_t* mdone = aempty + 1;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(mdone + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  // fills of the ring stages and (slot S) of the resident A tile
  FillLog* flog = reinterpret_cast<FillLog*>(bars + 32);
  static_assert(2 * S + 7 <= 31 && S + 1 <= 16, "barrier area");
  static_assert(32 * 8 + sizeof(FillLog) <= C::kBarBytes, "barrier area");

  // stage layout: RESA: [B hi | B lo]; else [A hi | A lo | B hi | B lo];
  // B hi and lo hold 256 rows each: the first permutation's 128 rows, then
  // the second's (or the unpermuted rows alone in the first 128)
  auto sB_hi = [&](int s) {
    return ring + s * C::kStageBytes + (RESA ? 0 : 2 * kPTile);
  };
  auto sB_lo = [&](int s) { return sB_hi(s) + C::kBHalf; };
  auto sA_hi = [&](int s, int kb) {
    return RESA ? aregion + kb * 2 * kPTile : ring + s * C::kStageBytes;
  };
  auto sA_lo = [&](int s, int kb) { return sA_hi(s, kb) + kPTile; };

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      // PAIR: the even CTA's barrier counts both CTAs' epilogue warps
      mbar_init(&tempty[a], PAIR ? 2 * kPEpiWarps : kPEpiWarps);
    }
    mbar_init(afull, 1);
    mbar_init(aempty, 1);
    mbar_init(mdone, 1);
    *abort_flag = 0;
    fill_log_init(flog);
    fence_barrier_init();
  }
  if (warp == 1) {
    if constexpr (PAIR) {
      tmem_alloc_pair(tmem_holder, 512);
      tmem_relinquish_pair();
    } else {
      tmem_alloc(tmem_holder, 512);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // both CTAs' barriers exist before the pair signals across them
  if constexpr (PAIR) cluster_sync();
  const uint32_t tmem_base = *tmem_holder;
  const uint32_t crank = PAIR ? cluster_ctarank() : 0u;
  // PAIR: work items go to clusters; each CTA of a pair takes one tile
  const int64_t wid = PAIR ? (int64_t)(blockIdx.x >> 1) : (int64_t)blockIdx.x;
  const int64_t wstride =
      PAIR ? (int64_t)(gridDim.x >> 1) : (int64_t)gridDim.x;
  WaitCtx w{abort_flag, p.status, p.wait_ns};
  const int64_t n = p.n;

  // items run chunk-major, and inside a chunk the tiles of the triangle go
  // column by column: CTAs working at the same time share the permuted
  // column panels of the same permutations in L2
  const int64_t tiles = PAIR ? col_pairs_before(p.m) : p.m * (p.m + 1) / 2;
  // PAIR: `dummy` marks the missing partner of a column's last, lone tile:
  // it repeats its partner's tile and its counts are dropped
  bool dummy = false;
  auto item_coords = [&](int64_t it, int64_t* row0, int64_t* col0, int* k0,
                         int* klen) {
    const int c = (int)(it / tiles);
    const int64_t t = it % tiles;
    int64_t yt, xt;
    if constexpr (PAIR) {
      int64_t r;
      col_pair_coords(t, &r, &xt);
      yt = 2 * r + (int64_t)crank;
      dummy = yt > xt;
      if (dummy) yt = 2 * r;
    } else {
      col_tri_coords(t, &yt, &xt);
    }
    *row0 = yt * kPT;
    *col0 = xt * kPT;
    *k0 = c * p.chunk;
    const int e = *k0 + p.chunk < p.kbatch ? *k0 + p.chunk : p.kbatch;
    *klen = e - *k0;
  };

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------- TMA producer
      const uint64_t pol = l2_policy_evict_last();
      int stage = 0;
      uint32_t phase = 0;
      uint32_t aph = 0;
      bool ok = true;
      for (int64_t it = wid; it < p.items && ok; it += wstride) {
        int64_t row0, col0;
        int k0, klen;
        item_coords(it, &row0, &col0, &k0, &klen);
        if (klen <= 0) continue;
        if (RESA) {
          if (!mbar_wait(aempty, aph ^ 1u, w)) break;
          flog->fills[S] += 1u;
          flog->bytes[S] = (uint32_t)(p.nkb * 2 * kPTile);
          if constexpr (PAIR) {
            // both CTAs' A tiles count on the even CTA's barrier
            if (crank == 0)
              mbar_arrive_expect_tx(afull, (uint32_t)(2 * p.nkb * 2 * kPTile));
            const uint32_t ab = cluster_addr(afull, 0);
            for (int kb = 0; kb < p.nkb; ++kb) {
              tma_load_2d_pair(sA_hi(0, kb), &tz_hi, ab, kb * KP, (int)row0,
                               pol);
              tma_load_2d_pair(sA_lo(0, kb), &tz_lo, ab, kb * KP, (int)row0,
                               pol);
            }
          } else {
            mbar_arrive_expect_tx(afull, (uint32_t)(p.nkb * 2 * kPTile));
            for (int kb = 0; kb < p.nkb; ++kb) {
              tma_load_2d_hint(sA_hi(0, kb), &tz_hi, afull, kb * KP,
                               (int)row0, pol);
              tma_load_2d_hint(sA_lo(0, kb), &tz_lo, afull, kb * KP,
                               (int)row0, pol);
            }
          }
          aph ^= 1u;
        }
        // pass -1: r_obs; pass q: permutations k0 + 2q and (if any) + 1
        const int npass = (klen + 1) / 2;
        for (int pass = -1; pass < npass && ok; ++pass) {
          const bool two = pass >= 0 && 2 * pass + 1 < klen;
          const uint32_t bytes = (RESA ? 0u : 2u * kPTile) +
                                 (two ? 4u : 2u) * (uint32_t)kPTile;
          for (int kb = 0; kb < p.nkb; ++kb) {
            if (!mbar_wait(&empty[stage], phase ^ 1u, w)) {
              ok = false;
              break;
            }
            const int kc = kb * KP;
            if constexpr (PAIR) {
              // each CTA: (its streamed A and) the 128 B rows of one
              // permutation, the even CTA k, the odd CTA k + 1 (r_obs and a
              // lone permutation: the same rows in both); both CTAs' bytes
              // count on the even CTA's barrier
              const uint32_t per_cta = (RESA ? 0u : 2u * kPTile) + 2u * kPTile;
              if (crank == 0)
                mbar_arrive_expect_tx(&full[stage], 2u * per_cta);
              const uint32_t fb = cluster_addr(&full[stage], 0);
              if (!RESA) {
                tma_load_2d_pair(sA_hi(stage, kb), &tz_hi, fb, kc, (int)row0,
                                 pol);
                tma_load_2d_pair(sA_lo(stage, kb), &tz_lo, fb, kc, (int)row0,
                                 pol);
              }
              if (pass < 0) {
                tma_load_2d_pair(sB_hi(stage), &tz_hi, fb, kc, (int)col0,
                                 pol);
                tma_load_2d_pair(sB_lo(stage), &tz_lo, fb, kc, (int)col0,
                                 pol);
              } else {
                const int kk = k0 + 2 * pass + ((two && crank) ? 1 : 0);
                tma_load_3d_pair(sB_hi(stage), &tp_hi, fb, kc, (int)col0, kk);
                tma_load_3d_pair(sB_lo(stage), &tp_lo, fb, kc, (int)col0, kk);
              }
            } else {
              mbar_arrive_expect_tx(&full[stage], bytes);
              if (!RESA) {
                tma_load_2d_hint(sA_hi(stage, kb), &tz_hi, &full[stage], kc,
                                 (int)row0, pol);
                tma_load_2d_hint(sA_lo(stage, kb), &tz_lo, &full[stage], kc,
                                 (int)row0, pol);
              }
              if (pass < 0) {
                tma_load_2d_hint(sB_hi(stage), &tz_hi, &full[stage], kc,
                                 (int)col0, pol);
                tma_load_2d_hint(sB_lo(stage), &tz_lo, &full[stage], kc,
                                 (int)col0, pol);
              } else {
                const int ka = k0 + 2 * pass;
                tma_load_3d(sB_hi(stage), &tp_hi, &full[stage], kc, (int)col0,
                            ka);
                tma_load_3d(sB_lo(stage), &tp_lo, &full[stage], kc, (int)col0,
                            ka);
                if (two) {
                  tma_load_3d(sB_hi(stage) + kPTile, &tp_hi, &full[stage], kc,
                              (int)col0, ka + 1);
                  tma_load_3d(sB_lo(stage) + kPTile, &tp_lo, &full[stage], kc,
                              (int)col0, ka + 1);
                }
              }
            }
            flog->fills[stage] += 1u;
            flog->bytes[stage] =
                PAIR ? (RESA ? 0u : 2u * kPTile) + 2u * kPTile : bytes;
            if (++stage == S) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && (!PAIR || crank == 0)) {
      // ------------------------------------------------------ MMA issuer
      // (PAIR: the even CTA issues for both)
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t aphase = 0;
      uint32_t aph = 0;
      bool ok = true;
      for (int64_t it = wid; it < p.items && ok; it += wstride) {
        int64_t row0, col0;
        int k0, klen;
        item_coords(it, &row0, &col0, &k0, &klen);
        if (klen <= 0) continue;
        if (RESA) {
          if (!mbar_wait(afull, aph, w)) break;
          aph ^= 1u;
        }
        const int npass = (klen + 1) / 2;
        for (int pass = -1; pass < npass && ok; ++pass) {
          const bool two = pass >= 0 && 2 * pass + 1 < klen;
          const uint32_t idesc = two ? kIdesc2 : kIdesc1;
          if (!mbar_wait(&tempty[acc], aphase ^ 1u, w)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + (uint32_t)(acc * kPAcc);
          for (int kb = 0; kb < p.nkb; ++kb) {
            if (!mbar_wait(&full[stage], phase, w)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t aH = smem_u32(sA_hi(stage, kb));
            const uint32_t aL = smem_u32(sA_lo(stage, kb));
            const uint32_t bH = smem_u32(sB_hi(stage));
            const uint32_t bL = smem_u32(sB_lo(stage));
#pragma unroll
            for (int ks = 0; ks < KP / kPUK; ++ks) {
              const uint32_t off = ks * kPUK * 2;
              const uint64_t dAH = kmajor_desc<2 * KP>(aH + off);
              const uint64_t dBH = kmajor_desc<2 * KP>(bH + off);
              const uint64_t dAL = kmajor_desc<2 * KP>(aL + off);
              const uint64_t dBL = kmajor_desc<2 * KP>(bL + off);
              auto mma = [&](uint64_t a, uint64_t b, uint32_t acc_in) {
                if constexpr (PAIR)
                  umma_f16_pair(d_tmem, a, b, idesc, acc_in);
                else
                  umma_f16(d_tmem, a, b, idesc, acc_in);
              };
              mma(dAH, dBH, (kb | ks) != 0);
              mma(dAH, dBL, 1u);
              mma(dAL, dBH, 1u);
              if (p.lolo) mma(dAL, dBL, 1u);
            }
            if constexpr (PAIR)
              umma_commit_pair(&empty[stage], 3);  // frees it in both CTAs
            else
              umma_commit(&empty[stage]);
            if (++stage == S) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (!ok) break;
          if constexpr (PAIR)
            umma_commit_pair(&tfull[acc], 3);  // each CTA reads its rows
          else
            umma_commit(&tfull[acc]);
          acc ^= 1;
          if (acc == 0) aphase ^= 1u;
        }
        // the resident A tile is free once this item's MMAs complete
        if (RESA && ok) {
          if constexpr (PAIR)
            umma_commit_pair(aempty, 3);
          else
            umma_commit(aempty);
        }
      }
      if constexpr (PAIR)
        umma_commit_pair(mdone, 1);
      else
        umma_commit(mdone);
      WaitCtx wd = w;
      volatile int never = 0;
      wd.abort_flag = &never;
      mbar_wait(mdone, 0, wd);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;          // TMEM lane quarter: rows 32q..32q+31
    const int h = (warp - 2) >> 2;   // columns 64h..64h+63
    int acc = 0;
    uint32_t aphase = 0;
    bool ok = true;
    for (int64_t it = wid; it < p.items && ok; it += wstride) {
      int64_t row0, col0;
      int k0, klen;
      item_coords(it, &row0, &col0, &k0, &klen);
      if (klen <= 0) continue;
      float robs[64];
      uint32_t cnt[32];  // two 16-bit counts per word
#pragma unroll
      for (int t = 0; t < 32; ++t) cnt[t] = 0u;
      const int npass = (klen + 1) / 2;
      for (int pass = -1; pass < npass; ++pass) {
        // permutations in this accumulator: columns [0, 128) and, for a
        // pair, [128, 256); this warp reads columns 64h.. of each
        const int nperm = pass < 0 ? 1 : (2 * pass + 1 < klen ? 2 : 1);
        bool got = true;
        if (lane == 0) got = mbar_wait(&tfull[acc], aphase, w);
        if (!__shfl_sync(0xffffffffu, got ? 1 : 0, 0)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) +
                               (uint32_t)(acc * kPAcc + h * 64);
        for (int e = 0; e < nperm; ++e) {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            uint32_t v[32];
            tmem_ld_32x32b_x32(taddr + (uint32_t)(e * kPT + c * 32), v);
            tmem_ld_wait();
            if (pass < 0) {
#pragma unroll
              for (int t = 0; t < 32; ++t)
                robs[c * 32 + t] = fabsf(__uint_as_float(v[t]));
            } else {
#pragma unroll
              for (int t = 0; t < 32; ++t) {
                const uint32_t hit =
                    fabsf(__uint_as_float(v[t])) >= robs[c * 32 + t] ? 1u
                                                                     : 0u;
                cnt[c * 16 + (t >> 1)] += hit << ((t & 1) * 16);
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if (PAIR && crank != 0)  // released to the even CTA's MMA issuer
            tmem_release_cluster(cluster_addr(&tempty[acc], 0));
          else
            tmem_release(&tempty[acc]);
        }
        acc ^= 1;
        if (acc == 0) aphase ^= 1u;
      }
      if (!ok) break;
      // add this item's counts to the packed output
      const int64_t i = row0 + q * 32 + lane;
      if (!dummy && i < n && p.flags[i] == 0) {
        const int64_t base = pair_row_base(n, i);
#pragma unroll
        for (int t = 0; t < 64; ++t) {
          const int64_t j = col0 + h * 64 + t;
          const uint32_t c = (cnt[t >> 1] >> ((t & 1) * 16)) & 0xFFFFu;
          if (c && j > i && j < n && p.flags[j] == 0)
            atomicAdd(p.counts + base + j, c);
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // every copy issued by this CTA (PAIR: by either CTA) has landed before
  // a CTA of the pair may exit
  drain_ring<PAIR>(full, RESA ? afull : nullptr, flog, S, w, crank);
  if (warp == 1) {
    __syncwarp();
    if constexpr (PAIR)
      tmem_dealloc_pair(tmem_base, 512);
    else
      tmem_dealloc(tmem_base, 512);
  }
}

template <bool BF16, bool RESA, bool PAIR, int KP>
cudaError_t launch_perm_kernel(const pcc_zmat* Z, const CUtensorMap& ph,
                               const CUtensorMap& pl, const PermParams& p,
                               cudaStream_t s) {
  auto fn = k_perm_tc<BF16, RESA, PAIR, KP>;
  const int smem = PCfg<RESA, PAIR, KP>::kSmemBytes;
  // Z's maps with the stage's box: 64 x 128 (128-B swizzle) or 32 x 128
  const CUtensorMap& zh = KP == 64 ? Z->tm_hi : Z->tm_hi32;
  const CUtensorMap& zl = KP == 64 ? Z->tm_lo : Z->tm_lo32;
  cudaError_t e = ensure_func_smem(reinterpret_cast<const void*>(fn), smem);
  if (e != cudaSuccess) return e;
  if constexpr (PAIR) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kPThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    static int max_clusters_of[kDeviceSlots] = {};  // per instance, device
    int& max_clusters = max_clusters_of[device_slot(Z->device)];
    if (max_clusters == 0) {
      cfg.gridDim = dim3(2 * (unsigned)(num_sms(Z->device) / 2), 1, 1);
      int mc = 0;
      if (cudaOccupancyMaxActiveClusters(&mc, fn, &cfg) != cudaSuccess ||
          mc <= 0) {
        cudaGetLastError();
        mc = num_sms(Z->device) / 2;
      }
      max_clusters = mc;
    }
    const int64_t ncl = p.items < max_clusters ? p.items : max_clusters;
    cfg.gridDim = dim3((unsigned)(2 * ncl), 1, 1);
    e = cudaLaunchKernelEx(&cfg, fn, zh, zl, ph, pl, p);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  int64_t grid = num_sms(Z->device);
  if (p.items < grid) grid = p.items;
  fn<<<(unsigned)grid, kPThreads, smem, s>>>(zh, zl, ph, pl, p);
  return cudaGetLastError();
}

size_t perm_ws_budget() {
  static size_t b = [] {
    const char* e = getenv("PCC_PERM_WS_BYTES");
    const long long v = e ? atoll(e) : 0;
    return (size_t)(v > 0 ? v : (4ll << 30));
  }();
  return b;
}

}  // namespace

pcc_status perm_test(pcc_zmat* Z, const int32_t* d_perms, int32_t P,
                     int32_t k0, int32_t k1, uint32_t* d_counts,
                     cudaStream_t s) {
  if (Z->prec != PCC_PREC_BF16X3 && Z->prec != PCC_PREC_FP16X3S &&
      Z->prec != PCC_PREC_BF16X4)
    return PCC_ERR_INVALID_ARG;
  // CTA pairs permute in shared memory where the rows fit: no workspace
  if (perm_smem_applies(Z))
    return perm_test_smem(Z, d_perms, k0, k1, d_counts, s);
  // or copy the permuted operand from a transposed Z
  if (perm_mn_applies(Z)) return perm_test_mn(Z, d_perms, k0, k1, d_counts, s);
  const int64_t n = Z->n, lpad = Z->lpad;
  const size_t per_k = (size_t)n * (size_t)lpad * 2 * 2;  // hi + lo
  int64_t kbmax = (int64_t)(perm_ws_budget() / per_k);
  if (kbmax < 1) kbmax = 1;
  const int64_t total = k1 - k0;
  const int64_t kb_alloc = total < kbmax ? total : kbmax;
  const size_t need = per_k * (size_t)kb_alloc;
  if (Z->perm_ws_bytes < need) {
    if (Z->perm_ws) {
      cudaStreamSynchronize(s);
      cudaFree(Z->perm_ws);
      Z->perm_ws = nullptr;
      Z->perm_ws_bytes = 0;
    }
    if (cudaMalloc(&Z->perm_ws, need) != cudaSuccess) {
      cudaGetLastError();
      return PCC_ERR_OOM;
    }
    Z->perm_ws_bytes = need;
  }
  uint16_t* wh = static_cast<uint16_t*>(Z->perm_ws);
  const bool bf16 = Z->prec != PCC_PREC_FP16X3S;
  const int64_t m = (n + kPT - 1) / kPT;
  // the CTA-pair form takes the tiles of a column two at a time
  const bool pair = tc_tuning().pair_mma != 0 && m >= 2;
  // the pair form follows the stage_k knob; single CTAs keep K = 32 (a
  // 64-sample stage next to the resident A tile leaves room for one stage)
  const int KP = pair && tc_tuning().stage_k == 64 ? 64 : 32;
  const int64_t tiles = pair ? col_pairs_before(m) : m * (m + 1) / 2;
  const int sms = num_sms(Z->device);
  if ((size_t)lpad * 4 + (size_t)kGatherWarps * 4 * lpad > 200 * 1024)
    return PCC_ERR_UNSUPPORTED;  // rows longer than the gather stages
  cudaError_t e = cudaSuccess;
  for (int64_t kb0 = k0; kb0 < k1; kb0 += kb_alloc) {
    const int64_t kbatch = (k1 - kb0) < kb_alloc ? (k1 - kb0) : kb_alloc;
    uint16_t* wl = wh + (size_t)kbatch * (size_t)n * (size_t)lpad;
    // gather the permuted halves of the batch
    const int64_t rpb = 64;
    dim3 g((unsigned)((n + rpb - 1) / rpb), (unsigned)kbatch, 1);
    const size_t rr = lpad <= 1024 ? 2 : 1;  // rows staged per warp
    const size_t gsmem =
        (size_t)lpad * 4 + (size_t)kGatherWarps * rr * 4 * (size_t)lpad;
    e = launch_gather(g, gsmem, s, static_cast<const uint16_t*>(Z->hi),
                      static_cast<const uint16_t*>(Z->lo), d_perms, n, Z->l,
                      lpad, kb0, rpb, wh, wl, Z->status);
    if (e != cudaSuccess) return cuda_status(e);
    CUtensorMap ph, pl;
    if (!encode_tmap_3d_u16(&ph, wh, kbatch, n, lpad, kPT, KP, bf16) ||
        !encode_tmap_3d_u16(&pl, wl, kbatch, n, lpad, kPT, KP, bf16))
      return PCC_ERR_CUDA;
    // chunks of about kPermChunk permutations, and at least ~8 items per
    // worker: each item repeats the r_obs pass, which costs more than the
    // L2 reuse of permuted panels that shorter chunks buy (4,096 x 256 x
    // 1,000 on CTA pairs: 48 -> 8.9 ms, 96 -> 8.7, 192 -> 8.5, 336 -> 8.4)
    const int64_t workers = pair ? sms / 2 : sms;  // CTAs or CTA pairs
    int64_t chunk = kPermChunk;
    if (tiles * ((kbatch + chunk - 1) / chunk) < 8 * workers)
      chunk = (kbatch * tiles + 8 * workers - 1) / (8 * workers);
    if (chunk < 1) chunk = 1;
    if (chunk > kbatch) chunk = kbatch;
    const int64_t nchunks = (kbatch + chunk - 1) / chunk;
    PermParams p;
    p.n = n;
    p.m = m;
    p.items = tiles * nchunks;
    p.nchunks = (int)nchunks;
    p.chunk = (int)chunk;
    p.kbatch = (int)kbatch;
    p.nkb = (int)(lpad / KP);
    p.lolo = Z->prec == PCC_PREC_BF16X4 ? 1 : 0;
    p.flags = Z->flags;
    p.counts = d_counts;
    p.status = Z->status;
    p.wait_ns = wait_limit_ns();
    const bool resa = lpad <= kPMaxResidentK;
    if (pair && KP == 64) {
      if (resa)
        e = bf16 ? launch_perm_kernel<true, true, true, 64>(Z, ph, pl, p, s)
                 : launch_perm_kernel<false, true, true, 64>(Z, ph, pl, p, s);
      else
        e = bf16 ? launch_perm_kernel<true, false, true, 64>(Z, ph, pl, p, s)
                 : launch_perm_kernel<false, false, true, 64>(Z, ph, pl, p,
                                                              s);
    } else if (pair) {
      if (resa)
        e = bf16 ? launch_perm_kernel<true, true, true, 32>(Z, ph, pl, p, s)
                 : launch_perm_kernel<false, true, true, 32>(Z, ph, pl, p, s);
      else
        e = bf16 ? launch_perm_kernel<true, false, true, 32>(Z, ph, pl, p, s)
                 : launch_perm_kernel<false, false, true, 32>(Z, ph, pl, p,
                                                              s);
    } else {
      if (resa)
        e = bf16
                ? launch_perm_kernel<true, true, false, 32>(Z, ph, pl, p, s)
                : launch_perm_kernel<false, true, false, 32>(Z, ph, pl, p, s);
      else
        e = bf16
                ? launch_perm_kernel<true, false, false, 32>(Z, ph, pl, p, s)
                : launch_perm_kernel<false, false, false, 32>(Z, ph, pl, p,
                                                              s);
    }
    if (e != cudaSuccess) return cuda_status(e);
  }
  return PCC_OK;
}

}  // namespace pcc
