// tc_perm_mn.cu -- K6 without a workspace, from a transposed copy of Z: the
// permutation test of Section IV-A on CTA pairs, the permuted operand copied
// straight from L2 into shared memory.
//
// For permutations pi_k of the l samples, r_k(i,j) = z_i . (z_j o pi_k) with
// (z_j o pi_k)[s] = z_j[pi_k[s]], and counts[J(i,j)] += #{k : |r_k(i,j)| >=
// |r(i,j)|} for i < j.  With Z also stored transposed (ZT: sample rows of
// npad genes, hi and lo halves), the permuted column operand of sample s is
// row pi_k[s] of ZT: 128 contiguous genes of a tile column.  So the B
// operand is taken in MN-major form (genes contiguous) and built by 16-byte
// cp.async copies, one per (sample, 8 genes), in the layout of a 128-byte
// swizzle: 1 KB atoms of 8 samples x 64 genes (sample r of the atom at
// 128 r, the 16-byte chunk of genes 8c..8c+7 at 16 (c ^ r)), the two gene
// atoms of a stage 1 KB apart and its 8-sample groups 2 KB apart.
//
// Work and tiles as in the workspace form (tc_perm.cu, pair form): a pair
// of CTAs runs one 2-SM MMA (M = 256: rows 2r and 2r + 1 of a tile column,
// A resident in each CTA), N = 256 = permutation k's 128 column genes from
// the even CTA and k + 1's from the odd one (r_obs and a lone last
// permutation: the same in both).  The passes of all tile pairs, tile by
// tile, are cut into one contiguous range per CTA pair; a tile's passes are
// a segment with one r_obs pass.
//
// Roles (12 warps): warp 0 loads each segment's A tile and forwards every
// filled B stage to the even CTA's MMA; warp 1 (lane 0 of the even CTA)
// issues the MMAs; warps 2-3 copy B stages (KP/4 samples x 2 halves per
// thread and stage, completion counted by cp.async.mbarrier.arrive on this
// CTA's barrier, so no thread waits for its copies); warps 4-11 read the
// accumulator of each pass (|r_obs| and 16-bit counts in registers, one
// atomic per pair and segment).  Every wait is bounded.
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

constexpr int kMCopyWarps = 2;
constexpr int kMCopiers = kMCopyWarps * 32;       // copying threads per CTA
constexpr int kMEpi0 = 2 + kMCopyWarps;           // first epilogue warp
constexpr int kMThreads = (kMEpi0 + kPEpiWarps) * 32;  // 12 warps
constexpr int kMATile = kPT * 64 * 2;             // A: 128 rows x 64 x 16 bit
constexpr int kMABytes = (kPMaxResidentK / 64) * 2 * kMATile;  // 128 KB
constexpr int kMRing = 96 * 1024;                 // B stages
constexpr int kMBarBytes = 512;
constexpr int kMSmemBytes = 1024 + kMABytes + kMRing + kMBarBytes;
static_assert(kMSmemBytes <= kPSmemBudget, "shared memory");
// MN-major B: gene atoms (64 genes) 1 KB apart, 8-sample groups 2 KB apart
constexpr uint32_t kMLbo = 1024, kMSbo = 2048;

// B stages of KP samples: [hi | lo], each 128 genes x KP samples
template <int KP>
struct MnStage {
  static constexpr int kTile = kPT * KP * 2;
  static constexpr int kBytes = 2 * kTile;
  static constexpr int kStages = kMRing / kBytes;
  static constexpr int kPer = KP / 4;  // samples per copying thread
  static_assert(kTile == (KP / 8) * (int)kMSbo, "B layout");
  static_assert(kPer * 4 * 16 == KP * 16 && kMCopiers == 64, "copy share");
  static_assert(kStages <= 6, "barrier area");
};

struct PermMnParams {
  int64_t n;
  int64_t m;          // 128-wide tiles per side
  int64_t tiles;      // tile pairs
  int64_t npass;      // passes per tile pair: ceil(P / 2)
  int64_t P;          // permutations tested
  int64_t kbase;      // index of the first one in perms
  int64_t l;
  int64_t lpad;
  int64_t npad;       // row length of ZT (genes, a multiple of 128)
  int nkb;            // B stages per pass: lpad / KP
  int lolo;           // 1: the fourth product lo.lo (BF16X4)
  const int32_t* perms;   // permutation k at perms + k * l
  const uint16_t* zt_hi;  // ZT halves, lpad x npad
  const uint16_t* zt_lo;
  const uint8_t* flags;
  uint32_t* counts;
  int* status;
  uint64_t wait_ns;
  int drop_loads;     // test hook (pcc_debug_drop_loads): 1 = no CTA loads
                      // A or forwards a stage, 2 = the odd CTA of a pair
                      // does neither, 3 = the even CTA (the waits run out)
};

// 16 bytes from global memory (cached in L2 only) into this CTA's shared
// memory, by the executing thread.
__device__ __forceinline__ void cp_async16_cg(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst),
               "l"(src)
               : "memory");
}

// An arrival on `bar` once every cp.async this thread issued so far has
// completed; the barrier's count includes it (no increment first).
__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// A read-only 32-bit load issued where it stands in program order (before
// a wait that follows it), so that its latency overlaps the wait.
__device__ __forceinline__ int32_t ld_nc_s32(const int32_t* p) {
  int32_t v;
  asm volatile("ld.global.nc.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

// Shared-memory descriptor of an MN-major operand with 128-byte swizzle:
// lbo = stride between 64-element blocks along M/N, sbo = stride between
// 8-row groups along K (field layout as in kmajor_desc).
__device__ __forceinline__ uint64_t mnmajor_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((kMLbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((kMSbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)2u << 61;
  return d;
}

// ZT[k][j] = Z[j][k] for both halves, k < lpad, j < npad (zero for j >= n),
// through a 32 x 33 shared tile so that reads and writes are coalesced.
__global__ void __launch_bounds__(256)
    k_transpose_u16(const uint16_t* __restrict__ hi,
                    const uint16_t* __restrict__ lo, int64_t n, int64_t lpad,
                    uint16_t* __restrict__ thi, uint16_t* __restrict__ tlo,
                    int64_t npad) {
  __shared__ uint16_t t[2][32][33];
  const int64_t j0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t j = j0 + r;
    const int64_t e = j * lpad + k0 + threadIdx.x;
    t[0][r][threadIdx.x] = j < n ? hi[e] : (uint16_t)0;
    t[1][r][threadIdx.x] = j < n ? lo[e] : (uint16_t)0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t e = (k0 + r) * npad + j0 + threadIdx.x;
    thi[e] = t[0][threadIdx.x][r];
    tlo[e] = t[1][threadIdx.x][r];
  }
}

template <bool BF16, int KP>
__global__ void __launch_bounds__(kMThreads, 1)
    k_perm_mn(const __grid_constant__ CUtensorMap tz_hi,
              const __grid_constant__ CUtensorMap tz_lo,
              const PermMnParams p) {
  using St = MnStage<KP>;
  constexpr int S = St::kStages;
  // M = 256 (both CTAs' tiles), N = 256 (128 genes from each CTA), A
  // K-major, B MN-major (bit 16 of the instruction descriptor)
  constexpr uint32_t kIdesc =
      make_idesc_f16(BF16, 2 * kPT, 2 * kPT) | (1u << 16);

  // 1024-byte aligned base, an offset from the shared array (shared-memory
  // instructions for every access below)
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem =
      smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t* aregion = smem;                   // resident A: [64 samples][hi|lo]
  uint8_t* ring = smem + kMABytes;           // B stages: [hi | lo]
  uint64_t* bars = reinterpret_cast<uint64_t*>(ring + kMRing);
  uint64_t* full = bars;                     // even CTA: both forwards
  uint64_t* empty = bars + 6;                // the MMA's commit, both CTAs
  uint64_t* bfull = bars + 12;               // this CTA's copies landed
  uint64_t* tfull = bars + 18;
  uint64_t* tempty = tfull + 2;
  uint64_t* afull = tempty + 2;
  uint64_t* aempty = afull + 1;
  uint64_t* mdone = aempty + 1;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(mdone + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  FillLog* flog = reinterpret_cast<FillLog*>(bars + 32);  // A copies
  static_assert(18 + 7 <= 31, "barrier area");
  static_assert(32 * 8 + sizeof(FillLog) <= kMBarBytes, "barrier area");

  auto sA_hi = [&](int a) { return aregion + a * 2 * kMATile; };
  auto sA_lo = [&](int a) { return sA_hi(a) + kMATile; };
  auto sB_hi = [&](int s) { return ring + s * St::kBytes; };
  auto sB_lo = [&](int s) { return sB_hi(s) + St::kTile; };

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 2);          // the forwarder of each CTA
      mbar_init(&empty[s], 1);
      mbar_init(&bfull[s], kMCopiers);  // every copying thread, no-inc
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 2 * kPEpiWarps);  // both CTAs' epilogue warps
    }
    mbar_init(afull, 1);
    mbar_init(aempty, 1);
    mbar_init(mdone, 1);
    *abort_flag = 0;
    fill_log_init(flog);
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc_pair(tmem_holder, 512);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  cluster_sync();  // both CTAs' barriers exist before either signals
  const uint32_t tmem_base = *tmem_holder;
  const uint32_t crank = cluster_ctarank();
  WaitCtx w{abort_flag, p.status, p.wait_ns};
  const int64_t n = p.n;

  // this CTA pair's range of (tile pair, pass) units, tile by tile
  const int64_t pw = (int64_t)(blockIdx.x >> 1);
  const int64_t npw = (int64_t)(gridDim.x >> 1);
  const int64_t units = p.tiles * p.npass;
  const int64_t u_begin = pw * units / npw;
  const int64_t u_end = (pw + 1) * units / npw;

  // `dummy` marks the missing partner of a column's last, lone tile: it
  // repeats its partner's tile and its counts are dropped
  bool dummy = false;
  auto seg_coords = [&](const Segment& g, int64_t* row0, int64_t* col0) {
    int64_t r, xt;
    col_pair_coords(g.t, &r, &xt);
    int64_t yt = 2 * r + (int64_t)crank;
    dummy = yt > xt;
    if (dummy) yt = 2 * r;
    *row0 = yt * kPT;
    *col0 = xt * kPT;
  };

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------- A tiles and stage forwarding
      const uint64_t pol = l2_policy_evict_last();
      const int na = (int)(p.lpad / 64);
      const uint32_t abytes = (uint32_t)(na * 2 * kMATile);
      const uint32_t full0 = cluster_addr(&full[0], 0);  // the even CTA's
      uint32_t aph = 0;
      int stage = 0;
      uint32_t phase = 0;
      bool ok = !(p.drop_loads == 1 || (p.drop_loads == 2 && crank == 1) ||
                  (p.drop_loads == 3 && crank == 0));
      for (int64_t u = u_begin; u < u_end && ok;) {
        const Segment g = next_segment(u, u_end, p.npass);
        u += g.q1 - g.q0;
        int64_t row0, col0;
        seg_coords(g, &row0, &col0);
        if (!mbar_wait(aempty, aph ^ 1u, w)) break;
        flog->fills[0] += 1u;
        flog->bytes[0] = abytes;
        // both CTAs' A tiles count on the even CTA's barrier
        if (crank == 0) mbar_arrive_expect_tx(afull, 2u * abytes);
        const uint32_t ab = cluster_addr(afull, 0);
        for (int a = 0; a < na; ++a) {
          tma_load_2d_pair(sA_hi(a), &tz_hi, ab, a * 64, (int)row0, pol);
          tma_load_2d_pair(sA_lo(a), &tz_lo, ab, a * 64, (int)row0, pol);
        }
        aph ^= 1u;
        // each B stage this CTA's copies filled goes to the MMA issuer:
        // the copies landed (this CTA's barrier), their stores are made
        // visible to the tensor cores and released over shared memory
        const int64_t nst = (g.q1 - g.q0 + 1) * p.nkb;
        for (int64_t sg = 0; sg < nst; ++sg) {
          if (!mbar_wait(&bfull[stage], phase, w)) {
            ok = false;
            break;
          }
          fence_proxy_async_smem();
          fence_release_smem_cluster();
          mbar_arrive_relaxed_cluster(full0 + (uint32_t)(stage * 8));
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && crank == 0) {
      // ------------------------------------------- MMA issuer (even CTA)
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t aphase = 0;
      uint32_t aph = 0;
      bool ok = true;
      for (int64_t u = u_begin; u < u_end && ok;) {
        const Segment g = next_segment(u, u_end, p.npass);
        u += g.q1 - g.q0;
        const int64_t nps = g.q1 - g.q0;
        if (!mbar_wait(afull, aph, w)) break;  // both CTAs' A tiles
        aph ^= 1u;
        tc_fence_after();
        for (int64_t pi = -1; pi < nps && ok; ++pi) {
          if (!mbar_wait(&tempty[acc], aphase ^ 1u, w)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + (uint32_t)(acc * kPAcc);
          for (int kb = 0; kb < p.nkb; ++kb) {
            if (!mbar_wait_acq_cluster(&full[stage], phase, w)) {
              ok = false;
              break;
            }
            tc_fence_after();
            // samples kb*KP.. of the A tiles: tile (kb*KP)/64, at byte
            // 2 ((kb*KP) mod 64) of its 128-byte rows
            const int a = (kb * KP) >> 6;
            const uint32_t aoff = (uint32_t)(((kb * KP) & 63) * 2);
            const uint32_t aH = smem_u32(sA_hi(a)) + aoff;
            const uint32_t aL = smem_u32(sA_lo(a)) + aoff;
            const uint32_t bH = smem_u32(sB_hi(stage));
            const uint32_t bL = smem_u32(sB_lo(stage));
#pragma unroll
            for (int ks = 0; ks < KP / kPUK; ++ks) {
              // A: +32 B per 16 samples inside its 128-byte rows; B: two
              // 8-sample groups per 16 samples
              const uint64_t dAH = kmajor_desc<128>(aH + ks * kPUK * 2);
              const uint64_t dAL = kmajor_desc<128>(aL + ks * kPUK * 2);
              const uint64_t dBH = mnmajor_desc_sw128(bH + ks * 2 * kMSbo);
              const uint64_t dBL = mnmajor_desc_sw128(bL + ks * 2 * kMSbo);
              umma_f16_pair(d_tmem, dAH, dBH, kIdesc, (kb | ks) != 0);
              umma_f16_pair(d_tmem, dAH, dBL, kIdesc, 1u);
              umma_f16_pair(d_tmem, dAL, dBH, kIdesc, 1u);
              if (p.lolo) umma_f16_pair(d_tmem, dAL, dBL, kIdesc, 1u);
            }
            umma_commit_pair(&empty[stage], 3);  // frees it in both CTAs
            if (++stage == S) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (!ok) break;
          umma_commit_pair(&tfull[acc], 3);  // each CTA reads its rows
          acc ^= 1;
          if (acc == 0) aphase ^= 1u;
        }
        if (ok) umma_commit_pair(aempty, 3);  // the A tiles may be replaced
      }
      umma_commit_pair(mdone, 1);
      WaitCtx wd = w;
      volatile int never = 0;
      wd.abort_flag = &never;
      mbar_wait(mdone, 0, wd);
    }
  } else if (warp < kMEpi0) {
    // ------------------------------------------------------- B copies
    // Thread t copies, for samples sr + 4i of a stage (i < KP/4), the 16
    // bytes of genes 8c..8c+7 of both halves.  The permutation indices of
    // a stage are loaded before its wait for a free slot.
    const int t = threadIdx.x - 64;
    const int sr = t >> 4;  // 0..3
    const int cch = t & 15;
    // byte offset of sample sr + 4i in a stage's tile: 8-sample group i/2,
    // gene atom cch/8, row sr + 4 (i & 1) of the atom, chunk (cch & 7) ^ row
    uint32_t dbase[2];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int r = sr + 4 * b;
      dbase[b] = (uint32_t)((cch >> 3) * (int)kMLbo + r * 128 +
                            (((cch & 7) ^ r) << 4));
    }
    const int l = (int)p.l;
    const uint32_t npad = (uint32_t)p.npad;
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    bool bad = false;
    for (int64_t u = u_begin; u < u_end && ok;) {
      const Segment g = next_segment(u, u_end, p.npass);
      u += g.q1 - g.q0;
      int64_t row0, col0;
      seg_coords(g, &row0, &col0);
      const uint16_t* src_hi = p.zt_hi + col0 + 8 * cch;
      const uint16_t* src_lo = p.zt_lo + col0 + 8 * cch;
      const int64_t nps = g.q1 - g.q0;
      for (int64_t pi = -1; pi < nps && ok; ++pi) {
        // the even CTA takes permutation k, the odd one k + 1 (a lone last
        // permutation: k in both); pi < 0: the identity (r_obs); a padding
        // sample s >= l reads the (zero) row s itself
        const int64_t k0 = 2 * (g.q0 + pi);
        const int64_t k =
            k0 + (int64_t)crank < p.P ? k0 + (int64_t)crank : k0;
        const int32_t* pr = p.perms + (p.kbase + (pi < 0 ? 0 : k)) * p.l;
        for (int kb = 0; kb < p.nkb; ++kb) {
          int32_t v[St::kPer];
#pragma unroll
          for (int i = 0; i < St::kPer; ++i) {
            const int s = kb * KP + sr + 4 * i;
            v[i] = (pi >= 0 && s < l) ? ld_nc_s32(pr + s) : s;
          }
          bool okw = true;
          if (lane == 0) okw = mbar_wait(&empty[stage], phase ^ 1u, w);
          if (!__shfl_sync(0xffffffffu, okw ? 1 : 0, 0)) {
            ok = false;
            break;
          }
          const uint32_t sb = smem_u32(sB_hi(stage));
#pragma unroll
          for (int i = 0; i < St::kPer; ++i) {
            const int s = kb * KP + sr + 4 * i;
            int32_t r = v[i];
            if (pi >= 0 && s < l && (uint32_t)r >= (uint32_t)l) {
              bad = true;  // recorded, read as sample 0
              r = 0;
            }
            const uint32_t off = (uint32_t)r * npad;
            const uint32_t dst =
                sb + (uint32_t)((i >> 1) * (int)kMSbo) + dbase[i & 1];
            cp_async16_cg(dst, src_hi + off);
            cp_async16_cg(dst + (uint32_t)St::kTile, src_lo + off);
          }
          // counted on this CTA's barrier once they have landed
          cp_async_arrive_noinc(&bfull[stage]);
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
    }
    if (bad) atomicCAS(p.status, 0, (int)PCC_ERR_INVALID_ARG);
    // no copy of this thread may still be in flight when the CTA leaves
    cp_async_wait_all();
  } else {
    // ----------------------------------------------------------- epilogue
    const int q = warp & 3;               // TMEM lane quarter: rows 32q..
    const int h = (warp - kMEpi0) >> 2;   // genes 64h..: columns 64h..
    int acc = 0;
    uint32_t aphase = 0;
    bool ok = true;
    for (int64_t u = u_begin; u < u_end && ok;) {
      const Segment g = next_segment(u, u_end, p.npass);
      u += g.q1 - g.q0;
      int64_t row0, col0;
      seg_coords(g, &row0, &col0);
      const int64_t nps = g.q1 - g.q0;
      float robs[64];
      uint32_t cnt[32];  // two 16-bit counts per word
#pragma unroll
      for (int i = 0; i < 32; ++i) cnt[i] = 0u;
      for (int64_t pe = -1; pe < nps; ++pe) {
        // pass pe (pe < 0: r_obs); permutation e of the pass at columns
        // 128e + 64h..
        const int nperm =
            pe < 0 ? 1 : (2 * (g.q0 + pe) + 1 < p.P ? 2 : 1);
        bool got = true;
        if (lane == 0) got = mbar_wait(&tfull[acc], aphase, w);
        if (!__shfl_sync(0xffffffffu, got ? 1 : 0, 0)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) +
                               (uint32_t)(acc * kPAcc + h * 64);
        for (int ep = 0; ep < nperm; ++ep) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            uint32_t v[16];
            tmem_ld_32x32b_x16(taddr + (uint32_t)(ep * 128 + c * 16), v);
            tmem_ld_wait();
            if (pe < 0) {
#pragma unroll
              for (int i = 0; i < 16; ++i)
                robs[c * 16 + i] = fabsf(__uint_as_float(v[i]));
            } else {
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                const uint32_t hit =
                    fabsf(__uint_as_float(v[i])) >= robs[c * 16 + i] ? 1u
                                                                     : 0u;
                cnt[c * 8 + (i >> 1)] += hit << ((i & 1) * 16);
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if (crank != 0)  // released to the even CTA's MMA issuer
            tmem_release_cluster(cluster_addr(&tempty[acc], 0));
          else
            tmem_release(&tempty[acc]);
        }
        acc ^= 1;
        if (acc == 0) aphase ^= 1u;
      }
      if (!ok) break;
      // add this segment's counts to the packed output
      const int64_t i = row0 + q * 32 + lane;
      if (!dummy && i < n && p.flags[i] == 0) {
        const int64_t base = pair_row_base(n, i);
#pragma unroll
        for (int c = 0; c < 64; ++c) {
          const int64_t j = col0 + h * 64 + c;
          const uint32_t v = (cnt[c >> 1] >> ((c & 1) * 16)) & 0xFFFFu;
          if (v && j > i && j < n && p.flags[j] == 0)
            atomicAdd(p.counts + base + j, v);
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // every A copy issued by either CTA has landed before a CTA may exit
  drain_ring<true>(afull, nullptr, flog, 1, w, crank);
  if (warp == 1) {
    __syncwarp();
    tmem_dealloc_pair(tmem_base, 512);
  }
}

// ZT (both halves, lpad x npad each) for the current contents of Z: built
// on the first call after each standardize, and by every call that a stream
// capture records (a replay may follow a later standardize).
cudaError_t ensure_zt16(pcc_zmat* Z, int64_t npad, cudaStream_t s) {
  if (Z->zt_valid && !stream_capturing(s)) return cudaSuccess;
  const size_t need = 2 * (size_t)npad * (size_t)Z->lpad * sizeof(uint16_t);
  if (Z->zt_bytes < need) {
    if (Z->zt) {
      cudaStreamSynchronize(s);
      cudaFree(Z->zt);
      Z->zt = nullptr;
      Z->zt_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&Z->zt, need);
    if (e != cudaSuccess) return e;
    Z->zt_bytes = need;
  }
  uint16_t* thi = static_cast<uint16_t*>(Z->zt);
  k_transpose_u16<<<dim3((unsigned)(npad / 32), (unsigned)(Z->lpad / 32)),
                    dim3(32, 8), 0, s>>>(
      static_cast<const uint16_t*>(Z->hi), static_cast<const uint16_t*>(Z->lo),
      Z->n, Z->lpad, thi, thi + (size_t)Z->lpad * (size_t)npad, npad);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) Z->zt_valid = 1;
  return e;
}

template <bool BF16, int KP>
cudaError_t launch_mn(const pcc_zmat* Z, const PermMnParams& p,
                      cudaStream_t s) {
  auto fn = k_perm_mn<BF16, KP>;
  cudaError_t e =
      ensure_func_smem(reinterpret_cast<const void*>(fn), kMSmemBytes);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(kMThreads, 1, 1);
  cfg.dynamicSmemBytes = kMSmemBytes;
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
  const int64_t units = p.tiles * p.npass;
  const int64_t ncl = units < max_clusters ? units : max_clusters;
  cfg.gridDim = dim3((unsigned)(2 * ncl), 1, 1);
  e = cudaLaunchKernelEx(&cfg, fn, Z->tm_hi, Z->tm_lo, p);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

int64_t mn_npad(int64_t n) { return (n + kPT - 1) / kPT * kPT; }

// samples per B stage: 64 (three stages) or, with PCC_PERM_MN_K=32, 32
// (six stages of half the size)
int mn_stage_k() {
  static const int k = [] {
    const char* e = getenv("PCC_PERM_MN_K");
    return (e && atoi(e) == 32) ? 32 : 64;
  }();
  return k;
}

}  // namespace

bool perm_mn_applies(const pcc_zmat* Z) {
  const int64_t m = (Z->n + kPT - 1) / kPT;
  // ZT offsets of a sample row are 32-bit element offsets
  return Z->lpad <= kPMaxResidentK && m >= 2 && tc_tuning().pair_mma != 0 &&
         tc_tuning().perm_form == PCC_PERM_TRANSPOSED &&
         (uint64_t)Z->lpad * (uint64_t)mn_npad(Z->n) < (1ull << 32);
}

pcc_status perm_test_mn(pcc_zmat* Z, const int32_t* d_perms, int32_t k0,
                        int32_t k1, uint32_t* d_counts, cudaStream_t s) {
  const int64_t n = Z->n;
  const int kp = mn_stage_k();
  PermMnParams p;
  p.n = n;
  p.m = (n + kPT - 1) / kPT;
  p.tiles = col_pairs_before(p.m);
  p.P = (int64_t)k1 - k0;
  p.npass = (p.P + 1) / 2;
  p.kbase = k0;
  p.l = Z->l;
  p.lpad = Z->lpad;
  p.npad = mn_npad(n);
  p.nkb = (int)(Z->lpad / kp);
  p.lolo = Z->prec == PCC_PREC_BF16X4 ? 1 : 0;
  p.perms = d_perms;
  p.flags = Z->flags;
  p.counts = d_counts;
  p.status = Z->status;
  p.wait_ns = wait_limit_ns();
  p.drop_loads = debug_drop_loads();
  if (p.P <= 0) return PCC_OK;
  const cudaError_t ez = ensure_zt16(Z, p.npad, s);
  if (ez != cudaSuccess) {
    cudaGetLastError();
    return ez == cudaErrorMemoryAllocation ? PCC_ERR_OOM : cuda_status(ez);
  }
  p.zt_hi = static_cast<const uint16_t*>(Z->zt);
  p.zt_lo = p.zt_hi + (size_t)p.lpad * (size_t)p.npad;
  const bool bf16 = Z->prec != PCC_PREC_FP16X3S;
  cudaError_t e;
  if (kp == 32)
    e = bf16 ? launch_mn<true, 32>(Z, p, s) : launch_mn<false, 32>(Z, p, s);
  else
    e = bf16 ? launch_mn<true, 64>(Z, p, s) : launch_mn<false, 64>(Z, p, s);
  return cuda_status(e);
}

}  // namespace pcc
