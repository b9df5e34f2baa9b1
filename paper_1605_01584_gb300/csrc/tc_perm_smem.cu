// tc_perm_smem.cu -- K6 without a permuted workspace: the permutation test
// of Section IV-A on CTA pairs, with each permuted operand built in shared
// memory from resident unpermuted rows.
//
// For permutations pi_k of the l samples, r_k(i,j) = z_i . (z_j o pi_k) with
// (z_j o pi_k)[s] = z_j[pi_k[s]], and counts[J(i,j)] += #{k : |r_k(i,j)| >=
// |r(i,j)|} for i < j.  Work: tile pairs of the triangle (two 128 x 128
// tiles of one tile column, rows 2r and 2r + 1, as one 2-SM MMA of M = 256)
// times passes of two permutations.  The passes of all tile pairs, tile by
// tile, are cut into one contiguous range per CTA pair; a range covers a few
// tiles, each a segment that starts with one r_obs pass.
//
// Per segment each CTA keeps resident in shared memory the source rows: its
// 64 of the tile column's 128 rows z_j, one 32-bit word per sample (hi | lo
// << 16), 256 words per row with the word index XOR-ed by the row's low
// five bits, so that 32 rows read at one sample index hit 32 banks.  A ring
// of 32-sample stages then carries, per stage,
//   - A: the CTA's 128 rows z_i, hi and lo (TMA, 64-byte swizzle; the rows
//     come from L2 for every pass);
//   - B: 128 K-major rows built from the source rows in the layout a
//     64-byte-swizzled TMA load would write: rows 0-63 permutation k, rows
//     64-127 permutation k + 1, for this CTA's 64 genes.
// The 2-SM MMA takes N = 128 B rows from each CTA, so accumulator columns
// are [k: genes 0-63 | k+1: genes 0-63 | k: genes 64-127 | k+1: genes
// 64-127] and epilogue half h reads columns 128h.. for genes 64h..64h+63.
// r_obs (the identity) and a lone last permutation fill both halves with
// the same rows, and only the first is read.
//
// Roles (10 warps): warp 0 loads A; warp 1 (lane 0 of the even CTA) issues
// the MMAs; warps 2-9 both gather and run the epilogue.  Warp 2 + e builds
// genes 8e..8e+7 of every B stage in both permutation slots, from the
// source rows it loaded itself, and after gathering a pass reads the
// accumulator of the previous one (|r_obs| and 16-bit counts in registers,
// one atomic per pair and segment).  A stage is full on the even CTA's
// barrier once both CTAs' A bytes have landed and the 16 warps of the pair
// have arrived.  Every wait is bounded.
//
// Cost: per 32-sample stage a CTA moves 96 KB through shared memory (the
// tensor cores' 48 KB of operand reads, 16 KB of gather reads and 16 KB of
// stores, 16 KB of A copies) against 64 KB when the permuted rows arrive by
// TMA next to a resident A tile: about as many cycles of shared-memory
// bandwidth as the stage's MMAs take, so this form can at best match the
// workspace form (tc_perm.cu).  As built it runs well below that bound,
// stalled on each stage's per-warp waits and hand-offs.  The transposed form
// (tc_perm_mn.cu) permutes with no shared-memory reads at all and is the
// default; this one stays selectable.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include "pcc_internal.h"
#include "pcc_ptx.cuh"
#include "pcc_sched.h"
#include "tc_common.cuh"
#include "tc_perm_common.cuh"

namespace pcc {
namespace {

constexpr int kSThreads = 320;            // 10 warps
constexpr int kSKP = 32;                  // samples per stage
constexpr int kSTile = kPT * kSKP * 2;    // 128 rows x 32 x 16 bit: 8 KB
constexpr int kSStages = 5;
constexpr int kSStageBytes = 4 * kSTile;  // [A hi | A lo | B hi | B lo]
constexpr int kSSrcPitch = 256;           // words per source row
constexpr int kSSrcBytes = 64 * kSSrcPitch * 4;                 // 64 KB
constexpr int kSBarBytes = 512;
constexpr int kSSmemBytes =
    1024 + kSStages * kSStageBytes + kSSrcBytes + kSBarBytes;
static_assert(kSSmemBytes <= kPSmemBudget, "shared memory");

struct PermSmemParams {
  int64_t n;
  int64_t m;          // 128-wide tiles per side
  int64_t tiles;      // tile pairs
  int64_t npass;      // passes per tile pair: ceil(P / 2)
  int64_t P;          // permutations tested
  int64_t kbase;      // index of the first one in perms
  int64_t l;
  int64_t lpad;
  int nkb;            // stages per pass: lpad / 32
  int lolo;           // 1: the fourth product lo.lo (BF16X4)
  const int32_t* perms;   // permutation k at perms + k * l
  const uint16_t* zhi;    // Z halves, n x lpad
  const uint16_t* zlo;
  const uint8_t* flags;
  uint32_t* counts;
  int* status;
  uint64_t wait_ns;
  int drop_loads;     // test hook (pcc_debug_drop_loads): 1 = no CTA loads
                      // A, 2 = the odd CTA of a pair loads none, 3 = the
                      // even CTA loads none (so the waits run out)
};

template <bool BF16>
__global__ void __launch_bounds__(kSThreads, 1)
    k_perm_smem(const __grid_constant__ CUtensorMap tz_hi,
                const __grid_constant__ CUtensorMap tz_lo,
                const PermSmemParams p) {
  // always M = 256 (both CTAs' tiles) and N = 256 (128 B rows per CTA)
  constexpr uint32_t kIdesc = make_idesc_f16(BF16, 2 * kPT, 2 * kPT);

  // 1024-byte aligned base, kept as an offset from the shared array so that
  // every access below compiles to shared-memory instructions
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem =
      smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t* ring = smem;  // kSStages x [A hi | A lo | B hi | B lo]
  uint32_t* src = reinterpret_cast<uint32_t*>(ring + kSStages * kSStageBytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(src + 64 * kSSrcPitch);
  uint64_t* full = bars;              // even CTA: A bytes + 16 warps
  uint64_t* empty = bars + kSStages;  // the MMA's commit, in both CTAs
  uint64_t* tfull = bars + 2 * kSStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* mdone = tempty + 2;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(mdone + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  FillLog* flog = reinterpret_cast<FillLog*>(bars + 32);  // A copies
  static_assert(2 * kSStages + 6 <= 31 && kSStages <= 16, "barrier area");
  static_assert(32 * 8 + sizeof(FillLog) <= kSBarBytes, "barrier area");

  auto sA_hi = [&](int s) { return ring + s * kSStageBytes; };
  auto sA_lo = [&](int s) { return sA_hi(s) + kSTile; };
  auto sB_hi = [&](int s) { return sA_hi(s) + 2 * kSTile; };
  auto sB_lo = [&](int s) { return sA_hi(s) + 3 * kSTile; };

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kSStages; ++s) {
      // the even producer's arrive (with both CTAs' A bytes) and the 8
      // gathering warps of each CTA
      mbar_init(&full[s], 1 + 2 * kPEpiWarps);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 2 * kPEpiWarps);  // both CTAs' epilogue warps
    }
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
      // ------------------------------------------------------ A producer
      const uint64_t pol = l2_policy_evict_last();
      constexpr uint32_t kABytes = 2u * kSTile;  // per CTA and stage
      int stage = 0;
      uint32_t phase = 0;
      bool ok = !(p.drop_loads == 1 || (p.drop_loads == 2 && crank == 1) ||
                  (p.drop_loads == 3 && crank == 0));
      for (int64_t u = u_begin; u < u_end && ok;) {
        const Segment g = next_segment(u, u_end, p.npass);
        u += g.q1 - g.q0;
        int64_t row0, col0;
        seg_coords(g, &row0, &col0);
        const int64_t nst = (g.q1 - g.q0 + 1) * p.nkb;  // r_obs + passes
        for (int64_t sg = 0; sg < nst; ++sg) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, w)) {
            ok = false;
            break;
          }
          const int kb = (int)(sg % p.nkb);
          // both CTAs' A bytes count on the even CTA's barrier
          if (crank == 0) mbar_arrive_expect_tx(&full[stage], 2u * kABytes);
          const uint32_t fb = cluster_addr(&full[stage], 0);
          tma_load_2d_pair(sA_hi(stage), &tz_hi, fb, kb * kSKP, (int)row0,
                           pol);
          tma_load_2d_pair(sA_lo(stage), &tz_lo, fb, kb * kSKP, (int)row0,
                           pol);
          flog->fills[stage] += 1u;
          flog->bytes[stage] = kABytes;
          if (++stage == kSStages) {
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
      bool ok = true;
      for (int64_t u = u_begin; u < u_end && ok;) {
        const Segment g = next_segment(u, u_end, p.npass);
        u += g.q1 - g.q0;
        const int64_t nps = g.q1 - g.q0;
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
            const uint32_t aH = smem_u32(sA_hi(stage));
            const uint32_t aL = smem_u32(sA_lo(stage));
            const uint32_t bH = smem_u32(sB_hi(stage));
            const uint32_t bL = smem_u32(sB_lo(stage));
#pragma unroll
            for (int ks = 0; ks < kSKP / kPUK; ++ks) {
              const uint32_t off = ks * kPUK * 2;
              const uint64_t dAH = kmajor_desc<2 * kSKP>(aH + off);
              const uint64_t dBH = kmajor_desc<2 * kSKP>(bH + off);
              const uint64_t dAL = kmajor_desc<2 * kSKP>(aL + off);
              const uint64_t dBL = kmajor_desc<2 * kSKP>(bL + off);
              umma_f16_pair(d_tmem, dAH, dBH, kIdesc, (kb | ks) != 0);
              umma_f16_pair(d_tmem, dAH, dBL, kIdesc, 1u);
              umma_f16_pair(d_tmem, dAL, dBH, kIdesc, 1u);
              if (p.lolo) umma_f16_pair(d_tmem, dAL, dBL, kIdesc, 1u);
            }
            umma_commit_pair(&empty[stage], 3);  // frees it in both CTAs
            if (++stage == kSStages) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (!ok) break;
          umma_commit_pair(&tfull[acc], 3);  // each CTA reads its rows
          acc ^= 1;
          if (acc == 0) aphase ^= 1u;
        }
      }
      umma_commit_pair(mdone, 1);
      WaitCtx wd = w;
      volatile int never = 0;
      wd.abort_flag = &never;
      mbar_wait(mdone, 0, wd);
    }
  } else {
    // ------------------------------------------------ gather and epilogue
    // Each warp gathers its share of every B stage (genes 8e..8e+7 of this
    // CTA's 64, in both permutation slots, from source rows it loaded
    // itself), in stage order, and reads its accumulator quarter after
    // each pass: pass pi: gather pi's stages, then the epilogue of pass
    // pi - 1.  The MMA of pass pi needs only epilogue pi - 2 (double
    // buffer), so the order cannot stall it; the ring keeps up to kSStages
    // stages gathered ahead while a warp runs an epilogue.
    const int q = warp & 3;          // TMEM lane quarter: rows 32q..32q+31
    const int h = (warp - 2) >> 2;   // genes 64h..64h+63: columns 128h..
    const int e = warp - 2;          // gather share: genes 8e..8e+7
    const int gq = lane >> 2;        // gather: gene 8e + gq,
    const int gc = lane & 3;         // samples 8gc..8gc+7 of a stage
    const int gg = 8 * e + gq;       // this lane's source row
    const uint32_t* srow = src + gg * kSSrcPitch;
    const uint32_t swz = (uint32_t)(gg & 31);
    const int64_t gene0 = (int64_t)crank * 64;
    const uint32_t full0 = cluster_addr(&full[0], 0);  // the even CTA's
    const int l = (int)p.l;  // <= lpad <= 256
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t aphase = 0;
    bool ok = true;
    bool bad = false;
    // this warp's share of one stage: lane (gq, gc) builds the 8 samples
    // 8gc.. of gene gg in slot 0 (indices v0 of samples 32 kb + lane, spread
    // by shuffles) and then in slot 1 (v1)
    auto gather_share = [&](int s, int32_t v0, int32_t v1) {
      uint8_t* bh = sB_hi(s);
      uint8_t* bl = sB_lo(s);
#pragma unroll
      for (int slot = 0; slot < 2; ++slot) {
        const int32_t vs = slot ? v1 : v0;
        uint32_t w8[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int32_t qi = __shfl_sync(0xffffffffu, vs, gc * 8 + t);
          const uint32_t x = srow[((uint32_t)qi & 255u) ^ swz];
          w8[t] = qi >= 0 ? x : 0u;  // padding sample: zero
        }
        // stage row of gene gg in this slot: 64 B of 32 samples, 16-byte
        // chunk gc at gc ^ ((row >> 1) & 3) (64-byte swizzle)
        const uint32_t rho = (uint32_t)(slot * 64 + gg);
        const uint32_t off =
            rho * 64u + 16u * ((uint32_t)gc ^ ((rho >> 1) & 3u));
        // hi: the low halves of the words, lo: the high halves
        uint4 ua, ub;
        ua.x = __byte_perm(w8[0], w8[1], 0x5410);
        ua.y = __byte_perm(w8[2], w8[3], 0x5410);
        ua.z = __byte_perm(w8[4], w8[5], 0x5410);
        ua.w = __byte_perm(w8[6], w8[7], 0x5410);
        ub.x = __byte_perm(w8[0], w8[1], 0x7632);
        ub.y = __byte_perm(w8[2], w8[3], 0x7632);
        ub.z = __byte_perm(w8[4], w8[5], 0x7632);
        ub.w = __byte_perm(w8[6], w8[7], 0x7632);
        *reinterpret_cast<uint4*>(bh + off) = ua;
        *reinterpret_cast<uint4*>(bl + off) = ub;
      }
    };
    for (int64_t u = u_begin; u < u_end && ok;) {
      const Segment g = next_segment(u, u_end, p.npass);
      u += g.q1 - g.q0;
      int64_t row0, col0;
      seg_coords(g, &row0, &col0);
      // 1. this warp's 8 source rows (word s of row r at s ^ (r & 31)),
      // two rows' loads in flight at a time; rows past n are zero.  This
      // warp's gathers of the previous segment are all done.
#pragma unroll 1
      for (int r0 = 0; r0 < 8; r0 += 2) {
        uint32_t hv[2][8], lv[2][8];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
          const int64_t j = col0 + gene0 + 8 * e + r0 + rr;
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int64_t sj = 32 * t + lane;
            const bool in = j < n && sj < p.lpad;
            hv[rr][t] = in ? (uint32_t)__ldg(p.zhi + j * p.lpad + sj) : 0u;
            lv[rr][t] = in ? (uint32_t)__ldg(p.zlo + j * p.lpad + sj) : 0u;
          }
        }
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
          const int r = 8 * e + r0 + rr;
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int sj = 32 * t + lane;
            if (sj < p.lpad)
              src[r * kSSrcPitch + (sj ^ (r & 31))] =
                  hv[rr][t] | (lv[rr][t] << 16);
          }
        }
      }
      __syncwarp();
      // 2. passes.  Lane t holds the indices of samples 32 kb + t, kb < 8,
      // of both slots; the next pass's load while the epilogue runs.
      const int64_t nps = g.q1 - g.q0;
      int32_t n0[8], n1[8];
      auto load_pass = [&](int64_t pi) {
        const int64_t k = 2 * (g.q0 + pi);
        // a lone last permutation fills both halves
        const int64_t k1 = k + 1 < p.P ? k + 1 : k;
        const int32_t* r0 = p.perms + (p.kbase + k) * p.l;
        const int32_t* r1 = p.perms + (p.kbase + k1) * p.l;
#pragma unroll
        for (int kb = 0; kb < 8; ++kb) {
          const int sj = kb * kSKP + lane;
          n0[kb] = sj < l ? __ldg(r0 + sj) : -1;
          n1[kb] = sj < l ? __ldg(r1 + sj) : -1;
        }
      };
      load_pass(0);
      float robs[64];
      uint32_t cnt[32];  // two 16-bit counts per word
#pragma unroll
      for (int t = 0; t < 32; ++t) cnt[t] = 0u;
      for (int64_t pi = -1; pi <= nps && ok; ++pi) {
        if (pi < nps) {
          // (a) gather pass pi: r_obs (the identity) for pi < 0; an index
          // outside [0, l) is recorded and read as sample 0
          if (pi >= 0) {
#pragma unroll
            for (int kb = 0; kb < 8; ++kb) {
              const int sj = kb * kSKP + lane;
              if (sj < l && (uint32_t)n0[kb] >= (uint32_t)l) {
                bad = true;
                n0[kb] = 0;
              }
              if (sj < l && (uint32_t)n1[kb] >= (uint32_t)l) {
                bad = true;
                n1[kb] = 0;
              }
            }
          }
#pragma unroll
          for (int kb = 0; kb < 8; ++kb) {
            if (kb >= p.nkb || !ok) break;
            bool okw = true;
            if (lane == 0) okw = mbar_wait(&empty[stage], phase ^ 1u, w);
            if (!__shfl_sync(0xffffffffu, okw ? 1 : 0, 0)) {
              ok = false;
              break;
            }
            const int sj = kb * kSKP + lane;
            const int32_t id = sj < l ? sj : -1;
            gather_share(stage, pi < 0 ? id : n0[kb], pi < 0 ? id : n1[kb]);
            // the stores reach the tensor cores (async proxy) of both
            // CTAs, ordered before the arrive by a release over shared
            // memory only
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
              fence_release_smem_cluster();
              mbar_arrive_relaxed_cluster(full0 + (uint32_t)(stage * 8));
            }
            if (++stage == kSStages) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (!ok) break;
          if (pi >= 0 && pi + 1 < nps) load_pass(pi + 1);
        }
        if (pi < 0) continue;
        // (b) the epilogue of pass pe = pi - 1 (pe < 0: r_obs); its
        // permutations: columns 128h + [0, 64) and, for two, 128h + [64, 128)
        const int64_t pe = pi - 1;
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
                               (uint32_t)(acc * kPAcc + h * 128);
        for (int ep = 0; ep < nperm; ++ep) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            uint32_t v[16];  // 16 columns at a time: registers are scarce
            tmem_ld_32x32b_x16(taddr + (uint32_t)(ep * 64 + c * 16), v);
            tmem_ld_wait();
            if (pe < 0) {
#pragma unroll
              for (int t = 0; t < 16; ++t)
                robs[c * 16 + t] = fabsf(__uint_as_float(v[t]));
            } else {
#pragma unroll
              for (int t = 0; t < 16; ++t) {
                const uint32_t hit =
                    fabsf(__uint_as_float(v[t])) >= robs[c * 16 + t] ? 1u
                                                                     : 0u;
                cnt[c * 8 + (t >> 1)] += hit << ((t & 1) * 16);
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
        for (int t = 0; t < 64; ++t) {
          const int64_t j = col0 + h * 64 + t;
          const uint32_t c = (cnt[t >> 1] >> ((t & 1) * 16)) & 0xFFFFu;
          if (c && j > i && j < n && p.flags[j] == 0)
            atomicAdd(p.counts + base + j, c);
        }
      }
    }
    if (bad) atomicCAS(p.status, 0, (int)PCC_ERR_INVALID_ARG);
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // every A copy issued by either CTA has landed before a CTA may exit.
  // After a wait ran out, a stage's phase may also lack gathering warps'
  // arrivals; the drain then ends on its own time limit, well after the
  // copies (issued before the first wait ran out) have landed.
  drain_ring<true>(full, nullptr, flog, kSStages, w, crank);
  if (warp == 1) {
    __syncwarp();
    tmem_dealloc_pair(tmem_base, 512);
  }
}

template <bool BF16>
cudaError_t launch_smem(const pcc_zmat* Z, const PermSmemParams& p,
                        cudaStream_t s) {
  auto fn = k_perm_smem<BF16>;
  cudaError_t e =
      ensure_func_smem(reinterpret_cast<const void*>(fn), kSSmemBytes);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(kSThreads, 1, 1);
  cfg.dynamicSmemBytes = kSSmemBytes;
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
  e = cudaLaunchKernelEx(&cfg, fn, Z->tm_hi32, Z->tm_lo32, p);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

bool perm_smem_applies(const pcc_zmat* Z) {
  const int64_t m = (Z->n + kPT - 1) / kPT;
  return Z->lpad <= kPMaxResidentK && m >= 2 && tc_tuning().pair_mma != 0 &&
         tc_tuning().perm_form == PCC_PERM_SMEM;
}

pcc_status perm_test_smem(pcc_zmat* Z, const int32_t* d_perms, int32_t k0,
                          int32_t k1, uint32_t* d_counts, cudaStream_t s) {
  const int64_t n = Z->n;
  PermSmemParams p;
  p.n = n;
  p.m = (n + kPT - 1) / kPT;
  p.tiles = col_pairs_before(p.m);
  p.P = (int64_t)k1 - k0;
  p.npass = (p.P + 1) / 2;
  p.kbase = k0;
  p.l = Z->l;
  p.lpad = Z->lpad;
  p.nkb = (int)(Z->lpad / kSKP);
  p.lolo = Z->prec == PCC_PREC_BF16X4 ? 1 : 0;
  p.perms = d_perms;
  p.zhi = static_cast<const uint16_t*>(Z->hi);
  p.zlo = static_cast<const uint16_t*>(Z->lo);
  p.flags = Z->flags;
  p.counts = d_counts;
  p.status = Z->status;
  p.wait_ns = wait_limit_ns();
  p.drop_loads = debug_drop_loads();
  if (p.P <= 0) return PCC_OK;
  const bool bf16 = Z->prec != PCC_PREC_FP16X3S;
  const cudaError_t e = bf16 ? launch_smem<true>(Z, p, s)
                             : launch_smem<false>(Z, p, s);
  return cuda_status(e);
}

}  // namespace pcc
