// tc_pairs.cu -- K2 / K3: all-pairs r(i,j) = z_i . z_j (Eq. (6)) on the
// tcgen05 tensor cores, with the packed-triangle and |r| >= tau epilogues
// fused.
//
// Precision: z = hi + lo (two 16-bit halves, written by the variable
// transformation).  Per tile the MMAs accumulate, in FP32 in TMEM,
//     hi_Y hi_X^T + hi_Y lo_X^T + lo_Y hi_X^T          (3 products)
// which recovers z_Y z_X^T up to the dropped lo lo^T term; BF16X4 adds
// that fourth product, BF16X1 runs the first product only.
//
// Work decomposition (pcc_sched.h): 256 x 256 super-tiles of the upper
// triangle in banded order, each split into two units of 128 rows x 256
// columns.  A persistent grid (one CTA per SM) strides over the units, as
// Algorithm 1 strides thread groups over tile ids.
//
// CTA roles (320 threads):
//   warp 0      TMA producer: per K block (32 or 64), loads A = rows of the
//               unit (hi, lo: 128 rows each) and B = its columns (hi, lo:
//               256 rows each) into a ring of shared-memory stages.
//   warp 1      allocates 512 TMEM columns (two 128 x 256 FP32
//               accumulators) and one elected thread issues the MMAs
//               (M = 128, N = 256, K = 16 per instruction), committing each
//               stage back to the producer and each finished accumulator to
//               the epilogue.
//   warps 2-9   epilogue: tcgen05.ld of the accumulator (warp w reads TMEM
//               lanes 32*(w%4)..+31 = its 32 rows, and one half of the
//               columns), a transpose through
//               shared memory so that a warp stores 32 consecutive pairs of
//               one row at a time (rows of the packed triangle are
//               contiguous), clamp to [-1,1], NaN for flagged rows, and the
//               optional warp-aggregated edge append.
// The two accumulators let the epilogue of one unit overlap the MMAs of the
// next.  Rows longer than 1,024 samples cut a unit's K blocks into chunks
// of at most 640 samples, each accumulated in a fresh buffer and added into
// the next by the epilogue (tc_common.cuh): the FP32 accumulation rounds
// its running sum toward zero, and a shorter running sum loses less.
//
// CROSS: the non-symmetric job matrix between the rows of two matrices
// (Section III-B, Eq. (7)-(8)): A rows come from the first, B rows from the
// second, every super-tile of the my x mx grid is computed, and the
// epilogue writes a dense row-major R (pitch ldr).  Super-tiles are taken
// in bands of G rows, column by column within a band (Eq. (7)-(8) with the
// roles of rows and columns swapped, per band), so that a band's A rows
// stay in L2 while B streams past them once.
//
// CTA pairs (the default: 2-CTA clusters).  The CTAs of a pair compute the
// two halves of one super-tile, which need the same 256 B rows, as one 2-SM
// MMA unit: each CTA loads its 128 A rows and 128 of the B rows into its own
// stage, and the even CTA issues tcgen05.mma.cta_group::2 with M = 256; the
// pair's tensor cores exchange the B halves, so each SM takes a third less
// operand data from L2 than a CTA that loads all 256 B rows, and a stage is
// a third smaller (six stages instead of four).  Both CTAs' copies count on
// the even CTA's stage barrier; its commits release the stage in both CTAs
// and hand each CTA its half of the accumulator; both epilogues release the
// accumulator to the even CTA.  Otherwise (pcc_set_pair_mma(0)) every CTA
// runs its own M = 128 MMA over all 256 B rows.
// Measured at 65,536 x 512: 4.76 ms (2-SM MMA), 5.42 ms (independent CTAs).
// Every wait is bounded (pcc_ptx.cuh): a wait that runs out records
// PCC_ERR_TIMEOUT; the CTA stops issuing, waits for every copy it (and, in
// the pair form, its partner) issued, frees TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdlib.h>

#include "pcc_internal.h"
#include "pcc_ptx.cuh"
#include "pcc_sched.h"
#include "tc_common.cuh"
#include "tc_epilogue.cuh"

namespace pcc {
namespace {

constexpr int kBM = 128;   // rows per unit (MMA M)
constexpr int kBN = 256;   // columns per unit (MMA N)
constexpr int kUK = 16;    // K per tcgen05.mma kind::f16
constexpr int kThreads = 320;
constexpr int kEpiWarps = 8;

struct TcParams {
  int64_t n;         // rows (of the first matrix)
  int64_t m;         // super-tiles per side (CROSS: super-tile rows)
  int64_t ncol;      // columns: n, or the second matrix's rows (CROSS)
  int64_t mcol;      // CROSS: super-tile columns
  int64_t ldr;       // CROSS: row pitch of R
  int64_t r_off;     // R holds the output from element r_off on (a window
                     // of whole rows, for passes that do not fit at once)
  const uint8_t* cflags;  // flags of the column variables
  int64_t G;         // super-tile rows per band (pcc_sched.h)
  int64_t u_begin;   // units [u_begin, u_end)
  int64_t u_end;
  int nkb;           // K blocks of KB
  int nch;           // accumulator chunks per unit (tc_common.cuh)
  float out_scale;   // 2^-2s for FP16X3S, else 1
  float tau;
  const uint8_t* flags;
  float* R;
  pcc_edge* edges;
  unsigned long long* count;
  uint64_t cap;
  int* status;
  uint64_t wait_ns;
  int drop_loads;    // test hook (pcc_debug_drop_loads): 1 = no producer
                     // issues loads, 2 / 3 = the odd / even CTA of each
                     // pair issues none, so an operand wait runs out
};

// KB = K per ring stage: 64 (one 128-B swizzle row of 16-bit elements, 2
// stages of 96 KB) or 32 (64-B swizzle, 4 stages of 48 KB: the same bytes in
// flight, refilled at half the granularity).
// PAIR (the 2-SM MMA of a CTA pair): each CTA holds only its 128 of the
// 256 B rows, so a stage is a third smaller and the ring holds six (K = 32)
// or three (K = 64).
template <int NPROD, int KB, bool PAIR = false>
struct Cfg {
  static constexpr int kTileA = kBM * KB * 2;
  static constexpr int kTileB = (PAIR ? kBM : kBN) * KB * 2;
  static constexpr int kSwz = KB * 2;  // swizzle span in bytes
  static constexpr int kStageBytes =
      NPROD == 1 ? (kTileA + kTileB) : 2 * (kTileA + kTileB);
  static constexpr int kStages = (4 * 49152) / kStageBytes;
  static constexpr int kRingBytes = kStages * kStageBytes;
  static constexpr int kEpiBytes = kEpiWarps * 32 * kStagePad * 4;
  static constexpr int kBarBytes = 512;
  static constexpr int kSmemBytes = 1024 + kRingBytes + kEpiBytes + kBarBytes;
  static_assert(kSmemBytes <= 232448, "shared memory budget");
};

template <bool CROSS>
__device__ __forceinline__ void unit_coords(BandCursor* cur, const TcParams& p,
                                            int64_t u, int64_t* row0,
                                            int64_t* col0) {
  int64_t yt, xt;
  if constexpr (CROSS) {
    const int64_t t = u >> 1;
    const int64_t per_band = p.G * p.mcol;
    const int64_t b = t / per_band;
    const int64_t tb = t - b * per_band;
    const int64_t rows = p.m - b * p.G < p.G ? p.m - b * p.G : p.G;
    xt = tb / rows;
    yt = b * p.G + (tb - xt * rows);
  } else {
    band_tile_coords(cur, p.m, p.G, u >> 1, &yt, &xt);
  }
  *row0 = yt * kTcSuper + (u & 1) * kBM;
  *col0 = xt * kTcSuper;
}

template <int NPROD, bool BF16, bool WRITE_R, bool EDGES, int KB, bool CROSS,
          bool PAIR>
__global__ void __launch_bounds__(kThreads, 1)
    k_pairs_tc(const __grid_constant__ CUtensorMap tm_hi,
               const __grid_constant__ CUtensorMap tm_lo,
               const __grid_constant__ CUtensorMap tmb_hi,
               const __grid_constant__ CUtensorMap tmb_lo, const TcParams p) {
  // B operand maps: the second matrix's for CROSS, else Z's own
  const CUtensorMap* mb_hi = CROSS ? &tmb_hi : &tm_hi;
  const CUtensorMap* mb_lo = CROSS ? &tmb_lo : &tm_lo;
  using C = Cfg<NPROD, KB, PAIR>;
  constexpr int kTileA = C::kTileA;
  constexpr int kTileB = C::kTileB;
  constexpr int S = C::kStages;
  static_assert(S <= 16, "fill log size");
  // PAIR: one instruction covers the pair's 256 rows
  constexpr uint32_t kIdesc = make_idesc_f16(BF16, PAIR ? 2 * kBM : kBM, kBN);

  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned base, kept as an offset from the shared array so
  // that accesses through it compile to shared-memory instructions
  uint8_t* smem =
      smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t* ring = smem;
  float* epi = reinterpret_cast<float*>(smem + C::kRingBytes);
  uint64_t* bars =
      reinterpret_cast<uint64_t*>(smem + C::kRingBytes + C::kEpiBytes);
  uint64_t* full = bars;            // [S]
  uint64_t* empty = bars + S;       // [S]
  uint64_t* tfull = bars + 2 * S;   // [2]
  uint64_t* tempty = tfull + 2;     // [2]
  uint64_t* mdone = tempty + 2;     // [1]
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(mdone + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  FillLog* flog = reinterpret_cast<FillLog*>(bars + 32);
  static_assert(2 * S + 5 <= 31, "barrier area");
  static_assert(32 * 8 + sizeof(FillLog) <= C::kBarBytes, "barrier area");

  auto sA_hi = [&](int s) { return ring + s * C::kStageBytes; };
  auto sB_hi = [&](int s) { return ring + s * C::kStageBytes + kTileA; };
  auto sA_lo = [&](int s) {
    return ring + s * C::kStageBytes + kTileA + kTileB;
  };
  auto sB_lo = [&](int s) {
    return ring + s * C::kStageBytes + 2 * kTileA + kTileB;
  };

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      // PAIR: the even CTA's accumulator barriers count both epilogues
      mbar_init(&tempty[a], PAIR ? 2 * kEpiWarps : kEpiWarps);
    }
    mbar_init(mdone, 1);
    *abort_flag = 0;
    fill_log_init(flog);
    fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    tma_prefetch_desc(&tm_hi);
    if (NPROD > 1) tma_prefetch_desc(&tm_lo);
    if (CROSS) {
      tma_prefetch_desc(&tmb_hi);
      if (NPROD > 1) tma_prefetch_desc(&tmb_lo);
    }
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
  // both CTAs' barriers are initialised before the pair signals across them
  if constexpr (PAIR) cluster_sync();
  const uint32_t tmem_base = *tmem_holder;
  const uint32_t crank = PAIR ? cluster_ctarank() : 0u;

  WaitCtx w{abort_flag, p.status, p.wait_ns};
  const int64_t n = p.n;
  const int nkb = p.nkb;
  const int nch = p.nch;

  if (warp == 0) {
    // ------------------------------------------------------ TMA producer
    if (lane == 0) {
      BandCursor cur;
      band_cursor_init(&cur, p.m, p.G);
      int stage = 0;
      uint32_t phase = 0;
      const uint64_t pol = l2_policy_evict_last();
      const bool drop = p.drop_loads == 1 ||
                        (PAIR && p.drop_loads == 2 && crank == 1) ||
                        (PAIR && p.drop_loads == 3 && crank == 0);
      for (int64_t u = p.u_begin + blockIdx.x; u < p.u_end && !drop;
           u += gridDim.x) {
        int64_t row0, col0;
        unit_coords<CROSS>(&cur, p, u, &row0, &col0);
        // the CTAs of a pair run their units in lockstep (they share B), so
        // only the single-CTA form skips units below the last row
        if (!PAIR && row0 >= n) continue;
        bool ok = true;
        for (int kb = 0; kb < nkb; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, w)) {
            ok = false;
            break;
          }
          const int kc = kb * KB;
          if constexpr (PAIR) {
            // each CTA loads its 128 A rows and its 128 of the 256 B rows
            // into its own stage; the even CTA's barrier counts the bytes
            // of both, since its one MMA reads both stages
            if (crank == 0)
              mbar_arrive_expect_tx(&full[stage], 2 * C::kStageBytes);
            const uint32_t fb = cluster_addr(&full[stage], 0);
            const int brow = (int)(col0 + crank * kBM);
            tma_load_2d_pair(sA_hi(stage), &tm_hi, fb, kc, (int)row0, pol);
            tma_load_2d_pair(sB_hi(stage), mb_hi, fb, kc, brow, pol);
            if (NPROD > 1) {
              tma_load_2d_pair(sA_lo(stage), &tm_lo, fb, kc, (int)row0, pol);
              tma_load_2d_pair(sB_lo(stage), mb_lo, fb, kc, brow, pol);
            }
          } else {
            mbar_arrive_expect_tx(&full[stage], C::kStageBytes);
            // Z is re-read by many tiles: keep it in L2 ahead of the
            // evict-first output stream
            tma_load_2d_hint(sA_hi(stage), &tm_hi, &full[stage], kc,
                             (int)row0, pol);
            tma_load_2d_hint(sB_hi(stage), mb_hi, &full[stage], kc,
                             (int)col0, pol);
            tma_load_2d_hint(sB_hi(stage) + kTileA, mb_hi, &full[stage], kc,
                             (int)col0 + kBM, pol);
            if (NPROD > 1) {
              tma_load_2d_hint(sA_lo(stage), &tm_lo, &full[stage], kc,
                               (int)row0, pol);
              tma_load_2d_hint(sB_lo(stage), mb_lo, &full[stage], kc,
                               (int)col0, pol);
              tma_load_2d_hint(sB_lo(stage) + kTileA, mb_lo, &full[stage],
                               kc, (int)col0 + kBM, pol);
            }
          }
          flog->fills[stage] += 1u;
          flog->bytes[stage] = (uint32_t)C::kStageBytes;
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------- MMA issuer
    // (PAIR: the even CTA issues for both)
    if (lane == 0 && (!PAIR || crank == 0)) {
      BandCursor cur;
      band_cursor_init(&cur, p.m, p.G);
      int stage = 0;
      uint32_t phase = 0;
      // the accumulator buffer alternates with every chunk
      int acc = 0;
      uint32_t aphase = 0;
      bool ok = true;
      for (int64_t u = p.u_begin + blockIdx.x; u < p.u_end && ok;
           u += gridDim.x) {
        int64_t row0, col0;
        unit_coords<CROSS>(&cur, p, u, &row0, &col0);
        if (!PAIR && row0 >= n) continue;
        for (int c = 0; c < nch && ok; ++c) {
          if (!mbar_wait(&tempty[acc], aphase ^ 1u, w)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + (uint32_t)(acc * kBN);
          const int kb0 = chunk_begin<KB>(nkb, nch, c);
          const int kb1 = chunk_begin<KB>(nkb, nch, c + 1);
          for (int kb = kb0; kb < kb1; ++kb) {
            if (!mbar_wait(&full[stage], phase, w)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t aH = smem_u32(sA_hi(stage));
            const uint32_t bH = smem_u32(sB_hi(stage));
            const uint32_t aL = smem_u32(sA_lo(stage));
            const uint32_t bL = smem_u32(sB_lo(stage));
#pragma unroll
            for (int ks = 0; ks < KB / kUK; ++ks) {
              const uint32_t off = ks * kUK * 2;  // bytes along K
              const uint64_t dAH = kmajor_desc<C::kSwz>(aH + off);
              const uint64_t dBH = kmajor_desc<C::kSwz>(bH + off);
              auto mma = [&](uint64_t a, uint64_t b, uint32_t acc_in) {
                if constexpr (PAIR)
                  umma_f16_pair(d_tmem, a, b, kIdesc, acc_in);
                else
                  umma_f16(d_tmem, a, b, kIdesc, acc_in);
              };
              mma(dAH, dBH, (kb == kb0 && ks == 0) ? 0u : 1u);
              if (NPROD >= 3) {
                const uint64_t dAL = kmajor_desc<C::kSwz>(aL + off);
                const uint64_t dBL = kmajor_desc<C::kSwz>(bL + off);
                mma(dAH, dBL, 1u);
                mma(dAL, dBH, 1u);
                if (NPROD == 4) mma(dAL, dBL, 1u);
              }
            }
            if constexpr (PAIR)
              umma_commit_pair(&empty[stage], 3);  // frees the stage in both
            else
              umma_commit(&empty[stage]);
            if (++stage == S) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (!ok) break;
          // PAIR: each CTA's epilogue reads its own half of the accumulator
          if constexpr (PAIR)
            umma_commit_pair(&tfull[acc], 3);
          else
            umma_commit(&tfull[acc]);
          acc ^= 1;
          if (acc == 0) aphase ^= 1u;
        }
      }
      // all MMAs issued by this thread complete before TMEM is released
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
    // ---------------------------------------------------------- epilogue
    // 8 warps: warp w reads TMEM lane quarter q = w % 4 (rows 32q..32q+31
    // of the unit) and column half h (columns 128h..128h+127).
    const int q = warp & 3;
    const int h = (warp - 2) >> 2;
    float* stg = epi + (warp - 2) * 32 * kStagePad;
    BandCursor cur;
    band_cursor_init(&cur, p.m, p.G);
    int acc = 0;
    uint32_t aphase = 0;
    const uint32_t lane_off = ((uint32_t)(q * 32) << 16) + (uint32_t)(h * 128);
    // release a TMEM buffer to the MMA issuer (PAIR: the even CTA's)
    auto release = [&](int a) {
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (PAIR && crank != 0)
          tmem_release_cluster(cluster_addr(&tempty[a], 0));
        else
          tmem_release(&tempty[a]);
      }
    };
    for (int64_t u = p.u_begin + blockIdx.x; u < p.u_end; u += gridDim.x) {
      int64_t row0, col0;
      unit_coords<CROSS>(&cur, p, u, &row0, &col0);
      if (!PAIR && row0 >= n) continue;
      const int64_t rbase = row0 + q * 32;  // first row of this warp
      const int64_t jw0 = col0 + h * 128;   // first column of this warp
      // flags do not depend on the accumulator: load them before waiting
      const int64_t my_i = rbase + lane;
      const int rf = (my_i < n) ? p.flags[my_i] : 1;
      int cfl[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int64_t jj = jw0 + c * 32 + lane;
        cfl[c] = (jj < p.ncol) ? p.cflags[jj] : 1;
      }
      // chunks: each finished chunk is added into the next one, whose
      // buffer then holds the unit's running sum
      int last = -1;
      bool ok = true;
      for (int c = 0; c < nch; ++c) {
        bool okw = true;
        if (lane == 0) okw = mbar_wait(&tfull[acc], aphase, w);
        if (!__shfl_sync(0xffffffffu, okw ? 1 : 0, 0)) {
          ok = false;
          break;
        }
        tc_fence_after();
        if (last >= 0) {
          fold_acc(tmem_base + lane_off + (uint32_t)(last * kBN),
                   tmem_base + lane_off + (uint32_t)(acc * kBN));
          release(last);
        }
        last = acc;
        acc ^= 1;
        if (acc == 0) aphase ^= 1u;
      }
      if (!ok) break;
      const uint32_t rflags = __ballot_sync(0xffffffffu, rf != 0);
      // packed index of (rbase, 0); row i+1 starts n - i - 2 later (dense:
      // rbase * ldr, rows ldr apart)
      const int64_t base0 =
          (CROSS ? rbase * p.ldr : pair_row_base(n, rbase)) - p.r_off;
      const EpiOut eo{p.R, p.out_scale, p.tau, p.edges, p.count, p.cap,
                      p.status};
      epilogue_rows<WRITE_R, EDGES, CROSS>(
          tmem_base + lane_off + (uint32_t)(last * kBN), stg, lane, n, rbase,
          jw0, base0, rflags, cfl, eo, p.ncol, p.ldr);
      release(last);
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // every copy issued by this CTA (PAIR: by either CTA) has landed before
  // a CTA of the cluster may exit
  drain_ring<PAIR>(full, nullptr, flog, S, w, crank);
  if (warp == 1) {
    __syncwarp();
    if constexpr (PAIR)
      tmem_dealloc_pair(tmem_base, 512);
    else
      tmem_dealloc(tmem_base, 512);
  }
}

template <int NPROD, bool BF16, bool WRITE_R, bool EDGES, int KB, bool CROSS>
cudaError_t launch_inst(const pcc_zmat* Z, const pcc_zmat* ZB,
                        const TcParams& p, int grid, cudaStream_t s) {
  const CUtensorMap& th = KB == 64 ? Z->tm_hi : Z->tm_hi32;
  const CUtensorMap& tl = KB == 64 ? Z->tm_lo : Z->tm_lo32;
  const CUtensorMap& tbh = KB == 64 ? ZB->tm_hi : ZB->tm_hi32;
  const CUtensorMap& tbl = KB == 64 ? ZB->tm_lo : ZB->tm_lo32;
  const int64_t tiles = (p.u_end - p.u_begin) / 2;
  const TcTuning tn = tc_tuning();
  {
    if (tn.cluster == 2 && tn.pair_mma != 0 && tiles >= 2) {
      auto fn = k_pairs_tc<NPROD, BF16, WRITE_R, EDGES, KB, CROSS, true>;
      const int smem = Cfg<NPROD, KB, true>::kSmemBytes;
      cudaError_t e =
          ensure_func_smem(reinterpret_cast<const void*>(fn), smem);
      if (e != cudaSuccess) return e;
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 2;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.blockDim = dim3(kThreads, 1, 1);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = s;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      // per template instance and device
      static int max_clusters_of[kDeviceSlots] = {};
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
      int64_t ncl = tiles < max_clusters ? tiles : max_clusters;
      cfg.gridDim = dim3((unsigned)(2 * ncl), 1, 1);
      e = cudaLaunchKernelEx(&cfg, fn, th, tl, tbh, tbl, p);
      if (e != cudaSuccess) return e;
      return cudaGetLastError();
    }
  }
  auto fn = k_pairs_tc<NPROD, BF16, WRITE_R, EDGES, KB, CROSS, false>;
  const int smem = Cfg<NPROD, KB, false>::kSmemBytes;
  cudaError_t e = ensure_func_smem(reinterpret_cast<const void*>(fn), smem);
  if (e != cudaSuccess) return e;
  fn<<<grid, kThreads, smem, s>>>(th, tl, tbh, tbl, p);
  return cudaGetLastError();
}

template <int NPROD, bool BF16, int KB, bool CROSS>
cudaError_t launch_prec(const pcc_zmat* Z, const pcc_zmat* ZB,
                        const TcParams& p, int grid, bool write_r,
                        bool edges_on, cudaStream_t s) {
  if (write_r && edges_on)
    return launch_inst<NPROD, BF16, true, true, KB, CROSS>(Z, ZB, p, grid, s);
  if (edges_on)
    return launch_inst<NPROD, BF16, false, true, KB, CROSS>(Z, ZB, p, grid,
                                                            s);
  return launch_inst<NPROD, BF16, true, false, KB, CROSS>(Z, ZB, p, grid, s);
}

template <int KB, bool CROSS>
cudaError_t launch_kb(const pcc_zmat* Z, const pcc_zmat* ZB, TcParams& p,
                      int grid, bool write_r, bool edges_on, cudaStream_t s) {
  p.nkb = (int)(Z->lpad / KB);
  p.nch = accum_chunks(Z->lpad);
  switch (Z->prec) {
    case PCC_PREC_BF16X3:
      return launch_prec<3, true, KB, CROSS>(Z, ZB, p, grid, write_r,
                                             edges_on, s);
    case PCC_PREC_FP16X3S:
      return launch_prec<3, false, KB, CROSS>(Z, ZB, p, grid, write_r,
                                              edges_on, s);
    case PCC_PREC_BF16X4:
      return launch_prec<4, true, KB, CROSS>(Z, ZB, p, grid, write_r,
                                             edges_on, s);
    case PCC_PREC_BF16X1:
      return launch_prec<1, true, KB, CROSS>(Z, ZB, p, grid, write_r,
                                             edges_on, s);
    default:
      return cudaErrorInvalidValue;
  }
}

TcParams base_params(const pcc_zmat* Z, float* R, float tau,
                     pcc_edge* edges, uint64_t cap,
                     unsigned long long* count) {
  TcParams p;
  p.n = Z->n;
  p.m = tc_super_count(Z->n);
  p.ncol = Z->n;
  p.mcol = 0;
  p.ldr = 0;
  p.r_off = 0;
  p.cflags = Z->flags;
  p.G = tc_tuning().band;
  p.out_scale = (float)ldexp(1.0, -2 * Z->scale_exp);
  p.tau = tau;
  p.flags = Z->flags;
  p.R = R;
  p.edges = edges;
  p.count = count;
  p.cap = cap;
  p.status = Z->status;
  p.wait_ns = wait_limit_ns();
  p.drop_loads = debug_drop_loads();
  return p;
}

}  // namespace

int64_t tc_num_tiles(int64_t n) {
  const int64_t m = tc_super_count(n);
  return m * (m + 1) / 2;
}

cudaError_t launch_tc_pairs(const pcc_zmat* Z, float* R, int64_t t0,
                            int64_t t1, bool edges_on, float tau,
                            pcc_edge* edges, uint64_t cap,
                            unsigned long long* count, cudaStream_t s,
                            int64_t r_off, int64_t G) {
  if (t1 <= t0) return cudaSuccess;
  TcParams p = base_params(Z, R, tau, edges, cap, count);
  p.r_off = r_off;
  if (G > 0) p.G = G;
  p.u_begin = 2 * t0;
  p.u_end = 2 * t1;
  const int64_t units = p.u_end - p.u_begin;
  int grid = num_sms(Z->device);
  if (units < grid) grid = (int)units;
  const bool write_r = R != nullptr;
  if (tc_tuning().stage_k == 64)
    return launch_kb<64, false>(Z, Z, p, grid, write_r, edges_on, s);
  return launch_kb<32, false>(Z, Z, p, grid, write_r, edges_on, s);
}

int64_t tc_cross_tiles(int64_t na, int64_t nb) {
  return tc_super_count(na) * tc_super_count(nb);
}

cudaError_t launch_tc_cross(const pcc_zmat* ZA, const pcc_zmat* ZB, float* R,
                            int64_t ldr, int64_t t0, int64_t t1,
                            bool edges_on, float tau, pcc_edge* edges,
                            uint64_t cap, unsigned long long* count,
                            cudaStream_t s, int64_t r_off, int64_t G) {
  if (t1 <= t0) return cudaSuccess;
  TcParams p = base_params(ZA, R, tau, edges, cap, count);
  p.r_off = r_off;
  if (G > 0) p.G = G;
  p.ncol = ZB->n;
  p.mcol = tc_super_count(ZB->n);
  p.ldr = ldr;
  p.cflags = ZB->flags;
  p.u_begin = 2 * t0;
  p.u_end = 2 * t1;
  const int64_t units = p.u_end - p.u_begin;
  int grid = num_sms(ZA->device);
  if (units < grid) grid = (int)units;
  if (tc_tuning().stage_k == 64)
    return launch_kb<64, true>(ZA, ZB, p, grid, R != nullptr, edges_on, s);
  return launch_kb<32, true>(ZA, ZB, p, grid, R != nullptr, edges_on, s);
}

}  // namespace pcc
