// tc_batched.cu -- K7: all pairs of many matrices of uneven n and l in one
// persistent tensor-core launch.
//
// Every matrix b keeps its own standardized halves, TMA maps, flags and
// packed output; a device array of descriptors holds them.  The work units
// of all matrices (128 x 256 halves of 256 x 256 super-tiles, banded order
// of pcc_sched.h per matrix) are assigned to the CTAs on the host: units
// are taken longest first and each goes to the CTA with the least estimated
// work so far (cost = c0 + c1 * K-blocks * products), then each CTA's list
// is put back in (matrix, unit) order so that CTAs walk the matrices
// together.  The split form (3 products or 1, BF16 or FP16 halves) is read
// per matrix at run time, so one kernel serves the whole batch.
//
// Same roles, pipeline and bounded waits as the single-matrix kernel
// (tc_pairs.cu), K = 32 or 64 per stage (the stage_k knob); matrices with
// rows longer than 1024 accumulate their units in chunks as that kernel does
// (tc_common.cuh).  With the pair form (pcc_set_pair_mma, the default) the plan hands whole super-tiles to
// CTA pairs, which run one 2-SM MMA per tile (M = 256, each CTA loading its
// 128 A rows and 128 of the B rows, as in tc_pairs.cu); otherwise single
// CTAs take units.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <queue>
#include <vector>

#include "pcc_internal.h"
#include "pcc_ptx.cuh"
#include "pcc_sched.h"
#include "tc_common.cuh"
#include "tc_epilogue.cuh"

namespace pcc {
namespace {

constexpr int kBM = 128, kBN = 256, kUK = 16;
constexpr int kThreads = 320, kEpiWarps = 8;
constexpr int kEpiBytes = kEpiWarps * 32 * kStagePad * 4;
// KB = K per stage (32 or 64, the stage_k knob); PAIR: each CTA holds 128
// of the 256 B rows, so its stages are a third smaller
template <bool PAIR, int KB>
struct BCfg {
  static constexpr int kTileA = kBM * KB * 2;
  static constexpr int kTileB = (PAIR ? kBM : kBN) * KB * 2;
  static constexpr int kStageBytes = 2 * (kTileA + kTileB);  // 3 products
  static constexpr int kStages = (4 * 49152) / kStageBytes;
  static constexpr int kBarBytes = 512;
  static constexpr int kSmemBytes =
      1024 + kStages * kStageBytes + kEpiBytes + kBarBytes;
  static_assert(kSmemBytes <= 232448, "shared memory budget");
};

// takes the 128-byte alignment of its tensor maps (TMA reads them from
// global memory)
struct MatDesc {
  CUtensorMap tm_hi;  // box 32 x 128, 64-B swizzle
  CUtensorMap tm_lo;
  int64_t n;
  int64_t m;          // super-tiles per side
  int nkb;            // K blocks of 32
  int nprod;          // 4, 3 or 1 products per K step
  int nch;            // accumulator chunks per unit (tc_common.cuh)
  int64_t G;          // super-tile rows per band of this matrix's order
  uint32_t idesc;     // MMA instruction descriptor (BF16 or FP16 halves)
  float scale;        // accumulator -> r
  const uint8_t* flags;
  float* R;
};

struct BatchParams {
  const MatDesc* descs;
  const uint64_t* items;   // (matrix << 40) | unit (PAIR: | tile)
  const int64_t* cta_off;  // items of CTA (PAIR: CTA pair) c:
                           // [cta_off[c], cta_off[c+1])
  int* status;
  uint64_t wait_ns;
};

constexpr int kItemShift = 40;
constexpr uint64_t kItemMask = (1ull << kItemShift) - 1;

template <bool PAIR, int KB>
__global__ void __launch_bounds__(kThreads, 1)
    k_pairs_tc_batched(const BatchParams p) {
  using C = BCfg<PAIR, KB>;
  constexpr int kTileA = C::kTileA;
  constexpr int kTileB = C::kTileB;
  constexpr int kStageBytes = C::kStageBytes;
  constexpr int kStages = C::kStages;
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned base, kept as an offset from the shared array so
  // that accesses through it compile to shared-memory instructions
  uint8_t* smem =
      smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t* ring = smem;
  float* epi = reinterpret_cast<float*>(smem + kStages * kStageBytes);
  uint64_t* bars =
      reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes + kEpiBytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + kStages;
  uint64_t* tfull = bars + 2 * kStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* mdone = tempty + 2;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(mdone + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  FillLog* flog = reinterpret_cast<FillLog*>(bars + 32);
  static_assert(2 * kStages + 5 <= 31, "barrier area");
  static_assert(32 * 8 + sizeof(FillLog) <= C::kBarBytes, "barrier area");
  auto sA_hi = [&](int s) { return ring + s * kStageBytes; };
  auto sB_hi = [&](int s) { return ring + s * kStageBytes + kTileA; };
  auto sA_lo = [&](int s) { return ring + s * kStageBytes + kTileA + kTileB; };
  auto sB_lo = [&](int s) {
    return ring + s * kStageBytes + 2 * kTileA + kTileB;
  };

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      // PAIR: the even CTA's barrier counts both CTAs' epilogue warps
      mbar_init(&tempty[a], PAIR ? 2 * kEpiWarps : kEpiWarps);
    }
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
  WaitCtx w{abort_flag, p.status, p.wait_ns};
  const int64_t wid = PAIR ? (int64_t)(blockIdx.x >> 1) : (int64_t)blockIdx.x;
  const int64_t it0 = p.cta_off[wid], it1 = p.cta_off[wid + 1];

  // unit coordinates; the band cursor restarts when the matrix changes
  struct Walk {
    int64_t b = -1;
    BandCursor cur;
  };
  auto coords = [&](Walk& wk, uint64_t item, const MatDesc*& d,
                    int64_t* row0, int64_t* col0) {
    const int64_t b = (int64_t)(item >> kItemShift);
    const int64_t u = (int64_t)(item & kItemMask);
    d = p.descs + b;
    if (b != wk.b) {
      wk.b = b;
      band_cursor_init(&wk.cur, d->m, d->G);
    }
    // PAIR items are tiles, CTA rank h takes half h; else items are units
    const int64_t t = PAIR ? u : (u >> 1);
    const int64_t half = PAIR ? (int64_t)crank : (u & 1);
    int64_t yt, xt;
    band_tile_coords(&wk.cur, d->m, d->G, t, &yt, &xt);
    *row0 = yt * kTcSuper + half * kBM;
    *col0 = xt * kTcSuper;
  };

  if (warp == 0) {
    if (lane == 0) {
      const uint64_t pol = l2_policy_evict_last();
      Walk wk;
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int64_t it = it0; it < it1 && ok; ++it) {
        const MatDesc* d;
        int64_t row0, col0;
        coords(wk, p.items[it], d, &row0, &col0);
        const int nkb = d->nkb, nprod = d->nprod;
        const uint32_t bytes =
            nprod >= 3 ? (uint32_t)kStageBytes : (uint32_t)(kTileA + kTileB);
        for (int kb = 0; kb < nkb; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, w)) {
            ok = false;
            break;
          }
          const int kc = kb * KB;
          if constexpr (PAIR) {
            // each CTA: its 128 A rows and 128 of the B rows; both CTAs'
            // bytes count on the even CTA's barrier
            if (crank == 0) mbar_arrive_expect_tx(&full[stage], 2 * bytes);
            const uint32_t fb = cluster_addr(&full[stage], 0);
            const int brow = (int)(col0 + crank * kBM);
            tma_load_2d_pair(sA_hi(stage), &d->tm_hi, fb, kc, (int)row0, pol);
            tma_load_2d_pair(sB_hi(stage), &d->tm_hi, fb, kc, brow, pol);
            if (nprod >= 3) {
              tma_load_2d_pair(sA_lo(stage), &d->tm_lo, fb, kc, (int)row0,
                               pol);
              tma_load_2d_pair(sB_lo(stage), &d->tm_lo, fb, kc, brow, pol);
            }
          } else {
            mbar_arrive_expect_tx(&full[stage], bytes);
            tma_load_2d_hint(sA_hi(stage), &d->tm_hi, &full[stage], kc,
                             (int)row0, pol);
            tma_load_2d_hint(sB_hi(stage), &d->tm_hi, &full[stage], kc,
                             (int)col0, pol);
            tma_load_2d_hint(sB_hi(stage) + kTileA, &d->tm_hi, &full[stage], kc,
                             (int)col0 + kBM, pol);
            if (nprod >= 3) {
              tma_load_2d_hint(sA_lo(stage), &d->tm_lo, &full[stage], kc,
                               (int)row0, pol);
              tma_load_2d_hint(sB_lo(stage), &d->tm_lo, &full[stage], kc,
                               (int)col0, pol);
              tma_load_2d_hint(sB_lo(stage) + kTileA, &d->tm_lo, &full[stage],
                               kc, (int)col0 + kBM, pol);
            }
          }
          flog->fills[stage] += 1u;
          flog->bytes[stage] = bytes;
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
    }
  } else if (warp == 1) {
    // MMA issuer (PAIR: the even CTA issues for both)
    if (lane == 0 && (!PAIR || crank == 0)) {
      Walk wk;
      int stage = 0, acc = 0;
      uint32_t phase = 0, aphase = 0;
      bool ok = true;
      for (int64_t it = it0; it < it1 && ok; ++it) {
        const MatDesc* d;
        int64_t row0, col0;
        coords(wk, p.items[it], d, &row0, &col0);
        const int nkb = d->nkb, nprod = d->nprod, nch = d->nch;
        const uint32_t idesc = d->idesc;
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
              const uint32_t off = ks * kUK * 2;
              const uint64_t dAH = kmajor_desc<2 * KB>(aH + off);
              const uint64_t dBH = kmajor_desc<2 * KB>(bH + off);
              auto mma = [&](uint64_t a, uint64_t b, uint32_t acc_in) {
                if constexpr (PAIR)
                  umma_f16_pair(d_tmem, a, b, idesc, acc_in);
                else
                  umma_f16(d_tmem, a, b, idesc, acc_in);
              };
              mma(dAH, dBH, (kb == kb0 && ks == 0) ? 0u : 1u);
              if (nprod >= 3) {
                mma(dAH, kmajor_desc<2 * KB>(bL + off), 1u);
                mma(kmajor_desc<2 * KB>(aL + off), dBH, 1u);
                if (nprod == 4)
                  mma(kmajor_desc<2 * KB>(aL + off), kmajor_desc<2 * KB>(bL + off),
                      1u);
              }
            }
            if constexpr (PAIR)
              umma_commit_pair(&empty[stage], 3);  // frees it in both CTAs
            else
              umma_commit(&empty[stage]);
            if (++stage == kStages) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (!ok) break;
          if constexpr (PAIR)
            umma_commit_pair(&tfull[acc], 3);
          else
            umma_commit(&tfull[acc]);
          acc ^= 1;
          if (acc == 0) aphase ^= 1u;
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
    const int q = warp & 3;
    const int h = (warp - 2) >> 2;
    float* stg = epi + (warp - 2) * 32 * kStagePad;
    Walk wk;
    int acc = 0;
    uint32_t aphase = 0;
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
    for (int64_t it = it0; it < it1; ++it) {
      const MatDesc* d;
      int64_t row0, col0;
      coords(wk, p.items[it], d, &row0, &col0);
      const int64_t n = d->n;
      const int64_t rbase = row0 + q * 32;
      const int64_t jw0 = col0 + h * 128;
      const int64_t my_i = rbase + lane;
      const int rf = (my_i < n) ? d->flags[my_i] : 1;
      int cfl[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int64_t jj = jw0 + c * 32 + lane;
        cfl[c] = (jj < n) ? d->flags[jj] : 1;
      }
      const EpiOut eo{d->R, d->scale, 2.f, nullptr, nullptr, 0, p.status};
      const uint32_t lane_off =
          ((uint32_t)(q * 32) << 16) + (uint32_t)(h * 128);
      // chunks: each finished chunk is added into the next one
      int last = -1;
      bool ok = true;
      for (int c = 0; c < d->nch; ++c) {
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
      const int64_t base0 = pair_row_base(n, rbase);
      epilogue_rows<true, false>(tmem_base + lane_off + (uint32_t)(last * kBN),
                                 stg, lane, n, rbase, jw0, base0, rflags, cfl,
                                 eo);
      release(last);
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // every copy issued by this CTA (PAIR: by either CTA) has landed before
  // a CTA of the pair may exit
  drain_ring<PAIR>(full, nullptr, flog, kStages, w, crank);
  if (warp == 1) {
    __syncwarp();
    if constexpr (PAIR)
      tmem_dealloc_pair(tmem_base, 512);
    else
      tmem_dealloc(tmem_base, 512);
  }
}

// ------------------------------------------------------------- host plan
// One persistent launch over the matrices of one CTA form (a kernel runs
// either 1-SM or 2-SM MMAs, never both).
struct Launch {
  bool pair = false;     // items are tiles for CTA pairs (2-SM MMA)
  int kb = 32;           // K per stage
  int grid = 0;          // CTAs
  void* dmem = nullptr;  // descs | cta_off | items
  MatDesc* d_descs = nullptr;
  int64_t* d_off = nullptr;
  uint64_t* d_items = nullptr;
};

struct Plan {
  std::vector<const pcc_zmat*> zs;
  std::vector<float*> rs;
  // per matrix: n, lpad, prec, hi address, pair form, band rows
  std::vector<int64_t> sig;
  double cost_c0 = 0, cost_c1 = 0;
  int64_t one_acc_l = 0, chunk_l = 0;
  int stage_k = 32;
  int device = -1;
  Launch L[2];  // 2-SM pair matrices, then single-CTA matrices
  int nlaunch = 0;
};

constexpr int kSig = 6;

std::mutex g_plan_mu;
std::vector<Plan*> g_plans;  // small cache, most recent last

void free_plan(Plan* P) {
  for (int k = 0; k < 2; ++k)
    if (P->L[k].dmem) cudaFree(P->L[k].dmem);
  delete P;
}

// CTA pairs of the pair form that can be resident at once
template <int KB>
int pair_workers(int device) {
  static int mc_of[kDeviceSlots] = {};
  int& mc = mc_of[device_slot(device)];
  if (mc == 0) {
    auto fn = k_pairs_tc_batched<true, KB>;
    const int smem = BCfg<true, KB>::kSmemBytes;
    int v = 0;
    if (ensure_func_smem(reinterpret_cast<const void*>(fn), smem) ==
        cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 2;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.blockDim = dim3(kThreads, 1, 1);
      cfg.dynamicSmemBytes = smem;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      cfg.gridDim = dim3(2 * (unsigned)(num_sms(device) / 2), 1, 1);
      if (cudaOccupancyMaxActiveClusters(&v, fn, &cfg) != cudaSuccess) v = 0;
    }
    cudaGetLastError();
    mc = v > 0 ? v : num_sms(device) / 2;
  }
  return mc;
}

// Work list of one launch over the matrices `mats` (indices into P->zs):
// every unit (pair form: every tile) costs c0 + c1 * K-blocks * products;
// longest first, each to the least-loaded worker, then each worker's list
// in (matrix, unit) order.
bool build_launch(Plan* P, Launch* L, const std::vector<int>& mats,
                  bool pair, int KB) {
  const int B = (int)mats.size();
  const int sms = num_sms(P->device);
  std::vector<MatDesc> descs(B);
  struct U {
    double cost;
    uint64_t item;
  };
  std::vector<U> units;
  for (int lb = 0; lb < B; ++lb) {
    const int b = mats[lb];
    const pcc_zmat* Z = P->zs[b];
    MatDesc& d = descs[lb];
    memset(&d, 0, sizeof(d));
    // K = 64 stages: box 64 x 128, 128-byte swizzle; K = 32: 32 x 128, 64-B
    d.tm_hi = KB == 64 ? Z->tm_hi : Z->tm_hi32;
    d.tm_lo = KB == 64 ? Z->tm_lo : Z->tm_lo32;
    d.n = Z->n;
    d.m = tc_super_count(Z->n);
    d.nkb = (int)(Z->lpad / KB);
    d.nprod = Z->prec == PCC_PREC_BF16X1   ? 1
              : Z->prec == PCC_PREC_BF16X4 ? 4
                                           : 3;
    d.nch = accum_chunks(Z->lpad);
    d.G = P->sig[kSig * b + 5];
    // the pair form's one instruction covers both CTAs' 128 rows
    d.idesc =
        make_idesc_f16(Z->prec != PCC_PREC_FP16X3S, pair ? 2 * kBM : kBM, kBN);
    d.scale = (float)ldexp(1.0, -2 * Z->scale_exp);
    d.flags = Z->flags;
    d.R = P->rs[b];
    // a unit's cost (c1 per 32 samples and product, whatever the stage
    // size); a tile of the pair form costs the same (its two halves run
    // side by side on the pair)
    const double cost =
        P->cost_c0 + P->cost_c1 * (double)(Z->lpad / 32) * d.nprod;
    if (pair) {
      const int64_t nt = tc_num_tiles(Z->n);
      for (int64_t t = 0; t < nt; ++t)
        units.push_back({cost, ((uint64_t)lb << kItemShift) | (uint64_t)t});
      continue;
    }
    const int64_t nu = 2 * tc_num_tiles(Z->n);
    BandCursor cur;
    band_cursor_init(&cur, d.m, d.G);
    for (int64_t u = 0; u < nu; ++u) {
      int64_t yt, xt;
      band_tile_coords(&cur, d.m, d.G, u >> 1, &yt, &xt);
      if (yt * kTcSuper + (u & 1) * kBM >= Z->n) continue;  // empty half
      units.push_back({cost, ((uint64_t)lb << kItemShift) | (uint64_t)u});
    }
  }
  const int64_t total = (int64_t)units.size();
  // workers: CTAs, or CTA pairs in the pair form
  const int64_t nw = pair ? (KB == 64 ? pair_workers<64>(P->device)
                                      : pair_workers<32>(P->device))
                         : sms;
  int grid = (int)std::min<int64_t>(nw, std::max<int64_t>(total, 1));
  std::stable_sort(units.begin(), units.end(),
                   [](const U& a, const U& b) { return a.cost > b.cost; });
  typedef std::pair<double, int> Ld;
  std::priority_queue<Ld, std::vector<Ld>, std::greater<Ld>> heap;
  for (int c = 0; c < grid; ++c) heap.push({0.0, c});
  std::vector<std::vector<uint64_t>> per(grid);
  for (const U& u : units) {
    Ld top = heap.top();
    heap.pop();
    per[top.second].push_back(u.item);
    heap.push({top.first + u.cost, top.second});
  }
  std::vector<int64_t> off(grid + 1, 0);
  std::vector<uint64_t> items;
  items.reserve(total);
  for (int c = 0; c < grid; ++c) {
    std::sort(per[c].begin(), per[c].end());
    off[c] = (int64_t)items.size();
    items.insert(items.end(), per[c].begin(), per[c].end());
  }
  off[grid] = (int64_t)items.size();
  const size_t bd = sizeof(MatDesc) * B;
  const size_t bo = sizeof(int64_t) * (grid + 1);
  const size_t bi = sizeof(uint64_t) * std::max<size_t>(items.size(), 1);
  const size_t o_off = (bd + 255) / 256 * 256;
  const size_t o_items = o_off + (bo + 255) / 256 * 256;
  if (cudaMalloc(&L->dmem, o_items + bi) != cudaSuccess) {
    cudaGetLastError();
    L->dmem = nullptr;
    return false;
  }
  uint8_t* base = static_cast<uint8_t*>(L->dmem);
  L->d_descs = reinterpret_cast<MatDesc*>(base);
  L->d_off = reinterpret_cast<int64_t*>(base + o_off);
  L->d_items = reinterpret_cast<uint64_t*>(base + o_items);
  if (cudaMemcpy(L->d_descs, descs.data(), bd, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(L->d_off, off.data(), bo, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      (!items.empty() &&
       cudaMemcpy(L->d_items, items.data(), sizeof(uint64_t) * items.size(),
                  cudaMemcpyHostToDevice) != cudaSuccess)) {
    cudaFree(L->dmem);
    L->dmem = nullptr;
    return false;
  }
  L->pair = pair;
  L->kb = KB;
  L->grid = pair ? 2 * grid : grid;
  return true;
}

bool build_plan(Plan* P) {
  std::vector<int> by_form[2];  // 0: pair form, 1: single CTAs
  for (int b = 0; b < (int)P->zs.size(); ++b)
    by_form[P->sig[kSig * b + 4] ? 0 : 1].push_back(b);
  for (int f = 0; f < 2; ++f) {
    if (by_form[f].empty()) continue;
    if (!build_launch(P, &P->L[P->nlaunch], by_form[f], f == 0,
                      P->stage_k))
      return false;
    ++P->nlaunch;
  }
  return true;
}

template <bool PAIR, int KB>
cudaError_t launch_form(const Launch& L, const BatchParams& bp,
                        cudaStream_t s) {
  auto fn = k_pairs_tc_batched<PAIR, KB>;
  const int smem = BCfg<PAIR, KB>::kSmemBytes;
  cudaError_t e = ensure_func_smem(reinterpret_cast<const void*>(fn), smem);
  if (e != cudaSuccess) return e;
  if constexpr (PAIR) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)L.grid, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, fn, bp);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  fn<<<L.grid, kThreads, smem, s>>>(bp);
  return cudaGetLastError();
}

cudaError_t launch_one(const Launch& L, const BatchParams& bp,
                       cudaStream_t s) {
  if (L.pair)
    return L.kb == 64 ? launch_form<true, 64>(L, bp, s)
                      : launch_form<true, 32>(L, bp, s);
  return L.kb == 64 ? launch_form<false, 64>(L, bp, s)
                    : launch_form<false, 32>(L, bp, s);
}

}  // namespace

pcc_status allpairs_batched(const pcc_zmat* const* Zs, int32_t B,
                            float* const* Rs, const int32_t* pair,
                            const int32_t* band, cudaStream_t s) {
  const TcTuning tn = tc_tuning();
  const int dev = Zs[0]->device;
  // per matrix: n, lpad, prec, hi address, form, band rows
  std::vector<int64_t> sig;
  sig.reserve((size_t)kSig * B);
  for (int b = 0; b < B; ++b) {
    sig.push_back(Zs[b]->n);
    sig.push_back(Zs[b]->lpad);
    sig.push_back((int64_t)Zs[b]->prec);
    sig.push_back((int64_t)(uintptr_t)Zs[b]->hi);
    sig.push_back(pair ? (pair[b] != 0) : (tn.pair_mma != 0 &&
                                           tn.cluster == 2));
    sig.push_back(band ? band[b] : tn.band);
  }
  Plan* P = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_plan_mu);
    for (Plan* q : g_plans) {
      if ((int)q->zs.size() != B || q->device != dev) continue;
      bool same = q->cost_c0 == tn.cost_c0 && q->cost_c1 == tn.cost_c1 &&
                  q->stage_k == tn.stage_k &&
                  q->one_acc_l == tn.one_acc_l && q->chunk_l == tn.chunk_l &&
                  q->sig == sig;
      for (int b = 0; b < B && same; ++b)
        same = q->zs[b] == Zs[b] && q->rs[b] == Rs[b];
      if (same) {
        P = q;
        break;
      }
    }
    if (!P) {
      P = new Plan();
      P->zs.assign(Zs, Zs + B);
      P->rs.assign(Rs, Rs + B);
      P->sig = sig;
      P->cost_c0 = tn.cost_c0;
      P->cost_c1 = tn.cost_c1;
      P->one_acc_l = tn.one_acc_l;
      P->chunk_l = tn.chunk_l;
      P->stage_k = tn.stage_k;
      P->device = dev;
      if (!build_plan(P)) {
        free_plan(P);
        return PCC_ERR_OOM;
      }
      g_plans.push_back(P);
      if (g_plans.size() > 8) {
        Plan* old = g_plans.front();
        cudaDeviceSynchronize();  // its last launch may be on any stream
        free_plan(old);
        g_plans.erase(g_plans.begin());
      }
    }
  }
  for (int k = 0; k < P->nlaunch; ++k) {
    BatchParams bp;
    bp.descs = P->L[k].d_descs;
    bp.items = P->L[k].d_items;
    bp.cta_off = P->L[k].d_off;
    bp.status = Zs[0]->status;
    bp.wait_ns = wait_limit_ns();
    const cudaError_t e = launch_one(P->L[k], bp, s);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return PCC_OK;
}

}  // namespace pcc
