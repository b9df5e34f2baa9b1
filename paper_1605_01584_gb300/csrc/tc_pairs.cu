// tc_pairs.cu -- K2 / K3: all-pairs r(i,j) = z_i . z_j (Eq. (6)) on the
// tcgen05 tensor cores, with the packed-triangle and |r| >= tau epilogues
// fused.
//
// Precision: z = hi + lo (two 16-bit halves, written by the variable
// transformation).  Per tile the MMAs accumulate, in FP32 in TMEM,
//     hi_Y hi_X^T + hi_Y lo_X^T + lo_Y hi_X^T          (3 products)
// which recovers z_Y z_X^T up to the dropped lo lo^T term; BF16X1 runs the
// first product only.
//
// Work decomposition (pcc_sched.h): 256 x 256 super-tiles of the upper
// triangle in banded order, each split into two units of 128 rows x 256
// columns.  A persistent grid (one CTA per SM) strides over the units, as
// Algorithm 1 strides thread groups over tile ids.
//
// CTA roles (192 threads):
//   warp 0      TMA producer: per K block of 64, loads A = rows of the unit
//               (hi, lo: 128 x 64 each) and B = its columns (hi, lo: 256 x
//               64 each) into a ring of shared-memory stages (128-B swizzle).
//   warp 1      allocates 512 TMEM columns (two 128 x 256 FP32
//               accumulators) and one elected thread issues the MMAs
//               (M = 128, N = 256, K = 16 per instruction), committing each
//               stage back to the producer and each finished accumulator to
//               the epilogue.
//   warps 2-5   epilogue: tcgen05.ld of the accumulator (warp w reads TMEM
//               lanes 32*(w%4)..+31 = its 32 rows), a transpose through
//               shared memory so that a warp stores 32 consecutive pairs of
//               one row at a time (rows of the packed triangle are
//               contiguous), clamp to [-1,1], NaN for flagged rows, and the
//               optional warp-aggregated edge append.
// The two accumulators let the epilogue of one unit overlap the MMAs of the
// next.  Every wait is bounded (pcc_ptx.cuh): a wait that runs out records
// PCC_ERR_TIMEOUT and the CTA drains its copies, frees TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include "pcc_internal.h"
#include "pcc_ptx.cuh"
#include "pcc_sched.h"

namespace pcc {
namespace {

constexpr int kBM = 128;   // rows per unit (MMA M)
constexpr int kBN = 256;   // columns per unit (MMA N)
constexpr int kBK = 64;    // K per stage: one 128-B swizzle row of 16-bit
constexpr int kUK = 16;    // K per tcgen05.mma kind::f16
constexpr int kThreads = 192;
constexpr int kEpiWarps = 4;
constexpr int kTileA = kBM * kBK * 2;  // 16 KB
constexpr int kTileB = kBN * kBK * 2;  // 32 KB
constexpr int kStagePad = 33;          // epilogue transpose row pitch
constexpr int kGroupG = 8;             // super-tile rows per band

struct TcParams {
  int64_t n;
  int64_t m;         // super-tiles per side
  int64_t u_begin;   // units [u_begin, u_end)
  int64_t u_end;
  int nkb;           // K blocks of 64
  float out_scale;   // 2^-2s for FP16X3S, else 1
  float tau;
  const uint8_t* flags;
  float* R;
  pcc_edge* edges;
  unsigned long long* count;
  uint64_t cap;
  int* status;
  uint64_t wait_ns;
};

template <int NPROD>
struct Cfg {
  static constexpr int kStages = NPROD == 1 ? 4 : 2;
  static constexpr int kStageBytes = NPROD == 1 ? (kTileA + kTileB)
                                                : 2 * (kTileA + kTileB);
  static constexpr int kRingBytes = kStages * kStageBytes;
  static constexpr int kEpiBytes = kEpiWarps * 32 * kStagePad * 4;
  static constexpr int kBarBytes = 256;
  static constexpr int kSmemBytes = 1024 + kRingBytes + kEpiBytes + kBarBytes;
};

__device__ __forceinline__ void unit_coords(BandCursor* cur, const TcParams& p,
                                            int64_t u, int64_t* row0,
                                            int64_t* col0) {
  int64_t yt, xt;
  band_tile_coords(cur, p.m, kGroupG, u >> 1, &yt, &xt);
  *row0 = yt * kTcSuper + (u & 1) * kBM;
  *col0 = xt * kTcSuper;
}

template <int NPROD, bool BF16, bool WRITE_R, bool EDGES>
__global__ void __launch_bounds__(kThreads, 1)
    k_pairs_tc(const __grid_constant__ CUtensorMap tm_hi,
               const __grid_constant__ CUtensorMap tm_lo, const TcParams p) {
  using C = Cfg<NPROD>;
  constexpr int S = C::kStages;
  constexpr uint32_t kIdesc = make_idesc_f16(BF16, kBM, kBN);

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
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
      mbar_init(&tempty[a], kEpiWarps);
    }
    mbar_init(mdone, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    tma_prefetch_desc(&tm_hi);
    if (NPROD > 1) tma_prefetch_desc(&tm_lo);
  }
  if (warp == 1) {
    tmem_alloc(tmem_holder, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;

  WaitCtx w{abort_flag, p.status, p.wait_ns};
  const int64_t n = p.n;

  if (warp == 0) {
    // ------------------------------------------------------ TMA producer
    if (lane == 0) {
      BandCursor cur;
      band_cursor_init(&cur, p.m, kGroupG);
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_mask = 0;
      uint32_t last_phase[S];
      for (int s = 0; s < S; ++s) last_phase[s] = 0;
      for (int64_t u = p.u_begin + blockIdx.x; u < p.u_end; u += gridDim.x) {
        int64_t row0, col0;
        unit_coords(&cur, p, u, &row0, &col0);
        if (row0 >= n) continue;
        bool ok = true;
        for (int kb = 0; kb < p.nkb; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, w)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[stage], C::kStageBytes);
          const int kc = kb * kBK;
          tma_load_2d(sA_hi(stage), &tm_hi, &full[stage], kc, (int)row0);
          tma_load_2d(sB_hi(stage), &tm_hi, &full[stage], kc, (int)col0);
          tma_load_2d(sB_hi(stage) + kTileA, &tm_hi, &full[stage], kc,
                      (int)col0 + kBM);
          if (NPROD > 1) {
            tma_load_2d(sA_lo(stage), &tm_lo, &full[stage], kc, (int)row0);
            tma_load_2d(sB_lo(stage), &tm_lo, &full[stage], kc, (int)col0);
            tma_load_2d(sB_lo(stage) + kTileA, &tm_lo, &full[stage], kc,
                        (int)col0 + kBM);
          }
          issued_mask |= 1u << stage;
          last_phase[stage] = phase;
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
      }
      // drain: every issued copy must land before the CTA may exit
      WaitCtx wd = w;
      volatile int never = 0;
      wd.abort_flag = &never;
      for (int s = 0; s < S; ++s)
        if (issued_mask & (1u << s)) mbar_wait(&full[s], last_phase[s], wd);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------- MMA issuer
    if (lane == 0) {
      BandCursor cur;
      band_cursor_init(&cur, p.m, kGroupG);
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t aphase = 0;
      for (int64_t u = p.u_begin + blockIdx.x; u < p.u_end; u += gridDim.x) {
        int64_t row0, col0;
        unit_coords(&cur, p, u, &row0, &col0);
        if (row0 >= n) continue;
        if (!mbar_wait(&tempty[acc], aphase ^ 1u, w)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(acc * kBN);
        bool ok = true;
        for (int kb = 0; kb < p.nkb; ++kb) {
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
          for (int ks = 0; ks < kBK / kUK; ++ks) {
            const uint32_t off = ks * kUK * 2;  // bytes along K
            const uint64_t dAH = sw128_kmajor_desc(aH + off);
            const uint64_t dBH = sw128_kmajor_desc(bH + off);
            umma_f16(d_tmem, dAH, dBH, kIdesc, (kb | ks) != 0);
            if (NPROD == 3) {
              const uint64_t dAL = sw128_kmajor_desc(aL + off);
              const uint64_t dBL = sw128_kmajor_desc(bL + off);
              umma_f16(d_tmem, dAH, dBL, kIdesc, 1u);
              umma_f16(d_tmem, dAL, dBH, kIdesc, 1u);
            }
          }
          umma_commit(&empty[stage]);
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        umma_commit(&tfull[acc]);
        acc ^= 1;
        if (acc == 0) aphase ^= 1u;
      }
      // all MMAs issued by this thread complete before TMEM is released
      umma_commit(mdone);
      WaitCtx wd = w;
      volatile int never = 0;
      wd.abort_flag = &never;
      mbar_wait(mdone, 0, wd);
    }
  } else {
    // ---------------------------------------------------------- epilogue
    const int q = warp & 3;  // TMEM lane quarter this warp may read
    float* stg = epi + (warp - 2) * 32 * kStagePad;
    BandCursor cur;
    band_cursor_init(&cur, p.m, kGroupG);
    int acc = 0;
    uint32_t aphase = 0;
    for (int64_t u = p.u_begin + blockIdx.x; u < p.u_end; u += gridDim.x) {
      int64_t row0, col0;
      unit_coords(&cur, p, u, &row0, &col0);
      if (row0 >= n) continue;
      if (!mbar_wait(&tfull[acc], aphase, w)) break;
      tc_fence_after();
      const int64_t rbase = row0 + q * 32;       // first row of this warp
      const int64_t my_i = rbase + lane;
      const int my_flag = (my_i < n) ? p.flags[my_i] : 1;
      const int64_t my_base = pair_row_base(n, my_i);
#pragma unroll 1
      for (int c = 0; c < kBN / 32; ++c) {
        const int64_t jc0 = col0 + c * 32;
        // warp-uniform: does this 32 x 32 block hold any pair i < j < n?
        if (rbase >= n || jc0 >= n || jc0 + 31 <= rbase) continue;
        uint32_t v[32];
        tmem_ld_32x32b_x32(
            tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * kBN + c * 32),
            v);
        tmem_ld_wait();
#pragma unroll
        for (int t = 0; t < 32; ++t)
          stg[lane * kStagePad + t] = __uint_as_float(v[t]);
        __syncwarp();
        const int64_t j = jc0 + lane;
        const int col_flag = (j < n) ? p.flags[j] : 1;
#pragma unroll 4
        for (int rr = 0; rr < 32; ++rr) {
          const int64_t i = rbase + rr;
          const int64_t base = __shfl_sync(0xffffffffu, my_base, rr);
          const int fl = __shfl_sync(0xffffffffu, my_flag, rr) | col_flag;
          const bool valid = (i < n) && (j < n) && (j > i);
          float r = stg[rr * kStagePad + lane] * p.out_scale;
          r = fminf(1.f, fmaxf(-1.f, r));
          if (fl) r = __int_as_float(0x7fc00000);
          if constexpr (WRITE_R) {
            if (valid) __stcs(p.R + base + j, r);
          }
          if constexpr (EDGES) {
            const bool e = valid && !fl && fabsf(r) >= p.tau;
            const unsigned mask = __ballot_sync(0xffffffffu, e);
            if (mask) {
              const int leader = __ffs(mask) - 1;
              unsigned long long b0 = 0;
              if (lane == leader)
                b0 = atomicAdd(p.count, (unsigned long long)__popc(mask));
              b0 = __shfl_sync(0xffffffffu, b0, leader);
              if (e) {
                const unsigned long long idx =
                    b0 + __popc(mask & ((1u << lane) - 1u));
                if (idx < p.cap) {
                  p.edges[idx].i = (uint32_t)i;
                  p.edges[idx].j = (uint32_t)j;
                  p.edges[idx].r = r;
                } else {
                  atomicCAS(p.status, 0, (int)PCC_ERR_CAPACITY);
                }
              }
            }
          }
        }
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[acc]);
      acc ^= 1;
      if (acc == 0) aphase ^= 1u;
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem_base, 512);
}

template <int NPROD, bool BF16, bool WRITE_R, bool EDGES>
cudaError_t launch_inst(const pcc_zmat* Z, const TcParams& p, int grid,
                        cudaStream_t s) {
  auto fn = k_pairs_tc<NPROD, BF16, WRITE_R, EDGES>;
  const int smem = Cfg<NPROD>::kSmemBytes;
  cudaError_t e = ensure_func_smem(reinterpret_cast<const void*>(fn), smem);
  if (e != cudaSuccess) return e;
  fn<<<grid, kThreads, smem, s>>>(Z->tm_hi, Z->tm_lo, p);
  return cudaGetLastError();
}

template <int NPROD, bool BF16>
cudaError_t launch_prec(const pcc_zmat* Z, const TcParams& p, int grid,
                        bool write_r, bool edges_on, cudaStream_t s) {
  if (write_r && edges_on) return launch_inst<NPROD, BF16, true, true>(Z, p, grid, s);
  if (edges_on) return launch_inst<NPROD, BF16, false, true>(Z, p, grid, s);
  return launch_inst<NPROD, BF16, true, false>(Z, p, grid, s);
}

}  // namespace

int64_t tc_num_tiles(int64_t n) {
  const int64_t m = tc_super_count(n);
  return m * (m + 1) / 2;
}

cudaError_t launch_tc_pairs(const pcc_zmat* Z, float* R, int64_t t0,
                            int64_t t1, bool edges_on, float tau,
                            pcc_edge* edges, uint64_t cap,
                            unsigned long long* count, cudaStream_t s) {
  if (t1 <= t0) return cudaSuccess;
  TcParams p;
  p.n = Z->n;
  p.m = tc_super_count(Z->n);
  p.u_begin = 2 * t0;
  p.u_end = 2 * t1;
  p.nkb = (int)(Z->lpad / kBK);
  p.out_scale = (float)ldexp(1.0, -2 * Z->scale_exp);
  p.tau = tau;
  p.flags = Z->flags;
  p.R = R;
  p.edges = edges;
  p.count = count;
  p.cap = cap;
  p.status = Z->status;
  p.wait_ns = wait_limit_ns();
  const int64_t units = p.u_end - p.u_begin;
  int grid = num_sms(Z->device);
  if (units < grid) grid = (int)units;
  const bool write_r = R != nullptr;
  switch (Z->prec) {
    case PCC_PREC_BF16X3:
      return launch_prec<3, true>(Z, p, grid, write_r, edges_on, s);
    case PCC_PREC_FP16X3S:
      return launch_prec<3, false>(Z, p, grid, write_r, edges_on, s);
    case PCC_PREC_BF16X1:
      return launch_prec<1, true>(Z, p, grid, write_r, edges_on, s);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace pcc
