// tc_perm_common.cuh -- what the two forms of the tensor-core permutation
// test share: the 128 x 128 tile of the triangle, the MMA step, and the
// numbering of tile pairs column by column for CTA pairs.
#pragma once
#include <math.h>
#include <stdint.h>

#include "pcc_ptx.cuh"

namespace pcc {

constexpr int kPT = 128;                 // tile side (M of one CTA)
constexpr int kPUK = 16;                 // K of one tcgen05.mma (16-bit)
constexpr int kPEpiWarps = 8;            // epilogue warps per CTA
constexpr int kPAcc = 2 * kPT;           // TMEM columns per accumulator
constexpr int kPMaxResidentK = 256;      // resident A tile up to lpad 256
constexpr int kPSmemBudget = 232448;     // dynamic shared memory per CTA

// PAIR items: the tiles of column x of the triangle taken two by two, rows
// (2r, 2r+1); column x holds floor((x+2)/2) pairs (the last one alone when
// x is even) and Q(x) = floor((x+1)/2) * floor((x+2)/2) pairs come before
// it.  The closed-form estimate is corrected by exact integer tests.
__host__ __device__ __forceinline__ int64_t col_pairs_before(int64_t x) {
  return ((x + 1) / 2) * ((x + 2) / 2);
}

__device__ __forceinline__ void col_pair_coords(int64_t t, int64_t* r,
                                                int64_t* x) {
  int64_t xx = (int64_t)(2.0 * sqrt((double)t));
  if (xx < 0) xx = 0;
  while (xx > 0 && col_pairs_before(xx) > t) --xx;
  while (col_pairs_before(xx + 1) <= t) ++xx;
  *x = xx;
  *r = t - col_pairs_before(xx);
}

// Counts are 16-bit per pair in registers: a segment of a CTA pair's range
// holds at most this many passes (two permutations each).
constexpr int64_t kPMaxSegPasses = 32767;

// Stage hand-off for operands that threads (not TMA) put in shared memory.

// Make this thread's shared-memory stores visible to the tensor cores
// (async proxy) before it signals that the stage is full.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Release over this CTA's shared memory only, at cluster scope: with the
// relaxed arrive after it, the gathered stage is visible to whoever
// acquires the barrier's phase, without waiting for this thread's global
// loads in flight (the next pass's indices), as a full release would.
__device__ __forceinline__ void fence_release_smem_cluster() {
  asm volatile("fence.release.sync_restrict::shared::cta.cluster;" :::
                   "memory");
}

// Arrive on an mbarrier of either CTA of the pair (shared::cluster
// address), relaxed: the ordering comes from the fence before it.
__device__ __forceinline__ void mbar_arrive_relaxed_cluster(uint32_t addr) {
  asm volatile(
      "mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(
          addr)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_acq_cluster(uint64_t* bar,
                                                          uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], "
      "%2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// mbar_wait with acquire at cluster scope (the phase was completed by
// threads of both CTAs); bounded like mbar_wait.
static __device__ __noinline__ bool mbar_wait_acq_cluster(uint64_t* bar,
                                                          uint32_t parity,
                                                          const WaitCtx w) {
  if (mbar_try_wait_acq_cluster(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  for (uint32_t spin = 1;; ++spin) {
    if (mbar_try_wait_acq_cluster(bar, parity)) return true;
    if ((spin & 15u) == 0) {
      if (*w.abort_flag) return false;
      if (global_timer_ns() - t0 > w.limit_ns) {
        wait_fail(w, 5 /* PCC_ERR_TIMEOUT */);
        return false;
      }
    }
  }
}

// One segment of a CTA pair's range: tile pair t, passes [q0, q1).
struct Segment {
  int64_t t, q0, q1;
};

// The next segment of the range [u, u1) of (tile pair, pass) units, numbered
// tile by tile.
__device__ __forceinline__ Segment next_segment(int64_t u, int64_t u1,
                                                int64_t npass) {
  Segment g;
  g.t = u / npass;
  g.q0 = u - g.t * npass;
  int64_t q1 = g.q0 + (u1 - u);
  if (q1 > npass) q1 = npass;
  if (q1 - g.q0 > kPMaxSegPasses) q1 = g.q0 + kPMaxSegPasses;
  g.q1 = q1;
  return g;
}

}  // namespace pcc
