// tc_common.cuh -- pieces shared by the persistent tensor-core kernels
// (tc_pairs.cu, tc_batched.cu): the accumulator chunk schedule of a work
// unit and the end-of-kernel drain of the TMA ring.
//
// Accumulator chunks.  The tensor cores add every product into the FP32
// accumulator with a rounding toward zero, so the error of a running sum
// grows with the number of updates made while it is large (on rows whose
// mass sits in one sample, r = 1, about 9e-9 per sample of the row after
// that sample).  A unit's K blocks are therefore cut into nch chunks of
// nearly equal length (whole groups of 64 samples), each accumulated into a
// fresh TMEM buffer,
// the two buffers alternating from chunk to chunk, and the epilogue adds
// each finished chunk into the next one with one round-to-nearest FP32 add
// per element (fold_acc) before that buffer is handed back.  nch = 1 keeps
// the whole row in one accumulator and lets the next unit's MMAs overlap the
// store of the previous one.
#pragma once
#include <stdint.h>

#include "pcc_ptx.cuh"

namespace pcc {

// First K block of chunk c of a unit of nkb blocks of KB samples cut into
// nch chunks.  Boundaries are set in groups of 64 samples (padded rows are
// a multiple of 64), so every stage size (KB = 32 or 64) cuts a row at the
// same samples and gives the same bits.
template <int KB>
__host__ __device__ __forceinline__ int chunk_begin(int nkb, int nch, int c) {
  static_assert(KB == 32 || KB == 64, "stage sizes");
  constexpr int per64 = 64 / KB;
  const int64_t groups = nkb / per64;
  return (int)((int64_t)c * groups / nch) * per64;
}

// Every fill of the ring, per stage: how many fills the producer issued and
// this CTA's bytes of the last one (slot S, after the S stages, may log one
// more barrier, such as that of a resident operand tile).  Kept in shared
// memory; in the 2-SM pair form the odd CTA copies its own counts into the
// even CTA's peer_* fields before the drain.
struct FillLog {
  uint32_t fills[16];
  uint32_t bytes[16];
  uint32_t peer_fills[16];
  uint32_t peer_bytes[16];
};

__device__ __forceinline__ void fill_log_init(FillLog* f) {
  for (int s = 0; s < 16; ++s) {
    f->fills[s] = 0;
    f->bytes[s] = 0;
    f->peer_fills[s] = 0;
    f->peer_bytes[s] = 0;
  }
}

// Single CTA: every copy completes on this CTA's own stage barriers, so the
// phase of the last fill of each stage completing means all its copies have
// landed.  Bounded by wd.
__device__ __forceinline__ uint64_t* log_bar(uint64_t* full, uint64_t* extra,
                                             int S, int s) {
  return s < S ? &full[s] : extra;
}

__device__ __forceinline__ void drain_own(uint64_t* full, uint64_t* extra,
                                          const FillLog* f, int S,
                                          const WaitCtx& wd) {
  const int slots = extra ? S + 1 : S;
  for (int s = 0; s < slots; ++s)
    if (f->fills[s])
      mbar_wait(log_bar(full, extra, S, s), (f->fills[s] - 1u) & 1u, wd);
}

// Pair form, one thread of the even CTA, after the odd CTA published its
// counts: both CTAs' copies complete on the even CTA's stage barriers, which
// the even producer arms for both.  A fill of stage s waits on the MMA's
// release of the previous fill of s, which needed both CTAs' copies of that
// one, so after the producers stop the two counts of a stage differ by at
// most one.  Where the even CTA armed a fill that the odd CTA never sent,
// the odd share is cancelled (complete_tx); where the odd CTA sent a fill
// that the even CTA never armed, it is armed now for the odd bytes alone.
// Then the last phase of every stage completes once every issued copy has
// landed.  Bounded by wd.
__device__ __forceinline__ void drain_pair_even(uint64_t* full,
                                                uint64_t* extra,
                                                const FillLog* f, int S,
                                                const WaitCtx& wd) {
  const int slots = extra ? S + 1 : S;
  for (int s = 0; s < slots; ++s) {
    uint64_t* bar = log_bar(full, extra, S, s);
    const uint32_t fe = f->fills[s], fo = f->peer_fills[s];
    const uint32_t F = fe > fo ? fe : fo;
    if (F == 0) continue;
    if (fe + 1u == F && fo == F)
      mbar_arrive_expect_tx(bar, f->peer_bytes[s]);
    else if (fo + 1u == F && fe == F)
      mbar_complete_tx(bar, f->bytes[s]);
    mbar_wait(bar, (F - 1u) & 1u, wd);
  }
}

// End of a persistent tensor-core kernel, called by every thread of the CTA
// after all roles have finished issuing: no copy may still be in flight
// into the shared memory of a CTA that exits.  PAIR: the odd CTA publishes
// its fill log to the even CTA, which drains both, and neither CTA leaves
// before that.
template <bool PAIR>
__device__ __forceinline__ void drain_ring(uint64_t* full, uint64_t* extra,
                                           FillLog* f, int S,
                                           const WaitCtx& w, uint32_t crank) {
  WaitCtx wd = w;
  volatile int never = 0;  // the drain ignores the CTA's abort flag
  wd.abort_flag = &never;
  if constexpr (PAIR) {
    if (crank == 1 && threadIdx.x == 0) {
      for (int s = 0; s < (extra ? S + 1 : S); ++s) {
        st_cluster_u32(cluster_addr(&f->peer_fills[s], 0), f->fills[s]);
        st_cluster_u32(cluster_addr(&f->peer_bytes[s], 0), f->bytes[s]);
      }
    }
    cluster_sync();
    if (crank == 0 && threadIdx.x == 0)
      drain_pair_even(full, extra, f, S, wd);
    cluster_sync();
  } else {
    if (threadIdx.x == 0) drain_own(full, extra, f, S, wd);
    __syncthreads();
  }
}

}  // namespace pcc
