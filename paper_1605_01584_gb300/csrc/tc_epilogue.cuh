// tc_epilogue.cuh -- the store side shared by the tensor-core pair kernels:
// one warp turns 32 rows x 128 columns of a TMEM accumulator into packed
// upper-triangle values (and optional |r| >= tau edges).
//
// Row i's pairs are contiguous in the packed layout, J(i,j) = base(i) + j,
// base(i+1) = base(i) + n - i - 2.  TMEM hands thread t the columns of row
// t, so each 32 x 32 block goes through a shared-memory transpose; the warp
// then stores 32 consecutive pairs of one row per instruction.  Blocks with
// no pair i < j < n are skipped, blocks that are entirely valid and
// unflagged take a branch-free path, and the (rare) edge append rescans a
// block only when some |r| >= tau.
//
// DENSE: the non-symmetric form (rows of one matrix against the rows of
// another): every (i < n, j < ncol) is a pair, and row i of R starts at
// base0 + (i - rbase) * ldr.
//
// Long rows: the K blocks of a unit are accumulated in chunks (see
// tc_common.cuh); fold_acc adds a finished chunk into the next one in TMEM
// so that the chunk's buffer can be handed back before the store pass.
#pragma once
#include <stdint.h>

#include "pcc.h"
#include "pcc_ptx.cuh"

namespace pcc {

constexpr int kStagePad = 33;  // transpose row pitch (conflict-free)

// second += first over one warp's 32 TMEM lanes x 128 columns (t_first,
// t_second: lane quarter and first column of the warp), one FP32
// round-to-nearest add per element, 16 columns at a time (few registers:
// the epilogue runs at the 168-register cap of a 10-warp CTA).
__device__ __forceinline__ void fold_acc(uint32_t t_first, uint32_t t_second) {
#pragma unroll 1
  for (int c = 0; c < 8; ++c) {
    uint32_t a[16], b[16];
    tmem_ld_32x32b_x16(t_first + (uint32_t)(c * 16), a);
    tmem_ld_32x32b_x16(t_second + (uint32_t)(c * 16), b);
    tmem_ld_wait();
#pragma unroll
    for (int t = 0; t < 16; ++t)
      b[t] = __float_as_uint(__uint_as_float(a[t]) + __uint_as_float(b[t]));
    tmem_st_32x32b_x16(t_second + (uint32_t)(c * 16), b);
  }
  tmem_st_wait();
}

struct EpiOut {
  float* R;                    // packed output (or null)
  float scale;                 // accumulator -> r (2^-2s for FP16X3S)
  float tau;                   // edge threshold
  pcc_edge* edges;
  unsigned long long* count;
  uint64_t cap;
  int* status;
};

// t_row: TMEM address of (lane 32q, first column of the warp's 128); stg:
// this warp's 32 x kStagePad floats; rbase: first row; jw0: first column;
// base0 = pair_row_base(n, rbase); rflags: bit rr = row rbase+rr flagged (or
// >= n); cfl[c]: flag of column jw0 + 32c + lane; ncol, ldr: DENSE only.
template <bool WRITE_R, bool EDGES, bool DENSE = false>
__device__ __forceinline__ void epilogue_rows(uint32_t t_row, float* stg,
                                              int lane, int64_t n,
                                              int64_t rbase, int64_t jw0,
                                              int64_t base0, uint32_t rflags,
                                              const int (&cfl)[4],
                                              const EpiOut& eo,
                                              int64_t ncol = 0,
                                              int64_t ldr = 0) {
  if constexpr (!DENSE) ncol = n;
  // warp-uniform: does 32 x 32 block c hold any pair?
  auto active = [&](int c) {
    const int64_t jc0 = jw0 + c * 32;
    if constexpr (DENSE) return !(rbase >= n || jc0 >= ncol);
    return !(rbase >= n || jc0 >= n || jc0 + 31 <= rbase);
  };
  auto next_active = [&](int c) {
    ++c;
    while (c < 4 && !active(c)) ++c;
    return c;
  };
  uint32_t v[32];
  int c = next_active(-1);
  if (c < 4) tmem_ld_32x32b_x32(t_row + (uint32_t)(c * 32), v);
  while (c < 4) {
    tmem_ld_wait();
#pragma unroll
    for (int t = 0; t < 32; ++t)
      stg[lane * kStagePad + t] = __uint_as_float(v[t]);
    __syncwarp();
    // the next block's TMEM load overlaps this block's stores
    const int cn = next_active(c);
    if (cn < 4) tmem_ld_32x32b_x32(t_row + (uint32_t)(cn * 32), v);
    const int64_t jc0 = jw0 + c * 32;
    const int64_t j = jc0 + lane;
    const bool cflag = cfl[c] != 0;
    const bool clean = (DENSE || jc0 > rbase + 31) && (jc0 + 31 < ncol) &&
                       (rbase + 31 < n) && rflags == 0 &&
                       !__any_sync(0xffffffffu, cflag);
    float* out = eo.R + base0 + j;
    // packed rows: row i+1 starts n - i - 2 after row i; dense rows: ldr
    int64_t step = DENSE ? ldr : n - rbase - 2;
    constexpr int64_t kDec = DENSE ? 0 : 1;
    bool hit = false;
    if (clean) {
      // every pair of the block is valid and unflagged
#pragma unroll 8
      for (int rr = 0; rr < 32; ++rr) {
        float r = stg[rr * kStagePad + lane] * eo.scale;
        r = fminf(1.f, fmaxf(-1.f, r));
        if constexpr (WRITE_R) __stcs(out, r);
        if constexpr (EDGES) hit |= fabsf(r) >= eo.tau;
        out += step;
        step -= kDec;
      }
    } else {
      hit = true;  // edges (if any) are handled by the scan below
      if constexpr (WRITE_R) {
#pragma unroll 4
        for (int rr = 0; rr < 32; ++rr) {
          const int64_t i = rbase + rr;
          float r = stg[rr * kStagePad + lane] * eo.scale;
          r = fminf(1.f, fmaxf(-1.f, r));
          if (((rflags >> rr) & 1u) || cflag) r = __int_as_float(0x7fc00000);
          if (i < n && j < ncol && (DENSE || j > i)) __stcs(out, r);
          out += step;
          step -= kDec;
        }
      }
    }
    if constexpr (EDGES) {
      if (__any_sync(0xffffffffu, hit)) {
        // rare: rescan the block and append its edges, one atomic per warp
        // and row
        for (int rr = 0; rr < 32; ++rr) {
          const int64_t i = rbase + rr;
          float r = stg[rr * kStagePad + lane] * eo.scale;
          r = fminf(1.f, fmaxf(-1.f, r));
          const bool fl = ((rflags >> rr) & 1u) || cflag;
          const bool e = i < n && j < ncol && (DENSE || j > i) && !fl &&
                         fabsf(r) >= eo.tau;
          const unsigned mask = __ballot_sync(0xffffffffu, e);
          if (mask) {
            const int leader = __ffs(mask) - 1;
            unsigned long long b0 = 0;
            if (lane == leader)
              b0 = atomicAdd(eo.count, (unsigned long long)__popc(mask));
            b0 = __shfl_sync(0xffffffffu, b0, leader);
            if (e) {
              const unsigned long long idx =
                  b0 + __popc(mask & ((1u << lane) - 1u));
              if (idx < eo.cap) {
                eo.edges[idx].i = (uint32_t)i;
                eo.edges[idx].j = (uint32_t)j;
                eo.edges[idx].r = r;
              } else {
                atomicCAS(eo.status, 0, (int)PCC_ERR_CAPACITY);
              }
            }
          }
        }
      }
    }
    __syncwarp();
    c = cn;
  }
}

}  // namespace pcc
