// stream.cu -- all pairs in passes, for outputs larger than the device
// (Section III-C's multi-pass execution and Algorithm 2's asynchronous
// double buffering).
//
// The paper computes a range of tile ids per pass into a tile-major buffer
// R', and while the next pass runs it copies the finished buffer to the
// host, which then has to place every tile.  Here a pass is a run of whole
// row blocks of the schedule instead: the bands of G super-tile rows of the
// tensor-core order (pcc_sched.h), or the tile rows of the paper's own
// triangular order for the CUDA-core forms, whose ids are contiguous (Eq.
// (9)-(10) numbers a row's tiles consecutively).  All the pairs of a run of
// rows form one contiguous slice of the packed triangle (or of the dense
// cross matrix), so the kernel writes the slice in its final layout into a
// device window (R offset by the slice's first element) and one copy puts
// it in place in the caller's host buffer: nothing is rearranged on the
// host.
//
// Pipeline (two device windows, two optional pinned staging buffers):
//   pass p:   [compute stream] wait until window p%2 was copied out (pass
//             p-2), run the kernel into window p%2
//             [copy streams]   wait for that kernel, copy window p%2 to the
//             host (caller's buffer or staging buffer p%2), in two halves
//             on two streams
//   host:     wait for the copy of pass p-1, hand it to the caller's sink
// so the kernel of pass p+1 overlaps the copy of pass p and the sink of
// pass p-1.
#include <stdlib.h>

#include <functional>
#include <vector>

#include "pcc_internal.h"
#include "pcc_sched.h"

namespace pcc {
namespace {

struct Block {      // one row block of the schedule
  int64_t t0, t1;   // its tile ids
  int64_t r0, r1;   // its rows (of the first matrix)
};

struct Pass {
  int64_t t0, t1, r0, r1;
  int64_t e0, e1;   // output elements [e0, e1)
};

int64_t pairs_before(int64_t n, int64_t i) { return i * (2 * n - i - 1) / 2; }

// Row blocks of each schedule.  cross_cols = 0 for the triangle, else the
// second matrix's rows.
std::vector<Block> tc_blocks(int64_t n, int64_t G, int64_t cross_cols) {
  std::vector<Block> v;
  const int64_t m = tc_super_count(n);
  const int64_t mc = cross_cols ? tc_super_count(cross_cols) : 0;
  int64_t start = 0;
  for (int64_t b = 0; b * G < m; ++b) {
    const int64_t g = m - b * G < G ? m - b * G : G;
    const int64_t cnt = cross_cols ? g * mc : band_tiles(m, G, b);
    const int64_t r0 = b * G * kTcSuper;
    const int64_t r1 = (b * G + g) * kTcSuper < n ? (b * G + g) * kTcSuper : n;
    v.push_back({start, start + cnt, r0, r1});
    start += cnt;
  }
  return v;
}

std::vector<Block> simt_blocks(int64_t n, int64_t BT, int64_t cross_cols) {
  std::vector<Block> v;
  const int64_t m = (n + BT - 1) / BT;
  const int64_t mc = cross_cols ? (cross_cols + BT - 1) / BT : 0;
  for (int64_t y = 0; y < m; ++y) {
    const int64_t t0 = cross_cols ? y * mc : tri_F(m, y);
    const int64_t t1 = cross_cols ? (y + 1) * mc : tri_F(m, y + 1);
    const int64_t r1 = (y + 1) * BT < n ? (y + 1) * BT : n;
    v.push_back({t0, t1, y * BT, r1});
  }
  return v;
}

// Greedy grouping of consecutive blocks into passes of at most cap output
// elements; false if one block alone exceeds cap.
bool group(const std::vector<Block>& bl, int64_t n, int64_t cross_cols,
           int64_t cap, std::vector<Pass>* out) {
  auto elem = [&](int64_t r) {
    return cross_cols ? r * cross_cols : pairs_before(n, r);
  };
  out->clear();
  size_t i = 0;
  while (i < bl.size()) {
    Pass p{bl[i].t0, bl[i].t1, bl[i].r0, bl[i].r1, elem(bl[i].r0),
           elem(bl[i].r1)};
    if (p.e1 - p.e0 > cap) return false;
    size_t j = i + 1;
    while (j < bl.size() && elem(bl[j].r1) - p.e0 <= cap) {
      p.t1 = bl[j].t1;
      p.r1 = bl[j].r1;
      p.e1 = elem(bl[j].r1);
      ++j;
    }
    out->push_back(p);
    i = j;
  }
  return true;
}

// The per-call objects; the windows and staging buffers themselves are
// cached in the pcc_zmat (grown when a call needs more).
// Each pass's copy is split in two halves on two copy streams: on GB300 one
// device-to-host copy ran at 150-193 GB/s from call to call, two
// concurrent ones at the link's 193.5 GB/s every time.
struct Resources {
  void* win[2] = {nullptr, nullptr};
  void* stage[2] = {nullptr, nullptr};
  cudaStream_t cs = nullptr;
  cudaStream_t cs2 = nullptr;
  cudaEvent_t k_done[2] = {nullptr, nullptr};
  cudaEvent_t c_done[2] = {nullptr, nullptr};
  cudaEvent_t c_half[2] = {nullptr, nullptr};
  ~Resources() {
    if (cs) cudaStreamSynchronize(cs);
    if (cs2) cudaStreamSynchronize(cs2);
    for (int k = 0; k < 2; ++k) {
      if (k_done[k]) cudaEventDestroy(k_done[k]);
      if (c_done[k]) cudaEventDestroy(c_done[k]);
      if (c_half[k]) cudaEventDestroy(c_half[k]);
    }
    if (cs) cudaStreamDestroy(cs);
    if (cs2) cudaStreamDestroy(cs2);
  }
};

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// two windows of `each` bytes in Z's device cache (and two pinned staging
// buffers when `staging`)
pcc_status take_workspace(pcc_zmat* Z, size_t each, bool staging,
                          Resources* r) {
  const size_t need = 2 * round256(each);
  if (Z->win_ws_bytes < need) {
    if (Z->win_ws) cudaFree(Z->win_ws);
    Z->win_ws = nullptr;
    Z->win_ws_bytes = 0;
    if (cudaMalloc(&Z->win_ws, need) != cudaSuccess) {
      cudaGetLastError();
      return PCC_ERR_OOM;
    }
    Z->win_ws_bytes = need;
  }
  r->win[0] = Z->win_ws;
  r->win[1] = static_cast<char*>(Z->win_ws) + round256(each);
  if (staging) {
    if (Z->stage_ws_bytes < need) {
      if (Z->stage_ws) cudaFreeHost(Z->stage_ws);
      Z->stage_ws = nullptr;
      Z->stage_ws_bytes = 0;
      if (cudaMallocHost(&Z->stage_ws, need) != cudaSuccess) {
        cudaGetLastError();
        return PCC_ERR_OOM;
      }
      Z->stage_ws_bytes = need;
    }
    r->stage[0] = Z->stage_ws;
    r->stage[1] = static_cast<char*>(Z->stage_ws) + round256(each);
  }
  return PCC_OK;
}

using LaunchFn =
    std::function<cudaError_t(void* win, const Pass& p, cudaStream_t s)>;

// The pass pipeline.  host: caller's buffer (NULL = staging); ldh: its row
// pitch for dense output (0 = packed, one contiguous slice per pass);
// ncols: dense row length on the device.
pcc_status run_passes(pcc_zmat* Zc, const std::vector<Pass>& passes,
                      size_t esize, int64_t ncols, void* host, int64_t ldh,
                      pcc_rows_sink sink, void* user, cudaStream_t s,
                      const LaunchFn& launch) {
  int64_t wmax = 0;
  for (const Pass& p : passes)
    if (p.e1 - p.e0 > wmax) wmax = p.e1 - p.e0;
  if (passes.empty() || wmax == 0) return PCC_OK;
  Resources r;
  const int nwin = passes.size() > 1 ? 2 : 1;
  // calls return only after their last copy, so Z's cached buffers are
  // free when the next call starts
  pcc_status ws = take_workspace(Zc, (size_t)wmax * esize, host == nullptr,
                                 &r);
  if (ws != PCC_OK) return ws;
  if (cudaStreamCreateWithFlags(&r.cs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&r.cs2, cudaStreamNonBlocking) != cudaSuccess)
    return PCC_ERR_CUDA;
  for (int k = 0; k < 2; ++k)
    if (cudaEventCreateWithFlags(&r.k_done[k], cudaEventDisableTiming) !=
            cudaSuccess ||
        cudaEventCreateWithFlags(&r.c_done[k], cudaEventDisableTiming) !=
            cudaSuccess ||
        cudaEventCreateWithFlags(&r.c_half[k], cudaEventDisableTiming) !=
            cudaSuccess)
      return PCC_ERR_CUDA;

  char* hb = static_cast<char*>(host);
  auto dst_of = [&](size_t p) -> char* {
    const Pass& q = passes[p];
    if (!host) return static_cast<char*>(r.stage[p & 1]);
    if (ldh) return hb + (size_t)(q.r0 * ldh) * esize;
    return hb + (size_t)q.e0 * esize;
  };
  auto deliver = [&](size_t p) -> pcc_status {
    if (cudaEventSynchronize(r.c_done[p & 1]) != cudaSuccess)
      return PCC_ERR_CUDA;
    if (sink && sink(user, passes[p].r0, passes[p].r1, dst_of(p)) != 0)
      return PCC_ERR_ABORTED;
    return PCC_OK;
  };
  auto fail = [&](pcc_status st) {
    cudaStreamSynchronize(s);
    cudaStreamSynchronize(r.cs);
    cudaStreamSynchronize(r.cs2);
    return st;
  };

  for (size_t p = 0; p < passes.size(); ++p) {
    const int k = (int)(p & 1) % nwin;
    const Pass& q = passes[p];
    // window k was last copied out by pass p-2
    if (p >= 2 && cudaStreamWaitEvent(s, r.c_done[k], 0) != cudaSuccess)
      return fail(PCC_ERR_CUDA);
    cudaError_t e = launch(r.win[k], q, s);
    if (e != cudaSuccess) return fail(cuda_status(e));
    if (cudaEventRecord(r.k_done[k], s) != cudaSuccess ||
        cudaStreamWaitEvent(r.cs, r.k_done[k], 0) != cudaSuccess ||
        cudaStreamWaitEvent(r.cs2, r.k_done[k], 0) != cudaSuccess)
      return fail(PCC_ERR_CUDA);
    const int64_t cnt = q.e1 - q.e0;
    char* dst = dst_of(p);
    const char* src = static_cast<const char*>(r.win[k]);
    if (host && ldh && ldh != ncols) {
      // rows [0, h) on one copy stream, [h, rows) on the other
      const size_t rows = (size_t)(q.r1 - q.r0), h = rows / 2;
      const size_t dp = (size_t)ldh * esize, sp = (size_t)ncols * esize;
      e = cudaMemcpy2DAsync(dst, dp, src, sp, sp, h, cudaMemcpyDeviceToHost,
                            r.cs);
      if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(dst + h * dp, dp, src + h * sp, sp, sp,
                              rows - h, cudaMemcpyDeviceToHost, r.cs2);
    } else {
      const size_t bytes = (size_t)cnt * esize, h = bytes / 2;
      e = cudaMemcpyAsync(dst, src, h, cudaMemcpyDeviceToHost, r.cs);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(dst + h, src + h, bytes - h,
                            cudaMemcpyDeviceToHost, r.cs2);
    }
    // c_done[k]: both halves are on the host
    if (e != cudaSuccess || cudaEventRecord(r.c_half[k], r.cs2) != cudaSuccess ||
        cudaStreamWaitEvent(r.cs, r.c_half[k], 0) != cudaSuccess ||
        cudaEventRecord(r.c_done[k], r.cs) != cudaSuccess)
      return fail(PCC_ERR_CUDA);
    // hand the previous pass to the caller while this one computes
    if (p >= 1) {
      pcc_status st = deliver(p - 1);
      if (st != PCC_OK) return fail(st);
    }
  }
  pcc_status st = deliver(passes.size() - 1);
  if (st != PCC_OK) return fail(st);
  return PCC_OK;
}

// elements per window: half the budget (both windows share it); default
// budget a quarter of the free device memory, at most 4 GiB
int64_t window_cap(int64_t device_bytes, size_t esize) {
  int64_t b = device_bytes;
  if (b <= 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      fr = (size_t)1 << 32;
    }
    b = (int64_t)(fr / 4);
    if (b > ((int64_t)4 << 30)) b = (int64_t)4 << 30;
  }
  return b / 2 / (int64_t)esize;
}

}  // namespace

pcc_status allpairs_host(const pcc_zmat* ZA, const pcc_zmat* ZB, void* host,
                         pcc_dtype rt, int64_t ldh, int64_t device_bytes,
                         pcc_rows_sink sink, void* user, cudaStream_t s,
                         const HostEdges* he) {
  const bool eo = he != nullptr;
  const float tau = eo ? he->tau : 0.f;
  pcc_edge* ed = eo ? he->edges : nullptr;
  const uint64_t ecap = eo ? he->cap : 0;
  unsigned long long* cnt = eo ? he->count : nullptr;
  const size_t esize = rt == PCC_F64 ? 8 : 4;
  const int64_t cap = window_cap(device_bytes, esize);
  const int64_t cross = ZB ? ZB->n : 0;
  const int64_t n = ZA->n;
  std::vector<Pass> passes;
  if (is_split(ZA->prec)) {
    // the widest first block must fit: halve the band height until it does
    int64_t G = tc_tuning().band;
    for (;;) {
      if (group(tc_blocks(n, G, cross), n, cross, cap, &passes)) break;
      if (G == 1) return PCC_ERR_OOM;
      G = (G + 1) / 2;
    }
    return run_passes(
        const_cast<pcc_zmat*>(ZA), passes, esize, cross, host, ZB ? ldh : 0,
        sink, user, s,
        [&](void* win, const Pass& q, cudaStream_t st) {
          float* w = static_cast<float*>(win);
          if (ZB)
            return launch_tc_cross(ZA, ZB, w, cross, q.t0, q.t1, eo, tau, ed,
                                   ecap, cnt, st, q.e0, G);
          return launch_tc_pairs(ZA, w, q.t0, q.t1, eo, tau, ed, ecap, cnt,
                                 st, q.e0, G);
        });
  }
  const int64_t BT = simt_tile_size(ZA->prec);
  if (!group(simt_blocks(n, BT, cross), n, cross, cap, &passes))
    return PCC_ERR_OOM;
  return run_passes(const_cast<pcc_zmat*>(ZA), passes, esize, cross, host,
                    ZB ? ldh : 0, sink, user, s,
                    [&](void* win, const Pass& q, cudaStream_t st) {
                      if (ZB)
                        return launch_simt_cross(ZA, ZB, win, rt, cross, q.t0,
                                                 q.t1, tau, ed, ecap, cnt, st,
                                                 q.e0);
                      return launch_simt_pairs(ZA, win, rt, q.t0, q.t1, tau,
                                               ed, ecap, cnt, st, q.e0);
                    });
}

}  // namespace pcc
