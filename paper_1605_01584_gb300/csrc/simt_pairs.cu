// simt_pairs.cu -- K4 / K5: CUDA-core pair kernels over a standardized Z in
// FP32 or FP64 (the plain-precision comparison path).
//
// Section III-C: the n x n job matrix is cut into BT x BT tiles, m =
// ceil(n/BT); the tiles of the upper triangle (diagonal included) are
// numbered by Eq. (16) and each block maps its id back to (yt, xt) with
// Eq. (17)-(19) (FP64 root + integer correction, pcc_sched.h).  Within a
// tile, r(i,j) = sum_k z_i[k] z_j[k] (Eq. (6)) for rows y in
// [yt*BT, (yt+1)*BT) and columns x in [xt*BT, (xt+1)*BT); pairs with
// x <= y are skipped (Algorithm 1 skips y > x; the diagonal is excluded
// here).  Instead of one thread per column (the Xeon Phi layout), 256
// threads each own a TT x TT register block, K is staged through shared
// memory BK at a time with a register prefetch of the next stage.
//
// CROSS: the non-symmetric job matrix between the rows of two matrices A
// (n rows) and B (nb rows), Section III-B: tile t of the ma x mb tile grid
// is numbered row-major, t = yt * mb + xt (Eq. (7)), and mapped back with
// Eq. (8); every pair of a tile is valid and R is dense, R[i * ldr + j].
#include <math.h>

#include "pcc_internal.h"
#include "pcc_sched.h"

namespace pcc {
namespace {

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int W = 4;
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int W = 2;
};

template <typename T, int H>
struct VecH;
template <>
struct VecH<float, 4> {
  using type = float4;
};
template <>
struct VecH<double, 2> {
  using type = double2;
};

template <typename V, typename T>
__device__ __forceinline__ T vget(const V& v, int q);
template <>
__device__ __forceinline__ float vget<float4, float>(const float4& v, int q) {
  return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}
template <>
__device__ __forceinline__ double vget<double2, double>(const double2& v,
                                                       int q) {
  return q == 0 ? v.x : v.y;
}

struct SimtCross {
  const void* Zb;          // B operand (== A for the triangle)
  const uint8_t* flagsb;
  int64_t nb;              // rows of B
  int64_t mb;              // tile columns (CROSS)
  int64_t ldr;             // row pitch of the dense R (CROSS)
  int64_t r_off;           // R holds the output from element r_off on
};

template <typename T, typename OutT, int BT, int TT, int BK, bool WRITE_R,
          bool EDGES, bool CROSS>
// FP32: two blocks per SM (at one, with 129 registers, the eight warps of a
// block idle together at every stage barrier); FP64: three
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 3)
    k_pairs_simt(const T* __restrict__ Z, const uint8_t* __restrict__ flags,
                 int64_t n, int64_t lpad, int64_t m, int64_t t0,
                 OutT* __restrict__ R, float tau, pcc_edge* __restrict__ edges,
                 uint64_t cap, unsigned long long* __restrict__ count,
                 int* __restrict__ status, const SimtCross cx) {
  const T* __restrict__ Zb = CROSS ? static_cast<const T*>(cx.Zb) : Z;
  const uint8_t* __restrict__ flagsb = CROSS ? cx.flagsb : flags;
  const int64_t nb = CROSS ? cx.nb : n;
  static_assert((BT / TT) * (BT / TT) == 256, "256 threads per tile");
  constexpr int H = TT / 2;
  constexpr int PAD = 4;
  using V = typename Vec16<T>::type;
  constexpr int VW = Vec16<T>::W;
  constexpr int NV = BT * BK / 256 / VW;  // vector loads per thread/operand
  using VH = typename VecH<T, H>::type;

  // operand stages; after the K loop the same memory stages the tile for
  // the stores, half of its rows at a time
  __shared__ __align__(16) T smem_ops[4 * BK * (BT + PAD)];
  static_assert(BT / 2 <= 4 * BK, "a half tile fits the operand stages");
  auto As = reinterpret_cast<T(*)[BK][BT + PAD]>(smem_ops);
  auto Bs = reinterpret_cast<T(*)[BK][BT + PAD]>(smem_ops +
                                                  2 * BK * (BT + PAD));
  __shared__ uint8_t fr[BT], fc[BT];

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  int64_t yt, xt;
  if constexpr (CROSS) {
    const int64_t t = t0 + (int64_t)blockIdx.x;
    yt = t / cx.mb;  // Eq. (8)
    xt = t - yt * cx.mb;
  } else {
    tri_coords(m, t0 + (int64_t)blockIdx.x, &yt, &xt);
  }
  const int64_t row0 = yt * BT, col0 = xt * BT;

  if (tid < BT) {
    fr[tid] = (row0 + tid < n) ? flags[row0 + tid] : 1;
    fc[tid] = (col0 + tid < nb) ? flagsb[col0 + tid] : 1;
  }

  V ra[NV], rb[NV];
  // thread -> (row, group of VW k values): four neighbouring threads read
  // 64 contiguous bytes of one row (coalesced); the transposed stores
  // As[k][r] of a warp then cover 8 rows at 4 k groups, and for FP32 the
  // k rows 8..15 keep their columns XOR 8 (whole float4 groups move) so
  // that those 4 groups fall on distinct banks (row pitch BT + 4 words)
  auto swz = [](int k) { return sizeof(T) == 4 ? ((k >> 3) & 1) * 8 : 0; };
  // a thread's NV vectors are rows r0, r0 + RV, ... at one k group
  constexpr int RV = 256 / (BK / VW);  // rows covered by one vector round
  const int r0 = tid / (BK / VW);
  const int kq0 = (tid % (BK / VW)) * VW;
  const T* __restrict__ pa = Z + (row0 + r0) * lpad + kq0;
  const T* __restrict__ pb = Zb + (col0 + r0) * lpad + kq0;
  const int64_t vstride = (int64_t)RV * lpad;
  auto gload = [&](int64_t kb) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int64_t off = v * vstride + kb * BK;
      ra[v] = (row0 + r0 + v * RV < n)
                  ? *reinterpret_cast<const V*>(pa + off) : V{};
      rb[v] = (col0 + r0 + v * RV < nb)
                  ? *reinterpret_cast<const V*>(pb + off) : V{};
    }
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int r = r0 + v * RV;
      const int kq = kq0;
#pragma unroll
      for (int q = 0; q < VW; ++q) {
        As[buf][kq + q][r ^ swz(kq + q)] = vget<V, T>(ra[v], q);
        Bs[buf][kq + q][r ^ swz(kq + q)] = vget<V, T>(rb[v], q);
      }
    }
  };

  T acc[TT][TT];
#pragma unroll
  for (int a = 0; a < TT; ++a)
#pragma unroll
    for (int b = 0; b < TT; ++b) acc[a][b] = T(0);

  const int64_t nkb = lpad / BK;
  gload(0);
  sstore(0);
  __syncthreads();
  for (int64_t kb = 0; kb < nkb; ++kb) {
    const int cur = kb & 1;
    if (kb + 1 < nkb) gload(kb + 1);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T a[TT], b[TT];
      const int sw = swz(k);
      const VH a0 =
          *reinterpret_cast<const VH*>(&As[cur][k][(ty * H) ^ sw]);
      const VH a1 =
          *reinterpret_cast<const VH*>(&As[cur][k][(BT / 2 + ty * H) ^ sw]);
      const VH b0 =
          *reinterpret_cast<const VH*>(&Bs[cur][k][(tx * H) ^ sw]);
      const VH b1 =
          *reinterpret_cast<const VH*>(&Bs[cur][k][(BT / 2 + tx * H) ^ sw]);
#pragma unroll
      for (int q = 0; q < H; ++q) {
        a[q] = vget<VH, T>(a0, q);
        a[H + q] = vget<VH, T>(a1, q);
        b[q] = vget<VH, T>(b0, q);
        b[H + q] = vget<VH, T>(b1, q);
      }
#pragma unroll
      for (int i = 0; i < TT; ++i)
#pragma unroll
        for (int j = 0; j < TT; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (kb + 1 < nkb) {
      sstore(cur ^ 1);
      __syncthreads();
    }
  }

  // Stores: each half of the tile's rows goes through shared memory, so
  // that a warp writes 32 consecutive pairs of one row per instruction (a
  // packed row's pairs are contiguous; thread blocks of 8 x 8 in registers
  // would touch 16 sectors per store instruction).
  const int lane = tid & 31, warp = tid >> 5;
  T(*tile)[BT + PAD] = reinterpret_cast<T(*)[BT + PAD]>(smem_ops);
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    __syncthreads();  // operand stages (or the previous half) are free
#pragma unroll
    for (int a = 0; a < H; ++a) {
      const int li = ty * H + a;  // row within the half
      const T* q = acc[half * H + a];
      VH v0, v1;
      if constexpr (H == 4) {
        v0 = make_float4(q[0], q[1], q[2], q[3]);
        v1 = make_float4(q[4], q[5], q[6], q[7]);
      } else {
        v0 = make_double2(q[0], q[1]);
        v1 = make_double2(q[2], q[3]);
      }
      *reinterpret_cast<VH*>(&tile[li][tx * H]) = v0;
      *reinterpret_cast<VH*>(&tile[li][BT / 2 + tx * H]) = v1;
    }
    __syncthreads();
    for (int li = warp; li < BT / 2; li += 8) {
      const int ri = half * (BT / 2) + li;  // row within the tile
      const int64_t i = row0 + ri;
      if (i >= n) break;
      const int64_t base =
          (CROSS ? i * cx.ldr : pair_row_base(n, i)) - cx.r_off;
#pragma unroll
      for (int c = 0; c < BT / 32; ++c) {
        const int lj = c * 32 + lane;
        const int64_t j = col0 + lj;
        const bool valid = (j < nb) && (CROSS || j > i);
        const bool flagged = (fr[ri] | fc[lj]) != 0;
        T v = tile[li][lj];
        v = v > T(1) ? T(1) : (v < T(-1) ? T(-1) : v);
        if (flagged) v = T(NAN);
        if constexpr (WRITE_R) {
          if (valid) R[base + j] = (OutT)v;
        }
        if constexpr (EDGES) {
          const bool e = valid && !flagged && fabs((double)v) >= (double)tau;
          const unsigned mask = __ballot_sync(0xffffffffu, e);
          if (mask) {
            const int leader = __ffs(mask) - 1;
            unsigned long long basei = 0;
            if (lane == leader)
              basei = atomicAdd(count, (unsigned long long)__popc(mask));
            basei = __shfl_sync(0xffffffffu, basei, leader);
            if (e) {
              const unsigned long long idx =
                  basei + __popc(mask & ((1u << lane) - 1u));
              if (idx < cap) {
                edges[idx].i = (uint32_t)i;
                edges[idx].j = (uint32_t)j;
                edges[idx].r = (float)v;
              } else {
                atomicCAS(status, 0, (int)PCC_ERR_CAPACITY);
              }
            }
          }
        }
      }
    }
  }
}

template <typename T, typename OutT, int BT, int TT, bool CROSS>
cudaError_t launch_t(const pcc_zmat* Z, OutT* R, int64_t t0, int64_t t1,
                     bool edges_on, float tau, pcc_edge* edges, uint64_t cap,
                     unsigned long long* count, cudaStream_t s,
                     const SimtCross& cx) {
  const int64_t m = (Z->n + BT - 1) / BT;
  const int64_t nblocks = t1 - t0;
  if (nblocks <= 0) return cudaSuccess;
  if (nblocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  const T* z = reinterpret_cast<const T*>(Z->z);
  if (edges_on && R)
    k_pairs_simt<T, OutT, BT, TT, 16, true, true, CROSS>
        <<<(unsigned)nblocks, 256, 0, s>>>(z, Z->flags, Z->n, Z->lpad, m, t0,
                                           R, tau, edges, cap, count,
                                           Z->status, cx);
  else if (edges_on)
    k_pairs_simt<T, OutT, BT, TT, 16, false, true, CROSS>
        <<<(unsigned)nblocks, 256, 0, s>>>(z, Z->flags, Z->n, Z->lpad, m, t0,
                                           R, tau, edges, cap, count,
                                           Z->status, cx);
  else
    k_pairs_simt<T, OutT, BT, TT, 16, true, false, CROSS>
        <<<(unsigned)nblocks, 256, 0, s>>>(z, Z->flags, Z->n, Z->lpad, m, t0,
                                           R, tau, edges, cap, count,
                                           Z->status, cx);
  return cudaGetLastError();
}

template <bool CROSS>
cudaError_t launch_prec(const pcc_zmat* Z, void* R, pcc_dtype rt, int64_t t0,
                        int64_t t1, float tau, pcc_edge* edges, uint64_t cap,
                        unsigned long long* count, cudaStream_t s,
                        const SimtCross& cx) {
  const bool edges_on = count != nullptr;
  if (Z->prec == PCC_PREC_FP32)
    return launch_t<float, float, 128, 8, CROSS>(
        Z, reinterpret_cast<float*>(R), t0, t1, edges_on, tau, edges, cap,
        count, s, cx);
  if (rt == PCC_F64)
    return launch_t<double, double, 64, 4, CROSS>(
        Z, reinterpret_cast<double*>(R), t0, t1, edges_on, tau, edges, cap,
        count, s, cx);
  return launch_t<double, float, 64, 4, CROSS>(Z, reinterpret_cast<float*>(R),
                                               t0, t1, edges_on, tau, edges,
                                               cap, count, s, cx);
}

}  // namespace

int simt_tile_size(pcc_prec p) { return p == PCC_PREC_FP64 ? 64 : 128; }

cudaError_t launch_simt_pairs(const pcc_zmat* Z, void* R, pcc_dtype rt,
                              int64_t t0, int64_t t1, float tau,
                              pcc_edge* edges, uint64_t cap,
                              unsigned long long* count, cudaStream_t s,
                              int64_t r_off) {
  const SimtCross cx{Z->z, Z->flags, Z->n, 0, 0, r_off};
  return launch_prec<false>(Z, R, rt, t0, t1, tau, edges, cap, count, s, cx);
}

int64_t simt_cross_tiles(const pcc_zmat* ZA, const pcc_zmat* ZB) {
  const int64_t t = simt_tile_size(ZA->prec);
  return ((ZA->n + t - 1) / t) * ((ZB->n + t - 1) / t);
}

cudaError_t launch_simt_cross(const pcc_zmat* ZA, const pcc_zmat* ZB, void* R,
                              pcc_dtype rt, int64_t ldr, int64_t t0,
                              int64_t t1, float tau, pcc_edge* edges,
                              uint64_t cap, unsigned long long* count,
                              cudaStream_t s, int64_t r_off) {
  const int64_t t = simt_tile_size(ZA->prec);
  const SimtCross cx{ZB->z, ZB->flags, ZB->n, (ZB->n + t - 1) / t, ldr,
                     r_off};
  return launch_prec<true>(ZA, R, rt, t0, t1, tau, edges, cap, count, s, cx);
}

}  // namespace pcc
