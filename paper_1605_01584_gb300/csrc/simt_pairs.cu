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
// here).  Instead of one thread per column (the Xeon Phi layout), the
// threads each own a register block of the tile, K is staged through shared
// memory BK at a time with a register prefetch of the next stage.
//
// CROSS: the non-symmetric job matrix between the rows of two matrices A
// (n rows) and B (nb rows), Section III-B: tile t of the ma x mb tile grid
// is numbered row-major, t = yt * mb + xt (Eq. (7)), and mapped back with
// Eq. (8); every pair of a tile is valid and R is dense, R[i * ldr + j].
#include <math.h>

#include "pcc_internal.h"
#include "pcc_ptx.cuh"
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

template <typename V, typename T>
__device__ __forceinline__ T vget(const V& v, int q);
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

// Stores of a finished tile, called by all NT threads of the block: thread
// (tx, ty) holds rows g * BT/GR + ty * W + a and columns h * BT/2 + tx * W + b
// of the tile in acc[g * W + a][h * W + b]; smem holds at least BT/2 rows of
// BT + 4 values (the operand stages, free once the K loop is over).  Each
// half of the tile's rows goes through shared memory, so that a warp writes
// 32 consecutive pairs of one row per instruction (a packed row's pairs are
// contiguous; the threads' register blocks would touch 16 sectors per store
// instruction).  fr/fc: flags of the tile's rows and columns.
template <typename T, typename OutT, int BT, int GR, int NT, bool WRITE_R,
          bool EDGES, bool CROSS>
__device__ __forceinline__ void store_tile(
    const T (&acc)[GR * Vec16<T>::W][2 * Vec16<T>::W], T* smem_ops,
    const uint8_t* fr, const uint8_t* fc, int tid, int64_t row0,
    int64_t col0, int64_t n, int64_t nb, OutT* R, float tau,
    pcc_edge* edges, uint64_t cap, unsigned long long* count, int* status,
    const SimtCross& cx) {
  using V = typename Vec16<T>::type;
  constexpr int W = Vec16<T>::W;
  constexpr int PAD = 4;
  constexpr int NWARP = NT / 32;
  const int tx = tid & 15, ty = tid >> 4;
  const int lane = tid & 31;
  // this lane's columns of the tile: flags and bounds, fixed for the tile
  bool cfl[BT / 32], cin[BT / 32];
#pragma unroll
  for (int c = 0; c < BT / 32; ++c) {
    cfl[c] = fc[c * 32 + lane] != 0;
    cin[c] = col0 + c * 32 + lane < nb;
  }
  const int warp = tid >> 5;
  T(*tile)[BT + PAD] = reinterpret_cast<T(*)[BT + PAD]>(smem_ops);
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    __syncthreads();  // operand stages (or the previous half) are free
    // row groups g of this half: g * BT/GR in [half * BT/2, (half+1) BT/2)
#pragma unroll
    for (int g = half * GR / 2; g < (half + 1) * GR / 2; ++g) {
#pragma unroll
      for (int a = 0; a < W; ++a) {
        const int li = g * (BT / GR) - half * (BT / 2) + ty * W + a;
        const T* q = acc[g * W + a];
        V v0, v1;
        if constexpr (W == 4) {
          v0 = make_float4(q[0], q[1], q[2], q[3]);
          v1 = make_float4(q[4], q[5], q[6], q[7]);
        } else {
          v0 = make_double2(q[0], q[1]);
          v1 = make_double2(q[2], q[3]);
        }
        *reinterpret_cast<V*>(&tile[li][tx * W]) = v0;
        *reinterpret_cast<V*>(&tile[li][BT / 2 + tx * W]) = v1;
      }
    }
    __syncthreads();
    // the value stored for row li, column chunk c of this half (clamped,
    // NaN when flagged), whether it is a pair of the output, and whether
    // it is an edge
    auto value = [&](int li, int c, int64_t i, bool rfl, bool* valid,
                     bool* edge) -> T {
      const int lj = c * 32 + lane;
      const int64_t j = col0 + lj;
      *valid = cin[c] && (CROSS || j > i);
      const bool flagged = rfl || cfl[c];
      T v = tile[li][lj];
      v = v > T(1) ? T(1) : (v < T(-1) ? T(-1) : v);
      if (flagged) v = T(NAN);
      // FP32 values compare in FP32: the same result as in FP64 (both
      // conversions are exact) without the slow FP64 pipe
      bool over;
      if constexpr (sizeof(T) == 4)
        over = fabsf((float)v) >= tau;
      else
        over = fabs((double)v) >= (double)tau;
      *edge = *valid && !flagged && over;
      return v;
    };
    bool hit = false;  // EDGES: some pair of this warp's rows is an edge
    for (int li = warp; li < BT / 2; li += NWARP) {
      const int ri = half * (BT / 2) + li;  // row within the tile
      const int64_t i = row0 + ri;
      if (i >= n) break;
      const int64_t base =
          (CROSS ? i * cx.ldr : pair_row_base(n, i)) - cx.r_off;
      const bool rfl = fr[ri] != 0;
#pragma unroll
      for (int c = 0; c < BT / 32; ++c) {
        bool valid, e;
        const T v = value(li, c, i, rfl, &valid, &e);
        if constexpr (WRITE_R) {
          if (valid) R[base + col0 + c * 32 + lane] = (OutT)v;
        }
        if constexpr (EDGES) hit |= e;
      }
    }
    // edges are rare: only a warp with one rescans its rows of the staged
    // half and appends them, one atomic per warp and 32 columns
    if constexpr (EDGES) {
      if (__any_sync(0xffffffffu, hit)) {
        for (int li = warp; li < BT / 2; li += NWARP) {
          const int ri = half * (BT / 2) + li;
          const int64_t i = row0 + ri;
          if (i >= n) break;
          const bool rfl = fr[ri] != 0;
          for (int c = 0; c < BT / 32; ++c) {
            bool valid, e;
            const T v = value(li, c, i, rfl, &valid, &e);
            const unsigned mask = __ballot_sync(0xffffffffu, e);
            if (!mask) continue;
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
                edges[idx].j = (uint32_t)(col0 + c * 32 + lane);
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

// Thread layout: NT threads as 16 columns (tx) x NT/16 rows (ty) of
// threads; with W = 16 bytes / sizeof(T) (one vector), thread (tx, ty) owns
// the W x W blocks at rows g * BT/GR + ty * W (g < GR groups) and columns
// h * BT/2 + tx * W (h < 2): TR = GR * W rows by TC = 2 * W columns, read per
// k as GR + 2 vectors of shared memory.  This row-major form serves FP64
// (256 threads of 4 x 4); FP32 uses the k-major form below with the same
// thread layout (256 threads of 8 x 8).
template <typename T, typename OutT, int BT, int GR, int NT, int BK,
          bool WRITE_R, bool EDGES, bool CROSS>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 3)
    k_pairs_simt(const T* __restrict__ Z, const uint8_t* __restrict__ flags,
                 int64_t n, int64_t lpad, int64_t m, int64_t t0,
                 OutT* __restrict__ R, float tau, pcc_edge* __restrict__ edges,
                 uint64_t cap, unsigned long long* __restrict__ count,
                 int* __restrict__ status, const SimtCross cx) {
  const T* __restrict__ Zb = CROSS ? static_cast<const T*>(cx.Zb) : Z;
  const uint8_t* __restrict__ flagsb = CROSS ? cx.flagsb : flags;
  const int64_t nb = CROSS ? cx.nb : n;
  using V = typename Vec16<T>::type;
  constexpr int W = Vec16<T>::W;        // elements per 16-byte vector
  constexpr int NTY = NT / 16;          // thread rows
  constexpr int TR = GR * W, TC = 2 * W;
  static_assert(NTY * W * GR == BT && 16 * W * 2 == BT, "thread layout");
  constexpr int PAD = 4;
  constexpr int NV = BT * BK / NT / W;  // vector loads per thread/operand

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

  for (int t = tid; t < BT; t += NT) {
    fr[t] = (row0 + t < n) ? flags[row0 + t] : 1;
    fc[t] = (col0 + t < nb) ? flagsb[col0 + t] : 1;
  }

  V ra[NV], rb[NV];
  // thread -> (row, group of W k values): four neighbouring threads read
  // 64 contiguous bytes of one row (coalesced); the transposed stores
  // As[k][r] of a warp then cover 8 rows at 4 k groups, and for FP32 the
  // k rows 8..15 keep their columns XOR 8 (whole float4 groups move) so
  // that those 4 groups fall on distinct banks (row pitch BT + 4 words)
  auto swz = [](int k) { return sizeof(T) == 4 ? ((k >> 3) & 1) * 8 : 0; };
  // a thread's NV vectors are rows r0, r0 + RV, ... at one k group
  constexpr int RV = NT / (BK / W);  // rows covered by one vector round
  const int r0 = tid / (BK / W);
  const int kq0 = (tid % (BK / W)) * W;
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
#pragma unroll
      for (int q = 0; q < W; ++q) {
        As[buf][kq0 + q][r ^ swz(kq0 + q)] = vget<V, T>(ra[v], q);
        Bs[buf][kq0 + q][r ^ swz(kq0 + q)] = vget<V, T>(rb[v], q);
      }
    }
  };

  T acc[TR][TC];
#pragma unroll
  for (int a = 0; a < TR; ++a)
#pragma unroll
    for (int b = 0; b < TC; ++b) acc[a][b] = T(0);

  const int64_t nkb = lpad / BK;
  gload(0);
  sstore(0);
  __syncthreads();
  for (int64_t kb = 0; kb < nkb; ++kb) {
    const int cur = kb & 1;
    if (kb + 1 < nkb) gload(kb + 1);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T a[TR], b[TC];
      const int sw = swz(k);
#pragma unroll
      for (int g = 0; g < GR; ++g) {
        const V v = *reinterpret_cast<const V*>(
            &As[cur][k][(g * (BT / GR) + ty * W) ^ sw]);
#pragma unroll
        for (int q = 0; q < W; ++q) a[g * W + q] = vget<V, T>(v, q);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const V v = *reinterpret_cast<const V*>(
            &Bs[cur][k][(h * (BT / 2) + tx * W) ^ sw]);
#pragma unroll
        for (int q = 0; q < W; ++q) b[h * W + q] = vget<V, T>(v, q);
      }
#pragma unroll
      for (int i = 0; i < TR; ++i)
#pragma unroll
        for (int j = 0; j < TC; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (kb + 1 < nkb) {
      sstore(cur ^ 1);
      __syncthreads();
    }
  }

  store_tile<T, OutT, BT, GR, NT, WRITE_R, EDGES, CROSS>(
      acc, smem_ops, fr, fc, tid, row0, col0, n, nb, R, tau, edges, cap,
      count, status, cx);
}

// ---------------------------------------------------------------- FP32, k-major
// FP32 pairs from k-major copies of Z (ZT: lpad rows of npad values, value
// (k, i) = z_i[k], npad = n rounded up to the tile with zeros beyond n).
// The BK x BT slice of a tile's rows at one K block is then BK contiguous
// runs of BT values, which 16-byte cp.async copies move to shared memory as
// they are, in a ring of kKmS stages: no staging through registers and no
// transposing stores, so the loop issues little besides the 64 FMAs per k
// of a thread's 8 x 8 block (same thread layout and store path as above).
// Stages of 32 samples ran 2.9% faster than 16 (half the barriers per K);
// 2 or 3 of them gave the same time.
constexpr int kKmBT = 128, kKmNT = 256, kKmBK = 32, kKmS = 3;
constexpr int kKmStage = 2 * kKmBK * kKmBT;         // floats: A, then B
constexpr int kKmSmemBytes = kKmS * kKmStage * 4;   // 96 KB
static_assert(kKmBT / 2 * (kKmBT + 4) <= kKmS * kKmStage,
              "the tile's staging for the stores fits the ring");

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst),
               "l"(src)
               : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <bool WRITE_R, bool EDGES, bool CROSS>
__global__ void __launch_bounds__(kKmNT, 2)
    k_pairs_simt_km(const float* __restrict__ ZT,
                    const float* __restrict__ ZTb,
                    const uint8_t* __restrict__ flags, int64_t n,
                    int64_t npad, int64_t npadb, int64_t lpad, int64_t m,
                    int64_t t0, float* __restrict__ R, float tau,
                    pcc_edge* __restrict__ edges, uint64_t cap,
                    unsigned long long* __restrict__ count,
                    int* __restrict__ status, const SimtCross cx) {
  constexpr int BT = kKmBT, BK = kKmBK, S = kKmS, NT = kKmNT;
  const uint8_t* __restrict__ flagsb = CROSS ? cx.flagsb : flags;
  const int64_t nb = CROSS ? cx.nb : n;
  extern __shared__ __align__(16) float km_smem[];
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
  for (int t = tid; t < BT; t += NT) {
    fr[t] = (row0 + t < n) ? flags[row0 + t] : 1;
    fc[t] = (col0 + t < nb) ? flagsb[col0 + t] : 1;
  }

  // stage s: A rows [BK][BT] at s * kKmStage, B rows right after; a thread
  // copies chunks tid + NT * i of the stage's 2 * BK * BT / 4 16-byte
  // chunks, so each warp copies 512 contiguous bytes of one k row
  constexpr int kChunks = 2 * BK * BT / 4;   // per stage
  constexpr int kOpChunks = BK * BT / 4;     // per operand
  static_assert(kChunks % NT == 0 && BT / 4 == 32, "chunk layout");
  const uint32_t sbase = smem_u32(km_smem);
  auto load_stage = [&](int s, int64_t kb) {
#pragma unroll
    for (int i = 0; i < kChunks / NT; ++i) {
      const int c = tid + i * NT;
      const int op = c / kOpChunks;  // 0: A (rows of the tile), 1: B
      const int kr = (c % kOpChunks) >> 5, c4 = c & 31;
      const int64_t k = kb * BK + kr;
      const float* src = op ? ZTb + k * npadb + col0 + c4 * 4
                            : ZT + k * npad + row0 + c4 * 4;
      cp_async16(sbase + (uint32_t)((s * kKmStage + op * BK * BT + kr * BT +
                                     c4 * 4) * 4),
                 src);
    }
  };

  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;

  const int64_t nkb = lpad / BK;
#pragma unroll
  for (int s = 0; s < S - 1; ++s) {
    if (s < nkb) load_stage(s, s);
    cp_async_commit();
  }
  for (int64_t kb = 0; kb < nkb; ++kb) {
    // stage kb has landed, and every thread is done with stage kb - 1,
    // whose buffer the next copy reuses
    cp_async_wait<S - 2>();
    __syncthreads();
    const int64_t kn = kb + S - 1;
    if (kn < nkb) load_stage((int)(kn % S), kn);
    cp_async_commit();
    const float* As = km_smem + (int)(kb % S) * kKmStage;
    const float* Bs = As + BK * BT;
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(As + k * BT + ty * 4);
      const float4 a1 =
          *reinterpret_cast<const float4*>(As + k * BT + BT / 2 + ty * 4);
      const float4 b0 = *reinterpret_cast<const float4*>(Bs + k * BT + tx * 4);
      const float4 b1 =
          *reinterpret_cast<const float4*>(Bs + k * BT + BT / 2 + tx * 4);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
  }
  cp_async_wait<0>();
  store_tile<float, float, BT, 2, NT, WRITE_R, EDGES, CROSS>(
      acc, km_smem, fr, fc, tid, row0, col0, n, nb, R, tau, edges, cap,
      count, status, cx);
}

// ZT[k][i] = Z[i][k] for k < lpad, i < npad (zero for i >= n), through a
// 32 x 33 shared tile so that both the reads and the writes are coalesced.
__global__ void __launch_bounds__(256)
    k_transpose_f32(const float* __restrict__ Z, int64_t n, int64_t lpad,
                    float* __restrict__ ZT, int64_t npad) {
  __shared__ float t[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t i = i0 + r;
    t[r][threadIdx.x] = i < n ? Z[i * lpad + k0 + threadIdx.x] : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8)
    ZT[(k0 + r) * npad + i0 + threadIdx.x] = t[threadIdx.x][r];
}

int64_t km_npad(int64_t n) { return (n + kKmBT - 1) / kKmBT * kKmBT; }

// The k-major copy of an FP32 Z, made once after each standardize (the
// standardize entry points clear zt_valid); kept in Z.
cudaError_t ensure_zt(const pcc_zmat* Zc, cudaStream_t s) {
  pcc_zmat* Z = const_cast<pcc_zmat*>(Zc);
  // a captured call transposes again: its replay may follow a standardize
  if (Z->zt_valid && !stream_capturing(s)) return cudaSuccess;
  const int64_t npad = km_npad(Z->n);
  const size_t need = (size_t)npad * (size_t)Z->lpad * sizeof(float);
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
  k_transpose_f32<<<dim3((unsigned)(npad / 32), (unsigned)(Z->lpad / 32)),
                    dim3(32, 8), 0, s>>>(static_cast<const float*>(Z->z),
                                         Z->n, Z->lpad,
                                         static_cast<float*>(Z->zt), npad);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) Z->zt_valid = 1;
  return e;
}

template <bool CROSS>
cudaError_t launch_km(const pcc_zmat* Z, const pcc_zmat* ZB, float* R,
                      int64_t t0, int64_t t1, bool edges_on, float tau,
                      pcc_edge* edges, uint64_t cap,
                      unsigned long long* count, cudaStream_t s,
                      const SimtCross& cx) {
  const int64_t m = (Z->n + kKmBT - 1) / kKmBT;
  const int64_t nblocks = t1 - t0;
  if (nblocks <= 0) return cudaSuccess;
  if (nblocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  cudaError_t e = ensure_zt(Z, s);
  if (e == cudaSuccess && CROSS) e = ensure_zt(ZB, s);
  if (e != cudaSuccess) return e;
  const float* zt = static_cast<const float*>(Z->zt);
  const float* ztb = static_cast<const float*>(CROSS ? ZB->zt : Z->zt);
  const int64_t npad = km_npad(Z->n), npadb = km_npad(ZB->n);
  auto go = [&](auto fn) {
    cudaError_t r = ensure_func_smem(reinterpret_cast<const void*>(fn),
                                     kKmSmemBytes);
    if (r != cudaSuccess) return r;
    fn<<<(unsigned)nblocks, kKmNT, kKmSmemBytes, s>>>(
        zt, ztb, Z->flags, Z->n, npad, npadb, Z->lpad, m, t0, R, tau, edges,
        cap, count, Z->status, cx);
    return cudaGetLastError();
  };
  if (edges_on && R) return go(k_pairs_simt_km<true, true, CROSS>);
  if (edges_on) return go(k_pairs_simt_km<false, true, CROSS>);
  return go(k_pairs_simt_km<true, false, CROSS>);
}

template <typename T, typename OutT, int BT, int GR, int NT, bool CROSS>
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
    k_pairs_simt<T, OutT, BT, GR, NT, 16, true, true, CROSS>
        <<<(unsigned)nblocks, NT, 0, s>>>(z, Z->flags, Z->n, Z->lpad, m, t0,
                                           R, tau, edges, cap, count,
                                           Z->status, cx);
  else if (edges_on)
    k_pairs_simt<T, OutT, BT, GR, NT, 16, false, true, CROSS>
        <<<(unsigned)nblocks, NT, 0, s>>>(z, Z->flags, Z->n, Z->lpad, m, t0,
                                           R, tau, edges, cap, count,
                                           Z->status, cx);
  else
    k_pairs_simt<T, OutT, BT, GR, NT, 16, true, false, CROSS>
        <<<(unsigned)nblocks, NT, 0, s>>>(z, Z->flags, Z->n, Z->lpad, m, t0,
                                           R, tau, edges, cap, count,
                                           Z->status, cx);
  return cudaGetLastError();
}

template <bool CROSS>
cudaError_t launch_prec(const pcc_zmat* Z, const pcc_zmat* ZB, void* R,
                        pcc_dtype rt, int64_t t0, int64_t t1, float tau,
                        pcc_edge* edges, uint64_t cap,
                        unsigned long long* count, cudaStream_t s,
                        const SimtCross& cx) {
  const bool edges_on = count != nullptr;
  if (Z->prec == PCC_PREC_FP32)
    return launch_km<CROSS>(Z, ZB, reinterpret_cast<float*>(R), t0, t1,
                            edges_on, tau, edges, cap, count, s, cx);
  if (rt == PCC_F64)
    return launch_t<double, double, 64, 2, 256, CROSS>(
        Z, reinterpret_cast<double*>(R), t0, t1, edges_on, tau, edges, cap,
        count, s, cx);
  return launch_t<double, float, 64, 2, 256, CROSS>(Z, reinterpret_cast<float*>(R),
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
  return launch_prec<false>(Z, Z, R, rt, t0, t1, tau, edges, cap, count, s,
                            cx);
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
  return launch_prec<true>(ZA, ZB, R, rt, t0, t1, tau, edges, cap, count, s,
                           cx);
}

}  // namespace pcc
