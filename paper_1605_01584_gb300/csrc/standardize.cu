// standardize.cu -- K1: the variable transformation of Eq. (5) / Algorithm 3.
//
// One warp per row.  Per row, in FP64 (where the cancellation of a large
// mean against small deviations needs it):
//   mean = sum_k x_k / l                       (pass 1, warp-shuffle sum)
//   S    = sum_k (x_k - mean)^2                (pass 2, warp-shuffle sum)
// then z_k = (x_k - mean) / sqrt(S) is formed element by element and
// stored in the form the pair kernels read:
//   BF16X3  hi = bf16(z), lo = bf16(z - hi)
//   FP16X3S hi = fp16(z 2^s), lo = fp16(z 2^s - hi)   (s >= 0 keeps the
//           low half out of the FP16 subnormal range)
//   BF16X1  hi = bf16(z)
//   FP32    z in FP32;  FP64  z in FP64
// For FP32 input the element-wise step runs in FP32 pairs: the FP64 mean is
// split into hi + lo floats and x - mean is formed by an exact two-term
// difference (Knuth's TwoSum), so the deviation keeps FP32 relative
// accuracy however large the mean is.  Rows are padded with zeros to lpad.
// The FP64 output form keeps every step in FP64.
// A row with S == 0 or a non-finite S is flagged and stored as zeros.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "pcc_internal.h"

namespace pcc {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

enum : int { M_BF16X3 = 0, M_FP16X3S = 1, M_BF16X1 = 2, M_FP32 = 3, M_FP64 = 4 };

// x - (mh + ml) for float x, with the rounding error of x - mh recovered
// exactly (TwoSum) and folded in before the final rounding.
__device__ __forceinline__ float dev_ff(float x, float mh, float ml) {
  float s = x - mh;
  float v = s - x;
  float e = (x - (s - v)) + (-mh - v);  // exact: x - mh = s + e
  return s + (e - ml);
}

// (s, c) += x: Knuth's TwoSum adds the exact rounding error of s + x to
// the compensation c (explicit _rn operations keep the compiler from
// reassociating or contracting them).
__device__ __forceinline__ void ff_add(float& s, float& c, float x) {
  const float t = __fadd_rn(s, x);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
  s = t;
  c = __fadd_rn(c, err);
}

// (s, c) += d*d with the product split exactly: p = fl(d*d), e = d*d - p.
__device__ __forceinline__ void ff_add_sq(float& s, float& c, float d) {
  const float p = __fmul_rn(d, d);
  const float e = fmaf(d, d, -p);
  ff_add(s, c, p);
  c = __fadd_rn(c, e);
}

template <typename TX, int MODE>
__global__ void __launch_bounds__(256)
    k_standardize(const TX* __restrict__ X, int64_t n, int64_t l, int64_t ldx,
                  int64_t lpad, float zscale, void* __restrict__ out0,
                  void* __restrict__ out1, uint8_t* __restrict__ flags) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp0; i < n; i += nwarps) {
    const TX* x = X + i * ldx;
    double s = 0.0;
    for (int64_t k = lane; k < l; k += 32) s += (double)x[k];
    const double mean = warp_sum(s) / (double)l;
    double q = 0.0;
    for (int64_t k = lane; k < l; k += 32) {
      const double d = (double)x[k] - mean;
      q = fma(d, d, q);
    }
    q = warp_sum(q);
    const bool bad = !(q > 0.0) || !isfinite(q);
    if (lane == 0) flags[i] = bad ? 1 : 0;
    const double inv = bad ? 0.0 : 1.0 / sqrt(q);

    if constexpr (MODE == M_FP64) {
      double* zr = reinterpret_cast<double*>(out0) + i * lpad;
      for (int64_t k = lane; k < lpad; k += 32)
        zr[k] = (k < l && !bad) ? ((double)x[k] - mean) * inv : 0.0;
    } else if constexpr (MODE == M_FP32) {
      float* zr = reinterpret_cast<float*>(out0) + i * lpad;
      const float mh = (float)mean, ml = (float)(mean - (double)mh);
      const float invf = (float)inv;
      for (int64_t k = lane; k < lpad; k += 32) {
        float z = 0.f;
        if (k < l && !bad) {
          if constexpr (sizeof(TX) == 8)
            z = (float)(((double)x[k] - mean) * inv);
          else
            z = dev_ff((float)x[k], mh, ml) * invf;
        }
        zr[k] = z;
      }
    } else {
      // split forms: each lane writes two adjacent 16-bit elements at once
      const float mh = (float)mean, ml = (float)(mean - (double)mh);
      const float invf = (float)(inv * (double)zscale);
      for (int64_t k = 2 * lane; k < lpad; k += 64) {
        float z0 = 0.f, z1 = 0.f;
        if (!bad) {
          if constexpr (sizeof(TX) == 8) {
            if (k < l) z0 = (float)(((double)x[k] - mean) * inv * zscale);
            if (k + 1 < l)
              z1 = (float)(((double)x[k + 1] - mean) * inv * zscale);
          } else {
            if (k < l) z0 = dev_ff((float)x[k], mh, ml) * invf;
            if (k + 1 < l) z1 = dev_ff((float)x[k + 1], mh, ml) * invf;
          }
        }
        if constexpr (MODE == M_FP16X3S) {
          const __half h0 = __float2half_rn(z0), h1 = __float2half_rn(z1);
          const __half g0 = __float2half_rn(z0 - __half2float(h0));
          const __half g1 = __float2half_rn(z1 - __half2float(h1));
          reinterpret_cast<__half2*>(out0)[(i * lpad + k) >> 1] =
              __halves2half2(h0, h1);
          reinterpret_cast<__half2*>(out1)[(i * lpad + k) >> 1] =
              __halves2half2(g0, g1);
        } else {
          const __nv_bfloat16 h0 = __float2bfloat16_rn(z0);
          const __nv_bfloat16 h1 = __float2bfloat16_rn(z1);
          reinterpret_cast<__nv_bfloat162*>(out0)[(i * lpad + k) >> 1] =
              __halves2bfloat162(h0, h1);
          if constexpr (MODE == M_BF16X3) {
            const __nv_bfloat16 g0 =
                __float2bfloat16_rn(z0 - __bfloat162float(h0));
            const __nv_bfloat16 g1 =
                __float2bfloat16_rn(z1 - __bfloat162float(h1));
            reinterpret_cast<__nv_bfloat162*>(out1)[(i * lpad + k) >> 1] =
                __halves2bfloat162(g0, g1);
          }
        }
      }
    }
  }
}

// FP32 input (16-byte loads when rows are 16-B aligned).  GB300 has
// little FP64 throughput, so each lane forms its partial sums of x and of
// d^2 as error-free float pairs (TwoSum, exact FMA-split squares, relative
// error ~2^-44) and only those partials are converted and summed across the
// row in FP64: the row mean and centred sum of squares are FP64 values at a
// cost of a few FP64 operations per lane instead of per element.
// sum over the 8 lanes of an 8-lane group (xor offsets stay in the group)
__device__ __forceinline__ double group8_sum(double v) {
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// four consecutive floats at x + k (ALIGNED: one 16-byte load)
template <bool ALIGNED>
__device__ __forceinline__ float4 load4(const float* x, int64_t k) {
  if constexpr (ALIGNED) {
    return *reinterpret_cast<const float4*>(x + k);
  } else {
    return make_float4(x[k], x[k + 1], x[k + 2], x[k + 3]);
  }
}

// The rows of one matrix, warps warp0, warp0 + nwarps, ... of a launch.
template <int MODE, bool ALIGNED>
__device__ __forceinline__ void standardize_rows_f32v(
    const float* __restrict__ X, int64_t n, int64_t l, int64_t ldx,
    int64_t lpad, double inv_l, float zscale, void* __restrict__ out0,
    void* __restrict__ out1, uint8_t* __restrict__ flags, int64_t warp0,
    int64_t nwarps) {
  // a warp standardizes 4 rows at a time, 8 lanes per row: the per-row
  // FP64 work (3 reduction steps, mean, 1/sqrt) is shared by 4 rows
  const int lane = threadIdx.x & 31;
  const int grp = lane >> 3, gl = lane & 7;
  const int64_t l4 = l & ~int64_t(3);
  for (int64_t i0 = 4 * warp0; i0 < n; i0 += 4 * nwarps) {
    const int64_t i = i0 + grp;
    const bool live = i < n;  // dead groups run along for the shuffles
    const float* x = X + (live ? i : i0) * ldx;
    // pass 1: float-pair partial sums, merged exactly in FP32 and summed
    // over the row's 8 lanes in FP64
    float sh[4] = {0.f, 0.f, 0.f, 0.f}, sl[4] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t k = 4 * gl; k < l4; k += 32) {
      const float4 v = load4<ALIGNED>(x, k);
      ff_add(sh[0], sl[0], v.x);
      ff_add(sh[1], sl[1], v.y);
      ff_add(sh[2], sl[2], v.z);
      ff_add(sh[3], sl[3], v.w);
    }
    for (int64_t k = l4 + gl; k < l; k += 8) ff_add(sh[0], sl[0], x[k]);
#pragma unroll
    for (int t = 1; t < 4; ++t) {
      ff_add(sh[0], sl[0], sh[t]);
      sl[0] = __fadd_rn(sl[0], sl[t]);
    }
    const double mean =
        group8_sum((double)sh[0] + (double)sl[0]) * inv_l;
    const float mh = (float)mean, ml = (float)(mean - (double)mh);
    // pass 2: deviations (one rounding), exact squares, float-pair sums
    float qh[4] = {0.f, 0.f, 0.f, 0.f}, ql[4] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t k = 4 * gl; k < l4; k += 32) {
      const float4 v = load4<ALIGNED>(x, k);
      ff_add_sq(qh[0], ql[0], dev_ff(v.x, mh, ml));
      ff_add_sq(qh[1], ql[1], dev_ff(v.y, mh, ml));
      ff_add_sq(qh[2], ql[2], dev_ff(v.z, mh, ml));
      ff_add_sq(qh[3], ql[3], dev_ff(v.w, mh, ml));
    }
    for (int64_t k = l4 + gl; k < l; k += 8)
      ff_add_sq(qh[0], ql[0], dev_ff(x[k], mh, ml));
#pragma unroll
    for (int t = 1; t < 4; ++t) {
      ff_add(qh[0], ql[0], qh[t]);
      ql[0] = __fadd_rn(ql[0], ql[t]);
    }
    const double q = group8_sum((double)qh[0] + (double)ql[0]);
    const bool bad = !(q > 0.0) || !isfinite(q) || !isfinite(mean);
    if (live && gl == 0) flags[i] = bad ? 1 : 0;
    // 1/sqrt(q): FP32 estimate, one Newton step in FP64 (error ~2^-44)
    double inv = 0.0;
    if (!bad) {
      const double y = (double)rsqrtf((float)q);
      inv = y * (1.5 - 0.5 * q * y * y);
    }
    const float invf = (float)(inv * (double)zscale);
    if (!live) continue;
    for (int64_t k = 4 * gl; k < lpad; k += 32) {
      float z[4] = {0.f, 0.f, 0.f, 0.f};
      if (!bad) {
        if (k + 3 < l) {
          const float4 v = load4<ALIGNED>(x, k);
          z[0] = dev_ff(v.x, mh, ml) * invf;
          z[1] = dev_ff(v.y, mh, ml) * invf;
          z[2] = dev_ff(v.z, mh, ml) * invf;
          z[3] = dev_ff(v.w, mh, ml) * invf;
        } else {
#pragma unroll
          for (int t = 0; t < 4; ++t)
            if (k + t < l) z[t] = dev_ff(x[k + t], mh, ml) * invf;
        }
      }
      const int64_t e = i * lpad + k;
      if constexpr (MODE == M_FP32) {
        *reinterpret_cast<float4*>(reinterpret_cast<float*>(out0) + e) =
            make_float4(z[0], z[1], z[2], z[3]);
      } else if constexpr (MODE == M_FP16X3S) {
        __half h[4], g[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          h[t] = __float2half_rn(z[t]);
          g[t] = __float2half_rn(z[t] - __half2float(h[t]));
        }
        __half2* o0 = reinterpret_cast<__half2*>(out0) + (e >> 1);
        __half2* o1 = reinterpret_cast<__half2*>(out1) + (e >> 1);
        o0[0] = __halves2half2(h[0], h[1]);
        o0[1] = __halves2half2(h[2], h[3]);
        o1[0] = __halves2half2(g[0], g[1]);
        o1[1] = __halves2half2(g[2], g[3]);
      } else {
        __nv_bfloat16 h[4], g[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          h[t] = __float2bfloat16_rn(z[t]);
          g[t] = __float2bfloat16_rn(z[t] - __bfloat162float(h[t]));
        }
        __nv_bfloat162* o0 = reinterpret_cast<__nv_bfloat162*>(out0) + (e >> 1);
        o0[0] = __halves2bfloat162(h[0], h[1]);
        o0[1] = __halves2bfloat162(h[2], h[3]);
        if constexpr (MODE == M_BF16X3) {
          __nv_bfloat162* o1 =
              reinterpret_cast<__nv_bfloat162*>(out1) + (e >> 1);
          o1[0] = __halves2bfloat162(g[0], g[1]);
          o1[1] = __halves2bfloat162(g[2], g[3]);
        }
      }
    }
  }
}

template <int MODE, bool ALIGNED>
__global__ void __launch_bounds__(256)
    k_standardize_f32v(const float* __restrict__ X, int64_t n, int64_t l,
                       int64_t ldx, int64_t lpad, double inv_l, float zscale,
                       void* __restrict__ out0, void* __restrict__ out1,
                       uint8_t* __restrict__ flags) {
  standardize_rows_f32v<MODE, ALIGNED>(
      X, n, l, ldx, lpad, inv_l, zscale, out0, out1, flags,
      ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
      ((int64_t)gridDim.x * blockDim.x) >> 5);
}

// Many matrices in one launch: block row y standardizes matrix y of the
// table (its rows in a grid-stride loop over blockIdx.x), with the same
// arithmetic as the one-matrix launch.
struct StdItem {
  const float* X;
  int64_t n, l, ldx, lpad;
  double inv_l;
  float zscale;
  int aligned;
  void* out0;
  void* out1;
  uint8_t* flags;
};

struct StdTable {
  StdItem it[kStdBatchMax];
};

template <int MODE>
__global__ void __launch_bounds__(256)
    k_standardize_batched(const __grid_constant__ StdTable t) {
  const StdItem& d = t.it[blockIdx.y];
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if (d.aligned)
    standardize_rows_f32v<MODE, true>(d.X, d.n, d.l, d.ldx, d.lpad, d.inv_l,
                                      d.zscale, d.out0, d.out1, d.flags, w0,
                                      nw);
  else
    standardize_rows_f32v<MODE, false>(d.X, d.n, d.l, d.ldx, d.lpad, d.inv_l,
                                       d.zscale, d.out0, d.out1, d.flags, w0,
                                       nw);
}

template <int MODE>
void launch_f32v(const float* X, int64_t ldx, pcc_zmat* Z, int blocks,
                 float zscale, void* o0, void* o1, cudaStream_t s) {
  const bool aligned =
      (ldx % 4) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  if (aligned)
    k_standardize_f32v<MODE, true><<<blocks, 256, 0, s>>>(
        X, Z->n, Z->l, ldx, Z->lpad, 1.0 / (double)Z->l, zscale, o0, o1,
        Z->flags);
  else
    k_standardize_f32v<MODE, false><<<blocks, 256, 0, s>>>(
        X, Z->n, Z->l, ldx, Z->lpad, 1.0 / (double)Z->l, zscale, o0, o1,
        Z->flags);
}

template <typename TX>
cudaError_t launch_mode(const TX* X, int64_t ldx, pcc_zmat* Z,
                        cudaStream_t s) {
  const int threads = 256;
  int64_t blocks = (Z->n + 7) / 8;
  const int64_t cap = (int64_t)num_sms(Z->device) * 8;
  if (blocks > cap) blocks = cap;
  const float zscale = (float)ldexp(1.0, Z->scale_exp);
  if constexpr (sizeof(TX) == 4) {
    if (Z->prec != PCC_PREC_FP64) {
      const float* Xf = reinterpret_cast<const float*>(X);
      switch (Z->prec) {
        case PCC_PREC_BF16X3:
        case PCC_PREC_BF16X4:  // the same halves; the pair kernel differs
          launch_f32v<M_BF16X3>(Xf, ldx, Z, (int)blocks, 1.f, Z->hi, Z->lo, s);
          break;
        case PCC_PREC_FP16X3S:
          launch_f32v<M_FP16X3S>(Xf, ldx, Z, (int)blocks, zscale, Z->hi,
                                 Z->lo, s);
          break;
        case PCC_PREC_BF16X1:
          launch_f32v<M_BF16X1>(Xf, ldx, Z, (int)blocks, 1.f, Z->hi, nullptr,
                                s);
          break;
        default:
          launch_f32v<M_FP32>(Xf, ldx, Z, (int)blocks, 1.f, Z->z, nullptr, s);
          break;
      }
      return cudaGetLastError();
    }
  }
  switch (Z->prec) {
    case PCC_PREC_BF16X3:
    case PCC_PREC_BF16X4:
      k_standardize<TX, M_BF16X3><<<(int)blocks, threads, 0, s>>>(
          X, Z->n, Z->l, ldx, Z->lpad, 1.f, Z->hi, Z->lo, Z->flags);
      break;
    case PCC_PREC_FP16X3S:
      k_standardize<TX, M_FP16X3S><<<(int)blocks, threads, 0, s>>>(
          X, Z->n, Z->l, ldx, Z->lpad, zscale, Z->hi, Z->lo, Z->flags);
      break;
    case PCC_PREC_BF16X1:
      k_standardize<TX, M_BF16X1><<<(int)blocks, threads, 0, s>>>(
          X, Z->n, Z->l, ldx, Z->lpad, 1.f, Z->hi, nullptr, Z->flags);
      break;
    case PCC_PREC_FP32:
      k_standardize<TX, M_FP32><<<(int)blocks, threads, 0, s>>>(
          X, Z->n, Z->l, ldx, Z->lpad, 1.f, Z->z, nullptr, Z->flags);
      break;
    case PCC_PREC_FP64:
      k_standardize<TX, M_FP64><<<(int)blocks, threads, 0, s>>>(
          X, Z->n, Z->l, ldx, Z->lpad, 1.f, Z->z, nullptr, Z->flags);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_standardize(const void* X, pcc_dtype xt, int64_t ldx,
                               pcc_zmat* Z, cudaStream_t s) {
  Z->zt_valid = 0;  // the FP32 form's k-major copy is out of date
  if (xt == PCC_F64)
    return launch_mode(reinterpret_cast<const double*>(X), ldx, Z, s);
  return launch_mode(reinterpret_cast<const float*>(X), ldx, Z, s);
}

cudaError_t launch_standardize_batched(const float* const* Xs,
                                       const int64_t* ldxs, pcc_zmat* const* Zs,
                                       int count, cudaStream_t s) {
  // one launch per stored form; the FP64 form has no FP32 row loop here
  const pcc_prec forms[4] = {PCC_PREC_BF16X3, PCC_PREC_FP16X3S,
                             PCC_PREC_BF16X1, PCC_PREC_FP32};
  for (int b = 0; b < count; ++b) Zs[b]->zt_valid = 0;
  for (int f = 0; f < 4; ++f) {
    int b = 0;
    while (b < count) {
      StdTable t;
      int c = 0;
      int64_t nmax = 0;
      for (; b < count && c < kStdBatchMax; ++b) {
        pcc_zmat* Z = Zs[b];
        const pcc_prec zp =
            Z->prec == PCC_PREC_BF16X4 ? PCC_PREC_BF16X3 : Z->prec;
        if (zp != forms[f]) continue;
        StdItem& d = t.it[c++];
        d.X = Xs[b];
        d.n = Z->n;
        d.l = Z->l;
        d.ldx = ldxs[b];
        d.lpad = Z->lpad;
        d.inv_l = 1.0 / (double)Z->l;
        d.zscale = forms[f] == PCC_PREC_FP16X3S
                       ? (float)ldexp(1.0, Z->scale_exp)
                       : 1.f;
        d.aligned = (ldxs[b] % 4) == 0 &&
                    (reinterpret_cast<uintptr_t>(Xs[b]) & 15) == 0;
        d.out0 = forms[f] == PCC_PREC_FP32 ? Z->z : Z->hi;
        d.out1 = (forms[f] == PCC_PREC_BF16X3 || forms[f] == PCC_PREC_FP16X3S)
                     ? Z->lo
                     : nullptr;
        d.flags = Z->flags;
        if (Z->n > nmax) nmax = Z->n;
      }
      if (c == 0) continue;
      // 32 rows per block and sweep; at most 8 blocks per SM per matrix
      int64_t bx = (nmax + 31) / 32;
      const int64_t cap = (int64_t)num_sms(Zs[0]->device) * 8;
      if (bx > cap) bx = cap;
      const dim3 grid((unsigned)bx, (unsigned)c, 1);
      switch (forms[f]) {
        case PCC_PREC_BF16X3:
          k_standardize_batched<M_BF16X3><<<grid, 256, 0, s>>>(t);
          break;
        case PCC_PREC_FP16X3S:
          k_standardize_batched<M_FP16X3S><<<grid, 256, 0, s>>>(t);
          break;
        case PCC_PREC_BF16X1:
          k_standardize_batched<M_BF16X1><<<grid, 256, 0, s>>>(t);
          break;
        default:
          k_standardize_batched<M_FP32><<<grid, 256, 0, s>>>(t);
          break;
      }
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  // FP64 outputs: one launch each
  for (int b = 0; b < count; ++b)
    if (Zs[b]->prec == PCC_PREC_FP64) {
      cudaError_t e = launch_standardize(Xs[b], PCC_F32, ldxs[b], Zs[b], s);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

}  // namespace pcc
