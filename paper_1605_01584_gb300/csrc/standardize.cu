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

// FP32 input, rows 16-B aligned (ldx % 4 == 0): float4 loads, four
// independent FP64 accumulators per lane, and the deviations of pass 2
// formed in FP32 pairs (dev_ff, one rounding) before their squares are
// accumulated in FP64, so a row costs 2 FP64 operations per element.
template <int MODE>
__global__ void __launch_bounds__(256)
    k_standardize_f32v(const float* __restrict__ X, int64_t n, int64_t l,
                       int64_t ldx, int64_t lpad, float zscale,
                       void* __restrict__ out0, void* __restrict__ out1,
                       uint8_t* __restrict__ flags) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t l4 = l & ~int64_t(3);
  for (int64_t i = warp0; i < n; i += nwarps) {
    const float* x = X + i * ldx;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int64_t k = 4 * lane; k < l4; k += 128) {
      const float4 v = *reinterpret_cast<const float4*>(x + k);
      s0 += (double)v.x;
      s1 += (double)v.y;
      s2 += (double)v.z;
      s3 += (double)v.w;
    }
    for (int64_t k = l4 + lane; k < l; k += 32) s0 += (double)x[k];
    const double mean = warp_sum((s0 + s1) + (s2 + s3)) / (double)l;
    const float mh = (float)mean, ml = (float)(mean - (double)mh);
    double q0 = 0.0, q1 = 0.0, q2 = 0.0, q3 = 0.0;
    for (int64_t k = 4 * lane; k < l4; k += 128) {
      const float4 v = *reinterpret_cast<const float4*>(x + k);
      const double d0 = (double)dev_ff(v.x, mh, ml);
      const double d1 = (double)dev_ff(v.y, mh, ml);
      const double d2 = (double)dev_ff(v.z, mh, ml);
      const double d3 = (double)dev_ff(v.w, mh, ml);
      q0 = fma(d0, d0, q0);
      q1 = fma(d1, d1, q1);
      q2 = fma(d2, d2, q2);
      q3 = fma(d3, d3, q3);
    }
    for (int64_t k = l4 + lane; k < l; k += 32) {
      const double d = (double)dev_ff(x[k], mh, ml);
      q0 = fma(d, d, q0);
    }
    const double q = warp_sum((q0 + q1) + (q2 + q3));
    const bool bad = !(q > 0.0) || !isfinite(q) || !isfinite(mean);
    if (lane == 0) flags[i] = bad ? 1 : 0;
    const double inv = bad ? 0.0 : 1.0 / sqrt(q);
    const float invf = (float)(inv * (double)zscale);
    for (int64_t k = 4 * lane; k < lpad; k += 128) {
      float z[4] = {0.f, 0.f, 0.f, 0.f};
      if (!bad) {
        if (k + 3 < l) {
          const float4 v = *reinterpret_cast<const float4*>(x + k);
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

template <int MODE>
void launch_f32v(const float* X, int64_t ldx, pcc_zmat* Z, int blocks,
                 float zscale, void* o0, void* o1, cudaStream_t s) {
  k_standardize_f32v<MODE><<<blocks, 256, 0, s>>>(X, Z->n, Z->l, ldx, Z->lpad,
                                                  zscale, o0, o1, Z->flags);
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
    if ((ldx % 4) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
        Z->prec != PCC_PREC_FP64) {
      const float* Xf = reinterpret_cast<const float*>(X);
      switch (Z->prec) {
        case PCC_PREC_BF16X3:
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
  if (xt == PCC_F64)
    return launch_mode(reinterpret_cast<const double*>(X), ldx, Z, s);
  return launch_mode(reinterpret_cast<const float*>(X), ldx, Z, s);
}

}  // namespace pcc
