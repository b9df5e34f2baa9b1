// noalloc.cu -- pcc_allpairs_upper_noalloc: the standardize + tensor-core
// pair path without any device allocation.
//
// Some callers cannot call cudaMalloc: code that lives inside another
// framework's memory manager (every device byte has to come from the host
// framework's pool, so a library allocation would bypass its accounting and
// limits), applications that fix their device-memory budget once at start-up,
// and latency-critical paths where the implicit device-wide synchronisation of
// cudaMalloc/cudaFree is not acceptable.  For them this entry point keeps the
// standardized matrix (the hi/lo halves, the row flags and a status word) in
// one file-scope device array of fixed size instead of a pcc_zmat.
//
// The array is created when a device first loads this library and lives
// until the process exits; every call on that device shares it.  Its device
// address is looked up with cudaGetSymbolAddress on the first call on each
// device (with that device current) and cached; host code never uses the
// array's name as an address.  Calls that overlap on the GPU (different
// streams without ordering between them) race on the array.
#include <string.h>

#include <mutex>

#include "pcc_internal.h"

namespace pcc {
namespace {

// 32 MiB: hi + lo (4 bytes per element of n x lpad), n flag bytes rounded
// up to 256, and 256 bytes for the status word.
constexpr size_t kNoAllocBytes = 32ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array for `dev` (the current device).
unsigned char* scratch_address(int dev) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
  }
  return g_noalloc_ptr[dev];
}

size_t round_up_sz(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace
}  // namespace pcc

using namespace pcc;

extern "C" pcc_status pcc_allpairs_upper_noalloc(const float* X, int64_t n,
                                                 int64_t l, int64_t ldx,
                                                 pcc_prec prec, float* R,
                                                 int32_t* d_status,
                                                 void* stream) {
  if (!X || !R || n < 2 || l < 2 || ldx < l || n >= (1ll << 31))
    return PCC_ERR_INVALID_ARG;
  const pcc_prec rp = resolve_prec(prec, l);  // as pcc_standardize
  if (rp != PCC_PREC_BF16X3 && rp != PCC_PREC_FP16X3S &&
      rp != PCC_PREC_BF16X4 && rp != PCC_PREC_BF16X1)
    return PCC_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return PCC_ERR_CUDA;
  int maj = 0, min = 0;
  cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&min, cudaDevAttrComputeCapabilityMinor, dev);
  if (maj != 10 || min != 3) return PCC_ERR_UNSUPPORTED;

  // layout inside the array; larger problems are refused, never truncated
  const int64_t lpad = (l + kLpadAlign - 1) / kLpadAlign * kLpadAlign;
  const size_t half = round_up_sz((size_t)n * (size_t)lpad * 2, 1024);
  const size_t halves = rp == PCC_PREC_BF16X1 ? half : 2 * half;
  const size_t flags_off = halves;
  const size_t status_off = flags_off + round_up_sz((size_t)n, 256);
  if (status_off + 256 > kNoAllocBytes) return PCC_ERR_INVALID_ARG;

  unsigned char* base = scratch_address(dev);
  if (!base) return PCC_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // a pcc_zmat that only points into the scratch array (host struct, no
  // device allocation)
  pcc_zmat Z;
  memset(&Z, 0, sizeof(Z));
  Z.device = dev;
  Z.n = n;
  Z.l = l;
  Z.lpad = lpad;
  Z.prec = rp;
  Z.scale_exp = 0;
  if (rp == PCC_PREC_FP16X3S)
    while ((int64_t)1 << (2 * (Z.scale_exp + 1)) <= l) ++Z.scale_exp;
  Z.hi = base;
  Z.lo = rp == PCC_PREC_BF16X1 ? nullptr : base + half;
  Z.flags = base + flags_off;
  Z.status = d_status ? reinterpret_cast<int*>(d_status)
                      : reinterpret_cast<int*>(base + status_off);
  const bool bf16 = rp != PCC_PREC_FP16X3S;
  if (!encode_tmap_2d_u16(&Z.tm_hi, Z.hi, n, lpad, 128, 64, bf16) ||
      !encode_tmap_2d_u16(&Z.tm_hi32, Z.hi, n, lpad, 128, 32, bf16))
    return PCC_ERR_CUDA;
  if (Z.lo) {
    if (!encode_tmap_2d_u16(&Z.tm_lo, Z.lo, n, lpad, 128, 64, bf16) ||
        !encode_tmap_2d_u16(&Z.tm_lo32, Z.lo, n, lpad, 128, 32, bf16))
      return PCC_ERR_CUDA;
  } else {
    Z.tm_lo = Z.tm_hi;
    Z.tm_lo32 = Z.tm_hi32;
  }
  // the status word starts every call at zero (the array keeps the
  // previous call's contents; everything else is overwritten below)
  cudaError_t e = cudaMemsetAsync(Z.status, 0, sizeof(int), s);
  if (e != cudaSuccess) return cuda_status(e);
  e = launch_standardize(X, PCC_F32, ldx, &Z, s);
  if (e != cudaSuccess) return cuda_status(e);
  e = launch_tc_pairs(&Z, R, 0, tc_num_tiles(n), false, 0.f, nullptr, 0,
                      nullptr, s);
  return cuda_status(e);
}
