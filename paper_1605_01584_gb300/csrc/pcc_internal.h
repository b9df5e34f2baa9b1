// pcc_internal.h -- library-private declarations shared by the .cu files.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "pcc.h"

// Library-owned standardized matrix (Eq. (5)): one device allocation holds
// the row data, the per-row flags and the device status word.
struct pcc_zmat {
  int device;
  int64_t n, l, lpad;      // lpad: row length rounded up to 64 elements
  pcc_prec prec;           // resolved (never PCC_PREC_AUTO)
  int32_t scale_exp;       // FP16X3S: z stored as z * 2^scale_exp
  void* base;              // the single allocation
  size_t bytes;
  void* hi;                // split forms: n x lpad 16-bit
  void* lo;                // split forms with 3 products: n x lpad 16-bit
  void* z;                 // FP32 / FP64 forms: n x lpad
  uint8_t* flags;          // n bytes
  int* status;             // device status word (pcc_status codes)
  CUtensorMap tm_hi;       // TMA maps over hi/lo: box 64 x 128, 128-B swizzle
  CUtensorMap tm_lo;
  CUtensorMap tm_hi32;     // the same with box 32 x 128, 64-B swizzle
  CUtensorMap tm_lo32;
  // permutation-test work buffer (allocated by the first pcc_perm_test)
  void* perm_ws;
  size_t perm_ws_bytes;
  // windows and pinned staging of the host-delivery passes (kept between
  // calls, grown when a call needs more)
  void* win_ws;
  size_t win_ws_bytes;
  void* stage_ws;
  size_t stage_ws_bytes;
  // device copy of a host input (pcc_standardize_host), kept between calls
  void* xin_ws;
  size_t xin_ws_bytes;
  // FP32 form: the k-major copy the CUDA-core pair kernel reads (made by
  // its first call after each standardize, which clears zt_valid)
  void* zt;
  size_t zt_bytes;
  int zt_valid;
};

namespace pcc {

constexpr int kLpadAlign = 64;

bool is_split(pcc_prec p);
// PCC_PREC_AUTO -> the split form for rows of length l; others unchanged
pcc_prec resolve_prec(pcc_prec p, int64_t l);
int num_sms(int device);
// Per-device slot of a small cache (devices 0 .. kDeviceSlots-1; larger ids
// share the last slot).
constexpr int kDeviceSlots = 64;
inline int device_slot(int device) {
  return device < 0 ? 0 : (device < kDeviceSlots ? device : kDeviceSlots - 1);
}
uint64_t wait_limit_ns();
// test hook of pcc_debug_drop_loads: 0 off, 1 every producer, 2 the odd
// CTA of each pair, 3 the even CTA of each pair
int debug_drop_loads();
cudaError_t ensure_func_smem(const void* func, int bytes);
// True while `s` is being captured into a CUDA graph.
bool stream_capturing(cudaStream_t s);
pcc_status cuda_status(cudaError_t e);

// TMA descriptor of a 2-D row-major 16-bit matrix rows x cols (cols a
// multiple of 8), box box_cols (64 or 32) columns x box_rows rows, swizzle of
// 2*box_cols bytes, zero fill out of bounds.
bool encode_tmap_2d_u16(CUtensorMap* map, const void* base, int64_t rows,
                        int64_t cols, int box_rows, int box_cols, bool bf16);
// 3-D variant: depth x rows x cols, box box_cols x box_rows x 1.
bool encode_tmap_3d_u16(CUtensorMap* map, const void* base, int64_t depth,
                        int64_t rows, int64_t cols, int box_rows, int box_cols,
                        bool bf16);

// Knobs of the tensor-core kernels (the tuner's choices).  Initial values
// come from PCC_TC_BK, PCC_TC_CLUSTER, PCC_TC_PAIR, PCC_TC_BAND,
// PCC_TC_ONEACC, PCC_TC_CHUNK; pcc_set_tuning changes them for later
// launches.
struct TcTuning {
  int stage_k;       // K per ring stage: 32 or 64
  int cluster;       // 2 = CTA pairs (with pair_mma), 1 = single CTAs
  int pair_mma;      // CTA pairs run one 2-SM MMA (M = 256), each CTA
                     // loading only its half of B; 0 = single CTAs
  int64_t band;      // super-tile rows per band of the pair schedule
  double cost_c0;    // batched plan: cycles per unit outside the K loop
  double cost_c1;    // batched plan: cycles per K block and product
  int64_t one_acc_l;  // padded rows up to this length use one accumulator
  int64_t chunk_l;    // longer rows: accumulator chunks of at most this
  int perm_form;       // pcc_perm_form of the permutation test
};
TcTuning tc_tuning();
void tc_set_tuning(const TcTuning& t);
// Accumulator chunks of a work unit with padded rows of lpad samples
// (tc_common.cuh): 1 up to one_acc_l samples, else enough chunks of at most
// chunk_l samples (at least 2, at most lpad / 64), whatever the stage size.
int accum_chunks(int64_t lpad);

// K1: standardize rows of X into Z's storage.
cudaError_t launch_standardize(const void* X, pcc_dtype xt, int64_t ldx,
                               pcc_zmat* Z, cudaStream_t s);
// K1 for many FP32 matrices: one launch per stored form and up to
// kStdBatchMax matrices (the matrix table is a kernel parameter).
constexpr int kStdBatchMax = 96;
cudaError_t launch_standardize_batched(const float* const* Xs,
                                       const int64_t* ldxs, pcc_zmat* const* Zs,
                                       int count, cudaStream_t s);

// K4/K5: CUDA-core pair kernels (FP32 / FP64 Z), tiles [t0, t1) of the
// paper's triangular tile order.
int simt_tile_size(pcc_prec p);
// r_off: R holds the output from element r_off on (a window of rows).
cudaError_t launch_simt_pairs(const pcc_zmat* Z, void* R, pcc_dtype rt,
                              int64_t t0, int64_t t1, float tau,
                              pcc_edge* edges, uint64_t cap,
                              unsigned long long* count, cudaStream_t s,
                              int64_t r_off = 0);

// K2/K3: tensor-core pair kernel, tiles [t0, t1) of the banded super-tile
// order (pcc_sched.h).
int64_t tc_num_tiles(int64_t n);
// G > 0 overrides the tuning's band rows (the tile numbering follows it).
cudaError_t launch_tc_pairs(const pcc_zmat* Z, float* R, int64_t t0,
                            int64_t t1, bool edges_on, float tau,
                            pcc_edge* edges, uint64_t cap,
                            unsigned long long* count, cudaStream_t s,
                            int64_t r_off = 0, int64_t G = 0);

// Non-symmetric pairs between the rows of ZA and ZB (Eq. (7)-(8)), dense R
// with row pitch ldr, tiles [t0, t1) of the cross schedule.
int64_t tc_cross_tiles(int64_t na, int64_t nb);
cudaError_t launch_tc_cross(const pcc_zmat* ZA, const pcc_zmat* ZB, float* R,
                            int64_t ldr, int64_t t0, int64_t t1,
                            bool edges_on, float tau, pcc_edge* edges,
                            uint64_t cap, unsigned long long* count,
                            cudaStream_t s, int64_t r_off = 0,
                            int64_t G = 0);
int64_t simt_cross_tiles(const pcc_zmat* ZA, const pcc_zmat* ZB);
cudaError_t launch_simt_cross(const pcc_zmat* ZA, const pcc_zmat* ZB, void* R,
                              pcc_dtype rt, int64_t ldr, int64_t t0,
                              int64_t t1, float tau, pcc_edge* edges,
                              uint64_t cap, unsigned long long* count,
                              cudaStream_t s, int64_t r_off = 0);

// Passes of whole row blocks into two device windows, copied to host memory
// while the next pass computes (ZB = NULL: the packed triangle of ZA).
struct HostEdges {   // the edge list written by the same passes
  float tau;
  pcc_edge* edges;
  uint64_t cap;
  unsigned long long* count;
};
pcc_status allpairs_host(const pcc_zmat* ZA, const pcc_zmat* ZB, void* host,
                         pcc_dtype rt, int64_t ldh, int64_t device_bytes,
                         pcc_rows_sink sink, void* user, cudaStream_t s,
                         const HostEdges* he = nullptr);

// K7: all pairs of B matrices in one persistent launch per CTA form; pair
// and band (B entries each, or NULL for the current tuning) choose each
// matrix's form (1 = 2-SM CTA pairs) and band rows.
pcc_status allpairs_batched(const pcc_zmat* const* Zs, int32_t B,
                            float* const* Rs, const int32_t* pair,
                            const int32_t* band, cudaStream_t s);

// K6: permutation test over permutations [k0, k1) of d_perms (P x l).
pcc_status perm_test(pcc_zmat* Z, const int32_t* d_perms, int32_t P,
                     int32_t k0, int32_t k1, uint32_t* d_counts,
                     cudaStream_t s);
// K6 on CTA pairs that permute the column rows in shared memory
// (tc_perm_smem.cu): for rows of up to 256 padded samples, when the pair
// form is on and the shared-memory form is selected (perm_form PCC_PERM_SMEM).
bool perm_smem_applies(const pcc_zmat* Z);
pcc_status perm_test_smem(pcc_zmat* Z, const int32_t* d_perms, int32_t k0,
                          int32_t k1, uint32_t* d_counts, cudaStream_t s);
// K6 on CTA pairs that copy the permuted column operand from a transposed
// copy of Z (tc_perm_mn.cu): rows of up to 256 padded samples, pair form on,
// perm_form PCC_PERM_TRANSPOSED.
bool perm_mn_applies(const pcc_zmat* Z);
pcc_status perm_test_mn(pcc_zmat* Z, const int32_t* d_perms, int32_t k0,
                        int32_t k1, uint32_t* d_counts, cudaStream_t s);

}  // namespace pcc
