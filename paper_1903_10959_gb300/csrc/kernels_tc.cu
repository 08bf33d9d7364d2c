// Mixed-precision kernels on the 5th-generation tensor cores (tcgen05,
// kind::tf32 and kind::f16, FP32 accumulation in TMEM) for sm_103a.
//
// Precision scheme (the mixed strategy of Secs. 3.4.2 and 3.5.2 of
// arXiv:1903.10959, moved onto tensor cores): every operand x is split into
// x_hi = tf32(x) and x_lo = tf32(x - x_hi); a product a.b is evaluated as
// a_lo.b_hi + a_hi.b_lo + a_hi.b_hi ("3xTF32", binary32-level accuracy) or
// as a_hi.b_hi alone ("1xTF32").  The cell products can instead split both
// operands into three bf16 terms (exact for binary32) and keep the six
// products down to 2^-24 ("BF16x3", kind::f16).  Wavefunction blocks are
// stored in binary32.  Diagonal blocks of the overlap / projected matrices
// and of the CholGS factor are evaluated in binary64 (the paper's S_d and
// L^{-1}_d).
//
//  tc_cell_r    : the cell-by-cell products H~_e Y_e of Sec. 3.3.1 for all
//                 cells in one launch, one CTA per (cell, 64-column tile);
//                 warp-specialised: warp 4 streams the pre-split cell matrix
//                 with bulk async copies, warps 0-3 gather + split the cell
//                 block of Y into shared memory and later store the result
//                 block, warp 5 issues the MMAs.
//  tc_cell_bf16 : the same products in BF16x3 as R_e^T = Y_e^T H~_e, one CTA
//                 per (cell, 128-column tile, part of <= 256 cell rows).
//  tc_assemble  : owner-computes sum of the cell blocks per unknown fused with
//                 the Chebyshev three-term update (Eq. chebFilter).
//  tc_gram      : lower tiles of A^T B over the unknowns (Algorithm CholGS
//                 step 1; H^ of Sec. 3.5), split-K, fixed-order reduction.
//  tc_tallgemm  : X U (Algorithm CholGS step 4, subspace rotation of Sec. 3.5).
#include <algorithm>
#include <cstdio>
#include <mutex>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"
#include "tc.h"
#include "tc_ptx.cuh"

namespace chfsi {

using namespace ptx;

__device__ int g_tc_status = 0;   // nonzero after a bounded wait gave up
// Test hook of the bounded waits (0 = off, the default): when set, gather warp
// 0 of the first CTA of the BF16x3 cell kernel (the shared-ring and the
// decoupled-ring forms) withholds its arrival on the first chunk's full
// barrier, so that the MMA warp's wait on it runs out.
__device__ int g_tc_withhold = 0;

constexpr int CELL_BN = 64;       // default columns per CTA (128 selectable)
constexpr int CELL_KC = 8;        // K per pipeline stage (one MMA K-step)
constexpr int CELL_THREADS = 192;

// ----------------------------------------------------------------- packing
// Cell matrix layout for the MMA A operand: per cell, per K-chunk of 8, the hi
// part for all M-tiles, then the lo part; each M-tile block is 128 rows x 8 K
// in the no-swizzle K-major core-matrix layout (LBO 128 B along K, SBO 256 B
// along M).
__device__ __host__ __forceinline__ int cell_elem_off(int r, int k) {
  return (r >> 3) * 64 + (k >> 2) * 32 + (r & 7) * 4 + (k & 3);   // in floats
}

__global__ void tc_pack_kernel(const double* __restrict__ Ht, float* __restrict__ out,
                               int64_t ncells, int ne, int mt, int nk) {
  const int64_t per_cell = (int64_t)nk * 2 * mt * 1024;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= ncells * per_cell / 2) return;
  // one thread per (cell, kc, mtile, r, k) of the hi half; writes hi and lo
  const int64_t e = idx / (per_cell / 2);
  int64_t rem = idx - e * (per_cell / 2);
  const int kc = (int)(rem / (mt * 1024));
  rem -= (int64_t)kc * mt * 1024;
  const int t = (int)(rem / 1024);
  const int w = (int)(rem - t * 1024);
  const int r = w / 8, k = w % 8;
  const int row = t * 128 + r, col = kc * CELL_KC + k;
  double v = (row < ne && col < ne) ? Ht[(e * ne + row) * (int64_t)ne + col] : 0.0;
  // round to TF32 (nearest, ties away), then the residual
  float hi = ptx::tf32_rna((float)v);
  float lo = ptx::tf32_rna((float)(v - (double)hi));
  float* base = out + e * per_cell + (int64_t)kc * 2 * mt * 1024;
  const int o = cell_elem_off(r, k);
  base[t * 1024 + o] = hi;
  base[mt * 1024 + t * 1024 + o] = lo;
}

cudaError_t tc_build(TcCellData& d, const std::vector<double>&, int64_t ncells, int ne,
                     cudaStream_t s, int64_t* dev_bytes) {
  // the device copy of the binary64 cell matrices is packed by tc_pack_from_device
  (void)s;
  (void)dev_bytes;
  d = TcCellData();
  d.ncells = ncells;
  d.ne = ne;
  d.mt = (ne + 127) / 128;
  d.kt = (ne + CELL_KC - 1) / CELL_KC * CELL_KC;
  return cudaSuccess;
}

cudaError_t tc_pack_from_device(TcCellData& d, const double* dHt, cudaStream_t s,
                                int64_t* dev_bytes) {
  const int nk = d.kt / CELL_KC;
  const size_t per_cell = (size_t)nk * 2 * d.mt * 1024 * sizeof(float);
  d.bytes = per_cell * d.ncells;
  cudaError_t e = cudaMalloc(&d.hi, d.bytes);
  if (e != cudaSuccess) {
    d.hi = nullptr;
    d.bytes = 0;
    return e;
  }
  if (dev_bytes) *dev_bytes += (int64_t)d.bytes;
  const int64_t n = d.ncells * (int64_t)nk * d.mt * 1024;
  note_launch();
  tc_pack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dHt, d.hi, d.ncells, d.ne, d.mt, nk);
  return cudaGetLastError();
}

void tc_free(TcCellData& d) {
  if (d.hi) cudaFree(d.hi);
  if (d.bf) cudaFree(d.bf);
  if (d.f16) cudaFree(d.f16);
  if (d.f16_inv) cudaFree(d.f16_inv);
  if (d.nl) cudaFree(d.nl);
  if (d.nl_off) cudaFree(d.nl_off);
  if (d.nl_zrow) cudaFree(d.nl_zrow);
  for (void* q : {(void*)d.pj, (void*)d.pj_np, (void*)d.pj_off, (void*)d.pj_row, (void*)d.pj_red_ptr,
                  (void*)d.pj_red_row})
    if (q) cudaFree(q);
  d = TcCellData();
}

// ----------------------------------------------------------------- BF16x3 packing
// Each value v ~ b1 + b2 + b3 with b1 = bf16(v), b2 = bf16(v - b1),
// b3 = bf16(v - b1 - b2) (about 24 significant bits together).  Layout: per
// cell, per K-chunk of 16, the three terms one after another, each holding all
// 128-row tiles; a tile block is 128 rows x 16 K bf16 in the no-swizzle
// K-major core-matrix layout (8 rows x 16 B; LBO 128 B along K, SBO 256 B
// along M), the same byte geometry as the TF32 blocks.
constexpr int BF_KC = 16;
__device__ __host__ __forceinline__ int bf_elem_off(int r, int k) {   // in bf16 elements
  return (r >> 3) * 128 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ void bf16_split3(double v, uint16_t& b1, uint16_t& b2, uint16_t& b3) {
  const __nv_bfloat16 h1 = __float2bfloat16_rn((float)v);
  const double r1 = v - (double)__bfloat162float(h1);
  const __nv_bfloat16 h2 = __float2bfloat16_rn((float)r1);
  const double r2 = r1 - (double)__bfloat162float(h2);
  const __nv_bfloat16 h3 = __float2bfloat16_rn((float)r2);
  b1 = __bfloat16_as_ushort(h1);
  b2 = __bfloat16_as_ushort(h2);
  b3 = __bfloat16_as_ushort(h3);
}

// The same split of a binary32 value in binary32 arithmetic: v - b1 and
// r1 - b2 are exact (each term keeps at most 8 significant bits of what is left).
__device__ __forceinline__ void bf16_split3f(float v, uint16_t& b1, uint16_t& b2, uint16_t& b3) {
  const __nv_bfloat16 h1 = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(h1);
  const __nv_bfloat16 h2 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(h2);
  b1 = __bfloat16_as_ushort(h1);
  b2 = __bfloat16_as_ushort(h2);
  b3 = __bfloat16_as_ushort(__float2bfloat16_rn(r2));
}

// The same three-term split for two binary32 values at once, packed the way
// the MMA operand holds them (x0 in the low half, x1 in the high half): one
// cvt.rn.bf16x2.f32 per term (round to nearest even, as __float2bfloat16_rn),
// the back-conversion by a shift or a mask, the remainders exact as above.
__device__ __forceinline__ uint32_t cvt_bf16x2(float hi, float lo) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ __forceinline__ void bf16_split3_pair(float x0, float x1, uint32_t& w1, uint32_t& w2,
                                                 uint32_t& w3) {
  w1 = cvt_bf16x2(x1, x0);
  const float r0 = x0 - __uint_as_float(w1 << 16);
  const float r1 = x1 - __uint_as_float(w1 & 0xffff0000u);
  w2 = cvt_bf16x2(r1, r0);
  const float s0 = r0 - __uint_as_float(w2 << 16);
  const float s1 = r1 - __uint_as_float(w2 & 0xffff0000u);
  w3 = cvt_bf16x2(s1, s0);
}

// Two-term fp16 split of two binary32 values, packed as the MMA operand holds
// them: one cvt.rn.f16x2.f32 per term, the remainders exact in binary32.
__device__ __forceinline__ uint32_t cvt_f16x2(float hi, float lo) {
  uint32_t r;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ __forceinline__ void f16_split2_pair(float x0, float x1, uint32_t& w1, uint32_t& w2) {
  w1 = cvt_f16x2(x1, x0);
  const float r0 = x0 - __half2float(__ushort_as_half((unsigned short)(w1 & 0xffffu)));
  const float r1 = x1 - __half2float(__ushort_as_half((unsigned short)(w1 >> 16)));
  w2 = cvt_f16x2(r1, r0);
}

// add (optional): an n_e x n_e matrix added to every cell's matrix first.
__global__ void tc_pack_bf16_kernel(const double* __restrict__ Ht, uint16_t* __restrict__ out,
                                    int64_t ncells, int ne, int mt, int nk16,
                                    const double* __restrict__ add = nullptr) {
  const int64_t per_chunk = (int64_t)mt * 2048;   // elements of one term, all tiles
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= ncells * nk16 * per_chunk) return;
  // one thread per (cell, chunk, tile, row, k); writes the three terms
  const int64_t e = idx / (nk16 * per_chunk);
  int64_t rem = idx - e * nk16 * per_chunk;
  const int kc = (int)(rem / per_chunk);
  rem -= (int64_t)kc * per_chunk;
  const int t = (int)(rem / 2048);
  const int w = (int)(rem - t * 2048);
  const int r = w / BF_KC, k = w % BF_KC;
  const int row = t * 128 + r, col = kc * BF_KC + k;
  double v = (row < ne && col < ne) ? Ht[(e * ne + row) * (int64_t)ne + col] : 0.0;
  if (add && row < ne && col < ne) v += add[(int64_t)row * ne + col];
  uint16_t b1, b2, b3;
  bf16_split3(v, b1, b2, b3);
  uint16_t* base = out + (e * nk16 + kc) * 3 * per_chunk + (int64_t)t * 2048 + bf_elem_off(r, k);
  base[0] = b1;
  base[per_chunk] = b2;
  base[2 * per_chunk] = b3;
}

cudaError_t tc_pack_bf16_matrices(const double* dH, const double* dadd, int64_t ncells, int ne, uint16_t** out,
                                  size_t* bytes, cudaStream_t s) {
  const int mt = (ne + 127) / 128, nk16 = (ne + BF_KC - 1) / BF_KC;
  const size_t need = (size_t)ncells * nk16 * 3 * mt * 2048 * sizeof(uint16_t);
  if (!*out) {
    cudaError_t e = cudaMalloc(out, need);
    if (e != cudaSuccess) {
      *out = nullptr;
      return e;
    }
    *bytes = need;
  }
  const int64_t n = ncells * (int64_t)nk16 * mt * 2048;
  note_launch();
  tc_pack_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dH, *out, ncells, ne, mt, nk16, dadd);
  return cudaGetLastError();
}

cudaError_t tc_pack_bf16_from_device(TcCellData& d, const double* dHt, cudaStream_t s,
                                     int64_t* dev_bytes) {
  const int nk16 = (d.ne + BF_KC - 1) / BF_KC;
  d.bf_bytes = (size_t)d.ncells * nk16 * 3 * d.mt * 2048 * sizeof(uint16_t);
  cudaError_t e = cudaMalloc(&d.bf, d.bf_bytes);
  if (e != cudaSuccess) {
    d.bf = nullptr;
    d.bf_bytes = 0;
    return e;
  }
  if (dev_bytes) *dev_bytes += (int64_t)d.bf_bytes;
  const int64_t n = d.ncells * (int64_t)nk16 * d.mt * 2048;
  note_launch();
  tc_pack_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dHt, d.bf, d.ncells, d.ne, d.mt, nk16);
  return cudaGetLastError();
}

// Projector chunks: scatter the three bf16 terms of each nonzero coefficient
// into the zeroed chunk array (positions from build_nl_cells, term 0; the
// other terms one term block further on).
__global__ void tc_pack_nl_kernel(const int64_t* __restrict__ pos, const double* __restrict__ val, int64_t nnz,
                                  int64_t per_chunk, uint16_t* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nnz) return;
  uint16_t b1, b2, b3;
  bf16_split3(val[i], b1, b2, b3);
  const int64_t p = pos[i];
  out[p] = b1;
  out[p + per_chunk] = b2;
  out[p + 2 * per_chunk] = b3;
}

cudaError_t tc_pack_nl(TcCellData& d, const int32_t* chunk_off, int64_t ncells, const int32_t* zrow,
                       const int64_t* nz_pos, const double* nz_val, int64_t nnz, cudaStream_t s,
                       int64_t* dev_bytes) {
  const int64_t nchunk = chunk_off[ncells];
  const int64_t per_chunk = (int64_t)d.mt * 2048;
  const size_t bytes = (size_t)nchunk * 3 * per_chunk * sizeof(uint16_t);
  int64_t* dpos = nullptr;
  double* dval = nullptr;
  cudaError_t e = cudaMalloc(&d.nl, std::max<size_t>(bytes, 16));
  if (e == cudaSuccess) e = cudaMalloc(&d.nl_off, (size_t)(ncells + 1) * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&d.nl_zrow, std::max<size_t>((size_t)nchunk * 16 * sizeof(int32_t), 16));
  if (e == cudaSuccess && nnz > 0) e = cudaMalloc(&dpos, (size_t)nnz * sizeof(int64_t));
  if (e == cudaSuccess && nnz > 0) e = cudaMalloc(&dval, (size_t)nnz * sizeof(double));
  if (e == cudaSuccess) e = cudaMemsetAsync(d.nl, 0, bytes, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d.nl_off, chunk_off, (size_t)(ncells + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nchunk > 0)
    e = cudaMemcpyAsync(d.nl_zrow, zrow, (size_t)nchunk * 16 * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(dpos, nz_pos, (size_t)nnz * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(dval, nz_val, (size_t)nnz * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nnz > 0) {
    note_launch();
    tc_pack_nl_kernel<<<(unsigned)((nnz + 255) / 256), 256, 0, s>>>(dpos, dval, nnz, per_chunk, d.nl);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (dpos) cudaFree(dpos);
  if (dval) cudaFree(dval);
  if (e != cudaSuccess) {
    if (d.nl) cudaFree(d.nl);
    if (d.nl_off) cudaFree(d.nl_off);
    if (d.nl_zrow) cudaFree(d.nl_zrow);
    d.nl = nullptr;
    d.nl_off = nullptr;
    d.nl_zrow = nullptr;
    d.nl_bytes = 0;
    return e;
  }
  d.nl_bytes = bytes + (size_t)(ncells + 1) * 4 + (size_t)nchunk * 64;
  if (dev_bytes) *dev_bytes += (int64_t)d.nl_bytes;
  return cudaSuccess;
}

// Projection blocks: the three bf16 terms of each coefficient at its
// position (term 0; the block of one chunk holds np[e] x 16 values per term).
__global__ void tc_pack_proj_kernel(const int64_t* __restrict__ pos, const double* __restrict__ val, int64_t nnz,
                                    const int64_t* __restrict__ poff, const int32_t* __restrict__ np,
                                    int64_t ncells, uint16_t* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nnz) return;
  const int64_t p = pos[i];
  int64_t lo = 0, hi = ncells - 1;   // the cell whose block holds p
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (poff[mid] <= p) lo = mid; else hi = mid - 1;
  }
  const int64_t term = (int64_t)np[lo] * 16;
  uint16_t b1, b2, b3;
  bf16_split3(val[i], b1, b2, b3);
  out[p] = b1;
  out[p + term] = b2;
  out[p + 2 * term] = b3;
}

cudaError_t tc_pack_proj(TcCellData& d, int64_t ncells, int nsite, const int32_t* np, const int64_t* poff,
                         const int64_t* prow, const int32_t* red_ptr, const int64_t* red_row,
                         const int64_t* pz_pos, const double* pz_val, int64_t nnz, cudaStream_t s,
                         int64_t* dev_bytes) {
  int npmax = 0;
  for (int64_t e = 0; e < ncells; ++e) npmax = std::max(npmax, np[e]);
  if (npmax > 256) return cudaErrorNotSupported;   // more than 64 sites on one cell's rows
  const size_t bytes = std::max<size_t>((size_t)poff[ncells] * sizeof(uint16_t), 16);
  const int64_t nred = red_ptr[nsite];
  int64_t* dpos = nullptr;
  double* dval = nullptr;
  cudaError_t e = cudaMalloc(&d.pj, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&d.pj_np, (size_t)ncells * 4);
  if (e == cudaSuccess) e = cudaMalloc(&d.pj_off, (size_t)(ncells + 1) * 8);
  if (e == cudaSuccess) e = cudaMalloc(&d.pj_row, (size_t)(ncells + 1) * 8);
  if (e == cudaSuccess) e = cudaMalloc(&d.pj_red_ptr, (size_t)(nsite + 1) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&d.pj_red_row, std::max<size_t>((size_t)nred * 8, 8));
  if (e == cudaSuccess && nnz > 0) e = cudaMalloc(&dpos, (size_t)nnz * 8);
  if (e == cudaSuccess && nnz > 0) e = cudaMalloc(&dval, (size_t)nnz * 8);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.pj, 0, bytes, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d.pj_np, np, (size_t)ncells * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d.pj_off, poff, (size_t)(ncells + 1) * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d.pj_row, prow, (size_t)(ncells + 1) * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d.pj_red_ptr, red_ptr, (size_t)(nsite + 1) * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nred > 0)
    e = cudaMemcpyAsync(d.pj_red_row, red_row, (size_t)nred * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(dpos, pz_pos, (size_t)nnz * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(dval, pz_val, (size_t)nnz * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nnz > 0) {
    note_launch();
    tc_pack_proj_kernel<<<(unsigned)((nnz + 255) / 256), 256, 0, s>>>(dpos, dval, nnz, d.pj_off, d.pj_np,
                                                                       ncells, d.pj);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (dpos) cudaFree(dpos);
  if (dval) cudaFree(dval);
  if (e != cudaSuccess) {
    for (void* q : {(void*)d.pj, (void*)d.pj_np, (void*)d.pj_off, (void*)d.pj_row, (void*)d.pj_red_ptr,
                    (void*)d.pj_red_row})
      if (q) cudaFree(q);
    d.pj = nullptr;
    d.pj_np = nullptr;
    d.pj_off = nullptr;
    d.pj_row = nullptr;
    d.pj_red_ptr = nullptr;
    d.pj_red_row = nullptr;
    return e;
  }
  d.pj_rows = prow[ncells];
  d.pj_npmax = npmax;
  d.pj_bytes = bytes + (size_t)ncells * 4 + (size_t)(ncells + 1) * 16 + (size_t)(nsite + 1) * 4 + (size_t)nred * 8;
  if (dev_bytes) *dev_bytes += (int64_t)d.pj_bytes;
  return cudaSuccess;
}

// Z[4 s + t][c] = sum over the (cell, slot) partial rows of site s, in the
// fixed (ascending cell) order of red_row.  One thread per (row of Z, column).
__global__ void nl_proj_reduce_kernel(const int32_t* __restrict__ red_ptr, const int64_t* __restrict__ red_row,
                                      const float* __restrict__ part, int nsite, int ncol,
                                      float* __restrict__ Z) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)4 * nsite * ncol) return;
  const int64_t zr = idx / ncol;
  const int c = (int)(idx - zr * ncol);
  const int site = (int)(zr >> 2), t = (int)(zr & 3);
  float v = 0.f;
  for (int k = red_ptr[site]; k < red_ptr[site + 1]; ++k) v += part[(red_row[k] + t) * ncol + c];
  Z[zr * ncol + c] = v;
}

// ----------------------------------------------------------------- FP16x2 packing
// Two fp16 terms carry about 22 significant bits, within a factor four of
// binary32, and fp16 MMAs run at the bf16 rate: three kind::f16 MMAs per
// chunk (h1 y2 + h2 y1 + h1 y1; the dropped h2 y2 is 2^-22 relative) against
// BF16x3's six.  fp16's range is narrow, so each operand is scaled by a power
// of two first (exact): each cell matrix by 2^s_e with max |2^s_e H~_e| in
// [2^13, 2^14), each column of the block likewise from its maximum, and the
// epilogue multiplies the product back by 2^-s_e 2^-t_c.  Same layout as the
// BF16x3 copy with two terms per chunk.

// Power-of-two scale taking a maximum m into [2^13, 2^14) (1 for m = 0 or not finite).
__device__ __forceinline__ float f16_scale_of(float m) {
  if (!(m > 0.f) || !(m <= 3.0e38f)) return 1.f;
  int E;
  frexpf(m, &E);                       // m = f 2^E, f in [0.5, 1)
  return ldexpf(1.f, max(-126, min(126, 14 - E)));   // a normal binary32 power of two
}

__global__ void __launch_bounds__(256) tc_cell_scale_kernel(const double* __restrict__ Ht, int ne,
                                                            float* __restrict__ inv) {
  const int64_t e = blockIdx.x;
  const double* h = Ht + e * (int64_t)ne * ne;
  double m = 0.0;
  for (int i = threadIdx.x; i < ne * ne; i += blockDim.x) m = fmax(m, fabs(h[i]));
  __shared__ double red[256];
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) inv[e] = 1.f / f16_scale_of((float)red[0]);
}

__global__ void tc_pack_f16_kernel(const double* __restrict__ Ht, const float* __restrict__ inv,
                                   uint16_t* __restrict__ out, int64_t ncells, int ne, int mt, int nk16) {
  const int64_t per_chunk = (int64_t)mt * 2048;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= ncells * nk16 * per_chunk) return;
  const int64_t e = idx / (nk16 * per_chunk);
  int64_t rem = idx - e * nk16 * per_chunk;
  const int kc = (int)(rem / per_chunk);
  rem -= (int64_t)kc * per_chunk;
  const int t = (int)(rem / 2048);
  const int w = (int)(rem - t * 2048);
  const int r = w / BF_KC, k = w % BF_KC;
  const int row = t * 128 + r, col = kc * BF_KC + k;
  const double v = (row < ne && col < ne) ? Ht[(e * ne + row) * (int64_t)ne + col] : 0.0;
  const double x = v * (double)(1.f / inv[e]);   // exact: a power of two
  const __half h1 = __float2half_rn((float)x);
  const __half h2 = __float2half_rn((float)(x - (double)__half2float(h1)));
  uint16_t* base = out + (e * nk16 + kc) * 2 * per_chunk + (int64_t)t * 2048 + bf_elem_off(r, k);
  base[0] = __half_as_ushort(h1);
  base[per_chunk] = __half_as_ushort(h2);
}

cudaError_t tc_pack_f16_from_device(TcCellData& d, const double* dHt, cudaStream_t s,
                                    int64_t* dev_bytes) {
  const int nk16 = (d.ne + BF_KC - 1) / BF_KC;
  const size_t terms = (size_t)d.ncells * nk16 * 2 * d.mt * 2048 * sizeof(uint16_t);
  cudaError_t e = cudaMalloc(&d.f16, terms);
  if (e == cudaSuccess) e = cudaMalloc(&d.f16_inv, (size_t)d.ncells * sizeof(float));
  if (e != cudaSuccess) {
    if (d.f16) cudaFree(d.f16);
    d.f16 = nullptr;
    d.f16_inv = nullptr;
    d.f16_bytes = 0;
    return e;
  }
  d.f16_bytes = terms + (size_t)d.ncells * sizeof(float);
  if (dev_bytes) *dev_bytes += (int64_t)d.f16_bytes;
  note_launch();
  tc_cell_scale_kernel<<<(unsigned)d.ncells, 256, 0, s>>>(dHt, d.ne, d.f16_inv);
  const int64_t n = d.ncells * (int64_t)nk16 * d.mt * 2048;
  note_launch();
  tc_pack_f16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dHt, d.f16_inv, d.f16, d.ncells, d.ne,
                                                                 d.mt, nk16);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- cell kernel
// Shared memory after the stages: barriers and flags (256 B), then the
// cell's dof map (n_e <= 729 ints for p <= 8).
constexpr int kCellSmemTail = 256 + 4 * 729 + 12;   // 3184 B, a multiple of 16
static_assert(kCellSmemTail % 16 == 0, "stage buffers stay 16-byte aligned");
struct CellSmem {
  int stages;
  int a_bytes;   // per stage
  int y_bytes;   // per stage (hi + lo)
  int total;
};

// Stage sizes of the cell kernel.  64-column tiles keep two CTAs per SM
// (about 110 KB each; 113 KB, three stages, for four 128-row tiles), three
// when the cell has at most two 128-row tiles (p <= 5: 72 KB each, TMEM 3 x
// 128 columns); 128-column tiles take the SM
// alone (TMEM holds one CTA's mt x 128 accumulator columns) and use up to
// 200 KB of stages.
__host__ __device__ inline CellSmem cell_smem(int mt, int split3, int bn = CELL_BN) {
  CellSmem c;
  c.a_bytes = mt * 4096 * (split3 ? 2 : 1);
  c.y_bytes = bn * CELL_KC * 4 * 2;
  const int stage = c.a_bytes + c.y_bytes;
  // CTAs per SM that TMEM allows (accumulator columns rounded to a power of two)
  const int cols = mt * bn;
  const int alloc = cols <= 64 ? 64 : (cols <= 128 ? 128 : (cols <= 256 ? 256 : 512));
  const int per_sm = 512 / alloc >= 3 ? 3 : 512 / alloc;
  const int budget_kb = per_sm >= 3 ? 72 : (per_sm == 2 ? 113 : 200);
  int S = (budget_kb * 1024 - kCellSmemTail) / stage;
  S = S < 2 ? 2 : (S > 6 ? 6 : S);
  c.stages = S;
  c.total = S * stage + kCellSmemTail;
  return c;
}

// ----------------------------------------------------------------- owner-computes cell kernel
// One CTA per (cell, 64-column tile) over ALL cells (no colour phases).
// Warp 4 streams the split cell matrix in K-chunks of 8 with bulk async
// copies, warps 0-3 gather + split the cell block of Y, warp 5 issues the
// MMAs into TMEM (one 64-column accumulator per 128-row tile); the epilogue
// only stores the dense cell block R_e = H~_e Y_e with 16-byte stores (no
// loads), so it never stalls on memory latency.  The assembly over cells and
// the Chebyshev update follow in tc_assemble_kernel.
struct RParams {
  const float* A;
  const int32_t* dofmap;
  const float* Yin;
  float* R;
  int64_t ld_in;
  int ncol, ne, mt, nk, split3;
  // multi-system mode: grid x runs over the items of all systems
  const TcBatchSys* sys;
  int nsys, parity;
  int64_t ldr;              // row stride of R (>= ncol)
  int64_t e_off;            // first cell of this launch (grids of at most 65535 cells)
  const uint32_t* cmax;     // FP16x2: column maxima of |Yin| (binary32 bits), index c0 + c
  const float* cinv;        // FP16x2: per-cell inverse scales
  // projector chunks of the BF16x3 ring kernel (null: none)
  const uint16_t* nlA;
  const int32_t* nl_off;
  const int32_t* nl_zrow;
  const float* Z;
  int64_t ldz;
  // projection mode: per cell rows np[e] (B operand rows, output rows), block
  // at element pj_off[e] of A, output rows from pj_row[e] of R
  const int32_t* pj_np;
  const int64_t* pj_off;
  const int64_t* pj_row;
  int pj_npmax;
  int tpc;                  // multi-tile kernel: column tiles per CTA
  int r_evict;              // write R under an evict_first L2 policy (R much larger than L2)
};

template <int BN, bool MULTI>
__global__ void __launch_bounds__(CELL_THREADS, 1) tc_cell_r_kernel(RParams P) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int64_t e = P.e_off + blockIdx.y;
  int c0 = blockIdx.x * BN;
  if (MULTI) {   // item -> (system, cell, tile): binary search over the systems' first items
    const int64_t item = blockIdx.x;
    int lo = 0, hi = P.nsys - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (P.sys[mid].item0 <= item) lo = mid; else hi = mid - 1;
    }
    const TcBatchSys& sy = P.sys[lo];
    const int64_t li = item - sy.item0;
    e = li / sy.tiles;
    c0 = (int)(li % sy.tiles) * BN;
    P.A = sy.A;
    P.dofmap = sy.dofmap;
    P.Yin = sy.Y[P.parity];
    P.ld_in = sy.ldY[P.parity];
    P.R = sy.R;
    P.ncol = sy.ncol;
    P.ldr = sy.ldr;
  }
  const int ncv = min(BN, P.ncol - c0);
  const int bne = ncv <= 16 ? 16 : (ncv + 15) / 16 * 16;
  const CellSmem L = cell_smem(P.mt, P.split3, BN);
  const int S = L.stages;
  const int stage_bytes = L.a_bytes + L.y_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * stage_bytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * S + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  int32_t* dm = reinterpret_cast<int32_t*>(smem + S * stage_bytes + 256);
  const uint32_t sbase = smem_u32(smem);
  auto fa = [&](int s) { return smem_u32(bars + s); };
  auto fy = [&](int s) { return smem_u32(bars + S + s); };
  auto em = [&](int s) { return smem_u32(bars + 2 * S + s); };
  const uint32_t accb = smem_u32(bars + 3 * S);
  const int tc_need = P.mt * BN;   // accumulator columns: one BN-wide block per 128-row tile
  const uint32_t tmem_cols = tc_need <= 64 ? 64 : (tc_need <= 128 ? 128 : (tc_need <= 256 ? 256 : 512));
  const int nk = P.nk, ne = P.ne;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(fa(s), 1);
      mbar_init(fy(s), 32);
      mbar_init(em(s), 1);
    }
    mbar_init(accb, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 5) {
    tmem_alloc(smem_u32(tmem_slot), tmem_cols);
    tmem_relinquish();
  }
  for (int l = tid; l < ne; l += CELL_THREADS) dm[l] = P.dofmap[e * ne + l];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 4) {
    if (lane == 0) {
      const char* Ae = reinterpret_cast<const char*>(P.A) + e * (int64_t)nk * P.mt * 8192;
      int issued = 0;
      for (int i = 0; i < nk; ++i) {
        const int s = i % S;
        if (i >= S && !mbar_wait(em(s), ((i / S) - 1) & 1)) {
          atomicExch(&g_tc_status, 21);
          *(volatile int*)abort_flag = 1;
          break;
        }
        if (*(volatile int*)abort_flag) break;
        mbar_arrive_expect_tx(fa(s), L.a_bytes);
        bulk_g2s(sbase + s * stage_bytes, Ae + (int64_t)i * P.mt * 8192, L.a_bytes, fa(s));
        ++issued;
      }
      if (*(volatile int*)abort_flag)
        for (int i = max(0, issued - S); i < issued; ++i) mbar_wait(fa(i % S), (i / S) & 1);
    }
  } else if (warp == 5) {
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(128, bne);
      for (int i = 0; i < nk; ++i) {
        const int s = i % S;
        if (!mbar_wait(fa(s), (i / S) & 1) || !mbar_wait(fy(s), (i / S) & 1) ||
            *(volatile int*)abort_flag) {
          atomicExch(&g_tc_status, 22);
          *(volatile int*)abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t sa = sbase + s * stage_bytes;
        const uint32_t sy = sa + L.a_bytes;
        const uint64_t yhi = umma_desc(sy, 128, 256);
        const uint64_t ylo = umma_desc(sy + BN * CELL_KC * 4, 128, 256);
        for (int t = 0; t < P.mt; ++t) {
          const uint32_t d = tmem + t * BN;
          const uint64_t ahi = umma_desc(sa + t * 4096, 128, 256);
          if (P.split3) {
            const uint64_t alo = umma_desc(sa + P.mt * 4096 + t * 4096, 128, 256);
            mma_tf32(d, alo, yhi, idesc, i > 0);
            mma_tf32(d, ahi, ylo, idesc, 1);
            mma_tf32(d, ahi, yhi, idesc, 1);
          } else {
            mma_tf32(d, ahi, yhi, idesc, i > 0);
          }
        }
        umma_commit(em(s));
      }
      umma_commit(accb);
    }
  } else {
    // gather + split (warp w: chunks w, w + G, ...; G = min(4, S) keeps parity waits sound)
    const bool vec = ((P.ld_in & 3) == 0) && ((reinterpret_cast<uintptr_t>(P.Yin) & 15) == 0);
    constexpr int CPT = BN / 16;   // columns per thread (16 threads span the tile)
    const int q = lane >> 4;
    const int cq = (lane & 15) * CPT;
    const int G = S < 4 ? S : 4;
    // rows l = 8 i + 4 q + a of the cell block, CPT columns per lane, zero-filled
    auto load_chunk = [&](int i, float (&v)[4][CPT]) {
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int l = i * CELL_KC + q * 4 + a;
        const int g = l < ne ? dm[l] : -1;
#pragma unroll
        for (int u = 0; u < CPT; ++u) v[a][u] = 0.f;
        if (g >= 0) {
          const float* src = P.Yin + (int64_t)g * P.ld_in + c0 + cq;
#pragma unroll
          for (int u4 = 0; u4 < CPT; u4 += 4) {
            if (vec && cq + u4 + 4 <= ncv) {
              const float4 t4 = __ldg(reinterpret_cast<const float4*>(src + u4));
              v[a][u4] = t4.x; v[a][u4 + 1] = t4.y; v[a][u4 + 2] = t4.z; v[a][u4 + 3] = t4.w;
            } else {
#pragma unroll
              for (int u = u4; u < u4 + 4; ++u)
                if (cq + u < ncv) v[a][u] = __ldg(src + u);
            }
          }
        }
      }
    };
    if (warp < G) {
      // (a second chunk prefetched into registers measured no faster: the two
      // co-resident CTAs per SM already overlap the gathers)
      float v[4][CPT];
      for (int i = warp; i < nk; i += G) {
        const int s = i % S;
        load_chunk(i, v);
        if (i >= S && !mbar_wait(em(s), ((i / S) - 1) & 1)) {
          atomicExch(&g_tc_status, 23);
          *(volatile int*)abort_flag = 1;
        }
        if (*(volatile int*)abort_flag) break;
        float* yh = reinterpret_cast<float*>(smem + s * stage_bytes + L.a_bytes);
        float* yl = yh + BN * CELL_KC;
#pragma unroll
        for (int u = 0; u < CPT; ++u) {
          const int n = cq + u;
          const int o = (n >> 3) * 64 + q * 32 + (n & 7) * 4;
          float4 h, lo;
          h.x = tf32_rna(v[0][u]); lo.x = v[0][u] - h.x;
          h.y = tf32_rna(v[1][u]); lo.y = v[1][u] - h.y;
          h.z = tf32_rna(v[2][u]); lo.z = v[2][u] - h.z;
          h.w = tf32_rna(v[3][u]); lo.w = v[3][u] - h.w;
          *reinterpret_cast<float4*>(yh + o) = h;
          *reinterpret_cast<float4*>(yl + o) = lo;
        }
        fence_proxy_async_smem();
        mbar_arrive(fy(s));
      }
    }
    // epilogue: TMEM row -> R row (16-byte stores only)
    const bool okacc = mbar_wait(accb, 0);
    if (!okacc) {
      atomicExch(&g_tc_status, 24);
      *(volatile int*)abort_flag = 1;
    }
    tc_fence_after();
    const bool run = __all_sync(0xffffffffu, okacc && !*(volatile int*)abort_flag);
    const bool vst = (P.ldr & 3) == 0;
    for (int t = 0; t < P.mt; ++t) {
      const int l = t * 128 + warp * 32 + lane;
      float* dst = P.R + ((int64_t)e * ne + l) * P.ldr + c0;
      for (int cb = 0; cb < bne; cb += 16) {
        float acc[16];
        __syncwarp();
        if (run) {
          tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + t * BN + cb, acc);
          tmem_wait_ld();
        }
        if (!run || l >= ne) continue;
        if (vst && cb + 16 <= ncv) {
#pragma unroll
          for (int u = 0; u < 16; u += 4)
            *reinterpret_cast<float4*>(dst + cb + u) = make_float4(acc[u], acc[u + 1], acc[u + 2], acc[u + 3]);
        } else {
#pragma unroll
          for (int u = 0; u < 16; ++u)
            if (cb + u < ncv) dst[cb + u] = acc[u];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 5) tmem_dealloc(tmem, tmem_cols);
}

cudaError_t tc_cell_r_launch(const TcCellData& d, const TcApplyArgs& a, cudaStream_t s) {
  if (a.ncells == 0 || a.ncol == 0) return cudaSuccess;
  if (!d.hi) return cudaErrorInvalidValue;
  // (128-column tiles with the 128-row tiles split over two CTAs per SM
  // measured slower than both variants here: the two halves gather Y twice)
  const int bn = a.tile == 128 ? 128 : 64;
  RParams P{d.hi, a.dofmap, a.Yin, a.R, a.ld_in, a.ncol, d.ne, d.mt, d.kt / CELL_KC, a.split3,
            nullptr, 0, 0, a.ncol, 0};
  tc_cell_prepare();
  const CellSmem L = cell_smem(d.mt, a.split3, bn);
  for (int64_t e0 = 0; e0 < a.ncells; e0 += 65535) {   // grid y is limited to 65535
    P.e_off = e0;
    dim3 grid((unsigned)((a.ncol + bn - 1) / bn),
              (unsigned)std::min<int64_t>(65535, a.ncells - e0));
    note_launch();
    if (bn == 128)
      tc_cell_r_kernel<128, false><<<grid, CELL_THREADS, L.total, s>>>(P);
    else
      tc_cell_r_kernel<64, false><<<grid, CELL_THREADS, L.total, s>>>(P);
  }
  return cudaGetLastError();
}

void tc_cell_prepare() {
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(tc_cell_r_kernel<64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(tc_cell_r_kernel<128, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
    cudaFuncSetAttribute(tc_cell_r_kernel<64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
}

cudaError_t tc_cell_multi_launch(const TcBatchSys* d_sys, int nsys, int64_t nitems, int ne, int mt,
                                 int nk, int split3, int parity, cudaStream_t s) {
  if (nitems == 0 || nsys == 0) return cudaSuccess;
  if (nitems > 0x7fffffff) return cudaErrorInvalidValue;
  RParams P{nullptr, nullptr, nullptr, nullptr, 0, 0, ne, mt, nk, split3, d_sys, nsys, parity, 0, 0};
  tc_cell_prepare();
  const CellSmem L = cell_smem(mt, split3, 64);
  note_launch();
  tc_cell_r_kernel<64, true><<<(unsigned)nitems, CELL_THREADS, L.total, s>>>(P);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- BF16x3 cell kernel
// R_e = H~_e Y_e computed as its transpose R_e^T = Y_e^T H~_e (H~_e is
// symmetric): the MMA's M = 128 columns of Y (A operand, gathered and split
// into three bf16 terms by warps 0-3), N = up to 256 rows of H~_e (B operand,
// streamed by bulk copies from the packed three-term matrix), K = 16 cell
// nodes per chunk, six kind::f16 MMAs per chunk (h3 y1 + h2 y2 + h1 y3 +
// h2 y1 + h1 y2 + h1 y1, smallest first) accumulated in FP32 in TMEM.
// Against 128-row x 64-column tiles this halves the shared-memory operand
// bytes per flop (the tensor core's shared-memory reads bounded that form)
// and pads the n_e rows only to a multiple of 16 per part.  A cell's rows are
// split into np parts of nh rows (one CTA each, nh <= 256 so that two CTAs
// share an SM's TMEM); grid x runs over (column tile, part) with the parts
// of a tile adjacent, grid y over cells.  Warp 4 issues the copies, warp 5
// the MMAs; warps 0-3 (two pairs, one chunk per pair, 8 rows per warp)
// gather, then store R with lanes over consecutive columns.
constexpr int BF_YT = 3 * 128 * BF_KC * 2;   // Y tile: three terms of 128 columns x 16
struct BfPlan {
  int np, nh, alloc, stages, total;
};
__host__ __device__ inline BfPlan bf_plan(int ne) {
  BfPlan b;
  b.np = (ne + 255) / 256;
  const int nh = (ne + b.np - 1) / b.np;
  b.nh = (nh + 15) / 16 * 16;
  b.alloc = b.nh <= 32 ? 32 : (b.nh <= 64 ? 64 : (b.nh <= 128 ? 128 : 256));
  const int per_sm = 512 / b.alloc >= 3 ? 3 : 512 / b.alloc;
  const int budget = (per_sm >= 3 ? 72 : (per_sm == 2 ? 113 : 200)) * 1024;
  const int stage = BF_YT + 3 * b.nh * 32;
  int S = (budget - kCellSmemTail) / stage;
  S = S < 2 ? 2 : (S > 6 ? 6 : S);
  b.stages = S;
  b.total = S * stage + kCellSmemTail;
  return b;
}

__global__ void __launch_bounds__(CELL_THREADS, 2) tc_cell_bf16_kernel(RParams P) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t e = P.e_off + blockIdx.y;
  const int ne = P.ne, nk = P.nk;   // nk: K-chunks of 16
  const BfPlan B = bf_plan(ne);
  const int h = blockIdx.x % B.np;
  const int c0 = (blockIdx.x / B.np) * 128;
  const int ncv = min(128, P.ncol - c0);
  const int r0 = h * B.nh;                 // first cell row of this part
  const int S = B.stages;
  const int hrow = B.nh * 32;              // one term of the part's rows for one chunk
  const int stage_bytes = BF_YT + 3 * hrow;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * stage_bytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * S + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  int32_t* dm = reinterpret_cast<int32_t*>(smem + S * stage_bytes + 256);
  const uint32_t sbase = smem_u32(smem);
  auto fa = [&](int s) { return smem_u32(bars + s); };
  auto fy = [&](int s) { return smem_u32(bars + S + s); };
  auto em = [&](int s) { return smem_u32(bars + 2 * S + s); };
  const uint32_t accb = smem_u32(bars + 3 * S);

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(fa(s), 1);
      mbar_init(fy(s), 64);
      mbar_init(em(s), 1);
    }
    mbar_init(accb, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 5) {
    tmem_alloc(smem_u32(tmem_slot), B.alloc);
    tmem_relinquish();
  }
  for (int l = tid; l < ne; l += CELL_THREADS) dm[l] = P.dofmap[e * ne + l];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 4) {
    if (lane == 0) {
      // term p of chunk i: rows [r0, r0 + nh) are contiguous (8-row groups of 256 B)
      const int64_t term_bytes = (int64_t)P.mt * 4096;
      const char* Ae = reinterpret_cast<const char*>(P.A) + e * (int64_t)nk * 3 * term_bytes + (int64_t)r0 * 32;
      int issued = 0;
      for (int i = 0; i < nk; ++i) {
        const int s = i % S;
        if (i >= S && !mbar_wait(em(s), ((i / S) - 1) & 1)) {
          atomicExch(&g_tc_status, 31);
          *(volatile int*)abort_flag = 1;
          break;
        }
        if (*(volatile int*)abort_flag) break;
        const uint32_t dst = sbase + s * stage_bytes + BF_YT;
        mbar_arrive_expect_tx(fa(s), 3 * hrow);
#pragma unroll
        for (int p = 0; p < 3; ++p)
          bulk_g2s(dst + p * hrow, Ae + ((int64_t)i * 3 + p) * term_bytes, hrow, fa(s));
        ++issued;
      }
      if (*(volatile int*)abort_flag)
        for (int i = max(0, issued - S); i < issued; ++i) mbar_wait(fa(i % S), (i / S) & 1);
    }
  } else if (warp == 5) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, B.nh);
      for (int i = 0; i < nk; ++i) {
        const int s = i % S;
        if (!mbar_wait(fa(s), (i / S) & 1) || !mbar_wait(fy(s), (i / S) & 1) ||
            *(volatile int*)abort_flag) {
          atomicExch(&g_tc_status, 32);
          *(volatile int*)abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t sy = sbase + s * stage_bytes;
        const uint32_t sh = sy + BF_YT;
        uint64_t y[3], hd[3];
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          y[p] = umma_desc(sy + p * 4096, 128, 256);
          hd[p] = umma_desc(sh + p * hrow, 128, 256);
        }
        mma_f16(tmem, y[0], hd[2], idesc, i > 0);
        mma_f16(tmem, y[1], hd[1], idesc, 1);
        mma_f16(tmem, y[2], hd[0], idesc, 1);
        mma_f16(tmem, y[0], hd[1], idesc, 1);
        mma_f16(tmem, y[1], hd[0], idesc, 1);
        mma_f16(tmem, y[0], hd[0], idesc, 1);
        umma_commit(em(s));
      }
      umma_commit(accb);
    }
  } else {
    // gather + split: pair (warp >> 1) takes chunks pair, pair + 2, ...; warp
    // half q takes rows 16 i + 8 q + a (a < 8); lane holds columns lane + 32 u,
    // so each load reads 128 contiguous bytes of a Y row and each 16-byte
    // store of 8 lanes fills one 128-byte core matrix (no bank conflicts)
    const int pair = warp >> 1, q = warp & 1;
    const bool withhold = g_tc_withhold != 0 && blockIdx.x == 0 && blockIdx.y == 0 && P.e_off == 0;
    for (int i = pair; i < nk; i += 2) {
      const int s = i % S;
      float v[8][4];
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int l = i * BF_KC + q * 8 + a;
        const int g = l < ne ? dm[l] : -1;
        const float* src = P.Yin + (int64_t)(g < 0 ? 0 : g) * P.ld_in + c0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = lane + 32 * u;
          v[a][u] = (g >= 0 && c < ncv) ? __ldg(src + c) : 0.f;
        }
      }
      if (i >= S && !mbar_wait(em(s), ((i / S) - 1) & 1)) {
        atomicExch(&g_tc_status, 33);
        *(volatile int*)abort_flag = 1;
      }
      if (*(volatile int*)abort_flag) break;
      uint16_t* ys = reinterpret_cast<uint16_t*>(smem + s * stage_bytes);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int o = bf_elem_off(lane + 32 * u, q * 8);
        uint32_t w[3][4];
#pragma unroll
        for (int a = 0; a < 8; a += 2)
          bf16_split3_pair(v[a][u], v[a + 1][u], w[0][a / 2], w[1][a / 2], w[2][a / 2]);
#pragma unroll
        for (int p = 0; p < 3; ++p)
          *reinterpret_cast<uint4*>(ys + p * 128 * BF_KC + o) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
      }
      fence_proxy_async_smem();
      if (!(withhold && warp == 0 && i == 0)) mbar_arrive(fy(s));
    }
    // epilogue: TMEM lane = column c0 + c, TMEM column = cell row r0 + j;
    // for each row the warp's lanes store 32 consecutive floats
    const bool okacc = mbar_wait(accb, 0);
    if (!okacc) {
      atomicExch(&g_tc_status, 34);
      *(volatile int*)abort_flag = 1;
    }
    tc_fence_after();
    const bool run = __all_sync(0xffffffffu, okacc && !*(volatile int*)abort_flag);
    const int c = warp * 32 + lane;
    float* dst = P.R + ((int64_t)e * ne + r0) * P.ldr + c0 + c;
    for (int cb = 0; cb < B.nh; cb += 16) {
      float acc[16];
      __syncwarp();
      if (run) {
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + cb, acc);
        tmem_wait_ld();
      }
      if (!run || c >= ncv) continue;
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (r0 + cb + j < ne) dst[(int64_t)(cb + j) * P.ldr] = acc[j];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 5) tmem_dealloc(tmem, B.alloc);
}

// ----------------------------------------------------------------- BF16x3 cell kernel, async gather
// The same product, tiling and arithmetic as tc_cell_bf16_kernel (bit-identical
// results), with the gather of the cell's rows of Y done by bulk async copies
// instead of register loads: warp 6 copies the 16 rows of each K-chunk (one
// copy of ncv * 4 bytes per row) into a ring of S_y binary32 staging slots,
// up to S_y chunks ahead; warps 0-3 split a staged chunk into its three bf16
// terms in the MMA layout (pairs on alternate chunks, as before) and release
// the slot.  The register gather keeps two chunks in flight per CTA; here
// S_y chunks are, so the gather's latency hides behind the MMAs.  Needs
// 16-byte aligned rows: Y 16-byte aligned, ld_in and ncol multiples of 4.
constexpr int BFA_THREADS = 224;
constexpr int BFA_ROWB = 128 * 4;             // one staged row: 128 binary32 columns
constexpr int BFA_SLOT = BF_KC * BFA_ROWB;    // one staged K-chunk (8 KB)
struct BfaPlan {
  int np, nh, alloc, st, sy, total;
};
__host__ __device__ inline BfaPlan bfa_plan(int ne) {
  const BfPlan b = bf_plan(ne);
  BfaPlan a;
  a.np = b.np;
  a.nh = b.nh;
  a.alloc = b.alloc;
  const int per_sm = 512 / b.alloc >= 3 ? 3 : 512 / b.alloc;
  const int budget = (per_sm >= 3 ? 72 : (per_sm == 2 ? 110 : 200)) * 1024 - kCellSmemTail;
  const int stage = BF_YT + 3 * b.nh * 32;
  a.st = 2;
  a.sy = (budget - a.st * stage) / BFA_SLOT;
  if (a.sy > 8) a.sy = 8;
  if (a.sy >= 6 && budget - 3 * stage >= 3 * BFA_SLOT) {   // room for a third term stage
    a.st = 3;
    a.sy = (budget - a.st * stage) / BFA_SLOT;
    if (a.sy > 8) a.sy = 8;
  }
  if (a.sy < 2) a.sy = 2;
  a.total = a.st * stage + a.sy * BFA_SLOT + kCellSmemTail;
  return a;
}

__global__ void __launch_bounds__(BFA_THREADS, 2) tc_cell_bf16_async_kernel(RParams P) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t e = P.e_off + blockIdx.y;
  const int ne = P.ne, nk = P.nk;   // nk: K-chunks of 16
  const BfaPlan B = bfa_plan(ne);
  const int h = blockIdx.x % B.np;
  const int c0 = (blockIdx.x / B.np) * 128;
  const int ncv = min(128, P.ncol - c0);
  const int r0 = h * B.nh;
  const int ST = B.st, SY = B.sy;
  const int hrow = B.nh * 32;
  const int stage_bytes = BF_YT + 3 * hrow;
  unsigned char* stg = smem + ST * stage_bytes;             // staging ring
  uint64_t* bars = reinterpret_cast<uint64_t*>(stg + SY * BFA_SLOT);
  // barriers: fa[ST], fy[ST], em[ST], sf[SY], se[SY], acc  (<= 3*3 + 2*8 + 1 = 26 x 8 B)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * ST + 2 * SY + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  int32_t* dm = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(bars) + 256);
  const uint32_t sbase = smem_u32(smem);
  const uint32_t gbase = smem_u32(stg);
  auto fa = [&](int s) { return smem_u32(bars + s); };
  auto fy = [&](int s) { return smem_u32(bars + ST + s); };
  auto em = [&](int s) { return smem_u32(bars + 2 * ST + s); };
  auto sf = [&](int s) { return smem_u32(bars + 3 * ST + s); };
  auto se = [&](int s) { return smem_u32(bars + 3 * ST + SY + s); };
  const uint32_t accb = smem_u32(bars + 3 * ST + 2 * SY);

  if (tid == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(fa(s), 1);
      mbar_init(fy(s), 64);
      mbar_init(em(s), 1);
    }
    for (int s = 0; s < SY; ++s) {
      mbar_init(sf(s), 1);
      mbar_init(se(s), 2);
    }
    mbar_init(accb, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 5) {
    tmem_alloc(smem_u32(tmem_slot), B.alloc);
    tmem_relinquish();
  }
  for (int l = tid; l < ne; l += BFA_THREADS) dm[l] = P.dofmap[e * ne + l];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 6) {
    // ---------------- producer of the staged rows of Y (bulk async copies)
    const uint32_t rowb = (uint32_t)ncv * 4;
    int issued = 0;
    for (int i = 0; i < nk; ++i) {
      const int s = i % SY;
      bool ok = true;
      if (lane == 0 && i >= SY) ok = mbar_wait(se(s), ((i / SY) - 1) & 1);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok && lane == 0) {
        atomicExch(&g_tc_status, 35);
        *(volatile int*)abort_flag = 1;
      }
      if (__shfl_sync(0xffffffffu, *(volatile int*)abort_flag, 0)) break;
      const int l = i * BF_KC + lane;
      const int g = (lane < BF_KC && l < ne) ? dm[l] : -1;
      const unsigned vmask = __ballot_sync(0xffffffffu, g >= 0);
      if (lane == 0) mbar_arrive_expect_tx(sf(s), (uint32_t)__popc(vmask) * rowb);
      __syncwarp();
      if (g >= 0)
        bulk_g2s(gbase + s * BFA_SLOT + lane * BFA_ROWB, P.Yin + (int64_t)g * P.ld_in + c0, rowb, sf(s));
      ++issued;
    }
    if (lane == 0 && *(volatile int*)abort_flag)   // let the copies in flight land before exit
      for (int i = max(0, issued - SY); i < issued; ++i) mbar_wait(sf(i % SY), (i / SY) & 1);
  } else if (warp == 4) {
    // ---------------- producer of the cell-matrix chunks (as tc_cell_bf16_kernel)
    if (lane == 0) {
      const int64_t term_bytes = (int64_t)P.mt * 4096;
      const char* Ae = reinterpret_cast<const char*>(P.A) + e * (int64_t)nk * 3 * term_bytes + (int64_t)r0 * 32;
      int issued = 0;
      for (int i = 0; i < nk; ++i) {
        const int s = i % ST;
        if (i >= ST && !mbar_wait(em(s), ((i / ST) - 1) & 1)) {
          atomicExch(&g_tc_status, 31);
          *(volatile int*)abort_flag = 1;
          break;
        }
        if (*(volatile int*)abort_flag) break;
        const uint32_t dst = sbase + s * stage_bytes + BF_YT;
        mbar_arrive_expect_tx(fa(s), 3 * hrow);
#pragma unroll
        for (int p = 0; p < 3; ++p)
          bulk_g2s(dst + p * hrow, Ae + ((int64_t)i * 3 + p) * term_bytes, hrow, fa(s));
        ++issued;
      }
      if (*(volatile int*)abort_flag)
        for (int i = max(0, issued - ST); i < issued; ++i) mbar_wait(fa(i % ST), (i / ST) & 1);
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer (as tc_cell_bf16_kernel)
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, B.nh);
      for (int i = 0; i < nk; ++i) {
        const int s = i % ST;
        if (!mbar_wait(fa(s), (i / ST) & 1) || !mbar_wait(fy(s), (i / ST) & 1) ||
            *(volatile int*)abort_flag) {
          atomicExch(&g_tc_status, 32);
          *(volatile int*)abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t sy = sbase + s * stage_bytes;
        const uint32_t sh = sy + BF_YT;
        uint64_t y[3], hd[3];
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          y[p] = umma_desc(sy + p * 4096, 128, 256);
          hd[p] = umma_desc(sh + p * hrow, 128, 256);
        }
        mma_f16(tmem, y[0], hd[2], idesc, i > 0);
        mma_f16(tmem, y[1], hd[1], idesc, 1);
        mma_f16(tmem, y[2], hd[0], idesc, 1);
        mma_f16(tmem, y[0], hd[1], idesc, 1);
        mma_f16(tmem, y[1], hd[0], idesc, 1);
        mma_f16(tmem, y[0], hd[0], idesc, 1);
        umma_commit(em(s));
      }
      umma_commit(accb);
    }
  } else {
    // ---------------- warps 0-3: split staged chunks into the three bf16 terms.
    // Pair (warp >> 1) takes chunks pair, pair + 2, ...; warp half q takes rows
    // 16 i + 8 q + a (a < 8), lane the columns lane + 32 u (u < 4), exactly as
    // the register gather, so the terms are the same bits.
    const int pair = warp >> 1, q = warp & 1;
    for (int i = pair; i < nk; i += 2) {
      const int s = i % ST, sl = i % SY;
      bool ok = mbar_wait(sf(sl), (i / SY) & 1);
      if (ok && i >= ST) ok = mbar_wait(em(s), ((i / ST) - 1) & 1);
      if (!ok) {
        atomicExch(&g_tc_status, 33);
        *(volatile int*)abort_flag = 1;
      }
      if (*(volatile int*)abort_flag) break;
      const float* rows = reinterpret_cast<const float*>(stg + sl * BFA_SLOT);
      float v[8][4];
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int r = q * 8 + a;
        const int l = i * BF_KC + r;
        const int g = l < ne ? dm[l] : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = lane + 32 * u;
          v[a][u] = (g >= 0 && c < ncv) ? rows[r * 128 + c] : 0.f;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(se(sl));      // the staged rows are in registers: free the slot
      uint16_t* ys = reinterpret_cast<uint16_t*>(smem + s * stage_bytes);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int o = bf_elem_off(lane + 32 * u, q * 8);
        uint32_t w[3][4];
#pragma unroll
        for (int a = 0; a < 8; a += 2) {
          uint16_t lo1, lo2, lo3, hi1, hi2, hi3;
          bf16_split3f(v[a][u], lo1, lo2, lo3);
          bf16_split3f(v[a + 1][u], hi1, hi2, hi3);
          w[0][a / 2] = (uint32_t)lo1 | ((uint32_t)hi1 << 16);
          w[1][a / 2] = (uint32_t)lo2 | ((uint32_t)hi2 << 16);
          w[2][a / 2] = (uint32_t)lo3 | ((uint32_t)hi3 << 16);
        }
#pragma unroll
        for (int p = 0; p < 3; ++p)
          *reinterpret_cast<uint4*>(ys + p * 128 * BF_KC + o) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
      }
      fence_proxy_async_smem();
      mbar_arrive(fy(s));
    }
    // epilogue (as tc_cell_bf16_kernel)
    const bool okacc = mbar_wait(accb, 0);
    if (!okacc) {
      atomicExch(&g_tc_status, 34);
      *(volatile int*)abort_flag = 1;
    }
    tc_fence_after();
    const bool run = __all_sync(0xffffffffu, okacc && !*(volatile int*)abort_flag);
    const int c = warp * 32 + lane;
    float* dst = P.R + ((int64_t)e * ne + r0) * P.ldr + c0 + c;
    for (int cb = 0; cb < B.nh; cb += 16) {
      float acc[16];
      __syncwarp();
      if (run) {
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + cb, acc);
        tmem_wait_ld();
      }
      if (!run || c >= ncv) continue;
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (r0 + cb + j < ne) dst[(int64_t)(cb + j) * P.ldr] = acc[j];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 5) tmem_dealloc(tmem, B.alloc);
}

bool tc_cell_bf16_async_ok(const TcApplyArgs& a) {
  return ((reinterpret_cast<uintptr_t>(a.Yin) & 15) == 0) && (a.ld_in % 4 == 0) && (a.ncol % 4 == 0);
}

// ----------------------------------------------------------------- BF16x3 cell kernel, decoupled rings
// The same product, tiling, gather and arithmetic as tc_cell_bf16_kernel
// (bit-identical results), with the cell-matrix chunks and the split Y chunks
// in two separate rings: SM matrix stages (one bulk-copied chunk of the
// part's rows each) and SY Y stages (three bf16 terms of 128 columns).  A
// chunk's matrix terms come from DRAM at about a microsecond of latency while
// its six MMAs take a quarter of that, so the matrix copies run SM chunks
// ahead of the products; the Y terms, gathered two chunks at a time by the
// warp pairs with a register prefetch, need only two stages.  The MMA warp
// releases both slots of a chunk with one commit each.
struct BfrPlan {
  int np, nh, alloc, sm, sy, total;
};
// npair gather warp pairs; each pair owns the Y stages i % npair of its
// chunks i = pair (mod npair), so its parity waits stay sound.  nt: terms per
// operand (3 for BF16x3, 2 for FP16x2).
__host__ __device__ inline BfrPlan bfr_plan(int ne, int npair, int nt = 3, int proj_nh = 0,
                                            bool one_cta = false) {
  BfPlan b = bf_plan(ne);
  if (proj_nh > 0) {   // projection blocks: one part of up to proj_nh rows
    b.np = 1;
    b.nh = proj_nh;
    b.alloc = proj_nh <= 32 ? 32 : (proj_nh <= 64 ? 64 : (proj_nh <= 128 ? 128 : 256));
  }
  BfrPlan r;
  r.np = b.np;
  r.nh = b.nh;
  r.alloc = b.alloc;
  const int per_sm = one_cta ? 1 : (512 / b.alloc >= 3 ? 3 : 512 / b.alloc);
  const int budget = (per_sm >= 3 ? 72 : (per_sm == 2 ? 111 : 200)) * 1024 - kCellSmemTail;
  const int mstage = nt * b.nh * 32, ystage = nt * 128 * BF_KC * 2;
  r.sy = npair;
  r.sm = (budget - r.sy * ystage) / mstage;
  if (r.sm > 8) r.sm = 8;
  if (r.sm < 2) r.sm = 2;
  r.total = r.sm * mstage + r.sy * ystage + kCellSmemTail;
  return r;
}

// MULTI: grid x runs over the (system, cell, column tile, row part) items of
// a batch (TcBatchSys: A = the system's packed BF16x3 copy, tiles = column
// tiles x parts, items of system s from item0), all systems of one degree.
// NT = 2: the FP16x2 form (P.A the fp16 terms, P.cinv the per-cell inverse
// scales, P.cmax the column maxima of Yin): three MMAs per chunk.
// NLC: the projector chunks are compiled in (a separate instantiation, so the
// kernel without projectors keeps its lean gather loop).  PROJ: the
// projection Z = C~^T Y instead of the cell products: the streamed operand is
// the cell's projection block (np[e] rows = its projectors, K = its nodes),
// the result (128 columns x np[e]) goes to rows pj_row[e] .. of R.
// KPT: the Bloch term of H~(k): the K loop continues over a second pass of
// the cell's nodes against one shared block (P.nlA: G~ = M^{-1/2} (k.G_e)
// M^{-1/2}, the same for every cell of the uniform periodic mesh), the rows
// of Y gathered with each (real, imaginary) column pair swapped and the new
// imaginary part negated, so R holds T~_e Y_r + G~ Y_i, T~_e Y_i - G~ Y_r.
template <int NPAIR, bool MULTI, int NT = 3, bool NLC = false, bool PROJ = false, bool KPT = false>
__global__ void __launch_bounds__((2 * NPAIR + 2) * 32, 2) tc_cell_bf16_rings_kernel(RParams P) {
  static_assert(NT == 3 || (NT == 2 && !MULTI), "BF16x3, or single-system FP16x2");
  static_assert(!NLC || (NT == 3 && !MULTI), "projector chunks: single-system BF16x3");
  static_assert(!PROJ || (NT == 3 && !MULTI && !NLC), "projection: single-system BF16x3");
  static_assert(!KPT || (NT == 3 && !MULTI && !NLC && !PROJ), "Bloch term: single-system BF16x3");
  constexpr int NTHR = (2 * NPAIR + 2) * 32;
  constexpr int WPROD = 2 * NPAIR, WMMA = 2 * NPAIR + 1;
  constexpr int YT = NT * 128 * BF_KC * 2;   // Y stage bytes
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int64_t e = P.e_off + blockIdx.y;
  const int ne = P.ne, nk = P.nk;
  const BfrPlan B = bfr_plan(ne, NPAIR, NT, PROJ ? P.pj_npmax : 0);
  const int nrow = PROJ ? P.pj_np[e] : B.nh;   // B-operand rows of this CTA
  if (PROJ && nrow == 0) return;                // a cell owning no projector rows: nothing to do
  int h = blockIdx.x % B.np;
  int c0 = (blockIdx.x / B.np) * 128;
  if (MULTI) {   // item -> (system, cell, tile, part): binary search over the systems' first items
    const int64_t item = blockIdx.x;
    int lo = 0, hi = P.nsys - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (P.sys[mid].item0 <= item) lo = mid; else hi = mid - 1;
    }
    const TcBatchSys& sy = P.sys[lo];
    const int64_t li = item - sy.item0;
    e = li / sy.tiles;
    const int t = (int)(li % sy.tiles);
    h = t % B.np;
    c0 = (t / B.np) * 128;
    P.A = sy.A;
    P.dofmap = sy.dofmap;
    P.Yin = sy.Y[P.parity];
    P.ld_in = sy.ldY[P.parity];
    P.R = sy.R;
    P.ncol = sy.ncol;
    P.ldr = sy.ldr;
  }
  const int ncv = min(128, P.ncol - c0);
  const int r0 = h * B.nh;
  const int SM = B.sm, SY = B.sy;
  const int hrow = nrow * 32;              // bytes of one term of a chunk (rows of 32 B)
  const int mstage = NT * B.nh * 32;       // stage stride (the launch's largest block)
  unsigned char* ybase = smem + SM * mstage;                   // Y term stages
  uint64_t* bars = reinterpret_cast<uint64_t*>(ybase + SY * YT);
  // fa[SM] (matrix full, tx), ea[SM] (matrix empty), fy[SY] (Y full, 64), ey[SY] (Y empty), acc
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * SM + 2 * SY + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  int32_t* dm = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(bars) + 256);
  const uint32_t mbase = smem_u32(smem);
  const uint32_t ysb = smem_u32(ybase);
  auto fa = [&](int s) { return smem_u32(bars + s); };
  auto ea = [&](int s) { return smem_u32(bars + SM + s); };
  auto fy = [&](int s) { return smem_u32(bars + 2 * SM + s); };
  auto ey = [&](int s) { return smem_u32(bars + 2 * SM + SY + s); };
  const uint32_t accb = smem_u32(bars + 2 * SM + 2 * SY);

  if (tid == 0) {
    for (int s = 0; s < SM; ++s) {
      mbar_init(fa(s), 1);
      mbar_init(ea(s), 1);
    }
    for (int s = 0; s < SY; ++s) {
      mbar_init(fy(s), 64);
      mbar_init(ey(s), 1);
    }
    mbar_init(accb, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == WMMA) {
    tmem_alloc(smem_u32(tmem_slot), B.alloc);
    tmem_relinquish();
  }
  for (int l = tid; l < ne; l += NTHR) dm[l] = P.dofmap[e * ne + l];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // projector chunks (BF16x3, single system): K continues over the cell's
  // 4 ns_e projectors with the rows of Z as the gathered operand
  const int nl0 = NLC ? P.nl_off[e] : 0;
  const int nkt = NLC ? nk + P.nl_off[e + 1] - nl0 : (KPT ? 2 * nk : nk);

  if (warp == WPROD) {
    if (lane == 0) {
      const int64_t term_bytes = (int64_t)P.mt * 4096;
      const char* Ae = PROJ ? reinterpret_cast<const char*>(P.A) + P.pj_off[e] * 2
                            : reinterpret_cast<const char*>(P.A) + e * (int64_t)nk * NT * term_bytes + (int64_t)r0 * 32;
      const int64_t tstride = PROJ ? (int64_t)hrow : term_bytes;   // bytes between terms and chunks
      const char* An = NLC || KPT ? reinterpret_cast<const char*>(P.nlA) + ((int64_t)nl0 - nk) * NT * term_bytes +
                                        (int64_t)r0 * 32
                                  : Ae;   // chunk i >= nk of the projector / Bloch block
      int issued = 0;
      for (int i = 0; i < nkt; ++i) {
        const int s = i % SM;
        if (i >= SM && !mbar_wait(ea(s), ((i / SM) - 1) & 1)) {
          atomicExch(&g_tc_status, 41);
          *(volatile int*)abort_flag = 1;
          break;
        }
        if (*(volatile int*)abort_flag) break;
        const uint32_t dst = mbase + s * mstage;
        mbar_arrive_expect_tx(fa(s), NT * hrow);
        const char* src = !(NLC || KPT) || i < nk ? Ae : An;
#pragma unroll
        for (int p = 0; p < NT; ++p)
          bulk_g2s(dst + p * hrow, src + ((int64_t)i * NT + p) * tstride, hrow, fa(s));
        ++issued;
      }
      if (*(volatile int*)abort_flag)
        for (int i = max(0, issued - SM); i < issued; ++i) mbar_wait(fa(i % SM), (i / SM) & 1);
    }
  } else if (warp == WMMA) {
    if (lane == 0) {
      const uint32_t idesc = NT == 3 ? idesc_bf16(128, nrow) : idesc_f16(128, nrow);
      for (int i = 0; i < nkt; ++i) {
        const int sa = i % SM, sy = i % SY;
        if (!mbar_wait(fa(sa), (i / SM) & 1) || !mbar_wait(fy(sy), (i / SY) & 1) ||
            *(volatile int*)abort_flag) {
          atomicExch(&g_tc_status, 42);
          *(volatile int*)abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t yb = ysb + sy * YT;
        const uint32_t hb = mbase + sa * mstage;
        uint64_t y[NT], hd[NT];
#pragma unroll
        for (int p = 0; p < NT; ++p) {
          y[p] = umma_desc(yb + p * 4096, 128, 256);
          hd[p] = umma_desc(hb + p * hrow, 128, 256);
        }
        if (NT == 3) {
          mma_f16(tmem, y[0], hd[NT - 1], idesc, i > 0);
          mma_f16(tmem, y[1], hd[1], idesc, 1);
          mma_f16(tmem, y[NT - 1], hd[0], idesc, 1);
          mma_f16(tmem, y[0], hd[1], idesc, 1);
          mma_f16(tmem, y[1], hd[0], idesc, 1);
          mma_f16(tmem, y[0], hd[0], idesc, 1);
        } else {
          mma_f16(tmem, y[0], hd[1], idesc, i > 0);
          mma_f16(tmem, y[1], hd[0], idesc, 1);
          mma_f16(tmem, y[0], hd[0], idesc, 1);
        }
        umma_commit(ea(sa));
        umma_commit(ey(sy));
      }
      umma_commit(accb);
    }
  } else {
    // gather + split exactly as tc_cell_bf16_kernel; Y stage of chunk i is i % SY
    const int pair = warp >> 1, q = warp & 1;
    // test hook (off by default): warp 0 of the first CTA withholds its first arrival
    const bool withhold = g_tc_withhold != 0 && blockIdx.x == 0 && blockIdx.y == 0 && P.e_off == 0;
    float tsc[4] = {1.f, 1.f, 1.f, 1.f};   // FP16x2: power-of-two scales of the lane's columns
    if (NT == 2) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = lane + 32 * u;
        if (c < ncv) tsc[u] = f16_scale_of(__uint_as_float(P.cmax[c0 + c]));
      }
    }
    for (int i = pair; i < nkt; i += NPAIR) {
      const int s = i % SY;
      float v[8][4];
      const bool zc = NLC && i >= nk;   // a projector chunk: rows of Z
      const bool sw = KPT && i >= nk;   // a Bloch chunk: the cell's rows again, columns swapped
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int l = (sw ? i - nk : i) * BF_KC + q * 8 + a;
        const int g = zc ? P.nl_zrow[(int64_t)(nl0 + i - nk) * BF_KC + q * 8 + a] : (l < ne ? dm[l] : -1);
        const float* src = zc ? P.Z + (int64_t)(g < 0 ? 0 : g) * P.ldz + c0
                              : P.Yin + (int64_t)(g < 0 ? 0 : g) * P.ld_in + c0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = lane + 32 * u;
          if (KPT && sw) {   // (re, im) -> (im, -re)
            const float y = (g >= 0 && c < ncv) ? __ldg(src + (c ^ 1)) : 0.f;
            v[a][u] = (c & 1) ? -y : y;
          } else {
            v[a][u] = (g >= 0 && c < ncv) ? __ldg(src + c) : 0.f;
          }
        }
      }
      if (i >= SY && !mbar_wait(ey(s), ((i / SY) - 1) & 1)) {
        atomicExch(&g_tc_status, 43);
        *(volatile int*)abort_flag = 1;
      }
      if (*(volatile int*)abort_flag) break;
      uint16_t* ys = reinterpret_cast<uint16_t*>(ybase + s * YT);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int o = bf_elem_off(lane + 32 * u, q * 8);
        uint32_t w[NT][4];
#pragma unroll
        for (int a = 0; a < 8; a += 2) {
          if (NT == 3)
            bf16_split3_pair(v[a][u], v[a + 1][u], w[0][a / 2], w[1][a / 2], w[NT - 1][a / 2]);
          else
            f16_split2_pair(v[a][u] * tsc[u], v[a + 1][u] * tsc[u], w[0][a / 2], w[1][a / 2]);
        }
#pragma unroll
        for (int p = 0; p < NT; ++p)
          *reinterpret_cast<uint4*>(ys + p * 128 * BF_KC + o) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
      }
      fence_proxy_async_smem();
      if (!(withhold && warp == 0 && i == 0)) mbar_arrive(fy(s));
    }
    // epilogue: warps 0-3 (TMEM lane quarter = warp % 4); further gather warps are done
    if (warp < 4) {
    const bool okacc = mbar_wait(accb, 0);
    if (!okacc) {
      atomicExch(&g_tc_status, 44);
      *(volatile int*)abort_flag = 1;
    }
    tc_fence_after();
    const bool run = __all_sync(0xffffffffu, okacc && !*(volatile int*)abort_flag);
    const int c = warp * 32 + lane;
    float* const rbase = P.R + (PROJ ? P.pj_row[e] : (int64_t)e * ne + r0) * P.ldr + c0;
    const int rend = min(nrow, PROJ ? nrow : ne - r0);   // rows of this CTA's result
    // FP16x2: undo the cell's and the column's scales (exact powers of two)
    const float back = NT == 2 && c < ncv ? P.cinv[e] / f16_scale_of(__uint_as_float(P.cmax[c0 + c])) : 1.f;
    // The result leaves through the rings, now idle (every MMA has completed):
    // the four warps write groups of up to `cap` rows into shared memory, row
    // r at [r][128 columns], and each thread then sends rows r = c (mod 128)
    // with one bulk copy of ncv columns; the warps wait only until the copies
    // have read shared memory, not for their writes to reach memory.
    // Without 16-byte rows (ld or ncv not a multiple of 4) the threads store
    // their column of each row directly.
    const int cap = (SM * mstage + SY * YT) / 512 / 16 * 16;
    if ((P.ldr & 3) == 0 && (ncv & 3) == 0 && cap >= 16) {
      float* stage = reinterpret_cast<float*>(smem);
      for (int g0 = 0; g0 < nrow; g0 += cap) {
        const int g1 = min(nrow, g0 + cap);
        for (int cb = g0; cb < g1; cb += 16) {
          float acc[16];
          __syncwarp();
          if (run) {
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + cb, acc);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (cb + j < g1) stage[(cb - g0 + j) * 128 + c] = NT == 2 ? acc[j] * back : acc[j];
          }
        }
        fence_proxy_async_smem();
        named_bar_sync(1, 128);
        if (run) {
          // R is read once, by the next launch: when it cannot stay in L2 it
          // is written as the first to be evicted, ahead of the Y rows and
          // cell matrices the other CTAs still read
          const uint64_t pol = l2_evict_first();
          for (int r = g0 + c; r < min(g1, rend); r += 128) {
            float* d = rbase + (int64_t)r * P.ldr;
            const uint32_t sa = smem_u32(stage + (r - g0) * 128);
            if (P.r_evict) bulk_s2g_hint(d, sa, (uint32_t)ncv * 4, pol);
            else bulk_s2g(d, sa, (uint32_t)ncv * 4);
          }
          bulk_commit();
          bulk_wait_read0();
        }
        named_bar_sync(1, 128);   // the staging rows are free again
      }
    } else {
      float* dst = rbase + c;
      for (int cb = 0; cb < nrow; cb += 16) {
        float acc[16];
        __syncwarp();
        if (run) {
          tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + cb, acc);
          tmem_wait_ld();
        }
        if (!run || c >= ncv) continue;
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (cb + j < rend) dst[(int64_t)(cb + j) * P.ldr] = NT == 2 ? acc[j] * back : acc[j];
      }
    }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == WMMA) tmem_dealloc(tmem, B.alloc);
}

// ----------------------------------------------------------------- BF16x3 cell kernel, several column tiles per CTA
// The product and arithmetic of the ring kernel (bit-identical results) with
// one CTA per (cell, row part, group of P.tpc consecutive 128-column tiles):
// the dof map is read once per group, both rings run on across the tiles
// (one chunk counter g = tile * nk + chunk for slots and parities), and four
// epilogue warps (6-9) drain each tile's accumulator while the gather warps
// and the matrix producer already fill the rings for the next tile.  The MMA
// warp starts a tile once the epilogue has released TMEM (tmem_empty).
// Warps: 0-3 gather (two pairs), 4 matrix producer, 5 MMA, 6-9 epilogue.
// NACC = 2: one CTA per SM with two TMEM accumulators (tile t in columns
// 256 (t % 2) ..), so the MMAs of tile t + 1 run while the epilogue drains
// tile t, deeper rings (the whole shared memory) and NPAIR gather pairs.
constexpr int kTilesPerCta = 3;
constexpr double kL2Bytes = 129.0 * 1024 * 1024;   // GB300 L2
template <int NPAIR, int NACC>
__global__ void __launch_bounds__((2 * NPAIR + 6) * 32, NACC == 1 ? 2 : 1) tc_cell_bf16_tiles_kernel(RParams P) {
  constexpr int NT = 3, WPROD = 2 * NPAIR, WMMA = 2 * NPAIR + 1, WEPI = 2 * NPAIR + 2;
  constexpr int BFT_THREADS = (2 * NPAIR + 6) * 32;
  constexpr int YT = NT * 128 * BF_KC * 2;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t e = P.e_off + blockIdx.y;
  const int ne = P.ne, nk = P.nk;
  const BfrPlan B = bfr_plan(ne, NPAIR, NT, 0, NACC == 2);
  const int nrow = B.nh;
  const int h = blockIdx.x % B.np;
  const int ntiles = (P.ncol + 127) / 128;
  const int t0 = (blockIdx.x / B.np) * P.tpc;
  const int nt = min(P.tpc, ntiles - t0);   // tiles of this CTA (>= 1)
  const int r0 = h * B.nh;
  const int SM = B.sm, SY = B.sy;
  const int hrow = nrow * 32;
  const int mstage = NT * B.nh * 32;
  unsigned char* ybase = smem + SM * mstage;
  uint64_t* bars = reinterpret_cast<uint64_t*>(ybase + SY * YT);
  // fa[SM], ea[SM], fy[SY], ey[SY], acc[NACC] (MMA -> epilogue), tmem_empty[NACC] (epilogue -> MMA)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * SM + 2 * SY + 2 * NACC);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  int32_t* dm = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(bars) + 256);
  const uint32_t mbase = smem_u32(smem);
  const uint32_t ysb = smem_u32(ybase);
  auto fa = [&](int q) { return smem_u32(bars + q); };
  auto ea = [&](int q) { return smem_u32(bars + SM + q); };
  auto fy = [&](int q) { return smem_u32(bars + 2 * SM + q); };
  auto ey = [&](int q) { return smem_u32(bars + 2 * SM + SY + q); };
  auto accb = [&](int b) { return smem_u32(bars + 2 * SM + 2 * SY + b); };
  auto tmeb = [&](int b) { return smem_u32(bars + 2 * SM + 2 * SY + NACC + b); };
  const uint32_t acols = NACC == 2 ? 512u : (uint32_t)B.alloc;

  if (tid == 0) {
    for (int q = 0; q < SM; ++q) {
      mbar_init(fa(q), 1);
      mbar_init(ea(q), 1);
    }
    for (int q = 0; q < SY; ++q) {
      mbar_init(fy(q), 64);
      mbar_init(ey(q), 1);
    }
    for (int b = 0; b < NACC; ++b) {
      mbar_init(accb(b), 1);
      mbar_init(tmeb(b), 128);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == WMMA) {
    tmem_alloc(smem_u32(tmem_slot), acols);
    tmem_relinquish();
  }
  for (int l = tid; l < ne; l += BFT_THREADS) dm[l] = P.dofmap[e * ne + l];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int G = nt * nk;   // chunks of this CTA

  if (warp == WPROD) {
    if (lane == 0) {
      const int64_t term_bytes = (int64_t)P.mt * 4096;
      const char* Ae = reinterpret_cast<const char*>(P.A) + e * (int64_t)nk * NT * term_bytes + (int64_t)r0 * 32;
      int issued = 0;
      for (int g = 0; g < G; ++g) {
        const int q = g % SM, i = g % nk;
        if (g >= SM && !mbar_wait(ea(q), ((g / SM) - 1) & 1)) {
          atomicExch(&g_tc_status, 51);
          *(volatile int*)abort_flag = 1;
          break;
        }
        if (*(volatile int*)abort_flag) break;
        const uint32_t dst = mbase + q * mstage;
        mbar_arrive_expect_tx(fa(q), NT * hrow);
#pragma unroll
        for (int p = 0; p < NT; ++p)
          bulk_g2s(dst + p * hrow, Ae + ((int64_t)i * NT + p) * term_bytes, hrow, fa(q));
        ++issued;
      }
      if (*(volatile int*)abort_flag)
        for (int g = max(0, issued - SM); g < issued; ++g) mbar_wait(fa(g % SM), (g / SM) & 1);
    }
  } else if (warp == WMMA) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, nrow);
      bool ok = true;
      for (int t = 0; t < nt && ok; ++t) {
        const int b = t % NACC;   // accumulator of tile t
        if (t >= NACC && !mbar_wait(tmeb(b), ((t / NACC) - 1) & 1)) {   // drained tile t - NACC
          atomicExch(&g_tc_status, 52);
          *(volatile int*)abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t dacc = tmem + (uint32_t)(b * 256);
        for (int i = 0; i < nk; ++i) {
          const int g = t * nk + i;
          const int sa = g % SM, sy = g % SY;
          if (!mbar_wait(fa(sa), (g / SM) & 1) || !mbar_wait(fy(sy), (g / SY) & 1) ||
              *(volatile int*)abort_flag) {
            atomicExch(&g_tc_status, 53);
            *(volatile int*)abort_flag = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t yb = ysb + sy * YT;
          const uint32_t hb = mbase + sa * mstage;
          uint64_t y[NT], hd[NT];
#pragma unroll
          for (int p = 0; p < NT; ++p) {
            y[p] = umma_desc(yb + p * 4096, 128, 256);
            hd[p] = umma_desc(hb + p * hrow, 128, 256);
          }
          mma_f16(dacc, y[0], hd[2], idesc, i > 0);
          mma_f16(dacc, y[1], hd[1], idesc, 1);
          mma_f16(dacc, y[2], hd[0], idesc, 1);
          mma_f16(dacc, y[0], hd[1], idesc, 1);
          mma_f16(dacc, y[1], hd[0], idesc, 1);
          mma_f16(dacc, y[0], hd[0], idesc, 1);
          umma_commit(ea(sa));
          umma_commit(ey(sy));
        }
        if (ok) umma_commit(accb(b));   // tile t's accumulator is complete
      }
    }
  } else if (warp < 2 * NPAIR) {
    // gather + split as the ring kernel; chunk g of this CTA is gathered by pair g % NPAIR
    const int pair = warp >> 1, qw = warp & 1;
    const bool withhold = g_tc_withhold != 0 && blockIdx.x == 0 && blockIdx.y == 0 && P.e_off == 0;
    for (int g = pair; g < G; g += NPAIR) {
      const int t = g / nk, i = g - t * nk;
      const int c0 = (t0 + t) * 128, ncv = min(128, P.ncol - c0);
      const int s = g % SY;
      float v[8][4];
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int l = i * BF_KC + qw * 8 + a;
        const int gr = l < ne ? dm[l] : -1;
        const float* src = P.Yin + (int64_t)(gr < 0 ? 0 : gr) * P.ld_in + c0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = lane + 32 * u;
          v[a][u] = (gr >= 0 && c < ncv) ? __ldg(src + c) : 0.f;
        }
      }
      if (g >= SY && !mbar_wait(ey(s), ((g / SY) - 1) & 1)) {
        atomicExch(&g_tc_status, 54);
        *(volatile int*)abort_flag = 1;
      }
      if (*(volatile int*)abort_flag) break;
      uint16_t* ys = reinterpret_cast<uint16_t*>(ybase + s * YT);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int o = bf_elem_off(lane + 32 * u, qw * 8);
        uint32_t w[NT][4];
#pragma unroll
        for (int a = 0; a < 8; a += 2) bf16_split3_pair(v[a][u], v[a + 1][u], w[0][a / 2], w[1][a / 2], w[2][a / 2]);
#pragma unroll
        for (int p = 0; p < NT; ++p)
          *reinterpret_cast<uint4*>(ys + p * 128 * BF_KC + o) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
      }
      fence_proxy_async_smem();
      if (!(withhold && warp == 0 && g == 0)) mbar_arrive(fy(s));
    }
  } else {
    // epilogue warps: TMEM lane quarter warp % 4, column c of each tile
    const int quarter = warp & 3, c = quarter * 32 + lane;
    const uint64_t pol = l2_evict_first();   // R is read once, by the next launch
    const int rend = min(nrow, ne - r0);
    for (int t = 0; t < nt; ++t) {
      const int b = t % NACC;
      const bool okacc = mbar_wait(accb(b), (t / NACC) & 1);
      if (!okacc) {
        atomicExch(&g_tc_status, 55);
        *(volatile int*)abort_flag = 1;
      }
      tc_fence_after();
      const bool run = __all_sync(0xffffffffu, okacc && !*(volatile int*)abort_flag);
      const int c0 = (t0 + t) * 128, ncv = min(128, P.ncol - c0);
      float* dst = P.R + ((int64_t)e * ne + r0) * P.ldr + c0 + c;
      for (int cb = 0; cb < nrow; cb += 16) {
        float acc[16];
        __syncwarp();
        if (run) {
          tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + b * 256 + cb, acc);
          tmem_wait_ld();
        }
        if (!run || c >= ncv) continue;
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (cb + j < rend) {
            if (P.r_evict) st_global_hint(dst + (int64_t)(cb + j) * P.ldr, acc[j], pol);
            else dst[(int64_t)(cb + j) * P.ldr] = acc[j];
          }
      }
      tc_fence_before();
      if (!run) break;
      mbar_arrive(tmeb(b));   // TMEM columns of tile t free for tile t + NACC
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == WMMA) tmem_dealloc(tmem, acols);
}

// ----------------------------------------------------------------- BF16x3 cell kernel, whole cell per CTA
// For cells split into two row parts (p = 6, 7): one CTA per (cell, 128-column
// tile) computes both parts into two TMEM accumulators (columns [0, nh) and
// [256, 256 + nh): all 512 columns, one CTA per SM), so every gathered value
// of Y is split once per cell instead of once per part.  Per K-chunk the
// producer copies the three terms of both parts' rows (contiguous in the
// packed layout) and the MMA warp issues the six products for each part.
// Four gather warp pairs own one Y stage each (chunks i = pair mod 4); the
// epilogue drains part 0 with warps 0-3 and part 1 with warps 4-7 (TMEM lane
// quarter = warp % 4).  Same per-part arithmetic as tc_cell_bf16_kernel:
// bit-identical results.
constexpr int BFW_NPAIR = 4, BFW_THREADS = (2 * BFW_NPAIR + 2) * 32;
struct BfwPlan {
  int nh, sm, sy, total;
};
__host__ __device__ inline BfwPlan bfw_plan(int ne) {
  const BfPlan b = bf_plan(ne);
  BfwPlan w;
  w.nh = b.nh;
  w.sy = BFW_NPAIR;
  const int budget = 200 * 1024 - kCellSmemTail;
  const int mstage = 3 * 2 * b.nh * 32;
  w.sm = (budget - w.sy * BF_YT) / mstage;
  if (w.sm > 6) w.sm = 6;
  if (w.sm < 2) w.sm = 2;
  w.total = w.sm * mstage + w.sy * BF_YT + kCellSmemTail;
  return w;
}
__host__ __device__ inline bool bfw_supported(int ne) {
  const BfPlan b = bf_plan(ne);
  return b.np == 2 && b.nh <= 256;
}

__global__ void __launch_bounds__(BFW_THREADS, 1) tc_cell_bf16_whole_kernel(RParams P) {
  constexpr int WPROD = 2 * BFW_NPAIR, WMMA = 2 * BFW_NPAIR + 1;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t e = P.e_off + blockIdx.y;
  const int ne = P.ne, nk = P.nk;
  const BfwPlan B = bfw_plan(ne);
  const int c0 = blockIdx.x * 128;
  const int ncv = min(128, P.ncol - c0);
  const int SM = B.sm, SY = B.sy;
  const int hrow = B.nh * 32;                 // one term of one part's rows, one chunk
  const int trow = 2 * hrow;                  // one term of both parts' rows
  const int mstage = 3 * trow;
  unsigned char* ybase = smem + SM * mstage;
  uint64_t* bars = reinterpret_cast<uint64_t*>(ybase + SY * BF_YT);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * SM + 2 * SY + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  int32_t* dm = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(bars) + 256);
  const uint32_t mbase = smem_u32(smem);
  const uint32_t ysb = smem_u32(ybase);
  auto fa = [&](int s) { return smem_u32(bars + s); };
  auto ea = [&](int s) { return smem_u32(bars + SM + s); };
  auto fy = [&](int s) { return smem_u32(bars + 2 * SM + s); };
  auto ey = [&](int s) { return smem_u32(bars + 2 * SM + SY + s); };
  const uint32_t accb = smem_u32(bars + 2 * SM + 2 * SY);

  if (tid == 0) {
    for (int s = 0; s < SM; ++s) {
      mbar_init(fa(s), 1);
      mbar_init(ea(s), 1);
    }
    for (int s = 0; s < SY; ++s) {
      mbar_init(fy(s), 64);
      mbar_init(ey(s), 1);
    }
    mbar_init(accb, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == WMMA) {
    tmem_alloc(smem_u32(tmem_slot), 512);
    tmem_relinquish();
  }
  for (int l = tid; l < ne; l += BFW_THREADS) dm[l] = P.dofmap[e * ne + l];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == WPROD) {
    if (lane == 0) {
      const int64_t term_bytes = (int64_t)P.mt * 4096;
      const char* Ae = reinterpret_cast<const char*>(P.A) + e * (int64_t)nk * 3 * term_bytes;
      int issued = 0;
      for (int i = 0; i < nk; ++i) {
        const int s = i % SM;
        if (i >= SM && !mbar_wait(ea(s), ((i / SM) - 1) & 1)) {
          atomicExch(&g_tc_status, 51);
          *(volatile int*)abort_flag = 1;
          break;
        }
        if (*(volatile int*)abort_flag) break;
        const uint32_t dst = mbase + s * mstage;
        mbar_arrive_expect_tx(fa(s), 3 * trow);
#pragma unroll
        for (int p = 0; p < 3; ++p)
          bulk_g2s(dst + p * trow, Ae + ((int64_t)i * 3 + p) * term_bytes, trow, fa(s));
        ++issued;
      }
      if (*(volatile int*)abort_flag)
        for (int i = max(0, issued - SM); i < issued; ++i) mbar_wait(fa(i % SM), (i / SM) & 1);
    }
  } else if (warp == WMMA) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, B.nh);
      for (int i = 0; i < nk; ++i) {
        const int sa = i % SM, sy = i % SY;
        if (!mbar_wait(fa(sa), (i / SM) & 1) || !mbar_wait(fy(sy), (i / SY) & 1) ||
            *(volatile int*)abort_flag) {
          atomicExch(&g_tc_status, 52);
          *(volatile int*)abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t yb = ysb + sy * BF_YT;
        const uint32_t hb = mbase + sa * mstage;
        uint64_t y[3];
#pragma unroll
        for (int p = 0; p < 3; ++p) y[p] = umma_desc(yb + p * 4096, 128, 256);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint64_t hd[3];
#pragma unroll
          for (int p = 0; p < 3; ++p) hd[p] = umma_desc(hb + p * trow + h * hrow, 128, 256);
          const uint32_t acc = tmem + h * 256;
          mma_f16(acc, y[0], hd[2], idesc, i > 0);
          mma_f16(acc, y[1], hd[1], idesc, 1);
          mma_f16(acc, y[2], hd[0], idesc, 1);
          mma_f16(acc, y[0], hd[1], idesc, 1);
          mma_f16(acc, y[1], hd[0], idesc, 1);
          mma_f16(acc, y[0], hd[0], idesc, 1);
        }
        umma_commit(ea(sa));
        umma_commit(ey(sy));
      }
      umma_commit(accb);
    }
  } else {
    // warps 0-7: gather + split (pair = warp >> 1 owns Y stage pair)
    const int pair = warp >> 1, q = warp & 1;
    for (int i = pair; i < nk; i += BFW_NPAIR) {
      const int s = i % SY;
      float v[8][4];
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int l = i * BF_KC + q * 8 + a;
        const int g = l < ne ? dm[l] : -1;
        const float* src = P.Yin + (int64_t)(g < 0 ? 0 : g) * P.ld_in + c0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = lane + 32 * u;
          v[a][u] = (g >= 0 && c < ncv) ? __ldg(src + c) : 0.f;
        }
      }
      if (i >= SY && !mbar_wait(ey(s), ((i / SY) - 1) & 1)) {
        atomicExch(&g_tc_status, 53);
        *(volatile int*)abort_flag = 1;
      }
      if (*(volatile int*)abort_flag) break;
      uint16_t* ys = reinterpret_cast<uint16_t*>(ybase + s * BF_YT);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int o = bf_elem_off(lane + 32 * u, q * 8);
        uint32_t w[3][4];
#pragma unroll
        for (int a = 0; a < 8; a += 2)
          bf16_split3_pair(v[a][u], v[a + 1][u], w[0][a / 2], w[1][a / 2], w[2][a / 2]);
#pragma unroll
        for (int p = 0; p < 3; ++p)
          *reinterpret_cast<uint4*>(ys + p * 128 * BF_KC + o) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
      }
      fence_proxy_async_smem();
      mbar_arrive(fy(s));
    }
    // epilogue: part h = warp / 4, TMEM lane quarter = warp % 4 (column c0 + 32 (warp % 4) + lane)
    const bool okacc = mbar_wait(accb, 0);
    if (!okacc) {
      atomicExch(&g_tc_status, 54);
      *(volatile int*)abort_flag = 1;
    }
    tc_fence_after();
    const bool run = __all_sync(0xffffffffu, okacc && !*(volatile int*)abort_flag);
    const int h = warp >> 2, wq = warp & 3;
    const int r0 = h * B.nh;
    const int c = wq * 32 + lane;
    float* dst = P.R + ((int64_t)e * ne + r0) * P.ldr + c0 + c;
    for (int cb = 0; cb < B.nh; cb += 16) {
      float acc[16];
      __syncwarp();
      if (run) {
        tmem_ld16(tmem + ((uint32_t)(wq * 32) << 16) + h * 256 + cb, acc);
        tmem_wait_ld();
      }
      if (!run || c >= ncv) continue;
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (r0 + cb + j < ne) dst[(int64_t)(cb + j) * P.ldr] = acc[j];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == WMMA) tmem_dealloc(tmem, 512);
}

cudaError_t tc_cell_bf16_launch(const TcCellData& d, const TcApplyArgs& a, cudaStream_t s) {
  if (a.ncells == 0 || a.ncol == 0) return cudaSuccess;
  if (!d.bf) return cudaErrorInvalidValue;
  const int nk16 = (d.ne + BF_KC - 1) / BF_KC;
  const BfPlan B = bf_plan(d.ne);
  if (B.np * B.nh > d.mt * 128) return cudaErrorInvalidValue;   // parts stay inside the packed rows
  RParams P{reinterpret_cast<const float*>(d.bf), a.dofmap, a.Yin, a.R, a.ld_in, a.ncol, d.ne, d.mt,
            nk16, 1, nullptr, 0, 0, a.ncol, 0};
  P.r_evict = (double)a.ncells * d.ne * a.ncol * 4 > 2.0 * kL2Bytes;
  if (a.Z) {   // projector chunks: only the ring kernels take them
    if (!d.nl || !tc_cell_bf16_nl_ok(a.gather)) return cudaErrorInvalidValue;
    P.nlA = d.nl;
    P.nl_off = d.nl_off;
    P.nl_zrow = d.nl_zrow;
    P.Z = a.Z;
    P.ldz = a.ldz;
  }
  if (a.kG) {   // the Bloch block: the ring kernel with two-column pairs
    if (a.Z || (a.ncol & 1) || (a.ld_in & 1)) return cudaErrorInvalidValue;
    P.nlA = a.kG;
    static std::once_flag attrk;
    std::call_once(attrk, [] {
      cudaFuncSetAttribute(tc_cell_bf16_rings_kernel<2, false, 3, false, false, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
    const BfrPlan BK = bfr_plan(d.ne, 2);
    for (int64_t e0 = 0; e0 < a.ncells; e0 += 65535) {
      P.e_off = e0;
      dim3 grid((unsigned)(((a.ncol + 127) / 128) * B.np), (unsigned)std::min<int64_t>(65535, a.ncells - e0));
      note_launch();
      tc_cell_bf16_rings_kernel<2, false, 3, false, false, true><<<grid, 6 * 32, BK.total, s>>>(P);
    }
    return cudaGetLastError();
  }
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(tc_cell_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(tc_cell_bf16_async_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(tc_cell_bf16_rings_kernel<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(tc_cell_bf16_rings_kernel<4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(tc_cell_bf16_rings_kernel<2, false, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    cudaFuncSetAttribute(tc_cell_bf16_rings_kernel<4, false, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    cudaFuncSetAttribute(tc_cell_bf16_rings_kernel<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(tc_cell_bf16_whole_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(tc_cell_bf16_tiles_kernel<2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(tc_cell_bf16_tiles_kernel<4, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  });
  const bool async = a.gather == 1 && tc_cell_bf16_async_ok(a);
  const BfaPlan BA = bfa_plan(d.ne);
  const BfrPlan BR = bfr_plan(d.ne, 2), BR4 = bfr_plan(d.ne, 4);
  const BfwPlan BW = bfw_plan(d.ne);
  if ((a.gather == 5 || a.gather == 6) && !P.nlA) {   // several column tiles per CTA
    const bool two = a.gather == 6;   // one CTA per SM, two accumulators, all tiles of a row part
    const int ntiles = (a.ncol + 127) / 128;
    P.tpc = two ? ntiles : std::min(ntiles, kTilesPerCta);
    const int ngroups = (ntiles + P.tpc - 1) / P.tpc;
    const BfrPlan BT = bfr_plan(d.ne, 4, 3, 0, true);
    for (int64_t e0 = 0; e0 < a.ncells; e0 += 65535) {
      P.e_off = e0;
      dim3 grid((unsigned)(ngroups * B.np), (unsigned)std::min<int64_t>(65535, a.ncells - e0));
      note_launch();
      if (two)
        tc_cell_bf16_tiles_kernel<4, 2><<<grid, 14 * 32, BT.total, s>>>(P);
      else
        tc_cell_bf16_tiles_kernel<2, 1><<<grid, 10 * 32, BR.total, s>>>(P);
    }
    return cudaGetLastError();
  }
  for (int64_t e0 = 0; e0 < a.ncells; e0 += 65535) {
    P.e_off = e0;
    dim3 grid((unsigned)(((a.ncol + 127) / 128) * B.np), (unsigned)std::min<int64_t>(65535, a.ncells - e0));
    note_launch();
    if (async)
      tc_cell_bf16_async_kernel<<<grid, BFA_THREADS, BA.total, s>>>(P);
    else if (a.gather == 2 && P.nlA)
      tc_cell_bf16_rings_kernel<2, false, 3, true><<<grid, 6 * 32, BR.total, s>>>(P);
    else if (a.gather == 3 && P.nlA)
      tc_cell_bf16_rings_kernel<4, false, 3, true><<<grid, 10 * 32, BR4.total, s>>>(P);
    else if (a.gather == 2)
      tc_cell_bf16_rings_kernel<2, false><<<grid, 6 * 32, BR.total, s>>>(P);
    else if (a.gather == 3)
      tc_cell_bf16_rings_kernel<4, false><<<grid, 10 * 32, BR4.total, s>>>(P);
    else if (a.gather == 4 && bfw_supported(d.ne))
      tc_cell_bf16_whole_kernel<<<dim3((unsigned)((a.ncol + 127) / 128), grid.y), BFW_THREADS, BW.total, s>>>(P);
    else if (a.gather == 4)
      tc_cell_bf16_rings_kernel<2, false><<<grid, 6 * 32, BR.total, s>>>(P);
    else
      tc_cell_bf16_kernel<<<grid, CELL_THREADS, B.total, s>>>(P);
  }
  return cudaGetLastError();
}

cudaError_t tc_cell_f16_launch(const TcCellData& d, const TcApplyArgs& a, const uint32_t* cmax,
                               cudaStream_t s) {
  if (a.ncells == 0 || a.ncol == 0) return cudaSuccess;
  if (!d.f16 || !d.f16_inv || !cmax) return cudaErrorInvalidValue;
  const int nk16 = (d.ne + BF_KC - 1) / BF_KC;
  const BfPlan B = bf_plan(d.ne);
  if (B.np * B.nh > d.mt * 128) return cudaErrorInvalidValue;
  RParams P{reinterpret_cast<const float*>(d.f16), a.dofmap, a.Yin, a.R, a.ld_in, a.ncol, d.ne, d.mt,
            nk16, 1, nullptr, 0, 0, a.ncol, 0, cmax, d.f16_inv};
  P.r_evict = (double)a.ncells * d.ne * a.ncol * 4 > 2.0 * kL2Bytes;
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(tc_cell_bf16_rings_kernel<2, false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
  });
  const BfrPlan BR = bfr_plan(d.ne, 2, 2);
  for (int64_t e0 = 0; e0 < a.ncells; e0 += 65535) {
    P.e_off = e0;
    dim3 grid((unsigned)(((a.ncol + 127) / 128) * B.np), (unsigned)std::min<int64_t>(65535, a.ncells - e0));
    note_launch();
    tc_cell_bf16_rings_kernel<2, false, 2><<<grid, 6 * 32, BR.total, s>>>(P);
  }
  return cudaGetLastError();
}

cudaError_t tc_nl_project_cells(const TcCellData& d, const int32_t* dofmap, int64_t ncells, int nsite,
                                const float* Y, int64_t ldy, int ncol, float* part, float* Z, cudaStream_t s) {
  if (ncells == 0 || ncol == 0 || nsite == 0) return cudaSuccess;
  if (!d.pj) return cudaErrorInvalidValue;
  const int nk16 = (d.ne + BF_KC - 1) / BF_KC;
  RParams P{reinterpret_cast<const float*>(d.pj), dofmap, Y, part, ldy, ncol, d.ne, d.mt, nk16, 1, nullptr, 0, 0,
            ncol, 0};
  P.pj_np = d.pj_np;
  P.pj_off = d.pj_off;
  P.pj_row = d.pj_row;
  P.pj_npmax = d.pj_npmax;
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(tc_cell_bf16_rings_kernel<2, false, 3, false, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  const BfrPlan BR = bfr_plan(d.ne, 2, 3, d.pj_npmax);
  for (int64_t e0 = 0; e0 < ncells; e0 += 65535) {
    P.e_off = e0;
    dim3 grid((unsigned)((ncol + 127) / 128), (unsigned)std::min<int64_t>(65535, ncells - e0));
    note_launch();
    tc_cell_bf16_rings_kernel<2, false, 3, false, true><<<grid, 6 * 32, BR.total, s>>>(P);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t tot = (int64_t)4 * nsite * ncol;
  note_launch();
  nl_proj_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(d.pj_red_ptr, d.pj_red_row, part, nsite,
                                                                      ncol, Z);
  return cudaGetLastError();
}

int tc_bf16_parts(int ne) { return bf_plan(ne).np; }

cudaError_t tc_cell_bf16_multi_launch(const TcBatchSys* d_sys, int nsys, int64_t nitems, int ne, int mt,
                                      int parity, cudaStream_t s) {
  if (nitems == 0 || nsys == 0) return cudaSuccess;
  if (nitems > 0x7fffffff) return cudaErrorInvalidValue;
  const int nk16 = (ne + BF_KC - 1) / BF_KC;
  const BfPlan B0 = bf_plan(ne);
  if (B0.np * B0.nh > mt * 128) return cudaErrorInvalidValue;
  RParams P{nullptr, nullptr, nullptr, nullptr, 0, 0, ne, mt, nk16, 1, d_sys, nsys, parity, 0, 0};
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(tc_cell_bf16_rings_kernel<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
  });
  const BfrPlan BR = bfr_plan(ne, 2);
  note_launch();
  tc_cell_bf16_rings_kernel<2, true><<<(unsigned)nitems, 6 * 32, BR.total, s>>>(P);
  return cudaGetLastError();
}

// Each thread: one unknown j, 4 consecutive columns.  Sums the cell rows
// holding j in ascending cell order, adds the projector term (when Z is set:
// sum over the sites touching j of the h-scaled coefficients times the
// projected block Z, the expansion half of H~_nl, in the order of j's site
// list), then applies the three-term update.  Y_out may alias Y_prev (each
// element is read before it is written by the same thread); it must not
// alias Y_in.
// The update of unknown j, columns c .. c + 3 (fewer at the block's edge);
// absout (when not null) receives |Y_out| of the four columns (0 past the edge).
template <bool NL>
__device__ __forceinline__ void assemble_quad(const AssembleParams& P, int64_t j, int c,
                                              float* absout = nullptr) {
  const int nc = min(4, P.ncol - c);
  const bool v4 = P.vec && nc == 4;
  float sum[4] = {0.f, 0.f, 0.f, 0.f};
  const int k0 = P.node_ptr[j], k1 = P.node_ptr[j + 1];
  for (int k = k0; k < k1; ++k) {
    const float* src = P.R + (int64_t)P.node_ent[k] * P.ncol + c;
    if (v4) {
      const float4 r = __ldg(reinterpret_cast<const float4*>(src));
      sum[0] += r.x; sum[1] += r.y; sum[2] += r.z; sum[3] += r.w;
    } else {
      for (int u = 0; u < nc; ++u) sum[u] += __ldg(src + u);
    }
  }
  if (NL) {
    float nl[4] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t e = P.dof_ptr[j]; e < P.dof_ptr[j + 1]; ++e) {
      const int64_t st = P.dof_site[e];
      const float4 cf = __ldg(reinterpret_cast<const float4*>(P.dof_c) + e);
      const float cq[4] = {cf.x, cf.y, cf.z, cf.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float* zr = P.Z + (4 * st + t) * P.ncol + c;
        if (v4) {
          const float4 z = __ldg(reinterpret_cast<const float4*>(zr));
          nl[0] = fmaf(cq[t], z.x, nl[0]);
          nl[1] = fmaf(cq[t], z.y, nl[1]);
          nl[2] = fmaf(cq[t], z.z, nl[2]);
          nl[3] = fmaf(cq[t], z.w, nl[3]);
        } else {
          for (int u = 0; u < nc; ++u) nl[u] = fmaf(cq[t], __ldg(zr + u), nl[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) sum[u] += nl[u];
  }
  float yin[4] = {0.f, 0.f, 0.f, 0.f}, yp[4] = {0.f, 0.f, 0.f, 0.f};
  const bool vin = v4 && P.vin, vprev = v4 && P.vprev, vout = v4 && P.vout;
  if (P.shift == 0.f) {
    // an application of H~ (no shift): Y_in is not read; sum - 0 * 0 equals sum - 0 * y_in
  } else if (vin) {
    const float4 t = *reinterpret_cast<const float4*>(P.Yin + j * P.ld_in + c);
    yin[0] = t.x; yin[1] = t.y; yin[2] = t.z; yin[3] = t.w;
  } else {
    for (int u = 0; u < nc; ++u) yin[u] = P.Yin[j * P.ld_in + c + u];
  }
  if (P.Yprev) {
    if (vprev) {
      const float4 t = *reinterpret_cast<const float4*>(P.Yprev + j * P.ld_prev + c);
      yp[0] = t.x; yp[1] = t.y; yp[2] = t.z; yp[3] = t.w;
    } else {
      for (int u = 0; u < nc; ++u) yp[u] = P.Yprev[j * P.ld_prev + c + u];
    }
  }
  float out[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    out[u] = P.alpha * (sum[u] - P.shift * yin[u]);
    if (P.Yprev) out[u] = fmaf(P.beta, yp[u], out[u]);
  }
  float* dst = P.Yout + j * P.ld_out + c;
  if (vout) {
    *reinterpret_cast<float4*>(dst) = make_float4(out[0], out[1], out[2], out[3]);
  } else {
    for (int u = 0; u < nc; ++u) dst[u] = out[u];
  }
  if (absout) {
#pragma unroll
    for (int u = 0; u < 4; ++u) absout[u] = u < nc ? fabsf(out[u]) : 0.f;
  }
}

// Each thread: one unknown j, 4 consecutive columns.  Sums the cell rows
// holding j in ascending cell order, adds the projector term (when Z is set:
// sum over the sites touching j of the h-scaled coefficients times the
// projected block Z, the expansion half of H~_nl, in the order of j's site
// list), then applies the three-term update.  Y_out may alias Y_prev (each
// element is read before it is written by the same thread); it must not
// alias Y_in.
template <bool NL>
__global__ void __launch_bounds__(256) tc_assemble_kernel(AssembleParams P) {
  const int nq = (P.ncol + 3) / 4;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= P.M * nq) return;
  const int64_t j = idx / nq;
  const int c = (int)(idx - j * nq) * 4;
  assemble_quad<NL>(P, j, c);
}

// The same per-element update with the column maxima of |Y_out|: block (32,
// 8) takes 128 columns (a quad per lane) of every 8-th row group; each thread
// keeps its quad's maximum over its rows, the block reduces over its 8 row
// lanes and adds one atomicMax per column (binary32 bits of a non-negative
// value order as unsigned integers).
template <bool NL>
__global__ void __launch_bounds__(256) tc_assemble_cmax_kernel(AssembleParams P, uint32_t* __restrict__ cmax) {
  const int nq = (P.ncol + 3) / 4;
  const int qd = blockIdx.x * 32 + threadIdx.x;
  float m[4] = {0.f, 0.f, 0.f, 0.f};
  if (qd < nq) {
    const int c = qd * 4;
    for (int64_t j = (int64_t)blockIdx.y * 8 + threadIdx.y; j < P.M; j += (int64_t)gridDim.y * 8) {
      float a[4];
      assemble_quad<NL>(P, j, c, a);
#pragma unroll
      for (int u = 0; u < 4; ++u) m[u] = fmaxf(m[u], a[u]);
    }
  }
  __shared__ float red[8][32][4];
#pragma unroll
  for (int u = 0; u < 4; ++u) red[threadIdx.y][threadIdx.x][u] = m[u];
  __syncthreads();
  if (threadIdx.y == 0 && qd < nq) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      float t = red[0][threadIdx.x][u];
      for (int w = 1; w < 8; ++w) t = fmaxf(t, red[w][threadIdx.x][u]);
      if (qd * 4 + u < P.ncol) atomicMax(cmax + qd * 4 + u, __float_as_uint(t));
    }
  }
}

// Column maxima of |Y| with the same mapping.
__global__ void __launch_bounds__(256) tc_colmax_kernel(const float* __restrict__ Y, int64_t ld, int64_t M,
                                                        int ncol, uint32_t* __restrict__ cmax) {
  const int nq = (ncol + 3) / 4;
  const int qd = blockIdx.x * 32 + threadIdx.x;
  float m[4] = {0.f, 0.f, 0.f, 0.f};
  if (qd < nq) {
    const int c = qd * 4;
    const int nc = min(4, ncol - c);
    for (int64_t j = (int64_t)blockIdx.y * 8 + threadIdx.y; j < M; j += (int64_t)gridDim.y * 8)
      for (int u = 0; u < nc; ++u) m[u] = fmaxf(m[u], fabsf(__ldg(Y + j * ld + c + u)));
  }
  __shared__ float red[8][32][4];
#pragma unroll
  for (int u = 0; u < 4; ++u) red[threadIdx.y][threadIdx.x][u] = m[u];
  __syncthreads();
  if (threadIdx.y == 0 && qd < nq) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      float t = red[0][threadIdx.x][u];
      for (int w = 1; w < 8; ++w) t = fmaxf(t, red[w][threadIdx.x][u]);
      if (qd * 4 + u < ncol) atomicMax(cmax + qd * 4 + u, __float_as_uint(t));
    }
  }
}

// Row groups of the column-maximum grids: about 8 blocks per SM over all columns.
static unsigned cmax_row_blocks(int64_t M, int ncol) {
  const int64_t xs = ((ncol + 3) / 4 + 31) / 32;
  int64_t ys = std::max<int64_t>(1, (8 * 152 + xs - 1) / xs);
  ys = std::min<int64_t>(ys, std::max<int64_t>(1, (M + 7) / 8));
  return (unsigned)std::min<int64_t>(ys, 65535);
}

cudaError_t tc_colmax_launch(const float* Y, int64_t ld, int64_t M, int ncol, uint32_t* cmax,
                             cudaStream_t s) {
  if (ncol <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(cmax, 0, (size_t)ncol * sizeof(uint32_t), s);
  if (e != cudaSuccess || M <= 0) return e;
  dim3 grid((unsigned)(((ncol + 3) / 4 + 31) / 32), cmax_row_blocks(M, ncol));
  note_launch();
  tc_colmax_kernel<<<grid, dim3(32, 8), 0, s>>>(Y, ld, M, ncol, cmax);
  return cudaGetLastError();
}

cudaError_t tc_assemble_launch(const AssembleParams& P0, cudaStream_t s) {
  const int64_t tot = P0.M * ((P0.ncol + 3) / 4);
  if (tot == 0) return cudaSuccess;
  AssembleParams P = P0;
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  P.vec = (P.ncol & 3) == 0 && al16(P.R) && (!P.Z || al16(P.Z));
  P.vin = (P.ld_in & 3) == 0 && al16(P.Yin);
  P.vprev = P.Yprev && (P.ld_prev & 3) == 0 && al16(P.Yprev);
  P.vout = (P.ld_out & 3) == 0 && al16(P.Yout);
  note_launch();
  if (P.Z)
    tc_assemble_kernel<true><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(P);
  else
    tc_assemble_kernel<false><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t tc_assemble_cmax_launch(const AssembleParams& P0, uint32_t* cmax, cudaStream_t s) {
  if (P0.ncol <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(cmax, 0, (size_t)P0.ncol * sizeof(uint32_t), s);
  if (e != cudaSuccess || P0.M <= 0) return e;
  AssembleParams P = P0;
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  P.vec = (P.ncol & 3) == 0 && al16(P.R) && (!P.Z || al16(P.Z));
  P.vin = (P.ld_in & 3) == 0 && al16(P.Yin);
  P.vprev = P.Yprev && (P.ld_prev & 3) == 0 && al16(P.Yprev);
  P.vout = (P.ld_out & 3) == 0 && al16(P.Yout);
  dim3 grid((unsigned)(((P.ncol + 3) / 4 + 31) / 32), cmax_row_blocks(P.M, P.ncol));
  note_launch();
  if (P.Z)
    tc_assemble_cmax_kernel<true><<<grid, dim3(32, 8), 0, s>>>(P, cmax);
  else
    tc_assemble_cmax_kernel<false><<<grid, dim3(32, 8), 0, s>>>(P, cmax);
  return cudaGetLastError();
}

cudaError_t tc_set_withhold(int on, cudaStream_t s) {
  const int v = on ? 1 : 0;
  cudaError_t e = cudaMemcpyToSymbolAsync(g_tc_withhold, &v, sizeof(int), 0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

int tc_read_status(cudaStream_t s) {
  int v = 0;
  cudaMemcpyFromSymbolAsync(&v, g_tc_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  if (v) {
    int z = 0;
    cudaMemcpyToSymbolAsync(g_tc_status, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
  }
  return v;
}

// ----------------------------------------------------------------- Gram (A^T B)
constexpr int GR_T = 128, GR_KC = 8, GR_THREADS = 160, GR_S = 6;
static_assert(GR_S >= 4, "parity waits of the 4 producer warps need at least 4 stages");

__host__ __device__ inline int gram_stage_bytes(int same) {
  return (same ? 1 : 2) * GR_T * GR_KC * 4 * 2;   // operands x (hi + lo)
}

struct GramParams {
  const float* A;
  const float* B;
  int64_t lda, ldb, M;
  int n1, n2, lower, split3;
  int64_t rows_per_split;
  double* partial;
};

// (row n, K index k) of a 128 x 8 operand block, K-major core matrices:
// LBO 128 B along K, SBO 256 B along the 128 rows.
__device__ __forceinline__ int k8_off(int n, int k) {
  return (n >> 3) * 64 + (k >> 2) * 32 + (n & 7) * 4 + (k & 3);
}

// Load 4 rows x the 4 columns col0 + 32 v (v = 0..3; one lane of a warp, so a
// warp reads 128 contiguous bytes per row and column block): v[a][u] = X[row0 + a][col0 + 32 u].
__device__ __forceinline__ void load4x4_strided(const float* __restrict__ X, int64_t ld, int64_t row0,
                                                int64_t r1, int col0, int nmax, float v[4][4]) {
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t row = row0 + a;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = col0 + 32 * u;
      v[a][u] = (row < r1 && c < nmax) ? __ldg(X + row * ld + c) : 0.f;
    }
  }
}
// Store of load4x4_strided's block: column n = nbase + 32 u, its 4 K values as
// one 16-byte store.  Eight consecutive lanes write one 128-byte core matrix,
// so each quarter-warp phase is free of bank conflicts.
__device__ __forceinline__ void store_split_t_strided(float* hi, float* lo, int nbase, int kq,
                                                      const float v[4][4]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int o = k8_off(nbase + 32 * u, kq * 4);
    float4 h, l;
    h.x = tf32_rna(v[0][u]); l.x = v[0][u] - h.x;
    h.y = tf32_rna(v[1][u]); l.y = v[1][u] - h.y;
    h.z = tf32_rna(v[2][u]); l.z = v[2][u] - h.z;
    h.w = tf32_rna(v[3][u]); l.w = v[3][u] - h.w;
    *reinterpret_cast<float4*>(hi + o) = h;
    *reinterpret_cast<float4*>(lo + o) = l;
  }
}
// Output tile 128 x 128 of C = A^T B (rows i of C <-> columns of A, columns j
// <-> columns of B); K = unknowns, split over grid.z.  Warps 0-3 produce the
// K-chunks (warp w: chunks w, w+4, ...; registers prefetched before the stage
// is free), warp 4 issues the MMAs.  Tiles strictly above the diagonal are
// skipped when `lower`; partial tiles (binary64) are reduced in fixed order.
__global__ void __launch_bounds__(GR_THREADS, 1) tc_gram_kernel(GramParams P) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int ti = blockIdx.x, tj = blockIdx.y, z = blockIdx.z;
  if (P.lower && ti < tj) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool same = (P.A == P.B) && (P.lda == P.ldb) && ti == tj;
  const int SB = gram_stage_bytes(same);
  const int S = GR_S;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * gram_stage_bytes(0));
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  const uint32_t sbase = smem_u32(smem);
  auto full = [&](int s) { return smem_u32(bars + s); };
  auto emp = [&](int s) { return smem_u32(bars + S + s); };
  const uint32_t accb = smem_u32(bars + 2 * S);
  const int64_t r0 = (int64_t)z * P.rows_per_split;
  const int64_t r1 = min(P.M, r0 + P.rows_per_split);
  const int nk = r1 > r0 ? (int)((r1 - r0 + GR_KC - 1) / GR_KC) : 0;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full(s), 32);
      mbar_init(emp(s), 1);
    }
    mbar_init(accb, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 4) {
    tmem_alloc(smem_u32(tmem_slot), 128);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 4) {
    if (lane == 0 && nk > 0) {
      const uint32_t idesc = idesc_tf32(128, 128);
      for (int i = 0; i < nk; ++i) {
        const int s = i % S;
        if (!mbar_wait(full(s), (i / S) & 1) || *(volatile int*)abort_flag) {
          atomicExch(&g_tc_status, 5);
          *(volatile int*)abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t sa = sbase + s * SB;
        const uint32_t sb = same ? sa : sa + GR_T * GR_KC * 8;
        const uint64_t ah = umma_desc(sa, 128, 256);
        const uint64_t al = umma_desc(sa + GR_T * GR_KC * 4, 128, 256);
        const uint64_t bh = umma_desc(sb, 128, 256);
        const uint64_t bl = umma_desc(sb + GR_T * GR_KC * 4, 128, 256);
        if (P.split3) {
          mma_tf32(tmem, al, bh, idesc, i > 0);
          mma_tf32(tmem, ah, bl, idesc, 1);
          mma_tf32(tmem, ah, bh, idesc, 1);
        } else {
          mma_tf32(tmem, ah, bh, idesc, i > 0);
        }
        umma_commit(emp(s));
      }
      umma_commit(accb);
    }
  } else {
    // lane l owns the tile columns l, l + 32, l + 64, l + 96 (conflict-free split stores)
    const int ia = ti * GR_T + lane, jb = tj * GR_T + lane;
    auto load_chunk = [&](int i, float (&va)[2][4][4], float (&vb)[2][4][4]) {
      const int64_t row0 = r0 + (int64_t)i * GR_KC;
#pragma unroll
      for (int kq = 0; kq < 2; ++kq) {
        load4x4_strided(P.A, P.lda, row0 + kq * 4, r1, ia, P.n1, va[kq]);
        if (!same) load4x4_strided(P.B, P.ldb, row0 + kq * 4, r1, jb, P.n2, vb[kq]);
      }
    };
    auto fill_stage = [&](int i, const float (&va)[2][4][4], const float (&vb)[2][4][4]) -> bool {
      const int s = i % S;
      if (i >= S && !mbar_wait(emp(s), ((i / S) - 1) & 1)) {
        atomicExch(&g_tc_status, 6);
        *(volatile int*)abort_flag = 1;
      }
      if (*(volatile int*)abort_flag) return false;
      float* sh = reinterpret_cast<float*>(smem + s * SB);
#pragma unroll
      for (int kq = 0; kq < 2; ++kq) {
        store_split_t_strided(sh, sh + GR_T * GR_KC, lane, kq, va[kq]);
        if (!same) store_split_t_strided(sh + GR_T * GR_KC * 2, sh + GR_T * GR_KC * 3, lane, kq, vb[kq]);
      }
      fence_proxy_async_smem();
      mbar_arrive(full(s));
      return true;
    };
    // chunks warp, warp + 4, ...: loads into registers before the stage is
    // free, then the split.  (A second register set for the next chunk costs
    // the second CTA per SM: 196 registers, measured 1.5x slower.)
    for (int i = warp; i < nk; i += 4) {
      float va[2][4][4], vb[2][4][4];
      load_chunk(i, va, vb);
      if (!fill_stage(i, va, vb)) break;
    }
    bool okacc = true;
    if (nk > 0) {
      okacc = mbar_wait(accb, 0);
      if (!okacc) atomicExch(&g_tc_status, 7);
    }
    tc_fence_after();
    // epilogue: thread row i = ti*128 + warp*32 + lane; consecutive lanes write
    // consecutive i of a column-major partial tile (coalesced)
    __syncwarp();   // tcgen05.ld is warp-aligned: reconverge after the polling above
    const int i = ti * GR_T + warp * 32 + lane;
    double* Pz = P.partial + (int64_t)z * P.n1 * P.n2;
    for (int cb = 0; cb < 128; cb += 16) {
      float acc[16];
      __syncwarp();
      if (nk > 0) {
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + cb, acc);
        tmem_wait_ld();
      } else {
        for (int u = 0; u < 16; ++u) acc[u] = 0.f;
      }
      if (i >= P.n1 || !okacc) continue;
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int j = tj * GR_T + cb + u;
        if (j < P.n2) Pz[i + (int64_t)j * P.n1] = (double)acc[u];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 4) tmem_dealloc(tmem, 128);
}

__global__ void tc_gram_reduce_kernel(const double* __restrict__ partial, int nsplit, int n1, int n2,
                                      double* __restrict__ C, int64_t ldc, int lower) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n1 * n2) return;
  const int i = (int)(idx % n1), j = (int)(idx / n1);
  if (lower && (i / GR_T) < (j / GR_T)) return;
  double s = 0.0;
  for (int zz = 0; zz < nsplit; ++zz) s += partial[(int64_t)zz * n1 * n2 + idx];
  C[i + (int64_t)j * ldc] = s;
}

// Diagonal blocks of A^T B in extended precision: C[i, j] = sum_r A[r, i] B[r, j]
// for i / bd == j / bd (i, j < min(n1, n2); BD divides 32).  Block: 8 row
// lanes x 32 columns; a thread owns column i and accumulates its BD block
// partners, whose B values come from neighbouring lanes by warp shuffles.
// Every product is split exactly into p + e (p = a b rounded, e = fma(a, b, -p))
// and summed as a float pair (Knuth's two-sum on the leading part, the
// rounding errors and e gathered in the trailing part); every 16 products per
// entry the pair is added into a binary64 partial sum.  This keeps the sums at
// binary64-class accuracy (relative error ~1e-13 of sum |a b| at these
// lengths) with two binary64 additions per 16 products: GB300's binary64 pipe
// issues 2 operations per clock and SM against 128 binary32 ones, and the
// plain binary64 form (two conversions and an FMA per product) was bound by
// it.  Rows are taken four at a time (four loads in flight per thread);
// partial sums over row chunks are reduced in fixed order.
// (explicitly rounded operations: the two-sum must not be contracted into FMAs)
__device__ __forceinline__ void ff_add_prod(float a, float b, float& sh, float& sl) {
  const float p = __fmul_rn(a, b);
  const float e = fmaf(a, b, -p);
  const float t = __fadd_rn(sh, p);
  const float bb = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(err, e));
}

template <int BD>
__global__ void __launch_bounds__(256) diag_gram_ff_kernel(const float* __restrict__ A, int64_t lda,
                                                           const float* __restrict__ B, int64_t ldb,
                                                           int64_t M, int nd, int64_t rows_per_chunk,
                                                           double* __restrict__ part) {
  const int lane = threadIdx.x & 31, rl = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t r1 = min(M, r0 + rows_per_chunk);
  const int jb = lane / BD * BD;            // first lane of this column's block
  const bool in = i < nd;
  double acc[BD];
  float sh[BD], sl[BD];
#pragma unroll
  for (int q = 0; q < BD; ++q) {
    acc[q] = 0.0;
    sh[q] = 0.f;
    sl[q] = 0.f;
  }
  auto flush = [&]() {
#pragma unroll
    for (int q = 0; q < BD; ++q) {
      acc[q] += (double)sh[q] + (double)sl[q];
      sh[q] = 0.f;
      sl[q] = 0.f;
    }
  };
  int64_t r = r0 + rl;
  int steps = 0;
  for (; r + 24 < r1; r += 32) {
    float a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a[u] = in ? A[(r + 8 * u) * lda + i] : 0.f;
      b[u] = in ? B[(r + 8 * u) * ldb + i] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int q = 0; q < BD; ++q) {
        const float bq = BD == 1 ? b[u] : __shfl_sync(0xffffffffu, b[u], jb + q);
        ff_add_prod(a[u], bq, sh[q], sl[q]);
      }
    if (++steps == 4) {
      flush();
      steps = 0;
    }
  }
  for (; r < r1; r += 8) {
    const float a = in ? A[r * lda + i] : 0.f;
    const float b = in ? B[r * ldb + i] : 0.f;
#pragma unroll
    for (int q = 0; q < BD; ++q) {
      const float bq = BD == 1 ? b : __shfl_sync(0xffffffffu, b, jb + q);
      ff_add_prod(a, bq, sh[q], sl[q]);
    }
  }
  flush();
  __shared__ double red[8][32];
#pragma unroll
  for (int q = 0; q < BD; ++q) {
    red[rl][lane] = acc[q];
    __syncthreads();
    if (rl == 0 && in) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += red[w][lane];
      part[((int64_t)blockIdx.y * gridDim.x * 32 + i) * BD + q] = t;
    }
    __syncthreads();
  }
}

__global__ void diag_reduce_kernel(const double* __restrict__ part, int nchunk, int ncols, int nd,
                                   int bd, double* __restrict__ C, int64_t ldc) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)nd * bd) return;
  const int i = (int)(idx / bd), q = (int)(idx % bd);
  const int j = i / bd * bd + q;
  if (j >= nd) return;
  double s = 0.0;
  for (int zz = 0; zz < nchunk; ++zz) s += part[((int64_t)zz * ncols + i) * bd + q];
  C[i + (int64_t)j * ldc] = s;
}

constexpr int GR_MAX_SPLIT = 16;
size_t tc_gram_partial_bytes(int64_t M, int n1, int n2) {
  (void)M;
  return (size_t)8 * GR_MAX_SPLIT * n1 * n2 + (size_t)64 * 1024 * 1024;
}

// K splits of the Gram grid: the grid runs in waves of `slots` CTAs (two per
// SM) and every CTA of a split takes the same time, so the launch lasts
// ceil(tiles * ns / slots) CTA times of 1 / ns of the rows each; take the ns
// that minimises that (the smaller on ties).
int64_t tc_gram_splits(int64_t tiles, int64_t max_split, int64_t slots) {
  int64_t best = 1;
  double tbest = 1e300;
  for (int64_t ns = 1; ns <= std::max<int64_t>(1, max_split); ++ns) {
    const double t = (double)((tiles * ns + slots - 1) / slots) / (double)ns;
    if (t < tbest * (1.0 - 1e-9)) {
      tbest = t;
      best = ns;
    }
  }
  return best;
}

cudaError_t tc_gram_mixed(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t M,
                          int n1, int n2, double* C, int64_t ldc, int lower, int diag_block,
                          int split3, void* partial, size_t partial_bytes, cudaStream_t s) {
  if (n1 == 0 || n2 == 0) return cudaSuccess;
  const int t1 = (n1 + GR_T - 1) / GR_T, t2 = (n2 + GR_T - 1) / GR_T;
  const int64_t tiles = lower ? (int64_t)t1 * (t1 + 1) / 2 : (int64_t)t1 * t2;
  const size_t diag_bytes = (size_t)64 * 1024 * 1024;
  int64_t max_split = (int64_t)((partial_bytes - diag_bytes) / (sizeof(double) * (size_t)n1 * n2));
  max_split = std::min<int64_t>(std::min<int64_t>(max_split, GR_MAX_SPLIT), (M + 1023) / 1024);
  int64_t nsplit = tc_gram_splits(tiles, max_split, 2 * 152);
  int64_t rps = ((M + nsplit - 1) / nsplit + GR_KC - 1) / GR_KC * GR_KC;
  nsplit = (M + rps - 1) / rps;
  GramParams P{A, B, lda, ldb, M, n1, n2, lower, split3, rps, (double*)partial};
  const int smem = GR_S * gram_stage_bytes(0) + 1024;
  static std::once_flag attr;
  std::call_once(attr, [&] {
    cudaFuncSetAttribute(tc_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  });
  note_launch();
  tc_gram_kernel<<<dim3(t1, t2, (unsigned)nsplit), GR_THREADS, smem, s>>>(P);
  const int64_t tot = (int64_t)n1 * n2;
  note_launch();
  tc_gram_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>((double*)partial, (int)nsplit,
                                                                      n1, n2, C, ldc, lower);
  // extended-precision diagonal blocks overwrite the tensor-core values there
  if (diag_block > 0) {
    int bd = 1;
    while (bd * 2 <= std::min(diag_block, 32)) bd *= 2;
    const int nd = std::min(n1, n2);
    const int ntile = (nd + 31) / 32;
    double* dpart = (double*)((char*)partial + (partial_bytes - diag_bytes));
    // about 64 resident blocks of 256 threads per SM's worth of row chunks
    int64_t nchunk = std::max<int64_t>(1, (64 * 152 + ntile - 1) / ntile);
    nchunk = std::min<int64_t>(nchunk, (int64_t)(diag_bytes / (8 * (size_t)ntile * 32 * bd)));
    nchunk = std::max<int64_t>(1, std::min<int64_t>(nchunk, (M + 255) / 256));
    int64_t rpc = (M + nchunk - 1) / nchunk;
    nchunk = (M + rpc - 1) / rpc;
    const dim3 dg(ntile, (unsigned)nchunk);
    note_launch();
    switch (bd) {
      case 1: diag_gram_ff_kernel<1><<<dg, 256, 0, s>>>(A, lda, B, ldb, M, nd, rpc, dpart); break;
      case 2: diag_gram_ff_kernel<2><<<dg, 256, 0, s>>>(A, lda, B, ldb, M, nd, rpc, dpart); break;
      case 4: diag_gram_ff_kernel<4><<<dg, 256, 0, s>>>(A, lda, B, ldb, M, nd, rpc, dpart); break;
      case 8: diag_gram_ff_kernel<8><<<dg, 256, 0, s>>>(A, lda, B, ldb, M, nd, rpc, dpart); break;
      case 16: diag_gram_ff_kernel<16><<<dg, 256, 0, s>>>(A, lda, B, ldb, M, nd, rpc, dpart); break;
      default: diag_gram_ff_kernel<32><<<dg, 256, 0, s>>>(A, lda, B, ldb, M, nd, rpc, dpart); break;
    }
    const int64_t tot2 = (int64_t)nd * bd;
    note_launch();
    diag_reduce_kernel<<<(unsigned)((tot2 + 255) / 256), 256, 0, s>>>(dpart, (int)nchunk, ntile * 32, nd,
                                                                       bd, C, ldc);
  }
  return cudaGetLastError();
}

// ----------------------------------------------------------------- tall GEMM (X U)
// C (M x n2) = A (M x n1, binary32) U (n1 x n2, binary64).  Tile: 128 rows x
// 128 columns; K-loop over n1 in chunks of 8.  U is split into TF32 hi / lo
// once per call into a chunked K-major layout (tc_splitu_kernel); diagonal
// blocks of U are excluded from the tensor-core product and added in binary64
// in the epilogue (the paper's Psi L^{-1}_d term).  Grid x runs over column
// tiles so the CTAs sharing a row block of A run together (A read once from
// HBM).  The epilogue stages the tile in shared memory and writes whole rows.
constexpr int TG_T = 128, TG_KC = 8, TG_THREADS = 160, TG_S = 6;
constexpr uint32_t TG_UBYTES = 2 * TG_T * TG_KC * 4;   // U chunk, hi + lo
static_assert(TG_S >= 4, "parity waits of the 4 producer warps need at least 4 stages");

// U split layout: [col tile][k chunk][hi|lo][128 cols x 8 K in k8_off layout]
__global__ void tc_splitu_kernel(const double* __restrict__ U, int64_t ldu, int n1, int n2, int upper,
                                 int trans, int bd, float* __restrict__ out) {
  const int nkc = (n1 + TG_KC - 1) / TG_KC;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int ntile = (n2 + TG_T - 1) / TG_T;
  if (idx >= (int64_t)ntile * nkc * TG_T * TG_KC) return;
  const int tile = (int)(idx / ((int64_t)nkc * TG_T * TG_KC));
  int rem = (int)(idx - (int64_t)tile * nkc * TG_T * TG_KC);
  const int kc = rem / (TG_T * TG_KC);
  rem -= kc * TG_T * TG_KC;
  const int n = rem / TG_KC, k = rem % TG_KC;
  const int col = tile * TG_T + n, kk = kc * TG_KC + k;
  double v = 0.0;
  if (col < n2 && kk < n1 && (!upper || kk <= col) && !(bd > 0 && kk / bd == col / bd))
    v = trans ? U[col + (int64_t)kk * ldu] : U[kk + (int64_t)col * ldu];
  const float h = tf32_rna((float)v);
  const float l = tf32_rna((float)(v - (double)h));
  float* base = out + ((int64_t)tile * nkc + kc) * 2 * TG_T * TG_KC;
  base[k8_off(n, k)] = h;
  base[TG_T * TG_KC + k8_off(n, k)] = l;
}

// Diagonal-block entries of U as float pairs: Ud[col * bd + q] = (hi, lo) of
// U[k0 + q, col] (k0 = col / bd * bd; zero outside U or, when upper, below
// the diagonal), hi + lo = U's entry to about 2^-48 relative.
__global__ void tc_diagu_kernel(const double* __restrict__ U, int64_t ldu, int n1, int n2, int upper,
                                int trans, int bd, float2* __restrict__ Ud) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n2 * bd) return;
  const int col = (int)(idx / bd), q = (int)(idx % bd);
  const int kk = col / bd * bd + q;
  double v = 0.0;
  if (kk < n1 && (!upper || kk <= col)) v = trans ? U[col + (int64_t)kk * ldu] : U[kk + (int64_t)col * ldu];
  const float h = (float)v;
  Ud[idx] = make_float2(h, (float)(v - (double)h));
}

// acc + sum over the diagonal block of col of A[row, kk] U[kk, col] (the
// paper's Psi L^{-1}_d term), in binary32 pairs: exact products of the
// leading parts, two-sum accumulation, the trailing parts of U by FMA.
__device__ __forceinline__ float tall_diag_add(float acc, const float* __restrict__ Arow,
                                               const float2* __restrict__ Ud, int col, int bd, int n1,
                                               int upper) {
  const int k0 = (col / bd) * bd;
  const int k1 = min(n1, k0 + bd);
  float sh = acc, sl = 0.f;
  for (int kk = k0; kk < k1; ++kk) {
    if (upper && kk > col) break;
    const float2 u = Ud[(int64_t)col * bd + (kk - k0)];
    const float a = Arow[kk];
    ff_add_prod(a, u.x, sh, sl);
    sl = __fmaf_rn(a, u.y, sl);
  }
  return __fadd_rn(sh, sl);
}

// bd = 1: the term is A[row, col] U[col, col] alone (zero for col >= n1).
__device__ __forceinline__ float tall_diag1(float acc, float a, float2 u) {
  float sh = acc, sl = 0.f;
  ff_add_prod(a, u.x, sh, sl);
  sl = __fmaf_rn(a, u.y, sl);
  return __fadd_rn(sh, sl);
}

struct TallParams {
  const float* A;
  int64_t lda, M;
  const float* Us;       // split U
  const float2* Ud;      // U's diagonal-block entries as float pairs (hi, lo), n2 x bd
  int64_t ldu;
  int n1, n2, upper, trans, bd, split3;
  float* C;
  int64_t ldc;
};

__global__ void __launch_bounds__(TG_THREADS, 1) tc_tall_kernel(TallParams P) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tj = blockIdx.x;
  const int64_t rb = (int64_t)blockIdx.y * TG_T;
  const int nkc_all = (P.n1 + TG_KC - 1) / TG_KC;
  int kend = P.n1;
  if (P.upper) kend = min(P.n1, (tj + 1) * TG_T);
  const int nk = (kend + TG_KC - 1) / TG_KC;
  const int SB = 2 * TG_T * TG_KC * 4 * 2;   // A (hi, lo) + U (hi, lo)
  const int S = TG_S;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * SB);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  const uint32_t sbase = smem_u32(smem);
  auto full = [&](int s) { return smem_u32(bars + s); };
  auto emp = [&](int s) { return smem_u32(bars + S + s); };
  const uint32_t accb = smem_u32(bars + 2 * S);
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full(s), 32);
      mbar_init(emp(s), 1);
    }
    mbar_init(accb, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 4) {
    tmem_alloc(smem_u32(tmem_slot), 128);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int ncv = min(TG_T, P.n2 - tj * TG_T);
  const int bne = (ncv + 15) / 16 * 16;

  if (warp == 4) {
    if (lane == 0 && nk > 0) {
      const uint32_t idesc = idesc_tf32(128, bne);
      for (int i = 0; i < nk; ++i) {
        const int s = i % S;
        if (!mbar_wait(full(s), (i / S) & 1) || *(volatile int*)abort_flag) {
          atomicExch(&g_tc_status, 8);
          *(volatile int*)abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t sa = sbase + s * SB;
        const uint32_t su = sa + TG_T * TG_KC * 8;
        const uint64_t ah = umma_desc(sa, 128, 256);
        const uint64_t al = umma_desc(sa + TG_T * TG_KC * 4, 128, 256);
        const uint64_t uh = umma_desc(su, 128, 256);
        const uint64_t ul = umma_desc(su + TG_T * TG_KC * 4, 128, 256);
        if (P.split3) {
          mma_tf32(tmem, al, uh, idesc, i > 0);
          mma_tf32(tmem, ah, ul, idesc, 1);
          mma_tf32(tmem, ah, uh, idesc, 1);
        } else {
          mma_tf32(tmem, ah, uh, idesc, i > 0);
        }
        umma_commit(emp(s));
      }
      umma_commit(accb);
    }
  } else {
    const bool vec = ((P.lda & 3) == 0) && ((reinterpret_cast<uintptr_t>(P.A) & 15) == 0);
    int last_issued = -1;
    for (int i = warp; i < nk; i += 4) {
      const int s = i % S;
      // A: rows rb + lane + 32 j, K quads kq: 4 consecutive K values (already K-major)
      float4 av[4][2];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t row = rb + lane + 32 * j;
#pragma unroll
        for (int kq = 0; kq < 2; ++kq) {
          const int k0 = i * TG_KC + kq * 4;
          float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
          if (row < P.M) {
            const float* src = P.A + row * P.lda + k0;
            if (vec && k0 + 4 <= P.n1) {
              t = __ldg(reinterpret_cast<const float4*>(src));
            } else {
              if (k0 + 0 < P.n1) t.x = __ldg(src + 0);
              if (k0 + 1 < P.n1) t.y = __ldg(src + 1);
              if (k0 + 2 < P.n1) t.z = __ldg(src + 2);
              if (k0 + 3 < P.n1) t.w = __ldg(src + 3);
            }
          }
          av[j][kq] = t;
        }
      }
      if (i >= S && !mbar_wait(emp(s), ((i / S) - 1) & 1)) {
        atomicExch(&g_tc_status, 9);
        *(volatile int*)abort_flag = 1;
      }
      if (*(volatile int*)abort_flag) break;
      float* sa = reinterpret_cast<float*>(smem + s * SB);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = lane + 32 * j;
#pragma unroll
        for (int kq = 0; kq < 2; ++kq) {
          const float4 t = av[j][kq];
          float4 h, l;
          h.x = tf32_rna(t.x); l.x = t.x - h.x;
          h.y = tf32_rna(t.y); l.y = t.y - h.y;
          h.z = tf32_rna(t.z); l.z = t.z - h.z;
          h.w = tf32_rna(t.w); l.w = t.w - h.w;
          const int o = k8_off(r, kq * 4);
          *reinterpret_cast<float4*>(sa + o) = h;
          *reinterpret_cast<float4*>(sa + TG_T * TG_KC + o) = l;
        }
      }
      // the pre-split U chunk (already in the operand layout): one bulk copy,
      // counted on the same barrier; issued after the stage is free and never
      // abandoned before this warp's arrivals, so the phase always completes
      if (lane == 0) {
        mbar_expect_tx(full(s), TG_UBYTES);
        bulk_g2s(smem_u32(sa + 2 * TG_T * TG_KC),
                 P.Us + ((int64_t)tj * nkc_all + i) * 2 * TG_T * TG_KC, TG_UBYTES, full(s));
        last_issued = i;
      }
      fence_proxy_async_smem();
      mbar_arrive(full(s));
    }
    // on an abort, wait (bounded) for this warp's last bulk copy before leaving
    if (lane == 0 && last_issued >= 0 && *(volatile int*)abort_flag)
      mbar_wait(full(last_issued % S), (last_issued / S) & 1);
    bool okacc = true;
    if (nk > 0) {
      okacc = mbar_wait(accb, 0);
      if (!okacc) atomicExch(&g_tc_status, 10);
    }
    tc_fence_after();
    const bool run = __all_sync(0xffffffffu, okacc && !*(volatile int*)abort_flag);
    // stage the 128 x 128 tile in shared memory (stage buffers are free), then
    // each warp writes whole rows with lanes over consecutive columns
    float* E = reinterpret_cast<float*>(smem);
    constexpr int EP = TG_T + 1;
    if (run) {
      for (int cb = 0; cb < bne; cb += 16) {
        float acc[16];
        __syncwarp();
        if (nk > 0) {
          tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + cb, acc);
          tmem_wait_ld();
        } else {
#pragma unroll
          for (int u = 0; u < 16; ++u) acc[u] = 0.f;
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) E[(warp * 32 + lane) * EP + cb + u] = acc[u];
      }
    }
    __syncwarp();
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if (run) {
      for (int r = warp; r < TG_T; r += 4) {
        const int64_t row = rb + r;
        if (row >= P.M) break;
        if (P.bd == 1) {   // the row's four diagonal-term loads issued together
          float a[4], v[4];
          float2 u[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = lane + 32 * q, col = tj * TG_T + c;
            const bool ok = c < ncv && col < P.n1;
            a[q] = ok ? __ldg(P.A + row * P.lda + col) : 0.f;
            u[q] = ok ? P.Ud[col] : make_float2(0.f, 0.f);
            v[q] = c < ncv ? E[r * EP + c] : 0.f;
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = lane + 32 * q;
            if (c < ncv) P.C[row * P.ldc + tj * TG_T + c] = tall_diag1(v[q], a[q], u[q]);
          }
          continue;
        }
        for (int c = lane; c < ncv; c += 32) {
          const int col = tj * TG_T + c;
          float v = E[r * EP + c];
          if (P.bd > 0) v = tall_diag_add(v, P.A + row * P.lda, P.Ud, col, P.bd, P.n1, P.upper);
          P.C[row * P.ldc + col] = v;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 4) tmem_dealloc(tmem, 128);
}

// kernel < 0: the 256-row kernel takes the tall products with at least two
// waves of its one-CTA-per-SM grid; 0 / 1 force the 128 x 128 / 256-row kernel.
bool tc_tall_use_wide(int64_t M, int n2, int kernel) {
  if (kernel >= 0) return kernel == 1;
  const int64_t ctas = (M + 255) / 256 * ((n2 + 255) / 256);
  return ctas >= 2 * 152;
}

// ----------------------------------------------------------------- tall GEMM, 256-row tiles
// The same product as tc_tall_kernel with a 256-row x BW-column CTA tile (BW
// <= 256, a multiple of 16, n2 split into equal column tiles): two TMEM
// accumulators (rows 0-127 at column 0, rows 128-255 at column 256; all 512
// columns, one CTA per SM) share every chunk of U, and every row block of A
// is read by ceil(n2 / 256) column tiles instead of ceil(n2 / 128), which
// halves the operand bytes each tensor-core flop pulls through L2.  Eight
// producer warps: warp w fills row half w & 1 of the chunks i = w >> 1
// (mod 4); the row-half-0 warp also issues the bulk copy of the chunk's
// pre-split U (layout as tc_splitu_kernel with tile width BW).  The epilogue
// (the same eight warps: TMEM lane quarter w % 4, accumulator w >> 2) reads
// its rows straight from TMEM and writes 16 consecutive columns per thread.
constexpr int TW_ROWS = 256, TW_PROD = 8, TW_THREADS = (TW_PROD + 1) * 32, TW_S = 6;
static_assert(TW_S >= 4, "parity waits of the 4 producer groups need at least 4 stages");

__host__ __device__ inline int tw_stage_bytes(int bw) { return TW_ROWS * TG_KC * 4 * 2 + bw * TG_KC * 4 * 2; }

// Column tiling of n2 for the 256-row kernel: ntile tiles of bw columns.
inline void tw_tiling(int n2, int& ntile, int& bw) {
  ntile = (n2 + 255) / 256;
  bw = ((n2 + ntile - 1) / ntile + 15) / 16 * 16;
}

// Bytes of the split U of either tall kernel (16-byte multiple).
inline size_t tall_split_bytes(int n1, int n2) {
  const int nkc = (n1 + TG_KC - 1) / TG_KC;
  const int ntile = (n2 + TG_T - 1) / TG_T;
  int ntw, bw;
  tw_tiling(n2, ntw, bw);
  const size_t narrow = (size_t)ntile * nkc * 2 * TG_T * TG_KC * 4;
  const size_t wide = (size_t)ntw * nkc * 2 * bw * TG_KC * 4;
  return (std::max(narrow, wide) + 15) / 16 * 16;
}

__global__ void tc_splitu_w_kernel(const double* __restrict__ U, int64_t ldu, int n1, int n2, int upper,
                                   int trans, int bd, int bw, float* __restrict__ out) {
  const int nkc = (n1 + TG_KC - 1) / TG_KC;
  const int64_t per_tile = (int64_t)nkc * bw * TG_KC;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int ntile = (n2 + bw - 1) / bw;
  if (idx >= (int64_t)ntile * per_tile) return;
  const int tile = (int)(idx / per_tile);
  int rem = (int)(idx - (int64_t)tile * per_tile);
  const int kc = rem / (bw * TG_KC);
  rem -= kc * bw * TG_KC;
  const int n = rem / TG_KC, k = rem % TG_KC;
  const int col = tile * bw + n, kk = kc * TG_KC + k;
  double v = 0.0;
  if (col < n2 && kk < n1 && (!upper || kk <= col) && !(bd > 0 && kk / bd == col / bd))
    v = trans ? U[col + (int64_t)kk * ldu] : U[kk + (int64_t)col * ldu];
  const float h = tf32_rna((float)v);
  const float l = tf32_rna((float)(v - (double)h));
  float* base = out + ((int64_t)tile * nkc + kc) * 2 * bw * TG_KC;
  base[k8_off(n, k)] = h;
  base[bw * TG_KC + k8_off(n, k)] = l;
}

__global__ void __launch_bounds__(TW_THREADS, 1) tc_tall_wide_kernel(TallParams P, int bw) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tj = blockIdx.x;
  const int64_t rb = (int64_t)blockIdx.y * TW_ROWS;
  const int nkc_all = (P.n1 + TG_KC - 1) / TG_KC;
  int kend = P.n1;
  if (P.upper) kend = min(P.n1, (tj + 1) * bw);
  const int nk = (kend + TG_KC - 1) / TG_KC;
  const int SB = tw_stage_bytes(bw);
  const uint32_t ubytes = (uint32_t)bw * TG_KC * 4 * 2;
  const int S = TW_S;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * SB);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  const uint32_t sbase = smem_u32(smem);
  auto full = [&](int s) { return smem_u32(bars + s); };
  auto emp = [&](int s) { return smem_u32(bars + S + s); };
  const uint32_t accb = smem_u32(bars + 2 * S);
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full(s), 64);
      mbar_init(emp(s), 1);
    }
    mbar_init(accb, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == TW_PROD) {
    tmem_alloc(smem_u32(tmem_slot), 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int ncv = min(bw, P.n2 - tj * bw);
  const int bne = (ncv + 15) / 16 * 16;

  if (warp == TW_PROD) {
    if (lane == 0 && nk > 0) {
      const uint32_t idesc = idesc_tf32(128, bne);
      for (int i = 0; i < nk; ++i) {
        const int s = i % S;
        if (!mbar_wait(full(s), (i / S) & 1) || *(volatile int*)abort_flag) {
          atomicExch(&g_tc_status, 11);
          *(volatile int*)abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t sa = sbase + s * SB;
        const uint32_t su = sa + TW_ROWS * TG_KC * 8;
        const uint64_t uh = umma_desc(su, 128, 256);
        const uint64_t ul = umma_desc(su + bw * TG_KC * 4, 128, 256);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t acc = tmem + h * 256;
          const uint32_t ah_a = sa + h * 128 * TG_KC * 4;
          const uint64_t ah = umma_desc(ah_a, 128, 256);
          const uint64_t al = umma_desc(ah_a + TW_ROWS * TG_KC * 4, 128, 256);
          if (P.split3) {
            mma_tf32(acc, al, uh, idesc, i > 0);
            mma_tf32(acc, ah, ul, idesc, 1);
            mma_tf32(acc, ah, uh, idesc, 1);
          } else {
            mma_tf32(acc, ah, uh, idesc, i > 0);
          }
        }
        umma_commit(emp(s));
      }
      umma_commit(accb);
    }
  } else {
    const bool vec = ((P.lda & 3) == 0) && ((reinterpret_cast<uintptr_t>(P.A) & 15) == 0);
    const int hw = warp & 1, grp = warp >> 1;
    int last_issued = -1;
    // rows hw*128 + lane + 32 j, K quads kq of chunk i, into registers
    auto load_chunk = [&](int i, float4 (&av)[4][2]) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t row = rb + hw * 128 + lane + 32 * j;
#pragma unroll
        for (int kq = 0; kq < 2; ++kq) {
          const int k0 = i * TG_KC + kq * 4;
          float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
          if (row < P.M) {
            const float* src = P.A + row * P.lda + k0;
            if (vec && k0 + 4 <= P.n1) {
              t = __ldg(reinterpret_cast<const float4*>(src));
            } else {
              if (k0 + 0 < P.n1) t.x = __ldg(src + 0);
              if (k0 + 1 < P.n1) t.y = __ldg(src + 1);
              if (k0 + 2 < P.n1) t.z = __ldg(src + 2);
              if (k0 + 3 < P.n1) t.w = __ldg(src + 3);
            }
          }
          av[j][kq] = t;
        }
      }
    };
    // wait for stage i % S, split the registers into it, add the U chunk, arrive
    auto fill_stage = [&](int i, const float4 (&av)[4][2]) -> bool {
      const int s = i % S;
      if (i >= S && !mbar_wait(emp(s), ((i / S) - 1) & 1)) {
        atomicExch(&g_tc_status, 12);
        *(volatile int*)abort_flag = 1;
      }
      if (*(volatile int*)abort_flag) return false;
      float* sa = reinterpret_cast<float*>(smem + s * SB);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = hw * 128 + lane + 32 * j;
#pragma unroll
        for (int kq = 0; kq < 2; ++kq) {
          const float4 t = av[j][kq];
          float4 h, l;
          h.x = tf32_rna(t.x); l.x = t.x - h.x;
          h.y = tf32_rna(t.y); l.y = t.y - h.y;
          h.z = tf32_rna(t.z); l.z = t.z - h.z;
          h.w = tf32_rna(t.w); l.w = t.w - h.w;
          const int o = k8_off(r, kq * 4);
          *reinterpret_cast<float4*>(sa + o) = h;
          *reinterpret_cast<float4*>(sa + TW_ROWS * TG_KC + o) = l;
        }
      }
      // the pre-split U chunk: one bulk copy on the same barrier, issued once
      // the stage is free and never abandoned before this warp's arrivals
      if (hw == 0 && lane == 0) {
        mbar_expect_tx(full(s), ubytes);
        bulk_g2s(smem_u32(sa + 2 * TW_ROWS * TG_KC),
                 P.Us + ((int64_t)tj * nkc_all + i) * 2 * bw * TG_KC, ubytes, full(s));
        last_issued = i;
      }
      fence_proxy_async_smem();
      mbar_arrive(full(s));
      return true;
    };
    // chunks grp, grp + 4, ...: the loads of the next chunk are in flight
    // while the current one is split (two register sets)
    float4 va[4][2], vb[4][2];
    if (grp < nk) load_chunk(grp, va);
    for (int i = grp; i < nk; i += 8) {
      const bool more = i + 4 < nk;
      if (more) load_chunk(i + 4, vb);
      if (!fill_stage(i, va) || !more) break;
      if (i + 8 < nk) load_chunk(i + 8, va);
      if (!fill_stage(i + 4, vb)) break;
    }
    if (lane == 0 && last_issued >= 0 && *(volatile int*)abort_flag)
      mbar_wait(full(last_issued % S), (last_issued / S) & 1);
    bool okacc = true;
    if (nk > 0) {
      okacc = mbar_wait(accb, 0);
      if (!okacc) atomicExch(&g_tc_status, 13);
    }
    tc_fence_after();
    const bool run = __all_sync(0xffffffffu, okacc && !*(volatile int*)abort_flag);
    const int q = warp & 3, h = warp >> 2;
    const int64_t row = rb + h * 128 + q * 32 + lane;
    const bool cvec = ((P.ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(P.C) & 15) == 0);
    for (int cb = 0; cb < bne; cb += 16) {
      float acc[16];
      __syncwarp();
      if (run && nk > 0) {
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + h * 256 + cb, acc);
        tmem_wait_ld();
      } else {
#pragma unroll
        for (int u = 0; u < 16; ++u) acc[u] = 0.f;
      }
      if (!run || row >= P.M) continue;
      const int c0 = tj * bw + cb;
      float out[16];
      if (P.bd == 1) {   // the 16 diagonal-term loads issued together
        float a[16];
        float2 ud[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int col = c0 + u;
          const bool ok = col < P.n2 && col < P.n1;
          a[u] = ok ? __ldg(P.A + row * P.lda + col) : 0.f;
          ud[u] = ok ? P.Ud[col] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) out[u] = tall_diag1(acc[u], a[u], ud[u]);
      } else {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int col = c0 + u;
          out[u] = acc[u];
          if (P.bd > 0 && col < P.n2)
            out[u] = tall_diag_add(acc[u], P.A + row * P.lda, P.Ud, col, P.bd, P.n1, P.upper);
        }
      }
      float* dst = P.C + row * P.ldc + c0;
      if (cvec && c0 + 16 <= tj * bw + ncv) {
#pragma unroll
        for (int u = 0; u < 16; u += 4)
          *reinterpret_cast<float4*>(dst + u) = make_float4(out[u], out[u + 1], out[u + 2], out[u + 3]);
      } else {
#pragma unroll
        for (int u = 0; u < 16; ++u)
          if (cb + u < ncv) dst[u] = out[u];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == TW_PROD) tmem_dealloc(tmem, 512);
}

cudaError_t tc_tallgemm_mixed(const float* A, int64_t lda, const double* U, int64_t ldu, int64_t M,
                              int n1, int n2, float* C, int64_t ldc, int upper, int trans,
                              int diag_block, int split3, void* work, cudaStream_t s, int kernel) {
  if (M == 0 || n2 == 0) return cudaSuccess;
  const int nkc = (n1 + TG_KC - 1) / TG_KC;
  const int ntile = (n2 + TG_T - 1) / TG_T;
  float* Us = (float*)work;
  float2* Ud = reinterpret_cast<float2*>((char*)work + tall_split_bytes(n1, n2));
  int bd = 0;
  if (diag_block > 0) {
    bd = 1;
    while (bd * 2 <= std::min(diag_block, 32)) bd *= 2;
    note_launch();
    tc_diagu_kernel<<<(unsigned)(((int64_t)n2 * bd + 255) / 256), 256, 0, s>>>(U, ldu, n1, n2, upper, trans,
                                                                               bd, Ud);
  }
  if (tc_tall_use_wide(M, n2, kernel)) {   // 256-row tiles
    int ntw, bw;
    tw_tiling(n2, ntw, bw);
    const int64_t totw = (int64_t)ntw * nkc * bw * TG_KC;
    note_launch();
    tc_splitu_w_kernel<<<(unsigned)((totw + 255) / 256), 256, 0, s>>>(U, ldu, n1, n2, upper, trans, bd, bw,
                                                                     Us);
    TallParams P{A, lda, M, Us, Ud, ldu, n1, n2, upper, trans, bd, split3, C, ldc};
    const int smem = TW_S * tw_stage_bytes(256) + 1024;
    static std::once_flag attrw;
    std::call_once(attrw, [&] {
      cudaFuncSetAttribute(tc_tall_wide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    });
    dim3 grid(ntw, (unsigned)((M + TW_ROWS - 1) / TW_ROWS));
    note_launch();
    tc_tall_wide_kernel<<<grid, TW_THREADS, TW_S * tw_stage_bytes(bw) + 1024, s>>>(P, bw);
    return cudaGetLastError();
  }
  const int64_t tot = (int64_t)ntile * nkc * TG_T * TG_KC;
  note_launch();
  tc_splitu_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(U, ldu, n1, n2, upper, trans, bd, Us);
  TallParams P{A, lda, M, Us, Ud, ldu, n1, n2, upper, trans, bd, split3, C, ldc};
  const int smem = TG_S * (2 * TG_T * TG_KC * 4 * 2) + 1024;
  static std::once_flag attr;
  std::call_once(attr, [&] {
    cudaFuncSetAttribute(tc_tall_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  });
  dim3 grid(ntile, (unsigned)((M + TG_T - 1) / TG_T));
  note_launch();
  tc_tall_kernel<<<grid, TG_THREADS, smem, s>>>(P);
  return cudaGetLastError();
}

size_t tc_tallgemm_work_bytes(int n1, int n2) {
  return tall_split_bytes(n1, n2) + (size_t)n2 * 32 * sizeof(float2) + 256;
}

// ----------------------------------------------------------------- nonlocal (binary32)
// Z[4 s + t][c] = sum over the support of site s of C~[s, j, t] Y[j][c].
// Block: one site x 128 columns, 8 warps; a lane owns 4 consecutive columns
// (16-byte loads).  Warp w takes the support entries w, w + 8, ...; four of
// them per step, with their unknown indices and rows loaded before the FMAs so
// four row gathers are in flight per lane.  Partial sums are combined in a
// fixed order (deterministic).
__global__ void __launch_bounds__(256) nl_project32_kernel(const int64_t* __restrict__ site_ptr,
                                                           const int32_t* __restrict__ site_dof,
                                                           const float* __restrict__ site_c,
                                                           const float* __restrict__ Y, int64_t ldy,
                                                           int ncol, int nsite,
                                                           float* __restrict__ Z) {
  // grid y strides over the sites; the column tiles of one site run together
  for (int s = blockIdx.y; s < nsite; s += gridDim.y) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int cb = blockIdx.x * 128;
  const int c0 = cb + lane * 4;
  const bool vec = ((ldy & 3) == 0) && ((reinterpret_cast<uintptr_t>(Y) & 15) == 0) && c0 + 4 <= ncol;
  float acc[4][4];
#pragma unroll
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[t][u] = 0.f;
  const int64_t e0 = site_ptr[s], e1 = site_ptr[s + 1];
  for (int64_t e = e0 + w; e < e1; e += 32) {
    int64_t row[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) row[q] = e + 8 * q < e1 ? (int64_t)site_dof[e + 8 * q] : -1;
    float y[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
      for (int u = 0; u < 4; ++u) y[q][u] = 0.f;
      if (row[q] < 0) continue;
      const float* src = Y + row[q] * ldy + c0;
      if (vec) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(src));
        y[q][0] = v.x; y[q][1] = v.y; y[q][2] = v.z; y[q][3] = v.w;
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (c0 + u < ncol) y[q][u] = __ldg(src + u);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (row[q] < 0) continue;
      const float4 cf = __ldg(reinterpret_cast<const float4*>(site_c) + (e + 8 * q));
      const float cq[4] = {cf.x, cf.y, cf.z, cf.w};
#pragma unroll
      for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[t][u] = fmaf(cq[t], y[q][u], acc[t][u]);
    }
  }
  __shared__ float red[8][4][128];
#pragma unroll
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int u = 0; u < 4; ++u) red[w][t][lane * 4 + u] = acc[t][u];
  __syncthreads();
  for (int o = threadIdx.x; o < 512; o += 256) {
    const int t = o >> 7, cc = o & 127;
    if (cb + cc >= ncol) continue;
    float v = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) v += red[q][t][cc];
    Z[(int64_t)(4 * s + t) * ncol + cb + cc] = v;
  }
  __syncthreads();   // red is reused by the next site
  }
}

cudaError_t tc_nl_project(const int64_t* site_ptr, const int32_t* site_dof, const float* site_c,
                          int nsite, const float* Y, int64_t ldy, int ncol, float* Z, cudaStream_t s) {
  if (nsite == 0 || ncol == 0) return cudaSuccess;
  note_launch();
  const unsigned gy = (unsigned)std::min(nsite, 65535);
  nl_project32_kernel<<<dim3((ncol + 127) / 128, gy), 256, 0, s>>>(site_ptr, site_dof, site_c, Y, ldy,
                                                                   ncol, nsite, Z);
  return cudaGetLastError();
}

}  // namespace chfsi
