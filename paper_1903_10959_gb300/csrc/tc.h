// Tensor-core (tcgen05, sm_103a) kernels of the mixed-precision path.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace chfsi {

// Device copies of the cell matrices for the tensor-core cell products.
struct TcCellData {
  float* hi = nullptr;     // TF32-rounded H~_e in the UMMA operand layout
  float* lo = nullptr;     // TF32-rounded residual H~_e - hi (same layout)
  size_t bytes = 0;        // bytes of each of hi / lo
  int64_t ncells = 0;
  int ne = 0, mt = 0, kt = 0;   // ne, row tiles of 128, K padded to a multiple of 8
  // BF16x3 copy (three bf16 terms per value), packed on first use
  uint16_t* bf = nullptr;
  size_t bf_bytes = 0;
  // FP16x2 copy (two fp16 terms of 2^s_e H~_e per value) and the per-cell
  // inverse scales 2^-s_e (float), packed on first use; f16_bytes covers both
  uint16_t* f16 = nullptr;
  float* f16_inv = nullptr;
  size_t f16_bytes = 0;
  // projector expansion as extra BF16x3 K-chunks per cell (NlCells layout),
  // packed on first use; nl_bytes covers the three arrays
  uint16_t* nl = nullptr;
  int32_t* nl_off = nullptr;       // ncells + 1 chunk offsets
  int32_t* nl_zrow = nullptr;      // 16 rows of Z per chunk (-1: padding)
  size_t nl_bytes = 0;
  // the projection Z = C~^T Y as per-cell BF16x3 blocks (NlCells::np / poff /
  // prow) and the per-site reduction lists; packed with the chunks above
  uint16_t* pj = nullptr;
  int32_t* pj_np = nullptr;
  int64_t* pj_off = nullptr;
  int64_t* pj_row = nullptr;
  int32_t* pj_red_ptr = nullptr;
  int64_t* pj_red_row = nullptr;
  int64_t pj_rows = 0;             // rows of the partial array
  int pj_npmax = 0;
  size_t pj_bytes = 0;
};

// Owner-computes form of one H~ Y step (no colouring): every cell writes its
// dense block R_e = H~_e Y_e (ne x ncol rows at R[(e * ne + l) * ncol]) with
// plain stores, then each unknown sums its 1..8 cell rows in ascending cell
// order and applies Y_out = alpha (sum + NL - shift Y_in) + beta Y_prev.
struct TcApplyArgs {
  const int32_t* dofmap;
  int64_t ncells;
  int ncol;
  const float* Yin;
  int64_t ld_in;
  float* R;                 // ncells * ne * ncol scratch
  int split3;
  int tile = 64;            // columns per CTA of the cell kernel: 64 or 128
  int gather = 2;           // BF16x3: 2 = decoupled matrix / Y rings, 0 = one shared ring, 1 = rows staged by
                            // bulk async copies (when aligned), 3 = rings with four gather warp pairs
  // BF16x3 ring kernels: when set, each cell's K loop continues over its
  // projector chunks (TcCellData::nl) with the rows of Z as the gathered
  // operand, so R holds H~_loc Y plus the owned rows' share of C~ h Z
  const float* Z = nullptr;
  int64_t ldz = 0;
  // Bloch term (complex blocks as (real, imaginary) column pairs): the shared
  // BF16x3 block of G~ = M^{-1/2} (k.G_e) M^{-1/2}; the cell data then holds
  // T~_e = H~_e + 1/2 |k|^2 M^{-1/2} A_e M^{-1/2}
  const uint16_t* kG = nullptr;
};
// Whether tc_cell_bf16_launch can add the projector chunks for this gather mode.
inline bool tc_cell_bf16_nl_ok(int gather) { return gather == 2 || gather == 3; }
// BF16x3 terms of ncells n_e x n_e binary64 matrices (plus add, an n_e x n_e
// matrix added to each, when not null) into *out (allocated on first use,
// *bytes set), in the packed cell-matrix layout.
cudaError_t tc_pack_bf16_matrices(const double* dH, const double* dadd, int64_t ncells, int ne, uint16_t** out,
                                  size_t* bytes, cudaStream_t s);
// Pack the projection blocks of build_nl_cells into d.pj (and its tables).
cudaError_t tc_pack_proj(TcCellData& d, int64_t ncells, int nsite, const int32_t* np, const int64_t* poff,
                         const int64_t* prow, const int32_t* red_ptr, const int64_t* red_row,
                         const int64_t* pz_pos, const double* pz_val, int64_t nnz, cudaStream_t s,
                         int64_t* dev_bytes);
// Z (4 nsite x ncol, row stride ncol) = C~^T Y by the projection blocks on the
// tensor cores: per cell the partial sums of its owned rows (a ring-kernel
// launch into part, pj_rows x ncol), then the per-site sums in a fixed order.
cudaError_t tc_nl_project_cells(const TcCellData& d, const int32_t* dofmap, int64_t ncells, int nsite,
                                const float* Y, int64_t ldy, int ncol, float* part, float* Z, cudaStream_t s);
// Pack the projector chunks (from build_nl_cells: nnz entries at nz_pos) into d.nl.
cudaError_t tc_pack_nl(TcCellData& d, const int32_t* chunk_off, int64_t ncells, const int32_t* zrow,
                       const int64_t* nz_pos, const double* nz_val, int64_t nnz, cudaStream_t s,
                       int64_t* dev_bytes);
cudaError_t tc_cell_r_launch(const TcCellData& d, const TcApplyArgs& a, cudaStream_t s);

// One system of a batched filter (device array, one entry per system).
struct TcBatchSys {
  const float* A;          // split cell matrices (tc_pack layout)
  const int32_t* dofmap;
  const float* Y[2];       // recurrence buffers: Y[0] = caller block, Y[1] = scratch
  int64_t ldY[2];
  float* R;                // dense cell blocks, ncells * ne rows of stride ldr
  int64_t ldr;             // ncol rounded up to a multiple of 4 (16-byte rows)
  const int32_t* node_ptr;
  const int32_t* node_ent;
  int64_t ncells, M;
  int ncol, tiles;         // tiles: 64-column tiles (multi-system kernel) or BN tiles
  int64_t item0;           // first (cell, tile) item of this system
  int64_t q0;              // first (unknown, column quad) of this system
};
// The cell kernel over the (cell, 64-column tile) items of every system of a
// batch in one launch (items of system s start at sys[s].item0, tiles fastest);
// Y[parity] of each system is the input.  All systems share n_e / mt / nk.
cudaError_t tc_cell_multi_launch(const TcBatchSys* d_sys, int nsys, int64_t nitems, int ne, int mt,
                                 int nk, int split3, int parity, cudaStream_t s);
// The BF16x3 cell kernel over the (cell, 128-column tile, row part) items of
// every system (A = each system's packed BF16x3 copy, tiles = column tiles x
// tc_bf16_parts(ne)); Y[parity] is the input.
cudaError_t tc_cell_bf16_multi_launch(const TcBatchSys* d_sys, int nsys, int64_t nitems, int ne, int mt,
                                      int parity, cudaStream_t s);
int tc_bf16_parts(int ne);
// Set the cell kernels' shared-memory attributes (before any stream capture).
void tc_cell_prepare();
// Owner-computes assembly fused with the Chebyshev update:
// Yout = alpha (sum_cells R + H~_nl Y - shift Yin) + beta Yprev (Yprev may be null).
struct AssembleParams {
  const int32_t* node_ptr;    // unknown -> rows of R (CSR, ascending cell order)
  const int32_t* node_ent;
  int64_t M;
  int ncol;
  const float* R;             // dense cell blocks, (cell, local node) rows x ncol
  const float* Yin;
  int64_t ld_in;
  float* Yout;
  int64_t ld_out;
  const float* Yprev;
  int64_t ld_prev;
  const int64_t* dof_ptr;     // projector expansion (when Z != null): unknown -> sites
  const int32_t* dof_site;
  const float* dof_c;         // 4 h-scaled coefficients per entry
  const float* Z;             // projected block, (4 nsite) x ncol
  float alpha, beta, shift;
  int vec, vin, vprev, vout;  // set by the launcher
};
cudaError_t tc_assemble_launch(const AssembleParams& P, cudaStream_t s);
// The same update with the column maxima of |Y_out| as a by-product: cmax
// (ncol words, the bits of non-negative binary32 values) is zeroed and filled.
cudaError_t tc_assemble_cmax_launch(const AssembleParams& P, uint32_t* cmax, cudaStream_t s);
// Column maxima of |Y| (M x ncol, leading dimension ld) into cmax (zeroed first).
cudaError_t tc_colmax_launch(const float* Y, int64_t ld, int64_t M, int ncol, uint32_t* cmax,
                             cudaStream_t s);
// FP16x2 cell kernel: as tc_cell_bf16_launch with two fp16 terms per operand,
// the block's columns scaled by powers of two from cmax (column maxima of Yin).
cudaError_t tc_cell_f16_launch(const TcCellData& d, const TcApplyArgs& a, const uint32_t* cmax,
                               cudaStream_t s);
cudaError_t tc_pack_f16_from_device(TcCellData& d, const double* dHt, cudaStream_t s,
                                    int64_t* dev_bytes);

cudaError_t tc_build(TcCellData& d, const std::vector<double>& Ht, int64_t ncells, int ne,
                     cudaStream_t s, int64_t* dev_bytes);
// Split the binary64 device cell matrices into three bf16 terms (BF16x3 layout).
cudaError_t tc_pack_bf16_from_device(TcCellData& d, const double* dHt, cudaStream_t s,
                                     int64_t* dev_bytes);
// The BF16x3 cell kernel (same contract as tc_cell_r_launch, 64-column tiles).
cudaError_t tc_cell_bf16_launch(const TcCellData& d, const TcApplyArgs& a, cudaStream_t s);
// Split the binary64 device cell matrices into the TF32 hi / lo operand layout.
cudaError_t tc_pack_from_device(TcCellData& d, const double* dHt, cudaStream_t s,
                                int64_t* dev_bytes);
// Read and clear the device status word of the bounded waits (0: no timeout).
int tc_read_status(cudaStream_t s);
// Test hook: withhold one gather arrival in the BF16x3 cell kernel (see kernels_tc.cu).
cudaError_t tc_set_withhold(int on, cudaStream_t s);
size_t tc_tallgemm_work_bytes(int n1, int n2);
void tc_free(TcCellData& d);
size_t tc_gram_partial_bytes(int64_t M, int n1, int n2);
cudaError_t tc_gram_mixed(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t M,
                          int n1, int n2, double* C, int64_t ldc, int lower, int diag_block,
                          int split3, void* partial, size_t partial_bytes, cudaStream_t s);
// kernel: -1 chooses by size, 0 the 128 x 128 tile kernel, 1 the 256-row tile kernel.
cudaError_t tc_tallgemm_mixed(const float* A, int64_t lda, const double* U, int64_t ldu, int64_t M,
                              int n1, int n2, float* C, int64_t ldc, int upper, int trans,
                              int diag_block, int split3, void* work, cudaStream_t s, int kernel = -1);
cudaError_t tc_nl_project(const int64_t* site_ptr, const int32_t* site_dof, const float* site_c,
                          int nsite, const float* Y, int64_t ldy, int ncol, float* Z,
                          cudaStream_t s);
}  // namespace chfsi
