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
};
cudaError_t tc_cell_r_launch(const TcCellData& d, const TcApplyArgs& a, cudaStream_t s);
cudaError_t tc_assemble_launch(const int32_t* node_ptr, const int32_t* node_ent, int64_t M,
                               int ncol, const float* R, const float* Yin, int64_t ld_in,
                               float* Yout, int64_t ld_out, const float* Yprev, int64_t ld_prev,
                               const float* NL, int64_t ld_nl, float alpha, float beta,
                               float shift, cudaStream_t s);

cudaError_t tc_build(TcCellData& d, const std::vector<double>& Ht, int64_t ncells, int ne,
                     cudaStream_t s, int64_t* dev_bytes);
// Split the binary64 device cell matrices into the TF32 hi / lo operand layout.
cudaError_t tc_pack_from_device(TcCellData& d, const double* dHt, cudaStream_t s,
                                int64_t* dev_bytes);
// Read and clear the device status word of the bounded waits (0: no timeout).
int tc_read_status(cudaStream_t s);
size_t tc_tallgemm_work_bytes(int n1, int n2);
void tc_free(TcCellData& d);
size_t tc_gram_partial_bytes(int64_t M, int n1, int n2);
cudaError_t tc_gram_mixed(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t M,
                          int n1, int n2, double* C, int64_t ldc, int lower, int diag_block,
                          int split3, void* partial, size_t partial_bytes, cudaStream_t s);
cudaError_t tc_tallgemm_mixed(const float* A, int64_t lda, const double* U, int64_t ldu, int64_t M,
                              int n1, int n2, float* C, int64_t ldc, int upper, int trans,
                              int diag_block, int split3, void* work, cudaStream_t s);
cudaError_t tc_nl_project(const int64_t* site_ptr, const int32_t* site_dof, const float* site_c,
                          int nsite, const float* Y, int64_t ldy, int ncol, float* Z,
                          cudaStream_t s);
cudaError_t tc_nl_expand(const int64_t* dof_ptr, const int32_t* dof_site, const float* dof_c,
                         int64_t M, const float* Z, int ncol, float* NL, int64_t ldn,
                         cudaStream_t s);

}  // namespace chfsi
