// ChFSI for a Bloch wavevector k (Eq. evp of the periodic problem, Sec. 2.1 of
// arXiv:1903.10959): the cell-periodic parts u of the Bloch states solve
// (-1/2 lap - i k.grad + 1/2 |k|^2 + V) u = eps u in the periodic box, so
// H~(k) = M^{-1/2} H(k) M^{-1/2} is complex Hermitian.  Blocks are complex,
// stored as interleaved (real, imaginary) binary64 column pairs: vector v at
// unknown j is X[j ldx + 2v] + i X[j ldx + 2v + 1].
//
//  apply   : the matrix-free Bloch cell kernel (kernels_mf.cu), colour by
//            colour, fused with the recurrence of Eq. chebFilter.
//  Gram    : X^H Y from the real Gram of the interleaved blocks,
//            (X^H Y)_ab = (G_{2a,2b} + G_{2a+1,2b+1}) + i (G_{2a,2b+1} - G_{2a+1,2b}).
//  CholGS  : S = X^H X = L L^H (cuSOLVER zpotrf), L^{-1} (ztrtri), X <- X L^{-H}
//            (Algorithm CholGS), the complex rotation as one real product
//            with the 2n x 2n real form of L^{-H} (upper triangular).
//  RR      : H^ = X^H H~ X, H^ Q = Q D (zheevd, ascending), X <- X Q (Sec. 3.5).
//  bounds  : k-step Lanczos on the real 2M-dimensional form of H~(k) (same
//            spectrum, each value twice).
//  mixed   : the filter on binary32 column pairs with BF16x3 cell products:
//            T~_e = H~_e + 1/2 |k|^2 A~ on both columns of a pair, and one
//            shared block G~ = M^{-1/2} (k.G) M^{-1/2} on the swapped pair
//            (re, im) -> (im, -re), in one ring-kernel launch per step; the
//            uniform periodic mesh gives every cell the same A~ and G~.
//            CholGS / RR stay binary64 on the binary64 block.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuComplex.h>
#include <cusolverDn.h>

#include "ctx.h"

using namespace chfsi;

namespace {

chfsi_status kfail(chfsi_ctx* ctx, chfsi_status st, const std::string& m) {
  ctx->err = m;
  if (st == CHFSI_ERR_CUDA) ctx->latched = st;
  return st;
}

#define KK(call)                                                                                 \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return kfail(ctx, CHFSI_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define KS(call)                                                                                 \
  do {                                                                                           \
    cusolverStatus_t s_ = (call);                                                                \
    if (s_ != CUSOLVER_STATUS_SUCCESS)                                                           \
      return kfail(ctx, CHFSI_ERR_CUDA, std::string(#call) + ": cusolver status " + std::to_string((int)s_)); \
  } while (0)

chfsi_status kgrow(chfsi_ctx* ctx, DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes) return CHFSI_OK;
  if (b.ptr) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(b.ptr);
    ctx->dev_bytes -= (int64_t)b.bytes;
  }
  b.ptr = nullptr;
  b.bytes = 0;
  if (cudaMalloc(&b.ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    return kfail(ctx, CHFSI_ERR_OOM, "k-point buffers: device allocation of " + std::to_string(bytes) + " bytes");
  }
  b.bytes = bytes;
  ctx->dev_bytes += (int64_t)bytes;
  return CHFSI_OK;
}

// complex (column-major, n1 x n2) from the real Gram (column-major, 2n1 x 2n2)
__global__ void gram_to_complex_kernel(const double* G, int ldg, int n1, int n2, cuDoubleComplex* C, int ldc) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n1 * n2) return;
  const int a = (int)(idx % n1), b = (int)(idx / n1);
  const double rr = G[(2 * a) + (int64_t)(2 * b) * ldg], ii = G[(2 * a + 1) + (int64_t)(2 * b + 1) * ldg];
  const double ri = G[(2 * a) + (int64_t)(2 * b + 1) * ldg], ir = G[(2 * a + 1) + (int64_t)(2 * b) * ldg];
  C[a + (int64_t)b * ldc] = make_cuDoubleComplex(rr + ii, ri - ir);
}

// Real 2n x 2n form (column-major) of the complex n x n matrix U acting on
// interleaved columns: new_b = sum_a x_a U_ab.  from_linv: U = L^{-H} read from
// the lower triangle of L^{-1} (U_ab = conj(Linv_ba) for a <= b, 0 below).
__global__ void real_form_kernel(const cuDoubleComplex* U, int ldu, int n, int from_linv, double* R) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int a = (int)(idx % n), b = (int)(idx / n);
  double ur = 0.0, ui = 0.0;
  if (from_linv) {
    if (a <= b) {
      const cuDoubleComplex l = U[b + (int64_t)a * ldu];
      ur = l.x;
      ui = -l.y;
    }
  } else {
    const cuDoubleComplex u = U[a + (int64_t)b * ldu];
    ur = u.x;
    ui = u.y;
  }
  const int64_t ld = 2 * (int64_t)n;
  R[(2 * a) + (2 * b) * ld] = ur;
  R[(2 * a + 1) + (2 * b) * ld] = -ui;
  R[(2 * a) + (2 * b + 1) * ld] = ui;
  R[(2 * a + 1) + (2 * b + 1) * ld] = ur;
}

__global__ void kaxpy2_kernel(double* w, const double* v, const double* vp, int64_t n, double a, double b) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) w[i] = fma(a, v[i], fma(b, vp[i], w[i]));
}
__global__ void kscal_kernel(double* v, const double* w, int64_t n, double s) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) v[i] = s * w[i];
}

unsigned kblk(int64_t n) { return (unsigned)((n + 255) / 256); }

chfsi_status kcheck(chfsi_ctx* ctx) {
  if (!ctx) return CHFSI_ERR_ARG;
  if (ctx->latched != CHFSI_OK) return ctx->latched;
  if (!ctx->kset) return kfail(ctx, CHFSI_ERR_STATE, "chfsi_set_kpoint has not been called");
  if (!ctx->built || !ctx->d_wv) return kfail(ctx, CHFSI_ERR_STATE, "the context has no potential (chfsi_build)");
  if (ctx->hproj.nsite > 0) return kfail(ctx, CHFSI_ERR_ARG, "projector Bloch phases are not modelled");
  return CHFSI_OK;
}

// Y = alpha (H~(k) Yin - shift Yin) + beta Yprev on nvec complex vectors.
chfsi_status kapply(chfsi_ctx* ctx, const double* Yin, int64_t ld_in, double* Yout, int64_t ld_out,
                    const double* Yprev, int64_t ld_prev, int nvec, double alpha, double beta, double shift) {
  const HostMesh& m = ctx->mesh;
  const int ncol = 2 * nvec;
  chfsi_status st;
  if ((st = kgrow(ctx, ctx->kW, (size_t)m.ndofs * ncol * 8)) != CHFSI_OK) return st;
  const int ncolour = (int)m.colour_offsets.size() - 1;
  for (int c = 0; c < ncolour; ++c) {
    MfLaunch L{};
    L.fac = ctx->d_kfac;
    L.wv = ctx->d_wv;
    L.minv_sqrt = ctx->d_msq;
    L.dofmap = ctx->d_dofmap;
    L.modes = ctx->d_modes;
    L.cells = ctx->d_cells + m.colour_offsets[c];
    L.ncells_colour = m.colour_offsets[c + 1] - m.colour_offsets[c];
    L.p = m.p;
    L.q = m.q;
    L.ncol = ncol;
    L.ld_in = ld_in;
    L.ld_out = ld_out;
    L.ld_prev = ld_prev;
    L.ld_w = ncol;
    KK(launch_mfk_cell_fp64(L, Yin, Yout, Yprev, (double*)ctx->kW.ptr, FilterStep{alpha, beta, shift},
                            ctx->stream));
  }
  return CHFSI_OK;
}

chfsi_status kfilter(chfsi_ctx* ctx, double* X, int64_t ldx, int n, int degree, double a, double b, double a0) {
  const HostMesh& m = ctx->mesh;
  chfsi_status st;
  if ((st = kgrow(ctx, ctx->kT1, (size_t)m.ndofs * 2 * n * 8)) != CHFSI_OK) return st;
  const double e = (b - a) / 2.0, c = (b + a) / 2.0, s1 = e / (a0 - c);
  double* bufs[2] = {X, (double*)ctx->kT1.ptr};
  int64_t lds[2] = {ldx, 2 * (int64_t)n};
  int cur = 0;
  double sig = s1;
  for (int k = 1; k <= degree; ++k) {
    double alpha, beta;
    if (k == 1) {
      alpha = s1 / e;
      beta = 0.0;
    } else {
      const double sn = 1.0 / (2.0 / s1 - sig);
      alpha = 2.0 * sn / e;
      beta = -sig * sn;
      sig = sn;
    }
    const int nxt = 1 - cur;
    if ((st = kapply(ctx, bufs[cur], lds[cur], bufs[nxt], lds[nxt], bufs[nxt], lds[nxt], n, alpha, beta, c)) != CHFSI_OK)
      return st;
    cur = nxt;
  }
  if (cur == 1)
    KK(cudaMemcpy2DAsync(X, ldx * 8, ctx->kT1.ptr, 2 * (size_t)n * 8, 2 * (size_t)n * 8, m.ndofs,
                         cudaMemcpyDeviceToDevice, ctx->stream));
  return CHFSI_OK;
}

// Pack the mixed-path blocks for the current k (after a rebuild or a new k).
chfsi_status kpack_mixed(chfsi_ctx* ctx) {
  if (ctx->kpack_valid) return CHFSI_OK;
  const HostMesh& m = ctx->mesh;
  if (!ctx->d_kA || !ctx->d_kG)
    return kfail(ctx, CHFSI_ERR_ARG, "mixed k-points need every cell to share the M^{-1/2} pattern");
  if (!ctx->d_Ht) return kfail(ctx, CHFSI_ERR_STATE, "no cell matrices (device-side potential)");
  const bool fresh_a = !ctx->kbf, fresh_g = !ctx->kgbf;
  KK(tc_pack_bf16_matrices(ctx->d_Ht, ctx->d_kA, m.ncells, m.ne, &ctx->kbf, &ctx->kbf_bytes, ctx->stream));
  KK(tc_pack_bf16_matrices(ctx->d_kG, nullptr, 1, m.ne, &ctx->kgbf, &ctx->kgbf_bytes, ctx->stream));
  if (fresh_a) ctx->dev_bytes += (int64_t)ctx->kbf_bytes;
  if (fresh_g) ctx->dev_bytes += (int64_t)ctx->kgbf_bytes;
  ctx->kpack_valid = true;
  return CHFSI_OK;
}

// Mixed Bloch step on binary32 column pairs (ld in floats, nvec complex vectors):
// Y = alpha (H~(k) Yin - shift Yin) + beta Yprev.
chfsi_status kapply_mixed(chfsi_ctx* ctx, const float* Yin, int64_t ld_in, float* Yout, int64_t ld_out,
                          const float* Yprev, int64_t ld_prev, int nvec, double alpha, double beta,
                          double shift) {
  const HostMesh& m = ctx->mesh;
  const int ncol = 2 * nvec;
  chfsi_status st;
  if ((st = kgrow(ctx, ctx->kY, (size_t)m.ncells * m.ne * ncol * 4)) != CHFSI_OK) return st;
  TcCellData view = ctx->tc;
  view.bf = ctx->kbf;
  TcApplyArgs ra{};
  ra.dofmap = ctx->d_dofmap;
  ra.ncells = m.ncells;
  ra.ncol = ncol;
  ra.Yin = Yin;
  ra.ld_in = ld_in;
  ra.R = (float*)ctx->kY.ptr;
  ra.split3 = 1;
  ra.gather = 2;
  ra.kG = ctx->kgbf;
  KK(tc_cell_bf16_launch(view, ra, ctx->stream));
  AssembleParams ap{};
  ap.node_ptr = ctx->d_node_ptr;
  ap.node_ent = ctx->d_node_ent;
  ap.M = m.ndofs;
  ap.ncol = ncol;
  ap.R = (const float*)ctx->kY.ptr;
  ap.Yin = Yin;
  ap.ld_in = ld_in;
  ap.Yout = Yout;
  ap.ld_out = ld_out;
  ap.Yprev = beta != 0.0 ? Yprev : nullptr;
  ap.ld_prev = ld_prev;
  ap.alpha = (float)alpha;
  ap.beta = (float)beta;
  ap.shift = (float)shift;
  KK(tc_assemble_launch(ap, ctx->stream));
  return CHFSI_OK;
}

// The Chebyshev filter (Eq. chebFilter) of a binary32 block of column pairs.
chfsi_status kfilter_mixed(chfsi_ctx* ctx, float* X, int64_t ldx, int n, int degree, double a, double b,
                           double a0) {
  const HostMesh& m = ctx->mesh;
  chfsi_status st;
  if ((st = kpack_mixed(ctx)) != CHFSI_OK) return st;
  if ((st = kgrow(ctx, ctx->kwork, (size_t)m.ndofs * 2 * n * 4)) != CHFSI_OK) return st;
  const double e = (b - a) / 2.0, c = (b + a) / 2.0, s1 = e / (a0 - c);
  float* bufs[2] = {X, (float*)ctx->kwork.ptr};
  int64_t lds[2] = {ldx, 2 * (int64_t)n};
  int cur = 0;
  double sig = s1;
  for (int k = 1; k <= degree; ++k) {
    double alpha, beta;
    if (k == 1) {
      alpha = s1 / e;
      beta = 0.0;
    } else {
      const double sn = 1.0 / (2.0 / s1 - sig);
      alpha = 2.0 * sn / e;
      beta = -sig * sn;
      sig = sn;
    }
    const int nxt = 1 - cur;
    if ((st = kapply_mixed(ctx, bufs[cur], lds[cur], bufs[nxt], lds[nxt], bufs[nxt], lds[nxt], n, alpha, beta,
                           c)) != CHFSI_OK)
      return st;
    cur = nxt;
  }
  if (cur == 1)
    KK(cudaMemcpy2DAsync(X, ldx * 4, ctx->kwork.ptr, 2 * (size_t)n * 4, 2 * (size_t)n * 4, m.ndofs,
                         cudaMemcpyDeviceToDevice, ctx->stream));
  return CHFSI_OK;
}

// C (n1 x n2 complex, column-major, ld n1) = A^H B over the unknowns.
chfsi_status kgram(chfsi_ctx* ctx, const double* A, int64_t lda, const double* B, int64_t ldb, int n1,
                   int n2, cuDoubleComplex* C) {
  const HostMesh& m = ctx->mesh;
  chfsi_status st;
  const size_t gbytes = (size_t)4 * n1 * n2 * 8;
  const size_t pbytes = (size_t)8 * 8 * 4 * n1 * n2;
  if ((st = kgrow(ctx, ctx->kG, gbytes + pbytes)) != CHFSI_OK) return st;
  double* G = (double*)ctx->kG.ptr;
  KK(launch_gram_fp64(A, lda, B, ldb, m.ndofs, 2 * n1, 2 * n2, G, 2 * n1, 0, G + 4 * (size_t)n1 * n2,
                      pbytes, ctx->stream));
  note_launch();
  gram_to_complex_kernel<<<kblk((int64_t)n1 * n2), 256, 0, ctx->stream>>>(G, 2 * n1, n1, n2, C, n1);
  KK(cudaGetLastError());
  return CHFSI_OK;
}

// X <- X R (R: 2n x 2n real form, column-major), through the tall-GEMM kernel.
chfsi_status krotate(chfsi_ctx* ctx, double* X, int64_t ldx, int n, const double* R, int upper) {
  const HostMesh& m = ctx->mesh;
  chfsi_status st;
  if ((st = kgrow(ctx, ctx->kT1, (size_t)m.ndofs * 2 * n * 8)) != CHFSI_OK) return st;
  double* T = (double*)ctx->kT1.ptr;
  KK(launch_tallgemm_fp64(X, ldx, R, 2 * n, m.ndofs, 2 * n, 2 * n, T, 2 * n, upper, 0, ctx->stream));
  KK(cudaMemcpy2DAsync(X, ldx * 8, T, 2 * (size_t)n * 8, 2 * (size_t)n * 8, m.ndofs,
                       cudaMemcpyDeviceToDevice, ctx->stream));
  return CHFSI_OK;
}

chfsi_status ksolver(chfsi_ctx* ctx) {
  if (!ctx->sol) {
    KS(cusolverDnCreate(&ctx->sol));
  }
  KS(cusolverDnSetStream(ctx->sol, ctx->stream));
  return CHFSI_OK;
}

chfsi_status kcholgs(chfsi_ctx* ctx, double* X, int64_t ldx, int n) {
  chfsi_status st;
  if ((st = ksolver(ctx)) != CHFSI_OK) return st;
  if ((st = kgrow(ctx, ctx->kS, (size_t)n * n * 16 + (size_t)4 * n * n * 8 + 64)) != CHFSI_OK) return st;
  cuDoubleComplex* S = (cuDoubleComplex*)ctx->kS.ptr;
  double* R = (double*)(S + (size_t)n * n);
  int* dinfo = (int*)(R + (size_t)4 * n * n);
  if ((st = kgram(ctx, X, ldx, X, ldx, n, n, S)) != CHFSI_OK) return st;
  int lw = 0;
  KS(cusolverDnZpotrf_bufferSize(ctx->sol, CUBLAS_FILL_MODE_LOWER, n, S, n, &lw));
  size_t dws = 0, hws = 0;
  KS(cusolverDnXtrtri_bufferSize(ctx->sol, CUBLAS_FILL_MODE_LOWER, CUBLAS_DIAG_NON_UNIT, n, CUDA_C_64F, S, n,
                                 &dws, &hws));
  if ((st = kgrow(ctx, ctx->kwork, std::max<size_t>((size_t)lw * 16, dws) + 256)) != CHFSI_OK) return st;
  KS(cusolverDnZpotrf(ctx->sol, CUBLAS_FILL_MODE_LOWER, n, S, n, (cuDoubleComplex*)ctx->kwork.ptr, lw, dinfo));
  int info = 0;
  KK(cudaMemcpyAsync(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  KK(cudaStreamSynchronize(ctx->stream));
  if (info != 0) return kfail(ctx, CHFSI_ERR_NOT_SPD, "k-point CholGS: zpotrf info = " + std::to_string(info));
  std::vector<char> hwork(hws + 16);
  KS(cusolverDnXtrtri(ctx->sol, CUBLAS_FILL_MODE_LOWER, CUBLAS_DIAG_NON_UNIT, n, CUDA_C_64F, S, n,
                      ctx->kwork.ptr, dws, hwork.data(), hws, dinfo));
  KK(cudaMemcpyAsync(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  KK(cudaStreamSynchronize(ctx->stream));
  if (info != 0) return kfail(ctx, CHFSI_ERR_NOT_SPD, "k-point CholGS: trtri info = " + std::to_string(info));
  note_launch();
  real_form_kernel<<<kblk((int64_t)n * n), 256, 0, ctx->stream>>>(S, n, n, 1, R);
  KK(cudaGetLastError());
  return krotate(ctx, X, ldx, n, R, 1);
}

chfsi_status krr(chfsi_ctx* ctx, double* X, int64_t ldx, int n, double* evals) {
  const HostMesh& m = ctx->mesh;
  chfsi_status st;
  if ((st = ksolver(ctx)) != CHFSI_OK) return st;
  if ((st = kgrow(ctx, ctx->kS, (size_t)n * n * 16 + (size_t)4 * n * n * 8 + 64)) != CHFSI_OK) return st;
  if ((st = kgrow(ctx, ctx->kY, (size_t)m.ndofs * 2 * n * 8 + (size_t)n * 8 + 64)) != CHFSI_OK) return st;
  cuDoubleComplex* Hh = (cuDoubleComplex*)ctx->kS.ptr;
  double* R = (double*)(Hh + (size_t)n * n);
  int* dinfo = (int*)(R + (size_t)4 * n * n);
  double* Y = (double*)ctx->kY.ptr;
  double* D = Y + (size_t)m.ndofs * 2 * n;
  if ((st = kapply(ctx, X, ldx, Y, 2 * n, nullptr, 0, n, 1.0, 0.0, 0.0)) != CHFSI_OK) return st;
  if ((st = kgram(ctx, X, ldx, Y, 2 * n, n, n, Hh)) != CHFSI_OK) return st;
  int lw = 0;
  KS(cusolverDnZheevd_bufferSize(ctx->sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, Hh, n, D, &lw));
  if ((st = kgrow(ctx, ctx->kwork, (size_t)lw * 16 + 256)) != CHFSI_OK) return st;
  KS(cusolverDnZheevd(ctx->sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, Hh, n, D,
                      (cuDoubleComplex*)ctx->kwork.ptr, lw, dinfo));
  int info = 0;
  KK(cudaMemcpyAsync(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  KK(cudaMemcpyAsync(evals, D, (size_t)n * 8, cudaMemcpyDeviceToHost, ctx->stream));
  KK(cudaStreamSynchronize(ctx->stream));
  if (info != 0) return kfail(ctx, CHFSI_ERR_EIG, "k-point RR: zheevd info = " + std::to_string(info));
  note_launch();
  real_form_kernel<<<kblk((int64_t)n * n), 256, 0, ctx->stream>>>(Hh, n, n, 0, R);
  KK(cudaGetLastError());
  return krotate(ctx, X, ldx, n, R, 0);
}

}  // namespace

extern "C" {

chfsi_status chfsi_set_kpoint(chfsi_ctx* ctx, const double* k) {
  if (!ctx || !k) return CHFSI_ERR_ARG;
  if (ctx->latched != CHFSI_OK) return ctx->latched;
  const HostMesh& m = ctx->mesh;
  if (!m.per[0] || !m.per[1] || !m.per[2]) return kfail(ctx, CHFSI_ERR_ARG, "Bloch states need a periodic box");
  if (!mf_supported(m.p, m.q)) return kfail(ctx, CHFSI_ERR_ARG, "k-points need 2 <= p <= 8 and q = p + 2");
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(k[d])) return kfail(ctx, CHFSI_ERR_ARG, "k must be finite");
  const int n1 = m.n1, q = m.q, nn = n1 * n1;
  std::vector<double> base, fac((size_t)9 * nn + 2 * q * n1);
  build_mf_factors(m, base);                       // A_x A_y A_z S_x S_y S_z B B^T
  const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
  std::copy(base.begin(), base.begin() + 6 * nn + 2 * q * n1, fac.begin());
  for (int i = 0; i < nn; ++i) fac[3 * nn + i] = base[3 * nn + i] + k2 * base[i];   // S'_x
  // 1-D derivative matrix C_il = int l_i l_l' = sum_a w_a B_ai D_al (no Jacobian)
  double* C = fac.data() + 6 * nn + 2 * q * n1;
  for (int i = 0; i < n1; ++i)
    for (int l = 0; l < n1; ++l) {
      double s = 0.0;
      for (int a = 0; a < q; ++a) s += m.gq_w[a] * m.B[a * n1 + i] * m.D[a * n1 + l];
      for (int d = 0; d < 3; ++d) C[d * nn + i * n1 + l] = k[d] * s;
    }
  if (!ctx->d_kfac) {
    if (cudaMalloc(&ctx->d_kfac, fac.size() * 8) != cudaSuccess) {
      cudaGetLastError();
      ctx->d_kfac = nullptr;
      return kfail(ctx, CHFSI_ERR_OOM, "k-point factors");
    }
    ctx->dev_bytes += (int64_t)fac.size() * 8;
  }
  KK(cudaMemcpyAsync(ctx->d_kfac, fac.data(), fac.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
  // dense shared blocks of the mixed path: A3 = A_z (x) A_y (x) A_x and
  // G3 = k_x A_z A_y C_x + k_y A_z C_y A_x + k_z C_z A_y A_x (node l = i + n1 (j + n1 kz)),
  // scaled by the cells' M^{-1/2} pattern when that pattern is the same in every cell
  const int ne = m.ne;
  bool uniform = true;
  std::vector<double> sc(ne);
  for (int l = 0; l < ne; ++l) sc[l] = 1.0 / std::sqrt(m.mass[m.dofmap[l]]);
  for (int64_t e = 1; e < m.ncells && uniform; ++e)
    for (int l = 0; l < ne; ++l)
      if (std::fabs(1.0 / std::sqrt(m.mass[m.dofmap[e * ne + l]]) - sc[l]) > 1e-12 * sc[l]) {
        uniform = false;
        break;
      }
  ctx->kpack_valid = false;
  if (uniform) {
    const double* Ax = base.data();
    const double* Ay = Ax + nn;
    const double* Az = Ay + nn;
    std::vector<double> A3((size_t)ne * ne), G3((size_t)ne * ne);
    for (int kz = 0; kz < n1; ++kz)
      for (int jy = 0; jy < n1; ++jy)
        for (int ix = 0; ix < n1; ++ix) {
          const int l = ix + n1 * (jy + n1 * kz);
          for (int kz2 = 0; kz2 < n1; ++kz2)
            for (int jy2 = 0; jy2 < n1; ++jy2)
              for (int ix2 = 0; ix2 < n1; ++ix2) {
                const int l2 = ix2 + n1 * (jy2 + n1 * kz2);
                const double az = Az[kz * n1 + kz2], ay = Ay[jy * n1 + jy2], ax = Ax[ix * n1 + ix2];
                const double a = az * ay * ax;
                const double g = az * ay * C[ix * n1 + ix2] + az * C[nn + jy * n1 + jy2] * ax +
                                 C[2 * nn + kz * n1 + kz2] * ay * ax;
                A3[(size_t)l * ne + l2] = 0.5 * k2 * a * sc[l] * sc[l2];
                G3[(size_t)l * ne + l2] = g * sc[l] * sc[l2];
              }
        }
    for (double** dp : {&ctx->d_kA, &ctx->d_kG})
      if (!*dp) {
        if (cudaMalloc(dp, (size_t)ne * ne * 8) != cudaSuccess) {
          cudaGetLastError();
          *dp = nullptr;
          return kfail(ctx, CHFSI_ERR_OOM, "k-point blocks");
        }
        ctx->dev_bytes += (int64_t)ne * ne * 8;
      }
    KK(cudaMemcpyAsync(ctx->d_kA, A3.data(), A3.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    KK(cudaMemcpyAsync(ctx->d_kG, G3.data(), G3.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
  } else {
    for (double** dp : {&ctx->d_kA, &ctx->d_kG})
      if (*dp) {
        cudaFree(*dp);
        *dp = nullptr;
        ctx->dev_bytes -= (int64_t)ne * ne * 8;
      }
  }
  KK(cudaStreamSynchronize(ctx->stream));
  for (int d = 0; d < 3; ++d) ctx->kpt[d] = k[d];
  ctx->kset = true;
  return CHFSI_OK;
}

chfsi_status chfsi_apply_kpoint(chfsi_ctx* ctx, const double* X, int64_t ldx, double* Y, int64_t ldy, int n) {
  chfsi_status st = kcheck(ctx);
  if (st != CHFSI_OK) return st;
  if (n < 0 || (n > 0 && (!X || !Y || ldx < 2 * n || ldy < 2 * n)))
    return kfail(ctx, CHFSI_ERR_ARG, "bad X / Y / leading dimensions (in doubles, >= 2 n)");
  if (n == 0) return CHFSI_OK;
  return kapply(ctx, X, ldx, Y, ldy, nullptr, 0, n, 1.0, 0.0, 0.0);
}

chfsi_status chfsi_bounds_kpoint(chfsi_ctx* ctx, int lanczos_steps, uint64_t seed, double* b_out) {
  chfsi_status st = kcheck(ctx);
  if (st != CHFSI_OK) return st;
  if (lanczos_steps < 1 || !b_out) return kfail(ctx, CHFSI_ERR_ARG, "bad Lanczos arguments");
  const int64_t M2 = 2 * ctx->mesh.ndofs;
  if ((st = kgrow(ctx, ctx->kvec, (size_t)M2 * 8 * 3 + 64)) != CHFSI_OK) return st;
  if ((st = kgrow(ctx, ctx->kG, (size_t)8 * 1024 + 64)) != CHFSI_OK) return st;
  double* v = (double*)ctx->kvec.ptr;
  double* vp = v + M2;
  double* w = vp + M2;
  double* dot = (double*)ctx->kG.ptr;
  double* part = dot + 8;
  KK(launch_fill_uniform(v, 1, M2, 1, stream_key(seed, 7), 1, ctx->stream));
  KK(cudaMemsetAsync(vp, 0, M2 * 8, ctx->stream));
  auto dotp = [&](const double* x, const double* y, double* r) -> chfsi_status {
    KK(launch_gram_fp64(x, 1, y, 1, M2, 1, 1, dot, 1, 0, part, 8 * 1000, ctx->stream));
    KK(cudaMemcpyAsync(r, dot, 8, cudaMemcpyDeviceToHost, ctx->stream));
    KK(cudaStreamSynchronize(ctx->stream));
    return CHFSI_OK;
  };
  double nv = 0.0;
  if ((st = dotp(v, v, &nv)) != CHFSI_OK) return st;
  note_launch();
  kscal_kernel<<<kblk(M2), 256, 0, ctx->stream>>>(v, v, M2, 1.0 / std::sqrt(nv));
  std::vector<double> al, be;
  double bprev = 0.0;
  for (int k = 0; k < lanczos_steps; ++k) {
    if ((st = kapply(ctx, v, 2, w, 2, nullptr, 0, 1, 1.0, 0.0, 0.0)) != CHFSI_OK) return st;
    note_launch();
    kaxpy2_kernel<<<kblk(M2), 256, 0, ctx->stream>>>(w, v, vp, M2, 0.0, -bprev);
    double a = 0.0;
    if ((st = dotp(w, v, &a)) != CHFSI_OK) return st;
    note_launch();
    kaxpy2_kernel<<<kblk(M2), 256, 0, ctx->stream>>>(w, v, vp, M2, -a, 0.0);
    double bb = 0.0;
    if ((st = dotp(w, w, &bb)) != CHFSI_OK) return st;
    bb = std::sqrt(bb);
    al.push_back(a);
    be.push_back(bb);
    if (bb == 0.0) break;
    KK(cudaMemcpyAsync(vp, v, M2 * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    note_launch();
    kscal_kernel<<<kblk(M2), 256, 0, ctx->stream>>>(v, w, M2, 1.0 / bb);
    bprev = bb;
  }
  // largest eigenvalue of the tridiagonal by bisection (Sturm counts)
  const int k = (int)al.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < k; ++i) {
    const double r = (i > 0 ? std::fabs(be[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(be[i]) : 0.0);
    lo = std::min(lo, al[i] - r);
    hi = std::max(hi, al[i] + r);
  }
  auto below = [&](double x) {
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < k; ++i) {
      d = (al[i] - x) - (i > 0 ? be[i - 1] * be[i - 1] / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0) cnt++;
    }
    return cnt;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-14 * std::max(1.0, std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (below(mid) >= k) hi = mid;
    else lo = mid;
  }
  *b_out = hi + std::fabs(be[k - 1]);
  return CHFSI_OK;
}

chfsi_status chfsi_apply_kpoint_mixed(chfsi_ctx* ctx, const float* X, int64_t ldx, float* Y, int64_t ldy,
                                      int n) {
  chfsi_status st = kcheck(ctx);
  if (st != CHFSI_OK) return st;
  if (n < 0 || (n > 0 && (!X || !Y || ldx < 2 * n || ldy < 2 * n || (ldx & 1))))
    return kfail(ctx, CHFSI_ERR_ARG, "bad X / Y / leading dimensions (in floats, even, >= 2 n)");
  if (n == 0) return CHFSI_OK;
  if ((st = kpack_mixed(ctx)) != CHFSI_OK) return st;
  return kapply_mixed(ctx, X, ldx, Y, ldy, nullptr, 0, n, 1.0, 0.0, 0.0);
}

chfsi_status chfsi_solve_kpoint_prec(chfsi_ctx* ctx, double* X, int64_t ldx, int n, int iters, int degree,
                                     double b, chfsi_precision filter_prec, double* evals_host) {
  if (filter_prec == CHFSI_FP64) return chfsi_solve_kpoint(ctx, X, ldx, n, iters, degree, b, evals_host);
  chfsi_status st = kcheck(ctx);
  if (st != CHFSI_OK) return st;
  if (filter_prec != CHFSI_MIXED_BF16X3) return kfail(ctx, CHFSI_ERR_ARG, "k-point filter: binary64 or BF16x3");
  if (n < 1 || !X || ldx < 2 * n || iters < 0 || degree < 1 || !evals_host)
    return kfail(ctx, CHFSI_ERR_ARG, "bad k-point solve arguments");
  const HostMesh& m = ctx->mesh;
  if ((st = kpack_mixed(ctx)) != CHFSI_OK) return st;
  // binary32 copy of the block for the filter; CholGS / RR on the binary64 block
  if ((st = kgrow(ctx, ctx->kvec, (size_t)m.ndofs * 2 * n * 4 + 16)) != CHFSI_OK) return st;
  float* X32 = (float*)ctx->kvec.ptr;
  const int64_t ld32 = 2 * (int64_t)n;
  std::vector<double> D(n);
  if ((st = kcholgs(ctx, X, ldx, n)) != CHFSI_OK) return st;
  if ((st = krr(ctx, X, ldx, n, D.data())) != CHFSI_OK) return st;
  for (int it = 0; it < iters; ++it) {
    double a = D[n - 1], a0 = D[0];
    if (!(a < b)) return kfail(ctx, CHFSI_ERR_ARG, "upper bound b must exceed the largest Ritz value");
    if (!(a0 < a)) a0 = a - 1e-3 * std::max(1.0, std::fabs(a));
    KK(launch_copy_cols(X, ldx, X32, ld32, m.ndofs, 2 * n, 1, 0, ctx->stream));
    if ((st = kfilter_mixed(ctx, X32, ld32, n, degree, a, b, a0)) != CHFSI_OK) return st;
    KK(launch_copy_cols(X32, ld32, X, ldx, m.ndofs, 2 * n, 0, 1, ctx->stream));
    if ((st = kcholgs(ctx, X, ldx, n)) != CHFSI_OK) return st;
    if ((st = krr(ctx, X, ldx, n, D.data())) != CHFSI_OK) return st;
  }
  if (tc_read_status(ctx->stream)) return kfail(ctx, CHFSI_ERR_TIMEOUT, "device wait timed out");
  KK(cudaStreamSynchronize(ctx->stream));
  std::memcpy(evals_host, D.data(), (size_t)n * 8);
  return CHFSI_OK;
}

chfsi_status chfsi_solve_kpoint(chfsi_ctx* ctx, double* X, int64_t ldx, int n, int iters, int degree,
                                double b, double* evals_host) {
  chfsi_status st = kcheck(ctx);
  if (st != CHFSI_OK) return st;
  if (n < 1 || !X || ldx < 2 * n || iters < 0 || degree < 1 || !evals_host)
    return kfail(ctx, CHFSI_ERR_ARG, "bad k-point solve arguments");
  std::vector<double> D(n);
  if ((st = kcholgs(ctx, X, ldx, n)) != CHFSI_OK) return st;
  if ((st = krr(ctx, X, ldx, n, D.data())) != CHFSI_OK) return st;
  for (int it = 0; it < iters; ++it) {
    double a = D[n - 1], a0 = D[0];
    if (!(a < b)) return kfail(ctx, CHFSI_ERR_ARG, "upper bound b must exceed the largest Ritz value");
    if (!(a0 < a)) a0 = a - 1e-3 * std::max(1.0, std::fabs(a));
    if ((st = kfilter(ctx, X, ldx, n, degree, a, b, a0)) != CHFSI_OK) return st;
    if ((st = kcholgs(ctx, X, ldx, n)) != CHFSI_OK) return st;
    if ((st = krr(ctx, X, ldx, n, D.data())) != CHFSI_OK) return st;
  }
  KK(cudaStreamSynchronize(ctx->stream));
  std::memcpy(evals_host, D.data(), (size_t)n * 8);
  return CHFSI_OK;
}

}  // extern "C"
