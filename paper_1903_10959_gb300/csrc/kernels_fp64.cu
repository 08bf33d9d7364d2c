#include <algorithm>
// Binary64 kernels of the ChFSI step (CUDA-core DFMA; GB300 runs binary64 at
// ~1 TFLOP/s, so these kernels are arithmetic-bound and kept simple), plus
// the precision-independent helpers (seeded fill, copies, scaling).
//
//  cell_fp64      : one colour of H~ Y = sum_e P_e^T H~_e P_e Y (Sec. 3.3.1:
//                   gather the cell block, dense cell product, assemble) fused
//                   with the Chebyshev three-term update (Eq. chebFilter).
//  gram_fp64      : S = A^T B over the unknowns (Algorithm CholGS step 1, and
//                   H^ = X^T (H~ X) of Sec. 3.5), split over row chunks with a
//                   fixed-order reduction (deterministic).
//  tallgemm_fp64  : X U for an N x N (optionally upper-triangular) U
//                   (Algorithm CholGS step 4; subspace rotation of Sec. 3.5).
//  resid_fp64     : column norms of H~ x - l x (binary64 accumulation).
//  nl_*_fp64      : separable projector term C~^T h C~ Y (Eqs. nlps,
//                   nonlocalHamDiscrete) in owner-computes form.
#include <cstdint>
#include <mutex>

#include "internal.h"

namespace chfsi {

// ---------------------------------------------------------------- cell apply
template <int BT>
__global__ void __launch_bounds__(256) cell_fp64_kernel(
    const double* __restrict__ Ht, const int32_t* __restrict__ dofmap,
    const uint8_t* __restrict__ modes, const int32_t* __restrict__ cells, int ne, int ncol,
    const double* __restrict__ Yin, int64_t ld_in, double* Yout, int64_t ld_out,
    const double* Yprev, int64_t ld_prev, double* __restrict__ W, int64_t ld_w,
    const double* __restrict__ NL, double alpha, double beta, double shift) {
  extern __shared__ double ys[];  // ne x BT, node-major
  const int64_t e = cells[blockIdx.x];
  const int c0 = blockIdx.y * BT;
  const int ncv = min(BT, ncol - c0);
  const int32_t* dm = dofmap + e * ne;
  const uint8_t* md = modes + e * ne;

  for (int idx = threadIdx.x; idx < ne * BT; idx += blockDim.x) {
    const int l = idx / BT, c = idx - (idx / BT) * BT;
    const int g = dm[l];
    double v = 0.0;
    if (g >= 0 && c < ncv) v = Yin[(int64_t)g * ld_in + c0 + c];
    ys[idx] = v;
  }
  __syncthreads();

  const double* H = Ht + e * (int64_t)ne * ne;
  for (int o = threadIdx.x; o < ne * BT; o += blockDim.x) {
    const int l = o / BT, c = o - (o / BT) * BT;
    const double* hr = H + (int64_t)l * ne;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int k = 0;
    for (; k + 4 <= ne; k += 4) {
      a0 = fma(__ldg(hr + k), ys[(k)*BT + c], a0);
      a1 = fma(__ldg(hr + k + 1), ys[(k + 1) * BT + c], a1);
      a2 = fma(__ldg(hr + k + 2), ys[(k + 2) * BT + c], a2);
      a3 = fma(__ldg(hr + k + 3), ys[(k + 3) * BT + c], a3);
    }
    for (; k < ne; ++k) a0 = fma(__ldg(hr + k), ys[k * BT + c], a0);
    double v = (a0 + a1) + (a2 + a3);
    const uint8_t mode = md[l];
    if (mode == MODE_SKIP || c >= ncv) continue;
    const int64_t g = dm[l];
    const int cc = c0 + c;
    if (mode == MODE_STORE) {
      W[g * ld_w + cc] = v;
    } else if (mode == MODE_ACCUM) {
      W[g * ld_w + cc] += v;
    } else {
      if (mode == MODE_FINAL) v += W[g * ld_w + cc];
      if (NL) v += NL[g * ld_w + cc];
      double out = alpha * (v - shift * ys[l * BT + c]);
      if (Yprev) out = fma(beta, Yprev[g * ld_prev + cc], out);
      Yout[g * ld_out + cc] = out;
    }
  }
}

cudaError_t launch_cell_fp64(const CellLaunch& L, const double* Yin, double* Yout,
                             const double* Yprev, double* W, const double* NL, int64_t ld_w,
                             FilterStep st, cudaStream_t s) {
  if (L.ncells_colour == 0 || L.ncol == 0) return cudaSuccess;
  const int bt = L.ncol >= 16 ? 16 : (L.ncol >= 4 ? 4 : 1);
  dim3 grid((unsigned)L.ncells_colour, (unsigned)((L.ncol + bt - 1) / bt));
  size_t smem = (size_t)L.ne * bt * sizeof(double);
  const double* prev = (st.beta != 0.0) ? Yprev : nullptr;
#define CHFSI_CELL_LAUNCH(B)                                                                      \
  do {                                                                                            \
    static std::once_flag attr_##B;                                                               \
    std::call_once(attr_##B, [] {                                                                 \
      cudaFuncSetAttribute(cell_fp64_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                           96 * 1024);                                                            \
    });                                                                                           \
    note_launch();                                                                                \
    cell_fp64_kernel<B><<<grid, 256, smem, s>>>(L.Ht, L.dofmap, L.modes, L.cells, L.ne, L.ncol,   \
                                                Yin, L.ld_in, Yout, L.ld_out, prev, L.ld_prev, W,  \
                                                ld_w, NL, st.alpha, st.beta, st.shift);           \
  } while (0)
  if (bt == 16) CHFSI_CELL_LAUNCH(16);
  else if (bt == 4) CHFSI_CELL_LAUNCH(4);
  else CHFSI_CELL_LAUNCH(1);
#undef CHFSI_CELL_LAUNCH
  return cudaGetLastError();
}

// ---------------------------------------------------------------- Gram (A^T B)
// 64 x 64 output tile per CTA, 256 threads with 4 x 4 micro-tiles, rows in
// chunks of 16 through shared memory; grid.z splits the rows, partial tiles
// go to `partial` and are summed in fixed order by gram_reduce.
constexpr int GT = 64, GK = 16;

__global__ void __launch_bounds__(256) gram_fp64_kernel(const double* __restrict__ A, int64_t lda,
                                                        const double* __restrict__ B, int64_t ldb,
                                                        int64_t M, int n1, int n2, int lower_only,
                                                        int64_t rows_per_split,
                                                        double* __restrict__ partial) {
  const int ti = blockIdx.x, tj = blockIdx.y, z = blockIdx.z;
  if (lower_only && (ti + 1) * GT <= tj * GT) return;   // tile strictly above the diagonal
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4] = {};
  const int64_t r0 = (int64_t)z * rows_per_split;
  const int64_t r1 = min(M, r0 + rows_per_split);
  for (int64_t r = r0; r < r1; r += GK) {
    for (int idx = threadIdx.x; idx < GK * GT; idx += 256) {
      const int kk = idx / GT, cc = idx % GT;
      const int64_t row = r + kk;
      const int ia = ti * GT + cc, jb = tj * GT + cc;
      As[kk][cc] = (row < r1 && ia < n1) ? A[row * lda + ia] : 0.0;
      Bs[kk][cc] = (row < r1 && jb < n2) ? B[row * ldb + jb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { a[u] = As[kk][ty * 4 + u]; b[u] = Bs[kk][tx * 4 + u]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
  double* P = partial + (int64_t)z * n1 * n2;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = ti * GT + ty * 4 + u, j = tj * GT + tx * 4 + v;
      if (i < n1 && j < n2) P[i + (int64_t)j * n1] = acc[u][v];
    }
}

__global__ void gram_reduce_kernel(const double* __restrict__ partial, int nsplit, int n1, int n2,
                                   double* __restrict__ C, int64_t ldc, int lower_only) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n1 * n2) return;
  const int i = (int)(idx % n1), j = (int)(idx / n1);
  if (lower_only && (i / GT) < (j / GT)) return;
  double s = 0.0;
  for (int z = 0; z < nsplit; ++z) s += partial[(int64_t)z * n1 * n2 + idx];
  C[i + (int64_t)j * ldc] = s;
}

cudaError_t launch_gram_fp64(const double* A, int64_t lda, const double* B, int64_t ldb,
                             int64_t M, int n1, int n2, double* C, int64_t ldc, int lower_only,
                             double* partial, size_t partial_bytes, cudaStream_t s) {
  if (n1 == 0 || n2 == 0) return cudaSuccess;
  const int t1 = (n1 + GT - 1) / GT, t2 = (n2 + GT - 1) / GT;
  int64_t tiles = (int64_t)t1 * t2;
  int64_t max_split = (int64_t)(partial_bytes / (sizeof(double) * (size_t)n1 * n2));
  int64_t want = (4 * 152 + tiles - 1) / tiles;
  int64_t nsplit = std::max<int64_t>(1, std::min<int64_t>(std::min(want, max_split), (M + 255) / 256));
  int64_t rps = ((M + nsplit - 1) / nsplit + GK - 1) / GK * GK;
  nsplit = (M + rps - 1) / rps;
  if (nsplit < 1) nsplit = 1;
  dim3 grid(t1, t2, (unsigned)nsplit);
  note_launch();
  gram_fp64_kernel<<<grid, 256, 0, s>>>(A, lda, B, ldb, M, n1, n2, lower_only, rps, partial);
  const int64_t tot = (int64_t)n1 * n2;
  note_launch();
  gram_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(partial, (int)nsplit, n1, n2, C,
                                                                   ldc, lower_only);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- tall GEMM (A U)
__global__ void __launch_bounds__(256) tallgemm_fp64_kernel(const double* __restrict__ A, int64_t lda,
                                                            const double* __restrict__ U, int64_t ldu,
                                                            int64_t M, int n1, int n2,
                                                            double* __restrict__ C, int64_t ldc,
                                                            int upper_tri, int trans_u) {
  __shared__ double As[GT][GK + 1];   // rows x k
  __shared__ double Us[GK][GT + 1];   // k x cols
  const int64_t rb = (int64_t)blockIdx.x * GT;
  const int cb = blockIdx.y * GT;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4] = {};
  const int kend = upper_tri ? min(n1, cb + GT) : n1;
  for (int k0 = 0; k0 < kend; k0 += GK) {
    for (int idx = threadIdx.x; idx < GT * GK; idx += 256) {
      const int rr = idx / GK, kk = idx % GK;
      const int64_t row = rb + rr;
      As[rr][kk] = (row < M && k0 + kk < n1) ? A[row * lda + k0 + kk] : 0.0;
      const int kk2 = idx % GK, cc = idx / GK;
      const int col = cb + cc, kx = k0 + kk2;
      double u = 0.0;
      if (col < n2 && kx < n1 && (!upper_tri || kx <= col))
        u = trans_u ? U[col + (int64_t)kx * ldu] : U[kx + (int64_t)col * ldu];
      Us[kk2][cc] = u;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { a[u] = As[ty * 4 + u][kk]; b[u] = Us[kk][tx * 4 + u]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t row = rb + ty * 4 + u;
    if (row >= M) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int col = cb + tx * 4 + v;
      if (col < n2) C[row * ldc + col] = acc[u][v];
    }
  }
}

cudaError_t launch_tallgemm_fp64(const double* A, int64_t lda, const double* U, int64_t ldu,
                                 int64_t M, int n1, int n2, double* C, int64_t ldc, int upper_tri,
                                 int trans_u, cudaStream_t s) {
  if (M == 0 || n2 == 0) return cudaSuccess;
  dim3 grid((unsigned)((M + GT - 1) / GT), (unsigned)((n2 + GT - 1) / GT));
  note_launch();
  tallgemm_fp64_kernel<<<grid, 256, 0, s>>>(A, lda, U, ldu, M, n1, n2, C, ldc, upper_tri, trans_u);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- residual norms
// out_sq[2*i]   = sum_r (Y - l X)^2,  out_sq[2*i+1] = sum_r w_r (Y - l X)^2,
// out_sq[2*n+i] = sum_r X^2.  With lam == nullptr, out_sq[i] = sum_r X Y instead
// (numerator of the Rayleigh quotient).  Block: 32 columns x 8 row lanes;
// fixed-order reductions.
__global__ void resid_partial_kernel(const double* __restrict__ Y, int64_t ldy,
                                     const double* __restrict__ X, int64_t ldx, int64_t M, int n,
                                     const double* __restrict__ lam, const double* __restrict__ wgt,
                                     int64_t rows_per_chunk, double* __restrict__ partial) {
  const int c = blockIdx.x * 32 + threadIdx.x % 32;
  const int ty = threadIdx.x / 32;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t r1 = min(M, r0 + rows_per_chunk);
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  if (c < n) {
    if (lam) {
      const double l = lam[c];
      for (int64_t r = r0 + ty; r < r1; r += 8) {
        const double x = X[r * ldx + c];
        const double d = Y[r * ldy + c] - l * x;
        s0 = fma(d, d, s0);
        if (wgt) s1 = fma(wgt[r] * d, d, s1);
        s2 = fma(x, x, s2);
      }
    } else {
      for (int64_t r = r0 + ty; r < r1; r += 8) {
        const double x = X[r * ldx + c];
        s0 = fma(x, Y[r * ldy + c], s0);
        s2 = fma(x, x, s2);
      }
    }
  }
  __shared__ double red[3][8][32];
  red[0][ty][threadIdx.x % 32] = s0;
  red[1][ty][threadIdx.x % 32] = s1;
  red[2][ty][threadIdx.x % 32] = s2;
  __syncthreads();
  if (ty == 0 && c < n) {
    double a = 0, b = 0, d = 0;
    for (int t = 0; t < 8; ++t) { a += red[0][t][threadIdx.x]; b += red[1][t][threadIdx.x]; d += red[2][t][threadIdx.x]; }
    double* P = partial + (int64_t)blockIdx.y * 3 * n;
    P[c] = a;
    P[n + c] = b;
    P[2 * n + c] = d;
  }
}

__global__ void resid_reduce_kernel(const double* __restrict__ partial, int nchunk, int n,
                                    double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * n) return;
  double s = 0.0;
  for (int z = 0; z < nchunk; ++z) s += partial[(int64_t)z * 3 * n + i];
  out[i] = s;
}

cudaError_t launch_resid_norms(const double* Y, int64_t ldy, const double* X, int64_t ldx,
                               int64_t M, int n, const double* lam, const double* wgt,
                               double* out_sq, double* partial, size_t partial_bytes,
                               cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int64_t max_chunks = (int64_t)(partial_bytes / (sizeof(double) * 3 * (size_t)n));
  int64_t nchunk = std::max<int64_t>(1, std::min<int64_t>(max_chunks, (M + 4095) / 4096));
  int64_t rpc = (M + nchunk - 1) / nchunk;
  nchunk = (M + rpc - 1) / rpc;
  dim3 grid((unsigned)((n + 31) / 32), (unsigned)nchunk);
  note_launch();
  resid_partial_kernel<<<grid, 256, 0, s>>>(Y, ldy, X, ldx, M, n, lam, wgt, rpc, partial);
  note_launch();
  resid_reduce_kernel<<<(3 * n + 255) / 256, 256, 0, s>>>(partial, (int)nchunk, n, out_sq);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- nonlocal projectors
// Z[4 s + t][c] = sum over the support of site s of C~[s, j, t] Y[j][c]
__global__ void nl_project_kernel(const int64_t* __restrict__ site_ptr,
                                  const int32_t* __restrict__ site_dof,
                                  const double* __restrict__ site_c, const double* __restrict__ Y,
                                  int64_t ldy, int ncol, double* __restrict__ Z) {
  const int s = blockIdx.x;
  const int c = blockIdx.y * 32 + threadIdx.x % 32;
  const int w = threadIdx.x / 32;  // 4 warps
  double acc[4] = {0, 0, 0, 0};
  if (c < ncol) {
    for (int64_t e = site_ptr[s] + w; e < site_ptr[s + 1]; e += 4) {
      const double y = Y[(int64_t)site_dof[e] * ldy + c];
#pragma unroll
      for (int t = 0; t < 4; ++t) acc[t] = fma(site_c[4 * e + t], y, acc[t]);
    }
  }
  __shared__ double red[4][4][32];
#pragma unroll
  for (int t = 0; t < 4; ++t) red[w][t][threadIdx.x % 32] = acc[t];
  __syncthreads();
  if (w == 0 && c < ncol) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      double v = ((red[0][t][threadIdx.x] + red[1][t][threadIdx.x]) + red[2][t][threadIdx.x]) +
                 red[3][t][threadIdx.x];
      Z[(int64_t)(4 * s + t) * ncol + c] = v;
    }
  }
}

// NL[j][c] = sum over sites touching j of C~[s, j, t] h[s, t] Z[4 s + t][c]
__global__ void nl_expand_kernel(const int64_t* __restrict__ dof_ptr,
                                 const int32_t* __restrict__ dof_site,
                                 const double* __restrict__ dof_c, int64_t M,
                                 const double* __restrict__ Z, int ncol, double* __restrict__ NL,
                                 int64_t ldn) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= M * ncol) return;
  const int64_t j = idx / ncol;
  const int c = (int)(idx - j * ncol);
  double v = 0.0;
  for (int64_t e = dof_ptr[j]; e < dof_ptr[j + 1]; ++e) {
    const int64_t s = dof_site[e];
#pragma unroll
    for (int t = 0; t < 4; ++t) v = fma(dof_c[4 * e + t], Z[(4 * s + t) * ncol + c], v);
  }
  NL[j * ldn + c] = v;
}

cudaError_t launch_nl_project_fp64(const int64_t* site_ptr, const int32_t* site_dof,
                                   const double* site_c, int nsite, const double* Y, int64_t ldy,
                                   int ncol, double* Z, cudaStream_t s) {
  if (nsite == 0 || ncol == 0) return cudaSuccess;
  dim3 grid(nsite, (ncol + 31) / 32);
  note_launch();
  nl_project_kernel<<<grid, 128, 0, s>>>(site_ptr, site_dof, site_c, Y, ldy, ncol, Z);
  return cudaGetLastError();
}

cudaError_t launch_nl_expand_fp64(const int64_t* dof_ptr, const int32_t* dof_site,
                                  const double* dof_c, int64_t M, const double* Z, int ncol,
                                  double* NL, int64_t ldn, cudaStream_t s) {
  const int64_t tot = M * ncol;
  if (tot == 0) return cudaSuccess;
  note_launch();
  nl_expand_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(dof_ptr, dof_site, dof_c, M, Z,
                                                                  ncol, NL, ldn);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ uint64_t splitmix_finalize(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void fill_uniform_kernel(void* X, int64_t ldx, int64_t rows, int ncol, uint64_t key,
                                    int is_double) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= rows * ncol) return;
  const int64_t r = idx / ncol;
  const int c = (int)(idx - r * ncol);
  const uint64_t state = key + (uint64_t)(idx + 1) * 0x9E3779B97F4A7C15ull;
  const double u = (double)(splitmix_finalize(state) >> 11) * (1.0 / 9007199254740992.0);
  const double v = 2.0 * u - 1.0;
  if (is_double) ((double*)X)[r * ldx + c] = v;
  else ((float*)X)[r * ldx + c] = (float)v;
}

uint64_t stream_key(uint64_t seed, uint64_t stream) {
  uint64_t z = seed;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return z ^ (stream * 0xD1B54A32D192ED03ull);
}

cudaError_t launch_fill_uniform(void* X, int64_t ldx, int64_t rows, int ncol, uint64_t key,
                                int is_double, cudaStream_t s) {
  const int64_t tot = rows * ncol;
  if (tot == 0) return cudaSuccess;
  note_launch();
  fill_uniform_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, ldx, rows, ncol, key,
                                                                     is_double);
  return cudaGetLastError();
}

__global__ void copy_cols_kernel(const void* src, int64_t lds, void* dst, int64_t ldd,
                                 int64_t rows, int ncol, int sd, int dd) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= rows * ncol) return;
  const int64_t r = idx / ncol;
  const int c = (int)(idx - r * ncol);
  const double v = sd ? ((const double*)src)[r * lds + c] : (double)((const float*)src)[r * lds + c];
  if (dd) ((double*)dst)[r * ldd + c] = v;
  else ((float*)dst)[r * ldd + c] = (float)v;
}

cudaError_t launch_copy_cols(const void* src, int64_t lds, void* dst, int64_t ldd, int64_t rows,
                             int ncol, int src_double, int dst_double, cudaStream_t s) {
  const int64_t tot = rows * ncol;
  if (tot == 0) return cudaSuccess;
  note_launch();
  copy_cols_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src, lds, dst, ldd, rows, ncol,
                                                                  src_double, dst_double);
  return cudaGetLastError();
}

// Row-by-row byte copy between two pitched 2-D buffers (either may be a
// device-mapped host buffer: the SMs then move the rows over the coherent
// host link).  16-byte vectors when every pointer, pitch and row length is a
// multiple of 16 bytes, else 4-byte words (row lengths are multiples of 4).
__global__ void copy2d_kernel(const char* __restrict__ src, int64_t sp, char* __restrict__ dst,
                              int64_t dp, int64_t rows, int64_t rb, int vec) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t w = vec ? 16 : 4;
  const int64_t per = rb / w, tot = rows * per;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += stride) {
    const int64_t r = i / per, c = i - r * per;
    if (vec)
      reinterpret_cast<uint4*>(dst + r * dp)[c] = reinterpret_cast<const uint4*>(src + r * sp)[c];
    else
      reinterpret_cast<uint32_t*>(dst + r * dp)[c] = reinterpret_cast<const uint32_t*>(src + r * sp)[c];
  }
}

cudaError_t launch_copy2d(const void* src, int64_t src_pitch, void* dst, int64_t dst_pitch,
                          int64_t rows, int64_t row_bytes, int nsm, cudaStream_t s) {
  if (rows == 0 || row_bytes == 0) return cudaSuccess;
  if (row_bytes % 4 || src_pitch % 4 || dst_pitch % 4 || ((uintptr_t)src & 3) || ((uintptr_t)dst & 3))
    return cudaErrorInvalidValue;
  const int vec = (row_bytes % 16 == 0 && src_pitch % 16 == 0 && dst_pitch % 16 == 0 &&
                   ((uintptr_t)src & 15) == 0 && ((uintptr_t)dst & 15) == 0);
  const int64_t tot = rows * (row_bytes / (vec ? 16 : 4));
  const int64_t blocks = std::min<int64_t>((tot + 255) / 256, (int64_t)std::max(nsm, 1) * 8);
  note_launch();
  copy2d_kernel<<<(unsigned)blocks, 256, 0, s>>>((const char*)src, src_pitch, (char*)dst, dst_pitch,
                                                 rows, row_bytes, vec);
  return cudaGetLastError();
}

__global__ void scale_rows_kernel(void* X, int64_t ldx, int64_t rows, int ncol,
                                  const double* __restrict__ sv, int is_double) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= rows * ncol) return;
  const int64_t r = idx / ncol;
  const int c = (int)(idx - r * ncol);
  if (is_double) ((double*)X)[r * ldx + c] *= sv[r];
  else ((float*)X)[r * ldx + c] = (float)((double)((float*)X)[r * ldx + c] * sv[r]);
}

cudaError_t launch_scale_rows(void* X, int64_t ldx, int64_t rows, int ncol, const double* sv,
                              int is_double, cudaStream_t s) {
  const int64_t tot = rows * ncol;
  if (tot == 0) return cudaSuccess;
  note_launch();
  scale_rows_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, ldx, rows, ncol, sv, is_double);
  return cudaGetLastError();
}

// w <- w + a v + b vp ; used by the Lanczos bound (binary64)
__global__ void axpy2_kernel(double* w, const double* v, const double* vp, int64_t M, double a,
                             double b) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < M) w[i] = fma(a, v[i], fma(b, vp[i], w[i]));
}
// v <- w * s
__global__ void scal_copy_kernel(double* v, const double* w, int64_t M, double s) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < M) v[i] = w[i] * s;
}

cudaError_t launch_axpy2(double* w, const double* v, const double* vp, int64_t M, double a,
                         double b, cudaStream_t s) {
  note_launch();
  axpy2_kernel<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(w, v, vp, M, a, b);
  return cudaGetLastError();
}
cudaError_t launch_scal_copy(double* v, const double* w, int64_t M, double sc, cudaStream_t s) {
  note_launch();
  scal_copy_kernel<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(v, w, M, sc);
  return cudaGetLastError();
}

// Inverse of a lower triangular binary64 matrix: the factor L of CholGS
// (Algorithm CholGS, S = L L^T, then X <- X L^{-T}).  Column j of L^{-1} is
// the forward substitution L x = e_j, one warp per column.  The warp walks its
// rows in blocks of 32: lane l holds row k0 + l of the block and its 32
// entries of L to the left of the diagonal; the block is solved in 32 steps
// (x_t = b_t / L_tt broadcast by shuffle, the lanes below subtract L_lt x_t);
// then every row below the block subtracts the block's 32 products at once,
// with 32 independent coalesced loads of L per row (lanes over consecutive
// rows), from a right-hand side kept in shared memory.  Summation order:
// along increasing k within and across blocks, as a column-oriented forward
// substitution.
constexpr int TRI_WARPS = 4;
__global__ void __launch_bounds__(TRI_WARPS * 32) trinv_lower_kernel(const double* __restrict__ L, int64_t ldl,
                                                                     int n, double* __restrict__ X, int64_t ldx) {
  extern __shared__ double tsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * TRI_WARPS + warp;
  if (j >= n) return;                         // warp-uniform; the kernel uses no block barrier
  double* b = tsm + (size_t)warp * (n + 32);  // right-hand side, b[r] for row j + r
  double* xs = b + n;                         // the current block's solution
  const int m = n - j;
  for (int r = lane; r < m; r += 32) b[r] = r == 0 ? 1.0 : 0.0;
  __syncwarp();
  for (int k0 = 0; k0 < m; k0 += 32) {
    const int kb = min(32, m - k0);
    const int r = k0 + lane;
    const bool own = lane < kb;
    const int64_t i = (int64_t)j + r;
    const double* Lrow = L + i + (int64_t)(j + k0) * ldl;   // L(i, j + k0 + t) at Lrow[t * ldl]
    double Ld[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) Ld[t] = (own && t < lane) ? Lrow[(int64_t)t * ldl] : 0.0;
    const double invd = own ? 1.0 / L[i + i * ldl] : 0.0;
    double bi = own ? b[r] : 0.0;
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      if (t < kb) {
        const double xt = __shfl_sync(0xffffffffu, bi * invd, t);
        if (lane > t) bi = fma(-Ld[t], xt, bi);
      }
    }
    const double x = bi * invd;
    if (own) {
      X[i + (int64_t)j * ldx] = x;
      xs[lane] = x;
    }
    __syncwarp();
    // rows below the block: b[r2] -= sum_t L(j + r2, j + k0 + t) x_t
    for (int r2 = k0 + 32 + lane; r2 < m; r2 += 32) {
      const double* Lr = L + (int64_t)j + r2 + (int64_t)(j + k0) * ldl;
      double acc = b[r2];
#pragma unroll
      for (int t = 0; t < 32; ++t)
        if (t < kb) acc = fma(-Lr[(int64_t)t * ldl], xs[t], acc);
      b[r2] = acc;
    }
    __syncwarp();
  }
}

bool trinv_lower_supported(int n) { return n > 0 && (size_t)TRI_WARPS * (n + 32) * 8 <= 200 * 1024; }

cudaError_t launch_trinv_lower_fp64(const double* L, int64_t ldl, int n, double* X, int64_t ldx,
                                    cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (!trinv_lower_supported(n)) return cudaErrorInvalidValue;
  const size_t smem = (size_t)TRI_WARPS * (n + 32) * 8;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(trinv_lower_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  note_launch();
  trinv_lower_kernel<<<(unsigned)((n + TRI_WARPS - 1) / TRI_WARPS), TRI_WARPS * 32, smem, s>>>(L, ldl, n, X, ldx);
  return cudaGetLastError();
}

}  // namespace chfsi
