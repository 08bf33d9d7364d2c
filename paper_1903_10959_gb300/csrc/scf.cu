// Self-consistent field loop on the GPU (Algorithm scf, Sec. 3.2 of
// arXiv:1903.10959) around the ChFSI step, for periodic Gaussian-charge
// systems, with every field kept on the device:
//
//  ES  (step 4): the electrostatic potential phi of -(1/4 pi) lap phi =
//      rho + b (Eq. ksproblemPer) in its FE form K phi = 4 pi F,
//      F_j = int N_j (rho + b) by the cells' Gauss rule, net charge
//      neutralised by a uniform background, int phi = 0; solved by conjugate
//      gradients on the scaled stiffness M^{-1/2} K M^{-1/2} (the matrix-free
//      cell kernel with the kinetic part alone).
//  V_eff (step 5) = phi + V_x(rho), V_x = -(3 rho / pi)^{1/3} (the exchange
//      part of the local-density approximation), at the Gauss points.
//  Steps 6-7: the matrix-free operator takes V_eff at the Gauss points
//      directly (no cell matrices are rebuilt); ChFSI passes warm-started
//      from the previous block (binary64).
//  DC  (step 8): Fermi-Dirac occupations of all states and the density at
//      the Gauss points (Eq. elecDensSP).
//  Mixing (step 9, Sec. 3.6): n-stage Anderson mixing of rho (Anderson 1965),
//      weighted by the quadrature weights.
//
// Reductions (dot products) use a fixed block partition and a fixed-order
// host sum, so a run is deterministic.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

using namespace chfsi;

namespace {

constexpr int SCF_THREADS = 256;
constexpr int RED_BLOCKS = 304;   // 2 x 152 SMs

// Nodal field -> its values at the q^3 Gauss points of every cell, by three
// passes of the 1-D basis matrix B (q x n1).  One CTA per cell.
__global__ void qp_interp_kernel(const double* __restrict__ u, const int32_t* __restrict__ dofmap,
                                 const double* __restrict__ B, int n1, int q,
                                 double* __restrict__ out) {
  extern __shared__ double qs[];
  const int64_t e = blockIdx.x;
  const int ne = n1 * n1 * n1;
  double* ue = qs;                       // n1^3
  double* t1 = ue + ne;                  // (n1, n1, q)
  double* t2 = t1 + n1 * n1 * q;         // (n1, q, q)
  double* sB = t2 + n1 * q * q;          // q x n1
  for (int t = threadIdx.x; t < q * n1; t += blockDim.x) sB[t] = B[t];
  for (int l = threadIdx.x; l < ne; l += blockDim.x) {
    const int g = dofmap[e * ne + l];
    ue[l] = g >= 0 ? u[g] : 0.0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n1 * n1 * q; t += blockDim.x) {   // z
    const int i = t % n1, j = (t / n1) % n1, c = t / (n1 * n1);
    double s = 0.0;
    for (int k = 0; k < n1; ++k) s = fma(sB[c * n1 + k], ue[(k * n1 + j) * n1 + i], s);
    t1[t] = s;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n1 * q * q; t += blockDim.x) {    // y
    const int i = t % n1, b = (t / n1) % q, c = t / (n1 * q);
    double s = 0.0;
    for (int j = 0; j < n1; ++j) s = fma(sB[b * n1 + j], t1[(c * n1 + j) * n1 + i], s);
    t2[t] = s;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < q * q * q; t += blockDim.x) {     // x
    const int a = t % q, b = (t / q) % q, c = t / (q * q);
    double s = 0.0;
    for (int i = 0; i < n1; ++i) s = fma(sB[a * n1 + i], t2[(c * q + b) * n1 + i], s);
    out[e * (int64_t)q * q * q + t] = s;
  }
}

// F_j += int N_j f over the cells of one colour (cells of a colour share no
// unknown, so the adds do not race): f at the Gauss points times the
// weights W (q^3, with the Jacobian), then B^T along the three axes.
__global__ void qp_load_kernel(const double* __restrict__ f, const double* __restrict__ W,
                               const int32_t* __restrict__ cells, const int32_t* __restrict__ dofmap,
                               const double* __restrict__ B, int n1, int q, double* F) {
  extern __shared__ double qs[];
  const int64_t e = cells[blockIdx.x];
  const int ne = n1 * n1 * n1, nq = q * q * q;
  double* fe = qs;                       // (q, q, q)
  double* t2 = fe + nq;                  // (n1, q, q)
  double* t1 = t2 + n1 * q * q;          // (n1, n1, q)
  double* sB = t1 + n1 * n1 * q;         // q x n1
  for (int t = threadIdx.x; t < q * n1; t += blockDim.x) sB[t] = B[t];
  for (int t = threadIdx.x; t < nq; t += blockDim.x) fe[t] = f[e * (int64_t)nq + t] * W[t];
  __syncthreads();
  for (int t = threadIdx.x; t < n1 * q * q; t += blockDim.x) {    // x: (a) -> (i)
    const int i = t % n1, b = (t / n1) % q, c = t / (n1 * q);
    double s = 0.0;
    for (int a = 0; a < q; ++a) s = fma(sB[a * n1 + i], fe[(c * q + b) * q + a], s);
    t2[t] = s;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n1 * n1 * q; t += blockDim.x) {   // y: (b) -> (j)
    const int i = t % n1, j = (t / n1) % n1, c = t / (n1 * n1);
    double s = 0.0;
    for (int b = 0; b < q; ++b) s = fma(sB[b * n1 + j], t2[(c * q + b) * n1 + i], s);
    t1[t] = s;
  }
  __syncthreads();
  for (int l = threadIdx.x; l < ne; l += blockDim.x) {            // z: (c) -> (k), scatter
    const int i = l % n1, j = (l / n1) % n1, k = l / (n1 * n1);
    double s = 0.0;
    for (int c = 0; c < q; ++c) s = fma(sB[c * n1 + k], t1[(c * n1 + j) * n1 + i], s);
    const int g = dofmap[e * ne + l];
    if (g >= 0) F[g] += s;
  }
}

// Partial sums of sum_i w_i a_i b_i (w: nw weights repeated, or none) over a
// fixed block partition.
__global__ void wdot_kernel(const double* __restrict__ a, const double* __restrict__ b,
                            const double* __restrict__ w, int nw, int64_t n, double* partial) {
  __shared__ double red[SCF_THREADS];
  double s = 0.0;
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * per, i1 = min(n, i0 + per);
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const double t = a[i] * b[i];
    s = w ? fma(w[i % nw], t, s) : s + t;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = SCF_THREADS / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// y = a x + b y (x may be null: y = b y); z = x - y variants below.
__global__ void axpby_kernel(double* y, const double* x, double a, double b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = x ? fma(a, x[i], b * y[i]) : b * y[i];
}
__global__ void scale_kernel(double* y, const double* x, const double* s, double c, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = c * s[i] * x[i];
}
__global__ void fill_kernel(double* y, double v, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = v;
}
__global__ void sub_kernel(double* z, const double* x, const double* y, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) z[i] = x[i] - y[i];
}
__global__ void add_kernel(double* z, const double* x, const double* y, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) z[i] = x[i] + y[i];
}
// V_eff = phi + V_x(rho), V_x = -(3 rho / pi)^{1/3} for rho >= 0 (0 below)
__global__ void veff_kernel(double* v, const double* phi_q, const double* rho, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) v[i] = phi_q[i] - cbrt(3.0 * fmax(rho[i], 0.0) / 3.14159265358979323846);
}
// w jac V at the Gauss points of every cell (the matrix-free potential factor)
__global__ void wv_kernel(double* wv, const double* v, const double* W, int nq, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) wv[i] = W[i % nq] * v[i];
}

unsigned nblk(int64_t n) { return (unsigned)((n + SCF_THREADS - 1) / SCF_THREADS); }

chfsi_status sfail(chfsi_ctx* ctx, chfsi_status st, const std::string& m) {
  ctx->err = m;
  if (st == CHFSI_ERR_CUDA) ctx->latched = st;
  return st;
}

#define SK(call)                                                                                 \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return sfail(ctx, CHFSI_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Device buffers of the SCF / Poisson solves, owned by the context.
struct ScfBufs {
  double *mload, *ones, *F, *x, *r, *p, *Ap, *W, *part;
};

chfsi_status scf_grow(chfsi_ctx* ctx, DevBuf& b, size_t bytes) {
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
    return sfail(ctx, CHFSI_ERR_OOM, "SCF buffers: device allocation of " + std::to_string(bytes) + " bytes");
  }
  b.bytes = bytes;
  ctx->dev_bytes += (int64_t)bytes;
  return CHFSI_OK;
}

// Gauss weights with the Jacobian, point a + q (b + q c).
std::vector<double> qp_weights(const HostMesh& m) {
  const int q = m.q;
  const double jac = m.h[0] * m.h[1] * m.h[2] / 8.0;
  std::vector<double> W((size_t)q * q * q);
  for (int c = 0; c < q; ++c)
    for (int b = 0; b < q; ++b)
      for (int a = 0; a < q; ++a) W[(c * q + b) * q + a] = m.gq_w[a] * m.gq_w[b] * m.gq_w[c] * jac;
  return W;
}

// The 1-D factors of the matrix-free apply on the device (built on first use
// when the context has not been built).
chfsi_status ensure_factors(chfsi_ctx* ctx) {
  if (ctx->d_fac) return CHFSI_OK;
  build_mf_factors(ctx->mesh, ctx->fac);
  if (cudaMalloc(&ctx->d_fac, ctx->fac.size() * 8) != cudaSuccess) {
    cudaGetLastError();
    ctx->d_fac = nullptr;
    return sfail(ctx, CHFSI_ERR_OOM, "matrix-free factors");
  }
  ctx->dev_bytes += (int64_t)ctx->fac.size() * 8;
  SK(cudaMemcpyAsync(ctx->d_fac, ctx->fac.data(), ctx->fac.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
  return CHFSI_OK;
}

chfsi_status wdot(chfsi_ctx* ctx, ScfBufs& b, const double* x, const double* y, const double* w, int nw,
                  int64_t n, double* out);

// F (zeroed here) = int N_j f for f at the Gauss points, colour by colour.
chfsi_status load_vector(chfsi_ctx* ctx, ScfBufs& b, const double* f_qp, double* F) {
  const HostMesh& m = ctx->mesh;
  const int nq = m.q * m.q * m.q;
  SK(cudaMemsetAsync(F, 0, m.ndofs * 8, ctx->stream));
  const int ncolour = (int)m.colour_offsets.size() - 1;
  const size_t smem = ((size_t)nq + m.n1 * m.q * m.q + m.n1 * m.n1 * m.q + m.q * m.n1) * 8;
  const double* Bd = ctx->d_fac + 6 * m.n1 * m.n1;
  for (int c = 0; c < ncolour; ++c) {
    const int64_t nc = m.colour_offsets[c + 1] - m.colour_offsets[c];
    if (!nc) continue;
    note_launch();
    qp_load_kernel<<<(unsigned)nc, 128, smem, ctx->stream>>>(f_qp, b.W, ctx->d_cells + m.colour_offsets[c],
                                                             ctx->d_dofmap, Bd, m.n1, m.q, F);
    SK(cudaGetLastError());
  }
  return CHFSI_OK;
}

chfsi_status setup_bufs(chfsi_ctx* ctx, ScfBufs& b) {
  const HostMesh& m = ctx->mesh;
  const int64_t M = m.ndofs;
  const int nq = m.q * m.q * m.q;
  chfsi_status st;
  if ((st = ensure_factors(ctx)) != CHFSI_OK) return st;
  const size_t bytes = ((size_t)7 * M + nq + RED_BLOCKS + 64) * 8;
  const bool fresh = ctx->scfb.bytes < bytes || !ctx->scf_setup;
  if ((st = scf_grow(ctx, ctx->scfb, bytes)) != CHFSI_OK) return st;
  double* d = (double*)ctx->scfb.ptr;
  b.mload = d;
  b.ones = d + M;
  b.F = d + 2 * M;
  b.x = d + 3 * M;
  b.r = d + 4 * M;
  b.p = d + 5 * M;
  b.Ap = d + 6 * M;
  b.W = d + 7 * M;
  b.part = b.W + nq;
  if (fresh) {
    const std::vector<double> W = qp_weights(m);
    SK(cudaMemcpyAsync(b.W, W.data(), W.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    note_launch();
    fill_kernel<<<nblk(M), SCF_THREADS, 0, ctx->stream>>>(b.ones, 1.0, M);
    // m_j = int N_j (the load of f = 1), used to neutralise and to fix the mean
    const int64_t nqa = m.ncells * (int64_t)nq;
    if ((st = scf_grow(ctx, ctx->scfq, (size_t)nqa * 8)) != CHFSI_OK) return st;
    note_launch();
    fill_kernel<<<nblk(nqa), SCF_THREADS, 0, ctx->stream>>>((double*)ctx->scfq.ptr, 1.0, nqa);
    SK(cudaMemsetAsync(b.mload, 0, M * 8, ctx->stream));
    if ((st = load_vector(ctx, b, (const double*)ctx->scfq.ptr, b.mload)) != CHFSI_OK) return st;
    if ((st = wdot(ctx, b, b.mload, b.ones, nullptr, 1, M, &ctx->scf_msum)) != CHFSI_OK) return st;
    ctx->scf_setup = true;
  }
  return CHFSI_OK;
}

// sum w a b over n entries (w repeated with period nw, or null)
chfsi_status wdot(chfsi_ctx* ctx, ScfBufs& b, const double* x, const double* y, const double* w, int nw,
                  int64_t n, double* out) {
  note_launch();
  wdot_kernel<<<RED_BLOCKS, SCF_THREADS, 0, ctx->stream>>>(x, y, w, nw, n, b.part);
  SK(cudaGetLastError());
  double h[RED_BLOCKS];
  SK(cudaMemcpyAsync(h, b.part, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  SK(cudaStreamSynchronize(ctx->stream));
  double s = 0.0;
  for (int i = 0; i < RED_BLOCKS; ++i) s += h[i];
  *out = s;
  return CHFSI_OK;
}

// out = M^{-1/2} K M^{-1/2} in (the matrix-free kernel, kinetic part alone, times 2)
chfsi_status stiffness_apply(chfsi_ctx* ctx, const double* in, double* out) {
  const HostMesh& m = ctx->mesh;
  chfsi_status st;
  if ((st = scf_grow(ctx, ctx->Wb, (size_t)m.ndofs * 8)) != CHFSI_OK) return st;
  const int ncolour = (int)m.colour_offsets.size() - 1;
  for (int c = 0; c < ncolour; ++c) {
    MfLaunch L{};
    L.fac = ctx->d_fac;
    L.wv = nullptr;
    L.minv_sqrt = ctx->d_msq;
    L.dofmap = ctx->d_dofmap;
    L.modes = ctx->d_modes;
    L.cells = ctx->d_cells + m.colour_offsets[c];
    L.ncells_colour = m.colour_offsets[c + 1] - m.colour_offsets[c];
    L.p = m.p;
    L.q = m.q;
    L.ncol = 1;
    L.ld_in = L.ld_out = L.ld_prev = L.ld_w = 1;
    L.kinetic_only = 1;
    SK(launch_mf_cell_fp64(L, in, out, nullptr, (double*)ctx->Wb.ptr, nullptr, FilterStep{2.0, 0.0, 0.0},
                           ctx->stream));
  }
  return CHFSI_OK;
}

// Poisson solve K phi = 4 pi F (F = int N (f), neutralised), int phi = 0.
chfsi_status poisson_impl(chfsi_ctx* ctx, const double* f_qp, double* phi, double tol, int max_iter,
                          int* iters, double* rel) {
  const HostMesh& m = ctx->mesh;
  const int64_t M = m.ndofs;
  const int nq = m.q * m.q * m.q;
  ScfBufs b{};
  chfsi_status st;
  if ((st = setup_bufs(ctx, b)) != CHFSI_OK) return st;
  // F = int N_j f, neutralised: F -= (sum F) m / sum m
  if ((st = load_vector(ctx, b, f_qp, b.F)) != CHFSI_OK) return st;
  double fsum = 0.0;
  const double msum = ctx->scf_msum;
  if ((st = wdot(ctx, b, b.F, b.ones, nullptr, 1, M, &fsum)) != CHFSI_OK) return st;
  note_launch();
  axpby_kernel<<<nblk(M), SCF_THREADS, 0, ctx->stream>>>(b.F, b.mload, -fsum / msum, 1.0, M);
  // scaled right-hand side r = 4 pi M^{-1/2} F, x = 0
  note_launch();
  scale_kernel<<<nblk(M), SCF_THREADS, 0, ctx->stream>>>(b.r, b.F, ctx->d_msq, 4.0 * M_PI, M);
  SK(cudaMemsetAsync(b.x, 0, M * 8, ctx->stream));
  SK(cudaMemcpyAsync(b.p, b.r, M * 8, cudaMemcpyDeviceToDevice, ctx->stream));
  double rr = 0.0, bb = 0.0;
  if ((st = wdot(ctx, b, b.r, b.r, nullptr, 1, M, &rr)) != CHFSI_OK) return st;
  bb = rr;
  int it = 0;
  double res = bb > 0.0 ? 1.0 : 0.0;
  for (; it < max_iter && bb > 0.0 && std::sqrt(rr) > tol * std::sqrt(bb); ++it) {
    if ((st = stiffness_apply(ctx, b.p, b.Ap)) != CHFSI_OK) return st;
    double pAp = 0.0;
    if ((st = wdot(ctx, b, b.p, b.Ap, nullptr, 1, M, &pAp)) != CHFSI_OK) return st;
    if (!(pAp > 0.0)) break;
    const double alpha = rr / pAp;
    note_launch();
    axpby_kernel<<<nblk(M), SCF_THREADS, 0, ctx->stream>>>(b.x, b.p, alpha, 1.0, M);
    note_launch();
    axpby_kernel<<<nblk(M), SCF_THREADS, 0, ctx->stream>>>(b.r, b.Ap, -alpha, 1.0, M);
    double rn = 0.0;
    if ((st = wdot(ctx, b, b.r, b.r, nullptr, 1, M, &rn)) != CHFSI_OK) return st;
    note_launch();
    axpby_kernel<<<nblk(M), SCF_THREADS, 0, ctx->stream>>>(b.p, b.r, 1.0, rn / rr, M);
    rr = rn;
  }
  if (bb > 0.0) res = std::sqrt(rr / bb);
  // phi = M^{-1/2} x, then the mean fixed: phi -= (m . phi) / sum m
  note_launch();
  scale_kernel<<<nblk(M), SCF_THREADS, 0, ctx->stream>>>(phi, b.x, ctx->d_msq, 1.0, M);
  double mphi = 0.0;
  if ((st = wdot(ctx, b, b.mload, phi, nullptr, 1, M, &mphi)) != CHFSI_OK) return st;
  note_launch();
  axpby_kernel<<<nblk(M), SCF_THREADS, 0, ctx->stream>>>(phi, b.ones, -mphi / msum, 1.0, M);
  SK(cudaStreamSynchronize(ctx->stream));
  if (iters) *iters = it;
  if (rel) *rel = res;
  if (res > tol && bb > 0.0)
    return sfail(ctx, CHFSI_ERR_EIG, "Poisson CG: relative residual " + std::to_string(res) + " after " +
                                         std::to_string(it) + " iterations");
  return CHFSI_OK;
}

}  // namespace

namespace {

// Gauss points of cell e, point a + q (b + q c).
void cell_qp(const HostMesh& m, int64_t e, std::vector<double>& xq) {
  const int q = m.q;
  const int c3[3] = {(int)(e % m.n[0]), (int)((e / m.n[0]) % m.n[1]), (int)(e / ((int64_t)m.n[0] * m.n[1]))};
  xq.resize((size_t)q * q * q * 3);
  for (int c = 0; c < q; ++c)
    for (int b = 0; b < q; ++b)
      for (int a = 0; a < q; ++a) {
        const int pt = (c * q + b) * q + a;
        const int ia[3] = {a, b, c};
        for (int ax = 0; ax < 3; ++ax)
          xq[pt * 3 + ax] = (c3[ax] + (m.gq_x[ia[ax]] + 1.0) / 2.0) * m.h[ax];
      }
}

// b(x) = -sum_I Z_I (2 pi s_I^2)^{-3/2} exp(-|x - R_I|^2 / (2 s_I^2)) over the
// 27 periodic images (the oracle's nuclear charge, reading R25).
double nuclear_charge(const double* x, const chfsi_scf_params& p, const double* len, double smin) {
  double b = 0.0;
  for (int I = 0; I < p.nnuclei; ++I) {
    const double s = std::max(p.sigma[I], smin);
    const double nrm = p.Z[I] / std::pow(2.0 * M_PI * s * s, 1.5);
    for (int sz = -1; sz <= 1; ++sz)
      for (int sy = -1; sy <= 1; ++sy)
        for (int sx = -1; sx <= 1; ++sx) {
          const double d0 = x[0] - (p.xyz[3 * I] + sx * len[0]);
          const double d1 = x[1] - (p.xyz[3 * I + 1] + sy * len[1]);
          const double d2 = x[2] - (p.xyz[3 * I + 2] + sz * len[2]);
          b -= nrm * std::exp(-(d0 * d0 + d1 * d1 + d2 * d2) / (2.0 * s * s));
        }
  }
  return b;
}

// Small dense solve G t = rhs (Gaussian elimination, partial pivoting); false
// when G is numerically singular.
bool small_solve(std::vector<double> G, std::vector<double> rhs, int n, std::vector<double>& t) {
  double scale = 0.0;
  for (int i = 0; i < n; ++i) scale = std::max(scale, std::fabs(G[i * n + i]));
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(G[i * n + k]) > std::fabs(G[piv * n + k])) piv = i;
    if (!(std::fabs(G[piv * n + k]) > 1e-13 * scale)) return false;
    if (piv != k) {
      for (int j = 0; j < n; ++j) std::swap(G[k * n + j], G[piv * n + j]);
      std::swap(rhs[k], rhs[piv]);
    }
    for (int i = k + 1; i < n; ++i) {
      const double f = G[i * n + k] / G[k * n + k];
      for (int j = k; j < n; ++j) G[i * n + j] -= f * G[k * n + j];
      rhs[i] -= f * rhs[k];
    }
  }
  t.assign(n, 0.0);
  for (int i = n - 1; i >= 0; --i) {
    double s = rhs[i];
    for (int j = i + 1; j < n; ++j) s -= G[i * n + j] * t[j];
    t[i] = s / G[i * n + i];
  }
  return true;
}

}  // namespace

extern "C" {

chfsi_status chfsi_set_potential_qp_device(chfsi_ctx* ctx, const double* v) {
  if (!ctx) return CHFSI_ERR_ARG;
  if (ctx->latched != CHFSI_OK) return ctx->latched;
  const HostMesh& m = ctx->mesh;
  if (!v) return sfail(ctx, CHFSI_ERR_ARG, "potential values: null pointer");
  if (!mf_supported(m.p, m.q))
    return sfail(ctx, CHFSI_ERR_ARG, "a device potential needs the matrix-free operator (2 <= p <= 8, q = p + 2)");
  chfsi_status st;
  if ((st = ensure_factors(ctx)) != CHFSI_OK) return st;
  const int nq = m.q * m.q * m.q;
  const int64_t n = m.ncells * (int64_t)nq;
  SK(cudaStreamSynchronize(ctx->stream));
  // the stored cell matrices (and their packed copies) belong to the old potential
  if (ctx->d_Ht) {
    cudaFree(ctx->d_Ht);
    ctx->dev_bytes -= (int64_t)m.ncells * m.ne * m.ne * 8;
    ctx->d_Ht = nullptr;
  }
  ctx->dev_bytes -= (int64_t)(ctx->tc.bytes + ctx->tc.bf_bytes + ctx->tc.f16_bytes + ctx->tc.nl_bytes +
                              ctx->tc.pj_bytes);
  ctx->kpack_valid = false;
  tc_free(ctx->tc);
  ctx->tc.ncells = m.ncells;
  ctx->tc.ne = m.ne;
  if (!ctx->d_wv || ctx->wv.size() != (size_t)n) {
    if (ctx->d_wv) {
      cudaFree(ctx->d_wv);
      ctx->dev_bytes -= (int64_t)ctx->wv.size() * 8;
      ctx->d_wv = nullptr;
    }
    ctx->wv.assign((size_t)n, 0.0);
    if (cudaMalloc(&ctx->d_wv, (size_t)n * 8) != cudaSuccess) {
      cudaGetLastError();
      ctx->d_wv = nullptr;
      ctx->wv.clear();
      return sfail(ctx, CHFSI_ERR_OOM, "potential factor");
    }
    ctx->dev_bytes += n * 8;
  }
  const std::vector<double> W = qp_weights(m);
  if ((st = scf_grow(ctx, ctx->scfw, W.size() * 8)) != CHFSI_OK) return st;
  SK(cudaMemcpyAsync(ctx->scfw.ptr, W.data(), W.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
  note_launch();
  wv_kernel<<<nblk(n), SCF_THREADS, 0, ctx->stream>>>(ctx->d_wv, v, (const double*)ctx->scfw.ptr, nq, n);
  SK(cudaGetLastError());
  SK(cudaStreamSynchronize(ctx->stream));
  ctx->fp64_op = 1;
  ctx->built = true;
  ++ctx->build_gen;
  return CHFSI_OK;
}

chfsi_status chfsi_poisson(chfsi_ctx* ctx, const double* f, double* phi, double tol, int max_iter,
                           int* iters, double* rel_residual) {
  if (!ctx) return CHFSI_ERR_ARG;
  if (ctx->latched != CHFSI_OK) return ctx->latched;
  const HostMesh& m = ctx->mesh;
  if (!f || !phi || !(tol > 0.0) || max_iter < 1) return sfail(ctx, CHFSI_ERR_ARG, "bad Poisson arguments");
  if (!m.per[0] || !m.per[1] || !m.per[2]) return sfail(ctx, CHFSI_ERR_ARG, "the Poisson solve is for periodic meshes");
  if (!mf_supported(m.p, m.q)) return sfail(ctx, CHFSI_ERR_ARG, "the Poisson solve needs 2 <= p <= 8, q = p + 2");
  return poisson_impl(ctx, f, phi, tol, max_iter, iters, rel_residual);
}

chfsi_status chfsi_scf(chfsi_ctx* ctx, const chfsi_scf_params* prm, double* X, int64_t ldx,
                       double* rho_host, double* evals_host, double* occ_host, double* mu_out,
                       double* res_hist, int* iters_out) {
  if (!ctx || !prm) return CHFSI_ERR_ARG;
  if (ctx->latched != CHFSI_OK) return ctx->latched;
  const chfsi_scf_params& P = *prm;
  const HostMesh& m = ctx->mesh;
  const int n = P.n_states;
  if (!m.per[0] || !m.per[1] || !m.per[2]) return sfail(ctx, CHFSI_ERR_ARG, "the SCF loop is for periodic meshes");
  if (!mf_supported(m.p, m.q)) return sfail(ctx, CHFSI_ERR_ARG, "the SCF loop needs 2 <= p <= 8, q = p + 2");
  if (P.nnuclei < 1 || !P.xyz || !P.Z || !P.sigma || n < 1 || !X || ldx < n || !(P.kT > 0.0) ||
      P.degree < 1 || P.passes < 1 || !(P.tol > 0.0) || P.max_iter < 1 || !(P.beta > 0.0) ||
      P.depth < 1 || P.depth > 16 || !(P.poisson_tol > 0.0) || P.lanczos_steps < 2 || !evals_host)
    return sfail(ctx, CHFSI_ERR_ARG, "bad SCF parameters");
  if (!ctx->proj.h.empty()) return sfail(ctx, CHFSI_ERR_ARG, "the SCF loop takes no nonlocal projectors");
  double n_el = 0.0;
  for (int I = 0; I < P.nnuclei; ++I) n_el += P.Z[I];
  if (!(2.0 * n >= n_el)) return sfail(ctx, CHFSI_ERR_ARG, "too few states for the electrons");
  chfsi_status st;
  ScfBufs b{};
  if ((st = setup_bufs(ctx, b)) != CHFSI_OK) return st;
  const int nq = m.q * m.q * m.q;
  const int64_t nqa = m.ncells * (int64_t)nq, M = m.ndofs;
  const int D = P.depth;
  // qp arrays: rho, bq, f, phiq, vq, rho_out, tmp, hist x[D], hist r[D]; nodal phi
  if ((st = scf_grow(ctx, ctx->scfr, ((size_t)(7 + 2 * D) * nqa + M) * 8)) != CHFSI_OK) return st;
  double* rho = (double*)ctx->scfr.ptr;
  double* bq = rho + nqa;
  double* f = bq + nqa;
  double* phiq = f + nqa;
  double* vq = phiq + nqa;
  double* rout = vq + nqa;
  double* tmp = rout + nqa;
  double* hx = tmp + nqa;
  double* hr = hx + (size_t)D * nqa;
  double* phi = hr + (size_t)D * nqa;
  // nuclear charge and the initial density (nuclei widened to 1 bohr, scaled to N_e)
  {
    std::vector<double> hb((size_t)nqa), hr0((size_t)nqa), xq;
    const std::vector<double> W = qp_weights(m);
    double tot = 0.0;
    for (int64_t e = 0; e < m.ncells; ++e) {
      cell_qp(m, e, xq);
      for (int pt = 0; pt < nq; ++pt) {
        hb[e * nq + pt] = nuclear_charge(&xq[pt * 3], P, m.len, 0.0);
        hr0[e * nq + pt] = -nuclear_charge(&xq[pt * 3], P, m.len, 1.0);
        tot += hr0[e * nq + pt] * W[pt];
      }
    }
    for (auto& v : hr0) v *= n_el / tot;
    SK(cudaMemcpyAsync(bq, hb.data(), nqa * 8, cudaMemcpyHostToDevice, ctx->stream));
    SK(cudaMemcpyAsync(rho, hr0.data(), nqa * 8, cudaMemcpyHostToDevice, ctx->stream));
    SK(cudaStreamSynchronize(ctx->stream));
  }
  // start block: the seeded uniform draws, orthonormalised by the first RR's CholGS
  if ((st = chfsi_fill_uniform(ctx, X, ldx, M, n, P.seed, 1, CHFSI_FP64)) != CHFSI_OK) return st;
  std::vector<double> Dv(n), occ(n), hist;
  std::vector<int> ring;                   // history slots, oldest first
  double mu = 0.0;
  bool first = true;
  int it = 0;
  for (; it < P.max_iter; ++it) {
    // ES and V_eff
    note_launch();
    add_kernel<<<nblk(nqa), SCF_THREADS, 0, ctx->stream>>>(f, rho, bq, nqa);
    if ((st = poisson_impl(ctx, f, phi, P.poisson_tol, 20000, nullptr, nullptr)) != CHFSI_OK) return st;
    const size_t ism = ((size_t)m.ne + m.n1 * m.n1 * m.q + m.n1 * m.q * m.q + m.q * m.n1) * 8;
    note_launch();
    qp_interp_kernel<<<(unsigned)m.ncells, 128, ism, ctx->stream>>>(phi, ctx->d_dofmap,
                                                                     ctx->d_fac + 6 * m.n1 * m.n1, m.n1,
                                                                     m.q, phiq);
    note_launch();
    veff_kernel<<<nblk(nqa), SCF_THREADS, 0, ctx->stream>>>(vq, phiq, rho, nqa);
    SK(cudaGetLastError());
    if ((st = chfsi_set_potential_qp_device(ctx, vq)) != CHFSI_OK) return st;
    // ChFSI passes (binary64, warm-started)
    double bup = 0.0;
    if ((st = chfsi_bounds(ctx, P.lanczos_steps, P.seed + 1000 + it, &bup)) != CHFSI_OK) return st;
    if (first && (st = chfsi_cholgs(ctx, X, ldx, n, CHFSI_FP64)) != CHFSI_OK) return st;
    first = false;
    if ((st = chfsi_rayleigh_ritz(ctx, X, ldx, n, CHFSI_FP64, Dv.data())) != CHFSI_OK) return st;
    for (int k = 0; k < P.passes; ++k) {
      double a = Dv[n - 1], a0 = Dv[0];
      if (!(a0 < a)) a0 = a - 1e-3 * std::max(1.0, std::fabs(a));
      if (!(a < bup)) bup = a + std::max(1.0, std::fabs(a));
      if ((st = chfsi_filter(ctx, X, ldx, n, P.degree, a, bup, a0, CHFSI_FP64)) != CHFSI_OK) return st;
      if ((st = chfsi_cholgs(ctx, X, ldx, n, CHFSI_FP64)) != CHFSI_OK) return st;
      if ((st = chfsi_rayleigh_ritz(ctx, X, ldx, n, CHFSI_FP64, Dv.data())) != CHFSI_OK) return st;
    }
    // DC: occupations of all states, density at the Gauss points
    if ((st = chfsi_fermi_level(n, Dv.data(), 0, n_el, P.kT, &mu, occ.data())) != CHFSI_OK)
      return sfail(ctx, st, "Fermi level");
    if ((st = chfsi_density(ctx, X, ldx, n, X, ldx, n, occ.data(), CHFSI_FP64, rout)) != CHFSI_OK) return st;
    // residual |rho_out - rho|_W
    note_launch();
    sub_kernel<<<nblk(nqa), SCF_THREADS, 0, ctx->stream>>>(tmp, rout, rho, nqa);
    double rr = 0.0;
    if ((st = wdot(ctx, b, tmp, tmp, b.W, nq, nqa, &rr)) != CHFSI_OK) return st;
    const double res = std::sqrt(rr);
    hist.push_back(res);
    if (res < P.tol) {
      SK(cudaMemcpyAsync(rho, rout, nqa * 8, cudaMemcpyDeviceToDevice, ctx->stream));
      ++it;
      break;
    }
    // Anderson mixing: history (x_i, r_i); minimise |r_m + sum t_i (r_i - r_m)|_W
    int slot = (int)ring.size() < D ? (int)ring.size() : ring.front();
    if ((int)ring.size() == D) ring.erase(ring.begin());
    ring.push_back(slot);
    SK(cudaMemcpyAsync(hx + (size_t)slot * nqa, rho, nqa * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    SK(cudaMemcpyAsync(hr + (size_t)slot * nqa, tmp, nqa * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    const int mh = (int)ring.size();
    std::vector<double> c(mh, 0.0);
    if (mh == 1) {
      c[0] = 1.0;
    } else {
      std::vector<double> Gr((size_t)mh * mh);
      for (int i = 0; i < mh; ++i)
        for (int j = 0; j <= i; ++j) {
          double v = 0.0;
          if ((st = wdot(ctx, b, hr + (size_t)ring[i] * nqa, hr + (size_t)ring[j] * nqa, b.W, nq, nqa, &v)) != CHFSI_OK)
            return st;
          Gr[i * mh + j] = Gr[j * mh + i] = v;
        }
      const int k = mh - 1, last = mh - 1;
      std::vector<double> G((size_t)k * k), g(k), t;
      for (int i = 0; i < k; ++i) {
        for (int j = 0; j < k; ++j)
          G[i * k + j] = Gr[i * mh + j] - Gr[i * mh + last] - Gr[last * mh + j] + Gr[last * mh + last];
        g[i] = -(Gr[i * mh + last] - Gr[last * mh + last]);
      }
      if (small_solve(G, g, k, t)) {
        double ts = 0.0;
        for (int i = 0; i < k; ++i) {
          c[i] = t[i];
          ts += t[i];
        }
        c[last] = 1.0 - ts;
      } else {
        c.assign(mh, 0.0);
        c[last] = 1.0;
      }
    }
    SK(cudaMemsetAsync(rho, 0, nqa * 8, ctx->stream));
    for (int i = 0; i < mh; ++i) {
      note_launch();
      axpby_kernel<<<nblk(nqa), SCF_THREADS, 0, ctx->stream>>>(rho, hx + (size_t)ring[i] * nqa, c[i], 1.0, nqa);
      note_launch();
      axpby_kernel<<<nblk(nqa), SCF_THREADS, 0, ctx->stream>>>(rho, hr + (size_t)ring[i] * nqa, c[i] * P.beta,
                                                                 1.0, nqa);
    }
    SK(cudaGetLastError());
  }
  SK(cudaStreamSynchronize(ctx->stream));
  if (rho_host) SK(cudaMemcpy(rho_host, rho, nqa * 8, cudaMemcpyDeviceToHost));
  std::memcpy(evals_host, Dv.data(), (size_t)n * 8);
  if (occ_host) std::memcpy(occ_host, occ.data(), (size_t)n * 8);
  if (mu_out) *mu_out = mu;
  if (res_hist) std::memcpy(res_hist, hist.data(), hist.size() * 8);
  if (iters_out) *iters_out = it;
  if (hist.empty() || hist.back() >= P.tol)
    return sfail(ctx, CHFSI_ERR_EIG, "SCF did not reach the residual tolerance in " + std::to_string(P.max_iter) +
                                         " iterations (last " + std::to_string(hist.empty() ? 0.0 : hist.back()) + ")");
  return CHFSI_OK;
}

}  // extern "C"
