// Electron density at the Gauss points of every cell (Algorithm dc, Eq.
// elecDensSP of arXiv:1903.10959) and the Fermi level of the partially
// occupied states.
//
//   rho(x_q) = 2 sum_i psi_i(x_q)^2 + 2 sum_j (f_j - 1) psi_fr,j(x_q)^2,
//   psi = M^{-1/2} x (x: columns of X or X_fr), interpolated from the cell's
//   GLL nodes to its q^3 Gauss points by sum factorisation: three passes of
//   the 1-D matrix B (q x (p+1)), one per direction, in the block's precision
//   (binary64 or binary32); the sum over the columns is binary64.
//
// One CTA per cell loops over the columns in chunks of CB and keeps the
// density of its points in registers, so every point is summed in a fixed
// order (deterministic, no atomics).
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace chfsi {

constexpr int DEN_THREADS = 256;
constexpr int DEN_MAXPT = 4;          // points per thread: q^3 <= 1024 (p <= 8)
constexpr int DEN_MAXN = 9;           // nodes per direction: p <= 8

struct DenSmem {
  int cb, psi, t1, t2, v, total;      // columns per chunk and region offsets (doubles)
};

__host__ __device__ inline DenSmem den_smem(int n1, int q, int cb) {   // in elements
  DenSmem d;
  d.cb = cb;
  const int ne = n1 * n1 * n1;
  d.psi = 0;
  d.t1 = d.psi + ne * cb;
  d.t2 = d.t1 + n1 * n1 * q * cb;
  d.v = d.t2 + n1 * q * q * cb;
  d.total = d.v + q * q * q * cb;
  return d;
}

template <typename T>
__global__ void __launch_bounds__(DEN_THREADS) density_kernel(
    const T* __restrict__ X, int64_t ldx, int n, const T* __restrict__ Xfr, int64_t ldfr, int nfr,
    const double* __restrict__ wfr, const int32_t* __restrict__ dofmap,
    const double* __restrict__ minv_sqrt, const double* __restrict__ Bg, int n1, int q, int cb,
    double* __restrict__ rho) {
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  T* dsm = reinterpret_cast<T*>(dsm_raw);
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x;
  const int ne = n1 * n1 * n1, nq = q * q * q;
  const DenSmem L = den_smem(n1, q, cb);
  __shared__ T sB[16 * 16];
  __shared__ T sms[1024];
  __shared__ int sdm[1024];
  for (int t = tid; t < q * n1; t += DEN_THREADS) sB[t] = (T)Bg[t];
  for (int l = tid; l < ne; l += DEN_THREADS) {
    const int g = dofmap[e * ne + l];
    sdm[l] = g;
    sms[l] = g >= 0 ? (T)minv_sqrt[g] : (T)0;
  }
  double acc[DEN_MAXPT];
#pragma unroll
  for (int u = 0; u < DEN_MAXPT; ++u) acc[u] = 0.0;
  T* Psi = dsm + L.psi;
  T* T1 = dsm + L.t1;
  T* T2 = dsm + L.t2;
  T* V = dsm + L.v;
  __syncthreads();
  const int nchunk_x = (n + cb - 1) / cb, nchunk = nchunk_x + (nfr + cb - 1) / cb;
  for (int ch = 0; ch < nchunk; ++ch) {
    const bool fr = ch >= nchunk_x;
    const int c0 = (fr ? ch - nchunk_x : ch) * cb;
    const int ncol = fr ? nfr : n;
    const int cv = min(cb, ncol - c0);
    const T* src = fr ? Xfr : X;
    const int64_t ld = fr ? ldfr : ldx;
    // 1. psi at the cell's nodes: M^{-1/2} x, zero at eliminated nodes and unused columns
    for (int t = tid; t < ne * cb; t += DEN_THREADS) {
      const int l = t / cb, c = t - l * cb;
      const int g = sdm[l];
      Psi[t] = (g >= 0 && c < cv) ? sms[l] * src[(int64_t)g * ld + c0 + c] : (T)0;
    }
    __syncthreads();
    // Each thread contracts one line: it keeps the line's n1 inputs in
    // registers and produces all q outputs, so the (line, column) index is
    // split once per line rather than once per output.
    // 2. x direction: T1[k][j][a][c] = sum_i B[a][i] Psi[(k n1 + j) n1 + i][c]
    for (int t = tid; t < n1 * n1 * cb; t += DEN_THREADS) {
      const int c = t % cb, kj = t / cb;
      T in[DEN_MAXN];
#pragma unroll
      for (int i = 0; i < DEN_MAXN; ++i) in[i] = i < n1 ? Psi[((int64_t)kj * n1 + i) * cb + c] : (T)0;
      for (int a = 0; a < q; ++a) {
        T s = 0;
#pragma unroll
        for (int i = 0; i < DEN_MAXN; ++i)
          if (i < n1) s = fma(sB[a * n1 + i], in[i], s);
        T1[((int64_t)kj * q + a) * cb + c] = s;
      }
    }
    __syncthreads();
    // 3. y direction: T2[k][b][a][c] = sum_j B[b][j] T1[k][j][a][c]
    for (int t = tid; t < n1 * q * cb; t += DEN_THREADS) {
      const int c = t % cb, r = t / cb;
      const int a = r % q, k = r / q;
      T in[DEN_MAXN];
#pragma unroll
      for (int j2 = 0; j2 < DEN_MAXN; ++j2)
        in[j2] = j2 < n1 ? T1[(((int64_t)k * n1 + j2) * q + a) * cb + c] : (T)0;
      for (int b = 0; b < q; ++b) {
        T s = 0;
#pragma unroll
        for (int j2 = 0; j2 < DEN_MAXN; ++j2)
          if (j2 < n1) s = fma(sB[b * n1 + j2], in[j2], s);
        T2[(((int64_t)k * q + b) * q + a) * cb + c] = s;
      }
    }
    __syncthreads();
    // 4. z direction: V[cz][b][a][c] = sum_k B[cz][k] T2[k][b][a][c]  (point a + q (b + q cz))
    for (int t = tid; t < q * q * cb; t += DEN_THREADS) {
      const int c = t % cb, ab = t / cb;
      T in[DEN_MAXN];
#pragma unroll
      for (int k = 0; k < DEN_MAXN; ++k)
        in[k] = k < n1 ? T2[((int64_t)k * q * q + ab) * cb + c] : (T)0;
      for (int cz = 0; cz < q; ++cz) {
        T s = 0;
#pragma unroll
        for (int k = 0; k < DEN_MAXN; ++k)
          if (k < n1) s = fma(sB[cz * n1 + k], in[k], s);
        V[((int64_t)cz * q * q + ab) * cb + c] = s;
      }
    }
    __syncthreads();
    // 5. rho += w_c psi_c^2 with w = 2 (X) or 2 (f - 1) (X_fr)
#pragma unroll
    for (int u = 0; u < DEN_MAXPT; ++u) {
      const int pt = tid + u * DEN_THREADS;
      if (pt >= nq) break;
      double s = 0.0;
      for (int c = 0; c < cv; ++c) {
        const double v = (double)V[pt * cb + c];
        s = fma(fr ? wfr[c0 + c] : 2.0, v * v, s);
      }
      acc[u] += s;
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < DEN_MAXPT; ++u) {
    const int pt = tid + u * DEN_THREADS;
    if (pt < nq) rho[e * nq + pt] = acc[u];
  }
}

cudaError_t launch_density(const DensityArgs& a, cudaStream_t s) {
  if (a.ncells == 0) return cudaSuccess;
  const int nq = a.q * a.q * a.q;
  if (a.q * a.n1 > 256 || nq > DEN_MAXPT * DEN_THREADS || a.n1 > DEN_MAXN)
    return cudaErrorInvalidValue;
  const size_t es = a.is_double ? 8 : 4;
  int cb = 8;
  while (cb > 1 && den_smem(a.n1, a.q, cb).total * es > 100 * 1024) cb /= 2;   // two CTAs per SM
  const size_t smem = (size_t)den_smem(a.n1, a.q, cb).total * es;
  if (a.is_double) {
    cudaFuncSetAttribute(density_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    note_launch();
    density_kernel<double><<<(unsigned)a.ncells, DEN_THREADS, smem, s>>>(
        (const double*)a.X, a.ldx, a.n, (const double*)a.Xfr, a.ldfr, a.nfr, a.wfr, a.dofmap,
        a.minv_sqrt, a.B, a.n1, a.q, cb, a.rho);
  } else {
    cudaFuncSetAttribute(density_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    note_launch();
    density_kernel<float><<<(unsigned)a.ncells, DEN_THREADS, smem, s>>>(
        (const float*)a.X, a.ldx, a.n, (const float*)a.Xfr, a.ldfr, a.nfr, a.wfr, a.dofmap,
        a.minv_sqrt, a.B, a.n1, a.q, cb, a.rho);
  }
  return cudaGetLastError();
}

// Fermi-Dirac occupation 1 / (1 + exp((eps - mu) / kT)), evaluated without overflow.
static double fermi_dirac(double eps, double mu, double kT) {
  const double t = (eps - mu) / kT;
  if (t > 0) {
    const double x = std::exp(-t);
    return x / (1.0 + x);
  }
  return 1.0 / (1.0 + std::exp(t));
}

}  // namespace chfsi

extern "C" chfsi_status chfsi_fermi_level(int n, const double* evals, int n_oc, double n_electrons,
                                         double kT, double* mu_out, double* occ_out) {
  using chfsi::fermi_dirac;
  if (n < 1 || !evals || n_oc < 0 || !(kT > 0) || !mu_out || !std::isfinite(n_electrons))
    return CHFSI_ERR_ARG;
  double lo = evals[0], hi = evals[0];
  for (int i = 0; i < n; ++i) {
    lo = std::min(lo, evals[i]);
    hi = std::max(hi, evals[i]);
  }
  lo -= 60.0 * kT;
  hi += 60.0 * kT;
  auto count = [&](double mu) {
    double f = 0.0;
    for (int i = 0; i < n; ++i) f += fermi_dirac(evals[i], mu, kT);
    return 2.0 * (n_oc + f);
  };
  if (!(count(lo) <= n_electrons && n_electrons <= count(hi))) return CHFSI_ERR_ARG;
  for (int it = 0; it < 400; ++it) {   // the count increases with mu: bisection
    const double mid = 0.5 * (lo + hi);
    if (count(mid) < n_electrons) lo = mid;
    else hi = mid;
    if (hi - lo <= 1e-15 * std::max(1.0, std::fabs(mid))) break;
  }
  const double mu = 0.5 * (lo + hi);
  *mu_out = mu;
  if (occ_out)
    for (int i = 0; i < n; ++i) occ_out[i] = fermi_dirac(evals[i], mu, kT);
  return CHFSI_OK;
}
