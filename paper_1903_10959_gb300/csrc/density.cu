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

// Binary32 blocks, q = n1 + 1 (the default rule): the same three passes with
// the lane as the column.  A CTA takes its cell's columns 32 at a time; every
// buffer is [line element][32 columns], so each warp access is one
// conflict-free row of shared memory and each gather load one 128-byte row of
// X.  The 1-D matrix B lives in the kernel's parameter space (its entries are
// constant-bank operands of the FMAs), the passes are fully unrolled for the
// degree, and the z pass never stores its output: each lane squares its q
// values, weights them by its column's weight, and the warp sums them over its
// 32 columns by a reduce-scatter (log2 of the padded q halving steps, then the
// remaining butterfly steps), which leaves every point's chunk sum on four
// lanes.  The lane with (lane & 3) == 0 adds it to that point's accumulator,
// a pair of binary32 words updated by Knuth's two-sum (about 44 bits; binary64
// adds would cost a pass of the GB300's two-per-clock binary64 pipe per line),
// so the column sum is binary32 within a chunk of 32 columns and carries the
// pair's precision across chunks, in a fixed order (deterministic).
constexpr int DEN32_THREADS = 256, DEN32_WARPS = DEN32_THREADS / 32;
struct DenB {
  float b[10 * 9];   // B (q x n1), row-major, q = n1 + 1 <= 10
};

template <int N1>
struct Den32 {
  static constexpr int Q = N1 + 1, NE = N1 * N1 * N1, NQ = Q * Q * Q;
  static constexpr int LA = NE > N1 * Q * Q ? NE : N1 * Q * Q;   // psi, then the y pass output
  static constexpr int LB = N1 * N1 * Q;                         // the x pass output
  static constexpr int P2 = Q <= 4 ? 4 : (Q <= 8 ? 8 : 16);      // q padded to a power of two
  static constexpr int LG = P2 == 4 ? 2 : (P2 == 8 ? 3 : 4);
  static constexpr int LPW = (Q * Q + DEN32_WARPS - 1) / DEN32_WARPS;   // z lines per warp
  static constexpr size_t SMEM = (size_t)(LA + LB) * 32 * 4 + (size_t)NE * 8;
  static constexpr int MINB = SMEM <= 110 * 1024 + 512 ? 2 : 1;   // CTAs per SM the shared memory allows
};

template <int N1>
__global__ void __launch_bounds__(DEN32_THREADS, Den32<N1>::MINB) density32_kernel(
    const float* __restrict__ X, int64_t ldx, int n, const float* __restrict__ Xfr, int64_t ldfr,
    int nfr, const double* __restrict__ wfr, const int32_t* __restrict__ dofmap,
    const double* __restrict__ minv_sqrt, const DenB Bc, double* __restrict__ rho) {
  using D = Den32<N1>;
  constexpr int Q = D::Q, NE = D::NE, P2 = D::P2;
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  float* bufA = reinterpret_cast<float*>(dsm_raw);
  float* bufB = bufA + D::LA * 32;
  int32_t* sdm = reinterpret_cast<int32_t*>(bufB + D::LB * 32);
  float* sms = reinterpret_cast<float*>(sdm + NE);
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int l = tid; l < NE; l += DEN32_THREADS) {
    const int g = dofmap[e * NE + l];
    sdm[l] = g;
    sms[l] = g >= 0 ? (float)minv_sqrt[g] : 0.f;
  }
  float acc_h[D::LPW], acc_l[D::LPW];   // the point's sum as hi + lo
#pragma unroll
  for (int m = 0; m < D::LPW; ++m) acc_h[m] = acc_l[m] = 0.f;
  __syncthreads();
  const int nchunk_x = (n + 31) / 32, nchunk = nchunk_x + (nfr + 31) / 32;
  for (int ch = 0; ch < nchunk; ++ch) {
    const bool fr = ch >= nchunk_x;
    const int c0 = (fr ? ch - nchunk_x : ch) * 32;
    const int cv = min(32, (fr ? nfr : n) - c0);
    const float* src = (fr ? Xfr : X) + c0 + lane;
    const int64_t ld = fr ? ldfr : ldx;
    const bool live = lane < cv;
    const float w = !live ? 0.f : (fr ? (float)wfr[c0 + lane] : 2.f);
    // 1. psi = M^{-1/2} x at the cell's nodes, one row of 32 columns per warp access
    for (int l0 = warp; l0 < NE; l0 += 4 * DEN32_WARPS) {
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int l = l0 + u * DEN32_WARPS;
        const int g = l < NE ? sdm[l] : -1;
        v[u] = (g >= 0 && live) ? __ldg(src + (int64_t)g * ld) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int l = l0 + u * DEN32_WARPS;
        if (l < NE) bufA[l * 32 + lane] = sms[l] * v[u];
      }
    }
    __syncthreads();
    // 2. x: bufB[(k n1 + j) q + a] = sum_i B[a][i] psi[(k n1 + j) n1 + i]
    for (int kj = warp; kj < N1 * N1; kj += DEN32_WARPS) {
      float in[N1];
#pragma unroll
      for (int i = 0; i < N1; ++i) in[i] = bufA[(kj * N1 + i) * 32 + lane];
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < N1; ++i) s = fmaf(Bc.b[a * N1 + i], in[i], s);
        bufB[(kj * Q + a) * 32 + lane] = s;
      }
    }
    __syncthreads();
    // 3. y: bufA[(k q + b) q + a] = sum_j B[b][j] bufB[(k n1 + j) q + a]
    for (int r = warp; r < N1 * Q; r += DEN32_WARPS) {
      const int k = r / Q, a = r - k * Q;
      float in[N1];
#pragma unroll
      for (int j = 0; j < N1; ++j) in[j] = bufB[((k * N1 + j) * Q + a) * 32 + lane];
#pragma unroll
      for (int b = 0; b < Q; ++b) {
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < N1; ++j) s = fmaf(Bc.b[b * N1 + j], in[j], s);
        bufA[((k * Q + b) * Q + a) * 32 + lane] = s;
      }
    }
    __syncthreads();
    // 4. z and the weighted squares: point ab + q^2 cz, psi = sum_k B[cz][k] bufA[k q^2 + ab]
#pragma unroll
    for (int m = 0; m < D::LPW; ++m) {
      const int ab = warp + m * DEN32_WARPS;
      if (ab >= Q * Q) break;
      float in[N1];
#pragma unroll
      for (int k = 0; k < N1; ++k) in[k] = bufA[(k * Q * Q + ab) * 32 + lane];
      float v[P2];
#pragma unroll
      for (int cz = 0; cz < P2; ++cz) {
        float s = 0.f;
        if (cz < Q) {
#pragma unroll
          for (int k = 0; k < N1; ++k) s = fmaf(Bc.b[cz * N1 + k], in[k], s);
        }
        v[cz] = w * (s * s);
      }
      // reduce-scatter over the lanes: after step t the lane keeps the half
      // of its values selected by lane bit (4 - t)
      int cnt = P2;
#pragma unroll
      for (int t = 0; t < D::LG; ++t) {
        const int off = 16 >> t;
        const bool upper = (lane & off) != 0;
        cnt >>= 1;
#pragma unroll
        for (int j = 0; j < P2 / 2; ++j) {
          if (j < cnt) {
            const float send = upper ? v[j] : v[j + cnt];
            const float keep = upper ? v[j + cnt] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, off);
          }
        }
      }
#pragma unroll
      for (int t = D::LG; t < 5; ++t) v[0] += __shfl_xor_sync(0xffffffffu, v[0], 16 >> t);
      int idx = 0;
#pragma unroll
      for (int t = 0; t < D::LG; ++t) idx |= ((lane >> (4 - t)) & 1) << (D::LG - 1 - t);
      if ((lane & ((1 << (5 - D::LG)) - 1)) == 0 && idx < Q) {   // two-sum into (hi, lo)
        const float x = v[0], t = __fadd_rn(acc_h[m], x), bp = __fsub_rn(t, acc_h[m]);
        acc_l[m] = __fadd_rn(acc_l[m], __fadd_rn(__fsub_rn(acc_h[m], __fsub_rn(t, bp)), __fsub_rn(x, bp)));
        acc_h[m] = t;
      }
    }
    __syncthreads();
  }
  int idx = 0;
#pragma unroll
  for (int t = 0; t < D::LG; ++t) idx |= ((lane >> (4 - t)) & 1) << (D::LG - 1 - t);
  if ((lane & ((1 << (5 - D::LG)) - 1)) == 0 && idx < Q) {
#pragma unroll
    for (int m = 0; m < D::LPW; ++m) {
      const int ab = warp + m * DEN32_WARPS;
      if (ab < Q * Q) rho[e * D::NQ + (int64_t)idx * Q * Q + ab] = (double)acc_h[m] + (double)acc_l[m];
    }
  }
}

template <int N1>
static cudaError_t launch_density32(const DensityArgs& a, cudaStream_t s) {
  using D = Den32<N1>;
  DenB Bc;
  for (int t = 0; t < D::Q * N1; ++t) Bc.b[t] = (float)a.Bh[t];
  cudaFuncSetAttribute(density32_kernel<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)D::SMEM);
  note_launch();
  density32_kernel<N1><<<(unsigned)a.ncells, DEN32_THREADS, D::SMEM, s>>>(
      (const float*)a.X, a.ldx, a.n, (const float*)a.Xfr, a.ldfr, a.nfr, a.wfr, a.dofmap, a.minv_sqrt, Bc,
      a.rho);
  return cudaGetLastError();
}

cudaError_t launch_density(const DensityArgs& a, cudaStream_t s) {
  if (a.ncells == 0) return cudaSuccess;
  const int nq = a.q * a.q * a.q;
  if (a.q * a.n1 > 256 || nq > DEN_MAXPT * DEN_THREADS || a.n1 > DEN_MAXN)
    return cudaErrorInvalidValue;
  if (!a.is_double && a.q == a.n1 + 1 && a.Bh && a.ncells <= 0x7fffffff) {
    switch (a.n1) {
      case 3: return launch_density32<3>(a, s);
      case 4: return launch_density32<4>(a, s);
      case 5: return launch_density32<5>(a, s);
      case 6: return launch_density32<6>(a, s);
      case 7: return launch_density32<7>(a, s);
      case 8: return launch_density32<8>(a, s);
      case 9: return launch_density32<9>(a, s);
      default: break;
    }
  }
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
