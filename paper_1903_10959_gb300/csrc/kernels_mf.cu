// Matrix-free binary64 cell apply (the alternative to stored cell matrices
// that the paper's Sec. 3.3.1 notes for the cell-level products).  On the
// tensor-product cell the action of H_e = 1/2 K_e + V_e (Eq. discreteHam)
// factors into 1-D contractions along the three axes:
//   K_e u = (S_x A_y A_z + A_x S_y A_z + A_x A_y S_z) u,
//     A = 1-D consistent mass, S = 1-D stiffness (Gauss rule, exact),
//   V_e u = B_x^T B_y^T B_z^T diag(w V jac) B_z B_y B_x u,
//     B = GLL Lagrange basis at the q Gauss points.
// With the scaled operator H~_e = D_e^{-1/2} H_e D_e^{-1/2} (Eq. hep) the
// cell vector is scaled by M^{-1/2} on the way in and out.  Per cell and
// vector this takes 14 n1^4 + 3 n1^3 (kinetic) + 4 (q n1^3 + q^2 n1^2 + q^3 n1)
// + q^3 (potential) + n1^3 flops instead of 2 n_e^2 (p = 6: 73k instead of
// 235k); binary64 on GB300 is ALU-bound, so the time follows the flops.
//
// One CTA per (cell of one colour, tile of T columns); the passes run out of
// shared memory, a thread per (pencil, column) contracting one axis in
// registers.  Assembly: the colour-ordered node modes of the binary64 path
// (store / accumulate / finish with the Chebyshev three-term update).
#include <algorithm>
#include <cstdint>
#include <mutex>

#include "internal.h"

namespace chfsi {

bool mf_supported(int p, int q);

namespace {

// Contract one axis of `in` (dims d0 (x) x d1 (y) x d2 (z), columns fastest,
// T per point) with the NOUT x NIN matrix M (row-major) into `out` (the same
// dims with the axis replaced by NOUT).  With M2 != nullptr a second
// contraction of the same pencils goes to out2 (shared loads).
template <int NIN, int NOUT, int T>
__device__ __forceinline__ void contract(const double* in, double* out, const double* M,
                                         double* out2, const double* M2, int axis, int d0, int d1,
                                         int d2) {
  // pencil index space: the two other dims x T columns
  const int oa = axis == 0 ? d1 : d0;                        // first other dim
  const int ob = axis == 2 ? d1 : d2;                        // second other dim
  const int npen = oa * ob * T;
  const int sin_ax = axis == 0 ? T : (axis == 1 ? d0 * T : d0 * d1 * T);
  for (int pid = threadIdx.x; pid < npen; pid += blockDim.x) {
    const int c = pid % T;
    const int r = pid / T;
    const int ia = r % oa, ib = r / oa;
    int x, y, z;                                              // pencil origin (axis coord 0)
    if (axis == 0) { x = 0; y = ia; z = ib; }
    else if (axis == 1) { x = ia; y = 0; z = ib; }
    else { x = ia; y = ib; z = 0; }
    const int in0 = ((z * d1 + y) * d0 + x) * T + c;
    double v[NIN];
#pragma unroll
    for (int i = 0; i < NIN; ++i) v[i] = in[in0 + i * sin_ax];
    // output dims: axis replaced by NOUT
    const int e0 = axis == 0 ? NOUT : d0, e1 = axis == 1 ? NOUT : d1;
    const int sout_ax = axis == 0 ? T : (axis == 1 ? e0 * T : e0 * e1 * T);
    const int out0 = ((z * e1 + y) * e0 + x) * T + c;
#pragma unroll 2
    for (int o = 0; o < NOUT; ++o) {
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < NIN; ++i) s = fma(M[o * NIN + i], v[i], s);
      out[out0 + o * sout_ax] = s;
    }
    if (M2) {
#pragma unroll 2
      for (int o = 0; o < NOUT; ++o) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < NIN; ++i) s = fma(M2[o * NIN + i], v[i], s);
        out2[out0 + o * sout_ax] = s;
      }
    }
  }
}

// Kinetic y pass: ayaz = A_y az and t = S_y az + A_y sz (y pencils of both inputs).
template <int N1, int T>
__device__ __forceinline__ void kinetic_y(const double* az, const double* sz, double* ayaz, double* t,
                                          const double* Ay, const double* Sy) {
  const int npen = N1 * N1 * T;
  const int st = N1 * T;
  for (int pid = threadIdx.x; pid < npen; pid += blockDim.x) {
    const int c = pid % T, r = pid / T;
    const int x = r % N1, z = r / N1;
    const int b0 = (z * N1 * N1 + x) * T + c;
    double a[N1], s[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) {
      a[i] = az[b0 + i * st];
      s[i] = sz[b0 + i * st];
    }
#pragma unroll 1
    for (int o = 0; o < N1; ++o) {
      double u = 0.0, w = 0.0;
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        u = fma(Ay[o * N1 + i], a[i], u);
        w = fma(Sy[o * N1 + i], a[i], w);
        w = fma(Ay[o * N1 + i], s[i], w);
      }
      ayaz[b0 + o * st] = u;
      t[b0 + o * st] = w;
    }
  }
}

// Kinetic x pass: kin = S_x ayaz + A_x t (x pencils).
template <int N1, int T>
__device__ __forceinline__ void kinetic_x(const double* ayaz, const double* t, double* kin,
                                          const double* Ax, const double* Sx) {
  const int npen = N1 * N1 * T;
  for (int pid = threadIdx.x; pid < npen; pid += blockDim.x) {
    const int c = pid % T, r = pid / T;            // r = y + N1 z
    const int b0 = r * N1 * T + c;
    double a[N1], s[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) {
      a[i] = ayaz[b0 + i * T];
      s[i] = t[b0 + i * T];
    }
#pragma unroll 2
    for (int o = 0; o < N1; ++o) {
      double u = 0.0;
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        u = fma(Sx[o * N1 + i], a[i], u);
        u = fma(Ax[o * N1 + i], s[i], u);
      }
      kin[b0 + o * T] = u;
    }
  }
}

}  // namespace

// Shared memory (doubles): the 1-D factors, M^{-1/2} at the cell's nodes,
// the raw and the scaled cell block (NE x T each), three buffers of
// max(q^3, NE) x T and one of NE x T.  Pass schedule (buffer <- buffer):
//   kinetic : b1, b2 <- A_z u, S_z u;  b3, kb <- A_y b1, S_y b1 + A_y b2;
//             b1 <- S_x b3 + A_x kb                      (kin, kept in b1)
//   potential: b2 <- B_z u;  b3 <- B_y b2;  b2 <- B_x b3, times w V jac;
//             b3 <- B_x^T b2;  b2 <- B_y^T b3;  kb <- B_z^T b2   (pot)
//   result  : r = M^{-1/2} (1/2 kin + pot), assembled by node mode.
__host__ __device__ constexpr int mf_fac_doubles(int n1, int q) { return 6 * n1 * n1 + 2 * q * n1; }
__host__ __device__ constexpr size_t mf_smem_bytes(int n1, int q, int t) {
  return sizeof(double) *
         ((size_t)((mf_fac_doubles(n1, q) + 1) & ~1) + (size_t)n1 * n1 * n1 +
          3 * (size_t)n1 * n1 * n1 * t + 3 * (size_t)(q * q * q > n1 * n1 * n1 ? q * q * q : n1 * n1 * n1) * t);
}

template <int N1, int Q, int T>
__global__ void __launch_bounds__(256) mf_cell_fp64_kernel(MfLaunch P, const double* __restrict__ Yin,
                                                          double* Yout, const double* Yprev,
                                                          double* W, const double* __restrict__ NL,
                                                          double alpha, double beta, double shift) {
  constexpr int NE = N1 * N1 * N1, NQ = Q * Q * Q;
  constexpr int NF = mf_fac_doubles(N1, Q);
  constexpr int BIG = (NQ > NE ? NQ : NE) * T;
  extern __shared__ double sm[];
  double* fac = sm;
  double* sv = fac + ((NF + 1) & ~1);                        // NE
  double* raw = sv + NE;                                     // NE x T
  double* u = raw + NE * T;                                  // NE x T
  double* kb = u + NE * T;                                   // NE x T
  double* b1 = kb + NE * T;
  double* b2 = b1 + BIG;
  double* b3 = b2 + BIG;
  const int64_t e = P.cells[blockIdx.x];
  const int c0 = blockIdx.y * T;
  const int ncv = min(T, P.ncol - c0);
  const int32_t* dm = P.dofmap + e * NE;
  const uint8_t* md = P.modes + e * NE;

  for (int i = threadIdx.x; i < NF; i += blockDim.x) fac[i] = P.fac[i];
  for (int l = threadIdx.x; l < NE; l += blockDim.x) {
    const int g = dm[l];
    sv[l] = g >= 0 ? P.minv_sqrt[g] : 0.0;
  }
  for (int idx = threadIdx.x; idx < NE * T; idx += blockDim.x) {
    const int l = idx / T, c = idx - l * T;
    const int g = dm[l];
    raw[idx] = (g >= 0 && c < ncv) ? Yin[(int64_t)g * P.ld_in + c0 + c] : 0.0;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < NE * T; idx += blockDim.x) u[idx] = raw[idx] * sv[idx / T];
  __syncthreads();
  const double* Ax = fac;
  const double* Ay = fac + N1 * N1;
  const double* Az = fac + 2 * N1 * N1;
  const double* Sx = fac + 3 * N1 * N1;
  const double* Sy = fac + 4 * N1 * N1;
  const double* Sz = fac + 5 * N1 * N1;
  const double* Bq = fac + 6 * N1 * N1;                      // Q x N1
  const double* Bt = Bq + Q * N1;                            // N1 x Q
  // kinetic part
  contract<N1, N1, T>(u, b1, Az, b2, Sz, 2, N1, N1, N1);
  __syncthreads();
  kinetic_y<N1, T>(b1, b2, b3, kb, Ay, Sy);
  __syncthreads();
  kinetic_x<N1, T>(b3, kb, b1, Ax, Sx);
  __syncthreads();
  // potential part (skipped for the stiffness operator alone)
  if (P.kinetic_only) {
    for (int idx = threadIdx.x; idx < NE * T; idx += blockDim.x) kb[idx] = 0.0;
  } else {
    contract<N1, Q, T>(u, b2, Bq, nullptr, nullptr, 2, N1, N1, N1);    // (N1, N1, Q)
    __syncthreads();
    contract<N1, Q, T>(b2, b3, Bq, nullptr, nullptr, 1, N1, N1, Q);    // (N1, Q, Q)
    __syncthreads();
    contract<N1, Q, T>(b3, b2, Bq, nullptr, nullptr, 0, N1, Q, Q);     // (Q, Q, Q)
    __syncthreads();
    const double* wv = P.wv + e * (int64_t)NQ;
    for (int idx = threadIdx.x; idx < NQ * T; idx += blockDim.x) b2[idx] *= __ldg(wv + idx / T);
    __syncthreads();
    contract<Q, N1, T>(b2, b3, Bt, nullptr, nullptr, 0, Q, Q, Q);      // (N1, Q, Q)
    __syncthreads();
    contract<Q, N1, T>(b3, b2, Bt, nullptr, nullptr, 1, N1, Q, Q);     // (N1, N1, Q)
    __syncthreads();
    contract<Q, N1, T>(b2, kb, Bt, nullptr, nullptr, 2, N1, N1, Q);    // (N1, N1, N1)
  }
  __syncthreads();
  // r = M^{-1/2} (1/2 kin + pot); node-mode assembly fused with the update
  for (int idx = threadIdx.x; idx < NE * T; idx += blockDim.x) {
    const int l = idx / T, c = idx - l * T;
    const uint8_t mode = md[l];
    if (mode == MODE_SKIP || c >= ncv) continue;
    double v = sv[l] * fma(0.5, b1[idx], kb[idx]);
    const int64_t g = dm[l];
    const int cc = c0 + c;
    if (mode == MODE_STORE) {
      W[g * P.ld_w + cc] = v;
    } else if (mode == MODE_ACCUM) {
      W[g * P.ld_w + cc] += v;
    } else {
      if (mode == MODE_FINAL) v += W[g * P.ld_w + cc];
      if (NL) v += NL[g * P.ld_w + cc];
      double out = alpha * (v - shift * raw[idx]);
      if (Yprev) out = fma(beta, Yprev[g * P.ld_prev + cc], out);
      Yout[g * P.ld_out + cc] = out;
    }
  }
}

// ---------------------------------------------------------------- Bloch (k-point) variant
// H_e(k) = 1/2 K_e - i k.G_e + 1/2 |k|^2 A_e + V_e (Eq. evp of the periodic
// problem, the cell-periodic part of a Bloch state) on a complex block stored
// as interleaved (real, imaginary) column pairs.  With T = 1/2 K + 1/2 |k|^2 A
// + V and G = k.G_e (real, cell-independent):
//   Re(H u) = T u_r + G u_i,   Im(H u) = T u_i - G u_r.
// 1/2 |k|^2 A folds into the kinetic x pass (S_x + |k|^2 A_x); G has the
// kinetic part's structure with the stiffness replaced by the 1-D derivative
// matrix C_il = int l_i l_l' (no Jacobian), scaled by k per axis:
//   G u = (k_x C_x) A_y A_z u + A_x (k_y C_y) A_z u + A_x A_y (k_z C_z) u.
// Factors: A_x, A_y, A_z, S'_x = S_x + |k|^2 A_x, S_y, S_z, B, B^T, k_x C, k_y C, k_z C.
__host__ __device__ constexpr int mfk_fac_doubles(int n1, int q) { return 9 * n1 * n1 + 2 * q * n1; }
__host__ __device__ constexpr size_t mfk_smem_bytes(int n1, int q, int t) {
  return sizeof(double) *
         ((size_t)((mfk_fac_doubles(n1, q) + 1) & ~1) + (size_t)n1 * n1 * n1 +
          5 * (size_t)n1 * n1 * n1 * t + 3 * (size_t)(q * q * q > n1 * n1 * n1 ? q * q * q : n1 * n1 * n1) * t);
}

// z pass of three matrices on the same pencils: out_m = M_m u along z.
template <int N1, int T>
__device__ __forceinline__ void z_pass3(const double* u, double* o1, double* o2, double* o3,
                                        const double* M1, const double* M2, const double* M3) {
  const int npen = N1 * N1 * T;
  const int st = N1 * N1 * T;
  for (int pid = threadIdx.x; pid < npen; pid += blockDim.x) {
    const int c = pid % T, r = pid / T;            // r = x + N1 y
    const int b0 = r * T + c;
    double v[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) v[i] = u[b0 + i * st];
#pragma unroll 1
    for (int o = 0; o < N1; ++o) {
      double a = 0.0, s = 0.0, g = 0.0;
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        a = fma(M1[o * N1 + i], v[i], a);
        s = fma(M2[o * N1 + i], v[i], s);
        g = fma(M3[o * N1 + i], v[i], g);
      }
      o1[b0 + o * st] = a;
      o2[b0 + o * st] = s;
      o3[b0 + o * st] = g;
    }
  }
}

// y pass: ayaz = A_y az, t = S_y az + A_y sz, gt = Cy az + A_y cz.
template <int N1, int T>
__device__ __forceinline__ void y_pass3(const double* az, const double* sz, const double* cz,
                                        double* ayaz, double* t, double* gt, const double* Ay,
                                        const double* Sy, const double* Cy) {
  const int npen = N1 * N1 * T;
  const int st = N1 * T;
  for (int pid = threadIdx.x; pid < npen; pid += blockDim.x) {
    const int c = pid % T, r = pid / T;
    const int x = r % N1, z = r / N1;
    const int b0 = (z * N1 * N1 + x) * T + c;
    double a[N1], s[N1], g[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) {
      a[i] = az[b0 + i * st];
      s[i] = sz[b0 + i * st];
      g[i] = cz[b0 + i * st];
    }
#pragma unroll 1
    for (int o = 0; o < N1; ++o) {
      double u = 0.0, w = 0.0, h = 0.0;
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        u = fma(Ay[o * N1 + i], a[i], u);
        w = fma(Sy[o * N1 + i], a[i], w);
        w = fma(Ay[o * N1 + i], s[i], w);
        h = fma(Cy[o * N1 + i], a[i], h);
        h = fma(Ay[o * N1 + i], g[i], h);
      }
      ayaz[b0 + o * st] = u;
      t[b0 + o * st] = w;
      gt[b0 + o * st] = h;
    }
  }
}

// x pass: kin = S'_x ayaz + A_x t, g = Cx ayaz + A_x gt.
template <int N1, int T>
__device__ __forceinline__ void x_pass2(const double* ayaz, const double* t, const double* gt,
                                        double* kin, double* g, const double* Ax, const double* Sx,
                                        const double* Cx) {
  const int npen = N1 * N1 * T;
  for (int pid = threadIdx.x; pid < npen; pid += blockDim.x) {
    const int c = pid % T, r = pid / T;
    const int b0 = r * N1 * T + c;
    double a[N1], s[N1], h[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) {
      a[i] = ayaz[b0 + i * T];
      s[i] = t[b0 + i * T];
      h[i] = gt[b0 + i * T];
    }
#pragma unroll 1
    for (int o = 0; o < N1; ++o) {
      double u = 0.0, w = 0.0;
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        u = fma(Sx[o * N1 + i], a[i], u);
        u = fma(Ax[o * N1 + i], s[i], u);
        w = fma(Cx[o * N1 + i], a[i], w);
        w = fma(Ax[o * N1 + i], h[i], w);
      }
      kin[b0 + o * T] = u;
      g[b0 + o * T] = w;
    }
  }
}

// Columns come in (real, imaginary) pairs; T is even and c0 is even.
template <int N1, int Q, int T>
__global__ void __launch_bounds__(256) mfk_cell_fp64_kernel(MfLaunch P, const double* __restrict__ Yin,
                                                           double* Yout, const double* Yprev,
                                                           double* W, double alpha, double beta,
                                                           double shift) {
  static_assert(T % 2 == 0, "column pairs");
  constexpr int NE = N1 * N1 * N1, NQ = Q * Q * Q;
  constexpr int NF = mfk_fac_doubles(N1, Q);
  constexpr int BIG = (NQ > NE ? NQ : NE) * T;
  extern __shared__ double sm[];
  double* fac = sm;
  double* sv = fac + ((NF + 1) & ~1);
  double* raw = sv + NE;
  double* u = raw + NE * T;
  double* kb = u + NE * T;
  double* x2 = kb + NE * T;
  double* x3 = x2 + NE * T;
  double* b1 = x3 + NE * T;
  double* b2 = b1 + BIG;
  double* b3 = b2 + BIG;
  const int64_t e = P.cells[blockIdx.x];
  const int c0 = blockIdx.y * T;
  const int ncv = min(T, P.ncol - c0);
  const int32_t* dm = P.dofmap + e * NE;
  const uint8_t* md = P.modes + e * NE;
  for (int i = threadIdx.x; i < NF; i += blockDim.x) fac[i] = P.fac[i];
  for (int l = threadIdx.x; l < NE; l += blockDim.x) {
    const int g = dm[l];
    sv[l] = g >= 0 ? P.minv_sqrt[g] : 0.0;
  }
  for (int idx = threadIdx.x; idx < NE * T; idx += blockDim.x) {
    const int l = idx / T, c = idx - l * T;
    const int g = dm[l];
    raw[idx] = (g >= 0 && c < ncv) ? Yin[(int64_t)g * P.ld_in + c0 + c] : 0.0;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < NE * T; idx += blockDim.x) u[idx] = raw[idx] * sv[idx / T];
  __syncthreads();
  const double* Ax = fac;
  const double* Ay = fac + N1 * N1;
  const double* Az = fac + 2 * N1 * N1;
  const double* Sx = fac + 3 * N1 * N1;
  const double* Sy = fac + 4 * N1 * N1;
  const double* Sz = fac + 5 * N1 * N1;
  const double* Bq = fac + 6 * N1 * N1;
  const double* Bt = Bq + Q * N1;
  const double* Cx = Bt + Q * N1;
  const double* Cy = Cx + N1 * N1;
  const double* Cz = Cy + N1 * N1;
  // potential first (into kb), using b2 / b3
  contract<N1, Q, T>(u, b2, Bq, nullptr, nullptr, 2, N1, N1, N1);
  __syncthreads();
  contract<N1, Q, T>(b2, b3, Bq, nullptr, nullptr, 1, N1, N1, Q);
  __syncthreads();
  contract<N1, Q, T>(b3, b2, Bq, nullptr, nullptr, 0, N1, Q, Q);
  __syncthreads();
  {
    const double* wv = P.wv + e * (int64_t)NQ;
    for (int idx = threadIdx.x; idx < NQ * T; idx += blockDim.x) b2[idx] *= __ldg(wv + idx / T);
  }
  __syncthreads();
  contract<Q, N1, T>(b2, b3, Bt, nullptr, nullptr, 0, Q, Q, Q);
  __syncthreads();
  contract<Q, N1, T>(b3, b2, Bt, nullptr, nullptr, 1, N1, Q, Q);
  __syncthreads();
  contract<Q, N1, T>(b2, kb, Bt, nullptr, nullptr, 2, N1, N1, Q);
  __syncthreads();
  // kinetic + mass + gradient parts
  z_pass3<N1, T>(u, b1, b2, b3, Az, Sz, Cz);                 // az, sz, cz
  __syncthreads();
  y_pass3<N1, T>(b1, b2, b3, u, x2, x3, Ay, Sy, Cy);          // ayaz (u), t (x2), gt (x3)
  __syncthreads();
  x_pass2<N1, T>(u, x2, x3, b1, b2, Ax, Sx, Cx);              // kin (b1), g (b2)
  __syncthreads();
  for (int idx = threadIdx.x; idx < NE * T; idx += blockDim.x) {
    const int l = idx / T, c = idx - l * T;
    const uint8_t mode = md[l];
    if (mode == MODE_SKIP || c >= ncv) continue;
    const bool im = (c & 1) != 0;
    const double gpart = im ? -b2[idx - 1] : b2[idx + 1];     // Re: + G u_i; Im: - G u_r
    double v = sv[l] * (fma(0.5, b1[idx], kb[idx]) + gpart);
    const int64_t g = dm[l];
    const int cc = c0 + c;
    if (mode == MODE_STORE) {
      W[g * P.ld_w + cc] = v;
    } else if (mode == MODE_ACCUM) {
      W[g * P.ld_w + cc] += v;
    } else {
      if (mode == MODE_FINAL) v += W[g * P.ld_w + cc];
      double out = alpha * (v - shift * raw[idx]);
      if (Yprev) out = fma(beta, Yprev[g * P.ld_prev + cc], out);
      Yout[g * P.ld_out + cc] = out;
    }
  }
}

namespace {
template <int N1, int T>
cudaError_t mfk_launch_t(const MfLaunch& L, const double* Yin, double* Yout, const double* Yprev,
                         double* W, FilterStep st, cudaStream_t s) {
  constexpr int Q = N1 + 1;
  constexpr size_t smem = mfk_smem_bytes(N1, Q, T);
  static_assert(smem <= 227 * 1024, "k-point cell kernel: shared memory");
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(mfk_cell_fp64_kernel<N1, Q, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  });
  dim3 grid((unsigned)L.ncells_colour, (unsigned)((L.ncol + T - 1) / T));
  note_launch();
  mfk_cell_fp64_kernel<N1, Q, T><<<grid, 256, smem, s>>>(L, Yin, Yout, Yprev, W, st.alpha, st.beta,
                                                          st.shift);
  return cudaGetLastError();
}
template <int N1>
cudaError_t mfk_launch_p(const MfLaunch& L, const double* Yin, double* Yout, const double* Yprev,
                         double* W, FilterStep st, cudaStream_t s) {
  constexpr int Q = N1 + 1;
  if (L.ncol >= 4 && mfk_smem_bytes(N1, Q, 4) <= 110 * 1024)
    return mfk_launch_t<N1, (mfk_smem_bytes(N1, Q, 4) <= 110 * 1024 ? 4 : 2)>(L, Yin, Yout, Yprev, W, st, s);
  return mfk_launch_t<N1, 2>(L, Yin, Yout, Yprev, W, st, s);
}
}  // namespace

cudaError_t launch_mfk_cell_fp64(const MfLaunch& L, const double* Yin, double* Yout,
                                 const double* Yprev, double* W, FilterStep st, cudaStream_t s) {
  if (L.ncells_colour == 0 || L.ncol == 0) return cudaSuccess;
  if (!mf_supported(L.p, L.q) || (L.ncol & 1)) return cudaErrorInvalidValue;
  const double* prev = st.beta != 0.0 ? Yprev : nullptr;
  switch (L.p) {
    case 2: return mfk_launch_p<3>(L, Yin, Yout, prev, W, st, s);
    case 3: return mfk_launch_p<4>(L, Yin, Yout, prev, W, st, s);
    case 4: return mfk_launch_p<5>(L, Yin, Yout, prev, W, st, s);
    case 5: return mfk_launch_p<6>(L, Yin, Yout, prev, W, st, s);
    case 6: return mfk_launch_p<7>(L, Yin, Yout, prev, W, st, s);
    case 7: return mfk_launch_p<8>(L, Yin, Yout, prev, W, st, s);
    default: return mfk_launch_p<9>(L, Yin, Yout, prev, W, st, s);
  }
}

namespace {
template <int N1, int T>
cudaError_t mf_launch_t(const MfLaunch& L, const double* Yin, double* Yout, const double* Yprev,
                        double* W, const double* NL, FilterStep st, cudaStream_t s) {
  constexpr int Q = N1 + 1;
  constexpr size_t smem = mf_smem_bytes(N1, Q, T);
  static_assert(smem <= 227 * 1024, "matrix-free cell kernel: shared memory");
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(mf_cell_fp64_kernel<N1, Q, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  });
  dim3 grid((unsigned)L.ncells_colour, (unsigned)((L.ncol + T - 1) / T));
  note_launch();
  mf_cell_fp64_kernel<N1, Q, T><<<grid, 256, smem, s>>>(L, Yin, Yout, Yprev, W, NL, st.alpha,
                                                         st.beta, st.shift);
  return cudaGetLastError();
}

// Column tile per CTA: the widest of 8 / 4 / 2 whose buffers fit in ~110 KB
// (two CTAs per SM), else the widest that fits in 227 KB.
template <int N1>
cudaError_t mf_launch_p(const MfLaunch& L, const double* Yin, double* Yout, const double* Yprev,
                        double* W, const double* NL, FilterStep st, cudaStream_t s) {
  constexpr int Q = N1 + 1;
  if (L.ncol >= 8 && mf_smem_bytes(N1, Q, 8) <= 110 * 1024)
    return mf_launch_t<N1, (mf_smem_bytes(N1, Q, 8) <= 110 * 1024 ? 8 : 2)>(L, Yin, Yout, Yprev, W, NL, st, s);
  if (L.ncol >= 4 && mf_smem_bytes(N1, Q, 4) <= 110 * 1024)
    return mf_launch_t<N1, (mf_smem_bytes(N1, Q, 4) <= 110 * 1024 ? 4 : 2)>(L, Yin, Yout, Yprev, W, NL, st, s);
  return mf_launch_t<N1, 2>(L, Yin, Yout, Yprev, W, NL, st, s);
}
}  // namespace

bool mf_supported(int p, int q) { return p >= 2 && p <= 8 && q == p + 2; }

cudaError_t launch_mf_cell_fp64(const MfLaunch& L, const double* Yin, double* Yout,
                                const double* Yprev, double* W, const double* NL, FilterStep st,
                                cudaStream_t s) {
  if (L.ncells_colour == 0 || L.ncol == 0) return cudaSuccess;
  if (!mf_supported(L.p, L.q)) return cudaErrorInvalidValue;
  const double* prev = st.beta != 0.0 ? Yprev : nullptr;
  switch (L.p) {
    case 2: return mf_launch_p<3>(L, Yin, Yout, prev, W, NL, st, s);
    case 3: return mf_launch_p<4>(L, Yin, Yout, prev, W, NL, st, s);
    case 4: return mf_launch_p<5>(L, Yin, Yout, prev, W, NL, st, s);
    case 5: return mf_launch_p<6>(L, Yin, Yout, prev, W, NL, st, s);
    case 6: return mf_launch_p<7>(L, Yin, Yout, prev, W, NL, st, s);
    case 7: return mf_launch_p<8>(L, Yin, Yout, prev, W, NL, st, s);
    default: return mf_launch_p<9>(L, Yin, Yout, prev, W, NL, st, s);
  }
}

}  // namespace chfsi
