// Host-side finite-element setup in binary64: quadrature rules, the
// cell -> unknown map with periodic identification, the colour schedule of
// the assembly, the diagonal GLL mass and the scaled cell Hamiltonians.
//
// arXiv:1903.10959 Sec. 2.4: C0 Lagrange basis on GLL nodes (Eq. fem), local
// Hamiltonian 1/2 int grad N_j . grad N_k + int V N_j N_k (Eq. discreteHam),
// GLL quadrature for the overlap matrix (diagonal M) and the standard form
// H~ = M^{-1/2} H M^{-1/2} (Eq. hep).  Sec. 3.3.1: the cell-level matrices
// are computed once and stored.  Because M is diagonal,
// H~ restricted to a cell is D_e^{-1/2} H_e D_e^{-1/2} with D_e the global
// mass at the cell's nodes, so the scaling is folded into the stored matrix.
//
// The Hamiltonian integrals use a Gauss-Legendre rule (q points per
// direction, default p + 2); the paper fixes only the mass quadrature.  The
// potential term is evaluated by sum factorisation over the three tensor
// directions.
#include <algorithm>
#include <array>
#include <cmath>
#include <stdexcept>

#include "internal.h"

namespace chfsi {

// Legendre P_n(x) and P_{n-1}(x) by the three-term recurrence.
static void legendre(int n, double x, double& pn, double& pn1) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { pn = 1.0; pn1 = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  pn = p1;
  pn1 = p0;
}

void gll_rule(int p, std::vector<double>& x, std::vector<double>& w) {
  // interior nodes: zeros of P_p' found by Newton from Chebyshev-Lobatto guesses,
  // using (1 - x^2) P_p' = p (P_{p-1} - x P_p) and the Legendre ODE for P_p''.
  x.assign(p + 1, 0.0);
  w.assign(p + 1, 0.0);
  x[0] = -1.0;
  x[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double t = -std::cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double pn, pn1;
      legendre(p, t, pn, pn1);
      double d1 = p * (pn1 - t * pn) / (1.0 - t * t);
      double d2 = (2.0 * t * d1 - p * (p + 1.0) * pn) / (1.0 - t * t);
      double dt = d1 / d2;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[i] = t;
  }
  for (int i = 0; i <= p; ++i) {
    double pn, pn1;
    legendre(p, x[i], pn, pn1);
    w[i] = 2.0 / (p * (p + 1.0) * pn * pn);
  }
}

void gauss_rule(int q, std::vector<double>& x, std::vector<double>& w) {
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  for (int i = 0; i < q; ++i) {
    double t = -std::cos(M_PI * (i + 0.75) / (q + 0.5));
    double d1 = 0.0;
    for (int it = 0; it < 100; ++it) {
      double pn, pn1;
      legendre(q, t, pn, pn1);
      d1 = q * (pn1 - t * pn) / (1.0 - t * t);
      double dt = pn / d1;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double pn, pn1;
    legendre(q, t, pn, pn1);
    d1 = q * (pn1 - t * pn) / (1.0 - t * t);
    x[i] = t;
    w[i] = 2.0 / ((1.0 - t * t) * d1 * d1);
  }
}

// Basis values and derivatives at points t via barycentric interpolation and
// the nodal differentiation matrix (exact for degree-p polynomials).
static void basis_at(const std::vector<double>& xn, const std::vector<double>& t,
                     std::vector<double>& B, std::vector<double>& Dd) {
  const int n1 = (int)xn.size(), nt = (int)t.size();
  std::vector<double> bw(n1, 1.0);
  for (int j = 0; j < n1; ++j)
    for (int k = 0; k < n1; ++k)
      if (k != j) bw[j] /= (xn[j] - xn[k]);
  std::vector<double> Dm(n1 * n1, 0.0);  // Dm[k*n1+j] = l_j'(x_k)
  for (int k = 0; k < n1; ++k) {
    double s = 0.0;
    for (int j = 0; j < n1; ++j)
      if (j != k) {
        Dm[k * n1 + j] = (bw[j] / bw[k]) / (xn[k] - xn[j]);
        s += Dm[k * n1 + j];
      }
    Dm[k * n1 + k] = -s;
  }
  B.assign(nt * n1, 0.0);
  Dd.assign(nt * n1, 0.0);
  for (int a = 0; a < nt; ++a) {
    int hit = -1;
    for (int j = 0; j < n1; ++j)
      if (std::fabs(t[a] - xn[j]) < 1e-15) hit = j;
    if (hit >= 0) {
      B[a * n1 + hit] = 1.0;
    } else {
      double den = 0.0;
      for (int j = 0; j < n1; ++j) den += bw[j] / (t[a] - xn[j]);
      for (int j = 0; j < n1; ++j) B[a * n1 + j] = (bw[j] / (t[a] - xn[j])) / den;
    }
    for (int j = 0; j < n1; ++j) {
      double s = 0.0;
      for (int k = 0; k < n1; ++k) s += B[a * n1 + k] * Dm[k * n1 + j];
      Dd[a * n1 + j] = s;
    }
  }
}

static int64_t global_1d(const HostMesh& m, int axis, int c, int i) {
  int64_t g = (int64_t)c * m.p + i;
  if (m.per[axis]) return g % ((int64_t)m.n[axis] * m.p);
  if (g == 0 || g == (int64_t)m.n[axis] * m.p) return -1;
  return g - 1;
}

static int colour_1d(const HostMesh& m, int axis, int c) {
  if (m.per[axis] && (m.n[axis] % 2 == 1) && c == m.n[axis] - 1) return 2;
  return c % 2;
}

void build_mesh(const chfsi_mesh_desc& d, HostMesh& m) {
  m.p = d.p;
  m.n1 = d.p + 1;
  m.ne = m.n1 * m.n1 * m.n1;
  m.q = d.quad_points > 0 ? d.quad_points : d.p + 2;
  for (int a = 0; a < 3; ++a) {
    m.per[a] = d.periodic[a] != 0;
    m.n[a] = d.ncell[a];
    m.len[a] = d.len[a];
    m.h[a] = d.len[a] / d.ncell[a];
    m.nd[a] = m.per[a] ? (int64_t)d.ncell[a] * d.p : (int64_t)d.ncell[a] * d.p - 1;
  }
  m.ndofs = m.nd[0] * m.nd[1] * m.nd[2];
  m.ncells = (int64_t)m.n[0] * m.n[1] * m.n[2];
  gll_rule(m.p, m.gll_x, m.gll_w);
  gauss_rule(m.q, m.gq_x, m.gq_w);
  basis_at(m.gll_x, m.gq_x, m.B, m.D);

  const int n1 = m.n1, ne = m.ne;
  m.dofmap.assign(m.ncells * ne, -1);
  for (int64_t e = 0; e < m.ncells; ++e) {
    int cx = (int)(e % m.n[0]), cy = (int)((e / m.n[0]) % m.n[1]), cz = (int)(e / ((int64_t)m.n[0] * m.n[1]));
    for (int k = 0; k < n1; ++k) {
      int64_t gz = global_1d(m, 2, cz, k);
      for (int j = 0; j < n1; ++j) {
        int64_t gy = global_1d(m, 1, cy, j);
        for (int i = 0; i < n1; ++i) {
          int64_t gx = global_1d(m, 0, cx, i);
          int l = i + n1 * (j + n1 * k);
          if (gx >= 0 && gy >= 0 && gz >= 0)
            m.dofmap[e * ne + l] = (int32_t)(gx + m.nd[0] * (gy + m.nd[1] * gz));
        }
      }
    }
  }

  // colours: parity per axis (a third colour closes odd periodic rings)
  std::vector<int> col(m.ncells);
  int used[27] = {0};
  for (int64_t e = 0; e < m.ncells; ++e) {
    int cx = (int)(e % m.n[0]), cy = (int)((e / m.n[0]) % m.n[1]), cz = (int)(e / ((int64_t)m.n[0] * m.n[1]));
    col[e] = colour_1d(m, 0, cx) + 3 * (colour_1d(m, 1, cy) + 3 * colour_1d(m, 2, cz));
    used[col[e]] = 1;
  }
  int rank[27], nc = 0;
  for (int c = 0; c < 27; ++c) rank[c] = used[c] ? nc++ : -1;
  m.colour_offsets.assign(nc + 1, 0);
  for (int64_t e = 0; e < m.ncells; ++e) m.colour_offsets[rank[col[e]] + 1]++;
  for (int c = 0; c < nc; ++c) m.colour_offsets[c + 1] += m.colour_offsets[c];
  m.colour_cells.assign(m.ncells, 0);
  {
    std::vector<int64_t> pos(m.colour_offsets.begin(), m.colour_offsets.end() - 1);
    for (int64_t e = 0; e < m.ncells; ++e) m.colour_cells[pos[rank[col[e]]]++] = (int32_t)e;
  }

  // modes: first / last colour touching each unknown
  std::vector<int> first(m.ndofs, 1 << 30), last(m.ndofs, -1), count(m.ndofs, 0);
  for (int64_t e = 0; e < m.ncells; ++e) {
    int r = rank[col[e]];
    for (int l = 0; l < ne; ++l) {
      int32_t g = m.dofmap[e * ne + l];
      if (g < 0) continue;
      first[g] = std::min(first[g], r);
      last[g] = std::max(last[g], r);
      count[g]++;
    }
  }
  m.modes.assign(m.ncells * ne, MODE_SKIP);
  for (int64_t e = 0; e < m.ncells; ++e) {
    int r = rank[col[e]];
    for (int l = 0; l < ne; ++l) {
      int32_t g = m.dofmap[e * ne + l];
      if (g < 0) continue;
      uint8_t md;
      if (count[g] == 1) md = MODE_FINAL_DIRECT;
      else if (r == first[g]) md = MODE_STORE;
      else if (r == last[g]) md = MODE_FINAL;
      else md = MODE_ACCUM;
      m.modes[e * ne + l] = md;
    }
  }

  // unknown -> (cell, local node) rows for the owner-computes assembly
  m.node_ptr.assign(m.ndofs + 1, 0);
  for (int64_t e = 0; e < m.ncells; ++e)
    for (int l = 0; l < ne; ++l)
      if (m.dofmap[e * ne + l] >= 0) m.node_ptr[m.dofmap[e * ne + l] + 1]++;
  for (int64_t j = 0; j < m.ndofs; ++j) m.node_ptr[j + 1] += m.node_ptr[j];
  m.node_ent.assign(m.node_ptr[m.ndofs], 0);
  {
    std::vector<int32_t> pos(m.node_ptr.begin(), m.node_ptr.end() - 1);
    for (int64_t e = 0; e < m.ncells; ++e)     // ascending e: fixed summation order
      for (int l = 0; l < ne; ++l) {
        const int32_t g = m.dofmap[e * ne + l];
        if (g >= 0) m.node_ent[pos[g]++] = (int32_t)(e * ne + l);
      }
  }

  // diagonal mass by GLL quadrature: node weight w_i w_j w_k hx hy hz / 8
  m.mass.assign(m.ndofs, 0.0);
  const double jac = m.h[0] * m.h[1] * m.h[2] / 8.0;
  for (int64_t e = 0; e < m.ncells; ++e)
    for (int k = 0; k < n1; ++k)
      for (int j = 0; j < n1; ++j)
        for (int i = 0; i < n1; ++i) {
          int32_t g = m.dofmap[e * ne + i + n1 * (j + n1 * k)];
          if (g >= 0) m.mass[g] += m.gll_w[i] * m.gll_w[j] * m.gll_w[k] * jac;
        }
}

// Potential of the wells at a point (wells pre-filtered to those in range).
static inline double well_sum(const double* x, const std::vector<double>& cx,
                              const std::vector<double>& dd, const std::vector<double>& inv2w2) {
  double v = 0.0;
  for (size_t a = 0; a < dd.size(); ++a) {
    double dx = x[0] - cx[3 * a], dy = x[1] - cx[3 * a + 1], dz = x[2] - cx[3 * a + 2];
    v -= dd[a] * std::exp(-(dx * dx + dy * dy + dz * dz) * inv2w2[a]);
  }
  return v;
}

void build_cell_matrices(const HostMesh& m, const Wells& wl, std::vector<double>& Ht,
                         std::vector<double>* wv) {
  const int n1 = m.n1, ne = m.ne, q = m.q;
  const int nn = n1 * n1;
  Ht.assign((size_t)m.ncells * ne * ne, 0.0);
  if (wv) wv->assign((size_t)m.ncells * q * q * q, 0.0);

  // 1-D consistent mass A and stiffness S per axis (Gauss rule, exact)
  std::vector<double> A[3], S[3];
  for (int ax = 0; ax < 3; ++ax) {
    A[ax].assign(nn, 0.0);
    S[ax].assign(nn, 0.0);
    for (int i = 0; i < n1; ++i)
      for (int l = 0; l < n1; ++l) {
        double sa = 0.0, ss = 0.0;
        for (int a = 0; a < q; ++a) {
          sa += m.gq_w[a] * m.B[a * n1 + i] * m.B[a * n1 + l];
          ss += m.gq_w[a] * m.D[a * n1 + i] * m.D[a * n1 + l];
        }
        A[ax][i * n1 + l] = sa * m.h[ax] / 2.0;
        S[ax][i * n1 + l] = ss * 2.0 / m.h[ax];
      }
  }
  // shared kinetic matrix 1/2 K (identical for every cell of the uniform mesh)
  std::vector<double> K(ne * ne);
  for (int k = 0; k < n1; ++k) for (int j = 0; j < n1; ++j) for (int i = 0; i < n1; ++i)
    for (int c = 0; c < n1; ++c) for (int b = 0; b < n1; ++b) for (int a = 0; a < n1; ++a) {
      int r = i + n1 * (j + n1 * k), s = a + n1 * (b + n1 * c);
      K[r * ne + s] = 0.5 * (S[0][i * n1 + a] * A[1][j * n1 + b] * A[2][k * n1 + c] +
                             A[0][i * n1 + a] * S[1][j * n1 + b] * A[2][k * n1 + c] +
                             A[0][i * n1 + a] * A[1][j * n1 + b] * S[2][k * n1 + c]);
    }
  // BB[a][i*n1+l] = w_a B[a][i] B[a][l]
  std::vector<double> BB(q * nn);
  for (int a = 0; a < q; ++a)
    for (int i = 0; i < n1; ++i)
      for (int l = 0; l < n1; ++l) BB[a * nn + i * n1 + l] = m.gq_w[a] * m.B[a * n1 + i] * m.B[a * n1 + l];

  // wells: images along the periodic axes as explicit centres; cut off where
  // the Gaussian is < 1e-18 D
  std::vector<double> ic, idp, iw;
  const int nw = (int)wl.depth.size();
  for (int a = 0; a < nw; ++a) {
    for (int sz = -1; sz <= 1; ++sz) for (int sy = -1; sy <= 1; ++sy) for (int sx = -1; sx <= 1; ++sx) {
      if ((!m.per[0] && sx) || (!m.per[1] && sy) || (!m.per[2] && sz)) continue;
      ic.push_back(wl.xyz[3 * a] + sx * m.len[0]);
      ic.push_back(wl.xyz[3 * a + 1] + sy * m.len[1]);
      ic.push_back(wl.xyz[3 * a + 2] + sz * m.len[2]);
      idp.push_back(wl.depth[a]);
      iw.push_back(wl.width[a]);
    }
  }
  const double jac = m.h[0] * m.h[1] * m.h[2] / 8.0;

#pragma omp parallel
  {
    std::vector<double> cx, dd, inv2w2, V(q * q * q), T1(q * q * nn), T2(q * nn * nn), He(ne * ne);
    double xq[3];
#pragma omp for schedule(dynamic, 4)
    for (int64_t e = 0; e < m.ncells; ++e) {
      int c3[3] = {(int)(e % m.n[0]), (int)((e / m.n[0]) % m.n[1]), (int)(e / ((int64_t)m.n[0] * m.n[1]))};
      double lo[3], hi[3];
      for (int ax = 0; ax < 3; ++ax) { lo[ax] = c3[ax] * m.h[ax]; hi[ax] = lo[ax] + m.h[ax]; }
      cx.clear(); dd.clear(); inv2w2.clear();
      for (size_t a = 0; a < idp.size(); ++a) {
        double r2 = 0.0;
        for (int ax = 0; ax < 3; ++ax) {
          double c = ic[3 * a + ax];
          double dlt = c < lo[ax] ? lo[ax] - c : (c > hi[ax] ? c - hi[ax] : 0.0);
          r2 += dlt * dlt;
        }
        if (r2 * 1.0 / (2.0 * iw[a] * iw[a]) > 41.5) continue;   // exp(-41.5) < 1e-18
        cx.push_back(ic[3 * a]); cx.push_back(ic[3 * a + 1]); cx.push_back(ic[3 * a + 2]);
        dd.push_back(idp[a]);
        inv2w2.push_back(1.0 / (2.0 * iw[a] * iw[a]));
      }
      const double* vq = wl.vqp.empty() ? nullptr : wl.vqp.data() + e * (int64_t)q * q * q;
      for (int c = 0; c < q; ++c) for (int b = 0; b < q; ++b) for (int a = 0; a < q; ++a) {
        xq[0] = lo[0] + (m.gq_x[a] + 1.0) * m.h[0] / 2.0;
        xq[1] = lo[1] + (m.gq_x[b] + 1.0) * m.h[1] / 2.0;
        xq[2] = lo[2] + (m.gq_x[c] + 1.0) * m.h[2] / 2.0;
        const int pt = (c * q + b) * q + a;
        V[pt] = (well_sum(xq, cx, dd, inv2w2) + (vq ? vq[pt] : 0.0)) * jac;
        if (wv) (*wv)[(size_t)e * q * q * q + pt] = V[pt] * m.gq_w[a] * m.gq_w[b] * m.gq_w[c];
      }
      // T1[c][b][il] = sum_a BB[a][il] V[c][b][a]
      for (int cb = 0; cb < q * q; ++cb)
        for (int il = 0; il < nn; ++il) {
          double s = 0.0;
          for (int a = 0; a < q; ++a) s += BB[a * nn + il] * V[cb * q + a];
          T1[cb * nn + il] = s;
        }
      // T2[c][jm][il] = sum_b BB[b][jm] T1[c][b][il]
      for (int c = 0; c < q; ++c)
        for (int jm = 0; jm < nn; ++jm)
          for (int il = 0; il < nn; ++il) {
            double s = 0.0;
            for (int b = 0; b < q; ++b) s += BB[b * nn + jm] * T1[(c * q + b) * nn + il];
            T2[(c * nn + jm) * nn + il] = s;
          }
      // V_e[(i j k),(l m n)] = sum_c BB[c][kn] T2[c][jm][il]
      for (int k = 0; k < n1; ++k) for (int nk = 0; nk < n1; ++nk) {
        int kn = k * n1 + nk;
        for (int j = 0; j < n1; ++j) for (int mj = 0; mj < n1; ++mj) {
          int jm = j * n1 + mj;
          for (int i = 0; i < n1; ++i) for (int li = 0; li < n1; ++li) {
            int il = i * n1 + li;
            double s = 0.0;
            for (int c = 0; c < q; ++c) s += BB[c * nn + kn] * T2[(c * nn + jm) * nn + il];
            int r = i + n1 * (j + n1 * k), col = li + n1 * (mj + n1 * nk);
            He[r * ne + col] = s;
          }
        }
      }
      // H~_e = D^{-1/2} (1/2 K + V_e) D^{-1/2}; rows/cols of eliminated nodes zero
      double* out = &Ht[(size_t)e * ne * ne];
      const int32_t* dm = &m.dofmap[e * ne];
      for (int r = 0; r < ne; ++r) {
        if (dm[r] < 0) continue;
        double sr = 1.0 / std::sqrt(m.mass[dm[r]]);
        for (int c = 0; c < ne; ++c) {
          if (dm[c] < 0) continue;
          out[(size_t)r * ne + c] = (K[r * ne + c] + He[r * ne + c]) * sr / std::sqrt(m.mass[dm[c]]);
        }
      }
    }
  }
}

void build_mf_factors(const HostMesh& m, std::vector<double>& fac) {
  const int n1 = m.n1, q = m.q, nn = n1 * n1;
  fac.assign((size_t)6 * nn + 2 * q * n1, 0.0);
  for (int ax = 0; ax < 3; ++ax)
    for (int i = 0; i < n1; ++i)
      for (int l = 0; l < n1; ++l) {
        double sa = 0.0, ss = 0.0;
        for (int a = 0; a < q; ++a) {
          sa += m.gq_w[a] * m.B[a * n1 + i] * m.B[a * n1 + l];
          ss += m.gq_w[a] * m.D[a * n1 + i] * m.D[a * n1 + l];
        }
        fac[(size_t)ax * nn + i * n1 + l] = sa * m.h[ax] / 2.0;          // A_ax
        fac[(size_t)(3 + ax) * nn + i * n1 + l] = ss * 2.0 / m.h[ax];    // S_ax
      }
  double* B = fac.data() + 6 * nn;
  double* Bt = B + q * n1;
  for (int a = 0; a < q; ++a)
    for (int i = 0; i < n1; ++i) {
      B[a * n1 + i] = m.B[a * n1 + i];
      Bt[i * q + a] = m.B[a * n1 + i];
    }
}

void build_projectors(const HostMesh& m, const Projectors& pr, HostProjectors& out) {
  const int ns = (int)pr.h.size() / 4;
  const int n1 = m.n1, ne = m.ne, q = m.q;
  out = HostProjectors();
  out.nsite = ns;
  out.site_ptr.assign(ns + 1, 0);
  const double jac = m.h[0] * m.h[1] * m.h[2] / 8.0;
  const double rc2 = pr.rcut * pr.rcut, is2 = 1.0 / (2.0 * pr.sigma * pr.sigma);
  std::vector<std::vector<std::pair<int32_t, std::array<double, 4>>>> per_site(ns);
#pragma omp parallel
  {
    std::vector<double> chi(4 * q * q * q), T1(4 * q * q * n1), T2(4 * q * n1 * n1), ce(4 * ne);
#pragma omp for schedule(dynamic, 1)
    for (int s = 0; s < ns; ++s) {
      std::vector<std::pair<int32_t, std::array<double, 4>>> ent;
      const double* R = &pr.xyz[3 * s];
      for (int64_t e = 0; e < m.ncells; ++e) {
        int c3[3] = {(int)(e % m.n[0]), (int)((e / m.n[0]) % m.n[1]), (int)(e / ((int64_t)m.n[0] * m.n[1]))};
        // quick reject: distance from R (nearest image) to the cell box
        double r2 = 0.0;
        for (int ax = 0; ax < 3; ++ax) {
          double lo = c3[ax] * m.h[ax], hi = lo + m.h[ax];
          double best = 1e300;
          for (int sh = -1; sh <= 1; ++sh) {
            if (!m.per[ax] && sh) continue;
            double c = R[ax] + sh * m.len[ax];
            double dl = c < lo ? lo - c : (c > hi ? c - hi : 0.0);
            best = std::min(best, dl);
          }
          r2 += best * best;
        }
        if (r2 > rc2) continue;
        // chi_t at the Gauss points, times the quadrature weight and Jacobian
        bool any = false;
        for (int c = 0; c < q; ++c) for (int b = 0; b < q; ++b) for (int a = 0; a < q; ++a) {
          double x[3] = {c3[0] * m.h[0] + (m.gq_x[a] + 1.0) * m.h[0] / 2.0,
                         c3[1] * m.h[1] + (m.gq_x[b] + 1.0) * m.h[1] / 2.0,
                         c3[2] * m.h[2] + (m.gq_x[c] + 1.0) * m.h[2] / 2.0};
          double d[3], rr = 0.0;
          for (int ax = 0; ax < 3; ++ax) {
            d[ax] = x[ax] - R[ax];
            if (m.per[ax]) d[ax] -= m.len[ax] * std::nearbyint(d[ax] / m.len[ax]);
            rr += d[ax] * d[ax];
          }
          int qi = (c * q + b) * q + a;
          if (rr > rc2) {
            for (int t = 0; t < 4; ++t) chi[4 * qi + t] = 0.0;
            continue;
          }
          any = true;
          double g = std::exp(-rr * is2) * m.gq_w[a] * m.gq_w[b] * m.gq_w[c] * jac;
          chi[4 * qi] = g;
          chi[4 * qi + 1] = g * d[0] / pr.sigma;
          chi[4 * qi + 2] = g * d[1] / pr.sigma;
          chi[4 * qi + 3] = g * d[2] / pr.sigma;
        }
        if (!any) continue;
        // sum factorisation: contract x (a -> i), then y (b -> j), then z (c -> k)
        for (int cb = 0; cb < q * q; ++cb)
          for (int i = 0; i < n1; ++i)
            for (int t = 0; t < 4; ++t) {
              double acc = 0.0;
              for (int a = 0; a < q; ++a) acc += m.B[a * n1 + i] * chi[4 * (cb * q + a) + t];
              T1[4 * (cb * n1 + i) + t] = acc;
            }
        for (int c = 0; c < q; ++c)
          for (int j = 0; j < n1; ++j)
            for (int i = 0; i < n1; ++i)
              for (int t = 0; t < 4; ++t) {
                double acc = 0.0;
                for (int b = 0; b < q; ++b) acc += m.B[b * n1 + j] * T1[4 * ((c * q + b) * n1 + i) + t];
                T2[4 * ((c * n1 + j) * n1 + i) + t] = acc;
              }
        for (int k = 0; k < n1; ++k)
          for (int j = 0; j < n1; ++j)
            for (int i = 0; i < n1; ++i)
              for (int t = 0; t < 4; ++t) {
                double acc = 0.0;
                for (int c = 0; c < q; ++c) acc += m.B[c * n1 + k] * T2[4 * ((c * n1 + j) * n1 + i) + t];
                ce[4 * (i + n1 * (j + n1 * k)) + t] = acc;
              }
        for (int l = 0; l < ne; ++l) {
          int32_t g = m.dofmap[e * ne + l];
          if (g < 0) continue;
          std::array<double, 4> v = {ce[4 * l], ce[4 * l + 1], ce[4 * l + 2], ce[4 * l + 3]};
          ent.push_back({g, v});
        }
      }
      std::stable_sort(ent.begin(), ent.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
      for (auto& it : ent) {   // merge duplicates (unknowns shared by several cells)
        if (!per_site[s].empty() && per_site[s].back().first == it.first)
          for (int t = 0; t < 4; ++t) per_site[s].back().second[t] += it.second[t];
        else
          per_site[s].push_back(it);
      }
    }
  }
  // by-site CSR with the M^{-1/2} scaling
  for (int s = 0; s < ns; ++s) out.site_ptr[s + 1] = out.site_ptr[s] + (int64_t)per_site[s].size();
  out.site_dof.resize(out.site_ptr[ns]);
  out.site_c.resize(4 * out.site_ptr[ns]);
  std::vector<int64_t> cnt(m.ndofs + 1, 0);
  for (int s = 0; s < ns; ++s)
    for (size_t i = 0; i < per_site[s].size(); ++i) {
      int64_t pos = out.site_ptr[s] + (int64_t)i;
      int32_t g = per_site[s][i].first;
      double sc = 1.0 / std::sqrt(m.mass[g]);
      out.site_dof[pos] = g;
      for (int t = 0; t < 4; ++t) out.site_c[4 * pos + t] = per_site[s][i].second[t] * sc;
      cnt[g + 1]++;
    }
  // by-dof CSR (transpose), coefficients multiplied by h
  out.dof_ptr.assign(m.ndofs + 1, 0);
  for (int64_t j = 0; j < m.ndofs; ++j) out.dof_ptr[j + 1] = out.dof_ptr[j] + cnt[j + 1];
  out.dof_site.resize(out.dof_ptr[m.ndofs]);
  out.dof_c.resize(4 * out.dof_ptr[m.ndofs]);
  std::vector<int64_t> fill(out.dof_ptr.begin(), out.dof_ptr.end() - 1);
  for (int s = 0; s < ns; ++s)
    for (int64_t pos = out.site_ptr[s]; pos < out.site_ptr[s + 1]; ++pos) {
      int32_t g = out.site_dof[pos];
      int64_t o = fill[g]++;
      out.dof_site[o] = s;
      for (int t = 0; t < 4; ++t) out.dof_c[4 * o + t] = out.site_c[4 * pos + t] * pr.h[4 * s + t];
    }
}

void build_nl_cells(const HostMesh& m, const HostProjectors& hp, NlCells& out) {
  out = NlCells();
  const int ne = m.ne, mt = (ne + 127) / 128;
  const int64_t per_chunk = (int64_t)mt * 2048;   // elements of one term of one K-chunk
  out.chunk_off.assign(m.ncells + 1, 0);
  if (hp.nsite == 0) return;
  // owner cell of each unknown: the first (lowest) cell holding it
  std::vector<int32_t> owner(m.ndofs);
  for (int64_t j = 0; j < m.ndofs; ++j) owner[j] = m.node_ent[m.node_ptr[j]] / ne;
  std::vector<std::vector<int32_t>> sites(m.ncells);
  for (int64_t e = 0; e < m.ncells; ++e) {
    std::vector<int32_t>& st = sites[e];
    for (int l = 0; l < ne; ++l) {
      const int32_t g = m.dofmap[e * ne + l];
      if (g < 0 || owner[g] != e) continue;
      for (int64_t k = hp.dof_ptr[g]; k < hp.dof_ptr[g + 1]; ++k) st.push_back(hp.dof_site[k]);
    }
    std::sort(st.begin(), st.end());
    st.erase(std::unique(st.begin(), st.end()), st.end());
    out.chunk_off[e + 1] = out.chunk_off[e] + (int32_t)((4 * st.size() + 15) / 16);
  }
  out.zrow.assign((size_t)out.chunk_off[m.ncells] * 16, -1);
  for (int64_t e = 0; e < m.ncells; ++e)
    for (size_t i = 0; i < sites[e].size(); ++i)
      for (int t = 0; t < 4; ++t) out.zrow[(size_t)out.chunk_off[e] * 16 + 4 * i + t] = 4 * sites[e][i] + t;
  // projection blocks
  const int nk16 = (ne + 15) / 16;
  out.np.assign(m.ncells, 0);
  out.poff.assign(m.ncells + 1, 0);
  out.prow.assign(m.ncells + 1, 0);
  for (int64_t e = 0; e < m.ncells; ++e) {
    out.np[e] = (int32_t)((4 * sites[e].size() + 15) / 16 * 16);
    out.poff[e + 1] = out.poff[e] + (int64_t)nk16 * 3 * out.np[e] * 16;
    out.prow[e + 1] = out.prow[e] + out.np[e];
  }
  for (int s = 0; s < hp.nsite; ++s)
    for (int64_t pos = hp.site_ptr[s]; pos < hp.site_ptr[s + 1]; ++pos) {
      const int32_t g = hp.site_dof[pos];
      const int32_t ent = m.node_ent[m.node_ptr[g]];   // the owner's row: e ne + l
      const int64_t e = ent / ne;
      const int l = ent % ne;
      const std::vector<int32_t>& st = sites[e];
      const int slot = (int)(std::lower_bound(st.begin(), st.end(), s) - st.begin());
      for (int t = 0; t < 4; ++t) {
        const int k = 4 * slot + t, kc = l % 16;
        const int64_t off = (k >> 3) * 128 + (kc >> 3) * 64 + (k & 7) * 8 + (kc & 7);
        out.pz_pos.push_back(out.poff[e] + (int64_t)(l / 16) * 3 * out.np[e] * 16 + off);
        out.pz_val.push_back(hp.site_c[4 * pos + t]);
      }
    }
  out.red_ptr.assign(hp.nsite + 1, 0);
  for (int64_t e = 0; e < m.ncells; ++e)
    for (int32_t s : sites[e]) out.red_ptr[s + 1]++;
  for (int s = 0; s < hp.nsite; ++s) out.red_ptr[s + 1] += out.red_ptr[s];
  out.red_row.assign(out.red_ptr[hp.nsite], 0);
  {
    std::vector<int32_t> fill(out.red_ptr.begin(), out.red_ptr.end() - 1);
    for (int64_t e = 0; e < m.ncells; ++e)     // ascending cells: fixed summation order
      for (size_t i = 0; i < sites[e].size(); ++i)
        out.red_row[fill[sites[e][i]]++] = out.prow[e] + 4 * (int64_t)i;
  }
  for (int64_t e = 0; e < m.ncells; ++e) {
    const std::vector<int32_t>& st = sites[e];
    for (int l = 0; l < ne; ++l) {
      const int32_t g = m.dofmap[e * ne + l];
      if (g < 0 || owner[g] != e) continue;
      const int tile = l / 128, r = l % 128;
      for (int64_t k = hp.dof_ptr[g]; k < hp.dof_ptr[g + 1]; ++k) {
        const int slot = (int)(std::lower_bound(st.begin(), st.end(), hp.dof_site[k]) - st.begin());
        for (int t = 0; t < 4; ++t) {
          const int kk = 4 * slot + t;
          const int64_t chunk = out.chunk_off[e] + kk / 16;
          const int kc = kk % 16;
          // element offset as bf_elem_off(r, kc) of the 128 x 16 tile block
          const int64_t off = (r >> 3) * 128 + (kc >> 3) * 64 + (r & 7) * 8 + (kc & 7);
          out.nz_pos.push_back(chunk * 3 * per_chunk + (int64_t)tile * 2048 + off);
          out.nz_val.push_back(hp.dof_c[4 * k + t]);
        }
      }
    }
  }
}

}  // namespace chfsi
