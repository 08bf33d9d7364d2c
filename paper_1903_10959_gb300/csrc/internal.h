// Internal declarations shared by the translation units of libchfsi.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/chfsi.h"

namespace chfsi {

// Assembly modes of one (cell, local node) pair.  Cells are processed colour
// by colour; cells of one colour share no unknown.  For each unknown the
// first cell (lowest colour) stores its contribution into the partial-sum
// buffer W, intermediate cells add into W, and the last cell adds W to its
// own contribution and finishes the Chebyshev update of that unknown.  An
// unknown covered by a single cell is finished directly.
enum NodeMode : uint8_t {
  MODE_FINAL_DIRECT = 0,  // only contributor: finish from the cell result
  MODE_STORE = 1,         // first of several: W = contribution
  MODE_ACCUM = 2,         // middle: W += contribution
  MODE_FINAL = 3,         // last: finish from W + contribution
  MODE_SKIP = 4           // eliminated (Dirichlet) node
};

// ---------------------------------------------------------------- host mesh
struct HostMesh {
  int n[3];
  double len[3], h[3];
  int p, n1, ne, q;            // degree, nodes per direction, nodes per cell, quad points
  bool per[3];                 // axis periodic (else Dirichlet)
  int64_t nd[3];               // unknowns per direction
  int64_t ndofs;
  int64_t ncells;
  std::vector<int32_t> dofmap; // ncells * ne, -1 for eliminated
  std::vector<uint8_t> modes;  // ncells * ne
  std::vector<int32_t> colour_cells;   // cells ordered by colour
  std::vector<int64_t> colour_offsets; // ncolours + 1
  std::vector<double> mass;    // ndofs
  // owner-computes assembly: the cell-local rows (e * ne + l) holding each
  // unknown, in ascending cell order (fixed summation order)
  std::vector<int32_t> node_ptr, node_ent;
  // 1-D rules
  std::vector<double> gll_x, gll_w, gq_x, gq_w;
  std::vector<double> B, D;    // (q x n1) basis values / d/dxi at Gauss points
};

void build_mesh(const chfsi_mesh_desc& d, HostMesh& m);        // map, colours, modes, mass

// Electron density at the Gauss points (density.cu).
struct DensityArgs {
  const void* X;             // M x n block (binary64 or binary32), columns weighted 2
  int64_t ldx;
  int n;
  const void* Xfr;           // M x nfr partially occupied block, columns weighted wfr
  int64_t ldfr;
  int nfr;
  const double* wfr;         // device, nfr weights 2 (f_j - 1)
  const int32_t* dofmap;     // device, ncells x n1^3
  const double* minv_sqrt;   // device, M^{-1/2} per unknown
  const double* B;           // device, q x n1 basis values at the Gauss points
  const double* Bh;          // host copy of B (the binary32 kernel takes it as a parameter), may be null
  int64_t ncells;
  int n1, q, is_double;
  double* rho;               // device, ncells x q^3
};
cudaError_t launch_density(const DensityArgs& a, cudaStream_t s);
void gll_rule(int p, std::vector<double>& x, std::vector<double>& w);
void gauss_rule(int q, std::vector<double>& x, std::vector<double>& w);

struct Wells {
  std::vector<double> xyz, depth, width;
  // optional potential values at the Gauss points of every cell, added to the
  // wells (cells x fastest, point a + q (b + q c)); empty when unset
  std::vector<double> vqp;
};
struct Projectors {
  std::vector<double> xyz, h;
  double sigma = 0.8, rcut = 3.0;
};

// Cell matrices H~_e (binary64, row-major ne x ne per cell) for all cells;
// wv (optional): per cell, w_a w_b w_c jac V at the q^3 Gauss points (the
// potential factor of the matrix-free apply).
void build_cell_matrices(const HostMesh& m, const Wells& w, std::vector<double>& Ht,
                         std::vector<double>* wv = nullptr);
// 1-D factors of the matrix-free apply: A_x, A_y, A_z, S_x, S_y, S_z (n1 x n1,
// consistent mass and stiffness by the Gauss rule), B (q x n1) and B^T.
void build_mf_factors(const HostMesh& m, std::vector<double>& fac);

// Scaled projector matrix C~ = C M^{-1/2} in two compressed forms:
//  by site: for site s, rows [site_ptr[s], site_ptr[s+1]) of (dof, c[4]);
//  by dof:  for unknown j, entries [dof_ptr[j], dof_ptr[j+1]) of (site, c[4]).
struct HostProjectors {
  int nsite = 0;
  std::vector<int64_t> site_ptr;
  std::vector<int32_t> site_dof;
  std::vector<double> site_c;      // 4 per entry
  std::vector<int64_t> dof_ptr;
  std::vector<int32_t> dof_site;
  std::vector<double> dof_c;       // 4 per entry, already multiplied by h
};
void build_projectors(const HostMesh& m, const Projectors& pr, HostProjectors& out);

// The projector expansion C~ h Z (Eq. nonlocalHamDiscrete) as extra K-chunks
// of the cell products: cell e takes the rows of the unknowns it owns (the
// first cell holding them, ascending cell order), and its K axis runs over
// the 4 projectors of the sites touching those rows (4 ns_e values, padded to
// chunks of 16).  chunk_off: ncells + 1 chunk offsets; zrow: per chunk 16 rows
// of Z (4 site + t, -1 for padding); nz_pos / nz_val: the nonzero entries
// B[k][l] = h-scaled coefficient of node l for projector k, at their element
// position in a K-chunk-major block layout (chunk, 128-row tile, 16 x 128
// core-matrix order, as the packed cell matrices), term 0.
struct NlCells {
  std::vector<int32_t> chunk_off;
  std::vector<int32_t> zrow;
  std::vector<int64_t> nz_pos;
  std::vector<double> nz_val;
  // the projection Z = C~^T Y as the transposed blocks: cell e contributes the
  // partial sums of its owned rows for its np[e] = 4 ns_e projectors (padded
  // to 16) as rows prow[e] .. prow[e] + np[e] of a partial array; its block
  // (K = the cell's nodes in chunks of 16, N = np[e]) starts at element
  // poff[e]; pz_pos / pz_val its nonzeros (term 0, coefficients without h);
  // red_ptr / red_row: per site, the partial rows (4 slot of its cells, in
  // ascending cell order) whose sums give Z's rows 4 s .. 4 s + 3
  std::vector<int32_t> np;
  std::vector<int64_t> poff, prow;
  std::vector<int64_t> pz_pos;
  std::vector<double> pz_val;
  std::vector<int32_t> red_ptr;
  std::vector<int64_t> red_row;
};
void build_nl_cells(const HostMesh& m, const HostProjectors& hp, NlCells& out);

// --------------------------------------------------------------- device side
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct FilterStep {       // one recurrence step Y_out = alpha (H~ Y_in - c Y_in) + beta Y_prev
  double alpha, beta, shift;
};

// Launchers implemented in kernels_fp64.cu / kernels_tc.cu.  All take the
// context stream and return cudaGetLastError() of the launch.
struct CellLaunch {
  const double* Ht;           // ncells * ne * ne (binary64)
  const float* Ht32;          // tensor-core layout (mixed), may be null
  const int32_t* dofmap;
  const uint8_t* modes;
  const int32_t* cells;       // cells of this colour
  int64_t ncells_colour;
  int ne;
  int ncol;
  int64_t ld;                 // leading dimension of Yin / Yout / Yprev / W / NL
  int64_t ld_in, ld_out, ld_prev;
};

cudaError_t launch_cell_fp64(const CellLaunch& L, const double* Yin, double* Yout,
                             const double* Yprev, double* W, const double* NL, int64_t ld_w,
                             FilterStep st, cudaStream_t s);

// Matrix-free binary64 cell apply (kernels_mf.cu): same contract as
// launch_cell_fp64 for one colour, with H~_e applied by sum factorisation.
struct MfLaunch {
  const double* fac;          // 1-D factors: A_x, A_y, A_z, S_x, S_y, S_z (n1 x n1), B (q x n1), B^T
  const double* wv;           // per cell, w_a w_b w_c jac V at the q^3 Gauss points
  const double* minv_sqrt;    // M^{-1/2} per unknown
  const int32_t* dofmap;
  const uint8_t* modes;
  const int32_t* cells;       // cells of this colour
  int64_t ncells_colour;
  int p, q, ncol;
  int64_t ld_in, ld_out, ld_prev, ld_w;
  int kinetic_only;           // 1: 1/2 K_e only (the scaled stiffness of the Poisson solve)
};
bool mf_supported(int p, int q);
// Bloch (k-point) form of the same apply on interleaved (real, imaginary)
// column pairs; L.fac holds the k-point factors (see kernels_mf.cu), ncol even.
cudaError_t launch_mfk_cell_fp64(const MfLaunch& L, const double* Yin, double* Yout,
                                 const double* Yprev, double* W, FilterStep st, cudaStream_t s);
cudaError_t launch_mf_cell_fp64(const MfLaunch& L, const double* Yin, double* Yout,
                                const double* Yprev, double* W, const double* NL, FilterStep st,
                                cudaStream_t s);

cudaError_t launch_fill_uniform(void* X, int64_t ldx, int64_t rows, int ncol, uint64_t key,
                                int is_double, cudaStream_t s);
cudaError_t launch_copy_cols(const void* src, int64_t lds, void* dst, int64_t ldd, int64_t rows,
                             int ncol, int src_double, int dst_double, cudaStream_t s);
// Pitched 2-D byte copy by the SMs (src / dst device or device-mapped host).
cudaError_t launch_copy2d(const void* src, int64_t src_pitch, void* dst, int64_t dst_pitch,
                          int64_t rows, int64_t row_bytes, int nsm, cudaStream_t s);
cudaError_t launch_scale_rows(void* X, int64_t ldx, int64_t rows, int ncol, const double* sv,
                              int is_double, cudaStream_t s);

// Gram: C(n1 x n2, column-major ldc) = A^T B over rows [0, M); A col offset
// handled by the caller through pointers.  lower_only: skip tiles strictly
// above the diagonal (i < j) when A == B geometry is square-symmetric.
cudaError_t launch_gram_fp64(const double* A, int64_t lda, const double* B, int64_t ldb,
                             int64_t M, int n1, int n2, double* C, int64_t ldc, int lower_only,
                             double* partial, size_t partial_bytes, cudaStream_t s);
// C(M x n2, row-major ldc) = A(M x n1, row-major lda) * U, U(n1 x n2) column-major ldu
// (trans_u: U(k, j) read from U[j + k*ldu]); upper_tri: U(k, j) = 0 for k > j.
cudaError_t launch_tallgemm_fp64(const double* A, int64_t lda, const double* U, int64_t ldu,
                                 int64_t M, int n1, int n2, double* C, int64_t ldc, int upper_tri,
                                 int trans_u, cudaStream_t s);
// col norms: out[i] = sum_j w_j (Y[j,i] - lam_i X[j,i])^2 (w null -> 1), binary64 accumulation
cudaError_t launch_resid_norms(const double* Y, int64_t ldy, const double* X, int64_t ldx,
                               int64_t M, int n, const double* lam, const double* wgt,
                               double* out_sq, double* partial, size_t partial_bytes,
                               cudaStream_t s);
cudaError_t launch_axpy2(double* w, const double* v, const double* vp, int64_t M, double a,
                         double b, cudaStream_t s);
cudaError_t launch_scal_copy(double* v, const double* w, int64_t M, double sc, cudaStream_t s);
// X (lower triangle, column-major ldx) = L^{-1} for a lower triangular L
// (column-major ldl, diagonal nonzero); X's strict upper triangle untouched.
bool trinv_lower_supported(int n);
cudaError_t launch_trinv_lower_fp64(const double* L, int64_t ldl, int n, double* X, int64_t ldx,
                                    cudaStream_t s);

// nonlocal: Z (nproj x ncol) = C~ Y ; NL (M x ncol) = C~^T h Z
cudaError_t launch_nl_project_fp64(const int64_t* site_ptr, const int32_t* site_dof,
                                   const double* site_c, int nsite, const double* Y, int64_t ldy,
                                   int ncol, double* Z, cudaStream_t s);
cudaError_t launch_nl_expand_fp64(const int64_t* dof_ptr, const int32_t* dof_site,
                                  const double* dof_c, int64_t M, const double* Z, int ncol,
                                  double* NL, int64_t ldn, cudaStream_t s);

uint64_t stream_key(uint64_t seed, uint64_t stream);

// Count of kernel launches issued by this library (all contexts, monotonic).
void note_launch();
int64_t launch_count();

}  // namespace chfsi
