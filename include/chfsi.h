/*
 * chfsi.h -- C ABI of a GB300 (sm_103a) library for one Chebyshev-filtered
 * subspace iteration (ChFSI) step of the real-space spectral finite-element
 * Kohn-Sham method of arXiv:1903.10959 (DFT-FE), for a fixed effective
 * potential on a uniform hexahedral mesh with Gauss-Lobatto-Legendre nodes.
 *
 * Problem statement (Sec. 2.4, Eqs. discreteHam, nonlocalHamDiscrete, hep):
 * the FE discretisation gives H Psi = eps M Psi with H = H_loc + H_nl and a
 * diagonal GLL mass M; the library works with the standard form
 *   H~ = M^{-1/2} H M^{-1/2},   x~ = M^{1/2} Psi                (Eq. hep)
 * and computes the lowest eigenpairs of H~ by ChFSI (step 7 of Algorithm scf):
 * Chebyshev filter (Eq. chebFilter, Sec. 3.3), CholGS (Algorithm CholGS,
 * Sec. 3.4) and Rayleigh-Ritz (Sec. 3.5).
 *
 * Conventions for every call:
 *  - Wavefunction blocks X are DEVICE pointers owned by the caller, row-major
 *    "DOF-major" (Sec. 3.3.1: the values of all vectors at one unknown are
 *    contiguous): element (unknown j, vector i) is at X[j * ldx + i],
 *    ldx >= ncol.  The element type is double for CHFSI_FP64 and float for
 *    the mixed precisions.  The library never frees caller memory.
 *  - Host arrays (eigenvalues, residuals, mass, inputs) are plain host
 *    pointers owned by the caller.
 *  - Every call runs on the context's CUDA stream.  Calls that return host
 *    values (bounds, eigenvalues, residuals, mass) synchronise that stream;
 *    the others are asynchronous.
 *  - Errors are returned as chfsi_status; no exception crosses the ABI.  A
 *    CUDA or cuSOLVER error is latched in the context (every later call
 *    returns CHFSI_ERR_CUDA) and described by chfsi_last_error().
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef CHFSI_H
#define CHFSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct chfsi_ctx chfsi_ctx;

typedef enum {
  CHFSI_OK = 0,
  CHFSI_ERR_ARG = 1,      /* invalid argument (null pointer, bad size, bad order of calls) */
  CHFSI_ERR_OOM = 2,      /* device allocation failed or exceeds the context's budget     */
  CHFSI_ERR_CUDA = 3,     /* CUDA / cuSOLVER failure; see chfsi_last_error                */
  CHFSI_ERR_NOT_SPD = 4,  /* CholGS: overlap matrix not positive definite (X unchanged)   */
  CHFSI_ERR_EIG = 5,      /* Rayleigh-Ritz: eigensolver did not converge                 */
  CHFSI_ERR_STATE = 6,    /* call made before the data it needs (e.g. filter before build) */
  CHFSI_ERR_TIMEOUT = 7   /* a bounded device-side wait gave up (kernel unwound; see last_error) */
} chfsi_status;

typedef enum {
  /* Everything in binary64: cell products, recurrence, overlap, projection. */
  CHFSI_FP64 = 0,
  /* X stored in binary32; filter cell products on tcgen05 tensor cores as
   * three TF32 products per term (hi*hi + hi*lo + lo*hi, FP32 accumulation),
   * which keeps binary32 accuracy; off-diagonal blocks of S and H^ likewise;
   * diagonal blocks, Cholesky, eigensolve and residuals in binary64. */
  CHFSI_MIXED_TF32X3 = 1,
  /* As above with one TF32 product per term (faster, ~5e-4 relative). */
  CHFSI_MIXED_TF32 = 2,
  /* Binary32 storage; cell products with both operands split into three
   * bf16 terms (about 24 bits) and six kind::f16 MMAs (K = 16) accumulated
   * in FP32; Gram / rotations as CHFSI_MIXED_TF32X3. */
  CHFSI_MIXED_BF16X3 = 3,
  /* Binary32 storage; cell products with both operands split into two fp16
   * terms (about 22 bits, as 3xTF32) after exact power-of-two scaling (each
   * cell matrix by its maximum, each column of the block by its maximum,
   * undone in the epilogue), three kind::f16 MMAs (K = 16) accumulated in
   * FP32: half the tensor work of BF16x3.  Gram / rotations as
   * CHFSI_MIXED_TF32X3.  Single-context calls only (not the batch API). */
  CHFSI_MIXED_F16X2 = 4
} chfsi_precision;

/* Uniform mesh of ncell[0] x ncell[1] x ncell[2] boxes on [0,len[0]] x ... .
 * p: FE degree (1..8), n_e = (p+1)^3 nodes per cell, GLL nodes (Sec. 2.4).
 * periodic[d] != 0: axis d periodic (opposite faces identified; requires
 * ncell[d] >= 2); otherwise homogeneous Dirichlet on the two faces normal to
 * axis d (boundary nodes eliminated; requires ncell[d] p >= 2).  All three
 * set: a periodic crystal; none: an isolated system; some: a semi-periodic
 * system such as a slab (the paper's periodic, non-periodic and
 * semi-periodic boundary conditions, Sec. 1).
 * quad_points: Gauss-Legendre points per direction for the Hamiltonian
 * integrals (0 selects p + 2); the mass always uses the GLL rule. */
typedef struct {
  int ncell[3];
  double len[3];
  int p;
  int periodic[3];
  int quad_points;
} chfsi_mesh_desc;

/* Create a context on the current CUDA device.  stream: a cudaStream_t (NULL
 * for the legacy default stream).  Builds the cell->unknown map, the colour
 * schedule of the assembly and the global diagonal GLL mass (Sec. 2.4). */
chfsi_status chfsi_create(const chfsi_mesh_desc* desc, void* stream, chfsi_ctx** out);
chfsi_status chfsi_destroy(chfsi_ctx* ctx);
const char*  chfsi_last_error(const chfsi_ctx* ctx);

/* Number of unknowns M: the product over the axes of n p (periodic axis) or
 * n p - 1 (Dirichlet axis). */
int64_t      chfsi_num_dofs(const chfsi_ctx* ctx);

/* Global diagonal mass M_jj (GLL quadrature; text after Eq. hep) -> host_out[M]. */
chfsi_status chfsi_mass_diag(chfsi_ctx* ctx, double* host_out);

/* Effective potential V(x) = -sum_a depth[a] exp(-|x - R_a|^2 / (2 width[a]^2)),
 * R_a = xyz[3a..3a+2]; each well is summed over its image shifts
 * {-1,0,1} len[d] along every periodic axis d (27 images when all three are).  Arrays are host, copied.  Invalidates any
 * previous chfsi_build. */
chfsi_status chfsi_set_potential_gaussians(chfsi_ctx* ctx, int n, const double* xyz,
                                           const double* depth, const double* width);

/* General effective potential (V_eff of Eq. discreteHam, e.g. the Hartree +
 * exchange-correlation + local pseudopotential field of an SCF step, Algorithm
 * scf) given by its values at the Gauss points of every cell, where the V_e
 * integrals are evaluated: v[e q^3 + a + q (b + q c)] for point (a, b, c) of
 * cell e (cells x fastest), q = p + 2 Gauss-Legendre points per direction --
 * the same points and layout as the output of chfsi_density.  The values are
 * added to the Gaussian wells of chfsi_set_potential_gaussians (set no wells
 * for a general field).  v: host, count = ncells * q^3 doubles, copied; all
 * finite.  v = NULL with count = 0 clears.  A wrong count returns
 * CHFSI_ERR_ARG.  Invalidates any previous chfsi_build. */
chfsi_status chfsi_set_potential_qp(chfsi_ctx* ctx, const double* v, int64_t count);

/* Separable nonlocal projectors (Eqs. nlps, nonlocalHamDiscrete): per site s,
 * four channels chi = g(r) {1, x/sigma, y/sigma, z/sigma}, g = exp(-r^2/(2 sigma^2))
 * for r <= rcut (0 beyond), r to the nearest image along the periodic axes, with couplings
 * h[4 s + k] (Ha).  H_nl = sum C^T h C, C_{k,j} = int chi_k N_j.  n = 0 clears. */
chfsi_status chfsi_set_projectors(chfsi_ctx* ctx, int n, const double* xyz, const double* h,
                                  double sigma, double rcut);

/* Build the cell matrices H~_e = D_e^{-1/2} (1/2 K_e + V_e) D_e^{-1/2}
 * (Eq. discreteHam scaled as in Eq. hep; D_e = global mass at the cell's
 * nodes) in binary64 on the host, and upload them together with the
 * precision-specific device copies and the projector data. */
chfsi_status chfsi_build(chfsi_ctx* ctx);

/* Column block size of the filter (Sec. 3.3.1 "B^f"; default 200 or ncol if
 * smaller) and diagonal block size of the mixed overlap/projection products
 * (default 1: the diagonal entries, as in the paper; a power of two <= 32).
 * Takes effect on the next call. */
chfsi_status chfsi_set_blocking(chfsi_ctx* ctx, int filter_block, int diag_block);

/* Columns per CTA of the tensor-core cell kernel (mixed precisions): 64
 * (default; two CTAs per SM) or 128 (one CTA per SM, wider MMAs).  Results
 * do not depend on it. */
chfsi_status chfsi_set_cell_tile(chfsi_ctx* ctx, int tile);

/* Filter lanes (mixed precisions; default 1): the columns of a filter call
 * are cut into up to `lanes` groups of whole 128-column tiles, each filtered
 * on its own stream with its own scratch, so the memory-bound assembly of one
 * lane overlaps the tensor-core cell products of another (the columns of the
 * Chebyshev filter, Eq. chebFilter, are independent).  Results are identical
 * to one lane.  Scratch per lane is sized by its columns, so the total equals
 * one lane's.  lanes in 1..4, else CHFSI_ERR_ARG. */
chfsi_status chfsi_set_filter_lanes(chfsi_ctx* ctx, int lanes);

/* Tile kernels of the mixed-precision block products of CholGS and
 * Rayleigh-Ritz (the overlap S = X^T X, the projection X^T H X and the
 * rotations X U, Sec. 3.3.2-3.3.3): tall = the rotation kernel, gram = the
 * overlap kernel; -1 (default) chooses by size, 0 = 128 x 128 output tiles,
 * 1 = 256-row tiles (two TMEM accumulators per CTA, each operand chunk
 * shared by twice the products).  Results are the same to rounding order
 * of the binary32 accumulators; CHFSI_ERR_ARG for other values. */
chfsi_status chfsi_set_gemm_kernels(chfsi_ctx* ctx, int tall, int gram);

/* Variant of the BF16x3 cell kernel (results are bit-identical): 2 (default)
 * = warps gather the cell's rows of Y into registers and split them, with the
 * cell-matrix chunks and the split Y chunks in separate shared-memory rings
 * (the matrix copies run up to five chunks ahead at p = 6); 0 = one ring
 * shared by both operands; 1 = the rows staged by bulk async copies several
 * chunks ahead and split from shared memory (used when the block is 16-byte
 * aligned with a leading dimension and a column count that are multiples of
 * 4, else 0); 3 = as 2 with four gather warp pairs instead of two; 4 = both
 * row parts of a cell per thread block (p = 6, 7; else 2); 5 = as 2 with
 * three 128-column tiles per thread block, the rings running on across them
 * and four epilogue warps; 6 = all column tiles per thread block, one block
 * per SM with two accumulators (the MMAs of a tile overlap the epilogue of
 * the previous one) and four gather warp pairs.  Modes 4-6 take no
 * projector chunks (the projector term then stays in the assembly). */
chfsi_status chfsi_set_cell_gather(chfsi_ctx* ctx, int mode);

/* Cell operator of the binary64 path (every CHFSI_FP64 apply, and the
 * binary64 products of the mixed precisions' last Rayleigh-Ritz, residuals
 * and polish): 0 = the stored cell matrices H~_e (dense n_e x n_e products,
 * Sec. 3.3.1); 1 = matrix-free, H_e applied by sum factorisation over the
 * tensor-product cell (1-D mass / stiffness / Gauss-point factors, the
 * alternative the paper notes for the cell-level products), 3.2x (p = 6) to
 * 5.5x (p = 8) fewer flops; -1 = the library's default: matrix-free where it
 * exists, else the cell matrices.  The matrix-free form
 * needs 2 <= p <= 8 and quad_points = p + 2 (CHFSI_ERR_ARG otherwise).  Both
 * give the same operator to rounding.  chfsi_fp64_operator returns the one in
 * use (0 or 1). */
chfsi_status chfsi_set_fp64_operator(chfsi_ctx* ctx, int op);
int          chfsi_fp64_operator(const chfsi_ctx* ctx);

/* Autotuner of the filter's blocking: times a degree-2 filter on a scratch
 * copy of X (M x n, device; X itself is not modified) for every candidate
 * (wavefunction block 200, ceil(n/2) and n, times cell tile 64 and 128 for
 * the mixed precisions), and keeps the fastest in the context (as
 * chfsi_set_blocking / chfsi_set_cell_tile would).  Needs a built context
 * and M * n element-sized bytes of free device memory for the copy.
 * A candidate whose scratch does not fit in device memory is skipped (its
 * ms_out entry is -1); CHFSI_ERR_OOM only when none fits.  The scratch grown
 * while tuning is released afterwards.  block_out, tile_out may be NULL;
 * ms_out (may be NULL) receives the time of each candidate in that order (at
 * most 6 entries).  Synchronises. */
chfsi_status chfsi_autotune(chfsi_ctx* ctx, const void* X, int64_t ldx, int n,
                            chfsi_precision prec, int* block_out, int* tile_out, double* ms_out);

/* Fill rows x ncol of X (device, leading dimension ldx) with the seeded
 * SplitMix64 stream (Steele, Lea & Flood 2014), mapped to [-1, 1): element
 * (r, c) is draw r * ncol + c of the stream keyed by (seed, stream). */
chfsi_status chfsi_fill_uniform(chfsi_ctx* ctx, void* X, int64_t ldx, int64_t rows, int ncol,
                                uint64_t seed, uint64_t stream, chfsi_precision prec);

/* Y = H~ X on ncol vectors (one application of Eq. hep's operator, the inner
 * operation of Eq. chebFilter).  X and Y: device, M x ncol, must not overlap.
 * The first call in a mixed precision packs the cell matrices for it (a
 * library-owned device copy: three bf16 terms, 6 B per entry, for
 * CHFSI_MIXED_BF16X3; the TF32 hi / lo pair, 8 B per entry, for the TF32
 * forms) and returns CHFSI_ERR_OOM when that copy does not fit.  The same
 * holds for every entry point below that takes a mixed precision. */
chfsi_status chfsi_apply(chfsi_ctx* ctx, const void* X, int64_t ldx, void* Y, int64_t ldy,
                         int ncol, chfsi_precision prec);

/* Y = H~ X in binary64 like chfsi_apply, but without allocating any device
 * memory.  The paper has no counterpart: this exists for callers that cannot
 * call cudaMalloc from inside their step -- for example host frameworks whose
 * own pool allocator owns the GPU's memory (a library allocation would fail
 * or escape their accounting), or latency-critical loops where cudaMalloc /
 * cudaFree would synchronise the device.  The caller passes X and Y (device,
 * M x ncol, not overlapping); the assembly scratch (the partial-sum buffer,
 * plus the projector buffers when projectors are set) lives in one fixed
 * file-scope device array of 64 MiB that every GPU loading the library keeps
 * until the process exits.  Limit: M * ncol * 8 bytes (twice that plus
 * 4 * nsite * ncol * 8 with projectors) must fit in 64 MiB; larger requests
 * return CHFSI_ERR_ARG with the sizes in chfsi_last_error, so split the
 * columns over several calls.  The context's device must be the current
 * device (CHFSI_ERR_STATE otherwise).  The first call on a context looks up
 * the array's device address (cudaGetSymbolAddress) and keeps it in the
 * context; make that first call before any stream capture.  A failed lookup
 * returns CHFSI_ERR_CUDA without latching the context.  All calls share the array and nothing in it needs to
 * start at zero (each call writes every scratch entry it reads); calls whose
 * work overlaps on the GPU (other streams, other contexts on the device)
 * race on it, so serialise them.  Asynchronous on the context's stream. */
chfsi_status chfsi_apply_noalloc(chfsi_ctx* ctx, const double* X, int64_t ldx, double* Y,
                                 int64_t ldy, int ncol);

/* Test hook of the bounded device waits (no counterpart in the paper; off by
 * default).  on != 0: in later BF16x3 cell-kernel launches on this device
 * (gather modes 0 and 2, the default), one
 * gather warp of the first thread block withholds its arrival on the first
 * K-chunk's barrier, so the MMA warp's bounded wait (2 s) runs out; the
 * kernel unwinds (waits for its own copies in flight, frees its TMEM) and the
 * call returns CHFSI_ERR_TIMEOUT without latching the context.  on = 0
 * restores normal operation; the next call gives the normal result.  For
 * tests of the error path only.  Synchronises the stream. */
chfsi_status chfsi_debug_withhold_arrival(chfsi_ctx* ctx, int on);

/* Degree-m Chebyshev filter (Eq. chebFilter) in the scaled form of Zhou &
 * Saad, in place on X (M x ncol): X <- T_m((H~ - c)/e) X / T_m((a0 - c)/e),
 * c = (a + b)/2, e = (b - a)/2; [a, b] is the damped interval, a0 < a the
 * lower end of the spectrum.  Requires a0 < a < b and degree >= 1. */
chfsi_status chfsi_filter(chfsi_ctx* ctx, void* X, int64_t ldx, int ncol, int degree,
                          double a, double b, double a0, chfsi_precision prec);

/* CholGS (Algorithm CholGS): S = X^T X, S = L L^T, X <- X L^{-T}, in place on
 * X (M x n).  Returns CHFSI_ERR_NOT_SPD and leaves X unchanged when the
 * Cholesky factorisation fails (cuSOLVER potrf + trtri, binary64). */
chfsi_status chfsi_cholgs(chfsi_ctx* ctx, void* X, int64_t ldx, int n, chfsi_precision prec);

/* Rayleigh-Ritz (Sec. 3.5): H^ = X^T H~ X, H^ Q = Q D (ascending, binary64
 * cuSOLVER syevd), X <- X Q in place.  evals_host[n] receives D. */
chfsi_status chfsi_rayleigh_ritz(chfsi_ctx* ctx, void* X, int64_t ldx, int n,
                                 chfsi_precision prec, double* evals_host);

/* Residuals in binary64 for n pairs (columns of X, evals_host):
 * res[i]  = ||H~ x_i - l_i x_i||_2 / ||x_i||_2, and, when gres != NULL,
 * gres[i] = ||H Psi_i - l_i M Psi_i||_2 with Psi_i = M^{-1/2} x_i / ||x_i||
 * (the generalized-problem residual of Eq. hep).  Either output may be NULL. */
chfsi_status chfsi_residuals(chfsi_ctx* ctx, const void* X, int64_t ldx, int n,
                             chfsi_precision prec, const double* evals_host,
                             double* res_host, double* gres_host);

/* Upper bound of spec(H~) by a k-step Lanczos run from the seeded start
 * vector (stream 7 of chfsi_fill_uniform): b = max Ritz value of the
 * tridiagonal + |beta_k| (the safeguard of Zhou & Saad; the paper ties the
 * filter to this bound, Sec. 3.3).  Binary64. */
chfsi_status chfsi_bounds(chfsi_ctx* ctx, int lanczos_steps, uint64_t seed, double* b_out);

/* Full ChFSI loop on X (M x n, in/out): CholGS + RR on the start block, then
 * `iters` times {filter(degree, a = max Ritz, b, a0 = min Ritz); CholGS; RR}
 * (step 7 of Algorithm scf).  b: upper bound (chfsi_bounds).  evals_host[n]
 * receives the final Ritz values.  When tol > 0 the loop stops early once
 * the largest residual of the lowest n_check pairs is below tol (adaptive
 * filtering, Sec. 3.3); n_check <= 0 means n.  iters_done may be NULL.
 * The stopping residual is the generalized one of chfsi_residuals (gres,
 * ||H Psi - l M Psi|| with Psi^T M Psi = 1) in binary64, with l the Ritz value
 * (FP64) or the column's binary64 Rayleigh quotient (mixed).
 * Mixed precisions: every RR but the last uses the tensor-core operator;
 * the last one applies H~ with binary64 cell products, so the returned
 * eigenvalues carry only second-order error from the binary32 subspace. */
chfsi_status chfsi_solve(chfsi_ctx* ctx, void* X, int64_t ldx, int n, int iters, int degree,
                         double b, double tol, int n_check, chfsi_precision prec,
                         double* evals_host, int* iters_done);

/* Mixed-precision ChFSI followed by a binary64 polish (the residual side of
 * the mixed-precision strategy, Secs. 3.4.2 and 3.5.2: binary32 arithmetic
 * where the subspace is still converging, binary64 where accuracy is set).
 * The binary32 filter's storage and FP32 accumulation leave the subspace with
 * a generalized residual near 1e-6; a few binary64 iterations from that
 * subspace remove it.  Steps:
 *  1. chfsi_solve on X (binary32, M x n) in precision prec (a mixed one),
 *     with iters, degree, b, tol, n_check as there, except that its last
 *     Rayleigh-Ritz stays in the tensor-core arithmetic;
 *  2. the binary64 copy X64 <- X (X64: caller-owned device block, M x n,
 *     leading dimension ldx64 >= n, not overlapping X; NULL: a library-owned
 *     staging block of M n 8 bytes);
 *  3. polish_iters binary64 iterations {filter of degree polish_degree with
 *     a = max Ritz, b, a0 = min Ritz of the previous Rayleigh-Ritz; CholGS;
 *     Rayleigh-Ritz} on X64;
 *  4. X <- the binary32 rounding of X64.
 * evals_host[n] receives the binary64 Ritz values of the last polish
 * iteration, iters_done (may be NULL) the mixed iterations run.  A polish
 * degree near the solve's degree damps the binary32 noise by the same factor
 * as one solve iteration; much lower degrees leave most of it.  Synchronises. */
chfsi_status chfsi_solve_polish(chfsi_ctx* ctx, float* X, int64_t ldx, int n, int iters, int degree,
                                double b, double tol, int n_check, chfsi_precision prec,
                                int polish_iters, int polish_degree, double* X64, int64_t ldx64,
                                double* evals_host, int* iters_done);

/* One ChFSI iteration (step 7 of Algorithm scf: filter of degree `degree`
 * with bounds a, b, a0, then CholGS and Rayleigh-Ritz) on a block held in HOST
 * memory, the transfers included: X_host (host, M x n, leading dimension
 * ldh, element type of prec) is copied into the caller's device block X
 * (M x n, ldx), the iteration runs on X, and the result is copied back into
 * X_host; evals_host[n] receives the Ritz values.  copy_mode: 0 = the SMs
 * move the rows over the coherent host link when the GPU can address X_host
 * (cudaHostGetDevicePointer succeeds: pinned memory from cudaHostAlloc or
 * cudaHostRegister, and on hosts whose GPU reaches pageable memory directly,
 * such as Grace, any host memory), else the copy engines; 1 = always the
 * copy engines (cudaMemcpy2DAsync); 2 = always the SMs (CHFSI_ERR_ARG when
 * the GPU cannot address X_host).  ms3 (may be NULL)
 * receives the device times of the host-to-device copy, the iteration and
 * the device-to-host copy (ms, CUDA events on the context stream).
 * Synchronises. */
chfsi_status chfsi_step_host(chfsi_ctx* ctx, void* X_host, int64_t ldh, void* X, int64_t ldx, int n,
                             int degree, double a, double b, double a0, chfsi_precision prec,
                             int copy_mode, double* evals_host, double* ms3);

/* Spectrum-splitting Rayleigh-Ritz (Algorithm rr, Sec. 3.5): H^ = X^T H~ X for
 * the CholGS output X (M x n, not modified), its n_fr largest eigenpairs in
 * binary64 (cuSOLVER syevdx, index range n-n_fr+1..n), and the partial
 * rotation X_fr = X Q_fr into the caller's block X_fr (device, M x n_fr,
 * leading dimension ldfr, same element type as X, must not overlap X).
 * evals_fr_host[n_fr] receives D_fr ascending.  CHFSI_ERR_EIG when syevdx
 * fails. */
chfsi_status chfsi_rayleigh_ritz_split(chfsi_ctx* ctx, const void* X, int64_t ldx, int n, int n_fr,
                                       void* Xfr, int64_t ldfr, chfsi_precision prec,
                                       double* evals_fr_host);

/* Fermi level (Algorithm dc, step 1): mu such that
 * 2 (n_oc + sum_i f(evals[i], mu)) = n_electrons, f the Fermi-Dirac function
 * 1 / (1 + exp((eps - mu) / kT)) (kT in Ha), over the n partially occupied
 * Ritz values; the n_oc lower states count as fully occupied.  Bisection on
 * the host to a relative width of 1e-15; occ_out[n] (may be NULL) receives
 * f(evals[i], mu).  CHFSI_ERR_ARG when the states cannot hold n_electrons.
 * Host only: needs no context or device. */
chfsi_status chfsi_fermi_level(int n, const double* evals, int n_oc, double n_electrons,
                               double kT, double* mu_out, double* occ_out);

/* Electron density (Algorithm dc, Eq. elecDensSP) at the Gauss points of
 * every cell (interpolation in the blocks' precision, binary64 sums):
 *   rho(x) = 2 sum_{i<n} psi_i(x)^2 + 2 sum_{j<n_fr} (f_j - 1) psi_fr,j(x)^2,
 * psi = M^{-1/2} x for the columns x of X (the CholGS output, M x n) and of
 * X_fr (chfsi_rayleigh_ritz_split), f_j = occ_fr_host[j] (chfsi_fermi_level).
 * n_fr = 0 gives the density of n doubly occupied states.  rho: device,
 * caller-owned, ncells * q^3 doubles with q = quad_points (p + 2 by default);
 * point (a, b, c) of cell e (cells x fastest) at rho[e q^3 + a + q (b + q c)].
 * Synchronises the stream. */
chfsi_status chfsi_density(chfsi_ctx* ctx, const void* X, int64_t ldx, int n, const void* Xfr,
                           int64_t ldfr, int n_fr, const double* occ_fr_host, chfsi_precision prec,
                           double* rho);

/* Psi^ = M^{-1/2} x~ in place (Eq. hep, recovery of the FE eigenvectors). */
chfsi_status chfsi_unscale(chfsi_ctx* ctx, void* X, int64_t ldx, int ncol, chfsi_precision prec);

/* Per-phase device times of the last chfsi_solve / filter / cholgs / rr call
 * (milliseconds, CUDA events): out[0] filter, out[1] cholgs, out[2] rr,
 * out[3] residual/other.  Synchronises. */
chfsi_status chfsi_last_timings(chfsi_ctx* ctx, double* out4);

/* Bytes of device memory the context currently holds. */
int64_t      chfsi_device_bytes(const chfsi_ctx* ctx);

/* Event timing of the filter kernels (on != 0: every cell-product and
 * assembly launch of this context is bracketed by CUDA events on its stream;
 * for measurement runs, the events cost a few microseconds per launch). */
chfsi_status chfsi_set_kernel_timing(chfsi_ctx* ctx, int on);

/* Accumulated device times since the last call, then reset:
 * out6[0] cell-product kernel ms, out6[1] assembly kernel ms, out6[2] and
 * out6[3] the numbers of launches timed, out6[4] ms of the binary32
 * projector kernels (projection + expansion), out6[5] their timed pairs.
 * Synchronises the stream. */
chfsi_status chfsi_kernel_timings(chfsi_ctx* ctx, double* out6);

/* Number of kernels this library has launched so far (all contexts; a
 * monotonic counter for accounting, e.g. launches per ChFSI iteration). */
int64_t      chfsi_kernel_launches(void);

/* ------------------------------------------------------------------- SCF
 * The self-consistent field loop around the ChFSI step (Algorithm scf,
 * Sec. 3.2), for periodic systems of Gaussian nuclear charges, on the device
 * with the matrix-free binary64 operator (needs 2 <= p <= 8 and
 * quad_points = p + 2, all three axes periodic). */

/* V_eff at the Gauss points given on the DEVICE (v: ncells * q^3 doubles,
 * the layout of chfsi_set_potential_qp), taken by the matrix-free operator
 * directly: the wells and any host values are replaced, the stored cell
 * matrices are released, and until the next chfsi_build only the binary64
 * precision is available (the mixed precisions return CHFSI_ERR_STATE).
 * Projectors set by an earlier chfsi_build stay.  Synchronises. */
chfsi_status chfsi_set_potential_qp_device(chfsi_ctx* ctx, const double* v);

/* Electrostatic potential (step 4 of Algorithm scf): phi with
 * -(1 / 4 pi) lap phi = f in the periodic box (Eq. ksproblemPer), in FE form
 * K phi = 4 pi F, F_j = int N_j f by the cells' Gauss rule, the net charge of
 * f neutralised by a uniform background, int phi = 0.  f: device, at the
 * Gauss points (ncells * q^3, chfsi_density layout); phi: device, M nodal
 * values.  Conjugate gradients on M^{-1/2} K M^{-1/2} (the matrix-free
 * stiffness) to relative residual tol, at most max_iter iterations;
 * iters / rel_residual (may be NULL) receive the count and the residual.
 * CHFSI_ERR_EIG when tol is not reached.  Synchronises. */
chfsi_status chfsi_poisson(chfsi_ctx* ctx, const double* f, double* phi, double tol, int max_iter,
                           int* iters, double* rel_residual);

typedef struct {
  int nnuclei;            /* Gaussian nuclear charges b = -sum Z_I g_I (normalised Gaussians) */
  const double* xyz;      /* host, 3 * nnuclei centres (bohr)                              */
  const double* Z;        /* host, nnuclei charges (N_e = sum Z)                            */
  const double* sigma;    /* host, nnuclei widths (bohr)                                    */
  int n_states;           /* states in the subspace (columns of X); 2 n_states >= N_e      */
  double kT;              /* Fermi-Dirac smearing (Ha)                                      */
  int degree;             /* Chebyshev degree of each ChFSI pass                            */
  int passes;             /* ChFSI passes per SCF step                                      */
  double tol;             /* stop when |rho_out - rho|_W < tol (quadrature-weighted L2)     */
  int max_iter;           /* SCF steps at most                                              */
  double beta;            /* Anderson mixing: step on the residual                          */
  int depth;              /* Anderson mixing: history length (1..16)                        */
  uint64_t seed;          /* start block (chfsi_fill_uniform stream 1) and Lanczos starts   */
  double poisson_tol;     /* relative residual of the Poisson CG                            */
  int lanczos_steps;      /* steps of the upper-bound estimate per SCF step                 */
} chfsi_scf_params;

/* The SCF loop: initial density = the nuclei widened to 1 bohr, scaled to N_e;
 * per step: phi (chfsi_poisson of rho + b), V_eff = phi + V_x(rho) with the
 * LDA exchange V_x = -(3 rho / pi)^{1/3} at the Gauss points
 * (chfsi_set_potential_qp_device), the upper bound (chfsi_bounds), a
 * Rayleigh-Ritz step and `passes` ChFSI passes on X (binary64, warm-started),
 * the Fermi level of all states (chfsi_fermi_level, n_oc = 0), the density
 * (chfsi_density), and n-stage Anderson mixing of rho weighted by the
 * quadrature weights.  X: device, M x n_states, binary64, caller-owned: filled
 * with the seeded start, returns the last eigenvectors.  Outputs (host; NULL
 * allowed except evals_host): rho_host[ncells q^3] the converged density,
 * evals_host / occ_host[n_states], mu_out, res_hist[max_iter] the residual of
 * every step, iters_out the steps run.  CHFSI_ERR_EIG when tol is not reached
 * in max_iter steps (the outputs then hold the last step).  Synchronises. */
chfsi_status chfsi_scf(chfsi_ctx* ctx, const chfsi_scf_params* prm, double* X, int64_t ldx,
                       double* rho_host, double* evals_host, double* occ_host, double* mu_out,
                       double* res_hist, int* iters_out);

/* -------------------------------------------------------------- k-points
 * Bloch states of a periodic crystal at wavevector k (Eq. evp of the periodic
 * problem, Sec. 2.1): the cell-periodic part u solves
 * (-1/2 lap - i k.grad + 1/2 |k|^2 + V) u = eps u, in FE form per cell
 * H_e(k) = 1/2 K_e - i k.G_e + 1/2 |k|^2 A_e + V_e (G^(d)_jl = int N_j d_d N_l,
 * A_e the consistent mass, the cell's Gauss rule), and H~(k) = M^{-1/2} H(k)
 * M^{-1/2} is complex Hermitian.  Applied matrix-free in binary64 (needs a
 * periodic box, 2 <= p <= 8, quad_points = p + 2, a built context or a device
 * potential, and no projectors: their Bloch phases are not modelled).
 * Complex blocks are binary64 (real, imaginary) column pairs: vector v at
 * unknown j is X[j ldx + 2 v] + i X[j ldx + 2 v + 1]; ldx counts doubles
 * (>= 2 n).  The real entry points above are unaffected. */

/* Set k (bohr^-1, three components) for the k-point entry points below. */
chfsi_status chfsi_set_kpoint(chfsi_ctx* ctx, const double* k);
/* Y = H~(k) X on n complex vectors (X, Y: device, must not overlap). */
chfsi_status chfsi_apply_kpoint(chfsi_ctx* ctx, const double* X, int64_t ldx, double* Y, int64_t ldy,
                                int n);
/* Upper bound of spec(H~(k)) by k-step Lanczos (as chfsi_bounds) on the real
 * 2M-dimensional form of H~(k), which has the same spectrum. */
chfsi_status chfsi_bounds_kpoint(chfsi_ctx* ctx, int lanczos_steps, uint64_t seed, double* b_out);
/* ChFSI at k (as chfsi_solve, binary64, fixed iteration count): CholGS + RR
 * on the start block, then `iters` x {filter, CholGS, RR}.  CholGS:
 * S = X^H X = L L^H (cuSOLVER zpotrf), L^{-1} (ztrtri), X <- X L^{-H}; RR:
 * H^ = X^H H~(k) X, zheevd (ascending), X <- X Q.  evals_host[n] receives
 * the Ritz values.  Synchronises. */
chfsi_status chfsi_solve_kpoint(chfsi_ctx* ctx, double* X, int64_t ldx, int n, int iters, int degree,
                                double b, double* evals_host);

/* Mixed precision at k: one application Y = H~(k) X on binary32 column pairs
 * (X, Y device, M x 2n floats, leading dimensions in floats, even, >= 2n),
 * the cell products in BF16x3: T~_e = H~_e + 1/2 |k|^2 M^{-1/2} A_e M^{-1/2}
 * on both columns of a pair and one shared block G~ = M^{-1/2} (k.G_e)
 * M^{-1/2} on the swapped pair (re, im) -> (im, -re), the assembly as for
 * the real operator.  Needs every cell to share the M^{-1/2} pattern (the
 * uniform periodic box; CHFSI_ERR_ARG otherwise) and the cell matrices
 * (CHFSI_ERR_STATE after a device-side potential). */
chfsi_status chfsi_apply_kpoint_mixed(chfsi_ctx* ctx, const float* X, int64_t ldx, float* Y, int64_t ldy,
                                      int n);

/* chfsi_solve_kpoint with a filter precision: CHFSI_FP64 (the binary64 solve)
 * or CHFSI_MIXED_BF16X3: each iteration filters a binary32 copy of the block
 * with the mixed application above (Eq. chebFilter), then CholGS and
 * Rayleigh-Ritz run in binary64 on X as in chfsi_solve_kpoint. */
chfsi_status chfsi_solve_kpoint_prec(chfsi_ctx* ctx, double* X, int64_t ldx, int n, int iters, int degree,
                                     double b, chfsi_precision filter_prec, double* evals_host);

/* ---------------------------------------------------------- domain decomposition
 * Partition of the mesh's cells over nranks ranks (the paper's primary level
 * of parallelism, Sec. 3.7: subdomains of the FE mesh on separate tasks; since
 * each basis function lives on the cells sharing its node, only unknowns on
 * subdomain boundaries are communicated).  Host-only (no device, no context):
 * every rank calls it for itself and all ranks agree on every list.
 * The ranks form a grid px x py x pz = nranks (the factorisation with the
 * smallest interface area, each factor at most the cells on its axis); rank
 * ix + px (iy + py iz) owns the cell block [ix n_x / px, (ix + 1) n_x / px) x ...
 * For rank `rank`:
 *  cells[ncells]        its cells (global index, cells x fastest), ascending;
 *  l2g[nlocal]          the global unknowns its cells touch, ascending: the
 *                       local numbering of its rows of X;
 *  owner[nlocal]        per local unknown the lowest rank whose cells touch it
 *                       (the rank that counts the row in sums over unknowns,
 *                       e.g. the overlap S = X^T X, Algorithm CholGS step 1);
 *  neighbors[nneighbors] the other ranks sharing unknowns with it, ascending;
 *  halo_ptr[nneighbors + 1], halo[nhalo]: for neighbor k, the local indices
 *                       halo[halo_ptr[k] .. halo_ptr[k+1]) of the shared
 *                       unknowns, in ascending global order (the same order on
 *                       both ranks, so exchanged rows line up).
 * A cell apply over the rank's cells gives partial sums on its local rows;
 * adding the partial sums that each neighbor sends for the shared rows gives
 * rows of H~ X (the halo sum).  Arrays are caller-owned host memory sized by
 * chfsi_partition_sizes.  CHFSI_ERR_ARG for an invalid mesh, rank outside
 * [0, nranks), or no factorisation fitting the cells. */
typedef struct {
  int64_t ncells, nlocal, nhalo;
  int nneighbors;
  int grid[3];
} chfsi_partition_info;

chfsi_status chfsi_partition_sizes(const chfsi_mesh_desc* desc, int nranks, int rank,
                                   chfsi_partition_info* out);
chfsi_status chfsi_partition_fill(const chfsi_mesh_desc* desc, int nranks, int rank, int32_t* cells,
                                  int32_t* l2g, int32_t* owner, int32_t* neighbors,
                                  int64_t* halo_ptr, int32_t* halo);

/* ---------------------------------------------------------------- batching
 * Many independent systems of the same FE degree (typically small and of
 * uneven size) filtered together on the tensor cores.  Per Chebyshev degree
 * step one launch of the cell kernel (a grid over, or a persistent loop over,
 * the (system, cell, column-tile) items of every system) and one launch of
 * the assembly kernel
 * covers every unknown of every system; the whole degree-m filter is
 * captured once into a CUDA graph and replayed while the buffers, widths,
 * degree and tile choice stay the same (the recurrence scalars live in device
 * memory and are refreshed by the graph).  Contexts must be built, share the
 * device, have no projectors and p <= 7. */
typedef struct chfsi_batch chfsi_batch;

chfsi_status chfsi_batch_create(int n, chfsi_ctx* const* ctxs, void* stream, chfsi_batch** out);
chfsi_status chfsi_batch_destroy(chfsi_batch* b);
const char*  chfsi_batch_last_error(const chfsi_batch* b);

/* Filter X[s] (device, binary32, M_s x ncol[s], leading dimension ldx[s]) of
 * every system in place with degree `degree` and bounds a[s] < b[s],
 * a0[s] < a[s] (scaled Eq. chebFilter), precision MIXED_BF16X3, MIXED_TF32X3 or
 * MIXED_TF32.  MIXED_BF16X3 runs one launch of the BF16x3 cell kernel per
 * degree step over the (system, cell, 128-column tile, row part) items (the
 * tile choice below applies to the TF32 kernels only); the first BF16x3 call
 * packs each member's three-term copy (3 x 2 bytes per cell-matrix element).
 * Synchronises the batch stream. */
chfsi_status chfsi_batch_filter(chfsi_batch* b, float* const* X, const int64_t* ldx,
                                const int* ncol, int degree, const double* a,
                                const double* bnd, const double* a0, chfsi_precision prec);

/* Autotuner of the batched cell kernel: times every candidate (column tile
 * width x pipeline depth, see chfsi_batch_candidates) on two degree steps of
 * this batch and keeps the fastest for later filter calls (TF32 precisions
 * only: CHFSI_ERR_ARG for MIXED_BF16X3, which has one kernel).  X is used as
 * scratch and overwritten.  choice (may be NULL) receives the winning index,
 * ms_out (may be NULL, one entry per candidate) the measured times. */
chfsi_status chfsi_batch_autotune(chfsi_batch* b, float* const* X, const int64_t* ldx,
                                  const int* ncol, chfsi_precision prec, int* choice,
                                  double* ms_out);

/* Candidate tile configurations: fills up to max (column tile, stages) pairs,
 * returns their number.  Stages -1 denotes the non-persistent multi-system
 * cell kernel (one CTA per (system, cell, 64-column tile) item, two CTAs per
 * SM), the default before autotuning; the others are the persistent kernel. */
int          chfsi_batch_candidates(const chfsi_batch* b, int* bn_out, int* stages_out, int max);

/* Select candidate k of chfsi_batch_candidates for later filter calls (as the
 * autotuner would).  CHFSI_ERR_ARG for an index out of range. */
chfsi_status chfsi_batch_set_candidate(chfsi_batch* b, int k);

/* ChFSI on every system: X[s] (device, binary64, M_s x n[s], in/out start
 * block), bnd[s] the upper bound of spec(H~_s); per iteration the batched
 * binary32 filter (filter_prec) followed, per system and concurrently, by
 * CholGS and Rayleigh-Ritz in orth_prec: CHFSI_FP64 (on the binary64 block)
 * or CHFSI_MIXED_TF32X3 / CHFSI_MIXED_BF16X3 (split-precision off-diagonal,
 * binary64 diagonal, on the binary32 working copy; the last Rayleigh-Ritz
 * applies H~ with binary64
 * products, as chfsi_solve does); X[s] receives the final block.
 * evals[s][n[s]] (host) receive the Ritz values. */
chfsi_status chfsi_batch_solve(chfsi_batch* b, double* const* X, const int64_t* ldx, const int* n,
                               int iters, int degree, const double* bnd,
                               chfsi_precision filter_prec, chfsi_precision orth_prec,
                               double* const* evals);

/* ----------------------------------------------------------------- serving
 * Continuous-batching request loop for SCF-like sequences of eigensolves.
 * The paper has no serving layer; this wraps the calls above.  A request is
 * one system (mesh, Gaussian wells) plus `resolves` follow-up potentials
 * (the same wells with new depths, e.g. a perturbed V_eff of the next SCF
 * step).  The server admits queued requests in FIFO order as soon as fewer
 * than max_active requests run and the request's device-memory estimate fits
 * in what is left of hbm_budget_bytes; every admitted request gets its own
 * host worker thread, CUDA stream and context, so the GPU work of admitted
 * requests overlaps.  A request keeps its block X (n columns, binary64 for
 * CHFSI_FP64, binary32 otherwise) and its upper bound b (one Lanczos run of
 * 20 steps on the first potential, raised by 2%) resident for all of its
 * solves: solve 0 starts from chfsi_fill_uniform(seed, stream 1) and runs
 * `iters` ChFSI iterations, every re-solve rebuilds the cell matrices and
 * runs `warm_iters` iterations from the previous X (warm start).  Each solve
 * uses chfsi_solve (tol, n_check as there), or chfsi_solve_polish when
 * polish_iters > 0 (mixed precisions: the polished block, rounded to
 * binary32, is the next solve's start), and then chfsi_residuals on the
 * lowest n_check pairs.  Requests share no device data, so a request's
 * results do not depend on what else runs.  A request whose estimate exceeds
 * the whole budget completes with CHFSI_ERR_OOM; one that only has to wait
 * for memory stays queued.  chfsi_server_destroy lets running requests finish,
 * fails the ones still queued (CHFSI_ERR_STATE) and joins every thread. */
#define CHFSI_MAX_SOLVES 16

typedef struct chfsi_server chfsi_server;

typedef struct {
  chfsi_mesh_desc mesh;
  int n;                  /* wanted + buffer states (columns of X)                    */
  int nwells;             /* Gaussian wells V(r) = -sum_k d_k exp(-|r-r_k|^2/(2 w_k^2)) */
  const double* xyz;      /* host, 3 * nwells (copied at submit)                       */
  const double* depth;    /* host, nwells: depths of solve 0 (copied)                  */
  const double* width;    /* host, nwells (copied)                                     */
  int resolves;           /* warm re-solves after solve 0, resolves + 1 <= CHFSI_MAX_SOLVES */
  const double* depth_seq;/* host, resolves * nwells: depths of re-solve k at k*nwells  */
  int degree;             /* Chebyshev degree m                                        */
  int iters;              /* ChFSI iterations of solve 0 (upper limit when tol > 0)     */
  int warm_iters;         /* iterations of each re-solve                               */
  double tol;             /* early stop on residual (chfsi_solve), 0 = fixed counts     */
  int n_check;            /* pairs checked by the early stop and reported residuals     */
  chfsi_precision prec;   /* filter / orthogonalisation precision                       */
  uint64_t seed;          /* start block and Lanczos seed                              */
  int polish_iters;       /* mixed precisions: > 0 runs every solve through           */
  int polish_degree;      /*   chfsi_solve_polish (degree 0 = the request's degree)      */
} chfsi_request;

typedef struct {
  int done;               /* 0 while queued or running                                 */
  chfsi_status status;    /* first error of the request, CHFSI_OK on success           */
  int nsolves;            /* solves completed                                          */
  double queue_ms;        /* submit -> admission (host clock)                          */
  double first_ms;        /* submit -> end of solve 0                                  */
  double total_ms;        /* submit -> end of the last solve                           */
  size_t est_bytes;       /* device-memory estimate used for admission                 */
  size_t used_bytes;      /* device bytes the request actually held (context + X)       */
  double solve_ms[CHFSI_MAX_SOLVES];     /* host wall time of each solve                */
  double max_residual[CHFSI_MAX_SOLVES]; /* max ||H~x - l x||/||x|| of the n_check pairs */
  double max_gresidual[CHFSI_MAX_SOLVES];/* max ||H Psi - l M Psi||, Psi^T M Psi = 1      */
  int iters[CHFSI_MAX_SOLVES];            /* ChFSI iterations each solve ran             */
  char error[160];        /* message of the first error                                */
} chfsi_result;

chfsi_status chfsi_server_create(size_t hbm_budget_bytes, int max_active, chfsi_server** out);
/* Copies the request (and its host arrays); *ticket identifies it. */
chfsi_status chfsi_server_submit(chfsi_server* sv, const chfsi_request* req, uint64_t* ticket);
/* Fills *out; with wait != 0 blocks until the request is done.  When done and
 * evals_host != NULL, copies the Ritz values of every solve, solve k at
 * evals_host[k * n], (resolves + 1) * n doubles. */
chfsi_status chfsi_server_poll(chfsi_server* sv, uint64_t ticket, int wait, chfsi_result* out,
                               double* evals_host);
/* Device-memory estimate the server admits a request by (bytes). */
size_t       chfsi_server_estimate(const chfsi_request* req);
chfsi_status chfsi_server_destroy(chfsi_server* sv);

#ifdef __cplusplus
}
#endif
#endif /* CHFSI_H */
