// C-ABI entry points of libchfsi (declared in include/chfsi.h): context and
// device-memory management, the filter / CholGS / Rayleigh-Ritz drivers and
// the ChFSI loop (step 7 of Algorithm scf in arXiv:1903.10959).
#include <algorithm>
#include <atomic>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cusolverDn.h>

#include "ctx.h"

using namespace chfsi;

namespace chfsi {
static std::atomic<int64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace chfsi



namespace {

cudaEvent_t kev_get(chfsi_ctx* ctx) {
  if (!ctx->kev_free.empty()) {
    cudaEvent_t e = ctx->kev_free.back();
    ctx->kev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
// Event pair around one kernel launch (kind 0: cell products, 1: assembly).
struct KTimer {
  chfsi_ctx* ctx;
  int kind;
  cudaEvent_t a = nullptr;
  KTimer(chfsi_ctx* c, int k) : ctx(c), kind(k) {
    if (ctx->ktiming) {
      a = kev_get(ctx);
      cudaEventRecord(a, ctx->stream);
    }
  }
  ~KTimer() {
    if (a) {
      cudaEvent_t b = kev_get(ctx);
      cudaEventRecord(b, ctx->stream);
      ctx->krec.push_back({kind, a, b});
    }
  }
};

chfsi_status fail(chfsi_ctx* c, chfsi_status st, const std::string& msg) {
  if (c) {
    c->err = msg;
    if (st == CHFSI_ERR_CUDA) c->latched = st;
  }
  return st;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(ctx, CHFSI_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define CS(call)                                                                          \
  do {                                                                                    \
    cusolverStatus_t s_ = (call);                                                         \
    if (s_ != CUSOLVER_STATUS_SUCCESS)                                                    \
      return fail(ctx, CHFSI_ERR_CUDA, std::string(#call) + ": cusolver status " +         \
                                           std::to_string((int)s_));                      \
  } while (0)
#define CHECK_CTX()                                                                       \
  do {                                                                                    \
    if (!ctx) return CHFSI_ERR_ARG;                                                       \
    if (ctx->latched != CHFSI_OK) return ctx->latched;                                    \
  } while (0)

cudaError_t dalloc(chfsi_ctx* ctx, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
  if (e == cudaSuccess) ctx->dev_bytes += (int64_t)std::max<size_t>(bytes, 16);
  return e;
}
void dfree(chfsi_ctx* ctx, void* p, size_t bytes) {
  if (p) {
    cudaFree(p);
    ctx->dev_bytes -= (int64_t)std::max<size_t>(bytes, 16);
  }
}
template <class T>
cudaError_t upload(chfsi_ctx* ctx, T** dst, const std::vector<T>& src) {
  if (*dst) return cudaErrorInvalidValue;
  cudaError_t e = dalloc(ctx, (void**)dst, src.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  if (src.empty()) return cudaSuccess;
  return cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream);
}
template <class T>
void release(chfsi_ctx* ctx, T*& p, size_t bytes) {
  dfree(ctx, (void*)p, bytes);
  p = nullptr;
}

chfsi_status grow(chfsi_ctx* ctx, DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes) return CHFSI_OK;
  if (b.ptr) {
    cudaStreamSynchronize(ctx->stream);
    dfree(ctx, b.ptr, b.bytes);
    b.ptr = nullptr;
    b.bytes = 0;
  }
  cudaError_t e = dalloc(ctx, &b.ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, CHFSI_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  }
  b.bytes = bytes;
  return CHFSI_OK;
}

bool is_mixed(chfsi_precision p) {
  return p == CHFSI_MIXED_TF32X3 || p == CHFSI_MIXED_TF32 || p == CHFSI_MIXED_BF16X3 ||
         p == CHFSI_MIXED_F16X2;
}
// Gram and tall GEMMs: 3xTF32 for the binary32-accurate precisions, 1xTF32 for TF32.
int split3_of(chfsi_precision p) { return p != CHFSI_MIXED_TF32; }
// Columns per block of the binary64 staging copies (residuals, binary64 RR apply).
constexpr int kStage64 = 512;
// Whether the binary64 path uses the matrix-free cell apply when the context
// leaves the choice open (chfsi_set_fp64_operator(-1)).
constexpr bool kMatrixFreeDefault = true;
// Free the per-call scratch that grows with the column block (filter, cell
// blocks, projector and binary64 staging buffers); later calls regrow it.
void release_scratch(chfsi_ctx* ctx) {
  cudaStreamSynchronize(ctx->stream);
  for (DevBuf* b : {&ctx->T1, &ctx->Wb, &ctx->NLb, &ctx->Zb, &ctx->Rb, &ctx->rot, &ctx->cmaxb, &ctx->pjb, &ctx->tinv}) {
    dfree(ctx, b->ptr, b->bytes);
    b->ptr = nullptr;
    b->bytes = 0;
  }
}

bool valid_prec(chfsi_precision p) { return p == CHFSI_FP64 || is_mixed(p); }
size_t esize(chfsi_precision p) { return p == CHFSI_FP64 ? 8 : 4; }

std::vector<double> minv_sqrt(const HostMesh& m) {
  std::vector<double> s(m.mass.size());
  for (size_t j = 0; j < s.size(); ++j) s[j] = 1.0 / std::sqrt(m.mass[j]);
  return s;
}

// Binary64 cell operator of this context: the sum-factorised (matrix-free)
// apply when selected, or by default when it exists for the degree and rule.
bool use_matrix_free(const chfsi_ctx* ctx) {
  if (!mf_supported(ctx->mesh.p, ctx->mesh.q)) return false;
  return ctx->fp64_op == 1 || (ctx->fp64_op < 0 && kMatrixFreeDefault);
}

void free_device_data(chfsi_ctx* ctx) {
  const HostMesh& m = ctx->mesh;
  release(ctx, ctx->d_Ht, (size_t)m.ncells * m.ne * m.ne * 8);
  release(ctx, ctx->d_wv, ctx->wv.size() * 8);
  release(ctx, ctx->d_fac, ctx->fac.size() * 8);
  ctx->dev_bytes -= (int64_t)(ctx->tc.bytes + ctx->tc.bf_bytes + ctx->tc.f16_bytes + ctx->tc.nl_bytes +
                              ctx->tc.pj_bytes);   // packed copies
  tc_free(ctx->tc);
  ctx->kpack_valid = false;   // the mixed Bloch packs hold the old cell matrices
  release(ctx, ctx->d_site_ptr, ctx->hproj.site_ptr.size() * 8);
  release(ctx, ctx->d_site_dof, ctx->hproj.site_dof.size() * 4);
  release(ctx, ctx->d_site_c, ctx->hproj.site_c.size() * 8);
  release(ctx, ctx->d_dof_ptr, ctx->hproj.dof_ptr.size() * 8);
  release(ctx, ctx->d_dof_site, ctx->hproj.dof_site.size() * 4);
  release(ctx, ctx->d_dof_c, ctx->hproj.dof_c.size() * 8);
  release(ctx, ctx->d_site_c32, ctx->hproj.site_c.size() * 4);
  release(ctx, ctx->d_dof_c32, ctx->hproj.dof_c.size() * 4);
  ctx->built = false;
  ++ctx->build_gen;   // device pointers captured elsewhere (batch graphs) are now stale
}

// The tensor-core copies of the cell data a mixed precision needs (packed on
// first use, on the context's stream): the BF16x3 / FP16x2 / TF32 cell
// matrices and, for the BF16x3 ring kernels, the projector chunks and the
// projection blocks.
chfsi_status ensure_tc_data(chfsi_ctx* ctx, chfsi_precision prec) {
  const HostMesh& m = ctx->mesh;
  const bool nl = ctx->hproj.nsite > 0;
  if (!ctx->d_Ht)
    return fail(ctx, CHFSI_ERR_STATE, "no cell matrices: the potential was set on the device "
                                      "(binary64 only until chfsi_build)");
  const bool bf16 = prec == CHFSI_MIXED_BF16X3;
  const bool f16 = prec == CHFSI_MIXED_F16X2;
  if (f16 && !ctx->tc.f16) {
    cudaError_t pe = tc_pack_f16_from_device(ctx->tc, ctx->d_Ht, ctx->stream, &ctx->dev_bytes);
    if (pe != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, pe == cudaErrorMemoryAllocation ? CHFSI_ERR_OOM : CHFSI_ERR_CUDA,
                  std::string("FP16x2 cell data: ") + cudaGetErrorString(pe));
    }
  }
  if (bf16 && !ctx->tc.bf) {
    cudaError_t pe = tc_pack_bf16_from_device(ctx->tc, ctx->d_Ht, ctx->stream, &ctx->dev_bytes);
    if (pe != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, pe == cudaErrorMemoryAllocation ? CHFSI_ERR_OOM : CHFSI_ERR_CUDA,
                  std::string("BF16x3 cell data: ") + cudaGetErrorString(pe));
    }
  }
  if (!bf16 && !f16 && !ctx->tc.hi) {
    cudaError_t pe = tc_pack_from_device(ctx->tc, ctx->d_Ht, ctx->stream, &ctx->dev_bytes);
    if (pe != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, pe == cudaErrorMemoryAllocation ? CHFSI_ERR_OOM : CHFSI_ERR_CUDA,
                  std::string("tensor-core cell data: ") + cudaGetErrorString(pe));
    }
  }
  // BF16x3 ring kernels take the projector terms on the tensor cores: the
  // projection Z = C~^T Y as per-cell blocks over the owned rows (partial sums
  // reduced per site in a fixed order) and the expansion C~ h Z as extra
  // K-chunks of the cell products; the assembly then has no projector term
  const bool nl_in_cells = nl && bf16 && tc_cell_bf16_nl_ok(ctx->cell_gather);
  if (nl_in_cells && !ctx->tc.nl) {
    NlCells nc;
    build_nl_cells(m, ctx->hproj, nc);
    cudaError_t pe = tc_pack_nl(ctx->tc, nc.chunk_off.data(), m.ncells, nc.zrow.data(), nc.nz_pos.data(),
                                nc.nz_val.data(), (int64_t)nc.nz_val.size(), ctx->stream, &ctx->dev_bytes);
    if (pe == cudaSuccess)
      pe = tc_pack_proj(ctx->tc, m.ncells, ctx->hproj.nsite, nc.np.data(), nc.poff.data(), nc.prow.data(),
                        nc.red_ptr.data(), nc.red_row.data(), nc.pz_pos.data(), nc.pz_val.data(),
                        (int64_t)nc.pz_val.size(), ctx->stream, &ctx->dev_bytes);
    if (pe == cudaErrorNotSupported) {
      cudaGetLastError();   // too many sites on one cell's rows: the projection stays by site
    } else if (pe != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, pe == cudaErrorMemoryAllocation ? CHFSI_ERR_OOM : CHFSI_ERR_CUDA,
                  std::string("projector chunks: ") + cudaGetErrorString(pe));
    }
  }
  return CHFSI_OK;
}

// One recurrence step over the ncol columns of a block:
// Yout = alpha (H~ Yin - shift Yin) + beta Yprev, colour by colour.
chfsi_status apply_step(chfsi_ctx* ctx, chfsi_precision prec, const void* Yin, int64_t ld_in,
                        void* Yout, int64_t ld_out, const void* Yprev, int64_t ld_prev, int ncol,
                        double alpha, double beta, double shift, const uint32_t* cmax_in = nullptr,
                        uint32_t* cmax_out = nullptr) {
  const HostMesh& m = ctx->mesh;
  const int B = std::max(ncol, 1);
  const size_t es = esize(prec);
  chfsi_status st;
  if (prec == CHFSI_FP64 && (st = grow(ctx, ctx->Wb, (size_t)m.ndofs * B * es)) != CHFSI_OK) return st;
  const bool nl = ctx->hproj.nsite > 0;
  if (nl) {
    if (prec == CHFSI_FP64 && (st = grow(ctx, ctx->NLb, (size_t)m.ndofs * B * es)) != CHFSI_OK) return st;
    if ((st = grow(ctx, ctx->Zb, (size_t)4 * ctx->hproj.nsite * B * es)) != CHFSI_OK) return st;
  }
  const int ncolour = (int)m.colour_offsets.size() - 1;
  if (prec == CHFSI_FP64) {
    if (nl) {
      CK(launch_nl_project_fp64(ctx->d_site_ptr, ctx->d_site_dof, ctx->d_site_c, ctx->hproj.nsite,
                                (const double*)Yin, ld_in, ncol, (double*)ctx->Zb.ptr, ctx->stream));
      CK(launch_nl_expand_fp64(ctx->d_dof_ptr, ctx->d_dof_site, ctx->d_dof_c, m.ndofs,
                               (const double*)ctx->Zb.ptr, ncol, (double*)ctx->NLb.ptr, B, ctx->stream));
    }
    const bool mf = use_matrix_free(ctx);
    if (!mf && !ctx->d_Ht) return fail(ctx, CHFSI_ERR_STATE, "no cell matrices for the binary64 operator");
    for (int c = 0; c < ncolour; ++c) {
      KTimer kt(ctx, 0);
      if (mf) {
        MfLaunch L{};
        L.fac = ctx->d_fac;
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
        L.ld_w = B;
        CK(launch_mf_cell_fp64(L, (const double*)Yin, (double*)Yout, (const double*)Yprev,
                               (double*)ctx->Wb.ptr, nl ? (const double*)ctx->NLb.ptr : nullptr,
                               FilterStep{alpha, beta, shift}, ctx->stream));
        continue;
      }
      CellLaunch L{};
      L.Ht = ctx->d_Ht;
      L.dofmap = ctx->d_dofmap;
      L.modes = ctx->d_modes;
      L.cells = ctx->d_cells + m.colour_offsets[c];
      L.ncells_colour = m.colour_offsets[c + 1] - m.colour_offsets[c];
      L.ne = m.ne;
      L.ncol = ncol;
      L.ld_in = ld_in;
      L.ld_out = ld_out;
      L.ld_prev = ld_prev;
      CK(launch_cell_fp64(L, (const double*)Yin, (double*)Yout, (const double*)Yprev,
                          (double*)ctx->Wb.ptr, nl ? (const double*)ctx->NLb.ptr : nullptr, B,
                          FilterStep{alpha, beta, shift}, ctx->stream));
    }
    return CHFSI_OK;
  }
  // mixed precisions: binary32 storage, tcgen05 TF32 (or BF16x3) cell products
  if ((st = ensure_tc_data(ctx, prec)) != CHFSI_OK) return st;
  const bool bf16 = prec == CHFSI_MIXED_BF16X3;
  const bool f16 = prec == CHFSI_MIXED_F16X2;
  const bool nl_in_cells = nl && bf16 && tc_cell_bf16_nl_ok(ctx->cell_gather);
  if (nl) {   // projection Z = C~^T Y
    KTimer kt(ctx, 2);
    if (nl_in_cells && ctx->tc.pj) {
      if ((st = grow(ctx, ctx->pjb, (size_t)ctx->tc.pj_rows * ncol * sizeof(float))) != CHFSI_OK) return st;
      CK(tc_nl_project_cells(ctx->tc, ctx->d_dofmap, m.ncells, ctx->hproj.nsite, (const float*)Yin, ld_in,
                             ncol, (float*)ctx->pjb.ptr, (float*)ctx->Zb.ptr, ctx->stream));
    } else {
      CK(tc_nl_project(ctx->d_site_ptr, ctx->d_site_dof, ctx->d_site_c32, ctx->hproj.nsite,
                       (const float*)Yin, ld_in, ncol, (float*)ctx->Zb.ptr, ctx->stream));
    }
  }
  // owner-computes: dense cell blocks R_e (one launch over all cells), then the
  // fixed-order assembly fused with the Chebyshev update
  if ((st = grow(ctx, ctx->Rb, (size_t)m.ncells * m.ne * ncol * sizeof(float))) != CHFSI_OK) return st;
  TcApplyArgs ra{};
  ra.dofmap = ctx->d_dofmap;
  ra.ncells = m.ncells;
  ra.ncol = ncol;
  ra.Yin = (const float*)Yin;
  ra.ld_in = ld_in;
  ra.R = (float*)ctx->Rb.ptr;
  ra.split3 = prec == CHFSI_MIXED_TF32X3;
  ra.tile = ctx->cell_tile;
  ra.gather = ctx->cell_gather;
  if (nl_in_cells) {
    ra.Z = (const float*)ctx->Zb.ptr;
    ra.ldz = ncol;
  }
  if (f16 && !cmax_in) {   // column maxima of the input block (the scales of its fp16 split)
    if ((st = grow(ctx, ctx->cmaxb, (size_t)3 * ncol * sizeof(uint32_t))) != CHFSI_OK) return st;
    uint32_t* cm = (uint32_t*)ctx->cmaxb.ptr + 2 * (size_t)ncol;
    CK(tc_colmax_launch((const float*)Yin, ld_in, m.ndofs, ncol, cm, ctx->stream));
    cmax_in = cm;
  }
  {
    KTimer kt(ctx, 0);
    if (f16) CK(tc_cell_f16_launch(ctx->tc, ra, cmax_in, ctx->stream));
    else if (bf16) CK(tc_cell_bf16_launch(ctx->tc, ra, ctx->stream));
    else CK(tc_cell_r_launch(ctx->tc, ra, ctx->stream));
  }
  KTimer kt(ctx, 1);
  AssembleParams ap{};
  ap.node_ptr = ctx->d_node_ptr;
  ap.node_ent = ctx->d_node_ent;
  ap.M = m.ndofs;
  ap.ncol = ncol;
  ap.R = (const float*)ctx->Rb.ptr;
  ap.Yin = (const float*)Yin;
  ap.ld_in = ld_in;
  ap.Yout = (float*)Yout;
  ap.ld_out = ld_out;
  ap.Yprev = beta != 0.0 ? (const float*)Yprev : nullptr;
  ap.ld_prev = ld_prev;
  if (nl && !nl_in_cells) {
    ap.dof_ptr = ctx->d_dof_ptr;
    ap.dof_site = ctx->d_dof_site;
    ap.dof_c = ctx->d_dof_c32;
    ap.Z = (const float*)ctx->Zb.ptr;
  }
  ap.alpha = (float)alpha;
  ap.beta = (float)beta;
  ap.shift = (float)shift;
  if (cmax_out) CK(tc_assemble_cmax_launch(ap, cmax_out, ctx->stream));
  else CK(tc_assemble_launch(ap, ctx->stream));
  return CHFSI_OK;
}

// Y = H~ X in column blocks (Y separate from X).
chfsi_status apply_blocks(chfsi_ctx* ctx, chfsi_precision prec, const void* X, int64_t ldx, void* Y,
                          int64_t ldy, int ncol) {
  const int B = std::max(1, std::min(ctx->filter_block, ncol));
  const size_t es = esize(prec);
  for (int b0 = 0; b0 < ncol; b0 += B) {
    const int nb = std::min(B, ncol - b0);
    chfsi_status st = apply_step(ctx, prec, (const char*)X + b0 * es, ldx, (char*)Y + b0 * es, ldy,
                                 nullptr, 0, nb, 1.0, 0.0, 0.0);
    if (st != CHFSI_OK) return st;
  }
  return CHFSI_OK;
}

chfsi_status check_x(chfsi_ctx* ctx, const void* X, int64_t ldx, int ncol, chfsi_precision prec) {
  if (!valid_prec(prec)) return fail(ctx, CHFSI_ERR_ARG, "unknown precision");
  if (!ctx->built) return fail(ctx, CHFSI_ERR_STATE, "chfsi_build has not been called");
  if (ncol < 0 || (ncol > 0 && (!X || ldx < ncol))) return fail(ctx, CHFSI_ERR_ARG, "bad X / ldx / ncol");
  return CHFSI_OK;
}

// Device-side bounded waits report through a status word; map it to an error.
chfsi_status check_device_status(chfsi_ctx* ctx, chfsi_precision prec) {
  if (!is_mixed(prec)) return CHFSI_OK;
  int v = tc_read_status(ctx->stream);
  if (v) return fail(ctx, CHFSI_ERR_TIMEOUT, "device wait timed out (site " + std::to_string(v) + ")");
  return CHFSI_OK;
}

void tic(chfsi_ctx* ctx) { cudaEventRecord(ctx->ev[0], ctx->stream); }
void toc(chfsi_ctx* ctx, int slot) {
  cudaEventRecord(ctx->ev[1], ctx->stream);
  cudaEventSynchronize(ctx->ev[1]);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
  ctx->times[slot] += ms;
}

// The filter of the columns [0, ncol) of X in blocks of the filter block size
// (every step on ctx->stream, scratch in ctx->T1 / Rb / Zb).
chfsi_status filter_range(chfsi_ctx* ctx, void* X, int64_t ldx, int ncol, int degree, double a,
                          double b, double a0, chfsi_precision prec) {
  const HostMesh& m = ctx->mesh;
  const int B = std::max(1, std::min(ctx->filter_block, ncol));
  const size_t es = esize(prec);
  chfsi_status st;
  if ((st = grow(ctx, ctx->T1, (size_t)m.ndofs * B * es)) != CHFSI_OK) return st;
  const double e = (b - a) / 2.0, c = (b + a) / 2.0;
  const double s1 = e / (a0 - c);
  for (int b0 = 0; b0 < ncol; b0 += B) {
    const int nb = std::min(B, ncol - b0);
    char* Xb = (char*)X + b0 * es;
    // Y0 = Xb, Y1 -> T1, then Y_{k+1} overwrites Y_{k-1}
    void* bufs[2] = {Xb, ctx->T1.ptr};
    int64_t lds[2] = {ldx, (int64_t)nb};
    int cur = 0;  // buffer holding Y_k
    double sig = s1;
    // FP16x2: each step's assembly leaves the column maxima of its output, the
    // next step's input (two alternating arrays; the first step measures X)
    uint32_t* cm[2] = {nullptr, nullptr};
    if (prec == CHFSI_MIXED_F16X2) {
      if ((st = grow(ctx, ctx->cmaxb, (size_t)3 * nb * sizeof(uint32_t))) != CHFSI_OK) return st;
      cm[0] = (uint32_t*)ctx->cmaxb.ptr;
      cm[1] = cm[0] + nb;
    }
    for (int k = 1; k <= degree; ++k) {
      double alpha, beta;
      if (k == 1) {
        alpha = s1 / e;
        beta = 0.0;
      } else {
        double sn = 1.0 / (2.0 / s1 - sig);
        alpha = 2.0 * sn / e;
        beta = -sig * sn;
        sig = sn;
      }
      const int nxt = 1 - cur;  // holds Y_{k-2} (or is free at k = 1)
      st = apply_step(ctx, prec, bufs[cur], lds[cur], bufs[nxt], lds[nxt], bufs[nxt], lds[nxt], nb,
                      alpha, beta, c, k == 1 ? nullptr : cm[cur], k == degree ? nullptr : cm[nxt]);
      if (st != CHFSI_OK) return st;
      cur = nxt;
    }
    if (cur == 1)
      CK(cudaMemcpy2DAsync(Xb, ldx * es, ctx->T1.ptr, nb * es, nb * es, m.ndofs,
                           cudaMemcpyDeviceToDevice, ctx->stream));
  }
  return CHFSI_OK;
}

// Lane l of a multi-lane filter: its stream and scratch take the place of the
// context's for the duration of the scope.
struct LaneScope {
  chfsi_ctx* ctx;
  int l;
  cudaStream_t saved;
  LaneScope(chfsi_ctx* c, int lane) : ctx(c), l(lane), saved(c->stream) {
    if (l == 0) return;
    ctx->stream = ctx->lane_stream[l];
    std::swap(ctx->T1, ctx->laneT1[l]);
    std::swap(ctx->Rb, ctx->laneR[l]);
    std::swap(ctx->Zb, ctx->laneZ[l]);
    std::swap(ctx->cmaxb, ctx->laneC[l]);
    std::swap(ctx->pjb, ctx->laneP[l]);
  }
  ~LaneScope() {
    if (l == 0) return;
    std::swap(ctx->T1, ctx->laneT1[l]);
    std::swap(ctx->Rb, ctx->laneR[l]);
    std::swap(ctx->Zb, ctx->laneZ[l]);
    std::swap(ctx->cmaxb, ctx->laneC[l]);
    std::swap(ctx->pjb, ctx->laneP[l]);
    ctx->stream = saved;
  }
};

// Chebyshev filter (Eq. chebFilter).  The columns are independent, so with
// L > 1 filter lanes (mixed precisions) they are cut into L groups of whole
// 128-column tiles, each filtered on its own stream with its own scratch: the
// memory-bound assembly of one lane then runs beside the tensor-core cell
// products of another.  Every column gets the same arithmetic as with one lane.
chfsi_status filter_impl(chfsi_ctx* ctx, void* X, int64_t ldx, int ncol, int degree, double a,
                         double b, double a0, chfsi_precision prec) {
  const int tiles = (ncol + 127) / 128;
  const int L = is_mixed(prec) ? std::min(ctx->filter_lanes, tiles) : 1;
  if (L <= 1) return filter_range(ctx, X, ldx, ncol, degree, a, b, a0, prec);
  // the shared cell data is packed before the lanes fork, so every lane's
  // stream is ordered after it
  chfsi_status st0 = ensure_tc_data(ctx, prec);
  if (st0 != CHFSI_OK) return st0;
  for (int l = 0; l < L; ++l) {
    if (l > 0 && !ctx->lane_stream[l])
      CK(cudaStreamCreateWithFlags(&ctx->lane_stream[l], cudaStreamNonBlocking));
    if (!ctx->lane_ev[l]) CK(cudaEventCreateWithFlags(&ctx->lane_ev[l], cudaEventDisableTiming));
  }
  // the lanes start after the work queued so far on the context's stream
  CK(cudaEventRecord(ctx->lane_ev[0], ctx->stream));
  for (int l = 1; l < L; ++l) CK(cudaStreamWaitEvent(ctx->lane_stream[l], ctx->lane_ev[0], 0));
  const size_t es = esize(prec);
  chfsi_status st = CHFSI_OK;
  int t0 = 0;
  for (int l = 0; l < L && st == CHFSI_OK; ++l) {
    const int nt = tiles / L + (l < tiles % L ? 1 : 0);
    const int c0 = t0 * 128, c1 = std::min(ncol, (t0 + nt) * 128);
    t0 += nt;
    LaneScope scope(ctx, l);
    st = filter_range(ctx, (char*)X + (size_t)c0 * es, ldx, c1 - c0, degree, a, b, a0, prec);
  }
  // the context's stream continues after every lane
  for (int l = 1; l < L; ++l) {
    CK(cudaEventRecord(ctx->lane_ev[l], ctx->lane_stream[l]));
    CK(cudaStreamWaitEvent(ctx->stream, ctx->lane_ev[l], 0));
  }
  return st;
}

// S(n x n, column-major, lower part) = A^T B for the precision's storage type.
chfsi_status gram_impl(chfsi_ctx* ctx, chfsi_precision prec, const void* A, int64_t lda,
                       const void* Bm, int64_t ldb, int n1, int n2, double* C, int64_t ldc,
                       int lower) {
  const HostMesh& m = ctx->mesh;
  chfsi_status st;
  if (prec == CHFSI_FP64) {
    size_t want = (size_t)8 * 8 * n1 * n2;
    if ((st = grow(ctx, ctx->part, want)) != CHFSI_OK) return st;
    CK(launch_gram_fp64((const double*)A, lda, (const double*)Bm, ldb, m.ndofs, n1, n2, C, ldc,
                        lower, (double*)ctx->part.ptr, ctx->part.bytes, ctx->stream));
    return CHFSI_OK;
  }
  size_t want = tc_gram_partial_bytes(m.ndofs, n1, n2);
  if ((st = grow(ctx, ctx->part, want)) != CHFSI_OK) return st;
  CK(tc_gram_mixed((const float*)A, lda, (const float*)Bm, ldb, m.ndofs, n1, n2, C, ldc, lower,
                   ctx->diag_block, split3_of(prec), ctx->part.ptr, ctx->part.bytes,
                   ctx->stream));
  return CHFSI_OK;
}

// X <- X U (U n x n column-major; trans / upper flags as launch_tallgemm_fp64).
chfsi_status rotate_impl(chfsi_ctx* ctx, chfsi_precision prec, void* X, int64_t ldx, int n,
                         const double* U, int upper, int trans) {
  const HostMesh& m = ctx->mesh;
  const size_t es = esize(prec);
  chfsi_status st;
  if ((st = grow(ctx, ctx->rot, (size_t)m.ndofs * n * es)) != CHFSI_OK) return st;
  if (prec == CHFSI_FP64) {
    CK(launch_tallgemm_fp64((const double*)X, ldx, U, n, m.ndofs, n, n, (double*)ctx->rot.ptr, n,
                            upper, trans, ctx->stream));
  } else {
    if ((st = grow(ctx, ctx->work, tc_tallgemm_work_bytes(n, n))) != CHFSI_OK) return st;
    CK(tc_tallgemm_mixed((const float*)X, ldx, U, n, m.ndofs, n, n, (float*)ctx->rot.ptr, n, upper,
                         trans, ctx->diag_block, split3_of(prec), ctx->work.ptr,
                         ctx->stream, ctx->tall_kernel));
  }
  CK(cudaMemcpy2DAsync(X, ldx * es, ctx->rot.ptr, n * es, n * es, m.ndofs, cudaMemcpyDeviceToDevice,
                       ctx->stream));
  return CHFSI_OK;
}

chfsi_status ensure_solver(chfsi_ctx* ctx) {
  if (!ctx->sol) {
    CS(cusolverDnCreate(&ctx->sol));
    CS(cusolverDnSetStream(ctx->sol, ctx->stream));
  }
  return CHFSI_OK;
}

chfsi_status cholgs_impl(chfsi_ctx* ctx, void* X, int64_t ldx, int n, chfsi_precision prec) {
  chfsi_status st;
  if (n == 0) return CHFSI_OK;
  if ((st = ensure_solver(ctx)) != CHFSI_OK) return st;
  if ((st = grow(ctx, ctx->Ssq, (size_t)n * n * 8 + 64)) != CHFSI_OK) return st;
  double* S = (double*)ctx->Ssq.ptr;
  int* dinfo = (int*)((char*)ctx->Ssq.ptr + (size_t)n * n * 8);
  // 1. S = X^T X (lower triangle)
  if ((st = gram_impl(ctx, prec, X, ldx, X, ldx, n, n, S, n, 1)) != CHFSI_OK) return st;
  // 2. S = L L^T
  int lw = 0;
  CS(cusolverDnDpotrf_bufferSize(ctx->sol, CUBLAS_FILL_MODE_LOWER, n, S, n, &lw));
  size_t dws = 0, hws = 0;
  CS(cusolverDnXtrtri_bufferSize(ctx->sol, CUBLAS_FILL_MODE_LOWER, CUBLAS_DIAG_NON_UNIT, n,
                                 CUDA_R_64F, S, n, &dws, &hws));
  size_t need = std::max<size_t>((size_t)lw * 8, dws) + 256;
  if ((st = grow(ctx, ctx->work, need)) != CHFSI_OK) return st;
  CS(cusolverDnDpotrf(ctx->sol, CUBLAS_FILL_MODE_LOWER, n, S, n, (double*)ctx->work.ptr, lw, dinfo));
  int info = 0;
  CK(cudaMemcpyAsync(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (info != 0)
    return fail(ctx, CHFSI_ERR_NOT_SPD, "CholGS: potrf info = " + std::to_string(info));
  // 3. L^{-1} (lower triangle; the strict upper triangle zero): the
  // warp-per-column forward substitution of kernels_fp64.cu (L_ii > 0 after
  // potrf), cuSOLVER's trtri in place beyond its shared-memory limit
  double* Linv = S;
  if (trinv_lower_supported(n)) {
    if ((st = grow(ctx, ctx->tinv, (size_t)n * n * 8)) != CHFSI_OK) return st;
    Linv = (double*)ctx->tinv.ptr;
    CK(cudaMemsetAsync(Linv, 0, (size_t)n * n * 8, ctx->stream));
    CK(launch_trinv_lower_fp64(S, n, n, Linv, n, ctx->stream));
  } else {
    std::vector<char> hwork(hws + 16);
    CS(cusolverDnXtrtri(ctx->sol, CUBLAS_FILL_MODE_LOWER, CUBLAS_DIAG_NON_UNIT, n, CUDA_R_64F, S, n,
                        ctx->work.ptr, dws, hwork.data(), hws, dinfo));
    CK(cudaMemcpyAsync(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (info != 0) return fail(ctx, CHFSI_ERR_NOT_SPD, "CholGS: trtri info = " + std::to_string(info));
  }
  // 4. X <- X L^{-T}: U(k, j) = Linv(j, k), nonzero for k <= j
  return rotate_impl(ctx, prec, X, ldx, n, Linv, 1, 1);
}

// Rayleigh-Ritz.  fp64_apply: for the mixed precisions, evaluate H~ X with the
// binary64 cell products (then round to binary32) so that H^ carries no
// binary32-accumulation bias; used for the last RR of a mixed solve.
// Step 1 of Rayleigh-Ritz: H^ = X^T (H~ X) (lower triangle, binary64, column
// major n x n) into ctx->Ssq, one column block at a time.  fp64_apply: H~ X
// with binary64 cell products for a binary32 block.
chfsi_status projected_impl(chfsi_ctx* ctx, const void* X, int64_t ldx, int n, chfsi_precision prec,
                            bool fp64_apply) {
  const HostMesh& m = ctx->mesh;
  chfsi_status st;
  if ((st = grow(ctx, ctx->Ssq, (size_t)n * n * 8 + 64)) != CHFSI_OK) return st;
  if ((st = grow(ctx, ctx->lam, (size_t)n * 8 + 64)) != CHFSI_OK) return st;
  double* Hh = (double*)ctx->Ssq.ptr;
  const size_t es = esize(prec);
  const bool via64 = fp64_apply && is_mixed(prec);
  // binary64 staging (X and H~X copies) is capped at kStage64 columns
  const int B = std::max(1, std::min({ctx->filter_block, n, via64 ? kStage64 : n}));
  if ((st = grow(ctx, ctx->T1, (size_t)m.ndofs * B * es)) != CHFSI_OK) return st;
  if (via64 && (st = grow(ctx, ctx->rot, (size_t)m.ndofs * B * 8 * 2)) != CHFSI_OK) return st;
  // 1. H^ = X^T (H~ X), lower triangle, one column block at a time
  for (int j0 = 0; j0 < n; j0 += B) {
    const int nb = std::min(B, n - j0);
    if (via64) {
      double* X64 = (double*)ctx->rot.ptr;
      double* Y64 = X64 + (size_t)m.ndofs * B;
      CK(launch_copy_cols((const char*)X + j0 * es, ldx, X64, nb, m.ndofs, nb, 0, 1, ctx->stream));
      if ((st = apply_step(ctx, CHFSI_FP64, X64, nb, Y64, nb, nullptr, 0, nb, 1.0, 0.0, 0.0)) != CHFSI_OK)
        return st;
      CK(launch_copy_cols(Y64, nb, ctx->T1.ptr, nb, m.ndofs, nb, 1, 0, ctx->stream));
    } else if ((st = apply_step(ctx, prec, (const char*)X + j0 * es, ldx, ctx->T1.ptr, nb, nullptr, 0,
                                nb, 1.0, 0.0, 0.0)) != CHFSI_OK) {
      return st;
    }
    if ((st = gram_impl(ctx, prec, (const char*)X + j0 * es, ldx, ctx->T1.ptr, nb, n - j0, nb,
                        Hh + j0 + (int64_t)j0 * n, n, 1)) != CHFSI_OK)
      return st;
  }
  return CHFSI_OK;
}

chfsi_status rr_impl(chfsi_ctx* ctx, void* X, int64_t ldx, int n, chfsi_precision prec,
                     double* evals_host, bool fp64_apply = false) {
  chfsi_status st;
  if (n == 0) return CHFSI_OK;
  if ((st = ensure_solver(ctx)) != CHFSI_OK) return st;
  // 1. H^ = X^T (H~ X)
  if ((st = projected_impl(ctx, X, ldx, n, prec, fp64_apply)) != CHFSI_OK) return st;
  double* Hh = (double*)ctx->Ssq.ptr;
  int* dinfo = (int*)((char*)ctx->Ssq.ptr + (size_t)n * n * 8);
  // 2. H^ Q = Q D (binary64 syevd, ascending)
  int lw = 0;
  double* W = (double*)ctx->lam.ptr;
  CS(cusolverDnDsyevd_bufferSize(ctx->sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, Hh, n,
                                 W, &lw));
  if ((st = grow(ctx, ctx->work, (size_t)lw * 8 + 256)) != CHFSI_OK) return st;
  CS(cusolverDnDsyevd(ctx->sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, Hh, n, W,
                      (double*)ctx->work.ptr, lw, dinfo));
  int info = 0;
  CK(cudaMemcpyAsync(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  if (evals_host)
    CK(cudaMemcpyAsync(evals_host, W, (size_t)n * 8, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (info != 0) return fail(ctx, CHFSI_ERR_EIG, "RR: syevd info = " + std::to_string(info));
  // 3. X <- X Q
  return rotate_impl(ctx, prec, X, ldx, n, Hh, 0, 0);
}

// Residual norms in binary64.  rayleigh: use each column's Rayleigh quotient
// x.H~x / x.x (computed here in binary64) instead of evals, so the norm
// measures the vector alone (stopping test of the mixed solve, whose Ritz
// values carry the first-order error of the binary32 projection).
chfsi_status residual_impl(chfsi_ctx* ctx, const void* X, int64_t ldx, int n, chfsi_precision prec,
                           const double* evals, double* res, double* gres, bool rayleigh = false) {
  const HostMesh& m = ctx->mesh;
  chfsi_status st;
  if (n == 0) return CHFSI_OK;
  const int B = std::max(1, std::min({ctx->filter_block, n, kStage64}));
  // binary64 copies of the block and of H~ x (residual check always in binary64)
  if ((st = grow(ctx, ctx->rot, (size_t)m.ndofs * B * 8 * 2)) != CHFSI_OK) return st;
  if ((st = grow(ctx, ctx->lam, (size_t)n * 8 * 4 + 64)) != CHFSI_OK) return st;
  if ((st = grow(ctx, ctx->part, (size_t)3 * n * 8 * 512)) != CHFSI_OK) return st;
  double* X64 = (double*)ctx->rot.ptr;
  double* Y64 = X64 + (size_t)m.ndofs * B;
  double* dl = (double*)ctx->lam.ptr;
  double* out = dl + n;
  CK(cudaMemcpyAsync(dl, evals, (size_t)n * 8, cudaMemcpyHostToDevice, ctx->stream));
  std::vector<double> sq(3 * (size_t)n);
  for (int j0 = 0; j0 < n; j0 += B) {
    const int nb = std::min(B, n - j0);
    CK(launch_copy_cols((const char*)X + j0 * esize(prec), ldx, X64, nb, m.ndofs, nb,
                        prec == CHFSI_FP64, 1, ctx->stream));
    if ((st = apply_step(ctx, CHFSI_FP64, X64, nb, Y64, nb, nullptr, 0, nb, 1.0, 0.0, 0.0)) != CHFSI_OK)
      return st;
    std::vector<double> h(3 * (size_t)nb);
    if (rayleigh) {
      CK(launch_resid_norms(Y64, nb, X64, nb, m.ndofs, nb, nullptr, nullptr, out,
                            (double*)ctx->part.ptr, ctx->part.bytes, ctx->stream));
      CK(cudaMemcpyAsync(h.data(), out, h.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      std::vector<double> rho(nb);
      for (int i = 0; i < nb; ++i) rho[i] = h[i] / h[2 * nb + i];
      CK(cudaMemcpyAsync(dl + j0, rho.data(), (size_t)nb * 8, cudaMemcpyHostToDevice, ctx->stream));
    }
    CK(launch_resid_norms(Y64, nb, X64, nb, m.ndofs, nb, dl + j0, ctx->d_mass, out,
                          (double*)ctx->part.ptr, ctx->part.bytes, ctx->stream));
    CK(cudaMemcpyAsync(h.data(), out, h.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < nb; ++i) {
      double xx = h[2 * nb + i];
      if (res) res[j0 + i] = std::sqrt(h[i] / xx);
      if (gres) gres[j0 + i] = std::sqrt(h[nb + i] / xx);
    }
  }
  return CHFSI_OK;
}

// The ChFSI loop of chfsi_solve (step 7 of Algorithm scf, repeated): CholGS +
// RR on the start block, then `iters` x {filter, CholGS, RR}, with the
// adaptive early stop on the binary64 generalized residual.  final_fp64_rr:
// for the mixed precisions, evaluate the last RR with binary64 cell products
// (second-order eigenvalue error); a caller that refines the block afterwards
// passes false.  D receives the Ritz values, *it_out the iterations run.
chfsi_status solve_impl(chfsi_ctx* ctx, void* X, int64_t ldx, int n, int iters, int degree, double b,
                        double tol, int n_check, chfsi_precision prec, bool final_fp64_rr,
                        std::vector<double>& D, int* it_out) {
  chfsi_status st;
  if (n_check <= 0 || n_check > n) n_check = n;
  std::vector<double> res(n);
  const bool fp64_last = final_fp64_rr && is_mixed(prec);
  tic(ctx);
  if ((st = cholgs_impl(ctx, X, ldx, n, prec)) != CHFSI_OK) return st;
  toc(ctx, 1);
  tic(ctx);
  if ((st = rr_impl(ctx, X, ldx, n, prec, D.data(), iters == 0 && fp64_last)) != CHFSI_OK) return st;
  toc(ctx, 2);
  int it = 0;
  for (; it < iters; ++it) {
    double a = D[n - 1], a0 = D[0];
    if (!(a < b)) return fail(ctx, CHFSI_ERR_ARG, "upper bound b must exceed the largest Ritz value");
    if (!(a0 < a)) a0 = a - 1e-3 * std::max(1.0, std::fabs(a));
    tic(ctx);
    if ((st = filter_impl(ctx, X, ldx, n, degree, a, b, a0, prec)) != CHFSI_OK) return st;
    toc(ctx, 0);
    tic(ctx);
    if ((st = cholgs_impl(ctx, X, ldx, n, prec)) != CHFSI_OK) return st;
    toc(ctx, 1);
    tic(ctx);
    const bool last = (it + 1 == iters);
    if ((st = rr_impl(ctx, X, ldx, n, prec, D.data(), last && fp64_last)) != CHFSI_OK) return st;
    toc(ctx, 2);
    if (tol > 0.0) {
      tic(ctx);
      if ((st = residual_impl(ctx, X, ldx, n_check, prec, D.data(), nullptr, res.data(),
                              is_mixed(prec))) != CHFSI_OK)
        return st;
      toc(ctx, 3);
      double mx = *std::max_element(res.begin(), res.begin() + n_check);
      if (mx < tol) {
        ++it;
        if (!last && fp64_last) {   // stopping early: redo the last RR with binary64 products
          tic(ctx);
          if ((st = rr_impl(ctx, X, ldx, n, prec, D.data(), true)) != CHFSI_OK) return st;
          toc(ctx, 2);
        }
        break;
      }
    }
  }
  *it_out = it;
  return CHFSI_OK;
}

}  // namespace

// ================================================== apply without device allocation
// Fixed device scratch for chfsi_apply_noalloc: the partial-sum buffer of the
// colour-ordered assembly and, with projectors, the projected coefficients and
// their expansion.  It is a file-scope device array, so every GPU that loads
// the library holds these bytes until the process exits.
constexpr size_t kNoallocScratchBytes = size_t(64) << 20;   // 64 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {
// Device address of the scratch for the context, resolved on the context's
// first allocation-free call with cudaGetSymbolAddress (the array's host-side
// name is only a stand-in and must never be handed to a kernel).  It is kept
// in the context, so it lives exactly as long as the context's other device
// pointers (a cudaDeviceReset invalidates both).
cudaError_t noalloc_scratch(chfsi_ctx* ctx, void** out) {
  if (!ctx->noalloc_scratch) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    ctx->noalloc_scratch = p;
  }
  *out = ctx->noalloc_scratch;
  return cudaSuccess;
}
}  // namespace

// ===================================================================== C ABI
namespace chfsi {
// Rayleigh-Ritz for the library's own drivers (batched solve): fp64_apply
// applies H~ with binary64 cell products to a binary32 block.
chfsi_status rayleigh_ritz_internal(chfsi_ctx* ctx, void* X, int64_t ldx, int n, chfsi_precision prec,
                                    double* evals_host, bool fp64_apply) {
  CHECK_CTX();
  chfsi_status st = check_x(ctx, X, ldx, n, prec);
  if (st != CHFSI_OK) return st;
  if ((st = rr_impl(ctx, X, ldx, n, prec, evals_host, fp64_apply)) != CHFSI_OK) return st;
  return check_device_status(ctx, prec);
}
}  // namespace chfsi

extern "C" {

chfsi_status chfsi_create(const chfsi_mesh_desc* desc, void* stream, chfsi_ctx** out) {
  if (!desc || !out) return CHFSI_ERR_ARG;
  *out = nullptr;
  if (desc->p < 1 || desc->p > 8) return CHFSI_ERR_ARG;
  for (int a = 0; a < 3; ++a) {
    if (desc->ncell[a] < 1 || !(desc->len[a] > 0.0)) return CHFSI_ERR_ARG;
    if (desc->periodic[a] && desc->ncell[a] < 2) return CHFSI_ERR_ARG;
    if (!desc->periodic[a] && desc->ncell[a] * desc->p < 2) return CHFSI_ERR_ARG;
  }
  if (desc->quad_points < 0 || desc->quad_points > 16) return CHFSI_ERR_ARG;
  int64_t nd = 1;
  for (int a = 0; a < 3; ++a) nd *= desc->periodic[a] ? (int64_t)desc->ncell[a] * desc->p
                                                      : (int64_t)desc->ncell[a] * desc->p - 1;
  if (nd >= (int64_t)1 << 31) return CHFSI_ERR_ARG;
  chfsi_ctx* ctx = new chfsi_ctx();
  ctx->stream = (cudaStream_t)stream;
  cudaGetDevice(&ctx->device);
  build_mesh(*desc, ctx->mesh);
  const HostMesh& m = ctx->mesh;
  cudaError_t e;
  if ((e = upload(ctx, &ctx->d_dofmap, m.dofmap)) != cudaSuccess ||
      (e = upload(ctx, &ctx->d_modes, m.modes)) != cudaSuccess ||
      (e = upload(ctx, &ctx->d_cells, m.colour_cells)) != cudaSuccess ||
      (e = upload(ctx, &ctx->d_mass, m.mass)) != cudaSuccess ||
      (e = upload(ctx, &ctx->d_node_ptr, m.node_ptr)) != cudaSuccess ||
      (e = upload(ctx, &ctx->d_node_ent, m.node_ent)) != cudaSuccess ||
      (e = upload(ctx, &ctx->d_msq, minv_sqrt(m))) != cudaSuccess ||
      (e = cudaEventCreate(&ctx->ev[0])) != cudaSuccess ||
      (e = cudaEventCreate(&ctx->ev[1])) != cudaSuccess ||
      (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) {
    chfsi_destroy(ctx);
    return e == cudaErrorMemoryAllocation ? CHFSI_ERR_OOM : CHFSI_ERR_CUDA;
  }
  *out = ctx;
  return CHFSI_OK;
}

chfsi_status chfsi_destroy(chfsi_ctx* ctx) {
  if (!ctx) return CHFSI_ERR_ARG;
  if (ctx->stream || true) cudaStreamSynchronize(ctx->stream);
  free_device_data(ctx);
  const HostMesh& m = ctx->mesh;
  release(ctx, ctx->d_dofmap, m.dofmap.size() * 4);
  release(ctx, ctx->d_modes, m.modes.size());
  release(ctx, ctx->d_cells, m.colour_cells.size() * 4);
  release(ctx, ctx->d_mass, m.mass.size() * 8);
  release(ctx, ctx->d_node_ptr, m.node_ptr.size() * 4);
  release(ctx, ctx->d_node_ent, m.node_ent.size() * 4);
  release(ctx, ctx->d_msq, m.mass.size() * 8);
  if (ctx->d_kfac) cudaFree(ctx->d_kfac);
  ctx->d_kfac = nullptr;
  for (void* q : {(void*)ctx->d_kA, (void*)ctx->d_kG, (void*)ctx->kbf, (void*)ctx->kgbf})
    if (q) cudaFree(q);
  for (DevBuf* b : {&ctx->T1, &ctx->Wb, &ctx->NLb, &ctx->Zb, &ctx->rot, &ctx->Ssq, &ctx->work,
                    &ctx->part, &ctx->vec, &ctx->lam, &ctx->Rb, &ctx->Db, &ctx->pol, &ctx->scfb, &ctx->scfq,
                    &ctx->cmaxb, &ctx->pjb, &ctx->tinv,
                    &ctx->scfr, &ctx->scfw, &ctx->kW, &ctx->kT1, &ctx->kG, &ctx->kS, &ctx->kwork,
                    &ctx->kY, &ctx->kvec})
    dfree(ctx, b->ptr, b->bytes);
  for (int l = 0; l < chfsi_ctx::kMaxLanes; ++l) {
    for (DevBuf* b : {&ctx->laneT1[l], &ctx->laneR[l], &ctx->laneZ[l], &ctx->laneC[l], &ctx->laneP[l]})
      dfree(ctx, b->ptr, b->bytes);
    if (ctx->lane_stream[l]) cudaStreamDestroy(ctx->lane_stream[l]);
    if (ctx->lane_ev[l]) cudaEventDestroy(ctx->lane_ev[l]);
  }
  if (ctx->sol) cusolverDnDestroy(ctx->sol);
  for (auto& ev : ctx->ev)
    if (ev) cudaEventDestroy(ev);
  for (auto& r : ctx->krec) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : ctx->kev_free) cudaEventDestroy(e);
  delete ctx;
  return CHFSI_OK;
}

const char* chfsi_last_error(const chfsi_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t chfsi_num_dofs(const chfsi_ctx* ctx) { return ctx ? ctx->mesh.ndofs : -1; }

int64_t chfsi_device_bytes(const chfsi_ctx* ctx) { return ctx ? ctx->dev_bytes : -1; }

int64_t chfsi_kernel_launches(void) { return launch_count(); }

chfsi_status chfsi_set_kernel_timing(chfsi_ctx* ctx, int on) {
  CHECK_CTX();
  ctx->ktiming = on != 0;
  return CHFSI_OK;
}

chfsi_status chfsi_kernel_timings(chfsi_ctx* ctx, double* out6) {
  double* out4 = out6;
  CHECK_CTX();
  if (!out4) return CHFSI_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  for (auto& r : ctx->krec) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    ctx->kms[r.kind] += ms;
    ctx->kcount[r.kind] += 1;
    ctx->kev_free.push_back(r.a);
    ctx->kev_free.push_back(r.b);
  }
  ctx->krec.clear();
  out4[0] = ctx->kms[0];
  out4[1] = ctx->kms[1];
  out4[2] = (double)ctx->kcount[0];
  out4[3] = (double)ctx->kcount[1];
  out4[4] = ctx->kms[2];
  out4[5] = (double)ctx->kcount[2];
  ctx->kms[0] = ctx->kms[1] = ctx->kms[2] = 0.0;
  ctx->kcount[0] = ctx->kcount[1] = ctx->kcount[2] = 0;
  return CHFSI_OK;
}

chfsi_status chfsi_mass_diag(chfsi_ctx* ctx, double* host_out) {
  CHECK_CTX();
  if (!host_out) return CHFSI_ERR_ARG;
  std::memcpy(host_out, ctx->mesh.mass.data(), ctx->mesh.mass.size() * 8);
  return CHFSI_OK;
}

chfsi_status chfsi_set_potential_gaussians(chfsi_ctx* ctx, int n, const double* xyz,
                                           const double* depth, const double* width) {
  CHECK_CTX();
  if (n < 0 || (n > 0 && (!xyz || !depth || !width))) return fail(ctx, CHFSI_ERR_ARG, "bad wells");
  for (int i = 0; i < n; ++i)
    if (!(width[i] > 0.0)) return fail(ctx, CHFSI_ERR_ARG, "well width must be positive");
  ctx->wells.xyz.assign(xyz, xyz + 3 * n);
  ctx->wells.depth.assign(depth, depth + n);
  ctx->wells.width.assign(width, width + n);
  ctx->built = false;
  return CHFSI_OK;
}

chfsi_status chfsi_set_potential_qp(chfsi_ctx* ctx, const double* v, int64_t count) {
  CHECK_CTX();
  const HostMesh& m = ctx->mesh;
  const int64_t want = m.ncells * (int64_t)m.q * m.q * m.q;
  if (count == 0 && !v) {
    ctx->wells.vqp.clear();
  } else {
    if (!v || count != want)
      return fail(ctx, CHFSI_ERR_ARG, "potential values: need ncells * q^3 = " + std::to_string(want) +
                                          ", got " + std::to_string(count));
    for (int64_t i = 0; i < count; ++i)
      if (!std::isfinite(v[i])) return fail(ctx, CHFSI_ERR_ARG, "potential values must be finite");
    ctx->wells.vqp.assign(v, v + count);
  }
  ctx->built = false;
  return CHFSI_OK;
}

chfsi_status chfsi_set_projectors(chfsi_ctx* ctx, int n, const double* xyz, const double* h,
                                  double sigma, double rcut) {
  CHECK_CTX();
  if (n < 0 || (n > 0 && (!xyz || !h || !(sigma > 0.0) || !(rcut > 0.0))))
    return fail(ctx, CHFSI_ERR_ARG, "bad projectors");
  ctx->proj.xyz.assign(xyz, xyz + 3 * (size_t)n);
  ctx->proj.h.assign(h, h + 4 * (size_t)n);
  ctx->proj.sigma = sigma;
  ctx->proj.rcut = rcut;
  ctx->built = false;
  return CHFSI_OK;
}

chfsi_status chfsi_build(chfsi_ctx* ctx) {
  CHECK_CTX();
  CK(cudaStreamSynchronize(ctx->stream));
  free_device_data(ctx);
  const HostMesh& m = ctx->mesh;
  std::vector<double> Ht;
  build_cell_matrices(m, ctx->wells, Ht, &ctx->wv);
  build_mf_factors(m, ctx->fac);
  build_projectors(m, ctx->proj, ctx->hproj);
  cudaError_t e;
  if ((e = upload(ctx, &ctx->d_Ht, Ht)) != cudaSuccess ||
      (e = upload(ctx, &ctx->d_wv, ctx->wv)) != cudaSuccess ||
      (e = upload(ctx, &ctx->d_fac, ctx->fac)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, e == cudaErrorMemoryAllocation ? CHFSI_ERR_OOM : CHFSI_ERR_CUDA,
                std::string("cell matrices: ") + cudaGetErrorString(e));
  }
  if (ctx->hproj.nsite > 0) {
    std::vector<float> sc32(ctx->hproj.site_c.begin(), ctx->hproj.site_c.end());
    std::vector<float> dc32(ctx->hproj.dof_c.begin(), ctx->hproj.dof_c.end());
    CK(upload(ctx, &ctx->d_site_ptr, ctx->hproj.site_ptr));
    CK(upload(ctx, &ctx->d_site_dof, ctx->hproj.site_dof));
    CK(upload(ctx, &ctx->d_site_c, ctx->hproj.site_c));
    CK(upload(ctx, &ctx->d_dof_ptr, ctx->hproj.dof_ptr));
    CK(upload(ctx, &ctx->d_dof_site, ctx->hproj.dof_site));
    CK(upload(ctx, &ctx->d_dof_c, ctx->hproj.dof_c));
    CK(upload(ctx, &ctx->d_site_c32, sc32));
    CK(upload(ctx, &ctx->d_dof_c32, dc32));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  cudaError_t te = tc_build(ctx->tc, Ht, m.ncells, m.ne, ctx->stream, &ctx->dev_bytes);   // packed lazily
  if (te != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, te == cudaErrorMemoryAllocation ? CHFSI_ERR_OOM : CHFSI_ERR_CUDA,
                std::string("tensor-core cell data: ") + cudaGetErrorString(te));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->built = true;
  ++ctx->build_gen;
  return CHFSI_OK;
}

chfsi_status chfsi_set_blocking(chfsi_ctx* ctx, int filter_block, int diag_block) {
  CHECK_CTX();
  if (filter_block < 1 || diag_block < 1) return fail(ctx, CHFSI_ERR_ARG, "block sizes must be >= 1");
  ctx->filter_block = filter_block;
  ctx->diag_block = diag_block;
  return CHFSI_OK;
}

chfsi_status chfsi_set_filter_lanes(chfsi_ctx* ctx, int lanes) {
  CHECK_CTX();
  if (lanes < 1 || lanes > chfsi_ctx::kMaxLanes) return fail(ctx, CHFSI_ERR_ARG, "lanes must be 1..4");
  ctx->filter_lanes = lanes;
  return CHFSI_OK;
}

chfsi_status chfsi_set_gemm_kernels(chfsi_ctx* ctx, int tall, int gram) {
  CHECK_CTX();
  if (tall < -1 || tall > 1 || gram < -1 || gram > 1) return fail(ctx, CHFSI_ERR_ARG, "kernel must be -1, 0 or 1");
  ctx->tall_kernel = tall;
  ctx->gram_kernel = gram;
  return CHFSI_OK;
}

chfsi_status chfsi_set_cell_tile(chfsi_ctx* ctx, int tile) {
  CHECK_CTX();
  if (tile != 64 && tile != 128) return fail(ctx, CHFSI_ERR_ARG, "cell tile must be 64 or 128");
  ctx->cell_tile = tile;
  return CHFSI_OK;
}

chfsi_status chfsi_set_cell_gather(chfsi_ctx* ctx, int mode) {
  CHECK_CTX();
  if (mode < 0 || mode > 6)
    return fail(ctx, CHFSI_ERR_ARG, "cell kernel variant: 0 one ring, 1 bulk async copies, 2 / 3 decoupled "
                                    "rings with 2 / 4 gather warp pairs, 4 whole cell per thread block, "
                                    "5 several column tiles per thread block, 6 the same with one thread block per SM "
                                    "and two accumulators");
  ctx->cell_gather = mode;
  return CHFSI_OK;
}

chfsi_status chfsi_set_fp64_operator(chfsi_ctx* ctx, int op) {
  CHECK_CTX();
  if (op < -1 || op > 1) return fail(ctx, CHFSI_ERR_ARG, "operator: -1 default, 0 cell matrices, 1 matrix-free");
  if (op == 1 && !mf_supported(ctx->mesh.p, ctx->mesh.q))
    return fail(ctx, CHFSI_ERR_ARG, "the matrix-free apply needs 2 <= p <= 8 and p + 2 Gauss points");
  ctx->fp64_op = op;
  return CHFSI_OK;
}

int chfsi_fp64_operator(const chfsi_ctx* ctx) { return ctx ? (use_matrix_free(ctx) ? 1 : 0) : -1; }

chfsi_status chfsi_autotune(chfsi_ctx* ctx, const void* X, int64_t ldx, int n, chfsi_precision prec,
                            int* block_out, int* tile_out, double* ms_out) {
  CHECK_CTX();
  chfsi_status st = check_x(ctx, X, ldx, n, prec);
  if (st != CHFSI_OK) return st;
  if (!ctx->built) return fail(ctx, CHFSI_ERR_STATE, "autotune before build");
  const HostMesh& m = ctx->mesh;
  const size_t es = esize(prec);
  // candidates: the paper-sized block of 200, half and all of the columns;
  // the tensor-core cell kernel with 64- and 128-column tiles
  std::vector<int> blocks;
  for (int bk : {200, (n + 1) / 2, n}) {
    bk = std::max(1, std::min(bk, n));
    if (std::find(blocks.begin(), blocks.end(), bk) == blocks.end()) blocks.push_back(bk);
  }
  std::vector<int> tiles = is_mixed(prec) ? std::vector<int>{64, 128} : std::vector<int>{64};
  void* scratch = nullptr;
  CK(dalloc(ctx, &scratch, (size_t)m.ndofs * n * es));
  CK(cudaMemcpy2DAsync(scratch, n * es, X, ldx * es, n * es, m.ndofs, cudaMemcpyDeviceToDevice,
                       ctx->stream));
  const int save_block = ctx->filter_block, save_tile = ctx->cell_tile;
  double best = 1e300;
  int best_block = save_block, best_tile = save_tile, k = 0;
  for (int bk : blocks) {
    for (int tl : tiles) {
      ctx->filter_block = bk;
      ctx->cell_tile = tl;
      float ms = 0.f;
      for (int rep = 0; rep < 2 && st == CHFSI_OK; ++rep) {   // first run grows the scratch
        cudaEventRecord(ctx->ev[0], ctx->stream);
        st = filter_impl(ctx, scratch, n, n, 2, 1.0, 2.0, 0.0, prec);
        cudaEventRecord(ctx->ev[1], ctx->stream);
        cudaEventSynchronize(ctx->ev[1]);
        cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
      }
      if (st == CHFSI_ERR_OOM) {   // candidate does not fit: skip it, free what it grew
        st = CHFSI_OK;
        release_scratch(ctx);
        if (ms_out) ms_out[k] = -1.0;
        ++k;
        continue;
      }
      if (st != CHFSI_OK) break;
      if (ms_out) ms_out[k] = ms;
      ++k;
      if (ms < best) {
        best = ms;
        best_block = bk;
        best_tile = tl;
      }
    }
    if (st != CHFSI_OK) break;
  }
  dfree(ctx, scratch, (size_t)m.ndofs * n * es);
  release_scratch(ctx);   // regrown at the chosen size by the next call
  if (st == CHFSI_OK && best > 1e299) st = fail(ctx, CHFSI_ERR_OOM, "no blocking candidate fits in device memory");
  ctx->filter_block = st == CHFSI_OK ? best_block : save_block;
  ctx->cell_tile = st == CHFSI_OK ? best_tile : save_tile;
  if (st != CHFSI_OK) return st;
  if ((st = check_device_status(ctx, prec)) != CHFSI_OK) return st;
  if (block_out) *block_out = best_block;
  if (tile_out) *tile_out = best_tile;
  return CHFSI_OK;
}

chfsi_status chfsi_fill_uniform(chfsi_ctx* ctx, void* X, int64_t ldx, int64_t rows, int ncol,
                                uint64_t seed, uint64_t stream, chfsi_precision prec) {
  CHECK_CTX();
  if (!valid_prec(prec) || rows < 0 || ncol < 0 || (rows * ncol > 0 && (!X || ldx < ncol)))
    return fail(ctx, CHFSI_ERR_ARG, "bad fill arguments");
  CK(launch_fill_uniform(X, ldx, rows, ncol, stream_key(seed, stream), prec == CHFSI_FP64, ctx->stream));
  return CHFSI_OK;
}

chfsi_status chfsi_apply(chfsi_ctx* ctx, const void* X, int64_t ldx, void* Y, int64_t ldy, int ncol,
                         chfsi_precision prec) {
  CHECK_CTX();
  chfsi_status st = check_x(ctx, X, ldx, ncol, prec);
  if (st != CHFSI_OK) return st;
  if (ncol > 0 && (!Y || ldy < ncol)) return fail(ctx, CHFSI_ERR_ARG, "bad Y / ldy");
  st = apply_blocks(ctx, prec, X, ldx, Y, ldy, ncol);
  if (st == CHFSI_OK) st = check_device_status(ctx, prec);
  return st;
}

chfsi_status chfsi_apply_noalloc(chfsi_ctx* ctx, const double* X, int64_t ldx, double* Y,
                                 int64_t ldy, int ncol) {
  CHECK_CTX();
  chfsi_status st = check_x(ctx, X, ldx, ncol, CHFSI_FP64);
  if (st != CHFSI_OK) return st;
  if (ncol > 0 && (!Y || ldy < ncol)) return fail(ctx, CHFSI_ERR_ARG, "bad Y / ldy");
  if (ncol == 0) return CHFSI_OK;
  if (!ctx->d_Ht) return fail(ctx, CHFSI_ERR_STATE, "no cell matrices: the potential was set on the device");
  const HostMesh& m = ctx->mesh;
  const int nsite = ctx->hproj.nsite;
  const size_t w_bytes = (size_t)m.ndofs * ncol * sizeof(double);
  const size_t z_bytes = (size_t)4 * nsite * ncol * sizeof(double);
  const size_t need = w_bytes + (nsite > 0 ? w_bytes + z_bytes : 0);
  if (need > kNoallocScratchBytes)
    return fail(ctx, CHFSI_ERR_ARG,
                "chfsi_apply_noalloc: needs " + std::to_string(need) + " bytes of scratch for " +
                    std::to_string(ncol) + " columns, more than the fixed " +
                    std::to_string(kNoallocScratchBytes) + " bytes; use fewer columns per call");
  // the scratch address belongs to the context's device, which must be current
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != ctx->device) {
    cudaGetLastError();
    ctx->err = "chfsi_apply_noalloc: the context's device (" + std::to_string(ctx->device) +
               ") is not the current device (" + std::to_string(cur) + ")";
    return CHFSI_ERR_STATE;
  }
  void* scratch = nullptr;
  cudaError_t se = noalloc_scratch(ctx, &scratch);
  if (se != cudaSuccess) {   // reported, not latched: the context stays usable
    cudaGetLastError();
    ctx->err = std::string("chfsi_apply_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(se);
    return CHFSI_ERR_CUDA;
  }
  double* W = (double*)scratch;                       // written before read (MODE_STORE first)
  double* NL = nsite > 0 ? W + (size_t)m.ndofs * ncol : nullptr;
  double* Z = nsite > 0 ? NL + (size_t)m.ndofs * ncol : nullptr;
  if (nsite > 0) {
    CK(launch_nl_project_fp64(ctx->d_site_ptr, ctx->d_site_dof, ctx->d_site_c, nsite, X, ldx, ncol,
                              Z, ctx->stream));
    CK(launch_nl_expand_fp64(ctx->d_dof_ptr, ctx->d_dof_site, ctx->d_dof_c, m.ndofs, Z, ncol, NL,
                             ncol, ctx->stream));
  }
  const int ncolour = (int)m.colour_offsets.size() - 1;
  for (int c = 0; c < ncolour; ++c) {
    CellLaunch L{};
    L.Ht = ctx->d_Ht;
    L.dofmap = ctx->d_dofmap;
    L.modes = ctx->d_modes;
    L.cells = ctx->d_cells + m.colour_offsets[c];
    L.ncells_colour = m.colour_offsets[c + 1] - m.colour_offsets[c];
    L.ne = m.ne;
    L.ncol = ncol;
    L.ld_in = ldx;
    L.ld_out = ldy;
    L.ld_prev = 0;
    CK(launch_cell_fp64(L, X, Y, nullptr, W, NL, ncol, FilterStep{1.0, 0.0, 0.0}, ctx->stream));
  }
  return CHFSI_OK;
}

chfsi_status chfsi_debug_withhold_arrival(chfsi_ctx* ctx, int on) {
  CHECK_CTX();
  CK(tc_set_withhold(on, ctx->stream));
  return CHFSI_OK;
}

chfsi_status chfsi_filter(chfsi_ctx* ctx, void* X, int64_t ldx, int ncol, int degree, double a,
                          double b, double a0, chfsi_precision prec) {
  CHECK_CTX();
  chfsi_status st = check_x(ctx, X, ldx, ncol, prec);
  if (st != CHFSI_OK) return st;
  if (degree < 1 || !(a0 < a) || !(a < b)) return fail(ctx, CHFSI_ERR_ARG, "filter needs degree >= 1 and a0 < a < b");
  std::fill(ctx->times, ctx->times + 4, 0.0);
  tic(ctx);
  st = filter_impl(ctx, X, ldx, ncol, degree, a, b, a0, prec);
  if (st == CHFSI_OK) toc(ctx, 0);
  if (st == CHFSI_OK) st = check_device_status(ctx, prec);
  return st;
}

chfsi_status chfsi_cholgs(chfsi_ctx* ctx, void* X, int64_t ldx, int n, chfsi_precision prec) {
  CHECK_CTX();
  chfsi_status st = check_x(ctx, X, ldx, n, prec);
  if (st != CHFSI_OK) return st;
  std::fill(ctx->times, ctx->times + 4, 0.0);
  tic(ctx);
  st = cholgs_impl(ctx, X, ldx, n, prec);
  if (st == CHFSI_OK) toc(ctx, 1);
  if (st == CHFSI_OK) st = check_device_status(ctx, prec);
  return st;
}

chfsi_status chfsi_rayleigh_ritz(chfsi_ctx* ctx, void* X, int64_t ldx, int n, chfsi_precision prec,
                                 double* evals_host) {
  CHECK_CTX();
  chfsi_status st = check_x(ctx, X, ldx, n, prec);
  if (st != CHFSI_OK) return st;
  std::fill(ctx->times, ctx->times + 4, 0.0);
  tic(ctx);
  st = rr_impl(ctx, X, ldx, n, prec, evals_host);
  if (st == CHFSI_OK) toc(ctx, 2);
  if (st == CHFSI_OK) st = check_device_status(ctx, prec);
  return st;
}

chfsi_status chfsi_rayleigh_ritz_split(chfsi_ctx* ctx, const void* X, int64_t ldx, int n, int n_fr,
                                       void* Xfr, int64_t ldfr, chfsi_precision prec,
                                       double* evals_fr_host) {
  CHECK_CTX();
  chfsi_status st = check_x(ctx, X, ldx, n, prec);
  if (st != CHFSI_OK) return st;
  if (n_fr < 1 || n_fr > n || !Xfr || ldfr < n_fr || !evals_fr_host)
    return fail(ctx, CHFSI_ERR_ARG, "bad split Rayleigh-Ritz arguments");
  const HostMesh& m = ctx->mesh;
  const size_t es = esize(prec);
  {   // the output block must not overlap X
    const char* x0 = (const char*)X;
    const char* x1 = x0 + ((m.ndofs - 1) * ldx + n) * es;
    const char* f0 = (const char*)Xfr;
    const char* f1 = f0 + ((m.ndofs - 1) * ldfr + n_fr) * es;
    if (f0 < x1 && x0 < f1) return fail(ctx, CHFSI_ERR_ARG, "X_fr overlaps X");
  }
  std::fill(ctx->times, ctx->times + 4, 0.0);
  tic(ctx);
  if ((st = ensure_solver(ctx)) != CHFSI_OK) return st;
  // 1. H^ = X^T H~ X
  if ((st = projected_impl(ctx, X, ldx, n, prec, false)) != CHFSI_OK) return st;
  double* Hh = (double*)ctx->Ssq.ptr;
  int* dinfo = (int*)((char*)ctx->Ssq.ptr + (size_t)n * n * 8);
  double* W = (double*)ctx->lam.ptr;
  // 2. the n_fr largest eigenpairs (binary64 syevdx, index range n - n_fr + 1 .. n);
  //    their eigenvectors overwrite the first n_fr columns of H^
  int lw = 0, meig = 0;
  const int il = n - n_fr + 1, iu = n;
  CS(cusolverDnDsyevdx_bufferSize(ctx->sol, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I,
                                  CUBLAS_FILL_MODE_LOWER, n, Hh, n, 0.0, 0.0, il, iu, &meig, W, &lw));
  if ((st = grow(ctx, ctx->work, (size_t)lw * 8 + 256)) != CHFSI_OK) return st;
  CS(cusolverDnDsyevdx(ctx->sol, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_LOWER,
                       n, Hh, n, 0.0, 0.0, il, iu, &meig, W, (double*)ctx->work.ptr, lw, dinfo));
  int info = 0;
  CK(cudaMemcpyAsync(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(evals_fr_host, W, (size_t)n_fr * 8, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (info != 0 || meig != n_fr)
    return fail(ctx, CHFSI_ERR_EIG, "split RR: syevdx info = " + std::to_string(info) +
                                        ", eigenpairs " + std::to_string(meig));
  // 3. X_fr = X Q_fr (the n x n_fr leading block of H^, leading dimension n)
  if (prec == CHFSI_FP64) {
    CK(launch_tallgemm_fp64((const double*)X, ldx, Hh, n, m.ndofs, n, n_fr, (double*)Xfr, ldfr, 0, 0,
                            ctx->stream));
  } else {
    if ((st = grow(ctx, ctx->work, tc_tallgemm_work_bytes(n, n_fr))) != CHFSI_OK) return st;
    CK(tc_tallgemm_mixed((const float*)X, ldx, Hh, n, m.ndofs, n, n_fr, (float*)Xfr, ldfr, 0, 0, 0,
                         split3_of(prec), ctx->work.ptr, ctx->stream, ctx->tall_kernel));
  }
  toc(ctx, 2);
  return check_device_status(ctx, prec);
}

chfsi_status chfsi_density(chfsi_ctx* ctx, const void* X, int64_t ldx, int n, const void* Xfr,
                           int64_t ldfr, int n_fr, const double* occ_fr_host, chfsi_precision prec,
                           double* rho) {
  CHECK_CTX();
  chfsi_status st = check_x(ctx, X, ldx, n, prec);
  if (st != CHFSI_OK) return st;
  if (n_fr < 0 || n_fr > 0 && (!Xfr || ldfr < n_fr || !occ_fr_host) || !rho)
    return fail(ctx, CHFSI_ERR_ARG, "bad density arguments");
  const HostMesh& m = ctx->mesh;
  // tables: basis at the Gauss points (q x n1), weights 2 (f - 1); M^{-1/2} is resident
  const size_t nb = (size_t)m.q * m.n1;
  if ((st = grow(ctx, ctx->Db, (nb + (size_t)n_fr + 8) * 8)) != CHFSI_OK) return st;
  std::vector<double> h(nb + (size_t)n_fr);
  std::copy(m.B.begin(), m.B.end(), h.begin());
  for (int j = 0; j < n_fr; ++j) h[nb + j] = 2.0 * (occ_fr_host[j] - 1.0);
  double* d = (double*)ctx->Db.ptr;
  CK(cudaMemcpyAsync(d, h.data(), h.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
  DensityArgs a{};
  a.X = X;
  a.ldx = ldx;
  a.n = n;
  a.Xfr = n_fr > 0 ? Xfr : X;
  a.ldfr = n_fr > 0 ? ldfr : ldx;
  a.nfr = n_fr;
  a.wfr = d + nb;
  a.dofmap = ctx->d_dofmap;
  a.minv_sqrt = ctx->d_msq;
  a.B = d;
  a.Bh = m.B.data();
  a.ncells = m.ncells;
  a.n1 = m.n1;
  a.q = m.q;
  a.is_double = prec == CHFSI_FP64;
  a.rho = rho;
  CK(launch_density(a, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));   // the host table must outlive its copy
  return CHFSI_OK;
}

chfsi_status chfsi_residuals(chfsi_ctx* ctx, const void* X, int64_t ldx, int n, chfsi_precision prec,
                             const double* evals_host, double* res_host, double* gres_host) {
  CHECK_CTX();
  chfsi_status st = check_x(ctx, X, ldx, n, prec);
  if (st != CHFSI_OK) return st;
  if (n > 0 && !evals_host) return fail(ctx, CHFSI_ERR_ARG, "evals required");
  return residual_impl(ctx, X, ldx, n, prec, evals_host, res_host, gres_host);
}

chfsi_status chfsi_bounds(chfsi_ctx* ctx, int lanczos_steps, uint64_t seed, double* b_out) {
  CHECK_CTX();
  if (!ctx->built) return fail(ctx, CHFSI_ERR_STATE, "chfsi_build has not been called");
  if (lanczos_steps < 1 || !b_out) return fail(ctx, CHFSI_ERR_ARG, "bad Lanczos arguments");
  const int64_t M = ctx->mesh.ndofs;
  chfsi_status st;
  if ((st = grow(ctx, ctx->vec, (size_t)M * 8 * 3 + 64)) != CHFSI_OK) return st;
  double* v = (double*)ctx->vec.ptr;
  double* vp = v + M;
  double* w = vp + M;
  double* dot = (double*)ctx->lam.ptr;
  if ((st = grow(ctx, ctx->lam, 64)) != CHFSI_OK) return st;
  dot = (double*)ctx->lam.ptr;
  if ((st = grow(ctx, ctx->part, (size_t)8 * 1024)) != CHFSI_OK) return st;
  CK(launch_fill_uniform(v, 1, M, 1, stream_key(seed, 7), 1, ctx->stream));
  CK(cudaMemsetAsync(vp, 0, M * 8, ctx->stream));
  auto dotp = [&](const double* x, const double* y, double* r) -> chfsi_status {
    CK(launch_gram_fp64(x, 1, y, 1, M, 1, 1, dot, 1, 0, (double*)ctx->part.ptr, ctx->part.bytes,
                        ctx->stream));
    CK(cudaMemcpyAsync(r, dot, 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return CHFSI_OK;
  };
  double nv = 0.0;
  if ((st = dotp(v, v, &nv)) != CHFSI_OK) return st;
  CK(launch_scal_copy(v, v, M, 1.0 / std::sqrt(nv), ctx->stream));
  std::vector<double> al, be;
  double bprev = 0.0;
  for (int k = 0; k < lanczos_steps; ++k) {
    if ((st = apply_step(ctx, CHFSI_FP64, v, 1, w, 1, nullptr, 0, 1, 1.0, 0.0, 0.0)) != CHFSI_OK) return st;
    CK(launch_axpy2(w, v, vp, M, 0.0, -bprev, ctx->stream));
    double a = 0.0;
    if ((st = dotp(w, v, &a)) != CHFSI_OK) return st;
    CK(launch_axpy2(w, v, vp, M, -a, 0.0, ctx->stream));
    double bb = 0.0;
    if ((st = dotp(w, w, &bb)) != CHFSI_OK) return st;
    bb = std::sqrt(bb);
    al.push_back(a);
    be.push_back(bb);
    if (bb == 0.0) break;
    CK(cudaMemcpyAsync(vp, v, M * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(launch_scal_copy(v, w, M, 1.0 / bb, ctx->stream));
    bprev = bb;
  }
  // largest eigenvalue of the k x k tridiagonal by bisection (Sturm counts)
  const int k = (int)al.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < k; ++i) {
    double r = (i > 0 ? std::fabs(be[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(be[i]) : 0.0);
    lo = std::min(lo, al[i] - r);
    hi = std::max(hi, al[i] + r);
  }
  auto count_below = [&](double x) {
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < k; ++i) {
      double off = i > 0 ? be[i - 1] * be[i - 1] : 0.0;
      d = (al[i] - x) - (i > 0 ? off / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0) cnt++;
    }
    return cnt;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-14 * std::max(1.0, std::fabs(hi)); ++it) {
    double mid = 0.5 * (lo + hi);
    if (count_below(mid) >= k) hi = mid;
    else lo = mid;
  }
  *b_out = hi + std::fabs(be[k - 1]);
  return CHFSI_OK;
}

chfsi_status chfsi_solve(chfsi_ctx* ctx, void* X, int64_t ldx, int n, int iters, int degree, double b,
                         double tol, int n_check, chfsi_precision prec, double* evals_host,
                         int* iters_done) {
  CHECK_CTX();
  chfsi_status st = check_x(ctx, X, ldx, n, prec);
  if (st != CHFSI_OK) return st;
  if (n < 1 || iters < 0 || degree < 1 || !evals_host) return fail(ctx, CHFSI_ERR_ARG, "bad solve arguments");
  std::fill(ctx->times, ctx->times + 4, 0.0);
  std::vector<double> D(n);
  int it = 0;
  if ((st = solve_impl(ctx, X, ldx, n, iters, degree, b, tol, n_check, prec, true, D, &it)) != CHFSI_OK)
    return st;
  if ((st = check_device_status(ctx, prec)) != CHFSI_OK) return st;
  std::memcpy(evals_host, D.data(), (size_t)n * 8);
  if (iters_done) *iters_done = it;
  return CHFSI_OK;
}

chfsi_status chfsi_solve_polish(chfsi_ctx* ctx, float* X, int64_t ldx, int n, int iters, int degree,
                                double b, double tol, int n_check, chfsi_precision prec,
                                int polish_iters, int polish_degree, double* X64, int64_t ldx64,
                                double* evals_host, int* iters_done) {
  CHECK_CTX();
  chfsi_status st = check_x(ctx, X, ldx, n, prec);
  if (st != CHFSI_OK) return st;
  if (!is_mixed(prec)) return fail(ctx, CHFSI_ERR_ARG, "the polish follows a mixed-precision solve");
  if (n < 1 || iters < 0 || degree < 1 || polish_iters < 1 || polish_degree < 1 || !evals_host ||
      (X64 && ldx64 < n))
    return fail(ctx, CHFSI_ERR_ARG, "bad polished-solve arguments");
  const HostMesh& m = ctx->mesh;
  if (X64) {   // the binary64 block must not overlap the binary32 one
    const char* x0 = (const char*)X;
    const char* x1 = x0 + ((m.ndofs - 1) * ldx + n) * 4;
    const char* y0 = (const char*)X64;
    const char* y1 = y0 + ((m.ndofs - 1) * ldx64 + n) * 8;
    if (y0 < x1 && x0 < y1) return fail(ctx, CHFSI_ERR_ARG, "X64 overlaps X");
  }
  std::fill(ctx->times, ctx->times + 4, 0.0);
  std::vector<double> D(n);
  int it = 0;
  // 1. the mixed-precision iterations; their last Rayleigh-Ritz stays in the
  //    tensor-core arithmetic (the polish recomputes the Ritz pairs)
  if ((st = solve_impl(ctx, X, ldx, n, iters, degree, b, tol, n_check, prec, false, D, &it)) != CHFSI_OK)
    return st;
  if ((st = check_device_status(ctx, prec)) != CHFSI_OK) return st;
  // 2. binary64 copy of the block (caller's X64, else library staging)
  double* P = X64;
  int64_t ldp = ldx64;
  if (!P) {
    if ((st = grow(ctx, ctx->pol, (size_t)m.ndofs * n * 8)) != CHFSI_OK) return st;
    P = (double*)ctx->pol.ptr;
    ldp = n;
  }
  CK(launch_copy_cols(X, ldx, P, ldp, m.ndofs, n, 0, 1, ctx->stream));
  // 3. binary64 ChFSI iterations from the mixed subspace (bounds from its last RR)
  for (int k = 0; k < polish_iters; ++k) {
    double a = D[n - 1], a0 = D[0];
    if (!(a < b)) return fail(ctx, CHFSI_ERR_ARG, "upper bound b must exceed the largest Ritz value");
    if (!(a0 < a)) a0 = a - 1e-3 * std::max(1.0, std::fabs(a));
    tic(ctx);
    if ((st = filter_impl(ctx, P, ldp, n, polish_degree, a, b, a0, CHFSI_FP64)) != CHFSI_OK) return st;
    toc(ctx, 0);
    tic(ctx);
    if ((st = cholgs_impl(ctx, P, ldp, n, CHFSI_FP64)) != CHFSI_OK) return st;
    toc(ctx, 1);
    tic(ctx);
    if ((st = rr_impl(ctx, P, ldp, n, CHFSI_FP64, D.data())) != CHFSI_OK) return st;
    toc(ctx, 2);
  }
  // 4. the polished block rounded back into the caller's binary32 block
  CK(launch_copy_cols(P, ldp, X, ldx, m.ndofs, n, 1, 0, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  std::memcpy(evals_host, D.data(), (size_t)n * 8);
  if (iters_done) *iters_done = it;
  return CHFSI_OK;
}

chfsi_status chfsi_step_host(chfsi_ctx* ctx, void* X_host, int64_t ldh, void* X, int64_t ldx, int n,
                             int degree, double a, double b, double a0, chfsi_precision prec,
                             int copy_mode, double* evals_host, double* ms3) {
  CHECK_CTX();
  chfsi_status st = check_x(ctx, X, ldx, n, prec);
  if (st != CHFSI_OK) return st;
  if (n < 1 || !X_host || ldh < n || degree < 1 || !(a0 < a) || !(a < b) || !evals_host ||
      copy_mode < 0 || copy_mode > 2)
    return fail(ctx, CHFSI_ERR_ARG, "bad host-step arguments");
  const HostMesh& m = ctx->mesh;
  const size_t es = esize(prec);
  // the SMs move the rows over the coherent host link when the host block is
  // device-mapped (pinned); otherwise, or when asked, the copy engines do
  void* hdev = nullptr;
  bool mapped = false;
  if (copy_mode != 1) {
    mapped = cudaHostGetDevicePointer(&hdev, X_host, 0) == cudaSuccess;
    if (!mapped) cudaGetLastError();
  }
  if (copy_mode == 2 && !mapped)
    return fail(ctx, CHFSI_ERR_ARG, "SM copies need a pinned (device-mapped) host block");
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  for (auto& e : ev) CK(cudaEventCreate(&e));
  auto destroy = [&] {
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
  };
  auto move = [&](const void* src, int64_t lds, void* dst, int64_t ldd, bool to_dev) -> cudaError_t {
    if (mapped)
      return launch_copy2d(to_dev ? hdev : src, lds * es, to_dev ? dst : hdev, ldd * es, m.ndofs,
                           (int64_t)n * es, nsm, ctx->stream);
    return cudaMemcpy2DAsync(dst, ldd * es, src, lds * es, n * es, m.ndofs,
                             to_dev ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost, ctx->stream);
  };
  std::fill(ctx->times, ctx->times + 4, 0.0);
  cudaError_t ce = cudaEventRecord(ev[0], ctx->stream);
  if (ce == cudaSuccess) ce = move(X_host, ldh, X, ldx, true);
  if (ce == cudaSuccess) ce = cudaEventRecord(ev[1], ctx->stream);
  if (ce != cudaSuccess) {
    destroy();
    return fail(ctx, CHFSI_ERR_CUDA, std::string("host-to-device copy: ") + cudaGetErrorString(ce));
  }
  std::vector<double> D(n);
  st = filter_impl(ctx, X, ldx, n, degree, a, b, a0, prec);
  if (st == CHFSI_OK) st = cholgs_impl(ctx, X, ldx, n, prec);
  if (st == CHFSI_OK) st = rr_impl(ctx, X, ldx, n, prec, D.data());
  if (st != CHFSI_OK) {
    destroy();
    return st;
  }
  ce = cudaEventRecord(ev[2], ctx->stream);
  if (ce == cudaSuccess) ce = move(X, ldx, X_host, ldh, false);
  if (ce == cudaSuccess) ce = cudaEventRecord(ev[3], ctx->stream);
  if (ce == cudaSuccess) ce = cudaEventSynchronize(ev[3]);
  if (ce != cudaSuccess) {
    destroy();
    return fail(ctx, CHFSI_ERR_CUDA, std::string("device-to-host copy: ") + cudaGetErrorString(ce));
  }
  if (ms3)
    for (int k = 0; k < 3; ++k) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
      ms3[k] = t;
    }
  destroy();
  std::memcpy(evals_host, D.data(), (size_t)n * 8);
  return check_device_status(ctx, prec);
}

chfsi_status chfsi_unscale(chfsi_ctx* ctx, void* X, int64_t ldx, int ncol, chfsi_precision prec) {
  CHECK_CTX();
  if (!valid_prec(prec) || ncol < 0 || (ncol > 0 && (!X || ldx < ncol))) return fail(ctx, CHFSI_ERR_ARG, "bad X");
  const HostMesh& m = ctx->mesh;
  chfsi_status st;
  if ((st = grow(ctx, ctx->vec, (size_t)m.ndofs * 8 * 3 + 64)) != CHFSI_OK) return st;
  std::vector<double> s(m.ndofs);
  for (int64_t j = 0; j < m.ndofs; ++j) s[j] = 1.0 / std::sqrt(m.mass[j]);
  CK(cudaMemcpyAsync(ctx->vec.ptr, s.data(), s.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
  CK(launch_scale_rows(X, ldx, m.ndofs, ncol, (const double*)ctx->vec.ptr, prec == CHFSI_FP64, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return CHFSI_OK;
}

chfsi_status chfsi_last_timings(chfsi_ctx* ctx, double* out4) {
  CHECK_CTX();
  if (!out4) return CHFSI_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < 4; ++i) out4[i] = ctx->times[i];
  return CHFSI_OK;
}

}  // extern "C"
