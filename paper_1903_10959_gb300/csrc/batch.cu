// Batched filtering of many independent systems (same FE degree) on the
// tensor cores: per Chebyshev degree step ONE persistent launch of the cell
// kernel covers the (system, cell, column-tile) items of every system and ONE
// launch of the assembly kernel covers every unknown of every system.  The
// whole degree-m filter is captured once into a CUDA graph and replayed; the
// per-system recurrence scalars (Eq. chebFilter, scaled form) are read from
// device memory, refreshed from a pinned host buffer by the graph's first
// node, so one graph serves every ChFSI iteration.  An autotuner times the
// column-tile width and pipeline depth of the cell kernel on the batch itself.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <thread>
#include <tuple>
#include <vector>

#include "ctx.h"
#include "tc_ptx.cuh"

using namespace chfsi;

namespace chfsi {

__device__ int g_batch_status = 0;

using BSys = TcBatchSys;

struct BParams {
  const BSys* sys;
  int nsys;
  int64_t nitems;
  int ne, mt, nk, split3, S, parity;
};

template <int BN>
struct BLayout {
  int a_bytes, y_bytes, stage, bar_off, total;
};
template <int BN>
__host__ __device__ inline BLayout<BN> b_layout(int mt, int split3, int S) {
  BLayout<BN> c;
  c.a_bytes = mt * 4096 * (split3 ? 2 : 1);
  c.y_bytes = BN * 8 * 4 * 2;
  c.stage = c.a_bytes + c.y_bytes;
  c.bar_off = S * c.stage;
  c.total = c.bar_off + 512;
  return c;
}
template <int BN>
int b_max_stages(int mt, int split3) {
  const BLayout<BN> l = b_layout<BN>(mt, split3, 1);
  int S = (226 * 1024 - 512) / l.stage;
  return std::min(S, 8);
}

// Persistent cell kernel: warp 0 streams the split cell matrices, warp 1
// issues the MMAs into a double-buffered TMEM accumulator, warps 2-5 gather +
// split the cell blocks of Y (stride 4 over the global chunk counter: needs
// S >= 4 for sound parity waits), warps 6-9 store the result blocks.
template <int BN>
__global__ void __launch_bounds__(320, 1) tc_cell_batched_kernel(BParams P) {
  using namespace ptx;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const BLayout<BN> L = b_layout<BN>(P.mt, P.split3, P.S);
  const int S = P.S;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * S + 4);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  const uint32_t sbase = smem_u32(smem);
  auto fa = [&](int s) { return smem_u32(bars + s); };
  auto fy = [&](int s) { return smem_u32(bars + S + s); };
  auto em = [&](int s) { return smem_u32(bars + 2 * S + s); };
  auto accf = [&](int b) { return smem_u32(bars + 3 * S + b); };
  auto acce = [&](int b) { return smem_u32(bars + 3 * S + 2 + b); };
  const int mt = P.mt, nk = P.nk, ne = P.ne;
  const uint32_t acc_cols = (uint32_t)(mt * BN);
  const uint32_t tmem_cols = 2 * acc_cols <= 64 ? 64 : (2 * acc_cols <= 128 ? 128 : (2 * acc_cols <= 256 ? 256 : 512));
  const int64_t my_items =
      P.nitems > blockIdx.x ? (P.nitems - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(fa(s), 1);
      mbar_init(fy(s), 32);
      mbar_init(em(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf(b), 1);
      mbar_init(acce(b), 128);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // item -> (system, cell, column offset); items of a CTA increase, so the
  // system index only moves forward
  struct Item {
    int s;
    int64_t e;
    int c0, ncv;
  };
  int s_hint = 0;
  auto item_at = [&](int64_t it) {
    const int64_t item = (int64_t)blockIdx.x + it * gridDim.x;
    while (s_hint + 1 < P.nsys && P.sys[s_hint + 1].item0 <= item) ++s_hint;
    const BSys& sy = P.sys[s_hint];
    const int64_t li = item - sy.item0;
    Item r;
    r.s = s_hint;
    r.e = li / sy.tiles;
    r.c0 = (int)(li % sy.tiles) * BN;
    r.ncv = min(BN, sy.ncol - r.c0);
    return r;
  };

  if (warp == 0) {
    if (lane == 0) {
      int64_t gi = 0, issued = 0;
      for (int64_t it = 0; it < my_items && !*(volatile int*)abort_flag; ++it) {
        const Item I = item_at(it);
        const char* Ae = reinterpret_cast<const char*>(P.sys[I.s].A) + I.e * (int64_t)nk * mt * 8192;
        for (int i = 0; i < nk; ++i, ++gi) {
          const int s = (int)(gi % S);
          if (gi >= S && !mbar_wait(em(s), (uint32_t)((gi / S) - 1) & 1)) {
            atomicExch(&g_batch_status, 1);
            *(volatile int*)abort_flag = 1;
            break;
          }
          mbar_arrive_expect_tx(fa(s), L.a_bytes);
          bulk_g2s(sbase + s * L.stage, Ae + (int64_t)i * mt * 8192, L.a_bytes, fa(s));
          ++issued;
        }
      }
      if (*(volatile int*)abort_flag)
        for (int64_t i = issued > S ? issued - S : 0; i < issued; ++i)
          mbar_wait(fa((int)(i % S)), (uint32_t)(i / S) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int64_t gi = 0;
      bool ok = true;
      for (int64_t it = 0; it < my_items && ok; ++it) {
        const int b = (int)(it & 1);
        if (it >= 2 && !mbar_wait(acce(b), (uint32_t)((it / 2) - 1) & 1)) {
          atomicExch(&g_batch_status, 2);
          *(volatile int*)abort_flag = 1;
          break;
        }
        tc_fence_after();
        const Item I = item_at(it);
        const int bne = I.ncv <= 16 ? 16 : (I.ncv + 15) / 16 * 16;
        const uint32_t idesc = idesc_tf32(128, bne);
        const uint32_t dbase = tmem + b * acc_cols;
        for (int i = 0; i < nk; ++i, ++gi) {
          const int s = (int)(gi % S);
          const uint32_t par = (uint32_t)(gi / S) & 1;
          if (!mbar_wait(fa(s), par) || !mbar_wait(fy(s), par) || *(volatile int*)abort_flag) {
            atomicExch(&g_batch_status, 3);
            *(volatile int*)abort_flag = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = sbase + s * L.stage;
          const uint32_t sy = sa + L.a_bytes;
          const uint64_t yhi = umma_desc(sy, 128, 256);
          const uint64_t ylo = umma_desc(sy + BN * 8 * 4, 128, 256);
          for (int t = 0; t < mt; ++t) {
            const uint32_t d = dbase + t * BN;
            const uint64_t ahi = umma_desc(sa + t * 4096, 128, 256);
            if (P.split3) {
              const uint64_t alo = umma_desc(sa + mt * 4096 + t * 4096, 128, 256);
              mma_tf32(d, alo, yhi, idesc, i > 0);
              mma_tf32(d, ahi, ylo, idesc, 1);
              mma_tf32(d, ahi, yhi, idesc, 1);
            } else {
              mma_tf32(d, ahi, yhi, idesc, i > 0);
            }
          }
          umma_commit(em(s));
        }
        umma_commit(accf(b));
      }
    }
  } else if (warp <= 5) {
    const int gw = warp - 2;
    constexpr int QPR = BN / 4;          // column quads per node row
    constexpr int NPL = 32 / QPR;        // node groups per warp pass (BN 64: 2, BN 32: 4)
    constexpr int NPT = 8 / NPL;         // nodes per lane
    const int q = lane / QPR;
    const int cq = (lane % QPR) * 4;
    const int64_t total = my_items * nk;
    auto load_chunk = [&](int64_t gi, float v[NPT][4]) {
      const int64_t it = gi / nk;
      const int i = (int)(gi - it * nk);
      const Item I = item_at(it);
      const BSys& sy = P.sys[I.s];
      const float* Y = sy.Y[P.parity];
      const int64_t ld = sy.ldY[P.parity];
      const bool vec = ((ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(Y) & 15) == 0);
#pragma unroll
      for (int a = 0; a < NPT; ++a) {
        const int l = i * 8 + q * NPT + a;
        const int g = l < ne ? sy.dofmap[I.e * ne + l] : -1;
        v[a][0] = v[a][1] = v[a][2] = v[a][3] = 0.f;
        if (g >= 0) {
          const float* src = Y + (int64_t)g * ld + I.c0 + cq;
          if (vec && cq + 4 <= I.ncv) {
            const float4 t4 = __ldg(reinterpret_cast<const float4*>(src));
            v[a][0] = t4.x; v[a][1] = t4.y; v[a][2] = t4.z; v[a][3] = t4.w;
          } else {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (cq + u < I.ncv) v[a][u] = __ldg(src + u);
          }
        }
      }
    };
    float va[NPT][4], vb[NPT][4];
    if (gw < total) load_chunk(gw, va);
    for (int64_t gi = gw; gi < total; gi += 4) {
      const bool more = gi + 4 < total;
      if (more) load_chunk(gi + 4, vb);
      const int s = (int)(gi % S);
      if (gi >= S && !mbar_wait(em(s), (uint32_t)((gi / S) - 1) & 1)) {
        atomicExch(&g_batch_status, 4);
        *(volatile int*)abort_flag = 1;
      }
      if (*(volatile int*)abort_flag) break;
      float* yh = reinterpret_cast<float*>(smem + s * L.stage + L.a_bytes);
      float* yl = yh + BN * 8;
      // the NPT K values of one column are consecutive in the K-major core
      // matrix: one 16-byte (NPT 4) or 8-byte (NPT 2) store each for hi and lo
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int n = cq + u;
        const int k0 = q * NPT;            // first K index of this lane within the chunk
        const int o = (n >> 3) * 64 + (k0 >> 2) * 32 + (n & 7) * 4 + (k0 & 3);
        float h[NPT], l[NPT];
#pragma unroll
        for (int a = 0; a < NPT; ++a) {
          h[a] = tf32_rna(va[a][u]);
          l[a] = va[a][u] - h[a];
        }
        if constexpr (NPT == 4) {
          *reinterpret_cast<float4*>(yh + o) = make_float4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<float4*>(yl + o) = make_float4(l[0], l[1], l[2], l[3]);
        } else if constexpr (NPT == 2) {
          *reinterpret_cast<float2*>(yh + o) = make_float2(h[0], h[1]);
          *reinterpret_cast<float2*>(yl + o) = make_float2(l[0], l[1]);
        } else {
#pragma unroll
          for (int a = 0; a < NPT; ++a) {
            yh[o + a] = h[a];
            yl[o + a] = l[a];
          }
        }
      }
      fence_proxy_async_smem();
      mbar_arrive(fy(s));
      if (more) {
#pragma unroll
        for (int a = 0; a < NPT; ++a)
#pragma unroll
          for (int u = 0; u < 4; ++u) va[a][u] = vb[a][u];
      }
    }
  } else {
    // store the result blocks: TMEM lane quadrant warp % 4, thread = row
    const int qd = warp & 3;
    for (int64_t it = 0; it < my_items; ++it) {
      const int b = (int)(it & 1);
      const Item I = item_at(it);
      const BSys& sy = P.sys[I.s];
      const int bne = I.ncv <= 16 ? 16 : (I.ncv + 15) / 16 * 16;
      const bool okw = !*(volatile int*)abort_flag && mbar_wait(accf(b), (uint32_t)(it / 2) & 1);
      if (!okw) {
        atomicExch(&g_batch_status, 5);
        *(volatile int*)abort_flag = 1;
      }
      tc_fence_after();
      const bool run = __all_sync(0xffffffffu, okw);
      const bool vst = (sy.ldr & 3) == 0;
      for (int t = 0; t < mt; ++t) {
        const int l = t * 128 + qd * 32 + lane;
        float* dst = sy.R + (I.e * ne + l) * sy.ldr + I.c0;
        for (int cb = 0; cb < bne; cb += 16) {
          float acc[16];
          __syncwarp();
          if (run) {
            tmem_ld16(tmem + ((uint32_t)(qd * 32) << 16) + b * acc_cols + t * BN + cb, acc);
            tmem_wait_ld();
          }
          if (!run || l >= ne) continue;
          if (vst && cb + 16 <= I.ncv) {
#pragma unroll
            for (int u = 0; u < 16; u += 4)
              *reinterpret_cast<float4*>(dst + cb + u) = make_float4(acc[u], acc[u + 1], acc[u + 2], acc[u + 3]);
          } else {
#pragma unroll
            for (int u = 0; u < 16; ++u)
              if (cb + u < I.ncv) dst[cb + u] = acc[u];
          }
        }
      }
      tc_fence_before();
      mbar_arrive(acce(b));     // TMEM buffer b is free again
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, tmem_cols);
}

// Assembly over all systems: thread = (system, unknown, 4 columns); sums the
// cell rows of the unknown in ascending cell order and applies
// Y_out = alpha (sum - shift Y_in) + beta Y_prev with the system's scalars of
// this degree step (coef[3 * s]); beta == 0 skips the read of Y_prev.
__global__ void __launch_bounds__(256) tc_assemble_batched_kernel(const BSys* __restrict__ sys, int nsys,
                                                                   int64_t nq_total,
                                                                   const float* __restrict__ coef,
                                                                   int parity) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= nq_total) return;
  int lo = 0, hi = nsys - 1;
  while (lo < hi) {             // last system with q0 <= idx
    const int mid = (lo + hi + 1) >> 1;
    if (sys[mid].q0 <= idx) lo = mid;
    else hi = mid - 1;
  }
  const BSys& sy = sys[lo];
  const int ncol = sy.ncol;
  const int nq = (ncol + 3) / 4;
  const int64_t li = idx - sy.q0;
  const int64_t j = li / nq;
  const int c = (int)(li - j * nq) * 4;
  const int nc = min(4, ncol - c);
  const float alpha = coef[3 * lo], beta = coef[3 * lo + 1], shift = coef[3 * lo + 2];
  const float* Yin = sy.Y[parity];
  float* Yout = const_cast<float*>(sy.Y[1 - parity]);
  const int64_t ldi = sy.ldY[parity], ldo = sy.ldY[1 - parity], ldr = sy.ldr;
  float sum[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k = sy.node_ptr[j]; k < sy.node_ptr[j + 1]; ++k) {   // R rows are 16-byte aligned
    const float4 r = __ldg(reinterpret_cast<const float4*>(sy.R + (int64_t)sy.node_ent[k] * ldr + c));
    sum[0] += r.x; sum[1] += r.y; sum[2] += r.z; sum[3] += r.w;
  }
  const bool vin = nc == 4 && (ldi & 3) == 0 && ((reinterpret_cast<uintptr_t>(Yin) & 15) == 0);
  const bool vout = nc == 4 && (ldo & 3) == 0 && ((reinterpret_cast<uintptr_t>(Yout) & 15) == 0);
  float yin[4] = {0.f, 0.f, 0.f, 0.f}, yp[4] = {0.f, 0.f, 0.f, 0.f};
  if (vin) {
    const float4 t = *reinterpret_cast<const float4*>(Yin + j * ldi + c);
    yin[0] = t.x; yin[1] = t.y; yin[2] = t.z; yin[3] = t.w;
  } else {
    for (int u = 0; u < nc; ++u) yin[u] = Yin[j * ldi + c + u];
  }
  if (beta != 0.f) {
    if (vout) {
      const float4 t = *reinterpret_cast<const float4*>(Yout + j * ldo + c);
      yp[0] = t.x; yp[1] = t.y; yp[2] = t.z; yp[3] = t.w;
    } else {
      for (int u = 0; u < nc; ++u) yp[u] = Yout[j * ldo + c + u];
    }
  }
  float out[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    out[u] = alpha * (sum[u] - shift * yin[u]);
    if (beta != 0.f) out[u] = fmaf(beta, yp[u], out[u]);
  }
  if (vout) {
    *reinterpret_cast<float4*>(Yout + j * ldo + c) = make_float4(out[0], out[1], out[2], out[3]);
  } else {
    for (int u = 0; u < nc; ++u) Yout[j * ldo + c + u] = out[u];
  }
}

}  // namespace chfsi

// ===================================================================== batch object
struct chfsi_batch {
  std::vector<chfsi_ctx*> ctx;
  cudaStream_t stream = nullptr;
  bool own_stream = false;       // created here (graphs cannot capture the legacy stream)
  int ne = 0, mt = 0, nk = 0;
  // device descriptors and buffers
  BSys* d_sys = nullptr;
  std::vector<BSys> h_sys;
  std::vector<DevBuf> T1, R;
  float* d_coef = nullptr;      // degree x nsys x 3
  float* h_coef = nullptr;      // pinned
  int coef_cap = 0;
  int64_t nitems = 0, nq = 0;
  // graph of the last filter configuration
  cudaGraphExec_t gexec = nullptr;
  std::vector<const void*> g_x;
  std::vector<int> g_ncol;
  std::vector<int64_t> g_ldx;
  std::vector<uint64_t> g_gen;   // build generation of each member context at capture
  int g_degree = -1, g_split3 = -1, g_bn = -1, g_S = -1;
  // tile choice: BN (32 / 64) and stages; set by the autotuner
  int bn = 64, S = -1;             // S < 0: the non-persistent multi-system kernel
  int nsm = 0;
  std::string err;
};

namespace {

void batch_free_graph(chfsi_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  b->g_degree = -1;
}

cudaError_t ensure_dbuf(DevBuf& d, size_t bytes) {
  if (d.bytes >= bytes) return cudaSuccess;
  if (d.ptr) cudaFree(d.ptr);
  d.ptr = nullptr;
  d.bytes = 0;
  cudaError_t e = cudaMalloc(&d.ptr, bytes);
  if (e == cudaSuccess) d.bytes = bytes;
  return e;
}

template <int BN>
cudaError_t launch_batched_cell(chfsi_batch* b, int split3, int S, int parity, cudaStream_t s) {
  BParams P{b->d_sys, (int)b->ctx.size(), b->nitems, b->ne, b->mt, b->nk, split3, S, parity};
  const BLayout<BN> L = b_layout<BN>(b->mt, split3, S);
  const int grid = (int)std::min<int64_t>(b->nitems, b->nsm);
  note_launch();
  tc_cell_batched_kernel<BN><<<grid, 320, L.total, s>>>(P);
  return cudaGetLastError();
}

// Cell-kernel modes of the batched filter (split3 argument of the helpers below).
constexpr int kBatchTf32 = 0, kBatchTf32x3 = 1, kBatchBf16x3 = 2;

int batch_mode(chfsi_precision prec) {
  return prec == CHFSI_MIXED_BF16X3 ? kBatchBf16x3 : (prec == CHFSI_MIXED_TF32X3 ? kBatchTf32x3 : kBatchTf32);
}

// Describe every system for the current filter call (pointers, items, quads).
// BF16x3: the packed three-term copy, items per (cell, 128-column tile, row part).
cudaError_t batch_describe(chfsi_batch* b, float* const* X, const int64_t* ldx, const int* ncol,
                           int bn, int mode) {
  const int n = (int)b->ctx.size();
  b->h_sys.assign(n, BSys{});
  int64_t item = 0, q = 0;
  for (int i = 0; i < n; ++i) {
    chfsi_ctx* c = b->ctx[i];
    const HostMesh& m = c->mesh;
    cudaError_t e;
    const int64_t ld4 = (ncol[i] + 3) / 4 * 4;   // 16-byte rows for the scratch and R
    if ((e = ensure_dbuf(b->T1[i], (size_t)m.ndofs * ld4 * 4 + 16)) != cudaSuccess) return e;
    if ((e = ensure_dbuf(b->R[i], (size_t)m.ncells * m.ne * ld4 * 4 + 16)) != cudaSuccess) return e;
    BSys& sy = b->h_sys[i];
    sy.A = mode == kBatchBf16x3 ? reinterpret_cast<const float*>(c->tc.bf) : c->tc.hi;
    sy.dofmap = c->d_dofmap;
    sy.Y[0] = X[i];
    sy.ldY[0] = ldx[i];
    sy.Y[1] = (const float*)b->T1[i].ptr;
    sy.ldY[1] = ld4;
    sy.R = (float*)b->R[i].ptr;
    sy.ldr = ld4;
    sy.node_ptr = c->d_node_ptr;
    sy.node_ent = c->d_node_ent;
    sy.ncells = m.ncells;
    sy.M = m.ndofs;
    sy.ncol = ncol[i];
    sy.tiles = mode == kBatchBf16x3 ? (ncol[i] + 127) / 128 * tc_bf16_parts(b->ne) : (ncol[i] + bn - 1) / bn;
    sy.item0 = item;
    sy.q0 = q;
    item += m.ncells * sy.tiles;
    q += m.ndofs * ((ncol[i] + 3) / 4);
  }
  b->nitems = item;
  b->nq = q;
  return cudaMemcpyAsync(b->d_sys, b->h_sys.data(), n * sizeof(BSys), cudaMemcpyHostToDevice,
                         b->stream);
}

// Enqueue the whole filter (degree steps) on b->stream (captured or not).
cudaError_t batch_enqueue(chfsi_batch* b, float* const* X, const int* ncol, int degree, int split3,
                          int bn, int S) {
  const int n = (int)b->ctx.size();
  cudaError_t e = cudaMemcpyAsync(b->d_coef, b->h_coef, (size_t)degree * n * 3 * sizeof(float),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e != cudaSuccess) return e;
  for (int k = 1; k <= degree; ++k) {
    const int parity = (k - 1) & 1;
    if (split3 == kBatchBf16x3)
      e = tc_cell_bf16_multi_launch(b->d_sys, n, b->nitems, b->ne, b->mt, parity, b->stream);
    else if (S < 0)
      e = tc_cell_multi_launch(b->d_sys, n, b->nitems, b->ne, b->mt, b->nk, split3, parity, b->stream);
    else
      e = bn == 64 ? launch_batched_cell<64>(b, split3, S, parity, b->stream)
                   : launch_batched_cell<32>(b, split3, S, parity, b->stream);
    if (e != cudaSuccess) return e;
    note_launch();
    tc_assemble_batched_kernel<<<(unsigned)((b->nq + 255) / 256), 256, 0, b->stream>>>(
        b->d_sys, n, b->nq, b->d_coef + (size_t)(k - 1) * n * 3, parity);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (degree & 1)   // Y_m sits in the scratch buffer: copy it back into X
    for (int i = 0; i < n; ++i) {
      const HostMesh& m = b->ctx[i]->mesh;
      e = cudaMemcpy2DAsync(X[i], b->h_sys[i].ldY[0] * 4, b->T1[i].ptr,
                            (size_t)b->h_sys[i].ldY[1] * 4, (size_t)ncol[i] * 4, m.ndofs,
                            cudaMemcpyDeviceToDevice, b->stream);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

void fill_coef(chfsi_batch* b, int degree, const double* a, const double* bb, const double* a0) {
  const int n = (int)b->ctx.size();
  for (int s = 0; s < n; ++s) {
    const double e = (bb[s] - a[s]) / 2.0, c = (bb[s] + a[s]) / 2.0;
    const double s1 = e / (a0[s] - c);
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
      float* cf = b->h_coef + ((size_t)(k - 1) * n + s) * 3;
      cf[0] = (float)alpha;
      cf[1] = (float)beta;
      cf[2] = (float)c;
    }
  }
}

chfsi_status bfail(chfsi_batch* b, chfsi_status st, const std::string& m) {
  b->err = m;
  return st;
}

chfsi_status batch_check(chfsi_batch* b, float* const* X, const int64_t* ldx, const int* ncol) {
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    const chfsi_ctx* c = b->ctx[i];
    if (!c->built || !c->d_Ht || c->hproj.nsite > 0 || c->latched != CHFSI_OK)
      return bfail(b, CHFSI_ERR_STATE, "system " + std::to_string(i) +
                                           " is not built, has projectors or has a latched error");
    if (!X || !X[i] || !ldx || !ncol || ncol[i] < 1 || ldx[i] < ncol[i])
      return bfail(b, CHFSI_ERR_ARG, "bad X / ldx / ncol for system " + std::to_string(i));
  }
  return CHFSI_OK;
}

chfsi_status batch_prepare(chfsi_batch* b, float* const* X, const int64_t* ldx, const int* ncol,
                           int degree, int bn, int mode) {
  const int n = (int)b->ctx.size();
  for (int i = 0; i < n; ++i) {
    chfsi_ctx* c = b->ctx[i];
    if (!c->tc.hi) {
      cudaError_t pe = tc_pack_from_device(c->tc, c->d_Ht, c->stream, &c->dev_bytes);
      if (pe != cudaSuccess) return bfail(b, CHFSI_ERR_OOM, "tensor-core cell data");
      cudaStreamSynchronize(c->stream);
    }
    if (mode == kBatchBf16x3 && !c->tc.bf) {
      cudaError_t pe = tc_pack_bf16_from_device(c->tc, c->d_Ht, c->stream, &c->dev_bytes);
      if (pe != cudaSuccess) return bfail(b, CHFSI_ERR_OOM, "BF16x3 cell data");
      cudaStreamSynchronize(c->stream);
    }
  }
  if (degree * n * 3 > b->coef_cap) {
    if (b->d_coef) cudaFree(b->d_coef);
    if (b->h_coef) cudaFreeHost(b->h_coef);
    b->coef_cap = degree * n * 3;
    if (cudaMalloc(&b->d_coef, b->coef_cap * sizeof(float)) != cudaSuccess ||
        cudaMallocHost(&b->h_coef, b->coef_cap * sizeof(float)) != cudaSuccess)
      return bfail(b, CHFSI_ERR_OOM, "coefficient buffers");
    batch_free_graph(b);
  }
  cudaError_t e = batch_describe(b, X, ldx, ncol, bn, mode);
  if (e != cudaSuccess) return bfail(b, CHFSI_ERR_OOM, cudaGetErrorString(e));
  return CHFSI_OK;
}

int batch_read_status_persistent(cudaStream_t s);
// Status words of both cell kernels (persistent batched, multi-system).
int batch_read_status(cudaStream_t s) {
  const int a = batch_read_status_persistent(s);
  const int c = tc_read_status(s);
  return a ? a : c;
}
int batch_read_status_persistent(cudaStream_t s) {
  int v = 0;
  cudaMemcpyFromSymbolAsync(&v, g_batch_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  if (v) {
    int z = 0;
    cudaMemcpyToSymbolAsync(g_batch_status, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
  }
  return v;
}

int default_stages(chfsi_batch* b, int bn, int split3) {
  const int S = bn == 64 ? b_max_stages<64>(b->mt, split3) : b_max_stages<32>(b->mt, split3);
  return S;
}

}  // namespace

extern "C" {

chfsi_status chfsi_batch_create(int n, chfsi_ctx* const* ctxs, void* stream, chfsi_batch** out) {
  if (n < 1 || !ctxs || !out) return CHFSI_ERR_ARG;
  *out = nullptr;
  const int p = ctxs[0] ? ctxs[0]->mesh.p : -1;
  for (int i = 0; i < n; ++i)
    if (!ctxs[i] || !ctxs[i]->built || !ctxs[i]->d_Ht || ctxs[i]->mesh.p != p || ctxs[i]->hproj.nsite > 0)
      return CHFSI_ERR_ARG;
  chfsi_batch* b = new chfsi_batch();
  b->ctx.assign(ctxs, ctxs + n);
  b->stream = (cudaStream_t)stream;
  b->ne = ctxs[0]->mesh.ne;
  b->mt = (b->ne + 127) / 128;
  b->nk = (b->ne + 7) / 8;
  if (b->mt > 4) {
    delete b;
    return CHFSI_ERR_ARG;
  }
  b->T1.resize(n);
  b->R.resize(n);
  if (!b->stream) {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return CHFSI_ERR_CUDA;
    }
    b->own_stream = true;
  }
  // kernel attributes are set here: they may not be changed during stream capture
  tc_cell_prepare();
  cudaFuncSetAttribute(tc_cell_batched_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  cudaFuncSetAttribute(tc_cell_batched_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaMalloc(&b->d_sys, n * sizeof(BSys)) != cudaSuccess) {
    delete b;
    return CHFSI_ERR_OOM;
  }
  *out = b;
  return CHFSI_OK;
}

chfsi_status chfsi_batch_destroy(chfsi_batch* b) {
  if (!b) return CHFSI_ERR_ARG;
  cudaStreamSynchronize(b->stream);
  batch_free_graph(b);
  for (auto& d : b->T1) cudaFree(d.ptr);
  for (auto& d : b->R) cudaFree(d.ptr);
  if (b->d_sys) cudaFree(b->d_sys);
  if (b->d_coef) cudaFree(b->d_coef);
  if (b->h_coef) cudaFreeHost(b->h_coef);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  return CHFSI_OK;
}

const char* chfsi_batch_last_error(const chfsi_batch* b) { return b ? b->err.c_str() : "null batch"; }

chfsi_status chfsi_batch_filter(chfsi_batch* b, float* const* X, const int64_t* ldx, const int* ncol,
                                int degree, const double* a, const double* bb, const double* a0,
                                chfsi_precision prec) {
  if (!b) return CHFSI_ERR_ARG;
  if (prec != CHFSI_MIXED_TF32X3 && prec != CHFSI_MIXED_TF32 && prec != CHFSI_MIXED_BF16X3)
    return bfail(b, CHFSI_ERR_ARG, "batched filter runs in a mixed precision");
  if (degree < 1 || !a || !bb || !a0) return bfail(b, CHFSI_ERR_ARG, "bad degree / bounds");
  chfsi_status st = batch_check(b, X, ldx, ncol);
  if (st != CHFSI_OK) return st;
  const int n = (int)b->ctx.size();
  for (int i = 0; i < n; ++i)
    if (!(a0[i] < a[i]) || !(a[i] < bb[i])) return bfail(b, CHFSI_ERR_ARG, "need a0 < a < b");
  const int split3 = batch_mode(prec);   // kBatchBf16x3: one multi-system BF16x3 launch per step
  const int bn = split3 == kBatchBf16x3 ? 128 : b->bn;
  const int S = split3 == kBatchBf16x3 ? -1 : (b->S != 0 ? b->S : default_stages(b, bn, split3));
  if (b->own_stream) cudaDeviceSynchronize();   // order after the caller's work on any stream
  // the graph is valid while pointers, widths, strides, degree and tile choice stay the
  // same and no member context has been rebuilt (a rebuild frees the cell data and
  // the dof map the graph's descriptors point to)
  bool same = b->gexec && b->g_degree == degree && b->g_split3 == split3 && b->g_bn == bn &&
              b->g_S == S && (int)b->g_x.size() == n;
  for (int i = 0; same && i < n; ++i)
    same = b->g_x[i] == X[i] && b->g_ncol[i] == ncol[i] && b->g_ldx[i] == ldx[i] &&
           b->g_gen[i] == b->ctx[i]->build_gen;
  cudaStreamSynchronize(b->stream);            // h_coef may still feed the previous replay
  if (!same) {
    batch_free_graph(b);
    if ((st = batch_prepare(b, X, ldx, ncol, degree, bn, split3)) != CHFSI_OK) return st;
    cudaStreamSynchronize(b->stream);
  }
  fill_coef(b, degree, a, bb, a0);
  if (!same) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e2 = batch_enqueue(b, X, ncol, degree, split3, bn, S);
      e = cudaStreamEndCapture(b->stream, &g);
      if (e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b->gexec = nullptr;
      return bfail(b, CHFSI_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    b->g_x.assign(X, X + n);
    b->g_ncol.assign(ncol, ncol + n);
    b->g_ldx.assign(ldx, ldx + n);
    b->g_gen.resize(n);
    for (int i = 0; i < n; ++i) b->g_gen[i] = b->ctx[i]->build_gen;
    b->g_degree = degree;
    b->g_split3 = split3;
    b->g_bn = bn;
    b->g_S = S;
  }
  cudaError_t e = cudaGraphLaunch(b->gexec, b->stream);
  if (e != cudaSuccess) return bfail(b, CHFSI_ERR_CUDA, cudaGetErrorString(e));
  if (batch_read_status(b->stream)) return bfail(b, CHFSI_ERR_TIMEOUT, "device wait timed out");
  return CHFSI_OK;
}

chfsi_status chfsi_batch_autotune(chfsi_batch* b, float* const* X, const int64_t* ldx,
                                  const int* ncol, chfsi_precision prec, int* choice,
                                  double* ms_out) {
  if (!b) return CHFSI_ERR_ARG;
  if (prec != CHFSI_MIXED_TF32X3 && prec != CHFSI_MIXED_TF32)
    return bfail(b, CHFSI_ERR_ARG, "autotuning is for the TF32 precisions (BF16x3 has one kernel)");
  chfsi_status st = batch_check(b, X, ldx, ncol);
  if (st != CHFSI_OK) return st;
  const int split3 = batch_mode(prec);
  const int n = (int)b->ctx.size();
  if (b->own_stream) cudaDeviceSynchronize();
  // candidates: the non-persistent multi-system kernel (64-column tiles), then
  // the persistent kernel with column tile 64 / 32 x deepest pipeline / 4 stages
  std::vector<std::pair<int, int>> cand{{64, -1}};
  for (int bn : {64, 32}) {
    const int smax = default_stages(b, bn, split3);
    cand.push_back({bn, smax});
    if (smax > 4) cand.push_back({bn, 4});
  }
  std::vector<double> lo(n, -2.0), hi(n, 50.0), mid(n, 0.0);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e300;
  int bi = 0;
  for (size_t c = 0; c < cand.size(); ++c) {
    const int bn = cand[c].first, S = cand[c].second;
    if ((st = batch_prepare(b, X, ldx, ncol, 2, bn, split3)) != CHFSI_OK) break;
    fill_coef(b, 2, mid.data(), hi.data(), lo.data());
    double t = 1e300;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, b->stream);
      cudaError_t e = batch_enqueue(b, X, ncol, 2, split3, bn, S);
      cudaEventRecord(e1, b->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        cudaGetLastError();
        ms = 1e30f;
      }
      t = std::min(t, (double)ms);
    }
    if (ms_out) ms_out[c] = t;
    if (t < best) {
      best = t;
      bi = (int)c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != CHFSI_OK) return st;
  if (batch_read_status(b->stream)) return bfail(b, CHFSI_ERR_TIMEOUT, "device wait timed out");
  b->bn = cand[bi].first;
  b->S = cand[bi].second;
  batch_free_graph(b);
  if (choice) *choice = bi;
  return CHFSI_OK;
}

chfsi_status chfsi_batch_set_candidate(chfsi_batch* b, int k) {
  if (!b) return CHFSI_ERR_ARG;
  const int n = chfsi_batch_candidates(b, nullptr, nullptr, 0);
  if (k < 0 || k >= n) return bfail(b, CHFSI_ERR_ARG, "no such candidate");
  std::vector<int> bn(n), st(n);
  chfsi_batch_candidates(b, bn.data(), st.data(), n);
  b->bn = bn[k];
  b->S = st[k];
  batch_free_graph(b);
  return CHFSI_OK;
}

int chfsi_batch_candidates(const chfsi_batch* b, int* bn_out, int* stages_out, int max) {
  if (!b) return 0;
  int k = 0;
  const int split3 = 1;
  if (max > 0) {
    if (bn_out) bn_out[0] = 64;
    if (stages_out) stages_out[0] = -1;
  }
  ++k;
  for (int bn : {64, 32}) {
    const int smax = bn == 64 ? b_max_stages<64>(b->mt, split3) : b_max_stages<32>(b->mt, split3);
    for (int S : {smax, 4}) {
      if (S == 4 && smax <= 4) continue;
      if (k < max) {
        if (bn_out) bn_out[k] = bn;
        if (stages_out) stages_out[k] = S;
      }
      ++k;
    }
  }
  return k;
}

chfsi_status chfsi_batch_solve(chfsi_batch* b, double* const* X, const int64_t* ldx, const int* n,
                               int iters, int degree, const double* bnd, chfsi_precision filter_prec,
                               chfsi_precision orth_prec, double* const* evals) {
  if (!b || !X || !ldx || !n || !bnd || !evals || iters < 0 || degree < 1) return CHFSI_ERR_ARG;
  if (orth_prec != CHFSI_FP64 && orth_prec != CHFSI_MIXED_TF32X3 && orth_prec != CHFSI_MIXED_BF16X3)
    return bfail(b, CHFSI_ERR_ARG, "batched CholGS / RR run in binary64, 3xTF32 or BF16x3");
  const bool mixed_orth = orth_prec != CHFSI_FP64;
  const int ns = (int)b->ctx.size();
  cudaDeviceSynchronize();   // the start blocks may come from any stream
  // binary32 working copies for the filter
  std::vector<DevBuf> X32(ns);
  std::vector<float*> xp(ns);
  std::vector<int64_t> ld32(ns);
  chfsi_status st = CHFSI_OK;
  for (int i = 0; i < ns; ++i) {
    if (!X[i] || n[i] < 1 || ldx[i] < n[i]) return bfail(b, CHFSI_ERR_ARG, "bad X");
    if (ensure_dbuf(X32[i], (size_t)b->ctx[i]->mesh.ndofs * n[i] * 4 + 16) != cudaSuccess) {
      for (auto& d : X32) cudaFree(d.ptr);
      return bfail(b, CHFSI_ERR_OOM, "binary32 copies");
    }
    xp[i] = (float*)X32[i].ptr;
    ld32[i] = n[i];
  }
  std::vector<std::vector<double>> D(ns);
  std::vector<chfsi_status> sts(ns, CHFSI_OK);
  // mixed orthogonalisation (3xTF32 or BF16x3) works on the binary32 copies in place; the last
  // Rayleigh-Ritz applies H~ with binary64 products (second-order eigenvalues)
  auto per_system_mixed = [&](int i, bool first, bool last) {
    chfsi_ctx* c = b->ctx[i];
    const int64_t M = c->mesh.ndofs;
    if (first && launch_copy_cols(X[i], ldx[i], xp[i], ld32[i], M, n[i], 1, 0, c->stream) != cudaSuccess) {
      sts[i] = CHFSI_ERR_CUDA;
      return;
    }
    D[i].resize(n[i]);
    chfsi_status s1 = chfsi_cholgs(c, xp[i], ld32[i], n[i], orth_prec);
    if (s1 == CHFSI_OK)
      s1 = rayleigh_ritz_internal(c, xp[i], ld32[i], n[i], orth_prec, D[i].data(), last);
    if (s1 == CHFSI_OK && last &&
        launch_copy_cols(xp[i], ld32[i], X[i], ldx[i], M, n[i], 0, 1, c->stream) != cudaSuccess)
      s1 = CHFSI_ERR_CUDA;
    if (s1 == CHFSI_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) s1 = CHFSI_ERR_CUDA;
    sts[i] = s1;
  };
  auto per_system = [&](int i, bool filtered) {
    chfsi_ctx* c = b->ctx[i];
    const int64_t M = c->mesh.ndofs;
    if (filtered) {   // binary32 filter output -> binary64 block
      if (launch_copy_cols(xp[i], ld32[i], X[i], ldx[i], M, n[i], 0, 1, c->stream) != cudaSuccess) {
        sts[i] = CHFSI_ERR_CUDA;
        return;
      }
    }
    D[i].resize(n[i]);
    chfsi_status s1 = chfsi_cholgs(c, X[i], ldx[i], n[i], CHFSI_FP64);
    if (s1 == CHFSI_OK) s1 = chfsi_rayleigh_ritz(c, X[i], ldx[i], n[i], CHFSI_FP64, D[i].data());
    if (s1 == CHFSI_OK &&
        launch_copy_cols(X[i], ldx[i], xp[i], ld32[i], M, n[i], 1, 0, c->stream) != cudaSuccess)
      s1 = CHFSI_ERR_CUDA;
    if (s1 == CHFSI_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) s1 = CHFSI_ERR_CUDA;
    sts[i] = s1;
  };
  auto run_all = [&](bool filtered, bool last) {
    std::vector<std::thread> th;
    for (int i = 0; i < ns; ++i) {
      if (mixed_orth) th.emplace_back(per_system_mixed, i, !filtered, last);
      else th.emplace_back(per_system, i, filtered);
    }
    for (auto& t : th) t.join();
    for (int i = 0; i < ns; ++i)
      if (sts[i] != CHFSI_OK) return bfail(b, sts[i], "system " + std::to_string(i) + ": " +
                                                           chfsi_last_error(b->ctx[i]));
    return CHFSI_OK;
  };
  if ((st = run_all(false, iters == 0)) == CHFSI_OK) {
    std::vector<double> a(ns), a0(ns);
    for (int it = 0; it < iters && st == CHFSI_OK; ++it) {
      for (int i = 0; i < ns; ++i) {
        a[i] = D[i][n[i] - 1];
        a0[i] = D[i][0];
        if (!(a0[i] < a[i])) a0[i] = a[i] - 1e-3 * std::max(1.0, std::fabs(a[i]));
      }
      st = chfsi_batch_filter(b, xp.data(), ld32.data(), n, degree, a.data(), bnd, a0.data(),
                              filter_prec);
      if (st == CHFSI_OK) st = run_all(true, it + 1 == iters);
    }
  }
  if (st == CHFSI_OK)
    for (int i = 0; i < ns; ++i) std::memcpy(evals[i], D[i].data(), (size_t)n[i] * 8);
  cudaStreamSynchronize(b->stream);
  batch_free_graph(b);     // the graph refers to the binary32 copies freed below
  for (auto& d : X32) cudaFree(d.ptr);
  return st;
}

}  // extern "C"
