// Private definition of the library context (shared by api.cu and batch.cu).
#pragma once

#include <string>
#include <vector>

#include <cusolverDn.h>

#include "internal.h"
#include "tc.h"

struct chfsi_ctx {
  chfsi::HostMesh mesh;
  chfsi::Wells wells;
  chfsi::Projectors proj;
  chfsi::HostProjectors hproj;
  cudaStream_t stream = nullptr;
  int device = 0;
  bool built = false;
  uint64_t build_gen = 0;
  void* noalloc_scratch = nullptr; // device address of the fixed no-allocation scratch          // bumped whenever the device cell data is rebuilt or freed
  chfsi_status latched = CHFSI_OK;
  std::string err;
  int filter_block = 200, diag_block = 1;
  int tall_kernel = -1, gram_kernel = -1;   // GEMM tile kernels: -1 by size, 0 128 x 128, 1 256-wide
  int cell_tile = 64;              // columns per CTA of the tensor-core cell kernel
  int cell_gather = 2;             // BF16x3 cell kernel: 2 decoupled rings (default), 0 one ring, 1 async gather, 3 rings with 4 gather pairs
  int64_t dev_bytes = 0;
  // resident device data
  double* d_Ht = nullptr;          // binary64 cell matrices
  double* d_wv = nullptr;          // matrix-free apply: w jac V at the Gauss points per cell
  double* d_fac = nullptr;         // matrix-free apply: 1-D factors
  double* d_msq = nullptr;         // M^{-1/2} per unknown
  std::vector<double> wv;          // host copy of d_wv (sizes)
  std::vector<double> fac;
  int fp64_op = -1;                // binary64 cell operator: 0 cell matrices, 1 matrix-free, -1 auto
  chfsi::TcCellData tc;                   // tensor-core copies (mixed precisions)
  int32_t* d_dofmap = nullptr;
  uint8_t* d_modes = nullptr;
  int32_t* d_cells = nullptr;
  double* d_mass = nullptr;
  int32_t* d_node_ptr = nullptr;
  int32_t* d_node_ent = nullptr;
  int64_t* d_site_ptr = nullptr;
  int32_t* d_site_dof = nullptr;
  double* d_site_c = nullptr;
  int64_t* d_dof_ptr = nullptr;
  int32_t* d_dof_site = nullptr;
  double* d_dof_c = nullptr;
  float* d_site_c32 = nullptr;
  float* d_dof_c32 = nullptr;
  // grown scratch
  chfsi::DevBuf T1, Wb, NLb, Zb, rot, Ssq, work, part, vec, lam, Rb;
  chfsi::DevBuf pol;               // binary64 staging block of the polish
  chfsi::DevBuf scfb, scfq, scfr, scfw;   // Poisson / SCF work arrays (scf.cu)
  chfsi::DevBuf kW, kT1, kG, kS, kwork, kY, kvec;   // Bloch (k-point) work arrays (kpoint.cu)
  double kpt[3] = {0, 0, 0};       // Bloch wavevector of the k-point entry points
  bool kset = false;
  double* d_kfac = nullptr;        // k-point factors of the matrix-free Bloch apply
  // mixed-precision Bloch apply: the shared cell blocks 1/2 |k|^2 A~ and G~
  // (binary64 n_e x n_e on the device; empty when the mesh's scaling pattern
  // differs between cells) and their BF16x3 packs for the current k
  double* d_kA = nullptr;
  double* d_kG = nullptr;
  uint16_t* kbf = nullptr;         // T~_e = H~_e + 1/2 |k|^2 A~, every cell
  uint16_t* kgbf = nullptr;        // G~, one block
  size_t kbf_bytes = 0, kgbf_bytes = 0;
  bool kpack_valid = false;
  bool scf_setup = false;          // scfb holds the load of 1 and the weights
  double scf_msum = 0.0;           // sum_j int N_j (the box volume)
  chfsi::DevBuf Db;                // density tables: M^{-1/2}, basis at Gauss points, weights
  // filter lanes (mixed precisions): column groups filtered concurrently on
  // their own streams, so one lane's assembly overlaps another's cell products
  static constexpr int kMaxLanes = 4;
  int filter_lanes = 1;
  cudaStream_t lane_stream[kMaxLanes] = {};   // lane 0 runs on `stream`
  cudaEvent_t lane_ev[kMaxLanes] = {};
  chfsi::DevBuf laneT1[kMaxLanes], laneR[kMaxLanes], laneZ[kMaxLanes], laneC[kMaxLanes], laneP[kMaxLanes];
  chfsi::DevBuf cmaxb;             // FP16x2: column maxima of the filter's blocks (3 x ncol words)
  chfsi::DevBuf pjb;               // partial projections of the cells (pj_rows x ncol)
  chfsi::DevBuf tinv;              // CholGS: L^{-1} (n x n binary64)
  cusolverDnHandle_t sol = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  double times[4] = {0, 0, 0, 0};
  // optional per-launch event timing of the filter kernels
  bool ktiming = false;
  std::vector<cudaEvent_t> kev_free;
  struct KRec {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<KRec> krec;
  double kms[3] = {0, 0, 0};       // cell products, assembly, projector kernels
  int64_t kcount[3] = {0, 0, 0};
};

namespace chfsi {
chfsi_status rayleigh_ritz_internal(chfsi_ctx* ctx, void* X, int64_t ldx, int n, chfsi_precision prec,
                                    double* evals_host, bool fp64_apply);
}  // namespace chfsi
