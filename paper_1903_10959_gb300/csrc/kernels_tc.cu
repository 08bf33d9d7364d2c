// Mixed-precision (tcgen05) kernels -- placeholder until the tensor-core path lands.
#include "internal.h"
#include "tc.h"

namespace chfsi {

cudaError_t tc_build(TcCellData& d, const std::vector<double>&, int64_t, int, cudaStream_t, int64_t*) {
  d = TcCellData();
  return cudaSuccess;
}
void tc_free(TcCellData& d) { d = TcCellData(); }
cudaError_t tc_cell_launch(const TcCellData&, const TcCellArgs&, cudaStream_t) { return cudaErrorNotSupported; }
size_t tc_gram_partial_bytes(int64_t, int, int) { return 16; }
cudaError_t tc_gram_mixed(const float*, int64_t, const float*, int64_t, int64_t, int, int, double*, int64_t,
                          int, int, int, void*, size_t, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t tc_tallgemm_mixed(const float*, int64_t, const double*, int64_t, int64_t, int, int, float*,
                              int64_t, int, int, int, int, void*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t tc_nl_project(const int64_t*, const int32_t*, const float*, int, const float*, int64_t, int,
                          float*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t tc_nl_expand(const int64_t*, const int32_t*, const float*, int64_t, const float*, int, float*,
                         int64_t, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace chfsi
