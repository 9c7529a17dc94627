// tcgen05 tensor-core MTTKRP passes (BF16 / TF32 in, FP32 accumulate in TMEM).
#include "mttkrp.cuh"

namespace gsp {

bool tc_supported(const MttkrpDims& d, int precision) {
  (void)d;
  (void)precision;
  return false;
}

int tc_mttkrp_xy(const void*, const void*, float*, const MttkrpDims&, int, cudaStream_t) {
  return GSP_ERR_UNSUPPORTED;
}

int tc_mttkrp_lst(const void*, const float*, const float*, float*, const MttkrpDims&, int, int,
                  cudaStream_t) {
  return GSP_ERR_UNSUPPORTED;
}

}  // namespace gsp
