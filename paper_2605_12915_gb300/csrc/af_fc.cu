// af_fc.cu -- launches of the foot-centred point update (af_fc.cuh), in a
// translation unit of their own so that the library's units compile in parallel.
#include "af_fc.cuh"

namespace af {

cudaError_t launch_fc_points(const StepArgs<double>& a, dim3 grd, dim3 blk, cudaStream_t s) {
  k_points_fc<0><<<grd, blk, 0, s>>>(a);
  k_points_fc<1><<<grd, blk, 0, s>>>(a);
  k_points_fc<2><<<grd, blk, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace af
