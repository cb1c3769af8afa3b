// L1 term of the training loss (Sec. 3.4): value and dL/dC in one pass.
#include <algorithm>

#include "common.cuh"

namespace sss {
namespace {

__global__ void __launch_bounds__(256) k_loss_l1(const float* __restrict__ pred, const float* __restrict__ target,
                                                 uint32_t count, float inv_count, float* __restrict__ grad,
                                                 float* __restrict__ loss) {
  __shared__ float warp_sum[8];
  float acc = 0.0f;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    const float d = pred[i] - target[i];
    acc += fabsf(d);
    grad[i] = d > 0.0f ? inv_count : (d < 0.0f ? -inv_count : 0.0f);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < 8; ++w) t += warp_sum[w];
    atomicAdd(loss, t * inv_count);
  }
}

}  // namespace
}  // namespace sss

extern "C" int sss_loss_l1(const float* pred, const float* target, uint32_t count, float* dL_dpred, float* loss_out,
                           sss_stream_t stream) {
  if (!pred || !target || !dL_dpred || !loss_out) return SSS_ERR_INVALID_ARG;
  if (count == 0) return SSS_OK;
  const unsigned blocks = std::min<unsigned>(sss::ceil_div(count, 256), 8 * sss::kNumSMs);
  sss::k_loss_l1<<<blocks, 256, 0, (cudaStream_t)stream>>>(pred, target, count, 1.0f / (float)count, dL_dpred,
                                                          loss_out);
  SSS_LAUNCH_CHECK();
  return SSS_OK;
}
