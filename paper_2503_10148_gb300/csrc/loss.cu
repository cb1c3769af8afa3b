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
    if (grad) grad[i] = d > 0.0f ? inv_count : (d < 0.0f ? -inv_count : 0.0f);
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

// dL/dpred = dL/dloss * sign(pred - target) / count, dL/dloss read on the
// device (1 when absent).
__global__ void __launch_bounds__(256) k_loss_l1_grad(const float* __restrict__ pred,
                                                      const float* __restrict__ target, uint32_t count,
                                                      float inv_count, const float* __restrict__ dl_dloss,
                                                      float* __restrict__ grad) {
  const float s = dl_dloss ? *dl_dloss * inv_count : inv_count;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    const float d = pred[i] - target[i];
    grad[i] = d > 0.0f ? s : (d < 0.0f ? -s : 0.0f);
  }
}

// reg_o |tanh(raw)| + reg_s sum_j exp(log_scale_j) summed over components.
__global__ void __launch_bounds__(256) k_regularizers(const float* __restrict__ opacity_raw,
                                                      const float* __restrict__ log_scale, uint32_t n, float reg_o,
                                                      float reg_s, float* __restrict__ loss) {
  __shared__ float warp_sum[8];
  float acc = 0.0f;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float s = expf(log_scale[i]) + expf(log_scale[n + i]) + expf(log_scale[2 * (size_t)n + i]);
    acc = fmaf(reg_o, fabsf(tanhf(opacity_raw[i])), fmaf(reg_s, s, acc));
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < 8; ++w) t += warp_sum[w];
    atomicAdd(loss, t);
  }
}

}  // namespace
}  // namespace sss

extern "C" int sss_loss_l1(const float* pred, const float* target, uint32_t count, float* dL_dpred, float* loss_out,
                           sss_stream_t stream) {
  if (!pred || !target || !loss_out) return SSS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(loss_out, 0, sizeof(float), st) != cudaSuccess) return SSS_ERR_CUDA;
  if (count == 0) return SSS_OK;
  const unsigned blocks = std::min<unsigned>(sss::ceil_div(count, 256), 8u * (unsigned)sss::device_sm_count());
  sss::k_loss_l1<<<blocks, 256, 0, st>>>(pred, target, count, 1.0f / (float)count, dL_dpred, loss_out);
  SSS_LAUNCH_CHECK();
  return SSS_OK;
}

extern "C" int sss_loss_l1_grad(const float* pred, const float* target, uint32_t count, const float* dL_dloss,
                                float* dL_dpred, sss_stream_t stream) {
  if (!pred || !target || !dL_dpred) return SSS_ERR_INVALID_ARG;
  if (count == 0) return SSS_OK;
  const unsigned blocks = std::min<unsigned>(sss::ceil_div(count, 256), 8u * (unsigned)sss::device_sm_count());
  sss::k_loss_l1_grad<<<blocks, 256, 0, (cudaStream_t)stream>>>(pred, target, count, 1.0f / (float)count, dL_dloss,
                                                               dL_dpred);
  SSS_LAUNCH_CHECK();
  return SSS_OK;
}

extern "C" int sss_regularizers(const sss_params* params, float reg_opacity, float reg_scale, float* loss_out,
                                sss_stream_t stream) {
  if (!params || !loss_out || params->n < 0) return SSS_ERR_INVALID_ARG;
  if (params->n > 0 && (!params->opacity_raw || !params->log_scale)) return SSS_ERR_INVALID_ARG;
  if (!(reg_opacity >= 0.0f) || !(reg_scale >= 0.0f)) return SSS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(loss_out, 0, sizeof(float), st) != cudaSuccess) return SSS_ERR_CUDA;
  if (params->n == 0) return SSS_OK;
  const unsigned blocks = std::min<unsigned>(sss::ceil_div((size_t)params->n, 256), 8u * (unsigned)sss::device_sm_count());
  sss::k_regularizers<<<blocks, 256, 0, st>>>(params->opacity_raw, params->log_scale, (uint32_t)params->n,
                                              reg_opacity, reg_scale, loss_out);
  SSS_LAUNCH_CHECK();
  return SSS_OK;
}
