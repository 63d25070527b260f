// Device helpers and small kernels of the network (CUDA cores).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "net_internal.h"

namespace ppe {

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad_f(float z)
{
    float cdf = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
    float pdf = 0.3989422804014327f * __expf(-0.5f * z * z);
    return cdf + z * pdf;
}

// Apply the epilogue to one output value (pixel p = (b*H + y)*W + x,
// image-local pixel q = y*W + x, channel co).
__device__ __forceinline__ void epi_store(const Epi &e, float z, size_t p, int q, int co, int cout)
{
    if (e.zf_out) e.zf_out[p * cout + co] = z;
    if (e.z_out) e.z_out[p * cout + co] = __float2bfloat16_rn(z);
    float y = e.act ? gelu_f(z) : z;
    if (e.out1) {
        float v = e.eta1 ? y * e.eta1[q] : y;
        e.out1[p * e.cs1 + e.co1 + co] = __float2bfloat16_rn(v);
    }
    if (e.out2) {
        float v = e.eta2 ? y * e.eta2[q] : y;
        e.out2[p * e.cs2 + e.co2 + co] = __float2bfloat16_rn(v);
    }
}

}  // namespace ppe
