// Network internals shared by the network translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "internal.h"

namespace ppe {

using bf16 = __nv_bfloat16;

// One 3x3 Mesh-Conv layer.
struct ConvLayer {
    std::string name;
    int cin, cout, level;
    int64_t off_w, off_b, off_p1w, off_p1b, off_p2w, off_p2b;   // offsets into the flat FP32 params
    int64_t off_wp;                                              // offset (elements) into packed BF16 weights
    int64_t off_wt;                                              // offset into packed transposed weights (dgrad)
};

// Epilogue of a convolution: z = acc + bias; optional outputs
//   z_out[p][co]                    (pre-activation, BF16)
//   out1[p*cs1 + co1 + co] = act(z) * eta1[pixel]   (BF16)
//   out2[p*cs2 + co2 + co] = act(z) * eta2[pixel]   (BF16)
struct Epi {
    float *zf_out = nullptr;   // FP32 pre-activation [p][co] (test hook)
    bf16 *z_out = nullptr;
    bf16 *out1 = nullptr;
    int cs1 = 0, co1 = 0;
    const float *eta1 = nullptr;
    bf16 *out2 = nullptr;
    int cs2 = 0, co2 = 0;
    const float *eta2 = nullptr;
    int act = 1;   // 1: GELU, 0: identity
    // tensor-core path only: the activation 2x2-averaged (the next level's
    // pooled input, times pool_eta at the coarse pixel; H and W even) and
    // nearest-2x up-sampled (times up_eta at the fine pixel)
    bf16 *pool_out = nullptr;
    int pool_cs = 0;
    const float *pool_eta = nullptr;
    bf16 *up_out = nullptr;
    int up_cs = 0;
    const float *up_eta = nullptr;
};

// Convolution problem: NHWC BF16 input [B][H][W][cin] (already eta-weighted),
// packed weights [cout][9][cin] BF16, bias FP32 [cout] (nullable).
struct ConvArgs {
    const bf16 *in = nullptr;
    const bf16 *w = nullptr;
    const float *bias = nullptr;
    int B = 0, H = 0, W = 0, cin = 0, cout = 0;
    Epi epi;
};

ppe_status conv3x3_simt(const ConvArgs &a, cudaStream_t s);
// tcgen05 implicit-GEMM convolution (sm_103a); returns PPE_ERR_ARG when the
// shape is outside what the kernel supports.
ppe_status conv3x3_tc(const ConvArgs &a, cudaStream_t s);
bool conv3x3_tc_supported(const ConvArgs &a);
ppe_status conv3x3_tc_prepare();
// tcgen05 weight gradient dW[co][ci][9] += (dZ, X); PPE_ERR_ARG for channel
// counts the kernel does not take (then the CUDA-core kernel runs)
bool wgrad_tc_supported(int cin, int cout);
ppe_status wgrad_tc(const bf16 *dZ, const bf16 *X, int B, int H, int W, int cin, int cout, float *dW, cudaStream_t s);

}  // namespace ppe
