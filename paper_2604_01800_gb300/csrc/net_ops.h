// Launchers of the network's CUDA-core kernels.
#pragma once

#include "net_internal.h"

namespace ppe {

// Source of the network input (1 channel).  Either a plain FP32 field
// r[b*bstride + y*pitch + x] * scale, or the current residual of a solver
// system, normalised as (r - mu) / sqrt(rho) from its device state.
struct InputSrc {
    const float *r = nullptr;
    int pitch = 0;
    size_t bstride = 0;
    float scale = 1.f;
    int nx = 0, ny = 0;
    const SysDesc *sd = nullptr;
    const SysState *st = nullptr;
};

ppe_status conv_in(const InputSrc &src, int B, int H, int W, const float *eta, const bf16 *w, const float *bias,
                   int C, const Epi &e, cudaStream_t s);
ppe_status pool2(const bf16 *in, bf16 *out, int B, int H, int W, int C, const float *eta, cudaStream_t s);
ppe_status up2(const bf16 *in, bf16 *out, int B, int H, int W, int C, const float *eta, cudaStream_t s);
ppe_status eta_layer(const float *delta, int HW, const float *w1, const float *b1, const float *w2, const float *b2,
                     int hid, int mesh, float *eta, float *phi_out, cudaStream_t s);
ppe_status sgemm(int M, int N, int K, const float *A, int lda, bool transA, const float *B, int ldb, bool transB,
                 float *C, int ldc, const float *bias, int act, bool accumulate, cudaStream_t s);
// The same on the tensor cores (kind::tf32) where the shape is one of the
// trunk's two forms (pixels as the long N or K dimension); the CUDA-core
// sgemm otherwise.  tgemm_form reports the form (1 pixel GEMM, 2 reduction
// GEMM, 0 CUDA cores); tgemm_error the device's bounded-wait flag.
int tgemm_form(int M, int N, int K, const float *A, int lda, bool transA, const float *B, int ldb, bool transB,
               const float *bias, int act);
ppe_status tgemm(int M, int N, int K, const float *A, int lda, bool transA, const float *B, int ldb, bool transB,
                 float *C, int ldc, const float *bias, int act, bool accumulate, cudaStream_t s,
                 float *scratch = nullptr, size_t scratch_floats = 0);
// Scratch (FP32 elements) that the reduction form needs for an M x N
// product; tgemm takes it from `scratch` when that is large enough, else
// from the device's stream-ordered pool.
size_t tgemm_scratch_floats(int M, int N);
int tgemm_error();
ppe_status fold_out(const bf16 *Y, const float *weff, const float *ceff, int B, int H, int W, int C, float *e,
                    int e_pitch, size_t e_bstride, int nx, int ny, cudaStream_t s);
ppe_status pack_conv_weights(const float *W, bf16 *Wp, bf16 *Wt, int cout, int cin, cudaStream_t s);

}  // namespace ppe
