// CUDA-core kernels of the network: the direct 3x3 convolution (reference
// path and 1-channel input layer), pooling, up-sampling, Mesh-Conv weights,
// a small FP32 GEMM for the trunk and head, the DeepONet fold, weight packing.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "net_kernels.cuh"
#include "net_ops.h"

namespace ppe {

namespace {

constexpr int ST_H = 8, ST_W = 16, ST_CO = 32, ST_CI = 16;

__global__ void __launch_bounds__(256) conv3x3_simt_kernel(ConvArgs a)
{
    __shared__ float xs[ST_CI][ST_H + 2][ST_W + 2];
    __shared__ float ws[ST_CI][9][ST_CO];
    const int tiles_w = (a.W + ST_W - 1) / ST_W;
    const int tile = blockIdx.x, b = blockIdx.z, co0 = blockIdx.y * ST_CO;
    const int ty0 = (tile / tiles_w) * ST_H, tx0 = (tile % tiles_w) * ST_W;
    const int tid = threadIdx.x, q = tid & 31, cq = tid >> 5;
    const int pr = q >> 2, pc = (q & 3) * 4;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int ci0 = 0; ci0 < a.cin; ci0 += ST_CI) {
        __syncthreads();
        for (int k = tid; k < ST_CI * (ST_H + 2) * (ST_W + 2); k += 256) {
            int ci = k % ST_CI, pix = k / ST_CI;
            int yy = pix / (ST_W + 2), xx = pix % (ST_W + 2);
            int y = ty0 - 1 + yy, x = tx0 - 1 + xx;
            float v = 0.f;
            if (y >= 0 && y < a.H && x >= 0 && x < a.W && ci0 + ci < a.cin)
                v = __bfloat162float(a.in[(((size_t)b * a.H + y) * a.W + x) * a.cin + ci0 + ci]);
            xs[ci][yy][xx] = v;
        }
        for (int k = tid; k < ST_CI * 9 * ST_CO; k += 256) {
            int ci = k % ST_CI, rest = k / ST_CI, tap = rest % 9, co = rest / 9;
            float v = 0.f;
            if (co0 + co < a.cout && ci0 + ci < a.cin)
                v = __bfloat162float(a.w[((size_t)(co0 + co) * 9 + tap) * a.cin + ci0 + ci]);
            ws[ci][tap][co] = v;
        }
        __syncthreads();
        for (int ci = 0; ci < ST_CI; ++ci) {
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                const int ky = tap / 3, kx = tap % 3;
                float wv[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) wv[c] = ws[ci][tap][cq * 4 + c];
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    float xv = xs[ci][pr + ky][pc + p + kx];
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[p][c] = fmaf(xv, wv[c], acc[p][c]);
                }
            }
        }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        int y = ty0 + pr, x = tx0 + pc + p;
        if (y >= a.H || x >= a.W) continue;
        size_t pg = ((size_t)b * a.H + y) * a.W + x;
        int ql = y * a.W + x;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int co = co0 + cq * 4 + c;
            if (co >= a.cout) continue;
            float z = acc[p][c] + (a.bias ? a.bias[co] : 0.f);
            epi_store(a.epi, z, pg, ql, co, a.cout);
        }
    }
}

__device__ __forceinline__ float input_at(const InputSrc &s, int b, int y, int x)
{
    if (y < 0 || x < 0 || y >= s.ny || x >= s.nx) return 0.f;
    if (s.st) {
        const SysState &st = *s.st;
        const SysDesc &sd = *s.sd;
        float scale = st.rho > 0.0 ? (float)(1.0 / sqrt(st.rho)) : 0.f;
        size_t k = (size_t)y * sd.pitch + x;
        double v = sd.precision == PPE_PREC_FP64 ? ((const double *)sd.r[st.cur])[k]
                                                 : (double)((const float *)sd.r[st.cur])[k];
        return (float)(v - st.mu) * scale;
    }
    return s.r[(size_t)b * s.bstride + (size_t)y * s.pitch + x] * s.scale;
}

// First layer (1 input channel): eta-weighted input, 3x3 conv, epilogue.
// Scalar form, for widths or destinations the staged form does not take.
__global__ void conv_in_kernel(InputSrc src, int B, int H, int W, const float *__restrict__ eta,
                               const bf16 *__restrict__ w, const float *__restrict__ bias, int C, Epi e)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y;
    int b = blockIdx.z;
    if (x >= W) return;
    float v[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
        float s = 0.f;
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
            s = input_at(src, b, yy, xx);
            if (eta) s *= eta[yy * W + xx];
        }
        v[t] = s;
    }
    size_t pg = ((size_t)b * H + y) * W + x;
    int q = y * W + x;
    for (int co = 0; co < C; ++co) {
        float z = bias ? bias[co] : 0.f;
#pragma unroll
        for (int t = 0; t < 9; ++t) z = fmaf(__bfloat162float(w[co * 9 + t]), v[t], z);
        epi_store(e, z, pg, q, co, C);
    }
}

// Staged form: a block computes CI_PX pixels of one row, 32 output channels
// at a time into registers; each BF16 destination is written through a
// shared-memory tile, so that consecutive lanes store consecutive 16-byte
// pieces of the NHWC rows.
constexpr int CI_PX = 128;
constexpr int CI_CH = 32;

__device__ __forceinline__ void ci_flush(const bf16 (*tile)[CI_CH + 8], bf16 *dst, int cs, int co, int np)
{
    // dst: pixel 0 of this block's run, channel 0 of the chunk; np valid pixels
    for (int k = threadIdx.x; k < np * (CI_CH / 8); k += blockDim.x) {
        const int px = k / (CI_CH / 8), part = k % (CI_CH / 8);
        *reinterpret_cast<uint4 *>(dst + (size_t)px * cs + co + 8 * part) =
            *reinterpret_cast<const uint4 *>(&tile[px][8 * part]);
    }
}

__global__ void __launch_bounds__(CI_PX) conv_in_staged_kernel(InputSrc src, int B, int H, int W,
                                                               const float *__restrict__ eta,
                                                               const bf16 *__restrict__ w,
                                                               const float *__restrict__ bias, int C, Epi e)
{
    // the next kernel (a tensor-core convolution launched as a programmatic
    // dependent) may start its set-up now; it waits for this grid's results
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __shared__ float ws[CI_CH][9];
    __shared__ float bs[CI_CH];
    __shared__ __align__(16) bf16 tile[CI_PX][CI_CH + 8];      // padded rows: conflict-free column writes
    // the solver state's residual, read once per block instead of per tap
    __shared__ const void *sr;
    __shared__ int sfp64, spitch;
    __shared__ double smu;
    __shared__ float sscale;
    if (threadIdx.x == 0 && src.st) {
        const SysState &st = *src.st;
        const SysDesc &sd = *src.sd;
        sr = sd.r[st.cur];
        sfp64 = sd.precision == PPE_PREC_FP64;
        spitch = sd.pitch;
        smu = st.mu;
        sscale = st.rho > 0.0 ? (float)(1.0 / sqrt(st.rho)) : 0.f;
    }
    __syncthreads();
    const int x0 = blockIdx.x * CI_PX, y = blockIdx.y, b = blockIdx.z;
    const int x = x0 + threadIdx.x;
    const int np = min(CI_PX, W - x0);
    float v[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
        float s = 0.f;
        if (x < W && yy >= 0 && yy < H && xx >= 0 && xx < W && yy < src.ny && xx < src.nx) {
            if (src.st) {
                const size_t k = (size_t)yy * spitch + xx;
                const double r = sfp64 ? ((const double *)sr)[k] : (double)((const float *)sr)[k];
                s = (float)(r - smu) * sscale;
            } else {
                s = src.r[(size_t)b * src.bstride + (size_t)yy * src.pitch + xx] * src.scale;
            }
            if (eta) s *= eta[yy * W + xx];
        }
        v[t] = s;
    }
    const size_t p0 = ((size_t)b * H + y) * W + x0;
    const int q = y * W + min(x, W - 1);
    const float s1 = (e.eta1 && x < W) ? e.eta1[q] : 1.f;
    const float s2 = (e.eta2 && x < W) ? e.eta2[q] : 1.f;
    for (int c0 = 0; c0 < C; c0 += CI_CH) {
        __syncthreads();
        for (int k = threadIdx.x; k < CI_CH * 9; k += blockDim.x)
            ws[k / 9][k % 9] = __bfloat162float(w[(c0 + k / 9) * 9 + k % 9]);
        if (threadIdx.x < CI_CH) bs[threadIdx.x] = bias ? bias[c0 + threadIdx.x] : 0.f;
        __syncthreads();
        float z[CI_CH];
#pragma unroll
        for (int c = 0; c < CI_CH; ++c) {
            float a = bs[c];
#pragma unroll
            for (int t = 0; t < 9; ++t) a = fmaf(ws[c][t], v[t], a);
            z[c] = a;
        }
        if (e.zf_out && x < W)
            for (int c = 0; c < CI_CH; ++c) e.zf_out[(p0 + threadIdx.x) * C + c0 + c] = z[c];
        if (e.z_out) {
#pragma unroll
            for (int c = 0; c < CI_CH; ++c) tile[threadIdx.x][c] = __float2bfloat16_rn(z[c]);
            __syncthreads();
            ci_flush(tile, e.z_out + p0 * C, C, c0, np);
            __syncthreads();
        }
        if (e.act) {
#pragma unroll
            for (int c = 0; c < CI_CH; ++c) z[c] = gelu_f(z[c]);
        }
        if (e.out1) {
#pragma unroll
            for (int c = 0; c < CI_CH; ++c) tile[threadIdx.x][c] = __float2bfloat16_rn(z[c] * s1);
            __syncthreads();
            ci_flush(tile, e.out1 + p0 * e.cs1 + e.co1, e.cs1, c0, np);
            __syncthreads();
        }
        if (e.out2) {
#pragma unroll
            for (int c = 0; c < CI_CH; ++c) tile[threadIdx.x][c] = __float2bfloat16_rn(z[c] * s2);
            __syncthreads();
            ci_flush(tile, e.out2 + p0 * e.cs2 + e.co2, e.cs2, c0, np);
        }
    }
}

// out[b][y][x][c] = 0.25 * sum of the 2x2 children * eta[y][x]
__global__ void pool2_kernel(const bf16 *__restrict__ in, bf16 *__restrict__ out, int B, int H, int W, int C,
                             const float *__restrict__ eta)
{
    const int cv = C / 8;
    size_t n = (size_t)B * H * W * cv;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        int c8 = k % cv;
        size_t pix = k / cv;
        int x = pix % W, y = (pix / W) % H, b = pix / ((size_t)W * H);
        float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            int yy = 2 * y + (t >> 1), xx = 2 * x + (t & 1);
            const uint4 raw = *reinterpret_cast<const uint4 *>(in + ((((size_t)b * 2 * H + yy) * 2 * W + xx) * C + c8 * 8));
            const bf16 *h = reinterpret_cast<const bf16 *>(&raw);
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[i] += __bfloat162float(h[i]);
        }
        float s = 0.25f * (eta ? eta[y * W + x] : 1.f);
        uint4 o;
        bf16 *oh = reinterpret_cast<bf16 *>(&o);
#pragma unroll
        for (int i = 0; i < 8; ++i) oh[i] = __float2bfloat16_rn(acc[i] * s);
        *reinterpret_cast<uint4 *>(out + pix * C + c8 * 8) = o;
    }
}

// out[b][y][x][c] = in[b][y/2][x/2][c] * eta[y][x]   (H, W: output dims)
__global__ void up2_kernel(const bf16 *__restrict__ in, bf16 *__restrict__ out, int B, int H, int W, int C,
                           const float *__restrict__ eta)
{
    const int cv = C / 8;
    size_t n = (size_t)B * H * W * cv;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        int c8 = k % cv;
        size_t pix = k / cv;
        int x = pix % W, y = (pix / W) % H, b = pix / ((size_t)W * H);
        const uint4 raw =
            *reinterpret_cast<const uint4 *>(in + ((((size_t)b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c8 * 8));
        const bf16 *h = reinterpret_cast<const bf16 *>(&raw);
        float s = eta ? eta[y * W + x] : 1.f;
        uint4 o;
        bf16 *oh = reinterpret_cast<bf16 *>(&o);
#pragma unroll
        for (int i = 0; i < 8; ++i) oh[i] = __float2bfloat16_rn(__bfloat162float(h[i]) * s);
        *reinterpret_cast<uint4 *>(out + pix * C + c8 * 8) = o;
    }
}

// eta[p] = exp(-Phi(Delta[:, p])^2), Phi = w2 . tanh(W1 Delta + b1) + b2
__global__ void eta_kernel(const float *__restrict__ delta, int HW, const float *__restrict__ w1,
                           const float *__restrict__ b1, const float *__restrict__ w2, const float *__restrict__ b2,
                           int hid, int mesh, float *__restrict__ eta, float *__restrict__ phi_out)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= HW) return;
    if (!mesh) {
        eta[p] = 1.f;
        if (phi_out) phi_out[p] = 0.f;
        return;
    }
    float d0 = delta[p], d1 = delta[HW + p], d2 = delta[2 * HW + p], d3 = delta[3 * HW + p];
    float phi = b2[0];
    for (int k = 0; k < hid; ++k) {
        float z = b1[k] + w1[4 * k] * d0 + w1[4 * k + 1] * d1 + w1[4 * k + 2] * d2 + w1[4 * k + 3] * d3;
        phi += w2[k] * tanhf(z);
    }
    eta[p] = __expf(-phi * phi);
    if (phi_out) phi_out[p] = phi;
}

// C[m][n] = act( sum_k A(m,k) B(k,n) + bias[m] ) (+ C if accumulate)
// A(m,k) = transA ? A[k*lda + m] : A[m*lda + k];  B(k,n) = transB ? B[n*ldb + k] : B[k*ldb + n]
constexpr int GT = 64, GK = 16;
__global__ void __launch_bounds__(256) sgemm_kernel(int M, int N, int K, const float *__restrict__ A, int lda,
                                                    int transA, const float *__restrict__ Bm, int ldb, int transB,
                                                    float *__restrict__ C, int ldc, const float *__restrict__ bias,
                                                    int act, int accumulate, int kchunk)
{
    __shared__ float As[GK][GT + 1];
    __shared__ float Bs[GK][GT + 1];
    const int tid = threadIdx.x, tr = tid / 16, tc = tid % 16;
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    // split-K: block z sums k in [kb, ke) and adds its share atomically
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    const bool split = gridDim.z > 1;
    float acc[4][4] = {};
    for (int k0 = kb; k0 < ke; k0 += GK) {
        for (int t = tid; t < GT * GK; t += 256) {
            int mm = t % GT, kk = t / GT;
            int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < ke) ? (transA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k]) : 0.f;
            int nn = t % GT;
            int n = n0 + nn;
            Bs[kk][nn] = (n < N && k < ke) ? (transB ? Bm[(size_t)n * ldb + k] : Bm[(size_t)k * ldb + n]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][tr * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tc * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int m = m0 + tr * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int n = n0 + tc * 4 + j;
            if (n >= N) continue;
            float *c = C + (size_t)m * ldc + n;
            if (split) {                       // identity epilogue, C accumulated
                atomicAdd(c, acc[i][j] + ((bias && blockIdx.z == 0) ? bias[m] : 0.f));
                continue;
            }
            float v = acc[i][j] + (bias ? bias[m] : 0.f);
            if (act == 1) v = tanhf(v);
            *c = accumulate ? *c + v : v;
        }
    }
}

// e[b][y][x] = sum_c Y[b][y][x][c] * weff[c][y*W+x] + ceff[y*W+x]   (cropped to nx x ny)
__global__ void fold_kernel(const bf16 *__restrict__ Y, const float *__restrict__ weff, const float *__restrict__ ceff,
                            int B, int H, int W, int C, float *__restrict__ e, int e_pitch, size_t e_bstride, int nx,
                            int ny)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y, b = blockIdx.z;
    if (x >= nx || y >= ny) return;
    int q = y * W + x;
    const bf16 *yp = Y + (((size_t)b * H + y) * W + x) * C;
    float s = ceff[q];
    size_t HW = (size_t)H * W;
    if ((C & 7) == 0) {
        // the pixel's channels as 16-byte pieces (rows are 16-byte aligned)
        for (int c = 0; c < C; c += 8) {
            const uint4 raw = *reinterpret_cast<const uint4 *>(yp + c);
            const bf16 *h = reinterpret_cast<const bf16 *>(&raw);
#pragma unroll
            for (int i = 0; i < 8; ++i) s = fmaf(__bfloat162float(h[i]), weff[(c + i) * HW + q], s);
        }
    } else {
        for (int c = 0; c < C; ++c) s = fmaf(__bfloat162float(yp[c]), weff[c * HW + q], s);
    }
    e[b * e_bstride + (size_t)y * e_pitch + x] = s;
}

// Wp[co][tap][ci] = W[co][ci][tap] (BF16)
__global__ void pack_w_kernel(const float *__restrict__ W, bf16 *__restrict__ Wp, int cout, int cin)
{
    size_t n = (size_t)cout * cin * 9;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        int ci = k % cin;
        int tap = (k / cin) % 9;
        int co = k / (9 * (size_t)cin);
        Wp[k] = __float2bfloat16_rn(W[((size_t)co * cin + ci) * 9 + tap]);
    }
}

// Wt[ci][tap][co] = W[co][ci][8 - tap]  (transposed, flipped: the data-gradient convolution)
__global__ void pack_wt_kernel(const float *__restrict__ W, bf16 *__restrict__ Wt, int cout, int cin)
{
    size_t n = (size_t)cout * cin * 9;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        int co = k % cout;
        int tap = (k / cout) % 9;
        int ci = k / (9 * (size_t)cout);
        Wt[k] = __float2bfloat16_rn(W[((size_t)co * cin + ci) * 9 + (8 - tap)]);
    }
}

inline unsigned grid1d(size_t n, int bs = 256)
{
    size_t g = (n + bs - 1) / bs;
    return (unsigned)(g > 65535u * 16u ? 65535u * 16u : (g == 0 ? 1 : g));
}

}  // namespace

ppe_status conv3x3_simt(const ConvArgs &a, cudaStream_t s)
{
    if (a.cin % 1 != 0 || a.B < 1) return PPE_ERR_ARG;
    int tiles = ((a.H + ST_H - 1) / ST_H) * ((a.W + ST_W - 1) / ST_W);
    dim3 grid(tiles, (a.cout + ST_CO - 1) / ST_CO, a.B);
    conv3x3_simt_kernel<<<grid, 256, 0, s>>>(a);
    PPE_CUDA_TRY(cudaGetLastError());
    return PPE_OK;
}

ppe_status conv_in(const InputSrc &src, int B, int H, int W, const float *eta, const bf16 *w, const float *bias, int C,
                   const Epi &e, cudaStream_t s)
{
    dim3 grid((W + 127) / 128, H, B);
    // the staged form needs whole 32-channel chunks and 16-byte aligned
    // destination rows and offsets
    auto aligned = [](const void *p, int cs, int co) {
        return ((uintptr_t)p & 15) == 0 && cs % 8 == 0 && co % 8 == 0;
    };
    const bool staged = C % CI_CH == 0 && (!e.z_out || aligned(e.z_out, C, 0)) &&
                        (!e.out1 || aligned(e.out1, e.cs1, e.co1)) && (!e.out2 || aligned(e.out2, e.cs2, e.co2));
    if (staged)
        conv_in_staged_kernel<<<grid, CI_PX, 0, s>>>(src, B, H, W, eta, w, bias, C, e);
    else
        conv_in_kernel<<<grid, 128, 0, s>>>(src, B, H, W, eta, w, bias, C, e);
    PPE_CUDA_TRY(cudaGetLastError());
    return PPE_OK;
}

ppe_status pool2(const bf16 *in, bf16 *out, int B, int H, int W, int C, const float *eta, cudaStream_t s)
{
    size_t n = (size_t)B * H * W * (C / 8);
    pool2_kernel<<<grid1d(n), 256, 0, s>>>(in, out, B, H, W, C, eta);
    PPE_CUDA_TRY(cudaGetLastError());
    return PPE_OK;
}

ppe_status up2(const bf16 *in, bf16 *out, int B, int H, int W, int C, const float *eta, cudaStream_t s)
{
    size_t n = (size_t)B * H * W * (C / 8);
    up2_kernel<<<grid1d(n), 256, 0, s>>>(in, out, B, H, W, C, eta);
    PPE_CUDA_TRY(cudaGetLastError());
    return PPE_OK;
}

ppe_status eta_layer(const float *delta, int HW, const float *w1, const float *b1, const float *w2, const float *b2,
                     int hid, int mesh, float *eta, float *phi_out, cudaStream_t s)
{
    eta_kernel<<<(HW + 255) / 256, 256, 0, s>>>(delta, HW, w1, b1, w2, b2, hid, mesh, eta, phi_out);
    PPE_CUDA_TRY(cudaGetLastError());
    return PPE_OK;
}

ppe_status sgemm(int M, int N, int K, const float *A, int lda, bool transA, const float *B, int ldb, bool transB,
                 float *C, int ldc, const float *bias, int act, bool accumulate, cudaStream_t s)
{
    dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT, 1);
    int kchunk = K;
    const int tiles = grid.x * grid.y;
    if (act == 0 && K >= 4096 && tiles < 296) {
        // long reductions over pixels with a small output: split K across blocks
        int splits = std::min((K + 1023) / 1024, std::max(1, 592 / tiles));
        kchunk = (K + splits - 1) / splits;
        kchunk = (kchunk + GK - 1) / GK * GK;
        grid.z = (K + kchunk - 1) / kchunk;
        if (grid.z > 1 && !accumulate) {      // the blocks add their shares into a cleared C
            cudaError_t e = ldc == N ? cudaMemsetAsync(C, 0, (size_t)M * N * sizeof(float), s)
                                     : cudaMemset2DAsync(C, (size_t)ldc * sizeof(float), 0, (size_t)N * sizeof(float),
                                                         M, s);
            if (e != cudaSuccess) return cuda_status(e, "sgemm split-K clear");
        }
    }
    sgemm_kernel<<<grid, 256, 0, s>>>(M, N, K, A, lda, transA, B, ldb, transB, C, ldc, bias, act, accumulate, kchunk);
    PPE_CUDA_TRY(cudaGetLastError());
    return PPE_OK;
}

ppe_status fold_out(const bf16 *Y, const float *weff, const float *ceff, int B, int H, int W, int C, float *e,
                    int e_pitch, size_t e_bstride, int nx, int ny, cudaStream_t s)
{
    dim3 grid((nx + 127) / 128, ny, B);
    fold_kernel<<<grid, 128, 0, s>>>(Y, weff, ceff, B, H, W, C, e, e_pitch, e_bstride, nx, ny);
    PPE_CUDA_TRY(cudaGetLastError());
    return PPE_OK;
}

ppe_status pack_conv_weights(const float *W, bf16 *Wp, bf16 *Wt, int cout, int cin, cudaStream_t s)
{
    size_t n = (size_t)cout * cin * 9;
    pack_w_kernel<<<grid1d(n), 256, 0, s>>>(W, Wp, cout, cin);
    if (Wt) pack_wt_kernel<<<grid1d(n), 256, 0, s>>>(W, Wt, cout, cin);
    PPE_CUDA_TRY(cudaGetLastError());
    return PPE_OK;
}

}  // namespace ppe
