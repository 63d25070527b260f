// Training of the DeepONet on the GPU (Sec. 2.4): the unsupervised loss of
// Eq. 18 through the volume-scaled PPE operator, hand-written backward
// kernels for every forward step, and the SAM + Adam update with cosine
// learning-rate decay.
//
// Backward of one Mesh-Conv layer Y = gelu(Z), Z = conv(eta * X) + b:
//   dZ = dY * gelu'(Z);  db = sum dZ;  dW = sum dZ (x) (eta X) shifted;
//   d(eta X) = conv of dZ with the transposed, flipped kernel (the forward
//   convolution kernel run on repacked weights);  dX = eta d(eta X);
//   d eta = sum_c X d(eta X) = sum_c (eta X) d(eta X) / eta;
//   eta = exp(-Phi^2):  dPhi = -2 Phi eta d eta, then the weight network.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "net_iface.h"
#include "net_impl.h"
#include "net_kernels.cuh"
#include "net_ops.h"

namespace ppe {

namespace {

unsigned g1d(size_t n, int bs = 256)
{
    size_t g = (n + bs - 1) / bs;
    if (g < 1) g = 1;
    if (g > 16384) g = 16384;
    return (unsigned)g;
}

// y = scale * A x for `batch` unpitched FP32 fields [ny][nx]
__global__ void apply_f32_kernel(const float *__restrict__ x, float *__restrict__ y, int nx, int ny, int batch,
                                 const float *__restrict__ dx, const float *__restrict__ dy,
                                 const float *__restrict__ fx, const float *__restrict__ fy, float scale)
{
    const size_t N = (size_t)nx * ny;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < N * batch; k += (size_t)gridDim.x * blockDim.x) {
        size_t c = k % N;
        int i = c % nx, j = c / nx;
        float v = x[k];
        float xe = i + 1 < nx ? x[k + 1] : 0.f, xw = i > 0 ? x[k - 1] : 0.f;
        float xn = j + 1 < ny ? x[k + nx] : 0.f, xs = j > 0 ? x[k - nx] : 0.f;
        float ax = fx[i + 1] * (v - xe) + fx[i] * (v - xw);
        float ay = fy[j + 1] * (v - xn) + fy[j] * (v - xs);
        y[k] = scale * (dy[j] * ax + dx[i] * ay);
    }
}

// res = R - Ae;  acc += sum res^2  (FP64)
__global__ void residual_kernel(const float *__restrict__ R, const float *__restrict__ Ae, float *__restrict__ res,
                                size_t n, double *acc)
{
    double s = 0.0;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        float r = R[k] - Ae[k];
        res[k] = r;
        s += (double)r * r;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        atomicAdd(acc, t);
    }
}

// Backward of e = sum_c U0_c weff_c + ceff (cropped to nx x ny).
__global__ void fold_bwd_kernel(const float *__restrict__ de, const bf16 *__restrict__ U0,
                                const float *__restrict__ weff, int B, int H, int W, int C, int nx, int ny,
                                float *__restrict__ dU0, float *__restrict__ dweff, float *__restrict__ dceff)
{
    const size_t HW = (size_t)H * W;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < HW; q += (size_t)gridDim.x * blockDim.x) {
        int x = q % W, y = q / W;
        bool in = x < nx && y < ny;
        float dc = 0.f;
        for (int c = 0; c < C; ++c) {
            float w = weff[c * HW + q], acc = 0.f;
            for (int b = 0; b < B; ++b) {
                float d = in ? de[((size_t)b * ny + y) * nx + x] : 0.f;
                size_t p = (size_t)b * HW + q;
                dU0[p * C + c] = d * w;
                acc += d * __bfloat162float(U0[p * C + c]);
            }
            dweff[c * HW + q] = acc;
        }
        for (int b = 0; b < B; ++b) dc += in ? de[((size_t)b * ny + y) * nx + x] : 0.f;
        dceff[q] = dc;
    }
}

// dZ = dY * gelu'(Z) (BF16); db[c] += sum over pixels.  The block size is a
// multiple of C (C <= 256), so that element k of the grid-stride loop always
// has channel threadIdx.x % C in a thread.
__global__ void act_bwd_kernel(const float *__restrict__ dY, const bf16 *__restrict__ Z, bf16 *__restrict__ dZ,
                               size_t n, int C, float *__restrict__ db)
{
    __shared__ float red[256];
    float acc = 0.f;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        float g = dY[k] * gelu_grad_f(__bfloat162float(Z[k]));
        dZ[k] = __float2bfloat16_rn(g);
        acc += g;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    if ((int)threadIdx.x < C) {
        // threads t = c, c + C, ... of the block all summed channel c
        float s = 0.f;
        for (int t = threadIdx.x; t < (int)blockDim.x; t += C) s += red[t];
        atomicAdd(&db[threadIdx.x], s);
    }
}

void act_bwd(const float *dY, const bf16 *Z, bf16 *dZ, size_t n, int C, float *db, cudaStream_t s)
{
    const int bs = (256 / C) * C;          // a multiple of C
    // a grid-stride loop over at most 1024 blocks: each block adds its channel
    // sums once, so the bias gradient's atomics stay few
    act_bwd_kernel<<<std::min(1024u, g1d(n, bs)), bs, 0, s>>>(dY, Z, dZ, n, C, db);
}

// dW[co][ci][tap] += sum_p dZ[p][co] * X[p + tap][ci]  (X: the layer's eta-weighted input)
//
// A block forms a (32 NCO) Cout x 32 Cin x 9-tap slab over its share of
// 8 x 16 pixel tiles; a thread owns NCO output channels (lane, lane + 32, ...)
// and four input channels, so every input value it loads feeds 9 NCO
// products per tap group.  The next tile's raw BF16 rows of dZ and X (16-byte
// pieces, zero-filled outside the image) are copied by cp.async while the
// current tile is computed, then widened to FP32 in shared memory.  Needs Cin
// and Cout multiples of 8.
constexpr int WG_H = 8, WG_W = 16, WG_P = WG_H * WG_W, WG_XP = (WG_H + 2) * (WG_W + 2);
template <int NCO> constexpr size_t wg_smem()
{
    return sizeof(float) * WG_P * (32 * NCO + 1) + sizeof(float) * WG_XP * 32 + sizeof(bf16) * (WG_P * 32 * NCO + WG_XP * 32);
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}

template <int NCO>
__global__ void __launch_bounds__(256) wgrad_kernel(const bf16 *__restrict__ dZ, const bf16 *__restrict__ X, int B,
                                                    int H, int W, int cin, int cout, float *__restrict__ dW,
                                                    int tiles_per_block)
{
    constexpr int NC = 32 * NCO;           // output channels of the block
    extern __shared__ __align__(16) unsigned char wg_smem[];
    float(*xs)[32] = reinterpret_cast<float(*)[32]>(wg_smem);                                   // [WG_XP][32]
    bf16(*xr)[32] = reinterpret_cast<bf16(*)[32]>(wg_smem + sizeof(float) * WG_XP * 32);      // [WG_XP][32]
    bf16(*dzr)[NC] = reinterpret_cast<bf16(*)[NC]>(wg_smem + sizeof(float) * WG_XP * 32 + sizeof(bf16) * WG_XP * 32);
    float(*dzs)[NC + 1] = reinterpret_cast<float(*)[NC + 1]>(wg_smem + sizeof(float) * WG_XP * 32 +
                                                             sizeof(bf16) * (WG_XP * 32 + WG_P * NC));   // [WG_P][NC+1]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int co0 = blockIdx.x * NC, ci0 = blockIdx.y * 32;
    const int tw = (W + WG_W - 1) / WG_W, th = (H + WG_H - 1) / WG_H;
    const long total = (long)B * tw * th;
    float acc[NCO][4][9];
#pragma unroll
    for (int u = 0; u < NCO; ++u)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int t = 0; t < 9; ++t) acc[u][j][t] = 0.f;
    const long t0 = (long)blockIdx.z * tiles_per_block;
    const long t1 = min(total, t0 + tiles_per_block);
    auto issue = [&](long tile) {
        const int b = tile / (tw * th), r = tile % (tw * th);
        const int y0 = (r / tw) * WG_H, x0 = (r % tw) * WG_W;
        for (int k = threadIdx.x; k < WG_P * 4 * NCO; k += 256) {
            const int q = k % (4 * NCO), p = k / (4 * NCO);
            const int y = y0 + p / WG_W, x = x0 + p % WG_W;
            const bool v = y < H && x < W && co0 + 8 * q < cout;
            cp_async16(&dzr[p][8 * q], v ? dZ + (((size_t)b * H + y) * W + x) * cout + co0 + 8 * q : dZ, v);
        }
        for (int k = threadIdx.x; k < WG_XP * 4; k += 256) {
            const int q = k & 3, p = k >> 2;
            const int y = y0 - 1 + p / (WG_W + 2), x = x0 - 1 + p % (WG_W + 2);
            const bool v = y >= 0 && y < H && x >= 0 && x < W && ci0 + 8 * q < cin;
            cp_async16(&xr[p][8 * q], v ? X + (((size_t)b * H + y) * W + x) * cin + ci0 + 8 * q : X, v);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if (t0 < t1) issue(t0);
    for (long tile = t0; tile < t1; ++tile) {
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();          // this tile's rows from every thread; the previous tile's products done
        for (int k = threadIdx.x; k < WG_P * 4 * NCO; k += 256) {
            const int q = k % (4 * NCO), p = k / (4 * NCO);
            const uint4 raw = *reinterpret_cast<const uint4 *>(&dzr[p][8 * q]);
            const bf16 *h = reinterpret_cast<const bf16 *>(&raw);
#pragma unroll
            for (int i = 0; i < 8; ++i) dzs[p][8 * q + i] = __bfloat162float(h[i]);
        }
        for (int k = threadIdx.x; k < WG_XP * 4; k += 256) {
            const int q = k & 3, p = k >> 2;
            const uint4 raw = *reinterpret_cast<const uint4 *>(&xr[p][8 * q]);
            const bf16 *h = reinterpret_cast<const bf16 *>(&raw);
            float4 *dst = reinterpret_cast<float4 *>(&xs[p][8 * q]);
            dst[0] = make_float4(__bfloat162float(h[0]), __bfloat162float(h[1]), __bfloat162float(h[2]),
                                 __bfloat162float(h[3]));
            dst[1] = make_float4(__bfloat162float(h[4]), __bfloat162float(h[5]), __bfloat162float(h[6]),
                                 __bfloat162float(h[7]));
        }
        __syncthreads();          // widened tiles visible; the raw buffers are free
        if (tile + 1 < t1) issue(tile + 1);
        for (int p = 0; p < WG_P; ++p) {
            float d[NCO];
#pragma unroll
            for (int u = 0; u < NCO; ++u) d[u] = dzs[p][lane + 32 * u];
            int py = p / WG_W, px = p % WG_W;
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                // the warp's four input channels in one 16-byte (broadcast) load
                const float4 xv = *reinterpret_cast<const float4 *>(&xs[(py + t / 3) * (WG_W + 2) + px + t % 3][warp * 4]);
#pragma unroll
                for (int u = 0; u < NCO; ++u) {
                    acc[u][0][t] = fmaf(d[u], xv.x, acc[u][0][t]);
                    acc[u][1][t] = fmaf(d[u], xv.y, acc[u][1][t]);
                    acc[u][2][t] = fmaf(d[u], xv.z, acc[u][2][t]);
                    acc[u][3][t] = fmaf(d[u], xv.w, acc[u][3][t]);
                }
            }
        }
    }
#pragma unroll
    for (int u = 0; u < NCO; ++u) {
        const int co = co0 + lane + 32 * u;
        if (co >= cout) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int ci = ci0 + warp * 4 + j;
            if (ci >= cin) continue;
#pragma unroll
            for (int t = 0; t < 9; ++t) atomicAdd(&dW[((size_t)co * cin + ci) * 9 + t], acc[u][j][t]);
        }
    }
}

// First layer (1 input channel X = eta R): dW[co][tap] and d(eta R)[p]
__device__ __forceinline__ float rin_at(const float *R, int b, int y, int x, int nx, int ny)
{
    return (y >= 0 && x >= 0 && y < ny && x < nx) ? R[((size_t)b * ny + y) * nx + x] : 0.f;
}

// dW[co][tap] of the first layer, dW[co][t] = sum_p dZ[p][co] V[p][t] with
// V[p][t] = (eta R) at the tap's neighbour of p.  A block stages a tile of
// WI_TP pixels (their dZ rows with 16-byte copies, their nine V values) in
// shared memory; thread k then owns the pairs (co, t) = k, k + 256, ... and
// sums over the tile's pixels; each pair is added to dW once per block.
constexpr int WI_THREADS = 256, WI_TP = 128, WI_MAXC = 128, WI_MAXK = (WI_MAXC * 9 + WI_THREADS - 1) / WI_THREADS;

int wg_sm_count_host()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

__global__ void __launch_bounds__(WI_THREADS) wgrad_in_kernel(const bf16 *__restrict__ dZ,
                                                             const float *__restrict__ R,
                                                             const float *__restrict__ eta, int B, int H, int W,
                                                             int C, int nx, int ny, float *__restrict__ dW)
{
    __shared__ float V[WI_TP * 9];
    __shared__ __align__(16) bf16 Z[WI_TP * WI_MAXC];
    const size_t P = (size_t)B * H * W;
    const int npair = C * 9;
    float acc[WI_MAXK];
#pragma unroll
    for (int j = 0; j < WI_MAXK; ++j) acc[j] = 0.f;
    const size_t ntiles = (P + WI_TP - 1) / WI_TP;
    for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const size_t p0 = tile * WI_TP;
        const int np = (int)min((size_t)WI_TP, P - p0);
        for (int i = threadIdx.x; i < WI_TP * 9; i += WI_THREADS) {
            const int pi = i / 9, t = i - pi * 9;
            float v = 0.f;
            if (pi < np) {
                const size_t p = p0 + pi;
                const int x = (int)(p % W), y = (int)((p / W) % H), b = (int)(p / ((size_t)W * H));
                const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
                if (yy >= 0 && xx >= 0 && yy < H && xx < W) v = rin_at(R, b, yy, xx, nx, ny) * eta[yy * W + xx];
            }
            V[i] = v;
        }
        // the tile's dZ rows are contiguous: np * C values, C a multiple of 8
        const uint4 *src = reinterpret_cast<const uint4 *>(dZ + p0 * C);
        uint4 *dst = reinterpret_cast<uint4 *>(Z);
        for (int i = threadIdx.x; i < np * C / 8; i += WI_THREADS) dst[i] = src[i];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < WI_MAXK; ++j) {
            const int k = threadIdx.x + WI_THREADS * j;
            if (k >= npair) break;
            const int co = k / 9, t = k - co * 9;
            float sacc = 0.f;
            for (int pi = 0; pi < np; ++pi) sacc = fmaf(__bfloat162float(Z[pi * C + co]), V[pi * 9 + t], sacc);
            acc[j] += sacc;
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < WI_MAXK; ++j) {
        const int k = threadIdx.x + WI_THREADS * j;
        if (k < npair) atomicAdd(&dW[k], acc[j]);
    }
}

__global__ void dgrad_in_kernel(const bf16 *__restrict__ dZ, const float *__restrict__ Wt /*[C][9] FP32 OIHW*/,
                                const float *__restrict__ R, int B, int H, int W, int C, int nx, int ny,
                                float *__restrict__ deta)
{
    const size_t P = (size_t)B * H * W;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        int x = p % W, y = (p / W) % H, b = p / ((size_t)W * H);
        float g = 0.f;   // d(eta R)[p] = sum_tap sum_co W[co][tap] dZ[p - offset(tap)][co]
        for (int t = 0; t < 9; ++t) {
            int yy = y - (t / 3 - 1), xx = x - (t % 3 - 1);
            if (yy < 0 || xx < 0 || yy >= H || xx >= W) continue;
            const bf16 *dz = dZ + (((size_t)b * H + yy) * W + xx) * C;
            if ((C & 7) == 0) {
                // the pixel's channels as 16-byte pieces, in channel order
                for (int co = 0; co < C; co += 8) {
                    const uint4 raw = *reinterpret_cast<const uint4 *>(dz + co);
                    const bf16 *hv = reinterpret_cast<const bf16 *>(&raw);
#pragma unroll
                    for (int i = 0; i < 8; ++i) g = fmaf(Wt[(co + i) * 9 + t], __bfloat162float(hv[i]), g);
                }
            } else {
                for (int co = 0; co < C; ++co) g = fmaf(Wt[co * 9 + t], __bfloat162float(dz[co]), g);
            }
        }
        float r = rin_at(R, b, y, x, nx, ny);
        atomicAdd(&deta[y * W + x], r * g);
    }
}

// dX = eta d(eta X);  d eta += sum_c (eta X) d(eta X) / eta
// A thread takes four channels of a pixel (16-byte loads and stores); the
// pixel's C/4 threads are consecutive lanes, summed by shuffles when C/4
// divides 32, and one of them adds to d eta.
__global__ void eta_bwd_kernel(const float4 *__restrict__ dXb, const uint2 *__restrict__ Xb,
                               const float *__restrict__ eta, size_t P, int HW, int C4, float4 *__restrict__ dX,
                               float *__restrict__ deta, int mesh)
{
    const size_t n = P * C4;
    const bool seg = C4 <= 32 && (32 % C4) == 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t base = (size_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const size_t k = base + threadIdx.x;
        const bool ok = k < n;
        float s = 0.f, e = 0.f;
        int q = 0;
        if (ok) {
            const size_t p = k / C4;
            q = (int)(p % HW);
            e = eta[q];
            const float4 g = dXb[k];
            dX[k] = make_float4(e * g.x, e * g.y, e * g.z, e * g.w);
            const uint2 raw = Xb[k];
            const bf16 *h = reinterpret_cast<const bf16 *>(&raw);
            s = __bfloat162float(h[0]) * g.x + __bfloat162float(h[1]) * g.y + __bfloat162float(h[2]) * g.z +
                __bfloat162float(h[3]) * g.w;
        }
        if (!mesh) continue;
        if (seg) {
            for (int o = 1; o < C4; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (ok && (threadIdx.x % C4) == 0 && e > 0.f) atomicAdd(&deta[q], s / e);
        } else if (ok && e > 0.f) {
            atomicAdd(&deta[q], s / e);
        }
    }
}

// Weight-network backward: phi = w2 . tanh(W1 D + b1) + b2, eta = exp(-phi^2).
// Each thread accumulates its pixels' contributions in registers (hid <= 16),
// then the block reduces them with warp shuffles and one atomic per value.
constexpr int PHI_MAXH = 16;
__global__ void __launch_bounds__(256) phi_bwd_kernel(const float *__restrict__ deta, const float *__restrict__ eta,
                               const float *__restrict__ phi, const float *__restrict__ D, int HW,
                               const float *__restrict__ W1, const float *__restrict__ b1, const float *__restrict__ w2,
                               int hid, float *__restrict__ gW1, float *__restrict__ gb1, float *__restrict__ gw2,
                               float *__restrict__ gb2)
{
    float a_w2[PHI_MAXH], a_b1[PHI_MAXH], a_W1[PHI_MAXH][4], a_b2 = 0.f;
#pragma unroll
    for (int k = 0; k < PHI_MAXH; ++k) {
        a_w2[k] = a_b1[k] = 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c) a_W1[k][c] = 0.f;
    }
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < HW; q += gridDim.x * blockDim.x) {
        float dphi = deta[q] * eta[q] * (-2.f * phi[q]);
        float d[4] = {D[q], D[HW + q], D[2 * HW + q], D[3 * HW + q]};
        a_b2 += dphi;
#pragma unroll
        for (int k = 0; k < PHI_MAXH; ++k) {
            if (k >= hid) break;
            float z = b1[k] + W1[4 * k] * d[0] + W1[4 * k + 1] * d[1] + W1[4 * k + 2] * d[2] + W1[4 * k + 3] * d[3];
            float h = tanhf(z);
            a_w2[k] += dphi * h;
            float dz = dphi * w2[k] * (1.f - h * h);
            a_b1[k] += dz;
#pragma unroll
            for (int c = 0; c < 4; ++c) a_W1[k][c] += dz * d[c];
        }
    }
    // warp sums, then the block's warps summed in shared memory: one atomic
    // per value and block (per warp, the ~100 values had drawn thousands of
    // atomics each)
    constexpr int NV = 1 + 6 * PHI_MAXH;
    __shared__ float red[8][NV];
    auto wsum = [](float v) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        return v;
    };
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float v = wsum(a_b2);
    if (lane == 0) red[warp][0] = v;
#pragma unroll
    for (int k = 0; k < PHI_MAXH; ++k) {
        if (k >= hid) break;
        v = wsum(a_w2[k]);
        if (lane == 0) red[warp][1 + 6 * k] = v;
        v = wsum(a_b1[k]);
        if (lane == 0) red[warp][2 + 6 * k] = v;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            v = wsum(a_W1[k][c]);
            if (lane == 0) red[warp][3 + 6 * k + c] = v;
        }
    }
    __syncthreads();
    const int nv = 1 + 6 * hid, nw = blockDim.x >> 5;
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
        float sum = 0.f;
        for (int w = 0; w < nw; ++w) sum += red[w][i];
        if (sum == 0.f) continue;
        if (i == 0) {
            atomicAdd(gb2, sum);
        } else {
            const int k = (i - 1) / 6, f = (i - 1) % 6;
            if (f == 0)
                atomicAdd(&gw2[k], sum);
            else if (f == 1)
                atomicAdd(&gb1[k], sum);
            else
                atomicAdd(&gW1[4 * k + (f - 2)], sum);
        }
    }
}

// dst[p][dco + c] += src[p][sco + c], c < nc
__global__ void add_slice_kernel(float *__restrict__ dst, int dcs, int dco, const float *__restrict__ src, int scs,
                                 int sco, int nc, size_t P)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < P * nc; k += (size_t)gridDim.x * blockDim.x) {
        size_t p = k / nc;
        int c = k % nc;
        dst[p * dcs + dco + c] += src[p * scs + sco + c];
    }
}

// coarse[b][y][x][c] += sum of the 4 fine children (fine: [B][2H][2W][C])
__global__ void up2_bwd_kernel(const float *__restrict__ fine, float *__restrict__ coarse, int B, int H, int W, int C)
{
    size_t n = (size_t)B * H * W * C;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        int c = k % C;
        size_t pix = k / C;
        int x = pix % W, y = (pix / W) % H, b = pix / ((size_t)W * H);
        float s = 0.f;
        for (int t = 0; t < 4; ++t)
            s += fine[((((size_t)b * 2 * H) + 2 * y + (t >> 1)) * 2 * W + 2 * x + (t & 1)) * C + c];
        coarse[k] += s;
    }
}

// fine[b][y][x][c] += 0.25 coarse[b][y/2][x/2][c]   (fine: [B][H][W][C])
__global__ void pool2_bwd_kernel(const float *__restrict__ coarse, float *__restrict__ fine, int B, int H, int W, int C)
{
    size_t n = (size_t)B * H * W * C;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        int c = k % C;
        size_t pix = k / C;
        int x = pix % W, y = (pix / W) % H, b = pix / ((size_t)W * H);
        fine[k] += 0.25f * coarse[((((size_t)b * (H / 2)) + y / 2) * (W / 2) + x / 2) * C + c];
    }
}

// dz = dt * (1 - t^2)
__global__ void tanh_bwd_kernel(const float *__restrict__ dt, const float *__restrict__ t, float *__restrict__ dz,
                                size_t n)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        dz[k] = dt[k] * (1.f - t[k] * t[k]);
}

__global__ void fill_kernel(float *p, size_t n, float v)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) p[k] = v;
}

__global__ void sumsq_kernel(const float *__restrict__ g, size_t n, double *acc)
{
    double s = 0.0;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        s += (double)g[k] * g[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        atomicAdd(acc, t);
    }
}

// P' = P + rho g / ||g||  (||g||^2 read from the device)
__global__ void perturb_kernel(const float *__restrict__ P, const float *__restrict__ g, float *__restrict__ Pp,
                               size_t n, double rho, const double *gsq)
{
    const float s = (float)(rho / (sqrt(*gsq) + 1e-12));
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        Pp[k] = P[k] + s * g[k];
}

__global__ void adam_kernel(float *__restrict__ P, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, size_t n, float lr, float b1, float b2, float eps, float bc1,
                            float bc2)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        float gk = g[k];
        float mk = b1 * m[k] + (1.f - b1) * gk;
        float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        P[k] -= lr * (mk / bc1) / (sqrtf(vk / bc2) + eps);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------

struct TrainWs {
    int capB = 0;
    std::vector<size_t> G;        // per-layer dL/dY offsets (FP32 elements)
    float *g = nullptr;           // all dL/dY buffers
    size_t g_elems = 0;
    float *dXb = nullptr, *dX = nullptr, *deta = nullptr;
    bf16 *dZ = nullptr;
    float *e = nullptr, *Ae = nullptr, *res = nullptr, *de = nullptr;
    float *dU0 = nullptr, *dweff = nullptr, *dceff = nullptr;
    float *dt3 = nullptr, *dt2 = nullptr, *dt1 = nullptr, *dz = nullptr, *ones = nullptr;
    float *gemm_part = nullptr;   // the trunk weight gradients' per-CTA slices
    size_t gemm_part_elems = 0;
    double *acc = nullptr;        // [0] loss sum, [1] grad sumsq
};

static void free_ws(TrainWs *w)
{
    if (!w) return;
    cudaFree(w->g); cudaFree(w->dXb); cudaFree(w->dX); cudaFree(w->deta); cudaFree(w->dZ);
    cudaFree(w->e); cudaFree(w->Ae); cudaFree(w->res); cudaFree(w->de); cudaFree(w->dU0);
    cudaFree(w->dweff); cudaFree(w->dceff); cudaFree(w->dt3); cudaFree(w->dt2); cudaFree(w->dt1);
    cudaFree(w->dz); cudaFree(w->ones); cudaFree(w->gemm_part); cudaFree(w->acc);
    delete w;
}

void net_free_train(NetCache *c)
{
    free_ws((TrainWs *)c->train);
    c->train = nullptr;
}

static ppe_status ensure_ws(ppe_net *n, NetCache *c, int B)
{
    TrainWs *w = (TrainWs *)c->train;
    if (w && w->capB >= B) return PPE_OK;
    free_ws(w);
    w = new TrainWs();
    c->train = w;
    w->capB = B;
    size_t off = 0, maxin = 0, maxout = 0;
    w->G.resize(n->layers.size());
    for (size_t i = 0; i < n->layers.size(); ++i) {
        const ConvLayer &l = n->layers[i];
        size_t px = (size_t)B * c->Hk[l.level] * c->Wk[l.level];
        w->G[i] = off;
        off += px * l.cout;
        maxin = std::max(maxin, px * l.cin);
        maxout = std::max(maxout, px * l.cout);
    }
    w->g_elems = off;
    const size_t P = (size_t)c->H * c->W, N = (size_t)c->nx * c->ny;
    const ppe_net_config &cf = n->cfg;
    PPE_CUDA_TRY(cudaMalloc(&w->g, off * 4));
    PPE_CUDA_TRY(cudaMalloc(&w->dXb, maxin * 4));
    PPE_CUDA_TRY(cudaMalloc(&w->dX, maxin * 4));
    PPE_CUDA_TRY(cudaMalloc(&w->dZ, maxout * 2));
    PPE_CUDA_TRY(cudaMalloc(&w->deta, P * 4));
    PPE_CUDA_TRY(cudaMalloc(&w->e, N * B * 4));
    PPE_CUDA_TRY(cudaMalloc(&w->Ae, N * B * 4));
    PPE_CUDA_TRY(cudaMalloc(&w->res, N * B * 4));
    PPE_CUDA_TRY(cudaMalloc(&w->de, N * B * 4));
    PPE_CUDA_TRY(cudaMalloc(&w->dU0, (size_t)B * P * cf.widths[0] * 4));
    PPE_CUDA_TRY(cudaMalloc(&w->dweff, P * cf.widths[0] * 4));
    PPE_CUDA_TRY(cudaMalloc(&w->dceff, P * 4));
    PPE_CUDA_TRY(cudaMalloc(&w->dt3, P * cf.c_last * 4));
    PPE_CUDA_TRY(cudaMalloc(&w->dt2, P * cf.trunk_hidden[1] * 4));
    PPE_CUDA_TRY(cudaMalloc(&w->dt1, P * cf.trunk_hidden[0] * 4));
    PPE_CUDA_TRY(cudaMalloc(&w->dz, P * std::max(cf.trunk_hidden[0], cf.trunk_hidden[1]) * 4));
    PPE_CUDA_TRY(cudaMalloc(&w->ones, P * 4));
    {
        const int cl = cf.c_last, h0 = cf.trunk_hidden[0], h1 = cf.trunk_hidden[1], C0 = cf.widths[0];
        w->gemm_part_elems = std::max({tgemm_scratch_floats(cl, C0), tgemm_scratch_floats(cl, h1),
                                       tgemm_scratch_floats(h1, h0)});
        PPE_CUDA_TRY(cudaMalloc(&w->gemm_part, w->gemm_part_elems * 4));
    }
    PPE_CUDA_TRY(cudaMalloc(&w->acc, 2 * sizeof(double)));
    fill_kernel<<<g1d(P), 256>>>(w->ones, P, 1.f);
    PPE_CUDA_TRY(cudaGetLastError());
    return PPE_OK;
}

// ---------------------------------------------------------------------------
// loss, backward
// ---------------------------------------------------------------------------

// L = mean (R - A e)^2 and de = -(2/(B N)) A (R - A e).  Loss sum lands in w->acc[0].
static ppe_status loss_de(ppe_grid *g, TrainWs *w, int B, const float *R, cudaStream_t s)
{
    const size_t N = (size_t)g->nx * g->ny;
    apply_f32_kernel<<<g1d(N * B), 256, 0, s>>>(w->e, w->Ae, g->nx, g->ny, B, g->dx32, g->dy32, g->fx32, g->fy32, 1.f);
    residual_kernel<<<g1d(N * B), 256, 0, s>>>(R, w->Ae, w->res, N * B, w->acc);
    apply_f32_kernel<<<g1d(N * B), 256, 0, s>>>(w->res, w->de, g->nx, g->ny, B, g->dx32, g->dy32, g->fx32, g->fy32,
                                                 (float)(-2.0 / ((double)B * N)));
    PPE_CUDA_TRY(cudaGetLastError());
    return PPE_OK;
}

// CUDA-core weight gradient dW[co][ci][9] += (dZ, X)
static ppe_status wgrad_simt(const bf16 *dZ, const bf16 *Xb, int B, int H, int W, int cin, int cout, float *dW,
                             cudaStream_t s)
{
    if (cin % 8 || cout % 8) {
        set_error("weight gradient: channel counts must be multiples of 8");
        return PPE_ERR_ARG;
    }
    // two output channels per thread from 64 on (each loaded input value
    // then feeds twice the products); one below
    const int nco = cout >= 64 ? 2 : 1;
    const int tiles = B * ((W + WG_W - 1) / WG_W) * ((H + WG_H - 1) / WG_H);
    dim3 grid((cout + 32 * nco - 1) / (32 * nco), (cin + 31) / 32, 1);
    int blocks_xy = grid.x * grid.y;
    int split = std::max(1, std::min(tiles, 592 / std::max(1, blocks_xy)));
    int per = (tiles + split - 1) / split;
    grid.z = (tiles + per - 1) / per;
    // the shared-memory opt-in is a per-device attribute of each kernel
    static PerDevice attrs;
    if (!once_per_device(attrs, [](int) {
            return cudaFuncSetAttribute(wgrad_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)wg_smem<1>()) == cudaSuccess &&
                   cudaFuncSetAttribute(wgrad_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)wg_smem<2>()) == cudaSuccess;
        }))
        return cuda_status(cudaGetLastError(), "cudaFuncSetAttribute(wgrad_kernel)");
    if (nco == 2)
        wgrad_kernel<2><<<grid, 256, wg_smem<2>(), s>>>(dZ, Xb, B, H, W, cin, cout, dW, per);
    else
        wgrad_kernel<1><<<grid, 256, wg_smem<1>(), s>>>(dZ, Xb, B, H, W, cin, cout, dW, per);
    PPE_CUDA_TRY(cudaGetLastError());
    return PPE_OK;
}

static ppe_status conv_backward(ppe_net *n, NetCache *c, TrainWs *w, int li, const bf16 *Xb, const float *P,
                                float *grads, int B, cudaStream_t s)
{
    const ConvLayer &l = n->layers[li];
    const int k = l.level, H = c->Hk[k], W = c->Wk[k];
    const size_t px = (size_t)B * H * W;
    const float *dY = w->g + w->G[li];
    const bf16 *Z = c->act + c->plan.Z[li];
    act_bwd(dY, Z, w->dZ, px * l.cout, l.cout, grads + l.off_b, s);
    // weight gradient: tensor cores where the kernel takes the channel counts
    if (n->use_tc && wgrad_tc_supported(l.cin, l.cout))
        PPE_TRY(wgrad_tc(w->dZ, Xb, B, H, W, l.cin, l.cout, grads + l.off_w, s));
    else
        PPE_TRY(wgrad_simt(w->dZ, Xb, B, H, W, l.cin, l.cout, grads + l.off_w, s));
    // data gradient: forward convolution of dZ with the transposed, flipped kernel
    ConvArgs a;
    a.in = w->dZ; a.w = n->wt + l.off_wt; a.bias = nullptr;
    a.B = B; a.H = H; a.W = W; a.cin = l.cout; a.cout = l.cin;
    a.epi.zf_out = w->dXb; a.epi.act = 0;
    PPE_TRY(run_conv(n, a, s));
    PPE_CUDA_TRY(cudaMemsetAsync(w->deta, 0, (size_t)H * W * 4, s));
    const float *eta = c->eta + c->eoff[li];
    eta_bwd_kernel<<<std::min(2048u, g1d(px * (l.cin / 4))), 256, 0, s>>>(
        reinterpret_cast<const float4 *>(w->dXb), reinterpret_cast<const uint2 *>(Xb), eta, px, H * W, l.cin / 4,
        reinterpret_cast<float4 *>(w->dX), w->deta, n->cfg.mesh_conv);
    if (n->cfg.mesh_conv) {
        int hid = n->cfg.phi_hidden;
        phi_bwd_kernel<<<std::min(128u, g1d((size_t)H * W)), 256, 0, s>>>(
            w->deta, eta, c->phi + c->eoff[li], c->delta + c->doff[k], H * W, P + l.off_p1w, P + l.off_p1b,
            P + l.off_p2w, hid, grads + l.off_p1w, grads + l.off_p1b, grads + l.off_p2w, grads + l.off_p2b);
    }
    PPE_CUDA_TRY(cudaGetLastError());
    return PPE_OK;
}

// Full backward: gradients of sum(de * e) into `grads` (zeroed here).
static ppe_status net_backward(ppe_net *n, NetCache *c, TrainWs *w, ppe_grid *g, int B, const float *R,
                               const float *P, float *grads, cudaStream_t s)
{
    const ppe_net_config &cf = n->cfg;
    const int L = c->L;
    const ActPlan &pl = c->plan;
    const int Pn = c->H * c->W;
    const int C0 = cf.widths[0];
    PPE_CUDA_TRY(cudaMemsetAsync(grads, 0, n->nparams * 4, s));
    PPE_CUDA_TRY(cudaMemsetAsync(w->g, 0, w->g_elems * 4, s));
    auto G = [&](const std::string &name) { return w->g + w->G[layer_index(n, name)]; };

    // DeepONet fold: e = sum_c U0_c weff_c + ceff
    float *gdec0b = G("dec0b");
    fold_bwd_kernel<<<g1d(Pn), 256, 0, s>>>(w->de, c->act + pl.U[0], c->weff, B, c->H, c->W, C0, g->nx, g->ny, gdec0b,
                                            w->dweff, w->dceff);
    // head + trunk: weff = head.w^T t3, ceff = head.b . t3 + out.b, t3 = T2 t2 + b2, t2 = tanh(T1 t1 + b1), ...
    float *t1 = c->trunk, *t2 = t1 + (size_t)cf.trunk_hidden[0] * Pn, *t3 = t2 + (size_t)cf.trunk_hidden[1] * Pn;
    const int h0 = cf.trunk_hidden[0], h1 = cf.trunk_hidden[1], cl = cf.c_last;
    PPE_TRY(tgemm(cl, C0, Pn, t3, Pn, false, w->dweff, Pn, true, grads + n->off_head_w, C0, nullptr, 0, false, s,
                  w->gemm_part, w->gemm_part_elems));
    PPE_TRY(tgemm(cl, 1, Pn, t3, Pn, false, w->dceff, 1, false, grads + n->off_head_b, 1, nullptr, 0, false, s));
    PPE_TRY(tgemm(1, 1, Pn, w->dceff, Pn, false, w->ones, 1, false, grads + n->off_out_b, 1, nullptr, 0, false, s));
    PPE_TRY(tgemm(cl, Pn, C0, P + n->off_head_w, C0, false, w->dweff, Pn, false, w->dt3, Pn, nullptr, 0, false, s));
    PPE_TRY(tgemm(cl, Pn, 1, P + n->off_head_b, 1, false, w->dceff, Pn, false, w->dt3, Pn, nullptr, 0, true, s));
    PPE_TRY(tgemm(cl, h1, Pn, w->dt3, Pn, false, t2, Pn, true, grads + n->off_tw[2], h1, nullptr, 0, false, s,
                  w->gemm_part, w->gemm_part_elems));
    PPE_TRY(tgemm(cl, 1, Pn, w->dt3, Pn, false, w->ones, 1, false, grads + n->off_tb[2], 1, nullptr, 0, false, s));
    PPE_TRY(tgemm(h1, Pn, cl, P + n->off_tw[2], h1, true, w->dt3, Pn, false, w->dt2, Pn, nullptr, 0, false, s));
    tanh_bwd_kernel<<<g1d((size_t)h1 * Pn), 256, 0, s>>>(w->dt2, t2, w->dz, (size_t)h1 * Pn);
    PPE_TRY(tgemm(h1, h0, Pn, w->dz, Pn, false, t1, Pn, true, grads + n->off_tw[1], h0, nullptr, 0, false, s,
                  w->gemm_part, w->gemm_part_elems));
    PPE_TRY(tgemm(h1, 1, Pn, w->dz, Pn, false, w->ones, 1, false, grads + n->off_tb[1], 1, nullptr, 0, false, s));
    PPE_TRY(tgemm(h0, Pn, h1, P + n->off_tw[1], h0, true, w->dz, Pn, false, w->dt1, Pn, nullptr, 0, false, s));
    tanh_bwd_kernel<<<g1d((size_t)h0 * Pn), 256, 0, s>>>(w->dt1, t1, w->dz, (size_t)h0 * Pn);
    PPE_TRY(tgemm(h0, 2, Pn, w->dz, Pn, false, c->xy, Pn, true, grads + n->off_tw[0], 2, nullptr, 0, false, s,
                  w->gemm_part, w->gemm_part_elems));
    PPE_TRY(tgemm(h0, 1, Pn, w->dz, Pn, false, w->ones, 1, false, grads + n->off_tb[0], 1, nullptr, 0, false, s));

    // decoder, level 0 upward
    for (int k = 0; k <= L - 2; ++k) {
        const std::string ks = std::to_string(k);
        const int Ck = cf.widths[k];
        const size_t px = (size_t)B * c->Hk[k] * c->Wk[k];
        PPE_TRY(conv_backward(n, c, w, layer_index(n, "dec" + ks + "b"), c->act + pl.D[k], P, grads, B, s));
        add_slice_kernel<<<g1d(px * Ck), 256, 0, s>>>(G("dec" + ks + "a"), Ck, 0, w->dX, Ck, 0, Ck, px);
        PPE_TRY(conv_backward(n, c, w, layer_index(n, "dec" + ks + "a"), c->act + pl.CAT[k], P, grads, B, s));
        add_slice_kernel<<<g1d(px * Ck), 256, 0, s>>>(G("up" + ks), Ck, 0, w->dX, 2 * Ck, 0, Ck, px);
        add_slice_kernel<<<g1d(px * Ck), 256, 0, s>>>(G("enc" + ks + "b"), Ck, 0, w->dX, 2 * Ck, Ck, Ck, px);
        PPE_TRY(conv_backward(n, c, w, layer_index(n, "up" + ks), c->act + pl.UP[k], P, grads, B, s));
        const std::string next = (k + 1 == L - 1) ? "enc" + std::to_string(k + 1) + "b" : "dec" + std::to_string(k + 1) + "b";
        const int C1 = cf.widths[k + 1];
        up2_bwd_kernel<<<g1d((size_t)B * c->Hk[k + 1] * c->Wk[k + 1] * C1), 256, 0, s>>>(w->dX, G(next), B, c->Hk[k + 1],
                                                                                        c->Wk[k + 1], C1);
    }
    // encoder, deepest level downward
    for (int k = L - 1; k >= 0; --k) {
        const std::string ks = std::to_string(k);
        const int Ck = cf.widths[k];
        const size_t px = (size_t)B * c->Hk[k] * c->Wk[k];
        PPE_TRY(conv_backward(n, c, w, layer_index(n, "enc" + ks + "b"), c->act + pl.A[k], P, grads, B, s));
        add_slice_kernel<<<g1d(px * Ck), 256, 0, s>>>(G("enc" + ks + "a"), Ck, 0, w->dX, Ck, 0, Ck, px);
        if (k > 0) {
            PPE_TRY(conv_backward(n, c, w, layer_index(n, "enc" + ks + "a"), c->act + pl.IN[k], P, grads, B, s));
            const int Cp = cf.widths[k - 1];
            pool2_bwd_kernel<<<g1d((size_t)B * c->Hk[k - 1] * c->Wk[k - 1] * Cp), 256, 0, s>>>(
                w->dX, G("enc" + std::to_string(k - 1) + "b"), B, c->Hk[k - 1], c->Wk[k - 1], Cp);
        }
    }
    // first layer (one input channel)
    {
        const int li = layer_index(n, "enc0a");
        const ConvLayer &l = n->layers[li];
        const size_t px = (size_t)B * c->H * c->W;
        act_bwd(G("enc0a"), c->act + pl.Z[li], w->dZ, px * l.cout, l.cout, grads + l.off_b, s);
        const float *eta = c->eta + c->eoff[li];
        if (l.cout > WI_MAXC || l.cout % 8 || ((uintptr_t)w->dZ & 15)) {
            set_error("first-layer weight gradient: at most 128 channels, a multiple of 8, 16-byte aligned rows");
            return PPE_ERR_ARG;
        }
        {
            const size_t tiles = (px + WI_TP - 1) / WI_TP;
            const unsigned gw = (unsigned)std::min<size_t>(tiles, 4 * (size_t)wg_sm_count_host());
            wgrad_in_kernel<<<gw, WI_THREADS, 0, s>>>(w->dZ, R, eta, B, c->H, c->W, l.cout, g->nx, g->ny,
                                                      grads + l.off_w);
        }
        if (cf.mesh_conv) {
            PPE_CUDA_TRY(cudaMemsetAsync(w->deta, 0, (size_t)c->H * c->W * 4, s));
            dgrad_in_kernel<<<g1d(px), 256, 0, s>>>(w->dZ, P + l.off_w, R, B, c->H, c->W, l.cout, g->nx, g->ny, w->deta);
            int hid = cf.phi_hidden;
            phi_bwd_kernel<<<std::min(128u, g1d((size_t)c->H * c->W)), 256, 0, s>>>(
                w->deta, eta, c->phi + c->eoff[li], c->delta + c->doff[0], c->H * c->W, P + l.off_p1w, P + l.off_p1b,
                P + l.off_p2w, hid, grads + l.off_p1w, grads + l.off_p1b, grads + l.off_p2w, grads + l.off_p2b);
        }
    }
    PPE_CUDA_TRY(cudaGetLastError());
    return PPE_OK;
}

// forward + loss + backward at parameters P; gradient into grads, loss sum into w->acc[0]
static ppe_status loss_and_grad(ppe_net *n, NetCache *c, TrainWs *w, ppe_grid *g, int B, const float *R, const float *P,
                                float *grads, cudaStream_t s)
{
    InputSrc src;
    src.r = R; src.pitch = g->nx; src.bstride = (size_t)g->nx * g->ny; src.nx = g->nx; src.ny = g->ny;
    PPE_TRY(net_forward(n, c, B, src, P, w->e, g->nx, (size_t)g->nx * g->ny, true, s));
    PPE_TRY(loss_de(g, w, B, R, s));
    return net_backward(n, c, w, g, B, R, P, grads, s);
}

}  // namespace ppe

extern "C" ppe_status ppe_debug_wgrad(const void *dZ, const void *X, int B, int H, int W, int cin, int cout, float *dW,
                                      int impl, void *stream)
{
    ppe::clear_error();
    if (!dZ || !X || !dW || B < 1 || H < 1 || W < 1 || cin < 1 || cout < 1) {
        ppe::set_error("ppe_debug_wgrad: bad arguments");
        return PPE_ERR_ARG;
    }
    const ppe::bf16 *z = (const ppe::bf16 *)dZ, *x = (const ppe::bf16 *)X;
    if (impl == 0) return ppe::wgrad_tc(z, x, B, H, W, cin, cout, dW, (cudaStream_t)stream);
    return ppe::wgrad_simt(z, x, B, H, W, cin, cout, dW, (cudaStream_t)stream);
}

extern "C" ppe_status ppe_debug_gemm(int M, int N, int K, const float *A, int lda, int transA, const float *B, int ldb,
                                     int transB, float *C, int ldc, const float *bias, int act, int accumulate, int impl,
                                     int *form, void *stream)
{
    ppe::clear_error();
    if (!A || !B || !C || M < 1 || N < 1 || K < 1 || lda < 1 || ldb < 1 || ldc < N || (act != 0 && act != 1)) {
        ppe::set_error("ppe_debug_gemm: bad arguments");
        return PPE_ERR_ARG;
    }
    const int f = impl == 0 ? ppe::tgemm_form(M, N, K, A, lda, transA != 0, B, ldb, transB != 0, bias, act) : 0;
    if (form) *form = f;
    if (impl == 0)
        return ppe::tgemm(M, N, K, A, lda, transA != 0, B, ldb, transB != 0, C, ldc, bias, act, accumulate != 0,
                          (cudaStream_t)stream);
    return ppe::sgemm(M, N, K, A, lda, transA != 0, B, ldb, transB != 0, C, ldc, bias, act, accumulate != 0,
                      (cudaStream_t)stream);
}


using namespace ppe;

extern "C" {

void net_default_hparams(ppe_train_hparams *hp)
{
    if (!hp) return;
    std::memset(hp, 0, sizeof(*hp));
    hp->lr0 = 2e-4;
    hp->total_steps = 1000000;
    hp->rho = 2e-4;
    hp->beta1 = 0.9;
    hp->beta2 = 0.999;
    hp->eps = 1e-8;
}

ppe_status net_get_step(const ppe_net *n, int64_t *step)
{
    if (!n || !step) { set_error("net_get_step: NULL argument"); return PPE_ERR_ARG; }
    *step = n->step;
    return PPE_OK;
}

static ppe_status train_prep(ppe_net *n, ppe_grid *g, int batch, const float *R, NetCache **cout, TrainWs **wout)
{
    if (!n || !g || !R || batch < 1) { set_error("net training: bad arguments"); return PPE_ERR_ARG; }
    PPE_TRY(net_check_grid(n, g));
    NetCache *c = (NetCache *)g->net_cache;
    PPE_TRY(ensure_acts(n, c, batch));
    PPE_TRY(ensure_ws(n, c, batch));
    *cout = c;
    *wout = (TrainWs *)c->train;
    return PPE_OK;
}

ppe_status net_loss_grad(ppe_net *n, ppe_grid *g, int batch, const float *R, void *stream, double *loss_out,
                         float *grad_host)
{
    clear_error();
    NetCache *c;
    TrainWs *w;
    PPE_TRY(train_prep(n, g, batch, R, &c, &w));
    cudaStream_t s = (cudaStream_t)stream;
    PPE_CUDA_TRY(cudaMemsetAsync(w->acc, 0, 2 * sizeof(double), s));
    PPE_TRY(loss_and_grad(n, c, w, g, batch, R, n->params, n->grads, s));
    double acc[2];
    PPE_CUDA_TRY(cudaMemcpyAsync(acc, w->acc, sizeof acc, cudaMemcpyDeviceToHost, s));
    if (grad_host) PPE_CUDA_TRY(cudaMemcpyAsync(grad_host, n->grads, n->nparams * 4, cudaMemcpyDeviceToHost, s));
    PPE_CUDA_TRY(cudaStreamSynchronize(s));
    if (loss_out) *loss_out = acc[0] / ((double)batch * g->nx * g->ny);
    return PPE_OK;
}

ppe_status net_train_step(ppe_net *n, ppe_grid *g, int batch, const float *R, const ppe_train_hparams *hp,
                          void *stream, double *loss_out)
{
    clear_error();
    if (!hp || !(hp->lr0 >= 0.0) || hp->total_steps < 1 || !(hp->rho >= 0.0)) {
        set_error("net_train_step: bad hyper-parameters");
        return PPE_ERR_ARG;
    }
    NetCache *c;
    TrainWs *w;
    PPE_TRY(train_prep(n, g, batch, R, &c, &w));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t np = n->nparams;
    PPE_CUDA_TRY(cudaMemsetAsync(w->acc, 0, 2 * sizeof(double), s));
    PPE_TRY(loss_and_grad(n, c, w, g, batch, R, n->params, n->grads, s));
    double loss_sum = 0.0;
    PPE_CUDA_TRY(cudaMemcpyAsync(&loss_sum, w->acc, sizeof(double), cudaMemcpyDeviceToHost, s));
    const float *gfinal = n->grads;
    if (hp->rho > 0.0) {
        sumsq_kernel<<<g1d(np), 256, 0, s>>>(n->grads, np, w->acc + 1);
        perturb_kernel<<<g1d(np), 256, 0, s>>>(n->params, n->grads, n->params_pert, np, hp->rho, w->acc + 1);
        PPE_TRY(loss_and_grad(n, c, w, g, batch, R, n->params_pert, n->grads2, s));
        gfinal = n->grads2;
    }
    const double t = (double)n->step;
    const double lr = 0.5 * hp->lr0 * (1.0 + std::cos(3.141592653589793 * std::min(t, (double)hp->total_steps) / hp->total_steps));
    const double bc1 = 1.0 - std::pow(hp->beta1, t + 1.0), bc2 = 1.0 - std::pow(hp->beta2, t + 1.0);
    adam_kernel<<<g1d(np), 256, 0, s>>>(n->params, gfinal, n->adam_m, n->adam_v, np, (float)lr, (float)hp->beta1,
                                       (float)hp->beta2, (float)hp->eps, (float)bc1, (float)bc2);
    PPE_CUDA_TRY(cudaGetLastError());
    PPE_CUDA_TRY(cudaStreamSynchronize(s));
    n->step++;
    n->version++;          // caches (packed weights, eta, trunk) follow the new parameters
    if (loss_out) *loss_out = loss_sum / ((double)batch * g->nx * g->ny);
    return PPE_OK;
}

}  // extern "C"
