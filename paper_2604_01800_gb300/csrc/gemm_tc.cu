// tcgen05 GEMMs of the DeepONet trunk and its head fold (Sec. 2.4: the
// trunk's MLP is evaluated at every cell of the grid; training
// back-propagates through it, Eq. 18).  The trunk's tensors are FP32
// [channels][P] with P = the network grid's cell count, so its GEMMs come in
// two shapes:
//
//  * pixel GEMM  C[m][p] = act(sum_k W(m, k) X[k][p] + bias[m]) (+ C):
//    M <= 256 output channels, the pixels are the long dimension.  The MMA
//    runs pixel-major: its M = 128 pixels of a tile, its N = the output
//    channels, K = the input channels.
//  * reduction GEMM  C[m][n] (+)= sum_p A[m][p] B[n][p]: the weight
//    gradients, K = the pixels.  A CTA owns an M block of 128 rows and a
//    range of pixels and writes its partial product to a scratch slice; a
//    second kernel adds the slices in a fixed order (the same result in
//    every run).
//
// Precision: the products are FP32-accurate.  The tensor cores take TF32
// operands (10 mantissa bits), so every operand is split as a = hi + lo
// with hi = a's top 10 mantissa bits (exact in TF32) and lo = a - hi (exact
// in FP32, its own TF32 rounding 2^-21 of a), and each product is summed as
// hi hi + hi lo + lo hi in the FP32 accumulator (the dropped lo lo term is
// 2^-20 of it): three MMAs per K step.  Plain TF32 was measured to leave
// the gradient of a block whose entries are sums with heavy cancellation
// (the head bias) visibly off the FP64 oracle's.
//
// Structure of both kernels: the threads copy each 32-deep K chunk of both
// operands into shared memory, split into hi and lo, in the K-major
// 128-byte-swizzled layout (four K values per 16-byte store), two stages
// deep, so that a chunk is copied while the tensor core works on the
// previous one; thread 0 issues the MMAs into a TMEM accumulator; all eight
// warps read it back.  For the pixel GEMM the copy is also the
// transposition (X's pixels are contiguous, its channels are not).  Every
// wait is bounded: on expiry the kernel raises the error flag, skips the
// rest of its work, lets the MMAs it issued finish, frees its TMEM and
// returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "net_internal.h"
#include "net_ops.h"
#include "tma.cuh"

namespace ppe {

namespace {

constexpr int GT_THREADS = 256;
constexpr long long GT_WAIT_NS = 1000000000LL;
constexpr int GT_KC = 32;                // K values per chunk (one 128-byte row)
constexpr uint32_t GT_ATOM = 1024;       // 8 rows of 128 bytes
constexpr uint32_t GT_AROWS_BYTES = 128u * 128u;   // the 128-row operand of a chunk

__device__ __forceinline__ bool gt_wait(uint32_t bar, uint32_t parity, int *err)
{
    if (mbar_wait_bounded(bar, parity, GT_WAIT_NS)) return true;
    atomicExch(err, 1);
    return false;
}

// K-major 128-byte-swizzled shared-memory descriptor: rows are M or N
// elements, a row holds 32 consecutive K values (FP32), 8 rows form an atom,
// sbo = 1024 between atoms, lbo unused for swizzled K-major operands.
__device__ __forceinline__ uint64_t gt_desc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(GT_ATOM >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;          // 128-byte swizzle
    return d;
}

// kind::tf32 instruction descriptor: TF32 x TF32 -> FP32, M = 128, both
// operands K-major.
__device__ __forceinline__ uint32_t gt_idesc(int n)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void gt_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void gt_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void gt_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void gt_tmem_alloc(uint32_t slot, int cols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void gt_tmem_free(uint32_t tmem, int cols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols) : "memory");
}

// Byte offset of K values 4q .. 4q + 3 of row `row` in a K-major
// 128-byte-swizzled chunk (32 K values per row): the 16-byte chunk index q is
// XORed with the row's index within its 8-row atom.
__device__ __forceinline__ uint32_t quad_off(int row, int q)
{
    return (uint32_t)(row >> 3) * GT_ATOM + (uint32_t)(row & 7) * 128u + (uint32_t)((q ^ (row & 7)) << 4);
}

// Store four K values of a row as their TF32 high parts (top 10 mantissa
// bits) and the FP32 remainders.
__device__ __forceinline__ void store_split(unsigned char *hi, unsigned char *lo, uint32_t off, const float (&v)[4])
{
    float h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        h[j] = __uint_as_float(__float_as_uint(v[j]) & 0xFFFFE000u);
        l[j] = v[j] - h[j];
    }
    *reinterpret_cast<float4 *>(hi + off) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4 *>(lo + off) = make_float4(l[0], l[1], l[2], l[3]);
}

// A stage holds the chunk's 128-row operand (hi, lo) and its np-row operand
// (hi, lo), each region 1024-byte aligned.
struct StageLayout {
    uint32_t a_lo, b_hi, b_lo, bytes;
    __host__ __device__ explicit StageLayout(int np)
    {
        a_lo = GT_AROWS_BYTES;
        b_hi = 2 * GT_AROWS_BYTES;
        b_lo = b_hi + (uint32_t)np * 128u;
        bytes = b_lo + (uint32_t)np * 128u;
    }
};

// The three MMAs of one 8-deep K step: hi hi, hi lo, lo hi.
__device__ __forceinline__ void mma_split(uint32_t tmem, uint32_t stage, const StageLayout &L, int k8, uint32_t idesc,
                                          bool first)
{
    const uint32_t o = 32u * (uint32_t)k8;
    const uint64_t ah = gt_desc(stage + o), al = gt_desc(stage + L.a_lo + o);
    const uint64_t bh = gt_desc(stage + L.b_hi + o), bl = gt_desc(stage + L.b_lo + o);
    gt_mma(tmem, ah, bh, idesc, first ? 0u : 1u);
    gt_mma(tmem, ah, bl, idesc, 1u);
    gt_mma(tmem, al, bh, idesc, 1u);
}

struct PxArgs {
    int M, K, P;                 // output channels, input channels, pixels
    int np;                      // M rounded up to 16 (the MMA's N)
    int ntiles;                  // pixel tiles of 128
    const float *X;              // X[k * ldx + p]
    int ldx;
    const float *W;              // W(m, k) = transW ? W[k * ldw + m] : W[m * ldw + k]
    int ldw, transW;
    const float *bias;           // nullable, [M]
    float *C;                    // C[m * ldc + p]
    int ldc, act, accumulate;
    uint32_t stage_bytes, bar_off;
    int *err;
};

// Pixel GEMM (see the file comment).  One CTA per SM walks the pixel tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...
__global__ void __launch_bounds__(GT_THREADS, 1) gemm_px_kernel(PxArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *gbase = smem_raw + (base - raw);
    const StageLayout L(a.np);
    const uint32_t bar0 = base + a.bar_off;
    const uint32_t mmad0 = bar0, accf = bar0 + 16;         // per stage: its MMAs are done; the tile is done
    const uint32_t tslot = accf + 8;
    uint32_t *tslot_ptr = reinterpret_cast<uint32_t *>(smem_raw + (tslot - raw));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = (a.K + GT_KC - 1) / GT_KC;              // K chunks per tile

    if (threadIdx.x == 0) {
        mbar_init(mmad0, 1);
        mbar_init(mmad0 + 8, 1);
        mbar_init(accf, 1);
        mbar_init_fence();
    }
    if (warp == 0) gt_tmem_alloc(tslot, 256);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot_ptr;
    const uint32_t idesc = gt_idesc(a.np);

    bool ok = true;
    int chunk = 0, ti = 0;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++ti) {
        const int p0 = t * 128;
        for (int kc = 0; kc < nk; ++kc, ++chunk) {
            const int s = chunk & 1;
            // the MMAs that read this stage two chunks ago are done
            if (chunk >= 2) ok = ok && gt_wait(mmad0 + 8 * s, ((chunk >> 1) - 1) & 1, a.err);
            if (ok) {
                unsigned char *st = gbase + a.stage_bytes * s;
                // X: a warp covers 32 consecutive pixels of one channel quad; the
                // four items of a thread are unrolled so their 16 loads are in
                // flight together (the copy is bound by load latency)
#pragma unroll
                for (int it = threadIdx.x; it < 128 * 8; it += GT_THREADS) {
                    const int px = it & 127, q = it >> 7;
                    const int p = p0 + px, k0 = kc * GT_KC + 4 * q;
                    float v[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        v[j] = (p < a.P && k0 + j < a.K) ? __ldg(a.X + (size_t)(k0 + j) * a.ldx + p) : 0.f;
                    store_split(st, st + L.a_lo, quad_off(px, q), v);
                }
                // W: rows = output channels, zero beyond M and K
                for (int it = threadIdx.x; it < a.np * 8; it += GT_THREADS) {
                    const int m = it >> 3, q = it & 7, k0 = kc * GT_KC + 4 * q;
                    float v[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int k = k0 + j;
                        v[j] = (m < a.M && k < a.K)
                                   ? __ldg(a.transW ? a.W + (size_t)k * a.ldw + m : a.W + (size_t)m * a.ldw + k)
                                   : 0.f;
                    }
                    store_split(st + L.b_hi, st + L.b_lo, quad_off(m, q), v);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // thread writes -> tensor-core reads
            if (!__syncthreads_and(ok)) {
                ok = false;
                break;
            }
            if (threadIdx.x == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sa = base + a.stage_bytes * s;
                const int k8n = min(4, (a.K - kc * GT_KC + 7) / 8);
                for (int k8 = 0; k8 < k8n; ++k8) mma_split(tmem, sa, L, k8, idesc, kc == 0 && k8 == 0);
                gt_commit(mmad0 + 8 * s);
                if (kc == nk - 1) gt_commit(accf);
            }
        }
        if (!ok) break;
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (pixels), 16-column
        // chunks h, h + 2, ... with h = w / 4
        ok = gt_wait(accf, ti & 1, a.err);
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int q4 = warp & 3, h = warp >> 2;
        const int p = p0 + 32 * q4 + lane;
        const uint32_t lane_off = (uint32_t)(32 * q4) << 16;
        for (int c0 = 16 * h; c0 < a.np; c0 += 32) {
            float v[16];
            gt_ld16(tmem + (uint32_t)c0 + lane_off, v);
            if (p >= a.P) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int m = c0 + j;
                if (m >= a.M) continue;
                float y = v[j] + (a.bias ? a.bias[m] : 0.f);
                if (a.act == 1) y = tanhf(y);
                float *c = a.C + (size_t)m * a.ldc + p;
                *c = a.accumulate ? *c + y : y;
            }
        }
        // the accumulator is free for the next tile's MMAs
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (!ok && threadIdx.x == 0) {
        // let the MMAs issued before the failed wait finish before the
        // accumulator is freed (the last use of each stage)
        for (int s = 0; s < 2; ++s)
            if (chunk > s) mbar_wait_bounded(mmad0 + 8 * s, ((chunk - 1 - s) >> 1) & 1, GT_WAIT_NS);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) gt_tmem_free(tmem, 256);
}

struct RedArgs {
    int M, N, K;                 // rows of A and of B (the output is M x N); pixels
    int np;                      // N rounded up to 16 (the MMA's N)
    const float *A, *B;          // A[m * lda + p], B[n * ldb + p]; lda, ldb multiples of 4, 16-byte aligned
    int lda, ldb;
    int nchunks, per;            // pixel chunks of 32; chunks per CTA
    int splits, mblocks;
    uint32_t stage_bytes, bar_off;
    float *part;                 // [splits][N][M]: the CTAs' slices of the product
    int *err;
};

// Four consecutive K values of row `row` (zero beyond rows / K); 16-byte
// loads where the four lie inside the row.
__device__ __forceinline__ void load_quad(const float *X, int ld, int row, int rows, int k0, int K, float (&v)[4])
{
    if (row >= rows || k0 >= K) {
        v[0] = v[1] = v[2] = v[3] = 0.f;
    } else if (k0 + 3 < K) {
        const float4 f = __ldg(reinterpret_cast<const float4 *>(X + (size_t)row * ld + k0));
        v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = k0 + j < K ? __ldg(X + (size_t)row * ld + k0 + j) : 0.f;
    }
}

// Reduction GEMM (see the file comment): CTA (mb, split) multiplies rows
// 128 mb .. of A by B over its pixel chunks and stores the 128 x N partial
// product to its slice.
__global__ void __launch_bounds__(GT_THREADS, 1) gemm_red_kernel(RedArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *gbase = smem_raw + (base - raw);
    const StageLayout L(a.np);
    const uint32_t bar0 = base + a.bar_off;
    const uint32_t mmad0 = bar0, accf = bar0 + 16;
    const uint32_t tslot = accf + 8;
    uint32_t *tslot_ptr = reinterpret_cast<uint32_t *>(smem_raw + (tslot - raw));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mb = blockIdx.x % a.mblocks, sp = blockIdx.x / a.mblocks;
    const int c0 = sp * a.per, c1 = min(a.nchunks, c0 + a.per);
    const int m0 = mb * 128;

    if (threadIdx.x == 0) {
        mbar_init(mmad0, 1);
        mbar_init(mmad0 + 8, 1);
        mbar_init(accf, 1);
        mbar_init_fence();
    }
    if (warp == 0) gt_tmem_alloc(tslot, 256);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot_ptr;
    const uint32_t idesc = gt_idesc(a.np);

    bool ok = true;
    int chunk = 0;
    for (int c = c0; c < c1; ++c, ++chunk) {
        const int s = chunk & 1;
        if (chunk >= 2) ok = ok && gt_wait(mmad0 + 8 * s, ((chunk >> 1) - 1) & 1, a.err);
        if (ok) {
            unsigned char *st = gbase + a.stage_bytes * s;
            const int k0 = c * GT_KC;
            // a warp covers 4 rows x 8 quads: 128-byte runs of each row
            for (int it = threadIdx.x; it < 128 * 8; it += GT_THREADS) {
                const int r = it >> 3, q = it & 7;
                float v[4];
                load_quad(a.A, a.lda, m0 + r, a.M, k0 + 4 * q, a.K, v);
                store_split(st, st + L.a_lo, quad_off(r, q), v);
            }
            for (int it = threadIdx.x; it < a.np * 8; it += GT_THREADS) {
                const int r = it >> 3, q = it & 7;
                float v[4];
                load_quad(a.B, a.ldb, r, a.N, k0 + 4 * q, a.K, v);
                store_split(st + L.b_hi, st + L.b_lo, quad_off(r, q), v);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // thread writes -> tensor-core reads
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = base + a.stage_bytes * s;
            for (int k8 = 0; k8 < 4; ++k8) mma_split(tmem, sa, L, k8, idesc, c == c0 && k8 == 0);
            gt_commit(mmad0 + 8 * s);
            if (c == c1 - 1) gt_commit(accf);
        }
    }
    if (ok && c1 > c0) ok = gt_wait(accf, 0, a.err);
    ok = __syncthreads_and(ok) && c1 > c0;
    // slice layout [N][M]: a warp stores 32 consecutive rows of one column
    float *dst = a.part + (size_t)sp * a.N * a.M;
    const int q4 = warp & 3, h = warp >> 2;
    const int m = m0 + 32 * q4 + lane;
    if (ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t lane_off = (uint32_t)(32 * q4) << 16;
        for (int cc = 16 * h; cc < a.np; cc += 32) {
            float v[16];
            gt_ld16(tmem + (uint32_t)cc + lane_off, v);
            if (m >= a.M) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (cc + j < a.N) dst[(size_t)(cc + j) * a.M + m] = v[j];
        }
    } else {
        if (threadIdx.x == 0)   // let the MMAs issued before a failed wait finish
            for (int s = 0; s < 2; ++s)
                if (chunk > s) mbar_wait_bounded(mmad0 + 8 * s, ((chunk - 1 - s) >> 1) & 1, GT_WAIT_NS);
        // no pixels (or an expired wait): this slice adds nothing
        if (m < a.M)
            for (int n = h; n < a.N; n += 2) dst[(size_t)n * a.M + m] = 0.f;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) gt_tmem_free(tmem, 256);
}

// C[m * ldc + n] (+)= sum over the slices, in slice order.
__global__ void gemm_red_sum_kernel(const float *__restrict__ part, int splits, int M, int N, float *C, int ldc,
                                    int accumulate)
{
    const size_t total = (size_t)M * N;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int n = (int)(i / M), m = (int)(i - (size_t)n * M);
        float s = 0.f;
        for (int k = 0; k < splits; ++k) s += part[(size_t)k * total + i];
        float *c = C + (size_t)m * ldc + n;
        *c = accumulate ? *c + s : s;
    }
}

std::mutex g_gt_mu;
int *g_gt_flag[MAX_DEVICES] = {};

int current_device()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return -1;
    return dev;
}

int *gt_flag(int dev)
{
    std::lock_guard<std::mutex> lk(g_gt_mu);
    if (!g_gt_flag[dev]) {
        int *f = nullptr;
        if (cudaMalloc(&f, sizeof(int)) != cudaSuccess) return nullptr;
        if (cudaMemset(f, 0, sizeof(int)) != cudaSuccess) {
            cudaFree(f);
            return nullptr;
        }
        g_gt_flag[dev] = f;
    }
    return g_gt_flag[dev];
}

int gt_sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

bool capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &st) != cudaSuccess || st != cudaStreamCaptureStatusNone;
}

constexpr int round_up_i(int v, int m) { return (v + m - 1) / m * m; }

}  // namespace

// Thin forms of the same product, memory-bound on the CUDA cores.
// Row dot: C[m][n] (+)= sum_p A[m][p] B(p, n) for N <= 4 (the bias gradients,
// B a vector of ones or the loss's gradient, and the first trunk layer's
// weight gradient, B the 2 coordinates).  One block per row, 16-byte loads,
// a fixed reduction order.
template <int N>
__global__ void __launch_bounds__(512) gemm_rowdot_kernel(int K, const float *__restrict__ A, int lda,
                                                         const float *__restrict__ B, int ldb, int transB,
                                                         float *C, int ldc, int accumulate)
{
    __shared__ float red[4][16];
    const int m = blockIdx.x;
    const float *a = A + (size_t)m * lda;
    float acc[N];
#pragma unroll
    for (int n = 0; n < N; ++n) acc[n] = 0.f;
    const bool vec = ((lda | (transB ? ldb : 4)) & 3) == 0 && ((uintptr_t)A & 15) == 0 &&
                     (!transB || ((uintptr_t)B & 15) == 0);
    const int kv = vec ? K / 4 * 4 : 0;
    // four 16-byte loads of a thread in flight at once (the loop is bound by
    // memory latency, not bandwidth, at one block per row)
#pragma unroll 4
    for (int k = 4 * threadIdx.x; k < kv; k += 4 * blockDim.x) {
        const float4 x = __ldg(reinterpret_cast<const float4 *>(a + k));
        for (int n = 0; n < N; ++n) {
            float b0, b1, b2, b3;
            if (transB) {
                const float4 y = __ldg(reinterpret_cast<const float4 *>(B + (size_t)n * ldb + k));
                b0 = y.x; b1 = y.y; b2 = y.z; b3 = y.w;
            } else {
                b0 = __ldg(B + (size_t)k * ldb + n); b1 = __ldg(B + (size_t)(k + 1) * ldb + n);
                b2 = __ldg(B + (size_t)(k + 2) * ldb + n); b3 = __ldg(B + (size_t)(k + 3) * ldb + n);
            }
            acc[n] += x.x * b0 + x.y * b1 + x.z * b2 + x.w * b3;
        }
    }
    for (int k = kv + threadIdx.x; k < K; k += blockDim.x)
        for (int n = 0; n < N; ++n) acc[n] += a[k] * (transB ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int n = 0; n < N; ++n) {
        float v = acc[n];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[n][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < N) {
        float v = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
        float *c = C + (size_t)m * ldc + threadIdx.x;
        *c = accumulate ? *c + v : v;
    }
}

// Small K: C[m][p] = act(sum_{k < K} W(m, k) X[k][p] + bias[m]) (+ C) for
// K <= 4 (the first trunk layer on the 2 coordinates; the head bias's
// rank-one term of the data gradient).  One thread per output, consecutive
// threads on consecutive pixels.
__global__ void __launch_bounds__(256) gemm_smallk_kernel(int M, int P, int K, const float *__restrict__ W, int ldw,
                                                         int transW, const float *__restrict__ X, int ldx,
                                                         const float *__restrict__ bias, float *C, int ldc, int act,
                                                         int accumulate)
{
    const size_t total = (size_t)M * P;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(i / P), p = (int)(i - (size_t)m * P);
        float y = bias ? __ldg(bias + m) : 0.f;
        for (int k = 0; k < K; ++k)
            y += __ldg(transW ? W + (size_t)k * ldw + m : W + (size_t)m * ldw + k) * __ldg(X + (size_t)k * ldx + p);
        if (act == 1) y = tanhf(y);
        float *c = C + (size_t)m * ldc + p;
        *c = accumulate ? *c + y : y;
    }
}

// Shape test of the forms (the arguments of sgemm): 1 pixel GEMM and 2
// reduction GEMM (tensor cores), 3 row dot and 4 small K (CUDA cores,
// memory-bound), 0 the general CUDA-core kernel.
int tgemm_form(int M, int N, int K, const float *A, int lda, bool transA, const float *B, int ldb, bool transB,
               const float *bias, int act)
{
    if (M < 1 || N < 1 || K < 1 || (act != 0 && act != 1)) return 0;
    if (!transB && N >= 1024 && M <= 256 && K >= 8 && K <= 4096 && ldb >= N && lda >= 1) return 1;
    if (!transA && transB && K >= 4096 && M >= 16 && N >= 16 && N <= 256 && !bias && act == 0 && lda % 4 == 0 &&
        ldb % 4 == 0 && lda >= K && ldb >= K && aligned16(A) && aligned16(B))
        return 2;
    if (!transA && N <= 4 && K >= 1024 && !bias && act == 0 && lda >= K) return 3;
    if (!transB && K <= 4 && N >= 1024 && M <= 65535 && ldb >= N) return 4;
    return 0;
}

// Pixel chunks per CTA and CTAs of a reduction GEMM over K pixels.
static void red_split(int M, int K, int nsm, int *per, int *splits)
{
    const int nchunks = (K + GT_KC - 1) / GT_KC, mblocks = (M + 127) / 128;
    const int target = std::max(1, nsm / mblocks);
    *per = std::max(8, (nchunks + target - 1) / target);      // at least 256 pixels per CTA
    *splits = (nchunks + *per - 1) / *per;
}

size_t tgemm_scratch_floats(int M, int N)
{
    // at most one slice per CTA, the CTAs at most one per SM per M block
    return (size_t)std::max(1, gt_sm_count()) * (size_t)M * (size_t)N;
}

ppe_status tgemm(int M, int N, int K, const float *A, int lda, bool transA, const float *B, int ldb, bool transB,
                 float *C, int ldc, const float *bias, int act, bool accumulate, cudaStream_t s, float *scratch,
                 size_t scratch_floats)
{
    const int form = tgemm_form(M, N, K, A, lda, transA, B, ldb, transB, bias, act);
    if (form == 3) {
        const int tb = transB ? 1 : 0, ac = accumulate ? 1 : 0;
        switch (N) {
        case 1: gemm_rowdot_kernel<1><<<M, 512, 0, s>>>(K, A, lda, B, ldb, tb, C, ldc, ac); break;
        case 2: gemm_rowdot_kernel<2><<<M, 512, 0, s>>>(K, A, lda, B, ldb, tb, C, ldc, ac); break;
        case 3: gemm_rowdot_kernel<3><<<M, 512, 0, s>>>(K, A, lda, B, ldb, tb, C, ldc, ac); break;
        default: gemm_rowdot_kernel<4><<<M, 512, 0, s>>>(K, A, lda, B, ldb, tb, C, ldc, ac); break;
        }
        PPE_CUDA_TRY(cudaGetLastError());
        return PPE_OK;
    }
    if (form == 4) {
        const size_t total = (size_t)M * N;
        const unsigned g = (unsigned)std::min<size_t>((total + 255) / 256, 65535u * 16u);
        gemm_smallk_kernel<<<g, 256, 0, s>>>(M, N, K, A, lda, transA ? 1 : 0, B, ldb, bias, C, ldc, act,
                                              accumulate ? 1 : 0);
        PPE_CUDA_TRY(cudaGetLastError());
        return PPE_OK;
    }
    const int dev = current_device();
    if (form == 0 || dev < 0 || (form == 2 && capturing(s)))
        return sgemm(M, N, K, A, lda, transA, B, ldb, transB, C, ldc, bias, act, accumulate, s);
    int *err = gt_flag(dev);
    if (!err) return cuda_status(cudaErrorMemoryAllocation, "tgemm error flag");
    static PerDevice attrs;
    const bool attr_ok = once_per_device(attrs, [](int) {
        const int cap = 227 * 1024;
        return cudaFuncSetAttribute(gemm_px_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) == cudaSuccess &&
               cudaFuncSetAttribute(gemm_red_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) == cudaSuccess;
    });
    if (!attr_ok) return cuda_status(cudaGetLastError(), "cudaFuncSetAttribute(tgemm)");
    const int nsm = gt_sm_count();

    if (form == 1) {
        // C[m][p] = act(W(m, k) X[k][p] + bias) with W = A, X = B
        PxArgs t{};
        t.M = M; t.K = K; t.P = N;
        t.np = round_up_i(M, 16);
        t.ntiles = (N + 127) / 128;
        t.X = B; t.ldx = ldb;
        t.W = A; t.ldw = lda; t.transW = transA ? 1 : 0;
        t.bias = bias; t.C = C; t.ldc = ldc; t.act = act; t.accumulate = accumulate ? 1 : 0;
        t.stage_bytes = StageLayout(t.np).bytes;
        t.bar_off = 2 * t.stage_bytes;
        t.err = err;
        const size_t smem = std::max<size_t>((size_t)t.bar_off + 64 + 1024, 116 * 1024);   // one CTA per SM
        gemm_px_kernel<<<std::min(t.ntiles, nsm), GT_THREADS, smem, s>>>(t);
        PPE_CUDA_TRY(cudaGetLastError());
        return PPE_OK;
    }

    // C[m][n] (+)= sum_p A[m][p] B[n][p]
    RedArgs t{};
    t.M = M; t.N = N; t.K = K;
    t.np = round_up_i(N, 16);
    t.A = A; t.B = B; t.lda = lda; t.ldb = ldb;
    t.nchunks = (K + GT_KC - 1) / GT_KC;
    t.mblocks = (M + 127) / 128;
    red_split(M, K, nsm, &t.per, &t.splits);
    t.stage_bytes = StageLayout(t.np).bytes;
    t.bar_off = 2 * t.stage_bytes;
    t.err = err;
    // the slices: the caller's scratch (its own stream), else stream-ordered
    // memory from the device's pool; GEMMs on different streams never share them
    const size_t need = (size_t)t.splits * M * N;
    const bool own = !(scratch && scratch_floats >= need);
    if (own) PPE_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void **>(&t.part), need * sizeof(float), s));
    else t.part = scratch;
    const size_t smem = std::max<size_t>((size_t)t.bar_off + 64 + 1024, 116 * 1024);
    gemm_red_kernel<<<t.mblocks * t.splits, GT_THREADS, smem, s>>>(t);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        const size_t total = (size_t)M * N;
        const unsigned g = (unsigned)std::min<size_t>((total + 255) / 256, 1024);
        gemm_red_sum_kernel<<<g, 256, 0, s>>>(t.part, t.splits, M, N, C, ldc, accumulate ? 1 : 0);
        e = cudaGetLastError();
    }
    if (own) cudaFreeAsync(t.part, s);
    if (e != cudaSuccess) return cuda_status(e, "tgemm reduction");
    return PPE_OK;
}

// Error flag raised by a tensor-core GEMM whose bounded wait expired.
int tgemm_error()
{
    const int dev = current_device();
    int *f = dev >= 0 ? gt_flag(dev) : nullptr;
    int v = 0;
    if (f) cudaMemcpy(&v, f, sizeof(int), cudaMemcpyDeviceToHost);
    return v;
}

}  // namespace ppe
