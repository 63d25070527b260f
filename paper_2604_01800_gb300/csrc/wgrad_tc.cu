// tcgen05 weight gradient of the 3x3 Mesh-Conv (the training step of
// Sec. 2.4, Eq. 18): for every tap (ky, kx)
//     dW[co][ci][3 ky + kx] += sum over pixels p of dZ[p][co] * X[p + (kx-1, ky-1)][ci]
// with X the layer's (eta-weighted) input, zero outside the image.
//
// GEMM view: D[m][n] = sum_k A[m][k] B[n][k] with K = pixels, so both operands
// are read MN-major: shared-memory rows are pixels, each row holds a run of
// channels (the NHWC tensors as they are).  A is the input X, B is dZ.
// A CTA owns one horizontal tap offset kx and walks a range of 8 x 16 pixel
// patches; per patch the TMA unit brings the 8 x 18 halo window of X at
// x0 + kx - 1, y0 - 1 and the patch of dZ.  A window row of 8 pixels is one
// 8-row swizzle atom along K, so the vertical taps are the window read from
// atom ky on.  For Cin <= 64 the three vertical taps share one MMA: M = 128
// rows are Cin-channel chunks whose stride is one window row, so chunk j is
// the window shifted by j rows (rows of a fourth, unused shift are dropped).
// For Cin >= 128 each vertical tap has its own accumulator over a 128-channel
// block.  The accumulators stay in TMEM over all of the CTA's patches; the
// epilogue adds them to dW once (FP32 atomics, other CTAs own other pixels).
//
// Every wait is bounded: on expiry the CTA raises the error flag, skips the
// remaining work, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "net_internal.h"
#include "tma.cuh"

namespace ppe {

namespace {

constexpr int WG_TW = 8, WG_TH = 16;                // pixel patch: one swizzle atom (8 pixels) per patch row
constexpr int WG_WIN_ROWS = WG_TW * (WG_TH + 2);    // 144 pixel rows of a halo window
constexpr int WG_THREADS = 256;                     // warp 0 TMA, warp 1 MMA, warps 4-7 epilogue
constexpr int WG_MAX_STAGES = 8;
constexpr long long WG_WAIT_NS = 1000000000LL;

struct WgArgs {
    int B, H, W, cin, cout;
    int tiles_x, tiles_y, npatch;   // patches of the batch
    int per;                        // patches per CTA
    int splits;                     // CTAs per (kx, channel block)
    int mblocks, nblocks;           // 128-channel blocks of Cin (Cin >= 128), output-channel blocks
    int ncols;                      // output channels per CTA (N of the MMA)
    int cx, cz;                     // channels per TMA box of X (32 or 64) and of dZ (32 or 64)
    int nacc;                       // accumulators (TMEM column blocks of ncols)
    int stages, tmem_cols;
    uint32_t x_bytes, z_off, stage_bytes, bar_off;   // X region, dZ region offset, stage stride, barriers
    float *dW;
    int *err;
};

__device__ __forceinline__ bool wg_wait(uint32_t bar, uint32_t parity, int *err)
{
    if (mbar_wait_bounded(bar, parity, WG_WAIT_NS)) return true;
    atomicExch(err, 1);
    return false;
}

// Descriptor of an MN-major operand in the swizzled canonical layout: rows of
// SW bytes hold SW/2 consecutive MN elements; 8 rows (consecutive K) form an
// atom; lbo = byte stride between MN chunks, sbo = between 8-row K groups.
template <int SW> __device__ __forceinline__ uint64_t mn_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    constexpr uint64_t layout = SW == 128 ? 2ull : (SW == 64 ? 4ull : 6ull);
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= layout << 61;
    return d;
}

// kind::f16, BF16 x BF16 -> FP32, M = 128, both operands MN-major.
__device__ __forceinline__ uint32_t wg_idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void wg_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void wg_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void wg_ld16(uint32_t taddr, float (&v)[16])
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

template <int SWX, int SWZ>
__global__ void __launch_bounds__(WG_THREADS, 1)
    wgrad_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmZ, WgArgs a)
{
    constexpr uint32_t ATOM_X = 8 * SWX, ATOM_Z = 8 * SWZ;   // one 8-pixel row of the window / patch
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t bar0 = base + a.bar_off;
    const uint32_t full0 = bar0, empty0 = bar0 + 8 * WG_MAX_STAGES, accf = bar0 + 16 * WG_MAX_STAGES;
    const uint32_t tslot = accf + 8;
    uint32_t *tslot_ptr = reinterpret_cast<uint32_t *>(smem_raw + (tslot - raw));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // CTA -> (kx, M block, N block, pixel split)
    int c = blockIdx.x;
    const int split = c % a.splits;
    c /= a.splits;
    const int nb = c % a.nblocks;
    c /= a.nblocks;
    const int mb = c % a.mblocks;
    const int kx = c / a.mblocks;
    const int p0 = split * a.per, p1 = min(a.npatch, p0 + a.per);
    const int co0 = nb * a.ncols, ci0 = mb * 128;
    const bool stacked = a.cin <= 64;                 // three vertical taps in one MMA
    const int xchunks = stacked ? 1 : 2;              // X boxes per stage
    const int zchunks = a.ncols / a.cz;               // dZ boxes per stage
    const uint32_t xbox = (uint32_t)WG_WIN_ROWS * SWX, zbox = (uint32_t)(WG_TW * WG_TH) * SWZ;
    const uint32_t tx_bytes = xchunks * xbox + zchunks * zbox;
    const int tiles_xy = a.tiles_x * a.tiles_y;

    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(accf, 1);
        mbar_init_fence();
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmX) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmZ) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tslot),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot_ptr;

    if (warp == 0) {
        if (lane == 0) {
            // producer: per patch, the X window of this kx (one or two channel
            // boxes) and the dZ patch (one box per channel chunk)
            bool ok = true;
            int it = 0, armed = 0;
            for (int p = p0; p < p1 && ok; ++p, ++it) {
                const int s = it % a.stages;
                ok = wg_wait(empty0 + 8 * s, ((it / a.stages) & 1) ^ 1, a.err);
                if (!ok) break;
                const int img = p / tiles_xy, t = p - img * tiles_xy;
                const int x0 = (t % a.tiles_x) * WG_TW, y0 = (t / a.tiles_x) * WG_TH;
                const uint32_t sx = base + a.stage_bytes * s, sz = sx + a.z_off;
                mbar_expect_tx(full0 + 8 * s, tx_bytes);
                for (int j = 0; j < xchunks; ++j)
                    tma_load_4d(sx + j * xbox, &tmX, full0 + 8 * s, ci0 + j * a.cx, x0 + kx - 1, y0 - 1, img);
                for (int j = 0; j < zchunks; ++j)
                    tma_load_4d(sz + j * zbox, &tmZ, full0 + 8 * s, co0 + j * a.cz, x0, y0, img);
                armed = it + 1;
            }
            if (!ok) {
                for (int k = (armed > a.stages ? armed - a.stages : 0); k < armed; ++k)
                    if (!mbar_wait_bounded(full0 + 8 * (k % a.stages), (k / a.stages) & 1, WG_WAIT_NS)) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = wg_idesc(a.ncols);
            // stacked: chunk stride one window row; per vertical tap: the second
            // 64-channel box of the window
            const uint32_t lbo_x = stacked ? ATOM_X : xbox, lbo_z = zbox;
            const int shift = stacked ? 128 / a.cin : 1;   // window rows between accumulators
            bool ok = true;
            int it = 0;
            for (int p = p0; p < p1 && ok; ++p, ++it) {
                const int s = it % a.stages;
                ok = wg_wait(full0 + 8 * s, (it / a.stages) & 1, a.err);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sx = base + a.stage_bytes * s, sz = sx + a.z_off;
#pragma unroll 1
                for (int k = 0; k < WG_TW * WG_TH / 16; ++k) {          // 16 pixels = two K atoms
                    const uint64_t bd = mn_desc<SWZ>(sz + 2 * k * ATOM_Z, lbo_z, ATOM_Z);
                    for (int q = 0; q < a.nacc; ++q) {
                        const uint64_t ad = mn_desc<SWX>(sx + (q * shift + 2 * k) * ATOM_X, lbo_x, ATOM_X);
                        wg_mma(tmem + (uint32_t)(q * a.ncols), ad, bd, idesc, (p > p0 || k > 0) ? 1u : 0u);
                    }
                }
                wg_commit(empty0 + 8 * s);
            }
            if (ok && p1 > p0) wg_commit(accf);
        }
    } else if (warp >= 4) {
        // epilogue: warp 4 + q reads TMEM lanes 32q .. 32q + 31 (D rows)
        const int q4 = warp - 4;
        const int r = 32 * q4 + lane;
        const bool ok = p1 > p0 && __all_sync(0xffffffffu, wg_wait(accf, 0, a.err));
        if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t lane_off = (uint32_t)(32 * q4) << 16;
            for (int q = 0; q < a.nacc; ++q) {
                // row r of accumulator q -> (ky, ci)
                int ky, ci;
                if (stacked) {
                    ky = q * (128 / a.cin) + r / a.cin;
                    ci = r % a.cin;
                } else {
                    ky = q;
                    ci = ci0 + r;
                }
                const bool valid = ky < 3 && ci < a.cin;
                for (int cc = 0; cc < a.ncols; cc += 16) {
                    float v[16];
                    wg_ld16(tmem + (uint32_t)(q * a.ncols + cc) + lane_off, v);
                    if (!valid) continue;
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const int co = co0 + cc + k;
                        atomicAdd(a.dW + ((size_t)co * a.cin + ci) * 9 + 3 * ky + kx, v[k]);
                    }
                }
            }
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
}

std::mutex g_wg_mu;
int *g_wg_flag[MAX_DEVICES] = {};

int *wg_flag()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return nullptr;
    std::lock_guard<std::mutex> lk(g_wg_mu);
    if (!g_wg_flag[dev]) {
        int *f = nullptr;
        if (cudaMalloc(&f, sizeof(int)) != cudaSuccess) return nullptr;
        if (cudaMemset(f, 0, sizeof(int)) != cudaSuccess) {
            cudaFree(f);
            return nullptr;
        }
        g_wg_flag[dev] = f;
    }
    return g_wg_flag[dev];
}

int wg_sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

}  // namespace

bool wgrad_tc_supported(int cin, int cout)
{
    const bool cin_ok = cin == 32 || cin == 64 || (cin % 128 == 0 && cin <= 1024);
    return cin_ok && cout % 32 == 0 && cout >= 32 && cout <= 1024 && tensor_map_encoder() != nullptr;
}

// dW[co][ci][9] += the weight gradient of one layer (dZ [B][H][W][cout] and
// X [B][H][W][cin], BF16 NHWC).  PPE_ERR_ARG for shapes outside the kernel.
ppe_status wgrad_tc(const bf16 *dZ, const bf16 *X, int B, int H, int W, int cin, int cout, float *dW,
                    cudaStream_t s)
{
    if (!wgrad_tc_supported(cin, cout) || B < 1 || H < 1 || W < 1) {
        set_error("wgrad_tc: unsupported shape");
        return PPE_ERR_ARG;
    }
    auto encode = tensor_map_encoder();
    int *err = wg_flag();
    if (!err) return cuda_status(cudaErrorMemoryAllocation, "wgrad_tc error flag");
    static PerDevice attrs;
    const bool attr_ok = once_per_device(attrs, [](int) {
        const int cap = 227 * 1024;
        return cudaFuncSetAttribute(wgrad_tc_kernel<64, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) ==
                   cudaSuccess &&
               cudaFuncSetAttribute(wgrad_tc_kernel<64, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) ==
                   cudaSuccess &&
               cudaFuncSetAttribute(wgrad_tc_kernel<128, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) ==
                   cudaSuccess &&
               cudaFuncSetAttribute(wgrad_tc_kernel<128, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) ==
                   cudaSuccess;
    });
    if (!attr_ok) return cuda_status(cudaGetLastError(), "cudaFuncSetAttribute(wgrad_tc_kernel)");

    WgArgs t{};
    t.B = B; t.H = H; t.W = W; t.cin = cin; t.cout = cout;
    t.tiles_x = (W + WG_TW - 1) / WG_TW;
    t.tiles_y = (H + WG_TH - 1) / WG_TH;
    t.npatch = B * t.tiles_x * t.tiles_y;
    const bool stacked = cin <= 64;
    t.cx = cin == 32 ? 32 : 64;
    t.mblocks = stacked ? 1 : cin / 128;
    t.nacc = stacked ? (cin == 32 ? 1 : 2) : 3;
    // output channels per CTA: the accumulators fit the 512 TMEM columns
    t.ncols = cout;
    while (t.nacc * t.ncols > 512 || t.ncols > 256) t.ncols /= 2;
    if (t.ncols % 32) {
        set_error("wgrad_tc: unsupported output-channel count");
        return PPE_ERR_ARG;
    }
    t.nblocks = cout / t.ncols;
    t.cz = t.ncols % 64 == 0 ? 64 : 32;             // dZ boxes of 64 channels where they divide the slice
    t.tmem_cols = 32;
    while (t.tmem_cols < t.nacc * t.ncols) t.tmem_cols *= 2;
    const uint32_t swx = 2 * t.cx, swz = 2 * t.cz;
    // X region: the window (one or two boxes) plus one window row read by the
    // unused fourth shift of the stacked form
    const uint32_t xrows = stacked ? WG_WIN_ROWS + 8 : 2 * WG_WIN_ROWS;
    t.x_bytes = xrows * swx;
    t.z_off = (t.x_bytes + 1023u) & ~1023u;
    const uint32_t zbytes = (uint32_t)(t.ncols / t.cz) * WG_TW * WG_TH * swz;
    t.stage_bytes = (t.z_off + zbytes + 1023u) & ~1023u;
    t.stages = std::min<int>(WG_MAX_STAGES, (200 * 1024) / t.stage_bytes);
    if (t.stages < 2) {
        set_error("wgrad_tc: stage does not fit shared memory");
        return PPE_ERR_ARG;
    }
    t.bar_off = t.stage_bytes * t.stages;
    const size_t smem = std::max<size_t>((size_t)t.bar_off + 256 + 1024, 116 * 1024);   // one CTA per SM
    // pixel splits: about one CTA per SM over (kx, M block, N block)
    const int nsm = wg_sm_count();
    const int groups = 3 * t.mblocks * t.nblocks;
    t.splits = std::max(1, std::min(t.npatch, nsm / groups));
    t.per = (t.npatch + t.splits - 1) / t.splits;
    t.splits = (t.npatch + t.per - 1) / t.per;
    t.dW = dW;
    t.err = err;

    CUtensorMap mX, mZ;
    {
        cuuint64_t dims[4] = {(cuuint64_t)cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
        cuuint64_t strides[3] = {(cuuint64_t)cin * 2, (cuuint64_t)W * cin * 2, (cuuint64_t)H * W * cin * 2};
        cuuint32_t box[4] = {(cuuint32_t)t.cx, (cuuint32_t)WG_TW, (cuuint32_t)(WG_TH + 2), 1};
        cuuint32_t es[4] = {1, 1, 1, 1};
        CUresult r = encode(&mX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)X, dims, strides, box, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE,
                            swx == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            set_error("cuTensorMapEncodeTiled(wgrad input) failed");
            return PPE_ERR_CUDA;
        }
    }
    {
        cuuint64_t dims[4] = {(cuuint64_t)cout, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
        cuuint64_t strides[3] = {(cuuint64_t)cout * 2, (cuuint64_t)W * cout * 2, (cuuint64_t)H * W * cout * 2};
        cuuint32_t box[4] = {(cuuint32_t)t.cz, (cuuint32_t)WG_TW, (cuuint32_t)WG_TH, 1};
        cuuint32_t es[4] = {1, 1, 1, 1};
        CUresult r = encode(&mZ, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)dZ, dims, strides, box, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE,
                            swz == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            set_error("cuTensorMapEncodeTiled(wgrad dZ) failed");
            return PPE_ERR_CUDA;
        }
    }
    const dim3 grid((unsigned)(groups * t.splits));
    if (swx == 64 && swz == 64)
        wgrad_tc_kernel<64, 64><<<grid, WG_THREADS, smem, s>>>(mX, mZ, t);
    else if (swx == 64)
        wgrad_tc_kernel<64, 128><<<grid, WG_THREADS, smem, s>>>(mX, mZ, t);
    else if (swz == 64)
        wgrad_tc_kernel<128, 64><<<grid, WG_THREADS, smem, s>>>(mX, mZ, t);
    else
        wgrad_tc_kernel<128, 128><<<grid, WG_THREADS, smem, s>>>(mX, mZ, t);
    PPE_CUDA_TRY(cudaGetLastError());
    return PPE_OK;
}

}  // namespace ppe
