// tcgen05 implicit-GEMM 3x3 convolution for sm_103a (the Mesh-Convs of the
// DeepONet branch, Sec. 2.4).
//
// GEMM view of one CTA: M = 128 output pixels (a TW x TH patch of one image),
// N = a slice of the output channels, K = 9 taps x Cin input channels.
// For every (tap, channel block) the A tile is a TMA box load of the NHWC
// activation tensor at the tap's shifted coordinates; coordinates outside the
// image are zero-filled by the TMA unit, which is exactly the convolution's
// zero padding.  The B tile is a TMA box load of the packed weights
// [Cout][9*Cin] (K-major).  Both land in shared memory in the swizzled
// K-major layout the tensor cores read; one elected thread issues
// tcgen05.mma (BF16 x BF16 -> FP32) into a TMEM accumulator, and all
// sixteen warps read it back with tcgen05.ld for the fused epilogue (bias,
// GELU, per-pixel Mesh-Conv weight of the consumer layer, BF16 stores): the
// epilogue's SIMT work, not the MMAs, sets the time of these small GEMMs, so
// it gets four warps per TMEM lane quarter.
//
// The input tensor arrives already multiplied by this layer's eta (the
// producing kernel applies it), so the A operand is loaded as is.
//
// Every wait is bounded: on expiry the CTA records an error flag, skips the
// remaining work, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "net_internal.h"
#include "net_kernels.cuh"
#include "tma.cuh"

namespace ppe {

namespace {

constexpr int TC_M = 128;
constexpr int TC_MAX_STAGES = 8;
constexpr long long TC_WAIT_NS = 1000000000LL;   // 1 s bound on every wait
constexpr int TC_THREADS = 512;                  // 16 warps: 2 issue roles, all 16 in the epilogue
constexpr int TC_GROUPS = TC_THREADS / 128;      // epilogue column groups
constexpr uint32_t TC_BAR_BYTES = 256;           // barriers and the TMEM slot, before the bias

struct TcArgs {
    int B, H, W, cin, cout, n_tile, tw, th, tiles_x, tiles_y, kblocks, stages, tmem_cols;
    uint32_t bar_off;       // byte offset of the barriers: past both the pipeline and the epilogue staging
    const float *bias;
    Epi epi;
    int *err;
};

// Bounded wait; returns false (and raises the error flag) on expiry.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *err)
{
    if (mbar_wait_bounded(bar, parity, TC_WAIT_NS)) return true;
    atomicExch(err, 1);
    return false;
}

// Shared-memory matrix descriptor of a K-major operand in the swizzled
// canonical layout: rows of SW bytes, 8-row atoms of 8*SW bytes.
template <int SW> __device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    constexpr uint64_t layout = SW == 128 ? 2ull : (SW == 64 ? 4ull : 6ull);
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);            // start address
    d |= (uint64_t)1 << 16;                              // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)((8 * SW) >> 4) << 32;                // stride byte offset: one 8-row atom
    d |= (uint64_t)1 << 46;                              // descriptor version
    d |= layout << 61;                                   // swizzle mode
    return d;
}

// kind::f16 instruction descriptor: BF16 x BF16 -> FP32, both K-major.
__device__ __forceinline__ uint32_t instr_desc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
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

template <int BK>
__global__ void __launch_bounds__(TC_THREADS, 2)
    conv_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcArgs a)
{
    constexpr int SW = BK * 2;                 // swizzle span = row bytes
    constexpr uint32_t A_BYTES = TC_M * BK * 2;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t b_bytes = (uint32_t)a.n_tile * BK * 2;
    const uint32_t tx_bytes = A_BYTES + b_bytes;                      // bytes landed per stage
    const uint32_t stage_bytes = (tx_bytes + 1023u) & ~1023u;         // 1024-aligned stage stride
    const uint32_t bar0 = base + a.bar_off;                    // full[8], empty[8], acc, TMEM slot, bias
    const uint32_t full0 = bar0, empty0 = bar0 + 8 * TC_MAX_STAGES, accb = bar0 + 16 * TC_MAX_STAGES;
    const uint32_t tslot = accb + 8;
    unsigned char *gbase = smem_raw + (base - raw);
    uint32_t *tslot_ptr = reinterpret_cast<uint32_t *>(gbase + (tslot - base));
    float *bias_s = reinterpret_cast<float *>(gbase + a.bar_off + TC_BAR_BYTES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x % (a.tiles_x * a.tiles_y), img = blockIdx.x / (a.tiles_x * a.tiles_y);
    const int x0 = (tile % a.tiles_x) * a.tw, y0 = (tile / a.tiles_x) * a.th;
    const int n0 = blockIdx.y * a.n_tile;
    const int cblocks = a.cin / BK;

    for (int i = threadIdx.x; i < a.n_tile; i += TC_THREADS) bias_s[i] = a.bias ? a.bias[n0 + i] : 0.f;
    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(accb, 1);
        mbar_init_fence();
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
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

    if (warp == 0 && lane == 0) {
        // producer: TMA loads of the A (activation) and B (weight) tiles
        bool ok = true;
        int armed = 0;
        for (int kb = 0; kb < a.kblocks && ok; ++kb) {
            int s = kb % a.stages;
            uint32_t ph = (kb / a.stages) & 1;
            ok = mbar_wait(empty0 + 8 * s, ph ^ 1, a.err);
            if (!ok) break;
            int tap = kb / cblocks, c0 = (kb % cblocks) * BK;
            int ky = tap / 3, kx = tap % 3;
            uint32_t sa = base + stage_bytes * s, sb = sa + A_BYTES;
            mbar_expect_tx(full0 + 8 * s, tx_bytes);
            tma_load_4d(sa, &tmA, full0 + 8 * s, c0, x0 + kx - 1, y0 + ky - 1, img);
            tma_load_2d(sb, &tmB, full0 + 8 * s, tap * a.cin + c0, n0);
            armed = kb + 1;
        }
        if (!ok) {
            // let copies already in flight land before the CTA leaves
            for (int kb = (armed > a.stages ? armed - a.stages : 0); kb < armed; ++kb)
                mbar_wait(full0 + 8 * (kb % a.stages), (kb / a.stages) & 1, a.err);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = instr_desc(a.n_tile);
        bool ok = true;
        for (int kb = 0; kb < a.kblocks; ++kb) {
            int s = kb % a.stages;
            uint32_t ph = (kb / a.stages) & 1;
            ok = mbar_wait(full0 + 8 * s, ph, a.err);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t sa = base + stage_bytes * s, sb = sa + A_BYTES;
#pragma unroll
            for (int k = 0; k < BK / 16; ++k)
                mma_bf16(tmem, smem_desc<SW>(sa + 32 * k), smem_desc<SW>(sb + 32 * k), idesc, (kb | k) != 0);
            mma_commit(empty0 + 8 * s);
        }
        mma_commit(accb);     // arrives once every MMA issued above has completed
    }
    __syncwarp();
    // epilogue: warp w reads TMEM lane quarter w % 4 (output pixels
    // m = 32 (w % 4) + lane) and the 16-column chunks g, g + G, g + 2G, ... of
    // the accumulator, g = w / 4 and G = TC_THREADS / 128 column groups.  The
    // outputs are staged [128 pixels][n_tile] in the (now idle) pipeline
    // shared memory and written back in 16-byte chunks, consecutive threads
    // taking consecutive chunks of a pixel's channel run.  Pass 0 writes the
    // FP32 pre-activation, pass 1 the BF16 pre-activation, pass 2 the
    // activation (computed once) into out1 and out2 with their per-pixel
    // Mesh-Conv weights.
    int ok = mbar_wait(accb, 0, a.err) ? 1 : 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    ok = __syncthreads_and(ok && *((volatile int *)a.err) == 0);
    const int quarter = warp & 3, group = warp >> 2;
    const int m = quarter * 32 + lane;
    const int px = x0 + m % a.tw, py = y0 + m / a.tw;
    const bool inside = px < a.W && py < a.H;
    const int q = py * a.W + px;
    const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
    unsigned char *stage = gbase;
    for (int pass = 0; pass < 3 && ok; ++pass) {
        void *dst0 = nullptr, *dst1 = nullptr;
        int cs0 = a.cout, co0 = 0, cs1 = a.cout, co1 = 0;
        float sc0 = 1.f, sc1 = 1.f;
        const int es = pass == 0 ? 4 : 2;
        if (pass == 0) {
            dst0 = a.epi.zf_out;
        } else if (pass == 1) {
            dst0 = a.epi.z_out;
        } else {
            // out1 and out2 share one staging layout; out2 alone moves into slot 0
            dst0 = a.epi.out1; cs0 = a.epi.cs1; co0 = a.epi.co1;
            sc0 = (a.epi.eta1 && inside) ? a.epi.eta1[q] : 1.f;
            dst1 = a.epi.out2; cs1 = a.epi.cs2; co1 = a.epi.co2;
            sc1 = (a.epi.eta2 && inside) ? a.epi.eta2[q] : 1.f;
            if (!dst0) { dst0 = dst1; cs0 = cs1; co0 = co1; sc0 = sc1; dst1 = nullptr; }
        }
        if (!dst0) continue;                          // uniform across the block
        const int nout = dst1 ? 2 : 1;
        const bool act = pass == 2 && a.epi.act != 0;
        const int rowb = a.n_tile * es + 16;          // padded staging row (bytes)
        const int plane = TC_M * rowb;                // one output's staging
        for (int c = 16 * group; c < a.n_tile; c += 16 * TC_GROUPS) {
            float v[16];
            tmem_ld16(trow + (uint32_t)c, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float z = v[i] + bias_s[c + i];
                v[i] = act ? gelu_f(z) : z;
            }
            for (int o = 0; o < nout; ++o) {
                const float sc = o == 0 ? sc0 : sc1;
                unsigned char *row = stage + (size_t)o * plane + (size_t)m * rowb + (size_t)c * es;
                if (es == 4) {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        *reinterpret_cast<float4 *>(row + 16 * i) =
                            make_float4(v[4 * i] * sc, v[4 * i + 1] * sc, v[4 * i + 2] * sc, v[4 * i + 3] * sc);
                } else {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        uint4 pk;
                        uint32_t *w = reinterpret_cast<uint32_t *>(&pk);
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            __nv_bfloat162 b2 = __floats2bfloat162_rn(v[8 * h + 2 * i] * sc, v[8 * h + 2 * i + 1] * sc);
                            w[i] = *reinterpret_cast<uint32_t *>(&b2);
                        }
                        *reinterpret_cast<uint4 *>(row + 16 * h) = pk;
                    }
                }
            }
        }
        __syncthreads();
        const int cpr = a.n_tile * es / 16;           // 16-byte chunks per pixel
        for (int k = threadIdx.x; k < nout * TC_M * cpr; k += TC_THREADS) {
            const int o = k / (TC_M * cpr), rem = k - o * (TC_M * cpr);
            const int mm = rem / cpr, off = rem - mm * cpr;
            const int qx = x0 + mm % a.tw, qy = y0 + mm / a.tw;
            if (qx >= a.W || qy >= a.H) continue;
            const size_t pp = ((size_t)img * a.H + qy) * a.W + qx;
            const int cs = o == 0 ? cs0 : cs1, co = o == 0 ? co0 : co1;
            unsigned char *dst = reinterpret_cast<unsigned char *>(o == 0 ? dst0 : dst1);
            const uint4 val = *reinterpret_cast<const uint4 *>(stage + (size_t)o * plane + (size_t)mm * rowb + 16 * off);
            *reinterpret_cast<uint4 *>(dst + (pp * cs + co + n0) * es + 16 * off) = val;
        }
        __syncthreads();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

int *err_flag()
{
    static int *flag = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        if (cudaMalloc(&flag, sizeof(int)) == cudaSuccess) cudaMemset(flag, 0, sizeof(int));
    });
    return flag;
}

int pick_bk(int cin) { return cin % 64 == 0 ? 64 : (cin % 32 == 0 ? 32 : 16); }

}  // namespace

// One-time set-up (driver entry point, error flag, kernel attributes); must
// run outside any stream capture.
ppe_status conv3x3_tc_prepare()
{
    if (!tensor_map_encoder()) {
        set_error("cuTensorMapEncodeTiled unavailable");
        return PPE_ERR_CUDA;
    }
    if (!err_flag()) return cuda_status(cudaErrorMemoryAllocation, "conv3x3_tc error flag");
    static std::once_flag attr_once;
    std::call_once(attr_once, [] {
        const int cap = 227 * 1024;
        cudaFuncSetAttribute(conv_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
        cudaFuncSetAttribute(conv_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
        cudaFuncSetAttribute(conv_tc_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    });
    return PPE_OK;
}

bool conv3x3_tc_supported(const ConvArgs &a)
{
    return a.cin % 16 == 0 && a.cout % 16 == 0 && a.cin >= 16 && a.cout >= 16 && a.H >= 1 && a.W >= 1 &&
           a.B >= 1 && tensor_map_encoder() != nullptr;
}

ppe_status conv3x3_tc(const ConvArgs &a, cudaStream_t s)
{
    if (!conv3x3_tc_supported(a)) {
        set_error("conv3x3_tc: unsupported shape");
        return PPE_ERR_ARG;
    }
    PPE_TRY(conv3x3_tc_prepare());
    auto encode = tensor_map_encoder();
    int *err = err_flag();
    const int bk = pick_bk(a.cin);
    // output patch of 128 pixels: TW x TH with TW a power of two <= 128
    int tw = 8;
    while (tw < a.W && tw < TC_M) tw *= 2;
    int th = TC_M / tw;
    // output-channel slice: the whole of Cout when it fits one MMA (<= 256)
    int n_tile = a.cout;
    while (n_tile > 256) n_tile /= 2;
    if (a.cout % n_tile) n_tile = 16;
    {
        // few output patches (deep U-Net levels): split the output channels so
        // that enough CTAs run; each slice re-reads the activations (L2-resident)
        const long mtiles = (long)((a.W + tw - 1) / tw) * ((a.H + th - 1) / th) * a.B;
        while (mtiles * (a.cout / n_tile) < 128 && n_tile % 32 == 0 && n_tile > 32 && a.cout % (n_tile / 2) == 0)
            n_tile /= 2;                                      // stays a multiple of 16
    }
    int tmem_cols = 32;
    while (tmem_cols < n_tile) tmem_cols *= 2;
    const int stage_bytes = ((TC_M + n_tile) * bk * 2 + 1023) / 1024 * 1024;
    int stages = std::min(TC_MAX_STAGES, (200 * 1024) / stage_bytes);
    stages = std::min(stages, 9 * (a.cin / bk));        // no deeper than the K loop
    if (stages < 2) stages = 2;
    // widest epilogue staging: one FP32 output, or two BF16 outputs
    const size_t staging = std::max((size_t)TC_M * (n_tile * 4 + 16), (size_t)2 * TC_M * (n_tile * 2 + 16));
    const size_t bar_off = (std::max((size_t)stage_bytes * stages, staging) + 127) / 128 * 128;
    const size_t smem = bar_off + TC_BAR_BYTES + (size_t)n_tile * 4 + 1024;   // + alignment slack

    CUtensorMap mA, mB;
    CUtensorMapSwizzle sw = bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                     : (bk == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
    {
        cuuint64_t dims[4] = {(cuuint64_t)a.cin, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.B};
        cuuint64_t strides[3] = {(cuuint64_t)a.cin * 2, (cuuint64_t)a.W * a.cin * 2, (cuuint64_t)a.H * a.W * a.cin * 2};
        cuuint32_t box[4] = {(cuuint32_t)bk, (cuuint32_t)tw, (cuuint32_t)th, 1};
        cuuint32_t es[4] = {1, 1, 1, 1};
        CUresult r = encode(&mA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)a.in, dims, strides, box, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            set_error("cuTensorMapEncodeTiled(activations) failed");
            return PPE_ERR_CUDA;
        }
    }
    {
        cuuint64_t dims[2] = {(cuuint64_t)9 * a.cin, (cuuint64_t)a.cout};
        cuuint64_t strides[1] = {(cuuint64_t)9 * a.cin * 2};
        cuuint32_t box[2] = {(cuuint32_t)bk, (cuuint32_t)n_tile};
        cuuint32_t es[2] = {1, 1};
        CUresult r = encode(&mB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)a.w, dims, strides, box, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            set_error("cuTensorMapEncodeTiled(weights) failed");
            return PPE_ERR_CUDA;
        }
    }
    TcArgs t;
    t.B = a.B; t.H = a.H; t.W = a.W; t.cin = a.cin; t.cout = a.cout; t.n_tile = n_tile;
    t.tw = tw; t.th = th;
    t.tiles_x = (a.W + tw - 1) / tw;
    t.tiles_y = (a.H + th - 1) / th;
    t.kblocks = 9 * (a.cin / bk);
    t.stages = stages;
    t.tmem_cols = tmem_cols;
    t.bar_off = (uint32_t)bar_off;
    t.bias = a.bias;
    t.epi = a.epi;
    t.err = err;
    dim3 grid(t.tiles_x * t.tiles_y * a.B, a.cout / n_tile);
    cudaError_t e;
    if (bk == 64)
        conv_tc_kernel<64><<<grid, TC_THREADS, smem, s>>>(mA, mB, t);
    else if (bk == 32)
        conv_tc_kernel<32><<<grid, TC_THREADS, smem, s>>>(mA, mB, t);
    else
        conv_tc_kernel<16><<<grid, TC_THREADS, smem, s>>>(mA, mB, t);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e, "conv_tc_kernel launch");
    return PPE_OK;
}

// Error flag raised by a tensor-core kernel whose bounded wait expired.
int conv_tc_error()
{
    int *f = err_flag();
    int v = 0;
    if (f) cudaMemcpy(&v, f, sizeof(int), cudaMemcpyDeviceToHost);
    return v;
}

}  // namespace ppe
