// tcgen05 implicit-GEMM 3x3 convolution for sm_103a (the Mesh-Convs of the
// DeepONet branch, Sec. 2.4).
//
// GEMM view of one tile: M = 128 output pixels (an 8 x 16 patch of one
// image), N = a slice of the output channels, K = 9 taps x Cin input channels.
// The activations come in as halo windows: for each channel block and each
// horizontal tap offset kx, one TMA box load brings the 8 x 18 pixel window
// at x0 + kx - 1, y0 - 1 of the NHWC tensor into shared memory, in the
// swizzled K-major layout the tensor cores read (one 8-row atom per window
// row).  The three vertical taps ky are the same window read from atom ky
// on, so one load serves three taps: 432 pixel rows per channel block where
// nine shifted tiles took 1,152.  Coordinates outside the image are
// zero-filled by the TMA unit, which is exactly the convolution's zero
// padding.  The B tiles are TMA box loads of the packed weights
// [Cout][9*Cin] (K-major).  One elected thread issues tcgen05.mma
// (BF16 x BF16 -> FP32) into a TMEM accumulator, and twelve epilogue warps
// read it back with tcgen05.ld for the fused epilogue (bias, GELU, per-pixel
// Mesh-Conv weight of the consumer layer, BF16 stores).
//
// The layers are small GEMMs (M <= 65,536 pixels, N <= 256, K <= 2,304)
// whose time goes into moving operands from L2, so the kernel shares loads
// across a thread-block cluster of cm x cn CTAs: the cn CTAs that compute
// different output-channel slices of one patch receive its activation
// windows from one multicast TMA load, and the cm CTAs that compute the same
// slice of different patches receive its weight tiles from one multicast.
// The issuing is spread over the cluster (the TMA unit's rate in rows is
// what limits a stage): each CTA of a patch row loads one piece of the
// window, and the three taps' weight tiles come from different CTAs of a
// slice column.
// Every CTA of the cluster releases a stage to all of them (multicast MMA
// commit), so a stage is refilled only when every CTA that received it has
// consumed it.
//
// The kernel is persistent: one or two CTAs per SM walk the tiles, the stage
// ring runs on from one tile to the next, and two TMEM accumulators let the
// epilogue of a tile overlap the MMAs of the following one.
//
// The input tensor arrives already multiplied by this layer's eta (the
// producing kernel applies it), so the A operand is loaded as is.
//
// Every wait is bounded: on expiry the CTA records an error flag, skips the
// remaining work, frees its TMEM and returns, after the cluster's CTAs have
// all stopped issuing copies into one another.
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
constexpr int TC_TW = 8, TC_TH = 16;             // output patch (pixels): one 8-row atom per patch row
constexpr int TC_WIN = TC_TW * (TC_TH + 2);      // pixel rows of a halo window (8 x 18)
constexpr int TC_MAX_STAGES = 8;
constexpr long long TC_WAIT_NS = 1000000000LL;   // 1 s bound on every wait
constexpr int TC_THREADS = 512;                  // warp 0: TMA producer, warp 1: MMA issuer, warps 4-15: epilogue
constexpr int TC_EPI_WARP0 = 4;
constexpr int TC_EPI_WARPS = TC_THREADS / 32 - TC_EPI_WARP0;   // three per TMEM lane quarter
constexpr int TC_GROUPS = TC_EPI_WARPS / 4;                      // epilogue column groups
constexpr uint32_t TC_BAR_BYTES = 256;           // barriers and the TMEM slot

struct TcArgs {
    int B, H, W, cin, cout, n_tile, tiles_x, tiles_y, stages, tmem_cols;
    int mtiles, nslices;    // image patches; output-channel slices
    int cm, cn;             // cluster shape: cm patches x cn slices (cm * cn CTAs)
    int units;              // cluster work units: ceil(mtiles / cm) x (nslices / cn)
    int qa, pa;             // a halo window is loaded as pa pieces of qa image rows, one per CTA of a patch row
    uint32_t bar_off;       // byte offset of the barriers, past the pipeline stages
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

// Arrive on the barrier at offset `bar` in every CTA of `mask` once the MMAs
// issued so far have completed.
__device__ __forceinline__ void mma_commit_mc(uint32_t bar, uint16_t mask)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
        "h"(mask)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}

// 16 consecutive BF16 channels (32 bytes, 16-byte aligned), each scaled by sc.
__device__ __forceinline__ void store_bf16x16(bf16 *dst, const float (&v)[16], float sc)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint4 pk;
        uint32_t *w = reinterpret_cast<uint32_t *>(&pk);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __nv_bfloat162 b2 = __floats2bfloat162_rn(v[8 * h + 2 * i] * sc, v[8 * h + 2 * i + 1] * sc);
            w[i] = *reinterpret_cast<uint32_t *>(&b2);
        }
        reinterpret_cast<uint4 *>(dst)[h] = pk;
    }
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
    constexpr int RB = BK * 2;                 // bytes per K-major row = swizzle span
    constexpr uint32_t A_BYTES = TC_WIN * RB;  // one halo window
    constexpr uint32_t ATOM = 8 * RB;          // one 8-row swizzle atom = one window row
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t b_bytes = (uint32_t)a.n_tile * RB;                 // one tap's weight tile
    const uint32_t piece_bytes = (uint32_t)(a.qa * TC_TW) * RB;       // qa window rows
    const uint32_t tx_bytes = a.pa * piece_bytes + 3 * b_bytes;       // bytes landed per stage
    const uint32_t stage_bytes = (tx_bytes + 1023u) & ~1023u;         // 1024-aligned stage stride
    // barriers: full[8], empty[8] of the stages; acc_full[2], acc_empty[2] of
    // the two TMEM accumulators; then the TMEM address slot
    const uint32_t bar0 = base + a.bar_off;
    const uint32_t full0 = bar0, empty0 = bar0 + 8 * TC_MAX_STAGES;
    const uint32_t accf0 = bar0 + 16 * TC_MAX_STAGES, acce0 = accf0 + 16, tslot = acce0 + 16;
    uint32_t *tslot_ptr = reinterpret_cast<uint32_t *>(smem_raw + (tslot - raw));

    // programmatic dependent launch: the next layer may start its set-up
    // (barriers, TMEM, cluster) while this one runs; it reads nothing the
    // previous kernel writes before griddepcontrol.wait below
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cblocks = a.cin / BK;
    const int kiters = 3 * cblocks;            // (channel block, kx) stages per tile
    const int tiles_xy = a.tiles_x * a.tiles_y;
    const int cs = a.cm * a.cn;
    const bool clustered = cs > 1;
    const int rank = clustered ? (int)cluster_rank() : 0;
    const int rm = rank / a.cn, rn = rank - rm * a.cn;
    const int cluster = blockIdx.x / cs, nclusters = gridDim.x / cs;
    const int sgroups = a.nslices / a.cn;
    // multicast masks: the CTAs of this patch row (activations), of this slice column (weights), all
    const uint16_t mask_a = (uint16_t)(((1u << a.cn) - 1u) << (rm * a.cn));
    uint16_t mask_b = 0;
    for (int i = 0; i < a.cm; ++i) mask_b |= (uint16_t)(1u << (i * a.cn + rn));
    const uint16_t mask_all = (uint16_t)((1u << cs) - 1u);

    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, cs);     // every CTA of the cluster releases every stage
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf0 + 8 * b, 1);
            mbar_init(acce0 + 8 * b, TC_EPI_WARPS);
        }
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
    // the cluster's barriers are initialised before any CTA sends it copies or arrivals
    if (clustered)
        cluster_sync();
    else
        __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot_ptr;
    // the previous kernel (this layer's input) has completed and its writes are visible
    asm volatile("griddepcontrol.wait;" ::: "memory");

    // Cluster c walks the units c, c + nclusters, ...; unit u is patch group
    // u / sgroups (patches cm * group + rm) and slice group u % sgroups
    // (slices cn * group + rn).  A patch past the last one (ragged cluster
    // row) is computed on zero-filled loads and not stored.
    if (warp == 0) {
        if (lane == 0) {
            // producer: the halo windows (one CTA per patch row multicasts) and
            // the weight tiles (one CTA per slice column multicasts)
            bool ok = true;
            int it = 0, armed = 0;
            for (int u = cluster; u < a.units && ok; u += nclusters) {
                const int mt = (u / sgroups) * a.cm + rm, ns = (u % sgroups) * a.cn + rn;
                const int img = mt / tiles_xy, tile = mt - img * tiles_xy;
                const int x0 = (tile % a.tiles_x) * TC_TW, y0 = (tile / a.tiles_x) * TC_TH, n0 = ns * a.n_tile;
                for (int kb = 0; kb < kiters; ++kb, ++it) {
                    const int s = it % a.stages;
                    const uint32_t ph = (it / a.stages) & 1;
                    ok = mbar_wait(empty0 + 8 * s, ph ^ 1, a.err);
                    if (!ok) break;
                    const int c0 = (kb / 3) * BK, kx = kb % 3;
                    const uint32_t sa = base + stage_bytes * s, sb = sa + A_BYTES;
                    mbar_expect_tx(full0 + 8 * s, tx_bytes);
                    // the window's piece rn (image rows rn*qa ..) to the CTAs of this patch row
                    if (rn < a.pa) {
                        const int r0 = rn * a.qa;
                        if (a.cn == 1)
                            tma_load_4d(sa, &tmA, full0 + 8 * s, c0, x0 + kx - 1, y0 - 1 + r0, img);
                        else
                            tma_load_4d_mc(sa + r0 * ATOM, &tmA, full0 + 8 * s, c0, x0 + kx - 1, y0 - 1 + r0, img,
                                           mask_a);
                    }
                    // weight tile of tap (ky, kx) from the CTA ky % cm of this slice column
#pragma unroll
                    for (int ky = 0; ky < 3; ++ky) {
                        if (ky % a.cm != rm) continue;
                        const int k0 = (3 * ky + kx) * a.cin + c0;
                        if (a.cm == 1)
                            tma_load_2d(sb + ky * b_bytes, &tmB, full0 + 8 * s, k0, n0);
                        else
                            tma_load_2d_mc(sb + ky * b_bytes, &tmB, full0 + 8 * s, k0, n0, mask_b);
                    }
                    armed = it + 1;
                }
            }
            if (!ok) {
                // let this CTA's own copies in flight land before it leaves
                for (int k = (armed > a.stages ? armed - a.stages : 0); k < armed; ++k)
                    if (!mbar_wait_bounded(full0 + 8 * (k % a.stages), (k / a.stages) & 1, TC_WAIT_NS)) break;
            }
            if (clustered) {
                // every CTA of the cluster has released the last stages: no
                // arrival of theirs is still on its way to this CTA
                for (int k = it; k < it + a.stages; ++k)
                    if (!mbar_wait(empty0 + 8 * (k % a.stages), ((k / a.stages) & 1) ^ 1, a.err)) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: per stage, the three vertical taps of the window
            const uint32_t idesc = instr_desc(a.n_tile);
            bool ok = true;
            int it = 0;
            for (int u = cluster, i = 0; u < a.units && ok; u += nclusters, ++i) {
                const int b = i & 1;
                ok = mbar_wait(acce0 + 8 * b, ((i >> 1) & 1) ^ 1, a.err);   // epilogue drained buffer b
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc = tmem + (uint32_t)(b * a.n_tile);
                for (int kb = 0; kb < kiters; ++kb, ++it) {
                    const int s = it % a.stages;
                    ok = mbar_wait(full0 + 8 * s, (it / a.stages) & 1, a.err);
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = base + stage_bytes * s, sb = sa + A_BYTES;
#pragma unroll
                    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                        for (int k = 0; k < BK / 16; ++k)
                            mma_bf16(acc, smem_desc<RB>(sa + ky * ATOM + 32 * k),
                                     smem_desc<RB>(sb + ky * b_bytes + 32 * k), idesc, (kb | ky | k) != 0);
                    if (clustered)
                        mma_commit_mc(empty0 + 8 * s, mask_all);
                    else
                        mma_commit(empty0 + 8 * s);
                }
                if (!ok) break;
                mma_commit(accf0 + 8 * b);      // arrives once every MMA of this tile has completed
            }
        }
    } else if (warp >= TC_EPI_WARP0) {
        // epilogue: warp w reads TMEM lane quarter w % 4 (output pixels
        // m = 32 (w % 4) + lane) and the 16-column chunks g, g + G, ... of the
        // accumulator, g its column group.  Each thread stores its pixel's
        // channel runs directly (32- or 64-byte pieces): bias, the FP32 and
        // BF16 pre-activations when asked for, and the activation (computed
        // once) into out1 and out2 with their per-pixel Mesh-Conv weights.
        const int quarter = warp & 3, group = (warp - TC_EPI_WARP0) >> 2;
        const int m = quarter * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        const Epi &e = a.epi;
        for (int u = cluster, i = 0; u < a.units; u += nclusters, ++i) {
            const int b = i & 1;
            const bool ok = __all_sync(0xffffffffu, mbar_wait(accf0 + 8 * b, (i >> 1) & 1, a.err));
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int mt = (u / sgroups) * a.cm + rm, ns = (u % sgroups) * a.cn + rn;
            const int img = mt / tiles_xy, tile = mt - img * tiles_xy;
            const int px = (tile % a.tiles_x) * TC_TW + m % TC_TW, py = (tile / a.tiles_x) * TC_TH + m / TC_TW;
            const int n0 = ns * a.n_tile;
            const bool inside = mt < a.mtiles && px < a.W && py < a.H;
            const int q = py * a.W + px;
            const size_t pp = ((size_t)img * a.H + py) * a.W + px;
            const float sc1 = (e.eta1 && inside) ? e.eta1[q] : 1.f;
            const float sc2 = (e.eta2 && inside) ? e.eta2[q] : 1.f;
            const bool act = e.act != 0;
            // pooling sums 2x2 pixel groups across lanes (l, l^1, l^8, l^9 of a
            // warp: two columns of two patch rows), so then every lane takes part
            const bool pool = e.pool_out != nullptr;
            for (int c = 16 * group; c < a.n_tile; c += 16 * TC_GROUPS) {
                float v[16];
                tmem_ld16(tmem + (uint32_t)(b * a.n_tile + c) + lane_off, v);
                if (!inside && !pool) continue;
                const int ch = n0 + c;
#pragma unroll
                for (int k = 0; k < 16; ++k) v[k] += a.bias ? __ldg(a.bias + ch + k) : 0.f;
                if (inside && e.zf_out) {
                    float4 *d = reinterpret_cast<float4 *>(e.zf_out + pp * a.cout + ch);
#pragma unroll
                    for (int k = 0; k < 4; ++k) d[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
                }
                if (inside && e.z_out) store_bf16x16(e.z_out + pp * a.cout + ch, v, 1.f);
                if (e.out1 || e.out2 || pool || e.up_out) {
                    if (act) {
#pragma unroll
                        for (int k = 0; k < 16; ++k) v[k] = gelu_f(v[k]);
                    }
                    if (inside && e.out1) store_bf16x16(e.out1 + pp * e.cs1 + e.co1 + ch, v, sc1);
                    if (inside && e.out2) store_bf16x16(e.out2 + pp * e.cs2 + e.co2 + ch, v, sc2);
                    if (inside && e.up_out) {
                        // nearest 2x: the pixel's four children on the fine grid
                        const int Wf = 2 * a.W;
#pragma unroll
                        for (int d = 0; d < 4; ++d) {
                            const int fx = 2 * px + (d & 1), fy = 2 * py + (d >> 1);
                            const size_t pf = ((size_t)img * 2 * a.H + fy) * Wf + fx;
                            store_bf16x16(e.up_out + pf * e.up_cs + ch, v, e.up_eta ? e.up_eta[fy * Wf + fx] : 1.f);
                        }
                    }
                    if (pool) {
#pragma unroll
                        for (int k = 0; k < 16; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], 1);
#pragma unroll
                        for (int k = 0; k < 16; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], 8);
                        if (inside && (lane & 9) == 0) {
                            const int Wc = a.W >> 1, Hc = a.H >> 1, xc = px >> 1, yc = py >> 1;
                            const size_t pc = ((size_t)img * Hc + yc) * Wc + xc;
                            store_bf16x16(e.pool_out + pc * e.pool_cs + ch, v,
                                          0.25f * (e.pool_eta ? e.pool_eta[yc * Wc + xc] : 1.f));
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(acce0 + 8 * b);     // buffer b may be overwritten
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
    // no CTA leaves while another of its cluster may still write into it
    if (clustered) cluster_sync();
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

// Error flag of the tensor-core kernels, one per device (allocated on first
// use with that device current).
std::mutex g_flag_mu;
int *g_flag[MAX_DEVICES] = {};

int *err_flag()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return nullptr;
    std::lock_guard<std::mutex> lk(g_flag_mu);
    if (!g_flag[dev]) {
        int *f = nullptr;
        if (cudaMalloc(&f, sizeof(int)) != cudaSuccess) return nullptr;
        if (cudaMemset(f, 0, sizeof(int)) != cudaSuccess) {
            cudaFree(f);
            return nullptr;
        }
        g_flag[dev] = f;
    }
    return g_flag[dev];
}

int sm_count()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    if (!cache[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = n > 0 ? n : 1;
    }
    return cache[dev];
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
    // the shared-memory opt-in is a per-device attribute of each kernel
    static PerDevice attrs;
    const bool ok = once_per_device(attrs, [](int) {
        const int cap = 227 * 1024;
        return cudaFuncSetAttribute(conv_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) ==
                   cudaSuccess &&
               cudaFuncSetAttribute(conv_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) ==
                   cudaSuccess &&
               cudaFuncSetAttribute(conv_tc_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) ==
                   cudaSuccess;
    });
    if (!ok) return cuda_status(cudaGetLastError(), "cudaFuncSetAttribute(conv_tc_kernel)");
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
    if (a.epi.pool_out && (a.H % 2 || a.W % 2)) {
        set_error("conv3x3_tc: a fused 2x2 pooling needs even H and W");
        return PPE_ERR_ARG;
    }
    auto encode = tensor_map_encoder();
    int *err = err_flag();
    const int bk = pick_bk(a.cin);
    const int rb = 2 * bk;
    // Output-channel slice.  A stage delivers a halo window (144 rows) and
    // three weight tiles (3 n rows) into every CTA that uses it, and what
    // bounds these layers is the bytes an SM takes in (about 30 per cycle,
    // measured, multicast or not).  Per SM that is ceil(tiles / SMs) x stages
    // per tile x the stage's rows: wide slices reuse a window over more output
    // channels, narrow ones spread few patches over more SMs.  Take the width
    // (a divisor of Cout, 16..128) that minimises it, the wider on ties.
    const int nsm = sm_count();
    const int tiles_x = (a.W + TC_TW - 1) / TC_TW, tiles_y = (a.H + TC_TH - 1) / TC_TH;
    const long mtiles = (long)tiles_x * tiles_y * a.B;
    const int kiters = 3 * (a.cin / bk);
    int n_tile = 0;
    double best = 0.0;
    for (int n = std::min(a.cout, 128); n >= 16; --n) {
        if (a.cout % n || n % 16) continue;
        const long tiles = mtiles * (a.cout / n);
        const double per_sm = (double)((tiles + nsm - 1) / nsm) * kiters * (TC_WIN + 3 * n);
        if (n_tile == 0 || per_sm < best) {
            best = per_sm;
            n_tile = n;
        }
    }
    const int nslices = a.cout / n_tile;
    // cluster: cn slices of one patch (multicast activations) x cm patches
    // of one slice (multicast weights), at most 4 CTAs: clusters of 8 at one
    // CTA per SM (about 190 KB of shared memory each) were measured to run
    // in two waves where those of 4 ran in one
    int cn = 1;
    for (int d = 4; d >= 2; --d)
        if (nslices % d == 0) { cn = d; break; }
    // pairs of patches share their weight loads when there are patches enough
    // to keep every SM busy with pairs
    const int cm = (cn <= 2 && mtiles >= nsm / 2) ? 2 : 1;
    const int cs = cm * cn;
    const long units = (mtiles + cm - 1) / cm * (nslices / cn);
    // the cn CTAs of a patch row each load a piece of its halo windows: qa
    // image rows, the smallest divisor of the window height that needs at
    // most cn pieces
    int qa = TC_TH + 2;
    for (int d = 1; d <= TC_TH + 2; ++d)
        if ((TC_TH + 2) % d == 0 && (TC_TH + 2) / d <= cn) { qa = d; break; }
    const int pa = (TC_TH + 2) / qa;
    int tmem_cols = 32;                                       // two accumulators of n_tile columns
    while (tmem_cols < 2 * n_tile) tmem_cols *= 2;
    const int stage_bytes = ((TC_WIN + 3 * n_tile) * rb + 1023) / 1024 * 1024;
    // two CTAs per SM when a pipeline of three or more stages fits in half the
    // shared memory and both CTAs' accumulators fit the 512 TMEM columns
    int ctas_per_sm = 2;
    int stages = std::min(TC_MAX_STAGES, (110 * 1024) / stage_bytes);
    if (stages < 3 || tmem_cols > 256 || mtiles * nslices <= nsm) {
        ctas_per_sm = 1;
        stages = std::min(TC_MAX_STAGES, (200 * 1024) / stage_bytes);
    }
    if (stages < 2) stages = 2;
    const size_t bar_off = (size_t)stage_bytes * stages;
    size_t smem = bar_off + TC_BAR_BYTES + 1024;             // + alignment slack
    // one CTA per SM: claim more than half the shared memory, so that no second
    // CTA lands on the SM and waits for the first one's TMEM
    if (ctas_per_sm == 1) smem = std::max(smem, (size_t)116 * 1024);

    CUtensorMap mA, mB;
    CUtensorMapSwizzle sw = bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                     : (bk == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
    {
        cuuint64_t dims[4] = {(cuuint64_t)a.cin, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.B};
        cuuint64_t strides[3] = {(cuuint64_t)a.cin * 2, (cuuint64_t)a.W * a.cin * 2, (cuuint64_t)a.H * a.W * a.cin * 2};
        cuuint32_t box[4] = {(cuuint32_t)bk, (cuuint32_t)TC_TW, (cuuint32_t)qa, 1};
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
    t.tiles_x = tiles_x;
    t.tiles_y = tiles_y;
    t.stages = stages;
    t.tmem_cols = tmem_cols;
    t.mtiles = (int)mtiles;
    t.nslices = nslices;
    t.cm = cm;
    t.cn = cn;
    t.units = (int)units;
    t.qa = qa;
    t.pa = pa;
    t.bar_off = (uint32_t)bar_off;
    t.bias = a.bias;
    t.epi = a.epi;
    t.err = err;
    // persistent: one or two CTAs per SM in clusters of cs, each cluster
    // walking its share of the units
    const long clusters = std::min<long>(units, std::max(1L, (long)nsm * ctas_per_sm / cs));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(clusters * cs));
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    // the layer's set-up overlaps the previous kernel's tail (measured: a
    // 256^2 inference 218 -> 196 us with L2 flushed)
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    cudaError_t e;
    if (bk == 64)
        e = cudaLaunchKernelEx(&cfg, conv_tc_kernel<64>, mA, mB, t);
    else if (bk == 32)
        e = cudaLaunchKernelEx(&cfg, conv_tc_kernel<32>, mA, mB, t);
    else
        e = cudaLaunchKernelEx(&cfg, conv_tc_kernel<16>, mA, mB, t);
    if (e == cudaSuccess) e = cudaGetLastError();
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
