// Persistent solver kernel: single-reduction Jacobi PCG (FP32 or FP64 inner
// vectors) with FP64 residual replacement, interleaved DLSM steps, and the
// compatibility projection / zero-mean normalisation of the Neumann problem.
//
// One cooperative launch runs the per-system state machine of every system of
// a batch.  Each block owns a contiguous range of tiles (of one or a few
// systems).  A step: every block runs the current pass of each of its systems
// over its tiles and writes one partial-sum record per system, then arrives
// at a per-system counter barrier.  After the barrier each block reads the
// partial records of its systems (fixed order, so every block obtains the
// same sums bit for bit) and advances its own copy of each system's state.
// There is no serial finisher: a step costs one barrier plus one read of the
// partial records.  The kernel returns when no system has a pass left (all
// are done or wait for a network direction).
//
// Operator (Sec. 2.1 Eq. 6, volume-scaled): for cell (i,j)
//   (A u)_ij = dy_j [fe_i (u_ij - u_E) + fw_i (u_ij - u_W)]
//            + dx_i [fn_j (u_ij - u_N) + fs_j (u_ij - u_S)]
// with face coefficients f = 2 / (width_left + width_right) and 0 at walls.
//
// PCG variant: Chronopoulos-Gear single-reduction CG with Jacobi
// preconditioning.  Per iteration, with u = D^-1 r:
//   p = u + beta p,  x += alpha p,  r -= alpha A p,
//   gamma' = r.u, delta' = (A u).u on the new residual, beta' = gamma'/gamma,
//   alpha' = gamma' / p'.A p'  with  p'.A p' = delta' + 2 beta' u'.(A p) + beta'^2 p.(A p).
// A p is not stored: each block rebuilds p on its tile plus a two-cell halo
// (from r and the previous p, both read two cells out), applies A on a
// one-cell ring, forms the new residual and u there, and applies A once more
// on the tile.  Stored per iteration: r, p (double-buffered) and the
// correction d, i.e. 12 bytes read and 12 written per cell in FP32.
//
// The iteration pass streams a block's tiles through two shared-memory
// stages: while one tile is computed, the TMA unit loads the next tile's r
// and p windows and its d tile (zero-filled outside the grid, which is the
// Neumann stencil's zero padding), and cp.async brings the next tile's 1-D
// coefficient arrays.  Tiles are 128 cells wide and 16, 8 or 4 rows high: a
// small grid takes the shorter tiles so that it spreads over more blocks
// (less work per block and step; more records to reduce).  For grids far
// larger than the block count a streaming variant has each warp march down
// rows of 120-wide strips instead.
//
// Mixed precision: the FP32 recursive residual is replaced by the FP64 true
// residual b - A(x + d) whenever it has dropped by a factor ru_delta since
// the last replacement, and before convergence is declared; the search
// direction is kept across a replacement (reliable updates), so the FP32
// iteration converges like the FP64 one.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "tma.cuh"

namespace ppe {

namespace {

// Geometry of a tile: TX columns (128 for the tile-cooperative kernels, 120
// for the streaming kernel) and TY rows (16, or 8 or 4 for the short-tile
// kernels that spread a small grid over more blocks), with its window (halo 4
// in x so that the window starts on a 16-byte boundary, halo 2 in y) and
// one-cell ring.  The template key GK packs both: TX * 32 + TY.
constexpr int geo_key(int tx, int ty) { return tx * 32 + ty; }
constexpr int GEO_TILE = geo_key(TILE_X, TILE_Y), GEO_R8 = geo_key(TILE_X, TILE_Y_R8), GEO_R4 = geo_key(TILE_X, TILE_Y_R4),
              GEO_STREAM = geo_key(TILE_X_STREAM, TILE_Y);
template <int GK> struct Geo {
    static constexpr int TX = GK / 32, TY = GK % 32;
    static constexpr int OX = WIN_OX, OY = WIN_OY;
    static constexpr int WX = TX + 2 * WIN_OX, WY = TY + 2 * WIN_OY, WN = WX * WY;
    static constexpr int WN_PAD = (WN + 31) / 32 * 32;     // window buffers padded to 128 bytes (FP32)
    static constexpr int RX = TX + 2, RY = TY + 2, RN = RX * RY;
    static constexpr int TN = TX * TY;
    static constexpr int NRL = (RN + SOLVER_THREADS - 1) / SOLVER_THREADS;   // ring loads per thread
    // the passes that work row by row: SOLVER_THREADS / TY threads per row,
    // up to CPT columns each
    static constexpr int TPR = SOLVER_THREADS / TY, CPT = (TX + TPR - 1) / TPR;
};
constexpr int NWARP = SOLVER_THREADS / 32;

template <typename T> __device__ __forceinline__ T ld_cg(const T *p) { return __ldcg(p); }

template <typename T> __device__ __forceinline__ T recip(T v);
template <> __device__ __forceinline__ float recip<float>(float v) { return v > 0.f ? __frcp_rn(v) : 0.f; }
template <> __device__ __forceinline__ double recip<double>(double v) { return v > 0.0 ? 1.0 / v : 0.0; }

// Coefficients over the tile window, in the arithmetic type C.
template <typename C, int GK> struct alignas(16) Coef {
    // the tile-cooperative geometry also keeps the window's Jacobi weights
    // D^-1 (computed once per tile, read every pass); the streaming pass
    // forms them from the 1-D arrays
    static constexpr bool KEEP_DINV = Geo<GK>::TX == TILE_X;
    C dx[Geo<GK>::WX], fw[Geo<GK>::WX], fe[Geo<GK>::WX], sx[Geo<GK>::WX];
    C dy[Geo<GK>::WY], fs[Geo<GK>::WY], fn[Geo<GK>::WY], sy[Geo<GK>::WY];
    C dinv[KEEP_DINV ? Geo<GK>::WN : 1];
};

// TMA destinations of one tile: r and p windows, d tile (sizes are multiples
// of 128 bytes, so every part stays 128-byte aligned).
template <typename T, int GK> struct Stage {
    T r[Geo<GK>::WN_PAD];
    T p[Geo<GK>::WN_PAD];
    T d[Geo<GK>::TN];
};
static_assert((Geo<GEO_TILE>::WN_PAD * 4) % 128 == 0 && (Geo<GEO_TILE>::TN * 4) % 128 == 0 &&
                  (Geo<GEO_R8>::WN_PAD * 4) % 128 == 0 && (Geo<GEO_R8>::TN * 4) % 128 == 0 &&
                  (Geo<GEO_R4>::WN_PAD * 4) % 128 == 0 && (Geo<GEO_R4>::TN * 4) % 128 == 0,
              "TMA destinations must stay 128-byte aligned");

// The 1-D coefficient arrays of a tile's window as stored in global memory
// (cell widths, face coefficients; zero outside the grid), staged by cp.async.
template <typename T, int GK> struct CoefRaw {
    T dx[Geo<GK>::WX], fx[Geo<GK>::WX + 1], dy[Geo<GK>::WY], fy[Geo<GK>::WY + 1];
};

template <typename T, int GK> struct IterBufs {
    Stage<T, GK> st[2];
    T un[Geo<GK>::WN_PAD];    // new u on the one-cell ring
    T q[Geo<GK>::WN_PAD];     // A p on the one-cell ring
    CoefRaw<T, GK> raw[2];    // the next tile's coefficient arrays, in flight during this tile
};

// Scratch windows of the other passes.
template <typename T, int GK> struct Work {
    T a0[Geo<GK>::WN_PAD], a1[Geo<GK>::WN_PAD], a2[Geo<GK>::WN_PAD];
};

// Per-warp TMA chunks of the streaming pass: two buffers of SRB rows of r and
// p (128 wide from i0 - 4), of d (120 wide from i0) and of the rows' y
// coefficients, each part padded to 128 bytes.
constexpr int SRB = 4;
constexpr int S_WX = TILE_X_STREAM + 8;
constexpr int S_RBYTES = S_WX * SRB * 4, S_RPAD = (S_RBYTES + 127) / 128 * 128;
constexpr int S_DBYTES = TILE_X_STREAM * SRB * 4, S_DPAD = (S_DBYTES + 127) / 128 * 128;
constexpr int S_YBYTES = 4 * SRB * 4;                    // dy, fy[j], fy[j+1], 0 of each row
constexpr int S_CHUNK = 2 * S_RPAD + S_DPAD + 128;
struct StreamBufs {
    unsigned char buf[SOLVER_THREADS / 32][2][S_CHUNK];
};

template <typename T, int GK> union PassBufs {
    IterBufs<T, GK> it;
    Work<T, GK> w;
};
template <typename T> union PassBufs<T, GEO_STREAM> {
    Work<T, GEO_STREAM> w;
    StreamBufs sb;
};

template <typename T, int GK_> struct SmemT {
    static constexpr int GK = GK_;
    PassBufs<T, GK_> u;                  // first member: 128-byte aligned
    unsigned long long bar[2];           // TMA completion barriers of the two stages
    unsigned long long sbar[NWARP][2];   // streaming pass: per-warp chunk barriers
    uint32_t sfills[NWARP];              // streaming pass: chunks issued per warp (buffer = fill & 1)
    Coef<double, GK_> cfd;
    Coef<float, GK_> cff;
    float red_hi[2][NPART][NWARP], red_lo[2][NPART][NWARP];   // per-warp partials, two buffers
    SysDesc sd[SMAX];
    SysState st[SMAX];
    int32_t ph0[2][SMAX];   // step timing, by step parity: each system's phase at the step's start
    uint64_t tstep[2];      // and the step's start time
    int32_t tag_d, tag_f;   // tile whose coefficients are in cfd / cff
    int32_t go;
    uint32_t fills;         // TMA stage fills issued so far (stage = fill & 1)
    // nonzero: another pass has written its scratch windows over the TMA
    // stages since the tile pass last took the full proxy fence
    uint32_t udirty;
    // step profile (block 0): iteration pass before and after its data wait,
    // after two stages, at its entry and after its loads are issued
    uint64_t ptime[6];
    unsigned long long pacc[16];   // step profile (block 0): accumulated ns, written to SolverArgs::prof at the end
};

// Dynamic shared memory of a block (plus 128 bytes of alignment slack): one
// block per SM in every variant.
static_assert(sizeof(SmemT<float, GEO_TILE>) + 128 <= 227 * 1024, "FP32 solver: one block per SM");
static_assert(SMAX <= NWARP, "one warp per system of a block in the step's reduction");
static_assert(sizeof(SmemT<double, GEO_TILE>) + 128 <= 227 * 1024, "FP64 solver: one block per SM");
static_assert(sizeof(SmemT<float, GEO_STREAM>) + 128 <= 227 * 1024, "streaming solver: one block per SM");

template <typename C, int GK>
__device__ void load_coef(Coef<C, GK> &cf, const SysDesc &sd, int i0, int j0, const C *DX, const C *FX,
                          const C *DY, const C *FY)
{
    constexpr int WX = Geo<GK>::WX, WY = Geo<GK>::WY, OX = Geo<GK>::OX, OY = Geo<GK>::OY;
    for (int k = threadIdx.x; k < WX; k += blockDim.x) {
        int i = i0 - OX + k;
        bool in = i >= 0 && i < sd.nx;
        C w = in ? DX[i] : C(0), a = in ? FX[i] : C(0), b = in ? FX[i + 1] : C(0);
        cf.dx[k] = w; cf.fw[k] = a; cf.fe[k] = b; cf.sx[k] = a + b;
    }
    for (int k = threadIdx.x; k < WY; k += blockDim.x) {
        int j = j0 - OY + k;
        bool in = j >= 0 && j < sd.ny;
        C w = in ? DY[j] : C(0), a = in ? FY[j] : C(0), b = in ? FY[j + 1] : C(0);
        cf.dy[k] = w; cf.fs[k] = a; cf.fn[k] = b; cf.sy[k] = a + b;
    }
    if constexpr (Coef<C, GK>::KEEP_DINV) {
        __syncthreads();
        for (int k = threadIdx.x; k < Geo<GK>::WN; k += blockDim.x) {
            const int wi = k % WX, wj = k / WX;
            cf.dinv[k] = recip<C>(cf.dy[wj] * cf.sx[wi] + cf.dx[wi] * cf.sy[wj]);
        }
    }
}

template <typename T, typename S> __device__ __forceinline__ Coef<T, S::GK> &coef_of(S &sm)
{
    if constexpr (sizeof(T) == 4)
        return sm.cff;
    else
        return sm.cfd;
}

// Coefficients of a tile do not change between steps: a block that keeps
// working on the same tile reuses them.  Every caller synchronises the block
// before it reads the coefficients.
// Every thread reads the tag before thread 0 may change it.  With the
// Jacobi weights kept, load_coef passes a block barrier before thread 0
// writes the tag, which orders the reads; without them a barrier comes first.
template <typename S> __device__ __forceinline__ void load_coef_f(S &sm, const SysDesc &sd, int i0, int j0, int tag)
{
    const int have = sm.tag_f;
    if constexpr (!Coef<float, S::GK>::KEEP_DINV) __syncthreads();
    if (have == tag) return;
    load_coef<float>(sm.cff, sd, i0, j0, sd.dx32, sd.fx32, sd.dy32, sd.fy32);
    if (threadIdx.x == 0) sm.tag_f = tag;
}

template <typename S> __device__ __forceinline__ void load_coef_d(S &sm, const SysDesc &sd, int i0, int j0, int tag)
{
    const int have = sm.tag_d;
    if constexpr (!Coef<double, S::GK>::KEEP_DINV) __syncthreads();
    if (have == tag) return;
    load_coef<double>(sm.cfd, sd, i0, j0, sd.dx, sd.fx, sd.dy, sd.fy);
    if (threadIdx.x == 0) sm.tag_d = tag;
}

template <typename T, typename S> __device__ __forceinline__ void load_coef_t(S &sm, const SysDesc &sd, int i0, int j0, int tag)
{
    if constexpr (sizeof(T) == 4)
        load_coef_f(sm, sd, i0, j0, tag);
    else
        load_coef_d(sm, sd, i0, j0, tag);
}

// Asynchronous 4- or 8-byte copy global -> shared; an invalid element is
// zero-filled without reading global memory (src then points at element 0).
__device__ __forceinline__ void cp_async_el(float *dst, const float *src, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_el(double *dst, const double *src, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Start copying the coefficient arrays of the tile at (i0, j0) into raw.
template <typename T, int GK>
__device__ __forceinline__ void issue_coef_raw(CoefRaw<T, GK> &raw, const SysDesc &sd, int i0, int j0)
{
    constexpr int WX = Geo<GK>::WX, WY = Geo<GK>::WY, OX = Geo<GK>::OX, OY = Geo<GK>::OY;
    const T *DX, *FX, *DY, *FY;
    if constexpr (sizeof(T) == 4) {
        DX = sd.dx32; FX = sd.fx32; DY = sd.dy32; FY = sd.fy32;
    } else {
        DX = sd.dx; FX = sd.fx; DY = sd.dy; FY = sd.fy;
    }
    static_assert(WX + 1 <= 256 && 256 + WY + 1 <= SOLVER_THREADS, "one copy per thread");
    const int k = threadIdx.x;
    if (k <= WX) {
        const int i = i0 - OX + k;
        if (k < WX) {
            const bool v = (unsigned)i < (unsigned)sd.nx;
            cp_async_el(&raw.dx[k], DX + (v ? i : 0), v);
        }
        const bool vf = (unsigned)i <= (unsigned)sd.nx;       // faces 0 .. nx
        cp_async_el(&raw.fx[k], FX + (vf ? i : 0), vf);
    } else if (k >= 256 && k <= 256 + WY) {
        const int kk = k - 256, j = j0 - OY + kk;
        if (kk < WY) {
            const bool v = (unsigned)j < (unsigned)sd.ny;
            cp_async_el(&raw.dy[kk], DY + (v ? j : 0), v);
        }
        const bool vf = (unsigned)j <= (unsigned)sd.ny;
        cp_async_el(&raw.fy[kk], FY + (vf ? j : 0), vf);
    }
    cp_async_commit();
}

// The tile's coefficients (and D^-1 window) from staged arrays, as load_coef
// forms them from global memory; the caller has waited for the copies and
// synchronised the block.
template <typename C, int GK>
__device__ void coef_from_raw(Coef<C, GK> &cf, const CoefRaw<C, GK> &raw, const SysDesc &sd, int i0, int j0)
{
    constexpr int WX = Geo<GK>::WX, WY = Geo<GK>::WY, OX = Geo<GK>::OX, OY = Geo<GK>::OY;
    for (int k = threadIdx.x; k < WX; k += blockDim.x) {
        const bool in = (unsigned)(i0 - OX + k) < (unsigned)sd.nx;
        const C a = in ? raw.fx[k] : C(0), b = in ? raw.fx[k + 1] : C(0);
        cf.dx[k] = raw.dx[k]; cf.fw[k] = a; cf.fe[k] = b; cf.sx[k] = a + b;
    }
    for (int k = threadIdx.x; k < WY; k += blockDim.x) {
        const bool in = (unsigned)(j0 - OY + k) < (unsigned)sd.ny;
        const C a = in ? raw.fy[k] : C(0), b = in ? raw.fy[k + 1] : C(0);
        cf.dy[k] = raw.dy[k]; cf.fs[k] = a; cf.fn[k] = b; cf.sy[k] = a + b;
    }
    if constexpr (Coef<C, GK>::KEEP_DINV) {
        __syncthreads();
        for (int k = threadIdx.x; k < Geo<GK>::WN; k += blockDim.x) {
            const int wi = k % WX, wj = k / WX;
            cf.dinv[k] = recip<C>(cf.dy[wj] * cf.sx[wi] + cf.dx[wi] * cf.sy[wj]);
        }
    }
}

template <typename T, typename S> __device__ __forceinline__ void set_coef_tag(S &sm, int tag)
{
    if (threadIdx.x == 0) {
        if constexpr (sizeof(T) == 4)
            sm.tag_f = tag;
        else
            sm.tag_d = tag;
    }
}

template <typename C, int GK> __device__ __forceinline__ C dinv_at(const Coef<C, GK> &cf, int wi, int wj)
{
    if constexpr (Coef<C, GK>::KEEP_DINV)
        return cf.dinv[wj * Geo<GK>::WX + wi];
    else
        return recip<C>(cf.dy[wj] * cf.sx[wi] + cf.dx[wi] * cf.sy[wj]);
}

// (A U) at window point (wi, wj); U holds the window, zero outside the domain.
template <typename C, int GK> __device__ __forceinline__ C stencil(const Coef<C, GK> &cf, const C *U, int wi, int wj)
{
    constexpr int WX = Geo<GK>::WX;
    int k = wj * WX + wi;
    C c = U[k];
    C ax = cf.fe[wi] * (c - U[k + 1]) + cf.fw[wi] * (c - U[k - 1]);
    C ay = cf.fn[wj] * (c - U[k + WX]) + cf.fs[wj] * (c - U[k - WX]);
    return cf.dy[wj] * ax + cf.dx[wi] * ay;
}

// Scalars of the current pass in the pass's arithmetic type (FP32 copies are
// made once per step by the state transition, not by every thread).
template <typename T> __device__ __forceinline__ T sc_alpha(const SysState &s);
template <typename T> __device__ __forceinline__ T sc_beta(const SysState &s);
template <typename T> __device__ __forceinline__ T sc_mu(const SysState &s);
template <typename T> __device__ __forceinline__ T sc_alpha_d(const SysState &s);
template <> __device__ __forceinline__ float sc_alpha<float>(const SysState &s) { return s.alpha_f; }
template <> __device__ __forceinline__ float sc_beta<float>(const SysState &s) { return s.beta_f; }
template <> __device__ __forceinline__ float sc_mu<float>(const SysState &s) { return s.mu_f; }
template <> __device__ __forceinline__ float sc_alpha_d<float>(const SysState &s) { return s.alpha_d_f; }
template <> __device__ __forceinline__ double sc_alpha<double>(const SysState &s) { return s.alpha; }
template <> __device__ __forceinline__ double sc_beta<double>(const SysState &s) { return s.beta; }
template <> __device__ __forceinline__ double sc_mu<double>(const SysState &s) { return s.mu; }
template <> __device__ __forceinline__ double sc_alpha_d<double>(const SysState &s) { return s.alpha_d; }

__device__ __forceinline__ bool in_dom(const SysDesc &sd, int i, int j)
{
    return (unsigned)i < (unsigned)sd.nx && (unsigned)j < (unsigned)sd.ny;
}

// k-th point of the one-cell ring around the tile, as window coordinates
template <int GK> __device__ __forceinline__ void ring_point(int k, int &wi, int &wj)
{
    wi = Geo<GK>::OX - 1 + k % Geo<GK>::RX;
    wj = Geo<GK>::OY - 1 + k / Geo<GK>::RX;
}

// Tiles are numbered column by column (a strip of tiles stacked in y), so a
// contiguous range of tiles is mostly a vertical strip: the streaming
// iteration pass marches down it.
template <int GK> __device__ __forceinline__ void tile_origin(const SysDesc &sd, int t, int &i0, int &j0)
{
    int lt = t - sd.tile0;
    i0 = (lt / sd.tiles_y) * Geo<GK>::TX;
    j0 = (lt % sd.tiles_y) * Geo<GK>::TY;
}

// Float-float (hi + lo) accumulation: ~48-bit sums on the FP32 pipes.  On
// this chip FP64 arithmetic runs at a small fraction of the FP32 rate, so the
// cross-warp and cross-block accumulation of the dot products uses the
// error-free TwoSum transformation in FP32 instead of FP64 adds.
struct Acc {
    float hi[NPART], lo[NPART];
};

__device__ __forceinline__ void ff_add(float &hi, float &lo, float bhi, float blo)
{
    float s = hi + bhi;
    float bb = s - hi;
    float e = (hi - (s - bb)) + (bhi - bb);
    e += lo + blo;
    float h = s + e;
    lo = e - (h - s);
    hi = h;
}

__device__ __forceinline__ void ff_from_double(double v, float &hi, float &lo)
{
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

__device__ __forceinline__ void acc_zero(Acc &a)
{
#pragma unroll
    for (int q = 0; q < NPART; ++q) a.hi[q] = a.lo[q] = 0.f;
}

// Warp-reduce the thread's tile sums; lane 0 adds them to its accumulator.
__device__ __forceinline__ void warp_accumulate(const float (&t)[NPART], Acc &acc)
{
    float v[NPART];
#pragma unroll
    for (int q = 0; q < NPART; ++q) {
        v[q] = t[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    }
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int q = 0; q < NPART; ++q) ff_add(acc.hi[q], acc.lo[q], v[q], 0.f);
}

__device__ __forceinline__ void warp_accumulate(const double (&t)[NPART], Acc &acc)
{
    double v[NPART];
#pragma unroll
    for (int q = 0; q < NPART; ++q) {
        v[q] = t[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    }
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int q = 0; q < NPART; ++q) {
            float h, l;
            ff_from_double(v[q], h, l);
            ff_add(acc.hi[q], acc.lo[q], h, l);
        }
}

// Division through an FP32 reciprocal refined by two Newton steps in FP64
// (a few FP64 instructions instead of a full IEEE division sequence).
__device__ __forceinline__ double fast_div(double a, double b)
{
    double ab = fabs(b);
    if (!(ab > 1e-30 && ab < 1e30)) return a / b;
    double r = (double)__frcp_rn((float)b);
    r = r * (2.0 - b * r);
    r = r * (2.0 - b * r);
    return a * r;
}

// ---------------------------------------------------------------------------
// passes over one tile; thread sums go to acc (lane 0 of each warp)
// ---------------------------------------------------------------------------

// The solve's power-of-two scale sigma = 2^-e, e the binary exponent of max |b|
// (1 for a zero or non-finite b).  Multiplying by it is exact, so the scaled
// solve is the unscaled one bit for bit wherever that one stays in range.
__device__ __forceinline__ double sys_scale(const SysState &s)
{
    const uint64_t bits = s.bmax_bits;
    if (bits == 0 || bits >= 0x7FF0000000000000ull) return 1.0;
    int e = 0;
    frexp(__longlong_as_double((long long)bits), &e);
    return ldexp(1.0, -max(e, -1020));
}

// 1 / sys_scale(s), also exact
__device__ __forceinline__ double sys_unscale(const SysState &s)
{
    const uint64_t bits = s.bmax_bits;
    if (bits == 0 || bits >= 0x7FF0000000000000ull) return 1.0;
    int e = 0;
    frexp(__longlong_as_double((long long)bits), &e);
    return ldexp(1.0, max(e, -1020));
}

// b statistics: b = -V S (scaled)
template <typename T, typename S>
__device__ void pass_init(S &sm, const SysDesc &sd, const SysState &st, int i0, int j0, Acc &acc)
{
    const double sg = sys_scale(st);
    using G = Geo<S::GK>;
    constexpr int WX = G::WX, WN = G::WN, OX = G::OX, OY = G::OY, RN = G::RN, NRL = G::NRL, TILE_X = G::TX;
    constexpr int TILE_N = G::TN;
    (void)WX; (void)WN; (void)OX; (void)OY; (void)RN; (void)NRL; (void)TILE_X; (void)TILE_N;
    double t[NPART] = {0, 0, 0, 0, 0, 0};
    const int ty = threadIdx.x / G::TPR, tx = threadIdx.x % G::TPR;
    int j = j0 + ty;
#pragma unroll
    for (int c = 0; c < G::CPT; ++c) {
        int i = i0 + tx + G::TPR * c;
        if (tx + G::TPR * c < TILE_X && i < sd.nx && j < sd.ny) {
            double b = -sd.dx[i] * sd.dy[j] * sd.f[(size_t)j * sd.nx + i] * sg;
            t[0] += b; t[1] += b * b; t[2] += fabs(b);
        }
    }
    warp_accumulate(t, acc);
}

// FP64 true residual r = (b - mu_b) - A (x + d); stored into the inner buffer.
template <typename T, typename S>
__device__ void pass_res(S &sm, const SysDesc &sd, const SysState &st, int i0, int j0, int tag, Acc &acc)
{
    using G = Geo<S::GK>;
    constexpr int WX = G::WX, WN = G::WN, OX = G::OX, OY = G::OY, RN = G::RN, NRL = G::NRL, TILE_X = G::TX;
    constexpr int TILE_N = G::TN;
    (void)WX; (void)WN; (void)OX; (void)OY; (void)RN; (void)NRL; (void)TILE_X; (void)TILE_N;
    auto &cf = sm.cfd;
    double *X = reinterpret_cast<double *>(&sm.u.w);
    load_coef_d(sm, sd, i0, j0, tag);
    const T *d = (const T *)sd.d;
    const double sg = sys_scale(st);
    double xv[NRL];
#pragma unroll
    for (int q = 0; q < NRL; ++q) {
        int k = threadIdx.x + q * SOLVER_THREADS, wi, wj;
        ring_point<S::GK>(k, wi, wj);
        int i = i0 - OX + wi, j = j0 - OY + wj;
        xv[q] = 0.0;
        if (k < RN && in_dom(sd, i, j)) {
            xv[q] = ld_cg(sd.x + (size_t)j * sd.nx + i) * sg;
            if (st.has_d) xv[q] += (double)ld_cg(d + (size_t)j * sd.pitch + i);
        }
    }
#pragma unroll
    for (int q = 0; q < NRL; ++q) {
        int k = threadIdx.x + q * SOLVER_THREADS, wi, wj;
        ring_point<S::GK>(k, wi, wj);
        if (k < RN) X[wj * WX + wi] = xv[q];
    }
    __syncthreads();
    double t[NPART] = {0, 0, 0, 0, 0, 0};
    const int ty = threadIdx.x / G::TPR, tx = threadIdx.x % G::TPR;
    int j = j0 + ty, wj = ty + OY;
    T *r = (T *)sd.r[st.cur];
#pragma unroll
    for (int c = 0; c < G::CPT; ++c) {
        int i = i0 + tx + G::TPR * c, wi = tx + G::TPR * c + OX;
        if (tx + G::TPR * c < TILE_X && i < sd.nx && j < sd.ny) {
            double b = -sd.dx[i] * sd.dy[j] * ld_cg(sd.f + (size_t)j * sd.nx + i) * sg - st.mu_b;
            double rv = b - stencil<double>(cf, X, wi, wj);
            r[(size_t)j * sd.pitch + i] = (T)rv;
            t[0] += rv; t[1] += rv * rv;
        }
    }
    warp_accumulate(t, acc);
    __syncthreads();
}

// u = D^-1 (r - mu), w = A u; dots r.u, w.u, r.r, sum r.  When the direction
// is kept (continuation), also u.(A p) and p.(A p) of the current p.  Folds d
// into x when a replacement is pending.
template <typename T, typename S>
__device__ void pass_restart(S &sm, const SysDesc &sd, const SysState &st, int i0, int j0, int tag, Acc &acc)
{
    using G = Geo<S::GK>;
    constexpr int WX = G::WX, WN = G::WN, OX = G::OX, OY = G::OY, RN = G::RN, NRL = G::NRL, TILE_X = G::TX;
    constexpr int TILE_N = G::TN;
    (void)WX; (void)WN; (void)OX; (void)OY; (void)RN; (void)NRL; (void)TILE_X; (void)TILE_N;
    auto &cf = coef_of<T>(sm);
    T *R = sm.u.w.a0, *U = sm.u.w.a1, *P = sm.u.w.a2;
    load_coef_t<T>(sm, sd, i0, j0, tag);
    const T *rin = (const T *)sd.r[st.cur];
    const T *pin = (const T *)sd.p[st.pcur];
    const bool keep = st.keep_dir != 0;
    const T mu = sc_mu<T>(st);
    T rv[NRL], pv[NRL];
#pragma unroll
    for (int q = 0; q < NRL; ++q) {
        int k = threadIdx.x + q * SOLVER_THREADS, wi, wj;
        ring_point<S::GK>(k, wi, wj);
        int i = i0 - OX + wi, j = j0 - OY + wj;
        rv[q] = 0; pv[q] = 0;
        if (k < RN && in_dom(sd, i, j)) {
            size_t gi = (size_t)j * sd.pitch + i;
            rv[q] = ld_cg(rin + gi) - mu;
            if (keep) pv[q] = ld_cg(pin + gi);
        }
    }
    __syncthreads();   // coefficients visible
#pragma unroll
    for (int q = 0; q < NRL; ++q) {
        int k = threadIdx.x + q * SOLVER_THREADS, wi, wj;
        ring_point<S::GK>(k, wi, wj);
        if (k < RN) {
            int w = wj * WX + wi;
            R[w] = rv[q];
            U[w] = rv[q] * dinv_at<T>(cf, wi, wj);
            P[w] = pv[q];
        }
    }
    __syncthreads();
    T t[NPART] = {0, 0, 0, 0, 0, 0};
    const int ty = threadIdx.x / G::TPR, tx = threadIdx.x % G::TPR;
    int j = j0 + ty, wj = ty + OY;
    T *dd = (T *)sd.d;
#pragma unroll
    for (int c = 0; c < G::CPT; ++c) {
        int i = i0 + tx + G::TPR * c, wi = tx + G::TPR * c + OX;
        if (tx + G::TPR * c < TILE_X && i < sd.nx && j < sd.ny) {
            int k = wj * WX + wi;
            T w = stencil<T>(cf, U, wi, wj);
            t[0] += R[k] * U[k]; t[1] += w * U[k]; t[2] += R[k] * R[k]; t[3] += R[k];
            if (keep) {   // continuation: u.(A p) and p.(A p) of the kept direction
                T ap = stencil<T>(cf, P, wi, wj);
                t[4] += U[k] * ap; t[5] += P[k] * ap;
            }
            if (st.reset_d) {
                size_t gi = (size_t)j * sd.pitch + i;
                if (st.fold_d) sd.x[(size_t)j * sd.nx + i] += (double)ld_cg(dd + gi) * sys_unscale(st);
                dd[gi] = T(0);
            }
        }
    }
    warp_accumulate(t, acc);
    __syncthreads();
}

// Issue the TMA loads of tile t into stage `fill & 1` (one thread).
// Four consecutive values (16-byte aligned): one 16-byte access in FP32, two
// in FP64.
__device__ __forceinline__ void ld4(const float *p, float (&v)[4])
{
    const float4 a = *reinterpret_cast<const float4 *>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&v)[4])
{
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float *p, const float (&v)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double *p, const double (&v)[4])
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}

// (A U) at the four window points w .. w + 3 of row wj (columns wc .. wc + 3).
template <typename C, int GK>
__device__ __forceinline__ void stencil4(const Coef<C, GK> &cf, const C *U, int w, int wc, int wj, C (&out)[4])
{
    constexpr int WX = Geo<GK>::WX;
    C c[4], n[4], sv[4], fe[4], fw[4], dx[4];
    ld4(U + w, c);
    ld4(U + w + WX, n);
    ld4(U + w - WX, sv);
    ld4(cf.fe + wc, fe);
    ld4(cf.fw + wc, fw);
    ld4(cf.dx + wc, dx);
    const C left = U[w - 1], right = U[w + 4];
    const C fn = cf.fn[wj], fs = cf.fs[wj], dy = cf.dy[wj];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const C e = k < 3 ? c[k + 1] : right, west = k > 0 ? c[k - 1] : left;
        const C ax = fe[k] * (c[k] - e) + fw[k] * (c[k] - west);
        const C ay = fn * (c[k] - n[k]) + fs * (c[k] - sv[k]);
        out[k] = dy * ax + dx[k] * ay;
    }
}

template <typename T, typename S>
__device__ __forceinline__ void iter_issue_at(S &sm, const SysDesc &sd, int cur, int pcur, bool first, int t,
                                              uint32_t fill, bool fence)
{
    using G = Geo<S::GK>;
    constexpr int WX = G::WX, WN = G::WN, OX = G::OX, OY = G::OY, RN = G::RN, NRL = G::NRL, TILE_X = G::TX;
    constexpr int TILE_N = G::TN;
    (void)WX; (void)WN; (void)OX; (void)OY; (void)RN; (void)NRL; (void)TILE_X; (void)TILE_N;
    int i0, j0;
    tile_origin<S::GK>(sd, t, i0, j0);
    const int s = fill & 1;
    Stage<T, S::GK> &stg = sm.u.it.st[s];
    const uint32_t bar = smem_u32(&sm.bar[s]);
    const uint32_t bytes = (uint32_t)(((first ? 1 : 2) * WN + TILE_N) * sizeof(T));
    // The grid's writes of the vectors (ordered by the step barrier) before
    // the async-proxy copies: needed once per pass; later tiles of the pass
    // read the same buffers, which the pass itself does not write (it writes
    // the other r and p buffers and other tiles' parts of d).  The stage a
    // copy lands in was last written by threads (the pass updates its
    // windows in place) before at least one block barrier, so the fence is
    // taken for global memory only: the full fence, with shared memory,
    // costs 0.3 us per pass at one tile per block (7.34 against 7.01 us per
    // c3 iteration on GB300).  After another pass has written its scratch
    // windows over the stages, the first load takes the full fence.
    if (fence && sm.udirty) {
        fence_proxy_async();
        sm.udirty = 0;
    } else if (fence) {
        fence_proxy_async_global();
    }
    mbar_expect_tx(bar, bytes);
    tma_load_2d(smem_u32(stg.r), sd.tmaps + MAP_R0 + cur, bar, i0 - OX, j0 - OY);
    if (!first) tma_load_2d(smem_u32(stg.p), sd.tmaps + MAP_P0 + pcur, bar, i0 - OX, j0 - OY);
    tma_load_2d(smem_u32(stg.d), sd.tmaps + MAP_D, bar, i0, j0);
}

template <typename T, typename S>
__device__ __forceinline__ void iter_issue(S &sm, const SysDesc &sd, const SysState &st, int t, uint32_t fill,
                                           bool fence)
{
    iter_issue_at<T>(sm, sd, st.cur, st.pcur, st.first != 0, t, fill, fence);
}

// One single-reduction PCG iteration over the tiles [t_lo, t_hi) of system q,
// two-stage TMA pipeline (the next tile loads while this one is computed).
template <typename T, typename S>
__device__ void pass_iter(S &sm, int q, int t_lo, int t_hi, Acc &acc, const SolverArgs &a)
{
    using G = Geo<S::GK>;
    constexpr int WX = G::WX, WN = G::WN, OX = G::OX, OY = G::OY, RN = G::RN, NRL = G::NRL, TILE_X = G::TX;
    constexpr int TILE_N = G::TN;
    (void)WX; (void)WN; (void)OX; (void)OY; (void)RN; (void)NRL; (void)TILE_X; (void)TILE_N;
    const SysDesc &sd = sm.sd[q];
    const SysState &st = sm.st[q];
    auto &cf = coef_of<T>(sm);
    IterBufs<T, S::GK> &ib = sm.u.it;
    T *Un = ib.un, *Q = ib.q;
    const int n = t_hi - t_lo;
    if (n <= 0) return;
    const uint32_t fill0 = sm.fills;
    const bool prof0 = a.prof && blockIdx.x == 0 && threadIdx.x == 0 && q == 0;
    if (prof0) sm.ptime[4] = gtimer();
    if (threadIdx.x == 0) iter_issue<T>(sm, sd, st, t_lo, fill0, true);
    if (prof0) sm.ptime[5] = gtimer();
    T *rout = (T *)sd.r[st.cur ^ 1];
    T *pout = (T *)sd.p[st.pcur ^ 1];
    T *dv = (T *)sd.d;
    const T mu = sc_mu<T>(st), alpha = sc_alpha<T>(st), beta = sc_beta<T>(st);
    const bool first = st.first != 0;
    for (int k = 0; k < n; ++k) {
        const int t = t_lo + k;
        const uint32_t fill = fill0 + k;
        if (threadIdx.x == 0 && k + 1 < n) iter_issue<T>(sm, sd, st, t + 1, fill + 1, false);
        int i0, j0;
        tile_origin<S::GK>(sd, t, i0, j0);
        if (k == 0) {
            load_coef_t<T>(sm, sd, i0, j0, t);
        } else {
            // this tile's arrays were copied while the previous tile was computed
            cp_async_wait_all();
            __syncthreads();
            coef_from_raw<T>(cf, ib.raw[k & 1], sd, i0, j0);
            set_coef_tag<T>(sm, t);
        }
        if (k + 1 < n) {
            int i1, j1;
            tile_origin<S::GK>(sd, t + 1, i1, j1);
            issue_coef_raw<T>(ib.raw[(k + 1) & 1], sd, i1, j1);
        }
        Stage<T, S::GK> &stg = ib.st[fill & 1];
        const bool prof = a.prof && blockIdx.x == 0 && threadIdx.x == 0 && q == 0;
        if (prof) sm.ptime[0] = gtimer();
        if (!mbar_wait_bounded(smem_u32(&sm.bar[fill & 1]), (fill >> 1) & 1, a.spin_limit_ns)) {
            if (threadIdx.x == 0) atomicExch(&a.ctl->err, (int32_t)PPE_ERR_TIMEOUT);
            sm.go = 0;
        }
        __syncthreads();   // coefficients visible
        if (prof) sm.ptime[1] = gtimer();
        // Every stage works on groups of four consecutive cells (16-byte
        // shared and global accesses); window rows (136), the tile's columns
        // (from window column 4) and the grid pitch are multiples of four.
        static_assert(Coef<T, S::GK>::KEEP_DINV && WX % 4 == 0 && OX % 4 == 0 && TILE_X % 4 == 0,
                      "four-cell groups stay aligned");
        constexpr int GX = WX / 4, TG = TILE_X / 4;
        // window: r - mu and the new direction p = u + beta p (zero outside the domain)
        T *Rw = stg.r, *Pw = stg.p;
        for (int g = threadIdx.x; g < G::WY * GX; g += SOLVER_THREADS) {
            const int wj = g / GX, wc = (g - wj * GX) * 4, w = wj * WX + wc;
            const int i = i0 - OX + wc;
            const bool row_in = (unsigned)(j0 - OY + wj) < (unsigned)sd.ny;
            T r[4], p[4], dinv[4];
            ld4(Rw + w, r);
            ld4(Pw + w, p);
            ld4(cf.dinv + w, dinv);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const bool in = row_in && (unsigned)(i + k) < (unsigned)sd.nx;
                const T rv = in ? r[k] - mu : T(0);
                const T u = rv * dinv[k];
                r[k] = rv;
                p[k] = first ? u : u + beta * p[k];
            }
            st4(Rw + w, r);
            st4(Pw + w, p);
        }
        __syncthreads();
        if (prof) sm.ptime[2] = gtimer();
        // one-cell ring: q = A p, r' = r - alpha q, u' = D^-1 r'; the tile's
        // columns in groups of four, the two edge columns one cell at a time
        constexpr int NRV = (TILE_N / TILE_X + 2) * TG;
        for (int g = threadIdx.x; g < NRV + 2 * (TILE_N / TILE_X + 2); g += SOLVER_THREADS) {
            if (g < NRV) {
                const int wj = OY - 1 + g / TG, wc = OX + (g % TG) * 4, w = wj * WX + wc;
                T qv[4], r[4], dinv[4], un[4];
                stencil4<T>(cf, Pw, w, wc, wj, qv);
                ld4(Rw + w, r);
                ld4(cf.dinv + w, dinv);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    r[k] -= alpha * qv[k];
                    un[k] = r[k] * dinv[k];
                }
                st4(Rw + w, r);
                st4(Un + w, un);
                st4(Q + w, qv);
            } else {
                const int e = g - NRV;
                const int wj = OY - 1 + (e >> 1), wi = (e & 1) ? OX + TILE_X : OX - 1;
                const int kk = wj * WX + wi;
                const T qv = stencil<T>(cf, Pw, wi, wj);
                const T rn = Rw[kk] - alpha * qv;
                Rw[kk] = rn;
                Un[kk] = rn * cf.dinv[kk];
                Q[kk] = qv;
            }
        }
        __syncthreads();
        if (prof) sm.ptime[3] = gtimer();
        // tile: store p, d, r'; dots r'.u', (A u').u', r'.r', sum r', u'.(A p), p.(A p)
        T tt[NPART] = {0, 0, 0, 0, 0, 0};
        for (int g = threadIdx.x; g < TILE_N / 4; g += SOLVER_THREADS) {
            const int ty = g / TG, cx = (g - ty * TG) * 4;
            const int j = j0 + ty, i = i0 + cx;
            if (j >= sd.ny || i >= sd.nx) continue;
            const int wj = OY + ty, wc = OX + cx, w = wj * WX + wc;
            T pn[4], rn[4], un[4], qv[4], dd[4], wn[4];
            ld4(Pw + w, pn);
            ld4(Rw + w, rn);
            ld4(Un + w, un);
            ld4(Q + w, qv);
            ld4(stg.d + ty * TILE_X + cx, dd);
            stencil4<T>(cf, Un, w, wc, wj, wn);
#pragma unroll
            for (int k = 0; k < 4; ++k) dd[k] += alpha * pn[k];
            const size_t gi = (size_t)j * sd.pitch + i;
            if (i + 3 < sd.nx) {
                st4(pout + gi, pn);
                st4(dv + gi, dd);
                st4(rout + gi, rn);
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (i + k < sd.nx) {
                        pout[gi + k] = pn[k];
                        dv[gi + k] = dd[k];
                        rout[gi + k] = rn[k];
                    }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (i + k >= sd.nx) continue;
                tt[0] += rn[k] * un[k]; tt[1] += wn[k] * un[k]; tt[2] += rn[k] * rn[k]; tt[3] += rn[k];
                tt[4] += un[k] * qv[k]; tt[5] += pn[k] * qv[k];
            }
        }
        warp_accumulate(tt, acc);
        // stage and ring buffers free for the next tile; after the last tile
        // the step's publish barrier (or the next pass's barriers, which all
        // come before any thread writes these buffers again) does it
        if (k + 1 < n) __syncthreads();
    }
    if (threadIdx.x == 0) sm.fills = fill0 + n;
}

// ---------------------------------------------------------------------------
// Streaming iteration pass (FP32, for grids far larger than the block
// count): the arithmetic of pass_iter organised for HBM bandwidth.  Each warp
// takes a contiguous run of the block's tiles (a vertical strip, the tiles
// being numbered column by column) and marches down it one row at a time.
// The warp covers the 128 columns i0 - 4 .. i0 + 123: the 120 tile columns
// and a four-cell halo on each side (two are needed; four keep every lane's
// columns on a 16-byte boundary).  Lane l holds columns i0 - 4 + 4l ..
// i0 - 1 + 4l: one 16-byte shared-memory load per vector and row, one
// 16-byte store per vector and row.  The TMA unit streams the strip into
// shared memory in chunks of four rows (r and p 128 wide from i0 - 4, d 120
// wide from i0, and the rows' y coefficients; zero outside the grid), two
// chunks in flight per warp.  For a new window row s:
//   row s:      P = D^-1 (r - mu) + beta p_old               (halo 2)
//   row s - 1:  Q = A P, r' = (r - mu) - alpha Q, u' = D^-1 r'   (halo 1);
//               on a tile row store p, r', d + alpha p and add r'.u', r'.r',
//               sum r', u'.Q, p.Q
//   row s - 2:  add (A u').u'
// Three rows of P and u' and one row of r - mu and D^-1 stay in registers;
// east and west neighbours come from the adjacent lane by shuffle.  Lanes 0
// and 31 hold only halo columns: their values feed their neighbours'
// stencils and are never stored or summed.  No block barrier is involved.
// ---------------------------------------------------------------------------

struct XCoef {
    float dx[4], fw[4], fe[4];
};

// A at one row on the lane's four columns, from the rows below (S), at (C)
// and above (N).
__device__ __forceinline__ void stencil_row(const XCoef &xc, float dyj, float fsj, float fnj, const float (&S)[4],
                                            const float (&C)[4], const float (&N)[4], float (&out)[4])
{
    const float w0 = __shfl_up_sync(0xffffffffu, C[3], 1);
    const float e3 = __shfl_down_sync(0xffffffffu, C[0], 1);
    const float W[4] = {w0, C[0], C[1], C[2]};
    const float E[4] = {C[1], C[2], C[3], e3};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float cc = C[c];
        const float ax = xc.fe[c] * (cc - E[c]) + xc.fw[c] * (cc - W[c]);
        const float ay = fnj * (cc - N[c]) + fsj * (cc - S[c]);
        out[c] = dyj * ax + xc.dx[c] * ay;
    }
}

// Issue the TMA loads of chunk k of a run (window rows jb - 2 + 4k .. +3 of r,
// p and the y coefficients, rows jb - 3 + 4k .. +3 of d, i.e. the ring rows
// of those window rows) into the warp's buffer g & 1.
template <typename S>
__device__ __forceinline__ void stream_issue(S &sm, const SysDesc &sd, const SysState &st, int warp, uint32_t g,
                                             int i0, int jb, int k)
{
    unsigned char *buf = sm.u.sb.buf[warp][g & 1];
    const uint32_t bar = smem_u32(&sm.sbar[warp][g & 1]);
    const bool first = st.first != 0;
    const uint32_t bytes = (first ? 1 : 2) * S_RBYTES + S_DBYTES + S_YBYTES;
    // The full proxy fence before every chunk.  Once per pass and warp would
    // do for ordering (threads only read the chunk buffers), but that was
    // measured to stream slower on GB300 (8192^2: 4,156 against 4,662 GB/s).
    fence_proxy_async();
    mbar_expect_tx(bar, bytes);
    tma_load_2d(smem_u32(buf), sd.tmaps + MAP_R0 + st.cur, bar, i0 - WIN_OX, jb - 2 + SRB * k);
    if (!first) tma_load_2d(smem_u32(buf + S_RPAD), sd.tmaps + MAP_P0 + st.pcur, bar, i0 - WIN_OX, jb - 2 + SRB * k);
    tma_load_2d(smem_u32(buf + 2 * S_RPAD), sd.tmaps + MAP_D, bar, i0, jb - 3 + SRB * k);
    tma_load_2d(smem_u32(buf + 2 * S_RPAD + S_DPAD), sd.tmaps + MAP_Y, bar, 0, jb - 2 + SRB * k);
}

// Not inlined: it gets its own register allocation (the kernel saves its
// live registers once per call instead of spilling inside the row loop).
template <typename S>
__device__ __noinline__ void pass_iter_stream(S &sm, int q, int t_lo, int t_hi, Acc &acc, const SolverArgs &a)
{
    const SysDesc &sd = sm.sd[q];
    const SysState &st = sm.st[q];
    StreamBufs &sb = sm.u.sb;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = t_hi - t_lo;
    // The block's tiles are consecutive rows of one strip or a few (a tile is
    // TILE_Y rows of a strip, tiles are numbered down the strips): split those
    // rows evenly over the warps, so that a block with fewer tiles than warps
    // still keeps every warp busy.
    const int rows_per_col = sd.tiles_y * TILE_Y;
    const int u_lo = (t_lo - sd.tile0) * TILE_Y, nu = n * TILE_Y;
    const int u0 = u_lo + (int)((long long)nu * warp / NWARP), u1 = u_lo + (int)((long long)nu * (warp + 1) / NWARP);
    float *rout = (float *)sd.r[st.cur ^ 1];
    float *pout = (float *)sd.p[st.pcur ^ 1];
    float *dv = (float *)sd.d;
    const float mu = st.mu_f, alpha = st.alpha_f, beta = st.beta_f;
    const bool first = st.first != 0;
    const int nx = sd.nx;
    const size_t pitch = (size_t)sd.pitch;
    float tt[NPART] = {0, 0, 0, 0, 0, 0};
    uint32_t gnext = sm.sfills[warp];      // global index of this warp's next chunk
    bool ok = true;

    for (int u = u0; u < u1;) {
        // the run of rows u .. u_end - 1 in one strip
        const int col = u / rows_per_col, r = u - col * rows_per_col;
        const int u_end = min(u1, u - r + rows_per_col);
        const int i0 = col * TILE_X_STREAM;
        const int jb = r, je = min(sd.ny, r + (u_end - u));
        u = u_end;
        if (jb >= je) continue;                    // rows of the strip's last tile below the grid
        const int nchunks = (je - jb + 4 + SRB - 1) / SRB;
        const uint32_t gb = gnext;
        gnext += nchunks;
        if (lane == 0) {
            stream_issue(sm, sd, st, warp, gb, i0, jb, 0);
            if (nchunks > 1) stream_issue(sm, sd, st, warp, gb + 1, i0, jb, 1);
        }

        const int x0 = i0 - 4 + 4 * lane;          // first column of the lane (16-byte aligned)
        XCoef xc;                                  // dx > 0 exactly on grid columns
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int x = x0 + c;
            const bool v = x >= 0 && x < nx;
            xc.dx[c] = v ? sd.dx32[x] : 0.f;
            xc.fw[c] = v ? sd.fx32[x] : 0.f;
            xc.fe[c] = v ? sd.fx32[x + 1] : 0.f;
        }
        // lanes 1..30 hold the tile columns; the float4 lies inside the row's pitch
        const bool own = lane >= 1 && lane <= 30 && x0 < nx;

        float P0[4], P1[4], P2[4];   // P of rows s-2, s-1, s
        float R1[4], D1[4];          // r - mu and D^-1 of row s-1
        float U0[4], U1[4], U2[4];   // u' of rows s-3, s-2, s-1
        float ydy1 = 0.f, yfs1 = 0.f, yfn1 = 0.f;   // y coefficients of row s-1
        float ydy0 = 0.f, yfs0 = 0.f, yfn0 = 0.f;   // and of row s-2
#pragma unroll
        for (int c = 0; c < 4; ++c) P0[c] = P1[c] = P2[c] = R1[c] = D1[c] = U0[c] = U1[c] = U2[c] = 0.f;

        // One chunk (SRB window rows) per outer iteration; the rows of a chunk
        // are unrolled, so the row windows rotate by renaming.  Rows before the
        // run (s < jb) and after it (s > je + 1) are computed on zeros or on
        // neighbouring data and never stored or summed.
        for (int k = 0; k < nchunks; ++k) {
            const uint32_t g = gb + k;
            if (!mbar_wait_bounded(smem_u32(&sm.sbar[warp][g & 1]), (g >> 1) & 1, a.spin_limit_ns)) {
                if (ok && lane == 0) atomicExch(&a.ctl->err, (int32_t)PPE_ERR_TIMEOUT);
                ok = false;
                sm.go = 0;
            }
            // chunk k - 1 is consumed: its buffer takes chunk k + 1
            __syncwarp();
            if (lane == 0 && k >= 1 && k + 1 < nchunks) stream_issue(sm, sd, st, warp, g + 1, i0, jb, k + 1);
            const unsigned char *cb = sb.buf[warp][g & 1];
            const float4 *rbuf = reinterpret_cast<const float4 *>(cb) + lane;
            const float4 *pbuf = reinterpret_cast<const float4 *>(cb + S_RPAD) + lane;
            // d rows hold the 120 tile columns; lane l >= 1 reads its four at 4l - 4
            const float4 *dbuf = reinterpret_cast<const float4 *>(cb + 2 * S_RPAD) + (lane >= 1 ? lane - 1 : 0);
            const float4 *ybuf = reinterpret_cast<const float4 *>(cb + 2 * S_RPAD + S_DPAD);
#pragma unroll
            for (int rr = 0; rr < SRB; ++rr) {
                const int s = jb - 2 + SRB * k + rr;
                const float4 a4 = rbuf[rr * (S_WX / 4)];
                float4 b4 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (!first) b4 = pbuf[rr * (S_WX / 4)];
                const float lr[4] = {a4.x, a4.y, a4.z, a4.w}, lp[4] = {b4.x, b4.y, b4.z, b4.w};
                const float4 yc = ybuf[rr];          // zero outside the grid
                const float dy = yc.x, fs = yc.y, fn = yc.z, sy = fs + fn;
                const float vy = dy > 0.f ? 1.f : 0.f;   // row inside the grid
                // row s: r - mu, D^-1, P (zero outside the grid)
                float R2[4], D2[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    P0[c] = P1[c];
                    P1[c] = P2[c];
                    const float in = xc.dx[c] > 0.f ? vy : 0.f;
                    const float r = in * (lr[c] - mu);
                    const float dg = dy * (xc.fw[c] + xc.fe[c]) + xc.dx[c] * sy;
                    D2[c] = dg > 0.f ? __frcp_rn(dg) : 0.f;
                    R2[c] = r;
                    P2[c] = first ? r * D2[c] : r * D2[c] + beta * (in * lp[c]);
                }
                // ring row s - 1: Q = A P, r', u'
                float qv[4], rn1[4];
                stencil_row(xc, ydy1, yfs1, yfn1, P0, P1, P2, qv);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    U0[c] = U1[c];
                    U1[c] = U2[c];
                    rn1[c] = R1[c] - alpha * qv[c];
                    U2[c] = rn1[c] * D1[c];
                }
                // row s - 2: (A u').u'
                float wv[4];
                stencil_row(xc, ydy0, yfs0, yfn0, U0, U1, U2, wv);
                const int jr = s - 1, jo = s - 2;
                const bool ring_out = jr >= jb && jr < je, w_out = jo >= jb && jo < je;
                const float m1 = ring_out && own ? 1.f : 0.f, m0 = w_out && own ? 1.f : 0.f;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float oc = xc.dx[c] > 0.f ? 1.f : 0.f;       // tile column inside the grid
                    const float rm = (m1 * oc) * rn1[c], qm = (m1 * oc) * qv[c];
                    tt[0] += rm * U2[c]; tt[2] += rm * rn1[c]; tt[3] += rm;
                    tt[4] += U2[c] * qm; tt[5] += P1[c] * qm;
                    tt[1] += (m0 * oc) * wv[c] * U1[c];
                }
                if (ring_out && own) {
                    // store p, r', d + alpha p of ring row s - 1 (a tile row)
                    const float4 d4 = dbuf[rr * (TILE_X_STREAM / 4)];
                    const size_t o = (size_t)jr * pitch + x0;
                    *reinterpret_cast<float4 *>(pout + o) = make_float4(P1[0], P1[1], P1[2], P1[3]);
                    *reinterpret_cast<float4 *>(rout + o) = make_float4(rn1[0], rn1[1], rn1[2], rn1[3]);
                    *reinterpret_cast<float4 *>(dv + o) = make_float4(d4.x + alpha * P1[0], d4.y + alpha * P1[1],
                                                                      d4.z + alpha * P1[2], d4.w + alpha * P1[3]);
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    R1[c] = R2[c];
                    D1[c] = D2[c];
                }
                ydy0 = ydy1; yfs0 = yfs1; yfn0 = yfn1;
                ydy1 = dy; yfs1 = fs; yfn1 = fn;
            }
        }
        __syncwarp();   // this run's buffers are read before the next run's loads reuse them
    }
    if (lane == 0) sm.sfills[warp] = gnext;
    warp_accumulate(tt, acc);
}

// DLSM dots r.e, e.(A e), e.e  (Eq. 11); with upd: d += alpha e, r_new = r - alpha A e (Eq. 12)
template <typename T, typename S, bool UPD>
__device__ void pass_dlsm(S &sm, const SysDesc &sd, const SysState &st, int i0, int j0, int tag, Acc &acc)
{
    using G = Geo<S::GK>;
    constexpr int WX = G::WX, WN = G::WN, OX = G::OX, OY = G::OY, RN = G::RN, NRL = G::NRL, TILE_X = G::TX;
    constexpr int TILE_N = G::TN;
    (void)WX; (void)WN; (void)OX; (void)OY; (void)RN; (void)NRL; (void)TILE_X; (void)TILE_N;
    // A e in the pass's precision: in FP64 mode the FP32 direction is applied
    // with the FP64 operator, as the FP64 iteration applies A to p
    auto &cf = coef_of<T>(sm);
    T *E = sm.u.w.a0;
    load_coef_t<T>(sm, sd, i0, j0, tag);
    float ev[NRL];
#pragma unroll
    for (int q = 0; q < NRL; ++q) {
        int k = threadIdx.x + q * SOLVER_THREADS, wi, wj;
        ring_point<S::GK>(k, wi, wj);
        int i = i0 - OX + wi, j = j0 - OY + wj;
        ev[q] = 0.f;
        if (k < RN && in_dom(sd, i, j)) ev[q] = ld_cg(sd.e + (size_t)j * sd.pitch + i);
    }
#pragma unroll
    for (int q = 0; q < NRL; ++q) {
        int k = threadIdx.x + q * SOLVER_THREADS, wi, wj;
        ring_point<S::GK>(k, wi, wj);
        if (k < RN) E[wj * WX + wi] = ev[q];
    }
    __syncthreads();
    const int cur = st.cur;
    const T *rin = (const T *)sd.r[cur];
    T *rout = (T *)sd.r[cur ^ 1];
    T *dv = (T *)sd.d;
    const T mu = sc_mu<T>(st), alpha = sc_alpha_d<T>(st);
    T t[NPART] = {0, 0, 0, 0, 0, 0};
    const int ty = threadIdx.x / G::TPR, tx = threadIdx.x % G::TPR;
    int j = j0 + ty, wj = ty + OY;
#pragma unroll
    for (int c = 0; c < G::CPT; ++c) {
        int i = i0 + tx + G::TPR * c, wi = tx + G::TPR * c + OX;
        if (tx + G::TPR * c < TILE_X && i < sd.nx && j < sd.ny) {
            int k = wj * WX + wi;
            size_t gi = (size_t)j * sd.pitch + i;
            T e = E[k];
            T q = stencil(cf, E, wi, wj);
            T r = ld_cg(rin + gi) - mu;
            if (UPD) {
                T rn = r - alpha * q;
                rout[gi] = rn;
                dv[gi] = ld_cg(dv + gi) + alpha * e;
                t[2] += rn * rn; t[3] += rn;
            } else {
                t[0] += r * e; t[1] += e * q; t[2] += e * e;
            }
        }
    }
    warp_accumulate(t, acc);
    __syncthreads();
}

// Fold d into x (if pending) and accumulate sum V, sum V x.
template <typename T, typename S>
__device__ void pass_final1(S &sm, const SysDesc &sd, const SysState &st, int i0, int j0, Acc &acc)
{
    using G = Geo<S::GK>;
    constexpr int WX = G::WX, WN = G::WN, OX = G::OX, OY = G::OY, RN = G::RN, NRL = G::NRL, TILE_X = G::TX;
    constexpr int TILE_N = G::TN;
    (void)WX; (void)WN; (void)OX; (void)OY; (void)RN; (void)NRL; (void)TILE_X; (void)TILE_N;
    const T *dd = (const T *)sd.d;
    const double sg = sys_scale(st);
    double t[NPART] = {0, 0, 0, 0, 0, 0};
    const int ty = threadIdx.x / G::TPR, tx = threadIdx.x % G::TPR;
    int j = j0 + ty;
#pragma unroll
    for (int c = 0; c < G::CPT; ++c) {
        int i = i0 + tx + G::TPR * c;
        if (tx + G::TPR * c < TILE_X && i < sd.nx && j < sd.ny) {
            size_t gx = (size_t)j * sd.nx + i;
            double x = st.zero_x ? 0.0 : ld_cg(sd.x + gx);
            if (st.fold_d && !st.zero_x) x += (double)ld_cg(dd + (size_t)j * sd.pitch + i) * sys_unscale(st);
            sd.x[gx] = x;
            double v = sd.dx[i] * sd.dy[j];
            t[0] += v; t[1] += v * (x * sg);
        }
    }
    warp_accumulate(t, acc);
}

template <typename T, typename S>
__device__ void pass_final2(S &sm, const SysDesc &sd, const SysState &st, int i0, int j0, Acc &acc)
{
    using G = Geo<S::GK>;
    constexpr int WX = G::WX, WN = G::WN, OX = G::OX, OY = G::OY, RN = G::RN, NRL = G::NRL, TILE_X = G::TX;
    constexpr int TILE_N = G::TN;
    (void)WX; (void)WN; (void)OX; (void)OY; (void)RN; (void)NRL; (void)TILE_X; (void)TILE_N;
    const int ty = threadIdx.x / G::TPR, tx = threadIdx.x % G::TPR;
    int j = j0 + ty;
#pragma unroll
    for (int c = 0; c < G::CPT; ++c) {
        int i = i0 + tx + G::TPR * c;
        if (tx + G::TPR * c < TILE_X && i < sd.nx && j < sd.ny) {
            size_t gx = (size_t)j * sd.nx + i;
            sd.x[gx] = ld_cg(sd.x + gx) - st.xmean * sys_unscale(st);
        }
    }
}

// ---------------------------------------------------------------------------
// state machine
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool is_pass_phase(int ph) { return ph != PH_NET && ph != PH_DONE; }

// max(v, 0) for a sum of squares that rounding may push below zero; a NaN
// stays NaN, so that a non-finite vector surfaces as PPE_ERR_NAN instead of
// reading as a zero norm
__device__ __forceinline__ double nonneg(double v) { return v > 0.0 ? v : (v == v ? 0.0 : v); }
__device__ __forceinline__ float nonneg(float v) { return v > 0.f ? v : (v == v ? 0.f : v); }

__device__ __forceinline__ int iter_cap(const SysDesc &sd)
{
    return sd.max_iters + (sd.mode == PPE_MODE_HYBRID ? sd.hybrid_budget : 0);
}

__device__ void to_res(SysState &s, int keep_dir)
{
    s.has_d = 1;
    s.keep_dir = keep_dir;
    s.phase = PH_RES;
}

// Transition of one system after a pass; t holds the reduced partial sums.
__device__ void advance(const SysDesc &sd, SysState &s, const double (&t)[NPART])
{
    const double N = sd.n_cells;
    (void)N;
    switch (s.phase) {
    case PH_INIT: {
        s.mu_b = t[0] * sd.inv_n;
        double bb = t[1] - N * s.mu_b * s.mu_b;
        s.bnorm = sqrt(nonneg(bb));
        s.incompat = t[2] > 0.0 ? fabs(t[0]) / t[2] : 0.0;
        s.cur = 0;
        s.pcur = 0;
        if (!isfinite(t[0]) || !isfinite(t[1]) || !isfinite(t[2])) {
            s.status = PPE_ERR_NAN;
            s.relres = t[1];
            s.phase = PH_FINAL1;
        } else if (!(s.incompat <= 1e-6)) {
            s.status = PPE_ERR_INCOMPATIBLE_RHS;
            s.phase = PH_DONE;
        } else if (!(s.bnorm > 0.0)) {
            s.zero_x = 1;
            s.relres = 0.0;
            s.phase = PH_FINAL1;
        } else {
            s.has_d = 0;
            s.keep_dir = 0;
            s.target = 0.9 * sd.tol * s.bnorm;
            s.phase = PH_RES;
        }
        break;
    }
    case PH_RES: {
        s.refinements++;
        s.mu = t[0] * sd.inv_n;
        double rr = t[1] - N * s.mu * s.mu;
        s.rnorm = sqrt(nonneg(rr));
        s.relres = fast_div(s.rnorm, s.bnorm);
        s.fold_d = s.has_d;
        // mixed precision: an FP32 inner solve normally cuts the true residual
        // by about inner_rtol; when the system's conditioning exceeds what
        // FP32 resolves, the inner iteration stalls and the true residual
        // stops falling.  Three refinements in a row that fail to cut it by
        // max(1/2, sqrt(inner_rtol)) end the mixed solve (the host continues
        // it in FP64); the square root keeps a planned reduction weaker than
        // one half from counting as a stall.
        if (sd.precision == PPE_PREC_MIXED && s.refinements > 1)
            s.stall = (s.relres > fmax(0.5, sqrt(sd.ru_delta)) * s.relres_prev || sd.force_stall) ? s.stall + 1 : 0;
        s.relres_prev = s.relres;
        // the budget of an inner solve follows the last one that reached its
        // reduction target (an overrun does not raise it)
        if (s.it_rep > 0 && !s.overran) s.it_rep_prev = s.it_rep;
        s.it_rep = 0;
        s.overran = 0;
        if (!isfinite(s.relres)) {
            s.status = PPE_ERR_NAN;
            s.fold_d = 0;
            s.phase = PH_FINAL1;
        } else if (s.relres <= sd.tol) {
            s.phase = PH_FINAL1;
        } else if (s.it_total >= iter_cap(sd) || s.refinements > 5000) {
            s.status = PPE_ERR_NOT_CONVERGED;
            s.phase = PH_FINAL1;
        } else if (s.stall >= 3) {
            s.status = PPE_ERR_NOT_CONVERGED;
            s.prec_stalled = 1;
            s.phase = PH_FINAL1;
        } else {
            s.rho_ref = s.rnorm;
            s.reset_d = 1;
            s.phase = PH_RESTART;
        }
        break;
    }
    case PH_RESTART: {
        // this pass summed r - mu; its mean is the further correction
        double dmu = t[3] * sd.inv_n;
        s.mu += dmu;
        double rr = t[2] - N * dmu * dmu;
        s.rho = nonneg(rr);
        s.reset_d = 0;
        s.fold_d = 0;
        s.has_d = 1;
        s.cg_count = 0;
        s.e_cg = 0.f;
        s.e_cg_n = 0;
        if (s.rho <= s.target * s.target || !(t[1] > 0.0) || !(t[0] > 0.0)) {
            to_res(s, 0);
            break;
        }
        bool cont = s.keep_dir && s.gamma > 0.0;
        if (cont) {
            // p' = u + beta p: p'.A p' = u.Au + 2 beta u.(Ap) + beta^2 p.(Ap)
            double beta = fast_div(t[0], s.gamma);
            double pap = t[1] + beta * (2.0 * t[4] + beta * t[5]);
            cont = pap > 0.0 && isfinite(beta);
            if (cont) {
                s.beta = beta;
                s.alpha = fast_div(t[0], pap);
                s.first = 0;
            }
        }
        if (!cont) {
            s.alpha = fast_div(t[0], t[1]);
            s.beta = 0.0;
            s.first = 1;
        }
        s.gamma = t[0];
        s.keep_dir = 0;
        s.phase = PH_ITER;
        break;
    }
    case PH_ITER: {
        // the pass stepped alpha along a direction with r.u = gamma: it removed
        // alpha gamma of the error's A-norm energy
        s.e_cg += (float)(s.alpha * s.gamma);
        s.e_cg_n++;
        s.it_pcg++;
        s.it_total++;
        s.cur ^= 1;
        s.pcur ^= 1;
        s.mu = t[3] * sd.inv_n;
        double rr = t[2] - N * s.mu * s.mu;
        s.rho = nonneg(rr);
        s.first = 0;
        s.cg_count++;
        if (sd.mode == PPE_MODE_HYBRID && !s.fell_back && s.it_total >= sd.hybrid_budget) s.fell_back = 1;
        const double rho = s.rho;
        if (!isfinite(rho)) { to_res(s, 0); break; }
        double gnew = t[0];
        double beta = fast_div(gnew, s.gamma);
        // next direction p' = u' + beta p: p'.A p' = u'.Au' + 2 beta u'.(Ap) + beta^2 p.(Ap)
        double denom = t[1] + beta * (2.0 * t[4] + beta * t[5]);
        bool ok = denom > 0.0 && isfinite(beta) && gnew > 0.0;
        const double ru = sd.ru_delta * s.rho_ref;
        if (rho <= s.target * s.target || s.it_total >= iter_cap(sd) || !ok || rho <= ru * ru) {
            // gamma and alpha of the direction in use stay the reference for the
            // continuation after the residual replacement
            to_res(s, ok ? 1 : 0);
            break;
        }
        s.beta = beta;
        s.alpha = fast_div(gnew, denom);
        s.gamma = gnew;
        if (sd.mode == PPE_MODE_HYBRID && !s.fell_back && s.cg_count >= sd.num_cg) {
            s.dlsm_count = 0;
            s.phase = PH_NET;
        } else {
            s.phase = PH_ITER;
        }
        break;
    }
    case PH_DLSM_DOT: {
        s.net_calls++;
        double re = t[0], eq = t[1], ee = t[2];
        double a = fast_div(re, eq);
        if (!(eq > sd.dlsm_guard * ee * sd.diag_max) || !isfinite(a)) {
            s.dlsm_skipped++;
            s.keep_dir = sd.keep_dir_after_dlsm;
            s.reset_d = 0;
            s.phase = PH_RESTART;
        } else {
            s.alpha_d = a;
            s.e_dlsm = (float)(a * re);           // (r.e)^2 / (e.Ae): the energy this step removes
            s.phase = PH_DLSM_UPD;
        }
        break;
    }
    case PH_DLSM_UPD: {
        s.it_dlsm++;
        s.it_total++;
        s.cur ^= 1;
        s.mu = t[3] * sd.inv_n;
        double rr = t[2] - N * s.mu * s.mu;
        s.rho = nonneg(rr);
        // the step is worth its inference if it removed at least as much error
        // energy as dlsm_cost iterations of the CG phase before it (at their
        // mean); after several unprofitable steps in a row continue as plain PCG
        const bool useful = s.e_cg_n == 0 || s.e_dlsm >= (float)sd.dlsm_cost * (s.e_cg / (float)s.e_cg_n);
        s.dlsm_useless = useful ? 0 : s.dlsm_useless + 1;
        if (sd.dlsm_stall_limit > 0 && s.dlsm_useless >= sd.dlsm_stall_limit) s.fell_back = 1;
        s.dlsm_count++;
        if (sd.mode == PPE_MODE_HYBRID && !s.fell_back && s.it_total >= sd.hybrid_budget) s.fell_back = 1;
        const double ru = sd.ru_delta * s.rho_ref;
        if (s.rho <= s.target * s.target || s.it_total >= iter_cap(sd) || !isfinite(s.rho)) {
            to_res(s, 0);
        } else if (s.rho <= ru * ru) {
            to_res(s, sd.keep_dir_after_dlsm);   // residual replacement (mixed precision)
        } else if (s.dlsm_count < sd.num_dlsm && !s.fell_back) {
            s.phase = PH_NET;
        } else {
            s.keep_dir = sd.keep_dir_after_dlsm;
            s.reset_d = 0;
            s.phase = PH_RESTART;
        }
        break;
    }
    case PH_FINAL1:
        s.xmean = fast_div(t[1], t[0]);
        s.phase = PH_FINAL2;
        break;
    case PH_FINAL2:
        s.phase = PH_DONE;
        break;
    default:
        break;
    }
    s.gamma_f = (float)s.gamma;
    s.rho_f = (float)s.rho;
    s.target_sq_f = (float)(s.target * s.target);
    s.ru_sq_f = (float)(sd.ru_delta * s.rho_ref * sd.ru_delta * s.rho_ref);
    s.alpha_f = (float)s.alpha;
    s.beta_f = (float)s.beta;
    s.mu_f = (float)s.mu;
    s.alpha_d_f = (float)s.alpha_d;
}


// float-float product with an FP32 factor: (h + l) * b
__device__ __forceinline__ void ff_mul(float &h, float &l, float b)
{
    const float p = h * b;
    float e = fmaf(h, b, -p);
    e = fmaf(l, b, e);
    h = p + e;
    l = e - (h - p);
}

// The transition after an iteration pass of the FP32 kernels, in FP32 and
// float-float arithmetic: GB300's FP64 pipe has a long latency, and this
// transition is on the critical path of every iteration.  It computes what
// the PH_ITER case of advance() computes (the denominator p'.A p', where
// two terms nearly cancel, in float-float from the float-float dot
// products) and keeps the FP64 state fields in step for the other phases.
__device__ void advance_iter_f32(const SysDesc &sd, SysState &s, const float (&h)[NPART], const float (&l)[NPART])
{
    // Every field the transition reads is loaded first and every result
    // stored last: the state lives in shared memory, and interleaved
    // read-modify-writes would each wait for the previous store.
    const float alpha0 = s.alpha_f, gamma0 = s.gamma_f, ru_sq = s.ru_sq_f, target_sq = s.target_sq_f;
    const float e_cg = s.e_cg;
    const int e_cg_n = s.e_cg_n, it_pcg = s.it_pcg, it_total = s.it_total + 1, cg_count = s.cg_count + 1;
    const int cur = s.cur, pcur = s.pcur, it_rep = s.it_rep + 1, it_rep_prev = s.it_rep_prev;
    int fell_back = s.fell_back;
    const float inv_n = sd.inv_n_f, n_cells = sd.n_cells_f;
    const bool hybrid = sd.mode == PPE_MODE_HYBRID;
    const int budget = sd.hybrid_budget, num_cg = sd.num_cg, cap = iter_cap(sd);

    const float mu = (h[3] + l[3]) * inv_n;
    const float rr = (h[2] + l[2]) - n_cells * mu * mu;
    const float rho = nonneg(rr);
    if (hybrid && !fell_back && it_total >= budget) fell_back = 1;
    const float gnew = h[0] + l[0];
    const float beta = __fdiv_rn(gnew, gamma0);
    // p'.A p' = u'.Au' + beta (2 u'.(Ap) + beta p.(Ap)), in float-float
    float wh = h[5], wl = l[5];
    ff_mul(wh, wl, beta);
    ff_add(wh, wl, 2.f * h[4], 2.f * l[4]);
    ff_mul(wh, wl, beta);
    ff_add(wh, wl, h[1], l[1]);
    const float denom = wh + wl;
    const bool ok = denom > 0.f && isfinite(beta) && gnew > 0.f;
    // an inner solve that runs far past the length of the previous one
    // (2000 + 4x) ends with a residual replacement, so a stalled FP32
    // iteration is noticed by the refinement's stall test
    const bool overrun = it_rep > 2000 + 4 * it_rep_prev;

    // the step the pass took removed alpha gamma of the error's A-norm energy
    s.e_cg = e_cg + alpha0 * gamma0;
    s.e_cg_n = e_cg_n + 1;
    s.it_pcg = it_pcg + 1;
    s.it_total = it_total;
    s.cur = cur ^ 1;
    s.pcur = pcur ^ 1;
    s.first = 0;
    s.cg_count = cg_count;
    s.mu_f = mu;
    s.rho_f = rho;
    s.mu = (double)mu;
    s.rho = (double)rho;
    s.fell_back = fell_back;
    if (!isfinite(rho)) {
        to_res(s, 0);
        return;
    }
    s.it_rep = it_rep;
    s.overran = overrun && !(rho <= ru_sq);
    if (rho <= target_sq || it_total >= cap || !ok || rho <= ru_sq || overrun) {
        // gamma and alpha of the direction in use stay the reference for the
        // continuation after the residual replacement
        to_res(s, ok ? 1 : 0);
        return;
    }
    const float alpha = __fdiv_rn(gnew, denom);
    s.beta_f = beta;
    s.alpha_f = alpha;
    s.gamma_f = gnew;
    s.beta = (double)beta;
    s.alpha = (double)alpha;
    s.gamma = (double)gnew;
    if (hybrid && !fell_back && cg_count >= num_cg) {
        s.dlsm_count = 0;
        s.phase = PH_NET;
    } else {
        s.phase = PH_ITER;
    }
}

template <typename T, typename S>
__device__ void run_pass(S &sm, int q, int ph, int t, Acc &acc)
{
    const SysDesc &sd = sm.sd[q];
    const SysState &st = sm.st[q];
    int i0, j0;
    tile_origin<S::GK>(sd, t, i0, j0);
    switch (ph) {
    case PH_INIT: pass_init<T>(sm, sd, st, i0, j0, acc); break;
    case PH_RES: pass_res<T>(sm, sd, st, i0, j0, t, acc); break;
    case PH_RESTART: pass_restart<T>(sm, sd, st, i0, j0, t, acc); break;
    case PH_DLSM_DOT: pass_dlsm<T, S, false>(sm, sd, st, i0, j0, t, acc); break;
    case PH_DLSM_UPD: pass_dlsm<T, S, true>(sm, sd, st, i0, j0, t, acc); break;
    case PH_FINAL1: pass_final1<T>(sm, sd, st, i0, j0, acc); break;
    case PH_FINAL2: pass_final2<T>(sm, sd, st, i0, j0, acc); break;
    default: break;
    }
}

// max |b| = max |V S| of each system into st[s].bmax_bits (states zeroed
// before); blockIdx.y is the system.  A NaN in b gives NaN bits above every
// finite value, which the scale ignores (the init pass then reports the NaN).
__global__ void __launch_bounds__(256) scale_kernel(const SysDesc *sys, SysState *st, int n)
{
    const int s = blockIdx.y;
    if (s >= n) return;
    const SysDesc &sd = sys[s];
    const size_t cells = (size_t)sd.nx * sd.ny;
    double m = 0.0;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < cells; k += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(k % sd.nx), j = (int)(k / sd.nx);
        const double b = fabs(sd.dx[i] * sd.dy[j] * sd.f[k]);
        if (!(b <= m)) m = b;
    }
    // non-negative doubles order like their bit patterns
    unsigned long long bits = (unsigned long long)__double_as_longlong(m);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bits = max(bits, __shfl_xor_sync(0xffffffffu, bits, o));
    if ((threadIdx.x & 31) == 0 && bits) atomicMax((unsigned long long *)&st[s].bmax_bits, bits);
}

__device__ __forceinline__ void red_release_add_u32(uint32_t *p, uint32_t v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Block-reduce the per-warp accumulators (lane 0 of each warp) into threads
// 0..NPART-1 (fixed order).
// Block sums of the pass's partials (fixed order: warp shuffles, then a
// shuffle tree over the warps in warp 0), written as the block's record for
// this step; lane 0 of warp 0 then bumps the system's arrival counter.  The
// per-warp scratch alternates between two buffers, so a warp that runs ahead
// into the next system's pass cannot overwrite what warp 0 still reads.
// A step's device time, charged by each system's first block to the kind of
// pass the system ran in it (ph0[par]).
template <typename S> __device__ void charge_step(S &sm, int nq, uint64_t dt, int par)
{
    for (int q = 0; q < nq; ++q) {
        if ((int)blockIdx.x != sm.sd[q].blk0) continue;
        const int ph = sm.ph0[par][q];
        if (ph == PH_ITER || ph == PH_RESTART)
            sm.st[q].ns_pcg += dt;
        else if (ph == PH_DLSM_DOT || ph == PH_DLSM_UPD)
            sm.st[q].ns_dlsm += dt;
        else if (is_pass_phase(ph))
            sm.st[q].ns_fp64 += dt;
    }
}

template <typename S>
__device__ void block_publish(S &sm, const Acc &acc, Slot *slot, uint32_t *counter, int par)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NPART; ++k) {
            sm.red_hi[par][k][warp] = acc.hi[k];
            sm.red_lo[par][k][warp] = acc.lo[k];
        }
    __syncthreads();
    if (warp == 0) {
        float h[NPART], l[NPART];
#pragma unroll
        for (int k = 0; k < NPART; ++k) {
            h[k] = lane < NWARP ? sm.red_hi[par][k][lane] : 0.f;
            l[k] = lane < NWARP ? sm.red_lo[par][k][lane] : 0.f;
        }
#pragma unroll
        for (int o = NWARP / 2; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < NPART; ++k) {
                const float oh = __shfl_down_sync(0xffffffffu, h[k], o);
                const float ol = __shfl_down_sync(0xffffffffu, l[k], o);
                ff_add(h[k], l[k], oh, ol);
            }
        if (lane == 0) {
            float4 *dst = reinterpret_cast<float4 *>(slot);
            dst[0] = make_float4(h[0], h[1], h[2], h[3]);
            dst[1] = make_float4(h[4], h[5], l[0], l[1]);
            dst[2] = make_float4(l[2], l[3], l[4], l[5]);
            // release: the record's stores are visible before the count is
            red_release_add_u32(counter, 1u);
        }
    }
}

// GK selects the tile geometry: GEO_TILE, GEO_R8 and GEO_R4 run the
// tile-cooperative iteration pass on 128x16, 128x8 or 128x4 tiles, GEO_STREAM
// (FP32 only) the streaming pass; their register needs allow one block per
// SM.
template <typename T, int GK_>
__global__ void __launch_bounds__(SOLVER_THREADS, 1)
    solver_kernel(SolverArgs a, int resume_net)
{
    constexpr bool STREAM = GK_ == GEO_STREAM;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations need 128-byte alignment: round the base up (the launch
    // reserves 128 extra bytes)
    using Sm = SmemT<T, GK_>;
    Sm &sm = *reinterpret_cast<Sm *>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    const BlockRange br = a.ranges[blockIdx.x];
    const int nq = br.s1 - br.s0 + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // per-system description and state of the systems this block works on
    for (int q = 0; q < nq; ++q) {
        const int32_t *dsrc = reinterpret_cast<const int32_t *>(a.sys + br.s0 + q);
        int32_t *ddst = reinterpret_cast<int32_t *>(&sm.sd[q]);
        for (int k = threadIdx.x; k < (int)(sizeof(SysDesc) / 4); k += blockDim.x) ddst[k] = dsrc[k];
        const int32_t *ssrc = reinterpret_cast<const int32_t *>(a.st + br.s0 + q);
        int32_t *sdst = reinterpret_cast<int32_t *>(&sm.st[q]);
        for (int k = threadIdx.x; k < (int)(sizeof(SysState) / 4); k += blockDim.x) sdst[k] = ld_cg(ssrc + k);
    }
    if (threadIdx.x == 0) {
        sm.tag_d = sm.tag_f = -1;
        sm.go = 1;
        sm.fills = 0;
        sm.udirty = 1;
        sm.ptime[0] = 0;
        for (int k = 0; k < 16; ++k) sm.pacc[k] = 0;
        mbar_init(smem_u32(&sm.bar[0]), 1);
        mbar_init(smem_u32(&sm.bar[1]), 1);
        if constexpr (STREAM) {
            for (int w = 0; w < NWARP; ++w) {
                mbar_init(smem_u32(&sm.sbar[w][0]), 1);
                mbar_init(smem_u32(&sm.sbar[w][1]), 1);
                sm.sfills[w] = 0;
            }
        }
        mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0 && resume_net)
        for (int q = 0; q < nq; ++q)
            if (sm.st[q].phase == PH_NET) {
                sm.st[q].phase = PH_DLSM_DOT;
                // the direction was computed since the segment that asked for it ended
                if ((int)blockIdx.x == sm.sd[q].blk0) sm.st[q].ns_net += gtimer() - sm.st[q].t_net0;
            }
    __syncthreads();
    const bool prof = a.prof && blockIdx.x == 0 && threadIdx.x == 0;
    // profile split of one step (block 0): pass, block reduce + publish,
    // wait for the other blocks, reduction of their records, state advance
    uint64_t t_a = prof ? gtimer() : 0, t_p = 0, t_b = 0, t_w = 0, t_r = 0, t_x = 0, t_c = 0;
    int red_par = 0;
    uint32_t last_step = 0;   // the last step that ran (thread 0)
    for (uint32_t step = 1;; ++step) {
        // a step budget ends the launch at the same step in every block, so each
        // system stops between two of its steps
        if (a.max_steps > 0 && step > (uint32_t)a.max_steps) break;
        // any system of this block still running?
        bool any = false;
        for (int q = 0; q < nq; ++q) any |= is_pass_phase(sm.st[q].phase);
        if (!any) break;
        const int bank = step & 1;
        if (threadIdx.x == 0) {
            sm.tstep[bank] = gtimer();
            for (int q = 0; q < nq; ++q) sm.ph0[bank][q] = sm.st[q].phase;
            last_step = step;
        }
        // 1) passes; publish one record per live system
        for (int q = 0; q < nq; ++q) {
            const SysDesc &sd = sm.sd[q];
            const int ph = sm.st[q].phase;
            if (!is_pass_phase(ph)) continue;
            Acc acc;
            acc_zero(acc);
            const int lo_t = max(br.t0, sd.tile0), hi_t = min(br.t1, sd.tile0 + sd.ntiles);
            if (ph == PH_ITER) {
                if constexpr (STREAM)
                    pass_iter_stream(sm, q, lo_t, hi_t, acc, a);
                else
                    pass_iter<T>(sm, q, lo_t, hi_t, acc, a);
            } else {
                // the other passes write their scratch windows over the TMA stages
                if (threadIdx.x == 0) sm.udirty = 1;
                for (int t = lo_t; t < hi_t; ++t) run_pass<T>(sm, q, ph, t, acc);
            }
            if (prof && q == 0) t_p = gtimer();
            // test hook: one block withholds its record once, so that the other
            // blocks' bounded waits expire (the failure path of the barrier)
            if (a.skip_block == (int)blockIdx.x + 1 && step == 2) continue;
            Slot *slot = a.slots + (size_t)bank * a.nslots + sd.part0 + (blockIdx.x - sd.blk0);
            block_publish(sm, acc, slot, a.arrive + br.s0 + q, red_par);
            red_par ^= 1;
        }
        if (prof) t_b = gtimer();
        // 2) wait for the records of every block of each live system, reduce,
        //    advance: system q in warp q mod 16, so the systems a block spans
        //    (at most SMAX) are served at once; one block barrier per step
        for (int q = warp; q < nq; q += NWARP) {
            const SysDesc &sd = sm.sd[q];
            if (!is_pass_phase(sm.st[q].phase)) continue;
            {
                if (lane == 0) {
                    // every block of this system has published step `step`
                    const uint32_t need = step * (uint32_t)sd.nparts;
                    const uint32_t *cnt = a.arrive + br.s0 + q;
                    if (ld_acquire_u32(cnt) < need) {
                        const uint64_t t0 = gtimer();
                        while (ld_acquire_u32(cnt) < need) {
                            if ((int64_t)(gtimer() - t0) > a.spin_limit_ns) {
                                atomicExch(&a.ctl->err, (int32_t)PPE_ERR_TIMEOUT);
                                sm.go = 0;
                                break;
                            }
                            __nanosleep(20);
                        }
                    }
                    if (prof && q == 0) t_w = gtimer();
                }
                // the acquire of lane 0 and the warp barrier order every lane's
                // record loads after the other blocks' releases
                __syncwarp();
                // lane l adds records l, l + 32, ... in order, then a fixed shuffle
                // tree: every block obtains the same sums bit for bit
                float h[NPART], l[NPART];
#pragma unroll
                for (int k = 0; k < NPART; ++k) h[k] = l[k] = 0.f;
                const Slot *base = a.slots + (size_t)bank * a.nslots + sd.part0;
                auto add_slot = [&](const float4 &v0, const float4 &v1, const float4 &v2) {
                    ff_add(h[0], l[0], v0.x, v1.z);
                    ff_add(h[1], l[1], v0.y, v1.w);
                    ff_add(h[2], l[2], v0.z, v2.x);
                    ff_add(h[3], l[3], v0.w, v2.y);
                    ff_add(h[4], l[4], v1.x, v2.z);
                    ff_add(h[5], l[5], v1.y, v2.w);
                };
                int b = lane;
                // four, then two records per lane with their loads in flight
                // together (the order of the additions stays l, l + 32, ...)
                for (; b + 96 < sd.nparts; b += 128) {
                    float4 v[4][3];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float4 *sl = reinterpret_cast<const float4 *>(base + b + 32 * u);
                        v[u][0] = __ldcg(sl); v[u][1] = __ldcg(sl + 1); v[u][2] = __ldcg(sl + 2);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) add_slot(v[u][0], v[u][1], v[u][2]);
                }
                for (; b + 32 < sd.nparts; b += 64) {
                    float4 v[2][3];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const float4 *sl = reinterpret_cast<const float4 *>(base + b + 32 * u);
                        v[u][0] = __ldcg(sl); v[u][1] = __ldcg(sl + 1); v[u][2] = __ldcg(sl + 2);
                    }
#pragma unroll
                    for (int u = 0; u < 2; ++u) add_slot(v[u][0], v[u][1], v[u][2]);
                }
                for (; b < sd.nparts; b += 32) {
                    const float4 *sl = reinterpret_cast<const float4 *>(base + b);
                    add_slot(__ldcg(sl), __ldcg(sl + 1), __ldcg(sl + 2));
                }
#pragma unroll
                for (int k = 0; k < NPART; ++k) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        float oh = __shfl_down_sync(0xffffffffu, h[k], o);
                        float ol = __shfl_down_sync(0xffffffffu, l[k], o);
                        ff_add(h[k], l[k], oh, ol);
                    }
                }
                if (lane == 0 && sm.go) {
                    if (prof && q == 0) t_r = gtimer();
                    if (sizeof(T) == 4 && sm.st[q].phase == PH_ITER) {
                        advance_iter_f32(sd, sm.st[q], h, l);
                    } else {
                        double tt[NPART];
#pragma unroll
                        for (int k = 0; k < NPART; ++k) tt[k] = (double)h[k] + (double)l[k];
                        advance(sd, sm.st[q], tt);
                    }
                    if (prof && q == 0) t_x = gtimer();
                }
            }
        }
        // the previous step's device time, charged by a lane that waits for no
        // system (off the step's critical path; the last step is charged on exit)
        if (threadIdx.x == 32 * (NWARP - 1) && step > 1)
            charge_step(sm, nq, sm.tstep[bank] - sm.tstep[bank ^ 1], bank ^ 1);
        __syncthreads();
        if (!sm.go) return;                             // a bounded wait expired: leave without writing state
        if (prof) {
            t_c = gtimer();
            if (t_p && t_w && t_r) {
                unsigned long long *pa = sm.pacc;
                pa[0] += t_p - t_a;
                pa[1] += t_b - t_p;
                pa[2] += t_w - t_b;
                pa[3] += t_r - t_w;
                pa[4] += t_c - t_r;
                pa[5] += t_x - t_r;
                pa[7] += 1;
                // the iteration pass's parts (steps that ran one)
                if (sm.ptime[0]) {
                    pa[8] += sm.ptime[0] - t_a;
                    pa[9] += sm.ptime[1] - sm.ptime[0];
                    pa[10] += sm.ptime[2] - sm.ptime[1];
                    pa[11] += sm.ptime[3] - sm.ptime[2];
                    pa[12] += t_p - sm.ptime[3];
                    pa[13] += 1;
                    pa[14] += sm.ptime[4] - t_a;
                    pa[15] += sm.ptime[5] - sm.ptime[4];
                }
            }
            sm.ptime[0] = 0;
            t_p = t_w = t_r = 0;
            t_a = t_c;
        }
    }
    if (prof)
        for (int k = 0; k < 16; ++k) a.prof[k] += sm.pacc[k];
    if (threadIdx.x == 0 && last_step > 0)
        charge_step(sm, nq, gtimer() - sm.tstep[last_step & 1], (int)(last_step & 1));
    // a system that waits for a network direction starts its network clock
    if (threadIdx.x == 0)
        for (int q = 0; q < nq; ++q)
            if ((int)blockIdx.x == sm.sd[q].blk0 && sm.st[q].phase == PH_NET) sm.st[q].t_net0 = gtimer();
    __syncthreads();
    // write back the states of the systems this block owns
    for (int q = 0; q < nq; ++q) {
        if ((int)blockIdx.x != sm.sd[q].blk0) continue;
        const int32_t *src = reinterpret_cast<const int32_t *>(&sm.st[q]);
        int32_t *dst = reinterpret_cast<int32_t *>(a.st + br.s0 + q);
        for (int k = threadIdx.x; k < (int)(sizeof(SysState) / 4); k += blockDim.x) dst[k] = src[k];
    }
}

size_t solver_smem(SolverVariant v)
{
    switch (v) {
    case SV_FP64: return sizeof(SmemT<double, GEO_TILE>) + 128;
    case SV_FP32_STREAM: return sizeof(SmemT<float, GEO_STREAM>) + 128;
    case SV_FP64_R8: return sizeof(SmemT<double, GEO_R8>) + 128;
    case SV_FP32_R8: return sizeof(SmemT<float, GEO_R8>) + 128;
    case SV_FP64_R4: return sizeof(SmemT<double, GEO_R4>) + 128;
    case SV_FP32_R4: return sizeof(SmemT<float, GEO_R4>) + 128;
    default: return sizeof(SmemT<float, GEO_TILE>) + 128;
    }
}

const void *solver_fn(SolverVariant v)
{
    switch (v) {
    case SV_FP64: return (const void *)solver_kernel<double, GEO_TILE>;
    case SV_FP32_STREAM: return (const void *)solver_kernel<float, GEO_STREAM>;
    case SV_FP64_R8: return (const void *)solver_kernel<double, GEO_R8>;
    case SV_FP32_R8: return (const void *)solver_kernel<float, GEO_R8>;
    case SV_FP64_R4: return (const void *)solver_kernel<double, GEO_R4>;
    case SV_FP32_R4: return (const void *)solver_kernel<float, GEO_R4>;
    default: return (const void *)solver_kernel<float, GEO_TILE>;
    }
}


}  // namespace

// The dynamic shared-memory opt-in is a per-function attribute of each
// device: set it once per device.
void set_solver_attributes()
{
    static PerDevice pd;
    once_per_device(pd, [](int) {
        for (int v = 0; v < SV_COUNT; ++v)
            if (cudaFuncSetAttribute(solver_fn((SolverVariant)v), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)solver_smem((SolverVariant)v)) != cudaSuccess)
                return false;
        return true;
    });
}

const void *solver_kernel_fn(SolverVariant v) { return solver_fn(v); }
size_t solver_smem_bytes(SolverVariant v) { return solver_smem(v); }

const void *scale_kernel_fn() { return (const void *)scale_kernel; }

dim3 scale_grid(int n, long max_cells)
{
    const long gx = std::min<long>(64, std::max<long>(1, (max_cells + 255) / 256));
    return dim3((unsigned)gx, (unsigned)n);
}

ppe_status launch_scale(const SysDesc *sys, SysState *st, int n, long max_cells, cudaStream_t s)
{
    scale_kernel<<<scale_grid(n, max_cells), 256, 0, s>>>(sys, st, n);
    PPE_CUDA_TRY(cudaGetLastError());
    return PPE_OK;
}

int solver_max_blocks(SolverVariant v, int blocks_per_sm_req)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    set_solver_attributes();
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solver_fn(v), SOLVER_THREADS, solver_smem(v));
    if (blocks_per_sm_req > 0 && blocks_per_sm_req < per_sm) per_sm = blocks_per_sm_req;
    return per_sm * sms;
}

ppe_status launch_solver_resume(const SolverArgs &a, SolverVariant v, int grid_blocks, cudaStream_t stream, int resume)
{
    SolverArgs args = a;
    int res = resume;
    void *params[] = {&args, &res};
    set_solver_attributes();
    cudaError_t e = cudaLaunchCooperativeKernel(solver_fn(v), dim3(grid_blocks), dim3(SOLVER_THREADS), params,
                                                solver_smem(v), stream);
    if (e != cudaSuccess) return cuda_status(e, "cudaLaunchCooperativeKernel(solver)");
    return PPE_OK;
}

ppe_status encode_solver_maps(void *const r[2], void *const p[2], void *d, const float *ycoef, int nx, int ny,
                              int pitch, SolverVariant v, CUtensorMap out[NMAPS])
{
    const bool fp64 = solver_variant_fp64(v), stream = v == SV_FP32_STREAM;
    // tile-cooperative kernels: one tile window (136 x (th + 4)) and one tile
    // (128 x th); streaming kernel: chunks of SRB rows of a 132-wide window
    // and of a 124-wide tile
    const cuuint32_t th = (cuuint32_t)solver_tile_h(v);
    const cuuint32_t win_w = stream ? S_WX : WIN_X, win_h = stream ? SRB : th + 2 * WIN_OY;
    const cuuint32_t tile_w = stream ? TILE_X_STREAM : TILE_X, tile_h = stream ? SRB : th;
    auto encode = tensor_map_encoder();
    if (!encode) {
        set_error("cuTensorMapEncodeTiled unavailable");
        return PPE_ERR_CUDA;
    }
    const size_t es = fp64 ? 8 : 4;
    if (pitch % 4 != 0 || pitch < nx) {
        set_error("encode_solver_maps: pitch must be a multiple of 4 and at least nx");
        return PPE_ERR_ARG;
    }
    void *const bufs[MAP_Y] = {r[0], r[1], p[0], p[1], d};
    std::memset(&out[MAP_Y], 0, sizeof(CUtensorMap));
    if (ycoef) {
        if ((uintptr_t)ycoef % 16 != 0) {
            set_error("encode_solver_maps: row coefficients not 16-byte aligned");
            return PPE_ERR_ARG;
        }
        cuuint64_t dims[2] = {4, (cuuint64_t)ny};
        cuuint64_t strides[1] = {16};
        cuuint32_t box[2] = {4, (cuuint32_t)(stream ? SRB : 1)};
        cuuint32_t estr[2] = {1, 1};
        CUresult cr = encode(&out[MAP_Y], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)ycoef, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) {
            set_error("cuTensorMapEncodeTiled(row coefficients) failed");
            return PPE_ERR_CUDA;
        }
    }
    for (int m = 0; m < MAP_Y; ++m) {
        if ((uintptr_t)bufs[m] % 16 != 0) {
            set_error("encode_solver_maps: vector not 16-byte aligned");
            return PPE_ERR_ARG;
        }
        const bool win = m != MAP_D;
        cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
        cuuint64_t strides[1] = {(cuuint64_t)pitch * es};
        cuuint32_t box[2] = {win ? win_w : tile_w, win ? win_h : tile_h};
        cuuint32_t estr[2] = {1, 1};
        CUresult cr = encode(&out[m], fp64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                             bufs[m], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) {
            set_error("cuTensorMapEncodeTiled(solver vectors) failed");
            return PPE_ERR_CUDA;
        }
    }
    return PPE_OK;
}

}  // namespace ppe
