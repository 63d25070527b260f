// Multigrid-preconditioned CG: the CG-type partner the paper calls MGPCG-4
// (Sec. 2.6, Tables 2-3: CG with one multigrid V-cycle per iteration as its
// preconditioner; there an algebraic hierarchy from PETSc), restated for the
// tensor-product grid:
//   * hierarchy: level l+1 merges neighbouring pairs of cells along each axis
//     (an odd last cell stays alone, an axis of one cell is kept), down to a
//     level of at most MG_COARSE_CELLS cells;
//   * operator on every level: the same volume-scaled 5-point operator built
//     from that level's widths;
//   * prolongation P: per axis, linear interpolation between a cell's parent
//     and the coarse neighbour on its side of the parent's centre (the
//     parent's value at walls); restriction R = P^T, so the V-cycle is
//     symmetric;
//   * smoother: damped line Jacobi (omega = 0.8), x-lines then y-lines before
//     the coarse correction, y then x after.  Each line is a tridiagonal system
//     (its diagonal and the couplings along the line), solved by a warp with
//     the partition method (segments per lane, parallel cyclic reduction of
//     the segments' interface system).  Line relaxation is what keeps the
//     smoother effective on stretched cells, whose couplings along the two
//     axes differ by the cell aspect ratio;
//   * coarsest level: the pseudo-inverse of its singular Neumann operator
//     applied to the zero-sum residual.
//
// One cooperative persistent kernel runs a whole solve: FP64 true residuals
// and iterative refinement around FP32 inner MG-PCG iterations.  Levels with
// more than MG_LOCAL_CELLS cells are processed by every block, with a bounded
// grid barrier between dependent passes; the smaller levels of a V-cycle run
// inside block 0 alone (block barriers only) while the other blocks wait.
// Every reduction sums per-block partials in a fixed order, so every block
// obtains the same scalars bit for bit.  Every wait is bounded: on expiry the
// kernel records PPE_ERR_TIMEOUT and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "tma.cuh"

namespace ppe {

namespace {

constexpr int MG_THREADS = 512;
constexpr int MG_WARPS = MG_THREADS / 32;
constexpr int MG_COARSE_CELLS = 256;
constexpr int MG_LOCAL_CELLS = 1024;     // levels at most this large run in block 0 (measured: 1024 beats 256, 512, 4096 and 16384)
constexpr int MG_MAX_LEVELS = 24;
constexpr float MG_OMEGA = 0.8f;
constexpr float MG_INNER_RTOL = 1e-4f;     // FP32 inner solve: residual drop per refinement
constexpr int MG_INNER_MAX = 200;           // inner iterations before a refinement is forced (the
                                            // preconditioned iteration needs about ten)

struct MgLevel {
    int nx, ny, cx, cy;                   // cx/cy: the axis is coarsened towards the next level
    const float *dx, *dy, *fx, *fy;       // widths, face coefficients (0 at walls)
    const int *pxp, *pxn, *pyp, *pyn;     // this level's cells: parent and side neighbour on the next level (-1: none)
    const float *pxw, *pyw;               // interpolation weight of the neighbour (parent: 1 - w)
    float *r, *za, *zb, *t;               // right-hand side, corrections (za holds the result), residual
    float *s1, *s2;                       // line-solve scratch (with t)
};

struct MgReport {
    int32_t status, iters, refinements, stalled;
    double relres, incompat;
    unsigned long long ns;
};

struct MgArgs {
    const MgLevel *lv;
    int nlev, local0;                     // levels; the first level block 0 runs alone
    const float *pinv;                    // coarsest-level pseudo-inverse [nc][nc]
    int nx, ny;
    const double *dx, *dy, *fx, *fy;      // the grid in FP64 (true residuals)
    const double *S;
    double *x, *r64;
    float *p, *q, *d;
    double tol;
    int max_iters;
    int mode;                             // 0: solve; 1: apply one V-cycle to lv[0].r (result in lv[0].za)
    double *part;                         // [2][gridDim.x][4] reduction partials
    unsigned *bar;                        // [0] arrivals, [1] generation
    int *err;
    long long spin_ns;
    MgReport *rep;
};

// ---------------------------------------------------------------------------
// synchronisation
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned ld_acq(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

struct Sync {
    unsigned gen;      // generations this block has passed
    int par;           // reduction buffer parity
};

// Bounded generation barrier over the grid; false (and PPE_ERR_TIMEOUT
// recorded) if the other blocks do not arrive within the limit.
__device__ bool grid_bar(const MgArgs &a, Sync &s)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = s.gen + 1;
        __threadfence();
        if (atomicAdd(&a.bar[0], 1u) == gridDim.x - 1) {
            atomicExch(&a.bar[0], 0u);
            __threadfence();
            atomicExch(&a.bar[1], target);
        } else if (ld_acq(&a.bar[1]) != target) {
            const uint64_t t0 = gtimer();
            while (ld_acq(&a.bar[1]) != target) {
                if ((long long)(gtimer() - t0) > a.spin_ns) {
                    ok = 0;
                    atomicExch(a.err, (int)PPE_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(32);
            }
        }
        // no fence here: the last block's fence above acquires the others'
        // arrivals, a waiter's acquire load the last block's release, and the
        // block barrier below orders the block's later loads after either
        s.gen = target;
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// Sum K doubles over the whole grid: the same result in every block.
template <int K> __device__ bool grid_sum(const MgArgs &a, Sync &s, double (&v)[K])
{
    __shared__ double red[MG_WARPS][4];
    __shared__ double res[4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double x = v[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp][k] = x;
    }
    __syncthreads();
    double *part = a.part + (size_t)s.par * gridDim.x * 4;
    if (threadIdx.x < K) {
        double x = 0.0;
        for (int w = 0; w < MG_WARPS; ++w) x += red[w][threadIdx.x];
        part[blockIdx.x * 4 + threadIdx.x] = x;
    }
    if (!grid_bar(a, s)) return false;
    if (threadIdx.x < K) {
        double x = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) x += __ldcg(&part[b * 4 + threadIdx.x]);
        res[threadIdx.x] = x;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = res[k];
    s.par ^= 1;
    return true;
}

// Work distribution: cells over (wid, nw) workers; lines in groups of 32
// consecutive lines per warp (coalesced along y-lines).
struct Dist {
    int wid, nw, g0, gs;
};
__device__ __forceinline__ Dist grid_dist()
{
    const int warp = threadIdx.x >> 5;
    return {(int)(blockIdx.x * blockDim.x + threadIdx.x), (int)(gridDim.x * blockDim.x),
            (int)(blockIdx.x + gridDim.x * warp), (int)(gridDim.x * MG_WARPS)};
}
__device__ __forceinline__ Dist local_dist() { return {(int)threadIdx.x, (int)blockDim.x, (int)(threadIdx.x >> 5), MG_WARPS}; }

// ---------------------------------------------------------------------------
// level operations
// ---------------------------------------------------------------------------

// (A z) at cell (i, j) of a level
__device__ __forceinline__ float apply_at(const MgLevel &L, const float *z, int i, int j)
{
    const int nx = L.nx;
    const size_t k = (size_t)j * nx + i;
    const float c = z[k];
    float ax = 0.f, ay = 0.f;
    if (i > 0) ax += L.fx[i] * (c - z[k - 1]);
    if (i + 1 < nx) ax += L.fx[i + 1] * (c - z[k + 1]);
    if (j > 0) ay += L.fy[j] * (c - z[k - nx]);
    if (j + 1 < L.ny) ay += L.fy[j + 1] * (c - z[k + nx]);
    return L.dy[j] * ax + L.dx[i] * ay;
}

// One line system T x = rhs of a sweep, solved by a whole warp with the
// partition method.  The line's n unknowns are split into K = min(32, n)
// contiguous segments, one per lane.  A lane eliminates the interior of its
// segment (all but its last unknown) for three right-hand sides at once: the
// line's, and the two spikes that carry the couplings to the last unknowns of
// the previous and of its own segment.  Substituting the interiors into the
// segments' last rows leaves a K x K tridiagonal system in those last
// unknowns, solved by parallel cyclic reduction across the lanes; each lane
// then forms its interior.  The serial work per lane is about n / 32 steps
// instead of n.  Scratch: t (modified super-diagonal), zout, s1, s2 (the
// three right-hand sides), indexed like the line's cells.
//
// LineX / LineY give, for position k of the line: its cell index, the
// tridiagonal coefficients (a k-1 coupling, b diagonal, c k+1 coupling) and
// the right-hand side r - mu - A zin at that cell.
struct LineX {
    const MgLevel &L;
    int j;
    float mu;
    const float *zin;
    __device__ int n() const { return L.nx; }
    __device__ size_t cell(int k) const { return (size_t)j * L.nx + k; }
    __device__ void coef(int k, float &a, float &b, float &c) const
    {
        const float dyj = L.dy[j], fl = L.fx[k], fr = L.fx[k + 1];
        a = -dyj * fl;
        c = -dyj * fr;
        b = dyj * (fl + fr) + L.dx[k] * (L.fy[j] + L.fy[j + 1]);
    }
    __device__ float rhs(int k) const
    {
        float v = L.r[cell(k)] - mu;
        if (zin) v -= apply_at(L, zin, k, j);
        return v;
    }
};
struct LineY {
    const MgLevel &L;
    int i;
    float mu;
    const float *zin;
    __device__ int n() const { return L.ny; }
    __device__ size_t cell(int k) const { return (size_t)k * L.nx + i; }
    __device__ void coef(int k, float &a, float &b, float &c) const
    {
        const float dxi = L.dx[i], fl = L.fy[k], fr = L.fy[k + 1];
        a = -dxi * fl;
        c = -dxi * fr;
        b = dxi * (fl + fr) + L.dy[k] * (L.fx[i] + L.fx[i + 1]);
    }
    __device__ float rhs(int k) const
    {
        float v = L.r[cell(k)] - mu;
        if (zin) v -= apply_at(L, zin, i, k);
        return v;
    }
};

// zout = zin + omega T^{-1} rhs on one line (zin = nullptr: zero); with dot,
// accumulate (r - mu) . zout.
template <class Line>
__device__ void warp_line(const Line &ln, const MgLevel &L, float mu, const float *zin, float *zout, double *dot)
{
    const int lane = threadIdx.x & 31;
    const int n = ln.n();
    const int K = n < 32 ? n : 32;
    const int base = n / K, extra = n % K;
    const bool has = lane < K;
    const int p = has ? lane * base + min(lane, extra) : n;
    const int m = has ? base + (lane < extra ? 1 : 0) : 0;
    const int mi = m - 1;                       // interior unknowns of the segment
    float *sc = L.t, *sy = zout, *sv = L.s1, *sw = L.s2;
    // forward elimination of the interior with three right-hand sides
    float cp = 0.f, yp = 0.f, vp = 0.f, wp = 0.f;
    for (int k = 0; k < mi; ++k) {
        float a, b, c;
        ln.coef(p + k, a, b, c);
        const float d = ln.rhs(p + k);
        const float rv = k == 0 ? -a : 0.f;     // coupling to the previous segment's last unknown
        const float rw = k == mi - 1 ? -c : 0.f;  // coupling to this segment's last unknown
        const float aa = k == 0 ? 0.f : a, cc = k == mi - 1 ? 0.f : c;
        const float inv = 1.f / (b - aa * cp);
        cp = cc * inv;
        yp = (d - aa * yp) * inv;
        vp = (rv - aa * vp) * inv;
        wp = (rw - aa * wp) * inv;
        const size_t q = ln.cell(p + k);
        sc[q] = cp;
        sy[q] = yp;
        sv[q] = vp;
        sw[q] = wp;
    }
    // back substitution: interior x = y + v * x_prev_last + w * x_last
    float xy = 0.f, xv = 0.f, xw = 0.f;
    for (int k = mi - 1; k >= 0; --k) {
        const size_t q = ln.cell(p + k);
        const float c = sc[q];
        xy = sy[q] - c * xy;
        xv = sv[q] - c * xv;
        xw = sw[q] - c * xw;
        sy[q] = xy;
        sv[q] = xv;
        sw[q] = xw;
    }
    // the segment's last row, in terms of the last unknowns L_{l-1}, L_l, L_{l+1}
    float A = 0.f, B = 1.f, C = 0.f, D = 0.f;
    // first interior of this segment (for the previous lane's row): x = y0 + v0 L_{l-1} + w0 L_l
    float y0 = 0.f, v0 = 0.f, w0 = 1.f;          // no interior: x_p is L_l itself
    if (mi >= 1) {
        const size_t q = ln.cell(p);
        y0 = sy[q];
        v0 = sv[q];
        w0 = sw[q];
    }
    const float y0n = __shfl_down_sync(0xffffffffu, y0, 1), v0n = __shfl_down_sync(0xffffffffu, v0, 1),
                w0n = __shfl_down_sync(0xffffffffu, w0, 1);
    if (has) {
        float a, b, c;
        const int kl = p + m - 1;
        ln.coef(kl, a, b, c);
        const float d = ln.rhs(kl);
        // x_{kl-1}: the last interior (or L_{l-1} when there is none)
        float yl = 0.f, vl = 1.f, wl = 0.f;
        if (mi >= 1) {
            const size_t q = ln.cell(kl - 1);
            yl = sy[q];
            vl = sv[q];
            wl = sw[q];
        }
        // x_{kl+1}: the next segment's first unknown, y0n + v0n L_l + w0n L_{l+1}
        // (c = 0 on the line's last row)
        const bool last_seg = lane == K - 1;
        const float cn = last_seg ? 0.f : c;
        A = a * vl;
        B = b + a * wl + cn * v0n;
        C = cn * w0n;
        D = d - a * yl - cn * y0n;
        if (lane == 0) A = 0.f;
        if (last_seg) C = 0.f;
    }
    // parallel cyclic reduction of the K x K system A L_{l-1} + B L_l + C L_{l+1} = D
    for (int s = 1; s < 32; s <<= 1) {
        const float Am = __shfl_up_sync(0xffffffffu, A, s), Bm = __shfl_up_sync(0xffffffffu, B, s),
                    Cm = __shfl_up_sync(0xffffffffu, C, s), Dm = __shfl_up_sync(0xffffffffu, D, s);
        const float Ap = __shfl_down_sync(0xffffffffu, A, s), Bp = __shfl_down_sync(0xffffffffu, B, s),
                    Cp = __shfl_down_sync(0xffffffffu, C, s), Dp = __shfl_down_sync(0xffffffffu, D, s);
        const bool lo = lane >= s, hi = lane + s < 32;
        const float k1 = lo ? A / Bm : 0.f, k2 = hi ? C / Bp : 0.f;
        const float nA = lo ? -Am * k1 : 0.f, nC = hi ? -Cp * k2 : 0.f;
        B = B - (lo ? Cm * k1 : 0.f) - (hi ? Ap * k2 : 0.f);
        D = D - (lo ? Dm * k1 : 0.f) - (hi ? Dp * k2 : 0.f);
        A = nA;
        C = nC;
    }
    const float Ll = D / B;
    float Lp = __shfl_up_sync(0xffffffffu, Ll, 1);      // every lane takes part in the shuffle
    if (lane == 0) Lp = 0.f;
    if (!has) return;
    // the segment's unknowns, and the update zout = zin + omega x
    for (int k = 0; k < m; ++k) {
        const size_t q = ln.cell(p + k);
        const float xk = k == m - 1 ? Ll : sy[q] + sv[q] * Lp + sw[q] * Ll;
        const float z = (zin ? zin[q] : 0.f) + MG_OMEGA * xk;
        zout[q] = z;
        if (dot) *dot += (double)(L.r[q] - mu) * (double)z;
    }
}

// Lines are spread over warps (consecutive lines in neighbouring warps of a
// block, which share cache lines along y).  grid: every block; local: block 0.
__device__ __forceinline__ void line_range(bool grid, int &w0, int &ws)
{
    const int warp = threadIdx.x >> 5;
    w0 = grid ? (int)(blockIdx.x * MG_WARPS + warp) : warp;
    ws = grid ? (int)(gridDim.x * MG_WARPS) : MG_WARPS;
}

// zout = zin + omega T_x^{-1} (r - mu - A zin) row by row (zin = nullptr: zero).
// With dot: accumulate (r - mu) . zout.
__device__ void xsweep(const MgLevel &L, float mu, const float *zin, float *zout, bool grid, double *dot)
{
    int w0, ws;
    line_range(grid, w0, ws);
    for (int j = w0; j < L.ny; j += ws) warp_line(LineX{L, j, mu, zin}, L, mu, zin, zout, dot);
}

// The same along columns, by whole blocks: a block takes 32 adjacent columns
// (lane = column, so that every load of a warp is one row segment) and cuts
// each column into MG_WARPS row segments, one per warp.  Each thread
// eliminates its segment's interior as in warp_line; the segments' last rows
// form a small tridiagonal system per column (one unknown per warp), solved
// by warp 0 through shared memory.  grid: the blocks take column groups in
// turn; local: block 0 takes them all.
__device__ void ysweep(const MgLevel &L, float mu, const float *zin, float *zout, bool grid)
{
    __shared__ float sh_y0[MG_WARPS][32], sh_v0[MG_WARPS][32], sh_w0[MG_WARPS][32];
    __shared__ float sh_A[MG_WARPS][32], sh_B[MG_WARPS][32], sh_C[MG_WARPS][32], sh_D[MG_WARPS][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ny = L.ny;
    const int K = ny < MG_WARPS ? ny : MG_WARPS;
    const int base = ny / K, extra = ny % K;
    const bool hasseg = warp < K;
    const int p = hasseg ? warp * base + min(warp, extra) : ny;
    const int m = hasseg ? base + (warp < extra ? 1 : 0) : 0;
    const int mi = m - 1;
    float *sc = L.t, *sy = zout, *sv = L.s1, *sw = L.s2;
    const int g0 = grid ? (int)blockIdx.x : 0, gs = grid ? (int)gridDim.x : 1;
    for (int cg = g0; cg * 32 < L.nx; cg += gs) {
        const int i = cg * 32 + lane;
        const bool col = i < L.nx;
        const bool has = hasseg && col;
        const LineY ln{L, col ? i : 0, mu, zin};
        float cp = 0.f, yp = 0.f, vp = 0.f, wp = 0.f;
        if (has) {
            for (int k = 0; k < mi; ++k) {
                float a, b, c;
                ln.coef(p + k, a, b, c);
                const float d = ln.rhs(p + k);
                const float rv = k == 0 ? -a : 0.f;
                const float rw = k == mi - 1 ? -c : 0.f;
                const float aa = k == 0 ? 0.f : a, cc = k == mi - 1 ? 0.f : c;
                const float inv = 1.f / (b - aa * cp);
                cp = cc * inv;
                yp = (d - aa * yp) * inv;
                vp = (rv - aa * vp) * inv;
                wp = (rw - aa * wp) * inv;
                const size_t q = ln.cell(p + k);
                sc[q] = cp;
                sy[q] = yp;
                sv[q] = vp;
                sw[q] = wp;
            }
            float xy = 0.f, xv = 0.f, xw = 0.f;
            for (int k = mi - 1; k >= 0; --k) {
                const size_t q = ln.cell(p + k);
                const float c = sc[q];
                xy = sy[q] - c * xy;
                xv = sv[q] - c * xv;
                xw = sw[q] - c * xw;
                sy[q] = xy;
                sv[q] = xv;
                sw[q] = xw;
            }
        }
        float y0 = 0.f, v0 = 0.f, w0 = 1.f;
        if (has && mi >= 1) {
            const size_t q = ln.cell(p);
            y0 = sy[q];
            v0 = sv[q];
            w0 = sw[q];
        }
        sh_y0[warp][lane] = y0;
        sh_v0[warp][lane] = v0;
        sh_w0[warp][lane] = w0;
        __syncthreads();
        float A = 0.f, B = 1.f, C = 0.f, D = 0.f;
        if (has) {
            float a, b, c;
            const int kl = p + m - 1;
            ln.coef(kl, a, b, c);
            const float d = ln.rhs(kl);
            float yl = 0.f, vl = 1.f, wl = 0.f;
            if (mi >= 1) {
                const size_t q = ln.cell(kl - 1);
                yl = sy[q];
                vl = sv[q];
                wl = sw[q];
            }
            const bool last_seg = warp == K - 1;
            const float cn = last_seg ? 0.f : c;
            const float y0n = last_seg ? 0.f : sh_y0[warp + 1][lane], v0n = last_seg ? 0.f : sh_v0[warp + 1][lane],
                        w0n = last_seg ? 0.f : sh_w0[warp + 1][lane];
            A = warp == 0 ? 0.f : a * vl;
            B = b + a * wl + cn * v0n;
            C = last_seg ? 0.f : cn * w0n;
            D = d - a * yl - cn * y0n;
        }
        sh_A[warp][lane] = A;
        sh_B[warp][lane] = B;
        sh_C[warp][lane] = C;
        sh_D[warp][lane] = D;
        __syncthreads();
        if (warp == 0 && col) {
            // Thomas over the K segment unknowns of column i (diagonally dominant)
            float cpr = 0.f, dpr = 0.f;
            for (int w = 0; w < K; ++w) {
                const float inv = 1.f / (sh_B[w][lane] - sh_A[w][lane] * cpr);
                cpr = sh_C[w][lane] * inv;
                dpr = (sh_D[w][lane] - sh_A[w][lane] * dpr) * inv;
                sh_C[w][lane] = cpr;
                sh_D[w][lane] = dpr;
            }
            float xn = 0.f;
            for (int w = K - 1; w >= 0; --w) {
                xn = sh_D[w][lane] - sh_C[w][lane] * xn;
                sh_D[w][lane] = xn;
            }
        }
        __syncthreads();
        if (has) {
            const float Ll = sh_D[warp][lane];
            const float Lp = warp == 0 ? 0.f : sh_D[warp - 1][lane];
            for (int k = 0; k < m; ++k) {
                const size_t q = ln.cell(p + k);
                const float xk = k == m - 1 ? Ll : sy[q] + sv[q] * Lp + sw[q] * Ll;
                zout[q] = (zin ? zin[q] : 0.f) + MG_OMEGA * xk;
            }
        }
        __syncthreads();           // the shared arrays are reused by the next column group
    }
}

// t = r - mu - A z
__device__ void residual(const MgLevel &L, float mu, const float *z, float *t, const Dist &d)
{
    const int n = L.nx * L.ny;
    for (int k = d.wid; k < n; k += d.nw) {
        const int i = k % L.nx, j = k / L.nx;
        t[k] = L.r[k] - mu - apply_at(L, z, i, j);
    }
}

// weight of fine index f for coarse index c along one axis
__device__ __forceinline__ float axis_w(const int *par, const int *nb, const float *w, int f, int c)
{
    return (par[f] == c ? 1.f - w[f] : 0.f) + (nb[f] == c ? w[f] : 0.f);
}

// rc = P^T t: each coarse cell gathers its fine contributors
__device__ void restrict_to(const MgLevel &F, const MgLevel &C, const float *t, const Dist &d)
{
    const int n = C.nx * C.ny;
    for (int k = d.wid; k < n; k += d.nw) {
        const int I = k % C.nx, J = k / C.nx;
        const int i0 = F.cx ? max(0, 2 * I - 1) : I, i1 = F.cx ? min(F.nx - 1, 2 * I + 2) : I;
        const int j0 = F.cy ? max(0, 2 * J - 1) : J, j1 = F.cy ? min(F.ny - 1, 2 * J + 2) : J;
        float s = 0.f;
        for (int j = j0; j <= j1; ++j) {
            const float wy = axis_w(F.pyp, F.pyn, F.pyw, j, J);
            if (wy == 0.f) continue;
            float sx = 0.f;
            for (int i = i0; i <= i1; ++i) {
                const float wx = axis_w(F.pxp, F.pxn, F.pxw, i, I);
                if (wx != 0.f) sx += wx * t[(size_t)j * F.nx + i];
            }
            s += wy * sx;
        }
        C.r[k] = s;
    }
}

// zout = zin + P zc
__device__ void prolong_add(const MgLevel &F, const MgLevel &C, const float *zc, const float *zin, float *zout,
                            const Dist &d)
{
    const int n = F.nx * F.ny;
    for (int k = d.wid; k < n; k += d.nw) {
        const int i = k % F.nx, j = k / F.nx;
        const int ip = F.pxp[i], in = F.pxn[i], jp = F.pyp[j], jn = F.pyn[j];
        const float wx = F.pxw[i], wy = F.pyw[j];
        float v = (1.f - wx) * (1.f - wy) * zc[(size_t)jp * C.nx + ip];
        if (in >= 0) v += wx * (1.f - wy) * zc[(size_t)jp * C.nx + in];
        if (jn >= 0) v += (1.f - wx) * wy * zc[(size_t)jn * C.nx + ip];
        if (in >= 0 && jn >= 0) v += wx * wy * zc[(size_t)jn * C.nx + in];
        zout[k] = zin[k] + v;
    }
}

// Coarsest level (block 0): za = pinv (r - mean r).  With dot (the level is
// the grid itself): accumulate (r - mu) . za.
__device__ void coarsest(const MgArgs &a, const MgLevel &L, float mu, double *dot)
{
    __shared__ float red[MG_WARPS];
    __shared__ float mean_s;
    const int n = L.nx * L.ny;
    float s = 0.f;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s += L.r[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < MG_WARPS; ++w) t += red[w];
        mean_s = t / (float)n;
    }
    __syncthreads();
    const float m = mean_s;
    for (int row = threadIdx.x; row < n; row += blockDim.x) {
        float z = 0.f;
        for (int c = 0; c < n; ++c) z += a.pinv[(size_t)row * n + c] * (L.r[c] - m);
        L.za[row] = z;
        if (dot) *dot += (double)(L.r[row] - mu) * (double)z;
    }
}

// Levels l0 .. nlev-1 of a V-cycle inside block 0 (block barriers only).
__device__ void local_vcycle(const MgArgs &a, int l0, float mu0, double *dot)
{
    const Dist d = local_dist();
    const int last = a.nlev - 1;
    for (int l = l0; l < last; ++l) {
        const MgLevel &L = a.lv[l];
        const float mu = l == 0 ? mu0 : 0.f;
        xsweep(L, mu, nullptr, L.za, false, nullptr);
        __syncthreads();
        ysweep(L, mu, L.za, L.zb, false);
        __syncthreads();
        residual(L, mu, L.zb, L.t, d);
        __syncthreads();
        restrict_to(L, a.lv[l + 1], L.t, d);
        __syncthreads();
    }
    coarsest(a, a.lv[last], last == 0 ? mu0 : 0.f, last == 0 ? dot : nullptr);
    __syncthreads();
    for (int l = last - 1; l >= l0; --l) {
        const MgLevel &L = a.lv[l];
        const float mu = l == 0 ? mu0 : 0.f;
        prolong_add(L, a.lv[l + 1], a.lv[l + 1].za, L.zb, L.za, d);
        __syncthreads();
        ysweep(L, mu, L.za, L.zb, false);
        __syncthreads();
        xsweep(L, mu, L.zb, L.za, false, l == 0 ? dot : nullptr);
        __syncthreads();
    }
}

// One V-cycle on lv[0].r - mu0; the result in lv[0].za; dot accumulates
// (r - mu0) . za in the threads that wrote za.  Ends with lv[0].za written by
// this block's share (the caller's barrier or reduction publishes it).
__device__ bool vcycle(const MgArgs &a, Sync &s, float mu0, double *dot)
{
    const Dist d = grid_dist();
    for (int l = 0; l < a.local0; ++l) {
        const MgLevel &L = a.lv[l];
        const float mu = l == 0 ? mu0 : 0.f;
        xsweep(L, mu, nullptr, L.za, true, nullptr);
        if (!grid_bar(a, s)) return false;
        ysweep(L, mu, L.za, L.zb, true);
        if (!grid_bar(a, s)) return false;
        residual(L, mu, L.zb, L.t, d);
        if (!grid_bar(a, s)) return false;
        restrict_to(L, a.lv[l + 1], L.t, d);
        if (!grid_bar(a, s)) return false;
    }
    if (blockIdx.x == 0) local_vcycle(a, a.local0, mu0, a.local0 == 0 ? dot : nullptr);
    if (a.local0 > 0 && !grid_bar(a, s)) return false;
    for (int l = a.local0 - 1; l >= 0; --l) {
        const MgLevel &L = a.lv[l];
        const float mu = l == 0 ? mu0 : 0.f;
        prolong_add(L, a.lv[l + 1], a.lv[l + 1].za, L.zb, L.za, d);
        if (!grid_bar(a, s)) return false;
        ysweep(L, mu, L.za, L.zb, true);
        if (!grid_bar(a, s)) return false;
        xsweep(L, mu, L.zb, L.za, true, l == 0 ? dot : nullptr);
        if (l > 0 && !grid_bar(a, s)) return false;
    }
    return true;
}

__device__ __forceinline__ double nonneg(double v) { return v > 0.0 ? v : (v == v ? 0.0 : v); }

// (A u) in FP64 at fine cell (i, j), u = x + d
// A (x + d / sigma) at cell (i, j), FP64; unsig = 1 / sigma (d holds the
// scaled FP32 correction of the current inner solve)
__device__ __forceinline__ double apply64(const MgArgs &a, int i, int j, double unsig)
{
    const int nx = a.nx;
    const size_t k = (size_t)j * nx + i;
    auto u = [&](size_t q) { return a.x[q] + (double)a.d[q] * unsig; };
    const double c = u(k);
    double ax = 0.0, ay = 0.0;
    if (i > 0) ax += a.fx[i] * (c - u(k - 1));
    if (i + 1 < nx) ax += a.fx[i + 1] * (c - u(k + 1));
    if (j > 0) ay += a.fy[j] * (c - u(k - nx));
    if (j + 1 < a.ny) ay += a.fy[j + 1] * (c - u(k + nx));
    return a.dy[j] * ax + a.dx[i] * ay;
}

__global__ void __launch_bounds__(MG_THREADS, 1) mg_kernel(MgArgs a)
{
    Sync s{0u, 0};
    const Dist dg = grid_dist();
    const uint64_t t_start = gtimer();
    if (a.mode == 1) {
        double dummy = 0.0;
        vcycle(a, s, 0.f, &dummy);
        return;
    }
    const int nx = a.nx, n = a.nx * a.ny;
    const MgLevel &L0 = a.lv[0];
    float *r = L0.r, *z = L0.za;
    // statistics of b = -V S; zero the correction
    double st[3] = {0.0, 0.0, 0.0};
    for (int k = dg.wid; k < n; k += dg.nw) {
        const double b = -a.dx[k % nx] * a.dy[k / nx] * a.S[k];
        st[0] += b;
        st[1] += b * b;
        st[2] += fabs(b);
        a.d[k] = 0.f;
    }
    if (!grid_sum(a, s, st)) return;
    const double mub = st[0] / n;
    const double bnorm = sqrt(nonneg(st[1] - n * mub * mub));
    const double incompat = st[2] > 0.0 ? fabs(st[0]) / st[2] : 0.0;
    int status = PPE_OK, iters = 0, refinements = 0, stall = 0, stalled = 0;
    double relres = 0.0, relres_prev = 0.0;
    // the FP32 inner solve works on 2^-e r, e the binary exponent of the true
    // residual's norm (exact scaling: the FP32 vectors stay in range whatever
    // the scale of the source); d is folded back with the inverse
    double sig = 1.0;
    if (!isfinite(st[0]) || !isfinite(st[1])) {
        status = PPE_ERR_NAN;
    } else if (!(incompat <= 1e-6)) {
        status = PPE_ERR_INCOMPATIBLE_RHS;
    } else if (!(bnorm > 0.0)) {
        for (int k = dg.wid; k < n; k += dg.nw) a.x[k] = 0.0;
    } else {
        for (;;) {
            // true residual of x + d / sigma in FP64
            const double unsig = 1.0 / sig;
            double rs[2] = {0.0, 0.0};
            for (int k = dg.wid; k < n; k += dg.nw) {
                const int i = k % nx, j = k / nx;
                const double b = -a.dx[i] * a.dy[j] * a.S[k] - mub;
                const double rv = b - apply64(a, i, j, unsig);
                a.r64[k] = rv;
                rs[0] += rv;
                rs[1] += rv * rv;
            }
            if (!grid_sum(a, s, rs)) return;
            const double mu = rs[0] / n;
            const double rsq = nonneg(rs[1] - n * mu * mu);
            relres = sqrt(rsq) / bnorm;
            ++refinements;
            // fold d into x; the FP32 residual of the next inner solve
            if (rsq > 0.0 && isfinite(rsq)) {
                int e = 0;
                frexp(sqrt(rsq), &e);
                sig = ldexp(1.0, -max(-1020, min(1020, e)));
            }
            for (int k = dg.wid; k < n; k += dg.nw) {
                a.x[k] += (double)a.d[k] * unsig;
                a.d[k] = 0.f;
                r[k] = (float)((a.r64[k] - mu) * sig);
            }
            if (!grid_bar(a, s)) return;
            if (!isfinite(relres)) { status = PPE_ERR_NAN; break; }
            if (relres <= a.tol) break;
            if (iters >= a.max_iters) { status = PPE_ERR_NOT_CONVERGED; break; }
            // an FP32 inner solve that cannot halve the true residual three
            // times in a row: the system is beyond what FP32 resolves
            stall = (refinements > 1 && relres > 0.5 * relres_prev) ? stall + 1 : 0;
            relres_prev = relres;
            if (stall >= 3) { status = PPE_ERR_NOT_CONVERGED; stalled = 1; break; }
            const double target_sq = fmax((double)MG_INNER_RTOL * MG_INNER_RTOL * rsq,
                                           0.25 * a.tol * a.tol * bnorm * bnorm) * sig * sig;
            // inner MG-PCG on A d = r (FP32 vectors, FP64 scalars)
            float mur = 0.f;                   // lagged mean of the FP32 residual
            double g[1] = {0.0};
            if (!vcycle(a, s, mur, &g[0])) return;
            if (!grid_sum(a, s, g)) return;
            double gamma = g[0], beta = 0.0;
            for (int inner = 0; inner < MG_INNER_MAX; ++inner) {
                const float bf = (float)beta;
                for (int k = dg.wid; k < n; k += dg.nw) a.p[k] = beta == 0.0 ? z[k] : z[k] + bf * a.p[k];
                if (!grid_bar(a, s)) return;
                double pq[1] = {0.0};
                for (int k = dg.wid; k < n; k += dg.nw) {
                    const float qv = apply_at(L0, a.p, k % nx, k / nx);
                    a.q[k] = qv;
                    pq[0] += (double)a.p[k] * qv;
                }
                if (!grid_sum(a, s, pq)) return;
                const double alpha = gamma / pq[0];
                if (!(pq[0] > 0.0) || !isfinite(alpha)) break;     // refine from the true residual
                const float af = (float)alpha;
                double rr[2] = {0.0, 0.0};
                for (int k = dg.wid; k < n; k += dg.nw) {
                    a.d[k] += af * a.p[k];
                    const float rv = r[k] - af * a.q[k];
                    r[k] = rv;
                    rr[0] += rv;
                    rr[1] += (double)rv * rv;
                }
                if (!grid_sum(a, s, rr)) return;
                ++iters;
                const double m = rr[0] / n;
                mur = (float)m;
                if (nonneg(rr[1] - n * m * m) <= target_sq || iters >= a.max_iters) break;
                double gn[1] = {0.0};
                if (!vcycle(a, s, mur, &gn[0])) return;
                if (!grid_sum(a, s, gn)) return;
                beta = gn[0] / gamma;
                gamma = gn[0];
                if (!(gamma > 0.0)) break;
            }
        }
        // zero volume-weighted mean
        double vm[2] = {0.0, 0.0};
        for (int k = dg.wid; k < n; k += dg.nw) {
            const double v = a.dx[k % nx] * a.dy[k / nx];
            vm[0] += v * a.x[k];
            vm[1] += v;
        }
        if (!grid_sum(a, s, vm)) return;
        const double xm = vm[0] / vm[1];
        for (int k = dg.wid; k < n; k += dg.nw) a.x[k] -= xm;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.rep->status = status;
        a.rep->iters = iters;
        a.rep->refinements = refinements;
        a.rep->stalled = stalled;
        a.rep->relres = relres;
        a.rep->incompat = incompat;
        a.rep->ns = gtimer() - t_start;
    }
}

// ---------------------------------------------------------------------------
// host side: the hierarchy
// ---------------------------------------------------------------------------

std::vector<double> coarsen(const std::vector<double> &w)
{
    const size_t n = w.size();
    if (n == 1) return w;
    std::vector<double> c((n + 1) / 2);
    for (size_t k = 0; k < n / 2; ++k) c[k] = w[2 * k] + w[2 * k + 1];
    if (n % 2) c.back() = w.back();
    return c;
}

std::vector<double> faces(const std::vector<double> &w)
{
    std::vector<double> f(w.size() + 1, 0.0);
    for (size_t k = 1; k < w.size(); ++k) f[k] = 2.0 / (w[k - 1] + w[k]);
    return f;
}

// per fine cell: parent, side neighbour (-1: none), neighbour weight
void prolong_tables(const std::vector<double> &wf, const std::vector<double> &wc, std::vector<int> &par,
                    std::vector<int> &nb, std::vector<float> &w)
{
    const size_t nf = wf.size(), nc = wc.size();
    par.assign(nf, 0);
    nb.assign(nf, -1);
    w.assign(nf, 0.f);
    std::vector<double> xf(nf), xc(nc);
    double e = 0.0;
    for (size_t i = 0; i < nf; ++i) { xf[i] = e + 0.5 * wf[i]; e += wf[i]; }
    e = 0.0;
    for (size_t I = 0; I < nc; ++I) { xc[I] = e + 0.5 * wc[I]; e += wc[I]; }
    for (size_t i = 0; i < nf; ++i) {
        const int p = nf == nc ? (int)i : (int)(i / 2);
        par[i] = p;
        if (nf == nc || xf[i] == xc[p]) continue;
        const int q = xf[i] < xc[p] ? p - 1 : p + 1;
        if (q < 0 || q >= (int)nc) continue;
        nb[i] = q;
        w[i] = (float)((xf[i] - xc[p]) / (xc[q] - xc[p]));
    }
}

// Pseudo-inverse of the coarsest operator by Jacobi eigenvalue iterations on
// the small dense symmetric matrix (FP64): A = V diag(l) V^T, A^+ = V diag(1/l, l > tol) V^T.
std::vector<double> pseudo_inverse(const std::vector<double> &dx, const std::vector<double> &dy)
{
    const int nx = (int)dx.size(), ny = (int)dy.size(), n = nx * ny;
    const std::vector<double> fx = faces(dx), fy = faces(dy);
    std::vector<double> A((size_t)n * n, 0.0), V((size_t)n * n, 0.0);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const int r = j * nx + i;
            auto add = [&](int c, double v) { A[(size_t)r * n + c] += v; };
            if (i > 0) { add(r, dy[j] * fx[i]); add(r - 1, -dy[j] * fx[i]); }
            if (i + 1 < nx) { add(r, dy[j] * fx[i + 1]); add(r + 1, -dy[j] * fx[i + 1]); }
            if (j > 0) { add(r, dx[i] * fy[j]); add(r - nx, -dx[i] * fy[j]); }
            if (j + 1 < ny) { add(r, dx[i] * fy[j + 1]); add(r + nx, -dx[i] * fy[j + 1]); }
        }
    for (int k = 0; k < n; ++k) V[(size_t)k * n + k] = 1.0;
    // cyclic Jacobi rotations until the off-diagonal part is negligible
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                const double v = A[(size_t)p * n + q] * A[(size_t)p * n + q];
                tot += v;
                if (p != q) off += v;
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    double lmax = 0.0;
    for (int k = 0; k < n; ++k) lmax = std::max(lmax, std::fabs(A[(size_t)k * n + k]));
    std::vector<double> P((size_t)n * n, 0.0);
    for (int k = 0; k < n; ++k) {
        const double l = A[(size_t)k * n + k];
        if (!(l > 1e-12 * lmax)) continue;          // the constant null space
        for (int r = 0; r < n; ++r) {
            const double vr = V[(size_t)r * n + k] / l;
            for (int c = 0; c < n; ++c) P[(size_t)r * n + c] += vr * V[(size_t)c * n + k];
        }
    }
    return P;
}

}  // namespace

// The hierarchy and the kernel's buffers of one grid (built on first use).
struct MgPlan {
    int nlev = 0, local0 = 0, ncoarse = 0, blocks = 0;
    MgLevel *lv_dev = nullptr;
    void *mem = nullptr;           // every level array, one allocation
    float *pinv = nullptr;
    double *r64 = nullptr, *part = nullptr;
    float *p = nullptr, *q = nullptr, *d = nullptr;
    unsigned *bar = nullptr;
    int *err = nullptr;
    MgReport *rep = nullptr;
    std::vector<MgLevel> lv;       // host copy (device pointers)
};

void mg_plan_destroy(MgPlan *m)
{
    if (!m) return;
    cudaFree(m->lv_dev);
    cudaFree(m->mem);
    delete m;
}

static ppe_status mg_plan_create(ppe_grid *g, MgPlan **out)
{
    *out = nullptr;
    struct HostLevel {
        std::vector<double> dx, dy;
        std::vector<int> pxp, pxn, pyp, pyn;
        std::vector<float> pxw, pyw;
    };
    std::vector<HostLevel> H(1);
    H[0].dx = g->hdx;
    H[0].dy = g->hdy;
    while ((long long)H.back().dx.size() * H.back().dy.size() > MG_COARSE_CELLS &&
           (H.back().dx.size() > 1 || H.back().dy.size() > 1) && (int)H.size() < MG_MAX_LEVELS) {
        HostLevel c;
        c.dx = coarsen(H.back().dx);
        c.dy = coarsen(H.back().dy);
        prolong_tables(H.back().dx, c.dx, H.back().pxp, H.back().pxn, H.back().pxw);
        prolong_tables(H.back().dy, c.dy, H.back().pyp, H.back().pyn, H.back().pyw);
        H.push_back(std::move(c));
    }
    if ((long long)H.back().dx.size() * H.back().dy.size() > 4096) {
        set_error("multigrid: the coarsest level is too large (grid too elongated)");
        return PPE_ERR_ARG;
    }
    const int nlev = (int)H.size();
    // byte layout of one allocation
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
    struct Off { size_t dx, dy, fx, fy, pxp, pxn, pyp, pyn, pxw, pyw, r, za, zb, t, s1, s2; };
    std::vector<Off> O(nlev);
    for (int l = 0; l < nlev; ++l) {
        const size_t nx = H[l].dx.size(), ny = H[l].dy.size(), n = nx * ny;
        O[l].dx = take(4 * nx); O[l].dy = take(4 * ny); O[l].fx = take(4 * (nx + 1)); O[l].fy = take(4 * (ny + 1));
        O[l].pxp = take(4 * nx); O[l].pxn = take(4 * nx); O[l].pyp = take(4 * ny); O[l].pyn = take(4 * ny);
        O[l].pxw = take(4 * nx); O[l].pyw = take(4 * ny);
        O[l].r = take(4 * n); O[l].za = take(4 * n); O[l].zb = take(4 * n); O[l].t = take(4 * n);
        O[l].s1 = take(4 * n); O[l].s2 = take(4 * n);
    }
    const size_t nc = H.back().dx.size() * H.back().dy.size();
    const size_t n0 = g->hdx.size() * g->hdy.size();
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = std::max(1, std::min(sms, (int)((n0 + MG_THREADS - 1) / MG_THREADS)));
    const size_t o_pinv = take(4 * nc * nc), o_r64 = take(8 * n0), o_p = take(4 * n0), o_q = take(4 * n0),
                 o_d = take(4 * n0), o_part = take(8 * 2 * 4 * (size_t)std::max(blocks, sms)), o_bar = take(8),
                 o_err = take(4), o_rep = take(sizeof(MgReport));
    MgPlan *m = new MgPlan();
    auto fail = [&](cudaError_t e, const char *what) {
        mg_plan_destroy(m);
        return cuda_status(e, what);
    };
    cudaError_t e;
    if ((e = cudaMalloc(&m->mem, off)) != cudaSuccess) return fail(e, "cudaMalloc(multigrid)");
    if ((e = cudaMalloc(&m->lv_dev, sizeof(MgLevel) * nlev)) != cudaSuccess) return fail(e, "cudaMalloc(multigrid)");
    char *base = (char *)m->mem;
    std::vector<char> host(off, 0);
    auto put = [&](size_t o, const void *src, size_t bytes) { std::memcpy(host.data() + o, src, bytes); };
    m->lv.resize(nlev);
    for (int l = 0; l < nlev; ++l) {
        const HostLevel &h = H[l];
        const int nx = (int)h.dx.size(), ny = (int)h.dy.size();
        std::vector<float> dx(h.dx.begin(), h.dx.end()), dy(h.dy.begin(), h.dy.end());
        std::vector<double> fxd = faces(h.dx), fyd = faces(h.dy);
        std::vector<float> fx(fxd.begin(), fxd.end()), fy(fyd.begin(), fyd.end());
        put(O[l].dx, dx.data(), 4 * nx); put(O[l].dy, dy.data(), 4 * ny);
        put(O[l].fx, fx.data(), 4 * (nx + 1)); put(O[l].fy, fy.data(), 4 * (ny + 1));
        if (l + 1 < nlev) {
            put(O[l].pxp, h.pxp.data(), 4 * nx); put(O[l].pxn, h.pxn.data(), 4 * nx); put(O[l].pxw, h.pxw.data(), 4 * nx);
            put(O[l].pyp, h.pyp.data(), 4 * ny); put(O[l].pyn, h.pyn.data(), 4 * ny); put(O[l].pyw, h.pyw.data(), 4 * ny);
        }
        MgLevel &L = m->lv[l];
        L.nx = nx; L.ny = ny;
        L.cx = l + 1 < nlev && H[l + 1].dx.size() < h.dx.size();
        L.cy = l + 1 < nlev && H[l + 1].dy.size() < h.dy.size();
        L.dx = (const float *)(base + O[l].dx); L.dy = (const float *)(base + O[l].dy);
        L.fx = (const float *)(base + O[l].fx); L.fy = (const float *)(base + O[l].fy);
        L.pxp = (const int *)(base + O[l].pxp); L.pxn = (const int *)(base + O[l].pxn);
        L.pyp = (const int *)(base + O[l].pyp); L.pyn = (const int *)(base + O[l].pyn);
        L.pxw = (const float *)(base + O[l].pxw); L.pyw = (const float *)(base + O[l].pyw);
        L.r = (float *)(base + O[l].r); L.za = (float *)(base + O[l].za);
        L.zb = (float *)(base + O[l].zb); L.t = (float *)(base + O[l].t);
        L.s1 = (float *)(base + O[l].s1); L.s2 = (float *)(base + O[l].s2);
    }
    {
        const std::vector<double> P = pseudo_inverse(H.back().dx, H.back().dy);
        std::vector<float> Pf(P.begin(), P.end());
        put(o_pinv, Pf.data(), 4 * nc * nc);
    }
    if ((e = cudaMemcpy(m->mem, host.data(), off, cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e, "cudaMemcpy(multigrid)");
    if ((e = cudaMemcpy(m->lv_dev, m->lv.data(), sizeof(MgLevel) * nlev, cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e, "cudaMemcpy(multigrid)");
    m->nlev = nlev;
    m->local0 = nlev - 1;
    for (int l = 0; l < nlev; ++l)
        if ((long long)H[l].dx.size() * H[l].dy.size() <= MG_LOCAL_CELLS) {
            m->local0 = l;
            break;
        }
    m->ncoarse = (int)nc;
    m->blocks = blocks;
    m->pinv = (float *)(base + o_pinv);
    m->r64 = (double *)(base + o_r64);
    m->p = (float *)(base + o_p);
    m->q = (float *)(base + o_q);
    m->d = (float *)(base + o_d);
    m->part = (double *)(base + o_part);
    m->bar = (unsigned *)(base + o_bar);
    m->err = (int *)(base + o_err);
    m->rep = (MgReport *)(base + o_rep);
    *out = m;
    return PPE_OK;
}

static ppe_status mg_launch(ppe_grid *g, MgPlan *m, const double *rhs, double *x, double tol, int mode,
                            cudaStream_t stream)
{
    MgArgs a;
    std::memset(&a, 0, sizeof a);
    a.lv = m->lv_dev; a.nlev = m->nlev; a.local0 = m->local0; a.pinv = m->pinv;
    a.nx = g->nx; a.ny = g->ny; a.dx = g->dx; a.dy = g->dy; a.fx = g->fx; a.fy = g->fy;
    a.S = rhs; a.x = x; a.r64 = m->r64; a.p = m->p; a.q = m->q; a.d = m->d;
    a.tol = tol; a.max_iters = g->opts.max_iters; a.mode = mode;
    a.part = m->part; a.bar = m->bar; a.err = m->err;
    a.spin_ns = (long long)(g->opts.spin_limit_ms > 0 ? g->opts.spin_limit_ms : 2000) * 1000000LL;
    a.rep = m->rep;
    PPE_CUDA_TRY(cudaMemsetAsync(m->bar, 0, 8, stream));
    PPE_CUDA_TRY(cudaMemsetAsync(m->err, 0, 4, stream));
    PPE_CUDA_TRY(cudaMemsetAsync(m->rep, 0, sizeof(MgReport), stream));
    void *params[] = {&a};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)mg_kernel, dim3(m->blocks), dim3(MG_THREADS), params, 0,
                                                stream);
    if (e != cudaSuccess) return cuda_status(e, "cudaLaunchCooperativeKernel(multigrid)");
    return PPE_OK;
}

static ppe_status mg_plan_of(ppe_grid *g, MgPlan **m)
{
    if (!g->mg) PPE_TRY(mg_plan_create(g, &g->mg));
    *m = g->mg;
    return PPE_OK;
}

// Solve with the multigrid partner (mixed precision: FP32 inner MG-PCG, FP64
// refinement); the report as ppe_solve's.
ppe_status mg_solve(ppe_grid *g, const double *rhs, double *x, double tol, cudaStream_t stream, ppe_solve_info *info)
{
    MgPlan *m = nullptr;
    PPE_TRY(mg_plan_of(g, &m));
    cudaEvent_t e0 = g->ls->ev0, e1 = g->ls->ev1;
    PPE_CUDA_TRY(cudaEventRecord(e0, stream));
    PPE_TRY(mg_launch(g, m, rhs, x, tol, 0, stream));
    PPE_CUDA_TRY(cudaEventRecord(e1, stream));
    MgReport rep;
    int err = 0;
    PPE_CUDA_TRY(cudaMemcpyAsync(&rep, m->rep, sizeof rep, cudaMemcpyDeviceToHost, stream));
    PPE_CUDA_TRY(cudaMemcpyAsync(&err, m->err, sizeof err, cudaMemcpyDeviceToHost, stream));
    PPE_CUDA_TRY(cudaStreamSynchronize(stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (err) {
        set_error("multigrid kernel: bounded grid-barrier wait expired");
        return (ppe_status)err;
    }
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->status = rep.status;
        info->iters_pcg = rep.iters;
        info->refinements = rep.refinements;
        info->launches = 1;
        info->rel_res_true = rep.relres;
        info->incompat = rep.incompat;
        info->ms_total = ms;
        info->ms_pcg = (double)rep.ns * 1e-6;
        info->precision_fallback = rep.stalled;
    }
    if (rep.status != PPE_OK) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "multigrid solve finished with status %d (relres %.3e)", rep.status,
                      rep.relres);
        set_error(buf);
    }
    return (ppe_status)rep.status;
}

}  // namespace ppe

using namespace ppe;

extern "C" ppe_status ppe_debug_mg_vcycle(ppe_grid *g, const float *r_dev, float *z_dev, void *stream)
{
    clear_error();
    if (!g || !r_dev || !z_dev) {
        set_error("ppe_debug_mg_vcycle: NULL argument");
        return PPE_ERR_ARG;
    }
    MgPlan *m = nullptr;
    PPE_TRY(mg_plan_of(g, &m));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)g->nx * g->ny * sizeof(float);
    PPE_CUDA_TRY(cudaMemcpyAsync(m->lv[0].r, r_dev, bytes, cudaMemcpyDeviceToDevice, st));
    PPE_TRY(mg_launch(g, m, nullptr, nullptr, 1.0, 1, st));
    PPE_CUDA_TRY(cudaMemcpyAsync(z_dev, m->lv[0].za, bytes, cudaMemcpyDeviceToDevice, st));
    int err = 0;
    PPE_CUDA_TRY(cudaMemcpyAsync(&err, m->err, sizeof err, cudaMemcpyDeviceToHost, st));
    PPE_CUDA_TRY(cudaStreamSynchronize(st));
    if (err) {
        set_error("multigrid kernel: bounded grid-barrier wait expired");
        return (ppe_status)err;
    }
    return PPE_OK;
}
