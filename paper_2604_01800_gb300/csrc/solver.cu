// Persistent solver kernel: iterative refinement (FP64) around a
// single-reduction Jacobi PCG (FP32 or FP64) with interleaved DLSM steps.
//
// One cooperative launch runs the whole per-system state machine of every
// system in a batch; grid-wide barriers separate the passes.  A pass sweeps
// the tiles of every system once; each tile writes FP64 partial sums, and the
// last block to reach the barrier reduces them (fixed order, so results are
// reproducible) and advances each system's state.  The kernel returns when
// every live system is done or waits for a network direction.
//
// Operator (Sec. 2.1 Eq. 6, volume-scaled): for cell (i,j)
//   (A u)_ij = dy_j [fe_i (u_ij - u_E) + fw_i (u_ij - u_W)]
//            + dx_i [fn_j (u_ij - u_N) + fs_j (u_ij - u_S)]
// with face coefficients f = 2 / (width_left + width_right) and 0 at walls.
//
// PCG variant: Chronopoulos-Gear single-reduction CG with Jacobi
// preconditioning.  Per iteration, with u = D^-1 r and w = A u:
//   p = u + beta p,  s = w + beta s  (s = A p),  x += alpha p,  r -= alpha s,
//   gamma' = r.u, delta' = (A u).u, beta' = gamma'/gamma,
//   alpha' = gamma' / (delta' - beta' gamma' / alpha).
// Each block recomputes the new residual on a one-cell halo of its tile
// (reading r two cells out) so that A u' is available in the same pass: one
// grid barrier per iteration.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "internal.h"

namespace ppe {

namespace {

constexpr int WX = TILE_X + 4;     // tile window with a two-cell halo
constexpr int WY = TILE_Y + 4;
constexpr int WN = WX * WY;

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename T> __device__ __forceinline__ T ld_cg(const T *p) { return __ldcg(p); }

template <typename T> __device__ __forceinline__ T recip(T v);
template <> __device__ __forceinline__ float recip<float>(float v) { return v > 0.f ? __frcp_rn(v) : 0.f; }
template <> __device__ __forceinline__ double recip<double>(double v) { return v > 0.0 ? 1.0 / v : 0.0; }

// Coefficients of the tile window, in the arithmetic type C.
template <typename C> struct Coef {
    C dx[WX], fw[WX], fe[WX], sx[WX];
    C dy[WY], fs[WY], fn[WY], sy[WY];
};

template <typename C> struct Work {
    C a0[WN], a1[WN], a2[WN], a3[WN], a4[WN], a5[WN];
};

template <typename T> struct SmemT {
    Coef<double> cfd;
    Coef<float> cff;
    Work<T> w;
    double red[NPART][TILE_Y];
    SysDesc sd;
    SysState st;
    int32_t last;
    uint32_t gen;
    int32_t go;
};

template <typename C>
__device__ void load_coef(Coef<C> &cf, const SysDesc &sd, int i0, int j0, const C *DX, const C *FX,
                          const C *DY, const C *FY)
{
    for (int k = threadIdx.x; k < WX; k += blockDim.x) {
        int i = i0 - 2 + k;
        bool in = i >= 0 && i < sd.nx;
        C w = in ? DX[i] : C(0), a = in ? FX[i] : C(0), b = in ? FX[i + 1] : C(0);
        cf.dx[k] = w; cf.fw[k] = a; cf.fe[k] = b; cf.sx[k] = a + b;
    }
    for (int k = threadIdx.x; k < WY; k += blockDim.x) {
        int j = j0 - 2 + k;
        bool in = j >= 0 && j < sd.ny;
        C w = in ? DY[j] : C(0), a = in ? FY[j] : C(0), b = in ? FY[j + 1] : C(0);
        cf.dy[k] = w; cf.fs[k] = a; cf.fn[k] = b; cf.sy[k] = a + b;
    }
}

template <typename T, typename S> __device__ __forceinline__ Coef<T> &coef_of(S &sm);
template <> __device__ __forceinline__ Coef<float> &coef_of<float, SmemT<float>>(SmemT<float> &sm) { return sm.cff; }
template <> __device__ __forceinline__ Coef<double> &coef_of<double, SmemT<double>>(SmemT<double> &sm) { return sm.cfd; }

template <typename T, typename S> __device__ __forceinline__ void load_coef_t(S &sm, const SysDesc &sd, int i0, int j0)
{
    if constexpr (sizeof(T) == 4)
        load_coef<float>(sm.cff, sd, i0, j0, sd.dx32, sd.fx32, sd.dy32, sd.fy32);
    else
        load_coef<double>(sm.cfd, sd, i0, j0, sd.dx, sd.fx, sd.dy, sd.fy);
}

template <typename C> __device__ __forceinline__ C dinv_at(const Coef<C> &cf, int wi, int wj)
{
    return recip<C>(cf.dy[wj] * cf.sx[wi] + cf.dx[wi] * cf.sy[wj]);
}

// (A U) at window point (wi, wj); U holds the window, zero outside the domain.
template <typename C> __device__ __forceinline__ C stencil(const Coef<C> &cf, const C *U, int wi, int wj)
{
    int k = wj * WX + wi;
    C c = U[k];
    C ax = cf.fe[wi] * (c - U[k + 1]) + cf.fw[wi] * (c - U[k - 1]);
    C ay = cf.fn[wj] * (c - U[k + WX]) + cf.fs[wj] * (c - U[k - WX]);
    return cf.dy[wj] * ax + cf.dx[wi] * ay;
}

__device__ __forceinline__ bool in_dom(const SysDesc &sd, int i, int j)
{
    return i >= 0 && j >= 0 && i < sd.nx && j < sd.ny;
}

// Block reduction of NPART values; thread k < NPART writes the tile partial.
template <typename T, typename S>
__device__ void block_partials(S &sm, T (&acc)[NPART], double *out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NPART; ++q) {
        T v = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sm.red[q][warp] = (double)v;
    }
    __syncthreads();
    if (threadIdx.x < NPART) {
        double s = 0.0;
        for (int w = 0; w < TILE_Y; ++w) s += sm.red[threadIdx.x][w];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// passes (one tile each)
// ---------------------------------------------------------------------------

// b statistics: b = -V S
template <typename T, typename S> __device__ void pass_init(S &sm, int i0, int j0, double *out)
{
    const SysDesc &sd = sm.sd;
    double acc[NPART] = {0, 0, 0, 0, 0, 0};
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    int j = j0 + ty;
    for (int c = 0; c < 4; ++c) {
        int i = i0 + tx + 32 * c;
        if (i < sd.nx && j < sd.ny) {
            double b = -sd.dx[i] * sd.dy[j] * sd.f[(size_t)j * sd.nx + i];
            acc[0] += b; acc[1] += b * b; acc[2] += fabs(b);
        }
    }
    block_partials(sm, acc, out);
}

// FP64 true residual r = (b - mu_b) - A (x + d); stores r into the inner buffer.
template <typename T, typename S> __device__ void pass_res(S &sm, int i0, int j0, double *out)
{
    const SysDesc &sd = sm.sd;
    const SysState &st = sm.st;
    Coef<double> &cf = sm.cfd;
    double *X = reinterpret_cast<double *>(&sm.w);
    load_coef<double>(cf, sd, i0, j0, sd.dx, sd.fx, sd.dy, sd.fy);
    const T *d = (const T *)sd.d;
    for (int k = threadIdx.x; k < WN; k += blockDim.x) {
        int wi = k % WX, wj = k / WX, i = i0 - 2 + wi, j = j0 - 2 + wj;
        double v = 0.0;
        if (wi >= 1 && wi < WX - 1 && wj >= 1 && wj < WY - 1 && in_dom(sd, i, j)) {
            v = ld_cg(sd.x + (size_t)j * sd.nx + i);
            if (st.has_d) v += (double)ld_cg(d + (size_t)j * sd.pitch + i);
        }
        X[k] = v;
    }
    __syncthreads();
    double acc[NPART] = {0, 0, 0, 0, 0, 0};
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    int j = j0 + ty, wj = ty + 2;
    T *r = (T *)sd.r[st.cur];
    for (int c = 0; c < 4; ++c) {
        int i = i0 + tx + 32 * c, wi = tx + 32 * c + 2;
        if (i < sd.nx && j < sd.ny) {
            double b = -sd.dx[i] * sd.dy[j] * ld_cg(sd.f + (size_t)j * sd.nx + i) - st.mu_b;
            double rv = b - stencil<double>(cf, X, wi, wj);
            r[(size_t)j * sd.pitch + i] = (T)rv;
            acc[0] += rv; acc[1] += rv * rv;
        }
    }
    block_partials(sm, acc, out);
}

// Start of a CG-type phase: u = D^-1 (r - mu), w = A u; dots r.u, w.u, r.r, sum r.
template <typename T, typename S> __device__ void pass_restart(S &sm, int i0, int j0, double *out)
{
    const SysDesc &sd = sm.sd;
    const SysState &st = sm.st;
    Coef<T> &cf = coef_of<T>(sm);
    T *R = sm.w.a0, *U = sm.w.a1;
    load_coef_t<T>(sm, sd, i0, j0);
    __syncthreads();
    const T *rin = (const T *)sd.r[st.cur];
    const T mu = (T)st.mu;
    for (int k = threadIdx.x; k < WN; k += blockDim.x) {
        int wi = k % WX, wj = k / WX, i = i0 - 2 + wi, j = j0 - 2 + wj;
        T rv = 0;
        if (wi >= 1 && wi < WX - 1 && wj >= 1 && wj < WY - 1 && in_dom(sd, i, j))
            rv = ld_cg(rin + (size_t)j * sd.pitch + i) - mu;
        R[k] = rv;
        U[k] = rv * dinv_at<T>(cf, wi, wj);
    }
    __syncthreads();
    T acc[NPART] = {0, 0, 0, 0, 0, 0};
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    int j = j0 + ty, wj = ty + 2;
    T *dd = (T *)sd.d;
    for (int c = 0; c < 4; ++c) {
        int i = i0 + tx + 32 * c, wi = tx + 32 * c + 2;
        if (i < sd.nx && j < sd.ny) {
            int k = wj * WX + wi;
            T w = stencil<T>(cf, U, wi, wj);
            acc[0] += R[k] * U[k]; acc[1] += w * U[k]; acc[2] += R[k] * R[k]; acc[3] += R[k];
            if (st.reset_d) {
                size_t gi = (size_t)j * sd.pitch + i;
                if (st.fold_d) sd.x[(size_t)j * sd.nx + i] += (double)ld_cg(dd + gi);
                dd[gi] = T(0);
            }
        }
    }
    block_partials(sm, acc, out);
}

// One single-reduction PCG iteration.
template <typename T, typename S> __device__ void pass_iter(S &sm, int i0, int j0, double *out)
{
    const SysDesc &sd = sm.sd;
    const SysState &st = sm.st;
    Coef<T> &cf = coef_of<T>(sm);
    T *R = sm.w.a0, *U = sm.w.a1, *Sv = sm.w.a2, *Rn = sm.w.a3, *Un = sm.w.a4, *Sn = sm.w.a5;
    load_coef_t<T>(sm, sd, i0, j0);
    __syncthreads();
    const int cur = st.cur;
    const T *rin = (const T *)sd.r[cur];
    const T *sin = (const T *)sd.s[cur];
    T *rout = (T *)sd.r[cur ^ 1];
    T *sout = (T *)sd.s[cur ^ 1];
    T *pv = (T *)sd.p;
    T *dv = (T *)sd.d;
    const T mu = (T)st.mu, alpha = (T)st.alpha, beta = (T)st.beta;
    const bool first = st.first != 0;
    for (int k = threadIdx.x; k < WN; k += blockDim.x) {
        int wi = k % WX, wj = k / WX, i = i0 - 2 + wi, j = j0 - 2 + wj;
        T rv = 0, sv = 0;
        if (in_dom(sd, i, j)) {
            size_t gi = (size_t)j * sd.pitch + i;
            rv = ld_cg(rin + gi) - mu;
            if (!first && wi >= 1 && wi < WX - 1 && wj >= 1 && wj < WY - 1) sv = ld_cg(sin + gi);
        }
        R[k] = rv;
        U[k] = rv * dinv_at<T>(cf, wi, wj);
        Sv[k] = sv;
    }
    __syncthreads();
    // new residual on the tile and its one-cell ring
    for (int k = threadIdx.x; k < WN; k += blockDim.x) {
        int wi = k % WX, wj = k / WX, i = i0 - 2 + wi, j = j0 - 2 + wj;
        T rn = 0, un = 0, sn = 0;
        if (wi >= 1 && wi < WX - 1 && wj >= 1 && wj < WY - 1 && in_dom(sd, i, j)) {
            T w = stencil<T>(cf, U, wi, wj);
            sn = w + beta * Sv[k];
            rn = R[k] - alpha * sn;
            un = rn * dinv_at<T>(cf, wi, wj);
        }
        Rn[k] = rn; Un[k] = un; Sn[k] = sn;
    }
    __syncthreads();
    T acc[NPART] = {0, 0, 0, 0, 0, 0};
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    int j = j0 + ty, wj = ty + 2;
    for (int c = 0; c < 4; ++c) {
        int i = i0 + tx + 32 * c, wi = tx + 32 * c + 2;
        if (i < sd.nx && j < sd.ny) {
            int k = wj * WX + wi;
            size_t gi = (size_t)j * sd.pitch + i;
            T pold = first ? T(0) : ld_cg(pv + gi);
            T pn = U[k] + beta * pold;
            pv[gi] = pn;
            dv[gi] = ld_cg(dv + gi) + alpha * pn;
            sout[gi] = Sn[k];
            T rn = Rn[k], un = Un[k];
            rout[gi] = rn;
            T wn = stencil<T>(cf, Un, wi, wj);
            acc[0] += rn * un; acc[1] += wn * un; acc[2] += rn * rn; acc[3] += rn;
        }
    }
    block_partials(sm, acc, out);
}

// DLSM dots: r.e, e.(A e), e.e  (Eq. 11)
template <typename T, typename S> __device__ void pass_dlsm_dot(S &sm, int i0, int j0, double *out)
{
    const SysDesc &sd = sm.sd;
    const SysState &st = sm.st;
    Coef<float> &cf = sm.cff;
    float *E = reinterpret_cast<float *>(&sm.w);
    load_coef<float>(cf, sd, i0, j0, sd.dx32, sd.fx32, sd.dy32, sd.fy32);
    for (int k = threadIdx.x; k < WN; k += blockDim.x) {
        int wi = k % WX, wj = k / WX, i = i0 - 2 + wi, j = j0 - 2 + wj;
        float v = 0.f;
        if (wi >= 1 && wi < WX - 1 && wj >= 1 && wj < WY - 1 && in_dom(sd, i, j))
            v = ld_cg(sd.e + (size_t)j * sd.pitch + i);
        E[k] = v;
    }
    __syncthreads();
    const T *rin = (const T *)sd.r[st.cur];
    const T mu = (T)st.mu;
    float acc[NPART] = {0, 0, 0, 0, 0, 0};
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    int j = j0 + ty, wj = ty + 2;
    for (int c = 0; c < 4; ++c) {
        int i = i0 + tx + 32 * c, wi = tx + 32 * c + 2;
        if (i < sd.nx && j < sd.ny) {
            int k = wj * WX + wi;
            float ev = E[k];
            float rv = (float)(ld_cg(rin + (size_t)j * sd.pitch + i) - mu);
            float q = stencil<float>(cf, E, wi, wj);
            acc[0] += rv * ev; acc[1] += ev * q; acc[2] += ev * ev;
        }
    }
    block_partials(sm, acc, out);
}

// DLSM update: d += alpha e, r_new = (r - mu) - alpha A e  (Eq. 12)
template <typename T, typename S> __device__ void pass_dlsm_upd(S &sm, int i0, int j0, double *out)
{
    const SysDesc &sd = sm.sd;
    const SysState &st = sm.st;
    Coef<float> &cf = sm.cff;
    float *E = reinterpret_cast<float *>(&sm.w);
    load_coef<float>(cf, sd, i0, j0, sd.dx32, sd.fx32, sd.dy32, sd.fy32);
    for (int k = threadIdx.x; k < WN; k += blockDim.x) {
        int wi = k % WX, wj = k / WX, i = i0 - 2 + wi, j = j0 - 2 + wj;
        float v = 0.f;
        if (wi >= 1 && wi < WX - 1 && wj >= 1 && wj < WY - 1 && in_dom(sd, i, j))
            v = ld_cg(sd.e + (size_t)j * sd.pitch + i);
        E[k] = v;
    }
    __syncthreads();
    const int cur = st.cur;
    const T *rin = (const T *)sd.r[cur];
    T *rout = (T *)sd.r[cur ^ 1];
    T *dv = (T *)sd.d;
    const T mu = (T)st.mu, alpha = (T)st.alpha_d;
    T acc[NPART] = {0, 0, 0, 0, 0, 0};
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    int j = j0 + ty, wj = ty + 2;
    for (int c = 0; c < 4; ++c) {
        int i = i0 + tx + 32 * c, wi = tx + 32 * c + 2;
        if (i < sd.nx && j < sd.ny) {
            int k = wj * WX + wi;
            size_t gi = (size_t)j * sd.pitch + i;
            T q = (T)stencil<float>(cf, E, wi, wj);
            T rn = (ld_cg(rin + gi) - mu) - alpha * q;
            rout[gi] = rn;
            dv[gi] = ld_cg(dv + gi) + alpha * (T)E[k];
            acc[2] += rn * rn; acc[3] += rn;
        }
    }
    block_partials(sm, acc, out);
}

// Fold d into x (if pending) and accumulate sum V, sum V x.
template <typename T, typename S> __device__ void pass_final1(S &sm, int i0, int j0, double *out)
{
    const SysDesc &sd = sm.sd;
    const SysState &st = sm.st;
    const T *dd = (const T *)sd.d;
    double acc[NPART] = {0, 0, 0, 0, 0, 0};
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    int j = j0 + ty;
    for (int c = 0; c < 4; ++c) {
        int i = i0 + tx + 32 * c;
        if (i < sd.nx && j < sd.ny) {
            size_t gx = (size_t)j * sd.nx + i;
            double x = st.zero_x ? 0.0 : ld_cg(sd.x + gx);
            if (st.fold_d && !st.zero_x) x += (double)ld_cg(dd + (size_t)j * sd.pitch + i);
            sd.x[gx] = x;
            double v = sd.dx[i] * sd.dy[j];
            acc[0] += v; acc[1] += v * x;
        }
    }
    block_partials(sm, acc, out);
}

template <typename T, typename S> __device__ void pass_final2(S &sm, int i0, int j0, double *out)
{
    const SysDesc &sd = sm.sd;
    const SysState &st = sm.st;
    double acc[NPART] = {0, 0, 0, 0, 0, 0};
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    int j = j0 + ty;
    for (int c = 0; c < 4; ++c) {
        int i = i0 + tx + 32 * c;
        if (i < sd.nx && j < sd.ny) {
            size_t gx = (size_t)j * sd.nx + i;
            sd.x[gx] = ld_cg(sd.x + gx) - st.xmean;
        }
    }
    block_partials(sm, acc, out);
}

// ---------------------------------------------------------------------------
// finisher: reduce the partials of every system and advance its state
// ---------------------------------------------------------------------------

template <typename S>
__device__ void reduce_system(S &sm, const double *partials, int tile0, int ntiles, double (&tot)[NPART])
{
    double acc[NPART] = {0, 0, 0, 0, 0, 0};
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        const double *p = partials + (size_t)(tile0 + t) * NPART;
#pragma unroll
        for (int q = 0; q < NPART; ++q) acc[q] += ld_cg(p + q);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NPART; ++q) {
        double v = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sm.red[q][warp] = v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NPART; ++q) {
        double s = 0.0;
        for (int w = 0; w < TILE_Y; ++w) s += sm.red[q][w];
        tot[q] = s;
    }
    __syncthreads();
}

__device__ void enter_inner_converged(SysState &s)
{
    s.has_d = 1;
    s.phase = PH_RES;
}

// State transition of one system after a pass (runs on one thread).
__device__ void advance(const SysDesc &sd, SysState &s, const double (&t)[NPART], bool resume_net)
{
    const double N = sd.n_cells;
    int ph = s.phase;
    if (ph == PH_NET && resume_net) ph = PH_DLSM_DOT;
    switch (ph) {
    case PH_INIT: {
        s.mu_b = t[0] / N;
        double bb = t[1] - N * s.mu_b * s.mu_b;
        s.bnorm = sqrt(bb > 0.0 ? bb : 0.0);
        s.incompat = t[2] > 0.0 ? fabs(t[0]) / t[2] : 0.0;
        s.cur = 0;
        if (!(s.incompat <= 1e-6)) {
            s.status = PPE_ERR_INCOMPATIBLE_RHS;
            s.phase = PH_DONE;
        } else if (!(s.bnorm > 0.0)) {
            s.zero_x = 1;
            s.relres = 0.0;
            s.phase = PH_FINAL1;
        } else {
            s.has_d = 0;
            s.phase = PH_RES;
        }
        break;
    }
    case PH_RES: {
        s.refinements++;
        s.mu = t[0] / N;
        double rr = t[1] - N * s.mu * s.mu;
        s.rnorm = sqrt(rr > 0.0 ? rr : 0.0);
        s.relres = s.rnorm / s.bnorm;
        s.fold_d = s.has_d;
        if (!isfinite(s.relres)) {
            s.status = PPE_ERR_NAN;
            s.fold_d = 0;
            s.phase = PH_FINAL1;
        } else if (s.relres <= sd.tol) {
            s.phase = PH_FINAL1;
        } else if (s.it_total >= sd.max_iters + (sd.mode == PPE_MODE_HYBRID ? sd.hybrid_budget : 0) ||
                   s.refinements > 200) {
            s.status = PPE_ERR_NOT_CONVERGED;
            s.phase = PH_FINAL1;
        } else {
            double tau = sd.inner_rtol * s.rnorm;
            double floor_ = 0.5 * sd.tol * s.bnorm;
            s.tau = tau > floor_ ? tau : floor_;
            s.reset_d = 1;
            s.cg_count = 0;
            s.phase = PH_RESTART;
        }
        break;
    }
    case PH_RESTART: {
        s.mu = t[3] / N;
        double rr = t[2] - N * s.mu * s.mu;
        s.rho = rr > 0.0 ? rr : 0.0;
        s.reset_d = 0;
        s.fold_d = 0;
        s.has_d = 1;
        if (sqrt(s.rho) <= s.tau || !(t[1] > 0.0) || !isfinite(t[0] / t[1])) {
            enter_inner_converged(s);
            break;
        }
        s.gamma = t[0];
        s.alpha = t[0] / t[1];
        s.beta = 0.0;
        s.first = 1;
        s.cg_count = 0;
        s.phase = PH_ITER;
        break;
    }
    case PH_ITER: {
        s.it_pcg++;
        s.it_total++;
        s.cur ^= 1;
        s.mu = t[3] / N;
        double rr = t[2] - N * s.mu * s.mu;
        s.rho = rr > 0.0 ? rr : 0.0;
        s.first = 0;
        s.cg_count++;
        if (sd.mode == PPE_MODE_HYBRID && !s.fell_back && s.it_total >= sd.hybrid_budget) s.fell_back = 1;
        if (sqrt(s.rho) <= s.tau || s.it_total >= sd.max_iters + (sd.mode == PPE_MODE_HYBRID ? sd.hybrid_budget : 0)) {
            enter_inner_converged(s);
            break;
        }
        double gnew = t[0];
        double beta = gnew / s.gamma;
        double denom = t[1] - beta * gnew / s.alpha;
        if (!(denom > 0.0) || !isfinite(beta)) {       // breakdown: restart from the true residual
            enter_inner_converged(s);
            break;
        }
        s.beta = beta;
        s.alpha = gnew / denom;
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
        double a = re / eq;
        if (!(eq > sd.dlsm_guard * ee * sd.diag_max) || !isfinite(a)) {
            s.dlsm_skipped++;
            s.phase = PH_RESTART;          // back to the CG-type method
            s.reset_d = 0;
        } else {
            s.alpha_d = a;
            s.phase = PH_DLSM_UPD;
        }
        break;
    }
    case PH_DLSM_UPD: {
        s.it_dlsm++;
        s.it_total++;
        s.cur ^= 1;
        s.mu = t[3] / N;
        double rr = t[2] - N * s.mu * s.mu;
        s.rho = rr > 0.0 ? rr : 0.0;
        s.dlsm_count++;
        if (sd.mode == PPE_MODE_HYBRID && !s.fell_back && s.it_total >= sd.hybrid_budget) s.fell_back = 1;
        if (sqrt(s.rho) <= s.tau) {
            enter_inner_converged(s);
        } else if (s.dlsm_count < sd.num_dlsm && !s.fell_back) {
            s.phase = PH_NET;
        } else {
            s.reset_d = 0;
            s.phase = PH_RESTART;
        }
        break;
    }
    case PH_FINAL1: {
        s.xmean = t[1] / t[0];
        s.phase = PH_FINAL2;
        break;
    }
    case PH_FINAL2:
        s.phase = PH_DONE;
        break;
    default:
        break;
    }
}

template <typename S> __device__ void copy_state_in(S &sm, const SolverArgs &a, int s)
{
    // state written by the finisher of the previous step: read through L2
    const int32_t *src = reinterpret_cast<const int32_t *>(a.st + s);
    int32_t *dst = reinterpret_cast<int32_t *>(&sm.st);
    for (int k = threadIdx.x; k < (int)(sizeof(SysState) / 4); k += blockDim.x) dst[k] = ld_cg(src + k);
    const int32_t *dsrc = reinterpret_cast<const int32_t *>(a.sys + s);
    int32_t *ddst = reinterpret_cast<int32_t *>(&sm.sd);
    for (int k = threadIdx.x; k < (int)(sizeof(SysDesc) / 4); k += blockDim.x) ddst[k] = dsrc[k];
}

template <typename T, typename S>
__device__ void finisher(S &sm, const SolverArgs &a, bool resume_net)
{
    bool any_active = false, any_net = false;
    for (int s = 0; s < a.nsys; ++s) {
        __syncthreads();
        copy_state_in(sm, a, s);
        __syncthreads();
        int ph = sm.st.phase;
        if (ph == PH_DONE || (ph == PH_NET && !resume_net)) {
            if (ph == PH_NET) any_net = true;
            continue;
        }
        double tot[NPART];
        reduce_system(sm, a.partials, sm.sd.tile0, sm.sd.ntiles, tot);
        if (threadIdx.x == 0) {
            SysState st = sm.st;
            advance(sm.sd, st, tot, resume_net);
            int32_t *dst = reinterpret_cast<int32_t *>(a.st + s);
            const int32_t *src = reinterpret_cast<const int32_t *>(&st);
            for (int k = 0; k < (int)(sizeof(SysState) / 4); ++k) dst[k] = src[k];
            sm.st = st;
        }
        __syncthreads();
        int nph = sm.st.phase;
        if (nph == PH_NET) any_net = true;
        else if (nph != PH_DONE) any_active = true;
    }
    if (threadIdx.x == 0) {
        a.ctl->exit_kernel = any_active ? 0 : 1;
        a.ctl->any_net = any_net ? 1 : 0;
    }
}

// Grid-wide barrier; the last block to arrive runs the finisher.  Waits are
// bounded: on expiry the block records PPE_ERR_TIMEOUT and the kernel ends.
template <typename T, typename S>
__device__ bool barrier_and_finish(S &sm, const SolverArgs &a, bool resume_net)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t gen = ld_acquire_u32(&a.ctl->bar_gen);
        __threadfence();
        uint32_t prev = atomicAdd(&a.ctl->bar_count, 1u);
        sm.last = (prev == gridDim.x - 1) ? 1 : 0;
        sm.gen = gen;
    }
    __syncthreads();
    if (sm.last) {
        __threadfence();
        finisher<T>(sm, a, resume_net);
        __syncthreads();
        if (threadIdx.x == 0) {
            a.ctl->bar_count = 0;
            __threadfence();
            st_release_u32(&a.ctl->bar_gen, sm.gen + 1);
        }
    } else if (threadIdx.x == 0) {
        uint64_t t0 = globaltimer_ns();
        while (ld_acquire_u32(&a.ctl->bar_gen) == sm.gen) {
            if ((int64_t)(globaltimer_ns() - t0) > a.spin_limit_ns) {
                atomicExch(&a.ctl->err, (int32_t)PPE_ERR_TIMEOUT);
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t err = ld_cg(&a.ctl->err);
        int32_t ex = ld_cg(&a.ctl->exit_kernel);
        sm.go = (err == 0 && ex == 0) ? 1 : 0;
    }
    __syncthreads();
    return sm.go != 0;
}

template <typename T>
__global__ void __launch_bounds__(SOLVER_THREADS, 1) solver_kernel(SolverArgs a, int resume_net)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemT<T> &sm = *reinterpret_cast<SmemT<T> *>(smem_raw);
    bool resume = resume_net != 0;
    for (int step = 0;; ++step) {
        for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
            int s = a.tile_sys[t];
            __syncthreads();
            copy_state_in(sm, a, s);
            __syncthreads();
            int ph = sm.st.phase;
            if (ph == PH_NET && resume) ph = PH_DLSM_DOT;
            int lt = t - sm.sd.tile0;
            int i0 = (lt % sm.sd.tiles_x) * TILE_X, j0 = (lt / sm.sd.tiles_x) * TILE_Y;
            double *out = a.partials + (size_t)t * NPART;
            switch (ph) {
            case PH_INIT: pass_init<T>(sm, i0, j0, out); break;
            case PH_RES: pass_res<T>(sm, i0, j0, out); break;
            case PH_RESTART: pass_restart<T>(sm, i0, j0, out); break;
            case PH_ITER: pass_iter<T>(sm, i0, j0, out); break;
            case PH_DLSM_DOT: pass_dlsm_dot<T>(sm, i0, j0, out); break;
            case PH_DLSM_UPD: pass_dlsm_upd<T>(sm, i0, j0, out); break;
            case PH_FINAL1: pass_final1<T>(sm, i0, j0, out); break;
            case PH_FINAL2: pass_final2<T>(sm, i0, j0, out); break;
            default: break;
            }
        }
        if (!barrier_and_finish<T>(sm, a, resume)) break;
        resume = false;
    }
}

}  // namespace

int solver_max_blocks(bool fp64, int blocks_per_sm_req)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    size_t smem = fp64 ? sizeof(SmemT<double>) : sizeof(SmemT<float>);
    if (fp64) {
        cudaFuncSetAttribute(solver_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solver_kernel<double>, SOLVER_THREADS, smem);
    } else {
        cudaFuncSetAttribute(solver_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solver_kernel<float>, SOLVER_THREADS, smem);
    }
    if (blocks_per_sm_req > 0 && blocks_per_sm_req < per_sm) per_sm = blocks_per_sm_req;
    return per_sm * sms;
}

ppe_status launch_solver_resume(const SolverArgs &a, bool fp64, int grid_blocks, cudaStream_t stream, int resume)
{
    size_t smem = fp64 ? sizeof(SmemT<double>) : sizeof(SmemT<float>);
    SolverArgs args = a;
    int res = resume;
    void *params[] = {&args, &res};
    cudaError_t e;
    if (fp64) {
        cudaFuncSetAttribute(solver_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        e = cudaLaunchCooperativeKernel((const void *)solver_kernel<double>, dim3(grid_blocks),
                                        dim3(SOLVER_THREADS), params, smem, stream);
    } else {
        cudaFuncSetAttribute(solver_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        e = cudaLaunchCooperativeKernel((const void *)solver_kernel<float>, dim3(grid_blocks),
                                        dim3(SOLVER_THREADS), params, smem, stream);
    }
    if (e != cudaSuccess) return cuda_status(e, "cudaLaunchCooperativeKernel(solver)");
    return PPE_OK;
}

}  // namespace ppe
