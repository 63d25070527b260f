// Persistent solver kernel: single-reduction Jacobi PCG (FP32 or FP64 inner
// vectors) with FP64 residual replacement, interleaved DLSM steps, and the
// compatibility projection / zero-mean normalisation of the Neumann problem.
//
// One cooperative launch runs the per-system state machine of every system of
// a batch.  Each block owns a contiguous range of tiles (of one or a few
// systems).  A step: every block runs the current pass of each of its systems
// over its tiles and writes one FP64 partial-sum record per system, then
// arrives at a grid-wide counter barrier.  After the barrier each block reads
// the partial records of its systems (fixed order, so every block obtains the
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
// preconditioning.  Per iteration, with u = D^-1 r and w = A u:
//   p = u + beta p,  s = w + beta s  (s = A p),  x += alpha p,  r -= alpha s,
//   gamma' = r.u, delta' = (A u).u, beta' = gamma'/gamma,
//   alpha' = gamma' / (delta' - beta' gamma' / alpha).
// Each block recomputes the new residual on a one-cell ring around its tile
// (reading r two cells out) so that A u' is available in the same pass.
//
// Mixed precision: the FP32 recursive residual is replaced by the FP64 true
// residual b - A(x + d) whenever it has dropped by a factor ru_delta since
// the last replacement, and before convergence is declared; the search
// direction is kept across a replacement (reliable updates), so the FP32
// iteration converges like the FP64 one.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "internal.h"

namespace ppe {

namespace {

constexpr int WX = TILE_X + 4;     // tile window with a two-cell halo
constexpr int WY = TILE_Y + 4;
constexpr int WN = WX * WY;
constexpr int NWARP = SOLVER_THREADS / 32;
constexpr int NL = (WN + SOLVER_THREADS - 1) / SOLVER_THREADS;   // window loads per thread

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
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
    float red_hi[NPART][NWARP], red_lo[NPART][NWARP];
    SysDesc sd[SMAX];
    SysState st[SMAX];
    double tot[NPART];
    int32_t tag_d, tag_f;   // tile whose coefficients are in cfd / cff
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

// Coefficients of a tile do not change between steps: a block that keeps
// working on the same tile reuses them.  Every caller synchronises the block
// before it reads the coefficients.
template <typename S> __device__ __forceinline__ void load_coef_f(S &sm, const SysDesc &sd, int i0, int j0, int tag)
{
    const int have = sm.tag_f;
    __syncthreads();
    if (have == tag) return;
    load_coef<float>(sm.cff, sd, i0, j0, sd.dx32, sd.fx32, sd.dy32, sd.fy32);
    if (threadIdx.x == 0) sm.tag_f = tag;
}

template <typename S> __device__ __forceinline__ void load_coef_d(S &sm, const SysDesc &sd, int i0, int j0, int tag)
{
    const int have = sm.tag_d;
    __syncthreads();
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
    return i >= 0 && j >= 0 && i < sd.nx && j < sd.ny;
}

__device__ __forceinline__ bool in_ring1(int wi, int wj) { return wi >= 1 && wi < WX - 1 && wj >= 1 && wj < WY - 1; }

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

// b statistics: b = -V S
template <typename T, typename S> __device__ void pass_init(S &sm, const SysDesc &sd, int i0, int j0, Acc &acc)
{
    double t[NPART] = {0, 0, 0, 0, 0, 0};
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    int j = j0 + ty;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int i = i0 + tx + 32 * c;
        if (i < sd.nx && j < sd.ny) {
            double b = -sd.dx[i] * sd.dy[j] * sd.f[(size_t)j * sd.nx + i];
            t[0] += b; t[1] += b * b; t[2] += fabs(b);
        }
    }
    warp_accumulate(t, acc);
}

// FP64 true residual r = (b - mu_b) - A (x + d); stored into the inner buffer.
template <typename T, typename S>
__device__ void pass_res(S &sm, const SysDesc &sd, const SysState &st, int i0, int j0, int tag, Acc &acc)
{
    Coef<double> &cf = sm.cfd;
    double *X = reinterpret_cast<double *>(&sm.w);
    load_coef_d(sm, sd, i0, j0, tag);
    const T *d = (const T *)sd.d;
    double xv[NL];
#pragma unroll
    for (int q = 0; q < NL; ++q) {
        int k = threadIdx.x + q * SOLVER_THREADS;
        xv[q] = 0.0;
        if (k < WN) {
            int wi = k % WX, wj = k / WX, i = i0 - 2 + wi, j = j0 - 2 + wj;
            if (in_ring1(wi, wj) && in_dom(sd, i, j)) {
                xv[q] = ld_cg(sd.x + (size_t)j * sd.nx + i);
                if (st.has_d) xv[q] += (double)ld_cg(d + (size_t)j * sd.pitch + i);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < NL; ++q) {
        int k = threadIdx.x + q * SOLVER_THREADS;
        if (k < WN) X[k] = xv[q];
    }
    __syncthreads();
    double t[NPART] = {0, 0, 0, 0, 0, 0};
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    int j = j0 + ty, wj = ty + 2;
    T *r = (T *)sd.r[st.cur];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int i = i0 + tx + 32 * c, wi = tx + 32 * c + 2;
        if (i < sd.nx && j < sd.ny) {
            double b = -sd.dx[i] * sd.dy[j] * ld_cg(sd.f + (size_t)j * sd.nx + i) - st.mu_b;
            double rv = b - stencil<double>(cf, X, wi, wj);
            r[(size_t)j * sd.pitch + i] = (T)rv;
            t[0] += rv; t[1] += rv * rv;
        }
    }
    warp_accumulate(t, acc);
    __syncthreads();
}

// u = D^-1 (r - mu), w = A u; dots r.u, w.u, r.r, sum r.  Folds d into x
// when a replacement is pending.
template <typename T, typename S>
__device__ void pass_restart(S &sm, const SysDesc &sd, const SysState &st, int i0, int j0, int tag, Acc &acc)
{
    Coef<T> &cf = coef_of<T>(sm);
    T *R = sm.w.a0, *U = sm.w.a1;
    load_coef_t<T>(sm, sd, i0, j0, tag);
    const T *rin = (const T *)sd.r[st.cur];
    const T mu = sc_mu<T>(st);
    T rv[NL];
#pragma unroll
    for (int q = 0; q < NL; ++q) {
        int k = threadIdx.x + q * SOLVER_THREADS;
        rv[q] = 0;
        if (k < WN) {
            int wi = k % WX, wj = k / WX, i = i0 - 2 + wi, j = j0 - 2 + wj;
            if (in_ring1(wi, wj) && in_dom(sd, i, j)) rv[q] = ld_cg(rin + (size_t)j * sd.pitch + i) - mu;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NL; ++q) {
        int k = threadIdx.x + q * SOLVER_THREADS;
        if (k < WN) {
            R[k] = rv[q];
            U[k] = rv[q] * dinv_at<T>(cf, k % WX, k / WX);
        }
    }
    __syncthreads();
    T t[NPART] = {0, 0, 0, 0, 0, 0};
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    int j = j0 + ty, wj = ty + 2;
    T *dd = (T *)sd.d;
    const T *pv = (const T *)sd.p;
    const T *sv = (const T *)sd.s[st.cur];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int i = i0 + tx + 32 * c, wi = tx + 32 * c + 2;
        if (i < sd.nx && j < sd.ny) {
            int k = wj * WX + wi;
            T w = stencil<T>(cf, U, wi, wj);
            t[0] += R[k] * U[k]; t[1] += w * U[k]; t[2] += R[k] * R[k]; t[3] += R[k];
            if (st.keep_dir) {   // continuation after a residual replacement: u.s and p.s of the kept direction
                size_t gi = (size_t)j * sd.pitch + i;
                T so = ld_cg(sv + gi);
                t[4] += U[k] * so; t[5] += ld_cg(pv + gi) * so;
            }
            if (st.reset_d) {
                size_t gi = (size_t)j * sd.pitch + i;
                if (st.fold_d) sd.x[(size_t)j * sd.nx + i] += (double)ld_cg(dd + gi);
                dd[gi] = T(0);
            }
        }
    }
    warp_accumulate(t, acc);
    __syncthreads();
}

// One single-reduction PCG iteration.
template <typename T, typename S>
__device__ void pass_iter(S &sm, const SysDesc &sd, const SysState &st, int i0, int j0, int tag, Acc &acc)
{
    Coef<T> &cf = coef_of<T>(sm);
    T *R = sm.w.a0, *U = sm.w.a1, *Sv = sm.w.a2, *Rn = sm.w.a3, *Un = sm.w.a4, *Sn = sm.w.a5;
    load_coef_t<T>(sm, sd, i0, j0, tag);
    const int cur = st.cur;
    const T *rin = (const T *)sd.r[cur];
    const T *sin = (const T *)sd.s[cur];
    T *rout = (T *)sd.r[cur ^ 1];
    T *sout = (T *)sd.s[cur ^ 1];
    T *pv = (T *)sd.p;
    T *dv = (T *)sd.d;
    const T mu = sc_mu<T>(st), alpha = sc_alpha<T>(st), beta = sc_beta<T>(st);
    const bool first = st.first != 0;
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    const int j = j0 + ty, wj0 = ty + 2;
    // issue every global load of this tile before using any of them
    T rv[NL], sv[NL], pold[4], dold[4];
#pragma unroll
    for (int q = 0; q < NL; ++q) {
        int k = threadIdx.x + q * SOLVER_THREADS;
        rv[q] = 0; sv[q] = 0;
        if (k < WN) {
            int wi = k % WX, wj = k / WX, i = i0 - 2 + wi, jj = j0 - 2 + wj;
            if (in_dom(sd, i, jj)) {
                size_t gi = (size_t)jj * sd.pitch + i;
                rv[q] = ld_cg(rin + gi);
                if (!first && in_ring1(wi, wj)) sv[q] = ld_cg(sin + gi);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int i = i0 + tx + 32 * c;
        pold[c] = 0; dold[c] = 0;
        if (i < sd.nx && j < sd.ny) {
            size_t gi = (size_t)j * sd.pitch + i;
            if (!first) pold[c] = ld_cg(pv + gi);
            dold[c] = ld_cg(dv + gi);
        }
    }
    __syncthreads();   // coefficients visible
#pragma unroll
    for (int q = 0; q < NL; ++q) {
        int k = threadIdx.x + q * SOLVER_THREADS;
        if (k < WN) {
            int wi = k % WX, wj = k / WX;
            bool in = in_dom(sd, i0 - 2 + wi, j0 - 2 + wj);
            T r = in ? rv[q] - mu : T(0);
            R[k] = r;
            U[k] = r * dinv_at<T>(cf, wi, wj);
            Sv[k] = sv[q];
        }
    }
    __syncthreads();
    // new residual on the tile and its one-cell ring
    for (int k = threadIdx.x; k < WN; k += blockDim.x) {
        int wi = k % WX, wj = k / WX, i = i0 - 2 + wi, jj = j0 - 2 + wj;
        T rn = 0, un = 0, sn = 0;
        if (in_ring1(wi, wj) && in_dom(sd, i, jj)) {
            T w = stencil<T>(cf, U, wi, wj);
            sn = w + beta * Sv[k];
            rn = R[k] - alpha * sn;
            un = rn * dinv_at<T>(cf, wi, wj);
        }
        Rn[k] = rn; Un[k] = un; Sn[k] = sn;
    }
    __syncthreads();
    T t[NPART] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int i = i0 + tx + 32 * c, wi = tx + 32 * c + 2;
        if (i < sd.nx && j < sd.ny) {
            int k = wj0 * WX + wi;
            size_t gi = (size_t)j * sd.pitch + i;
            T pn = U[k] + beta * pold[c];
            pv[gi] = pn;
            dv[gi] = dold[c] + alpha * pn;
            sout[gi] = Sn[k];
            T rn = Rn[k], un = Un[k];
            rout[gi] = rn;
            T wn = stencil<T>(cf, Un, wi, wj0);
            t[0] += rn * un; t[1] += wn * un; t[2] += rn * rn; t[3] += rn;
            t[4] += un * Sn[k]; t[5] += pn * Sn[k];
        }
    }
    warp_accumulate(t, acc);
    __syncthreads();
}

// DLSM dots r.e, e.(A e), e.e  (Eq. 11); with upd: d += alpha e, r_new = r - alpha A e (Eq. 12)
template <typename T, typename S, bool UPD>
__device__ void pass_dlsm(S &sm, const SysDesc &sd, const SysState &st, int i0, int j0, int tag, Acc &acc)
{
    Coef<float> &cf = sm.cff;
    float *E = reinterpret_cast<float *>(&sm.w);
    load_coef_f(sm, sd, i0, j0, tag);
    float ev[NL];
#pragma unroll
    for (int q = 0; q < NL; ++q) {
        int k = threadIdx.x + q * SOLVER_THREADS;
        ev[q] = 0.f;
        if (k < WN) {
            int wi = k % WX, wj = k / WX, i = i0 - 2 + wi, j = j0 - 2 + wj;
            if (in_ring1(wi, wj) && in_dom(sd, i, j)) ev[q] = ld_cg(sd.e + (size_t)j * sd.pitch + i);
        }
    }
#pragma unroll
    for (int q = 0; q < NL; ++q) {
        int k = threadIdx.x + q * SOLVER_THREADS;
        if (k < WN) E[k] = ev[q];
    }
    __syncthreads();
    const int cur = st.cur;
    const T *rin = (const T *)sd.r[cur];
    T *rout = (T *)sd.r[cur ^ 1];
    T *dv = (T *)sd.d;
    const T mu = sc_mu<T>(st), alpha = sc_alpha_d<T>(st);
    T t[NPART] = {0, 0, 0, 0, 0, 0};
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    int j = j0 + ty, wj = ty + 2;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int i = i0 + tx + 32 * c, wi = tx + 32 * c + 2;
        if (i < sd.nx && j < sd.ny) {
            int k = wj * WX + wi;
            size_t gi = (size_t)j * sd.pitch + i;
            T e = (T)E[k];
            T q = (T)stencil<float>(cf, E, wi, wj);
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
    const T *dd = (const T *)sd.d;
    double t[NPART] = {0, 0, 0, 0, 0, 0};
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    int j = j0 + ty;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int i = i0 + tx + 32 * c;
        if (i < sd.nx && j < sd.ny) {
            size_t gx = (size_t)j * sd.nx + i;
            double x = st.zero_x ? 0.0 : ld_cg(sd.x + gx);
            if (st.fold_d && !st.zero_x) x += (double)ld_cg(dd + (size_t)j * sd.pitch + i);
            sd.x[gx] = x;
            double v = sd.dx[i] * sd.dy[j];
            t[0] += v; t[1] += v * x;
        }
    }
    warp_accumulate(t, acc);
}

template <typename T, typename S>
__device__ void pass_final2(S &sm, const SysDesc &sd, const SysState &st, int i0, int j0, Acc &acc)
{
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    int j = j0 + ty;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int i = i0 + tx + 32 * c;
        if (i < sd.nx && j < sd.ny) {
            size_t gx = (size_t)j * sd.nx + i;
            sd.x[gx] = ld_cg(sd.x + gx) - st.xmean;
        }
    }
}

// ---------------------------------------------------------------------------
// state machine
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool is_pass_phase(int ph) { return ph != PH_NET && ph != PH_DONE; }

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
    const bool pcg_like = sd.mode == PPE_MODE_PCG || s.fell_back;
    switch (s.phase) {
    case PH_INIT: {
        s.mu_b = t[0] * sd.inv_n;
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
        s.rnorm = sqrt(rr > 0.0 ? rr : 0.0);
        s.relres = fast_div(s.rnorm, s.bnorm);
        s.fold_d = s.has_d;
        if (!isfinite(s.relres)) {
            s.status = PPE_ERR_NAN;
            s.fold_d = 0;
            s.phase = PH_FINAL1;
        } else if (s.relres <= sd.tol) {
            s.phase = PH_FINAL1;
        } else if (s.it_total >= iter_cap(sd) || s.refinements > 5000) {
            s.status = PPE_ERR_NOT_CONVERGED;
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
        s.rho = rr > 0.0 ? rr : 0.0;
        s.reset_d = 0;
        s.fold_d = 0;
        s.has_d = 1;
        s.cg_count = 0;
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
        s.it_pcg++;
        s.it_total++;
        s.cur ^= 1;
        s.mu = t[3] * sd.inv_n;
        double rr = t[2] - N * s.mu * s.mu;
        s.rho = rr > 0.0 ? rr : 0.0;
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
        if (rho <= s.target * s.target || s.it_total >= iter_cap(sd) || !ok || (pcg_like && rho <= ru * ru)) {
            // gamma and alpha of the direction in use stay the reference for the
            // continuation after the residual replacement
            to_res(s, pcg_like && ok ? 1 : 0);
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
        const double rho_before = s.rho;
        s.rho = rr > 0.0 ? rr : 0.0;
        // a direction that removes less than 10% of the residual norm is not
        // worth its inference; after several in a row continue as plain PCG
        s.dlsm_useless = s.rho > 0.81 * rho_before ? s.dlsm_useless + 1 : 0;
        if (s.dlsm_useless >= 6) s.fell_back = 1;
        s.dlsm_count++;
        if (sd.mode == PPE_MODE_HYBRID && !s.fell_back && s.it_total >= sd.hybrid_budget) s.fell_back = 1;
        if (s.rho <= s.target * s.target || s.it_total >= iter_cap(sd) || !isfinite(s.rho)) {
            to_res(s, 0);
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
    s.alpha_f = (float)s.alpha;
    s.beta_f = (float)s.beta;
    s.mu_f = (float)s.mu;
    s.alpha_d_f = (float)s.alpha_d;
}

template <typename T, typename S>
__device__ void run_pass(S &sm, int q, int ph, int t, Acc &acc)
{
    const SysDesc &sd = sm.sd[q];
    const SysState &st = sm.st[q];
    int lt = t - sd.tile0;
    int i0 = (lt % sd.tiles_x) * TILE_X, j0 = (lt / sd.tiles_x) * TILE_Y;
    switch (ph) {
    case PH_INIT: pass_init<T>(sm, sd, i0, j0, acc); break;
    case PH_RES: pass_res<T>(sm, sd, st, i0, j0, t, acc); break;
    case PH_RESTART: pass_restart<T>(sm, sd, st, i0, j0, t, acc); break;
    case PH_ITER: pass_iter<T>(sm, sd, st, i0, j0, t, acc); break;
    case PH_DLSM_DOT: pass_dlsm<T, S, false>(sm, sd, st, i0, j0, t, acc); break;
    case PH_DLSM_UPD: pass_dlsm<T, S, true>(sm, sd, st, i0, j0, t, acc); break;
    case PH_FINAL1: pass_final1<T>(sm, sd, st, i0, j0, acc); break;
    case PH_FINAL2: pass_final2<T>(sm, sd, st, i0, j0, acc); break;
    default: break;
    }
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

// Block-reduce the per-warp accumulators (lane 0 of each warp) into threads
// 0..NPART-1 (fixed order).
template <typename S> __device__ void block_reduce_acc(S &sm, const Acc &acc, float (&hi)[NPART], float (&lo)[NPART])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NPART; ++k) {
            sm.red_hi[k][warp] = acc.hi[k];
            sm.red_lo[k][warp] = acc.lo[k];
        }
    __syncthreads();
    if (threadIdx.x < NPART) {
        float h = 0.f, l = 0.f;
        for (int w = 0; w < NWARP; ++w) ff_add(h, l, sm.red_hi[threadIdx.x][w], sm.red_lo[threadIdx.x][w]);
        hi[threadIdx.x] = h;
        lo[threadIdx.x] = l;
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(SOLVER_THREADS) solver_kernel(SolverArgs a, int resume_net)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemT<T> &sm = *reinterpret_cast<SmemT<T> *>(smem_raw);
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
    }
    __syncthreads();
    if (threadIdx.x == 0 && resume_net)
        for (int q = 0; q < nq; ++q)
            if (sm.st[q].phase == PH_NET) sm.st[q].phase = PH_DLSM_DOT;
    __syncthreads();
    const bool prof = a.prof && blockIdx.x == 0 && threadIdx.x == 0;
    uint64_t t_a = prof ? globaltimer_ns() : 0, t_b = 0, t_c = 0;
    __shared__ float pub_hi[NPART], pub_lo[NPART];
    for (uint32_t step = 1;; ++step) {
        // any system of this block still running?
        bool any = false;
        for (int q = 0; q < nq; ++q) any |= is_pass_phase(sm.st[q].phase);
        if (!any) break;
        const int bank = step & 1;
        // 1) passes; publish one record per live system
        for (int q = 0; q < nq; ++q) {
            const SysDesc &sd = sm.sd[q];
            const int ph = sm.st[q].phase;
            if (!is_pass_phase(ph)) continue;
            Acc acc;
            acc_zero(acc);
            const int lo_t = max(br.t0, sd.tile0), hi_t = min(br.t1, sd.tile0 + sd.ntiles);
            for (int t = lo_t; t < hi_t; ++t) run_pass<T>(sm, q, ph, t, acc);
            block_reduce_acc(sm, acc, pub_hi, pub_lo);
            Slot *slot = a.slots + (size_t)bank * a.nslots + sd.part0 + (blockIdx.x - sd.blk0);
            if (threadIdx.x < NPART) {
                slot->hi[threadIdx.x] = pub_hi[threadIdx.x];
                slot->lo[threadIdx.x] = pub_lo[threadIdx.x];
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(&a.arrive[br.s0 + q], 1u);
            }
        }
        if (prof) t_b = globaltimer_ns();
        // 2) wait for the records of every block of each live system, reduce, advance
        for (int q = 0; q < nq; ++q) {
            const SysDesc &sd = sm.sd[q];
            if (!is_pass_phase(sm.st[q].phase)) continue;
            float h[NPART], l[NPART];
#pragma unroll
            for (int k = 0; k < NPART; ++k) h[k] = l[k] = 0.f;
            const Slot *base = a.slots + (size_t)bank * a.nslots + sd.part0;
            if (threadIdx.x == 0) {
                // every block of this system has published step `step`
                const uint32_t need = step * (uint32_t)sd.nparts;
                const uint32_t *cnt = a.arrive + br.s0 + q;
                if (ld_acquire_u32(cnt) < need) {
                    uint64_t t0 = globaltimer_ns();
                    while (ld_acquire_u32(cnt) < need) {
                        if ((int64_t)(globaltimer_ns() - t0) > a.spin_limit_ns) {
                            atomicExch(&a.ctl->err, (int32_t)PPE_ERR_TIMEOUT);
                            sm.go = 0;
                            break;
                        }
                        __nanosleep(20);
                    }
                }
                __threadfence();
            }
            __syncthreads();
            for (int b = threadIdx.x; b < sd.nparts; b += blockDim.x) {
                const Slot *sl = base + b;
#pragma unroll
                for (int k = 0; k < NPART; ++k) ff_add(h[k], l[k], ld_cg(&sl->hi[k]), ld_cg(&sl->lo[k]));
            }
            // block reduction in fixed order: warp shuffle, then warps
#pragma unroll
            for (int k = 0; k < NPART; ++k) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    float oh = __shfl_down_sync(0xffffffffu, h[k], o);
                    float ol = __shfl_down_sync(0xffffffffu, l[k], o);
                    ff_add(h[k], l[k], oh, ol);
                }
                if (lane == 0) {
                    sm.red_hi[k][warp] = h[k];
                    sm.red_lo[k][warp] = l[k];
                }
            }
            __syncthreads();
            if (!sm.go) return;                         // a bounded wait expired: leave without writing state
            if (threadIdx.x < NPART) {
                float th = 0.f, tl = 0.f;
                for (int w = 0; w < NWARP; ++w) ff_add(th, tl, sm.red_hi[threadIdx.x][w], sm.red_lo[threadIdx.x][w]);
                sm.tot[threadIdx.x] = (double)th + (double)tl;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double tt[NPART];
                for (int k = 0; k < NPART; ++k) tt[k] = sm.tot[k];
                advance(sd, sm.st[q], tt);
            }
            __syncthreads();
        }
        if (prof) {
            t_c = globaltimer_ns();
            atomicAdd(&a.prof[0], (unsigned long long)(t_b - t_a));
            atomicAdd(&a.prof[2], (unsigned long long)(t_c - t_b));
            atomicAdd(&a.prof[3], 1ull);
            t_a = t_c;
        }
    }
    // write back the states of the systems this block owns
    for (int q = 0; q < nq; ++q) {
        if ((int)blockIdx.x != sm.sd[q].blk0) continue;
        const int32_t *src = reinterpret_cast<const int32_t *>(&sm.st[q]);
        int32_t *dst = reinterpret_cast<int32_t *>(a.st + br.s0 + q);
        for (int k = threadIdx.x; k < (int)(sizeof(SysState) / 4); k += blockDim.x) dst[k] = src[k];
    }
}

// The dynamic shared-memory opt-in is a per-function attribute: set it once.
void set_solver_attributes()
{
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(solver_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(SmemT<double>));
        cudaFuncSetAttribute(solver_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(SmemT<float>));
    });
}

}  // namespace

int solver_max_blocks(bool fp64, int blocks_per_sm_req)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    size_t smem = fp64 ? sizeof(SmemT<double>) : sizeof(SmemT<float>);
    set_solver_attributes();
    if (fp64)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solver_kernel<double>, SOLVER_THREADS, smem);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solver_kernel<float>, SOLVER_THREADS, smem);
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
    set_solver_attributes();
    if (fp64)
        e = cudaLaunchCooperativeKernel((const void *)solver_kernel<double>, dim3(grid_blocks),
                                        dim3(SOLVER_THREADS), params, smem, stream);
    else
        e = cudaLaunchCooperativeKernel((const void *)solver_kernel<float>, dim3(grid_blocks),
                                        dim3(SOLVER_THREADS), params, smem, stream);
    if (e != cudaSuccess) return cuda_status(e, "cudaLaunchCooperativeKernel(solver)");
    return PPE_OK;
}

}  // namespace ppe
