// Host side of the C ABI: grid handles, options, the FP64 operator and
// residual, and the mean removal of DLSM directions.  The solve drivers are
// in drive.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "net_iface.h"

namespace ppe {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }
void clear_error() { g_err.clear(); }

ppe_status cuda_status(cudaError_t e, const char *what)
{
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return PPE_ERR_NOMEM;
    return PPE_ERR_CUDA;
}

static ppe_status arg_error(const std::string &msg)
{
    set_error(msg);
    return PPE_ERR_ARG;
}

// y = A x in FP64 (plain one-thread-per-cell kernel; reference operator).
__global__ void apply_kernel(int nx, int ny, const double *__restrict__ dx, const double *__restrict__ dy,
                             const double *__restrict__ fx, const double *__restrict__ fy,
                             const double *__restrict__ x, double *__restrict__ y)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= nx || j >= ny) return;
    size_t k = (size_t)j * nx + i;
    double c = x[k];
    double xe = i + 1 < nx ? x[k + 1] : 0.0, xw = i > 0 ? x[k - 1] : 0.0;
    double xn = j + 1 < ny ? x[k + nx] : 0.0, xs = j > 0 ? x[k - nx] : 0.0;
    double ax = fx[i + 1] * (c - xe) + fx[i] * (c - xw);
    double ay = fy[j + 1] * (c - xn) + fy[j] * (c - xs);
    y[k] = dy[j] * ax + dx[i] * ay;
}

// r = -V S - A x in FP64 (no projection).
__global__ void residual_kernel(int nx, int ny, const double *__restrict__ dx, const double *__restrict__ dy,
                                const double *__restrict__ fx, const double *__restrict__ fy,
                                const double *__restrict__ S, const double *__restrict__ x, double *__restrict__ r)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= nx || j >= ny) return;
    size_t k = (size_t)j * nx + i;
    double c = x[k];
    double xe = i + 1 < nx ? x[k + 1] : 0.0, xw = i > 0 ? x[k - 1] : 0.0;
    double xn = j + 1 < ny ? x[k + nx] : 0.0, xs = j > 0 ? x[k - nx] : 0.0;
    double ax = fx[i + 1] * (c - xe) + fx[i] * (c - xw);
    double ay = fy[j + 1] * (c - xn) + fy[j] * (c - xs);
    r[k] = -dx[i] * dy[j] * S[k] - (dy[j] * ax + dx[i] * ay);
}

// Mean removal of a DLSM direction (A annihilates constants, so the loss of
// Eq. 18 leaves the constant part of NN(r) free; removing it keeps the FP32
// correction d from carrying a large constant).  Two kernels: per-block
// partial sums, then every block forms the mean from the partials and
// subtracts it.
constexpr int DIR_PART_BLOCKS = 152;

__global__ void __launch_bounds__(512) dir_partial_kernel(const float *e, int nx, int ny, int pitch, double *part)
{
    __shared__ double wsum[16];
    const size_t n = (size_t)nx * ny;
    float s = 0.f;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        s += e[(k / nx) * pitch + k % nx];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = (double)s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
        part[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(512) dir_center_kernel(float *e, int nx, int ny, int pitch, const double *part,
                                                         int nparts)
{
    __shared__ float mean;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < nparts; ++b) t += part[b];
        mean = (float)(t / ((double)nx * ny));
    }
    __syncthreads();
    const float m = mean;
    const size_t n = (size_t)nx * ny;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        e[(k / nx) * pitch + k % nx] -= m;
}

ppe_status center_direction(ppe_grid *g, cudaStream_t stream)
{
    dir_partial_kernel<<<DIR_PART_BLOCKS, 512, 0, stream>>>(g->e, g->nx, g->ny, g->pitch, g->dir_part);
    const int nb = (int)std::min<size_t>(4 * DIR_PART_BLOCKS, ((size_t)g->nx * g->ny + 511) / 512);
    dir_center_kernel<<<nb, 512, 0, stream>>>(g->e, g->nx, g->ny, g->pitch, g->dir_part, DIR_PART_BLOCKS);
    PPE_CUDA_TRY(cudaGetLastError());
    return PPE_OK;
}

}  // namespace ppe

using namespace ppe;

extern "C" {

const char *ppe_last_error(void) { return g_err.c_str(); }
const char *ppe_version(void) { return "ppe-gb300 0.1 sm_103a"; }

void ppe_default_options(ppe_solve_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->max_iters = 200000;
    o->num_cg = 3;
    o->num_dlsm = 2;
    o->hybrid_budget = 20000;
    o->inner_rtol = 0.3;
    o->dlsm_guard = 1e-10;
    o->blocks_per_sm = 2;
    o->dlsm_stall_limit = 6;
    o->dlsm_cost_iters = 16;
    o->spin_limit_ms = 2000;
}

void ppe_destroy_grid(ppe_grid *g)
{
    if (!g) return;
    net_release_grid(g);
    cudaFree(g->dx); cudaFree(g->dy); cudaFree(g->fx); cudaFree(g->fy);
    cudaFree(g->dx32); cudaFree(g->dy32); cudaFree(g->fx32); cudaFree(g->fy32);
    cudaFree(g->vec); cudaFree(g->e); cudaFree(g->tmaps_dev); cudaFree(g->dir_part);
    cudaFree(g->ycoef);
    launch_set_destroy(g->ls);
    mg_plan_destroy(g->mg);
    cudaFree(g->dir_r); cudaFree(g->dir_e);
    delete g;
}

ppe_status ppe_create_grid(int nx, int ny, const double *dx, const double *dy, ppe_bc bc,
                           const uint8_t *mask, ppe_grid **out)
{
    clear_error();
    if (!out) return arg_error("ppe_create_grid: out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || (long long)nx * ny >= (1LL << 31)) return arg_error("ppe_create_grid: bad nx/ny");
    if (!dx || !dy) return arg_error("ppe_create_grid: dx/dy NULL");
    if (bc != PPE_BC_NEUMANN) return arg_error("ppe_create_grid: only PPE_BC_NEUMANN is supported");
    for (int i = 0; i < nx; ++i)
        if (!(dx[i] > 0.0) || !std::isfinite(dx[i])) return arg_error("ppe_create_grid: dx must be positive and finite");
    for (int j = 0; j < ny; ++j)
        if (!(dy[j] > 0.0) || !std::isfinite(dy[j])) return arg_error("ppe_create_grid: dy must be positive and finite");

    ppe_grid *g = new ppe_grid();
    g->nx = nx; g->ny = ny;
    g->pitch = round_up(nx, PITCH_ALIGN);
    g->tiles_x = (nx + TILE_X - 1) / TILE_X;
    g->tiles_y = (ny + TILE_Y - 1) / TILE_Y;
    g->hdx.assign(dx, dx + nx);
    g->hdy.assign(dy, dy + ny);
    if (mask) g->hmask.assign(mask, mask + (size_t)nx * ny);
    ppe_default_options(&g->opts);
    cudaGetDevice(&g->device);
    g->lx = 0; for (double v : g->hdx) g->lx += v;
    g->ly = 0; for (double v : g->hdy) g->ly += v;

    // face coefficients 2 / (w_left + w_right), zero at the walls
    std::vector<double> fx(nx + 1, 0.0), fy(ny + 1, 0.0);
    for (int i = 1; i < nx; ++i) fx[i] = 2.0 / (dx[i - 1] + dx[i]);
    for (int j = 1; j < ny; ++j) fy[j] = 2.0 / (dy[j - 1] + dy[j]);
    double dmax = 0.0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            dmax = std::max(dmax, dy[j] * (fx[i] + fx[i + 1]) + dx[i] * (fy[j] + fy[j + 1]));
    g->diag_max = dmax;
    std::vector<float> dx32(dx, dx + nx), dy32(dy, dy + ny), fx32(fx.begin(), fx.end()), fy32(fy.begin(), fy.end());

    auto fail = [&](ppe_status s) { ppe_destroy_grid(g); return s; };
#define G_ALLOC(ptr, bytes)                                                              \
    do {                                                                                 \
        cudaError_t _e = cudaMalloc((void **)&(ptr), (bytes));                           \
        if (_e != cudaSuccess) return fail(cuda_status(_e, "cudaMalloc(grid)"));         \
    } while (0)
#define G_COPY(dst, src, bytes)                                                          \
    do {                                                                                 \
        cudaError_t _e = cudaMemcpy((dst), (src), (bytes), cudaMemcpyHostToDevice);      \
        if (_e != cudaSuccess) return fail(cuda_status(_e, "cudaMemcpy(grid)"));         \
    } while (0)
    G_ALLOC(g->dx, nx * 8); G_COPY(g->dx, dx, nx * 8);
    G_ALLOC(g->dy, ny * 8); G_COPY(g->dy, dy, ny * 8);
    G_ALLOC(g->fx, (nx + 1) * 8); G_COPY(g->fx, fx.data(), (nx + 1) * 8);
    G_ALLOC(g->fy, (ny + 1) * 8); G_COPY(g->fy, fy.data(), (ny + 1) * 8);
    G_ALLOC(g->dx32, nx * 4); G_COPY(g->dx32, dx32.data(), nx * 4);
    G_ALLOC(g->dy32, ny * 4); G_COPY(g->dy32, dy32.data(), ny * 4);
    G_ALLOC(g->fx32, (nx + 1) * 4); G_COPY(g->fx32, fx32.data(), (nx + 1) * 4);
    G_ALLOC(g->fy32, (ny + 1) * 4); G_COPY(g->fy32, fy32.data(), (ny + 1) * 4);
    size_t vbytes = (size_t)g->pitch * ny * 8;
    G_ALLOC(g->vec, vbytes * 5);
    char *base = (char *)g->vec;
    g->r[0] = base; g->r[1] = base + vbytes; g->p[0] = base + 2 * vbytes; g->p[1] = base + 3 * vbytes;
    g->d = base + 4 * vbytes;
    {
        std::vector<float> yc((size_t)4 * ny);
        for (int j = 0; j < ny; ++j) {
            yc[4 * j] = (float)dy[j];
            yc[4 * j + 1] = (float)fy[j];
            yc[4 * j + 2] = (float)fy[j + 1];
            yc[4 * j + 3] = 0.f;
        }
        G_ALLOC(g->ycoef, yc.size() * sizeof(float));
        G_COPY(g->ycoef, yc.data(), yc.size() * sizeof(float));
        CUtensorMap maps[SV_COUNT * NMAPS];   // one set per kernel variant, in SolverVariant order
        ppe_status ms = PPE_OK;
        for (int v = 0; v < SV_COUNT && ms == PPE_OK; ++v)
            ms = encode_solver_maps(g->r, g->p, g->d, g->ycoef, nx, ny, g->pitch, (SolverVariant)v, maps + v * NMAPS);
        if (ms != PPE_OK) return fail(ms);
        G_ALLOC(g->tmaps_dev, sizeof maps);
        G_COPY(g->tmaps_dev, maps, sizeof maps);
    }
    G_ALLOC(g->e, (size_t)g->pitch * ny * 4);
    G_ALLOC(g->dir_part, DIR_PART_BLOCKS * sizeof(double));
    {
        cudaError_t _e = cudaMemset(g->e, 0, (size_t)g->pitch * ny * 4);
        if (_e != cudaSuccess) return fail(cuda_status(_e, "cudaMemset(e)"));
    }
    // tile counts of the tile shapes; workspaces are sized for the largest
    int ntiles = std::max(g->tiles_x, (nx + TILE_X_STREAM - 1) / TILE_X_STREAM) *
                 ((ny + TILE_Y_R4 - 1) / TILE_Y_R4);
    {
        ppe_status ls = launch_set_create(1, ntiles, ntiles + 1, &g->ls);
        if (ls != PPE_OK) return fail(ls);
    }
    {
        static std::atomic<uint64_t> next_id{1};
        g->id = next_id++;
    }
#undef G_ALLOC
#undef G_COPY
    *out = g;
    return PPE_OK;
}

ppe_status ppe_grid_shape(const ppe_grid *g, int *nx, int *ny)
{
    if (!g) return arg_error("ppe_grid_shape: NULL grid");
    if (nx) *nx = g->nx;
    if (ny) *ny = g->ny;
    return PPE_OK;
}

ppe_status ppe_set_options(ppe_grid *g, const ppe_solve_opts *o)
{
    clear_error();
    if (!g || !o) return arg_error("ppe_set_options: NULL argument");
    if (o->max_iters < 1 || o->num_cg < 1 || o->num_dlsm < 1 || o->hybrid_budget < 0 ||
        !(o->inner_rtol > 0.0 && o->inner_rtol < 1.0) || !(o->dlsm_guard >= 0.0) || o->blocks_per_sm < 0 ||
        o->iter_pass < 0 || o->iter_pass > 2 || o->dlsm_stall_limit < 0 ||
        o->dlsm_cost_iters < 0 || o->spin_limit_ms < 0 || o->host_loop < 0 || o->host_loop > 1 ||
        o->debug_skip_block < 0 || o->preconditioner < 0 || o->preconditioner > 1 || o->debug_force_stall < 0 ||
        (o->tile_rows != 0 && o->tile_rows != TILE_Y && o->tile_rows != TILE_Y_R8 && o->tile_rows != TILE_Y_R4))
        return arg_error("ppe_set_options: option out of range");
    g->opts = *o;
    return PPE_OK;
}

ppe_status ppe_residual(ppe_grid *g, const double *S, const double *x, double *r, void *stream)
{
    clear_error();
    if (!g || !S || !x || !r) return arg_error("ppe_residual: NULL argument");
    if (r == x || r == S) return arg_error("ppe_residual: r may not alias S or x");
    dim3 blk(32, 8), grd((g->nx + 31) / 32, (g->ny + 7) / 8);
    residual_kernel<<<grd, blk, 0, (cudaStream_t)stream>>>(g->nx, g->ny, g->dx, g->dy, g->fx, g->fy, S, x, r);
    PPE_CUDA_TRY(cudaGetLastError());
    return PPE_OK;
}

ppe_status ppe_set_direction_source(ppe_grid *g, ppe_direction_fn fn, void *user)
{
    clear_error();
    if (!g) return arg_error("ppe_set_direction_source: NULL grid");
    if (fn && !g->dir_r) {
        size_t bytes = (size_t)g->nx * g->ny * sizeof(float);
        PPE_CUDA_TRY(cudaMalloc(&g->dir_r, bytes));
        PPE_CUDA_TRY(cudaMalloc(&g->dir_e, bytes));
    }
    g->dir_fn = fn;
    g->dir_user = user;
    return PPE_OK;
}

ppe_status ppe_apply(ppe_grid *g, const double *x, double *y, void *stream)
{
    clear_error();
    if (!g || !x || !y) return arg_error("ppe_apply: NULL argument");
    if (x == y) return arg_error("ppe_apply: x and y may not alias");
    dim3 blk(32, 8), grd((g->nx + 31) / 32, (g->ny + 7) / 8);
    apply_kernel<<<grd, blk, 0, (cudaStream_t)stream>>>(g->nx, g->ny, g->dx, g->dy, g->fx, g->fy, x, y);
    PPE_CUDA_TRY(cudaGetLastError());
    return PPE_OK;
}

}  // extern "C"
