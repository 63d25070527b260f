// Host side of the C ABI: grid handles, the FP64 operator, and the solve
// drivers that launch the persistent solver kernel.
#include <cuda_runtime.h>

#include <algorithm>
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

static int g_spin_limit_ms = 2000;

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

// r_hat = (r - mu) / sqrt(rho) of a system's current residual, unpitched FP32.
__global__ void rhat_kernel(const SysDesc *sd, const SysState *st, float *out)
{
    const int nx = sd->nx, ny = sd->ny;
    const size_t n = (size_t)nx * ny;
    const double scale = st->rho > 0.0 ? 1.0 / sqrt(st->rho) : 0.0;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        size_t i = k % nx, j = k / nx, g = j * sd->pitch + i;
        double v = sd->precision == PPE_PREC_FP64 ? ((const double *)sd->r[st->cur])[g]
                                                  : (double)((const float *)sd->r[st->cur])[g];
        out[k] = (float)((v - st->mu) * scale);
    }
}

// e (pitched, solver layout) <- e_user (unpitched)
__global__ void pitch_copy_kernel(const float *src, float *dst, int nx, int ny, int pitch)
{
    const size_t n = (size_t)nx * ny;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        dst[(k / nx) * pitch + k % nx] = src[k];
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
    o->inner_rtol = 0.1;
    o->dlsm_guard = 1e-10;
    o->blocks_per_sm = 2;
    o->dlsm_stall_limit = 6;
    o->dlsm_cost_iters = 16;
}

void ppe_destroy_grid(ppe_grid *g)
{
    if (!g) return;
    net_release_grid(g);
    cudaFree(g->dx); cudaFree(g->dy); cudaFree(g->fx); cudaFree(g->fy);
    cudaFree(g->dx32); cudaFree(g->dy32); cudaFree(g->fx32); cudaFree(g->fy32);
    cudaFree(g->vec); cudaFree(g->e); cudaFree(g->tmaps_dev); cudaFree(g->dir_part);
    cudaFree(g->ycoef);
    cudaFree(g->sys_dev); cudaFree(g->st_dev); cudaFree(g->ranges_dev); cudaFree(g->slots_dev);
    cudaFree(g->ctl_dev);
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
        CUtensorMap maps[3 * NMAPS];     // one set per kernel variant, in SolverVariant order
        ppe_status ms = PPE_OK;
        for (int v = 0; v < 3 && ms == PPE_OK; ++v)
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
    // tile counts of the two tile widths; workspaces are sized for the larger
    int ntiles = std::max(g->tiles_x, (nx + TILE_X_STREAM - 1) / TILE_X_STREAM) * g->tiles_y;
    G_ALLOC(g->sys_dev, sizeof(SysDesc));
    G_ALLOC(g->st_dev, sizeof(SysState));
    g->ranges_blocks = ntiles;
    G_ALLOC(g->ranges_dev, (size_t)ntiles * sizeof(BlockRange));
    G_ALLOC(g->slots_dev, (size_t)2 * (ntiles + 1) * sizeof(Slot));
    G_ALLOC(g->ctl_dev, sizeof(Control));
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
        o->dlsm_cost_iters < 0)
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

namespace ppe {

static SysDesc make_desc(const ppe_grid *g, const double *rhs, double *x, double tol, ppe_mode mode,
                         ppe_precision prec, int tile0, SolverVariant v)
{
    SysDesc sd;
    std::memset(&sd, 0, sizeof(sd));
    const int tw = v == SV_FP32_STREAM ? TILE_X_STREAM : TILE_X;
    sd.nx = g->nx; sd.ny = g->ny; sd.pitch = g->pitch;
    sd.tiles_x = (g->nx + tw - 1) / tw; sd.tiles_y = g->tiles_y;
    sd.tile0 = tile0; sd.ntiles = sd.tiles_x * sd.tiles_y;
    sd.mode = mode; sd.precision = prec;
    sd.max_iters = g->opts.max_iters; sd.num_cg = g->opts.num_cg; sd.num_dlsm = g->opts.num_dlsm;
    sd.hybrid_budget = g->opts.hybrid_budget;
    sd.keep_dir_after_dlsm = g->opts.keep_dir_after_dlsm ? 1 : 0;
    sd.dlsm_stall_limit = g->opts.dlsm_stall_limit;
    sd.dlsm_cost = g->opts.dlsm_cost_iters;
    sd.tol = tol;
    sd.ru_delta = prec == PPE_PREC_MIXED ? g->opts.inner_rtol : 0.0;
    sd.dlsm_guard = g->opts.dlsm_guard;
    sd.diag_max = g->diag_max;
    sd.n_cells = (double)g->nx * (double)g->ny;
    sd.inv_n = 1.0 / sd.n_cells;
    sd.n_cells_f = (float)sd.n_cells;
    sd.inv_n_f = (float)sd.inv_n;
    sd.dx = g->dx; sd.dy = g->dy; sd.fx = g->fx; sd.fy = g->fy;
    sd.dx32 = g->dx32; sd.dy32 = g->dy32; sd.fx32 = g->fx32; sd.fy32 = g->fy32;
    sd.f = rhs; sd.x = x;
    sd.r[0] = g->r[0]; sd.r[1] = g->r[1]; sd.p[0] = g->p[0]; sd.p[1] = g->p[1];
    sd.d = g->d; sd.e = g->e;
    sd.tmaps = g->tmaps_dev + (int)v * NMAPS;
    return sd;
}

static void fill_info(ppe_solve_info *info, const SysState &s, double ms, double ms_net, int launches)
{
    if (!info) return;
    std::memset(info, 0, sizeof(*info));
    info->status = s.status;
    info->iters_pcg = s.it_pcg;
    info->iters_dlsm = s.it_dlsm;
    info->dlsm_skipped = s.dlsm_skipped;
    info->refinements = s.refinements;
    info->fell_back = s.fell_back;
    info->net_calls = s.net_calls;
    info->launches = launches;
    info->rel_res_true = s.relres;
    info->incompat = s.incompat;
    info->ms_total = ms;
    info->ms_net = ms_net;
}

// Split the tiles of n systems into contiguous block ranges (at most SMAX
// systems per block, at most max_blocks blocks) and assign the partial-sum
// slots of every system.
static bool plan_blocks(std::vector<SysDesc> &sds, int max_blocks, std::vector<BlockRange> &ranges, int &nslots)
{
    int total = 0;
    for (auto &d : sds) total += d.ntiles;
    std::vector<int> sys_of(total);
    for (size_t s = 0; s < sds.size(); ++s)
        for (int t = 0; t < sds[s].ntiles; ++t) sys_of[sds[s].tile0 + t] = (int)s;
    for (int chunk = std::max(1, (total + max_blocks - 1) / max_blocks);; ++chunk) {
        ranges.clear();
        int t = 0;
        while (t < total) {
            BlockRange r;
            r.t0 = t;
            r.s0 = sys_of[t];
            int e = t;
            while (e < total && e - t < chunk && sys_of[e] - r.s0 < SMAX) ++e;
            r.t1 = e;
            r.s1 = sys_of[e - 1];
            ranges.push_back(r);
            t = e;
        }
        if ((int)ranges.size() <= max_blocks) break;
        if (chunk > total) return false;
    }
    nslots = 0;
    for (size_t s = 0; s < sds.size(); ++s) {
        int first = -1, last = -1;
        for (size_t b = 0; b < ranges.size(); ++b)
            if ((int)s >= ranges[b].s0 && (int)s <= ranges[b].s1) {
                if (first < 0) first = (int)b;
                last = (int)b;
            }
        sds[s].blk0 = first;
        sds[s].nparts = last - first + 1;
        sds[s].part0 = nslots;
        nslots += sds[s].nparts;
    }
    return true;
}

// Drive the persistent launches of n systems until every one is done; run
// the network between launches for the systems that wait for a direction.
// Rebalancing of a batch: launches end every max_steps steps; when the tiles
// of the systems still running have dropped below a fraction of the planned
// ones, the host spreads them over all blocks again (finished systems get no
// tiles).  Systems of very different iteration counts otherwise leave most
// SMs idle at the end of a batch.
struct Replan {
    std::vector<SysDesc> *sds;      // host copy of the descriptions (updated in place)
    std::vector<int> full_tiles;    // tiles of each system
    int max_blocks = 0, slot_cap = 0, max_steps = 0;
    double fraction = 0.75;
};

static ppe_status drive(int n, ppe_grid *const *grids, SysDesc *sys_dev, SysState *st_dev, BlockRange *ranges_dev,
                        int blocks, Slot *slots_dev, int nslots, Control *ctl_dev, SolverVariant variant,
                        ppe_net *net, cudaStream_t stream, ppe_solve_info *info, Replan *rp = nullptr)
{
    const bool fp64 = variant == SV_FP64;
    SolverArgs a;
    a.sys = sys_dev; a.st = st_dev; a.ranges = ranges_dev; a.slots = slots_dev; a.nslots = nslots; a.ctl = ctl_dev;
    a.max_steps = rp ? rp->max_steps : 0;
    a.pad_ = 0;
    int planned_tiles = 0;
    if (rp)
        for (int s = 0; s < n; ++s) planned_tiles += (*rp->sds)[s].ntiles;
    a.arrive = nullptr;
    PPE_CUDA_TRY(cudaMallocAsync((void **)&a.arrive, sizeof(uint32_t) * n, stream));
    a.nsys = n; a.ntiles = 0;
    a.spin_limit_ns = (int64_t)g_spin_limit_ms * 1000000LL;
    a.prof = nullptr;
    static const bool want_prof = std::getenv("PPE_SOLVER_PROFILE") != nullptr;
    if (want_prof) {
        PPE_CUDA_TRY(cudaMalloc(&a.prof, 8 * sizeof(unsigned long long)));
        PPE_CUDA_TRY(cudaMemsetAsync(a.prof, 0, 8 * sizeof(unsigned long long), stream));
    }

    cudaEvent_t ev0, ev1;
    PPE_CUDA_TRY(cudaEventCreate(&ev0));
    PPE_CUDA_TRY(cudaEventCreate(&ev1));
    PPE_CUDA_TRY(cudaEventRecord(ev0, stream));
    PPE_CUDA_TRY(cudaMemsetAsync(st_dev, 0, sizeof(SysState) * n, stream));
    int launches = 0;
    double ms_net = 0.0;
    ppe_status status = PPE_OK;
    Control ctl_host;
    std::vector<SysState> st(n);
    int active = n;
    for (int round = 0;; ++round) {
        std::memset(&ctl_host, 0, sizeof ctl_host);
        ctl_host.active0 = active;
        PPE_CUDA_TRY(cudaMemcpyAsync(ctl_dev, &ctl_host, sizeof(Control), cudaMemcpyHostToDevice, stream));
        PPE_CUDA_TRY(cudaMemsetAsync(a.arrive, 0, sizeof(uint32_t) * n, stream));
        status = launch_solver_resume(a, variant, blocks, stream, round > 0 ? 1 : 0);
        if (status != PPE_OK) break;
        ++launches;
        PPE_CUDA_TRY(cudaMemcpyAsync(st.data(), st_dev, sizeof(SysState) * n, cudaMemcpyDeviceToHost, stream));
        PPE_CUDA_TRY(cudaMemcpyAsync(&ctl_host, ctl_dev, sizeof(Control), cudaMemcpyDeviceToHost, stream));
        PPE_CUDA_TRY(cudaStreamSynchronize(stream));
        if (ctl_host.err) {
            set_error("solver kernel: bounded grid-barrier wait expired");
            status = (ppe_status)ctl_host.err;
            break;
        }
        active = 0;
        int live = 0, live_tiles = 0;
        for (int s = 0; s < n; ++s) {
            active += st[s].phase == PH_NET;
            if (st[s].phase != PH_DONE) {
                ++live;
                if (rp) live_tiles += rp->full_tiles[s];
            }
        }
        if (!live) break;
        if (!active) {
            // the launch ended on its step budget
            if (!rp) { status = PPE_ERR_CUDA; set_error("solver kernel left with systems running"); break; }
            if (live_tiles < rp->fraction * planned_tiles) {
                std::vector<SysDesc> &sds = *rp->sds;
                int t0 = 0;
                for (int s = 0; s < n; ++s) {
                    sds[s].ntiles = st[s].phase != PH_DONE ? rp->full_tiles[s] : 0;
                    sds[s].tile0 = t0;
                    t0 += sds[s].ntiles;
                }
                std::vector<BlockRange> ranges;
                int ns = 0;
                if (plan_blocks(sds, std::min(rp->max_blocks, t0), ranges, ns) && ns <= rp->slot_cap) {
                    PPE_CUDA_TRY(cudaMemcpyAsync(sys_dev, sds.data(), sizeof(SysDesc) * n, cudaMemcpyHostToDevice,
                                                 stream));
                    PPE_CUDA_TRY(cudaMemcpyAsync(ranges_dev, ranges.data(), sizeof(BlockRange) * ranges.size(),
                                                 cudaMemcpyHostToDevice, stream));
                    blocks = (int)ranges.size();     // a.nslots (the bank stride) stays the capacity
                    planned_tiles = t0;
                }
            }
            continue;
        }
        float t = 0.f;
        for (int s = 0; s < n; ++s) {
            if (st[s].phase != PH_NET) continue;
            ppe_grid *g = grids[s];
            if (g->dir_fn) {
                const int nb = (int)std::min<size_t>(1184, ((size_t)g->nx * g->ny + 255) / 256);
                rhat_kernel<<<nb, 256, 0, stream>>>(sys_dev + s, st_dev + s, g->dir_r);
                g->dir_fn(g->dir_user, g->dir_r, g->dir_e, g->nx, g->ny, (void *)stream);
                pitch_copy_kernel<<<nb, 256, 0, stream>>>(g->dir_e, g->e, g->nx, g->ny, g->pitch);
                cudaError_t ce = cudaGetLastError();
                if (ce != cudaSuccess) { status = cuda_status(ce, "direction source"); break; }
                status = center_direction(g, stream);
                if (status != PPE_OK) break;
                continue;
            }
            if (!net) { set_error("hybrid solve without a network or direction source"); status = PPE_ERR_NO_NET; break; }
            ppe_status ns = net_direction(net, g, sys_dev + s, st_dev + s, fp64, stream, &t);
            if (ns != PPE_OK) { status = ns; break; }
            ms_net += t;
        }
        if (status != PPE_OK) break;
        if (launches > 10000000) { status = PPE_ERR_NOT_CONVERGED; break; }
    }
    if (a.prof) {
        unsigned long long pr[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        cudaMemcpyAsync(pr, a.prof, sizeof pr, cudaMemcpyDeviceToHost, stream);
        cudaStreamSynchronize(stream);
        double st_ = pr[7] ? (double)pr[7] * 1e3 : 1.0;
        std::fprintf(stderr, "[solver profile] blocks=%d steps=%llu  per step (us): pass %.2f, reduce+publish %.2f, "
                     "wait %.2f, gather %.2f, advance %.2f (state machine %.2f)\n", blocks, pr[7], pr[0] / st_,
                     pr[1] / st_, pr[2] / st_, pr[3] / st_, pr[4] / st_, pr[5] / st_);
        cudaFree(a.prof);
    }
    cudaFreeAsync(a.arrive, stream);
    float ms = 0.f;
    cudaEventRecord(ev1, stream);
    cudaEventSynchronize(ev1);
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (status != PPE_OK) return status;
    ppe_status worst = PPE_OK;
    for (int s = 0; s < n; ++s) {
        fill_info(info ? info + s : nullptr, st[s], ms, ms_net, launches);
        if (st[s].status != PPE_OK && worst == PPE_OK) worst = (ppe_status)st[s].status;
    }
    if (worst != PPE_OK) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "solve finished with status %d (relres %.3e)", (int)worst, st[0].relres);
        set_error(buf);
    }
    return worst;
}

// Kernel variant of a launch.  FP64 has one; in mixed precision the
// streaming iteration pass pays off once the grid has a few tiles per block.
// Measured on GB300 (per iteration, tile-cooperative / streaming): 896^2 =
// 392 tiles 18.7 / 21.9 us, 1024^2 = 512 tiles 21.4 / 18.3 us, 2048 x 1024 =
// 1024 tiles 33.1 / 22.0 us; on grids of a few hundred tiles or fewer the
// tile-cooperative pass has the lower latency (512^2: 8.1 / 17.3 us).
// ppe_autotune measures instead of guessing.
constexpr int STREAM_MIN_TILES = 448;
static SolverVariant pick_variant(ppe_precision prec, int iter_pass, int ntiles)
{
    if (prec == PPE_PREC_FP64) return SV_FP64;
    if (iter_pass == 1) return SV_FP32_TILE;
    if (iter_pass == 2) return SV_FP32_STREAM;
    return ntiles >= STREAM_MIN_TILES ? SV_FP32_STREAM : SV_FP32_TILE;
}

static ppe_status check_solve_args(ppe_grid *g, const double *rhs, double *x, double tol, ppe_mode mode,
                                   ppe_precision prec, ppe_net *net)
{
    if (!g || !rhs || !x) return arg_error("ppe_solve: NULL grid, rhs or x");
    if (!(tol > 0.0) || !std::isfinite(tol)) return arg_error("ppe_solve: tol_rel must be positive");
    if (mode != PPE_MODE_PCG && mode != PPE_MODE_HYBRID) return arg_error("ppe_solve: bad mode");
    if (prec != PPE_PREC_FP64 && prec != PPE_PREC_MIXED) return arg_error("ppe_solve: bad precision");
    if (mode == PPE_MODE_HYBRID && g->dir_fn) return PPE_OK;
    if (mode == PPE_MODE_HYBRID && !net) {
        set_error("ppe_solve: hybrid mode needs a network or a direction source");
        return PPE_ERR_NO_NET;
    }
    if (mode == PPE_MODE_HYBRID) return net_check_grid(net, g);
    return PPE_OK;
}

}  // namespace ppe

extern "C" {

ppe_status ppe_solve(ppe_grid *g, const double *rhs, double *x, double tol, ppe_mode mode, ppe_precision prec,
                     ppe_net *net, void *stream, ppe_solve_info *info)
{
    clear_error();
    PPE_TRY(check_solve_args(g, rhs, x, tol, mode, prec, net));
    cudaStream_t st = (cudaStream_t)stream;
    int pass = g->opts.iter_pass, bps = g->opts.blocks_per_sm;
    if (prec == PPE_PREC_MIXED && pass == 0) {
        if (g->tuned_pass) {
            pass = g->tuned_pass;
            bps = g->tuned_bps;
        } else {
            tune_lookup(g->nx, g->ny, &pass, &bps);
        }
    }
    const SolverVariant v = pick_variant(prec, pass, g->tiles_x * g->tiles_y);
    std::vector<SysDesc> sds(1, make_desc(g, rhs, x, tol, mode, prec, 0, v));
    int maxb = std::min(solver_max_blocks(v, bps), sds[0].ntiles);
    if (maxb < 1) return cuda_status(cudaErrorInvalidConfiguration, "solver occupancy");
    std::vector<BlockRange> ranges;
    int nslots = 0;
    if (!plan_blocks(sds, maxb, ranges, nslots)) return arg_error("ppe_solve: cannot partition tiles");
    PPE_CUDA_TRY(cudaMemcpyAsync(g->sys_dev, sds.data(), sizeof(SysDesc), cudaMemcpyHostToDevice, st));
    PPE_CUDA_TRY(cudaMemcpyAsync(g->ranges_dev, ranges.data(), sizeof(BlockRange) * ranges.size(),
                                 cudaMemcpyHostToDevice, st));
    ppe_grid *gs[1] = {g};
    return drive(1, gs, g->sys_dev, g->st_dev, g->ranges_dev, (int)ranges.size(), g->slots_dev, nslots, g->ctl_dev,
                 v, net, st, info);
}

ppe_status ppe_solve_batch(int n, ppe_grid *const *grids, const double *const *rhs, double *const *x, double tol,
                           ppe_mode mode, ppe_precision prec, ppe_net *net, void *stream, ppe_solve_info *info)
{
    clear_error();
    if (n < 1 || !grids || !rhs || !x) return arg_error("ppe_solve_batch: bad arguments");
    for (int i = 0; i < n; ++i) PPE_TRY(check_solve_args(grids[i], rhs[i], x[i], tol, mode, prec, net));
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < i; ++k)
            if (grids[i] == grids[k]) return arg_error("ppe_solve_batch: a grid handle may appear only once");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<SysDesc> sds(n);
    int ntiles = 0;
    for (int i = 0; i < n; ++i) ntiles += grids[i]->tiles_x * grids[i]->tiles_y;
    const SolverVariant v = pick_variant(prec, grids[0]->opts.iter_pass, ntiles);
    ntiles = 0;
    Replan rp;
    rp.sds = &sds;
    for (int i = 0; i < n; ++i) {
        sds[i] = make_desc(grids[i], rhs[i], x[i], tol, mode, prec, ntiles, v);
        ntiles += sds[i].ntiles;
        rp.full_tiles.push_back(sds[i].ntiles);
    }
    const int maxb_all = solver_max_blocks(v, grids[0]->opts.blocks_per_sm);
    int maxb = std::min(maxb_all, ntiles);
    std::vector<BlockRange> ranges;
    int nslots = 0;
    if (maxb < 1 || !plan_blocks(sds, maxb, ranges, nslots)) return arg_error("ppe_solve_batch: cannot partition");
    rp.max_blocks = maxb_all;
    rp.slot_cap = maxb_all + n + 1;          // parts of any plan: at most one per block plus one per system
    rp.max_steps = n > 1 ? 400 : 0;
    nslots = std::max(nslots, rp.slot_cap);
    SysDesc *sys_dev = nullptr;
    SysState *st_dev = nullptr;
    BlockRange *rg_dev = nullptr;
    Slot *part_dev = nullptr;
    Control *ctl_dev = nullptr;
    auto cleanup = [&]() {
        cudaFree(sys_dev); cudaFree(st_dev); cudaFree(rg_dev); cudaFree(part_dev); cudaFree(ctl_dev);
    };
    if (cudaMalloc(&sys_dev, sizeof(SysDesc) * n) != cudaSuccess || cudaMalloc(&st_dev, sizeof(SysState) * n) != cudaSuccess ||
        cudaMalloc(&rg_dev, sizeof(BlockRange) * std::max<size_t>(ranges.size(), (size_t)maxb_all)) != cudaSuccess ||
        cudaMalloc(&part_dev, sizeof(Slot) * 2 * (size_t)nslots) != cudaSuccess ||
        cudaMalloc(&ctl_dev, sizeof(Control)) != cudaSuccess) {
        cleanup();
        set_error("ppe_solve_batch: device allocation failed");
        return PPE_ERR_NOMEM;
    }
    cudaMemcpyAsync(sys_dev, sds.data(), sizeof(SysDesc) * n, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(rg_dev, ranges.data(), sizeof(BlockRange) * ranges.size(), cudaMemcpyHostToDevice, st);
    ppe_status status = drive(n, grids, sys_dev, st_dev, rg_dev, (int)ranges.size(), part_dev, nslots, ctl_dev, v, net,
                              st, info, rp.max_steps > 0 ? &rp : nullptr);
    cudaStreamSynchronize(st);
    cleanup();
    return status;
}

}  // extern "C"
