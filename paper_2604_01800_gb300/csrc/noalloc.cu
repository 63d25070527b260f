// Allocation-free PCG solve for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a host application whose device
// memory is entirely reserved up front by its own pool allocator (so a
// library allocation would fail or fragment it), a long-running loop that
// must not allocate after initialisation (allocation latency or failure in
// the middle of a time step is unacceptable), or a plugin whose host forbids
// plugins from allocating device memory.  For them ppe_solve_noalloc runs the
// same persistent solver kernel as ppe_solve, with every piece of scratch it
// needs (grid coefficients, inner vectors, partial-sum records, solver state)
// placed in one file-scope __device__ array of fixed size.  The caller passes
// only the grid widths, the source and the solution buffer.
//
// Limits: nx, ny <= 4096 and nx*ny <= 65536 cells, plain PCG.  Every GPU that
// loads the library holds the array (about 3.3 MB) until the process exits.
// All calls share the array and it keeps the last call's contents: each call
// clears what must start at zero, and calls whose work overlaps on the GPU
// race with each other.  The first call on a device looks the array's device
// address up (cudaGetSymbolAddress, with that device current); make that
// first call before any stream capture (a lookup that fails is retried by
// the next call).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace ppe {

namespace {

constexpr int NA_MAX_CELLS = 65536;
constexpr int NA_MAX_DIM = 4096;
constexpr int NA_MAX_BLOCKS = 1024;
// Rows are padded to a multiple of 4 elements (16 bytes in FP32, as the TMA
// unit requires); the padded vectors hold at most this many elements.
constexpr int NA_PITCH_ALIGN = 4;
constexpr size_t NA_MAX_PADDED = (size_t)NA_MAX_CELLS + (size_t)(NA_PITCH_ALIGN - 1) * NA_MAX_DIM;

// byte layout of the scratch array (every part 256-byte aligned)
constexpr size_t al(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t OFF_DESC = 0;
constexpr size_t OFF_STATE = OFF_DESC + al(sizeof(SysDesc));
constexpr size_t OFF_CTL = OFF_STATE + al(sizeof(SysState));
constexpr size_t OFF_ARRIVE = OFF_CTL + al(sizeof(Control));
constexpr size_t OFF_RANGES = OFF_ARRIVE + al(sizeof(uint32_t));
constexpr size_t OFF_SLOTS = OFF_RANGES + al(sizeof(BlockRange) * NA_MAX_BLOCKS);
constexpr size_t OFF_DX = OFF_SLOTS + al(sizeof(Slot) * 2 * (NA_MAX_BLOCKS + 1));
constexpr size_t OFF_DY = OFF_DX + al(8 * NA_MAX_DIM);
constexpr size_t OFF_FX = OFF_DY + al(8 * NA_MAX_DIM);
constexpr size_t OFF_FY = OFF_FX + al(8 * (NA_MAX_DIM + 1));
constexpr size_t OFF_DX32 = OFF_FY + al(8 * (NA_MAX_DIM + 1));
constexpr size_t OFF_DY32 = OFF_DX32 + al(4 * NA_MAX_DIM);
constexpr size_t OFF_FX32 = OFF_DY32 + al(4 * NA_MAX_DIM);
constexpr size_t OFF_FY32 = OFF_FX32 + al(4 * (NA_MAX_DIM + 1));
constexpr size_t OFF_MAPS = OFF_FY32 + al(4 * (NA_MAX_DIM + 1));
constexpr size_t OFF_VEC = OFF_MAPS + al(sizeof(CUtensorMap) * NMAPS);
constexpr size_t VEC_BYTES = al(8 * NA_MAX_PADDED);
constexpr size_t SCRATCH_BYTES = OFF_VEC + 5 * VEC_BYTES;

// The scratch.  In host code this name is only a stand-in symbol, never a
// device address: host code must use the address cudaGetSymbolAddress returns.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

// Face coefficients 2/(w_left + w_right) (0 at the walls) and FP32 copies.
__global__ void na_coeff_kernel(int n, const double *w, double *f, float *w32, float *f32)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= n; k += gridDim.x * blockDim.x) {
        double v = (k > 0 && k < n) ? 2.0 / (w[k - 1] + w[k]) : 0.0;
        f[k] = v;
        f32[k] = (float)v;
        if (k < n) w32[k] = (float)w[k];
    }
}

// Device address of the scratch array on the current device, looked up with
// that device current.  Only a successful lookup is kept: a failed one (for
// example a first call made during a stream capture) is retried by the next
// call instead of disabling the entry point for the rest of the process.
std::mutex g_base_mu;
unsigned char *g_base[MAX_DEVICES] = {};

unsigned char *scratch_base(int dev, cudaError_t *err)
{
    if (dev < 0 || dev >= MAX_DEVICES) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_base_mu);
    if (!g_base[dev]) {
        void *p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (*err != cudaSuccess) return nullptr;
        g_base[dev] = (unsigned char *)p;
    }
    *err = cudaSuccess;
    return g_base[dev];
}

}  // namespace
}  // namespace ppe

using namespace ppe;

extern "C" ppe_status ppe_solve_noalloc(int nx, int ny, const double *dx, const double *dy, const double *rhs_dev,
                                        double *x_dev, double tol_rel, ppe_precision precision, void *stream,
                                        ppe_solve_info *info)
{
    clear_error();
    char msg[200];
    if (nx < 1 || ny < 1 || nx > NA_MAX_DIM || ny > NA_MAX_DIM || (long)nx * ny > NA_MAX_CELLS) {
        std::snprintf(msg, sizeof msg,
                      "ppe_solve_noalloc: grid %d x %d exceeds the fixed scratch (nx, ny <= %d and nx*ny <= %d)", nx,
                      ny, NA_MAX_DIM, NA_MAX_CELLS);
        set_error(msg);
        return PPE_ERR_ARG;
    }
    if (!dx || !dy || !rhs_dev || !x_dev || !(tol_rel > 0.0) || !std::isfinite(tol_rel) ||
        (precision != PPE_PREC_FP64 && precision != PPE_PREC_MIXED)) {
        set_error("ppe_solve_noalloc: bad argument");
        return PPE_ERR_ARG;
    }
    for (int i = 0; i < nx; ++i)
        if (!(dx[i] > 0.0) || !std::isfinite(dx[i])) { set_error("ppe_solve_noalloc: dx must be positive"); return PPE_ERR_ARG; }
    for (int j = 0; j < ny; ++j)
        if (!(dy[j] > 0.0) || !std::isfinite(dy[j])) { set_error("ppe_solve_noalloc: dy must be positive"); return PPE_ERR_ARG; }

    int dev = 0;
    PPE_CUDA_TRY(cudaGetDevice(&dev));
    cudaError_t e;
    unsigned char *base = scratch_base(dev, &e);
    if (!base) return cuda_status(e, "cudaGetSymbolAddress(no-alloc scratch)");
    cudaStream_t st = (cudaStream_t)stream;

    double *d_dx = (double *)(base + OFF_DX), *d_dy = (double *)(base + OFF_DY);
    double *d_fx = (double *)(base + OFF_FX), *d_fy = (double *)(base + OFF_FY);
    float *d_dx32 = (float *)(base + OFF_DX32), *d_dy32 = (float *)(base + OFF_DY32);
    float *d_fx32 = (float *)(base + OFF_FX32), *d_fy32 = (float *)(base + OFF_FY32);
    PPE_CUDA_TRY(cudaMemcpyAsync(d_dx, dx, 8 * (size_t)nx, cudaMemcpyHostToDevice, st));
    PPE_CUDA_TRY(cudaMemcpyAsync(d_dy, dy, 8 * (size_t)ny, cudaMemcpyHostToDevice, st));
    na_coeff_kernel<<<(nx + 256) / 256, 256, 0, st>>>(nx, d_dx, d_fx, d_dx32, d_fx32);
    na_coeff_kernel<<<(ny + 256) / 256, 256, 0, st>>>(ny, d_dy, d_fy, d_dy32, d_fy32);
    PPE_CUDA_TRY(cudaGetLastError());

    // one system, contiguous tile ranges
    const bool fp64 = precision == PPE_PREC_FP64;
    const int tiles_x = (nx + TILE_X - 1) / TILE_X, tiles_y = (ny + TILE_Y - 1) / TILE_Y;
    const int ntiles = tiles_x * tiles_y;
    const SolverVariant v = fp64 ? SV_FP64 : SV_FP32_TILE;
    int maxb = solver_max_blocks(v, 1);
    if (maxb < 1) return cuda_status(cudaErrorInvalidConfiguration, "solver occupancy");
    if (maxb > NA_MAX_BLOCKS) maxb = NA_MAX_BLOCKS;
    const int chunk = (ntiles + maxb - 1) / maxb;
    const int blocks = (ntiles + chunk - 1) / chunk;
    BlockRange ranges[NA_MAX_BLOCKS];
    for (int b = 0; b < blocks; ++b) {
        ranges[b].t0 = b * chunk;
        ranges[b].t1 = std::min(ntiles, (b + 1) * chunk);
        ranges[b].s0 = ranges[b].s1 = 0;
    }

    ppe_solve_opts opts;
    ppe_default_options(&opts);
    SysDesc sd;
    std::memset(&sd, 0, sizeof sd);
    const int pitch = round_up(nx, NA_PITCH_ALIGN);
    sd.nx = nx; sd.ny = ny; sd.pitch = pitch; sd.tiles_x = tiles_x; sd.tiles_y = tiles_y; sd.tile0 = 0;
    sd.ntiles = ntiles;
    sd.mode = PPE_MODE_PCG; sd.precision = precision;
    sd.max_iters = opts.max_iters; sd.num_cg = opts.num_cg; sd.num_dlsm = opts.num_dlsm;
    sd.hybrid_budget = opts.hybrid_budget;
    sd.part0 = 0; sd.blk0 = 0; sd.nparts = blocks;
    sd.tol = tol_rel;
    sd.ru_delta = fp64 ? 0.0 : opts.inner_rtol;
    sd.dlsm_guard = opts.dlsm_guard;
    sd.diag_max = 0.0;
    sd.n_cells = (double)nx * ny;
    sd.inv_n = 1.0 / sd.n_cells;
    sd.n_cells_f = (float)sd.n_cells;
    sd.inv_n_f = (float)sd.inv_n;
    sd.dx = d_dx; sd.dy = d_dy; sd.fx = d_fx; sd.fy = d_fy;
    sd.dx32 = d_dx32; sd.dy32 = d_dy32; sd.fx32 = d_fx32; sd.fy32 = d_fy32;
    sd.f = rhs_dev; sd.x = x_dev;
    unsigned char *vec = base + OFF_VEC;
    sd.r[0] = vec; sd.r[1] = vec + VEC_BYTES; sd.p[0] = vec + 2 * VEC_BYTES; sd.p[1] = vec + 3 * VEC_BYTES;
    sd.d = vec + 4 * VEC_BYTES; sd.e = nullptr;
    CUtensorMap maps[NMAPS];
    PPE_TRY(encode_solver_maps(sd.r, sd.p, sd.d, nullptr, nx, ny, pitch, v, maps));
    CUtensorMap *d_maps = (CUtensorMap *)(base + OFF_MAPS);
    sd.tmaps = d_maps;

    SysDesc *d_sd = (SysDesc *)(base + OFF_DESC);
    SysState *d_st = (SysState *)(base + OFF_STATE);
    Control *d_ctl = (Control *)(base + OFF_CTL);
    uint32_t *d_arrive = (uint32_t *)(base + OFF_ARRIVE);
    BlockRange *d_ranges = (BlockRange *)(base + OFF_RANGES);
    Slot *d_slots = (Slot *)(base + OFF_SLOTS);
    PPE_CUDA_TRY(cudaMemcpyAsync(d_sd, &sd, sizeof sd, cudaMemcpyHostToDevice, st));
    PPE_CUDA_TRY(cudaMemcpyAsync(d_maps, maps, sizeof maps, cudaMemcpyHostToDevice, st));
    PPE_CUDA_TRY(cudaMemcpyAsync(d_ranges, ranges, sizeof(BlockRange) * blocks, cudaMemcpyHostToDevice, st));
    // what must start at zero: state (phase INIT), control block, arrival counter
    PPE_CUDA_TRY(cudaMemsetAsync(d_st, 0, sizeof(SysState), st));
    PPE_CUDA_TRY(cudaMemsetAsync(d_ctl, 0, sizeof(Control), st));
    PPE_CUDA_TRY(cudaMemsetAsync(d_arrive, 0, sizeof(uint32_t), st));
    PPE_TRY(launch_scale(d_sd, d_st, 1, (long)nx * ny, st));

    SolverArgs a;
    std::memset(&a, 0, sizeof a);
    a.sys = d_sd; a.st = d_st; a.ranges = d_ranges; a.slots = d_slots; a.nslots = blocks; a.ctl = d_ctl;
    a.arrive = d_arrive; a.nsys = 1; a.ntiles = ntiles; a.spin_limit_ns = 2000000000LL; a.prof = nullptr;
    PPE_TRY(launch_solver_resume(a, v, blocks, st, 0));

    SysState s;
    Control c;
    PPE_CUDA_TRY(cudaMemcpyAsync(&s, d_st, sizeof s, cudaMemcpyDeviceToHost, st));
    PPE_CUDA_TRY(cudaMemcpyAsync(&c, d_ctl, sizeof c, cudaMemcpyDeviceToHost, st));
    PPE_CUDA_TRY(cudaStreamSynchronize(st));
    if (c.err) {
        set_error("ppe_solve_noalloc: bounded grid wait expired");
        return (ppe_status)c.err;
    }
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->status = s.status;
        info->iters_pcg = s.it_pcg;
        info->refinements = s.refinements;
        info->launches = 1;
        info->rel_res_true = s.relres;
        info->incompat = s.incompat;
    }
    if (s.status != PPE_OK) {
        std::snprintf(msg, sizeof msg, "ppe_solve_noalloc: solve finished with status %d (relres %.3e)", s.status,
                      s.relres);
        set_error(msg);
    }
    return (ppe_status)s.status;
}
