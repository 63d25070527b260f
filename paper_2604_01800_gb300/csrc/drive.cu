// Solve drivers: segments of the persistent solver kernel, the network
// directions between them (Sec. 2.2's alternation of CG-type iterations and
// DLSM steps), and batches of independent systems.
//
// Default path: a whole solve -- one system or a batch, plain PCG or hybrid
// -- is one CUDA graph launch.  The graph holds
//   * an initialisation kernel (states, barrier counters, control block), and
//   * a conditional WHILE node whose body runs
//       - one solver segment: the cooperative persistent kernel, until every
//         system is done or waits for a network direction (or, in a batch, a
//         step budget ends the segment);
//       - a one-block decision kernel that reads the systems' phases on the
//         device and sets the conditions of the loop and of the branches;
//       - per system of a hybrid solve, a conditional IF node whose body is
//         that system's network forward pass and direction mean removal.
// The decision kernel also re-plans the tile ranges of a batch over the
// systems still running (the same planner the host uses).  The host launches
// the graph and reads the reports back once: there is no host round-trip per
// hybrid cycle.  Graphs are built once per launch set (grid or batch plan)
// and rebuilt only when the kernel variant, the launch shape, the network or
// its parameter version change.
//
// Host loop (opts.host_loop = 1, a user direction source, or the solver's
// step profile): the host launches each segment, reads the states back and
// runs the directions in between.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "net_iface.h"

namespace ppe {

namespace {

constexpr int DRIVE_THREADS = 256;
constexpr int LOOP_CAP = 4000000;       // segments per solve before the loop gives up
constexpr float REPLAN_FRACTION = 0.75f;
constexpr int BATCH_STEP_BUDGET = 400;

// ---------------------------------------------------------------------------
// device side of the loop
// ---------------------------------------------------------------------------

// States to zero (phase PH_INIT), barrier counters, control block, loop counters.
__global__ void __launch_bounds__(DRIVE_THREADS) drive_init_kernel(SysState *st, uint32_t *arrive, Control *ctl,
                                                                   DriveCtl *dc)
{
    const int n = dc->n;
    int32_t *w = reinterpret_cast<int32_t *>(st);
    const int nw = n * (int)(sizeof(SysState) / 4);
    for (int k = threadIdx.x; k < nw; k += blockDim.x) w[k] = 0;
    for (int s = threadIdx.x; s < n; s += blockDim.x) arrive[s] = 0;
    if (threadIdx.x == 0) {
        ctl->arrive = 0;
        ctl->err = 0;
        ctl->active0 = n;
        ctl->retired[0] = ctl->retired[1] = 0;
        dc->launches = 0;
        dc->err = 0;
    }
}

// After a segment: count it, stop on a bounded-wait error or the segment cap,
// end the loop when every system is done, re-plan a batch whose running
// systems hold few of the planned tiles, reset the barrier for the next
// segment, and open the network branches of the systems waiting for a
// direction.
__global__ void __launch_bounds__(DRIVE_THREADS)
    drive_decide_kernel(SysDesc *sys, const SysState *st, BlockRange *ranges, BlockRange *ranges_tmp,
                        uint32_t *arrive, Control *ctl, DriveCtl *dc, const int32_t *full_tiles,
                        int32_t *scratch, const cudaGraphConditionalHandle *if_h, cudaGraphConditionalHandle while_h)
{
    __shared__ int cont;
    const int n = dc->n;
    if (threadIdx.x == 0) {
        int c = 1;
        dc->launches++;
        if (ctl->err) {
            dc->err = ctl->err;
            c = 0;
        } else {
            int live = 0, active = 0, live_tiles = 0;
            for (int s = 0; s < n; ++s) {
                const int ph = st[s].phase;
                active += ph == PH_NET;
                if (ph != PH_DONE) {
                    ++live;
                    live_tiles += full_tiles[s];
                }
            }
            if (!live) {
                c = 0;
            } else if (dc->launches >= dc->loop_cap) {
                dc->err = PPE_ERR_NOT_CONVERGED;
                c = 0;
            } else if (!active && dc->max_steps > 0 && (float)live_tiles < dc->fraction * (float)dc->planned_tiles) {
                // the segment ended on its step budget: spread the running
                // systems' tiles over every block again (finished systems get none)
                int32_t *nt = scratch, *t0 = nt + n, *b0 = t0 + n, *np = b0 + n, *p0 = np + n;
                for (int s = 0; s < n; ++s) nt[s] = st[s].phase != PH_DONE ? full_tiles[s] : 0;
                int ns = 0;
                const int nr = plan_ranges(n, nt, dc->max_blocks, t0, b0, np, p0, ranges_tmp, dc->max_blocks, &ns);
                if (nr > 0 && ns <= dc->slot_cap) {
                    for (int s = 0; s < n; ++s) {
                        sys[s].ntiles = nt[s];
                        sys[s].tile0 = t0[s];
                        sys[s].blk0 = b0[s];
                        sys[s].nparts = np[s];
                        sys[s].part0 = p0[s];
                    }
                    for (int b = 0; b < dc->max_blocks; ++b) {
                        if (b < nr) {
                            ranges[b] = ranges_tmp[b];
                        } else {
                            ranges[b].t0 = ranges[b].t1 = 0;   // idle block: no systems
                            ranges[b].s0 = 1;
                            ranges[b].s1 = 0;
                        }
                    }
                    dc->planned_tiles = live_tiles;
                }
            }
        }
        if (c) {
            ctl->arrive = 0;
            ctl->active0 = n;
            ctl->retired[0] = ctl->retired[1] = 0;
        }
        cont = c;
    }
    __syncthreads();
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        if (cont) arrive[s] = 0;
        if (dc->with_net) cudaGraphSetConditional(if_h[s], (cont && st[s].phase == PH_NET) ? 1u : 0u);
    }
    if (threadIdx.x == 0) cudaGraphSetConditional(while_h, cont ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------

ppe_status arg_error(const std::string &msg)
{
    set_error(msg);
    return PPE_ERR_ARG;
}

SysDesc make_desc(const ppe_grid *g, const double *rhs, double *x, double tol, ppe_mode mode, ppe_precision prec,
                  int tile0, SolverVariant v)
{
    SysDesc sd;
    std::memset(&sd, 0, sizeof(sd));
    const int tw = solver_tile_w(v), th = solver_tile_h(v);
    sd.nx = g->nx; sd.ny = g->ny; sd.pitch = g->pitch;
    sd.tiles_x = (g->nx + tw - 1) / tw; sd.tiles_y = (g->ny + th - 1) / th;
    sd.tile0 = tile0; sd.ntiles = sd.tiles_x * sd.tiles_y;
    sd.mode = mode; sd.precision = prec;
    sd.max_iters = g->opts.max_iters; sd.num_cg = g->opts.num_cg; sd.num_dlsm = g->opts.num_dlsm;
    sd.hybrid_budget = g->opts.hybrid_budget;
    sd.keep_dir_after_dlsm = g->opts.keep_dir_after_dlsm ? 1 : 0;
    sd.dlsm_stall_limit = g->opts.dlsm_stall_limit;
    sd.dlsm_cost = g->opts.dlsm_cost_iters;
    sd.force_stall = g->opts.debug_force_stall ? 1 : 0;
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

void fill_info(ppe_solve_info *info, const SysState &s, double ms, int launches, int drive)
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
    info->ms_net = (double)s.ns_net * 1e-6;
    info->ms_pcg = (double)s.ns_pcg * 1e-6;
    info->ms_dlsm = (double)s.ns_dlsm * 1e-6;
    info->ms_refine = (double)s.ns_fp64 * 1e-6;
    info->drive = drive;
    info->precision_fallback = s.prec_stalled;
}

// A mixed solve whose FP32 inner iteration stalled, continued in FP64 from its
// iterate: the report of both parts together.
void merge_fallback(ppe_solve_info &fp64, const ppe_solve_info &mixed)
{
    fp64.iters_pcg += mixed.iters_pcg;
    fp64.iters_dlsm += mixed.iters_dlsm;
    fp64.dlsm_skipped += mixed.dlsm_skipped;
    fp64.refinements += mixed.refinements;
    fp64.fell_back |= mixed.fell_back;
    fp64.net_calls += mixed.net_calls;
    fp64.launches += mixed.launches;
    fp64.incompat = mixed.incompat;
    fp64.ms_total += mixed.ms_total;
    fp64.ms_net += mixed.ms_net;
    fp64.ms_pcg += mixed.ms_pcg;
    fp64.ms_dlsm += mixed.ms_dlsm;
    fp64.ms_refine += mixed.ms_refine;
    fp64.precision_fallback = 1;
}

// Kernel variant of a launch.  FP64 has one; in mixed precision the
// streaming iteration pass pays off once the grid has a few tiles per block.
// Measured on GB300 (per iteration, tile-cooperative / streaming): 896^2 =
// 392 tiles 18.7 / 21.9 us, 1024^2 = 512 tiles 21.4 / 18.3 us, 2048 x 1024 =
// 1024 tiles 33.1 / 22.0 us; on grids of a few hundred tiles or fewer the
// tile-cooperative pass has the lower latency (512^2: 8.1 / 17.3 us).
// ppe_autotune measures instead of guessing.
//
// ntiles counts 128x16 tiles.  Small grids take shorter tiles, one per
// block on two or four times the blocks: the per-block work of a step
// shrinks while its synchronisation grows with the number of records.
// Measured on GB300 (us per iteration, 16 / 8 / 4 rows): 256^2 (32 tiles of
// 16 rows) mixed 7.25 / 6.35 / 6.68, FP64 35.5 / 26.0 / 22.3; 64^2 (4 tiles)
// mixed 7.38 / 6.68 / 6.26, FP64 35.4 / 25.8 / 21.5.  FP64 passes are long,
// so FP64 takes the shortest tiles that still fit one per SM; FP32 takes 4
// rows only while the blocks stay few (16 ntiles <= SMs), else 8 rows while
// they fit (2 ntiles <= SMs).
constexpr int STREAM_MIN_TILES = 448;
SolverVariant pick_variant_for(ppe_precision prec, int iter_pass, int ntiles, int tile_rows, int sms)
{
    const bool fp64 = prec == PPE_PREC_FP64;
    int rows = tile_rows;
    if (!rows) {
        if (fp64)
            rows = 4 * ntiles <= sms ? TILE_Y_R4 : 2 * ntiles <= sms ? TILE_Y_R8 : TILE_Y;
        else
            rows = 16 * ntiles <= sms ? TILE_Y_R4 : 2 * ntiles <= sms ? TILE_Y_R8 : TILE_Y;
    }
    const SolverVariant v64 = rows == TILE_Y_R4 ? SV_FP64_R4 : rows == TILE_Y_R8 ? SV_FP64_R8 : SV_FP64;
    const SolverVariant v32 = rows == TILE_Y_R4 ? SV_FP32_R4 : rows == TILE_Y_R8 ? SV_FP32_R8 : SV_FP32_TILE;
    if (fp64) return v64;
    if (iter_pass == 2) return SV_FP32_STREAM;
    if (iter_pass == 1 || ntiles < STREAM_MIN_TILES) return v32;
    return SV_FP32_STREAM;
}

SolverVariant pick_variant(ppe_precision prec, int iter_pass, int ntiles, int tile_rows)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return pick_variant_for(prec, iter_pass, ntiles, tile_rows, sms);
}

ppe_status check_solve_args(ppe_grid *g, const double *rhs, double *x, double tol, ppe_mode mode,
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

int64_t spin_ns(const ppe_solve_opts &o)
{
    return (int64_t)(o.spin_limit_ms > 0 ? o.spin_limit_ms : 2000) * 1000000LL;
}

// r_hat = (r - mu) / sqrt(rho) of a system's current residual, unpitched FP32
// (input of a user direction source).
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

// The reports of a finished drive: per-system infos, worst status.
ppe_status finish(int n, const std::vector<SysState> &st, double ms, int launches, int drive, ppe_solve_info *info)
{
    ppe_status worst = PPE_OK;
    for (int s = 0; s < n; ++s) {
        fill_info(info ? info + s : nullptr, st[s], ms, launches, drive);
        if (st[s].status != PPE_OK && worst == PPE_OK) worst = (ppe_status)st[s].status;
    }
    if (worst != PPE_OK) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "solve finished with status %d (relres %.3e)", (int)worst, st[0].relres);
        set_error(buf);
    }
    return worst;
}

// Host-side rebalancing of a batch in the host loop (same rule as the
// decision kernel's).
struct Replan {
    std::vector<SysDesc> *sds;
    std::vector<int32_t> full_tiles;
    int max_blocks = 0, slot_cap = 0, max_steps = 0;
};

// ---------------------------------------------------------------------------
// host loop
// ---------------------------------------------------------------------------

ppe_status drive_host(int n, ppe_grid *const *grids, LaunchSet &ls, int blocks, int nslots, SolverVariant variant,
                      ppe_net *net, const ppe_solve_opts &opts, cudaStream_t stream, ppe_solve_info *info,
                      Replan *rp)
{
    const bool fp64 = solver_variant_fp64(variant);
    SolverArgs a;
    std::memset(&a, 0, sizeof a);
    a.sys = ls.sys; a.st = ls.st; a.ranges = ls.ranges; a.slots = ls.slots; a.nslots = nslots; a.ctl = ls.ctl;
    a.arrive = ls.arrive;
    a.max_steps = rp ? rp->max_steps : 0;
    a.skip_block = opts.debug_skip_block;
    a.nsys = n; a.ntiles = 0;
    a.spin_limit_ns = spin_ns(opts);
    int planned_tiles = 0;
    if (rp)
        for (int s = 0; s < n; ++s) planned_tiles += (*rp->sds)[s].ntiles;
    static const bool want_prof = std::getenv("PPE_SOLVER_PROFILE") != nullptr;
    if (want_prof) {
        PPE_CUDA_TRY(cudaMalloc(&a.prof, 16 * sizeof(unsigned long long)));
        PPE_CUDA_TRY(cudaMemsetAsync(a.prof, 0, 16 * sizeof(unsigned long long), stream));
    }
    PPE_CUDA_TRY(cudaEventRecord(ls.ev0, stream));
    PPE_CUDA_TRY(cudaMemsetAsync(ls.st, 0, sizeof(SysState) * n, stream));
    {
        long max_cells = 0;
        for (int s = 0; s < n; ++s) max_cells = std::max<long>(max_cells, (long)grids[s]->nx * grids[s]->ny);
        PPE_TRY(launch_scale(ls.sys, ls.st, n, max_cells, stream));
    }
    int launches = 0;
    ppe_status status = PPE_OK;
    Control ctl_host;
    std::vector<SysState> st(n);
    for (int round = 0;; ++round) {
        std::memset(&ctl_host, 0, sizeof ctl_host);
        ctl_host.active0 = n;
        PPE_CUDA_TRY(cudaMemcpyAsync(ls.ctl, &ctl_host, sizeof(Control), cudaMemcpyHostToDevice, stream));
        PPE_CUDA_TRY(cudaMemsetAsync(ls.arrive, 0, sizeof(uint32_t) * n, stream));
        status = launch_solver_resume(a, variant, blocks, stream, round > 0 ? 1 : 0);
        if (status != PPE_OK) break;
        ++launches;
        PPE_CUDA_TRY(cudaMemcpyAsync(st.data(), ls.st, sizeof(SysState) * n, cudaMemcpyDeviceToHost, stream));
        PPE_CUDA_TRY(cudaMemcpyAsync(&ctl_host, ls.ctl, sizeof(Control), cudaMemcpyDeviceToHost, stream));
        PPE_CUDA_TRY(cudaStreamSynchronize(stream));
        if (ctl_host.err) {
            set_error("solver kernel: bounded grid-barrier wait expired");
            status = (ppe_status)ctl_host.err;
            break;
        }
        int active = 0, live = 0, live_tiles = 0;
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
            if (live_tiles < REPLAN_FRACTION * planned_tiles) {
                std::vector<SysDesc> &sds = *rp->sds;
                std::vector<int32_t> nt(n), t0(n), b0(n), np(n), p0(n);
                for (int s = 0; s < n; ++s) nt[s] = st[s].phase != PH_DONE ? rp->full_tiles[s] : 0;
                std::vector<BlockRange> ranges(rp->max_blocks);
                int ns = 0;
                const int nr = plan_ranges(n, nt.data(), rp->max_blocks, t0.data(), b0.data(), np.data(), p0.data(),
                                           ranges.data(), rp->max_blocks, &ns);
                if (nr > 0 && ns <= rp->slot_cap) {
                    for (int s = 0; s < n; ++s) {
                        sds[s].ntiles = nt[s]; sds[s].tile0 = t0[s]; sds[s].blk0 = b0[s];
                        sds[s].nparts = np[s]; sds[s].part0 = p0[s];
                    }
                    PPE_CUDA_TRY(cudaMemcpyAsync(ls.sys, sds.data(), sizeof(SysDesc) * n, cudaMemcpyHostToDevice,
                                                 stream));
                    PPE_CUDA_TRY(cudaMemcpyAsync(ls.ranges, ranges.data(), sizeof(BlockRange) * nr,
                                                 cudaMemcpyHostToDevice, stream));
                    blocks = nr;     // a.nslots (the bank stride) stays the capacity
                    planned_tiles = live_tiles;
                }
            }
            continue;
        }
        for (int s = 0; s < n; ++s) {
            if (st[s].phase != PH_NET) continue;
            ppe_grid *g = grids[s];
            if (g->dir_fn) {
                const int nb = (int)std::min<size_t>(1184, ((size_t)g->nx * g->ny + 255) / 256);
                rhat_kernel<<<nb, 256, 0, stream>>>(ls.sys + s, ls.st + s, g->dir_r);
                g->dir_fn(g->dir_user, g->dir_r, g->dir_e, g->nx, g->ny, (void *)stream);
                pitch_copy_kernel<<<nb, 256, 0, stream>>>(g->dir_e, g->e, g->nx, g->ny, g->pitch);
                cudaError_t ce = cudaGetLastError();
                if (ce != cudaSuccess) { status = cuda_status(ce, "direction source"); break; }
                status = center_direction(g, stream);
                if (status != PPE_OK) break;
                continue;
            }
            if (!net) { set_error("hybrid solve without a network or direction source"); status = PPE_ERR_NO_NET; break; }
            float t = 0.f;
            ppe_status ns = net_direction(net, g, ls.sys + s, ls.st + s, fp64, stream, &t);
            if (ns != PPE_OK) { status = ns; break; }
        }
        if (status != PPE_OK) break;
        if (launches > LOOP_CAP) { status = PPE_ERR_NOT_CONVERGED; break; }
    }
    if (a.prof) {
        unsigned long long pr[16] = {};
        cudaMemcpyAsync(pr, a.prof, sizeof pr, cudaMemcpyDeviceToHost, stream);
        cudaStreamSynchronize(stream);
        double st_ = pr[7] ? (double)pr[7] * 1e3 : 1.0, si_ = pr[13] ? (double)pr[13] * 1e3 : 1.0;
        std::fprintf(stderr, "[solver profile] blocks=%d steps=%llu  per step (us): pass %.2f, reduce+publish %.2f, "
                     "wait %.2f, gather %.2f, advance %.2f (state machine %.2f)\n", blocks, pr[7], pr[0] / st_,
                     pr[1] / st_, pr[2] / st_, pr[3] / st_, pr[4] / st_, pr[5] / st_);
        std::fprintf(stderr, "[solver profile] iteration passes=%llu  per pass (us): to the data wait %.2f, data wait "
                     "%.2f, window stage %.2f, ring stage %.2f, tile stage and sums %.2f (to the pass %.2f, "
                     "issuing its loads %.2f)\n", pr[13], pr[8] / si_, pr[9] / si_, pr[10] / si_, pr[11] / si_,
                     pr[12] / si_, pr[14] / si_, pr[15] / si_);
        cudaFree(a.prof);
    }
    float ms = 0.f;
    cudaEventRecord(ls.ev1, stream);
    cudaEventSynchronize(ls.ev1);
    cudaEventElapsedTime(&ms, ls.ev0, ls.ev1);
    if (status != PPE_OK) return status;
    return finish(n, st, ms, launches, 1, info);
}

// ---------------------------------------------------------------------------
// graph path
// ---------------------------------------------------------------------------

uint64_t direction_key(const ppe_net *net, ppe_grid *const *grids, int n)
{
    uint64_t h = 0xcbf29ce484222325ull;
    for (int s = 0; s < n; ++s) h = (h ^ net_direction_key(net, grids[s])) * 0x100000001b3ull;
    return h;
}

void destroy_graph(LaunchSet &ls)
{
    if (ls.exec) cudaGraphExecDestroy(ls.exec);
    if (ls.graph) cudaGraphDestroy(ls.graph);
    ls.exec = nullptr;
    ls.graph = nullptr;
    ls.built_variant = -1;
}

// Build the solve graph of a launch set (see the file comment).
ppe_status build_graph(LaunchSet &ls, const SolverArgs &args_in, SolverVariant v, int blocks, int n,
                       ppe_grid *const *grids, ppe_net *net, bool with_net, cudaStream_t stream)
{
    destroy_graph(ls);
    set_solver_attributes();
    if (with_net)
        for (int s = 0; s < n; ++s) PPE_TRY(net_prepare_direction(net, grids[s], stream));
    if (!ls.cap) PPE_CUDA_TRY(cudaStreamCreateWithFlags(&ls.cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    PPE_CUDA_TRY(cudaGraphCreate(&g, 0));
    auto fail = [&](cudaError_t e, const char *what) {
        cudaGraphDestroy(g);
        return cuda_status(e, what);
    };
    cudaError_t e;
    cudaGraphConditionalHandle wh;
    if ((e = cudaGraphConditionalHandleCreate(&wh, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
        return fail(e, "cudaGraphConditionalHandleCreate(loop)");
    // initialisation
    cudaGraphNode_t init_node, while_node, solver_node, decide_node;
    {
        void *p[] = {&ls.st, &ls.arrive, &ls.ctl, &ls.dc};
        cudaKernelNodeParams kp = {};
        kp.func = (void *)drive_init_kernel;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(DRIVE_THREADS);
        kp.kernelParams = p;
        if ((e = cudaGraphAddKernelNode(&init_node, g, nullptr, 0, &kp)) != cudaSuccess)
            return fail(e, "cudaGraphAddKernelNode(init)");
    }
    // the power-of-two scale of every system (max |b|)
    cudaGraphNode_t scale_node;
    {
        long max_cells = 0;
        for (int s = 0; s < n; ++s) max_cells = std::max<long>(max_cells, (long)grids[s]->nx * grids[s]->ny);
        int nn = n;
        void *p[] = {&ls.sys, &ls.st, &nn};
        cudaKernelNodeParams kp = {};
        kp.func = const_cast<void *>(scale_kernel_fn());
        kp.gridDim = scale_grid(n, max_cells);
        kp.blockDim = dim3(256);
        kp.kernelParams = p;
        if ((e = cudaGraphAddKernelNode(&scale_node, g, &init_node, 1, &kp)) != cudaSuccess)
            return fail(e, "cudaGraphAddKernelNode(scale)");
    }
    // the loop
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = wh;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    if ((e = cudaGraphAddNode(&while_node, g, &scale_node, nullptr, 1, &wp)) != cudaSuccess)
        return fail(e, "cudaGraphAddNode(loop)");
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    // solver segment: the cooperative persistent kernel, resuming systems that
    // waited for a direction
    {
        SolverArgs args = args_in;
        int resume = 1;
        void *p[] = {&args, &resume};
        cudaKernelNodeParams kp = {};
        kp.func = const_cast<void *>(solver_kernel_fn(v));
        kp.gridDim = dim3(blocks);
        kp.blockDim = dim3(SOLVER_THREADS);
        kp.sharedMemBytes = (unsigned)solver_smem_bytes(v);
        kp.kernelParams = p;
        if ((e = cudaGraphAddKernelNode(&solver_node, body, nullptr, 0, &kp)) != cudaSuccess)
            return fail(e, "cudaGraphAddKernelNode(solver)");
        cudaLaunchAttributeValue av;
        std::memset(&av, 0, sizeof av);
        av.cooperative = 1;
        if ((e = cudaGraphKernelNodeSetAttribute(solver_node, cudaLaunchAttributeCooperative, &av)) != cudaSuccess)
            return fail(e, "cudaGraphKernelNodeSetAttribute(cooperative)");
    }
    {
        void *p[] = {&ls.sys, &ls.st, &ls.ranges, &ls.ranges_tmp, &ls.arrive, &ls.ctl, &ls.dc, &ls.full_tiles,
                     &ls.plan_scratch, &ls.if_handles, &wh};
        cudaKernelNodeParams kp = {};
        kp.func = (void *)drive_decide_kernel;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(DRIVE_THREADS);
        kp.kernelParams = p;
        if ((e = cudaGraphAddKernelNode(&decide_node, body, &solver_node, 1, &kp)) != cudaSuccess)
            return fail(e, "cudaGraphAddKernelNode(decide)");
    }
    // network branches, one per system, side by side
    if (with_net) {
        std::vector<cudaGraphConditionalHandle> hs(n);
        for (int s = 0; s < n; ++s) {
            if ((e = cudaGraphConditionalHandleCreate(&hs[s], body, 0, 0)) != cudaSuccess)
                return fail(e, "cudaGraphConditionalHandleCreate(branch)");
            cudaGraphNodeParams ip = {};
            ip.type = cudaGraphNodeTypeConditional;
            ip.conditional.handle = hs[s];
            ip.conditional.type = cudaGraphCondTypeIf;
            ip.conditional.size = 1;
            cudaGraphNode_t if_node;
            if ((e = cudaGraphAddNode(&if_node, body, &decide_node, nullptr, 1, &ip)) != cudaSuccess)
                return fail(e, "cudaGraphAddNode(branch)");
            cudaGraph_t ib = ip.conditional.phGraph_out[0];
            if ((e = cudaStreamBeginCaptureToGraph(ls.cap, ib, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
                cudaSuccess)
                return fail(e, "cudaStreamBeginCaptureToGraph(branch)");
            ppe_status rs = net_record_direction(net, grids[s], ls.sys + s, ls.st + s, ls.cap);
            cudaGraph_t got = nullptr;
            e = cudaStreamEndCapture(ls.cap, &got);
            if (rs != PPE_OK) {
                cudaGraphDestroy(g);
                return rs;
            }
            if (e != cudaSuccess) return fail(e, "cudaStreamEndCapture(branch)");
        }
        if ((e = cudaMemcpy(ls.if_handles, hs.data(), sizeof(cudaGraphConditionalHandle) * n,
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail(e, "cudaMemcpy(branch handles)");
    }
    cudaGraphExec_t ex = nullptr;
    if ((e = cudaGraphInstantiate(&ex, g, 0)) != cudaSuccess) return fail(e, "cudaGraphInstantiate(solve)");
    ls.graph = g;
    ls.exec = ex;
    ls.built_args = args_in;
    ls.built_variant = (int)v;
    ls.built_blocks = blocks;
    ls.built_with_net = with_net ? 1 : 0;
    ls.built_net = with_net ? (const void *)net : nullptr;
    ls.built_version = with_net ? direction_key(net, grids, n) : 0;
    return PPE_OK;
}

// One solve (or batch) as one graph launch.  ranges: the initial plan
// (nr ranges; the launch runs `blocks` blocks, the rest idle).
ppe_status drive_graph(int n, ppe_grid *const *grids, LaunchSet &ls, const std::vector<SysDesc> &sds,
                       const std::vector<BlockRange> &ranges, int blocks, int nslots, const std::vector<int32_t> &full,
                       int max_steps, SolverVariant variant, ppe_net *net, bool with_net, const ppe_solve_opts &opts,
                       cudaStream_t stream, ppe_solve_info *info)
{
    SolverArgs a;
    std::memset(&a, 0, sizeof a);
    a.sys = ls.sys; a.st = ls.st; a.ranges = ls.ranges; a.slots = ls.slots; a.nslots = nslots; a.ctl = ls.ctl;
    a.arrive = ls.arrive; a.nsys = n; a.ntiles = 0; a.spin_limit_ns = spin_ns(opts); a.max_steps = max_steps;
    a.skip_block = opts.debug_skip_block; a.prof = nullptr;
    if (with_net)
        for (int s = 0; s < n; ++s) PPE_TRY(net_prepare_direction(net, grids[s], stream));
    const bool same = ls.exec && ls.built_variant == (int)variant && ls.built_blocks == blocks &&
                      ls.built_with_net == (with_net ? 1 : 0) && std::memcmp(&ls.built_args, &a, sizeof a) == 0 &&
                      (!with_net || (ls.built_net == (const void *)net &&
                                     ls.built_version == direction_key(net, grids, n)));
    if (!same) PPE_TRY(build_graph(ls, a, variant, blocks, n, grids, net, with_net, stream));

    std::vector<BlockRange> rg(blocks);
    for (int b = 0; b < blocks; ++b) {
        if (b < (int)ranges.size()) {
            rg[b] = ranges[b];
        } else {
            rg[b].t0 = rg[b].t1 = 0;
            rg[b].s0 = 1;
            rg[b].s1 = 0;
        }
    }
    DriveCtl dch;
    std::memset(&dch, 0, sizeof dch);
    dch.n = n;
    dch.max_blocks = blocks;
    dch.slot_cap = nslots;
    dch.max_steps = max_steps;
    int planned = 0;
    for (int s = 0; s < n; ++s) planned += sds[s].ntiles;
    dch.planned_tiles = planned;
    dch.loop_cap = LOOP_CAP;
    dch.fraction = REPLAN_FRACTION;
    dch.with_net = with_net ? 1 : 0;
    PPE_CUDA_TRY(cudaMemcpyAsync(ls.sys, sds.data(), sizeof(SysDesc) * n, cudaMemcpyHostToDevice, stream));
    PPE_CUDA_TRY(cudaMemcpyAsync(ls.ranges, rg.data(), sizeof(BlockRange) * blocks, cudaMemcpyHostToDevice, stream));
    PPE_CUDA_TRY(cudaMemcpyAsync(ls.full_tiles, full.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, stream));
    PPE_CUDA_TRY(cudaMemcpyAsync(ls.dc, &dch, sizeof dch, cudaMemcpyHostToDevice, stream));
    PPE_CUDA_TRY(cudaEventRecord(ls.ev0, stream));
    PPE_CUDA_TRY(cudaGraphLaunch(ls.exec, stream));
    PPE_CUDA_TRY(cudaEventRecord(ls.ev1, stream));
    std::vector<SysState> st(n);
    PPE_CUDA_TRY(cudaMemcpyAsync(st.data(), ls.st, sizeof(SysState) * n, cudaMemcpyDeviceToHost, stream));
    PPE_CUDA_TRY(cudaMemcpyAsync(&dch, ls.dc, sizeof dch, cudaMemcpyDeviceToHost, stream));
    PPE_CUDA_TRY(cudaStreamSynchronize(stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ls.ev0, ls.ev1);
    if (dch.err == PPE_ERR_TIMEOUT) {
        set_error("solver kernel: bounded grid-barrier wait expired");
        return PPE_ERR_TIMEOUT;
    }
    if (dch.err) {
        set_error("solve loop stopped after its segment cap");
        return (ppe_status)dch.err;
    }
    return finish(n, st, ms, dch.launches, 0, info);
}

// Cached resources of batches, keyed by the grids' creation numbers.
struct BatchPlan {
    std::vector<uint64_t> ids;
    int device = 0, variant = -1, max_blocks = 0;
    LaunchSet *ls = nullptr;
};
std::mutex g_batch_mu;
std::vector<BatchPlan> g_batch_cache;   // most recent last
constexpr size_t BATCH_CACHE = 2;

}  // namespace

ppe_status launch_set_create(int n, int max_ranges, int slot_cap, LaunchSet **out)
{
    *out = nullptr;
    LaunchSet *ls = new LaunchSet();
    ls->n = n;
    ls->max_ranges = max_ranges;
    ls->slot_cap = slot_cap;
    cudaGetDevice(&ls->device);
    auto fail = [&](cudaError_t e, const char *what) {
        launch_set_destroy(ls);
        return cuda_status(e, what);
    };
    cudaError_t e;
#define LS_ALLOC(ptr, bytes)                                                                       \
    if ((e = cudaMalloc((void **)&(ptr), (bytes))) != cudaSuccess) return fail(e, "cudaMalloc(launch set)")
    LS_ALLOC(ls->sys, sizeof(SysDesc) * n);
    LS_ALLOC(ls->st, sizeof(SysState) * n);
    LS_ALLOC(ls->ranges, sizeof(BlockRange) * max_ranges);
    LS_ALLOC(ls->ranges_tmp, sizeof(BlockRange) * max_ranges);
    LS_ALLOC(ls->slots, sizeof(Slot) * 2 * (size_t)slot_cap);
    LS_ALLOC(ls->ctl, sizeof(Control));
    LS_ALLOC(ls->arrive, sizeof(uint32_t) * n);
    LS_ALLOC(ls->dc, sizeof(DriveCtl));
    LS_ALLOC(ls->full_tiles, sizeof(int32_t) * n);
    LS_ALLOC(ls->plan_scratch, sizeof(int32_t) * 5 * n);
    LS_ALLOC(ls->if_handles, sizeof(cudaGraphConditionalHandle) * n);
#undef LS_ALLOC
    if ((e = cudaEventCreate(&ls->ev0)) != cudaSuccess) return fail(e, "cudaEventCreate");
    if ((e = cudaEventCreate(&ls->ev1)) != cudaSuccess) return fail(e, "cudaEventCreate");
    *out = ls;
    return PPE_OK;
}

void launch_set_destroy(LaunchSet *ls)
{
    if (!ls) return;
    destroy_graph(*ls);
    if (ls->cap) cudaStreamDestroy(ls->cap);
    if (ls->ev0) cudaEventDestroy(ls->ev0);
    if (ls->ev1) cudaEventDestroy(ls->ev1);
    cudaFree(ls->sys); cudaFree(ls->st); cudaFree(ls->ranges); cudaFree(ls->ranges_tmp); cudaFree(ls->slots);
    cudaFree(ls->ctl); cudaFree(ls->arrive); cudaFree(ls->dc); cudaFree(ls->full_tiles); cudaFree(ls->plan_scratch);
    cudaFree(ls->if_handles);
    delete ls;
}

}  // namespace ppe

using namespace ppe;

namespace {

ppe_status solve_single(ppe_grid *g, const double *rhs, double *x, double tol, ppe_mode mode, ppe_precision prec,
                        ppe_net *net, cudaStream_t st, ppe_solve_info *info)
{
    int pass = g->opts.iter_pass, bps = g->opts.blocks_per_sm, rows = g->opts.tile_rows;
    if (prec == PPE_PREC_MIXED && pass == 0) {
        // the autotuner's choice: pass, CTAs per SM and (unless the options
        // fix it) the tile height
        int tuned_rows = 0;
        if (g->tuned_pass) {
            pass = g->tuned_pass;
            bps = g->tuned_bps;
            tuned_rows = g->tuned_rows;
        } else {
            tune_lookup(g->nx, g->ny, &pass, &bps, &tuned_rows);
        }
        if (!rows) rows = tuned_rows;
    }
    const SolverVariant v = pick_variant(prec, pass, g->tiles_x * g->tiles_y, rows);
    std::vector<SysDesc> sds(1, make_desc(g, rhs, x, tol, mode, prec, 0, v));
    const int maxb = std::min(solver_max_blocks(v, bps), sds[0].ntiles);
    if (maxb < 1) return cuda_status(cudaErrorInvalidConfiguration, "solver occupancy");
    LaunchSet &ls = *g->ls;
    std::vector<BlockRange> ranges(ls.max_ranges);
    int nslots = 0;
    std::vector<int32_t> nt(1, sds[0].ntiles), full(nt);
    int32_t t0, b0, np, p0;
    const int nr = plan_ranges(1, nt.data(), maxb, &t0, &b0, &np, &p0, ranges.data(), ls.max_ranges, &nslots);
    if (nr < 1) return arg_error("ppe_solve: cannot partition tiles");
    ranges.resize(nr);
    sds[0].tile0 = t0; sds[0].blk0 = b0; sds[0].nparts = np; sds[0].part0 = p0;
    ppe_grid *gs[1] = {g};
    static const bool want_prof = std::getenv("PPE_SOLVER_PROFILE") != nullptr;
    const bool with_net = mode == PPE_MODE_HYBRID;
    if (g->opts.host_loop || g->dir_fn || want_prof) {
        PPE_CUDA_TRY(cudaMemcpyAsync(ls.sys, sds.data(), sizeof(SysDesc), cudaMemcpyHostToDevice, st));
        PPE_CUDA_TRY(cudaMemcpyAsync(ls.ranges, ranges.data(), sizeof(BlockRange) * nr, cudaMemcpyHostToDevice, st));
        return drive_host(1, gs, ls, nr, nslots, v, net, g->opts, st, info, nullptr);
    }
    return drive_graph(1, gs, ls, sds, ranges, nr, ls.slot_cap, full, 0, v, net, with_net, g->opts, st, info);
}

}  // namespace

extern "C" {

ppe_status ppe_solve(ppe_grid *g, const double *rhs, double *x, double tol, ppe_mode mode, ppe_precision prec,
                     ppe_net *net, void *stream, ppe_solve_info *info)
{
    clear_error();
    PPE_TRY(check_solve_args(g, rhs, x, tol, mode, prec, net));
    cudaStream_t st = (cudaStream_t)stream;
    if (g->opts.preconditioner == 1) {
        // the multigrid partner (plain PCG, FP32 inner with FP64 refinement)
        if (mode != PPE_MODE_PCG || prec != PPE_PREC_MIXED)
            return arg_error("ppe_solve: the multigrid partner runs PPE_MODE_PCG in PPE_PREC_MIXED");
        return mg_solve(g, rhs, x, tol, st, info);
    }
    ppe_solve_info a;
    std::memset(&a, 0, sizeof a);
    ppe_status status = solve_single(g, rhs, x, tol, mode, prec, net, st, &a);
    if (status == PPE_ERR_NOT_CONVERGED && a.precision_fallback) {
        // the FP32 inner iteration stalled: continue in FP64 from the iterate
        clear_error();
        ppe_solve_info b;
        std::memset(&b, 0, sizeof b);
        status = solve_single(g, rhs, x, tol, mode, PPE_PREC_FP64, net, st, &b);
        merge_fallback(b, a);
        a = b;
    }
    if (info) *info = a;
    return status;
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
    for (int i = 0; i < n; ++i)
        if (grids[i]->opts.preconditioner != 0)
            return arg_error("ppe_solve_batch: batches run the Jacobi partner (preconditioner 0)");
    cudaStream_t st = (cudaStream_t)stream;
    int ntiles = 0;
    for (int i = 0; i < n; ++i) ntiles += grids[i]->tiles_x * grids[i]->tiles_y;
    // One kernel serves every system: the first grid's options choose it; in
    // mixed precision with the pass left to the library, an autotuned choice
    // (pass and tile height) shared by every system's shape is taken, else the
    // batch's total tile count decides.
    int pass = grids[0]->opts.iter_pass, rows = grids[0]->opts.tile_rows;
    if (prec == PPE_PREC_MIXED && pass == 0) {
        int p0 = -1, r0 = -1;
        bool same = true;
        for (int i = 0; i < n && same; ++i) {
            int p = 0, b = 0, r = 0;
            if (grids[i]->tuned_pass) {
                p = grids[i]->tuned_pass;
                r = grids[i]->tuned_rows;
            } else if (!tune_lookup(grids[i]->nx, grids[i]->ny, &p, &b, &r)) {
                same = false;
                break;
            }
            if (p0 < 0) {
                p0 = p;
                r0 = r;
            }
            same = p == p0 && r == r0;
        }
        if (same && p0 > 0) {
            pass = p0;
            if (!rows) rows = r0;
        }
    }
    const SolverVariant v = pick_variant(prec, pass, ntiles, rows);
    std::vector<SysDesc> sds(n);
    std::vector<int32_t> full(n);
    for (int i = 0; i < n; ++i) {
        sds[i] = make_desc(grids[i], rhs[i], x[i], tol, mode, prec, 0, v);
        full[i] = sds[i].ntiles;
    }
    const int maxb_all = solver_max_blocks(v, grids[0]->opts.blocks_per_sm);
    if (maxb_all < 1) return cuda_status(cudaErrorInvalidConfiguration, "solver occupancy");
    const int slot_cap = maxb_all + n + 1;   // records of any plan: at most one per block plus one per system
    // the batch's launch set (cached for the same grids on this device)
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<uint64_t> ids(n);
    for (int i = 0; i < n; ++i) ids[i] = grids[i]->id;
    std::unique_lock<std::mutex> lk(g_batch_mu);
    LaunchSet *ls = nullptr;
    for (size_t k = 0; k < g_batch_cache.size(); ++k) {
        BatchPlan &bp = g_batch_cache[k];
        if (bp.ids == ids && bp.device == dev && bp.max_blocks == maxb_all) {
            BatchPlan keep = bp;
            g_batch_cache.erase(g_batch_cache.begin() + k);
            g_batch_cache.push_back(keep);
            ls = keep.ls;
            break;
        }
    }
    if (!ls) {
        PPE_TRY(launch_set_create(n, maxb_all, slot_cap, &ls));
        if (g_batch_cache.size() >= BATCH_CACHE) {
            launch_set_destroy(g_batch_cache.front().ls);
            g_batch_cache.erase(g_batch_cache.begin());
        }
        BatchPlan bp;
        bp.ids = ids;
        bp.device = dev;
        bp.max_blocks = maxb_all;
        bp.ls = ls;
        g_batch_cache.push_back(bp);
    }
    std::vector<int32_t> t0(n), b0(n), np(n), p0(n);
    std::vector<BlockRange> ranges(maxb_all);
    int nslots = 0;
    const int nr = plan_ranges(n, full.data(), std::min(maxb_all, ntiles), t0.data(), b0.data(), np.data(),
                               p0.data(), ranges.data(), maxb_all, &nslots);
    if (nr < 1 || nslots > slot_cap) return arg_error("ppe_solve_batch: cannot partition");
    ranges.resize(nr);
    for (int i = 0; i < n; ++i) {
        sds[i].tile0 = t0[i]; sds[i].blk0 = b0[i]; sds[i].nparts = np[i]; sds[i].part0 = p0[i];
    }
    const int max_steps = n > 1 ? BATCH_STEP_BUDGET : 0;
    const ppe_solve_opts &opts = grids[0]->opts;
    bool any_dir_fn = false;
    for (int i = 0; i < n; ++i) any_dir_fn |= grids[i]->dir_fn != nullptr;
    static const bool want_prof = std::getenv("PPE_SOLVER_PROFILE") != nullptr;
    std::vector<ppe_solve_info> rep(n);
    ppe_status status;
    if (opts.host_loop || any_dir_fn || want_prof) {
        Replan rp;
        rp.sds = &sds;
        rp.full_tiles = full;
        rp.max_blocks = maxb_all;
        rp.slot_cap = slot_cap;
        rp.max_steps = max_steps;
        PPE_CUDA_TRY(cudaMemcpyAsync(ls->sys, sds.data(), sizeof(SysDesc) * n, cudaMemcpyHostToDevice, st));
        PPE_CUDA_TRY(cudaMemcpyAsync(ls->ranges, ranges.data(), sizeof(BlockRange) * nr, cudaMemcpyHostToDevice, st));
        status = drive_host(n, grids, *ls, nr, slot_cap, v, net, opts, st, rep.data(), max_steps > 0 ? &rp : nullptr);
    } else {
        // a batch that re-plans launches every block (idle ones leave at once)
        const int blocks = max_steps > 0 ? maxb_all : nr;
        status = drive_graph(n, grids, *ls, sds, ranges, blocks, slot_cap, full, max_steps, v, net,
                             mode == PPE_MODE_HYBRID, opts, st, rep.data());
    }
    lk.unlock();
    if (status == PPE_OK || status == PPE_ERR_NOT_CONVERGED) {
        // systems whose FP32 inner iteration stalled continue in FP64, one by one
        bool any = false;
        for (int i = 0; i < n; ++i) {
            if (!rep[i].precision_fallback) continue;
            ppe_solve_info b;
            std::memset(&b, 0, sizeof b);
            solve_single(grids[i], rhs[i], x[i], tol, mode, PPE_PREC_FP64, net, st, &b);
            merge_fallback(b, rep[i]);
            rep[i] = b;
            any = true;
        }
        if (any) {
            status = PPE_OK;
            clear_error();
            for (int i = 0; i < n && status == PPE_OK; ++i)
                if (rep[i].status != PPE_OK) {
                    status = (ppe_status)rep[i].status;
                    set_error("ppe_solve_batch: a system finished with status " + std::to_string(status));
                }
        }
    }
    if (info) std::memcpy(info, rep.data(), sizeof(ppe_solve_info) * n);
    return status;
}

ppe_status ppe_debug_pick_variant(int precision, int iter_pass, int ntiles, int tile_rows, int sms, int *pass_out,
                                  int *rows_out)
{
    clear_error();
    if ((precision != PPE_PREC_FP64 && precision != PPE_PREC_MIXED) || iter_pass < 0 || iter_pass > 2 || ntiles < 1 ||
        sms < 1 || (tile_rows != 0 && tile_rows != TILE_Y && tile_rows != TILE_Y_R8 && tile_rows != TILE_Y_R4)) {
        set_error("ppe_debug_pick_variant: argument out of range");
        return PPE_ERR_ARG;
    }
    const SolverVariant v = pick_variant_for((ppe_precision)precision, iter_pass, ntiles, tile_rows, sms);
    if (pass_out) *pass_out = v == SV_FP32_STREAM ? 2 : 1;
    if (rows_out) *rows_out = solver_tile_h(v);
    return PPE_OK;
}

ppe_status ppe_debug_plan_ranges(int n, const int32_t *ntiles, int max_blocks, int max_ranges, int32_t *tile0,
                                 int32_t *blk0, int32_t *nparts, int32_t *part0, int32_t *ranges, int *nranges,
                                 int *nslots)
{
    clear_error();
    if (n < 1 || !ntiles || max_ranges < 1 || !tile0 || !blk0 || !nparts || !part0 || !ranges || !nranges ||
        !nslots) {
        set_error("ppe_debug_plan_ranges: bad arguments");
        return PPE_ERR_ARG;
    }
    for (int i = 0; i < n; ++i)
        if (ntiles[i] < 0) {
            set_error("ppe_debug_plan_ranges: negative tile count");
            return PPE_ERR_ARG;
        }
    static_assert(sizeof(BlockRange) == 4 * sizeof(int32_t), "a range is four int32 values");
    *nranges = plan_ranges(n, ntiles, max_blocks, tile0, blk0, nparts, part0,
                           reinterpret_cast<BlockRange *>(ranges), max_ranges, nslots);
    return PPE_OK;
}

}  // extern "C"
