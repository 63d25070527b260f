// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ppe.h"

namespace ppe {

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);
void clear_error();
ppe_status cuda_status(cudaError_t e, const char *what);

#define PPE_CUDA_TRY(call)                                                     \
    do {                                                                       \
        cudaError_t _e = (call);                                               \
        if (_e != cudaSuccess) return ::ppe::cuda_status(_e, #call);           \
    } while (0)

#define PPE_TRY(call)                                                          \
    do {                                                                       \
        ppe_status _s = (call);                                                \
        if (_s != PPE_OK) return _s;                                           \
    } while (0)

// ---------------------------------------------------------------------------
// per-device one-time set-up (kernel attributes, lookups): fn runs with the
// device current until it succeeds once on that device
// ---------------------------------------------------------------------------
constexpr int MAX_DEVICES = 64;
struct PerDevice {
    std::mutex m;
    bool done[MAX_DEVICES] = {};
};
template <class F> bool once_per_device(PerDevice &pd, F fn)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return false;
    std::lock_guard<std::mutex> lk(pd.m);
    if (!pd.done[dev]) pd.done[dev] = fn(dev);
    return pd.done[dev];
}

// ---------------------------------------------------------------------------
// tiling of the persistent solver kernel
// ---------------------------------------------------------------------------
constexpr int TILE_X = 128;                 // cells per tile row (4 per lane)
constexpr int TILE_X_STREAM = 120;          // tile width of the streaming kernel: a warp row of
                                            // 128 cells covers it plus a four-cell halo per side
constexpr int TILE_Y = 16;                  // rows per tile (one warp each in the row-by-row passes)
constexpr int TILE_Y_R8 = 8, TILE_Y_R4 = 4; // rows per tile of the short-tile variants (2 or 4 warps a row)
constexpr int SOLVER_THREADS = 32 * TILE_Y;
constexpr int NPART = 6;                    // FP64 partial sums per tile
constexpr int PITCH_ALIGN = 32;             // inner-vector row pitch (elements)
// A pass reads its tile with a halo: two cells in y and, so that the window
// starts on a 16-byte boundary for the TMA unit, four cells in x.
constexpr int WIN_OX = 4, WIN_OY = 2;
constexpr int WIN_X = TILE_X + 2 * WIN_OX;  // 136 (window of a tile-cooperative tile)
constexpr int WIN_Y = TILE_Y + 2 * WIN_OY;  // 20 (16-row tiles; rows + 4 in general)
// Tensor maps of one system's inner vectors (per precision): the two residual
// buffers and the two direction buffers (window boxes), and d (tile box).
// MAP_Y: the per-row y coefficients (dy, fy[j], fy[j+1], 0) as an FP32 [ny][4]
// array, read by the streaming kernel.
enum SolverMap : int { MAP_R0 = 0, MAP_R1 = 1, MAP_P0 = 2, MAP_P1 = 3, MAP_D = 4, MAP_Y = 5, NMAPS = 6 };

inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Phases of the per-system state machine run by the solver kernel.
enum Phase : int32_t {
    PH_INIT = 0,      // b statistics: sum, sum of squares, sum of magnitudes
    PH_RES = 1,       // FP64 true residual of x + d (residual replacement / refinement)
    PH_RESTART = 2,   // u = D^-1 r, w = A u and the CG dots; fresh start or continuation
    PH_ITER = 3,      // one single-reduction PCG iteration
    PH_NET = 4,       // waiting for a network direction (kernel yields)
    PH_DLSM_DOT = 5,  // DLSM: r.e, e.Ae, e.e
    PH_DLSM_UPD = 6,  // DLSM: d += alpha e, r -= alpha A e
    PH_FINAL1 = 7,    // fold d into x; volume-weighted sum of x
    PH_FINAL2 = 8,    // remove the volume-weighted mean
    PH_DONE = 9
};

constexpr int SMAX = 8;   // systems one block may span

// Static description of one system (device memory, written by the host).
struct SysDesc {
    int32_t nx, ny, pitch, tiles_x, tiles_y, tile0, ntiles;   // tiles numbered column by column
    int32_t mode, precision;              // ppe_mode, ppe_precision
    int32_t max_iters, num_cg, num_dlsm, hybrid_budget;
    int32_t part0, blk0, nparts;          // partial slots part0.. for blocks blk0..blk0+nparts-1
    int32_t keep_dir_after_dlsm;          // 1: CG directions continue across DLSM steps
    int32_t dlsm_stall_limit;             // unprofitable DLSM steps in a row before plain PCG (0: never)
    int32_t dlsm_cost;                    // a DLSM step's cost in CG iterations (profitability threshold)
    int32_t force_stall;                  // test hook: every refinement after the first counts as stalled
    double tol, ru_delta, dlsm_guard, diag_max;
    double n_cells, inv_n;                // nx*ny and its reciprocal
    float n_cells_f, inv_n_f;             // the same in FP32
    const double *dx, *dy;                // widths [nx], [ny]
    const double *fx, *fy;                // face coefficients [nx+1], [ny+1]; 0 at walls
    const float *dx32, *dy32, *fx32, *fy32;
    const double *f;                      // source S [ny][nx] (caller)
    double *x;                            // solution [ny][nx] (caller)
    void *r[2], *p[2], *d;                // inner vectors [ny][pitch], FP32 or FP64 (r, p double-buffered)
    float *e;                             // DLSM direction [ny][pitch]
    const CUtensorMap *tmaps;             // NMAPS maps of r[0], r[1], p[0], p[1], d, y coefficients
};

// Mutable per-system state.  Every block that works on a system keeps an
// identical copy (each computes the same transition from the same partial
// sums); the system's first block writes it back when the kernel returns.
struct SysState {
    int32_t phase, status;
    int32_t it_pcg, it_dlsm, dlsm_skipped, refinements, it_total;
    int32_t cg_count, dlsm_count, fell_back, net_calls;
    int32_t has_d, fold_d, reset_d, first, cur, zero_x, keep_dir;
    double alpha, beta, gamma, mu, mu_b, bnorm, target, rnorm, relres, incompat;
    double alpha_d, xmean, rho, rho_ref;
    float alpha_f, beta_f, mu_f, alpha_d_f;   // FP32 copies for the FP32 passes
    int32_t dlsm_useless, pcur;           // pcur: which p buffer holds the current direction
    int32_t e_cg_n;                       // CG iterations of the current CG phase
    float e_cg, e_dlsm;                   // error energy (A-norm^2) they removed; the last DLSM step's
    float gamma_f, target_sq_f, ru_sq_f, rho_f;   // FP32 state of the FP32 iteration's transition
    // mixed precision: FP32 iterations since the last true residual and in
    // the inner solve before it; refinements in a row that did not halve the
    // true residual; 1 once the FP32 iteration is judged stalled
    int32_t it_rep, it_rep_prev, stall, prec_stalled, overran;
    double relres_prev;                   // true relative residual at the previous refinement
    // device time by kind of step (globaltimer ns, measured by the system's
    // first block): CG-type passes, DLSM passes, FP64 passes (statistics of b,
    // true residuals, finalisation), and the time between a segment that asked
    // for a network direction and the segment that used it
    uint64_t ns_pcg, ns_dlsm, ns_fp64, ns_net, t_net0;
    // bit pattern of max |b| over the system (set before the first segment by
    // the scale kernel): the solver works on 2^-e b and 2^-e x, e its binary
    // exponent, so that sums of squares stay inside the float-float range
    uint64_t bmax_bits;
};

// Tiles [t0, t1) of a block; they belong to systems s0..s1.
struct BlockRange {
    int32_t t0, t1, s0, s1;
};

// Partial-sum record of one block for one system and one step: float-float
// sums of the pass's dot products and the step number that published them.
// Two banks (by step parity) so that a block can publish step s+1 while a
// slower block still reads step s.
struct Slot {
    float hi[NPART];
    float lo[NPART];
    uint32_t pad[4];
};
static_assert(sizeof(Slot) == 64, "one record per 64-byte line");

// Global control block of one persistent launch.
// Retirements are counted in two slots by step parity: a block can only add
// to the slot of step s+2 after every block has read the slot of step s.
struct Control {
    unsigned long long arrive;   // cumulative barrier arrivals
    int32_t err;                 // PPE_ERR_TIMEOUT if a bounded wait expired
    int32_t active0;             // systems with passes left at launch
    int32_t retired[2];          // systems that stopped needing passes, by step parity
};

struct SolverArgs {
    SysDesc *sys;
    SysState *st;
    const BlockRange *ranges;  // one per block
    Slot *slots;               // [2][nslots]
    int32_t nslots;
    uint32_t *arrive;          // per system: cumulative count of published records
    Control *ctl;
    int32_t nsys, ntiles;
    int64_t spin_limit_ns;
    int32_t max_steps;         // > 0: every block leaves after this many steps (the host may re-plan)
    int32_t skip_block;        // test hook: block skip_block - 1 withholds its record at step 2 (0: off)
    unsigned long long *prof;  // nullable, 16 words: block 0's ns per step part [0..5], step count [7], iteration-pass parts [8..12], their count [13], pass entry and load issue [14..15]
};

// Solver kernel variants: FP64, FP32 with the tile-cooperative iteration
// pass, FP32 with the streaming iteration pass.
// The short-tile variants work on 128x8 or 128x4 tiles: a grid of few tiles
// spreads over two or four times the blocks, each with less work per step.
enum SolverVariant : int {
    SV_FP64 = 0, SV_FP32_TILE = 1, SV_FP32_STREAM = 2,
    SV_FP64_R8 = 3, SV_FP32_R8 = 4, SV_FP64_R4 = 5, SV_FP32_R4 = 6
};
constexpr int SV_COUNT = 7;
inline bool solver_variant_fp64(SolverVariant v) { return v == SV_FP64 || v == SV_FP64_R8 || v == SV_FP64_R4; }
inline int solver_tile_h(SolverVariant v)
{
    return v == SV_FP64_R8 || v == SV_FP32_R8 ? TILE_Y_R8 : v == SV_FP64_R4 || v == SV_FP32_R4 ? TILE_Y_R4 : TILE_Y;
}
inline int solver_tile_w(SolverVariant v) { return v == SV_FP32_STREAM ? TILE_X_STREAM : TILE_X; }

ppe_status launch_solver_resume(const SolverArgs &a, SolverVariant v, int grid_blocks, cudaStream_t stream,
                                int resume);
int solver_max_blocks(SolverVariant v, int blocks_per_sm_req);
// Kernel function and dynamic shared memory of a variant (graph nodes).
// max |b| of every system into its state (states zeroed before): the
// power-of-two scale of the solve; one launch for n systems
const void *scale_kernel_fn();
dim3 scale_grid(int n, long max_cells);
ppe_status launch_scale(const SysDesc *sys, SysState *st, int n, long max_cells, cudaStream_t s);
const void *solver_kernel_fn(SolverVariant v);
size_t solver_smem_bytes(SolverVariant v);
// Set the variants' shared-memory attributes on the current device.
void set_solver_attributes();

// Split the tiles of n systems into contiguous block ranges: every range
// holds at most `chunk` tiles (the smallest chunk for which at most
// max_blocks ranges result) and tiles of at most SMAX systems.  ntiles[s] = 0
// leaves system s without tiles.  Writes tile0 (prefix sums), blk0 and
// nparts (the ranges a system's tiles fall in, i.e. the blocks whose records
// it reduces), part0 (its first record slot) and the ranges; returns the
// number of ranges (-1 if more than max_ranges would be needed) and the
// record slots in *nslots.  Host and device (on-device re-planning of a
// batch) run the same function.
__host__ __device__ inline int plan_ranges(int n, const int32_t *ntiles, int max_blocks, int32_t *tile0,
                                           int32_t *blk0, int32_t *nparts, int32_t *part0, BlockRange *ranges,
                                           int max_ranges, int *nslots)
{
    int total = 0;
    for (int s = 0; s < n; ++s) {
        tile0[s] = total;
        total += ntiles[s];
    }
    int nr = 0;
    if (total > 0) {
        if (max_blocks < 1) return -1;
        for (int chunk = (total + max_blocks - 1) / max_blocks;; ++chunk) {
            nr = 0;
            int t = 0, s = 0;
            while (t < total) {
                while (tile0[s] + ntiles[s] <= t) ++s;              // the system holding tile t
                const int lim = s + SMAX < n ? tile0[s + SMAX] : total;
                const int e = t + chunk < lim ? t + chunk : lim;
                int s1 = s;
                while (tile0[s1] + ntiles[s1] <= e - 1) ++s1;
                if (nr < max_ranges) {
                    ranges[nr].t0 = t; ranges[nr].t1 = e; ranges[nr].s0 = s; ranges[nr].s1 = s1;
                }
                ++nr;
                t = e;
            }
            if (nr <= max_blocks && nr <= max_ranges) break;
            if (chunk > total) return -1;
        }
    }
    int slots = 0;
    for (int s = 0; s < n; ++s) {
        int first = -1, last = -1;
        for (int b = 0; b < nr; ++b)
            if (s >= ranges[b].s0 && s <= ranges[b].s1) {
                if (first < 0) first = b;
                last = b;
            }
        blk0[s] = first;
        nparts[s] = first < 0 ? 0 : last - first + 1;
        part0[s] = slots;
        slots += nparts[s];
    }
    *nslots = slots;
    return nr;
}

// Device-resident alternation of a solve (one CUDA graph launch): the loop
// control the decision kernel reads and updates between solver segments.
struct DriveCtl {
    int32_t n;              // systems
    int32_t max_blocks;     // blocks of every solver launch (ranges beyond the plan are empty)
    int32_t slot_cap;       // record slots per bank
    int32_t max_steps;      // > 0: segments end on this step budget and a batch may be re-planned
    int32_t planned_tiles;  // tiles of the current plan
    int32_t launches;       // solver segments run so far
    int32_t loop_cap;       // give up after this many segments
    int32_t err;            // ppe_status of the loop itself (timeout, cap)
    float fraction;         // re-plan when the running systems hold fewer tiles than this share of the plan
    int32_t with_net;       // 1: the graph has a network branch per system
    int32_t pad_[2];
};

// Encode the NMAPS tensor maps of one system's inner vectors for a kernel
// variant (element type FP32 or FP64, box shapes of the variant's tiles; row
// pitch `pitch` elements, a multiple of 4; every buffer 16-byte aligned).
// Cells outside [0,nx) x [0,ny) read as zero.  ycoef (nullable: the map is
// then left zero) is the FP32 [ny][4] row-coefficient array.
ppe_status encode_solver_maps(void *const r[2], void *const p[2], void *d, const float *ycoef, int nx, int ny,
                              int pitch, SolverVariant v, CUtensorMap out[NMAPS]);

// Autotuned launch configuration of a grid shape, if ppe_autotune measured
// one in this process (or the tuning cache file holds one).
bool tune_lookup(int nx, int ny, int *iter_pass, int *blocks_per_sm, int *tile_rows);

// Remove the mean of the grid's DLSM direction e (two kernels on `stream`;
// no allocation, so it may run inside a stream capture).
ppe_status center_direction(ppe_grid *g, cudaStream_t stream);

// Device resources of one set of solver launches (a grid's single solves, or
// a batch), allocated once and reused by every solve: descriptions, states,
// block ranges, record slots, barrier counters, loop control, events, and
// the solve graph with what it was built for.
struct LaunchSet {
    int n = 0, max_ranges = 0, slot_cap = 0, device = 0;
    SysDesc *sys = nullptr;
    SysState *st = nullptr;
    BlockRange *ranges = nullptr, *ranges_tmp = nullptr;
    Slot *slots = nullptr;               // 2 banks x slot_cap records
    Control *ctl = nullptr;
    uint32_t *arrive = nullptr;          // per system: cumulative count of published records
    DriveCtl *dc = nullptr;
    int32_t *full_tiles = nullptr;       // per system: tiles of its full plan
    int32_t *plan_scratch = nullptr;     // 5 n integers for on-device re-planning
    cudaGraphConditionalHandle *if_handles = nullptr;   // per system: its network branch
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaStream_t cap = nullptr;          // capture stream of the network branches
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // what the graph was built for
    SolverArgs built_args{};
    int built_variant = -1, built_blocks = 0, built_with_net = 0;
    const void *built_net = nullptr;
    uint64_t built_version = 0;
};
ppe_status launch_set_create(int n, int max_ranges, int slot_cap, LaunchSet **out);
void launch_set_destroy(LaunchSet *ls);

// The multigrid partner (mg.cu): hierarchy and buffers of a grid, built on
// its first multigrid solve; the solve itself (FP32 inner MG-PCG, FP64
// refinement).
struct MgPlan;
void mg_plan_destroy(MgPlan *m);
ppe_status mg_solve(ppe_grid *g, const double *rhs, double *x, double tol, cudaStream_t stream,
                    ppe_solve_info *info);

}  // namespace ppe

// The grid handle (opaque in the public header).
struct ppe_grid {
    int nx = 0, ny = 0, pitch = 0, tiles_x = 0, tiles_y = 0;
    double lx = 0, ly = 0, diag_max = 0;
    std::vector<double> hdx, hdy;
    std::vector<uint8_t> hmask;
    ppe_solve_opts opts{};
    int device = 0;
    // device copies
    double *dx = nullptr, *dy = nullptr, *fx = nullptr, *fy = nullptr;
    float *dx32 = nullptr, *dy32 = nullptr, *fx32 = nullptr, *fy32 = nullptr;
    void *vec = nullptr;                 // 5 inner vectors, 8 bytes per element
    float *e = nullptr;                  // DLSM direction
    double *dir_part = nullptr;          // partial sums of the direction's mean removal
    float *ycoef = nullptr;              // [ny][4] FP32: dy, fy[j], fy[j+1], 0 (streaming kernel)
    void *r[2] = {nullptr, nullptr}, *p[2] = {nullptr, nullptr}, *d = nullptr;
    CUtensorMap *tmaps_dev = nullptr;    // tensor maps of the inner vectors, one set per kernel variant
    int tuned_pass = 0, tuned_bps = 0, tuned_rows = 0;   // ppe_autotune's choice (0: none)
    uint64_t id = 0;                     // process-unique creation number (keys cached batch plans)
    ppe::LaunchSet *ls = nullptr;        // single-system launch resources and the solve graph
    ppe::MgPlan *mg = nullptr;           // multigrid hierarchy (first multigrid solve)
    ppe_direction_fn dir_fn = nullptr;   // user direction source (replaces the network)
    void *dir_user = nullptr;
    float *dir_r = nullptr, *dir_e = nullptr;   // [ny][nx] staging for dir_fn
    void *net_cache = nullptr;           // per-network data for this grid (owned by the net)
    const void *net_owner = nullptr;
};
