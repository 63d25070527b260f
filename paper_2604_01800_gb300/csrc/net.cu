// The grid-spacing-aware DeepONet (Sec. 2.4): parameters, per-grid caches
// (distance maps, Mesh-Conv weights eta, trunk features), forward pass, the
// DLSM direction hook of the solver, and the weights file.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "net_iface.h"
#include "net_impl.h"
#include "net_ops.h"

namespace ppe {

// ---------------------------------------------------------------------------
// parameter layout
// ---------------------------------------------------------------------------

static void build_layout(ppe_net *n)
{
    const ppe_net_config &c = n->cfg;
    const int L = c.levels;
    n->layers.clear();
    int64_t off = 0, offp = 0;
    auto add = [&](const std::string &name, int cin, int cout, int level) {
        ConvLayer l;
        l.name = name; l.cin = cin; l.cout = cout; l.level = level;
        l.off_w = off; off += (int64_t)cout * cin * 9;
        l.off_b = off; off += cout;
        l.off_p1w = off; off += (int64_t)c.phi_hidden * 4;
        l.off_p1b = off; off += c.phi_hidden;
        l.off_p2w = off; off += c.phi_hidden;
        l.off_p2b = off; off += 1;
        l.off_wp = offp; l.off_wt = offp;
        offp += (int64_t)cout * cin * 9;
        n->layers.push_back(l);
    };
    int cin = 1;
    for (int k = 0; k < L; ++k) {
        add("enc" + std::to_string(k) + "a", cin, c.widths[k], k);
        add("enc" + std::to_string(k) + "b", c.widths[k], c.widths[k], k);
        cin = c.widths[k];
    }
    for (int k = L - 2; k >= 0; --k) {
        add("up" + std::to_string(k), c.widths[k + 1], c.widths[k], k);
        add("dec" + std::to_string(k) + "a", 2 * c.widths[k], c.widths[k], k);
        add("dec" + std::to_string(k) + "b", c.widths[k], c.widths[k], k);
    }
    n->off_head_w = off; off += (int64_t)c.c_last * c.widths[0];
    n->off_head_b = off; off += c.c_last;
    int dims[4] = {2, c.trunk_hidden[0], c.trunk_hidden[1], c.c_last};
    for (int i = 0; i < 3; ++i) {
        n->off_tw[i] = off; off += (int64_t)dims[i + 1] * dims[i];
        n->off_tb[i] = off; off += dims[i + 1];
    }
    n->off_out_b = off; off += 1;
    n->nparams = off;
    n->npacked = offp;
}

int layer_index(const ppe_net *n, const std::string &name)
{
    for (size_t i = 0; i < n->layers.size(); ++i)
        if (n->layers[i].name == name) return (int)i;
    return -1;
}

static bool valid_config(const ppe_net_config &c)
{
    if (c.levels < 2 || c.levels > PPE_NET_MAX_LEVELS) return false;
    for (int k = 0; k < c.levels; ++k)
        if (c.widths[k] < 16 || c.widths[k] % 16 || c.widths[k] > 256) return false;
    if (c.c_last < 1 || c.c_last > 1024 || c.phi_hidden < 1 || c.phi_hidden > 16) return false;
    if (c.trunk_hidden[0] < 1 || c.trunk_hidden[1] < 1 || c.trunk_hidden[0] > 4096 || c.trunk_hidden[1] > 4096)
        return false;
    return true;
}

// splitmix64-based normal generator for net_create's own initial values
struct InitRng {
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double normal() { return std::sqrt(-2.0 * std::log(uniform())) * std::cos(6.283185307179586 * uniform()); }
};

static void init_params(ppe_net *n, uint64_t seed)
{
    InitRng g{seed};
    std::vector<float> &p = n->host_params;
    p.assign(n->nparams, 0.f);
    for (auto &l : n->layers) {
        double sd = std::sqrt(2.0 / (9.0 * l.cin));
        for (int64_t i = 0; i < (int64_t)l.cout * l.cin * 9; ++i) p[l.off_w + i] = (float)(g.normal() * sd);
        for (int i = 0; i < n->cfg.phi_hidden * 4; ++i) p[l.off_p1w + i] = (float)(0.1 * g.normal());
        for (int i = 0; i < n->cfg.phi_hidden; ++i) p[l.off_p2w + i] = (float)(0.1 * g.normal());
    }
    double sh = std::sqrt(1.0 / n->cfg.widths[0]);
    for (int64_t i = 0; i < (int64_t)n->cfg.c_last * n->cfg.widths[0]; ++i) p[n->off_head_w + i] = (float)(g.normal() * sh);
    int dims[4] = {2, n->cfg.trunk_hidden[0], n->cfg.trunk_hidden[1], n->cfg.c_last};
    for (int i = 0; i < 3; ++i) {
        double st = std::sqrt(2.0 / (dims[i] + dims[i + 1]));
        for (int64_t k = 0; k < (int64_t)dims[i] * dims[i + 1]; ++k) p[n->off_tw[i] + k] = (float)(g.normal() * st);
    }
}

static ppe_status upload_params(ppe_net *n)
{
    PPE_CUDA_TRY(cudaMemcpy(n->params, n->host_params.data(), n->nparams * 4, cudaMemcpyHostToDevice));
    n->version++;
    n->packed_version = 0;
    return PPE_OK;
}

ppe_status net_alloc(ppe_net *n)
{
    PPE_CUDA_TRY(cudaMalloc(&n->params, n->nparams * 4));
    PPE_CUDA_TRY(cudaMalloc(&n->grads, n->nparams * 4));
    PPE_CUDA_TRY(cudaMalloc(&n->grads2, n->nparams * 4));
    PPE_CUDA_TRY(cudaMalloc(&n->params_pert, n->nparams * 4));
    PPE_CUDA_TRY(cudaMalloc(&n->adam_m, n->nparams * 4));
    PPE_CUDA_TRY(cudaMalloc(&n->adam_v, n->nparams * 4));
    PPE_CUDA_TRY(cudaMemset(n->adam_m, 0, n->nparams * 4));
    PPE_CUDA_TRY(cudaMemset(n->adam_v, 0, n->nparams * 4));
    PPE_CUDA_TRY(cudaMalloc(&n->wp, n->npacked * 2));
    PPE_CUDA_TRY(cudaMalloc(&n->wt, n->npacked * 2));
    PPE_CUDA_TRY(cudaMalloc(&n->scratch, 64 * sizeof(double)));
    return PPE_OK;
}

// Re-pack BF16 conv weights from the FP32 master copy (active parameter set).
ppe_status ensure_packed(ppe_net *n, const float *P, cudaStream_t s)
{
    // the master parameters are cached by version; any other set (the SAM
    // perturbation) is packed every time
    uint64_t want = P == n->params ? n->version : 0;
    if (want && n->packed_version == want && n->packed_src == P) return PPE_OK;
    for (auto &l : n->layers)
        PPE_TRY(pack_conv_weights(P + l.off_w, n->wp + l.off_wp, n->wt + l.off_wt, l.cout, l.cin, s));
    n->packed_version = want;
    n->packed_src = P;
    return PPE_OK;
}

// ---------------------------------------------------------------------------
// per-grid cache
// ---------------------------------------------------------------------------

static void free_cache(NetCache *c)
{
    if (!c) return;
    net_free_train(c);
    if (c->dir_exec) cudaGraphExecDestroy(c->dir_exec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    cudaFree(c->delta); cudaFree(c->eta); cudaFree(c->phi); cudaFree(c->xy); cudaFree(c->trunk);
    cudaFree(c->weff); cudaFree(c->ceff); cudaFree(c->act); cudaFree(c->grad_act); cudaFree(c->efull);
    cudaFree(c->red);
    delete c;
}

void net_release_grid(ppe_grid *g)
{
    if (g && g->net_cache) {
        NetCache *c = (NetCache *)g->net_cache;
        if (c->net) {
            auto &v = c->net->grids;
            v.erase(std::remove(v.begin(), v.end(), g), v.end());
        }
        free_cache(c);
        g->net_cache = nullptr;
        g->net_owner = nullptr;
    }
}

ppe_status net_check_grid(ppe_net *net, ppe_grid *g)
{
    if (!net) return PPE_ERR_NO_NET;
    if (!g->net_cache || g->net_owner != net) {
        set_error("hybrid solve: network not attached to this grid (call net_attach)");
        return PPE_ERR_NO_NET;
    }
    return PPE_OK;
}

static std::vector<double> centres(const std::vector<double> &d)
{
    std::vector<double> c(d.size());
    double f = 0.0;
    for (size_t i = 0; i < d.size(); ++i) {
        c[i] = f + 0.5 * d[i];
        f += d[i];
    }
    return c;
}

// Distance-vector maps Delta_K [4][H_K][W_K] (left, right, up, down), scaled
// by the inverse mean spacing of the unpadded grid; nearest-neighbour values
// at the walls (Sec. 2.4).
static void distance_maps(const std::vector<double> &dxp, const std::vector<double> &dyp, double sx, double sy,
                          int L, std::vector<std::vector<float>> &out)
{
    std::vector<double> xc = centres(dxp), yc = centres(dyp);
    out.assign(L, {});
    for (int k = 0; k < L; ++k) {
        if (k > 0) {
            std::vector<double> nx(xc.size() / 2), ny(yc.size() / 2);
            for (size_t i = 0; i < nx.size(); ++i) nx[i] = 0.5 * (xc[2 * i] + xc[2 * i + 1]);
            for (size_t j = 0; j < ny.size(); ++j) ny[j] = 0.5 * (yc[2 * j] + yc[2 * j + 1]);
            xc.swap(nx);
            yc.swap(ny);
        }
        int W = (int)xc.size(), H = (int)yc.size();
        auto side = [](const std::vector<double> &c, std::vector<double> &prev, std::vector<double> &next) {
            int n = (int)c.size();
            prev.assign(n, 0.0);
            next.assign(n, 0.0);
            for (int i = 0; i + 1 < n; ++i) {
                double d = std::fabs(c[i + 1] - c[i]);
                next[i] = d;
                prev[i + 1] = d;
            }
            if (n > 1) {
                prev[0] = next[0];
                next[n - 1] = prev[n - 1];
            }
        };
        std::vector<double> left, right, down, up;
        side(xc, left, right);
        side(yc, down, up);
        std::vector<float> m((size_t)4 * H * W);
        for (int j = 0; j < H; ++j)
            for (int i = 0; i < W; ++i) {
                size_t q = (size_t)j * W + i;
                m[q] = (float)(left[i] * sx);
                m[(size_t)H * W + q] = (float)(right[i] * sx);
                m[(size_t)2 * H * W + q] = (float)(up[j] * sy);
                m[(size_t)3 * H * W + q] = (float)(down[j] * sy);
            }
        out[k].swap(m);
    }
}

static ppe_status make_cache(ppe_net *n, ppe_grid *g, NetCache **out)
{
    const int L = n->cfg.levels;
    const int m = 1 << L;
    NetCache *c = new NetCache();
    c->net = n;
    c->nx = g->nx; c->ny = g->ny;
    c->W = round_up(g->nx, m);
    c->H = round_up(g->ny, m);
    c->L = L;
    for (int k = 0; k < L; ++k) { c->Wk[k] = c->W >> k; c->Hk[k] = c->H >> k; }
    std::vector<double> dxp = g->hdx, dyp = g->hdy;
    while ((int)dxp.size() < c->W) dxp.push_back(g->hdx.back());
    while ((int)dyp.size() < c->H) dyp.push_back(g->hdy.back());
    double sx = g->nx / g->lx, sy = g->ny / g->ly;
    std::vector<std::vector<float>> maps;
    distance_maps(dxp, dyp, sx, sy, L, maps);
    size_t dtot = 0;
    for (int k = 0; k < L; ++k) { c->doff[k] = dtot; dtot += maps[k].size(); }
    auto fail = [&](cudaError_t e) { free_cache(c); return cuda_status(e, "net_attach allocation"); };
    cudaError_t e;
    if ((e = cudaMalloc(&c->delta, dtot * 4)) != cudaSuccess) return fail(e);
    for (int k = 0; k < L; ++k)
        if ((e = cudaMemcpy(c->delta + c->doff[k], maps[k].data(), maps[k].size() * 4, cudaMemcpyHostToDevice)) !=
            cudaSuccess)
            return fail(e);
    size_t etot = 0;
    c->eoff.resize(n->layers.size());
    for (size_t i = 0; i < n->layers.size(); ++i) {
        c->eoff[i] = etot;
        int k = n->layers[i].level;
        etot += (size_t)c->Hk[k] * c->Wk[k];
    }
    if ((e = cudaMalloc(&c->eta, etot * 4)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&c->phi, etot * 4)) != cudaSuccess) return fail(e);
    // trunk input: normalised cell-centre coordinates of the padded grid
    const size_t P = (size_t)c->H * c->W;
    std::vector<double> xc = centres(dxp), yc = centres(dyp);
    std::vector<float> xy(2 * P);
    for (int j = 0; j < c->H; ++j)
        for (int i = 0; i < c->W; ++i) {
            xy[(size_t)j * c->W + i] = (float)(xc[i] / g->lx);
            xy[P + (size_t)j * c->W + i] = (float)(yc[j] / g->ly);
        }
    if ((e = cudaMalloc(&c->xy, 2 * P * 4)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpy(c->xy, xy.data(), 2 * P * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
    const ppe_net_config &cf = n->cfg;
    size_t tr = (size_t)(cf.trunk_hidden[0] + cf.trunk_hidden[1] + cf.c_last) * P;
    if ((e = cudaMalloc(&c->trunk, tr * 4)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&c->weff, (size_t)cf.widths[0] * P * 4)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&c->ceff, P * 4)) != cudaSuccess) return fail(e);
    *out = c;
    return PPE_OK;
}

// Activation plan for batch B (offsets in BF16 elements).
static void plan_acts(const ppe_net *n, NetCache *c, int B)
{
    const int L = c->L;
    size_t off = 0;
    auto take = [&](size_t elems) { size_t o = off; off += (elems + 127) / 128 * 128; return o; };
    ActPlan &a = c->plan;
    for (int k = 0; k < L; ++k) {
        size_t px = (size_t)B * c->Hk[k] * c->Wk[k];
        int Ck = n->cfg.widths[k];
        a.A[k] = take(px * Ck);
        a.IN[k] = k > 0 ? take(px * n->cfg.widths[k - 1]) : 0;
        a.P[k] = k < L - 1 ? take(px * Ck) : 0;
        a.CAT[k] = k < L - 1 ? take(px * 2 * Ck) : 0;
        a.UP[k] = k < L - 1 ? take(px * n->cfg.widths[k + 1]) : 0;
        a.D[k] = k < L - 1 ? take(px * Ck) : 0;
        a.U[k] = take(px * Ck);
    }
    // pre-activations of every layer (training)
    a.Z.resize(n->layers.size());
    for (size_t i = 0; i < n->layers.size(); ++i) {
        int k = n->layers[i].level;
        a.Z[i] = take((size_t)B * c->Hk[k] * c->Wk[k] * n->layers[i].cout);
    }
    a.total = off;
}

ppe_status ensure_acts(ppe_net *n, NetCache *c, int B)
{
    if (c->capB >= B && c->act) return PPE_OK;
    cudaFree(c->act);
    c->act = nullptr;
    plan_acts(n, c, B);
    PPE_CUDA_TRY(cudaMalloc(&c->act, c->plan.total * 2));
    PPE_CUDA_TRY(cudaMemset(c->act, 0, c->plan.total * 2));
    c->capB = B;
    return PPE_OK;
}

// eta for every layer, trunk features, folded head (for parameters P).
ppe_status refresh_cache(ppe_net *n, NetCache *c, const float *P, cudaStream_t s)
{
    uint64_t want = P == n->params ? n->version : 0;
    if (want && c->version == want && c->src == P) return PPE_OK;
    const ppe_net_config &cf = n->cfg;
    for (size_t i = 0; i < n->layers.size(); ++i) {
        const ConvLayer &l = n->layers[i];
        int k = l.level;
        int HW = c->Hk[k] * c->Wk[k];
        PPE_TRY(eta_layer(c->delta + c->doff[k], HW, P + l.off_p1w, P + l.off_p1b, P + l.off_p2w, P + l.off_p2b,
                          cf.phi_hidden, cf.mesh_conv, c->eta + c->eoff[i], c->phi + c->eoff[i], s));
    }
    const int Pn = c->H * c->W;
    float *t1 = c->trunk, *t2 = t1 + (size_t)cf.trunk_hidden[0] * Pn, *t3 = t2 + (size_t)cf.trunk_hidden[1] * Pn;
    PPE_TRY(tgemm(cf.trunk_hidden[0], Pn, 2, P + n->off_tw[0], 2, false, c->xy, Pn, false, t1, Pn, P + n->off_tb[0], 1,
                  false, s));
    PPE_TRY(tgemm(cf.trunk_hidden[1], Pn, cf.trunk_hidden[0], P + n->off_tw[1], cf.trunk_hidden[0], false, t1, Pn,
                  false, t2, Pn, P + n->off_tb[1], 1, false, s));
    PPE_TRY(tgemm(cf.c_last, Pn, cf.trunk_hidden[1], P + n->off_tw[2], cf.trunk_hidden[1], false, t2, Pn, false, t3,
                  Pn, P + n->off_tb[2], 0, false, s));
    // weff[c0][p] = sum_c head.w[c][c0] t3[c][p];  ceff[p] = sum_c head.b[c] t3[c][p] + out.b
    PPE_TRY(tgemm(cf.widths[0], Pn, cf.c_last, P + n->off_head_w, cf.widths[0], true, t3, Pn, false, c->weff, Pn,
                  nullptr, 0, false, s));
    PPE_TRY(tgemm(1, Pn, cf.c_last, P + n->off_head_b, cf.c_last, false, t3, Pn, false, c->ceff, Pn,
                  P + n->off_out_b, 0, false, s));
    c->version = want;
    c->src = P;
    return PPE_OK;
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------

ppe_status run_conv(ppe_net *n, const ConvArgs &a, cudaStream_t s)
{
    if (n->use_tc && conv3x3_tc_supported(a)) return conv3x3_tc(a, s);
    return conv3x3_simt(a, s);
}

ppe_status net_forward(ppe_net *n, NetCache *c, int B, const InputSrc &src, const float *P, float *e, int e_pitch,
                       size_t e_bstride, bool keep_z, cudaStream_t s)
{
    PPE_TRY(ensure_packed(n, P, s));
    PPE_TRY(refresh_cache(n, c, P, s));
    PPE_TRY(ensure_acts(n, c, B));
    const ppe_net_config &cf = n->cfg;
    const int L = c->L;
    bf16 *act = c->act;
    const ActPlan &pl = c->plan;
    auto eta = [&](const std::string &name) { return c->eta + c->eoff[layer_index(n, name)]; };
    auto zbuf = [&](int li) { return keep_z ? act + pl.Z[li] : (bf16 *)nullptr; };
    auto args = [&](const std::string &name, const bf16 *in, int k, const Epi &ep) {
        int li = layer_index(n, name);
        const ConvLayer &l = n->layers[li];
        ConvArgs a;
        a.in = in; a.w = n->wp + l.off_wp; a.bias = P + l.off_b;
        a.B = B; a.H = c->Hk[k]; a.W = c->Wk[k]; a.cin = l.cin; a.cout = l.cout;
        a.epi = ep;
        a.epi.z_out = zbuf(li);
        return a;
    };
    auto conv = [&](const std::string &name, const bf16 *in, int k, const Epi &ep) -> ppe_status {
        return run_conv(n, args(name, in, k, ep), s);
    };
    // on the tensor-core path the 2x2 pooling and the nearest up-sampling
    // run in the producing convolution's epilogue; otherwise the raw output
    // goes to P[k] / U[k] and separate kernels pool or up-sample it
    auto fused = [&](const std::string &name, const bf16 *in, int k) {
        return n->use_tc && conv3x3_tc_supported(args(name, in, k, Epi()));
    };
    bool pooled[PPE_NET_MAX_LEVELS] = {}, upped[PPE_NET_MAX_LEVELS] = {};
    // enc0a: 1-channel input
    {
        int li = layer_index(n, "enc0a");
        const ConvLayer &l = n->layers[li];
        Epi ep;
        ep.z_out = zbuf(li);
        ep.out1 = act + pl.A[0]; ep.cs1 = cf.widths[0]; ep.co1 = 0; ep.eta1 = eta("enc0b");
        PPE_TRY(conv_in(src, B, c->H, c->W, eta("enc0a"), n->wp + l.off_wp, P + l.off_b, l.cout, ep, s));
    }
    for (int k = 0; k < L; ++k) {
        const int Ck = cf.widths[k];
        std::string ks = std::to_string(k);
        if (k > 0) {
            if (!pooled[k])
                PPE_TRY(pool2(act + pl.P[k - 1], act + pl.IN[k], B, c->Hk[k], c->Wk[k], cf.widths[k - 1],
                              eta("enc" + ks + "a"), s));
            Epi ep;
            ep.out1 = act + pl.A[k]; ep.cs1 = Ck; ep.eta1 = eta("enc" + ks + "b");
            PPE_TRY(conv("enc" + ks + "a", act + pl.IN[k], k, ep));
        }
        Epi ep;
        const bool f = fused("enc" + ks + "b", act + pl.A[k], k);
        if (k < L - 1) {
            ep.out1 = act + pl.CAT[k]; ep.cs1 = 2 * Ck; ep.co1 = Ck; ep.eta1 = eta("dec" + ks + "a");
            if (f) {
                ep.pool_out = act + pl.IN[k + 1]; ep.pool_cs = Ck; ep.pool_eta = eta("enc" + std::to_string(k + 1) + "a");
                pooled[k + 1] = true;
            } else {
                ep.out2 = act + pl.P[k]; ep.cs2 = Ck; ep.co2 = 0; ep.eta2 = nullptr;
            }
        } else if (f && k > 0) {
            ep.up_out = act + pl.UP[k - 1]; ep.up_cs = Ck; ep.up_eta = eta("up" + std::to_string(k - 1));
            upped[k - 1] = true;
        } else {
            ep.out1 = act + pl.U[k]; ep.cs1 = Ck;
        }
        PPE_TRY(conv("enc" + ks + "b", act + pl.A[k], k, ep));
    }
    for (int k = L - 2; k >= 0; --k) {
        const int Ck = cf.widths[k];
        std::string ks = std::to_string(k);
        if (!upped[k])
            PPE_TRY(up2(act + pl.U[k + 1], act + pl.UP[k], B, c->Hk[k], c->Wk[k], cf.widths[k + 1], eta("up" + ks),
                        s));
        Epi e1;
        e1.out1 = act + pl.CAT[k]; e1.cs1 = 2 * Ck; e1.co1 = 0; e1.eta1 = eta("dec" + ks + "a");
        PPE_TRY(conv("up" + ks, act + pl.UP[k], k, e1));
        Epi e2;
        e2.out1 = act + pl.D[k]; e2.cs1 = Ck; e2.eta1 = eta("dec" + ks + "b");
        PPE_TRY(conv("dec" + ks + "a", act + pl.CAT[k], k, e2));
        Epi e3;
        if (k > 0 && fused("dec" + ks + "b", act + pl.D[k], k)) {
            e3.up_out = act + pl.UP[k - 1]; e3.up_cs = Ck; e3.up_eta = eta("up" + std::to_string(k - 1));
            upped[k - 1] = true;
        } else {
            e3.out1 = act + pl.U[k]; e3.cs1 = Ck;
        }
        PPE_TRY(conv("dec" + ks + "b", act + pl.D[k], k, e3));
    }
    return fold_out(act + pl.U[0], c->weff, c->ceff, B, c->H, c->W, cf.widths[0], e, e_pitch, e_bstride, c->nx, c->ny,
                    s);
}

ppe_status net_prepare_direction(ppe_net *net, ppe_grid *g, cudaStream_t stream)
{
    PPE_TRY(net_check_grid(net, g));
    NetCache *c = (NetCache *)g->net_cache;
    PPE_TRY(ensure_packed(net, net->params, stream));
    PPE_TRY(refresh_cache(net, c, net->params, stream));
    PPE_TRY(ensure_acts(net, c, 1));
    if (net->use_tc) PPE_TRY(conv3x3_tc_prepare());     // one-time set-up cannot run inside a capture
    return PPE_OK;
}

ppe_status net_record_direction(ppe_net *net, ppe_grid *g, const SysDesc *sd_dev, const SysState *st_dev,
                                cudaStream_t stream)
{
    PPE_TRY(net_check_grid(net, g));
    NetCache *c = (NetCache *)g->net_cache;
    InputSrc src;
    src.sd = sd_dev; src.st = st_dev; src.nx = g->nx; src.ny = g->ny;
    PPE_TRY(net_forward(net, c, 1, src, net->params, g->e, g->pitch, 0, false, stream));
    return center_direction(g, stream);
}

uint64_t net_direction_key(const ppe_net *net, const ppe_grid *g)
{
    // what a captured direction bakes in: the parameter version (packed
    // weights, eta, trunk fold) and the grid's activation buffers
    const NetCache *c = g ? (const NetCache *)g->net_cache : nullptr;
    uint64_t h = net ? net->version : 0;
    h = h * 0x100000001b3ull ^ (uint64_t)(uintptr_t)c;
    h = h * 0x100000001b3ull ^ (uint64_t)(uintptr_t)(c ? c->act : nullptr);
    return h;
}

// The DLSM direction of a solver system: the forward pass on its normalised
// residual, with its mean removed.  The sequence of launches is the same on every call, so it is
// captured once into a CUDA graph (per grid and parameter version) and
// replayed with a single launch afterwards.
ppe_status net_direction(ppe_net *net, ppe_grid *g, const SysDesc *sd_dev, const SysState *st_dev, bool,
                         cudaStream_t stream, float *ms)
{
    PPE_TRY(net_check_grid(net, g));
    NetCache *c = (NetCache *)g->net_cache;
    if (ms) *ms = 0.f;
    PPE_TRY(ensure_packed(net, net->params, stream));
    PPE_TRY(refresh_cache(net, c, net->params, stream));
    PPE_TRY(ensure_acts(net, c, 1));
    if (!(c->dir_exec && c->dir_version == net->version && c->dir_key == (const void *)sd_dev &&
          c->dir_act == (const void *)c->act)) {
        if (c->dir_exec) {
            cudaGraphExecDestroy(c->dir_exec);
            c->dir_exec = nullptr;
        }
        if (!c->cap_stream) PPE_CUDA_TRY(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        if (net->use_tc) PPE_TRY(conv3x3_tc_prepare());     // one-time set-up cannot run inside a capture
        InputSrc src;
        src.sd = sd_dev; src.st = st_dev; src.nx = g->nx; src.ny = g->ny;
        cudaGraph_t graph = nullptr;
        PPE_CUDA_TRY(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        ppe_status fs = net_forward(net, c, 1, src, net->params, g->e, g->pitch, 0, false, c->cap_stream);
        if (fs == PPE_OK) fs = center_direction(g, c->cap_stream);
        cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &graph);
        if (fs != PPE_OK) {
            if (graph) cudaGraphDestroy(graph);
            return fs;
        }
        if (ce != cudaSuccess) return cuda_status(ce, "cudaStreamEndCapture(direction)");
        ce = cudaGraphInstantiate(&c->dir_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            c->dir_exec = nullptr;
            return cuda_status(ce, "cudaGraphInstantiate(direction)");
        }
        c->dir_version = net->version;
        c->dir_key = sd_dev;
        c->dir_act = c->act;
    }
    PPE_CUDA_TRY(cudaGraphLaunch(c->dir_exec, stream));
    return PPE_OK;
}

}  // namespace ppe

using namespace ppe;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

static uint32_t crc32_bytes(const unsigned char *p, size_t n, uint32_t crc = 0)
{
    crc = ~crc;
    for (size_t i = 0; i < n; ++i) {
        crc ^= p[i];
        for (int k = 0; k < 8; ++k) crc = (crc >> 1) ^ (0xEDB88320u & (0u - (crc & 1u)));
    }
    return ~crc;
}

extern "C" {

void net_default_config(ppe_net_config *c)
{
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->levels = 4;
    c->widths[0] = 32; c->widths[1] = 64; c->widths[2] = 128; c->widths[3] = 256;
    c->c_last = 100;
    c->trunk_hidden[0] = 100; c->trunk_hidden[1] = 200;
    c->phi_hidden = 16;
    c->mesh_conv = 1;
}

void net_destroy(ppe_net *n)
{
    if (!n) return;
    std::vector<ppe_grid *> gs = n->grids;
    for (ppe_grid *g : gs) net_release_grid(g);
    cudaFree(n->params); cudaFree(n->grads); cudaFree(n->grads2); cudaFree(n->params_pert);
    cudaFree(n->adam_m); cudaFree(n->adam_v); cudaFree(n->wp); cudaFree(n->wt); cudaFree(n->scratch);
    delete n;
}

ppe_status net_create(const ppe_net_config *cfg, uint64_t seed, ppe_net **out)
{
    clear_error();
    if (!cfg || !out) { set_error("net_create: NULL argument"); return PPE_ERR_ARG; }
    *out = nullptr;
    if (!valid_config(*cfg)) { set_error("net_create: invalid configuration"); return PPE_ERR_ARG; }
    ppe_net *n = new ppe_net();
    n->cfg = *cfg;
    build_layout(n);
    init_params(n, seed);
    ppe_status st = net_alloc(n);
    if (st == PPE_OK) st = upload_params(n);
    if (st != PPE_OK) { net_destroy(n); return st; }
    *out = n;
    return PPE_OK;
}

ppe_status net_param_count(const ppe_net *n, int64_t *count)
{
    if (!n || !count) { set_error("net_param_count: NULL argument"); return PPE_ERR_ARG; }
    *count = n->nparams;
    return PPE_OK;
}

ppe_status net_get_config(const ppe_net *n, ppe_net_config *cfg)
{
    if (!n || !cfg) { set_error("net_get_config: NULL argument"); return PPE_ERR_ARG; }
    *cfg = n->cfg;
    return PPE_OK;
}

ppe_status net_set_params(ppe_net *n, const float *params, int64_t count)
{
    clear_error();
    if (!n || !params || count != n->nparams) { set_error("net_set_params: bad arguments or count"); return PPE_ERR_ARG; }
    n->host_params.assign(params, params + count);
    return upload_params(n);
}

ppe_status net_get_params(const ppe_net *n, float *params, int64_t count)
{
    clear_error();
    if (!n || !params || count != n->nparams) { set_error("net_get_params: bad arguments or count"); return PPE_ERR_ARG; }
    PPE_CUDA_TRY(cudaDeviceSynchronize());
    PPE_CUDA_TRY(cudaMemcpy(params, n->params, count * 4, cudaMemcpyDeviceToHost));
    return PPE_OK;
}

static ppe_status save_impl(const ppe_net *n, const char *path, bool with_moments)
{
    clear_error();
    if (!n || !path) { set_error("net_save: NULL argument"); return PPE_ERR_ARG; }
    PPE_CUDA_TRY(cudaDeviceSynchronize());
    std::vector<unsigned char> buf;
    auto put = [&](const void *p, size_t k) {
        const unsigned char *c = (const unsigned char *)p;
        buf.insert(buf.end(), c, c + k);
    };
    const char magic[8] = {'P', 'P', 'E', 'N', 'E', 'T', '0', '1'};
    uint32_t version = 1, flags = with_moments ? 1u : 0u;
    put(magic, 8); put(&version, 4); put(&flags, 4); put(&n->cfg, sizeof(ppe_net_config));
    int64_t np = n->nparams, step = n->step;
    put(&np, 8); put(&step, 8);
    std::vector<float> tmp(np);
    std::vector<float *> arrays = {n->params};
    if (with_moments) { arrays.push_back(n->adam_m); arrays.push_back(n->adam_v); }
    for (float *src : arrays) {
        PPE_CUDA_TRY(cudaMemcpy(tmp.data(), src, np * 4, cudaMemcpyDeviceToHost));
        put(tmp.data(), np * 4);
    }
    uint32_t crc = crc32_bytes(buf.data(), buf.size());
    put(&crc, 4);
    FILE *f = std::fopen(path, "wb");
    if (!f) { set_error(std::string("net_save: cannot open ") + path); return PPE_ERR_ARG; }
    size_t w = std::fwrite(buf.data(), 1, buf.size(), f);
    std::fclose(f);
    if (w != buf.size()) { set_error("net_save: short write"); return PPE_ERR_ARG; }
    return PPE_OK;
}

ppe_status net_save(const ppe_net *n, const char *path) { return save_impl(n, path, true); }
ppe_status net_save_params(const ppe_net *n, const char *path) { return save_impl(n, path, false); }

ppe_status net_load(const char *path, ppe_net **out)
{
    clear_error();
    if (!path || !out) { set_error("net_load: NULL argument"); return PPE_ERR_ARG; }
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) { set_error(std::string("net_load: cannot open ") + path); return PPE_ERR_ARG; }
    std::vector<unsigned char> buf;
    unsigned char tmp[1 << 16];
    size_t r;
    while ((r = std::fread(tmp, 1, sizeof tmp, f)) > 0) buf.insert(buf.end(), tmp, tmp + r);
    std::fclose(f);
    const size_t head = 8 + 4 + 4 + sizeof(ppe_net_config) + 16;
    if (buf.size() < head + 4 || std::memcmp(buf.data(), "PPENET01", 8) != 0) {
        set_error("net_load: not a PPENET01 file");
        return PPE_ERR_FORMAT;
    }
    uint32_t crc;
    std::memcpy(&crc, buf.data() + buf.size() - 4, 4);
    if (crc != crc32_bytes(buf.data(), buf.size() - 4)) { set_error("net_load: CRC mismatch"); return PPE_ERR_FORMAT; }
    uint32_t flags;
    std::memcpy(&flags, buf.data() + 12, 4);
    ppe_net_config cfg;
    std::memcpy(&cfg, buf.data() + 16, sizeof cfg);
    int64_t np, step;
    std::memcpy(&np, buf.data() + 16 + sizeof cfg, 8);
    std::memcpy(&step, buf.data() + 24 + sizeof cfg, 8);
    if (!valid_config(cfg)) { set_error("net_load: invalid configuration"); return PPE_ERR_FORMAT; }
    const bool moments = (flags & 1u) != 0;
    ppe_net *n = new ppe_net();
    n->cfg = cfg;
    build_layout(n);
    if (n->nparams != np || buf.size() != head + (size_t)np * (moments ? 12 : 4) + 4) {
        delete n;
        set_error("net_load: size does not match the configuration");
        return PPE_ERR_FORMAT;
    }
    n->host_params.resize(np);
    std::memcpy(n->host_params.data(), buf.data() + head, np * 4);
    ppe_status st = net_alloc(n);
    if (st == PPE_OK) st = upload_params(n);
    if (st == PPE_OK && moments) {
        cudaError_t e1 = cudaMemcpy(n->adam_m, buf.data() + head + np * 4, np * 4, cudaMemcpyHostToDevice);
        cudaError_t e2 = cudaMemcpy(n->adam_v, buf.data() + head + np * 8, np * 4, cudaMemcpyHostToDevice);
        if (e1 != cudaSuccess || e2 != cudaSuccess) st = cuda_status(e1 != cudaSuccess ? e1 : e2, "net_load");
    }
    if (st != PPE_OK) { net_destroy(n); return st; }
    // Without its moments the optimiser restarts: Adam's bias correction and
    // the cosine schedule count from zero again (a fine-tuning run).
    n->step = moments ? step : 0;
    *out = n;
    return PPE_OK;
}

ppe_status net_attach(ppe_net *n, ppe_grid *g)
{
    clear_error();
    if (!n || !g) { set_error("net_attach: NULL argument"); return PPE_ERR_ARG; }
    if (g->net_cache && g->net_owner == n) return PPE_OK;
    net_release_grid(g);
    NetCache *c = nullptr;
    PPE_TRY(make_cache(n, g, &c));
    g->net_cache = c;
    g->net_owner = n;
    n->grids.push_back(g);
    PPE_TRY(refresh_cache(n, c, n->params, 0));
    PPE_CUDA_TRY(cudaDeviceSynchronize());
    return PPE_OK;
}

ppe_status net_infer_batch(ppe_net *n, ppe_grid *g, int batch, const float *r, float *e, void *stream)
{
    clear_error();
    if (!n || !g || !r || !e || batch < 1) { set_error("net_infer: bad arguments"); return PPE_ERR_ARG; }
    PPE_TRY(net_check_grid(n, g));
    NetCache *c = (NetCache *)g->net_cache;
    InputSrc src;
    src.r = r; src.pitch = g->nx; src.bstride = (size_t)g->nx * g->ny; src.nx = g->nx; src.ny = g->ny;
    return net_forward(n, c, batch, src, n->params, e, g->nx, (size_t)g->nx * g->ny, false, (cudaStream_t)stream);
}

ppe_status net_infer(ppe_net *n, ppe_grid *g, const float *r, float *e, void *stream)
{
    return net_infer_batch(n, g, 1, r, e, stream);
}

ppe_status ppe_debug_conv3x3(const void *in, const void *w, const float *bias, int B, int H, int W, int cin, int cout,
                             float *out, int impl, void *stream)
{
    clear_error();
    if (!in || !w || !out || B < 1 || H < 1 || W < 1 || cin < 1 || cout < 1) {
        set_error("ppe_debug_conv3x3: bad arguments");
        return PPE_ERR_ARG;
    }
    ConvArgs a;
    a.in = (const bf16 *)in; a.w = (const bf16 *)w; a.bias = bias;
    a.B = B; a.H = H; a.W = W; a.cin = cin; a.cout = cout;
    a.epi.zf_out = out;
    a.epi.act = 0;
    if (impl == 0) {
        if (!conv3x3_tc_supported(a)) {
            set_error("ppe_debug_conv3x3: shape not supported by the tensor-core kernel");
            return PPE_ERR_ARG;
        }
        return conv3x3_tc(a, (cudaStream_t)stream);
    }
    return conv3x3_simt(a, (cudaStream_t)stream);
}

}  // extern "C"
