// Network object, per-grid caches and the functions shared by net.cu and the
// training module.
#pragma once

#include <atomic>
#include <string>
#include <vector>

#include "net_internal.h"
#include "net_ops.h"

namespace ppe {

// Offsets (BF16 elements) of the activation buffers of one batch.
struct ActPlan {
    size_t A[PPE_NET_MAX_LEVELS] = {};    // input of enc{k}b (eta-weighted)
    size_t IN[PPE_NET_MAX_LEVELS] = {};   // pooled input of enc{k}a (k >= 1, eta-weighted)
    size_t P[PPE_NET_MAX_LEVELS] = {};    // raw output of enc{k}b (to pooling)
    size_t CAT[PPE_NET_MAX_LEVELS] = {};  // [up{k} out | enc{k}b out] (eta-weighted), input of dec{k}a
    size_t UP[PPE_NET_MAX_LEVELS] = {};   // up-sampled input of up{k} (eta-weighted)
    size_t D[PPE_NET_MAX_LEVELS] = {};    // input of dec{k}b (eta-weighted)
    size_t U[PPE_NET_MAX_LEVELS] = {};    // raw output of dec{k}b (U[L-1]: enc{L-1}b)
    std::vector<size_t> Z;                // pre-activation of every layer
    size_t total = 0;
};

struct NetCache {
    ppe_net *net = nullptr;
    uint64_t version = 0;
    const float *src = nullptr;
    int nx = 0, ny = 0, H = 0, W = 0, L = 0;
    int Hk[PPE_NET_MAX_LEVELS] = {}, Wk[PPE_NET_MAX_LEVELS] = {};
    float *delta = nullptr;                 // distance maps, all levels
    size_t doff[PPE_NET_MAX_LEVELS] = {};
    float *eta = nullptr, *phi = nullptr;   // per layer
    std::vector<size_t> eoff;
    float *xy = nullptr, *trunk = nullptr, *weff = nullptr, *ceff = nullptr;
    bf16 *act = nullptr;
    int capB = 0;
    ActPlan plan;
    // training scratch
    float *grad_act = nullptr;
    size_t grad_elems = 0;
    float *efull = nullptr;
    size_t efull_elems = 0;
    double *red = nullptr;
    void *train = nullptr;                  // training workspace (net_train.cu)
    // CUDA graph of the DLSM-direction forward (input: the solver state)
    cudaGraphExec_t dir_exec = nullptr;
    uint64_t dir_version = 0;
    const void *dir_key = nullptr;
    const void *dir_act = nullptr;          // activation buffer the graph was captured with
    cudaStream_t cap_stream = nullptr;
};

void net_free_train(NetCache *c);

int layer_index(const ppe_net *n, const std::string &name);
ppe_status ensure_packed(ppe_net *n, const float *P, cudaStream_t s);
ppe_status refresh_cache(ppe_net *n, NetCache *c, const float *P, cudaStream_t s);
ppe_status ensure_acts(ppe_net *n, NetCache *c, int B);
ppe_status run_conv(ppe_net *n, const ConvArgs &a, cudaStream_t s);
ppe_status net_forward(ppe_net *n, NetCache *c, int B, const InputSrc &src, const float *P, float *e, int e_pitch,
                       size_t e_bstride, bool keep_z, cudaStream_t s);

}  // namespace ppe

// Parameter versions are unique across the process: a network's versions
// start at a serial of its own (upper 32 bits), so a graph or cache keyed by
// (pointer, version) never matches a later network that happens to reuse a
// freed network's memory.
inline uint64_t net_version_base()
{
    static std::atomic<uint64_t> serial{0};
    return (serial.fetch_add(1) + 1) << 32;
}

struct ppe_net {
    ppe_net_config cfg{};
    std::vector<ppe::ConvLayer> layers;
    int64_t off_head_w = 0, off_head_b = 0, off_tw[3] = {}, off_tb[3] = {}, off_out_b = 0;
    int64_t nparams = 0, npacked = 0;
    std::vector<float> host_params;
    float *params = nullptr, *grads = nullptr, *grads2 = nullptr, *params_pert = nullptr;
    float *adam_m = nullptr, *adam_v = nullptr;
    ppe::bf16 *wp = nullptr, *wt = nullptr;
    double *scratch = nullptr;
    uint64_t version = net_version_base() + 1, packed_version = 0;
    const float *packed_src = nullptr;
    int64_t step = 0;
    bool use_tc = true;
    std::vector<ppe_grid *> grids;
};
