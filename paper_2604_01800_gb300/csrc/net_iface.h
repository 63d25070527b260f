// Interface between the solver driver and the network module.
#pragma once

#include "internal.h"

namespace ppe {

// Free whatever per-grid caches a network attached to this grid.
void net_release_grid(ppe_grid *g);
// PPE_OK if `net` has been attached to `g` (net_attach), else an error.
ppe_status net_check_grid(ppe_net *net, ppe_grid *g);
// Run the network on the current residual of system `st` (device state) and
// write the DLSM direction into the grid's direction buffer.  `ms` receives
// the elapsed time of the inference on `stream`.
ppe_status net_direction(ppe_net *net, ppe_grid *g, const SysDesc *sd_dev, const SysState *st_dev,
                         bool fp64_inner, cudaStream_t stream, float *ms);
// Bring the packed weights, the grid's caches and its activation buffers up
// to date for directions (kernels on `stream`; call outside any capture).
ppe_status net_prepare_direction(ppe_net *net, ppe_grid *g, cudaStream_t stream);
// Enqueue the direction's launches for system (sd_dev, st_dev) on a stream
// that is being captured (after net_prepare_direction): the forward pass on
// the normalised residual, then the mean removal of e.
ppe_status net_record_direction(ppe_net *net, ppe_grid *g, const SysDesc *sd_dev, const SysState *st_dev,
                                cudaStream_t stream);
// Key of what a captured direction of this grid bakes in (parameter version,
// activation buffers); a changed key means the capture must be redone.
uint64_t net_direction_key(const ppe_net *net, const ppe_grid *g);

}  // namespace ppe
