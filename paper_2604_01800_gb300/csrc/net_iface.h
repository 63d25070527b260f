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

}  // namespace ppe
