// Placeholder network hooks until the network module is built.
#include "net_iface.h"

namespace ppe {
void net_release_grid(ppe_grid *) {}
ppe_status net_check_grid(ppe_net *, ppe_grid *) { set_error("network module not built"); return PPE_ERR_NO_NET; }
ppe_status net_direction(ppe_net *, ppe_grid *, const SysDesc *, const SysState *, bool, cudaStream_t, float *)
{
    set_error("network module not built");
    return PPE_ERR_NO_NET;
}
}  // namespace ppe
