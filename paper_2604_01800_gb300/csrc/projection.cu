// The projection step around the PPE (Sec. 2.1): the source of Eq. 6 from a
// staggered intermediate velocity, and the correction of Eqs. 7-8.
//
// Staggered (MAC) layout, FP64, row-major: u [ny][nx+1] on the x faces
// (face i of row j lies between cells i-1 and i), v [ny+1][nx] on the y
// faces, p and dp [ny][nx] at cell centres.  The wall faces carry the
// prescribed normal velocity: their contribution to the divergence of u* is
// the known part bc2 of Eq. 6, and Eq. 7 does not change them (which is what
// makes dp's boundary condition homogeneous Neumann).  D G is then exactly
// the PPE operator M of the solver, and the source that makes u^{n+1}
// divergence free, walls included, is the whole divergence of u* over dt.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

namespace ppe {

namespace {

// S = divergence of the face field (wall faces included) / dt
__global__ void source_kernel(int nx, int ny, const double *__restrict__ dx, const double *__restrict__ dy,
                              const double *__restrict__ u, const double *__restrict__ v, double inv_dt,
                              double *__restrict__ S)
{
    const size_t n = (size_t)nx * ny;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(k % nx), j = (int)(k / nx);
        const size_t fu = (size_t)j * (nx + 1) + i, fv = (size_t)j * nx + i;
        S[k] = ((u[fu + 1] - u[fu]) / dx[i] + (v[fv + nx] - v[fv]) / dy[j]) * inv_dt;
    }
}

// u -= dt G dp on the interior x faces, v likewise on the interior y faces,
// p += dp at the cells; one index space over all three.
__global__ void project_kernel(int nx, int ny, const double *__restrict__ dx, const double *__restrict__ dy,
                               const double *__restrict__ dp, double dt, double *__restrict__ u,
                               double *__restrict__ v, double *__restrict__ p)
{
    const size_t nu = (size_t)ny * (nx + 1), nv = (size_t)(ny + 1) * nx, nc = (size_t)nx * ny;
    const size_t total = nu + nv + (p ? nc : 0);
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        if (k < nu) {
            const int i = (int)(k % (nx + 1)), j = (int)(k / (nx + 1));
            if (i == 0 || i == nx) continue;
            const size_t c = (size_t)j * nx + i;
            u[k] -= dt * (dp[c] - dp[c - 1]) / (0.5 * (dx[i - 1] + dx[i]));
        } else if (k < nu + nv) {
            const size_t f = k - nu;
            const int i = (int)(f % nx), j = (int)(f / nx);
            if (j == 0 || j == ny) continue;
            const size_t c = (size_t)j * nx + i;
            v[f] -= dt * (dp[c] - dp[c - nx]) / (0.5 * (dy[j - 1] + dy[j]));
        } else {
            const size_t c = k - nu - nv;
            p[c] += dp[c];
        }
    }
}

unsigned blocks_for(size_t n)
{
    size_t b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 16384 ? 16384 : b));
}

}  // namespace

}  // namespace ppe

using namespace ppe;

extern "C" {

ppe_status ppe_source(ppe_grid *g, const double *u, const double *v, double dt, double *S, void *stream)
{
    clear_error();
    if (!g || !u || !v || !S || !(dt > 0.0) || !std::isfinite(dt)) {
        set_error("ppe_source: NULL argument or dt not positive");
        return PPE_ERR_ARG;
    }
    const size_t n = (size_t)g->nx * g->ny;
    source_kernel<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(g->nx, g->ny, g->dx, g->dy, u, v, 1.0 / dt, S);
    PPE_CUDA_TRY(cudaGetLastError());
    return PPE_OK;
}

ppe_status ppe_project(ppe_grid *g, const double *dp, double dt, double *u, double *v, double *p, void *stream)
{
    clear_error();
    if (!g || !dp || !u || !v || !(dt > 0.0) || !std::isfinite(dt)) {
        set_error("ppe_project: NULL argument or dt not positive");
        return PPE_ERR_ARG;
    }
    const size_t n = (size_t)g->ny * (g->nx + 1) + (size_t)(g->ny + 1) * g->nx + (p ? (size_t)g->nx * g->ny : 0);
    project_kernel<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(g->nx, g->ny, g->dx, g->dy, dp, dt, u, v, p);
    PPE_CUDA_TRY(cudaGetLastError());
    return PPE_OK;
}

}  // extern "C"
