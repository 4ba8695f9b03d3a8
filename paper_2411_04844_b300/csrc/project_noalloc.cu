// dgr_project_noalloc: the projector of dgr_project for callers that cannot
// allocate device memory.  Its only scratch -- the per-(view, detector column)
// and per-row ray tables -- lives in a fixed file-scope device array instead of
// a dgr_ws, so a call needs no workspace and allocates nothing.
#include <math.h>

#include <mutex>

#include "dgr_internal.cuh"

namespace {

// Fixed scratch, DGR_NOALLOC_SCRATCH_BYTES, held by every device that loads
// this library until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[DGR_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
void *g_scratch_ptr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device.  The array's
// name is a host-side stand-in in host code, so the address is looked up once
// per device (with that device current) and cached.
cudaError_t scratch_of_current_device(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

bool args_ok(const dgr_grid *g, const dgr_geom *geo, const float *vol, const float *sino) {
    if (!g || !geo || !vol || !sino || !geo->angles) return false;
    if (g->nx <= 0 || g->ny <= 0 || g->nz <= 0 || g->nx > 32767 || g->ny > 32767 || g->nz > 32767)
        return false;
    if (!isfinite(g->h) || !(g->h > 0.f) || !isfinite(g->ox) || !isfinite(g->oy) || !isfinite(g->oz))
        return false;
    if (geo->beam != DGR_PARALLEL && geo->beam != DGR_CONE) return false;
    if (geo->n_views <= 0 || geo->nu <= 0 || geo->nv <= 0) return false;
    if (!(isfinite(geo->pu) && geo->pu > 0.f && isfinite(geo->pv) && geo->pv > 0.f)) return false;
    if (geo->beam == DGR_CONE) {
        if (!(isfinite(geo->dso) && isfinite(geo->dsd) && geo->dso > 0.f && geo->dsd > geo->dso))
            return false;
        // the grid must lie strictly inside the source circle
        const double o[2] = {g->ox, g->oy}, e[2] = {g->nx * (double)g->h, g->ny * (double)g->h};
        double r2 = 0;
        for (int a = 0; a < 2; ++a) {
            const double m = fmax(fabs(o[a]), fabs(o[a] + e[a]));
            r2 += m * m;
        }
        if (!(sqrt(r2) < 0.999 * geo->dso)) return false;
    }
    return true;
}

}  // namespace

extern "C" int dgr_project_noalloc(const dgr_grid *grid, const dgr_geom *geom, const float *vol,
                                   float *sino, cudaStream_t stream) {
    if (!args_ok(grid, geom, vol, sino)) return DGR_ERR_ARG;
    if (dgr::ray_table_bytes_single(*geom) > (size_t)DGR_NOALLOC_SCRATCH_BYTES)
        return DGR_ERR_WS_TOO_SMALL;
    if ((long long)grid->nx * grid->ny * grid->nz >= (1ll << 31)) return DGR_ERR_ARG;
    void *scratch = nullptr;
    if (scratch_of_current_device(&scratch) != cudaSuccess) return DGR_ERR_CUDA;
    dgr::RayXY *tab = static_cast<dgr::RayXY *>(scratch);
    const cudaError_t e = dgr::launch_project_single(*grid, *geom, tab, vol, sino, stream);
    return e == cudaSuccess ? DGR_OK : DGR_ERR_CUDA;
}
