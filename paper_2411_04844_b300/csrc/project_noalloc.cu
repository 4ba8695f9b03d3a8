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
// per device (with that device current) and cached.  The cache is keyed by
// device ordinal: after cudaDeviceReset (which unloads the module) or under a
// context other than the device's primary one the cached address is stale.
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

// Ray-table entries (one per view x detector column) the array can hold.
constexpr long long MAX_TABLE_ENTRIES = DGR_NOALLOC_SCRATCH_BYTES / (long long)sizeof(dgr::RayXY);

}  // namespace

extern "C" int dgr_project_noalloc(const dgr_grid *grid, const dgr_geom *geom, const float *vol,
                                   float *sino, cudaStream_t stream) {
    // the same validation as dgr_project (shared validators)
    if (!dgr::grid_ok(grid) || !dgr::geom_ok(geom) || !vol || !sino) return DGR_ERR_ARG;
    if (!dgr::geom_fits_grid(grid, geom)) return DGR_ERR_ARG;
    if ((long long)grid->nx * grid->ny * grid->nz >= (1ll << 31)) return DGR_ERR_ARG;
    // scratch capacity, in 64-bit counts before any int arithmetic on the tables
    if ((long long)geom->n_views * geom->nu > MAX_TABLE_ENTRIES ||
        dgr::ray_table_bytes_single(*geom) > (size_t)DGR_NOALLOC_SCRATCH_BYTES)
        return DGR_ERR_WS_TOO_SMALL;
    void *scratch = nullptr;
    if (scratch_of_current_device(&scratch) != cudaSuccess) return DGR_ERR_CUDA;
    dgr::RayXY *tab = static_cast<dgr::RayXY *>(scratch);
    const cudaError_t e = dgr::launch_project_single(*grid, *geom, tab, vol, sino, stream);
    return e == cudaSuccess ? DGR_OK : DGR_ERR_CUDA;
}
