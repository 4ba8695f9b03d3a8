// Internal definitions of libdgr (sm_103a).  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <utility>

#include "dgr.h"

namespace dgr {

// CTAs of one full wave of `kernel` on the current device (SMs x CTAs resident
// per SM at `threads` threads and `smem` dynamic shared bytes), looked up once
// per (device, kernel) and cached: launches do not query the device each time.
int wave_ctas(const void *kernel, int threads, size_t smem);

// Host-side argument validators (api.cu), shared by every entry point.
// slab_origin: the z origin of a slab's first layer, oz + z0 h (FP64, rounded once)
inline float slab_origin(const dgr_grid &g) { return (float)((double)g.oz + (double)g.z0 * (double)g.h); }
constexpr int MAX_DIM = 32767;          // grid side
constexpr int MAX_VIEWS_BP = 1 << 20;   // views of one geometry
bool grid_ok(const dgr_grid *g);
bool geom_ok(const dgr_geom *geo);
bool geom_fits_grid(const dgr_grid *g, const dgr_geom *geo);  // cone: grid inside the source circle

// Voxel tile of the forward voxelizer: 8 (x) x 16 (y) x 32 (z).  A CTA of four
// warps owns one tile; a warp owns an 8 x 4 patch in (x, y) and every lane
// keeps the 32 z-voxels of its (x, y) column in registers, so the per-Gaussian
// set-up of a lane is shared by up to 32 exponentials.
constexpr int TX = 8, TY = 16;
constexpr int TZ_MAX = 32;  // tile depth: 8, 16 or 32 (dgr_set_tile_depth; the autotuner's knob)
constexpr int TZG = 8;      // z handled in groups of 8 (a group outside the box is skipped)
int tile_depth();           // current tile depth
void set_tile_depth(int tz);
constexpr int VOX_THREADS = 128;
constexpr int VOX_CHUNK = 64;  // prep records staged in shared memory at a time

// Long tile lists are cut into segments taken by different CTAs (a grid of
// few tiles, each in the boxes of thousands of Gaussians, would otherwise
// leave most SMs idle): each segment's sums go to a partial slot of
// TZ_MAX x VOX_THREADS floats, the CTA finishing a tile's last segment adds
// the slots in segment order.  Per instance at most SPLIT_BUDGET slots; a
// tile splits into at most SPLIT_SMAX segments of at least SPLIT_LMIN list
// entries (see plan_tile).
constexpr int SPLIT_BUDGET = 1024;
constexpr int SPLIT_SMAX = 16;
constexpr int SPLIT_LMIN = 256;
constexpr int VOX_SLOT = TZ_MAX * VOX_THREADS;
// status-word slots: the voxelizer's unit queue head, the count of extra
// units (segments after the first of split tiles), per-instance slot counters
constexpr int VOX_QUEUE = 18, VOX_NEXTRA = 19, VOX_SLOTCTR = 20;  // .. VOX_SLOTCTR + MAX_INST - 1
// workspace ints of the split plan for `tiles` tiles and `ninst` instances:
// nseg [tiles] | slot [tiles] | done [tiles] | extra [ninst SPLIT_BUDGET]
inline size_t split_plan_ints(long long tiles, int ninst) {
    return (size_t)(3 * tiles + (long long)ninst * SPLIT_BUDGET);
}
struct VoxSplit {
    int *nseg;   // segments of each tile (1: not split)
    int *slot;   // first partial slot of a split tile (-1: not split)
    int *done;   // segments of a split tile finished
    int *extra;  // extra units: tile | segment << 24 (segments 1 .. nseg - 1 of split tiles)
    int *ctr;    // [0] extra units; [1 + i] partial slots taken by instance i
    float *part; // partial slots
};
inline VoxSplit vox_split_of(int *ints, float *part, int *status, long long tiles) {
    VoxSplit S;
    S.nseg = ints;
    S.slot = ints + tiles;
    S.done = S.slot + tiles;
    S.extra = S.done + tiles;
    S.ctr = status + VOX_NEXTRA;
    S.part = part;
    return S;
}

// Backward work item: a piece of one Gaussian's box holding at most about
// ITEM_VOX voxels (see item_count), processed by one warp.
constexpr int ITEM_VOX = 2048;
constexpr int NMOM = 10;  // moments per item: S0, S1[3], S2[6]

// Work items of the backward pass cover a box of ex * ey * ez voxels: a
// warp's lanes take the (x, y) columns of the item and walk its z range, so
// the z range is kept long (the per-column set-up is paid once per column):
//   zc = min(ez, max(1, ITEM_VOX / ex)) layers, yc = min(ey, max(1, ITEM_VOX /
//   (ex zc))) rows; items are the ceil(ey / yc) x ceil(ez / zc) blocks.
// a / b for 0 <= a, 1 <= b (exact); on the device for operands below 2^20 by a
// float reciprocal and one correction (the estimate is within 0.25 of a / b),
// else by the integer division
__host__ __device__ inline int div_small(int a, int b) {
#ifdef __CUDA_ARCH__
    if (a < (1 << 20) && b < (1 << 20)) {
        int q = (int)((float)a * __frcp_rn((float)b));
        const int r = a - q * b;
        if (r < 0) --q;
        else if (r >= b) ++q;
        return q;
    }
#endif
    return a / b;
}
__host__ __device__ inline void item_shape(int ex, int ey, int ez, int &yc, int &zc) {
    const int zmax = div_small(ITEM_VOX, ex);
    zc = ez < zmax ? ez : (zmax > 1 ? zmax : 1);
    const int xz = ex * zc;  // <= max(ITEM_VOX, ex)
    yc = xz < ITEM_VOX ? div_small(ITEM_VOX, xz) : 1;
    if (yc > ey) yc = ey;
}
__host__ __device__ inline uint32_t item_count(int ex, int ey, int ez) {
    if (ex <= 0 || ey <= 0 || ez <= 0) return 0u;
    int yc, zc;
    item_shape(ex, ey, ez, yc, zc);
    return (uint32_t)div_small(ey + yc - 1, yc) * (uint32_t)div_small(ez + zc - 1, zc);
}
// item c of a box with lower corner (ly, lz) and upper (hy, hz): y and z ranges
__host__ __device__ inline void item_range(int c, int ex, int ey, int ly, int hy, int lz, int hz,
                                           int &yb, int &ye, int &zb, int &ze) {
    int yc, zc;
    item_shape(ex, ey, hz - lz + 1, yc, zc);
    const int nyc = div_small(ey + yc - 1, yc);
    const int zi = div_small(c, nyc);
    yb = ly + (c - zi * nyc) * yc;
    ye = min(yb + yc - 1, hy);
    zb = lz + zi * zc;
    ze = min(zb + zc - 1, hz);
}

// log2(e): the exponent exp(-x/2) is evaluated as ex2(-x/2 * log2(e)).
constexpr float LOG2E = 1.4426950408889634f;

// Per-Gaussian record written by the prep kernel (96 bytes, 6 x 16).
// The exponent -1/2 log2(e) d^T A d is kept in column form: along the z column
// through (dx, dy) it peaks at dz* = zx dx + zy dy with the value
//     qmin = l1 (n1 . (dx, dy))^2 + l2 (n2 . (dx, dy))^2,
// n1 = (n1x, n1y), n2 = (-n1y, n1x) and l1, l2 the principal axes and values of
// (Sigma_xy)^-1 (scaled), and
//     q(dz) = qmin + a22 (dz - dz*)^2,
// a sum of terms <= 0: no cancellation however far the peak lies from the
// centre plane.  The FP64 copies of n1 and (zx, zy) let a caller evaluate the
// principal coordinates and the peak at a point far from the centre (a tile's
// centre) in FP64 once, so that lanes add only small FP32 offsets.  For a
// diagonal A: n1 = (1, 0), l1 = the x and l2 the y coefficient, zx = zy = 0.
struct __align__(16) Prep {
    float dx, dy, dz, rho;      // delta = u - a (voxel units), intensity
    float l1, l2, a22, n1x;     // x -1/2 log2(e): principal values of (Sigma_xy)^-1, A_zz
    float zx, zy;               // the column's peak: dz* = zx dx + zy dy
    int ax, ay;                 // anchor a = floor(u)
    int az;
    int bx, by, bz;             // box per axis: lo | hi << 16 (lo > hi: empty)
    double n1x_d, n1y_d;        // n1 in FP64
    double zx_d, zy_d;          // (zx, zy) in FP64
};
static_assert(sizeof(Prep) == 96, "Prep must be 96 bytes");

__host__ __device__ inline int box_lo(int p) { return (int)(short)(p & 0xffff); }
__host__ __device__ inline int box_hi(int p) { return (int)(short)((unsigned)p >> 16); }
__host__ __device__ inline int box_pack(int lo, int hi) {
    return (int)(((unsigned)lo & 0xffffu) | (((unsigned)hi & 0xffffu) << 16));
}

// Per (view, iu) ray data of the projector: the ray is X(t) = X0 + t D with
// X0 the point of the (x, y) line closest to the grid axis.  xi = (X - o)/h
// is the continuous voxel coordinate; e = D / h.
struct __align__(16) RayXY {
    float xi0x, xi0y, ex, ey;
    float inv_ex, inv_ey, tc, dxy2;  // 1/e (0 when e == 0), t-shift for z, |D_xy|^2
};

// Per detector row: zv = v / h (FP32), its reciprocal (0 when zv == 0), the
// FP64-snapped z layer used when the ray runs parallel to the z planes, and v.
struct __align__(16) RowZ {
    float zv, izv, zsnap, v;
};

// ---------------------------------------------------------------------------
// Batches: every kernel works on a batch of independent problems described by
// a struct passed by value (kernel parameter space, so a captured CUDA graph
// keeps it).  Global index spaces (Gaussians, tiles, rays, backprojector
// blocks, backward items) run over all instances back to back; a single call
// of the C ABI is a batch of one.
// ---------------------------------------------------------------------------
constexpr int MAX_INST = 16;
// status block (256 bytes of the workspace): [0] device status flags,
// [16] voxelizer tile queue head, [17] set when a Gaussian is not separable
constexpr int SEP_FLAG = 17;
constexpr int BIG_COUNT = 18;  // status word: Gaussians of the adjoint with more than BIG_ITEMS items
constexpr int ITEM_QUEUE = 19;  // status word: next run of the adjoint's work items (zeroed with BIG_COUNT)
constexpr int BIG_ITEMS = 256;

struct Inst {
    dgr_grid g;                       // the grid as the kernels see it: a z-slab's origin
                                      // moved to its first layer, z0 = 0
    int z0;                           // the slab's first layer in the whole grid
    float oz_full;                    // the whole grid's z origin (footprint frame)
    int beam, n_views, nu, nv;
    float pu, pv, dso, dsd;
    const float *angles;
    float k, zoff;  // truncation factor; -oz / h
    // Gaussians of this instance (device arrays, local index)
    const float *mu, *s, *q, *rho;
    float *g_mu, *g_s, *g_q, *g_rho;  // adjoint outputs
    int g0, n;                        // first global Gaussian, count
    int tile0, ntx, nty, ntz;         // first global tile, tiles per axis
    long long ray0;                   // first global ray
    int tab0, view0, row0;            // first RayXY entry, view, RowZ entry
    int blk0, nbx, nbz;               // column backprojector: first CTA, CTAs in x, z passes
    int bb0, nbbx, nbby, nbbz;        // brick backprojector: first brick, bricks per axis
    int col_u, col_v;                 // ray colour classes (footprint < col pixels)
    int multiz;                       // a ray may cross two z planes inside one (x, y) cell
    int pb0, npv;                     // projector / ray scatter: first CTA, row groups
    int kv0, nkv;                     // views of this launch (ray scatter: one view group)
    int fb0;                          // ray scatter fold: first tile
    int *acc;                         // ray scatter: integer sums (z fastest)
    int vsx, vsy, vsz;                // element strides of vol as voxelize output / project input
    float *vol;                       // volume (voxelize output, project input)
    float *gvol;                      // volume gradient, x fastest (backproject output, FVR adjoint input)
    float w_l1, w_ssim, w_tv;         // objective weights
    float ssim_c1, ssim_c2;           // SSIM constants
    int st0, nst, tv0, ntv;           // SSIM tiles, TV tiles: first and count
    float *sino;                      // projection (step: prediction, then residual)
    const float *meas;                // measured projections (step)
    float *loss;                      // loss scalar (step)
    // optimiser state and constants (step)
    float *theta, *m, *v;
    int *step;
    float *mu_w, *s_w, *q_w, *rho_w;  // parameters rewritten by Adam
    float *gacc;                      // optional |dL/dmu| accumulator (densification)
    float lr0, lr1, b1, b2, eps;
    int n_iters;
};

struct Batch {
    int n;             // instances
    int tz;            // voxelizer tile depth
    int tot_g;         // Gaussians of all instances
    int tot_tiles;
    int tot_tab, tot_rows, tot_views;
    int tot_blk;
    int tot_bricks;
    int tot_st, tot_tv;  // SSIM and TV tiles
    int tma_ch, tma_zcap;  // staged path walk: cells per stage, words per cell column
    int *status;           // device status word (bounded waits flag timeouts)
    float ssim_w[11];    // SSIM window taps
    long long tot_rays;
    Inst in[MAX_INST];
};

// instance owning a global index (linear scan of at most MAX_INST entries)
__device__ __forceinline__ int inst_of_g(const Batch &B, int g) {
    int i = 0;
    while (i + 1 < B.n && B.in[i + 1].g0 <= g) ++i;
    return i;
}
__device__ __forceinline__ int inst_of_tile(const Batch &B, int t) {
    int i = 0;
    while (i + 1 < B.n && B.in[i + 1].tile0 <= t) ++i;
    return i;
}
__device__ __forceinline__ int inst_of_ray(const Batch &B, long long r) {
    int i = 0;
    while (i + 1 < B.n && B.in[i + 1].ray0 <= r) ++i;
    return i;
}
__device__ __forceinline__ int inst_of_view(const Batch &B, int v) {
    int i = 0;
    while (i + 1 < B.n && B.in[i + 1].view0 <= v) ++i;
    return i;
}
__device__ __forceinline__ int inst_of_blk(const Batch &B, int b) {
    int i = 0;
    while (i + 1 < B.n && B.in[i + 1].blk0 <= b) ++i;
    return i;
}

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// host-side count of kernel launches issued by the library
extern std::atomic<long long> g_launches;
inline void counted(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// Programmatic dependent launch.  A kernel launched by launch_dep may be
// scheduled onto the SMs while the work before it in the stream is still
// draining; DEP_ENTER, the first statement of every such kernel, waits until
// that work has completed and its memory is visible (griddepcontrol.wait),
// then lets the next kernel in the stream be scheduled in turn
// (griddepcontrol.launch_dependents).  Nothing before DEP_ENTER touches
// global memory, so the order of every read and write is that of plain
// stream order; only the launch latency and the tail of each kernel are
// overlapped.  Launched without the attribute, both instructions do nothing.
#define DEP_ENTER()                                                   \
    do {                                                              \
        asm volatile("griddepcontrol.wait;" ::: "memory");             \
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); \
    } while (0)

// Bounds-checked build (-DDGR_CHECK_BOUNDS, libdgr_checked.so): the volume,
// integer-sum and gradient accesses of the walks, the FVR adjoint and the
// voxelizer's record loads test their index against the buffer's size; an
// index outside it sets DGR_STATUS_BOUNDS in the status word and the access
// is skipped (a load reads 0), so a bad index is reported instead of faulting.
// In the default build DGR_INB is the constant true and the code is unchanged.
#ifdef DGR_CHECK_BOUNDS
__device__ __forceinline__ bool dgr_inb(long long i, long long n, int *status) {
    if ((unsigned long long)i < (unsigned long long)n) return true;
    if (status) atomicOr(status, DGR_STATUS_BOUNDS);
    return false;
}
#define DGR_INB(i, n, status) dgr_inb((long long)(i), (long long)(n), (status))
#else
#define DGR_INB(i, n, status) true
#endif

template <typename... P, typename... A>
inline cudaError_t launch_dep(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              A &&...args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

}  // namespace dgr

// Workspace: one device arena and the plan that fixed its layout.
struct dgr_ws {
    char *base;
    size_t bytes;
    dgr_ws_plan plan;
    // byte offsets into base
    size_t status, prep, itemcnt, item_off, tile_cnt, tile_off, tile_fill, scan_tmp, list,
        partials, grads, vol, sino, loss_part, rayxy, sino_scaled, losses, list_tmp, acc, gvol, ssim_maps,
        ssim_g, ssim_part, tv_part, dens, vsplit, vpart;
    size_t scan_tmp_elems;
};

namespace dgr {
template <class T>
inline T *ws_ptr(dgr_ws *ws, size_t off) { return reinterpret_cast<T *>(ws->base + off); }

// scan.cu
// Exclusive scan of len uint32 counts into out[0..len] (out[len] = total).
// If the total exceeds cap, `flag` is OR-ed into *status and out[len] keeps
// the (saturated) total.
cudaError_t scan_u32(const uint32_t *in, uint32_t *out, int len, unsigned long long cap,
                     int *status, int flag, unsigned long long *tmp, cudaStream_t st);
size_t scan_tmp_elems(int len);

// voxelize.cu
int tile_dims(const dgr_grid &g, int &ntx, int &nty, int &ntz);
cudaError_t launch_prep(const Batch &B, Prep *prep, uint32_t *itemcnt, int *status, cudaStream_t st);
cudaError_t launch_count_pairs(const Batch &B, const Prep *prep, dgr_ws *ws, unsigned long long cap,
                               cudaStream_t st);
cudaError_t launch_voxelize(const Batch &B, const Prep *prep, dgr_ws *ws, int deterministic,
                            cudaStream_t st, const cudaEvent_t *kev = nullptr);
cudaError_t launch_footprint(const dgr_grid &g, int n, const float *mu, const float *s,
                             const float *q, float k, int *anchor, int *box, cudaStream_t st);

// voxelize_bwd.cu (grad_vol = Inst::vol; outputs Inst::g_*)
// kev (optional): two events recorded right before / after the main kernel
cudaError_t launch_voxelize_backward(const Batch &B, const Prep *prep, dgr_ws *ws, cudaStream_t st,
                                     const cudaEvent_t *kev = nullptr);

// project.cu
size_t ray_table_bytes(long long n_tab, long long n_views, long long n_rows);
cudaError_t launch_ray_tables(const Batch &B, RayXY *tab, cudaStream_t st);
// kev (optional): two events recorded right before / after the main kernel
cudaError_t launch_project(const Batch &B, const RayXY *tab, int *status, cudaStream_t st,
                           const cudaEvent_t *kev = nullptr);
void set_staged_walk(int on);
// x-fastest -> z-fastest copy of a volume (the row-warp projector's layout)
cudaError_t launch_vol_zfast(const dgr_grid &g, const float *src, float *dst, cudaStream_t st);
// sino_scaled: scratch of all instances' rays (residual x |D|, [view][u][v]); not aliasing sino
// densify.cu: adaptive density control; counts_dev: device int[3] (n_clone, n_split, n_out)
cudaError_t launch_densify(const dgr_grid &g, const dgr_densify_cfg &cfg, int iters, const dgr_params &in,
                           const float *normals, const dgr_params &out, dgr_ws *ws, int *counts_dev,
                           cudaStream_t st);
// loss.cu: SSIM and TV terms of the objective
void ssim_window(float *w);
void loss_tiles(Batch &B);
size_t ssim_tiles_cap(long long max_views, int max_nu, int max_nv, int ninst);
size_t tv_tiles_cap(long long max_vox, int ninst);
cudaError_t launch_ssim(const Batch &B, float *maps, float *spart, float *gout, cudaStream_t st);
cudaError_t launch_tv(const Batch &B, float *tpart, int accumulate, cudaStream_t st);
cudaError_t launch_loss_final(const Batch &B, const float *l1part, int l1_blocks, const float *spart,
                              const float *tpart, cudaStream_t st);
// acc: the workspace's integer sums (ray scatter), room for acc_vox voxels
cudaError_t launch_backproject(const Batch &B, const RayXY *tab, float *sino_scaled, int *acc,
                               long long acc_vox, int *status, cudaStream_t st,
                               const cudaEvent_t *kev = nullptr);
// the projector of one instance with caller-provided tables (no workspace)
cudaError_t launch_project_single(const dgr_grid &g, const dgr_geom &geo, RayXY *tab,
                                  const float *vol, float *sino, cudaStream_t st);
size_t ray_table_bytes_single(const dgr_geom &geo);  // 64-bit sizes: no wrap-around
// backprojector CTAs covering a grid (x blocks of 8 columns x ny x z passes)
int bp_blocks(const dgr_grid &g, int &nbx, int &nbz);
// brick backprojector: bricks per axis and the ray colour classes of a geometry
int bp_bricks(const dgr_grid &g, int &nbx, int &nby, int &nbz);
int multi_z(const dgr_geom &geo);
void set_separable(int on);
void bp_colours(const dgr_grid &g, const dgr_geom &geo, int &cu, int &cv);
int backprojector_variant();
void set_backprojector_variant(int v);

// step.cu
constexpr int L1_BLOCKS = 148 * 8;  // per instance (8 per SM); fixed so the loss reduction order is fixed
cudaError_t launch_l1(const Batch &B, float *part, const float *gadd, cudaStream_t st);
cudaError_t launch_l1_single(const float *pred, const float *meas, long long m, float w, float *resid,
                             float *loss, float *part, cudaStream_t st);
cudaError_t launch_params_init(const dgr_problem &P, const dgr_params &p, cudaStream_t st);
cudaError_t launch_adam(const Batch &B, cudaStream_t st);
}  // namespace dgr
