/*
 * dgr.h -- C ABI of the B300 (sm_103a) hot path of Discretized Gaussian
 * Representation (DGR, arxiv 2411.04844): Fast Volume Reconstruction (FVR),
 * the X-ray projector, their adjoints and one optimisation step.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Array arguments are DEVICE pointers to contiguous FP32 (or int32)
 *    memory owned by the caller; descriptor structs and the scalars they hold
 *    live in HOST memory and are read before the call returns.
 *  - Volumes are [nz][ny][nx] (x fastest).  Voxel (i, j, k) has its centre at
 *    (ox + (i + 1/2) h, oy + (j + 1/2) h, oz + (k + 1/2) h).
 *  - Sinograms are [n_views][nv][nu] (u fastest).
 *  - Gaussian parameters: mu [n][3] world units; s [n][3] per-axis standard
 *    deviations, world units, > 0; q [n][4] rotation quaternion (w, x, y, z),
 *    need not be normalised (it is normalised inside); rho [n] intensity
 *    (the paper's I).  Sigma = R(q) diag(s^2) R(q)^T.
 *  - Every call is asynchronous on `stream`, never synchronises (except the
 *    explicitly synchronous dgr_voxelize_count and dgr_status) and never
 *    allocates: device scratch comes from a dgr_ws made by dgr_ws_create.
 *  - Return value: DGR_OK, or a host-detected error (DGR_ERR_ARG,
 *    DGR_ERR_WS_TOO_SMALL, DGR_ERR_CUDA) in which case nothing was launched
 *    (DGR_ERR_CUDA: a launch failed; the stream may hold earlier launches).
 *    Errors found on the device (non-finite inputs, work-list overflow) are
 *    OR-ed into the workspace's device status word, read with dgr_status.
 *  - Thread safety: calls sharing one dgr_ws must be ordered on one stream.
 */
#ifndef DGR_H
#define DGR_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* host-detected return codes */
#define DGR_OK 0
#define DGR_ERR_ARG 1
#define DGR_ERR_WS_TOO_SMALL 2
#define DGR_ERR_CUDA 3
/* device status bits (dgr_status) */
#define DGR_STATUS_NONFINITE 0x10   /* a Gaussian had a non-finite parameter; it was skipped */
#define DGR_STATUS_PAIR_OVERFLOW 0x20 /* (tile, Gaussian) work list exceeded the plan; volume incomplete */
#define DGR_STATUS_ITEM_OVERFLOW 0x40 /* backward work items exceeded the plan; gradients incomplete */
#define DGR_STATUS_TIMEOUT 0x80      /* a bounded wait inside a kernel gave up; its output is invalid */
#define DGR_STATUS_BOUNDS 0x100      /* bounds-checked build only: an index fell outside its buffer; that access was skipped */

/* Voxel grid: nx, ny, nz <= 32767 voxels of size h, min corner (ox, oy, oz).
 * z0 (>= 0, usually 0): this grid is the z-slab of layers [z0, z0 + nz) of a
 * larger grid with the same origin (ox, oy, oz) and voxel size; voxel (i, j, k)
 * of the slab has centre (ox, oy, oz) + (i + 1/2, j + 1/2, z0 + k + 1/2) h.
 * Footprint integers are taken in the larger grid's frame, so a slab's
 * voxelized values are those of the same layers of the whole grid (bit for
 * bit when z0 is a multiple of the voxelizer's tile depth, 32).  The line
 * integral is additive over z-slabs (Sec. 4.3) and the voxel sum over
 * Gaussians (Eq. 4): the z-slab split of one reconstruction over several GPUs
 * runs voxelize, project, backproject and the voxelize adjoint on slab grids.
 * dgr_step, dgr_params_init, dgr_adam, dgr_densify and dgr_seed take whole
 * grids (z0 = 0). */
typedef struct {
    int nx, ny, nz;
    float h;
    float ox, oy, oz;
    int z0;
} dgr_grid;

#define DGR_PARALLEL 0
#define DGR_CONE 1

/* Scan geometry (paper Sec. 4.3: "general geometry projection transformation";
 * conventions fixed by this library):  views rotate about z by angles[k]
 * (radians, DEVICE array [n_views]); r = (cos a, sin a, 0), e_u = (-sin a,
 * cos a, 0), e_v = (0, 0, 1); detector pixel (iu, iv) sits at
 * u = (iu - (nu-1)/2) pu, v = (iv - (nv-1)/2) pv.
 *   parallel: the ray through u e_u + v e_v along r.
 *   cone:     source at -dso r, flat detector centred at (dsd - dso) r; the
 *             ray from the source through the pixel centre.
 * Line integrals are in (value x world length). */
typedef struct {
    int beam;          /* DGR_PARALLEL or DGR_CONE */
    int n_views, nu, nv;
    float pu, pv;      /* detector pitch, world units */
    float dso, dsd;    /* cone only: source-origin, source-detector distance */
    const float *angles; /* device [n_views] */
} dgr_geom;

/* Opaque device workspace: one cudaMalloc made by dgr_ws_create, carved by
 * every call according to the plan it was created with. */
typedef struct dgr_ws dgr_ws;

/* What a workspace must hold.  max_pairs bounds the (voxel tile, Gaussian)
 * work list of the voxelizer; max_items bounds the backward work items
 * (z-chunks of Gaussian boxes).  Use dgr_voxelize_count for exact values.
 * grid_vox/rays > 0 reserve the step's volume and sinogram buffers. */
typedef struct {
    int max_n;               /* largest Gaussian count */
    int max_tiles;           /* largest number of voxel tiles (dgr_tile_count) */
    long long max_pairs;
    long long max_items;
    long long max_vox;       /* dgr_step: voxels of the volume; dgr_project: optional room for a z-fastest copy */
    long long max_rays;      /* dgr_step only: rays of the sinogram (0 otherwise) */
    int max_views, max_nu, max_nv; /* projector tables (batches: sum of views, max nu, max nv) */
    int max_inst;            /* instances of dgr_step_batched (0 or 1: single problems) */
} dgr_ws_plan;

/* Bytes a workspace with this plan needs. */
int dgr_ws_bytes(const dgr_ws_plan *plan, size_t *bytes);
/* The only allocating calls: cudaMalloc / cudaFree of the workspace arena. */
int dgr_ws_create(dgr_ws **ws, const dgr_ws_plan *plan);
int dgr_ws_destroy(dgr_ws *ws);
/* Voxel tiles (8 x 16 x depth voxels) covering a grid, for the current tile
 * depth.  Plans and calls must use the same depth. */
int dgr_tile_count(const dgr_grid *grid, int *tiles);

/* Reads and clears the device status word (synchronises `stream`). */
int dgr_status(dgr_ws *ws, cudaStream_t stream, int *status);
const char *dgr_strerror(int code);
/* 1 (default): the voxelizer sorts each tile's Gaussian list, so results are
 * bit-reproducible run to run; 0: skip the sort (order follows atomics). */
int dgr_set_deterministic(int on);
/* Voxelizer tile depth along z: 8, 16 or 32 (default 32).  Deeper tiles share
 * each lane's per-Gaussian set-up over more voxels; shallower tiles make more
 * CTAs for small grids.  A process-wide setting, chosen by the autotuner
 * (paper_2411_04844_b300/autotune.py); workspace plans depend on it. */
int dgr_set_tile_depth(int tz);
/* 1 (default): when every Gaussian of a voxelize call has a diagonal A
 * (isotropic scales -- the paper's representation -- or an identity rotation),
 * the voxelizer uses its separable form, exp(-d^T A d / 2) = EXY(x, y) EZ(z):
 * per tile an outer-product sum, two small exponential tables per Gaussian
 * and one FMA per (Gaussian, voxel) pair (tile depth 32 only); 0: always the
 * general kernel.  A process-wide setting. */
int dgr_set_separable(int on);
/* 1: the path walks of dgr_project (with a workspace copy), of the
 * ray-scatter backprojector and of the step stage each (x, y) cell's z window
 * in shared memory with bulk asynchronous copies (projector) or add it back
 * with bulk asynchronous reductions (backprojector), two stages of up to 32
 * cells, when every volume has nz a multiple of 4 and at most 4096;
 * 0 (default): the walks read and add in global memory directly.  Same
 * results either way.  At 256^3 / 50 x 256^2 the staged walks take 1.48 ms
 * (project) and 1.99 ms (backproject) against 1.04 and 1.34 ms direct: the
 * volume already sits in L2 and the lanes' loads are 4-5 sectors, so the
 * stage synchronisation and the lower occupancy cost more than they save.
 * A process-wide setting. */
int dgr_set_staged_walk(int on);
/* Backprojector implementation (all exact transposes of dgr_project, all
 * bit-reproducible): 0 (default) = ray scatter -- a CTA per detector column
 * walks the column's path like the projector and adds into integer sums in
 * the workspace (needs a plan whose max_vox covers the volumes, else the
 * brick scatter runs); 1 = column gather -- a warp per voxel column finds the
 * candidate rays of each voxel in closed form; 2 = brick scatter -- a CTA
 * accumulates a voxel brick in shared memory, its warps walking the detector
 * columns that cross it, each lane carrying several detector rows.  The two
 * scatters add the same fixed-point integers (exact, order-independent; the
 * step is chosen per group of 128 views from the largest residual so that no
 * sum can overflow) and fold them into FP32 sums in a fixed order: they
 * return the same bits.  A process-wide setting. */
int dgr_set_backprojector(int variant);

/* Footprint integers (paper Sec. 4.1 "Gaussian Effect Confinement",
 * "Discretize and Align" Eq. 6; valid mask of Algorithm 1):
 * anchor a = floor(u), u = (mu - o)/h - 1/2 (voxel centres at integers);
 *   k_trunc > 0: per axis R = ceil(k_trunc * sigma_a), sigma_a = sqrt(Sigma_aa)/h,
 *                box [a - R, a + R + 1];
 *   k_trunc < 0: the paper's fixed odd box K = -k_trunc, [a - (K-1)/2, a + (K-1)/2];
 * clipped to the grid (axis empty when lo > hi).  Computed with a fixed FP32
 * operation sequence (every operation rounded on its own).
 * anchor [n][3], box [n][6] = (lo x, y, z, hi x, y, z), device int32. */
int dgr_footprint(const dgr_grid *grid, int n, const float *mu, const float *s, const float *q,
                  float k_trunc, int *anchor, int *box, cudaStream_t stream);

/* Exact work-list sizes for these Gaussians (synchronises `stream`). */
int dgr_voxelize_count(const dgr_grid *grid, int n, const float *mu, const float *s,
                       const float *q, float k_trunc, long long *pairs, long long *items,
                       dgr_ws *ws, cudaStream_t stream);

/* FVR forward (paper Eq. 4 with confinement, Eq. 6-7 alignment, Algorithm 1):
 * vol[v] = sum_g rho_g exp(-1/2 (v - u_g)^T A_g (v - u_g)) over the voxels of
 * each Gaussian's box, A_g = h^2 Sigma_g^-1.  Overwrites vol [nz][ny][nx]. */
int dgr_voxelize(const dgr_grid *grid, int n, const float *mu, const float *s, const float *q,
                 const float *rho, float k_trunc, float *vol, dgr_ws *ws, cudaStream_t stream);

/* Adjoint of dgr_voxelize: given grad_vol = dL/dV, writes dL/dmu [n][3],
 * dL/ds [n][3], dL/dq [n][4], dL/drho [n] (overwrites).  Box and anchor are
 * held fixed (piecewise-constant), the gradient to mu flowing through
 * u - a (paper Sec. 4.1, end of "Discretize and Align"). */
int dgr_voxelize_backward(const dgr_grid *grid, int n, const float *mu, const float *s,
                          const float *q, const float *rho, float k_trunc, const float *grad_vol,
                          float *g_mu, float *g_s, float *g_q, float *g_rho, dgr_ws *ws,
                          cudaStream_t stream);

/* Projector T (paper Sec. 4.3, Eq. 12, P_hat = T(V)): each detector pixel is
 * the exact line integral of the piecewise-constant voxel image along its ray
 * (Siddon's radiological path).  Overwrites sino [n_views][nv][nu].
 * If the workspace plan's max_vox covers the grid, the volume is first copied
 * into the workspace with z fastest and projected by the row-warp kernel (a
 * warp per 32 detector rows of one detector column); otherwise a per-ray
 * kernel reads it in place.  Both use the same chord lengths; their sums may
 * differ in rounding order. */
int dgr_project(const dgr_grid *grid, const dgr_geom *geom, const float *vol, float *sino,
                dgr_ws *ws, cudaStream_t stream);

/* Exact transpose of dgr_project: vol[v] = sum_rays L(ray, v) sino[ray], with
 * L the same chord lengths.  Gathers per voxel (no atomics).  Overwrites vol. */
int dgr_backproject(const dgr_grid *grid, const dgr_geom *geom, const float *sino, float *vol,
                    dgr_ws *ws, cudaStream_t stream);

/* L1 data term of the paper's objective (Sec. 4.3, Eq. 13, first term):
 * loss = weight x mean |pred - meas| (device scalar, fixed-order reduction)
 * and resid = weight x sign(pred - meas) / m (sign(0) = 0).  resid may alias
 * pred.  weight 1 is the term itself; a part of a sinogram (views split over
 * GPUs) takes weight = m / (all rays), so the parts' losses and residuals add
 * up to those of the whole. */
int dgr_l1_residual(const float *pred, const float *meas, long long m, float weight, float *resid,
                    float *loss, dgr_ws *ws, cudaStream_t stream);

/* SSIM term of the objective (paper Sec. 4.3, App. D.1) on its own:
 * loss_out (device scalar) = 1 - SSIM(pred, meas), the mean of the SSIM map
 * over every pixel of every view (statistics as in dgr_problem), and
 * grad = d loss / d pred.  pred, meas, grad: device [n_views][nv][nu] of geom.
 * The workspace plan must hold max_rays >= the projection size. */
int dgr_ssim_loss(const dgr_geom *geom, const float *pred, const float *meas, float data_range,
                  float *grad, float *loss_out, dgr_ws *ws, cudaStream_t stream);
/* TV term on its own: loss_out = sum over axes of |forward differences| of
 * vol divided by the voxel count; grad = d loss / d vol.  vol, grad: device
 * [nz][ny][nx].  The workspace plan must hold max_vox >= the voxel count. */
int dgr_tv_loss(const dgr_grid *grid, const float *vol, float *grad, float *loss_out, dgr_ws *ws,
                cudaStream_t stream);

/* One optimisation iteration (paper Sec. 4.3 "Global Optimization"; Adam with
 * lr decaying lr0 -> lr1, Sec. 5.1 "Implementation Details"). */
typedef struct {
    dgr_grid grid;
    dgr_geom geom;
    float k_trunc;
    float lr0, lr1;    /* lr(t) = lr0 (lr1/lr0)^((t-1)/(n_iters-1)), t = 1..n_iters */
    int n_iters;
    float beta1, beta2, eps;
    /* objective (paper Sec. 4.3, App. D.1; 0.6 / 0.2 / 1 there):
     *   loss = w_l1 mean|P_hat - P| + w_ssim (1 - SSIM(P_hat, P)) + w_tv TV(V),
     * SSIM over every projection image (11 x 11 Gaussian window, sigma 1.5,
     * zero outside the image, C1 = (0.01 L)^2, C2 = (0.03 L)^2 with
     * L = ssim_range, 1 if 0), TV = sum over axes of |forward differences| /
     * voxels.  All three weights 0: the L1 term alone with weight 1. */
    float w_l1, w_ssim, w_tv, ssim_range;
} dgr_problem;

/* Optimiser state.  theta/m/v are [11 n] laid out [mu 3n | s 3n | q 4n | rho n]
 * with theta = ((mu - c)/half, log s, q, softplus^-1(rho)), c and half the
 * grid centre and half-extent.  mu/s/q/rho are rewritten from theta by every
 * step; step is a device int counting completed steps. */
typedef struct {
    int n;
    float *mu, *s, *q, *rho;
    float *theta, *m, *v;
    int *step;
    float *grad_accum;  /* optional device [n] (NULL: none): every step adds |dL/dmu| (world
                         * units) of each Gaussian -- the statistic of dgr_densify */
} dgr_params;

/* theta from (mu, s, q, rho); m = v = 0; step = 0. */
int dgr_params_init(const dgr_problem *prob, const dgr_params *p, cudaStream_t stream);

/* The last phase of dgr_step on its own (Sec. 5.1): with the gradients of
 * the loss with respect to (mu, s, q, rho) given (device [n][3], [n][3],
 * [n][4], [n]), one Adam step on theta (chain factors half-extent, s and
 * sigmoid(theta_rho); learning rate of step *p->step + 1 on the problem's
 * schedule), mu/s/q/rho rewritten from theta, step incremented.  For a loss
 * whose gradients were assembled elsewhere (e.g. summed over the z-slabs of
 * several GPUs): on identical inputs every replica takes the identical step. */
int dgr_adam(const dgr_problem *prob, const dgr_params *p, const float *g_mu, const float *g_s,
             const float *g_q, const float *g_rho, cudaStream_t stream);

/* voxelize -> project -> loss and residual -> backproject (+ TV gradient) -> voxelize adjoint ->
 * chain rule to theta -> Adam.  measured: device [n_views][nv][nu];
 * loss_out: device scalar (the L1 loss before the update).  The workspace
 * plan must carry max_vox and max_rays of this problem. */
int dgr_step(const dgr_problem *prob, const dgr_params *p, const float *measured,
             float *loss_out, dgr_ws *ws, cudaStream_t stream);

/* Adaptive density control (paper App. F, Algorithm 2).  With avg = grad_accum
 * / iters and sigma = the largest axis scale of a Gaussian:
 *   clone  avg >= tau, sigma <= theta_frac x body diagonal of the grid: the
 *          n_clone of largest avg (ties: lower index), n_clone <= n_max - n;
 *          the original and its copy each get half the intensity;
 *   split  avg >= tau, sigma > theta: the n_split of largest avg, n_split <=
 *          n_max - n - n_clone; each is replaced by two children
 *          mu + R(q) diag(s) z (z: normals[i][c], standard normal 3-vectors
 *          supplied by the caller, device [n][2][3]), scales s / 2^(1/3), the
 *          same rotation and intensity;
 *   prune  the other originals with avg <= tau or sigma > 3 size h.
 * out receives surviving originals (index order; theta, m, v kept), clones
 * and children (theta from their parameters, zero moments, zero grad_accum);
 * its arrays must hold n_max Gaussians and must not alias in's; *out->step =
 * *in->step.  in->grad_accum is required.  *n_out (host) receives the new
 * count: the call synchronises the stream.  The decisions are taken on the
 * FP32 values.  The plan needs max_n >= in->n. */
typedef struct {
    float tau;         /* minimum mean gradient (2e-4 in the paper) */
    float theta_frac;  /* small/large threshold as a fraction of the body diagonal (0.005) */
    float size;        /* box size in voxels (17): wider than 3 size h is pruned */
    int n_max;         /* cap on the number of Gaussians (500,000) */
} dgr_densify_cfg;
int dgr_densify(const dgr_grid *grid, const dgr_densify_cfg *cfg, int iters, const dgr_params *in,
                const float *normals, dgr_params *out, int *n_out, dgr_ws *ws, cudaStream_t stream);

/* Many independent reconstructions in one call (the paper runs one problem
 * at a time): n_inst <= 16 problems, each with its own
 * grid, geometry, Gaussian count and optimiser state, advance by one dgr_step
 * each, every phase being ONE launch over the work of all instances (the
 * voxelizer's CTAs are persistent and pull tiles of every instance from one
 * queue; the projector and backprojector walks take one launch per detector
 * height class present -- at most 64 rows, at most 128, taller -- whose CTAs
 * cover that many rows).  probs, params, measured: host arrays [n_inst] (measured[i] a device
 * pointer); loss_out: device [n_inst].  The workspace plan must hold the sums
 * over instances: max_n, max_tiles, max_pairs, max_items, max_vox, max_rays,
 * max_views (sum of views), max_nu / max_nv (maxima) and max_inst >= n_inst.
 * Captured once in a CUDA graph, one replay advances every instance. */
int dgr_step_batched(int n_inst, const dgr_problem *probs, const dgr_params *params,
                     const float *const *measured, float *loss_out, dgr_ws *ws,
                     cudaStream_t stream);

/* dgr_step with CUDA events recorded on `stream` at its phase boundaries:
 * events[0] before voxelize, [1] after voxelize, [2] after project, [3] after
 * the L1 residual, [4] after backproject, [5] after the voxelize adjoint,
 * [6] after Adam.  With n_events >= DGR_STEP_KERNEL_EVENTS (15), also
 * [7] / [8] right before / after the backprojector's main kernel (the path
 * scatter, without the residual scaling and the fold), [9] / [10] around
 * the projector's main kernel, [11] / [12] around the voxelizer's main kernel
 * (the tile evaluation, without prep and binning) and [13] / [14] around the
 * voxelize adjoint's main kernel (the per-item moments).  events: host array
 * of n_events (>= 7) cudaEvent_t. */
#define DGR_STEP_EVENTS 7
#define DGR_STEP_KERNEL_EVENTS 15
int dgr_step_timed(const dgr_problem *prob, const dgr_params *p, const float *measured,
                   float *loss_out, dgr_ws *ws, cudaStream_t stream, cudaEvent_t *events,
                   int n_events);

/* Projector for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a library-level variant of dgr_project.
 *
 * Some callers may not call cudaMalloc at all: code hosted inside an
 * application that hands out all device memory from its own pool and forbids
 * driver allocations in plug-ins; loops with a latency budget in which an
 * allocation (which may synchronise the device) is not allowed; code that runs
 * after a one-time initialisation phase during which all memory was reserved.
 * For them this entry point computes what dgr_project computes (with the
 * per-ray kernel: the same chord lengths) without any dgr_ws: its scratch (the ray tables,
 * 32 bytes per (view, detector column) + 16 bytes per detector row + 8 bytes
 * per view, rounded) lives in one fixed device array of
 * DGR_NOALLOC_SCRATCH_BYTES that every GPU using the library holds until the
 * process exits.  The caller still passes vol and sino (device pointers).
 *  - Geometries whose ray tables exceed the array (e.g. more than ~130,000
 *    views x detector columns) return DGR_ERR_WS_TOO_SMALL; nothing runs.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current) and caches it per
 *    device ordinal.  The cached address is invalid after cudaDeviceReset and
 *    under a context other than the device's primary context: do not call
 *    this entry point after either.
 *  - Geometries are validated exactly as by dgr_project; the table size is
 *    checked in 64-bit arithmetic (views x columns) before anything runs.
 *  - It calls no cudaMalloc, cudaFree or other allocating routine.
 *  - All calls on a device share the one array (it keeps the last call's
 *    tables, every call rewrites them in full): calls that overlap on the GPU
 *    (e.g. on two streams at once) race and give wrong results.  Order them.
 * Arguments, layouts and errors otherwise as dgr_project. */
#define DGR_NOALLOC_SCRATCH_BYTES (4 << 20)
int dgr_project_noalloc(const dgr_grid *grid, const dgr_geom *geom, const float *vol,
                        float *sino, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Learned warm start (not in the paper: a network proposing the initial
 * Gaussians from a coarse backprojection; the plain initialisation remains
 * the fallback).  A 3D convolutional encoder-decoder on an n^3 grid (n a
 * multiple of 4, <= 256), channels 16-32-64-32-16, 3^3 kernels, 2^3 average
 * pooling and nearest upsampling, additive skips, a 1^3 head to 2 outputs
 * (density, log-scale in voxels).  Activations and weights BF16 (channels-last
 * [z][y][x][c]), every convolution accumulating in FP32; the four inner
 * convolutions are implicit GEMMs on the tcgen05 tensor cores (forward, data
 * and weight gradient; FP32 accumulators in tensor memory; halo tiles whose
 * taps are shared-memory descriptors into one input block).
 * params: FP32 [dgr_net_param_count()], per layer [tap][c_in][c_out] weights
 * then [c_out] biases.  input: FP32 [n^3]; output: FP32 [n^3][2].
 * ws: caller-owned device scratch of dgr_net_ws_bytes(n) bytes holding the
 * activations, so dgr_net_backward must follow the dgr_net_forward it
 * differentiates on the same ws. */
long long dgr_net_param_count(void);
int dgr_net_ws_bytes(int n, size_t *bytes);
int dgr_net_forward(int n, const float *params, const float *input, float *output, void *ws,
                    size_t ws_bytes, cudaStream_t stream);
/* grad_params (FP32, overwritten) = d loss / d params for d loss / d output. */
int dgr_net_backward(int n, const float *params, const float *input, const float *grad_output,
                     float *grad_params, void *ws, size_t ws_bytes, cudaStream_t stream);
/* loss = mean over voxels of w_density (y0 - t0)^2 + w_scale (y1 - t1)^2
 * (device scalar) and grad_output = d loss / d output. */
int dgr_net_loss(int n, const float *output, const float *target, float w_density, float w_scale,
                 float *grad_output, float *loss, void *ws, size_t ws_bytes, cudaStream_t stream);
/* Convolution engine: 2 = tcgen05 (default): forward and data gradient with
 * the three z taps of one (dy, dx) in one MMA (N = 3 x output channels) over
 * TMA-loaded halo blocks (an 8 x 16 x ZT output tile's input block with a
 * one-voxel halo, every tap a descriptor into it), weight gradient with the
 * input channels x z offsets on M and the y offsets x output channels on N;
 * 3 = tcgen05 on halo tiles with one MMA per tap (N = output channels) and
 * the weight gradient with the output channels on M; 1 = tcgen05 on gathered
 * 128-row tiles (im2col into shared memory) for forward and data gradient,
 * mma.sync for the weight gradient; 0 = mma.sync m16n8k16 for all.
 * Process-wide; DGR_ERR_ARG otherwise. */
int dgr_set_conv_engine(int engine);
/* The network's device status word on ws (DGR_STATUS_TIMEOUT when a bounded
 * wait of a tcgen05 convolution gave up; the output is then incomplete).
 * Cleared by dgr_net_forward; synchronous read. */
int dgr_net_status(int n, const void *ws, size_t ws_bytes, int *status);
/* Textbook Adam on a flat FP32 array (step t >= 1, host int). */
int dgr_adam_flat(long long n, float *params, const float *grads, float *m, float *v, int t,
                  float lr, float beta1, float beta2, float eps, cudaStream_t stream);
/* FDK-style filtering of projections for the network input: each detector
 * row is cosine-weighted (cone: dsd / sqrt(dsd^2 + u^2 + v^2)), convolved
 * with the Ram-Lak ramp kernel and multiplied by scale (the FBP constant,
 * pi / n_views x pu pv / (M h^3) with M = dsd / dso, so that dgr_backproject
 * of the result is the FDK volume); out has the sinogram layout. */
int dgr_fdk_filter(const dgr_geom *geom, float scale, const float *sino, float *out,
                   cudaStream_t stream);
/* Seeding proposals from a source volume of n_vox voxels with `channels`
 * values each: density = max(src[channels * i], 0); log_scale = src[2 i + 1]
 * (channels 2: the network's output) or log_scale_default (channels 1: an FDK
 * volume, the plain fallback). */
int dgr_proposals(long long n_vox, const float *src, int channels, float log_scale_default,
                  float *density, float *log_scale, cudaStream_t stream);
/* Training targets from a fit of the plain method: w[i] = rho[i] x mean over
 * axes of log(s / h) (voxelize it for the weighted log-scale sum), then
 * out[i] = (density[i], clamp(wsum[i] / density[i], log_lo, log_hi)) where
 * density > min_density, (density[i], log_default) elsewhere; out [n_vox][2]. */
int dgr_logscale_weight(int n, const float *s, const float *rho, float h, float *w,
                        cudaStream_t stream);
int dgr_fit_targets(long long n_vox, const float *density, const float *wsum, float min_density,
                    float log_lo, float log_hi, float log_default, float *out, cudaStream_t stream);
/* Seeding from proposals on a cubic grid: ns voxels drawn with probability
 * proportional to max(density, 0) (u: uniform [0,1) per seed, given), mu = the
 * voxel centre + jitter * h (jitter in [-1/2, 1/2)^3, given), isotropic s =
 * clamp(exp(log_scale), 0.3, 8) h, q = identity, rho = density; voxel[i] = the
 * drawn voxel.  scratch: dgr_seed_bytes(n) bytes of device memory. */
int dgr_seed_bytes(int n_side, size_t *bytes);
int dgr_seed(const dgr_grid *grid, const float *density, const float *log_scale, int ns,
             const float *u, const float *jitter, float *mu, float *s, float *q, float *rho,
             int *voxel, void *scratch, size_t scratch_bytes, cudaStream_t stream);
/* rho[i] *= clamp(density / vol, 1/4, 4) at each seed's voxel (a fixed-point
 * step matching the seeds' voxelized field vol to the proposed density). */
int dgr_seed_rescale(int ns, const int *voxel, const float *density, const float *vol, float *rho,
                     cudaStream_t stream);

/* Failure-detection check (the paper has no counterpart).  Every kernel of
 * this library that waits for asynchronous copies or tensor-core MMAs waits
 * on an mbarrier for a bounded number of polls; if the wait runs out it ORs
 * DGR_STATUS_TIMEOUT into the status word and returns, so the host detects the
 * failure and the context stays usable.  This launches one CTA whose bounded
 * wait (at most `polls` polls, 1 <= polls <= 2^18, the kernels' own limit;
 * an unsuccessful poll takes about 3 us on the B300)
 * runs out on purpose: it waits on an mbarrier that nothing arrives at, with
 * nothing in flight.  status: device int, OR-ed with DGR_STATUS_TIMEOUT;
 * gave_up: device int, set to 1 (0 if the wait had completed). */
int dgr_test_bounded_wait(int polls, int *status, int *gave_up, cudaStream_t stream);

/* Total number of kernels this library has launched in this process (a host
 * counter; lets callers count launches inside a timed region). */
long long dgr_launch_count(void);

/* Measurement utility (the paper has no counterpart): the rate of one
 * arithmetic pipe per SM clock on the running GPU, the peak the voxelizer
 * (exp2 per in-box pair, Eq. 4) and its adjoint (FP32 FMA) are judged by.
 * kind: DGR_PIPE_EX2 (ex2.approx.ftz.f32), DGR_PIPE_FFMA (FP32 fma) or
 * DGR_PIPE_FFMA2 (packed f32x2 fma; counted as two FMAs).  Launches n_blocks
 * CTAs of 256 threads, each thread iters x 32 operations in 8 independent
 * chains.  rec: device [4 n_blocks] uint64, per CTA: SM id, clock64 at start,
 * clock64 at end, operations; sink: device [256 n_blocks] floats (keeps the
 * results live).  Per SM, rate = its CTAs' operations / (latest end -
 * earliest start).  DGR_ERR_ARG for a bad kind or size (1 <= iters <= 2^20,
 * 1 <= n_blocks <= 2^16) or a null pointer; asynchronous on stream. */
#define DGR_PIPE_EX2 0
#define DGR_PIPE_FFMA 1
#define DGR_PIPE_FFMA2 2
int dgr_pipe_rate(int kind, int iters, int n_blocks, unsigned long long *rec, float *sink,
                  cudaStream_t stream);
/* Measurement utility (no paper counterpart): L2 bandwidth over a device
 * buffer of `bytes` (a multiple of 16, of 512 for kind 1; 16-byte aligned) small enough to stay
 * in L2, `passes` passes by n_blocks CTAs of 256 threads.  kind 0: streaming
 * 16-byte reads (sink: device [256 n_blocks] floats keeps them live); kind 1:
 * 32-bit integer reductions (+1 to every word, the backprojector's scatter
 * operation; buf is modified).  The caller times it (bytes x passes / time).
 * DGR_ERR_ARG for a bad kind, size or pointer; asynchronous on stream. */
int dgr_l2_rate(int kind, long long bytes, int passes, int n_blocks, void *buf, float *sink,
                cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* DGR_H */
