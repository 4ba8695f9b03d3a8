// C ABI of libdgr: argument validation, workspace layout, orchestration of the
// kernels on the caller's stream.  See include/dgr.h for the contract.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <new>

#include "dgr_internal.cuh"

using namespace dgr;

std::atomic<long long> dgr::g_launches{0};

int dgr::wave_ctas(const void *kernel, int threads, size_t smem) {
    struct Entry {
        const void *k;
        int dev, threads, ctas;
        size_t smem;
    };
    static std::mutex mu;
    static Entry cache[64];
    static int used = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < used; ++i)
        if (cache[i].k == kernel && cache[i].dev == dev && cache[i].threads == threads && cache[i].smem == smem)
            return cache[i].ctas;
    int sms = 148, per_sm = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int ctas = sms * per_sm;
    if (used < 64) cache[used++] = Entry{kernel, dev, threads, ctas, smem};
    return ctas;
}

// Host-side validators shared by every entry point (also the no-allocation
// projector).
bool dgr::grid_ok(const dgr_grid *g) {
    return g && g->nx > 0 && g->ny > 0 && g->nz > 0 && g->nx <= MAX_DIM && g->ny <= MAX_DIM &&
           g->nz <= MAX_DIM && isfinite(g->h) && g->h > 0.f && isfinite(g->ox) &&
           isfinite(g->oy) && isfinite(g->oz) && g->z0 >= 0 && g->z0 <= (1 << 24) &&
           isfinite(slab_origin(*g));
}

bool dgr::geom_ok(const dgr_geom *geo) {
    if (!geo || !geo->angles) return false;
    if (geo->beam != DGR_PARALLEL && geo->beam != DGR_CONE) return false;
    if (geo->n_views <= 0 || geo->nu <= 0 || geo->nv <= 0 || geo->n_views > MAX_VIEWS_BP) return false;
    if (!(isfinite(geo->pu) && geo->pu > 0.f && isfinite(geo->pv) && geo->pv > 0.f)) return false;
    if (geo->beam == DGR_CONE &&
        !(isfinite(geo->dso) && isfinite(geo->dsd) && geo->dso > 0.f && geo->dsd > geo->dso))
        return false;
    return true;
}

bool dgr::geom_fits_grid(const dgr_grid *g, const dgr_geom *geo) {
    // cone: the whole grid must lie in front of the source (every corner
    // strictly inside the source circle), so central projection is convex
    if (geo->beam != DGR_CONE) return true;
    double r2 = 0;
    const double o[2] = {g->ox, g->oy}, e[2] = {g->nx * (double)g->h, g->ny * (double)g->h};
    for (int a = 0; a < 2; ++a) {
        const double m = fmax(fabs(o[a]), fabs(o[a] + e[a]));
        r2 += m * m;
    }
    return sqrt(r2) < 0.999 * geo->dso;
}

namespace {

int g_deterministic = 1;

bool k_ok(float k) {
    if (!isfinite(k) || k == 0.f) return false;
    if (k > 0.f) return true;
    const float K = -k;
    return K == floorf(K) && ((int)K % 2 == 1) && K < 65536.f;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? DGR_OK : DGR_ERR_CUDA; }

struct Layout {
    size_t status, prep, itemcnt, item_off, tile_cnt, tile_off, tile_fill, scan_tmp, list,
        partials, grads, vol, sino, loss_part, rayxy, sino_scaled, list_tmp, gvol, ssim_maps, ssim_g,
        ssim_part, tv_part, dens, vsplit, vpart, acc, total;
    size_t scan_elems;
};

bool plan_ok(const dgr_ws_plan *p) {
    return p && p->max_n >= 0 && p->max_tiles >= 0 && p->max_pairs >= 0 && p->max_items >= 0 &&
           p->max_vox >= 0 && p->max_rays >= 0 && p->max_views >= 0 && p->max_nu >= 0 &&
           p->max_nv >= 0 && p->max_pairs < (1ll << 32) && p->max_items < (1ll << 32) &&
           p->max_n < (1 << 24) && p->max_tiles < (1 << 24) && p->max_inst >= 0 &&
           p->max_inst <= MAX_INST;
}

Layout layout_of(const dgr_ws_plan &p) {
    Layout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    const int scan_len = p.max_n > p.max_tiles ? p.max_n : p.max_tiles;
    L.scan_elems = scan_tmp_elems(scan_len);
    L.status = take(256);
    L.prep = take(sizeof(Prep) * (size_t)p.max_n);
    L.itemcnt = take(4 * ((size_t)p.max_n + 1));
    L.item_off = take(4 * ((size_t)p.max_n + 1));
    L.tile_cnt = take(4 * ((size_t)p.max_tiles + 1));
    L.tile_off = take(4 * ((size_t)p.max_tiles + 1));
    L.tile_fill = take(4 * ((size_t)p.max_tiles + 1));
    L.scan_tmp = take(8 * L.scan_elems);
    L.list = take(4 * (size_t)p.max_pairs);
    L.list_tmp = take(4 * (size_t)p.max_pairs);  // merge scratch of long tile lists
    L.partials = take(4 * (size_t)NMOM * (size_t)p.max_items);
    const int ninst = p.max_inst > 0 ? p.max_inst : 1;
    L.rayxy = take(ray_table_bytes((long long)p.max_views * p.max_nu, p.max_views,
                                   (long long)ninst * p.max_nv));
    // residual x |D| for the backprojector (standalone calls; the step reuses its sinogram)
    // scaled residual of the backprojector, then (64-float aligned) one maximum per view
    L.sino_scaled = take(4 * ((size_t)p.max_views * p.max_nu * p.max_nv + 64 + (size_t)p.max_views));
    L.loss_part = take(4 * (size_t)(L1_BLOCKS * ninst + 1));
    L.grads = take(4 * 11 * (size_t)p.max_n);
    // instance volumes start on 64-float boundaries (vectorised stores)
    L.vol = take(4 * ((size_t)p.max_vox + (size_t)64 * (p.max_inst > 1 ? p.max_inst : 1)));
    L.sino = take(4 * (size_t)p.max_rays);
    // step: the volume gradient (x fastest; the volume itself stays z fastest
    // for the TV term), SSIM maps A, B, C and gradient, SSIM and TV partial sums
    const size_t vpad = (size_t)64 * (p.max_inst > 1 ? p.max_inst : 1);
    const bool step = p.max_rays > 0 && p.max_vox > 0;
    L.gvol = take(step ? 4 * ((size_t)p.max_vox + vpad) : 0);
    L.ssim_maps = take(4 * 3 * (size_t)p.max_rays);
    L.ssim_g = take(4 * (size_t)p.max_rays);
    L.ssim_part = take(4 * ssim_tiles_cap(p.max_views, p.max_nu, p.max_nv, ninst));
    L.tv_part = take(4 * tv_tiles_cap(p.max_vox, ninst));
    // densification: keys, flags, three offset scans of max_n + 1, counts
    L.dens = take(4 * (5 * ((size_t)p.max_n + 1) + 8));
    // the voxelizer's split plan and partial slots (rewritten by every call)
    L.vsplit = take(p.max_tiles > 0 ? 4 * split_plan_ints(p.max_tiles, ninst) : 0);
    L.vpart = take(p.max_tiles > 0 ? 4 * (size_t)ninst * SPLIT_BUDGET * VOX_SLOT : 0);
    // integer sums of the ray-driven backprojector (z fastest), kept zero between calls
    L.acc = take(p.max_vox > 0 ? 4 * ((size_t)p.max_vox + vpad) : 0);
    L.total = o;
    return L;
}

}  // namespace

extern "C" {

int dgr_ws_bytes(const dgr_ws_plan *plan, size_t *bytes) {
    if (!plan_ok(plan) || !bytes) return DGR_ERR_ARG;
    *bytes = layout_of(*plan).total;
    return DGR_OK;
}

int dgr_ws_create(dgr_ws **ws, const dgr_ws_plan *plan) {
    if (!ws || !plan_ok(plan)) return DGR_ERR_ARG;
    *ws = nullptr;
    const Layout L = layout_of(*plan);
    dgr_ws *w = new (std::nothrow) dgr_ws;
    if (!w) return DGR_ERR_ARG;
    memset(w, 0, sizeof(*w));
    w->plan = *plan;
    w->bytes = L.total;
    if (cudaMalloc(&w->base, L.total) != cudaSuccess) {
        delete w;
        return DGR_ERR_CUDA;
    }
    w->status = L.status; w->prep = L.prep; w->itemcnt = L.itemcnt; w->item_off = L.item_off;
    w->tile_cnt = L.tile_cnt; w->tile_off = L.tile_off; w->tile_fill = L.tile_fill;
    w->scan_tmp = L.scan_tmp; w->list = L.list; w->partials = L.partials; w->grads = L.grads;
    w->vol = L.vol; w->sino = L.sino; w->loss_part = L.loss_part; w->rayxy = L.rayxy;
    w->sino_scaled = L.sino_scaled;
    w->list_tmp = L.list_tmp;
    w->acc = L.acc;
    w->gvol = L.gvol; w->ssim_maps = L.ssim_maps; w->ssim_g = L.ssim_g; w->ssim_part = L.ssim_part;
    w->tv_part = L.tv_part; w->dens = L.dens;
    w->vsplit = L.vsplit; w->vpart = L.vpart;
    w->scan_tmp_elems = L.scan_elems;
    if (cudaMemset(w->base + L.status, 0, 256) != cudaSuccess ||
        cudaMemset(w->base + L.acc, 0, L.total - L.acc) != cudaSuccess) {
        cudaFree(w->base);
        delete w;
        return DGR_ERR_CUDA;
    }
    *ws = w;
    return DGR_OK;
}

int dgr_ws_destroy(dgr_ws *ws) {
    if (!ws) return DGR_ERR_ARG;
    const cudaError_t e = cudaFree(ws->base);
    delete ws;
    return cuda_rc(e);
}

int dgr_tile_count(const dgr_grid *grid, int *tiles) {
    if (!grid_ok(grid) || !tiles) return DGR_ERR_ARG;
    int a, b, c;
    *tiles = tile_dims(*grid, a, b, c);
    return DGR_OK;
}

int dgr_status(dgr_ws *ws, cudaStream_t stream, int *status) {
    if (!ws || !status) return DGR_ERR_ARG;
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, ws->base + ws->status, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws->base + ws->status, 0, sizeof(int), stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    *status = v;
    return cuda_rc(e);
}

const char *dgr_strerror(int code) {
    switch (code) {
        case DGR_OK: return "ok";
        case DGR_ERR_ARG: return "invalid argument";
        case DGR_ERR_WS_TOO_SMALL: return "workspace plan too small for this call";
        case DGR_ERR_CUDA: return "CUDA error";
        case DGR_STATUS_NONFINITE: return "non-finite or invalid Gaussian parameter (skipped)";
        case DGR_STATUS_PAIR_OVERFLOW: return "voxelizer work list overflow (volume incomplete)";
        case DGR_STATUS_ITEM_OVERFLOW: return "backward work items overflow (gradients incomplete)";
        default: return "unknown dgr code";
    }
}

int dgr_set_deterministic(int on) {
    g_deterministic = on ? 1 : 0;
    return DGR_OK;
}

int dgr_set_backprojector(int variant) {
    if (variant < 0 || variant > 2) return DGR_ERR_ARG;
    set_backprojector_variant(variant);
    return DGR_OK;
}

int dgr_set_staged_walk(int on) {
    set_staged_walk(on);
    return DGR_OK;
}

int dgr_set_separable(int on) {
    set_separable(on);
    return DGR_OK;
}

int dgr_set_tile_depth(int tz) {
    if (tz != 8 && tz != 16 && tz != 32) return DGR_ERR_ARG;
    set_tile_depth(tz);
    return DGR_OK;
}

int dgr_footprint(const dgr_grid *grid, int n, const float *mu, const float *s, const float *q,
                  float k_trunc, int *anchor, int *box, cudaStream_t stream) {
    if (!grid_ok(grid) || n < 0 || !k_ok(k_trunc)) return DGR_ERR_ARG;
    if (n > 0 && (!mu || !s || !q || !anchor || !box || !aligned16(q))) return DGR_ERR_ARG;
    return cuda_rc(launch_footprint(*grid, n, mu, s, q, k_trunc, anchor, box, stream));
}

static int gauss_args_ok(const dgr_grid *grid, int n, const float *mu, const float *s,
                         const float *q, const float *rho, float k) {
    if (!grid_ok(grid) || n < 0 || !k_ok(k)) return 0;
    if ((long long)grid->nx * grid->ny * grid->nz >= (1ll << 31)) return 0;
    if (n > 0 && (!mu || !s || !q || !rho || !aligned16(q))) return 0;
    return 1;
}

// ---------------------------------------------------------------------------
// batch descriptors
// ---------------------------------------------------------------------------
namespace {

void set_grid(Inst &I, const dgr_grid &g, float k) {
    I.g = g;
    // a z-slab is an ordinary grid at its own origin for every kernel but the
    // prep (footprint integers in the whole grid's frame)
    I.g.oz = slab_origin(g);
    I.g.z0 = 0;
    I.z0 = g.z0;
    I.oz_full = g.oz;
    I.k = k;
    I.zoff = -I.g.oz / g.h;
    tile_dims(g, I.ntx, I.nty, I.ntz);
    I.vsx = 1;  // the C ABI's volume layout: [nz][ny][nx]
    I.vsy = g.nx;
    I.vsz = g.nx * g.ny;
}

void set_geom(Inst &I, const dgr_geom &geo) {
    I.beam = geo.beam;
    I.n_views = geo.n_views;
    I.nu = geo.nu;
    I.nv = geo.nv;
    I.pu = geo.pu;
    I.pv = geo.pv;
    I.dso = geo.dso;
    I.dsd = geo.dsd;
    I.angles = geo.angles;
    bp_blocks(I.g, I.nbx, I.nbz);
    bp_bricks(I.g, I.nbbx, I.nbby, I.nbbz);
    bp_colours(I.g, geo, I.col_u, I.col_v);
    I.multiz = multi_z(geo);
}

// offsets of each instance in the global index spaces
void finish(Batch &B, bool has_geom) {
    int g = 0, tiles = 0, tab = 0, views = 0, rows = 0, blk = 0, bricks = 0;
    long long rays = 0;
    for (int i = 0; i < B.n; ++i) {
        Inst &I = B.in[i];
        I.g0 = g;
        g += I.n;
        I.tile0 = tiles;
        tiles += I.ntx * I.nty * I.ntz;
        if (has_geom) {
            I.tab0 = tab;
            tab += I.n_views * I.nu;
            I.view0 = views;
            views += I.n_views;
            I.row0 = rows;
            rows += I.nv;
            I.ray0 = rays;
            rays += (long long)I.n_views * I.nu * I.nv;
            I.blk0 = blk;
            blk += I.nbx * I.g.ny * I.nbz;
            I.bb0 = bricks;
            bricks += I.nbbx * I.nbby * I.nbbz;
        }
    }
    B.tot_g = g;
    B.tot_tiles = tiles;
    B.tot_tab = tab;
    B.tot_views = views;
    B.tot_rows = rows;
    B.tot_rays = rays;
    B.tot_blk = blk;
    B.tot_bricks = bricks;
}

Batch *new_batch() {
    static thread_local Batch B;
    memset(&B, 0, sizeof(B));
    B.tz = tile_depth();
    return &B;
}

int check_batch_ws(dgr_ws *ws, const Batch &B, bool geom, bool step) {
    if (!ws) return DGR_ERR_ARG;
    const dgr_ws_plan &p = ws->plan;
    if (B.tot_g > p.max_n || B.tot_tiles > p.max_tiles) return DGR_ERR_WS_TOO_SMALL;
    if (B.n > (p.max_inst > 0 ? p.max_inst : 1)) return DGR_ERR_WS_TOO_SMALL;
    if (geom) {
        long long tab_cap = (long long)p.max_views * p.max_nu;
        long long rows_cap = (long long)(p.max_inst > 0 ? p.max_inst : 1) * p.max_nv;
        if (B.tot_tab > tab_cap || B.tot_views > p.max_views || B.tot_rows > rows_cap ||
            B.tot_rays > (long long)p.max_views * p.max_nu * p.max_nv)
            return DGR_ERR_WS_TOO_SMALL;
    }
    if (step) {
        long long vox = 0;
        for (int i = 0; i < B.n; ++i) vox += (long long)B.in[i].g.nx * B.in[i].g.ny * B.in[i].g.nz;
        if (vox > p.max_vox || B.tot_rays > p.max_rays) return DGR_ERR_WS_TOO_SMALL;
    }
    return DGR_OK;
}

}  // namespace

int dgr_voxelize_count(const dgr_grid *grid, int n, const float *mu, const float *s,
                       const float *q, float k_trunc, long long *pairs, long long *items,
                       dgr_ws *ws, cudaStream_t stream) {
    if (!gauss_args_ok(grid, n, mu, s, q, mu, k_trunc) || !pairs || !items) return DGR_ERR_ARG;
    Batch &B = *new_batch();
    B.n = 1;
    Inst &I = B.in[0];
    set_grid(I, *grid, k_trunc);
    I.n = n;
    // rho is not needed for the integers; mu stands in as a valid pointer
    I.mu = mu; I.s = s; I.q = q; I.rho = mu;
    finish(B, false);
    int rc = check_batch_ws(ws, B, false, false);
    if (rc) return rc;
    Prep *prep = ws_ptr<Prep>(ws, ws->prep);
    uint32_t *itemcnt = ws_ptr<uint32_t>(ws, ws->itemcnt);
    int *status = ws_ptr<int>(ws, ws->status);
    cudaError_t e = launch_prep(B, prep, itemcnt, status, stream);
    if (e == cudaSuccess) e = launch_count_pairs(B, prep, ws, ~0ull, stream);
    if (e == cudaSuccess && n > 0)
        e = scan_u32(itemcnt, ws_ptr<uint32_t>(ws, ws->item_off), n, ~0ull, status, 0,
                     ws_ptr<unsigned long long>(ws, ws->scan_tmp), stream);
    uint32_t tp = 0, ti = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&tp, ws_ptr<uint32_t>(ws, ws->tile_off) + B.tot_tiles, 4,
                            cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync(&ti, ws_ptr<uint32_t>(ws, ws->item_off) + n, 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    *pairs = tp;
    *items = ti;
    return cuda_rc(e);
}

int dgr_voxelize(const dgr_grid *grid, int n, const float *mu, const float *s, const float *q,
                 const float *rho, float k_trunc, float *vol, dgr_ws *ws, cudaStream_t stream) {
    if (!gauss_args_ok(grid, n, mu, s, q, rho, k_trunc) || !vol) return DGR_ERR_ARG;
    Batch &B = *new_batch();
    B.n = 1;
    Inst &I = B.in[0];
    set_grid(I, *grid, k_trunc);
    I.n = n; I.mu = mu; I.s = s; I.q = q; I.rho = rho; I.vol = vol;
    finish(B, false);
    int rc = check_batch_ws(ws, B, false, false);
    if (rc) return rc;
    Prep *prep = ws_ptr<Prep>(ws, ws->prep);
    cudaError_t e = launch_prep(B, prep, ws_ptr<uint32_t>(ws, ws->itemcnt), ws_ptr<int>(ws, ws->status), stream);
    if (e == cudaSuccess) e = launch_voxelize(B, prep, ws, g_deterministic, stream);
    return cuda_rc(e);
}

int dgr_voxelize_backward(const dgr_grid *grid, int n, const float *mu, const float *s,
                          const float *q, const float *rho, float k_trunc, const float *grad_vol,
                          float *g_mu, float *g_s, float *g_q, float *g_rho, dgr_ws *ws,
                          cudaStream_t stream) {
    if (!gauss_args_ok(grid, n, mu, s, q, rho, k_trunc) || !grad_vol) return DGR_ERR_ARG;
    if (n > 0 && (!g_mu || !g_s || !g_q || !g_rho)) return DGR_ERR_ARG;
    Batch &B = *new_batch();
    B.n = 1;
    Inst &I = B.in[0];
    set_grid(I, *grid, k_trunc);
    I.n = n; I.mu = mu; I.s = s; I.q = q; I.rho = rho;
    I.gvol = const_cast<float *>(grad_vol);
    I.g_mu = g_mu; I.g_s = g_s; I.g_q = g_q; I.g_rho = g_rho;
    finish(B, false);
    int rc = check_batch_ws(ws, B, false, false);
    if (rc) return rc;
    Prep *prep = ws_ptr<Prep>(ws, ws->prep);
    cudaError_t e = launch_prep(B, prep, ws_ptr<uint32_t>(ws, ws->itemcnt), ws_ptr<int>(ws, ws->status), stream);
    if (e == cudaSuccess) e = launch_voxelize_backward(B, prep, ws, stream);
    return cuda_rc(e);
}

static int proj_batch(const dgr_grid *grid, const dgr_geom *geom, const float *vol, const float *sino,
                      dgr_ws *ws, Batch *&Bout) {
    if (!grid_ok(grid) || !geom_ok(geom) || !vol || !sino || !ws) return DGR_ERR_ARG;
    if (!geom_fits_grid(grid, geom)) return DGR_ERR_ARG;
    if ((long long)grid->nx * grid->ny * grid->nz >= (1ll << 31)) return DGR_ERR_ARG;
    Batch &B = *new_batch();
    B.n = 1;
    Inst &I = B.in[0];
    set_grid(I, *grid, 3.0f);
    set_geom(I, *geom);
    I.vol = const_cast<float *>(vol);
    I.gvol = const_cast<float *>(vol);  // dgr_backproject writes here
    I.sino = const_cast<float *>(sino);
    finish(B, true);
    int rc = check_batch_ws(ws, B, true, false);
    if (rc) return rc;
    Bout = &B;
    return DGR_OK;
}

int dgr_project(const dgr_grid *grid, const dgr_geom *geom, const float *vol, float *sino,
                dgr_ws *ws, cudaStream_t stream) {
    Batch *B = nullptr;
    int rc = proj_batch(grid, geom, vol, sino, ws, B);
    if (rc) return rc;
    RayXY *tab = ws_ptr<RayXY>(ws, ws->rayxy);
    cudaError_t e = cudaSuccess;
    Inst &I = B->in[0];
    const long long vox = (long long)grid->nx * grid->ny * grid->nz;
    if (ws->plan.max_vox >= vox) {
        // a z-fastest copy in the workspace feeds the row-warp projector
        float *zf = ws_ptr<float>(ws, ws->vol);
        e = launch_vol_zfast(*grid, vol, zf, stream);
        I.vol = zf;
        I.vsz = 1;
        I.vsy = grid->nz;
        I.vsx = grid->ny * grid->nz;
    }
    if (e == cudaSuccess) e = launch_ray_tables(*B, tab, stream);
    if (e == cudaSuccess) e = launch_project(*B, tab, ws_ptr<int>(ws, ws->status), stream);
    return cuda_rc(e);
}

int dgr_backproject(const dgr_grid *grid, const dgr_geom *geom, const float *sino, float *vol,
                    dgr_ws *ws, cudaStream_t stream) {
    Batch *B = nullptr;
    int rc = proj_batch(grid, geom, vol, sino, ws, B);
    if (rc) return rc;
    RayXY *tab = ws_ptr<RayXY>(ws, ws->rayxy);
    cudaError_t e = launch_ray_tables(*B, tab, stream);
    if (e == cudaSuccess) e = launch_backproject(*B, tab, ws_ptr<float>(ws, ws->sino_scaled), ws_ptr<int>(ws, ws->acc), ws->plan.max_vox, ws_ptr<int>(ws, ws->status), stream);
    return cuda_rc(e);
}

int dgr_l1_residual(const float *pred, const float *meas, long long m, float weight, float *resid,
                    float *loss, dgr_ws *ws, cudaStream_t stream) {
    if (!pred || !meas || !resid || !loss || !ws || m <= 0 || !isfinite(weight)) return DGR_ERR_ARG;
    return cuda_rc(launch_l1_single(pred, meas, m, weight, resid, loss, ws_ptr<float>(ws, ws->loss_part),
                                    stream));
}

static bool weights_ok(const dgr_problem *P) {
    auto ok = [](float w) { return isfinite(w) && w >= 0.f; };
    return ok(P->w_l1) && ok(P->w_ssim) && ok(P->w_tv) && ok(P->ssim_range);
}

// objective weights and SSIM constants of an instance (all weights 0: L1 alone)
static void set_objective(Inst &I, const dgr_problem &P) {
    const bool none = P.w_l1 == 0.f && P.w_ssim == 0.f && P.w_tv == 0.f;
    I.w_l1 = none ? 1.f : P.w_l1;
    I.w_ssim = none ? 0.f : P.w_ssim;
    I.w_tv = none ? 0.f : P.w_tv;
    const float L = P.ssim_range > 0.f ? P.ssim_range : 1.f;
    I.ssim_c1 = (0.01f * L) * (0.01f * L);
    I.ssim_c2 = (0.03f * L) * (0.03f * L);
}

static int problem_ok(const dgr_problem *P) {
    return P && grid_ok(&P->grid) && P->grid.z0 == 0 && geom_ok(&P->geom) && k_ok(P->k_trunc) && weights_ok(P) &&
           geom_fits_grid(&P->grid, &P->geom) && isfinite(P->lr0) && isfinite(P->lr1) &&
           P->lr0 > 0.f && P->lr1 > 0.f && P->n_iters >= 1 && P->beta1 >= 0.f && P->beta1 < 1.f &&
           P->beta2 >= 0.f && P->beta2 < 1.f && P->eps > 0.f &&
           (long long)P->grid.nx * P->grid.ny * P->grid.nz < (1ll << 31);
}

static int params_ok(const dgr_params *p) {
    return p && p->n >= 0 &&
           (p->n == 0 || (p->mu && p->s && p->q && p->rho && p->theta && p->m && p->v &&
                          aligned16(p->q))) &&
           p->step;
}

int dgr_params_init(const dgr_problem *prob, const dgr_params *p, cudaStream_t stream) {
    if (!problem_ok(prob) || !params_ok(p)) return DGR_ERR_ARG;
    return cuda_rc(launch_params_init(*prob, *p, stream));
}

int dgr_adam(const dgr_problem *prob, const dgr_params *p, const float *g_mu, const float *g_s,
             const float *g_q, const float *g_rho, cudaStream_t stream) {
    if (!problem_ok(prob) || !params_ok(p) || (p->n > 0 && (!g_mu || !g_s || !g_q || !g_rho)))
        return DGR_ERR_ARG;
    Batch &B = *new_batch();
    B.n = 1;
    Inst &I = B.in[0];
    set_grid(I, prob->grid, prob->k_trunc);
    I.n = p->n;
    I.g0 = 0;
    I.mu = p->mu; I.s = p->s; I.q = p->q; I.rho = p->rho;
    I.mu_w = p->mu; I.s_w = p->s; I.q_w = p->q; I.rho_w = p->rho;
    I.theta = p->theta; I.m = p->m; I.v = p->v; I.step = p->step; I.gacc = p->grad_accum;
    I.lr0 = prob->lr0; I.lr1 = prob->lr1; I.b1 = prob->beta1; I.b2 = prob->beta2; I.eps = prob->eps;
    I.n_iters = prob->n_iters;
    I.g_mu = const_cast<float *>(g_mu); I.g_s = const_cast<float *>(g_s);
    I.g_q = const_cast<float *>(g_q); I.g_rho = const_cast<float *>(g_rho);
    B.tot_g = p->n;
    return cuda_rc(launch_adam(B, stream));
}

// voxelize -> project -> L1 -> backproject -> voxelize adjoint -> Adam, for a
// batch of problems, one launch per phase
// ev: phase events (DGR_STEP_EVENTS) or nullptr; kev: optional events
// around the main kernels of the backprojector, the projector, the voxelizer
// and the voxelize adjoint (2 each)
static int step_batch(int n_inst, const dgr_problem *probs, const dgr_params *params,
                      const float *const *measured, float *loss_out, dgr_ws *ws,
                      cudaStream_t stream, cudaEvent_t *ev, const cudaEvent_t *kev = nullptr) {
    if (n_inst < 1 || n_inst > MAX_INST || !probs || !params || !measured || !loss_out || !ws)
        return DGR_ERR_ARG;
    Batch &B = *new_batch();
    B.n = n_inst;
    for (int i = 0; i < n_inst; ++i) {
        const dgr_problem *P = probs + i;
        const dgr_params *p = params + i;
        if (!problem_ok(P) || !params_ok(p) || !measured[i]) return DGR_ERR_ARG;
        Inst &I = B.in[i];
        set_grid(I, P->grid, P->k_trunc);
        set_geom(I, P->geom);
        I.n = p->n;
        I.mu = p->mu; I.s = p->s; I.q = p->q; I.rho = p->rho;
        I.mu_w = p->mu; I.s_w = p->s; I.q_w = p->q; I.rho_w = p->rho;
        I.theta = p->theta; I.m = p->m; I.v = p->v; I.step = p->step; I.gacc = p->grad_accum;
        I.meas = measured[i];
        I.loss = loss_out + i;
        I.lr0 = P->lr0; I.lr1 = P->lr1; I.b1 = P->beta1; I.b2 = P->beta2; I.eps = P->eps;
        I.n_iters = P->n_iters;
        set_objective(I, *P);
    }
    finish(B, true);
    loss_tiles(B);
    int rc = check_batch_ws(ws, B, true, true);
    if (rc) return rc;
    {
        const dgr_ws_plan &p = ws->plan;
        const int ninst = p.max_inst > 0 ? p.max_inst : 1;
        if ((size_t)B.tot_st > ssim_tiles_cap(p.max_views, p.max_nu, p.max_nv, ninst) ||
            (size_t)B.tot_tv > tv_tiles_cap(p.max_vox, ninst))
            return DGR_ERR_WS_TOO_SMALL;
    }
    bool any_ssim = false, any_tv = false;
    for (int i = 0; i < n_inst; ++i) {
        any_ssim = any_ssim || B.in[i].w_ssim != 0.f;
        any_tv = any_tv || B.in[i].w_tv != 0.f;
    }
    // per-instance buffers in the workspace: volume (then its gradient),
    // sinogram (prediction, then residual), gradients [mu 3n | s 3n | q 4n | rho n]
    float *vol = ws_ptr<float>(ws, ws->vol);
    float *gvol = ws_ptr<float>(ws, ws->gvol);
    float *sino = ws_ptr<float>(ws, ws->sino);
    float *grads = ws_ptr<float>(ws, ws->grads);
    long long vo = 0;
    for (int i = 0; i < n_inst; ++i) {
        Inst &I = B.in[i];
        I.vol = vol + vo;
        I.gvol = gvol + vo;
        vo += ((long long)I.g.nx * I.g.ny * I.g.nz + 63) / 64 * 64;
        // the step's own volume is z fastest ([nx][ny][nz]): the projector's
        // lanes (consecutive detector rows) then read neighbouring words; the
        // backprojector writes the gradient in the C ABI's layout
        I.vsz = 1;
        I.vsy = I.g.nz;
        I.vsx = I.g.ny * I.g.nz;
        I.sino = sino + I.ray0;
        float *gr = grads + 11ll * I.g0;
        I.g_mu = gr; I.g_s = gr + 3 * I.n; I.g_q = gr + 6 * I.n; I.g_rho = gr + 10 * I.n;
    }
    Prep *prep = ws_ptr<Prep>(ws, ws->prep);
    RayXY *tab = ws_ptr<RayXY>(ws, ws->rayxy);
    int *status = ws_ptr<int>(ws, ws->status);
    auto mark = [&](int i) { return ev ? cudaEventRecord(ev[i], stream) : cudaSuccess; };
    cudaError_t e = mark(0);
    if (e == cudaSuccess) e = launch_prep(B, prep, ws_ptr<uint32_t>(ws, ws->itemcnt), status, stream);
    if (e == cudaSuccess) e = launch_voxelize(B, prep, ws, g_deterministic, stream, kev ? kev + 4 : nullptr);
    if (e == cudaSuccess) e = mark(1);
    if (e == cudaSuccess) e = launch_ray_tables(B, tab, stream);
    if (e == cudaSuccess) e = launch_project(B, tab, ws_ptr<int>(ws, ws->status), stream, kev ? kev + 2 : nullptr);
    if (e == cudaSuccess) e = mark(2);
    float *ssim_g = ws_ptr<float>(ws, ws->ssim_g);
    if (e == cudaSuccess && any_ssim)
        e = launch_ssim(B, ws_ptr<float>(ws, ws->ssim_maps), ws_ptr<float>(ws, ws->ssim_part), ssim_g, stream);
    if (e == cudaSuccess) e = launch_l1(B, ws_ptr<float>(ws, ws->loss_part), any_ssim ? ssim_g : nullptr, stream);
    if (e == cudaSuccess) e = mark(3);
    if (e == cudaSuccess)
        e = launch_backproject(B, tab, ws_ptr<float>(ws, ws->sino_scaled), ws_ptr<int>(ws, ws->acc),
                               ws->plan.max_vox, ws_ptr<int>(ws, ws->status), stream, kev);
    if (e == cudaSuccess && any_tv) e = launch_tv(B, ws_ptr<float>(ws, ws->tv_part), 1, stream);
    if (e == cudaSuccess)
        e = launch_loss_final(B, ws_ptr<float>(ws, ws->loss_part), L1_BLOCKS, ws_ptr<float>(ws, ws->ssim_part),
                              ws_ptr<float>(ws, ws->tv_part), stream);
    if (e == cudaSuccess) e = mark(4);
    if (e == cudaSuccess) e = launch_voxelize_backward(B, prep, ws, stream, kev ? kev + 6 : nullptr);
    if (e == cudaSuccess) e = mark(5);
    if (e == cudaSuccess) e = launch_adam(B, stream);
    if (e == cudaSuccess) e = mark(6);
    return cuda_rc(e);
}

int dgr_step(const dgr_problem *prob, const dgr_params *p, const float *measured,
             float *loss_out, dgr_ws *ws, cudaStream_t stream) {
    return step_batch(1, prob, p, &measured, loss_out, ws, stream, nullptr);
}

int dgr_step_timed(const dgr_problem *prob, const dgr_params *p, const float *measured,
                   float *loss_out, dgr_ws *ws, cudaStream_t stream, cudaEvent_t *events,
                   int n_events) {
    if (!events || n_events < DGR_STEP_EVENTS) return DGR_ERR_ARG;
    return step_batch(1, prob, p, &measured, loss_out, ws, stream, events,
                      n_events >= DGR_STEP_KERNEL_EVENTS ? events + DGR_STEP_EVENTS : nullptr);
}

int dgr_step_batched(int n_inst, const dgr_problem *probs, const dgr_params *params,
                     const float *const *measured, float *loss_out, dgr_ws *ws,
                     cudaStream_t stream) {
    return step_batch(n_inst, probs, params, measured, loss_out, ws, stream, nullptr);
}

int dgr_ssim_loss(const dgr_geom *geom, const float *pred, const float *meas, float data_range,
                  float *grad, float *loss_out, dgr_ws *ws, cudaStream_t stream) {
    if (!geom_ok(geom) || !pred || !meas || !grad || !loss_out || !ws || !isfinite(data_range) ||
        data_range < 0.f)
        return DGR_ERR_ARG;
    Batch &B = *new_batch();
    B.n = 1;
    Inst &I = B.in[0];
    I.n_views = geom->n_views; I.nu = geom->nu; I.nv = geom->nv;
    I.sino = const_cast<float *>(pred);
    I.meas = meas;
    I.loss = loss_out;
    dgr_problem P;
    memset(&P, 0, sizeof(P));
    P.w_ssim = 1.f;
    P.ssim_range = data_range;
    set_objective(I, P);
    B.tot_rays = (long long)I.n_views * I.nu * I.nv;
    loss_tiles(B);
    const dgr_ws_plan &p = ws->plan;
    if (B.tot_rays > p.max_rays || (size_t)B.tot_st > ssim_tiles_cap(p.max_views, p.max_nu, p.max_nv, 1))
        return DGR_ERR_WS_TOO_SMALL;
    cudaError_t e = launch_ssim(B, ws_ptr<float>(ws, ws->ssim_maps), ws_ptr<float>(ws, ws->ssim_part), grad, stream);
    if (e == cudaSuccess) e = launch_loss_final(B, nullptr, 0, ws_ptr<float>(ws, ws->ssim_part), nullptr, stream);
    return cuda_rc(e);
}

int dgr_tv_loss(const dgr_grid *grid, const float *vol, float *grad, float *loss_out, dgr_ws *ws,
                cudaStream_t stream) {
    if (!grid_ok(grid) || !vol || !grad || !loss_out || !ws) return DGR_ERR_ARG;
    if ((long long)grid->nx * grid->ny * grid->nz >= (1ll << 31)) return DGR_ERR_ARG;
    Batch &B = *new_batch();
    B.n = 1;
    Inst &I = B.in[0];
    set_grid(I, *grid, 3.0f);
    I.vol = const_cast<float *>(vol);
    I.gvol = grad;
    I.loss = loss_out;
    dgr_problem P;
    memset(&P, 0, sizeof(P));
    P.w_tv = 1.f;
    set_objective(I, P);
    loss_tiles(B);
    if ((size_t)B.tot_tv > tv_tiles_cap(ws->plan.max_vox, 1)) return DGR_ERR_WS_TOO_SMALL;
    cudaError_t e = launch_tv(B, ws_ptr<float>(ws, ws->tv_part), 0, stream);
    if (e == cudaSuccess) e = launch_loss_final(B, nullptr, 0, nullptr, ws_ptr<float>(ws, ws->tv_part), stream);
    return cuda_rc(e);
}

int dgr_densify(const dgr_grid *grid, const dgr_densify_cfg *cfg, int iters, const dgr_params *in,
                const float *normals, dgr_params *out, int *n_out, dgr_ws *ws, cudaStream_t stream) {
    if (!grid_ok(grid) || grid->z0 != 0 || !cfg || !in || !out || !n_out || !ws || iters < 1)
        return DGR_ERR_ARG;
    if (!(cfg->tau >= 0.f) || !(cfg->theta_frac >= 0.f) || !(cfg->size > 0.f) || cfg->n_max < 1 ||
        cfg->n_max >= (1 << 24))
        return DGR_ERR_ARG;
    if (!params_ok(in) || !in->grad_accum || (in->n > 0 && !normals)) return DGR_ERR_ARG;
    if (!out->mu || !out->s || !out->q || !out->rho || !out->theta || !out->m || !out->v || !out->step ||
        !aligned16(out->q))
        return DGR_ERR_ARG;
    if (in->n > ws->plan.max_n) return DGR_ERR_WS_TOO_SMALL;
    int *counts = reinterpret_cast<int *>(ws_ptr<unsigned>(ws, ws->dens) + 5 * ((size_t)ws->plan.max_n + 1));
    cudaError_t e = launch_densify(*grid, *cfg, iters, *in, normals, *out, ws, counts, stream);
    int h[3] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, counts, sizeof(h), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return DGR_ERR_CUDA;
    *n_out = h[2];
    return DGR_OK;
}

long long dgr_launch_count(void) { return g_launches.load(); }

}  // extern "C"
