// C ABI of libdgr: argument validation, workspace layout, orchestration of the
// kernels on the caller's stream.  See include/dgr.h for the contract.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "dgr_internal.cuh"

using namespace dgr;

std::atomic<long long> dgr::g_launches{0};

namespace {

int g_deterministic = 1;

constexpr int MAX_DIM = 32767;
constexpr int MAX_VIEWS_BP = 1 << 20;

bool grid_ok(const dgr_grid *g) {
    return g && g->nx > 0 && g->ny > 0 && g->nz > 0 && g->nx <= MAX_DIM && g->ny <= MAX_DIM &&
           g->nz <= MAX_DIM && isfinite(g->h) && g->h > 0.f && isfinite(g->ox) &&
           isfinite(g->oy) && isfinite(g->oz);
}

bool k_ok(float k) {
    if (!isfinite(k) || k == 0.f) return false;
    if (k > 0.f) return true;
    const float K = -k;
    return K == floorf(K) && ((int)K % 2 == 1) && K < 65536.f;
}

bool geom_ok(const dgr_geom *geo) {
    if (!geo || !geo->angles) return false;
    if (geo->beam != DGR_PARALLEL && geo->beam != DGR_CONE) return false;
    if (geo->n_views <= 0 || geo->nu <= 0 || geo->nv <= 0 || geo->n_views > MAX_VIEWS_BP) return false;
    if (!(isfinite(geo->pu) && geo->pu > 0.f && isfinite(geo->pv) && geo->pv > 0.f)) return false;
    if (geo->beam == DGR_CONE &&
        !(isfinite(geo->dso) && isfinite(geo->dsd) && geo->dso > 0.f && geo->dsd > geo->dso))
        return false;
    return true;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

bool geom_fits_grid(const dgr_grid *g, const dgr_geom *geo) {
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

int check_ws_grid(dgr_ws *ws, const dgr_grid *g, int n) {
    if (!ws) return DGR_ERR_ARG;
    int tx, ty, tz;
    const int tiles = tile_dims(*g, tx, ty, tz);
    if (n > ws->plan.max_n || tiles > ws->plan.max_tiles) return DGR_ERR_WS_TOO_SMALL;
    return DGR_OK;
}

int check_ws_geom(dgr_ws *ws, const dgr_geom *geo) {
    if (geo->n_views > ws->plan.max_views || geo->nu > ws->plan.max_nu || geo->nv > ws->plan.max_nv)
        return DGR_ERR_WS_TOO_SMALL;
    return DGR_OK;
}

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? DGR_OK : DGR_ERR_CUDA; }

struct Layout {
    size_t status, prep, itemcnt, item_off, tile_cnt, tile_off, tile_fill, scan_tmp, list,
        partials, grads, vol, sino, loss_part, rayxy, sino_scaled, total;
    size_t scan_elems;
};

bool plan_ok(const dgr_ws_plan *p) {
    return p && p->max_n >= 0 && p->max_tiles >= 0 && p->max_pairs >= 0 && p->max_items >= 0 &&
           p->max_vox >= 0 && p->max_rays >= 0 && p->max_views >= 0 && p->max_nu >= 0 &&
           p->max_nv >= 0 && p->max_pairs < (1ll << 32) && p->max_items < (1ll << 32) &&
           p->max_n < (1 << 24) && p->max_tiles < (1 << 24);
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
    L.partials = take(4 * (size_t)NMOM * (size_t)p.max_items);
    L.rayxy = take(ray_table_bytes(p.max_views, p.max_nu, p.max_nv));
    // residual x |D| for the backprojector (standalone calls; the step reuses its sinogram)
    L.sino_scaled = take(4 * (size_t)p.max_views * p.max_nu * p.max_nv);
    L.loss_part = take(4 * (size_t)(L1_BLOCKS + 1));
    L.grads = take(4 * 11 * (size_t)p.max_n);
    L.vol = take(4 * (size_t)p.max_vox);
    L.sino = take(4 * (size_t)p.max_rays);
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
    w->scan_tmp_elems = L.scan_elems;
    if (cudaMemset(w->base + L.status, 0, 256) != cudaSuccess) {
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

int dgr_footprint(const dgr_grid *grid, int n, const float *mu, const float *s, const float *q,
                  float k_trunc, int *anchor, int *box, cudaStream_t stream) {
    if (!grid_ok(grid) || n < 0 || !k_ok(k_trunc)) return DGR_ERR_ARG;
    if (n > 0 && (!mu || !s || !q || !anchor || !box || !aligned16(q))) return DGR_ERR_ARG;
    return cuda_rc(launch_footprint(*grid, n, mu, s, q, k_trunc, anchor, box, stream));
}

static int gauss_args_ok(const dgr_grid *grid, int n, const float *mu, const float *s,
                         const float *q, const float *rho, float k) {
    if (!grid_ok(grid) || n < 0 || !k_ok(k)) return 0;
    if (n > 0 && (!mu || !s || !q || !rho || !aligned16(q))) return 0;
    return 1;
}

int dgr_voxelize_count(const dgr_grid *grid, int n, const float *mu, const float *s,
                       const float *q, float k_trunc, long long *pairs, long long *items,
                       dgr_ws *ws, cudaStream_t stream) {
    if (!gauss_args_ok(grid, n, mu, s, q, mu, k_trunc) || !pairs || !items) return DGR_ERR_ARG;
    int rc = check_ws_grid(ws, grid, n);
    if (rc) return rc;
    Prep *prep = ws_ptr<Prep>(ws, ws->prep);
    uint32_t *itemcnt = ws_ptr<uint32_t>(ws, ws->itemcnt);
    int *status = ws_ptr<int>(ws, ws->status);
    // rho is not needed for the integers; mu stands in as a valid pointer
    cudaError_t e = launch_prep(*grid, n, mu, s, q, mu, k_trunc, prep, itemcnt, status, stream);
    if (e == cudaSuccess) e = launch_count_pairs(*grid, n, prep, ws, ~0ull, stream);
    if (e == cudaSuccess && n > 0)
        e = scan_u32(itemcnt, ws_ptr<uint32_t>(ws, ws->item_off), n, ~0ull, status, 0,
                     ws_ptr<unsigned long long>(ws, ws->scan_tmp), stream);
    int tx, ty, tz;
    const int tiles = tile_dims(*grid, tx, ty, tz);
    uint32_t tp = 0, ti = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&tp, ws_ptr<uint32_t>(ws, ws->tile_off) + tiles, 4, cudaMemcpyDeviceToHost, stream);
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
    int rc = check_ws_grid(ws, grid, n);
    if (rc) return rc;
    Prep *prep = ws_ptr<Prep>(ws, ws->prep);
    cudaError_t e = launch_prep(*grid, n, mu, s, q, rho, k_trunc, prep,
                                ws_ptr<uint32_t>(ws, ws->itemcnt), ws_ptr<int>(ws, ws->status), stream);
    if (e == cudaSuccess) e = launch_voxelize(*grid, n, prep, ws, vol, g_deterministic, stream);
    return cuda_rc(e);
}

int dgr_voxelize_backward(const dgr_grid *grid, int n, const float *mu, const float *s,
                          const float *q, const float *rho, float k_trunc, const float *grad_vol,
                          float *g_mu, float *g_s, float *g_q, float *g_rho, dgr_ws *ws,
                          cudaStream_t stream) {
    if (!gauss_args_ok(grid, n, mu, s, q, rho, k_trunc) || !grad_vol) return DGR_ERR_ARG;
    if (n > 0 && (!g_mu || !g_s || !g_q || !g_rho)) return DGR_ERR_ARG;
    int rc = check_ws_grid(ws, grid, n);
    if (rc) return rc;
    Prep *prep = ws_ptr<Prep>(ws, ws->prep);
    cudaError_t e = launch_prep(*grid, n, mu, s, q, rho, k_trunc, prep,
                                ws_ptr<uint32_t>(ws, ws->itemcnt), ws_ptr<int>(ws, ws->status), stream);
    if (e == cudaSuccess)
        e = launch_voxelize_backward(*grid, n, mu, s, q, rho, prep, grad_vol, g_mu, g_s, g_q, g_rho,
                                     ws, stream);
    return cuda_rc(e);
}

int dgr_project(const dgr_grid *grid, const dgr_geom *geom, const float *vol, float *sino,
                dgr_ws *ws, cudaStream_t stream) {
    if (!grid_ok(grid) || !geom_ok(geom) || !vol || !sino || !ws) return DGR_ERR_ARG;
    if (!geom_fits_grid(grid, geom)) return DGR_ERR_ARG;
    int rc = check_ws_geom(ws, geom);
    if (rc) return rc;
    RayXY *tab = ws_ptr<RayXY>(ws, ws->rayxy);
    cudaError_t e = launch_ray_tables(*grid, *geom, tab, stream);
    if (e == cudaSuccess) e = launch_project(*grid, *geom, tab, vol, sino, stream);
    return cuda_rc(e);
}

int dgr_backproject(const dgr_grid *grid, const dgr_geom *geom, const float *sino, float *vol,
                    dgr_ws *ws, cudaStream_t stream) {
    if (!grid_ok(grid) || !geom_ok(geom) || !vol || !sino || !ws) return DGR_ERR_ARG;
    if (!geom_fits_grid(grid, geom)) return DGR_ERR_ARG;
    int rc = check_ws_geom(ws, geom);
    if (rc) return rc;
    RayXY *tab = ws_ptr<RayXY>(ws, ws->rayxy);
    cudaError_t e = launch_ray_tables(*grid, *geom, tab, stream);
    if (e == cudaSuccess)
        e = launch_backproject(*grid, *geom, tab, sino, ws_ptr<float>(ws, ws->sino_scaled), vol, stream);
    return cuda_rc(e);
}

int dgr_l1_residual(const float *pred, const float *meas, long long m, float *resid, float *loss,
                    dgr_ws *ws, cudaStream_t stream) {
    if (!pred || !meas || !resid || !loss || !ws || m <= 0) return DGR_ERR_ARG;
    return cuda_rc(launch_l1(pred, meas, m, resid, loss, ws_ptr<float>(ws, ws->loss_part), stream));
}

static int problem_ok(const dgr_problem *P) {
    return P && grid_ok(&P->grid) && geom_ok(&P->geom) && k_ok(P->k_trunc) &&
           geom_fits_grid(&P->grid, &P->geom) && isfinite(P->lr0) && isfinite(P->lr1) &&
           P->lr0 > 0.f && P->lr1 > 0.f && P->n_iters >= 1 && P->beta1 >= 0.f && P->beta1 < 1.f &&
           P->beta2 >= 0.f && P->beta2 < 1.f && P->eps > 0.f;
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

static int step_impl(const dgr_problem *prob, const dgr_params *p, const float *measured,
                     float *loss_out, dgr_ws *ws, cudaStream_t stream, cudaEvent_t *ev) {
    if (!problem_ok(prob) || !params_ok(p) || !measured || !loss_out || !ws) return DGR_ERR_ARG;
    const dgr_grid &g = prob->grid;
    const dgr_geom &geo = prob->geom;
    int rc = check_ws_grid(ws, &g, p->n);
    if (rc) return rc;
    rc = check_ws_geom(ws, &geo);
    if (rc) return rc;
    const long long nvox = (long long)g.nx * g.ny * g.nz;
    const long long nrays = (long long)geo.n_views * geo.nv * geo.nu;
    if (nvox > ws->plan.max_vox || nrays > ws->plan.max_rays) return DGR_ERR_WS_TOO_SMALL;
    const int n = p->n;
    float *vol = ws_ptr<float>(ws, ws->vol);     // volume, then its gradient (same buffer)
    float *sino = ws_ptr<float>(ws, ws->sino);   // prediction, then residual (in place)
    float *grads = ws_ptr<float>(ws, ws->grads);
    Prep *prep = ws_ptr<Prep>(ws, ws->prep);
    RayXY *tab = ws_ptr<RayXY>(ws, ws->rayxy);
    int *status = ws_ptr<int>(ws, ws->status);
    auto mark = [&](int i) { return ev ? cudaEventRecord(ev[i], stream) : cudaSuccess; };
    cudaError_t e = mark(0);
    if (e == cudaSuccess)
        e = launch_prep(g, n, p->mu, p->s, p->q, p->rho, prob->k_trunc, prep,
                        ws_ptr<uint32_t>(ws, ws->itemcnt), status, stream);
    if (e == cudaSuccess) e = launch_voxelize(g, n, prep, ws, vol, g_deterministic, stream);
    if (e == cudaSuccess) e = mark(1);
    if (e == cudaSuccess) e = launch_ray_tables(g, geo, tab, stream);
    if (e == cudaSuccess) e = launch_project(g, geo, tab, vol, sino, stream);
    if (e == cudaSuccess) e = mark(2);
    if (e == cudaSuccess)
        e = launch_l1(sino, measured, nrays, sino, loss_out, ws_ptr<float>(ws, ws->loss_part), stream);
    if (e == cudaSuccess) e = mark(3);
    if (e == cudaSuccess)
        e = launch_backproject(g, geo, tab, sino, ws_ptr<float>(ws, ws->sino_scaled), vol, stream);
    if (e == cudaSuccess) e = mark(4);
    if (e == cudaSuccess)
        e = launch_voxelize_backward(g, n, p->mu, p->s, p->q, p->rho, prep, vol, grads,
                                     grads + 3 * (size_t)n, grads + 6 * (size_t)n,
                                     grads + 10 * (size_t)n, ws, stream);
    if (e == cudaSuccess) e = mark(5);
    if (e == cudaSuccess) e = launch_adam(*prob, *p, grads, stream);
    if (e == cudaSuccess) e = mark(6);
    return cuda_rc(e);
}

int dgr_step(const dgr_problem *prob, const dgr_params *p, const float *measured,
             float *loss_out, dgr_ws *ws, cudaStream_t stream) {
    return step_impl(prob, p, measured, loss_out, ws, stream, nullptr);
}

int dgr_step_timed(const dgr_problem *prob, const dgr_params *p, const float *measured,
                   float *loss_out, dgr_ws *ws, cudaStream_t stream, cudaEvent_t *events,
                   int n_events) {
    if (!events || n_events < DGR_STEP_EVENTS) return DGR_ERR_ARG;
    return step_impl(prob, p, measured, loss_out, ws, stream, events);
}

long long dgr_launch_count(void) { return g_launches.load(); }

}  // extern "C"
