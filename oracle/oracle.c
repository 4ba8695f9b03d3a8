/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the DGR hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference arm of bench.py may load this library.  It shares
 * no code, header, table or constant with the CUDA path.
 *
 * What it computes (paper: "Discretized Gaussian Representation for
 * Tomographic Reconstruction", arxiv 2411.04844):
 *
 *   voxelize   V(p) = sum_i G(p, mu_i, Sigma_i) * I_i            (Eq. 3, Eq. 4)
 *              restricted to each Gaussian's local box            (Sec. 4.1,
 *              "Gaussian Effect Confinement"), anchored at the floored centre
 *              ("Discretize and Align", Eq. 6-7), with out-of-volume voxels
 *              dropped (valid mask of Algorithm 1).  The quadratic form is the
 *              direct (p-mu)^T Sigma^-1 (p-mu); the paper's decomposition
 *              (Eq. 9) is algebraically identical and is not used here.
 *   project    P_hat = T(V) (Sec. 4.3): the exact line integral of the
 *              piecewise-constant voxel image along each detector ray,
 *              evaluated with Siddon's plane-crossing merge.
 *   backproject  the exact transpose of project (same segments).
 *   voxelize_backward  analytic gradient of <G_V, V> w.r.t. (mu, s, q, rho),
 *              the gradient flowing through Delta-mu with box and anchor held
 *              constant (Sec. 4.1, end of "Discretize and Align").
 *
 * Readings of the paper taken here:
 *   - voxel i has centre o + (i + 1/2) h; voxel-unit centre coordinate
 *     u = (mu - o)/h - 1/2, so voxel centres are at integers.
 *   - anchor a = floor(u) (mathematical floor, Eq. 6).
 *   - k_trunc > 0: per-axis box [a - R, a + R + 1], R = ceil(k * sigma_a)
 *     (smallest floor-anchored integer box holding the k-sigma bounding box);
 *     k_trunc < 0: the paper's fixed odd box K = -k_trunc, [a - (K-1)/2,
 *     a + (K-1)/2] (Algorithm 1, B' = meshgrid of -(K-1)/2 .. (K-1)/2).
 *   - box integers come from a fixed FP32 operation sequence (below), so that
 *     an FP32 implementation can reproduce them bit for bit; every value is
 *     then computed in FP64.
 *   - Sigma = R(q) diag(s^2) R(q)^T with q = (w, x, y, z) normalised.
 *   - geometry: rotation about z; parallel rays along (cos t, sin t, 0);
 *     cone source at -dso * (cos t, sin t, 0), flat detector at distance dsd
 *     from the source; detector axes e_u = (-sin t, cos t, 0), e_v = z;
 *     pixel centre offsets (i - (n-1)/2) * pitch.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Footprint integers: a fixed FP32 sequence, every operation rounded   */
/* on its own (this file is compiled with -ffp-contract=off).           */
/* ------------------------------------------------------------------ */
static void rot_from_quat_f32(const float qin[4], float R[9])
{
    float w = qin[0], x = qin[1], y = qin[2], z = qin[3];
    float n2 = w * w;
    n2 = n2 + x * x;
    n2 = n2 + y * y;
    n2 = n2 + z * z;
    float inv = 1.0f / sqrtf(n2);
    w = w * inv; x = x * inv; y = y * inv; z = z * inv;
    float xx = x * x, yy = y * y, zz = z * z;
    float xy = x * y, xz = x * z, yz = y * z;
    float wx = w * x, wy = w * y, wz = w * z;
    R[0] = 1.0f - 2.0f * (yy + zz);
    R[1] = 2.0f * (xy - wz);
    R[2] = 2.0f * (xz + wy);
    R[3] = 2.0f * (xy + wz);
    R[4] = 1.0f - 2.0f * (xx + zz);
    R[5] = 2.0f * (yz - wx);
    R[6] = 2.0f * (xz - wy);
    R[7] = 2.0f * (yz + wx);
    R[8] = 1.0f - 2.0f * (xx + yy);
}

/* dims = {nx, ny, nz}; org = grid min corner; outputs anchor[3n] and
 * box[6n] = {lo_x, lo_y, lo_z, hi_x, hi_y, hi_z} (inclusive, clipped to the
 * grid; an axis with lo > hi means the box misses the grid). */
void oracle_footprint(const int dims[3], float h, const float org[3], int n,
                      const float *mu, const float *s, const float *q,
                      float k_trunc, int *anchor, int *box)
{
    for (int g = 0; g < n; ++g) {
        float R[9];
        rot_from_quat_f32(q + 4 * g, R);
        int far = 0;
        for (int a = 0; a < 3; ++a) {
            float u = (mu[3 * g + a] - org[a]) / h;
            u = u - 0.5f;
            /* |u| >= 2^24 voxels: treated as outside the grid */
            if (!(fabsf(u) < 16777216.0f)) { far = 1; u = 0.0f; }
            int an = (int)floorf(u);
            int rad;
            if (k_trunc > 0.0f) {
                float t0 = R[3 * a + 0] * s[3 * g + 0];
                float t1 = R[3 * a + 1] * s[3 * g + 1];
                float t2 = R[3 * a + 2] * s[3 * g + 2];
                float var = t0 * t0;
                var = var + t1 * t1;
                var = var + t2 * t2;
                float sig = sqrtf(var) / h;
                float kr = k_trunc * sig;
                /* a radius beyond the grid only needs to cover the grid */
                rad = kr < 65536.0f ? (int)ceilf(kr) : 65536;
            } else {
                rad = 0; /* fixed box handled below */
            }
            int lo, hi;
            if (k_trunc > 0.0f) {
                lo = an - rad;
                hi = an + rad + 1;
            } else {
                int K = (int)(-k_trunc);
                int half = (K - 1) / 2;
                lo = an - half;
                hi = an + half;
            }
            if (lo < 0) lo = 0;
            if (hi > dims[a] - 1) hi = dims[a] - 1;
            anchor[3 * g + a] = an;
            box[6 * g + a] = lo;
            box[6 * g + 3 + a] = hi;
        }
        if (far)
            for (int a = 0; a < 3; ++a) { box[6 * g + a] = 1; box[6 * g + 3 + a] = 0; }
    }
}

/* ------------------------------------------------------------------ */
/* FP64 Gaussian pieces                                                */
/* ------------------------------------------------------------------ */
static void rot_from_quat_f64(const double qin[4], double R[9], double qn[4], double *qnorm)
{
    double nrm = sqrt(qin[0] * qin[0] + qin[1] * qin[1] + qin[2] * qin[2] + qin[3] * qin[3]);
    double w = qin[0] / nrm, x = qin[1] / nrm, y = qin[2] / nrm, z = qin[3] / nrm;
    if (qn) { qn[0] = w; qn[1] = x; qn[2] = y; qn[3] = z; }
    if (qnorm) *qnorm = nrm;
    R[0] = 1 - 2 * (y * y + z * z);
    R[1] = 2 * (x * y - w * z);
    R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);
    R[4] = 1 - 2 * (x * x + z * z);
    R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);
    R[7] = 2 * (y * z + w * x);
    R[8] = 1 - 2 * (x * x + y * y);
}

/* Precision matrix in voxel units: A = h^2 Sigma^-1 = h^2 R diag(1/s^2) R^T. */
static void precision_voxel(const double R[9], const double s[3], double h, double A[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k)
                acc += R[3 * i + k] * R[3 * j + k] / (s[k] * s[k]);
            A[3 * i + j] = h * h * acc;
        }
}

static double quad_form(const double A[9], const double d[3])
{
    double r = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            r += d[i] * A[3 * i + j] * d[j];
    return r;
}

typedef struct {
    double u[3];   /* voxel-unit centre */
    double A[9];   /* voxel-unit precision */
    double rho;
    int lo[3], hi[3];
} gauss64;

static void make_gauss(double h, const double org[3], const double *mu, const double *s,
                       const double *q, double rho, const int *box, gauss64 *G)
{
    double R[9];
    rot_from_quat_f64(q, R, 0, 0);
    precision_voxel(R, s, h, G->A);
    for (int a = 0; a < 3; ++a) {
        G->u[a] = (mu[a] - org[a]) / h - 0.5;
        G->lo[a] = box[a];
        G->hi[a] = box[3 + a];
    }
    G->rho = rho;
}

/* vol[nz][ny][nx] (x fastest) is overwritten.  brute != 0: every voxel is
 * tested against every Gaussian's box (Eq. 4 with the confinement mask);
 * brute == 0: each Gaussian loops over its own box. */
void oracle_voxelize_core(const int dims[3], double h, const double org[3], int n,
                          const double *mu, const double *s, const double *q,
                          const double *rho, const int *box, int brute, double *vol)
{
    const int nx = dims[0], ny = dims[1], nz = dims[2];
    gauss64 *G = (gauss64 *)malloc(sizeof(gauss64) * (size_t)(n > 0 ? n : 1));
    for (int g = 0; g < n; ++g)
        make_gauss(h, org, mu + 3 * g, s + 3 * g, q + 4 * g, rho[g], box + 6 * g, &G[g]);
    memset(vol, 0, sizeof(double) * (size_t)nx * ny * nz);
    if (brute) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    double acc = 0;
                    for (int g = 0; g < n; ++g) {
                        const gauss64 *P = &G[g];
                        if (x < P->lo[0] || x > P->hi[0] || y < P->lo[1] || y > P->hi[1] ||
                            z < P->lo[2] || z > P->hi[2])
                            continue;
                        double d[3] = {x - P->u[0], y - P->u[1], z - P->u[2]};
                        acc += P->rho * exp(-0.5 * quad_form(P->A, d));
                    }
                    vol[((size_t)z * ny + y) * nx + x] = acc;
                }
    } else {
        /* each z slice is owned by one thread; Gaussians are visited in index
         * order so the FP64 sum order is fixed */
#pragma omp parallel for schedule(dynamic, 1)
        for (int z = 0; z < nz; ++z)
            for (int g = 0; g < n; ++g) {
                const gauss64 *P = &G[g];
                if (z < P->lo[2] || z > P->hi[2]) continue;
                for (int y = P->lo[1]; y <= P->hi[1]; ++y)
                    for (int x = P->lo[0]; x <= P->hi[0]; ++x) {
                        double d[3] = {x - P->u[0], y - P->u[1], z - P->u[2]};
                        vol[((size_t)z * ny + y) * nx + x] += P->rho * exp(-0.5 * quad_form(P->A, d));
                    }
            }
    }
    free(G);
}

/* V at a list of voxels pts[npts][3] = (x, y, z): the brute-force definition
 * (every Gaussian's box tested) restricted to those voxels, for spot checks of
 * volumes too large to evaluate whole. */
void oracle_voxelize_points(const int dims[3], double h, const double org[3], int n,
                            const double *mu, const double *s, const double *q,
                            const double *rho, const int *box, int npts, const int *pts,
                            double *out)
{
    (void)dims;
    gauss64 *G = (gauss64 *)malloc(sizeof(gauss64) * (size_t)(n > 0 ? n : 1));
    for (int g = 0; g < n; ++g)
        make_gauss(h, org, mu + 3 * g, s + 3 * g, q + 4 * g, rho[g], box + 6 * g, &G[g]);
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < npts; ++p) {
        const int x = pts[3 * p], y = pts[3 * p + 1], z = pts[3 * p + 2];
        double acc = 0;
        for (int g = 0; g < n; ++g) {
            const gauss64 *P = &G[g];
            if (x < P->lo[0] || x > P->hi[0] || y < P->lo[1] || y > P->hi[1] || z < P->lo[2] ||
                z > P->hi[2])
                continue;
            double d[3] = {x - P->u[0], y - P->u[1], z - P->u[2]};
            acc += P->rho * exp(-0.5 * quad_form(P->A, d));
        }
        out[p] = acc;
    }
    free(G);
}

/* Analytic gradient of L = <grad_vol, V> with the integers (box, anchor) held
 * fixed.  Per Gaussian, with e = exp(-1/2 d^T A d), d = v - u:
 *   dL/drho = sum G e
 *   dL/du   = rho A sum G e d
 *   dL/dA   = -1/2 rho sum G e d d^T           (A treated as a full matrix)
 * then u = (mu - o)/h - 1/2, A = h^2 R diag(s^-2) R^T, R = R(q / |q|). */
void oracle_voxelize_backward_core(const int dims[3], double h, const double org[3], int n,
                                   const double *mu, const double *s, const double *q,
                                   const double *rho, const int *box, const double *grad_vol,
                                   double *g_mu, double *g_s, double *g_q, double *g_rho)
{
    const int nx = dims[0], ny = dims[1];
#pragma omp parallel for schedule(dynamic, 4)
    for (int g = 0; g < n; ++g) {
        double R[9], qn[4], qnorm, A[9];
        rot_from_quat_f64(q + 4 * g, R, qn, &qnorm);
        precision_voxel(R, s + 3 * g, h, A);
        double u[3];
        for (int a = 0; a < 3; ++a) u[a] = (mu[3 * g + a] - org[a]) / h - 0.5;
        const int *bx = box + 6 * g;
        double M0 = 0, M1[3] = {0, 0, 0}, M2[9] = {0};
        for (int z = bx[2]; z <= bx[5]; ++z)
            for (int y = bx[1]; y <= bx[4]; ++y)
                for (int x = bx[0]; x <= bx[3]; ++x) {
                    double d[3] = {x - u[0], y - u[1], z - u[2]};
                    double e = exp(-0.5 * quad_form(A, d));
                    double ge = grad_vol[((size_t)z * ny + y) * nx + x] * e;
                    M0 += ge;
                    for (int i = 0; i < 3; ++i) {
                        M1[i] += ge * d[i];
                        for (int j = 0; j < 3; ++j) M2[3 * i + j] += ge * d[i] * d[j];
                    }
                }
        double r = rho[g];
        g_rho[g] = M0;
        /* dL/du and dL/dmu */
        for (int i = 0; i < 3; ++i) {
            double acc = 0;
            for (int j = 0; j < 3; ++j) acc += A[3 * i + j] * M1[j];
            g_mu[3 * g + i] = r * acc / h;
        }
        /* dL/dA (full, symmetric) */
        double GA[9];
        for (int i = 0; i < 9; ++i) GA[i] = -0.5 * r * M2[i];
        /* A = h^2 R D R^T, D = diag(1/s^2) */
        const double *sg = s + 3 * g;
        double D[3] = {1 / (sg[0] * sg[0]), 1 / (sg[1] * sg[1]), 1 / (sg[2] * sg[2])};
        /* dL/dD_kk = h^2 (R^T GA R)_kk ; dD_kk/ds_k = -2 / s_k^3 */
        for (int k = 0; k < 3; ++k) {
            double acc = 0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) acc += R[3 * i + k] * GA[3 * i + j] * R[3 * j + k];
            g_s[3 * g + k] = h * h * acc * (-2.0 / (sg[k] * sg[k] * sg[k]));
        }
        /* dL/dR = h^2 (GA + GA^T) R D = 2 h^2 GA R D */
        double gR[9];
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) {
                double acc = 0;
                for (int j = 0; j < 3; ++j) acc += (GA[3 * i + j] + GA[3 * j + i]) * R[3 * j + k];
                gR[3 * i + k] = h * h * acc * D[k];
            }
        /* dR/dqn from the rotation formula */
        double w = qn[0], x = qn[1], y = qn[2], zq = qn[3];
        double gw = 2 * (-zq * gR[1] + y * gR[2] + zq * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
        double gx = 2 * (y * gR[1] + zq * gR[2] + y * gR[3] - 2 * x * gR[4] - w * gR[5] + zq * gR[6] +
                         w * gR[7] - 2 * x * gR[8]);
        double gy = 2 * (-2 * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] + zq * gR[5] - w * gR[6] +
                         zq * gR[7] - 2 * y * gR[8]);
        double gz = 2 * (-2 * zq * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] - 2 * zq * gR[4] +
                         y * gR[5] + x * gR[6] + y * gR[7]);
        double gqn[4] = {gw, gx, gy, gz};
        /* qn = q / |q| */
        double dot = qn[0] * gqn[0] + qn[1] * gqn[1] + qn[2] * gqn[2] + qn[3] * gqn[3];
        for (int i = 0; i < 4; ++i) g_q[4 * g + i] = (gqn[i] - qn[i] * dot) / qnorm;
    }
}

/* ------------------------------------------------------------------ */
/* Projector: Siddon's exact radiological path (Siddon 1985)           */
/* ------------------------------------------------------------------ */
typedef struct {
    int n[3];
    double h, o[3];
} grid64;

/* Ray for detector pixel (iu, iv) of a view at angle th; point S, direction D
 * (points S + alpha D).  The ray is a full line for parallel beam and the
 * line through the source for cone beam (the grid lies between source and
 * detector, so the line and the source->pixel segment cover the same voxels). */
static void ray_of(int beam, double th, int iu, int iv, int nu, int nv, double pu, double pv,
                   double dso, double dsd, double S[3], double D[3])
{
    double c = cos(th), sn = sin(th);
    double rh[3] = {c, sn, 0};
    double eu[3] = {-sn, c, 0};
    double uu = (iu - 0.5 * (nu - 1)) * pu;
    double vv = (iv - 0.5 * (nv - 1)) * pv;
    if (beam == 0) {
        for (int a = 0; a < 3; ++a) {
            S[a] = uu * eu[a] + (a == 2 ? vv : 0.0);
            D[a] = rh[a];
        }
    } else {
        for (int a = 0; a < 3; ++a) {
            double src = -dso * rh[a];
            double pix = (dsd - dso) * rh[a] + uu * eu[a] + (a == 2 ? vv : 0.0);
            S[a] = src;
            D[a] = pix - src;
        }
    }
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Calls f(voxel_index, length) for every segment of the ray inside the grid. */
typedef struct {
    size_t idx;
    double len;
} segment;

static int siddon_segments(const grid64 *G, const double S[3], const double D[3], double *alph,
                           segment *seg)
{
    double amin = -INFINITY, amax = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double lo = G->o[a], hi = G->o[a] + G->n[a] * G->h;
        if (D[a] != 0.0) {
            double a0 = (lo - S[a]) / D[a], a1 = (hi - S[a]) / D[a];
            double mn = a0 < a1 ? a0 : a1, mx = a0 < a1 ? a1 : a0;
            if (mn > amin) amin = mn;
            if (mx < amax) amax = mx;
        } else {
            /* parallel to the planes of this axis: inside iff lo <= S < hi */
            if (!(S[a] >= lo && S[a] < hi)) return 0;
        }
    }
    if (!(amax > amin)) return 0;
    int m = 0;
    alph[m++] = amin;
    alph[m++] = amax;
    for (int a = 0; a < 3; ++a) {
        if (D[a] == 0.0) continue;
        for (int k = 0; k <= G->n[a]; ++k) {
            double al = (G->o[a] + k * G->h - S[a]) / D[a];
            if (al > amin && al < amax) alph[m++] = al;
        }
    }
    qsort(alph, (size_t)m, sizeof(double), cmp_double);
    double dn = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
    int ns = 0;
    for (int k = 1; k < m; ++k) {
        double len = (alph[k] - alph[k - 1]) * dn;
        if (!(len > 0)) continue;
        double mid = 0.5 * (alph[k] + alph[k - 1]);
        int id[3];
        int ok = 1;
        for (int a = 0; a < 3; ++a) {
            id[a] = (int)floor((S[a] + mid * D[a] - G->o[a]) / G->h);
            if (id[a] < 0 || id[a] >= G->n[a]) ok = 0;
        }
        if (!ok) continue;
        seg[ns].idx = ((size_t)id[2] * G->n[1] + id[1]) * G->n[0] + id[0];
        seg[ns].len = len;
        ++ns;
    }
    return ns;
}

/* sino[n_views][nv][nu] (u fastest) is overwritten. */
void oracle_project(const int dims[3], double h, const double org[3], int beam, int n_views,
                    int nu, int nv, double pu, double pv, double dso, double dsd,
                    const double *angles, const double *vol, double *sino)
{
    grid64 G = {{dims[0], dims[1], dims[2]}, h, {org[0], org[1], org[2]}};
    int cap = dims[0] + dims[1] + dims[2] + 8;
    long nrays = (long)n_views * nv * nu;
#pragma omp parallel
    {
        double *alph = (double *)malloc(sizeof(double) * cap);
        segment *seg = (segment *)malloc(sizeof(segment) * cap);
#pragma omp for schedule(dynamic, 64)
        for (long r = 0; r < nrays; ++r) {
            int iu = (int)(r % nu);
            int iv = (int)((r / nu) % nv);
            int k = (int)(r / ((long)nu * nv));
            double S[3], D[3];
            ray_of(beam, angles[k], iu, iv, nu, nv, pu, pv, dso, dsd, S, D);
            int ns = siddon_segments(&G, S, D, alph, seg);
            double acc = 0;
            for (int i = 0; i < ns; ++i) acc += seg[i].len * vol[seg[i].idx];
            sino[r] = acc;
        }
        free(alph);
        free(seg);
    }
}

/* vol[nz][ny][nx] is overwritten with A^T sino (same segments as project). */
void oracle_backproject(const int dims[3], double h, const double org[3], int beam, int n_views,
                        int nu, int nv, double pu, double pv, double dso, double dsd,
                        const double *angles, const double *sino, double *vol)
{
    grid64 G = {{dims[0], dims[1], dims[2]}, h, {org[0], org[1], org[2]}};
    int cap = dims[0] + dims[1] + dims[2] + 8;
    size_t nvox = (size_t)dims[0] * dims[1] * dims[2];
    memset(vol, 0, sizeof(double) * nvox);
    long nrays = (long)n_views * nv * nu;
#pragma omp parallel
    {
        double *alph = (double *)malloc(sizeof(double) * cap);
        segment *seg = (segment *)malloc(sizeof(segment) * cap);
#pragma omp for schedule(dynamic, 64)
        for (long r = 0; r < nrays; ++r) {
            int iu = (int)(r % nu);
            int iv = (int)((r / nu) % nv);
            int k = (int)(r / ((long)nu * nv));
            double S[3], D[3];
            ray_of(beam, angles[k], iu, iv, nu, nv, pu, pv, dso, dsd, S, D);
            int ns = siddon_segments(&G, S, D, alph, seg);
            double w = sino[r];
            for (int i = 0; i < ns; ++i) {
#pragma omp atomic
                vol[seg[i].idx] += seg[i].len * w;
            }
        }
        free(alph);
        free(seg);
    }
}

/* Ray origin/direction exactly as the projector uses them (for tests that
 * build an independent chord matrix). */
void oracle_ray(int beam, double th, int iu, int iv, int nu, int nv, double pu, double pv,
                double dso, double dsd, double *S, double *D)
{
    ray_of(beam, th, iu, iv, nu, nv, pu, pv, dso, dsd, S, D);
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
