/*
 * csgs_oracle.c -- plain FP64 CPU oracle for sensitivity scoring of a 3D Gaussian
 * scene and for sensitivity sampling of a weighted coreset.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls this
 * file; only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg use it.  It shares no code, header, table or constant with the CUDA path.
 *
 * What it computes (paper, Sec. 3 "Scalar rendering function", "A pruned 3DGS
 * scene", Eq. (sen), Algorithm 1), written out literally and slowly:
 *   for every view and every pixel (brute force over ALL Gaussians, no tiles):
 *     k(g,q)    projected (EWA) Gaussian value at the pixel centre, truncated to
 *               the Mahalanobis ellipse d^T Sigma'^-1 d <= cut2 (3-sigma footprint,
 *               proof of Thm. 1 in the appendix);
 *     rho       = min(rho_max, alpha * k), pairs with rho < alpha_min are skipped;
 *     order     ascending camera-space depth of the means, ties by lower index;
 *     T         prefix transmittance prod_{j before i} (1 - rho_j); traversal stops
 *               before the Gaussian that would bring T below t_min;
 *     a         = c * rho * T per channel, A = sum_i a;
 *   imp(g,q) = a / A over queries with A > 0, s = max over queries (Eq. sen) or the
 *   aggregated variants of Sec. 3 "Sensitivity at Multiple Resolutions";
 *   p = s / S, i.i.d. inverse-CDF draws, w = n / (m p) (Algorithm 1, steps 3-5).
 *
 * Every quantity is FP64; inputs arrive as float32 arrays and are widened.
 * The only shortcut is an exact implication used to skip Gaussians early: the
 * ellipse d^T Sigma'^-1 d <= c satisfies |dx| <= sqrt(c Sigma'_xx) (and likewise
 * for y), so a Gaussian outside that box cannot pass the footprint test.
 *
 * Straddle flags: where the GPU (FP32) and this oracle (FP64) may take a
 * threshold decision differently, the query is flagged.  A query is flagged when a
 * tested value lies within a relative band of a threshold (footprint cut,
 * alpha_min, t_min) or two consecutive contributors have depths within a relative
 * band.  The bands are inputs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- types */

typedef struct {
    int64_t n;
    int32_t sh_degree;
    int32_t pad;
    const float* means;          /* [3][n] */
    const float* log_scales;     /* [3][n] */
    const float* quats;          /* [4][n] (w,x,y,z) */
    const float* opacity_logits; /* [n] */
    const float* sh;             /* [(d+1)^2][3][n] */
} or_scene;

typedef struct {
    double alpha_min;
    double rho_max;
    double t_min;
    double cut2;
    double dilation;
    double clamp_fov;
    double obj_w[3];
    double band_cut;
    double band_alpha;
    double band_tmin;  /* safety factor on the accumulated error bound of T */
    double band_depth;
    int32_t resolution; /* 0 pixel, 1 scene, 2 channel, 3 tile, 4 image */
    int32_t variant;    /* 0 L1 colour, 1 L2 colour, 2 no-colour */
    int32_t tile;       /* tile edge (pixels) for the per-tile resolution */
    int32_t pad;
} or_opts;

enum { RES_PIXEL = 0, RES_SCENE = 1, RES_CHANNEL = 2, RES_TILE = 3, RES_IMAGE = 4 };
enum { VAR_L1 = 0, VAR_L2 = 1, VAR_NC = 2 };

typedef struct {
    double R[9], t[3], fx, fy, cx, cy, near_z;
    int W, H;
} ocam;

/* per-view projected Gaussian (SoA for the scan fields, AoS for the rest) */
typedef struct {
    double a, b, c;   /* conic = Sigma'^-1 (symmetric: a, b, c) */
    double depth;
    double alpha;     /* weighted opacity w_i * alpha_i */
    double rgb[3];
} oattr;

typedef struct {
    int64_t n;
    double* mx;
    double* my;
    double* rx; /* half-width of the pre-test box, +inf if invalid -> use valid */
    double* ry;
    uint8_t* valid;
    oattr* at;
} oview;

typedef struct {
    double depth;
    int64_t gid;
    double rho;
    int viol;    /* w alpha k >= 1: the factor 1 - w rho would not be positive unclamped */
    int clamped; /* rho = rho_max exactly */
} ocand;

typedef struct {
    int64_t gid;
    double rho, T;
    double c[3];
} oterm;

/* ---------------------------------------------------------------- helpers */

static void read_cam(const float* r, ocam* c) {
    for (int k = 0; k < 9; ++k) c->R[k] = r[k];
    for (int k = 0; k < 3; ++k) c->t[k] = r[9 + k];
    c->fx = r[12];
    c->fy = r[13];
    c->cx = r[14];
    c->cy = r[15];
    c->W = (int)r[16];
    c->H = (int)r[17];
    c->near_z = r[18];
}

/* Real spherical harmonics up to degree 3, orthonormal on the unit sphere, with the
 * sign convention of the 3DGS colour model (cited by the paper, Sec. 2).  Each
 * constant is its closed-form normalisation sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!)
 * times the factor of the Cartesian polynomial. */
void or_sh_basis(int deg, const double* dir, double* Y) {
    const double pi = 3.14159265358979323846;
    double x = dir[0], y = dir[1], z = dir[2];
    Y[0] = 0.5 * sqrt(1.0 / pi);
    if (deg < 1) return;
    double c1 = sqrt(3.0 / (4.0 * pi));
    Y[1] = -c1 * y;
    Y[2] = c1 * z;
    Y[3] = -c1 * x;
    if (deg < 2) return;
    double xx = x * x, yy = y * y, zz = z * z;
    double c2a = 0.5 * sqrt(15.0 / pi), c2b = 0.25 * sqrt(5.0 / pi), c2c = 0.25 * sqrt(15.0 / pi);
    Y[4] = c2a * x * y;
    Y[5] = -c2a * y * z;
    Y[6] = c2b * (2.0 * zz - xx - yy);
    Y[7] = -c2a * x * z;
    Y[8] = c2c * (xx - yy);
    if (deg < 3) return;
    double c3a = 0.25 * sqrt(35.0 / (2.0 * pi)), c3b = 0.5 * sqrt(105.0 / pi);
    double c3c = 0.25 * sqrt(21.0 / (2.0 * pi)), c3d = 0.25 * sqrt(7.0 / pi);
    double c3e = 0.25 * sqrt(105.0 / pi);
    Y[9] = -c3a * y * (3.0 * xx - yy);
    Y[10] = c3b * x * y * z;
    Y[11] = -c3c * y * (4.0 * zz - xx - yy);
    Y[12] = c3d * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
    Y[13] = -c3c * x * (4.0 * zz - xx - yy);
    Y[14] = c3e * z * (xx - yy);
    Y[15] = -c3a * x * (xx - 3.0 * yy);
}

/* Projection of one Gaussian into one camera (EWA splatting, the kernel k of
 * Sec. 3 "Scalar rendering function"; readings of the unstated details: J
 * linearised at the mean with x/z, y/z clamped, low-pass dilation added to the
 * diagonal, pixel centres at integer coordinates).
 * out[16]: valid, mx, my, conic a, b, c, cov xx, xy, yy, depth, alpha, r, g, b,
 *          camera x, camera y. */
static int project_one(const or_scene* sc, int64_t i, const ocam* cm, const or_opts* o,
                       double wi, double* out) {
    const int64_t n = sc->n;
    memset(out, 0, 16 * sizeof(double));
    double mu[3] = {sc->means[i], sc->means[n + i], sc->means[2 * n + i]};
    double pc[3];
    for (int r = 0; r < 3; ++r)
        pc[r] = cm->R[3 * r] * mu[0] + cm->R[3 * r + 1] * mu[1] + cm->R[3 * r + 2] * mu[2] + cm->t[r];
    double x = pc[0], y = pc[1], z = pc[2];
    if (!(z > cm->near_z)) return 0;
    double alpha = wi / (1.0 + exp(-(double)sc->opacity_logits[i]));
    if (!(alpha > 0.0)) return 0;

    /* 3D covariance Sigma = Rq diag(s^2) Rq^T */
    double s[3];
    for (int k = 0; k < 3; ++k) s[k] = exp((double)sc->log_scales[k * n + i]);
    double qw = sc->quats[i], qx = sc->quats[n + i], qy = sc->quats[2 * n + i], qz = sc->quats[3 * n + i];
    double qn = sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
    qw /= qn; qx /= qn; qy /= qn; qz /= qn;
    double Rq[9] = {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy),
                    2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx),
                    2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)};
    double Sig[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += Rq[3 * r + k] * s[k] * s[k] * Rq[3 * c + k];
            Sig[3 * r + c] = acc;
        }
    /* camera-space covariance R Sigma R^T */
    double tmp[9], Sc[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += cm->R[3 * r + k] * Sig[3 * k + c];
            tmp[3 * r + c] = acc;
        }
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += tmp[3 * r + k] * cm->R[3 * c + k];
            Sc[3 * r + c] = acc;
        }
    /* Jacobian of the perspective map at the (clamped) mean */
    double limx = o->clamp_fov * 0.5 * cm->W / cm->fx;
    double limy = o->clamp_fov * 0.5 * cm->H / cm->fy;
    double txz = x / z, tyz = y / z;
    if (txz < -limx) txz = -limx;
    if (txz > limx) txz = limx;
    if (tyz < -limy) tyz = -limy;
    if (tyz > limy) tyz = limy;
    double J[6] = {cm->fx / z, 0.0, -cm->fx * txz / z, 0.0, cm->fy / z, -cm->fy * tyz / z};
    double JS[6];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += J[3 * r + k] * Sc[3 * k + c];
            JS[3 * r + c] = acc;
        }
    double cov[4];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += JS[3 * r + k] * J[3 * c + k];
            cov[2 * r + c] = acc;
        }
    double ca = cov[0] + o->dilation, cb = 0.5 * (cov[1] + cov[2]), cc = cov[3] + o->dilation;
    double det = ca * cc - cb * cb;
    if (!(det > 0.0)) return 0;

    /* view-dependent colour: SH evaluated along the direction camera -> mean */
    double cpos[3];
    for (int k = 0; k < 3; ++k)
        cpos[k] = -(cm->R[k] * cm->t[0] + cm->R[3 + k] * cm->t[1] + cm->R[6 + k] * cm->t[2]);
    double d[3] = {mu[0] - cpos[0], mu[1] - cpos[1], mu[2] - cpos[2]};
    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    d[0] /= dn; d[1] /= dn; d[2] /= dn;
    double Y[16];
    int deg = sc->sh_degree;
    int nk = (deg + 1) * (deg + 1);
    or_sh_basis(deg, d, Y);
    double rgb[3];
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.0;
        for (int k = 0; k < nk; ++k) acc += (double)sc->sh[(int64_t)(3 * k + ch) * n + i] * Y[k];
        acc += 0.5;
        rgb[ch] = acc > 0.0 ? acc : 0.0;
    }
    out[0] = 1.0;
    out[1] = cm->fx * x / z + cm->cx;
    out[2] = cm->fy * y / z + cm->cy;
    out[3] = cc / det;
    out[4] = -cb / det;
    out[5] = ca / det;
    out[6] = ca;
    out[7] = cb;
    out[8] = cc;
    out[9] = z;
    out[10] = alpha;
    out[11] = rgb[0];
    out[12] = rgb[1];
    out[13] = rgb[2];
    out[14] = x;
    out[15] = y;
    return 1;
}

/* Project every Gaussian of the scene into one camera.  w: per-Gaussian weight
 * (NULL = all ones). out: [n][16] as in project_one. */
int or_project(const or_scene* sc, const float* cam, const or_opts* o, const double* w, double* out) {
    ocam cm;
    read_cam(cam, &cm);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < sc->n; ++i) project_one(sc, i, &cm, o, w ? w[i] : 1.0, out + 16 * i);
    return 0;
}

static int build_view(const or_scene* sc, const float* cam, const or_opts* o, const double* w, oview* v,
                      ocam* cm) {
    read_cam(cam, cm);
    int64_t n = sc->n;
    v->n = n;
    v->mx = (double*)malloc(sizeof(double) * n);
    v->my = (double*)malloc(sizeof(double) * n);
    v->rx = (double*)malloc(sizeof(double) * n);
    v->ry = (double*)malloc(sizeof(double) * n);
    v->valid = (uint8_t*)malloc(n);
    v->at = (oattr*)malloc(sizeof(oattr) * n);
    if (!v->mx || !v->my || !v->rx || !v->ry || !v->valid || !v->at) return -1;
    const double grow = o->cut2 * (1.0 + o->band_cut);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double p[16];
        int ok = project_one(sc, i, cm, o, w ? w[i] : 1.0, p);
        v->valid[i] = (uint8_t)ok;
        v->mx[i] = p[1];
        v->my[i] = p[2];
        /* |dx| <= sqrt(c Sigma'_xx) on the ellipse; a hair of slack keeps the
         * implication exact under FP64 rounding */
        v->rx[i] = ok ? sqrt(grow * p[6]) * (1.0 + 1e-9) + 1e-9 : -1.0;
        v->ry[i] = ok ? sqrt(grow * p[8]) * (1.0 + 1e-9) + 1e-9 : -1.0;
        v->at[i].a = p[3];
        v->at[i].b = p[4];
        v->at[i].c = p[5];
        v->at[i].depth = p[9];
        v->at[i].alpha = p[10];
        v->at[i].rgb[0] = p[11];
        v->at[i].rgb[1] = p[12];
        v->at[i].rgb[2] = p[13];
    }
    return 0;
}

static void free_view(oview* v) {
    free(v->mx); free(v->my); free(v->rx); free(v->ry); free(v->valid); free(v->at);
}

static int cand_cmp(const void* pa, const void* pb) {
    const ocand* a = (const ocand*)pa;
    const ocand* b = (const ocand*)pb;
    if (a->depth < b->depth) return -1;
    if (a->depth > b->depth) return 1;
    return (a->gid > b->gid) - (a->gid < b->gid);
}

typedef struct {
    ocand* cand;
    int64_t cap;
    oterm* terms;
    int64_t tcap;
} obuf;

static void buf_reserve(obuf* b, int64_t need) {
    if (need > b->cap) {
        int64_t c = b->cap ? b->cap : 256;
        while (c < need) c *= 2;
        b->cand = (ocand*)realloc(b->cand, sizeof(ocand) * c);
        b->terms = (oterm*)realloc(b->terms, sizeof(oterm) * c);
        b->cap = c;
        b->tcap = c;
    }
}

typedef struct {
    double A[3];
    double T;           /* transmittance after the last contributor */
    int64_t n_terms;    /* contributors */
    int64_t evaluated;  /* Gaussians inside the footprint box before the stop */
    int64_t violations; /* pairs met before the stop with w*alpha*k >= 1 */
    int flag;           /* straddle */
} opix;

static int near_rel(double v, double thr, double band) { return fabs(v - thr) <= band * fabs(thr); }

/* Composite one pixel of one view: the definition of Sec. 3 written out.  The
 * candidates are all Gaussians (list == NULL) or the nlist Gaussians of list (the tiled
 * traversal); the test, the order and the compositing are the same either way. */
static void pixel_composite_from(const oview* v, const or_opts* o, double px, double py, const int64_t* list,
                                 int64_t nlist, obuf* b, opix* r) {
    int64_t nc = 0;
    memset(r, 0, sizeof(*r));
    r->T = 1.0;
    const int64_t ncand = list ? nlist : v->n;
    for (int64_t q = 0; q < ncand; ++q) {
        const int64_t i = list ? list[q] : q;
        if (!v->valid[i]) continue;
        double dx = px - v->mx[i];
        if (fabs(dx) > v->rx[i]) continue;
        double dy = py - v->my[i];
        if (fabs(dy) > v->ry[i]) continue;
        const oattr* g = &v->at[i];
        double m = g->a * dx * dx + 2.0 * g->b * dx * dy + g->c * dy * dy;
        if (near_rel(m, o->cut2, o->band_cut)) r->flag = 1;
        if (m > o->cut2) continue;
        double k = exp(-0.5 * m);
        double raw = g->alpha * k;
        double rho = raw < o->rho_max ? raw : o->rho_max;
        if (near_rel(rho, o->alpha_min, o->band_alpha)) r->flag = 1;
        if (rho < o->alpha_min) continue;
        buf_reserve(b, nc + 1);
        b->cand[nc].depth = g->depth;
        b->cand[nc].gid = i;
        b->cand[nc].rho = rho;
        b->cand[nc].viol = raw >= 1.0;
        b->cand[nc].clamped = raw >= o->rho_max;
        nc++;
    }
    qsort(b->cand, (size_t)nc, sizeof(ocand), cand_cmp);
    double T = 1.0;
    double relT = 0.0; /* error bound of an FP32 evaluation of T relative to T */
    int64_t nt = 0;
    for (int64_t j = 0; j < nc; ++j) {
        const ocand* c = &b->cand[j];
        if (j > 0 && fabs(c->depth - b->cand[j - 1].depth) <= o->band_depth * c->depth) r->flag = 1;
        double Tn = T * (1.0 - c->rho);
        /* each factor 1 - rho carries the relative error of rho (band_alpha, none when
         * rho is the clamp constant) amplified by rho / (1 - rho), plus one rounding */
        relT += (c->clamped ? 0.0 : o->band_alpha * c->rho / (1.0 - c->rho)) + 1.2e-7;
        if (fabs(Tn - o->t_min) <= o->band_tmin * relT * o->t_min) r->flag = 1;
        r->evaluated++;
        r->violations += c->viol; /* validity (Def. "valid") over the pairs the traversal meets */
        if (Tn < o->t_min) break;
        const oattr* g = &v->at[c->gid];
        oterm* t = &b->terms[nt++];
        t->gid = c->gid;
        t->rho = c->rho;
        t->T = T;
        for (int ch = 0; ch < 3; ++ch) {
            t->c[ch] = g->rgb[ch];
            r->A[ch] += g->rgb[ch] * c->rho * T;
        }
        T = Tn;
    }
    r->T = T;
    r->n_terms = nt;
}

static void pixel_composite(const oview* v, const or_opts* o, double px, double py, obuf* b, opix* r) {
    pixel_composite_from(v, o, px, py, NULL, 0, b, r);
}

/* ---------------------------------------------------------------- render */

/* Render pixels of one camera.  pix: optional list of npix (x, y) pairs; when NULL
 * every pixel is rendered in row-major order.  w: per-Gaussian weights (NULL = 1),
 * giving the weighted render A_w of Sec. 3 "A pruned 3DGS scene" (rho' = w alpha k).
 * Outputs per rendered pixel: rgb[3], T (final transmittance), n_terms, flag.
 * counters[0] += violations (w alpha k >= 1), counters[1] += flagged pixels. */
int or_render(const or_scene* sc, const float* cam, const or_opts* o, const double* w, int64_t npix,
              const int32_t* pix, double* rgb, double* Tout, int32_t* nterms, uint8_t* flags,
              int64_t* counters) {
    oview v;
    ocam cm;
    if (build_view(sc, cam, o, w, &v, &cm)) return -1;
    int64_t total = pix ? npix : (int64_t)cm.W * cm.H;
    int64_t viol = 0, nflag = 0;
#pragma omp parallel reduction(+ : viol, nflag)
    {
        obuf b = {0};
#pragma omp for schedule(dynamic, 16)
        for (int64_t q = 0; q < total; ++q) {
            int px = pix ? pix[2 * q] : (int)(q % cm.W);
            int py = pix ? pix[2 * q + 1] : (int)(q / cm.W);
            opix r;
            pixel_composite(&v, o, px, py, &b, &r);
            for (int ch = 0; ch < 3; ++ch) rgb[3 * q + ch] = r.A[ch];
            if (Tout) Tout[q] = r.T;
            if (nterms) nterms[q] = (int32_t)r.n_terms;
            if (flags) flags[q] = (uint8_t)r.flag;
            viol += r.violations;
            nflag += r.flag;
        }
        free(b.cand);
        free(b.terms);
    }
    if (counters) {
        counters[0] += viol;
        counters[1] += nflag;
    }
    free_view(&v);
    return 0;
}

/* The same render by tiles (the rasteriser's traversal): every valid Gaussian is listed
 * in the tiles of tile_w x tile_h pixels its footprint box [mx - rx, mx + rx] x
 * [my - ry, my + ry] reaches, and each pixel composites only its tile's list.  Since the
 * box contains every pixel of the footprint test, this must equal or_render exactly
 * (reading: results do not depend on tiling). */
int or_render_tiled(const or_scene* sc, const float* cam, const or_opts* o, const double* w, int32_t tile_w,
                    int32_t tile_h, double* rgb, double* Tout, int32_t* nterms) {
    if (tile_w < 1 || tile_h < 1) return -1;
    oview v;
    ocam cm;
    if (build_view(sc, cam, o, w, &v, &cm)) return -1;
    const int tx_n = (cm.W + tile_w - 1) / tile_w, ty_n = (cm.H + tile_h - 1) / tile_h;
    const int64_t ntiles = (int64_t)tx_n * ty_n;
    int64_t* count = (int64_t*)calloc((size_t)ntiles + 1, sizeof(int64_t));
    if (!count) {
        free_view(&v);
        return -1;
    }
    /* two sweeps over the Gaussians: count per tile, then fill (index order within a tile) */
    int64_t* start = (int64_t*)calloc((size_t)ntiles + 1, sizeof(int64_t));
    for (int64_t i = 0; i < v.n; ++i) {
        if (!v.valid[i]) continue;
        int x0 = (int)floor((v.mx[i] - v.rx[i]) / tile_w), x1 = (int)floor((v.mx[i] + v.rx[i]) / tile_w);
        int y0 = (int)floor((v.my[i] - v.ry[i]) / tile_h), y1 = (int)floor((v.my[i] + v.ry[i]) / tile_h);
        if (x0 < 0) x0 = 0;
        if (y0 < 0) y0 = 0;
        if (x1 >= tx_n) x1 = tx_n - 1;
        if (y1 >= ty_n) y1 = ty_n - 1;
        for (int ty = y0; ty <= y1; ++ty)
            for (int tx = x0; tx <= x1; ++tx) count[(int64_t)ty * tx_n + tx]++;
    }
    for (int64_t t = 0; t < ntiles; ++t) start[t + 1] = start[t] + count[t];
    int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(start[ntiles] > 0 ? start[ntiles] : 1));
    memset(count, 0, sizeof(int64_t) * (size_t)ntiles);
    for (int64_t i = 0; i < v.n; ++i) {
        if (!v.valid[i]) continue;
        int x0 = (int)floor((v.mx[i] - v.rx[i]) / tile_w), x1 = (int)floor((v.mx[i] + v.rx[i]) / tile_w);
        int y0 = (int)floor((v.my[i] - v.ry[i]) / tile_h), y1 = (int)floor((v.my[i] + v.ry[i]) / tile_h);
        if (x0 < 0) x0 = 0;
        if (y0 < 0) y0 = 0;
        if (x1 >= tx_n) x1 = tx_n - 1;
        if (y1 >= ty_n) y1 = ty_n - 1;
        for (int ty = y0; ty <= y1; ++ty)
            for (int tx = x0; tx <= x1; ++tx) {
                const int64_t t = (int64_t)ty * tx_n + tx;
                list[start[t] + count[t]++] = i;
            }
    }
    const int64_t total = (int64_t)cm.W * cm.H;
#pragma omp parallel
    {
        obuf b = {0};
#pragma omp for schedule(dynamic, 16)
        for (int64_t q = 0; q < total; ++q) {
            const int px = (int)(q % cm.W), py = (int)(q / cm.W);
            const int64_t t = (int64_t)(py / tile_h) * tx_n + px / tile_w;
            opix r;
            pixel_composite_from(&v, o, px, py, list + start[t], start[t + 1] - start[t], &b, &r);
            for (int ch = 0; ch < 3; ++ch) rgb[3 * q + ch] = r.A[ch];
            if (Tout) Tout[q] = r.T;
            if (nterms) nterms[q] = (int32_t)r.n_terms;
        }
        free(b.cand);
        free(b.terms);
    }
    free(list);
    free(start);
    free(count);
    free_view(&v);
    return 0;
}

/* Contributor list of one pixel: gid, rho, T, colour for each term in order.
 * Returns the number of terms (at most cap are written); -1 on error. */
int64_t or_pixel_terms(const or_scene* sc, const float* cam, const or_opts* o, const double* w, int32_t px,
                       int32_t py, int64_t cap, int64_t* gid, double* rho, double* T, double* rgb, int32_t* flag) {
    oview v;
    ocam cm;
    if (build_view(sc, cam, o, w, &v, &cm)) return -1;
    obuf b = {0};
    opix r;
    pixel_composite(&v, o, px, py, &b, &r);
    for (int64_t j = 0; j < r.n_terms && j < cap; ++j) {
        gid[j] = b.terms[j].gid;
        rho[j] = b.terms[j].rho;
        T[j] = b.terms[j].T;
        for (int ch = 0; ch < 3; ++ch) rgb[3 * j + ch] = b.terms[j].c[ch];
    }
    if (flag) *flag = r.flag;
    int64_t nt = r.n_terms;
    free(b.cand);
    free(b.terms);
    free_view(&v);
    return nt;
}

/* ---------------------------------------------------------------- scoring */

static void atomic_max_nonneg(double* dst, double v) {
    /* non-negative doubles order like their bit patterns */
    uint64_t nv, ov;
    memcpy(&nv, &v, 8);
    uint64_t* p = (uint64_t*)dst;
    ov = __atomic_load_n(p, __ATOMIC_RELAXED);
    while (nv > ov) {
        if (__atomic_compare_exchange_n(p, &ov, nv, 0, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) break;
    }
}

static void atomic_add_double(double* dst, double v) {
    uint64_t* p = (uint64_t*)dst;
    uint64_t ov = __atomic_load_n(p, __ATOMIC_RELAXED), nv;
    for (;;) {
        double cur, nxt;
        memcpy(&cur, &ov, 8);
        nxt = cur + v;
        memcpy(&nv, &nxt, 8);
        if (__atomic_compare_exchange_n(p, &ov, nv, 0, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) break;
    }
}

/* the per-query, per-Gaussian term of the chosen score variant (Sec. 3,
 * "Additional variants"): L1 colour c rho T, L2 colour (c rho T)^2, no-colour rho T */
static double term_channel(const or_opts* o, const oterm* t, int ch) {
    double base = t->rho * t->T;
    if (o->variant == VAR_NC) return base;
    double a = t->c[ch] * base;
    return o->variant == VAR_L2 ? a * a : a;
}

static double term_pixel(const or_opts* o, const oterm* t) {
    if (o->variant == VAR_NC) return t->rho * t->T;
    double acc = 0.0;
    for (int ch = 0; ch < 3; ++ch) acc += o->obj_w[ch] * term_channel(o, t, ch);
    return acc;
}

/* Sensitivity of every Gaussian over every pixel-query of every camera (rows
 * [row0,row1) of each view; row1 < 0 means all rows).
 *   s[n]        sensitivity under the chosen resolution
 *   s_clean[n]  same, over unflagged queries only (pixel and channel resolutions)
 *   touched[n]  1 if the Gaussian contributes to a flagged query
 *   counters    [0] queries with A > 0, [1] flagged pixels, [2] evaluated pairs,
 *               [3] contributing pairs, [4] pixels
 *   totals      [0] sum of A over all queries (scene resolution), [1] S = sum s
 */
int or_score(const or_scene* sc, const float* cams, int32_t n_views, const or_opts* o, int32_t row0,
             int32_t row1, double* s, double* s_clean, uint8_t* touched, int64_t* counters, double* totals) {
    const int64_t n = sc->n;
    memset(s, 0, sizeof(double) * n);
    if (s_clean) memset(s_clean, 0, sizeof(double) * n);
    if (touched) memset(touched, 0, n);
    int64_t cnt[5] = {0, 0, 0, 0, 0};
    double sumA = 0.0;
    double* acc = NULL; /* scene resolution: sum over queries of the term */
    if (o->resolution == RES_SCENE) acc = (double*)calloc((size_t)n, sizeof(double));

    for (int32_t v = 0; v < n_views; ++v) {
        oview view;
        ocam cm;
        if (build_view(sc, cams + 20 * v, o, NULL, &view, &cm)) return -1;
        int r0 = row0 > 0 ? row0 : 0;
        int r1 = (row1 < 0 || row1 > cm.H) ? cm.H : row1;
        if (o->resolution == RES_TILE || o->resolution == RES_IMAGE) {
            /* aggregated queries: a unit is a tile (or the whole image) */
            int ts = o->resolution == RES_TILE ? o->tile : (cm.W > cm.H ? cm.W : cm.H);
            int tx = (cm.W + ts - 1) / ts, ty = (cm.H + ts - 1) / ts;
            int64_t units = (int64_t)tx * ty;
#pragma omp parallel
            {
                obuf b = {0};
                double* loc = (double*)calloc((size_t)n, sizeof(double));
                int64_t* list = (int64_t*)malloc(sizeof(int64_t) * 1024);
                int64_t lcap = 1024;
                int64_t c0 = 0, c1 = 0, c2 = 0, c3 = 0, c4 = 0;
#pragma omp for schedule(dynamic, 1)
                for (int64_t u = 0; u < units; ++u) {
                    int ux = (int)(u % tx), uy = (int)(u / tx);
                    int64_t nl = 0;
                    double Au = 0.0;
                    int uflag = 0;
                    for (int py = uy * ts; py < (uy + 1) * ts && py < cm.H; ++py) {
                        if (py < r0 || py >= r1) continue;
                        for (int px = ux * ts; px < (ux + 1) * ts && px < cm.W; ++px) {
                            opix r;
                            pixel_composite(&view, o, px, py, &b, &r);
                            c4++;
                            c2 += r.evaluated;
                            c3 += r.n_terms;
                            uflag |= r.flag;
                            c1 += r.flag;
                            for (int64_t j = 0; j < r.n_terms; ++j) {
                                double a = term_pixel(o, &b.terms[j]);
                                int64_t g = b.terms[j].gid;
                                if (a == 0.0) continue;
                                if (loc[g] == 0.0) {
                                    if (nl == lcap) {
                                        lcap *= 2;
                                        list = (int64_t*)realloc(list, sizeof(int64_t) * lcap);
                                    }
                                    list[nl++] = g;
                                }
                                loc[g] += a;
                                Au += a;
                            }
                        }
                    }
                    if (Au > 0.0) {
                        c0++;
                        for (int64_t j = 0; j < nl; ++j) {
                            int64_t g = list[j];
                            double imp = loc[g] / Au;
                            atomic_max_nonneg(&s[g], imp);
                            if (s_clean && !uflag) atomic_max_nonneg(&s_clean[g], imp);
                            if (touched && uflag) touched[g] = 1;
                        }
                    }
                    for (int64_t j = 0; j < nl; ++j) loc[list[j]] = 0.0;
                }
#pragma omp critical
                {
                    cnt[0] += c0; cnt[1] += c1; cnt[2] += c2; cnt[3] += c3; cnt[4] += c4;
                }
                free(loc);
                free(list);
                free(b.cand);
                free(b.terms);
            }
            free_view(&view);
            continue;
        }
#pragma omp parallel
        {
            obuf b = {0};
            int64_t c0 = 0, c1 = 0, c2 = 0, c3 = 0, c4 = 0;
            double lsum = 0.0;
#pragma omp for schedule(dynamic, 1)
            for (int py = r0; py < r1; ++py) {
                for (int px = 0; px < cm.W; ++px) {
                    opix r;
                    pixel_composite(&view, o, px, py, &b, &r);
                    c4++;
                    c2 += r.evaluated;
                    c3 += r.n_terms;
                    c1 += r.flag;
                    if (o->resolution == RES_CHANNEL) {
                        for (int ch = 0; ch < 3; ++ch) {
                            double Ac = 0.0;
                            for (int64_t j = 0; j < r.n_terms; ++j) Ac += term_channel(o, &b.terms[j], ch);
                            if (!(Ac > 0.0)) continue;
                            c0++;
                            for (int64_t j = 0; j < r.n_terms; ++j) {
                                double imp = term_channel(o, &b.terms[j], ch) / Ac;
                                int64_t g = b.terms[j].gid;
                                atomic_max_nonneg(&s[g], imp);
                                if (s_clean && !r.flag) atomic_max_nonneg(&s_clean[g], imp);
                                if (touched && r.flag) touched[g] = 1;
                            }
                        }
                        continue;
                    }
                    double A = 0.0;
                    for (int64_t j = 0; j < r.n_terms; ++j) A += term_pixel(o, &b.terms[j]);
                    if (!(A > 0.0)) continue; /* queries with A = 0 are discarded */
                    c0++;
                    if (o->resolution == RES_SCENE) {
                        lsum += A;
                        for (int64_t j = 0; j < r.n_terms; ++j)
                            atomic_add_double(&acc[b.terms[j].gid], term_pixel(o, &b.terms[j]));
                        if (touched && r.flag)
                            for (int64_t j = 0; j < r.n_terms; ++j) touched[b.terms[j].gid] = 1;
                        continue;
                    }
                    for (int64_t j = 0; j < r.n_terms; ++j) {
                        double imp = term_pixel(o, &b.terms[j]) / A;
                        int64_t g = b.terms[j].gid;
                        atomic_max_nonneg(&s[g], imp);
                        if (s_clean && !r.flag) atomic_max_nonneg(&s_clean[g], imp);
                        if (touched && r.flag) touched[g] = 1;
                    }
                }
            }
#pragma omp critical
            {
                cnt[0] += c0; cnt[1] += c1; cnt[2] += c2; cnt[3] += c3; cnt[4] += c4;
                sumA += lsum;
            }
            free(b.cand);
            free(b.terms);
        }
        free_view(&view);
    }
    if (o->resolution == RES_SCENE) {
        for (int64_t i = 0; i < n; ++i) s[i] = sumA > 0.0 ? acc[i] / sumA : 0.0;
        if (s_clean) memcpy(s_clean, s, sizeof(double) * n);
        free(acc);
    }
    double S = 0.0;
    for (int64_t i = 0; i < n; ++i) S += s[i];
    if (counters)
        for (int k = 0; k < 5; ++k) counters[k] = cnt[k];
    if (totals) {
        totals[0] = sumA;
        totals[1] = S;
    }
    return 0;
}

/* ---------------------------------------------------------------- sampling */

/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64
 * multiplies with the round keys bumped by the Weyl constants between rounds. */
void or_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* p = s / S (Algorithm 1, step 3).  Returns S. */
double or_probabilities(const double* s, int64_t n, double* p) {
    double S = 0.0;
    for (int64_t i = 0; i < n; ++i) S += s[i];
    for (int64_t i = 0; i < n; ++i) p[i] = S > 0.0 ? s[i] / S : 0.0;
    return S;
}

/* Integer CDF used for the draws: P_i = round(p_i * 2^56), C = inclusive prefix sum. */
void or_cdf(const double* p, int64_t n, uint64_t* C) {
    uint64_t run = 0;
    for (int64_t i = 0; i < n; ++i) {
        run += (uint64_t)llrint(ldexp(p[i], 56));
        C[i] = run;
    }
}

/* The t-th uniform draw in [0, C_total): a 64-bit Philox word x mapped by
 * floor(x * C_total / 2^64). */
uint64_t or_uniform(uint64_t seed, uint64_t t, uint64_t ctotal) {
    uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(t >> 32), 0u, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    or_philox4x32_10(ctr, key, r);
    uint64_t x = ((uint64_t)r[1] << 32) | r[0];
    return (uint64_t)(((unsigned __int128)x * ctotal) >> 64);
}

/* Algorithm 1, steps 4-5: m i.i.d. draws J_t with P(J = i) = p_i (inverse CDF:
 * the smallest i with C_i > u), counts n_i and weights w_i = n_i / (m p_i).
 * J[m] (may be NULL), counts[n], w[n]. Returns the number of distinct indices. */
int64_t or_sample(const double* p, int64_t n, int64_t m, uint64_t seed, int32_t* J, int32_t* counts, double* w) {
    uint64_t* C = (uint64_t*)malloc(sizeof(uint64_t) * (n > 0 ? n : 1));
    if (!C) return -1;
    or_cdf(p, n, C);
    uint64_t total = n > 0 ? C[n - 1] : 0;
    memset(counts, 0, sizeof(int32_t) * n);
    if (total == 0 || m <= 0) {
        free(C);
        for (int64_t i = 0; i < n; ++i) w[i] = 0.0;
        return 0;
    }
    for (int64_t t = 0; t < m; ++t) {
        uint64_t u = or_uniform(seed, (uint64_t)t, total);
        int64_t lo = 0, hi = n - 1; /* smallest index with C > u; C[n-1] > u always */
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (C[mid] > u)
                hi = mid;
            else
                lo = mid + 1;
        }
        if (J) J[t] = (int32_t)lo;
        counts[lo]++;
    }
    int64_t distinct = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (counts[i] > 0) {
            w[i] = (double)counts[i] / ((double)m * p[i]);
            distinct++;
        } else {
            w[i] = 0.0;
        }
    }
    free(C);
    return distinct;
}

/* Theorem 2 sample size: m >= 3 S / eps^2 * log(2 |Q'| / delta). */
double or_theorem2_m(double S, double eps, double delta, double nq) {
    return 3.0 * S / (eps * eps) * log(2.0 * nq / delta);
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- transfer */

/* Per-pixel quantities of the transfer argument (Sec. 3.3 and its appendix proof):
 * along the full-scene front-to-back order, A = sum c rho T, the relaxed objective
 * A_th = sum w c rho T (terms frozen at the full-scene transmittance), the true
 * reduced render A_w = sum w c rho T_w with T_w = prod (1 - w rho), and
 * gamma_q = max over retained Gaussians of |log T - log T_w|.  Intended for the
 * pure definitions (alpha_min = 0, rho_max = 1, t_min = 0); the footprint cut
 * applies.  out per pixel: A[3], A_th[3], A_w[3], gamma_q, min(1 - w rho). */
int or_transfer(const or_scene* sc, const float* cam, const or_opts* o, const double* w, double* out) {
    oview v;
    ocam cm;
    if (build_view(sc, cam, o, NULL, &v, &cm)) return -1;
    int64_t total = (int64_t)cm.W * cm.H;
#pragma omp parallel
    {
        obuf b = {0};
#pragma omp for schedule(dynamic, 16)
        for (int64_t q = 0; q < total; ++q) {
            double px = (double)(q % cm.W), py = (double)(q / cm.W);
            int64_t nc = 0;
            for (int64_t i = 0; i < v.n; ++i) {
                if (!v.valid[i]) continue;
                double dx = px - v.mx[i];
                if (fabs(dx) > v.rx[i]) continue;
                double dy = py - v.my[i];
                if (fabs(dy) > v.ry[i]) continue;
                const oattr* g = &v.at[i];
                double m = g->a * dx * dx + 2.0 * g->b * dx * dy + g->c * dy * dy;
                if (m > o->cut2) continue;
                double rho = g->alpha * exp(-0.5 * m);
                if (rho > o->rho_max) rho = o->rho_max;
                if (rho < o->alpha_min) continue;
                buf_reserve(&b, nc + 1);
                b.cand[nc].depth = g->depth;
                b.cand[nc].gid = i;
                b.cand[nc].rho = rho;
                nc++;
            }
            qsort(b.cand, (size_t)nc, sizeof(ocand), cand_cmp);
            double T = 1.0, Tw = 1.0, gam = 0.0, minf = 1.0;
            double A[3] = {0, 0, 0}, Ath[3] = {0, 0, 0}, Aw[3] = {0, 0, 0};
            for (int64_t j = 0; j < nc; ++j) {
                const ocand* c = &b.cand[j];
                const oattr* g = &v.at[c->gid];
                double wi = w[c->gid];
                for (int ch = 0; ch < 3; ++ch) {
                    double a = g->rgb[ch] * c->rho * T;
                    A[ch] += a;
                    Ath[ch] += wi * a;
                    Aw[ch] += wi * g->rgb[ch] * c->rho * Tw;
                }
                if (wi > 0.0) {
                    double d = fabs(log(T) - log(Tw));
                    if (d > gam) gam = d;
                }
                double f = 1.0 - wi * c->rho;
                if (f < minf) minf = f;
                T *= 1.0 - c->rho;
                Tw *= f;
            }
            double* r = out + 11 * q;
            for (int ch = 0; ch < 3; ++ch) {
                r[ch] = A[ch];
                r[3 + ch] = Ath[ch];
                r[6 + ch] = Aw[ch];
            }
            r[9] = gam;
            r[10] = minf;
        }
        free(b.cand);
        free(b.terms);
    }
    free_view(&v);
    return 0;
}

/* Per-pixel-resolution sensitivity restricted to a list of pixels of one view:
 * s[i] = max over the listed queries of a_i / A (Eq. sen over that subset); used to
 * obtain the exact s_i of chosen Gaussians by listing every pixel of their
 * footprints.  flags[p] marks straddling pixels; touched[i] = 1 if Gaussian i
 * contributes to a flagged pixel. */
int or_score_pixels(const or_scene* sc, const float* cam, const or_opts* o, int64_t npix, const int32_t* pix,
                    double* s, uint8_t* touched, uint8_t* flags) {
    oview v;
    ocam cm;
    if (build_view(sc, cam, o, NULL, &v, &cm)) return -1;
    memset(s, 0, sizeof(double) * sc->n);
    if (touched) memset(touched, 0, sc->n);
#pragma omp parallel
    {
        obuf b = {0};
#pragma omp for schedule(dynamic, 4)
        for (int64_t q = 0; q < npix; ++q) {
            opix r;
            pixel_composite(&v, o, pix[2 * q], pix[2 * q + 1], &b, &r);
            if (flags) flags[q] = (uint8_t)r.flag;
            double A = 0.0;
            for (int64_t j = 0; j < r.n_terms; ++j) A += term_pixel(o, &b.terms[j]);
            if (!(A > 0.0)) continue;
            for (int64_t j = 0; j < r.n_terms; ++j) {
                atomic_max_nonneg(&s[b.terms[j].gid], term_pixel(o, &b.terms[j]) / A);
                if (touched && r.flag) touched[b.terms[j].gid] = 1;
            }
        }
        free(b.cand);
        free(b.terms);
    }
    free_view(&v);
    return 0;
}

/* ---------------------------------------------------------------- surrogate MLP */
/* The surrogate sensitivity model (not in the paper): x (64 features, zero-padded)
 * -> 256 (GELU) -> 256 (GELU) -> 1, predicting log-sensitivity.  FP64 arithmetic with
 * the GPU's BF16 rounding points emulated: the inputs, W1, W2, the first hidden
 * activation and the two back-propagated pre-activation gradients are rounded to
 * BF16 (round to nearest even, through float32); everything else stays FP64.
 * Parameter block (doubles): W1[256][64], b1[256], W2[256][256], b2[256], w3[256], b3. */
#define MLP_IN 64
#define MLP_H 256
#define MLP_NPARAM (MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1)

int or_mlp_nparam(void) { return MLP_NPARAM; }

double or_bf16(double x) {
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    u &= 0xFFFF0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

static double gelu(double z) { return 0.5 * z * (1.0 + erf(z / sqrt(2.0))); }
static double gelu_d(double z) {
    const double pi = 3.14159265358979323846;
    return 0.5 * (1.0 + erf(z / sqrt(2.0))) + z * exp(-0.5 * z * z) / sqrt(2.0 * pi);
}

double or_gelu(double z) { return gelu(z); }
double or_gelu_d(double z) { return gelu_d(z); }

/* Forward of B rows.  emulate: 1 = BF16 rounding points, 0 = plain FP64 (for finite
 * differences).  y[B]; when z1/h1/z2/h2 are non-NULL they receive [B][256]. */
void or_mlp_forward(const double* P, const float* X, int64_t B, int emulate, double* y, double* z1o, double* h1o,
                    double* z2o, double* h2o) {
    const double *W1 = P, *b1 = W1 + MLP_H * MLP_IN, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H, *w3 = b2 + MLP_H,
                 *b3 = w3 + MLP_H;
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < B; ++r) {
        double x[MLP_IN], z1[MLP_H], h1[MLP_H], z2[MLP_H], h2[MLP_H];
        for (int k = 0; k < MLP_IN; ++k) x[k] = emulate ? or_bf16(X[r * MLP_IN + k]) : X[r * MLP_IN + k];
        for (int o = 0; o < MLP_H; ++o) {
            double acc = 0.0;
            for (int k = 0; k < MLP_IN; ++k) acc += (emulate ? or_bf16(W1[o * MLP_IN + k]) : W1[o * MLP_IN + k]) * x[k];
            z1[o] = acc + b1[o];
            h1[o] = emulate ? or_bf16(gelu(z1[o])) : gelu(z1[o]);
        }
        for (int o = 0; o < MLP_H; ++o) {
            double acc = 0.0;
            for (int k = 0; k < MLP_H; ++k) acc += (emulate ? or_bf16(W2[o * MLP_H + k]) : W2[o * MLP_H + k]) * h1[k];
            z2[o] = acc + b2[o];
            h2[o] = gelu(z2[o]);
        }
        double acc = b3[0];
        for (int k = 0; k < MLP_H; ++k) acc += w3[k] * h2[k];
        y[r] = acc;
        if (z1o)
            for (int k = 0; k < MLP_H; ++k) {
                z1o[r * MLP_H + k] = z1[k];
                h1o[r * MLP_H + k] = h1[k];
                z2o[r * MLP_H + k] = z2[k];
                h2o[r * MLP_H + k] = h2[k];
            }
    }
}

/* Loss mean_r (y_r - t_r)^2 and its gradient with respect to every parameter (G has the
 * parameter block's layout).  Returns the loss. */
double or_mlp_backward(const double* P, const float* X, const float* t, int64_t B, int emulate, double* G) {
    const double *W1 = P, *b1 = W1 + MLP_H * MLP_IN, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H, *w3 = b2 + MLP_H;
    (void)b1;
    (void)b2;
    double* y = (double*)malloc(sizeof(double) * B);
    double* z1 = (double*)malloc(sizeof(double) * B * MLP_H);
    double* h1 = (double*)malloc(sizeof(double) * B * MLP_H);
    double* z2 = (double*)malloc(sizeof(double) * B * MLP_H);
    double* h2 = (double*)malloc(sizeof(double) * B * MLP_H);
    or_mlp_forward(P, X, B, emulate, y, z1, h1, z2, h2);
    memset(G, 0, sizeof(double) * MLP_NPARAM);
    double *gW1 = G, *gb1 = gW1 + MLP_H * MLP_IN, *gW2 = gb1 + MLP_H, *gb2 = gW2 + MLP_H * MLP_H, *gw3 = gb2 + MLP_H,
           *gb3 = gw3 + MLP_H;
    double loss = 0.0;
    for (int64_t r = 0; r < B; ++r) {
        const double e = y[r] - t[r];
        loss += e * e / (double)B;
        const double dy = 2.0 * e / (double)B;
        double dz2[MLP_H], dz2b[MLP_H], dz1[MLP_H];
        gb3[0] += dy;
        for (int o = 0; o < MLP_H; ++o) {
            gw3[o] += dy * h2[r * MLP_H + o];
            dz2[o] = dy * w3[o] * gelu_d(z2[r * MLP_H + o]);
            dz2b[o] = emulate ? or_bf16(dz2[o]) : dz2[o];
            gb2[o] += dz2[o];
        }
        for (int o = 0; o < MLP_H; ++o)
            for (int k = 0; k < MLP_H; ++k) gW2[o * MLP_H + k] += dz2b[o] * h1[r * MLP_H + k];
        for (int k = 0; k < MLP_H; ++k) {
            double acc = 0.0;
            for (int o = 0; o < MLP_H; ++o) acc += dz2b[o] * (emulate ? or_bf16(W2[o * MLP_H + k]) : W2[o * MLP_H + k]);
            dz1[k] = acc * gelu_d(z1[r * MLP_H + k]);
            gb1[k] += dz1[k];
        }
        for (int o = 0; o < MLP_H; ++o) {
            const double d = emulate ? or_bf16(dz1[o]) : dz1[o];
            for (int k = 0; k < MLP_IN; ++k)
                gW1[o * MLP_IN + k] += d * (emulate ? or_bf16(X[r * MLP_IN + k]) : X[r * MLP_IN + k]);
        }
    }
    (void)W1;
    free(y);
    free(z1);
    free(h1);
    free(z2);
    free(h2);
    return loss;
}

/* One Adam step (Kingma & Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). */
void or_adam(double* p, const double* g, double* m, double* v, int64_t n, double lr, double b1, double b2, double eps,
             int64_t step) {
    const double c1 = 1.0 - pow(b1, (double)step), c2 = 1.0 - pow(b2, (double)step);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        p[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}

/* ---------------------------------------------------------------- render gradient */
/* Gradient of L = sum_pixels grad_rgb . C (so grad_rgb = dL/dC) of the (weighted)
 * render of one view with respect to the means, the SH coefficients and the opacity
 * logits (scales and rotations fixed), by the chain rule through Sec. 3's compositing
 * (back to front: dC/drho_i = c_i T_i - (sum_{j>i} c_j rho_j T_j) / (1 - rho_i)) and the
 * EWA projection.  Accumulates (+=) into g_means[3][N], g_sh[(d+1)^2][3][N],
 * g_logit[N].  FP64 throughout. */

static void sh_grad(int deg, const double* d, double G[16][3]) {
    const double pi = 3.14159265358979323846;
    double x = d[0], y = d[1], z = d[2];
    memset(G, 0, sizeof(double) * 48);
    if (deg < 1) return;
    double c1 = sqrt(3.0 / (4.0 * pi));
    G[1][1] = -c1;
    G[2][2] = c1;
    G[3][0] = -c1;
    if (deg < 2) return;
    double c2a = 0.5 * sqrt(15.0 / pi), c2b = 0.25 * sqrt(5.0 / pi), c2c = 0.25 * sqrt(15.0 / pi);
    G[4][0] = c2a * y; G[4][1] = c2a * x;
    G[5][1] = -c2a * z; G[5][2] = -c2a * y;
    G[6][0] = -2.0 * c2b * x; G[6][1] = -2.0 * c2b * y; G[6][2] = 4.0 * c2b * z;
    G[7][0] = -c2a * z; G[7][2] = -c2a * x;
    G[8][0] = 2.0 * c2c * x; G[8][1] = -2.0 * c2c * y;
    if (deg < 3) return;
    double c3a = 0.25 * sqrt(35.0 / (2.0 * pi)), c3b = 0.5 * sqrt(105.0 / pi);
    double c3c = 0.25 * sqrt(21.0 / (2.0 * pi)), c3d = 0.25 * sqrt(7.0 / pi), c3e = 0.25 * sqrt(105.0 / pi);
    double xx = x * x, yy = y * y, zz = z * z;
    G[9][0] = -c3a * 6.0 * x * y; G[9][1] = -c3a * (3.0 * xx - 3.0 * yy);
    G[10][0] = c3b * y * z; G[10][1] = c3b * x * z; G[10][2] = c3b * x * y;
    G[11][0] = c3c * 2.0 * x * y; G[11][1] = -c3c * (4.0 * zz - xx - 3.0 * yy); G[11][2] = -c3c * 8.0 * y * z;
    G[12][0] = -c3d * 6.0 * x * z; G[12][1] = -c3d * 6.0 * y * z; G[12][2] = c3d * (6.0 * zz - 3.0 * xx - 3.0 * yy);
    G[13][0] = -c3c * (4.0 * zz - 3.0 * xx - yy); G[13][1] = c3c * 2.0 * x * y; G[13][2] = -c3c * 8.0 * x * z;
    G[14][0] = c3e * 2.0 * x * z; G[14][1] = -c3e * 2.0 * y * z; G[14][2] = c3e * (xx - yy);
    G[15][0] = -c3a * (3.0 * xx - 3.0 * yy); G[15][1] = c3a * 6.0 * x * y;
}

typedef struct {
    int64_t gid;
    double rho, T, k, dx, dy;
    int clamped;
} obterm;

int or_render_backward(const or_scene* sc, const float* cam, const or_opts* o, const double* w, const double* grad_rgb,
                       double* g_means, double* g_sh, double* g_logit) {
    oview v;
    ocam cm;
    if (build_view(sc, cam, o, w, &v, &cm)) return -1;
    const int64_t n = sc->n;
    double* g2 = (double*)calloc((size_t)n * 9, sizeof(double)); /* mean x,y; Q xx,xy,yy; alpha; r,g,b */
    int64_t total = (int64_t)cm.W * cm.H;
#pragma omp parallel
    {
        ocand* cand = NULL;
        obterm* tl = NULL;
        int64_t cap = 0;
#pragma omp for schedule(dynamic, 16)
        for (int64_t q = 0; q < total; ++q) {
            double px = (double)(q % cm.W), py = (double)(q / cm.W);
            int64_t nc = 0;
            for (int64_t i = 0; i < n; ++i) {
                if (!v.valid[i]) continue;
                double dx = px - v.mx[i];
                if (fabs(dx) > v.rx[i]) continue;
                double dy = py - v.my[i];
                if (fabs(dy) > v.ry[i]) continue;
                const oattr* g = &v.at[i];
                double m = g->a * dx * dx + 2.0 * g->b * dx * dy + g->c * dy * dy;
                if (m > o->cut2) continue;
                double raw = g->alpha * exp(-0.5 * m);
                double rho = raw < o->rho_max ? raw : o->rho_max;
                if (rho < o->alpha_min) continue;
                if (nc == cap) {
                    cap = cap ? 2 * cap : 256;
                    cand = (ocand*)realloc(cand, sizeof(ocand) * cap);
                    tl = (obterm*)realloc(tl, sizeof(obterm) * cap);
                }
                cand[nc].depth = g->depth;
                cand[nc].gid = i;
                cand[nc].rho = rho;
                cand[nc].viol = raw >= o->rho_max; /* reused: clamped */
                nc++;
            }
            qsort(cand, (size_t)nc, sizeof(ocand), cand_cmp);
            double T = 1.0;
            int64_t nt = 0;
            for (int64_t j = 0; j < nc; ++j) {
                double Tn = T * (1.0 - cand[j].rho);
                if (Tn < o->t_min) break;
                const oattr* g = &v.at[cand[j].gid];
                obterm* t = &tl[nt++];
                t->gid = cand[j].gid;
                t->rho = cand[j].rho;
                t->T = T;
                t->clamped = cand[j].viol;
                t->dx = px - v.mx[t->gid];
                t->dy = py - v.my[t->gid];
                t->k = exp(-0.5 * (g->a * t->dx * t->dx + 2.0 * g->b * t->dx * t->dy + g->c * t->dy * t->dy));
                T = Tn;
            }
            const double* gr = grad_rgb + 3 * q;
            double S[3] = {0.0, 0.0, 0.0};
            for (int64_t j = nt - 1; j >= 0; --j) {
                const obterm* t = &tl[j];
                const oattr* g = &v.at[t->gid];
                double* G = g2 + 9 * t->gid;
                double drho = 0.0;
                for (int ch = 0; ch < 3; ++ch) {
                    atomic_add_double(&G[6 + ch], gr[ch] * t->rho * t->T);
                    drho += gr[ch] * (g->rgb[ch] * t->T - S[ch] / (1.0 - t->rho));
                }
                for (int ch = 0; ch < 3; ++ch) S[ch] += g->rgb[ch] * t->rho * t->T;
                if (t->clamped) continue;
                /* rho = alpha k, k = exp(-m/2), m = d^T Q d with d = pixel - mean */
                atomic_add_double(&G[5], drho * t->k);
                const double dm = -0.5 * t->rho * drho;
                atomic_add_double(&G[0], dm * -2.0 * (g->a * t->dx + g->b * t->dy));
                atomic_add_double(&G[1], dm * -2.0 * (g->b * t->dx + g->c * t->dy));
                atomic_add_double(&G[2], dm * t->dx * t->dx);
                atomic_add_double(&G[3], dm * 2.0 * t->dx * t->dy);
                atomic_add_double(&G[4], dm * t->dy * t->dy);
            }
        }
        free(cand);
        free(tl);
    }
    /* projection backward, per Gaussian */
    const int deg = sc->sh_degree, nk = (deg + 1) * (deg + 1);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        if (!v.valid[i]) continue;
        const double* G = g2 + 9 * i;
        double mu[3] = {sc->means[i], sc->means[n + i], sc->means[2 * n + i]};
        double pc[3];
        for (int r = 0; r < 3; ++r)
            pc[r] = cm.R[3 * r] * mu[0] + cm.R[3 * r + 1] * mu[1] + cm.R[3 * r + 2] * mu[2] + cm.t[r];
        double x = pc[0], y = pc[1], z = pc[2];
        double a = 1.0 / (1.0 + exp(-(double)sc->opacity_logits[i]));
        double wi = w ? w[i] : 1.0;
        g_logit[i] += G[5] * wi * a * (1.0 - a);
        /* covariance pieces */
        double s[3];
        for (int k = 0; k < 3; ++k) s[k] = exp((double)sc->log_scales[k * n + i]);
        double qw = sc->quats[i], qx = sc->quats[n + i], qy = sc->quats[2 * n + i], qz = sc->quats[3 * n + i];
        double qn = sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
        qw /= qn; qx /= qn; qy /= qn; qz /= qn;
        double Rq[9] = {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy),
                        2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx),
                        2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)};
        double Sig[9], tmp[9], Sc[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += Rq[3 * r + k] * s[k] * s[k] * Rq[3 * c + k];
                Sig[3 * r + c] = acc;
            }
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += cm.R[3 * r + k] * Sig[3 * k + c];
                tmp[3 * r + c] = acc;
            }
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += tmp[3 * r + k] * cm.R[3 * c + k];
                Sc[3 * r + c] = acc;
            }
        double limx = o->clamp_fov * 0.5 * cm.W / cm.fx, limy = o->clamp_fov * 0.5 * cm.H / cm.fy;
        double ux = x / z, uy = y / z;
        int fx_in = ux >= -limx && ux <= limx, fy_in = uy >= -limy && uy <= limy;
        if (ux < -limx) ux = -limx;
        if (ux > limx) ux = limx;
        if (uy < -limy) uy = -limy;
        if (uy > limy) uy = limy;
        double J[6] = {cm.fx / z, 0.0, -cm.fx * ux / z, 0.0, cm.fy / z, -cm.fy * uy / z};
        const oattr* ga = &v.at[i];
        double Q[4] = {ga->a, ga->b, ga->b, ga->c};
        double Gq[4] = {G[2], 0.5 * G[3], 0.5 * G[3], G[4]};
        double QG[4], H[4];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) QG[2 * r + c] = Q[2 * r] * Gq[c] + Q[2 * r + 1] * Gq[2 + c];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) H[2 * r + c] = -(QG[2 * r] * Q[c] + QG[2 * r + 1] * Q[2 + c]);
        /* dL/dJ = 2 H J Sc */
        double JS[6], dJ[6];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += J[3 * r + k] * Sc[3 * k + c];
                JS[3 * r + c] = acc;
            }
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) dJ[3 * r + c] = 2.0 * (H[2 * r] * JS[c] + H[2 * r + 1] * JS[3 + c]);
        double dx = 0.0, dy = 0.0, dz = 0.0;
        /* J00 = fx/z, J11 = fy/z, J02 = -fx u / z, J12 = -fy v / z (u, v clamped x/z, y/z) */
        dz += dJ[0] * (-cm.fx / (z * z)) + dJ[4] * (-cm.fy / (z * z));
        dz += dJ[2] * (cm.fx * ux / (z * z)) + dJ[5] * (cm.fy * uy / (z * z));
        if (fx_in) {
            dx += dJ[2] * (-cm.fx / z) / z;
            dz += dJ[2] * (-cm.fx / z) * (-x / (z * z));
        }
        if (fy_in) {
            dy += dJ[5] * (-cm.fy / z) / z;
            dz += dJ[5] * (-cm.fy / z) * (-y / (z * z));
        }
        /* projected mean */
        dx += G[0] * cm.fx / z;
        dz += G[0] * (-cm.fx * x / (z * z));
        dy += G[1] * cm.fy / z;
        dz += G[1] * (-cm.fy * y / (z * z));
        double gm[3];
        for (int k = 0; k < 3; ++k) gm[k] = cm.R[k] * dx + cm.R[3 + k] * dy + cm.R[6 + k] * dz;
        /* colour */
        double cpos[3];
        for (int k = 0; k < 3; ++k)
            cpos[k] = -(cm.R[k] * cm.t[0] + cm.R[3 + k] * cm.t[1] + cm.R[6 + k] * cm.t[2]);
        double dv[3] = {mu[0] - cpos[0], mu[1] - cpos[1], mu[2] - cpos[2]};
        double len = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
        double dh[3] = {dv[0] / len, dv[1] / len, dv[2] / len};
        double Y[16], GY[16][3];
        or_sh_basis(deg, dh, Y);
        sh_grad(deg, dh, GY);
        double gdir[3] = {0.0, 0.0, 0.0};
        for (int ch = 0; ch < 3; ++ch) {
            double acc = 0.5;
            for (int k = 0; k < nk; ++k) acc += (double)sc->sh[(int64_t)(3 * k + ch) * n + i] * Y[k];
            if (!(acc > 0.0)) continue; /* clamped colour */
            for (int k = 0; k < nk; ++k) {
                g_sh[(int64_t)(3 * k + ch) * n + i] += G[6 + ch] * Y[k];
                for (int c = 0; c < 3; ++c) gdir[c] += G[6 + ch] * (double)sc->sh[(int64_t)(3 * k + ch) * n + i] * GY[k][c];
            }
        }
        /* d dir / d mu = (I - dir dir^T) / len */
        double dd = gdir[0] * dh[0] + gdir[1] * dh[1] + gdir[2] * dh[2];
        for (int k = 0; k < 3; ++k) gm[k] += (gdir[k] - dd * dh[k]) / len;
        for (int k = 0; k < 3; ++k) g_means[k * n + i] += gm[k];
    }
    free(g2);
    free_view(&v);
    return 0;
}
