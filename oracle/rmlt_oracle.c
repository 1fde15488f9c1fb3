/*
 * CPU oracle for Regional Adaptive Metropolis Light Transport, restated in
 * primary sample space (PSS).  TEST INFRASTRUCTURE: only the tests, the smoke
 * check and the benchmark's CPU-baseline leg load it; the CUDA product path
 * shares no code with it.
 *
 * Plain binary64 C.  Readings of the paper that this file takes (where the
 * paper is silent, garbled or inconsistent) are marked "Reading:".
 *
 * parity pins: Philox against an independent library generator; closest hit
 * against brute force; the region update against a literal sequential
 * transcription of Alg. 1; the furnace and uniform-emitter closed forms; the
 * toy integrand's closed-form region masses (App. B); detailed balance of the
 * state-dependent acceptance on an enumerated torus.  See tests/test_oracle_*.
 */
#include "rmlt_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_DIM 256
#define OR_MAX_GRAD 62          /* dimensions of the gradient (2 + 5 x 12) */
#define OR_MALA_TAU_MAX 0.01    /* Langevin step bound: std <= 0.1 keeps the nearest-image density exact */
#define OR_WIN 1e-4            /* scene-relative window of the decision margin (10x the exclusion threshold) */
#define OR_INF (1.0 / 0.0)
#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Philox4x32-10: ten rounds of two 32x32->64 multiplies, key bumped by the  */
/* Weyl constants after each round (Salmon et al., SC'11, Sec. 3.2).         */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* A uniform in [0,1) from the top 24 bits of a word; exact in binary32/64. */
static double u24(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

/* Counter layout of the draws (the paper does not specify its RNG):
 *   mutation draws  ctr = {mut lo, mut hi, chain, call}, key = {seed lo, seed hi}
 *   bootstrap draws ctr = {sample lo, sample hi, 0xFFFFFFFF, 0x8000 + call}
 *   starting state  ctr = {chain g, 0, 0xFFFFFFFF, 0x7FFE} (its point u_g)   */
static void draw(uint64_t seed, uint64_t a, uint32_t b, uint32_t call, uint32_t out[4])
{
    uint32_t ctr[4] = {(uint32_t)a, (uint32_t)(a >> 32), b, call};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* binary32 quantities that decide integers (proposal offsets, sigma_k)     */
/* ------------------------------------------------------------------------ */
float or_exp2_f32(float t)
{
    /* t = n + r, n = rint(t), |r| <= 1/2; 2^r by its Taylor series
     * sum_i (ln 2)^i r^i / i!, i <= 7, Horner with fused multiply-adds. */
    float n = rintf(t);
    float r = t - n;
    float p = 1.525273365e-05f;
    p = fmaf(p, r, 1.540352969e-04f);
    p = fmaf(p, r, 1.333355787e-03f);
    p = fmaf(p, r, 9.618128650e-03f);
    p = fmaf(p, r, 5.550410971e-02f);
    p = fmaf(p, r, 2.402265072e-01f);
    p = fmaf(p, r, 6.931471825e-01f);
    p = fmaf(p, r, 1.0f);
    int32_t e = (int32_t)n + 127;
    uint32_t bits = (uint32_t)e << 23;
    float s;
    memcpy(&s, &bits, sizeof s);
    return p * s;
}

/* Kelemen et al. (2002) small step: offset magnitude sigma s2 (s1/s2)^xi,
 * i.e. log-uniform on [sigma s1, sigma s2]; scaled by 2^32 and rounded to an
 * integer number of PSS quanta.  sigma_s2 = fl(sigma_k * fl(s2 * 2^32)),
 * log2_ratio = fl(log2(s2 / s1)). */
int64_t or_kelemen_delta(uint32_t xmag, float sigma_s2, float log2_ratio)
{
    float xi = (float)(xmag >> 8) * 5.9604644775390625e-08f;
    float t = -(xi * log2_ratio);
    float m = sigma_s2 * or_exp2_f32(t);
    return (int64_t)llrintf(m);
}

/* erf^-1 by Newton's method on the library erf, from Winitzki's closed-form
 * estimate (a = 0.147); four steps reach binary64 accuracy on |x| < 1 - 2^-24 */
static double or_erfinv(double x)
{
    if (x <= -1.0) return -OR_INF;
    if (x >= 1.0) return OR_INF;
    if (x == 0.0) return 0.0;
    const double ln = log((1.0 - x) * (1.0 + x)), a = 0.147, t = 2.0 / (OR_PI * a) + 0.5 * ln;
    double y = copysign(sqrt(sqrt(t * t - ln / a) - t), x);
    for (int i = 0; i < 4; ++i) y -= (erf(y) - x) / (2.0 / sqrt(OR_PI) * exp(-y * y));
    return y;
}

/* Truncated-normal kernel (the paper's family, Sec. 5.2, with angles in
 * [-pi, pi] mapped to torus offsets in (-1/2, 1/2)): inverse-CDF sample of a
 * normal of standard deviation sigma truncated to (-1/2, 1/2). */
int64_t or_truncnorm_delta(uint32_t xmag, double sigma)
{
    const double u = u24(xmag);
    const double Z = erf(1.0 / (2.0 * sqrt(2.0) * sigma));
    /* u = 0 with Z rounded to 1 (sigma below ~0.06) would ask for erfinv(-1) */
    const double x = fmax(-1.0 + 0x1p-52, (2.0 * u - 1.0) * Z);
    const double d = sigma * sqrt(2.0) * or_erfinv(x);
    return (int64_t)llrint(d * 4294967296.0);
}

/* sigma_k = sqrt(exp(lambda_k)) = 2^(lambda_k / (2 ln 2))  (Alg. 1; Sec. 5.3) */
static float sigma_of_lambda(double lambda)
{
    return or_exp2_f32((float)(lambda * 0.7213475204444817));
}

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                      */
/* ------------------------------------------------------------------------ */
static void v_sub(const double a[3], const double b[3], double o[3]) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static double v_dot(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void v_cross(const double a[3], const double b[3], double o[3])
{
    double x = a[1] * b[2] - a[2] * b[1];
    double y = a[2] * b[0] - a[0] * b[2];
    double z = a[0] * b[1] - a[1] * b[0];
    o[0] = x; o[1] = y; o[2] = z;
}
static double v_len(const double a[3]) { return sqrt(v_dot(a, a)); }
static void v_norm(double a[3]) { double l = v_len(a); a[0] /= l; a[1] /= l; a[2] /= l; }
static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }

/* Luminance l(f) (Sec. 3.2 leaves l unspecified; Rec. 709 weights). */
static double luminance(const double f[3]) { return 0.2126 * f[0] + 0.7152 * f[1] + 0.0722 * f[2]; }

/* ------------------------------------------------------------------------ */
/* scene                                                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    double v0[3], e1[3], e2[3], n[3];
    double area2;                 /* |e1 x e2| */
    double h_u, h_v, h_w;         /* area2 / |edge opposite to each weight|  */
    int32_t mat;
} or_tri;

typedef struct {
    int32_t type;                 /* 0 Lambert, 1 GGX */
    double albedo[3], emission[3], rough;
    int32_t emissive, black;
} or_mat;

typedef struct {
    double lo[3], hi[3];
    int32_t left, right, first, count;   /* leaf iff count > 0 */
} or_node;

struct or_scene {
    int32_t toy;
    double toy_p[10];
    int32_t nt, nm;
    or_tri* tri;
    or_mat* mat;
    int32_t nl;
    int32_t* light;
    double* light_cdf;            /* cumulative area / total, last = 1 */
    double light_area;
    double cam_pos[3], cam_fwd[3], cam_right[3], cam_up[3], tan_half;
    double scale, eps;
    int32_t use_bvh, n_node;
    or_node* node;
    int32_t* idx;
};

static const double* g_cent;
static int g_axis;
static int cmp_idx(const void* a, const void* b)
{
    double ka = g_cent[3 * *(const int32_t*)a + g_axis], kb = g_cent[3 * *(const int32_t*)b + g_axis];
    if (ka < kb) return -1;
    if (ka > kb) return 1;
    return (*(const int32_t*)a) - (*(const int32_t*)b);
}

/* Median-split BVH, leaves of <= 4 triangles, boxes inflated by the margin
 * window so that every near-miss candidate is visited. */
static int32_t bvh_build(or_scene* s, double* cent, int32_t first, int32_t count)
{
    int32_t id = s->n_node++;
    or_node* nd = &s->node[id];
    double infl = OR_WIN * s->scale;
    for (int a = 0; a < 3; ++a) { nd->lo[a] = OR_INF; nd->hi[a] = -OR_INF; }
    double clo[3] = {OR_INF, OR_INF, OR_INF}, chi[3] = {-OR_INF, -OR_INF, -OR_INF};
    for (int32_t i = first; i < first + count; ++i) {
        const or_tri* t = &s->tri[s->idx[i]];
        for (int a = 0; a < 3; ++a) {
            double p0 = t->v0[a], p1 = t->v0[a] + t->e1[a], p2 = t->v0[a] + t->e2[a];
            nd->lo[a] = dmin(nd->lo[a], dmin(p0, dmin(p1, p2)));
            nd->hi[a] = dmax(nd->hi[a], dmax(p0, dmax(p1, p2)));
            double c = cent[3 * s->idx[i] + a];
            clo[a] = dmin(clo[a], c);
            chi[a] = dmax(chi[a], c);
        }
    }
    for (int a = 0; a < 3; ++a) { nd->lo[a] -= infl; nd->hi[a] += infl; }
    if (count <= 4) {
        nd->first = first; nd->count = count; nd->left = nd->right = -1;
        return id;
    }
    int axis = 0;
    for (int a = 1; a < 3; ++a) if (chi[a] - clo[a] > chi[axis] - clo[axis]) axis = a;
    g_cent = cent;
    g_axis = axis;
    qsort(s->idx + first, (size_t)count, sizeof(int32_t), cmp_idx);
    int32_t half = count / 2;
    nd->count = 0;
    nd->first = -1;
    int32_t l = bvh_build(s, cent, first, half);
    int32_t r = bvh_build(s, cent, first + half, count - half);
    s->node[id].left = l;
    s->node[id].right = r;
    return id;
}

or_scene* or_scene_create(int32_t nv, const float* verts, int32_t nt, const uint32_t* tris,
                          const uint32_t* mat_id, int32_t nm, const int32_t* mat_type,
                          const float* albedo, const float* emission, const float* roughness,
                          const float* camera, int32_t use_bvh)
{
    if (nt <= 0 || nv <= 0 || nm <= 0) return NULL;
    or_scene* s = (or_scene*)calloc(1, sizeof(or_scene));
    s->nt = nt; s->nm = nm;
    s->tri = (or_tri*)calloc((size_t)nt, sizeof(or_tri));
    s->mat = (or_mat*)calloc((size_t)nm, sizeof(or_mat));
    for (int32_t m = 0; m < nm; ++m) {
        or_mat* M = &s->mat[m];
        M->type = mat_type[m];
        for (int a = 0; a < 3; ++a) { M->albedo[a] = albedo[3 * m + a]; M->emission[a] = emission[3 * m + a]; }
        M->rough = roughness[m];
        M->emissive = (M->emission[0] > 0 || M->emission[1] > 0 || M->emission[2] > 0);
        M->black = (M->albedo[0] <= 0 && M->albedo[1] <= 0 && M->albedo[2] <= 0);
    }
    double lo[3] = {OR_INF, OR_INF, OR_INF}, hi[3] = {-OR_INF, -OR_INF, -OR_INF};
    for (int32_t i = 0; i < nv; ++i)
        for (int a = 0; a < 3; ++a) { lo[a] = dmin(lo[a], verts[3 * i + a]); hi[a] = dmax(hi[a], verts[3 * i + a]); }
    double diag[3];
    v_sub(hi, lo, diag);
    s->scale = v_len(diag);
    s->eps = 1e-4 * s->scale;
    s->nl = 0;
    for (int32_t i = 0; i < nt; ++i) {
        or_tri* T = &s->tri[i];
        double p[3][3];
        for (int j = 0; j < 3; ++j) {
            uint32_t vi = tris[3 * i + j];
            if ((int64_t)vi >= nv) { or_scene_destroy(s); return NULL; }
            for (int a = 0; a < 3; ++a) p[j][a] = verts[3 * vi + a];
        }
        if ((int64_t)mat_id[i] >= nm) { or_scene_destroy(s); return NULL; }
        for (int a = 0; a < 3; ++a) { T->v0[a] = p[0][a]; T->e1[a] = p[1][a] - p[0][a]; T->e2[a] = p[2][a] - p[0][a]; }
        double c[3];
        v_cross(T->e1, T->e2, c);
        T->area2 = v_len(c);
        if (T->area2 > 0) { T->n[0] = c[0] / T->area2; T->n[1] = c[1] / T->area2; T->n[2] = c[2] / T->area2; }
        double e3[3];
        v_sub(T->e2, T->e1, e3);
        T->h_u = T->area2 / dmax(v_len(T->e2), 1e-300);
        T->h_v = T->area2 / dmax(v_len(T->e1), 1e-300);
        T->h_w = T->area2 / dmax(v_len(e3), 1e-300);
        T->mat = (int32_t)mat_id[i];
        if (s->mat[T->mat].emissive && T->area2 > 0) s->nl++;
    }
    /* light list, sampled proportionally to area */
    s->light = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s->nl > 0 ? s->nl : 1));
    s->light_cdf = (double*)malloc(sizeof(double) * (size_t)(s->nl > 0 ? s->nl : 1));
    double acc = 0;
    int32_t li = 0;
    for (int32_t i = 0; i < nt; ++i) {
        if (s->mat[s->tri[i].mat].emissive && s->tri[i].area2 > 0) {
            acc += 0.5 * s->tri[i].area2;
            s->light[li] = i;
            s->light_cdf[li] = acc;
            li++;
        }
    }
    s->light_area = acc;
    for (int32_t j = 0; j < s->nl; ++j) s->light_cdf[j] /= acc;
    if (s->nl > 0) s->light_cdf[s->nl - 1] = 1.0;
    /* pinhole camera */
    double pos[3] = {camera[0], camera[1], camera[2]}, look[3] = {camera[3], camera[4], camera[5]};
    double up[3] = {camera[6], camera[7], camera[8]};
    memcpy(s->cam_pos, pos, sizeof pos);
    v_sub(look, pos, s->cam_fwd);
    v_norm(s->cam_fwd);
    v_cross(s->cam_fwd, up, s->cam_right);
    v_norm(s->cam_right);
    v_cross(s->cam_right, s->cam_fwd, s->cam_up);
    s->tan_half = tan((double)camera[9] * OR_PI / 360.0);
    s->use_bvh = use_bvh;
    s->idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)nt);
    for (int32_t i = 0; i < nt; ++i) s->idx[i] = i;
    if (use_bvh) {
        double* cent = (double*)malloc(sizeof(double) * 3 * (size_t)nt);
        for (int32_t i = 0; i < nt; ++i)
            for (int a = 0; a < 3; ++a)
                cent[3 * i + a] = s->tri[i].v0[a] + (s->tri[i].e1[a] + s->tri[i].e2[a]) / 3.0;
        s->node = (or_node*)calloc((size_t)(2 * nt + 1), sizeof(or_node));
        s->n_node = 0;
        bvh_build(s, cent, 0, nt);
        free(cent);
    }
    return s;
}

or_scene* or_scene_create_toy(const double* p)
{
    or_scene* s = (or_scene*)calloc(1, sizeof(or_scene));
    s->toy = 1;
    memcpy(s->toy_p, p, sizeof(double) * 10);
    s->scale = 1.0;
    return s;
}

void or_scene_destroy(or_scene* s)
{
    if (!s) return;
    free(s->tri); free(s->mat); free(s->light); free(s->light_cdf); free(s->node); free(s->idx);
    free(s);
}

double or_scene_scale(const or_scene* s) { return s->scale; }

/* Tests only, a planted mistake: choose the next-event light triangle
 * uniformly instead of in proportion to its area (the weight still assumes
 * the area density).  The furnace pins must catch it. */
void or_scene_plant_uniform_lights(or_scene* s)
{
    for (int32_t j = 0; j < s->nl; ++j) s->light_cdf[j] = (double)(j + 1) / (double)s->nl;
}

/* ------------------------------------------------------------------------ */
/* ray casting                                                               */
/* ------------------------------------------------------------------------ */
/* Moller-Trumbore: plane parameter t and barycentrics (u, v) of the hit.  */
static int tri_plane(const or_tri* T, const double o[3], const double d[3], double* t, double* u, double* v)
{
    double p[3], s[3], q[3];
    v_cross(d, T->e2, p);
    double det = v_dot(T->e1, p);
    if (det == 0.0 || !isfinite(det)) return 0;
    double inv = 1.0 / det;
    v_sub(o, T->v0, s);
    *u = v_dot(s, p) * inv;
    v_cross(s, T->e1, q);
    *v = v_dot(d, q) * inv;
    *t = v_dot(T->e2, q) * inv;
    return 1;
}

/* signed distance (world units) of the plane hit from the nearest edge line;
 * positive inside the triangle */
static double edge_dist(const or_tri* T, double u, double v)
{
    double w = 1.0 - u - v;
    return dmin(u * T->h_u, dmin(v * T->h_v, w * T->h_w));
}

static int box_hit(const or_node* n, const double o[3], const double d[3], double t0, double t1)
{
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (o[a] < n->lo[a] || o[a] > n->hi[a]) return 0;
            continue;
        }
        double inv = 1.0 / d[a];
        double ta = (n->lo[a] - o[a]) * inv, tb = (n->hi[a] - o[a]) * inv;
        if (ta > tb) { double x = ta; ta = tb; tb = x; }
        t0 = dmax(t0, ta);
        t1 = dmin(t1, tb);
        if (t0 > t1) return 0;
    }
    return 1;
}

typedef int (*tri_visit)(void* st, int32_t tri);   /* returns 1 to stop */

/* visit every triangle whose (inflated) box the segment (t0, t1) touches;
 * t1 may shrink during the walk through *t1p */
static void walk(const or_scene* s, const double o[3], const double d[3], double t0, double* t1p,
                 int brute, tri_visit fn, void* st, uint64_t* nodes, uint64_t* tests)
{
    if (brute || !s->use_bvh) {
        for (int32_t i = 0; i < s->nt; ++i) { if (tests) (*tests)++; if (fn(st, i)) return; }
        return;
    }
    int32_t stack[128];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const or_node* n = &s->node[stack[--sp]];
        if (nodes) (*nodes)++;
        if (!box_hit(n, o, d, t0, *t1p)) continue;
        if (n->count > 0) {
            for (int32_t i = n->first; i < n->first + n->count; ++i) {
                if (tests) (*tests)++;
                if (fn(st, s->idx[i])) return;
            }
        } else {
            stack[sp++] = n->left;
            stack[sp++] = n->right;
        }
    }
}

typedef struct {
    const or_scene* s;
    const double *o, *d;
    double tmin, t1;
    int32_t best;
    double bt, win, m;
    int pass;
} hit_state;

static int closest_visit(void* vs, int32_t i)
{
    hit_state* h = (hit_state*)vs;
    const or_tri* T = &h->s->tri[i];
    double t, u, v;
    if (!tri_plane(T, h->o, h->d, &t, &u, &v)) return 0;
    if (h->pass == 0) {
        if (u >= 0 && v >= 0 && u + v <= 1.0 && t > h->tmin && t < h->t1) {
            h->t1 = t;
            h->best = i;
            h->bt = t;
        }
        return 0;
    }
    /* pass 1: margin of the closest-hit decision */
    if (!(t > h->tmin) || t > h->t1) return 0;
    double ed = edge_dist(T, u, v);
    if (ed < -h->win) return 0;
    double sc = h->s->scale;
    if (i == h->best) h->m = dmin(h->m, ed / sc);
    else if (ed >= 0) h->m = dmin(h->m, fabs(t - h->bt) / sc);
    else h->m = dmin(h->m, -ed / sc);
    return 0;
}

int32_t or_closest_hit(const or_scene* s, const double o[3], const double d[3],
                       double tmin, double tmax, int32_t brute,
                       double* t_out, int32_t* tri_out, double* margin)
{
    hit_state h = {s, o, d, tmin, tmax, -1, tmax, OR_WIN * s->scale, OR_INF, 0};
    walk(s, o, d, tmin, &h.t1, brute, closest_visit, &h, NULL, NULL);
    if (margin) {
        h.pass = 1;
        h.t1 = (h.best >= 0 ? h.bt : tmax) + h.win;
        double t1 = h.t1;
        walk(s, o, d, tmin, &t1, brute, closest_visit, &h, NULL, NULL);
        *margin = dmin(*margin, h.m);
    }
    if (t_out) *t_out = h.bt;
    if (tri_out) *tri_out = h.best;
    return h.best >= 0;
}

typedef struct {
    const or_scene* s;
    const double *o, *d;
    double tmin, tmax, win, m;
    int occ, want_margin;
} any_state;

static int any_visit(void* vs, int32_t i)
{
    any_state* h = (any_state*)vs;
    const or_tri* T = &h->s->tri[i];
    double t, u, v;
    if (!tri_plane(T, h->o, h->d, &t, &u, &v)) return 0;
    if (u >= 0 && v >= 0 && u + v <= 1.0 && t > h->tmin && t < h->tmax) h->occ = 1;
    if (!h->want_margin) return h->occ;
    if (t <= h->tmin - h->win || t >= h->tmax + h->win) return 0;
    double ed = edge_dist(T, u, v);
    if (ed < -h->win) return 0;
    double sc = h->s->scale;
    h->m = dmin(h->m, fabs(ed) / sc);
    if (ed >= 0) h->m = dmin(h->m, dmin(fabs(t - h->tmax), fabs(t - h->tmin)) / sc);
    return 0;
}

int32_t or_any_hit(const or_scene* s, const double o[3], const double d[3],
                   double tmin, double tmax, int32_t brute, double* margin)
{
    any_state h = {s, o, d, tmin, tmax, OR_WIN * s->scale, OR_INF, 0, margin != NULL};
    double t1 = tmax + h.win;
    walk(s, o, d, tmin - h.win, &t1, brute, any_visit, &h, NULL, NULL);
    if (margin) *margin = dmin(*margin, h.m);
    return h.occ;
}

/* ------------------------------------------------------------------------ */
/* path map  u -> f(u): pinhole camera, d surface interactions, next-event  */
/* estimation at each, BSDF sampling in between (PT + NEE in PSS).          */
/* ------------------------------------------------------------------------ */
/* orthonormal frame around n (switches helper axis at |n_z| = 0.9) */
static void frame(const double n[3], double t[3], double b[3], double* margin)
{
    double az = fabs(n[2]);
    if (margin) *margin = dmin(*margin, fabs(az - 0.9));
    if (az < 0.9) { t[0] = -n[1]; t[1] = n[0]; t[2] = 0.0; }
    else { t[0] = 0.0; t[1] = -n[2]; t[2] = n[1]; }
    v_norm(t);
    v_cross(n, t, b);
}

static void to_world(const double l[3], const double t[3], const double b[3], const double n[3], double w[3])
{
    for (int a = 0; a < 3; ++a) w[a] = l[0] * t[a] + l[1] * b[a] + l[2] * n[a];
}

/* Smith G1 for GGX */
static double ggx_g1(double c, double a2)
{
    if (c <= 0) return 0.0;
    return 2.0 * c / (c + sqrt(a2 + (1.0 - a2) * c * c));
}

static void bsdf_eval(const or_mat* M, const double wo[3], const double wi[3], const double n[3], double fr[3])
{
    if (M->type == 0) {
        for (int a = 0; a < 3; ++a) fr[a] = M->albedo[a] / OR_PI;
        return;
    }
    double co = v_dot(n, wo), ci = v_dot(n, wi);
    if (co <= 0 || ci <= 0) { fr[0] = fr[1] = fr[2] = 0; return; }
    double h[3] = {wo[0] + wi[0], wo[1] + wi[1], wo[2] + wi[2]};
    v_norm(h);
    double ch = v_dot(n, h), a2 = M->rough * M->rough;
    double den = 1.0 + (a2 - 1.0) * ch * ch;
    double D = a2 / (OR_PI * den * den);
    double G = ggx_g1(co, a2) * ggx_g1(ci, a2);
    double c5 = pow(1.0 - v_dot(wi, h), 5.0);
    for (int a = 0; a < 3; ++a) {
        double F = M->albedo[a] + (1.0 - M->albedo[a]) * c5;
        fr[a] = F * D * G / (4.0 * co * ci);
    }
}

/* GGX continuation at an interaction: the half vector m is drawn with
 * density D(m) cos(theta_m) (Walter et al. 2007: tan^2 theta_m = a^2 bu /
 * (1 - bu), phi = 2 pi bv), wi is wo reflected about m, and the throughput
 * weight is f_r cos(theta_i) / pdf(wi) with pdf(wi) = D(m) cos(theta_m) /
 * (4 wo.m), i.e. F G (wo.m) / (cos(theta_o) cos(theta_m)).  Returns 0 when
 * the path ends (m faces away from wo, or wi is below the surface).  m_out
 * (optional) receives m.  `planted` (tests only): 1 drops the reflection
 * Jacobian 4 (wo.m) from the weight, a planted mistake the pins must catch. */
static int ggx_continue(const or_mat* M, const double wo[3], const double ns[3], const double ft[3],
                        const double fb[3], double bu, double bv, double wi[3], double w[3], double* mloc,
                        double* m_out, int planted)
{
    double a2 = M->rough * M->rough;
    double tan2 = a2 * bu / (1.0 - bu);
    double cm = 1.0 / sqrt(1.0 + tan2);
    double sm = sqrt(dmax(0.0, 1.0 - cm * cm));
    double phi = 2.0 * OR_PI * bv;
    double loc[3] = {sm * cos(phi), sm * sin(phi), cm}, mv[3];
    to_world(loc, ft, fb, ns, mv);
    if (m_out) for (int a = 0; a < 3; ++a) m_out[a] = mv[a];
    double dom = v_dot(wo, mv);
    w[0] = w[1] = w[2] = 0.0;
    if (dom <= 0) return 0;
    for (int a = 0; a < 3; ++a) wi[a] = 2.0 * dom * mv[a] - wo[a];
    double ci = v_dot(wi, ns), co = v_dot(wo, ns);
    if (mloc) *mloc = dmin(*mloc, 0.01 * dmin(dom, dmin(fabs(ci), co)));
    if (ci <= 0) return 0;
    double G = ggx_g1(co, a2) * ggx_g1(ci, a2);
    double c5 = pow(1.0 - dom, 5.0);
    for (int a = 0; a < 3; ++a) {
        double F = M->albedo[a] + (1.0 - M->albedo[a]) * c5;
        w[a] = planted == 1 ? F * G / (4.0 * co * cm) : F * G * dom / (co * cm);
    }
    return 1;
}

/* test entry points: one GGX lobe in the local frame n = z */
static void local_material(or_mat* M, double alpha, const double F0[3])
{
    memset(M, 0, sizeof *M);
    M->type = 1;
    M->rough = alpha;
    for (int a = 0; a < 3; ++a) M->albedo[a] = F0[a];
}

void or_ggx_sample_n(double alpha, const double F0[3], const double wo[3], int64_t n, const double* bu,
                     const double* bv, int32_t planted, double* wi, double* w, double* m)
{
    or_mat M;
    local_material(&M, alpha, F0);
    const double ns[3] = {0, 0, 1}, ft[3] = {1, 0, 0}, fb[3] = {0, 1, 0};
    for (int64_t i = 0; i < n; ++i)
        ggx_continue(&M, wo, ns, ft, fb, bu[i], bv[i], &wi[3 * i], &w[3 * i], NULL, &m[3 * i], planted);
}

void or_ggx_eval_n(double alpha, const double F0[3], const double wo[3], int64_t n, const double* wi, double* fr)
{
    or_mat M;
    local_material(&M, alpha, F0);
    const double ns[3] = {0, 0, 1};
    for (int64_t i = 0; i < n; ++i) bsdf_eval(&M, wo, &wi[3 * i], ns, &fr[3 * i]);
}

double or_ggx_g1(double cos_theta, double alpha) { return ggx_g1(cos_theta, alpha * alpha); }

static double toy_eval(const double* p, double u0, double u1)
{
    double f = p[0];
    if (u0 >= p[2] && u0 < p[3] && u1 >= p[4] && u1 < p[5]) f += p[1];
    double dx = u0 - p[7], dy = u1 - p[8];
    f += p[6] * exp(-(dx * dx + dy * dy) / (2.0 * p[9] * p[9]));
    return f;
}

/* A first-order bound on what binary32 evaluation of the same path can
 * change (the kernel traces in binary32, this oracle in binary64).  With the
 * unit roundoff u = 2^-24 and the scene diagonal S (a bound on coordinate
 * magnitudes), the walk carries
 *   ep  position error of the ray origin (world units),
 *   ed  angle error of the ray direction (radians),
 *   eT  relative error of the throughput,
 * and propagates them through each step with its condition number: a plane
 * hit at incidence cosine c spreads the ray's perpendicular error
 * ep + t ed (plus the Moller-Trumbore rounding, ~8 u S) by 1 / c; a direction
 * between points a distance l apart errs by (position error) / l; a cosine
 * factor c errs relatively by (angle error) / c; 1 / l^2 by 2 (position
 * error) / l; the GGX density changes with the half vector's angle by at most
 * (2 / alpha) per radian (|d ln D / d theta_m| <= 2 (1 - alpha^2) / alpha).
 *   dec   the smallest distance to a decision flip (a triangle edge, a near
 *         tie, a sign of a cosine, the light CDF, the shading frame's axis
 *         switch) in units of that quantity's error bound: below a few, a
 *         binary32 evaluation may take the other branch;
 *   ferr  the absolute error bound of each channel of f: every emitted or
 *         next-event term times the relative error bound of its factors. */
typedef struct {
    double dec;
    double ferr[3];
} or_err;

static double or_div(double a, double b) { return b > 1e-300 ? a / b : OR_INF; }

/* path map with the geometric decision margin (margin, scene-relative) and
 * the binary32 error model (E); either may be NULL */
static int32_t path_eval_impl(const or_scene* s, int32_t width, int32_t height, int32_t max_depth,
                              const uint32_t* q, double f[3], double* margin, or_err* E, uint64_t counts[3])
{
    double mloc = OR_INF;
    double* mp = margin ? &mloc : NULL;
    const double u = 0x1p-24, S = s->scale;
    double ep = 4.0 * u * S, ed = 8.0 * u, eT = 0.0;   /* camera ray: position and normalize() rounding */
    if (E) {
        E->dec = OR_INF;
        E->ferr[0] = E->ferr[1] = E->ferr[2] = 0.0;
    }
    f[0] = f[1] = f[2] = 0.0;
    if (s->toy) {
        double v = toy_eval(s->toy_p, u24(q[0]), u24(q[1]));
        f[0] = f[1] = f[2] = v;
        if (margin) *margin = OR_INF;
        if (E) E->ferr[0] = E->ferr[1] = E->ferr[2] = 16.0 * u * fabs(v);
        return 1;
    }
    double L[3] = {0, 0, 0}, T[3] = {1, 1, 1};
    double aspect = (double)width / (double)height;
    double sx = (2.0 * u24(q[0]) - 1.0) * s->tan_half * aspect;
    double sy = (1.0 - 2.0 * u24(q[1])) * s->tan_half;
    double o[3], d[3];
    for (int a = 0; a < 3; ++a) {
        o[a] = s->cam_pos[a];
        d[a] = s->cam_fwd[a] + sx * s->cam_right[a] + sy * s->cam_up[a];
    }
    v_norm(d);
    for (int b = 0; b < max_depth; ++b) {
        double t, mh = OR_INF;
        int32_t ti;
        if (counts) counts[0]++;
        int hit = or_closest_hit(s, o, d, 0.0, OR_INF, 0, &t, &ti, (mp || E) ? &mh : NULL);
        if (mp) mloc = dmin(mloc, mh);
        if (!hit) {
            if (E) E->dec = dmin(E->dec, or_div(mh * S, ep + 8.0 * u * S));
            break;
        }
        const or_tri* Tr = &s->tri[ti];
        const or_mat* M = &s->mat[Tr->mat];
        double x[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
        double cosi = -v_dot(Tr->n, d);
        mloc = dmin(mloc, fabs(cosi));
        /* a short segment (a corner) amplifies the binary32 hit-point error
         * like 2^-24 scale / t: below t / scale = 6e-4 it counts as
         * near-degenerate */
        mloc = dmin(mloc, t / s->scale / 60.0);
        /* the hit point's error: the ray's perpendicular error at t spread
         * over the plane by 1 / |cos|; the edge and tie margins against it */
        const double eh = or_div(ep + t * ed + 8.0 * u * S, fabs(cosi));
        if (E) {
            E->dec = dmin(E->dec, or_div(mh * S, eh));
            E->dec = dmin(E->dec, or_div(fabs(cosi), ed + 4.0 * u));
        }
        double ns[3];
        for (int a = 0; a < 3; ++a) ns[a] = cosi > 0 ? Tr->n[a] : -Tr->n[a];
        if (b == 0 && M->emissive && cosi > 0)
            for (int a = 0; a < 3; ++a) {
                L[a] += T[a] * M->emission[a];
                if (E) E->ferr[a] += fabs(T[a] * M->emission[a]) * (eT + 2.0 * u);
            }
        if (M->black) break;
        double wo[3] = {-d[0], -d[1], -d[2]};
        /* next-event estimation: light triangle by area, uniform point on it */
        if (s->nl > 0) {
            double ls = u24(q[2 + 5 * b]), lu = u24(q[3 + 5 * b]), lv = u24(q[4 + 5 * b]);
            int32_t lo = 0, hi = s->nl - 1;
            while (lo < hi) { int32_t mid = (lo + hi) / 2; if (s->light_cdf[mid] > ls) hi = mid; else lo = mid + 1; }
            mloc = dmin(mloc, s->light_cdf[lo] - ls);
            if (lo > 0) mloc = dmin(mloc, ls - s->light_cdf[lo - 1]);
            if (E && s->nl > 1) {   /* the kernel's CDF is rounded to binary32 */
                E->dec = dmin(E->dec, or_div(s->light_cdf[lo] - ls, u));
                if (lo > 0) E->dec = dmin(E->dec, or_div(ls - s->light_cdf[lo - 1], u));
            }
            const or_tri* LT = &s->tri[s->light[lo]];
            const or_mat* LM = &s->mat[LT->mat];
            double su = sqrt(lu), b1 = su * (1.0 - lv), b2 = su * lv;
            double p[3], wi[3];
            for (int a = 0; a < 3; ++a) p[a] = LT->v0[a] + b1 * LT->e1[a] + b2 * LT->e2[a];
            v_sub(p, x, wi);
            double dist2 = v_dot(wi, wi), dist = sqrt(dist2);
            for (int a = 0; a < 3; ++a) wi[a] /= dist;
            double cx = v_dot(ns, wi), cl = -v_dot(LT->n, wi);
            /* the light direction's error: both end points over their distance */
            const double epl = eh + 4.0 * u * S, ew = or_div(epl, dist) + 4.0 * u;
            if (E) {
                E->dec = dmin(E->dec, or_div(fabs(cx), ew + 4.0 * u));
                E->dec = dmin(E->dec, or_div(fabs(cl), ew + 4.0 * u));
            }
            if (cx > 0 && cl > 0) {
                /* a grazing cosine makes the contribution ill-conditioned in
                 * binary32 (relative error ~ 2^-24 / cos): below 1e-3 it
                 * counts as a near-degenerate decision */
                mloc = dmin(mloc, 0.01 * dmin(cx, cl));
                /* and so does a light point close to x relative to the scene:
                 * the binary32 geometry term's relative error grows like
                 * 2^-24 scale / (dist cos); below dist cos / scale = 6e-4 it
                 * counts as near-degenerate */
                mloc = dmin(mloc, dist * dmin(cx, cl) / s->scale / 60.0);
                double xo[3], sd[3];
                for (int a = 0; a < 3; ++a) xo[a] = x[a] + s->eps * ns[a];
                v_sub(p, xo, sd);
                double sdist = v_len(sd);
                if (E) E->dec = dmin(E->dec, or_div(fabs(sdist - 2.0 * s->eps), epl));
                if (sdist > 2.0 * s->eps) {
                    for (int a = 0; a < 3; ++a) sd[a] /= sdist;
                    if (counts) counts[0]++;
                    double mv = OR_INF;
                    int occ = or_any_hit(s, xo, sd, 0.0, sdist - s->eps, 0, (mp || E) ? &mv : NULL);
                    if (mp) mloc = dmin(mloc, mv);
                    /* an occluder's edge against the shadow ray's error along its length */
                    if (E) E->dec = dmin(E->dec, or_div(mv * S, epl + sdist * ew + 8.0 * u * S));
                    if (!occ) {
                        double fr[3];
                        bsdf_eval(M, wo, wi, ns, fr);
                        double g = cx * cl / dist2 * s->light_area;
                        /* relative error of T fr Le g: the cosines, 1 / dist^2,
                         * the BSDF (GGX: its density's slope times the half
                         * vector's angle error) and a few roundings */
                        double eP = eT + or_div(ew + 4.0 * u, cx) + or_div(ew + 4.0 * u, cl) +
                                    2.0 * or_div(epl, dist) + 16.0 * u;
                        if (M->type == 1) {
                            const double co = v_dot(wo, ns);
                            eP += (2.0 / M->rough + or_div(2.0, co) + or_div(2.0, cx)) * (ed + ew) + 16.0 * u;
                        }
                        for (int a = 0; a < 3; ++a) {
                            const double c = T[a] * fr[a] * LM->emission[a] * g;
                            L[a] += c;
                            if (E) E->ferr[a] += fabs(c) * eP;
                        }
                    }
                }
            }
        }
        if (b == max_depth - 1) break;
        /* continue by sampling the BSDF with the bounce's last two dimensions */
        double bu = u24(q[5 + 5 * b]), bv = u24(q[6 + 5 * b]);
        double ft[3], fb[3], wi[3], loc[3];
        frame(ns, ft, fb, mp);
        if (E) E->dec = dmin(E->dec, or_div(fabs(fabs(ns[2]) - 0.9), 4.0 * u));
        double phi = 2.0 * OR_PI * bv;
        double ed_next;
        if (M->type == 0) {
            double r = sqrt(bu);
            loc[0] = r * cos(phi); loc[1] = r * sin(phi); loc[2] = sqrt(dmax(0.0, 1.0 - bu));
            mloc = dmin(mloc, 0.01 * loc[2]);
            to_world(loc, ft, fb, ns, wi);
            for (int a = 0; a < 3; ++a) T[a] *= M->albedo[a];
            /* a cosine sample depends on the normal only (and sqrt(1 - bu)
             * near the horizon); the throughput gains one rounding */
            ed_next = 16.0 * u + or_div(u, loc[2]);
            eT += u;
        } else {
            double w[3], m[3];
            const double co = v_dot(wo, ns);
            const int cont = ggx_continue(M, wo, ns, ft, fb, bu, bv, wi, w, &mloc, m, 0);
            const double dom = v_dot(wo, m);
            /* wi reflects wo about m: its angle error is wo's plus twice m's */
            ed_next = ed + 32.0 * u;
            if (E) {
                E->dec = dmin(E->dec, or_div(fabs(dom), ed + 8.0 * u));
                if (dom > 0) E->dec = dmin(E->dec, or_div(fabs(v_dot(wi, ns)), ed_next + 4.0 * u));
            }
            if (!cont) break;
            const double ci = v_dot(wi, ns);
            eT += or_div(ed + 8.0 * u, dom) + or_div(ed + 4.0 * u, co) + or_div(ed_next + 4.0 * u, ci) + 16.0 * u;
            for (int a = 0; a < 3; ++a) T[a] *= w[a];
        }
        for (int a = 0; a < 3; ++a) { o[a] = x[a] + s->eps * ns[a]; d[a] = wi[a]; }
        ep = eh + 2.0 * u * S;
        ed = ed_next;
    }
    int ok = isfinite(L[0]) && isfinite(L[1]) && isfinite(L[2]);
    if (ok) { f[0] = L[0]; f[1] = L[1]; f[2] = L[2]; }
    if (margin) *margin = mloc;
    return ok;
}

int32_t or_path_eval(const or_scene* s, int32_t width, int32_t height, int32_t max_depth,
                     const uint32_t* q, double f[3], double* margin, uint64_t counts[3])
{
    return path_eval_impl(s, width, height, max_depth, q, f, margin, NULL, counts);
}

int32_t or_path_eval_err(const or_scene* s, int32_t width, int32_t height, int32_t max_depth,
                         const uint32_t* q, double f[3], double* dec, double ferr[3], uint64_t counts[3])
{
    or_err E;
    int32_t ok = path_eval_impl(s, width, height, max_depth, q, f, NULL, &E, counts);
    if (dec) *dec = E.dec;
    if (ferr) for (int a = 0; a < 3; ++a) ferr[a] = E.ferr[a];
    return ok;
}

/* ------------------------------------------------------------------------ */
/* gradient of log pi(u) by forward-mode differentiation: every continuous  */
/* quantity of the path map carries its derivative with respect to all D    */
/* primary-sample coordinates (dual numbers); the discrete choices (hit      */
/* triangle, light triangle, visibility, branch taken) come from the primal  */
/* walk and are held fixed, so this is the gradient of the smooth piece of   */
/* f that contains u.                                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    double v;
    double g[OR_MAX_GRAD];
} dn;

typedef struct {
    dn c[3];
} dv3;

static int g_nd; /* dimensions carried by the dual numbers of the current call */

static dn dn_c(double v)
{
    dn r;
    r.v = v;
    memset(r.g, 0, sizeof(double) * (size_t)g_nd);
    return r;
}
static dn dn_var(double v, int j)
{
    dn r = dn_c(v);
    r.g[j] = 1.0;
    return r;
}
static dn dn_add(dn a, dn b) { for (int j = 0; j < g_nd; ++j) a.g[j] += b.g[j]; a.v += b.v; return a; }
static dn dn_sub(dn a, dn b) { for (int j = 0; j < g_nd; ++j) a.g[j] -= b.g[j]; a.v -= b.v; return a; }
static dn dn_scale(dn a, double s) { for (int j = 0; j < g_nd; ++j) a.g[j] *= s; a.v *= s; return a; }
static dn dn_addc(dn a, double c) { a.v += c; return a; }
static dn dn_mul(dn a, dn b)
{
    dn r;
    r.v = a.v * b.v;
    for (int j = 0; j < g_nd; ++j) r.g[j] = a.g[j] * b.v + a.v * b.g[j];
    return r;
}
static dn dn_div(dn a, dn b)
{
    dn r;
    r.v = a.v / b.v;
    for (int j = 0; j < g_nd; ++j) r.g[j] = (a.g[j] * b.v - a.v * b.g[j]) / (b.v * b.v);
    return r;
}
/* f(a) with f'(a.v) = df */
static dn dn_apply(dn a, double fv, double df)
{
    a.v = fv;
    for (int j = 0; j < g_nd; ++j) a.g[j] *= df;
    return a;
}
static dn dn_sqrt(dn a) { double r = sqrt(a.v); return dn_apply(a, r, r > 0 ? 0.5 / r : 0.0); }
static dn dn_cos(dn a) { return dn_apply(a, cos(a.v), -sin(a.v)); }
static dn dn_sin(dn a) { return dn_apply(a, sin(a.v), cos(a.v)); }
static dn dn_exp(dn a) { double e = exp(a.v); return dn_apply(a, e, e); }

static dv3 dv_c(const double a[3]) { dv3 r; for (int k = 0; k < 3; ++k) r.c[k] = dn_c(a[k]); return r; }
static dv3 dv_add(dv3 a, dv3 b) { for (int k = 0; k < 3; ++k) a.c[k] = dn_add(a.c[k], b.c[k]); return a; }
static dv3 dv_sub(dv3 a, dv3 b) { for (int k = 0; k < 3; ++k) a.c[k] = dn_sub(a.c[k], b.c[k]); return a; }
static dv3 dv_smul(dv3 a, dn s) { for (int k = 0; k < 3; ++k) a.c[k] = dn_mul(a.c[k], s); return a; }
/* constant vector times a dual scalar */
static dv3 dv_cs(const double a[3], dn s) { dv3 r; for (int k = 0; k < 3; ++k) r.c[k] = dn_scale(s, a[k]); return r; }
static dn dv_dotc(dv3 a, const double b[3])
{
    dn r = dn_scale(a.c[0], b[0]);
    r = dn_add(r, dn_scale(a.c[1], b[1]));
    return dn_add(r, dn_scale(a.c[2], b[2]));
}
static dn dv_dot(dv3 a, dv3 b)
{
    dn r = dn_mul(a.c[0], b.c[0]);
    r = dn_add(r, dn_mul(a.c[1], b.c[1]));
    return dn_add(r, dn_mul(a.c[2], b.c[2]));
}
static void dv_val(dv3 a, double o[3]) { for (int k = 0; k < 3; ++k) o[k] = a.c[k].v; }

int32_t or_path_grad(const or_scene* s, int32_t width, int32_t height, int32_t max_depth, const uint32_t* q,
                     double f[3], double* grad)
{
    const int D = s->toy ? 2 : 2 + 5 * max_depth;
    if (D > OR_MAX_GRAD) return -1;
    g_nd = D;
    memset(grad, 0, sizeof(double) * (size_t)D);
    f[0] = f[1] = f[2] = 0.0;
    dn u[OR_MAX_GRAD];
    for (int j = 0; j < D; ++j) u[j] = dn_var(u24(q[j]), j);
    if (s->toy) {
        const double* p = s->toy_p;
        double u0 = u[0].v, u1 = u[1].v;
        dn fv = dn_c(p[0] + ((u0 >= p[2] && u0 < p[3] && u1 >= p[4] && u1 < p[5]) ? p[1] : 0.0));
        dn dx = dn_addc(u[0], -p[7]), dy = dn_addc(u[1], -p[8]);
        dn r2 = dn_add(dn_mul(dx, dx), dn_mul(dy, dy));
        fv = dn_add(fv, dn_scale(dn_exp(dn_scale(r2, -1.0 / (2.0 * p[9] * p[9]))), p[6]));
        f[0] = f[1] = f[2] = fv.v;
        for (int j = 0; j < D; ++j) grad[j] = fv.g[j] / fv.v;
        return 1;
    }
    dv3 L = dv_c((double[3]){0, 0, 0});
    double T[3] = {1, 1, 1};
    const double aspect = (double)width / (double)height;
    dn sx = dn_scale(dn_addc(dn_scale(u[0], 2.0), -1.0), s->tan_half * aspect);
    dn sy = dn_scale(dn_addc(dn_scale(u[1], -2.0), 1.0), s->tan_half);
    dv3 o = dv_c(s->cam_pos);
    dv3 d = dv_add(dv_add(dv_c(s->cam_fwd), dv_cs(s->cam_right, sx)), dv_cs(s->cam_up, sy));
    dn dl = dn_sqrt(dv_dot(d, d));
    for (int k = 0; k < 3; ++k) d.c[k] = dn_div(d.c[k], dl);
    for (int b = 0; b < max_depth; ++b) {
        double ov[3], dvv[3], t;
        int32_t ti;
        dv_val(o, ov);
        dv_val(d, dvv);
        if (!or_closest_hit(s, ov, dvv, 0.0, OR_INF, 0, &t, &ti, NULL)) break;
        const or_tri* Tr = &s->tri[ti];
        const or_mat* M = &s->mat[Tr->mat];
        /* the hit on the triangle's plane: t = (v0 - o).n / d.n */
        dn tn = dn_div(dv_dotc(dv_sub(dv_c(Tr->v0), o), Tr->n), dv_dotc(d, Tr->n));
        dv3 x = dv_add(o, dv_smul(d, tn));
        double cosi = -v_dot(Tr->n, dvv);
        double ns[3];
        for (int a = 0; a < 3; ++a) ns[a] = cosi > 0 ? Tr->n[a] : -Tr->n[a];
        if (b == 0 && M->emissive && cosi > 0)
            for (int a = 0; a < 3; ++a) L.c[a] = dn_addc(L.c[a], T[a] * M->emission[a]);
        if (M->black) break;
        if (s->nl > 0) {
            dn lu = u[3 + 5 * b], lv = u[4 + 5 * b];
            double ls = u[2 + 5 * b].v;
            int32_t lo = 0, hi = s->nl - 1;
            while (lo < hi) { int32_t mid = (lo + hi) / 2; if (s->light_cdf[mid] > ls) hi = mid; else lo = mid + 1; }
            const or_tri* LT = &s->tri[s->light[lo]];
            const or_mat* LM = &s->mat[LT->mat];
            dn su = dn_sqrt(lu);
            dn b1 = dn_mul(su, dn_addc(dn_scale(lv, -1.0), 1.0)), b2 = dn_mul(su, lv);
            dv3 p = dv_add(dv_add(dv_c(LT->v0), dv_cs(LT->e1, b1)), dv_cs(LT->e2, b2));
            dv3 wi = dv_sub(p, x);
            dn dist2 = dv_dot(wi, wi), dist = dn_sqrt(dist2);
            for (int k = 0; k < 3; ++k) wi.c[k] = dn_div(wi.c[k], dist);
            dn cx = dv_dotc(wi, ns), cl = dn_scale(dv_dotc(wi, LT->n), -1.0);
            if (cx.v > 0 && cl.v > 0) {
                double xv[3], pv[3], xo[3], sd[3];
                dv_val(x, xv);
                dv_val(p, pv);
                for (int a = 0; a < 3; ++a) xo[a] = xv[a] + s->eps * ns[a];
                v_sub(pv, xo, sd);
                double sdist = v_len(sd);
                if (sdist > 2.0 * s->eps) {
                    for (int a = 0; a < 3; ++a) sd[a] /= sdist;
                    if (!or_any_hit(s, xo, sd, 0.0, sdist - s->eps, 0, NULL)) {
                        if (M->type != 0) return 0;   /* the gradient covers Lambertian surfaces */
                        dn g = dn_scale(dn_div(dn_mul(cx, cl), dist2), s->light_area);
                        for (int a = 0; a < 3; ++a)
                            L.c[a] = dn_add(L.c[a], dn_scale(g, T[a] * M->albedo[a] / OR_PI * LM->emission[a]));
                    }
                }
            }
        }
        if (b == max_depth - 1) break;
        if (M->type != 0) return 0;
        dn bu = u[5 + 5 * b], bv = u[6 + 5 * b];
        double ft[3], fb[3];
        frame(ns, ft, fb, NULL);
        dn phi = dn_scale(bv, 2.0 * OR_PI);
        dn r = dn_sqrt(bu);
        dn lz = dn_sqrt(dn_addc(dn_scale(bu, -1.0), 1.0));
        dv3 wi = dv_add(dv_add(dv_cs(ft, dn_mul(r, dn_cos(phi))), dv_cs(fb, dn_mul(r, dn_sin(phi)))), dv_cs(ns, lz));
        for (int a = 0; a < 3; ++a) T[a] *= M->albedo[a];
        double epsn[3] = {s->eps * ns[0], s->eps * ns[1], s->eps * ns[2]};
        o = dv_add(x, dv_c(epsn));
        d = wi;
    }
    dn pi = dn_add(dn_add(dn_scale(L.c[0], 0.2126), dn_scale(L.c[1], 0.7152)), dn_scale(L.c[2], 0.0722));
    for (int a = 0; a < 3; ++a) f[a] = L.c[a].v;
    if (!isfinite(pi.v)) return 0;
    if (pi.v > 0)
        for (int j = 0; j < D; ++j) grad[j] = pi.g[j] / pi.v;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* chains                                                                    */
/* ------------------------------------------------------------------------ */
struct or_ctx {
    const or_scene* s;
    or_params p;
    int32_t D, m, nx;
    uint32_t T_large;
    float S1, S2, log2_ratio;
    uint32_t* q;
    double* f;
    double* pi;
    int32_t* k;
    int64_t* boot;
    double* lam;
    int64_t* n;
    uint64_t *i, *A, *h, *h_prev;
    double *w, *Rc;
    float* sig;
    double* img;
    double* Bk;                   /* sum of pi over uniform samples landing in region k */
    uint64_t nU;                  /* number of uniform samples (bootstrap + large steps) */
    /* quadtree partition (Sec. 6.2): node children (-1 for a leaf), leaf region ids, depths */
    int32_t cap;                  /* region capacity */
    int32_t* qt_child;
    int32_t* qt_leaf;
    int32_t* qt_depth;
    int32_t qt_nodes;
    uint64_t since_refine;
    double bhat;
    uint64_t mut;
    uint64_t st[8];
    uint64_t mala_st[2];          /* Langevin moves proposed, accepted */
    uint32_t T_mala;
    double* g;                    /* [C][D] gradient of log pi at each chain's state (Langevin runs) */
    /* sharded stepping: i, A, h (cap each), large steps and nU at the start of the epoch; Bk */
    uint64_t* snap_i;
    double* snap_B;
    int inited;
    or_mut_hook mh;
    or_upd_hook uh;
    or_prop_hook ph;
    /* the last Langevin move (tests): drift, normal draws, tau_x, sensitivity */
    double lm_m[OR_MAX_GRAD], lm_z[OR_MAX_GRAD], lm_tau, lm_sens;
    void* user;
};

int32_t or_init_tables(or_ctx* c);

or_ctx* or_ctx_create(const or_scene* s, const or_params* p)
{
    if (!s || !p) return NULL;
    int32_t D = 2 + 5 * p->max_depth;
    if (D > OR_MAX_DIM || p->n_chains <= 0 || p->width <= 0 || p->height <= 0 || p->region_px <= 0)
        return NULL;
    if (p->chain_first < 0 || p->chains_total < 0 ||
        (p->chains_total > 0 && (int64_t)p->chain_first + p->n_chains > (int64_t)p->chains_total) ||
        (p->chains_total == 0 && p->chain_first != 0))
        return NULL;
    /* the truncated normal's sigma stays below 4 (lambda_max = 2 ln 4): wider
     * is uniform on the window for every purpose */
    if (p->kernel != 0 && !(p->kernel == 1 && p->lambda_max <= 2.0 * log(4.0) + 1e-12)) return NULL;
    or_ctx* c = (or_ctx*)calloc(1, sizeof(or_ctx));
    c->s = s;
    c->p = *p;
    c->D = D;
    c->nx = (p->width + p->region_px - 1) / p->region_px;
    int32_t ny = (p->height + p->region_px - 1) / p->region_px;
    c->m = c->nx * ny;
    if (p->dir_cells > 1) {
        if (p->partition != 0 || p->target_mode != 0 || p->max_depth < 1 || s->toy || p->dir_cells > 64) {
            free(c);
            return NULL;
        }
        c->m *= p->dir_cells * p->dir_cells;
    }
    c->cap = c->m;
    if (p->partition == 1) {
        if (p->qt_max_leaves < 1 || p->qt_max_depth < 0 || p->qt_max_depth > 24 || p->target_mode != 0) {
            free(c);
            return NULL;
        }
        c->m = 1;
        c->cap = p->qt_max_leaves;
        size_t nodes = (size_t)(4 * (size_t)c->cap / 3 + 8);
        c->qt_child = (int32_t*)malloc(sizeof(int32_t) * 4 * nodes);
        c->qt_leaf = (int32_t*)malloc(sizeof(int32_t) * nodes);
        c->qt_depth = (int32_t*)malloc(sizeof(int32_t) * nodes);
    }
    double tl = ceil(p->p_large * 16777216.0);
    c->T_large = (uint32_t)(tl < 0 ? 0 : (tl > 16777216.0 ? 16777216.0 : tl));
    double tm = ceil(p->p_mala * 16777216.0);
    c->T_mala = (uint32_t)(tm < 0 ? 0 : (tm > 16777216.0 ? 16777216.0 : tm));
    c->S1 = (float)(p->s1 * 4294967296.0);
    c->S2 = (float)(p->s2 * 4294967296.0);
    c->log2_ratio = (float)log2(p->s2 / p->s1);
    size_t C = (size_t)p->n_chains, m = (size_t)c->cap;
    c->q = (uint32_t*)calloc(C * (size_t)D, sizeof(uint32_t));
    c->f = (double*)calloc(C * 3, sizeof(double));
    c->pi = (double*)calloc(C, sizeof(double));
    c->k = (int32_t*)calloc(C, sizeof(int32_t));
    c->boot = (int64_t*)calloc(C, sizeof(int64_t));
    c->lam = (double*)calloc(m, sizeof(double));
    c->n = (int64_t*)calloc(m, sizeof(int64_t));
    c->i = (uint64_t*)calloc(m, sizeof(uint64_t));
    c->A = (uint64_t*)calloc(m, sizeof(uint64_t));
    c->h = (uint64_t*)calloc(m, sizeof(uint64_t));
    c->h_prev = (uint64_t*)calloc(m, sizeof(uint64_t));
    c->w = (double*)calloc(m, sizeof(double));
    c->Rc = (double*)calloc(m, sizeof(double));
    c->sig = (float*)calloc(m, sizeof(float));
    c->img = (double*)calloc((size_t)p->width * (size_t)p->height * 3, sizeof(double));
    c->Bk = (double*)calloc(m, sizeof(double));
    if (p->p_mala > 0) {
        /* the Langevin strategy differentiates the path map: Lambertian scenes,
         * D <= 62, a positive step and drift bound */
        int ok = D <= OR_MAX_GRAD && p->mala_tau > 0 && p->mala_drift_max > 0 && p->p_large + p->p_mala <= 1.0;
        for (int32_t mi = 0; mi < s->nm && ok && !s->toy; ++mi) ok = s->mat[mi].type == 0;
        if (!ok) {
            or_ctx_destroy(c);
            return NULL;
        }
        c->g = (double*)calloc(C * (size_t)D, sizeof(double));
    }
    return c;
}

void or_ctx_destroy(or_ctx* c)
{
    if (!c) return;
    free(c->q); free(c->f); free(c->pi); free(c->k); free(c->boot); free(c->lam); free(c->n);
    free(c->i); free(c->A); free(c->h); free(c->h_prev); free(c->w); free(c->Rc); free(c->sig);
    free(c->img); free(c->Bk);
    free(c->qt_child); free(c->qt_leaf); free(c->qt_depth);
    free(c->g);
    free(c->snap_i); free(c->snap_B);
    free(c);
}

void or_set_hooks(or_ctx* c, or_mut_hook mh, or_upd_hook uh, void* user)
{
    c->mh = mh; c->uh = uh; c->user = user;
}

void or_set_prop_hook(or_ctx* c, or_prop_hook ph) { c->ph = ph; }

void or_last_mala(const or_ctx* c, double* m, double* z, double out2[2])
{
    for (int32_t d = 0; d < c->D && d < OR_MAX_GRAD; ++d) {
        if (m) m[d] = c->lm_m[d];
        if (z) z[d] = c->lm_z[d];
    }
    if (out2) { out2[0] = c->lm_tau; out2[1] = c->lm_sens; }
}

static void pixel_of(const or_ctx* c, const uint32_t* q, int32_t* px, int32_t* py)
{
    *px = (int32_t)(((uint64_t)(q[0] >> 8) * (uint64_t)c->p.width) >> 24);
    *py = (int32_t)(((uint64_t)(q[1] >> 8) * (uint64_t)c->p.height) >> 24);
}

/* Region of a state in the 2-D screen-space partition (Sec. 5.4): a cell of
 * the uniform grid (Sec. 6.1), or the quadtree leaf containing (u0, u1)
 * (Sec. 6.2).  The quadtree halves [0,1)^2 per level, so the quadrant at
 * depth l is bit 31 - l of the state words u0, u1. */
int32_t or_region_of(const or_ctx* c, const uint32_t* q)
{
    if (c->p.partition == 1) {
        int32_t node = 0, depth = 0;
        while (c->qt_child[4 * node] >= 0) {
            int32_t bx = (int32_t)((q[0] >> (31 - depth)) & 1u), by = (int32_t)((q[1] >> (31 - depth)) & 1u);
            node = c->qt_child[4 * node + bx + 2 * by];
            depth++;
        }
        return c->qt_leaf[node];
    }
    int32_t px, py;
    pixel_of(c, q, &px, &py);
    int32_t k = px / c->p.region_px + (py / c->p.region_px) * c->nx;
    if (c->p.dir_cells > 1) {
        /* 4-D partition in PSS (analogue of Sec. 5.4): the screen region
         * crossed with a dir_cells^2 grid over the first bounce's BSDF
         * coordinates (u5, u6), cells taken like pixels */
        const int32_t g = c->p.dir_cells;
        const int32_t cu = (int32_t)(((uint64_t)(q[5] >> 8) * (uint64_t)g) >> 24);
        const int32_t cv = (int32_t)(((uint64_t)(q[6] >> 8) * (uint64_t)g) >> 24);
        k = k * g * g + cu + cv * g;
    }
    return k;
}

/* Refinement of the quadtree partition (Sec. 6.2), run once every qt_refine
 * mutations at an epoch boundary: every leaf visited more than qt_split times
 * since the previous pass splits into four children.  Children inherit the
 * scale parameter lambda, get n = n_parent / 4 updates (at least 1), and are
 * not split again in the same pass.  Readings: a visit is a post-MH state of
 * any mutation (the histogram h); i, A and the visit counts of the children
 * start at 0; the first child keeps the parent's region id and the other
 * three get the next free ids, leaves taken in node order; splitting stops at
 * qt_max_depth and qt_max_leaves. */
static void quadtree_refine(or_ctx* c)
{
    const or_params* p = &c->p;
    const int32_t nodes0 = c->qt_nodes;
    for (int32_t node = 0; node < nodes0; ++node) {
        if (c->qt_child[4 * node] >= 0) continue;
        const int32_t k = c->qt_leaf[node];
        if (c->h[k] - c->h_prev[k] <= (uint64_t)p->qt_split) continue;
        if (c->qt_depth[node] >= p->qt_max_depth || c->m + 3 > c->cap) continue;
        const double lam = c->lam[k];
        const int64_t nc = c->n[k] / 4 > 1 ? c->n[k] / 4 : 1;
        for (int32_t q = 0; q < 4; ++q) {
            const int32_t ch = c->qt_nodes++;
            const int32_t id = q == 0 ? k : c->m++;
            c->qt_child[4 * node + q] = ch;
            for (int32_t j = 0; j < 4; ++j) c->qt_child[4 * ch + j] = -1;
            c->qt_leaf[ch] = id;
            c->qt_depth[ch] = c->qt_depth[node] + 1;
            c->lam[id] = lam;
            c->n[id] = nc;
            c->i[id] = c->A[id] = c->h[id] = c->h_prev[id] = 0;
            c->w[id] = 1.0;
            c->Rc[id] = 0.0;
            c->Bk[id] = 0.0;
            c->sig[id] = sigma_of_lambda(lam);
        }
        c->qt_leaf[node] = -1;
    }
    for (int32_t k = 0; k < c->m; ++k) c->h_prev[k] = c->h[k];
    for (int32_t ch = 0; ch < c->p.n_chains; ++ch) c->k[ch] = or_region_of(c, &c->q[(size_t)ch * c->D]);
}

static double weight_of(const or_ctx* c, int32_t k) { return c->p.target_mode ? c->w[k] : 1.0; }

/* chains over the whole (possibly sharded) population, and the global id of
 * this context's chain `chain` (the Philox key of its draws) */
static int32_t chains_all(const or_ctx* c) { return c->p.chains_total > 0 ? c->p.chains_total : c->p.n_chains; }
static uint32_t gid(const or_ctx* c, uint32_t chain) { return (uint32_t)c->p.chain_first + chain; }

/* Large step: an independent uniform point of the PSS cube. */
static void large_step(const or_ctx* c, uint32_t chain, uint64_t mut, uint32_t* qy)
{
    for (int32_t j = 0; 4 * j < c->D; ++j) {
        uint32_t r[4];
        draw(c->p.seed, mut, gid(c, chain), 1u + (uint32_t)j, r);
        for (int a = 0; a < 4 && 4 * j + a < c->D; ++a) qy[4 * j + a] = r[a];
    }
}

/* Small step: every dimension perturbed with the one scale sigma_{k(x)}
 * (Alg. 1, region lookup, step size and proposal; Sec. 5.2 proposal of the current state's region). */
static void small_step(const or_ctx* c, uint32_t chain, uint64_t mut, int32_t kx,
                       const uint32_t* qx, uint32_t* qy)
{
    float sigS2 = c->sig[kx] * c->S2;
    for (int32_t j = 0; 2 * j < c->D; ++j) {
        uint32_t r[4];
        draw(c->p.seed, mut, gid(c, chain), 1u + (uint32_t)j, r);
        for (int a = 0; a < 2 && 2 * j + a < c->D; ++a) {
            int32_t dim = 2 * j + a;
            if (c->p.kernel == 1) {   /* signed offset; the sign word is not used */
                qy[dim] = qx[dim] + (uint32_t)(uint64_t)or_truncnorm_delta(r[2 * a], (double)c->sig[kx]);
                continue;
            }
            int64_t dq = or_kelemen_delta(r[2 * a], sigS2, c->log2_ratio);
            uint32_t off = (uint32_t)(uint64_t)dq;
            qy[dim] = (r[2 * a + 1] >> 31) ? qx[dim] - off : qx[dim] + off;
        }
    }
}

/* Ratio T_{k(y)}(x|y) / T_{k(x)}(y|x) of the truncated-normal kernel: per
 * dimension phi(delta / s) / (s Z(s)) with the nearest-image displacement
 * delta (|delta| < 1/2) and s = sigma of the state the move starts from. */
static double truncnorm_ratio(const or_ctx* c, int32_t kx, int32_t ky, const uint32_t* qx, const uint32_t* qy)
{
    const double sx = (double)c->sig[kx], sy = (double)c->sig[ky];
    if (sx == sy) return 1.0;
    const double zx = erf(1.0 / (2.0 * sqrt(2.0) * sx)), zy = erf(1.0 / (2.0 * sqrt(2.0) * sy));
    double s2 = 0.0;
    for (int32_t d = 0; d < c->D; ++d) {
        double dl = (double)(int32_t)(qy[d] - qx[d]) * (1.0 / 4294967296.0);
        s2 += dl * dl;
    }
    return exp(c->D * log((sx * zx) / (sy * zy)) - 0.5 * s2 * (1.0 / (sy * sy) - 1.0 / (sx * sx)));
}

/* Ratio T_{k(y)}(x|y) / T_{k(x)}(y|x) of the state-dependent mixture
 * (Sec. 5.2, eq. regional_proposal_mixture) for the Kelemen kernel.  Its
 * magnitude density 1 / (|delta| ln(s2/s1)) does not depend on sigma inside
 * its support [sigma s1, sigma s2], so the ratio is the indicator that every
 * offset lies in the reverse kernel's support.  Reading: the paper writes
 * only the generic MH ratio (Sec. 3.2); the reverse kernel is the one of the
 * proposal's region. */
static int reverse_support(const or_ctx* c, int32_t kx, int32_t ky, const uint32_t* qx, const uint32_t* qy)
{
    if (c->sig[ky] == c->sig[kx]) return 1;
    float lo = c->sig[ky] * c->S1, hi = c->sig[ky] * c->S2;
    for (int32_t d = 0; d < c->D; ++d) {
        int64_t dd = (int64_t)(int32_t)(qy[d] - qx[d]);
        float mag = (float)(dd < 0 ? -dd : dd);
        if (!(mag >= lo && mag <= hi)) return 0;
    }
    return 1;
}

/* MH acceptance of the mixture (Sec. 3.2, strategy-mixture form; Sec. 5.2):
 * a = min(1, pi~(y) T_{k(y)}(x|y) s(j|y) / (pi~(x) T_{k(x)}(y|x) s(j|x))),
 * pi~ = pi / w_k (w = 1 in plain mode).  The strategy probabilities s do not
 * depend on the state and cancel; R is the kernel ratio (1 for the large step,
 * whose density is uniform).  A zero-contribution current state (possible only
 * at initialisation) accepts any proposal the reverse kernel can undo. */
static double accept_prob(const or_ctx* c, int32_t kx, int32_t ky, double pix, double piy, double R)
{
    if (!(R > 0)) return 0.0;
    double ptx = pix / weight_of(c, kx), pty = piy / weight_of(c, ky);
    if (!(ptx > 0)) return 1.0;
    return dmin(1.0, pty / ptx * R);
}

/* kernel ratio of a proposal: 1 for the large step, the reverse-support
 * indicator for Kelemen, the density ratio for the truncated normal */
static double kernel_ratio(const or_ctx* c, int32_t large, int32_t kx, int32_t ky, const uint32_t* qx,
                           const uint32_t* qy)
{
    if (large) return 1.0;
    if (c->p.kernel == 1) return truncnorm_ratio(c, kx, ky, qx, qy);
    return (double)reverse_support(c, kx, ky, qx, qy);
}

double or_accept_prob(const or_ctx* c, const uint32_t* qx, const uint32_t* qy,
                      double pix, double piy, int32_t large)
{
    int32_t kx = or_region_of(c, qx), ky = or_region_of(c, qy);
    return accept_prob(c, kx, ky, pix, piy, kernel_ratio(c, large, kx, ky, qx, qy));
}

/* splat f(x) / pi(x) of the chain's current state at its pixel */
static void splat(or_ctx* c, int32_t chain)
{
    if (!(c->pi[chain] > 0)) return;
    int32_t px, py;
    pixel_of(c, &c->q[(size_t)chain * c->D], &px, &py);
    size_t o = ((size_t)py * c->p.width + px) * 3;
    for (int a = 0; a < 3; ++a) c->img[o + a] += c->f[3 * chain + a] / c->pi[chain];
}

/* ------------------------------------------------------------------------ */
/* Langevin strategy (MALA, Roberts & Tweedie 1996, with the drift's norm    */
/* bounded): y = x + m_x + sqrt(tau_x) xi, m_x = (tau_x / 2) grad log pi(x)  */
/* scaled to norm <= drift_max, xi ~ N(0, I) by Box-Muller from the          */
/* mutation's Philox draws (call 1 + j gives dims 4j..4j+3), on the torus    */
/* with nearest-image displacements.  tau_x = min(tau sigma_{k(x)}^2, 0.01): */
/* the step adapts with the region of the current state (a standard        */
/* deviation of at most 0.1 keeps the nearest-image density exact to       */
/* e^-12), so the reverse density uses                                      */
/* tau_{k(y)} and the ratio keeps its normalising factors.  Not in the      */
/* paper (gradient methods appear only as related work); the region weight  */
/* is constant inside a region, so grad log pi~ = grad log pi.              */
/* ------------------------------------------------------------------------ */
static void mala_drift(const or_ctx* c, const double* g, double tau, double* m)
{
    double n2 = 0.0;
    for (int32_t d = 0; d < c->D; ++d) {
        m[d] = 0.5 * tau * g[d];
        n2 += m[d] * m[d];
    }
    double n = sqrt(n2);
    if (n > c->p.mala_drift_max)
        for (int32_t d = 0; d < c->D; ++d) m[d] *= c->p.mala_drift_max / n;
}

/* log N(delta; m, tau I) */
static double mala_logq(int32_t D, double tau, const double* delta, const double* m)
{
    double s2 = 0.0;
    for (int32_t d = 0; d < D; ++d) {
        double e = delta[d] - m[d];
        s2 += e * e;
    }
    return -0.5 * D * log(2.0 * OR_PI * tau) - s2 / (2.0 * tau);
}

static void mala_mutate(or_ctx* c, uint32_t chain, double xi)
{
    const int32_t D = c->D;
    uint32_t qy[OR_MAX_DIM];
    uint32_t* qx = &c->q[(size_t)chain * D];
    const double* gx = &c->g[(size_t)chain * D];
    const int32_t kx = c->k[chain];
    const double tx = dmin(c->p.mala_tau * (double)c->sig[kx] * (double)c->sig[kx], OR_MALA_TAU_MAX);
    double mx[OR_MAX_GRAD], my[OR_MAX_GRAD], delta[OR_MAX_GRAD], gy[OR_MAX_GRAD], z[OR_MAX_GRAD + 3];
    mala_drift(c, gx, tx, mx);
    for (int32_t j = 0; 4 * j < D; ++j) {
        uint32_t r[4];
        draw(c->p.seed, c->mut, gid(c, chain), 1u + (uint32_t)j, r);
        for (int a = 0; a < 2; ++a) {
            double u1 = ((double)(r[2 * a] >> 8) + 0.5) * (1.0 / 16777216.0);
            double u2 = u24(r[2 * a + 1]);
            double rho = sqrt(-2.0 * log(u1));
            z[4 * j + 2 * a] = rho * cos(2.0 * OR_PI * u2);
            z[4 * j + 2 * a + 1] = rho * sin(2.0 * OR_PI * u2);
        }
    }
    const double st = sqrt(tx);
    for (int32_t d = 0; d < D; ++d) {
        double step = mx[d] + st * z[d];
        int64_t dq = (int64_t)llrint(step * 4294967296.0);
        qy[d] = qx[d] + (uint32_t)(uint64_t)dq;
        c->lm_m[d] = mx[d];
        c->lm_z[d] = z[d];
    }
    c->lm_tau = tx;
    if (c->ph) c->ph(c->user, chain, c->mut, 2, qy, D);
    for (int32_t d = 0; d < D; ++d) delta[d] = (double)(int32_t)(qy[d] - qx[d]) * (1.0 / 4294967296.0);
    int32_t ky = or_region_of(c, qy);
    double fy[3];
    if (or_path_grad(c->s, c->p.width, c->p.height, c->p.max_depth, qy, fy, gy) != 1) {
        fy[0] = fy[1] = fy[2] = 0.0;
        for (int32_t d = 0; d < D; ++d) gy[d] = 0.0;
        c->st[5]++;
    }
    const double ty = dmin(c->p.mala_tau * (double)c->sig[ky] * (double)c->sig[ky], OR_MALA_TAU_MAX);
    mala_drift(c, gy, ty, my);
    c->lm_sens = 0.0;
    for (int32_t d = 0; d < D; ++d)
        c->lm_sens += fabs(mx[d]) * fabs(delta[d] - mx[d]) / tx + fabs(my[d]) * fabs(delta[d] + my[d]) / ty;
    double piy = luminance(fy);
    double ptx = c->pi[chain] / weight_of(c, kx), pty = piy / weight_of(c, ky);
    double a;
    if (!(pty > 0)) {
        a = 0.0;
    } else if (!(ptx > 0)) {
        a = 1.0;
    } else {
        double lr = log(pty) - log(ptx);
        if (!(c->p.debug_flags & 2)) {   /* bit 1: planted mistake, proposal densities dropped */
            double back[OR_MAX_GRAD];
            for (int32_t d = 0; d < D; ++d) back[d] = -delta[d];
            lr += mala_logq(D, ty, back, my) - mala_logq(D, tx, delta, mx);
        }
        a = lr >= 0 ? 1.0 : exp(lr);
    }
    int32_t acc = xi < a;
    if (c->mh) {
        /* the test hook sees a Langevin move as kind 2, with the path's
         * binary32 error model */
        or_err E;
        double fe[3];
        path_eval_impl(c->s, c->p.width, c->p.height, c->p.max_depth, qy, fe, NULL, &E, NULL);
        c->mh(c->user, chain, c->mut, qy, D, 2, 0, E.dec, E.ferr, xi, fy, &a, &acc);
        piy = luminance(fy);
    }
    c->mala_st[0]++;
    if (acc) {
        memcpy(qx, qy, sizeof(uint32_t) * (size_t)D);
        for (int x = 0; x < 3; ++x) c->f[3 * chain + x] = fy[x];
        memcpy(&c->g[(size_t)chain * D], gy, sizeof(double) * (size_t)D);
        c->pi[chain] = piy;
        c->k[chain] = ky;
        c->st[1]++;
        c->mala_st[1]++;
    }
    c->h[c->k[chain]] += 1;
    c->st[0]++;
    splat(c, chain);
}

/* One Metropolis-Hastings mutation of chain `chain` (Alg. 1, mutation step). */
static void mutate(or_ctx* c, uint32_t chain)
{
    int32_t D = c->D;
    uint32_t r0[4], qy[OR_MAX_DIM];
    uint32_t* qx = &c->q[(size_t)chain * D];
    draw(c->p.seed, c->mut, gid(c, chain), 0u, r0);
    int32_t large = (r0[0] >> 8) < c->T_large;
    double xi = u24(r0[1]);
    if (!large && c->g && (r0[0] >> 8) < c->T_large + c->T_mala) {
        mala_mutate(c, chain, xi);
        return;
    }
    int32_t kx = c->k[chain];
    if (large) large_step(c, chain, c->mut, qy);
    else small_step(c, chain, c->mut, kx, qx, qy);
    if (c->ph) c->ph(c->user, chain, c->mut, large, qy, D);
    int32_t ky = or_region_of(c, qy);
    double R = kernel_ratio(c, large, kx, ky, qx, qy);
    if (c->p.debug_flags & 1) R = 1.0;   /* planted mistake for negative-control tests */
    double fy[3] = {0, 0, 0};
    or_err E = {OR_INF, {0, 0, 0}};
    /* early rejection: a proposal outside the reverse Kelemen kernel's support
     * has R = 0 by definition; the truncated normal's density ratio is
     * positive (if it underflows, a = 0 but the path is still evaluated) */
    const int early = c->p.kernel == 1 ? 0 : !(R > 0);
    if (!early) {
        uint64_t cnt[3] = {0, 0, 0};
        if (!path_eval_impl(c->s, c->p.width, c->p.height, c->p.max_depth, qy, fy, NULL, c->mh ? &E : NULL, cnt))
            c->st[5]++;
        c->st[6] += cnt[0];
    } else {
        c->st[4]++;
    }
    double piy = luminance(fy);
    double a = accept_prob(c, kx, ky, c->pi[chain], piy, R);
    int32_t acc = xi < a;
    if (c->mh) {
        c->mh(c->user, chain, c->mut, qy, D, large, early, E.dec, E.ferr, xi, fy, &a, &acc);
        piy = luminance(fy);
    }
    if (large) {
        c->st[2]++;
        c->Bk[ky] += piy;
        c->nU++;
    } else {
        /* adaptation statistics of the current state's region (Alg. 1, acceptance statistics) */
        c->st[3]++;
        c->i[kx] += 1;
        c->A[kx] += (uint64_t)llrint(a * 4294967296.0);
    }
    if (acc) {
        memcpy(qx, qy, sizeof(uint32_t) * (size_t)D);
        for (int x = 0; x < 3; ++x) c->f[3 * chain + x] = fy[x];
        c->pi[chain] = piy;
        c->k[chain] = ky;
        c->st[1]++;
        if (c->g) {   /* the Langevin strategy needs grad log pi of every state */
            double fg[3];
            or_path_grad(c->s, c->p.width, c->p.height, c->p.max_depth, qx, fg, &c->g[(size_t)chain * D]);
        }
    }
    c->h[c->k[chain]] += 1;
    c->st[0]++;
    /* splat the chain's current state (estimator of Sec. 3.2) */
    splat(c, chain);
}

/* Region-parameter update at an epoch boundary (Alg. 1, region update).
 * Reading: the trigger is i_k >= L and alpha_hat = A_k / i_k, which equals
 * eq. est_exp_acc (Alg. 1 tests i_k > L but divides by L).  The update follows
 * eq. update_lambda as printed: lambda grows when the acceptance estimate is
 * above the target (the prose after it states the opposite direction; the
 * equation agrees with adaptive scaling).  lambda is clamped to
 * [lambda_min, lambda_max] (Sec. 7.1 limits it below by -30).  At most one
 * update per region per epoch. */
static void region_update(or_ctx* c)
{
    const or_params* p = &c->p;
    for (int32_t k = 0; k < c->m; ++k) {
        if (c->i[k] >= (uint64_t)p->L) {
            double ah = (double)c->A[k] / (4294967296.0 * (double)c->i[k]);
            int32_t sg = ah > p->alpha_star ? 1 : (ah < p->alpha_star ? -1 : 0);
            if (c->uh) c->uh(c->user, k, c->i[k], c->A[k], ah, &sg);
            double g = dmin(p->gamma_max, p->gamma_scale / sqrt((double)c->n[k]));  /* eq. step_size_n */
            double lam = c->lam[k] + g * (double)sg;                                  /* eq. update_lambda */
            if (lam < p->lambda_min) lam = p->lambda_min;
            if (lam > p->lambda_max) lam = p->lambda_max;
            c->lam[k] = lam;
            c->n[k] += 1;
            c->i[k] = 0;
            c->A[k] = 0;
        }
        c->sig[k] = sigma_of_lambda(c->lam[k]);
    }
}

/* Region-weighted target (extension, not in the paper; modelled on two-stage
 * MLT, Sec. 8): w_k tracks the region's share of the true target, so pi / w
 * spreads the chains evenly over the regions.  Binary64, fixed region order. */
static void weight_update(or_ctx* c)
{
    double m = (double)c->m, S = 0.0;
    for (int32_t k = 0; k < c->m; ++k) S += c->w[k] * (double)(c->h[k] - c->h_prev[k]);
    if (S > 0) {
        for (int32_t k = 0; k < c->m; ++k) c->Rc[k] += c->w[k] * (double)(c->h[k] - c->h_prev[k]) / S;
        double T = 0.0;
        for (int32_t k = 0; k < c->m; ++k) T += c->Rc[k];
        for (int32_t k = 0; k < c->m; ++k) c->w[k] = m * dmax(c->Rc[k] / T, c->p.w_floor / m);
    }
    memcpy(c->h_prev, c->h, sizeof(uint64_t) * (size_t)c->m);
}

static void boot_sample(const or_ctx* c, uint64_t s, uint32_t* q)
{
    for (int32_t j = 0; 4 * j < c->D; ++j) {
        uint32_t r[4];
        draw(c->p.seed, s, 0xFFFFFFFFu, 0x8000u + (uint32_t)j, r);
        for (int a = 0; a < 4 && 4 * j + a < c->D; ++a) q[4 * j + a] = r[a];
    }
}

/* Bootstrap (Sec. 3.2: b estimated by independent Monte Carlo in a
 * preprocess) and the initial states.  Reading: the paper does not say how
 * the initial paths are chosen.  Every chain g of the population takes the
 * uniform sample s where the cumulative sum of pi over all n = K C samples
 * (K = n_boot / C) first exceeds t_g = (g + u_g) / C * sum(pi), u_g a
 * uniform of its own: systematic resampling in proportion to pi, so each
 * chain starts on a contributing path and the starting states follow pi.
 * Without a contributing sample, chain g starts at sample g K.
 * b = sum of all pi / n. */
int32_t or_init(or_ctx* c)
{
    const or_params* p = &c->p;
    const int32_t C_all = chains_all(c);
    int64_t K = p->n_bootstrap / C_all;
    if (K <= 0) return -1;
    const int64_t n = K * (int64_t)C_all;
    if (p->partition == 1) or_init_tables(c);   /* the region lookup needs the root */
    uint32_t q[OR_MAX_DIM];
    double f[3], total = 0.0;
    double* pis = (double*)malloc(sizeof(double) * (size_t)n);
    if (!pis) return -1;
    memset(c->Bk, 0, sizeof(double) * (size_t)c->m);
    /* every sample of the population (all shards): b and the distribution
     * need all of them; only this context's chains take a starting state */
    double* cum = (double*)malloc(sizeof(double) * (size_t)n);   /* inclusive cumulative sums */
    if (!cum) {
        free(pis);
        return -1;
    }
    for (int64_t s = 0; s < n; ++s) {
        boot_sample(c, (uint64_t)s, q);
        if (!or_path_eval(c->s, p->width, p->height, p->max_depth, q, f, NULL, NULL)) c->st[5]++;
        pis[s] = luminance(f);
        c->Bk[or_region_of(c, q)] += pis[s];
        total += pis[s];
        cum[s] = total;
    }
    for (int32_t ch = 0; ch < p->n_chains; ++ch) {
        const int32_t g = p->chain_first + ch;
        int64_t sel = (int64_t)g * K;
        if (total > 0.0) {
            uint32_t r[4];
            draw(p->seed, (uint64_t)g, 0xFFFFFFFFu, 0x7FFEu, r);
            const double t = ((double)g + u24(r[0])) / (double)C_all * total;
            int64_t lo = 0, hi = n;   /* the first s with cum[s] > t, n if none */
            while (lo < hi) {
                const int64_t mid = lo + (hi - lo) / 2;
                if (cum[mid] > t) hi = mid;
                else lo = mid + 1;
            }
            sel = lo < n ? lo : -1;
            for (int64_t s = n - 1; s >= 0 && sel < 0; --s)   /* t at the very end: rounding */
                if (pis[s] > 0.0) sel = s;
        }
        c->boot[ch] = sel;
        uint32_t* qc = &c->q[(size_t)ch * c->D];
        boot_sample(c, (uint64_t)sel, qc);
        or_path_eval(c->s, p->width, p->height, p->max_depth, qc, &c->f[3 * ch], NULL, NULL);
        c->pi[ch] = luminance(&c->f[3 * ch]);
        c->k[ch] = or_region_of(c, qc);
        if (c->g) {
            double fg[3];
            or_path_grad(c->s, p->width, p->height, p->max_depth, qc, fg, &c->g[(size_t)ch * c->D]);
        }
    }
    free(cum);
    free(pis);
    c->st[7] = (uint64_t)(K * C_all);
    c->nU = (uint64_t)(K * C_all);
    c->bhat = total / (double)(K * C_all);
    return or_init_tables(c);
}

/* Alg. 1, initialisation: lambda_k = initial scale, i_k = A_k = 0, n_k = 1 */
int32_t or_init_tables(or_ctx* c)
{
    if (c->p.partition == 1) {
        c->m = 1;
        c->qt_nodes = 1;
        for (int32_t j = 0; j < 4; ++j) c->qt_child[j] = -1;
        c->qt_leaf[0] = 0;
        c->qt_depth[0] = 0;
        c->since_refine = 0;
        for (int32_t ch = 0; ch < c->p.n_chains; ++ch) c->k[ch] = 0;
    }
    for (int32_t k = 0; k < c->m; ++k) {
        c->lam[k] = c->p.lambda_init;
        c->n[k] = 1;
        c->i[k] = c->A[k] = c->h[k] = c->h_prev[k] = 0;
        c->w[k] = 1.0;
        c->Rc[k] = 0.0;
        c->sig[k] = sigma_of_lambda(c->lam[k]);
    }
    c->mut = 0;
    c->inited = 1;
    return 0;
}

void or_refresh_sigma(or_ctx* c)
{
    for (int32_t k = 0; k < c->m; ++k) c->sig[k] = sigma_of_lambda(c->lam[k]);
}

int32_t or_set_state(or_ctx* c, uint32_t chain, const uint32_t* q)
{
    if ((int64_t)chain >= c->p.n_chains) return -1;
    uint32_t* qc = &c->q[(size_t)chain * c->D];
    memcpy(qc, q, sizeof(uint32_t) * (size_t)c->D);
    or_path_eval(c->s, c->p.width, c->p.height, c->p.max_depth, qc, &c->f[3 * chain], NULL, NULL);
    c->pi[chain] = luminance(&c->f[3 * chain]);
    c->k[chain] = or_region_of(c, qc);
    if (c->g) {
        double fg[3];
        or_path_grad(c->s, c->p.width, c->p.height, c->p.max_depth, qc, fg, &c->g[(size_t)chain * c->D]);
    }
    return 0;
}

int32_t or_mutate_one(or_ctx* c, uint32_t chain, uint64_t mut)
{
    if (!c->inited || (int64_t)chain >= c->p.n_chains) return -1;
    uint64_t keep = c->mut;
    c->mut = mut;
    mutate(c, chain);
    c->mut = keep;
    return 0;
}

/* E mutations of every chain of this context (Alg. 1, mutation step) */
static void epoch_mutations(or_ctx* c)
{
    uint64_t mut0 = c->mut;
    for (uint32_t ch = 0; ch < (uint32_t)c->p.n_chains; ++ch) {
        c->mut = mut0;
        for (int32_t j = 0; j < c->p.epoch_len; ++j) {
            mutate(c, ch);
            c->mut++;
        }
    }
    c->mut = mut0 + (uint64_t)c->p.epoch_len;
}

/* the epoch boundary: Alg. 1, region update, the weighted target's weights, and
 * a quadtree pass every qt_refine mutations of the whole population */
static void epoch_boundary(or_ctx* c)
{
    region_update(c);
    if (c->p.target_mode) weight_update(c);
    if (c->p.partition == 1) {
        c->since_refine += (uint64_t)chains_all(c) * (uint64_t)c->p.epoch_len;
        if (c->since_refine >= (uint64_t)c->p.qt_refine) {
            c->since_refine = 0;
            quadtree_refine(c);
        }
    }
}

int32_t or_run_epochs(or_ctx* c, int64_t n_epochs)
{
    if (!c->inited) return -1;
    for (int64_t e = 0; e < n_epochs; ++e) {
        epoch_mutations(c);
        epoch_boundary(c);
    }
    return 0;
}

int32_t or_region_capacity(const or_ctx* c) { return c->cap; }

/* Sharded stepping: the region tables every context shares are its own
 * tables at the start of the epoch plus what all contexts' chains added
 * during it (the paper's threads share i_k and A_k through atomics, Sec. 6;
 * integer sums do not depend on their order). */
int32_t or_epoch_mutate(or_ctx* c, uint64_t* counts, double* sums)
{
    if (!c->inited || c->snap_i) return -1;
    const size_t cap = (size_t)c->cap;
    c->snap_i = (uint64_t*)malloc(sizeof(uint64_t) * (3 * cap + 2));
    c->snap_B = (double*)malloc(sizeof(double) * cap);
    memcpy(c->snap_i, c->i, sizeof(uint64_t) * cap);
    memcpy(c->snap_i + cap, c->A, sizeof(uint64_t) * cap);
    memcpy(c->snap_i + 2 * cap, c->h, sizeof(uint64_t) * cap);
    c->snap_i[3 * cap] = c->st[2];
    c->snap_i[3 * cap + 1] = c->nU;
    memcpy(c->snap_B, c->Bk, sizeof(double) * cap);
    epoch_mutations(c);
    for (size_t k = 0; k < cap; ++k) {
        counts[k] = c->i[k] - c->snap_i[k];
        counts[cap + k] = c->A[k] - c->snap_i[cap + k];
        counts[2 * cap + k] = c->h[k] - c->snap_i[2 * cap + k];
        sums[k] = c->Bk[k] - c->snap_B[k];
    }
    counts[3 * cap] = c->st[2] - c->snap_i[3 * cap];
    return 0;
}

int32_t or_epoch_update(or_ctx* c, const uint64_t* counts, const double* sums)
{
    if (!c->snap_i) return -1;
    const size_t cap = (size_t)c->cap;
    for (size_t k = 0; k < cap; ++k) {
        c->i[k] = c->snap_i[k] + counts[k];
        c->A[k] = c->snap_i[cap + k] + counts[cap + k];
        c->h[k] = c->snap_i[2 * cap + k] + counts[2 * cap + k];
        c->Bk[k] = c->snap_B[k] + sums[k];
    }
    /* uniform samples of the whole population: the bootstrap plus every large step */
    c->nU = c->snap_i[3 * cap + 1] + counts[3 * cap];
    free(c->snap_i);
    free(c->snap_B);
    c->snap_i = NULL;
    c->snap_B = NULL;
    epoch_boundary(c);
    return 0;
}

int32_t or_refine(or_ctx* c)
{
    if (c->p.partition != 1 || !c->inited) return -1;
    quadtree_refine(c);
    return 0;
}

int32_t or_quadtree(const or_ctx* c, int32_t* child, int32_t* leaf, int32_t* depth, int32_t cap_nodes)
{
    if (c->p.partition != 1) return 0;
    for (int32_t n = 0; n < c->qt_nodes && n < cap_nodes; ++n) {
        for (int32_t j = 0; j < 4; ++j) child[4 * n + j] = c->qt_child[4 * n + j];
        leaf[n] = c->qt_leaf[n];
        depth[n] = c->qt_depth[n];
    }
    return c->qt_nodes;
}

/* Plain target: I_j = (b / N) sum_i f(x_i) / pi(x_i) over the chain states
 * at pixel j (Sec. 3.2), times W H for radiance units.
 * Region-weighted target (extension): the target changes between epochs, so
 * the chains' region occupancy lags behind it; within one region w is
 * constant and the visits follow pi restricted to the region.  Each region is
 * therefore normalised by its own mass, I_j = B_k sum_i f / pi / h_k, with
 * B_k = int_{P_k} pi estimated from the uniform samples (bootstrap and large
 * steps).  At equilibrium h_k / N = B_k / b and both forms agree. */
void or_read_image(const or_ctx* c, double* out)
{
    const or_params* p = &c->p;
    double N = (double)c->mut * (double)chains_all(c);   /* a shard returns its share of the image */
    double WH = (double)p->width * (double)p->height;
    for (int32_t y = 0; y < p->height; ++y)
        for (int32_t x = 0; x < p->width; ++x) {
            double s;
            if (!p->target_mode) {
                s = N > 0 ? c->bhat * WH / N : 0.0;
            } else {
                int32_t k = x / p->region_px + (y / p->region_px) * c->nx;
                s = (c->h[k] > 0 && c->nU > 0) ? WH * (c->Bk[k] / (double)c->nU) / (double)c->h[k] : 0.0;
            }
            size_t o = ((size_t)y * p->width + x) * 3;
            for (int a = 0; a < 3; ++a) out[o + a] = c->img[o + a] * s;
        }
}

int32_t or_dims(const or_ctx* c) { return c->D; }
int32_t or_regions(const or_ctx* c) { return c->m; }
uint64_t or_mutations_done(const or_ctx* c) { return c->mut; }
double or_bhat(const or_ctx* c) { return c->bhat; }
uint32_t* or_state_q(or_ctx* c) { return c->q; }
double* or_state_f(or_ctx* c) { return c->f; }
double* or_state_pi(or_ctx* c) { return c->pi; }
int32_t* or_state_k(or_ctx* c) { return c->k; }
int64_t* or_boot_choice(or_ctx* c) { return c->boot; }
double* or_lambda(or_ctx* c) { return c->lam; }
int64_t* or_n_updates(or_ctx* c) { return c->n; }
uint64_t* or_visits(or_ctx* c) { return c->i; }
uint64_t* or_accsum(or_ctx* c) { return c->A; }
uint64_t* or_hist(or_ctx* c) { return c->h; }
uint64_t* or_hist_prev(or_ctx* c) { return c->h_prev; }
double* or_weight(or_ctx* c) { return c->w; }
float* or_sigma(or_ctx* c) { return c->sig; }
double* or_image_acc(or_ctx* c) { return c->img; }
void or_stats(const or_ctx* c, uint64_t out[8]) { memcpy(out, c->st, sizeof c->st); }
void or_mala_stats(const or_ctx* c, uint64_t out[2]) { memcpy(out, c->mala_st, sizeof c->mala_st); }
const double* or_state_grad(const or_ctx* c, uint32_t chain) { return c->g ? &c->g[(size_t)chain * c->D] : NULL; }
