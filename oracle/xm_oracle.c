/*
 * xm_oracle.c -- plain FP64 CPU oracle of the sky cross-match.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the independent checker of the CUDA
 * library: only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py load it. The product path never calls it, and it
 * shares no code, header, table or constant with the CUDA sources.
 *
 * What it computes (paper §2.1, "Sky" functional case): every source A_i of
 * the first catalogue carries a region centred on its position -- a circle,
 * an ellipse or a rectangle -- whose size is a fixed value or a per-source
 * catalogue column and whose orientation is a position angle with a
 * configurable zero-point and direction of rotation. The members of A_i are
 * the sources B_j of the second catalogue inside that region, decided from
 * their distance to A_i and the limits of the region. Positions may be given
 * in equatorial or galactic coordinates (paper §2).
 *
 * The oracle is the plain definition, evaluated pair by pair in FP64:
 *   1. every position becomes an equatorial unit vector p; a galactic input is
 *      rotated by the IAU galactic frame (north galactic pole at
 *      RA 192.85948 deg, Dec 27.12825 deg; galactic longitude of the north
 *      celestial pole 122.93192 deg);
 *   2. A_i gets its local east/north basis (e, n) in its INPUT frame, rotated
 *      to equatorial with p, so the position angle counts from the north of
 *      the frame the catalogue was given in;
 *   3. for B_j: x = p_B.e, y = p_B.n, z = p_B.p_A; the angular separation is
 *      rho = atan2(hypot(x, y), z) and the bearing (east of north) is
 *      phi = atan2(x, y);
 *   4. with PA_eff = pa_zero + pa_dir * PA, the region frame coordinates are
 *      X = rho cos(phi - PA_eff) (along the major axis), Y = rho sin(...)
 *      (azimuthal-equidistant frame centred on A_i);
 *   5. circle: rho <= r; ellipse: (X/a)^2 + (Y/b)^2 <= 1;
 *      rectangle: |X| <= a and |Y| <= b (a, b half-sides); closed boundary;
 *   6. the separation is reported in arcsec;
 *   7. with every pair also its normalised distance: the factor by which the
 *      region must be scaled about A_i to reach B_j -- rho/r for a circle,
 *      sqrt((X/a)^2 + (Y/b)^2) for an ellipse, max(|X|/a, |Y|/b) for a
 *      rectangle -- so B_j is a member when it is at most 1. It orders the
 *      members by how deep inside the region they lie (the "best" pair by
 *      normalised distance) and places them among concentric scaled copies
 *      of the region (paper §3, ClumpPopulator).
 * A region with a zero size has no interior and matches nothing (whether a
 * separation is exactly zero depends on the order of rounding, so the closed
 * boundary would make every such candidate a last-ulp decision).
 *
 * Two ways of finding the candidates, with identical results:
 *   - brute force: every (i, j) pair;
 *   - a sparse 3-D voxel grid on the unit vectors with edge at least the
 *     chord of the largest region's bounding radius, so any member lies in
 *     one of the 27 voxels around A_i. This only prunes (§2.3 uses a sky
 *     partition the same way) and has no RA wrap or pole special case.
 *
 * Borderline report: a candidate whose decision margin (|rho/r - 1| for a
 * circle, |q - 1| for an ellipse, |max(|X|/a, |Y|/b) - 1| for a rectangle)
 * is below tau is listed, since the last-ulp differences between two correct
 * FP64 programs may decide it either way.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846
#define DEG (OR_PI / 180.0)
#define ARCSEC (OR_PI / 648000.0)

enum { OR_EQ = 0, OR_GAL = 1 };
enum { OR_CIRCLE = 0, OR_ELLIPSE = 1, OR_RECT = 2 };
enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2 };

/* ---------------------------------------------------------------- frames -- */

/* Rows of the equatorial -> galactic rotation: the galactic x (l=0,b=0),
 * y (l=90,b=0) and z (north galactic pole) axes written in equatorial
 * coordinates, built from the three defining angles of the galactic frame. */
static void eq_to_gal_rows(double xg[3], double yg[3], double zg[3]) {
    const double ra_ngp = 192.85948 * DEG, dec_ngp = 27.12825 * DEG;
    const double l_ncp = 122.93192 * DEG;
    zg[0] = cos(dec_ngp) * cos(ra_ngp);
    zg[1] = cos(dec_ngp) * sin(ra_ngp);
    zg[2] = sin(dec_ngp);
    /* w: the north celestial pole projected on the galactic plane; it points
     * to galactic longitude l_ncp. */
    double w[3] = {-zg[2] * zg[0], -zg[2] * zg[1], 1.0 - zg[2] * zg[2]};
    double nw = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    for (int k = 0; k < 3; k++) w[k] /= nw;
    /* k = zg x w points to longitude l_ncp + 90 deg */
    double kk[3] = {zg[1] * w[2] - zg[2] * w[1], zg[2] * w[0] - zg[0] * w[2],
                    zg[0] * w[1] - zg[1] * w[0]};
    for (int k = 0; k < 3; k++) {
        xg[k] = cos(l_ncp) * w[k] - sin(l_ncp) * kk[k];
        yg[k] = sin(l_ncp) * w[k] + cos(l_ncp) * kk[k];
    }
}

/* m (row-major) maps galactic vectors to equatorial: v_eq = m v_gal. */
void or_gal_to_eq_matrix(double m[9]) {
    double xg[3], yg[3], zg[3];
    eq_to_gal_rows(xg, yg, zg);
    for (int k = 0; k < 3; k++) {
        m[3 * k + 0] = xg[k];
        m[3 * k + 1] = yg[k];
        m[3 * k + 2] = zg[k];
    }
}

static void sph_vectors(double lon_deg, double lat_deg, double p[3], double e[3],
                        double n[3]) {
    double lam = fmod(lon_deg, 360.0);
    if (lam < 0) lam += 360.0;
    lam *= DEG;
    double bet = lat_deg * DEG;
    double cl = cos(lam), sl = sin(lam), cb = cos(bet), sb = sin(bet);
    p[0] = cb * cl; p[1] = cb * sl; p[2] = sb;
    if (e) { e[0] = -sl; e[1] = cl; e[2] = 0.0; }
    if (n) { n[0] = -sb * cl; n[1] = -sb * sl; n[2] = cb; }
}

static void mat_vec(const double m[9], const double v[3], double out[3]) {
    double r[3];
    for (int k = 0; k < 3; k++) r[k] = m[3 * k] * v[0] + m[3 * k + 1] * v[1] + m[3 * k + 2] * v[2];
    out[0] = r[0]; out[1] = r[1]; out[2] = r[2];
}

static int coord_ok(double lon, double lat) {
    return isfinite(lon) && isfinite(lat) && lat >= -90.0 && lat <= 90.0;
}

/* Equatorial unit vector (and, when asked, the input-frame east/north basis
 * rotated to equatorial) of one position. */
static void to_eq(double lon, double lat, int frame, const double m[9], double p[3],
                  double e[3], double n[3]) {
    sph_vectors(lon, lat, p, e, n);
    if (frame == OR_GAL) {
        mat_vec(m, p, p);
        if (e) mat_vec(m, e, e);
        if (n) mat_vec(m, n, n);
    }
}

static void vec_to_sph(const double p[3], double* lon_deg, double* lat_deg) {
    double lon = atan2(p[1], p[0]) / DEG;
    if (lon < 0) lon += 360.0;
    if (lon >= 360.0) lon -= 360.0;
    *lon_deg = lon;
    *lat_deg = atan2(p[2], hypot(p[0], p[1])) / DEG;
}

/* Converts positions given in `frame` to equatorial RA/Dec in degrees. */
int or_to_equatorial(int64_t n, const double* lon, const double* lat, int frame, double* ra,
                     double* dec) {
    double m[9];
    or_gal_to_eq_matrix(m);
    for (int64_t i = 0; i < n; i++) {
        if (!coord_ok(lon[i], lat[i])) return OR_EINVAL;
        double p[3];
        to_eq(lon[i], lat[i], frame, m, p, NULL, NULL);
        vec_to_sph(p, &ra[i], &dec[i]);
    }
    return OR_OK;
}

/* Converts equatorial RA/Dec (degrees) to `frame` longitude/latitude. */
int or_from_equatorial(int64_t n, const double* ra, const double* dec, int frame, double* lon,
                       double* lat) {
    double m[9], mt[9];
    or_gal_to_eq_matrix(m);
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) mt[3 * r + c] = m[3 * c + r];
    for (int64_t i = 0; i < n; i++) {
        if (!coord_ok(ra[i], dec[i])) return OR_EINVAL;
        double p[3];
        sph_vectors(ra[i], dec[i], p, NULL, NULL);
        if (frame == OR_GAL) mat_vec(mt, p, p);
        vec_to_sph(p, &lon[i], &lat[i]);
    }
    return OR_OK;
}

/* --------------------------------------------------------------- regions -- */

typedef struct {
    double p[3], e[3], n[3];
    double a, b;       /* radians: circle radius / semi-axes / half-sides */
    double theta;      /* PA_eff in radians, east of north of the input frame */
    double bound;      /* bounding angular radius of the region (radians) */
    int empty;         /* zero size: matches nothing */
} a_src;

typedef struct {
    int shape;
    const double *a_col, *b_col, *pa_col;
    double a_fix, b_fix, pa_fix;
    double scale, unit_arcsec, pa_zero_deg;
    int pa_dir;
} region_spec;

static int make_region(const region_spec* rs, int64_t i, a_src* s) {
    double a = rs->a_col ? rs->a_col[i] : rs->a_fix;
    double b = rs->b_col ? rs->b_col[i] : rs->b_fix;
    double pa = rs->pa_col ? rs->pa_col[i] : rs->pa_fix;
    if (rs->shape == OR_CIRCLE) b = a;
    if (!isfinite(a) || !isfinite(b) || !isfinite(pa) || a < 0 || b < 0) return OR_EINVAL;
    double k = rs->scale * rs->unit_arcsec * ARCSEC;
    s->a = a * k;
    s->b = b * k;
    s->theta = (rs->pa_zero_deg + rs->pa_dir * pa) * DEG;
    s->empty = (s->a == 0.0 || s->b == 0.0);
    if (rs->shape == OR_RECT)
        s->bound = hypot(s->a, s->b);
    else
        s->bound = s->a > s->b ? s->a : s->b;
    return OR_OK;
}

/* Membership of one candidate: returns 1 if inside; rho (radians) and the
 * decision margin are returned through the pointers. */
static int test_pair(int shape, const a_src* A, const double pb[3], double* rho_out,
                     double* margin_out, double* dist_out) {
    double x = pb[0] * A->e[0] + pb[1] * A->e[1] + pb[2] * A->e[2];
    double y = pb[0] * A->n[0] + pb[1] * A->n[1] + pb[2] * A->n[2];
    double z = pb[0] * A->p[0] + pb[1] * A->p[1] + pb[2] * A->p[2];
    double rho = atan2(hypot(x, y), z);
    *rho_out = rho;
    if (A->empty) { *margin_out = INFINITY; *dist_out = INFINITY; return 0; }
    if (shape == OR_CIRCLE) {
        *margin_out = fabs(rho / A->a - 1.0);
        *dist_out = rho / A->a;
        return rho <= A->a;
    }
    double phi = atan2(x, y);
    double X = rho * cos(phi - A->theta);
    double Y = rho * sin(phi - A->theta);
    if (shape == OR_ELLIPSE) {
        double q = (X / A->a) * (X / A->a) + (Y / A->b) * (Y / A->b);
        *margin_out = fabs(q - 1.0);
        *dist_out = sqrt(q);
        return q <= 1.0;
    }
    double m = fmax(fabs(X) / A->a, fabs(Y) / A->b);
    *margin_out = fabs(m - 1.0);
    *dist_out = m;
    return m <= 1.0;
}

/* ---------------------------------------------------------------- output -- */

typedef struct {
    int64_t *a, *b;
    double* sep;
    double* dist;
    int64_t n, cap;
    int64_t *ba, *bb;
    double* bm;
    int64_t nb, capb;
    int oom;
} pairbuf;

static void pb_push(pairbuf* P, int64_t a, int64_t b, double sep, double dist) {
    if (P->n == P->cap) {
        int64_t c = P->cap ? 2 * P->cap : 1024;
        int64_t* na = realloc(P->a, c * sizeof(int64_t));
        if (na) P->a = na;
        int64_t* nb = realloc(P->b, c * sizeof(int64_t));
        if (nb) P->b = nb;
        double* ns = realloc(P->sep, c * sizeof(double));
        if (ns) P->sep = ns;
        double* nd = realloc(P->dist, c * sizeof(double));
        if (nd) P->dist = nd;
        if (!na || !nb || !ns || !nd) { P->oom = 1; return; }
        P->cap = c;
    }
    P->a[P->n] = a; P->b[P->n] = b; P->sep[P->n] = sep; P->dist[P->n] = dist; P->n++;
}

static void pb_border(pairbuf* P, int64_t a, int64_t b, double m) {
    if (P->nb == P->capb) {
        int64_t c = P->capb ? 2 * P->capb : 64;
        int64_t* na = realloc(P->ba, c * sizeof(int64_t));
        if (na) P->ba = na;
        int64_t* nb = realloc(P->bb, c * sizeof(int64_t));
        if (nb) P->bb = nb;
        double* nm = realloc(P->bm, c * sizeof(double));
        if (nm) P->bm = nm;
        if (!na || !nb || !nm) { P->oom = 1; return; }
        P->capb = c;
    }
    P->ba[P->nb] = a; P->bb[P->nb] = b; P->bm[P->nb] = m; P->nb++;
}

typedef struct or_result {
    int64_t n, nb;
    int64_t *a, *b, *ba, *bb;
    double *sep, *dist, *bm;
} or_result;

/* --------------------------------------------------------------- matcher -- */

typedef struct { uint64_t key; int64_t row; } vox_entry;

static int vox_cmp(const void* x, const void* y) {
    const vox_entry* u = x;
    const vox_entry* v = y;
    if (u->key != v->key) return u->key < v->key ? -1 : 1;
    return (u->row > v->row) - (u->row < v->row);
}

static int64_t vox_axis(double c, double edge) {
    /* a component may round a hair below -1; merging it into voxel 0 only
     * widens the candidate set */
    int64_t k = (int64_t)floor((c + 1.0) / edge);
    return k < 0 ? 0 : k;
}

static uint64_t vox_key(int64_t ix, int64_t iy, int64_t iz) {
    return (uint64_t)ix | ((uint64_t)iy << 21) | ((uint64_t)iz << 42);
}

typedef struct { int64_t b; double sep, margin, dist; } member;

static int member_cmp(const void* x, const void* y) {
    const member* u = x;
    const member* v = y;
    return (u->b > v->b) - (u->b < v->b);
}

typedef struct {
    /* shared, read-only */
    int shape, mode;
    double tau, edge;
    const a_src* A;
    const int64_t* a_rows;   /* row of each a_src in the caller's catalogue */
    int64_t nA;
    const double* pB;        /* 3 * nB */
    int64_t nB;
    const vox_entry* vox;    /* sorted, grid mode */
    int64_t nvox;
    /* per thread */
    int64_t lo, hi;
    pairbuf out;
} worker;

static int64_t lower_key(const vox_entry* v, int64_t n, uint64_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (v[mid].key < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

static void consider(worker* w, const a_src* A, int64_t arow, int64_t j, member** mem,
                     int64_t* nm, int64_t* cm) {
    double rho, margin, dist;
    int in = test_pair(w->shape, A, w->pB + 3 * j, &rho, &margin, &dist);
    if (margin < w->tau) pb_border(&w->out, arow, j, margin);
    if (!in) return;
    if (*nm == *cm) {
        int64_t c = *cm ? 2 * *cm : 64;
        member* nmem = realloc(*mem, c * sizeof(member));
        if (!nmem) { w->out.oom = 1; return; }
        *mem = nmem;
        *cm = c;
    }
    (*mem)[*nm].b = j;
    (*mem)[*nm].sep = rho / ARCSEC;
    (*mem)[*nm].margin = margin;
    (*mem)[*nm].dist = dist;
    (*nm)++;
}

static void* run_worker(void* arg) {
    worker* w = arg;
    member* mem = NULL;
    int64_t cm = 0;
    for (int64_t i = w->lo; i < w->hi && !w->out.oom; i++) {
        const a_src* A = &w->A[i];
        int64_t arow = w->a_rows[i];
        int64_t nm = 0;
        if (w->mode == 0) {
            for (int64_t j = 0; j < w->nB; j++) consider(w, A, arow, j, &mem, &nm, &cm);
        } else {
            int64_t ix = vox_axis(A->p[0], w->edge), iy = vox_axis(A->p[1], w->edge),
                    iz = vox_axis(A->p[2], w->edge);
            for (int dz = -1; dz <= 1; dz++)
                for (int dy = -1; dy <= 1; dy++)
                    for (int dx = -1; dx <= 1; dx++) {
                        if (ix + dx < 0 || iy + dy < 0 || iz + dz < 0) continue;
                        uint64_t key = vox_key(ix + dx, iy + dy, iz + dz);
                        for (int64_t k = lower_key(w->vox, w->nvox, key);
                             k < w->nvox && w->vox[k].key == key; k++)
                            consider(w, A, arow, w->vox[k].row, &mem, &nm, &cm);
                    }
        }
        /* members of one A in ascending B row (canonical order) */
        qsort(mem, nm, sizeof(member), member_cmp);
        for (int64_t k = 0; k < nm; k++) pb_push(&w->out, arow, mem[k].b, mem[k].sep, mem[k].dist);
    }
    free(mem);
    return NULL;
}

static int key_in(const uint64_t* keys, int64_t n, uint64_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (keys[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo < n && keys[lo] == key;
}

static int u64_cmp(const void* x, const void* y) {
    uint64_t u = *(const uint64_t*)x, v = *(const uint64_t*)y;
    return (u > v) - (u < v);
}

typedef struct {
    const double* pB;
    const uint64_t* need;
    int64_t nneed, lo, hi;
    double edge;
    vox_entry* out;
    int64_t nout;
} vox_job;

static void* vox_fill(void* arg) {
    vox_job* J = arg;
    J->nout = 0;
    for (int64_t j = J->lo; j < J->hi; j++) {
        const double* p = J->pB + 3 * j;
        uint64_t key = vox_key(vox_axis(p[0], J->edge), vox_axis(p[1], J->edge),
                               vox_axis(p[2], J->edge));
        if (J->need && !key_in(J->need, J->nneed, key)) continue;
        J->out[J->lo + J->nout].key = key;
        J->out[J->lo + J->nout].row = j;
        J->nout++;
    }
    return NULL;
}

/*
 * Cross-match: members of each selected A source (all of them when a_subset
 * is NULL) among B. mode 0 = brute force, 1 = voxel grid. Pairs come out in
 * ascending (A row, B row). Returns NULL with *status set on invalid input or
 * exhausted memory.
 */
or_result* or_match(int64_t nA, const double* a_lon, const double* a_lat, int a_frame,
                    int shape, const double* a_col, const double* b_col, const double* pa_col,
                    double a_fix, double b_fix, double pa_fix, double scale,
                    double unit_arcsec, double pa_zero_deg, int pa_dir, int64_t nB,
                    const double* b_lon, const double* b_lat, int b_frame,
                    const int64_t* a_subset, int64_t n_subset, int mode, int nthreads,
                    double tau, int* status) {
    *status = OR_OK;
    if (shape < OR_CIRCLE || shape > OR_RECT || (pa_dir != 1 && pa_dir != -1) ||
        !isfinite(scale) || scale < 0 || !isfinite(unit_arcsec) || unit_arcsec <= 0 ||
        !isfinite(pa_zero_deg) || nA < 0 || nB < 0) {
        *status = OR_EINVAL;
        return NULL;
    }
    region_spec rs = {shape, a_col, b_col, pa_col, a_fix, b_fix, pa_fix,
                      scale, unit_arcsec, pa_zero_deg, pa_dir};
    double m[9];
    or_gal_to_eq_matrix(m);

    /* whole-catalogue validity, as the library checks it */
    for (int64_t i = 0; i < nA; i++) {
        a_src tmp;
        if (!coord_ok(a_lon[i], a_lat[i]) || make_region(&rs, i, &tmp) != OR_OK) {
            *status = OR_EINVAL;
            return NULL;
        }
    }
    for (int64_t j = 0; j < nB; j++)
        if (!coord_ok(b_lon[j], b_lat[j])) { *status = OR_EINVAL; return NULL; }

    int64_t nsel = a_subset ? n_subset : nA;
    a_src* A = malloc((nsel ? nsel : 1) * sizeof(a_src));
    int64_t* a_rows = malloc((nsel ? nsel : 1) * sizeof(int64_t));
    double* pB = malloc((nB ? 3 * nB : 3) * sizeof(double));
    if (!A || !a_rows || !pB) { free(A); free(a_rows); free(pB); *status = OR_ENOMEM; return NULL; }
    double bmax = 0.0;
    for (int64_t k = 0; k < nsel; k++) {
        int64_t i = a_subset ? a_subset[k] : k;
        if (i < 0 || i >= nA) { free(A); free(a_rows); free(pB); *status = OR_EINVAL; return NULL; }
        a_rows[k] = i;
        make_region(&rs, i, &A[k]);
        to_eq(a_lon[i], a_lat[i], a_frame, m, A[k].p, A[k].e, A[k].n);
        if (!A[k].empty && A[k].bound > bmax) bmax = A[k].bound;
    }
    for (int64_t j = 0; j < nB; j++) to_eq(b_lon[j], b_lat[j], b_frame, m, pB + 3 * j, NULL, NULL);

    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;

    /* voxel edge: the chord of the largest bounding radius, with a relative
     * margin far above FP64 rounding; regions of a third of the sky or more
     * fall back to brute force */
    double edge = 0.0;
    vox_entry* vox = NULL;
    int64_t nvox = 0;
    if (mode == 1) {
        if (bmax >= OR_PI / 3) {
            mode = 0;
        } else {
            edge = 2.0 * sin(bmax / 2.0) * (1.0 + 1e-6) + 1e-12;
            if (edge < 2.0 / 1048576.0) edge = 2.0 / 1048576.0;
        }
    }
    if (mode == 1) {
        /* with a subset of A, keep only the B in voxels some selected A can
         * reach (pure pruning: same results, less sorting) */
        uint64_t* need = NULL;
        int64_t nneed = 0;
        if (a_subset) {
            need = malloc((nsel > 0 ? 27 * nsel : 1) * sizeof(uint64_t));
            if (!need) { free(A); free(a_rows); free(pB); *status = OR_ENOMEM; return NULL; }
            for (int64_t k = 0; k < nsel; k++) {
                int64_t ix = vox_axis(A[k].p[0], edge), iy = vox_axis(A[k].p[1], edge),
                        iz = vox_axis(A[k].p[2], edge);
                for (int dz = -1; dz <= 1; dz++)
                    for (int dy = -1; dy <= 1; dy++)
                        for (int dx = -1; dx <= 1; dx++)
                            if (ix + dx >= 0 && iy + dy >= 0 && iz + dz >= 0)
                                need[nneed++] = vox_key(ix + dx, iy + dy, iz + dz);
            }
            qsort(need, nneed, sizeof(uint64_t), u64_cmp);
        }
        vox = malloc((nB ? nB : 1) * sizeof(vox_entry));
        if (!vox) { free(need); free(A); free(a_rows); free(pB); *status = OR_ENOMEM; return NULL; }
        vox_job jobs[256];
        pthread_t th[256];
        int nt = nthreads;
        for (int t = 0; t < nt; t++) {
            jobs[t].pB = pB; jobs[t].need = need; jobs[t].nneed = nneed; jobs[t].edge = edge;
            jobs[t].lo = nB * t / nt; jobs[t].hi = nB * (t + 1) / nt; jobs[t].out = vox;
            pthread_create(&th[t], NULL, vox_fill, &jobs[t]);
        }
        for (int t = 0; t < nt; t++) {
            pthread_join(th[t], NULL);
            memmove(vox + nvox, vox + jobs[t].lo, jobs[t].nout * sizeof(vox_entry));
            nvox += jobs[t].nout;
        }
        free(need);
        qsort(vox, nvox, sizeof(vox_entry), vox_cmp);
    }

    worker* W = calloc(nthreads, sizeof(worker));
    pthread_t th[256];
    if (!W) { free(vox); free(A); free(a_rows); free(pB); *status = OR_ENOMEM; return NULL; }
    for (int t = 0; t < nthreads; t++) {
        W[t].shape = shape; W[t].mode = mode; W[t].tau = tau; W[t].edge = edge;
        W[t].A = A; W[t].a_rows = a_rows; W[t].nA = nsel; W[t].pB = pB; W[t].nB = nB;
        W[t].vox = vox; W[t].nvox = nvox;
        W[t].lo = nsel * t / nthreads; W[t].hi = nsel * (t + 1) / nthreads;
        pthread_create(&th[t], NULL, run_worker, &W[t]);
    }
    int oom = 0;
    int64_t total = 0, totalb = 0;
    for (int t = 0; t < nthreads; t++) {
        pthread_join(th[t], NULL);
        oom |= W[t].out.oom;
        total += W[t].out.n;
        totalb += W[t].out.nb;
    }
    or_result* R = calloc(1, sizeof(or_result));
    if (R && !oom) {
        R->a = malloc((total ? total : 1) * sizeof(int64_t));
        R->b = malloc((total ? total : 1) * sizeof(int64_t));
        R->sep = malloc((total ? total : 1) * sizeof(double));
        R->dist = malloc((total ? total : 1) * sizeof(double));
        R->ba = malloc((totalb ? totalb : 1) * sizeof(int64_t));
        R->bb = malloc((totalb ? totalb : 1) * sizeof(int64_t));
        R->bm = malloc((totalb ? totalb : 1) * sizeof(double));
        oom = !R->a || !R->b || !R->sep || !R->dist || !R->ba || !R->bb || !R->bm;
    }
    if (R && !oom) {
        /* threads own contiguous, ascending slices of the selected A */
        for (int t = 0; t < nthreads; t++) {
            memcpy(R->a + R->n, W[t].out.a, W[t].out.n * sizeof(int64_t));
            memcpy(R->b + R->n, W[t].out.b, W[t].out.n * sizeof(int64_t));
            memcpy(R->sep + R->n, W[t].out.sep, W[t].out.n * sizeof(double));
            memcpy(R->dist + R->n, W[t].out.dist, W[t].out.n * sizeof(double));
            R->n += W[t].out.n;
            memcpy(R->ba + R->nb, W[t].out.ba, W[t].out.nb * sizeof(int64_t));
            memcpy(R->bb + R->nb, W[t].out.bb, W[t].out.nb * sizeof(int64_t));
            memcpy(R->bm + R->nb, W[t].out.bm, W[t].out.nb * sizeof(double));
            R->nb += W[t].out.nb;
        }
    }
    for (int t = 0; t < nthreads; t++) {
        free(W[t].out.a); free(W[t].out.b); free(W[t].out.sep); free(W[t].out.dist);
        free(W[t].out.ba); free(W[t].out.bb); free(W[t].out.bm);
    }
    free(W); free(vox); free(A); free(a_rows); free(pB);
    if (!R || oom) {
        if (R) {
            free(R->a); free(R->b); free(R->sep); free(R->dist);
            free(R->ba); free(R->bb); free(R->bm); free(R);
        }
        *status = OR_ENOMEM;
        return NULL;
    }
    return R;
}

int64_t or_result_npairs(const or_result* R) { return R->n; }
int64_t or_result_nborder(const or_result* R) { return R->nb; }

void or_result_copy(const or_result* R, int64_t* a, int64_t* b, double* sep) {
    memcpy(a, R->a, R->n * sizeof(int64_t));
    memcpy(b, R->b, R->n * sizeof(int64_t));
    memcpy(sep, R->sep, R->n * sizeof(double));
}

void or_result_copy_dist(const or_result* R, double* dist) {
    memcpy(dist, R->dist, R->n * sizeof(double));
}

void or_result_copy_border(const or_result* R, int64_t* a, int64_t* b, double* margin) {
    memcpy(a, R->ba, R->nb * sizeof(int64_t));
    memcpy(b, R->bb, R->nb * sizeof(int64_t));
    memcpy(margin, R->bm, R->nb * sizeof(double));
}

void or_result_free(or_result* R) {
    if (!R) return;
    free(R->a); free(R->b); free(R->sep); free(R->dist); free(R->ba); free(R->bb); free(R->bm);
    free(R);
}

/* Separation (arcsec) between two positions given in their frames. */
double or_separation(double lon1, double lat1, int frame1, double lon2, double lat2, int frame2) {
    double m[9], p1[3], p2[3];
    or_gal_to_eq_matrix(m);
    to_eq(lon1, lat1, frame1, m, p1, NULL, NULL);
    to_eq(lon2, lat2, frame2, m, p2, NULL, NULL);
    double c[3] = {p1[1] * p2[2] - p1[2] * p2[1], p1[2] * p2[0] - p1[0] * p2[2],
                   p1[0] * p2[1] - p1[1] * p2[0]};
    double s = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    double d = p1[0] * p2[0] + p1[1] * p2[1] + p1[2] * p2[2];
    return atan2(s, d) / ARCSEC;
}
