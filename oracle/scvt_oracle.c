/*
 * scvt_oracle.c -- plain, slow FP64 CPU oracle for spherical centroidal
 * Voronoi tessellations (SCVT) and the Lloyd-preconditioned LBFGS method.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into a stand-alone shared
 * library that the tests, the package's smoke check and the benchmark's CPU
 * baseline load; the product path (the CUDA library) never calls it and
 * shares no code with it.
 *
 * What it computes, and where the paper defines it:
 *   - spherical Voronoi regions with the Euclidean metric restricted to S^2
 *     (Sec. 2.1, definition of V_i^c; the metric note closing Sec. 2.1);
 *   - mass m_i = int_{V_i} rho, first moment c_i = int_{V_i} y rho and the
 *     energy F = sum_i int_{V_i} |y - z_i|^2 rho (Sec. 2.1, CCVT energy);
 *   - tangential gradient g_i = 2 (c_i.z_i) z_i - 2 c_i and the Lloyd
 *     preconditioner h_i = 1 / (2 c_i.z_i) (Sec. 3.1, spherical form);
 *   - cell integrals as sums over six signed sub-triangles per Delaunay
 *     triangle (vertex, edge midpoint, circumcentre; Sec. 3.2.2);
 *   - Lloyd map z_i <- c_i / |c_i| (Sec. 2.1 constrained centroid, Sec. 2.2.1);
 *   - LBFGS two-loop recursion with the initial inverse Hessian replaced by
 *     diag(h) (Sec. 2.2.2 two-loop; Sec. 3.1 Lloyd preconditioner), Wolfe
 *     line search started at step 1 (Sec. 3.1), re-projection onto S^2.
 *
 * Construction (independent of the GPU path): the spherical Delaunay
 * triangulation is the 3D convex hull of the generators, built by randomised
 * incremental insertion with exact orientation signs (floating-point
 * expansion arithmetic after Shewchuk 1997).  Voronoi vertices are the unit
 * outward normals of the hull facets.  Reductions use pairwise summation.
 *
 * Readings of the paper that this file fixes (ambiguities):
 *   - the 7-point degree-5 Radon rule on each sub-triangle, mapped to the
 *     sphere by radial projection of the planar points with weights scaled
 *     by the signed spherical area (Van Oosterom-Strackee formula);
 *   - tanh cap prefactor (1-gamma)/2, geodesic distance via atan2, and
 *     (1-gamma)/2 (tanh(x)+1) evaluated as (1-gamma)/(1+exp(-2x)) (equal,
 *     without the cancellation of tanh(x)+1 far outside the cap);
 *   - energy accumulated directly as rho |p - z_i|^2 (no 2m - 2 z.c identity);
 *   - line search: More-Thuente (1994) with c1 = 1e-4, c2 = 0.9, step bounds
 *     [1e-20, 1e20], derivative along the projected path
 *     phi'(a) = sum_i g_i(a).q_i / |z_i + a q_i|; a trial step whose
 *     generators do not form a valid tessellation is halved toward the best
 *     step so far and never exceeded again.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_INVALID 1
#define ORC_DEGENERATE 2
#define ORC_NOMEM 3
#define ORC_LINESEARCH 6

typedef struct {
    int kind; /* 0 uniform, 1 polar X3, 2 tanh cap, 3 tanh cap to the 4th power */
    double gamma, alpha, beta;
    double xc[3];
} orc_density;

/* ======================================================================
 * Exact sign of a 3x3 determinant (orientation of four points)
 * Floating-point expansions: two_sum / two_diff / two_prod are exact
 * error-free transformations; grow adds one double to a nonoverlapping
 * expansion (Shewchuk 1997, Grow-Expansion, with zero elimination).
 * Exact as long as no product underflows (the method's standing assumption;
 * coordinates of unit vectors are far from the subnormal range).
 * ====================================================================== */

static void two_sum(double a, double b, double *x, double *y)
{
    double s = a + b;
    double bv = s - a;
    double av = s - bv;
    double br = b - bv;
    double ar = a - av;
    *x = s;
    *y = ar + br;
}

static void two_diff(double a, double b, double *x, double *y)
{
    double d = a - b;
    double bv = a - d;
    double av = d + bv;
    double br = bv - b;
    double ar = a - av;
    *x = d;
    *y = ar + br;
}

static void two_prod(double a, double b, double *x, double *y)
{
    double p = a * b;
    *x = p;
    *y = fma(a, b, -p); /* the rounding error of a product is representable */
}

/* h <- e + b ; returns new length.  e must be nonoverlapping, increasing. */
static int grow(int elen, const double *e, double b, double *h)
{
    double q = b, t;
    int hl = 0;
    for (int i = 0; i < elen; i++) {
        two_sum(q, e[i], &q, &t);
        if (t != 0.0) h[hl++] = t;
    }
    if (q != 0.0 || hl == 0) h[hl++] = q;
    return hl;
}

#define EXP_CAP 512

/* out <- e * f (exact), by accumulating every two_prod term */
static int exp_mul(int elen, const double *e, int flen, const double *f, double *out)
{
    double buf[EXP_CAP];
    int len = 0;
    for (int j = 0; j < flen; j++)
        for (int i = 0; i < elen; i++) {
            double p, err;
            two_prod(e[i], f[j], &p, &err);
            len = grow(len, out, err, buf);
            memcpy(out, buf, sizeof(double) * len);
            len = grow(len, out, p, buf);
            memcpy(out, buf, sizeof(double) * len);
        }
    if (len == 0) { out[0] = 0.0; len = 1; }
    return len;
}

/* out <- e + s*f (exact), s = +1 or -1 */
static int exp_add(int elen, const double *e, int flen, const double *f, double s, double *out)
{
    double a[EXP_CAP], b[EXP_CAP];
    memcpy(a, e, sizeof(double) * elen);
    int len = elen;
    for (int j = 0; j < flen; j++) {
        len = grow(len, a, s * f[j], b);
        memcpy(a, b, sizeof(double) * len);
    }
    memcpy(out, a, sizeof(double) * len);
    return len;
}

static int exp_sign(int len, const double *e)
{
    for (int i = len - 1; i >= 0; i--) {
        if (e[i] > 0) return 1;
        if (e[i] < 0) return -1;
    }
    return 0;
}

/* exact sign of det[a-d ; b-d ; c-d] (rows) */
static int orient3d_exact(const double *a, const double *b, const double *c, const double *d)
{
    double ad[3][2], bd[3][2], cd[3][2];
    for (int k = 0; k < 3; k++) {
        double x, y;
        two_diff(a[k], d[k], &x, &y); ad[k][0] = y; ad[k][1] = x;
        two_diff(b[k], d[k], &x, &y); bd[k][0] = y; bd[k][1] = x;
        two_diff(c[k], d[k], &x, &y); cd[k][0] = y; cd[k][1] = x;
    }
    static const int perm[3][2] = {{1, 2}, {2, 0}, {0, 1}};
    double total[EXP_CAP];
    int tl = 1;
    total[0] = 0.0;
    for (int r = 0; r < 3; r++) {
        int u = perm[r][0], v = perm[r][1];
        double p1[EXP_CAP], p2[EXP_CAP], minor[EXP_CAP], term[EXP_CAP], nt[EXP_CAP];
        int l1 = exp_mul(2, bd[u], 2, cd[v], p1);
        int l2 = exp_mul(2, bd[v], 2, cd[u], p2);
        int lm = exp_add(l1, p1, l2, p2, -1.0, minor);
        int lt = exp_mul(2, ad[r], lm, minor, term);
        tl = exp_add(tl, total, lt, term, 1.0, nt);
        memcpy(total, nt, sizeof(double) * tl);
    }
    return exp_sign(tl, total);
}

/* sign of det[a-d ; b-d ; c-d]: floating filter, exact fallback */
static int orient3d(const double *a, const double *b, const double *c, const double *d)
{
    double adx = a[0] - d[0], ady = a[1] - d[1], adz = a[2] - d[2];
    double bdx = b[0] - d[0], bdy = b[1] - d[1], bdz = b[2] - d[2];
    double cdx = c[0] - d[0], cdy = c[1] - d[1], cdz = c[2] - d[2];
    double m1 = bdy * cdz - bdz * cdy;
    double m2 = bdz * cdx - bdx * cdz;
    double m3 = bdx * cdy - bdy * cdx;
    double det = adx * m1 + ady * m2 + adz * m3;
    double perm = (fabs(bdy * cdz) + fabs(bdz * cdy)) * fabs(adx)
                + (fabs(bdz * cdx) + fabs(bdx * cdz)) * fabs(ady)
                + (fabs(bdx * cdy) + fabs(bdy * cdx)) * fabs(adz);
    double bound = 1.0e-15 * perm; /* > (7 + 56 eps) eps * permanent */
    if (det > bound) return 1;
    if (-det > bound) return -1;
    return orient3d_exact(a, b, c, d);
}

/* exported for the predicate pins */
int orc_orient3d(const double *a, const double *b, const double *c, const double *d, int exact_only)
{
    return exact_only ? orient3d_exact(a, b, c, d) : orient3d(a, b, c, d);
}

/* ======================================================================
 * Convex hull of points on S^2 == spherical Delaunay triangulation
 * Facet (v0,v1,v2) is counter-clockwise seen from outside; edge k runs
 * v[k] -> v[k+1] and nb[k] is the facet across it.  A point p is strictly
 * outside facet (a,b,c) iff orient3d(a,b,c,p) < 0.
 * ====================================================================== */

typedef struct {
    int v[3];
    int nb[3];
    int head;  /* first point of the conflict list */
    int alive;
} hfacet;

typedef struct {
    int n;
    const double *z;
    hfacet *f;
    int nf, capf;
    int *freel;
    int nfree;
    int *pnext; /* conflict list links (per point) */
    int *pfac;  /* per point: the facet whose conflict list holds it */
    int *vis;   /* per facet: stamp when found visible */
    int *nvis;  /* per facet: stamp when found not visible */
    int stamp;
    int *smap, *emap; /* per vertex: new facet starting / ending at it */
} hull_t;

#define P(i) (H->z + 3 * (size_t)(i))

static int outside(const hull_t *H, int fi, int p)
{
    const hfacet *F = &H->f[fi];
    return orient3d(P(F->v[0]), P(F->v[1]), P(F->v[2]), P(p)) < 0;
}

static int facet_new(hull_t *H, int a, int b, int c)
{
    int id;
    if (H->nfree > 0) {
        id = H->freel[--H->nfree];
    } else {
        if (H->nf == H->capf) {
            int nc = H->capf * 2 + 16;
            hfacet *nfp = (hfacet *)realloc(H->f, sizeof(hfacet) * nc);
            int *nv = (int *)realloc(H->vis, sizeof(int) * nc);
            int *nn = (int *)realloc(H->nvis, sizeof(int) * nc);
            int *nfl = (int *)realloc(H->freel, sizeof(int) * nc);
            if (!nfp || !nv || !nn || !nfl) return -1;
            H->f = nfp; H->vis = nv; H->nvis = nn; H->freel = nfl;
            for (int i = H->capf; i < nc; i++) { H->vis[i] = 0; H->nvis[i] = 0; }
            H->capf = nc;
        }
        id = H->nf++;
    }
    hfacet *F = &H->f[id];
    F->v[0] = a; F->v[1] = b; F->v[2] = c;
    F->nb[0] = F->nb[1] = F->nb[2] = -1;
    F->head = -1;
    F->alive = 1;
    H->vis[id] = 0;
    H->nvis[id] = 0;
    return id;
}

static uint64_t splitmix64(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static void hull_free(hull_t *H)
{
    free(H->f); free(H->freel); free(H->pnext); free(H->pfac); free(H->vis); free(H->nvis);
    free(H->smap); free(H->emap);
    memset(H, 0, sizeof(*H));
}

static void conflict_push(hull_t *H, int fi, int p)
{
    H->pnext[p] = H->f[fi].head;
    H->f[fi].head = p;
    H->pfac[p] = fi;
}

/* Build the hull.  Returns ORC_OK, ORC_DEGENERATE (duplicate / coplanar start
 * / a point not strictly outside the current hull / origin not strictly
 * inside) or ORC_NOMEM. */
static int hull_build(hull_t *H, int n, const double *z)
{
    memset(H, 0, sizeof(*H));
    H->n = n;
    H->z = z;
    if (n < 4) return ORC_INVALID;
    H->pnext = (int *)malloc(sizeof(int) * n);
    H->pfac = (int *)malloc(sizeof(int) * n);
    H->smap = (int *)malloc(sizeof(int) * n);
    H->emap = (int *)malloc(sizeof(int) * n);
    int *order = (int *)malloc(sizeof(int) * n);
    int *vlist = NULL, *hf = NULL, *hk = NULL, *newf = NULL, *pts = NULL;
    int capv = 64, caph = 64, capp = 64;
    vlist = (int *)malloc(sizeof(int) * capv);
    hf = (int *)malloc(sizeof(int) * caph);
    hk = (int *)malloc(sizeof(int) * caph);
    newf = (int *)malloc(sizeof(int) * caph);
    pts = (int *)malloc(sizeof(int) * capp);
    int rc = ORC_OK;
    if (!H->pnext || !H->pfac || !H->smap || !H->emap || !order || !vlist || !hf || !hk || !newf || !pts) {
        rc = ORC_NOMEM;
        goto done;
    }
    for (int i = 0; i < n; i++) { order[i] = i; H->smap[i] = -1; H->emap[i] = -1; H->pnext[i] = -1; H->pfac[i] = -1; }
    /* deterministic random insertion order */
    uint64_t seed = 0x5C4D7E11ULL;
    for (int i = n - 1; i > 0; i--) {
        int j = (int)(splitmix64(&seed) % (uint64_t)(i + 1));
        int t = order[i]; order[i] = order[j]; order[j] = t;
    }
    /* initial tetrahedron from the first four points in general position */
    int t0 = order[0], t1 = -1, t2 = -1, t3 = -1, i1 = -1, i2 = -1, i3 = -1;
    for (int i = 1; i < n && t1 < 0; i++) {
        const double *a = P(t0), *b = P(order[i]);
        if (a[0] != b[0] || a[1] != b[1] || a[2] != b[2]) { t1 = order[i]; i1 = i; }
    }
    if (t1 < 0) { rc = ORC_DEGENERATE; goto done; }
    for (int i = 1; i < n && t2 < 0; i++) {
        if (i == i1) continue;
        const double *a = P(t0), *b = P(t1), *c = P(order[i]);
        double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        double w[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        double cr[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
        if (cr[0] != 0 || cr[1] != 0 || cr[2] != 0) { t2 = order[i]; i2 = i; }
    }
    if (t2 < 0) { rc = ORC_DEGENERATE; goto done; }
    for (int i = 1; i < n && t3 < 0; i++) {
        if (i == i1 || i == i2) continue;
        if (orient3d(P(t0), P(t1), P(t2), P(order[i])) != 0) { t3 = order[i]; i3 = i; }
    }
    if (t3 < 0) { rc = ORC_DEGENERATE; goto done; }
    {
        int tv[4] = {t0, t1, t2, t3};
        static const int fc[4][4] = {{0, 1, 2, 3}, {0, 1, 3, 2}, {0, 2, 3, 1}, {1, 2, 3, 0}};
        int fid[4];
        for (int k = 0; k < 4; k++) {
            int a = tv[fc[k][0]], b = tv[fc[k][1]], c = tv[fc[k][2]], d = tv[fc[k][3]];
            if (orient3d(P(a), P(b), P(c), P(d)) < 0) { int t = b; b = c; c = t; }
            fid[k] = facet_new(H, a, b, c);
            if (fid[k] < 0) { rc = ORC_NOMEM; goto done; }
        }
        for (int x = 0; x < 4; x++)
            for (int ex = 0; ex < 3; ex++) {
                int a = H->f[fid[x]].v[ex], b = H->f[fid[x]].v[(ex + 1) % 3];
                for (int y = 0; y < 4; y++) {
                    if (y == x) continue;
                    for (int ey = 0; ey < 3; ey++)
                        if (H->f[fid[y]].v[ey] == b && H->f[fid[y]].v[(ey + 1) % 3] == a)
                            H->f[fid[x]].nb[ex] = fid[y];
                }
            }
        /* assign every other point to a facet it sees */
        for (int i = 1; i < n; i++) {
            if (i == i1 || i == i2 || i == i3) continue;
            int p = order[i], got = 0;
            for (int k = 0; k < 4 && !got; k++)
                if (outside(H, fid[k], p)) { conflict_push(H, fid[k], p); got = 1; }
            if (!got) { rc = ORC_DEGENERATE; goto done; }
        }
    }
    /* insertion in the random order; pfac[p] is a facet that p sees */
    for (int i = 1; i < n; i++) {
        if (i == i1 || i == i2 || i == i3) continue;
        int p = order[i];
        int f0 = H->pfac[p];
        if (f0 < 0 || !H->f[f0].alive) { rc = ORC_DEGENERATE; goto done; }
        H->stamp++;
        int st = H->stamp;
        int nv = 0, nh = 0;
        vlist[nv++] = f0;
        H->vis[f0] = st;
        for (int qi = 0; qi < nv; qi++) {
            int fcur = vlist[qi];
            for (int k = 0; k < 3; k++) {
                int g = H->f[fcur].nb[k];
                if (H->vis[g] == st) continue;
                int isvis = 0;
                if (H->nvis[g] != st) {
                    if (outside(H, g, p)) isvis = 1;
                    else H->nvis[g] = st;
                }
                if (isvis) {
                    H->vis[g] = st;
                    if (nv == capv) { capv *= 2; vlist = (int *)realloc(vlist, sizeof(int) * capv); if (!vlist) { rc = ORC_NOMEM; goto done; } }
                    vlist[nv++] = g;
                } else {
                    if (nh == caph) {
                        caph *= 2;
                        hf = (int *)realloc(hf, sizeof(int) * caph);
                        hk = (int *)realloc(hk, sizeof(int) * caph);
                        newf = (int *)realloc(newf, sizeof(int) * caph);
                        if (!hf || !hk || !newf) { rc = ORC_NOMEM; goto done; }
                    }
                    hf[nh] = fcur; hk[nh] = k; nh++;
                }
            }
        }
        /* collect conflict points of the visible facets */
        int np = 0;
        for (int qi = 0; qi < nv; qi++) {
            int fcur = vlist[qi];
            for (int q = H->f[fcur].head; q >= 0; q = H->pnext[q]) {
                if (q == p) continue;
                if (np == capp) { capp *= 2; pts = (int *)realloc(pts, sizeof(int) * capp); if (!pts) { rc = ORC_NOMEM; goto done; } }
                pts[np++] = q;
            }
        }
        /* retire the visible facets before allocating the cone (slots reuse) */
        for (int qi = 0; qi < nv; qi++) {
            int fcur = vlist[qi];
            H->f[fcur].alive = 0;
            H->f[fcur].head = -1;
        }
        /* cone of new facets over the horizon; horizon data is read from the
         * retired facets, which are only recycled after this loop */
        for (int e = 0; e < nh; e++) {
            int fcur = hf[e], k = hk[e];
            int a = H->f[fcur].v[k], b = H->f[fcur].v[(k + 1) % 3], g = H->f[fcur].nb[k];
            hk[e] = a; /* keep a, b, g for the linking pass */
            hf[e] = g;
            newf[e] = b;
        }
        for (int qi = 0; qi < nv; qi++) H->freel[H->nfree++] = vlist[qi];
        for (int e = 0; e < nh; e++) {
            int a = hk[e], b = newf[e], g = hf[e];
            int nfid = facet_new(H, a, b, p);
            if (nfid < 0) { rc = ORC_NOMEM; goto done; }
            newf[e] = nfid;
            H->f[nfid].nb[0] = g;
            for (int kk = 0; kk < 3; kk++)
                if (H->f[g].v[kk] == b && H->f[g].v[(kk + 1) % 3] == a) H->f[g].nb[kk] = nfid;
            H->smap[a] = nfid;
            H->emap[b] = nfid;
        }
        for (int e = 0; e < nh; e++) {
            hfacet *F = &H->f[newf[e]];
            int a = F->v[0], b = F->v[1];
            F->nb[1] = H->smap[b];
            F->nb[2] = H->emap[a];
            if (F->nb[1] < 0 || F->nb[2] < 0) { rc = ORC_DEGENERATE; goto done; }
        }
        for (int e = 0; e < nh; e++) {
            H->smap[H->f[newf[e]].v[0]] = -1;
            H->emap[H->f[newf[e]].v[1]] = -1;
        }
        H->pfac[p] = -1;
        /* reassign: a point that saw a retired facet now sees a new facet or
         * the surviving facet across a horizon edge */
        for (int t = 0; t < np; t++) {
            int q = pts[t], got = 0;
            for (int e = 0; e < nh && !got; e++) {
                if (outside(H, newf[e], q)) { conflict_push(H, newf[e], q); got = 1; }
                else {
                    int g = H->f[newf[e]].nb[0];
                    if (outside(H, g, q)) { conflict_push(H, g, q); got = 1; }
                }
            }
            if (!got) { rc = ORC_DEGENERATE; goto done; }
        }
    }
    /* checks: 2n-4 facets, origin strictly inside every facet */
    {
        int alive = 0;
        const double o[3] = {0, 0, 0};
        for (int i = 0; i < H->nf; i++) {
            if (!H->f[i].alive) continue;
            alive++;
            if (orient3d(P(H->f[i].v[0]), P(H->f[i].v[1]), P(H->f[i].v[2]), o) <= 0) { rc = ORC_DEGENERATE; goto done; }
        }
        if (alive != 2 * n - 4) rc = ORC_DEGENERATE;
    }
done:
    free(order); free(vlist); free(hf); free(hk); free(newf); free(pts);
    return rc;
}

/* ======================================================================
 * Voronoi cells from the hull (duality, Sec. 2.1 / Sec. 3.2.2)
 * Cell i has corners V_0..V_{d-1} counter-clockwise seen from outside;
 * edge t runs V_t -> V_{t+1} and is dual to Delaunay edge (i, nbr_t).
 * ====================================================================== */

typedef struct {
    int n;
    int *off;    /* n+1 */
    int *nbr;    /* off[n] */
    double *vx;  /* 3*off[n] corner coordinates (rounded to FP64) */
    double *vxl; /* 3*off[n] their remainders: the corner is vx + vxl to ~106 bits */
} vor_t;

static void vor_free(vor_t *V)
{
    free(V->off); free(V->nbr); free(V->vx); free(V->vxl);
    memset(V, 0, sizeof(*V));
}

/* ======================================================================
 * Double-double arithmetic: a value is the unevaluated sum hi + lo of two
 * doubles (about 106 significant bits), built from Knuth's TwoSum, the
 * fast variant for ordered operands and the exact product by FMA.  The
 * cell integrals below form unit vectors (Voronoi corners, edge midpoints,
 * projected rule points) and then quantities much smaller than them: the
 * offsets p - z_i of the energy and the signed areas of sub-triangles a
 * few 1e-4 wide.  Formed from FP64 unit vectors, those lose up to 1.6e-12
 * of the energy of the smallest, most irregular cells of a 2.6M-generator
 * mesh (measured against a 40-digit evaluation of the same formulas); in
 * double-double the loss is far below the 1e-12 the parity tests require.
 * The formulas are unchanged; only these steps carry more bits.
 * ====================================================================== */

typedef struct { double hi, lo; } dd_t;

static dd_t dd_two_sum(double a, double b)
{
    double s = a + b;
    double bb = s - a;
    dd_t r = {s, (a - (s - bb)) + (b - bb)};
    return r;
}

static dd_t dd_fast_sum(double a, double b) /* |a| >= |b| or a == 0 */
{
    double s = a + b;
    dd_t r = {s, b - (s - a)};
    return r;
}

static dd_t dd_d(double a) { dd_t r = {a, 0.0}; return r; }

static dd_t dd_add(dd_t x, dd_t y)
{
    dd_t s = dd_two_sum(x.hi, y.hi);
    dd_t t = dd_two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = dd_fast_sum(s.hi, s.lo);
    s.lo += t.lo;
    return dd_fast_sum(s.hi, s.lo);
}

static dd_t dd_neg(dd_t x) { dd_t r = {-x.hi, -x.lo}; return r; }
static dd_t dd_sub(dd_t x, dd_t y) { return dd_add(x, dd_neg(y)); }

static dd_t dd_mul(dd_t x, dd_t y)
{
    double p = x.hi * y.hi;
    double e = fma(x.hi, y.hi, -p);
    e += x.hi * y.lo;
    e += x.lo * y.hi;
    return dd_fast_sum(p, e);
}

static dd_t dd_div(dd_t x, dd_t y)
{
    double q1 = x.hi / y.hi;
    dd_t r = dd_sub(x, dd_mul(y, dd_d(q1)));
    double q2 = r.hi / y.hi;
    r = dd_sub(r, dd_mul(y, dd_d(q2)));
    double q3 = r.hi / y.hi;
    return dd_add(dd_fast_sum(q1, q2), dd_d(q3));
}

static dd_t dd_sqrt(dd_t a)
{
    if (a.hi <= 0.0) return dd_d(0.0);
    double s = sqrt(a.hi);
    dd_t r = dd_sub(a, dd_mul(dd_d(s), dd_d(s)));
    return dd_fast_sum(s, r.hi / (2.0 * s));
}

typedef struct { dd_t c[3]; } dd3_t;

static dd3_t dd3_of(const double *hi, const double *lo)
{
    dd3_t r;
    for (int k = 0; k < 3; k++) { r.c[k].hi = hi[k]; r.c[k].lo = lo ? lo[k] : 0.0; }
    return r;
}

static dd3_t dd3_sub(dd3_t a, dd3_t b)
{
    dd3_t r;
    for (int k = 0; k < 3; k++) r.c[k] = dd_sub(a.c[k], b.c[k]);
    return r;
}

static dd_t dd3_dot(dd3_t a, dd3_t b)
{
    return dd_add(dd_add(dd_mul(a.c[0], b.c[0]), dd_mul(a.c[1], b.c[1])), dd_mul(a.c[2], b.c[2]));
}

static dd3_t dd3_cross(dd3_t a, dd3_t b)
{
    dd3_t r;
    r.c[0] = dd_sub(dd_mul(a.c[1], b.c[2]), dd_mul(a.c[2], b.c[1]));
    r.c[1] = dd_sub(dd_mul(a.c[2], b.c[0]), dd_mul(a.c[0], b.c[2]));
    r.c[2] = dd_sub(dd_mul(a.c[0], b.c[1]), dd_mul(a.c[1], b.c[0]));
    return r;
}

static dd3_t dd3_unit(dd3_t a)
{
    dd_t r = dd_sqrt(dd3_dot(a, a));
    dd3_t o;
    for (int k = 0; k < 3; k++) o.c[k] = dd_div(a.c[k], r);
    return o;
}

static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* circumcentre of a facet on S^2: unit outward normal of its plane,
 * (b - a) x (c - a) with the base a taken opposite the longest edge (the two
 * shortest edges meet at the largest angle, >= 60 degrees, so the cross
 * product does not cancel even for near-coincident generators); ties go to
 * the smallest index.  Rotating (a,b,c) keeps the orientation. */
static void facet_vertex(const double *z, const int *v, double *out, double *outl)
{
    double L[3];
    for (int k = 0; k < 3; k++) { /* L[k]: squared length of the edge opposite v[k] */
        const double *p = z + 3 * (size_t)v[(k + 1) % 3], *q = z + 3 * (size_t)v[(k + 2) % 3];
        double d[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
        L[k] = dot3(d, d);
    }
    int r = 0;
    for (int k = 1; k < 3; k++)
        if (L[k] > L[r] || (L[k] == L[r] && v[k] < v[r])) r = k;
    const double *a = z + 3 * (size_t)v[r], *b = z + 3 * (size_t)v[(r + 1) % 3], *c = z + 3 * (size_t)v[(r + 2) % 3];
    /* in double-double: the differences are exact, the unit normal carries ~106 bits */
    dd3_t A = dd3_of(a, NULL), B = dd3_of(b, NULL), C = dd3_of(c, NULL);
    dd3_t nrm = dd3_unit(dd3_cross(dd3_sub(B, A), dd3_sub(C, A)));
    for (int k = 0; k < 3; k++) {
        out[k] = nrm.c[k].hi;
        outl[k] = nrm.c[k].lo;
    }
}

static int voronoi_from_hull(const hull_t *H, vor_t *V)
{
    int n = H->n;
    memset(V, 0, sizeof(*V));
    V->n = n;
    int *inc = (int *)malloc(sizeof(int) * n);      /* one incident facet per point */
    double *fv = (double *)malloc(sizeof(double) * 6 * (size_t)H->nf);  /* hi, then lo */
    V->off = (int *)malloc(sizeof(int) * (n + 1));
    if (!inc || !fv || !V->off) { free(inc); free(fv); return ORC_NOMEM; }
    for (int i = 0; i < n; i++) inc[i] = -1;
    for (int f = 0; f < H->nf; f++) {
        if (!H->f[f].alive) continue;
        facet_vertex(H->z, H->f[f].v, fv + 6 * (size_t)f, fv + 6 * (size_t)f + 3);
        for (int k = 0; k < 3; k++) inc[H->f[f].v[k]] = f;
    }
    /* degrees: walk around each point */
    V->off[0] = 0;
    for (int i = 0; i < n; i++) {
        if (inc[i] < 0) { free(inc); free(fv); return ORC_DEGENERATE; }
        int f = inc[i], d = 0;
        do {
            int k = (H->f[f].v[0] == i) ? 0 : (H->f[f].v[1] == i) ? 1 : 2;
            f = H->f[f].nb[(k + 2) % 3];
            d++;
            if (d > n) { free(inc); free(fv); return ORC_DEGENERATE; }
        } while (f != inc[i]);
        V->off[i + 1] = V->off[i] + d;
    }
    V->nbr = (int *)malloc(sizeof(int) * (size_t)V->off[n]);
    V->vx = (double *)malloc(sizeof(double) * 3 * (size_t)V->off[n]);
    V->vxl = (double *)malloc(sizeof(double) * 3 * (size_t)V->off[n]);
    if (!V->nbr || !V->vx || !V->vxl) { free(inc); free(fv); return ORC_NOMEM; }
    for (int i = 0; i < n; i++) {
        int f = inc[i], t = V->off[i];
        do {
            int k = (H->f[f].v[0] == i) ? 0 : (H->f[f].v[1] == i) ? 1 : 2;
            memcpy(V->vx + 3 * (size_t)t, fv + 6 * (size_t)f, sizeof(double) * 3);
            memcpy(V->vxl + 3 * (size_t)t, fv + 6 * (size_t)f + 3, sizeof(double) * 3);
            V->nbr[t] = H->f[f].v[(k + 2) % 3];
            f = H->f[f].nb[(k + 2) % 3];
            t++;
        } while (f != inc[i]);
    }
    free(inc);
    free(fv);
    return ORC_OK;
}

static int build_voronoi(int n, const double *z, vor_t *V)
{
    hull_t H;
    int rc = hull_build(&H, n, z);
    if (rc == ORC_OK) rc = voronoi_from_hull(&H, V);
    hull_free(&H);
    return rc;
}

/* Voronoi topology for the tests: degrees, CCW neighbour lists and corners.
 * deg[n]; nbr and vx must hold cap entries (cap >= 6n).  */
int orc_voronoi(int n, const double *z, int *deg, int *nbr, double *vx, int cap)
{
    vor_t V;
    int rc = build_voronoi(n, z, &V);
    if (rc != ORC_OK) return rc;
    if (V.off[n] > cap) { vor_free(&V); return ORC_INVALID; }
    for (int i = 0; i < n; i++) deg[i] = V.off[i + 1] - V.off[i];
    memcpy(nbr, V.nbr, sizeof(int) * (size_t)V.off[n]);
    if (vx) memcpy(vx, V.vx, sizeof(double) * 3 * (size_t)V.off[n]);
    vor_free(&V);
    return ORC_OK;
}

static double arc3(const double *a, const double *b)
{
    double c[3];
    cross3(a, b, c);
    return atan2(sqrt(dot3(c, c)), dot3(a, b));
}

static int cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

static int cmp_tri(const void *a, const void *b)
{
    const int *x = (const int *)a, *y = (const int *)b;
    for (int k = 0; k < 3; k++)
        if (x[k] != y[k]) return (x[k] > y[k]) - (x[k] < y[k]);
    return 0;
}

/* Bisection refinement (Sec. 4.3, the optimisation-bisection initialisation):
 * the n generators followed by the midpoints normalize(z_i + z_j) of the
 * Delaunay edges (i < j), in lexicographic (i, j) order.  *n_out = n + E. */
int orc_bisect(int n, const double *z, double *out, int cap, int *n_out)
{
    vor_t V;
    int rc = build_voronoi(n, z, &V);
    if (rc != ORC_OK) return rc;
    int m = n + V.off[n] / 2;
    if (m > cap) { vor_free(&V); return ORC_INVALID; }
    memcpy(out, z, sizeof(double) * 3 * (size_t)n);
    int t = n, js[256];
    for (int i = 0; i < n; i++) {
        int d = 0;
        for (int e = V.off[i]; e < V.off[i + 1]; e++)
            if (V.nbr[e] > i && d < 256) js[d++] = V.nbr[e];
        qsort(js, (size_t)d, sizeof(int), cmp_int);
        for (int k = 0; k < d; k++) {
            double mp[3];
            for (int c = 0; c < 3; c++) mp[c] = z[3 * (size_t)i + c] + z[3 * (size_t)js[k] + c];
            double r = sqrt(dot3(mp, mp));
            for (int c = 0; c < 3; c++) out[3 * (size_t)t + c] = mp[c] / r;
            t++;
        }
    }
    vor_free(&V);
    *n_out = t;
    return t == m ? ORC_OK : ORC_DEGENERATE;
}

/* Mesh quality measures (Sec. 4): cellQ(V) = min / max edge length of the
 * Voronoi cell, triQ = (a+b-c)(b+c-a)(c+a-b)/(abc) of a Delaunay triangle
 * with edge lengths a, b, c; lengths are great-circle arc lengths.  cellq:
 * n values (nullable); triq: the triangles ordered by their sorted vertex
 * triple (i < j < k), *n_tri of them (2n - 4). */
int orc_mesh_quality(int n, const double *z, double *cellq, double *triq, int tri_cap, int *n_tri)
{
    hull_t H;
    int rc = hull_build(&H, n, z);
    if (rc != ORC_OK) return rc;
    vor_t V;
    rc = voronoi_from_hull(&H, &V);
    if (rc != ORC_OK) { hull_free(&H); return rc; }
    if (cellq) {
        for (int i = 0; i < n; i++) {
            int d = V.off[i + 1] - V.off[i];
            double lo = INFINITY, hi = 0.0;
            for (int k = 0; k < d; k++) {
                const double *a = V.vx + 3 * (size_t)(V.off[i] + k);
                const double *b = V.vx + 3 * (size_t)(V.off[i] + (k + 1) % d);
                double L = arc3(a, b);
                if (L < lo) lo = L;
                if (L > hi) hi = L;
            }
            cellq[i] = lo / hi;
        }
    }
    int nt = 0;
    for (int f = 0; f < H.nf; f++)
        if (H.f[f].alive) nt++;
    int *tri = (int *)malloc(sizeof(int) * 3 * (size_t)(nt ? nt : 1));
    if (!tri) { vor_free(&V); hull_free(&H); return ORC_NOMEM; }
    int t = 0;
    for (int f = 0; f < H.nf; f++) {
        if (!H.f[f].alive) continue;
        int v[3] = {H.f[f].v[0], H.f[f].v[1], H.f[f].v[2]};
        qsort(v, 3, sizeof(int), cmp_int);
        memcpy(tri + 3 * (size_t)t, v, sizeof(v));
        t++;
    }
    qsort(tri, (size_t)nt, 3 * sizeof(int), cmp_tri);
    if (triq) {
        if (nt > tri_cap) { free(tri); vor_free(&V); hull_free(&H); return ORC_INVALID; }
        for (int k = 0; k < nt; k++) {
            const double *A = z + 3 * (size_t)tri[3 * k], *B = z + 3 * (size_t)tri[3 * k + 1];
            const double *Cp = z + 3 * (size_t)tri[3 * k + 2];
            double a = arc3(B, Cp), b = arc3(Cp, A), c = arc3(A, B);
            triq[k] = (a + b - c) * (b + c - a) * (c + a - b) / (a * b * c);
        }
    }
    if (n_tri) *n_tri = nt;
    free(tri);
    vor_free(&V);
    hull_free(&H);
    return ORC_OK;
}

/* ======================================================================
 * Point densities (Sec. 4)
 * ====================================================================== */

static double rho_eval(const orc_density *r, const double *p)
{
    switch (r->kind) {
    case 0:
        return 1.0;
    case 1: { /* X3: (1 - gamma) z^4 + gamma */
        double z2 = p[2] * p[2];
        return (1.0 - r->gamma) * z2 * z2 + r->gamma;
    }
    case 2:
    case 3: { /* tanh cap on the geodesic distance to x_c */
        double cr[3];
        cross3(p, r->xc, cr);
        double d = atan2(sqrt(dot3(cr, cr)), dot3(p, r->xc));
        /* (tanh(x) + 1)/2 written as 1/(1 + exp(-2x)): the same function
         * without the cancellation of tanh(x) + 1 for x << 0 */
        double x = (r->beta - d) / r->alpha;
        double v = (1.0 - r->gamma) / (1.0 + exp(-2.0 * x)) + r->gamma;
        if (r->kind == 3) { v = v * v; v = v * v; }
        return v;
    }
    default:
        return NAN;
    }
}

double orc_rho(const orc_density *r, const double *p) { return rho_eval(r, p); }

/* largest value of the density on S^2: 1 for rho = 1 and X3 (at the poles);
 * the tanh cap at its centre (d = 0), to the 4th power for that kind */
static double rho_max(const orc_density *r)
{
    if (r->kind == 0 || r->kind == 1) return 1.0;
    double v = (1.0 - r->gamma) / (1.0 + exp(-2.0 * r->beta / r->alpha)) + r->gamma;
    if (r->kind == 3) { v = v * v; v = v * v; }
    return v;
}

/* rho^e: e = 1 and e = 1/2 exactly, pow otherwise */
static double rho_pow(double v, double e)
{
    return e == 1.0 ? v : (e == 0.5 ? sqrt(v) : pow(v, e));
}

/* Monte Carlo initialisation by the density (Sec. 4.1): candidate k (a
 * uniform point on S^2) is kept when u_k rho_max^e <= rho(cand_k)^e, u_k
 * uniform on [0, 1); the first n_target kept candidates, in candidate order,
 * are the generators (e = 1: sampled by rho; e = 1/2: by the asymptotic CVT
 * point density rho^(1/2) of a surface).  Returns the number written (fewer
 * than n_target when the candidates run out). */
long long orc_sample_density(const orc_density *r, double e, const double *cand, const double *u, long long m,
                             long long n_target, double *z_out)
{
    const double rm = rho_pow(rho_max(r), e);
    long long k = 0;
    for (long long i = 0; i < m && k < n_target; i++) {
        if (u[i] * rm <= rho_pow(rho_eval(r, cand + 3 * i), e)) {
            for (int d = 0; d < 3; d++) z_out[3 * k + d] = cand[3 * i + d];
            k++;
        }
    }
    return k;
}

/* ======================================================================
 * Quadrature over signed spherical sub-triangles (Sec. 3.2.2)
 * ====================================================================== */

typedef struct {
    int nq;
    double bary[64][3];
    double w[64];     /* weights summing to 1 over the triangle */
    int exact_jac;    /* 0: area-scaled radial projection, 1: exact Jacobian */
    int fan;          /* 1: one triangle (z_i, v_a, v_b) per Voronoi edge instead of the
                         two sub-triangles through the Delaunay-edge midpoint */
} qrule_t;

/* 7-point degree-5 rule (Radon): centroid, and two orbits (a, a, 1-2a) with
 * a = (6 -+ sqrt 15)/21 */
static void rule_radon7(qrule_t *R)
{
    double s15 = sqrt(15.0);
    double a1 = (6.0 - s15) / 21.0, a2 = (6.0 + s15) / 21.0;
    double w1 = (155.0 - s15) / 1200.0, w2 = (155.0 + s15) / 1200.0;
    R->nq = 7;
    R->exact_jac = 0;
    R->fan = 0;
    R->bary[0][0] = R->bary[0][1] = R->bary[0][2] = 1.0 / 3.0;
    R->w[0] = 9.0 / 40.0;
    double orb[2][2] = {{a1, w1}, {a2, w2}};
    int k = 1;
    for (int o = 0; o < 2; o++)
        for (int r = 0; r < 3; r++) {
            double a = orb[o][0], b = 1.0 - 2.0 * a;
            R->bary[k][0] = (r == 0) ? b : a;
            R->bary[k][1] = (r == 1) ? b : a;
            R->bary[k][2] = (r == 2) ? b : a;
            R->w[k] = orb[o][1];
            k++;
        }
}

/* accumulate sum w rho, sum w rho p, sum w rho |p - zi|^2 over the signed
 * spherical triangle (a,b,c).  The corners are double-double; the area's
 * determinant and denominator, the rule points, their projection onto S^2
 * and the offsets p - zi are formed in double-double, then rounded (the
 * density and the sums are FP64). */
static void tri_accum(const qrule_t *R, const orc_density *rho, const double *zi,
                      dd3_t a, dd3_t b, dd3_t c, double *m, double *cm, double *e)
{
    const dd3_t Z = dd3_of(zi, NULL);
    /* signed spherical area: tan(E/2) = det[a,b,c] / (1 + a.b + b.c + c.a) */
    dd_t det = dd3_dot(a, dd3_cross(dd3_sub(b, a), dd3_sub(c, a)));
    dd_t den = dd_add(dd_add(dd_add(dd_d(1.0), dd3_dot(a, b)), dd3_dot(b, c)), dd3_dot(c, a));
    double A = 2.0 * atan2(det.hi, den.hi);
    for (int k = 0; k < R->nq; k++) {
        dd3_t x;
        for (int d = 0; d < 3; d++)
            x.c[d] = dd_add(dd_add(dd_mul(dd_d(R->bary[k][0]), a.c[d]), dd_mul(dd_d(R->bary[k][1]), b.c[d])),
                            dd_mul(dd_d(R->bary[k][2]), c.c[d]));
        dd_t r = dd_sqrt(dd3_dot(x, x));
        dd3_t pp;
        for (int d = 0; d < 3; d++) pp.c[d] = dd_div(x.c[d], r);
        double p[3] = {pp.c[0].hi, pp.c[1].hi, pp.c[2].hi};
        double wk = R->exact_jac ? R->w[k] * det.hi / (2.0 * r.hi * r.hi * r.hi) : R->w[k] * A;
        double rv = rho_eval(rho, p);
        dd3_t dp = dd3_sub(pp, Z);
        double dp2 = dd3_dot(dp, dp).hi;
        *m += wk * rv;
        cm[0] += wk * rv * p[0];
        cm[1] += wk * rv * p[1];
        cm[2] += wk * rv * p[2];
        *e += wk * rv * dp2;
    }
}

static void cell_integrals(const vor_t *V, const double *z, int i, const qrule_t *R, const orc_density *rho,
                           double *m, double *cm, double *e)
{
    const double *zi = z + 3 * (size_t)i;
    const dd3_t Zi = dd3_of(zi, NULL);
    int b0 = V->off[i], d = V->off[i + 1] - V->off[i];
    *m = 0; cm[0] = cm[1] = cm[2] = 0; *e = 0;
    for (int t = 0; t < d; t++) {
        const size_t ka = 3 * (size_t)(b0 + t), kb = 3 * (size_t)(b0 + (t + 1) % d);
        const dd3_t va = dd3_of(V->vx + ka, V->vxl + ka);
        const dd3_t vb = dd3_of(V->vx + kb, V->vxl + kb);
        if (R->fan) {
            tri_accum(R, rho, zi, Zi, va, vb, m, cm, e);
            continue;
        }
        /* Delaunay-edge midpoint normalize(z_i + z_j): the sum is exact in double-double */
        const double *zj = z + 3 * (size_t)V->nbr[b0 + t];
        dd3_t s;
        for (int k = 0; k < 3; k++) s.c[k] = dd_two_sum(zi[k], zj[k]);
        const dd3_t mu = dd3_unit(s);
        tri_accum(R, rho, zi, Zi, va, mu, m, cm, e);
        tri_accum(R, rho, zi, Zi, mu, vb, m, cm, e);
    }
}

/* pairwise (cascade) summation */
static double psum(const double *x, size_t n, size_t stride)
{
    if (n <= 8) {
        double s = 0;
        for (size_t i = 0; i < n; i++) s += x[i * stride];
        return s;
    }
    size_t h = n / 2;
    return psum(x, h, stride) + psum(x + h * stride, n - h, stride);
}

static double pdot(const double *a, const double *b, size_t n)
{
    double *t = (double *)malloc(sizeof(double) * (n ? n : 1));
    for (size_t i = 0; i < n; i++) t[i] = a[i] * b[i];
    double s = psum(t, n, 1);
    free(t);
    return s;
}

typedef struct {
    double F;       /* total energy */
    double gnorm;   /* ||g||_2 over all 3n components */
} orc_eval_out;

/* Full evaluation of Sec. 3.1 quantities.  Any output pointer may be NULL.
 * rule: NULL = Radon 7-point with area scaling. */
static int eval_all(int n, const double *z, const orc_density *rho, const qrule_t *rule,
                    double *F, double *g, double *h, double *m, double *c, double *Fi,
                    double *gnorm, int *deg_out, int nthreads)
{
    qrule_t R7;
    if (!rule) { rule_radon7(&R7); rule = &R7; }
    vor_t V;
    int rc = build_voronoi(n, z, &V);
    if (rc != ORC_OK) return rc;
    double *mm = (double *)malloc(sizeof(double) * n);
    double *cc = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *ee = (double *)malloc(sizeof(double) * n);
    double *gg = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    if (!mm || !cc || !ee || !gg) { free(mm); free(cc); free(ee); free(gg); vor_free(&V); return ORC_NOMEM; }
    int bad = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads) reduction(| : bad)
#endif
    for (int i = 0; i < n; i++) {
        double mi, ci[3], ei;
        cell_integrals(&V, z, i, rule, rho, &mi, ci, &ei);
        const double *zi = z + 3 * (size_t)i;
        double cz = dot3(ci, zi);
        mm[i] = mi;
        cc[3 * (size_t)i] = ci[0]; cc[3 * (size_t)i + 1] = ci[1]; cc[3 * (size_t)i + 2] = ci[2];
        ee[i] = ei;
        for (int d = 0; d < 3; d++) gg[3 * (size_t)i + d] = 2.0 * cz * zi[d] - 2.0 * ci[d];
        if (!(cz > 0)) bad = 1;
        if (h) h[i] = 1.0 / (2.0 * cz);
    }
    (void)nthreads;
    if (F) *F = psum(ee, (size_t)n, 1);
    if (gnorm) *gnorm = sqrt(pdot(gg, gg, 3 * (size_t)n));
    if (g) memcpy(g, gg, sizeof(double) * 3 * (size_t)n);
    if (m) memcpy(m, mm, sizeof(double) * n);
    if (c) memcpy(c, cc, sizeof(double) * 3 * (size_t)n);
    if (Fi) memcpy(Fi, ee, sizeof(double) * n);
    if (deg_out) for (int i = 0; i < n; i++) deg_out[i] = V.off[i + 1] - V.off[i];
    free(mm); free(cc); free(ee); free(gg);
    vor_free(&V);
    return bad ? ORC_DEGENERATE : ORC_OK;
}

/* Exported evaluation.  rule_mode 0: Radon 7-point (the method's rule).
 * rule_mode | 4: the fan decomposition (one triangle per Voronoi edge).
 * rule_mode 1/2: caller-supplied rule (nq points, barycentric qb[nq*3], weights
 * qw[nq] summing to 1) with area scaling (1) or the exact Jacobian of the
 * radial projection det[a,b,c]/|x|^3 (2). */
int orc_energy_grad(int n, const double *z, const orc_density *rho, int rule_mode, int nq,
                    const double *qb, const double *qw, double *F, double *g, double *h,
                    double *m, double *c, double *Fi, double *gnorm, int nthreads)
{
    if (n < 4 || !z || !rho) return ORC_INVALID;
    qrule_t R, *rp = NULL;
    const int fan = (rule_mode & 4) != 0;
    rule_mode &= 3;
    if (rule_mode == 0 && fan) {
        rule_radon7(&R);
        R.fan = 1;
        rp = &R;
    }
    if (rule_mode != 0) {
        if (nq < 1 || nq > 64 || !qb || !qw) return ORC_INVALID;
        R.nq = nq;
        R.fan = fan;
        R.exact_jac = (rule_mode == 2);
        for (int k = 0; k < nq; k++) {
            R.bary[k][0] = qb[3 * k]; R.bary[k][1] = qb[3 * k + 1]; R.bary[k][2] = qb[3 * k + 2];
            R.w[k] = qw[k];
        }
        rp = &R;
    }
    return eval_all(n, z, rho, rp, F, g, h, m, c, Fi, gnorm, NULL, nthreads);
}

/* Lloyd map (Sec. 2.2.1 on S^2): z_i <- c_i / |c_i| */
int orc_lloyd_step(int n, const double *z, const orc_density *rho, double *zout, int nthreads)
{
    double *c = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    if (!c) return ORC_NOMEM;
    int rc = eval_all(n, z, rho, NULL, NULL, NULL, NULL, NULL, c, NULL, NULL, NULL, nthreads);
    if (rc == ORC_OK)
        for (int i = 0; i < n; i++) {
            double *ci = c + 3 * (size_t)i;
            double r = sqrt(dot3(ci, ci));
            zout[3 * (size_t)i] = ci[0] / r;
            zout[3 * (size_t)i + 1] = ci[1] / r;
            zout[3 * (size_t)i + 2] = ci[2] / r;
        }
    free(c);
    return rc;
}

/* ======================================================================
 * LBFGS two-loop recursion (Sec. 2.2.2) with the boxed initial inverse
 * Hessian replaced by diag(h) (Sec. 3.1): q = -H g.
 * S, Y hold mcount pairs, oldest first, each of length 3n.
 * ====================================================================== */
/* h == NULL: the plain LBFGS initial matrix gamma I instead (Sec. 2.2.2) */
static int two_loop_h0(int n, const double *g, const double *h, double gamma, int mcount,
                       const double *S, const double *Y, double *q)
{
    size_t L = 3 * (size_t)n;
    double alpha[64], rho[64];
    if (mcount < 0 || mcount > 64) return ORC_INVALID;
    for (size_t k = 0; k < L; k++) q[k] = -g[k];
    for (int i = mcount - 1; i >= 0; i--) {
        const double *s = S + (size_t)i * L, *y = Y + (size_t)i * L;
        rho[i] = 1.0 / pdot(y, s, L);
        alpha[i] = rho[i] * pdot(s, q, L);
        for (size_t k = 0; k < L; k++) q[k] -= alpha[i] * y[k];
    }
    for (size_t k = 0; k < L; k++) q[k] *= h ? h[k / 3] : gamma;
    for (int i = 0; i < mcount; i++) {
        const double *s = S + (size_t)i * L, *y = Y + (size_t)i * L;
        double beta = rho[i] * pdot(y, q, L);
        for (size_t k = 0; k < L; k++) q[k] += s[k] * (alpha[i] - beta);
    }
    return ORC_OK;
}

int orc_two_loop(int n, const double *g, const double *h, int mcount,
                 const double *S, const double *Y, double *q)
{
    return two_loop_h0(n, g, h, 1.0, mcount, S, Y, q);
}

/* plain LBFGS (Sec. 2.2.2): H0 = gamma I, gamma = y.s / y.y of the newest
 * pair (the caller passes it; 1 with an empty history) */
int orc_two_loop_scalar(int n, const double *g, double gamma, int mcount,
                        const double *S, const double *Y, double *q)
{
    return two_loop_h0(n, g, NULL, gamma, mcount, S, Y, q);
}

/* ======================================================================
 * More-Thuente line search (More & Thuente 1994), written from the paper's
 * description: sufficient decrease + curvature (strong Wolfe), interval
 * updating with cubic / quadratic / secant safeguarded steps, the modified
 * function psi in the first stage, bisection when the bracket shrinks slowly.
 * ====================================================================== */

typedef int (*orc_phi_fn)(void *ctx, double a, double *f, double *g);

/* minimiser of the cubic interpolating (u,fu,du), (v,fv,dv) */
static double cubic_min(double u, double fu, double du, double v, double fv, double dv, int *ok)
{
    double d1 = du + dv - 3.0 * (fu - fv) / (u - v);
    double disc = d1 * d1 - du * dv;
    *ok = disc >= 0.0;
    if (disc < 0.0) disc = 0.0;
    double d2 = sqrt(disc);
    if (v < u) d2 = -d2;
    double den = dv - du + 2.0 * d2;
    if (den == 0.0) { *ok = 0; return u; }
    return v - (v - u) * (dv + d2 - d1) / den;
}

typedef struct {
    double x, fx, dx;   /* best step */
    double y, fy, dy;   /* other end of the interval */
    int brackt;
} mt_state;

static double mt_step(mt_state *S, double t, double ft, double dt, double tmin, double tmax)
{
    double newt;
    double sdx = (double)((S->dx > 0.0) - (S->dx < 0.0));
    double sgn = (dt * sdx < 0.0) ? -1.0 : 1.0; /* -1: derivatives differ in sign */
    int ok;
    if (ft > S->fx) {
        /* case 1: higher function value -- the minimum is bracketed */
        double tc = cubic_min(S->x, S->fx, S->dx, t, ft, dt, &ok);
        double tq = S->x + (S->dx / ((S->fx - ft) / (t - S->x) + S->dx)) / 2.0 * (t - S->x);
        newt = (fabs(tc - S->x) < fabs(tq - S->x)) ? tc : tc + (tq - tc) / 2.0;
        S->brackt = 1;
    } else if (sgn < 0) {
        /* case 2: lower value, derivatives of opposite sign -- bracketed */
        double tc = cubic_min(S->x, S->fx, S->dx, t, ft, dt, &ok);
        double ts = t + dt / (dt - S->dx) * (S->x - t);
        newt = (fabs(tc - t) > fabs(ts - t)) ? tc : ts;
        S->brackt = 1;
    } else if (fabs(dt) < fabs(S->dx)) {
        /* case 3: lower value, same sign, derivative magnitude decreases */
        double tc = cubic_min(S->x, S->fx, S->dx, t, ft, dt, &ok);
        int toward = ok && ((t > S->x) ? (tc > t) : (tc < t));
        if (!toward) tc = (t > S->x) ? tmax : tmin;
        double ts = t + dt / (dt - S->dx) * (S->x - t);
        if (S->brackt) {
            newt = (fabs(tc - t) < fabs(ts - t)) ? tc : ts;
            if (t > S->x) newt = fmin(t + 0.66 * (S->y - t), newt);
            else newt = fmax(t + 0.66 * (S->y - t), newt);
        } else {
            newt = (fabs(tc - t) > fabs(ts - t)) ? tc : ts;
            newt = fmin(tmax, fmax(tmin, newt));
        }
    } else {
        /* case 4: lower value, same sign, derivative does not decrease */
        if (S->brackt) newt = cubic_min(t, ft, dt, S->y, S->fy, S->dy, &ok);
        else newt = (t > S->x) ? tmax : tmin;
    }
    /* update the interval */
    if (ft > S->fx) {
        S->y = t; S->fy = ft; S->dy = dt;
    } else {
        if (sgn < 0) { S->y = S->x; S->fy = S->fx; S->dy = S->dx; }
        S->x = t; S->fx = ft; S->dx = dt;
    }
    return newt;
}

typedef struct {
    double ftol, gtol, xtol, stpmin, stpmax;
    int maxfev;
} mt_opts;

/* info: 1 converged (strong Wolfe), 2 interval too small, 3 maxfev,
 * 4 at stpmin, 5 at stpmax, 6 rounding prevents progress, <0 callback error.
 * On return *stp, *f, *g hold the last evaluated point. */
static int mt_search(orc_phi_fn phi, void *ctx, double f0, double g0, const mt_opts *o,
                     double *stp, double *f, double *g, int *nfev)
{
    if (!(g0 < 0.0) || !(*stp > 0.0)) return 7;
    mt_state S = {0.0, f0, g0, 0.0, f0, g0, 0};
    int stage1 = 1, info = 0;
    double gtest = o->ftol * g0;
    double width = o->stpmax - o->stpmin, width1 = 2.0 * width;
    double tmin = 0.0, tmax = *stp + 4.0 * *stp;
    double t = *stp;
    double cap = INFINITY; /* smallest step whose trial point was not a tessellation */
    *nfev = 0;
    for (;;) {
        t = fmax(t, o->stpmin);
        t = fmin(t, o->stpmax);
        if (t >= cap) t = S.x + 0.5 * (cap - S.x);
        if ((S.brackt && (t <= tmin || t >= tmax)) || *nfev >= o->maxfev - 1 ||
            (S.brackt && tmax - tmin <= o->xtol * tmax))
            t = S.x; /* an unusual end is coming: evaluate the best step */
        double ft, dt;
        int cb = phi(ctx, t, &ft, &dt);
        (*nfev)++;
        *stp = t; *f = ft; *g = dt;
        if (cb == 2) {
            /* invalid trial point: halve the step toward the best one */
            *f = INFINITY;
            if (*nfev >= o->maxfev) return 3;
            cap = t;
            t = S.x + 0.5 * (t - S.x);
            continue;
        }
        if (cb != 0) return -1;
        double ftest = f0 + t * gtest;
        if ((S.brackt && (t <= tmin || t >= tmax))) info = 6;
        if (t == o->stpmax && ft <= ftest && dt <= gtest) info = 5;
        if (t == o->stpmin && (ft > ftest || dt >= gtest)) info = 4;
        if (*nfev >= o->maxfev) info = 3;
        if (S.brackt && tmax - tmin <= o->xtol * tmax) info = 2;
        if (ft <= ftest && fabs(dt) <= o->gtol * (-g0)) info = 1;
        if (info) return info;
        if (stage1 && ft <= ftest && dt >= fmin(o->ftol, o->gtol) * g0) stage1 = 0;
        double nt;
        if (stage1 && ft <= S.fx && ft > ftest) {
            /* modified function psi(a) = phi(a) - phi(0) - ftol a phi'(0) */
            mt_state M = S;
            M.fx = S.fx - S.x * gtest; M.dx = S.dx - gtest;
            M.fy = S.fy - S.y * gtest; M.dy = S.dy - gtest;
            nt = mt_step(&M, t, ft - t * gtest, dt - gtest, tmin, tmax);
            S.brackt = M.brackt;
            S.x = M.x; S.fx = M.fx + M.x * gtest; S.dx = M.dx + gtest;
            S.y = M.y; S.fy = M.fy + M.y * gtest; S.dy = M.dy + gtest;
        } else {
            nt = mt_step(&S, t, ft, dt, tmin, tmax);
        }
        if (S.brackt) {
            if (fabs(S.y - S.x) >= 0.66 * width1) nt = S.x + 0.5 * (S.y - S.x);
            width1 = width;
            width = fabs(S.y - S.x);
            tmin = fmin(S.x, S.y);
            tmax = fmax(S.x, S.y);
        } else {
            tmin = S.x;
            tmax = nt + 4.0 * (nt - S.x);
        }
        t = nt;
    }
}

/* exported for the line-search pins: phi is a C callback */
int orc_line_search(orc_phi_fn phi, void *ctx, double f0, double g0, double stp0,
                    double ftol, double gtol, double xtol, double stpmin, double stpmax, int maxfev,
                    double *stp, double *f, double *g, int *nfev)
{
    mt_opts o = {ftol, gtol, xtol, stpmin, stpmax, maxfev};
    *stp = stp0;
    return mt_search(phi, ctx, f0, g0, &o, stp, f, g, nfev);
}

/* ======================================================================
 * Lloyd-preconditioned LBFGS on S^2 (Sec. 3.1; the serial core of the
 * parallel algorithm of Sec. 3.3 without communication)
 * ====================================================================== */

typedef struct {
    int max_iter;
    double grad_tol, rel_grad_tol, rel_df_tol, step_tol;
    int ls_max_evals;
    double c1, c2;
    int lbfgs_m;
    int nthreads;
    int method;  /* 0 Lloyd-preconditioned LBFGS, 1 LBFGS with gamma_n I, 2 Lloyd */
} orc_opts;

typedef struct {
    int iters, fevals, resets, skipped;
    double energy, grad_norm;
    int converged, status;
} orc_report;

typedef struct {
    int n;
    const double *z;     /* base point */
    const double *q;     /* direction */
    const orc_density *rho;
    double *zt, *gt, *ht; /* trial point and its gradient / preconditioner */
    double Ft;
    int nthreads;
    int rc;
} ls_ctx;

static int phi_eval(void *vctx, double a, double *f, double *dphi)
{
    ls_ctx *C = (ls_ctx *)vctx;
    int n = C->n;
    double *nrm = (double *)malloc(sizeof(double) * n);
    double *tmp = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    if (!nrm || !tmp) { free(nrm); free(tmp); C->rc = ORC_NOMEM; return 1; }
    for (int i = 0; i < n; i++) {
        double x[3];
        for (int d = 0; d < 3; d++) x[d] = C->z[3 * (size_t)i + d] + a * C->q[3 * (size_t)i + d];
        double r = sqrt(dot3(x, x));
        nrm[i] = r;
        for (int d = 0; d < 3; d++) C->zt[3 * (size_t)i + d] = x[d] / r;
    }
    int rc = eval_all(n, C->zt, C->rho, NULL, &C->Ft, C->gt, C->ht, NULL, NULL, NULL, NULL, NULL, C->nthreads);
    if (rc == ORC_DEGENERATE || rc == ORC_INVALID) { free(nrm); free(tmp); return 2; } /* not a tessellation */
    if (rc != ORC_OK) { free(nrm); free(tmp); C->rc = rc; return 1; }
    for (int i = 0; i < n; i++)
        for (int d = 0; d < 3; d++)
            tmp[3 * (size_t)i + d] = C->gt[3 * (size_t)i + d] * C->q[3 * (size_t)i + d] / nrm[i];
    *f = C->Ft;
    *dphi = psum(tmp, 3 * (size_t)n, 1);
    free(nrm);
    free(tmp);
    return 0;
}

/* Per-iteration trace (optional, arrays of length >= max_iter):
 * energy after the iteration, ||g|| after, accepted step, evaluations used.
 * method 0: the Lloyd-preconditioned LBFGS (Sec. 3.1); method 1: LBFGS with
 * H0 = gamma_n I, gamma_n = y.s / y.y of the newest stored pair and H0 = I
 * with an empty memory (Sec. 2.2.2); method 2: Lloyd's iteration (Sec. 2.2.1)
 * written as the step alpha = 1 along the Lloyd direction q = -h g, whose
 * trial point normalize(z - h g) = c / |c| (since z - h g = c / (c.z)), with
 * no line search and no memory. */
int orc_lbfgs_solve(int n, double *z, const orc_density *rho, const orc_opts *o, orc_report *rep,
                    double *tr_F, double *tr_g, double *tr_a, int *tr_nfev)
{
    size_t L = 3 * (size_t)n;
    int M = o->lbfgs_m;
    memset(rep, 0, sizeof(*rep));
    if (n < 4 || M < 0 || M > 64 || o->method < 0 || o->method > 2) return ORC_INVALID;
    if (o->method == 2) M = 0;
    double *g = (double *)malloc(sizeof(double) * L);
    double *h = (double *)malloc(sizeof(double) * n);
    double *q = (double *)malloc(sizeof(double) * L);
    double *zt = (double *)malloc(sizeof(double) * L);
    double *gt = (double *)malloc(sizeof(double) * L);
    double *ht = (double *)malloc(sizeof(double) * n);
    double *S = (double *)malloc(sizeof(double) * L * (M ? M : 1));
    double *Y = (double *)malloc(sizeof(double) * L * (M ? M : 1));
    double *tmp = (double *)malloc(sizeof(double) * L);
    int rc = ORC_OK;
    if (!g || !h || !q || !zt || !gt || !ht || !S || !Y || !tmp) { rc = ORC_NOMEM; goto out; }
    double F;
    rc = eval_all(n, z, rho, NULL, &F, g, h, NULL, NULL, NULL, NULL, NULL, o->nthreads);
    rep->fevals = 1;
    if (rc != ORC_OK) goto out;
    int hist = 0;
    double gamma = 1.0;  /* method 1: y.s / y.y of the newest stored pair */
    mt_opts mo = {o->c1, o->c2, 1e-16, 1e-20, 1e20, o->ls_max_evals};
    double Fprev = F;
    for (;;) {
        double gn = sqrt(pdot(g, g, L));
        rep->energy = F;
        rep->grad_norm = gn;
        if (gn <= o->grad_tol) { rep->converged = 1; break; }
        if (o->rel_grad_tol > 0 && gn / F <= o->rel_grad_tol) { rep->converged = 1; break; }
        if (rep->iters > 0 && o->rel_df_tol > 0 && fabs(F - Fprev) / Fprev < o->rel_df_tol) { rep->converged = 1; break; }
        if (rep->iters >= o->max_iter) break;
        if (o->method == 1) two_loop_h0(n, g, NULL, hist ? gamma : 1.0, hist, S, Y, q);
        else orc_two_loop(n, g, h, hist, S, Y, q);
        double d0 = pdot(g, q, L);
        if (!(d0 < 0.0)) {
            hist = 0;
            rep->resets++;
            if (o->method == 1) two_loop_h0(n, g, NULL, 1.0, 0, S, Y, q);
            else orc_two_loop(n, g, h, 0, S, Y, q);
            d0 = pdot(g, q, L);
            if (!(d0 < 0.0)) { rc = ORC_DEGENERATE; break; }
        }
        ls_ctx C = {n, z, q, rho, zt, gt, ht, 0.0, o->nthreads, ORC_OK};
        double a = 1.0, fa, ga;
        int nfev = 0;
        int info;
        if (o->method == 2) {
            /* Lloyd: the trial point at alpha = 1, accepted as it is */
            int cb = phi_eval(&C, 1.0, &fa, &ga);
            nfev = 1;
            if (cb == 2) { rep->fevals += 1; rc = ORC_DEGENERATE; break; }
            info = cb ? -1 : 1;
        } else {
            info = mt_search(phi_eval, &C, F, d0, &mo, &a, &fa, &ga, &nfev);
        }
        rep->fevals += nfev;
        if (info < 0) { rc = C.rc; break; }
        if (info != 1) {
            if (!(fa < F)) {
                if (hist == 0) { rc = ORC_LINESEARCH; break; }
                hist = 0;
                rep->resets++;
                continue;
            }
            hist = 0; /* accept the best point but restart the memory */
            rep->resets++;
        }
        /* accept: s = z+ - z, y = g+ - g */
        double maxmove = 0.0;
        double *s_new = tmp;
        for (size_t k = 0; k < L; k++) s_new[k] = zt[k] - z[k];
        for (int i = 0; i < n; i++) {
            double mv = sqrt(dot3(s_new + 3 * (size_t)i, s_new + 3 * (size_t)i));
            if (mv > maxmove) maxmove = mv;
        }
        double *y_new = q; /* q is no longer needed */
        for (size_t k = 0; k < L; k++) y_new[k] = gt[k] - g[k];
        double ys = pdot(y_new, s_new, L);
        double yy = sqrt(pdot(y_new, y_new, L)), ss = sqrt(pdot(s_new, s_new, L));
        if (M > 0 && ys > 1e-12 * yy * ss) {
            if (hist == M) {
                memmove(S, S + L, sizeof(double) * L * (M - 1));
                memmove(Y, Y + L, sizeof(double) * L * (M - 1));
                hist--;
            }
            memcpy(S + L * hist, s_new, sizeof(double) * L);
            memcpy(Y + L * hist, y_new, sizeof(double) * L);
            hist++;
            gamma = ys / pdot(y_new, y_new, L);
        } else if (o->method != 2) {
            rep->skipped++;
        }
        memcpy(z, zt, sizeof(double) * L);
        memcpy(g, gt, sizeof(double) * L);
        memcpy(h, ht, sizeof(double) * n);
        Fprev = F;
        F = fa;
        if (tr_F) tr_F[rep->iters] = F;
        if (tr_g) tr_g[rep->iters] = sqrt(pdot(g, g, L));
        if (tr_a) tr_a[rep->iters] = a;
        if (tr_nfev) tr_nfev[rep->iters] = nfev;
        rep->iters++;
        if (o->step_tol > 0 && maxmove <= o->step_tol) {
            rep->energy = F;
            rep->grad_norm = sqrt(pdot(g, g, L));
            rep->converged = 1;
            break;
        }
    }
out:
    rep->status = rc;
    free(g); free(h); free(q); free(zt); free(gt); free(ht); free(S); free(Y); free(tmp);
    return rc;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
