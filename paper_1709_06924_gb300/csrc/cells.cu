// cells.cu -- spherical Voronoi cells and their integrals, one thread per
// generator.
//
// Per evaluation:
//   1. cube-map binning: face = argmax |z_k|, (s, t) = the other two
//      coordinates over |z_face|, G x G bins per face, counting sort, each
//      bin ordered by coordinates;
//   2. per generator z_i: its K nearest neighbours by chord distance, found by
//      a complete cap query over the bins (every point within the cap's chord
//      radius is seen, so "not kept" implies "at least d_K away");
//   3. the cell V_i = {x in S^2 : x.(z_i - z_j) >= 0 for all j} (Sec. 2.1,
//      Euclidean distance on the sphere) is clipped in the gnomonic plane at
//      z_i, where each bisector great circle is a straight line; neighbours
//      are taken nearest first and clipping stops once the next neighbour is
//      farther than twice the largest vertex distance (security radius).  A
//      cell that cannot be certified is queued for a pass with more
//      neighbours;
//   4. the cell is integrated over the paper's signed sub-triangles (Sec.
//      3.2.2: generator, Delaunay-edge midpoint normalize(z_i+z_j), Voronoi
//      vertex) with the 7-point degree-5 rule mapped radially to the sphere,
//      weights scaled by the signed spherical area (Van Oosterom-Strackee);
//   5. g_i = 2 (c_i.z_i) z_i - 2 c_i and h_i = 1/(2 c_i.z_i) (Sec. 3.1).
// Results are written at the generator's original index, so that every
// later reduction runs in index order and is independent of the binning.
#include <math.h>

#include "scvt_internal.cuh"

namespace scvt {

namespace {

constexpr double kBoxL = 1.0e3;         // half-width of the starting square (gnomonic)
constexpr double kCertMargin = 1.0 + 1e-9;

// Radon's 7-point degree-5 rule: centroid (weight 9/40) and the orbits
// (a, a, 1 - 2a) with a = (6 -+ sqrt 15)/21, weights (155 -+ sqrt 15)/1200.
__constant__ double kQb[7][3] = {
    {1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0},
    {0.7974269853530873224, 0.1012865073234563388, 0.1012865073234563388},
    {0.1012865073234563388, 0.7974269853530873224, 0.1012865073234563388},
    {0.1012865073234563388, 0.1012865073234563388, 0.7974269853530873224},
    {0.059715871789769820459, 0.47014206410511508977, 0.47014206410511508977},
    {0.47014206410511508977, 0.059715871789769820459, 0.47014206410511508977},
    {0.47014206410511508977, 0.47014206410511508977, 0.059715871789769820459},
};
__constant__ double kQw[7] = {0.225,
                              0.1259391805448271526, 0.1259391805448271526, 0.1259391805448271526,
                              0.13239415278850618074, 0.13239415278850618074, 0.13239415278850618074};

struct V3 {
    double x, y, z;
};
__device__ __forceinline__ V3 mk(double x, double y, double z) { return V3{x, y, z}; }
__device__ __forceinline__ V3 sub(V3 a, V3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ V3 add(V3 a, V3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ V3 scl(V3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 crs(V3 a, V3 b) {
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ V3 unit(V3 a) { return scl(a, 1.0 / sqrt(dot(a, a))); }
__device__ __forceinline__ V3 ld(const P4 *p) {
    const P4 v = p[0];
    return mk(v.x, v.y, v.z);
}

__device__ __forceinline__ int bin_index(double x, double y, double z, int G) {
    double ax = fabs(x), ay = fabs(y), az = fabs(z);
    int a;
    double m, pb, pc;
    if (ax >= ay && ax >= az) { a = 0; m = x; pb = y; pc = z; }
    else if (ay >= az) { a = 1; m = y; pb = z; pc = x; }
    else { a = 2; m = z; pb = x; pc = y; }
    double am = fabs(m);
    double s = pb / am, t = pc / am;
    int iu = (int)floor((s + 1.0) * 0.5 * G);
    int iv = (int)floor((t + 1.0) * 0.5 * G);
    iu = min(max(iu, 0), G - 1);
    iv = min(max(iv, 0), G - 1);
    int face = 2 * a + (m < 0.0 ? 1 : 0);
    return (face * G + iv) * G + iu;
}

// ---------------------------------------------------------------- binning
__global__ void k_bin_count(const double *__restrict__ z, int n, int G, int *__restrict__ bin_of,
                            int *__restrict__ count, DevStatus *st) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = z[3 * (size_t)i], y = z[3 * (size_t)i + 1], w = z[3 * (size_t)i + 2];
    double r2 = x * x + y * y + w * w;
    if (!(fabs(r2 - 1.0) <= 2e-12)) {  // also catches NaN / inf
        atomicOr(&st->flags, FLAG_BAD_POINT);
        bin_of[i] = 0;
        atomicAdd(&count[0], 1);
        return;
    }
    int b = bin_index(x, y, w, G);
    bin_of[i] = b;
    atomicAdd(&count[b], 1);
}

__global__ void k_bin_scatter(const double *__restrict__ z, int n, const int *__restrict__ bin_of,
                              int *__restrict__ cursor, P4 *__restrict__ zs, float4 *__restrict__ zf,
                              int *__restrict__ sidx) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int pos = atomicAdd(&cursor[bin_of[i]], 1);
    sidx[pos] = i;
    double x = z[3 * (size_t)i], y = z[3 * (size_t)i + 1], w = z[3 * (size_t)i + 2];
    zs[pos] = P4{x, y, w, 0.0};
    zf[pos] = make_float4((float)x, (float)y, (float)w, 0.0f);
}

// Order each bin's generators by their coordinates (lexicographic x, y, z).
// The scatter above fills a bin in atomic order; sorting makes the bin
// layout a function of the point set alone, so every later step (kNN ties,
// the edge list of the quadrature and its reduction tree) is reproducible and
// independent of the input order.  Bins hold a few generators: insertion sort.
__global__ void k_bin_sort(const int *__restrict__ start, int nbins, P4 *__restrict__ zs, float4 *__restrict__ zf,
                           int *__restrict__ sidx) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    const int p0 = start[b], p1 = start[b + 1];
    for (int p = p0 + 1; p < p1; ++p) {
        const P4 v = zs[p];
        const float4 vf = zf[p];
        const int id = sidx[p];
        int q = p;
        while (q > p0) {
            const P4 u = zs[q - 1];
            const bool greater = u.x > v.x || (u.x == v.x && (u.y > v.y || (u.y == v.y && u.z > v.z)));
            if (!greater) break;
            zs[q] = u;
            zf[q] = zf[q - 1];
            sidx[q] = sidx[q - 1];
            --q;
        }
        zs[q] = v;
        zf[q] = vf;
        sidx[q] = id;
    }
}

// exclusive scan of 2048-element tiles; writes tile totals
__global__ void k_scan_tiles(const int *__restrict__ in, int *__restrict__ out, int len, int *__restrict__ totals) {
    __shared__ int warp_sums[32];
    int base = blockIdx.x * 2048;
    int t = threadIdx.x;  // 1024 threads, 2 elements each
    int i0 = base + 2 * t, i1 = i0 + 1;
    int v0 = (i0 < len) ? in[i0] : 0;
    int v1 = (i1 < len) ? in[i1] : 0;
    int s = v0 + v1;
    int lane = t & 31, w = t >> 5;
    int incl = s;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[w] = incl;
    __syncthreads();
    if (w == 0) {
        int ws = warp_sums[lane];
        int wi = ws;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        warp_sums[lane] = wi - ws;  // exclusive
    }
    __syncthreads();
    int excl = warp_sums[w] + incl - s;
    if (i0 < len) out[i0] = excl;
    if (i1 < len) out[i1] = excl + v0;
    if (t == 1023 && totals) totals[blockIdx.x] = excl + s;
}

__global__ void k_scan_add(int *__restrict__ out, int len, const int *__restrict__ offs) {
    int i = blockIdx.x * 2048 + threadIdx.x * 2;
    int add = offs[blockIdx.x];
    if (i < len) out[i] += add;
    if (i + 1 < len) out[i + 1] += add;
}

// recursive exclusive scan; tmp must hold sum over levels of ceil(len/2048)
void exclusive_scan(const int *in, int *out, int len, int *tmp, cudaStream_t s, int64_t *launches) {
    int tiles = (len + 2047) / 2048;
    if (tiles <= 1) {
        k_scan_tiles<<<1, 1024, 0, s>>>(in, out, len, nullptr);
        (*launches)++;
        return;
    }
    int *totals = tmp, *tot_scan = tmp + tiles;
    k_scan_tiles<<<tiles, 1024, 0, s>>>(in, out, len, totals);
    exclusive_scan(totals, tot_scan, tiles, tmp + 2 * tiles, s, launches);
    k_scan_add<<<tiles, 1024, 0, s>>>(out, len, tot_scan);
    (*launches) += 2;
}

__global__ void k_set_total(int *start, int nbins, int n) { start[nbins] = n; }

// ------------------------------------------------------------ k-nearest
// The neighbour search runs on FP32 copies of the coordinates (the FP32 pipe
// is ~70x the FP64 pipe on this part); it only has to produce candidates and a
// certified lower bound on the distance of every generator it did not keep.
// With coordinates rounded to FP32 (error <= 6e-8 each) and the FP32
// difference and squared norm, the true chord d of a scanned point satisfies
// d >= sqrt(d2f) (1 - 3e-7) - 4e-7; lower_d2() returns the square of that.
__device__ __forceinline__ double lower_d2(float d2f) {
    double d = sqrt((double)d2f) * (1.0 - 3e-7) - 4e-7;
    return d > 0.0 ? d * d : 0.0;
}

template <int K>
struct KnnList {
    float d[K];
    int j[K];
    int cnt;
    __device__ __forceinline__ void push(float d2, int jj) {
        if (cnt == K && (d2 > d[K - 1] || (d2 == d[K - 1] && jj > j[K - 1]))) return;
        int p = (cnt < K) ? cnt++ : K - 1;
        while (p > 0 && (d[p - 1] > d2 || (d[p - 1] == d2 && j[p - 1] > jj))) {
            d[p] = d[p - 1];
            j[p] = j[p - 1];
            --p;
        }
        d[p] = d2;
        j[p] = jj;
    }
};

__device__ __forceinline__ float4 ldf(const float4 *p) { return p[0]; }

// exact duplicate test on the FP64 coordinates for FP32 near-coincidences
__device__ __forceinline__ void check_duplicate(const Grid &g, V3 q, int p, unsigned *flags) {
    V3 d = sub(ld(g.zs + p), q);
    if (d.x == 0.0 && d.y == 0.0 && d.z == 0.0) atomicOr(flags, FLAG_DUPLICATE);
}

// Every generator p (bin order) within chord r of q, found through the bins
// that the cap {x : x.q >= cos theta} can reach (sin theta = S < 0.28), is
// scanned; those with d2f <= r2acc are offered to the list.  For face
// (a, sign) the values s = x_b / |x_a| attained in the cap lie between the
// roots of (q_b - s sign q_a)^2 = S^2 (1 + s^2): the planes of constant s are
// great circles through the c axis, and one meets the cap iff q's distance
// to it is at most S.
template <int K>
__device__ void cap_query(const Grid &g, V3 q, float4 qf, int self, double S, float r2acc, KnnList<K> &L,
                          unsigned *flags) {
    const double S2 = S * S;
    const double qv[3] = {q.x, q.y, q.z};
    for (int a = 0; a < 3; ++a) {
        double qa = qv[a];
        double A = qa * qa - S2;
        if (A <= 0.0) continue;  // the cap cannot reach face a (|x_a| >= 1/sqrt3 there)
        double sg = qa > 0.0 ? 1.0 : -1.0;
        int face = 2 * a + (qa < 0.0 ? 1 : 0);
        int lo[2], hi[2];
        bool empty = false;
        for (int r = 0; r < 2; ++r) {
            double qb = qv[(a + 1 + r) % 3];
            double disc = qa * qa + qb * qb - S2;
            double rt = S * sqrt(fmax(disc, 0.0));
            double s0 = (sg * qa * qb - rt) / A - 1e-9;
            double s1 = (sg * qa * qb + rt) / A + 1e-9;
            if (s0 > 1.0 || s1 < -1.0) { empty = true; break; }
            s0 = fmax(s0, -1.0);
            s1 = fmin(s1, 1.0);
            lo[r] = min(max((int)floor((s0 + 1.0) * 0.5 * g.G), 0), g.G - 1);
            hi[r] = min(max((int)floor((s1 + 1.0) * 0.5 * g.G), 0), g.G - 1);
        }
        if (empty) continue;
        for (int iv = lo[1]; iv <= hi[1]; ++iv) {
            int row = (face * g.G + iv) * g.G;
            int p0 = g.bstart[row + lo[0]], p1 = g.bstart[row + hi[0] + 1];
            for (int p = p0; p < p1; ++p) {
                if (p == self) continue;
                float4 c = ldf(g.zf + p);
                float dx = c.x - qf.x, dy = c.y - qf.y, dz = c.z - qf.z;
                float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if (d2 == 0.0f) check_duplicate(g, q, p, flags);
                if (d2 <= r2acc) L.push(d2, p);
            }
        }
    }
}

template <int K>
__device__ void all_query(const Grid &g, V3 q, float4 qf, int self, KnnList<K> &L, unsigned *flags) {
    for (int p = 0; p < g.n; ++p) {
        if (p == self) continue;
        float4 c = ldf(g.zf + p);
        float dx = c.x - qf.x, dy = c.y - qf.y, dz = c.z - qf.z;
        float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (d2 == 0.0f) check_duplicate(g, q, p, flags);
        L.push(d2, p);
    }
}

// ---------------------------------------------------------------- clipping
// Convex polygon in the gnomonic plane at z_i: edge k runs from vertex k to
// vertex k+1 on line ln[k] (a u + b w <= c).  Lines live in a side table:
// slots 0..K-1 follow the kNN list, K..K+3 are the starting square, and
// K+4.. hold generators met by the exhaustive last-resort scan (ids in jx).
// Each line is computed once in FP64 and kept with an FP32 copy.  Vertex k
// is the intersection of lines ln[k-1] and ln[k]; it is carried as an FP32
// approximation (uf, wf) with a flag `ill` when that 2x2 system is poorly
// conditioned.  Its FP64 value is only ever computed from its two lines
// (meet64), so the final corners do not depend on the order of clipping.
//
// Inside/outside decisions are filtered: the FP32 side value
// sd = a u + b w - c decides when |sd| > 2e-4 (|a u| + |b w| + |c|) and the
// vertex is well conditioned (|det| >= (|a1 b2| + |a2 b1|)/30).  FP32 lines
// carry a relative error of 6e-8 and the FP32 intersection an error of about
// kappa * 3e-7 of the vertex scale (kappa <= 30 here), so the FP32 side value
// is within 1e-5 of the magnitude and the filtered sign equals the FP64 sign.
// Every other decision is taken in FP64.
template <int K, int VMAX>
struct Poly {
    float uf[2][VMAX], wf[2][VMAX];
    unsigned char ln[2][VMAX];
    unsigned char ill[2][VMAX];
    double la[K + 4 + VMAX], lb[K + 4 + VMAX], lc[K + 4 + VMAX];
    float laf[K + 4 + VMAX], lbf[K + 4 + VMAX], lcf[K + 4 + VMAX];
    int jx[VMAX];
    int nv, cur;

    __device__ __forceinline__ void set_line(int l, double a, double b, double c) {
        la[l] = a; lb[l] = b; lc[l] = c;
        laf[l] = (float)a; lbf[l] = (float)b; lcf[l] = (float)c;
    }
    __device__ __forceinline__ void meet64(int l1, int l2, double &u, double &w) const {
        double inv = 1.0 / (la[l1] * lb[l2] - la[l2] * lb[l1]);
        u = (lc[l1] * lb[l2] - lc[l2] * lb[l1]) * inv;
        w = (la[l1] * lc[l2] - la[l2] * lc[l1]) * inv;
    }
    // FP32 intersection; returns true if it is ill conditioned
    __device__ __forceinline__ bool meet32(int l1, int l2, float &u, float &w) const {
        float p1 = laf[l1] * lbf[l2], p2 = laf[l2] * lbf[l1];
        float det = p1 - p2;
        u = (lcf[l1] * lbf[l2] - lcf[l2] * lbf[l1]) / det;
        w = (laf[l1] * lcf[l2] - laf[l2] * lcf[l1]) / det;
        return !(fabsf(det) * 30.0f >= fabsf(p1) + fabsf(p2));
    }
};

__device__ __forceinline__ double chord2_of_r2(double r2) {
    // |normalize(z_i + u e1 + w e2) - z_i|^2 = 2 - 2/sqrt(1 + r^2), without cancellation
    double q = sqrt(1.0 + r2);
    return 2.0 * r2 / (q * (1.0 + q));
}

// clip by line slot l; returns 1 if the polygon changed, 0 if not, -1 on
// capacity / empty errors
template <int K, int VMAX>
__device__ int clip(Poly<K, VMAX> &P, int l, unsigned *flags, unsigned long long *amb) {
    const int c0 = P.cur, nv = P.nv;
    const float laf = P.laf[l], lbf = P.lbf[l], lcf = P.lcf[l];
    unsigned long long out = 0ull;
    int namb = 0;
    for (int k = 0; k < nv; ++k) {
        const float uk = P.uf[c0][k], wk = P.wf[c0][k];
        const float sd = fmaf(laf, uk, fmaf(lbf, wk, -lcf));
        const float mag = fabsf(laf * uk) + fabsf(lbf * wk) + fabsf(lcf);
        bool outside;
        if (!P.ill[c0][k] && fabsf(sd) > 2e-4f * mag) {
            outside = sd > 0.0f;
        } else {
            const int kp = (k == 0) ? nv - 1 : k - 1;
            double u, w;
            P.meet64(P.ln[c0][kp], P.ln[c0][k], u, w);
            const double la = P.la[l], lb = P.lb[l], lc = P.lc[l];
            const double sd64 = la * u + lb * w - lc;
            if (fabs(sd64) <= 1e-14 * (fabs(la * u) + fabs(lb * w) + fabs(lc))) ++namb;
            outside = sd64 > 0.0;
        }
        if (outside) out |= (1ull << k);
    }
    if (namb) atomicAdd(amb, (unsigned long long)namb);
    if (!out) return 0;
    unsigned long long full = (nv == 64) ? ~0ull : ((1ull << nv) - 1ull);
    if (out == full) {
        atomicOr(flags, FLAG_EMPTY);
        return -1;
    }
    // the outside vertices form one cyclic run k0..k1 (convexity)
    int k0 = -1, runs = 0;
    for (int k = 0; k < nv; ++k) {
        int prev = (k == 0) ? nv - 1 : k - 1;
        if (((out >> k) & 1ull) && !((out >> prev) & 1ull)) {
            if (k0 < 0) k0 = k;
            ++runs;
        }
    }
    if (runs > 1) atomicOr(flags, FLAG_NONCONVEX);
    int k1 = k0, runlen = 1;
    while (true) {
        int nx = (k1 + 1 == nv) ? 0 : k1 + 1;
        if (!((out >> nx) & 1ull)) break;
        k1 = nx;
        ++runlen;
    }
    int nnew = nv - runlen + 2;
    if (nnew > VMAX) return -1;
    const int c1 = c0 ^ 1;
    const int kin = (k0 == 0) ? nv - 1 : k0 - 1;  // last inside vertex before the run
    const int lin = P.ln[c0][kin], lout = P.ln[c0][k1];
    float pu, pw, qu, qw;
    bool pill = P.meet32(lin, l, pu, pw);
    bool qill = P.meet32(l, lout, qu, qw);
    P.uf[c1][0] = pu; P.wf[c1][0] = pw; P.ln[c1][0] = (unsigned char)l; P.ill[c1][0] = pill;
    P.uf[c1][1] = qu; P.wf[c1][1] = qw; P.ln[c1][1] = (unsigned char)lout; P.ill[c1][1] = qill;
    int o = 2;
    int k = (k1 + 1 == nv) ? 0 : k1 + 1;
    for (int cnt = 0; cnt < nv - runlen; ++cnt) {
        P.uf[c1][o] = P.uf[c0][k];
        P.wf[c1][o] = P.wf[c0][k];
        P.ln[c1][o] = P.ln[c0][k];
        P.ill[c1][o] = P.ill[c0][k];
        ++o;
        k = (k + 1 == nv) ? 0 : k + 1;
    }
    P.nv = nnew;
    P.cur = c1;
    return 1;
}

// an upper bound of the largest squared chord from z_i to a vertex
template <int K, int VMAX>
__device__ __forceinline__ double poly_R2(const Poly<K, VMAX> &P) {
    const int c = P.cur;
    double r2 = 0.0;
    for (int v = 0; v < P.nv; ++v) {
        double rv;
        if (P.ill[c][v]) {
            double u, w;
            P.meet64(P.ln[c][(v == 0) ? P.nv - 1 : v - 1], P.ln[c][v], u, w);
            rv = u * u + w * w;
        } else {
            rv = (double)P.uf[c][v] * P.uf[c][v] + (double)P.wf[c][v] * P.wf[c][v];
        }
        r2 = fmax(r2, rv);
    }
    return chord2_of_r2(r2 * 1.001);
}

// ------------------------------------------------------------- quadrature
struct Acc {
    double m, cx, cy, cz, e;
};

// signed spherical triangle (A, B, C) with the 7-point rule; A = z_i.
// inv_alpha: 1/alpha of the tanh cap.
__device__ __forceinline__ void tri(const Density &r, double inv_alpha, V3 A, V3 B, V3 C, Acc &acc) {
    V3 cr = crs(sub(B, A), sub(C, A));
    double det = dot(A, cr);
    double den = 1.0 + dot(A, B) + dot(B, C) + dot(C, A);
    double area = 2.0 * atan2(det, den);
    const V3 xc = mk(r.xc0, r.xc1, r.xc2);
#pragma unroll 1
    for (int k = 0; k < 7; ++k) {
        V3 x = add(add(scl(A, kQb[k][0]), scl(B, kQb[k][1])), scl(C, kQb[k][2]));
        V3 p = scl(x, rsqrt(dot(x, x)));
        double rv;
        if (r.kind == 0) {
            rv = 1.0;
        } else if (r.kind == 1) {
            double z2 = p.z * p.z;
            rv = (1.0 - r.gamma) * z2 * z2 + r.gamma;
        } else {
            V3 cx = crs(p, xc);
            double d = atan2(sqrt(dot(cx, cx)), dot(p, xc));
            rv = 0.5 * (1.0 - r.gamma) * (tanh((r.beta - d) * inv_alpha) + 1.0) + r.gamma;
            if (r.kind == 3) { rv = rv * rv; rv = rv * rv; }
        }
        double wr = kQw[k] * area * rv;
        V3 dp = sub(p, A);
        acc.m += wr;
        acc.cx += wr * p.x;
        acc.cy += wr * p.y;
        acc.cz += wr * p.z;
        acc.e += wr * dot(dp, dp);
    }
}

__device__ __forceinline__ void write_cell(const CellOut &out, int i, V3 zi, const Acc &acc, DevStatus *st) {
    const double cz = acc.cx * zi.x + acc.cy * zi.y + acc.cz * zi.z;
    if (!(cz > 0.0)) atomicOr(&st->flags, FLAG_NONPOSITIVE);
    if (out.grad) {
        out.grad[3 * (size_t)i] = 2.0 * cz * zi.x - 2.0 * acc.cx;
        out.grad[3 * (size_t)i + 1] = 2.0 * cz * zi.y - 2.0 * acc.cy;
        out.grad[3 * (size_t)i + 2] = 2.0 * cz * zi.z - 2.0 * acc.cz;
    }
    if (out.hdiag) out.hdiag[i] = 1.0 / (2.0 * cz);
    if (out.mass) out.mass[i] = acc.m;
    if (out.moment) {
        out.moment[3 * (size_t)i] = acc.cx;
        out.moment[3 * (size_t)i + 1] = acc.cy;
        out.moment[3 * (size_t)i + 2] = acc.cz;
    }
    if (out.fcell) out.fcell[i] = acc.e;
}

__device__ __forceinline__ bool lex_less(V3 a, V3 b) {
    return a.x < b.x || (a.x == b.x && (a.y < b.y || (a.y == b.y && a.z < b.z)));
}

// -------------------------------------------------------------- topology
// One thread per cell.  mode: list == nullptr -> all bin positions, else the
// retry list.  The certified polygon is written to the cell buffer with its
// edges rotated to start at the neighbour with the lexicographically
// smallest coordinates (so the layout is the same for any input order).
// Cells with more than kCellSlots edges are integrated here, in-thread.
template <int K, int VMAX>
__global__ void __launch_bounds__(128) k_topo(Grid g, Density rho, CellOut out, CellBuf cb,
                                              const int *__restrict__ list, const unsigned *__restrict__ list_count,
                                              int *__restrict__ next_list, unsigned *__restrict__ next_count,
                                              int last_pass, int scan_all, DevStatus *st) {
    int nwork = list ? (int)*list_count : g.n;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nwork; t += gridDim.x * blockDim.x) {
        const int p = list ? list[t] : t;
        const V3 zi = ld(g.zs + p);
        const float4 zif = ldf(g.zf + p);
        const int i = g.sidx[p];

        // ---- neighbours (FP32): list of up to K, bound D2 on everything else
        KnnList<K> L;
        L.cnt = 0;
        double D2;
        if (scan_all || g.n - 1 <= K) {
            all_query<K>(g, zi, zif, p, L, &st->flags);
            D2 = (L.cnt == g.n - 1) ? INFINITY : lower_d2(L.d[K - 1]);
        } else {
            // caps are chord balls |x - z_i| <= r; sin(theta) = r sqrt(1 - r^2/4)
            const double rmax = 0.28291;  // sin(theta) <= 0.28 keeps caps off the far faces
            double r;
            float hint = out.radius ? out.radius[i] : 0.0f;
            if (hint > 0.0f && !last_pass) {
                r = 1.1 * (double)hint;
            } else {
                // local density from the own bin: lambda = count / solid angle
                int b = bin_index(zi.x, zi.y, zi.z, g.G);
                int cbn = g.bstart[b + 1] - g.bstart[b];
                double ax = fabs(zi.x), ay = fabs(zi.y), az = fabs(zi.z);
                double am = fmax(ax, fmax(ay, az));
                double s2 = (ax * ax + ay * ay + az * az) / (am * am);  // 1 + s^2 + t^2
                double omega = (4.0 / ((double)g.G * g.G)) / (s2 * sqrt(s2));
                double lam = fmax((double)cbn, 1.0) / omega;
                r = sqrt(1.5 * K / (3.141592653589793 * lam));
                if (last_pass) r *= 2.0;
            }
            r = fmin(r, rmax);
            double r2 = 0.0;
            float r2acc = 0.0f;
            for (int attempt = 0;; ++attempt) {
                r2 = r * r;
                const double S = r * sqrt(1.0 - 0.25 * r2) * (1.0 + 1e-9);
                r2acc = (float)(r2 * 1.001) + 1e-12f;
                L.cnt = 0;
                cap_query<K>(g, zi, zif, p, S, r2acc, L, &st->flags);
                if (L.cnt == K || r >= rmax || attempt > 8) break;
                double grow = (L.cnt > 0) ? sqrt(1.3 * K / (double)L.cnt) : 2.0;
                r = fmin(r * fmax(grow, 1.25), rmax);
            }
            // unkept: inside the list's range -> >= lower(d_K); outside the cap -> > r
            D2 = (L.cnt == K) ? fmin(lower_d2(L.d[K - 1]), r2) : fmin(lower_d2(r2acc), r2);
        }
        if (out.radius) out.radius[i] = sqrtf(L.cnt ? L.d[L.cnt - 1] : 0.0f);

        // ---- gnomonic frame at z_i: e1 x e2 = z_i
        V3 ax;
        {
            double fx = fabs(zi.x), fy = fabs(zi.y), fz = fabs(zi.z);
            ax = (fx <= fy && fx <= fz) ? mk(1, 0, 0) : ((fy <= fz) ? mk(0, 1, 0) : mk(0, 0, 1));
        }
        const V3 e1 = unit(crs(zi, ax));
        const V3 e2 = crs(zi, e1);

        // ---- clip nearest first, with the security radius
        Poly<K, VMAX> P;
        P.cur = 0;
        P.nv = 4;
        {
            // square lines: K right (u <= L), K+1 top (w <= L), K+2 left, K+3 bottom
            const double la[4] = {1, 0, -1, 0}, lb[4] = {0, 1, 0, -1};
            const float vu[4] = {(float)kBoxL, (float)kBoxL, -(float)kBoxL, -(float)kBoxL};
            const float vw[4] = {-(float)kBoxL, (float)kBoxL, (float)kBoxL, -(float)kBoxL};
            for (int k = 0; k < 4; ++k) {
                P.set_line(K + k, la[k], lb[k], kBoxL);
                P.ln[0][k] = (unsigned char)(K + k);
                P.uf[0][k] = vu[k];
                P.wf[0][k] = vw[k];
                P.ill[0][k] = 0;
            }
        }
        double R2 = chord2_of_r2(2.0 * kBoxL * kBoxL);
        bool ok = true, early = false;
        for (int k = 0; k < L.cnt; ++k) {
            const double bound = fmin(lower_d2(L.d[k]), D2);
            if (bound > 4.0 * R2 * kCertMargin) { early = true; break; }
            const V3 d = sub(ld(g.zs + L.j[k]), zi);
            P.set_line(k, dot(e1, d), dot(e2, d), -dot(zi, d));
            int rc = clip<K, VMAX>(P, k, &st->flags, &st->ambiguous);
            if (rc < 0) { ok = false; break; }
            if (rc > 0) R2 = poly_R2(P);
        }
        bool boxed = false;
        for (int v = 0; v < P.nv; ++v) boxed |= (P.ln[P.cur][v] >= K);  // no extra slots yet
        bool certified = ok && !boxed && (early || D2 > 4.0 * R2 * kCertMargin);
        if (ok && !certified && last_pass) {
            // last resort: clip by every generator (the exact cell); points
            // that cannot reach the polygon are skipped.  A new line goes to
            // an extra slot that no current edge uses.
            for (int q = 0; q < g.n && ok; ++q) {
                if (q == p) continue;
                const V3 d = sub(ld(g.zs + q), zi);
                if (dot(d, d) > 4.0 * R2 * kCertMargin) continue;
                unsigned long long used = 0ull;
                for (int v = 0; v < P.nv; ++v)
                    if (P.ln[P.cur][v] >= K + 4) used |= 1ull << (P.ln[P.cur][v] - (K + 4));
                int x = __ffsll((long long)~used) - 1;
                if (x < 0 || x >= VMAX) { ok = false; break; }
                const int l = K + 4 + x;
                P.set_line(l, dot(e1, d), dot(e2, d), -dot(zi, d));
                P.jx[x] = q;
                int rc = clip<K, VMAX>(P, l, &st->flags, &st->ambiguous);
                if (rc < 0) { ok = false; break; }
                if (rc > 0) R2 = poly_R2(P);
            }
            boxed = false;
            for (int v = 0; v < P.nv; ++v) boxed |= (P.ln[P.cur][v] >= K && P.ln[P.cur][v] < K + 4);
            if (ok && boxed) atomicOr(&st->flags, FLAG_UNBOUNDED);
            certified = ok && !boxed;
        }
        if (!certified) {
            if (last_pass) {
                atomicOr(&st->flags, ok ? FLAG_EXHAUSTED : FLAG_VMAX);
            } else {
                unsigned pos = atomicAdd(next_count, 1u);
                next_list[pos] = p;
            }
            cb.deg[p] = 0;
            continue;
        }

        // ---- canonical edge order: start at the lexicographically smallest neighbour
        const int c = P.cur, nv = P.nv;
        auto nbj = [&](int k) -> int {
            int l = P.ln[c][k];
            return (l < K) ? L.j[l] : P.jx[l - (K + 4)];
        };
        int k0 = 0;
        V3 best = ld(g.zs + nbj(0));
        for (int k = 1; k < nv; ++k) {
            V3 zn = ld(g.zs + nbj(k));
            if (lex_less(zn, best)) { best = zn; k0 = k; }
        }
        auto corner = [&](int k) -> V3 {  // FP64 corner k from its two lines
            double u, w;
            P.meet64(P.ln[c][(k == 0) ? nv - 1 : k - 1], P.ln[c][k], u, w);
            return unit(add(zi, add(scl(e1, u), scl(e2, w))));
        };
        if (out.deg) {
            out.deg[i] = nv;
            if (nv <= out.max_deg)
                for (int t2 = 0; t2 < nv; ++t2)
                    out.nbr[(size_t)i * out.max_deg + t2] = g.sidx[nbj((k0 + t2 < nv) ? k0 + t2 : k0 + t2 - nv)];
        }
        if (nv <= kCellSlots) {
            cb.deg[p] = nv;
            for (int t2 = 0; t2 < nv; ++t2) {
                const int k = (k0 + t2 < nv) ? k0 + t2 : k0 + t2 - nv;
                V3 v = corner(k);
                cb.vx[(size_t)p * kCellSlots + t2] = P4{v.x, v.y, v.z, 0.0};
                cb.nb[(size_t)p * kCellSlots + t2] = nbj(k);
            }
        } else {
            // large cell: integrate here, edges in the canonical order
            cb.deg[p] = 0;
            const double inv_alpha = 1.0 / rho.alpha;
            Acc acc = {0, 0, 0, 0, 0};
            V3 vfirst = corner(k0);
            V3 va = vfirst;
            for (int t2 = 0; t2 < nv; ++t2) {
                const int k = (k0 + t2 < nv) ? k0 + t2 : k0 + t2 - nv;
                const int k1 = (k + 1 == nv) ? 0 : k + 1;
                V3 vb = (t2 + 1 == nv) ? vfirst : corner(k1);
                V3 mu = unit(add(zi, ld(g.zs + nbj(k))));
                tri(rho, inv_alpha, zi, va, mu, acc);
                tri(rho, inv_alpha, zi, mu, vb, acc);
                va = vb;
            }
            write_cell(out, i, zi, acc, st);
        }
    }
}

// -------------------------------------------------------------- quadrature
// Edge list: cells' edges laid end to end in bin order (eoff = exclusive
// scan of the degrees), ecell[e] = the cell of edge e.
__global__ void k_edge_cells(int n, const int *__restrict__ deg, const int *__restrict__ eoff,
                             int *__restrict__ ecell) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int d = deg[p], o = eoff[p];
    for (int k = 0; k < d; ++k) ecell[o + k] = p;
}

// One thread per Voronoi edge (two signed sub-triangles of Sec. 3.2.2, 14
// rule points).  The warp sums each cell's edges with a fixed segmented
// suffix reduction; a cell whose edges straddle two warps is finished by the
// second of its two parts to arrive, which adds them in a fixed order (the
// part holding the cell's first edge + the other part), so results do not
// depend on timing.
__global__ void __launch_bounds__(256) k_quad(Grid g, Density rho, CellOut out, CellBuf cb, const int *eoff,
                                              const int *ecell, double *__restrict__ parts_val,
                                              int *__restrict__ parts_cnt, DevStatus *st) {
    const int nedges = eoff[g.n];
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const long long wbase = e - lane;
    int p = -1;
    Acc acc = {0, 0, 0, 0, 0};
    V3 zi = mk(0, 0, 0);
    int e0 = 0, deg = 0;
    if (e < nedges) {
        p = ecell[e];
        e0 = eoff[p];
        deg = cb.deg[p];
        const int k = (int)(e - e0);
        zi = ld(g.zs + p);
        const P4 *vx = cb.vx + (size_t)p * kCellSlots;
        const V3 va = ld(vx + k);
        const V3 vb = ld(vx + ((k + 1 == deg) ? 0 : k + 1));
        const V3 mu = unit(add(zi, ld(g.zs + cb.nb[(size_t)p * kCellSlots + k])));
        const double inv_alpha = 1.0 / rho.alpha;
        tri(rho, inv_alpha, zi, va, mu, acc);
        tri(rho, inv_alpha, zi, mu, vb, acc);
    }
    // segmented suffix sums: lane l ends with the sum of its segment from l on
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int po = __shfl_down_sync(0xffffffffu, p, o);
        const double m = __shfl_down_sync(0xffffffffu, acc.m, o);
        const double cx = __shfl_down_sync(0xffffffffu, acc.cx, o);
        const double cy = __shfl_down_sync(0xffffffffu, acc.cy, o);
        const double cz = __shfl_down_sync(0xffffffffu, acc.cz, o);
        const double ee = __shfl_down_sync(0xffffffffu, acc.e, o);
        if (lane + o < 32 && po == p) {
            acc.m += m;
            acc.cx += cx;
            acc.cy += cy;
            acc.cz += cz;
            acc.e += ee;
        }
    }
    const int pprev = __shfl_up_sync(0xffffffffu, p, 1);
    const bool head = (p >= 0) && (lane == 0 || pprev != p);
    if (!head) return;
    const bool starts_here = e0 >= wbase;
    const bool ends_here = e0 + deg <= wbase + 32;
    if (starts_here && ends_here) {
        write_cell(out, g.sidx[p], zi, acc, st);
        return;
    }
    // split cell: publish this part, then the second arrival finishes
    double *slot = parts_val + (size_t)p * 10 + (starts_here ? 0 : 5);
    slot[0] = acc.m; slot[1] = acc.cx; slot[2] = acc.cy; slot[3] = acc.cz; slot[4] = acc.e;
    __threadfence();
    if (atomicAdd(&parts_cnt[p], 1) == 1) {
        __threadfence();
        const volatile double *a = parts_val + (size_t)p * 10;
        Acc tot;
        tot.m = a[0] + a[5];
        tot.cx = a[1] + a[6];
        tot.cy = a[2] + a[7];
        tot.cz = a[3] + a[8];
        tot.e = a[4] + a[9];
        parts_cnt[p] = 0;  // ready for the next evaluation
        write_cell(out, g.sidx[p], zi, tot, st);
    }
}

}  // namespace

void bin_points(const double *z, int n, int G, int *bin_of, int *count, int *start, int *cursor, int *scan_tmp,
                P4 *zs, float4 *zf, int *sidx, DevStatus *st, cudaStream_t s, int64_t *launches) {
    const int nbins = 6 * G * G;
    cudaMemsetAsync(count, 0, sizeof(int) * nbins, s);
    int blocks = (n + 255) / 256;
    k_bin_count<<<blocks, 256, 0, s>>>(z, n, G, bin_of, count, st);
    exclusive_scan(count, start, nbins, scan_tmp, s, launches);
    k_set_total<<<1, 1, 0, s>>>(start, nbins, n);
    cudaMemcpyAsync(cursor, start, sizeof(int) * nbins, cudaMemcpyDeviceToDevice, s);
    k_bin_scatter<<<blocks, 256, 0, s>>>(z, n, bin_of, cursor, zs, zf, sidx);
    k_bin_sort<<<(nbins + 255) / 256, 256, 0, s>>>(start, nbins, zs, zf, sidx);
    (*launches) += 4;
}

__global__ void k_set_total_from(int *arr, int n, const int *last_in) {
    // arr[n] = arr[n-1] + last_in[n-1]: total of an exclusive scan
    arr[n] = arr[n - 1] + last_in[n - 1];
}

void cell_passes(const Grid &g, const Density &rho, const CellOut &out, const CellBuf &cb, int *list1, int *list2,
                 DevStatus *st, int knn_k0, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, int64_t *launches,
                 int64_t *cell_launches) {
    const int blocks0 = (g.n + 127) / 128;
    if (knn_k0 <= 16)
        k_topo<16, 32><<<blocks0, 128, 0, s>>>(g, rho, out, cb, nullptr, nullptr, list1, &st->retry_count[0], 0, 0, st);
    else
        k_topo<32, 32><<<blocks0, 128, 0, s>>>(g, rho, out, cb, nullptr, nullptr, list1, &st->retry_count[0], 0, 0, st);
    // retry passes: sized for the worst case, they read their work count on the device
    const int rblocks = 2 * 152;
    k_topo<64, 64><<<rblocks, 64, 0, s>>>(g, rho, out, cb, list1, &st->retry_count[0], list2, &st->retry_count[1], 0,
                                          0, st);
    int scan_all = g.n <= 20000 ? 1 : 0;
    k_topo<128, 64><<<rblocks, 64, 0, s>>>(g, rho, out, cb, list2, &st->retry_count[1], nullptr, &st->retry_count[2],
                                           1, scan_all, st);
    // edge list for the quadrature
    exclusive_scan(cb.deg, cb.eoff, g.n, cb.scan_tmp, s, launches);
    k_set_total_from<<<1, 1, 0, s>>>(cb.eoff, g.n, cb.deg);
    k_edge_cells<<<(g.n + 255) / 256, 256, 0, s>>>(g.n, cb.deg, cb.eoff, cb.ecell);
    if (ev0) cudaEventRecord(ev0, s);
    // Euler: a full tessellation has 6N - 12 edge sides; failed cells only lower the count
    const long long max_edges = 6LL * g.n;
    k_quad<<<(unsigned)((max_edges + 255) / 256), 256, 0, s>>>(g, rho, out, cb, cb.eoff, cb.ecell, cb.parts_val,
                                                               cb.parts_cnt, st);
    if (ev1) cudaEventRecord(ev1, s);
    (*launches) += 6;
    (*cell_launches) += 4;
}

}  // namespace scvt
