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
#include <string.h>

#include <algorithm>

#include "df.cuh"
#include "scvt_internal.cuh"

namespace scvt {

namespace {

constexpr double kBoxL = 1.0e3;         // half-width of the starting square (gnomonic)

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

// the same rule as double-float pairs: weights b1, b2 of the 2nd and 3rd
// vertex, point weight W, and b1^2, 2 b1 b2, b2^2
#define SCVT_DF(x) {(float)(x), (float)((x) - (double)(float)(x))}
#define SCVT_QP(b1, b2, w) {SCVT_DF(b1), SCVT_DF(b2), SCVT_DF(w), SCVT_DF((b1) * (b1)), SCVT_DF(2.0 * (b1) * (b2)), \
                            SCVT_DF((b2) * (b2))}
__constant__ float kQdf[7][6][2] = {
    SCVT_QP(1.0 / 3.0, 1.0 / 3.0, 0.225),
    SCVT_QP(0.1012865073234563388, 0.1012865073234563388, 0.1259391805448271526),
    SCVT_QP(0.7974269853530873224, 0.1012865073234563388, 0.1259391805448271526),
    SCVT_QP(0.1012865073234563388, 0.7974269853530873224, 0.1259391805448271526),
    SCVT_QP(0.47014206410511508977, 0.47014206410511508977, 0.13239415278850618074),
    SCVT_QP(0.059715871789769820459, 0.47014206410511508977, 0.13239415278850618074),
    SCVT_QP(0.47014206410511508977, 0.059715871789769820459, 0.13239415278850618074),
};
#undef SCVT_QP
#undef SCVT_DF

// the same rule in FP32 for the mixed-precision quadrature
__constant__ float kQbf[7][2] = {
    {1.0f / 3.0f, 1.0f / 3.0f},
    {0.1012865073234563388f, 0.1012865073234563388f},
    {0.7974269853530873224f, 0.1012865073234563388f},
    {0.1012865073234563388f, 0.7974269853530873224f},
    {0.47014206410511508977f, 0.47014206410511508977f},
    {0.059715871789769820459f, 0.47014206410511508977f},
    {0.47014206410511508977f, 0.059715871789769820459f},
};
__constant__ float kQwf[7] = {0.225f,
                              0.1259391805448271526f, 0.1259391805448271526f, 0.1259391805448271526f,
                              0.13239415278850618074f, 0.13239415278850618074f, 0.13239415278850618074f};

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

// The problem a position (or original index) belongs to, with its range,
// bin resolution and bins; a single problem is problem 0 of itself.
struct View {
    int b, p0, n, G;
    const int *bstart;
};
__device__ __forceinline__ View view_of(const Grid &g, int p) {
    if (!g.inst) return View{0, 0, g.n, g.G, g.bstart};
    const int b = g.pinst[p];
    const InstGeom I = g.inst[b];
    return View{b, I.p0, I.n, I.G, g.bstart + I.bin0};
}
__device__ __forceinline__ unsigned *flags_of(const Grid &g, DevStatus *st, int b) {
    return g.ist ? &g.ist[b].flags : &st->flags;
}
__device__ __forceinline__ bool inactive(const Grid &g, int b) { return g.active && !g.active[b]; }

// One chunk of the cell pipeline: cells [p0, p1) in bin order, their edges
// [*e0, *e0 + *etot) of the edge list (both known on the device only: a
// chunk's edges follow the previous chunk's).
struct Span {
    int p0, p1;
    const int *e0, *etot;
};

// Cube-map bin of a unit vector: face = its largest component, then the
// gnomonic coordinates s, t in [-1, 1] on G x G bins.  In FP32 from the
// rounded coordinates: s and t are within 2e-7 of their exact values, and
// the cap queries widen their bin ranges by at least 1e-6 in s and t; a
// point whose two largest components agree to 1e-7 may take either face,
// and a query takes every face its cap reaches (|q_a| + S >= 1/sqrt3 - 1e-6).
__device__ __forceinline__ int bin_index(float x, float y, float z, int G) {
    const float ax = fabsf(x), ay = fabsf(y), az = fabsf(z);
    int a;
    float m, pb, pc;
    if (ax >= ay && ax >= az) { a = 0; m = x; pb = y; pc = z; }
    else if (ay >= az) { a = 1; m = y; pb = z; pc = x; }
    else { a = 2; m = z; pb = x; pc = y; }
    const float inv = 1.0f / fabsf(m);
    int iu = (int)floorf((pb * inv + 1.0f) * 0.5f * G);
    int iv = (int)floorf((pc * inv + 1.0f) * 0.5f * G);
    iu = min(max(iu, 0), G - 1);
    iv = min(max(iv, 0), G - 1);
    const int face = 2 * a + (m < 0.0f ? 1 : 0);
    return (face * G + iv) * G + iu;
}

// ---------------------------------------------------------------- binning
__global__ void k_bin_count(const double *__restrict__ z, Grid g, int *__restrict__ bin_of,
                            int *__restrict__ count, DevStatus *st) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const View v = view_of(g, i);
    const int base = (int)(v.bstart - g.bstart);
    double x = z[3 * (size_t)i], y = z[3 * (size_t)i + 1], w = z[3 * (size_t)i + 2];
    double r2 = x * x + y * y + w * w;
    if (!(fabs(r2 - 1.0) <= 2e-12)) {  // also catches NaN / inf
        atomicOr(flags_of(g, st, v.b), FLAG_BAD_POINT);
        bin_of[i] = base;
        atomicAdd(&count[base], 1);
        return;
    }
    int b = base + bin_index((float)x, (float)y, (float)w, v.G);
    bin_of[i] = b;
    atomicAdd(&count[b], 1);
}

// fullest bin of each problem (blockIdx.y; gridDim.x blocks share its bins)
// into its status block
__global__ void k_bin_max(Grid g, const int *__restrict__ count, DevStatus *st) {
    int b0 = 0, nb = g.nbins;
    DevStatus *dst = st;
    if (g.inst) {
        const InstGeom I = g.inst[blockIdx.y];
        b0 = I.bin0;
        nb = 6 * I.G * I.G;
        dst = g.ist + blockIdx.y;
        if (inactive(g, blockIdx.y)) return;
    }
    int m = 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += gridDim.x * blockDim.x) m = max(m, count[b0 + k]);
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0) atomicMax(&dst->max_bin, (unsigned)m);
}

// The FP32 copy carries the generator's search-radius hint (from the previous
// evaluation, 0 = none) in its w component, so the topology pass reads it with
// the coordinates instead of through the original index.
// Third FP32 part of a point (z - hi - lo, exact: hi + lo + ll == z since
// z - hi and then the remainder after lo are exact in FP64 and the last fits
// in 24 bits) and |z|^2 - 1: the squares by the FMA form of TwoProduct,
// their sum by TwoSum, so s - 1 plus the error terms is |z|^2 - 1 to ~1e-32.
__device__ __forceinline__ float4 fine_parts(double x, double y, double w, float4 h, float4 l) {
    const double rx = (x - (double)h.x) - (double)l.x, ry = (y - (double)h.y) - (double)l.y,
                 rz = (w - (double)h.z) - (double)l.z;
    const double px = x * x, py = y * y, pz = w * w;
    const double ex = fma(x, x, -px), ey = fma(y, y, -py), ez = fma(w, w, -pz);
    const double s1 = px + py, b1 = s1 - px, t1 = (px - (s1 - b1)) + (py - b1);
    const double s2 = s1 + pz, b2 = s2 - s1, t2 = (s1 - (s2 - b2)) + (pz - b2);
    const double eps = (s2 - 1.0) + ((t1 + t2) + (ex + ey + ez));
    return make_float4((float)rx, (float)ry, (float)rz, (float)eps);
}

__global__ void k_bin_scatter(const double *__restrict__ z, int n, const int *__restrict__ bin_of,
                              int *__restrict__ cursor, P4 *__restrict__ zs, float4 *__restrict__ zf,
                              float4 *__restrict__ zl, float4 *__restrict__ zll, int *__restrict__ sidx,
                              const float *__restrict__ hint) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int pos = atomicAdd(&cursor[bin_of[i]], 1);
    sidx[pos] = i;
    double x = z[3 * (size_t)i], y = z[3 * (size_t)i + 1], w = z[3 * (size_t)i + 2];
    zs[pos] = P4{x, y, w, 0.0};
    const float hx = (float)x, hy = (float)y, hw = (float)w;
    const float4 h = make_float4(hx, hy, hw, hint ? hint[i] : 0.0f);
    const float4 l = make_float4((float)(x - (double)hx), (float)(y - (double)hy), (float)(w - (double)hw), 0.0f);
    zf[pos] = h;
    zl[pos] = l;
    if (zll) zll[pos] = fine_parts(x, y, w, h, l);
}

// Order each bin's generators by their coordinates (lexicographic x, y, z).
// The scatter above fills a bin in atomic order; sorting makes the bin
// layout a function of the point set alone, so every later step (kNN ties,
// the edge list of the quadrature and its reduction tree) is reproducible and
// independent of the input order.  Bins hold a few generators: insertion sort.
__global__ void k_bin_sort(const int *__restrict__ start, int nbins, P4 *__restrict__ zs, float4 *__restrict__ zf,
                           float4 *__restrict__ zl, float4 *__restrict__ zll, int *__restrict__ sidx) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    const int p0 = start[b], p1 = start[b + 1];
    for (int p = p0 + 1; p < p1; ++p) {
        const P4 v = zs[p];
        const float4 vf = zf[p], vl = zl[p], vll = zll ? zll[p] : make_float4(0, 0, 0, 0);
        const int id = sidx[p];
        int q = p;
        while (q > p0) {
            const P4 u = zs[q - 1];
            const bool greater = u.x > v.x || (u.x == v.x && (u.y > v.y || (u.y == v.y && u.z > v.z)));
            if (!greater) break;
            zs[q] = u;
            zf[q] = zf[q - 1];
            zl[q] = zl[q - 1];
            if (zll) zll[q] = zll[q - 1];
            sidx[q] = sidx[q - 1];
            --q;
        }
        zs[q] = v;
        zf[q] = vf;
        zl[q] = vl;
        if (zll) zll[q] = vll;
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
void scan_rec(const int *in, int *out, int len, int *tmp, cudaStream_t s, int64_t *launches) {
    int tiles = (len + 2047) / 2048;
    if (tiles <= 1) {
        k_scan_tiles<<<1, 1024, 0, s>>>(in, out, len, nullptr);
        (*launches)++;
        return;
    }
    int *totals = tmp, *tot_scan = tmp + tiles;
    k_scan_tiles<<<tiles, 1024, 0, s>>>(in, out, len, totals);
    scan_rec(totals, tot_scan, tiles, tmp + 2 * tiles, s, launches);
    k_scan_add<<<tiles, 1024, 0, s>>>(out, len, tot_scan);
    (*launches) += 2;
}

__global__ void k_set_total(int *start, int nbins, int n) { start[nbins] = n; }

// ------------------------------------------------------------ k-nearest
// The neighbour search runs on FP32 copies of the coordinates (the FP32 pipe
// is ~70x the FP64 pipe on this part); it only has to produce candidates and a
// certified lower bound on the distance of every generator it did not keep.
// FP32 coordinates are within 3e-8 of the FP64 ones, so an FP32 difference is
// within 1.1e-7 + 6e-8 |d| of the true one, and the FP32 squared norm and
// square root add 1.8e-7 relative: the true chord is at least
// sqrt(d2f) (1 - 2.6e-7) - 1.1e-7.  lower32() uses (1 - 1e-6) and 5e-7, and
// rounds its own square down.
__device__ __forceinline__ float lower32(float d2f) {
    float d = sqrtf(d2f) * (1.0f - 1e-6f) - 5e-7f;
    return d > 0.0f ? d * d * (1.0f - 1e-6f) : 0.0f;
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

// Every generator p (bin order) within chord r of z_i is scanned; those with
// d2f <= r2acc are offered to the list.  S >= sin(theta) of that ball, with
// FP32 rounding and the FP32 centre already covered.  For face (a, sign) the
// values s = x_b / |x_a| attained in the cap lie between the roots of
// (q_b - s sign q_a)^2 = S^2 (1 + s^2): the planes of constant s are great
// circles through the c axis, and one meets the cap iff q's distance to it is
// at most S.  The FP32 roots are widened by 4e-6/A + 1e-6 (their error is
// below 4e-7/A).
template <int K>
__device__ void cap_query(const Grid &g, const View &v, V3 q, float4 qf, int self, float S, float r2acc,
                          KnnList<K> &L, unsigned *flags) {
    const float S2 = S * S;
    const float qv[3] = {qf.x, qf.y, qf.z};
    for (int a = 0; a < 3; ++a) {
        const float qa = qv[a];
        const float A = qa * qa - S2;
        if (A <= 0.0f) continue;  // the cap cannot reach face a (|x_a| >= 1/sqrt3 there)
        // nor when |x_a| <= |q_a| + S stays below 1/sqrt3 on the whole cap; this
        // also keeps A away from 0, where the roots below lose their accuracy
        if (fabsf(qa) + S + 1e-6f < 0.5773f) continue;
        const float sg = qa > 0.0f ? 1.0f : -1.0f;
        const int face = 2 * a + (qa < 0.0f ? 1 : 0);
        const float invA = 1.0f / A;
        const float margin = 4e-6f * invA + 1e-6f;
        int lo[2], hi[2];
        bool empty = false;
        for (int r = 0; r < 2; ++r) {
            const float qb = qv[(a + 1 + r) % 3];
            const float disc = qa * qa + qb * qb - S2;
            const float rt = S * sqrtf(fmaxf(disc, 0.0f));
            float s0 = (sg * qa * qb - rt) * invA - margin;
            float s1 = (sg * qa * qb + rt) * invA + margin;
            if (s0 > 1.0f || s1 < -1.0f) { empty = true; break; }
            s0 = fmaxf(s0, -1.0f);
            s1 = fminf(s1, 1.0f);
            lo[r] = min(max((int)floorf((s0 + 1.0f) * 0.5f * v.G), 0), v.G - 1);
            hi[r] = min(max((int)floorf((s1 + 1.0f) * 0.5f * v.G), 0), v.G - 1);
        }
        if (empty) continue;
        for (int iv = lo[1]; iv <= hi[1]; ++iv) {
            int row = (face * v.G + iv) * v.G;
            int p0 = v.bstart[row + lo[0]], p1 = v.bstart[row + hi[0] + 1];
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
__device__ void all_query(const Grid &g, const View &v, V3 q, float4 qf, int self, KnnList<K> &L, unsigned *flags) {
    for (int p = v.p0; p < v.p0 + v.n; ++p) {
        if (p == self) continue;
        float4 c = ldf(g.zf + p);
        float dx = c.x - qf.x, dy = c.y - qf.y, dz = c.z - qf.z;
        float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (d2 == 0.0f) check_duplicate(g, q, p, flags);
        L.push(d2, p);
    }
}

// ---------------------------------------------------------------- clipping
// Convex polygon in the gnomonic plane at z_i (frame e1, e2): edge k runs
// from vertex k to vertex k+1 on line ln[k]: a u + b w <= c with
// (a, b, c) = (e1.d, e2.d, -z_i.d), d = z_j - z_i.  Line slots: 0..K-1 follow
// the kNN list, K..K+3 are the starting square, K+4.. hold generators met by
// the exhaustive last-resort scan (ids in jx).  The table keeps FP32 lines
// (d taken in FP64, then rounded; c = -z_i.d in FP64, then rounded); an FP64
// line is recomputed from the generator when needed.  Vertex k is the
// intersection of lines ln[k-1] and ln[k], carried as an FP32 approximation
// with a flag `ill` when that 2x2 system is poorly conditioned; its FP64
// value is only ever computed from its two FP64 lines, so the final corners
// do not depend on the order of clipping.
//
// Inside/outside decisions are filtered: the FP32 side value
// sd = a u + b w - c decides when |sd| > 2e-4 M, M = (|a|+|b|)(|u|+|w|) + |c|,
// and the vertex is well conditioned (|det| >= (|a1 b2| + |a2 b1|)/30).
// FP32 lines are within ~2e-7 of M's line part and the FP32 vertex within
// kappa * 3e-7 <= 1e-5 of its scale, so the FP32 side value is within ~1e-5 M
// and its sign equals the FP64 sign.  Every other decision is taken in FP64.
struct Frame {
    V3 zi, e1, e2;
    float3 e1f, e2f;
    const P4 *zs;
};

template <int K, int VMAX, int EXTRA>
struct Poly {
    float uf[2][VMAX], wf[2][VMAX];
    unsigned char ln[2][VMAX];
    unsigned char ill[2][VMAX];
    float la[K + 4 + EXTRA], lb[K + 4 + EXTRA], lc[K + 4 + EXTRA];
    int jx[EXTRA > 0 ? EXTRA : 1];
    const int *kj;  // kNN list ids
    int nv, cur;

    __device__ __forceinline__ int gen_of(int l) const {
        return (l < K) ? kj[l] : ((l < K + 4) ? -1 - (l - K) : jx[l - (K + 4)]);
    }
    __device__ __forceinline__ void set_line(const Frame &F, int l, int j) {
        const V3 d = sub(ld(F.zs + j), F.zi);
        const float dx = (float)d.x, dy = (float)d.y, dz = (float)d.z;
        la[l] = F.e1f.x * dx + F.e1f.y * dy + F.e1f.z * dz;
        lb[l] = F.e2f.x * dx + F.e2f.y * dy + F.e2f.z * dz;
        lc[l] = (float)(-dot(F.zi, d));
    }
    __device__ __forceinline__ void line64(const Frame &F, int l, double &a, double &b, double &c) const {
        if (l >= K && l < K + 4) {
            const int k = l - K;  // square: right, top, left, bottom
            a = (k == 0) ? 1.0 : ((k == 2) ? -1.0 : 0.0);
            b = (k == 1) ? 1.0 : ((k == 3) ? -1.0 : 0.0);
            c = kBoxL;
            return;
        }
        const V3 d = sub(ld(F.zs + gen_of(l)), F.zi);
        a = dot(F.e1, d);
        b = dot(F.e2, d);
        c = -dot(F.zi, d);
    }
    __device__ __forceinline__ static void meet(double a1, double b1, double c1, double a2, double b2, double c2,
                                                double &u, double &w) {
        double inv = 1.0 / (a1 * b2 - a2 * b1);
        u = (c1 * b2 - c2 * b1) * inv;
        w = (a1 * c2 - a2 * c1) * inv;
    }
    __device__ __forceinline__ void meet64(const Frame &F, int l1, int l2, double &u, double &w) const {
        double a1, b1, c1, a2, b2, c2;
        line64(F, l1, a1, b1, c1);
        line64(F, l2, a2, b2, c2);
        meet(a1, b1, c1, a2, b2, c2, u, w);
    }
    // FP32 intersection; returns true if it is ill conditioned
    __device__ __forceinline__ bool meet32(int l1, int l2, float &u, float &w) const {
        float p1 = la[l1] * lb[l2], p2 = la[l2] * lb[l1];
        float det = p1 - p2;
        u = (lc[l1] * lb[l2] - lc[l2] * lb[l1]) / det;
        w = (la[l1] * lc[l2] - la[l2] * lc[l1]) / det;
        return !(fabsf(det) * 30.0f >= fabsf(p1) + fabsf(p2));
    }
};

// FP32 upper bound of 2 - 2/sqrt(1 + r2) (the squared chord of a vertex at
// gnomonic radius^2 r2), inflated past its own rounding
__device__ __forceinline__ float chord2_up(float r2) {
    float q = sqrtf(1.0f + r2);
    return 2.0f * r2 / (q * (1.0f + q)) * (1.0f + 1e-5f);
}

// clip by line slot l; returns 1 if the polygon changed, 0 if not, -1 on
// capacity / empty errors
template <int K, int VMAX, int EXTRA>
__device__ int clip(Poly<K, VMAX, EXTRA> &P, const Frame &F, int l, unsigned *flags, unsigned long long *amb) {
    const int c0 = P.cur, nv = P.nv;
    const float la = P.la[l], lb = P.lb[l], lc = P.lc[l];
    const float lab = fabsf(la) + fabsf(lb);
    unsigned long long out = 0ull;
    int namb = 0;
    for (int k = 0; k < nv; ++k) {
        const float uk = P.uf[c0][k], wk = P.wf[c0][k];
        const float sd = fmaf(la, uk, fmaf(lb, wk, -lc));
        const float mag = lab * (fabsf(uk) + fabsf(wk)) + fabsf(lc);
        bool outside;
        if (!P.ill[c0][k] && fabsf(sd) > 2e-4f * mag) {
            outside = sd > 0.0f;
        } else {
            const int kp = (k == 0) ? nv - 1 : k - 1;
            double u, w, a, b, c;
            P.meet64(F, P.ln[c0][kp], P.ln[c0][k], u, w);
            P.line64(F, l, a, b, c);
            const double sd64 = a * u + b * w - c;
            if (fabs(sd64) <= 1e-14 * (fabs(a * u) + fabs(b * w) + fabs(c))) ++namb;
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
template <int K, int VMAX, int EXTRA>
__device__ __forceinline__ float poly_R2(const Poly<K, VMAX, EXTRA> &P, const Frame &F) {
    const int c = P.cur;
    float r2 = 0.0f;
    for (int v = 0; v < P.nv; ++v) {
        float rv;
        if (P.ill[c][v]) {
            double u, w;
            P.meet64(F, P.ln[c][(v == 0) ? P.nv - 1 : v - 1], P.ln[c][v], u, w);
            rv = (float)(u * u + w * w);
        } else {
            rv = P.uf[c][v] * P.uf[c][v] + P.wf[c][v] * P.wf[c][v];
        }
        r2 = fmaxf(r2, rv);
    }
    return chord2_up(r2 * 1.001f);
}

// ------------------------------------------------------------- quadrature
struct Acc {
    double m, cx, cy, cz, e;
};

// the density at a unit vector p, directly from its definition (kinds 2, 3:
// geodesic distance d to x_c, the tanh cap in its logistic form)
__device__ __forceinline__ double rho_direct(const Density &r, double inv_alpha, V3 p) {
    const V3 xc = mk(r.xc0, r.xc1, r.xc2);
    V3 cx = crs(p, xc);
    double d = atan2(sqrt(dot(cx, cx)), dot(p, xc));
    // (1 - gamma)/2 (tanh(x) + 1) + gamma, as (1 - gamma)/(1 + exp(-2x)) + gamma:
    // the same function without the cancellation of tanh(x) + 1 for x << 0
    double rv = (1.0 - r.gamma) / (1.0 + exp(-2.0 * (r.beta - d) * inv_alpha)) + r.gamma;
    if (r.kind == 3) { rv = rv * rv; rv = rv * rv; }
    return rv;
}

__device__ __forceinline__ double horner(const double *__restrict__ cf, int K, double u) {
    double r = cf[K - 1];
    for (int j = K - 2; j >= 0; --j) r = fma(r, u, cf[j]);
    return r;
}

// Offsets from z_i (FP64).  A point x = z_i + w near the sphere projects to
// p = x / |x|, and p - z_i = (1 + m) w + m z_i with m = 1/|x| - 1 and
// |x|^2 - 1 = (|z_i|^2 - 1) + 2 z_i.w + |w|^2; m comes from the binomial
// series of (1 + e)^(-1/2) - 1 for |e| < 1e-4 (exact to 3e-21 relative to e),
// else from the square root.  The tangential part of p - z_i is then exact
// to rounding relative to |w| (the radial part, m z_i, moves the point off
// the sphere only at second order), so no difference of nearby unit vectors
// is ever formed.
__device__ __forceinline__ double inv_norm_minus1(double e) {
    if (fabs(e) < 1e-4) return e * (-0.5 + e * (0.375 + e * (-0.3125 + e * 0.2734375)));
    const double r = sqrt(1.0 + e);
    return -e / (r * (1.0 + r));
}

__device__ __forceinline__ V3 project_offset(V3 zi, double aA1, V3 w) {
    const double m = inv_norm_minus1(aA1 + 2.0 * dot(zi, w) + dot(w, w));
    return add(scl(w, 1.0 + m), scl(zi, m));
}

// the edge midpoint mu_ij = normalize(z_i + z_j) as the offset mu - z_i
__device__ __forceinline__ V3 midpoint_offset(V3 zi, double aA1, V3 zj) {
    return project_offset(zi, aA1, scl(sub(zj, zi), 0.5));
}

// signed spherical triangle (A, A + ob, A + oc) with the 7-point rule; A = z_i,
// ob, oc: offsets of the other two corners from z_i, aA1 = |A|^2 - 1.
// inv_alpha: 1/alpha of the tanh cap.  cf / K / cj: the density's series
// about x_c.p = cj from the density table (K = 0: evaluate the density
// directly).  Accumulates m, the moment relative to z_i (sum w rho (p - z_i);
// the caller adds m z_i) and the energy.
__device__ __forceinline__ void tri(const Density &r, double inv_alpha, V3 A, double aA1, V3 ob, V3 oc, Acc &acc,
                                    const double *cf = nullptr, int K = 0, double cj = 0.0) {
    // Van Oosterom-Strackee with B = A + ob, C = A + oc:
    // det[A,B,C] = A.(ob x oc), 1 + A.B + B.C + C.A = 4 + 3 (|A|^2 - 1) + 2 A.(ob + oc) + ob.oc
    const double det = dot(A, crs(ob, oc));
    const double den = 4.0 + 3.0 * aA1 + 2.0 * dot(A, add(ob, oc)) + dot(ob, oc);
    // signed area 2 atan(det / den); for the small triangles of a cell
    // |det / den| < 1e-2 and the odd Taylor series of atan to the x^7 term is
    // exact to 1e-17 relative
    double area;
    const double xa = det / den;
    if (den > 0.0 && fabs(xa) < 1e-2) {
        const double x2 = xa * xa;
        area = 2.0 * xa * (1.0 + x2 * (-1.0 / 3.0 + x2 * (0.2 + x2 * (-1.0 / 7.0))));
    } else {
        area = 2.0 * atan2(det, den);
    }
    const V3 xc = mk(r.xc0, r.xc1, r.xc2);
    const double u0 = (K > 0) ? dot(xc, A) - cj : 0.0;
#pragma unroll 1
    for (int k = 0; k < 7; ++k) {
        // rule point x = A + b1 ob + b2 oc, projected: p - A from the offsets
        const V3 w = add(scl(ob, kQb[k][1]), scl(oc, kQb[k][2]));
        const V3 dp = project_offset(A, aA1, w);
        double rv;
        if (r.kind == 0) {
            rv = 1.0;
        } else if (r.kind == 1) {
            const double pz = A.z + dp.z, z2 = pz * pz;
            rv = (1.0 - r.gamma) * z2 * z2 + r.gamma;
        } else if (K > 0) {
            rv = horner(cf, K, u0 + dot(xc, dp));
        } else {
            rv = rho_direct(r, inv_alpha, add(A, dp));
        }
        const double wr = kQw[k] * area * rv;
        acc.m += wr;
        acc.cx = fma(wr, dp.x, acc.cx);
        acc.cy = fma(wr, dp.y, acc.cy);
        acc.cz = fma(wr, dp.z, acc.cz);
        acc.e = fma(wr, dot(dp, dp), acc.e);
    }
}

// moment relative to z_i -> moment c = m z_i + sum w rho (p - z_i)
__device__ __forceinline__ void moment_from_offsets(V3 zi, Acc &acc) {
    acc.cx = fma(zi.x, acc.m, acc.cx);
    acc.cy = fma(zi.y, acc.m, acc.cy);
    acc.cz = fma(zi.z, acc.m, acc.cz);
}

__device__ __forceinline__ void write_cell(const CellOut &out, int i, V3 zi, const Acc &acc, unsigned *flags) {
    const double cz = acc.cx * zi.x + acc.cy * zi.y + acc.cz * zi.z;
    if (!(cz > 0.0)) atomicOr(flags, FLAG_NONPOSITIVE);
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

// order-preserving unsigned image of a float's bits (negative values reversed)
__device__ __forceinline__ unsigned okey32(float x) {
    const unsigned b = __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Canonical start of a cell's edge cycle: the neighbour whose FP32 pair
// coordinates (hi.x, lo.x, hi.y, lo.y, hi.z, lo.z) are lexicographically
// smallest -- a function of the point alone, so the edge order (and every
// per-cell sum) is the same whichever pass certifies the cell.
__device__ __forceinline__ bool ckey_less(const Grid &g, int a, int b) {
    const float4 ha = g.zf[a], hb = g.zf[b], la = g.zl[a], lb = g.zl[b];
    const unsigned ka[6] = {okey32(ha.x), okey32(la.x), okey32(ha.y), okey32(la.y), okey32(ha.z), okey32(la.z)};
    const unsigned kb[6] = {okey32(hb.x), okey32(lb.x), okey32(hb.y), okey32(lb.y), okey32(hb.z), okey32(lb.z)};
#pragma unroll
    for (int k = 0; k < 6; ++k)
        if (ka[k] != kb[k]) return ka[k] < kb[k];
    return false;
}

// -------------------------------------------------------------- topology
// One thread per cell.  list == nullptr -> all bin positions, else the retry
// list.  The certified polygon is written to the cell buffer with its edges
// rotated to start at the neighbour with the lexicographically smallest
// coordinates (so the layout is the same for any input order).  Cells with
// more than kCellSlots edges are integrated here, in-thread.  EXTRA > 0 only
// in the last pass, which may clip by every generator.
template <int K, int VMAX, int EXTRA>
__global__ void __launch_bounds__(128) k_topo(Grid g, CellOut out, CellBuf cb,
                                              const int *__restrict__ list, const unsigned *__restrict__ list_count,
                                              int *__restrict__ next_list, unsigned *__restrict__ next_count,
                                              int last_pass, int scan_all_max, DevStatus *st) {
    int nwork = list ? (int)*list_count : g.n;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nwork; t += gridDim.x * blockDim.x) {
        const int p = list ? list[t] : t;
        const View v = view_of(g, p);
        if (!list && inactive(g, v.b)) {
            cb.deg[p] = 0;
            continue;
        }
        unsigned *flags = flags_of(g, st, v.b);
        const V3 zi = ld(g.zs + p);
        const float4 zif = ldf(g.zf + p);
        const int i = g.sidx[p];
        const bool scan_all = v.n <= scan_all_max;

        // ---- neighbours (FP32): list of up to K, bound D2 on everything else
        KnnList<K> L;
        L.cnt = 0;
        float D2;
        if (scan_all || v.n - 1 <= K) {
            all_query<K>(g, v, zi, zif, p, L, flags);
            D2 = (L.cnt == v.n - 1) ? INFINITY : lower32(L.d[K - 1]);
        } else {
            // caps are chord balls |x - z_i| <= r; sin(theta) = r sqrt(1 - r^2/4)
            const float rmax = 0.2829f;  // sin(theta) <= 0.28 keeps caps off the far faces
            float r;
            const float hint = out.radius ? out.radius[i] : 0.0f;
            if (hint > 0.0f && !last_pass) {
                r = 1.1f * hint;
            } else {
                // local density from the own bin: lambda = count / solid angle
                int b = bin_index((float)zi.x, (float)zi.y, (float)zi.z, v.G);
                int cbn = v.bstart[b + 1] - v.bstart[b];
                float ax = fabsf(zif.x), ay = fabsf(zif.y), az = fabsf(zif.z);
                float am = fmaxf(ax, fmaxf(ay, az));
                float s2 = (ax * ax + ay * ay + az * az) / (am * am);  // 1 + s^2 + t^2
                float omega = (4.0f / ((float)v.G * v.G)) / (s2 * sqrtf(s2));
                float lam = fmaxf((float)cbn, 1.0f) / omega;
                r = sqrtf(1.5f * K / (3.14159265f * lam));
                if (last_pass) r *= 2.0f;
            }
            r = fminf(r, rmax);
            float r2lo = 0.0f, r2acc = 0.0f;
            for (int attempt = 0;; ++attempt) {
                const float rs = r * (1.0f + 1e-5f) + 1e-7f;  // covers the FP32 centre
                const float S = rs * sqrtf(1.0f - 0.25f * rs * rs) * (1.0f + 1e-5f);
                r2lo = r * r * (1.0f - 1e-6f);
                r2acc = r * r * 1.001f + 1e-12f;
                L.cnt = 0;
                cap_query<K>(g, v, zi, zif, p, S, r2acc, L, flags);
                if (L.cnt == K || r >= rmax || attempt > 8) break;
                float grow = (L.cnt > 0) ? sqrtf(1.3f * K / (float)L.cnt) : 2.0f;
                r = fminf(r * fmaxf(grow, 1.25f), rmax);
            }
            // unkept: in the list's range -> >= lower(d_K); beyond r2acc -> >= lower(r2acc);
            // never scanned -> farther than r
            D2 = (L.cnt == K) ? fminf(lower32(L.d[K - 1]), r2lo) : fminf(lower32(r2acc), r2lo);
        }
        if (out.radius) out.radius[i] = sqrtf(L.cnt ? L.d[L.cnt - 1] : 0.0f);

        // ---- gnomonic frame at z_i: e1 x e2 = z_i
        Frame F;
        F.zi = zi;
        F.zs = g.zs;
        {
            double fx = fabs(zi.x), fy = fabs(zi.y), fz = fabs(zi.z);
            V3 ax = (fx <= fy && fx <= fz) ? mk(1, 0, 0) : ((fy <= fz) ? mk(0, 1, 0) : mk(0, 0, 1));
            V3 c = crs(zi, ax);
            F.e1 = scl(c, rsqrt(dot(c, c)));
            F.e2 = crs(zi, F.e1);
            F.e1f = make_float3((float)F.e1.x, (float)F.e1.y, (float)F.e1.z);
            F.e2f = make_float3((float)F.e2.x, (float)F.e2.y, (float)F.e2.z);
        }

        // ---- clip nearest first, with the security radius
        Poly<K, VMAX, EXTRA> P;
        P.kj = L.j;
        P.cur = 0;
        P.nv = 4;
        {
            // square lines: K right (u <= L), K+1 top (w <= L), K+2 left, K+3 bottom
            const float la[4] = {1, 0, -1, 0}, lb[4] = {0, 1, 0, -1};
            const float vu[4] = {(float)kBoxL, (float)kBoxL, -(float)kBoxL, -(float)kBoxL};
            const float vw[4] = {-(float)kBoxL, (float)kBoxL, (float)kBoxL, -(float)kBoxL};
            for (int k = 0; k < 4; ++k) {
                P.la[K + k] = la[k];
                P.lb[K + k] = lb[k];
                P.lc[K + k] = (float)kBoxL;
                P.ln[0][k] = (unsigned char)(K + k);
                P.uf[0][k] = vu[k];
                P.wf[0][k] = vw[k];
                P.ill[0][k] = 0;
            }
        }
        float R2 = chord2_up(2.0f * (float)kBoxL * (float)kBoxL);
        bool ok = true, early = false;
        for (int k = 0; k < L.cnt; ++k) {
            const float bound = fminf(lower32(L.d[k]), D2);
            if (bound > 4.0f * R2 * (1.0f + 1e-6f)) { early = true; break; }
            P.set_line(F, k, L.j[k]);
            int rc = clip<K, VMAX, EXTRA>(P, F, k, flags, &st->ambiguous);
            if (rc < 0) { ok = false; break; }
            if (rc > 0) R2 = poly_R2(P, F);
        }
        bool boxed = false;
        for (int v = 0; v < P.nv; ++v) boxed |= (P.ln[P.cur][v] >= K);  // no extra slots yet
        bool certified = ok && !boxed && (early || D2 > 4.0f * R2 * (1.0f + 1e-6f));
        if (EXTRA > 0 && ok && !certified && last_pass) {
            // last resort: clip by every generator (the exact cell); points
            // that cannot reach the polygon are skipped.  A new line goes to
            // an extra slot that no current edge uses.
            for (int q = v.p0; q < v.p0 + v.n && ok; ++q) {
                if (q == p) continue;
                const V3 d = sub(ld(g.zs + q), zi);
                if (dot(d, d) > 4.0 * (double)R2 * (1.0 + 1e-6)) continue;
                // every listed neighbour has been clipped by already: its bisector
                // may be an edge now, and clipping by a line of the polygon again
                // would solve two identical lines for a corner.  The list is sorted
                // by (FP32 d2, index) with d2 computed as here: binary search
                bool listed = false;
                if (L.cnt > 0) {
                    const float4 c = ldf(g.zf + q);
                    const float dx = c.x - zif.x, dy = c.y - zif.y, dz = c.z - zif.z;
                    const float d2f = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    int lo = 0, hi = L.cnt;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (L.d[mid] < d2f || (L.d[mid] == d2f && L.j[mid] < q)) lo = mid + 1;
                        else hi = mid;
                    }
                    listed = lo < L.cnt && L.d[lo] == d2f && L.j[lo] == q;
                }
                if (listed) continue;
                unsigned long long used = 0ull;
                for (int v = 0; v < P.nv; ++v)
                    if (P.ln[P.cur][v] >= K + 4) used |= 1ull << (P.ln[P.cur][v] - (K + 4));
                int x = __ffsll((long long)~used) - 1;
                if (x < 0 || x >= EXTRA) { ok = false; break; }
                const int l = K + 4 + x;
                P.jx[x] = q;
                P.set_line(F, l, q);
                int rc = clip<K, VMAX, EXTRA>(P, F, l, flags, &st->ambiguous);
                if (rc < 0) { ok = false; break; }
                if (rc > 0) R2 = poly_R2(P, F);
            }
            boxed = false;
            for (int v = 0; v < P.nv; ++v) boxed |= (P.ln[P.cur][v] >= K && P.ln[P.cur][v] < K + 4);
            if (ok && boxed) atomicOr(flags, FLAG_UNBOUNDED);
            certified = ok && !boxed;
        }
        if (!certified) {
            if (last_pass) {
                atomicOr(flags, ok ? FLAG_EXHAUSTED : FLAG_VMAX);
            } else {
                unsigned pos = atomicAdd(next_count, 1u);
                next_list[pos] = p;
            }
            cb.deg[p] = 0;
            continue;
        }
        // the next evaluation's first pass starts from this cell's own size
        if (out.radius) out.radius[i] = fminf(2.2f * sqrtf(R2), 2.0f);

        // ---- canonical edge order: start at the neighbour with the smallest key
        const int c = P.cur, nv = P.nv;
        int k0 = 0;
        for (int k = 1; k < nv; ++k)
            if (ckey_less(g, P.gen_of(P.ln[c][k]), P.gen_of(P.ln[c][k0]))) k0 = k;
        if (out.deg) {
            out.deg[i] = nv;
            if (nv <= out.max_deg)
                for (int t2 = 0; t2 < nv; ++t2)
                    out.nbr[(size_t)i * out.max_deg + t2] =
                        g.sidx[P.gen_of(P.ln[c][(k0 + t2 < nv) ? k0 + t2 : k0 + t2 - nv])];
        }
        // FP64 corners in canonical order; each edge's FP64 line is computed once
        double pa, pb, pc;
        P.line64(F, P.ln[c][(k0 == 0) ? nv - 1 : k0 - 1], pa, pb, pc);
        if (nv <= kCellSlots) {
            // corners are computed from these lines by k_corners
            cb.deg[p] = nv;
            for (int t2 = 0; t2 < nv; ++t2)
                cb.nb[(size_t)p * kCellSlots + t2] = P.gen_of(P.ln[c][(k0 + t2 < nv) ? k0 + t2 : k0 + t2 - nv]);
        } else {
            // large cell: integrate here, edges in the canonical order
            cb.deg[p] = 0;
            const Density rho = g.rho ? g.rho[v.b] : g.rho0;
            const double inv_alpha = rho.inv_alpha;
            const double aA1 = dot(zi, zi) - 1.0;
            Acc acc = {0, 0, 0, 0, 0};
            V3 corners_first, va;  // corners as offsets from z_i
            for (int t2 = 0; t2 <= nv; ++t2) {
                const int k = (k0 + t2) % nv;
                double a, b, cc, u, w;
                P.line64(F, P.ln[c][k], a, b, cc);
                P.meet(pa, pb, pc, a, b, cc, u, w);
                pa = a; pb = b; pc = cc;
                V3 vb = (t2 == nv) ? corners_first : project_offset(zi, aA1, add(scl(F.e1, u), scl(F.e2, w)));
                if (t2 == 0) {
                    corners_first = vb;
                } else {
                    const int kprev = (k0 + t2 - 1) % nv;
                    if (g.fan) {
                        tri(rho, inv_alpha, zi, aA1, va, vb, acc);
                    } else {
                        const V3 om = midpoint_offset(zi, aA1, ld(g.zs + P.gen_of(P.ln[c][kprev])));
                        tri(rho, inv_alpha, zi, aA1, va, om, acc);
                        tri(rho, inv_alpha, zi, aA1, om, vb, acc);
                    }
                }
                va = vb;
            }
            moment_from_offsets(zi, acc);
            write_cell(out, i, zi, acc, flags);
        }
    }
}

// ------------------------------------------------- topology, warp per cell
// The first pass gives each cell one warp, so that control flow is uniform:
// lanes scan candidate generators together, the polygon keeps one vertex
// per lane in registers, and a clip is a per-lane side test, a ballot and a
// shuffle compaction.  A vertex whose two lines meet at a small angle
// (|det| < (|a1 b2| + |a2 b1|)/30) is solved once in FP64 when it is created
// and kept rounded to FP32, so later side tests on it stay FP32-filtered.
// Differences z_j - z_i come from the FP32 pairs
// (hi, lo) of the coordinates: fl(hi_j - hi_i) is within 6e-8 of its value
// and the lo parts (<= 3e-8 each) add the rest, so d is within ~2e-7 of |d|
// and no FP64 arithmetic is needed except in rare per-lane fallbacks.  Cells
// this pass cannot certify (or with more than 16 edges, or 32 vertices at
// some point) go to the retry list of the thread-per-cell passes.

__device__ __forceinline__ float3 dfdiff(const Grid &g, int q, float4 hp, float4 lp) {
    const float4 hq = g.zf[q], lq = g.zl[q];
    return make_float3((hq.x - hp.x) + (lq.x - lp.x), (hq.y - hp.y) + (lq.y - lp.y), (hq.z - hp.z) + (lq.z - lp.z));
}

__device__ __forceinline__ void frame64(V3 zi, V3 &e1, V3 &e2) {
    double fx = fabs(zi.x), fy = fabs(zi.y), fz = fabs(zi.z);
    V3 ax = (fx <= fy && fx <= fz) ? mk(1, 0, 0) : ((fy <= fz) ? mk(0, 1, 0) : mk(0, 0, 1));
    V3 c = crs(zi, ax);
    e1 = scl(c, rsqrt(dot(c, c)));
    e2 = crs(zi, e1);
}

// FP64 line of generator `gen` (< 0: the starting square) in the frame at z_i
__device__ __forceinline__ void line_of(const Grid &g, V3 zi, V3 e1, V3 e2, int gen, double &a, double &b,
                                        double &c) {
    if (gen < 0) {
        const int k = -1 - gen;  // right, top, left, bottom
        a = (k == 0) ? 1.0 : ((k == 2) ? -1.0 : 0.0);
        b = (k == 1) ? 1.0 : ((k == 3) ? -1.0 : 0.0);
        c = kBoxL;
        return;
    }
    const V3 d = sub(ld(g.zs + gen), zi);
    a = dot(e1, d);
    b = dot(e2, d);
    c = -dot(zi, d);
}

// FP64 vertex of lines (gin, gout) at cell p
__device__ __forceinline__ void vertex64(const Grid &g, int p, int gin, int gout, double &u, double &w) {
    const V3 zi = ld(g.zs + p);
    V3 e1, e2;
    frame64(zi, e1, e2);
    double a1, b1, c1, a2, b2, c2;
    line_of(g, zi, e1, e2, gin, a1, b1, c1);
    line_of(g, zi, e1, e2, gout, a2, b2, c2);
    double inv = 1.0 / (a1 * b2 - a2 * b1);
    u = (c1 * b2 - c2 * b1) * inv;
    w = (a1 * c2 - a2 * c1) * inv;
}

// FP64 side test of vertex (gin, gout) against generator gnew: true = outside
__device__ bool outside64(const Grid &g, int p, int gin, int gout, int gnew, unsigned long long *amb) {
    const V3 zi = ld(g.zs + p);
    V3 e1, e2;
    frame64(zi, e1, e2);
    double a1, b1, c1, a2, b2, c2, a, b, c;
    line_of(g, zi, e1, e2, gin, a1, b1, c1);
    line_of(g, zi, e1, e2, gout, a2, b2, c2);
    line_of(g, zi, e1, e2, gnew, a, b, c);
    double inv = 1.0 / (a1 * b2 - a2 * b1);
    double u = (c1 * b2 - c2 * b1) * inv;
    double w = (a1 * c2 - a2 * c1) * inv;
    double sd = a * u + b * w - c;
    if (fabs(sd) <= 1e-14 * (fabs(a * u) + fabs(b * w) + fabs(c))) atomicAdd(amb, 1ull);
    return sd > 0.0;
}


// append every q in [q0, q1), q != p, with d2 <= r2acc, scanned by the L lanes
// of a sub-warp (lane sl, first lane sbase, mask smask); cnt may exceed 2L
template <int L>
__device__ __forceinline__ int gather(const Grid &g, int p, float4 hp, float4 lp, int q0, int q1, float r2acc, int cnt,
                                      float *cd, int *cj, int sl, int sbase, unsigned smask, unsigned *flags) {
    constexpr unsigned lfull = (L == 32) ? 0xffffffffu : ((1u << L) - 1u);
    for (int base = q0; base < q1; base += L) {
        const int q = base + sl;
        bool pred = false;
        float d2 = 0.0f;
        if (q < q1 && q != p) {
            const float3 d = dfdiff(g, q, hp, lp);
            d2 = fmaf(d.x, d.x, fmaf(d.y, d.y, d.z * d.z));
            if (d2 == 0.0f) check_duplicate(g, ld(g.zs + p), q, flags);
            pred = d2 <= r2acc;
        }
        const unsigned m = (__ballot_sync(smask, pred) >> sbase) & lfull;
        const int pos = cnt + __popc(m & ((1u << sl) - 1u));
        if (pred && pos < 2 * L) {
            cd[pos] = d2;
            cj[pos] = q;
        }
        cnt += __popc(m);
    }
    return cnt;
}

// append every generator of up to L bin rows, scanned as one list: lane k < nr
// holds row k's range [q0, q0 + len); the L lanes of the sub-warp take the
// rows' generators L at a time in row order, so the candidates arrive in the
// same order as row by row, with fewer partly filled rounds and the rows'
// ranges loaded in one round.  (Faster on the small caps of cells with radius
// hints; the large caps of a random start's first evaluations take longer
// than row by row.)
template <int L>
__device__ __forceinline__ int gather_rows(const Grid &g, int p, float4 hp, float4 lp, int q0, int len, int nr,
                                           float r2acc, int cnt, float *cd, int *cj, int sl, int sbase, unsigned smask,
                                           unsigned *flags) {
    constexpr unsigned lfull = (L == 32) ? 0xffffffffu : ((1u << L) - 1u);
    int inc = len;
#pragma unroll
    for (int o = 1; o < L; o <<= 1) {
        const int t = __shfl_up_sync(smask, inc, o, L);
        if (sl >= o) inc += t;
    }
    const int total = __shfl_sync(smask, inc, L - 1, L);
    const int pre = inc - len;  // first list position of this lane's row
    for (int base = 0; base < total; base += L) {
        const int f = base + sl;
        // the row holding position f: the last k < nr with pre_k <= f (pre is
        // non-decreasing; a binary search in log2(L) shuffles)
        int k = 0;
#pragma unroll
        for (int step = L / 2; step > 0; step >>= 1) {
            const int c = k + step;
            const int pc = __shfl_sync(smask, pre, c < L ? c : L - 1, L);
            if (c < nr && pc <= f) k = c;
        }
        const int q = __shfl_sync(smask, q0, k, L) + f - __shfl_sync(smask, pre, k, L);
        bool pred = false;
        float d2 = 0.0f;
        if (f < total && q != p) {
            const float3 d = dfdiff(g, q, hp, lp);
            d2 = fmaf(d.x, d.x, fmaf(d.y, d.y, d.z * d.z));
            if (d2 == 0.0f) check_duplicate(g, ld(g.zs + p), q, flags);
            pred = d2 <= r2acc;
        }
        const unsigned m = (__ballot_sync(smask, pred) >> sbase) & lfull;
        const int pos = cnt + __popc(m & ((1u << sl) - 1u));
        if (pred && pos < 2 * L) {
            cd[pos] = d2;
            cj[pos] = q;
        }
        cnt += __popc(m);
    }
    return cnt;
}

// WPB warps per block, L lanes per cell (32: one cell per warp, 16: two);
// every collective runs on the cell's sub-warp.  knn_target: the number of
// candidates the first radius aims at when the cell has no radius hint.
// At most 64 registers a thread (32 warps per SM): the few spills cost less
// than the occupancy they buy (2-10 % faster than at 80 registers).
template <int WPB, int L>
__global__ void __launch_bounds__(WPB * 32, 32 / WPB) k_topo_warp(Grid g, CellOut out, CellBuf cb, int *__restrict__ next_list,
                                                        unsigned *__restrict__ next_count, DevStatus *st,
                                                        float knn_target, int pbeg, int pend) {
    constexpr int C = 2 * L;  // candidate slots per cell
    constexpr unsigned lfull = (L == 32) ? 0xffffffffu : ((1u << L) - 1u);
    __shared__ float s_d2[WPB * 32 / L][C];
    __shared__ int s_j[WPB * 32 / L][C];
    __shared__ float4 s_ln[WPB * 32 / L][L];
    const int lane = threadIdx.x & 31;
    const int sl = lane & (L - 1), sbase = lane & ~(L - 1);
    const unsigned smask = lfull << sbase;
    float *cd = s_d2[threadIdx.x / L];
    int *cj = s_j[threadIdx.x / L];
    float4 *ln = s_ln[threadIdx.x / L];
    const int gs = (blockIdx.x * blockDim.x + threadIdx.x) / L;
    const int ns = (gridDim.x * blockDim.x) / L;
    const float INF = __int_as_float(0x7f800000);
    for (int p = pbeg + gs; p < pend; p += ns) {
        const View v = view_of(g, p);
        if (inactive(g, v.b)) {
            if (sl == 0) cb.deg[p] = 0;
            continue;
        }
        unsigned *flags = flags_of(g, st, v.b);
        const float4 hp = g.zf[p], lp = g.zl[p];
        const int i = g.sidx[p];
        // FP32 frame (any orthonormal frame gives the same vertex directions)
        float3 e1, e2;
        {
            const float fx = fabsf(hp.x), fy = fabsf(hp.y), fz = fabsf(hp.z);
            float3 ax = (fx <= fy && fx <= fz) ? make_float3(1, 0, 0)
                                               : ((fy <= fz) ? make_float3(0, 1, 0) : make_float3(0, 0, 1));
            float3 c = make_float3(hp.y * ax.z - hp.z * ax.y, hp.z * ax.x - hp.x * ax.z, hp.x * ax.y - hp.y * ax.x);
            const float inv = rsqrtf(c.x * c.x + c.y * c.y + c.z * c.z);
            e1 = make_float3(c.x * inv, c.y * inv, c.z * inv);
            e2 = make_float3(hp.y * e1.z - hp.z * e1.y, hp.z * e1.x - hp.x * e1.z, hp.x * e1.y - hp.y * e1.x);
        }
        const bool all_mode = v.n - 1 <= C;
        // caps up to chord rmax are cube-map queries (sin(theta) <= 0.28 keeps
        // them off the far faces); wider ones, for cells that large, scan every
        // generator of the problem (chord 2 takes them all) in problems of up to
        // 131,072 generators, where such cells occur; in larger problems the
        // thread passes take a cell that needs more than rmax
        const float rmax = 0.2829f, rwide = (v.n <= (1 << 17)) ? 2.0f : rmax;
        float r;
        {
            const float hint = hp.w;  // the radius hint travels with the coordinates
            if (hint > 0.0f) {
                r = hint;
            } else {
                const int b = bin_index(hp.x, hp.y, hp.z, v.G);
                const int cbn = v.bstart[b + 1] - v.bstart[b];
                const float ax = fabsf(hp.x), ay = fabsf(hp.y), az = fabsf(hp.z);
                const float am = fmaxf(ax, fmaxf(ay, az));
                const float s2 = (ax * ax + ay * ay + az * az) / (am * am);
                const float omega = (4.0f / ((float)v.G * v.G)) / (s2 * sqrtf(s2));
                r = sqrtf(knn_target * omega / (3.14159265f * fmaxf((float)cbn, 1.0f)));
            }
            r = fminf(r, rwide);
        }
        bool certified = false, ok = true;
        int nv = 0;
        float R2 = 0.0f;
        // polygon: sub-warp lane k < nv holds vertex k and its outgoing edge's line
        float vu = 0.0f, vw = 0.0f, la_o = 0.0f, lb_o = 0.0f, lc_o = 0.0f;
        int vill = 0, g_o = 0, g_i = 0;
        for (int attempt = 0; attempt < 8 && ok && !certified; ++attempt) {
            // ---- candidates within chord r (every one of them; the rest are farther than r)
            const float rs = r * (1.0f + 1e-5f) + 1e-7f;  // covers the FP32 centre
            const float S = rs * sqrtf(fmaxf(1.0f - 0.25f * rs * rs, 0.0f)) * (1.0f + 1e-5f);
            const float r2acc = all_mode ? INF : r * r * 1.001f;
            const float D2 = (all_mode || r >= 2.0f) ? INF : r * r * (1.0f - 1e-6f);  // chord 2: every generator
            int cnt = 0;
            if (all_mode || r > rmax) {
                cnt = gather<L>(g, p, hp, lp, v.p0, v.p0 + v.n, r2acc, cnt, cd, cj, sl, sbase, smask, flags);
            } else {
                const float S2 = S * S;
                const float qv[3] = {hp.x, hp.y, hp.z};
                for (int a = 0; a < 3; ++a) {
                    const float qa = qv[a];
                    const float A = qa * qa - S2;
                    if (A <= 0.0f || fabsf(qa) + S + 1e-6f < 0.5773f) continue;  // cap off face a
                    const float sg = qa > 0.0f ? 1.0f : -1.0f;
                    const int face = 2 * a + (qa < 0.0f ? 1 : 0);
                    const float invA = 1.0f / A;
                    const float margin = 4e-6f * invA + 1e-6f;
                    int lo[2], hi[2];
                    bool empty = false;
                    for (int rr = 0; rr < 2; ++rr) {
                        const float qb = qv[(a + 1 + rr) % 3];
                        const float rt = S * sqrtf(fmaxf(qa * qa + qb * qb - S2, 0.0f));
                        float s0 = (sg * qa * qb - rt) * invA - margin;
                        float s1 = (sg * qa * qb + rt) * invA + margin;
                        if (s0 > 1.0f || s1 < -1.0f) { empty = true; break; }
                        s0 = fmaxf(s0, -1.0f);
                        s1 = fminf(s1, 1.0f);
                        lo[rr] = min(max((int)floorf((s0 + 1.0f) * 0.5f * v.G), 0), v.G - 1);
                        hi[rr] = min(max((int)floorf((s1 + 1.0f) * 0.5f * v.G), 0), v.G - 1);
                    }
                    if (empty) continue;
                    // the face's bin rows lo[1] .. hi[1], up to L at a time
                    for (int iv0 = lo[1]; iv0 <= hi[1]; iv0 += L) {
                        const int nr = min(L, hi[1] - iv0 + 1);
                        int q0 = 0, len = 0;
                        if (sl < nr) {
                            const int row = (face * v.G + iv0 + sl) * v.G;
                            q0 = v.bstart[row + lo[0]];
                            len = v.bstart[row + hi[0] + 1] - q0;
                        }
                        cnt = gather_rows<L>(g, p, hp, lp, q0, len, nr, r2acc, cnt, cd, cj, sl, sbase, smask, flags);
                    }
                }
            }
            __syncwarp(smask);
            if (cnt > C) {
                // too many: the cap that holds about 90 % of the slots (counts
                // grow as r^2), at least halving r; the bound stays r-based
                r *= fmaxf(0.5f, sqrtf(0.9f * (float)C / (float)cnt));
                continue;
            }
            if (cnt < 3 && !all_mode && r < rwide) {
                r = fminf(r * 2.0f, rwide);
                continue;
            }
            bool early = false, fast = false;
            if (cnt <= L) {
                // ---- all lines at once: lane l holds candidate l's line and
                // proposes the piece of it inside every other line, the lines
                // bounding that piece at its two ends being its polygon
                // neighbours.  The proposal is then certified with the clipping
                // test's own FP32 filter: every proposed vertex well conditioned and
                // strictly inside every other line, the neighbour links one
                // counter-clockwise cycle.  Then it is the exact cell.  A
                // polygon the candidates leave open has lines with an unbounded
                // piece, which breaks the cycle; such cells, like any other that
                // fails, are clipped one candidate at a time from the square below.
                const int nl = cnt;
                float fa = 0.0f, fb = 0.0f, fc = 0.0f;
                int gen = 0;
                if (sl < cnt) {
                    gen = cj[sl];
                    const float3 d = dfdiff(g, gen, hp, lp);
                    fa = e1.x * d.x + e1.y * d.y + e1.z * d.z;
                    fb = e2.x * d.x + e2.y * d.y + e2.z * d.z;
                    fc = 0.5f * fmaf(d.x, d.x, fmaf(d.y, d.y, d.z * d.z));
                }
                ln[sl] = make_float4(fa, fb, fc, 0.0f);
                __syncwarp(smask);
                // line l: the point pu, pw on it, direction (-fb, fa) (counter-clockwise
                // along the boundary); line i bounds the parameter t by h / s
                const float n2 = fa * fa + fb * fb;
                const float pu = __fdividef(fc * fa, n2), pw = __fdividef(fc * fb, n2);
                float tmax = INF, tmin = -INF;
                int imax = -1, imin = -1;
                bool infeasible = false;
                for (int i = 0; i < nl; ++i) {
                    const float4 li = ln[i];
                    const float sv = li.y * fa - li.x * fb;
                    const float h = li.z - fmaf(li.x, pu, li.y * pw);
                    const float t = __fdividef(h, sv);
                    if (i != sl) {
                        if (sv > 0.0f) {
                            if (t < tmax) { tmax = t; imax = i; }
                        } else if (sv < 0.0f) {
                            if (t > tmin) { tmin = t; imin = i; }
                        } else if (h < 0.0f) {
                            infeasible = true;
                        }
                    }
                }
                const bool present = sl < nl && !infeasible && imax >= 0 && imin >= 0 && tmin < tmax;
                const unsigned pm = (__ballot_sync(smask, present) >> sbase) & lfull;
                const int m = __popc(pm);
                const int nx = present ? imax : sl;  // successor (counter-clockwise)
                const int pv = __shfl_sync(smask, imin, sbase + (nx & (L - 1)));
                bool good = !present || ((((pm >> nx) & 1u) != 0u) && pv == sl);
                int pos = -1;
                if (m >= 3) {
                    const int start = __ffs(pm) - 1;
                    int cur = start;
                    if (sl == start) pos = 0;
                    for (int k = 1; k < m; ++k) {
                        cur = __shfl_sync(smask, nx, sbase + cur);
                        if (sl == cur) pos = k;
                    }
                    cur = __shfl_sync(smask, nx, sbase + cur);
                    good = good && cur == start && (!present || pos >= 0);
                } else {
                    good = false;
                }
                float r2v = 0.0f;
                if (good && present) {
                    const float4 ls = ln[nx];
                    const float p1 = fa * ls.y, p2 = ls.x * fb, det = p1 - p2;
                    if (!(det > 0.0f) || !(fabsf(det) * 30.0f >= fabsf(p1) + fabsf(p2))) {
                        good = false;
                    } else {
                        const float inv = __fdividef(1.0f, det);
                        const float xu = (fc * ls.y - ls.z * fb) * inv;
                        const float xw = (fa * ls.z - ls.x * fc) * inv;
                        const float su = fabsf(xu) + fabsf(xw);
                        for (int i = 0; i < nl; ++i) {
                            const float4 li = ln[i];
                            const float sd = fmaf(li.x, xu, fmaf(li.y, xw, -li.z));
                            const float mag = (fabsf(li.x) + fabsf(li.y)) * su + fabsf(li.z);
                            if (i != sl && i != nx && !(sd < -2e-4f * mag)) good = false;
                        }
                        r2v = xu * xu + xw * xw;
                    }
                }
                fast = ((__ballot_sync(smask, !good) >> sbase) & lfull) == 0u;
                if (fast) {
                    // lane k takes the edge at position k of the cycle
                    if (present) cj[pos] = sl;
                    __syncwarp(smask);
                    const int from = (sl < m) ? cj[sl] : sl;
                    g_o = __shfl_sync(smask, gen, sbase + (from & (L - 1)));
                    nv = m;
#pragma unroll
                    for (int o = L / 2; o > 0; o >>= 1) r2v = fmaxf(r2v, __shfl_xor_sync(smask, r2v, o));
                    R2 = r2v * (1.001f * (1.0f + 1e-5f));
                }
                __syncwarp(smask);
            }
            if (!fast) {
            // ---- sort the candidates once by (d2, index), a total order, so the
            // result does not depend on the network: up to L candidates one per
            // lane over the next power of two >= cnt; more, two per lane over 2L
            if (cnt <= L) {
                int S = 2;
                while (S < cnt) S <<= 1;
                float dv = (sl < cnt) ? cd[sl] : INF;
                int jv = (sl < cnt) ? cj[sl] : 0x7fffffff;
                __syncwarp(smask);
                for (int k = 2; k <= S; k <<= 1) {
                    for (int j = k >> 1; j > 0; j >>= 1) {
                        const float od = __shfl_xor_sync(smask, dv, j);
                        const int oj = __shfl_xor_sync(smask, jv, j);
                        const bool ascending = (sl & k) == 0, lower = (sl & j) == 0;
                        const bool other_less = od < dv || (od == dv && oj < jv);
                        if ((lower == ascending) ? other_less : !other_less) {
                            dv = od;
                            jv = oj;
                        }
                    }
                }
                cd[sl] = dv;
                cj[sl] = jv;
                __syncwarp(smask);
            } else {
                float cdd[2];
                int cjj[2];
#pragma unroll
                for (int s2 = 0; s2 < 2; ++s2) {
                    const int idx = 2 * sl + s2;
                    cdd[s2] = (idx < cnt) ? cd[idx] : INF;
                    cjj[s2] = (idx < cnt) ? cj[idx] : 0x7fffffff;
                }
                __syncwarp(smask);
#pragma unroll
                for (int k = 2; k <= C; k <<= 1) {
#pragma unroll
                    for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
                        for (int s2 = 0; s2 < 2; ++s2) {
                            const int e = 2 * sl + s2;
                            float od;
                            int oj;
                            if (j == 1) {
                                od = cdd[s2 ^ 1];
                                oj = cjj[s2 ^ 1];
                            } else {
                                // partner lane sl ^ (j / 2): inside the sub-warp
                                od = __shfl_xor_sync(smask, cdd[s2], j >> 1);
                                oj = __shfl_xor_sync(smask, cjj[s2], j >> 1);
                            }
                            const bool ascending = (e & k) == 0, lower = (e & j) == 0;
                            const bool other_less = od < cdd[s2] || (od == cdd[s2] && oj < cjj[s2]);
                            const bool take = (lower == ascending) ? other_less : !other_less;
                            if (j == 1) {
                                // both slots of the lane are the pair: decide once, from slot 0
                                if (s2 == 0) {
                                    if (take) {
                                        const float td = cdd[0];
                                        const int tj = cjj[0];
                                        cdd[0] = cdd[1]; cjj[0] = cjj[1];
                                        cdd[1] = td; cjj[1] = tj;
                                    }
                                }
                            } else if (take) {
                                cdd[s2] = od;
                                cjj[s2] = oj;
                            }
                        }
                    }
                }
                // sorted order back to shared memory: step t reads slot t by broadcast
#pragma unroll
                for (int s2 = 0; s2 < 2; ++s2) {
                    cd[2 * sl + s2] = cdd[s2];
                    cj[2 * sl + s2] = cjj[s2];
                }
                __syncwarp(smask);
            }
            // ---- the starting square
            nv = 4;
            {
                const float Lb = (float)kBoxL;
                vu = (sl == 0 || sl == 1) ? Lb : -Lb;
                vw = (sl == 1 || sl == 2) ? Lb : -Lb;
                la_o = (sl == 0) ? 1.0f : ((sl == 2) ? -1.0f : 0.0f);
                lb_o = (sl == 1) ? 1.0f : ((sl == 3) ? -1.0f : 0.0f);
                lc_o = Lb;
                g_o = -1 - sl;
                g_i = -1 - ((sl + 3) & 3);
                vill = 0;
            }
            R2 = chord2_up(2.0f * (float)kBoxL * (float)kBoxL);
            const int ncand = min(cnt, C);
            for (int t = 0; t < ncand; ++t) {
                // candidate t (nearest first)
                const float wd = cd[t];
                const int wj = cj[t];
                // security radius: everything left is at least this far
                const float bound = fminf(wd * (1.0f - 2e-6f), D2);
                if (bound > 4.0f * R2 * (1.0f + 1e-6f)) { early = true; break; }
                // the bisector of (z_i, z_wj) as a line a u + b w <= c
                const float3 d = dfdiff(g, wj, hp, lp);
                const float la = e1.x * d.x + e1.y * d.y + e1.z * d.z;
                const float lb = e2.x * d.x + e2.y * d.y + e2.z * d.z;
                const float lc = 0.5f * fmaf(d.x, d.x, fmaf(d.y, d.y, d.z * d.z));
                bool outside = false;
                if (sl < nv) {
                    const float sd = fmaf(la, vu, fmaf(lb, vw, -lc));
                    const float mag = (fabsf(la) + fabsf(lb)) * (fabsf(vu) + fabsf(vw)) + fabsf(lc);
                    if (!vill && fabsf(sd) > 2e-4f * mag) outside = sd > 0.0f;
                    else outside = outside64(g, p, g_i, g_o, wj, &st->ambiguous);
                }
                const unsigned m = (__ballot_sync(smask, outside) >> sbase) & lfull;
                if (m == 0u) continue;
                const unsigned full = (nv == 32) ? 0xffffffffu : ((1u << nv) - 1u);
                if (m == full) {
                    if (sl == 0) atomicOr(flags, FLAG_EMPTY);
                    ok = false;
                    break;
                }
                const unsigned rot = ((m << 1) | (m >> (nv - 1))) & full;  // bit k = bit k-1 of m
                const unsigned starts = m & ~rot;
                if (__popc(starts) > 1 && sl == 0) atomicOr(flags, FLAG_NONCONVEX);
                // indices mod nv by one conditional subtraction (operands < 2 nv)
                const int k0 = __ffs(starts) - 1;
                const unsigned mr = (k0 == 0) ? m : (((m >> k0) | (m << (nv - k0))) & full);
                const int runlen = __ffs(~mr) - 1;
                const int k1r = k0 + runlen - 1;
                const int k1 = (k1r >= nv) ? k1r - nv : k1r;
                const int kin = (k0 == 0) ? nv - 1 : k0 - 1;
                const int nnew = nv - runlen + 2;
                if (nnew > L) { ok = false; break; }
                const float ai = __shfl_sync(smask, la_o, sbase + kin), bi = __shfl_sync(smask, lb_o, sbase + kin),
                            ci = __shfl_sync(smask, lc_o, sbase + kin);
                const int gkin = __shfl_sync(smask, g_o, sbase + kin);
                // new vertices P = (edge kin) x (new line), Q = (new line) x (edge k1);
                // lanes 2 .. nnew-1 take the surviving vertices k1+1 .. kin (k1 + sl - 1
                // < 2 nv there); the lanes above carry any lane's values, unused
                const int sr = (sl >= 2) ? k1 + sl - 1 : k1;
                const int src = sbase + (((sr >= nv) ? sr - nv : sr) & (L - 1));
                const float su = __shfl_sync(smask, vu, src), sw = __shfl_sync(smask, vw, src);
                const int sill = __shfl_sync(smask, vill, src), sg = __shfl_sync(smask, g_o, src);
                const int sgi = __shfl_sync(smask, g_i, src);
                const float sa = __shfl_sync(smask, la_o, src), sb = __shfl_sync(smask, lb_o, src),
                            sc = __shfl_sync(smask, lc_o, src);
                if (sl < 2) {
                    // lane 0: P meets lines (kin, new); lane 1: Q meets lines (new, k1's outgoing)
                    const bool l0 = sl == 0;
                    const float a1 = l0 ? ai : la, b1 = l0 ? bi : lb, c1 = l0 ? ci : lc;
                    const float a2 = l0 ? la : sa, b2 = l0 ? lb : sb, c2 = l0 ? lc : sc;
                    const int gA = l0 ? gkin : wj, gB = l0 ? wj : sg;
                    const float p1 = a1 * b2, p2 = a2 * b1, det = p1 - p2, inv = __fdividef(1.0f, det);
                    vu = (c1 * b2 - c2 * b1) * inv;
                    vw = (a1 * c2 - a2 * c1) * inv;
                    vill = 0;
                    if (!(fabsf(det) * 30.0f >= fabsf(p1) + fabsf(p2))) {
                        // poorly conditioned in FP32: solve once in FP64, keep the rounded vertex
                        double u, w;
                        vertex64(g, p, gA, gB, u, w);
                        vu = (float)u;
                        vw = (float)w;
                    }
                    la_o = l0 ? la : sa; lb_o = l0 ? lb : sb; lc_o = l0 ? lc : sc;
                    g_o = gB; g_i = gA;
                } else {
                    vu = su; vw = sw; vill = sill; la_o = sa; lb_o = sb; lc_o = sc; g_o = sg; g_i = sgi;
                }
                nv = nnew;
                // R2: an upper bound of the largest squared vertex chord; the
                // squared gnomonic radius t^2 bounds the squared chord
                // 2 - 2 / sqrt(1 + t^2) of its point from above
                float r2v = (sl < nv) ? vu * vu + vw * vw : 0.0f;
#pragma unroll
                for (int o = L / 2; o > 0; o >>= 1) r2v = fmaxf(r2v, __shfl_xor_sync(smask, r2v, o));
                R2 = r2v * (1.001f * (1.0f + 1e-5f));
            }
            if (!ok) break;
            }
            const bool boxed = ((__ballot_sync(smask, sl < nv && g_o < 0) >> sbase) & lfull) != 0u;
            certified = !boxed && (early || D2 > 4.0f * R2 * (1.0f + 1e-6f));
            if (!certified) {
                if (all_mode || r >= rwide) break;
                // an open polygon says nothing of the cell's size: widen the cap; a
                // closed one needs chord 2 sqrt(R2) (taken with 2.5 % to spare, so
                // that large cells' caps still fit the slots), but R2 of a polygon
                // clipped by too few candidates overstates the cell, so grow at
                // most twofold
                r = boxed ? fminf(2.0f * r, rwide)
                          : fminf(fmaxf(fminf(2.05f * sqrtf(R2), 2.0f * r), 1.25f * r), rwide);
            }
        }
        if (!certified || nv > kCellSlots) {
            if (sl == 0) {
                unsigned pos = atomicAdd(next_count, 1u);
                next_list[pos] = p;
                cb.deg[p] = 0;
            }
            continue;
        }
        // ---- canonical order: start at the neighbour with the smallest key
        // (hi.x, lo.x, hi.y, lo.y, hi.z, lo.z) of its FP32 pair coordinates, a
        // function of the point alone; the first key decides unless it ties
        int best;
        {
            unsigned k0 = 0xffffffffu;
            float4 nh = make_float4(0, 0, 0, 0);
            if (sl < nv) {
                nh = g.zf[g_o];
                k0 = okey32(nh.x);
            }
            const unsigned kmin = __reduce_min_sync(smask, k0);
            const unsigned tie = (__ballot_sync(smask, k0 == kmin) >> sbase) & lfull;
            best = __ffs(tie) - 1;
            if (__popc(tie) > 1) {
                // rare: resolve on the whole key among the tied lanes
                unsigned long long kx = ~0ull, ky = kx, kz = kx;
                if ((tie >> sl) & 1u) {
                    const float4 nl = g.zl[g_o];
                    kx = ((unsigned long long)okey32(nh.x) << 32) | okey32(nl.x);
                    ky = ((unsigned long long)okey32(nh.y) << 32) | okey32(nl.y);
                    kz = ((unsigned long long)okey32(nh.z) << 32) | okey32(nl.z);
                }
                best = sl;
#pragma unroll
                for (int o = L / 2; o > 0; o >>= 1) {
                    const unsigned long long ox = __shfl_xor_sync(smask, kx, o), oy = __shfl_xor_sync(smask, ky, o),
                                             oz = __shfl_xor_sync(smask, kz, o);
                    const int ob = __shfl_xor_sync(smask, best, o);
                    const bool less =
                        ox < kx || (ox == kx && (oy < ky || (oy == ky && (oz < kz || (oz == kz && ob < best)))));
                    if (less) { kx = ox; ky = oy; kz = oz; best = ob; }
                }
            }
        }
        const int rgs = best + sl;  // < 2 nv on the lanes that keep it
        const int rg = __shfl_sync(smask, g_o, sbase + (((rgs >= nv) ? rgs - nv : rgs) & (L - 1)));
        if (sl < nv) {
            cb.nb[(size_t)p * kCellSlots + sl] = rg;
            if (out.deg && nv <= out.max_deg) out.nbr[(size_t)i * out.max_deg + sl] = g.sidx[rg];
        }
        if (sl == 0) {
            cb.deg[p] = nv;
            if (out.deg) out.deg[i] = nv;
            if (out.radius) out.radius[i] = fminf(2.2f * sqrtf(R2), rwide);
        }
    }
}

// z_q - z_p as a double-float from the three FP32 parts of each coordinate
// (both differences of parts are exact by TwoSum; the third parts are tiny)
__device__ __forceinline__ df3 gen_diff(const Grid &g, int q, float4 hp, float4 lp, float4 llp) {
    const float4 hq = g.zf[q], lq = g.zl[q], llq = g.zll[q];
    return df3{df_norm(dfl_add_f(dfl_add(two_sum(hq.x, -hp.x), two_sum(lq.x, -lp.x)), llq.x - llp.x)),
               df_norm(dfl_add_f(dfl_add(two_sum(hq.y, -hp.y), two_sum(lq.y, -lp.y)), llq.y - llp.y)),
               df_norm(dfl_add_f(dfl_add(two_sum(hq.z, -hp.z), two_sum(lq.z, -lp.z)), llq.z - llp.z))};
}

// 1/|x| - 1 for delta = 1 - |x|^2 <= 1e-3 (binomial series, exact to 3e-19)
__device__ __forceinline__ df inv_norm_m1(df dl) {
    const df d2 = dfl_mul(dl, dl);
    const float tail = d2.hi * dl.hi * (0.3125f + dl.hi * (0.2734375f + dl.hi * 0.24609375f));
    return df_norm(dfl_add_f(dfl_add(df{0.5f * dl.hi, 0.5f * dl.lo}, dfl_mul_f(d2, 0.375f)), tail));
}

// FP64 line of neighbour gen in the frame at z_i for the corners: (a, b) =
// (e1.d, e2.d), d = z_j - z_i, and c = -z_i.d taken as (|d|^2 + (|z_i|^2 - 1)
// - (|z_j|^2 - 1)) / 2 with the exact |z|^2 - 1 of the binning (zll[].w):
// the dot product -z_i.d cancels to |d|^2 / 2 and would carry an error of
// 1e-16 |d|, a relative 2e-16 / |d| of the line's offset, which moves the
// corners of close neighbours by ~1e-16 -- up to 1e-12 of a small cell's
// energy.  Without zll (mixed form) the dot product is used.
__device__ __forceinline__ void corner_line64(const Grid &g, int p, V3 zi, V3 e1, V3 e2, int gen, double &a,
                                              double &b, double &c) {
    const V3 d = sub(ld(g.zs + gen), zi);
    a = dot(e1, d);
    b = dot(e2, d);
    c = g.zll ? 0.5 * (dot(d, d) + ((double)g.zll[p].w - (double)g.zll[gen].w)) : -dot(zi, d);
}

// Corner of every edge: vertex k of a cell is where the bisector planes of
// edges k-1 and k meet the plane z_i + u e1 + w e2 (then projected).
// Double-float path: e1, e2 are any FP32 vectors spanning a plane through
// z_i (the two bisector planes meet in a line through the origin, which
// crosses it at the corner's direction whatever the tilt); the line of
// neighbour j is a u + b w = c with (a, b) = (e1.d, e2.d), d = z_j - z_i from
// the three-part coordinates, and c = -z_i.d = (|d|^2 + (|z_i|^2 - 1) -
// (|z_j|^2 - 1)) / 2 without cancellation.  The 2x2 solve (well conditioned:
// |det| >= (|a1 b2| + |a2 b1|) / 8, so the pairs' 2^-47 stays below 3e-14 of
// u and w) gives the offset x - z_i = u e1 + w e2;
// projecting, v - z_i = (1 + m)(x - z_i) + m z_i with m = 1/|x| - 1 from
// delta = -(|z_i|^2 - 1) - 2 z_i.(x - z_i) - |x - z_i|^2.  Corners farther
// than chord 0.03 or poorly conditioned, and every corner of the plain FP64
// form, are solved in FP64 in the gnomonic frame at z_i and projected the
// same way (project_offset).  The cell buffer keeps each corner as its
// offset v - z_i in FP64, exact to rounding relative to the cell's size
// (an absolute unit vector would carry 1e-16 of absolute error, up to 1e-12
// of the smallest cells' energies).
// Corner slots: FP64 offsets v - z_i (P4) in the plain FP64 form; in the
// FP64 form the same 32 bytes hold the offset as double-float pairs (hi.x,
// hi.y, hi.z, lo.x | lo.y, lo.z), the form the quadrature computes in.
__device__ __forceinline__ void store_corner_df(P4 *slot, df3 o) {
    float4 *f = reinterpret_cast<float4 *>(slot);
    f[0] = make_float4(o.x.hi, o.y.hi, o.z.hi, o.x.lo);
    f[1] = make_float4(o.y.lo, o.z.lo, 0.0f, 0.0f);
}
__device__ __forceinline__ df3 load_corner_df(const P4 *slot) {
    const float4 *f = reinterpret_cast<const float4 *>(slot);
    const float4 a = f[0], b = f[1];
    return df3{df{a.x, a.w}, df{a.y, b.x}, df{a.z, b.y}};
}

template <bool PLAIN>
__global__ void __launch_bounds__(256) k_corners(Grid g, CellBuf cb, Span sp) {
    const int ne = *sp.etot, eb = *sp.e0;
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < ne; it += gridDim.x * blockDim.x) {
        const int e = eb + it;
        const int p = cb.ecell[e];
        const int k = e - cb.eoff[p];
        const int deg = cb.deg[p];
        const int *nb = cb.nb + (size_t)p * kCellSlots;
        const int ga = nb[(k == 0) ? deg - 1 : k - 1], gb = nb[k];
        const V3 zi = ld(g.zs + p);
        if constexpr (!PLAIN) {
            const float4 hp = g.zf[p], lp = g.zl[p], llp = g.zll[p];
            float3 e1, e2;
            {
                const float fx = fabsf(hp.x), fy = fabsf(hp.y), fz = fabsf(hp.z);
                const float3 ax = (fx <= fy && fx <= fz) ? make_float3(1, 0, 0)
                                                         : ((fy <= fz) ? make_float3(0, 1, 0) : make_float3(0, 0, 1));
                const float3 c = make_float3(hp.y * ax.z - hp.z * ax.y, hp.z * ax.x - hp.x * ax.z,
                                             hp.x * ax.y - hp.y * ax.x);
                const float inv = rsqrtf(c.x * c.x + c.y * c.y + c.z * c.z);
                e1 = make_float3(c.x * inv, c.y * inv, c.z * inv);
                e2 = make_float3(hp.y * e1.z - hp.z * e1.y, hp.z * e1.x - hp.x * e1.z, hp.x * e1.y - hp.y * e1.x);
            }
            df la[2], lb[2], lc[2];
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int q = t == 0 ? ga : gb;
                const df3 d = gen_diff(g, q, hp, lp, llp);
                // unnormalized chains (dfl_*), normalized where sums cancel
                la[t] = df_norm(dfl_add(dfl_add(dfl_mul_f(d.x, e1.x), dfl_mul_f(d.y, e1.y)), dfl_mul_f(d.z, e1.z)));
                lb[t] = df_norm(dfl_add(dfl_add(dfl_mul_f(d.x, e2.x), dfl_mul_f(d.y, e2.y)), dfl_mul_f(d.z, e2.z)));
                const df c2 = df_norm(dfl_add_f(df3_dot_n(d, d), llp.w - g.zll[q].w));
                lc[t] = df{0.5f * c2.hi, 0.5f * c2.lo};
            }
            const df p1 = dfl_mul(la[0], lb[1]), p2 = dfl_mul(la[1], lb[0]);
            const df det = df_norm(dfl_add(p1, df_neg(p2)));
            if (fabsf(det.hi) * 8.0f >= fabsf(p1.hi) + fabsf(p2.hi)) {
                const df u = df_div(df_norm(dfl_add(dfl_mul(lc[0], lb[1]), df_neg(dfl_mul(lc[1], lb[0])))), det);
                const df w = df_div(df_norm(dfl_add(dfl_mul(la[0], lc[1]), df_neg(dfl_mul(la[1], lc[0])))), det);
                const df3 dx{df_norm(dfl_add(dfl_mul_f(u, e1.x), dfl_mul_f(w, e2.x))),
                             df_norm(dfl_add(dfl_mul_f(u, e1.y), dfl_mul_f(w, e2.y))),
                             df_norm(dfl_add(dfl_mul_f(u, e1.z), dfl_mul_f(w, e2.z)))};
                const float r2 = dx.x.hi * dx.x.hi + dx.y.hi * dx.y.hi + dx.z.hi * dx.z.hi;
                if (r2 <= 0.9e-3f) {
                    const df3 Z{df{hp.x, lp.x}, df{hp.y, lp.y}, df{hp.z, lp.z}};
                    const df zd = df3_dot_n(Z, dx);
                    const df dl =
                        df_norm(df_neg(dfl_add(dfl_add_f(df{2.0f * zd.hi, 2.0f * zd.lo}, llp.w), df3_dot_n(dx, dx))));
                    const df m = inv_norm_m1(dl);
                    const df ox = df_norm(dfl_add(dx.x, dfl_mul(m, dfl_add(Z.x, dx.x))));
                    const df oy = df_norm(dfl_add(dx.y, dfl_mul(m, dfl_add(Z.y, dx.y))));
                    const df oz = df_norm(dfl_add(dx.z, dfl_mul(m, dfl_add(Z.z, dx.z))));
                    store_corner_df(cb.vx + (size_t)p * kCellSlots + k, df3{ox, oy, oz});
                    continue;
                }
            }
        }
        V3 e1, e2;
        frame64(zi, e1, e2);
        double a1, b1, c1, a2, b2, c2;
        corner_line64(g, p, zi, e1, e2, ga, a1, b1, c1);
        corner_line64(g, p, zi, e1, e2, gb, a2, b2, c2);
        const double inv = 1.0 / (a1 * b2 - a2 * b1);
        const double u = (c1 * b2 - c2 * b1) * inv;
        const double w = (a1 * c2 - a2 * c1) * inv;
        const V3 o = project_offset(zi, dot(zi, zi) - 1.0, add(scl(e1, u), scl(e2, w)));
        if constexpr (PLAIN) cb.vx[(size_t)p * kCellSlots + k] = P4{o.x, o.y, o.z, 0.0};
        else store_corner_df(cb.vx + (size_t)p * kCellSlots + k, df3_from(o.x, o.y, o.z));
    }
}

// ------------------------------------------------------ density table
// The tanh cap depends on p only through c = x_c.p.  At each centre c_j =
// cos(theta_j) the table holds the Taylor series of rho in u = c - c_j, built
// by power-series arithmetic on the exact composition rho = gamma + (1 -
// gamma) / (1 + exp(-x)), x = 2 (beta - acos c) / alpha:  (1 - (c_j + u)^2)^(-1/2)
// by the binomial recurrence of h^(-1/2), h = 1 + tau1 u + tau2 u^2,
// integrated to acos; the exponential of a series; the reciprocal of a
// series; squared twice for the 4th power.  A range |u| <= U takes the
// terms up to the first two successive ones below 1e-17 of the value; the
// centre's validated radius r_j is the largest r = 0.05 2^(-q/4) whose
// truncated series matches the direct formula at u = +-r, +-r/2, +-r/8 to
// 1e-14 (the direct formula's own sensitivity is ~1e-14 for alpha = 0.05;
// the parity budget is 1e-12).  Near the cap centre and its antipode, where
// acos is singular, and where cells are wide against alpha, the radius is
// small or 0 and those edges evaluate the density directly.
__constant__ double kInv[kTabK + 1] = {0.0,       1.0,       1.0 / 2,  1.0 / 3,  1.0 / 4,  1.0 / 5,  1.0 / 6,
                                       1.0 / 7,   1.0 / 8,   1.0 / 9,  1.0 / 10, 1.0 / 11, 1.0 / 12, 1.0 / 13,
                                       1.0 / 14,  1.0 / 15,  1.0 / 16, 1.0 / 17, 1.0 / 18, 1.0 / 19, 1.0 / 20,
                                       1.0 / 21,  1.0 / 22,  1.0 / 23, 1.0 / 24};

// the density as a function of c = x_c.p, from its definition
__device__ double rho_of_c(const Density &r, double c) {
    double rv = (1.0 - r.gamma) / (1.0 + exp(-2.0 * (r.beta - acos(c)) * r.inv_alpha)) + r.gamma;
    if (r.kind == 3) { rv = rv * rv; rv = rv * rv; }
    return rv;
}

// terms needed over |u| <= U: the first K with terms K and K+1 below 1e-17 of
// the value (0: none within kTabK)
__device__ int series_terms(const double *cf, double U) {
    const double tol = 1e-17 * fabs(cf[0]);
    double Uk = 1.0;
    int small = 0;
    for (int k = 1; k < kTabK; ++k) {
        Uk *= U;
        small = (fabs(cf[k]) * Uk <= tol) ? small + 1 : 0;
        if (small == 2) return k - 1;
    }
    return 0;
}

__global__ void k_dens_table(Density r, int M, double dth, TabCentre *meta, double *cfo, float2 *cdf, float *mag) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    // the centre c_j = cos(j dth) as rounded; sqrt(1 - c_j^2) and acos c_j from it
    const double ci = cos(j * dth);
    const double si = sqrt((1.0 - ci) * (1.0 + ci));
    const double th = atan2(si, ci);
    double cf[kTabK];
    for (int k = 0; k < kTabK; ++k) cf[k] = 0.0;
    double rj = 0.0;
    int Kj = 0;
    if (si > 1e-6) {
        const double isi = 1.0 / si;
        const double tau1 = -2.0 * ci * isi * isi, tau2 = -isi * isi;
        const double c2a = 2.0 * r.inv_alpha * isi;
        const double om = 1.0 - r.gamma;
        double gs[kTabK], xs[kTabK], es[kTabK], rs[kTabK], sq[kTabK];
        gs[0] = 1.0;
        xs[0] = 2.0 * (r.beta - th) * r.inv_alpha;
        es[0] = exp(-xs[0]);
        const double r0 = 1.0 / (1.0 + es[0]);
        rs[0] = r0;
        cf[0] = om * r0 + r.gamma;
        if (r.kind == 3) {
            sq[0] = cf[0] * cf[0];
            cf[0] = sq[0] * sq[0];
        }
        for (int k = 1; k < kTabK; ++k) {
            const double ik = kInv[k];
            double t = (0.5 - k) * tau1 * gs[k - 1];
            if (k >= 2) t += (1.0 - k) * tau2 * gs[k - 2];
            gs[k] = t * ik;
            xs[k] = c2a * gs[k - 1] * ik;  // -2 a_k / alpha, a_k the terms of acos
            t = 0.0;
            for (int i = 1; i <= k; ++i) t += i * xs[i] * es[k - i];
            es[k] = -t * ik;
            t = 0.0;
            for (int i = 1; i <= k; ++i) t += es[i] * rs[k - i];
            rs[k] = -r0 * t;
            if (r.kind == 3) {
                // (gamma + om r)^4 as the square of the square
                t = 0.0;
                for (int i = 0; i <= k; ++i) {
                    const double ri = i == 0 ? om * rs[0] + r.gamma : om * rs[i];
                    const double rk = (k - i) == 0 ? om * rs[0] + r.gamma : om * rs[k - i];
                    t += ri * rk;
                }
                sq[k] = t;
                t = 0.0;
                for (int i = 0; i <= k; ++i) t += sq[i] * sq[k - i];
                cf[k] = t;
            } else {
                cf[k] = om * rs[k];
            }
        }
        for (int q = 0; q < 80 && rj == 0.0; ++q) {
            const double rr = 0.05 * exp2(-0.25 * q);
            const int K = series_terms(cf, rr);
            if (K == 0) continue;
            bool ok = true;
            const double us[6] = {rr, -rr, 0.5 * rr, -0.5 * rr, 0.125 * rr, -0.125 * rr};
            for (int t = 0; t < 6 && ok; ++t) {
                const double c = ci + us[t];
                if (c > 1.0 || c < -1.0) continue;
                const double d = rho_of_c(r, c);
                ok = fabs(horner(cf, K, us[t]) - d) <= 1e-14 * d;
            }
            if (ok) {
                rj = rr;
                Kj = K;
            }
        }
    }
    // double-float copy of the series in v = u 2^-e, 2^e >= r_j (exact
    // scaling; keeps the coefficients in FP32 range), and |cf_k| r_j^k
    int ex = 0;
    if (rj > 0.0) frexp(rj, &ex);
    meta[j] = TabCentre{ci, rj, (float)ldexp(1.0, -ex), (float)rj, (float)Kj, 0.0f};
    double rk = 1.0;
    for (int k = 0; k < kTabK; ++k) {
        cfo[(size_t)j * kTabK + k] = cf[k];
        const df c = df_from(ldexp(cf[k], ex * k));
        cdf[(size_t)j * kTabK + k] = make_float2(c.hi, c.lo);
        mag[(size_t)j * kTabK + k] = (float)(fabs(cf[k]) * rk);
        rk *= rj;
    }
}

// The edge's series: the centre nearest in angle to x_c.z_i = ci, and the
// terms its range needs.  xa, xb, xm: x_c.(v - z_i) at the edge's two
// corners and its midpoint (FP32; the radial parts of the projected rule
// points, |x_c.(p - z_i)| <= (1 + r2) max |x_c.o| + r2 |ci| for offsets of
// squared length <= r2 <= 1/2, are covered by the bound's terms).  Returns 0
// when the range exceeds the centre's validated radius (direct evaluation).
// the centre nearest in angle to c = x_c.z_i
__device__ __forceinline__ int table_centre(const DensTab &T, double ci) {
    const float th = (ci >= 0.0) ? 2.0f * asinf(sqrtf((float)(0.5 * (1.0 - ci))))
                                 : 3.14159265f - 2.0f * asinf(sqrtf((float)(0.5 * (1.0 + ci))));
    return min(T.M - 1, max(0, __float2int_rn(th / T.dth)));
}

// the terms of centre j's series over |u| <= U (0: U beyond its radius)
__device__ __forceinline__ int terms_within(const DensTab &T, int j, float U) {
    const float R = T.meta[j].rf;
    if (!(U <= R)) return 0;
    // terms |cf_k| U^k = mag_k (U / r_j)^k, no overflow
    const float *mg = T.mag + (size_t)j * kTabK;
    const float tol = 1e-17f * mg[0], x = U / R;
    float xk = 1.0f;
    int small = 0;
    for (int k = 1; k < kTabK; ++k) {
        xk *= x;
        small = (mg[k] * xk <= tol) ? small + 1 : 0;
        if (small == 2) return k - 1;
    }
    return 0;
}

__device__ __forceinline__ int table_terms(const DensTab &T, double ci, float xa, float xb, float xm, float r2,
                                           int &j, double &cj) {
    j = table_centre(T, ci);
    const TabCentre mt = T.meta[j];
    cj = mt.c;
    if (!(mt.r > 0.0)) return 0;
    const float U = (float)fabs(ci - cj) + (1.0f + r2) * fmaxf(fmaxf(fabsf(xa), fabsf(xb)), fabsf(xm)) +
                    r2 * fabsf((float)ci) + 1e-6f * sqrtf(r2) + 1e-12f;
    return terms_within(T, j, U);
}

// The FP64 form takes the centre per cell (k_cell_table): the record holds j,
// the scale, and u0 = x_c.z_i - c_j as a pair; then per edge only the range
// bound, with |x_c.z_i| <= 1 for its radial term.
__device__ __forceinline__ float4 cell_table_record(const DensTab &T, const Density &rho, V3 zi) {
    const double ci = rho.xc0 * zi.x + rho.xc1 * zi.y + rho.xc2 * zi.z;
    const int j = table_centre(T, ci);
    const TabCentre mt = T.meta[j];
    if (!(mt.r > 0.0)) return make_float4(__int_as_float(-1), 1.0f, 0.0f, 0.0f);
    const df u = df_from(ci - mt.c);
    return make_float4(__int_as_float(j), mt.scale, u.hi, u.lo);
}

// thread per cell of cells [p0, p1): the cells' table records
__global__ void __launch_bounds__(256) k_cell_table(Grid g, CellBuf cb, int p0, int p1) {
    const int p = p0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= p1) return;
    const int b = view_of(g, p).b;
    const Density rho = g.rho ? g.rho[b] : g.rho0;
    const DensTab T = g.tabs ? g.tabs[b] : g.tab0;
    cb.ctab[p] = (rho.kind >= 2 && T.M > 0) ? cell_table_record(T, rho, ld(g.zs + p))
                                             : make_float4(__int_as_float(-1), 1.0f, 0.0f, 0.0f);
}

// -------------------------------------------------------------- quadrature
// Edge list: cells' edges laid end to end in bin order (eoff = exclusive
// scan of the degrees), ecell[e] = the cell of edge e.
// Edges past the list's capacity ecap are dropped (k_rebase has flagged the
// evaluation); a consistent tessellation has 6N - 12 < ecap edge sides.
__global__ void k_edge_cells(int p0, int p1, const int *__restrict__ deg, const int *__restrict__ eoff,
                             int *__restrict__ ecell, int ecap) {
    int p = p0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= p1) return;
    int d = deg[p], o = eoff[p];
    for (int k = 0; k < d && o + k < ecap; ++k) ecell[o + k] = p;
}

// Chunk words (kChunkWords per chunk): retry counts of the three topology
// passes, the chunk's edge count, the chunk's first edge.
constexpr int kChunkWords = 8;
enum { CW_R0 = 0, CW_R1 = 1, CW_R2 = 2, CW_ETOT = 3, CW_EBASE = 4 };

// a chunk's exclusive scan of the degrees, moved to the chunk's first edge,
// which follows the previous chunk's edges (prev: that chunk's words, null
// for the first chunk); the last cell writes the chunk's edge count, cut to
// the list's capacity ecap (FLAG_ECAP when cut: the edge kernels then stop
// at the capacity and the evaluation reports the inconsistent cells)
__global__ void k_rebase(int p0, int p1, const int *__restrict__ deg, int *__restrict__ eoff,
                         const int *__restrict__ prev, int *__restrict__ mine, int ecap, unsigned *flags) {
    const int p = p0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= p1) return;
    const int base = prev ? prev[CW_EBASE] + prev[CW_ETOT] : 0;
    const int local = eoff[p];
    eoff[p] = local + base;
    if (p == p1 - 1) {
        const int tot = local + deg[p], room = ecap - base;
        if (tot > room) atomicOr(flags, FLAG_ECAP);
        mine[CW_ETOT] = tot > room ? (room > 0 ? room : 0) : tot;
        mine[CW_EBASE] = base;
    }
}

// retry counts of all chunks into the evaluation's status block
__global__ void k_sum_counts(const unsigned *__restrict__ counts, int nch, DevStatus *st) {
    for (int k = 0; k < 3; ++k) {
        unsigned t = 0;
        for (int c = 0; c < nch; ++c) t += counts[kChunkWords * c + k];
        st->retry_count[k] = t;
    }
}

// ------------------------------------------- quadrature in double-float
// The FP64 form's rule points in double-float arithmetic (df.cuh): FP32
// pairs carrying ~48 bits, several times cheaper here than FP64.  Everything
// is taken relative to z_i: a sub-triangle (A, A + b, A + c) has FP64
// offsets b, c (rounded to pairs: 3.6e-15 of their size), and rule point k
// is x = A + w, w = b1 b + b2 c, projected to p = x / |x| = A + q,
// q = (1 + m) w + m A, m = 1/|x| - 1.  Every per-point quantity is a
// combination of per-triangle scalars (A.b, A.c, b.b, b.c, c.c, e.b, e.c,
// e.A for the density's direction e) with the rule's constants:
//   A.w   = b1 A.b + b2 A.c,   |w|^2 = b1^2 b.b + 2 b1 b2 b.c + b2^2 c.c
//   delta = 1 - |x|^2 = -(|A|^2 - 1) - 2 A.w - |w|^2   (|A|^2 - 1 from FP64)
//   m     = delta/2 + 3 delta^2/8 + 5 delta^3/16 + 35 delta^4/128 + 63 delta^5/256,
//           exact to 3e-19 for delta <= 1e-3
//   e.q   = e.w + m (e.A + e.w)  (the density's argument: x_c.p - c_i = (x_c.z_i - c_i)
//           + x_c.q for the tanh cap, p_z = A_z + e_z.q for X3)
//   |q|^2 = |w|^2 + 2 m (|w|^2 + A.w) + m^2 |x|^2 = |p - z_i|^2
// and sum wr q = b S1 + c S2 + A T0 with S1, S2 the sums of wr (1 + m) b1,
// wr (1 + m) b2 and T0 that of wr m, so wr p sums to z_i sum wr + sum wr q.
// No difference of nearby values is formed.  The signed area is 2 atan(t),
// t = A.(b x c) / (4 + 3 (|A|^2 - 1) + 2 A.(b + c) + b.c) (Van Oosterom-Strackee
// with B = A + b, C = A + c), atan(t) = t - t^3/3 to 1e-18 for the t <= 3e-4
// of such triangles.  Per-edge mass, moment and energy match the FP64
// evaluation to ~1e-14 relative.
struct AccDF {
    df m, qx, qy, qz, e;
};

__device__ __forceinline__ void tri_df(int kind, df g1, df gam, df3 A, df aA1, df3 b, df3 c, df3 ev, df eA, df u0,
                                       const float2 *__restrict__ sdf, float vs, int K, AccDF &acc) {
    const df Ab = df3_dot_n(A, b), Ac = df3_dot_n(A, c);
    const df bb = df3_dot_n(b, b), cc = df3_dot_n(c, c), bc = df3_dot_n(b, c);
    const df eb = df3_dot_n(ev, b), ec = df3_dot_n(ev, c);
    const df det = df3_dot_n(A, df3_cross_n(b, c));
    const df den = df_norm(dfl_add(dfl_add_f(dfl_mul_f(aA1, 3.0f), 4.0f), dfl_add(dfl_mul_f(dfl_add(Ab, Ac), 2.0f), bc)));
    const df t = df_div(det, den);
    const df area = df_mul_f(df_add_f(t, -t.hi * t.hi * t.hi * (1.0f / 3.0f)), 2.0f);
    df S0{0.0f, 0.0f}, S1{0.0f, 0.0f}, S2{0.0f, 0.0f}, T0{0.0f, 0.0f}, E{0.0f, 0.0f};
#pragma unroll 1
    for (int k = 0; k < 7; ++k) {
        const df b1{kQdf[k][0][0], kQdf[k][0][1]}, b2{kQdf[k][1][0], kQdf[k][1][1]}, W{kQdf[k][2][0], kQdf[k][2][1]};
        const df B11{kQdf[k][3][0], kQdf[k][3][1]}, B12{kQdf[k][4][0], kQdf[k][4][1]}, B22{kQdf[k][5][0], kQdf[k][5][1]};
        // unnormalized chains (dfl_*); the sums that cancel (delta, |w|^2 + A.w,
        // the series argument) are normalized before they are multiplied (m
        // and the weight come from sums and products of one sign)
        const df Aw = dfl_add(dfl_mul(b1, Ab), dfl_mul(b2, Ac));
        const df ww = dfl_add(dfl_add(dfl_mul(B11, bb), dfl_mul(B12, bc)), dfl_mul(B22, cc));
        const df dl = df_norm(df_neg(dfl_add(dfl_add(aA1, df{2.0f * Aw.hi, 2.0f * Aw.lo}), ww)));
        const df d2 = dfl_mul(dl, dl);
        const float tail = d2.hi * dl.hi * (0.3125f + dl.hi * (0.2734375f + dl.hi * 0.24609375f));
        const df m = dfl_add_f(dfl_add(df{0.5f * dl.hi, 0.5f * dl.lo}, dfl_mul_f(d2, 0.375f)), tail);
        const df xw = dfl_add(dfl_mul(b1, eb), dfl_mul(b2, ec));
        const df eq = dfl_add(xw, dfl_mul(m, dfl_add(eA, xw)));
        df rv;
        if (kind == 0) {
            rv = df{1.0f, 0.0f};
        } else if (kind == 1) {
            const df pz = df_norm(dfl_add(eA, eq)), z2 = df_norm(dfl_mul(pz, pz));
            rv = dfl_add(dfl_mul(g1, dfl_mul(z2, z2)), gam);
        } else {
            // the argument of the cell's series, scaled by its power of two
            const df u = df_norm(dfl_add(u0, eq));
            const df v{u.hi * vs, u.lo * vs};
            rv = df{sdf[K - 1].x, sdf[K - 1].y};
            for (int j = K - 2; j >= 0; --j) rv = dfl_fma(rv, v, df{sdf[j].x, sdf[j].y});
        }
        const df wr = dfl_mul(dfl_mul(W, area), rv);
        const df wm = dfl_mul(wr, m);
        // |q|^2 = |w|^2 + 2 m (|w|^2 + A.w) + m^2 - m^2 delta
        const df mwa = dfl_mul(m, df_norm(dfl_add(ww, Aw))), msq = dfl_mul(m, m);
        const df e = dfl_add_f(dfl_add(dfl_add(ww, df{2.0f * mwa.hi, 2.0f * mwa.lo}), msq), -msq.hi * dl.hi);
        // wr q = (wr + wm) w + wm A: sums of (wr + wm) b1, (wr + wm) b2 and wm
        const df wp = dfl_add(wr, wm);
        S0 = dfl_add(S0, wr);
        S1 = dfl_add(S1, dfl_mul(wp, b1));
        S2 = dfl_add(S2, dfl_mul(wp, b2));
        T0 = dfl_add(T0, wm);
        E = dfl_add(E, dfl_mul(wr, e));
    }
    S0 = df_norm(S0);
    S1 = df_norm(S1);
    S2 = df_norm(S2);
    T0 = df_norm(T0);
    E = df_norm(E);
    const df a1 = S1, a2 = S2;
    acc.m = df_norm(dfl_add(acc.m, S0));
    acc.qx = df_norm(dfl_add(acc.qx, dfl_add(dfl_add(dfl_mul(a1, b.x), dfl_mul(a2, c.x)), dfl_mul(T0, A.x))));
    acc.qy = df_norm(dfl_add(acc.qy, dfl_add(dfl_add(dfl_mul(a1, b.y), dfl_mul(a2, c.y)), dfl_mul(T0, A.y))));
    acc.qz = df_norm(dfl_add(acc.qz, dfl_add(dfl_add(dfl_mul(a1, b.z), dfl_mul(a2, c.z)), dfl_mul(T0, A.z))));
    acc.e = df_norm(dfl_add(acc.e, E));
}

// One thread per Voronoi edge (two signed sub-triangles of Sec. 3.2.2, 14
// rule points, summed in order).  The edge's five sums go to the edge list;
// k_cell_sum adds a cell's edges in edge order, so a cell's result depends
// on its own edges only (not on where they fall in the launch).

template <bool PLAIN>
__global__ void __launch_bounds__(512) k_quad(Grid g, CellBuf cb, int ecap, Span sp, DevStatus *st) {
    const int ne = *sp.etot, eb = *sp.e0;
    const DensDF dd0 = dens_df(g.rho0);  // single-problem density, converted once
    unsigned n_ser = 0, n_terms = 0;
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < ne; it += gridDim.x * blockDim.x) {
        const int e = eb + it;
        const int p = cb.ecell[e];
        const int k = e - cb.eoff[p];
        const int deg = cb.deg[p];
        const V3 zi = ld(g.zs + p);
        const P4 *vx = cb.vx + (size_t)p * kCellSlots;
        const int kb = (k + 1 == deg) ? 0 : k + 1;
        // corner offsets from z_i: FP64, or double-float pairs in the FP64 form
        df3 da, db;
        V3 va, vb;
        if constexpr (PLAIN) {
            va = ld(vx + k);
            vb = ld(vx + kb);
        } else {
            da = load_corner_df(vx + k);
            db = load_corner_df(vx + kb);
        }
        const int b = view_of(g, p).b;
        const Density rho = g.rho ? g.rho[b] : g.rho0;
        const int q = cb.nb[(size_t)p * kCellSlots + k];
        double *ea = cb.eacc;
        // the edge's density series from the table (tanh-cap kinds): its range
        // bound in FP32 from the corner offsets and z_j - z_i (FP32 pairs),
        // x_c.z_i in FP64 (it sets the series' argument)
        int K = 0, j = 0;
        double cj = 0.0, ci = 0.0;
        df u0c{0.0f, 0.0f};  // FP64 form: x_c.z_i - c_j from the cell's record
        float vsc = 1.0f;
        const double *tcf = nullptr;
        const float2 *tcdf = nullptr;
        if (rho.kind >= 2) {
            const DensTab T = g.tabs ? g.tabs[b] : g.tab0;
            if (T.M > 0) {
                float3 fa, fb;
                if constexpr (PLAIN) {
                    fa = make_float3((float)va.x, (float)va.y, (float)va.z);
                    fb = make_float3((float)vb.x, (float)vb.y, (float)vb.z);
                } else {
                    fa = make_float3(da.x.hi, da.y.hi, da.z.hi);
                    fb = make_float3(db.x.hi, db.y.hi, db.z.hi);
                }
                const float3 fh = dfdiff(g, q, g.zf[p], g.zl[p]);
                const float r2 = fmaxf(fmaxf(fa.x * fa.x + fa.y * fa.y + fa.z * fa.z, fb.x * fb.x + fb.y * fb.y + fb.z * fb.z),
                                       0.25f * (fh.x * fh.x + fh.y * fh.y + fh.z * fh.z));
                if (r2 <= 0.5f) {
                    const DensityF rf = g.rhof ? g.rhof[b] : g.rho0f;
                    const float xa = rf.xc0 * fa.x + rf.xc1 * fa.y + rf.xc2 * fa.z;
                    const float xb = rf.xc0 * fb.x + rf.xc1 * fb.y + rf.xc2 * fb.z;
                    const float xm = 0.5f * (rf.xc0 * fh.x + rf.xc1 * fh.y + rf.xc2 * fh.z);
                    if constexpr (PLAIN) {
                        ci = rho.xc0 * zi.x + rho.xc1 * zi.y + rho.xc2 * zi.z;
                        K = table_terms(T, ci, xa, xb, xm, r2, j, cj);
                    } else {
                        const float4 rec = cb.ctab[p];
                        j = __float_as_int(rec.x);
                        if (j >= 0) {
                            const float U = fabsf(rec.z) + (1.0f + r2) * fmaxf(fmaxf(fabsf(xa), fabsf(xb)), fabsf(xm)) +
                                            r2 + 1e-6f * sqrtf(r2) + 1e-12f;
                            K = terms_within(T, j, U);
                            cj = T.meta[j].c;
                            vsc = rec.y;
                            u0c = df{rec.z, rec.w};
                        } else {
                            j = 0;
                        }
                    }
                    tcf = T.cf + (size_t)j * kTabK;
                    tcdf = T.cdf + (size_t)j * kTabK;
                }
            }
        }
        if (K > 0) {
            n_ser++;
            n_terms += K;
        }
        // double-float path: offsets of the edge's points from z_i below chord
        // 0.03 (then delta <= 1e-3 at every rule point) and a density without
        // direct evaluation; otherwise FP64.  The FP64 form's edge sums are
        // stored as double-float pairs (m, o = sum w rho (p - z_i), F), the
        // plain form's in FP64 (m, c, F).
        float2 *ef = reinterpret_cast<float2 *>(cb.eacc);
        if constexpr (!PLAIN) {
            const float4 hp = g.zf[p], lp = g.zl[p], llp = g.zll[p];
            const df3 dj = gen_diff(g, q, hp, lp, llp);
            const float r2 = fmaxf(fmaxf(da.x.hi * da.x.hi + da.y.hi * da.y.hi + da.z.hi * da.z.hi,
                                         db.x.hi * db.x.hi + db.y.hi * db.y.hi + db.z.hi * db.z.hi),
                                   0.25f * (dj.x.hi * dj.x.hi + dj.y.hi * dj.y.hi + dj.z.hi * dj.z.hi));
            if (r2 <= 0.9e-3f && (rho.kind < 2 || K > 0)) {
                const df3 A{df{hp.x, lp.x}, df{hp.y, lp.y}, df{hp.z, lp.z}};
                const df aA1{llp.w, 0.0f};
                const DensDF dd = g.rho ? g.rhodf[b] : dd0;
                const df eA = df3_dot_n(dd.ev, A);
                const df u0 = (K > 0) ? u0c : df{0.0f, 0.0f};
                const float vs = (K > 0) ? vsc : 1.0f;
                // edge midpoint mu = (z_i + z_j) / |z_i + z_j|: with h = (z_j - z_i) / 2,
                // mu - z_i = h + m (A + h), 1 - |A + h|^2 = -(|A|^2 - 1) - 2 A.h - |h|^2
                const df3 hh{df{0.5f * dj.x.hi, 0.5f * dj.x.lo}, df{0.5f * dj.y.hi, 0.5f * dj.y.lo},
                             df{0.5f * dj.z.hi, 0.5f * dj.z.lo}};
                const df Ah = df3_dot_n(A, hh);
                const df dl = df_norm(df_neg(dfl_add(dfl_add(aA1, df{2.0f * Ah.hi, 2.0f * Ah.lo}), df3_dot_n(hh, hh))));
                const df mm = inv_norm_m1(dl);
                const df3 dm{df_norm(dfl_add(hh.x, dfl_mul(mm, dfl_add(A.x, hh.x)))),
                             df_norm(dfl_add(hh.y, dfl_mul(mm, dfl_add(A.y, hh.y)))),
                             df_norm(dfl_add(hh.z, dfl_mul(mm, dfl_add(A.z, hh.z))))};
                AccDF ad{};
                // the edge's sub-triangles (z_i, v_a, mu), (z_i, mu, v_b), or the fan's
                // (z_i, v_a, v_b), in order, through one copy of the rule's code
                const int ntri = g.fan ? 1 : 2;
#pragma unroll 1
                for (int t = 0; t < ntri; ++t) {
                    const df3 tb = (t == 0) ? da : dm;
                    const df3 tc = (t == 0 && !g.fan) ? dm : db;
                    tri_df(rho.kind, dd.g1, dd.gam, A, aA1, tb, tc, dd.ev, eA, u0, tcdf, vs, K, ad);
                }
                ef[e] = make_float2(ad.m.hi, ad.m.lo);
                ef[(size_t)ecap + e] = make_float2(ad.qx.hi, ad.qx.lo);
                ef[2 * (size_t)ecap + e] = make_float2(ad.qy.hi, ad.qy.lo);
                ef[3 * (size_t)ecap + e] = make_float2(ad.qz.hi, ad.qz.lo);
                ef[4 * (size_t)ecap + e] = make_float2(ad.e.hi, ad.e.lo);
                continue;
            }
            va = V3{df_to(da.x), df_to(da.y), df_to(da.z)};
            vb = V3{df_to(db.x), df_to(db.y), df_to(db.z)};
        }
        // FP64: every point relative to z_i (corner and midpoint offsets)
        const double inv_alpha = rho.inv_alpha;
        const double aA1 = dot(zi, zi) - 1.0;
        Acc acc = {0, 0, 0, 0, 0};
        if (g.fan) {
            tri(rho, inv_alpha, zi, aA1, va, vb, acc, tcf, K, cj);
        } else {
            const V3 om = midpoint_offset(zi, aA1, ld(g.zs + q));
            tri(rho, inv_alpha, zi, aA1, va, om, acc, tcf, K, cj);
            tri(rho, inv_alpha, zi, aA1, om, vb, acc, tcf, K, cj);
        }
        if constexpr (!PLAIN) {
            const df em = df_from(acc.m), ex = df_from(acc.cx), ey = df_from(acc.cy), ez = df_from(acc.cz),
                     ee = df_from(acc.e);
            ef[e] = make_float2(em.hi, em.lo);
            ef[(size_t)ecap + e] = make_float2(ex.hi, ex.lo);
            ef[2 * (size_t)ecap + e] = make_float2(ey.hi, ey.lo);
            ef[3 * (size_t)ecap + e] = make_float2(ez.hi, ez.lo);
            ef[4 * (size_t)ecap + e] = make_float2(ee.hi, ee.lo);
            continue;
        }
        moment_from_offsets(zi, acc);
        ea[e] = acc.m;
        ea[(size_t)ecap + e] = acc.cx;
        ea[2 * (size_t)ecap + e] = acc.cy;
        ea[3 * (size_t)ecap + e] = acc.cz;
        ea[4 * (size_t)ecap + e] = acc.e;
    }
    // edges that took the density table, and their terms: one pair of
    // atomics per block
    __shared__ unsigned cnt[2];
    if (threadIdx.x == 0) cnt[0] = cnt[1] = 0u;
    __syncthreads();
    n_ser = __reduce_add_sync(0xffffffffu, n_ser);
    n_terms = __reduce_add_sync(0xffffffffu, n_terms);
    if ((threadIdx.x & 31) == 0 && n_ser) {
        atomicAdd(&cnt[0], n_ser);
        atomicAdd(&cnt[1], n_terms);
    }
    __syncthreads();
    if (threadIdx.x == 0 && cnt[0]) {
        atomicAdd(&st->ser_edges, (unsigned long long)cnt[0]);
        atomicAdd(&st->ser_terms, (unsigned long long)cnt[1]);
    }
}

// ------------------------------------------------ mixed precision (FP32)
// Corners, edge midpoints and rule points are handled as offsets from z_i in
// FP32: every quantity is formed without cancellation at the cell scale h,
// so FP32 keeps ~1e-7 of h.  Per edge the 14 rule points are summed in FP32;
// edges and cells are summed in FP64, and c_i = m_i z_i + sum w rho (p - z_i)
// so that the gradient g_i = -2 (o - (o.z_i) z_i), o = sum w rho (p - z_i),
// never subtracts m_i z_i from itself.

// FP32 lines of generators gin, gout in the FP32 frame at z_p, their
// intersection (u, w), and whether it is ill conditioned
__device__ __forceinline__ bool vertex32(const Grid &g, int p, float4 hp, float4 lp, float3 e1, float3 e2, int gin,
                                         int gout, float &u, float &w) {
    const float3 d1 = dfdiff(g, gin, hp, lp), d2 = dfdiff(g, gout, hp, lp);
    const float a1 = e1.x * d1.x + e1.y * d1.y + e1.z * d1.z, b1 = e2.x * d1.x + e2.y * d1.y + e2.z * d1.z;
    const float c1 = 0.5f * fmaf(d1.x, d1.x, fmaf(d1.y, d1.y, d1.z * d1.z));
    const float a2 = e1.x * d2.x + e1.y * d2.y + e1.z * d2.z, b2 = e2.x * d2.x + e2.y * d2.y + e2.z * d2.z;
    const float c2 = 0.5f * fmaf(d2.x, d2.x, fmaf(d2.y, d2.y, d2.z * d2.z));
    const float p1 = a1 * b2, p2 = a2 * b1, det = p1 - p2;
    u = (c1 * b2 - c2 * b1) / det;
    w = (a1 * c2 - a2 * c1) / det;
    return !(fabsf(det) * 30.0f >= fabsf(p1) + fabsf(p2));
}

__device__ __forceinline__ void frame32(float4 hp, float3 &e1, float3 &e2) {
    const float fx = fabsf(hp.x), fy = fabsf(hp.y), fz = fabsf(hp.z);
    float3 ax = (fx <= fy && fx <= fz) ? make_float3(1, 0, 0)
                                       : ((fy <= fz) ? make_float3(0, 1, 0) : make_float3(0, 0, 1));
    float3 c = make_float3(hp.y * ax.z - hp.z * ax.y, hp.z * ax.x - hp.x * ax.z, hp.x * ax.y - hp.y * ax.x);
    const float inv = rsqrtf(c.x * c.x + c.y * c.y + c.z * c.z);
    e1 = make_float3(c.x * inv, c.y * inv, c.z * inv);
    e2 = make_float3(hp.y * e1.z - hp.z * e1.y, hp.z * e1.x - hp.x * e1.z, hp.x * e1.y - hp.y * e1.x);
}

// offset of normalize(z + u e1 + w e2) from z: (u e1 + w e2)/q - z r^2/(q (1+q)), q = sqrt(1 + r^2)
__device__ __forceinline__ float3 gnomonic_offset(float4 z, float3 e1, float3 e2, float u, float w) {
    const float r2 = u * u + w * w;
    const float q = sqrtf(1.0f + r2);
    const float iq = 1.0f / q, t = r2 / (q * (1.0f + q));
    return make_float3((u * e1.x + w * e2.x) * iq - z.x * t, (u * e1.y + w * e2.y) * iq - z.y * t,
                       (u * e1.z + w * e2.z) * iq - z.z * t);
}

__global__ void __launch_bounds__(256) k_corners32(Grid g, CellBuf cb, Span sp) {
    const int ne = *sp.etot, eb = *sp.e0;
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < ne; it += gridDim.x * blockDim.x) {
        const int e = eb + it;
        const int p = cb.ecell[e];
        const int k = e - cb.eoff[p];
        const int deg = cb.deg[p];
        const int *nb = cb.nb + (size_t)p * kCellSlots;
        const int gin = nb[(k == 0) ? deg - 1 : k - 1], gout = nb[k];
        const float4 hp = g.zf[p], lp = g.zl[p];
        float3 e1, e2;
        frame32(hp, e1, e2);
        float u, w;
        float3 o;
        if (!vertex32(g, p, hp, lp, e1, e2, gin, gout, u, w)) {
            o = gnomonic_offset(hp, e1, e2, u, w);
        } else {
            // ill conditioned: the corner in FP64, then its offset
            const V3 zi = ld(g.zs + p);
            V3 f1, f2;
            frame64(zi, f1, f2);
            double a1, b1, c1, a2, b2, c2;
            line_of(g, zi, f1, f2, gin, a1, b1, c1);
            line_of(g, zi, f1, f2, gout, a2, b2, c2);
            const double inv = 1.0 / (a1 * b2 - a2 * b1);
            const double uu = (c1 * b2 - c2 * b1) * inv, ww = (a1 * c2 - a2 * c1) * inv;
            const double r2 = uu * uu + ww * ww, q = sqrt(1.0 + r2), t = r2 / (q * (1.0 + q));
            o = make_float3((float)((uu * f1.x + ww * f2.x) / q - zi.x * t), (float)((uu * f1.y + ww * f2.y) / q - zi.y * t),
                            (float)((uu * f1.z + ww * f2.z) / q - zi.z * t));
        }
        cb.vo[(size_t)p * kCellSlots + k] = make_float4(o.x, o.y, o.z, 0.0f);
    }
}

struct AccF {
    float m, ox, oy, oz, e;
};

__device__ __forceinline__ float rho32(const DensityF &r, float px, float py, float pz) {
    if (r.kind == 0) return 1.0f;
    if (r.kind == 1) {
        const float z2 = pz * pz;
        return (1.0f - r.gamma) * z2 * z2 + r.gamma;
    }
    const float cx = py * r.xc2 - pz * r.xc1, cy = pz * r.xc0 - px * r.xc2, cz = px * r.xc1 - py * r.xc0;
    const float d = atan2f(sqrtf(cx * cx + cy * cy + cz * cz), px * r.xc0 + py * r.xc1 + pz * r.xc2);
    // logistic form of (1 - gamma)/2 (tanh(x) + 1) + gamma: no cancellation in the tail
    float v = (1.0f - r.gamma) / (1.0f + expf(-2.0f * (r.beta - d) * r.inv_alpha)) + r.gamma;
    if (r.kind == 3) { v = v * v; v = v * v; }
    return v;
}

// signed sub-triangle (z, z + oa, z + ob) with the 7-point rule, FP32
__device__ __forceinline__ void tri32(const DensityF &r, float4 z, float3 oa, float3 ob, AccF &acc) {
    const float cx = oa.y * ob.z - oa.z * ob.y, cy = oa.z * ob.x - oa.x * ob.z, cz = oa.x * ob.y - oa.y * ob.x;
    const float det = z.x * cx + z.y * cy + z.z * cz;
    const float zoa = z.x * oa.x + z.y * oa.y + z.z * oa.z, zob = z.x * ob.x + z.y * ob.y + z.z * ob.z;
    const float den = 4.0f + 2.0f * zoa + 2.0f * zob + (oa.x * ob.x + oa.y * ob.y + oa.z * ob.z);
    const float area = 2.0f * atan2f(det, den);
#pragma unroll 1
    for (int k = 0; k < 7; ++k) {
        const float b1 = kQbf[k][0], b2 = kQbf[k][1];  // weights of the 2nd and 3rd vertex
        const float dx = b1 * oa.x + b2 * ob.x, dy = b1 * oa.y + b2 * ob.y, dz = b1 * oa.z + b2 * ob.z;
        const float zd = z.x * dx + z.y * dy + z.z * dz, dd = dx * dx + dy * dy + dz * dz;
        const float n = sqrtf(1.0f + 2.0f * zd + dd);
        const float t = (2.0f * zd + dd) / (n + 1.0f), in = 1.0f / n;
        const float ox = (dx - z.x * t) * in, oy = (dy - z.y * t) * in, oz = (dz - z.z * t) * in;
        const float wr = kQwf[k] * area * rho32(r, z.x + ox, z.y + oy, z.z + oz);
        acc.m += wr;
        acc.ox += wr * ox;
        acc.oy += wr * oy;
        acc.oz += wr * oz;
        acc.e += wr * (ox * ox + oy * oy + oz * oz);
    }
}

__device__ __forceinline__ void write_cell_offsets(const CellOut &out, int i, V3 zi, const Acc &a, unsigned *flags) {
    // a.cx, a.cy, a.cz hold o = sum w rho (p - z_i)
    const double oz = a.cx * zi.x + a.cy * zi.y + a.cz * zi.z;
    const double cz = a.m + oz;  // c.z_i with |z_i| = 1
    if (!(cz > 0.0)) atomicOr(flags, FLAG_NONPOSITIVE);
    if (out.grad) {
        out.grad[3 * (size_t)i] = -2.0 * (a.cx - oz * zi.x);
        out.grad[3 * (size_t)i + 1] = -2.0 * (a.cy - oz * zi.y);
        out.grad[3 * (size_t)i + 2] = -2.0 * (a.cz - oz * zi.z);
    }
    if (out.hdiag) out.hdiag[i] = 1.0 / (2.0 * cz);
    if (out.mass) out.mass[i] = a.m;
    if (out.moment) {
        out.moment[3 * (size_t)i] = a.m * zi.x + a.cx;
        out.moment[3 * (size_t)i + 1] = a.m * zi.y + a.cy;
        out.moment[3 * (size_t)i + 2] = a.m * zi.z + a.cz;
    }
    if (out.fcell) out.fcell[i] = a.e;
}

// one thread per edge; the 14 rule points of the edge's two sub-triangles
// summed in FP32, the edge's five sums stored in FP32 (edges and cells are
// summed in FP64 by k_cell_sum)
__global__ void __launch_bounds__(512) k_quad32(Grid g, CellBuf cb, int ecap, Span sp) {
    const int ne = *sp.etot, eb = *sp.e0;
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < ne; it += gridDim.x * blockDim.x) {
        const int e = eb + it;
        const int p = cb.ecell[e];
        const int k = e - cb.eoff[p];
        const int deg = cb.deg[p];
        const float4 hp = g.zf[p], lp = g.zl[p];
        const float4 va = cb.vo[(size_t)p * kCellSlots + k];
        const float4 vb = cb.vo[(size_t)p * kCellSlots + ((k + 1 == deg) ? 0 : k + 1)];
        // edge midpoint normalize(z_i + z_j) as an offset: d/s + z |d|^2 / (s (2 + s)), s = sqrt(4 - |d|^2)
        const float3 d = dfdiff(g, cb.nb[(size_t)p * kCellSlots + k], hp, lp);
        const float dd = fmaf(d.x, d.x, fmaf(d.y, d.y, d.z * d.z));
        const float sq = sqrtf(4.0f - dd), is = 1.0f / sq, t = dd / (sq * (2.0f + sq));
        const float3 om = make_float3(d.x * is + hp.x * t, d.y * is + hp.y * t, d.z * is + hp.z * t);
        const DensityF rf = g.rhof ? g.rhof[view_of(g, p).b] : g.rho0f;
        AccF a = {0, 0, 0, 0, 0};
        if (g.fan) {
            tri32(rf, hp, make_float3(va.x, va.y, va.z), make_float3(vb.x, vb.y, vb.z), a);
        } else {
            tri32(rf, hp, make_float3(va.x, va.y, va.z), om, a);
            tri32(rf, hp, om, make_float3(vb.x, vb.y, vb.z), a);
        }
        float *ea = (float *)cb.eacc;
        ea[e] = a.m;
        ea[(size_t)ecap + e] = a.ox;
        ea[2 * (size_t)ecap + e] = a.oy;
        ea[3 * (size_t)ecap + e] = a.oz;
        ea[4 * (size_t)ecap + e] = a.e;
    }
}

// thread per cell: the cell's edge sums added in edge order, then the cell's
// outputs (g_i, h_i, m_i, c_i, F_i at the original index).  KIND 0: the FP64
// form's double-float pairs (m, o, F), added as pairs; 1: the mixed form's
// FP32 sums (m, o, F), added as pairs (FP32 operations instead of FP64 ones
// on GB300's narrow FP64 pipe); 2: the plain form's FP64 sums (m, c, F).
// With o = sum w rho (p - z_i) the gradient -2 (o - (o.z_i) z_i) never
// subtracts m_i z_i from itself.
template <int KIND>
__global__ void __launch_bounds__(256) k_cell_sum(Grid g, CellOut out, CellBuf cb, int ecap, DevStatus *st, Span sp) {
    const int p = sp.p0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= sp.p1) return;
    const int deg = cb.deg[p];
    if (deg == 0) return;  // integrated by the topology kernel, failed, or inactive
    const int e0 = cb.eoff[p];
    if (e0 + deg > ecap) return;  // past the edge list (FLAG_ECAP is set)
    Acc acc = {0, 0, 0, 0, 0};
    if (KIND == 0) {
        const float2 *ef = reinterpret_cast<const float2 *>(cb.eacc);
        df s[5] = {};
        for (int k = 0; k < deg; ++k) {
            const int e = e0 + k;
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                const float2 v = ef[(size_t)c * ecap + e];
                s[c] = df_add(s[c], df{v.x, v.y});
            }
        }
        acc = Acc{df_to(s[0]), df_to(s[1]), df_to(s[2]), df_to(s[3]), df_to(s[4])};
    } else if (KIND == 1) {
        // FP32 edge sums added exactly enough as pairs (no FP64 instruction per edge)
        const float *ea = (const float *)cb.eacc;
        df s[5] = {};
        for (int k = 0; k < deg; ++k) {
            const int e = e0 + k;
#pragma unroll
            for (int c = 0; c < 5; ++c) s[c] = df_add_f(s[c], ea[(size_t)c * ecap + e]);
        }
        acc = Acc{df_to(s[0]), df_to(s[1]), df_to(s[2]), df_to(s[3]), df_to(s[4])};
    } else {
        const double *ea = cb.eacc;
        for (int k = 0; k < deg; ++k) {
            const int e = e0 + k;
            acc.m += ea[e];
            acc.cx += ea[(size_t)ecap + e];
            acc.cy += ea[2 * (size_t)ecap + e];
            acc.cz += ea[3 * (size_t)ecap + e];
            acc.e += ea[4 * (size_t)ecap + e];
        }
    }
    const V3 zi = ld(g.zs + p);
    unsigned *flags = flags_of(g, st, view_of(g, p).b);
    if (KIND == 2) write_cell(out, g.sidx[p], zi, acc, flags);
    else write_cell_offsets(out, g.sidx[p], zi, acc, flags);
}

}  // namespace

void bin_points(const double *z, const Grid &g, int *bin_of, int *count, int *start, int *cursor, int *scan_tmp,
                P4 *zs, float4 *zf, float4 *zl, float4 *zll, int *sidx, const float *hint, DevStatus *st, cudaStream_t s,
                int64_t *launches) {
    const int n = g.n, nbins = g.nbins;
    Grid gb = g;
    gb.bstart = start;
    cudaMemsetAsync(count, 0, sizeof(int) * nbins, s);
    int blocks = (n + 255) / 256;
    k_bin_count<<<blocks, 256, 0, s>>>(z, gb, bin_of, count, st);
    k_bin_max<<<dim3(g.inst ? 32 : 4 * 152, g.inst ? g.nprob : 1), 256, 0, s>>>(gb, count, st);
    exclusive_scan(count, start, nbins, scan_tmp, s, launches);
    k_set_total<<<1, 1, 0, s>>>(start, nbins, n);
    cudaMemcpyAsync(cursor, start, sizeof(int) * nbins, cudaMemcpyDeviceToDevice, s);
    k_bin_scatter<<<blocks, 256, 0, s>>>(z, n, bin_of, cursor, zs, zf, zl, zll, sidx, hint);
    k_bin_sort<<<(nbins + 255) / 256, 256, 0, s>>>(start, nbins, zs, zf, zl, zll, sidx);
    (*launches) += 5;
}


void exclusive_scan(const int *in, int *out, int len, int *tmp, cudaStream_t s, int64_t *launches) {
    scan_rec(in, out, len, tmp, s, launches);
}

int bins_per_edge(int64_t n, int bin_load) {
    const int G = (int)ceil(sqrt((double)n / (6.0 * (double)bin_load)));
    return std::max(1, std::min(G, 4096));
}

int adapt_bins(int G0, int Gcur, int Gmax, unsigned max_bin, int bin_load) {
    if (max_bin == 0 || Gcur <= 0) return Gcur;
    const double r = (double)Gcur / (double)G0;
    const double m0 = (double)max_bin * r * r;
    double G = G0 * sqrt(m0 / (6.0 * bin_load));
    G = std::max((double)G0, std::min((double)Gmax, ceil(G)));
    if (fabs(G - Gcur) <= 0.15 * Gcur) return Gcur;
    return (int)G;
}

scvt_status tune_from(const scvt_tuning &t, Tune *out) {
    if (t.bin_load < 1 || t.bin_load > 16) return SCVT_ERR_INVALID;
    if (t.knn_target < 8 || t.knn_target > 64) return SCVT_ERR_INVALID;
    if (t.topo_warps != 2 && t.topo_warps != 4 && t.topo_warps != 8) return SCVT_ERR_INVALID;
    if (t.topo_blocks_per_sm < 1 || t.topo_blocks_per_sm > 64) return SCVT_ERR_INVALID;
    if (t.quad_block != 128 && t.quad_block != 256 && t.quad_block != 512) return SCVT_ERR_INVALID;
    if (t.topo_cell_lanes != 16 && t.topo_cell_lanes != 32) return SCVT_ERR_INVALID;
    if (t.chunks < 1 || t.chunks > kMaxChunks) return SCVT_ERR_INVALID;
    out->bin_load = t.bin_load;
    out->knn_target = t.knn_target;
    out->topo_warps = t.topo_warps;
    out->topo_bpsm = t.topo_blocks_per_sm;
    out->quad_block = t.quad_block;
    out->topo_lanes = t.topo_cell_lanes;
    out->chunks = t.chunks;
    return SCVT_OK;
}

scvt_tuning tuning_of(const Tune &u) {
    scvt_tuning t;
    t.bin_load = u.bin_load;
    t.knn_target = u.knn_target;
    t.topo_warps = u.topo_warps;
    t.topo_blocks_per_sm = u.topo_bpsm;
    t.quad_block = u.quad_block;
    t.topo_cell_lanes = u.topo_lanes;
    t.chunks = u.chunks;
    return t;
}

Density to_device_density(const scvt_density &r) {
    Density d;
    d.kind = r.kind;
    d.gamma = r.gamma;
    d.alpha = r.alpha;
    d.beta = r.beta;
    d.xc0 = r.xc[0];
    d.xc1 = r.xc[1];
    d.xc2 = r.xc[2];
    d.inv_alpha = 1.0 / r.alpha;
    return d;
}

DensityF to_density32(const Density &d) {
    DensityF f;
    f.kind = d.kind;
    f.gamma = (float)d.gamma;
    f.beta = (float)d.beta;
    f.inv_alpha = (float)(1.0 / d.alpha);
    f.xc0 = (float)d.xc0;
    f.xc1 = (float)d.xc1;
    f.xc2 = (float)d.xc2;
    return f;
}

int dens_table_centres(int64_t n) {
    // theta spacing about half the smallest cells' angular size for a cap
    // holding most generators at 8x the density contrast: 8 sqrt(n) centres
    const double m = 8.0 * sqrt((double)n);
    return (int)std::max(1024.0, std::min(32768.0, ceil(m)));
}

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t dens_table_bytes(int M) {
    return up256(sizeof(TabCentre) * M) + up256(sizeof(double) * kTabK * M) + up256(sizeof(float2) * kTabK * M) +
           up256(sizeof(float) * kTabK * M);
}

cudaError_t dens_table_build(const Density &r, int M, void *buf, DensTab *out, cudaStream_t s) {
    memset(out, 0, sizeof(*out));
    if (r.kind < 2 || M < 2 || !buf) return cudaSuccess;
    unsigned char *b = (unsigned char *)buf;
    TabCentre *meta = (TabCentre *)b;
    b += up256(sizeof(TabCentre) * M);
    double *cf = (double *)b;
    b += up256(sizeof(double) * kTabK * M);
    float2 *cdf = (float2 *)b;
    b += up256(sizeof(float2) * kTabK * M);
    float *mag = (float *)b;
    const double dth = 3.14159265358979323846 / (M - 1);
    k_dens_table<<<(M + 127) / 128, 128, 0, s>>>(r, M, dth, meta, cf, cdf, mag);
    out->M = M;
    out->dth = (float)dth;
    out->meta = meta;
    out->cf = cf;
    out->cdf = cdf;
    out->mag = mag;
    return cudaGetLastError();
}

void cell_passes(const Grid &g, const CellOut &out, const CellBuf &cb, int *list1, int *list2, DevStatus *st,
                 int precision, const Tune &t, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, int64_t *launches,
                 int64_t *cell_launches, const Pipes *px, const cudaEvent_t *topo_ev) {
    // the cells are cut into nch chunks of consecutive bin positions, each run
    // through the whole pipeline on its own stream (the first on s); chunks
    // share nothing but the read-only generators, so their kernels overlap
    const int nch = std::max(1, std::min(t.chunks, px->n_aux + 1));
    unsigned *counts = px->counts;
    cudaMemsetAsync(counts, 0, sizeof(unsigned) * kChunkWords * kMaxChunks, s);
    if (nch > 1) {
        cudaEventRecord(px->fork, s);
        for (int c = 1; c < nch; ++c) cudaStreamWaitEvent(px->aux[c - 1], px->fork, 0);
    }
    const int scan_len = 2 * (g.n / 2048 + 64) + 64;
    const int wpb = t.topo_warps;
    const int cpw = 32 / t.topo_lanes;  // cells per warp
    const float kt = (float)t.knn_target;
    const int qb = t.quad_block;
    for (int c = 0; c < nch; ++c) {
        const cudaStream_t sc = (c == 0) ? s : px->aux[c - 1];
        const int p0 = (int)((long long)g.n * c / nch), p1 = (int)((long long)g.n * (c + 1) / nch);
        const int len = p1 - p0;
        if (len <= 0) continue;
        unsigned *rc = counts + kChunkWords * c;
        int *cw = (int *)rc;  // this chunk's words
        const bool timed = (c == 0 && nch == 1);
        nvtxRangePushA("scvt topology");
        if (timed && topo_ev) cudaEventRecord(topo_ev[0], sc);
        // first pass: a warp (or half warp) per cell, grid capped at topo_bpsm blocks per SM
        const int wblocks =
            (int)std::max<long long>(1, std::min<long long>((len + wpb * cpw - 1) / (wpb * cpw), 152LL * t.topo_bpsm / nch));
        if (t.topo_lanes == 16) {
            if (wpb == 2) k_topo_warp<2, 16><<<wblocks, 64, 0, sc>>>(g, out, cb, list1 + p0, rc, st, kt, p0, p1);
            else if (wpb == 8) k_topo_warp<8, 16><<<wblocks, 256, 0, sc>>>(g, out, cb, list1 + p0, rc, st, kt, p0, p1);
            else k_topo_warp<4, 16><<<wblocks, 128, 0, sc>>>(g, out, cb, list1 + p0, rc, st, kt, p0, p1);
        } else {
            if (wpb == 2) k_topo_warp<2, 32><<<wblocks, 64, 0, sc>>>(g, out, cb, list1 + p0, rc, st, kt, p0, p1);
            else if (wpb == 8) k_topo_warp<8, 32><<<wblocks, 256, 0, sc>>>(g, out, cb, list1 + p0, rc, st, kt, p0, p1);
            else k_topo_warp<4, 32><<<wblocks, 128, 0, sc>>>(g, out, cb, list1 + p0, rc, st, kt, p0, p1);
        }
        if (timed && topo_ev) cudaEventRecord(topo_ev[1], sc);
        // retry passes (thread per cell): sized for the worst case, they read their work count on the device
        const int rblocks = std::max(1, 2 * 152 / nch);
        k_topo<64, 64, 0><<<rblocks, 64, 0, sc>>>(g, out, cb, list1 + p0, rc, list2 + p0, rc + 1, 0, 0, st);
        // the last pass scans every generator of problems up to 20,000 generators
        k_topo<128, 64, 64><<<rblocks, 64, 0, sc>>>(g, out, cb, list2 + p0, rc + 1, nullptr, rc + 2, 1, 20000, st);
        // the chunk's edge list follows the previous chunk's: its first edge is
        // known once that chunk's count is, so the rebase waits for it
        exclusive_scan(cb.deg + p0, cb.eoff + p0, len, cb.scan_tmp + (size_t)c * scan_len, sc, launches);
        if (c > 0) cudaStreamWaitEvent(sc, px->rebased[c - 1], 0);
        const int ecap = 6 * g.n;
        k_rebase<<<(len + 255) / 256, 256, 0, sc>>>(p0, p1, cb.deg, cb.eoff,
                                                     c > 0 ? (const int *)(counts + kChunkWords * (c - 1)) : nullptr, cw,
                                                     ecap, &st->flags);
        if (c + 1 < nch) cudaEventRecord(px->rebased[c], sc);
        k_edge_cells<<<(len + 255) / 256, 256, 0, sc>>>(p0, p1, cb.deg, cb.eoff, cb.ecell, ecap);
        // the edge kernels loop over the chunk's edges (grid sized for about 6 per
        // cell; Euler: a full tessellation has 6N - 12 edge sides in all)
        const Span sp{p0, p1, cw + CW_EBASE, cw + CW_ETOT};
        const unsigned eblocks = (unsigned)((6 * len + qb - 1) / qb);
        const unsigned e256 = (unsigned)((6 * len + 255) / 256);
        const unsigned cblocks = (unsigned)((len + 255) / 256);
        nvtxRangePop();
        Phase pq("scvt corners, quadrature, cell sums");
        if (precision == 1) {
            k_corners32<<<e256, 256, 0, sc>>>(g, cb, sp);
            if (timed && ev0) cudaEventRecord(ev0, sc);
            k_quad32<<<eblocks, qb, 0, sc>>>(g, cb, ecap, sp);
            if (timed && ev1) cudaEventRecord(ev1, sc);
            k_cell_sum<1><<<cblocks, 256, 0, sc>>>(g, out, cb, ecap, st, sp);
        } else {
            const bool plain = precision == 2;
            if (plain) {
                k_corners<true><<<e256, 256, 0, sc>>>(g, cb, sp);
            } else {
                if (cb.ctab) {
                    k_cell_table<<<cblocks, 256, 0, sc>>>(g, cb, p0, p1);
                    (*launches)++;
                }
                k_corners<false><<<e256, 256, 0, sc>>>(g, cb, sp);
            }
            if (timed && ev0) cudaEventRecord(ev0, sc);
            if (plain) k_quad<true><<<eblocks, qb, 0, sc>>>(g, cb, ecap, sp, st);
            else k_quad<false><<<eblocks, qb, 0, sc>>>(g, cb, ecap, sp, st);
            if (timed && ev1) cudaEventRecord(ev1, sc);
            if (plain) k_cell_sum<2><<<cblocks, 256, 0, sc>>>(g, out, cb, ecap, st, sp);
            else k_cell_sum<0><<<cblocks, 256, 0, sc>>>(g, out, cb, ecap, st, sp);
        }
        (*launches) += 10;
        (*cell_launches) += 5;
    }
    if (nch > 1) {
        for (int c = 1; c < nch; ++c) {
            cudaEventRecord(px->join[c - 1], px->aux[c - 1]);
            cudaStreamWaitEvent(s, px->join[c - 1], 0);
        }
    }
    k_sum_counts<<<1, 1, 0, s>>>(counts, nch, st);
    (*launches)++;
}

}  // namespace scvt

namespace scvt {

cudaError_t pipes_create(Pipes &px, int n_aux) {
    px = Pipes();
    cudaError_t e = cudaMalloc((void **)&px.counts, sizeof(unsigned) * kChunkWords * kMaxChunks);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&px.fork, cudaEventDisableTiming);
    for (int k = 0; k < n_aux && k < kMaxChunks - 1 && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&px.aux[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&px.join[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&px.rebased[k], cudaEventDisableTiming);
        if (e == cudaSuccess) px.n_aux = k + 1;
    }
    return e;
}

void pipes_destroy(Pipes &px) {
    for (int k = 0; k < px.n_aux; ++k) {
        if (px.aux[k]) cudaStreamDestroy(px.aux[k]);
        if (px.join[k]) cudaEventDestroy(px.join[k]);
        if (px.rebased[k]) cudaEventDestroy(px.rebased[k]);
    }
    if (px.fork) cudaEventDestroy(px.fork);
    if (px.counts) cudaFree(px.counts);
    px = Pipes();
}

}  // namespace scvt
