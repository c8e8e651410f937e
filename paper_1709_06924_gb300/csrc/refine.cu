// refine.cu -- bisection refinement and mesh quality on a Voronoi topology
// (include/scvt.h, scvt_bisect and scvt_mesh_quality).
//
// Both read the neighbour cycles of every generator (original ids, as
// scvt_voronoi returns them).  Bisection (Sec. 4.3) appends the midpoint
// normalize(z_i + z_j) of every Delaunay edge i < j; the quality measures of
// Sec. 4 are cellQ = min / max great-circle length of a cell's edges and
// triQ = (a+b-c)(b+c-a)(c+a-b)/(abc) of each Delaunay triangle.  Each item is
// owned by its smallest generator id and listed in lexicographic order: a
// count per generator, an exclusive scan, then a write pass.
#include <cuda_runtime.h>
#include <math.h>

#include "scvt_internal.cuh"

namespace scvt {

namespace {

constexpr int kMaxNb = 32;

__device__ __forceinline__ void load3(const double *z, int i, double *p) {
    p[0] = z[3 * (size_t)i];
    p[1] = z[3 * (size_t)i + 1];
    p[2] = z[3 * (size_t)i + 2];
}

// great-circle length atan2(|a x b|, a.b)
__device__ __forceinline__ double arc(const double *a, const double *b) {
    const double cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2], cz = a[0] * b[1] - a[1] * b[0];
    return atan2(sqrt(cx * cx + cy * cy + cz * cz), a[0] * b[0] + a[1] * b[1] + a[2] * b[2]);
}

__global__ void k_edge_count(int n, const int *__restrict__ deg, const int *__restrict__ nbr, int maxd,
                             int *__restrict__ cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = 0;
    for (int k = 0; k < deg[i]; ++k) c += nbr[(size_t)i * maxd + k] > i;
    cnt[i] = c;
}

// the generators, then the midpoints of their edges to larger ids, ascending;
// the midpoint is rounded like (z_i + z_j) / sqrt(x^2 + y^2 + z^2) summed left
// to right without fused operations
__global__ void k_bisect_write(int n, const double *__restrict__ z, const int *__restrict__ deg,
                               const int *__restrict__ nbr, int maxd, const int *__restrict__ off,
                               double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double zi[3];
    load3(z, i, zi);
    out[3 * (size_t)i] = zi[0];
    out[3 * (size_t)i + 1] = zi[1];
    out[3 * (size_t)i + 2] = zi[2];
    int js[kMaxNb];
    int d = 0;
    for (int k = 0; k < deg[i]; ++k) {
        const int j = nbr[(size_t)i * maxd + k];
        if (j > i) {
            int p = d++;
            while (p > 0 && js[p - 1] > j) {
                js[p] = js[p - 1];
                --p;
            }
            js[p] = j;
        }
    }
    for (int t = 0; t < d; ++t) {
        double zj[3];
        load3(z, js[t], zj);
        const double x = __dadd_rn(zi[0], zj[0]), y = __dadd_rn(zi[1], zj[1]), w = __dadd_rn(zi[2], zj[2]);
        const double r = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(w, w)));
        const size_t o = 3 * ((size_t)n + off[i] + t);
        out[o] = __ddiv_rn(x, r);
        out[o + 1] = __ddiv_rn(y, r);
        out[o + 2] = __ddiv_rn(w, r);
    }
}

// corner between neighbours a and b of cell i: the circumcentre direction of
// (z_i, z_a, z_b) on the side of z_i
__device__ __forceinline__ void corner(const double *zi, const double *za, const double *zb, double *v) {
    const double u0 = za[0] - zi[0], u1 = za[1] - zi[1], u2 = za[2] - zi[2];
    const double w0 = zb[0] - zi[0], w1 = zb[1] - zi[1], w2 = zb[2] - zi[2];
    double c0 = u1 * w2 - u2 * w1, c1 = u2 * w0 - u0 * w2, c2 = u0 * w1 - u1 * w0;
    const double s = c0 * zi[0] + c1 * zi[1] + c2 * zi[2];
    const double inv = (s >= 0.0 ? 1.0 : -1.0) / sqrt(c0 * c0 + c1 * c1 + c2 * c2);
    v[0] = c0 * inv;
    v[1] = c1 * inv;
    v[2] = c2 * inv;
}

__global__ void k_cell_quality(int n, const double *__restrict__ z, const int *__restrict__ deg,
                               const int *__restrict__ nbr, int maxd, double *__restrict__ cellq) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int d = deg[i];
    const int *nb = nbr + (size_t)i * maxd;
    double zi[3], za[3], zb[3], v0[3], vp[3], vc[3];
    load3(z, i, zi);
    load3(z, nb[0], za);
    load3(z, nb[1 % d], zb);
    corner(zi, za, zb, v0);
    vp[0] = v0[0]; vp[1] = v0[1]; vp[2] = v0[2];
    double lo = INFINITY, hi = 0.0;
    for (int k = 1; k <= d; ++k) {
        if (k < d) {
            load3(z, nb[k], za);
            load3(z, nb[(k + 1) % d], zb);
            corner(zi, za, zb, vc);
        } else {
            vc[0] = v0[0]; vc[1] = v0[1]; vc[2] = v0[2];
        }
        const double L = arc(vp, vc);
        lo = fmin(lo, L);
        hi = fmax(hi, L);
        vp[0] = vc[0]; vp[1] = vc[1]; vp[2] = vc[2];
    }
    cellq[i] = lo / hi;
}

__global__ void k_tri_count(int n, const int *__restrict__ deg, const int *__restrict__ nbr, int maxd,
                            int *__restrict__ cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int d = deg[i];
    const int *nb = nbr + (size_t)i * maxd;
    int c = 0;
    for (int k = 0; k < d; ++k) c += (nb[k] > i && nb[(k + 1) % d] > i);
    cnt[i] = c;
}

// triangles (i, j, k), i < j < k, owned by i, in ascending (j, k)
__global__ void k_tri_write(int n, const double *__restrict__ z, const int *__restrict__ deg,
                            const int *__restrict__ nbr, int maxd, const int *__restrict__ off,
                            double *__restrict__ triq) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int d = deg[i];
    const int *nb = nbr + (size_t)i * maxd;
    long long keys[kMaxNb];
    int m = 0;
    for (int k = 0; k < d; ++k) {
        int a = nb[k], b = nb[(k + 1) % d];
        if (a > i && b > i) {
            if (a > b) { const int t = a; a = b; b = t; }
            const long long key = ((long long)a << 32) | (unsigned)b;
            int p = m++;
            while (p > 0 && keys[p - 1] > key) {
                keys[p] = keys[p - 1];
                --p;
            }
            keys[p] = key;
        }
    }
    double A[3], B[3], C[3];
    load3(z, i, A);
    for (int t = 0; t < m; ++t) {
        load3(z, (int)(keys[t] >> 32), B);
        load3(z, (int)(keys[t] & 0xffffffffLL), C);
        const double a = arc(B, C), b = arc(C, A), c = arc(A, B);
        triq[off[i] + t] = (a + b - c) * (b + c - a) * (c + a - b) / (a * b * c);
    }
}

}  // namespace

cudaError_t bisect_midpoints(int n, const double *z, const int *deg, const int *nbr, int maxd, int *cnt, int *off,
                             int *scan_tmp, double *out, int64_t cap, int64_t *n_out, cudaStream_t s) {
    const unsigned blocks = (unsigned)((n + 255) / 256);
    int64_t launches = 0;
    k_edge_count<<<blocks, 256, 0, s>>>(n, deg, nbr, maxd, cnt);
    exclusive_scan(cnt, off, n, scan_tmp, s, &launches);
    int last[2];
    cudaError_t e = cudaMemcpyAsync(&last[0], off + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last[1], cnt + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    *n_out = (int64_t)n + last[0] + last[1];
    if (*n_out > cap) return cudaSuccess;  // the caller reports the size
    k_bisect_write<<<blocks, 256, 0, s>>>(n, z, deg, nbr, maxd, off, out);
    return cudaGetLastError();
}

cudaError_t mesh_quality(int n, const double *z, const int *deg, const int *nbr, int maxd, int *cnt, int *off,
                         int *scan_tmp, double *cellq, double *triq, int64_t cap, int64_t *n_tri, cudaStream_t s) {
    const unsigned blocks = (unsigned)((n + 255) / 256);
    int64_t launches = 0;
    if (cellq) k_cell_quality<<<blocks, 256, 0, s>>>(n, z, deg, nbr, maxd, cellq);
    k_tri_count<<<blocks, 256, 0, s>>>(n, deg, nbr, maxd, cnt);
    exclusive_scan(cnt, off, n, scan_tmp, s, &launches);
    int last[2];
    cudaError_t e = cudaMemcpyAsync(&last[0], off + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last[1], cnt + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    *n_tri = (int64_t)last[0] + last[1];
    if (triq && *n_tri <= cap) k_tri_write<<<blocks, 256, 0, s>>>(n, z, deg, nbr, maxd, off, triq);
    return cudaGetLastError();
}

}  // namespace scvt
