// lbfgs.cu -- HBM-streaming kernels of the LBFGS iteration and the
// deterministic reductions.
//
// Every reduction uses a fixed partition: the index range is cut into
// reduce_blocks(n) contiguous chunks, each summed by one block in a fixed
// order, and the chunk sums are added by one block in a fixed order.  The
// result therefore depends only on n and the data, never on launch timing or
// on the binning of an evaluation.
//
// The two-loop recursion (Sec. 2.2.2) keeps its scalars alpha_k, beta_k on
// the device.  With up to kCmpMax pairs it runs as three gathered passes
// (each vector of the history read once or twice per direction, see the
// comment above cmp_pass_a); otherwise one pass per step, each fusing the
// axpy of one step with the dot product of the next.  A pass's last block
// to finish turns the chunk sums into the next scalars, so the direction
// runs back to back without a host round trip.
#include <math.h>
#include <string.h>

#include "scvt_internal.cuh"

namespace scvt {

namespace {

constexpr int kRT = 256;  // threads of the chunk kernels

template <int NQ>
__device__ __forceinline__ void block_sum_store(double (&v)[NQ], double *dst) {
    __shared__ double sh[NQ][kRT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double x = v[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[q][w] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double s = 0.0;
            for (int k = 0; k < kRT / 32; ++k) s += sh[q][k];
            dst[q] = s;
        }
    }
}

// contiguous chunk k of nb chunks of [0, n)
__device__ __forceinline__ void chunk_range(int64_t n, int nb, int k, int64_t &b0, int64_t &b1) {
    int64_t chunk = (n + nb - 1) / nb;
    b0 = (int64_t)k * chunk;
    b1 = b0 + chunk < n ? b0 + chunk : n;
}

__device__ __forceinline__ void chunk_of(int64_t n, int64_t &b0, int64_t &b1) {
    chunk_range(n, gridDim.x, blockIdx.x, b0, b1);
}

__global__ void k_reduce_eval(int n, const double *__restrict__ fcell, const double *__restrict__ g,
                              const double *__restrict__ q, const double *__restrict__ nrm,
                              double *__restrict__ partials) {
    int64_t b0, b1;
    chunk_of(n, b0, b1);
    double v[3] = {0.0, 0.0, 0.0};
    for (int64_t i = b0 + threadIdx.x; i < b1; i += kRT) {
        double gx = g[3 * i], gy = g[3 * i + 1], gz = g[3 * i + 2];
        v[0] += fcell[i];
        v[1] += gx * gx + gy * gy + gz * gz;
        if (q) v[2] += (gx * q[3 * i] + gy * q[3 * i + 1] + gz * q[3 * i + 2]) * nrm[i];
    }
    block_sum_store<3>(v, partials + 4 * blockIdx.x);
}

// one block: out[q] = sum_b partials[stride*b + q] in a fixed order
template <int NQ>
__global__ void k_finish(const double *__restrict__ partials, int nb, int stride, double *out) {
    double v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = 0.0;
    for (int b = threadIdx.x; b < nb; b += kRT)
#pragma unroll
        for (int q = 0; q < NQ; ++q) v[q] += partials[(size_t)stride * b + q];
    double res[NQ];
    block_sum_store<NQ>(v, res);
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < NQ; ++q) out[q] = res[q];
}

// out = scale * sum (scale may be null); if minus_from: out = *minus_from - out
__global__ void k_finish_scalar(const double *__restrict__ partials, int nb, const double *scale,
                                const double *minus_from, double *out) {
    double v[1] = {0.0};
    for (int b = threadIdx.x; b < nb; b += kRT) v[0] += partials[b];
    double res[1];
    block_sum_store<1>(v, res);
    if (threadIdx.x == 0) {
        double r = scale ? scale[0] * res[0] : res[0];
        if (minus_from) r = minus_from[0] - r;
        out[0] = r;
    }
}

__global__ void k_dot(int64_t len, const double *__restrict__ x, const double *__restrict__ y,
                      double *__restrict__ partials) {
    int64_t b0, b1;
    chunk_of(len, b0, b1);
    double v[1] = {0.0};
    for (int64_t i = b0 + threadIdx.x; i < b1; i += kRT) v[0] += x[i] * y[i];
    block_sum_store<1>(v, partials + blockIdx.x);
}

__global__ void k_trial(int n, const double *__restrict__ z, const double *__restrict__ q, double alpha,
                        double *__restrict__ zt, double *__restrict__ nrm) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = z[3 * (size_t)i] + alpha * q[3 * (size_t)i];
    double y = z[3 * (size_t)i + 1] + alpha * q[3 * (size_t)i + 1];
    double w = z[3 * (size_t)i + 2] + alpha * q[3 * (size_t)i + 2];
    // one reciprocal square root (FP64 divisions and square roots are
    // sequences on the FP64 pipe, which bounds these vector kernels)
    double r = rsqrt(x * x + y * y + w * w);
    zt[3 * (size_t)i] = x * r;
    zt[3 * (size_t)i + 1] = y * r;
    zt[3 * (size_t)i + 2] = w * r;
    nrm[i] = r;
}

__global__ void k_lloyd(int n, const double *__restrict__ c, double *__restrict__ zout) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = c[3 * (size_t)i], y = c[3 * (size_t)i + 1], w = c[3 * (size_t)i + 2];
    double r = sqrt(x * x + y * y + w * w);
    zout[3 * (size_t)i] = x / r;
    zout[3 * (size_t)i + 1] = y / r;
    zout[3 * (size_t)i + 2] = w / r;
}

// *out = max(*out, sqrt of the warp's largest v) for v >= 0: one atomic per
// warp (nonnegative doubles order like their bit patterns)
__device__ __forceinline__ void warp_max_to(double v, unsigned long long *out) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(sqrt(v)));
}

// s = zt - z, y = gt - g; partial sums of y.s, y.y, s.s; max |s_i|
__global__ void k_accept(int n, const double *__restrict__ zt, const double *__restrict__ z,
                         const double *__restrict__ gt, const double *__restrict__ g, double *__restrict__ S,
                         double *__restrict__ Y, double *__restrict__ partials, unsigned long long *maxmove) {
    int64_t b0, b1;
    chunk_of(n, b0, b1);
    double v[3] = {0.0, 0.0, 0.0};
    double mv = 0.0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += kRT) {
        double s2 = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double s = zt[3 * i + d] - z[3 * i + d];
            double y = gt[3 * i + d] - g[3 * i + d];
            S[3 * i + d] = s;
            Y[3 * i + d] = y;
            v[0] += y * s;
            v[1] += y * y;
            s2 += s * s;
        }
        v[2] += s2;
        mv = fmax(mv, s2);
    }
    warp_max_to(mv, maxmove);
    block_sum_store<3>(v, partials + 4 * blockIdx.x);
}

// the same per problem: blockIdx.y = problem, blockIdx.x = chunk of that
// problem (reduce_blocks(n_b) chunks, as for a single problem of size n_b)
__global__ void k_reduce_eval_batch(const InstGeom *__restrict__ inst, const int *__restrict__ pbase,
                                    const int *__restrict__ active, const double *__restrict__ fcell,
                                    const double *__restrict__ g, const double *__restrict__ q,
                                    const double *__restrict__ nrm, double *__restrict__ partials) {
    const int b = blockIdx.y;
    if (active && !active[b]) return;
    const InstGeom I = inst[b];
    int64_t nb = (I.n + 4095) / 4096;
    nb = nb < 1 ? 1 : (nb > 1024 ? 1024 : nb);
    if (blockIdx.x >= nb) return;
    const int64_t chunk = (I.n + nb - 1) / nb;
    const int64_t b0 = (int64_t)blockIdx.x * chunk, b1 = b0 + chunk < I.n ? b0 + chunk : I.n;
    double v[3] = {0.0, 0.0, 0.0};
    for (int64_t j = b0 + threadIdx.x; j < b1; j += kRT) {
        const int64_t i = I.p0 + j;
        double gx = g[3 * i], gy = g[3 * i + 1], gz = g[3 * i + 2];
        v[0] += fcell[i];
        v[1] += gx * gx + gy * gy + gz * gz;
        if (q) v[2] += (gx * q[3 * i] + gy * q[3 * i + 1] + gz * q[3 * i + 2]) * nrm[i];
    }
    block_sum_store<3>(v, partials + 4 * ((int64_t)pbase[b] + blockIdx.x));
}

// block b: ist[b].red[q] = sum of problem b's chunk sums, in chunk order
__global__ void k_finish_batch(const InstGeom *__restrict__ inst, const int *__restrict__ pbase,
                               const int *__restrict__ active, const double *__restrict__ partials,
                               DevStatus *ist) {
    const int b = blockIdx.x;
    if (active && !active[b]) return;
    int nb = (inst[b].n + 4095) / 4096;
    nb = nb < 1 ? 1 : (nb > 1024 ? 1024 : nb);
    const double *pp = partials + 4 * (int64_t)pbase[b];
    double v[3] = {0.0, 0.0, 0.0};
    for (int k = threadIdx.x; k < nb; k += kRT)
#pragma unroll
        for (int q = 0; q < 3; ++q) v[q] += pp[4 * k + q];
    double res[3];
    block_sum_store<3>(v, res);
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < 3; ++q) ist[b].red[q] = res[q];
}

__global__ void k_set_rho(double *rho, const DevStatus *st) { rho[0] = 1.0 / st->dots[0]; }

// plain LBFGS: gamma = y.s / y.y of the newest pair (Sec. 2.2.2)
__global__ void k_set_gamma(double *gamma, const DevStatus *st) { gamma[0] = st->dots[0] / st->dots[1]; }

// ---- direction passes (two-loop recursion) ----
// Vectors read once per pass (the history pairs, g) are loaded with an L2
// evict-first policy, so the direction q -- written and read again by every
// pass, 24 bytes per generator -- stays resident in L2 between passes.
__device__ __forceinline__ unsigned long long policy_evict_first() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ double ld_stream(const double *a, unsigned long long pol) {
    double v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(a), "l"(pol));
    return v;
}

// The scalar a pass leaves for the next one, taken by the last of its
// blocks to finish: the chunk sums in block order (the same fixed partition
// as every reduction here), out = scale * sum, or minus_from - scale * sum.
// Each block's chunk sum is published before its ticket; the last ticket
// holder therefore reads every sum (at L2, where they were published: the
// loads bypass L1 and need not be ordered among themselves), and resets the
// ticket counter for the next pass.
// (nb chunks; this block's chunk is k)
__device__ __forceinline__ void finish_by_last_block(double v, double *__restrict__ partials, unsigned *ticket, int nb,
                                                     int k, const double *scale, const double *minus_from,
                                                     double *out) {
    double vv[1] = {v};
    block_sum_store<1>(vv, partials + k);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == (unsigned)nb - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double w[1] = {0.0};
    for (int b = threadIdx.x; b < nb; b += kRT) w[0] += __ldcg(partials + b);
    double res[1];
    block_sum_store<1>(w, res);
    if (threadIdx.x == 0) {
        double r = scale ? scale[0] * res[0] : res[0];
        if (minus_from) r = minus_from[0] - r;
        out[0] = r;
        *ticket = 0u;
    }
}

// one step of the recursion over the chunk [b0, b1): q = (q0 + sign coef x)
// [* h or * hs[0]] with q0 = q (or -x for the first pass: coef = null);
// returns this thread's share of w.q
__device__ __forceinline__ double step_chunk(int64_t b0, int64_t b1, double *__restrict__ q,
                                             const double *__restrict__ coef, double sign, const double *__restrict__ x,
                                             const double *__restrict__ h, const double *__restrict__ hs,
                                             const double *__restrict__ w) {
    const unsigned long long pol = policy_evict_first();
    const double a = coef ? sign * coef[0] : 0.0;
    const double sc = hs ? hs[0] : 1.0;
    double v = 0.0;
    // four elements per thread and iteration, their loads issued together
    constexpr int U = 4;
    for (int64_t i0 = b0 + threadIdx.x; i0 < b1; i0 += U * kRT) {
        double xv[U], wv[U], qv[U], hv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + (int64_t)u * kRT;
            if (i < b1) {
                xv[u] = ld_stream(x + i, pol);
                wv[u] = ld_stream(w + i, pol);
                qv[u] = coef ? q[i] : 0.0;
                hv[u] = h ? h[i / 3] : sc;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + (int64_t)u * kRT;
            if (i < b1) {
                double t = coef ? qv[u] + a * xv[u] : -xv[u];
                if (h || hs) t *= hv[u];
                q[i] = t;
                v += wv[u] * t;
            }
        }
    }
    return v;
}

// one step of the recursion, then the next scalar from w.q (finish_by_last_block)
__global__ void __launch_bounds__(kRT) k_step(int64_t len, double *__restrict__ q, const double *__restrict__ coef,
                                              double sign, const double *__restrict__ x,
                                              const double *__restrict__ h, const double *__restrict__ hs,
                                              const double *__restrict__ w, double *__restrict__ partials,
                                              unsigned *ticket, const double *scale, const double *minus_from,
                                              double *out) {
    int64_t b0, b1;
    chunk_of(len, b0, b1);
    const double v = step_chunk(b0, b1, q, coef, sign, x, h, hs, w);
    finish_by_last_block(v, partials, ticket, gridDim.x, blockIdx.x, scale, minus_from, out);
}

// ---- segmented LBFGS kernels (many problems per launch) ----
// the problem whose blocks hold block `blk` (first block of each problem in
// `first`, ascending)
__device__ __forceinline__ int lane_of_block(const SegLane *__restrict__ L, int nl, int blk, bool acc) {
    int lo = 0, hi = nl - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((acc ? L[mid].blk1 : L[mid].blk3) <= blk) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// pass t of the two-loop recursion of every problem with 0 or more than
// kCmpMax pairs: t = 0 sets q = -g, passes 1..c are the backward steps
// (newest pair first; the last applies the initial matrix), passes c+1..2c
// the forward steps -- the same steps, pointers and scalars as two_loop()
// for one problem
__global__ void __launch_bounds__(kRT) k_seg_step(const SegLane *__restrict__ lanes, int nl, int t,
                                                  double *__restrict__ q_rows) {
    const int b = lane_of_block(lanes, nl, blockIdx.x, false);
    const SegLane &L = lanes[b];
    const int c = L.count;
    if (!L.dir || (c >= 1 && c <= kCmpMax) || t > 2 * c) return;
    const int k = blockIdx.x - L.blk3;
    if (k >= L.nb3) return;
    const int64_t len = 3 * (int64_t)L.n;
    double *q = q_rows + 3 * L.row;
    double *alpha = L.scal + kScalAlpha, *coef = L.scal + kScalCoef;
    unsigned *ticket = reinterpret_cast<unsigned *>(L.scal + kScalTicket);
    auto S = [&](int j) { return (const double *)(L.hist + (size_t)L.slots[j] * L.slot_stride); };
    auto Y = [&](int j) { return (const double *)(L.yhist + (size_t)L.slots[j] * L.slot_stride); };
    auto R = [&](int j) { return (const double *)(L.rho + L.slots[j]); };
    // initial matrix: diag(h), or gamma I (plain LBFGS with pairs), or I
    const double *h0 = L.method == 1 ? nullptr : L.h;
    const double *hs0 = (L.method == 1 && c > 0) ? L.rho + kLaneMaxM + 1 : nullptr;
    const double *coef_p = nullptr, *x, *h = nullptr, *hs = nullptr, *w, *scale = nullptr, *minus = nullptr;
    double sign = 0.0, *out;
    if (t == 0) {
        x = L.g;
        if (c == 0) {
            h = h0;
            hs = hs0;
            w = L.g;
            out = &L.st->dots[3];
        } else {
            w = S(c - 1);
            scale = R(c - 1);
            out = alpha + c - 1;
        }
    } else if (t <= c) {
        const int j = c - t;
        coef_p = alpha + j;
        sign = -1.0;
        x = Y(j);
        if (j > 0) {
            w = S(j - 1);
            scale = R(j - 1);
            out = alpha + j - 1;
        } else {
            h = h0;
            hs = hs0;
            w = Y(0);
            scale = R(0);
            minus = alpha;
            out = coef;
        }
    } else {
        const int j = t - c - 1;
        coef_p = coef + j;
        sign = 1.0;
        x = S(j);
        if (j + 1 < c) {
            w = Y(j + 1);
            scale = R(j + 1);
            minus = alpha + j + 1;
            out = coef + j + 1;
        } else {
            w = L.g;
            out = &L.st->dots[3];
        }
    }
    int64_t b0, b1;
    chunk_range(len, L.nb3, k, b0, b1);
    const double v = step_chunk(b0, b1, q, coef_p, sign, x, h, hs, w);
    finish_by_last_block(v, L.partials, ticket, L.nb3, k, scale, minus, out);
}

__global__ void k_seg_trial(const SegLane *__restrict__ lanes, const int *__restrict__ pinst, int64_t ntot,
                            const double *__restrict__ q_rows, double *__restrict__ zt_rows,
                            double *__restrict__ nrm_rows) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= ntot) return;
    const SegLane &L = lanes[pinst[r]];
    if (!L.trial) return;
    const int64_t i = r - L.row;
    const double a = L.alpha;
    // the arithmetic of k_trial
    double x = L.z[3 * i] + a * q_rows[3 * r];
    double y = L.z[3 * i + 1] + a * q_rows[3 * r + 1];
    double w = L.z[3 * i + 2] + a * q_rows[3 * r + 2];
    double nr = rsqrt(x * x + y * y + w * w);
    zt_rows[3 * r] = x * nr;
    zt_rows[3 * r + 1] = y * nr;
    zt_rows[3 * r + 2] = w * nr;
    nrm_rows[r] = nr;
}

__global__ void __launch_bounds__(kRT) k_seg_accept(const SegLane *__restrict__ lanes, int nl,
                                                    const double *__restrict__ zt_rows,
                                                    const double *__restrict__ gt_rows,
                                                    const double *__restrict__ ht_rows) {
    const int b = lane_of_block(lanes, nl, blockIdx.x, true);
    const SegLane &L = lanes[b];
    if (!L.accept) return;
    const int k = blockIdx.x - L.blk1;
    if (k >= L.nb1) return;
    double *S = L.hist + (size_t)L.spare * L.slot_stride;
    double *Y = L.yhist + (size_t)L.spare * L.slot_stride;
    const double *zt = zt_rows + 3 * L.row, *gt = gt_rows + 3 * L.row, *ht = ht_rows + L.row;
    int64_t b0, b1;
    chunk_range(L.n, L.nb1, k, b0, b1);
    // the arithmetic of k_accept, then the iterate moves to the trial point
    double v[3] = {0.0, 0.0, 0.0};
    double mv = 0.0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += kRT) {
        double s2 = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double zn = zt[3 * i + d], gn = gt[3 * i + d];
            double s = zn - L.z[3 * i + d];
            double y = gn - L.g[3 * i + d];
            S[3 * i + d] = s;
            Y[3 * i + d] = y;
            v[0] += y * s;
            v[1] += y * y;
            s2 += s * s;
            L.z[3 * i + d] = zn;
            L.g[3 * i + d] = gn;
        }
        v[2] += s2;
        L.h[i] = ht[i];
        mv = fmax(mv, s2);
    }
    warp_max_to(mv, &L.st->maxmove_bits);
    // chunk sums, then the last block: the dots in the order of k_finish<3>,
    // and 1/(y.s) (gamma) when the curvature test passes
    block_sum_store<3>(v, L.partials + 4 * k);
    __shared__ bool last;
    unsigned *ticket = reinterpret_cast<unsigned *>(L.scal + kScalAcceptTicket);
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == (unsigned)L.nb1 - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double w[3] = {0.0, 0.0, 0.0};
    for (int c = threadIdx.x; c < L.nb1; c += kRT)
#pragma unroll
        for (int q = 0; q < 3; ++q) w[q] += __ldcg(L.partials + 4 * c + q);
    double res[3];
    block_sum_store<3>(w, res);
    if (threadIdx.x == 0) {
        L.st->dots[0] = res[0];
        L.st->dots[1] = res[1];
        L.st->dots[2] = res[2];
        if (L.method != 2 && L.m > 0 && res[0] > 1e-12 * sqrt(res[1]) * sqrt(res[2])) {
            L.rho[L.spare] = 1.0 / res[0];
            if (L.method == 1) L.rho[kLaneMaxM + 1] = res[0] / res[1];
        }
        *ticket = 0u;
    }
}

// ---- gathered direction passes (1 .. kCmpMax pairs) ----
// The two-loop recursion with each loop's vector updates gathered into one
// pass.  Backward loop: q_c = -g, alpha_j = rho_j s_j.q_{j+1}, q_j = q_{j+1}
// - alpha_j y_j; as q_{j+1} = -g - sum_{i>j} alpha_i y_i,
//     s_j.q_{j+1} = -s_j.g - sum_{i>j} alpha_i (s_j.y_i).
// Forward loop: r_0 = H0 q_0, beta_j = rho_j y_j.r_j, r_{j+1} = r_j +
// coef_j s_j with coef_j = alpha_j - beta_j; as r_j = r_0 + sum_{i<j} coef_i
// s_i,
//     y_j.r_j = y_j.r_0 + sum_{i<j} coef_i (s_i.y_j).
// The products s_a.y_b (a older than b) stay in the problem's scalars by
// history slot.  The newest pair's products with the older pairs come from
// the s_a.g of two successive directions: y = g' - g, so s_a.y = s_a.g' -
// s_a.g, with g the gradient its direction used and g' the next one.  That
// saves count - 1 FP64 multiply-adds per component, and on this GPU the
// FP64 pipe, not HBM, bounds the direction: one FP64 multiply-add per
// component and step of the recursion (4 count + 2 in all) against
// 8 bytes moved per component and step.
//   A: s_j.g for every pair; the last block forms the newest pair's
//      products (if it is new), keeps s_j.g, and runs the backward
//      recursion, newest first;
//   B: q_0 = -g - sum alpha_j y_j (newest first), r_0 = H0 q_0 into q;
//      y_j.r_0 and g.r_0; the last block runs the forward recursion, oldest
//      first, and leaves g.q = g.r_0 + sum coef_j s_j.g;
//   C: q = r_0 + sum coef_j s_j (oldest first).
// Per component, q is formed by the fused multiply-adds of the step-by-step
// passes in their order; the dot products are summed differently, so the two
// agree to rounding.  Each block takes one chunk of the 3n components (the
// partition of every reduction here) with kCT threads and at most 72
// registers a thread, so that the 1024 chunks of the largest problems are
// resident at once on 152 SMs (7 blocks each).
constexpr int kCT = 128;

__device__ __forceinline__ const double *lane_S(const SegLane &L, int j) {
    return L.hist + (size_t)L.slots[j] * L.slot_stride;
}
__device__ __forceinline__ const double *lane_Y(const SegLane &L, int j) {
    return L.yhist + (size_t)L.slots[j] * L.slot_stride;
}

// The block's sums of v go to partials[q nb + k]; the last block to finish
// (ticket counter) returns true, its thread 0 holding in res the sums over
// all chunks in chunk order, and resets the counter.
template <int NQ>
__device__ __forceinline__ bool cmp_sums(const double (&v)[NQ], double *__restrict__ partials, unsigned *ticket,
                                         int nb, int k, double (&res)[NQ]) {
    __shared__ double sh[NQ][kCT / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double x = v[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[q][w] = x;
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
        double t = 0.0;
#pragma unroll
        for (int j = 0; j < kCT / 32; ++j) t += sh[threadIdx.x][j];
        partials[(size_t)threadIdx.x * nb + k] = t;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == (unsigned)nb - 1;
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double a[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) a[q] = 0.0;
    for (int b = threadIdx.x; b < nb; b += kCT)
#pragma unroll
        for (int q = 0; q < NQ; ++q) a[q] += __ldcg(partials + (size_t)q * nb + b);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double x = a[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[q][w] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double t = 0.0;
#pragma unroll
            for (int j = 0; j < kCT / 32; ++j) t += sh[q][j];
            res[q] = t;
        }
        *ticket = 0u;
    }
    return true;
}

// The pair count C is a compile-time constant of each pass (the kernels
// switch on the lane's count): FP64 instructions of absent pairs, even
// predicated off, would hold the FP64 pipe.
// DIRECT: the newest pair's products as dot products s_j.y_newest (for a
// history given from outside, without the previous directions' s_j.g)
template <bool DIRECT, int C>
__device__ __forceinline__ void cmp_pass_a(const SegLane &L, int k) {
    int64_t b0, b1;
    chunk_range(3 * (int64_t)L.n, L.nb3, k, b0, b1);
    const unsigned long long pol = policy_evict_first();
    const double *S[C];
#pragma unroll
    for (int j = 0; j < C; ++j) S[j] = lane_S(L, j);
    const double *yn = lane_Y(L, C - 1);
    constexpr int NQ = DIRECT ? 2 * C - 1 : C;
    double v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = 0.0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += kCT) {
        const double gi = ld_stream(L.g + i, pol);
        const double yi = DIRECT ? ld_stream(yn + i, pol) : 0.0;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const double sj = ld_stream(S[j] + i, pol);
            v[j] = fma(sj, gi, v[j]);
            if constexpr (DIRECT)
                if (j + 1 < C) v[C + j] = fma(sj, yi, v[C + j]);
        }
    }
    double res[NQ];
    if (!cmp_sums<NQ>(v, L.partials, reinterpret_cast<unsigned *>(L.scal + kScalTicket), L.nb3, k, res)) return;
    if (threadIdx.x != 0) return;
    double *alpha = L.scal + kScalAlpha, *u = L.scal + kScalU, *G = L.rho + kLaneGram, *sg = L.rho + kLaneSg;
    const int sn = L.slots[C - 1];
    if (DIRECT)
        for (int j = 0; j + 1 < C; ++j) G[L.slots[j] * kGramDim + sn] = res[C + j];
    else if (L.new_pair)
        for (int j = 0; j + 1 < C; ++j) G[L.slots[j] * kGramDim + sn] = res[j] - sg[L.slots[j]];
    for (int j = 0; j < C; ++j) {
        u[j] = res[j];
        sg[L.slots[j]] = res[j];
    }
    for (int j = C - 1; j >= 0; --j) {
        const int sj = L.slots[j];
        double d = -res[j];
        for (int i = C - 1; i > j; --i) d = fma(-alpha[i], G[sj * kGramDim + L.slots[i]], d);
        alpha[j] = L.rho[sj] * d;
    }
}

template <int C>
__device__ __forceinline__ void cmp_pass_b(const SegLane &L, int k, double *__restrict__ q) {
    int64_t b0, b1;
    chunk_range(3 * (int64_t)L.n, L.nb3, k, b0, b1);
    const unsigned long long pol = policy_evict_first();
    const double *alpha = L.scal + kScalAlpha;
    const double *Y[C];
    double na[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
        Y[j] = lane_Y(L, j);
        na[j] = -alpha[j];
    }
    // initial matrix: diag(h), or gamma I (plain LBFGS)
    const double *h = L.method == 1 ? nullptr : L.h;
    const double gam = L.method == 1 ? L.rho[kLaneMaxM + 1] : 1.0;
    constexpr int NQ = C + 1;
    double v[NQ];
#pragma unroll
    for (int j = 0; j < NQ; ++j) v[j] = 0.0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += kCT) {
        const double gi = ld_stream(L.g + i, pol);
        double yv[C];
#pragma unroll
        for (int j = 0; j < C; ++j) yv[j] = ld_stream(Y[j] + i, pol);
        const double hv = h ? h[i / 3] : gam;
        double t = -gi;
#pragma unroll
        for (int j = C - 1; j >= 0; --j) t = fma(na[j], yv[j], t);
        t *= hv;
        q[i] = t;
#pragma unroll
        for (int j = 0; j < C; ++j) v[j] = fma(yv[j], t, v[j]);
        v[C] = fma(gi, t, v[C]);
    }
    double res[NQ];
    if (!cmp_sums<NQ>(v, L.partials, reinterpret_cast<unsigned *>(L.scal + kScalTicket), L.nb3, k, res)) return;
    if (threadIdx.x != 0) return;
    double *coef = L.scal + kScalCoef;
    const double *u = L.scal + kScalU, *G = L.rho + kLaneGram;
    for (int j = 0; j < C; ++j) {
        const int sj = L.slots[j];
        double d = res[j];
        for (int i = 0; i < j; ++i) d = fma(coef[i], G[L.slots[i] * kGramDim + sj], d);
        coef[j] = fma(-L.rho[sj], d, alpha[j]);
    }
    double gd = res[C];
    for (int j = 0; j < C; ++j) gd = fma(coef[j], u[j], gd);
    L.st->dots[3] = gd;
}

template <int C>
__device__ __forceinline__ void cmp_pass_c(const SegLane &L, int k, double *__restrict__ q) {
    int64_t b0, b1;
    chunk_range(3 * (int64_t)L.n, L.nb3, k, b0, b1);
    const unsigned long long pol = policy_evict_first();
    const double *coef = L.scal + kScalCoef;
    const double *S[C];
    double cf[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
        S[j] = lane_S(L, j);
        cf[j] = coef[j];
    }
    for (int64_t i = b0 + threadIdx.x; i < b1; i += kCT) {
        double sv[C];
#pragma unroll
        for (int j = 0; j < C; ++j) sv[j] = ld_stream(S[j] + i, pol);
        double t = q[i];
#pragma unroll
        for (int j = 0; j < C; ++j) t = fma(cf[j], sv[j], t);
        q[i] = t;
    }
}

// the lane and chunk of this block: the one lane (chunk = block), or the
// block's problem in the segmented grid; null if the block has no work here
template <bool SEG>
__device__ __forceinline__ const SegLane *cmp_lane(const SegLane *__restrict__ lanes, int nl, const SegLane &one,
                                                   int &k) {
    if (!SEG) {
        k = blockIdx.x;
        return &one;
    }
    const SegLane &L = lanes[lane_of_block(lanes, nl, blockIdx.x, false)];
    k = blockIdx.x - L.blk3;
    if (!L.dir || L.count < 1 || L.count > kCmpMax || k >= L.nb3) return nullptr;
    return &L;
}

// the pass for the lane's pair count (1 .. kCmpMax, uniform over a block)
#define SCVT_CMP_COUNTS(F) \
    switch (L->count) {    \
        case 1: F(1); break; \
        case 2: F(2); break; \
        case 3: F(3); break; \
        case 4: F(4); break; \
        case 5: F(5); break; \
        case 6: F(6); break; \
        case 7: F(7); break; \
        case 8: F(8); break; \
    }
static_assert(kCmpMax == 8, "SCVT_CMP_COUNTS lists the counts 1 .. kCmpMax");

template <bool SEG, bool DIRECT>
__global__ void __launch_bounds__(kCT, 7) k_cmp_a(const SegLane *__restrict__ lanes, int nl,
                                                  const __grid_constant__ SegLane one) {
    int k;
    const SegLane *L = cmp_lane<SEG>(lanes, nl, one, k);
    if (!L) return;
#define SCVT_A(C) cmp_pass_a<DIRECT, C>(*L, k)
    SCVT_CMP_COUNTS(SCVT_A)
#undef SCVT_A
}

template <bool SEG>
__global__ void __launch_bounds__(kCT, 7) k_cmp_b(const SegLane *__restrict__ lanes, int nl,
                                                  const __grid_constant__ SegLane one, double *__restrict__ q_rows) {
    int k;
    const SegLane *L = cmp_lane<SEG>(lanes, nl, one, k);
    if (!L) return;
    double *q = q_rows + 3 * L->row;
#define SCVT_B(C) cmp_pass_b<C>(*L, k, q)
    SCVT_CMP_COUNTS(SCVT_B)
#undef SCVT_B
}

template <bool SEG>
__global__ void __launch_bounds__(kCT, 7) k_cmp_c(const SegLane *__restrict__ lanes, int nl,
                                                  const __grid_constant__ SegLane one, double *__restrict__ q_rows) {
    int k;
    const SegLane *L = cmp_lane<SEG>(lanes, nl, one, k);
    if (!L) return;
    double *q = q_rows + 3 * L->row;
#define SCVT_C(C) cmp_pass_c<C>(*L, k, q)
    SCVT_CMP_COUNTS(SCVT_C)
#undef SCVT_C
}
#undef SCVT_CMP_COUNTS

__global__ void k_differs(int64_t len, const double *__restrict__ a, const double *__restrict__ b, unsigned *flag) {
    int any = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        any |= (__double_as_longlong(a[i]) != __double_as_longlong(b[i]));
    if (__syncthreads_or(any) && threadIdx.x == 0) atomicOr(flag, 1u);
}

}  // namespace

int reduce_blocks(int64_t n) {
    int64_t b = (n + 4095) / 4096;
    if (b < 1) b = 1;
    if (b > 1024) b = 1024;
    return (int)b;
}

void reduce_eval(int n, const double *fcell, const double *grad, const double *q, const double *nrm,
                 double *partials, DevStatus *st, cudaStream_t s, int64_t *launches) {
    int nb = reduce_blocks(n);
    k_reduce_eval<<<nb, kRT, 0, s>>>(n, fcell, grad, q, nrm, partials);
    k_finish<3><<<1, kRT, 0, s>>>(partials, nb, 4, st->red);
    (*launches) += 2;
}

void reduce_eval_batch(int nprob, int max_nb, const InstGeom *inst, const int *pbase, const int *active,
                       const double *fcell, const double *grad, const double *q, const double *nrm, double *partials,
                       DevStatus *ist, cudaStream_t s, int64_t *launches) {
    k_reduce_eval_batch<<<dim3(max_nb, nprob), kRT, 0, s>>>(inst, pbase, active, fcell, grad, q, nrm, partials);
    k_finish_batch<<<nprob, kRT, 0, s>>>(inst, pbase, active, partials, ist);
    (*launches) += 2;
}

void dot_to(int64_t len, const double *x, const double *y, double *partials, double *out, cudaStream_t s,
            int64_t *launches) {
    int nb = reduce_blocks(len);
    k_dot<<<nb, kRT, 0, s>>>(len, x, y, partials);
    k_finish_scalar<<<1, kRT, 0, s>>>(partials, nb, nullptr, nullptr, out);
    (*launches) += 2;
}

void trial_point(int n, const double *z, const double *q, double alpha, double *zt, double *nrm, cudaStream_t s,
                 int64_t *launches) {
    k_trial<<<(n + 255) / 256, 256, 0, s>>>(n, z, q, alpha, zt, nrm);
    (*launches)++;
}

void lloyd_project(int n, const double *c, double *zout, cudaStream_t s, int64_t *launches) {
    k_lloyd<<<(n + 255) / 256, 256, 0, s>>>(n, c, zout);
    (*launches)++;
}

void accept_pair(int n, const double *zt, const double *z, const double *gt, const double *g, double *S, double *Y,
                 double *partials, DevStatus *st, cudaStream_t s, int64_t *launches) {
    int nb = reduce_blocks(n);
    k_accept<<<nb, kRT, 0, s>>>(n, zt, z, gt, g, S, Y, partials, &st->maxmove_bits);
    k_finish<3><<<1, kRT, 0, s>>>(partials, nb, 4, st->dots);
    (*launches) += 2;
}

void vec_differs(int64_t len, const double *a, const double *b, DevStatus *st, cudaStream_t s, int64_t *launches) {
    cudaMemsetAsync(&st->differs, 0, sizeof(unsigned), s);
    k_differs<<<4 * 152, 256, 0, s>>>(len, a, b, &st->differs);
    (*launches)++;
}

void set_rho(double *rho_dev, int k, const DevStatus *st, cudaStream_t s, int64_t *launches) {
    k_set_rho<<<1, 1, 0, s>>>(rho_dev + k, st);
    (*launches)++;
}

void set_gamma(double *gamma_dev, const DevStatus *st, cudaStream_t s, int64_t *launches) {
    k_set_gamma<<<1, 1, 0, s>>>(gamma_dev, st);
    (*launches)++;
}

void seg_direction(const SegLane *lanes, int nl, bool any_gathered, int max_step_count, int nblk3, double *q_rows,
                   cudaStream_t s, int64_t *launches) {
    if (any_gathered) {
        SegLane none;
        memset(&none, 0, sizeof(none));
        k_cmp_a<true, false><<<nblk3, kCT, 0, s>>>(lanes, nl, none);
        k_cmp_b<true><<<nblk3, kCT, 0, s>>>(lanes, nl, none, q_rows);
        k_cmp_c<true><<<nblk3, kCT, 0, s>>>(lanes, nl, none, q_rows);
        (*launches) += 3;
    }
    for (int t = 0; t <= 2 * max_step_count; ++t) {
        k_seg_step<<<nblk3, kRT, 0, s>>>(lanes, nl, t, q_rows);
        (*launches)++;
    }
}

void lane_direction(const SegLane &L, double *q, cudaStream_t s, int64_t *launches) {
    const int c = L.count;
    if (c >= 1 && c <= kCmpMax) {
        cudaMemsetAsync(L.scal + kScalTicket, 0, sizeof(unsigned), s);
        k_cmp_a<false, false><<<L.nb3, kCT, 0, s>>>(nullptr, 1, L);
        k_cmp_b<false><<<L.nb3, kCT, 0, s>>>(nullptr, 1, L, q);
        k_cmp_c<false><<<L.nb3, kCT, 0, s>>>(nullptr, 1, L, q);
        (*launches) += 3;
        return;
    }
    const double *S[kLaneMaxM], *Y[kLaneMaxM], *R[kLaneMaxM];
    for (int k = 0; k < c; ++k) {
        S[k] = L.hist + (size_t)L.slots[k] * L.slot_stride;
        Y[k] = L.yhist + (size_t)L.slots[k] * L.slot_stride;
        R[k] = L.rho + L.slots[k];
    }
    two_loop(L.n, L.g, L.method == 1 ? nullptr : L.h, (L.method == 1 && c > 0) ? L.rho + kLaneMaxM + 1 : nullptr, c,
             S, Y, R, q, L.partials, L.scal, L.st, s, launches);
}

void lane_pair_products(const SegLane &L, cudaStream_t s, int64_t *launches) {
    // pass A over the first k pairs forms pair k-1's products with the older
    // ones as dot products (its scalars alpha are left unused)
    cudaMemsetAsync(L.scal + kScalTicket, 0, sizeof(unsigned), s);
    for (int k = 2; k <= L.count; ++k) {
        SegLane P = L;
        P.count = k;
        k_cmp_a<false, true><<<P.nb3, kCT, 0, s>>>(nullptr, 1, P);
        (*launches)++;
    }
}

void seg_trial(const SegLane *lanes, const int *pinst, int64_t ntot, const double *q_rows, double *zt_rows,
               double *nrm_rows, cudaStream_t s, int64_t *launches) {
    k_seg_trial<<<(unsigned)((ntot + 255) / 256), 256, 0, s>>>(lanes, pinst, ntot, q_rows, zt_rows, nrm_rows);
    (*launches)++;
}

void seg_accept(const SegLane *lanes, int nl, int nblk1, const double *zt_rows, const double *gt_rows,
                const double *ht_rows, cudaStream_t s, int64_t *launches) {
    k_seg_accept<<<nblk1, kRT, 0, s>>>(lanes, nl, zt_rows, gt_rows, ht_rows);
    (*launches)++;
}

void two_loop(int n, const double *g, const double *h, const double *hs, int count, const double *const *S,
              const double *const *Y, const double *const *rho, double *q, double *partials, double *scal,
              DevStatus *st, cudaStream_t s, int64_t *launches) {
    // one pass per step of the recursion (Sec. 2.2.2): q = -g, then per pair
    // (newest first) q -= alpha_k y_k, the initial matrix (diag(h) per
    // generator, hs[0] I or I) with the last backward step, then per pair
    // (oldest first) q += (alpha_k - beta_k) s_k; each pass's last block turns
    // the chunk sums of its dot product into the next step's scalar, so the
    // 2 count + 1 passes run back to back without a host round trip
    const int64_t len = 3 * (int64_t)n;
    const int nb = reduce_blocks(len);
    double *alpha = scal + kScalAlpha, *coef = scal + kScalCoef;
    unsigned *ticket = reinterpret_cast<unsigned *>(scal + kScalTicket);
    cudaMemsetAsync(ticket, 0, sizeof(unsigned), s);
    if (count == 0) {
        k_step<<<nb, kRT, 0, s>>>(len, q, nullptr, 0.0, g, h, hs, g, partials, ticket, nullptr, nullptr,
                                  &st->dots[3]);
        (*launches)++;
        return;
    }
    // backward: newest (count-1) .. oldest (0); the first pass gives alpha_{count-1}
    k_step<<<nb, kRT, 0, s>>>(len, q, nullptr, 0.0, g, nullptr, nullptr, S[count - 1], partials, ticket,
                              rho[count - 1], nullptr, alpha + count - 1);
    (*launches)++;
    for (int k = count - 1; k >= 0; --k) {
        if (k > 0) {
            // q -= alpha_k y_k; alpha_{k-1} = rho_{k-1} s_{k-1}.q
            k_step<<<nb, kRT, 0, s>>>(len, q, alpha + k, -1.0, Y[k], nullptr, nullptr, S[k - 1], partials, ticket,
                                      rho[k - 1], nullptr, alpha + k - 1);
        } else {
            // q = H0 (q - alpha_0 y_0); coef_0 = alpha_0 - rho_0 y_0.q
            k_step<<<nb, kRT, 0, s>>>(len, q, alpha, -1.0, Y[0], h, hs, Y[0], partials, ticket, rho[0], alpha,
                                      coef);
        }
        (*launches)++;
    }
    // forward: oldest .. newest; q += coef_k s_k, coef_{k+1} = alpha_{k+1} - rho_{k+1} y_{k+1}.q, the
    // last pass leaves g.q
    for (int k = 0; k < count; ++k) {
        if (k + 1 < count)
            k_step<<<nb, kRT, 0, s>>>(len, q, coef + k, 1.0, S[k], nullptr, nullptr, Y[k + 1], partials, ticket,
                                      rho[k + 1], alpha + k + 1, coef + k + 1);
        else
            k_step<<<nb, kRT, 0, s>>>(len, q, coef + k, 1.0, S[k], nullptr, nullptr, g, partials, ticket, nullptr,
                                      nullptr, &st->dots[3]);
        (*launches)++;
    }
}

}  // namespace scvt
