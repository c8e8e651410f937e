// capi.cu -- the C ABI (include/scvt.h): handle, workspace, evaluation
// driver and the Lloyd-preconditioned LBFGS driver.
//
// The host side of the solver moves scalars only: per evaluation one
// device-to-host copy of a small status block (energy, |g|^2, phi'(alpha),
// flags); per iteration one more for the curvature pair's dot products.
// Vectors (Z, g, h, q, the history ring) stay in HBM.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "scvt_internal.cuh"
#include "autotune.h"
#include "wolfe.h"

using namespace scvt;

namespace {

constexpr int kMaxM = kLaneMaxM;  // history pairs
constexpr int kDefaultK0 = 32;

struct Bufs {
    double *z = nullptr, *zt = nullptr;      // current iterate, trial point
    double *g = nullptr, *gt = nullptr;      // gradients
    double *h = nullptr, *ht = nullptr;      // preconditioner
    double *fc = nullptr;                    // per-cell energy (scratch)
    double *q = nullptr;                     // direction
    double *yv = nullptr;                    // y of the newest candidate pair (scratch)
    double *nrm = nullptr;                   // 1 / |z + alpha q|
    double *mass = nullptr, *moment = nullptr;
    double *stage_a = nullptr, *stage_b = nullptr;  // host-pointer staging (3n each)
    double *partials = nullptr;              // kCmpQ * 1024 chunk sums
    double *scal = nullptr;                  // two-loop scalars (kTwoLoopScratch)
    double *rho = nullptr;                   // kLaneRho: 1/(y.s) per slot, gamma, the products s_a.y_b
    double *hist = nullptr;                  // (m + 1) slots of S and Y, 3n each
    P4 *zs = nullptr;
    float4 *zf = nullptr, *zl = nullptr, *zll = nullptr;
    P4 *cvx = nullptr;
    int *cdeg = nullptr, *cnb = nullptr, *eoff = nullptr, *ecell = nullptr, *escan = nullptr;
    double *eacc = nullptr;
    void *tab = nullptr;                     // density table (FP64 forms, tanh-cap densities)
    float4 *vo = nullptr, *ctab = nullptr;
    int *bin_of = nullptr, *count = nullptr, *start = nullptr, *cursor = nullptr, *scan_tmp = nullptr;
    int *sidx = nullptr, *list1 = nullptr, *list2 = nullptr;
    int *deg = nullptr;
    float *radius = nullptr;
    DevStatus *st = nullptr;
};

}  // namespace

struct scvt_handle {
    scvt_config cfg;
    int n = 0;
    int G = 1;      // bins per face edge of the next evaluation (adapted to the generators' spread)
    int Gmax = 1;   // largest the workspace holds
    int m = 0;
    Tune tune;
    Pipes pipes;
    cudaStream_t stream = nullptr;
    Bufs b;
    DensTab tab{};                 // the density table in b.tab (M = 0: none)
    DevStatus *st_host = nullptr;  // pinned
    int64_t bytes = 0;
    // history ring: slot order (oldest first) and one spare slot
    int hist_slots[kMaxM + 1];
    int hist_count = 0;
    bool new_pair = false;  // a pair was stored after the last direction
    int spare = 0;
    bool state_valid = false;  // z, g, h, F describe the current iterate
    double F = 0.0, gnorm = 0.0;
    bool radius_valid = false;
    // stats
    scvt_stats stats;
    bool profiling = false;
    cudaEvent_t ev_topo[2] = {nullptr, nullptr};
    cudaEvent_t ev_cell0 = nullptr, ev_cell1 = nullptr, ev_e0 = nullptr, ev_e1 = nullptr, ev_l0 = nullptr,
                ev_l1 = nullptr;
    std::string err;
};

namespace {

scvt_status fail(scvt_handle *h, scvt_status s, const std::string &msg) {
    if (h) h->err = msg;
    return s;
}

scvt_status cuda_fail(scvt_handle *h, cudaError_t e, const char *what) {
    cudaGetLastError();
    return fail(h, e == cudaErrorMemoryAllocation ? SCVT_ERR_OOM : SCVT_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(H, e_, what); \
    } while (0)

template <class T>
cudaError_t alloc(scvt_handle *H, T **p, size_t count) {
    size_t bytes = sizeof(T) * (count ? count : 1);
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e == cudaSuccess) H->bytes += (int64_t)bytes;
    return e;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

double *slot_S(scvt_handle *H, int slot) { return H->b.hist + (size_t)slot * 2 * 3 * H->n; }
double *slot_Y(scvt_handle *H, int slot) { return slot_S(H, slot) + (size_t)3 * H->n; }

void profile_accumulate(scvt_handle *H) {
    if (!H->profiling) return;
    float ms = 0.0f;
    // the cell kernels are timed only when the cells run as one pipeline
    const bool one = H->tune.chunks <= 1 || H->pipes.n_aux == 0;
    if (one && cudaEventElapsedTime(&ms, H->ev_cell0, H->ev_cell1) == cudaSuccess) {
        H->stats.cell_kernel_ms += ms;
        H->stats.cell_kernel_timed++;
    }
    if (one && cudaEventElapsedTime(&ms, H->ev_topo[0], H->ev_topo[1]) == cudaSuccess) {
        H->stats.topo_kernel_ms += ms;
        H->stats.topo_kernel_timed++;
    }
    if (cudaEventElapsedTime(&ms, H->ev_e0, H->ev_e1) == cudaSuccess) H->stats.eval_ms += ms;
    cudaGetLastError();
}

// One energy/gradient evaluation at zdev (device).  Outputs go to the given
// device arrays (grad, hdiag and fcell are required).  If q is given, phi'
// (Sec. 3.1 line search on the projected path) is accumulated with nrm.
scvt_status evaluate_dev(scvt_handle *H, const double *zdev, double *grad, double *hdiag, double *fcell,
                         double *mass, double *moment, int *deg, int *nbr, int max_deg, const double *q,
                         const double *nrm, double *F, double *gn2, double *dphi) {
    const int n = H->n;
    Bufs &B = H->b;
    cudaStream_t s = H->stream;
    int64_t *L = &H->stats.kernel_launches;
    Phase ph("scvt evaluate");
    if (H->profiling) cudaEventRecord(H->ev_e0, s);
    CK(cudaMemsetAsync(B.st, 0, sizeof(DevStatus), s), "reset status");
    Grid g;
    memset(&g, 0, sizeof(g));
    g.n = n;
    g.G = H->G;
    g.nbins = 6 * H->G * H->G;
    g.zs = B.zs;
    g.zf = B.zf;
    g.zl = B.zl;
    g.zll = H->cfg.precision != 1 ? B.zll : nullptr;  // not computed in the mixed form
    g.sidx = B.sidx;
    g.bstart = B.start;
    g.rho0 = to_device_density(H->cfg.rho);
    g.rho0f = to_density32(g.rho0);
    g.tab0 = H->tab;
    g.fan = H->cfg.decomposition;
    if (!H->radius_valid) {
        CK(cudaMemsetAsync(B.radius, 0, sizeof(float) * n, s), "reset radius hints");
        H->radius_valid = true;
    }
    {
        Phase pb("scvt bin");
        bin_points(zdev, g, B.bin_of, B.count, B.start, B.cursor, B.scan_tmp, B.zs, B.zf, B.zl,
                   H->cfg.precision != 1 ? B.zll : nullptr, B.sidx, B.radius, B.st, s, L);
    }
    CellOut out;
    out.grad = grad;
    out.hdiag = hdiag;
    out.mass = mass;
    out.moment = moment;
    out.fcell = fcell;
    out.deg = deg;
    out.nbr = nbr;
    out.max_deg = max_deg;
    out.radius = B.radius;
    CellBuf cb;
    cb.deg = B.cdeg;
    cb.vx = B.cvx;
    cb.nb = B.cnb;
    cb.eoff = B.eoff;
    cb.ecell = B.ecell;
    cb.scan_tmp = B.escan;
    cb.eacc = B.eacc;
    cb.vo = B.vo;
    cb.ctab = B.ctab;
    cell_passes(g, out, cb, B.list1, B.list2, B.st, H->cfg.precision, H->tune, s,
                H->profiling ? H->ev_cell0 : nullptr, H->profiling ? H->ev_cell1 : nullptr, L,
                &H->stats.cell_launches, &H->pipes, H->profiling ? H->ev_topo : nullptr);
    {
        Phase pr("scvt reduce");
        reduce_eval(n, fcell, grad, q, nrm, B.partials, B.st, s, L);
    }
    if (H->profiling) cudaEventRecord(H->ev_e1, s);
    CK(cudaGetLastError(), "launch");
    CK(cudaMemcpyAsync(H->st_host, B.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s), "status copy");
    CK(cudaStreamSynchronize(s), "evaluation");
    profile_accumulate(H);
    const DevStatus &st = *H->st_host;
    H->stats.evaluations++;
    H->stats.knn_retries += st.retry_count[0];
    H->stats.ambiguous += (int64_t)st.ambiguous;
    H->stats.series_edges += (int64_t)st.ser_edges;
    H->G = adapt_bins(bins_per_edge(n, H->tune.bin_load), H->G, H->Gmax, st.max_bin, H->tune.bin_load);
    H->stats.series_terms += (int64_t)st.ser_terms;
    if (st.flags & FLAG_BAD_POINT)
        return fail(H, SCVT_ERR_INVALID, "a generator is not finite or not on the unit sphere (| |z|^2 - 1 | > 2e-12)");
    if (st.flags & FLAG_DUPLICATE) return fail(H, SCVT_ERR_INVALID, "duplicate generators");
    if (st.flags & (FLAG_UNBOUNDED | FLAG_EMPTY))
        return fail(H, SCVT_ERR_DEGENERATE, "origin not strictly inside the convex hull of the generators");
    if (st.flags & FLAG_EXHAUSTED)
        return fail(H, SCVT_ERR_KNN_EXHAUSTED, "a Voronoi cell could not be certified by the security radius");
    if (st.flags & FLAG_VMAX) return fail(H, SCVT_ERR_KNN_EXHAUSTED, "a Voronoi cell has more than 64 vertices");
    if (st.flags & FLAG_NONPOSITIVE) return fail(H, SCVT_ERR_DEGENERATE, "a cell has c_i . z_i <= 0");
    if (st.flags & FLAG_ECAP)
        return fail(H, SCVT_ERR_DEGENERATE, "neighbouring cells disagree on a Voronoi vertex (cocircular generators)");
    if (F) *F = st.red[0];
    if (gn2) *gn2 = st.red[1];
    if (dphi) *dphi = st.red[2];
    H->err.clear();
    return SCVT_OK;
}

// Resolve an input array of 3n (or n) doubles: device pointers are used
// as they are, host pointers are copied into the given staging buffer.
scvt_status stage_in(scvt_handle *H, const double *p, size_t count, double *stage, const double **dev) {
    if (is_device_ptr(p)) {
        *dev = p;
        return SCVT_OK;
    }
    CK(cudaMemcpyAsync(stage, p, sizeof(double) * count, cudaMemcpyHostToDevice, H->stream), "host to device");
    *dev = stage;
    return SCVT_OK;
}

scvt_status copy_out(scvt_handle *H, double *dst, const double *src, size_t count) {
    if (!dst) return SCVT_OK;
    cudaMemcpyKind k = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (dst != src) CK(cudaMemcpyAsync(dst, src, sizeof(double) * count, k, H->stream), "copy out");
    return SCVT_OK;
}

// history bookkeeping
void hist_reset(scvt_handle *H) {
    H->hist_count = 0;
    H->new_pair = false;
    for (int k = 0; k <= H->m; ++k) H->hist_slots[k] = k;
    H->spare = H->m;  // slot m is the first spare
}

// method 0: H0 = diag(h); 1: gamma I (I with an empty memory); 2: Lloyd, diag(h) and no memory
// the handle's LBFGS state as the direction kernels see one problem
SegLane single_lane(scvt_handle *H, int count, int method) {
    SegLane L;
    memset(&L, 0, sizeof(L));
    L.n = H->n;
    L.count = count;
    L.method = method;
    L.m = H->m;
    L.dir = 1;
    L.nb3 = reduce_blocks(3 * (int64_t)H->n);
    L.nb1 = reduce_blocks(H->n);
    for (int k = 0; k < count; ++k) L.slots[k] = H->hist_slots[k];
    L.z = H->b.z;
    L.g = H->b.g;
    L.h = H->b.h;
    L.hist = slot_S(H, 0);
    L.yhist = slot_Y(H, 0);
    L.slot_stride = 2 * 3 * (int64_t)H->n;
    L.rho = H->b.rho;
    L.scal = H->b.scal;
    L.partials = H->b.partials;
    L.st = H->b.st;
    return L;
}

scvt_status make_direction(scvt_handle *H, double *d0, int method) {
    const int count = (method == 2) ? 0 : H->hist_count;
    Phase ph("scvt direction");
    if (H->profiling) cudaEventRecord(H->ev_l0, H->stream);
    SegLane L = single_lane(H, count, method);
    L.new_pair = H->new_pair ? 1 : 0;
    H->new_pair = false;
    lane_direction(L, H->b.q, H->stream, &H->stats.kernel_launches);
    if (H->profiling) cudaEventRecord(H->ev_l1, H->stream);
    CK(cudaGetLastError(), "two-loop launch");
    CK(cudaMemcpyAsync(&H->st_host->dots[3], &H->b.st->dots[3], sizeof(double), cudaMemcpyDeviceToHost, H->stream),
       "direction copy");
    CK(cudaStreamSynchronize(H->stream), "two-loop");
    if (H->profiling) {
        float ms;
        if (cudaEventElapsedTime(&ms, H->ev_l0, H->ev_l1) == cudaSuccess) H->stats.lbfgs_ms += ms;
        cudaGetLastError();
    }
    *d0 = H->st_host->dots[3];
    return SCVT_OK;
}

}  // namespace

namespace {

// topology of z into deg (n) and nbr (n x 32) allocated on the stream; every
// cell must have at most 32 neighbours
scvt_status topology32(scvt_handle *H, const double *zd, int **deg, int **nbr) {
    const size_t n = H->n;
    *deg = nullptr;
    *nbr = nullptr;
    CK(cudaMallocAsync((void **)deg, sizeof(int) * n, H->stream), "degree buffer");
    CK(cudaMallocAsync((void **)nbr, sizeof(int) * n * 32, H->stream), "neighbour buffer");
    double F, g2;
    scvt_status s = evaluate_dev(H, zd, H->b.gt, H->b.ht, H->b.fc, nullptr, nullptr, *deg, *nbr, 32, nullptr,
                                 nullptr, &F, &g2, nullptr);
    if (s) return s;
    std::vector<int> hd(n);
    CK(cudaMemcpy(hd.data(), *deg, sizeof(int) * n, cudaMemcpyDeviceToHost), "degree check");
    for (size_t i = 0; i < n; ++i)
        if (hd[i] > 32) return fail(H, SCVT_ERR_INVALID, "a cell has more than 32 neighbours");
    return SCVT_OK;
}

}  // namespace

// ======================================================================
extern "C" {

const char *scvt_status_string(scvt_status s) {
    switch (s) {
    case SCVT_OK: return "ok";
    case SCVT_ERR_INVALID: return "invalid argument";
    case SCVT_ERR_DEGENERATE: return "degenerate input";
    case SCVT_ERR_OOM: return "out of device memory";
    case SCVT_ERR_CUDA: return "CUDA error";
    case SCVT_ERR_KNN_EXHAUSTED: return "neighbour search exhausted";
    case SCVT_ERR_LINESEARCH: return "line search failed";
    case SCVT_ERR_TIMEOUT: return "device wait timed out";
    case SCVT_ERR_UNIMPLEMENTED: return "not implemented";
    }
    return "unknown status";
}

const char *scvt_last_error(const scvt_handle *h) { return h ? h->err.c_str() : ""; }

const char *scvt_version(void) { return "scvt-gb300 0.3 (sm_103a; FP64 form (double-float rule points), mixed FP32/FP64 form, plain FP64 form)"; }

void scvt_destroy(scvt_handle *H) {
    if (!H) return;
    Bufs &b = H->b;
    void *ptrs[] = {b.z, b.zt, b.g, b.gt, b.h, b.ht, b.fc, b.q, b.yv, b.nrm, b.mass, b.moment, b.stage_a, b.stage_b,
                    b.partials, b.scal, b.rho, b.hist, b.zs, b.zf, b.zl, b.zll, b.cvx, b.cnb, b.cdeg, b.eoff, b.ecell, b.escan, b.eacc, b.vo, b.ctab, b.tab, b.bin_of, b.count, b.start, b.cursor, b.scan_tmp,
                    b.sidx, b.list1, b.list2, b.deg, b.radius, b.st};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (H->st_host) cudaFreeHost(H->st_host);
    pipes_destroy(H->pipes);
    cudaEvent_t evs[] = {H->ev_cell0, H->ev_cell1, H->ev_e0, H->ev_e1, H->ev_l0, H->ev_l1, H->ev_topo[0], H->ev_topo[1]};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    delete H;
}

scvt_status scvt_create(const scvt_config *cfg, void *cuda_stream, scvt_handle **out) {
    if (!cfg || !out) return SCVT_ERR_INVALID;
    *out = nullptr;
    if (cfg->n < 4 || cfg->n > (int64_t)200000000) return SCVT_ERR_INVALID;
    if (cfg->lbfgs_m < 0 || cfg->lbfgs_m > kMaxM) return SCVT_ERR_INVALID;
    if (cfg->quad_points != 0 && cfg->quad_points != 7) return SCVT_ERR_INVALID;
    if (cfg->precision < 0 || cfg->precision > 2) return SCVT_ERR_INVALID;
    if (cfg->decomposition != 0 && cfg->decomposition != 1) return SCVT_ERR_INVALID;
    if (cfg->rho.kind < 0 || cfg->rho.kind > 3) return SCVT_ERR_INVALID;
    if (cfg->rho.kind != SCVT_RHO_UNIFORM) {
        if (!(cfg->rho.gamma > 0.0) || !(cfg->rho.gamma <= 1.0)) return SCVT_ERR_INVALID;
        if (cfg->rho.kind >= 2) {
            double r = sqrt(cfg->rho.xc[0] * cfg->rho.xc[0] + cfg->rho.xc[1] * cfg->rho.xc[1] +
                            cfg->rho.xc[2] * cfg->rho.xc[2]);
            if (!(fabs(r - 1.0) < 1e-9) || !(cfg->rho.alpha > 0.0)) return SCVT_ERR_INVALID;
        }
    }
    if (cfg->knn_k0 != 0 && (cfg->knn_k0 < 8 || cfg->knn_k0 > 32)) return SCVT_ERR_INVALID;
    scvt_handle *H = new (std::nothrow) scvt_handle();
    if (!H) return SCVT_ERR_OOM;
    H->cfg = *cfg;
    if (H->cfg.knn_k0 == 0) H->cfg.knn_k0 = kDefaultK0;
    if (H->cfg.knn_kmax == 0) H->cfg.knn_kmax = 128;
    H->n = (int)cfg->n;
    H->m = cfg->lbfgs_m;
    H->stream = (cudaStream_t)cuda_stream;
    memset(&H->stats, 0, sizeof(H->stats));
    // ~2 generators per bin on average; bins are allocated for the finest tuning (1 per bin)
    H->G = bins_per_edge(H->n, H->tune.bin_load);
    const int n = H->n;
    const size_t n3 = 3 * (size_t)n;
    H->Gmax = max_bins_per_edge(H->n);
    const int nbins = 6 * H->Gmax * H->Gmax;
    Bufs &b = H->b;
    cudaError_t e = cudaSuccess;
#define AL(ptr, cnt) \
    if (e == cudaSuccess) e = alloc(H, &(ptr), (cnt))
    AL(b.z, n3); AL(b.zt, n3); AL(b.g, n3); AL(b.gt, n3); AL(b.h, n); AL(b.ht, n); AL(b.fc, n);
    AL(b.q, n3); AL(b.yv, n3); AL(b.nrm, n); AL(b.mass, n); AL(b.moment, n3);
    AL(b.stage_a, n3); AL(b.stage_b, n3);
    AL(b.partials, kCmpQ * 1024); AL(b.scal, kTwoLoopScratch); AL(b.rho, kLaneRho);
    AL(b.hist, (size_t)(H->m + 1) * 2 * n3);
    AL(b.zs, n); AL(b.zf, n); AL(b.zl, n); AL(b.zll, n); AL(b.cvx, (size_t)n * kCellSlots); AL(b.cnb, (size_t)n * kCellSlots);
    AL(b.cdeg, n); AL(b.eoff, n + 1); AL(b.ecell, 6 * (size_t)n); AL(b.escan, scan_tmp_ints(n));
    AL(b.eacc, 5 * 6 * (size_t)n);
    if (cfg->precision == 1) AL(b.vo, (size_t)n * kCellSlots);
    if (cfg->precision == 0) AL(b.ctab, n);
    const Density dens = to_device_density(cfg->rho);
    const int tabM = (cfg->precision != 1 && dens.kind >= 2) ? dens_table_centres(n) : 0;
    if (tabM > 0 && e == cudaSuccess) {
        e = cudaMalloc(&b.tab, dens_table_bytes(tabM));
        if (e == cudaSuccess) H->bytes += (int64_t)dens_table_bytes(tabM);
    }
    AL(b.bin_of, n); AL(b.count, nbins); AL(b.start, nbins + 1); AL(b.cursor, nbins);
    AL(b.scan_tmp, 2 * (nbins / 2048 + 64) + 64);
    AL(b.sidx, n); AL(b.list1, n); AL(b.list2, n); AL(b.deg, n); AL(b.radius, n);
    AL(b.st, 1);
#undef AL
    if (e == cudaSuccess && tabM > 0) e = dens_table_build(dens, tabM, b.tab, &H->tab, H->stream);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&H->st_host, sizeof(DevStatus));
    if (e == cudaSuccess) e = pipes_create(H->pipes, kMaxChunks - 1);
    cudaEvent_t *evs[] = {&H->ev_cell0, &H->ev_cell1, &H->ev_e0, &H->ev_e1, &H->ev_l0, &H->ev_l1, &H->ev_topo[0],
                          &H->ev_topo[1]};
    for (cudaEvent_t *ev : evs)
        if (e == cudaSuccess) e = cudaEventCreate(ev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        scvt_destroy(H);
        return e == cudaErrorMemoryAllocation ? SCVT_ERR_OOM : SCVT_ERR_CUDA;
    }
    H->stats.bytes_device = H->bytes;
    hist_reset(H);
    *out = H;
    return SCVT_OK;
}

scvt_status scvt_evaluate(scvt_handle *H, const double *z, scvt_eval_out *o) {
    if (!H) return SCVT_ERR_INVALID;
    if (!z || !o) return fail(H, SCVT_ERR_INVALID, "null argument");
    const size_t n = H->n, n3 = 3 * n;
    const double *zd;
    scvt_status s = stage_in(H, z, n3, H->b.stage_a, &zd);
    if (s) return s;
    // kernels write into device memory; host outputs are copied afterwards
    double *grad = (o->grad && is_device_ptr(o->grad)) ? o->grad : H->b.gt;
    double *hd = (o->precond && is_device_ptr(o->precond)) ? o->precond : H->b.ht;
    double *mass = o->mass ? ((is_device_ptr(o->mass)) ? o->mass : H->b.mass) : nullptr;
    double *mom = o->moment ? ((is_device_ptr(o->moment)) ? o->moment : H->b.moment) : nullptr;
    double *fc = (o->cell_energy && is_device_ptr(o->cell_energy)) ? o->cell_energy : H->b.fc;
    double F, g2;
    s = evaluate_dev(H, zd, grad, hd, fc, mass, mom, nullptr, nullptr, 0, nullptr, nullptr, &F, &g2, nullptr);
    if (s) return s;
    if ((s = copy_out(H, o->grad, grad, n3))) return s;
    if ((s = copy_out(H, o->precond, hd, n))) return s;
    if ((s = copy_out(H, o->mass, mass, n))) return s;
    if ((s = copy_out(H, o->moment, mom, n3))) return s;
    if ((s = copy_out(H, o->cell_energy, fc, n))) return s;
    CK(cudaStreamSynchronize(H->stream), "copy out");
    o->energy = F;
    o->grad_norm = sqrt(g2);
    return SCVT_OK;
}

scvt_status scvt_energy_grad(scvt_handle *H, const double *z, double *energy, double *grad, double *mass,
                             double *moment) {
    if (!H) return SCVT_ERR_INVALID;
    if (!energy) return fail(H, SCVT_ERR_INVALID, "energy pointer is null");
    scvt_eval_out o;
    memset(&o, 0, sizeof(o));
    o.grad = grad;
    o.mass = mass;
    o.moment = moment;
    scvt_status s = scvt_evaluate(H, z, &o);
    if (s == SCVT_OK) *energy = o.energy;
    return s;
}

scvt_status scvt_lloyd_step(scvt_handle *H, const double *z_in, double *z_out) {
    if (!H) return SCVT_ERR_INVALID;
    if (!z_in || !z_out) return fail(H, SCVT_ERR_INVALID, "null argument");
    const size_t n3 = 3 * (size_t)H->n;
    const double *zd;
    scvt_status s = stage_in(H, z_in, n3, H->b.stage_a, &zd);
    if (s) return s;
    double F, g2;
    s = evaluate_dev(H, zd, H->b.gt, H->b.ht, H->b.fc, nullptr, H->b.moment, nullptr, nullptr, 0, nullptr, nullptr,
                     &F, &g2, nullptr);
    if (s) return s;
    bool dev_out = is_device_ptr(z_out);
    double *dst = dev_out ? z_out : H->b.stage_b;
    lloyd_project(H->n, H->b.moment, dst, H->stream, &H->stats.kernel_launches);
    CK(cudaGetLastError(), "lloyd launch");
    if (!dev_out) CK(cudaMemcpyAsync(z_out, dst, sizeof(double) * n3, cudaMemcpyDeviceToHost, H->stream), "copy out");
    CK(cudaStreamSynchronize(H->stream), "lloyd step");
    return SCVT_OK;
}

scvt_status scvt_voronoi(scvt_handle *H, const double *z, int *deg, int *nbr, int max_deg) {
    if (!H) return SCVT_ERR_INVALID;
    if (!z || !deg || !nbr || max_deg < 3) return fail(H, SCVT_ERR_INVALID, "bad argument");
    const size_t n = H->n;
    const double *zd;
    scvt_status s = stage_in(H, z, 3 * n, H->b.stage_a, &zd);
    if (s) return s;
    bool dev_deg = is_device_ptr(deg), dev_nbr = is_device_ptr(nbr);
    int *ddeg = dev_deg ? deg : H->b.deg;
    int *dnbr = nbr;
    int *tmp = nullptr;
    if (!dev_nbr) {
        CK(cudaMallocAsync((void **)&tmp, sizeof(int) * n * max_deg, H->stream), "topology buffer");
        dnbr = tmp;
    }
    double F, g2;
    s = evaluate_dev(H, zd, H->b.gt, H->b.ht, H->b.fc, nullptr, nullptr, ddeg, dnbr, max_deg, nullptr, nullptr, &F,
                     &g2, nullptr);
    if (s == SCVT_OK) {
        if (!dev_deg) cudaMemcpyAsync(deg, ddeg, sizeof(int) * n, cudaMemcpyDeviceToHost, H->stream);
        if (!dev_nbr) cudaMemcpyAsync(nbr, dnbr, sizeof(int) * n * max_deg, cudaMemcpyDeviceToHost, H->stream);
    }
    if (tmp) cudaFreeAsync(tmp, H->stream);
    CK(cudaStreamSynchronize(H->stream), "topology copy");
    if (s) return s;
    // degree check on the host copy
    std::vector<int> hd;
    const int *dp = deg;
    if (dev_deg) {
        hd.resize(n);
        CK(cudaMemcpy(hd.data(), deg, sizeof(int) * n, cudaMemcpyDeviceToHost), "degree check");
        dp = hd.data();
    }
    for (size_t i = 0; i < n; ++i)
        if (dp[i] > max_deg) return fail(H, SCVT_ERR_INVALID, "a cell has more neighbours than max_deg");
    return SCVT_OK;
}

scvt_status scvt_bisect(scvt_handle *H, const double *z, double *z_out, int64_t cap, int64_t *n_out) {
    if (!H) return SCVT_ERR_INVALID;
    if (!z || !z_out || !n_out || cap < 0) return fail(H, SCVT_ERR_INVALID, "bad argument");
    const int n = H->n;
    const double *zd;
    scvt_status s = stage_in(H, z, 3 * (size_t)n, H->b.stage_a, &zd);
    if (s) return s;
    int *deg = nullptr, *nbr = nullptr;
    double *tmp = nullptr;
    s = topology32(H, zd, &deg, &nbr);
    const bool dev_out = is_device_ptr(z_out);
    if (s == SCVT_OK && !dev_out && cap > 0) {
        cudaError_t e = cudaMallocAsync((void **)&tmp, sizeof(double) * 3 * (size_t)cap, H->stream);
        if (e != cudaSuccess) s = cuda_fail(H, e, "output buffer");
    }
    if (s == SCVT_OK) {
        cudaError_t e = bisect_midpoints(n, zd, deg, nbr, 32, H->b.list1, H->b.list2, H->b.escan,
                                         dev_out ? z_out : tmp, cap, n_out, H->stream);
        if (e != cudaSuccess) s = cuda_fail(H, e, "bisection");
        else if (*n_out > cap) s = fail(H, SCVT_ERR_INVALID, "z_out holds fewer points than the refinement");
        else if (!dev_out && *n_out > 0) {
            e = cudaMemcpyAsync(z_out, tmp, sizeof(double) * 3 * (size_t)*n_out, cudaMemcpyDeviceToHost, H->stream);
            if (e != cudaSuccess) s = cuda_fail(H, e, "copy out");
        }
    }
    void *bufs[] = {deg, nbr, tmp};
    for (void *p : bufs)
        if (p) cudaFreeAsync(p, H->stream);
    cudaError_t e = cudaStreamSynchronize(H->stream);
    if (s == SCVT_OK && e != cudaSuccess) s = cuda_fail(H, e, "bisection");
    return s;
}

scvt_status scvt_mesh_quality(scvt_handle *H, const double *z, double *cellq, double *triq,
                                         int64_t tri_cap, int64_t *n_tri) {
    if (!H) return SCVT_ERR_INVALID;
    if (!z || !n_tri || (triq && tri_cap < 0)) return fail(H, SCVT_ERR_INVALID, "bad argument");
    const int n = H->n;
    const double *zd;
    scvt_status s = stage_in(H, z, 3 * (size_t)n, H->b.stage_a, &zd);
    if (s) return s;
    int *deg = nullptr, *nbr = nullptr;
    double *tc = nullptr, *tt = nullptr;
    s = topology32(H, zd, &deg, &nbr);
    const bool dev_c = cellq && is_device_ptr(cellq), dev_t = triq && is_device_ptr(triq);
    cudaError_t e = cudaSuccess;
    if (s == SCVT_OK && cellq && !dev_c) e = cudaMallocAsync((void **)&tc, sizeof(double) * (size_t)n, H->stream);
    if (s == SCVT_OK && e == cudaSuccess && triq && !dev_t && tri_cap > 0)
        e = cudaMallocAsync((void **)&tt, sizeof(double) * (size_t)tri_cap, H->stream);
    if (e != cudaSuccess) s = cuda_fail(H, e, "output buffers");
    if (s == SCVT_OK) {
        e = mesh_quality(n, zd, deg, nbr, 32, H->b.list1, H->b.list2, H->b.escan, cellq ? (dev_c ? cellq : tc) : nullptr,
                         triq ? (dev_t ? triq : tt) : nullptr, tri_cap, n_tri, H->stream);
        if (e != cudaSuccess) s = cuda_fail(H, e, "mesh quality");
        else if (triq && *n_tri > tri_cap) s = fail(H, SCVT_ERR_INVALID, "triq holds fewer values than triangles");
        else {
            if (tc) e = cudaMemcpyAsync(cellq, tc, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, H->stream);
            if (e == cudaSuccess && tt && *n_tri > 0)
                e = cudaMemcpyAsync(triq, tt, sizeof(double) * (size_t)*n_tri, cudaMemcpyDeviceToHost, H->stream);
            if (e != cudaSuccess) s = cuda_fail(H, e, "copy out");
        }
    }
    void *bufs[] = {deg, nbr, tc, tt};
    for (void *p : bufs)
        if (p) cudaFreeAsync(p, H->stream);
    e = cudaStreamSynchronize(H->stream);
    if (s == SCVT_OK && e != cudaSuccess) s = cuda_fail(H, e, "mesh quality");
    return s;
}

scvt_status scvt_lbfgs_direction(scvt_handle *H, const double *g, const double *hdiag, int count,
                                            const double *S,
                                 const double *Y, double *q) {
    if (!H) return SCVT_ERR_INVALID;
    if (!g || !hdiag || !q || count < 0 || count > 64 || (count > 0 && (!S || !Y)))
        return fail(H, SCVT_ERR_INVALID, "bad argument");
    for (const void *p : {(const void *)g, (const void *)hdiag, (const void *)q})
        if (!is_device_ptr(p)) return fail(H, SCVT_ERR_INVALID, "scvt_lbfgs_direction takes device pointers");
    if (count > 0 && (!is_device_ptr(S) || !is_device_ptr(Y)))
        return fail(H, SCVT_ERR_INVALID, "scvt_lbfgs_direction takes device pointers");
    const size_t n3 = 3 * (size_t)H->n;
    std::vector<const double *> Sp(count), Yp(count), Rp(count);
    // 1/(y.s) of each pair (and, for the gathered passes, the products
    // s_a.y_b), and the direction's own scratch: the handle's solver state
    // stays untouched
    double *rho = nullptr;
    const size_t nrho = count > kCmpMax ? (size_t)count : (size_t)kLaneRho;
    CK(cudaMallocAsync((void **)&rho, sizeof(double) * (nrho + kTwoLoopScratch), H->stream), "rho buffer");
    double *scal = rho + nrho;
    int64_t *L = &H->stats.kernel_launches;
    for (int k = 0; k < count; ++k) {
        Sp[k] = S + k * n3;
        Yp[k] = Y + k * n3;
        Rp[k] = rho + k;
        dot_to((int64_t)n3, Yp[k], Sp[k], H->b.partials, &H->b.st->dots[0], H->stream, L);
        set_rho(rho, k, H->b.st, H->stream, L);
    }
    if (count >= 1 && count <= kCmpMax) {
        SegLane D = single_lane(H, 0, 0);
        D.count = count;
        for (int k = 0; k < count; ++k) D.slots[k] = k;
        D.g = const_cast<double *>(g);
        D.h = const_cast<double *>(hdiag);
        D.hist = const_cast<double *>(S);
        D.yhist = const_cast<double *>(Y);
        D.slot_stride = (int64_t)n3;
        D.rho = rho;
        D.scal = scal;
        lane_pair_products(D, H->stream, L);
        lane_direction(D, q, H->stream, L);
    } else {
        two_loop(H->n, g, hdiag, nullptr, count, Sp.data(), Yp.data(), Rp.data(), q, H->b.partials, scal, H->b.st,
                 H->stream, L);
    }
    cudaFreeAsync(rho, H->stream);
    CK(cudaGetLastError(), "two-loop launch");
    CK(cudaStreamSynchronize(H->stream), "two-loop");
    return SCVT_OK;
}

scvt_status scvt_lbfgs_solve(scvt_handle *H, double *z, const scvt_solve_opts *opts_in, scvt_solve_report *rep_out) {
    if (!H) return SCVT_ERR_INVALID;
    if (!z) return fail(H, SCVT_ERR_INVALID, "null argument");
    scvt_solve_opts o;
    memset(&o, 0, sizeof(o));
    if (opts_in) o = *opts_in;
    else { o.max_iter = 200; o.grad_tol = 1e-8; }
    if (o.ls_max_evals <= 0) o.ls_max_evals = 10;
    if (o.c1 <= 0.0) o.c1 = 1e-4;
    if (o.c2 <= 0.0) o.c2 = 0.9;
    if (o.max_iter < 0 || !(o.c1 < o.c2) || o.c2 >= 1.0 || o.method < 0 || o.method > 2)
        return fail(H, SCVT_ERR_INVALID, "bad solve options");
    scvt_solve_report rep;
    memset(&rep, 0, sizeof(rep));
    const int n = H->n;
    const size_t n3 = 3 * (size_t)n;
    Bufs &B = H->b;
    cudaStream_t s = H->stream;
    scvt_status st = SCVT_OK;
    const int64_t retries0 = H->stats.knn_retries;
    bool resume = o.warm_start && H->state_valid;
    const double *zin = nullptr;
    if (resume && o.warm_start == 2) {
        // resume only if the caller passes back the engine's own iterate
        if ((st = stage_in(H, z, n3, B.stage_a, &zin))) return st;
        vec_differs((int64_t)n3, zin, B.z, B.st, s, &H->stats.kernel_launches);
        CK(cudaMemcpyAsync(&H->st_host->differs, &B.st->differs, sizeof(unsigned), cudaMemcpyDeviceToHost, s),
           "compare copy");
        CK(cudaStreamSynchronize(s), "compare");
        resume = H->st_host->differs == 0;
    }
    if (!resume) {
        const double *zd = zin;
        if (!zd && (st = stage_in(H, z, n3, B.stage_a, &zd))) return st;
        if (zd != B.z) CK(cudaMemcpyAsync(B.z, zd, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s), "copy in");
        double F, g2;
        st = evaluate_dev(H, B.z, B.g, B.h, B.fc, nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr, &F, &g2,
                          nullptr);
        rep.fevals = 1;
        if (st) {
            H->state_valid = false;
            if (rep_out) { rep.status = st; *rep_out = rep; }
            return st;
        }
        H->F = F;
        H->gnorm = sqrt(g2);
        H->state_valid = true;
        hist_reset(H);
    }
    WolfeSearch ls;
    ls.ftol = o.c1;
    ls.gtol = o.c2;
    ls.maxfev = o.ls_max_evals;
    double Fprev = H->F;
    int iters = 0;
    for (;;) {
        rep.energy = H->F;
        rep.grad_norm = H->gnorm;
        if (H->gnorm <= o.grad_tol) { rep.converged = 1; break; }
        if (o.rel_grad_tol > 0 && H->gnorm / H->F <= o.rel_grad_tol) { rep.converged = 1; break; }
        if (iters > 0 && o.rel_df_tol > 0 && fabs(H->F - Fprev) / Fprev < o.rel_df_tol) { rep.converged = 1; break; }
        if (iters >= o.max_iter) break;
        double d0;
        if ((st = make_direction(H, &d0, o.method))) break;
        if (!(d0 < 0.0)) {
            hist_reset(H);
            rep.resets++;
            if ((st = make_direction(H, &d0, o.method))) break;
            if (!(d0 < 0.0)) { st = fail(H, SCVT_ERR_DEGENERATE, "Lloyd direction is not a descent direction"); break; }
        }
        scvt_status cb_status = SCVT_OK;
        auto phi = [&](double a, double &f, double &d) -> int {
            {
                Phase pt("scvt trial point");
                trial_point(n, B.z, B.q, a, B.zt, B.nrm, s, &H->stats.kernel_launches);
            }
            double g2;
            cb_status = evaluate_dev(H, B.zt, B.gt, B.ht, B.fc, nullptr, nullptr, nullptr, nullptr, 0, B.q, B.nrm, &f,
                                     &g2, &d);
            if (cb_status == SCVT_OK) return 0;
            // a step that breaks the tessellation is a failed trial, not an error
            if (cb_status == SCVT_ERR_DEGENERATE || cb_status == SCVT_ERR_INVALID ||
                cb_status == SCVT_ERR_KNN_EXHAUSTED) {
                cb_status = SCVT_OK;
                return 1;
            }
            return -1;
        };
        double a = 1.0, fa = 0.0, da = 0.0;
        int nfev = 0;
        int info;
        if (o.method == 2) {
            // Lloyd: the unit step, accepted as it is
            const int cb = phi(1.0, fa, da);
            nfev = 1;
            if (cb > 0) {
                rep.fevals += 1;
                st = fail(H, SCVT_ERR_DEGENERATE, "the Lloyd step is not a valid tessellation");
                break;
            }
            info = cb < 0 ? -1 : 1;
        } else {
            Phase pl("scvt line search");
            info = ls.run(phi, H->F, d0, a, fa, da, nfev);
        }
        rep.fevals += nfev;
        if (info < 0) { st = cb_status; break; }
        if (info != 1) {
            if (!(fa < H->F)) {
                if (H->hist_count == 0) { st = fail(H, SCVT_ERR_LINESEARCH, "no decrease along the Lloyd direction"); break; }
                hist_reset(H);
                rep.resets++;
                continue;
            }
            hist_reset(H);
            rep.resets++;
        }
        // accept the last evaluated point: s = z+ - z, y = g+ - g into the spare slot
        Phase pa("scvt accept");
        const int slot = H->spare;
        CK(cudaMemsetAsync(&B.st->maxmove_bits, 0, sizeof(unsigned long long), s), "reset max move");
        accept_pair(n, B.zt, B.z, B.gt, B.g, slot_S(H, slot), slot_Y(H, slot), B.partials, B.st, s,
                    &H->stats.kernel_launches);
        CK(cudaGetLastError(), "accept launch");
        CK(cudaMemcpyAsync(H->st_host, B.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s), "pair copy");
        CK(cudaStreamSynchronize(s), "accept");
        const double ys = H->st_host->dots[0], yy = H->st_host->dots[1], ss = H->st_host->dots[2];
        unsigned long long mb = H->st_host->maxmove_bits;
        double maxmove;
        memcpy(&maxmove, &mb, sizeof(double));
        if (o.method != 2 && H->m > 0 && ys > 1e-12 * sqrt(yy) * sqrt(ss)) {
            set_rho(B.rho, slot, B.st, s, &H->stats.kernel_launches);
            if (o.method == 1) set_gamma(B.rho + kLaneMaxM + 1, B.st, s, &H->stats.kernel_launches);
            if (H->hist_count == H->m) {
                // the oldest pair's slot becomes the spare
                int old = H->hist_slots[0];
                for (int k = 1; k < H->hist_count; ++k) H->hist_slots[k - 1] = H->hist_slots[k];
                H->hist_count--;
                H->spare = old;
            } else {
                // take any slot not in use as the next spare
                bool used[kMaxM + 1] = {false};
                for (int k = 0; k < H->hist_count; ++k) used[H->hist_slots[k]] = true;
                used[slot] = true;
                for (int k = 0; k <= H->m; ++k)
                    if (!used[k]) { H->spare = k; break; }
            }
            H->hist_slots[H->hist_count++] = slot;
            H->new_pair = true;
        } else if (o.method != 2) {
            rep.skipped++;
        }
        std::swap(B.z, B.zt);
        std::swap(B.g, B.gt);
        std::swap(B.h, B.ht);
        Fprev = H->F;
        H->F = fa;
        // |g| at the accepted point: the last evaluation's reduction
        H->gnorm = sqrt(H->st_host->red[1]);
        iters++;
        rep.iters = iters;
        if (o.step_tol > 0 && maxmove <= o.step_tol) {
            rep.energy = H->F;
            rep.grad_norm = H->gnorm;
            rep.converged = 1;
            break;
        }
    }
    rep.iters = iters;
    rep.knn_retries = (int)(H->stats.knn_retries - retries0);
    if (st == SCVT_OK || st == SCVT_ERR_LINESEARCH) {
        rep.energy = H->F;
        rep.grad_norm = H->gnorm;
        scvt_status c = copy_out(H, z, B.z, n3);
        if (c == SCVT_OK) {
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) c = cuda_fail(H, e, "copy out");
        }
        if (c) st = c;
    } else {
        H->state_valid = false;
    }
    rep.status = st;
    if (rep_out) *rep_out = rep;
    return st;
}

scvt_status scvt_set_tuning(scvt_handle *H, const scvt_tuning *t) {
    if (!H) return SCVT_ERR_INVALID;
    if (!t) return fail(H, SCVT_ERR_INVALID, "null argument");
    Tune u;
    scvt_status s = tune_from(*t, &u);
    if (s) return fail(H, s, "tuning out of range");
    H->tune = u;
    H->G = bins_per_edge(H->n, u.bin_load);
    return SCVT_OK;
}

scvt_status scvt_tune(scvt_handle *H, const double *z, scvt_tuning *chosen) {
    if (!H) return SCVT_ERR_INVALID;
    if (!z) return fail(H, SCVT_ERR_INVALID, "null argument");
    const size_t n3 = 3 * (size_t)H->n;
    const double *zd;
    scvt_status s = stage_in(H, z, n3, H->b.stage_a, &zd);
    if (s) return s;
    Bufs &B = H->b;
    double F, g2;
    // one evaluation leaves radius hints for the warm timings; it must succeed
    s = evaluate_dev(H, zd, B.gt, B.ht, B.fc, nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr, &F, &g2,
                     nullptr);
    if (s) return s;
    auto time_cfg = [&](const Tune &u, bool cold, float *ms) -> scvt_status {
        H->tune = u;
        H->G = bins_per_edge(H->n, u.bin_load);
        float best = INFINITY;
        for (int rep = 0; rep < 2; ++rep) {
            if (cold) CK(cudaMemsetAsync(B.radius, 0, sizeof(float) * H->n, H->stream), "clear hints");
            CK(cudaEventRecord(H->ev_l0, H->stream), "event");
            scvt_status r = evaluate_dev(H, zd, B.gt, B.ht, B.fc, nullptr, nullptr, nullptr, nullptr, 0, nullptr,
                                         nullptr, &F, &g2, nullptr);
            if (r) return r;
            CK(cudaEventRecord(H->ev_l1, H->stream), "event");
            CK(cudaEventSynchronize(H->ev_l1), "event");
            float t_ms = 0.0f;
            CK(cudaEventElapsedTime(&t_ms, H->ev_l0, H->ev_l1), "event time");
            best = std::min(best, t_ms);
        }
        *ms = best;
        return SCVT_OK;
    };
    const Tune start = H->tune;
    Tune best;
    s = autotune(start, time_cfg, &best);
    if (s) {
        H->tune = start;
        H->G = bins_per_edge(H->n, start.bin_load);
        return s;
    }
    H->tune = best;
    H->G = bins_per_edge(H->n, best.bin_load);
    // leave warm hints for the chosen configuration
    s = evaluate_dev(H, zd, B.gt, B.ht, B.fc, nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr, &F, &g2,
                     nullptr);
    if (s) return s;
    if (chosen) *chosen = tuning_of(best);
    return SCVT_OK;
}

scvt_status scvt_get_tuning(const scvt_handle *H, scvt_tuning *t) {
    if (!H || !t) return SCVT_ERR_INVALID;
    *t = tuning_of(H->tune);
    return SCVT_OK;
}

scvt_status scvt_get_stats(const scvt_handle *H, scvt_stats *out) {
    if (!H || !out) return SCVT_ERR_INVALID;
    *out = H->stats;
    out->bytes_device = H->bytes;
    return SCVT_OK;
}

scvt_status scvt_reset_stats(scvt_handle *H) {
    if (!H) return SCVT_ERR_INVALID;
    memset(&H->stats, 0, sizeof(H->stats));
    H->stats.bytes_device = H->bytes;
    return SCVT_OK;
}

scvt_status scvt_set_profiling(scvt_handle *H, int enabled) {
    if (!H) return SCVT_ERR_INVALID;
    H->profiling = enabled != 0;
    return SCVT_OK;
}

}  // extern "C"
