// batch.cu -- batches of independent problems (include/scvt.h, "Batches").
//
// The problems' generators are concatenated; problem b owns rows
// [off_b, off_b + n_b) of every per-generator array and its own block of
// cube-map bins.  One evaluation bins every problem, runs the topology
// passes, the corners, the per-edge quadrature and the per-cell sums over all
// problems' cells at once (the cell kernels look up their problem's range,
// bins and density), and reduces each problem separately with the chunking a
// single problem of its size uses.  That sequence has fixed pointers and
// launch shapes, so it is captured once as a CUDA graph and replayed; the
// host only changes the `active` mask (problems whose line search still
// needs an evaluation) between replays.
//
// The LBFGS runs per problem on the problem's row range with the same
// vector kernels and the same host logic as a single-problem handle
// (two-loop, Wolfe search, curvature test, history ring), stepped in
// lockstep: every outer round computes all directions, then runs line-search
// rounds until every search has ended, then accepts.  Each problem therefore
// reproduces a single-problem solve bit for bit.
#include <cuda_runtime.h>
#include <math.h>
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

constexpr int kMaxM = 32;

// solver state of one problem (mirrors a single-problem handle)
struct Prob {
    int n = 0;
    int64_t off = 0;  // first row
    int slots[kMaxM + 1];
    int count = 0, spare = 0;
    double F = 0.0, gnorm = 0.0, Fprev = 0.0;
    bool done = false, state_valid = false;
    scvt_solve_report rep;
    WolfeSearch ls;
    int ls_state = 0;  // 0 running, else the search's result
    double d0 = 0.0, g2_last = 0.0;
};

}  // namespace

struct scvt_batch {
    int B = 0;
    int64_t ntot = 0;
    int m = 0;
    int precision = 0;
    std::vector<scvt_config> cfg;
    std::vector<InstGeom> geom;   // host copy
    std::vector<int> pbase;       // first chunk of each problem's reduction
    int max_nb = 1;
    int nbins = 0;
    cudaStream_t ustream = nullptr, stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_a = nullptr, ev_b = nullptr;
    Tune tune;
    // device tables
    InstGeom *d_inst = nullptr;
    int *d_pinst = nullptr, *d_pbase = nullptr, *d_active = nullptr;
    Density *d_rho = nullptr;
    DensityF *d_rhof = nullptr;
    DevStatus *d_ist = nullptr, *d_st = nullptr;
    // pinned host mirrors
    DevStatus *h_ist = nullptr, *h_st = nullptr;
    int *h_active = nullptr;
    // vectors (concatenated)
    double *z = nullptr, *zt = nullptr, *g = nullptr, *gt = nullptr, *h = nullptr, *ht = nullptr, *fc = nullptr;
    double *q = nullptr, *nrm = nullptr, *stage = nullptr, *partials = nullptr, *scal = nullptr;
    double *rho_hist = nullptr, *hist = nullptr;
    // evaluation workspace
    P4 *zs = nullptr, *cvx = nullptr;
    float4 *zf = nullptr, *zl = nullptr, *vo = nullptr;
    int *cdeg = nullptr, *cnb = nullptr, *eoff = nullptr, *ecell = nullptr, *escan = nullptr;
    double *eacc = nullptr;
    int *bin_of = nullptr, *count = nullptr, *start = nullptr, *cursor = nullptr, *scan_tmp = nullptr;
    int *sidx = nullptr, *list1 = nullptr, *list2 = nullptr;
    float *radius = nullptr;
    // the captured evaluation
    cudaGraphExec_t graph = nullptr;
    int64_t graph_launches = 0, graph_cell_launches = 0;
    std::vector<Prob> prob;
    bool solved_once = false;
    scvt_stats stats;
    int64_t bytes = 0;
    std::string err;
};

namespace {

scvt_status bfail(scvt_batch *b, scvt_status s, const std::string &msg) {
    if (b) b->err = msg;
    return s;
}

scvt_status bcuda(scvt_batch *b, cudaError_t e, const char *what) {
    cudaGetLastError();
    return bfail(b, e == cudaErrorMemoryAllocation ? SCVT_ERR_OOM : SCVT_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

#define BK(call, what)                                     \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return bcuda(BT, e_, what); \
    } while (0)

template <class T>
cudaError_t balloc(scvt_batch *BT, T **p, size_t count) {
    size_t bytes = sizeof(T) * (count ? count : 1);
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e == cudaSuccess) BT->bytes += (int64_t)bytes;
    return e;
}

bool dev_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

scvt_status status_of_flags(unsigned f) {
    if (f & (FLAG_BAD_POINT | FLAG_DUPLICATE)) return SCVT_ERR_INVALID;
    if (f & (FLAG_UNBOUNDED | FLAG_EMPTY)) return SCVT_ERR_DEGENERATE;
    if (f & (FLAG_EXHAUSTED | FLAG_VMAX)) return SCVT_ERR_KNN_EXHAUSTED;
    if (f & FLAG_NONPOSITIVE) return SCVT_ERR_DEGENERATE;
    return SCVT_OK;
}

scvt_status validate_config(const scvt_config &c) {
    if (c.n < 4 || c.n > (int64_t)200000000) return SCVT_ERR_INVALID;
    if (c.lbfgs_m < 0 || c.lbfgs_m > kMaxM) return SCVT_ERR_INVALID;
    if (c.quad_points != 0 && c.quad_points != 7) return SCVT_ERR_INVALID;
    if (c.precision != 0 && c.precision != 1) return SCVT_ERR_INVALID;
    if (c.rho.kind < 0 || c.rho.kind > 3) return SCVT_ERR_INVALID;
    if (c.rho.kind != SCVT_RHO_UNIFORM) {
        if (!(c.rho.gamma > 0.0) || !(c.rho.gamma <= 1.0)) return SCVT_ERR_INVALID;
        if (c.rho.kind >= 2) {
            double r = sqrt(c.rho.xc[0] * c.rho.xc[0] + c.rho.xc[1] * c.rho.xc[1] + c.rho.xc[2] * c.rho.xc[2]);
            if (!(fabs(r - 1.0) < 1e-9) || !(c.rho.alpha > 0.0)) return SCVT_ERR_INVALID;
        }
    }
    return SCVT_OK;
}

// per-problem bins for the current tuning; uploads the geometry table
scvt_status layout_bins(scvt_batch *BT) {
    int bin0 = 0;
    for (int b = 0; b < BT->B; ++b) {
        const int G = bins_per_edge(BT->geom[b].n, BT->tune.bin_load);
        BT->geom[b].G = G;
        BT->geom[b].bin0 = bin0;
        bin0 += 6 * G * G;
    }
    BT->nbins = bin0;
    BK(cudaMemcpyAsync(BT->d_inst, BT->geom.data(), sizeof(InstGeom) * BT->B, cudaMemcpyHostToDevice, BT->stream),
       "problem table");
    BK(cudaStreamSynchronize(BT->stream), "problem table");
    return SCVT_OK;
}

Grid make_grid(const scvt_batch *BT) {
    Grid g;
    memset(&g, 0, sizeof(g));
    g.n = (int)BT->ntot;
    g.G = BT->geom[0].G;
    g.nbins = BT->nbins;
    g.zs = BT->zs;
    g.zf = BT->zf;
    g.zl = BT->zl;
    g.sidx = BT->sidx;
    g.bstart = BT->start;
    g.inst = BT->d_inst;
    g.pinst = BT->d_pinst;
    g.rho = BT->d_rho;
    g.rhof = BT->d_rhof;
    g.ist = BT->d_ist;
    g.active = BT->d_active;
    return g;
}

// the evaluation at zt of the active problems: gt, ht, fc, per-problem sums
// (phi' along q with nrm), statuses copied to the pinned mirrors
void enqueue_eval(scvt_batch *BT, int64_t *launches, int64_t *cell_launches) {
    cudaStream_t s = BT->stream;
    cudaMemsetAsync(BT->d_st, 0, sizeof(DevStatus), s);
    cudaMemsetAsync(BT->d_ist, 0, sizeof(DevStatus) * BT->B, s);
    Grid g = make_grid(BT);
    bin_points(BT->zt, g, BT->bin_of, BT->count, BT->start, BT->cursor, BT->scan_tmp, BT->zs, BT->zf, BT->zl,
               BT->sidx, BT->d_st, s, launches);
    CellOut out;
    memset(&out, 0, sizeof(out));
    out.grad = BT->gt;
    out.hdiag = BT->ht;
    out.fcell = BT->fc;
    out.radius = BT->radius;
    CellBuf cb;
    cb.deg = BT->cdeg;
    cb.vx = BT->cvx;
    cb.nb = BT->cnb;
    cb.eoff = BT->eoff;
    cb.ecell = BT->ecell;
    cb.scan_tmp = BT->escan;
    cb.eacc = BT->eacc;
    cb.vo = BT->vo;
    cell_passes(g, out, cb, BT->list1, BT->list2, BT->d_st, BT->precision == 1, BT->tune, s, nullptr, nullptr,
                launches, cell_launches);
    reduce_eval_batch(BT->B, BT->max_nb, BT->d_inst, BT->d_pbase, BT->d_active, BT->fc, BT->gt, BT->q, BT->nrm,
                      BT->partials, BT->d_ist, s, launches);
    cudaMemcpyAsync(BT->h_ist, BT->d_ist, sizeof(DevStatus) * BT->B, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(BT->h_st, BT->d_st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s);
}

scvt_status capture(scvt_batch *BT) {
    if (BT->graph) {
        cudaGraphExecDestroy(BT->graph);
        BT->graph = nullptr;
    }
    cudaGraph_t gr = nullptr;
    BK(cudaStreamBeginCapture(BT->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    int64_t l = 0, c = 0;
    enqueue_eval(BT, &l, &c);
    cudaError_t e = cudaStreamEndCapture(BT->stream, &gr);
    if (e != cudaSuccess) return bcuda(BT, e, "capture of the evaluation");
    e = cudaGraphInstantiate(&BT->graph, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
        BT->graph = nullptr;
        return bcuda(BT, e, "graph instantiation");
    }
    BT->graph_launches = l;
    BT->graph_cell_launches = c;
    return SCVT_OK;
}

// one batched evaluation of the problems marked in h_active; synchronises
scvt_status run_eval(scvt_batch *BT) {
    if (!BT->graph) {
        scvt_status s = capture(BT);
        if (s) return s;
    }
    BK(cudaMemcpyAsync(BT->d_active, BT->h_active, sizeof(int) * BT->B, cudaMemcpyHostToDevice, BT->stream),
       "active mask");
    BK(cudaGraphLaunch(BT->graph, BT->stream), "graph launch");
    BK(cudaStreamSynchronize(BT->stream), "evaluation");
    BT->stats.evaluations++;
    BT->stats.kernel_launches += BT->graph_launches;
    BT->stats.cell_launches += BT->graph_cell_launches;
    BT->stats.knn_retries += BT->h_st->retry_count[0];
    BT->stats.ambiguous += (int64_t)BT->h_st->ambiguous;
    return SCVT_OK;
}

scvt_status stage_in(scvt_batch *BT, const double *p, size_t count, double *dst) {
    BK(cudaMemcpyAsync(dst, p, sizeof(double) * count, dev_ptr(p) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       BT->stream),
       "copy in");
    return SCVT_OK;
}

scvt_status copy_to_caller(scvt_batch *BT, double *dst, const double *src, size_t count) {
    BK(cudaMemcpyAsync(dst, src, sizeof(double) * count,
                       dev_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, BT->stream),
       "copy out");
    return SCVT_OK;
}

void enter(scvt_batch *BT) {
    cudaEventRecord(BT->ev_in, BT->ustream);
    cudaStreamWaitEvent(BT->stream, BT->ev_in, 0);
}

double *slot_S(scvt_batch *BT, int slot) { return BT->hist + (size_t)slot * 2 * 3 * BT->ntot; }
double *slot_Y(scvt_batch *BT, int slot) { return slot_S(BT, slot) + (size_t)3 * BT->ntot; }
double *rho_of(scvt_batch *BT, int b) { return BT->rho_hist + (size_t)b * (kMaxM + 1); }

void hist_reset(Prob &P, int m) {
    P.count = 0;
    for (int k = 0; k <= m; ++k) P.slots[k] = k;
    P.spare = m;
}

// the two-loop direction of problem b into q (its rows); g.q is left in
// the problem's status block
void enqueue_direction(scvt_batch *BT, int b) {
    Prob &P = BT->prob[b];
    const double *S[kMaxM], *Y[kMaxM], *R[kMaxM];
    const size_t o3 = 3 * (size_t)P.off;
    for (int k = 0; k < P.count; ++k) {
        const int sl = P.slots[k];
        S[k] = slot_S(BT, sl) + o3;
        Y[k] = slot_Y(BT, sl) + o3;
        R[k] = rho_of(BT, b) + sl;
    }
    two_loop(P.n, BT->g + o3, BT->h + P.off, P.count, S, Y, R, BT->q + o3, BT->partials, BT->scal, &BT->d_ist[b],
             BT->stream, &BT->stats.kernel_launches);
}

scvt_status sync_statuses(scvt_batch *BT) {
    BK(cudaMemcpyAsync(BT->h_ist, BT->d_ist, sizeof(DevStatus) * BT->B, cudaMemcpyDeviceToHost, BT->stream),
       "status copy");
    BK(cudaStreamSynchronize(BT->stream), "status");
    return SCVT_OK;
}

}  // namespace

extern "C" {

void scvt_batch_destroy(scvt_batch *BT) {
    if (!BT) return;
    if (BT->graph) cudaGraphExecDestroy(BT->graph);
    void *ptrs[] = {BT->d_inst, BT->d_pinst, BT->d_pbase, BT->d_active, BT->d_rho, BT->d_rhof, BT->d_ist, BT->d_st,
                    BT->z, BT->zt, BT->g, BT->gt, BT->h, BT->ht, BT->fc, BT->q, BT->nrm, BT->stage, BT->partials,
                    BT->scal, BT->rho_hist, BT->hist, BT->zs, BT->cvx, BT->zf, BT->zl, BT->vo, BT->cdeg, BT->cnb,
                    BT->eoff, BT->ecell, BT->escan, BT->eacc, BT->bin_of, BT->count, BT->start, BT->cursor,
                    BT->scan_tmp, BT->sidx, BT->list1, BT->list2, BT->radius};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    void *hp[] = {BT->h_ist, BT->h_st, BT->h_active};
    for (void *p : hp)
        if (p) cudaFreeHost(p);
    cudaEvent_t evs[] = {BT->ev_in, BT->ev_a, BT->ev_b};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    if (BT->stream) cudaStreamDestroy(BT->stream);
    delete BT;
}

scvt_status scvt_batch_create(const scvt_config *cfgs, int count, void *cuda_stream, scvt_batch **out) {
    if (!cfgs || !out || count < 1 || count > 65535) return SCVT_ERR_INVALID;
    *out = nullptr;
    int64_t ntot = 0;
    for (int b = 0; b < count; ++b) {
        if (validate_config(cfgs[b])) return SCVT_ERR_INVALID;
        if (cfgs[b].precision != cfgs[0].precision || cfgs[b].lbfgs_m != cfgs[0].lbfgs_m) return SCVT_ERR_INVALID;
        ntot += cfgs[b].n;
    }
    if (ntot > (int64_t)200000000) return SCVT_ERR_INVALID;
    scvt_batch *BT = new (std::nothrow) scvt_batch();
    if (!BT) return SCVT_ERR_OOM;
    BT->B = count;
    BT->ntot = ntot;
    BT->m = cfgs[0].lbfgs_m;
    BT->precision = cfgs[0].precision;
    BT->cfg.assign(cfgs, cfgs + count);
    BT->ustream = (cudaStream_t)cuda_stream;
    memset(&BT->stats, 0, sizeof(BT->stats));
    BT->geom.resize(count);
    BT->pbase.resize(count);
    BT->prob.resize(count);
    int64_t off = 0, nb_total = 0, bins1 = 0;
    for (int b = 0; b < count; ++b) {
        const int n = (int)cfgs[b].n;
        BT->geom[b].p0 = (int)off;
        BT->geom[b].n = n;
        BT->prob[b].n = n;
        BT->prob[b].off = off;
        const int nb = reduce_blocks(n);
        BT->pbase[b] = (int)nb_total;
        nb_total += nb;
        BT->max_nb = std::max(BT->max_nb, nb);
        const int g1 = bins_per_edge(n, 1);
        bins1 += 6LL * g1 * g1;
        off += n;
    }
    const size_t N = (size_t)ntot, n3 = 3 * N;
    const size_t nbins_max = (size_t)bins1;
    cudaError_t e = cudaStreamCreateWithFlags(&BT->stream, cudaStreamNonBlocking);
#define AL(ptr, cnt) \
    if (e == cudaSuccess) e = balloc(BT, &(ptr), (cnt))
    AL(BT->d_inst, count); AL(BT->d_pinst, N); AL(BT->d_pbase, count); AL(BT->d_active, count);
    AL(BT->d_rho, count); AL(BT->d_rhof, count); AL(BT->d_ist, count); AL(BT->d_st, 1);
    AL(BT->z, n3); AL(BT->zt, n3); AL(BT->g, n3); AL(BT->gt, n3); AL(BT->h, N); AL(BT->ht, N); AL(BT->fc, N);
    AL(BT->q, n3); AL(BT->nrm, N); AL(BT->stage, n3);
    AL(BT->partials, std::max<size_t>(4 * 1024, 4 * (size_t)nb_total)); AL(BT->scal, 128);
    AL(BT->rho_hist, (size_t)count * (kMaxM + 1));
    AL(BT->hist, (size_t)(BT->m + 1) * 2 * n3);
    AL(BT->zs, N); AL(BT->zf, N); AL(BT->zl, N); AL(BT->cvx, N * kCellSlots); AL(BT->cnb, N * kCellSlots);
    AL(BT->cdeg, N); AL(BT->eoff, N + 1); AL(BT->ecell, 6 * N); AL(BT->escan, 2 * (N / 2048 + 64) + 64);
    AL(BT->eacc, 5 * 6 * N);
    if (BT->precision == 1) AL(BT->vo, N * kCellSlots);
    AL(BT->bin_of, N); AL(BT->count, nbins_max); AL(BT->start, nbins_max + 1); AL(BT->cursor, nbins_max);
    AL(BT->scan_tmp, 2 * (nbins_max / 2048 + 64) + 64);
    AL(BT->sidx, N); AL(BT->list1, N); AL(BT->list2, N); AL(BT->radius, N);
#undef AL
    if (e == cudaSuccess) e = cudaMallocHost((void **)&BT->h_ist, sizeof(DevStatus) * count);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&BT->h_st, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&BT->h_active, sizeof(int) * count);
    cudaEvent_t *evs[] = {&BT->ev_in, &BT->ev_a, &BT->ev_b};
    for (cudaEvent_t *ev : evs)
        if (e == cudaSuccess) e = cudaEventCreate(ev);
    if (e == cudaSuccess) {
        // static tables: problem of each row, densities, reduction bases
        std::vector<int> pinst(N);
        std::vector<Density> rho(count);
        std::vector<DensityF> rhof(count);
        for (int b = 0; b < count; ++b) {
            for (int i = 0; i < BT->geom[b].n; ++i) pinst[BT->geom[b].p0 + i] = b;
            rho[b] = to_device_density(cfgs[b].rho);
            rhof[b] = to_density32(rho[b]);
        }
        e = cudaMemcpy(BT->d_pinst, pinst.data(), sizeof(int) * N, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(BT->d_rho, rho.data(), sizeof(Density) * count, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(BT->d_rhof, rhof.data(), sizeof(DensityF) * count, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(BT->d_pbase, BT->pbase.data(), sizeof(int) * count, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(BT->radius, 0, sizeof(float) * N);
        if (e == cudaSuccess) e = cudaMemset(BT->q, 0, sizeof(double) * n3);
        if (e == cudaSuccess) e = cudaMemset(BT->nrm, 0, sizeof(double) * N);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        scvt_batch_destroy(BT);
        return e == cudaErrorMemoryAllocation ? SCVT_ERR_OOM : SCVT_ERR_CUDA;
    }
    if (layout_bins(BT) != SCVT_OK) {
        scvt_batch_destroy(BT);
        return SCVT_ERR_CUDA;
    }
    BT->stats.bytes_device = BT->bytes;
    *out = BT;
    return SCVT_OK;
}

scvt_status scvt_batch_energy_grad(scvt_batch *BT, const double *z, double *energy, double *grad) {
    if (!BT) return SCVT_ERR_INVALID;
    if (!z || !energy) return bfail(BT, SCVT_ERR_INVALID, "null argument");
    enter(BT);
    const size_t n3 = 3 * (size_t)BT->ntot;
    scvt_status s = stage_in(BT, z, n3, BT->zt);
    if (s) return s;
    for (int b = 0; b < BT->B; ++b) BT->h_active[b] = 1;
    if ((s = run_eval(BT))) return s;
    scvt_status first = SCVT_OK;
    for (int b = 0; b < BT->B; ++b) {
        energy[b] = BT->h_ist[b].red[0];
        scvt_status sb = status_of_flags(BT->h_ist[b].flags);
        if (sb && !first) {
            first = sb;
            BT->err = "problem " + std::to_string(b) + ": " + scvt_status_string(sb);
        }
    }
    if (grad) {
        if ((s = copy_to_caller(BT, grad, BT->gt, n3))) return s;
        BK(cudaStreamSynchronize(BT->stream), "copy out");
    }
    if (!first) BT->err.clear();
    return first;
}

scvt_status scvt_batch_lbfgs_solve(scvt_batch *BT, double *z, const scvt_solve_opts *opts_in,
                                   scvt_solve_report *reports) {
    if (!BT) return SCVT_ERR_INVALID;
    if (!z || !reports) return bfail(BT, SCVT_ERR_INVALID, "null argument");
    scvt_solve_opts o;
    memset(&o, 0, sizeof(o));
    if (opts_in) o = *opts_in;
    else { o.max_iter = 200; o.grad_tol = 1e-8; }
    if (o.ls_max_evals <= 0) o.ls_max_evals = 10;
    if (o.c1 <= 0.0) o.c1 = 1e-4;
    if (o.c2 <= 0.0) o.c2 = 0.9;
    if (o.max_iter < 0 || !(o.c1 < o.c2) || o.c2 >= 1.0 || o.warm_start < 0 || o.warm_start > 1)
        return bfail(BT, SCVT_ERR_INVALID, "bad solve options");
    enter(BT);
    const int B = BT->B, m = BT->m;
    const size_t n3 = 3 * (size_t)BT->ntot;
    cudaStream_t s = BT->stream;
    int64_t *L = &BT->stats.kernel_launches;
    std::vector<Prob> &P = BT->prob;
    scvt_status st;
    const bool resume = o.warm_start == 1 && BT->solved_once;
    for (int b = 0; b < B; ++b) {
        memset(&P[b].rep, 0, sizeof(scvt_solve_report));
        P[b].done = false;
    }
    if (!resume || [&] {
            for (int b = 0; b < B; ++b)
                if (!P[b].state_valid) return true;
            return false;
        }()) {
        // initial evaluation of every problem at z
        if ((st = stage_in(BT, z, n3, BT->z))) return st;
        BK(cudaMemcpyAsync(BT->zt, BT->z, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s), "copy in");
        for (int b = 0; b < B; ++b) BT->h_active[b] = 1;
        if ((st = run_eval(BT))) return st;
        BK(cudaMemcpyAsync(BT->g, BT->gt, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s), "gradient");
        BK(cudaMemcpyAsync(BT->h, BT->ht, sizeof(double) * BT->ntot, cudaMemcpyDeviceToDevice, s), "precond");
        for (int b = 0; b < B; ++b) {
            Prob &p = P[b];
            p.rep.fevals = 1;
            scvt_status sb = status_of_flags(BT->h_ist[b].flags);
            if (sb) {
                p.rep.status = sb;
                p.done = true;
                p.state_valid = false;
                continue;
            }
            p.F = BT->h_ist[b].red[0];
            p.gnorm = sqrt(BT->h_ist[b].red[1]);
            p.state_valid = true;
            hist_reset(p, m);
        }
    }
    for (int b = 0; b < B; ++b) {
        P[b].ls.ftol = o.c1;
        P[b].ls.gtol = o.c2;
        P[b].ls.maxfev = o.ls_max_evals;
        P[b].Fprev = P[b].F;
    }
    for (;;) {
        // ---- stopping tests
        std::vector<int> act;
        for (int b = 0; b < B; ++b) {
            Prob &p = P[b];
            if (p.done) continue;
            p.rep.energy = p.F;
            p.rep.grad_norm = p.gnorm;
            bool stop = false;
            if (p.gnorm <= o.grad_tol) { p.rep.converged = 1; stop = true; }
            else if (o.rel_grad_tol > 0 && p.gnorm / p.F <= o.rel_grad_tol) { p.rep.converged = 1; stop = true; }
            else if (p.rep.iters > 0 && o.rel_df_tol > 0 && fabs(p.F - p.Fprev) / p.Fprev < o.rel_df_tol) {
                p.rep.converged = 1;
                stop = true;
            } else if (p.rep.iters >= o.max_iter) {
                stop = true;
            }
            if (stop) p.done = true;
            else act.push_back(b);
        }
        if (act.empty()) break;
        // ---- directions (a second round for problems whose direction is not a descent direction)
        for (int b : act) enqueue_direction(BT, b);
        if ((st = sync_statuses(BT))) return st;
        std::vector<int> redo;
        for (int b : act) {
            P[b].d0 = BT->h_ist[b].dots[3];
            if (!(P[b].d0 < 0.0)) redo.push_back(b);
        }
        if (!redo.empty()) {
            for (int b : redo) {
                hist_reset(P[b], m);
                P[b].rep.resets++;
                enqueue_direction(BT, b);
            }
            if ((st = sync_statuses(BT))) return st;
            for (int b : redo) {
                P[b].d0 = BT->h_ist[b].dots[3];
                if (!(P[b].d0 < 0.0)) {
                    P[b].rep.status = SCVT_ERR_DEGENERATE;
                    P[b].done = true;
                    P[b].state_valid = false;
                }
            }
        }
        // ---- line searches in lockstep
        std::vector<int> ls;
        for (int b : act) {
            if (P[b].done) continue;
            P[b].ls_state = P[b].ls.begin(P[b].F, P[b].d0, 1.0);
            if (P[b].ls_state == 0) ls.push_back(b);
        }
        while (!ls.empty()) {
            for (int b = 0; b < B; ++b) BT->h_active[b] = 0;
            for (int b : ls) {
                Prob &p = P[b];
                const size_t o3 = 3 * (size_t)p.off;
                trial_point(p.n, BT->z + o3, BT->q + o3, p.ls.trial(), BT->zt + o3, BT->nrm + p.off, s, L);
                BT->h_active[b] = 1;
            }
            if ((st = run_eval(BT))) return st;
            std::vector<int> next;
            for (int b : ls) {
                Prob &p = P[b];
                const DevStatus &ds = BT->h_ist[b];
                const scvt_status sb = status_of_flags(ds.flags);
                // a step that breaks the tessellation is a failed trial, not an error
                const int cb = sb ? 1 : 0;
                p.g2_last = ds.red[1];
                p.ls_state = p.ls.feed(cb, sb ? 0.0 : ds.red[0], sb ? 0.0 : ds.red[2]);
                if (p.ls_state == 0) next.push_back(b);
            }
            ls.swap(next);
        }
        // ---- accept (or restart) per problem
        std::vector<int> acc;
        for (int b : act) {
            Prob &p = P[b];
            if (p.done) continue;
            p.rep.fevals += p.ls.nfev;
            const int info = p.ls_state;
            const double fa = p.ls.last_f;
            if (info != 1) {
                if (!(fa < p.F)) {
                    if (p.count == 0) {
                        p.rep.status = SCVT_ERR_LINESEARCH;
                        p.done = true;
                        continue;
                    }
                    hist_reset(p, m);
                    p.rep.resets++;
                    continue;
                }
                hist_reset(p, m);
                p.rep.resets++;
            }
            const size_t o3 = 3 * (size_t)p.off;
            const int slot = p.spare;
            cudaMemsetAsync(&BT->d_ist[b].maxmove_bits, 0, sizeof(unsigned long long), s);
            accept_pair(p.n, BT->zt + o3, BT->z + o3, BT->gt + o3, BT->g + o3, slot_S(BT, slot) + o3,
                        slot_Y(BT, slot) + o3, BT->partials, &BT->d_ist[b], s, L);
            acc.push_back(b);
        }
        if (!acc.empty()) {
            BK(cudaGetLastError(), "accept launch");
            if ((st = sync_statuses(BT))) return st;
        }
        for (int b : acc) {
            Prob &p = P[b];
            const DevStatus &ds = BT->h_ist[b];
            const double ys = ds.dots[0], yy = ds.dots[1], ss = ds.dots[2];
            double maxmove;
            unsigned long long mb = ds.maxmove_bits;
            memcpy(&maxmove, &mb, sizeof(double));
            const int slot = p.spare;
            if (m > 0 && ys > 1e-12 * sqrt(yy) * sqrt(ss)) {
                set_rho(rho_of(BT, b), slot, &BT->d_ist[b], s, L);
                if (p.count == m) {
                    int old = p.slots[0];
                    for (int k = 1; k < p.count; ++k) p.slots[k - 1] = p.slots[k];
                    p.count--;
                    p.spare = old;
                } else {
                    bool used[kMaxM + 1] = {false};
                    for (int k = 0; k < p.count; ++k) used[p.slots[k]] = true;
                    used[slot] = true;
                    for (int k = 0; k <= m; ++k)
                        if (!used[k]) { p.spare = k; break; }
                }
                p.slots[p.count++] = slot;
            } else {
                p.rep.skipped++;
            }
            const size_t o3 = 3 * (size_t)p.off;
            cudaMemcpyAsync(BT->z + o3, BT->zt + o3, sizeof(double) * 3 * p.n, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(BT->g + o3, BT->gt + o3, sizeof(double) * 3 * p.n, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(BT->h + p.off, BT->ht + p.off, sizeof(double) * p.n, cudaMemcpyDeviceToDevice, s);
            p.Fprev = p.F;
            p.F = p.ls.last_f;
            p.gnorm = sqrt(p.g2_last);
            p.rep.iters++;
            if (o.step_tol > 0 && maxmove <= o.step_tol) {
                p.rep.energy = p.F;
                p.rep.grad_norm = p.gnorm;
                p.rep.converged = 1;
                p.done = true;
            }
        }
        BK(cudaGetLastError(), "history update");
    }
    // ---- results
    scvt_status ret = SCVT_OK;
    for (int b = 0; b < B; ++b) {
        Prob &p = P[b];
        if (p.rep.status == SCVT_OK || p.rep.status == SCVT_ERR_LINESEARCH) {
            p.rep.energy = p.F;
            p.rep.grad_norm = p.gnorm;
        }
        reports[b] = p.rep;
        if (p.rep.status == SCVT_ERR_LINESEARCH && ret == SCVT_OK) ret = SCVT_ERR_LINESEARCH;
        if (p.rep.status != SCVT_OK && p.rep.status != SCVT_ERR_LINESEARCH &&
            (ret == SCVT_OK || ret == SCVT_ERR_LINESEARCH)) {
            ret = (scvt_status)p.rep.status;
            BT->err = "problem " + std::to_string(b) + ": " + scvt_status_string(ret);
        }
    }
    if ((st = copy_to_caller(BT, z, BT->z, n3))) return st;
    BK(cudaStreamSynchronize(s), "copy out");
    BT->solved_once = true;
    if (ret == SCVT_OK) BT->err.clear();
    return ret;
}

scvt_status scvt_batch_set_tuning(scvt_batch *BT, const scvt_tuning *t) {
    if (!BT) return SCVT_ERR_INVALID;
    if (!t) return bfail(BT, SCVT_ERR_INVALID, "null argument");
    Tune u;
    if (tune_from(*t, &u)) return bfail(BT, SCVT_ERR_INVALID, "tuning out of range");
    BT->tune = u;
    scvt_status s = layout_bins(BT);
    if (s) return s;
    if (BT->graph) {
        cudaGraphExecDestroy(BT->graph);
        BT->graph = nullptr;
    }
    return SCVT_OK;
}

scvt_status scvt_batch_get_tuning(const scvt_batch *BT, scvt_tuning *t) {
    if (!BT || !t) return SCVT_ERR_INVALID;
    *t = tuning_of(BT->tune);
    return SCVT_OK;
}

scvt_status scvt_batch_tune(scvt_batch *BT, const double *z, scvt_tuning *chosen) {
    if (!BT) return SCVT_ERR_INVALID;
    if (!z) return bfail(BT, SCVT_ERR_INVALID, "null argument");
    enter(BT);
    scvt_status s = stage_in(BT, z, 3 * (size_t)BT->ntot, BT->zt);
    if (s) return s;
    for (int b = 0; b < BT->B; ++b) BT->h_active[b] = 1;
    // one evaluation leaves radius hints for the warm timings; it must succeed
    if ((s = run_eval(BT))) return s;
    for (int b = 0; b < BT->B; ++b)
        if ((s = status_of_flags(BT->h_ist[b].flags))) return bfail(BT, s, "tuning input is not a valid batch");
    // time one configuration: best of two evaluations (cold: radius hints cleared first)
    auto time_cfg = [&](const Tune &u, bool cold, float *ms) -> scvt_status {
        scvt_tuning t = tuning_of(u);
        scvt_status r = scvt_batch_set_tuning(BT, &t);
        if (r) return r;
        if ((r = capture(BT))) return r;
        float best = INFINITY;
        for (int rep = 0; rep < 2; ++rep) {
            if (cold) BK(cudaMemsetAsync(BT->radius, 0, sizeof(float) * BT->ntot, BT->stream), "clear hints");
            BK(cudaEventRecord(BT->ev_a, BT->stream), "event");
            if ((r = run_eval(BT))) return r;
            BK(cudaEventRecord(BT->ev_b, BT->stream), "event");
            BK(cudaEventSynchronize(BT->ev_b), "event");
            float t_ms = 0.0f;
            BK(cudaEventElapsedTime(&t_ms, BT->ev_a, BT->ev_b), "event time");
            best = std::min(best, t_ms);
        }
        *ms = best;
        return SCVT_OK;
    };
    Tune cur;
    if ((s = autotune(BT->tune, time_cfg, &cur))) return s;
    scvt_tuning t = tuning_of(cur);
    if ((s = scvt_batch_set_tuning(BT, &t))) return s;
    // leave warm hints for the chosen configuration
    if ((s = run_eval(BT))) return s;
    if (chosen) *chosen = t;
    return SCVT_OK;
}

scvt_status scvt_batch_get_stats(const scvt_batch *BT, scvt_stats *out) {
    if (!BT || !out) return SCVT_ERR_INVALID;
    *out = BT->stats;
    out->bytes_device = BT->bytes;
    return SCVT_OK;
}

scvt_status scvt_batch_reset_stats(scvt_batch *BT) {
    if (!BT) return SCVT_ERR_INVALID;
    memset(&BT->stats, 0, sizeof(BT->stats));
    BT->stats.bytes_device = BT->bytes;
    return SCVT_OK;
}

const char *scvt_batch_last_error(const scvt_batch *BT) { return BT ? BT->err.c_str() : ""; }

}  // extern "C"
