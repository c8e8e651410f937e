// batch.cu -- batches of independent problems (include/scvt.h, "Batches").
//
// The problems' generators are concatenated; problem b owns rows
// [off_b, off_b + n_b) of every per-generator array (iterate, gradient,
// preconditioner, history) and of the evaluation workspace (evalset.cuh:
// one captured graph evaluates every problem's cells, one reduction per
// problem).  The LBFGS runs per problem with the single-problem logic,
// stepped in lockstep (lockstep.cuh), so each problem reproduces a
// single-problem solve bit for bit.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "autotune.h"
#include "evalset.cuh"
#include "lockstep.cuh"

using namespace scvt;

struct scvt_batch {
    int B = 0;
    int64_t ntot = 0;
    int m = 0;
    std::vector<scvt_config> cfg;
    std::vector<int64_t> off;
    cudaStream_t ustream = nullptr, stream = nullptr;
    cudaEvent_t ev_in = nullptr;
    EvalSet E;
    // resident vectors (concatenated)
    double *z = nullptr, *g = nullptr, *h = nullptr, *hist = nullptr, *rho_hist = nullptr;
    std::vector<Lane> lanes;
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

scvt_status validate_config(const scvt_config &c) {
    if (c.n < 4 || c.n > (int64_t)200000000) return SCVT_ERR_INVALID;
    if (c.lbfgs_m < 0 || c.lbfgs_m > kLaneMaxM) return SCVT_ERR_INVALID;
    if (c.quad_points != 0 && c.quad_points != 7) return SCVT_ERR_INVALID;
    if (c.precision < 0 || c.precision > 2) return SCVT_ERR_INVALID;
    if (c.decomposition != 0 && c.decomposition != 1) return SCVT_ERR_INVALID;
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

scvt_status copy_in(scvt_batch *BT, const double *p, size_t count, double *dst) {
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

}  // namespace

extern "C" {

void scvt_batch_destroy(scvt_batch *BT) {
    if (!BT) return;
    evalset_free(BT->E);
    void *ptrs[] = {BT->z, BT->g, BT->h, BT->hist, BT->rho_hist};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (BT->ev_in) cudaEventDestroy(BT->ev_in);
    if (BT->stream) cudaStreamDestroy(BT->stream);
    delete BT;
}

scvt_status scvt_batch_create(const scvt_config *cfgs, int count, void *cuda_stream, scvt_batch **out) {
    if (!cfgs || !out || count < 1 || count > 65535) return SCVT_ERR_INVALID;
    *out = nullptr;
    int64_t ntot = 0;
    for (int b = 0; b < count; ++b) {
        if (validate_config(cfgs[b])) return SCVT_ERR_INVALID;
        if (cfgs[b].precision != cfgs[0].precision || cfgs[b].lbfgs_m != cfgs[0].lbfgs_m ||
            cfgs[b].decomposition != cfgs[0].decomposition)
            return SCVT_ERR_INVALID;
        ntot += cfgs[b].n;
    }
    if (ntot > (int64_t)200000000) return SCVT_ERR_INVALID;
    scvt_batch *BT = new (std::nothrow) scvt_batch();
    if (!BT) return SCVT_ERR_OOM;
    BT->B = count;
    BT->ntot = ntot;
    BT->m = cfgs[0].lbfgs_m;
    BT->cfg.assign(cfgs, cfgs + count);
    BT->ustream = (cudaStream_t)cuda_stream;
    memset(&BT->stats, 0, sizeof(BT->stats));
    const size_t N = (size_t)ntot, n3 = 3 * N;
    cudaError_t e = cudaStreamCreateWithFlags(&BT->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&BT->ev_in);
    if (e == cudaSuccess) e = evalset_alloc(BT->E, ntot, count, cfgs[0].precision, BT->stream);
    BT->E.fan = cfgs[0].decomposition;
#define AL(ptr, cnt) \
    if (e == cudaSuccess) e = balloc(BT, &(ptr), (cnt))
    AL(BT->z, n3); AL(BT->g, n3); AL(BT->h, N);
    AL(BT->hist, (size_t)(BT->m + 1) * 2 * n3); AL(BT->rho_hist, (size_t)count * kLaneRho);
#undef AL
    std::vector<int> ns(count);
    std::vector<scvt_density> rhos(count);
    for (int b = 0; b < count; ++b) {
        ns[b] = (int)cfgs[b].n;
        rhos[b] = cfgs[b].rho;
    }
    if (e == cudaSuccess) e = evalset_layout(BT->E, count, ns.data(), rhos.data());
    if (e != cudaSuccess) {
        cudaGetLastError();
        scvt_batch_destroy(BT);
        return e == cudaErrorMemoryAllocation ? SCVT_ERR_OOM : SCVT_ERR_CUDA;
    }
    BT->lanes.resize(count);
    BT->off.resize(count);
    int64_t off = 0;
    for (int b = 0; b < count; ++b) {
        Lane &L = BT->lanes[b];
        L.b = b;
        L.n = ns[b];
        L.row = off;
        L.z = BT->z + 3 * off;
        L.g = BT->g + 3 * off;
        L.h = BT->h + off;
        L.hist = BT->hist + 3 * off;
        L.slot_stride = 2 * n3;
        L.y_off = n3;
        L.rho = BT->rho_hist + (size_t)b * kLaneRho;
        BT->off[b] = off;
        off += ns[b];
    }
    BT->bytes += BT->E.bytes;
    BT->stats.bytes_device = BT->bytes;
    *out = BT;
    return SCVT_OK;
}

scvt_status scvt_batch_energy_grad(scvt_batch *BT, const double *z, double *energy, double *grad) {
    if (!BT) return SCVT_ERR_INVALID;
    if (!z || !energy) return bfail(BT, SCVT_ERR_INVALID, "null argument");
    enter(BT);
    EvalSet &E = BT->E;
    const size_t n3 = 3 * (size_t)BT->ntot;
    scvt_status s = copy_in(BT, z, n3, E.zt);
    if (s) return s;
    for (int b = 0; b < BT->B; ++b) E.h_active[b] = 1;
    BK(evalset_run(E, &BT->stats), "evaluation");
    scvt_status first = SCVT_OK;
    for (int b = 0; b < BT->B; ++b) {
        energy[b] = E.h_ist[b].red[0];
        scvt_status sb = status_of_flags(E.h_ist[b].flags);
        if (sb && !first) {
            first = sb;
            BT->err = "problem " + std::to_string(b) + ": " + scvt_status_string(sb);
        }
    }
    if (grad) {
        if ((s = copy_to_caller(BT, grad, E.gt, n3))) return s;
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
    if (lane_options(opts_in, &o) || o.warm_start < 0 || o.warm_start > 1)
        return bfail(BT, SCVT_ERR_INVALID, "bad solve options");
    enter(BT);
    const size_t n3 = 3 * (size_t)BT->ntot;
    bool resume = o.warm_start == 1 && BT->solved_once;
    for (Lane &L : BT->lanes) resume = resume && L.state_valid;
    std::vector<Lane *> lanes;
    for (Lane &L : BT->lanes) {
        memset(&L.rep, 0, sizeof(L.rep));
        L.opt = o;
        L.done = false;
        L.need_init = !resume;
        lanes.push_back(&L);
    }
    scvt_status st;
    if (!resume && (st = copy_in(BT, z, n3, BT->z))) return st;
    for (;;) {
        bool any = false;
        for (Lane *L : lanes) any = any || !L->done;
        if (!any) break;
        BK(lockstep_round(BT->E, lanes, BT->m, &BT->stats), "lockstep iteration");
    }
    scvt_status ret = SCVT_OK;
    for (int b = 0; b < BT->B; ++b) {
        Lane &L = BT->lanes[b];
        if (L.rep.status == SCVT_OK || L.rep.status == SCVT_ERR_LINESEARCH) {
            L.rep.energy = L.F;
            L.rep.grad_norm = L.gnorm;
        }
        reports[b] = L.rep;
        if (L.rep.status == SCVT_ERR_LINESEARCH && ret == SCVT_OK) ret = SCVT_ERR_LINESEARCH;
        if (L.rep.status != SCVT_OK && L.rep.status != SCVT_ERR_LINESEARCH &&
            (ret == SCVT_OK || ret == SCVT_ERR_LINESEARCH)) {
            ret = (scvt_status)L.rep.status;
            BT->err = "problem " + std::to_string(b) + ": " + scvt_status_string(ret);
        }
    }
    if ((st = copy_to_caller(BT, z, BT->z, n3))) return st;
    BK(cudaStreamSynchronize(BT->stream), "copy out");
    BT->solved_once = true;
    if (ret == SCVT_OK) BT->err.clear();
    return ret;
}

scvt_status scvt_batch_set_tuning(scvt_batch *BT, const scvt_tuning *t) {
    if (!BT) return SCVT_ERR_INVALID;
    if (!t) return bfail(BT, SCVT_ERR_INVALID, "null argument");
    Tune u;
    if (tune_from(*t, &u)) return bfail(BT, SCVT_ERR_INVALID, "tuning out of range");
    BK(evalset_set_tune(BT->E, u), "tuning");
    return SCVT_OK;
}

scvt_status scvt_batch_get_tuning(const scvt_batch *BT, scvt_tuning *t) {
    if (!BT || !t) return SCVT_ERR_INVALID;
    *t = tuning_of(BT->E.tune);
    return SCVT_OK;
}

scvt_status scvt_batch_tune(scvt_batch *BT, const double *z, scvt_tuning *chosen) {
    if (!BT) return SCVT_ERR_INVALID;
    if (!z) return bfail(BT, SCVT_ERR_INVALID, "null argument");
    enter(BT);
    EvalSet &E = BT->E;
    scvt_status s = copy_in(BT, z, 3 * (size_t)BT->ntot, E.zt);
    if (s) return s;
    for (int b = 0; b < BT->B; ++b) E.h_active[b] = 1;
    // one evaluation leaves radius hints for the warm timings; it must succeed
    BK(evalset_run(E, &BT->stats), "evaluation");
    for (int b = 0; b < BT->B; ++b)
        if ((s = status_of_flags(E.h_ist[b].flags))) return bfail(BT, s, "tuning input is not a valid batch");
    auto time_cfg = [&](const Tune &u, bool cold, float *ms) -> scvt_status {
        BK(evalset_time(E, u, cold, ms, &BT->stats), "timed evaluation");
        return SCVT_OK;
    };
    Tune best;
    if ((s = autotune(E.tune, time_cfg, &best))) return s;
    BK(evalset_set_tune(E, best), "tuning");
    // leave warm hints for the chosen configuration
    BK(evalset_run(E, &BT->stats), "evaluation");
    if (chosen) *chosen = tuning_of(best);
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
