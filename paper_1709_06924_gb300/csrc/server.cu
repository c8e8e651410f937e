// server.cu -- continuous batching of solve requests (include/scvt.h,
// "Serving").
//
// Jobs wait in a FIFO queue.  A step admits queued jobs in order while the
// memory budget (workspace + every running job's resident buffers), the
// workspace rows (sum of N) and the job slots allow; a job's iterate,
// gradient, preconditioner, LBFGS history and radius hints are allocated at
// admission (stream-ordered) and stay on the device until it retires.  The
// running jobs are laid out in the shared evaluation workspace (evalset.cuh)
// in admission order; when the set changes the layout is rebuilt (the
// radius hints follow their jobs) and the evaluation graph is re-captured.
// Every step then advances all running jobs by one LBFGS iteration with the
// lockstep solver (lockstep.cuh): new jobs get their first evaluation in the
// same evaluation round as the others' trial points.  Jobs that stopped are
// retired: their generators go back to host memory and their device memory
// returns to the budget.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "evalset.cuh"
#include "lockstep.cuh"

using namespace scvt;

namespace {

struct Job {
    int64_t id = 0;
    int n = 0;
    scvt_density rho;
    int state = SCVT_JOB_QUEUED;
    double t_submit = -1.0, t_admit = -1.0, t_done = -1.0;
    std::vector<double> z_host;  // the start until admission, the result after retirement
    int64_t bytes = 0;
    void *block = nullptr;       // one device allocation for the resident buffers
    float *hints = nullptr;
    Lane lane;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// device bytes of a job's resident buffers: z, g (3n), h (n), (m+1) history
// slots of S and Y (3n each), 1/(y.s) per slot, radius hints (n floats)
size_t job_bytes(int64_t n, int m) {
    const size_t n3 = 3 * (size_t)n;
    return align256(8 * n3) * 2 + align256(8 * (size_t)n) + align256(8 * (size_t)(m + 1) * 2 * n3) +
           align256(8 * kLaneRho) + align256(4 * (size_t)n);
}

bool dev_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

struct scvt_server {
    scvt_server_config cfg;
    cudaStream_t ustream = nullptr, stream = nullptr;
    cudaEvent_t ev_in = nullptr;
    EvalSet E;
    int64_t ws_bytes = 0, budget = 0, resident = 0, active_n = 0;
    std::vector<std::unique_ptr<Job>> jobs;  // by id
    std::deque<int64_t> queue;
    std::vector<int64_t> running;            // layout order
    std::vector<int64_t> laid_out;           // jobs in the current layout, in order
    bool relayout = false;
    std::chrono::steady_clock::time_point t0;
    scvt_stats stats;
    std::string err;
};

namespace {

scvt_status sfail(scvt_server *S, scvt_status s, const std::string &msg) {
    if (S) S->err = msg;
    return s;
}

scvt_status scuda(scvt_server *S, cudaError_t e, const char *what) {
    cudaGetLastError();
    return sfail(S, e == cudaErrorMemoryAllocation ? SCVT_ERR_OOM : SCVT_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

#define SK(call, what)                                    \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return scuda(S, e_, what); \
    } while (0)

double now(const scvt_server *S) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - S->t0).count();
}

bool valid_density(const scvt_density &r) {
    if (r.kind < 0 || r.kind > 3) return false;
    if (r.kind == SCVT_RHO_UNIFORM) return true;
    if (!(r.gamma > 0.0) || !(r.gamma <= 1.0)) return false;
    if (r.kind >= 2) {
        const double l = sqrt(r.xc[0] * r.xc[0] + r.xc[1] * r.xc[1] + r.xc[2] * r.xc[2]);
        if (!(fabs(l - 1.0) < 1e-9) || !(r.alpha > 0.0)) return false;
    }
    return true;
}

// admit queued jobs in order while they fit
scvt_status admit(scvt_server *S) {
    const int m = S->cfg.lbfgs_m;
    while (!S->queue.empty()) {
        Job &J = *S->jobs[S->queue.front()];
        if ((int)S->running.size() >= S->cfg.max_jobs) break;
        if (S->active_n + J.n > S->cfg.max_generators) break;
        if (S->ws_bytes + S->resident + J.bytes > S->budget) break;
        SK(cudaMallocAsync(&J.block, J.bytes, S->stream), "job buffers");
        const size_t n = (size_t)J.n, n3 = 3 * n;
        char *p = (char *)J.block;
        Lane &L = J.lane;
        L.z = (double *)p;
        p += align256(8 * n3);
        L.g = (double *)p;
        p += align256(8 * n3);
        L.h = (double *)p;
        p += align256(8 * n);
        L.hist = (double *)p;
        p += align256(8 * (size_t)(m + 1) * 2 * n3);
        L.rho = (double *)p;
        p += align256(8 * kLaneRho);
        J.hints = (float *)p;
        L.n = J.n;
        L.slot_stride = 2 * n3;
        L.y_off = n3;
        L.need_init = true;
        L.done = false;
        memset(&L.rep, 0, sizeof(L.rep));
        SK(cudaMemcpyAsync(L.z, J.z_host.data(), sizeof(double) * n3, cudaMemcpyHostToDevice, S->stream), "job start");
        SK(cudaMemsetAsync(J.hints, 0, sizeof(float) * n, S->stream), "job hints");
        SK(cudaStreamSynchronize(S->stream), "admission");
        std::vector<double>().swap(J.z_host);
        J.state = SCVT_JOB_RUNNING;
        J.t_admit = now(S);
        S->running.push_back(J.id);
        S->resident += J.bytes;
        S->active_n += J.n;
        S->queue.pop_front();
        S->relayout = true;
    }
    return SCVT_OK;
}

// lay the running jobs out in the workspace; radius hints follow their jobs
scvt_status lay_out(scvt_server *S) {
    EvalSet &E = S->E;
    for (int64_t id : S->laid_out) {
        Job &J = *S->jobs[id];
        if (J.state != SCVT_JOB_RUNNING) continue;
        SK(cudaMemcpyAsync(J.hints, E.radius + J.lane.row, sizeof(float) * J.n, cudaMemcpyDeviceToDevice, S->stream),
           "save hints");
    }
    const int B = (int)S->running.size();
    std::vector<int> ns(B);
    std::vector<scvt_density> rhos(B);
    for (int k = 0; k < B; ++k) {
        const Job &J = *S->jobs[S->running[k]];
        ns[k] = J.n;
        rhos[k] = J.rho;
    }
    SK(evalset_layout(E, B, ns.data(), rhos.data()), "layout");
    int64_t row = 0;
    for (int k = 0; k < B; ++k) {
        Job &J = *S->jobs[S->running[k]];
        J.lane.b = k;
        J.lane.row = row;
        SK(cudaMemcpyAsync(E.radius + row, J.hints, sizeof(float) * J.n, cudaMemcpyDeviceToDevice, S->stream),
           "load hints");
        row += J.n;
    }
    SK(cudaStreamSynchronize(S->stream), "layout");
    S->laid_out = S->running;
    S->relayout = false;
    return SCVT_OK;
}

scvt_status retire(scvt_server *S) {
    std::vector<int64_t> keep;
    for (int64_t id : S->running) {
        Job &J = *S->jobs[id];
        Lane &L = J.lane;
        if (!L.done) {
            keep.push_back(id);
            continue;
        }
        if (L.rep.status == SCVT_OK || L.rep.status == SCVT_ERR_LINESEARCH) {
            L.rep.energy = L.F;
            L.rep.grad_norm = L.gnorm;
            J.state = SCVT_JOB_DONE;
        } else {
            J.state = SCVT_JOB_FAILED;
        }
        J.z_host.resize(3 * (size_t)J.n);
        SK(cudaMemcpyAsync(J.z_host.data(), L.z, sizeof(double) * 3 * J.n, cudaMemcpyDeviceToHost, S->stream),
           "job result");
        SK(cudaFreeAsync(J.block, S->stream), "job buffers");
        SK(cudaStreamSynchronize(S->stream), "retire");
        J.block = nullptr;
        J.t_done = now(S);
        S->resident -= J.bytes;
        S->active_n -= J.n;
        S->relayout = true;
    }
    S->running.swap(keep);
    return SCVT_OK;
}

}  // namespace

extern "C" {

void scvt_server_destroy(scvt_server *S) {
    if (!S) return;
    if (S->stream) cudaStreamSynchronize(S->stream);
    for (auto &J : S->jobs)
        if (J && J->block) cudaFreeAsync(J->block, S->stream);
    if (S->stream) cudaStreamSynchronize(S->stream);
    evalset_free(S->E);
    if (S->ev_in) cudaEventDestroy(S->ev_in);
    if (S->stream) cudaStreamDestroy(S->stream);
    delete S;
}

scvt_status scvt_server_create(const scvt_server_config *cfg, void *cuda_stream, scvt_server **out) {
    if (!cfg || !out) return SCVT_ERR_INVALID;
    *out = nullptr;
    if (cfg->max_jobs < 1 || cfg->max_jobs > 65535) return SCVT_ERR_INVALID;
    if (cfg->max_generators < 4 || cfg->max_generators > (int64_t)200000000) return SCVT_ERR_INVALID;
    if (cfg->precision < 0 || cfg->precision > 2) return SCVT_ERR_INVALID;
    if (cfg->lbfgs_m < 0 || cfg->lbfgs_m > kLaneMaxM) return SCVT_ERR_INVALID;
    if (cfg->memory_budget < 0) return SCVT_ERR_INVALID;
    const int64_t ws = evalset_bytes(cfg->max_generators, cfg->max_jobs, cfg->precision);
    int64_t budget = cfg->memory_budget;
    if (budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            return SCVT_ERR_CUDA;
        }
        budget = (int64_t)(0.8 * (double)fr);
    }
    if (ws >= budget) return SCVT_ERR_INVALID;
    scvt_server *S = new (std::nothrow) scvt_server();
    if (!S) return SCVT_ERR_OOM;
    S->cfg = *cfg;
    S->budget = budget;
    S->ustream = (cudaStream_t)cuda_stream;
    S->t0 = std::chrono::steady_clock::now();
    memset(&S->stats, 0, sizeof(S->stats));
    cudaError_t e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&S->ev_in);
    if (e == cudaSuccess) e = evalset_alloc(S->E, cfg->max_generators, cfg->max_jobs, cfg->precision, S->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        scvt_server_destroy(S);
        return e == cudaErrorMemoryAllocation ? SCVT_ERR_OOM : SCVT_ERR_CUDA;
    }
    S->ws_bytes = std::max<int64_t>(ws, S->E.bytes);
    *out = S;
    return SCVT_OK;
}

scvt_status scvt_server_submit(scvt_server *S, int64_t n, const scvt_density *rho, const double *z0,
                               const scvt_solve_opts *opts, int64_t *job_id) {
    if (!S) return SCVT_ERR_INVALID;
    if (!rho || !z0 || !job_id) return sfail(S, SCVT_ERR_INVALID, "null argument");
    if (n < 4 || n > S->cfg.max_generators) return sfail(S, SCVT_ERR_INVALID, "job size outside 4..max_generators");
    if (!valid_density(*rho)) return sfail(S, SCVT_ERR_INVALID, "bad density");
    scvt_solve_opts o;
    if (lane_options(opts, &o) || o.warm_start != 0) return sfail(S, SCVT_ERR_INVALID, "bad solve options");
    const size_t bytes = job_bytes(n, S->cfg.lbfgs_m);
    if (S->ws_bytes + (int64_t)bytes > S->budget) return sfail(S, SCVT_ERR_INVALID, "job exceeds the memory budget");
    std::unique_ptr<Job> J(new (std::nothrow) Job());
    if (!J) return sfail(S, SCVT_ERR_OOM, "host memory");
    J->id = (int64_t)S->jobs.size();
    J->n = (int)n;
    J->rho = *rho;
    J->bytes = (int64_t)bytes;
    J->lane.opt = o;
    J->z_host.resize(3 * (size_t)n);
    cudaEventRecord(S->ev_in, S->ustream);
    cudaStreamWaitEvent(S->stream, S->ev_in, 0);
    SK(cudaMemcpyAsync(J->z_host.data(), z0, sizeof(double) * 3 * n,
                       dev_ptr(z0) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, S->stream),
       "job start");
    SK(cudaStreamSynchronize(S->stream), "job start");
    J->t_submit = now(S);
    *job_id = J->id;
    S->queue.push_back(J->id);
    S->jobs.push_back(std::move(J));
    return SCVT_OK;
}

scvt_status scvt_server_step(scvt_server *S, int *running, int *queued) {
    if (!S) return SCVT_ERR_INVALID;
    cudaEventRecord(S->ev_in, S->ustream);
    cudaStreamWaitEvent(S->stream, S->ev_in, 0);
    scvt_status s = admit(S);
    if (s) return s;
    if (!S->running.empty()) {
        if (S->relayout && (s = lay_out(S))) return s;
        std::vector<Lane *> lanes;
        for (int64_t id : S->running) lanes.push_back(&S->jobs[id]->lane);
        SK(lockstep_round(S->E, lanes, S->cfg.lbfgs_m, &S->stats), "lockstep iteration");
        if ((s = retire(S))) return s;
    }
    if (running) *running = (int)S->running.size();
    if (queued) *queued = (int)S->queue.size();
    S->err.clear();
    return SCVT_OK;
}

scvt_status scvt_server_job(const scvt_server *S, int64_t id, scvt_job_info *info) {
    if (!S || !info || id < 0 || id >= (int64_t)S->jobs.size()) return SCVT_ERR_INVALID;
    const Job &J = *S->jobs[id];
    memset(info, 0, sizeof(*info));
    info->state = J.state;
    info->n = J.n;
    info->t_submit = J.t_submit;
    info->t_admit = J.t_admit;
    info->t_done = J.t_done;
    info->bytes_resident = J.bytes;
    info->report = J.lane.rep;
    return SCVT_OK;
}

scvt_status scvt_server_fetch(scvt_server *S, int64_t id, double *z_out) {
    if (!S) return SCVT_ERR_INVALID;
    if (!z_out || id < 0 || id >= (int64_t)S->jobs.size()) return sfail(S, SCVT_ERR_INVALID, "bad argument");
    Job &J = *S->jobs[id];
    if (J.state != SCVT_JOB_DONE && J.state != SCVT_JOB_FAILED) return sfail(S, SCVT_ERR_INVALID, "job not finished");
    SK(cudaMemcpyAsync(z_out, J.z_host.data(), sizeof(double) * 3 * J.n,
                       dev_ptr(z_out) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, S->stream),
       "fetch");
    SK(cudaStreamSynchronize(S->stream), "fetch");
    std::vector<double>().swap(J.z_host);
    J.state = SCVT_JOB_FETCHED;
    return SCVT_OK;
}

double scvt_server_clock(const scvt_server *S) { return S ? now(S) : 0.0; }

scvt_status scvt_server_get_stats(const scvt_server *S, scvt_stats *out) {
    if (!S || !out) return SCVT_ERR_INVALID;
    *out = S->stats;
    out->bytes_device = S->ws_bytes + S->resident;
    return SCVT_OK;
}

const char *scvt_server_last_error(const scvt_server *S) { return S ? S->err.c_str() : ""; }

}  // extern "C"
