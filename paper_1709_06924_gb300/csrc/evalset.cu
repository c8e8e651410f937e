// evalset.cu -- evaluation workspace of batches and the server (see evalset.cuh).
#include <math.h>
#include <string.h>

#include <algorithm>

#include "evalset.cuh"

namespace scvt {

namespace {

template <class T>
cudaError_t ealloc(EvalSet &E, T **p, size_t count) {
    size_t bytes = sizeof(T) * (count ? count : 1);
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e == cudaSuccess) E.bytes += (int64_t)bytes;
    return e;
}

// bins of the finest adapted resolution (max_bins_per_edge: twice the bins per
// edge of one generator per bin) over at most cap_b problems of cap_n
// generators in total: sum 6 (2 ceil(sqrt(n_b/6)))^2 <= 4 (cap_n + 2 sqrt(6
// cap_n cap_b) + 6 cap_b)
size_t max_bins(int64_t cap_n, int cap_b) {
    return 4 * ((size_t)cap_n + (size_t)(2.0 * sqrt(6.0 * (double)cap_n * (double)cap_b)) + 6 * (size_t)cap_b) + 64;
}

size_t max_partials(int64_t cap_n, int cap_b) { return 4 * ((size_t)cap_n / 4096 + (size_t)cap_b + 1024); }

// chunk sums of the segmented LBFGS kernels: per problem max(kCmpQ nb3,
// 4 nb1) <= kCmpQ (3n/4096 + 1) + 4 (n/4096 + 1), nb3 = reduce_blocks(3n),
// nb1 = reduce_blocks(n)
size_t max_seg_partials(int64_t cap_n, int cap_b) {
    return (3 * kCmpQ + 4) * ((size_t)cap_n / 4096) + (kCmpQ + 4) * (size_t)cap_b + 64 + 3 * kCmpQ + 4;
}

// density-table pool: the tables of any layout of at most cap_b problems with
// cap_n generators in all fit (sum of 8 sqrt(n_b) <= 8 sqrt(cap_n cap_b), plus
// the 1,024-centre minimum per problem), capped at 1 GiB; a problem whose
// table does not fit evaluates its density directly
size_t tab_pool_size(int64_t cap_n, int cap_b) {
    const double centres = 8.0 * sqrt((double)cap_n * (double)cap_b) + 1024.0 * cap_b + 32768.0;
    const double bytes = centres * (double)dens_table_bytes(1024) / 1024.0 + 1024.0 * cap_b;
    return (size_t)std::min(bytes, (double)(1ull << 30));
}

// problem of every row, by binary search over the problems' first rows
__global__ void k_fill_pinst(const InstGeom *__restrict__ inst, int B, int *__restrict__ pinst, int ntot) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ntot) return;
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (inst[mid].p0 <= i) lo = mid;
        else hi = mid - 1;
    }
    pinst[i] = lo;
}

Grid make_grid(const EvalSet &E) {
    Grid g;
    memset(&g, 0, sizeof(g));
    g.n = (int)E.ntot;
    g.G = E.geom.empty() ? 1 : E.geom[0].G;
    g.nbins = E.nbins;
    g.zs = E.zs;
    g.zf = E.zf;
    g.zl = E.zl;
    g.zll = E.precision != 1 ? E.zll : nullptr;  // not computed in the mixed form
    g.sidx = E.sidx;
    g.bstart = E.start;
    g.inst = E.d_inst;
    g.pinst = E.d_pinst;
    g.rho = E.d_rho;
    g.rhof = E.d_rhof;
    g.rhodf = E.d_rhodf;
    g.tabs = E.precision != 1 ? E.d_tabs : nullptr;
    g.ist = E.d_ist;
    g.active = E.d_active;
    g.nprob = E.B;
    g.fan = E.fan;
    return g;
}

void enqueue_eval(EvalSet &E, int64_t *launches, int64_t *cell_launches) {
    cudaStream_t s = E.stream;
    cudaMemsetAsync(E.d_st, 0, sizeof(DevStatus), s);
    cudaMemsetAsync(E.d_ist, 0, sizeof(DevStatus) * E.B, s);
    Grid g = make_grid(E);
    bin_points(E.zt, g, E.bin_of, E.count, E.start, E.cursor, E.scan_tmp, E.zs, E.zf, E.zl, E.precision != 1 ? E.zll : nullptr, E.sidx, E.radius, E.d_st,
               s, launches);
    CellOut out;
    memset(&out, 0, sizeof(out));
    out.grad = E.gt;
    out.hdiag = E.ht;
    out.fcell = E.fc;
    out.radius = E.radius;
    CellBuf cb;
    cb.deg = E.cdeg;
    cb.vx = E.cvx;
    cb.nb = E.cnb;
    cb.eoff = E.eoff;
    cb.ecell = E.ecell;
    cb.scan_tmp = E.escan;
    cb.eacc = E.eacc;
    cb.vo = E.vo;
    cb.ctab = E.ctab;
    cell_passes(g, out, cb, E.list1, E.list2, E.d_st, E.precision, E.tune, s, nullptr, nullptr, launches,
                cell_launches, &E.pipes);
    reduce_eval_batch(E.B, E.max_nb, E.d_inst, E.d_pbase, E.d_active, E.fc, E.gt, E.q, E.nrm, E.partials, E.d_ist, s,
                      launches);
    cudaMemcpyAsync(E.h_ist, E.d_ist, sizeof(DevStatus) * E.B, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(E.h_st, E.d_st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s);
}

cudaError_t capture(EvalSet &E) {
    if (E.graph) {
        cudaGraphExecDestroy(E.graph);
        E.graph = nullptr;
    }
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamBeginCapture(E.stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    int64_t l = 0, c = 0;
    enqueue_eval(E, &l, &c);
    e = cudaStreamEndCapture(E.stream, &gr);
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&E.graph, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
        E.graph = nullptr;
        return e;
    }
    E.graph_launches = l;
    E.graph_cell_launches = c;
    return cudaSuccess;
}

cudaError_t rebin(EvalSet &E) {
    int bin0 = 0;
    for (int b = 0; b < E.B; ++b) {
        const int G = E.gsel[b] > 0 ? E.gsel[b] : bins_per_edge(E.geom[b].n, E.tune.bin_load);
        E.geom[b].G = G;
        E.geom[b].bin0 = bin0;
        bin0 += 6 * G * G;
    }
    E.nbins = bin0;
    if (E.graph) {
        cudaGraphExecDestroy(E.graph);
        E.graph = nullptr;
    }
    if (E.B == 0) return cudaSuccess;
    cudaError_t e =
        cudaMemcpyAsync(E.d_inst, E.geom.data(), sizeof(InstGeom) * E.B, cudaMemcpyHostToDevice, E.stream);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(E.stream);
}

}  // namespace

scvt_status status_of_flags(unsigned f) {
    if (f & (FLAG_BAD_POINT | FLAG_DUPLICATE)) return SCVT_ERR_INVALID;
    if (f & (FLAG_UNBOUNDED | FLAG_EMPTY)) return SCVT_ERR_DEGENERATE;
    if (f & (FLAG_EXHAUSTED | FLAG_VMAX)) return SCVT_ERR_KNN_EXHAUSTED;
    if (f & (FLAG_NONPOSITIVE | FLAG_ECAP)) return SCVT_ERR_DEGENERATE;
    return SCVT_OK;
}

int64_t evalset_bytes(int64_t cap_n, int cap_b, int precision) {
    const int64_t N = cap_n, nb = (int64_t)max_bins(cap_n, cap_b);
    int64_t per_row = 24 * 2 + 8 * 4 + 4      // zt, gt, q; ht, fc, nrm, (pinst); radius
                      + 32 + 48 + 16 * 32 + 16 * 4 + 4 + 4 + 24 + 240  // zs, zf+zl+zll, cvx, cnb, cdeg, eoff, ecell, eacc
                      + 4 * 4;                // bin_of, sidx, list1, list2
    if (precision == 1) per_row += 16 * 16;   // vo
    if (precision == 0) per_row += 16;        // ctab
    const int64_t tabs = precision != 1 ? (int64_t)tab_pool_size(cap_n, cap_b) + (int64_t)cap_b * (int64_t)sizeof(DensTab) : 0;
    const int64_t seg = (int64_t)cap_b * (int64_t)(sizeof(SegLane) + 8 * kTwoLoopScratch) +
                        8 * (int64_t)max_seg_partials(cap_n, cap_b);
    return N * per_row + nb * 12 + (int64_t)max_partials(cap_n, cap_b) * 8 + (int64_t)cap_b * 512 + tabs + seg +
           (1 << 20);
}

cudaError_t evalset_alloc(EvalSet &E, int64_t cap_n, int cap_b, int precision, cudaStream_t s) {
    E.cap_n = cap_n;
    E.cap_b = cap_b;
    E.precision = precision;
    E.stream = s;
    const size_t N = (size_t)cap_n, n3 = 3 * N, nb = max_bins(cap_n, cap_b);
    E.partials_len = max_partials(cap_n, cap_b);
    cudaError_t e = cudaSuccess;
#define AL(ptr, cnt) \
    if (e == cudaSuccess) e = ealloc(E, &(ptr), (cnt))
    AL(E.d_inst, cap_b); AL(E.d_pinst, N); AL(E.d_pbase, cap_b); AL(E.d_active, cap_b);
    AL(E.d_rho, cap_b); AL(E.d_rhof, cap_b); AL(E.d_rhodf, cap_b); AL(E.d_ist, cap_b); AL(E.d_st, 1);
    AL(E.zt, n3); AL(E.gt, n3); AL(E.ht, N); AL(E.fc, N); AL(E.q, n3); AL(E.nrm, N); AL(E.radius, N);
    AL(E.partials, E.partials_len);
    E.seg_partials_len = max_seg_partials(cap_n, cap_b);
    AL(E.d_seg, cap_b); AL(E.seg_partials, E.seg_partials_len); AL(E.seg_scal, (size_t)cap_b * kTwoLoopScratch);
    AL(E.zs, N); AL(E.zf, N); AL(E.zl, N); AL(E.zll, N); AL(E.cvx, N * kCellSlots); AL(E.cnb, N * kCellSlots);
    AL(E.cdeg, N); AL(E.eoff, N + 1); AL(E.ecell, 6 * N); AL(E.escan, scan_tmp_ints(N));
    AL(E.eacc, 5 * 6 * N);
    if (precision == 1) AL(E.vo, N * kCellSlots);
    if (precision == 0) AL(E.ctab, N);
    if (precision != 1) {
        E.tab_pool_bytes = tab_pool_size(cap_n, cap_b);
        AL(E.d_tabs, cap_b);
        if (e == cudaSuccess) e = ealloc(E, (unsigned char **)&E.tab_pool, E.tab_pool_bytes);
    }
    AL(E.bin_of, N); AL(E.count, nb); AL(E.start, nb + 1); AL(E.cursor, nb); AL(E.scan_tmp, 2 * (nb / 2048 + 64) + 64);
    AL(E.sidx, N); AL(E.list1, N); AL(E.list2, N);
#undef AL
    if (e == cudaSuccess) e = pipes_create(E.pipes, kMaxChunks - 1);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&E.h_ist, sizeof(DevStatus) * cap_b);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&E.h_st, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&E.h_active, sizeof(int) * cap_b);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&E.h_seg, sizeof(SegLane) * cap_b);
    // the segmented kernels' ticket counters start at 0 (each pass's last block resets its own)
    if (e == cudaSuccess) e = cudaMemsetAsync(E.seg_scal, 0, sizeof(double) * cap_b * kTwoLoopScratch, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(E.radius, 0, sizeof(float) * N, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(E.q, 0, sizeof(double) * n3, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(E.nrm, 0, sizeof(double) * N, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

void evalset_free(EvalSet &E) {
    if (E.graph) cudaGraphExecDestroy(E.graph);
    E.graph = nullptr;
    void *ptrs[] = {E.d_inst, E.d_pinst, E.d_pbase, E.d_active, E.d_rho, E.d_rhof, E.d_rhodf, E.d_ist, E.d_st, E.zt, E.gt,
                    E.ht, E.fc, E.q, E.nrm, E.radius, E.partials, E.zs, E.zf, E.zl, E.zll, E.cvx, E.cnb, E.cdeg, E.eoff,
                    E.ecell, E.escan, E.eacc, E.vo, E.ctab, E.tab_pool, E.d_tabs, E.d_seg, E.seg_partials, E.seg_scal, E.bin_of, E.count, E.start, E.cursor, E.scan_tmp, E.sidx,
                    E.list1, E.list2};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    void *hp[] = {E.h_ist, E.h_st, E.h_active, E.h_seg};
    for (void *p : hp)
        if (p) cudaFreeHost(p);
    pipes_destroy(E.pipes);
    E = EvalSet();
}

cudaError_t evalset_layout(EvalSet &E, int B, const int *ns, const scvt_density *rhos) {
    if (B < 0 || B > E.cap_b) return cudaErrorInvalidValue;
    int64_t ntot = 0;
    for (int b = 0; b < B; ++b) ntot += ns[b];
    if (ntot > E.cap_n) return cudaErrorInvalidValue;
    E.B = B;
    E.ntot = ntot;
    E.geom.resize(B);
    E.pbase.resize(B);
    E.max_nb = 1;
    E.gsel.assign(B, 0);
    E.tabs.assign(B, DensTab{});
    std::vector<Density> rho(B);
    std::vector<DensityF> rhof(B);
    std::vector<DensDF> rhodf(B);
    int64_t off = 0, nbt = 0;
    for (int b = 0; b < B; ++b) {
        E.geom[b].p0 = (int)off;
        E.geom[b].n = ns[b];
        const int nb = reduce_blocks(ns[b]);
        E.pbase[b] = (int)nbt;
        nbt += nb;
        E.max_nb = std::max(E.max_nb, nb);
        rho[b] = to_device_density(rhos[b]);
        rhof[b] = to_density32(rho[b]);
        rhodf[b] = dens_df(rho[b]);
        off += ns[b];
    }
    if (B == 0) return cudaSuccess;
    cudaError_t e = rebin(E);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(E.d_rho, rho.data(), sizeof(Density) * B, cudaMemcpyHostToDevice, E.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(E.d_rhof, rhof.data(), sizeof(DensityF) * B, cudaMemcpyHostToDevice, E.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(E.d_rhodf, rhodf.data(), sizeof(DensDF) * B, cudaMemcpyHostToDevice, E.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(E.d_pbase, E.pbase.data(), sizeof(int) * B, cudaMemcpyHostToDevice, E.stream);
    // each problem's density table, laid out in the pool in problem order
    if (E.precision != 1) {
        size_t used = 0;
        for (int b = 0; b < B && e == cudaSuccess; ++b) {
            if (rho[b].kind < 2) continue;
            const int M = dens_table_centres(ns[b]);
            const size_t need = dens_table_bytes(M);
            if (used + need > E.tab_pool_bytes) continue;  // direct evaluation
            e = dens_table_build(rho[b], M, (unsigned char *)E.tab_pool + used, &E.tabs[b], E.stream);
            used += need;
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(E.d_tabs, E.tabs.data(), sizeof(DensTab) * B, cudaMemcpyHostToDevice, E.stream);
    }
    if (e == cudaSuccess && ntot > 0)
        k_fill_pinst<<<(unsigned)((ntot + 255) / 256), 256, 0, E.stream>>>(E.d_inst, B, E.d_pinst, (int)ntot);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(E.stream);
    return e;
}

cudaError_t evalset_set_tune(EvalSet &E, const Tune &t) {
    E.tune = t;
    E.gsel.assign(E.B, 0);
    return rebin(E);
}

cudaError_t evalset_run(EvalSet &E, scvt_stats *stats) {
    Phase ph("scvt batch evaluate");
    cudaError_t e;
    if (!E.graph && (e = capture(E)) != cudaSuccess) return e;
    e = cudaMemcpyAsync(E.d_active, E.h_active, sizeof(int) * E.B, cudaMemcpyHostToDevice, E.stream);
    if (e == cudaSuccess) e = cudaGraphLaunch(E.graph, E.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(E.stream);
    if (e != cudaSuccess) return e;
    // an edge list overflow is global: every evaluated problem reports it
    if (E.h_st->flags & FLAG_ECAP)
        for (int b = 0; b < E.B; ++b)
            if (E.h_active[b]) E.h_ist[b].flags |= FLAG_ECAP;
    // bins refined (or relaxed) where an evaluated problem's generators
    // concentrate; a change re-lays the bins out and drops the graph
    bool rebinned = false;
    for (int b = 0; b < E.B; ++b) {
        if (!E.h_active[b]) continue;
        const int n = E.geom[b].n;
        const int G = adapt_bins(bins_per_edge(n, E.tune.bin_load), E.geom[b].G, max_bins_per_edge(n),
                                 E.h_ist[b].max_bin, E.tune.bin_load);
        if (G != E.geom[b].G) {
            E.gsel[b] = G;
            rebinned = true;
        }
    }
    if (rebinned && (e = rebin(E)) != cudaSuccess) return e;
    if (stats) {
        stats->evaluations++;
        stats->kernel_launches += E.graph_launches;
        stats->cell_launches += E.graph_cell_launches;
        stats->knn_retries += E.h_st->retry_count[0];
        stats->ambiguous += (int64_t)E.h_st->ambiguous;
        stats->series_edges += (int64_t)E.h_st->ser_edges;
        stats->series_terms += (int64_t)E.h_st->ser_terms;
    }
    return cudaSuccess;
}

cudaError_t evalset_time(EvalSet &E, const Tune &u, bool cold, float *ms, scvt_stats *stats) {
    cudaError_t e = evalset_set_tune(E, u);
    if (e != cudaSuccess) return e;
    if ((e = capture(E)) != cudaSuccess) return e;
    cudaEvent_t a, b;
    if ((e = cudaEventCreate(&a)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&b)) != cudaSuccess) {
        cudaEventDestroy(a);
        return e;
    }
    float best = INFINITY;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        if (cold) e = cudaMemsetAsync(E.radius, 0, sizeof(float) * E.ntot, E.stream);
        if (e == cudaSuccess) e = cudaEventRecord(a, E.stream);
        if (e == cudaSuccess) e = evalset_run(E, stats);
        if (e == cudaSuccess) e = cudaEventRecord(b, E.stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float t = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
        if (e == cudaSuccess) best = std::min(best, t);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ms = best;
    return e;
}

}  // namespace scvt
