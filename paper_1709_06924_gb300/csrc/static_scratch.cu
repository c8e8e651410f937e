// static_scratch.cu -- energy and gradient without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need an
// evaluation: code that runs inside a memory budget fixed up front (a
// pool owned by someone else, an allocator that must not be re-entered from
// a callback), or embedded hosts that forbid cudaMalloc after start-up.  This
// entry point serves them: it runs the same binning, topology, quadrature and
// reduction kernels as the handle-based API, but all of its scratch lives in
// one file-scope __device__ array of fixed size, present on every GPU that
// loads the library until the process exits.
//
// Limits and rules (also in include/scvt.h):
//   - N <= SCVT_STATIC_MAX_N (16,384); larger N is rejected with
//     SCVT_ERR_INVALID before any device work;
//   - the array's device address is looked up once per device (first call
//     on that device, with the device current) and kept for the life of the
//     process; make that first call before any stream capture, and do not
//     use this entry point on a device after cudaDeviceReset (the address
//     kept from before the reset is no longer valid);
//   - every call shares the one array and it keeps the last call's contents;
//     whatever must start at zero is cleared on the stream by each call.
//     Calls whose work overlaps on the GPU (other streams, other host
//     threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "scvt_internal.cuh"

using namespace scvt;

namespace {

constexpr int kMaxN = SCVT_STATIC_MAX_N;
constexpr int kMaxG = 37;  // ceil(sqrt(kMaxN / 12)): bins per face edge at kMaxN
constexpr int kMaxBins = 6 * kMaxG * kMaxG;
constexpr int kScanTmp = 2 * (kMaxBins / 2048 + 64) + 64;

constexpr size_t up(size_t x) { return (x + 255) & ~(size_t)255; }

// byte offsets of the regions inside the array
constexpr size_t oSt = 0;
constexpr size_t oPartials = oSt + up(sizeof(DevStatus));
constexpr size_t oCount = oPartials + up(sizeof(double) * 4 * 1024);
constexpr size_t oStart = oCount + up(sizeof(int) * kMaxBins);
constexpr size_t oCursor = oStart + up(sizeof(int) * (kMaxBins + 1));
constexpr size_t oScan = oCursor + up(sizeof(int) * kMaxBins);
constexpr size_t oBinOf = oScan + up(sizeof(int) * kScanTmp);
constexpr size_t oSidx = oBinOf + up(sizeof(int) * kMaxN);
constexpr size_t oList1 = oSidx + up(sizeof(int) * kMaxN);
constexpr size_t oList2 = oList1 + up(sizeof(int) * kMaxN);
constexpr size_t oCdeg = oList2 + up(sizeof(int) * kMaxN);
constexpr size_t oZs = oCdeg + up(sizeof(int) * kMaxN);
constexpr size_t oZf = oZs + up(sizeof(P4) * kMaxN);
constexpr size_t oZl = oZf + up(sizeof(float4) * kMaxN);
constexpr size_t oZll = oZl + up(sizeof(float4) * kMaxN);
constexpr size_t oCvx = oZll + up(sizeof(float4) * kMaxN);
constexpr size_t oCnb = oCvx + up(sizeof(P4) * kMaxN * kCellSlots);
constexpr size_t oFc = oCnb + up(sizeof(int) * kMaxN * kCellSlots);
constexpr size_t oH = oFc + up(sizeof(double) * kMaxN);
constexpr size_t oG = oH + up(sizeof(double) * kMaxN);
constexpr size_t oEoff = oG + up(sizeof(double) * 3 * kMaxN);
constexpr size_t oEcell = oEoff + up(sizeof(int) * (kMaxN + 1));
constexpr size_t oEscan = oEcell + up(sizeof(int) * 6 * kMaxN);
constexpr size_t oEacc = oEscan + up(sizeof(int) * (2 * (kMaxN / 2048 + 64) + 64));
constexpr size_t oCounts = oEacc + up(sizeof(double) * 5 * 6 * kMaxN);
constexpr size_t kBytes = oCounts + up(sizeof(unsigned) * 8 * kMaxChunks);  // about 16.4 MB

__device__ __align__(256) unsigned char g_scratch[kBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {nullptr};

// device address of g_scratch on the current device (looked up once per device)
cudaError_t scratch_address(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = (unsigned char *)p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

bool device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" scvt_status scvt_energy_grad_static(int64_t n, const scvt_density *rho, const double *z,
                                               void *cuda_stream, double *energy, double *grad, double *mass,
                                               double *moment) {
    if (!rho || !z || !energy) return SCVT_ERR_INVALID;
    if (n < 4 || n > kMaxN) return SCVT_ERR_INVALID;
    if (rho->kind < 0 || rho->kind > 3) return SCVT_ERR_INVALID;
    if (rho->kind != SCVT_RHO_UNIFORM) {
        if (!(rho->gamma > 0.0) || !(rho->gamma <= 1.0)) return SCVT_ERR_INVALID;
        if (rho->kind >= 2) {
            double r = sqrt(rho->xc[0] * rho->xc[0] + rho->xc[1] * rho->xc[1] + rho->xc[2] * rho->xc[2]);
            if (!(fabs(r - 1.0) < 1e-9) || !(rho->alpha > 0.0)) return SCVT_ERR_INVALID;
        }
    }
    if (!device_ptr(z) || (grad && !device_ptr(grad)) || (mass && !device_ptr(mass)) ||
        (moment && !device_ptr(moment)))
        return SCVT_ERR_INVALID;
    unsigned char *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) {
        cudaGetLastError();
        return SCVT_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int N = (int)n;
    const int G = (int)ceil(sqrt((double)N / 12.0));  // the handle API's bin resolution
    DevStatus *st = (DevStatus *)(base + oSt);
    double *partials = (double *)(base + oPartials);
    int *count = (int *)(base + oCount), *start = (int *)(base + oStart), *cursor = (int *)(base + oCursor);
    int *scan_tmp = (int *)(base + oScan), *bin_of = (int *)(base + oBinOf), *sidx = (int *)(base + oSidx);
    int *list1 = (int *)(base + oList1), *list2 = (int *)(base + oList2), *cdeg = (int *)(base + oCdeg);
    P4 *zs = (P4 *)(base + oZs);
    float4 *zf = (float4 *)(base + oZf);
    float4 *zl = (float4 *)(base + oZl);
    float4 *zll = (float4 *)(base + oZll);
    P4 *cvx = (P4 *)(base + oCvx);
    int *cnb = (int *)(base + oCnb);
    double *fc = (double *)(base + oFc), *hd = (double *)(base + oH);
    double *g = grad ? grad : (double *)(base + oG);

    int64_t launches = 0, cell_launches = 0;
    if (cudaMemsetAsync(st, 0, sizeof(DevStatus), s) != cudaSuccess) {
        cudaGetLastError();
        return SCVT_ERR_CUDA;
    }
    Grid grid;
    memset(&grid, 0, sizeof(grid));
    grid.n = N;
    grid.G = G;
    grid.nbins = 6 * G * G;
    grid.zs = zs;
    grid.zf = zf;
    grid.zl = zl;
    grid.zll = zll;
    grid.sidx = sidx;
    grid.bstart = start;
    grid.rho0 = to_device_density(*rho);
    grid.rho0f = to_density32(grid.rho0);
    bin_points(z, grid, bin_of, count, start, cursor, scan_tmp, zs, zf, zl, zll, sidx, nullptr, st, s, &launches);
    CellOut out;
    out.grad = g;
    out.hdiag = hd;
    out.mass = mass;
    out.moment = moment;
    out.fcell = fc;
    out.deg = nullptr;
    out.nbr = nullptr;
    out.max_deg = 0;
    out.radius = nullptr;
    CellBuf cb;
    cb.deg = cdeg;
    cb.vx = cvx;
    cb.nb = cnb;
    cb.eoff = (int *)(base + oEoff);
    cb.ecell = (int *)(base + oEcell);
    cb.scan_tmp = (int *)(base + oEscan);
    cb.eacc = (double *)(base + oEacc);
    cb.vo = nullptr;
    cb.ctab = nullptr;  // the density is evaluated directly (no table)
    Pipes px;  // one pipeline on the caller's stream, its counters in the scratch array
    px.counts = (unsigned *)(base + oCounts);
    cell_passes(grid, out, cb, list1, list2, st, 0, Tune(), s, nullptr, nullptr, &launches, &cell_launches, &px);
    reduce_eval(N, fc, g, nullptr, nullptr, partials, st, s, &launches);
    // a launch that failed (configuration, resources) leaves the status block
    // as it was cleared: report it instead of the energy
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return SCVT_ERR_CUDA;
    DevStatus hs;
    e = cudaMemcpyAsync(&hs, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SCVT_ERR_CUDA;
    }
    if (hs.flags & (FLAG_BAD_POINT | FLAG_DUPLICATE)) return SCVT_ERR_INVALID;
    if (hs.flags & (FLAG_UNBOUNDED | FLAG_EMPTY | FLAG_NONPOSITIVE | FLAG_ECAP)) return SCVT_ERR_DEGENERATE;
    if (hs.flags & (FLAG_EXHAUSTED | FLAG_VMAX)) return SCVT_ERR_KNN_EXHAUSTED;
    *energy = hs.red[0];
    return SCVT_OK;
}
