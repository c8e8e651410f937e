// sample.cu -- Monte Carlo initialisation by the density (include/scvt.h,
// scvt_sample_density).
//
// Candidate k (a point on S^2) is kept when u_k rho_max <= rho(cand_k), u_k
// uniform on [0, 1): the kept points are distributed with density
// proportional to rho (Sec. 4.1 initialises the serial tests this way).  The
// decision is one thread per candidate; the kept candidates keep their order
// (an exclusive scan gives each its slot) and the first n_target are written.
#include <cuda_runtime.h>
#include <math.h>

#include <climits>

#include "scvt_internal.cuh"

using namespace scvt;

namespace {

// rho^e: e = 1 and e = 1/2 exactly, pow otherwise
__host__ __device__ __forceinline__ double rho_pow(double v, double e) {
    return e == 1.0 ? v : (e == 0.5 ? sqrt(v) : pow(v, e));
}

__global__ void k_sample_flags(Density r, double e, double rmax, const double *__restrict__ cand,
                               const double *__restrict__ u, int m, int *__restrict__ flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const double v = rho_value(r, cand[3 * (size_t)i], cand[3 * (size_t)i + 1], cand[3 * (size_t)i + 2]);
    flag[i] = (u[i] * rmax <= rho_pow(v, e)) ? 1 : 0;
}

__global__ void k_sample_scatter(const double *__restrict__ cand, const int *__restrict__ flag,
                                 const int *__restrict__ pos, int m, long long n_target, double *__restrict__ out,
                                 long long *count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    if (flag[i] && pos[i] < n_target) {
        const size_t k = (size_t)pos[i];
        out[3 * k] = cand[3 * (size_t)i];
        out[3 * k + 1] = cand[3 * (size_t)i + 1];
        out[3 * k + 2] = cand[3 * (size_t)i + 2];
    }
    if (i == m - 1) *count = (long long)pos[i] + flag[i];
}

bool device_pointer(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// the largest value of the density on S^2 (at the poles for X3, at the cap
// centre for the tanh kinds)
double rho_max(const Density &r) {
    if (r.kind == 0 || r.kind == 1) return 1.0;
    const double inv_alpha = r.inv_alpha;
    double v = (1.0 - r.gamma) / (1.0 + exp(-2.0 * r.beta * inv_alpha)) + r.gamma;
    if (r.kind == 3) {
        v = v * v;
        v = v * v;
    }
    return v;
}

}  // namespace

extern "C" scvt_status scvt_sample_density(const scvt_density *rho, double exponent, const double *cand,
                                           const double *u, int64_t m, int64_t n_target, double *z_out,
                                           int64_t *n_out, void *cuda_stream) {
    if (!rho || !cand || !u || !z_out || !n_out || m < 1 || m > INT_MAX - 1 || n_target < 0) return SCVT_ERR_INVALID;
    if (!(exponent > 0.0) || !(exponent <= 4.0)) return SCVT_ERR_INVALID;
    if (rho->kind < 0 || rho->kind > 3) return SCVT_ERR_INVALID;
    if (rho->kind >= 2 && !(rho->alpha > 0.0)) return SCVT_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int M = (int)m;
    const Density d = to_device_density(*rho);
    double *dc = nullptr, *du = nullptr, *dout = nullptr;
    int *flag = nullptr, *pos = nullptr, *tmp = nullptr;
    long long *cnt = nullptr;
    const bool cand_dev = device_pointer(cand), u_dev = device_pointer(u), out_dev = device_pointer(z_out);
    cudaError_t e = cudaSuccess;
    if (!cand_dev) e = cudaMallocAsync((void **)&dc, sizeof(double) * 3 * (size_t)M, s);
    if (e == cudaSuccess && !u_dev) e = cudaMallocAsync((void **)&du, sizeof(double) * (size_t)M, s);
    if (e == cudaSuccess && !out_dev && n_target > 0)
        e = cudaMallocAsync((void **)&dout, sizeof(double) * 3 * (size_t)n_target, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&flag, sizeof(int) * (size_t)M, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&pos, sizeof(int) * (size_t)M, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&tmp, sizeof(int) * (2 * ((size_t)M / 2048 + 64) + 64), s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&cnt, sizeof(long long), s);
    if (e == cudaSuccess && dc)
        e = cudaMemcpyAsync(dc, cand, sizeof(double) * 3 * (size_t)M, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && du) e = cudaMemcpyAsync(du, u, sizeof(double) * (size_t)M, cudaMemcpyHostToDevice, s);
    long long host_cnt = 0;
    if (e == cudaSuccess) {
        const double *c = dc ? dc : cand, *uu = du ? du : u;
        double *o = dout ? dout : z_out;
        int64_t launches = 0;
        const unsigned blocks = (unsigned)((M + 255) / 256);
        k_sample_flags<<<blocks, 256, 0, s>>>(d, exponent, rho_pow(rho_max(d), exponent), c, uu, M, flag);
        exclusive_scan(flag, pos, M, tmp, s, &launches);
        k_sample_scatter<<<blocks, 256, 0, s>>>(c, flag, pos, M, (long long)n_target, o, cnt);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&host_cnt, cnt, sizeof(long long), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        const long long k = host_cnt < n_target ? host_cnt : n_target;
        if (e == cudaSuccess && dout && k > 0)
            e = cudaMemcpyAsync(z_out, dout, sizeof(double) * 3 * (size_t)k, cudaMemcpyDeviceToHost, s);
        *n_out = k;
    }
    void *bufs[] = {dc, du, dout, flag, pos, tmp, cnt};
    for (void *p : bufs)
        if (p) cudaFreeAsync(p, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? SCVT_ERR_OOM : SCVT_ERR_CUDA;
    }
    return SCVT_OK;
}
