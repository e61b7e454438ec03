// gf_misc_kernels.cu -- small HBM-bound helpers: model validation and update coefficients,
// residual + L2 misfit (Eq. objective), and the sum of per-shot gradients.
#include "gf_internal.cuh"

namespace gf {
namespace {

constexpr int kRedThreads = 256;

// eps_r >= 1, sigma >= 0 and both finite (the physical ranges the paper clamps to, Sec. 3.1),
// and the update coefficients of every cell of the pitched [ny][pitch] planes:
// Ca = (1 - a)/(1 + a), Cb = (dt/eps)/(1 + a), a = sigma dt / (2 eps), EB/EA and 1/EA of the
// Sec. 3.2 coefficient listing.  The PEC ring (outermost cells), perfect conductors
// (sigma > 100 S/m, the listing's rule) and the row padding get Ca = Cb = 0.
__global__ void prepare_model_kernel(const float* __restrict__ eps_r,
                                     const float* __restrict__ sigma, int nx, int ny, int pitch,
                                     float dt_eps0, float* __restrict__ ca, float* __restrict__ cb,
                                     int* status) {
    int bad = 0;
    const long long total = (long long)pitch * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / pitch), x = (int)(k - (long long)y * pitch);
        float a_ = 0.f, b_ = 0.f;
        if (x < nx) {
            const float e = eps_r[(long long)y * nx + x], s = sigma[(long long)y * nx + x];
            bad |= !(e >= 1.0f && s >= 0.0f && isfinite(e) && isfinite(s));
            const bool ring = x == 0 || y == 0 || x == nx - 1 || y == ny - 1;
            if (!ring && !(s > 100.0f)) {
                const float dte = dt_eps0 / e;
                const float a = 0.5f * s * dte;
                const float inv = 1.0f / (1.0f + a);
                a_ = (1.0f - a) * inv;
                b_ = dte * inv;
            }
        }
        ca[k] = a_;
        cb[k] = b_;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, kStatusBadModel);
}

// resid = traces - observed (skipped if resid is NULL); per-block partial sums of resid^2 / 2
// in FP64 (fixed order).
__global__ void residual_misfit_kernel(const float* __restrict__ traces,
                                       const float* __restrict__ observed, float* resid,
                                       long long count, double* partial, int* status) {
    __shared__ double red[kRedThreads];
    double acc = 0.0;
    int bad = 0;
    for (long long k = blockIdx.x * (long long)kRedThreads + threadIdx.x; k < count;
         k += (long long)gridDim.x * kRedThreads) {
        const float r = traces[k] - observed[k];
        if (resid) resid[k] = r;
        bad |= !isfinite(r);
        acc += 0.5 * (double)r * (double)r;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, kStatusNonFinite);
}

__global__ void finish_misfit_kernel(const double* partial, int nblocks, double* misfit) {
    __shared__ double red[kRedThreads];
    double acc = 0.0;
    for (int k = threadIdx.x; k < nblocks; k += kRedThreads) acc += partial[k];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *misfit = red[0];
}

// out[y * nx + x] = sum_s per_shot[s][y * pitch + x] in shot order (deterministic).
__global__ void sum_shots_kernel(const float* __restrict__ per_shot, int nshots, int nx, int ny,
                                 int pitch, float* __restrict__ out, int* status) {
    int bad = 0;
    const long long N = (long long)nx * ny, Np = (long long)pitch * ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(c / nx), x = (int)(c - (long long)y * nx);
        const long long m = (long long)y * pitch + x;
        float acc = 0.f;
        for (int s = 0; s < nshots; ++s) acc += per_shot[(long long)s * Np + m];
        out[c] = acc;
        bad |= !isfinite(acc);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, kStatusNonFinite);
}

int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return (int)b;
}

}  // namespace

cudaError_t launch_prepare_model(const float* eps_r, const float* sigma, int nx, int ny,
                                 int pitch, float dt_eps0, float* ca, float* cb, int* status,
                                 cudaStream_t st) {
    prepare_model_kernel<<<grid_for((long long)pitch * ny, 256), 256, 0, st>>>(
        eps_r, sigma, nx, ny, pitch, dt_eps0, ca, cb, status);
    return cudaGetLastError();
}

cudaError_t launch_residual_misfit(const float* traces, const float* observed, float* resid,
                                   long long count, double* partial, int nblocks, int* status,
                                   cudaStream_t st) {
    residual_misfit_kernel<<<nblocks, kRedThreads, 0, st>>>(traces, observed, resid, count,
                                                            partial, status);
    return cudaGetLastError();
}

cudaError_t launch_finish_misfit(const double* partial, int nblocks, double* misfit,
                                 cudaStream_t st) {
    finish_misfit_kernel<<<1, kRedThreads, 0, st>>>(partial, nblocks, misfit);
    return cudaGetLastError();
}

cudaError_t launch_sum_shots(const float* per_shot, int nshots, int nx, int ny, int pitch,
                             float* out, int* status, cudaStream_t st) {
    sum_shots_kernel<<<grid_for((long long)nx * ny, 256), 256, 0, st>>>(per_shot, nshots, nx, ny,
                                                                       pitch, out, status);
    return cudaGetLastError();
}

}  // namespace gf
