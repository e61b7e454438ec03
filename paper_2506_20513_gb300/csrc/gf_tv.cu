// gf_tv.cu -- total-variation regularisation of a model gradient (Algorithm 3, Sec. 3.4).
//
// The paper lists the steps of its TV term (backward difference with circular boundary, a
// right-hand side, an average of neighbours by convolution, forward difference with circular
// boundary, soft-thresholding of the auxiliary variables Z, multiplier update, restoring the
// scale) and the functional TV(X) = sum sqrt((Dx X)^2 + (Dy X)^2).  Read as split Bregman for
// the TV-denoising problem  min_u 1/2 |u - x|^2 + lambda TV(u)  on the normalised model
// x = X / max|X|, from u = x, Z = D x, B = 0, with u updated by one Jacobi sweep of
// (1 + 4 mu) u - mu * sum(neighbours) = x + mu D^T (Z - B) per iteration,
// Z = shrink(D u + B, lambda / mu) (isotropic) and B += D u - Z.  The TV gradient pulls the
// model towards its denoised version, in normalised units: G += weight * max|G| * (x - u).
//
// Also here: the Adam update of one model parameter (Sec. 2.3), the other model-space kernel
// of the inversion drivers.
#include "gf_internal.cuh"

namespace gf {
namespace {

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// max |a| (and max |b| if given) over n values into bits[0], bits[1] (non-negative floats
// order like their bit patterns, so an integer atomicMax is exact and order-independent).
__global__ void max_abs_kernel(const float* __restrict__ a, const float* __restrict__ b,
                               long long n, unsigned* bits) {
    float ma = 0.f, mb = 0.f;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        ma = fmaxf(ma, fabsf(a[k]));
        if (b) mb = fmaxf(mb, fabsf(b[k]));
    }
    atomicMax(&bits[0], __float_as_uint(ma));
    if (b) atomicMax(&bits[1], __float_as_uint(mb));
}

// x = X / s; u = x; Z = D x (forward differences, circular); B = 0
__global__ void tv_init_kernel(const float* __restrict__ X, const unsigned* bits, int nx, int ny,
                               float* x, float* u, float* zx, float* zy, float* bx, float* by) {
    const float s = __uint_as_float(bits[0]);
    const float inv = s > 0.f ? 1.f / s : 0.f;
    const long long n = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k % nx), j = (int)(k / nx);
        const float v = X[k] * inv;
        x[k] = v;
        u[k] = v;
        zx[k] = X[(long long)j * nx + wrap(i + 1, nx)] * inv - v;
        zy[k] = X[(long long)wrap(j + 1, ny) * nx + i] * inv - v;
        bx[k] = 0.f;
        by[k] = 0.f;
    }
}

// One Jacobi sweep: u_new = (x + mu D^T(Z - B) + mu * sum of the four neighbours of u) /
// (1 + 4 mu), with D^T v (i) = v(i-1) - v(i) (circular backward difference).
__global__ void tv_u_kernel(const float* __restrict__ x, const float* __restrict__ u,
                            const float* __restrict__ zx, const float* __restrict__ zy,
                            const float* __restrict__ bx, const float* __restrict__ by,
                            int nx, int ny, float mu, float* __restrict__ u_new) {
    const long long n = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k % nx), j = (int)(k / nx);
        const long long kl = (long long)j * nx + wrap(i - 1, nx);
        const long long kd = (long long)wrap(j - 1, ny) * nx + i;
        const long long kr = (long long)j * nx + wrap(i + 1, nx);
        const long long ku = (long long)wrap(j + 1, ny) * nx + i;
        const float div = (zx[kl] - bx[kl]) - (zx[k] - bx[k]) + (zy[kd] - by[kd]) - (zy[k] - by[k]);
        const float nb = u[kl] + u[kr] + u[kd] + u[ku];
        u_new[k] = (x[k] + mu * div + mu * nb) / (1.f + 4.f * mu);
    }
}

// Forward differences of u (circular), isotropic soft threshold, multiplier update.
__global__ void tv_zb_kernel(const float* __restrict__ u, int nx, int ny, float thresh,
                             float* zx, float* zy, float* bx, float* by) {
    const long long n = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k % nx), j = (int)(k / nx);
        const float dx = u[(long long)j * nx + wrap(i + 1, nx)] - u[k];
        const float dy = u[(long long)wrap(j + 1, ny) * nx + i] - u[k];
        const float sx = dx + bx[k], sy = dy + by[k];
        const float mag = sqrtf(sx * sx + sy * sy);
        const float f = mag > thresh ? (mag - thresh) / mag : 0.f;
        const float nzx = f * sx, nzy = f * sy;
        zx[k] = nzx;
        zy[k] = nzy;
        bx[k] = sx - nzx;
        by[k] = sy - nzy;
    }
}

// G += weight * max|G| * (x - u)  (bits[1] = max|G|)
__global__ void tv_apply_kernel(const float* __restrict__ x, const float* __restrict__ u,
                                const unsigned* bits, long long n, float weight, float* G) {
    const float w = weight * __uint_as_float(bits[1]);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        G[k] += w * (x[k] - u[k]);
}

int blocks_for(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 152 * 8 ? 152 * 8 : b));
}

// One Adam step where the mask is non-zero: g' = gscale g, first and second moments
// m = b1 m + (1 - b1) g', v = b2 v + (1 - b2) g'^2, then
// x = max(xmin, x - lr (m c1) / (sqrt(v c2) + eps)) with the bias corrections
// c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t).  Masked cells keep x, m and v.
__global__ void adam_kernel(long long n, float* __restrict__ x, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ mask, float gscale, float lr, float b1,
                            float b2, float eps, float c1, float c2, float xmin) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        if (mask && mask[k] == 0.f) continue;
        const float gk = gscale * g[k];
        const float mk = b1 * m[k] + (1.f - b1) * gk;
        const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        x[k] = fmaxf(xmin, x[k] - lr * (mk * c1) / (sqrtf(vk * c2) + eps));
    }
}

}  // namespace

cudaError_t adam_update(long long n, float* x, const float* g, float* m, float* v,
                        const float* mask, float gscale, float lr, float b1, float b2, float eps,
                        int t, float xmin, cudaStream_t st) {
    const float c1 = (float)(1.0 / (1.0 - pow((double)b1, t)));
    const float c2 = (float)(1.0 / (1.0 - pow((double)b2, t)));
    adam_kernel<<<blocks_for(n), 256, 0, st>>>(n, x, g, m, v, mask, gscale, lr, b1, b2, eps, c1,
                                               c2, xmin);
    return cudaGetLastError();
}

size_t tv_scratch_floats(long long n) { return 7 * (size_t)n + 64; }

cudaError_t tv_gradient(int nx, int ny, const float* X, float* G, float* scratch, float lambda,
                        float mu, int iters, float weight, cudaStream_t st) {
    const long long n = (long long)nx * ny;
    float* x = scratch;
    float* u = x + n;
    float* u2 = u + n;
    float* zx = u2 + n;
    float* zy = zx + n;
    float* bx = zy + n;
    float* by = bx + n;
    unsigned* bits = reinterpret_cast<unsigned*>(by + n);
    cudaError_t e = cudaMemsetAsync(bits, 0, 4 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    const int nb = blocks_for(n);
    max_abs_kernel<<<nb, 256, 0, st>>>(X, G, n, bits);
    tv_init_kernel<<<nb, 256, 0, st>>>(X, bits, nx, ny, x, u, zx, zy, bx, by);
    for (int it = 0; it < iters; ++it) {
        tv_u_kernel<<<nb, 256, 0, st>>>(x, u, zx, zy, bx, by, nx, ny, mu, u2);
        float* t = u;
        u = u2;
        u2 = t;
        tv_zb_kernel<<<nb, 256, 0, st>>>(u, nx, ny, lambda / mu, zx, zy, bx, by);
    }
    tv_apply_kernel<<<nb, 256, 0, st>>>(x, u, bits, n, weight, G);
    return cudaGetLastError();
}

}  // namespace gf
