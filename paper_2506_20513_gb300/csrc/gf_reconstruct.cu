// gf_reconstruct.cu -- reverse-time reconstruction of the forward wavefield inside a
// checkpoint segment (storage mode GF_STORE_RECONSTRUCT, sm_103a).
//
// Instead of keeping Ez of every step of a segment, the segment's forward recomputation keeps
// only the fields of a boundary ring (the CPML strips and two cells more) per step; the
// adjoint then runs the Yee updates of Algorithm 1 backwards from the segment's last state:
// with state_n = (Ez^n, H^{n-1/2}), undoing step n is
//   Ez^n = (Ez^{n+1} + Cb w^n / (dx dy) [source cells] - Cb Q(H^{n+1/2})) / Ca,
//   Hy^{n-1/2} = Hy^{n+1/2} - (dt/mu0) (Ez^n(i+1,j) - Ez^n(i,j)) / dx,
//   Hx^{n-1/2} = Hx^{n+1/2} + (dt/mu0) (Ez^n(i,j+1) - Ez^n(i,j)) / dy,
// Q = (Hy(i,j) - Hy(i-1,j)) / dx - (Hx(i,j) - Hx(i,j-1)) / dy, on the cells outside the ring
// (where no CPML memory takes part in the updates and all neighbours exist); ring cells take
// their stored values.  Perfect conductors (Ca = 0) stay 0.  In lossy cells Ca < 1, so the
// reversed E update amplifies FP32 rounding by about 1 / Ca per step (e^{a k} over a k-step
// segment, a = sigma dt / eps): the scheme is only usable inside short segments.
#include "gf_internal.cuh"

namespace gf {
namespace {

// Ring fields of every shot at one step: slot [3][nshots][ring_cells] <- Ez, Hx, Hy.
__global__ void ring_store_kernel(const float* __restrict__ st, long long F, long long Np,
                                  int pitch, int nx, int ny, int nshots,
                                  const int* __restrict__ ring_map, int ring_cells,
                                  float* __restrict__ slot) {
    const long long N = (long long)nx * ny;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N * nshots;
         t += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(t / N);
        const long long c = t - s * N;
        const int r = __ldg(ring_map + c);
        if (r < 0) continue;
        const int j = (int)(c / nx), i = (int)(c - (long long)j * nx);
        const long long o = s * Np + (long long)j * pitch + i;
        for (int f = 0; f < 3; ++f)
            slot[((long long)f * nshots + s) * ring_cells + r] = st[f * F + o];
    }
}

// Undo step n's E update (and its source) of every shot; also write Ez^n to the history
// plane `hist` of each shot (hist + s * hist_stride_np).
__global__ void reverse_e_kernel(float* __restrict__ st, long long F, long long Np, int pitch,
                                 int nx, int ny, int nshots, const int* __restrict__ ring_map,
                                 int ring_cells, const float* __restrict__ slot,
                                 const float* __restrict__ ca, const float* __restrict__ cb,
                                 float rdx, float rdy, const int2* __restrict__ src_xy, int nsrc,
                                 const float* __restrict__ wavelet, int nt, int n,
                                 float src_scale, float* __restrict__ hist,
                                 long long hist_stride_np) {
    const long long N = (long long)nx * ny;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N * nshots;
         t += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(t / N);
        const long long c = t - s * N;
        const int j = (int)(c / nx), i = (int)(c - (long long)j * nx);
        const long long m = (long long)j * pitch + i;
        const long long o = s * Np + m;
        const int r = __ldg(ring_map + c);
        float ez;
        if (r >= 0) {
            ez = slot[(long long)s * ring_cells + r];
        } else {
            const float a = ca[m], b = cb[m];
            float e1 = st[o];
            for (int k = 0; k < nsrc; ++k) {
                const int2 xy = __ldg(src_xy + s * nsrc + k);
                if (xy.x == i && xy.y == j)
                    e1 += b * src_scale * __ldg(wavelet + ((long long)s * nsrc + k) * nt + n);
            }
            const float* hx = st + F + o;
            const float* hy = st + 2 * F + o;
            float q = rdx * (hy[0] - hy[-1]);
            q = fmaf(-rdy, hx[0] - hx[-pitch], q);
            ez = a != 0.f ? (e1 - b * q) / a : 0.f;
        }
        st[o] = ez;
        hist[s * hist_stride_np + m] = ez;
    }
}

// Undo step n's H update from Ez^n (all of it already reconstructed).
__global__ void reverse_h_kernel(float* __restrict__ st, long long F, long long Np, int pitch,
                                 int nx, int ny, int nshots, const int* __restrict__ ring_map,
                                 int ring_cells, const float* __restrict__ slot, float chx,
                                 float chy) {
    const long long N = (long long)nx * ny;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N * nshots;
         t += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(t / N);
        const long long c = t - s * N;
        const int j = (int)(c / nx), i = (int)(c - (long long)j * nx);
        const long long o = s * Np + (long long)j * pitch + i;
        const int r = __ldg(ring_map + c);
        if (r >= 0) {
            st[F + o] = slot[((long long)nshots + s) * ring_cells + r];
            st[2 * F + o] = slot[((long long)2 * nshots + s) * ring_cells + r];
        } else {
            const float e = st[o];
            st[2 * F + o] = fmaf(-chx, st[o + 1] - e, st[2 * F + o]);
            st[F + o] = fmaf(chy, st[o + pitch] - e, st[F + o]);
        }
    }
}

int grid_for(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

}  // namespace

cudaError_t launch_ring_store(const float* st, int nshots, long long Np, int pitch, int nx,
                             int ny, const int* ring_map, int ring_cells, float* slot,
                             cudaStream_t stream) {
    const long long F = (long long)nshots * Np;
    ring_store_kernel<<<grid_for((long long)nx * ny * nshots), 256, 0, stream>>>(
        st, F, Np, pitch, nx, ny, nshots, ring_map, ring_cells, slot);
    return cudaGetLastError();
}

cudaError_t launch_reverse_step(float* st, int nshots, long long Np, int pitch, int nx, int ny,
                                const int* ring_map, int ring_cells, const float* slot,
                                const float* ca, const float* cb, float rdx, float rdy,
                                float ch, const int2* src_xy, int nsrc, const float* wavelet,
                                int nt, int n, float src_scale, float* hist,
                                long long hist_stride_np, cudaStream_t stream) {
    const long long F = (long long)nshots * Np;
    const int g = grid_for((long long)nx * ny * nshots);
    reverse_e_kernel<<<g, 256, 0, stream>>>(st, F, Np, pitch, nx, ny, nshots, ring_map,
                                            ring_cells, slot, ca, cb, rdx, rdy, src_xy, nsrc,
                                            wavelet, nt, n, src_scale, hist, hist_stride_np);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reverse_h_kernel<<<g, 256, 0, stream>>>(st, F, Np, pitch, nx, ny, nshots, ring_map,
                                            ring_cells, slot, ch * rdx, ch * rdy);
    return cudaGetLastError();
}

}  // namespace gf
