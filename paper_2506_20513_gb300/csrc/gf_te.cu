// gf_te.cu -- forward model of the TE mode (sm_103a): the fields Ex, Ey, Hz that an x- or
// y-polarised hertzian line source excites in 2-D (Sec. 3.2 source listing, polarisations
// 0 and 1; the z-polarised source drives the TM mode of the tile kernels).
//
//   Hz(i,j) at (i+1/2, j+1/2), Ex(i,j) at (i+1/2, j), Ey(i,j) at (i, j+1/2);
//   mu0 dHz/dt = dEx/dy - dEy/dx;  eps dEx/dt + sigma Ex = dHz/dy - Jx;
//   eps dEy/dt + sigma Ey = -dHz/dx - Jy.
// Each E component takes the update coefficients Ca, Cb of the cell whose index it carries;
// PEC walls hold Ex on rows 0 and ny-1 and Ey on columns 0 and nx-1 at zero; the CPML uses
// the context's axis profiles (Hz's x difference on half-integer x nodes, Ex's y difference
// of Hz on integer y nodes, and so on).
//
// One time step is two launches over the cells (x <= nx-2, y <= ny-2) of every shot, one
// thread per cell, consecutive threads on consecutive x (coalesced rows):
//   H launch: Hz^{n+1/2} from Ex^n, Ey^n into the other Hz buffer, so that extra blocks of
//             the same launch can record Ex^n, Ey^n, Hz^{n-1/2} at the receivers;
//   E launch: Ex^{n+1}, Ey^{n+1} from Hz^{n+1/2}, the source current in its component.
// The CPML memory of a cell is read and written only where its profile is non-zero (it is
// zero, and stays zero, everywhere else).
#include "gf_internal.cuh"

namespace gf {
namespace {

constexpr int kTeThreads = 256;

// Update coefficients of the coefficient listing without the TM ring rule (the TE walls are
// the loop bounds): Ca = (eps/dt - sigma/2) / (eps/dt + sigma/2), Cb = 1 / (eps/dt +
// sigma/2), both 0 in perfect conductors (sigma > 100 S/m) and in the row padding.
__global__ void te_coef_kernel(const float* __restrict__ eps_r, const float* __restrict__ sigma,
                               int nx, int ny, int pitch, float dt_eps0, float* __restrict__ ca,
                               float* __restrict__ cb, int* status) {
    int bad = 0;
    const long long total = (long long)pitch * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / pitch), x = (int)(k - (long long)y * pitch);
        float a_ = 0.f, b_ = 0.f;
        if (x < nx) {
            const float e = eps_r[(long long)y * nx + x], s = sigma[(long long)y * nx + x];
            bad |= !(e >= 1.0f && s >= 0.0f && isfinite(e) && isfinite(s));
            if (!(s > 100.0f)) {
                const float dte = dt_eps0 / e;
                const float h = 0.5f * s * dte;
                const float inv = 1.0f / (1.0f + h);
                a_ = (1.0f - h) * inv;
                b_ = dte * inv;
            }
        }
        ca[k] = a_;
        cb[k] = b_;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, kStatusBadModel);
}

// Cell t of the launch: shot s, column x in [0, nx-2], row y in [0, ny-2].
struct TeCell {
    int s, x, y;
    long long o;  // offset in a field plane [nshots][ny][pitch]
};

__device__ __forceinline__ TeCell te_cell(const TeParams& p, long long t) {
    const long long per = (long long)(p.nx - 1) * (p.ny - 1);
    TeCell c;
    c.s = (int)(t / per);
    const long long r = t - (long long)c.s * per;
    c.y = (int)(r / (p.nx - 1));
    c.x = (int)(r - (long long)c.y * (p.nx - 1));
    c.o = (long long)c.s * p.Np + (long long)c.y * p.pitch + c.x;
    return c;
}

__global__ void __launch_bounds__(kTeThreads) te_h_kernel(const TeParams p, int n,
                                                          const float* __restrict__ hz_old,
                                                          float* __restrict__ hz_new) {
    const long long cells = (long long)p.nshots * (p.nx - 1) * (p.ny - 1);
    const long long t = blockIdx.x * (long long)kTeThreads + threadIdx.x;
    if (t >= cells) {
        // receiver blocks: Ex^n, Ey^n, Hz^{n-1/2} (nothing in this launch writes them)
        const long long r = t - (((cells + kTeThreads - 1) / kTeThreads) * kTeThreads);
        if (r < 0 || r >= (long long)p.nshots * p.nrec) return;
        const int s = (int)(r / p.nrec);
        const int2 xy = __ldg(p.rec_xy + r);
        const long long o = (long long)s * p.Np + (long long)xy.y * p.pitch + xy.x;
        const long long k = ((long long)s * p.nt + n) * p.nrec + (r - (long long)s * p.nrec);
        if (p.traces) {
            p.traces[3 * k] = p.ex[o];
            p.traces[3 * k + 1] = p.ey[o];
            p.traces[3 * k + 2] = hz_old[o];
        }
        if (p.traces_p) p.traces_p[k] = p.pol == 0 ? p.ex[o] : p.ey[o];
        return;
    }
    const TeCell c = te_cell(p, t);
    const float dyr = p.ex[c.o + p.pitch] - p.ex[c.o];
    const float dxr = p.ey[c.o + 1] - p.ey[c.o];
    float ty = __ldg(p.py.aH + c.y) * dyr;
    float tx = __ldg(p.px.aH + c.x) * dxr;
    const float cy = __ldg(p.py.cH + c.y);
    if (cy != 0.f) {
        const float q = fmaf(__ldg(p.py.bH + c.y), p.psi_hzy[c.o], cy * dyr);
        p.psi_hzy[c.o] = q;
        ty += q;
    }
    const float cx = __ldg(p.px.cH + c.x);
    if (cx != 0.f) {
        const float q = fmaf(__ldg(p.px.bH + c.x), p.psi_hzx[c.o], cx * dxr);
        p.psi_hzx[c.o] = q;
        tx += q;
    }
    hz_new[c.o] = fmaf(p.ch, ty - tx, hz_old[c.o]);
}

__global__ void __launch_bounds__(kTeThreads) te_e_kernel(const TeParams p, int n,
                                                          const float* __restrict__ hz) {
    const long long cells = (long long)p.nshots * (p.nx - 1) * (p.ny - 1);
    const long long t = blockIdx.x * (long long)kTeThreads + threadIdx.x;
    if (t >= cells) return;
    const TeCell c = te_cell(p, t);
    const long long m = (long long)c.y * p.pitch + c.x;
    const float a = __ldg(p.ca + m), b = __ldg(p.cb + m);
    // source current of this cell (x-directed sources on Ex, y-directed on Ey)
    float w = 0.f;
    for (int k = 0; k < p.nsrc; ++k) {
        const int2 xy = __ldg(p.src_xy + c.s * p.nsrc + k);
        if (xy.x == c.x && xy.y == c.y)
            w += __ldg(p.wavelet + ((long long)c.s * p.nsrc + k) * p.nt + n);
    }
    w *= p.src_scale;
    const float h = hz[c.o];
    if (c.y >= 1) {
        const float d = h - hz[c.o - p.pitch];
        float q = __ldg(p.py.aE + c.y) * d;
        const float cy = __ldg(p.py.cE + c.y);
        if (cy != 0.f) {
            const float s = fmaf(__ldg(p.py.bE + c.y), p.psi_exy[c.o], cy * d);
            p.psi_exy[c.o] = s;
            q += s;
        }
        if (p.pol == 0) q -= w;
        const float e = fmaf(a, p.ex[c.o], b * q);
        p.ex[c.o] = e;
        if (p.hist) p.hist[(long long)n * 2 * p.F + c.o] = e;
    }
    if (c.x >= 1) {
        const float d = h - hz[c.o - 1];
        float q = __ldg(p.px.aE + c.x) * d;
        const float cx = __ldg(p.px.cE + c.x);
        if (cx != 0.f) {
            const float s = fmaf(__ldg(p.px.bE + c.x), p.psi_eyx[c.o], cx * d);
            p.psi_eyx[c.o] = s;
            q += s;
        }
        q = -q;
        if (p.pol == 1) q -= w;
        const float e = fmaf(a, p.ey[c.o], b * q);
        p.ey[c.o] = e;
        if (p.hist) p.hist[(long long)n * 2 * p.F + p.F + c.o] = e;
    }
}

// ---- adjoint ---------------------------------------------------------------------------
// Step n reversed.  On entry aex, aey hold dJ/dE^{n+1} and ahz dJ/dHz^{n+1/2} (without the
// E updates' share); the CPML memories' adjoints follow A_n = b A_{n+1} + (cotangent of the
// bracket that uses the memory of step n), and only inside the strips (c != 0: outside,
// b = 0 and the memory's adjoint only ever meets c = 0).

// E updates reversed: lam = Cb aE^{n+1}; the zero-lag gradients of both components of the
// cell; the bracket's cotangent goes through its CPML memory to the Hz difference (d_ex,
// d_ey, gathered by the next launch); aE becomes Ca aE^{n+1}.
__global__ void __launch_bounds__(kTeThreads) te_adj_e_kernel(const TeParams p, int n) {
    const long long cells = (long long)p.nshots * (p.nx - 1) * (p.ny - 1);
    const long long t = blockIdx.x * (long long)kTeThreads + threadIdx.x;
    if (t >= cells) return;
    const TeCell c = te_cell(p, t);
    const long long m = (long long)c.y * p.pitch + c.x;
    const float a = __ldg(p.ca + m), b = __ldg(p.cb + m);
    const float* h1 = p.hist + (long long)n * 2 * p.F;
    const float* h0 = n > 0 ? h1 - 2 * p.F : nullptr;
    float ge = 0.f, gs = 0.f;
    if (c.y >= 1) {
        const float ae = p.aex[c.o];
        const float lam = b * ae;
        const float e1 = h1[c.o], e0 = h0 ? h0[c.o] : 0.f;
        ge = fmaf(-lam, e1 - e0, ge);
        gs = fmaf(-0.5f * lam, e1 + e0, gs);
        float d = __ldg(p.py.aE + c.y) * lam;
        const float cy = __ldg(p.py.cE + c.y);
        if (cy != 0.f) {
            const float A = fmaf(__ldg(p.py.bE + c.y), p.a_exy[c.o], lam);
            p.a_exy[c.o] = A;
            d = fmaf(cy, A, d);
        }
        p.d_ex[c.o] = d;
        p.aex[c.o] = a * ae;
    }
    if (c.x >= 1) {
        const float ae = p.aey[c.o];
        const float lam = b * ae;
        const float e1 = h1[p.F + c.o], e0 = h0 ? h0[p.F + c.o] : 0.f;
        ge = fmaf(-lam, e1 - e0, ge);
        gs = fmaf(-0.5f * lam, e1 + e0, gs);
        // Qy = -(a D + psi): the bracket's cotangent is -lam
        float d = -__ldg(p.px.aE + c.x) * lam;
        const float cx = __ldg(p.px.cE + c.x);
        if (cx != 0.f) {
            const float A = fmaf(__ldg(p.px.bE + c.x), p.a_eyx[c.o], -lam);
            p.a_eyx[c.o] = A;
            d = fmaf(cx, A, d);
        }
        p.d_ey[c.o] = d;
        p.aey[c.o] = a * ae;
    }
    p.g_eps[c.o] = fmaf(ge, p.geps, p.g_eps[c.o]);
    p.g_sig[c.o] += gs;
}

// Hz update reversed: dJ/dHz^{n+1/2} gathers the E brackets' cotangents of the four E
// nodes around the cell; it is also dJ/dHz^{n-1/2}; the Hz bracket's cotangent goes through
// the memories to the E differences (d_hy for Ex, d_hx for Ey).
__global__ void __launch_bounds__(kTeThreads) te_adj_h_kernel(const TeParams p) {
    const long long cells = (long long)p.nshots * (p.nx - 1) * (p.ny - 1);
    const long long t = blockIdx.x * (long long)kTeThreads + threadIdx.x;
    if (t >= cells) return;
    const TeCell c = te_cell(p, t);
    const float ah = p.ahz[c.o] + (p.d_ex[c.o] - p.d_ex[c.o + p.pitch]) +
                     (p.d_ey[c.o] - p.d_ey[c.o + 1]);
    p.ahz[c.o] = ah;
    const float h = p.ch * ah;
    float dy = __ldg(p.py.aH + c.y) * h;
    const float cy = __ldg(p.py.cH + c.y);
    if (cy != 0.f) {
        const float B = fmaf(__ldg(p.py.bH + c.y), p.b_hzy[c.o], h);
        p.b_hzy[c.o] = B;
        dy = fmaf(cy, B, dy);
    }
    float dx = -__ldg(p.px.aH + c.x) * h;
    const float cx = __ldg(p.px.cH + c.x);
    if (cx != 0.f) {
        const float B = fmaf(__ldg(p.px.bH + c.x), p.b_hzx[c.o], -h);
        p.b_hzx[c.o] = B;
        dx = fmaf(cx, B, dx);
    }
    p.d_hy[c.o] = dy;
    p.d_hx[c.o] = dx;
}

// dJ/dE^n of the updated E nodes: Ca aE^{n+1} plus the two Hz cells whose differences use it.
__global__ void __launch_bounds__(kTeThreads) te_adj_gather_kernel(const TeParams p) {
    const long long cells = (long long)p.nshots * (p.nx - 1) * (p.ny - 1);
    const long long t = blockIdx.x * (long long)kTeThreads + threadIdx.x;
    if (t >= cells) return;
    const TeCell c = te_cell(p, t);
    if (c.y >= 1) p.aex[c.o] += p.d_hy[c.o - p.pitch] - p.d_hy[c.o];
    if (c.x >= 1) p.aey[c.o] += p.d_hx[c.o - 1] - p.d_hx[c.o];
}

// The recording of step n reversed: the residual enters the source component's adjoint at
// each receiver node (atomic: receivers may share a cell).
__global__ void te_adj_rec_kernel(const TeParams p, int n) {
    const long long r = blockIdx.x * (long long)kTeThreads + threadIdx.x;
    if (r >= (long long)p.nshots * p.nrec) return;
    const int s = (int)(r / p.nrec);
    const int2 xy = __ldg(p.rec_xy + r);
    const long long o = (long long)s * p.Np + (long long)xy.y * p.pitch + xy.x;
    float* ae = p.pol == 0 ? p.aex : p.aey;
    atomicAdd(ae + o, __ldg(p.resid + ((long long)s * p.nt + n) * p.nrec + (r - (long long)s * p.nrec)));
}

long long te_blocks(long long n) { return (n + kTeThreads - 1) / kTeThreads; }

}  // namespace

cudaError_t launch_te_coef(const float* eps_r, const float* sigma, int nx, int ny, int pitch,
                           float dt_eps0, float* ca, float* cb, int* status, cudaStream_t st) {
    const long long b = te_blocks((long long)pitch * ny);
    te_coef_kernel<<<(int)(b < 152 * 8 ? b : 152 * 8), kTeThreads, 0, st>>>(
        eps_r, sigma, nx, ny, pitch, dt_eps0, ca, cb, status);
    return cudaGetLastError();
}

cudaError_t launch_te_h(const TeParams& p, int n, cudaStream_t st) {
    const long long cells = (long long)p.nshots * (p.nx - 1) * (p.ny - 1);
    const long long bc = te_blocks(cells);
    const long long br = te_blocks((long long)p.nshots * p.nrec);
    const float* hz_old = (n & 1) ? p.hz1 : p.hz0;
    float* hz_new = (n & 1) ? p.hz0 : p.hz1;
    te_h_kernel<<<(unsigned)(bc + br), kTeThreads, 0, st>>>(p, n, hz_old, hz_new);
    return cudaGetLastError();
}

cudaError_t launch_te_adj_step(const TeParams& p, int n, int part, cudaStream_t st) {
    const long long cells = (long long)p.nshots * (p.nx - 1) * (p.ny - 1);
    const unsigned bc = (unsigned)te_blocks(cells);
    switch (part) {
        case 0: te_adj_e_kernel<<<bc, kTeThreads, 0, st>>>(p, n); break;
        case 1: te_adj_h_kernel<<<bc, kTeThreads, 0, st>>>(p); break;
        case 2: te_adj_gather_kernel<<<bc, kTeThreads, 0, st>>>(p); break;
        default:
            te_adj_rec_kernel<<<(unsigned)te_blocks((long long)p.nshots * p.nrec), kTeThreads, 0,
                                st>>>(p, n);
    }
    return cudaGetLastError();
}

cudaError_t launch_te_e(const TeParams& p, int n, cudaStream_t st) {
    const long long cells = (long long)p.nshots * (p.nx - 1) * (p.ny - 1);
    const float* hz_new = (n & 1) ? p.hz0 : p.hz1;
    te_e_kernel<<<(unsigned)te_blocks(cells), kTeThreads, 0, st>>>(p, n, hz_new);
    return cudaGetLastError();
}

}  // namespace gf
