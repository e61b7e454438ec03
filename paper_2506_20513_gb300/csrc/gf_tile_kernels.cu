// gf_tile_kernels.cu -- temporally blocked 2-D TM FDTD forward and adjoint kernels (sm_103a).
//
// One CTA owns an interior tile of tile_w x tile_h cells of one shot and advances it K time
// steps per launch.  The tile plus a K-cell halo is staged in shared memory; every time step
// the valid region shrinks by one cell on each side (an H update needs Ez at +1, an E update
// needs H at -1), so after K steps exactly the interior is valid and is written back to the
// other ping-pong state buffer.  Halo cells are recomputed redundantly by neighbouring CTAs
// from the same inputs, so every copy of a cell holds the same value.  Sources and adjoint
// sources are injected into every staged copy of their cell; receivers and the wavefield
// history are written only by the owning (interior) CTA.
//
// Forward time step n (Algorithm 1, Sec. 3.3): record d^n = Ez^n at the receivers, update
// H and the magnetic CPML memories from Ez^n, update Ez and the electric CPML memories from
// H^{n+1/2} with Ez^{n+1} = Ca Ez^n + Cb Q (Eqs. 3-5 in the time-averaged loss form of the
// Sec. 3.2 coefficient listing), inject the source into Q (Sec. 3.2 source listing), store
// Ez^{n+1}.
//
// Adjoint time step n (Algorithm 2): the exact transpose of the forward step, in reverse:
// lam = Cb * adj(Ez^{n+1}) accumulates the zero-lag gradients (Eqs. grad_eps, grad_sigma in
// discrete form), feeds the electric CPML memories and, through the transposed differences,
// adj(H); adj(H) feeds the magnetic CPML memories and adj(Ez^n); the receiver residual of
// step n is added last.
#include "gf_internal.cuh"

namespace gf {
namespace {

constexpr int kTX = 32;  // threads along x (one warp per row: coalesced rows)
constexpr int kTY = kThreads / kTX;

// Ca = (1 - a)/(1 + a), Cb = (dt/eps)/(1 + a), a = sigma dt / (2 eps): EB/EA and 1/EA of the
// coefficient listing.  The PEC ring and perfect conductors (sigma > 100 S/m) get 0.
__device__ __forceinline__ void coefficients(float er, float sg, float dt_eps0, bool fixed,
                                             float& Ca, float& Cb) {
    if (fixed || sg > 100.0f) {
        Ca = 0.0f;
        Cb = 0.0f;
        return;
    }
    const float dte = dt_eps0 / er;
    const float a = 0.5f * sg * dte;
    const float inv = 1.0f / (1.0f + a);
    Ca = (1.0f - a) * inv;
    Cb = dte * inv;
}

__device__ __forceinline__ bool in_xstrip(int gx, const TileParams& p) {
    return gx < p.npml || gx >= p.nx - p.npml - 1;
}
__device__ __forceinline__ bool in_ystrip(int gy, const TileParams& p) {
    return gy < p.npml || gy >= p.ny - p.npml - 1;
}

// Stage the six profile arrays of one axis for local indices 0..E-1 starting at global O.
__device__ __forceinline__ void stage_profile(float* dst, const AxisProfile& a, int O, int E,
                                              int n, int tid) {
    for (int i = tid; i < E; i += kThreads) {
        const int g = min(max(O + i, 0), n - 1);
        dst[i] = __ldg(a.aE + g);
        dst[E + i] = __ldg(a.bE + g);
        dst[2 * E + i] = __ldg(a.cE + g);
        dst[3 * E + i] = __ldg(a.aH + g);
        dst[4 * E + i] = __ldg(a.bH + g);
        dst[5 * E + i] = __ldg(a.cH + g);
    }
}

// ---------------------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------------------
template <bool kHist, bool kIllum>
__global__ void __launch_bounds__(kThreads) fwd_tile_kernel(const TileParams p) {
    extern __shared__ float4 smem_raw[];
    float* sm = reinterpret_cast<float*>(smem_raw);
    const int K = p.K, TW = p.tile_w, TH = p.tile_h;
    const int EW = TW + 2 * K, EH = TH + 2 * K, EN = EW * EH;
    float* Ez = sm;
    float* Hx = Ez + EN;
    float* Hy = Hx + EN;
    float* Ca = Hy + EN;
    float* Cb = Ca + EN;
    float* PEx = Cb + EN;
    float* PEy = PEx + EN;
    float* PHx = PEy + EN;
    float* PHy = PHx + EN;
    float* xp = PHy + EN;     // [6][EW]
    float* yp = xp + 6 * EW;  // [6][EH]
    float* ill = yp + 6 * EH; // [TH][TW]
    __shared__ int s_src[kMaxSrc];

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kTX + tx;
    const int shot = blockIdx.y;
    const int X0 = (blockIdx.x % p.tiles_x) * TW - K;
    const int Y0 = (blockIdx.x / p.tiles_x) * TH - K;
    const long long F = (long long)p.nshots * p.N;
    const long long sbase = (long long)shot * p.N;

    for (int ly = ty; ly < EH; ly += kTY) {
        const int gy = Y0 + ly;
        for (int lx = tx; lx < EW; lx += kTX) {
            const int gx = X0 + lx, l = ly * EW + lx;
            float ez = 0.f, hx = 0.f, hy = 0.f, ca = 0.f, cb = 0.f;
            float pex = 0.f, pey = 0.f, phx = 0.f, phy = 0.f;
            if (gx >= 0 && gx < p.nx && gy >= 0 && gy < p.ny) {
                const long long g = (long long)gy * p.nx + gx, sg = sbase + g;
                ez = p.st_in[sg];
                hx = p.st_in[F + sg];
                hy = p.st_in[2 * F + sg];
                if (in_xstrip(gx, p)) {
                    pex = p.st_in[3 * F + sg];
                    phy = p.st_in[6 * F + sg];
                }
                if (in_ystrip(gy, p)) {
                    pey = p.st_in[4 * F + sg];
                    phx = p.st_in[5 * F + sg];
                }
                const bool ring = gx == 0 || gy == 0 || gx == p.nx - 1 || gy == p.ny - 1;
                coefficients(__ldg(p.eps_r + g), __ldg(p.sigma + g), p.dt_eps0, ring, ca, cb);
            }
            Ez[l] = ez; Hx[l] = hx; Hy[l] = hy; Ca[l] = ca; Cb[l] = cb;
            PEx[l] = pex; PEy[l] = pey; PHx[l] = phx; PHy[l] = phy;
        }
    }
    stage_profile(xp, p.px, X0, EW, p.nx, tid);
    stage_profile(yp, p.py, Y0, EH, p.ny, tid);
    if (kIllum)
        for (int i = tid; i < TW * TH; i += kThreads) ill[i] = 0.f;
    if (tid < kMaxSrc) {
        int li = -1;
        if (tid < p.nsrc) {
            const int cell = p.src_cell[shot * p.nsrc + tid];
            const int lx = cell % p.nx - X0, ly = cell / p.nx - Y0;
            if (lx >= 0 && lx < EW && ly >= 0 && ly < EH) li = ly * EW + lx;
        }
        s_src[tid] = li;
    }
    __syncthreads();

    for (int s = 0; s < K; ++s) {
        const int n = p.n0 + s;
        // 1. receivers: d^n = Ez^n, written by the CTA that owns the receiver cell
        for (int r = tid; r < p.nrec; r += kThreads) {
            const int cell = __ldg(p.rec_cell + shot * p.nrec + r);
            const int lx = cell % p.nx - X0, ly = cell / p.nx - Y0;
            if (lx >= K && lx < K + TW && ly >= K && ly < K + TH)
                p.traces[((long long)shot * p.nt + n) * p.nrec + r] = Ez[ly * EW + lx];
        }
        // 2-3. H and magnetic CPML from Ez^n
        for (int ly = s + ty; ly <= EH - 2 - s; ly += kTY) {
            const float ayH = yp[3 * EH + ly], byH = yp[4 * EH + ly], cyH = yp[5 * EH + ly];
            for (int lx = s + tx; lx <= EW - 2 - s; lx += kTX) {
                const int l = ly * EW + lx;
                const float ez = Ez[l];
                const float dyE = Ez[l + EW] - ez, dxE = Ez[l + 1] - ez;
                const float phx = byH * PHx[l] + cyH * dyE;
                PHx[l] = phx;
                Hx[l] -= p.ch * (ayH * dyE + phx);
                const float phy = xp[4 * EW + lx] * PHy[l] + xp[5 * EW + lx] * dxE;
                PHy[l] = phy;
                Hy[l] += p.ch * (xp[3 * EW + lx] * dxE + phy);
            }
        }
        __syncthreads();
        // 4-6. E, electric CPML and the source term, giving Ez^{n+1}
        float wsrc[kMaxSrc];
        int lsrc[kMaxSrc];
#pragma unroll
        for (int k = 0; k < kMaxSrc; ++k) {
            lsrc[k] = -1;
            wsrc[k] = 0.f;
            if (k < p.nsrc) {
                lsrc[k] = s_src[k];
                wsrc[k] = p.src_scale * __ldg(p.wavelet + ((long long)shot * p.nsrc + k) * p.nt + n);
            }
        }
        for (int ly = s + 1 + ty; ly <= EH - 2 - s; ly += kTY) {
            const float ayE = yp[ly], byE = yp[EH + ly], cyE = yp[2 * EH + ly];
            const int gy = Y0 + ly;
            const bool row_in = ly >= K && ly < K + TH && gy < p.ny;
            for (int lx = s + 1 + tx; lx <= EW - 2 - s; lx += kTX) {
                const int l = ly * EW + lx;
                const float dxH = Hy[l] - Hy[l - 1], dyH = Hx[l] - Hx[l - EW];
                const float pex = xp[EW + lx] * PEx[l] + xp[2 * EW + lx] * dxH;
                PEx[l] = pex;
                const float pey = byE * PEy[l] + cyE * dyH;
                PEy[l] = pey;
                float q = xp[lx] * dxH + pex - (ayE * dyH + pey);
#pragma unroll
                for (int k = 0; k < kMaxSrc; ++k)
                    if (l == lsrc[k]) q -= wsrc[k];
                const float ez = Ca[l] * Ez[l] + Cb[l] * q;
                Ez[l] = ez;
                const int gx = X0 + lx;
                if (row_in && lx >= K && lx < K + TW && gx < p.nx) {
                    if (kHist)
                        __stcs(p.hist + ((long long)shot * p.nt + n) * p.N +
                                   (long long)gy * p.nx + gx, ez);
                    if (kIllum) ill[(ly - K) * TW + (lx - K)] += ez * ez;
                }
            }
        }
        __syncthreads();
    }

    // write the interior back
    for (int ly = K + ty; ly < K + TH; ly += kTY) {
        const int gy = Y0 + ly;
        if (gy >= p.ny) break;
        for (int lx = K + tx; lx < K + TW; lx += kTX) {
            const int gx = X0 + lx;
            if (gx >= p.nx) break;
            const int l = ly * EW + lx;
            const long long g = (long long)gy * p.nx + gx, sg = sbase + g;
            p.st_out[sg] = Ez[l];
            p.st_out[F + sg] = Hx[l];
            p.st_out[2 * F + sg] = Hy[l];
            if (in_xstrip(gx, p)) {
                p.st_out[3 * F + sg] = PEx[l];
                p.st_out[6 * F + sg] = PHy[l];
            }
            if (in_ystrip(gy, p)) {
                p.st_out[4 * F + sg] = PEy[l];
                p.st_out[5 * F + sg] = PHx[l];
            }
            if (kIllum) p.illum[sg] += ill[(ly - K) * TW + (lx - K)];
        }
    }
}

// ---------------------------------------------------------------------------------------
// Adjoint
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) adj_tile_kernel(const TileParams p) {
    extern __shared__ float4 smem_raw[];
    float* sm = reinterpret_cast<float*>(smem_raw);
    const int K = p.K, TW = p.tile_w, TH = p.tile_h;
    const int EW = TW + 2 * K, EH = TH + 2 * K, EN = EW * EH, IN = TW * TH;
    float* Ez = sm;  // adjoint of Ez^{n+1}
    float* Hx = Ez + EN;
    float* Hy = Hx + EN;
    float* Ca = Hy + EN;
    float* Cb = Ca + EN;
    float* PEx = Cb + EN;
    float* PEy = PEx + EN;
    float* PHx = PEy + EN;
    float* PHy = PHx + EN;
    float* Sx = PHy + EN;  // transposed-difference weights of the E step
    float* Sy = Sx + EN;
    float* Tx = Sy + EN;   // transposed-difference weights of the H step
    float* Ty = Tx + EN;
    float* xp = Ty + EN;
    float* yp = xp + 6 * EW;
    float* E1 = yp + 6 * EH;  // [IN] forward Ez^{n+1} of the interior
    float* Ge = E1 + IN;      // [IN] eps_r gradient accumulator
    float* Gs = Ge + IN;      // [IN] sigma gradient accumulator

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kTX + tx;
    const int shot = blockIdx.y;
    const int X0 = (blockIdx.x % p.tiles_x) * TW - K;
    const int Y0 = (blockIdx.x / p.tiles_x) * TH - K;
    const long long F = (long long)p.nshots * p.N;
    const long long sbase = (long long)shot * p.N;
    const int n1 = p.n0 + K - 1;  // first (latest) step of this launch

    for (int ly = ty; ly < EH; ly += kTY) {
        const int gy = Y0 + ly;
        for (int lx = tx; lx < EW; lx += kTX) {
            const int gx = X0 + lx, l = ly * EW + lx;
            float ez = 0.f, hx = 0.f, hy = 0.f, ca = 0.f, cb = 0.f;
            float pex = 0.f, pey = 0.f, phx = 0.f, phy = 0.f;
            const bool in = gx >= 0 && gx < p.nx && gy >= 0 && gy < p.ny;
            if (in) {
                const long long g = (long long)gy * p.nx + gx, sg = sbase + g;
                ez = p.st_in[sg];
                hx = p.st_in[F + sg];
                hy = p.st_in[2 * F + sg];
                if (in_xstrip(gx, p)) {
                    pex = p.st_in[3 * F + sg];
                    phy = p.st_in[6 * F + sg];
                }
                if (in_ystrip(gy, p)) {
                    pey = p.st_in[4 * F + sg];
                    phx = p.st_in[5 * F + sg];
                }
                const bool ring = gx == 0 || gy == 0 || gx == p.nx - 1 || gy == p.ny - 1;
                coefficients(__ldg(p.eps_r + g), __ldg(p.sigma + g), p.dt_eps0, ring, ca, cb);
            }
            Ez[l] = ez; Hx[l] = hx; Hy[l] = hy; Ca[l] = ca; Cb[l] = cb;
            PEx[l] = pex; PEy[l] = pey; PHx[l] = phx; PHy[l] = phy;
            if (lx >= K && lx < K + TW && ly >= K && ly < K + TH) {
                const int il = (ly - K) * TW + (lx - K);
                E1[il] = in ? __ldcs(p.hist + ((long long)shot * p.nt + n1) * p.N +
                                     (long long)gy * p.nx + gx)
                            : 0.f;
                Ge[il] = 0.f;
                Gs[il] = 0.f;
            }
        }
    }
    stage_profile(xp, p.px, X0, EW, p.nx, tid);
    stage_profile(yp, p.py, Y0, EH, p.ny, tid);
    __syncthreads();

    for (int s = 0; s < K; ++s) {
        const int n = n1 - s;
        // A: lam = Cb adj(Ez^{n+1}); zero-lag gradients; electric CPML memories; the E-step
        //    difference weights; adj(Ez^n) starts as Ca adj(Ez^{n+1})
        for (int ly = s + ty; ly <= EH - 1 - s; ly += kTY) {
            const float ayE = yp[ly], byE = yp[EH + ly], cyE = yp[2 * EH + ly];
            const int gy = Y0 + ly;
            const bool row_in = ly >= K && ly < K + TH && gy < p.ny;
            for (int lx = s + tx; lx <= EW - 1 - s; lx += kTX) {
                const int l = ly * EW + lx;
                const float lam = Cb[l] * Ez[l];
                const int gx = X0 + lx;
                if (row_in && lx >= K && lx < K + TW && gx < p.nx) {
                    const int il = (ly - K) * TW + (lx - K);
                    const float e1 = E1[il];
                    const float e0 = n > 0 ? __ldcs(p.hist + ((long long)shot * p.nt + n - 1) * p.N +
                                                    (long long)gy * p.nx + gx)
                                           : 0.f;
                    Ge[il] -= p.geps * lam * (e1 - e0);
                    Gs[il] -= 0.5f * lam * (e1 + e0);
                    E1[il] = e0;
                }
                const float pex = PEx[l] + lam, pey = PEy[l] - lam;
                Sx[l] = lam * xp[lx] + xp[2 * EW + lx] * pex;
                Sy[l] = -lam * ayE + cyE * pey;
                PEx[l] = xp[EW + lx] * pex;
                PEy[l] = byE * pey;
                Ez[l] = Ca[l] * Ez[l];
            }
        }
        __syncthreads();
        // B: adj(H) += transposed differences of the E step; magnetic CPML memories; the
        //    H-step difference weights
        for (int ly = s + ty; ly <= EH - 2 - s; ly += kTY) {
            const float ayH = yp[3 * EH + ly], byH = yp[4 * EH + ly], cyH = yp[5 * EH + ly];
            for (int lx = s + tx; lx <= EW - 2 - s; lx += kTX) {
                const int l = ly * EW + lx;
                const float hy = Hy[l] + Sx[l] - Sx[l + 1];
                const float hx = Hx[l] + Sy[l] - Sy[l + EW];
                Hy[l] = hy;
                Hx[l] = hx;
                const float phy = PHy[l] + p.ch * hy;
                Tx[l] = p.ch * hy * xp[3 * EW + lx] + xp[5 * EW + lx] * phy;
                PHy[l] = xp[4 * EW + lx] * phy;
                const float phx = PHx[l] - p.ch * hx;
                Ty[l] = -p.ch * hx * ayH + cyH * phx;
                PHx[l] = byH * phx;
            }
        }
        __syncthreads();
        // C: adj(Ez^n) += transposed differences of the H step
        for (int ly = s + 1 + ty; ly <= EH - 2 - s; ly += kTY) {
            for (int lx = s + 1 + tx; lx <= EW - 2 - s; lx += kTX) {
                const int l = ly * EW + lx;
                Ez[l] += Tx[l - 1] - Tx[l] + Ty[l - EW] - Ty[l];
            }
        }
        __syncthreads();
        // adjoint source: the residual of step n at every staged copy of a receiver cell
        for (int r = tid; r < p.nrec; r += kThreads) {
            const int cell = __ldg(p.rec_cell + shot * p.nrec + r);
            const int lx = cell % p.nx - X0, ly = cell / p.nx - Y0;
            if (lx >= 0 && lx < EW && ly >= 0 && ly < EH)
                atomicAdd(&Ez[ly * EW + lx], __ldg(p.resid + ((long long)shot * p.nt + n) * p.nrec + r));
        }
        __syncthreads();
    }

    for (int ly = K + ty; ly < K + TH; ly += kTY) {
        const int gy = Y0 + ly;
        if (gy >= p.ny) break;
        for (int lx = K + tx; lx < K + TW; lx += kTX) {
            const int gx = X0 + lx;
            if (gx >= p.nx) break;
            const int l = ly * EW + lx, il = (ly - K) * TW + (lx - K);
            const long long g = (long long)gy * p.nx + gx, sg = sbase + g;
            p.st_out[sg] = Ez[l];
            p.st_out[F + sg] = Hx[l];
            p.st_out[2 * F + sg] = Hy[l];
            if (in_xstrip(gx, p)) {
                p.st_out[3 * F + sg] = PEx[l];
                p.st_out[6 * F + sg] = PHy[l];
            }
            if (in_ystrip(gy, p)) {
                p.st_out[4 * F + sg] = PEy[l];
                p.st_out[5 * F + sg] = PHx[l];
            }
            p.grad[sg] += Ge[il];
            p.grad[F + sg] += Gs[il];
        }
    }
}

}  // namespace

size_t fwd_tile_smem_bytes(int tile_w, int tile_h, int K) {
    const size_t EW = tile_w + 2 * K, EH = tile_h + 2 * K;
    return sizeof(float) * (9 * EW * EH + 6 * (EW + EH) + (size_t)tile_w * tile_h);
}

size_t adj_tile_smem_bytes(int tile_w, int tile_h, int K) {
    const size_t EW = tile_w + 2 * K, EH = tile_h + 2 * K;
    return sizeof(float) * (13 * EW * EH + 6 * (EW + EH) + 3 * (size_t)tile_w * tile_h);
}

// Allow each kernel the largest dynamic shared memory that fits beside its static shared
// memory within the per-block opt-in limit `optin`.
template <class Kern>
static cudaError_t allow_smem(Kern k, size_t optin) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(optin - a.sharedSizeBytes));
}

cudaError_t configure_tile_kernels(size_t optin) {
    cudaError_t e;
    if ((e = allow_smem(fwd_tile_kernel<true, true>, optin))) return e;
    if ((e = allow_smem(fwd_tile_kernel<true, false>, optin))) return e;
    if ((e = allow_smem(fwd_tile_kernel<false, true>, optin))) return e;
    if ((e = allow_smem(fwd_tile_kernel<false, false>, optin))) return e;
    return allow_smem(adj_tile_kernel, optin);
}

size_t tile_static_smem_bytes() { return sizeof(int) * kMaxSrc; }

cudaError_t launch_fwd_tile(const TileParams& p, int tiles, cudaStream_t st) {
    const dim3 grid(tiles, p.nshots), block(kTX, kTY);
    const size_t smem = fwd_tile_smem_bytes(p.tile_w, p.tile_h, p.K);
    if (p.hist && p.illum)
        fwd_tile_kernel<true, true><<<grid, block, smem, st>>>(p);
    else if (p.hist)
        fwd_tile_kernel<true, false><<<grid, block, smem, st>>>(p);
    else if (p.illum)
        fwd_tile_kernel<false, true><<<grid, block, smem, st>>>(p);
    else
        fwd_tile_kernel<false, false><<<grid, block, smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_adj_tile(const TileParams& p, int tiles, cudaStream_t st) {
    const dim3 grid(tiles, p.nshots), block(kTX, kTY);
    adj_tile_kernel<<<grid, block, adj_tile_smem_bytes(p.tile_w, p.tile_h, p.K), st>>>(p);
    return cudaGetLastError();
}

}  // namespace gf
