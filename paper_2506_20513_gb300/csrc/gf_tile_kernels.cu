// gf_tile_kernels.cu -- temporally blocked 2-D TM FDTD forward and adjoint kernels (sm_103a).
//
// Tiling.  One CTA (64 x BY threads) owns an interior tile of tile_w x tile_h cells of one
// shot and advances it K time steps per launch.  The tile plus a K-cell halo (at most 64 x 64
// cells) stays on chip for the whole launch: thread (tx, ty) owns column tx and the RY
// consecutive rows RY*ty .. RY*ty + RY - 1 (RY * BY = 64, or 32 for the 512-thread 64 x 32
// variant), keeping their field values in registers.  Shared memory carries what neighbours
// exchange: two x-neighbour planes (Ez for the H update and Hy for the E update; the
// transposed difference weights S and T in the adjoint) and one row per thread segment for
// the y-neighbour across segments; besides, per owned cell, the CPML memory variables of strip
// cells and the update coefficients Ca, Cb (and in the adjoint the carried Ez^{n+1} and the
// two gradient accumulators), which would not fit the 64-register budget of a 1024-thread
// CTA, plus the launch's source samples and, in the adjoint, the tile's receiver positions
// and residual samples.  Each time step the valid
// region shrinks by one cell on every side (an H update reads Ez at +1, an E update reads H
// at -1), so after K steps exactly the interior is valid; it is written to the other
// ping-pong state buffer.  Halo cells are recomputed redundantly by neighbouring CTAs from
// identical inputs.  Sources and adjoint sources are injected into every staged copy of their
// cell; receivers and the wavefield history are written only by the CTA owning the cell.
// Tiles whose staged window misses every CPML strip run a specialised body without the
// memory variables (a CTA-uniform branch).
//
// Forward time step n (Algorithm 1, Sec. 3.3): record d^n = Ez^n at the receivers, update H
// and the magnetic CPML memories from Ez^n, update Ez and the electric CPML memories from
// H^{n+1/2} with Ez^{n+1} = Ca Ez^n + Cb Q (Eqs. 3-5 in the time-averaged loss form of the
// Sec. 3.2 coefficient listing), inject the source into Q (Sec. 3.2 source listing), store
// Ez^{n+1}.
//
// Adjoint time step n (Algorithm 2): the exact transpose of the forward step, in reverse:
// (A) lam = Cb * adj(Ez^{n+1}) accumulates the zero-lag gradients (Eqs. grad_eps and
// grad_sigma in discrete form) and feeds the electric CPML memories, giving the weights S of
// the transposed E-step differences, and adj(Ez^n) starts as Ca adj(Ez^{n+1}); (B) adj(H)
// receives the transposed differences of S and feeds the magnetic CPML memories, giving the
// weights T; (C) adj(Ez^n) receives the transposed differences of T and the receiver residual
// of step n.
#include "gf_internal.cuh"

namespace gf {
namespace {

constexpr int BX = 64;        // threads along x = staged tile width
constexpr int kMaxK = 31;     // tile + 2K <= 64 with tile >= 2
// The staged tile height is EHM = RY * BY (64 for variants 0 and 1, 32 for variant 3); a
// plane of the staged window holds PLANE = EHM * BX floats.

__host__ __device__ constexpr size_t smem_floats(int ry, int by) {
    return 11 * (size_t)(ry * by) * BX + 2 * by * BX + 6 * (ry * by) + 6 * BX +
           (kMaxK + 1) * kMaxSrc + kRecStage;
}

// Shared-memory carve-up (floats).
struct Smem {
    float* xplane;   // [EHM][BX] x-neighbour exchange (Ez, or S in the adjoint)
    float* xplane2;  // [EHM][BX] (Hy, or T in the adjoint)
    float* rowA;     // [BY][BX] one row per thread segment (bottom Hx, or top S_y)
    float* rowB;     // [BY][BX] (adjoint: bottom T_y)
    float* psi;      // [4][EHM][BX] CPML memories: Ex, Ey, Hx, Hy
    float* yprof;    // [6][EHM] row profiles aE bE cE aH bH cH
    float* xprof;    // [6][BX] column profiles aE bE cE aH bH cH
    float* wsrc;     // [kMaxK + 1][kMaxSrc] scaled source samples of this launch
    float* coef;     // [5][EHM][BX] adjoint: Ca, Cb, the carried Ez^{n+1} and the two
                     // gradient accumulators of the owned cells (kept here rather than in
                     // registers, which would spill)
    float* rstage;   // [kRecStage] adjoint: residual samples of the launch [entry][step] from
                     // the start, window positions lx | ly << 8 of the entries from the end
};

template <int RY, int BY>
__device__ __forceinline__ Smem carve(float* sm) {
    constexpr int EHM = RY * BY, PLANE = EHM * BX;
    Smem s;
    s.xplane = sm;
    s.xplane2 = s.xplane + PLANE;
    s.rowA = s.xplane2 + PLANE;
    s.rowB = s.rowA + BY * BX;
    s.psi = s.rowB + BY * BX;
    s.yprof = s.psi + 4 * PLANE;
    s.xprof = s.yprof + 6 * EHM;
    s.wsrc = s.xprof + 6 * BX;
    s.coef = s.wsrc + (kMaxK + 1) * kMaxSrc;
    s.rstage = s.coef + 5 * PLANE;
    return s;
}

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

// Per-thread geometry shared by both kernels.
template <int RY>
struct Cell {
    int lx, ly0, gx, X0, Y0, EWe, EHe;
    bool col_active;  // column inside the staged window and the grid
    bool col_int;     // column inside this CTA's interior and the grid
    bool xs;          // column inside an x CPML strip
    bool tile_strip;  // the staged window touches a CPML strip (CTA-uniform)

    __device__ __forceinline__ void init(const TileParams& p) {
        lx = threadIdx.x;
        ly0 = threadIdx.y * RY;
        EWe = p.tile_w + 2 * p.K;
        EHe = p.tile_h + 2 * p.K;
        X0 = (blockIdx.x % p.tiles_x) * p.tile_w - p.K;
        Y0 = (blockIdx.x / p.tiles_x) * p.tile_h - p.K;
        gx = X0 + lx;
        col_active = lx < EWe && gx >= 0 && gx < p.nx;
        col_int = lx >= p.K && lx < p.K + p.tile_w && gx < p.nx;
        xs = col_active && in_xstrip(gx, p);
        // strips: x in [0, npml) U [nx - npml - 1, nx), same for y
        const int xe = X0 + EWe - 1, ye = Y0 + EHe - 1;
        tile_strip = X0 < p.npml || xe >= p.nx - p.npml - 1 || Y0 < p.npml ||
                     ye >= p.ny - p.npml - 1;
    }
};

// Row and column CPML profiles of the staged window (clamped to the grid).
template <int EHM>
__device__ __forceinline__ void stage_profiles(const Smem& s, const TileParams& p, int X0, int Y0,
                                               int tid) {
    if (tid < EHM) {
        const int g = min(max(Y0 + tid, 0), p.ny - 1);
        s.yprof[tid] = __ldg(p.py.aE + g);
        s.yprof[EHM + tid] = __ldg(p.py.bE + g);
        s.yprof[2 * EHM + tid] = __ldg(p.py.cE + g);
        s.yprof[3 * EHM + tid] = __ldg(p.py.aH + g);
        s.yprof[4 * EHM + tid] = __ldg(p.py.bH + g);
        s.yprof[5 * EHM + tid] = __ldg(p.py.cH + g);
    } else if (tid < EHM + BX) {
        const int i = tid - EHM, g = min(max(X0 + i, 0), p.nx - 1);
        s.xprof[i] = __ldg(p.px.aE + g);
        s.xprof[BX + i] = __ldg(p.px.bE + g);
        s.xprof[2 * BX + i] = __ldg(p.px.cE + g);
        s.xprof[3 * BX + i] = __ldg(p.px.aH + g);
        s.xprof[4 * BX + i] = __ldg(p.px.bH + g);
        s.xprof[5 * BX + i] = __ldg(p.px.cH + g);
    }
}

// Load the time-stepping state of the owned cells; CPML memories of strip cells go to
// shared memory (zero elsewhere), and with kCoefSmem the update coefficients too (ca, cb are
// then left untouched).  Returns the row bit masks (y strip, interior).
template <int RY, int BY, bool kCoefSmem = false>
__device__ __forceinline__ void load_state(const TileParams& p, const Cell<RY>& c, const Smem& s,
                                           long long sbase, float* f0, float* f1, float* f2,
                                           float* ca, float* cb, unsigned& ystrip,
                                           unsigned& interior) {
    constexpr int EHM = RY * BY, PLANE = EHM * BX;
    const long long F = (long long)p.nshots * p.N;
    ystrip = 0;
    interior = 0;
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        const int ly = c.ly0 + r, gy = c.Y0 + ly, l = ly * BX + c.lx;
        const bool in = c.col_active && ly < c.EHe && gy >= 0 && gy < p.ny;
        float a = 0.f, b = 0.f, d = 0.f, cav = 0.f, cbv = 0.f;
        float pex = 0.f, pey = 0.f, phx = 0.f, phy = 0.f;
        if (in) {
            const long long g = (long long)gy * p.nx + c.gx, sg = sbase + g;
            a = p.st_in[sg];
            b = p.st_in[F + sg];
            d = p.st_in[2 * F + sg];
            const bool ys = in_ystrip(gy, p);
            if (ys) ystrip |= 1u << r;
            if (c.xs) {
                pex = p.st_in[3 * F + sg];
                phy = p.st_in[6 * F + sg];
            }
            if (ys) {
                pey = p.st_in[4 * F + sg];
                phx = p.st_in[5 * F + sg];
            }
            const bool ring = c.gx == 0 || gy == 0 || c.gx == p.nx - 1 || gy == p.ny - 1;
            coefficients(__ldg(p.eps_r + g), __ldg(p.sigma + g), p.dt_eps0, ring, cav, cbv);
            if (c.col_int && ly >= p.K && ly < p.K + p.tile_h) interior |= 1u << r;
        }
        f0[r] = a; f1[r] = b; f2[r] = d;
        if (kCoefSmem) {
            s.coef[l] = cav;
            s.coef[PLANE + l] = cbv;
        } else {
            ca[r] = cav;
            cb[r] = cbv;
        }
        if (c.tile_strip) {
            s.psi[l] = pex;
            s.psi[PLANE + l] = pey;
            s.psi[2 * PLANE + l] = phx;
            s.psi[3 * PLANE + l] = phy;
        }
    }
}

// Write the owned interior cells (fields and strip memories) to the output state.
template <int RY, int BY>
__device__ __forceinline__ void store_state(const TileParams& p, const Cell<RY>& c, const Smem& s,
                                            long long sbase, const float* f0, const float* f1,
                                            const float* f2, unsigned ystrip, unsigned interior) {
    constexpr int EHM = RY * BY, PLANE = EHM * BX;
    const long long F = (long long)p.nshots * p.N;
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        if (!((interior >> r) & 1u)) continue;
        const int ly = c.ly0 + r, l = ly * BX + c.lx;
        const long long sg = sbase + (long long)(c.Y0 + ly) * p.nx + c.gx;
        p.st_out[sg] = f0[r];
        p.st_out[F + sg] = f1[r];
        p.st_out[2 * F + sg] = f2[r];
        if (c.xs) {
            p.st_out[3 * F + sg] = s.psi[l];
            p.st_out[6 * F + sg] = s.psi[3 * PLANE + l];
        }
        if ((ystrip >> r) & 1u) {
            p.st_out[4 * F + sg] = s.psi[PLANE + l];
            p.st_out[5 * F + sg] = s.psi[2 * PLANE + l];
        }
    }
}

// Range [first, end) of the entries of this CTA's receiver list (host-built, sorted by row,
// at most 65535 entries) that covers every entry on this thread's cells, packed as
// first | end << 16 (0 when there is none).  Computed once per launch so that the per-step
// injection visits only this range (usually one entry) rather than decoding the whole list
// on every step: a thread that did so became the straggler of its CTA at every barrier.
template <int RY>
__device__ __forceinline__ unsigned owned_range(const int* __restrict__ idx, int count,
                                                const int* __restrict__ cells, int nx,
                                                const Cell<RY>& c) {
    unsigned first = 0, end = 0;
    for (int e = 0; e < count; ++e) {
        const int cell = __ldg(cells + __ldg(idx + e));
        const int lx = cell % nx - c.X0, ly = cell / nx - c.Y0 - c.ly0;
        if (lx == c.lx && ly >= 0 && ly < RY && c.lx < c.EWe && c.ly0 + ly < c.EHe) {
            if (end == 0) first = e;
            end = e + 1;
        }
    }
    return first | end << 16;
}

// ---------------------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------------------
template <int RY, int BY, bool kStrip, bool kHist, bool kIllum>
__device__ __forceinline__ void fwd_body(const TileParams& p, const Cell<RY>& c, const Smem& s,
                                         float* ez, float* hx, float* hy, float* ill, unsigned ystrip,
                                         unsigned interior, unsigned srcmask, const int* rlist,
                                         int nrl, int shot, int tid) {
    constexpr int EHM = RY * BY, PLANE = EHM * BX;
    constexpr int NTHR = BX * BY;
    const int ty = threadIdx.y, K = p.K;
    float* sEz = s.xplane;
    float* sHy = s.xplane2;
    float* sHxB = s.rowA;
    float* sPEx = s.psi;
    float* sPEy = s.psi + PLANE;
    float* sPHx = s.psi + 2 * PLANE;
    float* sPHy = s.psi + 3 * PLANE;
    const float chx = p.ch * p.rdx, chy = p.ch * p.rdy;
    // the history column of this thread: slot n, row r at hcol + n N + r nx
    float* hcol = kHist ? p.hist + ((long long)shot * p.hist_stride - p.hist_slot0) * p.N +
                              (long long)(c.Y0 + c.ly0) * p.nx + c.gx
                        : nullptr;
    const int* rec_cells = p.rec_cell + (long long)shot * p.nrec;
    float* trace_base = p.traces + (long long)shot * p.nt * p.nrec;

    for (int st = 0; st < K; ++st) {
        const int n = p.n0 + st;
        // 1. receivers of this CTA's interior: d^n = Ez^n
        for (int e = tid; e < nrl; e += NTHR) {
            const int ri = __ldg(rlist + e);
            const int cell = __ldg(rec_cells + ri);
            const int lx = cell % p.nx - c.X0, ly = cell / p.nx - c.Y0;
            if (lx >= K && lx < K + p.tile_w && ly >= K && ly < K + p.tile_h)
                trace_base[(long long)n * p.nrec + ri] = sEz[ly * BX + lx];
        }
        // 2-3. H and magnetic CPML from Ez^n
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            const int ly = c.ly0 + r, l = ly * BX + c.lx;
            const float e = ez[r];
            const float er = sEz[c.lx < BX - 1 ? l + 1 : l];
            const float ed = r < RY - 1 ? ez[r + 1] : (ly + 1 < EHM ? sEz[l + BX] : e);
            const float dxE = er - e, dyE = ed - e;
            if (kStrip && (c.xs || ((ystrip >> r) & 1u))) {
                const float ayH = s.yprof[3 * EHM + ly], byH = s.yprof[4 * EHM + ly],
                            cyH = s.yprof[5 * EHM + ly];
                const float phx = byH * sPHx[l] + cyH * dyE;
                sPHx[l] = phx;
                hx[r] -= p.ch * (ayH * dyE + phx);
                const float phy = s.xprof[4 * BX + c.lx] * sPHy[l] + s.xprof[5 * BX + c.lx] * dxE;
                sPHy[l] = phy;
                hy[r] += p.ch * (s.xprof[3 * BX + c.lx] * dxE + phy);
            } else {
                hx[r] -= chy * dyE;
                hy[r] += chx * dxE;
            }
            sHy[l] = hy[r];
        }
        sHxB[ty * BX + c.lx] = hx[RY - 1];
        __syncthreads();
        // 4-6. E, electric CPML and the source term, giving Ez^{n+1}
        float q[RY];
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            const int ly = c.ly0 + r, l = ly * BX + c.lx;
            const float hl = sHy[c.lx > 0 ? l - 1 : l];
            const float hu = r > 0 ? hx[r - 1] : (ty > 0 ? sHxB[(ty - 1) * BX + c.lx] : hx[0]);
            const float dxH = hy[r] - hl, dyH = hx[r] - hu;
            if (kStrip && (c.xs || ((ystrip >> r) & 1u))) {
                const float ayE = s.yprof[ly], byE = s.yprof[EHM + ly], cyE = s.yprof[2 * EHM + ly];
                const float pex = s.xprof[BX + c.lx] * sPEx[l] + s.xprof[2 * BX + c.lx] * dxH;
                sPEx[l] = pex;
                const float pey = byE * sPEy[l] + cyE * dyH;
                sPEy[l] = pey;
                q[r] = s.xprof[c.lx] * dxH + pex - (ayE * dyH + pey);
            } else {
                q[r] = p.rdx * dxH - p.rdy * dyH;
            }
        }
        if (srcmask) {
            for (int k = 0; k < p.nsrc; ++k) {
                const int cell = __ldg(p.src_cell + shot * p.nsrc + k);
                const int lx = cell % p.nx - c.X0, r0 = cell / p.nx - c.Y0 - c.ly0;
                if (lx != c.lx) continue;
#pragma unroll
                for (int r = 0; r < RY; ++r)
                    if (r == r0 && ((srcmask >> r) & 1u)) q[r] -= s.wsrc[st * kMaxSrc + k];
            }
        }
        float* hrow = kHist ? hcol + (long long)n * p.N : nullptr;
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            const int l = (c.ly0 + r) * BX + c.lx;
            const float v = s.coef[l] * ez[r] + s.coef[PLANE + l] * q[r];
            ez[r] = v;
            sEz[l] = v;
            if ((interior >> r) & 1u) {
                if (kHist) __stcs(hrow + r * p.nx, v);
                if (kIllum) ill[r] += v * v;
            }
        }
        __syncthreads();
    }
}

template <int RY, int BY, bool kHist, bool kIllum>
__global__ void __launch_bounds__(BX* BY, BY <= 8 && RY <= 4 ? 2 : 1) fwd_tile_kernel(const TileParams p) {
    constexpr int EHM = RY * BY, PLANE = EHM * BX;
    extern __shared__ float4 smem_raw[];
    const Smem s = carve<RY, BY>(reinterpret_cast<float*>(smem_raw));
    const int tid = threadIdx.y * BX + threadIdx.x;
    const int shot = blockIdx.y, K = p.K;
    Cell<RY> c;
    c.init(p);
    const long long sbase = (long long)shot * p.N;

    float ez[RY], hx[RY], hy[RY], ill[RY];
    unsigned ystrip, interior;
    load_state<RY, BY, true>(p, c, s, sbase, ez, hx, hy, nullptr, nullptr, ystrip, interior);
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        s.xplane[(c.ly0 + r) * BX + c.lx] = ez[r];
        ill[r] = 0.f;
    }
    stage_profiles<EHM>(s, p, c.X0, c.Y0, tid);
    for (int k = tid; k < K * kMaxSrc; k += BX * BY) {
        const int st = k / kMaxSrc, src = k % kMaxSrc;
        s.wsrc[k] = src < p.nsrc
                        ? p.src_scale * __ldg(p.wavelet + ((long long)shot * p.nsrc + src) * p.nt + p.n0 + st)
                        : 0.f;
    }
    // rows of this thread holding a source (every staged copy injects)
    unsigned srcmask = 0;
    for (int k = 0; k < p.nsrc; ++k) {
        const int cell = __ldg(p.src_cell + shot * p.nsrc + k);
        const int lx = cell % p.nx - c.X0, r0 = cell / p.nx - c.Y0 - c.ly0;
        if (lx == c.lx && r0 >= 0 && r0 < RY && c.lx < c.EWe && c.ly0 + r0 < c.EHe)
            srcmask |= 1u << r0;
    }
    const int tile = blockIdx.x;
    const long long lo = p.tile_rec_off[(long long)shot * p.ntiles + tile];
    const int nrl = (int)(p.tile_rec_off[(long long)shot * p.ntiles + tile + 1] - lo);
    const int* rlist = p.tile_rec_idx + lo;
    __syncthreads();

    if (c.tile_strip)
        fwd_body<RY, BY, true, kHist, kIllum>(p, c, s, ez, hx, hy, ill, ystrip, interior,
                                              srcmask, rlist, nrl, shot, tid);
    else
        fwd_body<RY, BY, false, kHist, kIllum>(p, c, s, ez, hx, hy, ill, ystrip, interior,
                                               srcmask, rlist, nrl, shot, tid);

    store_state<RY, BY>(p, c, s, sbase, ez, hx, hy, ystrip, interior);
    if (kIllum) {
#pragma unroll
        for (int r = 0; r < RY; ++r)
            if ((interior >> r) & 1u)
                p.illum[sbase + (long long)(c.Y0 + c.ly0 + r) * p.nx + c.gx] += ill[r];
    }
}

// ---------------------------------------------------------------------------------------
// Adjoint
// ---------------------------------------------------------------------------------------
template <int RY, int BY, bool kStrip, bool kStaged>
__device__ __forceinline__ void adj_body(const TileParams& p, const Cell<RY>& c, const Smem& s,
                                         float* aez, float* ahx, float* ahy,
                                         unsigned ystrip, unsigned interior, unsigned rrange,
                                         const int* rlist, int shot) {
    constexpr int EHM = RY * BY, PLANE = EHM * BX;
    const int ty = threadIdx.y, K = p.K;
    float* sSx = s.xplane;
    float* sTx = s.xplane2;
    float* sSyT = s.rowA;
    float* sTyB = s.rowB;
    float* sPEx = s.psi;
    float* sPEy = s.psi + PLANE;
    float* sPHx = s.psi + 2 * PLANE;
    float* sPHy = s.psi + 3 * PLANE;
    const float chx = p.ch * p.rdx, chy = p.ch * p.rdy;
    const int n1 = p.n0 + K - 1;
    const float* hcol = p.hist + ((long long)shot * p.hist_stride - p.hist_slot0) * p.N +
                        (long long)(c.Y0 + c.ly0) * p.nx + c.gx;
    const int* rec_cells = p.rec_cell + (long long)shot * p.nrec;
    const float* resid_base = p.resid + (long long)shot * p.nt * p.nrec;
    float wx[RY], wy[RY], pf[RY];

    // Ez^n of the owned cells (Ez^0 = 0), for the gradient of step n
    auto load_e0 = [&](int n) {
#pragma unroll
        for (int r = 0; r < RY; ++r)
            pf[r] = (n >= 1 && ((interior >> r) & 1u))
                        ? __ldcs(hcol + (long long)(n - 1) * p.N + r * p.nx)
                        : 0.f;
    };
    // A: gradient, electric CPML and the S weights; adj(Ez^n) starts as Ca adj(Ez^{n+1})
    auto phase_a = [&]() {
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            const int ly = c.ly0 + r, l = ly * BX + c.lx;
            const float lam = s.coef[PLANE + l] * aez[r];
            if ((interior >> r) & 1u) {
                const float en1 = s.coef[2 * PLANE + l];
                s.coef[3 * PLANE + l] -= p.geps * lam * (en1 - pf[r]);
                s.coef[4 * PLANE + l] -= 0.5f * lam * (en1 + pf[r]);
                s.coef[2 * PLANE + l] = pf[r];
            }
            if (kStrip && (c.xs || ((ystrip >> r) & 1u))) {
                const float ayE = s.yprof[ly], byE = s.yprof[EHM + ly], cyE = s.yprof[2 * EHM + ly];
                const float pex = sPEx[l] + lam, pey = sPEy[l] - lam;
                wx[r] = lam * s.xprof[c.lx] + s.xprof[2 * BX + c.lx] * pex;
                wy[r] = -lam * ayE + cyE * pey;
                sPEx[l] = s.xprof[BX + c.lx] * pex;
                sPEy[l] = byE * pey;
            } else {
                wx[r] = lam * p.rdx;
                wy[r] = -lam * p.rdy;
            }
            sSx[l] = wx[r];
            aez[r] *= s.coef[l];
        }
        sSyT[ty * BX + c.lx] = wy[0];
    };

    load_e0(n1);
    phase_a();
    for (int st = 0; st < K; ++st) {
        const int n = n1 - st;
        __syncthreads();
        if (st < K - 1) load_e0(n - 1);  // prefetch for the gradient of step n - 1
        // B: adj(H) += transposed S differences; magnetic CPML; T weights.  Rows go upwards
        // so that wy[r + 1] still holds S_y when row r reads it.
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            const int ly = c.ly0 + r, l = ly * BX + c.lx;
            const float sxr = sSx[c.lx < BX - 1 ? l + 1 : l];
            const float syd = r < RY - 1 ? wy[r + 1] : (ty < BY - 1 ? sSyT[(ty + 1) * BX + c.lx] : wy[r]);
            const float hyv = ahy[r] + wx[r] - sxr;
            const float hxv = ahx[r] + wy[r] - syd;
            ahy[r] = hyv;
            ahx[r] = hxv;
            if (kStrip && (c.xs || ((ystrip >> r) & 1u))) {
                const float ayH = s.yprof[3 * EHM + ly], byH = s.yprof[4 * EHM + ly],
                            cyH = s.yprof[5 * EHM + ly];
                const float phy = sPHy[l] + p.ch * hyv;
                wx[r] = p.ch * hyv * s.xprof[3 * BX + c.lx] + s.xprof[5 * BX + c.lx] * phy;
                sPHy[l] = s.xprof[4 * BX + c.lx] * phy;
                const float phx = sPHx[l] - p.ch * hxv;
                wy[r] = -p.ch * hxv * ayH + cyH * phx;
                sPHx[l] = byH * phx;
            } else {
                wx[r] = chx * hyv;
                wy[r] = -chy * hxv;
            }
            sTx[l] = wx[r];
        }
        sTyB[ty * BX + c.lx] = wy[RY - 1];
        __syncthreads();
        // C: adj(Ez^n) += transposed T differences; adjoint source of step n
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            const int l = (c.ly0 + r) * BX + c.lx;
            const float tl = sTx[c.lx > 0 ? l - 1 : l];
            const float tu = r > 0 ? wy[r - 1] : (ty > 0 ? sTyB[(ty - 1) * BX + c.lx] : wy[0]);
            aez[r] += tl - wx[r] + tu - wy[r];
        }
        for (int e = rrange & 0xffffu; e < (int)(rrange >> 16); ++e) {
            int r0;
            float v;
            if (kStaged) {
                const int pos = __float_as_int(s.rstage[kRecStage - 1 - e]);
                r0 = (pos >> 8) - c.ly0;
                if ((pos & 0xff) != c.lx || r0 < 0 || r0 >= RY) continue;
                v = s.rstage[e * K + st];
            } else {
                const int ri = __ldg(rlist + e);
                const int cell = __ldg(rec_cells + ri);
                r0 = cell / p.nx - c.Y0 - c.ly0;
                if (cell % p.nx - c.X0 != c.lx || r0 < 0 || r0 >= RY) continue;
                v = __ldg(resid_base + (long long)n * p.nrec + ri);
            }
#pragma unroll
            for (int r = 0; r < RY; ++r)
                if (r == r0) aez[r] += v;
        }
        if (st < K - 1) phase_a();
    }
}

template <int RY, int BY, bool kStaged>
__global__ void __launch_bounds__(BX* BY, BY <= 8 && RY <= 4 ? 2 : 1) adj_tile_kernel(const TileParams p) {
    constexpr int EHM = RY * BY, PLANE = EHM * BX;
    extern __shared__ float4 smem_raw[];
    const Smem s = carve<RY, BY>(reinterpret_cast<float*>(smem_raw));
    const int tid = threadIdx.y * BX + threadIdx.x;
    const int shot = blockIdx.y, K = p.K;
    Cell<RY> c;
    c.init(p);
    const long long sbase = (long long)shot * p.N;
    const int n1 = p.n0 + K - 1;

    float aez[RY], ahx[RY], ahy[RY];
    unsigned ystrip, interior;
    load_state<RY, BY, true>(p, c, s, sbase, aez, ahx, ahy, nullptr, nullptr, ystrip, interior);
    const float* hcol = p.hist + ((long long)shot * p.hist_stride - p.hist_slot0) * p.N +
                        (long long)(c.Y0 + c.ly0) * p.nx + c.gx;
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        s.coef[3 * PLANE + (c.ly0 + r) * BX + c.lx] = 0.f;
        s.coef[4 * PLANE + (c.ly0 + r) * BX + c.lx] = 0.f;
        s.coef[2 * PLANE + (c.ly0 + r) * BX + c.lx] =
            ((interior >> r) & 1u) ? __ldcs(hcol + (long long)n1 * p.N + r * p.nx) : 0.f;
    }
    stage_profiles<EHM>(s, p, c.X0, c.Y0, tid);
    const int tile = blockIdx.x;
    const long long lo = p.tile_rec_off[(long long)shot * p.ntiles + tile];
    const int nrl = (int)(p.tile_rec_off[(long long)shot * p.ntiles + tile + 1] - lo);
    const int* rlist = p.tile_rec_idx + lo;
    const unsigned rrange =
        owned_range<RY>(rlist, nrl, p.rec_cell + (long long)shot * p.nrec, p.nx, c);
    if (kStaged) {
        // the receivers' window positions and the residual samples of this launch, so that
        // the per-step injection reads shared memory only (nrl * (K + 1) <= kRecStage)
        const int* rc = p.rec_cell + (long long)shot * p.nrec;
        for (int e = tid; e < nrl; e += BX * BY) {
            const int cell = __ldg(rc + __ldg(rlist + e));
            s.rstage[kRecStage - 1 - e] =
                __int_as_float((cell % p.nx - c.X0) | (cell / p.nx - c.Y0) << 8);
        }
        const float* rb = p.resid + (long long)shot * p.nt * p.nrec;
        for (int i = tid; i < nrl * K; i += BX * BY) {
            const int e = i / K, st = i - e * K;
            s.rstage[i] = __ldg(rb + (long long)(n1 - st) * p.nrec + __ldg(rlist + e));
        }
    }
    __syncthreads();

    if (c.tile_strip)
        adj_body<RY, BY, true, kStaged>(p, c, s, aez, ahx, ahy, ystrip, interior, rrange, rlist,
                                        shot);
    else
        adj_body<RY, BY, false, kStaged>(p, c, s, aez, ahx, ahy, ystrip, interior, rrange, rlist,
                                         shot);

    store_state<RY, BY>(p, c, s, sbase, aez, ahx, ahy, ystrip, interior);
    const long long F = (long long)p.nshots * p.N;
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        if (!((interior >> r) & 1u)) continue;
        const long long sg = sbase + (long long)(c.Y0 + c.ly0 + r) * p.nx + c.gx;
        // one writer per cell per launch and launches in stream order: a fire-and-forget
        // reduction is deterministic and hides the read latency of += at the end of the CTA
        const int l = (c.ly0 + r) * BX + c.lx;
        atomicAdd(p.grad + sg, s.coef[3 * PLANE + l]);
        atomicAdd(p.grad + F + sg, s.coef[4 * PLANE + l]);
    }
}

// Allow a kernel the largest dynamic shared memory that fits beside its static shared memory
// within the per-block opt-in limit.
template <class Kern>
cudaError_t allow_smem(Kern k, size_t optin) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(optin - a.sharedSizeBytes));
}

template <int RY, int BY>
cudaError_t configure_variant(size_t optin) {
    cudaError_t e;
    if ((e = allow_smem(fwd_tile_kernel<RY, BY, true, true>, optin))) return e;
    if ((e = allow_smem(fwd_tile_kernel<RY, BY, true, false>, optin))) return e;
    if ((e = allow_smem(fwd_tile_kernel<RY, BY, false, true>, optin))) return e;
    if ((e = allow_smem(fwd_tile_kernel<RY, BY, false, false>, optin))) return e;
    if ((e = allow_smem(adj_tile_kernel<RY, BY, true>, optin))) return e;
    return allow_smem(adj_tile_kernel<RY, BY, false>, optin);
}

template <int RY, int BY>
cudaError_t launch_fwd_variant(const TileParams& p, cudaStream_t st) {
    const dim3 grid(p.ntiles, p.nshots), block(BX, BY);
    const size_t smem = sizeof(float) * smem_floats(RY, BY);
    if (p.hist && p.illum)
        fwd_tile_kernel<RY, BY, true, true><<<grid, block, smem, st>>>(p);
    else if (p.hist)
        fwd_tile_kernel<RY, BY, true, false><<<grid, block, smem, st>>>(p);
    else if (p.illum)
        fwd_tile_kernel<RY, BY, false, true><<<grid, block, smem, st>>>(p);
    else
        fwd_tile_kernel<RY, BY, false, false><<<grid, block, smem, st>>>(p);
    return cudaGetLastError();
}

template <int RY, int BY>
cudaError_t launch_adj_variant(const TileParams& p, cudaStream_t st) {
    const dim3 grid(p.ntiles, p.nshots), block(BX, BY);
    const size_t smem = sizeof(float) * smem_floats(RY, BY);
    if (p.rec_staged)
        adj_tile_kernel<RY, BY, true><<<grid, block, smem, st>>>(p);
    else
        adj_tile_kernel<RY, BY, false><<<grid, block, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace

int max_tile_extent() { return BX; }
int max_tile_height(int variant) { return variant == 3 ? 32 : 64; }
int num_tile_variants() { return 3; }

size_t tile_smem_bytes(int variant) {
    return sizeof(float) * (variant == 0 ? smem_floats(4, 16)
                            : variant == 1 ? smem_floats(8, 8)
                                           : smem_floats(4, 8));
}

cudaError_t configure_tile_kernels(size_t optin) {
    cudaError_t e = configure_variant<4, 16>(optin);
    if (e != cudaSuccess) return e;
    if ((e = configure_variant<8, 8>(optin)) != cudaSuccess) return e;
    return configure_variant<4, 8>(optin);
}

// Variant 0: 4 rows per thread, 1024 threads, 64 x 64 window; variant 1: 8 rows per thread,
// 512 threads, 64 x 64; variant 3: 4 rows per thread, 512 threads, 64 x 32 window, two CTAs
// per SM (one CTA's barrier waits and state loads overlap the other's work).
cudaError_t launch_fwd_tile(const TileParams& p, int variant, cudaStream_t st) {
    return variant == 0   ? launch_fwd_variant<4, 16>(p, st)
           : variant == 1 ? launch_fwd_variant<8, 8>(p, st)
                          : launch_fwd_variant<4, 8>(p, st);
}

cudaError_t launch_adj_tile(const TileParams& p, int variant, cudaStream_t st) {
    return variant == 0   ? launch_adj_variant<4, 16>(p, st)
           : variant == 1 ? launch_adj_variant<8, 8>(p, st)
                          : launch_adj_variant<4, 8>(p, st);
}

}  // namespace gf
