// gf_tile_kernels.cu -- temporally blocked 2-D TM FDTD forward and adjoint kernels (sm_103a).
//
// Tiling.  One CTA (64 x 8 threads) owns an interior tile of tile_w x tile_h cells of one
// shot and advances it K time steps per launch.  The tile plus a K-cell halo (at most 64 x 64
// cells) is held on chip for the whole launch: thread (tx, ty) owns column tx and the eight
// consecutive rows 8 ty .. 8 ty + 7, keeping their field values, update coefficients and
// accumulators in registers.  Shared memory only carries what neighbours need: the x-neighbour
// planes (Ez for the H update, Hy for the E update; the transposed-difference weights in the
// adjoint), one row per thread segment for the y-neighbour across segments, and the CPML memory
// variables of the cells in the absorbing strips.  Each time step the valid region shrinks by
// one cell on every side (an H update reads Ez at +1, an E update reads H at -1), so after K
// steps exactly the interior is valid and is written to the other ping-pong state buffer; halo
// cells are recomputed redundantly by neighbouring CTAs from identical inputs.  Sources and
// adjoint sources are injected into every staged copy of their cell; receivers and the
// wavefield history are written only by the CTA that owns the cell.
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

constexpr int BX = 64;                // threads along x = staged tile width
constexpr int BY = 8;                 // thread rows
constexpr int RY = 8;                 // cells per thread along y
constexpr int EHM = BY * RY;          // staged tile height
constexpr int NTHR = BX * BY;         // 512 threads
constexpr int PLANE = EHM * BX;       // cells of one staged plane
constexpr int kMaxK = 31;             // tile_w + 2K <= 64 with tile_w >= 2

struct Entry {
    int l;    // staged cell index ly * BX + lx
    int idx;  // receiver or source index within the shot
};

// Shared-memory layout common to both kernels (floats unless noted).
struct Smem {
    float* xplane;   // [EHM][BX] x-neighbour exchange (Ez or S)
    float* xplane2;  // [EHM][BX] second x-neighbour plane (Hy or T)
    float* rowA;     // [BY][BX] one row per thread segment (bottom Hx, or top S_y)
    float* rowB;     // [BY][BX] (adjoint: bottom T_y)
    float* psi;      // [4][EHM][BX] CPML memories of strip cells: Ex, Ey, Hx, Hy
    float* yprof;    // [6][EHM] row profiles aE bE cE aH bH cH
    float* wsrc;     // [kMaxK + 1][kMaxSrc] scaled source samples of this launch
    int* scan;       // [NTHR]
    unsigned* mask;  // [BY][BX] per-thread-segment bit masks of listed cells
    Entry* list;     // [kMaxCtaRec] receivers (or sources) of this CTA, in index order
};

__host__ __device__ constexpr size_t smem_floats() {
    return 2 * PLANE + 2 * BY * BX + 4 * PLANE + 6 * EHM + (kMaxK + 1) * kMaxSrc;
}
__host__ __device__ constexpr size_t smem_bytes() {
    return sizeof(float) * smem_floats() + sizeof(int) * NTHR + sizeof(unsigned) * BY * BX +
           sizeof(Entry) * kMaxCtaRec;
}

__device__ __forceinline__ Smem carve(float* sm) {
    Smem s;
    s.xplane = sm;
    s.xplane2 = s.xplane + PLANE;
    s.rowA = s.xplane2 + PLANE;
    s.rowB = s.rowA + BY * BX;
    s.psi = s.rowB + BY * BX;
    s.yprof = s.psi + 4 * PLANE;
    s.wsrc = s.yprof + 6 * EHM;
    s.scan = reinterpret_cast<int*>(s.wsrc + (kMaxK + 1) * kMaxSrc);
    s.mask = reinterpret_cast<unsigned*>(s.scan + NTHR);
    s.list = reinterpret_cast<Entry*>(s.mask + BY * BX);
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

// Exclusive prefix sum of one int per thread (shared-memory Hillis-Steele), block total.
__device__ int block_exclusive_scan(int v, int* buf, int tid, int& total) {
    buf[tid] = v;
    __syncthreads();
    for (int off = 1; off < NTHR; off <<= 1) {
        const int t = tid >= off ? buf[tid - off] : 0;
        __syncthreads();
        buf[tid] += t;
        __syncthreads();
    }
    total = buf[NTHR - 1];
    const int incl = buf[tid];
    __syncthreads();
    return incl - v;
}

// Collect, in index order, the items k < count whose cell lies in the staged window
// [xlo, xhi) x [ylo, yhi); set the owning thread's mask bit for each.  Returns the count (the
// host guarantees it fits the list).
__device__ int collect(const int* __restrict__ cells, int count, int nx, int X0, int Y0,
                       int xlo, int xhi, int ylo, int yhi, const Smem& s, int tid) {
    const int chunk = (count + NTHR - 1) / NTHR;
    const int k0 = min(tid * chunk, count), k1 = min(k0 + chunk, count);
    int mine = 0;
    for (int k = k0; k < k1; ++k) {
        const int c = __ldg(cells + k);
        const int lx = c % nx - X0, ly = c / nx - Y0;
        mine += (lx >= xlo && lx < xhi && ly >= ylo && ly < yhi);
    }
    int total;
    int off = block_exclusive_scan(mine, s.scan, tid, total);
    for (int k = k0; k < k1; ++k) {
        const int c = __ldg(cells + k);
        const int lx = c % nx - X0, ly = c / nx - Y0;
        if (lx >= xlo && lx < xhi && ly >= ylo && ly < yhi) {
            if (off < kMaxCtaRec) s.list[off] = Entry{ly * BX + lx, k};
            ++off;
            atomicOr(&s.mask[(ly / RY) * BX + lx], 1u << (ly % RY));
        }
    }
    __syncthreads();
    return min(total, kMaxCtaRec);
}

// Row profiles of the staged rows (clamped to the grid).
__device__ __forceinline__ void stage_rows(const Smem& s, const AxisProfile& a, int Y0, int ny,
                                           int tid) {
    if (tid < EHM) {
        const int g = min(max(Y0 + tid, 0), ny - 1);
        s.yprof[tid] = __ldg(a.aE + g);
        s.yprof[EHM + tid] = __ldg(a.bE + g);
        s.yprof[2 * EHM + tid] = __ldg(a.cE + g);
        s.yprof[3 * EHM + tid] = __ldg(a.aH + g);
        s.yprof[4 * EHM + tid] = __ldg(a.bH + g);
        s.yprof[5 * EHM + tid] = __ldg(a.cH + g);
    }
}

// Per-thread geometry shared by both kernels.
struct Cell {
    int lx, ly0, gx, X0, Y0, EWe, EHe;
    bool col_active;  // column inside the staged window and the grid
    bool xs;          // column inside an x CPML strip
    float axE, bxE, cxE, axH, bxH, cxH;  // column profiles
};

__device__ __forceinline__ Cell cell_geometry(const TileParams& p) {
    Cell c;
    c.lx = threadIdx.x;
    c.ly0 = threadIdx.y * RY;
    c.EWe = p.tile_w + 2 * p.K;
    c.EHe = p.tile_h + 2 * p.K;
    c.X0 = (blockIdx.x % p.tiles_x) * p.tile_w - p.K;
    c.Y0 = (blockIdx.x / p.tiles_x) * p.tile_h - p.K;
    c.gx = c.X0 + c.lx;
    c.col_active = c.lx < c.EWe && c.gx >= 0 && c.gx < p.nx;
    c.xs = c.col_active && in_xstrip(c.gx, p);
    const int g = min(max(c.gx, 0), p.nx - 1);
    c.axE = __ldg(p.px.aE + g);
    c.bxE = __ldg(p.px.bE + g);
    c.cxE = __ldg(p.px.cE + g);
    c.axH = __ldg(p.px.aH + g);
    c.bxH = __ldg(p.px.bH + g);
    c.cxH = __ldg(p.px.cH + g);
    return c;
}

// ---------------------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------------------
template <bool kHist, bool kIllum>
__global__ void __launch_bounds__(NTHR, 1) fwd_tile_kernel(const TileParams p) {
    extern __shared__ float4 smem_raw[];
    const Smem s = carve(reinterpret_cast<float*>(smem_raw));
    float* sEz = s.xplane;
    float* sHy = s.xplane2;
    float* sHxB = s.rowA;
    float* sPEx = s.psi;
    float* sPEy = s.psi + PLANE;
    float* sPHx = s.psi + 2 * PLANE;
    float* sPHy = s.psi + 3 * PLANE;
    __shared__ Entry s_src[kMaxSrc];

    const int tid = threadIdx.y * BX + threadIdx.x, ty = threadIdx.y;
    const int shot = blockIdx.y, K = p.K;
    const Cell c = cell_geometry(p);
    const long long F = (long long)p.nshots * p.N;
    const long long sbase = (long long)shot * p.N;
    // off the CPML strips kappa = 1 and the memories vanish: a = 1/d, plain differences
    const float chx = p.ch * p.rdx, chy = p.ch * p.rdy;

    float ez[RY], hx[RY], hy[RY], ca[RY], cb[RY], ill[RY];
    unsigned ystrip = 0;     // rows inside a y CPML strip
    unsigned interior = 0;   // rows of cells this CTA owns (written back, history)
    const bool col_int = c.lx >= K && c.lx < K + p.tile_w && c.gx < p.nx;
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        const int ly = c.ly0 + r, gy = c.Y0 + ly, l = ly * BX + c.lx;
        const bool in = c.col_active && ly < c.EHe && gy >= 0 && gy < p.ny;
        float e = 0.f, hxv = 0.f, hyv = 0.f, cav = 0.f, cbv = 0.f;
        float pex = 0.f, pey = 0.f, phx = 0.f, phy = 0.f;
        if (in) {
            const long long g = (long long)gy * p.nx + c.gx, sg = sbase + g;
            e = p.st_in[sg];
            hxv = p.st_in[F + sg];
            hyv = p.st_in[2 * F + sg];
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
            if (col_int && ly >= K && ly < K + p.tile_h) interior |= 1u << r;
        }
        ez[r] = e; hx[r] = hxv; hy[r] = hyv; ca[r] = cav; cb[r] = cbv; ill[r] = 0.f;
        sPEx[l] = pex; sPEy[l] = pey; sPHx[l] = phx; sPHy[l] = phy;
        sEz[l] = e;
    }
    stage_rows(s, p.py, c.Y0, p.ny, tid);
    for (int k = tid; k < K * kMaxSrc; k += NTHR) {
        const int st = k / kMaxSrc, src = k % kMaxSrc;
        s.wsrc[k] = src < p.nsrc ? p.src_scale * __ldg(p.wavelet + ((long long)shot * p.nsrc + src) * p.nt + p.n0 + st)
                                 : 0.f;
    }
    s.mask[tid] = 0u;
    if (tid < kMaxSrc) {
        int l = -1;
        if (tid < p.nsrc) {
            const int cell = __ldg(p.src_cell + shot * p.nsrc + tid);
            const int lx = cell % p.nx - c.X0, ly = cell / p.nx - c.Y0;
            if (lx >= 0 && lx < c.EWe && ly >= 0 && ly < c.EHe) l = ly * BX + lx;
        }
        s_src[tid] = Entry{l, tid};
    }
    // receivers owned by this CTA (interior window), in index order (collect() synchronises)
    const int nrl = collect(p.rec_cell + (long long)shot * p.nrec, p.nrec, p.nx, c.X0, c.Y0, K,
                           K + p.tile_w, K, K + p.tile_h, s, tid);
    // rows of this thread that hold a source (every staged copy injects)
    unsigned srcmask = 0;
#pragma unroll
    for (int k = 0; k < kMaxSrc; ++k) {
        const int l = s_src[k].l;
        if (l >= 0 && l % BX == c.lx && l / BX >= c.ly0 && l / BX < c.ly0 + RY)
            srcmask |= 1u << (l / BX - c.ly0);
    }

    for (int st = 0; st < K; ++st) {
        const int n = p.n0 + st;
        // 1. receivers: d^n = Ez^n
        for (int e = tid; e < nrl; e += NTHR)
            p.traces[((long long)shot * p.nt + n) * p.nrec + s.list[e].idx] = sEz[s.list[e].l];
        // 2-3. H and magnetic CPML from Ez^n
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            const int ly = c.ly0 + r, l = ly * BX + c.lx;
            const float e = ez[r];
            const float er = sEz[c.lx < BX - 1 ? l + 1 : l];
            const float ed = r < RY - 1 ? ez[r + 1] : (ly + 1 < EHM ? sEz[l + BX] : e);
            const float dxE = er - e, dyE = ed - e;
            if (c.xs || ((ystrip >> r) & 1u)) {
                const float ayH = s.yprof[3 * EHM + ly], byH = s.yprof[4 * EHM + ly],
                            cyH = s.yprof[5 * EHM + ly];
                const float phx = byH * sPHx[l] + cyH * dyE;
                sPHx[l] = phx;
                hx[r] -= p.ch * (ayH * dyE + phx);
                const float phy = c.bxH * sPHy[l] + c.cxH * dxE;
                sPHy[l] = phy;
                hy[r] += p.ch * (c.axH * dxE + phy);
            } else {
                hx[r] -= chy * dyE;
                hy[r] += chx * dxE;
            }
            sHy[l] = hy[r];
        }
        sHxB[ty * BX + c.lx] = hx[RY - 1];
        __syncthreads();
        // 4-6. E, electric CPML and the source term, giving Ez^{n+1}
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            const int ly = c.ly0 + r, l = ly * BX + c.lx;
            const float hl = sHy[c.lx > 0 ? l - 1 : l];
            const float hu = r > 0 ? hx[r - 1] : (ty > 0 ? sHxB[(ty - 1) * BX + c.lx] : hx[0]);
            const float dxH = hy[r] - hl, dyH = hx[r] - hu;
            float q;
            if (c.xs || ((ystrip >> r) & 1u)) {
                const float ayE = s.yprof[ly], byE = s.yprof[EHM + ly], cyE = s.yprof[2 * EHM + ly];
                const float pex = c.bxE * sPEx[l] + c.cxE * dxH;
                sPEx[l] = pex;
                const float pey = byE * sPEy[l] + cyE * dyH;
                sPEy[l] = pey;
                q = c.axE * dxH + pex - (ayE * dyH + pey);
            } else {
                q = p.rdx * dxH - p.rdy * dyH;
            }
            if ((srcmask >> r) & 1u) {
#pragma unroll
                for (int k = 0; k < kMaxSrc; ++k)
                    if (s_src[k].l == l) q -= s.wsrc[st * kMaxSrc + k];
            }
            const float v = ca[r] * ez[r] + cb[r] * q;
            ez[r] = v;
            sEz[l] = v;
            if ((interior >> r) & 1u) {
                const long long g = (long long)(c.Y0 + ly) * p.nx + c.gx;
                if (kHist) __stcs(p.hist + ((long long)shot * p.nt + n) * p.N + g, v);
                if (kIllum) ill[r] += v * v;
            }
        }
        __syncthreads();
    }

    // write the interior back
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        if (!((interior >> r) & 1u)) continue;
        const int ly = c.ly0 + r, gy = c.Y0 + ly, l = ly * BX + c.lx;
        const long long g = (long long)gy * p.nx + c.gx, sg = sbase + g;
        p.st_out[sg] = ez[r];
        p.st_out[F + sg] = hx[r];
        p.st_out[2 * F + sg] = hy[r];
        if (c.xs) {
            p.st_out[3 * F + sg] = sPEx[l];
            p.st_out[6 * F + sg] = sPHy[l];
        }
        if ((ystrip >> r) & 1u) {
            p.st_out[4 * F + sg] = sPEy[l];
            p.st_out[5 * F + sg] = sPHx[l];
        }
        if (kIllum) p.illum[sg] += ill[r];
    }
}

// ---------------------------------------------------------------------------------------
// Adjoint
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(NTHR, 1) adj_tile_kernel(const TileParams p) {
    extern __shared__ float4 smem_raw[];
    const Smem s = carve(reinterpret_cast<float*>(smem_raw));
    float* sSx = s.xplane;    // S_x weights (x-neighbour exchange)
    float* sTx = s.xplane2;   // T_x weights
    float* sSyT = s.rowA;     // S_y of each segment's top row
    float* sTyB = s.rowB;     // T_y of each segment's bottom row
    float* sPEx = s.psi;
    float* sPEy = s.psi + PLANE;
    float* sPHx = s.psi + 2 * PLANE;
    float* sPHy = s.psi + 3 * PLANE;

    const int tid = threadIdx.y * BX + threadIdx.x, ty = threadIdx.y;
    const int shot = blockIdx.y, K = p.K;
    const Cell c = cell_geometry(p);
    const long long F = (long long)p.nshots * p.N;
    const long long sbase = (long long)shot * p.N;
    const long long hbase = (long long)shot * p.nt * p.N;
    const float chx = p.ch * p.rdx, chy = p.ch * p.rdy;
    const int n1 = p.n0 + K - 1;  // latest step of this launch

    float aez[RY], ahx[RY], ahy[RY], ca[RY], cb[RY], ge[RY], gs[RY], e1[RY], wx[RY], wy[RY];
    unsigned ystrip = 0, interior = 0;
    const bool col_int = c.lx >= K && c.lx < K + p.tile_w && c.gx < p.nx;
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        const int ly = c.ly0 + r, gy = c.Y0 + ly, l = ly * BX + c.lx;
        const bool in = c.col_active && ly < c.EHe && gy >= 0 && gy < p.ny;
        float e = 0.f, hxv = 0.f, hyv = 0.f, cav = 0.f, cbv = 0.f, h1 = 0.f;
        float pex = 0.f, pey = 0.f, phx = 0.f, phy = 0.f;
        if (in) {
            const long long g = (long long)gy * p.nx + c.gx, sg = sbase + g;
            e = p.st_in[sg];
            hxv = p.st_in[F + sg];
            hyv = p.st_in[2 * F + sg];
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
            if (col_int && ly >= K && ly < K + p.tile_h) {
                interior |= 1u << r;
                h1 = __ldcs(p.hist + hbase + (long long)n1 * p.N + g);  // Ez^{n1+1}
            }
        }
        aez[r] = e; ahx[r] = hxv; ahy[r] = hyv; ca[r] = cav; cb[r] = cbv;
        ge[r] = 0.f; gs[r] = 0.f; e1[r] = h1;
        sPEx[l] = pex; sPEy[l] = pey; sPHx[l] = phx; sPHy[l] = phy;
    }
    stage_rows(s, p.py, c.Y0, p.ny, tid);
    s.mask[tid] = 0u;
    __syncthreads();
    // receivers of every staged cell (all copies inject), in index order
    const int nrl = collect(p.rec_cell + (long long)shot * p.nrec, p.nrec, p.nx, c.X0, c.Y0, 0,
                           c.EWe, 0, c.EHe, s, tid);
    const unsigned recmask = s.mask[ty * BX + c.lx];

    // Ez^n of the owned cells for the gradient of step n (Ez^0 = 0)
    auto load_e0 = [&](int n, float* dst) {
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            float v = 0.f;
            if (n >= 1 && ((interior >> r) & 1u)) {
                const long long g = (long long)(c.Y0 + c.ly0 + r) * p.nx + c.gx;
                v = __ldcs(p.hist + hbase + (long long)(n - 1) * p.N + g);
            }
            dst[r] = v;
        }
    };
    // A: gradient, electric CPML, S weights; adj(Ez^n) starts as Ca adj(Ez^{n+1})
    auto phase_a = [&](const float* e0) {
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            const int ly = c.ly0 + r, l = ly * BX + c.lx;
            const float lam = cb[r] * aez[r];
            if ((interior >> r) & 1u) {
                ge[r] -= p.geps * lam * (e1[r] - e0[r]);
                gs[r] -= 0.5f * lam * (e1[r] + e0[r]);
                e1[r] = e0[r];
            }
            float sx, sy;
            if (c.xs || ((ystrip >> r) & 1u)) {
                const float ayE = s.yprof[ly], byE = s.yprof[EHM + ly], cyE = s.yprof[2 * EHM + ly];
                const float pex = sPEx[l] + lam, pey = sPEy[l] - lam;
                sx = lam * c.axE + c.cxE * pex;
                sy = -lam * ayE + cyE * pey;
                sPEx[l] = c.bxE * pex;
                sPEy[l] = byE * pey;
            } else {
                sx = lam * p.rdx;
                sy = -lam * p.rdy;
            }
            wx[r] = sx;
            wy[r] = sy;
            sSx[l] = sx;
            aez[r] *= ca[r];
        }
        sSyT[ty * BX + c.lx] = wy[0];
    };

    float pf[RY];
    load_e0(n1, pf);
    phase_a(pf);
    for (int st = 0; st < K; ++st) {
        const int n = n1 - st;
        __syncthreads();
        // prefetch Ez^{n-1} for the gradient of step n - 1
        if (st < K - 1) load_e0(n - 1, pf);
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
            float tx, tyv;
            if (c.xs || ((ystrip >> r) & 1u)) {
                const float ayH = s.yprof[3 * EHM + ly], byH = s.yprof[4 * EHM + ly],
                            cyH = s.yprof[5 * EHM + ly];
                const float phy = sPHy[l] + p.ch * hyv;
                tx = p.ch * hyv * c.axH + c.cxH * phy;
                sPHy[l] = c.bxH * phy;
                const float phx = sPHx[l] - p.ch * hxv;
                tyv = -p.ch * hxv * ayH + cyH * phx;
                sPHx[l] = byH * phx;
            } else {
                tx = chx * hyv;
                tyv = -chy * hxv;
            }
            wx[r] = tx;
            wy[r] = tyv;
            sTx[l] = tx;
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
        if (recmask) {
            for (int e = 0; e < nrl; ++e) {
                const int l = s.list[e].l;
                const int r = l / BX - c.ly0;
                if (l % BX != c.lx || r < 0 || r >= RY) continue;
                const float v = __ldg(p.resid + ((long long)shot * p.nt + n) * p.nrec + s.list[e].idx);
#pragma unroll
                for (int q = 0; q < RY; ++q)
                    if (q == r) aez[q] += v;
            }
        }
        if (st < K - 1) phase_a(pf);
    }

#pragma unroll
    for (int r = 0; r < RY; ++r) {
        if (!((interior >> r) & 1u)) continue;
        const int ly = c.ly0 + r, gy = c.Y0 + ly, l = ly * BX + c.lx;
        const long long g = (long long)gy * p.nx + c.gx, sg = sbase + g;
        p.st_out[sg] = aez[r];
        p.st_out[F + sg] = ahx[r];
        p.st_out[2 * F + sg] = ahy[r];
        if (c.xs) {
            p.st_out[3 * F + sg] = sPEx[l];
            p.st_out[6 * F + sg] = sPHy[l];
        }
        if ((ystrip >> r) & 1u) {
            p.st_out[4 * F + sg] = sPEy[l];
            p.st_out[5 * F + sg] = sPHx[l];
        }
        p.grad[sg] += ge[r];
        p.grad[F + sg] += gs[r];
    }
}

}  // namespace

int max_tile_extent() { return BX; }
size_t fwd_tile_smem_bytes() { return smem_bytes(); }
size_t adj_tile_smem_bytes() { return smem_bytes(); }
size_t tile_static_smem_bytes() { return sizeof(Entry) * kMaxSrc; }

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

cudaError_t launch_fwd_tile(const TileParams& p, int tiles, cudaStream_t st) {
    const dim3 grid(tiles, p.nshots), block(BX, BY);
    const size_t smem = smem_bytes();
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
    const dim3 grid(tiles, p.nshots), block(BX, BY);
    adj_tile_kernel<<<grid, block, smem_bytes(), st>>>(p);
    return cudaGetLastError();
}

}  // namespace gf
