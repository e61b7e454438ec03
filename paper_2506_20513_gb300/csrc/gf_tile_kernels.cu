// gf_tile_kernels.cu -- temporally blocked 2-D TM FDTD forward and adjoint kernels (sm_103a).
//
// Tiling.  One CTA owns an interior tile of tile_w x tile_h cells of one shot and advances it
// K time steps per launch on a staged window of 64 x WY cells (the tile plus a halo of kl >= K
// columns on the left, >= K on the right and K rows above and below).  The window lives in
// registers: warp w owns the R rows w*R .. w*R + R - 1 of the window and lane l of every warp
// owns the column pair (2l, 2l + 1), so one warp spans the window's width.  Consequences:
//   * every global access of a thread is an 8-byte pair (state, wavefield store, update
//     coefficients, gradients), every row of a warp one 256-byte segment;
//   * x-neighbours come from the thread itself or from the next / previous lane by a warp
//     shuffle: no shared memory and no barrier for the x differences;
//   * y-neighbours come from the thread's own rows, except across warps: the top row of each
//     warp (Ez, or the adjoint's S_y weights) and the bottom row (Hx, or T_y) are exchanged
//     through shared memory, with two block barriers per time step.
// Each time step the valid region shrinks by one cell on every side (an H update reads Ez at
// +1, an E update reads H at -1; the window edges read their own values), so after K steps
// exactly the interior is valid; it is written to the other ping-pong state buffer.  Halo
// cells are recomputed redundantly by neighbouring CTAs from identical inputs.  Sources and
// adjoint sources are injected into every staged copy of their cell; receivers and the
// wavefield store are written only by the CTA owning the cell.
//
// CPML.  The convolutional PML memories live in shared memory (four window planes).  CTAs
// whose live columns reach an x strip take the x-CPML form of the H and E updates in every
// column (outside the strips its profile is a = 1/d, b = c = 0, which reduces it to the plain
// update and keeps the memory at zero): a CTA-uniform branch, chosen once per launch.  Rows in
// a y strip take the y-CPML form, a warp-uniform branch per row.
//
// Forward time step n (Algorithm 1, Sec. 3.3): record d^n = Ez^n at the receivers, update H
// and the magnetic CPML memories from Ez^n, update Ez and the electric CPML memories from
// H^{n+1/2} with Ez^{n+1} = Ca Ez^n + Cb Q (Eqs. 3-5 in the time-averaged loss form of the
// Sec. 3.2 coefficient listing), inject the source (Sec. 3.2 source listing: Q -= w^n / (dx
// dy), applied as Ez^{n+1} -= Cb w^n / (dx dy)), store Ez^{n+1}.
//
// Adjoint time step n (Algorithm 2): the exact transpose of the forward step, in reverse:
// (A) lam = Cb * adj(Ez^{n+1}) accumulates the zero-lag gradients (Eqs. grad_eps and
// grad_sigma in discrete form) and feeds the electric CPML memories, giving the weights S of
// the transposed E-step differences, and adj(Ez^n) starts as Ca adj(Ez^{n+1}); (B) adj(H)
// receives the transposed differences of S and feeds the magnetic CPML memories, giving the
// weights T; (C) adj(Ez^n) receives the transposed differences of T and the receiver residual
// of step n.  The stored Ez^n of the gradient is read through a shared-memory ring filled by
// cp.async kRingLead steps ahead of its use; the ring also holds the previous step's Ez^{n+1}.
#include "gf_internal.cuh"

namespace gf {
namespace {

constexpr int WX = 64;               // staged window width: one warp, two columns per lane
constexpr unsigned kFull = 0xffffffffu;
constexpr int kRing = 5;             // adjoint: slots of the wavefield ring
constexpr int kRingLead = 3;         // steps between a slot's cp.async and its use

// Shared-memory carve-up of a variant (offsets in floats; every region 16-byte aligned).
template <int R, int NW>
struct G {
    static constexpr int WY = R * NW;                    // window height
    static constexpr int NT = 32 * NW;                   // threads per CTA
    static constexpr int PL = WY * 32;                   // float2 per window plane
    static constexpr int oPsi = 0;                       // [4][WY][32] float2: Ex Ey Hx Hy
    static constexpr int oTop = oPsi + 8 * PL;           // [NW][32] float2
    static constexpr int oBot = oTop + 64 * NW;          // [NW][32] float2
    static constexpr int oYp = oBot + 64 * NW;           // [WY][2] float4: E, H row profiles
    static constexpr int oXp = oYp + 8 * WY;             // [6][32] float2: column profiles
    static constexpr int oWs = oXp + 6 * WX;             // [kMaxK + 1][kMaxSrc] source samples
    static constexpr int oSp = oWs + (kMaxK + 1) * kMaxSrc;  // [kMaxSrc] source positions
    static constexpr int oRec = oSp + kMaxSrc;           // [kRecStage] staged receivers
    static constexpr int oCoef = oRec + kRecStage;       // [WY][32] float4: Ca, Cb of the pair
    static constexpr int oRing = oCoef + 4 * PL;         // adjoint: [kRing][WY][32] float2
    static constexpr int fwd_floats = oRing;
    static constexpr int adj_floats = oRing + kRing * 2 * PL;
};

__device__ __forceinline__ bool in_xstrip(int gx, const TileParams& p) {
    return p.npml > 0 && (gx < p.npml || gx >= p.nx - p.npml - 1);
}
__device__ __forceinline__ bool in_ystrip(int gy, const TileParams& p) {
    return p.npml > 0 && (gy < p.npml || gy >= p.ny - p.npml - 1);
}

// Position of a thread in the staged window.
template <int R>
struct Pos {
    int lane, warp, ly0;   // lane, warp, first window row of the warp
    int X0, Y0, gx0;       // window origin (X0 even); global column of the lane's first column
    bool lane_in;          // the lane's first column lies in the grid (the second one may be
                           // the row padding when nx is odd: its coefficients are zero)
    bool lane_int;         // the lane's columns are interior columns of the tile
    bool tile_xs;          // the window's live columns reach an x CPML strip (CTA-uniform)
    bool xs0, xs1;         // the lane's columns lie in an x strip (only set when tile_xs)
    unsigned row_in;       // bit r: row ly0 + r lies in the grid
    unsigned row_int;      // bit r: row ly0 + r is an interior row
    unsigned ymask;        // bit r: row ly0 + r lies in a y CPML strip (warp-uniform)
    bool ys;               // some row of the warp lies in a y strip: the warp takes the y-CPML
                           // form in all its rows (warp-uniform)
};

template <int R>
__device__ __forceinline__ Pos<R> position(const TileParams& p) {
    Pos<R> w;
    w.lane = threadIdx.x & 31;
    w.warp = threadIdx.x >> 5;
    w.ly0 = w.warp * R;
    const int tx = blockIdx.x % p.tiles_x, ty = blockIdx.x / p.tiles_x;
    w.X0 = tx * p.tile_w - p.kl;
    w.Y0 = ty * p.tile_h - p.K;
    w.gx0 = w.X0 + 2 * w.lane;
    w.lane_in = w.gx0 >= 0 && w.gx0 < p.nx;
    w.lane_int = 2 * w.lane >= p.kl && 2 * w.lane < p.kl + p.tile_w && w.gx0 < p.nx;
    const int xa = tx * p.tile_w - p.K, xb = tx * p.tile_w + p.tile_w + p.K;  // live columns
    w.tile_xs = p.npml > 0 && (xa < p.npml || xb - 1 >= p.nx - p.npml - 1);
    w.xs0 = w.tile_xs && in_xstrip(w.gx0, p);
    w.xs1 = w.tile_xs && in_xstrip(w.gx0 + 1, p);
    w.row_in = w.row_int = w.ymask = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int ly = w.ly0 + r, gy = w.Y0 + ly;
        if (gy >= 0 && gy < p.ny) {
            w.row_in |= 1u << r;
            if (in_ystrip(gy, p)) w.ymask |= 1u << r;
            if (ly >= p.K && ly < p.K + p.tile_h) w.row_int |= 1u << r;
        }
    }
    w.ys = w.ymask != 0;
    return w;
}

__device__ __forceinline__ float2 ld2(const float* a) { return *reinterpret_cast<const float2*>(a); }
__device__ __forceinline__ void st2(float* a, float2 v) { *reinterpret_cast<float2*>(a) = v; }

// Value of cell (r, c) of a thread's register block (r, c run-time, warp-divergent callers).
template <int R>
__device__ __forceinline__ float pick(const float2 (&f)[R], int r, int c) {
    float v = 0.f;
#pragma unroll
    for (int k = 0; k < R; ++k)
        if (k == r) v = c ? f[k].y : f[k].x;
    return v;
}
template <int R>
__device__ __forceinline__ void add_at(float2 (&f)[R], int r, int c, float v) {
#pragma unroll
    for (int k = 0; k < R; ++k)
        if (k == r) {
            if (c) f[k].y += v;
            else f[k].x += v;
        }
}

// Load the owned cells' state (f0, f1, f2 = Ez, Hx, Hy or their adjoints); the update
// coefficients go to the shared-memory plane coef (Ca, Cb of both columns as one float4),
// the CPML memories of strip cells to the psi planes (zero elsewhere in the planes the strip
// forms read: x planes of x-strip CTAs, y planes of every row of a y-strip warp).  Every
// global load is issued before the first shared-memory store, so that the prologue waits
// for one memory round trip, not one per row.
template <int R, int NW>
__device__ __forceinline__ void load_state(const TileParams& p, const Pos<R>& w, float* sm,
                                           int shot, float2 (&f0)[R], float2 (&f1)[R],
                                           float2 (&f2)[R]) {
    using Gm = G<R, NW>;
    const long long F = (long long)p.nshots * p.Np;
    const long long sb = (long long)shot * p.Np;
    const float2 z = make_float2(0.f, 0.f);
    float2 u[R], v[R], pex[R], phy[R], pey[R], phx[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const bool in = w.lane_in && ((w.row_in >> r) & 1u);
        const long long m = (long long)(w.Y0 + w.ly0 + r) * p.pitch + w.gx0;
        const float* s = p.st_in + sb + m;
        f0[r] = f1[r] = f2[r] = u[r] = v[r] = z;
        pex[r] = phy[r] = pey[r] = phx[r] = z;
        if (in) {
            f0[r] = ld2(s);
            f1[r] = ld2(s + F);
            f2[r] = ld2(s + 2 * F);
            u[r] = __ldg(reinterpret_cast<const float2*>(p.ca + m));
            v[r] = __ldg(reinterpret_cast<const float2*>(p.cb + m));
            if (w.xs0 || w.xs1) {
                pex[r] = ld2(s + 3 * F);
                phy[r] = ld2(s + 6 * F);
            }
            if ((w.ymask >> r) & 1u) {
                pey[r] = ld2(s + 4 * F);
                phx[r] = ld2(s + 5 * F);
            }
        }
    }
    float2* psi = reinterpret_cast<float2*>(sm + Gm::oPsi) + w.ly0 * 32 + w.lane;
    float4* coef = reinterpret_cast<float4*>(sm + Gm::oCoef) + w.ly0 * 32 + w.lane;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        coef[r * 32] = make_float4(u[r].x, v[r].x, u[r].y, v[r].y);
        if (w.tile_xs) {
            if (!w.xs0) pex[r].x = phy[r].x = 0.f;
            if (!w.xs1) pex[r].y = phy[r].y = 0.f;
            psi[r * 32] = pex[r];
            psi[3 * Gm::PL + r * 32] = phy[r];
        }
        if (w.ys) {
            psi[Gm::PL + r * 32] = pey[r];
            psi[2 * Gm::PL + r * 32] = phx[r];
        }
    }
}

// Write the owned interior cells (fields and strip memories) to the output state.
template <int R, int NW>
__device__ __forceinline__ void store_state(const TileParams& p, const Pos<R>& w, const float* sm,
                                            int shot, const float2 (&f0)[R], const float2 (&f1)[R],
                                            const float2 (&f2)[R]) {
    using Gm = G<R, NW>;
    const long long F = (long long)p.nshots * p.Np;
    const long long sb = (long long)shot * p.Np;
    const float2* psi = reinterpret_cast<const float2*>(sm + Gm::oPsi) + w.ly0 * 32 + w.lane;
    if (!w.lane_int) return;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (!((w.row_int >> r) & 1u)) continue;
        float* s = p.st_out + sb + (long long)(w.Y0 + w.ly0 + r) * p.pitch + w.gx0;
        st2(s, f0[r]);
        st2(s + F, f1[r]);
        st2(s + 2 * F, f2[r]);
        if (w.xs0 || w.xs1) {
            st2(s + 3 * F, psi[r * 32]);
            st2(s + 6 * F, psi[3 * Gm::PL + r * 32]);
        }
        if ((w.ymask >> r) & 1u) {
            st2(s + 4 * F, psi[Gm::PL + r * 32]);
            st2(s + 5 * F, psi[2 * Gm::PL + r * 32]);
        }
    }
}

// Row and column CPML profiles of the staged window (clamped to the grid).
template <int R, int NW>
__device__ __forceinline__ void stage_profiles(const TileParams& p, const Pos<R>& w, float* sm) {
    using Gm = G<R, NW>;
    for (int i = threadIdx.x; i < Gm::WY + WX; i += Gm::NT) {
        if (i < Gm::WY) {
            const int g = min(max(w.Y0 + i, 0), p.ny - 1);
            float4* yp = reinterpret_cast<float4*>(sm + Gm::oYp) + 2 * i;
            yp[0] = make_float4(__ldg(p.py.aE + g), __ldg(p.py.bE + g), __ldg(p.py.cE + g), 0.f);
            yp[1] = make_float4(__ldg(p.py.aH + g), __ldg(p.py.bH + g), __ldg(p.py.cH + g), 0.f);
        } else {
            const int c = i - Gm::WY, g = min(max(w.X0 + c, 0), p.nx - 1);
            float* xp = sm + Gm::oXp + c;  // plane k, column c at xp[k * 64]
            xp[0] = __ldg(p.px.aE + g);
            xp[WX] = __ldg(p.px.bE + g);
            xp[2 * WX] = __ldg(p.px.cE + g);
            xp[3 * WX] = __ldg(p.px.aH + g);
            xp[4 * WX] = __ldg(p.px.bH + g);
            xp[5 * WX] = __ldg(p.px.cH + g);
        }
    }
}

// Window receivers.  With kStaged the list is staged in shared memory: rec[e] = position
// lx | (ly + kRowBias) << 8 | interior << 16, rec[nrl + e] = receiver index (and, in the
// adjoint, rec[2 nrl + e K + st] = residual sample of launch step st); otherwise entries are
// decoded from global memory when used.  The lists are built for the context's time-block
// depth; a shorter last launch starts its window lower, so a few entries can sit above row 0
// (they match no thread).  The bias keeps the packed rows non-negative and in list order.
constexpr int kRowBias = 64;
__device__ __forceinline__ int rec_position(const TileParams& p, int cell, int X0, int Y0) {
    const int y = cell / p.nx, x = cell - y * p.nx;
    const int lx = x - X0, ly = y - Y0;
    const bool interior =
        lx >= p.kl && lx < p.kl + p.tile_w && ly >= p.K && ly < p.K + p.tile_h;
    return (lx & 0xff) | (ly + kRowBias) << 8 | (interior ? 1 << 16 : 0);
}
__device__ __forceinline__ int rec_row(int pos) { return ((pos >> 8) & 0xff) - kRowBias; }

template <bool kStaged>
__device__ __forceinline__ void rec_entry(const TileParams& p, const int* srec, const int* rlist,
                                          const int* rcells, int nrl, int e, int X0, int Y0,
                                          int& pos, int& ri) {
    if (kStaged) {
        pos = srec[e];
        ri = srec[nrl + e];
    } else {
        ri = __ldg(rlist + e);
        pos = rec_position(p, __ldg(rcells + ri), X0, Y0);
    }
}

// Entries [lo, hi) of the row-sorted list on the warp's rows [ly0, ly0 + R).
template <bool kStaged, int R>
__device__ __forceinline__ void warp_rec_range(const TileParams& p, const Pos<R>& w,
                                               const int* srec, const int* rlist,
                                               const int* rcells, int nrl, int& lo, int& hi) {
    lo = hi = 0;
    for (int base = 0; base < nrl; base += 32) {
        const int e = base + w.lane;
        int ly = 1 << 20;
        if (e < nrl) {
            int pos, ri;
            rec_entry<kStaged>(p, srec, rlist, rcells, nrl, e, w.X0, w.Y0, pos, ri);
            ly = rec_row(pos);
        }
        lo += __popc(__ballot_sync(kFull, ly < w.ly0));
        hi += __popc(__ballot_sync(kFull, ly < w.ly0 + R));
    }
}

// ---------------------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------------------
// H update of the warp's rows from Ez^n (eb: Ez of the row below the warp), with the x-CPML
// form in every column when XS and the y-CPML form in every row when YS (both reduce to the
// plain update outside the strips).  No per-row branches: the rows are independent chains.
template <int R, int NW, bool XS, bool YS>
__device__ __forceinline__ void h_rows(const TileParams& p, float2* psi, const float2* xp,
                                       const float4* yp, const float2 (&ez)[R], float2 eb,
                                       float2 (&hx)[R], float2 (&hy)[R]) {
    using Gm = G<R, NW>;
    const float ch = p.ch, chx = p.ch * p.rdx, chy = p.ch * p.rdy;
    float2 axH, bxH, cxH;
    if (XS) {
        axH = xp[3 * 32];
        bxH = xp[4 * 32];
        cxH = xp[5 * 32];
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float2 e = ez[r];
        const float2 ed = r < R - 1 ? ez[r + 1] : eb;
        const float er = __shfl_down_sync(kFull, e.x, 1);
        const float dx0 = e.y - e.x, dx1 = er - e.y;
        const float dy0 = ed.x - e.x, dy1 = ed.y - e.y;
        if (XS) {
            float2 ph = psi[3 * Gm::PL + r * 32];
            ph.x = fmaf(bxH.x, ph.x, cxH.x * dx0);
            ph.y = fmaf(bxH.y, ph.y, cxH.y * dx1);
            psi[3 * Gm::PL + r * 32] = ph;
            hy[r].x = fmaf(ch, fmaf(axH.x, dx0, ph.x), hy[r].x);
            hy[r].y = fmaf(ch, fmaf(axH.y, dx1, ph.y), hy[r].y);
        } else {
            hy[r].x = fmaf(chx, dx0, hy[r].x);
            hy[r].y = fmaf(chx, dx1, hy[r].y);
        }
        if (YS) {
            const float4 pr = yp[2 * r + 1];
            float2 ph = psi[2 * Gm::PL + r * 32];
            ph.x = fmaf(pr.y, ph.x, pr.z * dy0);
            ph.y = fmaf(pr.y, ph.y, pr.z * dy1);
            psi[2 * Gm::PL + r * 32] = ph;
            hx[r].x = fmaf(-ch, fmaf(pr.x, dy0, ph.x), hx[r].x);
            hx[r].y = fmaf(-ch, fmaf(pr.x, dy1, ph.y), hx[r].y);
        } else {
            hx[r].x = fmaf(-chy, dy0, hx[r].x);
            hx[r].y = fmaf(-chy, dy1, hx[r].y);
        }
    }
}

// E update of the warp's rows from H^{n+1/2} (ha: Hx of the row above the warp):
// Ez^{n+1} = Ca Ez^n + Cb Q.
template <int R, int NW, bool XS, bool YS>
__device__ __forceinline__ void e_rows(const TileParams& p, float2* psi, const float2* xp,
                                       const float4* yp, const float4* coef, float2 (&ez)[R],
                                       const float2 (&hx)[R], const float2 (&hy)[R], float2 ha) {
    using Gm = G<R, NW>;
    const float rdx = p.rdx, rdy = p.rdy;
    float2 axE, bxE, cxE;
    if (XS) {
        axE = xp[0];
        bxE = xp[32];
        cxE = xp[2 * 32];
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float2 h = hy[r];
        const float hl = __shfl_up_sync(kFull, h.y, 1);
        const float2 hu = r > 0 ? hx[r - 1] : ha;
        const float dx0 = h.x - hl, dx1 = h.y - h.x;
        const float dy0 = hx[r].x - hu.x, dy1 = hx[r].y - hu.y;
        float q0, q1;
        if (XS) {
            float2 pe = psi[r * 32];
            pe.x = fmaf(bxE.x, pe.x, cxE.x * dx0);
            pe.y = fmaf(bxE.y, pe.y, cxE.y * dx1);
            psi[r * 32] = pe;
            q0 = fmaf(axE.x, dx0, pe.x);
            q1 = fmaf(axE.y, dx1, pe.y);
        } else {
            q0 = rdx * dx0;
            q1 = rdx * dx1;
        }
        if (YS) {
            const float4 pr = yp[2 * r];
            float2 pe = psi[Gm::PL + r * 32];
            pe.x = fmaf(pr.y, pe.x, pr.z * dy0);
            pe.y = fmaf(pr.y, pe.y, pr.z * dy1);
            psi[Gm::PL + r * 32] = pe;
            q0 -= fmaf(pr.x, dy0, pe.x);
            q1 -= fmaf(pr.x, dy1, pe.y);
        } else {
            q0 = fmaf(-rdy, dy0, q0);
            q1 = fmaf(-rdy, dy1, q1);
        }
        const float4 c = coef[r * 32];
        ez[r].x = fmaf(c.x, ez[r].x, c.y * q0);
        ez[r].y = fmaf(c.z, ez[r].y, c.w * q1);
    }
}

template <int R, int NW, bool XS, bool kHist, bool kIllum, bool kStaged>
__device__ __forceinline__ void fwd_steps(const TileParams& p, const Pos<R>& w, float* sm,
                                          float2 (&ez)[R], float2 (&hx)[R], float2 (&hy)[R],
                                          float2 (&ill)[R], int rlo, int rhi, int nrl,
                                          const int* rlist, bool srcany, int shot) {
    using Gm = G<R, NW>;
    float2* top = reinterpret_cast<float2*>(sm + Gm::oTop);
    float2* bot = reinterpret_cast<float2*>(sm + Gm::oBot);
    float2* psi = reinterpret_cast<float2*>(sm + Gm::oPsi) + w.ly0 * 32 + w.lane;
    const float2* xp = reinterpret_cast<const float2*>(sm + Gm::oXp) + w.lane;
    const float4* yp = reinterpret_cast<const float4*>(sm + Gm::oYp) + 2 * w.ly0;
    const float4* coef = reinterpret_cast<const float4*>(sm + Gm::oCoef) + w.ly0 * 32 + w.lane;
    const int* srec = reinterpret_cast<const int*>(sm + Gm::oRec);
    const int* srcpos = reinterpret_cast<const int*>(sm + Gm::oSp);
    const float* wsrc = sm + Gm::oWs;
    const int* rcells = p.rec_cell + (long long)shot * p.nrec;
    float* tr = p.traces + (long long)shot * p.nt * p.nrec;
    // the wavefield store of the owned cells: row r of step n at hp + n Np + r pitch
    float* hp = kHist ? p.hist + ((long long)shot * p.hist_stride - p.hist_slot0) * p.Np +
                            (long long)(w.Y0 + w.ly0) * p.pitch + w.gx0
                      : nullptr;
    bool own[R];
#pragma unroll
    for (int r = 0; r < R; ++r) own[r] = w.lane_int && ((w.row_int >> r) & 1u);
    const float2* below = top + (w.warp + 1) * 32 + w.lane;
    const float2* above = bot + (w.warp - 1) * 32 + w.lane;

    for (int st = 0; st < p.K; ++st) {
        const int n = p.n0 + st;
        // 1. receivers in this CTA's interior: d^n = Ez^n (loop bounds are warp-uniform)
        for (int e = rlo; e < rhi; ++e) {
            int pos, ri;
            rec_entry<kStaged>(p, srec, rlist, rcells, nrl, e, w.X0, w.Y0, pos, ri);
            if (((pos & 0xff) >> 1) == w.lane && (pos >> 16))
                tr[(long long)n * p.nrec + ri] = pick<R>(ez, rec_row(pos) - w.ly0, pos & 1);
        }
        top[w.warp * 32 + w.lane] = ez[0];
        __syncthreads();
        const float2 eb = w.warp < NW - 1 ? *below : ez[R - 1];
        // 2-3. H and magnetic CPML from Ez^n
        if (w.ys)
            h_rows<R, NW, XS, true>(p, psi, xp, yp, ez, eb, hx, hy);
        else
            h_rows<R, NW, XS, false>(p, psi, xp, yp, ez, eb, hx, hy);
        bot[w.warp * 32 + w.lane] = hx[R - 1];
        __syncthreads();
        const float2 ha = w.warp > 0 ? *above : hx[0];
        // 4-5. E and electric CPML from H^{n+1/2}, giving Ez^{n+1}
        if (w.ys)
            e_rows<R, NW, XS, true>(p, psi, xp, yp, coef, ez, hx, hy, ha);
        else
            e_rows<R, NW, XS, false>(p, psi, xp, yp, coef, ez, hx, hy, ha);
        // 6. sources: Ez^{n+1} -= Cb w^n / (dx dy) in every staged copy
        if (srcany) {
            for (int k = 0; k < p.nsrc; ++k) {
                const int pos = srcpos[k];
                const int r = (pos >> 8) - w.ly0, c = pos & 1;
                if (pos >= 0 && ((pos & 0xff) >> 1) == w.lane && r >= 0 && r < R) {
                    const float4 cc = coef[r * 32];
                    add_at<R>(ez, r, c, -(c ? cc.w : cc.y) * wsrc[st * kMaxSrc + k]);
                }
            }
        }
        // 7. wavefield store and illumination of the owned cells
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (kHist && own[r])
                __stcs(reinterpret_cast<float2*>(hp + (long long)n * p.Np + (long long)r * p.pitch),
                       ez[r]);
            if (kIllum) {
                ill[r].x = fmaf(ez[r].x, ez[r].x, ill[r].x);
                ill[r].y = fmaf(ez[r].y, ez[r].y, ill[r].y);
            }
        }
    }
}

template <int R, int NW, bool kHist, bool kIllum, bool kStaged>
__global__ void __launch_bounds__(32 * NW, NW <= 8 && R <= 4 ? 2 : 1) fwd_tile_kernel(const TileParams p) {
    using Gm = G<R, NW>;
    extern __shared__ float4 smem_raw[];
    float* sm = reinterpret_cast<float*>(smem_raw);
    const Pos<R> w = position<R>(p);
    const int shot = blockIdx.y, K = p.K, tid = threadIdx.x;

    float2 ez[R], hx[R], hy[R], ill[R];
    load_state<R, NW>(p, w, sm, shot, ez, hx, hy);
#pragma unroll
    for (int r = 0; r < R; ++r) ill[r] = make_float2(0.f, 0.f);
    stage_profiles<R, NW>(p, w, sm);
    float* wsrc = sm + Gm::oWs;
    int* srcpos = reinterpret_cast<int*>(sm + Gm::oSp);
    for (int k = tid; k < K * kMaxSrc; k += Gm::NT) {
        const int st = k / kMaxSrc, src = k - st * kMaxSrc;
        wsrc[k] = src < p.nsrc ? p.src_scale * __ldg(p.wavelet + ((long long)shot * p.nsrc + src) *
                                                                     p.nt + p.n0 + st)
                               : 0.f;
    }
    if (tid < kMaxSrc) {
        int pos = -1;
        if (tid < p.nsrc) {
            const int cell = __ldg(p.src_cell + shot * p.nsrc + tid);
            const int y = cell / p.nx, x = cell - y * p.nx, lx = x - w.X0, ly = y - w.Y0;
            if (lx >= 0 && lx < WX && ly >= 0 && ly < Gm::WY) pos = lx | ly << 8;
        }
        srcpos[tid] = pos;
    }
    const long long lo = p.tile_rec_off[(long long)shot * p.ntiles + blockIdx.x];
    const int nrl = (int)(p.tile_rec_off[(long long)shot * p.ntiles + blockIdx.x + 1] - lo);
    const int* rlist = p.tile_rec_idx + lo;
    const int* rcells = p.rec_cell + (long long)shot * p.nrec;
    int* srec = reinterpret_cast<int*>(sm + Gm::oRec);
    if (kStaged) {
        for (int e = tid; e < nrl; e += Gm::NT) {
            const int ri = __ldg(rlist + e);
            srec[e] = rec_position(p, __ldg(rcells + ri), w.X0, w.Y0);
            srec[nrl + e] = ri;
        }
    }
    __syncthreads();
    int rlo, rhi;
    warp_rec_range<kStaged, R>(p, w, srec, rlist, rcells, nrl, rlo, rhi);
    bool srcany = false;
    for (int k = 0; k < p.nsrc; ++k) {
        const int pos = srcpos[k], r = (pos >> 8) - w.ly0;
        srcany |= pos >= 0 && ((pos & 0xff) >> 1) == w.lane && r >= 0 && r < R;
    }

    if (w.tile_xs)
        fwd_steps<R, NW, true, kHist, kIllum, kStaged>(p, w, sm, ez, hx, hy, ill, rlo, rhi, nrl,
                                                       rlist, srcany, shot);
    else
        fwd_steps<R, NW, false, kHist, kIllum, kStaged>(p, w, sm, ez, hx, hy, ill, rlo, rhi, nrl,
                                                        rlist, srcany, shot);

    store_state<R, NW>(p, w, sm, shot, ez, hx, hy);
    if (kIllum && w.lane_int) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (!((w.row_int >> r) & 1u)) continue;
            float* a = p.illum + (long long)shot * p.Np + (long long)(w.Y0 + w.ly0 + r) * p.pitch + w.gx0;
            float2 v = ld2(a);
            v.x += ill[r].x;
            v.y += ill[r].y;
            st2(a, v);
        }
    }
}

// ---------------------------------------------------------------------------------------
// Adjoint
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// cp.async of 8 bytes that reads `bytes` (8 or 0) from global memory and zero-fills the rest.
__device__ __forceinline__ void cp_async8_zfill(void* dst_smem, const void* src, int bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(bytes)
                 : "memory");
}

// Phase A of the warp's rows: lam = Cb adj(Ez^{n+1}); zero-lag gradient sums with Ez^{n+1}
// (ring slot `prev`) and Ez^n (ring slot `slot`); electric CPML and the S weights (wx, wy);
// adj(Ez^n) starts as Ca adj(Ez^{n+1}).  The gradient sums carry no constant factor (applied
// once at the end of the launch).
template <int R, int NW, bool XS, bool YS>
__device__ __forceinline__ void a_rows(const TileParams& p, float2* psi, const float2* xp,
                                       const float4* yp, const float4* coef, const float2* slot,
                                       const float2* prev, float2 (&aez)[R], float2 (&ge)[R],
                                       float2 (&gs)[R], float2 (&wx)[R], float2 (&wy)[R]) {
    using Gm = G<R, NW>;
    const float rdx = p.rdx, rdy = p.rdy;
    float2 axE, bxE, cxE;
    if (XS) {
        axE = xp[0];
        bxE = xp[32];
        cxE = xp[2 * 32];
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float2 pf = slot[r * 32], en1 = prev[r * 32];
        const float4 c = coef[r * 32];
        const float l0 = c.y * aez[r].x, l1 = c.w * aez[r].y;
        ge[r].x = fmaf(l0, en1.x - pf.x, ge[r].x);
        ge[r].y = fmaf(l1, en1.y - pf.y, ge[r].y);
        gs[r].x = fmaf(l0, en1.x + pf.x, gs[r].x);
        gs[r].y = fmaf(l1, en1.y + pf.y, gs[r].y);
        if (XS) {
            float2 pe = psi[r * 32];
            pe.x += l0;
            pe.y += l1;
            wx[r].x = fmaf(l0, axE.x, cxE.x * pe.x);
            wx[r].y = fmaf(l1, axE.y, cxE.y * pe.y);
            pe.x *= bxE.x;
            pe.y *= bxE.y;
            psi[r * 32] = pe;
        } else {
            wx[r].x = l0 * rdx;
            wx[r].y = l1 * rdx;
        }
        if (YS) {
            const float4 pr = yp[2 * r];
            float2 pe = psi[Gm::PL + r * 32];
            pe.x -= l0;
            pe.y -= l1;
            wy[r].x = fmaf(-l0, pr.x, pr.z * pe.x);
            wy[r].y = fmaf(-l1, pr.x, pr.z * pe.y);
            pe.x *= pr.y;
            pe.y *= pr.y;
            psi[Gm::PL + r * 32] = pe;
        } else {
            wy[r].x = -l0 * rdy;
            wy[r].y = -l1 * rdy;
        }
        aez[r].x *= c.x;
        aez[r].y *= c.z;
    }
}

// Phase B: adj(H) += transposed S differences (sb_: S_y of the row below the warp); magnetic
// CPML; the T weights replace S in wx, wy.  Rows in ascending order, so that wy[r + 1] still
// holds S_y when row r reads it.
template <int R, int NW, bool XS, bool YS>
__device__ __forceinline__ void b_rows(const TileParams& p, float2* psi, const float2* xp,
                                       const float4* yp, float2 sb_, float2 (&ahx)[R],
                                       float2 (&ahy)[R], float2 (&wx)[R], float2 (&wy)[R]) {
    using Gm = G<R, NW>;
    const float ch = p.ch, chx = p.ch * p.rdx, chy = p.ch * p.rdy;
    float2 axH, bxH, cxH;
    if (XS) {
        axH = xp[3 * 32];
        bxH = xp[4 * 32];
        cxH = xp[5 * 32];
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float sxr = __shfl_down_sync(kFull, wx[r].x, 1);
        const float2 syd = r < R - 1 ? wy[r + 1] : sb_;
        const float hy0 = ahy[r].x + wx[r].x - wx[r].y, hy1 = ahy[r].y + wx[r].y - sxr;
        const float hx0 = ahx[r].x + wy[r].x - syd.x, hx1 = ahx[r].y + wy[r].y - syd.y;
        ahy[r] = make_float2(hy0, hy1);
        ahx[r] = make_float2(hx0, hx1);
        if (XS) {
            float2 ph = psi[3 * Gm::PL + r * 32];
            ph.x = fmaf(ch, hy0, ph.x);
            ph.y = fmaf(ch, hy1, ph.y);
            wx[r].x = fmaf(ch * hy0, axH.x, cxH.x * ph.x);
            wx[r].y = fmaf(ch * hy1, axH.y, cxH.y * ph.y);
            ph.x *= bxH.x;
            ph.y *= bxH.y;
            psi[3 * Gm::PL + r * 32] = ph;
        } else {
            wx[r].x = chx * hy0;
            wx[r].y = chx * hy1;
        }
        if (YS) {
            const float4 pr = yp[2 * r + 1];
            float2 ph = psi[2 * Gm::PL + r * 32];
            ph.x = fmaf(-ch, hx0, ph.x);
            ph.y = fmaf(-ch, hx1, ph.y);
            wy[r].x = fmaf(-ch * hx0, pr.x, pr.z * ph.x);
            wy[r].y = fmaf(-ch * hx1, pr.x, pr.z * ph.y);
            ph.x *= pr.y;
            ph.y *= pr.y;
            psi[2 * Gm::PL + r * 32] = ph;
        } else {
            wy[r].x = -chy * hx0;
            wy[r].y = -chy * hx1;
        }
    }
}

// Ez^n of the owned cells for phase A number a (step n = n1 - a; a = -1 gives Ez^{n1+1}) into
// ring slot (a + kRing) % kRing, zero when n = 0 (Ez^0 = 0); one cp.async group per a, empty
// beyond the launch.  Cells the thread does not own are not fetched: their ring entries only
// feed gradient sums that are never stored.  hp: the owned cells' store, Ez^{m+1} of row r at
// hp + m Np + r pitch.
template <int R, int NW>
__device__ __forceinline__ void ring_fetch(const TileParams& p, float2* ring, const float* hp,
                                           const bool (&own)[R], int n1, int a) {
    using Gm = G<R, NW>;
    if (a < p.K) {
        const int n = n1 - a;
        float2* slot = ring + ((a + kRing) % kRing) * Gm::PL;
        const float* h = hp + (long long)(n >= 1 ? n - 1 : 0) * p.Np;
        const int bytes = n >= 1 ? 8 : 0;
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (own[r]) cp_async8_zfill(slot + r * 32, h + (long long)r * p.pitch, bytes);
    }
    cp_async_commit();
}

template <int R, int NW, bool XS, bool kStaged>
__device__ __forceinline__ void adj_steps(const TileParams& p, const Pos<R>& w, float* sm,
                                          float2 (&aez)[R], float2 (&ahx)[R], float2 (&ahy)[R],
                                          float2 (&ge)[R], float2 (&gs)[R], const float* hp,
                                          const bool (&own)[R], int rlo, int rhi, int nrl,
                                          const int* rlist, int shot) {
    using Gm = G<R, NW>;
    const int K = p.K, n1 = p.n0 + K - 1;
    float2* top = reinterpret_cast<float2*>(sm + Gm::oTop);
    float2* bot = reinterpret_cast<float2*>(sm + Gm::oBot);
    float2* psi = reinterpret_cast<float2*>(sm + Gm::oPsi) + w.ly0 * 32 + w.lane;
    float2* ring = reinterpret_cast<float2*>(sm + Gm::oRing) + w.ly0 * 32 + w.lane;
    const float2* xp = reinterpret_cast<const float2*>(sm + Gm::oXp) + w.lane;
    const float4* yp = reinterpret_cast<const float4*>(sm + Gm::oYp) + 2 * w.ly0;
    const float4* coef = reinterpret_cast<const float4*>(sm + Gm::oCoef) + w.ly0 * 32 + w.lane;
    const int* srec = reinterpret_cast<const int*>(sm + Gm::oRec);
    const int* rcells = p.rec_cell + (long long)shot * p.nrec;
    const float* rbase = p.resid + (long long)shot * p.nt * p.nrec;
    const float2* below = top + (w.warp + 1) * 32 + w.lane;
    const float2* above = bot + (w.warp - 1) * 32 + w.lane;
    float2 wx[R], wy[R];
    auto phase_a = [&](int a) {
        ring_fetch<R, NW>(p, ring, hp, own, n1, a + kRingLead);
        cp_async_wait<kRingLead>();
        const float2* slot = ring + (a % kRing) * Gm::PL;
        const float2* prev = ring + ((a + kRing - 1) % kRing) * Gm::PL;
        if (w.ys)
            a_rows<R, NW, XS, true>(p, psi, xp, yp, coef, slot, prev, aez, ge, gs, wx, wy);
        else
            a_rows<R, NW, XS, false>(p, psi, xp, yp, coef, slot, prev, aez, ge, gs, wx, wy);
    };

    phase_a(0);
    for (int st = 0; st < K; ++st) {
        const int n = n1 - st;
        top[w.warp * 32 + w.lane] = wy[0];
        __syncthreads();
        const float2 sb_ = w.warp < NW - 1 ? *below : wy[R - 1];
        // B: adj(H) += transposed S differences; magnetic CPML; T weights
        if (w.ys)
            b_rows<R, NW, XS, true>(p, psi, xp, yp, sb_, ahx, ahy, wx, wy);
        else
            b_rows<R, NW, XS, false>(p, psi, xp, yp, sb_, ahx, ahy, wx, wy);
        bot[w.warp * 32 + w.lane] = wy[R - 1];
        __syncthreads();
        const float2 ta = w.warp > 0 ? *above : wy[0];
        // C: adj(Ez^n) += transposed T differences
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float tl = __shfl_up_sync(kFull, wx[r].y, 1);
            const float2 tu = r > 0 ? wy[r - 1] : ta;
            aez[r].x += (tl - wx[r].x) + (tu.x - wy[r].x);
            aez[r].y += (wx[r].x - wx[r].y) + (tu.y - wy[r].y);
        }
        // adjoint source of step n: the residual at the receivers (every staged copy)
        for (int e = rlo; e < rhi; ++e) {
            int pos, ri;
            rec_entry<kStaged>(p, srec, rlist, rcells, nrl, e, w.X0, w.Y0, pos, ri);
            if (((pos & 0xff) >> 1) == w.lane) {
                const float v = kStaged ? __int_as_float(srec[2 * nrl + e * K + st])
                                        : __ldg(rbase + (long long)n * p.nrec + ri);
                add_at<R>(aez, rec_row(pos) - w.ly0, pos & 1, v);
            }
        }
        if (st < K - 1) phase_a(st + 1);
    }
    cp_async_wait<0>();
}

template <int R, int NW, bool kStaged>
__global__ void __launch_bounds__(32 * NW, NW <= 8 && R <= 4 ? 2 : 1) adj_tile_kernel(const TileParams p) {
    using Gm = G<R, NW>;
    extern __shared__ float4 smem_raw[];
    float* sm = reinterpret_cast<float*>(smem_raw);
    const Pos<R> w = position<R>(p);
    const int shot = blockIdx.y, K = p.K, tid = threadIdx.x;
    const int n1 = p.n0 + K - 1;

    float2 aez[R], ahx[R], ahy[R], ge[R], gs[R];
    load_state<R, NW>(p, w, sm, shot, aez, ahx, ahy);
    // the stored Ez of the owned cells: Ez^{m+1} of row r at hp + m Np + r pitch; the ring's
    // first slots are requested before anything else of the prologue
    const float* hp = p.hist + ((long long)shot * p.hist_stride - p.hist_slot0) * p.Np +
                      (long long)(w.Y0 + w.ly0) * p.pitch + w.gx0;
    bool own[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        own[r] = w.lane_int && ((w.row_int >> r) & 1u);
        ge[r] = gs[r] = make_float2(0.f, 0.f);
    }
    float2* ring = reinterpret_cast<float2*>(sm + Gm::oRing) + w.ly0 * 32 + w.lane;
    for (int a = -1; a < kRingLead; ++a) ring_fetch<R, NW>(p, ring, hp, own, n1, a);
    stage_profiles<R, NW>(p, w, sm);
    const long long lo = p.tile_rec_off[(long long)shot * p.ntiles + blockIdx.x];
    const int nrl = (int)(p.tile_rec_off[(long long)shot * p.ntiles + blockIdx.x + 1] - lo);
    const int* rlist = p.tile_rec_idx + lo;
    const int* rcells = p.rec_cell + (long long)shot * p.nrec;
    int* srec = reinterpret_cast<int*>(sm + Gm::oRec);
    if (kStaged) {
        // positions, indices and the residual samples of this launch, so that the per-step
        // injection reads shared memory only (nrl * (K + 2) <= kRecStage)
        for (int e = tid; e < nrl; e += Gm::NT) {
            const int ri = __ldg(rlist + e);
            srec[e] = rec_position(p, __ldg(rcells + ri), w.X0, w.Y0);
            srec[nrl + e] = ri;
        }
        const float* rb = p.resid + (long long)shot * p.nt * p.nrec;
        for (int i = tid; i < nrl * K; i += Gm::NT) {
            const int e = i / K, st = i - e * K;
            srec[2 * nrl + i] =
                __float_as_int(__ldg(rb + (long long)(n1 - st) * p.nrec + __ldg(rlist + e)));
        }
    }
    __syncthreads();
    int rlo, rhi;
    warp_rec_range<kStaged, R>(p, w, srec, rlist, rcells, nrl, rlo, rhi);

    if (w.tile_xs)
        adj_steps<R, NW, true, kStaged>(p, w, sm, aez, ahx, ahy, ge, gs, hp, own, rlo, rhi, nrl,
                                        rlist, shot);
    else
        adj_steps<R, NW, false, kStaged>(p, w, sm, aez, ahx, ahy, ge, gs, hp, own, rlo, rhi, nrl,
                                         rlist, shot);

    store_state<R, NW>(p, w, sm, shot, aez, ahx, ahy);
    if (w.lane_int) {
        const long long F = (long long)p.nshots * p.Np;
        const float se = -p.geps;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (!((w.row_int >> r) & 1u)) continue;
            float* g = p.grad + (long long)shot * p.Np + (long long)(w.Y0 + w.ly0 + r) * p.pitch + w.gx0;
            // one writer per cell per launch and launches in stream order: a fire-and-forget
            // reduction is deterministic and hides the read latency of += at the end of the CTA
            atomicAdd(reinterpret_cast<float2*>(g), make_float2(se * ge[r].x, se * ge[r].y));
            atomicAdd(reinterpret_cast<float2*>(g + F),
                      make_float2(-0.5f * gs[r].x, -0.5f * gs[r].y));
        }
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

template <int R, int NW>
cudaError_t configure_variant(size_t optin) {
    cudaError_t e;
#define GF_ALLOW(...) \
    if ((e = allow_smem(__VA_ARGS__, optin)) != cudaSuccess) return e
    GF_ALLOW(fwd_tile_kernel<R, NW, true, true, true>);
    GF_ALLOW(fwd_tile_kernel<R, NW, true, false, true>);
    GF_ALLOW(fwd_tile_kernel<R, NW, false, true, true>);
    GF_ALLOW(fwd_tile_kernel<R, NW, false, false, true>);
    GF_ALLOW(fwd_tile_kernel<R, NW, true, true, false>);
    GF_ALLOW(fwd_tile_kernel<R, NW, true, false, false>);
    GF_ALLOW(fwd_tile_kernel<R, NW, false, true, false>);
    GF_ALLOW(fwd_tile_kernel<R, NW, false, false, false>);
    GF_ALLOW(adj_tile_kernel<R, NW, true>);
    GF_ALLOW(adj_tile_kernel<R, NW, false>);
#undef GF_ALLOW
    return cudaSuccess;
}

template <int R, int NW, bool kHist, bool kIllum>
cudaError_t launch_fwd_variant(const TileParams& p, bool staged, cudaStream_t st) {
    using Gm = G<R, NW>;
    const dim3 grid(p.ntiles, p.nshots), block(Gm::NT);
    const size_t smem = sizeof(float) * Gm::fwd_floats;
    if (staged)
        fwd_tile_kernel<R, NW, kHist, kIllum, true><<<grid, block, smem, st>>>(p);
    else
        fwd_tile_kernel<R, NW, kHist, kIllum, false><<<grid, block, smem, st>>>(p);
    return cudaGetLastError();
}

template <int R, int NW>
cudaError_t launch_fwd_r(const TileParams& p, bool staged, cudaStream_t st) {
    if (p.hist && p.illum) return launch_fwd_variant<R, NW, true, true>(p, staged, st);
    if (p.hist) return launch_fwd_variant<R, NW, true, false>(p, staged, st);
    if (p.illum) return launch_fwd_variant<R, NW, false, true>(p, staged, st);
    return launch_fwd_variant<R, NW, false, false>(p, staged, st);
}

template <int R, int NW>
cudaError_t launch_adj_r(const TileParams& p, bool staged, cudaStream_t st) {
    using Gm = G<R, NW>;
    const dim3 grid(p.ntiles, p.nshots), block(Gm::NT);
    const size_t smem = sizeof(float) * Gm::adj_floats;
    if (staged)
        adj_tile_kernel<R, NW, true><<<grid, block, smem, st>>>(p);
    else
        adj_tile_kernel<R, NW, false><<<grid, block, smem, st>>>(p);
    return cudaGetLastError();
}
}  // namespace

int max_tile_extent() { return WX; }
int max_tile_height(int variant) { return variant == 1 ? G<4, 8>::WY : 64; }
int num_tile_variants() { return 3; }

size_t tile_smem_bytes(int variant) {
    return sizeof(float) * (variant == 0   ? G<4, 16>::adj_floats
                            : variant == 1 ? G<4, 8>::adj_floats
                                           : G<8, 8>::adj_floats);
}

cudaError_t configure_tile_kernels(size_t optin) {
    cudaError_t e = configure_variant<4, 16>(optin);
    if (e != cudaSuccess) return e;
    if ((e = configure_variant<4, 8>(optin)) != cudaSuccess) return e;
    return configure_variant<8, 8>(optin);
}

// Variant 0: 4 rows per thread, 512 threads, 64 x 64 window, one CTA per SM; variant 1: 4 rows
// per thread, 256 threads, 64 x 32 window, two CTAs per SM (one CTA's loads and barrier waits
// overlap the other's work); variant 2: 8 rows per thread, 256 threads, 64 x 64.  Receiver
// lists are staged in shared memory when the longest one fits (forward: 2 words per entry,
// adjoint: K + 2), else read from global memory.
cudaError_t launch_fwd_tile(const TileParams& p, int variant, cudaStream_t st) {
    const bool staged = 2LL * p.rec_max <= kRecStage;
    return variant == 0   ? launch_fwd_r<4, 16>(p, staged, st)
           : variant == 1 ? launch_fwd_r<4, 8>(p, staged, st)
                          : launch_fwd_r<8, 8>(p, staged, st);
}

cudaError_t launch_adj_tile(const TileParams& p, int variant, cudaStream_t st) {
    const bool staged = (long long)p.rec_max * (p.K + 2) <= kRecStage;
    return variant == 0   ? launch_adj_r<4, 16>(p, staged, st)
           : variant == 1 ? launch_adj_r<4, 8>(p, staged, st)
                          : launch_adj_r<8, 8>(p, staged, st);
}

}  // namespace gf
