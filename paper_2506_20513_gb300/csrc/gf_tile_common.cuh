// gf_tile_common.cuh -- device building blocks shared by the per-launch tile kernels
// (gf_tile_kernels.cu) and the persistent dataflow kernels (gf_flow_kernels.cu): the 2-D TM
// FDTD forward step (Algorithm 1) and its exact transpose (Algorithm 2) on a staged window.
//
// Layout.  A CTA advances one tile of tile_w x tile_h cells of one shot by K time steps on a
// staged window of 64 x WY cells: the tile plus kl >= K columns on the left, >= K on the right
// and K rows above and below.  The window lives in registers: warp w owns the R rows
// w*R .. w*R + R - 1 and lane l of every warp the column pair (2l, 2l + 1), so one warp spans
// the window's width.  Every global access of a thread is an 8-byte pair and every row of a
// warp a 256-byte segment; x-neighbours come from the thread itself or from the next /
// previous lane by a warp shuffle; y-neighbours come from the thread's own rows, except
// across warps, where the top row of each warp (Ez, or the adjoint's S_y weights) and the
// bottom row (Hx, or T_y) are exchanged through shared memory (two block barriers per time
// step).  Each time step the valid region shrinks by one cell on every side (an H update
// reads Ez at +1, an E update reads H at -1; the window edges read their own values), so
// after K steps exactly the interior is valid.  Halo cells are recomputed redundantly by
// neighbouring tiles from identical inputs.  Sources and adjoint sources are injected into
// every staged copy of their cell; receivers and the wavefield store are written only by the
// tile owning the cell.
//
// CPML.  The convolutional PML memories live in shared memory (four window planes).  Tiles
// whose live columns reach an x strip take the x-CPML form of the H and E updates in every
// column (outside the strips its profile is a = 1/d, b = c = 0, which reduces it to the plain
// update and keeps the memory at zero): a CTA-uniform choice, made once per tile.  A warp with
// a row in a y strip takes the y-CPML form in all its rows (warp-uniform, no per-row branch).
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
// of step n.  The stored Ez^n of the owned cells is read through a shared-memory ring filled
// by cp.async kRingLead steps ahead of its use; the ring also holds the previous step's
// Ez^{n+1}.
#pragma once
#include "gf_internal.cuh"

namespace gf {
namespace {

constexpr int WX = 64;               // staged window width: one warp, two columns per lane
constexpr unsigned kFull = 0xffffffffu;
constexpr int kRing = 5;             // adjoint: slots of the wavefield ring
constexpr int kRingLead = 3;         // steps between a slot's cp.async and its use

// Shared-memory carve-up of a variant (offsets in floats).  Window planes are [WY][64]
// floats, row-major like the global planes, so that one TMA box fills one plane; they come
// first, 1024-byte aligned.  The adjoint appends the ring of kRing interior slots; the
// persistent forward appends the next tile's update coefficients.
template <int R, int NW>
struct G {
    static constexpr int WY = R * NW;                    // window height
    static constexpr int NT = 32 * NW;                   // threads per CTA
    static constexpr int PL = WY * 32;                   // float2 per window plane
    static constexpr int oPsi = 0;                       // 4 planes: psi Ex, Ey, Hx, Hy
    static constexpr int oCoef = oPsi + 8 * PL;          // 2 planes: Ca, Cb
    static constexpr int oStage = oCoef + 4 * PL;        // 3 planes: state staged by TMA / cp.async
    static constexpr int oTop = oStage + 6 * PL;         // [NW][32] float2
    static constexpr int oBot = oTop + 64 * NW;          // [NW][32] float2
    static constexpr int oYp = oBot + 64 * NW;           // [WY][2] float4: E, H row profiles
    static constexpr int oXp = oYp + 8 * WY;             // [6][64]: column profiles
    static constexpr int oWs = oXp + 6 * WX;             // [kMaxK + 1][kMaxSrc] source samples
    static constexpr int oSp = oWs + (kMaxK + 1) * kMaxSrc;  // [kMaxSrc] source positions
    static constexpr int oRec = oSp + kMaxSrc;           // [kRecStage] staged receivers
    static constexpr int oFlag = oRec + kRecStage;       // [4] ints: persistent-kernel flags
    static constexpr int oBar = oFlag + 4;               // mbarrier of the prologue's TMA loads
    static constexpr int oEnd = oBar + 4;
    static constexpr int oCoef2 = oEnd;                  // persistent forward: 2 planes
    static constexpr int fwd_floats = oEnd;
    static constexpr int fwd_flow_floats = oCoef2 + 4 * PL;
    static constexpr int adj_ring_off = oEnd;            // adjoint ring (both kinds)
    static_assert((oCoef * 4) % 1024 == 0 && (oStage * 4) % 1024 == 0, "TMA planes");
};

__device__ __forceinline__ bool in_xstrip(int gx, const TileParams& p) {
    return p.npml > 0 && (gx < p.npml || gx >= p.nx - p.npml - 1);
}
__device__ __forceinline__ bool in_ystrip(int gy, const TileParams& p) {
    return p.npml > 0 && (gy < p.npml || gy >= p.ny - p.npml - 1);
}

// Position of a thread in the staged window of one tile.
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
    unsigned ymask;        // bit r: row ly0 + r is a live row in a y CPML strip (warp-uniform)
    bool ys;               // some row of the warp lies in a y strip: the warp takes the y-CPML
                           // form in all its rows (warp-uniform)
};

// Window of tile `tile` advanced by K steps (p.kl: the context's left halo).
template <int R>
__device__ __forceinline__ Pos<R> position(const TileParams& p, int tile, int K) {
    Pos<R> w;
    w.lane = threadIdx.x & 31;
    w.warp = threadIdx.x >> 5;
    w.ly0 = w.warp * R;
    const int tx = tile % p.tiles_x, ty = tile / p.tiles_x;
    w.X0 = tx * p.tile_w - p.kl;
    w.Y0 = ty * p.tile_h - K;
    w.gx0 = w.X0 + 2 * w.lane;
    w.lane_in = w.gx0 >= 0 && w.gx0 < p.nx;
    w.lane_int = 2 * w.lane >= p.kl && 2 * w.lane < p.kl + p.tile_w && w.gx0 < p.nx;
    const int xa = tx * p.tile_w - K, xb = tx * p.tile_w + p.tile_w + K;  // live columns
    w.tile_xs = p.npml > 0 && (xa < p.npml || xb - 1 >= p.nx - p.npml - 1);
    w.xs0 = w.tile_xs && in_xstrip(w.gx0, p);
    w.xs1 = w.tile_xs && in_xstrip(w.gx0 + 1, p);
    w.row_in = w.row_int = w.ymask = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int ly = w.ly0 + r, gy = w.Y0 + ly;
        if (gy >= 0 && gy < p.ny) {
            w.row_in |= 1u << r;
            // only rows of the live window (the tile and its K-row halos) count: rows beyond
            // it hold values that never reach the tile, whatever form updates them
            if (ly < p.tile_h + 2 * K && in_ystrip(gy, p)) w.ymask |= 1u << r;
            if (ly >= K && ly < K + p.tile_h) w.row_int |= 1u << r;
        }
    }
    w.ys = w.ymask != 0;
    return w;
}

__device__ __forceinline__ float2 ld2(const float* a) { return *reinterpret_cast<const float2*>(a); }
__device__ __forceinline__ void st2(float* a, float2 v) { *reinterpret_cast<float2*>(a) = v; }
// 8-byte load through L2 only: data written by other CTAs of the same (persistent) kernel
__device__ __forceinline__ float2 ld2cg(const float* a) {
    return __ldcg(reinterpret_cast<const float2*>(a));
}

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

__device__ __forceinline__ uint32_t smem_u32(const void* a) {
    return (uint32_t)__cvta_generic_to_shared(a);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
                 : "memory");
}
// Programmatic dependent launch (the tile kernels of a pass are launched with programmatic
// stream serialisation): launch_dependents lets the next launch's CTAs start their prologue
// on the SMs this launch's last wave leaves idle; wait blocks the calling thread until the
// previous kernel on the stream has completed and its memory operations are visible.  Data a
// previous launch writes or reads (the state buffers, the gradient and illumination sums,
// the wavefield store) are touched only after the wait.
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// One 3-D TMA box (fp32, 64 x WY x 1 at (x, y, z)) into shared memory, completion counted in
// bytes on the mbarrier.  x must be a multiple of 4 (16 bytes); x, y may lie outside the
// array (zero fill).
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}
// Wait for phase `parity` of the mbarrier, at most `limit` polls; false when it ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned limit) {
    for (unsigned i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
// cp.async of 8 bytes through L1 that reads `bytes` (8 or 0) and zero-fills the rest.
__device__ __forceinline__ void cp_async8(void* dst_smem, const void* src, int bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(bytes)
                 : "memory");
}
// cp.async of 16 bytes through L2 only that reads `bytes` (16 or 0) and zero-fills the rest.
__device__ __forceinline__ void cp_async16cg(void* dst_smem, const void* src, int bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(bytes)
                 : "memory");
}

// ---------------------------------------------------------------------------------------
// A tile's prologue: global loads first (one memory round trip for most tiles), then the
// shared-memory stores that consume them.  A store of a loaded value makes the warp wait for
// it, so loads placed after one would start a second round trip.
// ---------------------------------------------------------------------------------------
// Does the live window of `w` (K steps) touch a CPML strip (CTA-uniform)?
template <int R>
__device__ __forceinline__ bool tile_in_strip(const TileParams& p, const Pos<R>& w, int K) {
    if (p.npml <= 0) return false;
    const int ya = w.Y0, yb = w.Y0 + p.tile_h + 2 * K;  // live rows [ya, yb)
    return w.tile_xs || ya < p.npml || yb - 1 >= p.ny - p.npml - 1;
}

// Registers of a tile's prologue loads.
template <int R>
struct TileLoads {
    int4 d;                                  // tile descriptor {first entry, entries, source mask}
    float2 f0[R], f1[R], f2[R];              // state (Ez, Hx, Hy or their adjoints)
    float2 u[R], v[R];                       // update coefficients Ca, Cb of the column pair
    float2 pex[R], phy[R], pey[R], phx[R];   // CPML memories of strip cells
    float prof[6];                           // one row's or one column's profiles
    float wv;                                // one source sample (thread k < K kMaxSrc)
    int2 sxy;                                // one source position (thread k < nsrc)
};

// Issue the prologue loads of (shot, tile) for the K steps from n0: tile descriptor, state
// (kFields, from the state buffer st), coefficients (kCoef), CPML memories and profiles
// (strip tiles), source samples and positions.  kCG: read the state through L2 only (the
// persistent kernels read what other CTAs of the same launch wrote).
template <int R, int NW, bool kFields, bool kCoef, bool kPsi, bool kCG, bool kSrc>
__device__ __forceinline__ void issue_loads(const TileParams& p, const Pos<R>& w, const float* st,
                                            int shot, int tile, int n0, int K, bool strip,
                                            TileLoads<R>& L) {
    using Gm = G<R, NW>;
    const int tid = threadIdx.x;
    const float2 z = make_float2(0.f, 0.f);
    L.d = __ldg(p.tile_desc + (long long)shot * p.ntiles + tile);
    const long long F = (long long)p.nshots * p.Np;
    const long long sb = (long long)shot * p.Np;
    auto ld = [&](const float* a) { return kCG ? ld2cg(a) : ld2(a); };
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const bool in = w.lane_in && ((w.row_in >> r) & 1u);
        const long long m = (long long)(w.Y0 + w.ly0 + r) * p.pitch + w.gx0;
        const float* s = st + sb + m;
        L.f0[r] = L.f1[r] = L.f2[r] = L.u[r] = L.v[r] = z;
        L.pex[r] = L.phy[r] = L.pey[r] = L.phx[r] = z;
        if (in) {
            if (kFields) {
                L.f0[r] = ld(s);
                L.f1[r] = ld(s + F);
                L.f2[r] = ld(s + 2 * F);
            }
            if (kCoef) {
                L.u[r] = __ldg(reinterpret_cast<const float2*>(p.ca + m));
                L.v[r] = __ldg(reinterpret_cast<const float2*>(p.cb + m));
            }
            if (kPsi && strip && (w.xs0 || w.xs1)) {
                L.pex[r] = ld(s + 3 * F);
                L.phy[r] = ld(s + 6 * F);
            }
            if (kPsi && strip && ((w.ymask >> r) & 1u)) {
                L.pey[r] = ld(s + 4 * F);
                L.phx[r] = ld(s + 5 * F);
            }
        }
    }
    if (strip && tid < Gm::WY + WX) {
        const AxisProfile& a = tid < Gm::WY ? p.py : p.px;
        const int g = tid < Gm::WY ? min(max(w.Y0 + tid, 0), p.ny - 1)
                                   : min(max(w.X0 + tid - Gm::WY, 0), p.nx - 1);
        L.prof[0] = __ldg(a.aE + g);
        L.prof[1] = __ldg(a.bE + g);
        L.prof[2] = __ldg(a.cE + g);
        L.prof[3] = __ldg(a.aH + g);
        L.prof[4] = __ldg(a.bH + g);
        L.prof[5] = __ldg(a.cH + g);
    }
    L.wv = 0.f;
    if (kSrc && tid < K * kMaxSrc) {
        const int stp = tid / kMaxSrc, src = tid - stp * kMaxSrc;
        if (src < p.nsrc)
            L.wv = __ldg(p.wavelet + ((long long)shot * p.nsrc + src) * p.nt + n0 + stp);
    }
    if (kSrc && tid < p.nsrc) L.sxy = __ldg(p.src_xy + (long long)shot * p.nsrc + tid);
}

// Shared-memory stores of the prologue loads: coefficients (kCoef), CPML memories and
// profiles (strip tiles; zero memories elsewhere in the planes the strip forms read: x planes
// of x-strip tiles, y planes of every row of a y-strip warp), source samples wsrc[st][k] and
// window positions srcpos[k] (lx | ly << 8, -1 for sources outside the live window).
template <int R, int NW, bool kCoef, bool kPsi, bool kSrc>
__device__ __forceinline__ void store_loads(const TileParams& p, const Pos<R>& w, float* sm,
                                            int K, bool strip, TileLoads<R>& L) {
    using Gm = G<R, NW>;
    const int tid = threadIdx.x;
    float2* psi = reinterpret_cast<float2*>(sm + Gm::oPsi) + w.ly0 * 32 + w.lane;
    float2* coef = reinterpret_cast<float2*>(sm + Gm::oCoef) + w.ly0 * 32 + w.lane;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (kCoef) {
            coef[r * 32] = L.u[r];
            coef[Gm::PL + r * 32] = L.v[r];
        }
        if (kPsi && strip && w.tile_xs) {
            if (!w.xs0) L.pex[r].x = L.phy[r].x = 0.f;
            if (!w.xs1) L.pex[r].y = L.phy[r].y = 0.f;
            psi[r * 32] = L.pex[r];
            psi[3 * Gm::PL + r * 32] = L.phy[r];
        }
        if (kPsi && strip && w.ys) {
            psi[Gm::PL + r * 32] = L.pey[r];
            psi[2 * Gm::PL + r * 32] = L.phx[r];
        }
    }
    if (strip && tid < Gm::WY + WX) {
        if (tid < Gm::WY) {
            float4* yp = reinterpret_cast<float4*>(sm + Gm::oYp) + 2 * tid;
            yp[0] = make_float4(L.prof[0], L.prof[1], L.prof[2], 0.f);
            yp[1] = make_float4(L.prof[3], L.prof[4], L.prof[5], 0.f);
        } else {
            float* xp = sm + Gm::oXp + tid - Gm::WY;  // plane k, column c at xp[k * 64]
#pragma unroll
            for (int k = 0; k < 6; ++k) xp[k * WX] = L.prof[k];
        }
    }
    if (!kSrc) return;
    const int mask = L.d.z;
    if (tid < K * kMaxSrc) {
        const int src = tid % kMaxSrc;
        (sm + Gm::oWs)[tid] = ((mask >> src) & 1) ? p.src_scale * L.wv : 0.f;
    }
    if (tid < kMaxSrc) {
        int pos = -1;
        if (tid < p.nsrc && ((mask >> tid) & 1)) {
            const int lx = L.sxy.x - w.X0, ly = L.sxy.y - w.Y0;
            if (lx >= 0 && lx < WX && ly >= 0 && ly < Gm::WY) pos = lx | ly << 8;
        }
        reinterpret_cast<int*>(sm + Gm::oSp)[tid] = pos;
    }
}

// Thread 0: TMA boxes of the window at (X0, Y0) for `shot` into the shared-memory planes,
// counted on the mbarrier `bar` (initialised here): the state (fields 0-2 into the staging
// planes), the update coefficients (Ca, Cb planes) and, for strip tiles, the CPML memories
// (fields 3-6 into the psi planes; zero outside the strips in the buffers, so the planes need
// no clearing).  Zero fill outside the grid.
template <int R, int NW>
__device__ __forceinline__ void tma_window(const TileMaps& m, float* sm, uint32_t bar, int nshots,
                                           int shot, int X0, int Y0, bool strip) {
    using Gm = G<R, NW>;
    constexpr uint32_t kPlane = Gm::WY * WX * sizeof(float);
    mbar_init(bar, 1);
    mbar_expect_tx(bar, (strip ? 9u : 5u) * kPlane);
    // the coefficients first: no kernel of the pass writes them, so they may load while the
    // previous launch of the pass still runs; the state only after it has completed
#pragma unroll
    for (int c = 0; c < 2; ++c)
        tma_load_3d(smem_u32(sm + Gm::oCoef + c * 2 * Gm::PL), &m.coef, X0, Y0, c, bar);
    pdl_wait();
#pragma unroll
    for (int f = 0; f < 3; ++f)
        tma_load_3d(smem_u32(sm + Gm::oStage + f * 2 * Gm::PL), &m.st, X0, Y0, f * nshots + shot, bar);
    if (strip) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            tma_load_3d(smem_u32(sm + Gm::oPsi + i * 2 * Gm::PL), &m.st, X0, Y0,
                        (3 + i) * nshots + shot, bar);
    }
}

// Wait (bounded) for the window's TMA boxes, then read the thread's state from the staging
// planes.  On expiry the timeout is recorded and the wait repeated once (the CTA must not end
// with copies in flight); the results of the launch are then not to be trusted.
template <int R, int NW>
__device__ __forceinline__ void tma_finish(const TileParams& p, const Pos<R>& w, float* sm,
                                           uint32_t bar, float2 (&f0)[R], float2 (&f1)[R],
                                           float2 (&f2)[R]) {
    using Gm = G<R, NW>;
    constexpr unsigned kPolls = 1u << 24;
    if (!mbar_wait(bar, 0, kPolls)) {
        if (threadIdx.x == 0) atomicOr(p.status, kStatusTimeout);
        mbar_wait(bar, 0, kPolls);
    }
    const float2* s = reinterpret_cast<const float2*>(sm + Gm::oStage) + w.ly0 * 32 + w.lane;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        f0[r] = s[r * 32];
        f1[r] = s[Gm::PL + r * 32];
        f2[r] = s[2 * Gm::PL + r * 32];
    }
}

// Write the owned interior cells (fields and strip memories) to the state buffer `st`.
template <int R, int NW>
__device__ __forceinline__ void store_state(const TileParams& p, const Pos<R>& w, const float* sm,
                                            float* st, int shot, const float2 (&f0)[R],
                                            const float2 (&f1)[R], const float2 (&f2)[R]) {
    using Gm = G<R, NW>;
    const long long F = (long long)p.nshots * p.Np;
    const long long sb = (long long)shot * p.Np;
    const float2* psi = reinterpret_cast<const float2*>(sm + Gm::oPsi) + w.ly0 * 32 + w.lane;
    if (!w.lane_int) return;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (!((w.row_int >> r) & 1u)) continue;
        float* s = st + sb + (long long)(w.Y0 + w.ly0 + r) * p.pitch + w.gx0;
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

// Does one of the thread's cells hold a source (after store_loads and a barrier)?
template <int R, int NW>
__device__ __forceinline__ bool thread_has_source(const TileParams& p, const Pos<R>& w,
                                                  const float* sm) {
    using Gm = G<R, NW>;
    const int* srcpos = reinterpret_cast<const int*>(sm + Gm::oSp);
    bool any = false;
    for (int k = 0; k < p.nsrc; ++k) {
        const int pos = srcpos[k], r = (pos >> 8) - w.ly0;
        any |= pos >= 0 && ((pos & 0xff) >> 1) == w.lane && r >= 0 && r < R;
    }
    return any;
}

// ---------------------------------------------------------------------------------------
// Receivers
// ---------------------------------------------------------------------------------------
// A tile's receiver list (host-built, sorted by row) holds entries {receiver index, packed
// position (x - tx tile_w + kRel) | (y - ty tile_h + kRel) << 16} of the receivers in the
// window [tx tile_w - K, tx tile_w + tile_w + K) x [ty tile_h - K, ty tile_h + tile_h + K)
// of the context's K.  In a window of the kernels the entry sits at lx = x - X0, ly = y - Y0,
// packed as lx | (ly + kRowBias) << 8 | interior << 16: a shorter last block starts its window
// lower, so a few entries can sit above row 0 (they match no thread); the bias keeps the packed
// rows non-negative and in list order.  With kStaged the packed positions and receiver indices
// are staged in shared memory (rec[e], rec[nrl + e]; in the adjoint also the residual samples
// rec[2 nrl + e K + st] of steps n1 - st); otherwise they are read from the list when used.
constexpr int kRel = 64;
constexpr int kRowBias = 64;
__device__ __forceinline__ int rec_position(const TileParams& p, int2 ent, int K) {
    const int lx = (ent.y & 0xffff) - kRel + p.kl, ly = (ent.y >> 16) - kRel + K;
    const bool interior = lx >= p.kl && lx < p.kl + p.tile_w && ly >= K && ly < K + p.tile_h;
    return (lx & 0xff) | (ly + kRowBias) << 8 | (interior ? 1 << 16 : 0);
}
__device__ __forceinline__ int rec_row(int pos) { return ((pos >> 8) & 0xff) - kRowBias; }

template <bool kStaged>
__device__ __forceinline__ void rec_entry(const TileParams& p, const int* srec, const int2* ents,
                                          int nrl, int e, int K, int& pos, int& ri) {
    if (kStaged) {
        pos = srec[e];
        ri = srec[nrl + e];
    } else {
        const int2 ent = __ldg(ents + e);
        ri = ent.x;
        pos = rec_position(p, ent, K);
    }
}

// Stage the receiver list of a tile (descriptor d: first entry, entries) and, with kAdj, the
// residual samples of steps n1, n1 - 1, .., n1 - K + 1.  Returns the list's entries.
template <int R, int NW, bool kStaged, bool kAdj>
__device__ __forceinline__ const int2* stage_receivers(const TileParams& p, float* sm, int shot,
                                                       int4 d, int n1, int K) {
    using Gm = G<R, NW>;
    const int tid = threadIdx.x, nrl = d.y;
    const int2* ents = p.tile_rec + d.x;
    if (kStaged && nrl > 0) {
        int* srec = reinterpret_cast<int*>(sm + Gm::oRec);
        for (int e = tid; e < nrl; e += Gm::NT) {
            const int2 ent = __ldg(ents + e);
            srec[e] = rec_position(p, ent, K);
            srec[nrl + e] = ent.x;
        }
        if (kAdj) {
            const float* rb = p.resid + (long long)shot * p.nt * p.nrec;
            for (int i = tid; i < nrl * K; i += Gm::NT) {
                const int e = i / K, st = i - e * K;
                srec[2 * nrl + i] =
                    __float_as_int(__ldg(rb + (long long)(n1 - st) * p.nrec + __ldg(ents + e).x));
            }
        }
    }
    return ents;
}

// Entries [lo, hi) of the row-sorted list on the warp's rows [ly0, ly0 + R).
template <bool kStaged, int R>
__device__ __forceinline__ void warp_rec_range(const TileParams& p, const Pos<R>& w,
                                               const int* srec, const int2* ents, int nrl, int K,
                                               int& lo, int& hi) {
    lo = hi = 0;
    for (int base = 0; base < nrl; base += 32) {
        const int e = base + w.lane;
        int ly = 1 << 20;
        if (e < nrl) {
            int pos, ri;
            rec_entry<kStaged>(p, srec, ents, nrl, e, K, pos, ri);
            ly = rec_row(pos);
        }
        lo += __popc(__ballot_sync(kFull, ly < w.ly0));
        hi += __popc(__ballot_sync(kFull, ly < w.ly0 + R));
    }
}

// The receiver entries of a thread's cells, found once per tile so that every step records
// (or injects) them in parallel across the warp instead of one warp walking the list: at
// most two per thread, each packed as entry << 4 | row << 1 | column (-1 = none); `walk`
// (warp-uniform) when some lane holds more, and the warp then walks its range every step.
struct OwnRec {
    int e0, e1;
    bool walk;
};

template <bool kStaged, int R>
__device__ __forceinline__ OwnRec own_receivers(const TileParams& p, const Pos<R>& w,
                                                const int* srec, const int2* ents, int nrl, int K,
                                                int rlo, int rhi, bool interior_only) {
    OwnRec o;
    o.e0 = o.e1 = -1;
    int n = 0;
    for (int e = rlo; e < rhi; ++e) {
        int pos, ri;
        rec_entry<kStaged>(p, srec, ents, nrl, e, K, pos, ri);
        if (((pos & 0xff) >> 1) == w.lane && (!interior_only || (pos >> 16))) {
            const int code = e << 4 | (rec_row(pos) - w.ly0) << 1 | (pos & 1);
            if (n == 0) o.e0 = code;
            else if (n == 1) o.e1 = code;
            ++n;
        }
    }
    o.walk = __any_sync(kFull, n > 2);
    return o;
}

// ---------------------------------------------------------------------------------------
// Row updates of one warp (no per-row branches: the rows are independent chains)
// ---------------------------------------------------------------------------------------
// H update of the warp's rows from Ez^n (eb: Ez of the row below the warp), with the x-CPML
// form in every column when XS and the y-CPML form in every row when YS (both reduce to the
// plain update outside the strips).
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
                                       const float4* yp, const float2* coef, float2 (&ez)[R],
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
        const float2 ca = coef[r * 32], cb = coef[G<R, NW>::PL + r * 32];
        ez[r].x = fmaf(ca.x, ez[r].x, cb.x * q0);
        ez[r].y = fmaf(ca.y, ez[r].y, cb.y * q1);
    }
}

// Phase A of the warp's rows: lam = Cb adj(Ez^{n+1}); zero-lag gradient sums with Ez^{n+1}
// (ring slot `prev`) and Ez^n (ring slot `slot`) on the owned cells; electric CPML and the S
// weights (wx, wy); adj(Ez^n) starts as Ca adj(Ez^{n+1}).  The gradient sums carry no
// constant factor (applied once per tile).  rs: ring row stride in float2.
template <int R, int NW, bool XS, bool YS>
__device__ __forceinline__ void a_rows(const TileParams& p, float2* psi, const float2* xp,
                                       const float4* yp, const float2* coef, const float2* slot,
                                       const float2* prev, int rs, const bool (&own)[R],
                                       float2 (&aez)[R], float2 (&ge)[R], float2 (&gs)[R],
                                       float2 (&wx)[R], float2 (&wy)[R]) {
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
        float2 pf = make_float2(0.f, 0.f), en1 = pf;
        if (own[r]) {
            pf = slot[r * rs];
            en1 = prev[r * rs];
        }
        const float2 ca = coef[r * 32], cb = coef[G<R, NW>::PL + r * 32];
        const float l0 = cb.x * aez[r].x, l1 = cb.y * aez[r].y;
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
        aez[r].x *= ca.x;
        aez[r].y *= ca.y;
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

// The adjoint's wavefield ring: kRing slots of the tile interior (tile_h rows of rs =
// tile_w / 2 float2); the owned cell (row r, lane) of a thread at ring + r rs in a slot.
struct Ring {
    float2* base;   // thread's cell of row 0 in slot 0
    int rs;         // row stride (float2)
    int slot;       // slot stride (float2)
};

// Ez^n of the owned cells for phase A number a (step n = n1 - a; a = -1 gives Ez^{n1+1}) into
// ring slot (a + kRing) % kRing, zero when n = 0 (Ez^0 = 0); one cp.async group per a, empty
// when a >= K.  Cells the thread does not own are not fetched.  hp: the owned cells' store,
// Ez^{m+1} of row r at hp + m Np + r pitch.
template <int R>
__device__ __forceinline__ void ring_fetch(const TileParams& p, const Ring& rg, const float* hp,
                                           const bool (&own)[R], int n1, int K, int a) {
    if (a < K) {
        const int n = n1 - a;
        float2* slot = rg.base + ((a + kRing) % kRing) * rg.slot;
        const float* h = hp + (long long)(n >= 1 ? n - 1 : 0) * p.Np;
        const int bytes = n >= 1 ? 8 : 0;
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (own[r]) cp_async8(slot + r * rg.rs, h + (long long)r * p.pitch, bytes);
    }
    cp_async_commit();
}

// The magnetic components of receiver ri at step n (H^{n-1/2}: Hx at (i, j+1/2), Hy at
// (i+1/2, j), the values the registers hold before the step's H update).
template <int R>
__device__ __forceinline__ void record_h(const TileParams& p, int shot, int n, int ri,
                                         const float2 (&hx)[R], const float2 (&hy)[R], int r,
                                         int c) {
    float* th = p.traces_h + (((long long)shot * p.nt + n) * p.nrec + ri) * 2;
    th[0] = pick<R>(hx, r, c);
    th[1] = pick<R>(hy, r, c);
}

// ---------------------------------------------------------------------------------------
// Time-step loops of one tile
// ---------------------------------------------------------------------------------------
// Forward steps n0 .. n0 + K - 1 of (shot, tile) with the window state in ez, hx, hy (and the
// strip memories, coefficients, profiles, sources and receivers staged in shared memory).
template <int R, int NW, bool XS, bool kHist, bool kIllum, bool kStaged>
__device__ __forceinline__ void fwd_steps(const TileParams& p, const Pos<R>& w, float* sm,
                                          int shot, int n0, int K, float2 (&ez)[R],
                                          float2 (&hx)[R], float2 (&hy)[R], float2 (&ill)[R],
                                          int rlo, int rhi, int nrl, const int2* ents,
                                          const OwnRec& orc, bool srcany) {
    using Gm = G<R, NW>;
    float2* top = reinterpret_cast<float2*>(sm + Gm::oTop);
    float2* bot = reinterpret_cast<float2*>(sm + Gm::oBot);
    float2* psi = reinterpret_cast<float2*>(sm + Gm::oPsi) + w.ly0 * 32 + w.lane;
    const float2* xp = reinterpret_cast<const float2*>(sm + Gm::oXp) + w.lane;
    const float4* yp = reinterpret_cast<const float4*>(sm + Gm::oYp) + 2 * w.ly0;
    const float2* coef = reinterpret_cast<const float2*>(sm + Gm::oCoef) + w.ly0 * 32 + w.lane;
    const int* srec = reinterpret_cast<const int*>(sm + Gm::oRec);
    const int* srcpos = reinterpret_cast<const int*>(sm + Gm::oSp);
    const float* wsrc = sm + Gm::oWs;
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

    for (int st = 0; st < K; ++st) {
        const int n = n0 + st;
        // 1. receivers in this tile's interior: d^n = Ez^n (loop bounds are warp-uniform)
        if (orc.walk) {
            for (int e = rlo; e < rhi; ++e) {
                int pos, ri;
                rec_entry<kStaged>(p, srec, ents, nrl, e, K, pos, ri);
                if (((pos & 0xff) >> 1) == w.lane && (pos >> 16)) {
                    const int rr = rec_row(pos) - w.ly0, cc = pos & 1;
                    tr[(long long)n * p.nrec + ri] = pick<R>(ez, rr, cc);
                    if (kIllum && p.traces_h) record_h<R>(p, shot, n, ri, hx, hy, rr, cc);
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int code = q ? orc.e1 : orc.e0;
                if (code >= 0) {
                    const int e = code >> 4;
                    const int ri = kStaged ? srec[nrl + e] : __ldg(ents + e).x;
                    tr[(long long)n * p.nrec + ri] = pick<R>(ez, (code >> 1) & 7, code & 1);
                    if (kIllum && p.traces_h)
                        record_h<R>(p, shot, n, ri, hx, hy, (code >> 1) & 7, code & 1);
                }
            }
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
                    const float2 cb = coef[Gm::PL + r * 32];
                    add_at<R>(ez, r, c, -(c ? cb.y : cb.x) * wsrc[st * kMaxSrc + k]);
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

// Accumulate the illumination of the owned cells into the per-shot planes.
template <int R>
__device__ __forceinline__ void add_illumination(const TileParams& p, const Pos<R>& w, int shot,
                                                 const float2 (&ill)[R]) {
    if (!w.lane_int) return;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (!((w.row_int >> r) & 1u)) continue;
        float* a = p.illum + (long long)shot * p.Np + (long long)(w.Y0 + w.ly0 + r) * p.pitch + w.gx0;
        float2 v = ld2cg(a);  // earlier blocks of this tile may have run on another SM
        v.x += ill[r].x;
        v.y += ill[r].y;
        st2(a, v);
    }
}

// Adjoint steps n0 + K - 1 down to n0 of (shot, tile) with the adjoint window state in aez,
// ahx, ahy; gradient sums in ge, gs.  The ring's first kRingLead + 1 groups (a = -1 .. 2) must
// have been requested (ring_fetch) before.  after_a(a) runs after phase A number a (the
// persistent kernel issues prefetches there).
template <int R, int NW, bool XS, bool kStaged, class AfterA>
__device__ __forceinline__ void adj_steps(const TileParams& p, const Pos<R>& w, float* sm,
                                          int shot, int n0, int K, float2 (&aez)[R],
                                          float2 (&ahx)[R], float2 (&ahy)[R], float2 (&ge)[R],
                                          float2 (&gs)[R], const float* hp, const bool (&own)[R],
                                          const Ring& rg, int rlo, int rhi, int nrl,
                                          const int2* ents, const OwnRec& orc, AfterA after_a) {
    using Gm = G<R, NW>;
    const int n1 = n0 + K - 1;
    float2* top = reinterpret_cast<float2*>(sm + Gm::oTop);
    float2* bot = reinterpret_cast<float2*>(sm + Gm::oBot);
    float2* psi = reinterpret_cast<float2*>(sm + Gm::oPsi) + w.ly0 * 32 + w.lane;
    const float2* xp = reinterpret_cast<const float2*>(sm + Gm::oXp) + w.lane;
    const float4* yp = reinterpret_cast<const float4*>(sm + Gm::oYp) + 2 * w.ly0;
    const float2* coef = reinterpret_cast<const float2*>(sm + Gm::oCoef) + w.ly0 * 32 + w.lane;
    const int* srec = reinterpret_cast<const int*>(sm + Gm::oRec);
    const float* rbase = p.resid + (long long)shot * p.nt * p.nrec;
    const float2* below = top + (w.warp + 1) * 32 + w.lane;
    const float2* above = bot + (w.warp - 1) * 32 + w.lane;
    float2 wx[R], wy[R];
    auto phase_a = [&](int a) {
        ring_fetch<R>(p, rg, hp, own, n1, K, a + kRingLead);
        cp_async_wait<kRingLead>();
        const float2* slot = rg.base + (a % kRing) * rg.slot;
        const float2* prev = rg.base + ((a + kRing - 1) % kRing) * rg.slot;
        if (w.ys)
            a_rows<R, NW, XS, true>(p, psi, xp, yp, coef, slot, prev, rg.rs, own, aez, ge, gs, wx, wy);
        else
            a_rows<R, NW, XS, false>(p, psi, xp, yp, coef, slot, prev, rg.rs, own, aez, ge, gs, wx, wy);
        after_a(a);
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
        if (orc.walk) {
            for (int e = rlo; e < rhi; ++e) {
                int pos, ri;
                rec_entry<kStaged>(p, srec, ents, nrl, e, K, pos, ri);
                if (((pos & 0xff) >> 1) == w.lane) {
                    const float v = kStaged ? __int_as_float(srec[2 * nrl + e * K + st])
                                            : __ldg(rbase + (long long)n * p.nrec + ri);
                    add_at<R>(aez, rec_row(pos) - w.ly0, pos & 1, v);
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int code = q ? orc.e1 : orc.e0;
                if (code >= 0) {
                    const int e = code >> 4;
                    const float v = kStaged ? __int_as_float(srec[2 * nrl + e * K + st])
                                            : __ldg(rbase + (long long)n * p.nrec + __ldg(ents + e).x);
                    add_at<R>(aez, (code >> 1) & 7, code & 1, v);
                }
            }
        }
        if (st < K - 1) phase_a(st + 1);
    }
}

// a[0] += x, a[1] += y as one fire-and-forget vector reduction (no value returned, so the
// thread does not wait for it)
__device__ __forceinline__ void red_add2(float* a, float x, float y) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};\n" ::"l"(a), "f"(x), "f"(y) : "memory");
}

// Add the tile's gradient sums (owned cells) to the per-shot accumulators: g_eps_r gets
// -eps0/dt sum lam (Ez^{n+1} - Ez^n), g_sigma gets -1/2 sum lam (Ez^{n+1} + Ez^n).  One writer
// per cell per tile and tiles of a cell in a fixed order: a fire-and-forget reduction is
// deterministic and hides the read latency of +=.
template <int R>
__device__ __forceinline__ void add_gradients(const TileParams& p, const Pos<R>& w, int shot,
                                              const float2 (&ge)[R], const float2 (&gs)[R]) {
    if (!w.lane_int) return;
    const long long F = (long long)p.nshots * p.Np;
    const float se = -p.geps;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (!((w.row_int >> r) & 1u)) continue;
        float* g = p.grad + (long long)shot * p.Np + (long long)(w.Y0 + w.ly0 + r) * p.pitch + w.gx0;
        red_add2(g, se * ge[r].x, se * ge[r].y);
        red_add2(g + F, -0.5f * gs[r].x, -0.5f * gs[r].y);
    }
}

// Ring of a tile (see Ring) in the shared-memory region at ring_off.
template <int R, int NW>
__device__ __forceinline__ Ring make_ring(const TileParams& p, const Pos<R>& w, float* sm,
                                          int ring_off, int K) {
    Ring rg;
    rg.rs = p.tile_w / 2;
    rg.slot = rg.rs * p.tile_h;
    rg.base = reinterpret_cast<float2*>(sm + ring_off) + (w.ly0 - K) * rg.rs + (w.lane - p.kl / 2);
    return rg;
}

}  // namespace
}  // namespace gf
