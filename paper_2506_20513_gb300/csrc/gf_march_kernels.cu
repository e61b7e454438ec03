// gf_march_kernels.cu -- barrier-free "warp march" forward kernel (sm_103a).
//
// Each warp owns a strip of 64 staged columns (two per lane: lane and lane + 32) of one shot
// and a chunk of H interior rows, and advances it K time steps (levels) in one pass down
// the rows: at march iteration i, level 0 loads row i of the input state, and level s
// (1 <= s <= K) advances row i - s from time n0 + s - 1 to n0 + s.  This is valid because an
// H update at row y reads Ez at rows y and y + 1 of the previous level (row y + 1 was just
// produced by level s - 1 in the same iteration) and an E update at row y reads Hx at row
// y - 1 of its own level (produced one iteration earlier).  The field values of the last
// two rows of every level stay in registers (row parity selects the slot); x-neighbours come
// from warp shuffles; update coefficients and CPML memories of the K + 1 rows in flight sit
// in a per-warp shared-memory ring, each lane touching only its own columns.  No CTA-wide
// barrier is needed.  The halo (K columns on each side of the strip, K rows above and below
// the chunk) is recomputed redundantly, exactly as in the tile kernels, and only the owned
// interior is written back.  The step order is that of Algorithm 1 (Sec. 3.3), in the Ca/Cb
// form of the Sec. 3.2 coefficient listing.
#include "gf_internal.cuh"

namespace gf {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMW = 4;          // warps per CTA
constexpr int kCols = 64;       // staged columns per warp
constexpr int kRing = 8;        // rows in flight (>= K + 1)
constexpr int kMaxWarpRec = 128;

struct RecEntry {
    int row, col, idx;  // global row, staged column, receiver index
};

struct WarpSmem {
    float coef[kRing][2][kCols];  // Ca, Cb
    float psi[kRing][4][kCols];   // CPML memories Ex, Ey, Hx, Hy
    float xprof[6][kCols];        // column profiles aE bE cE aH bH cH
    RecEntry rec[kMaxWarpRec];    // owned receivers, sorted by (row, index)
    int src_row[kMaxSrc], src_col[kMaxSrc];
    int nrec;
};

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

// Value one column to the right for columns (lane, lane + 32); the last staged column has
// no right neighbour (halo edge) and gets its own value.
__device__ __forceinline__ void right_of(float a, float b, int lane, float& ra, float& rb) {
    const float da = __shfl_down_sync(kFull, a, 1);
    const float db = __shfl_down_sync(kFull, b, 1);
    const float b0 = __shfl_sync(kFull, b, 0);
    ra = lane < 31 ? da : b0;
    rb = lane < 31 ? db : b;
}
// Value one column to the left; the first staged column gets its own value.
__device__ __forceinline__ void left_of(float a, float b, int lane, float& la, float& lb) {
    const float ua = __shfl_up_sync(kFull, a, 1);
    const float ub = __shfl_up_sync(kFull, b, 1);
    const float a31 = __shfl_sync(kFull, a, 31);
    la = lane > 0 ? ua : a;
    lb = lane > 0 ? ub : a31;
}

struct MarchGeom {
    int lane, X0, Y0, Ys, gx[2];
    bool in[2], own[2], xs[2];
    int shot;
};

template <int K, bool kHist>
struct FwdMarch {
    const TileParams& p;
    WarpSmem& w;
    const MarchGeom& g;
    float E[K + 1][2][2], HX[K + 1][2][2], HY[K + 1][2][2];  // [level][row parity][column]
    int rcur[K];                                             // receiver cursor per level

    __device__ FwdMarch(const TileParams& p_, WarpSmem& w_, const MarchGeom& g_)
        : p(p_), w(w_), g(g_) {
#pragma unroll
        for (int s = 0; s <= K; ++s)
#pragma unroll
            for (int q = 0; q < 2; ++q)
#pragma unroll
                for (int c = 0; c < 2; ++c) E[s][q][c] = HX[s][q][c] = HY[s][q][c] = 0.f;
#pragma unroll
        for (int s = 0; s < K; ++s) rcur[s] = 0;
    }

    __device__ __forceinline__ bool ystrip(int y) const {
        return y < p.npml || y >= p.ny - p.npml - 1;
    }

    // record d^{n0+s} = Ez^{n0+s} of row y for the receivers this warp owns
    __device__ __forceinline__ void record(int s, int y, const float (&e)[2]) {
        int c = rcur[s];
        while (c < w.nrec && w.rec[c].row < y) ++c;
        while (c < w.nrec && w.rec[c].row == y) {
            const RecEntry r = w.rec[c];
            const int col = r.col;
            if ((col & 31) == g.lane)
                p.traces[((long long)g.shot * p.nt + p.n0 + s) * p.nrec + r.idx] =
                    col >= 32 ? e[1] : e[0];
            ++c;
        }
        rcur[s] = c;
    }

    template <int P>
    __device__ __forceinline__ void row(int i) {
        const long long F = (long long)p.nshots * p.N;
        const long long sbase = (long long)g.shot * p.N;
        // level 0: load row i of the input state into registers and the ring
        {
            const int y = i, rr = y & (kRing - 1);
            const bool yin = y >= 0 && y < p.ny;
            const bool ys = yin && ystrip(y);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int col = g.lane + 32 * c;
                float e = 0.f, hx = 0.f, hy = 0.f, ca = 0.f, cb = 0.f;
                float pex = 0.f, pey = 0.f, phx = 0.f, phy = 0.f;
                if (yin && g.in[c]) {
                    const long long gi = (long long)y * p.nx + g.gx[c], sg = sbase + gi;
                    e = p.st_in[sg];
                    hx = p.st_in[F + sg];
                    hy = p.st_in[2 * F + sg];
                    if (g.xs[c]) {
                        pex = p.st_in[3 * F + sg];
                        phy = p.st_in[6 * F + sg];
                    }
                    if (ys) {
                        pey = p.st_in[4 * F + sg];
                        phx = p.st_in[5 * F + sg];
                    }
                    const bool ring = g.gx[c] == 0 || y == 0 || g.gx[c] == p.nx - 1 || y == p.ny - 1;
                    coefficients(__ldg(p.eps_r + gi), __ldg(p.sigma + gi), p.dt_eps0, ring, ca, cb);
                }
                E[0][P][c] = e;
                HX[0][P][c] = hx;
                HY[0][P][c] = hy;
                w.coef[rr][0][col] = ca;
                w.coef[rr][1][col] = cb;
                w.psi[rr][0][col] = pex;
                w.psi[rr][1][col] = pey;
                w.psi[rr][2][col] = phx;
                w.psi[rr][3][col] = phy;
            }
            if (yin && K > 0) record(0, y, E[0][P]);
        }
        // levels 1..K: level s advances row i - s from time n0 + s - 1 to n0 + s
#pragma unroll
        for (int s = 1; s <= K; ++s) {
            const int y = i - s, rr = y & (kRing - 1);
            const int q = (P - s) & 1;  // parity slot of row y (rows y -/+ 1 use q ^ 1)
            const bool ys = y >= 0 && y < p.ny && ystrip(y);
            // H and magnetic CPML from Ez^{n0+s-1} (rows y, y + 1, column + 1)
            float ezr[2];
            right_of(E[s - 1][q][0], E[s - 1][q][1], g.lane, ezr[0], ezr[1]);
            float ayH = p.rdy, byH = 0.f, cyH = 0.f, ayE = p.rdy, byE = 0.f, cyE = 0.f;
            if (ys) {
                ayE = __ldg(p.py.aE + y);
                byE = __ldg(p.py.bE + y);
                cyE = __ldg(p.py.cE + y);
                ayH = __ldg(p.py.aH + y);
                byH = __ldg(p.py.bH + y);
                cyH = __ldg(p.py.cH + y);
            }
            float hyv[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int col = g.lane + 32 * c;
                const float e = E[s - 1][q][c];
                const float dyE = E[s - 1][q ^ 1][c] - e, dxE = ezr[c] - e;
                float hx = HX[s - 1][q][c], hy = HY[s - 1][q][c];
                if (g.xs[c] || ys) {
                    const float phx = byH * w.psi[rr][2][col] + cyH * dyE;
                    w.psi[rr][2][col] = phx;
                    hx -= p.ch * (ayH * dyE + phx);
                    const float phy = w.xprof[4][col] * w.psi[rr][3][col] + w.xprof[5][col] * dxE;
                    w.psi[rr][3][col] = phy;
                    hy += p.ch * (w.xprof[3][col] * dxE + phy);
                } else {
                    hx -= p.ch * (p.rdy * dyE);
                    hy += p.ch * (p.rdx * dxE);
                }
                HX[s][q][c] = hx;
                HY[s][q][c] = hy;
                hyv[c] = hy;
            }
            // E, electric CPML and the source, giving Ez^{n0+s}
            float hyl[2];
            left_of(hyv[0], hyv[1], g.lane, hyl[0], hyl[1]);
            float enew[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int col = g.lane + 32 * c;
                const float dxH = hyv[c] - hyl[c], dyH = HX[s][q][c] - HX[s][q ^ 1][c];
                float qq;
                if (g.xs[c] || ys) {
                    const float pex = w.xprof[1][col] * w.psi[rr][0][col] + w.xprof[2][col] * dxH;
                    w.psi[rr][0][col] = pex;
                    const float pey = byE * w.psi[rr][1][col] + cyE * dyH;
                    w.psi[rr][1][col] = pey;
                    qq = w.xprof[0][col] * dxH + pex - (ayE * dyH + pey);
                } else {
                    qq = p.rdx * dxH - p.rdy * dyH;
                }
                for (int k = 0; k < p.nsrc; ++k)
                    if (w.src_row[k] == y && w.src_col[k] == col)
                        qq -= p.src_scale *
                              __ldg(p.wavelet + ((long long)g.shot * p.nsrc + k) * p.nt + p.n0 + s - 1);
                const float v = w.coef[rr][0][col] * E[s - 1][q][c] + w.coef[rr][1][col] * qq;
                E[s][q][c] = v;
                enew[c] = v;
                if (kHist && g.own[c] && y >= g.Y0 && y < g.Y0 + p.tile_h && y < p.ny)
                    __stcs(p.hist + ((long long)g.shot * p.hist_stride + p.n0 + s - 1 - p.hist_slot0) * p.N +
                               (long long)y * p.nx + g.gx[c],
                           v);
            }
            const bool yown = y >= g.Y0 && y < g.Y0 + p.tile_h && y < p.ny;
            if (s < K && yown) record(s, y, enew);
            if (s == K && yown) {
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    if (!g.own[c]) continue;
                    const int col = g.lane + 32 * c;
                    const long long sg = sbase + (long long)y * p.nx + g.gx[c];
                    p.st_out[sg] = E[K][q][c];
                    p.st_out[F + sg] = HX[K][q][c];
                    p.st_out[2 * F + sg] = HY[K][q][c];
                    if (g.xs[c]) {
                        p.st_out[3 * F + sg] = w.psi[rr][0][col];
                        p.st_out[6 * F + sg] = w.psi[rr][3][col];
                    }
                    if (ys) {
                        p.st_out[4 * F + sg] = w.psi[rr][1][col];
                        p.st_out[5 * F + sg] = w.psi[rr][2][col];
                    }
                }
            }
        }
    }
};

// The receivers of this warp's interior from the host-built list of its tile (already in
// (row, index) order), compacted in order with a warp ballot; and the sources inside its
// staged columns.
__device__ void stage_lists(const TileParams& p, WarpSmem& w, const MarchGeom& g, int tile) {
    const long long lo = p.tile_rec_off[(long long)g.shot * p.ntiles + tile];
    const int n = (int)(p.tile_rec_off[(long long)g.shot * p.ntiles + tile + 1] - lo);
    const int* rl = p.tile_rec_idx + lo;
    const int* cells = p.rec_cell + (long long)g.shot * p.nrec;
    int count = 0;
    for (int base = 0; base < n; base += 32) {
        const int e = base + g.lane;
        RecEntry r{0, 0, 0};
        bool keep = false;
        if (e < n) {
            const int ri = __ldg(rl + e), cell = __ldg(cells + ri);
            r = RecEntry{cell / p.nx, cell % p.nx - g.X0, ri};
            keep = r.col >= p.halo && r.col < p.halo + p.tile_w && r.row >= g.Y0 &&
                   r.row < g.Y0 + p.tile_h;
        }
        const unsigned m = __ballot_sync(kFull, keep);
        const int pos = count + __popc(m & ((1u << g.lane) - 1u));
        if (keep && pos < kMaxWarpRec) w.rec[pos] = r;
        count += __popc(m);
    }
    if (g.lane == 0) w.nrec = count < kMaxWarpRec ? count : kMaxWarpRec;
    if (g.lane < kMaxSrc) {
        int row = -(1 << 30), col = -1;
        if (g.lane < p.nsrc) {
            const int cell = __ldg(p.src_cell + g.shot * p.nsrc + g.lane);
            const int c = cell % p.nx - g.X0;
            if (c >= 0 && c < kCols) {
                row = cell / p.nx;
                col = c;
            }
        }
        w.src_row[g.lane] = row;
        w.src_col[g.lane] = col;
    }
    // rows that level 0 never loads (above the march start) read zeros
    for (int r = 0; r < kRing; ++r)
        for (int c = 0; c < 2; ++c) {
            const int col = g.lane + 32 * c;
            w.coef[r][0][col] = 0.f;
            w.coef[r][1][col] = 0.f;
            for (int k = 0; k < 4; ++k) w.psi[r][k][col] = 0.f;
        }
    __syncwarp();
}

template <int K, bool kHist>
__global__ void __launch_bounds__(kMW * 32) fwd_march_kernel(const TileParams p, int chunks) {
    extern __shared__ float4 smem_raw[];
    const int warp = threadIdx.x >> 5;
    WarpSmem& w = reinterpret_cast<WarpSmem*>(smem_raw)[warp];
    const int gw = blockIdx.x * kMW + warp;
    const int strips = p.tiles_x;
    if (gw >= p.nshots * strips * chunks) return;  // whole warp
    MarchGeom g;
    g.lane = threadIdx.x & 31;
    g.shot = gw / (strips * chunks);
    const int rem = gw % (strips * chunks);
    const int strip = rem % strips, chunk = rem / strips;
    g.X0 = strip * p.tile_w - p.halo;
    g.Y0 = chunk * p.tile_h;
    g.Ys = g.Y0 - K;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int col = g.lane + 32 * c;
        g.gx[c] = g.X0 + col;
        g.in[c] = g.gx[c] >= 0 && g.gx[c] < p.nx;
        g.own[c] = col >= p.halo && col < p.halo + p.tile_w && g.gx[c] < p.nx;
        g.xs[c] = g.in[c] && (g.gx[c] < p.npml || g.gx[c] >= p.nx - p.npml - 1);
        const int gc = min(max(g.gx[c], 0), p.nx - 1);
        w.xprof[0][col] = __ldg(p.px.aE + gc);
        w.xprof[1][col] = __ldg(p.px.bE + gc);
        w.xprof[2][col] = __ldg(p.px.cE + gc);
        w.xprof[3][col] = __ldg(p.px.aH + gc);
        w.xprof[4][col] = __ldg(p.px.bH + gc);
        w.xprof[5][col] = __ldg(p.px.cH + gc);
    }
    stage_lists(p, w, g, chunk * strips + strip);
    FwdMarch<K, kHist> m(p, w, g);
    // level K reaches the chunk's last row at i = last; row<P> needs P = parity of i
    const int last = g.Y0 + p.tile_h - 1 + K;
    if (g.Ys & 1) {
        for (int i = g.Ys; i <= last; i += 2) {
            m.template row<1>(i);
            m.template row<0>(i + 1);
        }
    } else {
        for (int i = g.Ys; i <= last; i += 2) {
            m.template row<0>(i);
            m.template row<1>(i + 1);
        }
    }
}

}  // namespace

size_t march_smem_bytes() { return sizeof(WarpSmem) * kMW; }
int march_max_steps() { return kRing - 1; }

template <int K, bool H>
static cudaError_t allow_march(size_t optin) {
    return cudaFuncSetAttribute(fwd_march_kernel<K, H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)march_smem_bytes());
}

cudaError_t configure_march_kernels(size_t optin) {
    cudaError_t e = cudaSuccess;
#define GF_ALLOW(K)                                                   \
    if (e == cudaSuccess) e = allow_march<K, true>(optin);            \
    if (e == cudaSuccess) e = allow_march<K, false>(optin);
    GF_ALLOW(1) GF_ALLOW(2) GF_ALLOW(3) GF_ALLOW(4) GF_ALLOW(5) GF_ALLOW(6) GF_ALLOW(7)
#undef GF_ALLOW
    return e;
}

cudaError_t launch_fwd_march(const TileParams& p, int chunks, cudaStream_t st) {
    const long long warps = (long long)p.nshots * p.tiles_x * chunks;
    const dim3 grid((unsigned)((warps + kMW - 1) / kMW)), block(kMW * 32);
    const size_t smem = march_smem_bytes();
    const bool h = p.hist != nullptr;
    switch (p.K) {
#define GF_CASE(K)                                                                          \
    case K:                                                                                 \
        if (h) fwd_march_kernel<K, true><<<grid, block, smem, st>>>(p, chunks);             \
        else fwd_march_kernel<K, false><<<grid, block, smem, st>>>(p, chunks);              \
        break;
        GF_CASE(1) GF_CASE(2) GF_CASE(3) GF_CASE(4) GF_CASE(5) GF_CASE(6) GF_CASE(7)
#undef GF_CASE
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace gf
