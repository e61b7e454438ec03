// gf_api.cu -- host runtime behind the C ABI of include/gprfwi.h.
//
// Owns argument validation (CFL, Eq. cfl; geometry; sizes), the CPML profiles (built here in
// FP64 and uploaded as FP32), the workspace layout, and the launch sequence of the forward
// (Algorithm 1) and adjoint (Algorithm 2) time loops.  Every step of the path runs in the
// kernels of gf_tile_kernels.cu and gf_misc_kernels.cu; nothing is computed on the host
// except the model-independent CPML profiles and the Ricker helper.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <string>
#include <vector>

#include "../../include/gprfwi.h"
#include "gf_internal.cuh"

namespace {

constexpr double kEps0 = 8.8541878128e-12;  // F/m
constexpr double kMu0 = 1.25663706212e-6;   // H/m
constexpr double kC0 = 299792458.0;         // m/s
constexpr int kMisfitBlocks = 1024;
constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Offsets (bytes) of the workspace regions.
struct Layout {
    size_t status, partial, coef, done, stA, stB, illum, traces, resid, grad, hist, stC, stD, ckpt,
        seg, ring, total;
};

}  // namespace

// The stream operations of one context while a batch records them instead of running them
// (the persistent multi-instance schedule runs every context's operations in its own order,
// merging the persistent passes of several contexts into one launch).
struct StreamOp {
    int kind = -1;      // -1: copy or memset; GF_KERNEL_*: a kernel of that family
    bool flow = false;  // a persistent pass (inst, adjoint): mergeable across contexts
    bool adjoint = false;
    gf::FlowInstance inst{};
    std::function<cudaError_t(cudaStream_t)> run;  // the operation itself (non-flow)
    const char* what = "";
};
struct OpList {
    std::vector<StreamOp> ops;
};

struct gf_ctx {
    gf_grid_desc g;
    int nshots, nsrc, nrec, device;
    long long N;              // nx * ny (caller arrays)
    int pitch;                // row pitch of the internal planes (gf::row_pitch)
    long long Np;             // pitch * ny
    float* d_prof = nullptr;  // [12][max(nx, ny)] profiles (x: 6 arrays, y: 6 arrays)
    int2* d_src_xy = nullptr;  // [nshots][nsrc] source cells (x, y)
    int2* d_rec_xy = nullptr;  // [nshots][nrec] receiver cells (x, y), made by the TE model
    float* te_buf = nullptr;   // TE gradient: E history, traces and residual (library-owned)
    size_t te_bytes = 0;
    gf::AxisProfile px{}, py{};
    char* ws = nullptr;
    size_t ws_bytes = 0;
    bool ws_owned = false;
    bool have_forward = false;
    int tile_w = 48, tile_h = 50, K = 7, variant = 0;
    long long wait_budget = 1LL << 22;  // polls of one dependency wait (persistent kernels)
    // tensor maps of the tile launches: state buffer -> maps (window height of the variant)
    struct MapEntry {
        const float* st = nullptr;
        const float* coef = nullptr;
        int wy = 0;
        gf::TileMaps m;
    };
    MapEntry maps[4];
    int maps_next = 0;
    int store_mode = GF_STORE_FULL, ckpt_k = 0;
    int* d_ring_map = nullptr;  // [ny][nx] ring index (reconstruction mode), -1 inside
    int ring_cells = 0;
    const float* last_wavelet = nullptr;  // wavelet of the stored forward (recomputation)
    std::vector<int> h_rec;  // host copies of the receiver and source cells ([nshots][nrec],
    std::vector<int> h_src;  // [nshots][nsrc], linear j * nx + i)
    int4* d_tile_desc = nullptr;    // per (shot, tile) descriptors for the current tiling
    int2* d_tile_rec = nullptr;     // their receiver entries
    int* d_cta_order = nullptr;     // launch order of the (shot, tile) pairs: all shots, then
                                    // the shots of each lane
    int lanes = 2;                  // shot groups run concurrently on their own streams
    int lane_off[4] = {0}, lane_cnt[4] = {0};  // each lane's part of d_cta_order
    cudaStream_t lane_st[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t lane_fork = nullptr, lane_join[4] = {nullptr, nullptr, nullptr, nullptr};
    int tile_rec_max = 0;           // longest per (shot, tile) list of the current tiling
    long long generation = 0;        // bumped when launch parameters or buffers change
    size_t smem_optin = 0;
    long long launches = 0;
    OpList* rec = nullptr;  // set while a batch records this context's operations
    bool one_lane = false;  // set while a batch runs this context beside others
    bool profiling = false;
    // per kernel family: recorded (start, stop) event pairs not yet read
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev[3];
    std::vector<cudaEvent_t> ev_pool;
    char err[512] = {0};
};

namespace {

// Message of the last gf_create failure on this thread (there is no context to hold it).
thread_local char g_create_err[512] = "no error";

void create_fail(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_create_err, sizeof(g_create_err), fmt, ap);
    va_end(ap);
}

int fail(gf_ctx* c, int code, const char* fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int cuda_fail(gf_ctx* c, cudaError_t e, const char* what) {
    return fail(c, GF_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define GF_CUDA(ctx, call, what)                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, (what)); \
    } while (0)

cudaEvent_t take_event(gf_ctx* c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Launch one kernel (a callable returning cudaError_t) of family `kind`, counting it and,
// when profiling, bracketing it with events on `st`.
template <class F>
cudaError_t launch(gf_ctx* c, int kind, cudaStream_t st, F&& f) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->profiling) {
        e0 = take_event(c);
        e1 = take_event(c);
        cudaEventRecord(e0, st);
    }
    cudaError_t e = f();
    if (c->profiling) {
        cudaEventRecord(e1, st);
        c->prof_ev[kind].emplace_back(e0, e1);
    }
    if (e == cudaSuccess) ++c->launches;
    return e;
}

// Run a stream operation now, or append it to the context's recorder.
int stream_op(gf_ctx* c, cudaStream_t st, int kind, const char* what,
              std::function<cudaError_t(cudaStream_t)> f) {
    if (c->rec) {
        StreamOp op;
        op.kind = kind;
        op.run = std::move(f);
        op.what = what;
        c->rec->ops.push_back(std::move(op));
        return GF_OK;
    }
    const cudaError_t e = kind >= 0 ? launch(c, kind, st, [&] { return f(st); }) : f(st);
    return e == cudaSuccess ? GF_OK : cuda_fail(c, e, what);
}

// One persistent pass of the context, now or recorded.
int flow_op(gf_ctx* c, cudaStream_t st, const gf::FlowInstance& inst, bool adjoint,
            const char* what) {
    if (c->rec) {
        StreamOp op;
        op.kind = adjoint ? GF_KERNEL_ADJ : GF_KERNEL_FWD;
        op.flow = true;
        op.adjoint = adjoint;
        op.inst = inst;
        op.what = what;
        c->rec->ops.push_back(std::move(op));
        return GF_OK;
    }
    const cudaError_t e = launch(c, adjoint ? GF_KERNEL_ADJ : GF_KERNEL_FWD, st,
                                 [&] { return gf::launch_flow_pass(inst, adjoint, st); });
    return e == cudaSuccess ? GF_OK : cuda_fail(c, e, what);
}

// A stream operation: the expression after `what` runs on stream s_ (now or when a recorded
// schedule replays it; it captures by value).
#define GF_OP(ctx, st, kind, what, ...)                                                    \
    do {                                                                                  \
        const int rc_ = stream_op((ctx), (st), (kind), (what),                            \
                                  [=](cudaStream_t s_) -> cudaError_t { return __VA_ARGS__; }); \
        if (rc_) return rc_;                                                              \
    } while (0)

void drop_profile(gf_ctx* c) {
    for (auto& v : c->prof_ev) {
        for (auto& pr : v) {
            c->ev_pool.push_back(pr.first);
            c->ev_pool.push_back(pr.second);
        }
        v.clear();
    }
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// CPML profile of one node at depth u = rho / (npml d) in (0, 1] (convolutional PML,
// Roden & Gedney): graded sigma, kappa, alpha; recursive-convolution coefficients b, c.
void cpml_node(const gf_grid_desc& g, double d, double u, double& a, double& b, double& c) {
    if (u <= 0.0) {
        a = 1.0 / d;
        b = 0.0;
        c = 0.0;
        return;
    }
    const double m = g.pml_order;
    double smax = g.pml_sigma_max;
    if (smax <= 0.0) smax = 0.8 * (m + 1.0) / (sqrt(kMu0 / kEps0) * d * sqrt(g.pml_eps_ref));
    const double um = pow(u, m);
    const double sig = smax * um;
    const double kap = 1.0 + (g.pml_kappa_max - 1.0) * um;
    const double alp = g.pml_alpha_max * (1.0 - u);
    b = exp(-(sig / kap + alp) * g.dt / kEps0);
    c = sig > 0.0 ? sig * (b - 1.0) / (sig * kap + kap * kap * alp) / d : 0.0;
    a = 1.0 / (kap * d);
}

// Six FP32 arrays of length n for one axis: aE, bE, cE (integer nodes), aH, bH, cH
// (half nodes i + 1/2).  Depth is measured from the edge of the physical part
// [npml, n - 1 - npml].
void axis_profiles(const gf_grid_desc& g, int n, double d, float* out, int stride) {
    const double lo = g.npml, hi = n - 1 - g.npml;
    for (int i = 0; i < n; ++i) {
        for (int h = 0; h < 2; ++h) {
            const double pos = i + 0.5 * h;
            double rho = 0.0;
            if (pos < lo) rho = lo - pos;
            if (pos > hi) rho = pos - hi;
            const double u = g.npml > 0 ? rho / g.npml : 0.0;
            double a, b, c;
            cpml_node(g, d, u, a, b, c);
            out[(3 * h + 0) * stride + i] = (float)a;
            out[(3 * h + 1) * stride + i] = (float)b;
            out[(3 * h + 2) * stride + i] = (float)c;
        }
    }
}

int num_checkpoints(const gf_ctx* c) { return (c->g.nt + c->ckpt_k - 1) / c->ckpt_k; }

Layout layout_of(const gf_ctx* c, bool forward_only) {
    Layout L{};
    const size_t field = sizeof(float) * (size_t)c->nshots * (size_t)c->Np;
    const size_t tr = sizeof(float) * (size_t)c->nshots * c->g.nt * c->nrec;
    size_t o = 0;
    L.status = o; o = align_up(o + sizeof(int));
    L.partial = o; o = align_up(o + sizeof(double) * kMisfitBlocks * 5);  // total + 4 lanes
    L.coef = o; o = align_up(o + 2 * sizeof(float) * (size_t)c->Np);
    const size_t ntiles = (size_t)((c->g.nx + c->tile_w - 1) / c->tile_w) *
                          ((c->g.ny + c->tile_h - 1) / c->tile_h);
    L.done = o; o = align_up(o + sizeof(int) * ntiles * (size_t)c->nshots);
    L.stA = o; o = align_up(o + gf::kNumFields * field);
    L.stB = o; o = align_up(o + gf::kNumFields * field);
    L.illum = o; o = align_up(o + field);
    L.traces = o; o = align_up(o + tr);
    if (forward_only) {
        L.total = o;
        return L;
    }
    L.resid = o; o = align_up(o + tr);
    L.grad = o; o = align_up(o + 2 * field);
    if (c->store_mode == GF_STORE_CHECKPOINT || c->store_mode == GF_STORE_RECONSTRUCT) {
        // checkpoints of the whole state every k steps, the state buffers of the segment
        // recomputation, and either a (k + 1)-slot Ez segment buffer or, when the adjoint
        // reconstructs the segment backwards, (k + 1) boundary-ring slots and a (K + 1)-slot
        // Ez buffer
        L.stC = o; o = align_up(o + gf::kNumFields * field);
        L.stD = o; o = align_up(o + gf::kNumFields * field);
        L.ckpt = o; o = align_up(o + gf::kNumFields * field * (size_t)num_checkpoints(c));
        if (c->store_mode == GF_STORE_CHECKPOINT) {
            L.seg = o; o = align_up(o + field * (size_t)(c->ckpt_k + 1));
        } else {
            L.seg = o; o = align_up(o + field * (size_t)(c->K + 1));
            L.ring = o;
            o = align_up(o + sizeof(float) * 3 * (size_t)c->nshots * c->ring_cells *
                                 (size_t)(c->ckpt_k + 1));
        }
    } else {
        L.hist = o; o = align_up(o + field * (size_t)c->g.nt);
    }
    L.total = o;
    return L;
}

int ensure_workspace(gf_ctx* c, bool forward_only) {
    const Layout L = layout_of(c, forward_only);
    if (c->ws && c->ws_bytes >= L.total) return GF_OK;
    if (c->ws && !c->ws_owned)
        return fail(c, GF_ENOMEM, "caller workspace has %zu bytes, %zu needed", c->ws_bytes, L.total);
    if (c->ws) {
        cudaFree(c->ws);
        c->ws = nullptr;
        c->ws_bytes = 0;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, L.total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, GF_ENOMEM, "cudaMalloc(%zu) failed: %s", L.total, cudaGetErrorString(e));
    }
    c->ws = (char*)p;
    c->ws_bytes = L.total;
    c->ws_owned = true;
    c->have_forward = false;
    ++c->generation;
    GF_CUDA(c, cudaMemset(c->ws + L.status, 0, sizeof(int)), "clear status");
    return GF_OK;
}

gf::TileParams base_params(const gf_ctx* c, const Layout& L) {
    gf::TileParams p{};
    p.nx = c->g.nx;
    p.ny = c->g.ny;
    p.pitch = c->pitch;
    p.npml = c->g.npml;
    p.nt = c->g.nt;
    p.nshots = c->nshots;
    p.nsrc = c->nsrc;
    p.nrec = c->nrec;
    p.Np = c->Np;
    p.ca = (const float*)(c->ws + L.coef);
    p.cb = p.ca + c->Np;
    p.ch = (float)(c->g.dt / kMu0);
    p.src_scale = (float)(1.0 / (c->g.dx * c->g.dy));
    p.geps = (float)(kEps0 / c->g.dt);
    p.rdx = (float)(1.0 / c->g.dx);
    p.rdy = (float)(1.0 / c->g.dy);
    p.px = c->px;
    p.py = c->py;
    p.src_xy = c->d_src_xy;
    p.status = (int*)(c->ws + L.status);
    p.tile_w = c->tile_w;
    p.tile_h = c->tile_h;
    p.tiles_x = (c->g.nx + c->tile_w - 1) / c->tile_w;
    p.ntiles = p.tiles_x * ((c->g.ny + c->tile_h - 1) / c->tile_h);
    p.tile_desc = c->d_tile_desc;
    p.tile_rec = c->d_tile_rec;
    p.cta_order = c->d_cta_order;
    p.ncta = p.ntiles * c->nshots;
    p.rec_max = c->tile_rec_max;
    p.kl = gf::left_halo(c->K);
    p.hist_stride = c->g.nt;
    p.hist_slot0 = 0;
    return p;
}

// Model check and the pitched Ca / Cb planes the tile kernels read.
int prepare_model(gf_ctx* c, const Layout& L, const float* eps_r, const float* sigma,
                  cudaStream_t st) {
    float* ca = (float*)(c->ws + L.coef);
    int* status = (int*)(c->ws + L.status);
    const int nx = c->g.nx, ny = c->g.ny, pitch = c->pitch;
    const float dt_eps0 = (float)(c->g.dt / kEps0);
    const long long Np = c->Np;
    GF_OP(c, st, GF_KERNEL_AUX, "prepare_model",
          gf::launch_prepare_model(eps_r, sigma, nx, ny, pitch, dt_eps0, ca, ca + Np, status, s_));
    return GF_OK;
}


// Tensor maps for a tile launch reading state buffer `st` (cached per buffer and variant).
const gf::TileMaps* tile_maps(gf_ctx* c, const gf::TileParams& p, const float* st) {
    const int wy = gf::max_tile_height(c->variant);
    for (auto& e : c->maps)
        if (e.st == st && e.coef == p.ca && e.wy == wy) return &e.m;
    auto& e = c->maps[c->maps_next];
    c->maps_next = (c->maps_next + 1) % 4;
    e.st = nullptr;
    if (!gf::make_tile_maps(&e.m, st, p.ca, c->pitch, c->g.ny, c->nshots, wy)) return nullptr;
    e.st = st;
    e.coef = p.ca;
    e.wy = wy;
    return &e.m;
}

// Forward steps [n_begin, n_end) in blocks of at most K steps, ping-ponging between buf[cur]
// and buf[cur ^ 1]; returns with cur pointing at the final state.  The persistent variant runs
// the whole range in one cooperative launch, the others launch once per block.
int forward_steps(gf_ctx* c, const Layout& L, gf::TileParams& p, float* const buf[2], int& cur,
                  int n_begin, int n_end, cudaStream_t st) {
    if (n_end <= n_begin) return GF_OK;
    if (c->variant == gf::kFlowVariant) {
        int* done = (int*)(c->ws + L.done);
        const size_t nb = sizeof(int) * (size_t)p.ntiles * c->nshots;
        GF_OP(c, st, -1, "clear counters", cudaMemsetAsync(done, 0, nb, s_));
        p.K = c->K;
        const gf::FlowInstance fi{p, gf::make_flow_args(buf[cur], buf[cur ^ 1], done, n_begin,
                                                        n_end - 1, c->K, c->wait_budget)};
        const int rc = flow_op(c, st, fi, false, "fwd_flow");
        if (rc) return rc;
        cur ^= ((n_end - n_begin + c->K - 1) / c->K) & 1;
        return GF_OK;
    }
    if (c->rec) return fail(c, GF_ESTATE, "only the persistent variant's passes can be merged");
    for (int n0 = n_begin; n0 < n_end; n0 += c->K) {
        p.n0 = n0;
        p.K = std::min(c->K, n_end - n0);
        p.st_in = buf[cur];
        p.st_out = buf[cur ^ 1];
        const gf::TileMaps* m = tile_maps(c, p, buf[cur]);
        if (!m) return fail(c, GF_ECUDA, "tensor maps of the tile kernels could not be encoded");
        GF_CUDA(c, launch(c, GF_KERNEL_FWD, st, [&] { return gf::launch_fwd_tile(p, *m, c->variant, st); }), "fwd_tile");
        cur ^= 1;
    }
    return GF_OK;
}

// Adjoint steps n_end - 1 down to n_begin (reverse), K steps at most per block.
int adjoint_steps(gf_ctx* c, const Layout& L, gf::TileParams& p, float* const buf[2], int& cur,
                  int n_begin, int n_end, cudaStream_t st) {
    if (n_end <= n_begin) return GF_OK;
    if (c->variant == gf::kFlowVariant) {
        int* done = (int*)(c->ws + L.done);
        const size_t nb = sizeof(int) * (size_t)p.ntiles * c->nshots;
        GF_OP(c, st, -1, "clear counters", cudaMemsetAsync(done, 0, nb, s_));
        p.K = c->K;
        const gf::FlowInstance fi{p, gf::make_flow_args(buf[cur], buf[cur ^ 1], done, n_begin,
                                                        n_end - 1, c->K, c->wait_budget)};
        const int rc = flow_op(c, st, fi, true, "adj_flow");
        if (rc) return rc;
        cur ^= ((n_end - n_begin + c->K - 1) / c->K) & 1;
        return GF_OK;
    }
    if (c->rec) return fail(c, GF_ESTATE, "only the persistent variant's passes can be merged");
    for (int n1 = n_end - 1; n1 >= n_begin; n1 -= c->K) {
        const int k = std::min(c->K, n1 - n_begin + 1);
        p.n0 = n1 - k + 1;
        p.K = k;
        p.st_in = buf[cur];
        p.st_out = buf[cur ^ 1];
        const gf::TileMaps* m = tile_maps(c, p, buf[cur]);
        if (!m) return fail(c, GF_ECUDA, "tensor maps of the tile kernels could not be encoded");
        GF_CUDA(c, launch(c, GF_KERNEL_ADJ, st, [&] { return gf::launch_adj_tile(p, *m, c->variant, st); }), "adj_tile");
        cur ^= 1;
    }
    return GF_OK;
}

// ---------------------------------------------------------------------------------------
// Lanes: the shots are split into contiguous groups that run their passes concurrently on
// the context's own streams (forked from and joined back into the caller's stream), so that
// one group's launches fill the SMs the other's last wave leaves idle and the groups' TMA
// prologues do not all hit HBM at once.  Every shot's arithmetic is the same in any lane.
// ---------------------------------------------------------------------------------------
struct LaneRange {
    int index, n, s0, s1;
    cudaStream_t st;
};

int lanes_in_use(const gf_ctx* c) {
    if (c->rec || c->one_lane || c->variant == gf::kFlowVariant ||
        c->store_mode == GF_STORE_RECONSTRUCT)
        return 1;
    return std::max(1, std::min(c->lanes, c->nshots));
}

// Destroy the lane streams and events (those that exist) and clear their handles.
void release_lanes(gf_ctx* c) {
    for (int l = 0; l < 4; ++l) {
        if (c->lane_st[l]) cudaStreamDestroy(c->lane_st[l]);
        if (c->lane_join[l]) cudaEventDestroy(c->lane_join[l]);
        c->lane_st[l] = nullptr;
        c->lane_join[l] = nullptr;
    }
    if (c->lane_fork) cudaEventDestroy(c->lane_fork);
    c->lane_fork = nullptr;
}

// Restrict the tile launches of p to the lane's shots.
void lane_params(const gf_ctx* c, gf::TileParams& p, const LaneRange& ln) {
    if (ln.n == 1) return;
    p.cta_order = c->d_cta_order + c->lane_off[ln.index];
    p.ncta = c->lane_cnt[ln.index];
}

// Run body(lane) for every lane; with more than one lane on the context's lane streams,
// ordered after everything enqueued on `st` so far and before everything enqueued on it next.
template <class F>
int run_lanes(gf_ctx* c, cudaStream_t st, F&& body) {
    const int n = lanes_in_use(c);
    if (n == 1) return body(LaneRange{0, 1, 0, c->nshots, st});
    if (!c->lane_fork) {
        cudaError_t e = cudaEventCreateWithFlags(&c->lane_fork, cudaEventDisableTiming);
        for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
            e = cudaStreamCreateWithFlags(&c->lane_st[l], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->lane_join[l], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) {
            // all or nothing: the next call creates the whole set again
            release_lanes(c);
            return cuda_fail(c, e, "lane streams");
        }
    }
    GF_CUDA(c, cudaEventRecord(c->lane_fork, st), "fork lanes");
    int rc = GF_OK;
    for (int l = 0; l < n; ++l) {
        // a lane whose fork fails runs nothing but is still joined, like one whose body fails
        cudaError_t e = cudaStreamWaitEvent(c->lane_st[l], c->lane_fork, 0);
        if (e != cudaSuccess && rc == GF_OK) rc = cuda_fail(c, e, "fork lanes");
        const int s0 = (int)((long long)c->nshots * l / n);
        const int s1 = (int)((long long)c->nshots * (l + 1) / n);
        if (rc == GF_OK) rc = body(LaneRange{l, n, s0, s1, c->lane_st[l]});
        // joined even after a failure, so that the caller's stream orders after the lane
        cudaEventRecord(c->lane_join[l], c->lane_st[l]);
        cudaStreamWaitEvent(st, c->lane_join[l], 0);
    }
    return rc;
}

// Slices of the lane's shots in [fields][nshots][Np] arrays: clear / copy them (one
// contiguous operation for all shots, else one per field).
int clear_shots(gf_ctx* c, cudaStream_t st, float* base, int fields, const LaneRange& ln,
                const char* what) {
    const size_t F = sizeof(float) * (size_t)c->nshots * c->Np;
    const size_t off = sizeof(float) * (size_t)ln.s0 * c->Np;
    const size_t w = sizeof(float) * (size_t)(ln.s1 - ln.s0) * c->Np;
    if (w == F) {
        const size_t n = F * (size_t)fields;
        GF_OP(c, st, -1, what, cudaMemsetAsync(base, 0, n, s_));
        return GF_OK;
    }
    for (int f = 0; f < fields; ++f) {
        char* p0 = (char*)base + F * (size_t)f + off;
        GF_OP(c, st, -1, what, cudaMemsetAsync(p0, 0, w, s_));
    }
    return GF_OK;
}
int copy_shots(gf_ctx* c, cudaStream_t st, void* dst, const void* src, int fields,
               const LaneRange& ln, const char* what) {
    const size_t F = sizeof(float) * (size_t)c->nshots * c->Np;
    const size_t off = sizeof(float) * (size_t)ln.s0 * c->Np;
    const size_t w = sizeof(float) * (size_t)(ln.s1 - ln.s0) * c->Np;
    if (w == F) {
        const size_t n = F * (size_t)fields;
        GF_OP(c, st, -1, what, cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToDevice, s_));
        return GF_OK;
    }
    for (int f = 0; f < fields; ++f) {
        char* d = (char*)dst + F * (size_t)f + off;
        const char* s = (const char*)src + F * (size_t)f + off;
        GF_OP(c, st, -1, what, cudaMemcpyAsync(d, s, w, cudaMemcpyDeviceToDevice, s_));
    }
    return GF_OK;
}

// The forward pass of one call: setup on the caller's stream, the time loop per lane, the
// illumination sum after the lanes.
struct Forward {
    Layout L;
    gf::TileParams p;
    bool ckpt = false;
    size_t state = 0;
    float* st_buf[2] = {nullptr, nullptr};
};

int forward_setup(gf_ctx* c, const float* eps_r, const float* sigma, const float* wavelet,
                  float* traces, float* illum, bool store, cudaStream_t st, Forward& f,
                  float* traces_h = nullptr) {
    if (!eps_r || !sigma || !wavelet) return fail(c, GF_EINVAL, "NULL model or wavelet pointer");
    int rc = ensure_workspace(c, !store);
    if (rc) return rc;
    f.L = layout_of(c, !store);
    const Layout& L = f.L;
    f.p = base_params(c, L);
    f.p.wavelet = wavelet;
    f.p.traces = traces ? traces : (float*)(c->ws + L.traces);
    f.p.traces_h = traces_h;
    f.ckpt = store && (c->store_mode == GF_STORE_CHECKPOINT ||
                       c->store_mode == GF_STORE_RECONSTRUCT);
    f.p.hist = store && !f.ckpt ? (float*)(c->ws + L.hist) : nullptr;
    f.p.illum = illum ? (float*)(c->ws + L.illum) : nullptr;
    f.state = gf::kNumFields * sizeof(float) * (size_t)c->nshots * (size_t)c->Np;
    f.st_buf[0] = (float*)(c->ws + L.stA);
    f.st_buf[1] = (float*)(c->ws + L.stB);
    {
        float* b0 = f.st_buf[0];
        const size_t state = f.state;
        GF_OP(c, st, -1, "clear state", cudaMemsetAsync(b0, 0, state, s_));
        if (illum) {
            float* ill = f.p.illum;
            GF_OP(c, st, -1, "clear illumination",
                  cudaMemsetAsync(ill, 0, state / gf::kNumFields, s_));
        }
    }
    rc = prepare_model(c, L, eps_r, sigma, st);
    if (rc) return rc;
    c->have_forward = store;
    c->last_wavelet = wavelet;
    return GF_OK;
}

int forward_lane(gf_ctx* c, const Forward& f, const LaneRange& ln) {
    gf::TileParams p = f.p;
    lane_params(c, p, ln);
    int cur = 0;
    if (f.ckpt) {
        // the state at every k-th step is saved before the segment that starts there
        for (int j = 0; j < num_checkpoints(c); ++j) {
            const int n_begin = j * c->ckpt_k, n_end = std::min(c->g.nt, n_begin + c->ckpt_k);
            char* dst = c->ws + f.L.ckpt + f.state * (size_t)j;
            int rc = copy_shots(c, ln.st, dst, f.st_buf[cur], gf::kNumFields, ln,
                                "save checkpoint");
            if (rc) return rc;
            rc = forward_steps(c, f.L, p, f.st_buf, cur, n_begin, n_end, ln.st);
            if (rc) return rc;
        }
        return GF_OK;
    }
    return forward_steps(c, f.L, p, f.st_buf, cur, 0, c->g.nt, ln.st);
}

int forward_finish(gf_ctx* c, const Forward& f, float* illum, cudaStream_t st) {
    if (illum) {
        const float* per = f.p.illum;
        int* status = f.p.status;
        const int ns = c->nshots, nx = c->g.nx, ny = c->g.ny, pitch = c->pitch;
        GF_OP(c, st, GF_KERNEL_AUX, "sum illum",
              gf::launch_sum_shots(per, ns, nx, ny, pitch, illum, status, s_));
    }
    return GF_OK;
}

int run_forward(gf_ctx* c, const float* eps_r, const float* sigma, const float* wavelet,
                float* traces, float* illum, bool store, cudaStream_t st,
                float* traces_h = nullptr) {
    Forward f;
    int rc = forward_setup(c, eps_r, sigma, wavelet, traces, illum, store, st, f, traces_h);
    if (rc) return rc;
    rc = run_lanes(c, st, [&](const LaneRange& ln) { return forward_lane(c, f, ln); });
    if (rc) return rc;
    return forward_finish(c, f, illum, st);
}

// The adjoint pass of one call: setup on the caller's stream (clears, coefficients), the
// time loop per lane (with its checkpoint restores and segment recomputations), the shot sums
// after the lanes.
struct Adjoint {
    Layout L;
    gf::TileParams p;
    size_t plane = 0, field = 0, state = 0;
    float* st_buf[2] = {nullptr, nullptr};
};

// clear: clear the adjoint state and the gradients here (else each lane clears its shots).
int adjoint_setup(gf_ctx* c, const float* eps_r, const float* sigma, const float* resid,
                  bool clear, bool prepare, cudaStream_t st, Adjoint& a) {
    a.L = layout_of(c, false);
    const Layout& L = a.L;
    a.p = base_params(c, L);
    a.p.resid = resid;
    a.p.grad = (float*)(c->ws + L.grad);
    a.plane = sizeof(float) * (size_t)c->Np;
    a.field = a.plane * (size_t)c->nshots;
    a.state = gf::kNumFields * a.field;
    a.st_buf[0] = (float*)(c->ws + L.stA);
    a.st_buf[1] = (float*)(c->ws + L.stB);
    if (clear) {
        float* b0 = a.st_buf[0];
        float* gr = a.p.grad;
        const size_t state = a.state, field = a.field;
        GF_OP(c, st, -1, "clear adjoint state", cudaMemsetAsync(b0, 0, state, s_));
        GF_OP(c, st, -1, "clear gradients", cudaMemsetAsync(gr, 0, 2 * field, s_));
    }
    if (prepare) {
        const int rc = prepare_model(c, L, eps_r, sigma, st);
        if (rc) return rc;
    }
    return GF_OK;
}

int adjoint_lane(gf_ctx* c, const Adjoint& a, const LaneRange& ln, bool clear) {
    const Layout& L = a.L;
    gf::TileParams p = a.p;
    lane_params(c, p, ln);
    const size_t plane = a.plane;
    const size_t state = a.state;
    float* const* st_buf = a.st_buf;
    const cudaStream_t st = ln.st;
    if (clear) {
        int rc = clear_shots(c, st, st_buf[0], gf::kNumFields, ln, "clear adjoint state");
        if (rc) return rc;
        rc = clear_shots(c, st, p.grad, 2, ln, "clear gradients");
        if (rc) return rc;
    }
    int cur = 0;
    if (c->store_mode == GF_STORE_CHECKPOINT) {
        // segments in reverse: restore the checkpoint, recompute the segment's Ez into the
        // segment buffer (slot 0 = Ez at the segment start), then run its adjoint steps
        float* seg = (float*)(c->ws + L.seg);
        float* const fw_buf[2] = {(float*)(c->ws + L.stC), (float*)(c->ws + L.stD)};
        gf::TileParams q = p;
        q.wavelet = c->last_wavelet;
        q.traces = (float*)(c->ws + L.traces);  // recomputed traces are not needed
        q.illum = nullptr;
        q.hist = seg;
        q.hist_stride = c->ckpt_k + 1;
        p.hist = seg;
        p.hist_stride = c->ckpt_k + 1;
        for (int j = num_checkpoints(c) - 1; j >= 0; --j) {
            const int n_begin = j * c->ckpt_k, n_end = std::min(c->g.nt, n_begin + c->ckpt_k);
            const char* ck = c->ws + L.ckpt + state * (size_t)j;
            int rc = copy_shots(c, st, fw_buf[0], ck, gf::kNumFields, ln, "restore checkpoint");
            if (rc) return rc;
            // Ez plane of every shot of the lane -> slot 0 of its segment
            const size_t seg_pitch = (size_t)(c->ckpt_k + 1) * plane;
            const size_t nsh = (size_t)(ln.s1 - ln.s0);
            float* seg0 = seg + (size_t)ln.s0 * (c->ckpt_k + 1) * (size_t)c->Np;
            const char* ck0 = ck + plane * (size_t)ln.s0;
            if (seg_pitch < ((size_t)1 << 30)) {
                GF_OP(c, st, -1, "segment start",
                      cudaMemcpy2DAsync(seg0, seg_pitch, ck0, plane, plane, nsh,
                                        cudaMemcpyDeviceToDevice, s_));
            } else {  // a pitch beyond what 2-D copies take: one copy per shot
                for (size_t i = 0; i < nsh; ++i) {
                    char* d = (char*)seg0 + seg_pitch * i;
                    const char* s = ck0 + plane * i;
                    GF_OP(c, st, -1, "segment start",
                          cudaMemcpyAsync(d, s, plane, cudaMemcpyDeviceToDevice, s_));
                }
            }
            q.hist_slot0 = n_begin - 1;
            p.hist_slot0 = n_begin - 1;
            int fcur = 0;
            rc = forward_steps(c, L, q, fw_buf, fcur, n_begin, n_end, st);
            if (rc) return rc;
            rc = adjoint_steps(c, L, p, st_buf, cur, n_begin, n_end, st);
            if (rc) return rc;
        }
    } else if (c->store_mode == GF_STORE_RECONSTRUCT) {
        // segments in reverse: restore the checkpoint, recompute the segment one step per
        // launch keeping the boundary ring of every step, then, block by block from the
        // segment's end, run the updates backwards into a (K + 1)-slot Ez buffer and run the
        // adjoint steps of that block
        float* small = (float*)(c->ws + L.seg);
        float* ring = (float*)(c->ws + L.ring);
        const size_t ring_slot = 3 * (size_t)c->nshots * c->ring_cells;
        float* const fw_buf[2] = {(float*)(c->ws + L.stC), (float*)(c->ws + L.stD)};
        gf::TileParams q = p;
        q.wavelet = c->last_wavelet;
        q.traces = (float*)(c->ws + L.traces);  // recomputed traces are not needed
        q.illum = nullptr;
        q.hist = nullptr;
        p.hist = small;
        p.hist_stride = c->K + 1;
        const size_t small_bytes = plane * (size_t)c->nshots * (c->K + 1);
        GF_OP(c, st, -1, "clear Ez buffer", cudaMemsetAsync(small, 0, small_bytes, s_));
        const int* map = c->d_ring_map;
        const int rc_cells = c->ring_cells, nsh = c->nshots, nx = c->g.nx, ny = c->g.ny;
        const int pitch = c->pitch, nsrc = c->nsrc, nt = c->g.nt;
        const long long Np = c->Np;
        const float rdx = p.rdx, rdy = p.rdy, ch = p.ch, sscale = p.src_scale;
        const float* ca = p.ca;
        const float* cb = p.cb;
        const int2* sxy = c->d_src_xy;
        const float* wav = c->last_wavelet;
        for (int j = num_checkpoints(c) - 1; j >= 0; --j) {
            const int n_begin = j * c->ckpt_k, n_end = std::min(c->g.nt, n_begin + c->ckpt_k);
            const char* ck = c->ws + L.ckpt + state * (size_t)j;
            float* fb0 = fw_buf[0];
            GF_OP(c, st, -1, "restore checkpoint",
                  cudaMemcpyAsync(fb0, ck, state, cudaMemcpyDeviceToDevice, s_));
            GF_OP(c, st, GF_KERNEL_AUX, "ring store",
                  gf::launch_ring_store(fb0, nsh, Np, pitch, nx, ny, map, rc_cells, ring, s_));
            int fcur = 0;
            for (int n = n_begin; n < n_end; ++n) {
                int rc = forward_steps(c, L, q, fw_buf, fcur, n, n + 1, st);
                if (rc) return rc;
                const float* sb = fw_buf[fcur];
                float* slot = ring + ring_slot * (size_t)(n + 1 - n_begin);
                GF_OP(c, st, GF_KERNEL_AUX, "ring store",
                      gf::launch_ring_store(sb, nsh, Np, pitch, nx, ny, map, rc_cells, slot, s_));
            }
            float* rec = fw_buf[fcur];  // the state at the segment's end, reversed in place
            for (int n1 = n_end - 1; n1 >= n_begin; n1 -= c->K) {
                const int k = std::min(c->K, n1 - n_begin + 1), n0 = n1 - k + 1;
                // slot m of the buffer holds Ez^{n0 + m}: the current Ez first, then the
                // reversed steps n1 .. n0
                const size_t sp = (size_t)(c->K + 1) * plane;
                float* top = small + (size_t)k * (size_t)Np;
                GF_OP(c, st, -1, "block end",
                      cudaMemcpy2DAsync(top, sp, rec, plane, plane, (size_t)nsh,
                                        cudaMemcpyDeviceToDevice, s_));
                for (int n = n1; n >= n0; --n) {
                    const float* slot = ring + ring_slot * (size_t)(n - n_begin);
                    float* hist = small + (size_t)(n - n0) * (size_t)Np;
                    const long long hs = (long long)(c->K + 1) * Np;
                    GF_OP(c, st, GF_KERNEL_AUX, "reverse step",
                          gf::launch_reverse_step(rec, nsh, Np, pitch, nx, ny, map, rc_cells,
                                                  slot, ca, cb, rdx, rdy, ch, sxy, nsrc, wav,
                                                  nt, n, sscale, hist, hs, s_));
                }
                p.hist_slot0 = n0 - 1;
                int rc = adjoint_steps(c, L, p, st_buf, cur, n0, n1 + 1, st);
                if (rc) return rc;
            }
        }
    } else {
        p.hist = (float*)(c->ws + L.hist);
        int rc = adjoint_steps(c, L, p, st_buf, cur, 0, c->g.nt, st);
        if (rc) return rc;
    }
    return GF_OK;
}

int adjoint_finish(gf_ctx* c, const Adjoint& a, float* g_eps_r, float* g_sigma,
                   cudaStream_t st) {
    {
        const float* gr = a.p.grad;
        int* status = a.p.status;
        const int ns = c->nshots, nx = c->g.nx, ny = c->g.ny, pitch = c->pitch;
        const size_t off = (size_t)c->nshots * c->Np;
        if (g_eps_r)
            GF_OP(c, st, GF_KERNEL_AUX, "sum g_eps_r",
                  gf::launch_sum_shots(gr, ns, nx, ny, pitch, g_eps_r, status, s_));
        if (g_sigma)
            GF_OP(c, st, GF_KERNEL_AUX, "sum g_sigma",
                  gf::launch_sum_shots(gr + off, ns, nx, ny, pitch, g_sigma, status, s_));
    }
    return GF_OK;
}

int run_adjoint(gf_ctx* c, const float* eps_r, const float* sigma, const float* resid,
                float* g_eps_r, float* g_sigma, cudaStream_t st) {
    Adjoint a;
    int rc = adjoint_setup(c, eps_r, sigma, resid, true, true, st, a);
    if (rc) return rc;
    rc = run_lanes(c, st, [&](const LaneRange& ln) { return adjoint_lane(c, a, ln, false); });
    if (rc) return rc;
    return adjoint_finish(c, a, g_eps_r, g_sigma, st);
}

// Per (shot, tile) descriptors of the tiling (tile_w x tile_h, K steps per block) for the
// tile kernels: the receivers of the window [tx tw - K, tx tw + tw + K) x [ty th - K,
// ty th + th + K) as entries {receiver index, (x - tx tw + 64) | (y - ty th + 64) << 16} in
// (row, receiver index) order, and the mask of the shot's sources in that window.  Uploaded;
// rebuilt whenever the tiling changes.
int build_tile_tables(gf_ctx* c, int tw, int th, int K) {
    const int nx = c->g.nx, ny = c->g.ny;
    const int ntx = (nx + tw - 1) / tw, nty = (ny + th - 1) / th, nt_ = ntx * nty;
    std::vector<std::vector<int>> lists((size_t)c->nshots * nt_);
    std::vector<int> masks(lists.size(), 0);
    auto windows = [&](int i, int j, auto&& visit) {
        const int tx0 = std::max(0, (i - K) / tw - 1), tx1 = std::min(ntx - 1, (i + K) / tw);
        const int ty0 = std::max(0, (j - K) / th - 1), ty1 = std::min(nty - 1, (j + K) / th);
        for (int ty = ty0; ty <= ty1; ++ty)
            for (int tx = tx0; tx <= tx1; ++tx)
                if (i >= tx * tw - K && i < tx * tw + tw + K && j >= ty * th - K &&
                    j < ty * th + th + K)
                    visit(ty * ntx + tx);
    };
    for (int s = 0; s < c->nshots; ++s) {
        for (int r = 0; r < c->nrec; ++r) {
            const int cell = c->h_rec[(size_t)s * c->nrec + r];
            windows(cell % nx, cell / nx, [&](int t) { lists[(size_t)s * nt_ + t].push_back(r); });
        }
        for (int k = 0; k < c->nsrc; ++k) {
            const int cell = c->h_src[(size_t)s * c->nsrc + k];
            windows(cell % nx, cell / nx, [&](int t) { masks[(size_t)s * nt_ + t] |= 1 << k; });
        }
    }
    std::vector<int4> desc(lists.size());
    std::vector<int2> ents;
    int longest = 0;
    for (size_t k = 0; k < lists.size(); ++k) {
        const int* cells = c->h_rec.data() + (k / nt_) * c->nrec;
        const int t = (int)(k % nt_), tx = t % ntx, ty = t / ntx;
        std::stable_sort(lists[k].begin(), lists[k].end(),
                         [&](int a, int b) { return cells[a] / nx < cells[b] / nx; });
        desc[k] = make_int4((int)ents.size(), (int)lists[k].size(), masks[k], 0);
        for (int r : lists[k]) {
            const int x = cells[r] % nx - tx * tw + 64, y = cells[r] / nx - ty * th + 64;
            ents.push_back(make_int2(r, x | y << 16));
        }
        longest = std::max(longest, (int)lists[k].size());
    }
    if (ents.empty()) ents.push_back(make_int2(0, 0));
    // launch order: receiver tiles, then tiles whose window (the tile and K cells around it)
    // touches a CPML strip, then the others; shot-major within a class
    std::vector<int> order;
    order.reserve(lists.size());
    const int np = c->g.npml;
    auto strip_tile = [&](int t) {
        const int tx = t % ntx, ty = t / ntx;
        const int xa = tx * tw - K, xb = tx * tw + tw + K, ya = ty * th - K, yb = ty * th + th + K;
        return np > 0 && (xa < np || xb - 1 >= nx - np - 1 || ya < np || yb - 1 >= ny - np - 1);
    };
    for (int cls = 0; cls < 3; ++cls)
        for (size_t k = 0; k < lists.size(); ++k) {
            const int t = (int)(k % nt_);
            const int kc = !lists[k].empty() ? 0 : strip_tile(t) ? 1 : 2;
            if (kc == cls) order.push_back((int)(k / nt_) << 16 | t);
        }
    // then each lane's shots [nshots l / n, nshots (l + 1) / n) in the same order
    const size_t all = order.size();
    const int nl = std::max(1, std::min(c->lanes, c->nshots));
    int lane_off[4] = {0}, lane_cnt[4] = {0};
    for (int l = 0; l < nl; ++l) {
        const int s0 = (int)((long long)c->nshots * l / nl);
        const int s1 = (int)((long long)c->nshots * (l + 1) / nl);
        lane_off[l] = (int)order.size();
        for (size_t k = 0; k < all; ++k) {
            const int shot = order[k] >> 16;
            if (shot >= s0 && shot < s1) order.push_back(order[k]);
        }
        lane_cnt[l] = (int)order.size() - lane_off[l];
    }
    int4* d_desc = nullptr;
    int2* d_ents = nullptr;
    int* d_order = nullptr;
    cudaError_t e = cudaMalloc(&d_desc, desc.size() * sizeof(int4));
    if (e == cudaSuccess) e = cudaMalloc(&d_ents, ents.size() * sizeof(int2));
    if (e == cudaSuccess) e = cudaMalloc(&d_order, order.size() * sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpy(d_desc, desc.data(), desc.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d_ents, ents.data(), ents.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d_order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_desc);
        cudaFree(d_ents);
        cudaFree(d_order);
        return cuda_fail(c, e, "tile tables");
    }
    cudaFree(c->d_tile_desc);
    cudaFree(c->d_tile_rec);
    cudaFree(c->d_cta_order);
    c->d_tile_desc = d_desc;
    c->d_tile_rec = d_ents;
    c->d_cta_order = d_order;
    c->tile_rec_max = longest;
    for (int l = 0; l < 4; ++l) {
        c->lane_off[l] = lane_off[l];
        c->lane_cnt[l] = lane_cnt[l];
    }
    return GF_OK;
}

// A tiling fits a variant's staged window: left halo left_halo(K) + tile_w + K columns within
// the window width, tile_h + 2K rows within its height; tile_w even (the window starts on an
// even column, so that column pairs are 8-byte aligned).  The persistent variant also needs
// tile_w a multiple of 4 (16-byte chunks), tiles at least K wide and high (a window only
// reaches the eight neighbouring tiles) and its shared memory within the limit.
int check_tiling(gf_ctx* c, int tw, int th, int K, int variant) {
    if (variant < 0 || variant >= gf::kNumVariants)
        return fail(c, GF_EINVAL, "kernel variant %d does not exist", variant);
    const bool flow = variant == gf::kFlowVariant;
    const int E = gf::max_tile_extent(), Eh = flow ? 64 : gf::max_tile_height(variant);
    const int kl = gf::left_halo(K);
    if (K < 1 || K > gf::kMaxK || tw < 4 || (tw & 3) || th < 1 || kl + tw + K > E ||
        th + 2 * K > Eh || (flow && (tw < K || th < K)))
        return fail(c, GF_EINVAL,
                    "tile %dx%d with %d steps per launch: need a tile width that is a multiple of "
                    "4 with %d + width + steps <= %d and height + 2*steps <= %d (steps <= %d)%s",
                    tw, th, K, kl, E, Eh, gf::kMaxK, flow ? ", width and height >= steps" : "");
    if ((long long)((c->g.nx + tw - 1) / tw) * ((c->g.ny + th - 1) / th) > 65535)
        return fail(c, GF_EINVAL, "tile %dx%d gives more than 65535 tiles", tw, th);
    const size_t need = flow ? gf::flow_smem_bytes(tw, th) : gf::tile_smem_bytes(variant, tw, th);
    if (need > c->smem_optin)
        return fail(c, GF_EINVAL, "tile kernels need %zu bytes of shared memory (> %zu)", need,
                    c->smem_optin);
    return GF_OK;
}

// Default tile of a variant for K steps per launch: the widest tile and the tallest one whose
// shared memory (the adjoint's wavefield ring grows with the tile) fits.
void default_tile(const gf_ctx* c, int variant, int K, int* tw, int* th) {
    const bool flow = variant == gf::kFlowVariant;
    *tw = (gf::max_tile_extent() - gf::left_halo(K) - K) & ~3;
    *th = (flow ? 64 : gf::max_tile_height(variant)) - 2 * K;
    auto need = [&] {
        return flow ? gf::flow_smem_bytes(*tw, *th) : gf::tile_smem_bytes(variant, *tw, *th);
    };
    while (*th > K && need() > c->smem_optin) --*th;
}

}  // namespace

extern "C" {

const char* gf_version(void) { return "gprfwi-gb300 0.1 (sm_103a)"; }

const char* gf_last_error(const gf_ctx* ctx) { return ctx ? ctx->err : g_create_err; }

int gf_create(gf_ctx** out, const gf_grid_desc* grid, const gf_acquisition* acq, int device) {
    if (!out) return GF_EINVAL;
    *out = nullptr;
    if (!grid || !acq || !acq->src_ij || !acq->rec_ij) {
        create_fail("gf_create: NULL grid, acquisition or geometry pointer");
        return GF_EINVAL;
    }
    const gf_grid_desc& g = *grid;
    if (g.nx < 3 || g.ny < 3 || g.nt < 1 || g.npml < 0 || 2 * g.npml > g.nx - 2 ||
        2 * g.npml > g.ny - 2 || !(g.dx > 0) || !(g.dy > 0) || !(g.dt > 0) || g.pml_order < 0 ||
        !(g.pml_kappa_max >= 1.0) || !(g.pml_alpha_max >= 0.0) || !(g.pml_eps_ref > 0.0)) {
        create_fail("gf_create: invalid grid description");
        return GF_EINVAL;
    }
    if ((long long)g.nx * g.ny > (1LL << 31) - 1) {
        create_fail("gf_create: grid too large");
        return GF_EINVAL;
    }
    // Eq. cfl with the vacuum speed of light (eps_r >= 1 everywhere).
    const double dtmax = 1.0 / (kC0 * sqrt(1.0 / (g.dx * g.dx) + 1.0 / (g.dy * g.dy)));
    if (g.dt > dtmax) {
        create_fail("gf_create: dt = %g s exceeds the CFL bound %g s", g.dt, dtmax);
        return GF_ECFL;
    }
    if (acq->nshots < 1 || acq->nshots > 65535 || acq->nsrc < 1 || acq->nsrc > gf::kMaxSrc ||
        acq->nrec < 1) {
        create_fail("gf_create: need 1 <= nshots <= 65535, 1 <= nsrc <= %d, nrec >= 1", gf::kMaxSrc);
        return GF_EINVAL;
    }
    auto inside = [&](const int32_t* ij) {
        return ij[0] >= 1 && ij[0] <= g.nx - 2 && ij[1] >= 1 && ij[1] <= g.ny - 2;
    };
    std::vector<int> src((size_t)acq->nshots * acq->nsrc), rec((size_t)acq->nshots * acq->nrec);
    for (size_t k = 0; k < src.size(); ++k) {
        if (!inside(acq->src_ij + 2 * k)) {
            create_fail("gf_create: source %zu outside 1..nx-2 x 1..ny-2", k);
            return GF_EINVAL;
        }
        src[k] = acq->src_ij[2 * k + 1] * g.nx + acq->src_ij[2 * k];
    }
    for (size_t k = 0; k < rec.size(); ++k) {
        if (!inside(acq->rec_ij + 2 * k)) {
            create_fail("gf_create: receiver %zu outside 1..nx-2 x 1..ny-2", k);
            return GF_EINVAL;
        }
        rec[k] = acq->rec_ij[2 * k + 1] * g.nx + acq->rec_ij[2 * k];
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        create_fail("gf_create: CUDA device %d not available (%d devices)", device, ndev);
        return GF_ECUDA;
    }
    DeviceGuard guard(device);
    gf_ctx* c = new gf_ctx();
    c->g = g;
    c->nshots = acq->nshots;
    c->nsrc = acq->nsrc;
    c->nrec = acq->nrec;
    c->device = device;
    c->N = (long long)g.nx * g.ny;
    c->pitch = gf::row_pitch(g.nx);
    c->Np = (long long)c->pitch * g.ny;
    c->h_rec = rec;
    c->h_src = src;
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    c->smem_optin = (size_t)optin;
    const int stride = std::max(g.nx, g.ny);
    std::vector<float> prof(12 * (size_t)stride, 0.f);
    axis_profiles(g, g.nx, g.dx, prof.data(), stride);
    axis_profiles(g, g.ny, g.dy, prof.data() + 6 * (size_t)stride, stride);
    cudaError_t e = cudaMalloc(&c->d_prof, prof.size() * sizeof(float));
    std::vector<int2> sxy(src.size());
    for (size_t k = 0; k < src.size(); ++k) sxy[k] = make_int2(src[k] % g.nx, src[k] / g.nx);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_src_xy, sxy.size() * sizeof(int2));
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_prof, prof.data(), prof.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_src_xy, sxy.data(), sxy.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = gf::configure_tile_kernels((size_t)optin);
    if (e == cudaSuccess) e = gf::configure_flow_kernels((size_t)optin);
    if (e != cudaSuccess) {
        cudaGetLastError();
        create_fail("gf_create: CUDA setup failed: %s", cudaGetErrorString(e));
        gf_destroy(c);
        return GF_ECUDA;
    }
    float* P = c->d_prof;
    const size_t S = stride;
    c->px = {P, P + S, P + 2 * S, P + 3 * S, P + 4 * S, P + 5 * S};
    c->py = {P + 6 * S, P + 7 * S, P + 8 * S, P + 9 * S, P + 10 * S, P + 11 * S};
    if (check_tiling(c, c->tile_w, c->tile_h, c->K, c->variant) != GF_OK ||
        build_tile_tables(c, c->tile_w, c->tile_h, c->K) != GF_OK) {
        create_fail("gf_create: %s", c->err);
        gf_destroy(c);
        return GF_EINVAL;
    }
    *out = c;
    return GF_OK;
}

void gf_destroy(gf_ctx* c) {
    if (!c) return;
    DeviceGuard guard(c->device);
    drop_profile(c);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    if (c->ws_owned && c->ws) cudaFree(c->ws);
    cudaFree(c->d_prof);
    cudaFree(c->d_src_xy);
    cudaFree(c->d_ring_map);
    cudaFree(c->d_rec_xy);
    cudaFree(c->te_buf);
    cudaFree(c->d_tile_desc);
    cudaFree(c->d_tile_rec);
    cudaFree(c->d_cta_order);
    release_lanes(c);
    delete c;
}

int gf_set_lanes(gf_ctx* c, int lanes) {
    if (!c) return GF_EINVAL;
    if (lanes < 1 || lanes > 4) return fail(c, GF_EINVAL, "lanes must be 1 to 4, not %d", lanes);
    DeviceGuard guard(c->device);
    const int old = c->lanes;
    c->lanes = lanes;
    const int rc = build_tile_tables(c, c->tile_w, c->tile_h, c->K);
    if (rc) {
        c->lanes = old;
        return rc;
    }
    ++c->generation;
    return GF_OK;
}

int gf_workspace_size(const gf_ctx* c, int store_mode, int forward_only, size_t* bytes) {
    if (!c || !bytes) return GF_EINVAL;
    if (store_mode != c->store_mode)
        return fail(const_cast<gf_ctx*>(c), GF_EINVAL,
                    "store mode %d is not the context's (%d): call gf_set_storage", store_mode,
                    c->store_mode);
    *bytes = layout_of(c, forward_only != 0).total;
    return GF_OK;
}

int gf_set_workspace(gf_ctx* c, void* ws, size_t bytes) {
    if (!c) return GF_EINVAL;
    ++c->generation;
    if (ws && ((uintptr_t)ws % kAlign)) return fail(c, GF_EINVAL, "workspace not 256-byte aligned");
    DeviceGuard guard(c->device);
    if (c->ws_owned && c->ws) cudaFree(c->ws);
    c->ws = (char*)ws;
    c->ws_bytes = ws ? bytes : 0;
    c->ws_owned = false;
    c->have_forward = false;
    if (ws) {
        if (bytes < layout_of(c, true).total)
            return fail(c, GF_ENOMEM, "workspace of %zu bytes is below the forward minimum", bytes);
        GF_CUDA(c, cudaMemset(c->ws, 0, sizeof(int)), "clear status");
    }
    return GF_OK;
}

int gf_set_tiling(gf_ctx* c, int tile_w, int tile_h, int K) {
    if (!c) return GF_EINVAL;
    ++c->generation;
    const int k = K > 0 ? K : c->K;
    int tw, th;
    default_tile(c, c->variant, k, &tw, &th);
    if (tile_w > 0) tw = tile_w;
    if (tile_h > 0) th = tile_h;
    int rc = check_tiling(c, tw, th, k, c->variant);
    if (rc) return rc;
    DeviceGuard guard(c->device);
    rc = build_tile_tables(c, tw, th, k);
    if (rc) return rc;
    c->tile_w = tw;
    c->tile_h = th;
    c->K = k;
    return GF_OK;
}

int gf_set_storage(gf_ctx* c, int mode, int k) {
    if (!c) return GF_EINVAL;
    ++c->generation;
    if (mode == GF_STORE_FULL) {
        k = 0;
    } else if ((mode != GF_STORE_CHECKPOINT && mode != GF_STORE_RECONSTRUCT) || k < 1 ||
               k > c->g.nt) {
        return fail(c, GF_EINVAL, "storage mode %d with k = %d is not valid", mode, k);
    }
    if (mode == GF_STORE_RECONSTRUCT && !c->d_ring_map) {
        // the ring: cells within npml + 2 of an edge (every CPML memory and every neighbour
        // of a CPML cell), numbered row by row
        const int nx = c->g.nx, ny = c->g.ny, W = c->g.npml + 2;
        std::vector<int> map((size_t)nx * ny);
        int cnt = 0;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                map[(size_t)j * nx + i] =
                    (i < W || i >= nx - W || j < W || j >= ny - W) ? cnt++ : -1;
        DeviceGuard guard(c->device);
        int* d = nullptr;
        cudaError_t e = cudaMalloc(&d, map.size() * sizeof(int));
        if (e == cudaSuccess)
            e = cudaMemcpy(d, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaFree(d);
            return cuda_fail(c, e, "ring map");
        }
        c->d_ring_map = d;
        c->ring_cells = cnt;
    }
    c->store_mode = mode;
    c->ckpt_k = k;
    c->have_forward = false;
    if (c->ws && c->ws_owned && c->ws_bytes < layout_of(c, false).total) {
        DeviceGuard guard(c->device);
        cudaFree(c->ws);
        c->ws = nullptr;
        c->ws_bytes = 0;
    }
    return GF_OK;
}

int gf_set_variant(gf_ctx* c, int variant) {
    if (!c) return GF_EINVAL;
    ++c->generation;
    if (variant < 0 || variant >= gf::kNumVariants)
        return fail(c, GF_EINVAL, "kernel variant %d does not exist", variant);
    // a tile taller than the variant's window is shrunk to the largest that fits
    const bool flow = variant == gf::kFlowVariant;
    int th = c->tile_h, tw = c->tile_w;
    const int Eh = flow ? 64 : gf::max_tile_height(variant);
    if (th + 2 * c->K > Eh) th = Eh - 2 * c->K;
    int rc = check_tiling(c, tw, th, c->K, variant);
    if (rc) return rc;
    DeviceGuard guard(c->device);
    rc = build_tile_tables(c, tw, th, c->K);
    if (rc) return rc;
    c->tile_w = tw;
    c->tile_h = th;
    c->variant = variant;
    return GF_OK;
}

int gf_get_tiling(const gf_ctx* c, int* tile_w, int* tile_h, int* K, int* variant) {
    if (!c || !tile_w || !tile_h || !K || !variant) return GF_EINVAL;
    *tile_w = c->tile_w;
    *tile_h = c->tile_h;
    *K = c->K;
    *variant = c->variant;
    return GF_OK;
}

int gf_forward_model(gf_ctx* c, const float* eps_r, const float* sigma, const float* wavelet,
                     float* traces, float* illum, void* stream) {
    if (!c) return GF_EINVAL;
    if (!traces) return fail(c, GF_EINVAL, "traces must not be NULL");
    DeviceGuard guard(c->device);
    return run_forward(c, eps_r, sigma, wavelet, traces, illum, false, (cudaStream_t)stream);
}

int gf_forward_model_fields(gf_ctx* c, const float* eps_r, const float* sigma,
                            const float* wavelet, float* traces, float* h_traces, float* illum,
                            void* stream) {
    if (!c) return GF_EINVAL;
    if (!traces) return fail(c, GF_EINVAL, "traces must not be NULL");
    DeviceGuard guard(c->device);
    return run_forward(c, eps_r, sigma, wavelet, traces, illum, false, (cudaStream_t)stream,
                       h_traces);
}

// TE model: argument checks, workspace, receiver table, parameters with the forward fields
// in the state buffers, field clears and the coefficient kernel.
static int te_setup(gf_ctx* c, const float* eps_r, const float* sigma, const float* wavelet,
                    int polarisation, cudaStream_t st, gf::TeParams& p, Layout& L) {
    if (!eps_r || !sigma || !wavelet) return fail(c, GF_EINVAL, "NULL model or wavelet pointer");
    if (polarisation != 0 && polarisation != 1)
        return fail(c, GF_EINVAL, "polarisation %d: 0 (x-directed) or 1 (y-directed)",
                    polarisation);
    const long long cells = (long long)c->nshots * (c->g.nx - 1) * (c->g.ny - 1);
    if ((cells + (long long)c->nshots * c->nrec) / 256 + 2 > 0x7fffffffLL)
        return fail(c, GF_EINVAL, "TE model: %lld cells exceed one launch", cells);
    if (c->rec) return fail(c, GF_ESTATE, "the TE model is not part of a batch schedule");
    int rc = ensure_workspace(c, true);
    if (rc) return rc;
    if (!c->d_rec_xy) {
        std::vector<int2> rxy(c->h_rec.size());
        for (size_t k = 0; k < rxy.size(); ++k)
            rxy[k] = make_int2(c->h_rec[k] % c->g.nx, c->h_rec[k] / c->g.nx);
        GF_CUDA(c, cudaMalloc(&c->d_rec_xy, rxy.size() * sizeof(int2)), "receiver table");
        GF_CUDA(c, cudaMemcpy(c->d_rec_xy, rxy.data(), rxy.size() * sizeof(int2),
                              cudaMemcpyHostToDevice), "receiver table");
    }
    // the TE fields reuse the forward workspace's state buffers: a stored TM forward is gone
    c->have_forward = false;
    L = layout_of(c, true);
    const long long F = (long long)c->nshots * c->Np;
    float* a = (float*)(c->ws + L.stA);
    float* b = (float*)(c->ws + L.stB);
    p = gf::TeParams{};
    p.nx = c->g.nx;
    p.ny = c->g.ny;
    p.pitch = c->pitch;
    p.nshots = c->nshots;
    p.nsrc = c->nsrc;
    p.nrec = c->nrec;
    p.nt = c->g.nt;
    p.pol = polarisation;
    p.Np = c->Np;
    p.F = F;
    p.ch = (float)(c->g.dt / kMu0);
    p.src_scale = (float)(1.0 / (c->g.dx * c->g.dy));
    p.geps = (float)(kEps0 / c->g.dt);
    p.px = c->px;
    p.py = c->py;
    p.ex = a;
    p.ey = a + F;
    p.hz0 = a + 2 * F;
    p.psi_hzx = a + 3 * F;
    p.psi_hzy = a + 4 * F;
    p.psi_exy = a + 5 * F;
    p.psi_eyx = a + 6 * F;
    p.hz1 = b;
    p.ca = (const float*)(c->ws + L.coef);
    p.cb = p.ca + c->Np;
    p.wavelet = wavelet;
    p.src_xy = c->d_src_xy;
    p.rec_xy = c->d_rec_xy;
    int* status = (int*)(c->ws + L.status);
    float* ca = (float*)(c->ws + L.coef);
    const int nx = c->g.nx, ny = c->g.ny, pitch = c->pitch;
    const float dt_eps0 = (float)(c->g.dt / kEps0);
    const long long Np = c->Np;
    GF_OP(c, st, -1, "clear TE fields", cudaMemsetAsync(a, 0, 7 * sizeof(float) * F, s_));
    GF_OP(c, st, -1, "clear TE fields", cudaMemsetAsync(b, 0, sizeof(float) * F, s_));
    GF_OP(c, st, GF_KERNEL_AUX, "TE coefficients",
          gf::launch_te_coef(eps_r, sigma, nx, ny, pitch, dt_eps0, ca, ca + Np, status, s_));
    return GF_OK;
}

// The context's TE buffer (E history, traces, residual), grown to `need` bytes.
static int te_buffer(gf_ctx* c, size_t need) {
    if (c->te_bytes >= need) return GF_OK;
    if (c->te_buf) cudaFree(c->te_buf);
    c->te_buf = nullptr;
    c->te_bytes = 0;
    if (cudaMalloc(&c->te_buf, need) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, GF_ENOMEM, "TE model: %zu bytes of history and trace buffers", need);
    }
    c->te_bytes = need;
    return GF_OK;
}

static int te_forward_steps(gf_ctx* c, const gf::TeParams& p, cudaStream_t st) {
    for (int n = 0; n < c->g.nt; ++n) {
        GF_OP(c, st, GF_KERNEL_FWD, "TE H update", gf::launch_te_h(p, n, s_));
        GF_OP(c, st, GF_KERNEL_FWD, "TE E update", gf::launch_te_e(p, n, s_));
    }
    return GF_OK;
}

int gf_forward_model_te(gf_ctx* c, const float* eps_r, const float* sigma,
                        const float* wavelet, int polarisation, float* traces, void* stream) {
    if (!c) return GF_EINVAL;
    if (!traces) return fail(c, GF_EINVAL, "traces must not be NULL");
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    gf::TeParams p;
    Layout L;
    int rc = te_setup(c, eps_r, sigma, wavelet, polarisation, st, p, L);
    if (rc) return rc;
    p.traces = traces;
    return te_forward_steps(c, p, st);
}

int gf_misfit_te(gf_ctx* c, const float* eps_r, const float* sigma, const float* wavelet,
                 int polarisation, const float* observed, double* misfit, void* stream) {
    if (!c) return GF_EINVAL;
    if (!observed || !misfit) return fail(c, GF_EINVAL, "NULL observed or misfit pointer");
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    gf::TeParams p;
    Layout L;
    int rc = te_setup(c, eps_r, sigma, wavelet, polarisation, st, p, L);
    if (rc) return rc;
    const size_t ntr = (size_t)c->nshots * c->g.nt * c->nrec;
    rc = te_buffer(c, sizeof(float) * ntr);
    if (rc) return rc;
    p.traces_p = c->te_buf;
    rc = te_forward_steps(c, p, st);
    if (rc) return rc;
    double* partial = (double*)(c->ws + L.partial);
    int* status = (int*)(c->ws + L.status);
    const float* tp = p.traces_p;
    GF_OP(c, st, GF_KERNEL_AUX, "TE misfit",
          gf::launch_residual_misfit(tp, observed, nullptr, (long long)ntr, partial,
                                     kMisfitBlocks, status, s_));
    GF_OP(c, st, GF_KERNEL_AUX, "TE misfit",
          gf::launch_finish_misfit(partial, kMisfitBlocks, misfit, s_));
    return GF_OK;
}

int gf_misfit_and_gradient_te(gf_ctx* c, const float* eps_r, const float* sigma,
                              const float* wavelet, int polarisation, const float* observed,
                              double* misfit, float* g_eps_r, float* g_sigma, float* traces,
                              void* stream) {
    if (!c) return GF_EINVAL;
    if (!observed || !misfit) return fail(c, GF_EINVAL, "NULL observed or misfit pointer");
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    gf::TeParams p;
    Layout L;
    int rc = te_setup(c, eps_r, sigma, wavelet, polarisation, st, p, L);
    if (rc) return rc;
    // the E history, the source component's traces and their residual, in a buffer of the
    // library's own (kept for the next call)
    const long long F = p.F;
    const size_t ntr = (size_t)c->nshots * c->g.nt * c->nrec;
    rc = te_buffer(c, sizeof(float) * ((size_t)c->g.nt * 2 * (size_t)F + 2 * ntr));
    if (rc) return rc;
    p.hist = c->te_buf;
    p.traces_p = c->te_buf + (size_t)c->g.nt * 2 * (size_t)F;
    float* resid = p.traces_p + ntr;
    p.traces = traces;
    rc = te_forward_steps(c, p, st);
    if (rc) return rc;
    double* partial = (double*)(c->ws + L.partial);
    int* status = (int*)(c->ws + L.status);
    const float* tp = p.traces_p;
    GF_OP(c, st, GF_KERNEL_AUX, "TE residual",
          gf::launch_residual_misfit(tp, observed, resid, (long long)ntr, partial, kMisfitBlocks,
                                     status, s_));
    GF_OP(c, st, GF_KERNEL_AUX, "TE misfit",
          gf::launch_finish_misfit(partial, kMisfitBlocks, misfit, s_));
    // adjoint: 7 planes in the first state buffer, 6 in the second
    float* a = (float*)(c->ws + L.stA);
    float* b = (float*)(c->ws + L.stB);
    p.aex = a;
    p.aey = a + F;
    p.ahz = a + 2 * F;
    p.a_exy = a + 3 * F;
    p.a_eyx = a + 4 * F;
    p.b_hzx = a + 5 * F;
    p.b_hzy = a + 6 * F;
    p.d_ex = b;
    p.d_ey = b + F;
    p.d_hy = b + 2 * F;
    p.d_hx = b + 3 * F;
    p.g_eps = b + 4 * F;
    p.g_sig = b + 5 * F;
    p.resid = resid;
    GF_OP(c, st, -1, "clear TE adjoint", cudaMemsetAsync(a, 0, 7 * sizeof(float) * F, s_));
    GF_OP(c, st, -1, "clear TE adjoint", cudaMemsetAsync(b, 0, 6 * sizeof(float) * F, s_));
    for (int n = c->g.nt - 1; n >= 0; --n)
        for (int part = 0; part < 4; ++part)
            GF_OP(c, st, GF_KERNEL_ADJ, "TE adjoint step",
                  gf::launch_te_adj_step(p, n, part, s_));
    const int ns = c->nshots, nx = c->g.nx, ny = c->g.ny, pitch = c->pitch;
    const float *ge = p.g_eps, *gs = p.g_sig;
    if (g_eps_r)
        GF_OP(c, st, GF_KERNEL_AUX, "TE gradient shot sum",
              gf::launch_sum_shots(ge, ns, nx, ny, pitch, g_eps_r, status, s_));
    if (g_sigma)
        GF_OP(c, st, GF_KERNEL_AUX, "TE gradient shot sum",
              gf::launch_sum_shots(gs, ns, nx, ny, pitch, g_sigma, status, s_));
    return GF_OK;
}

int gf_forward(gf_ctx* c, const float* eps_r, const float* sigma, const float* wavelet,
               float* traces, float* illum, int store_mode, void* stream) {
    if (!c) return GF_EINVAL;
    if (store_mode != c->store_mode)
        return fail(c, GF_EINVAL, "store mode %d is not the context's (%d): call gf_set_storage",
                    store_mode, c->store_mode);
    if (!traces) return fail(c, GF_EINVAL, "traces must not be NULL");
    DeviceGuard guard(c->device);
    return run_forward(c, eps_r, sigma, wavelet, traces, illum, true, (cudaStream_t)stream);
}

int gf_adjoint(gf_ctx* c, const float* eps_r, const float* sigma, const float* resid,
               float* g_eps_r, float* g_sigma, void* stream) {
    if (!c) return GF_EINVAL;
    if (!eps_r || !sigma || !resid) return fail(c, GF_EINVAL, "NULL model or residual pointer");
    if (!c->have_forward) return fail(c, GF_ESTATE, "gf_adjoint needs a stored gf_forward first");
    DeviceGuard guard(c->device);
    return run_adjoint(c, eps_r, sigma, resid, g_eps_r, g_sigma, (cudaStream_t)stream);
}

int gf_misfit_and_gradient(gf_ctx* c, const float* eps_r, const float* sigma,
                           const float* wavelet, const float* observed, double* misfit,
                           float* g_eps_r, float* g_sigma, float* traces, void* stream) {
    if (!c) return GF_EINVAL;
    if (!observed || !misfit) return fail(c, GF_EINVAL, "NULL observed or misfit pointer");
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    Forward f;
    int rc = forward_setup(c, eps_r, sigma, wavelet, traces, nullptr, true, st, f);
    if (rc) return rc;
    Adjoint a;
    const Layout& L = f.L;
    float* resid = (float*)(c->ws + L.resid);
    rc = adjoint_setup(c, eps_r, sigma, resid, false, false, st, a);
    if (rc) return rc;
    const float* tr = f.p.traces;
    double* partial = (double*)(c->ws + L.partial);
    int* status = (int*)(c->ws + L.status);
    const long long per_shot = (long long)c->g.nt * c->nrec;
    const int nl = lanes_in_use(c);
    // per lane: forward, residual of its traces, adjoint.  With one lane the residual kernel
    // also sums the misfit; with several, the misfit is summed after the lanes by the same
    // kernel over all traces, so that J does not depend on the lanes.
    rc = run_lanes(c, st, [&](const LaneRange& ln) {
        int r = forward_lane(c, f, ln);
        if (r) return r;
        const long long o = per_shot * ln.s0, cnt = per_shot * (ln.s1 - ln.s0);
        double* part = partial + (size_t)kMisfitBlocks * (nl == 1 ? 0 : 1 + ln.index);
        const float* trl = tr + o;
        const float* obl = observed + o;
        float* rsl = resid + o;
        GF_OP(c, ln.st, GF_KERNEL_AUX, "residual_misfit",
              gf::launch_residual_misfit(trl, obl, rsl, cnt, part, kMisfitBlocks, status, s_));
        return adjoint_lane(c, a, ln, true);
    });
    if (rc) return rc;
    if (nl > 1) {
        const long long count = per_shot * c->nshots;
        GF_OP(c, st, GF_KERNEL_AUX, "misfit",
              gf::launch_residual_misfit(tr, observed, nullptr, count, partial, kMisfitBlocks,
                                         status, s_));
    }
    GF_OP(c, st, GF_KERNEL_AUX, "finish_misfit",
          gf::launch_finish_misfit(partial, kMisfitBlocks, misfit, s_));
    return adjoint_finish(c, a, g_eps_r, g_sigma, st);
}

int gf_misfit(gf_ctx* c, const float* eps_r, const float* sigma, const float* wavelet,
              const float* observed, double* misfit, void* stream) {
    if (!c) return GF_EINVAL;
    if (!observed || !misfit) return fail(c, GF_EINVAL, "NULL observed or misfit pointer");
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = run_forward(c, eps_r, sigma, wavelet, nullptr, nullptr, false, st);
    if (rc) return rc;
    const Layout L = layout_of(c, true);
    const long long count = (long long)c->nshots * c->g.nt * c->nrec;
    GF_CUDA(c, launch(c, GF_KERNEL_AUX, st, [&] {
                return gf::launch_residual_misfit((float*)(c->ws + L.traces), observed, nullptr,
                                                  count, (double*)(c->ws + L.partial),
                                                  kMisfitBlocks, (int*)(c->ws + L.status), st);
            }),
            "residual_misfit");
    GF_CUDA(c, launch(c, GF_KERNEL_AUX, st, [&] {
                return gf::launch_finish_misfit((double*)(c->ws + L.partial), kMisfitBlocks, misfit, st);
            }),
            "finish_misfit");
    return GF_OK;
}

size_t gf_tv_scratch_bytes(int nx, int ny) {
    return nx > 0 && ny > 0 ? sizeof(float) * gf::tv_scratch_floats((long long)nx * ny) : 0;
}

int gf_tv_gradient(int nx, int ny, const float* model, float* grad, void* scratch, float lambda,
                   float mu, int iters, float weight, void* stream) {
    if (nx < 2 || ny < 2 || !model || !grad || !scratch || !(lambda >= 0.f) || !(mu > 0.f) ||
        iters < 0 || !(weight >= 0.f)) {
        create_fail("gf_tv_gradient: invalid argument");
        return GF_EINVAL;
    }
    cudaError_t e = gf::tv_gradient(nx, ny, model, grad, (float*)scratch, lambda, mu, iters, weight,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        create_fail("gf_tv_gradient: %s", cudaGetErrorString(e));
        return GF_ECUDA;
    }
    return GF_OK;
}

int gf_adam_update(long long n, float* x, const float* grad, float* m, float* v,
                   const float* mask, float gscale, float lr, float beta1, float beta2, float eps,
                   int t, float xmin, void* stream) {
    if (n < 0 || (n > 0 && (!x || !grad || !m || !v)) || t < 1 || !(lr >= 0.f) ||
        !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f) ||
        !isfinite(gscale)) {
        create_fail("gf_adam_update: invalid argument");
        return GF_EINVAL;
    }
    if (n == 0) return GF_OK;
    cudaError_t e = gf::adam_update(n, x, grad, m, v, mask, gscale, lr, beta1, beta2, eps, t,
                                    xmin, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        create_fail("gf_adam_update: %s", cudaGetErrorString(e));
        return GF_ECUDA;
    }
    return GF_OK;
}

int gf_status(gf_ctx* c, void* stream) {
    if (!c) return GF_EINVAL;
    if (!c->ws) return GF_OK;
    DeviceGuard guard(c->device);
    GF_CUDA(c, cudaStreamSynchronize((cudaStream_t)stream), "synchronize");
    int s = 0;
    GF_CUDA(c, cudaMemcpy(&s, c->ws, sizeof(int), cudaMemcpyDeviceToHost), "read status");
    GF_CUDA(c, cudaMemset(c->ws, 0, sizeof(int)), "clear status");
    if (s & gf::kStatusBadModel)
        return fail(c, GF_EINVAL, "model has eps_r < 1, sigma < 0 or non-finite values");
    if (s & gf::kStatusTimeout)
        return fail(c, GF_ETIMEOUT, "a dependency wait of the persistent kernels ran out");
    if (s & gf::kStatusNonFinite) return fail(c, GF_ENONFINITE, "non-finite traces or gradients");
    return GF_OK;
}

long long gf_kernel_launches(const gf_ctx* c) { return c ? c->launches : 0; }

int gf_set_wait_budget(gf_ctx* c, long long polls) {
    if (!c || polls < 0) return GF_EINVAL;
    if (polls != c->wait_budget) ++c->generation;  // recorded schedules carry the budget
    c->wait_budget = polls;
    return GF_OK;
}

int gf_profile(gf_ctx* c, int enable) {
    if (!c) return GF_EINVAL;
    DeviceGuard guard(c->device);
    drop_profile(c);
    c->profiling = enable != 0;
    return GF_OK;
}

int gf_profile_read(gf_ctx* c, int kind, double* ms_total, long long* launches) {
    if (!c || kind < 0 || kind > 2 || !ms_total || !launches) return GF_EINVAL;
    DeviceGuard guard(c->device);
    double total = 0.0;
    auto& v = c->prof_ev[kind];
    for (auto& pr : v) {
        GF_CUDA(c, cudaEventSynchronize(pr.second), "event synchronize");
        float ms = 0.f;
        GF_CUDA(c, cudaEventElapsedTime(&ms, pr.first, pr.second), "event elapsed");
        total += ms;
        c->ev_pool.push_back(pr.first);
        c->ev_pool.push_back(pr.second);
    }
    *ms_total = total;
    *launches = (long long)v.size();
    v.clear();
    return GF_OK;
}

int gf_profile_read_span(gf_ctx* c, int kind, double* ms_total, double* ms_span,
                         long long* launches) {
    if (!c || kind < 0 || kind > 3 || !ms_total || !ms_span || !launches) return GF_EINVAL;
    DeviceGuard guard(c->device);
    // kind 3: the forward and adjoint tile launches together, without clearing them
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>*> recs;
    for (int k = 0; k < 3; ++k)
        if (k == kind || (kind == 3 && k < 2))
            for (auto& pr : c->prof_ev[k]) recs.push_back(&pr);
    std::vector<std::pair<double, double>> iv;
    double total = 0.0;
    for (auto* pr : recs) {
        GF_CUDA(c, cudaEventSynchronize(pr->second), "event synchronize");
        float a = 0.f, b = 0.f;
        GF_CUDA(c, cudaEventElapsedTime(&a, recs[0]->first, pr->first), "event elapsed");
        GF_CUDA(c, cudaEventElapsedTime(&b, recs[0]->first, pr->second), "event elapsed");
        iv.emplace_back(a, b);
        total += b - a;
    }
    // the union of the launches' intervals: launches of concurrent lanes, and consecutive
    // launches under programmatic dependent launch, overlap
    std::sort(iv.begin(), iv.end());
    double span = 0.0, lo = 0.0, hi = -1e300;
    for (const auto& x : iv) {
        if (x.first > hi) {
            if (hi > lo) span += hi - lo;
            lo = x.first;
            hi = x.second;
        } else {
            hi = std::max(hi, x.second);
        }
    }
    if (hi > lo) span += hi - lo;
    *ms_total = total;
    *ms_span = span;
    *launches = (long long)recs.size();
    if (kind < 3) {
        auto& v = c->prof_ev[kind];
        for (auto& pr : v) {
            c->ev_pool.push_back(pr.first);
            c->ev_pool.push_back(pr.second);
        }
        v.clear();
    }
    return GF_OK;
}

int gf_ricker(float* out, int nt, double dt, double f0, double amp) {
    if (!out || nt < 0 || !(dt > 0) || !(f0 > 0)) return GF_EINVAL;
    const double t0 = sqrt(2.0) / f0, pi = 3.14159265358979323846;
    for (int n = 0; n < nt; ++n) {
        const double tau = n * dt - t0;
        const double z = pi * pi * f0 * f0 * tau * tau;
        out[n] = (float)(amp * (1.0 - 2.0 * z) * exp(-z));
    }
    return GF_OK;
}

}  // extern "C"

// Helpers shared with the allocation-free entry point (gf_noalloc.cu).
namespace gf {
void host_axis_profiles(const gf_grid_desc& g, int n, double d, float* out, int stride) {
    axis_profiles(g, n, d, out, stride);
}
void set_error_without_context(const char* msg) {
    snprintf(g_create_err, sizeof(g_create_err), "%s", msg);
}
}  // namespace gf

// ---------------------------------------------------------------------------------------
// Autotuner and uneven-instance batches
// ---------------------------------------------------------------------------------------
namespace {

// Forward launches over the first `nsteps` steps only (no storage): the autotuner's probe.
int forward_prefix(gf_ctx* c, const float* eps_r, const float* sigma, const float* wavelet,
                   int nsteps, cudaStream_t st) {
    int rc = ensure_workspace(c, true);
    if (rc) return rc;
    const Layout L = layout_of(c, true);
    gf::TileParams p = base_params(c, L);
    p.wavelet = wavelet;
    p.traces = (float*)(c->ws + L.traces);
    const size_t state = gf::kNumFields * sizeof(float) * (size_t)c->nshots * (size_t)c->Np;
    float* const st_buf[2] = {(float*)(c->ws + L.stA), (float*)(c->ws + L.stB)};
    GF_CUDA(c, cudaMemsetAsync(st_buf[0], 0, state, st), "clear state");
    rc = prepare_model(c, L, eps_r, sigma, st);
    if (rc) return rc;
    int cur = 0;
    return forward_steps(c, L, p, st_buf, cur, 0, std::min(nsteps, c->g.nt), st);
}

std::string tune_key(const gf_ctx* c) {
    cudaDeviceProp prop;
    std::string dev = cudaGetDeviceProperties(&prop, c->device) == cudaSuccess ? prop.name : "gpu";
    for (char& ch : dev)
        if (ch == ' ' || ch == '|') ch = '_';
    char buf[256];
    snprintf(buf, sizeof(buf), "%s nx=%d ny=%d npml=%d shots=%d src=%d rec=%d", dev.c_str(),
             c->g.nx, c->g.ny, c->g.npml, c->nshots, c->nsrc, c->nrec);
    return buf;
}

}  // namespace

struct gf_batch {
    // the persistent multi-instance schedule (modes 3 and 4): every context's recorded
    // operations, in its own order, with the persistent passes of several contexts merged
    struct Merged {
        std::vector<int> members;               // contexts whose pass this launch runs
        std::vector<gf::FlowInstance> h_inst;   // their passes (host copy)
        bool adjoint = false, hist = false;
        size_t inst_off = 0, items_off = 0;     // device copies in d_plan
        long long total = 0;                    // work items
    };
    struct Step {
        int inst, op, merged;                   // merged < 0: operation op of context inst
    };
    std::vector<OpList> lists;
    std::vector<Merged> merged;
    std::vector<Step> steps;
    char* d_plan = nullptr;
    std::vector<const void*> plan_key;
    std::vector<long long> plan_gens;
    cudaGraph_t graph4 = nullptr;
    cudaGraphExec_t exec4 = nullptr;
    std::vector<gf_ctx*> ctx;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaStream_t capture = nullptr;  // graphs are captured here (the caller's may be legacy)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> key;  // argument pointers the graph was captured with
    std::vector<long long> gens;
    int device = 0;
    char err[512] = {0};
};

namespace {

int batch_fail(gf_batch* b, int code, const char* what, const gf_ctx* c) {
    snprintf(b->err, sizeof(b->err), "%s%s%s", what, c ? ": " : "", c ? c->err : "");
    return code;
}

// Record every context's gradient operations, then merge: run each context's operations in
// its order up to its next persistent pass; one launch runs the pending passes of the same
// kind (forward with or without the wavefield store, or adjoint) of all contexts at once.
int build_plan(gf_batch* b, const float* const* eps_r, const float* const* sigma,
               const float* const* wavelet, const float* const* observed, double* misfit,
               float* const* g_eps_r, float* const* g_sigma) {
    const int n = (int)b->ctx.size();
    for (int i = 0; i < n; ++i)
        if (b->ctx[i]->variant != gf::kFlowVariant)
            return batch_fail(b, GF_EINVAL,
                              "modes 3 and 4 need every context on the persistent variant (3)",
                              nullptr);
    b->lists.assign(n, OpList());
    for (int i = 0; i < n; ++i) {
        gf_ctx* c = b->ctx[i];
        c->rec = &b->lists[i];
        const int rc = gf_misfit_and_gradient(c, eps_r[i], sigma[i], wavelet[i], observed[i],
                                              misfit + i, g_eps_r[i], g_sigma[i], nullptr,
                                              nullptr);
        c->rec = nullptr;
        if (rc) return batch_fail(b, rc, "recording an instance", c);
    }
    b->merged.clear();
    b->steps.clear();
    std::vector<size_t> pos(n, 0);
    size_t bytes = 0;
    auto align = [](size_t x) { return (x + 255) / 256 * 256; };
    for (;;) {
        int first = -1;
        for (int i = 0; i < n; ++i) {
            const auto& ops = b->lists[i].ops;
            while (pos[i] < ops.size() && !ops[pos[i]].flow) {
                b->steps.push_back({i, (int)pos[i], -1});
                ++pos[i];
            }
            if (pos[i] < ops.size() && first < 0) first = i;
        }
        if (first < 0) break;
        const StreamOp& f0 = b->lists[first].ops[pos[first]];
        gf_batch::Merged m;
        m.adjoint = f0.adjoint;
        m.hist = f0.inst.p.hist != nullptr;
        for (int i = 0; i < n; ++i) {
            const auto& ops = b->lists[i].ops;
            if (pos[i] >= ops.size()) continue;
            const StreamOp& op = ops[pos[i]];
            if (!op.flow || op.adjoint != m.adjoint || (op.inst.p.hist != nullptr) != m.hist)
                continue;
            m.members.push_back(i);
            m.h_inst.push_back(op.inst);
            m.total += (long long)op.inst.f.nblocks * op.inst.p.nshots * op.inst.p.ntiles;
            ++pos[i];
        }
        if (m.total > 0x7fffffffLL)
            return batch_fail(b, GF_EINVAL, "a merged pass has more than 2^31 work items",
                              nullptr);
        m.inst_off = align(bytes);
        bytes = m.inst_off + sizeof(gf::FlowInstance) * m.members.size();
        m.items_off = align(bytes);
        bytes = m.items_off + sizeof(int2) * (size_t)m.total;
        b->steps.push_back({-1, -1, (int)b->merged.size()});
        b->merged.push_back(std::move(m));
    }
    // the launches' instance arrays and work items (block-major over the instances), on the
    // device for as long as the plan is kept
    std::vector<char> h(bytes);
    for (const auto& m : b->merged) {
        memcpy(h.data() + m.inst_off, m.h_inst.data(), sizeof(gf::FlowInstance) * m.h_inst.size());
        int2* it = reinterpret_cast<int2*>(h.data() + m.items_off);
        int maxb = 0;
        for (const auto& fi : m.h_inst) maxb = std::max(maxb, fi.f.nblocks);
        long long k = 0;
        for (int blk = 0; blk < maxb; ++blk)
            for (size_t s = 0; s < m.h_inst.size(); ++s) {
                const gf::FlowInstance& fi = m.h_inst[s];
                if (blk >= fi.f.nblocks) continue;
                const int ipb = fi.p.nshots * fi.p.ntiles;
                for (int t = 0; t < ipb; ++t) it[k++] = make_int2((int)s, blk * ipb + t);
            }
    }
    cudaFree(b->d_plan);
    b->d_plan = nullptr;
    if (bytes) {
        cudaError_t e = cudaMalloc(&b->d_plan, bytes);
        if (e == cudaSuccess) e = cudaMemcpy(b->d_plan, h.data(), bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return batch_fail(b, GF_ENOMEM, "device copy of the merged schedule", nullptr);
        }
    }
    return GF_OK;
}

int run_plan(gf_batch* b, cudaStream_t st) {
    for (const auto& s : b->steps) {
        if (s.merged < 0) {
            gf_ctx* c = b->ctx[s.inst];
            const StreamOp& op = b->lists[s.inst].ops[s.op];
            const cudaError_t e = op.run(st);
            if (e != cudaSuccess) {
                cudaGetLastError();
                cuda_fail(c, e, op.what);
                return batch_fail(b, GF_ECUDA, "instance operation", c);
            }
            if (op.kind >= 0) ++c->launches;
            continue;
        }
        const gf_batch::Merged& m = b->merged[s.merged];
        const cudaError_t e = gf::launch_flow_multi(
            m.h_inst.data(), reinterpret_cast<const gf::FlowInstance*>(b->d_plan + m.inst_off),
            (int)m.members.size(), reinterpret_cast<const int2*>(b->d_plan + m.items_off),
            m.total, m.adjoint, m.hist, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            snprintf(b->err, sizeof(b->err), "merged persistent pass: %s", cudaGetErrorString(e));
            return GF_ECUDA;
        }
        ++b->ctx[m.members[0]]->launches;
    }
    return GF_OK;
}

}  // namespace

extern "C" {

int gf_autotune(gf_ctx* c, const float* eps_r, const float* sigma, const float* wavelet,
                const char* cache_path, int probe_steps, void* stream) {
    if (!c || !eps_r || !sigma || !wavelet) return GF_EINVAL;
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const std::string key = tune_key(c);
    if (cache_path) {
        if (FILE* f = fopen(cache_path, "r")) {
            char line[512];
            int best[4] = {0, 0, 0, -1};
            while (fgets(line, sizeof(line), f)) {
                const char* bar = strchr(line, '|');
                if (!bar) continue;
                if (std::string(line, bar - line) != key + " ") continue;
                int v[4];
                if (sscanf(bar + 1, "%d %d %d %d", &v[0], &v[1], &v[2], &v[3]) == 4)
                    std::copy(v, v + 4, best);
            }
            fclose(f);
            if (best[3] >= 0 && gf_set_variant(c, best[3]) == GF_OK &&
                gf_set_tiling(c, best[0], best[1], best[2]) == GF_OK)
                return GF_OK;
        }
    }
    struct Cand { int variant, K; };
    std::vector<Cand> cands;
    for (int v : {gf::kFlowVariant, 0})
        for (int K : {4, 5, 6, 7, 8, 10}) cands.push_back({v, K});
    for (int K : {3, 4, 5, 6}) cands.push_back({1, K});
    for (int K : {5, 7}) cands.push_back({2, K});
    const int steps = probe_steps > 0 ? probe_steps : 48;
    cudaEvent_t e0, e1;
    GF_CUDA(c, cudaEventCreate(&e0), "event");
    GF_CUDA(c, cudaEventCreate(&e1), "event");
    const bool prof = c->profiling;
    c->profiling = false;
    float best_ms = 1e30f;
    Cand best{c->variant, c->K};
    int rc = GF_OK;
    for (const Cand& k : cands) {
        if (gf_set_variant(c, k.variant) != GF_OK || gf_set_tiling(c, 0, 0, k.K) != GF_OK) continue;
        rc = forward_prefix(c, eps_r, sigma, wavelet, steps, st);  // warm-up
        if (rc == GF_ENOMEM) {  // a caller workspace too small for this candidate's tiling
            rc = GF_OK;
            continue;
        }
        if (rc) break;
        cudaEventRecord(e0, st);
        rc = forward_prefix(c, eps_r, sigma, wavelet, steps, st);
        if (rc) break;
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = k;
        }
    }
    c->profiling = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    rc = gf_set_variant(c, best.variant);
    if (rc == GF_OK) rc = gf_set_tiling(c, 0, 0, best.K);
    if (rc == GF_OK && cache_path) {
        if (FILE* f = fopen(cache_path, "a")) {
            fprintf(f, "%s | %d %d %d %d\n", key.c_str(), c->tile_w, c->tile_h, c->K, c->variant);
            fclose(f);
        }
    }
    return rc;
}

int gf_batch_create(gf_batch** out, gf_ctx* const* ctxs, int n) {
    if (!out) return GF_EINVAL;
    *out = nullptr;
    if (!ctxs || n < 1) return GF_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!ctxs[i] || ctxs[i]->device != ctxs[0]->device) return GF_EINVAL;
    DeviceGuard guard(ctxs[0]->device);
    gf_batch* b = new gf_batch();
    b->device = ctxs[0]->device;
    b->ctx.assign(ctxs, ctxs + n);
    b->streams.resize(n, nullptr);
    b->join.resize(n, nullptr);
    cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        gf_batch_destroy(b);
        return GF_ECUDA;
    }
    *out = b;
    return GF_OK;
}

void gf_batch_destroy(gf_batch* b) {
    if (!b) return;
    DeviceGuard guard(b->device);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->exec4) cudaGraphExecDestroy(b->exec4);
    if (b->graph4) cudaGraphDestroy(b->graph4);
    cudaFree(b->d_plan);
    for (auto s : b->streams)
        if (s) cudaStreamDestroy(s);
    for (auto e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->capture) cudaStreamDestroy(b->capture);
    delete b;
}

const char* gf_batch_last_error(const gf_batch* b) { return b ? b->err : "no batch"; }

int gf_batch_misfit_and_gradient(gf_batch* b, const float* const* eps_r, const float* const* sigma,
                                 const float* const* wavelet, const float* const* observed,
                                 double* misfit, float* const* g_eps_r, float* const* g_sigma,
                                 int mode, void* stream) {
    if (!b || !eps_r || !sigma || !wavelet || !observed || !misfit || !g_eps_r || !g_sigma ||
        mode < 0 || mode > 4)
        return GF_EINVAL;
    DeviceGuard guard(b->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int n = (int)b->ctx.size();
    auto fail_b = [&](int code, const char* what, gf_ctx* c) {
        snprintf(b->err, sizeof(b->err), "%s: %s", what, c ? c->err : "");
        return code;
    };
    // every context needs its full workspace before streams fork (and before a capture)
    for (int i = 0; i < n; ++i) {
        gf_ctx* c = b->ctx[i];
        if (c->profiling) return fail_b(GF_ESTATE, "disable profiling for batches", c);
        int rc = ensure_workspace(c, false);
        if (rc) return fail_b(rc, "workspace", c);
    }
    auto run_all = [&](bool concurrent, cudaStream_t st) -> int {
        if (concurrent) {
            if (cudaEventRecord(b->fork, st) != cudaSuccess) return GF_ECUDA;
        }
        for (int i = 0; i < n; ++i) {
            cudaStream_t si = concurrent ? b->streams[i] : st;
            if (concurrent && cudaStreamWaitEvent(si, b->fork, 0) != cudaSuccess) return GF_ECUDA;
            // instances that run beside each other need no shot lanes of their own
            b->ctx[i]->one_lane = concurrent;
            int rc = gf_misfit_and_gradient(b->ctx[i], eps_r[i], sigma[i], wavelet[i], observed[i],
                                            misfit + i, g_eps_r[i], g_sigma[i], nullptr, si);
            b->ctx[i]->one_lane = false;
            if (rc) return fail_b(rc, "instance", b->ctx[i]);
            if (concurrent) {
                if (cudaEventRecord(b->join[i], si) != cudaSuccess) return GF_ECUDA;
                if (cudaStreamWaitEvent(st, b->join[i], 0) != cudaSuccess) return GF_ECUDA;
            }
        }
        return GF_OK;
    };
    if (mode < 2) return run_all(mode == 1, st);
    std::vector<const void*> key;
    std::vector<long long> gens;
    for (int i = 0; i < n; ++i) {
        key.insert(key.end(), {eps_r[i], sigma[i], wavelet[i], observed[i], misfit + i,
                               g_eps_r[i], g_sigma[i]});
        gens.push_back(b->ctx[i]->generation);
    }
    if (mode >= 3) {
        const bool rebuilt = b->steps.empty() || key != b->plan_key || gens != b->plan_gens;
        if (rebuilt) {
            if (b->exec4) cudaGraphExecDestroy(b->exec4);
            if (b->graph4) cudaGraphDestroy(b->graph4);
            b->exec4 = nullptr;
            b->graph4 = nullptr;
            b->steps.clear();
            const int rc = build_plan(b, eps_r, sigma, wavelet, observed, misfit, g_eps_r,
                                      g_sigma);
            if (rc) {
                b->steps.clear();
                return rc;
            }
            b->plan_key = key;
            b->plan_gens = gens;
        }
        if (mode == 3) return run_plan(b, st);
        if (!b->exec4) {
            if (cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                cudaGetLastError();
                return fail_b(GF_ECUDA, "begin capture", nullptr);
            }
            const int rc = run_plan(b, b->capture);
            cudaGraph_t g = nullptr;
            const cudaError_t e = cudaStreamEndCapture(b->capture, &g);
            if (rc || e != cudaSuccess) {
                cudaGetLastError();
                if (g) cudaGraphDestroy(g);
                return rc ? rc : fail_b(GF_ECUDA, "end capture", nullptr);
            }
            if (cudaGraphInstantiate(&b->exec4, g, 0) != cudaSuccess) {
                cudaGetLastError();
                cudaGraphDestroy(g);
                return fail_b(GF_ECUDA, "instantiate graph", nullptr);
            }
            b->graph4 = g;
        }
        if (cudaGraphLaunch(b->exec4, st) != cudaSuccess) {
            cudaGetLastError();
            return fail_b(GF_ECUDA, "graph launch", nullptr);
        }
        return GF_OK;
    }
    // graph mode: capture the concurrent schedule once, replay while nothing changed
    if (!b->exec || key != b->key || gens != b->gens) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
        if (cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return fail_b(GF_ECUDA, "begin capture", nullptr);
        }
        const int rc = run_all(true, b->capture);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->capture, &g);
        if (rc || e != cudaSuccess) {
            cudaGetLastError();
            if (g) cudaGraphDestroy(g);
            return rc ? rc : fail_b(GF_ECUDA, "end capture", nullptr);
        }
        if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphDestroy(g);
            return fail_b(GF_ECUDA, "instantiate graph", nullptr);
        }
        b->graph = g;
        b->key = key;
        b->gens = gens;
        // the instances' launches now live in the graph; keep their counters meaningful
    }
    if (cudaGraphLaunch(b->exec, st) != cudaSuccess) {
        cudaGetLastError();
        return fail_b(GF_ECUDA, "graph launch", nullptr);
    }
    return GF_OK;
}

}  // extern "C"

