// gf_noalloc.cu -- forward modelling that allocates no memory: gf_forward_model_noalloc.
//
// Some callers cannot allocate device memory at the moment they need a forward model:
// programs whose device memory is owned and handed out by another runtime or a fixed pool
// (so a cudaMalloc from a library would bypass or break its accounting), services that run
// under a hard memory budget set by their host, and real-time loops that must never enter
// the allocator.  This entry point serves them.  It
// keeps everything the forward tile kernels need besides the caller's inputs and outputs --
// the two time-stepping state buffers, the update coefficients, the CPML profiles, the
// geometry and the per-tile receiver lists -- in one file-scope device array of fixed size (kScratchBytes), which every
// GPU that loads this library holds until the process exits.  It never calls cudaMalloc,
// cudaFree or any allocating routine.
//
// The array is shared by every call on a device and keeps the last call's contents; each call
// clears the state it needs to start from zero.  Calls whose work overlaps on the GPU (two
// streams, two threads) race on the array and must be serialised by the caller.
//
// The first call on each device looks up the array's device address with
// cudaGetSymbolAddress and sets the kernels' shared-memory limits, with that device current;
// make that first call before any stream capture begins.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/gprfwi.h"
#include "gf_internal.cuh"

namespace gf {
void host_axis_profiles(const gf_grid_desc& g, int n, double d, float* out, int stride);
void set_error_without_context(const char* msg);
}  // namespace gf

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB per device
constexpr int kMaxAxis = 16384;                     // cells per axis
constexpr int kMaxDevices = 64;
constexpr int kTileW = 48, kTileH = 48, kSteps = 8, kVariant = 0;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceSlot {
    unsigned char* ptr = nullptr;  // device address of g_scratch on this device
    bool ready = false;
};
DeviceSlot g_slots[kMaxDevices];
std::mutex g_mutex;
// host staging for the CPML profiles (static: no heap use)
float g_prof_host[12 * kMaxAxis];

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

int fail(int code, const char* fmt, ...) {
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    gf::set_error_without_context(msg);
    return code;
}

// Per (shot, tile) window [tx tw - K, tx tw + tw + K) x [ty th - K, ty th + th + K): the
// number of its receivers (desc.y) and the mask of its sources (desc.z); positions (x, y).
__global__ void count_windows(const int2* rec, const int2* src, int nshots, int nrec, int nsrc,
                              int tw, int th, int K, int tiles_x, int ntiles, int4* desc) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nshots * ntiles) return;
    const int s = k / ntiles, t = k % ntiles;
    const int x0 = (t % tiles_x) * tw - K, y0 = (t / tiles_x) * th - K;
    auto inside = [&](int2 c) {
        return c.x >= x0 && c.x < x0 + tw + 2 * K && c.y >= y0 && c.y < y0 + th + 2 * K;
    };
    int n = 0, mask = 0;
    for (int r = 0; r < nrec; ++r) n += inside(rec[s * nrec + r]);
    for (int q = 0; q < nsrc; ++q)
        if (inside(src[s * nsrc + q])) mask |= 1 << q;
    desc[k] = make_int4(0, n, mask, 0);
}

// desc[0..n).y -> exclusive offsets desc[k].x (one block, sequential chunks, fixed order).
__global__ void exclusive_offsets(int4* desc, int n) {
    __shared__ int part[1024];
    const int t = threadIdx.x, chunk = (n + blockDim.x - 1) / blockDim.x;
    const int a = min(t * chunk, n), b = min(a + chunk, n);
    int sum = 0;
    for (int k = a; k < b; ++k) sum += desc[k].y;
    part[t] = sum;
    __syncthreads();
    if (t == 0) {
        int run = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) {
            const int v = part[k];
            part[k] = run;
            run += v;
        }
    }
    __syncthreads();
    int run = part[t];
    for (int k = a; k < b; ++k) {
        desc[k].x = run;
        run += desc[k].y;
    }
}

// Receiver entries of each window {index, (x - tx tw + 64) | (y - ty th + 64) << 16}, sorted
// by row (insertion sort of the window's short list, stable: index order within a row).
__global__ void fill_windows(const int2* rec, int nshots, int nrec, int tw, int th, int K,
                             int tiles_x, int ntiles, const int4* desc, int2* ents) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nshots * ntiles) return;
    const int s = k / ntiles, t = k % ntiles;
    const int tx = t % tiles_x, ty = t / tiles_x;
    const int x0 = tx * tw - K, y0 = ty * th - K;
    int2* out = ents + desc[k].x;
    int n = 0;
    for (int r = 0; r < nrec; ++r) {
        const int2 c = rec[s * nrec + r];
        if (c.x >= x0 && c.x < x0 + tw + 2 * K && c.y >= y0 && c.y < y0 + th + 2 * K) {
            const int2 e = make_int2(r, (c.x - tx * tw + 64) | (c.y - ty * th + 64) << 16);
            int q = n++;
            while (q > 0 && (out[q - 1].y >> 16) > (e.y >> 16)) {
                out[q] = out[q - 1];
                --q;
            }
            out[q] = e;
        }
    }
}

// Launch order of the (shot, tile) pairs: shot << 16 | tile, in index order.
__global__ void fill_order(int nshots, int ntiles, int* order) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nshots * ntiles) order[k] = (k / ntiles) << 16 | (k % ntiles);
}

// Once per device, with that device current: the scratch address and kernel attributes.
int setup_device(int device, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceSlot& slot = g_slots[device];
    if (!slot.ready) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(GF_ECUDA, "gf_forward_model_noalloc: cudaGetSymbolAddress: %s",
                        cudaGetErrorString(e));
        }
        int optin = 0;
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
        if (e == cudaSuccess) e = gf::configure_tile_kernels((size_t)optin);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(GF_ECUDA, "gf_forward_model_noalloc: kernel set-up: %s",
                        cudaGetErrorString(e));
        }
        if (gf::tile_smem_bytes(kVariant, kTileW, kTileH) > (size_t)optin)
            return fail(GF_ECUDA, "gf_forward_model_noalloc: not enough shared memory per block");
        slot.ptr = (unsigned char*)p;
        slot.ready = true;
    }
    *out = slot.ptr;
    return GF_OK;
}

}  // namespace

extern "C" int gf_forward_model_noalloc(const gf_grid_desc* grid, const gf_acquisition* acq,
                                        int device, const float* eps_r, const float* sigma,
                                        const float* wavelet, float* traces, void* stream) {
    if (!grid || !acq || !acq->src_ij || !acq->rec_ij || !eps_r || !sigma || !wavelet || !traces)
        return fail(GF_EINVAL, "gf_forward_model_noalloc: NULL argument");
    const gf_grid_desc& g = *grid;
    if (g.nx < 3 || g.ny < 3 || g.nt < 1 || g.npml < 0 || 2 * g.npml > g.nx - 2 ||
        2 * g.npml > g.ny - 2 || !(g.dx > 0) || !(g.dy > 0) || !(g.dt > 0) || g.pml_order < 0 ||
        !(g.pml_kappa_max >= 1.0) || !(g.pml_alpha_max >= 0.0) || !(g.pml_eps_ref > 0.0))
        return fail(GF_EINVAL, "gf_forward_model_noalloc: invalid grid description");
    if (g.nx > kMaxAxis || g.ny > kMaxAxis)
        return fail(GF_EINVAL, "gf_forward_model_noalloc: grid %dx%d exceeds %d cells per axis",
                    g.nx, g.ny, kMaxAxis);
    const double dtmax = 1.0 / (299792458.0 * sqrt(1.0 / (g.dx * g.dx) + 1.0 / (g.dy * g.dy)));
    if (g.dt > dtmax)
        return fail(GF_ECFL, "gf_forward_model_noalloc: dt exceeds the CFL bound %g s", dtmax);
    if (acq->nshots < 1 || acq->nshots > 65535 || acq->nsrc < 1 || acq->nsrc > gf::kMaxSrc ||
        acq->nrec < 1)
        return fail(GF_EINVAL, "gf_forward_model_noalloc: need nshots >= 1, 1 <= nsrc <= %d, "
                    "nrec >= 1", gf::kMaxSrc);
    const long long nsrc_all = (long long)acq->nshots * acq->nsrc;
    const long long nrec_all = (long long)acq->nshots * acq->nrec;
    for (long long k = 0; k < nsrc_all + nrec_all; ++k) {
        const int32_t* ij = k < nsrc_all ? acq->src_ij + 2 * k : acq->rec_ij + 2 * (k - nsrc_all);
        if (ij[0] < 1 || ij[0] > g.nx - 2 || ij[1] < 1 || ij[1] > g.ny - 2)
            return fail(GF_EINVAL, "gf_forward_model_noalloc: source or receiver off 1..n-2");
    }
    cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &capture) != cudaSuccess) {
        cudaGetLastError();
        return fail(GF_ECUDA, "gf_forward_model_noalloc: cannot query the stream");
    }
    if (capture != cudaStreamCaptureStatusNone)
        return fail(GF_EINVAL, "gf_forward_model_noalloc: the stream is capturing (the call "
                    "synchronises it and cannot be captured)");

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev ||
        device >= kMaxDevices) {
        cudaGetLastError();
        return fail(GF_ECUDA, "gf_forward_model_noalloc: device %d not available", device);
    }

    // scratch layout (256-byte aligned regions)
    const int pitch = gf::row_pitch(g.nx);
    const long long Np = (long long)pitch * g.ny;
    const int S = g.nx > g.ny ? g.nx : g.ny;
    const int tiles_x = (g.nx + kTileW - 1) / kTileW;
    const int ntiles = tiles_x * ((g.ny + kTileH - 1) / kTileH);
    const long long nwin = (long long)acq->nshots * ntiles;
    // a receiver lies in at most 3 x 3 windows when tile >= 2K
    const long long max_entries = 9 * nrec_all;
    size_t o = 0;
    const size_t o_status = o; o = up256(o + sizeof(int));
    const size_t o_coef = o; o = up256(o + sizeof(float) * 2 * (size_t)Np);
    const size_t o_prof = o; o = up256(o + sizeof(float) * 12 * (size_t)S);
    const size_t o_srcij = o; o = up256(o + sizeof(int) * 2 * (size_t)nsrc_all);
    const size_t o_recij = o; o = up256(o + sizeof(int) * 2 * (size_t)nrec_all);
    const size_t o_desc = o; o = up256(o + sizeof(int4) * (size_t)nwin);
    const size_t o_ents = o; o = up256(o + sizeof(int2) * (size_t)max_entries);
    const size_t o_order = o; o = up256(o + sizeof(int) * (size_t)nwin);
    const size_t field = sizeof(float) * (size_t)acq->nshots * (size_t)Np;
    const size_t o_stA = o; o = up256(o + gf::kNumFields * field);
    const size_t o_stB = o; o = up256(o + gf::kNumFields * field);
    if (o > kScratchBytes)
        return fail(GF_ENOMEM, "gf_forward_model_noalloc: needs %zu bytes of scratch; the static "
                    "scratch holds %zu (nshots * nx * ny is about %zu at most)", o, kScratchBytes,
                    kScratchBytes / (2 * gf::kNumFields * sizeof(float)));

    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != device) cudaSetDevice(device);
    struct Restore {
        int prev, dev;
        ~Restore() {
            if (prev >= 0 && prev != dev) cudaSetDevice(prev);
        }
    } restore{prev, device};
    unsigned char* base = nullptr;
    int rc = setup_device(device, &base);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;

    // CPML profiles (host FP64 -> static host staging -> scratch)
    std::unique_lock<std::mutex> lock(g_mutex);
    gf::host_axis_profiles(g, g.nx, g.dx, g_prof_host, S);
    gf::host_axis_profiles(g, g.ny, g.dy, g_prof_host + 6 * (size_t)S, S);
    cudaError_t e = cudaMemcpyAsync(base + o_prof, g_prof_host, sizeof(float) * 12 * (size_t)S,
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + o_srcij, acq->src_ij, sizeof(int) * 2 * (size_t)nsrc_all,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + o_recij, acq->rec_ij, sizeof(int) * 2 * (size_t)nrec_all,
                            cudaMemcpyHostToDevice, st);
    // the host staging is reused by the next call, and the caller's geometry arrays are only
    // read during this call: every host read completes here
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    lock.unlock();
    // (i, j) pairs are (x, y) cells as they come
    const int2* src = (const int2*)(base + o_srcij);
    const int2* rec = (const int2*)(base + o_recij);
    int4* desc = (int4*)(base + o_desc);
    int2* ents = (int2*)(base + o_ents);
    if (e == cudaSuccess) {
        const int wb = (int)((nwin + 255) / 256);
        count_windows<<<wb, 256, 0, st>>>(rec, src, acq->nshots, acq->nrec, acq->nsrc, kTileW,
                                          kTileH, kSteps, tiles_x, ntiles, desc);
        exclusive_offsets<<<1, 1024, 0, st>>>(desc, (int)nwin);
        fill_windows<<<wb, 256, 0, st>>>(rec, acq->nshots, acq->nrec, kTileW, kTileH, kSteps,
                                         tiles_x, ntiles, desc, ents);
        fill_order<<<wb, 256, 0, st>>>(acq->nshots, ntiles, (int*)(base + o_order));
        e = cudaGetLastError();
    }
    // the state starts from zero on every call (the array keeps the previous call's contents);
    // the update coefficients of this call's model fill the pitched planes
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_stA, 0, gf::kNumFields * field, st);
    float* ca = (float*)(base + o_coef);
    if (e == cudaSuccess)
        e = gf::launch_prepare_model(eps_r, sigma, g.nx, g.ny, pitch,
                                     (float)(g.dt / 8.8541878128e-12), ca, ca + Np,
                                     (int*)(base + o_status), st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(GF_ECUDA, "gf_forward_model_noalloc: %s", cudaGetErrorString(e));
    }

    gf::TileParams p{};
    p.nx = g.nx;
    p.ny = g.ny;
    p.pitch = pitch;
    p.npml = g.npml;
    p.nt = g.nt;
    p.nshots = acq->nshots;
    p.nsrc = acq->nsrc;
    p.nrec = acq->nrec;
    p.Np = Np;
    p.ca = ca;
    p.cb = ca + Np;
    p.ch = (float)(g.dt / 1.25663706212e-6);
    p.src_scale = (float)(1.0 / (g.dx * g.dy));
    p.geps = (float)(8.8541878128e-12 / g.dt);
    p.rdx = (float)(1.0 / g.dx);
    p.rdy = (float)(1.0 / g.dy);
    float* P = (float*)(base + o_prof);
    p.px = {P, P + S, P + 2 * S, P + 3 * S, P + 4 * S, P + 5 * S};
    p.py = {P + 6 * S, P + 7 * S, P + 8 * S, P + 9 * S, P + 10 * S, P + 11 * S};
    p.wavelet = wavelet;
    p.src_xy = src;
    p.traces = traces;
    p.hist = nullptr;
    p.illum = nullptr;
    p.tile_w = kTileW;
    p.tile_h = kTileH;
    p.tiles_x = tiles_x;
    p.ntiles = ntiles;
    p.tile_desc = desc;
    p.tile_rec = ents;
    p.cta_order = (const int*)(base + o_order);
    p.rec_max = acq->nrec;  // no window holds more than a shot's receivers
    p.status = (int*)(base + o_status);
    p.kl = gf::left_halo(kSteps);
    float* buf[2] = {(float*)(base + o_stA), (float*)(base + o_stB)};
    int cur = 0;
    for (int n0 = 0; n0 < g.nt; n0 += kSteps) {
        p.n0 = n0;
        p.K = g.nt - n0 < kSteps ? g.nt - n0 : kSteps;
        p.st_in = buf[cur];
        p.st_out = buf[cur ^ 1];
        gf::TileMaps maps;
        if (!gf::make_tile_maps(&maps, buf[cur], ca, pitch, g.ny, acq->nshots,
                                gf::max_tile_height(kVariant)))
            return fail(GF_ECUDA, "gf_forward_model_noalloc: tensor maps could not be encoded");
        e = gf::launch_fwd_tile(p, maps, kVariant, st);
        if (e != cudaSuccess)
            return fail(GF_ECUDA, "gf_forward_model_noalloc: tile launch: %s", cudaGetErrorString(e));
        cur ^= 1;
    }
    return GF_OK;
}
