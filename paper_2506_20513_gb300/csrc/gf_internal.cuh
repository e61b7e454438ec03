// gf_internal.cuh -- types shared by the host runtime and the sm_103a kernels of libgprfwi.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace gf {

constexpr int kMaxSrc = 8;        // sources per shot
constexpr int kNumFields = 7;     // Ez, Hx, Hy, psiEx, psiEy, psiHx, psiHy (or their adjoints)
constexpr int kMaxK = 31;         // time steps per tile launch
// Shared-memory words in which a tile kernel stages its window's receiver list: positions
// and receiver indices (2 words per entry) and, in the adjoint, the residual samples of the
// launch (K more words per entry).  Longer lists are read from global memory.
constexpr int kRecStage = 2048;

// Device-status bits (OR-ed into the workspace status word by kernels).
constexpr int kStatusBadModel = 1;   // eps_r < 1, sigma < 0 or non-finite model value
constexpr int kStatusNonFinite = 2;  // non-finite trace or gradient
constexpr int kStatusTimeout = 4;    // a persistent kernel's dependency wait ran out

// Row pitch (floats) of the library's internal [ny][pitch] planes (state, wavefield store,
// per-shot gradients and illumination, update coefficients): nx rounded up to a multiple of
// 4, so that every row starts 16-byte aligned and column pairs (2i, 2i + 1) are 8-byte
// aligned.  Caller arrays (model, gradients, illumination) stay [ny][nx].
inline int row_pitch(int nx) { return (nx + 3) & ~3; }

// Left halo of a tile launch with K steps: K rounded up to a multiple of 4, so that the staged
// window starts on a 16-byte boundary (tile widths are multiples of 4): its rows are loaded by
// TMA boxes or 16-byte copies.
inline int left_halo(int K) { return (K + 3) & ~3; }

// CPML profiles of one axis (FP32, uploaded once per context).  For a node at index i:
//   a = 1 / (kappa * d), b = exp(-(sigma/kappa + alpha) dt / eps0),
//   c = sigma (b - 1) / (sigma kappa + kappa^2 alpha) / d  (0 outside the CPML),
// "E" arrays at integer nodes, "H" arrays at the half node i + 1/2.
struct AxisProfile {
    const float *aE, *bE, *cE, *aH, *bH, *cH;
};

// Everything one tile launch needs.  State arrays are packed as [kNumFields][nshots][Np] with
// Np = pitch * ny (row gy of a plane at gy * pitch).
struct TileParams {
    int nx, ny, pitch, npml, nt, nshots, nsrc, nrec;
    long long Np;        // pitch * ny
    float ch;            // dt / mu0
    float src_scale;     // 1 / (dx dy)
    float geps;          // eps0 / dt (zero-lag eps_r gradient scale)
    float rdx, rdy;      // 1 / dx, 1 / dy
    AxisProfile px, py;
    const float* ca;     // update coefficients Ca, Cb of the model, [Np] each (0 on the PEC
    const float* cb;     // ring, in perfect conductors and in the row padding)
    const float* wavelet;   // [nshots][nsrc][nt]
    const int2* src_xy;     // [nshots][nsrc] source cells (x, y)
    const float* st_in;     // time-stepping state at the start of the launch
    float* st_out;          // state at the end of the launch (other ping-pong buffer)
    float* hist;            // wavefield store, NULL = not stored: Ez^{n+1} of shot s at
                            // hist + (s * hist_stride + n - hist_slot0) * Np
    int hist_stride;        // slots per shot (nt for the full store, k + 1 for a segment)
    int hist_slot0;         // step whose Ez^{n+1} is slot 0 (0, or the segment start - 1)
    float* traces;          // forward: [nshots][nt][nrec] output
    float* traces_h;        // forward: [nshots][nt][nrec][2] Hx, Hy output (NULL = skip)
    const float* resid;     // adjoint: [nshots][nt][nrec] trace cotangent
    float* illum;           // forward: [nshots][Np] accumulated (NULL = skip)
    float* grad;            // adjoint: [2][nshots][Np] accumulated
    int n0, K;              // first time step of the launch, steps in the launch
    int tile_w, tile_h;     // interior tile size (tile_w even)
    int kl;                 // left halo of the staged window (left_halo(K)); K elsewhere
    int tiles_x, ntiles;
    // Per (shot, tile) descriptor {first entry, entries, source mask, 0} of the window
    // [tx*tile_w - K, tx*tile_w + tile_w + K) x [ty*tile_h - K, ty*tile_h + tile_h + K) (K of
    // the context): its receiver list tile_rec[first .. first + entries) sorted by row, each
    // entry {receiver index, (x - tx*tile_w + 64) | (y - ty*tile_h + 64) << 16}, and bit k set
    // when source k of the shot lies in the window.  Host-built per tiling.
    const int4* tile_desc;  // [nshots][ntiles]
    const int2* tile_rec;
    // Launch order of the (shot, tile) pairs, shot << 16 | tile: tiles with receivers first,
    // then tiles touching a CPML strip, then the rest (the slow ones start early, the last wave
    // is short)
    const int* cta_order;   // [nshots * ntiles], or one lane's part of it
    int ncta;               // CTAs of a per-launch tile kernel: entries of cta_order (0: all)
    int rec_max;            // longest list (decides shared-memory staging)
    int* status;
};

// Tensor maps of one tile launch (TMA loads of the staged window, fp32, box 64 x WY, zero
// outside the arrays): the state buffer the launch reads ([kNumFields * nshots][ny][pitch],
// plane z = field * nshots + shot) and the update coefficients ([2][ny][pitch]: Ca, Cb).
struct TileMaps {
    CUtensorMap st;
    CUtensorMap coef;
};

// Encode a TileMaps for state buffer `st` and coefficient planes `coef` (window height wy);
// false when the driver's encoder is unavailable or rejects the layout.
bool make_tile_maps(TileMaps* m, const float* st, const float* coef, int pitch, int ny,
                    int nshots, int wy);

// Host-side launchers.  Kernel variants: 0 = one launch per time block, 4 rows per thread,
// 512 threads, 64 x 64 window; 1 = the same with 256 threads and a 64 x 32 window (two CTAs
// per SM); 2 = 8 rows per thread, 256 threads, 64 x 64; 3 = the persistent dataflow kernels
// (one cooperative launch per pass, variant 0's window).
constexpr int kFlowVariant = 3;
constexpr int kNumVariants = 4;
cudaError_t launch_fwd_tile(const TileParams& p, const TileMaps& m, int variant, cudaStream_t st);
cudaError_t launch_adj_tile(const TileParams& p, const TileMaps& m, int variant, cudaStream_t st);
int max_tile_extent();              // staged window width
int max_tile_height(int variant);   // staged window height of a per-launch variant (0-2)
size_t tile_smem_bytes(int variant, int tile_w, int tile_h);  // per-launch variants (0-2)
cudaError_t configure_tile_kernels(size_t optin);
// Persistent dataflow passes.  One pass of one instance (a context's shots on its grid):
// forward steps [n_first, n_last] in blocks of kb steps, or the adjoint steps n_last down to
// n_first, ping-ponging from buf0 (the pass ends in buf[nblocks % 2]); done: nshots * ntiles
// zeroed ints (completed blocks per (shot, tile)); budget: polls of one dependency wait.
struct FlowArgs {
    float* buf0;
    float* buf1;
    int* done;
    int n_first, n_last;
    int kb;
    int nblocks;
    long long budget;
};
struct FlowInstance {
    TileParams p;
    FlowArgs f;
};
FlowArgs make_flow_args(float* buf0, float* buf1, int* done, int n_first, int n_last, int kb,
                        long long budget);
// One cooperative launch for one instance's pass.  The tiling needs tile_w a multiple of 4,
// kl a multiple of 4 and tile_w, tile_h >= kb.
cudaError_t launch_flow_pass(const FlowInstance& inst, bool adjoint, cudaStream_t st);
// One cooperative launch for the passes of several instances (host array h_inst, its device
// copy d_inst): work item k of the launch is items[k] = {instance, item of that instance},
// block-major over all instances (an item may only depend on earlier items).  All instances
// store the forward wavefield (hist) or none does; ring = largest tile_w * tile_h (adjoint).
cudaError_t launch_flow_multi(const FlowInstance* h_inst, const FlowInstance* d_inst, int n,
                              const int2* d_items, long long total, bool adjoint, bool hist,
                              cudaStream_t st);
size_t flow_smem_bytes(int tile_w, int tile_h);
cudaError_t configure_flow_kernels(size_t optin);

// Model check (eps_r >= 1, sigma >= 0, finite) and the update coefficients Ca, Cb of every
// cell of the pitched planes.
cudaError_t launch_prepare_model(const float* eps_r, const float* sigma, int nx, int ny,
                                 int pitch, float dt_eps0, float* ca, float* cb, int* status,
                                 cudaStream_t st);
cudaError_t launch_residual_misfit(const float* traces, const float* observed, float* resid,
                                   long long count, double* partial, int nblocks, int* status,
                                   cudaStream_t st);
cudaError_t launch_finish_misfit(const double* partial, int nblocks, double* misfit,
                                 cudaStream_t st);
size_t tv_scratch_floats(long long n);
cudaError_t adam_update(long long n, float* x, const float* g, float* m, float* v,
                        const float* mask, float gscale, float lr, float b1, float b2, float eps,
                        int t, float xmin, cudaStream_t st);
cudaError_t tv_gradient(int nx, int ny, const float* X, float* G, float* scratch, float lambda,
                        float mu, int iters, float weight, cudaStream_t st);
// TE-mode forward model (gf_te.cu): fields of every shot as [nshots][ny][pitch] planes,
// CPML memory planes touched only inside the strips, Hz in two buffers (step n reads hz0 if
// n is even, else hz1, and writes the other).
struct TeParams {
    int nx, ny, pitch, nshots, nsrc, nrec, nt, pol;  // pol: 0 = x-directed source, 1 = y
    long long Np;        // pitch * ny
    float ch;            // dt / mu0
    float src_scale;     // 1 / (dx dy)
    AxisProfile px, py;
    float *ex, *ey, *hz0, *hz1, *psi_hzx, *psi_hzy, *psi_exy, *psi_eyx;
    const float* ca;     // [ny][pitch] Ca, Cb without the TM ring rule
    const float* cb;
    const float* wavelet;  // [nshots][nsrc][nt]
    const int2* src_xy;    // [nshots][nsrc]
    const int2* rec_xy;    // [nshots][nrec]
    float* traces;         // [nshots][nt][nrec][3]: Ex^n, Ey^n, Hz^{n-1/2} (NULL = skip)
    long long F;           // nshots * Np: one field plane of every shot
    float* traces_p;       // [nshots][nt][nrec] the source component's traces (NULL = skip)
    float* hist;           // [nt][2][nshots][Np]: Ex^{n+1}, Ey^{n+1} of step n (NULL = none)
    // adjoint (planes [nshots][Np]): adjoint fields, the CPML memories' adjoints, the
    // differences' cotangents passed between the launches of one step, per-shot gradients
    float *aex, *aey, *ahz, *a_exy, *a_eyx, *b_hzx, *b_hzy, *d_ex, *d_ey, *d_hy, *d_hx;
    float *g_eps, *g_sig;
    const float* resid;    // [nshots][nt][nrec] cotangent of traces_p
    float geps;            // eps0 / dt
};
cudaError_t launch_te_coef(const float* eps_r, const float* sigma, int nx, int ny, int pitch,
                           float dt_eps0, float* ca, float* cb, int* status, cudaStream_t st);
// one time step: the H launch (with the receivers of step n), then the E launch
cudaError_t launch_te_h(const TeParams& p, int n, cudaStream_t st);
cudaError_t launch_te_e(const TeParams& p, int n, cudaStream_t st);
// one adjoint step n (reverse order): E updates reversed with the zero-lag gradients, Hz
// update reversed, the E cotangents gathered, the residual of step n injected
cudaError_t launch_te_adj_step(const TeParams& p, int n, int part, cudaStream_t st);
// Reverse-time reconstruction inside checkpoint segments (gf_reconstruct.cu).  ring_map:
// [ny][nx] ring index of each cell (-1 outside the ring); a ring slot holds Ez, Hx, Hy of the
// ring cells of every shot ([3][nshots][ring_cells]).
cudaError_t launch_ring_store(const float* st, int nshots, long long Np, int pitch, int nx,
                             int ny, const int* ring_map, int ring_cells, float* slot,
                             cudaStream_t stream);
// Undo step n (state_{n+1} -> state_n in place) and write Ez^n of shot s to
// hist + s * hist_stride_np.
cudaError_t launch_reverse_step(float* st, int nshots, long long Np, int pitch, int nx, int ny,
                                const int* ring_map, int ring_cells, const float* slot,
                                const float* ca, const float* cb, float rdx, float rdy,
                                float ch, const int2* src_xy, int nsrc, const float* wavelet,
                                int nt, int n, float src_scale, float* hist,
                                long long hist_stride_np, cudaStream_t stream);
// out[gy * nx + gx] = sum over shots of per_shot[s * pitch * ny + gy * pitch + gx].
cudaError_t launch_sum_shots(const float* per_shot, int nshots, int nx, int ny, int pitch,
                             float* out, int* status, cudaStream_t st);

}  // namespace gf
