// gf_internal.cuh -- types shared by the host runtime and the sm_103a kernels of libgprfwi.
#pragma once
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
constexpr int kRecStage = 4096;

// Device-status bits (OR-ed into the workspace status word by kernels).
constexpr int kStatusBadModel = 1;   // eps_r < 1, sigma < 0 or non-finite model value
constexpr int kStatusNonFinite = 2;  // non-finite trace or gradient

// Row pitch (floats) of the library's internal [ny][pitch] planes (state, wavefield store,
// per-shot gradients and illumination, update coefficients): nx rounded up to a multiple of
// 4, so that every row starts 16-byte aligned and column pairs (2i, 2i + 1) are 8-byte
// aligned.  Caller arrays (model, gradients, illumination) stay [ny][nx].
inline int row_pitch(int nx) { return (nx + 3) & ~3; }

// Left halo of a tile launch with K steps: K rounded up to even, so that the staged window
// starts on an even column (tile widths are even).
inline int left_halo(int K) { return (K + 1) & ~1; }

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
    const int* src_cell;    // [nshots][nsrc] linear cell index j*nx+i
    const int* rec_cell;    // [nshots][nrec]
    const float* st_in;     // time-stepping state at the start of the launch
    float* st_out;          // state at the end of the launch (other ping-pong buffer)
    float* hist;            // wavefield store, NULL = not stored: Ez^{n+1} of shot s at
                            // hist + (s * hist_stride + n - hist_slot0) * Np
    int hist_stride;        // slots per shot (nt for the full store, k + 1 for a segment)
    int hist_slot0;         // step whose Ez^{n+1} is slot 0 (0, or the segment start - 1)
    float* traces;          // forward: [nshots][nt][nrec] output
    const float* resid;     // adjoint: [nshots][nt][nrec] trace cotangent
    float* illum;           // forward: [nshots][Np] accumulated (NULL = skip)
    float* grad;            // adjoint: [2][nshots][Np] accumulated
    int n0, K;              // first time step of the launch, steps in the launch
    int tile_w, tile_h;     // interior tile size (tile_w even)
    int kl;                 // left halo of the staged window (left_halo(K)); K elsewhere
    int tiles_x, ntiles;
    // receivers of each (shot, tile) window [tx*tile_w - K, tx*tile_w + tile_w + K) x
    // [ty*tile_h - K, ty*tile_h + tile_h + K), host-built CSR sorted by row: entries
    // tile_rec_idx[off[s*ntiles+t] .. off[s*ntiles+t+1]) are receiver indices
    const int* tile_rec_off;
    const int* tile_rec_idx;
    int rec_max;            // longest of these lists (decides shared-memory staging)
    int* status;
};

// Host-side launchers.  Tile-kernel variants: 0 = 4 rows per thread, 512 threads, 64 x 64
// window; 1 = 4 rows per thread, 256 threads, 64 x 32 (two CTAs per SM); 2 = 8 rows per
// thread, 256 threads, 64 x 64.
cudaError_t launch_fwd_tile(const TileParams& p, int variant, cudaStream_t st);
cudaError_t launch_adj_tile(const TileParams& p, int variant, cudaStream_t st);
int max_tile_extent();              // staged window width
int max_tile_height(int variant);   // staged window height of a tile-kernel variant
int num_tile_variants();
size_t tile_smem_bytes(int variant);
cudaError_t configure_tile_kernels(size_t optin);

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
cudaError_t tv_gradient(int nx, int ny, const float* X, float* G, float* scratch, float lambda,
                        float mu, int iters, float weight, cudaStream_t st);
// out[gy * nx + gx] = sum over shots of per_shot[s * pitch * ny + gy * pitch + gx].
cudaError_t launch_sum_shots(const float* per_shot, int nshots, int nx, int ny, int pitch,
                             float* out, int* status, cudaStream_t st);

}  // namespace gf
