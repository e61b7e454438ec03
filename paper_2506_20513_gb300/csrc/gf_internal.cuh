// gf_internal.cuh -- types shared by the host runtime and the sm_103a kernels of libgprfwi.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace gf {

constexpr int kMaxSrc = 8;        // sources per shot
constexpr int kNumFields = 7;     // Ez, Hx, Hy, psiEx, psiEy, psiHx, psiHy (or their adjoints)
// Shared-memory words in which the adjoint tile kernel stages its tile's receiver positions
// and the residual samples of its launch (entries x (K + 1) words must fit).
constexpr int kRecStage = 1536;

// Device-status bits (OR-ed into the workspace status word by kernels).
constexpr int kStatusBadModel = 1;   // eps_r < 1, sigma < 0 or non-finite model value
constexpr int kStatusNonFinite = 2;  // non-finite trace or gradient

// CPML profiles of one axis (FP32, uploaded once per context).  For a node at index i:
//   a = 1 / (kappa * d), b = exp(-(sigma/kappa + alpha) dt / eps0),
//   c = sigma (b - 1) / (sigma kappa + kappa^2 alpha) / d  (0 outside the CPML),
// "E" arrays at integer nodes, "H" arrays at the half node i + 1/2.
struct AxisProfile {
    const float *aE, *bE, *cE, *aH, *bH, *cH;
};

// Everything one tile launch needs.  State arrays are packed as [kNumFields][nshots][N].
struct TileParams {
    int nx, ny, npml, nt, nshots, nsrc, nrec;
    long long N;         // nx * ny
    float dt_eps0;       // dt / eps0
    float ch;            // dt / mu0
    float src_scale;     // 1 / (dx dy)
    float geps;          // eps0 / dt (zero-lag eps_r gradient scale)
    float rdx, rdy;      // 1 / dx, 1 / dy
    AxisProfile px, py;
    const float* eps_r;
    const float* sigma;
    const float* wavelet;   // [nshots][nsrc][nt]
    const int* src_cell;    // [nshots][nsrc] linear cell index j*nx+i
    const int* rec_cell;    // [nshots][nrec]
    const float* st_in;     // time-stepping state at the start of the launch
    float* st_out;          // state at the end of the launch (other ping-pong buffer)
    float* hist;            // wavefield store, NULL = not stored: Ez^{n+1} of shot s at
                            // hist + (s * hist_stride + n - hist_slot0) * N
    int hist_stride;        // slots per shot (nt for the full store, k + 1 for a segment)
    int hist_slot0;         // step whose Ez^{n+1} is slot 0 (0, or the segment start - 1)
    float* traces;          // forward: [nshots][nt][nrec] output
    const float* resid;     // adjoint: [nshots][nt][nrec] trace cotangent
    float* illum;           // forward: [nshots][N] accumulated (NULL = skip)
    float* grad;            // adjoint: [2][nshots][N] accumulated
    int n0, K;              // first time step of the launch, steps in the launch
    int tile_w, tile_h;     // interior tile size; the staged tile has a K-cell halo
    int tiles_x, ntiles;
    int halo;               // staged halo of the warp-march kernel (>= K)
    // receivers of each (shot, tile) staged window, host-built CSR: entries
    // tile_rec_idx[off[s*ntiles+t] .. off[s*ntiles+t+1]) are receiver indices in index order
    const int* tile_rec_off;
    const int* tile_rec_idx;
    int* status;
    int rec_staged;         // adjoint: every tile's receiver list fits the staging area
};

// Host-side launchers (one per kernel family).
// Tile-kernel variants: 0 = 4 rows per thread (1024 threads), 1 = 8 rows (512 threads).
cudaError_t launch_fwd_tile(const TileParams& p, int variant, cudaStream_t st);
cudaError_t launch_adj_tile(const TileParams& p, int variant, cudaStream_t st);
// Warp-march forward kernel: 64-column strips, chunks of tile_h rows, K <= march_max_steps().
cudaError_t launch_fwd_march(const TileParams& p, int chunks, cudaStream_t st);
cudaError_t configure_march_kernels(size_t optin);
size_t march_smem_bytes();
int march_max_steps();
int max_tile_extent();              // staged tile (interior + 2K halo) width limit
int max_tile_height(int variant);   // staged tile height limit of a tile-kernel variant
int num_tile_variants();
size_t tile_smem_bytes(int variant);
cudaError_t configure_tile_kernels(size_t optin);

cudaError_t launch_check_model(const float* eps_r, const float* sigma, long long N, int* status,
                               cudaStream_t st);
cudaError_t launch_residual_misfit(const float* traces, const float* observed, float* resid,
                                   long long count, double* partial, int nblocks, int* status,
                                   cudaStream_t st);
cudaError_t launch_finish_misfit(const double* partial, int nblocks, double* misfit,
                                 cudaStream_t st);
size_t tv_scratch_floats(long long n);
cudaError_t tv_gradient(int nx, int ny, const float* X, float* G, float* scratch, float lambda,
                        float mu, int iters, float weight, cudaStream_t st);
cudaError_t launch_sum_shots(const float* per_shot, int nshots, long long N, float* out,
                             int* status, cudaStream_t st);

}  // namespace gf
