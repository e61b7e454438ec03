/*
 * gprfwi.h -- C ABI of the GB300 (sm_103a) library for the hot path of dual-parameter GPR
 * full waveform inversion (arXiv 2506.20513): the 2-D TM Maxwell FDTD time loop with CPML
 * absorbing boundaries and its exact discrete adjoint with zero-lag gradients (and the TE
 * mode that x- and y-polarised sources excite: gf_forward_model_te,
 * gf_misfit_and_gradient_te).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid.      Arrays are [ny][nx], x (horizontal) fastest, y (depth) second, FP32.  The
 *            absorbing layer (npml cells on each side) lies INSIDE the arrays, as the
 *            paper's model arrays do (Sec. 3.1, the demo strips pmlthick cells before
 *            saving).  Ez lives on integer nodes, Hx at (i, j+1/2), Hy at (i+1/2, j)
 *            (Sec. 2.1, Eqs. 3-5).  The outermost ring of Ez nodes is a PEC wall behind
 *            the CPML and is never updated.
 * Model.     eps_r (relative permittivity, >= 1) and sigma (conductivity in S/m, >= 0),
 *            both [ny][nx].  Cells with sigma > 100 S/m are perfect conductors (Sec. 3.2,
 *            coefficient listing).  Relative permeability is 1.
 * Shots.     A context holds nshots independent experiments ("step" in the paper's
 *            Table 1; every kernel carries a shot index, Sec. 3.2).  Each shot has nsrc
 *            z-polarised line sources and nrec receivers given as cell indices (i, j).
 * Wavelet.   Device FP32 [nshots][nsrc][nt]: w^n is injected into Ez^{n+1} as
 *            Ez(src) -= Cb(src) w^n / (dx dy)  (Sec. 3.2, hertzian-dipole listing with
 *            dl = dz = 1).
 * Traces.    Device FP32 [nshots][nt][nrec]: d^n = Ez^n sampled before the updates of
 *            step n (Algorithm 1, stage 1), so d^0 = 0.
 * Pointers.  Every array argument of a compute call is a DEVICE pointer on the context's
 *            device unless stated otherwise.  The caller owns every argument buffer; the
 *            library never frees or retains them beyond the call.  Calls are asynchronous
 *            on the given stream (a cudaStream_t passed as void*, NULL = legacy default
 *            stream) and return after enqueueing.
 * Errors.    Every call returns 0 (GF_OK) or a negative GF_E* code; gf_last_error() gives
 *            a one-line message.  Host-side argument errors are detected before anything
 *            is enqueued.  Errors found on the device (invalid model values, non-finite
 *            traces, exhausted bounded waits) are recorded in a device status word that
 *            gf_status() reads.  No call throws, traps or aborts.
 * Threads.   A context is not thread-safe; distinct contexts are independent.
 * Readings.  The calls follow the statement of the problem (forward_model(eps_r, sigma,
 *            sources, receivers) -> traces; misfit_and_gradient(eps_r, sigma, observed) ->
 *            J, g_eps_r, g_sigma) with these deliberate choices: the acquisition (sources,
 *            receivers) is fixed per context, as the paper's configuration fixes it per
 *            run; the wavefield storage (full, checkpoints every k steps, or checkpoints
 *            with reverse reconstruction) is a property of the context, set once with
 *            gf_set_storage, because it decides the workspace size, instead of an argument
 *            of every call; the misfit is written to device memory (a call enqueues and
 *            returns, and the next FWI step reads it there); host arrays are copied by the
 *            caller (the library's compute calls take device pointers only).
 */
#ifndef GPRFWI_H
#define GPRFWI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GF_OK 0
#define GF_EINVAL (-1)     /* bad argument: shape, index, NULL pointer, eps_r < 1, sigma < 0 */
#define GF_ECFL (-2)       /* time step violates the CFL bound (Sec. 2.1, Eq. cfl) */
#define GF_ENOMEM (-3)     /* device allocation failed or caller workspace too small */
#define GF_ECUDA (-4)      /* a CUDA runtime call failed (message in gf_last_error) */
#define GF_ENONFINITE (-5) /* non-finite trace or gradient detected on the device */
#define GF_ETIMEOUT (-6)   /* a bounded device-side wait ran out */
#define GF_ESTATE (-7)     /* call out of order (e.g. adjoint without a saved forward) */

/* Padded grid and CPML description (Sec. 4 parameter tables: dx, nx, ny, dt, pmlthick;
 * CPML grading per the convolutional PML of Roden & Gedney, which the paper names only as
 * "PML" kernels, Sec. 3.2). */
typedef struct gf_grid_desc {
    int32_t nx, ny;        /* array size in cells, CPML included */
    int32_t npml;          /* CPML width in cells on each side (0 = PEC box) */
    int32_t nt;            /* number of time steps */
    double dx, dy, dt;     /* cell size (m) and time step (s) */
    int32_t pml_order;     /* grading exponent m (e.g. 3) */
    double pml_sigma_max;  /* S/m; <= 0 selects 0.8 (m+1) / (eta0 d sqrt(pml_eps_ref)) */
    double pml_kappa_max;  /* >= 1 */
    double pml_alpha_max;  /* S/m (complex-frequency shift, linear taper to 0 at depth) */
    double pml_eps_ref;    /* reference relative permittivity of the sigma_max default */
} gf_grid_desc;

/* Acquisition geometry (Sec. 3.2 source / receiver listings; Table 1 source_location,
 * receiver_location, step, nsrc, nrx).  HOST pointers, copied during gf_create. */
typedef struct gf_acquisition {
    int32_t nshots;         /* >= 1 */
    int32_t nsrc;           /* sources per shot, 1..8 */
    int32_t nrec;           /* receivers per shot, >= 1; at most 65535 of them may fall in
                               one staged tile window (GF_EINVAL from gf_create or
                               gf_set_tiling otherwise) */
    const int32_t* src_ij;  /* [nshots][nsrc][2] cell indices (i, j), 1 <= i <= nx-2 ... */
    const int32_t* rec_ij;  /* [nshots][nrec][2] cell indices, same range (off the ring) */
} gf_acquisition;

typedef struct gf_ctx gf_ctx;

/* Wavefield storage for the adjoint (the forward wavefield store of Algorithm 1, stage 7;
 * checkpointing is the paper's stated future work for large models, Sec. 5). */
#define GF_STORE_FULL 0       /* every Ez^n of every shot kept in the workspace */
#define GF_STORE_CHECKPOINT 1 /* whole state every k steps; the adjoint recomputes each
                                 k-step segment from its checkpoint (one extra forward) */
#define GF_STORE_RECONSTRUCT 2 /* checkpoints every k steps; the adjoint recomputes each
                                  segment keeping only a boundary ring per step, then runs
                                  the updates backwards inside the segment (experimental) */

/* Create a context on CUDA device `device`: validates the grid (CFL, Eq. cfl) and the
 * geometry, builds the CPML profiles in FP64 on the host and uploads them with the
 * geometry (device memory owned by the context, freed by gf_destroy).  No workspace is
 * allocated here.  *out is set to NULL on failure; the returned code says why. */
int gf_create(gf_ctx** out, const gf_grid_desc* grid, const gf_acquisition* acq, int device);

/* Free everything the context owns (never a caller workspace).  NULL is accepted. */
void gf_destroy(gf_ctx* ctx);

/* Message of the last error on this context (static text for ctx == NULL). */
const char* gf_last_error(const gf_ctx* ctx);

/* Bytes of device workspace that gf_misfit_and_gradient / gf_forward with saving need for
 * the context's storage mode (store_mode must equal it; see gf_set_storage).
 * forward_only != 0 gives the smaller forward-only figure. */
int gf_workspace_size(const gf_ctx* ctx, int store_mode, int forward_only, size_t* bytes);

/* Hand the context a caller-owned device workspace (>= gf_workspace_size bytes, 256-byte
 * aligned).  The caller keeps ownership and must keep it alive and unused by others while
 * calls on this context are in flight.  Without it the library allocates its own workspace
 * with cudaMalloc on first use (freed by gf_destroy).  ws == NULL reverts to that. */
int gf_set_workspace(gf_ctx* ctx, void* ws, size_t bytes);

/* Time-blocking options: tile interior width/height in cells and time steps per block K.
 * A tile is advanced K steps at a time on a staged window of 64 x 64 cells (64 x 32 for
 * variant 1): the interior plus a left halo of K rounded up to even (to a multiple of 4 for
 * variant 3), a right halo of at least K and K rows above and below.  The tile width must be
 * even (a multiple of 4, and tiles at least K wide and high, for variant 3).  K = 0 keeps the
 * current K, a tile size of 0 selects the largest that fits.  Default: 48 x 50 interior,
 * K = 7.  Returns GF_EINVAL (and keeps the old tiling) when the shape does not fit. */
int gf_set_tiling(gf_ctx* ctx, int tile_w, int tile_h, int steps_per_launch);

/* Select how gf_forward / gf_misfit_and_gradient keep the forward wavefield for the adjoint:
 * GF_STORE_FULL (default; k ignored) or GF_STORE_CHECKPOINT with 1 <= k <= nt.  Checkpointing
 * needs ceil(nt/k) * 7 * nshots * nx * ny * 4 bytes of checkpoints plus (k + 1) * nshots * nx
 * * ny * 4 bytes of segment buffer instead of nt * nshots * nx * ny * 4, for one extra
 * forward pass.  Results agree with GF_STORE_FULL up to FP32 rounding (launches split at
 * segment boundaries group some sums differently).  GF_STORE_RECONSTRUCT with 1 <= k <= nt:
 * the same checkpoints; each segment's recomputation (one step per launch) keeps Ez, Hx, Hy
 * of a boundary ring (cells within npml + 2 of an edge) per step, (k + 1) * 3 * nshots *
 * ring_cells * 4 bytes, and the adjoint reconstructs Ez backwards from the segment's last
 * state (Algorithm 1's updates run in reverse outside the ring) into a (K + 1)-slot buffer
 * before each adjoint launch.  In lossy media the reversed E update divides by Ca < 1, so
 * FP32 rounding grows by about e^{sigma dt k / eps} over a segment: the gradient error
 * depends on k and sigma (experimental; GF_STORE_CHECKPOINT is exact to FP32 rounding).
 * Invalidates a stored forward. */
int gf_set_storage(gf_ctx* ctx, int mode, int k);

/* Kernel variant.  0-2: one kernel launch per time block, one CTA per (tile, shot): 0
 * (default) = four rows per thread, 512-thread CTAs, 64 x 64 window; 1 = four rows per
 * thread, 256-thread CTAs
 * on a 64 x 32 window, two CTAs per SM (tile height + 2 steps <= 32; a taller current tile is
 * shrunk to fit); 2 = eight rows per thread, 256-thread CTAs, 64 x 64.  3 = the
 * persistent dataflow kernels: one cooperative launch per pass, CTAs pulling (time block,
 * shot, tile) items with per-tile completion counters and bounded waits (GF_ETIMEOUT from
 * gf_status when one runs out), variant 0's window, the next item's state prefetched while
 * the current one runs (the tile width is rounded down to a multiple of 4).  All compute the
 * same result up to FP32 rounding. */
int gf_set_variant(gf_ctx* ctx, int variant);

/* Shot lanes (1-4, default 2): the shots are split into that many contiguous groups whose
 * passes run concurrently on the context's own streams, forked from and joined back into the
 * caller's stream, so that one group's launches fill the SMs the other's last wave leaves
 * idle.  Results do not depend on the lanes (every shot's arithmetic and every sum's order
 * are the same).  Used by the per-launch variants (0-2) with GF_STORE_FULL or
 * GF_STORE_CHECKPOINT; the persistent variant, GF_STORE_RECONSTRUCT and recorded batch
 * schedules run one lane. */
int gf_set_lanes(gf_ctx* ctx, int lanes);

/* Current tiling and variant (for autotuners). */
int gf_get_tiling(const gf_ctx* ctx, int* tile_w, int* tile_h, int* steps_per_launch,
                  int* variant);

/* forward_model(eps_r, sigma, sources, receivers) -> traces (Algorithm 1 for all shots).
 * traces: [nshots][nt][nrec] written.  illum: optional [ny][nx], receives the illumination
 * sum over shots and n = 1..nt of (Ez^n)^2 (NULL to skip).  Nothing is kept for an adjoint. */
int gf_forward_model(gf_ctx* ctx, const float* eps_r, const float* sigma, const float* wavelet,
                     float* traces, float* illum, void* stream);

/* gf_forward_model that also records the receivers' magnetic components (the paper's
 * receivers store every field component, Sec. 3.2 store_outputs; in the 2-D TM mode those
 * are Ez, Hx, Hy): h_traces, device [nshots][nt][nrec][2] or NULL, gets Hx^{n-1/2} at (i,
 * j+1/2) and Hy^{n-1/2} at (i+1/2, j) of each receiver cell (i, j), sampled with d^n = Ez^n
 * (before step n's updates; zero at n = 0).  Forward only: the misfit and its gradient use
 * Ez. */
int gf_forward_model_fields(gf_ctx* ctx, const float* eps_r, const float* sigma,
                            const float* wavelet, float* traces, float* h_traces, float* illum,
                            void* stream);

/* Forward model of the TE mode: the fields of an x-directed (polarisation 0) or y-directed
 * (polarisation 1) hertzian line source (Sec. 3.2 source listing, polarisations 0 and 1; in
 * 2-D they excite Ex, Ey, Hz, while the z-directed source of the calls above drives the TM
 * mode).  Same context, grid, CPML, acquisition and wavelet layout as gf_forward_model; the
 * sources and receivers sit at the E node of their component in cell (i, j): Ex at
 * (i+1/2, j), Ey at (i, j+1/2), Hz at (i+1/2, j+1/2).  Every E component takes Ca, Cb of the
 * cell whose index it carries (the coefficient listing's per-index material); PEC walls on
 * the outermost rows and columns; perfect conductors (sigma > 100 S/m) hold E at zero.
 * One step n: record, H update, E update with the source current w^n / (dx dy) of the
 * polarisation's component (as for Ez).
 * traces: device [nshots][nt][nrec][3] written with Ex^n, Ey^n and Hz^{n-1/2} of each
 * receiver cell (before step n's updates; zero at n = 0).  Forward only, one step per
 * launch pair (no temporal blocking, no lanes); it uses the forward workspace's state
 * buffers, so a wavefield stored by gf_forward is dropped (gf_adjoint then returns
 * GF_ESTATE).  A bad model sets the status word (gf_status).  GF_EINVAL for a NULL
 * pointer or another polarisation. */
int gf_forward_model_te(gf_ctx* ctx, const float* eps_r, const float* sigma,
                        const float* wavelet, int polarisation, float* traces, void* stream);

/* misfit_and_gradient for the TE mode: J = 1/2 sum (d - o)^2 over the traces of the
 * source's own component (Ex^n for polarisation 0, Ey^n for 1) and its exact discrete
 * gradients, summed over shots.  The forward keeps Ex and Ey of every step; the adjoint
 * transposes each step in reverse (E updates with their CPML memories, Hz update with its
 * memories, recording).  Each cell's gradient is the zero-lag form of both of its E
 * components: with lam = Cb * adjoint(E^{n+1}),
 *   dJ/deps_r = -sum_n lam (E^{n+1} - E^n) eps0 / dt,  dJ/dsigma = -sum_n lam (E^{n+1} + E^n) / 2
 * (the TE counterpart of Eqs. grad_eps / grad_sigma).
 * observed: device [nshots][nt][nrec].  misfit: device FP64 scalar.  g_eps_r, g_sigma:
 * device [ny][nx] or NULL.  traces: optional device [nshots][nt][nrec][3] as in
 * gf_forward_model_te.  The E history (nt * 2 * nshots * ny * pitch floats) and the trace
 * buffers are held by the context until gf_destroy; GF_ENOMEM if they cannot be allocated.
 * One step per launch group, no lanes; it drops a wavefield stored by gf_forward, like
 * gf_forward_model_te. */
int gf_misfit_and_gradient_te(gf_ctx* ctx, const float* eps_r, const float* sigma,
                              const float* wavelet, int polarisation, const float* observed,
                              double* misfit, float* g_eps_r, float* g_sigma, float* traces,
                              void* stream);

/* The misfit of gf_misfit_and_gradient_te alone (a line-search evaluation): the TE forward
 * model and J = 1/2 sum (d - o)^2 over the source component's traces, no history, no
 * adjoint.  Bit-identical to the J of gf_misfit_and_gradient_te on the same inputs.
 * observed: device [nshots][nt][nrec]; misfit: device FP64 scalar.  Uses the context's TE
 * trace buffer (held until gf_destroy). */
int gf_misfit_te(gf_ctx* ctx, const float* eps_r, const float* sigma, const float* wavelet,
                 int polarisation, const float* observed, double* misfit, void* stream);

/* Forward run that also stores the wavefield (mode GF_STORE_FULL) in the workspace for a
 * later gf_adjoint on the same model, wavelet and stream. */
int gf_forward(gf_ctx* ctx, const float* eps_r, const float* sigma, const float* wavelet,
               float* traces, float* illum, int store_mode, void* stream);

/* Adjoint run (Algorithm 2) of the last gf_forward, driven by the trace cotangent
 * resid = dL/dtraces [nshots][nt][nrec].  Writes g_eps_r = dL/deps_r and g_sigma =
 * dL/dsigma (per S/m), [ny][nx], summed over shots: the discrete zero-lag gradients
 * -sum_n lam^{n+1} (Ez^{n+1} - Ez^n) eps0/dt and -sum_n lam^{n+1} (Ez^{n+1} + Ez^n)/2 with
 * lam = Cb * adjoint(Ez) (Sec. 2.1, Eqs. grad_eps and grad_sigma).  Either output may be
 * NULL.  Returns GF_ESTATE if no stored forward exists. */
int gf_adjoint(gf_ctx* ctx, const float* eps_r, const float* sigma, const float* resid,
               float* g_eps_r, float* g_sigma, void* stream);

/* misfit_and_gradient(eps_r, sigma, observed) -> J, g_eps_r, g_sigma: the L2 misfit
 * J = 1/2 sum_{s,n,r} (d - o)^2 (Sec. 2.1, Eq. objective) written as one FP64 value to
 * *misfit (device), and its exact gradients as in gf_adjoint.  observed: [nshots][nt][nrec].
 * traces (optional, may be NULL) receives the modelled data.  Equivalent to gf_forward +
 * residual + gf_adjoint, enqueued on one stream. */
int gf_misfit_and_gradient(gf_ctx* ctx, const float* eps_r, const float* sigma,
                           const float* wavelet, const float* observed, double* misfit,
                           float* g_eps_r, float* g_sigma, float* traces, void* stream);

/* Misfit only (a line-search evaluation): forward model of all shots and J = 1/2 sum (d - o)^2
 * (Eq. objective) into *misfit (device FP64).  Nothing is kept for an adjoint. */
int gf_misfit(gf_ctx* ctx, const float* eps_r, const float* sigma, const float* wavelet,
              const float* observed, double* misfit, void* stream);

/* Total-variation term of Algorithm 3 (Sec. 3.4), read as split Bregman for
 * min_u 1/2 |u - x|^2 + lambda TV(u), TV(u) = sum sqrt((Dx u)^2 + (Dy u)^2) with circular
 * differences, on x = model / max|model|, from u = x, Z = D x, B = 0 (lambda = 0 changes
 * nothing): `iters` sweeps of u = (x + mu D^T(Z - B) + mu * sum
 * of the 4 neighbours of u) / (1 + 4 mu), Z = shrink(Du + B, lambda/mu), B += Du - Z; then
 * grad += weight * max|grad| * (x - u) (normalised units).  One
 * neighbour average per iteration converges for small mu (0.2 is a safe choice).
 * model, grad: device [ny][nx]; scratch: device, gf_tv_scratch_bytes(nx, ny) bytes, owned by
 * the caller.  Asynchronous on `stream`; errors via gf_last_error(NULL). */
size_t gf_tv_scratch_bytes(int nx, int ny);
int gf_tv_gradient(int nx, int ny, const float* model, float* grad, void* scratch, float lambda,
                   float mu, int iters, float weight, void* stream);

/* One Adam step (Sec. 2.3: the updates of eps_r and sigma with bias-corrected first and
 * second moments) on n cells of one model parameter, in place, on `stream`:
 *   g' = gscale * grad;  m = beta1 m + (1 - beta1) g';  v = beta2 v + (1 - beta2) g'^2;
 *   x  = max(xmin, x - lr * (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps))
 * at the cells where mask != 0 (mask NULL: every cell); masked cells keep x, m and v.
 * x, grad, m, v, mask: device float32 [n], owned by the caller (m, v zeroed before t = 1).
 * t >= 1 is this parameter's step count; 0 <= beta < 1, eps > 0, lr >= 0, else GF_EINVAL
 * (message via gf_last_error(NULL)).  The clamp at xmin is the paper's eps_r >= 1,
 * sigma >= 0 projection (Sec. 3.1 demo). */
int gf_adam_update(long long n, float* x, const float* grad, float* m, float* v,
                   const float* mask, float gscale, float lr, float beta1, float beta2, float eps,
                   int t, float xmin, void* stream);

/* Synchronise `stream` and return the device status word (GF_OK or the first device-side
 * error since the last gf_status call), then clear it. */
int gf_status(gf_ctx* ctx, void* stream);

/* Host helper: Ricker wavelet w(n dt) = amp (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2),
 * tau = n dt - sqrt(2)/f0, n = 0..nt-1, into the HOST array out[nt] (the paper's
 * source_amplitudes = ['ricker', amplitude, f0], Sec. 4 tables). */
int gf_ricker(float* out, int nt, double dt, double f0, double amp);

/* Kernel families for the profiling counters below. */
#define GF_KERNEL_FWD 0 /* temporally blocked forward tile kernel (Algorithm 1) */
#define GF_KERNEL_ADJ 1 /* temporally blocked adjoint tile kernel (Algorithm 2) */
#define GF_KERNEL_AUX 2 /* model check, residual / misfit, shot sums */

/* Number of kernels this context has launched since gf_create (all families). */
long long gf_kernel_launches(const gf_ctx* ctx);

/* Polls of one dependency wait of the persistent kernels (variant 3) before it gives up and
 * records GF_ETIMEOUT (default 4194304, about a second; polls >= 0).  A wait that runs out
 * ends its CTA; the results of that call are then undefined, the next call starts afresh.
 * Fault-injection hook for tests: a budget of 0 makes any wait that is not already satisfied
 * run out. */
int gf_set_wait_budget(gf_ctx* ctx, long long polls);

/* enable != 0: from now on bracket every kernel launch with CUDA events on its stream (no
 * synchronisation is added); enable == 0 stops and drops what was recorded. */
int gf_profile(gf_ctx* ctx, int enable);

/* Synchronise on the recorded events and return, for one kernel family, the summed device
 * time in milliseconds and the number of launches recorded since the last read (or since
 * profiling was enabled); the family's record is then cleared. */
int gf_profile_read(gf_ctx* ctx, int kind, double* ms_total, long long* launches);

/* As gf_profile_read, and also the length in milliseconds of the union of the launches'
 * intervals (launches of concurrent lanes, and consecutive launches under programmatic
 * dependent launch, overlap: the union is the time the family kept the GPU busy).  kind 3:
 * the forward and adjoint families together, read without clearing them. */
int gf_profile_read_span(gf_ctx* ctx, int kind, double* ms_total, double* ms_span,
                         long long* launches);

/* Forward model without any memory allocation.  The paper has no counterpart: this is a
 * service for callers that may not allocate device memory (their memory belongs to another
 * runtime or a fixed pool, or they run under a hard budget or in a loop that must not enter
 * the allocator).  It computes the same forward model as gf_forward_model, to FP32 rounding,
 * with its own fixed tiling (48 x 48 tiles, 8 steps per launch), without a context: grid and
 * acq are as for gf_create (HOST pointers, read only before the call returns); eps_r, sigma,
 * wavelet are device inputs and traces the device output [nshots][nt][nrec], all owned by the
 * caller, on `device`.  All working memory (time-stepping state, CPML profiles, geometry,
 * per-tile receiver lists) lives in one static 64 MiB device array that every GPU loading
 * this library holds until the process exits; the call never calls cudaMalloc, cudaFree or
 * another allocating routine.  Limits: nx, ny <= 16384 and about nshots * nx * ny <= 1.1e6
 * cells (GF_ENOMEM with the exact need otherwise); GF_EINVAL and GF_ECFL as for gf_create;
 * messages via gf_last_error(NULL).  Model values are not checked on the device.  The array
 * is shared by all calls on a device and keeps the last call's contents (each call clears
 * what must start at zero); calls that overlap on the GPU race and must be serialised by the
 * caller.  Every call copies the geometry from host memory and synchronises `stream` once, so
 * no call can be captured into a CUDA graph: on a stream that is capturing, the call returns
 * GF_EINVAL before it touches the stream (the capture stays valid). */
int gf_forward_model_noalloc(const gf_grid_desc* grid, const gf_acquisition* acq, int device,
                             const float* eps_r, const float* sigma, const float* wavelet,
                             float* traces, void* stream);

/* Autotuner (tile shape, time-block depth, kernel variant).  Looks up the context's shape
 * (device name, nx, ny, npml, shots, sources, receivers) in the text cache `cache_path`
 * (NULL = no cache); on a miss, times a forward pass over the first `probe_steps` steps (0 =
 * 48) for each candidate (variants 0 and 3 with 4, 5, 6, 7, 8 or 10 steps per launch,
 * variant 1 with 3..6, variant 2 with 5 and 7; each with its default tile for that depth),
 * with CUDA events on `stream`, keeps the fastest and appends it to the cache.  Candidates a
 * caller workspace cannot hold are skipped (give the context no workspace, or a library-
 * owned one, to probe them all).  Leaves the chosen tiling set on the context (read it back
 * with gf_get_tiling).  Synchronises `stream`.  eps_r, sigma, wavelet: device inputs as for
 * gf_forward_model. */
int gf_autotune(gf_ctx* ctx, const float* eps_r, const float* sigma, const float* wavelet,
                const char* cache_path, int probe_steps, void* stream);

/* Batches of independent instances (contexts of possibly different grids, shots and nt on
 * one device), for many small inversions at once.  The batch owns one stream per instance;
 * it does not own the contexts, which must outlive it. */
typedef struct gf_batch gf_batch;
int gf_batch_create(gf_batch** out, gf_ctx* const* ctxs, int n);
void gf_batch_destroy(gf_batch* batch);
const char* gf_batch_last_error(const gf_batch* batch);

/* misfit_and_gradient for every instance i (arrays of n device pointers, as for
 * gf_misfit_and_gradient; misfit: device double[n]).  mode 0: one instance after the other on
 * `stream`; mode 1: all instances concurrently on the batch's streams, forked from and joined
 * back into `stream`; mode 2: mode 1 captured once into a CUDA graph and replayed (a single
 * graph launch per call) while the argument pointers and every context's configuration stay
 * the same, re-captured otherwise; mode 3: the persistent multi-instance schedule (every
 * context must use the persistent variant 3): each context's operations run in its own order
 * on `stream`, and the persistent passes that the contexts have pending at the same point
 * (forward with the wavefield store, forward without it, or adjoint) run as ONE cooperative
 * launch over all of their work items, block-major across the instances, each item waiting
 * (bounded, GF_ETIMEOUT via gf_status of its context) only for its own instance's neighbours;
 * mode 4: mode 3 captured once into a CUDA graph and replayed under the same rule as mode 2.
 * The schedule of modes 3 and 4 is recorded on the first call and kept (with a device copy of
 * its work items) while the argument pointers and the contexts' configuration, wait budget
 * included, stay the same.  Each context's workspace is allocated before the first fork;
 * profiling must be off.  Asynchronous on `stream`. */
int gf_batch_misfit_and_gradient(gf_batch* batch, const float* const* eps_r,
                                 const float* const* sigma, const float* const* wavelet,
                                 const float* const* observed, double* misfit,
                                 float* const* g_eps_r, float* const* g_sigma, int mode,
                                 void* stream);

/* Library version string. */
const char* gf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GPRFWI_H */
