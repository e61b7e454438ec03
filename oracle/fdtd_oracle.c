/*
 * fdtd_oracle.c -- plain FP64 CPU oracle for the 2-D TM FDTD forward model and its
 * exact discrete adjoint (dual-parameter GPR full waveform inversion, arXiv 2506.20513).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py may load this code.  It shares no code, header, table or
 * constant with the CUDA library: every formula below is written out again here, in double
 * precision, with plain loops and no blocking, fusion or reordering beyond what the method
 * states.
 *
 * What is computed (paper notation; x is the fast array axis, y the second axis):
 *   fields  Ez(i,j) at integer nodes, Hx(i,j) at (i, j+1/2), Hy(i,j) at (i+1/2, j)
 *           (Sec. 2.1, Eqs. 3-5: 2-D TM Yee discretisation).
 *   arrays  [ny][nx], index j*nx + i, the CPML of width npml lies inside the arrays.
 *   E update uses the time-averaged loss form of the paper's coefficient listing
 *   (Sec. 3.2, "ucget"): EA = eps/dt + sigma/2, EB = eps/dt - sigma/2,
 *   Ca = EB/EA, Cb = 1/EA, Cb = Ca = 0 where sigma > 100 S/m (PEC rule);
 *   H update coefficient Ch = dt / mu0 (relative permeability 1).
 *   The outermost ring of Ez nodes is held at zero (PEC behind the CPML); Ez is updated for
 *   1 <= i <= nx-2, 1 <= j <= ny-2, Hx for 0 <= j <= ny-2 (all i), Hy for 0 <= i <= nx-2
 *   (all j).
 *   CPML: convolutional PML (Roden & Gedney, 2000) with graded profiles
 *     sigma(u) = sigma_max u^m, kappa(u) = 1 + (kappa_max-1) u^m, alpha(u) = alpha_max (1-u),
 *     u = depth / (npml * d), b = exp(-(sigma/kappa + alpha) dt / eps0),
 *     c = sigma (b - 1) / (sigma kappa + kappa^2 alpha),
 *     sigma_max = 0.8 (m+1) / (eta0 d sqrt(eps_ref)) unless given.
 *   One time step n (Algorithm 1 order):
 *     1 record d^n = Ez^n at each receiver
 *     2-3 H and magnetic-CPML update from Ez^n  -> H^{n+1/2}
 *     4-5 E and electric-CPML update from H^{n+1/2} -> Ez^{n+1}
 *     6 hertzian line source: Ez(src) -= Cb(src) * w^n / (dx dy)   (Sec. 3.2 source listing,
 *       dl = dz = 1 in 2-D)
 *     7 store Ez^{n+1} (full history, for the adjoint)
 *   Misfit J = 1/2 sum_{n,r} (d^n_r - o^n_r)^2 (Eq. objective).
 *   Adjoint: the exact transpose of every step above, taken in reverse (Algorithm 2 order:
 *   adjoint source, E, E-PML, H, H-PML, gradients).  Two equivalent gradient forms are
 *   produced:
 *     coefficient form  dJ/deps = sum_n Ebar^{n+1}(dCa/deps Ez^n + dCb/deps Q^n), same for sigma,
 *     zero-lag form     dJ/deps = -sum_n lam^{n+1} (Ez^{n+1}-Ez^n)/dt,
 *                       dJ/dsigma = -sum_n lam^{n+1} (Ez^{n+1}+Ez^n)/2,  lam = Cb Ebar
 *   (the discrete counterpart of Eqs. grad_eps / grad_sigma), returned per relative
 *   permittivity (times eps0) and per S/m.
 *
 * The TE mode an x- or y-polarised source excites (Ex, Ey, Hz) has its own forward model,
 * or_forward_te_shot, at the end of this file.
 *
 * Nothing here is tuned.  Shots are independent and may run on separate OpenMP threads;
 * the per-shot gradients are then summed in shot order, so results do not depend on the
 * thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_EPS0 8.8541878128e-12  /* F/m, CODATA 2018 */
#define OR_MU0 1.25663706212e-6   /* H/m, CODATA 2018 */

typedef struct {
    int32_t nx, ny, npml, nt;
    double dx, dy, dt;
    int32_t pml_order;
    double pml_sigma_max; /* <= 0: use the optimal-grading default */
    double pml_kappa_max;
    double pml_alpha_max;
    double pml_eps_ref;
} or_grid;

/* CPML profiles of one axis: E nodes at integer positions, H nodes at half-integer ones. */
typedef struct {
    double *bE, *cE, *kE; /* [n]  */
    double *bH, *cH, *kH; /* [n]  (H node i sits at i+1/2) */
} or_axis;

static void or_axis_free(or_axis* a) {
    free(a->bE); free(a->cE); free(a->kE);
    free(a->bH); free(a->cH); free(a->kH);
}

/* One profile value at normalised depth u in (0,1]; u <= 0 means "not in the CPML". */
static void or_cpml_point(const or_grid* g, double d, double u, double* b, double* c, double* k) {
    if (u <= 0.0) { *b = 0.0; *c = 0.0; *k = 1.0; return; }
    double m = (double)g->pml_order;
    double smax = g->pml_sigma_max;
    if (smax <= 0.0) {
        double eta0 = sqrt(OR_MU0 / OR_EPS0);
        smax = 0.8 * (m + 1.0) / (eta0 * d * sqrt(g->pml_eps_ref));
    }
    double s = smax * pow(u, m);
    double kap = 1.0 + (g->pml_kappa_max - 1.0) * pow(u, m);
    double al = g->pml_alpha_max * (1.0 - u);
    *b = exp(-(s / kap + al) * g->dt / OR_EPS0);
    *c = (s > 0.0) ? s * (*b - 1.0) / (s * kap + kap * kap * al) : 0.0;
    *k = kap;
}

/* Depth into the CPML, in cells, of a node at (possibly half-integer) position p on an axis
 * of n nodes whose physical part spans [npml, n-1-npml]. */
static double or_depth(int n, int npml, double p) {
    double lo = (double)npml, hi = (double)(n - 1 - npml);
    if (p < lo) return lo - p;
    if (p > hi) return p - hi;
    return 0.0;
}

static int or_axis_init(const or_grid* g, int n, double d, or_axis* a) {
    a->bE = calloc(n, sizeof(double)); a->cE = calloc(n, sizeof(double)); a->kE = calloc(n, sizeof(double));
    a->bH = calloc(n, sizeof(double)); a->cH = calloc(n, sizeof(double)); a->kH = calloc(n, sizeof(double));
    if (!a->bE || !a->cE || !a->kE || !a->bH || !a->cH || !a->kH) return -1;
    for (int i = 0; i < n; ++i) {
        double uE = g->npml > 0 ? or_depth(n, g->npml, (double)i) / g->npml : 0.0;
        double uH = g->npml > 0 ? or_depth(n, g->npml, (double)i + 0.5) / g->npml : 0.0;
        or_cpml_point(g, d, uE, &a->bE[i], &a->cE[i], &a->kE[i]);
        or_cpml_point(g, d, uH, &a->bH[i], &a->cH[i], &a->kH[i]);
    }
    return 0;
}

/* Update coefficients of the paper's "ucget" listing, per cell, in FP64.  Ring cells and
 * PEC cells (sigma > 100 S/m) get Ca = Cb = 0. */
static void or_coefficients(const or_grid* g, const double* eps_r, const double* sigma, double* Ca, double* Cb) {
    int nx = g->nx, ny = g->ny;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int c = j * nx + i;
            int ring = (i == 0 || j == 0 || i == nx - 1 || j == ny - 1);
            if (ring || sigma[c] > 100.0) { Ca[c] = 0.0; Cb[c] = 0.0; continue; }
            double EA = OR_EPS0 * eps_r[c] / g->dt + 0.5 * sigma[c];
            double EB = OR_EPS0 * eps_r[c] / g->dt - 0.5 * sigma[c];
            Ca[c] = EB / EA;
            Cb[c] = 1.0 / EA;
        }
}

/* ---------------------------------------------------------------------------------------
 * Forward model of one shot (Algorithm 1).  Outputs (each may be NULL):
 *   traces [nt][nrec]            d^n = Ez^n at the receivers
 *   h_traces [nt][nrec][2]       Hx^{n-1/2} at (i, j+1/2) and Hy^{n-1/2} at (i+1/2, j) of
 *                                the receiver cells, sampled with d^n (the paper's receivers
 *                                store every field component, Sec. 3.2 store_outputs)
 *   ez_hist [(nt+1)][ny*nx]      Ez^0 .. Ez^nt
 *   q_hist [nt][ny*nx]           Q^n, the bracket multiplied by Cb in the step-n E update,
 *                                including the source term
 *   energy [nt]                  W^n = dx dy sum(eps Ez^n^2 + mu0 (Hx^{n-1/2} Hx^{n+1/2}
 *                                + Hy^{n-1/2} Hy^{n+1/2})), the conserved discrete energy of
 *                                the lossless Yee scheme
 * -------------------------------------------------------------------------------------*/
int or_forward_shot(const or_grid* g, const double* eps_r, const double* sigma,
                    int nsrc, const int32_t* src, const double* wav,
                    int nrec, const int32_t* rec,
                    double* traces, double* h_traces, double* ez_hist, double* q_hist,
                    double* energy) {
    const int nx = g->nx, ny = g->ny, nt = g->nt;
    const size_t N = (size_t)nx * ny;
    const double dx = g->dx, dy = g->dy, dt = g->dt;
    const double Ch = dt / OR_MU0;
    or_axis ax, ay;
    if (or_axis_init(g, nx, dx, &ax) || or_axis_init(g, ny, dy, &ay)) return -1;
    double *Ez = calloc(N, sizeof(double)), *Hx = calloc(N, sizeof(double)), *Hy = calloc(N, sizeof(double));
    double *pEx = calloc(N, sizeof(double)), *pEy = calloc(N, sizeof(double));
    double *pHx = calloc(N, sizeof(double)), *pHy = calloc(N, sizeof(double));
    double *Ca = calloc(N, sizeof(double)), *Cb = calloc(N, sizeof(double)), *Q = calloc(N, sizeof(double));
    if (!Ez || !Hx || !Hy || !pEx || !pEy || !pHx || !pHy || !Ca || !Cb || !Q) return -1;
    or_coefficients(g, eps_r, sigma, Ca, Cb);
    if (ez_hist) memset(ez_hist, 0, N * sizeof(double)); /* Ez^0 = 0 */

    for (int n = 0; n < nt; ++n) {
        /* 1. save receiver data (Ez^n, before this step's updates) */
        if (traces)
            for (int r = 0; r < nrec; ++r)
                traces[(size_t)n * nrec + r] = Ez[(size_t)rec[2 * r + 1] * nx + rec[2 * r]];
        if (h_traces)
            for (int r = 0; r < nrec; ++r) {
                const size_t c = (size_t)rec[2 * r + 1] * nx + rec[2 * r];
                h_traces[((size_t)n * nrec + r) * 2] = Hx[c];
                h_traces[((size_t)n * nrec + r) * 2 + 1] = Hy[c];
            }
        double wsum = 0.0;
        if (energy)
            for (size_t c = 0; c < N; ++c) wsum += OR_EPS0 * eps_r[c] * Ez[c] * Ez[c];
        /* 2-3. magnetic field and magnetic CPML (Eqs. hx_update, hy_update) */
        for (int j = 0; j <= ny - 2; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = (size_t)j * nx + i;
                double D = (Ez[c + nx] - Ez[c]) / dy;
                pHx[c] = ay.bH[j] * pHx[c] + ay.cH[j] * D;
                double old = Hx[c];
                Hx[c] = old - Ch * (D / ay.kH[j] + pHx[c]);
                if (energy) wsum += OR_MU0 * old * Hx[c];
            }
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i <= nx - 2; ++i) {
                size_t c = (size_t)j * nx + i;
                double D = (Ez[c + 1] - Ez[c]) / dx;
                pHy[c] = ax.bH[i] * pHy[c] + ax.cH[i] * D;
                double old = Hy[c];
                Hy[c] = old + Ch * (D / ax.kH[i] + pHy[c]);
                if (energy) wsum += OR_MU0 * old * Hy[c];
            }
        if (energy) energy[n] = wsum * dx * dy;
        /* 4-5. electric field and electric CPML (Eq. ez_explicit in the Ca/Cb form) */
        for (int j = 1; j <= ny - 2; ++j)
            for (int i = 1; i <= nx - 2; ++i) {
                size_t c = (size_t)j * nx + i;
                double Dx = (Hy[c] - Hy[c - 1]) / dx;
                double Dy = (Hx[c] - Hx[c - nx]) / dy;
                pEx[c] = ax.bE[i] * pEx[c] + ax.cE[i] * Dx;
                pEy[c] = ay.bE[j] * pEy[c] + ay.cE[j] * Dy;
                Q[c] = Dx / ax.kE[i] + pEx[c] - Dy / ay.kE[j] - pEy[c];
            }
        /* 6. source injection enters the same bracket: Ez(src) -= Cb w^n / (dx dy) */
        for (int s = 0; s < nsrc; ++s) {
            size_t c = (size_t)src[2 * s + 1] * nx + src[2 * s];
            Q[c] -= wav[(size_t)s * nt + n] / (dx * dy);
        }
        for (int j = 1; j <= ny - 2; ++j)
            for (int i = 1; i <= nx - 2; ++i) {
                size_t c = (size_t)j * nx + i;
                Ez[c] = Ca[c] * Ez[c] + Cb[c] * Q[c];
            }
        /* 7. save the wavefield */
        if (q_hist) memcpy(q_hist + (size_t)n * N, Q, N * sizeof(double));
        if (ez_hist) memcpy(ez_hist + (size_t)(n + 1) * N, Ez, N * sizeof(double));
    }
    free(Ez); free(Hx); free(Hy); free(pEx); free(pEy); free(pHx); free(pHy);
    free(Ca); free(Cb); free(Q);
    or_axis_free(&ax); or_axis_free(&ay);
    return 0;
}

/* ---------------------------------------------------------------------------------------
 * Exact discrete adjoint of or_forward_shot for one shot (Algorithm 2), driven by the
 * trace residual resid [nt][nrec] (= dJ/dd for J of Eq. objective).  Needs ez_hist
 * (and q_hist for the coefficient form).  Outputs (each may be NULL; all are ADDED to):
 *   g_eps_r, g_sigma    zero-lag form, per unit relative permittivity and per S/m
 *   gc_eps_r, gc_sigma  coefficient form (needs q_hist)
 *   g_wav [nsrc][nt]    dJ/dw^n for each source waveform sample
 * -------------------------------------------------------------------------------------*/
int or_adjoint_shot(const or_grid* g, const double* eps_r, const double* sigma,
                    int nsrc, const int32_t* src, int nrec, const int32_t* rec,
                    const double* resid, const double* ez_hist, const double* q_hist,
                    double* g_eps_r, double* g_sigma, double* gc_eps_r, double* gc_sigma,
                    double* g_wav) {
    const int nx = g->nx, ny = g->ny, nt = g->nt;
    const size_t N = (size_t)nx * ny;
    const double dx = g->dx, dy = g->dy, dt = g->dt;
    const double Ch = dt / OR_MU0;
    or_axis ax, ay;
    if (or_axis_init(g, nx, dx, &ax) || or_axis_init(g, ny, dy, &ay)) return -1;
    /* adjoint state: aEz = adjoint of Ez^{n+1}, aHx/aHy of H^{n+1/2}, aP* of the CPML
     * memory variables after their step-n update */
    double *aEz = calloc(N, sizeof(double)), *aHx = calloc(N, sizeof(double)), *aHy = calloc(N, sizeof(double));
    double *aPEx = calloc(N, sizeof(double)), *aPEy = calloc(N, sizeof(double));
    double *aPHx = calloc(N, sizeof(double)), *aPHy = calloc(N, sizeof(double));
    double *Ca = calloc(N, sizeof(double)), *Cb = calloc(N, sizeof(double));
    if (!aEz || !aHx || !aHy || !aPEx || !aPEy || !aPHx || !aPHy || !Ca || !Cb) return -1;
    or_coefficients(g, eps_r, sigma, Ca, Cb);

    for (int n = nt - 1; n >= 0; --n) {
        const double* E1 = ez_hist + (size_t)(n + 1) * N; /* Ez^{n+1} */
        const double* E0 = ez_hist + (size_t)n * N;       /* Ez^n */
        /* 1. adjoint of the source injection: dJ/dw^n = -Cb(src) aEz(src) / (dx dy) */
        if (g_wav)
            for (int s = 0; s < nsrc; ++s) {
                size_t c = (size_t)src[2 * s + 1] * nx + src[2 * s];
                g_wav[(size_t)s * nt + n] += -Cb[c] * aEz[c] / (dx * dy);
            }
        /* 6. gradients of Ez^{n+1} = Ca Ez^n + Cb Q^n with respect to eps and sigma */
        for (int j = 1; j <= ny - 2; ++j)
            for (int i = 1; i <= nx - 2; ++i) {
                size_t c = (size_t)j * nx + i;
                if (Cb[c] == 0.0) continue; /* PEC cell: coefficients do not depend on the model */
                double eps = OR_EPS0 * eps_r[c];
                double a = sigma[c] * dt / (2.0 * eps);
                double lam = Cb[c] * aEz[c];
                if (g_eps_r) g_eps_r[c] += OR_EPS0 * (-lam * (E1[c] - E0[c]) / dt);
                if (g_sigma) g_sigma[c] += -lam * 0.5 * (E1[c] + E0[c]);
                if (q_hist && (gc_eps_r || gc_sigma)) {
                    double Qn = q_hist[(size_t)n * N + c];
                    double opa2 = (1.0 + a) * (1.0 + a);
                    double dCa_de = 2.0 * a / (eps * opa2);
                    double dCb_de = -dt / (eps * eps * opa2);
                    double dCa_ds = -dt / (eps * opa2);
                    double dCb_ds = -dt * dt / (2.0 * eps * eps * opa2);
                    if (gc_eps_r) gc_eps_r[c] += OR_EPS0 * aEz[c] * (dCa_de * E0[c] + dCb_de * Qn);
                    if (gc_sigma) gc_sigma[c] += aEz[c] * (dCa_ds * E0[c] + dCb_ds * Qn);
                }
            }
        /* 2-3. transpose of the E and electric-CPML update: the bracket Q receives
         * lam = Cb aEz; it reaches the CPML memories and, through the differences, H */
        for (int j = 1; j <= ny - 2; ++j)
            for (int i = 1; i <= nx - 2; ++i) {
                size_t c = (size_t)j * nx + i;
                double lam = Cb[c] * aEz[c];
                aPEx[c] += lam;
                aPEy[c] -= lam;
                double aDx = lam / ax.kE[i] + ax.cE[i] * aPEx[c];
                double aDy = -lam / ay.kE[j] + ay.cE[j] * aPEy[c];
                aPEx[c] *= ax.bE[i];
                aPEy[c] *= ay.bE[j];
                aHy[c] += aDx / dx;
                aHy[c - 1] -= aDx / dx;
                aHx[c] += aDy / dy;
                aHx[c - nx] -= aDy / dy;
                aEz[c] = Ca[c] * aEz[c];
            }
        /* 4-5. transpose of the H and magnetic-CPML update (H^{n+1/2} = H^{n-1/2} + ...):
         * aH carries over unchanged, the differences of Ez^n receive Ch aH */
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i <= nx - 2; ++i) {
                size_t c = (size_t)j * nx + i;
                aPHy[c] += Ch * aHy[c];
                double aD = Ch * aHy[c] / ax.kH[i] + ax.cH[i] * aPHy[c];
                aPHy[c] *= ax.bH[i];
                aEz[c + 1] += aD / dx;
                aEz[c] -= aD / dx;
            }
        for (int j = 0; j <= ny - 2; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = (size_t)j * nx + i;
                aPHx[c] -= Ch * aHx[c];
                double aD = -Ch * aHx[c] / ay.kH[j] + ay.cH[j] * aPHx[c];
                aPHx[c] *= ay.bH[j];
                aEz[c + nx] += aD / dy;
                aEz[c] -= aD / dy;
            }
        /* the PEC ring is not a state variable: its adjoint is dropped */
        for (int i = 0; i < nx; ++i) { aEz[i] = 0.0; aEz[(size_t)(ny - 1) * nx + i] = 0.0; }
        for (int j = 0; j < ny; ++j) { aEz[(size_t)j * nx] = 0.0; aEz[(size_t)j * nx + nx - 1] = 0.0; }
        /* adjoint source: transpose of "save receiver data" at step n (dJ/dd^n) */
        for (int r = 0; r < nrec; ++r)
            aEz[(size_t)rec[2 * r + 1] * nx + rec[2 * r]] += resid[(size_t)n * nrec + r];
    }
    free(aEz); free(aHx); free(aHy); free(aPEx); free(aPEy); free(aPHx); free(aPHy);
    free(Ca); free(Cb);
    or_axis_free(&ax); or_axis_free(&ay);
    return 0;
}

/* ---------------------------------------------------------------------------------------
 * Tangent-linear model of one shot: the derivative of the traces along the model
 * perturbation (d_eps_r, d_sigma), obtained by differentiating every forward step
 * (forward mode).  Used to pin the adjoint with the dot-product test.
 * -------------------------------------------------------------------------------------*/
int or_tangent_shot(const or_grid* g, const double* eps_r, const double* sigma,
                    const double* d_eps_r, const double* d_sigma,
                    int nsrc, const int32_t* src, const double* wav,
                    int nrec, const int32_t* rec, double* d_traces) {
    const int nx = g->nx, ny = g->ny, nt = g->nt;
    const size_t N = (size_t)nx * ny;
    const double dx = g->dx, dy = g->dy, dt = g->dt;
    const double Ch = dt / OR_MU0;
    or_axis ax, ay;
    if (or_axis_init(g, nx, dx, &ax) || or_axis_init(g, ny, dy, &ay)) return -1;
    double* buf = calloc(16 * N, sizeof(double));
    if (!buf) return -1;
    double *Ez = buf, *Hx = buf + N, *Hy = buf + 2 * N, *pEx = buf + 3 * N, *pEy = buf + 4 * N;
    double *pHx = buf + 5 * N, *pHy = buf + 6 * N, *Q = buf + 7 * N;
    double *tEz = buf + 8 * N, *tHx = buf + 9 * N, *tHy = buf + 10 * N, *tpEx = buf + 11 * N;
    double *tpEy = buf + 12 * N, *tpHx = buf + 13 * N, *tpHy = buf + 14 * N, *tQ = buf + 15 * N;
    double *Ca = calloc(N, sizeof(double)), *Cb = calloc(N, sizeof(double));
    double *tCa = calloc(N, sizeof(double)), *tCb = calloc(N, sizeof(double));
    if (!Ca || !Cb || !tCa || !tCb) return -1;
    or_coefficients(g, eps_r, sigma, Ca, Cb);
    for (size_t c = 0; c < N; ++c) {
        if (Cb[c] == 0.0) continue;
        double eps = OR_EPS0 * eps_r[c];
        double a = sigma[c] * dt / (2.0 * eps);
        double opa2 = (1.0 + a) * (1.0 + a);
        double de = OR_EPS0 * d_eps_r[c];
        tCa[c] = 2.0 * a / (eps * opa2) * de - dt / (eps * opa2) * d_sigma[c];
        tCb[c] = -dt / (eps * eps * opa2) * de - dt * dt / (2.0 * eps * eps * opa2) * d_sigma[c];
    }
    for (int n = 0; n < nt; ++n) {
        for (int r = 0; r < nrec; ++r)
            d_traces[(size_t)n * nrec + r] = tEz[(size_t)rec[2 * r + 1] * nx + rec[2 * r]];
        for (int j = 0; j <= ny - 2; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = (size_t)j * nx + i;
                double D = (Ez[c + nx] - Ez[c]) / dy, tD = (tEz[c + nx] - tEz[c]) / dy;
                pHx[c] = ay.bH[j] * pHx[c] + ay.cH[j] * D;
                tpHx[c] = ay.bH[j] * tpHx[c] + ay.cH[j] * tD;
                Hx[c] -= Ch * (D / ay.kH[j] + pHx[c]);
                tHx[c] -= Ch * (tD / ay.kH[j] + tpHx[c]);
            }
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i <= nx - 2; ++i) {
                size_t c = (size_t)j * nx + i;
                double D = (Ez[c + 1] - Ez[c]) / dx, tD = (tEz[c + 1] - tEz[c]) / dx;
                pHy[c] = ax.bH[i] * pHy[c] + ax.cH[i] * D;
                tpHy[c] = ax.bH[i] * tpHy[c] + ax.cH[i] * tD;
                Hy[c] += Ch * (D / ax.kH[i] + pHy[c]);
                tHy[c] += Ch * (tD / ax.kH[i] + tpHy[c]);
            }
        for (int j = 1; j <= ny - 2; ++j)
            for (int i = 1; i <= nx - 2; ++i) {
                size_t c = (size_t)j * nx + i;
                double Dx = (Hy[c] - Hy[c - 1]) / dx, Dy = (Hx[c] - Hx[c - nx]) / dy;
                double tDx = (tHy[c] - tHy[c - 1]) / dx, tDy = (tHx[c] - tHx[c - nx]) / dy;
                pEx[c] = ax.bE[i] * pEx[c] + ax.cE[i] * Dx;
                pEy[c] = ay.bE[j] * pEy[c] + ay.cE[j] * Dy;
                tpEx[c] = ax.bE[i] * tpEx[c] + ax.cE[i] * tDx;
                tpEy[c] = ay.bE[j] * tpEy[c] + ay.cE[j] * tDy;
                Q[c] = Dx / ax.kE[i] + pEx[c] - Dy / ay.kE[j] - pEy[c];
                tQ[c] = tDx / ax.kE[i] + tpEx[c] - tDy / ay.kE[j] - tpEy[c];
            }
        for (int s = 0; s < nsrc; ++s) {
            size_t c = (size_t)src[2 * s + 1] * nx + src[2 * s];
            Q[c] -= wav[(size_t)s * nt + n] / (dx * dy);
        }
        for (int j = 1; j <= ny - 2; ++j)
            for (int i = 1; i <= nx - 2; ++i) {
                size_t c = (size_t)j * nx + i;
                /* product rule on Ez^{n+1} = Ca Ez^n + Cb Q^n (tEz uses the old Ez) */
                tEz[c] = tCa[c] * Ez[c] + Ca[c] * tEz[c] + tCb[c] * Q[c] + Cb[c] * tQ[c];
                Ez[c] = Ca[c] * Ez[c] + Cb[c] * Q[c];
            }
    }
    free(buf); free(Ca); free(Cb); free(tCa); free(tCb);
    or_axis_free(&ax); or_axis_free(&ay);
    return 0;
}

/* ---------------------------------------------------------------------------------------
 * Multi-shot drivers.  Layouts: src [nshots][nsrc][2], rec [nshots][nrec][2] (cell indices
 * i, j), wav [nshots][nsrc][nt], traces / observed [nshots][nt][nrec].
 * -------------------------------------------------------------------------------------*/
int or_forward(const or_grid* g, const double* eps_r, const double* sigma,
               int nshots, int nsrc, const int32_t* src, const double* wav,
               int nrec, const int32_t* rec, double* traces, int nthreads) {
    int err = 0;
    (void)nthreads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1) reduction(| : err)
    for (int s = 0; s < nshots; ++s)
        err |= or_forward_shot(g, eps_r, sigma, nsrc, src + (size_t)s * nsrc * 2,
                               wav + (size_t)s * nsrc * g->nt, nrec, rec + (size_t)s * nrec * 2,
                               traces + (size_t)s * g->nt * nrec, NULL, NULL, NULL, NULL);
    return err ? -1 : 0;
}

/* Misfit J = 1/2 sum (d - o)^2 over all shots and the summed zero-lag gradients. */
int or_misfit_gradient(const or_grid* g, const double* eps_r, const double* sigma,
                       int nshots, int nsrc, const int32_t* src, const double* wav,
                       int nrec, const int32_t* rec, const double* observed,
                       double* misfit, double* g_eps_r, double* g_sigma,
                       double* traces_out, int nthreads) {
    const size_t N = (size_t)g->nx * g->ny;
    const int nt = g->nt;
    double* ge = calloc((size_t)nshots * N, sizeof(double));
    double* gs = calloc((size_t)nshots * N, sizeof(double));
    double* Js = calloc((size_t)nshots, sizeof(double));
    if (!ge || !gs || !Js) return -1;
    int err = 0;
    (void)nthreads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1) reduction(| : err)
    for (int s = 0; s < nshots; ++s) {
        double* hist = malloc((size_t)(nt + 1) * N * sizeof(double));
        double* tr = malloc((size_t)nt * nrec * sizeof(double));
        double* res = malloc((size_t)nt * nrec * sizeof(double));
        if (!hist || !tr || !res) { err |= 1; free(hist); free(tr); free(res); continue; }
        const int32_t* ss = src + (size_t)s * nsrc * 2;
        const int32_t* rr = rec + (size_t)s * nrec * 2;
        err |= or_forward_shot(g, eps_r, sigma, nsrc, ss, wav + (size_t)s * nsrc * nt, nrec, rr,
                               tr, NULL, hist, NULL, NULL);
        double J = 0.0;
        for (size_t k = 0; k < (size_t)nt * nrec; ++k) {
            res[k] = tr[k] - observed[(size_t)s * nt * nrec + k];
            J += 0.5 * res[k] * res[k];
        }
        Js[s] = J;
        if (traces_out) memcpy(traces_out + (size_t)s * nt * nrec, tr, (size_t)nt * nrec * sizeof(double));
        err |= or_adjoint_shot(g, eps_r, sigma, nsrc, ss, nrec, rr, res, hist, NULL,
                               ge + (size_t)s * N, gs + (size_t)s * N, NULL, NULL, NULL);
        free(hist); free(tr); free(res);
    }
    double J = 0.0;
    memset(g_eps_r, 0, N * sizeof(double));
    memset(g_sigma, 0, N * sizeof(double));
    for (int s = 0; s < nshots; ++s) {
        J += Js[s];
        for (size_t c = 0; c < N; ++c) {
            g_eps_r[c] += ge[(size_t)s * N + c];
            g_sigma[c] += gs[(size_t)s * N + c];
        }
    }
    *misfit = J;
    free(ge); free(gs); free(Js);
    return err ? -1 : 0;
}

/* ---------------------------------------------------------------------------------------
 * TE-mode forward model of one shot: the fields an x- or y-polarised hertzian line source
 * excites (Sec. 3.2 source listing, polarisation 0 / 1; in 2-D they drive Ex, Ey, Hz,
 * the dual of the TM mode above).
 *   fields  Hz(i,j) at (i+1/2, j+1/2), Ex(i,j) at (i+1/2, j), Ey(i,j) at (i, j+1/2).
 *   Faraday:  mu0 dHz/dt = dEx/dy - dEy/dx
 *   Ampere:   eps dEx/dt + sigma Ex = dHz/dy - Jx,  eps dEy/dt + sigma Ey = -dHz/dx - Jy
 *   Each E component takes Ca, Cb of the cell whose index it carries (the coefficient
 *   listing evaluates every component's coefficients from the material at that index).
 *   PEC walls on the outermost nodes: Ex is held at zero on rows j = 0 and j = ny-1, Ey on
 *   columns i = 0 and i = nx-1 (their tangential components); Hz is updated for
 *   0 <= i <= nx-2, 0 <= j <= ny-2; Ex for 0 <= i <= nx-2, 1 <= j <= ny-2; Ey for
 *   1 <= i <= nx-2, 0 <= j <= ny-2.  PEC cells (sigma > 100 S/m) hold their E at zero.
 *   CPML: the same profiles as the TM model; Hz's x difference sits on half-integer x
 *   nodes (H profile), its y difference on half-integer y nodes; Ex's y difference of Hz on
 *   integer y nodes (E profile), Ey's x difference on integer x nodes.
 *   One step n: record Ex^n, Ey^n, Hz^{n-1/2} at the receiver cells; Hz update; E update;
 *   the source enters the bracket of its component: Q(src) -= w^n / (dx dy).
 * Outputs (each may be NULL):
 *   traces [nt][nrec][3]   Ex^n, Ey^n, Hz^{n-1/2} at each receiver cell's nodes
 *   energy [nt]            dx dy sum(eps (Ex^n^2 + Ey^n^2) + mu0 Hz^{n-1/2} Hz^{n+1/2}),
 *                          conserved by the lossless scheme
 *   ex_hist, ey_hist [(nt+1)][ny*nx]   Ex^0 .. Ex^nt and Ey^0 .. Ey^nt (for the adjoint)
 * -------------------------------------------------------------------------------------*/
int or_forward_te_shot(const or_grid* g, const double* eps_r, const double* sigma, int pol,
                       int nsrc, const int32_t* src, const double* wav,
                       int nrec, const int32_t* rec, double* traces, double* energy,
                       double* ex_hist, double* ey_hist) {
    const int nx = g->nx, ny = g->ny, nt = g->nt;
    const size_t N = (size_t)nx * ny;
    const double dx = g->dx, dy = g->dy, dt = g->dt;
    const double Ch = dt / OR_MU0;
    if (pol != 0 && pol != 1) return -2;
    or_axis ax, ay;
    if (or_axis_init(g, nx, dx, &ax) || or_axis_init(g, ny, dy, &ay)) return -1;
    double *Ex = calloc(N, sizeof(double)), *Ey = calloc(N, sizeof(double)), *Hz = calloc(N, sizeof(double));
    double *pHzx = calloc(N, sizeof(double)), *pHzy = calloc(N, sizeof(double));
    double *pExy = calloc(N, sizeof(double)), *pEyx = calloc(N, sizeof(double));
    double *Ca = calloc(N, sizeof(double)), *Cb = calloc(N, sizeof(double));
    double *Qx = calloc(N, sizeof(double)), *Qy = calloc(N, sizeof(double));
    if (!Ex || !Ey || !Hz || !pHzx || !pHzy || !pExy || !pEyx || !Ca || !Cb || !Qx || !Qy)
        return -1;
    /* per-cell coefficients without the ring rule (the walls are handled by the loop
     * bounds below) */
    for (size_t c = 0; c < N; ++c) {
        if (sigma[c] > 100.0) { Ca[c] = 0.0; Cb[c] = 0.0; continue; }
        double EA = OR_EPS0 * eps_r[c] / dt + 0.5 * sigma[c];
        double EB = OR_EPS0 * eps_r[c] / dt - 0.5 * sigma[c];
        Ca[c] = EB / EA;
        Cb[c] = 1.0 / EA;
    }
    if (ex_hist) memset(ex_hist, 0, N * sizeof(double));
    if (ey_hist) memset(ey_hist, 0, N * sizeof(double));
    for (int n = 0; n < nt; ++n) {
        if (traces)
            for (int r = 0; r < nrec; ++r) {
                const size_t c = (size_t)rec[2 * r + 1] * nx + rec[2 * r];
                traces[((size_t)n * nrec + r) * 3 + 0] = Ex[c];
                traces[((size_t)n * nrec + r) * 3 + 1] = Ey[c];
                traces[((size_t)n * nrec + r) * 3 + 2] = Hz[c];
            }
        double wsum = 0.0;
        if (energy)
            for (size_t c = 0; c < N; ++c)
                wsum += OR_EPS0 * eps_r[c] * (Ex[c] * Ex[c] + Ey[c] * Ey[c]);
        /* magnetic field and its CPML memory */
        for (int j = 0; j <= ny - 2; ++j)
            for (int i = 0; i <= nx - 2; ++i) {
                size_t c = (size_t)j * nx + i;
                double Dy = (Ex[c + nx] - Ex[c]) / dy;
                double Dx = (Ey[c + 1] - Ey[c]) / dx;
                pHzy[c] = ay.bH[j] * pHzy[c] + ay.cH[j] * Dy;
                pHzx[c] = ax.bH[i] * pHzx[c] + ax.cH[i] * Dx;
                double old = Hz[c];
                Hz[c] = old + Ch * (Dy / ay.kH[j] + pHzy[c] - Dx / ax.kH[i] - pHzx[c]);
                if (energy) wsum += OR_MU0 * old * Hz[c];
            }
        if (energy) energy[n] = wsum * dx * dy;
        /* electric brackets and their CPML memory */
        for (int j = 1; j <= ny - 2; ++j)
            for (int i = 0; i <= nx - 2; ++i) {
                size_t c = (size_t)j * nx + i;
                double D = (Hz[c] - Hz[c - nx]) / dy;
                pExy[c] = ay.bE[j] * pExy[c] + ay.cE[j] * D;
                Qx[c] = D / ay.kE[j] + pExy[c];
            }
        for (int j = 0; j <= ny - 2; ++j)
            for (int i = 1; i <= nx - 2; ++i) {
                size_t c = (size_t)j * nx + i;
                double D = (Hz[c] - Hz[c - 1]) / dx;
                pEyx[c] = ax.bE[i] * pEyx[c] + ax.cE[i] * D;
                Qy[c] = -(D / ax.kE[i] + pEyx[c]);
            }
        /* the source current enters the bracket of its component */
        for (int s = 0; s < nsrc; ++s) {
            size_t c = (size_t)src[2 * s + 1] * nx + src[2 * s];
            double* Q = pol == 0 ? Qx : Qy;
            Q[c] -= wav[(size_t)s * nt + n] / (dx * dy);
        }
        for (int j = 1; j <= ny - 2; ++j)
            for (int i = 0; i <= nx - 2; ++i) {
                size_t c = (size_t)j * nx + i;
                Ex[c] = Ca[c] * Ex[c] + Cb[c] * Qx[c];
            }
        for (int j = 0; j <= ny - 2; ++j)
            for (int i = 1; i <= nx - 2; ++i) {
                size_t c = (size_t)j * nx + i;
                Ey[c] = Ca[c] * Ey[c] + Cb[c] * Qy[c];
            }
        if (ex_hist) memcpy(ex_hist + (size_t)(n + 1) * N, Ex, N * sizeof(double));
        if (ey_hist) memcpy(ey_hist + (size_t)(n + 1) * N, Ey, N * sizeof(double));
    }
    free(Ex); free(Ey); free(Hz); free(pHzx); free(pHzy); free(pExy); free(pEyx);
    free(Ca); free(Cb); free(Qx); free(Qy);
    or_axis_free(&ax); or_axis_free(&ay);
    return 0;
}

/* ---------------------------------------------------------------------------------------
 * Exact discrete adjoint of or_forward_te_shot for one shot, driven by the residual of the
 * source's own component: resid [nt][nrec] = dJ/d(E_pol^n at receiver r) (Ex for
 * polarisation 0, Ey for 1).  Needs ex_hist and ey_hist.  Every forward operation is
 * transposed in reverse order: for n = nt-1 .. 0, the E updates (with their CPML memories),
 * then the Hz update (with its memories), then the recording of step n.  Adjoint fields
 * aEx, aEy hold dJ/dE^{n+1} on entry to step n's reversal and dJ/dE^n after it; aHz holds
 * dJ/dHz^{n+1/2}, then dJ/dHz^{n-1/2}.  The CPML memories' adjoints follow the recursion
 * backwards: A_n = b A_{n+1} + (cotangent of the bracket that uses the memory of step n).
 * Gradients (ADDED to g_eps_r, per unit relative permittivity, and g_sigma, per S/m), the
 * zero-lag form of both E components of each cell, lam = Cb aE^{n+1}:
 *   dJ/deps_r += -sum_n lam (E^{n+1} - E^n) eps0 / dt,  dJ/dsigma += -sum_n lam (E^{n+1} + E^n) / 2
 * (the derivative of the update's residual EA E^{n+1} - EB E^n - Q).
 * -------------------------------------------------------------------------------------*/
int or_adjoint_te_shot(const or_grid* g, const double* eps_r, const double* sigma, int pol,
                       int nrec, const int32_t* rec, const double* resid,
                       const double* ex_hist, const double* ey_hist,
                       double* g_eps_r, double* g_sigma) {
    const int nx = g->nx, ny = g->ny, nt = g->nt;
    const size_t N = (size_t)nx * ny;
    const double dx = g->dx, dy = g->dy, dt = g->dt;
    const double Ch = dt / OR_MU0;
    if (pol != 0 && pol != 1) return -2;
    or_axis ax, ay;
    if (or_axis_init(g, nx, dx, &ax) || or_axis_init(g, ny, dy, &ay)) return -1;
    double *aEx = calloc(N, sizeof(double)), *aEy = calloc(N, sizeof(double)), *aHz = calloc(N, sizeof(double));
    double *aPExy = calloc(N, sizeof(double)), *aPEyx = calloc(N, sizeof(double));
    double *aPHzx = calloc(N, sizeof(double)), *aPHzy = calloc(N, sizeof(double));
    double *Ca = calloc(N, sizeof(double)), *Cb = calloc(N, sizeof(double));
    if (!aEx || !aEy || !aHz || !aPExy || !aPEyx || !aPHzx || !aPHzy || !Ca || !Cb) return -1;
    for (size_t c = 0; c < N; ++c) {
        if (sigma[c] > 100.0) { Ca[c] = 0.0; Cb[c] = 0.0; continue; }
        double EA = OR_EPS0 * eps_r[c] / dt + 0.5 * sigma[c];
        double EB = OR_EPS0 * eps_r[c] / dt - 0.5 * sigma[c];
        Ca[c] = EB / EA;
        Cb[c] = 1.0 / EA;
    }
    for (int n = nt - 1; n >= 0; --n) {
        const double *X1 = ex_hist + (size_t)(n + 1) * N, *X0 = ex_hist + (size_t)n * N;
        const double *Y1 = ey_hist + (size_t)(n + 1) * N, *Y0 = ey_hist + (size_t)n * N;
        /* E updates of step n, reversed (Ex: rows 1..ny-2, columns 0..nx-2) */
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = (size_t)j * nx + i;
                if (j < 1 || j > ny - 2 || i > nx - 2) { aEx[c] = 0.0; continue; } /* held */
                double ae = aEx[c];
                double lam = Cb[c] * ae;
                if (g_eps_r) g_eps_r[c] += -lam * (X1[c] - X0[c]) * OR_EPS0 / dt;
                if (g_sigma) g_sigma[c] += -lam * 0.5 * (X1[c] + X0[c]);
                /* Qx = D / k + psi, psi = b psi_prev + c D, D = (Hz[c] - Hz[c-nx]) / dy */
                aPExy[c] = ay.bE[j] * aPExy[c] + lam;
                double aD = ay.cE[j] * aPExy[c] + lam / ay.kE[j];
                aHz[c] += aD / dy;
                aHz[c - nx] -= aD / dy;
                aEx[c] = Ca[c] * ae;
            }
        /* Ey: rows 0..ny-2, columns 1..nx-2; Qy = -(D / k + psi), D = (Hz[c] - Hz[c-1]) / dx */
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = (size_t)j * nx + i;
                if (j > ny - 2 || i < 1 || i > nx - 2) { aEy[c] = 0.0; continue; }
                double ae = aEy[c];
                double lam = Cb[c] * ae;
                if (g_eps_r) g_eps_r[c] += -lam * (Y1[c] - Y0[c]) * OR_EPS0 / dt;
                if (g_sigma) g_sigma[c] += -lam * 0.5 * (Y1[c] + Y0[c]);
                aPEyx[c] = ax.bE[i] * aPEyx[c] - lam;
                double aD = ax.cE[i] * aPEyx[c] - lam / ax.kE[i];
                aHz[c] += aD / dx;
                aHz[c - 1] -= aD / dx;
                aEy[c] = Ca[c] * ae;
            }
        /* Hz update of step n, reversed: Hz^{n+1/2} = Hz^{n-1/2} + Ch (Dy / ky + psi_y
         * - Dx / kx - psi_x), Dy = (Ex[c+nx] - Ex[c]) / dy, Dx = (Ey[c+1] - Ey[c]) / dx */
        for (int j = 0; j <= ny - 2; ++j)
            for (int i = 0; i <= nx - 2; ++i) {
                size_t c = (size_t)j * nx + i;
                double ah = Ch * aHz[c];
                aPHzy[c] = ay.bH[j] * aPHzy[c] + ah;
                double aDy = ay.cH[j] * aPHzy[c] + ah / ay.kH[j];
                aPHzx[c] = ax.bH[i] * aPHzx[c] - ah;
                double aDx = ax.cH[i] * aPHzx[c] - ah / ax.kH[i];
                aEx[c + nx] += aDy / dy;
                aEx[c] -= aDy / dy;
                aEy[c + 1] += aDx / dx;
                aEy[c] -= aDx / dx;
            }
        /* recording of step n: d^n = E_pol^n at the receivers */
        double* aE = pol == 0 ? aEx : aEy;
        for (int r = 0; r < nrec; ++r)
            aE[(size_t)rec[2 * r + 1] * nx + rec[2 * r]] += resid[(size_t)n * nrec + r];
    }
    free(aEx); free(aEy); free(aHz); free(aPExy); free(aPEyx); free(aPHzx); free(aPHzy);
    free(Ca); free(Cb);
    or_axis_free(&ax); or_axis_free(&ay);
    return 0;
}
