/*
 * Oracle: plain FP64 loops for the stencil sweeps (test infrastructure).
 *
 * This file is the slow, obviously-correct CPU definition that the CUDA
 * library is checked against.  It is NOT part of the product: only tests/,
 * the smoke check and the CPU-baseline leg of the benchmark load it.  It
 * shares no code with the CUDA path.
 *
 * What it computes (paper, Section 2 and Section 5.1):
 *  - a grid point at time n+1 is a function of its neighbours at earlier
 *    times; the halo ("ghost") region is read-only and as wide as the stencil
 *    radius r (Section 2, the 1D 3-point Jacobi description);
 *  - heat diffusion u_t = alpha * Laplacian(u), solved for u.forward with
 *    forward Euler (the Devito listing in Section 5.1):
 *        u^{n+1}_p = u^n_p + a * L(u^n)_p,   a = alpha dt / h^2;
 *  - the isotropic acoustic wave equation, second order in time
 *    (Section 6.1), leapfrog with three time levels:
 *        u^{n+1}_p = 2 u^n_p - u^{n-1}_p + kappa_p * L(u^n)_p,
 *        kappa_p = c_p^2 dt^2 / h^2;
 *  - L is the star stencil  L(u)_p = sum_axes sum_{m=-r..r} w_|m| u_{p+m e};
 *  - a Ricker point source is added to u^{n+1} at the end of step n.
 *
 * Layout: every field is a padded array with r ghost cells on both sides of
 * every stencil axis (2D grids have nz = 1 and no z ghosts), x fastest:
 *   index(i,j,k) = ((k+rz)*(ny+2r) + (j+r))*(nx+2r) + (i+r),  i in [-r, nx+r).
 * Ghost cells hold zero (Dirichlet, the paper's read-only halo) or, for the
 * periodic test mode, copies of the opposite interior faces.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t nx, ny, nz;  /* interior sizes */
    int64_t r, rz;       /* ghost width on x/y and on z (0 for 2D) */
    int64_t px, py, pz;  /* padded sizes */
} lay_t;

static lay_t mk_layout(int ndim, const int64_t n[3], int r)
{
    lay_t L;
    L.nx = n[0];
    L.ny = n[1];
    L.nz = ndim == 3 ? n[2] : 1;
    L.r = r;
    L.rz = ndim == 3 ? r : 0;
    L.px = L.nx + 2 * r;
    L.py = L.ny + 2 * r;
    L.pz = L.nz + 2 * L.rz;
    return L;
}

static inline int64_t at(const lay_t *L, int64_t i, int64_t j, int64_t k)
{
    return ((k + L->rz) * L->py + (j + L->r)) * L->px + (i + L->r);
}

int64_t orc_padded_size(int ndim, const int64_t n[3], int r)
{
    lay_t L = mk_layout(ndim, n, r);
    return L.px * L.py * L.pz;
}

/* Ghost cells: bc 0 = zero (Dirichlet), bc 1 = periodic faces. */
void orc_fill_ghosts(int ndim, const int64_t n[3], int r, int bc, double *u)
{
    lay_t L = mk_layout(ndim, n, r);
    int64_t i, j, k, g;
    if (bc == 0) {
        for (k = -L.rz; k < L.nz + L.rz; k++)
            for (j = -L.r; j < L.ny + L.r; j++)
                for (i = -L.r; i < L.nx + L.r; i++) {
                    int inside = i >= 0 && i < L.nx && j >= 0 && j < L.ny && k >= 0 && k < L.nz;
                    if (!inside)
                        u[at(&L, i, j, k)] = 0.0;
                }
        return;
    }
    /* periodic: each face ghost slab is the opposite interior slab */
    for (k = 0; k < L.nz; k++)
        for (j = 0; j < L.ny; j++)
            for (g = 1; g <= L.r; g++) {
                u[at(&L, -g, j, k)] = u[at(&L, L.nx - g, j, k)];
                u[at(&L, L.nx - 1 + g, j, k)] = u[at(&L, g - 1, j, k)];
            }
    for (k = 0; k < L.nz; k++)
        for (i = 0; i < L.nx; i++)
            for (g = 1; g <= L.r; g++) {
                u[at(&L, i, -g, k)] = u[at(&L, i, L.ny - g, k)];
                u[at(&L, i, L.ny - 1 + g, k)] = u[at(&L, i, g - 1, k)];
            }
    if (ndim == 3)
        for (j = 0; j < L.ny; j++)
            for (i = 0; i < L.nx; i++)
                for (g = 1; g <= L.r; g++) {
                    u[at(&L, i, j, -g)] = u[at(&L, i, j, L.nz - g)];
                    u[at(&L, i, j, L.nz - 1 + g)] = u[at(&L, i, j, g - 1)];
                }
}

/* L(u)_p = sum over axes, sum over m = -r..r of w_|m| u_{p + m e_axis} */
static inline double star(const lay_t *L, int ndim, const double *w, const double *u,
                          int64_t i, int64_t j, int64_t k)
{
    double s = 0.0;
    int64_t m;
    int r = (int)L->r;
    for (m = -r; m <= r; m++)
        s += w[m < 0 ? -m : m] * u[at(L, i + m, j, k)];
    for (m = -r; m <= r; m++)
        s += w[m < 0 ? -m : m] * u[at(L, i, j + m, k)];
    if (ndim == 3)
        for (m = -r; m <= r; m++)
            s += w[m < 0 ? -m : m] * u[at(L, i, j, k + m)];
    return s;
}

/* One forward-Euler heat step over the interior: out = u + a * L(u). */
void orc_sweep_heat(int ndim, const int64_t n[3], int r, const double *w, double a,
                    const double *u, double *out)
{
    lay_t L = mk_layout(ndim, n, r);
    int64_t k;
#pragma omp parallel for schedule(static)
    for (k = 0; k < L.nz; k++) {
        int64_t i, j;
        for (j = 0; j < L.ny; j++)
            for (i = 0; i < L.nx; i++) {
                int64_t p = at(&L, i, j, k);
                out[p] = u[p] + a * star(&L, ndim, w, u, i, j, k);
            }
    }
}

/* One leapfrog wave step: out = 2u - uprev + kappa * L(u); kappa is dense (interior only). */
void orc_sweep_wave(int ndim, const int64_t n[3], int r, const double *w, const double *kappa,
                    const double *u, const double *uprev, double *out)
{
    lay_t L = mk_layout(ndim, n, r);
    int64_t k;
#pragma omp parallel for schedule(static)
    for (k = 0; k < L.nz; k++) {
        int64_t i, j;
        for (j = 0; j < L.ny; j++)
            for (i = 0; i < L.nx; i++) {
                int64_t p = at(&L, i, j, k);
                double kap = kappa[(k * L.ny + j) * L.nx + i];
                out[p] = 2.0 * u[p] - uprev[p] + kap * star(&L, ndim, w, u, i, j, k);
            }
    }
}

/* Ricker wavelet R(t) = (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2). */
double orc_ricker(double t, double f0, double t0)
{
    const double pi = 3.14159265358979323846;
    double a = pi * f0 * (t - t0);
    a = a * a;
    return (1.0 - 2.0 * a) * exp(-a);
}

static void dense_to_padded(const lay_t *L, const double *d, double *p)
{
    int64_t i, j, k;
    for (k = 0; k < L->nz; k++)
        for (j = 0; j < L->ny; j++)
            for (i = 0; i < L->nx; i++)
                p[at(L, i, j, k)] = d[(k * L->ny + j) * L->nx + i];
}

static void padded_to_dense(const lay_t *L, const double *p, double *d)
{
    int64_t i, j, k;
    for (k = 0; k < L->nz; k++)
        for (j = 0; j < L->ny; j++)
            for (i = 0; i < L->nx; i++)
                d[(k * L->ny + j) * L->nx + i] = p[at(L, i, j, k)];
}

/* nsteps heat steps on a dense interior field u (in place).  Returns 0 or -2 (no memory). */
int orc_heat_run(int ndim, const int64_t n[3], int r, const double *w, double a, int bc,
                 double *u, int64_t nsteps)
{
    lay_t L = mk_layout(ndim, n, r);
    int64_t sz = L.px * L.py * L.pz, s;
    double *A = calloc((size_t)sz, sizeof(double));
    double *B = calloc((size_t)sz, sizeof(double));
    if (!A || !B) {
        free(A);
        free(B);
        return -2;
    }
    dense_to_padded(&L, u, A);
    for (s = 0; s < nsteps; s++) {
        double *t;
        orc_fill_ghosts(ndim, n, r, bc, A);
        orc_sweep_heat(ndim, n, r, w, a, A, B);
        t = A;
        A = B;
        B = t;
    }
    padded_to_dense(&L, A, u);
    free(A);
    free(B);
    return 0;
}

/*
 * nsteps steps of a coupled system of nf fields (several stencils in one sweep,
 * a synthetic multi-field workload): for every field k,
 *     u_k^{n+1} = u_k^n + sum_j A[k][j] L(u_j^n)
 * with A an nf x nf matrix (row-major).  A = a I is nf independent heat
 * equations.  u holds the nf dense fields one after another.
 */
int orc_system_run(int ndim, const int64_t n[3], int r, const double *w, int nf, const double *A, int bc,
                   double *u, int64_t nsteps)
{
    lay_t L = mk_layout(ndim, n, r);
    int64_t sz = L.px * L.py * L.pz, s, dn = L.nx * L.ny * L.nz;
    int f;
    double *X = calloc((size_t)(sz * nf), sizeof(double));
    double *Y = calloc((size_t)(sz * nf), sizeof(double));
    if (!X || !Y) {
        free(X);
        free(Y);
        return -2;
    }
    for (f = 0; f < nf; f++)
        dense_to_padded(&L, u + f * dn, X + f * sz);
    for (s = 0; s < nsteps; s++) {
        double *t;
        int64_t k;
        for (f = 0; f < nf; f++)
            orc_fill_ghosts(ndim, n, r, bc, X + f * sz);
#pragma omp parallel for schedule(static)
        for (k = 0; k < L.nz; k++) {
            int64_t i, j;
            double lap[16];
            for (j = 0; j < L.ny; j++)
                for (i = 0; i < L.nx; i++) {
                    int64_t p = at(&L, i, j, k);
                    int a, b;
                    for (b = 0; b < nf; b++)
                        lap[b] = star(&L, ndim, w, X + b * sz, i, j, k);
                    for (a = 0; a < nf; a++) {
                        double acc = 0.0;
                        for (b = 0; b < nf; b++)
                            acc += A[a * nf + b] * lap[b];
                        Y[a * sz + p] = X[a * sz + p] + acc;
                    }
                }
        }
        t = X;
        X = Y;
        Y = t;
    }
    for (f = 0; f < nf; f++)
        padded_to_dense(&L, X + f * sz, u + f * dn);
    free(X);
    free(Y);
    return 0;
}

/*
 * nsteps wave steps.  uprev = u^{n-1}, u = u^n on entry (dense), u^{n-1+s}, u^{n+s} on exit.
 * step0 is the global index n of the first step (the source time is t_n = n dt).
 * src == NULL: no source; else the value amp * kappa_s * h^2 * R(t_n) = amp c_s^2 dt^2 R(t_n)
 * is added to u^{n+1} at src = (i, j, k) after the stencil update.
 */
int orc_wave_run(int ndim, const int64_t n[3], int r, const double *w, int bc,
                 const double *kappa, double *uprev, double *u, int64_t nsteps, int64_t step0,
                 const int64_t *src, double f0, double t0, double amp, double dt, double h)
{
    lay_t L = mk_layout(ndim, n, r);
    int64_t sz = L.px * L.py * L.pz, s;
    double *P = calloc((size_t)sz, sizeof(double));
    double *C = calloc((size_t)sz, sizeof(double));
    double *N = calloc((size_t)sz, sizeof(double));
    if (!P || !C || !N) {
        free(P);
        free(C);
        free(N);
        return -2;
    }
    dense_to_padded(&L, uprev, P);
    dense_to_padded(&L, u, C);
    for (s = 0; s < nsteps; s++) {
        double *t;
        orc_fill_ghosts(ndim, n, r, bc, C);
        orc_sweep_wave(ndim, n, r, w, kappa, C, P, N);
        if (src) {
            int64_t sk = ndim == 3 ? src[2] : 0;
            double ks = kappa[(sk * L.ny + src[1]) * L.nx + src[0]];
            double tn = (double)(step0 + s) * dt;
            N[at(&L, src[0], src[1], sk)] += amp * ks * h * h * orc_ricker(tn, f0, t0);
        }
        t = P;
        P = C;
        C = N;
        N = t;
    }
    padded_to_dense(&L, P, uprev);
    padded_to_dense(&L, C, u);
    free(P);
    free(C);
    free(N);
    return 0;
}

/*
 * Adjoint (transpose) of one source-free leapfrog step, dense inputs, zero ghosts.
 * The step maps (u^n, u^{n-1}) to (u^{n+1}, u^n) with
 *     u^{n+1} = 2 u^n - u^{n-1} + K L u^n,   K = diag(kappa),
 * a linear map whose transpose takes cotangents (lam^{n+1}, lam^n) to
 *     lam^n'     = lam^n + 2 lam^{n+1} + L (K lam^{n+1})     (L is symmetric)
 *     lam^{n-1}' = -lam^{n+1}.
 * lam_cur holds lam^n on entry and lam^n' on exit; lam_prev receives lam^{n-1}'.
 * Used to train a closure through whole coarse-grid rollouts (backpropagation
 * through the time steps of Section 6.1's scheme).
 */
int orc_wave_adjoint(int ndim, const int64_t n[3], int r, const double *w, const double *kappa,
                     const double *lam_next, double *lam_cur, double *lam_prev)
{
    lay_t L = mk_layout(ndim, n, r);
    int64_t sz = L.px * L.py * L.pz, dn = L.nx * L.ny * L.nz, d;
    double *P = calloc((size_t)sz, sizeof(double));
    if (!P)
        return -2;
    /* K lam^{n+1} on a padded array with zero ghosts */
    {
        int64_t i, j, k;
        for (k = 0; k < L.nz; k++)
            for (j = 0; j < L.ny; j++)
                for (i = 0; i < L.nx; i++) {
                    d = (k * L.ny + j) * L.nx + i;
                    P[at(&L, i, j, k)] = kappa[d] * lam_next[d];
                }
    }
    {
        int64_t k;
#pragma omp parallel for schedule(static)
        for (k = 0; k < L.nz; k++) {
            int64_t i, j, dd;
            for (j = 0; j < L.ny; j++)
                for (i = 0; i < L.nx; i++) {
                    dd = (k * L.ny + j) * L.nx + i;
                    lam_cur[dd] += 2.0 * lam_next[dd] + star(&L, ndim, w, P, i, j, k);
                }
        }
    }
    for (d = 0; d < dn; d++)
        lam_prev[d] = -lam_next[d];
    free(P);
    return 0;
}

/*
 * Discrete leapfrog energy between levels u^{n-1} (uprev) and u^n (u), dense inputs:
 *   E = sum_p (u_p - uprev_p)^2 / kappa_p + sum_p u_p (A uprev)_p,   A = -L,
 * with the ghosts of uprev given by bc.  For the source-free scheme this is
 * conserved exactly (up to rounding) from step to step.
 */
int orc_energy(int ndim, const int64_t n[3], int r, const double *w, int bc, const double *kappa,
               const double *u, const double *uprev, double *out)
{
    lay_t L = mk_layout(ndim, n, r);
    int64_t sz = L.px * L.py * L.pz, i, j, k;
    double e = 0.0;
    double *P = calloc((size_t)sz, sizeof(double));
    if (!P)
        return -2;
    dense_to_padded(&L, uprev, P);
    orc_fill_ghosts(ndim, n, r, bc, P);
    for (k = 0; k < L.nz; k++)
        for (j = 0; j < L.ny; j++)
            for (i = 0; i < L.nx; i++) {
                int64_t d = (k * L.ny + j) * L.nx + i;
                double v = u[d] - uprev[d];
                e += v * v / kappa[d];
                e += u[d] * (-star(&L, ndim, w, P, i, j, k));
            }
    free(P);
    *out = e;
    return 0;
}

/* ------------------------------------------------------------------------
 * 3x3x3 convolution with zero padding (cross-correlation), FP64.
 * x[ci][z][y][x], wt[co][ci][dz][dy][dx] (taps index offset+1), y[co][z][y][x].
 * ---------------------------------------------------------------------- */
static inline int inb(int64_t v, int64_t n) { return v >= 0 && v < n; }

void orc_conv3d_fwd(int cin, int cout, const int64_t n[3], const double *x, const double *wt,
                    const double *b, double *y)
{
    int64_t nx = n[0], ny = n[1], nz = n[2], N = nx * ny * nz;
    int co;
#pragma omp parallel for schedule(static)
    for (co = 0; co < cout; co++) {
        int64_t i, j, k;
        int ci, dz, dy, dx;
        for (k = 0; k < nz; k++)
            for (j = 0; j < ny; j++)
                for (i = 0; i < nx; i++) {
                    double s = b ? b[co] : 0.0;
                    for (ci = 0; ci < cin; ci++)
                        for (dz = -1; dz <= 1; dz++)
                            for (dy = -1; dy <= 1; dy++)
                                for (dx = -1; dx <= 1; dx++) {
                                    int64_t ii = i + dx, jj = j + dy, kk = k + dz;
                                    if (!inb(ii, nx) || !inb(jj, ny) || !inb(kk, nz))
                                        continue;
                                    s += wt[(((int64_t)co * cin + ci) * 3 + dz + 1) * 9 + (dy + 1) * 3 + dx + 1] *
                                         x[(int64_t)ci * N + (kk * ny + jj) * nx + ii];
                                }
                    y[(int64_t)co * N + (k * ny + j) * nx + i] = s;
                }
    }
}

/* dx[ci][q] = sum_co sum_t wt[co][ci][t] dy[co][q - t]  (gradient of fwd w.r.t. x) */
void orc_conv3d_bwd_data(int cin, int cout, const int64_t n[3], const double *dy, const double *wt,
                         double *dx_out)
{
    int64_t nx = n[0], ny = n[1], nz = n[2], N = nx * ny * nz;
    int ci;
#pragma omp parallel for schedule(static)
    for (ci = 0; ci < cin; ci++) {
        int64_t i, j, k;
        int co, dz, dyy, dxx;
        for (k = 0; k < nz; k++)
            for (j = 0; j < ny; j++)
                for (i = 0; i < nx; i++) {
                    double s = 0.0;
                    for (co = 0; co < cout; co++)
                        for (dz = -1; dz <= 1; dz++)
                            for (dyy = -1; dyy <= 1; dyy++)
                                for (dxx = -1; dxx <= 1; dxx++) {
                                    int64_t ii = i - dxx, jj = j - dyy, kk = k - dz;
                                    if (!inb(ii, nx) || !inb(jj, ny) || !inb(kk, nz))
                                        continue;
                                    s += wt[(((int64_t)co * cin + ci) * 3 + dz + 1) * 9 + (dyy + 1) * 3 + dxx + 1] *
                                         dy[(int64_t)co * N + (kk * ny + jj) * nx + ii];
                                }
                    dx_out[(int64_t)ci * N + (k * ny + j) * nx + i] = s;
                }
    }
}

/* dw[co][ci][t] = sum_p dy[co][p] x[ci][p + t];  db[co] = sum_p dy[co][p] */
void orc_conv3d_bwd_weight(int cin, int cout, const int64_t n[3], const double *x, const double *dy,
                           double *dw, double *db)
{
    int64_t nx = n[0], ny = n[1], nz = n[2], N = nx * ny * nz;
    int co;
#pragma omp parallel for schedule(static)
    for (co = 0; co < cout; co++) {
        int ci, dz, dyy, dxx;
        int64_t i, j, k;
        double sb = 0.0;
        for (k = 0; k < N; k++)
            sb += dy[(int64_t)co * N + k];
        if (db)
            db[co] = sb;
        for (ci = 0; ci < cin; ci++)
            for (dz = -1; dz <= 1; dz++)
                for (dyy = -1; dyy <= 1; dyy++)
                    for (dxx = -1; dxx <= 1; dxx++) {
                        double s = 0.0;
                        for (k = 0; k < nz; k++)
                            for (j = 0; j < ny; j++)
                                for (i = 0; i < nx; i++) {
                                    int64_t ii = i + dxx, jj = j + dyy, kk = k + dz;
                                    if (!inb(ii, nx) || !inb(jj, ny) || !inb(kk, nz))
                                        continue;
                                    s += dy[(int64_t)co * N + (k * ny + j) * nx + i] *
                                         x[(int64_t)ci * N + (kk * ny + jj) * nx + ii];
                                }
                        dw[(((int64_t)co * cin + ci) * 3 + dz + 1) * 9 + (dyy + 1) * 3 + dxx + 1] = s;
                    }
    }
}
