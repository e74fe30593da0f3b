/*
 * FP64 dense CPU oracle for the explicit reaction-diffusion step of
 * Stark & Sbalzarini (arXiv 2304.11165) on a level-set-masked voxel box.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * definition that the CUDA library is checked against.  Only the tests, the
 * smoke check and the bench's CPU-baseline leg load it; the library never
 * does, and the two share no code, header or table.
 *
 * Everything is a plain loop over every voxel of a dense box, in FP64, in the
 * order the paper states it.  Arrays are dense, shaped [Nz][Ny][Nx] with x
 * fastest; a voxel's linear index is (z*Ny + y)*Nx + x.  Multi-species arrays
 * are [S][Nz][Ny][Nx].
 *
 * Readings of the paper taken here (the paper is silent or loose on them):
 *  - active (pore) voxel: phi > FLT_EPSILON, compared in FP32 (the point
 *    insertion rule of the sparse-grid construction, Appendix B Listing 5,
 *    with lower bound 0 and no upper cut; the no-flux test of the functor,
 *    Appendix B Listing 6, phi <= 0 + eps, is its complement);
 *  - voxels outside the box are outside Omega (mirrored, i.e. no flux through
 *    box faces) unless the face is Dirichlet;
 *  - a Dirichlet face holds its *active* voxels of that voxel plane fixed at
 *    their current value; they are ordinary neighbours of free voxels;
 *  - surface reaction weight: smoothed delta w = (1 + cos(pi phi / eps_b)) /
 *    (2 eps_b) for active voxels with phi < eps_b, else 0;
 *  - species 0 loses T = k w u0 per unit time, species 1 gains the same T;
 *  - the explicit limit is the 3-D, reactive form of Eq. 10.
 *
 * Sums (mass, fluxes, norms, dot products, gradient sums) are accumulated per
 * z-slice with Kahan compensation, then the slices are added in order, so the
 * result does not depend on the thread count.
 *
 * Parity pins for every function live in tests/test_oracle_*.py.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(x, y, z) (((int64_t)(z) * ny + (y)) * nx + (x))

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Kahan-compensated accumulator. */
typedef struct { double s, c; } ksum;
static inline void kadd(ksum *k, double v)
{
    double y = v - k->c;
    double t = k->s + y;
    k->c = (t - k->s) - y;
    k->s = t;
}

/* Adds per-slice partial sums in slice order. */
static double sum_slices(const double *part, int64_t nz)
{
    ksum k = {0.0, 0.0};
    for (int64_t z = 0; z < nz; ++z) kadd(&k, part[z]);
    return k.s;
}

/* ------------------------------------------------------------------------ */
/* Geometry: which voxels belong to Omega (Sec. 3.2; point insertion in
 * Appendix B Listing 5; the functor's no-flux test in Listing 6).            */
void oracle_active_mask(const float *phi, int64_t n, float eps_mask, uint8_t *active)
{
    for (int64_t i = 0; i < n; ++i) active[i] = (phi[i] > eps_mask) ? 1 : 0;
}

/* Dirichlet-held voxels: active voxels on a face flagged Dirichlet.
 * face order: x-low, x-high, y-low, y-high, z-low, z-high.                   */
void oracle_fixed_mask(const int64_t dims[3], const uint8_t *active, const int dirichlet[6],
                       uint8_t *fixed)
{
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                int on = (dirichlet[0] && x == 0) || (dirichlet[1] && x == nx - 1) ||
                         (dirichlet[2] && y == 0) || (dirichlet[3] && y == ny - 1) ||
                         (dirichlet[4] && z == 0) || (dirichlet[5] && z == nz - 1);
                fixed[IDX(x, y, z)] = (uint8_t)(active[IDX(x, y, z)] && on);
            }
}

/* Smoothed surface delta that restricts the reaction to the interface band
 * (Sec. 3.5: a sink rate on the surface, localised by the level set).       */
void oracle_surface_weight(const float *phi, const uint8_t *active, int64_t n, double band_eps,
                           double *w)
{
    const double pi = 3.14159265358979323846;
    for (int64_t i = 0; i < n; ++i) {
        double p = (double)phi[i];
        w[i] = (active[i] && p < band_eps) ? (1.0 + cos(pi * p / band_eps)) / (2.0 * band_eps) : 0.0;
    }
}

/* Explicit stability limit: Eq. 10 gives dt < 1/(2 max D) * 1/sum_a dx_a^-2
 * for pure diffusion in 2-D.  Here every axis with more than one voxel counts,
 * and each species' largest linear loss rate is added to its diffusive rate;
 * the result is the smallest over species.                                  */
double oracle_stability_limit(const int64_t dims[3], const double dx[3], int nspecies,
                              const double *D, const double *decay, double k_surf, double band_eps)
{
    double inv2 = 0.0;
    for (int a = 0; a < 3; ++a)
        if (dims[a] > 1) inv2 += 1.0 / (dx[a] * dx[a]);
    double lim = INFINITY;
    for (int s = 0; s < nspecies; ++s) {
        double rate = 2.0 * D[s] * inv2 + decay[s];
        if (s == 0 && k_surf > 0.0) rate += k_surf / band_eps;  /* max of w is 1/eps_b */
        double l = (rate > 0.0) ? 1.0 / rate : INFINITY;
        if (l < lim) lim = l;
    }
    return lim;
}

/* ------------------------------------------------------------------------ */
/* Value of the neighbour across axis a, direction dir (+1/-1), with the
 * no-flux rule: a neighbour outside Omega (or outside the box) takes the
 * centre's value, so the gradient towards it is zero (Sec. 2.3; Appendix B
 * Listing 6).                                                                */
static inline double nbr_value(const double *u, const uint8_t *active, int64_t nx, int64_t ny,
                               int64_t nz, int64_t x, int64_t y, int64_t z, int a, int dir,
                               double uc)
{
    int64_t xx = x, yy = y, zz = z;
    if (a == 0) xx += dir;
    else if (a == 1) yy += dir;
    else zz += dir;
    if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz) return uc;
    int64_t j = IDX(xx, yy, zz);
    return active[j] ? u[j] : uc;
}

/* Bracketed right-hand side of the FTCS update for species s at voxel
 * (x,y,z): sum_a D_s/dx_a^2 [(u_{+a} - u) - (u - u_{-a})] - decay_s u + reaction.
 * `lap_only` returns just sum_a 1/dx_a^2 [...] (no D, no reaction).        */
static double rhs_at(const double *u, const uint8_t *active, const double *w, int nspecies,
                     int64_t nx, int64_t ny, int64_t nz, int64_t x, int64_t y, int64_t z, int s,
                     const double dx[3], const double *D, const double *decay, double k_surf,
                     int lap_only)
{
    const int64_t n = nx * ny * nz;
    const int64_t i = IDX(x, y, z);
    const double *us = u + (int64_t)s * n;
    const double uc = us[i];
    double lap = 0.0;
    for (int a = 0; a < 3; ++a) {
        double up = nbr_value(us, active, nx, ny, nz, x, y, z, a, +1, uc);
        double um = nbr_value(us, active, nx, ny, nz, x, y, z, a, -1, uc);
        double coef = (lap_only ? 1.0 : D[s]) / (dx[a] * dx[a]);
        lap += coef * ((up - uc) - (uc - um));
    }
    if (lap_only) return lap;
    double transfer = (w && k_surf != 0.0) ? k_surf * w[i] * u[i] : 0.0;  /* k w u_A, species 0 */
    double react = -decay[s] * uc;
    if (s == 0) react -= transfer;
    else if (s == 1) react += transfer;
    (void)nspecies;
    return lap + react;
}

/* One forward-Euler FTCS step of Eq. 1 (Sec. 2.3: FTCS, explicit Euler; a
 * Jacobi sweep from the state at step n into a separate output, like the
 * two concentration properties of Appendix B Listing 7).  Inactive voxels are set to 0; Dirichlet-held
 * voxels are copied.  `src` (nullable, [S][N]) is an extra source term added
 * inside the bracket, used by the manufactured-solution check of Sec. 3.1.  */
void oracle_step(const int64_t dims[3], const uint8_t *active, const uint8_t *fixed,
                 const double *w, int nspecies, const double *u, double *u_next,
                 const double dx[3], double dt, const double *D, const double *decay,
                 double k_surf, const double *src)
{
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    const int64_t n = nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t i = IDX(x, y, z);
                for (int s = 0; s < nspecies; ++s) {
                    const int64_t si = (int64_t)s * n + i;
                    if (!active[i]) { u_next[si] = 0.0; continue; }
                    if (fixed[i]) { u_next[si] = u[si]; continue; }
                    double r = rhs_at(u, active, w, nspecies, nx, ny, nz, x, y, z, s, dx, D, decay,
                                      k_surf, 0);
                    if (src) r += src[si];
                    u_next[si] = u[si] + dt * r;
                }
            }
}

/* nsteps forward-Euler steps in place on u ([S][N]).  Returns 0, or -1 when
 * the scratch state cannot be allocated.                                     */
int oracle_run(const int64_t dims[3], const uint8_t *active, const uint8_t *fixed, const double *w,
               int nspecies, double *u, const double dx[3], double dt, const double *D,
               const double *decay, double k_surf, int64_t nsteps)
{
    const int64_t n = dims[0] * dims[1] * dims[2] * (int64_t)nspecies;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)n);
    if (!tmp) return -1;
    double *a = u, *b = tmp;
    for (int64_t t = 0; t < nsteps; ++t) {
        oracle_step(dims, active, fixed, w, nspecies, a, b, dx, dt, D, decay, k_surf, NULL);
        double *c = a; a = b; b = c;
    }
    if (a != u) memcpy(u, a, sizeof(double) * (size_t)n);
    free(tmp);
    return 0;
}

/* (L_h u)_i: the bracketed right-hand side per species, 0 on inactive and
 * Dirichlet-held voxels.                                                     */
void oracle_rhs(const int64_t dims[3], const uint8_t *active, const uint8_t *fixed, const double *w,
                int nspecies, const double *u, const double dx[3], const double *D,
                const double *decay, double k_surf, double *rhs)
{
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    const int64_t n = nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t i = IDX(x, y, z);
                for (int s = 0; s < nspecies; ++s)
                    rhs[(int64_t)s * n + i] =
                        (active[i] && !fixed[i])
                            ? rhs_at(u, active, w, nspecies, nx, ny, nz, x, y, z, s, dx, D, decay,
                                     k_surf, 0)
                            : 0.0;
            }
}

/* Monitoring reductions, per species s, written to out[s*5 + q]:
 *   q=0 mass      M = sum_{active} u dV                 (mass curve, Sec. 3.4)
 *   q=1 J_in      x-flux through the plane between x=0 and x=1
 *   q=2 J_out     x-flux through the plane between x=Nx-2 and x=Nx-1
 *   q=3 residual  ||L_h u||_2 over free active voxels
 *   q=4 n_active
 * J_p = sum over (y,z) with both (p,y,z) and (p+1,y,z) active of
 *       D_s (u_p - u_{p+1}) / dx * dy dz.                                   */
void oracle_reduce(const int64_t dims[3], const uint8_t *active, const uint8_t *fixed,
                   const double *w, int nspecies, const double *u, const double dx[3],
                   const double *D, const double *decay, double k_surf, double *out)
{
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    const int64_t n = nx * ny * nz;
    const double dv = dx[0] * dx[1] * dx[2];
    const double area = dx[1] * dx[2];
    double *part = (double *)calloc((size_t)(5 * nz), sizeof(double));
    if (!part) return;
    for (int s = 0; s < nspecies; ++s) {
        const double *us = u + (int64_t)s * n;
#pragma omp parallel for schedule(static)
        for (int64_t z = 0; z < nz; ++z) {
            ksum m = {0, 0}, jin = {0, 0}, jout = {0, 0}, r2 = {0, 0}, cnt = {0, 0};
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) {
                    const int64_t i = IDX(x, y, z);
                    if (!active[i]) continue;
                    kadd(&cnt, 1.0);
                    kadd(&m, us[i] * dv);
                    if (!fixed[i]) {
                        double r = rhs_at(u, active, w, nspecies, nx, ny, nz, x, y, z, s, dx, D,
                                          decay, k_surf, 0);
                        kadd(&r2, r * r);
                    }
                    if (nx >= 2 && (x == 0 || x == nx - 2) && active[i + 1]) {
                        double j = D[s] * (us[i] - us[i + 1]) / dx[0] * area;
                        if (x == 0) kadd(&jin, j);
                        if (x == nx - 2) kadd(&jout, j);
                    }
                }
            part[0 * nz + z] = m.s;
            part[1 * nz + z] = jin.s;
            part[2 * nz + z] = jout.s;
            part[3 * nz + z] = r2.s;
            part[4 * nz + z] = cnt.s;
        }
        out[s * 5 + 0] = sum_slices(part + 0 * nz, nz);
        out[s * 5 + 1] = sum_slices(part + 1 * nz, nz);
        out[s * 5 + 2] = sum_slices(part + 2 * nz, nz);
        out[s * 5 + 3] = sqrt(sum_slices(part + 3 * nz, nz));
        out[s * 5 + 4] = sum_slices(part + 4 * nz, nz);
    }
    free(part);
}

/* Effective diffusivity and diffusive tortuosity (Eq. 2: tau = D_f / D_eff).
 * D_eff is the superficial value J L / (dC A) with J the mean of the inlet
 * and outlet fluxes, L = (Nx-1) dx the distance between the two held planes
 * and A = Ny dy Nz dz the box cross-section.  The pore-space (intrinsic)
 * effective diffusivity is D_eff / psi, so tau = D psi / D_eff.            */
void oracle_effective_D(const int64_t dims[3], const double dx[3], double J_in, double J_out,
                        double dC, double D, double n_active, double *D_eff, double *tau,
                        double *psi)
{
    const double L = (double)(dims[0] - 1) * dx[0];
    const double A = (double)dims[1] * dx[1] * (double)dims[2] * dx[2];
    const double J = 0.5 * (J_in + J_out);
    *psi = n_active / ((double)dims[0] * (double)dims[1] * (double)dims[2]);
    *D_eff = J * L / (dC * A);
    *tau = (*D_eff > 0.0) ? (*psi) * D / (*D_eff) : INFINITY;
}

/* ------------------------------------------------------------------------ */
/* Steady state by a second, independent method: the discrete steady state
 * solves L_h u = 0 on the free voxels with the Dirichlet voxels held.  With
 * the no-flux rule L_h is the (negative) graph Laplacian of the active-voxel
 * graph, so -L_h restricted to free voxels is symmetric positive
 * semi-definite and conjugate gradients apply.  Jacobi preconditioner.
 * u holds the start (with the held values) and receives the solution.
 * Returns the final relative residual ||b - A x|| / ||b||.                  */
static void cg_apply(const int64_t dims[3], const uint8_t *active, const uint8_t *fixed,
                     const double *eps, const double dx[3], double D, const double *v, double *Av)
{
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t i = IDX(x, y, z);
                if (!active[i] || fixed[i]) { Av[i] = 0.0; continue; }
                double acc = 0.0;
                for (int a = 0; a < 3; ++a)
                    for (int dir = -1; dir <= 1; dir += 2) {
                        int64_t xx = x + (a == 0 ? dir : 0), yy = y + (a == 1 ? dir : 0),
                                zz = z + (a == 2 ? dir : 0);
                        if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz) continue;
                        int64_t j = IDX(xx, yy, zz);
                        if (!active[j]) continue;
                        double c = D / (dx[a] * dx[a]) * (eps ? 0.5 * (eps[i] + eps[j]) : 1.0);
                        /* held neighbours enter as value 0 (their values are in b) */
                        acc += c * (v[i] - (fixed[j] ? 0.0 : v[j]));
                    }
                Av[i] = acc;
            }
}

static double cg_dot(const int64_t dims[3], const double *a, const double *b, double *part)
{
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < nz; ++z) {
        ksum k = {0, 0};
        for (int64_t i = IDX(0, 0, z); i < IDX(0, 0, z + 1); ++i) kadd(&k, a[i] * b[i]);
        part[z] = k.s;
    }
    return sum_slices(part, nz);
}

static double steady_cg(const int64_t dims[3], const uint8_t *active, const uint8_t *fixed,
                        const double *eps, const double dx[3], double D, double *u, double tol,
                        int64_t maxit, int64_t *iters)
{
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    const int64_t n = nx * ny * nz;
    double *x = (double *)calloc((size_t)n, sizeof(double));
    double *b = (double *)calloc((size_t)n, sizeof(double));
    double *r = (double *)calloc((size_t)n, sizeof(double));
    double *zv = (double *)calloc((size_t)n, sizeof(double));
    double *p = (double *)calloc((size_t)n, sizeof(double));
    double *Ap = (double *)calloc((size_t)n, sizeof(double));
    double *dinv = (double *)calloc((size_t)n, sizeof(double));
    double *part = (double *)calloc((size_t)nz, sizeof(double));
    double rel = -1.0;
    *iters = 0;
    if (!x || !b || !r || !zv || !p || !Ap || !dinv || !part) goto done;

    /* b_i = sum over held neighbours j of c_a u_j;  x = start on free voxels */
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t xx0 = 0; xx0 < nx; ++xx0) {
                const int64_t i = IDX(xx0, y, z);
                if (!active[i] || fixed[i]) continue;
                x[i] = u[i];
                double diag = 0.0, bi = 0.0;
                for (int a = 0; a < 3; ++a)
                    for (int dir = -1; dir <= 1; dir += 2) {
                        int64_t xx = xx0 + (a == 0 ? dir : 0), yy = y + (a == 1 ? dir : 0),
                                zz = z + (a == 2 ? dir : 0);
                        if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz) continue;
                        int64_t j = IDX(xx, yy, zz);
                        if (!active[j]) continue;
                        double c = D / (dx[a] * dx[a]) * (eps ? 0.5 * (eps[i] + eps[j]) : 1.0);
                        diag += c;
                        if (fixed[j]) bi += c * u[j];
                    }
                b[i] = bi;
                dinv[i] = diag > 0.0 ? 1.0 / diag : 0.0;
            }
    double bnorm = sqrt(cg_dot(dims, b, b, part));
    cg_apply(dims, active, fixed, eps, dx, D, x, Ap);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - Ap[i];
    if (bnorm == 0.0) { rel = sqrt(cg_dot(dims, r, r, part)); goto store; }
    for (int64_t i = 0; i < n; ++i) { zv[i] = dinv[i] * r[i]; p[i] = zv[i]; }
    double rz = cg_dot(dims, r, zv, part);
    rel = sqrt(cg_dot(dims, r, r, part)) / bnorm;
    while (rel >= tol && *iters < maxit) {
        cg_apply(dims, active, fixed, eps, dx, D, p, Ap);
        double pAp = cg_dot(dims, p, Ap, part);
        if (!(pAp > 0.0)) break;
        double alpha = rz / pAp;
        for (int64_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * Ap[i]; }
        ++*iters;
        rel = sqrt(cg_dot(dims, r, r, part)) / bnorm;
        for (int64_t i = 0; i < n; ++i) zv[i] = dinv[i] * r[i];
        double rz_new = cg_dot(dims, r, zv, part);
        double beta = rz_new / rz;
        rz = rz_new;
        for (int64_t i = 0; i < n; ++i) p[i] = zv[i] + beta * p[i];
    }
store:
    for (int64_t i = 0; i < n; ++i)
        if (active[i] && !fixed[i]) u[i] = x[i];
done:
    free(x); free(b); free(r); free(zv); free(p); free(Ap); free(dinv); free(part);
    return rel;
}

/* ------------------------------------------------------------------------ */
double oracle_steady_cg(const int64_t dims[3], const uint8_t *active, const uint8_t *fixed,
                        const double dx[3], double D, double *u, double tol, int64_t maxit,
                        int64_t *iters)
{
    return steady_cg(dims, active, fixed, NULL, dx, D, u, tol, maxit, iters);
}

/* Sum of u over the active voxels of the box lo <= (x, y, z) < hi, and their
 * count: the mass of the bleached region of a simulated FRAP experiment
 * (Sec. 3.3, the normalised mass in the initially bleached box).  out[2].   */
void oracle_box_sum(const int64_t dims[3], const uint8_t *active, const double *u, const int64_t lo[3],
                    const int64_t hi[3], double *out)
{
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    ksum m = {0, 0};
    double cnt = 0.0;
    for (int64_t z = lo[2] < 0 ? 0 : lo[2]; z < (hi[2] > nz ? nz : hi[2]); ++z)
        for (int64_t y = lo[1] < 0 ? 0 : lo[1]; y < (hi[1] > ny ? ny : hi[1]); ++y)
            for (int64_t x = lo[0] < 0 ? 0 : lo[0]; x < (hi[0] > nx ? nx : hi[0]); ++x) {
                const int64_t i = IDX(x, y, z);
                if (!active[i]) continue;
                kadd(&m, u[i]);
                cnt += 1.0;
            }
    out[0] = m.s;
    out[1] = cnt;
}

/* ------------------------------------------------------------------------ */
/* Inhomogeneous diffusion (Eq. 6 and the functor of Appendix B Listing 6;
 * the paper's fertilizer application, Sec. 3.4): one species whose
 * diffusivity is D * eps_i per voxel.  The flux between a voxel and a face
 * neighbour uses the arithmetic mean of their diffusivities, and a neighbour
 * outside Omega takes the centre's value and the centre's eps (no flux):
 *   u'_i = u_i + dt ( sum_a 1/dx_a^2 [ D_{+a} (u~_{i+a} - u_i) - D_{-a} (u_i - u~_{i-a}) ] - decay u_i ),
 *   D_{+-a} = D (eps_i + eps~_{i+-a}) / 2.                                   */

/* Eq. 6: eps = d_min + d_max / (1 + exp(-(g1 + g2 phi))), per voxel.        */
void oracle_eps_sigmoid(const float *phi, int64_t n, double d_min, double d_max, double g1,
                        double g2, double *eps)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) eps[i] = d_min + d_max / (1.0 + exp(-(g1 + g2 * (double)phi[i])));
}

static double rhs_inhom_at(const double *u, const double *eps, const uint8_t *active, int64_t nx,
                           int64_t ny, int64_t nz, int64_t x, int64_t y, int64_t z,
                           const double dx[3], double D, double decay)
{
    const int64_t i = IDX(x, y, z);
    const double uc = u[i], ec = eps[i];
    double lap = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double up = nbr_value(u, active, nx, ny, nz, x, y, z, a, +1, uc);
        const double um = nbr_value(u, active, nx, ny, nz, x, y, z, a, -1, uc);
        const double ep = nbr_value(eps, active, nx, ny, nz, x, y, z, a, +1, ec);
        const double em = nbr_value(eps, active, nx, ny, nz, x, y, z, a, -1, ec);
        const double dp = D * (ec + ep) / 2.0, dm = D * (ec + em) / 2.0;
        lap += (dp * (up - uc) - dm * (uc - um)) / (dx[a] * dx[a]);
    }
    return lap - decay * uc;
}

void oracle_step_inhom(const int64_t dims[3], const uint8_t *active, const uint8_t *fixed,
                       const double *eps, const double *u, double *u_next, const double dx[3],
                       double dt, double D, double decay)
{
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t i = IDX(x, y, z);
                if (!active[i]) { u_next[i] = 0.0; continue; }
                if (fixed[i]) { u_next[i] = u[i]; continue; }
                u_next[i] = u[i] + dt * rhs_inhom_at(u, eps, active, nx, ny, nz, x, y, z, dx, D, decay);
            }
}

int oracle_run_inhom(const int64_t dims[3], const uint8_t *active, const uint8_t *fixed,
                     const double *eps, double *u, const double dx[3], double dt, double D,
                     double decay, int64_t nsteps)
{
    const int64_t n = dims[0] * dims[1] * dims[2];
    double *tmp = (double *)malloc(sizeof(double) * (size_t)n);
    if (!tmp) return -1;
    double *a = u, *b = tmp;
    for (int64_t t = 0; t < nsteps; ++t) {
        oracle_step_inhom(dims, active, fixed, eps, a, b, dx, dt, D, decay);
        double *c = a; a = b; b = c;
    }
    if (a != u) memcpy(u, a, sizeof(double) * (size_t)n);
    free(tmp);
    return 0;
}

/* Reductions of the inhomogeneous case, out[5] as oracle_reduce; the x-face
 * flux uses the face diffusivity D (eps_p + eps_{p+1}) / 2.                  */
void oracle_reduce_inhom(const int64_t dims[3], const uint8_t *active, const uint8_t *fixed,
                         const double *eps, const double *u, const double dx[3], double D,
                         double decay, double *out)
{
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    const double dv = dx[0] * dx[1] * dx[2];
    const double area = dx[1] * dx[2];
    double *part = (double *)calloc((size_t)(5 * nz), sizeof(double));
    if (!part) return;
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < nz; ++z) {
        ksum m = {0, 0}, jin = {0, 0}, jout = {0, 0}, r2 = {0, 0}, cnt = {0, 0};
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t i = IDX(x, y, z);
                if (!active[i]) continue;
                kadd(&cnt, 1.0);
                kadd(&m, u[i] * dv);
                if (!fixed[i]) {
                    const double r = rhs_inhom_at(u, eps, active, nx, ny, nz, x, y, z, dx, D, decay);
                    kadd(&r2, r * r);
                }
                if (nx >= 2 && (x == 0 || x == nx - 2) && active[i + 1]) {
                    const double j = D * (eps[i] + eps[i + 1]) / 2.0 * (u[i] - u[i + 1]) / dx[0] * area;
                    if (x == 0) kadd(&jin, j);
                    if (x == nx - 2) kadd(&jout, j);
                }
            }
        part[0 * nz + z] = m.s;
        part[1 * nz + z] = jin.s;
        part[2 * nz + z] = jout.s;
        part[3 * nz + z] = r2.s;
        part[4 * nz + z] = cnt.s;
    }
    out[0] = sum_slices(part + 0 * nz, nz);
    out[1] = sum_slices(part + 1 * nz, nz);
    out[2] = sum_slices(part + 2 * nz, nz);
    out[3] = sqrt(sum_slices(part + 3 * nz, nz));
    out[4] = sum_slices(part + 4 * nz, nz);
    free(part);
}

/* Steady state of the inhomogeneous case by CG (face coefficients
 * D (eps_i + eps_j) / 2 dx_a^-2: still a symmetric graph Laplacian).       */
double oracle_steady_cg_inhom(const int64_t dims[3], const uint8_t *active, const uint8_t *fixed,
                              const double *eps, const double dx[3], double D, double *u,
                              double tol, int64_t maxit, int64_t *iters)
{
    return steady_cg(dims, active, fixed, eps, dx, D, u, tol, maxit, iters);
}

/* Adjoint of one step.  The forward step is linear, u^{n+1} = M u^n, with
 * (free voxel i, species s)
 *   M_ii = 1 - dt sum_{active nbr j} c_a - dt decay_s - [s=0] dt k w_i,
 *   M_ij = dt c_a for every active neighbour j (held ones included),
 *   d u_B,i^{n+1} / d u_A,i^n = dt k w_i   (two species),
 * and Dirichlet-held rows are the identity.  The held values are not free
 * parameters, so lambda is kept at 0 on held (and inactive) voxels, and
 *   lambda^n = M^T lambda^{n+1}
 * runs over free voxels only.  Gradient contributions of this step, added
 * into grad[] = {dL/dD_0, ..., dL/dD_{S-1}, dL/dk}:
 *   dL/dD_s += sum_i lambda_{s,i}^{n+1} dt g_{s,i}(u^n), g = sum_a [..]/dx_a^2
 *   dL/dk   += sum_i dt w_i u_{A,i}^n (lambda_{B,i}^{n+1} - lambda_{A,i}^{n+1}).
 * No counterpart in the paper: the adjoint is this library's addition.     */
void oracle_adjoint_step(const int64_t dims[3], const uint8_t *active, const uint8_t *fixed,
                         const double *w, int nspecies, const double *u_n,
                         const double *lam_next, double *lam_n, const double dx[3], double dt,
                         const double *D, const double *decay, double k_surf, double *grad)
{
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    const int64_t n = nx * ny * nz;
    double *part = (double *)calloc((size_t)((nspecies + 1) * nz), sizeof(double));
    if (!part) return;
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < nz; ++z) {
        ksum gD[2] = {{0, 0}, {0, 0}}, gk = {0, 0};
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t i = IDX(x, y, z);
                if (!active[i] || fixed[i]) {
                    for (int s = 0; s < nspecies; ++s) lam_n[(int64_t)s * n + i] = 0.0;
                    continue;
                }
                const double wi = w ? w[i] : 0.0;
                for (int s = 0; s < nspecies; ++s) {
                    const double *ls = lam_next + (int64_t)s * n;
                    double sum_c = 0.0, off = 0.0;
                    for (int a = 0; a < 3; ++a)
                        for (int dir = -1; dir <= 1; dir += 2) {
                            int64_t xx = x + (a == 0 ? dir : 0), yy = y + (a == 1 ? dir : 0),
                                    zz = z + (a == 2 ? dir : 0);
                            if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz)
                                continue;
                            int64_t j = IDX(xx, yy, zz);
                            if (!active[j]) continue;
                            double c = D[s] / (dx[a] * dx[a]);
                            sum_c += c;
                            if (!fixed[j]) off += c * ls[j];
                        }
                    double rate = decay[s] + ((s == 0) ? k_surf * wi : 0.0);
                    double diag = 1.0 - dt * sum_c - dt * rate;
                    double val = diag * ls[i] + dt * off;
                    if (s == 0 && nspecies == 2) val += dt * k_surf * wi * lam_next[n + i];
                    lam_n[(int64_t)s * n + i] = val;
                    double g = rhs_at(u_n, active, w, nspecies, nx, ny, nz, x, y, z, s, dx, D,
                                      decay, k_surf, 1);
                    kadd(&gD[s], ls[i] * dt * g);
                }
                double lb = (nspecies == 2) ? lam_next[n + i] : 0.0;
                kadd(&gk, dt * wi * u_n[i] * (lb - lam_next[i]));
            }
        for (int s = 0; s < nspecies; ++s) part[(int64_t)s * nz + z] = gD[s].s;
        part[(int64_t)nspecies * nz + z] = gk.s;
    }
    for (int s = 0; s <= nspecies; ++s) grad[s] += sum_slices(part + (int64_t)s * nz, nz);
    free(part);
}

/* Full adjoint: stores every forward state u^0..u^N (no checkpointing on the
 * CPU), then runs lambda^n = M^T lambda^{n+1} from lambda^N = dL/du^N.
 * Writes lambda^0 (= dL/du^0 on free voxels), grad[] (see above, zeroed
 * first) and u^N.  Returns 0, or -1 when the state history cannot be stored. */
int oracle_adjoint_run(const int64_t dims[3], const uint8_t *active, const uint8_t *fixed,
                       const double *w, int nspecies, const double *u0, const double dx[3],
                       double dt, const double *D, const double *decay, double k_surf,
                       int64_t nsteps, const double *lam_N, double *lam_0, double *grad,
                       double *u_N)
{
    const int64_t n = dims[0] * dims[1] * dims[2] * (int64_t)nspecies;
    double *hist = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(nsteps + 1));
    double *la = (double *)malloc(sizeof(double) * (size_t)n);
    double *lb = (double *)malloc(sizeof(double) * (size_t)n);
    if (!hist || !la || !lb) { free(hist); free(la); free(lb); return -1; }
    memcpy(hist, u0, sizeof(double) * (size_t)n);
    for (int64_t t = 0; t < nsteps; ++t)
        oracle_step(dims, active, fixed, w, nspecies, hist + t * n, hist + (t + 1) * n, dx, dt, D,
                    decay, k_surf, NULL);
    if (u_N) memcpy(u_N, hist + nsteps * n, sizeof(double) * (size_t)n);
    for (int s = 0; s <= nspecies; ++s) grad[s] = 0.0;
    memcpy(la, lam_N, sizeof(double) * (size_t)n);
    for (int64_t t = nsteps - 1; t >= 0; --t) {
        oracle_adjoint_step(dims, active, fixed, w, nspecies, hist + t * n, la, lb, dx, dt, D,
                            decay, k_surf, grad);
        double *c = la; la = lb; lb = c;
    }
    memcpy(lam_0, la, sizeof(double) * (size_t)n);
    free(hist); free(la); free(lb);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sussman redistancing (Sec. 2.1, the redistancing PDE with the smoothed
 * sign of Peng et al.): phi is driven to the steady state of
 *   d phi / d alpha = sigma(phi) (1 - |grad phi|),
 *   sigma(phi) = phi / sqrt(phi^2 + |grad phi|^2 h^2),
 * by forward Euler in the artificial time alpha with first-order upwind
 * (Godunov) differences, the scheme the paper uses for its results.
 * Readings: |grad phi| is the Godunov magnitude for the sign of phi at the
 * voxel, and the same magnitude enters sigma; h = min(dx); a neighbour beyond
 * the box takes the voxel's own value (zero gradient); a voxel with phi = 0
 * does not move; every voxel is updated from the previous iterate (Jacobi).
 *   D-_a = (phi_i - phi_{i-a}) / dx_a,  D+_a = (phi_{i+a} - phi_i) / dx_a,
 *   phi > 0: G^2 = sum_a max(max(D-_a, 0)^2, min(D+_a, 0)^2),
 *   phi < 0: G^2 = sum_a max(min(D-_a, 0)^2, max(D+_a, 0)^2),
 *   phi' = phi + dalpha sigma (1 - G).                                       */
static double godunov_mag(const double *p, int64_t nx, int64_t ny, int64_t nz, int64_t x, int64_t y,
                          int64_t z, const double dx[3])
{
    const double c = p[IDX(x, y, z)];
    const int64_t lo[3] = {x > 0 ? x - 1 : x, y > 0 ? y - 1 : y, z > 0 ? z - 1 : z};
    const int64_t hi[3] = {x < nx - 1 ? x + 1 : x, y < ny - 1 ? y + 1 : y, z < nz - 1 ? z + 1 : z};
    const double vm[3] = {p[IDX(lo[0], y, z)], p[IDX(x, lo[1], z)], p[IDX(x, y, lo[2])]};
    const double vp[3] = {p[IDX(hi[0], y, z)], p[IDX(x, hi[1], z)], p[IDX(x, y, hi[2])]};
    double g2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double dm = (c - vm[a]) / dx[a];
        const double dp = (vp[a] - c) / dx[a];
        double s1, s2;
        if (c > 0.0) {
            s1 = dm > 0.0 ? dm : 0.0;
            s2 = dp < 0.0 ? dp : 0.0;
        } else {
            s1 = dm < 0.0 ? dm : 0.0;
            s2 = dp > 0.0 ? dp : 0.0;
        }
        const double q1 = s1 * s1, q2 = s2 * s2;
        g2 += q1 > q2 ? q1 : q2;
    }
    return sqrt(g2);
}

/* `iters` iterations from phi0 into out (both dense [Nz][Ny][Nx]); dalpha =
 * cfl * min(dx).  Returns 0, or -1 when the work array cannot be allocated. */
int oracle_sussman(const int64_t dims[3], const double dx[3], const double *phi0, double cfl, int64_t iters,
                   double *out)
{
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    const int64_t n = nx * ny * nz;
    double h = dx[0];
    if (dx[1] < h) h = dx[1];
    if (dx[2] < h) h = dx[2];
    const double dalpha = cfl * h;
    double *a = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!a) return -1;
    memcpy(a, phi0, sizeof(double) * (size_t)n);
    for (int64_t it = 0; it < iters; ++it) {
#pragma omp parallel for schedule(static)
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) {
                    const double c = a[IDX(x, y, z)];
                    if (c == 0.0) {
                        out[IDX(x, y, z)] = c;
                        continue;
                    }
                    const double g = godunov_mag(a, nx, ny, nz, x, y, z, dx);
                    const double sigma = c / sqrt(c * c + g * g * h * h);
                    out[IDX(x, y, z)] = c + dalpha * sigma * (1.0 - g);
                }
        memcpy(a, out, sizeof(double) * (size_t)n);
    }
    memcpy(out, a, sizeof(double) * (size_t)n);
    free(a);
    return 0;
}

/* The Godunov magnitude |grad phi| per voxel (the quantity the steady state
 * drives to 1), for the pins. */
void oracle_upwind_grad(const int64_t dims[3], const double dx[3], const double *phi, double *out)
{
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) out[IDX(x, y, z)] = godunov_mag(phi, nx, ny, nz, x, y, z, dx);
}
