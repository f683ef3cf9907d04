/*
 * Plain FP64 CPU oracle of one explicit electromagnetic PIC cycle (KEMPIC-3D,
 * arxiv 2609.16575).  TEST INFRASTRUCTURE ONLY: this file is built and called by
 * the tests, by the package's smoke check and by the benchmark's CPU-baseline leg.
 * The product path never links, loads or calls it, and it shares no code, header
 * or constant with the CUDA library.
 *
 * It is deliberately slow and literal: one loop per operation, no blocking, no
 * fusion.  Every routine cites the passage of the paper it follows.
 *
 * Conventions (the paper's normalised units, section 2.3 and 3.1):
 *   c = eps0 = mu0 = 1; lengths in c/omega_p, times in 1/omega_p.
 *   Grid of n[0] x n[1] x n[2] cells with spacings d[0..2], periodic.
 *   Arrays hold one value per cell, index (k*ny + j)*nx + i, for each Yee
 *   component at its own staggered location (section 2.3):
 *     Ex(i+1/2,j,k)  Ey(i,j+1/2,k)  Ez(i,j,k+1/2)       (also Jx, Jy, Jz)
 *     Bx(i,j+1/2,k+1/2)  By(i+1/2,j,k+1/2)  Bz(i+1/2,j+1/2,k)
 *   Charge density rho lives on the nodes (i,j,k).
 *   Particle positions are kept in cell units, X_d = x_d / d_d in [0, n_d), as an
 *   integer cell index plus an in-cell offset in [0, 1) (two FP64 arrays), so that
 *   FP64 resolves 2^-53 of a cell anywhere in the box; momenta are u = gamma v.
 *   A species has charge q and mass m per physical particle; a super-particle of
 *   weight w carries q w and m w (Eqs. (9)-(11)).
 *
 * Time levels (section 2.2, Fig. 2): a state holds E^n, B^{n-1/2}, x^n, u^{n-1/2}.
 */
#include <math.h>
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

typedef struct {
    int n[3];
    double d[3];
    double dt;
    int open_x;    /* 1: x is bounded (absorbing faces), not periodic */
    long nxs;      /* values stored per x line: n[0], or n[0] + 1 nodes when open_x */
} or_grid;

/* The exported functions take n as 4 ints: n[0..2] cells, n[3] = open_x.  With an
 * open x dimension the arrays store nx + 1 values per x line (nodes 0..nx), so the
 * node-located components (Ey, Ez, Bx, Jy, Jz, rho) include the boundary plane x = nx;
 * the half-located ones (Ex, By, Bz, Jx) leave index nx unused.                   */
static or_grid mkgrid(const int* n, const double* d, double dt)
{
    or_grid g = {{n[0], n[1], n[2]}, {d[0], d[1], d[2]}, dt, n[3], n[0] + (n[3] ? 1 : 0)};
    return g;
}

static long wrapi(long i, long n) {
    long r = i % n;
    return r < 0 ? r + n : r;
}

/* Index of (i, j, k); y and z are periodic, x periodic or open.  Outside an open x
 * range (i < 0 or i > nx) there is no value: -1.                                  */
static long cell_index(const or_grid* g, long i, long j, long k) {
    if (g->open_x) {
        if (i < 0 || i > g->n[0]) return -1;
    } else {
        i = wrapi(i, g->n[0]);
    }
    j = wrapi(j, g->n[1]);
    k = wrapi(k, g->n[2]);
    return (k * g->n[1] + j) * g->nxs + i;
}

static long ncells(const or_grid* g) {
    return g->nxs * g->n[1] * g->n[2];
}

/* value at (i, j, k), zero outside an open x range */
static double at(const or_grid* g, const double* F, long i, long j, long k) {
    long c = cell_index(g, i, j, k);
    return c < 0 ? 0.0 : F[c];
}

/* ------------------------------------------------------------------------ */
/* Faraday's law on the Yee grid, section 2.3, Eq. (13) for Bx and its cyclic
 * permutations for By and Bz:  B <- B - frac*dt * curl E.
 * frac = 1 is one full step B^{n-1/2} -> B^{n+1/2}.                          */
void or_faraday(const int* n, const double* d, double dt, const double* E, double* B, double frac)
{
    or_grid g = mkgrid(n, d, dt);
    long N = ncells(&g);
    const double *Ex = E, *Ey = E + N, *Ez = E + 2 * N;
    double *Bx = B, *By = B + N, *Bz = B + 2 * N;
    double cx = frac * dt / d[0], cy = frac * dt / d[1], cz = frac * dt / d[2];
    for (long k = 0; k < n[2]; k++)
        for (long j = 0; j < n[1]; j++)
            for (long i = 0; i < g.nxs; i++) {
                long c = cell_index(&g, i, j, k);
                /* Bx(i, j+1/2, k+1/2): -dt/dy [Ez(j+1)-Ez(j)] + dt/dz [Ey(k+1)-Ey(k)] */
                Bx[c] += -cy * (at(&g, Ez, i, j + 1, k) - Ez[c])
                         + cz * (at(&g, Ey, i, j, k + 1) - Ey[c]);
                if (i == n[0]) continue;   /* By, Bz sit at x = i + 1/2: none beyond the last cell */
                /* By(i+1/2, j, k+1/2): -dt/dz [Ex(k+1)-Ex(k)] + dt/dx [Ez(i+1)-Ez(i)] */
                By[c] += -cz * (at(&g, Ex, i, j, k + 1) - Ex[c])
                         + cx * (at(&g, Ez, i + 1, j, k) - Ez[c]);
                /* Bz(i+1/2, j+1/2, k): -dt/dx [Ey(i+1)-Ey(i)] + dt/dy [Ex(j+1)-Ex(j)] */
                Bz[c] += -cx * (at(&g, Ey, i + 1, j, k) - Ey[c])
                         + cy * (at(&g, Ex, i, j + 1, k) - Ex[c]);
            }
}

/* Ampere-Maxwell law on the Yee grid, section 2.3, Eq. (14) for Ex and its
 * cyclic permutations:  E <- E + dt (curl B - J).                            */
void or_ampere(const int* n, const double* d, double dt, double* E, const double* B, const double* J)
{
    or_grid g = mkgrid(n, d, dt);
    long N = ncells(&g);
    double *Ex = E, *Ey = E + N, *Ez = E + 2 * N;
    const double *Bx = B, *By = B + N, *Bz = B + 2 * N;
    const double *Jx = J, *Jy = J + N, *Jz = J + 2 * N;
    double cx = dt / d[0], cy = dt / d[1], cz = dt / d[2];
    for (long k = 0; k < n[2]; k++)
        for (long j = 0; j < n[1]; j++)
            for (long i = 0; i < n[0]; i++) {
                long c = cell_index(&g, i, j, k);
                /* Ex(i+1/2, j, k): +dt/dy [Bz(j+1/2)-Bz(j-1/2)] - dt/dz [By(k+1/2)-By(k-1/2)] - dt Jx */
                Ex[c] += cy * (Bz[c] - at(&g, Bz, i, j - 1, k))
                         - cz * (By[c] - at(&g, By, i, j, k - 1))
                         - dt * Jx[c];
                /* with open x the boundary nodes x = 0 (and x = nx, outside this loop) of
                 * Ey and Ez belong to the absorbing boundary, not to this update */
                if (g.open_x && i == 0) continue;
                /* Ey(i, j+1/2, k): +dt/dz [Bx(k+1/2)-Bx(k-1/2)] - dt/dx [Bz(i+1/2)-Bz(i-1/2)] - dt Jy */
                Ey[c] += cz * (Bx[c] - at(&g, Bx, i, j, k - 1))
                         - cx * (Bz[c] - at(&g, Bz, i - 1, j, k))
                         - dt * Jy[c];
                /* Ez(i, j, k+1/2): +dt/dx [By(i+1/2)-By(i-1/2)] - dt/dy [Bx(j+1/2)-Bx(j-1/2)] - dt Jz */
                Ez[c] += cx * (By[c] - at(&g, By, i - 1, j, k))
                         - cy * (Bx[c] - at(&g, Bx, i, j - 1, k))
                         - dt * Jz[c];
            }
}

/* First-order Mur absorbing condition on the tangential E (Ey, Ez) of the two x faces
 * of an open x dimension, for a wave leaving along -x at x = 0 and +x at x = nx:
 *   E^{n+1}(0)  = E^n(1)    + k (E^{n+1}(1)    - E^n(0)),   k = (dt - dx) / (dt + dx),
 * and the mirror image at nx.  old holds Ey, Ez of planes 0, 1, nx-1, nx before the
 * Ampere update (layout [comp][plane][k][j]).                                     */
static void mur_x(const or_grid* g, const double* old, double* E)
{
    long N = ncells(g);
    long P = (long)g->n[1] * g->n[2];
    double kk = (g->dt - g->d[0]) / (g->dt + g->d[0]);
    int nx = g->n[0];
    for (int comp = 1; comp <= 2; comp++) {
        double* F = E + comp * N;
        const double* o = old + (comp - 1) * 4 * P;
        for (long k = 0; k < g->n[2]; k++)
            for (long j = 0; j < g->n[1]; j++) {
                long p = k * g->n[1] + j;
                F[cell_index(g, 0, j, k)] = o[1 * P + p] + kk * (F[cell_index(g, 1, j, k)] - o[0 * P + p]);
                F[cell_index(g, nx, j, k)] = o[2 * P + p] + kk * (F[cell_index(g, nx - 1, j, k)] - o[3 * P + p]);
            }
    }
}

/* ------------------------------------------------------------------------ */
/* Staggered cloud-in-cell interpolation, section 2.5: each component is
 * interpolated from its own Yee location with the first-order B-spline b1
 * (Eqs. (17)-(18) with b0 clouds).  half[d] = 1 when the component sits at a
 * half-integer position along d.                                            */
static double interp_component(const or_grid* g, const double* F, const int half[3], const long cell[3],
                               const double off[3])
{
    long base[3];
    double s[3];
    for (int d = 0; d < 3; d++) {
        double p = half[d] ? off[d] - 0.5 : off[d];   /* offset relative to the sample lattice */
        double f = floor(p);
        base[d] = cell[d] + (long)f;
        s[d] = p - f;
    }
    double v = 0.0;
    for (int c = 0; c < 2; c++)
        for (int b = 0; b < 2; b++)
            for (int a = 0; a < 2; a++) {
                double wgt = (a ? s[0] : 1.0 - s[0]) * (b ? s[1] : 1.0 - s[1]) * (c ? s[2] : 1.0 - s[2]);
                v += wgt * at(g, F, base[0] + a, base[1] + b, base[2] + c);
            }
    return v;
}

static const int HALF_E[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
static const int HALF_B[3][3] = {{0, 1, 1}, {1, 0, 1}, {1, 1, 0}};

static void gather(const or_grid* g, const double* E, const double* B, const long cell[3], const double off[3],
                   double Ep[3], double Bp[3])
{
    long N = ncells(g);
    for (int c = 0; c < 3; c++) {
        Ep[c] = interp_component(g, E + c * N, HALF_E[c], cell, off);
        Bp[c] = interp_component(g, B + c * N, HALF_B[c], cell, off);
    }
}

/* split a position in cell units into cell index and offset */
static void split(const double X[3], long cell[3], double off[3])
{
    for (int d = 0; d < 3; d++) {
        double f = floor(X[d]);
        cell[d] = (long)f;
        off[d] = X[d] - f;
    }
}

void or_gather(const int* n, const double* d, const double* E, const double* B, const double* X, double* Ep, double* Bp)
{
    or_grid g = mkgrid(n, d, 0.0);
    long cell[3];
    double off[3];
    split(X, cell, off);
    gather(&g, E, B, cell, off, Ep, Bp);
}

/* ------------------------------------------------------------------------ */
/* Higher-order particle shape (section 2.5, Eq. (16) with l = 1; section 5 lists
 * higher-order shapes as an extension).  The cloud b1 is a triangle two cells wide;
 * its overlap with the unit cell around a sample point gives the quadratic B-spline
 * weight (the triangular-shaped cloud, TSC) of a sample at distance r, in cell units:
 *   W2(r) = 3/4 - r^2              for |r| <= 1/2,
 *           (3/2 - |r|)^2 / 2      for 1/2 <= |r| <= 3/2,
 *           0                      beyond.
 * As with b0 (CIC), every field component is interpolated from its own Yee location
 * (Eqs. (17)-(18)): the three samples nearest the particle along each dimension.     */
static double tsc_w(double r)
{
    r = fabs(r);
    if (r <= 0.5) return 0.75 - r * r;
    if (r < 1.5) return 0.5 * (1.5 - r) * (1.5 - r);
    return 0.0;
}

static double interp_component_tsc(const or_grid* g, const double* F, const int half[3], const long cell[3],
                                   const double off[3])
{
    long base[3];
    double w[3][3];
    for (int d = 0; d < 3; d++) {
        double p = half[d] ? off[d] - 0.5 : off[d];   /* offset relative to the sample lattice */
        double m = floor(p + 0.5);                     /* the nearest sample */
        base[d] = cell[d] + (long)m - 1;
        for (int a = 0; a < 3; a++) w[d][a] = tsc_w(p - (m - 1.0 + a));
    }
    double v = 0.0;
    for (int c = 0; c < 3; c++)
        for (int b = 0; b < 3; b++)
            for (int a = 0; a < 3; a++)
                v += w[0][a] * w[1][b] * w[2][c] * at(g, F, base[0] + a, base[1] + b, base[2] + c);
    return v;
}

static void gather_tsc(const or_grid* g, const double* E, const double* B, const long cell[3], const double off[3],
                       double Ep[3], double Bp[3])
{
    long N = ncells(g);
    for (int c = 0; c < 3; c++) {
        Ep[c] = interp_component_tsc(g, E + c * N, HALF_E[c], cell, off);
        Bp[c] = interp_component_tsc(g, B + c * N, HALF_B[c], cell, off);
    }
}

void or_gather_tsc(const int* n, const double* d, const double* E, const double* B, const double* X, double* Ep,
                   double* Bp)
{
    or_grid g = mkgrid(n, d, 0.0);
    long cell[3];
    double off[3];
    split(X, cell, off);
    gather_tsc(&g, E, B, cell, off, Ep, Bp);
}

/* ------------------------------------------------------------------------ */
/* Relativistic Boris push, section 2.4 (leapfrog Eqs. (19)-(20), Boris 1970):
 * half electric kick, magnetic rotation, half electric kick.
 * eps = q dt / (2 m).  u enters as u^{n-1/2} and leaves as u^{n+1/2}.       */
void or_boris(double eps, const double* E, const double* B, double* u)
{
    double um[3], t[3], s[3], up[3], upl[3];
    for (int c = 0; c < 3; c++) um[c] = u[c] + eps * E[c];
    double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    for (int c = 0; c < 3; c++) t[c] = eps * B[c] / gm;
    double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int c = 0; c < 3; c++) s[c] = 2.0 * t[c] / (1.0 + t2);
    /* u' = u- + u- x t */
    up[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
    up[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
    up[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
    /* u+ = u- + u' x s */
    upl[0] = um[0] + (up[1] * s[2] - up[2] * s[1]);
    upl[1] = um[1] + (up[2] * s[0] - up[0] * s[2]);
    upl[2] = um[2] + (up[0] * s[1] - up[1] * s[0]);
    for (int c = 0; c < 3; c++) u[c] = upl[c] + eps * E[c];
}

static double gamma_of(const double* u)
{
    return sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
}

/* Single particle in uniform fields (the verification problems of section 3.1):
 * physical coordinates (unit cell), nsteps Boris steps, trajectory written to
 * xs[(nsteps+1)*3] and us[(nsteps+1)*3] (us[k] holds u^{k-1/2}, us[0] the
 * initial momentum after the optional half back-push).                      */
void or_boris_orbit(const double* E, const double* B, double qm, double dt, const double* x0, const double* u0,
                    long nsteps, int backpush, double* xs, double* us)
{
    double x[3] = {x0[0], x0[1], x0[2]}, u[3] = {u0[0], u0[1], u0[2]};
    if (backpush) or_boris(qm * (-0.5 * dt) / 2.0, E, B, u);
    for (int c = 0; c < 3; c++) { xs[c] = x[c]; us[c] = u[c]; }
    for (long s = 1; s <= nsteps; s++) {
        or_boris(qm * dt / 2.0, E, B, u);
        double g = gamma_of(u);
        for (int c = 0; c < 3; c++) x[c] += dt * u[c] / g;
        for (int c = 0; c < 3; c++) { xs[3 * s + c] = x[c]; us[3 * s + c] = u[c]; }
    }
}

/* ------------------------------------------------------------------------ */
/* Charge-conserving current deposition, section 2.5: the zigzag scheme of
 * Umeda et al. (2003).  Per dimension, in cell units, the move X1 -> X2 is split
 * at the relay point
 *     Xr = min( min(i1,i2)+1, max( max(i1,i2), (X1+X2)/2 ) )
 * into two straight segments, each inside one cell.  A segment with
 * displacement D (cell units) and midpoint offset W (relative to its cell)
 * contributes to the 4 x-edges of its cell
 *     Jx(i+1/2, j+b, k+c) += q w / (dt dy dz) * Dx * [ Wy^(b) Wz^(c) + s_bc Dy Dz / 12 ]
 * (W^(0) = 1-W, W^(1) = W, s_bc = +1 if b == c else -1), and cyclically for Jy,
 * Jz.  The product of midpoint weights is Umeda's form; the Dy Dz / 12 term is
 * the exact charge flux of a straight segment through a trilinear (CIC) charge
 * cloud (Villasenor & Buneman 1992).  It vanishes for moves in one or two
 * dimensions (all of the paper's tests) and is what makes the deposit satisfy
 * the discrete continuity equation (12) exactly for moves in three dimensions,
 * the property section 2.5 requires of the scheme.
 * X1 and X2 are given relative to an origin cell c0 (so that they stay small and
 * FP64 keeps full resolution); X2 must be unwrapped (|floor(X2) - floor(X1)| <= 1
 * per dimension).                                                             */
static void segment_current(const or_grid* g, double qw, const long cell[3], const double D[3], const double W[3], double* J)
{
    long N = ncells(g);
    double C[3] = {qw / (g->dt * g->d[1] * g->d[2]),
                   qw / (g->dt * g->d[2] * g->d[0]),
                   qw / (g->dt * g->d[0] * g->d[1])};
    for (int comp = 0; comp < 3; comp++) {
        int p = (comp + 1) % 3, r = (comp + 2) % 3;   /* the two transverse dimensions */
        for (int b = 0; b < 2; b++)
            for (int c = 0; c < 2; c++) {
                double wp = b ? W[p] : 1.0 - W[p];
                double wr = c ? W[r] : 1.0 - W[r];
                double sgn = (b == c) ? 1.0 : -1.0;
                double val = C[comp] * D[comp] * (wp * wr + sgn * D[p] * D[r] / 12.0);
                long idx[3] = {cell[0], cell[1], cell[2]};
                idx[p] += b;
                idx[r] += c;
                long e = cell_index(g, idx[0], idx[1], idx[2]);
                if (e >= 0) J[comp * N + e] += val;   /* deposits outside an open x range leave the box */
            }
    }
}

static void zigzag(const or_grid* g, double qw, const long c0[3], const double X1[3], const double X2[3], double* J)
{
    long i1[3], i2[3], cell1[3], cell2[3];
    double Xr[3], D1[3], D2[3], W1[3], W2[3];
    for (int d = 0; d < 3; d++) {
        i1[d] = (long)floor(X1[d]);
        i2[d] = (long)floor(X2[d]);
        double lo = (double)((i1[d] < i2[d] ? i1[d] : i2[d]) + 1);
        double hi = (double)(i1[d] > i2[d] ? i1[d] : i2[d]);
        double mid = 0.5 * (X1[d] + X2[d]);
        Xr[d] = fmin(lo, fmax(hi, mid));
        D1[d] = Xr[d] - X1[d];
        D2[d] = X2[d] - Xr[d];
        W1[d] = 0.5 * (X1[d] + Xr[d]) - (double)i1[d];
        W2[d] = 0.5 * (Xr[d] + X2[d]) - (double)i2[d];
        cell1[d] = c0[d] + i1[d];
        cell2[d] = c0[d] + i2[d];
    }
    segment_current(g, qw, cell1, D1, W1, J);
    segment_current(g, qw, cell2, D2, W2, J);
}

/* Esirkepov's charge-conserving deposit (Esirkepov 2001; section 2.5 names it among
 * the charge-conserving schemes, the paper's runs use ZigZag) with the same first-order
 * (CIC) particle shape.  For a straight move X1 -> X2 (cell units relative to cell c0,
 * less than one cell per dimension) let S0, S1 be the node weights 1 - |X - node| before
 * and after, DS = S1 - S0 (on the three nodes b .. b + 2 per dimension, b the lower of
 * the two cells), and
 *   Wx = DSx (S0y S0z + DSy S0z / 2 + S0y DSz / 2 + DSy DSz / 3)   (y, z cyclically);
 * then Jx(i + 1/2) = -(q w / (dt dy dz)) sum_{i' <= i} Wx(i'), the sum along x from the
 * support's first node, and likewise Jy, Jz.  The W sum to the change of the node
 * charge, so the discrete continuity equation holds exactly.                        */
static double cic(double r) { r = fabs(r); return r < 1.0 ? 1.0 - r : 0.0; }

static void esirkepov(const or_grid* g, double qw, const long c0[3], const double X1[3], const double X2[3], double* J)
{
    long N = ncells(g);
    double C[3] = {qw / (g->dt * g->d[1] * g->d[2]),
                   qw / (g->dt * g->d[2] * g->d[0]),
                   qw / (g->dt * g->d[0] * g->d[1])};
    long b[3];
    double S0[3][3], DS[3][3];
    for (int d = 0; d < 3; d++) {
        long f1 = (long)floor(X1[d]), f2 = (long)floor(X2[d]);
        b[d] = f1 < f2 ? f1 : f2;
        for (int m = 0; m < 3; m++) {
            double node = (double)(b[d] + m);
            S0[d][m] = cic(X1[d] - node);
            DS[d][m] = cic(X2[d] - node) - S0[d][m];
        }
    }
    for (int comp = 0; comp < 3; comp++) {
        int p = (comp + 1) % 3, r = (comp + 2) % 3;
        for (int jp = 0; jp < 3; jp++)
            for (int jr = 0; jr < 3; jr++) {
                double acc = 0.0;
                for (int i = 0; i < 2; i++) {   /* edges b + 1/2 and b + 3/2 along comp */
                    double W = DS[comp][i] * (S0[p][jp] * S0[r][jr] + 0.5 * DS[p][jp] * S0[r][jr]
                                              + 0.5 * S0[p][jp] * DS[r][jr] + DS[p][jp] * DS[r][jr] / 3.0);
                    acc += W;
                    long idx[3];
                    idx[comp] = c0[comp] + b[comp] + i;
                    idx[p] = c0[p] + b[p] + jp;
                    idx[r] = c0[r] + b[r] + jr;
                    long e = cell_index(g, idx[0], idx[1], idx[2]);
                    if (e >= 0 && acc != 0.0) J[comp * N + e] += -C[comp] * acc;
                }
            }
    }
}

void or_esirkepov(const int* n, const double* d, double dt, double qw, const double* X1, const double* X2, double* J)
{
    or_grid g = mkgrid(n, d, dt);
    long c0[3];
    double a[3], bb[3];
    for (int k = 0; k < 3; k++) {
        c0[k] = (long)floor(X1[k]);
        a[k] = X1[k] - (double)c0[k];
        bb[k] = X2[k] - (double)c0[k];
    }
    esirkepov(&g, qw, c0, a, bb, J);
}

/* Esirkepov's deposit with the quadratic (TSC) shape above (Esirkepov 2001 holds for any
 * shape factorised over the dimensions).  For a straight move X1 -> X2 (cell units
 * relative to cell c0, less than one cell per dimension) the node weights before and
 * after, S0 = W2(X1 - node) and S1 = W2(X2 - node), are taken on the four nodes
 * b .. b + 3 per dimension, b = min(m1, m2) - 1 with m the node nearest to X; DS =
 * S1 - S0 and
 *   Wx = DSx (S0y S0z + DSy S0z / 2 + S0y DSz / 2 + DSy DSz / 3)   (y, z cyclically),
 *   Jx(i + 1/2) = -(q w / (dt dy dz)) sum_{i' <= i} Wx(i'),
 * the running sum along x from the support's first node (the sum over all four nodes
 * is zero, so the edges b + 1/2 .. b + 5/2 carry the current).                      */
static void esirkepov_tsc(const or_grid* g, double qw, const long c0[3], const double X1[3], const double X2[3],
                          double* J)
{
    long N = ncells(g);
    double C[3] = {qw / (g->dt * g->d[1] * g->d[2]),
                   qw / (g->dt * g->d[2] * g->d[0]),
                   qw / (g->dt * g->d[0] * g->d[1])};
    long b[3];
    double S0[3][4], DS[3][4];
    for (int d = 0; d < 3; d++) {
        long m1 = (long)floor(X1[d] + 0.5), m2 = (long)floor(X2[d] + 0.5);
        b[d] = (m1 < m2 ? m1 : m2) - 1;
        for (int m = 0; m < 4; m++) {
            double node = (double)(b[d] + m);
            S0[d][m] = tsc_w(X1[d] - node);
            DS[d][m] = tsc_w(X2[d] - node) - S0[d][m];
        }
    }
    for (int comp = 0; comp < 3; comp++) {
        int p = (comp + 1) % 3, r = (comp + 2) % 3;
        for (int jp = 0; jp < 4; jp++)
            for (int jr = 0; jr < 4; jr++) {
                double acc = 0.0;
                for (int i = 0; i < 3; i++) {   /* edges b + 1/2 .. b + 5/2 along comp */
                    double W = DS[comp][i] * (S0[p][jp] * S0[r][jr] + 0.5 * DS[p][jp] * S0[r][jr]
                                              + 0.5 * S0[p][jp] * DS[r][jr] + DS[p][jp] * DS[r][jr] / 3.0);
                    acc += W;
                    long idx[3];
                    idx[comp] = c0[comp] + b[comp] + i;
                    idx[p] = c0[p] + b[p] + jp;
                    idx[r] = c0[r] + b[r] + jr;
                    long e = cell_index(g, idx[0], idx[1], idx[2]);
                    if (e >= 0 && acc != 0.0) J[comp * N + e] += -C[comp] * acc;
                }
            }
    }
}

void or_esirkepov_tsc(const int* n, const double* d, double dt, double qw, const double* X1, const double* X2,
                      double* J)
{
    or_grid g = mkgrid(n, d, dt);
    long c0[3];
    double a[3], bb[3];
    for (int k = 0; k < 3; k++) {
        c0[k] = (long)floor(X1[k]);
        a[k] = X1[k] - (double)c0[k];
        bb[k] = X2[k] - (double)c0[k];
    }
    esirkepov_tsc(&g, qw, c0, a, bb, J);
}

void or_zigzag(const int* n, const double* d, double dt, double qw, const double* X1, const double* X2, double* J)
{
    or_grid g = mkgrid(n, d, dt);
    long c0[3];
    double a[3], b[3];
    for (int k = 0; k < 3; k++) {
        c0[k] = (long)floor(X1[k]);
        a[k] = X1[k] - (double)c0[k];
        b[k] = X2[k] - (double)c0[k];
    }
    zigzag(&g, qw, c0, a, b, J);
}

/* Cloud-in-cell charge density on the nodes, section 2.5 (b1 weights),
 * rho(i+a, j+b, k+c) += q w / dV * W(dx,a) W(dy,b) W(dz,c).  A species is held
 * as C (3 rows of np integer cell indices) and P (7 rows of np values: offsets in
 * x, y, z within the cell, ux, uy, uz, w).                                     */
void or_rho(const int* n, const double* d, double q, long np, const double* P, const double* C, double* rho)
{
    or_grid g = mkgrid(n, d, 0.0);
    double dV = d[0] * d[1] * d[2];
    for (long p = 0; p < np; p++) {
        long base[3];
        double s[3];
        for (int dd = 0; dd < 3; dd++) {
            base[dd] = (long)C[dd * np + p];
            s[dd] = P[dd * np + p];
        }
        double qw = q * P[6 * np + p] / dV;
        for (int c = 0; c < 2; c++)
            for (int b = 0; b < 2; b++)
                for (int a = 0; a < 2; a++) {
                    double wgt = (a ? s[0] : 1.0 - s[0]) * (b ? s[1] : 1.0 - s[1]) * (c ? s[2] : 1.0 - s[2]);
                    long e = cell_index(&g, base[0] + a, base[1] + b, base[2] + c);
                    if (e >= 0) rho[e] += qw * wgt;
                }
    }
}

/* Charge density on the nodes with the quadratic (TSC) shape: rho(node) += q w / dV *
 * W2(X - node_x) W2(Y - node_y) W2(Z - node_z) over the 3 x 3 x 3 nearest nodes.     */
void or_rho_tsc(const int* n, const double* d, double q, long np, const double* P, const double* C, double* rho)
{
    or_grid g = mkgrid(n, d, 0.0);
    double dV = d[0] * d[1] * d[2];
    for (long p = 0; p < np; p++) {
        long base[3];
        double w[3][3];
        for (int dd = 0; dd < 3; dd++) {
            double off = P[dd * np + p];
            double m = floor(off + 0.5);
            base[dd] = (long)C[dd * np + p] + (long)m - 1;
            for (int a = 0; a < 3; a++) w[dd][a] = tsc_w(off - (m - 1.0 + a));
        }
        double qw = q * P[6 * np + p] / dV;
        for (int c = 0; c < 3; c++)
            for (int b = 0; b < 3; b++)
                for (int a = 0; a < 3; a++) {
                    long e = cell_index(&g, base[0] + a, base[1] + b, base[2] + c);
                    if (e >= 0) rho[e] += qw * w[0][a] * w[1][b] * w[2][c];
                }
    }
}

/* Discrete divergence at the nodes (backward differences of the edge
 * components), the operator of Gauss's law (2) and of continuity (12).      */
void or_divergence(const int* n, const double* d, const double* F, double* out)
{
    or_grid g = mkgrid(n, d, 0.0);
    long N = ncells(&g);
    for (long k = 0; k < n[2]; k++)
        for (long j = 0; j < n[1]; j++)
            for (long i = 0; i < n[0]; i++) {
                long c = cell_index(&g, i, j, k);
                out[c] = (F[c] - at(&g, F, i - 1, j, k)) / d[0]
                       + (F[N + c] - at(&g, F + N, i, j - 1, k)) / d[1]
                       + (F[2 * N + c] - at(&g, F + 2 * N, i, j, k - 1)) / d[2];
            }
}

/* Divergence of the magnetic field at the cell centres (i+1/2, j+1/2, k+1/2),
 * forward differences; zero by construction of the Yee scheme (section 2.3). */
void or_divergence_b(const int* n, const double* d, const double* B, double* out)
{
    or_grid g = mkgrid(n, d, 0.0);
    long N = ncells(&g);
    for (long k = 0; k < n[2]; k++)
        for (long j = 0; j < n[1]; j++)
            for (long i = 0; i < n[0]; i++) {
                long c = cell_index(&g, i, j, k);
                out[c] = (at(&g, B, i + 1, j, k) - B[c]) / d[0]
                       + (at(&g, B + N, i, j + 1, k) - B[N + c]) / d[1]
                       + (at(&g, B + 2 * N, i, j, k + 1) - B[2 * N + c]) / d[2];
            }
}

/* ------------------------------------------------------------------------ */
/* Initial momentum staggering: a Boris half step backwards in time on the
 * momentum only, u^0 -> u^{-1/2} (section 2.4, momenta at half-integer times),
 * with E^0 and B^0 = B^{-1/2} - (dt/2) curl E^0.                             */
void or_backpush(const int* n, const double* d, double dt, const double* E, const double* Bhalf,
                 double q, double m, long np, double* P, const double* C, int shape)
{
    or_grid g = mkgrid(n, d, dt);
    long N = ncells(&g);
    double* B0 = (double*)malloc(sizeof(double) * 3 * N);
    memcpy(B0, Bhalf, sizeof(double) * 3 * N);
    or_faraday(n, d, dt, E, B0, 0.5);
    for (long p = 0; p < np; p++) {
        long cell[3] = {(long)C[p], (long)C[np + p], (long)C[2 * np + p]};
        double off[3] = {P[p], P[np + p], P[2 * np + p]};
        double u[3] = {P[3 * np + p], P[4 * np + p], P[5 * np + p]};
        double Ep[3], Bp[3];
        if (shape == 2) gather_tsc(&g, E, B0, cell, off, Ep, Bp);
        else gather(&g, E, B0, cell, off, Ep, Bp);
        or_boris(q * (-0.5 * dt) / (2.0 * m), Ep, Bp, u);
        P[3 * np + p] = u[0];
        P[4 * np + p] = u[1];
        P[5 * np + p] = u[2];
    }
    free(B0);
}

/* ------------------------------------------------------------------------ */
/* One PIC cycle in the order of Fig. 2 (section 2.2):
 *   1. B^{n+1/2} = B^{n-1/2} - dt curl E^n                  (Faraday, Eq. (13))
 *   2. B^n = (B^{n+1/2} + B^{n-1/2}) / 2                     (Eq. (21))
 *   3. gather E^n, B^n at x^n; Boris u^{n-1/2} -> u^{n+1/2}; x^{n+1} = x^n + dt u/gamma
 *   4. zigzag J^{n+1/2} from the move x^n -> x^{n+1}         (section 2.5)
 *   5. E^{n+1} = E^n + dt (curl B^{n+1/2} - J^{n+1/2})       (Ampere, Eq. (14))
 * F holds 9*N values: Ex Ey Ez Bx By Bz Jx Jy Jz.  On return J holds J^{n+1/2}.
 * Species s has charge qm[2s], mass qm[2s+1], count np[s], offsets/momenta/weights
 * P[s] (7 rows) and cell indices C[s] (3 rows).
 * diag receives the energies of time level n:
 *   diag[0] = U_E = 1/2 dV sum E^n^2, diag[1] = U_B = 1/2 dV sum B^n^2,
 *   diag[2] = K = sum w m ((gamma^{n-1/2} + gamma^{n+1/2})/2 - 1).
 * Particles leaving the periodic box re-enter on the other side.  With an open x
 * dimension (n[3] = 1) particles that leave in x are removed (their weight is set
 * to 0 and they are skipped from then on), Ey and Ez of the two x faces follow the
 * first-order Mur condition, and an optional laser sheet adds to J (laser != NULL).
 * step is the index n of the cycle (time of J^{n+1/2} = (n + 1/2) dt).         */
/* Soft laser source (the external electromagnetic source module of section 2.6,
 * parameters of the laser-wakefield setup of section 4): a sheet of current J_y on the
 * node plane x = i_s, J_y = -2 a(t) exp(-r^2 / w0^2) / dx with
 * a(t) = a0 exp(-2 ln2 (t - t_p)^2 / tau^2) sin(omega (t - t_p)), tau the intensity FWHM,
 * r the distance from (yc, zc) (cell units) of the J_y point (y_{j+1/2}, z_k).  In
 * vacuum it radiates a wave of field amplitude a(t) to each side.
 * laser = {a0, omega, w0, tau, t_p, i_s, yc, zc}; t is the time of J^{n+1/2}.      */
static void laser_source(const or_grid* g, const double* laser, double t, double* J)
{
    long N = ncells(g);
    double a0 = laser[0], om = laser[1], w0 = laser[2], tau = laser[3], tp = laser[4];
    long is = (long)laser[5];
    double yc = laser[6] * g->d[1], zc = laser[7] * g->d[2];
    double s = t - tp;
    double a = a0 * exp(-2.0 * log(2.0) * s * s / (tau * tau)) * sin(om * s);
    for (long k = 0; k < g->n[2]; k++)
        for (long j = 0; j < g->n[1]; j++) {
            double y = (j + 0.5) * g->d[1] - yc, z = k * g->d[2] - zc;
            J[N + cell_index(g, is, j, k)] += -2.0 * a * exp(-(y * y + z * z) / (w0 * w0)) / g->d[0];
        }
}

/* ------------------------------------------------------------------------ */
/* Compensated binomial current filter: section 2.2 counts "compensated smoothing"
 * among the operations of a cycle and section 2.6 lists a current-filtering module,
 * without giving a scheme (the runs of section 4 use none).  Reading: along each
 * dimension, one convolution of every J component with the kernel made of `passes`
 * binomial stencils (1/4, 1/2, 1/4) and, when compensate is set, the compensating
 * stencil (-p/4, 1 + p/2, -p/4), p = passes.  Per dimension a mode of wave number k
 * is multiplied by (1 - s)^p, times (1 + p s) when compensated, s = sin^2(k d / 2):
 * the compensated product is flat to fourth order in k.  Periodic dimensions wrap;
 * along an open x the values x = 0 .. nx - 1 are filtered with zero outside them (the
 * face plane x = nx of Jy, Jz is left as it is).  It acts on the particles' current
 * after the deposit, before the laser sheet and Ampere's law.                      */
static int filter_kernel(int passes, int compensate, double* K)
{
    double cur[64] = {1.0}, nxt[64];
    int len = 1;
    double b[3] = {0.25, 0.5, 0.25};
    double c[3] = {-passes / 4.0, 1.0 + passes / 2.0, -passes / 4.0};
    int steps = passes + (compensate ? 1 : 0);
    for (int q = 0; q < steps; q++) {
        const double* st = q < passes ? b : c;
        for (int i = 0; i < len + 2; i++) nxt[i] = 0.0;
        for (int i = 0; i < len; i++)
            for (int m = 0; m < 3; m++) nxt[i + m] += cur[i] * st[m];
        len += 2;
        for (int i = 0; i < len; i++) cur[i] = nxt[i];
    }
    for (int i = 0; i < len; i++) K[i] = cur[i];
    return (len - 1) / 2;   /* half width */
}

void or_current_filter(const int* n, const double* d, double* J, int passes, int compensate)
{
    or_grid g = mkgrid(n, d, 0.0);
    long N = ncells(&g);
    double K[64];
    int h = filter_kernel(passes, compensate, K);
    long nxf = n[0];   /* x values filtered per line (the face plane of an open x is not) */
    double* tmp = (double*)malloc(sizeof(double) * N);
    for (int comp = 0; comp < 3; comp++) {
        double* A = J + comp * N;
        for (int dim = 0; dim < 3; dim++) {
            for (long k = 0; k < n[2]; k++)
                for (long j = 0; j < n[1]; j++)
                    for (long i = 0; i < nxf; i++) {
                        double sum = 0.0;
                        for (int m = -h; m <= h; m++) {
                            long ii = i + (dim == 0 ? m : 0), jj = j + (dim == 1 ? m : 0), kk = k + (dim == 2 ? m : 0);
                            if (g.open_x && (ii < 0 || ii >= nxf)) continue;   /* zero outside */
                            sum += K[m + h] * A[cell_index(&g, ii, jj, kk)];
                        }
                        tmp[cell_index(&g, i, j, k)] = sum;
                    }
            for (long k = 0; k < n[2]; k++)
                for (long j = 0; j < n[1]; j++)
                    for (long i = 0; i < nxf; i++) A[cell_index(&g, i, j, k)] = tmp[cell_index(&g, i, j, k)];
        }
    }
    free(tmp);
}

/* ------------------------------------------------------------------------ */
/* Perfectly conducting walls and a waveguide port (section 3.2: the Yee solver is
 * verified on the TE10 mode of a perfectly conducting rectangular guide driven at its
 * input plane; the paper gives no discretisation of either).
 * guide = {pec_y, pec_z, port, e0, omega, tau, mode_y, deposit, shape}; deposit = 1
 * selects Esirkepov's deposit instead of ZigZag (see esirkepov); shape = 2 selects the
 * quadratic (TSC) particle shape for the gather and Esirkepov's deposit (see tsc_w).
 * pec_y: the node plane y = 0 is a perfect conductor, its tangential Ex and Ez are
 *   held at zero; with y periodic that plane is both walls of a guide 0 <= y <= ny.
 * pec_z: likewise the plane z = 0 (Ex, Ey).
 * port (open x only): a hard source on the face x = 0 that replaces the absorbing
 *   condition there: Ez(0, j, k) = e0 g(t) sin(mode_y pi j / ny) sin(omega t), Ey(0, j, k)
 *   = 0, g(t) = 1 - exp(-t / tau), t the time of the new E (the envelope of section
 *   3.2 that suppresses the start-up transient).
 * Applied after Ampere's law (and the Mur faces): port first, then the walls.       */
static void port_source(const or_grid* g, const double* guide, double t, double* E)
{
    long N = ncells(g);
    double e0 = guide[3], om = guide[4], tau = guide[5];
    double m = guide[6];
    double amp = e0 * (1.0 - exp(-t / tau)) * sin(om * t);
    for (long k = 0; k < g->n[2]; k++)
        for (long j = 0; j < g->n[1]; j++) {
            E[N + cell_index(g, 0, j, k)] = 0.0;
            E[2 * N + cell_index(g, 0, j, k)] = amp * sin(m * M_PI * (double)j / g->n[1]);
        }
}

static void pec_walls(const or_grid* g, const double* guide, double* E)
{
    long N = ncells(g);
    for (long k = 0; k < g->n[2]; k++)
        for (long j = 0; j < g->n[1]; j++)
            for (long i = 0; i < g->nxs; i++) {
                long c = cell_index(g, i, j, k);
                if (guide[0] != 0 && j == 0) { E[c] = 0.0; E[2 * N + c] = 0.0; }
                if (guide[1] != 0 && k == 0) { E[c] = 0.0; E[N + c] = 0.0; }
            }
}

/* The particle part of the cycle (section 2.2, Fig. 2, steps 3-4) for one species of
 * charge q and mass m: gather E^n, B^n at x^n (Bn holds B^n), Boris push, move, and the
 * current of the move into J (ZigZag, or Esirkepov when esk is set); a particle that
 * leaves an open x is removed (weight 0).  Returns the species' kinetic energy at time
 * level n, sum w m ((gamma^{n-1/2} + gamma^{n+1/2}) / 2 - 1).                       */
static double push_species(const or_grid* gp, double q, double m, long cnt, double* Ps, double* Cs,
                           const double* E, const double* Bn, double* J, int esk, int shape)
{
    const or_grid g = *gp;
    const int* n = g.n;
    const double* d = g.d;
    double dt = g.dt;
    double K = 0.0;
    for (long p = 0; p < cnt; p++) {
        if (Ps[6 * cnt + p] == 0.0) continue;   /* removed through an open face */
        long cell[3] = {(long)Cs[p], (long)Cs[cnt + p], (long)Cs[2 * cnt + p]};
        double X1[3] = {Ps[p], Ps[cnt + p], Ps[2 * cnt + p]};          /* offsets: X relative to cell */
        double u[3] = {Ps[3 * cnt + p], Ps[4 * cnt + p], Ps[5 * cnt + p]};
        double w = Ps[6 * cnt + p];
        double Ep[3], Bp[3];
        if (shape == 2) gather_tsc(&g, E, Bn, cell, X1, Ep, Bp);
        else gather(&g, E, Bn, cell, X1, Ep, Bp);
        double g_old = gamma_of(u);
        or_boris(q * dt / (2.0 * m), Ep, Bp, u);
        double g_new = gamma_of(u);
        K += w * m * (0.5 * (g_old + g_new) - 1.0);
        double X2[3];
        for (int dd = 0; dd < 3; dd++) X2[dd] = X1[dd] + dt * u[dd] / (g_new * d[dd]);
        if (shape == 2) esirkepov_tsc(&g, q * w, cell, X1, X2, J);
        else if (esk) esirkepov(&g, q * w, cell, X1, X2, J);
        else zigzag(&g, q * w, cell, X1, X2, J);
        int gone = 0;
        for (int dd = 0; dd < 3; dd++) {
            /* new cell and offset; an offset that rounds to 1 starts the next cell */
            double f = floor(X2[dd]);
            double o = X2[dd] - f;
            long cn = cell[dd] + (long)f;
            if (o >= 1.0) { o = 0.0; cn += 1; }
            if (dd == 0 && g.open_x && (cn < 0 || cn >= n[0])) gone = 1;
            Cs[dd * cnt + p] = (double)wrapi(cn, n[dd]);
            Ps[dd * cnt + p] = o;
        }
        if (gone) Ps[6 * cnt + p] = 0.0;
        Ps[3 * cnt + p] = u[0];
        Ps[4 * cnt + p] = u[1];
        Ps[5 * cnt + p] = u[2];
    }
    return K;
}

/* push_species as an entry point: E and Bn (B^n) are read, J is added to.             */
double or_push(const int* n, const double* d, double dt, const double* E, const double* Bn, double q, double m, long np,
               double* P, double* C, double* J, int esk, int shape)
{
    or_grid g = mkgrid(n, d, dt);
    return push_species(&g, q, m, np, P, C, E, Bn, J, esk, shape);
}

void or_step(const int* n, const double* d, double dt, double* F, int ns, const double* qm, const long* np,
             double** P, double** C, double* diag, long step, const double* laser, const double* filt,
             const double* guide)
{
    or_grid g = mkgrid(n, d, dt);
    long N = ncells(&g);
    double dV = d[0] * d[1] * d[2];
    double *E = F, *B = F + 3 * N, *J = F + 6 * N;

    double* Bold = (double*)malloc(sizeof(double) * 3 * N);
    double* Bn = (double*)malloc(sizeof(double) * 3 * N);
    memcpy(Bold, B, sizeof(double) * 3 * N);
    or_faraday(n, d, dt, E, B, 1.0);                      /* B now holds B^{n+1/2} */
    for (long c = 0; c < 3 * N; c++) Bn[c] = 0.5 * (B[c] + Bold[c]);

    double UE = 0.0, UB = 0.0, K = 0.0;
    for (long c = 0; c < 3 * N; c++) { UE += E[c] * E[c]; UB += Bn[c] * Bn[c]; }

    for (long c = 0; c < 3 * N; c++) J[c] = 0.0;
    for (int s = 0; s < ns; s++) {
        double q = qm[2 * s], m = qm[2 * s + 1];
        double* Ps = P[s];
        double* Cs = C[s];
        long cnt = np[s];
        K += push_species(&g, q, m, cnt, Ps, Cs, E, Bn, J, guide && guide[7] != 0, guide ? (int)guide[8] : 1);
    }
    if (filt && filt[0] > 0) or_current_filter(n, d, J, (int)filt[0], (int)filt[1]);
    if (laser) laser_source(&g, laser, (step + 0.5) * dt, J);
    double* old = NULL;
    if (g.open_x) {
        /* Ey, Ez of planes 0, 1, nx-1, nx before the update, for the Mur condition */
        long Pn = (long)n[1] * n[2];
        long planes[4] = {0, 1, n[0] - 1, n[0]};
        old = (double*)malloc(sizeof(double) * 8 * Pn);
        for (int comp = 1; comp <= 2; comp++)
            for (int q = 0; q < 4; q++)
                for (long k = 0; k < n[2]; k++)
                    for (long j = 0; j < n[1]; j++)
                        old[((comp - 1) * 4 + q) * Pn + k * n[1] + j] = E[comp * N + cell_index(&g, planes[q], j, k)];
    }
    or_ampere(n, d, dt, E, B, J);
    if (old) {
        mur_x(&g, old, E);
        free(old);
    }
    if (guide) {
        if (guide[2] != 0 && g.open_x) port_source(&g, guide, (step + 1) * dt, E);
        if (guide[0] != 0 || guide[1] != 0) pec_walls(&g, guide, E);
    }
    diag[0] = 0.5 * dV * UE;
    diag[1] = 0.5 * dV * UB;
    diag[2] = K;
    free(Bold);
    free(Bn);
}

/* Several cycles; diag receives 3 values per step.                          */
void or_run(const int* n, const double* d, double dt, double* F, int ns, const double* qm, const long* np,
            double** P, double** C, long nsteps, double* diag, long step0, const double* laser, const double* filt,
            const double* guide)
{
    for (long s = 0; s < nsteps; s++)
        or_step(n, d, dt, F, ns, qm, np, P, C, diag + 3 * s, step0 + s, laser, filt, guide);
}

/* ------------------------------------------------------------------------ */
/* Moving window (section 2.2: one of the operations at the end of a cycle, before the
 * next one begins; section 4: the laser-wakefield run moves its window).  On an open x
 * dimension (n[3] = 1) the window moves one cell along +x:
 *   - every E and B value takes the value one cell further along x, and the new last
 *     value of each line is vacuum (zero): the x-node components Ey, Ez, Bx end at the
 *     face plane x = nx, the x-half components Ex, By, Bz at x = nx - 1/2;
 *   - every particle's x cell drops by one; a particle that was in cell 0 leaves the
 *     window (its weight is set to 0, as for a particle leaving through a face).
 * J is left as it is (the next cycle recomputes it).  The new plasma of the last
 * column is added by the caller.                                                  */
void or_window_shift(const int* n, const double* d, double* F, int ns, const long* np, double** P, double** C)
{
    or_grid g = mkgrid(n, d, 0.0);
    long N = ncells(&g);
    int nx = n[0];
    if (!g.open_x) return;
    for (int comp = 0; comp < 6; comp++) {
        int x_node = (comp == 1 || comp == 2 || comp == 3);   /* Ey, Ez, Bx */
        long last = x_node ? nx : nx - 1;
        double* A = F + comp * N;
        for (long k = 0; k < n[2]; k++)
            for (long j = 0; j < n[1]; j++) {
                for (long i = 0; i < last; i++) A[cell_index(&g, i, j, k)] = A[cell_index(&g, i + 1, j, k)];
                A[cell_index(&g, last, j, k)] = 0.0;
            }
    }
    for (int s = 0; s < ns; s++) {
        long cnt = np[s];
        for (long p = 0; p < cnt; p++) {
            if (P[s][6 * cnt + p] == 0.0) continue;   /* already removed */
            if (C[s][p] < 1.0) {
                P[s][6 * cnt + p] = 0.0;               /* cell 0 leaves the window */
            } else {
                C[s][p] -= 1.0;
            }
        }
    }
}

/* Gauss's law for an initial state whose charge varies along x only
 * (section 2.3, Eq. (2) in discrete form): Ex(i+1/2) = Ex(i-1/2) + dx rho(i)
 * along every x line, with zero line mean.  rho_total includes the ion
 * background.  Ey = Ez = 0.  Returns the largest |line mean of rho_total|,
 * which must vanish for the result to satisfy div E = rho exactly.          */
double or_gauss_x(const int* n, const double* d, const double* rho_total, double* E)
{
    or_grid g = mkgrid(n, d, 0.0);
    long N = ncells(&g);
    double worst = 0.0;
    for (long c = 0; c < 3 * N; c++) E[c] = 0.0;
    for (long k = 0; k < n[2]; k++)
        for (long j = 0; j < n[1]; j++) {
            double mean_rho = 0.0;
            for (long i = 0; i < n[0]; i++) mean_rho += rho_total[cell_index(&g, i, j, k)];
            mean_rho /= n[0];
            if (fabs(mean_rho) > worst) worst = fabs(mean_rho);
            /* Ex(i+1/2) - Ex(i-1/2) = dx rho(i)  <=>  Ex[i] = Ex[i-1] + dx rho(i) */
            double acc = 0.0, mean_e = 0.0;
            for (long i = 0; i < n[0]; i++) {
                acc += d[0] * rho_total[cell_index(&g, i, j, k)];
                E[cell_index(&g, i, j, k)] = acc;
                mean_e += acc;
            }
            mean_e /= n[0];
            for (long i = 0; i < n[0]; i++) E[cell_index(&g, i, j, k)] -= mean_e;
        }
    return worst;
}
