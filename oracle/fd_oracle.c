/*
 * Plain FP64 CPU oracle for the sixth-order finite-difference, 2N-storage
 * RK3 solver of isothermal compressible hydrodynamics described in
 * Pekkila, Vaisala, Kapyla, Kapyla & Anjum (2017), "Methods for compressible
 * fluid simulation on GPUs using high-order finite differences".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline / reference legs load this library; the product
 * path (the CUDA library) never calls it and shares no code with it.
 *
 * Everything here is the paper's definitions written out point by point:
 *   - first derivative ............... Eq. 6  (Sect. 2.3)
 *   - second derivative .............. Eq. 7  (read with 1/(180 dx^2); the
 *                                      printed 1/(180 dx) is dimensionally
 *                                      inconsistent)
 *   - bidiagonal mixed derivative .... Eq. 8
 *   - nested first derivatives ....... Eq. 9  (19-point form: D1 of the
 *                                      stored D1-divergence)
 *   - continuity ..................... Eq. 1, log-density form
 *   - momentum ....................... Eq. 2; the body force f = 0, or the
 *                                      non-helical random-k forcing of
 *                                      Sect. 6 (Eqs. 20-21) for one step:
 *                                      f = N f_k cos(k.x + phi),
 *                                      N = f0 c_s sqrt(|k| c_s / dt),
 *                                      f_k = k x e / sqrt(|k|^2 - (k.e)^2)
 *   - traceless rate of strain ....... Eq. 3
 *   - 2N-storage RK3 ................. Eq. 10, Algorithm 2 (55-point,
 *                                      single pass) and Algorithm 3 with
 *                                      Eqs. 14-16 / Appendix A (19-point,
 *                                      two passes)
 * The RK3 coefficients are not printed in the paper (Sect. 2.4 only fixes
 * alpha_1 = 0); they are Williamson's (1980) low-storage third-order set
 * alpha = (0, -5/9, -153/128), beta = (1/3, 15/16, 8/15).
 *
 * Grid (Sect. 2.3): N_i equidistant points per axis, spacing L_i / N_i,
 * periodic in every axis (Sect. 4); periodic wrap is plain modular indexing,
 * there are no ghost zones.  The wall variant (the "_wall" routines) keeps x
 * and y periodic and bounds z by two walls through the grid points z = 0
 * and z = Lz (spacing Lz / (N_z - 1)); the paper's ghost zones (Sect. 4,
 * Algorithm 1's boundary step) then carry the boundary condition: arrays
 * hold 3 ghost planes below and above the N_z interior planes, and before
 * each substep (and before the 19-point form's second pass, for the stored
 * divergence) they are filled as the mirror images of the interior about
 * the wall points, f(-k) = p f(k) and f(N_z-1+k) = p f(N_z-1-k), with parity
 * p = +1 for lnrho, u_x, u_y, s and the divergence and p = -1 for u_z: an
 * impermeable, free-slip wall.  The paper defines no boundary condition
 * besides periodic; this one is the reading of the ghost-zone mechanism
 * whose exact solution is known: the periodic solution on 2 (N_z - 1)
 * planes of the mirror-extended state.  Fields are stored [field][z][y][x] with x
 * fastest; the field order is (lnrho, u_x, u_y, u_z[, s]).  The paper's model
 * is isothermal and carries no energy variable: with entropy_mode = 0 the
 * state has the paper's four fields; with entropy_mode = 1 a fifth field s is
 * carried and advected passively (ds/dt = -u . grad s), with no feedback on
 * the flow.
 *
 * No blocking, fusion or reordering beyond what the definitions state.  The
 * file is compiled with -ffp-contract=off so that the compiler introduces no
 * fused multiply-adds.  Sums in the diagnostics use Neumaier's compensated
 * summation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Point stencils: one definition each, used by every grid routine.     */
/* ------------------------------------------------------------------ */

/* Eq. 6: d f / dx at sample 3 of s[0..6] (offsets -3..+3), spacing h. */
double or_d1_point(const double *s, double h)
{
    return (-s[0] + 9.0 * s[1] - 45.0 * s[2] + 45.0 * s[4] - 9.0 * s[5] + s[6]) / (60.0 * h);
}

/* Eq. 7: d^2 f / dx^2 at sample 3 of s[0..6], spacing h (1/(180 h^2)). */
double or_d2_point(const double *s, double h)
{
    return (2.0 * s[0] - 27.0 * s[1] + 270.0 * s[2] - 490.0 * s[3] + 270.0 * s[4] - 27.0 * s[5] +
            2.0 * s[6]) /
           (180.0 * h * h);
}

/* Eq. 8: d^2 f / (da db) at the centre of a 7x7 sample patch,
 * s[7*ia + ib] = f(a + (ia-3) ha, b + (ib-3) hb).  Only the two diagonals
 * of the patch enter (the "bidiagonal" scheme). */
double or_dmix_point(const double *s, double ha, double hb)
{
#define S(ia, ib) s[7 * ((ia) + 3) + ((ib) + 3)]
    double k1 = S(1, 1) - S(-1, 1) + S(-1, -1) - S(1, -1);
    double k2 = S(2, 2) - S(-2, 2) + S(-2, -2) - S(2, -2);
    double k3 = S(3, 3) - S(-3, 3) + S(-3, -3) - S(3, -3);
#undef S
    return (270.0 * k1 - 27.0 * k2 + 2.0 * k3) / (720.0 * ha * hb);
}

/* ------------------------------------------------------------------ */
/* Periodic grid                                                        */
/* ------------------------------------------------------------------ */

typedef struct {
    long n[3];   /* points per axis: x, y, z (interior points) */
    double h[3]; /* spacing L_i / N_i (L_z / (N_z - 1) between walls) */
    long gz;     /* ghost planes below and above the interior in z: 0
                    (periodic z) or 3 (walls) */
    long npts;   /* values stored per field: N_x N_y (N_z + 2 gz) */
} grid_t;

#define GZ_WALL 3

/* gz = 0: periodic z; gz = 3 with walls (spacing lz / (nz - 1)), or a
 * z-slab of a periodic domain whose ghost planes hold the neighbouring
 * slabs' planes (walls = 0: spacing lz / nz) */
static grid_t make_grid_gw(long nx, long ny, long nz, double lx, double ly, double lz, long gz,
                           int walls)
{
    grid_t g;
    g.n[0] = nx;
    g.n[1] = ny;
    g.n[2] = nz;
    g.h[0] = lx / (double)nx;
    g.h[1] = ly / (double)ny;
    g.h[2] = walls ? lz / (double)(nz - 1) : lz / (double)nz;
    g.gz = gz;
    g.npts = nx * ny * (nz + 2 * gz);
    return g;
}

static grid_t make_grid_bc(long nx, long ny, long nz, double lx, double ly, double lz, long gz)
{
    return make_grid_gw(nx, ny, nz, lx, ly, lz, gz, gz != 0);
}

static grid_t make_grid(long nx, long ny, long nz, double lx, double ly, double lz)
{
    return make_grid_bc(nx, ny, nz, lx, ly, lz, 0);
}

static inline long wrap(long i, long n)
{
    long r = i % n;
    return r < 0 ? r + n : r;
}

/* linear index of point p = (x, y, z): x and y wrapped periodically; z
 * wrapped too, or (walls) taken as is from the ghost-extended array, whose
 * z = -gz .. N_z - 1 + gz planes are all stored */
static inline long at(const grid_t *g, const long *p)
{
    const long z = g->gz ? p[2] + g->gz : wrap(p[2], g->n[2]);
    return (z * g->n[1] + wrap(p[1], g->n[1])) * g->n[0] + wrap(p[0], g->n[0]);
}

/* 7 samples of f along `axis` centred on p */
static void gather_axis(const double *f, const grid_t *g, const long *p, int axis, double *s)
{
    for (int m = -3; m <= 3; ++m) {
        long q[3] = {p[0], p[1], p[2]};
        q[axis] += m;
        s[m + 3] = f[at(g, q)];
    }
}

/* 7x7 samples of f in the (a, b) plane centred on p */
static void gather_plane(const double *f, const grid_t *g, const long *p, int a, int b, double *s)
{
    for (int ia = -3; ia <= 3; ++ia)
        for (int ib = -3; ib <= 3; ++ib) {
            long q[3] = {p[0], p[1], p[2]};
            q[a] += ia;
            q[b] += ib;
            s[7 * (ia + 3) + (ib + 3)] = f[at(g, q)];
        }
}

static double d1(const double *f, const grid_t *g, const long *p, int axis)
{
    double s[7];
    gather_axis(f, g, p, axis, s);
    return or_d1_point(s, g->h[axis]);
}

static double d2(const double *f, const grid_t *g, const long *p, int axis)
{
    double s[7];
    gather_axis(f, g, p, axis, s);
    return or_d2_point(s, g->h[axis]);
}

static double dmix(const double *f, const grid_t *g, const long *p, int a, int b)
{
    double s[49];
    gather_plane(f, g, p, a, b, s);
    return or_dmix_point(s, g->h[a], g->h[b]);
}

/* Whole-grid derivative operators (used by the stencil pins). */
void or_grid_d1(const double *f, double *out, long nx, long ny, long nz, double lx, double ly,
                double lz, int axis)
{
    grid_t g = make_grid(nx, ny, nz, lx, ly, lz);
    for (long z = 0; z < nz; ++z)
        for (long y = 0; y < ny; ++y)
            for (long x = 0; x < nx; ++x) {
                long p[3] = {x, y, z};
                out[at(&g, p)] = d1(f, &g, p, axis);
            }
}

void or_grid_d2(const double *f, double *out, long nx, long ny, long nz, double lx, double ly,
                double lz, int axis)
{
    grid_t g = make_grid(nx, ny, nz, lx, ly, lz);
    for (long z = 0; z < nz; ++z)
        for (long y = 0; y < ny; ++y)
            for (long x = 0; x < nx; ++x) {
                long p[3] = {x, y, z};
                out[at(&g, p)] = d2(f, &g, p, axis);
            }
}

void or_grid_dmix(const double *f, double *out, long nx, long ny, long nz, double lx, double ly,
                  double lz, int a, int b)
{
    grid_t g = make_grid(nx, ny, nz, lx, ly, lz);
    for (long z = 0; z < nz; ++z)
        for (long y = 0; y < ny; ++y)
            for (long x = 0; x < nx; ++x) {
                long p[3] = {x, y, z};
                out[at(&g, p)] = dmix(f, &g, p, a, b);
            }
}

/* ------------------------------------------------------------------ */
/* Right-hand side, Eqs. 1-3                                            */
/* ------------------------------------------------------------------ */

typedef struct {
    double cs2; /* c_s^2 */
    double nu;  /* kinematic viscosity */
    int entropy_mode;
    int nfields;
} phys_t;

/* The external force of Eq. 2 for one time step, Sect. 6 (Eqs. 20-21):
 * f(x) = Re{ N f_k exp(i k.x + i phi) } = N f_k cos(k.x + phi), f_k real. */
typedef struct {
    int on;
    double k[3];   /* wave vector, physical units */
    double phi;    /* phase */
    double amp[3]; /* N f_k */
} forcing_t;

/* N f_k of Eq. 21 for the integer wave vector kint (physical k_i =
 * 2 pi kint_i / L_i), the unit vector e, the scale f0, the sound speed and
 * the time step:  N = f0 c_s sqrt(|k| c_s / dt),
 * f_k = (k x e) / sqrt(|k|^2 - (k.e)^2).  Returns 0, or -1 when k is zero
 * or parallel to e (f_k undefined). */
int or_forcing_amplitude(const long *kint, const double *e, double f0, double cs, double dt,
                         double lx, double ly, double lz, double *amp)
{
    const double two_pi = 6.283185307179586476925286766559;
    const double k[3] = {two_pi * (double)kint[0] / lx, two_pi * (double)kint[1] / ly,
                         two_pi * (double)kint[2] / lz};
    const double kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    const double ke = k[0] * e[0] + k[1] * e[1] + k[2] * e[2];
    const double den2 = kk - ke * ke;
    if (!(kk > 0.0) || !(den2 > 1e-24 * kk))
        return -1;
    const double kn = sqrt(kk);
    const double N = f0 * cs * sqrt(kn * cs / dt);
    const double kxe[3] = {k[1] * e[2] - k[2] * e[1], k[2] * e[0] - k[0] * e[2],
                           k[0] * e[1] - k[1] * e[0]};
    const double den = sqrt(den2);
    for (int i = 0; i < 3; ++i)
        amp[i] = N * kxe[i] / den;
    return 0;
}

static int make_forcing(forcing_t *fo, const long *kint, double phi, const double *e, double f0,
                        double cs, double dt, double lx, double ly, double lz)
{
    const double two_pi = 6.283185307179586476925286766559;
    fo->on = 1;
    fo->k[0] = two_pi * (double)kint[0] / lx;
    fo->k[1] = two_pi * (double)kint[1] / ly;
    fo->k[2] = two_pi * (double)kint[2] / lz;
    fo->phi = phi;
    return or_forcing_amplitude(kint, e, f0, cs, dt, lx, ly, lz, fo->amp);
}

/* Terms of Eqs. 1-3 at point p that need only first and second derivatives
 * along the axes (everything except the grad(div u) term of Eq. 2).
 * rhs[0] = d lnrho/dt, rhs[1..3] = du_i/dt without (nu/3) grad(div u),
 * rhs[4] = ds/dt (when carried).  Also returns div u and the first
 * derivatives it was built from. */
static void rhs_axial(const double *state, const grid_t *g, const phys_t *ph, const long *p,
                      const forcing_t *fo, double *rhs)
{
    const long n = g->npts;
    const double *lnrho = state;
    const double *u[3] = {state + n, state + 2 * n, state + 3 * n};
    const long c = at(g, p);

    double uc[3], glnrho[3], gu[3][3]; /* gu[i][j] = d_j u_i */
    for (int i = 0; i < 3; ++i)
        uc[i] = u[i][c];
    for (int j = 0; j < 3; ++j)
        glnrho[j] = d1(lnrho, g, p, j);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            gu[i][j] = d1(u[i], g, p, j);

    double divu = gu[0][0] + gu[1][1] + gu[2][2];

    /* Eq. 1: d lnrho / dt = -u . grad lnrho - div u */
    double adv_lnrho = 0.0;
    for (int j = 0; j < 3; ++j)
        adv_lnrho += uc[j] * glnrho[j];
    rhs[0] = -adv_lnrho - divu;

    /* Eq. 3: S_ij = (d_j u_i + d_i u_j - (2/3) delta_ij div u) / 2 */
    double S[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            S[i][j] = 0.5 * (gu[i][j] + gu[j][i] - (i == j ? (2.0 / 3.0) * divu : 0.0));

    /* Eq. 2 without the (nu/3) grad(div u) term and with f = 0:
     * du_i/dt = -(u . grad) u_i - c_s^2 d_i lnrho
     *           + nu (lap u_i + 2 (S . grad lnrho)_i) */
    for (int i = 0; i < 3; ++i) {
        double adv = 0.0, lap = 0.0, sgl = 0.0;
        for (int j = 0; j < 3; ++j) {
            adv += uc[j] * gu[i][j];
            lap += d2(u[i], g, p, j);
            sgl += S[i][j] * glnrho[j];
        }
        rhs[1 + i] = -adv - ph->cs2 * glnrho[i] + ph->nu * (lap + 2.0 * sgl);
    }

    /* Eq. 2's f: the forcing of Eq. 20 at x = (x_i, y_j, z_l) = grid point p */
    if (fo && fo->on) {
        const double phase = fo->k[0] * (double)p[0] * g->h[0] + fo->k[1] * (double)p[1] * g->h[1] +
                             fo->k[2] * (double)p[2] * g->h[2] + fo->phi;
        const double cph = cos(phase);
        for (int i = 0; i < 3; ++i)
            rhs[1 + i] += fo->amp[i] * cph;
    }

    /* passive entropy: ds/dt = -u . grad s */
    if (ph->nfields == 5) {
        const double *s = state + 4 * n;
        double adv_s = 0.0;
        for (int j = 0; j < 3; ++j)
            adv_s += uc[j] * d1(s, g, p, j);
        rhs[4] = -adv_s;
    }
}

/* d_i (div u) at p in the 55-point form: d_i d_j u_j with the second
 * derivative (Eq. 7) for i == j and the bidiagonal scheme (Eq. 8) for
 * i != j. */
static void graddiv55(const double *state, const grid_t *g, const long *p, double *gd)
{
    const long n = g->npts;
    const double *u[3] = {state + n, state + 2 * n, state + 3 * n};
    for (int i = 0; i < 3; ++i) {
        double acc = 0.0;
        for (int j = 0; j < 3; ++j)
            acc += (i == j) ? d2(u[j], g, p, i) : dmix(u[j], g, p, i, j);
        gd[i] = acc;
    }
}

/* div u at p from first derivatives (Eq. 6); the stored field of the
 * 19-point form's first pass. */
static double divergence(const double *state, const grid_t *g, const long *p)
{
    const long n = g->npts;
    return d1(state + n, g, p, 0) + d1(state + 2 * n, g, p, 1) + d1(state + 3 * n, g, p, 2);
}

static phys_t make_phys(double cs, double nu, int entropy_mode)
{
    phys_t ph;
    ph.cs2 = cs * cs;
    ph.nu = nu;
    ph.entropy_mode = entropy_mode;
    ph.nfields = entropy_mode ? 5 : 4;
    return ph;
}

/* Full right-hand side d(state)/dt of Eqs. 1-3 on the whole grid.
 * form 0: 55-point (grad div u from Eqs. 7-8);
 * form 1: 19-point (grad div u as D1 of the D1-divergence, Eq. 9). */
static void rhs_grid(const double *state, double *rhs, long nx, long ny, long nz, double lx,
                     double ly, double lz, double cs, double nu, int entropy_mode, int form,
                     const forcing_t *fo)
{
    grid_t g = make_grid(nx, ny, nz, lx, ly, lz);
    phys_t ph = make_phys(cs, nu, entropy_mode);
    const long n = g.npts;
    double *divf = NULL;
    if (form == 1) {
        divf = (double *)malloc(sizeof(double) * n);
        for (long z = 0; z < nz; ++z)
            for (long y = 0; y < ny; ++y)
                for (long x = 0; x < nx; ++x) {
                    long p[3] = {x, y, z};
                    divf[at(&g, p)] = divergence(state, &g, p);
                }
    }
    for (long z = 0; z < nz; ++z)
        for (long y = 0; y < ny; ++y)
            for (long x = 0; x < nx; ++x) {
                long p[3] = {x, y, z};
                long c = at(&g, p);
                double r[5], gd[3];
                rhs_axial(state, &g, &ph, p, fo, r);
                if (form == 1) {
                    for (int i = 0; i < 3; ++i)
                        gd[i] = d1(divf, &g, p, i);
                } else {
                    graddiv55(state, &g, p, gd);
                }
                for (int i = 0; i < 3; ++i)
                    r[1 + i] += (ph.nu / 3.0) * gd[i];
                for (int f = 0; f < ph.nfields; ++f)
                    rhs[f * n + c] = r[f];
            }
    free(divf);
}

void or_rhs(const double *state, double *rhs, long nx, long ny, long nz, double lx, double ly,
            double lz, double cs, double nu, int entropy_mode, int form)
{
    rhs_grid(state, rhs, nx, ny, nz, lx, ly, lz, cs, nu, entropy_mode, form, NULL);
}

/* The right-hand side with the forcing of Sect. 6 (Eqs. 20-21) for wave
 * vector kint (integers, k_i = 2 pi kint_i / L_i), phase phi, unit vector e,
 * scale f0 and time step dt (N depends on dt).  Returns -1 when f_k is
 * undefined (k zero or parallel to e). */
int or_rhs_forced(const double *state, double *rhs, long nx, long ny, long nz, double lx,
                  double ly, double lz, double cs, double nu, int entropy_mode, int form,
                  double dt, double f0, const long *kint, double phi, const double *e)
{
    forcing_t fo;
    if (make_forcing(&fo, kint, phi, e, f0, cs, dt, lx, ly, lz))
        return -1;
    rhs_grid(state, rhs, nx, ny, nz, lx, ly, lz, cs, nu, entropy_mode, form, &fo);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Ghost zones of the wall variant (Sect. 4; Algorithm 1's boundary step) */
/* ------------------------------------------------------------------ */

/* Fill the 3 ghost planes below and above the N_z interior planes of each
 * of nf fields of a ghost-extended array (N_z + 6 planes of N_y x N_x per
 * field, interior plane z at index z + 3): mirror images about the wall
 * points z = 0 and z = N_z - 1, scaled by the field's parity (+1 or -1):
 *   f(-k) = parity f(k),  f(N_z - 1 + k) = parity f(N_z - 1 - k),  k = 1..3. */
void or_fill_ghosts_z(double *st, long nx, long ny, long nz, int nf, const double *parity)
{
    const long plane = nx * ny;
    const long fpitch = plane * (nz + 2 * GZ_WALL);
    for (int f = 0; f < nf; ++f) {
        double *a = st + f * fpitch + GZ_WALL * plane; /* interior plane 0 */
        for (long k = 1; k <= GZ_WALL; ++k)
            for (long c = 0; c < plane; ++c) {
                a[-k * plane + c] = parity[f] * a[k * plane + c];
                a[(nz - 1 + k) * plane + c] = parity[f] * a[(nz - 1 - k) * plane + c];
            }
    }
}

/* ------------------------------------------------------------------ */
/* 2N-storage RK3, Eq. 10                                               */
/* ------------------------------------------------------------------ */

static const double RK3_ALPHA[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
static const double RK3_BETA[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};

void or_rk3_coefficients(double *alpha, double *beta)
{
    for (int s = 0; s < 3; ++s) {
        alpha[s] = RK3_ALPHA[s];
        beta[s] = RK3_BETA[s];
    }
}

/* Eq. 10 for one value: w <- alpha w + dt r (alpha_1 = 0, so the first
 * substep does not look at the previous w), out <- in + beta w. */
static inline void rk3_update(int s, double dt, double r, double in, double *w, double *out)
{
    double wn = (s == 0) ? dt * r : RK3_ALPHA[s] * (*w) + dt * r;
    *w = wn;
    *out = in + RK3_BETA[s] * wn;
}

/* One substep s (0, 1, 2) of Algorithm 2 (55-point, single pass): reads
 * `in` and `w` (the 2N register, u-tilde), writes `out` and `w`. */
static void substep55(const double *in, double *w, double *out, int s, double dt, long nx,
                      long ny, long nz, double lx, double ly, double lz, double cs, double nu,
                      int entropy_mode, const forcing_t *fo, long gz, int walls)
{
    grid_t g = make_grid_gw(nx, ny, nz, lx, ly, lz, gz, walls);
    phys_t ph = make_phys(cs, nu, entropy_mode);
    const long n = g.npts;
#pragma omp parallel for schedule(static)
    for (long z = 0; z < nz; ++z)
        for (long y = 0; y < ny; ++y)
            for (long x = 0; x < nx; ++x) {
                long p[3] = {x, y, z};
                long c = at(&g, p);
                double r[5], gd[3];
                rhs_axial(in, &g, &ph, p, fo, r);
                graddiv55(in, &g, p, gd);
                for (int i = 0; i < 3; ++i)
                    r[1 + i] += (ph.nu / 3.0) * gd[i];
                for (int f = 0; f < ph.nfields; ++f)
                    rk3_update(s, dt, r[f], in[f * n + c], &w[f * n + c], &out[f * n + c]);
            }
}

/* One substep s of Algorithm 3 (19-point, two passes, Eqs. 14-16).
 * Pass 1 stores div u in `divf` and completes lnrho (and s) while the
 * velocity gets the partial update without (nu/3) grad(div u); pass 2
 * adds dt (nu/3) grad(div u) to w and beta dt (nu/3) grad(div u) to out,
 * with grad taken by Eq. 6 on the stored divergence (Eq. 9). */
static void substep19(const double *in, double *w, double *out, double *divf, int s, double dt,
                      long nx, long ny, long nz, double lx, double ly, double lz, double cs,
                      double nu, int entropy_mode, const forcing_t *fo, long gz)
{
    grid_t g = make_grid_bc(nx, ny, nz, lx, ly, lz, gz);
    phys_t ph = make_phys(cs, nu, entropy_mode);
    const long n = g.npts;
    /* pass 1 */
#pragma omp parallel for schedule(static)
    for (long z = 0; z < nz; ++z)
        for (long y = 0; y < ny; ++y)
            for (long x = 0; x < nx; ++x) {
                long p[3] = {x, y, z};
                long c = at(&g, p);
                double r[5];
                divf[c] = divergence(in, &g, p);
                rhs_axial(in, &g, &ph, p, fo, r);
                for (int f = 0; f < ph.nfields; ++f)
                    rk3_update(s, dt, r[f], in[f * n + c], &w[f * n + c], &out[f * n + c]);
            }
    /* the stored divergence is symmetric about a wall: its ghost planes
     * are the mirror images of the interior (the boundary step between
     * the passes) */
    if (gz) {
        const double even = 1.0;
        or_fill_ghosts_z(divf, nx, ny, nz, 1, &even);
    }
    /* pass 2 (periodic wrap of the divergence field by modular indexing, or
     * its ghost planes) */
#pragma omp parallel for schedule(static)
    for (long z = 0; z < nz; ++z)
        for (long y = 0; y < ny; ++y)
            for (long x = 0; x < nx; ++x) {
                long p[3] = {x, y, z};
                long c = at(&g, p);
                for (int i = 0; i < 3; ++i) {
                    double gdi = d1(divf, &g, p, i);
                    w[(1 + i) * n + c] += dt * (ph.nu / 3.0) * gdi;
                    out[(1 + i) * n + c] += RK3_BETA[s] * dt * (ph.nu / 3.0) * gdi;
                }
            }
}

void or_substep55(const double *in, double *w, double *out, int s, double dt, long nx, long ny,
                  long nz, double lx, double ly, double lz, double cs, double nu, int entropy_mode)
{
    substep55(in, w, out, s, dt, nx, ny, nz, lx, ly, lz, cs, nu, entropy_mode, NULL, 0, 0);
}

void or_substep19(const double *in, double *w, double *out, double *divf, int s, double dt,
                  long nx, long ny, long nz, double lx, double ly, double lz, double cs, double nu,
                  int entropy_mode)
{
    substep19(in, w, out, divf, s, dt, nx, ny, nz, lx, ly, lz, cs, nu, entropy_mode, NULL, 0);
}

/* Wall variant (z bounded by walls through z = 0 and z = Lz, spacing
 * Lz / (N_z - 1); x, y periodic): the same substeps on ghost-extended arrays
 * of N_z + 6 planes per field (interior plane z at index z + 3), whose ghost
 * planes the caller has filled by or_fill_ghosts_z (Algorithm 1's boundary
 * step) before the call.  Only interior planes of out, w and divf are
 * written (divf's ghosts are filled between the passes). */
void or_substep55_wall(const double *in, double *w, double *out, int s, double dt, long nx,
                       long ny, long nz, double lx, double ly, double lz, double cs, double nu,
                       int entropy_mode)
{
    substep55(in, w, out, s, dt, nx, ny, nz, lx, ly, lz, cs, nu, entropy_mode, NULL, GZ_WALL, 1);
}

/* One substep of Algorithm 2 on a z-slab of a periodic domain split along z
 * (the domain decomposition of Sect. 7): ghost-extended arrays as for the
 * wall variant, whose ghost planes the caller has filled with the
 * neighbouring slabs' boundary planes; z spacing lz / nz. */
void or_substep55_slab(const double *in, double *w, double *out, int s, double dt, long nx,
                       long ny, long nz, double lx, double ly, double lz, double cs, double nu,
                       int entropy_mode)
{
    substep55(in, w, out, s, dt, nx, ny, nz, lx, ly, lz, cs, nu, entropy_mode, NULL, GZ_WALL, 0);
}

void or_substep19_wall(const double *in, double *w, double *out, double *divf, int s, double dt,
                       long nx, long ny, long nz, double lx, double ly, double lz, double cs,
                       double nu, int entropy_mode)
{
    substep19(in, w, out, divf, s, dt, nx, ny, nz, lx, ly, lz, cs, nu, entropy_mode, NULL,
              GZ_WALL);
}

/* One substep with the forcing of the current time step (k, phi and e are
 * fixed over the step's three substeps; N uses the step's dt).  form 0:
 * Algorithm 2, form 1: Algorithm 3 (divf is then required).  Returns -1
 * when f_k is undefined. */
int or_substep_forced(const double *in, double *w, double *out, double *divf, int s, double dt,
                      int form, long nx, long ny, long nz, double lx, double ly, double lz,
                      double cs, double nu, int entropy_mode, double f0, const long *kint,
                      double phi, const double *e)
{
    forcing_t fo;
    if (make_forcing(&fo, kint, phi, e, f0, cs, dt, lx, ly, lz))
        return -1;
    if (form == 1)
        substep19(in, w, out, divf, s, dt, nx, ny, nz, lx, ly, lz, cs, nu, entropy_mode, &fo, 0);
    else
        substep55(in, w, out, s, dt, nx, ny, nz, lx, ly, lz, cs, nu, entropy_mode, &fo, 0, 0);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Diagnostics (FP64 reductions)                                        */
/* ------------------------------------------------------------------ */

typedef struct {
    double sum, comp;
} neumaier_t;

static inline void nadd(neumaier_t *a, double v)
{
    double t = a->sum + v;
    if (fabs(a->sum) >= fabs(v))
        a->comp += (a->sum - t) + v;
    else
        a->comp += (v - t) + a->sum;
    a->sum = t;
}

static inline double nval(const neumaier_t *a) { return a->sum + a->comp; }

/* out[0] mass        = dV sum exp(lnrho)
 * out[1] kinetic     = dV sum exp(lnrho) |u|^2 / 2
 * out[2] max |u|     (Euclidean)
 * out[3] rms |u|     = sqrt(sum |u|^2 / N)
 * out[4..8]   rms of each field   (sqrt(sum f^2 / N)); 0 for absent fields
 * out[9..13]  max |f| of each field
 * out[14]     1.0 if any value of the state is not finite, else 0.0 */
void or_diagnostics(const double *state, long nx, long ny, long nz, double lx, double ly,
                    double lz, int entropy_mode, double *out)
{
    grid_t g = make_grid(nx, ny, nz, lx, ly, lz);
    const long n = g.npts;
    const int nf = entropy_mode ? 5 : 4;
    const double dv = g.h[0] * g.h[1] * g.h[2];
    neumaier_t mass = {0, 0}, ekin = {0, 0}, u2 = {0, 0}, f2[5];
    double umax = 0.0, fmax[5];
    int nonfinite = 0;
    for (int f = 0; f < 5; ++f) {
        f2[f].sum = f2[f].comp = 0.0;
        fmax[f] = 0.0;
    }
    for (long c = 0; c < n; ++c) {
        double rho = exp(state[c]);
        double ux = state[n + c], uy = state[2 * n + c], uz = state[3 * n + c];
        double uu = ux * ux + uy * uy + uz * uz;
        nadd(&mass, rho);
        nadd(&ekin, 0.5 * rho * uu);
        nadd(&u2, uu);
        if (sqrt(uu) > umax)
            umax = sqrt(uu);
        for (int f = 0; f < nf; ++f) {
            double v = state[f * n + c];
            if (!isfinite(v))
                nonfinite = 1;
            nadd(&f2[f], v * v);
            if (fabs(v) > fmax[f])
                fmax[f] = fabs(v);
        }
    }
    out[0] = dv * nval(&mass);
    out[1] = dv * nval(&ekin);
    out[2] = umax;
    out[3] = sqrt(nval(&u2) / (double)n);
    for (int f = 0; f < 5; ++f) {
        out[4 + f] = sqrt(nval(&f2[f]) / (double)n);
        out[9 + f] = fmax[f];
    }
    out[14] = nonfinite ? 1.0 : 0.0;
}

/* Time step from the step-start state (the paper gives no rule):
 * dt = min(cfl * dmin / (max|u| + c_s), cnu * dmin^2 / nu). */
double or_cfl_dt(const double *state, long nx, long ny, long nz, double lx, double ly, double lz,
                 double cs, double nu, double cfl, double cnu)
{
    grid_t g = make_grid(nx, ny, nz, lx, ly, lz);
    const long n = g.npts;
    double umax = 0.0;
    for (long c = 0; c < n; ++c) {
        double ux = state[n + c], uy = state[2 * n + c], uz = state[3 * n + c];
        double m = sqrt(ux * ux + uy * uy + uz * uz);
        if (m > umax)
            umax = m;
    }
    double dmin = g.h[0];
    if (g.h[1] < dmin)
        dmin = g.h[1];
    if (g.h[2] < dmin)
        dmin = g.h[2];
    double dt = cfl * dmin / (umax + cs);
    if (nu > 0.0) {
        double dtn = cnu * dmin * dmin / nu;
        if (dtn < dt)
            dt = dtn;
    }
    return dt;
}

/* ------------------------------------------------------------------ */
/* Box filter (coarse vertex I sits on fine vertex r I)                 */
/* ------------------------------------------------------------------ */

/* Per axis, weights (1/2, 1, ..., 1, 1/2) / r over fine indices
 * r I - r/2 .. r I + r/2 (r even), periodic; the 3D filter is the product
 * of the three axis weights.  Applied to each of nf fields. */
void or_box_filter(const double *fine, double *coarse, long nfx, long nfy, long nfz, int r,
                   int nf)
{
    const long ncx = nfx / r, ncy = nfy / r, ncz = nfz / r;
    const long nfine = nfx * nfy * nfz, ncoarse = ncx * ncy * ncz;
    const int h = r / 2;
    for (int f = 0; f < nf; ++f)
        for (long Z = 0; Z < ncz; ++Z)
            for (long Y = 0; Y < ncy; ++Y)
                for (long X = 0; X < ncx; ++X) {
                    double acc = 0.0;
                    for (int a = -h; a <= h; ++a)
                        for (int b = -h; b <= h; ++b)
                            for (int c = -h; c <= h; ++c) {
                                double wz = (a == -h || a == h) ? 0.5 : 1.0;
                                double wy = (b == -h || b == h) ? 0.5 : 1.0;
                                double wx = (c == -h || c == h) ? 0.5 : 1.0;
                                long z = wrap(r * Z + a, nfz), y = wrap(r * Y + b, nfy),
                                     x = wrap(r * X + c, nfx);
                                acc += wz * wy * wx * fine[f * nfine + (z * nfy + y) * nfx + x];
                            }
                    coarse[f * ncoarse + (Z * ncy + Y) * ncx + X] =
                        acc / ((double)r * (double)r * (double)r);
                }
}

/* ------------------------------------------------------------------ */

int or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
