/*
 * lbgb_oracle.c -- plain, slow FP64 CPU oracle of one time step of the
 * two-component Shan-Chen lattice-Boltzmann fluid (D3Q19, BGK + Exact
 * Difference Method forcing) coupled to Ladd spherical colloids, as described
 * in "LBsoft: a parallel open-source software for simulation of colloidal
 * systems" (Bonaccorso et al., arXiv:2004.04080).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference that the CUDA library
 * is checked against.  Only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header or
 * table with the CUDA library: the lattice tables, equilibrium, forces and
 * integrator below are written out here on their own.
 *
 * The step follows the paper's particle-coupled call sequence (Sec. 3.1):
 *   1. moments (Eqs. 6, 7, 14)
 *   2. destroy / create fluid nodes under moving particles (Eqs. 24, 25)
 *   3. particle-particle forces (Eqs. 26, 27)
 *   4. LB force term: virtual wetting densities and Shan-Chen forces
 *      (Eqs. 11, 20, 21)
 *   5. collision with the exact-difference source (Eqs. 13-16)
 *   6. halfway bounce-back at particle surfaces and walls with the link
 *      forces (Eqs. 8, 9, 17-19, 22, 23)
 *   7. rotational leap-frog of the particles (Eqs. 28-35)
 *   8. streaming (Eq. 3)
 * Every loop is a plain loop over lattice sites or particles; nothing is
 * fused, blocked or reordered beyond what the equations state.  Build with
 * -O2 -ffp-contract=off so that no multiply-add is contracted.  Loops whose
 * iterations each write only their own site's values are shared out over
 * threads with OpenMP (-fopenmp); a site's arithmetic does not depend on the
 * thread count, so every thread count gives the same bits.  Sums into
 * per-particle totals stay single-threaded, in site order.
 *
 * Readings taken where the paper is silent or garbled (each is also used by
 * the CUDA library, which is written independently):
 *  - Shan-Chen force sign: F^k = -G rho^k sum_i w_i psi^kbar(x+c_i) c_i, so
 *    that G > 0 is repulsive between the components (Eq. 11 prints no sign;
 *    Eq. 12 needs repulsion).  The same sign is used for the solid-node force
 *    of Eq. 21.
 *  - Mixture relaxation: omega_eff = 1 / (nubar/cs^2 + 1/2) with
 *    1/nubar = sum_k (rho^k/rho)/nu_k and nu_k = cs^2 (tau_k - 1/2) (the
 *    printed omega_eff of Sec. 2.3 divides by zero at tau = 1).
 *  - Mixture velocity (Eq. 14) uses the bare moments j^k = sum_i f_i c_i with
 *    omega^k = 1/tau_k; the reported velocity adds half the force (end of
 *    Sec. 2.3).
 *  - Wall velocity at a particle link (Eq. 18) is the rigid-body velocity
 *    u_w = v_p + omega_p x (r_w - r_p).
 *  - Bounce-back density rho in Eqs. 9, 17, 19 is rho^k of the boundary fluid
 *    node, per component; the particle velocities in Eqs. 17-19 are the
 *    latest stored half-step values v(t-1/2), omega(t-1/2).
 *  - The wetting reaction force of Eq. 21 enters the particle force and
 *    torque together with the terms of Eq. 28.
 *  - Virtual density (Eq. 20) and refill density (Sec. 2.4, creation) are
 *    w_i-weighted means over fluid neighbours; for a refilled node the
 *    neighbours are nodes that are fluid both before and after the remap.  A
 *    refilled node with no such neighbour takes rho0^k.
 *  - A node is solid iff |x - r_p|^2 < R_p^2 (minimum image).  The first map
 *    after particles are added removes fluid without momentum bookkeeping.
 *  - Hertz force (Eq. 26): on particle i, F = -(5/2) K (sigma - r)^{3/2}
 *    r_ij/|r_ij| for r < sigma, with r floored at r_cap and
 *    r_ij = r_j - r_i (the printed derivative points the wrong way; sigma
 *    and r_cap are the "field pair hz" distances of the benchmark input).
 *  - Lubrication (Eq. 27), optional: F_i = -6 pi nu s (R_i R_j/(R_i+R_j))^2
 *    (1/h - 1/h_n) [(v_i - v_j).rhat] rhat with h floored at h_min.
 *  - Walls (normal to z) are halfway bounce-back planes at z = -1/2 and
 *    z = nz - 1/2 moving with a fixed velocity (Eq. 9 with the local density);
 *    for the Shan-Chen force a wall node carries the w_i-weighted mean density
 *    of its fluid neighbours ("wetting mode 0", neutral).
 *  - Open z faces (Sec. 2.2): a pressure face (Eq. 10) with a given rho_w
 *    and u_w the velocity of the boundary node (Eq. 14); a velocity face
 *    (Eq. 9) with the density of the boundary node; an equilibrium face that
 *    sends in f^eq(rho_w, u_w).  With open_extrap the face values of the
 *    first two are extrapolated from the boundary node b and the next
 *    interior node b+1, q_w = q_b + (q_b - q_{b+1})/2 (Sec. 2.2), where b+1
 *    exists and is fluid.
 *  - Soft harmonic side wall on particles: F_z = k (d - h) away from the wall
 *    when the centre is closer than d to a wall plane (h = distance).
 *  - First step: F_liq(-1/2) := F_liq(+1/2) (Eq. 35).
 *  - Spheres have isotropic inertia I = (2/5) m R^2, so the angular velocity is
 *    kept in the space frame; the body-frame omega* needed by Eq. 33 is
 *    R(q)^T omega with R evaluated at the normalised mid-step quaternion.
 *    The implicit mid-step of Eq. 34 is iterated until the quaternion rate
 *    changes by at most 1e-14 (at most 20 times), then q is normalised.
 *  - Every per-particle sum is a Neumaier-compensated FP64 sum (the paper's
 *    QUAD_FORCEINT concern, Sec. 3.1).
 */
#define _DEFAULT_SOURCE
#ifdef _OPENMP
#include <omp.h>
#endif
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
    ORC_OK = 0,
    ORC_ERR_ARG = -1,
    ORC_ERR_STATE = -2,
    ORC_ERR_NOMEM = -4,
    ORC_ERR_NONFINITE = -5,
    ORC_ERR_OVERLAP = -6
};

/* ---- D3Q19 lattice (Sec. 2.1): rest, 6 links of length 1, 12 of sqrt 2 ---- */
#define NQ 19
static const int CX[NQ] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[NQ] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[NQ] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static const double WT[NQ] = {
    1.0 / 3.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;

/* index of the link opposite to i (searched once, then remembered) */
static int opposite(int i)
{
    static int table[NQ];
    static int ready = 0;
    int a, j;
    if (!ready) {
        for (a = 0; a < NQ; a++) {
            table[a] = -1;
            for (j = 0; j < NQ; j++)
                if (CX[j] == -CX[a] && CY[j] == -CY[a] && CZ[j] == -CZ[a])
                    table[a] = j;
        }
        ready = 1;
    }
    return table[i];
}

typedef struct {
    double tau[2];
    double G;
    double zeta[2];
    double rho0[2];
    int bc[3];
    double wall_u_lo[3];
    double wall_u_hi[3];
    double body_force[3];
    double hertz_K, hertz_sigma, hertz_rcap;
    int lub_on;
    double lub_hn, lub_hmin, lub_scale;
    double side_wall_k, side_wall_d;
    int rotate;
    int janus;                         /* Janus wettability on/off          */
    double janus_theta0, janus_width;  /* switch centre and width, degrees  */
    int open[2];                       /* z faces (lo, hi) with walls: 0 wall,
                                          1 pressure, 2 velocity, 3 equilibrium */
    double open_rho[2][2];             /* face density per component        */
    int open_extrap;                   /* 1: the face values of pressure and
                                          velocity faces extrapolated to first
                                          order from the next interior node   */
} orc_params;

/* Neumaier compensated sum */
typedef struct { double s, c; } nsum;
static void nadd(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}
static double nval(const nsum *a) { return a->s + a->c; }

typedef struct {
    int nx, ny, nz;
    long N;
    orc_params P;
    int have_params, have_fields;
    double *f[2];      /* populations f[k][i*N + s] at the current time      */
    double *fpost[2];  /* post-collision populations                          */
    double *fnext[2];  /* populations at t+1, filled by streaming/bounce-back */
    double *rho[2];    /* rho^k per site (0 on solid)                          */
    double *jm[2];     /* bare momentum j^k, [3][N]                            */
    double *frc[2];    /* Shan-Chen + body force F^k, [3][N]                   */
    double *psi[2];    /* virtual density on frontier solid nodes              */
    double *psi_lo[2], *psi_hi[2]; /* wall virtual density, [nx*ny]            */
    int *owner, *owner_new;
    /* particles */
    int maxc, nc;
    double *pos, *vel, *omg, *quat, *rad, *mass;
    double *Fliq, *Tliq, *Fliq_prev, *Tliq_prev;
    unsigned char *prev_valid;
    double *Fd, *Td, *Fc, *Tc, *Fs, *Ts, *Fpair, *Ftot, *Ttot;
    int err;
} orc_t;

/* ---------------------------------------------------------------- helpers */
static long site(const orc_t *o, int x, int y, int z)
{
    return (long)x + (long)o->nx * ((long)y + (long)o->ny * (long)z);
}

/* neighbour of site (x,y,z) along link i; -1 if it lies beyond a wall */
static long neighbour(const orc_t *o, int x, int y, int z, int i)
{
    int xn = x + CX[i], yn = y + CY[i], zn = z + CZ[i];
    int L[3] = {o->nx, o->ny, o->nz};
    int c[3] = {xn, yn, zn};
    int d;
    for (d = 0; d < 3; d++) {
        if (c[d] < 0 || c[d] >= L[d]) {
            if (!o->P.bc[d])
                return -1;
            c[d] = (c[d] + L[d]) % L[d];
        }
    }
    return site(o, c[0], c[1], c[2]);
}

static void coords(const orc_t *o, long s, int *x, int *y, int *z)
{
    *x = (int)(s % o->nx);
    *y = (int)((s / o->nx) % o->ny);
    *z = (int)(s / ((long)o->nx * o->ny));
}

/* minimum-image component of a displacement */
static double mimg(double d, int L, int periodic)
{
    if (!periodic)
        return d;
    return d - (double)L * floor(d / (double)L + 0.5);
}

static void cross(const double a[3], const double b[3], double out[3])
{
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

/* Eq. 5: second-order equilibrium f_i^eq = w_i rho (1 + u_i + q_i/2) with
 * u_i = c_i.u/cs^2 and q_i = ((c_i.u)^2 - cs^2 u.u)/cs^4. */
static double feq_i(int i, double rho, const double u[3])
{
    double cu = CX[i] * u[0] + CY[i] * u[1] + CZ[i] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double ui = cu / CS2;
    double qi = (cu * cu - CS2 * uu) / (CS2 * CS2);
    return WT[i] * rho * (1.0 + ui + 0.5 * qi);
}

void orc_feq(double rho, const double *u, double *out)
{
    int i;
    for (i = 0; i < NQ; i++)
        out[i] = feq_i(i, rho, u);
}

void orc_lattice(int *cx, int *cy, int *cz, double *w, int *opp)
{
    int i;
    for (i = 0; i < NQ; i++) {
        cx[i] = CX[i];
        cy[i] = CY[i];
        cz[i] = CZ[i];
        w[i] = WT[i];
        opp[i] = opposite(i);
    }
}

/* ------------------------------------------------------------- lifecycle */
static void *zalloc(size_t n) { return calloc(n ? n : 1, 1); }

void orc_destroy(orc_t *o)
{
    int k;
    if (!o)
        return;
    for (k = 0; k < 2; k++) {
        free(o->f[k]); free(o->fpost[k]); free(o->fnext[k]);
        free(o->rho[k]); free(o->jm[k]); free(o->frc[k]); free(o->psi[k]);
        free(o->psi_lo[k]); free(o->psi_hi[k]);
    }
    free(o->owner); free(o->owner_new);
    free(o->pos); free(o->vel); free(o->omg); free(o->quat); free(o->rad); free(o->mass);
    free(o->Fliq); free(o->Tliq); free(o->Fliq_prev); free(o->Tliq_prev); free(o->prev_valid);
    free(o->Fd); free(o->Td); free(o->Fc); free(o->Tc); free(o->Fs); free(o->Ts);
    free(o->Fpair); free(o->Ftot); free(o->Ttot);
    free(o);
}

orc_t *orc_create(int nx, int ny, int nz, int maxc)
{
    orc_t *o;
    int k;
    long N, nxy;
    if (nx < 3 || ny < 3 || nz < 3 || maxc < 0)
        return NULL;
    o = (orc_t *)zalloc(sizeof(orc_t));
    if (!o)
        return NULL;
    o->nx = nx; o->ny = ny; o->nz = nz;
    N = (long)nx * ny * nz;
    nxy = (long)nx * ny;
    o->N = N;
    o->maxc = maxc;
    for (k = 0; k < 2; k++) {
        o->f[k] = zalloc(sizeof(double) * NQ * N);
        o->fpost[k] = zalloc(sizeof(double) * NQ * N);
        o->fnext[k] = zalloc(sizeof(double) * NQ * N);
        o->rho[k] = zalloc(sizeof(double) * N);
        o->jm[k] = zalloc(sizeof(double) * 3 * N);
        o->frc[k] = zalloc(sizeof(double) * 3 * N);
        o->psi[k] = zalloc(sizeof(double) * N);
        o->psi_lo[k] = zalloc(sizeof(double) * nxy);
        o->psi_hi[k] = zalloc(sizeof(double) * nxy);
        if (!o->f[k] || !o->fpost[k] || !o->fnext[k] || !o->rho[k] || !o->jm[k] ||
            !o->frc[k] || !o->psi[k] || !o->psi_lo[k] || !o->psi_hi[k]) {
            orc_destroy(o);
            return NULL;
        }
    }
    o->owner = zalloc(sizeof(int) * N);
    o->owner_new = zalloc(sizeof(int) * N);
#define PA(field, n) o->field = zalloc(sizeof(double) * (size_t)(n) * (maxc ? maxc : 1))
    PA(pos, 3); PA(vel, 3); PA(omg, 3); PA(quat, 4); PA(rad, 1); PA(mass, 1);
    PA(Fliq, 3); PA(Tliq, 3); PA(Fliq_prev, 3); PA(Tliq_prev, 3);
    PA(Fd, 3); PA(Td, 3); PA(Fc, 3); PA(Tc, 3); PA(Fs, 3); PA(Ts, 3);
    PA(Fpair, 3); PA(Ftot, 3); PA(Ttot, 3);
#undef PA
    o->prev_valid = zalloc((size_t)(maxc ? maxc : 1));
    if (!o->owner || !o->owner_new || !o->pos || !o->prev_valid || !o->Ttot) {
        orc_destroy(o);
        return NULL;
    }
    for (k = 0; k < N; k++)
        o->owner[k] = -1;
    return o;
}

int orc_set_params(orc_t *o, const orc_params *p)
{
    if (!o || !p)
        return ORC_ERR_ARG;
    if (!(p->tau[0] > 0.5) || !(p->tau[1] > 0.5))
        return ORC_ERR_ARG;
    if (!p->bc[0] || !p->bc[1])
        return ORC_ERR_ARG; /* walls only normal to z */
    if (p->janus && !(p->janus_width >= 0.0 && isfinite(p->janus_width) && isfinite(p->janus_theta0)))
        return ORC_ERR_ARG;
    if (p->open[0] < 0 || p->open[0] > 3 || p->open[1] < 0 || p->open[1] > 3)
        return ORC_ERR_ARG;
    if (p->open_extrap != 0 && p->open_extrap != 1)
        return ORC_ERR_ARG;
    o->P = *p;
    o->have_params = 1;
    return ORC_OK;
}

/* f = f^eq(rho^k, u) everywhere; u may be NULL (zero). */
int orc_init_fields(orc_t *o, const double *rhoA, const double *rhoB, const double *u)
{
    long s;
    int i;
    if (!o || !rhoA || !rhoB)
        return ORC_ERR_ARG;
    if (!o->have_params)
        return ORC_ERR_STATE;
    for (s = 0; s < o->N; s++) {
        double us[3] = {0.0, 0.0, 0.0};
        if (u) {
            us[0] = u[s];
            us[1] = u[o->N + s];
            us[2] = u[2 * o->N + s];
        }
        for (i = 0; i < NQ; i++) {
            o->f[0][i * o->N + s] = feq_i(i, rhoA[s], us);
            o->f[1][i * o->N + s] = feq_i(i, rhoB[s], us);
        }
    }
    o->have_fields = 1;
    return ORC_OK;
}

/* ----------------------------------------------------------- step pieces */

/* Eqs. 6 and 7 per component on fluid nodes; solid nodes hold zero. */
static void moments(orc_t *o)
{
    long s, N = o->N;
    int k, i, bad = 0;
#pragma omp parallel for private(k, i) reduction(| : bad) schedule(static)
    for (s = 0; s < N; s++) {
        for (k = 0; k < 2; k++) {
            double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
            if (o->owner[s] < 0) {
                for (i = 0; i < NQ; i++) {
                    double fi = o->f[k][i * N + s];
                    r += fi;
                    jx += fi * CX[i];
                    jy += fi * CY[i];
                    jz += fi * CZ[i];
                }
                if (!isfinite(r) || r < 0.0 || !isfinite(jx) || !isfinite(jy) || !isfinite(jz))
                    bad = 1;
            }
            o->rho[k][s] = r;
            o->jm[k][s] = jx;
            o->jm[k][N + s] = jy;
            o->jm[k][2 * N + s] = jz;
        }
    }
    if (bad)
        o->err = ORC_ERR_NONFINITE;
}

/* Eq. 14: u = sum_k omega^k j^k / sum_k omega^k rho^k, omega^k = 1/tau_k */
static void mix_velocity(const orc_t *o, long s, double u[3])
{
    long N = o->N;
    double w0 = 1.0 / o->P.tau[0], w1 = 1.0 / o->P.tau[1];
    double den = w0 * o->rho[0][s] + w1 * o->rho[1][s];
    int d;
    for (d = 0; d < 3; d++)
        u[d] = (w0 * o->jm[0][d * N + s] + w1 * o->jm[1][d * N + s]) / den;
}

/* The next interior node r_{b+1} of the boundary node s on z face `side`
 * (Sec. 2.2: one site inward along the face normal), or -1 where the face
 * values are not extrapolated: extrapolation off, no such node (nz < 2), or
 * a particle node there. */
static long next_interior(const orc_t *o, long s, int side)
{
    int x, y, z, zi;
    long n;
    if (!o->P.open_extrap)
        return -1;
    coords(o, s, &x, &y, &z);
    zi = side == 0 ? z + 1 : z - 1;
    if (zi < 0 || zi >= o->nz)
        return -1;
    n = site(o, x, y, zi);
    return o->owner[n] < 0 ? n : -1;
}

/* rho_w^k of a velocity face (Eq. 9): the first-order extrapolation of
 * Sec. 2.2, rho_w = rho(r_b) + [rho(r_b) - rho(r_{b+1})] / 2, else the
 * density of the boundary node */
static double face_density(const orc_t *o, long s, int side, int k)
{
    long n = next_interior(o, s, side);
    if (n < 0)
        return o->rho[k][s];
    return o->rho[k][s] + 0.5 * (o->rho[k][s] - o->rho[k][n]);
}

/* u_w of a pressure face (Eq. 10): the same extrapolation of the velocity
 * of Eq. 14, else the velocity of the boundary node */
static void face_velocity(const orc_t *o, long s, int side, double u[3])
{
    long n = next_interior(o, s, side);
    double ub[3], ui[3];
    int d;
    mix_velocity(o, s, ub);
    if (n < 0) {
        for (d = 0; d < 3; d++)
            u[d] = ub[d];
        return;
    }
    mix_velocity(o, n, ui);
    for (d = 0; d < 3; d++)
        u[d] = ub[d] + 0.5 * (ub[d] - ui[d]);
}

/* position of site s relative to particle p (minimum image), plus offset */
static void rel_pos(const orc_t *o, long s, int p, const double off[3], double out[3])
{
    int x, y, z;
    int L[3] = {o->nx, o->ny, o->nz};
    double c[3];
    int d;
    coords(o, s, &x, &y, &z);
    c[0] = x + off[0];
    c[1] = y + off[1];
    c[2] = z + off[2];
    for (d = 0; d < 3; d++)
        out[d] = mimg(c[d] - o->pos[3 * p + d], L[d], o->P.bc[d]);
}

/* Eq. 18 (rigid-body reading): u_w = v_p + omega_p x (r_w - r_p) */
static void wall_velocity(const orc_t *o, int p, const double rel[3], double uw[3])
{
    double wxr[3];
    int d;
    cross(&o->omg[3 * p], rel, wxr);
    for (d = 0; d < 3; d++)
        uw[d] = o->vel[3 * p + d] + wxr[d];
}

/* Sec. 2.4: node map.  owner_new[s] = lowest-index particle p with
 * |x_s - r_p|^2 < R_p^2; sets an overlap error if a node lies in two. */
static void build_map(orc_t *o)
{
    long s;
    int p;
    int L[3] = {o->nx, o->ny, o->nz};
    for (s = 0; s < o->N; s++)
        o->owner_new[s] = -1;
    for (p = 0; p < o->nc; p++) {
        double R = o->rad[p];
        int lo[3], hi[3], d, a, b, c;
        for (d = 0; d < 3; d++) {
            lo[d] = (int)floor(o->pos[3 * p + d] - R);
            hi[d] = (int)ceil(o->pos[3 * p + d] + R);
        }
        for (c = lo[2]; c <= hi[2]; c++)
            for (b = lo[1]; b <= hi[1]; b++)
                for (a = lo[0]; a <= hi[0]; a++) {
                    int q[3] = {a, b, c};
                    double d2 = 0.0;
                    int ok = 1;
                    for (d = 0; d < 3; d++) {
                        double dd = (double)q[d] - o->pos[3 * p + d];
                        d2 += dd * dd;
                        if (q[d] < 0 || q[d] >= L[d]) {
                            if (!o->P.bc[d])
                                ok = 0;
                            else
                                q[d] = ((q[d] % L[d]) + L[d]) % L[d];
                        }
                    }
                    if (!ok || !(d2 < R * R))
                        continue;
                    s = site(o, q[0], q[1], q[2]);
                    if (o->owner_new[s] < 0)
                        o->owner_new[s] = p;
                    else if (o->owner_new[s] != p)
                        o->err = ORC_ERR_OVERLAP;
                }
    }
}

/* Step 2: destroy (Eq. 24) and create (Eq. 25) fluid nodes. */
static void remap(orc_t *o, int first)
{
    long s, N = o->N;
    int p, k, i, d;
    nsum *acc;
    build_map(o);
    if (first) {
        for (s = 0; s < N; s++)
            o->owner[s] = o->owner_new[s];
        return;
    }
    acc = (nsum *)zalloc(sizeof(nsum) * 12 * (size_t)(o->nc ? o->nc : 1));
    /* Eq. 24: a fluid node covered by particle p hands its momentum to p */
    for (s = 0; s < N; s++) {
        int old = o->owner[s], nw = o->owner_new[s];
        if (old >= 0 && nw >= 0 && old != nw)
            o->err = ORC_ERR_OVERLAP;
        if (old < 0 && nw >= 0) {
            double u[3], mom[3], rel[3], tq[3], zero[3] = {0, 0, 0};
            double rt = o->rho[0][s] + o->rho[1][s];
            mix_velocity(o, s, u);
            for (d = 0; d < 3; d++)
                mom[d] = rt * u[d];
            rel_pos(o, s, nw, zero, rel);
            cross(rel, mom, tq);
            for (d = 0; d < 3; d++) {
                nadd(&acc[12 * nw + d], mom[d]);
                nadd(&acc[12 * nw + 3 + d], tq[d]);
            }
        }
    }
    /* Eq. 25: a node released by particle p is refilled with f^eq(rhobar^k, u_w) */
    for (s = 0; s < N; s++) {
        int old = o->owner[s], nw = o->owner_new[s];
        if (old >= 0 && nw < 0) {
            int x, y, z;
            double rb[2], uw[3], rel[3], mom[3], tq[3], zero[3] = {0, 0, 0};
            coords(o, s, &x, &y, &z);
            for (k = 0; k < 2; k++) {
                double num = 0.0, den = 0.0;
                for (i = 1; i < NQ; i++) {
                    long n = neighbour(o, x, y, z, i);
                    if (n < 0 || o->owner[n] >= 0 || o->owner_new[n] >= 0)
                        continue;
                    num += WT[i] * o->rho[k][n];
                    den += WT[i];
                }
                rb[k] = den > 0.0 ? num / den : o->P.rho0[k];
            }
            p = old;
            rel_pos(o, s, p, zero, rel);
            wall_velocity(o, p, rel, uw);
            for (k = 0; k < 2; k++)
                for (i = 0; i < NQ; i++)
                    o->f[k][i * N + s] = feq_i(i, rb[k], uw);
            for (d = 0; d < 3; d++)
                mom[d] = -(rb[0] + rb[1]) * uw[d];
            cross(rel, mom, tq);
            for (d = 0; d < 3; d++) {
                nadd(&acc[12 * p + 6 + d], mom[d]);
                nadd(&acc[12 * p + 9 + d], tq[d]);
            }
        }
    }
    for (p = 0; p < o->nc; p++)
        for (d = 0; d < 3; d++) {
            o->Fd[3 * p + d] = nval(&acc[12 * p + d]);
            o->Td[3 * p + d] = nval(&acc[12 * p + 3 + d]);
            o->Fc[3 * p + d] = nval(&acc[12 * p + 6 + d]);
            o->Tc[3 * p + d] = nval(&acc[12 * p + 9 + d]);
        }
    free(acc);
    for (s = 0; s < N; s++)
        o->owner[s] = o->owner_new[s];
    /* moments of the refilled nodes (and zero on the covered ones) */
    moments(o);
}

/* Eq. 26 (Hertz) and Eq. 27 (lubrication) on particle i due to particle j,
 * given r_ij = r_j - r_i (minimum image) and the two velocities. */
void orc_pair_force(const orc_params *P, const double *rij, double Ri, double Rj,
                    const double *vi, const double *vj, double *out)
{
    double r = sqrt(rij[0] * rij[0] + rij[1] * rij[1] + rij[2] * rij[2]);
    int d;
    out[0] = out[1] = out[2] = 0.0;
    if (!(r > 0.0))
        return;
    if (r < P->hertz_sigma && P->hertz_K != 0.0) {
        double rr = r < P->hertz_rcap ? P->hertz_rcap : r;
        double mag = 2.5 * P->hertz_K * pow(P->hertz_sigma - rr, 1.5);
        for (d = 0; d < 3; d++)
            out[d] += -mag * rij[d] / r;
    }
    if (P->lub_on) {
        double h = r - (Ri + Rj);
        if (h < P->lub_hn) {
            double nu = 0.5 * (CS2 * (P->tau[0] - 0.5) + CS2 * (P->tau[1] - 0.5));
            double red = Ri * Rj / (Ri + Rj);
            double vr = 0.0, mag;
            if (h < P->lub_hmin)
                h = P->lub_hmin;
            for (d = 0; d < 3; d++)
                vr += (vi[d] - vj[d]) * rij[d] / r;
            mag = -6.0 * 3.14159265358979323846 * nu * P->lub_scale * red * red * (1.0 / h - 1.0 / P->lub_hn) * vr;
            for (d = 0; d < 3; d++)
                out[d] += mag * rij[d] / r;
        }
    }
}

/* Step 3: particle-particle forces, summed for particle i over j in index order */
static void pair_forces(orc_t *o)
{
    int i, j, d;
    int L[3] = {o->nx, o->ny, o->nz};
    for (i = 0; i < o->nc; i++) {
        nsum a[3] = {{0, 0}, {0, 0}, {0, 0}};
        for (j = 0; j < o->nc; j++) {
            double rij[3], fo[3];
            if (j == i)
                continue;
            for (d = 0; d < 3; d++)
                rij[d] = mimg(o->pos[3 * j + d] - o->pos[3 * i + d], L[d], o->P.bc[d]);
            orc_pair_force(&o->P, rij, o->rad[i], o->rad[j], &o->vel[3 * i], &o->vel[3 * j], fo);
            for (d = 0; d < 3; d++)
                nadd(&a[d], fo[d]);
        }
        if (!o->P.bc[2] && o->P.side_wall_k != 0.0) {
            double hlo = o->pos[3 * i + 2] + 0.5;
            double hhi = ((double)o->nz - 0.5) - o->pos[3 * i + 2];
            if (hlo < o->P.side_wall_d)
                nadd(&a[2], o->P.side_wall_k * (o->P.side_wall_d - hlo));
            if (hhi < o->P.side_wall_d)
                nadd(&a[2], -o->P.side_wall_k * (o->P.side_wall_d - hhi));
        }
        for (d = 0; d < 3; d++)
            o->Fpair[3 * i + d] = nval(&a[d]);
    }
}

/* psi^k seen from a fluid node at (x,y,z) along link i: rho on fluid nodes,
 * the virtual density on particle nodes, the wall density beyond a wall. */
static double psi_at(const orc_t *o, int k, int x, int y, int z, int i)
{
    long n = neighbour(o, x, y, z, i);
    if (n < 0) {
        int xn = ((x + CX[i]) % o->nx + o->nx) % o->nx;
        int yn = ((y + CY[i]) % o->ny + o->ny) % o->ny;
        long w = (long)xn + (long)o->nx * yn;
        return (z + CZ[i] < 0) ? o->psi_lo[k][w] : o->psi_hi[k][w];
    }
    if (o->owner[n] < 0)
        return o->rho[k][n];
    return o->psi[k][n];
}

/* Janus wettability (Sec. 5.1, the colloid benchmarks; App. A, the MD
 * room's wettability-angle directive): the particle's wetting varies with
 * the polar angle theta between the direction from its centre to the node
 * and its first body axis x* (the first column of the rotation matrix of
 * Eq. 31, body to space).  The switch s goes smoothly from -1 to 1 across
 * [theta0 - width/2, theta0 + width/2] (a cubic smoothstep; a step at
 * theta0 for width 0).  With it on, the node's wetting constants are
 * s zeta^A and -s zeta^B, so the caps theta < theta0 and theta > theta0 wet
 * oppositely.  Returns s, or 1 with the switch off (plain zeta^k). */
static double janus_switch(const orc_t *o, int p, long s)
{
    const double *q = &o->quat[4 * p];
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double a = q[0] / n, b = q[1] / n, c = q[2] / n, e = q[3] / n;
    double ax[3], d[3], zero[3] = {0.0, 0.0, 0.0}, dn, ct, th, lo, t;
    if (!o->P.janus)
        return 1.0;
    ax[0] = a * a + b * b - c * c - e * e;
    ax[1] = 2.0 * (b * c + a * e);
    ax[2] = 2.0 * (b * e - a * c);
    rel_pos(o, s, p, zero, d);
    dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (dn == 0.0)
        return 0.0; /* the centre node: no direction */
    ct = (ax[0] * d[0] + ax[1] * d[1] + ax[2] * d[2]) / dn;
    ct = ct > 1.0 ? 1.0 : (ct < -1.0 ? -1.0 : ct);
    th = acos(ct) * (180.0 / M_PI);
    lo = o->P.janus_theta0 - 0.5 * o->P.janus_width;
    if (o->P.janus_width <= 0.0)
        return th < o->P.janus_theta0 ? -1.0 : 1.0;
    t = (th - lo) / o->P.janus_width;
    t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
    return -1.0 + 2.0 * t * t * (3.0 - 2.0 * t);
}

/* Step 4: Eq. 20 virtual densities, Eq. 11 on fluid, Eq. 21 on solid. */
static void lb_forces(orc_t *o, int store_particle_terms)
{
    long s, N = o->N;
    int k, i, d, x, y, z;
    double sw;
    nsum *acc = (nsum *)zalloc(sizeof(nsum) * 6 * (size_t)(o->nc ? o->nc : 1));
    /* Eq. 20 on every solid node that has a fluid neighbour */
#pragma omp parallel for private(k, i, x, y, z, sw) schedule(static)
    for (s = 0; s < N; s++) {
        o->psi[0][s] = 0.0;
        o->psi[1][s] = 0.0;
        if (o->owner[s] < 0)
            continue;
        coords(o, s, &x, &y, &z);
        sw = janus_switch(o, o->owner[s], s);
        for (k = 0; k < 2; k++) {
            double num = 0.0, den = 0.0;
            /* wetting constant of this node: zeta^k, or with the Janus
             * switch on s zeta^A and -s zeta^B */
            double zk = o->P.janus ? (k == 0 ? sw : -sw) * o->P.zeta[k] : o->P.zeta[k];
            for (i = 1; i < NQ; i++) {
                long n = neighbour(o, x, y, z, i);
                if (n < 0 || o->owner[n] >= 0)
                    continue;
                num += WT[i] * o->rho[k][n];
                den += WT[i];
            }
            if (den > 0.0)
                o->psi[k][s] = (1.0 + zk) * num / den;
        }
    }
    /* wall nodes (wetting mode 0): mean density of their fluid neighbours */
    if (!o->P.bc[2]) {
        int side;
        for (side = 0; side < 2; side++)
            for (y = 0; y < o->ny; y++)
                for (x = 0; x < o->nx; x++) {
                    int zf = side == 0 ? 0 : o->nz - 1;
                    int dz = side == 0 ? 1 : -1;
                    for (k = 0; k < 2; k++) {
                        double num = 0.0, den = 0.0;
                        for (i = 1; i < NQ; i++) {
                            long n;
                            if (CZ[i] != dz)
                                continue;
                            n = site(o, ((x + CX[i]) % o->nx + o->nx) % o->nx,
                                     ((y + CY[i]) % o->ny + o->ny) % o->ny, zf);
                            if (o->owner[n] >= 0)
                                continue;
                            num += WT[i] * o->rho[k][n];
                            den += WT[i];
                        }
                        /* a pressure or equilibrium face: its density */
                        if (o->P.open[side] == 1 || o->P.open[side] == 3)
                            (side == 0 ? o->psi_lo : o->psi_hi)[k][x + (long)o->nx * y] =
                                o->P.open_rho[side][k];
                        else
                            (side == 0 ? o->psi_lo : o->psi_hi)[k][x + (long)o->nx * y] =
                                den > 0.0 ? num / den : 0.0;
                    }
                }
    }
    /* Eq. 11 on fluid nodes (plus the body force rho^k g) */
#pragma omp parallel for private(k, i, d, x, y, z) schedule(static)
    for (s = 0; s < N; s++) {
        for (k = 0; k < 2; k++)
            for (d = 0; d < 3; d++)
                o->frc[k][d * N + s] = 0.0;
        if (o->owner[s] >= 0)
            continue;
        coords(o, s, &x, &y, &z);
        for (k = 0; k < 2; k++) {
            int kb = 1 - k;
            double sx = 0.0, sy = 0.0, sz = 0.0;
            for (i = 1; i < NQ; i++) {
                double ps = psi_at(o, kb, x, y, z, i);
                sx += WT[i] * ps * CX[i];
                sy += WT[i] * ps * CY[i];
                sz += WT[i] * ps * CZ[i];
            }
            o->frc[k][s] = -o->P.G * o->rho[k][s] * sx + o->rho[k][s] * o->P.body_force[0];
            o->frc[k][N + s] = -o->P.G * o->rho[k][s] * sy + o->rho[k][s] * o->P.body_force[1];
            o->frc[k][2 * N + s] = -o->P.G * o->rho[k][s] * sz + o->rho[k][s] * o->P.body_force[2];
        }
    }
    /* Eq. 21 on frontier solid nodes; net force and torque per particle */
    for (s = 0; s < N; s++) {
        int p = o->owner[s];
        double fs[3] = {0.0, 0.0, 0.0}, rel[3], tq[3], zero[3] = {0, 0, 0};
        int frontier = 0;
        if (p < 0)
            continue;
        coords(o, s, &x, &y, &z);
        for (k = 0; k < 2; k++) {
            int kb = 1 - k;
            double sx = 0.0, sy = 0.0, sz = 0.0;
            for (i = 1; i < NQ; i++) {
                long n = neighbour(o, x, y, z, i);
                if (n < 0 || o->owner[n] >= 0)
                    continue;
                frontier = 1;
                sx += WT[i] * o->rho[kb][n] * CX[i];
                sy += WT[i] * o->rho[kb][n] * CY[i];
                sz += WT[i] * o->rho[kb][n] * CZ[i];
            }
            fs[0] += -o->P.G * o->psi[k][s] * sx;
            fs[1] += -o->P.G * o->psi[k][s] * sy;
            fs[2] += -o->P.G * o->psi[k][s] * sz;
        }
        if (!frontier)
            continue;
        rel_pos(o, s, p, zero, rel);
        cross(rel, fs, tq);
        for (d = 0; d < 3; d++) {
            nadd(&acc[6 * p + d], fs[d]);
            nadd(&acc[6 * p + 3 + d], tq[d]);
        }
    }
    if (store_particle_terms)
        for (k = 0; k < o->nc; k++)
            for (d = 0; d < 3; d++) {
                o->Fs[3 * k + d] = nval(&acc[6 * k + d]);
                o->Ts[3 * k + d] = nval(&acc[6 * k + 3 + d]);
            }
    free(acc);
}

/* Step 5: Eq. 16 (BGK with the exact-difference source of Eq. 15) */
static void collide(orc_t *o)
{
    long s, N = o->N;
    int k, i;
    double nu0 = CS2 * (o->P.tau[0] - 0.5), nu1 = CS2 * (o->P.tau[1] - 0.5);
#pragma omp parallel for private(k, i) schedule(static)
    for (s = 0; s < N; s++) {
        double u[3], rt, inv_nu, nubar, om;
        if (o->owner[s] >= 0)
            continue;
        mix_velocity(o, s, u);
        rt = o->rho[0][s] + o->rho[1][s];
        inv_nu = (o->rho[0][s] / rt) / nu0 + (o->rho[1][s] / rt) / nu1;
        nubar = 1.0 / inv_nu;
        om = 1.0 / (nubar / CS2 + 0.5);
        for (k = 0; k < 2; k++) {
            double r = o->rho[k][s], us[3];
            us[0] = u[0]; us[1] = u[1]; us[2] = u[2];
            if (r > 1e-300) {
                us[0] = u[0] + o->frc[k][s] / r;
                us[1] = u[1] + o->frc[k][N + s] / r;
                us[2] = u[2] + o->frc[k][2 * N + s] / r;
            }
            for (i = 0; i < NQ; i++) {
                double e0 = feq_i(i, r, u);
                double e1 = feq_i(i, r, us);
                o->fpost[k][i * N + s] = (1.0 - om) * (o->f[k][i * N + s] - e0) + e1;
            }
        }
    }
}

/* Steps 6 and 8: bounce-back on particle and wall links (Eqs. 9, 17) with the
 * link forces of Eq. 19 summed into Eqs. 22-23, and streaming (Eq. 3). */
static void bounce_and_stream(orc_t *o)
{
    long s, N = o->N;
    int k, i, d, x, y, z, p;
    nsum *acc = (nsum *)zalloc(sizeof(nsum) * 6 * (size_t)(o->nc ? o->nc : 1));
    /* every (link, target) is written by one source site; the particle-link
     * sums run in site order, so with particles the loop is single-threaded */
#pragma omp parallel for private(k, i, d, x, y, z, p) schedule(static) if (o->nc == 0)
    for (s = 0; s < N; s++) {
        if (o->owner[s] >= 0)
            continue;
        coords(o, s, &x, &y, &z);
        for (i = 0; i < NQ; i++) {
            long n = neighbour(o, x, y, z, i);
            int ib = opposite(i);
            if (n >= 0 && o->owner[n] < 0) {
                for (k = 0; k < 2; k++)
                    o->fnext[k][i * N + n] = o->fpost[k][i * N + s];
            } else if (n < 0) {
                const int side = z + CZ[i] < 0 ? 0 : 1;
                const double *uw = side == 0 ? o->P.wall_u_lo : o->P.wall_u_hi;
                const int type = o->P.open[side];
                double cu = CX[i] * uw[0] + CY[i] * uw[1] + CZ[i] * uw[2];
                if (type == 1) {
                    /* pressure face (Eq. 10, anti-bounce-back): rho_w given,
                     * u_w the velocity of the boundary node (Eq. 14), or its
                     * first-order extrapolation to the face */
                    double um[3], cum, uu;
                    face_velocity(o, s, side, um);
                    cum = CX[i] * um[0] + CY[i] * um[1] + CZ[i] * um[2];
                    uu = um[0] * um[0] + um[1] * um[1] + um[2] * um[2];
                    for (k = 0; k < 2; k++)
                        o->fnext[k][ib * N + s] =
                            -o->fpost[k][i * N + s] +
                            2.0 * WT[i] * o->P.open_rho[side][k] *
                                (1.0 + cum * cum / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
                } else if (type == 3) {
                    /* equilibrium face: the incoming population is
                     * f^eq_ibar(rho_w, u_w) (Eq. 5) */
                    for (k = 0; k < 2; k++)
                        o->fnext[k][ib * N + s] = feq_i(ib, o->P.open_rho[side][k], uw);
                } else {
                    /* wall or velocity face (Eq. 9); rho_w the density of
                     * the boundary node, or on a velocity face its
                     * first-order extrapolation to the face */
                    for (k = 0; k < 2; k++) {
                        double rw = type == 2 ? face_density(o, s, side, k) : o->rho[k][s];
                        o->fnext[k][ib * N + s] = o->fpost[k][i * N + s] - 2.0 * WT[i] * rw * cu / CS2;
                    }
                }
            } else {
                double off[3], rel[3], uw[3], cu, fl = 0.0, fv[3], tq[3];
                p = o->owner[n];
                off[0] = 0.5 * CX[i];
                off[1] = 0.5 * CY[i];
                off[2] = 0.5 * CZ[i];
                rel_pos(o, s, p, off, rel);
                wall_velocity(o, p, rel, uw);
                cu = CX[i] * uw[0] + CY[i] * uw[1] + CZ[i] * uw[2];
                for (k = 0; k < 2; k++) {
                    double corr = 2.0 * WT[i] * o->rho[k][s] * cu / CS2;
                    o->fnext[k][ib * N + s] = o->fpost[k][i * N + s] - corr;
                    fl += 2.0 * o->fpost[k][i * N + s] - corr;
                }
                fv[0] = fl * CX[i];
                fv[1] = fl * CY[i];
                fv[2] = fl * CZ[i];
                cross(rel, fv, tq);
                for (d = 0; d < 3; d++) {
                    nadd(&acc[6 * p + d], fv[d]);
                    nadd(&acc[6 * p + 3 + d], tq[d]);
                }
            }
        }
    }
    for (p = 0; p < o->nc; p++)
        for (d = 0; d < 3; d++) {
            o->Fliq[3 * p + d] = nval(&acc[6 * p + d]);
            o->Tliq[3 * p + d] = nval(&acc[6 * p + 3 + d]);
        }
    free(acc);
    for (k = 0; k < 2; k++) {
        double *t = o->f[k];
        o->f[k] = o->fnext[k];
        o->fnext[k] = t;
    }
}

/* Eq. 33: qdot = 1/2 Q(q) (0, w*) */
static void quat_rate(const double q[4], const double w[3], double qd[4])
{
    qd[0] = 0.5 * (-q[1] * w[0] - q[2] * w[1] - q[3] * w[2]);
    qd[1] = 0.5 * (q[0] * w[0] - q[3] * w[1] + q[2] * w[2]);
    qd[2] = 0.5 * (q[3] * w[0] + q[0] * w[1] - q[1] * w[2]);
    qd[3] = 0.5 * (-q[2] * w[0] + q[1] * w[1] + q[0] * w[2]);
}

/* body-frame angular velocity w* = R(q/|q|)^T w with R from Eq. 31 */
static void body_omega(const double q[4], const double w[3], double wb[3])
{
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double a = q[0] / n, b = q[1] / n, c = q[2] / n, e = q[3] / n;
    double R[3][3];
    int i, j;
    R[0][0] = a * a + b * b - c * c - e * e;
    R[0][1] = 2.0 * (b * c - a * e);
    R[0][2] = 2.0 * (b * e + a * c);
    R[1][0] = 2.0 * (b * c + a * e);
    R[1][1] = a * a - b * b + c * c - e * e;
    R[1][2] = 2.0 * (c * e - a * b);
    R[2][0] = 2.0 * (b * e - a * c);
    R[2][1] = 2.0 * (c * e + a * b);
    R[2][2] = a * a - b * b - c * c + e * e;
    for (i = 0; i < 3; i++) {
        wb[i] = 0.0;
        for (j = 0; j < 3; j++)
            wb[i] += R[j][i] * w[j];
    }
}

/* Step 7 for one particle: Eq. 32 (leap-frog) with Eqs. 33-34 (Svanberg's
 * implicit mid-step quaternion).  F and T are the totals of Eq. 35.
 * L[d] > 0 wraps the position periodically along d. */
void orc_integrate_one(double *r, double *v, double *w, double *q, double m, double R,
                       const double *F, const double *T, int rotate, const int *L)
{
    int d, it;
    for (d = 0; d < 3; d++) {
        v[d] = v[d] + F[d] / m;
        r[d] = r[d] + v[d];
        if (L[d] > 0)
            r[d] = r[d] - (double)L[d] * floor(r[d] / (double)L[d]);
    }
    if (rotate) {
        double I = 0.4 * m * R * R;
        double wb[3], qd[4], qd_old[4], qh[4], nq;
        for (d = 0; d < 3; d++)
            w[d] = w[d] + T[d] / I;
        body_omega(q, w, wb);
        quat_rate(q, wb, qd_old);
        for (d = 0; d < 4; d++)
            qh[d] = q[d] + 0.5 * qd_old[d];
        for (it = 0; it < 20; it++) {
            double delta = 0.0;
            body_omega(qh, w, wb);
            quat_rate(qh, wb, qd);
            for (d = 0; d < 4; d++) {
                double dd = fabs(qd[d] - qd_old[d]);
                if (dd > delta)
                    delta = dd;
                qh[d] = q[d] + 0.5 * qd[d];
                qd_old[d] = qd[d];
            }
            if (delta <= 1e-14)
                break;
        }
        for (d = 0; d < 4; d++)
            q[d] = q[d] + qd_old[d];
        nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        for (d = 0; d < 4; d++)
            q[d] = q[d] / nq;
    }
}

static void integrate(orc_t *o)
{
    int p, d;
    int L[3];
    L[0] = o->P.bc[0] ? o->nx : 0;
    L[1] = o->P.bc[1] ? o->ny : 0;
    L[2] = o->P.bc[2] ? o->nz : 0;
    for (p = 0; p < o->nc; p++) {
        if (!o->prev_valid[p])
            for (d = 0; d < 3; d++) {
                o->Fliq_prev[3 * p + d] = o->Fliq[3 * p + d];
                o->Tliq_prev[3 * p + d] = o->Tliq[3 * p + d];
            }
        for (d = 0; d < 3; d++) {
            o->Ftot[3 * p + d] = 0.5 * (o->Fliq_prev[3 * p + d] + o->Fliq[3 * p + d]) +
                                 o->Fd[3 * p + d] + o->Fc[3 * p + d] + o->Fs[3 * p + d] +
                                 o->Fpair[3 * p + d];
            o->Ttot[3 * p + d] = 0.5 * (o->Tliq_prev[3 * p + d] + o->Tliq[3 * p + d]) +
                                 o->Td[3 * p + d] + o->Tc[3 * p + d] + o->Ts[3 * p + d];
        }
        orc_integrate_one(&o->pos[3 * p], &o->vel[3 * p], &o->omg[3 * p], &o->quat[4 * p],
                          o->mass[p], o->rad[p], &o->Ftot[3 * p], &o->Ttot[3 * p], o->P.rotate, L);
        for (d = 0; d < 3; d++) {
            o->Fliq_prev[3 * p + d] = o->Fliq[3 * p + d];
            o->Tliq_prev[3 * p + d] = o->Tliq[3 * p + d];
        }
        o->prev_valid[p] = 1;
    }
}

/* -------------------------------------------------------------- public */
int orc_add_colloids(orc_t *o, int n, const double *pos, const double *vel, const double *omega,
                     const double *quat, const double *radius, const double *mass)
{
    int p, d;
    int L[3];
    if (!o || n < 0 || !pos || !radius || !mass)
        return ORC_ERR_ARG;
    if (!o->have_fields)
        return ORC_ERR_STATE;
    if (o->nc + n > o->maxc)
        return ORC_ERR_STATE;
    L[0] = o->nx; L[1] = o->ny; L[2] = o->nz;
    for (p = 0; p < n; p++) {
        int q = o->nc + p;
        if (!(radius[p] > 0.0) || !(mass[p] > 0.0))
            return ORC_ERR_ARG;
        for (d = 0; d < 3; d++) {
            double x = pos[3 * p + d];
            if (o->P.bc[d]) {
                if (2.0 * radius[p] + 4.0 > (double)L[d])
                    return ORC_ERR_ARG;
                x = x - (double)L[d] * floor(x / (double)L[d]);
            } else if (x < 0.0 || x > (double)L[d] - 1.0) {
                return ORC_ERR_ARG;
            }
            o->pos[3 * q + d] = x;
            o->vel[3 * q + d] = vel ? vel[3 * p + d] : 0.0;
            o->omg[3 * q + d] = omega ? omega[3 * p + d] : 0.0;
        }
        for (d = 0; d < 4; d++)
            o->quat[4 * q + d] = quat ? quat[4 * p + d] : (d == 0 ? 1.0 : 0.0);
        o->rad[q] = radius[p];
        o->mass[q] = mass[p];
        o->prev_valid[q] = 0;
    }
    o->nc += n;
    o->err = ORC_OK;
    remap(o, 1);
    return o->err;
}

int orc_step(orc_t *o, int nsteps)
{
    int t;
    if (!o || nsteps < 0)
        return ORC_ERR_ARG;
    if (!o->have_fields)
        return ORC_ERR_STATE;
    for (t = 0; t < nsteps; t++) {
        o->err = ORC_OK;
        moments(o);            /* 1 */
        if (o->nc > 0)
            remap(o, 0);       /* 2 */
        pair_forces(o);        /* 3 */
        lb_forces(o, 1);       /* 4 */
        collide(o);            /* 5 */
        bounce_and_stream(o);  /* 6 and 8 (targets are disjoint) */
        integrate(o);          /* 7 */
        if (o->err)
            return o->err;
    }
    return ORC_OK;
}

/* rho^k and the half-force-corrected mixture velocity
 * u = sum_k (j^k + F^k/2) / rho (end of Sec. 2.3) of the current state, with
 * the forces evaluated on the current node map.  Solid nodes read zero. */
int orc_get_fields(orc_t *o, double *rhoA, double *rhoB, double *u)
{
    long s, N;
    int d;
    if (!o)
        return ORC_ERR_ARG;
    if (!o->have_fields)
        return ORC_ERR_STATE;
    N = o->N;
    moments(o);
    lb_forces(o, 0);
    for (s = 0; s < N; s++) {
        double rt = o->rho[0][s] + o->rho[1][s];
        if (rhoA)
            rhoA[s] = o->rho[0][s];
        if (rhoB)
            rhoB[s] = o->rho[1][s];
        if (u)
            for (d = 0; d < 3; d++)
                u[d * N + s] = o->owner[s] >= 0 ? 0.0
                    : (o->jm[0][d * N + s] + 0.5 * o->frc[0][d * N + s] +
                       o->jm[1][d * N + s] + 0.5 * o->frc[1][d * N + s]) / rt;
    }
    return ORC_OK;
}

/* out: mass^A, mass^B, sum j (3), sum (j + F/2) (3) over fluid nodes */
int orc_totals(orc_t *o, double *out)
{
    long s, N;
    int k, d;
    nsum a[8];
    if (!o || !out)
        return ORC_ERR_ARG;
    memset(a, 0, sizeof(a));
    N = o->N;
    moments(o);
    lb_forces(o, 0);
    for (s = 0; s < N; s++) {
        if (o->owner[s] >= 0)
            continue;
        for (k = 0; k < 2; k++) {
            nadd(&a[k], o->rho[k][s]);
            for (d = 0; d < 3; d++) {
                nadd(&a[2 + d], o->jm[k][d * N + s]);
                nadd(&a[5 + d], o->jm[k][d * N + s] + 0.5 * o->frc[k][d * N + s]);
            }
        }
    }
    for (k = 0; k < 8; k++)
        out[k] = nval(&a[k]);
    return ORC_OK;
}

int orc_get_colloids(orc_t *o, double *pos, double *vel, double *omega, double *quat,
                     double *force, double *torque)
{
    int p, d;
    if (!o)
        return ORC_ERR_ARG;
    for (p = 0; p < o->nc; p++) {
        for (d = 0; d < 3; d++) {
            if (pos) pos[3 * p + d] = o->pos[3 * p + d];
            if (vel) vel[3 * p + d] = o->vel[3 * p + d];
            if (omega) omega[3 * p + d] = o->omg[3 * p + d];
            if (force) force[3 * p + d] = o->Ftot[3 * p + d];
            if (torque) torque[3 * p + d] = o->Ttot[3 * p + d];
        }
        for (d = 0; d < 4; d++)
            if (quat) quat[4 * p + d] = o->quat[4 * p + d];
    }
    return o->nc;
}

/* per-particle force terms of the last step, [nc][3]:
 * 0 F_liq(t+1/2), 1 T_liq, 2 F_d, 3 T_d, 4 F_c, 5 T_c, 6 F_s, 7 T_s,
 * 8 F_pair, 9 F_total, 10 T_total */
int orc_get_colloid_terms(orc_t *o, int which, double *out)
{
    const double *src[11];
    int p, d;
    if (!o || !out || which < 0 || which > 10)
        return ORC_ERR_ARG;
    src[0] = o->Fliq; src[1] = o->Tliq; src[2] = o->Fd; src[3] = o->Td;
    src[4] = o->Fc; src[5] = o->Tc; src[6] = o->Fs; src[7] = o->Ts;
    src[8] = o->Fpair; src[9] = o->Ftot; src[10] = o->Ttot;
    for (p = 0; p < o->nc; p++)
        for (d = 0; d < 3; d++)
            out[3 * p + d] = src[which][3 * p + d];
    return ORC_OK;
}

/* raw populations of component k, [19][N] */
int orc_get_populations(orc_t *o, int k, double *out)
{
    if (!o || !out || k < 0 || k > 1)
        return ORC_ERR_ARG;
    memcpy(out, o->f[k], sizeof(double) * NQ * o->N);
    return ORC_OK;
}

int orc_set_populations(orc_t *o, int k, const double *in)
{
    if (!o || !in || k < 0 || k > 1)
        return ORC_ERR_ARG;
    memcpy(o->f[k], in, sizeof(double) * NQ * o->N);
    o->have_fields = 1;
    return ORC_OK;
}

/* psi^k of the last force evaluation, [N]: the virtual density (Eq. 20) on
 * particle frontier nodes, 0 elsewhere */
int orc_get_psi(orc_t *o, int k, double *out)
{
    if (!o || !out || k < 0 || k > 1)
        return ORC_ERR_ARG;
    memcpy(out, o->psi[k], sizeof(double) * o->N);
    return ORC_OK;
}

/* node map: -1 fluid, else the owning particle */
int orc_get_owner(orc_t *o, int *out)
{
    if (!o || !out)
        return ORC_ERR_ARG;
    memcpy(out, o->owner, sizeof(int) * o->N);
    return ORC_OK;
}

int orc_set_colloid_state(orc_t *o, int p, const double *pos, const double *vel,
                          const double *omega, const double *quat)
{
    int d;
    if (!o || p < 0 || p >= o->nc)
        return ORC_ERR_ARG;
    for (d = 0; d < 3; d++) {
        if (pos) o->pos[3 * p + d] = pos[d];
        if (vel) o->vel[3 * p + d] = vel[d];
        if (omega) o->omg[3 * p + d] = omega[d];
    }
    if (quat)
        for (d = 0; d < 4; d++)
            o->quat[4 * p + d] = quat[d];
    return ORC_OK;
}

/* OpenMP threads used by the site loops (n <= 0: all available); returns the
 * count now in effect, 1 in a build without OpenMP. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n <= 0)
        n = omp_get_num_procs();
    omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
