/*
 * pic_oracle.c -- plain FP64 CPU oracle for the 1D electrostatic electron
 * Particle-in-Cell method of Markidis & Lapenta, "Development and
 * performance analysis of a UPC Particle-in-Cell code" (PGAS10).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this code.  The CUDA library never calls
 * it, and the two share no code, header or constant table.
 *
 * Every function restates one passage of the paper in its own notation
 * (xg, rho, phi, E, xp, vp, Q0, qoms0, rho_init0, dx, ig, w1, w2):
 *   Sec. 2.1, Eqs. 2-3     leapfrog mover (position, velocity)
 *   Sec. 2.2, Eqs. 6-7     finite-difference Poisson, central-difference E
 *   Sec. 2.3               linear (two-cell) charge and field interpolation
 *   Appendix A             the periodic wrap, the CG solver, the cycle
 *                          order, the lattice ("quiet start") loading
 *   Sec. 4, Fig. 1         the two-stream beams and the phase-space
 *                          snapshot counts
 * Equation numbers count the displayed lines of Sec. 2: Eq. 1 equation of
 * motion, Eqs. 2-3 leapfrog, Eq. 4 Poisson, Eq. 5 E = -dPhi/dx, Eq. 6
 * discrete Poisson, Eq. 7 discrete E.
 *
 * Readings where the paper is ambiguous:
 *   R1  field solve: the converged solution of Eq. 6 with Phi_0 = 0 (the
 *       listing's CG with 150 fixed iterations is kept as orc_field_cg);
 *   R2  weights: the listing's cell-centred linear weighting, not the
 *       garbled "w1 = (x_p - x_g)/dx" sentence of Sec. 2.3;
 *   R3  wrap: positions live in [0, Lx);
 *   R5  fixed-point deposit (orc_deposit_fixed): the build's exact integer
 *       form of the Sec. 2.3 weighting, stated at the function;
 *   R13 nearest-grid-point weighting (shape ORC_NGP): the cell xp belongs
 *       to, trunc(xp/dx), takes the whole charge and gives its field;
 *   R6  loading: beams by particle parity, the thermal spread by Box-Muller
 *       on a named counter-based generator (orc_load_two_stream).
 *
 * Parity status: every exported function is pinned by a test against
 * something other than itself (closed forms, invariants, brute force, a
 * library solve); no function here is "parity unpinned".
 *
 * Build: plain C99, -O2 -ffp-contract=off (no fused multiply-add, so float
 * and double expressions round exactly as written).
 */
#define _POSIX_C_SOURCE 200809L
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Run parameters, named as in the Appendix A parameter block. */
typedef struct orc_params {
    int32_t ng;        /* NG: number of cells (grid points)              */
    int32_t shape;     /* ORC_CIC (the listing's two-cell weighting) or
                          ORC_NGP (the cell's own node, Sec. 2)          */
    int64_t np;        /* NP: number of particles                        */
    double  lx;        /* Lx: box length                                 */
    double  dt;        /* dt: time step                                  */
    double  qoms0;     /* qoms0: charge-to-mass ratio (-1 for electrons) */
    double  rho_init0; /* rho_init0: density of the immobile ions        */
} orc_params;

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ERANGE (-2)

#define ORC_CIC 0
#define ORC_NGP 1

static double orc_dx(const orc_params *p) { return p->lx / (double)p->ng; }

/* Particle charge Q0 (Appendix A parameter block): the ion charge of the box
 * rho_init0*Lx shared over NP particles, with the sign of qoms0. */
static double orc_q0(const orc_params *p)
{
    return (p->rho_init0 * p->lx / (double)p->np) * (p->qoms0 / fabs(p->qoms0));
}

/* Particle mass m = Q0 / qoms0. */
double orc_particle_mass(const orc_params *p) { return orc_q0(p) / p->qoms0; }

/* Periodic boundary (Appendix A, the wrap in the particle loop), reading R3:
 * x < 0 gains Lx, x >= Lx loses Lx; a negative x so small that x + Lx rounds
 * to Lx is the point 0.  One wrap per step suffices because |v dt| < Lx. */
static double orc_wrap(double x, double lx)
{
    if (x < 0.0) x += lx;
    else if (x >= lx) x -= lx;
    if (x >= lx) x = 0.0;
    return x;
}

/* Charge deposit, particle to grid (Sec. 2.3; Appendix A "Interpolation
 * particle to grid"), reading R2.  The ions add rho_init0 to every node
 * (Sec. 2: immobile neutralising protons).  A particle at xp with
 * ig = trunc(xp/dx + 1/2) gives w2 = 1 - w1 of its charge density Q0/dx to
 * node ig and w1 = (xg[ig] - xp)/dx to node ig - 1; node indices are taken
 * periodically (ig = 0 shares with node NG-1, ig = NG is node 0), which is
 * what the listing's ghost cells do with a single domain.
 * Returns ORC_ERANGE if a position lies outside [0, Lx]. */
/* Nearest-grid-point weighting (Sec. 2: the density at a grid point counts
 * the particles of its cell, and a particle feels the field of the cell it
 * belongs to).  With nodes at the cell centres, the cell of xp is
 * ig = trunc(xp/dx) and its node is the nearest one; xp == Lx is the periodic
 * image of 0 (cell 0). */
static int orc_cell_ngp(const orc_params *p, double x)
{
    int ig = (int)(x / orc_dx(p));
    return ig >= p->ng ? ig - p->ng : ig;
}

static int orc_deposit_ngp(const orc_params *p, const double *xp, double *rho)
{
    const int ng = p->ng;
    const double dx = orc_dx(p), Q0 = orc_q0(p);
    for (int ic = 0; ic < ng; ic++) rho[ic] = p->rho_init0;
    for (int64_t ip = 0; ip < p->np; ip++) {
        double x = xp[ip];
        if (!(x >= 0.0 && x <= p->lx)) return ORC_ERANGE;
        rho[orc_cell_ngp(p, x)] += Q0 / dx;
    }
    return ORC_OK;
}

/* The linear weighting of one particle at x (Sec. 2.3, reading R2):
 * ig = trunc(x/dx + 1/2); node *a (the node at or above x) takes w2 = 1 - w1
 * and node *b (the one below) w1 = (xg[a] - x)/dx, with the periodic ends
 * (ig = 0: a = 0, b = NG-1; ig = NG: a = NG-1, b = 0, the weights measured
 * from the last centre).  Returns ig. */
static int orc_cic(const orc_params *p, double x, double dx, double xg_last,
                   int *a, int *b, double *w1, double *w2)
{
    const int ng = p->ng;
    int ig = (int)(x / dx + 0.5);
    if (ig == 0) {
        *w1 = (dx / 2.0 - x) / dx; *w2 = 1 - *w1;
        *a = 0; *b = ng - 1;
    } else if (ig >= ng) {
        *w1 = (x - xg_last) / dx; *w2 = 1 - *w1;
        *a = ng - 1; *b = 0;
    } else {
        double xg = dx / 2.0 + dx * ig;
        *w1 = (xg - x) / dx; *w2 = 1 - *w1;
        *a = ig; *b = ig - 1;
    }
    return ig;
}

int orc_deposit(const orc_params *p, const double *xp, double *rho)
{
    if (p->shape == ORC_NGP) return orc_deposit_ngp(p, xp, rho);
    const int ng = p->ng;
    const double dx = orc_dx(p), Q0 = orc_q0(p);
    const double xg_last = dx / 2.0 + dx * (ng - 1);
    for (int ic = 0; ic < ng; ic++) rho[ic] = p->rho_init0;
    for (int64_t ip = 0; ip < p->np; ip++) {
        double x = xp[ip];
        if (!(x >= 0.0 && x <= p->lx)) return ORC_ERANGE;
        int a, b;
        double w1, w2;
        orc_cic(p, x, dx, xg_last, &a, &b, &w1, &w2);
        rho[a] += w2 * Q0 / dx;
        rho[b] += w1 * Q0 / dx;
    }
    return ORC_OK;
}

/* Field solve (Sec. 2.2, Eq. 6), reading R1: the exact solution of
 *   Phi[g+1] - 2 Phi[g] + Phi[g-1] = -rho[g] dx^2,  g = 1 .. NG-1,
 * with Phi[0] = 0 pinned as the listing's CG pins it, and Phi[NG] = Phi[0]
 * (periodic).  The g = 0 equation is the sum of the others when the box is
 * neutral.  Solved directly by the tridiagonal (Thomas) elimination.
 * work must hold 2*NG doubles. */
int orc_field_solve(const orc_params *p, const double *rho, double *phi,
                    double *work)
{
    const int ng = p->ng;
    const double dx = orc_dx(p);
    double *cp = work, *dp = work + ng;
    phi[0] = 0.0;
    int m = ng - 1; /* unknowns Phi[1..NG-1] */
    if (m <= 0) return ORC_OK;
    /* a = 1 (sub), b = -2 (diagonal), c = 1 (super), rhs d = -rho dx^2 */
    cp[1] = 1.0 / -2.0;
    dp[1] = (-rho[1] * dx * dx) / -2.0;
    for (int g = 2; g <= m; g++) {
        double den = -2.0 - cp[g - 1];
        cp[g] = 1.0 / den;
        dp[g] = ((-rho[g] * dx * dx) - dp[g - 1]) / den;
    }
    phi[m] = dp[m];
    for (int g = m - 1; g >= 1; g--) phi[g] = dp[g] - cp[g] * phi[g + 1];
    return ORC_OK;
}

/* The listing's matrix-free Conjugate Gradient (Sec. 2.2, Sec. 3.3,
 * Appendix A "CG SOLVER"): x = 0, r = v = -rho dx^2 except r[0] = v[0] = 0,
 * c = r.r; then maxit iterations of z = A v (row 0 the identity for the
 * pinned Phi[0], row NG-1 taking Phi[NG] = 0), t = c/(z.v), x += t v,
 * r -= t z, d = r.r, v = (d/c) v + r, c = d.  The listing stops on nothing
 * but maxit; here a zero residual (r.r == 0 or z.v == 0, where the next
 * step would divide by zero) also ends it.  Returns the iterations done.
 * work must hold 3*NG doubles. */
int orc_field_cg(const orc_params *p, const double *rho, int maxit,
                 double *phi, double *work)
{
    const int ng = p->ng;
    const double dx = orc_dx(p);
    double *r = work, *v = work + ng, *z = work + 2 * ng, *xk = phi;
    for (int ic = 0; ic < ng; ic++) xk[ic] = 0.0;
    r[0] = 0.0; v[0] = 0.0;
    for (int ic = 1; ic < ng; ic++) { r[ic] = -rho[ic] * dx * dx; v[ic] = r[ic]; }
    double c = 0.0;
    for (int ic = 0; ic < ng; ic++) c += r[ic] * r[ic];
    int it = 0;
    if (sqrt(c) > 1e-16 && ng > 1) {
        while (it < maxit) {
            z[0] = v[0];
            z[ng - 1] = v[ng - 2] - 2 * v[ng - 1];
            for (int ic = 1; ic < ng - 1; ic++) z[ic] = v[ic - 1] - 2 * v[ic] + v[ic + 1];
            double dotzv = 0.0;
            for (int ic = 0; ic < ng; ic++) dotzv += z[ic] * v[ic];
            if (!(dotzv != 0.0)) break;
            double t = c / dotzv;
            if (!isfinite(t)) break;
            for (int ic = 0; ic < ng; ic++) xk[ic] += t * v[ic];
            for (int ic = 0; ic < ng; ic++) r[ic] -= t * z[ic];
            double d = 0.0;
            for (int ic = 0; ic < ng; ic++) d += r[ic] * r[ic];
            it++;
            if (!(d > 0.0)) break;
            for (int ic = 0; ic < ng; ic++) v[ic] = (d / c) * v[ic] + r[ic];
            c = d;
        }
    }
    return it;
}

/* Electric field by central difference (Sec. 2.2, Eq. 7) with periodic
 * neighbours at both ends (Appendix A, the electric-field step). */
void orc_efield(const orc_params *p, const double *phi, double *E)
{
    const int ng = p->ng;
    const double dx = orc_dx(p);
    for (int ic = 0; ic < ng; ic++) {
        int ir = (ic + 1 == ng) ? 0 : ic + 1;
        int il = (ic == 0) ? ng - 1 : ic - 1;
        E[ic] = -(phi[ir] - phi[il]) / (2 * dx);
    }
}

/* Field at the particles, grid to particle (Sec. 2.3: the deposit's weighting
 * used in reverse; Appendix A velocity loop): Ex = w2 E[ig] + w1 E[ig-1] with the same
 * weights and periodic ends as orc_deposit. */
int orc_gather(const orc_params *p, const double *xp, const double *E,
               double *Ex)
{
    if (p->shape == ORC_NGP) {
        for (int64_t ip = 0; ip < p->np; ip++) {
            double x = xp[ip];
            if (!(x >= 0.0 && x <= p->lx)) return ORC_ERANGE;
            Ex[ip] = E[orc_cell_ngp(p, x)];
        }
        return ORC_OK;
    }
    const int ng = p->ng;
    const double dx = orc_dx(p);
    const double xg_last = dx / 2.0 + dx * (ng - 1);
    for (int64_t ip = 0; ip < p->np; ip++) {
        double x = xp[ip];
        if (!(x >= 0.0 && x <= p->lx)) return ORC_ERANGE;
        int a, b;
        double w1, w2;
        orc_cic(p, x, dx, xg_last, &a, &b, &w1, &w2);
        Ex[ip] = w2 * E[a] + w1 * E[b];
    }
    return ORC_OK;
}

/* Velocity update (Sec. 2.1, Eq. 3): v^{n+1/2} = v^{n-1/2} + qoms0 E_p dt. */
void orc_kick(const orc_params *p, const double *Ex, double *vp)
{
    for (int64_t ip = 0; ip < p->np; ip++) vp[ip] += p->qoms0 * Ex[ip] * p->dt;
}

/* Position update (Sec. 2.1, Eq. 2) and the periodic wrap:
 * x^{n+1} = wrap(x^n + v^{n+1/2} dt). */
void orc_drift(const orc_params *p, const double *vp, double *xp)
{
    for (int64_t ip = 0; ip < p->np; ip++)
        xp[ip] = orc_wrap(xp[ip] + vp[ip] * p->dt, p->lx);
}

/* rho -> phi -> E for one density: Eq. 6 then Eq. 7. work: 2*NG doubles. */
int orc_field(const orc_params *p, const double *rho, double *phi, double *E,
              double *work)
{
    int rc = orc_field_solve(p, rho, phi, work);
    if (rc) return rc;
    orc_efield(p, phi, E);
    return ORC_OK;
}

/* Set-up of the step state (x^0 given): rho^0, phi^0, E^0. */
int orc_prepare(const orc_params *p, const double *xp, double *rho,
                double *phi, double *E, double *work)
{
    int rc = orc_deposit(p, xp, rho);
    if (rc) return rc;
    return orc_field(p, rho, phi, E, work);
}

/* One step in the library's order, from the state (x^n, v^{n-1/2}, E^n):
 * gather E^n at x^n, kick to v^{n+1/2} (Eq. 3), drift and wrap to x^{n+1}
 * (Eq. 2), deposit rho^{n+1}, solve phi^{n+1} (Eq. 6), E^{n+1} (Eq. 7).
 * sums (may be NULL) receives sum v^{n-1/2} v^{n+1/2} and sum v^{n+1/2}.
 * work: NP + 2*NG doubles. */
int orc_step(const orc_params *p, double *xp, double *vp, double *rho,
             double *phi, double *E, double *work, double *sums)
{
    double *Ex = work, *fw = work + p->np;
    int rc = orc_gather(p, xp, E, Ex);
    if (rc) return rc;
    double svv = 0.0, sv = 0.0;
    for (int64_t ip = 0; ip < p->np; ip++) {
        double vold = vp[ip];
        vp[ip] = vold + p->qoms0 * Ex[ip] * p->dt;
        svv += vold * vp[ip];
        sv += vp[ip];
    }
    if (sums) { sums[0] = svv; sums[1] = sv; }
    orc_drift(p, vp, xp);
    return orc_prepare(p, xp, rho, phi, E, fw);
}

/* ---------------------------------------------------------------------
 * orc_step on several host threads, for timing the oracle on all cores.
 * The state it leaves (x, v, rho, phi, E) is bit for bit that of orc_step:
 *   - the gather, kick, drift and wrap of each particle are the serial
 *     code's operations on that particle, the particles split in ranges;
 *   - the deposit is split by nodes, not particles: each thread owns a
 *     range of nodes, scans every particle in order and adds only to its
 *     own nodes, so every node receives the serial code's additions in the
 *     serial order;
 *   - the field solve is the serial one.
 * Only the two sums (sum v_old v_new, sum v_new) add the same terms in
 * another grouping (per thread range, then over the ranges in order).
 * CIC shape only.  ig: NP ints of work.
 * --------------------------------------------------------------------- */
#include <pthread.h>

typedef struct {
    const orc_params *p;
    double *xp, *vp;
    const double *E;
    int32_t *ig;
    int64_t lo, hi;
    double svv, sv;
    int rc;
} orc_push_job;

static void *orc_push_range(void *arg)
{
    orc_push_job *j = (orc_push_job *)arg;
    const orc_params *p = j->p;
    const double dx = orc_dx(p);
    const double xg_last = dx / 2.0 + dx * (p->ng - 1);
    double svv = 0.0, sv = 0.0;
    j->rc = ORC_OK;
    for (int64_t ip = j->lo; ip < j->hi; ip++) {
        double x = j->xp[ip];
        if (!(x >= 0.0 && x <= p->lx)) { j->rc = ORC_ERANGE; return NULL; }
        int a, b;
        double w1, w2;
        orc_cic(p, x, dx, xg_last, &a, &b, &w1, &w2);
        double Ex = w2 * j->E[a] + w1 * j->E[b];
        double vold = j->vp[ip];
        j->vp[ip] = vold + p->qoms0 * Ex * p->dt;
        svv += vold * j->vp[ip];
        sv += j->vp[ip];
        x = orc_wrap(j->xp[ip] + j->vp[ip] * p->dt, p->lx);
        j->xp[ip] = x;
        if (!(x >= 0.0 && x <= p->lx)) { j->rc = ORC_ERANGE; return NULL; }
        j->ig[ip] = (int32_t)(x / dx + 0.5);
    }
    j->svv = svv;
    j->sv = sv;
    return NULL;
}

typedef struct {
    const orc_params *p;
    const double *xp;
    const int32_t *ig;
    double *rho;
    int g0, g1;
} orc_dep_job;

/* Does a particle with this ig touch a node in [g0, g1)? (the nodes orc_cic
 * picks: ig and ig-1, NG-1 for ig = 0, 0 and NG-1 for ig >= NG) */
static int orc_touches(int ig, int ng, int g0, int g1)
{
    int a = ig >= ng ? ng - 1 : ig;
    int b = ig == 0 ? ng - 1 : (ig >= ng ? 0 : ig - 1);
    return (a >= g0 && a < g1) || (b >= g0 && b < g1);
}

static void *orc_deposit_nodes(void *arg)
{
    orc_dep_job *j = (orc_dep_job *)arg;
    const orc_params *p = j->p;
    const int ng = p->ng;
    const double dx = orc_dx(p), Q0 = orc_q0(p);
    const double xg_last = dx / 2.0 + dx * (ng - 1);
    for (int ic = j->g0; ic < j->g1; ic++) j->rho[ic] = p->rho_init0;
    for (int64_t ip = 0; ip < p->np; ip++) {
        if (!orc_touches(j->ig[ip], ng, j->g0, j->g1)) continue;
        int a, b;
        double w1, w2;
        orc_cic(p, j->xp[ip], dx, xg_last, &a, &b, &w1, &w2);
        if (a >= j->g0 && a < j->g1) j->rho[a] += w2 * Q0 / dx;
        if (b >= j->g0 && b < j->g1) j->rho[b] += w1 * Q0 / dx;
    }
    return NULL;
}

#define ORC_MAX_THREADS 256

int orc_step_threads(const orc_params *p, double *xp, double *vp, double *rho,
                     double *phi, double *E, double *work, double *sums,
                     int32_t *ig, int nthreads)
{
    if (p->shape != ORC_CIC || nthreads < 1 || nthreads > ORC_MAX_THREADS)
        return ORC_EINVAL;
    pthread_t th[ORC_MAX_THREADS];
    orc_push_job pj[ORC_MAX_THREADS];
    orc_dep_job dj[ORC_MAX_THREADS];
    int nt = nthreads;
    for (int t = 0; t < nt; t++) {
        pj[t].p = p; pj[t].xp = xp; pj[t].vp = vp; pj[t].E = E; pj[t].ig = ig;
        pj[t].lo = p->np * t / nt;
        pj[t].hi = p->np * (t + 1) / nt;
        pj[t].svv = 0.0; pj[t].sv = 0.0;
        if (pthread_create(&th[t], NULL, orc_push_range, &pj[t]) != 0) return ORC_EINVAL;
    }
    int rc = ORC_OK;
    double svv = 0.0, sv = 0.0;
    for (int t = 0; t < nt; t++) {
        pthread_join(th[t], NULL);
        if (pj[t].rc) rc = pj[t].rc;
        svv += pj[t].svv;
        sv += pj[t].sv;
    }
    if (rc) return rc;
    if (sums) { sums[0] = svv; sums[1] = sv; }
    int ntd = nt < p->ng ? nt : p->ng;
    for (int t = 0; t < ntd; t++) {
        dj[t].p = p; dj[t].xp = xp; dj[t].ig = ig; dj[t].rho = rho;
        dj[t].g0 = (int)((int64_t)p->ng * t / ntd);
        dj[t].g1 = (int)((int64_t)p->ng * (t + 1) / ntd);
        if (pthread_create(&th[t], NULL, orc_deposit_nodes, &dj[t]) != 0) return ORC_EINVAL;
    }
    for (int t = 0; t < ntd; t++) pthread_join(th[t], NULL);
    return orc_field(p, rho, phi, E, work + p->np);
}

/* nt cycles in the order of the Appendix A time loop and the summary of
 * Sec. 2.4: drift + wrap (Eq. 2), deposit, solve (Eq. 6), E (Eq. 7), then
 * gather and kick (Eq. 3).  The listing drifts first, so vp enters as
 * v^{1/2}.  On return x = x^{nt}, v = v^{nt+1/2}, E = E^{nt}.
 * work: NP + 2*NG doubles. */
int orc_run_paper_order(const orc_params *p, double *xp, double *vp,
                        double *rho, double *phi, double *E, int64_t nt,
                        double *work)
{
    double *Ex = work, *fw = work + p->np;
    for (int64_t it = 0; it < nt; it++) {
        orc_drift(p, vp, xp);
        int rc = orc_prepare(p, xp, rho, phi, E, fw);
        if (rc) return rc;
        rc = orc_gather(p, xp, E, Ex);
        if (rc) return rc;
        orc_kick(p, Ex, vp);
    }
    return ORC_OK;
}

/* n steps of orc_step, recording per step n (0..nsteps-1) the history
 * row [sum v^{n-1/2} v^{n+1/2}, sum v^{n+1/2}, field energy of E^n,
 * amplitudes of modes 1..nmodes of E^n] (3 + nmodes doubles). */
double orc_field_energy(const orc_params *p, const double *E);
void orc_mode_amplitudes(const orc_params *p, const double *E, int nmodes,
                         double *amp);

int orc_run(const orc_params *p, double *xp, double *vp, double *rho,
            double *phi, double *E, int64_t nsteps, int nmodes, double *hist,
            double *work)
{
    const int row = 3 + nmodes;
    for (int64_t n = 0; n < nsteps; n++) {
        double fe = orc_field_energy(p, E);
        if (hist) {
            hist[n * row + 2] = fe;
            orc_mode_amplitudes(p, E, nmodes, hist + n * row + 3);
        }
        double sums[2];
        int rc = orc_step(p, xp, vp, rho, phi, E, work, sums);
        if (rc) return rc;
        if (hist) { hist[n * row + 0] = sums[0]; hist[n * row + 1] = sums[1]; }
    }
    return ORC_OK;
}

/* Field energy (1/2) sum_g E_g^2 dx (eps0 = 1). */
double orc_field_energy(const orc_params *p, const double *E)
{
    double s = 0.0;
    for (int ic = 0; ic < p->ng; ic++) s += E[ic] * E[ic];
    return 0.5 * s * orc_dx(p);
}

/* Amplitude of Fourier mode m of the grid field, m = 1..nmodes:
 * 2 |(1/NG) sum_g E_g exp(-2 pi i m g / NG)| (the amplitude A of a field
 * A cos(k_m x + phase)). */
void orc_mode_amplitudes(const orc_params *p, const double *E, int nmodes,
                         double *amp)
{
    const int ng = p->ng;
    const double two_pi = 6.283185307179586476925286766559;
    for (int m = 1; m <= nmodes; m++) {
        double re = 0.0, im = 0.0;
        for (int g = 0; g < ng; g++) {
            double th = two_pi * (double)((int64_t)m * g % ng) / (double)ng;
            re += E[g] * cos(th);
            im -= E[g] * sin(th);
        }
        amp[m - 1] = 2.0 * sqrt(re * re + im * im) / (double)ng;
    }
}

/* ---------------------------------------------------------------------
 * Fixed-point deposit, reading R5 (not in the paper; the build's exact form
 * of the Sec. 2.3 linear weighting, so that a density summed in any order is
 * the same integer).  The library keeps a float32 position as its cell
 * coordinate u = xp/dx in [0, NG) (node ic at u = ic + 1/2).  For each u:
 *   s = u - 0.5f;  fl = floorf(s);  f = s - fl
 *                                   (single float operations, round to nearest)
 *   i = (int)fl                     (left node, -1 .. NG-1)
 *   W = (uint32) trunc(f * 2^24)    (the right node's share, 0 .. 2^24)
 *   rho_q[(i+1) mod NG] += W;  rho_q[i mod NG] += 2^24 - W
 * Each particle adds exactly 2^24 to the total.  The FP64 density is
 *   rho_g = rho_init0 + (Q0/dx) rho_q[g] 2^-24.
 * --------------------------------------------------------------------- */
#define ORC_FIX_BITS 24

int orc_deposit_fixed(int32_t ng, int64_t np, const float *u, int64_t *rho_q)
{
    const float scale = 16777216.0f; /* 2^24 */
    for (int g = 0; g < ng; g++) rho_q[g] = 0;
    for (int64_t ip = 0; ip < np; ip++) {
        float s = u[ip] - 0.5f;
        float fl = floorf(s);
        float f = s - fl;
        if (!(fl >= -1.0f && fl <= (float)ng)) return ORC_ERANGE;
        int i = (int)fl;
        uint32_t W = (uint32_t)(f * scale);
        int il = ((i % ng) + ng) % ng;
        int ir = (il + 1 == ng) ? 0 : il + 1;
        rho_q[ir] += (int64_t)W;
        rho_q[il] += (int64_t)((1u << ORC_FIX_BITS) - W);
    }
    return ORC_OK;
}

/* The fixed-point form of the nearest-grid-point weighting (reading R13) on
 * cell coordinates: i = (int)floorf(u), cell NG (a coordinate at the box
 * end) is cell 0, rho_q[i] += 2^24. */
int orc_deposit_fixed_ngp(int32_t ng, int64_t np, const float *u, int64_t *rho_q)
{
    for (int g = 0; g < ng; g++) rho_q[g] = 0;
    for (int64_t ip = 0; ip < np; ip++) {
        float fl = floorf(u[ip]);
        if (!(fl >= 0.0f && fl <= (float)ng)) return ORC_ERANGE;
        int i = (int)fl;
        if (i == ng) i = 0;
        rho_q[i] += (int64_t)1 << ORC_FIX_BITS;
    }
    return ORC_OK;
}

/* FP64 density from the fixed-point sums (reading R5):
 * rho_g = rho_init0 + (Q0/dx) rho_q[g] 2^-24. */
void orc_rho_from_fixed(const orc_params *p, const int64_t *rho_q, double *rho)
{
    const double dx = orc_dx(p), Q0 = orc_q0(p);
    const double unit = ldexp(1.0, -ORC_FIX_BITS);
    for (int g = 0; g < p->ng; g++)
        rho[g] = p->rho_init0 + (Q0 / dx) * ((double)rho_q[g] * unit);
}

int orc_fix_bits(void) { return ORC_FIX_BITS; }

/* ---------------------------------------------------------------------
 * Initial loading (Sec. 2: positions and velocities sampled from the
 * problem's distribution; Appendix A set-up: particles on a uniform lattice;
 * Sec. 4: two beams at +-v0), reading R6, with the counter-based generator
 * SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014) written out from its published definition:
 * output k >= 1 of the generator seeded with `seed` is the mixing function
 * applied to seed + k * 0x9E3779B97F4A7C15 (mod 2^64).
 * --------------------------------------------------------------------- */
uint64_t orc_splitmix64(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + k * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Particle j of NP (float64 throughout; the library rounds to float32):
 *   x0 = (j + 1/2) Lx / NP                         the lattice
 *   x  = x0 - sum_m (eps_m / k_m) sin(k_m x0 + phase_m),  k_m = 2 pi m / Lx,
 *        folded once into [0, Lx)                  density perturbation
 *        sum_m eps_m cos(k_m x + phase_m) to first order
 *   v  = s_j v0 + vth sqrt(-2 ln u1) cos(2 pi u2)  Box-Muller
 * s_j = +1 for even j, -1 for odd j; u1 = (top 24 bits of z_{2j+1} + 1) 2^-24
 * in (0, 1], u2 = (top 24 bits of z_{2j+2}) 2^-24 in [0, 1), z_k =
 * orc_splitmix64(seed, k). */
int orc_load_two_stream(int64_t np, double lx, double v0, double vth,
                        uint64_t seed, int nmodes, const int32_t *mode,
                        const double *eps, const double *phase, double *x,
                        double *v)
{
    const double two_pi = 6.283185307179586476925286766559;
    if (np < 1 || !(lx > 0.0) || nmodes < 0) return ORC_EINVAL;
    for (int m = 0; m < nmodes; m++)
        if (mode[m] < 1) return ORC_EINVAL;
    for (int64_t j = 0; j < np; j++) {
        double x0 = ((double)j + 0.5) * (lx / (double)np);
        double xi = 0.0;
        for (int m = 0; m < nmodes; m++) {
            double k = two_pi * mode[m] / lx;
            xi += (eps[m] / k) * sin(k * x0 + phase[m]);
        }
        double xj = x0 - xi;
        if (xj < 0.0) xj += lx;
        else if (xj >= lx) xj -= lx;
        uint64_t z1 = orc_splitmix64(seed, 2 * (uint64_t)j + 1);
        uint64_t z2 = orc_splitmix64(seed, 2 * (uint64_t)j + 2);
        double u1 = ((double)(z1 >> 40) + 1.0) * ldexp(1.0, -24);
        double u2 = (double)(z2 >> 40) * ldexp(1.0, -24);
        double g = sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
        double s = (j % 2 == 0) ? 1.0 : -1.0;
        x[j] = xj;
        v[j] = s * v0 + vth * g;
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------------
 * Phase-space snapshot (Sec. 4, Fig. 1: the electrons in the (x, v) plane),
 * as counts of an nx by nv grid of bins over [0, Lx) x [vmin, vmax).  The
 * bin rule is the library's, stated in float32 so that the counts can be
 * compared exactly:  sx = (float)(nx / Lx), sv = (float)(nv / (vmax - vmin)),
 *   ix = min(nx - 1, trunc(x sx)),  iv = floor((v - (float)vmin) sv),
 * each product and difference one float operation; a particle with x sx not
 * >= 0 or iv outside [0, nv) is not counted.  counts[iv * nx + ix].
 * --------------------------------------------------------------------- */
int orc_phase_space(int32_t nx, int32_t nv, double lx, double vmin,
                    double vmax, int64_t np, const float *x, const float *v,
                    uint32_t *counts)
{
    if (nx < 1 || nv < 1 || !(lx > 0.0) || !(vmax > vmin)) return ORC_EINVAL;
    const float sx = (float)((double)nx / lx);
    const float sv = (float)((double)nv / (vmax - vmin));
    const float fvmin = (float)vmin;
    for (int64_t b = 0; b < (int64_t)nx * nv; b++) counts[b] = 0;
    for (int64_t ip = 0; ip < np; ip++) {
        float fx = x[ip] * sx;
        float dv = v[ip] - fvmin;
        float fv = floorf(dv * sv);
        if (!(fx >= 0.0f) || !(fv >= 0.0f) || !(fv < (float)nv)) continue;
        int ix = (int)fx;
        if (ix > nx - 1) ix = nx - 1;
        counts[(int64_t)fv * nx + ix] += 1;
    }
    return ORC_OK;
}
