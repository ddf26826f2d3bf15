/*
 * lbm_oracle.c -- plain, slow, FP64 CPU oracle of the lattice Boltzmann model
 * with fully resolved moving rigid particles (Sec. 4 of Bartuschat et al.).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * bench's CPU-baseline leg; never by the product path.  Shares no code with
 * the GPU library.
 *
 * One time step, in the paper's order:
 *   1. collide every fluid cell with the TRT operator (Eqs. TRTOp, EqPDF_TRT,
 *      LBMCollide) using the incompressible equilibrium (Eq. fequ_Incompr);
 *   2. stream (Eq. LBMStream) with a second array (push); links that end in a
 *      wall or particle cell are bounced back with the surface velocity
 *      (Eqs. BBBC, LBMMovWall) and their momentum is summed into the particle
 *      force and torque (Eqs. TransferredMomentum, LBMhydrodynForce);
 *   3. advance each rigid body with that force and torque (Sec. 4.3);
 *   4. re-map the obstacle cells from the new poses (Sec. 4.2: a cell belongs to
 *      a particle iff its centre lies inside it) and refill uncovered cells
 *      with the equilibrium at rho0 and the surface velocity of the previous
 *      time step.
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes): the weight in Eqs. LBMMovWall/LBMhydrodynForce is the lattice
 * weight w_q, so the factor 2 w_q / c_s^2 is 6 w_q; the torque of a link is
 * (x_s - x_C) x dF with x_s the obstacle-cell centre; the surface velocity
 * uses the particle state before this step's rigid-body update; covered cells
 * drop their populations; the rigid-body integrator (not described in the
 * paper) is semi-implicit Euler on U and on the world-frame angular momentum
 * with a quaternion exponential update; a body force g enters as the odd
 * source 3 w_q rho0 c_q.g after collision and the reported velocity is
 * sum(c f)/rho0 + g/2.
 *
 * Built with -ffp-contract=off so that every product and sum rounds
 * separately; the inside test is defined with that rounding.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19

/* D3Q19 velocity set and weights (Eq. SpeedOfSound and the weights under it:
   1/3 rest, 1/18 axis, 1/36 diagonal). */
static const int CX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static const int OPP[Q] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
static const double W[Q] = {1.0 / 3.0,
                            1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;

enum { FL_FLUID = 0, FL_WALL = 1, FL_PARTICLE = 2 };

typedef struct {
    double rec[ORC_PSTRIDE]; /* current state, record layout of lbm_oracle.h */
    double L[3];             /* world-frame angular momentum */
    double old[ORC_PSTRIDE]; /* state before this step's update */
    double F[3], M[3];       /* hydrodynamic force/torque of the last step */
} orc_particle;

struct orc_sim {
    int nx, ny, nz;
    long n;
    double tau, magic, rho0, omega, omega_odd;
    int periodic[3];
    double wall_lo[3], wall_hi[3], g[3];
    double *f, *fnew;
    uint8_t *flag;
    uint32_t *pid;
    int np;
    orc_particle *p;
    double Fwall[2][3];
    long t;
    int stab;         /* momentum stabilisation on (Sec. 4.1) */
    double ubar[3];   /* mean fluid velocity of the current step */
    int free_slip[3]; /* wall layers of a non-periodic axis reflect (Eq. FreeSlipBC) */
};

static int g_threads = 1;

void orc_set_threads(int nthreads) { g_threads = nthreads > 0 ? nthreads : 1; }

void orc_lattice(int *cx, int *cy, int *cz, double *w, int *opp) {
    for (int q = 0; q < Q; ++q) {
        cx[q] = CX[q];
        cy[q] = CY[q];
        cz[q] = CZ[q];
        w[q] = W[q];
        opp[q] = OPP[q];
    }
}

/* Odd relaxation rate from the TRT "magic" product
   Lambda = (1/omega - 1/2)(1/omega_odd - 1/2)  (Sec. 4.1; Lambda = 3/16 puts
   bounce-back walls half-way between cells). */
double orc_omega_odd(double tau, double magic) {
    double tau_odd = magic / (tau - 0.5) + 0.5;
    return 1.0 / tau_odd;
}

/* Incompressible equilibrium of He and Luo (Eq. fequ_Incompr). */
void orc_equilibrium(double rho, const double u[3], double rho0, double *feq) {
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int q = 0; q < Q; ++q) {
        double cu = CX[q] * u[0] + CY[q] * u[1] + CZ[q] * u[2];
        feq[q] = W[q] * (rho + rho0 * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2)));
    }
}

/* Moments of one cell (the density and velocity of Sec. 4.1; u uses rho0). */
static void moments(const double *f, double rho0, double *rho, double u[3]) {
    double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    for (int q = 0; q < Q; ++q) {
        r += f[q];
        jx += CX[q] * f[q];
        jy += CY[q] * f[q];
        jz += CZ[q] * f[q];
    }
    *rho = r;
    u[0] = jx / rho0;
    u[1] = jy / rho0;
    u[2] = jz / rho0;
}

/* TRT collision of one cell (Eqs. TRTOp, EqPDF_TRT, LBMCollide):
   f~_q = f_q + lambda_e (f^e_q - f^eq,e_q) + lambda_o (f^o_q - f^eq,o_q),
   lambda_e = -omega, lambda_o = -omega_odd; plus the body-force source
   3 w_q rho0 c_q.g.  The equilibrium is taken at the velocity u - ubar:
   ubar is the domain-mean velocity under momentum stabilisation (Sec. 4.1),
   zero otherwise. */
void orc_collide_cell(const double *f, double omega, double omega_odd, double rho0,
                      const double g[3], const double ubar[3], double *ft) {
    double rho, u[3];
    moments(f, rho0, &rho, u);
    for (int a = 0; a < 3; ++a) u[a] -= ubar[a];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int q = 0; q < Q; ++q) {
        int qb = OPP[q];
        double cu = CX[q] * u[0] + CY[q] * u[1] + CZ[q] * u[2];
        double fe = 0.5 * (f[q] + f[qb]);
        double fo = 0.5 * (f[q] - f[qb]);
        double feq_e = W[q] * (rho - rho0 * uu / (2.0 * CS2) + rho0 * cu * cu / (2.0 * CS2 * CS2));
        double feq_o = W[q] * rho0 * cu / CS2;
        double src = W[q] * rho0 * (CX[q] * g[0] + CY[q] * g[1] + CZ[q] * g[2]) / CS2;
        ft[q] = f[q] - omega * (fe - feq_e) - omega_odd * (fo - feq_o) + src;
    }
}

/* Rotation matrix (row-major) of the unit quaternion (w,x,y,z); every product
   and sum rounds separately, in the order written. */
void orc_quat_to_matrix(const double q[4], double R[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.0 - 2.0 * (y * y + z * z);
    R[1] = 2.0 * (x * y - w * z);
    R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);
    R[4] = 1.0 - 2.0 * (x * x + z * z);
    R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);
    R[7] = 2.0 * (y * z + w * x);
    R[8] = 1.0 - 2.0 * (x * x + y * y);
}

/* Displacement from a particle centre to a cell centre along one axis, taken
   to the nearest periodic image. */
static double min_image(double d, int n, int periodic) {
    if (periodic) {
        if (d > 0.5 * n)
            d -= n;
        else if (d < -0.5 * n)
            d += n;
    }
    return d;
}

/* Obstacle mapping of Sec. 4.2: cell (i,j,k) is covered iff its centre lies
   inside the body, with p = R^T d the centre in the body frame:
   ellipsoid: (p0/a)^2 + (p1/b)^2 + (p2/c)^2 <= 1;
   spherocylinder of radius r and half length L/2 = a along body x: the
   distance from p to the axis segment |p0| <= a - r is at most r, i.e.
   t^2 + p1^2 + p2^2 <= r^2 with t = max(|p0| - (a - r), 0). */
int orc_inside(const double *rec, int nx, int ny, int nz, const int periodic[3], int i, int j,
               int k) {
    double d0 = min_image((double)i - rec[0], nx, periodic[0]);
    double d1 = min_image((double)j - rec[1], ny, periodic[1]);
    double d2 = min_image((double)k - rec[2], nz, periodic[2]);
    double R[9];
    orc_quat_to_matrix(rec + 3, R);
    double p0 = R[0] * d0 + R[3] * d1 + R[6] * d2;
    double p1 = R[1] * d0 + R[4] * d1 + R[7] * d2;
    double p2 = R[2] * d0 + R[5] * d1 + R[8] * d2;
    if (rec[25] == ORC_SHAPE_SPHEROCYLINDER) {
        double r = rec[14];
        double t = fabs(p0) - (rec[13] - r);
        if (t < 0.0) t = 0.0;
        double s = t * t + p1 * p1 + p2 * p2;
        return s <= r * r;
    }
    double t0 = p0 / rec[13], t1 = p1 / rec[14], t2 = p2 / rec[15];
    double s = t0 * t0 + t1 * t1 + t2 * t2;
    return s <= 1.0;
}

/* Mass and principal moments of inertia of a homogeneous body of density
   rec[16].  Spherocylinder: a cylinder of length 2h = L - 2r (mass m_c) and
   two hemispherical caps forming a sphere of radius r (mass m_s).  About the
   axis: m_c r^2/2 + 2 m_s r^2/5.  About a transverse axis through the
   centre: the cylinder's m_c (r^2/4 + (2h)^2/12), and for each cap (mass
   m_s/2, centroid 3r/8 from its flat face, which lies h from the centre) its
   moment about the face, m_s r^2/5, moved to the centroid and then to the
   centre by the parallel-axis theorem: in total m_s (2r^2/5 + h^2 + 3hr/4). */
void orc_particle_mass_inertia(const double *rec, double *mass, double inertia[3]) {
    if (rec[25] == ORC_SHAPE_SPHEROCYLINDER) {
        double r = rec[14], h = rec[13] - rec[14];
        double mc = rec[16] * M_PI * r * r * (2.0 * h);
        double ms = rec[16] * (4.0 / 3.0) * M_PI * r * r * r;
        *mass = mc + ms;
        inertia[0] = mc * r * r / 2.0 + 2.0 * ms * r * r / 5.0;
        inertia[1] = mc * (r * r / 4.0 + (2.0 * h) * (2.0 * h) / 12.0) +
                     ms * (2.0 * r * r / 5.0 + h * h + 3.0 * h * r / 4.0);
        inertia[2] = inertia[1];
        return;
    }
    double a = rec[13], b = rec[14], c = rec[15];
    double m = rec[16] * (4.0 / 3.0) * M_PI * a * b * c;
    *mass = m;
    inertia[0] = m * (b * b + c * c) / 5.0;
    inertia[1] = m * (a * a + c * c) / 5.0;
    inertia[2] = m * (a * a + b * b) / 5.0;
}

/* Surface velocity of a rigid body at a cell centre: U + Omega x (x - x_C). */
static void surface_velocity(const double *rec, const orc_sim *s, int i, int j, int k,
                             double us[3]) {
    double d0 = min_image((double)i - rec[0], s->nx, s->periodic[0]);
    double d1 = min_image((double)j - rec[1], s->ny, s->periodic[1]);
    double d2 = min_image((double)k - rec[2], s->nz, s->periodic[2]);
    const double *U = rec + 7, *Om = rec + 10;
    us[0] = U[0] + (Om[1] * d2 - Om[2] * d1);
    us[1] = U[1] + (Om[2] * d0 - Om[0] * d2);
    us[2] = U[2] + (Om[0] * d1 - Om[1] * d0);
}

static void normalise_quat(double q[4]) {
    double nrm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) q[i] /= nrm;
}

/* omega = R diag(1/I) R^T L */
static void omega_from_L(const double q[4], const double I[3], const double L[3], double Om[3]) {
    double R[9];
    orc_quat_to_matrix(q, R);
    double lb[3];
    for (int a = 0; a < 3; ++a) lb[a] = (R[0 + a] * L[0] + R[3 + a] * L[1] + R[6 + a] * L[2]) / I[a];
    for (int a = 0; a < 3; ++a) Om[a] = R[3 * a + 0] * lb[0] + R[3 * a + 1] * lb[1] + R[3 * a + 2] * lb[2];
}

static void L_from_omega(const double q[4], const double I[3], const double Om[3], double L[3]) {
    double R[9];
    orc_quat_to_matrix(q, R);
    double ob[3];
    for (int a = 0; a < 3; ++a) ob[a] = (R[0 + a] * Om[0] + R[3 + a] * Om[1] + R[6 + a] * Om[2]) * I[a];
    for (int a = 0; a < 3; ++a) L[a] = R[3 * a + 0] * ob[0] + R[3 * a + 1] * ob[1] + R[3 * a + 2] * ob[2];
}

/* Rigid-body step with dt = 1 (the paper delegates this to its physics engine
   and does not state the integrator):
     U <- U + F/m ;  x <- x + U ;  L <- L + M ;
     Omega <- R(q) I^-1 R(q)^T L ;  q <- normalise(exp(Omega/2) * q). */
void orc_rigid_body_step(double *rec, double *L, const double F[3], const double M[3]) {
    double m, I[3];
    orc_particle_mass_inertia(rec, &m, I);
    for (int a = 0; a < 3; ++a) rec[7 + a] += F[a] / m;
    for (int a = 0; a < 3; ++a) rec[a] += rec[7 + a];
    for (int a = 0; a < 3; ++a) L[a] += M[a];
    double Om[3];
    omega_from_L(rec + 3, I, L, Om);
    for (int a = 0; a < 3; ++a) rec[10 + a] = Om[a];
    double th = sqrt(Om[0] * Om[0] + Om[1] * Om[1] + Om[2] * Om[2]);
    double dq[4] = {1.0, 0.0, 0.0, 0.0};
    if (th > 0.0) {
        double sh = sin(0.5 * th) / th;
        dq[0] = cos(0.5 * th);
        dq[1] = Om[0] * sh;
        dq[2] = Om[1] * sh;
        dq[3] = Om[2] * sh;
    }
    double *q = rec + 3;
    double nq[4];
    nq[0] = dq[0] * q[0] - (dq[1] * q[1] + dq[2] * q[2] + dq[3] * q[3]);
    nq[1] = dq[0] * q[1] + q[0] * dq[1] + (dq[2] * q[3] - dq[3] * q[2]);
    nq[2] = dq[0] * q[2] + q[0] * dq[2] + (dq[3] * q[1] - dq[1] * q[3]);
    nq[3] = dq[0] * q[3] + q[0] * dq[3] + (dq[1] * q[2] - dq[2] * q[1]);
    normalise_quat(nq);
    for (int a = 0; a < 4; ++a) q[a] = nq[a];
}

static long cell_index(const orc_sim *s, int i, int j, int k) {
    return (long)i + (long)s->nx * ((long)j + (long)s->ny * (long)k);
}

static int wrap(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

orc_sim *orc_create(int nx, int ny, int nz, double tau, double magic, double rho0,
                    const int periodic[3], const double wall_lo[3], const double wall_hi[3],
                    const double body_force[3]) {
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->nx = nx;
    s->ny = ny;
    s->nz = nz;
    s->n = (long)nx * ny * nz;
    s->tau = tau;
    s->magic = magic;
    s->rho0 = rho0;
    s->omega = 1.0 / tau;
    s->omega_odd = orc_omega_odd(tau, magic);
    for (int a = 0; a < 3; ++a) {
        s->periodic[a] = periodic[a];
        s->wall_lo[a] = wall_lo[a];
        s->wall_hi[a] = wall_hi[a];
        s->g[a] = body_force ? body_force[a] : 0.0;
    }
    s->f = (double *)calloc((size_t)Q * s->n, sizeof(double));
    s->fnew = (double *)calloc((size_t)Q * s->n, sizeof(double));
    s->flag = (uint8_t *)calloc((size_t)s->n, 1);
    s->pid = (uint32_t *)malloc((size_t)s->n * sizeof(uint32_t));
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long x = cell_index(s, i, j, k);
                uint32_t id = ORC_PID_FLUID;
                if (!periodic[1] && j == 0)
                    id = ORC_PID_WALL_YLO;
                else if (!periodic[1] && j == ny - 1)
                    id = ORC_PID_WALL_YHI;
                else if ((!periodic[0] && (i == 0 || i == nx - 1)) ||
                         (!periodic[2] && (k == 0 || k == nz - 1)))
                    id = ORC_PID_WALL;
                s->pid[x] = id;
                s->flag[x] = id == ORC_PID_FLUID ? FL_FLUID : FL_WALL;
                /* fluid at rest with density rho0 */
                for (int q = 0; q < Q; ++q) s->f[q * s->n + x] = (id == ORC_PID_FLUID) ? W[q] * rho0 : 0.0;
            }
    return s;
}

void orc_destroy(orc_sim *s) {
    if (!s) return;
    free(s->f);
    free(s->fnew);
    free(s->flag);
    free(s->pid);
    free(s->p);
    free(s);
}

long orc_step_count(const orc_sim *s) { return s->t; }

/* Re-map every non-wall cell from the current poses.  A cell inside several
   bodies belongs to the lowest index.  Cells that stop being obstacle cells get
   the equilibrium at rho0 and the surface velocity of their previous owner;
   `use_old` selects that owner's pre-update state (time stepping) and
   otherwise the refill is at rest (a fresh particle set). */
static void remap(orc_sim *s, int use_old) {
    double feq[Q];
    for (int k = 0; k < s->nz; ++k)
        for (int j = 0; j < s->ny; ++j)
            for (int i = 0; i < s->nx; ++i) {
                long x = cell_index(s, i, j, k);
                if (s->flag[x] == FL_WALL) continue;
                uint32_t old = s->pid[x];
                uint32_t nw = ORC_PID_FLUID;
                for (int p = 0; p < s->np; ++p)
                    if (orc_inside(s->p[p].rec, s->nx, s->ny, s->nz, s->periodic, i, j, k)) {
                        nw = (uint32_t)p;
                        break;
                    }
                if (old != ORC_PID_FLUID && nw == ORC_PID_FLUID) {
                    double us[3] = {0.0, 0.0, 0.0};
                    if (use_old && old < (uint32_t)s->np) surface_velocity(s->p[old].old, s, i, j, k, us);
                    orc_equilibrium(s->rho0, us, s->rho0, feq);
                    for (int q = 0; q < Q; ++q) s->f[q * s->n + x] = feq[q];
                }
                if (old == ORC_PID_FLUID && nw != ORC_PID_FLUID)
                    for (int q = 0; q < Q; ++q) s->f[q * s->n + x] = 0.0;
                s->pid[x] = nw;
                s->flag[x] = nw == ORC_PID_FLUID ? FL_FLUID : FL_PARTICLE;
            }
}

int orc_set_particles(orc_sim *s, const double *state, int n) {
    free(s->p);
    s->p = n > 0 ? (orc_particle *)calloc((size_t)n, sizeof(orc_particle)) : NULL;
    s->np = n;
    for (int p = 0; p < n; ++p) {
        memcpy(s->p[p].rec, state + (size_t)p * ORC_PSTRIDE, ORC_PSTRIDE * sizeof(double));
        normalise_quat(s->p[p].rec + 3);
        double m, I[3];
        orc_particle_mass_inertia(s->p[p].rec, &m, I);
        L_from_omega(s->p[p].rec + 3, I, s->p[p].rec + 10, s->p[p].L);
        memcpy(s->p[p].old, s->p[p].rec, sizeof(s->p[p].rec));
    }
    remap(s, 0);
    return 0;
}

/* Velocity of the obstacle cell xn = (i,j,k) as seen by a bounce-back link. */
static void obstacle_velocity(const orc_sim *s, uint32_t id, int i, int j, int k, double us[3]) {
    if (id == ORC_PID_WALL_YLO) {
        us[0] = s->wall_lo[0];
        us[1] = s->wall_lo[1];
        us[2] = s->wall_lo[2];
    } else if (id == ORC_PID_WALL_YHI) {
        us[0] = s->wall_hi[0];
        us[1] = s->wall_hi[1];
        us[2] = s->wall_hi[2];
    } else if (id == ORC_PID_WALL) {
        us[0] = us[1] = us[2] = 0.0;
    } else {
        surface_velocity(s->p[id].rec, s, i, j, k, us);
    }
}

/* Index of the lattice direction (cx, cy, cz), -1 if none. */
static int direction(int cx, int cy, int cz) {
    for (int q = 0; q < Q; ++q)
        if (CX[q] == cx && CY[q] == cy && CZ[q] == cz) return q;
    return -1;
}

/* Free-slip wall (Eq. FreeSlipBC): the population f~_q leaving fluid cell
   x_F = (i,j,k) into a wall cell is reflected at the wall, n the wall normal:
   it arrives at x_F + c_q - n (n.c_q) with direction c_q - 2 n (n.c_q).  At an
   edge or corner every wall layer the link crosses reflects its component.
   Applies when every layer the link crosses belongs to a free-slip axis and
   the arrival cell is fluid; returns 0 otherwise (the link bounces back).
   No momentum is booked to the wall. */
static int free_slip_link(orc_sim *s, int i, int j, int k, int q, double val) {
    const int dims[3] = {s->nx, s->ny, s->nz}, at[3] = {i, j, k};
    const int c[3] = {CX[q], CY[q], CZ[q]};
    int d[3], r[3], crossed = 0;
    for (int a = 0; a < 3; ++a) {
        const int to = at[a] + c[a];
        const int layer = !s->periodic[a] && c[a] != 0 && (to == 0 || to == dims[a] - 1);
        if (layer && !s->free_slip[a]) return 0;
        crossed |= layer;
        d[a] = layer ? at[a] : wrap(to, dims[a]);
        r[a] = layer ? -c[a] : c[a];
    }
    if (!crossed) return 0;
    const long xd = cell_index(s, d[0], d[1], d[2]);
    if (s->flag[xd] != FL_FLUID) return 0;
    s->fnew[direction(r[0], r[1], r[2]) * s->n + xd] = val;
    return 1;
}

void orc_set_free_slip(orc_sim *s, const int free_slip[3]) {
    for (int a = 0; a < 3; ++a) s->free_slip[a] = free_slip[a] != 0 && !s->periodic[a];
}

/* Momentum stabilisation (Sec. 4.1): the mean velocity sum(c f)/rho0 over
   the fluid cells of the whole domain, taken before the collision of this
   step and subtracted from every cell's velocity in its equilibrium. */
static void mean_fluid_velocity(orc_sim *s) {
    double j[3] = {0.0, 0.0, 0.0}, cnt = 0.0;
    for (long x = 0; x < s->n; ++x) {
        if (s->flag[x] != FL_FLUID) continue;
        double f[Q], rho, u[3];
        for (int q = 0; q < Q; ++q) f[q] = s->f[q * s->n + x];
        moments(f, s->rho0, &rho, u);
        for (int a = 0; a < 3; ++a) j[a] += u[a];
        cnt += 1.0;
    }
    for (int a = 0; a < 3; ++a) s->ubar[a] = cnt > 0.0 ? j[a] / cnt : 0.0;
}

void orc_set_momentum_stabilisation(orc_sim *s, int enable) {
    s->stab = enable != 0;
    for (int a = 0; a < 3; ++a) s->ubar[a] = 0.0;
}

static void collide_and_stream(orc_sim *s) {
    const long n = s->n;
    if (s->stab) mean_fluid_velocity(s);
    for (int p = 0; p < s->np; ++p)
        for (int a = 0; a < 3; ++a) s->p[p].F[a] = s->p[p].M[a] = 0.0;
    for (int w = 0; w < 2; ++w)
        for (int a = 0; a < 3; ++a) s->Fwall[w][a] = 0.0;

    int nthr = g_threads;
    int np = s->np;
    /* per-thread accumulators: [thread][particle][F0..2, M0..2], then walls */
    double *acc = (double *)calloc((size_t)nthr * (size_t)(np * 6 + 6), sizeof(double));
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthr) schedule(static)
#endif
    for (int k = 0; k < s->nz; ++k) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *my = acc + (size_t)tid * (size_t)(np * 6 + 6);
        double f[Q], ft[Q];
        for (int j = 0; j < s->ny; ++j)
            for (int i = 0; i < s->nx; ++i) {
                long x = cell_index(s, i, j, k);
                if (s->flag[x] != FL_FLUID) continue;
                for (int q = 0; q < Q; ++q) f[q] = s->f[q * n + x];
                orc_collide_cell(f, s->omega, s->omega_odd, s->rho0, s->g, s->ubar, ft);
                for (int q = 0; q < Q; ++q) {
                    int ii = wrap(i + CX[q], s->nx), jj = wrap(j + CY[q], s->ny),
                        kk = wrap(k + CZ[q], s->nz);
                    long xn = cell_index(s, ii, jj, kk);
                    if (s->flag[xn] == FL_FLUID) {
                        s->fnew[q * n + xn] = ft[q];
                        continue;
                    }
                    if (s->flag[xn] == FL_WALL && free_slip_link(s, i, j, k, q, ft[q])) continue;
                    /* velocity bounce-back (Eq. LBMMovWall) */
                    uint32_t id = s->pid[xn];
                    double us[3];
                    obstacle_velocity(s, id, ii, jj, kk, us);
                    double cu = CX[q] * us[0] + CY[q] * us[1] + CZ[q] * us[2];
                    double val = ft[q] - 2.0 * W[q] / CS2 * s->rho0 * cu;
                    s->fnew[OPP[q] * n + x] = val;
                    /* momentum handed to the obstacle along this link
                       (Eqs. TransferredMomentum, LBMhydrodynForce) */
                    double mag = ft[q] + val;
                    double dF[3] = {mag * CX[q], mag * CY[q], mag * CZ[q]};
                    if (id < (uint32_t)np) {
                        const double *rec = s->p[id].rec;
                        double r0 = min_image((double)ii - rec[0], s->nx, s->periodic[0]);
                        double r1 = min_image((double)jj - rec[1], s->ny, s->periodic[1]);
                        double r2 = min_image((double)kk - rec[2], s->nz, s->periodic[2]);
                        double *a = my + (size_t)id * 6;
                        a[0] += dF[0];
                        a[1] += dF[1];
                        a[2] += dF[2];
                        a[3] += r1 * dF[2] - r2 * dF[1];
                        a[4] += r2 * dF[0] - r0 * dF[2];
                        a[5] += r0 * dF[1] - r1 * dF[0];
                    } else if (id == ORC_PID_WALL_YLO || id == ORC_PID_WALL_YHI) {
                        double *a = my + (size_t)np * 6 + (id == ORC_PID_WALL_YLO ? 0 : 3);
                        a[0] += dF[0];
                        a[1] += dF[1];
                        a[2] += dF[2];
                    }
                }
            }
    }
    for (int t = 0; t < nthr; ++t) {
        const double *my = acc + (size_t)t * (size_t)(np * 6 + 6);
        for (int p = 0; p < np; ++p)
            for (int a = 0; a < 3; ++a) {
                s->p[p].F[a] += my[p * 6 + a];
                s->p[p].M[a] += my[p * 6 + 3 + a];
            }
        for (int a = 0; a < 3; ++a) {
            s->Fwall[0][a] += my[np * 6 + a];
            s->Fwall[1][a] += my[np * 6 + 3 + a];
        }
    }
    free(acc);
    double *tmp = s->f;
    s->f = s->fnew;
    s->fnew = tmp;
    /* non-fluid cells carry no populations */
    for (long x = 0; x < n; ++x)
        if (s->flag[x] != FL_FLUID)
            for (int q = 0; q < Q; ++q) s->f[q * n + x] = 0.0;
}

void orc_step(orc_sim *s, int nsteps) {
    for (int it = 0; it < nsteps; ++it) {
        collide_and_stream(s);
        for (int p = 0; p < s->np; ++p) {
            orc_particle *P = &s->p[p];
            memcpy(P->old, P->rec, sizeof(P->rec));
            if (P->rec[23] != 0.0) continue; /* fixed body */
            double F[3], M[3];
            for (int a = 0; a < 3; ++a) {
                F[a] = P->F[a] + P->rec[17 + a];
                M[a] = P->M[a] + P->rec[20 + a];
            }
            orc_rigid_body_step(P->rec, P->L, F, M);
            for (int a = 0; a < 3; ++a) {
                int n = a == 0 ? s->nx : (a == 1 ? s->ny : s->nz);
                if (s->periodic[a]) {
                    if (P->rec[a] >= n)
                        P->rec[a] -= n;
                    else if (P->rec[a] < 0.0)
                        P->rec[a] += n;
                }
            }
        }
        if (s->np > 0) remap(s, 1);
        s->t++;
    }
}

void orc_get_fields(const orc_sim *s, double *rho, double *u3, uint8_t *flags, uint32_t *pid,
                    double *pdfs) {
    const long n = s->n;
    for (long x = 0; x < n; ++x) {
        double f[Q], r = 0.0, u[3] = {0.0, 0.0, 0.0};
        int fluid = s->flag[x] == FL_FLUID;
        if (fluid) {
            for (int q = 0; q < Q; ++q) f[q] = s->f[q * n + x];
            moments(f, s->rho0, &r, u);
            for (int a = 0; a < 3; ++a) u[a] += 0.5 * s->g[a];
        }
        if (rho) rho[x] = r;
        if (u3)
            for (int a = 0; a < 3; ++a) u3[a * n + x] = u[a];
        if (flags) flags[x] = s->flag[x];
        if (pid) pid[x] = s->pid[x];
        if (pdfs)
            for (int q = 0; q < Q; ++q) pdfs[q * n + x] = fluid ? s->f[q * n + x] : 0.0;
    }
}

void orc_set_pdfs(orc_sim *s, const double *pdfs) {
    for (long x = 0; x < s->n; ++x)
        if (s->flag[x] == FL_FLUID)
            for (int q = 0; q < Q; ++q) s->f[q * s->n + x] = pdfs[q * s->n + x];
}

void orc_get_forces(const orc_sim *s, double *F, double *M) {
    for (int p = 0; p < s->np; ++p)
        for (int a = 0; a < 3; ++a) {
            if (F) F[3 * p + a] = s->p[p].F[a];
            if (M) M[3 * p + a] = s->p[p].M[a];
        }
}

void orc_get_wall_forces(const orc_sim *s, double *f6) {
    for (int a = 0; a < 3; ++a) {
        f6[a] = s->Fwall[0][a];
        f6[3 + a] = s->Fwall[1][a];
    }
}

void orc_get_particles(const orc_sim *s, double *state) {
    for (int p = 0; p < s->np; ++p)
        memcpy(state + (size_t)p * ORC_PSTRIDE, s->p[p].rec, ORC_PSTRIDE * sizeof(double));
}

/* Boundary links {(x_F, q): x_F fluid, x_F + c_q an obstacle}, ordered by cell
   index then direction (the sets D_s of Eq. LBMhydrodynForce, walls included). */
int orc_get_links(const orc_sim *s, int32_t *cell, int8_t *qq, uint32_t *pid, int cap) {
    int cnt = 0;
    for (int k = 0; k < s->nz; ++k)
        for (int j = 0; j < s->ny; ++j)
            for (int i = 0; i < s->nx; ++i) {
                long x = cell_index(s, i, j, k);
                if (s->flag[x] != FL_FLUID) continue;
                for (int q = 1; q < Q; ++q) {
                    long xn = cell_index(s, wrap(i + CX[q], s->nx), wrap(j + CY[q], s->ny),
                                         wrap(k + CZ[q], s->nz));
                    if (s->flag[xn] == FL_FLUID) continue;
                    if (cnt < cap) {
                        if (cell) cell[cnt] = (int32_t)x;
                        if (qq) qq[cnt] = (int8_t)q;
                        if (pid) pid[cnt] = s->pid[xn];
                    }
                    ++cnt;
                }
            }
    return cnt;
}
