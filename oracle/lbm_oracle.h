/*
 * lbm_oracle.h -- plain FP64 CPU oracle of the fully resolved particle model
 * (lattice Boltzmann method with moving-obstacle bounce-back, Sec. 4 of
 * Bartuschat et al., "Two computational models for simulating the tumbling
 * motion of elongated particles in fluids").
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the GPU library; only
 * the tests, the smoke check and the bench's CPU-baseline leg load it.  It
 * shares no code, header, table or helper with the GPU path.
 *
 * Conventions (lattice units, dx = dt = 1): cell (i,j,k) has centre (i,j,k)
 * and linear index i + nx*(j + ny*k).  Populations are canonical post-stream
 * values f[q*n + idx].  D3Q19 numbering: 0 rest; 1..6 = +x,-x,+y,-y,+z,-z;
 * 7..18 = (1,1,0),(-1,-1,0),(1,-1,0),(-1,1,0),(1,0,1),(-1,0,-1),(1,0,-1),
 * (-1,0,1),(0,1,1),(0,-1,-1),(0,1,-1),(0,-1,1).  Opposite of q (q>0) is the
 * other member of its adjacent pair.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* doubles per particle record: pos3 quat4(w,x,y,z) vel3 omega3 semi3 density
   extF3 extM3 fixed(0/1) cell(ignored by the oracle) shape.
   shape 0: ellipsoid with semi-axes (a, b, c) along body x, y, z;
   shape 1: spherocylinder (Sec. 5.1, Fig. Capsule) of total length L and
   radius r along body x, given as semi = (L/2, r, r). */
#define ORC_PSTRIDE 26
#define ORC_SHAPE_ELLIPSOID 0
#define ORC_SHAPE_SPHEROCYLINDER 1

#define ORC_PID_FLUID    0xFFFFFFFFu
#define ORC_PID_WALL_YLO 0xFFFFFFFEu
#define ORC_PID_WALL_YHI 0xFFFFFFFDu
#define ORC_PID_WALL     0xFFFFFFFCu

typedef struct orc_sim orc_sim;

orc_sim *orc_create(int nx, int ny, int nz, double tau, double magic, double rho0,
                    const int periodic[3], const double wall_lo[3],
                    const double wall_hi[3], const double body_force[3]);
void orc_destroy(orc_sim *s);
int orc_set_particles(orc_sim *s, const double *state, int n);
void orc_step(orc_sim *s, int nsteps);
long orc_step_count(const orc_sim *s);
void orc_get_fields(const orc_sim *s, double *rho, double *u3, uint8_t *flags,
                    uint32_t *pid, double *pdfs);
void orc_set_pdfs(orc_sim *s, const double *pdfs);
void orc_get_forces(const orc_sim *s, double *force3n, double *torque3n);
void orc_get_wall_forces(const orc_sim *s, double *f6);
void orc_get_particles(const orc_sim *s, double *state);
int orc_get_links(const orc_sim *s, int32_t *cell, int8_t *q, uint32_t *pid, int cap);
void orc_set_threads(int nthreads);
/* Momentum stabilisation (Sec. 4.1): each step's equilibria use u - ubar,
   ubar the mean velocity of all fluid cells before that step's collision. */
void orc_set_momentum_stabilisation(orc_sim *s, int enable);
/* Free-slip walls (Eq. FreeSlipBC) on the wall layers of each non-periodic
   axis a with free_slip[a] != 0 (the moving-wall velocities of y are then
   unused). */
void orc_set_free_slip(orc_sim *s, const int free_slip[3]);

/* building blocks, exposed for the pin tests */
void orc_lattice(int *cx, int *cy, int *cz, double *w, int *opp);
double orc_omega_odd(double tau, double magic);
void orc_equilibrium(double rho, const double u[3], double rho0, double *feq);
void orc_collide_cell(const double *f, double omega, double omega_odd, double rho0,
                      const double g[3], const double ubar[3], double *ft);
int orc_inside(const double *particle, int nx, int ny, int nz, const int periodic[3],
               int i, int j, int k);
void orc_quat_to_matrix(const double q[4], double R[9]);
void orc_rigid_body_step(double *particle, double *L, const double F[3], const double M[3]);
void orc_particle_mass_inertia(const double *particle, double *mass, double inertia[3]);

#ifdef __cplusplus
}
#endif
#endif
