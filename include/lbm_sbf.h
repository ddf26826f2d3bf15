/*
 * lbm_sbf.h -- slender-body formulation (Sec. 3 of Bartuschat et al.) of rigid
 * straight fibres in unbounded Stokes flow, on the GPU in FP64.
 *
 * Fibre m has centre x_m, unit tangent p_m, half length l_m and radius r_m.
 * Given external forces F_m and torques M_m, lbm_sbf_solve returns the
 * translational velocity xdot_m and the rate of change of the tangent pdot_m
 * of Eqs. xadot and padot: the line force of each fibre is expanded in
 * Legendre polynomials of degree 1..n_modes (Eq. force_exp), the non-local
 * slender body equation (Eq. sev_fils, with the operator of Eq. Kbar and the
 * fibre-fibre interaction of Eqs. Ucontr_def and Gnonper) is projected on
 * them, and the dense system for the coefficients is solved; the interaction
 * integrals use n_quad-point Gauss-Legendre quadrature along each fibre.
 * Units are the caller's (SI in the paper); mu is the dynamic viscosity.
 *
 * Sizes: 1 <= nfibres <= 64, 2 <= n_modes <= 10, 2 <= n_quad <= 64.  The
 * context holds O(nfibres^2 n_modes^2) device memory.  All host arrays are
 * owned by the caller and read or written during the call only.
 */
#ifndef LBM_SBF_H
#define LBM_SBF_H
#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_sbf lbm_sbf;

/* Create a context for nfibres fibres on the given CUDA stream (NULL: the
 * legacy default stream).  Errors: LBM_ERR_ARG for sizes out of range or
 * mu <= 0; LBM_ERR_OOM. */
lbm_status lbm_sbf_create(int nfibres, int n_modes, int n_quad, double mu, void *cuda_stream, lbm_sbf **out);

/* Set the fibre geometry (host arrays: centres[3m], tangents[3m] (normalised
 * by the library), half_lengths[m], radii[m]) and compute the interaction
 * integrals.  Errors: LBM_ERR_ARG for a NULL pointer, a zero tangent, a
 * non-positive length or radius, a radius not below the half length, or a
 * slenderness at which a mode's local operator is singular; LBM_ERR_CUDA. */
lbm_status lbm_sbf_set_fibres(lbm_sbf *s, const double *centres, const double *tangents, const double *half_lengths,
                              const double *radii);

/* Velocities for external forces force3m[3m] and torques torque3m[3m]:
 * xdot3m[3m] and pdot3m[3m] (host arrays).  Synchronises.  Errors:
 * LBM_ERR_ARG for a NULL pointer; LBM_ERR_STATE before lbm_sbf_set_fibres;
 * LBM_ERR_NUMERIC for a singular system; LBM_ERR_CUDA. */
lbm_status lbm_sbf_solve(lbm_sbf *s, const double *force3m, const double *torque3m, double *xdot3m, double *pdot3m);

lbm_status lbm_sbf_destroy(lbm_sbf *s);

#ifdef __cplusplus
}
#endif
#endif
