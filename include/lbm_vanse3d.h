/*
 * lbm_vanse3d.h -- C ABI of the three-dimensional (D3Q19) form of the MRTLB-VANSE
 * scheme (arXiv:2409.02964, Sec. 2.3; the 3-D extension its Sec. 4 names), on a
 * GB300 (sm_103a). Lattice units (dx = dt = c = 1, cs^2 = 1/3).
 *
 * What one step computes, per cell (the 2-D step of Eq. (5)-(7), (10), (13)-(20)
 * with its ingredients taken to D3Q19):
 *   - density rho = sum f / phi (Eq. 7); gradient by Eq. (10) with the D3Q19 weights,
 *     grad psi = 3 sum_i w_i psi(x + e_i) e_i;
 *   - force F = (kappa - phi) cs^2 grad rho (Eq. 13) + F^B, velocity
 *     u = (sum e f + F/2) / sum f (Eq. 7);
 *   - moments m = M f in the D3Q19 basis of d'Humieres et al. (2002)
 *     (rho, e, eps, j_x, q_x, j_y, q_y, j_z, q_z, 3p_xx, 3pi_xx, p_ww, pi_ww, p_xy,
 *     p_yz, p_xz, m_x, m_y, m_z);
 *   - equilibrium moments that give f^eq the velocity moments of Eq. (15): mass
 *     phi rho, momentum phi rho u, second moment phi rho u u + kappa rho cs^2 I,
 *     third moment kappa rho cs^2 (u delta + ...) apart from the e_a^3 = e_a
 *     components, which the lattice fixes to phi rho u_a (as in 2-D);
 *   - the Guo force moments (Eq. 6, 19), and the penalty source of Eq. (16) derived
 *     for the D3Q19 stress moments by the Chapman-Enskog bookkeeping of App. A:
 *       C_e      = 19 [(1 - X) div(phi rho u) - X rho d_t phi + 2/3 (kappa - phi) rho div u],
 *       C(3p_xx) = sum_a w_a [-kappa d_a(rho u_a) + 2/3 (kappa - phi) rho d_a u_a
 *                             + d_a(phi rho u_a)],  w = (2, -1, -1); p_ww: w = (0, 1, -1),
 *       C(p_ab)  = 1/3 (kappa - phi) rho (d_a u_b + d_b u_a),
 *     X = kappa / phi, d_t phi = phi(t+1) - phi(t);
 *   - relaxation m+ = m - Gamma (m - m^eq) + (I - Gamma/2)(S + C), f+ = M^-1 m+, and
 *     streaming, periodic in x and z, periodic or half-way bounce-back walls in y.
 * The scheme recovers Eq. (A12) in 3-D with the stress
 *   tau = rho nu (grad u + grad u^T - 2/3 div u I) + 2/3 rho nu_e div u I,
 * nu = cs^2 (1/s_nu - 1/2), nu_e = cs^2 (1/s_e - 1/2).
 *
 * Conventions as in lbm_vanse.h: one handle = one lattice on the current CUDA device;
 * every call runs on the stream given at creation and calls that return values in
 * host memory synchronise it; every entry point returns an lbm_status and keeps a
 * message (lbm_vanse3d_last_error). "on_device" = 1: device pointer; 0: host memory,
 * only read or written during the call.
 *
 * Layouts seen by callers: fields are [nz][ny][nx] doubles (cell (x, y, z) at
 * (z*ny + y)*nx + x); vector fields and forces [3][nz][ny][nx] (x component first);
 * populations [19][nz][ny][nx] doubles, post-streaming f_i(x, t), in the velocity
 * order e_0 = 0; e_1..e_6 = +x, -x, +y, -y, +z, -z; e_7..e_10 = (1,1,0), (-1,-1,0),
 * (1,-1,0), (-1,1,0); e_11..e_14 = (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1);
 * e_15..e_18 = (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1). The library stores the
 * populations as the same SoA planes in the precision chosen at creation, as
 * deviations from the rest state (w_i kappa rho0 for i >= 1, (phi - 2 kappa / 3) rho0
 * for i = 0); callers always see the populations themselves.
 */
#ifndef LBM_VANSE3D_H
#define LBM_VANSE3D_H

#include "lbm_vanse.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Problem statement: lattice size (each >= 1); relaxation TIME tau_nu of the stress
 * moments (s_nu = 1/tau_nu, nu = (tau_nu - 1/2)/3, tau_nu > 1/2); the other rates of
 * Gamma: s_e (<= 0 derives it from nu_e = nu/3, the 2-D choice; s_e = 2 would give
 * the Stokes stress but leaves the energy mode undamped), s_eps, s_q (energy flux),
 * s_pi (the fourth-order pi moments), s_m (the third-order m moments), each in (0, 2];
 * kappa of the provisional equation of state (Eq. 13-14); rho0 (> 0); bc_y
 * (lbm_bc: periodic, or half-way bounce-back walls at y = -1/2 and ny - 1/2; x and z
 * are periodic); storage (LBM_FP64, which computes in FP64, or LBM_FP32, which
 * computes in FP32).
 */
typedef struct {
    int nx, ny, nz;
    double tau_nu;
    double s_e, s_eps, s_q, s_pi, s_m;
    double kappa;
    double rho0;
    int bc_y;
    int storage;
} lbm_vanse3d_params;

typedef struct lbm_vanse3d* lbm_vanse3d_t;

/* Defaults: tau_nu = 0.8, s_e derived, s_eps = s_q = s_pi = s_m = 1.2, kappa = 0.5,
 * rho0 = 1, periodic, FP32; nx = ny = nz = 0 (the caller sets them). */
void lbm_vanse3d_default_params(lbm_vanse3d_params* p);

/* Allocate the lattice (two population buffers of 19 nx ny nz values, the
 * void-fraction fields and per-cell scratch) on the current device; stream may be
 * NULL (the default stream). LBM_ERR_ARG for invalid parameters, LBM_ERR_OOM when
 * the device memory does not suffice. On success *out owns the memory until
 * lbm_vanse3d_destroy. */
lbm_status lbm_vanse3d_create(const lbm_vanse3d_params* p, void* stream, lbm_vanse3d_t* out);

/* Free everything the handle holds (NULL is allowed). */
void lbm_vanse3d_destroy(lbm_vanse3d_t h);

/* phi(x, t) and optionally phi(x, t+1) (each nx ny nz doubles, every value in (0, 1]).
 * With phi_next the next step takes d_t phi = phi_next - phi_t and afterwards
 * phi(t) <- phi_next (steady again); NULL phi_next means steady. Required before
 * init_fields. A new phi(t) keeps the populations the steps left. LBM_ERR_ARG for a
 * NULL phi_t or a value outside (0, 1] (the lattice keeps its previous phi). */
lbm_status lbm_vanse3d_set_void_fraction(lbm_vanse3d_t h, const double* phi_t, const double* phi_next,
                                         int on_device);

/* Body force F^B = phi (gx, gy, gz) + field ([3][nz][ny][nx] doubles, may be NULL),
 * in effect until the next call. */
lbm_status lbm_vanse3d_set_body_force(lbm_vanse3d_t h, double gx, double gy, double gz, const double* field,
                                      int on_device);

/* Initial populations f = f^eq(rho, u, phi) - F_i/2 with F = F^p(rho) + F^B (each
 * field nx ny nz doubles; u the physical velocity). LBM_ERR_STATE before
 * set_void_fraction. */
lbm_status lbm_vanse3d_init_fields(lbm_vanse3d_t h, const double* rho, const double* ux, const double* uy,
                                   const double* uz, int on_device);

/* Advance nsteps (>= 0) time steps, queued on the handle's stream (asynchronous).
 * LBM_ERR_STATE before init_fields. */
lbm_status lbm_vanse3d_step(lbm_vanse3d_t h, int nsteps);

/* Wait for the handle's stream; reports a CUDA error raised by earlier launches. */
lbm_status lbm_vanse3d_sync(lbm_vanse3d_t h);

/* Post-streaming populations out (19 nx ny nz doubles) / in. set_populations marks
 * the lattice initialised (LBM_ERR_STATE before set_void_fraction). */
lbm_status lbm_vanse3d_get_populations(lbm_vanse3d_t h, double* f, int on_device);
lbm_status lbm_vanse3d_set_populations(lbm_vanse3d_t h, const double* f, int on_device);

/* rho (nx ny nz doubles) and the velocity u ([3][nz][ny][nx] doubles) of Eq. (7),
 * with the force of the current phi and F^B; either pointer may be NULL. */
lbm_status lbm_vanse3d_macros(lbm_vanse3d_t h, double* rho, double* u, int on_device);

/* FP64 sums over the lattice: mass = sum_x sum_i f_i, mom[3] = sum_x sum_i e_i f_i
 * (host pointers; synchronises). LBM_ERR_DIVERGED when a sum is not finite. */
lbm_status lbm_vanse3d_reduce(lbm_vanse3d_t h, double* mass, double* mom);

/* Steps taken since init_fields / set_populations. */
long long lbm_vanse3d_step_count(lbm_vanse3d_t h);

/* The last error message of h (or of the last failed create when h is NULL). */
const char* lbm_vanse3d_last_error(lbm_vanse3d_t h);

#ifdef __cplusplus
}
#endif

#endif
