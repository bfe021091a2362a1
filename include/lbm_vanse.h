/*
 * lbm_vanse.h -- C ABI of the GB300 (sm_103a) library for the consistent
 * multiple-relaxation-time lattice Boltzmann method for the volume-averaged
 * Navier-Stokes equations (MRTLB-VANSE; Liu, Zhang, Min, Wu, arXiv:2409.02964),
 * D2Q9, lattice units (dx = dt = c = 1, cs^2 = 1/3).
 *
 * One handle = one lattice resident on the current CUDA device. Every call is
 * issued on the CUDA stream given at creation; calls that hand results back to
 * host memory synchronise that stream. No C++ exception crosses this boundary:
 * every entry point returns an lbm_status and keeps a message per handle
 * (lbm_vanse_last_error).
 *
 * Layouts seen by callers: scalar fields are row-major [ny][nx] doubles (cell
 * (x, y) at y*nx + x); population arrays are [9][ny][nx] doubles with the D2Q9
 * order of Eq. (5): e_0 = (0,0), e_1..e_4 = E, N, W, S, e_5..e_8 = NE, NW, SW, SE.
 * "on_device" = 1 means the pointer is a device pointer on the handle's device,
 * 0 means host memory. Caller memory is only read or written during the call.
 * Internally the library stores populations as SoA planes with a padded row
 * pitch, in the precision chosen at creation; callers never see that layout.
 */
#ifndef LBM_VANSE_H
#define LBM_VANSE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,       /* invalid argument (sizes, rates, pointers, unsupported option) */
    LBM_ERR_CUDA = -2,      /* a CUDA runtime call failed; see lbm_vanse_last_error */
    LBM_ERR_OOM = -3,       /* device allocation failed */
    LBM_ERR_DIVERGED = -4,  /* a reduction found NaN/Inf in the populations */
    LBM_ERR_STATE = -5,     /* call out of order (e.g. step before init_fields) */
    LBM_ERR_TIMEOUT = -6    /* a kernel's bounded wait on its copy engine gave up */
} lbm_status;

/* Storage precision of the populations. FP64 computes in FP64; the others
 * compute in FP32. FP16 and BF16 store deviations from the rest state,
 * (f_i - f_i^rest) * 2^storage_scale_log2, with f_i^rest = w_i kappa rho0 for
 * i >= 1 and (phi - 5 kappa / 9) rho0 for i = 0 (the rest equilibrium of Eq. 14). */
typedef enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16 = 2, LBM_BF16 = 3 } lbm_storage;

/* The base FP16 / BF16 deviations are taken from. LBM_BASE_REST: f_i^rest as above.
 * LBM_BASE_MOMENTUM: f_i^rest + 3 w_i e_i . J, the linear (momentum) term of the
 * Eq. (14) equilibrium, with J the post-collision momentum m_3+, m_5+ of the cell
 * that holds the slot (the slot of population i at cell c holds f_i+(c)); J, rounded
 * to the storage type and scaled like the deviations, is stored in two more planes of
 * each population buffer (2 more values per cell read and written). The remainders
 * are an order smaller than the deviations from rest, so their rounding is too: with
 * BF16 the manufactured-solution error of Eq. (26) stays within a few per cent of
 * FP64's instead of doubling. Step kernel 5 only; not with solid cells. */
typedef enum { LBM_BASE_REST = 0, LBM_BASE_MOMENTUM = 1 } lbm_dev_base;

/* Boundary type of an axis pair: periodic (Sec. 3, default) or half-way
 * bounce-back no-slip walls at both ends (Sec. 3.1). Walls are supported on y. */
typedef enum { LBM_BC_PERIODIC = 0, LBM_BC_BOUNCEBACK = 1 } lbm_bc;

/*
 * Problem statement (Sec. 2.3 and 3): lattice size; relaxation TIME tau_nu of the
 * shear moments (rate s_nu = 1/tau_nu, viscosity nu = (tau_nu - 1/2)/3, Eq. 3-4);
 * the other diagonal entries of Gamma as RATES (s_e <= 0 derives s_e from the bulk
 * viscosity nu_e = nu/3 that Eq. (A12) requires); kappa of the provisional
 * equation of state (Eq. 13-14, default 0.5, Sec. 3); reference density rho0;
 * boundary types; storage precision; model_b = 1 selects the model-B variant
 * (kappa - phi -> kappa - 1 in Eq. 13 and 20, Sec. 2.3).
 */
typedef struct {
    int nx, ny;
    double tau_nu;
    double s_e, s_eps, s_q, s_c;
    double kappa;
    double rho0;
    int bc_x, bc_y;              /* lbm_bc */
    int storage;                 /* lbm_storage */
    int model_b;
    int storage_scale_log2;      /* FP16/BF16 deviation scale exponent (default 16 / 0) */
    int strip_rows;              /* rows per CTA strip of the step kernel; 0 = automatic */
    int eager;                   /* 1 = launch each step on its own; 0 = replay runs of steady
                                    steps as a captured CUDA graph (default) */
    int kernel;                  /* step-kernel variant: 0 = automatic; 1 = one column per thread
                                    (any storage); 2, 3, 4 = two columns per thread on packed FP32
                                    pairs with 64 / 96 / 128-thread CTAs; 5 = one warp per CTA,
                                    two columns per lane (2..5: not FP64) */
    int eq_order;                /* 3 (or 0): the 3rd-order equilibrium of Eq. (14) with Eq. (18), (20);
                                    2: App. B, Eq. (B1)-(B3) (kernels 1 and 5) */
    int dev_base;                /* lbm_dev_base of FP16 / BF16 storage (default LBM_BASE_REST) */
} lbm_vanse_params;

typedef struct lbm_vanse* lbm_vanse_t;

/* Fill *p with the paper's defaults: tau_nu = 0.8 (nu = 0.1), s_e derived,
 * s_eps = 1.2, s_q = 1.4, s_c = 1 (Sec. 2.3), kappa = 0.5, rho0 = 1 (Sec. 3),
 * periodic, FP32 storage. nx, ny are left at 0. */
void lbm_vanse_default_params(lbm_vanse_params* p);

/* Create a lattice on the current device. cuda_stream is a cudaStream_t (NULL =
 * legacy default stream). Allocates the two population buffers, the void-fraction
 * and body-force buffers. Errors: LBM_ERR_ARG (sizes < 1, tau_nu <= 1/2, rates
 * outside (0, 2), kappa outside [0, 1], bc_x = bounce-back with kernels 2-5),
 * LBM_ERR_OOM. Walls in x (bc_x = bounce-back, step kernel 1, chosen by default for
 * them) follow the rule of the y walls: half-way bounce-back links, and in the
 * Eq. (10) stencil the ghost cell past a wall mirrors the cell next to it, vector
 * components negated once even past two walls (a corner). */
lbm_status lbm_vanse_create(const lbm_vanse_params* p, void* cuda_stream, lbm_vanse_t* out);

/* Void fraction phi(x, t) of the next step and phi(x, t+1) (Eq. 7, 13, 14, 20;
 * d_t phi = phi(t+1) - phi(t), Sec. 2.3). phi_next = NULL means steady. After a
 * step, phi(t) takes the value of phi(t+1) and the field is steady until the next
 * call. Values must lie in (0, 1] (phi divides in Eq. 7 and in X = kappa / phi of
 * Eq. 20). Both fields are checked on the device before either replaces the
 * lattice's: a NaN, a negative value or a value above 1 returns LBM_ERR_ARG and
 * leaves the lattice unchanged. The check is waited for: device arrays and pageable
 * host arrays synchronise the lattice's stream; pinned host arrays wait only for their
 * own copy and check (below). A zero marks a solid cell (lbm_vanse_set_solid_cells);
 * without solid cells it is reported by the next lbm_vanse_sync.
 * Must be called before lbm_vanse_init_fields.
 * A new phi(t) keeps the populations the steps left (FP32/FP16/BF16 move their
 * stored f_0 deviation to the new rest value; FP16/BF16 round it again).
 * Host arrays in pinned (page-locked) memory are copied on a stream of the
 * library's own, so the copy overlaps the steps still queued on the lattice's
 * stream; the call returns once the arrays have been read, as for any host array. */
lbm_status lbm_vanse_set_void_fraction(lbm_vanse_t h, const double* phi_t, const double* phi_next,
                                       int on_device);

/* The same with float arrays [ny][nx] (same meaning, ownership and errors). The
 * FP32/FP16/BF16 storages compute with phi in FP32, so this form moves half the bytes
 * of the double one and gives identical results for values that are floats already;
 * FP64 storage widens the floats exactly. */
lbm_status lbm_vanse_set_void_fraction_f32(lbm_vanse_t h, const float* phi_t, const float* phi_next,
                                           int on_device);

/* Body force F^B(x, t) = phi(x, t) * (gx, gy) + field(x) (Eq. 6; the phi G form of
 * Sec. 3.1 plus an optional per-cell part, [2][ny][nx], x component first, e.g.
 * the manufactured force of Eq. 25). field may be NULL. Stays in effect until the
 * next call. */
lbm_status lbm_vanse_set_body_force(lbm_vanse_t h, double gx, double gy, const double* field,
                                    int on_device);

/* Linear drag added to the body force (Sec. 3.1, Eq. 21 and 23):
 *   F^B += -beta (u - u_s),  beta(x) = phi(x)^2 (d0 + d1 (1 - phi(x))),
 * so d0 = nu / k0 gives the Darcy resistance phi nu u / k0 of Sec. 3.1 (with F^B =
 * phi G from set_body_force) and d1 = 1 the fluid-solid drag of Eq. (23). Because the
 * drag is linear in u, Eq. (7) is solved exactly for u each step. d0, d1 >= 0;
 * d0 = d1 = 0 removes it. Runs on step kernels 1 and 5 (LBM_ERR_ARG on 2-4); it
 * takes the row loop's general path. Also used by init_fields and macros. */
lbm_status lbm_vanse_set_drag(lbm_vanse_t h, double d0, double d1, double us_x, double us_y);

/* Moving wall (Sec. 3.1, the Couette case of Eq. 22 II): with enable = 1 the top row
 * y = ny-1 becomes a row of wall nodes moving at (uw_x, uw_y), imposed by
 * non-equilibrium extrapolation, the scheme the paper uses: before each collision
 * the wall node's populations become f^eq(rho_f, u_w, phi_b) + f(x_f) - f^eq(rho_f,
 * u_f, phi_f), x_f = (x, ny-2) the fluid node below, rho_f and u_f its Eq. (7) values
 * (F^p there uses rho_b = rho_f), f^eq of Eq. (14) (B1 with eq_order 2). The wall
 * row's Eq. (10) stencil reads a ghost row extrapolated linearly from rows ny-1 and
 * ny-2. The bottom stays a half-way bounce-back wall, so the channel height is
 * ny - 1/2. Needs bc_y = LBM_BC_BOUNCEBACK, periodic x, ny >= 3 and step kernel 1
 * or 5 (LBM_ERR_ARG otherwise; on kernel 5 the rows next to the wall take the row
 * loop's general path); enable = 0 restores the half-way wall. lbm_vanse_macros reports the
 * wall row from its populations before the replacement. */
lbm_status lbm_vanse_set_moving_wall(lbm_vanse_t h, int enable, double uw_x, double uw_y);

/* Solid cells (the impermeable block of Sec. 3.3, Eq. 24 with phi_0 = 0): with
 * enable = 1, a cell whose void fraction is exactly 0 is solid. It holds no
 * populations (reported as zeros; macros report rho = u = p = 0 there), every link
 * from a fluid cell into it is a half-way bounce-back link, and in the Eq. (10)
 * stencil of a fluid cell it reads a ghost value mirrored about the solid surface: an
 * axis neighbour the cell itself, a diagonal neighbour the mean of the fluid ones of
 * its two axis images (the cell itself if both are solid), vector components negated.
 * Solid cells must stay solid (phi(t+1) = 0 where phi(t) = 0). Step kernels 1 and 5
 * (LBM_ERR_ARG otherwise; kernel 5 then runs every row on its general path and leaves
 * the stored values of solid cells as they are, since no link reads them); call
 * before lbm_vanse_init_fields. Without it a zero in
 * phi is an error, reported by the next lbm_vanse_sync. */
lbm_status lbm_vanse_set_solid_cells(lbm_vanse_t h, int enable);

/* Initial populations f = f^eq(rho, u, phi) - F_i(u, F)/2 (Eq. 14, Eq. 6 with
 * F = F^p + F^B, F^p from grad rho by Eq. 10 and 13), so that Eq. (7) returns u.
 * rho, ux, uy: [ny][nx]. Uses the void fraction and body force set before. */
lbm_status lbm_vanse_init_fields(lbm_vanse_t h, const double* rho, const double* ux,
                                 const double* uy, int on_device);

/* Advance nsteps time steps: per cell the fused stream + collide of Eq. (16)
 * (moments Eq. 17/A1, equilibrium Eq. 18, force moments Eq. 19 with F^p of Eq. 13,
 * penalty source Eq. 20 with gradients by Eq. 10, back-transform A1), streaming
 * with periodic wrap or half-way bounce-back. Asynchronous on the stream. Unless
 * params.eager is set, runs of steady steps are replayed as a CUDA graph captured
 * on first use (re-captured when phi, the force or the buffer parity change). */
lbm_status lbm_vanse_step(lbm_vanse_t h, int nsteps);

/* Macroscopic fields at the current time (Eq. 7): rho = sum f / phi,
 * u = (sum e f + F/2) / sum f with F = F^p + F^B, p = rho cs^2. Any output may
 * be NULL. Arrays [ny][nx]. */
lbm_status lbm_vanse_macros(lbm_vanse_t h, double* rho, double* ux, double* uy, double* p,
                            int on_device);

/* Post-streaming populations f_i(x, t) as [9][ny][nx] doubles (get), or replace
 * them (set; e.g. to restore a checkpoint). */
lbm_status lbm_vanse_get_populations(lbm_vanse_t h, double* f, int on_device);
lbm_status lbm_vanse_set_populations(lbm_vanse_t h, const double* f, int on_device);

/* Domain sums accumulated in FP64 on the device: mass = sum_x sum_i f_i and
 * momentum sum_x sum_i e_i f_i (= sum of j = phi rho u - F/2, Eq. 17). Results to
 * host memory (synchronises). Returns LBM_ERR_DIVERGED if any is NaN/Inf. */
lbm_status lbm_vanse_reduce(lbm_vanse_t h, double* mass, double* momx, double* momy);

/* The same three sums without waiting for them: the reduction and a copy of the
 * result to out[0..2] (mass, momentum x, momentum y; FP64) are queued on the
 * lattice's stream and the call returns at once. out is device memory when
 * on_device, else host memory (pinned, for the copy to be asynchronous); it must
 * stay valid until the stream has passed the copy, and holds the sums only then
 * (after lbm_vanse_sync, or an event recorded on the stream after this call). No
 * divergence check: the caller tests the values for finiteness. */
lbm_status lbm_vanse_reduce_async(lbm_vanse_t h, double* out, int on_device);

/* One step (as lbm_vanse_step(h, 1)) whose kernel also sums, over the lattice, the
 * post-collision moments it writes: out[0] = sum m_0+ (the mass, which Eq. 16
 * conserves), out[1..2] = sum j+ = sum (j + F) (Eq. 16 with S_3 = F_x, S_5 = F_y):
 * the momentum of the new populations before they stream. FP64 sums of per-thread
 * compensated partials; no separate pass over the populations. Queued like
 * lbm_vanse_reduce_async (same rules for out and on_device; no waiting, no
 * divergence check). Step kernels 1 and 5 (the defaults); LBM_ERR_ARG for 2-4. */
lbm_status lbm_vanse_step_sums(lbm_vanse_t h, double* out, int on_device);

/* Velocity error of Eq. (26), accumulated in FP64:
 * *num = sum |u - u_ref|^2, *den = sum |u_ref|^2 (E_u = sqrt(num/den)).
 * ux_ref, uy_ref: [ny][nx]. Results to host memory. */
lbm_status lbm_vanse_velocity_error(lbm_vanse_t h, const double* ux_ref, const double* uy_ref,
                                    int on_device, double* num, double* den);

/* Largest ny that lbm_vanse_reduce_noalloc accepts: its scratch holds one partial
 * (mass, momx, momy) triple per lattice row. */
#define LBM_VANSE_NOALLOC_MAX_ROWS 8192

/* Allocation-free form of lbm_vanse_reduce, for callers that cannot allocate device
 * memory while they run: a host loop whose memory is planned once and must not grow,
 * an application whose allocator owns all device memory (cudaMalloc from a library
 * would fragment or bypass it), or code that must not synchronise the device, which
 * cudaMalloc and cudaFree may do. This method's paper has no counterpart; it is a
 * service of this library.
 *
 * Computes the same FP64 sums as lbm_vanse_reduce (mass = sum_x sum_i f_i, momentum
 * sum_x sum_i e_i f_i) and writes them to out_dev[0..2], a caller-owned DEVICE array
 * of 3 doubles, asynchronously on the handle's stream (read it after synchronising).
 * Nothing is allocated or freed: the per-row partial sums live in one fixed device
 * array of LBM_VANSE_NOALLOC_MAX_ROWS x 3 doubles (192 KiB) inside the library, which
 * every GPU that loads the library keeps until the process exits.
 *
 * The first call on a device looks up that array's device address with that device
 * current; make that first call before starting any stream capture (a first call on
 * a capturing stream returns LBM_ERR_STATE). The kernels run on the handle's device
 * whichever device the calling thread has current; the caller's current device is
 * restored before the call returns. Every call on a
 * device shares the one array: calls whose kernels overlap on the GPU (two streams,
 * two handles, two threads) race on it and may return mixed sums, so keep such calls
 * ordered. Each call writes every partial it reads, so no clearing is needed and a
 * previous call's leftovers never leak into a result.
 *
 * Errors: LBM_ERR_ARG for a NULL handle or output, or ny > LBM_VANSE_NOALLOC_MAX_ROWS;
 * LBM_ERR_STATE before initialisation, or for a first call on a capturing stream;
 * LBM_ERR_CUDA if the address lookup, a device switch or a launch fails. It does not check the sums for NaN (the caller reads them). */
lbm_status lbm_vanse_reduce_noalloc(lbm_vanse_t h, double* out_dev);

/* ======================================================================== batches
 * Many independent n x n periodic lattices advanced together, each with its own
 * relaxation time and its own spatiotemporal manufactured solution (Sec. 3.4):
 * phi = phi0 + A sin(2 pi x/n) sin(2 pi y/n) cos(2 pi t/T), phi u = grad psi +
 * rot Psi with lap psi = -d_t phi and Psi = (U0 n / 2 pi) sin sin, rho = rho0, and the
 * body force of Eq. (25) without its pressure term. The void fraction and the force
 * are evaluated inside the step kernel, so a step reads and writes only populations.
 * One step of the whole batch is one persistent kernel that hands out work units
 * (60 columns x H rows of one lattice, largest lattices first) from a device
 * counter, followed by a one-thread kernel that advances the device-side clock; runs
 * of steps are replayed as a captured CUDA graph. */
typedef struct {
    int n;                /* lattice size (n x n), >= 1 */
    double tau_nu;        /* relaxation time of the shear moments (> 1/2) */
    double amplitude;     /* A */
    double period;        /* T in steps (> 0) */
    double u0;            /* U0 */
} lbm_vanse_batch_lattice;

typedef struct {
    int storage;          /* LBM_FP32, LBM_FP16 or LBM_BF16 */
    double s_e;           /* energy rate; <= 0 derives it per lattice from nu_e = nu/3 (App. A) */
    double s_eps, s_q;    /* rates shared by all lattices */
    double kappa, rho0, phi0;
    int strip_rows;       /* rows per work unit; 0 = a default (see lbm_vanse_batch_autotune) */
    int eager;            /* 1 = launch every step on its own (no CUDA graph) */
} lbm_vanse_batch_params;

typedef struct lbm_vanse_batch* lbm_vanse_batch_t;

/* Defaults: FP32, s_e = s_eps = s_q = 1.2, kappa = 0.5, rho0 = 1, phi0 = 0.7. */
void lbm_vanse_batch_default_params(lbm_vanse_batch_params* p);

/* Allocate count lattices (two population buffers each) on the current device.
 * Errors: LBM_ERR_ARG (count < 1, a bad lattice or parameter), LBM_ERR_OOM. */
lbm_status lbm_vanse_batch_create(const lbm_vanse_batch_lattice* lattices, int count,
                                  const lbm_vanse_batch_params* p, void* cuda_stream,
                                  lbm_vanse_batch_t* out);

/* t = 0 and every lattice at f = f^eq(rho0, u(0), phi(0)) - F_i/2 (Eq. 14, 6). */
lbm_status lbm_vanse_batch_init(lbm_vanse_batch_t b);

/* Advance every lattice nsteps steps (one persistent kernel per step). */
lbm_status lbm_vanse_batch_step(lbm_vanse_batch_t b, int nsteps);

/* The same steps with one kernel launch per lattice per step (the form the
 * persistent kernel replaces; for comparison). Each lattice is cut into strips as
 * a lone lattice would be (about five waves of resident CTAs, >= 16 rows). */
lbm_status lbm_vanse_batch_step_each(lbm_vanse_batch_t b, int nsteps);

/* Time trial_steps steps for each work-unit height of {16, 24, 32, 48, 64, 96, 128,
 * 192, 256}, keep the fastest, write it to *rows_out (may be NULL) and
 * re-initialise the batch (t = 0). */
lbm_status lbm_vanse_batch_autotune(lbm_vanse_batch_t b, int trial_steps, int* rows_out);

/* Eq. (26) sums for lattice index at the current step against its manufactured
 * velocity: *num = sum |u - u_ref|^2, *den = sum |u_ref|^2 (FP64, to host). */
lbm_status lbm_vanse_batch_velocity_error(lbm_vanse_batch_t b, int index, double* num, double* den);

/* Post-streaming populations of lattice index as [9][n][n] doubles. */
lbm_status lbm_vanse_batch_get_populations(lbm_vanse_batch_t b, int index, double* f, int on_device);

/* Total cells of the batch; steps taken since init. */
long long lbm_vanse_batch_cells(lbm_vanse_batch_t b);
long long lbm_vanse_batch_step_count(lbm_vanse_batch_t b);
const char* lbm_vanse_batch_last_error(lbm_vanse_batch_t b);
void lbm_vanse_batch_destroy(lbm_vanse_batch_t b);

/* ------------------------------------------------------------------------------
 * Gradient with respect to the void fraction (discrete adjoint, FP64).
 *
 * Problem: steady phi(x) on the lattice of p (x periodic, y as p->bc_y; bc_x must
 * be periodic); body force F^B = phi (gx, gy) (the Eq. 6 forcing of Sec. 3.1);
 * initial populations f(0) = f^eq(rho = 1, u = 0, phi) - F_i/2 (Eq. 14, 6); then
 * nsteps steps of Eq. (16) with streaming. After step n the objective samples
 *   O(n) = sum over y of (phi rho u_x)(x_out, y) = sum_y (j_x + F_x / 2)(x_out, y)
 * (Eq. 7), and J = sum of O(n) over n = nsteps - avg_steps + 1 .. nsteps divided by
 * avg_steps * ny: the mean outlet x-momentum over the last avg_steps steps.
 * dJ/dphi(x) is the exact derivative of this discrete J (every path by which phi
 * enters: Eq. 7 rho, Eq. 13 F^p, X = kappa / phi in Eq. 18 and Eq. 20, F^B and
 * f(0)), computed by a hand-written adjoint of the step run backwards in time. The
 * forward pass stores a checkpoint every K = checkpoint_every steps; the backward
 * pass recomputes one segment of K steps at a time. With dense_segments = 0 (the
 * default) the checkpoints live in pinned host memory, and inside a segment the
 * states every K2 = ceil(sqrt(K)) steps are recomputed and also kept on the host;
 * the device holds one sub-segment of K2 states (about 2 + K2 population arrays and
 * a few fields in all; every step is recomputed twice in the backward pass). With
 * dense_segments = 1 the checkpoints and a whole segment of K states stay on the
 * device (one recomputation, K + T/K population arrays). Both give bit-identical
 * results. Everything runs in FP64 on the stream given, whatever p->storage says.
 * The paper has no adjoint; this is the differentiable-design use of its method. */
typedef struct {
    int nsteps;            /* >= 1 */
    int avg_steps;         /* 1 .. nsteps */
    int checkpoint_every;  /* >= 1 */
    int x_out;             /* outlet column, 0 .. nx - 1 */
    double gx, gy;         /* F^B = phi (gx, gy) */
    int dense_segments;    /* 0: checkpoints on the host, K2-state sub-segments; 1: all on the device */
} lbm_vanse_adjoint_params;

typedef struct {
    double forward_ms;     /* device time of the forward pass (with checkpoints) */
    double backward_ms;    /* device time of the backward pass (with recomputation) */
    long long device_bytes;  /* device memory the call held at its peak */
    long long host_bytes;    /* pinned host memory it held for checkpoints */
} lbm_vanse_adjoint_stats;

/* phi: [ny][nx] doubles, on the device (on_device = 1) or host; read only. J
 * receives the objective (host pointer). dJdphi: [ny][nx] doubles, device or host
 * like phi, or NULL for the objective alone (no backward pass). stats may be NULL.
 * The call allocates its own device memory on cuda_stream and frees it before it
 * returns; it synchronises the stream. Errors: LBM_ERR_ARG (a bad parameter or
 * NULL), LBM_ERR_OOM, LBM_ERR_CUDA; the message is in lbm_vanse_last_error(NULL). */
lbm_status lbm_vanse_outlet_momentum_grad(const lbm_vanse_params* p, const lbm_vanse_adjoint_params* a,
                                          const double* phi, int on_device, void* cuda_stream, double* J,
                                          double* dJdphi, lbm_vanse_adjoint_stats* stats);

/* Checkpoint and resume (no counterpart in the paper; a service of this library).
 * A state is everything a later step depends on: the stored populations as they are
 * (the current buffer with its padding and ghost columns; FP16/BF16 deviations
 * bit for bit), phi(x, t), a pending phi(x, t+1), the body force (constant and
 * field), the drag and moving-wall settings, the step count and the device step
 * counter that seeds the stochastic rounding of FP16/BF16 stores. Loading it into a
 * lattice created with the same nx, ny, storage and solid-cell setting continues the
 * run bit for bit. Layout: a 512-byte header, then the raw device contents.
 *
 * lbm_vanse_state_bytes: the size of the state now (it depends on a pending
 * phi(t+1) and on a force field), or -1 before initialisation.
 * lbm_vanse_save_state: writes it to buf (host memory, or device memory with
 * on_device = 1; at least lbm_vanse_state_bytes bytes); synchronises the stream.
 * lbm_vanse_load_state: reads it back; synchronises the stream. Errors: LBM_ERR_ARG
 * for a NULL argument, a buffer that is not a state, or a state of another lattice;
 * LBM_ERR_STATE (save) before initialisation; LBM_ERR_CUDA for a failed copy. */
long long lbm_vanse_state_bytes(lbm_vanse_t h);
lbm_status lbm_vanse_save_state(lbm_vanse_t h, void* buf, int on_device);
lbm_status lbm_vanse_load_state(lbm_vanse_t h, const void* buf, int on_device);

/* Synchronise the stream and report any deferred kernel error (LBM_ERR_TIMEOUT
 * if a bounded wait gave up, LBM_ERR_CUDA for a launch/runtime error). After a
 * timeout the populations are not valid; the flag stays set. */
lbm_status lbm_vanse_sync(lbm_vanse_t h);

/* Test hook for the timeout path (no counterpart in the paper): every wait of the
 * step kernels for a staged source row gives up after `polls` polls of its mbarrier.
 * The default, restored by polls < 0, is the library's bound of kWaitTries polls
 * (seconds, far above a row's latency); larger values are capped at it, and 0 makes
 * every wait give up at once. A wait that gives up sets the lattice's timeout flag;
 * the kernel finishes its group of rows, waits with the full bound for every copy it
 * issued (so no copy lands after it exits) and returns; the next lbm_vanse_sync
 * returns LBM_ERR_TIMEOUT. Takes effect from the next step. LBM_ERR_ARG for a NULL
 * handle. */
lbm_status lbm_vanse_set_row_wait_limit(lbm_vanse_t h, long long polls);

/* Steps taken since init_fields / set_populations. */
long long lbm_vanse_step_count(lbm_vanse_t h);

/* Device bytes one step reads and writes per cell as the method requires them
 * (9 populations in and out, phi, plus phi(t+1) and the force field when set). */
double lbm_vanse_bytes_per_cell(lbm_vanse_t h);

/* Launch shape of the step kernel: threads per CTA, output columns per CTA,
 * rows per strip, CTAs in x and y, dynamic shared memory bytes. Any may be NULL. */
lbm_status lbm_vanse_launch_shape(lbm_vanse_t h, int* threads, int* cols, int* rows, int* grid_x,
                                  int* grid_y, int* smem_bytes);

/* Message of the last failed call on h (or of the last failed create when h is NULL). */
const char* lbm_vanse_last_error(lbm_vanse_t h);

/* Free every device buffer of h. Safe on NULL. */
void lbm_vanse_destroy(lbm_vanse_t h);

#ifdef __cplusplus
}
#endif

#endif /* LBM_VANSE_H */
