/*
 * vanse_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of one time step of the consistent
 * multiple-relaxation-time lattice Boltzmann method for the volume-averaged
 * Navier-Stokes equations (MRTLB-VANSE; Liu, Zhang, Min, Wu, arXiv:2409.02964),
 * D2Q9, lattice units (dx = dt = c = 1, cs^2 = 1/3).
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg load this
 * code. It shares no source, header, table or helper with the CUDA library, and
 * the CUDA library never loads it.
 *
 * What each function follows (section / equation of the paper):
 *   vo_lattice          Eq. (5)             D2Q9 velocities e_i and weights w_i
 *   vo_M, vo_Minv       Eq. (17), (A1)      moment matrix and its printed inverse
 *   vo_feq              Eq. (14)            adjusted 3rd-order density equilibrium
 *   vo_guo_force        Eq. (6)             velocity-space forcing term F_i
 *   vo_meq              Eq. (18)            equilibrium moments
 *   vo_force_moments    Eq. (19)            force moments S
 *   vo_penalty          Eq. (20) (+ Sec. 2.3 model-B variant)   penalty source C
 *   vo_gradient         Eq. (10)            isotropic finite-difference gradient
 *   vo_macros           Eq. (7), (13)       density, pressure-correction force, velocity
 *   vo_step             Eq. (16) + streaming (Sec. 2.3) + half-way bounce-back (Sec. 3.1)
 *   vo_init             f = f^eq - F_i/2    (the paper is silent; reading c7)
 *   eq_order = 2        App. B: Eq. (B1) equilibrium, (B2) moments, (B3) penalty
 *   phi = 0             a solid (impermeable) cell: half-way bounce-back links and a
 *                       mirrored Eq. (10) ghost (solid_ghost; the phi_0 = 0 block of
 *                       Sec. 3.3)
 *   nee_top, uw_x, uw_y the moving wall of the Couette case (Sec. 3.1, Eq. 22 II) by
 *                       non-equilibrium extrapolation (the scheme the paper cites);
 *                       the readings it needs are listed at nee_fill below
 *   drag_d0, drag_d1,   a body force linear in u, F^B += -beta (u - u_s) with
 *   us_x, us_y          beta = phi^2 (d0 + d1 (1 - phi)): the Darcy term of Sec. 3.1
 *                       (d0 = nu / k0) and the drag law of Eq. (23) (d1 = 1); u is
 *                       solved implicitly from Eq. (7) (reading c8)
 *
 * Readings where the paper is silent or garbled (all listed in the design notes):
 *   - the relaxation "tau"s of the paper are rates (the diagonal of Gamma);
 *   - relaxation is m - Gamma (m - m^eq) (Eq. 16; the sign in (A2) is garbled);
 *   - m_3 = j_x and m_5 = j_y (Eq. 17 / (A1) rows; App. A's m_4/m_6 is garbled);
 *   - rho and X use phi(x,t); d_t phi = phi(x,t+1) - phi(x,t); F^B is taken at t;
 *   - next to a half-way bounce-back wall the gradient stencil reads a ghost cell
 *     mirrored about the wall: rho and phi keep the mirror value, every component
 *     of the vector fields (u, rho u, phi rho u) changes sign (no-slip);
 *   - the initial populations are f^eq(rho, u, phi) - F_i(u, F)/2.
 *
 * Parity pins (tests/test_oracle_*.py): M M^-1 = I and the rows of M against the
 * moment definitions; M f^eq = m^eq and M F = S for random inputs; the Eq. (15)
 * moments; exactness of Eq. (10) on quadratics; Eq. (20) against the
 * Chapman-Enskog difference (A9) - (A10); reduction to a textbook BGK with Guo
 * forcing when phi = kappa and all rates are equal; the rest-state fixed point;
 * mass and momentum balance; exact Poiseuille flow at the "magic" MRT rates; and
 * second-order convergence on manufactured solutions.
 *
 * Array layout: row-major [ny][nx] fields, populations [9][ny][nx], body force
 * [2][ny][nx] (x component first). Cell (x, y) has index y*nx + x.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9

typedef struct {
    int nx, ny;
    /* diagonal of Gamma (relaxation rates), Sec. 2.3 */
    double s_c, s_e, s_eps, s_q, s_nu;
    double kappa;      /* provisional equation-of-state constant, Eq. (13) */
    int bc_x, bc_y;    /* 0 = periodic, 1 = half-way bounce-back walls at both ends */
    int model_b;       /* 1: kappa - phi -> kappa - 1 in Eq. (13) and Eq. (20) */
    int nthreads;      /* OpenMP threads for the cell loops; <= 0 keeps the default */
    int eq_order;      /* 3: Eq. (14), (18), (20) (default); 2: App. B, Eq. (B1)-(B3) */
    double drag_d0, drag_d1, us_x, us_y;   /* linear drag, see the header */
    int nee_top;       /* 1 (with bc_y = 1): the top row ny-1 is a velocity wall by
                        * non-equilibrium extrapolation (Sec. 3.1), wall velocity uw */
    double uw_x, uw_y;
} vo_params;

/* ---------------------------------------------------------------- Eq. (5) */
void vo_lattice(int e[Q][2], double w[Q])
{
    const double pi = acos(-1.0);
    e[0][0] = 0; e[0][1] = 0; w[0] = 4.0 / 9.0;
    for (int i = 1; i <= 4; ++i) {
        double a = (i - 1) * pi / 2.0;
        e[i][0] = (int)lround(cos(a));
        e[i][1] = (int)lround(sin(a));
        w[i] = 1.0 / 9.0;
    }
    for (int i = 5; i <= 8; ++i) {
        double a = (2 * i - 9) * pi / 4.0;
        e[i][0] = (int)lround(sqrt(2.0) * cos(a));
        e[i][1] = (int)lround(sqrt(2.0) * sin(a));
        w[i] = 1.0 / 36.0;
    }
}

/* --------------------------------------------------------------- Eq. (A1) */
static const double M_TAB[Q][Q] = {
    { 1,  1,  1,  1,  1,  1,  1,  1,  1},
    {-4, -1, -1, -1, -1,  2,  2,  2,  2},
    { 4, -2, -2, -2, -2,  1,  1,  1,  1},
    { 0,  1,  0, -1,  0,  1, -1, -1,  1},
    { 0, -2,  0,  2,  0,  1, -1, -1,  1},
    { 0,  0,  1,  0, -1,  1,  1, -1, -1},
    { 0,  0, -2,  0,  2,  1,  1, -1, -1},
    { 0,  1, -1,  1, -1,  0,  0,  0,  0},
    { 0,  0,  0,  0,  0,  1, -1,  1, -1},
};

/* the printed inverse, without its common factor 1/36 */
static const double MINV36_TAB[Q][Q] = {
    {4, -4,  4,  0,  0,  0,  0,  0,  0},
    {4, -1, -2,  6, -6,  0,  0,  9,  0},
    {4, -1, -2,  0,  0,  6, -6, -9,  0},
    {4, -1, -2, -6,  6,  0,  0,  9,  0},
    {4, -1, -2,  0,  0, -6,  6, -9,  0},
    {4,  2,  1,  6,  3,  6,  3,  0,  9},
    {4,  2,  1, -6, -3,  6,  3,  0, -9},
    {4,  2,  1, -6, -3, -6, -3,  0,  9},
    {4,  2,  1,  6,  3, -6, -3,  0, -9},
};

void vo_M(double M[Q][Q])
{
    memcpy(M, M_TAB, sizeof(M_TAB));
}

void vo_Minv(double Minv[Q][Q])
{
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j)
            Minv[i][j] = MINV36_TAB[i][j] / 36.0;
}

/* generic dense matrix-vector product, y = A x */
static void matvec(const double A[Q][Q], const double* x, double* y)
{
    for (int i = 0; i < Q; ++i) {
        double s = 0.0;
        for (int j = 0; j < Q; ++j) s += A[i][j] * x[j];
        y[i] = s;
    }
}

/* f = M^-1 m with the printed inverse (A1) applied as its integer matrix followed by
 * one division by the common factor 36. Multiplying by rounded entries such as 4/36
 * instead would scale the mass sum_i f_i = m_0 by 9 * fl(1/9) != 1 on every step,
 * a steady drift of the quantity the step conserves exactly (S_0 = C_0 = 0). */
static void apply_minv(const double* m, double* f)
{
    for (int i = 0; i < Q; ++i) {
        double s = 0.0;
        for (int j = 0; j < Q; ++j) s += MINV36_TAB[i][j] * m[j];
        f[i] = s / 36.0;
    }
}

/* m = M f, Eq. (17) */
void vo_moments(const double* f, double* m)
{
    matvec(M_TAB, f, m);
}

/* ---------------------------------------------------------------- Eq. (14) */
void vo_feq_order(int order, double kappa, double phi, double rho, double ux, double uy, double* feq)
{
    int e[Q][2];
    double w[Q];
    vo_lattice(e, w);
    const double cs2 = 1.0 / 3.0;
    const double X = kappa / phi;
    const double uu = ux * ux + uy * uy;
    double sum_w_nonzero = 0.0;
    for (int i = 1; i < Q; ++i) sum_w_nonzero += w[i];
    feq[0] = phi * rho - sum_w_nonzero * kappa * rho - w[0] * phi * rho * uu / (2.0 * cs2);
    for (int i = 1; i < Q; ++i) {
        double eu = e[i][0] * ux + e[i][1] * uy;
        double ee = (double)(e[i][0] * e[i][0] + e[i][1] * e[i][1]);
        /* Eq. (14) adjusts the first-order term by X; Eq. (B1) keeps the plain one */
        double first = order == 2 ? eu / cs2 : eu / cs2 * (1.0 + 0.5 * (X - 1.0) * (ee / cs2 - 4.0));
        double second = eu * eu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2);
        feq[i] = w[i] * (kappa * rho + phi * rho * (first + second));
    }
}

void vo_feq(double kappa, double phi, double rho, double ux, double uy, double* feq)
{
    vo_feq_order(3, kappa, phi, rho, ux, uy, feq);
}

/* ----------------------------------------------------------------- Eq. (6) */
void vo_guo_force(double ux, double uy, double Fx, double Fy, double* Fi)
{
    int e[Q][2];
    double w[Q];
    vo_lattice(e, w);
    const double cs2 = 1.0 / 3.0;
    for (int i = 0; i < Q; ++i) {
        double eu = e[i][0] * ux + e[i][1] * uy;
        double cx = (e[i][0] - ux) / cs2 + eu / (cs2 * cs2) * e[i][0];
        double cy = (e[i][1] - uy) / cs2 + eu / (cs2 * cs2) * e[i][1];
        Fi[i] = w[i] * (cx * Fx + cy * Fy);
    }
}

/* ---------------------------------------------------------------- Eq. (18) */
void vo_meq_order(int order, double kappa, double phi, double rho, double ux, double uy, double* meq)
{
    const double X = kappa / phi;
    const double pr = phi * rho;
    const double uu = ux * ux + uy * uy;
    meq[0] = pr;
    meq[1] = pr * (-4.0 + 3.0 * uu + 2.0 * X);
    meq[2] = pr * (4.0 - 3.0 * uu - 3.0 * X);
    meq[3] = pr * ux;
    /* Eq. (18): (X - 2) on the energy fluxes; Eq. (B2): -1 */
    const double qf = order == 2 ? -1.0 : (X - 2.0);
    meq[4] = pr * qf * ux;
    meq[5] = pr * uy;
    meq[6] = pr * qf * uy;
    meq[7] = pr * (ux * ux - uy * uy);
    meq[8] = pr * ux * uy;
}

void vo_meq(double kappa, double phi, double rho, double ux, double uy, double* meq)
{
    vo_meq_order(3, kappa, phi, rho, ux, uy, meq);
}

/* ---------------------------------------------------------------- Eq. (19) */
void vo_force_moments(double ux, double uy, double Fx, double Fy, double* S)
{
    const double uF = ux * Fx + uy * Fy;
    S[0] = 0.0;
    S[1] = 6.0 * uF;
    S[2] = -6.0 * uF;
    S[3] = Fx;
    S[4] = -Fx;
    S[5] = Fy;
    S[6] = -Fy;
    S[7] = 2.0 * (ux * Fx - uy * Fy);
    S[8] = ux * Fy + uy * Fx;
}

/*
 * ---------------------------------------------------------------- Eq. (20)
 * dA, dB, dD hold the four derivatives (d_x X_x, d_y X_y, d_x X_y, d_y X_x) of
 * A = rho u, B = u and D = phi rho u; dtphi = phi(t+1) - phi(t).
 * Model B (Sec. 2.3): every "kappa - phi" factor becomes "kappa - 1".
 * C is returned as the 9-vector (0, C_a, 0, 0, 0, 0, 0, C_b, C_c).
 */
void vo_penalty_order(int order, double kappa, double phi, double rho, const double* dA, const double* dB,
                      const double* dD, double dtphi, int model_b, double* C)
{
    const double X = kappa / phi;
    const double kp = model_b ? (kappa - 1.0) : (kappa - phi);
    const double divA = dA[0] + dA[1], difA = dA[0] - dA[1];
    const double divB = dB[0] + dB[1], difB = dB[0] - dB[1];
    const double crsB = dB[2] + dB[3];
    const double divD = dD[0] + dD[1], difD = dD[0] - dD[1];
    double Ca, Cb, Cc;
    if (order == 2) {
        /* Eq. (B3) */
        const double crsA = dA[2] + dA[3], crsD = dD[2] + dD[3];
        Ca = -2.0 * kappa * divA + 2.0 * kp * rho * divB + (4.0 - 2.0 * X) * divD - 2.0 * X * rho * dtphi;
        Cb = -(2.0 / 3.0) * kappa * difA + (2.0 / 3.0) * kp * rho * difB + (2.0 / 3.0) * difD;
        Cc = -(kappa / 3.0) * crsA + (1.0 / 3.0) * kp * rho * crsB + (1.0 / 3.0) * crsD;
    } else {
        Ca = -kappa * divA + 2.0 * kp * rho * divB + (3.0 - 2.0 * X) * divD - 2.0 * X * rho * dtphi;
        Cb = -kappa * difA + (2.0 / 3.0) * kp * rho * difB + difD;
        Cc = (1.0 / 3.0) * kp * rho * crsB;
    }
    for (int k = 0; k < Q; ++k) C[k] = 0.0;
    C[1] = Ca;
    C[7] = Cb;
    C[8] = Cc;
}

void vo_penalty(double kappa, double phi, double rho, const double* dA, const double* dB,
                const double* dD, double dtphi, int model_b, double* C)
{
    vo_penalty_order(3, kappa, phi, rho, dA, dB, dD, dtphi, model_b, C);
}

/* --------------------------------------------------------- neighbour rule */
/*
 * Returns the cell that stands for (x, y) (possibly outside the domain) and the
 * sign a vector field takes there. Periodic axes wrap. On a wall axis the ghost
 * cell is the mirror image about the half-way wall: -1 -> 0, -2 -> 1, n -> n-1,
 * and a vector field takes the negated mirror value (sign -1) whenever at least
 * one wall was crossed.
 */
static int neighbour(const vo_params* p, int x, int y, int* sign)
{
    int wall = 0;
    if (x < 0 || x >= p->nx) {
        if (p->bc_x == 0) {
            x = ((x % p->nx) + p->nx) % p->nx;
        } else {
            x = (x < 0) ? (-1 - x) : (2 * p->nx - 1 - x);
            wall = 1;
        }
    }
    if (y < 0 || y >= p->ny) {
        if (p->bc_y == 0) {
            y = ((y % p->ny) + p->ny) % p->ny;
        } else {
            y = (y < 0) ? (-1 - y) : (2 * p->ny - 1 - y);
            wall = 1;
        }
    }
    *sign = wall ? -1 : 1;
    return y * p->nx + x;
}

/*
 * ---------------------------------------------------------------- Eq. (10)
 * d_alpha psi(x) = (1/cs^2) sum_i w_i psi(x + e_i) e_{i alpha}.
 * odd = 1 for a vector-field component (negated in a wall ghost cell),
 * odd = 0 for a scalar (copied).
 */
/*
 * Solid cells (phi = 0, the impermeable block of Sec. 3.3 with phi_0 = 0) are not
 * part of the fluid. Their links are half-way bounce-back links (stream below); in
 * the Eq. (10) stencil of a fluid cell x a solid neighbour x + e_i reads a ghost
 * value mirrored about the solid surface, the rule of the straight walls above
 * applied link by link (the paper is silent):
 *   - an axis neighbour mirrors onto x itself;
 *   - a diagonal neighbour mirrors onto x + (e_ix, 0) and onto x + (0, e_iy); the
 *     fluid ones of these two are averaged (a straight wall leaves exactly the one
 *     the wall rule uses); if both are solid it mirrors onto x;
 *   - a vector-field component takes the negated mirror value (no-slip).
 */
static double solid_ghost(const vo_params* p, const double* psi, const double* phi, int odd, int x, int y,
                          int ex, int ey)
{
    const double sg = odd ? -1.0 : 1.0;
    if (ex == 0 || ey == 0) return sg * psi[(size_t)y * p->nx + x];
    double acc = 0.0;
    int n = 0;
    int sa, sb;
    const int a = neighbour(p, x + ex, y, &sa);
    const int b = neighbour(p, x, y + ey, &sb);
    if (phi[a] != 0.0) { acc += (odd && sa < 0) ? -psi[a] : psi[a]; ++n; }
    if (phi[b] != 0.0) { acc += (odd && sb < 0) ? -psi[b] : psi[b]; ++n; }
    if (n == 0) return sg * psi[(size_t)y * p->nx + x];
    return sg * (acc / n);
}

/* Eq. (10) with solid cells (phi[c] = 0) treated by solid_ghost; phi may be NULL (no
 * solid cells). The gradient at a solid cell is set to zero (never used). */
static void gradient_masked(const vo_params* p, const double* psi, int odd, const double* phi, double* gx,
                            double* gy);

void vo_gradient(const vo_params* p, const double* psi, int odd, double* gx, double* gy)
{
    gradient_masked(p, psi, odd, NULL, gx, gy);
}

static void gradient_masked(const vo_params* p, const double* psi, int odd, const double* phi, double* gx,
                            double* gy)
{
    int e[Q][2];
    double w[Q];
    vo_lattice(e, w);
    const double cs2 = 1.0 / 3.0;
    const int nx = p->nx, ny = p->ny;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (p->nthreads != 1) num_threads(p->nthreads > 0 ? p->nthreads : omp_get_max_threads())
#endif
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            double sx = 0.0, sy = 0.0;
            if (phi && phi[(size_t)y * nx + x] == 0.0) {
                gx[y * nx + x] = 0.0;
                gy[y * nx + x] = 0.0;
                continue;
            }
            for (int i = 0; i < Q; ++i) {
                double v;
                int sn;
                const int cn = neighbour(p, x + e[i][0], y + e[i][1], &sn);
                if (phi && phi[cn] == 0.0 && !(p->nee_top && y + e[i][1] == ny)) {
                    v = solid_ghost(p, psi, phi, odd, x, y, e[i][0], e[i][1]);
                } else if (p->nee_top && y + e[i][1] == ny) {
                    /* past the NEE wall row: linear extrapolation from rows ny-1, ny-2 */
                    int s1, s2;
                    const int c1 = neighbour(p, x + e[i][0], ny - 1, &s1);
                    const int c2 = neighbour(p, x + e[i][0], ny - 2, &s2);
                    v = 2.0 * psi[c1] - psi[c2];
                } else {
                    int sgn;
                    int c = neighbour(p, x + e[i][0], y + e[i][1], &sgn);
                    v = psi[c];
                    if (odd && sgn < 0) v = -v;
                }
                sx += w[i] * v * e[i][0];
                sy += w[i] * v * e[i][1];
            }
            gx[y * nx + x] = sx / cs2;
            gy[y * nx + x] = sy / cs2;
        }
    }
}

/*
 * Eq. (7) at one cell c of the post-streaming populations f (N cells per plane),
 * given the Eq. (10) gradient of rho there and the prescribed part of F^B:
 * F = F^p + F^B with F^p = (kappa - phi) cs^2 grad rho (model B: kappa - 1);
 * a drag -beta (u - u_s) in F makes Eq. (7) implicit in u, and being linear it
 * is solved exactly: u (sum f + beta / 2) = j + (F_rest + beta u_s) / 2.
 */
static void cell_velocity(const vo_params* p, const double* f, size_t N, size_t c, double phi, double grx,
                          double gry, double fbx, double fby, double* ux, double* uy, double* Fx, double* Fy)
{
    static const int ex[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    static const int ey[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const double cs2 = 1.0 / 3.0;
    double s = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < Q; ++i) {
        s += f[i * N + c];
        jx += ex[i] * f[i * N + c];
        jy += ey[i] * f[i * N + c];
    }
    const double kp = p->model_b ? (p->kappa - 1.0) : (p->kappa - phi);
    double fx = kp * cs2 * grx + fbx;
    double fy = kp * cs2 * gry + fby;
    const double beta = phi * phi * (p->drag_d0 + p->drag_d1 * (1.0 - phi));
    const double vx = (jx + 0.5 * (fx + beta * p->us_x)) / (s + 0.5 * beta);
    const double vy = (jy + 0.5 * (fy + beta * p->us_y)) / (s + 0.5 * beta);
    fx -= beta * (vx - p->us_x);
    fy -= beta * (vy - p->us_y);
    *ux = vx;
    *uy = vy;
    *Fx = fx;
    *Fy = fy;
}

/*
 * ----------------------------------------------------------- Eq. (7), (13)
 * From post-streaming populations f at time t: rho = sum f / phi,
 * F = F^p + F^B with F^p = (kappa - phi) cs^2 grad rho (model B: kappa - 1),
 * u = (sum e f + F/2) / sum f. Any output pointer may be NULL except rho.
 */
void vo_macros(const vo_params* p, const double* f, const double* phi, const double* fb,
               double* rho, double* ux, double* uy, double* Fx, double* Fy)
{
    const size_t N = (size_t)p->nx * p->ny;
    double* gx = (double*)malloc(N * sizeof(double));
    double* gy = (double*)malloc(N * sizeof(double));
    for (size_t c = 0; c < N; ++c) {
        double s = 0.0;
        for (int i = 0; i < Q; ++i) s += f[i * N + c];
        rho[c] = phi[c] != 0.0 ? s / phi[c] : 0.0;   /* solid cells report zeros */
    }
    gradient_masked(p, rho, 0, phi, gx, gy);
    for (size_t c = 0; c < N; ++c) {
        double vx, vy, fx, fy;
        if (phi[c] == 0.0) {
            if (ux) ux[c] = 0.0;
            if (uy) uy[c] = 0.0;
            if (Fx) Fx[c] = 0.0;
            if (Fy) Fy[c] = 0.0;
            continue;
        }
        cell_velocity(p, f, N, c, phi[c], gx[c], gy[c], fb ? fb[c] : 0.0, fb ? fb[N + c] : 0.0, &vx, &vy, &fx, &fy);
        if (ux) ux[c] = vx;
        if (uy) uy[c] = vy;
        if (Fx) Fx[c] = fx;
        if (Fy) Fy[c] = fy;
    }
    free(gx);
    free(gy);
}

/*
 * Moving wall by non-equilibrium extrapolation (Sec. 3.1; the scheme of the paper's
 * reference [47], Guo, Zheng and Shi). Readings where the paper is silent:
 *   - the wall nodes are the top row y = ny-1 (the wall passes through them); the
 *     fluid node next to each is (x, ny-2); the bottom stays a half-way bounce-back
 *     wall, so the channel height is H = ny - 1/2;
 *   - before the collision of each step, every population of a wall node is
 *     replaced by f_i = f_i^eq(rho_b, u_w, phi_b) + f_i(x_f) - f_i^eq(rho_f, u_f, phi_f)
 *     with rho_b = rho_f (extrapolated density) and f^eq of Eq. (14) (Eq. B1 when
 *     eq_order = 2);
 *   - u_f is Eq. (7) at the fluid node, with F^p from the Eq. (10) gradient of rho
 *     that already uses rho_b in the wall row, and the drag solved implicitly;
 *   - the Eq. (10) stencil of a wall node reads a ghost row above the wall that
 *     extrapolates linearly from rows ny-1 and ny-2 (every field; vo_gradient);
 *   - the wall node then collides like a fluid node; what it streams upward is
 *     replaced again at the next step.
 * f_out = f with the wall row replaced (f itself unchanged).
 */
static void nee_fill(const vo_params* p, const double* f, const double* phi, const double* fb, double* f_out)
{
    const int nx = p->nx, ny = p->ny;
    const size_t N = (size_t)nx * ny;
    double* rho = (double*)malloc(N * sizeof(double));
    double* gx = (double*)malloc(N * sizeof(double));
    double* gy = (double*)malloc(N * sizeof(double));
    memcpy(f_out, f, Q * N * sizeof(double));
    for (size_t c = 0; c < N; ++c) {
        double s = 0.0;
        for (int i = 0; i < Q; ++i) s += f[i * N + c];
        rho[c] = phi[c] != 0.0 ? s / phi[c] : 0.0;
    }
    for (int x = 0; x < nx; ++x) rho[(size_t)(ny - 1) * nx + x] = rho[(size_t)(ny - 2) * nx + x];
    gradient_masked(p, rho, 0, phi, gx, gy);
    for (int x = 0; x < nx; ++x) {
        const size_t cf = (size_t)(ny - 2) * nx + x, cb = (size_t)(ny - 1) * nx + x;
        double vx, vy, fx, fy;
        cell_velocity(p, f, N, cf, phi[cf], gx[cf], gy[cf], fb ? fb[cf] : 0.0, fb ? fb[N + cf] : 0.0,
                      &vx, &vy, &fx, &fy);
        double eb[Q], ef[Q];
        vo_feq_order(p->eq_order, p->kappa, phi[cb], rho[cf], p->uw_x, p->uw_y, eb);
        vo_feq_order(p->eq_order, p->kappa, phi[cf], rho[cf], vx, vy, ef);
        for (int i = 0; i < Q; ++i) f_out[i * N + cb] = eb[i] + (f[i * N + cf] - ef[i]);
    }
    free(rho);
    free(gx);
    free(gy);
}

static int opposite(int i)
{
    static const int opp[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    return opp[i];
}

/*
 * Streaming f_i(x + e_i, t+1) = f_i^+(x, t) with periodic wrap; a link that
 * leaves the fluid through a half-way bounce-back wall returns to the same cell
 * in the opposite direction (Sec. 3.1).
 */
static void stream(const vo_params* p, const double* fplus, double* fout, const double* phi)
{
    int e[Q][2];
    double w[Q];
    vo_lattice(e, w);
    const int nx = p->nx, ny = p->ny;
    const size_t N = (size_t)nx * ny;
    /* a solid cell (phi = 0) neither sends nor receives: its populations stay zero,
     * and a fluid link into it bounces back half-way like a wall link */
    memset(fout, 0, Q * N * sizeof(double));
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            if (phi[(size_t)y * nx + x] == 0.0) continue;
            for (int i = 0; i < Q; ++i) {
                int xd = x + e[i][0], yd = y + e[i][1];
                int wall = 0;
                if (xd < 0 || xd >= nx) {
                    if (p->bc_x == 0) xd = (xd + nx) % nx; else wall = 1;
                }
                if (yd < 0 || yd >= ny) {
                    if (p->bc_y == 0) yd = (yd + ny) % ny; else wall = 1;
                }
                if (!wall && phi[(size_t)yd * nx + xd] == 0.0) wall = 1;
                double v = fplus[i * N + (size_t)y * nx + x];
                if (wall)
                    fout[opposite(i) * N + (size_t)y * nx + x] = v;
                else
                    fout[i * N + (size_t)yd * nx + xd] = v;
            }
        }
    }
}

/*
 * --------------------------------------------------- one step, Eq. (16)
 * f: post-streaming populations at t. phi_t, phi_next: phi(x,t), phi(x,t+1)
 * (phi_next may be NULL for a steady field). fb: F^B(x,t) or NULL.
 * f_new receives the post-streaming populations at t+1 (must not alias f).
 * Returns 0.
 */
int vo_step(const vo_params* p, const double* f, double* f_new, const double* phi_t,
            const double* phi_next, const double* fb)
{
    const size_t N = (size_t)p->nx * p->ny;
    const double kappa = p->kappa;
    const double G[Q] = {p->s_c, p->s_e, p->s_eps, p->s_c, p->s_q, p->s_c, p->s_q, p->s_nu, p->s_nu};
    double* rho = (double*)malloc(N * sizeof(double));
    double* ux = (double*)malloc(N * sizeof(double));
    double* uy = (double*)malloc(N * sizeof(double));
    double* Fx = (double*)malloc(N * sizeof(double));
    double* Fy = (double*)malloc(N * sizeof(double));
    /* fields whose Eq. (10) gradients enter Eq. (20): A = rho u, B = u, D = phi rho u */
    double* fld = (double*)malloc(6 * N * sizeof(double));
    double* grd = (double*)malloc(12 * N * sizeof(double));
    double* fplus = (double*)malloc(Q * N * sizeof(double));
    double* fnee = NULL;
    if (p->nee_top && p->bc_y == 1 && p->ny >= 3) {
        /* the moving wall's populations, before anything reads them */
        fnee = (double*)malloc(Q * N * sizeof(double));
        nee_fill(p, f, phi_t, fb, fnee);
        f = fnee;
    }

    /* steps 1-3: rho, F, u (Eq. 7, 10, 13) */
    vo_macros(p, f, phi_t, fb, rho, ux, uy, Fx, Fy);

    /* step 4: the penalty-source fields and their gradients */
    for (size_t c = 0; c < N; ++c) {
        fld[0 * N + c] = rho[c] * ux[c];
        fld[1 * N + c] = rho[c] * uy[c];
        fld[2 * N + c] = ux[c];
        fld[3 * N + c] = uy[c];
        fld[4 * N + c] = phi_t[c] * rho[c] * ux[c];
        fld[5 * N + c] = phi_t[c] * rho[c] * uy[c];
    }
    for (int k = 0; k < 6; ++k)
        gradient_masked(p, fld + k * N, 1, phi_t, grd + (2 * k) * N, grd + (2 * k + 1) * N);

    /* steps 5-6: moments, relaxation (Eq. 16), back-transform (A1) */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (p->nthreads != 1) num_threads(p->nthreads > 0 ? p->nthreads : omp_get_max_threads())
#endif
    for (long long cc = 0; cc < (long long)N; ++cc) {
        const size_t c = (size_t)cc;
        double fc[Q], m[Q], meq[Q], S[Q], C[Q], mp[Q], fp[Q];
        if (phi_t[c] == 0.0) {   /* solid cell: nothing to collide */
            for (int i = 0; i < Q; ++i) fplus[i * N + c] = 0.0;
            continue;
        }
        for (int i = 0; i < Q; ++i) fc[i] = f[i * N + c];
        vo_moments(fc, m);
        vo_meq_order(p->eq_order, kappa, phi_t[c], rho[c], ux[c], uy[c], meq);
        vo_force_moments(ux[c], uy[c], Fx[c], Fy[c], S);
        /* derivative sets (d_x X_x, d_y X_y, d_x X_y, d_y X_x) */
        const double dA[4] = {grd[0 * N + c], grd[3 * N + c], grd[2 * N + c], grd[1 * N + c]};
        const double dB[4] = {grd[4 * N + c], grd[7 * N + c], grd[6 * N + c], grd[5 * N + c]};
        const double dD[4] = {grd[8 * N + c], grd[11 * N + c], grd[10 * N + c], grd[9 * N + c]};
        const double dtphi = phi_next ? (phi_next[c] - phi_t[c]) : 0.0;
        vo_penalty_order(p->eq_order, kappa, phi_t[c], rho[c], dA, dB, dD, dtphi, p->model_b, C);
        for (int k = 0; k < Q; ++k)
            mp[k] = m[k] - G[k] * (m[k] - meq[k]) + (1.0 - 0.5 * G[k]) * (S[k] + C[k]);
        apply_minv(mp, fp);
        for (int i = 0; i < Q; ++i) fplus[i * N + c] = fp[i];
    }

    /* step 7: streaming and bounce-back */
    stream(p, fplus, f_new, phi_t);

    free(rho); free(ux); free(uy); free(Fx); free(Fy);
    free(fld); free(grd); free(fplus);
    free(fnee);
    return 0;
}

/*
 * Initial populations (reading c7): f = f^eq(rho, u, phi) - F_i(u, F)/2 with
 * F = F^p + F^B and F^p from the given rho (Eq. 13). With these, Eq. (7)
 * returns exactly the given u.
 */
void vo_init(const vo_params* p, const double* rho, const double* ux, const double* uy,
             const double* phi, const double* fb, double* f)
{
    const size_t N = (size_t)p->nx * p->ny;
    const double cs2 = 1.0 / 3.0;
    double* gx = (double*)malloc(N * sizeof(double));
    double* gy = (double*)malloc(N * sizeof(double));
    gradient_masked(p, rho, 0, phi, gx, gy);
    for (size_t c = 0; c < N; ++c) {
        double feq[Q], Fi[Q];
        if (phi[c] == 0.0) {   /* solid cell */
            for (int i = 0; i < Q; ++i) f[i * N + c] = 0.0;
            continue;
        }
        const double kp = p->model_b ? (p->kappa - 1.0) : (p->kappa - phi[c]);
        const double beta = phi[c] * phi[c] * (p->drag_d0 + p->drag_d1 * (1.0 - phi[c]));
        const double fx = kp * cs2 * gx[c] + (fb ? fb[c] : 0.0) - beta * (ux[c] - p->us_x);
        const double fy = kp * cs2 * gy[c] + (fb ? fb[N + c] : 0.0) - beta * (uy[c] - p->us_y);
        vo_feq_order(p->eq_order, p->kappa, phi[c], rho[c], ux[c], uy[c], feq);
        vo_guo_force(ux[c], uy[c], fx, fy, Fi);
        for (int i = 0; i < Q; ++i) f[i * N + c] = feq[i] - 0.5 * Fi[i];
    }
    free(gx);
    free(gy);
}

/* number of OpenMP threads a parallel region would use (1 without OpenMP) */
int vo_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
