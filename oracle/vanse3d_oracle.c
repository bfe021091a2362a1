/*
 * vanse3d_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of one time step of the MRTLB-VANSE scheme
 * (arXiv:2409.02964) carried to three dimensions on the D3Q19 lattice, the
 * extension Sec. 4 names as future work. Lattice units (dx = dt = c = 1,
 * cs^2 = 1/3). Only the tests and the smoke check load this code; it shares no
 * source, header, table or helper with the CUDA library.
 *
 * The paper gives the scheme in 2-D only. The 3-D scheme here keeps each of its
 * ingredients and the properties the paper derives them from:
 *   v3_lattice     D3Q19 velocities and weights (Eq. (5)'s role in 3-D)
 *   v3_M           the D3Q19 moment basis of d'Humieres et al. (2002): rho, e, eps,
 *                  (j, q) per axis, 3p_xx, 3pi_xx, p_ww, pi_ww, p_xy, p_yz, p_xz,
 *                  m_x, m_y, m_z, each row the polynomial of its definition
 *                  evaluated on the velocities (Eq. (17)'s role); its inverse is
 *                  M^T diag(1/|row|^2), the rows being orthogonal
 *   v3_meq         equilibrium moments chosen so that the velocity moments of
 *                  f^eq are those of Eq. (15): sum f = phi rho, sum e f = phi rho u,
 *                  sum e e f = phi rho u u + kappa rho cs^2 I, the third moment
 *                  kappa rho cs^2 (u d + ...) in every component the lattice can
 *                  hold apart from e_a^3 = e_a (there it stays phi rho u_a, as in
 *                  2-D): e^eq = 19 (kappa rho + phi rho |u|^2) - 30 phi rho,
 *                  q^eq = (10 X / 3 - 4) phi rho u, the second-order (stress)
 *                  moments phi rho u u, and the fourth-order ghosts those of the
 *                  second-order Hermite equilibrium with the adjusted rest state of
 *                  Eq. (14) (eps^eq = 12 phi rho - 9 kappa rho - 11/2 phi rho |u|^2,
 *                  pi^eq = -p^eq / 2, m^eq = 0); with phi = kappa these are the
 *                  standard D3Q19 equilibria
 *   v3_guo_force   Eq. (6) in 3-D; v3_force_moments = M F (Eq. (19)'s role)
 *   v3_penalty     the penalty source of Eq. (16), derived for D3Q19 by the
 *                  Chapman-Enskog bookkeeping of App. A: for every stress moment the
 *                  first-order non-equilibrium of the scheme minus that of the target
 *                  stress cs^2 phi rho (grad u + grad u^T), with d_t rho replaced as
 *                  App. A does. Trace (e):
 *                    C_e = 19 [(1 - X) div(phi rho u) - X rho d_t phi
 *                              + 2/3 (kappa - phi) rho div u]
 *                  traceless diagonal moments sum_a w_a e_a^2 (w = (2,-1,-1) for
 *                  3p_xx, (0,1,-1) for p_ww), the C_b form of Eq. (20):
 *                    sum_a w_a [-kappa d_a(rho u_a) + 2/3 (kappa - phi) rho d_a u_a
 *                               + d_a(phi rho u_a)]
 *                  off-diagonal moments p_ab, the C_c form of Eq. (20):
 *                    1/3 (kappa - phi) rho (d_a u_b + d_b u_a)
 *   v3_gradient    Eq. (10) with the D3Q19 weights: grad psi = 3 sum_i w_i psi(x+e_i) e_i
 *   v3_macros      Eq. (7), (13)
 *   v3_step        Eq. (16) + streaming + half-way bounce-back walls in y
 *   v3_init        f = f^eq - F_i / 2 (as in 2-D)
 *
 * The scheme recovers Eq. (A12) in 3-D with the viscous stress
 *   tau = rho nu (grad u + grad u^T - 2/3 div u I) + 2/3 rho nu_e div u I,
 * nu = cs^2 (1/s_nu - 1/2), nu_e = cs^2 (1/s_e - 1/2): the Stokes form of Eq. (1)
 * needs nu_e = 0 (s_e = 2), the 3-D counterpart of nu_e = nu/3 in 2-D.
 *
 * Readings as in 2-D: rates are the diagonal of Gamma; relaxation is
 * m - Gamma (m - m^eq); rho and X use phi(x,t); d_t phi = phi(x,t+1) - phi(x,t);
 * next to a wall the gradient stencil reads a ghost cell mirrored about the wall
 * (scalars keep the mirror value, vector components change sign).
 *
 * Parity pins (tests/test_oracle_d3q19.py): lattice isotropy; the rows of M
 * against their polynomials (recomputed in the test), M M^-1 = I; the velocity
 * moments of f^eq summed by brute force; the moments of F_i; reduction to a
 * textbook D3Q19 BGK with Guo forcing when phi = kappa and all rates are equal;
 * the rest-state fixed point; mass and momentum balance; and second-order
 * convergence on a 3-D manufactured solution with a moving phi.
 *
 * Array layout: fields [nz][ny][nx]; populations [19][nz][ny][nx]; body force
 * [3][nz][ny][nx]. Cell (x, y, z) has index (z*ny + y)*nx + x.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q3 19

typedef struct {
    int nx, ny, nz;
    double s_c, s_e, s_eps, s_q, s_nu, s_pi, s_m;
    double kappa;
    int bc_y;       /* 0 periodic, 1 half-way bounce-back walls at y = -1/2 and ny - 1/2 */
    int nthreads;
    int no_penalty; /* tests only: leave the penalty source out (a planted mistake) */
} V3Params;

static const int E3[Q3][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double w3(int i) {
    if (i == 0) return 1.0 / 3.0;
    return i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0;
}

static int opposite3(int i) {
    for (int k = 0; k < Q3; ++k)
        if (E3[k][0] == -E3[i][0] && E3[k][1] == -E3[i][1] && E3[k][2] == -E3[i][2]) return k;
    return -1;
}

void v3_lattice(int* e, double* w) {
    for (int i = 0; i < Q3; ++i) {
        for (int a = 0; a < 3; ++a) e[3 * i + a] = E3[i][a];
        w[i] = w3(i);
    }
}

/* the basis polynomial of moment k at velocity (x, y, z) */
static double basis(int k, double x, double y, double z) {
    const double c2 = x * x + y * y + z * z;
    switch (k) {
        case 0: return 1.0;
        case 1: return 19.0 * c2 - 30.0;
        case 2: return (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0;
        case 3: return x;
        case 4: return (5.0 * c2 - 9.0) * x;
        case 5: return y;
        case 6: return (5.0 * c2 - 9.0) * y;
        case 7: return z;
        case 8: return (5.0 * c2 - 9.0) * z;
        case 9: return 3.0 * x * x - c2;
        case 10: return (3.0 * c2 - 5.0) * (3.0 * x * x - c2);
        case 11: return y * y - z * z;
        case 12: return (3.0 * c2 - 5.0) * (y * y - z * z);
        case 13: return x * y;
        case 14: return y * z;
        case 15: return x * z;
        case 16: return (y * y - z * z) * x;
        case 17: return (z * z - x * x) * y;
        case 18: return (x * x - y * y) * z;
    }
    return 0.0;
}

void v3_M(double* M) {
    for (int k = 0; k < Q3; ++k)
        for (int i = 0; i < Q3; ++i) M[k * Q3 + i] = basis(k, E3[i][0], E3[i][1], E3[i][2]);
}

/* M^-1 = M^T diag(1 / |row k|^2) (orthogonal rows) */
void v3_Minv(double* Mi) {
    double M[Q3 * Q3];
    v3_M(M);
    for (int k = 0; k < Q3; ++k) {
        double n2 = 0.0;
        for (int i = 0; i < Q3; ++i) n2 += M[k * Q3 + i] * M[k * Q3 + i];
        for (int i = 0; i < Q3; ++i) Mi[i * Q3 + k] = M[k * Q3 + i] / n2;
    }
}

/* both matrices, filled once (before any parallel loop) */
static double gM[Q3 * Q3], gMi[Q3 * Q3];
static int g_ready = 0;
static void tables(void) {
    if (g_ready) return;
    v3_M(gM);
    v3_Minv(gMi);
    g_ready = 1;
}

void v3_moments(const double* f, double* m) {
    tables();
    for (int k = 0; k < Q3; ++k) {
        double s = 0.0;
        for (int i = 0; i < Q3; ++i) s += gM[k * Q3 + i] * f[i];
        m[k] = s;
    }
}

static void from_moments(const double* m, double* f) {
    tables();
    for (int i = 0; i < Q3; ++i) {
        double s = 0.0;
        for (int k = 0; k < Q3; ++k) s += gMi[i * Q3 + k] * m[k];
        f[i] = s;
    }
}

void v3_meq(double kappa, double phi, double rho, double ux, double uy, double uz, double* m) {
    const double m0 = phi * rho, X = kappa / phi;
    const double u2 = ux * ux + uy * uy + uz * uz;
    const double pxx3 = m0 * (3.0 * ux * ux - u2), pww = m0 * (uy * uy - uz * uz);
    const double qf = 10.0 * X / 3.0 - 4.0;
    m[0] = m0;
    m[1] = 19.0 * (kappa * rho + m0 * u2) - 30.0 * m0;
    m[2] = 12.0 * m0 - 9.0 * kappa * rho - 5.5 * m0 * u2;
    m[3] = m0 * ux;
    m[4] = qf * m0 * ux;
    m[5] = m0 * uy;
    m[6] = qf * m0 * uy;
    m[7] = m0 * uz;
    m[8] = qf * m0 * uz;
    m[9] = pxx3;
    m[10] = -0.5 * pxx3;
    m[11] = pww;
    m[12] = -0.5 * pww;
    m[13] = m0 * ux * uy;
    m[14] = m0 * uy * uz;
    m[15] = m0 * ux * uz;
    m[16] = 0.0;
    m[17] = 0.0;
    m[18] = 0.0;
}

void v3_feq(double kappa, double phi, double rho, double ux, double uy, double uz, double* f) {
    double m[Q3];
    v3_meq(kappa, phi, rho, ux, uy, uz, m);
    from_moments(m, f);
}

/* Eq. (6): F_i = w_i [(e_i - u)/cs^2 + (e_i . u) e_i / cs^4] . F */
void v3_guo_force(double ux, double uy, double uz, double Fx, double Fy, double Fz, double* Fi) {
    const double u[3] = {ux, uy, uz}, F[3] = {Fx, Fy, Fz};
    for (int i = 0; i < Q3; ++i) {
        double eu = 0.0;
        for (int a = 0; a < 3; ++a) eu += E3[i][a] * u[a];
        double s = 0.0;
        for (int a = 0; a < 3; ++a) s += (3.0 * (E3[i][a] - u[a]) + 9.0 * eu * E3[i][a]) * F[a];
        Fi[i] = w3(i) * s;
    }
}

void v3_force_moments(double ux, double uy, double uz, double Fx, double Fy, double Fz, double* S) {
    double Fi[Q3];
    v3_guo_force(ux, uy, uz, Fx, Fy, Fz, Fi);
    v3_moments(Fi, S);
}

/* dA[a] = d_a (rho u)_a, dD[a] = d_a (phi rho u)_a, dB[3a+b] = d_a u_b */
void v3_penalty(double kappa, double phi, double rho, const double* dA, const double* dB,
                const double* dD, double dtphi, double* C) {
    const double X = kappa / phi, kp = kappa - phi;
    for (int k = 0; k < Q3; ++k) C[k] = 0.0;
    const double divB = dB[0] + dB[4] + dB[8], divD = dD[0] + dD[1] + dD[2];
    C[1] = 19.0 * ((1.0 - X) * divD - X * rho * dtphi + (2.0 / 3.0) * kp * rho * divB);
    double diag[3];
    for (int a = 0; a < 3; ++a) diag[a] = -kappa * dA[a] + (2.0 / 3.0) * kp * rho * dB[4 * a] + dD[a];
    C[9] = 2.0 * diag[0] - diag[1] - diag[2];
    C[11] = diag[1] - diag[2];
    C[13] = kp * rho * (dB[1] + dB[3]) / 3.0;   /* x, y */
    C[14] = kp * rho * (dB[5] + dB[7]) / 3.0;   /* y, z */
    C[15] = kp * rho * (dB[2] + dB[6]) / 3.0;   /* x, z */
}

/* ------------------------------------------------------------------ fields */
static long long cell3(const V3Params* p, int x, int y, int z) {
    return ((long long)z * p->ny + y) * p->nx + x;
}

static int wrap(int v, int n) { return ((v % n) + n) % n; }

/* value of a field at (x, y, z) with periodic x, z; in y periodic or, with walls,
 * the ghost mirrored about the half-way wall (sign for vector components) */
static double field_at(const V3Params* p, const double* psi, int x, int y, int z, int odd) {
    x = wrap(x, p->nx);
    z = wrap(z, p->nz);
    double sgn = 1.0;
    if (p->bc_y == 0) {
        y = wrap(y, p->ny);
    } else {
        if (y < 0) { y = -1 - y; sgn = odd ? -1.0 : 1.0; }
        else if (y >= p->ny) { y = 2 * p->ny - 1 - y; sgn = odd ? -1.0 : 1.0; }
    }
    return sgn * psi[cell3(p, x, y, z)];
}

void v3_gradient(const V3Params* p, const double* psi, int odd, double* gx, double* gy, double* gz) {
#ifdef _OPENMP
#pragma omp parallel for num_threads(p->nthreads > 0 ? p->nthreads : 1)
#endif
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                double g[3] = {0.0, 0.0, 0.0};
                for (int i = 1; i < Q3; ++i) {
                    const double v = field_at(p, psi, x + E3[i][0], y + E3[i][1], z + E3[i][2], odd);
                    for (int a = 0; a < 3; ++a) g[a] += 3.0 * w3(i) * v * E3[i][a];
                }
                const long long c = cell3(p, x, y, z);
                gx[c] = g[0];
                gy[c] = g[1];
                gz[c] = g[2];
            }
}

/* Eq. (7), (13): rho, F = F^p + F^B, u (arrays of N; F and u as [3][N]) */
void v3_macros(const V3Params* p, const double* f, const double* phi, const double* fb, double* rho,
               double* F, double* u) {
    const long long N = (long long)p->nx * p->ny * p->nz;
    double* m0 = (double*)malloc(sizeof(double) * N);
    for (long long c = 0; c < N; ++c) {
        double s = 0.0;
        for (int i = 0; i < Q3; ++i) s += f[i * N + c];
        m0[c] = s;
        rho[c] = s / phi[c];
    }
    double* g = (double*)malloc(sizeof(double) * 3 * N);
    v3_gradient(p, rho, 0, g, g + N, g + 2 * N);
    for (long long c = 0; c < N; ++c) {
        double j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q3; ++i)
            for (int a = 0; a < 3; ++a) j[a] += E3[i][a] * f[i * N + c];
        for (int a = 0; a < 3; ++a) {
            const double Fa = (p->kappa - phi[c]) / 3.0 * g[a * N + c] + (fb ? fb[a * N + c] : 0.0);
            F[a * N + c] = Fa;
            u[a * N + c] = (j[a] + 0.5 * Fa) / m0[c];
        }
    }
    free(g);
    free(m0);
}

/* one step: f (post-streaming at t) -> out (post-streaming at t+1) */
int v3_step(const V3Params* p, const double* f, double* out, const double* phi_t, const double* phi_next,
            const double* fb) {
    const long long N = (long long)p->nx * p->ny * p->nz;
    double* rho = (double*)malloc(sizeof(double) * N);
    double* F = (double*)malloc(sizeof(double) * 3 * N);
    double* u = (double*)malloc(sizeof(double) * 3 * N);
    v3_macros(p, f, phi_t, fb, rho, F, u);
    /* fields A = rho u, B = u, D = phi rho u and their gradients */
    double* fld = (double*)malloc(sizeof(double) * 9 * N);
    double* grd = (double*)malloc(sizeof(double) * 27 * N);
    for (long long c = 0; c < N; ++c)
        for (int a = 0; a < 3; ++a) {
            fld[(0 + a) * N + c] = rho[c] * u[a * N + c];
            fld[(3 + a) * N + c] = u[a * N + c];
            fld[(6 + a) * N + c] = phi_t[c] * rho[c] * u[a * N + c];
        }
    for (int k = 0; k < 9; ++k)   /* grd[(3k + a) N + c] = d_a field_k */
        v3_gradient(p, fld + k * N, 1, grd + (3 * k) * N, grd + (3 * k + 1) * N, grd + (3 * k + 2) * N);
    const double G[Q3] = {p->s_c, p->s_e, p->s_eps, p->s_c, p->s_q, p->s_c, p->s_q, p->s_c, p->s_q,
                          p->s_nu, p->s_pi, p->s_nu, p->s_pi, p->s_nu, p->s_nu, p->s_nu,
                          p->s_m, p->s_m, p->s_m};
    double* post = (double*)malloc(sizeof(double) * Q3 * N);
    tables();
#ifdef _OPENMP
#pragma omp parallel for num_threads(p->nthreads > 0 ? p->nthreads : 1)
#endif
    for (long long c = 0; c < N; ++c) {
        double fc[Q3], m[Q3], meq[Q3], S[Q3], C[Q3], fp[Q3];
        for (int i = 0; i < Q3; ++i) fc[i] = f[i * N + c];
        v3_moments(fc, m);
        const double ux = u[c], uy = u[N + c], uz = u[2 * N + c];
        v3_meq(p->kappa, phi_t[c], rho[c], ux, uy, uz, meq);
        v3_force_moments(ux, uy, uz, F[c], F[N + c], F[2 * N + c], S);
        double dA[3], dB[9], dD[3];
        for (int a = 0; a < 3; ++a) {
            dA[a] = grd[(3 * a + a) * N + c];            /* d_a (rho u)_a */
            dD[a] = grd[(3 * (6 + a) + a) * N + c];      /* d_a (phi rho u)_a */
            for (int b = 0; b < 3; ++b) dB[3 * a + b] = grd[(3 * (3 + b) + a) * N + c];   /* d_a u_b */
        }
        const double dtphi = phi_next ? phi_next[c] - phi_t[c] : 0.0;
        v3_penalty(p->kappa, phi_t[c], rho[c], dA, dB, dD, dtphi, C);
        if (p->no_penalty)
            for (int k = 0; k < Q3; ++k) C[k] = 0.0;
        double mp[Q3];
        for (int k = 0; k < Q3; ++k) mp[k] = m[k] - G[k] * (m[k] - meq[k]) + (1.0 - 0.5 * G[k]) * (S[k] + C[k]);
        from_moments(mp, fp);
        for (int i = 0; i < Q3; ++i) post[i * N + c] = fp[i];
    }
    /* pull streaming with half-way bounce-back at the y walls */
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                const long long c = cell3(p, x, y, z);
                for (int i = 0; i < Q3; ++i) {
                    const int sy = y - E3[i][1];
                    if (p->bc_y == 1 && (sy < 0 || sy >= p->ny)) {
                        out[i * N + c] = post[opposite3(i) * N + c];
                    } else {
                        const int sx = wrap(x - E3[i][0], p->nx), sz = wrap(z - E3[i][2], p->nz);
                        out[i * N + c] = post[i * N + cell3(p, sx, wrap(sy, p->ny), sz)];
                    }
                }
            }
    free(post);
    free(grd);
    free(fld);
    free(u);
    free(F);
    free(rho);
    return 0;
}

/* f = f^eq(rho, u, phi) - F_i(u, F)/2 with F = F^p(rho) + F^B */
void v3_init(const V3Params* p, const double* rho, const double* ux, const double* uy, const double* uz,
             const double* phi, const double* fb, double* f) {
    const long long N = (long long)p->nx * p->ny * p->nz;
    double* g = (double*)malloc(sizeof(double) * 3 * N);
    v3_gradient(p, rho, 0, g, g + N, g + 2 * N);
    for (long long c = 0; c < N; ++c) {
        double fe[Q3], Fi[Q3], F[3];
        for (int a = 0; a < 3; ++a) F[a] = (p->kappa - phi[c]) / 3.0 * g[a * N + c] + (fb ? fb[a * N + c] : 0.0);
        v3_feq(p->kappa, phi[c], rho[c], ux[c], uy[c], uz[c], fe);
        v3_guo_force(ux[c], uy[c], uz[c], F[0], F[1], F[2], Fi);
        for (int i = 0; i < Q3; ++i) f[i * N + c] = fe[i] - 0.5 * Fi[i];
    }
    free(g);
}
