// vanse_adjoint.cuh -- FP64 discrete adjoint of the MRTLB-VANSE step with respect to
// the void fraction (the differentiation workload).
//
// Problem: steady phi(x); F^B = phi g with constant g; f(0) = f^eq(1, 0, phi) - F_i/2
// (Eq. 14, 6; F^p = 0 at uniform rho); T steps; after step n the objective samples
// O(n) = sum_y (j_x + F_x / 2)(x_out, y) = sum_y (phi rho u_x)(x_out, y), and
// J = sum over the last M steps of O(n) / (M ny). The gradient dJ/dphi(x) includes
// every way phi enters: rho = sum f / phi (Eq. 7), F^p (Eq. 13), X = kappa / phi in
// m^eq (Eq. 18) and C (Eq. 20), F^B and the initial populations.
//
// Layout: dense FP64, populations [9][ny][nx], fields [ny][nx]; x periodic, y
// periodic or half-way bounce-back walls. One thread per cell, grid-stride loops.
//
// Forward step = three kernels: adj_fwd_rho (Eq. 7: sum f, rho), adj_fwd_u (Eq. 10
// gradient of rho, Eq. 13 F, Eq. 7 u, the Eq. 20 fields rho u, u, phi rho u) and
// adj_fwd_collide (Eq. 10 gradients of the fields, Eq. 20 C, Eq. 18/19, Eq. 16
// relaxation, (A1) back-transform, push streaming with bounce-back).
//
// Backward step n (lambda(n+1) -> lambda(n), the adjoint of the post-streaming
// populations, plus the contribution of O(n)), with rho, u, F and the fields of f(n)
// recomputed by the two forward kernels first:
//   adj_bwd_collide  transpose of streaming, then the adjoint of the collision at each
//                    cell: lambda of the moments, of u, F, rho, phi and of the eight
//                    Eq. (10) derivatives the penalty C reads;
//   adj_bwd_u        the transposed Eq. (10) stencil gathers the field adjoints from
//                    the neighbours' derivative adjoints; the objective's source; the
//                    adjoint of F and u (Eq. 13, 7): lambda of sum f, j, rho, phi and
//                    of grad rho;
//   adj_bwd_rho      the transposed stencil gathers lambda rho from grad rho; rho =
//                    sum f / phi; lambda(n) = M^T lambda_m.
// The transposed Eq. (10) stencil at cell x sums, over the cells y whose stencil
// reads x (directly or through the mirrored wall ghost), 3 w_i e_i sign lambda(y).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vanse_common.cuh"

namespace lbmv {

namespace adj {

// D2Q9 (Eq. 5) and the moment basis of Eq. (17) / (A1) as compile-time functions, so
// that unrolled loops fold the zero and unit entries. The rows of M are orthogonal,
// M M^T = diag(9, 36, 36, 6, 12, 6, 12, 4, 4), hence M^-1 = M^T diag(1 / |row|^2).
__host__ __device__ constexpr double w_of(int i) { return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }
__host__ __device__ constexpr double m_of(int k, int i) {
    // rows: 1, e = -4 + 3|c|^2, eps = 4 - 21|c|^2/2 + 9|c|^4/2, c_x, q_x = (-5 + 3|c|^2) c_x,
    // c_y, q_y, c_x^2 - c_y^2, c_x c_y
    return k == 0 ? 1.0
         : k == 1 ? -4.0 + 3.0 * (ex_of(i) * ex_of(i) + ey_of(i) * ey_of(i))
         : k == 2 ? 4.0 - 10.5 * (ex_of(i) * ex_of(i) + ey_of(i) * ey_of(i)) +
                        4.5 * (ex_of(i) * ex_of(i) + ey_of(i) * ey_of(i)) * (ex_of(i) * ex_of(i) + ey_of(i) * ey_of(i))
         : k == 3 ? (double)ex_of(i)
         : k == 4 ? (-5.0 + 3.0 * (ex_of(i) * ex_of(i) + ey_of(i) * ey_of(i))) * ex_of(i)
         : k == 5 ? (double)ey_of(i)
         : k == 6 ? (-5.0 + 3.0 * (ex_of(i) * ex_of(i) + ey_of(i) * ey_of(i))) * ey_of(i)
         : k == 7 ? (double)(ex_of(i) * ex_of(i) - ey_of(i) * ey_of(i))
                  : (double)(ex_of(i) * ey_of(i));
}
__host__ __device__ constexpr double mnorm_of(int k) {
    return k == 0 ? 9.0 : (k <= 2 ? 36.0 : (k == 4 || k == 6 ? 12.0 : (k == 3 || k == 5 ? 6.0 : 4.0)));
}
__host__ __device__ constexpr double minv_of(int i, int k) { return m_of(k, i) / mnorm_of(k); }

struct Params {
    int nx, ny;
    long long N;
    int wall_y, model_b;
    double kappa, gx, gy;
    double s_e, s_eps, s_q, s_nu;
    int x_out;
};

// Work arrays of one forward recompute (each [N] unless noted).
struct Fields {
    double *s, *rho;                 // sum f, rho
    double *ux, *uy, *Fx, *Fy;       // u, F
    double *drx, *dry;               // grad rho
    double *fld;                     // [6][N]: rho u_x, rho u_y, u_x, u_y, phi rho u_x, phi rho u_y
};

// Adjoint work arrays (each [N] unless noted).
struct Adj {
    double* lm;      // [9][N] lambda of the moments of f(n)
    double *lux, *luy, *lFx, *lFy, *lrho;
    double* lg;      // [8][N] lambda of d_x A_x, d_y A_y, d_x B_x, d_y B_y, d_x B_y, d_y B_x, d_x D_x, d_y D_y
    double *ldrx, *ldry;
};

#define ADJ_LOOP(c, N) for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < (N); c += (long long)gridDim.x * blockDim.x)

// cell of the Eq. (10) stencil point (x + ex, y + ey); sign -1 when a wall was crossed
__device__ __forceinline__ long long stencil_cell(const Params& p, int x, int y, int ex, int ey, double& sign) {
    int x2 = x + ex;
    x2 = x2 < 0 ? x2 + p.nx : (x2 >= p.nx ? x2 - p.nx : x2);
    int y2 = y + ey;
    sign = 1.0;
    if (y2 < 0 || y2 >= p.ny) {
        if (p.wall_y) {
            y2 = y2 < 0 ? -1 - y2 : 2 * p.ny - 1 - y2;
            sign = -1.0;
        } else {
            y2 = y2 < 0 ? y2 + p.ny : y2 - p.ny;
        }
    }
    return (long long)y2 * p.nx + x2;
}

// Eq. (10) at (x, y): odd = vector component (negated in a wall ghost)
__device__ __forceinline__ void grad_at(const Params& p, const double* v, int x, int y, bool odd, double& gx,
                                        double& gy) {
    gx = 0.0;
    gy = 0.0;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        double sg;
        const long long c = stencil_cell(p, x, y, ex_of(i), ey_of(i), sg);
        const double val = odd ? sg * v[c] : v[c];
        gx += 3.0 * w_of(i) * ex_of(i) * val;
        gy += 3.0 * w_of(i) * ey_of(i) * val;
    }
}

// Transpose of Eq. (10) at (x, y): sum over the cells whose stencil reads (x, y) of
// 3 w_i (e_ix lx + e_iy ly) sign, with lx, ly the adjoints of their x / y derivatives
// (either may be null).
__device__ __forceinline__ double grad_T_at(const Params& p, const double* lx, const double* ly, int x, int y,
                                            bool odd) {
    double acc = 0.0;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const int ex = ex_of(i), ey = ey_of(i);
        const double wgt = 3.0 * w_of(i);
        int xs = x - ex;
        xs = xs < 0 ? xs + p.nx : (xs >= p.nx ? xs - p.nx : xs);
        // direct: the stencil point (xs, ys) + e_i is (x, y)
        int ys = y - ey;
        bool ok = true;
        if (ys < 0 || ys >= p.ny) {
            if (p.wall_y) ok = false;
            else ys = ys < 0 ? ys + p.ny : ys - p.ny;
        }
        if (ok) {
            const long long c = (long long)ys * p.nx + xs;
            acc += wgt * ((lx ? ex * lx[c] : 0.0) + (ly ? ey * ly[c] : 0.0));
        }
        // through the wall ghost: (xs, y) + e_i lies beyond the wall next to row y
        if (p.wall_y && ((y == 0 && ey == -1) || (y == p.ny - 1 && ey == 1))) {
            const long long c = (long long)y * p.nx + xs;
            const double sg = odd ? -1.0 : 1.0;
            acc += sg * wgt * ((lx ? ex * lx[c] : 0.0) + (ly ? ey * ly[c] : 0.0));
        }
    }
    return acc;
}

// ------------------------------------------------------------------ forward
// f(0) = f^eq(1, 0, phi) - F_i(0, phi g)/2
__global__ void adj_init_kernel(Params p, const double* __restrict__ phi, double* __restrict__ f) {
    ADJ_LOOP(c, p.N) {
    #pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double feq = i == 0 ? phi[c] - (5.0 / 9.0) * p.kappa : w_of(i) * p.kappa;
            const double Fi = 3.0 * w_of(i) * (ex_of(i) * p.gx + ey_of(i) * p.gy) * phi[c];
            f[i * p.N + c] = feq - 0.5 * Fi;
        }
    }
}

__global__ void adj_fwd_rho(Params p, const double* __restrict__ f, const double* __restrict__ phi, Fields F) {
    ADJ_LOOP(c, p.N) {
        double s = 0.0;
    #pragma unroll
        for (int i = 0; i < 9; ++i) s += f[i * p.N + c];
        F.s[c] = s;
        F.rho[c] = s / phi[c];
    }
}

__global__ void adj_fwd_u(Params p, const double* __restrict__ f, const double* __restrict__ phi, Fields F) {
    ADJ_LOOP(c, p.N) {
        const int x = (int)(c % p.nx), y = (int)(c / p.nx);
        double jx = 0.0, jy = 0.0;
    #pragma unroll
        for (int i = 1; i < 9; ++i) {
            jx += ex_of(i) * f[i * p.N + c];
            jy += ey_of(i) * f[i * p.N + c];
        }
        double gx, gy;
        grad_at(p, F.rho, x, y, false, gx, gy);
        const double ph = phi[c], s = F.s[c], rho = F.rho[c];
        const double kp = p.model_b ? p.kappa - 1.0 : p.kappa - ph;
        const double Fx = kp / 3.0 * gx + ph * p.gx, Fy = kp / 3.0 * gy + ph * p.gy;
        const double ux = (jx + 0.5 * Fx) / s, uy = (jy + 0.5 * Fy) / s;
        F.drx[c] = gx;
        F.dry[c] = gy;
        F.Fx[c] = Fx;
        F.Fy[c] = Fy;
        F.ux[c] = ux;
        F.uy[c] = uy;
        F.fld[0 * p.N + c] = rho * ux;
        F.fld[1 * p.N + c] = rho * uy;
        F.fld[2 * p.N + c] = ux;
        F.fld[3 * p.N + c] = uy;
        F.fld[4 * p.N + c] = s * ux;
        F.fld[5 * p.N + c] = s * uy;
    }
}

// the eight Eq. (10) derivatives of the Eq. (20) fields at (x, y)
__device__ __forceinline__ void field_grads(const Params& p, const Fields& F, int x, int y, double g[8]) {
    double a, b;
    grad_at(p, F.fld + 0 * p.N, x, y, true, g[0], a);   // d_x A_x
    grad_at(p, F.fld + 1 * p.N, x, y, true, a, g[1]);   // d_y A_y
    grad_at(p, F.fld + 2 * p.N, x, y, true, g[2], g[5]);  // d_x B_x, d_y B_x
    grad_at(p, F.fld + 3 * p.N, x, y, true, g[4], g[3]);  // d_x B_y, d_y B_y
    grad_at(p, F.fld + 4 * p.N, x, y, true, g[6], b);   // d_x D_x
    grad_at(p, F.fld + 5 * p.N, x, y, true, b, g[7]);   // d_y D_y
}

struct Local {
    double m[9];
    double s, rho, ux, uy, Fx, Fy, phi, X, kp;
    double g[8];
};

__device__ __forceinline__ void load_local(const Params& p, const double* f, const double* phi, const Fields& F,
                                           long long c, int x, int y, Local& L) {
    double fc[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) fc[i] = f[i * p.N + c];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        double a = 0.0;
    #pragma unroll
        for (int i = 0; i < 9; ++i) a += m_of(k, i) * fc[i];
        L.m[k] = a;
    }
    L.s = F.s[c];
    L.rho = F.rho[c];
    L.ux = F.ux[c];
    L.uy = F.uy[c];
    L.Fx = F.Fx[c];
    L.Fy = F.Fy[c];
    L.phi = phi[c];
    L.X = p.kappa / L.phi;
    L.kp = p.model_b ? p.kappa - 1.0 : p.kappa - L.phi;
    field_grads(p, F, x, y, L.g);
}

// Eq. (18), (19), (20), (16): post-collision moments (steady phi: no d_t phi term;
// the conserved moments: m0+ = m0, j+ = j + F)
__device__ __forceinline__ void collide(const Params& p, const Local& L, double mp[9]) {
    const double kr = L.kp * L.rho;
    const double divA = L.g[0] + L.g[1], difA = L.g[0] - L.g[1];
    const double divB = L.g[2] + L.g[3], difB = L.g[2] - L.g[3], crsB = L.g[4] + L.g[5];
    const double divD = L.g[6] + L.g[7], difD = L.g[6] - L.g[7];
    const double Ca = -p.kappa * divA + 2.0 * kr * divB + (3.0 - 2.0 * L.X) * divD;
    const double Cb = -p.kappa * difA + (2.0 / 3.0) * kr * difB + difD;
    const double Cc = (1.0 / 3.0) * kr * crsB;
    const double ux = L.ux, uy = L.uy, s = L.s, uu = ux * ux + uy * uy, uF = ux * L.Fx + uy * L.Fy;
    const double he = 1.0 - 0.5 * p.s_e, heps = 1.0 - 0.5 * p.s_eps, hq = 1.0 - 0.5 * p.s_q, hnu = 1.0 - 0.5 * p.s_nu;
    mp[0] = L.m[0];
    mp[1] = L.m[1] - p.s_e * (L.m[1] - s * (-4.0 + 3.0 * uu + 2.0 * L.X)) + he * (6.0 * uF + Ca);
    mp[2] = L.m[2] - p.s_eps * (L.m[2] - s * (4.0 - 3.0 * uu - 3.0 * L.X)) + heps * (-6.0 * uF);
    mp[3] = L.m[3] + L.Fx;
    mp[4] = L.m[4] - p.s_q * (L.m[4] - s * (L.X - 2.0) * ux) + hq * (-L.Fx);
    mp[5] = L.m[5] + L.Fy;
    mp[6] = L.m[6] - p.s_q * (L.m[6] - s * (L.X - 2.0) * uy) + hq * (-L.Fy);
    mp[7] = L.m[7] - p.s_nu * (L.m[7] - s * (ux * ux - uy * uy)) + hnu * (2.0 * (ux * L.Fx - uy * L.Fy) + Cb);
    mp[8] = L.m[8] - p.s_nu * (L.m[8] - s * ux * uy) + hnu * (ux * L.Fy + uy * L.Fx + Cc);
}

// collide and push-stream into fn (bounce-back links return to the same cell)
__global__ void adj_fwd_collide(Params p, const double* __restrict__ f, const double* __restrict__ phi, Fields F,
                                double* __restrict__ fn) {
    ADJ_LOOP(c, p.N) {
        const int x = (int)(c % p.nx), y = (int)(c / p.nx);
        Local L;
        load_local(p, f, phi, F, c, x, y, L);
        double mp[9];
        collide(p, L, mp);
    #pragma unroll
        for (int i = 0; i < 9; ++i) {
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < 9; ++k) v += minv_of(i, k) * mp[k];
            int xd = x + ex_of(i);
            xd = xd < 0 ? xd + p.nx : (xd >= p.nx ? xd - p.nx : xd);
            int yd = y + ey_of(i);
            if (yd < 0 || yd >= p.ny) {
                if (p.wall_y) {
                    fn[opp_of(i) * p.N + c] = v;
                    continue;
                }
                yd = yd < 0 ? yd + p.ny : yd - p.ny;
            }
            fn[i * p.N + (long long)yd * p.nx + xd] = v;
        }
    }
}

// O(n): sum over y of j_x + F_x / 2 at column x_out, added to *acc (one block)
__global__ void adj_objective(Params p, const double* __restrict__ f, Fields F, double* acc) {
    __shared__ double part[256];
    double v = 0.0;
    for (int y = threadIdx.x; y < p.ny; y += blockDim.x) {
        const long long c = (long long)y * p.nx + p.x_out;
        double jx = 0.0;
    #pragma unroll
        for (int i = 1; i < 9; ++i) jx += ex_of(i) * f[i * p.N + c];
        v += jx + 0.5 * F.Fx[c];
    }
    part[threadIdx.x] = v;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) part[threadIdx.x] += part[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *acc += part[0];
}

// ------------------------------------------------------------------ backward
// lam_next = lambda(n+1) (null: zero); f = f(n) with F recomputed from it.
__global__ void adj_bwd_collide(Params p, const double* __restrict__ f, const double* __restrict__ phi, Fields F,
                                const double* __restrict__ lam_next, Adj A, double* __restrict__ gphi) {
    ADJ_LOOP(c, p.N) {
        const int x = (int)(c % p.nx), y = (int)(c / p.nx);
        double lmp[9], lm[9];
    #pragma unroll
        for (int k = 0; k < 9; ++k) lm[k] = 0.0;
        double lux = 0, luy = 0, lFx = 0, lFy = 0, lrho = 0, lphi = 0;
        double lg[8];
    #pragma unroll
        for (int k = 0; k < 8; ++k) lg[k] = 0.0;
        if (lam_next) {
            // transpose of streaming
            double lp[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                int xd = x + ex_of(i);
                xd = xd < 0 ? xd + p.nx : (xd >= p.nx ? xd - p.nx : xd);
                int yd = y + ey_of(i);
                if (yd < 0 || yd >= p.ny) {
                    if (p.wall_y) {
                        lp[i] = lam_next[opp_of(i) * p.N + c];
                        continue;
                    }
                    yd = yd < 0 ? yd + p.ny : yd - p.ny;
                }
                lp[i] = lam_next[i * p.N + (long long)yd * p.nx + xd];
            }
            // f+ = M^-1 m+  ->  lambda m+ = M^-T lambda f+
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                double a = 0.0;
#pragma unroll
                for (int i = 0; i < 9; ++i) a += minv_of(i, k) * lp[i];
                lmp[k] = a;
            }
            Local L;
            load_local(p, f, phi, F, c, x, y, L);
            const double he = 1.0 - 0.5 * p.s_e, heps = 1.0 - 0.5 * p.s_eps, hq = 1.0 - 0.5 * p.s_q,
                         hnu = 1.0 - 0.5 * p.s_nu;
            // relaxation (Eq. 16) and the conserved moments
            lm[0] = lmp[0];
            lm[3] = lmp[3];
            lFx += lmp[3];
            lm[5] = lmp[5];
            lFy += lmp[5];
            lm[1] = (1.0 - p.s_e) * lmp[1];
            lm[2] = (1.0 - p.s_eps) * lmp[2];
            lm[4] = (1.0 - p.s_q) * lmp[4];
            lm[6] = (1.0 - p.s_q) * lmp[6];
            lm[7] = (1.0 - p.s_nu) * lmp[7];
            lm[8] = (1.0 - p.s_nu) * lmp[8];
            const double lq1 = p.s_e * lmp[1], lq2 = p.s_eps * lmp[2], lq4 = p.s_q * lmp[4], lq6 = p.s_q * lmp[6],
                         lq7 = p.s_nu * lmp[7], lq8 = p.s_nu * lmp[8];   // lambda of m^eq_k
            const double lS1 = he * lmp[1], lS2 = heps * lmp[2], lS4 = hq * lmp[4], lS6 = hq * lmp[6],
                         lS7 = hnu * lmp[7], lS8 = hnu * lmp[8];
            const double lCa = he * lmp[1], lCb = hnu * lmp[7], lCc = hnu * lmp[8];
            const double ux = L.ux, uy = L.uy, s = L.s, X = L.X, uu = ux * ux + uy * uy;
            // Eq. (18)
            double ls = lq1 * (-4.0 + 3.0 * uu + 2.0 * X) + lq2 * (4.0 - 3.0 * uu - 3.0 * X) + lq4 * (X - 2.0) * ux +
                        lq6 * (X - 2.0) * uy + lq7 * (ux * ux - uy * uy) + lq8 * ux * uy;
            lux += s * (6.0 * ux * lq1 - 6.0 * ux * lq2 + (X - 2.0) * lq4 + 2.0 * ux * lq7 + uy * lq8);
            luy += s * (6.0 * uy * lq1 - 6.0 * uy * lq2 + (X - 2.0) * lq6 - 2.0 * uy * lq7 + ux * lq8);
            double lX = s * (2.0 * lq1 - 3.0 * lq2 + ux * lq4 + uy * lq6);
            // Eq. (19)
            const double luF = 6.0 * lS1 - 6.0 * lS2;
            lux += luF * L.Fx + 2.0 * lS7 * L.Fx + lS8 * L.Fy;
            luy += luF * L.Fy - 2.0 * lS7 * L.Fy + lS8 * L.Fx;
            lFx += luF * ux - lS4 + 2.0 * lS7 * ux + lS8 * uy;
            lFy += luF * uy - lS6 - 2.0 * lS7 * uy + lS8 * ux;
            // Eq. (20)
            const double kr = L.kp * L.rho;
            const double divB = L.g[2] + L.g[3], difB = L.g[2] - L.g[3], crsB = L.g[4] + L.g[5];
            const double divD = L.g[6] + L.g[7];
            const double ldivA = -p.kappa * lCa, ldifA = -p.kappa * lCb;
            const double lkr = 2.0 * divB * lCa + (2.0 / 3.0) * difB * lCb + (1.0 / 3.0) * crsB * lCc;
            const double ldivB = 2.0 * kr * lCa, ldifB = (2.0 / 3.0) * kr * lCb, lcrsB = (1.0 / 3.0) * kr * lCc;
            const double ldivD = (3.0 - 2.0 * X) * lCa, ldifD = lCb;
            lX += -2.0 * divD * lCa;
            lrho += L.kp * lkr;
            const double lkp = L.rho * lkr;
            lphi += -(p.kappa / (L.phi * L.phi)) * lX;
            if (!p.model_b) lphi += -lkp;
            lg[0] = ldivA + ldifA;
            lg[1] = ldivA - ldifA;
            lg[2] = ldivB + ldifB;
            lg[3] = ldivB - ldifB;
            lg[4] = lcrsB;
            lg[5] = lcrsB;
            lg[6] = ldivD + ldifD;
            lg[7] = ldivD - ldifD;
            lm[0] += ls;
        }
    #pragma unroll
        for (int k = 0; k < 9; ++k) A.lm[k * p.N + c] = lm[k];
    #pragma unroll
        for (int k = 0; k < 8; ++k) A.lg[k * p.N + c] = lg[k];
        A.lux[c] = lux;
        A.luy[c] = luy;
        A.lFx[c] = lFx;
        A.lFy[c] = lFy;
        A.lrho[c] = lrho;
        gphi[c] += lphi;
    }
}

// gather the field adjoints, add the objective's source, adjoint of Eq. (13), (7)
__global__ void adj_bwd_u(Params p, const double* __restrict__ f, const double* __restrict__ phi, Fields F, Adj A,
                          double obj_weight, double* __restrict__ gphi) {
    ADJ_LOOP(c, p.N) {
        const int x = (int)(c % p.nx), y = (int)(c / p.nx);
        const long long N = p.N;
        // lambda of the fields A = rho u, B = u, D = phi rho u (transposed Eq. 10)
        const double lAx = grad_T_at(p, A.lg + 0 * N, nullptr, x, y, true);
        const double lAy = grad_T_at(p, nullptr, A.lg + 1 * N, x, y, true);
        const double lBx = grad_T_at(p, A.lg + 2 * N, A.lg + 5 * N, x, y, true);
        const double lBy = grad_T_at(p, A.lg + 4 * N, A.lg + 3 * N, x, y, true);
        const double lDx = grad_T_at(p, A.lg + 6 * N, nullptr, x, y, true);
        const double lDy = grad_T_at(p, nullptr, A.lg + 7 * N, x, y, true);
        const double s = F.s[c], rho = F.rho[c], ux = F.ux[c], uy = F.uy[c], ph = phi[c];
        const double lux = A.lux[c] + lBx + rho * lAx + s * lDx;
        const double luy = A.luy[c] + lBy + rho * lAy + s * lDy;
        double lrho = A.lrho[c] + ux * lAx + uy * lAy;
        double ls = ux * lDx + uy * lDy;
        double ljx = lux / s, ljy = luy / s;
        double lFx = A.lFx[c] + 0.5 * lux / s, lFy = A.lFy[c] + 0.5 * luy / s;
        ls += -(ux * lux + uy * luy) / s;
        if (obj_weight != 0.0 && x == p.x_out) {
            ljx += obj_weight;
            lFx += 0.5 * obj_weight;
        }
        // F = kp/3 grad rho + phi g
        const double kp = p.model_b ? p.kappa - 1.0 : p.kappa - ph;
        A.ldrx[c] = kp / 3.0 * lFx;
        A.ldry[c] = kp / 3.0 * lFy;
        const double lkp = (F.drx[c] * lFx + F.dry[c] * lFy) / 3.0;
        double lphi = p.gx * lFx + p.gy * lFy;
        if (!p.model_b) lphi -= lkp;
        A.lm[0 * N + c] += ls;
        A.lm[3 * N + c] += ljx;
        A.lm[5 * N + c] += ljy;
        A.lrho[c] = lrho;
        gphi[c] += lphi;
    }
}

// gather lambda rho from grad rho, rho = sum f / phi, lambda(n) = M^T lambda_m
__global__ void adj_bwd_rho(Params p, const double* __restrict__ phi, Fields F, Adj A, double* __restrict__ lam,
                            double* __restrict__ gphi) {
    ADJ_LOOP(c, p.N) {
        const int x = (int)(c % p.nx), y = (int)(c / p.nx);
        const double lrho = A.lrho[c] + grad_T_at(p, A.ldrx, A.ldry, x, y, false);
        const double ph = phi[c];
        double lm[9];
    #pragma unroll
        for (int k = 0; k < 9; ++k) lm[k] = A.lm[k * p.N + c];
        lm[0] += lrho / ph;
        gphi[c] += -lrho * F.s[c] / (ph * ph);
    #pragma unroll
        for (int i = 0; i < 9; ++i) {
            double a = 0.0;
#pragma unroll
            for (int k = 0; k < 9; ++k) a += m_of(k, i) * lm[k];
            lam[i * p.N + c] = a;
        }
    }
}

// adjoint of the initial populations: gphi += d f(0) / d phi . lambda(0)
__global__ void adj_bwd_init(Params p, const double* __restrict__ lam, double* __restrict__ gphi) {
    ADJ_LOOP(c, p.N) {
        double a = lam[c];
    #pragma unroll
        for (int i = 1; i < 9; ++i) a -= 1.5 * w_of(i) * (ex_of(i) * p.gx + ey_of(i) * p.gy) * lam[i * p.N + c];
        gphi[c] += a;
    }
}

#undef ADJ_LOOP

}  // namespace adj
}  // namespace lbmv
