// The three-dimensional (D3Q19) MRTLB-VANSE step and the C ABI of
// include/lbm_vanse3d.h.
//
// One step is three kernels over the cells (x fastest, one thread per cell):
//   v3_moments   sum f and sum e f of the post-streaming populations, rho = sum f / phi
//                (Eq. 7);
//   v3_velocity  grad rho by Eq. (10) with the D3Q19 weights, F = (kappa - phi)/3 grad rho
//                + F^B (Eq. 13), u = (j + F/2) / sum f (Eq. 7);
//   v3_collide   the gradients of rho u, u and phi rho u (Eq. 10), the D3Q19 penalty
//                source, m = M f, the relaxation of Eq. (16) with the equilibrium and
//                Guo force moments, f+ = M^-1 m+, and push streaming (periodic x, z;
//                periodic or half-way bounce-back in y).
// The population buffers hold post-streaming deviations from the rest state,
// d_i = f_i - f_i^rest with f_i^rest = w_i kappa rho0 (i >= 1) and (phi - 2 kappa / 3) rho0
// (i = 0, phi of the lattice's current time level: the rest equilibrium of Eq. (14) on
// D3Q19), as [19][nz][ny][nx] planes in the storage type T (double or float), which is
// also the compute type; the density scratch holds rho - rho0. Every rounding then
// sits at the scale of the deviations rather than of the populations. Next to a wall
// the gradient stencils read a ghost cell mirrored about it (scalars keep the mirror
// value, vector components change sign).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <utility>

#include "lbm_vanse3d.h"

namespace lbmv3 {

constexpr int Q = 19;

// D3Q19 velocities (the order of the ABI)
constexpr int kE[Q][3] = {{0, 0, 0},   {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                          {0, 0, 1},   {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                          {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                          {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

// The same velocities, the opposite directions, the weights and the integer moment
// basis as compile-time functions: inside fully unrolled loops they fold into
// immediates, so the 19 x 19 transforms drop their zero products and turn the +-1
// entries into adds.
__host__ __device__ constexpr int vel(int i, int a) {
    return a == 0 ? ((i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
                     : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0)
         : a == 1 ? ((i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
                     : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0)
                  : ((i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
                     : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0);
}

__host__ __device__ constexpr int opp(int i) {
    int r = 0;
    for (int k = 0; k < Q; ++k)
        if (vel(k, 0) == -vel(i, 0) && vel(k, 1) == -vel(i, 1) && vel(k, 2) == -vel(i, 2)) r = k;
    return r;
}

// the basis polynomial of moment k at e_i (d'Humieres et al. 2002); all integers
__host__ __device__ constexpr int mcoef(int k, int i) {
    const int x = vel(i, 0), y = vel(i, 1), z = vel(i, 2), c2 = x * x + y * y + z * z;
    switch (k) {
        case 0: return 1;
        case 1: return 19 * c2 - 30;
        case 2: return (21 * c2 * c2 - 53 * c2 + 24) / 2;
        case 3: return x;
        case 4: return (5 * c2 - 9) * x;
        case 5: return y;
        case 6: return (5 * c2 - 9) * y;
        case 7: return z;
        case 8: return (5 * c2 - 9) * z;
        case 9: return 3 * x * x - c2;
        case 10: return (3 * c2 - 5) * (3 * x * x - c2);
        case 11: return y * y - z * z;
        case 12: return (3 * c2 - 5) * (y * y - z * z);
        case 13: return x * y;
        case 14: return y * z;
        case 15: return x * z;
        case 16: return (y * y - z * z) * x;
        case 17: return (z * z - x * x) * y;
        default: return (x * x - y * y) * z;
    }
}

__host__ __device__ constexpr int mnorm2(int k) {
    int s = 0;
    for (int i = 0; i < Q; ++i) s += mcoef(k, i) * mcoef(k, i);
    return s;
}

constexpr bool tables_agree() {
    for (int i = 0; i < Q; ++i)
        for (int a = 0; a < 3; ++a)
            if (vel(i, a) != kE[i][a]) return false;
    for (int k = 0; k < Q; ++k)            // orthogonal rows
        for (int l = 0; l < k; ++l) {
            int d = 0;
            for (int i = 0; i < Q; ++i) d += mcoef(k, i) * mcoef(l, i);
            if (d != 0) return false;
        }
    return true;
}
static_assert(tables_agree(), "velocity table and moment basis disagree");

template <typename T>
__host__ __device__ constexpr T weight(int i) {
    return i == 0 ? (T)1 / (T)3 : (i <= 6 ? (T)1 / (T)18 : (T)1 / (T)36);
}

// Transforms with compile-time coefficients: index sequences over the rows and the
// columns, `if constexpr` on each coefficient (zeros skipped, +-1 as adds), so no
// coefficient is looked up or tested while the kernel runs.
template <int K, int I, typename T>
__device__ __forceinline__ void row_acc(T& a, const T* v) {
    if constexpr (I < Q) {
        constexpr int c = mcoef(K, I);
        if constexpr (c == 1) a += v[I];
        else if constexpr (c == -1) a -= v[I];
        else if constexpr (c != 0) a += (T)c * v[I];
        row_acc<K, I + 1>(a, v);
    }
}

template <int I, int K, typename T>
__device__ __forceinline__ void col_acc(T& a, const T* v) {
    if constexpr (K < Q) {
        constexpr int c = mcoef(K, I);
        if constexpr (c == 1) a += v[K];
        else if constexpr (c == -1) a -= v[K];
        else if constexpr (c != 0) a += (T)c * v[K];
        col_acc<I, K + 1>(a, v);
    }
}

// out_k = sum_i M_ki v_i
template <typename T, int... K>
__device__ __forceinline__ void to_moments(const T* v, T* out, std::integer_sequence<int, K...>) {
    ((out[K] = (T)0, row_acc<K, 0>(out[K], v)), ...);
}

// out_i = sum_k M_ki v_k / |row k|^2 (v is scaled in place first)
template <typename T, int... K>
__device__ __forceinline__ void from_moments(T* v, T* out, std::integer_sequence<int, K...>) {
    ((v[K] *= (T)1 / (T)mnorm2(K)), ...);
    ((out[K] = (T)0, col_acc<K, 0>(out[K], v)), ...);
}

// Eq. (6) for every direction: F_i = w_i [3 (e_i - u) + 9 (e_i . u) e_i] . F
template <int I, typename T>
__device__ __forceinline__ T guo_one(const T* u, const T* F) {
    constexpr int ex = vel(I, 0), ey = vel(I, 1), ez = vel(I, 2);
    const T eu = (T)ex * u[0] + (T)ey * u[1] + (T)ez * u[2];
    const T s = ((T)3 * ((T)ex - u[0]) + (T)9 * eu * (T)ex) * F[0] +
                ((T)3 * ((T)ey - u[1]) + (T)9 * eu * (T)ey) * F[1] +
                ((T)3 * ((T)ez - u[2]) + (T)9 * eu * (T)ez) * F[2];
    return weight<T>(I) * s;
}

template <typename T, int... I>
__device__ __forceinline__ void guo_all(const T* u, const T* F, T* out, std::integer_sequence<int, I...>) {
    ((out[I] = guo_one<I>(u, F)), ...);
}

using Seq = std::make_integer_sequence<int, 19>;

struct Geo {
    int nx, ny, nz;
    long long N;
    int walls;   // 1: half-way bounce-back walls in y
};

template <typename T> struct Rates {
    T s[Q];
    T kappa, rho0;
};

__device__ __forceinline__ void decode(const Geo& g, long long c, int& x, int& y, int& z) {
    x = (int)(c % g.nx);
    const long long r = c / g.nx;
    y = (int)(r % g.ny);
    z = (int)(r / g.ny);
}

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// neighbour (x + e) for the gradient stencils: periodic x, z; y periodic or mirrored
// about the wall (mirror = true when the ghost is a mirror image)
__device__ __forceinline__ long long neighbour(const Geo& g, int x, int y, int z, int i, bool& mirror) {
    const int xn = wrapi(x + vel(i, 0), g.nx), zn = wrapi(z + vel(i, 2), g.nz);
    int yn = y + vel(i, 1);
    mirror = false;
    if (g.walls) {
        if (yn < 0) { yn = -1 - yn; mirror = true; }
        else if (yn >= g.ny) { yn = 2 * g.ny - 1 - yn; mirror = true; }
    } else {
        yn = wrapi(yn, g.ny);
    }
    return ((long long)zn * g.ny + yn) * g.nx + xn;
}

template <typename T>
__global__ void v3_moments(const T* __restrict__ f, const T* __restrict__ phi, T* __restrict__ rho,
                           T* __restrict__ j, Geo g) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    T m0 = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T v = f[i * g.N + c];
        m0 += v;
        jx += (T)vel(i, 0) * v;
        jy += (T)vel(i, 1) * v;
        jz += (T)vel(i, 2) * v;
    }
    rho[c] = m0 / phi[c];
    j[c] = jx;
    j[g.N + c] = jy;
    j[2 * g.N + c] = jz;
}

// F = (kappa - phi)/3 grad rho + phi G + field, u = (j + F/2) / (phi rho)
template <typename T>
__global__ void v3_velocity(const T* __restrict__ rho, const T* __restrict__ j, const T* __restrict__ phi,
                            const T* __restrict__ fb, T gx, T gy, T gz, T kappa, T rho0, T* __restrict__ u,
                            T* __restrict__ F, Geo g) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    int x, y, z;
    decode(g, c, x, y, z);
    T gr[3] = {0, 0, 0};
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        bool mir;
        const T v = (T)3 * weight<T>(i) * rho[neighbour(g, x, y, z, i, mir)];
        gr[0] += (T)vel(i, 0) * v;
        gr[1] += (T)vel(i, 1) * v;
        gr[2] += (T)vel(i, 2) * v;
    }
    const T ph = phi[c], r = rho[c];
    const T G[3] = {gx, gy, gz};
    const T m0 = ph * (rho0 + r);   // r = rho - rho0
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T Fa = (kappa - ph) / (T)3 * gr[a] + ph * G[a];
        if (fb) Fa += fb[a * g.N + c];
        F[a * g.N + c] = Fa;
        u[a * g.N + c] = (j[a * g.N + c] + (T)0.5 * Fa) / m0;
    }
}

template <typename T>
__device__ __forceinline__ void equilibrium_moments(T kappa, T phi, T rho, const T* u, T* m) {
    const T m0 = phi * rho, X = kappa / phi;
    const T u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const T pxx3 = m0 * ((T)3 * u[0] * u[0] - u2), pww = m0 * (u[1] * u[1] - u[2] * u[2]);
    const T qf = (T)10 * X / (T)3 - (T)4;
    m[0] = m0;
    m[1] = (T)19 * (kappa * rho + m0 * u2) - (T)30 * m0;
    m[2] = (T)12 * m0 - (T)9 * kappa * rho - (T)5.5 * m0 * u2;
    m[3] = m0 * u[0];
    m[4] = qf * m0 * u[0];
    m[5] = m0 * u[1];
    m[6] = qf * m0 * u[1];
    m[7] = m0 * u[2];
    m[8] = qf * m0 * u[2];
    m[9] = pxx3;
    m[10] = (T)-0.5 * pxx3;
    m[11] = pww;
    m[12] = (T)-0.5 * pww;
    m[13] = m0 * u[0] * u[1];
    m[14] = m0 * u[1] * u[2];
    m[15] = m0 * u[0] * u[2];
    m[16] = 0;
    m[17] = 0;
    m[18] = 0;
}

// m^eq minus the rest state's moments (rho0, u = 0): only m_0, e and eps carry a rest
// part; drho = rho - rho0
template <typename T>
__device__ __forceinline__ void equilibrium_deviation(T kappa, T phi, T rho, T drho, const T* u, T* m) {
    equilibrium_moments<T>(kappa, phi, rho, u, m);
    const T m0u2 = phi * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    m[0] = phi * drho;
    m[1] = (T)19 * (kappa * drho + m0u2) - (T)30 * phi * drho;
    m[2] = (T)12 * phi * drho - (T)9 * kappa * drho - (T)5.5 * m0u2;
}

// the collision's tile: 32 x 2 x 2 cells (one thread each) and a one-cell halo (larger
// tiles, 32 x 4 x 2 to 32 x 4 x 4, stage fewer halo cells per cell but ran slower)
#ifndef LBMV3_TY
#define LBMV3_TY 2
#endif
#ifndef LBMV3_TZ
#define LBMV3_TZ 2
#endif
// resident collision CTAs per SM the register allocation is sized for: 7 (72 registers,
// about 150 bytes of L1-cached spills per thread) ran the 256^3 FP32 step 11 % faster
// than the unbounded 96 registers (5 CTAs)
#ifndef LBMV3_MINB
#define LBMV3_MINB 7
#endif
constexpr int TX = 32, TY = LBMV3_TY, TZ = LBMV3_TZ, HX = TX + 2, HY = TY + 2, HZ = TZ + 2, HN = HX * HY * HZ;

__device__ __forceinline__ int modp(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

template <typename T>
__global__ void __launch_bounds__(TX * TY * TZ, LBMV3_MINB) v3_collide(const T* __restrict__ f, T* __restrict__ fo,
                                                           const T* __restrict__ rho, const T* __restrict__ u,
                                                           const T* __restrict__ F, const T* __restrict__ phi,
                                                           const T* __restrict__ phin, Rates<T> R, Geo g) {
    // rho, phi and u of the tile and its halo, staged once: the wall ghosts are
    // mirrored here (u with its sign changed), periodic axes wrap
    __shared__ T s_r[HN], s_p[HN], s_u[3][HN];
    const int nbx = (g.nx + TX - 1) / TX, nby = (g.ny + TY - 1) / TY;
    const int bx = (int)(blockIdx.x % nbx), by = (int)((blockIdx.x / nbx) % nby), bz = (int)(blockIdx.x / (nbx * nby));
    const int x0 = bx * TX, y0 = by * TY, z0 = bz * TZ;
    for (int q = threadIdx.x; q < HN; q += TX * TY * TZ) {
        const int hx = q % HX, hy = (q / HX) % HY, hz = q / (HX * HY);
        const int gx = modp(x0 - 1 + hx, g.nx), gz = modp(z0 - 1 + hz, g.nz);
        int gy = y0 - 1 + hy;
        T sg = 1;
        if (g.walls) {
            if (gy < 0) { gy = -1 - gy; sg = -1; }
            else if (gy >= g.ny) { gy = 2 * g.ny - 1 - gy; sg = -1; }
            gy = gy < 0 ? 0 : (gy >= g.ny ? g.ny - 1 : gy);   // beyond one ghost: only idle threads read it
        } else {
            gy = modp(gy, g.ny);
        }
        const long long n = ((long long)gz * g.ny + gy) * g.nx + gx;
        s_r[q] = rho[n];
        s_p[q] = phi[n];
        s_u[0][q] = sg * u[n];
        s_u[1][q] = sg * u[g.N + n];
        s_u[2][q] = sg * u[2 * g.N + n];
    }
    __syncthreads();
    const int tx = threadIdx.x % TX, ty = (threadIdx.x / TX) % TY, tz = threadIdx.x / (TX * TY);
    const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
    if (x >= g.nx || y >= g.ny || z >= g.nz) return;
    const long long c = ((long long)z * g.ny + y) * g.nx + x;
    const int hc = ((tz + 1) * HY + (ty + 1)) * HX + (tx + 1);
    const T kappa = R.kappa;
    // gradients of A = rho u (diagonal), B = u (all nine), D = phi rho u (diagonal)
    T dA[3] = {0, 0, 0}, dD[3] = {0, 0, 0}, dB[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int hn = hc + (vel(i, 2) * HY + vel(i, 1)) * HX + vel(i, 0);
        const T rn = R.rho0 + s_r[hn], pn = s_p[hn];
        const T un[3] = {s_u[0][hn], s_u[1][hn], s_u[2][hn]};
        const T wv = (T)3 * weight<T>(i);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const T ca = wv * (T)vel(i, a);
            dA[a] += ca * rn * un[a];
            dD[a] += ca * pn * rn * un[a];
#pragma unroll
            for (int b = 0; b < 3; ++b) dB[3 * a + b] += ca * un[b];
        }
    }
    const T ph = s_p[hc], dr = s_r[hc], r = R.rho0 + dr;
    const T uc[3] = {s_u[0][hc], s_u[1][hc], s_u[2][hc]};
    const T Fc[3] = {F[c], F[g.N + c], F[2 * g.N + c]};
    const T X = kappa / ph, kp = kappa - ph;
    const T dtphi = phin ? phin[c] - ph : (T)0;
    T C[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) C[k] = 0;
    {
        const T divB = dB[0] + dB[4] + dB[8], divD = dD[0] + dD[1] + dD[2];
        C[1] = (T)19 * (((T)1 - X) * divD - X * r * dtphi + (T)2 / (T)3 * kp * r * divB);
        T dg[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) dg[a] = -kappa * dA[a] + (T)2 / (T)3 * kp * r * dB[4 * a] + dD[a];
        C[9] = (T)2 * dg[0] - dg[1] - dg[2];
        C[11] = dg[1] - dg[2];
        C[13] = kp * r * (dB[1] + dB[3]) / (T)3;
        C[14] = kp * r * (dB[5] + dB[7]) / (T)3;
        C[15] = kp * r * (dB[2] + dB[6]) / (T)3;
    }
    T fl[Q], Fi[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fl[i] = f[i * g.N + c];
    guo_all<T>(uc, Fc, Fi, Seq{});
    T meq[Q], m[Q], S[Q];
    equilibrium_deviation<T>(kappa, ph, r, dr, uc, meq);
    to_moments<T>(fl, m, Seq{});
    to_moments<T>(Fi, S, Seq{});
    T mp[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const T s = R.s[k];
        mp[k] = m[k] - s * (m[k] - meq[k]) + ((T)1 - (T)0.5 * s) * (S[k] + C[k]);
    }
    T fp[Q];
    from_moments<T>(mp, fp, Seq{});
    fp[0] -= dtphi * R.rho0;   // f_0's rest value moves to phi(t+1)
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T v = fp[i];
        // push: f+_i(x) -> f_i(x + e_i); a link into a y wall returns as f_opp(x)
        const int yd = y + vel(i, 1);
        if (g.walls && (yd < 0 || yd >= g.ny)) {
            fo[opp(i) * g.N + c] = v;
        } else {
            const int xd = wrapi(x + vel(i, 0), g.nx), zd = wrapi(z + vel(i, 2), g.nz);
            fo[i * g.N + ((long long)zd * g.ny + wrapi(yd, g.ny)) * g.nx + xd] = v;
        }
    }
}

// f = f^eq(rho, u, phi) - F_i/2 (F from v3_velocity's force part)
template <typename T>
__global__ void v3_init(T* __restrict__ f, const T* __restrict__ rho, const T* __restrict__ u,
                        const T* __restrict__ F, const T* __restrict__ phi, T kappa, T rho0, Geo g) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    const T uc[3] = {u[c], u[g.N + c], u[2 * g.N + c]};
    const T Fc[3] = {F[c], F[g.N + c], F[2 * g.N + c]};
    T meq[Q], fe[Q], Fi[Q];
    equilibrium_deviation<T>(kappa, phi[c], rho[c], rho[c] - rho0, uc, meq);
    from_moments<T>(meq, fe, Seq{});
    guo_all<T>(uc, Fc, Fi, Seq{});
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        f[i * g.N + c] = fe[i] - (T)0.5 * Fi[i];
    }
}

// F only (init: the velocity is given)
template <typename T>
__global__ void v3_force(const T* __restrict__ rho, const T* __restrict__ phi, const T* __restrict__ fb, T gx,
                         T gy, T gz, T kappa, T* __restrict__ F, Geo g) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    int x, y, z;
    decode(g, c, x, y, z);
    T gr[3] = {0, 0, 0};
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        bool mir;
        const T v = (T)3 * weight<T>(i) * rho[neighbour(g, x, y, z, i, mir)];
#pragma unroll
        for (int a = 0; a < 3; ++a) gr[a] += (T)vel(i, a) * v;
    }
    const T ph = phi[c], G[3] = {gx, gy, gz};
    for (int a = 0; a < 3; ++a) F[a * g.N + c] = (kappa - ph) / (T)3 * gr[a] + ph * G[a] + (fb ? fb[a * g.N + c] : (T)0);
}

// populations to / from the caller's f: out = in + sign * f_i^rest, in FP64
template <typename Tin, typename Tout, typename T>
__global__ void v3_pop_io(const Tin* __restrict__ a, Tout* __restrict__ b, const T* __restrict__ phi, double kappa,
                          double rho0, double sign, long long N) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < (long long)Q * N;
         k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k / N);
        const double rest = i == 0 ? ((double)phi[k] - 2.0 * kappa / 3.0) * rho0
                                   : (i <= 6 ? kappa * rho0 / 18.0 : kappa * rho0 / 36.0);
        b[k] = (Tout)((double)a[k] + sign * rest);
    }
}

// a new phi(t) where the lattice holds populations: f_0's rest value follows phi, so the
// stored d_0 moves by (phi_old - phi_new) rho0 where phi changes
template <typename T>
__global__ void v3_rebase(const double* __restrict__ phin_src, T* __restrict__ phi, T* __restrict__ d0, T rho0,
                          long long N) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (long long)gridDim.x * blockDim.x) {
        const T v = (T)phin_src[k], old = phi[k];
        if (v != old) {
            d0[k] += (old - v) * rho0;
            phi[k] = v;
        }
    }
}

template <typename Tin, typename Tout>
__global__ void v3_convert(const Tin* __restrict__ a, Tout* __restrict__ b, long long n, double offset = 0.0) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        b[k] = (Tout)((double)a[k] + offset);
}

// FP64 mass and momentum sums: out[0..3] += per-block partials
template <typename T>
__global__ void v3_reduce(const T* __restrict__ f, const T* __restrict__ phi, double rho0, long long N,
                          double* __restrict__ out) {
    __shared__ double sh[4][256];
    double s[4] = {0, 0, 0, 0};
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        s[0] += (double)phi[c] * rho0;   // the rest state's mass
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double v = (double)f[i * N + c];
            s[0] += v;
            s[1] += vel(i, 0) * v;
            s[2] += vel(i, 1) * v;
            s[3] += vel(i, 2) * v;
        }
    }
    for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 4; ++q) atomicAdd(out + q, sh[q][0]);
}

__global__ void v3_check_phi(const double* __restrict__ phi, long long n, int* __restrict__ bad) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        if (!(phi[k] > 0.0 && phi[k] <= 1.0)) atomicExch(bad, 1);
}

}  // namespace lbmv3

using namespace lbmv3;

namespace {
thread_local std::string g_err3;
}

struct lbm_vanse3d {
    lbm_vanse3d_params prm{};
    cudaStream_t stream = nullptr;
    Geo geo{};
    int fp64 = 0;
    size_t tb = 4;               // bytes of T
    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    void *phi = nullptr, *phin = nullptr, *fb = nullptr;
    void *rho = nullptr, *j = nullptr, *u = nullptr, *F = nullptr;
    double* red = nullptr;
    int* bad = nullptr;
    double g[3] = {0, 0, 0};
    bool phi_set = false, phin_set = false, fb_set = false, initialised = false;
    long long steps = 0;
    double s[Q];
    std::string msg;
};

static lbm_status fail3(lbm_vanse3d* h, lbm_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->msg = buf; else g_err3 = buf;
    return st;
}

#define CK3(h, call)                                                                        \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return fail3((h), LBM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// stage n doubles from the caller into device memory (a device copy when on the host)
static lbm_status stage_in3(lbm_vanse3d* h, const double* src, long long n, int on_device, const double** out,
                            double** owned) {
    *owned = nullptr;
    if (on_device) { *out = src; return LBM_OK; }
    double* d = nullptr;
    CK3(h, cudaMallocAsync((void**)&d, n * sizeof(double), h->stream));
    CK3(h, cudaMemcpyAsync(d, src, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    *out = d;
    *owned = d;
    return LBM_OK;
}

static void convert_in(lbm_vanse3d* h, const double* d, void* dst, long long n) {
    const unsigned nb = blocks_for(n, 256) < 4096 ? blocks_for(n, 256) : 4096;
    if (h->fp64) v3_convert<double, double><<<nb, 256, 0, h->stream>>>(d, (double*)dst, n);
    else v3_convert<double, float><<<nb, 256, 0, h->stream>>>(d, (float*)dst, n);
}

template <typename T>
static Rates<T> rates(const lbm_vanse3d* h) {
    Rates<T> R;
    for (int k = 0; k < Q; ++k) R.s[k] = (T)h->s[k];
    R.kappa = (T)h->prm.kappa;
    R.rho0 = (T)h->prm.rho0;
    return R;
}

template <typename T>
static void enqueue_step(lbm_vanse3d* h) {
    const Geo& g = h->geo;
    const unsigned nb = (unsigned)(((g.nx + TX - 1) / TX) * (long long)((g.ny + TY - 1) / TY) * ((g.nz + TZ - 1) / TZ));
    const T* src = (const T*)h->f[h->cur];
    T* dst = (T*)h->f[1 - h->cur];
    v3_moments<T><<<blocks_for(g.N, 256), 256, 0, h->stream>>>(src, (const T*)h->phi, (T*)h->rho, (T*)h->j, g);
    v3_velocity<T><<<blocks_for(g.N, 256), 256, 0, h->stream>>>(
        (const T*)h->rho, (const T*)h->j, (const T*)h->phi, h->fb_set ? (const T*)h->fb : nullptr, (T)h->g[0],
        (T)h->g[1], (T)h->g[2], (T)h->prm.kappa, (T)h->prm.rho0, (T*)h->u, (T*)h->F, g);
    v3_collide<T><<<nb, TX * TY * TZ, 0, h->stream>>>(src, dst, (const T*)h->rho, (const T*)h->u, (const T*)h->F,
                                               (const T*)h->phi, h->phin_set ? (const T*)h->phin : nullptr,
                                               rates<T>(h), g);
}

extern "C" void lbm_vanse3d_default_params(lbm_vanse3d_params* p) {
    if (!p) return;
    *p = lbm_vanse3d_params{};
    p->tau_nu = 0.8;
    p->s_e = 0.0;
    p->s_eps = p->s_q = p->s_pi = p->s_m = 1.2;
    p->kappa = 0.5;
    p->rho0 = 1.0;
    p->bc_y = LBM_BC_PERIODIC;
    p->storage = LBM_FP32;
}

extern "C" const char* lbm_vanse3d_last_error(lbm_vanse3d_t h) { return h ? h->msg.c_str() : g_err3.c_str(); }

extern "C" void lbm_vanse3d_destroy(lbm_vanse3d_t h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    void* ptrs[] = {h->f[0], h->f[1], h->phi, h->phin, h->fb, h->rho, h->j, h->u, h->F, h->red, h->bad};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete h;
}

extern "C" lbm_status lbm_vanse3d_create(const lbm_vanse3d_params* p, void* stream, lbm_vanse3d_t* out) {
    if (!out) return fail3(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!p) return fail3(nullptr, LBM_ERR_ARG, "params is NULL");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail3(nullptr, LBM_ERR_ARG, "lattice size must be >= 1");
    const long long N = (long long)p->nx * p->ny * p->nz;
    if (N > (1LL << 40)) return fail3(nullptr, LBM_ERR_ARG, "lattice too large");
    if (!(p->tau_nu > 0.5)) return fail3(nullptr, LBM_ERR_ARG, "tau_nu must exceed 1/2");
    const double rates_in[] = {p->s_eps, p->s_q, p->s_pi, p->s_m};
    for (double r : rates_in)
        if (!(r > 0.0 && r <= 2.0)) return fail3(nullptr, LBM_ERR_ARG, "rates must lie in (0, 2]");
    if (p->s_e > 2.0) return fail3(nullptr, LBM_ERR_ARG, "s_e must lie in (0, 2] (or <= 0: derived)");
    if (!(p->rho0 > 0.0)) return fail3(nullptr, LBM_ERR_ARG, "rho0 must be positive");
    if (p->bc_y != LBM_BC_PERIODIC && p->bc_y != LBM_BC_BOUNCEBACK) return fail3(nullptr, LBM_ERR_ARG, "bad bc_y");
    if (p->storage != LBM_FP64 && p->storage != LBM_FP32)
        return fail3(nullptr, LBM_ERR_ARG, "3-D storage must be LBM_FP64 or LBM_FP32");
    lbm_vanse3d* h = new lbm_vanse3d();
    h->prm = *p;
    h->stream = (cudaStream_t)stream;
    h->geo = Geo{p->nx, p->ny, p->nz, N, p->bc_y == LBM_BC_BOUNCEBACK ? 1 : 0};
    h->fp64 = p->storage == LBM_FP64;
    h->tb = h->fp64 ? sizeof(double) : sizeof(float);
    const double s_nu = 1.0 / p->tau_nu, nu = (p->tau_nu - 0.5) / 3.0;
    const double s_e = p->s_e > 0.0 ? p->s_e : 1.0 / (nu + 0.5);   // nu_e = nu/3
    const double s[Q] = {1.0, s_e, p->s_eps, 1.0, p->s_q, 1.0, p->s_q, 1.0, p->s_q, s_nu,
                         p->s_pi, s_nu, p->s_pi, s_nu, s_nu, s_nu, p->s_m, p->s_m, p->s_m};
    for (int k = 0; k < Q; ++k) h->s[k] = s[k];
    cudaError_t e;
    struct A { void** p; size_t b; } allocs[] = {
        {&h->f[0], Q * N * h->tb}, {&h->f[1], Q * N * h->tb}, {&h->phi, N * h->tb}, {&h->phin, N * h->tb},
        {&h->fb, 3 * N * h->tb}, {&h->rho, N * h->tb}, {&h->j, 3 * N * h->tb}, {&h->u, 3 * N * h->tb},
        {&h->F, 3 * N * h->tb}, {(void**)&h->red, 4 * sizeof(double)}, {(void**)&h->bad, sizeof(int)}};
    for (auto& a : allocs) {
        e = cudaMalloc(a.p, a.b);
        if (e != cudaSuccess) {
            cudaGetLastError();
            g_err3 = std::string("cudaMalloc: ") + cudaGetErrorString(e);
            lbm_vanse3d_destroy(h);
            return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
        }
    }
    *out = h;
    return LBM_OK;
}

extern "C" lbm_status lbm_vanse3d_set_void_fraction(lbm_vanse3d_t h, const double* phi_t, const double* phi_next,
                                                    int on_device) {
    if (!h) return fail3(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!phi_t) return fail3(h, LBM_ERR_ARG, "phi_t is NULL");
    const long long N = h->geo.N;
    const double* srcs[2] = {phi_t, phi_next};
    const double* staged[2] = {nullptr, nullptr};
    double* owned[2] = {nullptr, nullptr};
    // stage and check both fields before either replaces the lattice's own
    lbm_status st = LBM_OK;
    CK3(h, cudaMemsetAsync(h->bad, 0, sizeof(int), h->stream));
    for (int k = 0; k < 2 && st == LBM_OK; ++k) {
        if (!srcs[k]) continue;
        st = stage_in3(h, srcs[k], N, on_device, &staged[k], &owned[k]);
        if (st == LBM_OK)
            v3_check_phi<<<blocks_for(N, 256) < 2048 ? blocks_for(N, 256) : 2048, 256, 0, h->stream>>>(staged[k], N,
                                                                                                     h->bad);
    }
    int bad = 0;
    if (st == LBM_OK) {
        cudaError_t e = cudaMemcpyAsync(&bad, h->bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) st = fail3(h, LBM_ERR_CUDA, "void fraction check: %s", cudaGetErrorString(e));
        else if (bad) st = fail3(h, LBM_ERR_ARG, "void fraction outside (0, 1]");
    }
    if (st == LBM_OK) {
        if (h->initialised) {   // keep the populations: d_0 follows the new rest value
            const unsigned nb = blocks_for(N, 256) < 4096 ? blocks_for(N, 256) : 4096;
            if (h->fp64)
                v3_rebase<double><<<nb, 256, 0, h->stream>>>(staged[0], (double*)h->phi, (double*)h->f[h->cur],
                                                             h->prm.rho0, N);
            else
                v3_rebase<float><<<nb, 256, 0, h->stream>>>(staged[0], (float*)h->phi, (float*)h->f[h->cur],
                                                            (float)h->prm.rho0, N);
        } else {
            convert_in(h, staged[0], h->phi, N);
        }
        if (staged[1]) convert_in(h, staged[1], h->phin, N);
    }
    for (double* o : owned)
        if (o) cudaFreeAsync(o, h->stream);
    if (st != LBM_OK) return st;
    CK3(h, cudaGetLastError());
    h->phi_set = true;
    h->phin_set = phi_next != nullptr;
    return LBM_OK;
}

extern "C" lbm_status lbm_vanse3d_set_body_force(lbm_vanse3d_t h, double gx, double gy, double gz,
                                                 const double* field, int on_device) {
    if (!h) return fail3(nullptr, LBM_ERR_ARG, "handle is NULL");
    h->g[0] = gx;
    h->g[1] = gy;
    h->g[2] = gz;
    h->fb_set = false;
    if (field) {
        const double* d;
        double* owned;
        lbm_status st = stage_in3(h, field, 3 * h->geo.N, on_device, &d, &owned);
        if (st != LBM_OK) return st;
        convert_in(h, d, h->fb, 3 * h->geo.N);
        if (owned) CK3(h, cudaFreeAsync(owned, h->stream));
        CK3(h, cudaGetLastError());
        h->fb_set = true;
    }
    return LBM_OK;
}

template <typename T>
static void enqueue_init(lbm_vanse3d* h) {
    const Geo& g = h->geo;
    v3_force<T><<<blocks_for(g.N, 256), 256, 0, h->stream>>>(
        (const T*)h->rho, (const T*)h->phi, h->fb_set ? (const T*)h->fb : nullptr, (T)h->g[0], (T)h->g[1],
        (T)h->g[2], (T)h->prm.kappa, (T*)h->F, g);
    v3_init<T><<<blocks_for(g.N, 128), 128, 0, h->stream>>>((T*)h->f[h->cur], (const T*)h->rho, (const T*)h->u,
                                                            (const T*)h->F, (const T*)h->phi, (T)h->prm.kappa,
                                                            (T)h->prm.rho0, g);
}

extern "C" lbm_status lbm_vanse3d_init_fields(lbm_vanse3d_t h, const double* rho, const double* ux,
                                              const double* uy, const double* uz, int on_device) {
    if (!h) return fail3(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!rho || !ux || !uy || !uz) return fail3(h, LBM_ERR_ARG, "a field is NULL");
    if (!h->phi_set) return fail3(h, LBM_ERR_STATE, "set the void fraction before init_fields");
    const long long N = h->geo.N;
    const double* srcs[4] = {rho, ux, uy, uz};
    char* ub = (char*)h->u;
    void* dsts[4] = {h->rho, ub, ub + N * h->tb, ub + 2 * N * h->tb};
    for (int k = 0; k < 4; ++k) {
        const double* d;
        double* owned;
        lbm_status st = stage_in3(h, srcs[k], N, on_device, &d, &owned);
        if (st != LBM_OK) return st;
        convert_in(h, d, dsts[k], N);
        if (owned) CK3(h, cudaFreeAsync(owned, h->stream));
    }
    h->cur = 0;
    if (h->fp64) enqueue_init<double>(h); else enqueue_init<float>(h);
    CK3(h, cudaGetLastError());
    h->initialised = true;
    h->steps = 0;
    return LBM_OK;
}

extern "C" lbm_status lbm_vanse3d_step(lbm_vanse3d_t h, int nsteps) {
    if (!h) return fail3(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (nsteps < 0) return fail3(h, LBM_ERR_ARG, "nsteps must be >= 0");
    if (!h->initialised) return fail3(h, LBM_ERR_STATE, "lattice not initialised");
    for (int s = 0; s < nsteps; ++s) {
        if (h->fp64) enqueue_step<double>(h); else enqueue_step<float>(h);
        CK3(h, cudaGetLastError());
        h->cur = 1 - h->cur;
        ++h->steps;
        if (h->phin_set) {   // phi(t) <- phi(t+1); steady afterwards
            std::swap(h->phi, h->phin);
            h->phin_set = false;
        }
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_vanse3d_sync(lbm_vanse3d_t h) {
    if (!h) return fail3(nullptr, LBM_ERR_ARG, "handle is NULL");
    CK3(h, cudaStreamSynchronize(h->stream));
    CK3(h, cudaGetLastError());
    return LBM_OK;
}

// device values out to the caller as doubles: plus `offset`, or, for the populations
// (pops = true), plus their rest state
static lbm_status copy_out(lbm_vanse3d* h, const void* src, double* dst, long long n, int on_device,
                           double offset = 0.0, bool pops = false) {
    double* d = dst;
    if (!on_device) CK3(h, cudaMallocAsync((void**)&d, n * sizeof(double), h->stream));
    const unsigned nb = blocks_for(n, 256) < 4096 ? blocks_for(n, 256) : 4096;
    const double k = h->prm.kappa, r0 = h->prm.rho0;
    if (pops) {
        if (h->fp64)
            v3_pop_io<double, double, double><<<nb, 256, 0, h->stream>>>((const double*)src, d, (const double*)h->phi,
                                                                         k, r0, 1.0, h->geo.N);
        else
            v3_pop_io<float, double, float><<<nb, 256, 0, h->stream>>>((const float*)src, d, (const float*)h->phi, k,
                                                                       r0, 1.0, h->geo.N);
    } else if (h->fp64) {
        v3_convert<double, double><<<nb, 256, 0, h->stream>>>((const double*)src, d, n, offset);
    } else {
        v3_convert<float, double><<<nb, 256, 0, h->stream>>>((const float*)src, d, n, offset);
    }
    CK3(h, cudaGetLastError());
    if (!on_device) {
        CK3(h, cudaMemcpyAsync(dst, d, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK3(h, cudaFreeAsync(d, h->stream));
        CK3(h, cudaStreamSynchronize(h->stream));
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_vanse3d_get_populations(lbm_vanse3d_t h, double* f, int on_device) {
    if (!h) return fail3(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!f) return fail3(h, LBM_ERR_ARG, "f is NULL");
    if (!h->initialised) return fail3(h, LBM_ERR_STATE, "lattice not initialised");
    return copy_out(h, h->f[h->cur], f, Q * h->geo.N, on_device, 0.0, true);
}

extern "C" lbm_status lbm_vanse3d_set_populations(lbm_vanse3d_t h, const double* f, int on_device) {
    if (!h) return fail3(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!f) return fail3(h, LBM_ERR_ARG, "f is NULL");
    if (!h->phi_set) return fail3(h, LBM_ERR_STATE, "set the void fraction before set_populations");
    const double* d;
    double* owned;
    lbm_status st = stage_in3(h, f, Q * h->geo.N, on_device, &d, &owned);
    if (st != LBM_OK) return st;
    h->cur = 0;
    {
        const long long n = Q * h->geo.N;
        const unsigned nb = blocks_for(n, 256) < 4096 ? blocks_for(n, 256) : 4096;
        const double k = h->prm.kappa, r0 = h->prm.rho0;
        if (h->fp64)
            v3_pop_io<double, double, double><<<nb, 256, 0, h->stream>>>(d, (double*)h->f[0], (const double*)h->phi, k,
                                                                         r0, -1.0, h->geo.N);
        else
            v3_pop_io<double, float, float><<<nb, 256, 0, h->stream>>>(d, (float*)h->f[0], (const float*)h->phi, k, r0,
                                                                       -1.0, h->geo.N);
    }
    if (owned) CK3(h, cudaFreeAsync(owned, h->stream));
    CK3(h, cudaGetLastError());
    h->initialised = true;
    h->steps = 0;
    return LBM_OK;
}

extern "C" lbm_status lbm_vanse3d_macros(lbm_vanse3d_t h, double* rho, double* u, int on_device) {
    if (!h) return fail3(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!h->initialised) return fail3(h, LBM_ERR_STATE, "lattice not initialised");
    const Geo& g = h->geo;
    if (h->fp64) {
        v3_moments<double><<<blocks_for(g.N, 256), 256, 0, h->stream>>>((const double*)h->f[h->cur],
                                                                         (const double*)h->phi, (double*)h->rho,
                                                                         (double*)h->j, g);
        v3_velocity<double><<<blocks_for(g.N, 256), 256, 0, h->stream>>>(
            (const double*)h->rho, (const double*)h->j, (const double*)h->phi,
            h->fb_set ? (const double*)h->fb : nullptr, h->g[0], h->g[1], h->g[2], h->prm.kappa, h->prm.rho0,
            (double*)h->u, (double*)h->F, g);
    } else {
        v3_moments<float><<<blocks_for(g.N, 256), 256, 0, h->stream>>>((const float*)h->f[h->cur],
                                                                        (const float*)h->phi, (float*)h->rho,
                                                                        (float*)h->j, g);
        v3_velocity<float><<<blocks_for(g.N, 256), 256, 0, h->stream>>>(
            (const float*)h->rho, (const float*)h->j, (const float*)h->phi,
            h->fb_set ? (const float*)h->fb : nullptr, (float)h->g[0], (float)h->g[1], (float)h->g[2],
            (float)h->prm.kappa, (float)h->prm.rho0, (float*)h->u, (float*)h->F, g);
    }
    CK3(h, cudaGetLastError());
    lbm_status st = LBM_OK;
    if (rho) st = copy_out(h, h->rho, rho, g.N, on_device, h->prm.rho0);   // the scratch holds rho - rho0
    if (st == LBM_OK && u) st = copy_out(h, h->u, u, 3 * g.N, on_device);
    return st;
}

extern "C" lbm_status lbm_vanse3d_reduce(lbm_vanse3d_t h, double* mass, double* mom) {
    if (!h) return fail3(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!h->initialised) return fail3(h, LBM_ERR_STATE, "lattice not initialised");
    CK3(h, cudaMemsetAsync(h->red, 0, 4 * sizeof(double), h->stream));
    const unsigned nb = blocks_for(h->geo.N, 256) < 1024 ? blocks_for(h->geo.N, 256) : 1024;
    if (h->fp64)
        v3_reduce<double><<<nb, 256, 0, h->stream>>>((const double*)h->f[h->cur], (const double*)h->phi, h->prm.rho0,
                                                     h->geo.N, h->red);
    else
        v3_reduce<float><<<nb, 256, 0, h->stream>>>((const float*)h->f[h->cur], (const float*)h->phi, h->prm.rho0,
                                                    h->geo.N, h->red);
    CK3(h, cudaGetLastError());
    double r[4];
    CK3(h, cudaMemcpyAsync(r, h->red, sizeof r, cudaMemcpyDeviceToHost, h->stream));
    CK3(h, cudaStreamSynchronize(h->stream));
    if (mass) *mass = r[0];
    if (mom) { mom[0] = r[1]; mom[1] = r[2]; mom[2] = r[3]; }
    for (double v : r)
        if (!std::isfinite(v)) return fail3(h, LBM_ERR_DIVERGED, "non-finite populations (mass %g)", r[0]);
    return LBM_OK;
}

extern "C" long long lbm_vanse3d_step_count(lbm_vanse3d_t h) { return h ? h->steps : -1; }
