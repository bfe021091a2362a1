// vanse_aux.cuh -- the non-hot kernels: field padding, initial populations,
// population get/set, macroscopic fields and FP64 reductions.
//
// Storage convention (shared with the step kernel): population plane i, padded
// row pitch P, cell (x, y) at i*plane + y*P + kPadCols + x, holding f_i+(x, t-1);
// cell x at time t pulls f_i(x, t) = f_i+(x - e_i, t-1), or, across a half-way
// bounce-back wall, f_opp(i)+(x, t-1). Periodic x is served by kGhost ghost
// columns on each side, rewritten whenever a cell near the edge is written.
#pragma once

#include "vanse_common.cuh"

namespace lbmv {

template <typename R>
struct Lattice {
    long long plane;   // elements per padded plane
    int nx, ny, P;
    int wall_y, model_b;
    int wall_x = 0;                    // half-way bounce-back walls at x = -1/2, nx - 1/2
    R kappa, gx, gy;
    R scale, inv_scale;
    Rest<R> rest;
    int eq2 = 0;                       // App. B equilibrium (B1) instead of Eq. (14)
    int has_drag = 0;                  // F^B += -beta (u - u_s), beta = phi^2 (d0 + d1 (1 - phi))
    R drag_d0 = 0, drag_d1 = 0, us_x = 0, us_y = 0;
    int has_solid = 0;                 // cells with phi = 0 are solid (half-way bounce-back links)
    // momentum base (FP16 / BF16 on the one-warp kernel): slot (i, c) holds the deviation
    // from f_i^rest + 3 w_i e_i . J(c), J(c) the post-collision momentum of cell c stored
    // (scaled like the deviations) in planes 9 (x) and 10 (y) of the same buffer
    int jbase = 0;
};

// the linear drag coefficient beta(phi) of a lattice (0 without drag)
template <typename R>
__device__ __forceinline__ R drag_beta(const Lattice<R>& L, R ph) {
    return L.has_drag ? ph * ph * (L.drag_d0 + L.drag_d1 * ((R)1 - ph)) : (R)0;
}

__device__ __forceinline__ long long cell_off(int P, int x, int y) { return (long long)y * P + kPadCols + x; }

// Write v at padded column x of row y and at every periodic ghost image of x.
template <typename T>
__device__ __forceinline__ void put_with_ghosts(T* plane_base, int P, int nx, int x, int y, T v) {
    const long long ro = (long long)y * P + kPadCols;
    plane_base[ro + x] = v;
    for (int g = x - nx; g >= -kGhost; g -= nx) plane_base[ro + g] = v;
    for (int g = x + nx; g < nx + kGhost; g += nx) plane_base[ro + g] = v;
}

// Periodic ghost columns of the 9 population planes, refreshed from the columns
// they image: column g in [-kGhost, 0) and [nx, nx + kGhost) takes column g mod nx
// (a verbatim copy: an FP16 / BF16 value stays encoded against the same phi, whose
// ghosts are images too). Runs after a step kernel that writes columns 0 .. nx-1
// only. One thread per (plane, row, ghost column).
template <typename S>
__device__ __forceinline__ void fill_ghosts(S* __restrict__ buf, long long plane, int nx, int ny, int P, long long k) {
    const int g6 = (int)(k % (2 * kGhost));
    const long long rest = k / (2 * kGhost);
    const int y = (int)(rest % ny), i = (int)(rest / ny);
    const int g = g6 < kGhost ? g6 - kGhost : nx + g6 - kGhost;
    const int sx = ((g % nx) + nx) % nx;
    S* row = buf + i * plane + (long long)y * P + kPadCols;
    row[g] = row[sx];
}

// step_ctr (optional): the one-warp kernel's step count, advanced here once per step
// (it seeds the stochastic rounding of FP16/BF16 stores).
// npl: the planes of the buffer (9 populations, 11 with the momentum base's J planes).
template <typename S>
__global__ void ghost_fill_kernel(S* __restrict__ buf, long long plane, int nx, int ny, int P,
                                  unsigned* __restrict__ step_ctr = nullptr, int npl = 9) {
    const long long n = (long long)npl * ny * 2 * kGhost;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        fill_ghosts<S>(buf, plane, nx, ny, P, k);
    if (step_ctr && blockIdx.x == 0 && threadIdx.x == 0) *step_ctr += 1u;
}

// Solid-cell tiles of the one-warp kernel: per CTA (its 60 columns x0 .., its strip's
// rows y0 .. y1-1), 1 when the void fraction phi(t) or phi(t+1) is 0 anywhere in what
// the CTA stages: rows y0-3 .. y1+2 (past a y wall none, periodic rows wrapped) and
// columns x0-3 .. x0+63 that lie within the lattice or its ghost columns (the columns
// beyond hold no value a written cell reads). One CTA per tile.
template <typename R>
__global__ void solid_tiles_kernel(const R* __restrict__ phi, const R* __restrict__ phin,
                                   unsigned char* __restrict__ tiles, int nx, int ny, int P, int W, int H,
                                   int wall_y) {
    const int x0 = blockIdx.x * W, y0 = blockIdx.y * H, y1 = min(y0 + H, ny);
    const int xlo = x0 - kGhost, xhi = min(x0 + 64, nx + kGhost);
    const int ncol = xhi - xlo, nrow = (y1 + 2) - (y0 - 3) + 1;
    int found = 0;
    for (int k = threadIdx.x; k < nrow * ncol; k += blockDim.x) {
        int y = y0 - 3 + k / ncol;
        const int x = xlo + k % ncol;
        if (y < 0 || y >= ny) {
            if (wall_y) continue;
            y = ((y % ny) + ny) % ny;
        }
        const long long o = (long long)y * P + kPadCols + x;
        if (phi[o] == (R)0 || (phin && phin[o] == (R)0)) found = 1;
    }
    found = __syncthreads_or(found);
    if (threadIdx.x == 0) tiles[blockIdx.y * gridDim.x + blockIdx.x] = (unsigned char)(found != 0);
}

// The launch order of the tiles: those with solid cells first (their CTAs take the
// longer solid path, and started first they overlap the others instead of trailing
// them), then the rest. cnt[0..1] must be zero on entry. One thread per tile.
__global__ void solid_order_kernel(const unsigned char* __restrict__ tiles, int n, int* __restrict__ order,
                                   int* __restrict__ cnt) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        if (tiles[t]) order[atomicAdd(cnt, 1)] = t;
        else order[n - 1 - atomicAdd(cnt + 1, 1)] = t;
    }
}

// Void-fraction check of a dense field before it replaces the lattice's: every value
// must lie in [0, 1]; NaN fails. (Zeros are solid cells: without solid cells enabled
// they are reported later, by the sync-time check of pad_field_kernel's flag.) Sets
// the bit `which` of *bad when any value fails; block size a multiple of 32.
template <typename T>
__global__ void check_phi_kernel(const T* __restrict__ src, long long n, int which, int* __restrict__ bad) {
    bool ok = true;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const T v = src[k];
        ok = ok && v >= (T)0 && v <= (T)1;
    }
    if (!__all_sync(0xffffffffu, ok) && (threadIdx.x & 31) == 0) atomicOr(bad, which);
}

// Copy a dense [ny][nx] field (double or float) into a padded R field (with
// ghosts). Rows are dealt to blocks and columns to threads (32-bit indices).
// zero_seen (optional): set to 1 when a value is exactly zero (a solid cell in phi).
template <typename Tin, typename R>
__global__ void pad_field_kernel(const Tin* __restrict__ src, R* __restrict__ dst, int nx, int ny, int P,
                                 int* __restrict__ zero_seen = nullptr) {
    bool zero = false;
    for (int y = blockIdx.x; y < ny; y += gridDim.x) {
        const Tin* row = src + (long long)y * nx;
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const R v = (R)row[x];
            zero = zero || v == (R)0;
            put_with_ghosts<R>(dst, P, nx, x, y, v);
        }
    }
    if (zero_seen && zero) *zero_seen = 1;
}

// Replace phi(t) of a lattice that already holds FP32/FP16/BF16 populations. Those
// store f_0 as a deviation from the rest value (phi - 5 kappa / 9) rho0 of the
// lattice's current phi, so where phi changes the stored deviation moves by
// (phi_old - phi_new) rho0 (times the storage scale) and the populations themselves
// stay as they are, as with FP64 storage. Cells whose phi is unchanged are not
// written. Each thread reads only its interior cell and writes that cell and its
// ghost images.
template <typename Tin, typename R, typename S>
__global__ void pad_phi_rebase_kernel(const Tin* __restrict__ src, R* __restrict__ phi, S* __restrict__ plane0,
                                      int nx, int ny, int P, R rho0_scaled, int* __restrict__ zero_seen) {
    bool zero = false;
    for (int y = blockIdx.x; y < ny; y += gridDim.x) {
        const Tin* row = src + (long long)y * nx;
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const R v = (R)row[x];
            zero = zero || v == (R)0;
            const long long o = cell_off(P, x, y);
            const R old = phi[o];
            if (old != v) {
                const R d = dec(plane0[o], (R)0, (R)1) + (old - v) * rho0_scaled;
                put_with_ghosts<S>(plane0, P, nx, x, y, enc<S, R>(d, (R)0, (R)1));
                put_with_ghosts<R>(phi, P, nx, x, y, v);
            }
        }
    }
    if (zero_seen && zero) *zero_seen = 1;
}

// Pull the post-streaming populations of cell (x, y) from the stored planes.
// With solid cells: a solid cell has no populations (zeros), and a population whose
// source cell is solid comes back from the half-way link (opposite slot, same cell).
// T: the type f is decoded to (R, or double for the read-back kernels, with the rest
// values of a Lattice<double>).
template <typename S, typename R, typename T = R>
__device__ __forceinline__ void pull_cell(const S* __restrict__ buf, const R* __restrict__ phi, const Lattice<T>& L,
                                          int x, int y, T f[9]) {
    const T ph = (T)phi[cell_off(L.P, x, y)];
    if (L.has_solid && ph == (T)0) {
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = (T)0;
        return;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int sx = x - ex_of(i), sy = y - ey_of(i);
        int pi = i;
        if (L.wall_x && (sx < 0 || sx >= L.nx)) { sx = x; sy = y; pi = opp_of(i); }
        if (sy < 0 || sy >= L.ny) {
            if (L.wall_y) { sx = x; sy = y; pi = opp_of(i); }
            else sy = (sy + L.ny) % L.ny;
        }
        if (L.has_solid && pi == i && phi[cell_off(L.P, sx, sy)] == (R)0) { sx = x; sy = y; pi = opp_of(i); }
        const long long so = cell_off(L.P, sx, sy);
        const S v = buf[pi * L.plane + so];
        const T rest = (i == 0) ? L.rest.r0(ph) : L.rest.ri(i);
        f[i] = dec_as<T>(v, rest, L.inv_scale);
        if (L.jbase && pi != 0) {
            // the slot's own base: 3 w_pi e_pi . J of the cell it sits in
            const T jx = dec_as<T>(buf[9 * L.plane + so], (T)0, L.inv_scale);
            const T jy = dec_as<T>(buf[10 * L.plane + so], (T)0, L.inv_scale);
            f[i] += w3_of<T>(pi) * ((T)ex_of(pi) * jx + (T)ey_of(pi) * jy);
        }
    }
}

// Store post-streaming value f_i(x, y) where the next pull will find it (the value,
// rest state and deviation in T: R, or double for the write-back kernel).
template <typename S, typename R, typename T = R>
__device__ __forceinline__ void scatter_cell(S* __restrict__ buf, const Lattice<T>& L, int x, int y, int i, T fi,
                                             T phi_cell, const R* __restrict__ phi = nullptr) {
    int tx = x - ex_of(i), ty = y - ey_of(i);
    int pi = i;
    if (L.wall_x && (tx < 0 || tx >= L.nx)) { tx = x; ty = y; pi = opp_of(i); }
    if (ty < 0 || ty >= L.ny) {
        if (L.wall_y) { tx = x; ty = y; pi = opp_of(i); }
        else ty = (ty + L.ny) % L.ny;
    }
    if (L.has_solid && pi == i && phi[cell_off(L.P, tx, ty)] == (R)0) { tx = x; ty = y; pi = opp_of(i); }
    tx = (tx + L.nx) % L.nx;
    const T rest = (i == 0) ? L.rest.r0(phi_cell) : L.rest.ri(i);
    put_with_ghosts<S>(buf + pi * L.plane, L.P, L.nx, tx, ty, enc<S, T>(fi, rest, L.scale));
}

// the row a stencil row y + dy maps to: periodic wrap, or the mirror row at a wall
template <typename R>
__device__ __forceinline__ int map_row(const Lattice<R>& L, int yy) {
    if (yy < 0 || yy >= L.ny) {
        if (L.wall_y) return yy < 0 ? -1 - yy : 2 * L.ny - 1 - yy;
        return (yy + L.ny) % L.ny;
    }
    return yy;
}

// Eq. (10) on a dense [ny][nx] double field; rho-like (even) ghost rule at walls. With
// solid cells (phi = 0) a solid neighbour reads the mirrored value: an axis neighbour
// the cell itself, a diagonal one the mean of the fluid ones of its two axis images
// (the cell itself if both are solid).
template <typename R, typename PT = R>
__device__ __forceinline__ void grad_dense_even(const double* __restrict__ a, const Lattice<R>& L, int x, int y, R& gx,
                                                R& gy, const PT* __restrict__ phi = nullptr) {
    R sx = 0, sy = 0;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        int nx_ = x + ex_of(i);
        if (nx_ < 0 || nx_ >= L.nx) nx_ = L.wall_x ? (nx_ < 0 ? -1 - nx_ : 2 * L.nx - 1 - nx_) : (nx_ + L.nx) % L.nx;
        int ny_ = map_row(L, y + ey_of(i));
        const R w = (i <= 4) ? (R)(1.0 / 9.0) : (R)(1.0 / 36.0);
        R v = (R)a[(long long)ny_ * L.nx + nx_];
        if (L.has_solid && phi[cell_off(L.P, nx_, ny_)] == (PT)0) {
            const R own = (R)a[(long long)y * L.nx + x];
            v = own;
            if (ex_of(i) != 0 && ey_of(i) != 0) {
                const int ax = nx_, by = map_row(L, y + ey_of(i));
                const bool fa = phi[cell_off(L.P, ax, y)] != (PT)0, fb_ = phi[cell_off(L.P, x, by)] != (PT)0;
                const R va = (R)a[(long long)y * L.nx + ax], vb = (R)a[(long long)by * L.nx + x];
                if (fa && fb_) v = (va + vb) / (R)2;
                else if (fa) v = va;
                else if (fb_) v = vb;
            }
        }
        sx += w * v * (R)ex_of(i);
        sy += w * v * (R)ey_of(i);
    }
    gx = (R)3 * sx;
    gy = (R)3 * sy;
}

// Initial populations f = f^eq(rho, u, phi) - F_i(u, F)/2 (Eq. 14, 6), F = F^p + F^B.
template <typename S, typename R>
__global__ void init_kernel(S* __restrict__ buf, const R* __restrict__ phi, const R* __restrict__ fb,
                            const double* __restrict__ rho_in, const double* __restrict__ ux_in,
                            const double* __restrict__ uy_in, const Lattice<R> L) {
    const long long n = (long long)L.nx * L.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / L.nx), x = (int)(k % L.nx);
        const long long co = cell_off(L.P, x, y);
        const R ph = phi[co];
        if (L.has_solid && ph == (R)0) continue;   // a solid cell holds no populations
        const R rho = (R)rho_in[k], ux = (R)ux_in[k], uy = (R)uy_in[k];
        R gx, gy;
        grad_dense_even<R>(rho_in, L, x, y, gx, gy, phi);
        const R kp = (L.model_b ? (L.kappa - (R)1) : (L.kappa - ph)) / (R)3;
        R Fx = kp * gx + ph * L.gx, Fy = kp * gy + ph * L.gy;
        if (fb) { Fx += fb[co]; Fy += fb[L.plane + co]; }
        const R beta = drag_beta(L, ph);
        Fx -= beta * (ux - L.us_x);
        Fy -= beta * (uy - L.us_y);
        const R X = L.kappa / ph;
        const R pr = ph * rho;
        const R uu = ux * ux + uy * uy;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const R exi = (R)ex_of(i), eyi = (R)ey_of(i);
            const R eu = exi * ux + eyi * uy;
            R feq;
            if (i == 0) {
                feq = pr - (R)(5.0 / 9.0) * L.kappa * rho - (R)(2.0 / 3.0) * pr * uu;
            } else {
                const R w = (i <= 4) ? (R)(1.0 / 9.0) : (R)(1.0 / 36.0);
                // Eq. (14): 1 + (X-1)(3|e|^2 - 4)/2 on the first-order term; (B1): 1
                const R g = L.eq2 ? (R)1 : ((i <= 4) ? ((R)3 - X) * (R)0.5 : X);
                feq = w * (L.kappa * rho + pr * ((R)3 * eu * g + (R)4.5 * eu * eu - (R)1.5 * uu));
            }
            const R w = (i == 0) ? (R)(4.0 / 9.0) : ((i <= 4) ? (R)(1.0 / 9.0) : (R)(1.0 / 36.0));
            const R Fi = w * (((R)3 * (exi - ux) + (R)9 * eu * exi) * Fx + ((R)3 * (eyi - uy) + (R)9 * eu * eyi) * Fy);
            scatter_cell<S, R>(buf, L, x, y, i, feq - (R)0.5 * Fi, ph, phi);
        }
    }
}

// Read-back and write-back of the post-streaming populations, decoded / encoded in
// FP64 (L: the lattice's Lattice<double>): a stored deviation d reads back as
// d / scale + f^rest with f^rest in FP64, so the value carries no rounding at the
// scale of f, and writing it back returns d.
template <typename S, typename R>
__global__ void get_pop_kernel(const S* __restrict__ buf, const R* __restrict__ phi, double* __restrict__ out,
                               const Lattice<double> L) {
    const long long n = (long long)L.nx * L.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / L.nx), x = (int)(k % L.nx);
        double f[9];
        pull_cell<S, R, double>(buf, phi, L, x, y, f);
#pragma unroll
        for (int i = 0; i < 9; ++i) out[i * n + k] = f[i];
    }
}

template <typename S, typename R>
__global__ void set_pop_kernel(S* __restrict__ buf, const R* __restrict__ phi, const double* __restrict__ in,
                               const Lattice<double> L) {
    const long long n = (long long)L.nx * L.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / L.nx), x = (int)(k % L.nx);
        const double ph = (double)phi[cell_off(L.P, x, y)];
        if (L.has_solid && ph == 0.0) continue;
#pragma unroll
        for (int i = 0; i < 9; ++i) scatter_cell<S, R, double>(buf, L, x, y, i, in[i * n + k], ph, phi);
    }
}

// Macroscopic pass 1: rho = sum f / phi (Eq. 7) into a dense double array.
// (Both macroscopic passes decode and compute in FP64 for every storage, L being
// the lattice's Lattice<double>: off the step path, and free of FP32 rounding at
// the scale of f.)
template <typename S, typename R>
__global__ void rho_kernel(const S* __restrict__ buf, const R* __restrict__ phi, double* __restrict__ rho,
                           const Lattice<double> L) {
    const long long n = (long long)L.nx * L.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / L.nx), x = (int)(k % L.nx);
        double f[9];
        pull_cell<S, R, double>(buf, phi, L, x, y, f);
        double s = 0;
#pragma unroll
        for (int i = 0; i < 9; ++i) s += f[i];
        const double ph = (double)phi[cell_off(L.P, x, y)];
        rho[k] = (L.has_solid && ph == 0.0) ? 0.0 : s / ph;
    }
}

// Macroscopic pass 2: F = F^p + F^B (Eq. 13), u = (sum e f + F/2) / sum f, p = rho/3.
template <typename S, typename R>
__global__ void vel_kernel(const S* __restrict__ buf, const R* __restrict__ phi, const R* __restrict__ fb,
                           const double* __restrict__ rho, double* __restrict__ ux, double* __restrict__ uy,
                           double* __restrict__ pr, const Lattice<double> L) {
    const long long n = (long long)L.nx * L.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / L.nx), x = (int)(k % L.nx);
        const long long co = cell_off(L.P, x, y);
        double f[9];
        pull_cell<S, R, double>(buf, phi, L, x, y, f);
        double s = 0, jx = 0, jy = 0;
#pragma unroll
        for (int i = 0; i < 9; ++i) { s += f[i]; jx += (double)ex_of(i) * f[i]; jy += (double)ey_of(i) * f[i]; }
        const double ph = (double)phi[co];
        if (L.has_solid && ph == 0.0) {   // a solid cell reports zeros
            if (ux) ux[k] = 0.0;
            if (uy) uy[k] = 0.0;
            if (pr) pr[k] = 0.0;
            continue;
        }
        double gx, gy;
        grad_dense_even<double>(rho, L, x, y, gx, gy, phi);
        const double kp = (L.model_b ? (L.kappa - 1.0) : (L.kappa - ph)) / 3.0;
        double Fx = kp * gx + ph * L.gx, Fy = kp * gy + ph * L.gy;
        if (fb) { Fx += (double)fb[co]; Fy += (double)fb[L.plane + co]; }
        // Eq. (7) with the drag -beta (u - u_s) inside F, solved for u
        const double beta = drag_beta(L, ph);
        if (ux) ux[k] = (jx + 0.5 * (Fx + beta * L.us_x)) / (s + 0.5 * beta);
        if (uy) uy[k] = (jy + 0.5 * (Fy + beta * L.us_y)) / (s + 0.5 * beta);
        if (pr) pr[k] = rho[k] / 3.0;
    }
}

// FP64 block reduction of three sums into partial[blockIdx.x * 3 + j].
__device__ __forceinline__ void block_reduce3(double a, double b, double c, double* partial) {
    __shared__ double sh[3][32];
    a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sh[0][wid] = a; sh[1][wid] = b; sh[2][wid] = c; }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        a = lane < nw ? sh[0][lane] : 0.0;
        b = lane < nw ? sh[1][lane] : 0.0;
        c = lane < nw ? sh[2][lane] : 0.0;
        a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
        if (lane == 0) { partial[blockIdx.x * 3 + 0] = a; partial[blockIdx.x * 3 + 1] = b; partial[blockIdx.x * 3 + 2] = c; }
    }
}

// Mass sum f and momentum sum e f of one cell's nine populations, in the compute
// type R. Used by both reductions below so that their per-cell terms are identical.
template <typename R>
__device__ __forceinline__ void cell_moments(const R f[9], R& m, R& jx, R& jy) {
    m = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    jx = (f[1] - f[3]) + ((f[5] - f[6]) + (f[8] - f[7]));
    jy = (f[2] - f[4]) + ((f[5] + f[6]) - (f[7] + f[8]));
}

// Compensated (Kahan) accumulation in R: s + c carries the sum to about one ulp of s
// however many terms are added.
template <typename R>
__device__ __forceinline__ void kahan_add(R& s, R& c, R v) {
    const R y = v - c;
    const R t = s + y;
    c = (t - s) - y;
    s = t;
}

// This thread's share of row y (columns threadIdx.x, + blockDim.x, ...): the three
// sums of cell_moments, accumulated in R with compensation and added to m, jx, jy
// in FP64. The FP64 pipe runs at a small fraction of the FP32 rate on this part, so
// it sees three additions per thread and row instead of three per cell. Both
// reductions below call this with the same block size, so their per-thread terms
// are identical.
template <typename S, typename R>
__device__ __forceinline__ void row_thread_moments(const S* __restrict__ buf, const R* __restrict__ phi,
                                                   const Lattice<R>& L, int y, double& m, double& jx, double& jy) {
    R sm = 0, sx = 0, sy = 0, cm = 0, cx = 0, cy = 0;
    for (int x = threadIdx.x; x < L.nx; x += blockDim.x) {
        R f[9], vm, vx, vy;
        pull_cell<S, R>(buf, phi, L, x, y, f);
        cell_moments(f, vm, vx, vy);
        kahan_add(sm, cm, vm);
        kahan_add(sx, cx, vx);
        kahan_add(sy, cy, vy);
    }
    m += (double)sm - (double)cm;
    jx += (double)sx - (double)cx;
    jy += (double)sy - (double)cy;
}

// Mass and momentum sums, FP64 partial sums per block; rows are dealt to blocks and
// columns to threads (32-bit indices, coalesced pulls).
template <typename S, typename R>
__global__ void moments_reduce_kernel(const S* __restrict__ buf, const R* __restrict__ phi, double* __restrict__ partial,
                                      const Lattice<R> L) {
    double m = 0, jx = 0, jy = 0;
    for (int y = blockIdx.x; y < L.ny; y += gridDim.x) row_thread_moments<S, R>(buf, phi, L, y, m, jx, jy);
    block_reduce3(m, jx, jy, partial);
}

// Eq. (26) sums: sum |u - u_ref|^2 and sum |u_ref|^2 (third slot unused).
__global__ void velocity_error_kernel(const double* __restrict__ ux, const double* __restrict__ uy,
                                      const double* __restrict__ uxr, const double* __restrict__ uyr, long long n,
                                      double* __restrict__ partial) {
    double num = 0, den = 0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const double dx = ux[k] - uxr[k], dy = uy[k] - uyr[k];
        num += dx * dx + dy * dy;
        den += uxr[k] * uxr[k] + uyr[k] * uyr[k];
    }
    block_reduce3(num, den, 0.0, partial);
}

// Mass and momentum sums per lattice row: one partial triple per row, written to
// partial[3*y .. 3*y+2] (rows are shared out over the blocks, grid-stride). Every
// row 0..ny-1 gets its triple written, so the caller never needs to clear partial.
template <typename S, typename R>
__global__ void row_moments_kernel(const S* __restrict__ buf, const R* __restrict__ phi, double* __restrict__ partial,
                                   const Lattice<R> L) {
    __shared__ double sh[3][32];
    for (int y = blockIdx.x; y < L.ny; y += gridDim.x) {
        double m = 0, jx = 0, jy = 0;
        row_thread_moments<S, R>(buf, phi, L, y, m, jx, jy);
        m = warp_sum(m); jx = warp_sum(jx); jy = warp_sum(jy);
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) { sh[0][wid] = m; sh[1][wid] = jx; sh[2][wid] = jy; }
        __syncthreads();
        if (wid == 0) {
            const int nw = blockDim.x >> 5;
            m = lane < nw ? sh[0][lane] : 0.0;
            jx = lane < nw ? sh[1][lane] : 0.0;
            jy = lane < nw ? sh[2][lane] : 0.0;
            m = warp_sum(m); jx = warp_sum(jx); jy = warp_sum(jy);
            if (lane == 0) { partial[3 * y + 0] = m; partial[3 * y + 1] = jx; partial[3 * y + 2] = jy; }
        }
        __syncthreads();
    }
}

// Sum nblocks partial triples in a fixed order (deterministic) into out[0..2].
__global__ void finish_reduce_kernel(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
    double a = 0, b = 0, c = 0;
    for (int k = threadIdx.x; k < nblocks; k += blockDim.x) {
        a += partial[k * 3 + 0]; b += partial[k * 3 + 1]; c += partial[k * 3 + 2];
    }
    __shared__ double sh[3][32];
    a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sh[0][wid] = a; sh[1][wid] = b; sh[2][wid] = c; }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        a = lane < nw ? sh[0][lane] : 0.0;
        b = lane < nw ? sh[1][lane] : 0.0;
        c = lane < nw ? sh[2][lane] : 0.0;
        a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
        if (lane == 0) { out[0] = a; out[1] = b; out[2] = c; }
    }
}

}  // namespace lbmv
