// vanse_step.cuh -- the fused D2Q9 MRTLB-VANSE stream + collide kernel.
//
// One time step per launch, pull streaming between two SoA buffers (the source
// buffer holds the post-collision populations f+(x, t-1); cell x pulls
// f_i(x, t) = f_i+(x - e_i, t-1), Sec. 2.3), periodic x, periodic or half-way
// bounce-back y (Sec. 3.1).
//
// Work decomposition: a CTA of T threads owns W = T - 4 columns of a strip of
// rows and marches up the strip one row per iteration. Thread t sits on column
// x0 - 2 + t for the whole strip. The method's data dependency is radius 3 in
// the pre-stream populations (C at x needs grad u at x, u needs F^p = (kappa -
// phi) cs^2 grad rho at x +- e_i, rho needs the pulled populations there), so
// each iteration runs three phases that trail each other by one row:
//   phase 1, row p1:   pull the 9 populations, moments m = M f (Eq. 17, A1),
//                      rho = m_0 / phi (Eq. 7)              (columns x0-2 .. x0+W+1)
//   phase 2, row p1-1: grad rho (Eq. 10), F = F^p + F^B (Eq. 13), u (Eq. 7) and
//                      the fields rho u, u, phi rho u       (columns x0-1 .. x0+W)
//   phase 3, row p1-2: their Eq. (10) gradients, penalty C (Eq. 20), m^eq
//                      (Eq. 18), S (Eq. 19), relaxation (Eq. 16), f+ = M^-1 m+
//                      (A1) and the store                  (columns x0 .. x0+W-1)
// x-neighbours are exchanged through one shared-memory row per field; the y
// direction lives in registers: Eq. (10) factorises into a central difference
// times a [1 4 1]/6 smoothing across, so each field keeps, per row, its x-difference
// d = v(x+1) - v(x-1) and w = 4 v(x) + v(x+1) + v(x-1); then
//   d_x v(y) = (d(y-1) + 4 d(y) + d(y+1)) / 12,   d_y v(y) = (w(y+1) - w(y-1)) / 12.
// Three row states rotate through the unrolled loop, so no register moves occur.
//
// Source rows (9 population rows + phi, and phi(t+1) / the force field when
// present) are staged in an 8-slot shared-memory ring by 1-D bulk async copies
// (cp.async.bulk, completing on one mbarrier per slot) issued up to 4 rows ahead
// of the newest row in use.
#pragma once

#include "vanse_common.cuh"

namespace lbmv {

constexpr int kSlots = 8;              // ring slots (power of two)
constexpr uint32_t kWaitTries = 1u << 22;  // bounded mbarrier polls (seconds, far above a row's latency)

template <typename R>
struct StepParams {
    const void* src;      // source population planes (storage type), padded rows
    void* dst;            // destination population planes
    const R* phi;         // phi(x, t), padded rows
    const R* phin;        // phi(x, t+1) (== phi when steady)
    const R* fb;          // F^B field planes (x then y), padded rows, or nullptr
    long long plane;      // elements per population / field plane (ny * P)
    int nx, ny, P;        // lattice size, row pitch (elements)
    int W, H;             // output columns per CTA, rows per strip
    int wall_y, unsteady, has_fb, model_b;
    int slot_stride;      // bytes per ring slot
    int wwmax;            // elements per staged row
    R kappa, gx, gy;
    R s_c, s_e, s_eps, s_q, s_nu;
    R scale, inv_scale;   // deviation-storage scale (FP16/BF16)
    Rest<R> rest;
    int* err;             // set to 1 when a bounded wait gives up
};

// Per-row register state (see the header comment for who writes what when).
template <typename R>
struct RowState {
    R m[9];                        // moments of the pulled populations (phase 1)
    R rho;                         // rho (phase 1)
    R dr, wr;                      // x-difference / smoothed sum of rho (phase 2)
    R Fx, Fy, ux, uy;              // force and velocity (phase 2)
    R dAx, dBx, dBy, dDx;          // x-differences of rho u_x, u_x, u_y, phi rho u_x
    R wAy, wBy, wBx, wDy;          // smoothed sums of rho u_y, u_y, u_x, phi rho u_y
};

template <typename S, typename R>
struct StepCtx {
    const StepParams<R>& p;
    unsigned char* ring;
    uint64_t* bar;
    R* rbuf;       // rho row, T entries
    R* fbuf;       // 6 field rows, 6*T entries
    int* abort_flag;
    int t, T, xc, sc;   // thread, CTA size, global column, smem column
    int x0, y0, y1;
    int wsp, ww;        // staged window start (padded column) and width
    int rlo, rhi;       // source rows this CTA loads
    int nR;             // staged R rows per slot
    int waited;         // newest row waited for
    int issued;         // newest row issued (thread 0 only)

    __device__ __forceinline__ unsigned char* slot_of(int r) const { return ring + (r & (kSlots - 1)) * p.slot_stride; }
    __device__ __forceinline__ const S* pop_row(int r, int i) const {
        return reinterpret_cast<const S*>(slot_of(r)) + i * p.wwmax;
    }
    __device__ __forceinline__ const R* r_row(int r, int k) const {
        return reinterpret_cast<const R*>(slot_of(r) + 9 * p.wwmax * (int)sizeof(S)) + k * p.wwmax;
    }
    __device__ __forceinline__ bool row_valid(int r) const { return !p.wall_y || (r >= 0 && r < p.ny); }

    // thread 0: load source row r (all staged rows) into its slot
    __device__ __forceinline__ void issue(int r) {
        issued = r;
        uint64_t* b = &bar[r & (kSlots - 1)];
        int gr = r;
        if (!p.wall_y) { gr %= p.ny; if (gr < 0) gr += p.ny; }
        unsigned char* slot = slot_of(r);
        const uint32_t bs = (uint32_t)(ww * (int)sizeof(S));
        const uint32_t br = (uint32_t)(ww * (int)sizeof(R));
        mbar_expect_tx(b, 9u * bs + (uint32_t)nR * br);
        const S* src = reinterpret_cast<const S*>(p.src) + (long long)gr * p.P + wsp;
#pragma unroll
        for (int i = 0; i < 9; ++i)
            bulk_g2s(slot + i * p.wwmax * (int)sizeof(S), src + i * p.plane, bs, b);
        R* rr = reinterpret_cast<R*>(slot + 9 * p.wwmax * (int)sizeof(S));
        const long long off = (long long)gr * p.P + wsp;
        int k = 0;
        bulk_g2s(rr + (k++) * p.wwmax, p.phi + off, br, b);
        if (p.unsteady) bulk_g2s(rr + (k++) * p.wwmax, p.phin + off, br, b);
        if (p.has_fb) {
            bulk_g2s(rr + (k++) * p.wwmax, p.fb + off, br, b);
            bulk_g2s(rr + (k++) * p.wwmax, p.fb + p.plane + off, br, b);
        }
    }
    // all threads: make sure every source row up to r has landed
    __device__ __forceinline__ void wait_upto(int r) {
        r = min(r, rhi);
        while (waited < r) {
            ++waited;
            const uint32_t parity = (uint32_t)(((waited - rlo) >> 3) & 1);
            if (!mbar_wait_bounded(&bar[waited & (kSlots - 1)], parity, kWaitTries)) {
                *abort_flag = 1;
                atomicExch(p.err, 1);
            }
        }
    }
};

// Phase 1: pull + moments + rho for row r into st.
template <typename S, typename R>
__device__ __forceinline__ void phase1(StepCtx<S, R>& c, RowState<R>& st, int r) {
    const StepParams<R>& p = c.p;
    const int s = c.sc;
    const R phi = c.r_row(r, 0)[s];
    const Rest<R>& rs = p.rest;
    const R ia = p.inv_scale;
    const S* rc = nullptr;
    R f0, f1, f2, f3, f4, f5, f6, f7, f8;
    rc = c.pop_row(r, 0);
    f0 = dec(rc[s], rs.r0(phi), ia);
    f1 = dec(c.pop_row(r, 1)[s - 1], rs.ax, ia);
    f3 = dec(c.pop_row(r, 3)[s + 1], rs.ax, ia);
    if (p.wall_y && r == 0) {  // links from y = -1 come back from the wall: opposite slot, same cell
        f2 = dec(c.pop_row(r, 4)[s], rs.ax, ia);
        f5 = dec(c.pop_row(r, 7)[s], rs.dg, ia);
        f6 = dec(c.pop_row(r, 8)[s], rs.dg, ia);
    } else {
        f2 = dec(c.pop_row(r - 1, 2)[s], rs.ax, ia);
        f5 = dec(c.pop_row(r - 1, 5)[s - 1], rs.dg, ia);
        f6 = dec(c.pop_row(r - 1, 6)[s + 1], rs.dg, ia);
    }
    if (p.wall_y && r == p.ny - 1) {
        f4 = dec(c.pop_row(r, 2)[s], rs.ax, ia);
        f7 = dec(c.pop_row(r, 5)[s], rs.dg, ia);
        f8 = dec(c.pop_row(r, 6)[s], rs.dg, ia);
    } else {
        f4 = dec(c.pop_row(r + 1, 4)[s], rs.ax, ia);
        f7 = dec(c.pop_row(r + 1, 7)[s + 1], rs.dg, ia);
        f8 = dec(c.pop_row(r + 1, 8)[s - 1], rs.dg, ia);
    }
    // m = M f with the row structure of (A1)
    const R a13 = f1 + f3, a24 = f2 + f4, b57 = f5 + f7, b68 = f6 + f8;
    const R sax = a13 + a24, sdg = b57 + b68;
    const R d13 = f1 - f3, d24 = f2 - f4;
    const R dx = (f5 - f7) + (f8 - f6);
    const R dy = (f5 - f7) + (f6 - f8);
    st.m[0] = f0 + sax + sdg;
    st.m[1] = (R)-4 * f0 - sax + (R)2 * sdg;
    st.m[2] = (R)4 * f0 - (R)2 * sax + sdg;
    st.m[3] = d13 + dx;
    st.m[4] = (R)-2 * d13 + dx;
    st.m[5] = d24 + dy;
    st.m[6] = (R)-2 * d24 + dy;
    st.m[7] = a13 - a24;
    st.m[8] = b57 - b68;
    st.rho = st.m[0] / phi;
}

template <typename S, typename R, int T>
__global__ void __launch_bounds__(T) vanse_step_kernel(const __grid_constant__ StepParams<R> p) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_abort;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    R* rbuf = reinterpret_cast<R*>(smem + 128);
    R* fbuf = rbuf + T;
    const int ring_off = (128 + 7 * T * (int)sizeof(R) + 127) & ~127;
    unsigned char* ring = smem + ring_off;

    const int t = threadIdx.x;
    constexpr int A = 16 / (int)sizeof(S);
    const int x0 = blockIdx.x * p.W;
    const int y0 = blockIdx.y * p.H;
    const int y1 = min(y0 + p.H, p.ny);

    StepCtx<S, R> c{p, ring, bar, rbuf, fbuf, &s_abort, t, T, 0, 0, x0, y0, y1, 0, 0, 0, 0, 0, 0, 0};
    c.wsp = ((kPadCols + x0 - kGhost) / A) * A;
    c.ww = ((kPadCols + x0 + p.W + kGhost + A - 1) / A) * A - c.wsp;
    c.xc = x0 - 2 + t;
    c.sc = kPadCols + c.xc - c.wsp;
    c.nR = 1 + (p.unsteady ? 1 : 0) + (p.has_fb ? 2 : 0);
    c.rlo = y0 - 3;
    c.rhi = y1 + 2;
    if (p.wall_y) { c.rlo = max(c.rlo, 0); c.rhi = min(c.rhi, p.ny - 1); }
    c.waited = c.rlo - 1;
    c.issued = c.rlo - 1;

    if (t == 0) {
        s_abort = 0;
        for (int k = 0; k < kSlots; ++k) mbar_init(&bar[k], 1);
        fence_mbar_init();
        for (int r = c.rlo; r <= min(y0 + 2, c.rhi); ++r) c.issue(r);
    }
    __syncthreads();

    const R kappa = p.kappa;
    const R third = (R)1 / (R)3;
    const R twelfth = (R)1 / (R)12;
    const bool ph3_thread = (t >= 2 && t < T - 2);
    const bool ph2_thread = (t >= 1 && t < T - 1);

    RowState<R> s0, s1, s2;

    // one iteration: new row p1 -> A, row p1-1 -> B, row p1-2 -> Cs
    auto iter = [&](RowState<R>& An, RowState<R>& Bs, RowState<R>& Cs, const int p1) -> bool {
        const int p2 = p1 - 1, p3 = p1 - 2;
        c.wait_upto(p1 + 1);
        const bool ph1 = (p1 <= y1 + 1) && c.row_valid(p1);
        if (ph1) {
            phase1<S, R>(c, An, p1);
            rbuf[t] = An.rho;
        }
        __syncthreads();  // A: rho row p1 visible; slot p1-3 free
        if (s_abort) return false;
        if (t == 0 && p1 + 5 <= c.rhi && p1 + 5 >= c.rlo) {
            fence_proxy_async();
            c.issue(p1 + 5);
        }
        // ---- phase 2 on row p2
        const bool ph2 = (p2 >= y0 - 1) && (p2 <= y1) && c.row_valid(p2);
        if (ph1 && ph2_thread) {
            const R l = rbuf[t - 1], r = rbuf[t + 1];
            An.dr = r - l;
            An.wr = (R)4 * An.rho + (r + l);
        }
        if (ph2 && ph2_thread) {
            // rows p2-1 (Cs), p2 (Bs), p2+1 (An), with the wall mirror of rho
            R dlo = Cs.dr, wlo = Cs.wr, dhi = An.dr, whi = An.wr;
            if (p.wall_y && p2 == 0) { dlo = Bs.dr; wlo = Bs.wr; }
            if (p.wall_y && p2 == p.ny - 1) { dhi = Bs.dr; whi = Bs.wr; }
            const R gx = (dlo + (R)4 * Bs.dr + dhi) * twelfth;
            const R gy = (whi - wlo) * twelfth;
            const R phi = c.r_row(p2, 0)[c.sc];
            const R kp = (p.model_b ? (kappa - (R)1) : (kappa - phi)) * third;
            R Fx = kp * gx + phi * p.gx;
            R Fy = kp * gy + phi * p.gy;
            if (p.has_fb) {
                const int k = p.unsteady ? 2 : 1;
                Fx += c.r_row(p2, k)[c.sc];
                Fy += c.r_row(p2, k + 1)[c.sc];
            }
            const R m0 = Bs.m[0];
            const R inv = (R)1 / m0;
            const R ux = (Bs.m[3] + (R)0.5 * Fx) * inv;
            const R uy = (Bs.m[5] + (R)0.5 * Fy) * inv;
            Bs.Fx = Fx; Bs.Fy = Fy; Bs.ux = ux; Bs.uy = uy;
            fbuf[0 * T + t] = Bs.rho * ux;
            fbuf[1 * T + t] = Bs.rho * uy;
            fbuf[2 * T + t] = ux;
            fbuf[3 * T + t] = uy;
            fbuf[4 * T + t] = m0 * ux;
            fbuf[5 * T + t] = m0 * uy;
        }
        __syncthreads();  // B: field row p2 visible
        if (ph2 && ph3_thread) {
            const R* F0 = fbuf;
            const R Axl = F0[t - 1], Axr = F0[t + 1];
            const R Ayl = F0[T + t - 1], Ayr = F0[T + t + 1];
            const R Bxl = F0[2 * T + t - 1], Bxr = F0[2 * T + t + 1];
            const R Byl = F0[3 * T + t - 1], Byr = F0[3 * T + t + 1];
            const R Dxl = F0[4 * T + t - 1], Dxr = F0[4 * T + t + 1];
            const R Dyl = F0[5 * T + t - 1], Dyr = F0[5 * T + t + 1];
            const R ay = Bs.rho * Bs.uy, dyv = Bs.m[0] * Bs.uy;
            Bs.dAx = Axr - Axl;
            Bs.dBx = Bxr - Bxl;
            Bs.dBy = Byr - Byl;
            Bs.dDx = Dxr - Dxl;
            Bs.wAy = (R)4 * ay + (Ayr + Ayl);
            Bs.wBy = (R)4 * Bs.uy + (Byr + Byl);
            Bs.wBx = (R)4 * Bs.ux + (Bxr + Bxl);
            Bs.wDy = (R)4 * dyv + (Dyr + Dyl);
        }
        // ---- phase 3 on row p3
        const bool ph3 = (p3 >= y0) && (p3 < y1);
        if (ph3 && ph3_thread && c.xc < p.nx) {
            // rows p3-1 (An holds row p1-3), p3 (Cs), p3+1 (Bs); walls mirror with a sign flip
            R dAx_l = An.dAx, dBx_l = An.dBx, dBy_l = An.dBy, dDx_l = An.dDx;
            R wAy_l = An.wAy, wBy_l = An.wBy, wBx_l = An.wBx, wDy_l = An.wDy;
            R dAx_h = Bs.dAx, dBx_h = Bs.dBx, dBy_h = Bs.dBy, dDx_h = Bs.dDx;
            R wAy_h = Bs.wAy, wBy_h = Bs.wBy, wBx_h = Bs.wBx, wDy_h = Bs.wDy;
            if (p.wall_y && p3 == 0) {
                dAx_l = -Cs.dAx; dBx_l = -Cs.dBx; dBy_l = -Cs.dBy; dDx_l = -Cs.dDx;
                wAy_l = -Cs.wAy; wBy_l = -Cs.wBy; wBx_l = -Cs.wBx; wDy_l = -Cs.wDy;
            }
            if (p.wall_y && p3 == p.ny - 1) {
                dAx_h = -Cs.dAx; dBx_h = -Cs.dBx; dBy_h = -Cs.dBy; dDx_h = -Cs.dDx;
                wAy_h = -Cs.wAy; wBy_h = -Cs.wBy; wBx_h = -Cs.wBx; wDy_h = -Cs.wDy;
            }
            // 12 x the Eq. (10) derivatives
            const R xAx = dAx_l + (R)4 * Cs.dAx + dAx_h;
            const R xBx = dBx_l + (R)4 * Cs.dBx + dBx_h;
            const R xBy = dBy_l + (R)4 * Cs.dBy + dBy_h;
            const R xDx = dDx_l + (R)4 * Cs.dDx + dDx_h;
            const R yAy = wAy_h - wAy_l;
            const R yBy = wBy_h - wBy_l;
            const R yBx = wBx_h - wBx_l;
            const R yDy = wDy_h - wDy_l;

            const R phi = c.r_row(p3, 0)[c.sc];
            const R phin = p.unsteady ? c.r_row(p3, 1)[c.sc] : phi;
            const R rho = Cs.rho;
            const R X = kappa / phi;
            const R kp = p.model_b ? (kappa - (R)1) : (kappa - phi);
            // Eq. (20)
            const R Ca = (-kappa * (xAx + yAy) + (R)2 * kp * rho * (xBx + yBy) + ((R)3 - (R)2 * X) * (xDx + yDy)) * twelfth
                         - (R)2 * X * rho * (phin - phi);
            const R Cb = (-kappa * (xAx - yAy) + ((R)2 / (R)3) * kp * rho * (xBx - yBy) + (xDx - yDy)) * twelfth;
            const R Cc = third * kp * rho * (xBy + yBx) * twelfth;

            // Eq. (18), (19), (16)
            const R m0 = Cs.m[0], ux = Cs.ux, uy = Cs.uy, Fx = Cs.Fx, Fy = Cs.Fy;
            const R uu = ux * ux + uy * uy;
            const R uF = ux * Fx + uy * Fy;
            const R jxe = m0 * ux, jye = m0 * uy;
            const R q = (X - (R)2);
            const R hc = (R)1 - (R)0.5 * p.s_c, he = (R)1 - (R)0.5 * p.s_e, hs = (R)1 - (R)0.5 * p.s_eps;
            const R hq = (R)1 - (R)0.5 * p.s_q, hn = (R)1 - (R)0.5 * p.s_nu;
            R a[9];
            a[0] = m0;
            a[1] = Cs.m[1] + p.s_e * (m0 * ((R)-4 + (R)3 * uu + (R)2 * X) - Cs.m[1]) + he * ((R)6 * uF + Ca);
            a[2] = Cs.m[2] + p.s_eps * (m0 * ((R)4 - (R)3 * uu - (R)3 * X) - Cs.m[2]) - hs * ((R)6 * uF);
            a[3] = Cs.m[3] + p.s_c * (jxe - Cs.m[3]) + hc * Fx;
            a[4] = Cs.m[4] + p.s_q * (q * jxe - Cs.m[4]) - hq * Fx;
            a[5] = Cs.m[5] + p.s_c * (jye - Cs.m[5]) + hc * Fy;
            a[6] = Cs.m[6] + p.s_q * (q * jye - Cs.m[6]) - hq * Fy;
            a[7] = Cs.m[7] + p.s_nu * (m0 * (ux * ux - uy * uy) - Cs.m[7]) + hn * ((R)2 * (ux * Fx - uy * Fy) + Cb);
            a[8] = Cs.m[8] + p.s_nu * (jxe * uy - Cs.m[8]) + hn * ((ux * Fy + uy * Fx) + Cc);

            // f+ = M^-1 m+ (A1), the 1/36 folded into the coefficients
            R fo[9];
            const R ninth = (R)1 / (R)9;
            fo[0] = (a[0] - a[1] + a[2]) * ninth;
            const R bax = ((R)4 * a[0] - a[1] - (R)2 * a[2]) * ((R)1 / (R)36);
            const R bdg = ((R)4 * a[0] + (R)2 * a[1] + a[2]) * ((R)1 / (R)36);
            const R xa = (a[3] - a[4]) * ((R)1 / (R)6);
            const R ya = (a[5] - a[6]) * ((R)1 / (R)6);
            const R pq = a[7] * (R)0.25;
            const R xd = ((R)2 * a[3] + a[4]) * twelfth;
            const R yd = ((R)2 * a[5] + a[6]) * twelfth;
            const R pd = a[8] * (R)0.25;
            const R t13 = bax + pq, t24 = bax - pq;
            fo[1] = t13 + xa;
            fo[3] = t13 - xa;
            fo[2] = t24 + ya;
            fo[4] = t24 - ya;
            const R t57 = bdg + pd, t68 = bdg - pd;
            const R sp = xd + yd, sm = xd - yd;
            fo[5] = t57 + sp;
            fo[7] = t57 - sp;
            fo[6] = t68 - sm;
            fo[8] = t68 + sm;

            // store (own cell: pull streaming) + periodic ghost images
            S* dst = reinterpret_cast<S*>(p.dst);
            const long long rowo = (long long)p3 * p.P + kPadCols;
            const R r0 = p.rest.r0(phin);
            S e[9];
            e[0] = enc<S, R>(fo[0], r0, p.scale);
#pragma unroll
            for (int i = 1; i < 9; ++i) e[i] = enc<S, R>(fo[i], p.rest.ri(i), p.scale);
#pragma unroll
            for (int i = 0; i < 9; ++i) dst[i * p.plane + rowo + c.xc] = e[i];
            if (c.xc < kGhost || c.xc >= p.nx - kGhost) {
                for (int g = c.xc - p.nx; g >= -kGhost; g -= p.nx)
#pragma unroll
                    for (int i = 0; i < 9; ++i) dst[i * p.plane + rowo + g] = e[i];
                for (int g = c.xc + p.nx; g < p.nx + kGhost; g += p.nx)
#pragma unroll
                    for (int i = 0; i < 9; ++i) dst[i * p.plane + rowo + g] = e[i];
            }
        }
        return true;
    };

    const int n_it = (y1 + 1) - (y0 - 2) + 1;  // p1 = y0-2 .. y1+1
    bool ok = true;
    for (int it = 0; it < n_it && ok; it += 3) {
        const int p1 = y0 - 2 + it;
        ok = iter(s0, s2, s1, p1);
        if (ok && it + 1 < n_it) ok = iter(s1, s0, s2, p1 + 1);
        if (ok && it + 2 < n_it) ok = iter(s2, s1, s0, p1 + 2);
    }
    if (!ok && t == 0) {
        // drain: wait (bounded) for every copy issued, so none lands after exit
        for (int r = c.waited + 1; r <= c.issued; ++r) {
            const uint32_t parity = (uint32_t)(((r - c.rlo) >> 3) & 1);
            mbar_wait_bounded(&bar[r & (kSlots - 1)], parity, kWaitTries);
        }
    }
}

}  // namespace lbmv
