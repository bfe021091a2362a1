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
// Source rows are staged in an 8-slot shared-memory ring by 1-D bulk async copies
// (cp.async.bulk, completing on one mbarrier per slot) issued up to 4 rows ahead
// of the newest row in use: the 9 population rows of a slot sit at fixed offsets
// (compile-time layout), the phi / phi(t+1) / force rows in a second ring whose row
// count depends on what is present.
#pragma once

#include "vanse_common.cuh"

namespace lbmv {

constexpr int kSlots = 8;                  // ring slots (power of two)
constexpr uint32_t kWaitTries = 1u << 22;  // bounded mbarrier polls (seconds, far above a row's latency)
// The default bound of a staged-row wait is kWaitTries (StepParams::wait_tries; a test may
// lower it to make the waits give up). Whatever that bound, a CTA drains the copies it
// issued with kWaitTries before it exits: from the first row whose wait gave up (its copy
// may still be in flight) to the newest row issued, so no copy lands after the exit.

// Compile-time shared-memory layout of the step kernel.
template <typename S, typename R, int T>
struct StepLayout {
    static constexpr int A = 16 / (int)sizeof(S);             // elements per 16 bytes
    static constexpr int WW = T + 2 * A;                       // staged row width (elements)
    static constexpr int kBuf = 128;                           // mbarriers
    static constexpr int kRho = kBuf;                          // rho row, T R
    static constexpr int kFld = kRho + T * (int)sizeof(R);     // 6 field rows, 6T R
    static constexpr int kPop = (kFld + 6 * T * (int)sizeof(R) + 127) & ~127;
    static constexpr int kPopRow = WW * (int)sizeof(S);
    static constexpr int kPopSlot = 9 * kPopRow;
    static constexpr int kAux = kPop + kSlots * kPopSlot;     // aux ring: kSlots x nR rows of WW R
    static constexpr int kAuxRow = WW * (int)sizeof(R);
    __host__ __device__ static constexpr size_t bytes(int nR) { return (size_t)kAux + (size_t)kSlots * nR * kAuxRow; }
    // with solid cells: rho, the six Eq. (20) fields and phi of the last three rows
    // (8 x 3 x T R; phase 3 cannot read phi of row p3-1 from the staging ring, whose slot
    // is refilled in the same row iteration)
    __host__ __device__ static constexpr size_t solid_bytes() { return (size_t)24 * T * sizeof(R); }
};

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
    int wall_x;           // half-way bounce-back walls at x = -1/2 and x = nx - 1/2 (kernel 1)
    int nR;               // staged aux rows per slot (phi, [phi(t+1)], [F^B x, y])
    R kappa, gx, gy;
    R s_e, s_eps, s_q, s_nu;      // relaxation rates (Gamma)
    R h_e, h_eps, h_q, h_nu;      // 1 - s/2
    R scale, inv_scale;   // deviation-storage scale (FP16/BF16)
    Rest<R> rest;
    int* err;             // set to 1 when a bounded wait gives up
    int eq2;              // App. B: (B2) energy-flux equilibria and the (B3) penalty (kernel 1 only)
    int has_drag;         // F^B += -beta (u - u_s), beta = phi^2 (d0 + d1 (1 - phi)); u solved implicitly
    R drag_d0, drag_d1, us_x, us_y;
    double* sums;         // step-sum variants: FP64 sums of m_0+, j_x+, j_y+ over the cells written (added)
    int nee_top;          // row ny-1 is a moving wall by non-equilibrium extrapolation (kernels 1 and 5)
    R uw_x, uw_y;         // its velocity
    int has_solid;        // cells with phi = 0 are solid (the SOLID variants of kernels 1 and 5)
    // one-warp kernel with solid cells: per CTA (blockIdx.y * gridDim.x + blockIdx.x), 1
    // when a solid cell lies in the rows and columns the CTA stages (else it runs the
    // solid-free path), or nullptr (every CTA takes the solid path)
    const unsigned char* solid_tiles;
    const int* tile_order;   // with solid_tiles: the tile (y * gridDim.x + x) CTA number k runs
    // the one-warp kernel collides FP16/BF16 deviations in the storage's scaled units:
    // h_* x scale, rho0 x scale and inv_scale / 3 (equal to h_*, rho0, 1/3 at scale 1)
    R hs_e, hs_eps, hs_q, hs_nu, rho0s, kp3;
    const unsigned* step_ctr;   // one-warp kernel: steps taken (seeds the stochastic rounding), or nullptr
    uint32_t wait_tries;        // polls of a staged-row wait before it gives up (kWaitTries by default)
    // one-warp kernel: the source buffer as a tensor [9 or 11][ny][P] whose box (the
    // staged width x 1 row x all planes) stages a row's population rows in one copy
    CUtensorMap pop_map;
};

// Compensated (Kahan) sums of the post-collision m_0, j_x, j_y of the cells one
// thread writes, for the step-sum kernel variants: the running sums stay within
// about one ulp of their value over the whole strip.
template <typename R>
struct MomentSums {
    R s[3] = {0, 0, 0}, c[3] = {0, 0, 0};
    __device__ __forceinline__ void add(int k, R v) {
        const R y = v - c[k];
        const R t = s[k] + y;
        c[k] = (t - s[k]) - y;
        s[k] = t;
    }
    __device__ __forceinline__ double value(int k) const { return (double)s[k] - (double)c[k]; }
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
    R dAy, wAx, dDy, wDx;          // App. B only: the cross derivatives of rho u and phi rho u
};

__device__ __forceinline__ float rcp_r(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp_r(double x) { return 1.0 / x; }

template <typename S, typename R, int T>
struct StepCtx {
    using L = StepLayout<S, R, T>;
    const StepParams<R>& p;
    unsigned char* smem;
    int* abort_flag;
    int t, xc, sc;      // thread, global column, smem column
    int y0, y1;
    int wsp, ww;        // staged window start (padded column) and width
    int rlo, rhi;       // source rows this CTA loads
    int waited;         // newest row waited for
    int issued;         // newest row issued (thread 0 only)
    int first_bad = 0x7fffffff;   // first row whose wait gave up (this thread)

    __device__ __forceinline__ uint64_t* bar(int r) const {
        return reinterpret_cast<uint64_t*>(smem) + (r & (kSlots - 1));
    }
    // this thread's element of population row 0 of the slot holding source row r
    __device__ __forceinline__ const S* pop(int r) const {
        return reinterpret_cast<const S*>(smem + L::kPop + (r & (kSlots - 1)) * L::kPopSlot) + sc;
    }
    // this thread's element of aux row k of the slot holding source row r
    __device__ __forceinline__ const R* aux(int r, int k) const {
        return reinterpret_cast<const R*>(smem + L::kAux) + ((r & (kSlots - 1)) * p.nR + k) * L::WW + sc;
    }
    __device__ __forceinline__ bool row_valid(int r) const { return !p.wall_y || (r >= 0 && r < p.ny); }

    // thread 0: load source row r into its slot
    __device__ __forceinline__ void issue(int r) {
        issued = r;
        uint64_t* b = bar(r);
        int gr = r;
        if (!p.wall_y) { gr %= p.ny; if (gr < 0) gr += p.ny; }
        const uint32_t bs = (uint32_t)(ww * (int)sizeof(S));
        const uint32_t br = (uint32_t)(ww * (int)sizeof(R));
        mbar_expect_tx(b, 9u * bs + (uint32_t)p.nR * br);
        const long long off = (long long)gr * p.P + wsp;
        const S* src = reinterpret_cast<const S*>(p.src) + off;
        unsigned char* ps = smem + L::kPop + (r & (kSlots - 1)) * L::kPopSlot;
#pragma unroll
        for (int i = 0; i < 9; ++i) bulk_g2s(ps + i * L::kPopRow, src + i * p.plane, bs, b);
        R* rr = reinterpret_cast<R*>(smem + L::kAux) + (r & (kSlots - 1)) * p.nR * L::WW;
        int k = 0;
        bulk_g2s(rr + (k++) * L::WW, p.phi + off, br, b);
        if (p.unsteady) bulk_g2s(rr + (k++) * L::WW, p.phin + off, br, b);
        if (p.has_fb) {
            bulk_g2s(rr + (k++) * L::WW, p.fb + off, br, b);
            bulk_g2s(rr + (k++) * L::WW, p.fb + p.plane + off, br, b);
        }
    }
    // all threads: make sure every source row up to r has landed
    __device__ __forceinline__ void wait_upto(int r) {
        r = min(r, rhi);
        while (waited < r) {
            ++waited;
            const uint32_t parity = (uint32_t)(((waited - rlo) >> 3) & 1);
            if (!mbar_wait_bounded(bar(waited), parity, p.wait_tries)) {
                first_bad = min(first_bad, waited);
                *abort_flag = 1;
                atomicExch(p.err, 1);
            }
        }
    }
};

// Phase 1: pull + moments + rho for row r into st.
template <typename S, typename R, int T, bool SOLID = false>
__device__ __forceinline__ void phase1(const StepCtx<S, R, T>& c, RowState<R>& st, int r) {
    using L = StepLayout<S, R, T>;
    constexpr int RW = L::WW;  // elements between population rows of a slot
    const StepParams<R>& p = c.p;
    const R phi = *c.aux(r, 0);
    const Rest<R>& rs = p.rest;
    const R ia = p.inv_scale;
    const S* cur = c.pop(r);
    R f0, f1, f2, f3, f4, f5, f6, f7, f8;
    f0 = dec(cur[0 * RW], rs.r0(phi), ia);
    f1 = dec(cur[1 * RW - 1], rs.ax, ia);
    f3 = dec(cur[3 * RW + 1], rs.ax, ia);
    if (p.wall_y && r == 0) {  // links from y = -1 come back from the wall: opposite slot, same cell
        f2 = dec(cur[4 * RW], rs.ax, ia);
        f5 = dec(cur[7 * RW], rs.dg, ia);
        f6 = dec(cur[8 * RW], rs.dg, ia);
    } else {
        const S* lo = c.pop(r - 1);
        f2 = dec(lo[2 * RW], rs.ax, ia);
        f5 = dec(lo[5 * RW - 1], rs.dg, ia);
        f6 = dec(lo[6 * RW + 1], rs.dg, ia);
    }
    if (p.wall_y && r == p.ny - 1) {
        f4 = dec(cur[2 * RW], rs.ax, ia);
        f7 = dec(cur[5 * RW], rs.dg, ia);
        f8 = dec(cur[6 * RW], rs.dg, ia);
    } else {
        const S* hi = c.pop(r + 1);
        f4 = dec(hi[4 * RW], rs.ax, ia);
        f7 = dec(hi[7 * RW + 1], rs.dg, ia);
        f8 = dec(hi[8 * RW - 1], rs.dg, ia);
    }
    if (p.wall_x) {   // links from x = -1 or x = nx come back from the wall: opposite slot, same cell
        if (c.xc == 0) {
            f1 = dec(cur[3 * RW], rs.ax, ia);
            f5 = dec(cur[7 * RW], rs.dg, ia);
            f8 = dec(cur[6 * RW], rs.dg, ia);
        }
        if (c.xc == p.nx - 1) {
            f3 = dec(cur[1 * RW], rs.ax, ia);
            f6 = dec(cur[8 * RW], rs.dg, ia);
            f7 = dec(cur[5 * RW], rs.dg, ia);
        }
    }
    if constexpr (SOLID) {
        // a solid cell (phi = 0) has no populations; a link from a solid cell is a
        // half-way bounce-back link: the population comes from the opposite slot of
        // this cell
        if (phi == (R)0) {
#pragma unroll
            for (int k = 0; k < 9; ++k) st.m[k] = (R)0;
            st.rho = (R)0;
            return;
        }
        const R* ph0 = c.aux(r, 0);
        if (ph0[-1] == (R)0) f1 = dec(cur[3 * RW], rs.ax, ia);
        if (ph0[1] == (R)0) f3 = dec(cur[1 * RW], rs.ax, ia);
        if (!(p.wall_y && r == 0)) {
            const R* phl = c.aux(r - 1, 0);
            if (phl[0] == (R)0) f2 = dec(cur[4 * RW], rs.ax, ia);
            if (phl[-1] == (R)0) f5 = dec(cur[7 * RW], rs.dg, ia);
            if (phl[1] == (R)0) f6 = dec(cur[8 * RW], rs.dg, ia);
        }
        if (!(p.wall_y && r == p.ny - 1)) {
            const R* phh = c.aux(r + 1, 0);
            if (phh[0] == (R)0) f4 = dec(cur[2 * RW], rs.ax, ia);
            if (phh[1] == (R)0) f7 = dec(cur[5 * RW], rs.dg, ia);
            if (phh[-1] == (R)0) f8 = dec(cur[6 * RW], rs.dg, ia);
        }
    }
    // m = M f with the row structure of (A1)
    const R a13 = f1 + f3, a24 = f2 + f4, b57 = f5 + f7, b68 = f6 + f8;
    const R sax = a13 + a24, sdg = b57 + b68;
    const R d13 = f1 - f3, d24 = f2 - f4;
    const R d57 = f5 - f7;
    const R dx = d57 + (f8 - f6);
    const R dy = d57 + (f6 - f8);
    st.m[0] = f0 + sax + sdg;
    st.m[1] = (R)-4 * f0 - sax + (R)2 * sdg;
    st.m[2] = (R)4 * f0 - (R)2 * sax + sdg;
    st.m[3] = d13 + dx;
    st.m[4] = (R)-2 * d13 + dx;
    st.m[5] = d24 + dy;
    st.m[6] = (R)-2 * d24 + dy;
    st.m[7] = a13 - a24;
    st.m[8] = b57 - b68;
    st.rho = st.m[0] * rcp_r(phi);
}

// 3-row ring index of a (possibly negative) row number
__device__ __forceinline__ int ring3(int r) { return ((r % 3) + 3) % 3; }

// 12 x the Eq. (10) gradient of a field at the fluid cell (thread column, row y) when
// solid cells (phi = 0) may be among its neighbours. val(row, dx) reads the field of
// a staged row, phi_at(row, dx) its void fraction. Neighbours map as everywhere (a row
// past a half-way wall is the mirror row, a vector component changing sign; the row
// past the moving wall extrapolates linearly); a solid neighbour then reads the ghost
// value mirrored about the solid surface: an axis neighbour the cell itself, a
// diagonal one the mean of the fluid ones of its two axis images (the cell itself if
// both are solid), negated for a vector component (odd). Returns false (and leaves
// g unset) when no neighbour is solid.
template <typename R, typename Val, typename Phi>
__device__ __forceinline__ bool solid_grad12(const StepParams<R>& p, int y, bool odd, Val val, Phi phi_at, R& gx12,
                                             R& gy12) {
    auto rowsel = [&](int dy, int& sg) {
        const int yy = y + dy;
        sg = 1;
        if (p.wall_y && (yy < 0 || yy >= p.ny)) { sg = -1; return y; }
        return yy;
    };
    bool any = false;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            if (dx == 0 && dy == 0) continue;
            int sg;
            const int rr = rowsel(dy, sg);
            const bool nee_row = p.nee_top && y + dy == p.ny;
            any = any || (!nee_row && phi_at(rr, dx) == (R)0);
        }
    if (!any) return false;
    const R osg = odd ? (R)-1 : (R)1;
    R sx = 0, sy = 0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            if (dx == 0 && dy == 0) continue;
            int sg;
            const int rr = rowsel(dy, sg);
            const bool nee_row = p.nee_top && y + dy == p.ny;
            R v;
            if (!nee_row && phi_at(rr, dx) == (R)0) {
                v = val(y, 0);
                if (dx != 0 && dy != 0) {
                    int sb;
                    const int rb = rowsel(dy, sb);
                    const bool fa = phi_at(y, dx) != (R)0, fb = phi_at(rb, 0) != (R)0;
                    const R va = val(y, dx), vb = (odd && sb < 0) ? -val(rb, 0) : val(rb, 0);
                    if (fa && fb) v = (va + vb) / (R)2;
                    else if (fa) v = va;
                    else if (fb) v = vb;
                }
                v = osg * v;
            } else if (nee_row) {
                v = (R)2 * val(y, dx) - val(y - 1, dx);
            } else {
                v = (odd && sg < 0) ? -val(rr, dx) : val(rr, dx);
            }
            const R cw = (dx != 0 && dy != 0) ? (R)1 : (R)4;   // 36 w_i
            sx += cw * v * (R)dx;
            sy += cw * v * (R)dy;
        }
    gx12 = sx;
    gy12 = sy;
    return true;
}

// Phase 2 for row p2 (state Bs), rows p2-1 / p2+1 in Cs / An.
template <typename S, typename R, int T, bool SOLID = false>
__device__ __forceinline__ void phase2(const StepCtx<S, R, T>& c, const RowState<R>& An, RowState<R>& Bs,
                                       const RowState<R>& Cs, int p2, R* fbuf, const R* rho3 = nullptr) {
    const StepParams<R>& p = c.p;
    const R twelfth = (R)1 / (R)12;
    if (SOLID && *c.aux(p2, 0) == (R)0) {   // solid cell: no velocity, no force, zero fields
        Bs.Fx = Bs.Fy = Bs.ux = Bs.uy = (R)0;
#pragma unroll
        for (int k = 0; k < 6; ++k) fbuf[k * T + c.t] = (R)0;
        return;
    }
    R dlo = Cs.dr, wlo = Cs.wr, dhi = An.dr, whi = An.wr;
    if (p.wall_y && (p2 == 0 || p2 == p.ny - 1)) {  // rho's wall ghost: the mirror row itself
        if (p2 == 0) { dlo = Bs.dr; wlo = Bs.wr; }
        if (p2 == p.ny - 1) {
            if (p.nee_top) { dhi = (R)2 * Bs.dr - Cs.dr; whi = (R)2 * Bs.wr - Cs.wr; }   // linear extrapolation
            else { dhi = Bs.dr; whi = Bs.wr; }
        }
    }
    R gx = (dlo + (R)4 * Bs.dr + dhi) * twelfth;
    R gy = (whi - wlo) * twelfth;
    if constexpr (SOLID) {
        R gx12, gy12;
        const int t = c.t;
        auto val = [&](int row, int dx) { return rho3[ring3(row) * T + t + dx]; };
        auto phi_at = [&](int row, int dx) { return c.aux(row, 0)[dx]; };
        if (solid_grad12(p, p2, false, val, phi_at, gx12, gy12)) { gx = gx12 * twelfth; gy = gy12 * twelfth; }
    }
    const R phi = *c.aux(p2, 0);
    const R kp = (p.model_b ? (p.kappa - (R)1) : (p.kappa - phi)) * ((R)1 / (R)3);
    R Fx = kp * gx + phi * p.gx;
    R Fy = kp * gy + phi * p.gy;
    if (p.has_fb) {
        const int k = p.unsteady ? 2 : 1;
        Fx += *c.aux(p2, k);
        Fy += *c.aux(p2, k + 1);
    }
    const R m0 = Bs.m[0];
    R ux, uy;
    if (p.has_drag) {
        // Eq. (7) with F^B += -beta (u - u_s): linear in u, solved exactly
        const R beta = phi * phi * (p.drag_d0 + p.drag_d1 * ((R)1 - phi));
        const R inv = (R)1 / (m0 + (R)0.5 * beta);
        ux = (Bs.m[3] + (R)0.5 * (Fx + beta * p.us_x)) * inv;
        uy = (Bs.m[5] + (R)0.5 * (Fy + beta * p.us_y)) * inv;
        Fx -= beta * (ux - p.us_x);
        Fy -= beta * (uy - p.us_y);
    } else {
        const R inv = rcp_r(m0);
        ux = (Bs.m[3] + (R)0.5 * Fx) * inv;
        uy = (Bs.m[5] + (R)0.5 * Fy) * inv;
    }
    Bs.Fx = Fx; Bs.Fy = Fy; Bs.ux = ux; Bs.uy = uy;
    const int t = c.t;
    fbuf[0 * T + t] = Bs.rho * ux;
    fbuf[1 * T + t] = Bs.rho * uy;
    fbuf[2 * T + t] = ux;
    fbuf[3 * T + t] = uy;
    fbuf[4 * T + t] = m0 * ux;
    fbuf[5 * T + t] = m0 * uy;
}

// Phase 3 for row p3 (state Cs), rows p3-1 / p3+1 in An / Bs: C, collision, store.
template <typename S, typename R, int T, bool SUMS = false, bool SOLID = false>
__device__ __forceinline__ void phase3(const StepCtx<S, R, T>& c, const RowState<R>& An, const RowState<R>& Bs,
                                       const RowState<R>& Cs, int p3, MomentSums<R>* sums = nullptr,
                                       const R* fld3 = nullptr) {
    const StepParams<R>& p = c.p;
    const R twelfth = (R)1 / (R)12;
    if (SOLID && *c.aux(p3, 0) == (R)0) return;   // a solid cell neither collides nor stores
    // 12 x the Eq. (10) derivatives
    R xAx = An.dAx + (R)4 * Cs.dAx + Bs.dAx;
    R xBx = An.dBx + (R)4 * Cs.dBx + Bs.dBx;
    R xBy = An.dBy + (R)4 * Cs.dBy + Bs.dBy;
    R xDx = An.dDx + (R)4 * Cs.dDx + Bs.dDx;
    R yAy = Bs.wAy - An.wAy;
    R yBy = Bs.wBy - An.wBy;
    R yBx = Bs.wBx - An.wBx;
    R yDy = Bs.wDy - An.wDy;
    // the row above a wall row: past a half-way wall the negated mirror row (no-slip),
    // past the moving (NEE) wall row the linear extrapolation 2 (row ny-1) - (row ny-2)
    const bool nee_hi = p.nee_top && p3 == p.ny - 1;
    auto ghi = [&](R cs, R an, R bs) { return nee_hi ? (R)2 * cs - an : (p3 == p.ny - 1 ? -cs : bs); };
    if (p.wall_y && (p3 == 0 || p3 == p.ny - 1)) {
        const bool lo = (p3 == 0);
        const R dAl = lo ? -Cs.dAx : An.dAx, dAh = ghi(Cs.dAx, An.dAx, Bs.dAx);
        const R dBxl = lo ? -Cs.dBx : An.dBx, dBxh = ghi(Cs.dBx, An.dBx, Bs.dBx);
        const R dByl = lo ? -Cs.dBy : An.dBy, dByh = ghi(Cs.dBy, An.dBy, Bs.dBy);
        const R dDl = lo ? -Cs.dDx : An.dDx, dDh = ghi(Cs.dDx, An.dDx, Bs.dDx);
        const R wAl = lo ? -Cs.wAy : An.wAy, wAh = ghi(Cs.wAy, An.wAy, Bs.wAy);
        const R wByl = lo ? -Cs.wBy : An.wBy, wByh = ghi(Cs.wBy, An.wBy, Bs.wBy);
        const R wBxl = lo ? -Cs.wBx : An.wBx, wBxh = ghi(Cs.wBx, An.wBx, Bs.wBx);
        const R wDl = lo ? -Cs.wDy : An.wDy, wDh = ghi(Cs.wDy, An.wDy, Bs.wDy);
        xAx = dAl + (R)4 * Cs.dAx + dAh;
        xBx = dBxl + (R)4 * Cs.dBx + dBxh;
        xBy = dByl + (R)4 * Cs.dBy + dByh;
        xDx = dDl + (R)4 * Cs.dDx + dDh;
        yAy = wAh - wAl;
        yBy = wByh - wByl;
        yBx = wBxh - wBxl;
        yDy = wDh - wDl;
        if (p.wall_x && (c.xc == 0 || c.xc == p.nx - 1)) {
            // Corner cell: the ghost row's diagonal ghost lies past both walls and holds the
            // negated cell value once (-psi), while the negated mirror row carries the
            // x-wall ghost negated twice (+psi); the ghost row's x-difference and smoothed
            // sum of a field component psi move by cd psi and cw psi.
            const R cd = (c.xc == 0 ? (R)2 : (R)0) - (c.xc == p.nx - 1 ? (R)2 : (R)0);
            const R cw = (c.xc == 0 ? (R)-2 : (R)0) + (c.xc == p.nx - 1 ? (R)-2 : (R)0);
            const R ng = (R)((p3 == 0 ? 1 : 0) + (p3 == p.ny - 1 ? 1 : 0));   // ghost rows at this row
            const R Ax = Cs.rho * Cs.ux, Ay = Cs.rho * Cs.uy, Dx = Cs.m[0] * Cs.ux, Dy = Cs.m[0] * Cs.uy;
            // x-derivatives take each ghost row's d with weight 1; y-derivatives take the
            // upper ghost's w with +1 and the lower's with -1
            const R sy = (R)((p3 == p.ny - 1 ? 1 : 0) - (p3 == 0 ? 1 : 0));
            xAx += ng * cd * Ax;
            xBx += ng * cd * Cs.ux;
            xBy += ng * cd * Cs.uy;
            xDx += ng * cd * Dx;
            yAy += sy * cw * Ay;
            yBy += sy * cw * Cs.uy;
            yBx += sy * cw * Cs.ux;
            yDy += sy * cw * Dy;
        }
    }

    // App. B cross derivatives, replaced below next to solid cells
    R xAy_s = 0, yAx_s = 0, xDy_s = 0, yDx_s = 0;
    bool solid_nb = false;
    if constexpr (SOLID) {
        const int t = c.t;
        // phi of rows p3-1 .. p3+1 from the ring phase 2 fills (the staging slot of row
        // p3-1 is being refilled by now)
        auto phi_at = [&](int row, int dx) { return fld3[18 * T + ring3(row) * T + t + dx]; };
        R g[6][2];
        for (int k = 0; k < 6 && (k == 0 || solid_nb); ++k) {
            auto val = [&](int row, int dx) { return fld3[(ring3(row) * 6 + k) * T + t + dx]; };
            const bool any = solid_grad12(p, p3, true, val, phi_at, g[k][0], g[k][1]);
            if (k == 0) solid_nb = any;
        }
        if (solid_nb) {
            // fields 0..5: rho u_x, rho u_y, u_x, u_y, phi rho u_x, phi rho u_y
            xAx = g[0][0]; yAy = g[1][1];
            xBx = g[2][0]; yBy = g[3][1]; xBy = g[3][0]; yBx = g[2][1];
            xDx = g[4][0]; yDy = g[5][1];
            xAy_s = g[1][0]; yAx_s = g[0][1]; xDy_s = g[5][0]; yDx_s = g[4][1];
        }
    }

    const R phi = *c.aux(p3, 0);
    const R phin = p.unsteady ? *c.aux(p3, 1) : phi;
    const R rho = Cs.rho;
    const R X = p.kappa * rcp_r(phi);
    const R kp = p.model_b ? (p.kappa - (R)1) : (p.kappa - phi);
    const R kr = kp * rho;
    R Ca, Cb, Cc;
    if (!p.eq2) {
        // Eq. (20)
        Ca = (-p.kappa * (xAx + yAy) + (R)2 * kr * (xBx + yBy) + ((R)3 - (R)2 * X) * (xDx + yDy)) * twelfth
             - (R)2 * X * rho * (phin - phi);
        Cb = (-p.kappa * (xAx - yAy) + ((R)2 / (R)3) * kr * (xBx - yBy) + (xDx - yDy)) * twelfth;
        Cc = kr * (xBy + yBx) * ((R)1 / (R)36);
    } else {
        // Eq. (B3): 12 x the cross derivatives d_x(rho u_y), d_y(rho u_x), d_x(phi rho u_y), d_y(phi rho u_x)
        R xAy = An.dAy + (R)4 * Cs.dAy + Bs.dAy, yAx = Bs.wAx - An.wAx;
        R xDy = An.dDy + (R)4 * Cs.dDy + Bs.dDy, yDx = Bs.wDx - An.wDx;
        if (p.wall_y && (p3 == 0 || p3 == p.ny - 1)) {
            const bool lo = (p3 == 0);
            xAy = (lo ? -Cs.dAy : An.dAy) + (R)4 * Cs.dAy + ghi(Cs.dAy, An.dAy, Bs.dAy);
            xDy = (lo ? -Cs.dDy : An.dDy) + (R)4 * Cs.dDy + ghi(Cs.dDy, An.dDy, Bs.dDy);
            yAx = ghi(Cs.wAx, An.wAx, Bs.wAx) - (lo ? -Cs.wAx : An.wAx);
            yDx = ghi(Cs.wDx, An.wDx, Bs.wDx) - (lo ? -Cs.wDx : An.wDx);
            if (p.wall_x && (c.xc == 0 || c.xc == p.nx - 1)) {   // corner cell, as above
                const R cd = (c.xc == 0 ? (R)2 : (R)0) - (c.xc == p.nx - 1 ? (R)2 : (R)0);
                const R cw = (c.xc == 0 ? (R)-2 : (R)0) + (c.xc == p.nx - 1 ? (R)-2 : (R)0);
                const R ng = (R)((p3 == 0 ? 1 : 0) + (p3 == p.ny - 1 ? 1 : 0));
                const R sy = (R)((p3 == p.ny - 1 ? 1 : 0) - (p3 == 0 ? 1 : 0));
                xAy += ng * cd * (Cs.rho * Cs.uy);
                xDy += ng * cd * (Cs.m[0] * Cs.uy);
                yAx += sy * cw * (Cs.rho * Cs.ux);
                yDx += sy * cw * (Cs.m[0] * Cs.ux);
            }
        }
        if (solid_nb) { xAy = xAy_s; yAx = yAx_s; xDy = xDy_s; yDx = yDx_s; }
        const R t3 = (R)2 / (R)3;
        Ca = ((R)-2 * p.kappa * (xAx + yAy) + (R)2 * kr * (xBx + yBy) + ((R)4 - (R)2 * X) * (xDx + yDy)) * twelfth
             - (R)2 * X * rho * (phin - phi);
        Cb = (-t3 * p.kappa * (xAx - yAy) + t3 * kr * (xBx - yBy) + t3 * (xDx - yDy)) * twelfth;
        Cc = (-p.kappa * (xAy + yAx) + kr * (xBy + yBx) + (xDy + yDx)) * ((R)1 / (R)36);
    }

    // Eq. (18), (19), (16); the conserved moments map to m_0 and j + F for any s_c
    const R m0 = Cs.m[0], ux = Cs.ux, uy = Cs.uy, Fx = Cs.Fx, Fy = Cs.Fy;
    const R uu = ux * ux + uy * uy;
    const R uF = ux * Fx + uy * Fy;
    const R jxe = m0 * ux, jye = m0 * uy;
    const R q = p.eq2 ? (R)-1 : X - (R)2;   // Eq. (18) / (B2) energy-flux equilibria
    R a[9];
    a[0] = m0;
    a[1] = Cs.m[1] + p.s_e * (m0 * ((R)-4 + (R)3 * uu + (R)2 * X) - Cs.m[1]) + p.h_e * ((R)6 * uF + Ca);
    a[2] = Cs.m[2] + p.s_eps * (m0 * ((R)4 - (R)3 * uu - (R)3 * X) - Cs.m[2]) - p.h_eps * ((R)6 * uF);
    a[3] = Cs.m[3] + Fx;
    a[4] = Cs.m[4] + p.s_q * (q * jxe - Cs.m[4]) - p.h_q * Fx;
    a[5] = Cs.m[5] + Fy;
    a[6] = Cs.m[6] + p.s_q * (q * jye - Cs.m[6]) - p.h_q * Fy;
    a[7] = Cs.m[7] + p.s_nu * (m0 * (ux * ux - uy * uy) - Cs.m[7]) + p.h_nu * ((R)2 * (ux * Fx - uy * Fy) + Cb);
    a[8] = Cs.m[8] + p.s_nu * (jxe * uy - Cs.m[8]) + p.h_nu * ((ux * Fy + uy * Fx) + Cc);

    if constexpr (SUMS) { sums->add(0, a[0]); sums->add(1, a[3]); sums->add(2, a[5]); }

    // f+ = M^-1 m+ (A1), the 1/36 folded into the coefficients. f_0 and the
    // diagonal-link x/y parts are formed as what m_0 and j leave after the other
    // populations (equal to (A1)'s rows; s = bax + bdg first, bdg = s - bax, exact
    // near rest), so the rounded 1/9, 1/36, 1/6 and 1/12 do not scale the cell's mass
    // and momentum by a fixed factor every step.
    R fo[9];
    const R bax = ((R)4 * a[0] - a[1] - (R)2 * a[2]) * ((R)1 / (R)36);
    const R sbd = ((R)8 * a[0] + (a[1] - a[2])) * ((R)1 / (R)36);
    const R bdg = sbd - bax;
    fo[0] = a[0] - (R)4 * sbd;
    const R xa = (a[3] - a[4]) * ((R)1 / (R)6);
    const R ya = (a[5] - a[6]) * ((R)1 / (R)6);
    const R pq = a[7] * (R)0.25;
    const R xd = (a[3] - (R)2 * xa) * (R)0.25;
    const R yd = (a[5] - (R)2 * ya) * (R)0.25;
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
    S* row = reinterpret_cast<S*>(p.dst) + (long long)p3 * p.P + kPadCols;
    S e[9];
    e[0] = enc<S, R>(fo[0], p.rest.r0(phin), p.scale);
#pragma unroll
    for (int i = 1; i < 9; ++i) e[i] = enc<S, R>(fo[i], p.rest.ri(i), p.scale);
    S* cell = row + c.xc;
#pragma unroll
    for (int i = 0; i < 9; ++i) cell[i * p.plane] = e[i];
    if (c.xc < kGhost || c.xc >= p.nx - kGhost) {
        // ghost images: at most one per side unless nx < kGhost
        int g = c.xc >= p.nx - kGhost ? c.xc - p.nx : c.xc + p.nx;
        while (g >= -kGhost && g < p.nx + kGhost) {
            S* gc = row + g;
            gc[0] = enc<S, R>(fo[0], p.rest.r0(phin), p.scale);
#pragma unroll
            for (int i = 1; i < 9; ++i) gc[i * p.plane] = enc<S, R>(fo[i], p.rest.ri(i), p.scale);
            // next image on the same side, then the other side
            if (g < 0) { g -= p.nx; if (g < -kGhost) { g = c.xc + p.nx; if (g >= p.nx + kGhost) break; } }
            else { g += p.nx; if (g >= p.nx + kGhost) break; }
        }
    }
}

// The equilibrium moments M f^eq of Eq. (18) (App. B: Eq. B2, eq2) at (phi, rho, u).
template <typename R>
__device__ __forceinline__ void eq_moments(const StepParams<R>& p, R phi, R rho, R ux, R uy, R m[9]) {
    const R m0 = phi * rho, X = p.kappa / phi, uu = ux * ux + uy * uy;
    const R q = p.eq2 ? (R)-1 : X - (R)2;
    m[0] = m0;
    m[1] = m0 * ((R)-4 + (R)3 * uu + (R)2 * X);
    m[2] = m0 * ((R)4 - (R)3 * uu - (R)3 * X);
    m[3] = m0 * ux;
    m[4] = q * (m0 * ux);
    m[5] = m0 * uy;
    m[6] = q * (m0 * uy);
    m[7] = m0 * (ux * ux - uy * uy);
    m[8] = (m0 * ux) * uy;
}

// Moving wall by non-equilibrium extrapolation (Sec. 3.1) on row ny-1 (Wa), next to
// fluid row ny-2 (Fl, its Eq. 7 velocity done): the wall node's moments become
// M f^eq(rho_f, u_w, phi_b) + m_f - M f^eq(rho_f, u_f, phi_f), with rho_b = rho_f
// (already in Wa.rho). In moment space, since M is linear.
template <typename R>
__device__ __forceinline__ void nee_wall_moments(const StepParams<R>& p, RowState<R>& Wa, const RowState<R>& Fl,
                                                 R phi_b, R phi_f) {
    R eb[9], ef[9];
    eq_moments(p, phi_b, Fl.rho, p.uw_x, p.uw_y, eb);
    eq_moments(p, phi_f, Fl.rho, Fl.ux, Fl.uy, ef);
#pragma unroll
    for (int k = 0; k < 9; ++k) Wa.m[k] = eb[k] + (Fl.m[k] - ef[k]);
}

template <typename S, typename R, int T, bool SUMS = false, bool SOLID = false>
__global__ void __launch_bounds__(T) vanse_step_kernel(const __grid_constant__ StepParams<R> p) {
    using L = StepLayout<S, R, T>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_abort;
    R* rbuf = reinterpret_cast<R*>(smem + L::kRho);
    R* fbuf = reinterpret_cast<R*>(smem + L::kFld);

    const int t = threadIdx.x;
    constexpr int A = L::A;
    const int x0 = blockIdx.x * p.W;
    const int y0 = blockIdx.y * p.H;
    const int y1 = min(y0 + p.H, p.ny);

    StepCtx<S, R, T> c{p, smem, &s_abort, t, 0, 0, y0, y1, 0, 0, 0, 0, 0, 0};
    c.wsp = ((kPadCols + x0 - kGhost) / A) * A;
    c.ww = ((kPadCols + x0 + p.W + kGhost + A - 1) / A) * A - c.wsp;
    c.xc = x0 - 2 + t;
    c.sc = kPadCols + c.xc - c.wsp;
    c.rlo = y0 - 3;
    c.rhi = y1 + 2;
    if (p.wall_y) { c.rlo = max(c.rlo, 0); c.rhi = min(c.rhi, p.ny - 1); }
    c.waited = c.rlo - 1;
    c.issued = c.rlo - 1;

    if (t == 0) {
        s_abort = 0;
        for (int k = 0; k < kSlots; ++k) mbar_init(reinterpret_cast<uint64_t*>(smem) + k, 1);
        fence_mbar_init();
        for (int r = c.rlo; r <= min(y0 + 2, c.rhi); ++r) c.issue(r);
    }
    __syncthreads();

    const bool ph3_thread = (t >= 2 && t < T - 2);
    const bool ph2_thread = (t >= 1 && t < T - 1);

    RowState<R> s0, s1, s2;
    MomentSums<R> sums;
    // with solid cells: rho and the six fields of the last three rows, for the
    // neighbour-by-neighbour stencil next to solid cells
    R* rho3 = SOLID ? reinterpret_cast<R*>(smem + L::bytes(p.nR)) : nullptr;
    R* fld3 = SOLID ? rho3 + 3 * T : nullptr;        // [3][6][T]; phi of the same rows follows at fld3 + 18 T

    // one iteration: new row p1 -> An, row p1-1 -> Bs, row p1-2 -> Cs
    auto iter = [&](RowState<R>& An, RowState<R>& Bs, RowState<R>& Cs, const int p1) -> bool {
        const int p2 = p1 - 1, p3 = p1 - 2;
        c.wait_upto(p1 + 1);
        const bool ph1 = (p1 <= y1 + 1) && c.row_valid(p1);
        if (ph1) {
            phase1<S, R, T, SOLID>(c, An, p1);
            // moving wall row: rho_b = rho of the fluid row below (its moments follow below)
            if (p.nee_top && p1 == p.ny - 1) An.rho = Bs.rho;
            rbuf[t] = An.rho;
            if constexpr (SOLID) rho3[ring3(p1) * T + t] = An.rho;
        }
        __syncthreads();  // A: rho row p1 visible; slot p1-3 free
        if (s_abort) return false;
        if (t == 0 && p1 + 5 <= c.rhi && p1 + 5 >= c.rlo) {
            fence_proxy_async();
            c.issue(p1 + 5);
        }
        const bool ph2 = (p2 >= y0 - 1) && (p2 <= y1) && c.row_valid(p2);
        if (ph1 && ph2_thread) {
            // past an x wall rho's ghost is the cell itself (the mirror about the wall)
            const R l = (p.wall_x && c.xc == 0) ? An.rho : rbuf[t - 1];
            const R r = (p.wall_x && c.xc == p.nx - 1) ? An.rho : rbuf[t + 1];
            An.dr = r - l;
            An.wr = (R)4 * An.rho + (r + l);
        }
        if (ph2 && ph2_thread) {
            phase2<S, R, T, SOLID>(c, An, Bs, Cs, p2, fbuf, rho3);
            if constexpr (SOLID) {
#pragma unroll
                for (int k = 0; k < 6; ++k) fld3[(ring3(p2) * 6 + k) * T + t] = fbuf[k * T + t];
                fld3[18 * T + ring3(p2) * T + t] = *c.aux(p2, 0);
            }
            if (p.nee_top && p1 == p.ny - 1 && ph1) nee_wall_moments(p, An, Bs, *c.aux(p1, 0), *c.aux(p2, 0));
        }
        __syncthreads();  // B: field row p2 visible
        if (ph2 && ph3_thread) {
            const R* F0 = fbuf + t;
            // past an x wall every field component's ghost is the negated cell value (no-slip)
            const bool xl = p.wall_x && c.xc == 0, xr = p.wall_x && c.xc == p.nx - 1;
            auto nb = [&](int k, int dx) { return ((dx < 0 && xl) || (dx > 0 && xr)) ? -F0[k * T] : F0[k * T + dx]; };
            const R Axl = nb(0, -1), Axr = nb(0, 1);
            const R Ayl = nb(1, -1), Ayr = nb(1, 1);
            const R Bxl = nb(2, -1), Bxr = nb(2, 1);
            const R Byl = nb(3, -1), Byr = nb(3, 1);
            const R Dxl = nb(4, -1), Dxr = nb(4, 1);
            const R Dyl = nb(5, -1), Dyr = nb(5, 1);
            Bs.dAx = Axr - Axl;
            Bs.dBx = Bxr - Bxl;
            Bs.dBy = Byr - Byl;
            Bs.dDx = Dxr - Dxl;
            Bs.wAy = (R)4 * (Bs.rho * Bs.uy) + (Ayr + Ayl);
            Bs.wBy = (R)4 * Bs.uy + (Byr + Byl);
            Bs.wBx = (R)4 * Bs.ux + (Bxr + Bxl);
            Bs.wDy = (R)4 * (Bs.m[0] * Bs.uy) + (Dyr + Dyl);
            if (p.eq2) {
                Bs.dAy = Ayr - Ayl;
                Bs.wAx = (R)4 * (Bs.rho * Bs.ux) + (Axr + Axl);
                Bs.dDy = Dyr - Dyl;
                Bs.wDx = (R)4 * (Bs.m[0] * Bs.ux) + (Dxr + Dxl);
            }
        }
        const bool ph3 = (p3 >= y0) && (p3 < y1);
        if (ph3 && ph3_thread && c.xc < p.nx) phase3<S, R, T, SUMS, SOLID>(c, An, Bs, Cs, p3, &sums, fld3);
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
        // drain: wait (bounded) for every copy that may still be in flight, so none
        // lands after exit (the rows whose wait gave up and those not waited for yet)
        for (int r = min(c.first_bad, c.waited + 1); r <= c.issued; ++r) {
            const uint32_t parity = (uint32_t)(((r - c.rlo) >> 3) & 1);
            mbar_wait_bounded(c.bar(r), parity, kWaitTries);
        }
    }
    if constexpr (SUMS) {
        // one FP64 atomic per CTA and sum (warps reduce by shuffles, then lane 0 adds)
        for (int k = 0; k < 3; ++k) {
            double v = sums.value(k);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((t & 31) == 0) atomicAdd(p.sums + k, v);
        }
    }
}

}  // namespace lbmv
