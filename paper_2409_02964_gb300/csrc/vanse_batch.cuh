// vanse_batch.cuh -- many independent lattices advanced by one persistent kernel
// per time step.
//
// Each lattice of a batch is an n x n periodic MRTLB-VANSE lattice with its own
// relaxation rates and its own spatiotemporal manufactured solution (Sec. 3.4):
// phi = phi0 + A sin(kx) sin(ky) cos(wt) and the body force of Eq. (25)
// (mms_force.cuh). Both are evaluated inside the kernel from the cell's
// coordinates and the step count, so the step reads and writes only the
// populations (no phi / force arrays).
//
// Work decomposition: every lattice is cut into units of 60 columns x H rows (the
// one-warp kernel's tile). A persistent grid of one-warp CTAs takes units from a
// global counter (largest lattices first) and runs the same row pipeline as the
// single-lattice one-warp kernel (warp_run_strip). The time step t lives in device
// memory and is advanced, with the unit counter reset, by a one-thread kernel
// after each step, so a captured CUDA graph of (step, tick) pairs replays without
// host involvement.
#pragma once

#include "vanse_aux.cuh"
#include "vanse_warp.cuh"
// after vanse_warp.cuh: the generated code needs the pair type and mms_rcp
#include "mms_force.cuh"

namespace lbmv {

struct BatchLattice {
    CUtensorMap map[2];        // each buffer as a tensor [9][ny][P] (box: staged width x 1 x 9)
    void* buf[2];              // population buffers (ping-pong by the parity of t)
    long long plane;           // elements per population plane
    int nx, ny, P;
    int tiles_x, strips, H;    // units: tiles_x x strips
    int unit0;                 // first unit of this lattice
    float s_e, s_eps, s_q, s_nu, h_e, h_eps, h_q, h_nu;
    float kappa, rho0;
    float k, w, A, U0, phi0, nu;   // manufactured solution
};

struct BatchParams {
    const BatchLattice* lat;
    const int* unit_lattice;   // lattice index of each unit
    int nunits;
    int* counter;              // next unit to hand out
    const int* clock;          // time step t
    float scale, inv_scale;    // FP16 / BF16 deviation scale
    int* err;
};

// Eq. (25) force at a lane's two columns. Kept out of line: inlined into each of the
// row loop's unrolled copies it makes the loop too large for the row states to stay
// in registers.
struct ForcePair {
    V2 fx, fy;
};
__device__ __forceinline__ ForcePair mms_force_pair(V2 sx, V2 cx, float sy, float cy, float ct, float st, float k,
                                                 float w, float A, float U0, float phi0, float nu) {
    ForcePair r;
    mms_force<V2>(sx, cx, bc(sy), bc(cy), ct, st, k, w, A, U0, phi0, nu, r.fx, r.fy);
    return r;
}

// Per-unit view with the interface warp_run_strip expects.
template <typename S>
struct BatchCtx {
    using L = WarpLayout<S>;
    static constexpr bool kUnsteady = true;
    static constexpr bool kSums = false;
    static constexpr bool kEq2 = false;
    static constexpr bool kSolid = false;
    static constexpr bool kJB = false;
    static constexpr bool kNee = false;
    StepParams<float> p;       // this lattice's scalars (pointers and sizes included)
    unsigned char* smem;
    int lane, xa, sa;
    int y0, y1;
    int wsp, ww;
    int rlo, rhi;
    int waited, issued;
    bool aborted;
    bool fast_strip;
    int fast_lo, fast_hi;
    uint32_t phase;            // parity of the next completion of each ring slot
    int first_bad;             // first row of this unit whose wait gave up (this lane)
    RowCopy cp;
    bool st_pair;              // this lane stores its pair (lanes 1..30, first column inside)
    uint32_t step = 0, salt = 0;   // seed of the stochastic rounding of FP16/BF16 stores
    // manufactured solution at this step
    V2 sx2, cx2;               // sin, cos of k x of the lane's two columns
    float k, w, A, U0, phi0, nu, rho0;
    float ct, st, ct1;         // cos(wt), sin(wt), cos(w(t+1))

    __device__ __forceinline__ uint64_t* bar(int r) const { return reinterpret_cast<uint64_t*>(smem) + wslot(r); }
    __device__ __forceinline__ const S* pop(int r) const {
        return reinterpret_cast<const S*>(smem + L::kPop + wslot(r) * L::kPopSlot) + sa;
    }
    __device__ __forceinline__ bool row_valid(int) const { return true; }

    __device__ __forceinline__ void row_setup(int r, PRow& st) const {
        sincospif(2.0f * (float)r / (float)p.ny, &st.sy, &st.cy);
    }
    __device__ __forceinline__ V2 phi2(int, const PRow& st) const { return fma2(A * ct * st.sy, sx2, bc(phi0)); }
    template <bool FAST>
    __device__ __forceinline__ V2 phin2(int, const PRow& st) const { return fma2(A * ct1 * st.sy, sx2, bc(phi0)); }
    template <bool FAST>
    __device__ __forceinline__ void add_field_force(int, const PRow& st, V2& Fx, V2& Fy) const {
        const ForcePair f = mms_force_pair(sx2, cx2, st.sy, st.cy, ct, this->st, k, w, A, U0, phi0, nu);
        Fx = fma2(rho0, f.fx, Fx);
        Fy = fma2(rho0, f.fy, Fy);
    }

    // this lane's part of staging a source row: lane 0 copies the nine population rows
    // with one 3-D tensor copy of the lattice's buffer (map: its tensor map in the
    // lattice descriptor, in global memory; a box of the whole staged width, starting
    // on the 16-byte aligned column wsp)
    __device__ __forceinline__ void setup_copies(const CUtensorMap* map) {
        const uint32_t base = smem_u32(smem);
        cp = RowCopy{};
        cp.bar0 = base;
        cp.tx = 9u * (uint32_t)(L::WW * (int)sizeof(S));
        if (lane == 0) {
            cp.map = map;
            cp.xcol = wsp;
            cp.dst = base + (uint32_t)L::kPop;
            cp.stride = (uint32_t)L::kPopSlot;
        }
    }
    // all lanes: load source row r (periodic) into its slot
    __device__ __forceinline__ void issue(int r) {
        issued = r;
        int gr = r % p.ny;
        if (gr < 0) gr += p.ny;
        cp.issue(lane, wslot(r), gr);
    }
    __device__ __forceinline__ void wait_upto(int r) {
        r = min(r, rhi);
        while (waited < r) {
            ++waited;
            const int s = wslot(waited);
            if (!mbar_wait_bounded(bar(waited), (phase >> s) & 1u, kWaitTries)) {
                first_bad = min(first_bad, waited);
                aborted = true;
                atomicExch(p.err, 1);
            }
            phase ^= 1u << s;
        }
    }
};

// After a wait gave up: wait (bounded by kWaitTries) for every copy of the unit that
// may still be in flight, so none lands after the CTA exits. Rows first_bad .. waited
// have toggled their slot's parity bit already (their completion has the other
// parity); rows waited+1 .. issued have not. These at most kWarpSlots rows lie in
// distinct slots (warp_run_strip never re-arms a slot whose wait gave up).
template <typename S>
__device__ __forceinline__ void batch_drain(const BatchCtx<S>& c, uint32_t& phase) {
    for (int r = min(c.first_bad, c.waited + 1); r <= c.issued; ++r) {
        const int s = wslot(r);
        if (r <= c.waited) {
            mbar_wait_bounded(c.bar(r), ((phase >> s) & 1u) ^ 1u, kWaitTries);
        } else {
            mbar_wait_bounded(c.bar(r), (phase >> s) & 1u, kWaitTries);
            phase ^= 1u << s;
        }
    }
}

template <typename S, int MINB>
__global__ void __launch_bounds__(32, MINB) vanse_batch_kernel(const __grid_constant__ BatchParams bp) {
    using L = WarpLayout<S>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x;
    constexpr int A = L::A;
    if (lane == 0) {
        for (int k = 0; k < kWarpSlots; ++k) mbar_init(reinterpret_cast<uint64_t*>(smem) + k, 1);
        fence_mbar_init();
    }
    __syncwarp();
    const int t = *bp.clock;
    uint32_t phase = 0;
    for (;;) {
        int u = 0;
        if (lane == 0) u = atomicAdd(bp.counter, 1);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= bp.nunits) break;
        const BatchLattice& Lt = bp.lat[bp.unit_lattice[u]];
        const int v = u - Lt.unit0;
        const int tx = v % Lt.tiles_x, ty = v / Lt.tiles_x;

        BatchCtx<S> c;
        c.smem = smem;
        c.lane = lane;
        c.step = (uint32_t)t;
        c.salt = (uint32_t)bp.unit_lattice[u] * 0x27d4eb2fu;
        c.aborted = false;
        c.first_bad = 0x7fffffff;
        c.phase = phase;
        StepParams<float>& p = c.p;
        p.src = Lt.buf[t & 1];
        p.dst = Lt.buf[(t + 1) & 1];
        p.plane = Lt.plane;
        p.nx = Lt.nx;
        p.ny = Lt.ny;
        p.P = Lt.P;
        p.W = 60;
        p.H = Lt.H;
        p.wall_y = 0;
        p.unsteady = 1;
        p.has_fb = 1;
        p.model_b = 0;
        p.nR = 0;
        p.kappa = Lt.kappa;
        p.gx = 0.f;
        p.gy = 0.f;
        p.s_e = Lt.s_e; p.s_eps = Lt.s_eps; p.s_q = Lt.s_q; p.s_nu = Lt.s_nu;
        p.h_e = Lt.h_e; p.h_eps = Lt.h_eps; p.h_q = Lt.h_q; p.h_nu = Lt.h_nu;
        p.scale = bp.scale;
        p.inv_scale = bp.inv_scale;
        p.hs_e = Lt.h_e * bp.scale; p.hs_eps = Lt.h_eps * bp.scale;
        p.hs_q = Lt.h_q * bp.scale; p.hs_nu = Lt.h_nu * bp.scale;
        p.rho0s = Lt.rho0 * bp.scale;
        p.kp3 = bp.inv_scale * (1.f / 3.f);
        p.rest.ax = Lt.kappa * Lt.rho0 * (1.f / 9.f);
        p.rest.dg = Lt.kappa * Lt.rho0 * (1.f / 36.f);
        p.rest.k59 = Lt.kappa * Lt.rho0 * (5.f / 9.f);
        p.rest.rho0 = Lt.rho0;
        p.err = bp.err;
        p.wait_tries = kWaitTries;
        p.eq2 = 0;
        p.has_drag = 0;
        p.drag_d0 = p.drag_d1 = p.us_x = p.us_y = 0.f;
        c.k = Lt.k; c.w = Lt.w; c.A = Lt.A; c.U0 = Lt.U0; c.phi0 = Lt.phi0; c.nu = Lt.nu; c.rho0 = Lt.rho0;
        sincosf(Lt.w * (float)t, &c.st, &c.ct);
        c.ct1 = cosf(Lt.w * (float)(t + 1));

        const int x0 = tx * 60;
        c.y0 = ty * Lt.H;
        c.y1 = min(c.y0 + Lt.H, Lt.ny);
        c.wsp = ((kPadCols + x0 - kGhost) / A) * A;
        c.ww = ((kPadCols + x0 + 63 + A - 1) / A) * A - c.wsp;
        c.xa = x0 - 2 + 2 * lane;
        c.sa = kPadCols + c.xa - c.wsp;
        c.st_pair = lane >= 1 && lane < 31 && c.xa < Lt.nx;
        float sa_, ca_, sb_, cb_;
        sincospif(2.0f * (float)c.xa / (float)Lt.nx, &sa_, &ca_);
        sincospif(2.0f * (float)(c.xa + 1) / (float)Lt.nx, &sb_, &cb_);
        c.sx2 = mk(sa_, sb_);
        c.cx2 = mk(ca_, cb_);
        c.rlo = c.y0 - 3;
        c.rhi = c.y1 + 2;
        c.waited = c.rlo - 1;
        c.issued = c.rlo - 1;
        c.fast_strip = true;
        c.fast_lo = c.y0;
        c.fast_hi = c.y1 + 1;

        c.setup_copies(&Lt.map[t & 1]);
        __syncwarp();
        fence_proxy_async();
        for (int r = c.rlo; r <= min(c.y0 + kWarpSlots - 6, c.rhi); ++r) c.issue(r);
        __syncwarp();
        const bool ok = warp_run_strip<S, true>(c);
        phase = c.phase;
        if (!ok) {
            if (lane == 0) batch_drain(c, phase);
            break;
        }
    }
}

// After each batched step, before the tick: refresh the periodic ghost columns of the
// buffer every lattice's step just wrote (blockIdx.y = lattice).
template <typename S>
__global__ void batch_ghost_fill_kernel(const BatchLattice* lats, const int* clock) {
    const BatchLattice& L = lats[blockIdx.y];
    S* buf = reinterpret_cast<S*>(L.buf[(*clock + 1) & 1]);
    const long long n = 9LL * L.ny * 2 * kGhost;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        fill_ghosts<S>(buf, L.plane, L.nx, L.ny, L.P, k);
}

// After each batched step: advance the clock and re-arm the unit counter.
__global__ void batch_tick_kernel(int* clock, int* counter) {
    *clock += 1;
    *counter = 0;
}

}  // namespace lbmv

namespace lbmv {

// ---------------------------------------------------------------- batch support
// phi(x, y, t) of a batch lattice (FP32 evaluation, as in the step kernel)
__device__ __forceinline__ float batch_phi(const BatchLattice& L, int x, int y, float ct) {
    float sx, cx, sy, cy;
    sincospif(2.0f * (float)x / (float)L.nx, &sx, &cx);
    sincospif(2.0f * (float)y / (float)L.ny, &sy, &cy);
    return L.phi0 + L.A * ct * sx * sy;
}

// manufactured velocity u = (grad psi + rot Psi) / phi at (x, y, t)
__device__ __forceinline__ void batch_velocity(const BatchLattice& L, int x, int y, float ct, float st, float& ux,
                                               float& uy) {
    float sx, cx, sy, cy;
    sincospif(2.0f * (float)x / (float)L.nx, &sx, &cx);
    sincospif(2.0f * (float)y / (float)L.ny, &sy, &cy);
    const float phi = L.phi0 + L.A * ct * sx * sy;
    const float a = -(L.A * L.w / (2.0f * L.k)) * st;
    ux = (a * cx * sy + L.U0 * sx * cy) / phi;
    uy = (a * sx * cy - L.U0 * cx * sy) / phi;
}

__device__ __forceinline__ Lattice<float> batch_as_lattice(const BatchLattice& L, float scale, float inv_scale) {
    Lattice<float> Q;
    Q.plane = L.plane;
    Q.nx = L.nx;
    Q.ny = L.ny;
    Q.P = L.P;
    Q.wall_y = 0;
    Q.model_b = 0;
    Q.kappa = L.kappa;
    Q.gx = 0.f;
    Q.gy = 0.f;
    Q.scale = scale;
    Q.inv_scale = inv_scale;
    Q.rest.ax = L.kappa * L.rho0 * (1.f / 9.f);
    Q.rest.dg = L.kappa * L.rho0 * (1.f / 36.f);
    Q.rest.k59 = L.kappa * L.rho0 * (5.f / 9.f);
    Q.rest.rho0 = L.rho0;
    return Q;
}

// t = 0: f = f^eq(rho0, u(0), phi(0)) - F_i(u, F^B(0))/2 (F^p = 0 for uniform rho),
// written where the first pull finds it (buffer 0).
template <typename S>
__global__ void batch_init_kernel(const BatchLattice* lats, int index, float scale, float inv_scale) {
    const BatchLattice& L = lats[index];
    const Lattice<float> Q = batch_as_lattice(L, scale, inv_scale);
    const long long n = (long long)L.nx * L.ny;
    for (long long kk = blockIdx.x * (long long)blockDim.x + threadIdx.x; kk < n; kk += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(kk / L.nx), x = (int)(kk % L.nx);
        float sx, cx, sy, cy;
        sincospif(2.0f * (float)x / (float)L.nx, &sx, &cx);
        sincospif(2.0f * (float)y / (float)L.ny, &sy, &cy);
        const float ph = L.phi0 + L.A * sx * sy;
        float ux, uy;
        batch_velocity(L, x, y, 1.0f, 0.0f, ux, uy);
        float Fx, Fy;
        mms_force<float>(sx, cx, sy, cy, 1.0f, 0.0f, L.k, L.w, L.A, L.U0, L.phi0, L.nu, Fx, Fy);
        Fx *= L.rho0;
        Fy *= L.rho0;
        const float rho = L.rho0, X = L.kappa / ph, pr = ph * rho, uu = ux * ux + uy * uy;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const float exi = (float)ex_of(i), eyi = (float)ey_of(i);
            const float eu = exi * ux + eyi * uy;
            float feq;
            if (i == 0) {
                feq = pr - (5.0f / 9.0f) * L.kappa * rho - (2.0f / 3.0f) * pr * uu;
            } else {
                const float w = (i <= 4) ? (1.0f / 9.0f) : (1.0f / 36.0f);
                const float g = (i <= 4) ? (3.0f - X) * 0.5f : X;
                feq = w * (L.kappa * rho + pr * (3.0f * eu * g + 4.5f * eu * eu - 1.5f * uu));
            }
            const float w = (i == 0) ? (4.0f / 9.0f) : ((i <= 4) ? (1.0f / 9.0f) : (1.0f / 36.0f));
            const float Fi = w * ((3.0f * (exi - ux) + 9.0f * eu * exi) * Fx + (3.0f * (eyi - uy) + 9.0f * eu * eyi) * Fy);
            scatter_cell<S, float>(reinterpret_cast<S*>(L.buf[0]), Q, x, y, i, feq - 0.5f * Fi, ph);
        }
    }
}

// Post-streaming populations of cell (x, y) of a batch lattice at step t, decoded in
// FP64: the stored deviation (scaled) plus the FP64 rest value at the kernel's own FP32
// phi(x, y, t), so the read-back adds no rounding at the scale of f.
template <typename S>
__device__ __forceinline__ void batch_pull(const BatchLattice& L, const Lattice<float>& Q, int t, int x, int y,
                                           double f[9]) {
    const S* buf = reinterpret_cast<const S*>(L.buf[t & 1]);
    const double ph = (double)batch_phi(L, x, y, cosf(L.w * (float)t));
    const double kr = (double)L.kappa * (double)L.rho0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int sx = x - ex_of(i);
        const int sy = (y - ey_of(i) + L.ny) % L.ny;
        const S v = buf[i * L.plane + cell_off(L.P, sx, sy)];
        const double rest = i == 0 ? ph * (double)L.rho0 - kr * (5.0 / 9.0) : kr * (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
        f[i] = decd(v, rest, (double)Q.inv_scale);
    }
}

template <typename S>
__global__ void batch_get_kernel(const BatchLattice* lats, int index, const int* clock, double* out, float scale,
                                 float inv_scale) {
    const BatchLattice& L = lats[index];
    const Lattice<float> Q = batch_as_lattice(L, scale, inv_scale);
    const int t = *clock;
    const long long n = (long long)L.nx * L.ny;
    for (long long kk = blockIdx.x * (long long)blockDim.x + threadIdx.x; kk < n; kk += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(kk / L.nx), x = (int)(kk % L.nx);
        double f[9];
        batch_pull<S>(L, Q, t, x, y, f);
#pragma unroll
        for (int i = 0; i < 9; ++i) out[i * n + kk] = f[i];
    }
}

// Eq. (7): rho = sum f / phi into a dense array (pass 1 of the velocity error)
template <typename S>
__global__ void batch_rho_kernel(const BatchLattice* lats, int index, const int* clock, double* rho, float scale,
                                 float inv_scale) {
    const BatchLattice& L = lats[index];
    const Lattice<float> Q = batch_as_lattice(L, scale, inv_scale);
    const int t = *clock;
    const float ct = cosf(L.w * (float)t);
    const long long n = (long long)L.nx * L.ny;
    for (long long kk = blockIdx.x * (long long)blockDim.x + threadIdx.x; kk < n; kk += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(kk / L.nx), x = (int)(kk % L.nx);
        double f[9];
        batch_pull<S>(L, Q, t, x, y, f);
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) s += f[i];
        rho[kk] = s / (double)batch_phi(L, x, y, ct);
    }
}

// Eq. (7), (13), (26): u from the populations with F = F^p + F^B(t), against the
// manufactured velocity at t; partial sums of |u - u_ref|^2 and |u_ref|^2 per block
template <typename S>
__global__ void batch_err_kernel(const BatchLattice* lats, int index, const int* clock, const double* rho,
                                 double* partial, float scale, float inv_scale) {
    const BatchLattice& L = lats[index];
    const Lattice<float> Q = batch_as_lattice(L, scale, inv_scale);
    const int t = *clock;
    float st, ct;
    sincosf(L.w * (float)t, &st, &ct);
    const long long n = (long long)L.nx * L.ny;
    double num = 0, den = 0;
    for (long long kk = blockIdx.x * (long long)blockDim.x + threadIdx.x; kk < n; kk += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(kk / L.nx), x = (int)(kk % L.nx);
        double f[9];
        batch_pull<S>(L, Q, t, x, y, f);
        double s = 0, jx = 0, jy = 0;
#pragma unroll
        for (int i = 0; i < 9; ++i) { s += f[i]; jx += (double)ex_of(i) * f[i]; jy += (double)ey_of(i) * f[i]; }
        float gx, gy;
        grad_dense_even<float>(rho, Q, x, y, gx, gy);
        float sx, cx, sy, cy;
        sincospif(2.0f * (float)x / (float)L.nx, &sx, &cx);
        sincospif(2.0f * (float)y / (float)L.ny, &sy, &cy);
        const float ph = L.phi0 + L.A * ct * sx * sy;
        float Fx, Fy;
        mms_force<float>(sx, cx, sy, cy, ct, st, L.k, L.w, L.A, L.U0, L.phi0, L.nu, Fx, Fy);
        const float kp = (L.kappa - ph) * (1.0f / 3.0f);
        Fx = kp * gx + L.rho0 * Fx;
        Fy = kp * gy + L.rho0 * Fy;
        const double ux = (jx + 0.5 * (double)Fx) / s, uy = (jy + 0.5 * (double)Fy) / s;
        float uxr, uyr;
        batch_velocity(L, x, y, ct, st, uxr, uyr);
        num += (ux - uxr) * (ux - uxr) + (uy - uyr) * (uy - uyr);
        den += (double)uxr * uxr + (double)uyr * uyr;
    }
    block_reduce3(num, den, 0.0, partial);
}

// One lattice as an ordinary grid of tiles_x x ceil(ny / H) CTAs (one strip of H rows
// each): the launch-per-lattice form the persistent kernel is compared against.
template <typename S, int MINB>
__global__ void __launch_bounds__(32, MINB) vanse_batch_one_kernel(const __grid_constant__ BatchParams bp, int index,
                                                                  int H) {
    using L = WarpLayout<S>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x;
    constexpr int A = L::A;
    if (lane == 0) {
        for (int k = 0; k < kWarpSlots; ++k) mbar_init(reinterpret_cast<uint64_t*>(smem) + k, 1);
        fence_mbar_init();
    }
    __syncwarp();
    const int t = *bp.clock;
    const BatchLattice& Lt = bp.lat[index];
    const int tx = blockIdx.x % Lt.tiles_x, ty = blockIdx.x / Lt.tiles_x;
    BatchCtx<S> c;
    c.smem = smem;
    c.lane = lane;
    c.step = (uint32_t)t;
    c.salt = (uint32_t)index * 0x27d4eb2fu;
    c.aborted = false;
    c.first_bad = 0x7fffffff;
    c.phase = 0;
    StepParams<float>& p = c.p;
    p.src = Lt.buf[t & 1];
    p.dst = Lt.buf[(t + 1) & 1];
    p.plane = Lt.plane;
    p.nx = Lt.nx;
    p.ny = Lt.ny;
    p.P = Lt.P;
    p.W = 60;
    p.H = H;
    p.wall_y = 0;
    p.unsteady = 1;
    p.has_fb = 1;
    p.model_b = 0;
    p.nR = 0;
    p.kappa = Lt.kappa;
    p.gx = 0.f;
    p.gy = 0.f;
    p.s_e = Lt.s_e; p.s_eps = Lt.s_eps; p.s_q = Lt.s_q; p.s_nu = Lt.s_nu;
    p.h_e = Lt.h_e; p.h_eps = Lt.h_eps; p.h_q = Lt.h_q; p.h_nu = Lt.h_nu;
    p.scale = bp.scale;
    p.inv_scale = bp.inv_scale;
    p.hs_e = Lt.h_e * bp.scale; p.hs_eps = Lt.h_eps * bp.scale;
    p.hs_q = Lt.h_q * bp.scale; p.hs_nu = Lt.h_nu * bp.scale;
    p.rho0s = Lt.rho0 * bp.scale;
    p.kp3 = bp.inv_scale * (1.f / 3.f);
    p.rest.ax = Lt.kappa * Lt.rho0 * (1.f / 9.f);
    p.rest.dg = Lt.kappa * Lt.rho0 * (1.f / 36.f);
    p.rest.k59 = Lt.kappa * Lt.rho0 * (5.f / 9.f);
    p.rest.rho0 = Lt.rho0;
    p.err = bp.err;
    p.wait_tries = kWaitTries;
    p.eq2 = 0;
    p.has_drag = 0;
    p.drag_d0 = p.drag_d1 = p.us_x = p.us_y = 0.f;
    c.k = Lt.k; c.w = Lt.w; c.A = Lt.A; c.U0 = Lt.U0; c.phi0 = Lt.phi0; c.nu = Lt.nu; c.rho0 = Lt.rho0;
    sincosf(Lt.w * (float)t, &c.st, &c.ct);
    c.ct1 = cosf(Lt.w * (float)(t + 1));
    const int x0 = tx * 60;
    c.y0 = ty * H;
    c.y1 = min(c.y0 + H, Lt.ny);
    c.wsp = ((kPadCols + x0 - kGhost) / A) * A;
    c.ww = ((kPadCols + x0 + 63 + A - 1) / A) * A - c.wsp;
    c.xa = x0 - 2 + 2 * lane;
    c.sa = kPadCols + c.xa - c.wsp;
    c.st_pair = lane >= 1 && lane < 31 && c.xa < Lt.nx;
    float sa_, ca_, sb_, cb_;
    sincospif(2.0f * (float)c.xa / (float)Lt.nx, &sa_, &ca_);
    sincospif(2.0f * (float)(c.xa + 1) / (float)Lt.nx, &sb_, &cb_);
    c.sx2 = mk(sa_, sb_);
    c.cx2 = mk(ca_, cb_);
    c.rlo = c.y0 - 3;
    c.rhi = c.y1 + 2;
    c.waited = c.rlo - 1;
    c.issued = c.rlo - 1;
    c.fast_strip = true;
    c.fast_lo = c.y0;
    c.fast_hi = c.y1 + 1;
    c.setup_copies(&Lt.map[t & 1]);
    for (int r = c.rlo; r <= min(c.y0 + kWarpSlots - 6, c.rhi); ++r) c.issue(r);
    __syncwarp();
    const bool ok = warp_run_strip<S, true>(c);
    if (!ok && lane == 0) batch_drain(c, c.phase);
}

}  // namespace lbmv
