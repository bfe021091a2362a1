// vanse_warp.cuh -- the fused D2Q9 MRTLB-VANSE stream + collide kernel with one
// warp per CTA, two adjacent columns per lane on packed FP32 pairs.
//
// Same method and the same three row phases as vanse_step.cuh; the differences:
//   * a CTA is one warp: lane l owns columns xa = x0 - 2 + 2l, xb = xa + 1, the
//     warp covers 64 columns and stores W = 60 of them;
//   * x-neighbours come from the adjacent lanes by shuffles (no shared exchange
//     rows, no CTA barriers), so every warp runs its row pipeline independently and
//     a stalled warp never holds the others up;
//   * arithmetic on the packed FP32 pairs of vanse_pair.cuh (FFMA2 / FADD2 / FMUL2);
//   * the source-row ring (8 slots, mbarriers) is per warp; the slot of row p - 3 is
//     refilled with row p + 5 at the start of iteration p: the nine population rows
//     by one 3-D tensor copy (cp.async.bulk.tensor, lane 0), the phi / phi(t+1) /
//     force rows by 1-D bulk copies (lanes 1..4);
//   * interior rows of steady, field-free strips run one branch-free block (no
//     wall / validity / field tests), so the collision of one row can overlap the
//     pulls and shuffles of the next two.
// Lanes 0 and 31 carry the halo columns: lane 0 finishes nothing, lane 31 nothing;
// lanes 1..30 store their two columns.
#pragma once

#include "vanse_common.cuh"
#include "vanse_pair.cuh"
#include "vanse_step.cuh"

namespace lbmv {

// source-row ring of the one-warp kernel: rows p-2 .. p+1 in use, the rest prefetch
#ifndef LBMV_WARP_SLOTS
#define LBMV_WARP_SLOTS 8
#endif
constexpr int kWarpSlots = LBMV_WARP_SLOTS;

// resident one-warp CTAs per SM the register allocation is sized for
#ifndef LBMV_WARP_MINB
#define LBMV_WARP_MINB 8
#endif

// NPL: planes staged per source row (the 9 populations; 11 with the momentum base,
// whose J planes follow them in the same buffer)
template <typename S, int NPL = 9>
struct WarpLayout {
    static constexpr int A = 16 / (int)sizeof(S);
    static constexpr int WW = 64 + 2 * A;           // staged row width (elements)
    static constexpr int kPop = 128;                // after the mbarriers
    static constexpr int kPopRow = WW * (int)sizeof(S);
    static constexpr int kPopSlot = (NPL * kPopRow + 127) / 128 * 128;   // tensor-copy destinations: 128-byte aligned
    static constexpr int kAux = kPop + kWarpSlots * kPopSlot;
    static constexpr int kAuxRow = WW * 4;
    static constexpr size_t bytes(int nR) { return (size_t)kAux + (size_t)kWarpSlots * nR * kAuxRow; }
};

// ring slot of source row r (r >= -3); a mask when the ring size is a power of two
__device__ __forceinline__ int wslot(int r) {
    if constexpr ((kWarpSlots & (kWarpSlots - 1)) == 0) return r & (kWarpSlots - 1);
    else return ((r % kWarpSlots) + kWarpSlots) % kWarpSlots;
}

// One source row of a strip is staged by a few copies into one ring slot, each issued
// by one lane; lane 0 first arms the slot's mbarrier with the row's total byte count.
// The one-warp step kernel stages the nine population rows with one 3-D tensor copy
// (lane 0; a copy costs its warp hundreds of cycles to issue, so one request instead
// of nine took the step from 67.7 to 73.8 GLUPS) and phi, phi(t+1), F^B_x, F^B_y with
// 1-D bulk copies; the batch kernels issue one 1-D bulk copy per population row.
struct RowCopy {
    const char* src = nullptr;   // this lane's source at row 0
    uint32_t pitch = 0;          // bytes per source row
    uint32_t dst = 0;            // shared address of this lane's destination in slot 0
    uint32_t stride = 0;         // bytes between ring slots
    uint32_t bytes = 0;          // bytes of this lane's copy (0: none)
    uint32_t tx = 0;             // bytes of the whole row (every lane)
    uint32_t bar0 = 0;           // shared address of the slot-0 mbarrier
    const CUtensorMap* map = nullptr;   // this lane copies a tensor box: the map, its first column
    int xcol = 0;

    // all lanes: stage global row gr into ring slot s
    __device__ __forceinline__ void issue(int lane, int s, int gr) const {
        const uint32_t b = bar0 + 8u * (uint32_t)s;
        if (lane == 0) mbar_expect_tx_at(b, tx);
        __syncwarp();
        if (map) tma_load_3d(dst + (uint32_t)s * stride, map, xcol, gr, 0, b);
        else if (bytes) bulk_g2s_at(dst + (uint32_t)s * stride, src + (long long)gr * (long long)pitch, bytes, b);
    }
};

// Compensated sums of the post-collision m_0, j_x, j_y of the column pairs a lane
// writes (step-sum variants of the one-warp kernel).
struct PairSums {
    V2 s[3] = {bc(0.f), bc(0.f), bc(0.f)}, c[3] = {bc(0.f), bc(0.f), bc(0.f)};
    __device__ __forceinline__ void add(int k, V2 v) {
        const V2 y = v - c[k];
        const V2 t = s[k] + y;
        c[k] = (t - s[k]) - y;
        s[k] = t;
    }
    __device__ __forceinline__ double value(int k) const {
        return ((double)s[k].v.x - (double)c[k].v.x) + ((double)s[k].v.y - (double)c[k].v.y);
    }
};

template <typename S, bool SUMS = false, bool EQ2 = false, bool SOLID = false, bool JB = false, bool NEE = false>
struct WarpCtx {
    static constexpr int kNPL = JB ? 11 : 9;   // planes per staged row
    using L = WarpLayout<S, kNPL>;
    static constexpr bool kUnsteady = false;   // the fast path runs only on steady strips
    static constexpr bool kSums = SUMS;        // accumulate the written cells' m_0+, j+ (PairSums)
    static constexpr bool kEq2 = EQ2;          // App. B: (B2) energy-flux equilibria, (B3) penalty
    static constexpr bool kSolid = SOLID;      // phi = 0 marks solid cells (general path only)
    static constexpr bool kJB = JB;            // FP16 / BF16 deviations from the momentum base
    // the moving wall's code (row ny-1 by non-equilibrium extrapolation): compiled only
    // into the instances that may meet it, since even untaken it slows the general row
    // path by about 7 % (instruction-cache footprint)
    static constexpr bool kNee = NEE || SOLID || JB;
    const StepParams<float>& p;
    unsigned char* smem;
    int lane, xa, sa;
    int y0, y1;
    int wsp, ww;
    int rlo, rhi;
    int waited, issued;
    bool aborted;
    bool fast_strip;
    int fast_lo, fast_hi;
    RowCopy cp;
    bool st_pair;              // this lane stores its pair (lanes 1..30, first column inside)
    mutable PairSums sums;     // used when kSums
    int first_bad = 0x7fffffff;   // first row whose wait gave up (this lane)
    uint32_t step = 0, salt = 0;   // seed of the stochastic rounding of FP16/BF16 stores

    __device__ __forceinline__ uint64_t* bar(int r) const { return reinterpret_cast<uint64_t*>(smem) + wslot(r); }
    __device__ __forceinline__ const S* pop(int r) const {
        return reinterpret_cast<const S*>(smem + L::kPop + wslot(r) * L::kPopSlot) + sa;
    }
    __device__ __forceinline__ const float* aux(int r, int k) const {
        return reinterpret_cast<const float*>(smem + L::kAux) + (wslot(r) * p.nR + k) * L::WW + sa;
    }
    __device__ __forceinline__ bool row_valid(int r) const { return !p.wall_y || (r >= 0 && r < p.ny); }
    __device__ __forceinline__ uint32_t parity(int r) const { return (uint32_t)(((r - rlo) / kWarpSlots) & 1); }

    // the per-cell sources of the step for row r (this lane's two columns): phi(t),
    // phi(t+1) and the field part of F^B, staged with the populations
    __device__ __forceinline__ void row_setup(int, PRow&) const {}
    __device__ __forceinline__ V2 phi2(int r, const PRow&) const {
        return V2{*reinterpret_cast<const float2*>(aux(r, 0))};
    }
    template <bool FAST>
    __device__ __forceinline__ V2 phin2(int r, const PRow& st) const {
        return (!FAST && p.unsteady) ? V2{*reinterpret_cast<const float2*>(aux(r, 1))} : phi2(r, st);
    }
    template <bool FAST>
    __device__ __forceinline__ void add_field_force(int r, const PRow&, V2& Fx, V2& Fy) const {
        if (!FAST && p.has_fb) {
            const int k = p.unsteady ? 2 : 1;
            Fx = Fx + V2{*reinterpret_cast<const float2*>(aux(r, k))};
            Fy = Fy + V2{*reinterpret_cast<const float2*>(aux(r, k + 1))};
        }
    }

    // this lane's part of staging a source row (see RowCopy): lane 0 the nine
    // population rows, a box of the whole staged width WW (wsp is a multiple of 16
    // bytes, so the box starts on a 16-byte boundary, and wsp + WW stays inside the
    // padded row); lanes 1..nR the aux rows
    __device__ __forceinline__ void setup_copies() {
        const uint32_t base = smem_u32(smem);
        cp.bar0 = base;
        cp.tx = (uint32_t)kNPL * (uint32_t)(L::WW * (int)sizeof(S)) + (uint32_t)p.nR * (uint32_t)(ww * 4);
        if (lane == 0) {
            cp.map = &p.pop_map;
            cp.xcol = wsp;
            cp.dst = base + (uint32_t)L::kPop;
            cp.stride = (uint32_t)L::kPopSlot;
        } else if (lane <= p.nR) {
            // aux rows in the order phi, phi(t+1) (unsteady), F^B_x, F^B_y (force field)
            const int k = lane - 1;
            const float* a = p.phi;
            if (k == 1 && p.unsteady) a = p.phin;
            else if (k >= 1) a = p.fb + (k - (p.unsteady ? 2 : 1)) * p.plane;
            cp.src = reinterpret_cast<const char*>(a + wsp);
            cp.pitch = (uint32_t)(p.P * 4);
            cp.dst = base + (uint32_t)(L::kAux + k * L::kAuxRow);
            cp.stride = (uint32_t)(p.nR * L::kAuxRow);
            cp.bytes = (uint32_t)(ww * 4);
        }
    }
    // all lanes: load source row r into its slot
    __device__ __forceinline__ void issue(int r) {
        issued = r;
        int gr = r;
        if (!p.wall_y) { gr %= p.ny; if (gr < 0) gr += p.ny; }
        cp.issue(lane, wslot(r), gr);
    }
    __device__ __forceinline__ void wait_upto(int r) {
        r = min(r, rhi);
        while (waited < r) {
            ++waited;
            if (!mbar_wait_bounded(bar(waited), parity(waited), p.wait_tries)) {
                first_bad = min(first_bad, waited);
                aborted = true;
                atomicExch(p.err, 1);
            }
        }
    }
};

// 32-bit integer mixer (xor-shift / multiply rounds); seeds the stochastic rounding
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// neighbour values across lanes: the left neighbour of xa is lane-1's xb, the right
// neighbour of xb is lane+1's xa
__device__ __forceinline__ float left_of(V2 v) { return __shfl_up_sync(0xffffffffu, v.v.y, 1); }
__device__ __forceinline__ float right_of(V2 v) { return __shfl_down_sync(0xffffffffu, v.v.x, 1); }

// ------------------------------------------------------------------ solid cells
// The Eq. (10) stencil next to solid cells (phi = 0). A solid neighbour reads the value
// mirrored about the solid surface: an axis neighbour the cell itself; a diagonal one
// the mean of its two axis images (x+dx, y), (x, y+dy) when both are fluid, the fluid
// one when one is, the cell itself when neither is; negated for a vector component.
// Being linear in the field, the rule is a set of 3 x 3 weights per cell, built once
// from the solid mask (branch-free) and applied to every field with that parity.
// m9: the solid bits of column C's neighbourhood (bit 3 (dy + 1) + dx + 1); sg = -1
// for a vector component, +1 for a scalar. kx, ky: 12 x the d/dx, d/dy weights at
// [dy + 1][dx + 1].
__device__ __forceinline__ void solid_weights(uint32_t m9, float sg, float (&kx)[3][3], float (&ky)[3][3]) {
    auto bit = [&](int dx, int dy) { return ((m9 >> (3 * (dy + 1) + dx + 1)) & 1u) != 0u; };
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            const float cw = (dx != 0 && dy != 0) ? 1.f : 4.f;   // 36 w_i
            kx[dy + 1][dx + 1] = (dx == 0 && dy == 0) ? 0.f : cw * (float)dx;
            ky[dy + 1][dx + 1] = (dx == 0 && dy == 0) ? 0.f : cw * (float)dy;
        }
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            if (dx == 0 && dy == 0) continue;
            const float cw = (dx != 0 && dy != 0) ? 1.f : 4.f;
            const bool sol = bit(dx, dy);
            const float wx = sol ? cw * (float)dx : 0.f, wy = sol ? cw * (float)dy : 0.f;
            kx[dy + 1][dx + 1] -= wx;
            ky[dy + 1][dx + 1] -= wy;
            if (dx == 0 || dy == 0) {
                kx[1][1] = fmaf(sg, wx, kx[1][1]);
                ky[1][1] = fmaf(sg, wy, ky[1][1]);
            } else {
                const bool fa = !bit(dx, 0), fb = !bit(0, dy);
                const float ca = fa ? (fb ? 0.5f : 1.f) : 0.f, cb = fb ? (fa ? 0.5f : 1.f) : 0.f;
                const float cc = (fa || fb) ? 0.f : 1.f;
                kx[1][dx + 1] = fmaf(sg * ca, wx, kx[1][dx + 1]);
                ky[1][dx + 1] = fmaf(sg * ca, wy, ky[1][dx + 1]);
                kx[dy + 1][1] = fmaf(sg * cb, wx, kx[dy + 1][1]);
                ky[dy + 1][1] = fmaf(sg * cb, wy, ky[dy + 1][1]);
                kx[1][1] = fmaf(sg * cc, wx, kx[1][1]);
                ky[1][1] = fmaf(sg * cc, wy, ky[1][1]);
            }
        }
}

// sum_{dy, dx} k[dy + 1][dx + 1] w[dy + 1][1 + C + dx]: column C of the pair
template <int C>
__device__ __forceinline__ float solid_apply(const float (&w)[3][4], const float (&k)[3][3]) {
    float a = 0.f;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) a = fmaf(k[r][c], w[r][C + c], a);
    return a;
}

// the 4-wide row window of a pair field: xa-1 (from the lane below), xa, xb, xb+1
__device__ __forceinline__ void win_row(float (&w)[4], V2 v) {
    w[0] = __shfl_up_sync(0xffffffffu, v.v.y, 1);
    w[1] = v.v.x;
    w[2] = v.v.y;
    w[3] = __shfl_down_sync(0xffffffffu, v.v.x, 1);
}

// Solid bits of the pair's neighbourhoods at row y (bit layout of PRow::sm), from the
// staged phi rows y-1 .. y+1: past a half-way y wall the mirror row (the row itself),
// past the moving wall the extrapolated row, which is never solid.
template <typename Ctx>
__device__ __forceinline__ uint32_t solid_mask(const Ctx& c, int y) {
    const auto& p = c.p;
    const float* q0 = c.aux(y, 0);
    const bool lo_m = p.wall_y && y == 0;
    const bool hi_m = p.wall_y && y == p.ny - 1;
    const float* ql = lo_m ? q0 : c.aux(y - 1, 0);
    const float* qh = hi_m ? q0 : c.aux(y + 1, 0);
    const bool hi_fluid = hi_m && p.nee_top;
    uint32_t m = 0;
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
        const uint32_t bl = ql[jj - 1] == 0.f, bm = q0[jj - 1] == 0.f, bh = !hi_fluid && qh[jj - 1] == 0.f;
#pragma unroll
        for (int col = 0; col < 2; ++col) {
            const int dx = jj - 1 - col;
            if (dx < -1 || dx > 1) continue;
            m |= (bl << (9 * col + dx + 1)) | (bm << (9 * col + 3 + dx + 1)) | (bh << (9 * col + 6 + dx + 1));
        }
    }
    return m;
}
__device__ __forceinline__ bool solid_own(uint32_t m, int col) { return (m >> (9 * col + 4)) & 1u; }
// a fluid cell with at least one solid neighbour
__device__ __forceinline__ bool solid_next(uint32_t m, int col) {
    return !solid_own(m, col) && ((m >> (9 * col)) & 0x1EFu) != 0;
}

template <typename S, bool FAST, typename Ctx>
__device__ __forceinline__ void warp_phase1(const Ctx& c, PRow& st, int r) {
    using IO = PairIO<S>;
    constexpr int RW = WarpLayout<S>::WW;
    const auto& p = c.p;
    c.row_setup(r, st);
    const V2 phi = c.phi2(r, st);
    const float ia = p.inv_scale;
    // the stored values are deviations from the rest state of Eq. (14) times the
    // storage scale (1 for FP32, a power of two for FP16/BF16); this kernel keeps them
    // as they are: f0..f8 below are scale x (f_i - f_i^rest), the rest state's moments
    // are added back analytically, and the collision runs in these scaled units (the
    // scale is a power of two, so this changes no rounding)
    const S* cur = c.pop(r);
    V2 f0, f1, f2, f3, f4, f5, f6, f7, f8;
    f0 = IO::dev(IO::al(cur), ia);
    f1 = IO::dev(IO::un(cur + 1 * RW - 1), ia);
    f3 = IO::dev(IO::un(cur + 3 * RW + 1), ia);
    if (!FAST && p.wall_y && r == 0) {
        f2 = IO::dev(IO::al(cur + 4 * RW), ia);
        f5 = IO::dev(IO::al(cur + 7 * RW), ia);
        f6 = IO::dev(IO::al(cur + 8 * RW), ia);
    } else {
        const S* lo = c.pop(r - 1);
        f2 = IO::dev(IO::al(lo + 2 * RW), ia);
        f5 = IO::dev(IO::un(lo + 5 * RW - 1), ia);
        f6 = IO::dev(IO::un(lo + 6 * RW + 1), ia);
    }
    if (!FAST && p.wall_y && r == p.ny - 1) {
        f4 = IO::dev(IO::al(cur + 2 * RW), ia);
        f7 = IO::dev(IO::al(cur + 5 * RW), ia);
        f8 = IO::dev(IO::al(cur + 6 * RW), ia);
    } else {
        const S* hi = c.pop(r + 1);
        f4 = IO::dev(IO::al(hi + 4 * RW), ia);
        f7 = IO::dev(IO::un(hi + 7 * RW + 1), ia);
        f8 = IO::dev(IO::un(hi + 8 * RW - 1), ia);
    }
    if constexpr (Ctx::kJB) {
        // momentum base: the value in slot k of cell c is the deviation from f_k^rest +
        // 3 w_k e_k . J(c), J(c) in the slot row's planes 9 and 10 (scaled units); add
        // back each pulled slot's term at the cell it was read from
        auto jx = [&](const S* row, int off, bool aligned) {
            return aligned ? IO::dev(IO::al(row + 9 * RW + off), ia) : IO::dev(IO::un(row + 9 * RW + off), ia);
        };
        auto jy = [&](const S* row, int off, bool aligned) {
            return aligned ? IO::dev(IO::al(row + 10 * RW + off), ia) : IO::dev(IO::un(row + 10 * RW + off), ia);
        };
        constexpr float t3 = 1.f / 3.f, t12 = 1.f / 12.f;
        f1 = fma2(t3, jx(cur, -1, false), f1);     // slot 1 of (x-1, y): e = (1, 0)
        f3 = fma2(-t3, jx(cur, 1, false), f3);     // slot 3 of (x+1, y): e = (-1, 0)
        if (!FAST && p.wall_y && r == 0) {         // slots 4, 7, 8 of the cell itself
            const V2 ox = jx(cur, 0, true), oy = jy(cur, 0, true);
            f2 = fma2(-t3, oy, f2);
            f5 = fma2(-t12, ox + oy, f5);
            f6 = fma2(t12, ox - oy, f6);
        } else {
            const S* lo = c.pop(r - 1);
            f2 = fma2(t3, jy(lo, 0, true), f2);                             // slot 2 of (x, y-1)
            f5 = fma2(t12, jx(lo, -1, false) + jy(lo, -1, false), f5);      // slot 5 of (x-1, y-1)
            f6 = fma2(t12, jy(lo, 1, false) - jx(lo, 1, false), f6);        // slot 6 of (x+1, y-1)
        }
        if (!FAST && p.wall_y && r == p.ny - 1) {  // slots 2, 5, 6 of the cell itself
            const V2 ox = jx(cur, 0, true), oy = jy(cur, 0, true);
            f4 = fma2(t3, oy, f4);
            f7 = fma2(t12, ox + oy, f7);
            f8 = fma2(t12, oy - ox, f8);
        } else {
            const S* hi = c.pop(r + 1);
            f4 = fma2(-t3, jy(hi, 0, true), f4);                            // slot 4 of (x, y+1)
            f7 = fma2(-t12, jx(hi, 1, false) + jy(hi, 1, false), f7);       // slot 7 of (x+1, y+1)
            f8 = fma2(t12, jx(hi, -1, false) - jy(hi, -1, false), f8);      // slot 8 of (x-1, y+1)
        }
    }
    bool sol_a = false, sol_b = false;
    if constexpr (Ctx::kSolid) {
        // a link whose source cell is solid (phi = 0) is a half-way bounce-back link:
        // the population comes from the opposite slot of this cell (the rows past a
        // y wall were handled above). The solid flags of the 3 x 4 window first; rows
        // of warps with no solid cell in it keep the pulls as they are (one vote), the
        // others select branch-free.
        const float* q0 = c.aux(r, 0);
        const bool lo_in = !(p.wall_y && r == 0), hi_in = !(p.wall_y && r == p.ny - 1);
        const float* ql = lo_in ? c.aux(r - 1, 0) : q0;
        const float* qh = hi_in ? c.aux(r + 1, 0) : q0;
        bool s0[4], sl[4], sh[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            s0[j] = q0[j - 1] == 0.f;
            sl[j] = lo_in && ql[j - 1] == 0.f;
            sh[j] = hi_in && qh[j - 1] == 0.f;
        }
        sol_a = s0[1];
        sol_b = s0[2];
        const bool any = s0[0] | s0[1] | s0[2] | s0[3] | sl[0] | sl[1] | sl[2] | sl[3] | sh[0] | sh[1] | sh[2] | sh[3];
        if (__any_sync(0xffffffffu, any)) {
            auto pick = [&](V2 f, int slot, bool ka, bool kb) {
                const V2 o = IO::dev(IO::al(cur + slot * RW), ia);
                return mk(ka ? o.v.x : f.v.x, kb ? o.v.y : f.v.y);
            };
            f1 = pick(f1, 3, s0[0], s0[1]);
            f3 = pick(f3, 1, s0[2], s0[3]);
            f2 = pick(f2, 4, sl[1], sl[2]);
            f5 = pick(f5, 7, sl[0], sl[1]);
            f6 = pick(f6, 8, sl[2], sl[3]);
            f4 = pick(f4, 2, sh[1], sh[2]);
            f7 = pick(f7, 5, sh[2], sh[3]);
            f8 = pick(f8, 6, sh[0], sh[1]);
        }
    }
    const V2 a13 = f1 + f3, a24 = f2 + f4, b57 = f5 + f7, b68 = f6 + f8;
    const V2 sax = a13 + a24, sdg = b57 + b68;
    const V2 d13 = f1 - f3, d24 = f2 - f4, d57 = f5 - f7;
    const V2 dx = d57 + (f8 - f6);
    const V2 dy = d57 + (f6 - f8);
    st.m[0] = f0 + sax + sdg;
    st.m[1] = fma2(-4.f, f0, fma2(2.f, sdg, -sax));
    st.m[2] = fma2(4.f, f0, fma2(-2.f, sax, sdg));
    st.m[3] = d13 + dx;
    st.m[4] = fma2(-2.f, d13, dx);
    st.m[5] = d24 + dy;
    st.m[6] = fma2(-2.f, d24, dy);
    st.m[7] = a13 - a24;
    st.m[8] = b57 - b68;
    // m[0..2] are the deviations of sum f, e and eps from the rest state's phi rho0,
    // rho0 (2 kappa - 4 phi) and rho0 (4 phi - 3 kappa); rho holds rho - rho0. 1/phi,
    // the full sum f and the full rho are kept for phases 2 and 3 (cheaper than
    // forming them there)
    st.iphi = rcp2(phi);
    st.rho = st.m[0] * st.iphi;   // scale x (rho - rho0)
    if constexpr (sizeof(S) == 4) {
        st.mf = fma2(p.rest.rho0, phi, st.m[0]);
        st.rf = st.rho + p.rest.rho0;
    } else {
        st.mf = fma2(p.rest.rho0, phi, ia * st.m[0]);
        st.rf = fma2(ia, st.rho, bc(p.rest.rho0));
    }
    if constexpr (Ctx::kSolid) {
        // a solid cell holds no populations: a finite zero state (its neighbours read it
        // through the mirrored ghost values of the solid stencil, never directly)
        if (sol_a || sol_b) {
            auto z = [&](V2 v) { return mk(sol_a ? 0.f : v.v.x, sol_b ? 0.f : v.v.y); };
#pragma unroll
            for (int k = 0; k < 9; ++k) st.m[k] = z(st.m[k]);
            st.iphi = z(st.iphi);
            st.rho = z(st.rho);
            st.mf = z(st.mf);
            st.rf = z(st.rf);
        }
    }
}

template <typename S, bool FAST, typename Ctx>
__device__ __forceinline__ void warp_phase2(const Ctx& c, const PRow& An, PRow& Bs, const PRow& Cs, int p2) {
    const auto& p = c.p;
    constexpr float tw = 1.0f / 12.0f;
    V2 dlo = Cs.dr, wlo = Cs.wr, dhi = An.dr, whi = An.wr;
    if (!FAST && p.wall_y && (p2 == 0 || p2 == p.ny - 1)) {
        if (p2 == 0) { dlo = Bs.dr; wlo = Bs.wr; }
        if (p2 == p.ny - 1) {
            // rho's ghost past a half-way wall is the mirror row (the row itself); past
            // the moving wall row it extrapolates linearly, 2 (row ny-1) - (row ny-2)
            if (Ctx::kNee && p.nee_top) { dhi = fma2(2.f, Bs.dr, -Cs.dr); whi = fma2(2.f, Bs.wr, -Cs.wr); }
            else { dhi = Bs.dr; whi = Bs.wr; }
        }
    }
    V2 gx = tw * fma2(4.f, Bs.dr, dlo + dhi);
    V2 gy = tw * (whi - wlo);
    bool sol_a = false, sol_b = false;
    if constexpr (Ctx::kSolid) {
        const uint32_t sm = solid_mask(c, p2);
        Bs.sm = sm;
        sol_a = solid_own(sm, 0);
        sol_b = solid_own(sm, 1);
        const bool na = solid_next(sm, 0), nb = solid_next(sm, 1);
        if (__any_sync(0xffffffffu, na || nb)) {
            // rho of the rows below and above: past a wall the row itself, past the
            // moving wall 2 (row ny-1) - (row ny-2)
            V2 lo = Cs.rho, hi = An.rho;
            if (p.wall_y && p2 == 0) lo = Bs.rho;
            if (p.wall_y && p2 == p.ny - 1) hi = p.nee_top ? fma2(2.f, Bs.rho, -Cs.rho) : Bs.rho;
            float w[3][4];
            win_row(w[0], lo);
            win_row(w[1], Bs.rho);
            win_row(w[2], hi);
            float kx[3][3], ky[3][3];
            solid_weights(sm & 0x1FFu, 1.f, kx, ky);
            if (na) { gx.v.x = tw * solid_apply<0>(w, kx); gy.v.x = tw * solid_apply<0>(w, ky); }
            solid_weights((sm >> 9) & 0x1FFu, 1.f, kx, ky);
            if (nb) { gx.v.y = tw * solid_apply<1>(w, kx); gy.v.y = tw * solid_apply<1>(w, ky); }
        }
    }
    const V2 phi = c.phi2(p2, Bs);
    // (kappa - phi) / 3 times 1/scale: the rho differences are in scaled units
    const float k3 = sizeof(S) == 4 ? 1.f / 3.f : p.kp3;
    const V2 kp = p.model_b ? bc((p.kappa - 1.f) * k3) : k3 * (bc(p.kappa) - phi);
    V2 Fx = fma2(kp, gx, p.gx * phi);
    V2 Fy = fma2(kp, gy, p.gy * phi);
    c.template add_field_force<FAST>(p2, Bs, Fx, Fy);
    const V2 m0 = Bs.mf;
    const V2 jx = sizeof(S) == 4 ? Bs.m[3] : p.inv_scale * Bs.m[3];
    const V2 jy = sizeof(S) == 4 ? Bs.m[5] : p.inv_scale * Bs.m[5];
    V2 ux, uy;
    if (!FAST && p.has_drag) {
        // Eq. (7) with F^B += -beta (u - u_s): linear in u, solved exactly (never on the fast path)
        const V2 beta = (phi * phi) * fma2(-p.drag_d1, phi, bc(p.drag_d0 + p.drag_d1));
        const V2 inv = rcp2(fma2(0.5f, beta, m0));
        ux = fma2(0.5f, fma2(p.us_x, beta, Fx), jx) * inv;
        uy = fma2(0.5f, fma2(p.us_y, beta, Fy), jy) * inv;
        Fx = Fx - beta * (ux + (-p.us_x));
        Fy = Fy - beta * (uy + (-p.us_y));
    } else {
        const V2 inv = rcp2(m0);
        ux = fma2(0.5f, Fx, jx) * inv;
        uy = fma2(0.5f, Fy, jy) * inv;
    }
    if constexpr (Ctx::kSolid) {
        // a solid cell: no velocity, no force, zero fields
        if (sol_a || sol_b) {
            auto z = [&](V2 v) { return mk(sol_a ? 0.f : v.v.x, sol_b ? 0.f : v.v.y); };
            ux = z(ux); uy = z(uy); Fx = z(Fx); Fy = z(Fy);
        }
        Bs.rfu = Bs.rf;
        Bs.mfu = Bs.mf;
    }
    Bs.Fx = Fx; Bs.Fy = Fy; Bs.ux = ux; Bs.uy = uy;
    // the Eq. (10) x-differences / smoothed sums of rho u, u, phi rho u on row p2
    const V2 rho = Bs.rf;
    const V2 Ax = rho * ux, Ay = rho * uy, Dx = m0 * ux, Dy = m0 * uy;
    const float Axl = left_of(Ax), Axr = right_of(Ax);
    const float Ayl = left_of(Ay), Ayr = right_of(Ay);
    const float Bxl = left_of(ux), Bxr = right_of(ux);
    const float Byl = left_of(uy), Byr = right_of(uy);
    const float Dxl = left_of(Dx), Dxr = right_of(Dx);
    const float Dyl = left_of(Dy), Dyr = right_of(Dy);
    Bs.dAx = rpair(Ax, Axr) - lpair(Ax, Axl);
    Bs.dBx = rpair(ux, Bxr) - lpair(ux, Bxl);
    Bs.dBy = rpair(uy, Byr) - lpair(uy, Byl);
    Bs.dDx = rpair(Dx, Dxr) - lpair(Dx, Dxl);
    Bs.wAy = fma2(4.f, Ay, rpair(Ay, Ayr) + lpair(Ay, Ayl));
    Bs.wBy = fma2(4.f, uy, rpair(uy, Byr) + lpair(uy, Byl));
    Bs.wBx = fma2(4.f, ux, rpair(ux, Bxr) + lpair(ux, Bxl));
    Bs.wDy = fma2(4.f, Dy, rpair(Dy, Dyr) + lpair(Dy, Dyl));
    if constexpr (Ctx::kEq2) {
        // (B3) needs the cross derivatives d_x(rho u_y), d_y(rho u_x), d_x(phi rho u_y),
        // d_y(phi rho u_x) only as -kappa (d_x A_y + d_y A_x) + (d_x D_y + d_y D_x), the
        // cross derivatives of G = D - kappa A
        const V2 Gx = fma2(-p.kappa, Ax, Dx), Gy = fma2(-p.kappa, Ay, Dy);
        const float Gyl = left_of(Gy), Gyr = right_of(Gy);
        const float Gxl = left_of(Gx), Gxr = right_of(Gx);
        Bs.dGy = rpair(Gy, Gyr) - lpair(Gy, Gyl);
        Bs.wGx = fma2(4.f, Gx, rpair(Gx, Gxr) + lpair(Gx, Gxl));
    }
}

// Moving wall by non-equilibrium extrapolation (Sec. 3.1) on the top row ny-1 (Wa),
// next to the fluid row ny-2 (Fl, its Eq. 7 velocity done by phase 2): the wall
// node's moments become M f^eq(rho_f, u_w, phi_b) + m_f - M f^eq(rho_f, u_f, phi_f),
// rho_b = rho_f (Wa.rho and Wa.rf already hold rho_f). On the stored deviations:
// with E(phi, u) = M f^eq(rho_f, u, phi) - m^rest(phi), whose parts are
// (phi drho, drho (2 kappa - 4 phi) + 3 phi rho |u|^2, drho (4 phi - 3 kappa) - 3 phi
// rho |u|^2, phi rho u_x, q phi rho u_x, phi rho u_y, q phi rho u_y, phi rho (u_x^2 -
// u_y^2), phi rho u_x u_y) with drho = rho_f - rho0 and q phi = kappa - 2 phi (Eq. 18)
// or -phi (B2), the wall's deviations are Fl.m + E(phi_b, u_w) - E(phi_f, u_f), in
// the storage's scaled units.
template <typename S, typename Ctx>
__device__ __forceinline__ void warp_nee_moments(const Ctx& c, PRow& Wa, const PRow& Fl, int pw) {
    const auto& p = c.p;
    const V2 pb = c.phi2(pw, Wa), pf = c.phi2(pw - 1, Fl);
    const V2 drs = Fl.rho;                                         // scale x (rho_f - rho0)
    const V2 sr = sizeof(S) == 4 ? Fl.rf : p.scale * Fl.rf;        // scale x rho_f
    const V2 bw = pb * sr, bf = pf * sr;                           // scale x phi rho_f
    const float wx = p.uw_x, wy = p.uw_y;
    const V2 fx = Fl.ux, fy = Fl.uy;
    const V2 ufu = fma2(fx, fx, fy * fy);
    const V2 uu3 = fma2(3.f * (wx * wx + wy * wy), bw, -(3.f * (bf * ufu)));   // 3 (phi_b rho uw^2 - phi_f rho uf^2)
    const V2 dp4 = 4.f * (drs * (pf - pb));                                   // 4 drho (phi_f - phi_b)
    const V2 jx = fma2(wx, bw, -(bf * fx)), jy = fma2(wy, bw, -(bf * fy));
    // q phi rho u: (kappa - 2 phi) rho u, or -phi rho u with (B2)
    V2 qx, qy;
    if constexpr (Ctx::kEq2) {
        qx = -jx;
        qy = -jy;
    } else {
        const V2 qb = fma2(-2.f, pb, bc(p.kappa)) * sr, qf = fma2(-2.f, pf, bc(p.kappa)) * sr;
        qx = fma2(wx, qb, -(qf * fx));
        qy = fma2(wy, qb, -(qf * fy));
    }
    Wa.m[0] = fma2(pb - pf, drs, Fl.m[0]);
    Wa.m[1] = Fl.m[1] + (dp4 + uu3);
    Wa.m[2] = Fl.m[2] - (dp4 + uu3);
    Wa.m[3] = Fl.m[3] + jx;
    Wa.m[4] = Fl.m[4] + qx;
    Wa.m[5] = Fl.m[5] + jy;
    Wa.m[6] = Fl.m[6] + qy;
    Wa.m[7] = Fl.m[7] + fma2(wx * wx - wy * wy, bw, -(bf * fma2(fx, fx, -(fy * fy))));
    Wa.m[8] = Fl.m[8] + fma2(wx * wy, bw, -(bf * (fx * fy)));
    // the full sum f of the wall node, as phase 1 keeps it
    if constexpr (sizeof(S) == 4) Wa.mf = fma2(p.rest.rho0, pb, Wa.m[0]);
    else Wa.mf = fma2(p.rest.rho0, pb, p.inv_scale * Wa.m[0]);
}

template <typename S, bool FAST, typename Ctx>
__device__ __forceinline__ void warp_phase3(const Ctx& c, const PRow& An, const PRow& Bs, const PRow& Cs,
                                            int p3, bool lane_ok) {
    using IO = PairIO<S>;
    const auto& p = c.p;
    constexpr float tw = 1.0f / 12.0f;
    V2 xAx = fma2(4.f, Cs.dAx, An.dAx + Bs.dAx);
    V2 xBx = fma2(4.f, Cs.dBx, An.dBx + Bs.dBx);
    V2 xBy = fma2(4.f, Cs.dBy, An.dBy + Bs.dBy);
    V2 xDx = fma2(4.f, Cs.dDx, An.dDx + Bs.dDx);
    V2 yAy = Bs.wAy - An.wAy;
    V2 yBy = Bs.wBy - An.wBy;
    V2 yBx = Bs.wBx - An.wBx;
    V2 yDy = Bs.wDy - An.wDy;
    // the rows around row p3: An holds row p3-1, Bs row p3+1. Past a half-way wall the
    // ghost row is the negated mirror row (no-slip); past the moving wall row (the
    // top row with nee_top) the linear extrapolation 2 (row ny-1) - (row ny-2)
    const bool nee_hi = !FAST && Ctx::kNee && p.nee_top && p3 == p.ny - 1;
    auto ghi = [&](V2 cs, V2 an, V2 bs) { return nee_hi ? fma2(2.f, cs, -an) : (p3 == p.ny - 1 ? -cs : bs); };
    if (!FAST && p.wall_y && (p3 == 0 || p3 == p.ny - 1)) {
        const bool lo = (p3 == 0);
        const V2 dAl = lo ? -Cs.dAx : An.dAx, dAh = ghi(Cs.dAx, An.dAx, Bs.dAx);
        const V2 dBxl = lo ? -Cs.dBx : An.dBx, dBxh = ghi(Cs.dBx, An.dBx, Bs.dBx);
        const V2 dByl = lo ? -Cs.dBy : An.dBy, dByh = ghi(Cs.dBy, An.dBy, Bs.dBy);
        const V2 dDl = lo ? -Cs.dDx : An.dDx, dDh = ghi(Cs.dDx, An.dDx, Bs.dDx);
        const V2 wAl = lo ? -Cs.wAy : An.wAy, wAh = ghi(Cs.wAy, An.wAy, Bs.wAy);
        const V2 wByl = lo ? -Cs.wBy : An.wBy, wByh = ghi(Cs.wBy, An.wBy, Bs.wBy);
        const V2 wBxl = lo ? -Cs.wBx : An.wBx, wBxh = ghi(Cs.wBx, An.wBx, Bs.wBx);
        const V2 wDl = lo ? -Cs.wDy : An.wDy, wDh = ghi(Cs.wDy, An.wDy, Bs.wDy);
        xAx = fma2(4.f, Cs.dAx, dAl + dAh);
        xBx = fma2(4.f, Cs.dBx, dBxl + dBxh);
        xBy = fma2(4.f, Cs.dBy, dByl + dByh);
        xDx = fma2(4.f, Cs.dDx, dDl + dDh);
        yAy = wAh - wAl;
        yBy = wByh - wByl;
        yBx = wBxh - wBxl;
        yDy = wDh - wDl;
    }
    // next to solid cells: 12 x the gradients of the six fields (rho u_x, rho u_y, u_x,
    // u_y, phi rho u_x, phi rho u_y) neighbour by neighbour, from the velocities of rows
    // p3-1 (An), p3 (Cs), p3+1 (Bs) and their rho, sum f kept by phase 2
    bool sna = false, snb = false;
    float sGy[2] = {0.f, 0.f}, sGx[2] = {0.f, 0.f};   // (B3): x-derivative of G_y, y-derivative of G_x
    if constexpr (Ctx::kSolid) {
        sna = solid_next(Cs.sm, 0);
        snb = solid_next(Cs.sm, 1);
        if (__any_sync(0xffffffffu, sna || snb)) {
            const bool lo_w = p.wall_y && p3 == 0, hi_w = p.wall_y && p3 == p.ny - 1;
            // the weights of both columns (vector components), once for the six fields
            float ka_x[3][3], ka_y[3][3], kb_x[3][3], kb_y[3][3];
            solid_weights(Cs.sm & 0x1FFu, -1.f, ka_x, ka_y);
            solid_weights((Cs.sm >> 9) & 0x1FFu, -1.f, kb_x, kb_y);
            // a rolled loop: this block runs only next to solid cells, and six unrolled
            // copies (three times over in the unrolled row loop) crowd the instruction
            // cache that the solid-free CTAs on the same SM share
#pragma unroll 1
            for (int k = 0; k < 6; ++k) {
                auto fld = [&](const PRow& R) {
                    const V2 u = (k & 1) ? R.uy : R.ux;
                    return k < 2 ? R.rfu * u : (k < 4 ? u : R.mfu * u);
                };
                const V2 l0 = fld(An), m = fld(Cs), h0 = fld(Bs);
                // past a half-way wall the negated mirror row (no-slip); past the
                // moving wall row 2 (row ny-1) - (row ny-2)
                const V2 l = lo_w ? -m : l0;
                const V2 h = hi_w ? (p.nee_top ? fma2(2.f, m, -l0) : -m) : h0;
                float w[3][4];
                win_row(w[0], l);
                win_row(w[1], m);
                win_row(w[2], h);
                float g[2][2];   // column, x / y
                g[0][0] = solid_apply<0>(w, ka_x);
                g[0][1] = solid_apply<0>(w, ka_y);
                g[1][0] = solid_apply<1>(w, kb_x);
                g[1][1] = solid_apply<1>(w, kb_y);
                auto put = [&](V2& d, int xy) {
                    if (sna) d.v.x = g[0][xy];
                    if (snb) d.v.y = g[1][xy];
                };
                switch (k) {
                    case 0: put(xAx, 0); break;
                    case 1: put(yAy, 1); break;
                    case 2: put(xBx, 0); put(yBx, 1); break;
                    case 3: put(yBy, 1); put(xBy, 0); break;
                    case 4: put(xDx, 0); break;
                    default: put(yDy, 1); break;
                }
                if constexpr (Ctx::kEq2) {
                    // G = D - kappa A
#pragma unroll
                    for (int cc = 0; cc < 2; ++cc) {
                        if (k == 0) sGx[cc] = -p.kappa * g[cc][1];
                        if (k == 1) sGy[cc] = -p.kappa * g[cc][0];
                        if (k == 4) sGx[cc] += g[cc][1];
                        if (k == 5) sGy[cc] += g[cc][0];
                    }
                }
            }
        }
    }
    const V2 phi = c.phi2(p3, Cs);
    const V2 phin = c.template phin2<FAST>(p3, Cs);
    const V2 rho = Cs.rf;
    const V2 X = p.kappa * Cs.iphi;
    const V2 kp = p.model_b ? bc(p.kappa - 1.f) : bc(p.kappa) - phi;
    const V2 kr = kp * rho;
    const V2 divD = xDx + yDy, difD = xDx - yDy;
    V2 Ca, Cb, Cc;
    if constexpr (Ctx::kEq2) {
        // Eq. (B3)
        V2 xGy = fma2(4.f, Cs.dGy, An.dGy + Bs.dGy);
        V2 yGx = Bs.wGx - An.wGx;
        if (!FAST && p.wall_y && (p3 == 0 || p3 == p.ny - 1)) {
            const bool lo = (p3 == 0);
            xGy = fma2(4.f, Cs.dGy, (lo ? -Cs.dGy : An.dGy) + ghi(Cs.dGy, An.dGy, Bs.dGy));
            yGx = ghi(Cs.wGx, An.wGx, Bs.wGx) - (lo ? -Cs.wGx : An.wGx);
        }
        if constexpr (Ctx::kSolid) {
            if (sna) { xGy.v.x = sGy[0]; yGx.v.x = sGx[0]; }
            if (snb) { xGy.v.y = sGy[1]; yGx.v.y = sGx[1]; }
        }
        Ca = tw * fma2(-2.f * p.kappa, xAx + yAy, fma2(2.f * kr, xBx + yBy, fma2(-2.f, X, bc(4.f)) * divD));
        Cb = (tw * (2.f / 3.f)) * fma2(-p.kappa, xAx - yAy, fma2(kr, xBx - yBy, difD));
        Cc = (1.f / 36.f) * fma2(kr, xBy + yBx, xGy + yGx);
    } else {
        // Eq. (20)
        Ca = fma2(tw, fma2(-p.kappa, xAx + yAy, fma2(2.f * kr, xBx + yBy, fma2(-2.f, X, bc(3.f)) * divD)), bc(0.f));
        Cb = tw * fma2(-p.kappa, xAx - yAy, fma2((2.f / 3.f) * kr, xBx - yBy, difD));
        Cc = (1.f / 36.f) * (kr * (xBy + yBx));
    }
    if (!FAST || Ctx::kUnsteady) Ca = fma2(-2.f, (X * rho) * (phin - phi), Ca);
    // Eq. (18), (19), (16) on the deviations from the rest state: the rest state's
    // moments (phi rho0, rho0 (2 kappa - 4 phi), rho0 (4 phi - 3 kappa), 0, ...) leave
    // m_0, e and eps; the equilibria of e and eps then differ from them by
    // dm0 (2X - 4) + 3 m0 |u|^2 and dm0 (4 - 3X) - 3 m0 |u|^2 (rho - rho0 = dm0 / phi)
    const V2 dm0 = Cs.m[0], ux = Cs.ux, uy = Cs.uy, Fx = Cs.Fx, Fy = Cs.Fy;
    const V2 m0 = Cs.mf;
    const V2 uu = fma2(ux, ux, uy * uy);
    const V2 uF = fma2(ux, Fx, uy * Fy);
    // equilibrium and source terms in the storage's scaled units
    const V2 m0s = sizeof(S) == 4 ? m0 : p.scale * m0;
    const V2 jxe = m0s * ux, jye = m0s * uy;
    const V2 q = Ctx::kEq2 ? bc(-1.f) : X - bc(2.f);   // Eq. (18) / (B2) energy-flux equilibria
    const V2 m0uu3 = m0s * (3.f * uu);
    V2 a[9];
    a[0] = dm0;
    const V2 me1 = fma2(dm0, fma2(2.f, X, bc(-4.f)), m0uu3);
    const V2 me2 = fma2(dm0, fma2(-3.f, X, bc(4.f)), -m0uu3);
    constexpr bool kUnit = sizeof(S) == 4;   // FP32: scale 1, the plain coefficients
    const float hs_e = kUnit ? p.h_e : p.hs_e, hs_eps = kUnit ? p.h_eps : p.hs_eps;
    const float hs_q = kUnit ? p.h_q : p.hs_q, hs_nu = kUnit ? p.h_nu : p.hs_nu;
    a[1] = fma2(hs_e, fma2(6.f, uF, Ca), fma2(p.s_e, me1 - Cs.m[1], Cs.m[1]));
    a[2] = fma2(-hs_eps * 6.f, uF, fma2(p.s_eps, me2 - Cs.m[2], Cs.m[2]));
    a[3] = sizeof(S) == 4 ? Cs.m[3] + Fx : fma2(p.scale, Fx, Cs.m[3]);
    a[4] = fma2(-hs_q, Fx, fma2(p.s_q, fma2(q, jxe, -Cs.m[4]), Cs.m[4]));
    a[5] = sizeof(S) == 4 ? Cs.m[5] + Fy : fma2(p.scale, Fy, Cs.m[5]);
    a[6] = fma2(-hs_q, Fy, fma2(p.s_q, fma2(q, jye, -Cs.m[6]), Cs.m[6]));
    const V2 me7 = m0s * fma2(ux, ux, -(uy * uy));
    const V2 S7 = 2.f * fma2(ux, Fx, -(uy * Fy));
    a[7] = fma2(hs_nu, S7 + Cb, fma2(p.s_nu, me7 - Cs.m[7], Cs.m[7]));
    const V2 S8 = fma2(ux, Fy, uy * Fx);
    a[8] = fma2(hs_nu, S8 + Cc, fma2(p.s_nu, fma2(jxe, uy, -Cs.m[8]), Cs.m[8]));
    // f+ = M^-1 m+ (A1). The 1/9, 1/36, 1/6 and 1/12 of M^-1 round in FP32, and
    // written directly they scale the cell's mass and momentum by the same rounding
    // factor every step. Instead f_0 and the diagonal-link x/y parts are taken as what
    // m_0 and j leave after the other populations: with s = bax + bdg formed first and
    // bdg = s - bax, f_0 = m_0 - 4 s and xd = (j_x - 2 xa) / 4 equal (A1)'s rows and
    // keep both sums exact up to rounding at the scale of the deviations.
    // f+ - f^rest = M^-1 (m+ - m^rest), all nine outputs deviations
    V2 fo[9];
    const V2 bax = (1.f / 36.f) * fma2(4.f, a[0], -fma2(2.f, a[2], a[1]));
    const V2 sbd = (1.f / 36.f) * fma2(8.f, a[0], a[1] - a[2]);
    const V2 bdg = sbd - bax;
    fo[0] = fma2(-4.f, sbd, a[0]);
    const V2 xa = (1.f / 6.f) * (a[3] - a[4]);
    const V2 ya = (1.f / 6.f) * (a[5] - a[6]);
    const V2 pq = 0.25f * a[7];
    const V2 xd = 0.25f * fma2(-2.f, xa, a[3]);
    const V2 yd = 0.25f * fma2(-2.f, ya, a[5]);
    const V2 pd = 0.25f * a[8];
    const V2 t13 = bax + pq, t24 = bax - pq;
    fo[1] = t13 + xa;
    fo[3] = t13 - xa;
    fo[2] = t24 + ya;
    fo[4] = t24 - ya;
    const V2 t57 = bdg + pd, t68 = bdg - pd;
    const V2 spp = xd + yd, smm = xd - yd;
    fo[5] = t57 + spp;
    fo[7] = t57 - spp;
    fo[6] = t68 - smm;
    fo[8] = t68 + smm;

    // f_0's rest value follows phi to t+1 (it is stored against phi(t+1))
    if (!FAST || Ctx::kUnsteady) fo[0] = fma2(sizeof(S) == 4 ? p.rest.rho0 : p.rho0s, phi - phin, fo[0]);
    // momentum base: this cell's post-collision momentum (m_3+, m_5+), rounded to the
    // storage type, is stored with the slots and each slot keeps its deviation from
    // 3 w_i e_i . J as well (these remainders carry no momentum)
    V2 Jq{}, Jqy{};
    if constexpr (Ctx::kJB) {
        Jq = IO::round_rn(a[3]);
        Jqy = IO::round_rn(a[5]);
        constexpr float t3 = 1.f / 3.f, t12 = 1.f / 12.f;
        const V2 sp = t12 * (Jq + Jqy), sm = t12 * (Jq - Jqy);
        fo[1] = fma2(-t3, Jq, fo[1]);
        fo[3] = fma2(t3, Jq, fo[3]);
        fo[2] = fma2(-t3, Jqy, fo[2]);
        fo[4] = fma2(t3, Jqy, fo[4]);
        fo[5] = fo[5] - sp;
        fo[7] = fo[7] + sp;
        fo[6] = fo[6] + sm;
        fo[8] = fo[8] - sm;
    }
    // one 2-wide store per population for every lane whose first column is inside
    // the lattice; the second column may then be the first ghost column, which the
    // ghost refresh after the step overwrites (the one-warp kernels leave all ghost
    // columns to ghost_fill_kernel, so the row loop holds no edge code)
    if (lane_ok) {
        if constexpr (Ctx::kSums) {
            // the second column of the pair may lie past nx (its store lands in the
            // first ghost column, overwritten by the ghost refresh): count it only when inside
            const V2 in = V2{make_float2(1.f, c.xa + 1 < p.nx ? 1.f : 0.f)};
            c.sums.add(0, m0 * in);
            const V2 ins = sizeof(S) == 4 ? in : p.inv_scale * in;
            c.sums.add(1, a[3] * ins);
            c.sums.add(2, a[5] * ins);
        }
        S* cell = reinterpret_cast<S*>(p.dst) + (long long)p3 * p.P + kPadCols + c.xa;
        if constexpr (sizeof(S) == 4) {
            IO::st(cell, fo[0]);
#pragma unroll
            for (int i = 1; i < 9; ++i) IO::st(cell + i * p.plane, fo[i]);
        } else {
            // FP16/BF16: stochastic rounding. Round-to-nearest loses every increment
            // below half a unit of the stored deviation (a slowly forced flow then
            // stalls); rounding up with probability equal to the discarded fraction
            // keeps each stored value unbiased. One hashed 32-bit word per column pair
            // (its column, row and step); population i takes it times an odd constant,
            // a bijection of 32-bit words, so every population's bits are uniform too.
            const uint32_t h0 = mix32(((uint32_t)c.xa * 0x9E3779B1u) ^ ((uint32_t)p3 * 0x85EBCA77u) ^
                                      ((c.step ^ c.salt) * 0xC2B2AE3Du));
#pragma unroll
            for (int i = 0; i < 9; ++i)
                IO::st_sr(cell + i * p.plane, fo[i], h0 * (0x2545F491u + 0x9E3779B8u * (uint32_t)i));
            if constexpr (Ctx::kJB) {
                IO::st(cell + 9 * p.plane, Jq);     // exact: already rounded
                IO::st(cell + 10 * p.plane, Jqy);
            }
        }
    }
}

// The row pipeline of one strip, shared by every one-warp kernel. Ctx supplies the
// staged rows (issue / wait_upto / pop), the per-cell sources (phi2, phin2,
// add_field_force, row_setup), the strip (y0, y1, source rows rlo .. rhi) and which
// rows may take the branch-free path (fast_strip, fast_lo, fast_hi).
//
// ONLY_FAST: every row takes the branch-free path, including the first four rows of
// the strip, whose phase-2/3 work on rows below y0 reads row states no phase 1 has
// filled; those results feed only phase 3 of rows below y0, which store nothing.
// Valid for strips whose staged rows y0-3 .. y1+2 hold no wall row and whose sources
// need no per-cell field handling (the caller checks).
template <typename S, bool ONLY_FAST, typename Ctx>
__device__ __forceinline__ bool warp_run_strip(Ctx& c) {
    const int lane = c.lane, y0 = c.y0, y1 = c.y1;
    PRow s0{}, s1{}, s2{};
    auto iter = [&](PRow& An, PRow& Bs, PRow& Cs, const int p1) {
        const int p2 = p1 - 1, p3 = p1 - 2;
        // the slot of row p1-3 is no longer read: refill it with row p1-3+kWarpSlots
        __syncwarp();
        if (p1 + kWarpSlots - 3 <= c.rhi && p1 + kWarpSlots - 3 >= c.rlo) {
            fence_proxy_async();
            c.issue(p1 + kWarpSlots - 3);
        }
        c.wait_upto(p1 + 1);
        const bool lane_ok = c.st_pair;
        if constexpr (ONLY_FAST) {
            warp_phase1<S, true>(c, An, p1);
            const float l = left_of(An.rho), r = right_of(An.rho);
            An.dr = rpair(An.rho, r) - lpair(An.rho, l);
            An.wr = fma2(4.f, An.rho, rpair(An.rho, r) + lpair(An.rho, l));
            warp_phase2<S, true>(c, An, Bs, Cs, p2);
            warp_phase3<S, true>(c, An, Bs, Cs, p3, lane_ok && p3 >= y0);
            return;
        }
        if constexpr (!Ctx::kSolid) {
            if (c.fast_strip && p3 >= c.fast_lo && p1 <= c.fast_hi) {
                // interior row: one branch-free block, so the collision of row p3 overlaps
                // the pulls and shuffles of rows p1, p2
                warp_phase1<S, true>(c, An, p1);
                const float l = left_of(An.rho), r = right_of(An.rho);
                An.dr = rpair(An.rho, r) - lpair(An.rho, l);
                An.wr = fma2(4.f, An.rho, rpair(An.rho, r) + lpair(An.rho, l));
                warp_phase2<S, true>(c, An, Bs, Cs, p2);
                warp_phase3<S, true>(c, An, Bs, Cs, p3, lane_ok);
                return;
            }
        }
        const bool ph1 = (p1 <= y1 + 1) && c.row_valid(p1);
        // the moving wall row (its moments follow once row ny-2 has its velocity)
        const bool nee_row = Ctx::kNee && c.p.nee_top && p1 == c.p.ny - 1;
        if (ph1) {
            warp_phase1<S, false>(c, An, p1);
            if (nee_row) { An.rho = Bs.rho; An.rf = Bs.rf; }   // rho_b = rho_f
            const float l = left_of(An.rho), r = right_of(An.rho);
            An.dr = rpair(An.rho, r) - lpair(An.rho, l);
            An.wr = fma2(4.f, An.rho, rpair(An.rho, r) + lpair(An.rho, l));
        }
        const bool ph2 = (p2 >= y0 - 1) && (p2 <= y1) && c.row_valid(p2);
        if (ph2) warp_phase2<S, false>(c, An, Bs, Cs, p2);
        if (ph1 && nee_row) warp_nee_moments<S>(c, An, Bs, p1);
        const bool ph3 = (p3 >= y0) && (p3 < y1);
        if (ph3) warp_phase3<S, false>(c, An, Bs, Cs, p3, lane_ok);
    };

    const int n_it = (y1 + 1) - (y0 - 2) + 1;
    // The rows the first iteration needs (y0-3 .. y0-1) are waited for here, with a vote:
    // inside the loop each iteration then waits for one new row r (iteration r-1), whose
    // slot is refilled at iteration r+3, after the vote that ends the group of three rows
    // holding iteration r-1. So a slot whose wait gave up is never armed again.
    c.wait_upto(y0 - 1);
    bool ok = !__any_sync(0xffffffffu, c.aborted);
    for (int it = 0; it < n_it && ok; it += 3) {
        const int p1 = y0 - 2 + it;
        iter(s0, s2, s1, p1);
        if (it + 1 < n_it) iter(s1, s0, s2, p1 + 1);
        if (it + 2 < n_it) iter(s2, s1, s0, p1 + 2);
        // a timed-out wait (bounded, flagged by wait_upto) ends the strip after
        // this group of three rows
        ok = !__any_sync(0xffffffffu, c.aborted);
    }
    __syncwarp();
    return ok;
}

// One CTA of the one-warp step kernel (the kernel below picks the instance).
template <typename S, bool SUMS, bool EQ2, bool SOLID, bool JB, bool NEE>
__device__ __forceinline__ void warp_step_cta(const StepParams<float>& p, unsigned char* smem, int bx, int by) {
    using L = WarpLayout<S, JB ? 11 : 9>;
    const int lane = threadIdx.x;
    constexpr int A = L::A;
    const int x0 = bx * p.W;
    const int y0 = by * p.H;
    const int y1 = min(y0 + p.H, p.ny);

    WarpCtx<S, SUMS, EQ2, SOLID, JB, NEE> c{p, smem, lane, 0, 0, y0, y1, 0, 0, 0, 0, 0, 0, false};
    if constexpr (sizeof(S) == 2) c.step = p.step_ctr ? *p.step_ctr : 0u;
    c.wsp = ((kPadCols + x0 - kGhost) / A) * A;
    c.ww = ((kPadCols + x0 + 63 + A - 1) / A) * A - c.wsp;
    c.xa = x0 - 2 + 2 * lane;
    c.sa = kPadCols + c.xa - c.wsp;
    c.st_pair = lane >= 1 && lane < 31 && c.xa < p.nx;
    c.rlo = y0 - 3;
    c.rhi = y1 + 2;
    if (p.wall_y) { c.rlo = max(c.rlo, 0); c.rhi = min(c.rhi, p.ny - 1); }
    c.waited = c.rlo - 1;
    c.issued = c.rlo - 1;
    // rows whose three phases need no wall, validity or field handling
    // (the EQ2 instance's fast path evaluates B3; the SOLID instance has none)
    c.fast_strip = !SOLID && !p.unsteady && !p.has_fb && !p.has_drag;
    c.fast_lo = p.wall_y ? max(y0, 1) : y0;                 // lowest phase-3 row
    c.fast_hi = p.wall_y ? min(y1 + 1, p.ny - 2) : y1 + 1;  // highest phase-1 row

    c.setup_copies();
    if (lane == 0) {
        for (int k = 0; k < kWarpSlots; ++k) mbar_init(reinterpret_cast<uint64_t*>(smem) + k, 1);
        fence_mbar_init();
    }
    __syncwarp();
    for (int r = c.rlo; r <= min(y0 + kWarpSlots - 6, c.rhi); ++r) c.issue(r);
    __syncwarp();
    // strips that stage no wall row run the loop that holds only the branch-free path
    if constexpr (SOLID) {
        warp_run_strip<S, false>(c);
    } else {
        if (c.fast_strip && (!p.wall_y || (y0 >= 3 && y1 <= p.ny - 3))) warp_run_strip<S, true>(c);
        else warp_run_strip<S, false>(c);
    }
    if (lane == 0) {
        // every copy that may still be in flight is waited for before the CTA exits
        // (the rows whose wait gave up and those not waited for yet; see kWaitTries)
        for (int r = min(c.first_bad, c.waited + 1); r <= c.issued; ++r)
            mbar_wait_bounded(c.bar(r), c.parity(r), kWaitTries);
    }
    if constexpr (SUMS) {
        for (int k = 0; k < 3; ++k) {
            double v = c.sums.value(k);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) atomicAdd(p.sums + k, v);
        }
    }
}

template <typename S, int MINB, bool SUMS = false, bool EQ2 = false, bool SOLID = false, bool JB = false,
          bool NEE = false>
__global__ void __launch_bounds__(32, MINB) vanse_warp_kernel(const __grid_constant__ StepParams<float> p) {
    extern __shared__ __align__(128) unsigned char smem[];
    if constexpr (SOLID) {
        // the tiles with solid cells run first (tile_order); a CTA whose staged rows and
        // columns hold no solid cell runs the solid-free path (with its branch-free
        // interior rows)
        int t = blockIdx.y * gridDim.x + blockIdx.x;
        if (p.solid_tiles && p.tile_order) t = p.tile_order[t];
        const int bx = t % gridDim.x, by = t / gridDim.x;
        if (p.solid_tiles && !p.solid_tiles[t])
            warp_step_cta<S, SUMS, EQ2, false, JB, true>(p, smem, bx, by);
        else
            warp_step_cta<S, SUMS, EQ2, true, JB, true>(p, smem, bx, by);
    } else {
        warp_step_cta<S, SUMS, EQ2, false, JB, NEE>(p, smem, blockIdx.x, blockIdx.y);
    }
}

}  // namespace lbmv

namespace lbmv {

// The one-warp kernel's instances with solid cells (the SOLID template argument),
// compiled in vanse_warp_solid.cu. configure sets their shared-memory attributes;
// launch starts the step-sum (sums) or plain instance, with App. B (eq2) or Eq. (18).
template <typename S>
cudaError_t warp_solid_configure(size_t smem_max);
template <typename S>
cudaError_t warp_solid_launch(const StepParams<float>& p, dim3 grid, size_t smem, cudaStream_t stream, bool sums,
                              bool eq2);

// The FP16 / BF16 instances with the momentum base (the JB template argument),
// compiled in vanse_warp_jb.cu; kernel returns the plain (sums = eq2 = false) instance
// for occupancy queries.
template <typename S>
cudaError_t warp_jb_configure(size_t smem_max);
template <typename S>
cudaError_t warp_jb_launch(const StepParams<float>& p, dim3 grid, size_t smem, cudaStream_t stream, bool sums,
                           bool eq2);
template <typename S>
const void* warp_jb_kernel();

// The instances with the moving wall's code (the NEE template argument), compiled in
// vanse_warp_nee.cu.
template <typename S>
cudaError_t warp_nee_configure(size_t smem_max);
template <typename S>
cudaError_t warp_nee_launch(const StepParams<float>& p, dim3 grid, size_t smem, cudaStream_t stream, bool sums,
                            bool eq2);

}  // namespace lbmv
