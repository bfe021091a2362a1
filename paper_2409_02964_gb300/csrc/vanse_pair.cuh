// vanse_pair.cuh -- the fused D2Q9 MRTLB-VANSE stream + collide kernel, two
// adjacent columns per thread with packed FP32 arithmetic (FFMA2 / FADD2 / FMUL2).
//
// Same method, same row-marching decomposition and the same three phases as
// vanse_step.cuh (see there for the derivation); differences:
//   * thread t owns columns xa = x0 - 2 + 2t and xb = xa + 1; a CTA of T threads
//     covers 2T columns and stores W = 2T - 4 of them;
//   * every per-cell quantity is a pair (V2) and the arithmetic runs on the packed
//     two-lane FP32 instructions, so one instruction updates both columns;
//   * per-row bookkeeping (waits, barriers, slot addressing, phase predicates) is
//     paid once per two cells, the x-neighbour exchange needs two scalar shared
//     loads per field per two cells, and the stores are 2-wide;
//   * a 6-slot ring (4 rows in use + 2 rows of prefetch) keeps the shared-memory
//     footprint at ~36 KB for 128 columns.
// Reduced-precision storage (FP16 / BF16) decodes pairs with one conversion.
#pragma once

#include "vanse_common.cuh"
#include "vanse_step.cuh"

namespace lbmv {

// ------------------------------------------------------------------ pair type
struct V2 {
    float2 v;
};
__device__ __forceinline__ V2 mk(float a, float b) { return V2{make_float2(a, b)}; }
__device__ __forceinline__ V2 bc(float s) { return V2{make_float2(s, s)}; }
__device__ __forceinline__ V2 operator+(V2 a, V2 b) { return V2{__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ V2 operator-(V2 a, V2 b) { return V2{__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)}; }
__device__ __forceinline__ V2 operator*(V2 a, V2 b) { return V2{__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ V2 operator*(float s, V2 b) { return V2{__fmul2_rn(make_float2(s, s), b.v)}; }
__device__ __forceinline__ V2 operator-(V2 a) { return V2{__fmul2_rn(make_float2(-1.f, -1.f), a.v)}; }
__device__ __forceinline__ V2 fma2(V2 a, V2 b, V2 c) { return V2{__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ V2 fma2(float s, V2 b, V2 c) { return V2{__ffma2_rn(make_float2(s, s), b.v, c.v)}; }
// 1/a by the approximate reciprocal instruction (rcp.approx, relative error below
// 2^-23; the operands here are densities and void fractions of order one)
__device__ __forceinline__ float rcp_approx(float a) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ V2 rcp2(V2 a) { return mk(rcp_approx(a.v.x), rcp_approx(a.v.y)); }
__device__ __forceinline__ V2 operator+(V2 a, float s) { return V2{__fadd2_rn(a.v, make_float2(s, s))}; }
__device__ __forceinline__ V2 operator+(float s, V2 a) { return a + s; }
__device__ __forceinline__ V2 operator*(V2 a, float s) { return s * a; }
__device__ __forceinline__ V2 mms_rcp(V2 a) { return rcp2(a); }
__device__ __forceinline__ float mms_rcp(float a) { return 1.0f / a; }

// storage loads of a pair at an even (aligned) element index, or a pair shifted by one
template <typename S> struct PairIO;
template <> struct PairIO<float> {
    __device__ static V2 al(const float* p) { return V2{*reinterpret_cast<const float2*>(p)}; }
    __device__ static V2 un(const float* p) { return mk(p[0], p[1]); }
    __device__ static V2 dec(V2 d, V2 rest, float) { return d + rest; }
    __device__ static V2 dev(V2 d, float) { return d; }
    __device__ static void st(float* p, V2 v) { *reinterpret_cast<float2*>(p) = v.v; }
    __device__ static float enc1(float f, float rest, float) { return f - rest; }
    __device__ static V2 round_rn(V2 v) { return v; }
};
template <> struct PairIO<__half> {
    __device__ static V2 al(const __half* p) { return V2{__half22float2(*reinterpret_cast<const __half2*>(p))}; }
    __device__ static V2 un(const __half* p) { return V2{__half22float2(__halves2half2(p[0], p[1]))}; }
    __device__ static V2 dec(V2 d, V2 rest, float ia) { return fma2(ia, d, rest); }
    __device__ static V2 dev(V2 d, float) { return d; }   // the storage's scaled units
    __device__ static void st(__half* p, V2 v) { *reinterpret_cast<__half2*>(p) = __float22half2_rn(v.v); }
    // stochastic rounding (the conversion's .rs mode) with 32 random bits r
    __device__ static void st_sr(__half* p, V2 v, uint32_t r) {
        uint32_t d;
        asm("cvt.rs.satfinite.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(v.v.y), "f"(v.v.x), "r"(r));
        *reinterpret_cast<uint32_t*>(p) = d;
    }
    __device__ static __half enc1(float f, float rest, float s) { return __float2half_rn((f - rest) * s); }
    // a pair rounded to the storage type (to nearest) and back: stored as it is, exactly
    __device__ static V2 round_rn(V2 v) { return V2{__half22float2(__float22half2_rn(v.v))}; }
};
template <> struct PairIO<__nv_bfloat16> {
    __device__ static V2 al(const __nv_bfloat16* p) {
        return V2{__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p))};
    }
    __device__ static V2 un(const __nv_bfloat16* p) { return V2{__bfloat1622float2(__halves2bfloat162(p[0], p[1]))}; }
    __device__ static V2 dec(V2 d, V2 rest, float ia) { return fma2(ia, d, rest); }
    __device__ static V2 dev(V2 d, float) { return d; }   // the storage's scaled units
    __device__ static void st(__nv_bfloat16* p, V2 v) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __float22bfloat162_rn(v.v);
    }
    __device__ static void st_sr(__nv_bfloat16* p, V2 v, uint32_t r) {
        uint32_t d;
        asm("cvt.rs.satfinite.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(v.v.y), "f"(v.v.x), "r"(r));
        *reinterpret_cast<uint32_t*>(p) = d;
    }
    __device__ static __nv_bfloat16 enc1(float f, float rest, float s) { return __float2bfloat16_rn((f - rest) * s); }
    __device__ static V2 round_rn(V2 v) { return V2{__bfloat1622float2(__float22bfloat162_rn(v.v))}; }
};

constexpr int kPairSlots = 6;   // ring slots: rows p-2 .. p+1 in use, two rows of prefetch

template <typename S, int T>
struct PairLayout {
    static constexpr int A = 16 / (int)sizeof(S);
    static constexpr int WW = 2 * T + 2 * A;                   // staged row width (elements)
    static constexpr int XB = 2 * T + 4;                        // exchange row: 2 pad + 2T + 2 pad
    static constexpr int kRho = 128;
    static constexpr int kFld = kRho + XB * 4;
    static constexpr int kPop = (kFld + 6 * XB * 4 + 127) & ~127;
    static constexpr int kPopRow = WW * (int)sizeof(S);
    static constexpr int kPopSlot = 9 * kPopRow;
    static constexpr int kAux = kPop + kPairSlots * kPopSlot;
    static constexpr int kAuxRow = WW * 4;
    static constexpr size_t bytes(int nR) { return (size_t)kAux + (size_t)kPairSlots * nR * kAuxRow; }
};

struct PRow {
    float sy, cy;   // sin, cos of k y of this row (analytic sources only)
    V2 m[9];
    V2 rho;
    V2 iphi, mf, rf;   // one-warp kernel: 1/phi, the full sum f and the full rho, kept from phase 1
    V2 dr, wr;
    V2 Fx, Fy, ux, uy;
    V2 dAx, dBx, dBy, dDx;
    V2 wAy, wBy, wBx, wDy;
    V2 dGy, wGx;       // one-warp kernel with App. B: G = phi rho u - kappa rho u (the (B3) cross terms)
    // one-warp kernel with solid cells: rho and the full sum f of the row whose velocity
    // ux, uy hold (phase 1 of a later row overwrites rf, mf first), and the pair's
    // solid-neighbour mask (bit 9 c + 3 (dy + 1) + dx + 1 for column c of the pair,
    // the rows past a wall mapped as the stencil maps them; bit 9 c + 4: the cell itself)
    V2 rfu, mfu;
    uint32_t sm;
};

__device__ __forceinline__ int pslot(int r) { return ((r % kPairSlots) + kPairSlots) % kPairSlots; }

template <typename S, int T>
struct PairCtx {
    using L = PairLayout<S, T>;
    const StepParams<float>& p;
    unsigned char* smem;
    int* abort_flag;
    int t, xa, sa;      // thread, first global column, its smem column (even)
    int y0, y1;
    int wsp, ww;
    int rlo, rhi;
    int waited, issued;
    int first_bad = 0x7fffffff;   // first row whose wait gave up (this thread)

    __device__ __forceinline__ uint64_t* bar(int r) const { return reinterpret_cast<uint64_t*>(smem) + pslot(r); }
    __device__ __forceinline__ const S* pop(int r) const {
        return reinterpret_cast<const S*>(smem + L::kPop + pslot(r) * L::kPopSlot) + sa;
    }
    __device__ __forceinline__ const float* aux(int r, int k) const {
        return reinterpret_cast<const float*>(smem + L::kAux) + (pslot(r) * p.nR + k) * L::WW + sa;
    }
    __device__ __forceinline__ bool row_valid(int r) const { return !p.wall_y || (r >= 0 && r < p.ny); }
    __device__ __forceinline__ uint32_t parity(int r) const { return (uint32_t)(((r - rlo) / kPairSlots) & 1); }

    __device__ __forceinline__ void issue(int r) {
        issued = r;
        uint64_t* b = bar(r);
        int gr = r;
        if (!p.wall_y) { gr %= p.ny; if (gr < 0) gr += p.ny; }
        const uint32_t bs = (uint32_t)(ww * (int)sizeof(S));
        const uint32_t br = (uint32_t)(ww * 4);
        mbar_expect_tx(b, 9u * bs + (uint32_t)p.nR * br);
        const long long off = (long long)gr * p.P + wsp;
        const S* src = reinterpret_cast<const S*>(p.src) + off;
        unsigned char* ps = smem + L::kPop + pslot(r) * L::kPopSlot;
#pragma unroll
        for (int i = 0; i < 9; ++i) bulk_g2s(ps + i * L::kPopRow, src + i * p.plane, bs, b);
        float* rr = reinterpret_cast<float*>(smem + L::kAux) + pslot(r) * p.nR * L::WW;
        int k = 0;
        bulk_g2s(rr + (k++) * L::WW, p.phi + off, br, b);
        if (p.unsteady) bulk_g2s(rr + (k++) * L::WW, p.phin + off, br, b);
        if (p.has_fb) {
            bulk_g2s(rr + (k++) * L::WW, p.fb + off, br, b);
            bulk_g2s(rr + (k++) * L::WW, p.fb + p.plane + off, br, b);
        }
    }
    __device__ __forceinline__ void wait_upto(int r) {
        r = min(r, rhi);
        while (waited < r) {
            ++waited;
            if (!mbar_wait_bounded(bar(waited), parity(waited), p.wait_tries)) {
                first_bad = min(first_bad, waited);
                *abort_flag = 1;
                atomicExch(p.err, 1);
            }
        }
    }
};

template <typename S, int T>
__device__ __forceinline__ void pair_phase1(const PairCtx<S, T>& c, PRow& st, int r) {
    using IO = PairIO<S>;
    constexpr int RW = PairLayout<S, T>::WW;
    const StepParams<float>& p = c.p;
    const V2 phi = V2{*reinterpret_cast<const float2*>(c.aux(r, 0))};
    const float ia = p.inv_scale;
    const V2 rax = bc(p.rest.ax), rdg = bc(p.rest.dg);
    const V2 r0 = fma2(p.rest.rho0, phi, bc(-p.rest.k59));
    const S* cur = c.pop(r);
    V2 f0, f1, f2, f3, f4, f5, f6, f7, f8;
    f0 = IO::dec(IO::al(cur), r0, ia);
    f1 = IO::dec(IO::un(cur + 1 * RW - 1), rax, ia);
    f3 = IO::dec(IO::un(cur + 3 * RW + 1), rax, ia);
    if (p.wall_y && r == 0) {
        f2 = IO::dec(IO::al(cur + 4 * RW), rax, ia);
        f5 = IO::dec(IO::al(cur + 7 * RW), rdg, ia);
        f6 = IO::dec(IO::al(cur + 8 * RW), rdg, ia);
    } else {
        const S* lo = c.pop(r - 1);
        f2 = IO::dec(IO::al(lo + 2 * RW), rax, ia);
        f5 = IO::dec(IO::un(lo + 5 * RW - 1), rdg, ia);
        f6 = IO::dec(IO::un(lo + 6 * RW + 1), rdg, ia);
    }
    if (p.wall_y && r == p.ny - 1) {
        f4 = IO::dec(IO::al(cur + 2 * RW), rax, ia);
        f7 = IO::dec(IO::al(cur + 5 * RW), rdg, ia);
        f8 = IO::dec(IO::al(cur + 6 * RW), rdg, ia);
    } else {
        const S* hi = c.pop(r + 1);
        f4 = IO::dec(IO::al(hi + 4 * RW), rax, ia);
        f7 = IO::dec(IO::un(hi + 7 * RW + 1), rdg, ia);
        f8 = IO::dec(IO::un(hi + 8 * RW - 1), rdg, ia);
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
    st.rho = st.m[0] * rcp2(phi);
}

// (left, own.x) and (own.y, right) pairs of a field around the thread's two columns
__device__ __forceinline__ V2 lpair(V2 own, float left) { return mk(left, own.v.x); }
__device__ __forceinline__ V2 rpair(V2 own, float right) { return mk(own.v.y, right); }

template <typename S, int T>
__device__ __forceinline__ void pair_phase2(const PairCtx<S, T>& c, const PRow& An, PRow& Bs, const PRow& Cs, int p2,
                                            float* fbuf) {
    using L = PairLayout<S, T>;
    const StepParams<float>& p = c.p;
    constexpr float tw = 1.0f / 12.0f;
    V2 dlo = Cs.dr, wlo = Cs.wr, dhi = An.dr, whi = An.wr;
    if (p.wall_y && (p2 == 0 || p2 == p.ny - 1)) {
        if (p2 == 0) { dlo = Bs.dr; wlo = Bs.wr; }
        if (p2 == p.ny - 1) { dhi = Bs.dr; whi = Bs.wr; }
    }
    const V2 gx = tw * fma2(4.f, Bs.dr, dlo + dhi);
    const V2 gy = tw * (whi - wlo);
    const V2 phi = V2{*reinterpret_cast<const float2*>(c.aux(p2, 0))};
    const V2 kp = p.model_b ? bc((p.kappa - 1.f) * (1.f / 3.f)) : (1.f / 3.f) * (bc(p.kappa) - phi);
    V2 Fx = fma2(kp, gx, p.gx * phi);
    V2 Fy = fma2(kp, gy, p.gy * phi);
    if (p.has_fb) {
        const int k = p.unsteady ? 2 : 1;
        Fx = Fx + V2{*reinterpret_cast<const float2*>(c.aux(p2, k))};
        Fy = Fy + V2{*reinterpret_cast<const float2*>(c.aux(p2, k + 1))};
    }
    const V2 m0 = Bs.m[0];
    const V2 inv = rcp2(m0);
    const V2 ux = fma2(0.5f, Fx, Bs.m[3]) * inv;
    const V2 uy = fma2(0.5f, Fy, Bs.m[5]) * inv;
    Bs.Fx = Fx; Bs.Fy = Fy; Bs.ux = ux; Bs.uy = uy;
    float2* F = reinterpret_cast<float2*>(fbuf + 2 + 2 * c.t);
    F[0 * L::XB / 2] = (Bs.rho * ux).v;
    F[1 * L::XB / 2] = (Bs.rho * uy).v;
    F[2 * L::XB / 2] = ux.v;
    F[3 * L::XB / 2] = uy.v;
    F[4 * L::XB / 2] = (m0 * ux).v;
    F[5 * L::XB / 2] = (m0 * uy).v;
}

template <typename S, int T>
__device__ __forceinline__ void pair_fields(const PairCtx<S, T>& c, PRow& Bs, const float* fbuf) {
    using L = PairLayout<S, T>;
    const float* F = fbuf + 2 + 2 * c.t;
    // left neighbour of xa is F[-1], right neighbour of xb is F[2] (per field row)
    const V2 Ax = Bs.rho * Bs.ux, Ay = Bs.rho * Bs.uy;
    const V2 Dx = Bs.m[0] * Bs.ux, Dy = Bs.m[0] * Bs.uy;
    const float Axl = F[0 * L::XB - 1], Axr = F[0 * L::XB + 2];
    const float Ayl = F[1 * L::XB - 1], Ayr = F[1 * L::XB + 2];
    const float Bxl = F[2 * L::XB - 1], Bxr = F[2 * L::XB + 2];
    const float Byl = F[3 * L::XB - 1], Byr = F[3 * L::XB + 2];
    const float Dxl = F[4 * L::XB - 1], Dxr = F[4 * L::XB + 2];
    const float Dyl = F[5 * L::XB - 1], Dyr = F[5 * L::XB + 2];
    Bs.dAx = rpair(Ax, Axr) - lpair(Ax, Axl);
    Bs.dBx = rpair(Bs.ux, Bxr) - lpair(Bs.ux, Bxl);
    Bs.dBy = rpair(Bs.uy, Byr) - lpair(Bs.uy, Byl);
    Bs.dDx = rpair(Dx, Dxr) - lpair(Dx, Dxl);
    Bs.wAy = fma2(4.f, Ay, rpair(Ay, Ayr) + lpair(Ay, Ayl));
    Bs.wBy = fma2(4.f, Bs.uy, rpair(Bs.uy, Byr) + lpair(Bs.uy, Byl));
    Bs.wBx = fma2(4.f, Bs.ux, rpair(Bs.ux, Bxr) + lpair(Bs.ux, Bxl));
    Bs.wDy = fma2(4.f, Dy, rpair(Dy, Dyr) + lpair(Dy, Dyl));
}

template <typename S, int T>
__device__ __forceinline__ void pair_phase3(const PairCtx<S, T>& c, const PRow& An, const PRow& Bs, const PRow& Cs,
                                            int p3) {
    using IO = PairIO<S>;
    const StepParams<float>& p = c.p;
    constexpr float tw = 1.0f / 12.0f;
    V2 xAx = fma2(4.f, Cs.dAx, An.dAx + Bs.dAx);
    V2 xBx = fma2(4.f, Cs.dBx, An.dBx + Bs.dBx);
    V2 xBy = fma2(4.f, Cs.dBy, An.dBy + Bs.dBy);
    V2 xDx = fma2(4.f, Cs.dDx, An.dDx + Bs.dDx);
    V2 yAy = Bs.wAy - An.wAy;
    V2 yBy = Bs.wBy - An.wBy;
    V2 yBx = Bs.wBx - An.wBx;
    V2 yDy = Bs.wDy - An.wDy;
    if (p.wall_y && (p3 == 0 || p3 == p.ny - 1)) {
        const bool lo = (p3 == 0), hi = (p3 == p.ny - 1);
        const V2 dAl = lo ? -Cs.dAx : An.dAx, dAh = hi ? -Cs.dAx : Bs.dAx;
        const V2 dBxl = lo ? -Cs.dBx : An.dBx, dBxh = hi ? -Cs.dBx : Bs.dBx;
        const V2 dByl = lo ? -Cs.dBy : An.dBy, dByh = hi ? -Cs.dBy : Bs.dBy;
        const V2 dDl = lo ? -Cs.dDx : An.dDx, dDh = hi ? -Cs.dDx : Bs.dDx;
        const V2 wAl = lo ? -Cs.wAy : An.wAy, wAh = hi ? -Cs.wAy : Bs.wAy;
        const V2 wByl = lo ? -Cs.wBy : An.wBy, wByh = hi ? -Cs.wBy : Bs.wBy;
        const V2 wBxl = lo ? -Cs.wBx : An.wBx, wBxh = hi ? -Cs.wBx : Bs.wBx;
        const V2 wDl = lo ? -Cs.wDy : An.wDy, wDh = hi ? -Cs.wDy : Bs.wDy;
        xAx = fma2(4.f, Cs.dAx, dAl + dAh);
        xBx = fma2(4.f, Cs.dBx, dBxl + dBxh);
        xBy = fma2(4.f, Cs.dBy, dByl + dByh);
        xDx = fma2(4.f, Cs.dDx, dDl + dDh);
        yAy = wAh - wAl;
        yBy = wByh - wByl;
        yBx = wBxh - wBxl;
        yDy = wDh - wDl;
    }
    const V2 phi = V2{*reinterpret_cast<const float2*>(c.aux(p3, 0))};
    const V2 phin = p.unsteady ? V2{*reinterpret_cast<const float2*>(c.aux(p3, 1))} : phi;
    const V2 rho = Cs.rho;
    const V2 X = p.kappa * rcp2(phi);
    const V2 kp = p.model_b ? bc(p.kappa - 1.f) : bc(p.kappa) - phi;
    const V2 kr = kp * rho;
    // Eq. (20)
    const V2 divD = xDx + yDy, difD = xDx - yDy;
    const V2 Ca = fma2(tw, fma2(-p.kappa, xAx + yAy, fma2(2.f * kr, xBx + yBy, fma2(-2.f, X, bc(3.f)) * divD)),
                       (-2.f) * (X * rho) * (phin - phi));
    const V2 Cb = tw * fma2(-p.kappa, xAx - yAy, fma2((2.f / 3.f) * kr, xBx - yBy, difD));
    const V2 Cc = (1.f / 36.f) * (kr * (xBy + yBx));
    // Eq. (18), (19), (16)
    const V2 m0 = Cs.m[0], ux = Cs.ux, uy = Cs.uy, Fx = Cs.Fx, Fy = Cs.Fy;
    const V2 uu = fma2(ux, ux, uy * uy);
    const V2 uF = fma2(ux, Fx, uy * Fy);
    const V2 jxe = m0 * ux, jye = m0 * uy;
    const V2 q = X - bc(2.f);
    V2 a[9];
    a[0] = m0;
    // m + s (m_eq - m) + h (S + C)
    const V2 me1 = m0 * fma2(3.f, uu, fma2(2.f, X, bc(-4.f)));
    const V2 me2 = m0 * fma2(-3.f, uu, fma2(-3.f, X, bc(4.f)));
    a[1] = fma2(p.h_e, fma2(6.f, uF, Ca), fma2(p.s_e, me1 - Cs.m[1], Cs.m[1]));
    a[2] = fma2(-p.h_eps * 6.f, uF, fma2(p.s_eps, me2 - Cs.m[2], Cs.m[2]));
    a[3] = Cs.m[3] + Fx;
    a[4] = fma2(-p.h_q, Fx, fma2(p.s_q, fma2(q, jxe, -Cs.m[4]), Cs.m[4]));
    a[5] = Cs.m[5] + Fy;
    a[6] = fma2(-p.h_q, Fy, fma2(p.s_q, fma2(q, jye, -Cs.m[6]), Cs.m[6]));
    const V2 me7 = m0 * fma2(ux, ux, -(uy * uy));
    const V2 S7 = 2.f * fma2(ux, Fx, -(uy * Fy));
    a[7] = fma2(p.h_nu, S7 + Cb, fma2(p.s_nu, me7 - Cs.m[7], Cs.m[7]));
    const V2 S8 = fma2(ux, Fy, uy * Fx);
    a[8] = fma2(p.h_nu, S8 + Cc, fma2(p.s_nu, fma2(jxe, uy, -Cs.m[8]), Cs.m[8]));
    // f+ = M^-1 m+ (A1); f_0 and the diagonal-link x/y parts as what m_0 and j leave
    // after the other populations, so the rounded fractions of M^-1 do not scale the
    // cell's mass and momentum by a fixed factor every step
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

    // encode and store
    const V2 r0 = fma2(p.rest.rho0, phin, bc(-p.rest.k59));
    S* row = reinterpret_cast<S*>(p.dst) + (long long)p3 * p.P + kPadCols;
    const int xa0 = c.xa;
    const bool va = xa0 < p.nx, vb = xa0 + 1 < p.nx;
    if (va && vb) {
        S* cell = row + xa0;
        IO::st(cell, sizeof(S) == 4 ? fo[0] - r0 : p.scale * (fo[0] - r0));
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const V2 ri = bc(i <= 4 ? p.rest.ax : p.rest.dg);
            IO::st(cell + i * p.plane, sizeof(S) == 4 ? fo[i] - ri : p.scale * (fo[i] - ri));
        }
    } else if (va) {
        S* cell = row + xa0;
        cell[0] = IO::enc1(fo[0].v.x, r0.v.x, p.scale);
#pragma unroll
        for (int i = 1; i < 9; ++i) cell[i * p.plane] = IO::enc1(fo[i].v.x, i <= 4 ? p.rest.ax : p.rest.dg, p.scale);
    }
    // periodic ghost images of columns near the x edges
    for (int k = 0; k < 2; ++k) {
        const int x = xa0 + k;
        if (x >= p.nx || !(x < kGhost || x >= p.nx - kGhost)) continue;
        int g = x >= p.nx - kGhost ? x - p.nx : x + p.nx;
        while (g >= -kGhost && g < p.nx + kGhost) {
            S* gc = row + g;
            gc[0] = IO::enc1(k ? fo[0].v.y : fo[0].v.x, k ? r0.v.y : r0.v.x, p.scale);
#pragma unroll
            for (int i = 1; i < 9; ++i)
                gc[i * p.plane] = IO::enc1(k ? fo[i].v.y : fo[i].v.x, i <= 4 ? p.rest.ax : p.rest.dg, p.scale);
            if (g < 0) { g -= p.nx; if (g < -kGhost) { g = x + p.nx; if (g >= p.nx + kGhost) break; } }
            else { g += p.nx; if (g >= p.nx + kGhost) break; }
        }
    }
}

template <typename S, int T, int MINB>
__global__ void __launch_bounds__(T, MINB) vanse_pair_kernel(const __grid_constant__ StepParams<float> p) {
    using L = PairLayout<S, T>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_abort;
    float* rbuf = reinterpret_cast<float*>(smem + L::kRho);
    float* fbuf = reinterpret_cast<float*>(smem + L::kFld);

    const int t = threadIdx.x;
    constexpr int A = L::A;
    const int x0 = blockIdx.x * p.W;
    const int y0 = blockIdx.y * p.H;
    const int y1 = min(y0 + p.H, p.ny);

    PairCtx<S, T> c{p, smem, &s_abort, t, 0, 0, y0, y1, 0, 0, 0, 0, 0, 0};
    c.wsp = ((kPadCols + x0 - kGhost) / A) * A;
    c.ww = ((kPadCols + x0 + 2 * T - 1 + A - 1) / A) * A - c.wsp;
    c.xa = x0 - 2 + 2 * t;
    c.sa = kPadCols + c.xa - c.wsp;
    c.rlo = y0 - 3;
    c.rhi = y1 + 2;
    if (p.wall_y) { c.rlo = max(c.rlo, 0); c.rhi = min(c.rhi, p.ny - 1); }
    c.waited = c.rlo - 1;
    c.issued = c.rlo - 1;

    if (t == 0) {
        s_abort = 0;
        for (int k = 0; k < kPairSlots; ++k) mbar_init(reinterpret_cast<uint64_t*>(smem) + k, 1);
        fence_mbar_init();
        for (int r = c.rlo; r <= min(y0, c.rhi); ++r) c.issue(r);
    }
    __syncthreads();

    PRow s0, s1, s2;
    auto iter = [&](PRow& An, PRow& Bs, PRow& Cs, const int p1) -> bool {
        const int p2 = p1 - 1, p3 = p1 - 2;
        c.wait_upto(p1 + 1);
        const bool ph1 = (p1 <= y1 + 1) && c.row_valid(p1);
        if (ph1) {
            pair_phase1<S, T>(c, An, p1);
            *reinterpret_cast<float2*>(rbuf + 2 + 2 * t) = An.rho.v;
        }
        __syncthreads();  // A: rho row p1 visible; slot of row p1-3 free
        if (s_abort) return false;
        if (t == 0 && p1 + 3 <= c.rhi && p1 + 3 >= c.rlo) {
            fence_proxy_async();
            c.issue(p1 + 3);
        }
        const bool ph2 = (p2 >= y0 - 1) && (p2 <= y1) && c.row_valid(p2);
        if (ph1) {
            const float l = rbuf[1 + 2 * t], r = rbuf[4 + 2 * t];
            An.dr = rpair(An.rho, r) - lpair(An.rho, l);
            An.wr = fma2(4.f, An.rho, rpair(An.rho, r) + lpair(An.rho, l));
        }
        if (ph2) pair_phase2<S, T>(c, An, Bs, Cs, p2, fbuf);
        __syncthreads();  // B: field row p2 visible
        if (ph2) pair_fields<S, T>(c, Bs, fbuf);
        const bool ph3 = (p3 >= y0) && (p3 < y1);
        if (ph3 && t >= 1 && t < T - 1) pair_phase3<S, T>(c, An, Bs, Cs, p3);
        return true;
    };

    const int n_it = (y1 + 1) - (y0 - 2) + 1;
    bool ok = true;
    for (int it = 0; it < n_it && ok; it += 3) {
        const int p1 = y0 - 2 + it;
        ok = iter(s0, s2, s1, p1);
        if (ok && it + 1 < n_it) ok = iter(s1, s0, s2, p1 + 1);
        if (ok && it + 2 < n_it) ok = iter(s2, s1, s0, p1 + 2);
    }
    if (!ok && t == 0) {
        // every copy that may still be in flight (see kWaitTries)
        for (int r = min(c.first_bad, c.waited + 1); r <= c.issued; ++r)
            mbar_wait_bounded(c.bar(r), c.parity(r), kWaitTries);
    }
}

}  // namespace lbmv
