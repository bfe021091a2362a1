// vanse_common.cuh -- lattice constants, storage encodings and the inline-PTX
// wrappers (mbarrier, bulk async copy) shared by the MRTLB-VANSE kernels.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace lbmv {

// D2Q9 velocities in the order of Eq. (5): rest, E, N, W, S, NE, NW, SW, SE.
__host__ __device__ constexpr int ex_of(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0); }
__host__ __device__ constexpr int ey_of(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0); }
__host__ __device__ constexpr int opp_of(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5); }
// 3 w_i of Eq. (5): the weight of the linear (momentum) term 3 w_i e_i . j of f^eq_i
template <typename T> __host__ __device__ constexpr T w3_of(int i) {
    return i == 0 ? (T)0 : (i <= 4 ? (T)1 / (T)3 : (T)1 / (T)12);
}

// Ghost columns kept on each side of a periodic x axis (the pull at halo radius 2
// reads 3 columns beyond a CTA's cells), and the column offset of cell x = 0 in a
// padded row (a multiple of every alignment unit used).
constexpr int kGhost = 3;
constexpr int kPadCols = 32;

// ------------------------------------------------------------------ storage
// Populations are stored in S and computed in R. FP16/BF16 hold scaled
// deviations from the rest state; FP32/FP64 hold f itself.
template <typename S> struct Prec;
template <> struct Prec<double> { using R = double; static constexpr bool kDev = false; };
template <> struct Prec<float> { using R = float; static constexpr bool kDev = true; };
template <> struct Prec<__half> { using R = float; static constexpr bool kDev = true; };
template <> struct Prec<__nv_bfloat16> { using R = float; static constexpr bool kDev = true; };

template <typename R> __device__ __forceinline__ R to_r(double v) { return (R)v; }

__device__ __forceinline__ double dec(double s, double, double) { return s; }
__device__ __forceinline__ float dec(float s, float rest, float inv_scale) { return fmaf(s, inv_scale, rest); }
__device__ __forceinline__ float dec(__half s, float rest, float inv_scale) { return fmaf(__half2float(s), inv_scale, rest); }
__device__ __forceinline__ float dec(__nv_bfloat16 s, float rest, float inv_scale) { return fmaf(__bfloat162float(s), inv_scale, rest); }

// The same decode in FP64 (the read-back kernels): the stored deviation and the rest
// value are added without the FP32 rounding at the scale of f.
__device__ __forceinline__ double decd(double s, double, double) { return s; }
__device__ __forceinline__ double decd(float s, double rest, double inv_scale) { return fma((double)s, inv_scale, rest); }
__device__ __forceinline__ double decd(__half s, double rest, double inv_scale) {
    return fma((double)__half2float(s), inv_scale, rest);
}
__device__ __forceinline__ double decd(__nv_bfloat16 s, double rest, double inv_scale) {
    return fma((double)__bfloat162float(s), inv_scale, rest);
}
template <typename T, typename S> __device__ __forceinline__ T dec_as(S s, T rest, T inv_scale) {
    if constexpr (sizeof(T) == 8) return decd(s, rest, inv_scale);
    else return dec(s, rest, inv_scale);
}

template <typename S, typename R> __device__ __forceinline__ S enc(R f, R rest, R scale);
template <> __device__ __forceinline__ double enc<double, double>(double f, double, double) { return f; }
template <> __device__ __forceinline__ float enc<float, float>(float f, float rest, float scale) { return (f - rest) * scale; }
template <> __device__ __forceinline__ __half enc<__half, float>(float f, float rest, float scale) { return __float2half_rn((f - rest) * scale); }
template <> __device__ __forceinline__ __nv_bfloat16 enc<__nv_bfloat16, float>(float f, float rest, float scale) { return __float2bfloat16_rn((f - rest) * scale); }
// FP64 values into every storage (the write-back kernel): the deviation is formed in FP64
template <> __device__ __forceinline__ float enc<float, double>(double f, double rest, double scale) { return (float)((f - rest) * scale); }
template <> __device__ __forceinline__ __half enc<__half, double>(double f, double rest, double scale) {
    return __float2half_rn((float)((f - rest) * scale));
}
template <> __device__ __forceinline__ __nv_bfloat16 enc<__nv_bfloat16, double>(double f, double rest, double scale) {
    return __float2bfloat16_rn((float)((f - rest) * scale));
}

// Rest-state populations of Eq. (14) (u = 0, rho = rho0): w_i kappa rho0 for
// i >= 1 and (phi - 5 kappa / 9) rho0 for i = 0.
template <typename R> struct Rest {
    R ax, dg, k59;  // kappa rho0 / 9, kappa rho0 / 36, 5 kappa rho0 / 9
    R rho0;
    __device__ __forceinline__ R r0(R phi) const { return phi * rho0 - k59; }
    __device__ __forceinline__ R ri(int i) const { return i <= 4 ? ax : dg; }
};

// ------------------------------------------------------------------ PTX
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after max_tries polls (each poll may suspend the thread
// for a hardware-chosen time), so a copy that never lands cannot hang the GPU.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t max_tries) {
    for (uint32_t k = 0; k < max_tries; ++k)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// 1-D bulk async copy global -> shared, completing on an mbarrier. Both addresses
// 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// The same two operations on shared-window addresses (no generic-to-shared
// conversion at the call site).
__device__ __forceinline__ void mbar_expect_tx_at(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s_at(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst), "l"(src),
        "r"(bytes), "r"(bar)
        : "memory");
}

// 3-D tiled tensor copy global -> shared: the box of the tensor map at coordinates
// (x, y, z), completing on an mbarrier. The map lives in the kernel's parameters; x
// times the element size must be a multiple of 16 bytes, the destination 128-byte
// aligned.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace lbmv
