// lbm_vanse.cu -- host side of the C ABI declared in include/lbm_vanse.h.
//
// Owns the device buffers of one lattice (two population buffers used in
// ping-pong, phi(t), phi(t+1), the optional body-force field, reduction scratch)
// and launches the kernels of vanse_step.cuh / vanse_aux.cuh on the handle's
// stream. Every entry point converts failures into an lbm_status and a message.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>
#include <type_traits>

#include "lbm_vanse.h"
#include "vanse_adjoint.cuh"
#include "vanse_aux.cuh"
#include "vanse_batch.cuh"
#include "vanse_pair.cuh"
#include "vanse_step.cuh"
#include "vanse_warp.cuh"

using namespace lbmv;

namespace {

constexpr int kThreads = 128;       // one-column step kernel: CTA size (W = kThreads - 4 columns)

// Step-kernel variants (params.kernel): 1 = one column per thread; 2..4 = two
// columns per thread on packed FP32 pairs with CTAs of 64 / 96 / 128 threads
// (W = 2T - 4 columns), register-capped for 6 / 4 / 3 resident CTAs per SM;
// 5 = one warp per CTA, two columns per lane, shuffle exchange (W = 60).
constexpr int kNumKernels = 5;
constexpr int kPairT[3] = {64, 96, 128};
constexpr int kDefaultKernel = 5;
constexpr int kAuxThreads = 256;
constexpr int kReduceBlocks = 1024;
constexpr int kGraphSteps = 32;     // steps per replayed CUDA graph (even: ping-pong returns to its buffer)

thread_local std::string g_create_error;

int storage_bytes(int storage) {
    switch (storage) {
        case LBM_FP64: return 8;
        case LBM_FP32: return 4;
        default: return 2;
    }
}

}  // namespace

struct lbm_vanse {
    lbm_vanse_params prm;
    cudaStream_t stream = nullptr;
    int device = 0;
    int sbytes = 4, rbytes = 4;   // storage and compute element sizes
    int P = 0;                    // padded row pitch (elements)
    long long plane = 0;          // elements per plane
    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    void* phi = nullptr;          // phi(t), R, padded
    void* phin = nullptr;         // phi(t+1), R, padded
    void* fb = nullptr;           // body-force field (2 planes), R, padded
    bool unsteady = false, has_fb = false, phi_set = false, initialised = false;
    double gx = 0, gy = 0;
    bool has_drag = false;        // F^B += -beta (u - u_s), beta = phi^2 (d0 + d1 (1 - phi))
    double drag_d0 = 0, drag_d1 = 0, us_x = 0, us_y = 0;
    bool nee_top = false;         // row ny-1: moving wall by non-equilibrium extrapolation
    double uw_x = 0, uw_y = 0;
    bool has_solid = false;       // phi = 0 marks solid cells (kernels 1 and 5)
    bool jbase = false;           // FP16/BF16 deviations from the momentum base (kernel 5)
    unsigned char* solid_tiles = nullptr;   // kernel 5 with solid cells: CTAs whose staged region holds one
    int* tile_order = nullptr;              // ... their launch order (those tiles first), and 2 counters
    int npl = 9;                  // planes per population buffer (11 with the momentum base)
    int* zero_phi = nullptr;      // device flag: the last phi upload held a zero
    unsigned* step_ctr = nullptr; // device step count of the one-warp kernel (seeds stochastic rounding)
    double s_nu = 0, s_e = 0;
    double scale = 1, inv_scale = 1;
    int* err = nullptr;           // device flag set by bounded waits
    uint32_t wait_tries = kWaitTries;   // polls of a staged-row wait (lowered only to test the timeout path)
    int* bad_phi = nullptr;       // device flags of the void-fraction check (1: phi_t, 2: phi_next)
    int* bad_phi_host = nullptr;  // pinned copy of them
    double* partial = nullptr;    // reduction partials (kReduceBlocks * 3)
    double* red_out = nullptr;    // reduction result (3)
    double* scratch = nullptr;    // 3 dense double fields (macros / error norms)
    long long steps = 0;
    // step-kernel launch shape
    int W = 0, H = 0, gridx = 0, gridy = 0;
    int resident = 1;             // step-kernel CTAs resident on the device
    // replayed graph of kGraphSteps steady steps, valid while its key matches
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    struct GraphKey {
        const void* phi; const void* fb; int has_fb; double gx, gy; int cur; double drag[4]; int has_drag;
        int nee; double uw[2];
        bool operator==(const GraphKey& o) const {
            return phi == o.phi && fb == o.fb && has_fb == o.has_fb && gx == o.gx && gy == o.gy && cur == o.cur &&
                   has_drag == o.has_drag && drag[0] == o.drag[0] && drag[1] == o.drag[1] && drag[2] == o.drag[2] &&
                   drag[3] == o.drag[3] && nee == o.nee && uw[0] == o.uw[0] && uw[1] == o.uw[1];
        }
    } gkey{};
    bool use_graphs = true;
    bool sums_configured = false; // shared-memory attributes set on the step-sum kernel variant
    bool solid_configured = false;  // ... and on the solid-cell variants
    bool nee_configured = false;    // ... and on kernel 5's moving-wall instances
    // uploads from pinned host memory: copied on their own stream into device staging
    // buffers (phi(t), phi(t+1)), so the copy overlaps the work already queued on
    // `stream`; staging_free marks the last read of the staging buffers on `stream`
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_done = nullptr, staging_free = nullptr;
    void* staging[2] = {nullptr, nullptr};
    CUtensorMap pop_map[2];       // kernel 5: each population buffer as a tensor [9][ny][P] (tma_load_3d)
    int kernel = 1;               // step-kernel variant (see kNumKernels)
    bool pair = false;            // two columns per thread (packed FP32) step kernel
    std::string msg;
};

namespace {

lbm_status fail(lbm_vanse* h, lbm_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) h->msg = buf; else g_create_error = buf;
    return st;
}

lbm_status cuda_fail(lbm_vanse* h, cudaError_t e, const char* what) {
    return fail(h, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(h, call)                                                      \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);         \
    } while (0)

template <typename R>
Rest<R> make_rest(const lbm_vanse* h) {
    Rest<R> r;
    const double k = h->prm.kappa, r0 = h->prm.rho0;
    r.ax = (R)(k * r0 / 9.0);
    r.dg = (R)(k * r0 / 36.0);
    r.k59 = (R)(5.0 * k * r0 / 9.0);
    r.rho0 = (R)r0;
    return r;
}

template <typename R>
Lattice<R> make_lattice(const lbm_vanse* h) {
    Lattice<R> L;
    L.plane = h->plane;
    L.nx = h->prm.nx;
    L.ny = h->prm.ny;
    L.P = h->P;
    L.wall_y = h->prm.bc_y == LBM_BC_BOUNCEBACK;
    L.wall_x = h->prm.bc_x == LBM_BC_BOUNCEBACK;
    L.model_b = h->prm.model_b;
    L.kappa = (R)h->prm.kappa;
    L.gx = (R)h->gx;
    L.gy = (R)h->gy;
    L.scale = (R)h->scale;
    L.inv_scale = (R)h->inv_scale;
    L.rest = make_rest<R>(h);
    L.eq2 = h->prm.eq_order == 2;
    L.has_drag = h->has_drag;
    L.drag_d0 = (R)h->drag_d0;
    L.drag_d1 = (R)h->drag_d1;
    L.us_x = (R)h->us_x;
    L.us_y = (R)h->us_y;
    L.has_solid = h->has_solid;
    L.jbase = h->jbase;
    return L;
}

int aux_blocks(long long n) {
    long long b = (n + kAuxThreads - 1) / kAuxThreads;
    return (int)std::max<long long>(1, std::min<long long>(b, 65535LL * 8));
}

template <typename S>
size_t step_smem_bytes(const lbm_vanse* h, int nR) {
    using R = typename Prec<S>::R;
    switch (h->kernel) {
        case 2: return PairLayout<S, 64>::bytes(nR);
        case 3: return PairLayout<S, 96>::bytes(nR);
        case 4: return PairLayout<S, 128>::bytes(nR);
        case 5: return h->jbase ? WarpLayout<S, 11>::bytes(nR) : WarpLayout<S>::bytes(nR);
        default:
            return StepLayout<S, R, kThreads>::bytes(nR) +
                   (h->has_solid ? StepLayout<S, R, kThreads>::solid_bytes() : 0);
    }
}

// the largest dynamic shared memory a launch of the handle's step kernel may ask for
template <typename S>
size_t step_smem_max(const lbm_vanse* h) {
    using R = typename Prec<S>::R;
    const size_t b = step_smem_bytes<S>(h, 4);
    return (h->kernel >= 2 && h->kernel <= 5) ? b : b + (h->has_solid ? 0 : StepLayout<S, R, kThreads>::solid_bytes());
}

int step_threads(const lbm_vanse* h) {
    if (h->kernel == 5) return 32;
    return h->kernel >= 2 ? kPairT[h->kernel - 2] : kThreads;
}

template <typename S>
const void* step_kernel_ptr(const lbm_vanse* h) {
    using R = typename Prec<S>::R;
    if constexpr (!std::is_same<S, double>::value) {
        switch (h->kernel) {
            case 2: return (const void*)vanse_pair_kernel<S, 64, 6>;
            case 3: return (const void*)vanse_pair_kernel<S, 96, 4>;
            case 4: return (const void*)vanse_pair_kernel<S, 128, 3>;
            case 5:
                if constexpr (sizeof(S) == 2) {
                    if (h->jbase) return warp_jb_kernel<S>();
                }
                return h->prm.eq_order == 2 ? (const void*)vanse_warp_kernel<S, LBMV_WARP_MINB, false, true>
                                            : (const void*)vanse_warp_kernel<S, LBMV_WARP_MINB>;
            default: break;
        }
    }
    return (const void*)vanse_step_kernel<S, R, kThreads>;
}

// Rows per strip (CTA): strip_rows, or automatically about five waves of resident
// CTAs (short strips cost halo rows, long ones leave SMs idle in the last wave); ten
// on kernel 5 with solid cells, whose CTAs next to a solid take several times as long
// as the others: shorter strips shorten the longest CTA (on the 4096^2 channel with
// a solid block 56 GLUPS at 24 rows against 49 at 47).
void pick_strip_height(lbm_vanse* h) {
    int H = h->prm.strip_rows;
    if (H <= 0) {
        const int waves = (h->has_solid && h->kernel == 5) ? 10 : 5;
        const int nstrips = std::max(1, (waves * h->resident + h->gridx - 1) / h->gridx);
        H = (h->prm.ny + nstrips - 1) / nstrips;
        H = std::max(H, 16);
    }
    h->H = std::min(H, h->prm.ny);
    h->gridy = (h->prm.ny + h->H - 1) / h->H;
}

template <typename S>
lbm_status configure(lbm_vanse* h) {
    using R = typename Prec<S>::R;
    (void)sizeof(R);
    const void* kern = step_kernel_ptr<S>(h);
    const int threads = step_threads(h);
    const size_t smax = step_smem_max<S>(h);
    CK(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
    CK(h, cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared));
    if constexpr (sizeof(S) == 2) {
        if (h->jbase) CK(h, warp_jb_configure<S>(smax));
    }
    const size_t s1 = step_smem_bytes<S>(h, 1);
    int per_sm = 0, nsm = 0;
    CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, s1));
    CK(h, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
    h->resident = std::max(1, per_sm * nsm);
    pick_strip_height(h);
    return LBM_OK;
}

// The step-sum variant of the handle's step kernel (kernels 1 and 5; nullptr for
// the others).
template <typename S>
const void* step_sums_kernel_ptr(const lbm_vanse* h) {
    using R = typename Prec<S>::R;
    if constexpr (!std::is_same<S, double>::value) {
        if (h->kernel == 5)
            return h->prm.eq_order == 2 ? (const void*)vanse_warp_kernel<S, LBMV_WARP_MINB, true, true>
                                        : (const void*)vanse_warp_kernel<S, LBMV_WARP_MINB, true>;
        if (h->kernel != 1) return nullptr;
    }
    return (const void*)vanse_step_kernel<S, R, kThreads, true>;   // (solid cells: launch_solid_step)
}

// Kernel 5 with the moving wall: its instances' shared-memory attributes, on first use.
template <typename S>
lbm_status configure_nee(lbm_vanse* h) {
    if constexpr (!std::is_same<S, double>::value) {
        if (!h->nee_configured) {
            CK(h, warp_nee_configure<S>(step_smem_max<S>(h)));
            h->nee_configured = true;
        }
    }
    return LBM_OK;
}

// Kernel 1 with solid cells: a variant of its own (the neighbour-by-neighbour stencil
// and the 3-row rings stay out of the other kernels); shared-memory attributes set on
// first use.
template <typename S>
lbm_status launch_solid_step(lbm_vanse* h, const StepParams<typename Prec<S>::R>& p, dim3 grid, size_t smem,
                             cudaStream_t stream, bool sums) {
    using R = typename Prec<S>::R;
    if constexpr (!std::is_same<S, double>::value) {
        if (h->kernel == 5) {
            if (!h->solid_configured) {
                CK(h, warp_solid_configure<S>(step_smem_max<S>(h)));
                h->solid_configured = true;
            }
            CK(h, warp_solid_launch<S>(p, grid, smem, stream, sums, p.eq2 != 0));
            // the one-warp kernel writes columns 0 .. nx-1 only
            const long long ng = (long long)h->npl * h->prm.ny * 2 * kGhost;
            ghost_fill_kernel<S><<<(int)std::min<long long>((ng + 255) / 256, 4096), 256, 0, stream>>>(
                (S*)p.dst, h->plane, h->prm.nx, h->prm.ny, h->P, h->step_ctr, h->npl);
            CK(h, cudaGetLastError());
            return LBM_OK;
        }
    }
    if (!h->solid_configured) {
        for (const void* k : {(const void*)vanse_step_kernel<S, R, kThreads, true, true>,
                              (const void*)vanse_step_kernel<S, R, kThreads, false, true>}) {
            CK(h, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)step_smem_max<S>(h)));
            CK(h, cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       cudaSharedmemCarveoutMaxShared));
        }
        h->solid_configured = true;
    }
    if (sums) vanse_step_kernel<S, R, kThreads, true, true><<<grid, kThreads, smem, stream>>>(p);
    else vanse_step_kernel<S, R, kThreads, false, true><<<grid, kThreads, smem, stream>>>(p);
    CK(h, cudaGetLastError());
    return LBM_OK;
}

template <typename S>
lbm_status enqueue_step(lbm_vanse* h, cudaStream_t stream, int src, double* sums = nullptr) {
    using R = typename Prec<S>::R;
    StepParams<R> p;
    p.src = h->f[src];
    p.dst = h->f[1 - src];
    p.phi = (const R*)h->phi;
    p.phin = h->unsteady ? (const R*)h->phin : (const R*)h->phi;
    p.fb = h->has_fb ? (const R*)h->fb : nullptr;
    p.plane = h->plane;
    p.nx = h->prm.nx;
    p.ny = h->prm.ny;
    p.P = h->P;
    p.W = h->W;
    p.H = h->H;
    p.wall_y = h->prm.bc_y == LBM_BC_BOUNCEBACK;
    p.wall_x = h->prm.bc_x == LBM_BC_BOUNCEBACK;
    p.unsteady = h->unsteady;
    p.has_fb = h->has_fb;
    p.model_b = h->prm.model_b;
    const int nR = 1 + (h->unsteady ? 1 : 0) + (h->has_fb ? 2 : 0);
    const size_t smem = step_smem_bytes<S>(h, nR);
    p.nR = nR;
    p.kappa = (R)h->prm.kappa;
    p.gx = (R)h->gx;
    p.gy = (R)h->gy;
    p.s_e = (R)h->s_e;
    p.s_eps = (R)h->prm.s_eps;
    p.s_q = (R)h->prm.s_q;
    p.s_nu = (R)h->s_nu;
    p.h_e = (R)(1.0 - 0.5 * h->s_e);
    p.h_eps = (R)(1.0 - 0.5 * h->prm.s_eps);
    p.h_q = (R)(1.0 - 0.5 * h->prm.s_q);
    p.h_nu = (R)(1.0 - 0.5 * h->s_nu);
    p.hs_e = (R)((1.0 - 0.5 * h->s_e) * h->scale);
    p.hs_eps = (R)((1.0 - 0.5 * h->prm.s_eps) * h->scale);
    p.hs_q = (R)((1.0 - 0.5 * h->prm.s_q) * h->scale);
    p.hs_nu = (R)((1.0 - 0.5 * h->s_nu) * h->scale);
    p.rho0s = (R)(h->prm.rho0 * h->scale);
    p.kp3 = (R)(h->inv_scale / 3.0);
    p.scale = (R)h->scale;
    p.inv_scale = (R)h->inv_scale;
    p.rest = make_rest<R>(h);
    p.err = h->err;
    p.eq2 = h->prm.eq_order == 2;
    p.has_drag = h->has_drag;
    p.drag_d0 = (R)h->drag_d0;
    p.drag_d1 = (R)h->drag_d1;
    p.us_x = (R)h->us_x;
    p.us_y = (R)h->us_y;
    p.sums = sums;
    p.nee_top = h->nee_top;
    p.uw_x = (R)h->uw_x;
    p.uw_y = (R)h->uw_y;
    p.has_solid = h->has_solid;
    p.solid_tiles = (h->has_solid && h->kernel == 5) ? h->solid_tiles : nullptr;
    p.tile_order = p.solid_tiles ? h->tile_order : nullptr;
    p.step_ctr = h->step_ctr;
    p.wait_tries = h->wait_tries;
    if (h->kernel == 5) p.pop_map = h->pop_map[src];
    dim3 grid(h->gridx, h->gridy);
    if (h->has_solid) return launch_solid_step<S>(h, p, grid, smem, stream, sums != nullptr);
    if (sums) {
        if (!h->sums_configured) {
            const void* kern = step_sums_kernel_ptr<S>(h);
            if (!kern) return fail(h, LBM_ERR_ARG, "step sums need step kernel 1 or 5 (kernel %d)", h->kernel);
            CK(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)step_smem_max<S>(h)));
            CK(h, cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       cudaSharedmemCarveoutMaxShared));
            h->sums_configured = true;
        }
        if constexpr (!std::is_same<S, double>::value) {
            if (h->kernel == 5) {
                if constexpr (sizeof(S) == 2) {
                    if (h->jbase) CK(h, warp_jb_launch<S>(p, grid, smem, stream, true, p.eq2 != 0));
                }
                if (!h->jbase && h->nee_top) {
                    lbm_status st = configure_nee<S>(h);
                    if (st != LBM_OK) return st;
                    CK(h, warp_nee_launch<S>(p, grid, smem, stream, true, p.eq2 != 0));
                } else if (!h->jbase) {
                    if (p.eq2) vanse_warp_kernel<S, LBMV_WARP_MINB, true, true><<<grid, 32, smem, stream>>>(p);
                    else vanse_warp_kernel<S, LBMV_WARP_MINB, true><<<grid, 32, smem, stream>>>(p);
                }
                CK(h, cudaGetLastError());
                const long long ng = (long long)h->npl * h->prm.ny * 2 * kGhost;
                ghost_fill_kernel<S><<<(int)std::min<long long>((ng + 255) / 256, 4096), 256, 0, stream>>>(
                    (S*)h->f[1 - src], h->plane, h->prm.nx, h->prm.ny, h->P, h->step_ctr, h->npl);
                CK(h, cudaGetLastError());
                return LBM_OK;
            }
        }
        vanse_step_kernel<S, R, kThreads, true><<<grid, kThreads, smem, stream>>>(p);
        CK(h, cudaGetLastError());
        return LBM_OK;
    }
    if constexpr (!std::is_same<S, double>::value) {
        switch (h->kernel) {
            case 2: vanse_pair_kernel<S, 64, 6><<<grid, 64, smem, stream>>>(p); CK(h, cudaGetLastError()); return LBM_OK;
            case 3: vanse_pair_kernel<S, 96, 4><<<grid, 96, smem, stream>>>(p); CK(h, cudaGetLastError()); return LBM_OK;
            case 4: vanse_pair_kernel<S, 128, 3><<<grid, 128, smem, stream>>>(p); CK(h, cudaGetLastError()); return LBM_OK;
            case 5: {
                if constexpr (sizeof(S) == 2) {
                    if (h->jbase) CK(h, warp_jb_launch<S>(p, grid, smem, stream, false, p.eq2 != 0));
                }
                if (!h->jbase && h->nee_top) {
                    lbm_status st = configure_nee<S>(h);
                    if (st != LBM_OK) return st;
                    CK(h, warp_nee_launch<S>(p, grid, smem, stream, false, p.eq2 != 0));
                } else if (!h->jbase) {
                    if (p.eq2) vanse_warp_kernel<S, LBMV_WARP_MINB, false, true><<<grid, 32, smem, stream>>>(p);
                    else vanse_warp_kernel<S, LBMV_WARP_MINB><<<grid, 32, smem, stream>>>(p);
                }
                CK(h, cudaGetLastError());
                // the one-warp kernel writes columns 0 .. nx-1 only
                const long long ng = (long long)h->npl * h->prm.ny * 2 * kGhost;
                ghost_fill_kernel<S><<<(int)std::min<long long>((ng + 255) / 256, 4096), 256, 0, stream>>>(
                    (S*)h->f[1 - src], h->plane, h->prm.nx, h->prm.ny, h->P, h->step_ctr, h->npl);
                CK(h, cudaGetLastError());
                return LBM_OK;
            }
            default: break;
        }
    }
    vanse_step_kernel<S, R, kThreads><<<grid, kThreads, smem, stream>>>(p);
    CK(h, cudaGetLastError());
    return LBM_OK;
}

template <typename S>
lbm_status launch_step(lbm_vanse* h, double* sums = nullptr) {
    lbm_status st = enqueue_step<S>(h, h->stream, h->cur, sums);
    if (st != LBM_OK) return st;
    h->cur = 1 - h->cur;
    if (h->unsteady) {
        // phi(t) <- phi(t+1); the field stays steady until the next set call
        std::swap(h->phi, h->phin);
        h->unsteady = false;
    }
    h->steps++;
    return LBM_OK;
}

// Capture kGraphSteps steady steps starting from buffer h->cur into an executable
// graph. Capture runs on a private stream (the caller's may be the legacy default
// stream, which cannot be captured); the graph is then launched on h->stream.
template <typename S>
lbm_status build_graph(lbm_vanse* h) {
    if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
    if (!h->cap_stream) CK(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    lbm_status st = LBM_OK;
    for (int k = 0; k < kGraphSteps && st == LBM_OK; ++k) st = enqueue_step<S>(h, h->cap_stream, h->cur ^ (k & 1));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (st != LBM_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { h->gexec = nullptr; return cuda_fail(h, e, "cudaGraphInstantiate"); }
    h->gkey = {h->phi, h->fb, (int)h->has_fb, h->gx, h->gy, h->cur, {h->drag_d0, h->drag_d1, h->us_x, h->us_y},
               (int)h->has_drag, (int)h->nee_top, {h->uw_x, h->uw_y}};
    return LBM_OK;
}

template <typename S>
lbm_status replay_graph(lbm_vanse* h) {
    lbm_vanse::GraphKey key{h->phi, h->fb, (int)h->has_fb, h->gx, h->gy, h->cur,
                            {h->drag_d0, h->drag_d1, h->us_x, h->us_y}, (int)h->has_drag,
                            (int)h->nee_top, {h->uw_x, h->uw_y}};
    if (!h->gexec || !(key == h->gkey)) {
        lbm_status st = build_graph<S>(h);
        if (st != LBM_OK) return st;
    }
    CK(h, cudaGraphLaunch(h->gexec, h->stream));
    h->steps += kGraphSteps;   // even count: h->cur is unchanged
    return LBM_OK;
}

// The momentum base's J planes of buffer b set to zero: the auxiliary writers encode
// every slot against f^rest alone (J = 0 is a valid base; the next step stores its own).
cudaError_t zero_j_planes(lbm_vanse* h, int b) {
    return cudaMemsetAsync((char*)h->f[b] + (size_t)9 * h->plane * h->sbytes, 0, (size_t)2 * h->plane * h->sbytes,
                           h->stream);
}

template <typename S>
lbm_status run_init(lbm_vanse* h, const double* rho, const double* ux, const double* uy) {
    using R = typename Prec<S>::R;
    const long long n = (long long)h->prm.nx * h->prm.ny;
    Lattice<R> L = make_lattice<R>(h);
    if (h->jbase) CK(h, zero_j_planes(h, h->cur));
    init_kernel<S, R><<<aux_blocks(n), kAuxThreads, 0, h->stream>>>(
        (S*)h->f[h->cur], (const R*)h->phi, h->has_fb ? (const R*)h->fb : nullptr, rho, ux, uy, L);
    CK(h, cudaGetLastError());
    return LBM_OK;
}

template <typename S>
lbm_status run_get(lbm_vanse* h, double* out) {
    using R = typename Prec<S>::R;
    const long long n = (long long)h->prm.nx * h->prm.ny;
    get_pop_kernel<S, R><<<aux_blocks(n), kAuxThreads, 0, h->stream>>>((const S*)h->f[h->cur], (const R*)h->phi, out,
                                                                       make_lattice<double>(h));
    CK(h, cudaGetLastError());
    return LBM_OK;
}

template <typename S>
lbm_status run_set(lbm_vanse* h, const double* in) {
    using R = typename Prec<S>::R;
    const long long n = (long long)h->prm.nx * h->prm.ny;
    if (h->jbase) CK(h, zero_j_planes(h, h->cur));
    set_pop_kernel<S, R><<<aux_blocks(n), kAuxThreads, 0, h->stream>>>((S*)h->f[h->cur], (const R*)h->phi, in,
                                                                       make_lattice<double>(h));
    CK(h, cudaGetLastError());
    return LBM_OK;
}

template <typename S>
lbm_status run_macros(lbm_vanse* h, double* rho, double* ux, double* uy, double* p) {
    using R = typename Prec<S>::R;
    const long long n = (long long)h->prm.nx * h->prm.ny;
    const Lattice<double> L = make_lattice<double>(h);   // the macroscopic passes compute in FP64
    rho_kernel<S, R><<<aux_blocks(n), kAuxThreads, 0, h->stream>>>((const S*)h->f[h->cur], (const R*)h->phi, rho, L);
    CK(h, cudaGetLastError());
    if (ux || uy || p) {
        vel_kernel<S, R><<<aux_blocks(n), kAuxThreads, 0, h->stream>>>(
            (const S*)h->f[h->cur], (const R*)h->phi, h->has_fb ? (const R*)h->fb : nullptr, rho, ux, uy, p, L);
        CK(h, cudaGetLastError());
    }
    return LBM_OK;
}

template <typename S>
lbm_status run_reduce(lbm_vanse* h) {
    using R = typename Prec<S>::R;
    moments_reduce_kernel<S, R><<<kReduceBlocks, kAuxThreads, 0, h->stream>>>((const S*)h->f[h->cur],
                                                                               (const R*)h->phi, h->partial,
                                                                               make_lattice<R>(h));
    CK(h, cudaGetLastError());
    finish_reduce_kernel<<<1, 1024, 0, h->stream>>>(h->partial, kReduceBlocks, h->red_out);
    CK(h, cudaGetLastError());
    return LBM_OK;
}

#define DISPATCH(h, fn, ...)                                                     \
    ([&]() -> lbm_status {                                                       \
        switch ((h)->prm.storage) {                                              \
            case LBM_FP64: return fn<double>((h), ##__VA_ARGS__);                \
            case LBM_FP32: return fn<float>((h), ##__VA_ARGS__);                 \
            case LBM_FP16: return fn<__half>((h), ##__VA_ARGS__);                \
            default: return fn<__nv_bfloat16>((h), ##__VA_ARGS__);               \
        }                                                                        \
    }())

bool host_pinned(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeHost;
}

// Copy a caller array to device memory if it lives on the host; returns the
// device pointer to use (caller's own pointer when on_device). A copy from pinned
// memory is asynchronous, so the call waits for it: the caller may reuse its array
// as soon as the entry point returns.
template <typename T>
lbm_status stage_in(lbm_vanse* h, const T* src, long long count, int on_device, T** dev, bool* owned) {
    *owned = false;
    if (on_device) { *dev = const_cast<T*>(src); return LBM_OK; }
    CK(h, cudaMallocAsync((void**)dev, (size_t)count * sizeof(T), h->stream));
    *owned = true;
    CK(h, cudaMemcpyAsync(*dev, src, (size_t)count * sizeof(T), cudaMemcpyHostToDevice, h->stream));
    if (host_pinned(src)) CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

template <typename T>
lbm_status pad_into(lbm_vanse* h, const T* dev_src, void* dst, int* zero_seen = nullptr) {
    const int blocks = std::min(h->prm.ny, 65535);
    if (h->rbytes == 8)
        pad_field_kernel<T, double><<<blocks, kAuxThreads, 0, h->stream>>>(dev_src, (double*)dst, h->prm.nx,
                                                                           h->prm.ny, h->P, zero_seen);
    else
        pad_field_kernel<T, float><<<blocks, kAuxThreads, 0, h->stream>>>(dev_src, (float*)dst, h->prm.nx,
                                                                          h->prm.ny, h->P, zero_seen);
    CK(h, cudaGetLastError());
    return LBM_OK;
}

template <typename T, typename S>
lbm_status rebase_pad(lbm_vanse* h, const T* dev_src) {
    using R = typename Prec<S>::R;
    const int blocks = std::min(h->prm.ny, 65535);
    pad_phi_rebase_kernel<T, R, S><<<blocks, kAuxThreads, 0, h->stream>>>(
        dev_src, (R*)h->phi, (S*)h->f[h->cur], h->prm.nx, h->prm.ny, h->P, (R)(h->prm.rho0 * h->scale), h->zero_phi);
    CK(h, cudaGetLastError());
    return LBM_OK;
}

// phi(t) into the lattice: a plain copy while no populations are stored (or they are
// FP64, stored as they are); otherwise the copy that also keeps the populations
// (pad_phi_rebase_kernel).
template <typename T>
lbm_status put_phi_t(lbm_vanse* h, const T* dev_src) {
    if (!h->initialised || h->prm.storage == LBM_FP64) return pad_into<T>(h, dev_src, h->phi, h->zero_phi);
    switch (h->prm.storage) {
        case LBM_FP32: return rebase_pad<T, float>(h, dev_src);
        case LBM_FP16: return rebase_pad<T, __half>(h, dev_src);
        default: return rebase_pad<T, __nv_bfloat16>(h, dev_src);
    }
}

// The void-fraction check (check_phi_kernel) of the staged fields on stream s, then
// its verdict: the flags are copied to pinned host memory and s is synchronised. A
// bad field fails the call before anything of the lattice changes.
lbm_status ensure_phi_check(lbm_vanse* h) {
    if (h->bad_phi) return LBM_OK;
    CK(h, cudaMalloc((void**)&h->bad_phi, sizeof(int)));
    CK(h, cudaMallocHost((void**)&h->bad_phi_host, sizeof(int)));
    return LBM_OK;
}

template <typename T>
lbm_status check_phi_fields(lbm_vanse* h, const T* phi_t, const T* phi_next, cudaStream_t s) {
    lbm_status st = ensure_phi_check(h);
    if (st != LBM_OK) return st;
    const long long n = (long long)h->prm.nx * h->prm.ny;
    const int blocks = (int)std::min<long long>((n + kAuxThreads - 1) / kAuxThreads, 2048);
    CK(h, cudaMemsetAsync(h->bad_phi, 0, sizeof(int), s));
    check_phi_kernel<T><<<blocks, kAuxThreads, 0, s>>>(phi_t, n, 1, h->bad_phi);
    CK(h, cudaGetLastError());
    if (phi_next) {
        check_phi_kernel<T><<<blocks, kAuxThreads, 0, s>>>(phi_next, n, 2, h->bad_phi);
        CK(h, cudaGetLastError());
    }
    CK(h, cudaMemcpyAsync(h->bad_phi_host, h->bad_phi, sizeof(int), cudaMemcpyDeviceToHost, s));
    return LBM_OK;
}

// after the check's stream has been synchronised
lbm_status phi_verdict(lbm_vanse* h) {
    const int b = *h->bad_phi_host;
    if (!b) return LBM_OK;
    return fail(h, LBM_ERR_ARG, "%s outside [0, 1] (NaN, negative or above 1); the lattice is unchanged",
                b == 1 ? "phi_t holds values" : (b == 2 ? "phi_next holds values" : "phi_t and phi_next hold values"));
}

// Upload of phi(t) [and phi(t+1)] from pinned host arrays: the copies run on the
// copy stream into the staging buffers, overlapping whatever `stream` is still
// executing (e.g. the previous step); the call returns once the caller's arrays
// have been read, and the padding kernels follow on `stream`.
template <typename T>
lbm_status upload_void_fraction_pinned(lbm_vanse* h, const T* phi_t, const T* phi_next) {
    const long long n = (long long)h->prm.nx * h->prm.ny;
    const size_t bytes = (size_t)n * sizeof(T);
    if (!h->copy_stream) {
        CK(h, cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
        CK(h, cudaEventCreateWithFlags(&h->copy_done, cudaEventDisableTiming));
        CK(h, cudaEventCreateWithFlags(&h->staging_free, cudaEventDisableTiming));
        CK(h, cudaEventRecord(h->staging_free, h->stream));
    }
    for (int k = 0; k < (phi_next ? 2 : 1); ++k)
        if (!h->staging[k]) CK(h, cudaMalloc(&h->staging[k], (size_t)n * sizeof(double)));
    CK(h, cudaStreamWaitEvent(h->copy_stream, h->staging_free, 0));
    CK(h, cudaMemcpyAsync(h->staging[0], phi_t, bytes, cudaMemcpyHostToDevice, h->copy_stream));
    if (phi_next) CK(h, cudaMemcpyAsync(h->staging[1], phi_next, bytes, cudaMemcpyHostToDevice, h->copy_stream));
    // the check runs on the copy stream too, so the wait for the copies covers it
    lbm_status chk = check_phi_fields<T>(h, (const T*)h->staging[0], phi_next ? (const T*)h->staging[1] : nullptr,
                                         h->copy_stream);
    if (chk != LBM_OK) return chk;
    CK(h, cudaEventRecord(h->copy_done, h->copy_stream));
    CK(h, cudaEventSynchronize(h->copy_done));
    chk = phi_verdict(h);
    if (chk != LBM_OK) return chk;
    CK(h, cudaStreamWaitEvent(h->stream, h->copy_done, 0));
    CK(h, cudaMemsetAsync(h->zero_phi, 0, sizeof(int), h->stream));
    lbm_status st = put_phi_t<T>(h, (const T*)h->staging[0]);
    if (st == LBM_OK && phi_next) st = pad_into<T>(h, (const T*)h->staging[1], h->phin, h->zero_phi);
    if (st != LBM_OK) return st;
    CK(h, cudaEventRecord(h->staging_free, h->stream));
    return LBM_OK;
}

// Kernel 5 with solid cells: flag the CTAs whose staged region holds a solid cell of
// phi(t) or phi(t+1) (solid_tiles_kernel), after every change of phi. The others run
// the solid-free path. (Solid cells stay solid, so the flags of phi(t) and phi(t+1)
// also cover the steady steps after phi(t+1) has become phi(t).)
lbm_status update_solid_tiles(lbm_vanse* h) {
    if (!h->has_solid || h->kernel != 5 || !h->phi_set) return LBM_OK;
    const int nt = h->gridx * h->gridy;
    if (!h->solid_tiles) CK(h, cudaMallocAsync((void**)&h->solid_tiles, (size_t)nt, h->stream));
    if (!h->tile_order) CK(h, cudaMallocAsync((void**)&h->tile_order, (size_t)(nt + 2) * sizeof(int), h->stream));
    solid_tiles_kernel<float><<<dim3(h->gridx, h->gridy), 256, 0, h->stream>>>(
        (const float*)h->phi, h->unsteady ? (const float*)h->phin : nullptr, h->solid_tiles, h->prm.nx, h->prm.ny, h->P,
        h->W, h->H, h->prm.bc_y == LBM_BC_BOUNCEBACK);
    CK(h, cudaGetLastError());
    CK(h, cudaMemsetAsync(h->tile_order + nt, 0, 2 * sizeof(int), h->stream));
    solid_order_kernel<<<(nt + 255) / 256, 256, 0, h->stream>>>(h->solid_tiles, nt, h->tile_order, h->tile_order + nt);
    CK(h, cudaGetLastError());
    return LBM_OK;
}

// lbm_vanse_set_void_fraction for double or float caller arrays.
template <typename T>
lbm_status set_void_fraction_impl(lbm_vanse* h, const T* phi_t, const T* phi_next, int on_device) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!phi_t) return fail(h, LBM_ERR_ARG, "phi_t is NULL");
    const long long n = (long long)h->prm.nx * h->prm.ny;
    if (!on_device && host_pinned(phi_t) && (!phi_next || host_pinned(phi_next))) {
        lbm_status st = upload_void_fraction_pinned<T>(h, phi_t, phi_next);
        if (st != LBM_OK) return st;
        h->unsteady = phi_next != nullptr;
        h->phi_set = true;
        return update_solid_tiles(h);
    }
    // stage and check both fields before either replaces the lattice's own
    T* d[2] = {nullptr, nullptr};
    bool owned[2] = {false, false};
    auto release = [&]() {
        for (int k = 0; k < 2; ++k)
            if (owned[k]) cudaFreeAsync(d[k], h->stream);
    };
    lbm_status st = stage_in<T>(h, phi_t, n, on_device, &d[0], &owned[0]);
    if (st == LBM_OK && phi_next) st = stage_in<T>(h, phi_next, n, on_device, &d[1], &owned[1]);
    if (st == LBM_OK) st = check_phi_fields<T>(h, d[0], d[1], h->stream);
    if (st == LBM_OK) {
        const cudaError_t e = cudaStreamSynchronize(h->stream);
        st = e == cudaSuccess ? phi_verdict(h) : cuda_fail(h, e, "void fraction check");
    }
    if (st != LBM_OK) { release(); return st; }
    CK(h, cudaMemsetAsync(h->zero_phi, 0, sizeof(int), h->stream));
    st = put_phi_t<T>(h, d[0]);
    if (st == LBM_OK && phi_next) st = pad_into<T>(h, d[1], h->phin, h->zero_phi);
    release();
    if (st != LBM_OK) return st;
    h->unsteady = phi_next != nullptr;
    h->phi_set = true;
    return update_solid_tiles(h);
}

lbm_status ensure_scratch(lbm_vanse* h) {
    if (h->scratch) return LBM_OK;
    const long long n = (long long)h->prm.nx * h->prm.ny;
    CK(h, cudaMallocAsync((void**)&h->scratch, (size_t)(3 * n) * sizeof(double), h->stream));
    return LBM_OK;
}

bool rate_ok(double s) { return s > 0.0 && s < 2.0; }

// The tensor map of one population buffer for the one-warp kernel: a 3-D tensor
// [9 planes][ny rows][P columns] of the storage type (row and plane strides are
// multiples of 16 bytes: P is a multiple of 32), box = the staged width WW x 1 row x 9
// planes. cuTensorMapEncodeTiled comes from the driver through the runtime's entry
// point, so the library links no driver library of its own.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Encodes the map of one population buffer (P columns per row, ny rows, planes of
// `plane` elements, storage `storage`); returns an empty string or the failure.
std::string encode_pop_map_raw(void* buf, int P, int ny, long long plane, int storage, CUtensorMap* out,
                               int npl = 9) {
    static EncodeTiledFn enc = nullptr;
    static std::mutex mu;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!enc) {
            cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
            void* fn = nullptr;
            const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                                   cudaEnableDefault, &q);
            if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
                return "cuTensorMapEncodeTiled is not available from the driver";
            enc = (EncodeTiledFn)fn;
        }
    }
    const int sb = storage_bytes(storage);
    const cuuint64_t dims[3] = {(cuuint64_t)P, (cuuint64_t)ny, (cuuint64_t)npl};
    const cuuint64_t strides[2] = {(cuuint64_t)P * sb, (cuuint64_t)plane * sb};
    // the staged width WarpLayout<S>::WW: 64 columns plus 16 bytes on each side
    const cuuint32_t box[3] = {(cuuint32_t)(64 + 2 * (16 / sb)), 1, (cuuint32_t)npl};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt = storage == LBM_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : (storage == LBM_FP16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                          : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    const CUresult r = enc(out, dt, 3, buf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    return std::string();
}

template <typename S>
lbm_status encode_pop_map(lbm_vanse* h, void* buf, CUtensorMap* out) {
    static_assert(WarpLayout<S>::WW == 64 + 2 * (16 / (int)sizeof(S)), "box width of encode_pop_map_raw");
    const std::string e = encode_pop_map_raw(buf, h->P, h->prm.ny, h->plane, h->prm.storage, out, h->npl);
    if (!e.empty()) return fail(h, LBM_ERR_CUDA, "%s", e.c_str());
    return LBM_OK;
}

template <typename S>
lbm_status encode_pop_maps(lbm_vanse* h) {
    if constexpr (std::is_same<S, double>::value) {
        return LBM_OK;
    } else {
        if (h->kernel != 5) return LBM_OK;
        for (int b = 0; b < 2; ++b) {
            const lbm_status st = encode_pop_map<S>(h, h->f[b], &h->pop_map[b]);
            if (st != LBM_OK) return st;
        }
        return LBM_OK;
    }
}

}  // namespace

// ================================================== allocation-free reduction
// Per-row partial sums for lbm_vanse_reduce_noalloc live in this fixed array, so
// that call needs no cudaMalloc. In host code the name is only a stand-in for the
// device copy: its device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) double g_noalloc_rows[LBM_VANSE_NOALLOC_MAX_ROWS * 3];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_addr[kMaxDevices] = {};

// Device address of g_noalloc_rows on h's device (looked up on first use, with that
// device current). The lookup is refused while h's stream is capturing a graph: it
// must happen once, outside any capture.
lbm_status noalloc_rows(lbm_vanse* h, double** out) {
    if (h->device < 0 || h->device >= kMaxDevices) return fail(h, LBM_ERR_ARG, "device %d out of range", h->device);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[h->device]) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        CK(h, cudaStreamIsCapturing(h->stream, &cap));
        if (cap != cudaStreamCaptureStatusNone)
            return fail(h, LBM_ERR_STATE,
                        "the first lbm_vanse_reduce_noalloc call on device %d must come before any stream capture "
                        "(it looks up the address of the fixed scratch)", h->device);
        int prev = -1;
        CK(h, cudaGetDevice(&prev));
        if (prev != h->device) CK(h, cudaSetDevice(h->device));
        void* addr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_rows);
        if (prev != h->device) cudaSetDevice(prev);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaGetSymbolAddress(reduction rows)");
        g_noalloc_addr[h->device] = static_cast<double*>(addr);
    }
    *out = g_noalloc_addr[h->device];
    return LBM_OK;
}

template <typename S>
lbm_status run_reduce_noalloc(lbm_vanse* h, double* rows, double* out) {
    using R = typename Prec<S>::R;
    const int blocks = std::min(h->prm.ny, 1024);
    row_moments_kernel<S, R><<<blocks, kAuxThreads, 0, h->stream>>>((const S*)h->f[h->cur], (const R*)h->phi, rows,
                                                                     make_lattice<R>(h));
    CK(h, cudaGetLastError());
    finish_reduce_kernel<<<1, 1024, 0, h->stream>>>(rows, h->prm.ny, out);
    CK(h, cudaGetLastError());
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_vanse_reduce_noalloc(lbm_vanse_t h, double* out_dev) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!out_dev) return fail(h, LBM_ERR_ARG, "out_dev is NULL");
    if (h->prm.ny > LBM_VANSE_NOALLOC_MAX_ROWS)
        return fail(h, LBM_ERR_ARG, "ny = %d exceeds the %d rows the fixed reduction scratch holds", h->prm.ny,
                    LBM_VANSE_NOALLOC_MAX_ROWS);
    if (!h->initialised) return fail(h, LBM_ERR_STATE, "lattice not initialised");
    double* rows = nullptr;
    lbm_status st = noalloc_rows(h, &rows);
    if (st != LBM_OK) return st;
    // the scratch address belongs to h's device: launch there even when the calling
    // thread has another device current, and put the caller's device back afterwards
    int prev = -1;
    CK(h, cudaGetDevice(&prev));
    if (prev != h->device) CK(h, cudaSetDevice(h->device));
    st = DISPATCH(h, run_reduce_noalloc, rows, out_dev);
    if (prev != h->device) {
        const cudaError_t e = cudaSetDevice(prev);
        if (st == LBM_OK && e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice(caller's device)");
    }
    return st;
}

// ============================================================================ C ABI

extern "C" void lbm_vanse_default_params(lbm_vanse_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->tau_nu = 0.8;
    p->s_e = 0.0;
    p->s_eps = 1.2;
    p->s_q = 1.4;
    p->s_c = 1.0;
    p->kappa = 0.5;
    p->rho0 = 1.0;
    p->bc_x = LBM_BC_PERIODIC;
    p->bc_y = LBM_BC_PERIODIC;
    p->storage = LBM_FP32;
    p->model_b = 0;
    p->storage_scale_log2 = -1000;  // sentinel: per-precision default
    p->strip_rows = 0;
    p->eager = 0;
    p->eq_order = 3;
    p->dev_base = LBM_BASE_REST;
}

extern "C" lbm_status lbm_vanse_create(const lbm_vanse_params* p, void* cuda_stream, lbm_vanse_t* out) {
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!p) return fail(nullptr, LBM_ERR_ARG, "params is NULL");
    if (p->nx < 1 || p->ny < 1) return fail(nullptr, LBM_ERR_ARG, "nx, ny must be >= 1 (got %d, %d)", p->nx, p->ny);
    if ((long long)p->nx * p->ny > (1LL << 31)) return fail(nullptr, LBM_ERR_ARG, "lattice too large");
    if (!(p->tau_nu > 0.5)) return fail(nullptr, LBM_ERR_ARG, "tau_nu must exceed 1/2 (got %g)", p->tau_nu);
    if (!(p->kappa >= 0.0 && p->kappa <= 1.0)) return fail(nullptr, LBM_ERR_ARG, "kappa must lie in [0, 1]");
    if (!(p->rho0 > 0.0)) return fail(nullptr, LBM_ERR_ARG, "rho0 must be positive");
    if (!rate_ok(p->s_eps) || !rate_ok(p->s_q) || !rate_ok(p->s_c) || (p->s_e > 0 && !rate_ok(p->s_e)))
        return fail(nullptr, LBM_ERR_ARG, "relaxation rates must lie in (0, 2)");
    if (p->bc_x != LBM_BC_PERIODIC && p->bc_x != LBM_BC_BOUNCEBACK) return fail(nullptr, LBM_ERR_ARG, "bad bc_x");
    if (p->bc_x == LBM_BC_BOUNCEBACK && p->kernel >= 2)
        return fail(nullptr, LBM_ERR_ARG, "x walls run on step kernel 1");
    if (p->bc_y != LBM_BC_PERIODIC && p->bc_y != LBM_BC_BOUNCEBACK) return fail(nullptr, LBM_ERR_ARG, "bad bc_y");
    if (p->storage < LBM_FP64 || p->storage > LBM_BF16) return fail(nullptr, LBM_ERR_ARG, "bad storage");
    if (p->strip_rows < 0) return fail(nullptr, LBM_ERR_ARG, "strip_rows must be >= 0");
    if (p->dev_base != LBM_BASE_REST && p->dev_base != LBM_BASE_MOMENTUM)
        return fail(nullptr, LBM_ERR_ARG, "dev_base must be LBM_BASE_REST or LBM_BASE_MOMENTUM");
    if (p->dev_base == LBM_BASE_MOMENTUM) {
        if (p->storage != LBM_FP16 && p->storage != LBM_BF16)
            return fail(nullptr, LBM_ERR_ARG, "the momentum base is an FP16 / BF16 storage form");
        // the kernel the lattice would run (the default rule below)
        const int k = p->kernel ? p->kernel : (p->bc_x == LBM_BC_BOUNCEBACK ? 1 : kDefaultKernel);
        if (k != 5)
            return fail(nullptr, LBM_ERR_ARG, "the momentum base runs on step kernel 5 (this lattice: kernel %d)", k);
    }

    lbm_vanse* h = new lbm_vanse();
    h->prm = *p;
    h->stream = (cudaStream_t)cuda_stream;
    h->use_graphs = p->eager == 0;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) { delete h; return fail(nullptr, LBM_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e)); }
    h->sbytes = storage_bytes(p->storage);
    h->rbytes = p->storage == LBM_FP64 ? 8 : 4;
    h->s_nu = 1.0 / p->tau_nu;
    if (p->s_e > 0) h->s_e = p->s_e;
    else {
        const double nu = (p->tau_nu - 0.5) / 3.0;  // Eq. (3)-(4): tau^-1 = nu / cs^2 + 1/2
        const double nu_e = nu / 3.0;               // Eq. (A12)
        h->s_e = 1.0 / (3.0 * nu_e + 0.5);
    }
    int k = p->storage_scale_log2;
    if (k == -1000) k = (p->storage == LBM_FP16) ? 16 : 0;
    if (p->storage == LBM_FP16 || p->storage == LBM_BF16) {
        h->scale = std::ldexp(1.0, k);
        h->inv_scale = std::ldexp(1.0, -k);
    }
    if (p->kernel < 0 || p->kernel > kNumKernels) {
        delete h;
        return fail(nullptr, LBM_ERR_ARG, "kernel must lie in 0..%d", kNumKernels);
    }
    if (p->kernel >= 2 && p->storage == LBM_FP64) {
        delete h;
        return fail(nullptr, LBM_ERR_ARG, "the two-column kernels run packed FP32 arithmetic; FP64 storage needs kernel 1");
    }
    if (p->eq_order != 0 && p->eq_order != 2 && p->eq_order != 3) {
        delete h;
        return fail(nullptr, LBM_ERR_ARG, "eq_order must be 2 (App. B) or 3 (Eq. 14; 0 = 3)");
    }
    if (p->eq_order == 2 && p->kernel >= 2 && p->kernel <= 4) {
        delete h;
        return fail(nullptr, LBM_ERR_ARG, "the App. B equilibrium runs on kernels 1 and 5");
    }
    if (h->prm.eq_order == 0) h->prm.eq_order = 3;
    h->kernel = p->kernel ? p->kernel
                          : ((p->storage == LBM_FP64 || p->bc_x == LBM_BC_BOUNCEBACK) ? 1 : kDefaultKernel);
    h->jbase = p->dev_base == LBM_BASE_MOMENTUM;   // (checked above)
    h->npl = h->jbase ? 11 : 9;
    h->pair = h->kernel >= 2;
    h->W = h->kernel == 5 ? 60 : (h->pair ? 2 * kPairT[h->kernel - 2] - 4 : kThreads - 4);
    h->gridx = (p->nx + h->W - 1) / h->W;
    h->P = ((kPadCols + h->gridx * h->W + kPadCols) + 31) / 32 * 32;
    h->plane = (long long)p->ny * h->P;

    lbm_status st = LBM_OK;
    auto alloc = [&](void** ptr, size_t bytes) -> bool {
        cudaError_t ee = cudaMallocAsync(ptr, bytes, h->stream);
        if (ee != cudaSuccess) { st = cuda_fail(h, ee, "cudaMallocAsync"); return false; }
        ee = cudaMemsetAsync(*ptr, 0, bytes, h->stream);
        if (ee != cudaSuccess) { st = cuda_fail(h, ee, "cudaMemsetAsync"); return false; }
        return true;
    };
    const size_t popb = (size_t)h->npl * h->plane * h->sbytes;
    const size_t fldb = (size_t)h->plane * h->rbytes;
    bool ok = alloc(&h->f[0], popb) && alloc(&h->f[1], popb) && alloc(&h->phi, fldb) && alloc(&h->phin, fldb) &&
              alloc((void**)&h->err, sizeof(int)) && alloc((void**)&h->zero_phi, sizeof(int)) &&
              alloc((void**)&h->step_ctr, sizeof(unsigned)) &&
              alloc((void**)&h->partial, kReduceBlocks * 3 * sizeof(double)) &&
              alloc((void**)&h->red_out, 4 * sizeof(double));
    if (ok) st = DISPATCH(h, configure);
    if (ok && st == LBM_OK) st = DISPATCH(h, encode_pop_maps);
    if (!ok || st != LBM_OK) {
        g_create_error = h->msg;
        lbm_vanse_destroy(h);
        return st == LBM_OK ? LBM_ERR_CUDA : st;
    }
    *out = h;
    return LBM_OK;
}

extern "C" lbm_status lbm_vanse_set_void_fraction(lbm_vanse_t h, const double* phi_t, const double* phi_next,
                                                  int on_device) {
    return set_void_fraction_impl<double>(h, phi_t, phi_next, on_device);
}

extern "C" lbm_status lbm_vanse_set_void_fraction_f32(lbm_vanse_t h, const float* phi_t, const float* phi_next,
                                                      int on_device) {
    return set_void_fraction_impl<float>(h, phi_t, phi_next, on_device);
}

extern "C" lbm_status lbm_vanse_set_body_force(lbm_vanse_t h, double gx, double gy, const double* field,
                                               int on_device) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!std::isfinite(gx) || !std::isfinite(gy)) return fail(h, LBM_ERR_ARG, "non-finite body force");
    h->gx = gx;
    h->gy = gy;
    if (!field) { h->has_fb = false; return LBM_OK; }
    const long long n = (long long)h->prm.nx * h->prm.ny;
    if (!h->fb) {
        cudaError_t e = cudaMallocAsync(&h->fb, (size_t)2 * h->plane * h->rbytes, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMallocAsync(body force)");
        e = cudaMemsetAsync(h->fb, 0, (size_t)2 * h->plane * h->rbytes, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync(body force)");
    }
    double* d = nullptr;
    bool owned = false;
    lbm_status st = stage_in(h, field, 2 * n, on_device, &d, &owned);
    if (st != LBM_OK) return st;
    st = pad_into(h, d, h->fb);
    if (st == LBM_OK) st = pad_into(h, d + n, (char*)h->fb + (size_t)h->plane * h->rbytes);
    if (owned) cudaFreeAsync(d, h->stream);
    if (st != LBM_OK) return st;
    h->has_fb = true;
    return LBM_OK;
}

extern "C" lbm_status lbm_vanse_set_drag(lbm_vanse_t h, double d0, double d1, double us_x, double us_y) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!std::isfinite(d0) || !std::isfinite(d1) || !std::isfinite(us_x) || !std::isfinite(us_y) || d0 < 0 || d1 < 0)
        return fail(h, LBM_ERR_ARG, "drag coefficients must be finite and >= 0, u_s finite");
    const bool on = d0 > 0 || d1 > 0;
    if (on && h->kernel >= 2 && h->kernel <= 4)
        return fail(h, LBM_ERR_ARG, "the drag runs on kernels 1 and 5 (this lattice uses kernel %d)", h->kernel);
    h->has_drag = on;
    h->drag_d0 = d0;
    h->drag_d1 = d1;
    h->us_x = us_x;
    h->us_y = us_y;
    return LBM_OK;
}

extern "C" lbm_status lbm_vanse_set_solid_cells(lbm_vanse_t h, int enable) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (enable && h->kernel != 1 && h->kernel != 5)
        return fail(h, LBM_ERR_ARG, "solid cells run on step kernels 1 and 5 (this lattice uses kernel %d)",
                    h->kernel);
    if (enable && h->prm.bc_x == LBM_BC_BOUNCEBACK)
        return fail(h, LBM_ERR_ARG, "solid cells and x walls together are not supported (use a solid frame)");
    if (enable && h->jbase)
        return fail(h, LBM_ERR_ARG, "solid cells and the momentum base together are not supported");
    h->has_solid = enable != 0;
    if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }   // the step's shared memory changes
    if (h->kernel == 5) {
        // the strip height follows (pick_strip_height); the tile flags are re-sized
        const int gy = h->gridy;
        pick_strip_height(h);
        if (h->gridy != gy) {
            if (h->solid_tiles) { cudaFreeAsync(h->solid_tiles, h->stream); h->solid_tiles = nullptr; }
            if (h->tile_order) { cudaFreeAsync(h->tile_order, h->stream); h->tile_order = nullptr; }
        }
    }
    return update_solid_tiles(h);
}

extern "C" lbm_status lbm_vanse_set_row_wait_limit(lbm_vanse_t h, long long polls) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    const uint32_t v = polls < 0 ? kWaitTries : (uint32_t)std::min<long long>(polls, (long long)kWaitTries);
    if (v != h->wait_tries) {
        h->wait_tries = v;
        if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }   // the steps' parameters change
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_vanse_set_moving_wall(lbm_vanse_t h, int enable, double uw_x, double uw_y) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!enable) { h->nee_top = false; h->uw_x = h->uw_y = 0; return LBM_OK; }
    if (!std::isfinite(uw_x) || !std::isfinite(uw_y)) return fail(h, LBM_ERR_ARG, "wall velocity must be finite");
    if (h->prm.bc_y != LBM_BC_BOUNCEBACK) return fail(h, LBM_ERR_ARG, "the moving wall needs bc_y = bounce-back");
    if (h->prm.ny < 3) return fail(h, LBM_ERR_ARG, "the moving wall needs ny >= 3");
    if (h->prm.bc_x == LBM_BC_BOUNCEBACK) return fail(h, LBM_ERR_ARG, "the moving wall needs periodic x");
    if (h->kernel != 1 && h->kernel != 5)
        return fail(h, LBM_ERR_ARG, "the moving wall runs on step kernels 1 and 5 (this lattice uses kernel %d)",
                    h->kernel);
    h->nee_top = true;
    h->uw_x = uw_x;
    h->uw_y = uw_y;
    return LBM_OK;
}

extern "C" lbm_status lbm_vanse_init_fields(lbm_vanse_t h, const double* rho, const double* ux, const double* uy,
                                            int on_device) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!rho || !ux || !uy) return fail(h, LBM_ERR_ARG, "rho, ux, uy must be non-NULL");
    if (!h->phi_set) return fail(h, LBM_ERR_STATE, "set the void fraction before init_fields");
    const long long n = (long long)h->prm.nx * h->prm.ny;
    double *dr, *dx, *dy;
    bool o1, o2, o3;
    lbm_status st = stage_in(h, rho, n, on_device, &dr, &o1);
    if (st != LBM_OK) return st;
    st = stage_in(h, ux, n, on_device, &dx, &o2);
    if (st != LBM_OK) return st;
    st = stage_in(h, uy, n, on_device, &dy, &o3);
    if (st != LBM_OK) return st;
    h->cur = 0;
    st = DISPATCH(h, run_init, dr, dx, dy);
    if (o1) cudaFreeAsync(dr, h->stream);
    if (o2) cudaFreeAsync(dx, h->stream);
    if (o3) cudaFreeAsync(dy, h->stream);
    if (st != LBM_OK) return st;
    h->initialised = true;
    h->steps = 0;
    return LBM_OK;
}

extern "C" lbm_status lbm_vanse_step(lbm_vanse_t h, int nsteps) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (nsteps < 0) return fail(h, LBM_ERR_ARG, "nsteps must be >= 0");
    if (!h->initialised) return fail(h, LBM_ERR_STATE, "init_fields or set_populations must come first");
    int left = nsteps;
    while (left > 0 && h->unsteady) {   // the step that consumes phi(t+1) runs on its own
        lbm_status st = DISPATCH(h, launch_step);
        if (st != LBM_OK) return st;
        --left;
    }
    while (h->use_graphs && left >= kGraphSteps) {
        lbm_status st = DISPATCH(h, replay_graph);
        if (st != LBM_OK) return st;
        left -= kGraphSteps;
    }
    while (left-- > 0) {
        lbm_status st = DISPATCH(h, launch_step);
        if (st != LBM_OK) return st;
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_vanse_macros(lbm_vanse_t h, double* rho, double* ux, double* uy, double* p, int on_device) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!h->initialised) return fail(h, LBM_ERR_STATE, "lattice not initialised");
    const long long n = (long long)h->prm.nx * h->prm.ny;
    lbm_status st = ensure_scratch(h);
    if (st != LBM_OK) return st;
    double* dr = (on_device && rho) ? rho : h->scratch;
    double* dx = (on_device && ux) ? ux : (ux ? h->scratch + n : nullptr);
    double* dy = (on_device && uy) ? uy : (uy ? h->scratch + 2 * n : nullptr);
    double* dp = (on_device && p) ? p : nullptr;
    st = DISPATCH(h, run_macros, dr, dx, dy, dp);
    if (st != LBM_OK) return st;
    if (!on_device) {
        if (rho) CK(h, cudaMemcpyAsync(rho, dr, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        if (ux) CK(h, cudaMemcpyAsync(ux, dx, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        if (uy) CK(h, cudaMemcpyAsync(uy, dy, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        if (p) {
            if (rho) { for (long long k = 0; k < n; ++k) p[k] = rho[k] / 3.0; }
            else {
                CK(h, cudaMemcpy(p, dr, n * sizeof(double), cudaMemcpyDeviceToHost));
                for (long long k = 0; k < n; ++k) p[k] /= 3.0;
            }
        }
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_vanse_get_populations(lbm_vanse_t h, double* f, int on_device) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!f) return fail(h, LBM_ERR_ARG, "f is NULL");
    if (!h->initialised) return fail(h, LBM_ERR_STATE, "lattice not initialised");
    const long long n9 = 9LL * h->prm.nx * h->prm.ny;
    double* d = f;
    if (!on_device) CK(h, cudaMallocAsync((void**)&d, n9 * sizeof(double), h->stream));
    lbm_status st = DISPATCH(h, run_get, d);
    if (st == LBM_OK && !on_device) {
        cudaError_t e = cudaMemcpyAsync(f, d, n9 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) st = cuda_fail(h, e, "copy populations to host");
    }
    if (!on_device) cudaFreeAsync(d, h->stream);
    return st;
}

extern "C" lbm_status lbm_vanse_set_populations(lbm_vanse_t h, const double* f, int on_device) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!f) return fail(h, LBM_ERR_ARG, "f is NULL");
    if (!h->phi_set) return fail(h, LBM_ERR_STATE, "set the void fraction before set_populations");
    const long long n9 = 9LL * h->prm.nx * h->prm.ny;
    double* d = nullptr;
    bool owned = false;
    lbm_status st = stage_in(h, f, n9, on_device, &d, &owned);
    if (st != LBM_OK) return st;
    h->cur = 0;
    st = DISPATCH(h, run_set, d);
    if (owned) cudaFreeAsync(d, h->stream);
    if (st != LBM_OK) return st;
    h->initialised = true;
    h->steps = 0;
    return LBM_OK;
}

// ============================================================ checkpoint / resume
namespace {

// A snapshot: this header (512 bytes) and then the raw device contents, in order: the
// current population buffer (9 planes with their padding and ghost columns, as
// stored), phi(t), phi(t+1) if pending, the force field if set.
struct StateHeader {
    char magic[8];
    int version, nx, ny, P, storage, kernel, has_solid;
    int unsteady, has_fb, has_drag, nee_top;
    long long plane, steps;
    unsigned step_ctr, pad0;
    double gx, gy, drag[4], uw[2];
    int dev_base, pad1;
};
static_assert(sizeof(StateHeader) <= 512, "state header");
constexpr size_t kStateHeader = 512;
constexpr char kStateMagic[8] = {'L', 'B', 'M', 'V', 'S', 'N', 'A', 'P'};

size_t state_bytes(const lbm_vanse* h) {
    const size_t pop = (size_t)h->npl * h->plane * h->sbytes, fld = (size_t)h->plane * h->rbytes;
    return kStateHeader + pop + fld * (1 + (h->unsteady ? 1 : 0) + (h->has_fb ? 2 : 0));
}

}  // namespace

extern "C" long long lbm_vanse_state_bytes(lbm_vanse_t h) { return h && h->initialised ? (long long)state_bytes(h) : -1; }

extern "C" lbm_status lbm_vanse_save_state(lbm_vanse_t h, void* buf, int on_device) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!buf) return fail(h, LBM_ERR_ARG, "buf is NULL");
    if (!h->initialised) return fail(h, LBM_ERR_STATE, "lattice not initialised");
    StateHeader hd{};
    std::memcpy(hd.magic, kStateMagic, 8);
    hd.version = 1;
    hd.nx = h->prm.nx; hd.ny = h->prm.ny; hd.P = h->P; hd.storage = h->prm.storage;
    hd.kernel = h->kernel; hd.has_solid = h->has_solid;
    hd.unsteady = h->unsteady; hd.has_fb = h->has_fb; hd.has_drag = h->has_drag; hd.nee_top = h->nee_top;
    hd.plane = h->plane; hd.steps = h->steps;
    hd.gx = h->gx; hd.gy = h->gy;
    hd.drag[0] = h->drag_d0; hd.drag[1] = h->drag_d1; hd.drag[2] = h->us_x; hd.drag[3] = h->us_y;
    hd.uw[0] = h->uw_x; hd.uw[1] = h->uw_y;
    hd.dev_base = h->jbase ? 1 : 0;
    CK(h, cudaMemcpyAsync(&hd.step_ctr, h->step_ctr, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    char* out = static_cast<char*>(buf);
    const cudaMemcpyKind hk = on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    const cudaMemcpyKind dk = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    char header[kStateHeader] = {};
    std::memcpy(header, &hd, sizeof(hd));
    CK(h, cudaMemcpyAsync(out, header, kStateHeader, hk, h->stream));
    size_t off = kStateHeader;
    const size_t pop = (size_t)h->npl * h->plane * h->sbytes, fld = (size_t)h->plane * h->rbytes;
    CK(h, cudaMemcpyAsync(out + off, h->f[h->cur], pop, dk, h->stream));
    off += pop;
    CK(h, cudaMemcpyAsync(out + off, h->phi, fld, dk, h->stream));
    off += fld;
    if (h->unsteady) { CK(h, cudaMemcpyAsync(out + off, h->phin, fld, dk, h->stream)); off += fld; }
    if (h->has_fb) CK(h, cudaMemcpyAsync(out + off, h->fb, 2 * fld, dk, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

extern "C" lbm_status lbm_vanse_load_state(lbm_vanse_t h, const void* buf, int on_device) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!buf) return fail(h, LBM_ERR_ARG, "buf is NULL");
    const char* in = static_cast<const char*>(buf);
    StateHeader hd{};
    CK(h, cudaMemcpy(&hd, in, sizeof(hd), on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
    if (std::memcmp(hd.magic, kStateMagic, 8) != 0 || hd.version != 1)
        return fail(h, LBM_ERR_ARG, "not a lattice state (bad magic or version)");
    if (hd.nx != h->prm.nx || hd.ny != h->prm.ny || hd.P != h->P || hd.storage != h->prm.storage ||
        hd.plane != h->plane || hd.has_solid != (int)h->has_solid || hd.dev_base != (h->jbase ? 1 : 0))
        return fail(h, LBM_ERR_ARG,
                    "the state is of another lattice (size %dx%d, storage %d, solid cells %d, deviation base %d)",
                    hd.nx, hd.ny, hd.storage, hd.has_solid, hd.dev_base);
    if (hd.nee_top && h->kernel != 1 && h->kernel != 5)
        return fail(h, LBM_ERR_ARG, "the state has a moving wall: kernel 1 or 5 needed");
    if (hd.has_fb && !h->fb) {
        CK(h, cudaMallocAsync(&h->fb, (size_t)2 * h->plane * h->rbytes, h->stream));
    }
    const cudaMemcpyKind dk = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    size_t off = kStateHeader;
    const size_t pop = (size_t)h->npl * h->plane * h->sbytes, fld = (size_t)h->plane * h->rbytes;
    CK(h, cudaMemcpyAsync(h->f[h->cur], in + off, pop, dk, h->stream));
    off += pop;
    CK(h, cudaMemcpyAsync(h->phi, in + off, fld, dk, h->stream));
    off += fld;
    if (hd.unsteady) { CK(h, cudaMemcpyAsync(h->phin, in + off, fld, dk, h->stream)); off += fld; }
    if (hd.has_fb) CK(h, cudaMemcpyAsync(h->fb, in + off, 2 * fld, dk, h->stream));
    CK(h, cudaMemcpyAsync(h->step_ctr, &hd.step_ctr, sizeof(unsigned), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->unsteady = hd.unsteady != 0;
    h->has_fb = hd.has_fb != 0;
    h->gx = hd.gx; h->gy = hd.gy;
    h->has_drag = hd.has_drag != 0;
    h->drag_d0 = hd.drag[0]; h->drag_d1 = hd.drag[1]; h->us_x = hd.drag[2]; h->us_y = hd.drag[3];
    h->nee_top = hd.nee_top != 0;
    h->uw_x = hd.uw[0]; h->uw_y = hd.uw[1];
    h->steps = hd.steps;
    h->phi_set = true;
    h->initialised = true;
    if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
    return update_solid_tiles(h);
}

extern "C" lbm_status lbm_vanse_reduce(lbm_vanse_t h, double* mass, double* momx, double* momy) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!h->initialised) return fail(h, LBM_ERR_STATE, "lattice not initialised");
    lbm_status st = DISPATCH(h, run_reduce);
    if (st != LBM_OK) return st;
    double r[3];
    CK(h, cudaMemcpyAsync(r, h->red_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (mass) *mass = r[0];
    if (momx) *momx = r[1];
    if (momy) *momy = r[2];
    if (!std::isfinite(r[0]) || !std::isfinite(r[1]) || !std::isfinite(r[2]))
        return fail(h, LBM_ERR_DIVERGED, "non-finite populations (mass %g)", r[0]);
    return LBM_OK;
}

extern "C" lbm_status lbm_vanse_step_sums(lbm_vanse_t h, double* out, int on_device) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!out) return fail(h, LBM_ERR_ARG, "out is NULL");
    if (!h->initialised) return fail(h, LBM_ERR_STATE, "init_fields or set_populations must come first");
    if (h->kernel != 1 && h->kernel != 5)
        return fail(h, LBM_ERR_ARG, "step sums need step kernel 1 or 5 (kernel %d)", h->kernel);
    CK(h, cudaMemsetAsync(h->red_out, 0, 3 * sizeof(double), h->stream));
    lbm_status st = DISPATCH(h, launch_step, h->red_out);
    if (st != LBM_OK) return st;
    CK(h, cudaMemcpyAsync(out, h->red_out, 3 * sizeof(double),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    return LBM_OK;
}

extern "C" lbm_status lbm_vanse_reduce_async(lbm_vanse_t h, double* out, int on_device) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!out) return fail(h, LBM_ERR_ARG, "out is NULL");
    if (!h->initialised) return fail(h, LBM_ERR_STATE, "lattice not initialised");
    lbm_status st = DISPATCH(h, run_reduce);
    if (st != LBM_OK) return st;
    CK(h, cudaMemcpyAsync(out, h->red_out, 3 * sizeof(double),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    return LBM_OK;
}

extern "C" lbm_status lbm_vanse_velocity_error(lbm_vanse_t h, const double* ux_ref, const double* uy_ref,
                                               int on_device, double* num, double* den) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!ux_ref || !uy_ref) return fail(h, LBM_ERR_ARG, "reference velocity is NULL");
    if (!h->initialised) return fail(h, LBM_ERR_STATE, "lattice not initialised");
    const long long n = (long long)h->prm.nx * h->prm.ny;
    lbm_status st = ensure_scratch(h);
    if (st != LBM_OK) return st;
    st = DISPATCH(h, run_macros, h->scratch, h->scratch + n, h->scratch + 2 * n, (double*)nullptr);
    if (st != LBM_OK) return st;
    double *rx, *ry;
    bool ox, oy;
    st = stage_in(h, ux_ref, n, on_device, &rx, &ox);
    if (st != LBM_OK) return st;
    st = stage_in(h, uy_ref, n, on_device, &ry, &oy);
    if (st != LBM_OK) return st;
    velocity_error_kernel<<<kReduceBlocks, kAuxThreads, 0, h->stream>>>(h->scratch + n, h->scratch + 2 * n, rx, ry, n,
                                                                         h->partial);
    CK(h, cudaGetLastError());
    finish_reduce_kernel<<<1, 1024, 0, h->stream>>>(h->partial, kReduceBlocks, h->red_out);
    CK(h, cudaGetLastError());
    double r[3];
    CK(h, cudaMemcpyAsync(r, h->red_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (ox) cudaFreeAsync(rx, h->stream);
    if (oy) cudaFreeAsync(ry, h->stream);
    if (num) *num = r[0];
    if (den) *den = r[1];
    return LBM_OK;
}

extern "C" lbm_status lbm_vanse_sync(lbm_vanse_t h) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    CK(h, cudaStreamSynchronize(h->stream));
    int flag = 0;
    CK(h, cudaMemcpy(&flag, h->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) return fail(h, LBM_ERR_TIMEOUT, "a step kernel gave up waiting for its staged rows");
    if (!h->has_solid) {
        CK(h, cudaMemcpy(&flag, h->zero_phi, sizeof(int), cudaMemcpyDeviceToHost));
        if (flag) return fail(h, LBM_ERR_ARG, "phi holds zeros: solid cells need lbm_vanse_set_solid_cells (kernels 1 and 5)");
    }
    return LBM_OK;
}

extern "C" long long lbm_vanse_step_count(lbm_vanse_t h) { return h ? h->steps : -1; }

extern "C" double lbm_vanse_bytes_per_cell(lbm_vanse_t h) {
    if (!h) return 0.0;
    double b = 2.0 * h->npl * h->sbytes + h->rbytes;  // 9 populations (+ J) read and written, phi(t)
    if (h->unsteady) b += h->rbytes;
    if (h->has_fb) b += 2.0 * h->rbytes;
    return b;
}

extern "C" lbm_status lbm_vanse_launch_shape(lbm_vanse_t h, int* threads, int* cols, int* rows, int* grid_x,
                                             int* grid_y, int* smem_bytes) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (threads) *threads = step_threads(h);
    if (cols) *cols = h->W;
    if (rows) *rows = h->H;
    if (grid_x) *grid_x = h->gridx;
    if (grid_y) *grid_y = h->gridy;
    if (smem_bytes) {
        const int nR = 1 + (h->unsteady ? 1 : 0) + (h->has_fb ? 2 : 0);
        size_t s = 0;
        switch (h->prm.storage) {
            case LBM_FP64: s = step_smem_bytes<double>(h, nR); break;
            case LBM_FP32: s = step_smem_bytes<float>(h, nR); break;
            case LBM_FP16: s = step_smem_bytes<__half>(h, nR); break;
            default: s = step_smem_bytes<__nv_bfloat16>(h, nR); break;
        }
        *smem_bytes = (int)s;
    }
    return LBM_OK;
}

extern "C" const char* lbm_vanse_last_error(lbm_vanse_t h) { return h ? h->msg.c_str() : g_create_error.c_str(); }

extern "C" void lbm_vanse_destroy(lbm_vanse_t h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->copy_stream) {
        cudaStreamSynchronize(h->copy_stream);
        cudaStreamDestroy(h->copy_stream);
        cudaEventDestroy(h->copy_done);
        cudaEventDestroy(h->staging_free);
    }
    void* ptrs[] = {h->f[0], h->f[1], h->phi, h->phin, h->fb, h->err, h->partial, h->red_out, h->scratch,
                    h->staging[0], h->staging[1], h->zero_phi, h->step_ctr, h->bad_phi, h->solid_tiles,
                    h->tile_order};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (h->bad_phi_host) cudaFreeHost(h->bad_phi_host);
    delete h;
}

// ============================================================================ batches

struct lbm_vanse_batch {
    lbm_vanse_batch_params prm;
    cudaStream_t stream = nullptr;
    int device = 0;
    int sbytes = 4;
    float scale = 1.f, inv_scale = 1.f;
    std::vector<lbm_vanse_batch_lattice> lat;
    std::vector<BatchLattice> desc;      // host copy of the device descriptors
    std::vector<size_t> offsets;         // byte offset of each lattice's two buffers
    void* pool = nullptr;                // every population buffer
    BatchLattice* d_desc = nullptr;
    int* d_units = nullptr;              // lattice of each unit
    int* d_clock = nullptr;              // [0] = t, [1] = unit counter, [2] = error flag
    double* scratch = nullptr;           // dense rho of the largest lattice
    double* partial = nullptr;
    double* red_out = nullptr;
    int nunits = 0, H = 0, grid = 0;
    int ghost_blocks = 1;                // x blocks of the ghost refresh (y = lattice)
    std::vector<int> H_each;             // strip height of each lattice launched on its own
    long long cells = 0, steps = 0;
    bool initialised = false;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::string msg;
};

namespace {

constexpr int kBatchMinBlocks = LBMV_WARP_MINB;
constexpr int kBatchGraphSteps = 16;

lbm_status bfail(lbm_vanse_batch* b, lbm_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (b) b->msg = buf; else g_create_error = buf;
    return st;
}

#define BCK(b, call)                                                                                      \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return bfail((b), e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, "%s: %s", #call, \
                         cudaGetErrorString(e_));                                                         \
    } while (0)

#define BDISPATCH(b, fn, ...)                                                    \
    ([&]() -> lbm_status {                                                       \
        switch ((b)->prm.storage) {                                              \
            case LBM_FP16: return fn<__half>((b), ##__VA_ARGS__);                \
            case LBM_BF16: return fn<__nv_bfloat16>((b), ##__VA_ARGS__);         \
            default: return fn<float>((b), ##__VA_ARGS__);                       \
        }                                                                        \
    }())

// Work units of height H for every lattice, largest lattices first.
lbm_status batch_decompose(lbm_vanse_batch* b, int H) {
    const int n = (int)b->lat.size();
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->lat[a].n > b->lat[c].n; });
    std::vector<int> units;
    for (int idx : order) {
        BatchLattice& L = b->desc[idx];
        L.H = std::min(H, L.ny);
        L.strips = (L.ny + L.H - 1) / L.H;
        L.unit0 = (int)units.size();
        for (int u = 0; u < L.tiles_x * L.strips; ++u) units.push_back(idx);
    }
    b->H = H;
    b->nunits = (int)units.size();
    if (b->d_units) cudaFree(b->d_units);
    b->d_units = nullptr;
    BCK(b, cudaMalloc((void**)&b->d_units, units.size() * sizeof(int)));
    BCK(b, cudaMemcpyAsync(b->d_units, units.data(), units.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaMemcpyAsync(b->d_desc, b->desc.data(), b->desc.size() * sizeof(BatchLattice), cudaMemcpyHostToDevice,
                           b->stream));
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    return LBM_OK;
}

BatchParams batch_params(const lbm_vanse_batch* b) {
    BatchParams bp;
    bp.lat = b->d_desc;
    bp.unit_lattice = b->d_units;
    bp.nunits = b->nunits;
    bp.counter = b->d_clock + 1;
    bp.clock = b->d_clock;
    bp.scale = b->scale;
    bp.inv_scale = b->inv_scale;
    bp.err = b->d_clock + 2;
    return bp;
}

template <typename S>
lbm_status batch_configure(lbm_vanse_batch* b) {
    const size_t smem = WarpLayout<S>::bytes(0);
    auto k1 = vanse_batch_kernel<S, kBatchMinBlocks>;
    auto k2 = vanse_batch_one_kernel<S, kBatchMinBlocks>;
    BCK(b, cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    BCK(b, cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    BCK(b, cudaFuncSetAttribute(k1, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared));
    BCK(b, cudaFuncSetAttribute(k2, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared));
    int per_sm = 0, nsm = 0;
    BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k1, 32, smem));
    BCK(b, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device));
    b->grid = std::max(1, per_sm * nsm);
    // launched on its own, a lattice gets the single-lattice rule: about five waves
    // of resident CTAs, strips of at least 16 rows
    b->H_each.resize(b->desc.size());
    for (size_t i = 0; i < b->desc.size(); ++i) {
        const BatchLattice& L = b->desc[i];
        const int nstrips = std::max(1, (5 * b->grid + L.tiles_x - 1) / L.tiles_x);
        b->H_each[i] = std::min(L.ny, std::max(16, (L.ny + nstrips - 1) / nstrips));
    }
    return LBM_OK;
}

template <typename S>
lbm_status batch_enqueue_step(lbm_vanse_batch* b, cudaStream_t stream) {
    const size_t smem = WarpLayout<S>::bytes(0);
    vanse_batch_kernel<S, kBatchMinBlocks><<<b->grid, 32, smem, stream>>>(batch_params(b));
    BCK(b, cudaGetLastError());
    batch_ghost_fill_kernel<S><<<dim3(b->ghost_blocks, (unsigned)b->desc.size()), 256, 0, stream>>>(b->d_desc, b->d_clock);
    BCK(b, cudaGetLastError());
    batch_tick_kernel<<<1, 1, 0, stream>>>(b->d_clock, b->d_clock + 1);
    BCK(b, cudaGetLastError());
    return LBM_OK;
}

template <typename S>
lbm_status batch_step_graph(lbm_vanse_batch* b) {
    if (!b->gexec) {
        if (!b->cap_stream) BCK(b, cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
        BCK(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        lbm_status st = LBM_OK;
        for (int k = 0; k < kBatchGraphSteps && st == LBM_OK; ++k) st = batch_enqueue_step<S>(b, b->cap_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
        if (st != LBM_OK) { if (g) cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { b->gexec = nullptr; return bfail(b, LBM_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e)); }
    }
    BCK(b, cudaGraphLaunch(b->gexec, b->stream));
    return LBM_OK;
}

template <typename S>
lbm_status batch_run(lbm_vanse_batch* b, int nsteps) {
    int left = nsteps;
    while (!b->prm.eager && left >= kBatchGraphSteps) {
        lbm_status st = batch_step_graph<S>(b);
        if (st != LBM_OK) return st;
        left -= kBatchGraphSteps;
        b->steps += kBatchGraphSteps;
    }
    while (left-- > 0) {
        lbm_status st = batch_enqueue_step<S>(b, b->stream);
        if (st != LBM_OK) return st;
        b->steps++;
    }
    return LBM_OK;
}

template <typename S>
lbm_status batch_run_each(lbm_vanse_batch* b, int nsteps) {
    const size_t smem = WarpLayout<S>::bytes(0);
    const BatchParams bp = batch_params(b);
    for (int s = 0; s < nsteps; ++s) {
        for (size_t i = 0; i < b->desc.size(); ++i) {
            const BatchLattice& L = b->desc[i];
            const int H = b->H_each[i], strips = (L.ny + H - 1) / H;
            vanse_batch_one_kernel<S, kBatchMinBlocks><<<L.tiles_x * strips, 32, smem, b->stream>>>(bp, (int)i, H);
            BCK(b, cudaGetLastError());
        }
        batch_ghost_fill_kernel<S><<<dim3(b->ghost_blocks, (unsigned)b->desc.size()), 256, 0, b->stream>>>(b->d_desc,
                                                                                                      b->d_clock);
        BCK(b, cudaGetLastError());
        batch_tick_kernel<<<1, 1, 0, b->stream>>>(b->d_clock, b->d_clock + 1);
        BCK(b, cudaGetLastError());
        b->steps++;
    }
    return LBM_OK;
}

template <typename S>
lbm_status batch_do_init(lbm_vanse_batch* b) {
    BCK(b, cudaMemsetAsync(b->d_clock, 0, 3 * sizeof(int), b->stream));
    for (size_t i = 0; i < b->desc.size(); ++i) {
        const long long n = (long long)b->desc[i].nx * b->desc[i].ny;
        batch_init_kernel<S><<<aux_blocks(n), kAuxThreads, 0, b->stream>>>(b->d_desc, (int)i, b->scale, b->inv_scale);
        BCK(b, cudaGetLastError());
    }
    b->steps = 0;
    b->initialised = true;
    return LBM_OK;
}

template <typename S>
lbm_status batch_do_error(lbm_vanse_batch* b, int index, double* out3) {
    const long long n = (long long)b->desc[index].nx * b->desc[index].ny;
    batch_rho_kernel<S><<<aux_blocks(n), kAuxThreads, 0, b->stream>>>(b->d_desc, index, b->d_clock, b->scratch,
                                                                       b->scale, b->inv_scale);
    BCK(b, cudaGetLastError());
    batch_err_kernel<S><<<kReduceBlocks, kAuxThreads, 0, b->stream>>>(b->d_desc, index, b->d_clock, b->scratch,
                                                                      b->partial, b->scale, b->inv_scale);
    BCK(b, cudaGetLastError());
    finish_reduce_kernel<<<1, 1024, 0, b->stream>>>(b->partial, kReduceBlocks, b->red_out);
    BCK(b, cudaGetLastError());
    BCK(b, cudaMemcpyAsync(out3, b->red_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

template <typename S>
lbm_status batch_do_get(lbm_vanse_batch* b, int index, double* dev_out) {
    const long long n = (long long)b->desc[index].nx * b->desc[index].ny;
    batch_get_kernel<S><<<aux_blocks(n), kAuxThreads, 0, b->stream>>>(b->d_desc, index, b->d_clock, dev_out, b->scale,
                                                                       b->inv_scale);
    BCK(b, cudaGetLastError());
    return LBM_OK;
}

}  // namespace

extern "C" void lbm_vanse_batch_default_params(lbm_vanse_batch_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->storage = LBM_FP32;
    p->s_e = 1.2;
    p->s_eps = 1.2;
    p->s_q = 1.2;
    p->kappa = 0.5;
    p->rho0 = 1.0;
    p->phi0 = 0.7;
    p->strip_rows = 0;
    p->eager = 0;
}

extern "C" lbm_status lbm_vanse_batch_create(const lbm_vanse_batch_lattice* lattices, int count,
                                             const lbm_vanse_batch_params* p, void* cuda_stream,
                                             lbm_vanse_batch_t* out) {
    if (!out) return bfail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!lattices || count < 1) return bfail(nullptr, LBM_ERR_ARG, "need at least one lattice");
    if (!p) return bfail(nullptr, LBM_ERR_ARG, "params is NULL");
    if (p->storage != LBM_FP32 && p->storage != LBM_FP16 && p->storage != LBM_BF16)
        return bfail(nullptr, LBM_ERR_ARG, "batches store FP32, FP16 or BF16 populations");
    if (!rate_ok(p->s_eps) || !rate_ok(p->s_q) || (p->s_e > 0 && !rate_ok(p->s_e)))
        return bfail(nullptr, LBM_ERR_ARG, "rates must lie in (0, 2)");
    if (!(p->kappa >= 0 && p->kappa <= 1) || !(p->rho0 > 0) || !(p->phi0 > 0 && p->phi0 <= 1))
        return bfail(nullptr, LBM_ERR_ARG, "bad kappa, rho0 or phi0");
    if (p->strip_rows < 0) return bfail(nullptr, LBM_ERR_ARG, "strip_rows must be >= 0");
    for (int i = 0; i < count; ++i) {
        const lbm_vanse_batch_lattice& q = lattices[i];
        if (q.n < 1 || q.n > 65536) return bfail(nullptr, LBM_ERR_ARG, "lattice %d: n = %d out of range", i, q.n);
        if (!(q.tau_nu > 0.5)) return bfail(nullptr, LBM_ERR_ARG, "lattice %d: tau_nu must exceed 1/2", i);
        if (!(q.period > 0)) return bfail(nullptr, LBM_ERR_ARG, "lattice %d: period must be positive", i);
        if (!(std::fabs(q.amplitude) < p->phi0)) return bfail(nullptr, LBM_ERR_ARG, "lattice %d: |A| must be < phi0", i);
    }
    lbm_vanse_batch* b = new lbm_vanse_batch();
    b->prm = *p;
    b->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&b->device);
    b->sbytes = storage_bytes(p->storage);
    if (p->storage == LBM_FP16) { b->scale = 65536.f; b->inv_scale = 1.f / 65536.f; }
    b->lat.assign(lattices, lattices + count);
    b->desc.resize(count);
    size_t total = 0;
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < count; ++i) {
        const lbm_vanse_batch_lattice& q = lattices[i];
        BatchLattice& L = b->desc[i];
        std::memset(&L, 0, sizeof(L));
        L.nx = L.ny = q.n;
        L.tiles_x = (q.n + 59) / 60;
        L.P = ((kPadCols + L.tiles_x * 60 + kPadCols) + 31) / 32 * 32;
        L.plane = (long long)L.ny * L.P;
        const double nu = (q.tau_nu - 0.5) / 3.0, s_nu = 1.0 / q.tau_nu;
        const double s_e = p->s_e > 0 ? p->s_e : 1.0 / (nu + 0.5);  // nu_e = nu/3
        L.s_e = (float)s_e; L.s_eps = (float)p->s_eps; L.s_q = (float)p->s_q; L.s_nu = (float)s_nu;
        L.h_e = (float)(1 - 0.5 * s_e); L.h_eps = (float)(1 - 0.5 * p->s_eps);
        L.h_q = (float)(1 - 0.5 * p->s_q); L.h_nu = (float)(1 - 0.5 * s_nu);
        L.kappa = (float)p->kappa; L.rho0 = (float)p->rho0;
        L.k = (float)(2 * pi / q.n); L.w = (float)(2 * pi / q.period);
        L.A = (float)q.amplitude; L.U0 = (float)q.u0; L.phi0 = (float)p->phi0; L.nu = (float)nu;
        const size_t bytes = ((size_t)9 * L.plane * b->sbytes + 255) / 256 * 256;
        b->offsets.push_back(total);
        total += 2 * bytes;
        b->cells += (long long)q.n * q.n;
    }
    lbm_status st = LBM_OK;
    cudaError_t e = cudaMalloc(&b->pool, total);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->pool, 0, total, b->stream);
    if (e != cudaSuccess) { st = bfail(nullptr, LBM_ERR_OOM, "batch populations (%zu bytes): %s", total, cudaGetErrorString(e)); }
    int nmax = 0;
    for (auto& q : b->lat) nmax = std::max(nmax, q.n);
    b->ghost_blocks = (int)std::min<long long>((9LL * nmax * 2 * kGhost + 255) / 256, 32);
    if (st == LBM_OK) {
        for (int i = 0; i < count; ++i) {
            const size_t bytes = ((size_t)9 * b->desc[i].plane * b->sbytes + 255) / 256 * 256;
            b->desc[i].buf[0] = (char*)b->pool + b->offsets[i];
            b->desc[i].buf[1] = (char*)b->pool + b->offsets[i] + bytes;
            for (int k = 0; k < 2 && st == LBM_OK; ++k) {
                const std::string err = encode_pop_map_raw(b->desc[i].buf[k], b->desc[i].P, b->desc[i].ny,
                                                           b->desc[i].plane, p->storage, &b->desc[i].map[k]);
                if (!err.empty()) st = bfail(nullptr, LBM_ERR_CUDA, "batch tensor maps: %s", err.c_str());
            }
        }
        e = cudaMalloc((void**)&b->d_desc, count * sizeof(BatchLattice));
        if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_clock, 4 * sizeof(int));
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_clock, 0, 4 * sizeof(int), b->stream);
        if (e == cudaSuccess) e = cudaMalloc((void**)&b->scratch, (size_t)nmax * nmax * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc((void**)&b->partial, kReduceBlocks * 3 * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc((void**)&b->red_out, 4 * sizeof(double));
        if (e != cudaSuccess) st = bfail(nullptr, LBM_ERR_OOM, "batch buffers: %s", cudaGetErrorString(e));
    }
    if (st == LBM_OK) st = BDISPATCH(b, batch_configure);
    if (st == LBM_OK) st = batch_decompose(b, p->strip_rows > 0 ? p->strip_rows : 48);
    if (st != LBM_OK) {
        if (b->msg.size()) g_create_error = b->msg;
        lbm_vanse_batch_destroy(b);
        return st;
    }
    *out = b;
    return LBM_OK;
}

extern "C" lbm_status lbm_vanse_batch_init(lbm_vanse_batch_t b) {
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "batch is NULL");
    return BDISPATCH(b, batch_do_init);
}

extern "C" lbm_status lbm_vanse_batch_step(lbm_vanse_batch_t b, int nsteps) {
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "batch is NULL");
    if (nsteps < 0) return bfail(b, LBM_ERR_ARG, "nsteps must be >= 0");
    if (!b->initialised) return bfail(b, LBM_ERR_STATE, "call lbm_vanse_batch_init first");
    return BDISPATCH(b, batch_run, nsteps);
}

extern "C" lbm_status lbm_vanse_batch_step_each(lbm_vanse_batch_t b, int nsteps) {
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "batch is NULL");
    if (nsteps < 0) return bfail(b, LBM_ERR_ARG, "nsteps must be >= 0");
    if (!b->initialised) return bfail(b, LBM_ERR_STATE, "call lbm_vanse_batch_init first");
    return BDISPATCH(b, batch_run_each, nsteps);
}

extern "C" lbm_status lbm_vanse_batch_autotune(lbm_vanse_batch_t b, int trial_steps, int* rows_out) {
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "batch is NULL");
    if (trial_steps < 1) return bfail(b, LBM_ERR_ARG, "trial_steps must be >= 1");
    static const int candidates[] = {16, 24, 32, 48, 64, 96, 128, 192, 256};
    cudaEvent_t e0, e1;
    BCK(b, cudaEventCreate(&e0));
    BCK(b, cudaEventCreate(&e1));
    int best = b->H;
    float best_ms = 1e30f;
    for (int H : candidates) {
        lbm_status st = batch_decompose(b, H);
        if (st == LBM_OK) st = lbm_vanse_batch_init(b);
        if (st == LBM_OK) st = lbm_vanse_batch_step(b, 2);  // warm-up (and graph capture)
        if (st != LBM_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return st; }
        BCK(b, cudaEventRecord(e0, b->stream));
        st = lbm_vanse_batch_step(b, trial_steps);
        if (st != LBM_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return st; }
        BCK(b, cudaEventRecord(e1, b->stream));
        BCK(b, cudaEventSynchronize(e1));
        float ms = 0.f;
        BCK(b, cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_ms) { best_ms = ms; best = H; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    lbm_status st = batch_decompose(b, best);
    if (st == LBM_OK) st = lbm_vanse_batch_init(b);
    if (st == LBM_OK && rows_out) *rows_out = best;
    return st;
}

extern "C" lbm_status lbm_vanse_batch_velocity_error(lbm_vanse_batch_t b, int index, double* num, double* den) {
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "batch is NULL");
    if (index < 0 || index >= (int)b->desc.size()) return bfail(b, LBM_ERR_ARG, "index %d out of range", index);
    if (!b->initialised) return bfail(b, LBM_ERR_STATE, "call lbm_vanse_batch_init first");
    double r[3];
    lbm_status st = BDISPATCH(b, batch_do_error, index, r);
    if (st != LBM_OK) return st;
    if (num) *num = r[0];
    if (den) *den = r[1];
    return LBM_OK;
}

extern "C" lbm_status lbm_vanse_batch_get_populations(lbm_vanse_batch_t b, int index, double* f, int on_device) {
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "batch is NULL");
    if (index < 0 || index >= (int)b->desc.size()) return bfail(b, LBM_ERR_ARG, "index %d out of range", index);
    if (!f) return bfail(b, LBM_ERR_ARG, "f is NULL");
    if (!b->initialised) return bfail(b, LBM_ERR_STATE, "call lbm_vanse_batch_init first");
    const long long n9 = 9LL * b->desc[index].nx * b->desc[index].ny;
    double* d = f;
    if (!on_device) BCK(b, cudaMallocAsync((void**)&d, n9 * sizeof(double), b->stream));
    lbm_status st = BDISPATCH(b, batch_do_get, index, d);
    if (st == LBM_OK && !on_device) {
        cudaError_t e = cudaMemcpyAsync(f, d, n9 * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) st = bfail(b, LBM_ERR_CUDA, "copy populations: %s", cudaGetErrorString(e));
    }
    if (!on_device) cudaFreeAsync(d, b->stream);
    return st;
}

extern "C" long long lbm_vanse_batch_cells(lbm_vanse_batch_t b) { return b ? b->cells : -1; }
extern "C" long long lbm_vanse_batch_step_count(lbm_vanse_batch_t b) { return b ? b->steps : -1; }
extern "C" const char* lbm_vanse_batch_last_error(lbm_vanse_batch_t b) {
    return b ? b->msg.c_str() : g_create_error.c_str();
}

extern "C" void lbm_vanse_batch_destroy(lbm_vanse_batch_t b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    void* ptrs[] = {b->pool, b->d_desc, b->d_units, b->d_clock, b->scratch, b->partial, b->red_out};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete b;
}

// ============================================================================ adjoint

namespace {

struct AdjBuffers {
    std::vector<void*> held;
    long long bytes = 0;
    void* host = nullptr;         // pinned host checkpoints
    long long host_bytes = 0;
    cudaStream_t st = nullptr;
    cudaError_t err = cudaSuccess;
    double* get(long long n) {
        void* q = nullptr;
        if (err == cudaSuccess) err = cudaMallocAsync(&q, (size_t)n * sizeof(double), st);
        if (err != cudaSuccess) return nullptr;
        held.push_back(q);
        bytes += n * (long long)sizeof(double);
        return (double*)q;
    }
    double* get_host(long long n) {
        if (err == cudaSuccess) err = cudaMallocHost(&host, (size_t)n * sizeof(double));
        if (err != cudaSuccess) { host = nullptr; return nullptr; }
        host_bytes = n * (long long)sizeof(double);
        return (double*)host;
    }
    ~AdjBuffers() {
        for (void* q : held) cudaFreeAsync(q, st);
        cudaStreamSynchronize(st);
        if (host) cudaFreeHost(host);
    }
};

struct AdjEvents {
    cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
    ~AdjEvents() {
        for (cudaEvent_t x : e)
            if (x) cudaEventDestroy(x);
    }
};

}  // namespace

extern "C" lbm_status lbm_vanse_outlet_momentum_grad(const lbm_vanse_params* p, const lbm_vanse_adjoint_params* a,
                                                     const double* phi, int on_device, void* cuda_stream, double* J,
                                                     double* dJdphi, lbm_vanse_adjoint_stats* stats) {
    if (!p || !a || !phi || !J) return fail(nullptr, LBM_ERR_ARG, "p, a, phi and J must not be NULL");
    if (p->nx < 1 || p->ny < 1 || p->nx > 65536 || p->ny > 65536) return fail(nullptr, LBM_ERR_ARG, "bad lattice size");
    if (!(p->tau_nu > 0.5)) return fail(nullptr, LBM_ERR_ARG, "tau_nu must exceed 1/2");
    if (!rate_ok(p->s_eps) || !rate_ok(p->s_q) || (p->s_e > 0 && !rate_ok(p->s_e)))
        return fail(nullptr, LBM_ERR_ARG, "rates must lie in (0, 2)");
    if (p->bc_x != LBM_BC_PERIODIC) return fail(nullptr, LBM_ERR_ARG, "bc_x must be periodic");
    if (p->eq_order == 2) return fail(nullptr, LBM_ERR_ARG, "the adjoint covers the Eq. (14) equilibrium only");
    if (a->nsteps < 1 || a->avg_steps < 1 || a->avg_steps > a->nsteps || a->checkpoint_every < 1)
        return fail(nullptr, LBM_ERR_ARG, "need nsteps >= 1, 1 <= avg_steps <= nsteps, checkpoint_every >= 1");
    if (a->x_out < 0 || a->x_out >= p->nx) return fail(nullptr, LBM_ERR_ARG, "x_out out of range");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const long long N = (long long)p->nx * p->ny, N9 = 9 * N;
    const double nu = (p->tau_nu - 0.5) / 3.0;
    adj::Params P;
    P.nx = p->nx;
    P.ny = p->ny;
    P.N = N;
    P.wall_y = p->bc_y == LBM_BC_BOUNCEBACK;
    P.model_b = p->model_b;
    P.kappa = p->kappa;
    P.gx = a->gx;
    P.gy = a->gy;
    P.s_e = p->s_e > 0 ? p->s_e : 1.0 / (nu + 0.5);   // nu_e = nu / 3
    P.s_eps = p->s_eps;
    P.s_q = p->s_q;
    P.s_nu = 1.0 / p->tau_nu;
    P.x_out = a->x_out;
    const int T = a->nsteps, M = a->avg_steps, K = a->checkpoint_every;
    const int nck = (T - 1) / K + 1;
    const bool want_grad = dJdphi != nullptr;
    // Two levels (dense_segments = 0): the checkpoints every K steps and, while a
    // segment is processed backwards, its states every K2 steps are kept in pinned host
    // memory; the device holds one sub-segment of K2 states. One level: checkpoints and
    // a whole segment of K states on the device.
    const bool dense = a->dense_segments != 0;
    const int K2 = dense ? std::min(K, T) : std::max(1, (int)std::ceil(std::sqrt((double)std::min(K, T))));
    const int nsub = (std::min(K, T) - 1) / K2 + 1;   // sub-checkpoints per segment

    AdjBuffers B;
    B.st = st;
    double* d_phi = B.get(N);
    double* fa = B.get(N9);
    double* fb = B.get(N9);
    double* ck = dense ? B.get((long long)nck * N9) : B.get_host((long long)(nck + (want_grad ? nsub : 0)) * N9);
    double* ck1 = dense ? nullptr : ck + (long long)nck * N9;   // host: a segment's sub-checkpoints
    adj::Fields F;
    F.s = B.get(N); F.rho = B.get(N); F.ux = B.get(N); F.uy = B.get(N); F.Fx = B.get(N); F.Fy = B.get(N);
    F.drx = B.get(N); F.dry = B.get(N); F.fld = B.get(6 * N);
    double* acc = B.get(1);
    double *seg = nullptr, *lam = nullptr, *lam2 = nullptr, *gphi = nullptr;
    adj::Adj A;
    if (want_grad) {
        seg = B.get((long long)K2 * N9);
        lam = B.get(N9);
        lam2 = B.get(N9);
        gphi = B.get(N);
        A.lm = B.get(N9);
        A.lux = B.get(N); A.luy = B.get(N); A.lFx = B.get(N); A.lFy = B.get(N); A.lrho = B.get(N);
        A.lg = B.get(8 * N);
        A.ldrx = B.get(N); A.ldry = B.get(N);
    }
    if (B.err != cudaSuccess)
        return fail(nullptr, B.err == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,
                    "adjoint buffers (%lld device bytes, %lld host bytes): %s", B.bytes, B.host_bytes,
                    cudaGetErrorString(B.err));
#define ACK(call)                                                                                              \
    do {                                                                                                       \
        cudaError_t e_ = (call);                                                                               \
        if (e_ != cudaSuccess) return fail(nullptr, LBM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
    } while (0)
    ACK(cudaMemcpyAsync(d_phi, phi, N * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    ACK(cudaMemsetAsync(acc, 0, sizeof(double), st));
    const int nb = aux_blocks(N), nt = kAuxThreads;
    AdjEvents ev;
    for (cudaEvent_t& x : ev.e) ACK(cudaEventCreate(&x));
    cudaEvent_t e0 = ev.e[0], e1 = ev.e[1], e2 = ev.e[2];
    ACK(cudaEventRecord(e0, st));
    auto fwd_fields = [&](const double* f) {
        adj::adj_fwd_rho<<<nb, nt, 0, st>>>(P, f, d_phi, F);
        adj::adj_fwd_u<<<nb, nt, 0, st>>>(P, f, d_phi, F);
    };
    auto fwd_step = [&](const double* f, double* fn) {
        fwd_fields(f);
        adj::adj_fwd_collide<<<nb, nt, 0, st>>>(P, f, d_phi, F, fn);
    };
    // forward: f(0), checkpoints every K steps, objective over the last M steps
    adj::adj_init_kernel<<<nb, nt, 0, st>>>(P, d_phi, fa);
    double *cur = fa, *nxt = fb;
    const cudaMemcpyKind to_ck = dense ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const cudaMemcpyKind from_ck = dense ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int n = 0; n < T; ++n) {
        if (n % K == 0) ACK(cudaMemcpyAsync(ck + (long long)(n / K) * N9, cur, N9 * sizeof(double), to_ck, st));
        fwd_step(cur, nxt);
        std::swap(cur, nxt);
        if (n + 1 > T - M) {
            fwd_fields(cur);
            adj::adj_objective<<<1, 256, 0, st>>>(P, cur, F, acc);
        }
    }
    ACK(cudaGetLastError());
    ACK(cudaEventRecord(e1, st));
    double Jsum = 0.0;
    ACK(cudaMemcpyAsync(&Jsum, acc, sizeof(double), cudaMemcpyDeviceToHost, st));
    const double wgt = 1.0 / ((double)M * p->ny);
    if (want_grad) {
        ACK(cudaMemsetAsync(gphi, 0, N * sizeof(double), st));
        // n = T: only the objective (lambda(T+1) = 0); cur holds f(T)
        fwd_fields(cur);
        adj::adj_bwd_collide<<<nb, nt, 0, st>>>(P, cur, d_phi, F, nullptr, A, gphi);
        adj::adj_bwd_u<<<nb, nt, 0, st>>>(P, cur, d_phi, F, A, wgt, gphi);
        adj::adj_bwd_rho<<<nb, nt, 0, st>>>(P, d_phi, F, A, lam, gphi);
        // backward over the steps m1 - 1 .. m0, whose states are seg[0 .. m1 - m0 - 1]
        auto backward = [&](int m0, int m1) {
            for (int n = m1 - 1; n >= m0; --n) {
                const double* fn = seg + (long long)(n - m0) * N9;
                fwd_fields(fn);
                adj::adj_bwd_collide<<<nb, nt, 0, st>>>(P, fn, d_phi, F, lam, A, gphi);
                adj::adj_bwd_u<<<nb, nt, 0, st>>>(P, fn, d_phi, F, A, n > T - M ? wgt : 0.0, gphi);
                adj::adj_bwd_rho<<<nb, nt, 0, st>>>(P, d_phi, F, A, lam2, gphi);
                std::swap(lam, lam2);
            }
        };
        for (int k = nck - 1; k >= 0; --k) {
            const int n0 = k * K, n1 = std::min(n0 + K, T);
            if (dense) {
                ACK(cudaMemcpyAsync(seg, ck + (long long)k * N9, N9 * sizeof(double), from_ck, st));
                for (int j = 1; j < n1 - n0; ++j) fwd_step(seg + (long long)(j - 1) * N9, seg + (long long)j * N9);
                backward(n0, n1);
                continue;
            }
            // the segment's states every K2 steps to the host (fa, fb: the running state)
            const int ns = (n1 - n0 - 1) / K2 + 1;
            ACK(cudaMemcpyAsync(fa, ck + (long long)k * N9, N9 * sizeof(double), from_ck, st));
            double *c0 = fa, *c1 = fb;
            for (int j = 0; j < ns; ++j) {
                ACK(cudaMemcpyAsync(ck1 + (long long)j * N9, c0, N9 * sizeof(double), cudaMemcpyDeviceToHost, st));
                if (j + 1 < ns)
                    for (int i = 0; i < K2; ++i) { fwd_step(c0, c1); std::swap(c0, c1); }
            }
            for (int j = ns - 1; j >= 0; --j) {
                const int m0 = n0 + j * K2, m1 = std::min(m0 + K2, n1);
                ACK(cudaMemcpyAsync(seg, ck1 + (long long)j * N9, N9 * sizeof(double), cudaMemcpyHostToDevice, st));
                for (int i = 1; i < m1 - m0; ++i) fwd_step(seg + (long long)(i - 1) * N9, seg + (long long)i * N9);
                backward(m0, m1);
            }
        }
        adj::adj_bwd_init<<<nb, nt, 0, st>>>(P, lam, gphi);
        ACK(cudaGetLastError());
        ACK(cudaMemcpyAsync(dJdphi, gphi, N * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    }
    ACK(cudaEventRecord(e2, st));
    ACK(cudaStreamSynchronize(st));
    *J = Jsum * wgt;
    if (stats) {
        float f_ms = 0.f, b_ms = 0.f;
        cudaEventElapsedTime(&f_ms, e0, e1);
        cudaEventElapsedTime(&b_ms, e1, e2);
        stats->forward_ms = f_ms;
        stats->backward_ms = want_grad ? b_ms : 0.0;
        stats->device_bytes = B.bytes;
        stats->host_bytes = B.host_bytes;
    }
#undef ACK
    return LBM_OK;
}
