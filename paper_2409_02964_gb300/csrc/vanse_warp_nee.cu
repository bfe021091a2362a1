// vanse_warp_nee.cu -- the one-warp step kernel with the moving wall's code (row
// ny-1 by non-equilibrium extrapolation, Sec. 3.1; vanse_warp.cuh, NEE): lattices
// with a moving wall launch these instances, the others the ones without that code,
// whose general row path it would slow. A translation unit of its own, so that its
// twelve instances compile in parallel with the rest of the library.
#include "vanse_warp.cuh"

namespace lbmv {

template <typename S>
cudaError_t warp_nee_configure(size_t smem_max) {
    for (const void* k : {(const void*)vanse_warp_kernel<S, LBMV_WARP_MINB, false, false, false, false, true>,
                          (const void*)vanse_warp_kernel<S, LBMV_WARP_MINB, true, false, false, false, true>,
                          (const void*)vanse_warp_kernel<S, LBMV_WARP_MINB, false, true, false, false, true>,
                          (const void*)vanse_warp_kernel<S, LBMV_WARP_MINB, true, true, false, false, true>}) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename S>
cudaError_t warp_nee_launch(const StepParams<float>& p, dim3 grid, size_t smem, cudaStream_t stream, bool sums,
                            bool eq2) {
    if (sums) {
        if (eq2) vanse_warp_kernel<S, LBMV_WARP_MINB, true, true, false, false, true><<<grid, 32, smem, stream>>>(p);
        else vanse_warp_kernel<S, LBMV_WARP_MINB, true, false, false, false, true><<<grid, 32, smem, stream>>>(p);
    } else {
        if (eq2) vanse_warp_kernel<S, LBMV_WARP_MINB, false, true, false, false, true><<<grid, 32, smem, stream>>>(p);
        else vanse_warp_kernel<S, LBMV_WARP_MINB, false, false, false, false, true><<<grid, 32, smem, stream>>>(p);
    }
    return cudaGetLastError();
}

template cudaError_t warp_nee_configure<float>(size_t);
template cudaError_t warp_nee_configure<__half>(size_t);
template cudaError_t warp_nee_configure<__nv_bfloat16>(size_t);
template cudaError_t warp_nee_launch<float>(const StepParams<float>&, dim3, size_t, cudaStream_t, bool, bool);
template cudaError_t warp_nee_launch<__half>(const StepParams<float>&, dim3, size_t, cudaStream_t, bool, bool);
template cudaError_t warp_nee_launch<__nv_bfloat16>(const StepParams<float>&, dim3, size_t, cudaStream_t, bool,
                                                    bool);

}  // namespace lbmv
