// vanse_warp_solid.cu -- the one-warp step kernel with solid cells (phi = 0: the
// impermeable block of Sec. 3.3, half-way bounce-back links and the neighbour-by-
// neighbour Eq. (10) stencil next to them; vanse_warp.cuh), in a translation unit of
// its own so that its twelve instances compile in parallel with the rest of the library.
#include "vanse_warp.cuh"

namespace lbmv {

template <typename S>
cudaError_t warp_solid_configure(size_t smem_max) {
    for (const void* k : {(const void*)vanse_warp_kernel<S, LBMV_WARP_MINB, false, false, true>,
                          (const void*)vanse_warp_kernel<S, LBMV_WARP_MINB, true, false, true>,
                          (const void*)vanse_warp_kernel<S, LBMV_WARP_MINB, false, true, true>,
                          (const void*)vanse_warp_kernel<S, LBMV_WARP_MINB, true, true, true>}) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename S>
cudaError_t warp_solid_launch(const StepParams<float>& p, dim3 grid, size_t smem, cudaStream_t stream, bool sums,
                              bool eq2) {
    if (sums) {
        if (eq2) vanse_warp_kernel<S, LBMV_WARP_MINB, true, true, true><<<grid, 32, smem, stream>>>(p);
        else vanse_warp_kernel<S, LBMV_WARP_MINB, true, false, true><<<grid, 32, smem, stream>>>(p);
    } else {
        if (eq2) vanse_warp_kernel<S, LBMV_WARP_MINB, false, true, true><<<grid, 32, smem, stream>>>(p);
        else vanse_warp_kernel<S, LBMV_WARP_MINB, false, false, true><<<grid, 32, smem, stream>>>(p);
    }
    return cudaGetLastError();
}

template cudaError_t warp_solid_configure<float>(size_t);
template cudaError_t warp_solid_configure<__half>(size_t);
template cudaError_t warp_solid_configure<__nv_bfloat16>(size_t);
template cudaError_t warp_solid_launch<float>(const StepParams<float>&, dim3, size_t, cudaStream_t, bool, bool);
template cudaError_t warp_solid_launch<__half>(const StepParams<float>&, dim3, size_t, cudaStream_t, bool, bool);
template cudaError_t warp_solid_launch<__nv_bfloat16>(const StepParams<float>&, dim3, size_t, cudaStream_t, bool,
                                                      bool);

}  // namespace lbmv
