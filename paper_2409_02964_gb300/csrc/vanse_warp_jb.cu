// vanse_warp_jb.cu -- the one-warp step kernel with FP16 / BF16 deviations from the
// momentum base (vanse_warp.cuh, JB): each slot is stored against f_i^rest plus the
// linear term 3 w_i e_i . J of Eq. (14) with J the cell's post-collision momentum,
// which the buffer holds in two more planes. A translation unit of its own, so that
// its eight instances compile in parallel with the rest of the library.
#include "vanse_warp.cuh"

namespace lbmv {

template <typename S>
cudaError_t warp_jb_configure(size_t smem_max) {
    for (const void* k : {(const void*)vanse_warp_kernel<S, LBMV_WARP_MINB, false, false, false, true>,
                          (const void*)vanse_warp_kernel<S, LBMV_WARP_MINB, true, false, false, true>,
                          (const void*)vanse_warp_kernel<S, LBMV_WARP_MINB, false, true, false, true>,
                          (const void*)vanse_warp_kernel<S, LBMV_WARP_MINB, true, true, false, true>}) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename S>
cudaError_t warp_jb_launch(const StepParams<float>& p, dim3 grid, size_t smem, cudaStream_t stream, bool sums,
                           bool eq2) {
    if (sums) {
        if (eq2) vanse_warp_kernel<S, LBMV_WARP_MINB, true, true, false, true><<<grid, 32, smem, stream>>>(p);
        else vanse_warp_kernel<S, LBMV_WARP_MINB, true, false, false, true><<<grid, 32, smem, stream>>>(p);
    } else {
        if (eq2) vanse_warp_kernel<S, LBMV_WARP_MINB, false, true, false, true><<<grid, 32, smem, stream>>>(p);
        else vanse_warp_kernel<S, LBMV_WARP_MINB, false, false, false, true><<<grid, 32, smem, stream>>>(p);
    }
    return cudaGetLastError();
}

template <typename S>
const void* warp_jb_kernel() {
    return (const void*)vanse_warp_kernel<S, LBMV_WARP_MINB, false, false, false, true>;
}

template cudaError_t warp_jb_configure<__half>(size_t);
template cudaError_t warp_jb_configure<__nv_bfloat16>(size_t);
template cudaError_t warp_jb_launch<__half>(const StepParams<float>&, dim3, size_t, cudaStream_t, bool, bool);
template cudaError_t warp_jb_launch<__nv_bfloat16>(const StepParams<float>&, dim3, size_t, cudaStream_t, bool,
                                                   bool);
template const void* warp_jb_kernel<__half>();
template const void* warp_jb_kernel<__nv_bfloat16>();

}  // namespace lbmv
