// drt_k_redo_out.cu -- the FP64 redo of the FP32-bulk path-steps that FP32 cannot resolve, written in
// place into the caller's per-path-step outputs and records.
#include "drt_launch.cuh"

namespace drt {

// FP64 redo of the queued path-steps: a fixed grid strides over the device-side count, one warp per
// block (the few queued steps spread over all SMs; each is a long FP64 chain), grid row y taking the
// chains of length y (one code instance per length: a warp runs one of them)
template <bool DUAL>
__global__ void __launch_bounds__(32)
k_redo(const LinkDev L, const TimeGridD tg, const FreqGridD fg, const OutD out, const RecD rec, const RedoList redo,
       const double *__restrict__ warm) {
    int n = min(*redo.count, redo.cap);
    const int warp = blockIdx.y * gridDim.x + blockIdx.x;
    if (n <= (int)(gridDim.x * gridDim.y)) {   // few queued steps: one per warp (see k_redo_rec)
        if (threadIdx.x == 0 && warp < n) {
            const int4 it = redo.items[warp];
            if constexpr (DUAL) path_step_redo_as<true>(L, tg, fg, it.y, it.z, out, rec, warm);
            else path_step_redo_as<false>(L, tg, fg, it.y, it.z, out, rec, warm);
        }
        return;
    }
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int4 it = redo.items[k];
        if (chain_length(L, it.y) != (int)blockIdx.y) continue;
        if constexpr (DUAL) path_step_redo_as<true>(L, tg, fg, it.y, it.z, out, rec, warm);
        else path_step_redo_as<false>(L, tg, fg, it.y, it.z, out, rec, warm);
    }
}

cudaError_t launch_redo(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, const OutD &out, const RecD &rec,
                        void *redo, const double *warm, cudaStream_t s) {
    if (L.n_paths == 0 || tg.n_steps == 0) return cudaSuccess;
    const dim3 grid(152 * 4, MAXI + 1);
    if (out.doppler) k_redo<true><<<grid, 32, 0, s>>>(L, tg, fg, out, rec, redo_list(redo, L, tg), warm);
    else k_redo<false><<<grid, 32, 0, s>>>(L, tg, fg, out, rec, redo_list(redo, L, tg), warm);
    return cudaGetLastError();
}

}  // namespace drt
