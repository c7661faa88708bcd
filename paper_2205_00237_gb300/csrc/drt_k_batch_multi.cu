// drt_k_batch_multi.cu -- stage 4 of a batch plan for the multi-diffraction chains of 2 and 3 vertices:
// code compiled for the chain length (the Newton state in registers), carrier pairs as for the other
// lengths.
#include "drt_batch_unit.cuh"

namespace drt {

cudaError_t launch_batch_bulk_multi(int N, bool pair, const BatchDev &B, int grid, cudaStream_t s) {
    if (N == 2) {
        if (pair) k_batch_bulk<2, false, true, true><<<grid, 128, 0, s>>>(B);
        else k_batch_bulk<2, false, false, true><<<grid, 128, 0, s>>>(B);
    } else {
        if (pair) k_batch_bulk<3, false, true, true><<<grid, 128, 0, s>>>(B);
        else k_batch_bulk<3, false, false, true><<<grid, 128, 0, s>>>(B);
    }
    return cudaGetLastError();
}

}  // namespace drt
