// drt_k_batch_gen_dual.cu -- stage 4 of a batch plan for the chains of the generic range, carrying the
// rates the Doppler output needs (delta numbers with time derivatives).
#include "drt_batch_unit.cuh"

namespace drt {

cudaError_t launch_batch_bulk_gen_dual(const BatchDev &B, int grid, cudaStream_t s) {
    k_batch_bulk<-1, true, false><<<grid, 128, 0, s>>>(B);
    return cudaGetLastError();
}

}  // namespace drt
