// drt_k_batch_gen.cu -- stage 4 of a batch plan for the chains of the generic range (several
// diffractions in a segment, 4 vertices, or any chain of a batch that writes per-path-step records),
// values only; the form with rates (Doppler output) is in drt_k_batch_gen_dual.cu.
#include "drt_batch_unit.cuh"

namespace drt {

cudaError_t launch_batch_bulk_gen_dual(const BatchDev &B, int grid, cudaStream_t s);

cudaError_t launch_batch_bulk_gen(bool dual, const BatchDev &B, int grid, cudaStream_t s) {
    if (dual) return launch_batch_bulk_gen_dual(B, grid, s);
    k_batch_bulk<-1, false, false><<<grid, 128, 0, s>>>(B);
    return cudaGetLastError();
}

}  // namespace drt
