// drt_k_batch.cu -- stage 4 of a batch plan (drt_batch.cu): the FP32-bulk extrapolation of every
// (link, path, 32 consecutive steps) unit of a wave, one warp per unit claimed from an atomic counter.
//
// The lanes of a unit share the chain signature.  Chains of up to 3 vertices with at most one
// diffraction between point sources run code unrolled for their length, one persistent launch per
// length (the signature sort makes each length a contiguous path range of its link, so each length
// has its own unit range) with the register budget of that length; the other chains (several
// diffractions in a segment, 4 vertices) and batches that write per-path-step records run the generic
// code.  A carrier pair (two entries of one link over one time grid) evaluates the geometry of its
// chains of 2 and 3 vertices and of its generic range once, with the coefficients and records of both
// carriers (PAIR instantiations, or a run-time branch in the generic code); the line of sight and the
// single interactions, whose geometry is a few posed points, run per carrier.
#include "drt_batch_unit.cuh"

namespace drt {

int batch_bulk_blocks(int N, bool multi) {
    if (multi) return N == 2 ? BatchBlocks<2, true>::v : BatchBlocks<3, true>::v;
    return N < 0 ? BatchBlocks<-1>::v : N <= 1 ? BatchBlocks<1>::v : N == 2 ? BatchBlocks<2>::v : BatchBlocks<3>::v;
}

cudaError_t launch_batch_bulk(int N, bool dual, bool pair, const BatchDev &B, int grid, cudaStream_t s) {
    if (N < 0) return launch_batch_bulk_gen(dual, B, grid, s);
    if (pair && N >= 2) {   // lengths 0 and 1 are never paired (see the planner)
        if (N == 2) k_batch_bulk<2, false, true><<<grid, 128, 0, s>>>(B);
        else k_batch_bulk<3, false, true><<<grid, 128, 0, s>>>(B);
    } else {
        switch (N) {
        case 0: k_batch_bulk<0, false, false><<<grid, 128, 0, s>>>(B); break;
        case 1: k_batch_bulk<1, false, false><<<grid, 128, 0, s>>>(B); break;
        case 2: k_batch_bulk<2, false, false><<<grid, 128, 0, s>>>(B); break;
        default: k_batch_bulk<3, false, false><<<grid, 128, 0, s>>>(B); break;
        }
    }
    return cudaGetLastError();
}

}  // namespace drt
