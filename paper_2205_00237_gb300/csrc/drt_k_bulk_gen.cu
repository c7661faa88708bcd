// drt_k_bulk_gen.cu -- the FP32-bulk kernel for the generic range of chains (several diffractions in a
// segment, or 4 vertices): per block one path, the chain length selecting an instance compiled for it.
#include <type_traits>

#include "drt_launch.cuh"

namespace drt {

// the generic range (several diffractions in a segment, 4 vertices; every chain when records are
// asked for): each path runs the instance compiled for its chain length
template <bool DUAL>
__global__ void __launch_bounds__(EXT_T, 4)
k_extrapolate_bulk_gen(const LinkDev L, const TimeGridD tg, const FreqGridD fg, const PoseB *__restrict__ poseb,
                       const BaseRec *__restrict__ base, const double *__restrict__ warm, const OutD out,
                       const RecD rec, const RedoList redo, int p0, int p1) {
    const int p = p0 + blockIdx.y;
    const int ti = blockIdx.x * EXT_T + threadIdx.x;
    if (p >= p1 || ti >= tg.n_steps) return;
    const BulkRows R = bulk_rows_global(L, poseb, base, nullptr, (tg.n_steps + tg.chunk - 1) / tg.chunk, p);
    typedef std::conditional_t<DUAL, dd, de> S;
    path_step_bulk<LEN_GEN, true, true, S>(L, tg, fg, R, warm, p, ti, out, rec, redo);
}

cudaError_t launch_extrapolate_bulk_generic(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, const PoseB *pb,
                                            const BaseRec *bs, const double *warm, const OutD &out, const RecD &rec,
                                            const RedoList &rl, cudaStream_t s) {
    const int tx = (tg.n_steps + EXT_T - 1) / EXT_T;
    const bool outs = any_output(out), dual = out.doppler != nullptr;
    return for_generic_ranges(L, 0, L.n_paths, !outs, [&](int kind, int a, int b) {
        const dim3 grid(tx, b - a);
        if (kind == 2) k_extrapolate_bulk_n<2, true><<<grid, EXT_T, 0, s>>>(L, tg, fg, pb, bs, warm, out, rec, rl, a, b);
        else if (kind == 3) k_extrapolate_bulk_n<3, true><<<grid, EXT_T, 0, s>>>(L, tg, fg, pb, bs, warm, out, rec, rl, a, b);
        else if (dual) k_extrapolate_bulk_gen<true><<<grid, EXT_T, 0, s>>>(L, tg, fg, pb, bs, warm, out, rec, rl, a, b);
        else k_extrapolate_bulk_gen<false><<<grid, EXT_T, 0, s>>>(L, tg, fg, pb, bs, warm, out, rec, rl, a, b);
        return cudaGetLastError();
    });
}

}  // namespace drt
