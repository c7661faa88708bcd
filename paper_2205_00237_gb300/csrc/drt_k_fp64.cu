// drt_k_fp64.cu -- a3-a8 in FP64: the per-(path, time-step) extrapolation kernels of the FP64 form and
// the warm starts of the multi-diffraction chains.
//
// A block covers 128 consecutive time steps of ONE path, so every lane of a warp runs the same chain
// signature (no type divergence); branches that remain (validity, Newton iteration counts,
// transition-function ranges) are correlated between neighbouring instants.  Chains with at most one
// diffraction between point sources run code unrolled for their length (paths of one length are
// contiguous after the signature sort, so each length is one launch with its own register budget);
// chains with several diffractions in a segment, and the rare 4-vertex chains (the generic range), run
// in launches of their own (drt_k_fp64_gen.cu), so the Newton solver costs the common chains nothing.
#include <algorithm>

#include "drt_launch.cuh"

namespace drt {

// user outputs (with or without Doppler): lengths 0..3 in one launch, chosen per block
template <bool DUAL>
__global__ void __launch_bounds__(EXT_T)
k_extrapolate_fp64_out(const LinkDev L, const TimeGridD tg, const FreqGridD fg, const double *__restrict__ pose,
                       const OutD out, const RecD rec, int p0, int p1, int f32out, const double *__restrict__ warm) {
    const int p = p0 + blockIdx.x;
    const int ti = blockIdx.y * EXT_T + threadIdx.x;
    if (p >= p1 || ti >= tg.n_steps) return;
    const bool f32 = f32out != 0;
    switch (chain_length(L, p)) {
    case 0: path_step_fp64<DUAL, 0, false, true>(L, tg, fg, pose, p, ti, out, rec, f32, warm); break;
    case 1: path_step_fp64<DUAL, 1, false, true>(L, tg, fg, pose, p, ti, out, rec, f32, warm); break;
    case 2: path_step_fp64<DUAL, 2, false, true>(L, tg, fg, pose, p, ti, out, rec, f32, warm); break;
    default: path_step_fp64<DUAL, 3, false, true>(L, tg, fg, pose, p, ti, out, rec, f32, warm); break;
    }
}

cudaError_t launch_extrapolate_fp64(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg,
                                    const double *pose, const OutD &out, const RecD &rec, cudaStream_t s, int p0,
                                    int p1, bool f32out, double *warm, cudaStream_t s_multi) {
    if (p1 < 0) p1 = L.n_paths;
    if (p1 <= p0 || tg.n_steps == 0) return cudaSuccess;
    const int f32 = f32out ? 1 : 0, ty = (tg.n_steps + EXT_T - 1) / EXT_T;
    const bool outs = any_output(out);
    // unrolled lengths 0..3 over [p0, p1) clipped to their ranges
    if (!outs) {
        for (int n = 0; n < MAXI; ++n) {
            const int a = std::max(p0, L.len_start[n]), b = std::min(p1, L.len_start[n + 1]);
            if (b <= a) continue;
            const dim3 grid(b - a, ty);
            switch (n) {
            case 0: k_extrapolate_fp64_n<0><<<grid, EXT_T, 0, s>>>(L, tg, fg, pose, out, rec, a, b, f32, warm); break;
            case 1: k_extrapolate_fp64_n<1><<<grid, EXT_T, 0, s>>>(L, tg, fg, pose, out, rec, a, b, f32, warm); break;
            case 2: k_extrapolate_fp64_n<2><<<grid, EXT_T, 0, s>>>(L, tg, fg, pose, out, rec, a, b, f32, warm); break;
            default: k_extrapolate_fp64_n<3><<<grid, EXT_T, 0, s>>>(L, tg, fg, pose, out, rec, a, b, f32, warm); break;
            }
            if (cudaError_t e = cudaGetLastError()) return e;
        }
    } else {
        const int a = p0, b = std::min(p1, L.len_start[MAXI]);
        if (b > a) {
            const dim3 grid(b - a, ty);
            // the Doppler shift needs the interaction points' velocities (dual numbers); nothing else does
            if (out.doppler) k_extrapolate_fp64_out<true><<<grid, EXT_T, 0, s>>>(L, tg, fg, pose, out, rec, a, b, f32, warm);
            else k_extrapolate_fp64_out<false><<<grid, EXT_T, 0, s>>>(L, tg, fg, pose, out, rec, a, b, f32, warm);
            if (cudaError_t e = cudaGetLastError()) return e;
        }
    }
    return launch_extrapolate_fp64_generic(L, tg, fg, pose, out, rec, p0, p1, f32, warm, s_multi ? s_multi : s);
}

}  // namespace drt
