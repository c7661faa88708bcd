// drt_k_fp64.cu -- a3-a8 in FP64: the per-(path, time-step) extrapolation kernels of the FP64 form and
// the warm starts of the multi-diffraction chains.
//
// A block covers 128 consecutive time steps of ONE path, so every lane of a warp runs the same chain
// signature (no type divergence); branches that remain (validity, Newton iteration counts,
// transition-function ranges) are correlated between neighbouring instants.  Chains with at most one
// diffraction between point sources run code unrolled for their length (paths of one length are
// contiguous after the signature sort, so each length is one launch with its own register budget);
// chains with several diffractions in a segment, and the rare 4-vertex chains, run the generic code
// in a launch of their own, so its Newton solver and dynamically indexed arrays cost the common chains
// nothing.
#include <algorithm>

#include "drt_launch.cuh"

namespace drt {

// the H-synthesis path (values, no user outputs), one chain length N per launch
template <int N>
__global__ void __launch_bounds__(EXT_T)
k_extrapolate_fp64_n(const LinkDev L, const TimeGridD tg, const FreqGridD fg, const double *__restrict__ pose,
                     const OutD out, const RecD rec, int p0, int p1, int f32out, const double *__restrict__ warm) {
    const int p = p0 + blockIdx.x;
    const int ti = blockIdx.y * EXT_T + threadIdx.x;
    if (p >= p1 || ti >= tg.n_steps) return;
    path_step_fp64<false, N, false, false>(L, tg, fg, pose, p, ti, out, rec, f32out != 0, warm);
}

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

// any chain (several diffractions in a segment, 4 vertices), generic code
template <bool DUAL>
__global__ void __launch_bounds__(EXT_T)
k_extrapolate_fp64_gen(const LinkDev L, const TimeGridD tg, const FreqGridD fg, const double *__restrict__ pose,
                       const OutD out, const RecD rec, int p0, int p1, int f32out, const double *__restrict__ warm) {
    const int p = p0 + blockIdx.x;
    const int ti = blockIdx.y * EXT_T + threadIdx.x;
    if (p >= p1 || ti >= tg.n_steps) return;
    path_step_fp64<DUAL, -1, true, true>(L, tg, fg, pose, p, ti, out, rec, f32out != 0, warm);
}

// warm-start pre-pass over (multi-diffraction path, chunk)
constexpr int WARM_T = 32;
__global__ void __launch_bounds__(WARM_T)
k_warm_fp64(const LinkDev L, const TimeGridD tg, double *__restrict__ warm) {
    int p = L.n_bulk + blockIdx.x;
    int c = blockIdx.y * WARM_T + threadIdx.x;
    if (p >= L.n_paths || c > n_chunks_of(tg)) return;   // rows 0..n_chunks
    path_warm_fp64(L, tg, p, c, warm);
}

__global__ void __launch_bounds__(32) k_t0par(const LinkDev L, double *__restrict__ t0par) {
    const int p = L.n_bulk + blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= L.n_paths) return;
    path_t0par_fp64(L, p, t0par + (size_t)(p - L.n_bulk) * (2 * MAXI));
}

cudaError_t launch_t0par(const LinkDev &L, double *t0par, cudaStream_t s) {
    const int n = L.n_paths - L.n_bulk;
    if (n <= 0) return cudaSuccess;
    k_t0par<<<(n + 31) / 32, 32, 0, s>>>(L, t0par);
    return cudaGetLastError();
}

cudaError_t launch_warm_fp64(const LinkDev &L, const TimeGridD &tg, double *warm, cudaStream_t s) {
    if (!warm || L.n_bulk >= L.n_paths || tg.n_steps == 0) return cudaSuccess;
    dim3 gw(L.n_paths - L.n_bulk, (n_chunks_of(tg) + 1 + WARM_T - 1) / WARM_T);
    k_warm_fp64<<<gw, WARM_T, 0, s>>>(L, tg, warm);
    return cudaGetLastError();
}

size_t warm_bytes(const LinkDev &L, const TimeGridD &tg) {
    return (size_t)(L.n_paths - L.n_bulk) * (n_chunks_of(tg) + 1) * 2 * MAXI * sizeof(double);
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
    const int m0 = std::max(p0, L.len_start[MAXI]);
    if (p1 > m0) {
        const dim3 grid(p1 - m0, ty);
        cudaStream_t sm = s_multi ? s_multi : s;
        if (out.doppler) k_extrapolate_fp64_gen<true><<<grid, EXT_T, 0, sm>>>(L, tg, fg, pose, out, rec, m0, p1, f32, warm);
        else k_extrapolate_fp64_gen<false><<<grid, EXT_T, 0, sm>>>(L, tg, fg, pose, out, rec, m0, p1, f32, warm);
    }
    return cudaGetLastError();
}

}  // namespace drt
