// drt_k_fp64_gen.cu -- the FP64 form's kernels for the generic range of chains (several diffractions
// in a segment, or 4 vertices) and the warm starts of the multi-diffraction chains.  Each block runs
// one path; inside, the chain length selects an instance compiled for that length, so every
// per-vertex array, the Newton state included, is indexed by constants and stays in registers.
#include <algorithm>

#include "drt_launch.cuh"

namespace drt {

// the generic range (several diffractions in a segment, 4 vertices): each path runs the instance
// compiled for its chain length
template <bool DUAL>
__global__ void __launch_bounds__(EXT_T)
k_extrapolate_fp64_gen(const LinkDev L, const TimeGridD tg, const FreqGridD fg, const double *__restrict__ pose,
                       const OutD out, const RecD rec, int p0, int p1, int f32out, const double *__restrict__ warm) {
    const int p = p0 + blockIdx.x;
    const int ti = blockIdx.y * EXT_T + threadIdx.x;
    if (p >= p1 || ti >= tg.n_steps) return;
    path_step_fp64<DUAL, LEN_GEN, true, true>(L, tg, fg, pose, p, ti, out, rec, f32out != 0, warm);
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

// one path per warp (lane 0): the chains' lengths differ, and each length is its own code instance
__global__ void __launch_bounds__(32) k_t0par(const LinkDev L, double *__restrict__ t0par) {
    const int p = L.n_bulk + blockIdx.x;
    if (threadIdx.x != 0 || p >= L.n_paths) return;
    path_t0par_fp64(L, p, t0par + (size_t)(p - L.n_bulk) * (2 * MAXI));
}

cudaError_t launch_t0par(const LinkDev &L, double *t0par, cudaStream_t s) {
    const int n = L.n_paths - L.n_bulk;
    if (n <= 0) return cudaSuccess;
    k_t0par<<<n, 32, 0, s>>>(L, t0par);
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

cudaError_t launch_extrapolate_fp64_generic(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg,
                                            const double *pose, const OutD &out, const RecD &rec, int p0, int p1,
                                            int f32, const double *warm, cudaStream_t s) {
    if (p1 < 0) p1 = L.n_paths;
    const int ty = (tg.n_steps + EXT_T - 1) / EXT_T;
    if (tg.n_steps == 0) return cudaSuccess;
    const bool dual = out.doppler != nullptr;
    // One launch over the whole range: FP64-pipe bound, the kernel gains nothing from a register budget
    // per length, while launches of their own for the few multi-diffraction chains of each length
    // (20 and 31 paths of the canyon link: 320 and 496 blocks, under two waves at 2 blocks per SM)
    // measured 15 % slower than one launch of all 51.
    return for_generic_ranges(L, p0, p1, false, [&](int, int a, int b) {
        const dim3 grid(b - a, ty);
        if (dual) k_extrapolate_fp64_gen<true><<<grid, EXT_T, 0, s>>>(L, tg, fg, pose, out, rec, a, b, f32, warm);
        else k_extrapolate_fp64_gen<false><<<grid, EXT_T, 0, s>>>(L, tg, fg, pose, out, rec, a, b, f32, warm);
        return cudaGetLastError();
    });
}

}  // namespace drt
