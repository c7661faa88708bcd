// drt_k_redo.cu -- the FP64 redo of the FP32-bulk path-steps that FP32 cannot resolve, beside the
// synthesis, with their contributions added to H afterwards (the records form is in drt_k_redo_out.cu).
#include "drt_launch.cuh"

namespace drt {

// The same redo beside the H synthesis: each queued step's (Re a, Im a, tau) goes to out3 (its record
// keeps a = 0, so the synthesis skips it), and k_redo_add then adds a exp(-j 2 pi f tau) into H.
// A queued step is one long dependent FP64 chain, so the kernel's time is the latency of its slowest
// warp.  With no more queued steps than warps, each warp takes one step on one lane: no two chains
// share a warp, so none waits for another's branches.  Otherwise grid row y takes the steps of chains
// of length y (each length is its own code instance, which lanes of one warp would run in turn).
__global__ void __launch_bounds__(32)
k_redo_rec(const LinkDev L, const TimeGridD tg, const FreqGridD fg, const RedoList redo, const double *__restrict__ warm,
           double *__restrict__ out3) {
    const int n = min(*redo.count, redo.cap);
    const OutD none{};
    const RecD nor{nullptr, nullptr};
    const int warp = blockIdx.y * gridDim.x + blockIdx.x;
    if (n <= (int)(gridDim.x * gridDim.y)) {
        if (threadIdx.x == 0 && warp < n) {
            const int4 it = redo.items[warp];
            path_step_redo_as<false>(L, tg, fg, it.y, it.z, none, nor, warm, out3 + 3 * (size_t)warp);
        }
        return;
    }
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int4 it = redo.items[k];
        if (chain_length(L, it.y) != (int)blockIdx.y) continue;
        path_step_redo_as<false>(L, tg, fg, it.y, it.z, none, nor, warm, out3 + 3 * (size_t)k);
    }
}

// one thread per (queued step, 16-bin tile): FP64-reduced seed, FP32 rotation across the tile
__global__ void __launch_bounds__(128)
k_redo_add(const FreqGridD fg, const RedoList redo, const double *__restrict__ in3, float2 *__restrict__ H, int ld) {
    const int n = min(*redo.count, redo.cap);
    const int F = fg.n_bins, ntile = (F + 15) / 16;
    const double f0 = fg.f0, df = fg.df;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < (long long)n * ntile;
         q += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(q / ntile), k0 = (int)(q % ntile) * 16;
        const double ar = in3[3 * (size_t)k], ai = in3[3 * (size_t)k + 1], tau = in3[3 * (size_t)k + 2];
        if (ar == 0.0 && ai == 0.0) continue;
        float2 *row = H + (size_t)redo.items[k].z * ld;
        double x = (f0 + k0 * df) * tau, xs = df * tau;
        float sn, cs, ws, wc;
        sincospif(2.f * (float)(x - floor(x)), &sn, &cs);
        sincospif(2.f * (float)(xs - floor(xs)), &ws, &wc);
        float zr = fmaf((float)ar, cs, (float)ai * sn), zi = fmaf((float)ai, cs, -(float)ar * sn);
        for (int j = 0; j < 16 && k0 + j < F; ++j) {
            atomicAdd(&row[k0 + j].x, zr);
            atomicAdd(&row[k0 + j].y, zi);
            const float nr = fmaf(zr, wc, zi * ws);
            zi = fmaf(zi, wc, -zr * ws);
            zr = nr;
        }
    }
}

cudaError_t launch_redo_rec(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, void *redo, const double *warm,
                            double *out3, cudaStream_t s) {
    if (L.n_paths == 0 || tg.n_steps == 0) return cudaSuccess;
    k_redo_rec<<<dim3(152 * 4, MAXI + 1), 32, 0, s>>>(L, tg, fg, redo_list(redo, L, tg), warm, out3);
    return cudaGetLastError();
}

cudaError_t launch_redo_add(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, void *redo, const double *in3,
                            float2 *H, cudaStream_t s, int ld) {
    if (L.n_paths == 0 || tg.n_steps == 0) return cudaSuccess;
    if (ld < 0) ld = fg.n_bins;
    k_redo_add<<<152 * 4, 128, 0, s>>>(fg, redo_list(redo, L, tg), in3, H, ld);
    return cudaGetLastError();
}

}  // namespace drt
