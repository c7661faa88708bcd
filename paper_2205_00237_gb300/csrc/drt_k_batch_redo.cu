// drt_k_batch_redo.cu -- the FP64 redo at the end of a batch wave: each queued path-step recomputed
// in FP64 and its contribution added to H.  Compiled twice: values only, and (drt_k_batch_redo_dual.cu,
// DRT_BATCH_REDO_DUAL) with the rates the Doppler output needs.
#include "drt_batch.cuh"

namespace drt {

// FP64 redo of queued steps; their contribution is added to H (all bins) with atomics, for the entry
// and, for a carrier pair, its partner
template <bool DUAL>
__device__ void redo_add_entry(const BatchLink &BL, int p, int ti) {
    double r[3];
    const RecD nor{nullptr, nullptr};
    path_step_redo_as<DUAL>(BL.L, BL.tg, BL.fg, p, ti, BL.out, nor, BL.warm, r);
    if (r[0] == 0.0 && r[1] == 0.0) return;
    // a exp(-j 2 pi f_k tau): FP64-reduced seed per 16-bin tile, FP32 rotation across the tile
    const double f0 = BL.fg.f0, df = BL.fg.df;
    const int F = BL.fg.n_bins;
    float2 *row = BL.H + (size_t)ti * F;
    double xs = df * r[2];
    float ws, wc;
    sincospif(2.f * (float)(xs - floor(xs)), &ws, &wc);
    for (int k0 = 0; k0 < F; k0 += 16) {
        double x = (f0 + k0 * df) * r[2];
        float sn, cs;
        sincospif(2.f * (float)(x - floor(x)), &sn, &cs);
        const float ar = (float)r[0], ai = (float)r[1];
        float zr = fmaf(ar, cs, ai * sn), zi = fmaf(ai, cs, -ar * sn);
        for (int j = 0; j < 16 && k0 + j < F; ++j) {
            atomicAdd(&row[k0 + j].x, zr);
            atomicAdd(&row[k0 + j].y, zi);
            const float nr = fmaf(zr, wc, zi * ws);
            zi = fmaf(zi, wc, -zr * ws);
            zr = nr;
        }
    }
}

template <bool DUAL>
__global__ void __launch_bounds__(32) k_batch_redo(const BatchDev B) {   // one warp per block, spread over SMs
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {   // the run's total; a wave whose count exceeds the list
        unsigned long long *hdr = reinterpret_cast<unsigned long long *>(B.redo.count);   // marks the run
        atomicAdd(hdr + 1, (unsigned long long)*B.redo.count);
        if (*B.redo.count > B.redo.cap) atomicOr(hdr + 2, 1ull);
    }
    const int n = min(*B.redo.count, B.redo.cap);
    // few queued steps: one per warp, on one lane (a step is one long dependent FP64 chain; lanes of
    // different chains would wait for each other's branches); otherwise grid row y takes the chains of
    // length y, whose code is one instance
    const bool one = n <= (int)(gridDim.x * gridDim.y);
    const int k0 = one ? blockIdx.y * gridDim.x + blockIdx.x : blockIdx.x * blockDim.x + threadIdx.x;
    const int kstep = one ? n + 1 : gridDim.x * blockDim.x;
    if (one && threadIdx.x != 0) return;
    for (int k = k0; k < n; k += kstep) {
        const int4 itm = B.redo.items[k];
        const BatchLink &BL = B.links[itm.x];
        if (!one && chain_length(BL.L, itm.y) != (int)blockIdx.y) continue;
        redo_add_entry<DUAL>(BL, itm.y, itm.z);
        if (BL.partner >= 0 && itm.y >= BL.pair_p0) redo_add_entry<DUAL>(B.links[BL.partner], itm.y, itm.z);
    }
}

#ifdef DRT_BATCH_REDO_DUAL
cudaError_t launch_batch_redo_dual(const BatchDev &B, int grid, cudaStream_t s) {
    k_batch_redo<true><<<dim3(grid, MAXI + 1), 32, 0, s>>>(B);
    return cudaGetLastError();
}
#else
cudaError_t launch_batch_redo_dual(const BatchDev &B, int grid, cudaStream_t s);

// dual: some entry asks for the Doppler shift (the redo then carries rates)
cudaError_t launch_batch_redo(bool dual, const BatchDev &B, int grid, cudaStream_t s) {
    if (dual) return launch_batch_redo_dual(B, grid, s);
    k_batch_redo<false><<<dim3(grid, MAXI + 1), 32, 0, s>>>(B);
    return cudaGetLastError();
}
#endif

}  // namespace drt
