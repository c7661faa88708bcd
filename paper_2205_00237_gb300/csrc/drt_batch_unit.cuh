// drt_batch_unit.cuh -- the extrapolation unit of a batch plan (stage 4: one warp, one (link, path,
// 32 steps) unit), shared by the unrolled per-length kernels (drt_k_batch.cu) and the generic-code
// kernel (drt_k_batch_gen.cu), which compile in separate translation units.
#pragma once
#include <type_traits>

#include "drt_batch.cuh"

namespace drt {

template <int N, bool MULTI, bool OUT, bool PAIR, class S>
__device__ __forceinline__ void batch_unit(const BatchDev &B, const BatchLink &BL, const BatchLink *Q, int li, int p,
                                           int t, const BulkRows &R) {
    Rec5 r, r2;
    if (PAIR && Q)
        bulk_eval<N, MULTI, OUT, S>(BL.L, BL.tg, BL.fg, R, BL.warm, p, t, BL.out, r, B.redo, li, &Q->fg, &r2);
    else
        bulk_eval<N, MULTI, OUT, S>(BL.L, BL.tg, BL.fg, R, BL.warm, p, t, BL.out, r, B.redo, li);
    const size_t ri = BL.rec0 + (size_t)t * BL.L.n_paths + p;
    B.rec_a[ri] = make_float4(r.ar, r.ai, r.ph, r.hi);
    B.rec_b[ri] = r.lo;
    if (PAIR && Q) {
        const size_t r2i = Q->rec0 + (size_t)t * BL.L.n_paths + p;
        B.rec_a[r2i] = make_float4(r2.ar, r2.ai, r2.ph, r2.hi);
        B.rec_b[r2i] = r2.lo;
    }
}

// blocks of 4 warps per SM (the register budget) per stage-4 kernel: the 3-vertex kernel at 4 blocks
// (128 registers, ~0.5 KB of L1-resident spills) measured 2 % faster on a 64-link batch than at 3
template <int N, bool MULTI = false> struct BatchBlocks {
    static constexpr int v = N < 0 ? 4 : MULTI ? 3 : N <= 1 ? 6 : 4;
};

// N >= 0: the units of the chains of length N (no records), MULTI: of the multi-diffraction chains of
// length N (2 or 3); N < 0: the units of the generic range
template <int N, bool DUAL, bool PAIR, bool MULTI = false>
__global__ void __launch_bounds__(128, BatchBlocks<N, MULTI>::v) k_batch_bulk(const BatchDev B) {
    typedef std::conditional_t<DUAL, dd, de> S;
    constexpr int slot = N < 0 ? ST_BULKM : MULTI ? ST_BULKD + N - 2 : ST_BULK + N;
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(B.counter, 1ull);
        it = __shfl_sync(0xffffffffu, it, 0);
        if ((long long)it >= B.n_items) break;
        const int li = find_link(B, slot, (long long)it);
        const BatchLink &BL = B.links[li];
        const long long local = (long long)it - BL.it0[slot];
        const int nb = (BL.tg.n_steps + BULK_W - 1) / BULK_W;
        const int p0 = N < 0 ? BL.gen_p0 : MULTI ? BL.L.multi_start[N - 2] : BL.L.len_start[N];
        const int p = p0 + (int)(local / nb), t = (int)(local % nb) * BULK_W + lane;
        if (N < 0 && p >= BL.skip_p0 && p < BL.skip_p1) continue;   // units of their own (warp-uniform)
        if (t < BL.tg.n_steps) {
            // the unit's chunk-base rows, and those of a pair's second carrier
            const BatchLink *Q = ((PAIR || N < 0) && BL.partner >= 0) ? &B.links[BL.partner] : nullptr;
            const BulkRows R = bulk_rows_global(BL.L, BL.poseb, BL.base, Q ? Q->base : nullptr,
                                                (BL.tg.n_steps + BL.tg.chunk - 1) / BL.tg.chunk, p);
            // the generic range: one instance per chain length, each taking a carrier pair or one carrier
            if constexpr (N >= 0) batch_unit<N, MULTI, false, PAIR, S>(B, BL, Q, li, p, t, R);
            else batch_unit<LEN_ANY, true, true, true, S>(B, BL, Q, li, p, t, R);
        }
    }
}

cudaError_t launch_batch_bulk_gen(bool dual, const BatchDev &B, int grid, cudaStream_t s);

}  // namespace drt
