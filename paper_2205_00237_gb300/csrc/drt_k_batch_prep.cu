// drt_k_batch_prep.cu -- stages 0-3 of a batch plan: FP32 base poses, FP64 chunk-base poses,
// multi-diffraction warm starts and FP64 chunk anchors, each a persistent launch over its
// (link, item) list.
#include "drt_batch.cuh"

namespace drt {

// stages 0-3: block-wide claims of blockDim.x consecutive items
template <int STAGE>
__global__ void __launch_bounds__(128) k_stage(const BatchDev B) {
    __shared__ long long s_start;
    const long long total = B.n_items;
    for (;;) {
        if (threadIdx.x == 0) s_start = (long long)atomicAdd(B.counter, (unsigned long long)blockDim.x);
        __syncthreads();
        long long q = s_start + threadIdx.x;
        bool done = s_start >= total;
        __syncthreads();
        if (done) break;
        if (q >= total) continue;
        const long long it = B.it_base + q;
        int li = find_link(B, STAGE, it);
        const BatchLink &BL = B.links[li];
        long long local = it - BL.it0[STAGE];
        int nch = chunks_of(BL.tg);
        if (STAGE == ST_POSEB) {
            int b = (int)(local / nch), c = (int)(local - (long long)b * nch);
            double tb = BL.tg.t_start + (double)c * BL.tg.chunk * BL.tg.dt;
            if (b < BL.L.n_bodies) body_pose_base(BL.L.bodies[b], tb, BL.poseb[local]);
            else terminal_base(b == BL.L.n_bodies ? BL.L.tx : BL.L.rx, tb, BL.poseb[local]);
        } else if (STAGE == ST_POSE64) {
            int b = (int)(local / nch), c = (int)(local - (long long)b * nch);
            body_pose_row(BL.L.bodies[b], BL.tg.t_start + (double)c * BL.tg.chunk * BL.tg.dt,
                          BL.pose64 + local * POSE_W);
        } else if (STAGE == ST_WARM) {   // rows 0..nch
            int p = BL.L.n_bulk + (int)(local / (nch + 1)), c = (int)(local % (nch + 1));
            path_warm_fp64(BL.L, BL.tg, p, c, BL.warm);
        } else {
            int p = (int)(local / nch), c = (int)(local % nch);
            path_base_fp64(BL.L, BL.tg, BL.fg, BL.pose64, p, c, BL.base, BL.warm);
        }
    }
}

cudaError_t launch_batch_stage(int stage, const BatchDev &B, int grid, cudaStream_t s) {
    switch (stage) {
    case ST_POSEB: k_stage<ST_POSEB><<<grid, 128, 0, s>>>(B); break;
    case ST_POSE64: k_stage<ST_POSE64><<<grid, 128, 0, s>>>(B); break;
    case ST_WARM: k_stage<ST_WARM><<<grid, 128, 0, s>>>(B); break;
    default: k_stage<ST_BASE><<<grid, 128, 0, s>>>(B); break;
    }
    return cudaGetLastError();
}

}  // namespace drt
