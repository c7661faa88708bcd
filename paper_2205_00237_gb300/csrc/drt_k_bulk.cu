// drt_k_bulk.cu -- the FP32-bulk form's kernels: FP32 base poses per chunk of steps and the FP32
// delta-number geometry and field per (path, step) for the chains of lengths 0..3 (the generic range
// in drt_k_bulk_gen.cu, the FP64 anchors in drt_k_base.cu, the FP64 redo in drt_k_redo.cu).
#include <algorithm>
#include <type_traits>

#include "drt_launch.cuh"

namespace drt {

// ------------------------------------------------------------------------------------------------
// FP32-bulk form: base poses per (body or terminal, chunk), FP64 anchors per (path, chunk), then
// the per-(path, step) delta-number kernel with the same block mapping as the FP64 form
size_t bulk_pose_bytes(const LinkDev &L, const TimeGridD &tg) {
    return (size_t)(L.n_bodies + 2) * n_chunks_of(tg) * sizeof(PoseB);
}
size_t bulk_base_bytes(const LinkDev &L, const TimeGridD &tg) {
    return (size_t)L.n_paths * n_chunks_of(tg) * sizeof(BaseRec);
}

__global__ void k_pose_bulk(const BodyD *__restrict__ bodies, int n_bodies, TermD tx, TermD rx, double t_start,
                            double dt, int n_chunks, int chunk, PoseB *__restrict__ poseb) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (n_bodies + 2) * n_chunks) return;
    int b = i / n_chunks, c = i - b * n_chunks;
    double tb = t_start + (double)c * chunk * dt;
    if (b < n_bodies) body_pose_base(bodies[b], tb, poseb[i]);
    else terminal_base(b == n_bodies ? tx : rx, tb, poseb[i]);
}

cudaError_t launch_pose_bulk(const LinkDev &L, const TimeGridD &tg, void *poseb, cudaStream_t s) {
    int n = (L.n_bodies + 2) * n_chunks_of(tg);
    if (tg.n_steps == 0) return cudaSuccess;
    k_pose_bulk<<<(n + 127) / 128, 128, 0, s>>>(L.bodies, L.n_bodies, L.tx, L.rx, tg.t_start, tg.dt, n_chunks_of(tg),
                                                tg.chunk, reinterpret_cast<PoseB *>(poseb));
    return cudaGetLastError();
}

size_t bulk_pose64_bytes(const LinkDev &L, const TimeGridD &tg) {
    return (size_t)L.n_bodies * n_chunks_of(tg) * POSE_W * sizeof(double);
}
size_t bulk_redo_bytes(const LinkDev &L, const TimeGridD &tg) {
    return 256 + (size_t)L.n_paths * tg.n_steps * sizeof(int4);
}

// user outputs: lengths 0..3 in one launch, chosen per block; rates (dual parts) only when the
// Doppler shift is asked for
template <bool DUAL>
__global__ void __launch_bounds__(EXT_T, 4)
k_extrapolate_bulk_out(const LinkDev L, const TimeGridD tg, const FreqGridD fg, const PoseB *__restrict__ poseb,
                       const BaseRec *__restrict__ base, const double *__restrict__ warm, const OutD out,
                       const RecD rec, const RedoList redo, int p0, int p1) {
    const int p = p0 + blockIdx.y;
    const int ti = blockIdx.x * EXT_T + threadIdx.x;
    if (p >= p1 || ti >= tg.n_steps) return;
    const int n = chain_length(L, p);
    const BulkRows R = bulk_rows_global(L, poseb, base, nullptr, (tg.n_steps + tg.chunk - 1) / tg.chunk, p);
    typedef std::conditional_t<DUAL, dd, de> S;
    switch (n) {
    case 0: path_step_bulk<0, false, true, S>(L, tg, fg, R, warm, p, ti, out, rec, redo); break;
    case 1: path_step_bulk<1, false, true, S>(L, tg, fg, R, warm, p, ti, out, rec, redo); break;
    case 2: path_step_bulk<2, false, true, S>(L, tg, fg, R, warm, p, ti, out, rec, redo); break;
    default: path_step_bulk<3, false, true, S>(L, tg, fg, R, warm, p, ti, out, rec, redo); break;
    }
}

cudaError_t launch_extrapolate_bulk(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, const void *poseb,
                                    const void *base, const double *warm, const OutD &out, const RecD &rec, void *redo,
                                    cudaStream_t s, cudaStream_t s_multi, bool lengths, bool generic, bool zero) {
    cudaError_t e = zero ? cudaMemsetAsync(redo, 0, sizeof(int), s) : cudaSuccess;
    if (e != cudaSuccess) return e;
    if (L.n_paths == 0 || tg.n_steps == 0) return cudaSuccess;
    const int tx = (tg.n_steps + EXT_T - 1) / EXT_T;
    const PoseB *pb = reinterpret_cast<const PoseB *>(poseb);
    const BaseRec *bs = reinterpret_cast<const BaseRec *>(base);
    const RedoList rl = redo_list(redo, L, tg);
    if (!lengths) {
    } else if (!any_output(out)) {
        for (int n = 0; n < MAXI; ++n) {
            const int a = L.len_start[n], b = L.len_start[n + 1];
            if (b <= a) continue;
            const dim3 grid(tx, b - a);
            switch (n) {
            case 0: k_extrapolate_bulk_n<0><<<grid, EXT_T, 0, s>>>(L, tg, fg, pb, bs, warm, out, rec, rl, a, b); break;
            case 1: k_extrapolate_bulk_n<1><<<grid, EXT_T, 0, s>>>(L, tg, fg, pb, bs, warm, out, rec, rl, a, b); break;
            case 2: k_extrapolate_bulk_n<2><<<grid, EXT_T, 0, s>>>(L, tg, fg, pb, bs, warm, out, rec, rl, a, b); break;
            default: k_extrapolate_bulk_n<3><<<grid, EXT_T, 0, s>>>(L, tg, fg, pb, bs, warm, out, rec, rl, a, b); break;
            }
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    } else if (L.len_start[MAXI] > 0) {
        const dim3 grid(tx, L.len_start[MAXI]);
        if (out.doppler) k_extrapolate_bulk_out<true><<<grid, EXT_T, 0, s>>>(L, tg, fg, pb, bs, warm, out, rec, rl, 0, L.len_start[MAXI]);
        else k_extrapolate_bulk_out<false><<<grid, EXT_T, 0, s>>>(L, tg, fg, pb, bs, warm, out, rec, rl, 0, L.len_start[MAXI]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (generic && L.n_paths > L.len_start[MAXI]) {
        cudaStream_t sm = s_multi ? s_multi : s;
        return launch_extrapolate_bulk_generic(L, tg, fg, pb, bs, warm, out, rec, rl, sm);
    }
    return cudaGetLastError();
}

}  // namespace drt
