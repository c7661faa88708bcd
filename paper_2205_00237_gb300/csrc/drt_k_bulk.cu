// drt_k_bulk.cu -- the FP32-bulk form's kernels: FP32 base poses and FP64 path-length / phase anchors
// per chunk of steps, the FP32 delta-number geometry and field per (path, step), and the FP64 redo of
// the steps FP32 cannot resolve (beside the synthesis, its contributions added to H afterwards).
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

// one block per path, one thread per chunk: lanes share the chain signature; body poses at the
// chunk bases come from an FP64 pose table [body][chunk] built first
constexpr int BASE_T = 64;
__global__ void __launch_bounds__(BASE_T)
k_base_fp64(const LinkDev L, const TimeGridD tg, const FreqGridD fg, const double *__restrict__ pose64,
            BaseRec *__restrict__ base, const double *__restrict__ warm, int p0) {
    int p = p0 + blockIdx.x;
    int c = blockIdx.y * BASE_T + threadIdx.x;
    if (p >= L.n_paths || c >= n_chunks_of(tg)) return;
    path_base_fp64(L, tg, fg, pose64, p, c, base, warm);
}

cudaError_t launch_base_pose64(const LinkDev &L, const TimeGridD &tg, double *pose64, cudaStream_t s) {
    if (L.n_paths == 0 || tg.n_steps == 0) return cudaSuccess;
    TimeGridD tc = make_tgrid(tg.t_start, tg.dt * tg.chunk, n_chunks_of(tg), 1);   // chunk bases
    return launch_pose(L, tc, pose64, s);
}

// anchors of paths [p0, p1); the multi-diffraction paths [n_bulk, n_paths) read the warm starts
cudaError_t launch_base_paths(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, const double *pose64,
                              void *base, const double *warm, int p0, int p1, cudaStream_t s) {
    if (p1 <= p0 || tg.n_steps == 0) return cudaSuccess;
    dim3 grid(p1 - p0, (n_chunks_of(tg) + BASE_T - 1) / BASE_T);
    k_base_fp64<<<grid, BASE_T, 0, s>>>(L, tg, fg, pose64, reinterpret_cast<BaseRec *>(base), warm, p0);
    return cudaGetLastError();
}

// The FP32-bulk step with the block mapping of the FP64 form (time-major block order: an SM's resident
// blocks are nearby paths, so nearby signatures).  The H-synthesis path runs one launch per chain
// length with the register budget of that length (72, 107 and ~150 registers for 1, 2 and 3 vertices
// unbounded): 1-vertex chains (most of the scattering tiles) get 12 warps per SM more than a bound set
// for the longest chain would give them.
template <int N> struct BulkBlocks { static constexpr int v = N <= 1 ? 6 : 4; };

template <int N>
__global__ void __launch_bounds__(EXT_T, BulkBlocks<N>::v)
k_extrapolate_bulk_n(const LinkDev L, const TimeGridD tg, const FreqGridD fg, const PoseB *__restrict__ poseb,
                     const BaseRec *__restrict__ base, const double *__restrict__ warm, const OutD out, const RecD rec,
                     const RedoList redo, int p0, int p1) {
    const int p = p0 + blockIdx.y;
    const int ti = blockIdx.x * EXT_T + threadIdx.x;
    if (p >= p1 || ti >= tg.n_steps) return;
    path_step_bulk<N, false, false, de>(L, tg, fg, poseb, base, warm, p, ti, out, rec, redo);
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
    typedef std::conditional_t<DUAL, dd, de> S;
    switch (chain_length(L, p)) {
    case 0: path_step_bulk<0, false, true, S>(L, tg, fg, poseb, base, warm, p, ti, out, rec, redo); break;
    case 1: path_step_bulk<1, false, true, S>(L, tg, fg, poseb, base, warm, p, ti, out, rec, redo); break;
    case 2: path_step_bulk<2, false, true, S>(L, tg, fg, poseb, base, warm, p, ti, out, rec, redo); break;
    default: path_step_bulk<3, false, true, S>(L, tg, fg, poseb, base, warm, p, ti, out, rec, redo); break;
    }
}

// chains with several diffractions in a segment and 4-vertex chains: generic code
template <bool DUAL>
__global__ void __launch_bounds__(EXT_T, 4)
k_extrapolate_bulk_gen(const LinkDev L, const TimeGridD tg, const FreqGridD fg, const PoseB *__restrict__ poseb,
                       const BaseRec *__restrict__ base, const double *__restrict__ warm, const OutD out,
                       const RecD rec, const RedoList redo, int p0, int p1) {
    const int p = p0 + blockIdx.y;
    const int ti = blockIdx.x * EXT_T + threadIdx.x;
    if (p >= p1 || ti >= tg.n_steps) return;
    typedef std::conditional_t<DUAL, dd, de> S;
    path_step_bulk<-1, true, true, S>(L, tg, fg, poseb, base, warm, p, ti, out, rec, redo);
}

cudaError_t launch_extrapolate_bulk(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, const void *poseb,
                                    const void *base, const double *warm, const OutD &out, const RecD &rec, void *redo,
                                    cudaStream_t s, cudaStream_t s_multi) {
    cudaError_t e = cudaMemsetAsync(redo, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (L.n_paths == 0 || tg.n_steps == 0) return cudaSuccess;
    const int tx = (tg.n_steps + EXT_T - 1) / EXT_T;
    const PoseB *pb = reinterpret_cast<const PoseB *>(poseb);
    const BaseRec *bs = reinterpret_cast<const BaseRec *>(base);
    const RedoList rl = redo_list(redo, L, tg);
    if (!any_output(out)) {
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
    if (L.n_paths > L.len_start[MAXI]) {
        const dim3 grid(tx, L.n_paths - L.len_start[MAXI]);
        cudaStream_t sm = s_multi ? s_multi : s;
        if (out.doppler) k_extrapolate_bulk_gen<true><<<grid, EXT_T, 0, sm>>>(L, tg, fg, pb, bs, warm, out, rec, rl, L.len_start[MAXI], L.n_paths);
        else k_extrapolate_bulk_gen<false><<<grid, EXT_T, 0, sm>>>(L, tg, fg, pb, bs, warm, out, rec, rl, L.len_start[MAXI], L.n_paths);
    }
    return cudaGetLastError();
}

// FP64 redo of the queued path-steps: a fixed grid strides over the device-side count
// one warp per block: the few queued steps spread over all SMs (each is a long FP64 chain)
__global__ void __launch_bounds__(32)
k_redo(const LinkDev L, const TimeGridD tg, const FreqGridD fg, const OutD out, const RecD rec, const RedoList redo,
       const double *__restrict__ warm) {
    int n = min(*redo.count, redo.cap);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int4 it = redo.items[k];
        path_step_redo(L, tg, fg, it.y, it.z, out, rec, warm);
    }
}

cudaError_t launch_redo(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, const OutD &out, const RecD &rec,
                        void *redo, const double *warm, cudaStream_t s) {
    if (L.n_paths == 0 || tg.n_steps == 0) return cudaSuccess;
    k_redo<<<152 * 8, 32, 0, s>>>(L, tg, fg, out, rec, redo_list(redo, L, tg), warm);
    return cudaGetLastError();
}

// The same redo beside the H synthesis: each queued step's (Re a, Im a, tau) goes to out3 (its record
// keeps a = 0, so the synthesis skips it), and k_redo_add then adds a exp(-j 2 pi f tau) into H
__global__ void __launch_bounds__(32)
k_redo_rec(const LinkDev L, const TimeGridD tg, const FreqGridD fg, const RedoList redo, const double *__restrict__ warm,
           double *__restrict__ out3) {
    const int n = min(*redo.count, redo.cap);
    const OutD none{};
    const RecD nor{nullptr, nullptr};
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int4 it = redo.items[k];
        path_step_redo(L, tg, fg, it.y, it.z, none, nor, warm, out3 + 3 * (size_t)k);
    }
}

// one thread per (queued step, 16-bin tile): FP64-reduced seed, FP32 rotation across the tile
__global__ void __launch_bounds__(128)
k_redo_add(const FreqGridD fg, const RedoList redo, const double *__restrict__ in3, float2 *__restrict__ H, int ld) {
    const int n = min(*redo.count, redo.cap);
    const int F = fg.n_bins, ntile = (F + 15) / 16;
    const double f0 = fg.fc - 0.5 * fg.bandwidth, df = fg.bandwidth / F;
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
    k_redo_rec<<<152 * 8, 32, 0, s>>>(L, tg, fg, redo_list(redo, L, tg), warm, out3);
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
