// drt_kernels.cu -- kernels of the DRT hot path on sm_103a:
//   k_pose           a2: per (time-step, body) pose table R(t), O(t), v_O(t), omega(t) (FP64)
//   k_extrapolate    a3-a8: one thread per (path, time-step); a warp covers 32 consecutive time
//                    steps of one path, so all its lanes run the same chain signature
//   k_warm_fp64      warm starts of the multi-diffraction chains at the chunk bases (FP64)
//   k_pose_bulk, k_base_fp64, k_extrapolate_bulk, k_redo
//                    FP32-bulk form: FP32 base poses and FP64 path-length / phase anchors per
//                    16-step chunk, FP32 delta-number geometry and field per (path, step), FP64
//                    redo of the steps FP32 cannot resolve
//   k_synth          a9: H(t, f) = sum_p a_p exp(-j 2 pi f tau_p); one thread per (time-step,
//                    16-bin frequency tile, path group), sincos seed per tile and a complex
//                    rotation recurrence inside it, FP32 FMA accumulation, groups added in
//                    shared memory
//   k_probe          FMA issue-rate probe for the roofline denominators
#include <algorithm>
#include "drt_internal.h"
#include "drt_physics.cuh"

namespace drt {

DRT_HD int n_chunks_of(const TimeGridD &tg) { return (tg.n_steps + tg.chunk - 1) / tg.chunk; }

// ------------------------------------------------------------------------------------------------
// a2: poses.  theta(t) = w0 t + wdot t^2 / 2 about the fixed axis k (Rodrigues), O(t) by Eq. Taylor,
// v_O(t) = v + a t, omega(t) = (w0 + wdot t) k.
__global__ void k_pose(const BodyD *__restrict__ bodies, int n_bodies, double t_start, double dt, int n_steps,
                       double *__restrict__ pose) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_steps * n_bodies) return;
    int b = i / n_steps, ti = i - b * n_steps;   // layout [body][time-step]
    body_pose_row(bodies[b], t_start + ti * dt, pose + (size_t)i * POSE_W);
}

cudaError_t launch_pose(const LinkDev &L, const TimeGridD &tg, double *pose, cudaStream_t s) {
    int n = tg.n_steps * L.n_bodies;
    if (n == 0) return cudaSuccess;
    k_pose<<<(n + 255) / 256, 256, 0, s>>>(L.bodies, L.n_bodies, tg.t_start, tg.dt, tg.n_steps, pose);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// a3-a8 in FP64.  A block covers 128 consecutive time steps of ONE path, so every lane of a warp
// runs the same chain signature (no type divergence); branches that remain (validity, Newton
// iteration counts, transition-function ranges) are correlated between neighbouring instants.
constexpr int EXT_T = 128;

template <bool DUAL>
__global__ void __launch_bounds__(EXT_T)
k_extrapolate_fp64(const LinkDev L, const TimeGridD tg, const FreqGridD fg, const double *__restrict__ pose,
                   const OutD out, const RecD rec, int p0, int f32out, const double *__restrict__ warm) {
    int p = p0 + blockIdx.x;
    int ti = blockIdx.y * EXT_T + threadIdx.x;
    if (p >= L.n_paths || ti >= tg.n_steps) return;
    path_step_fp64<DUAL>(L, tg, fg, pose, p, ti, out, rec, f32out != 0, warm);
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
                                    int p1, bool f32out, double *warm) {
    if (p1 < 0) p1 = L.n_paths;
    if (p1 <= p0 || tg.n_steps == 0) return cudaSuccess;
    dim3 grid(p1 - p0, (tg.n_steps + EXT_T - 1) / EXT_T);
    // the Doppler shift needs the interaction points' velocities (dual numbers); nothing else does
    if (out.doppler) k_extrapolate_fp64<true><<<grid, EXT_T, 0, s>>>(L, tg, fg, pose, out, rec, p0, f32out ? 1 : 0, warm);
    else k_extrapolate_fp64<false><<<grid, EXT_T, 0, s>>>(L, tg, fg, pose, out, rec, p0, f32out ? 1 : 0, warm);
    return cudaGetLastError();
}

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

static RedoList redo_list(void *redo, const LinkDev &L, const TimeGridD &tg) {
    RedoList r;
    r.count = reinterpret_cast<int *>(redo);
    r.items = reinterpret_cast<int4 *>(reinterpret_cast<char *>(redo) + 256);
    r.cap = L.n_paths * tg.n_steps;
    return r;
}

// at most 128 registers (4 blocks of 4 warps per SM): the latency-bound FP32 step gains more from
// the extra warps than it loses to spills (2048-path link 1.47 -> 1.12 ms, canyon within 3 %)
template <bool DUAL>
__global__ void __launch_bounds__(EXT_T, 4)
k_extrapolate_bulk(const LinkDev L, const TimeGridD tg, const FreqGridD fg, const PoseB *__restrict__ poseb,
                   const BaseRec *__restrict__ base, const double *__restrict__ warm, const OutD out, const RecD rec,
                   const RedoList redo) {
    int p = blockIdx.y;   // time-major block order: an SM's resident blocks are nearby paths (signatures)
    int ti = blockIdx.x * EXT_T + threadIdx.x;
    if (p >= L.n_paths || ti >= tg.n_steps) return;
    if constexpr (DUAL) path_step_bulk<dd>(L, tg, fg, poseb, base, warm, p, ti, out, rec, redo);
    else path_step_bulk<de>(L, tg, fg, poseb, base, warm, p, ti, out, rec, redo);
}

cudaError_t launch_extrapolate_bulk(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, const void *poseb,
                                    const void *base, const double *warm, const OutD &out, const RecD &rec, void *redo,
                                    cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(redo, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (L.n_paths == 0 || tg.n_steps == 0) return cudaSuccess;
    dim3 grid((tg.n_steps + EXT_T - 1) / EXT_T, L.n_paths);
    const PoseB *pb = reinterpret_cast<const PoseB *>(poseb);
    const BaseRec *bs = reinterpret_cast<const BaseRec *>(base);
    // rates (dual parts) only when the Doppler shift is asked for
    if (out.doppler) k_extrapolate_bulk<true><<<grid, EXT_T, 0, s>>>(L, tg, fg, pb, bs, warm, out, rec, redo_list(redo, L, tg));
    else k_extrapolate_bulk<false><<<grid, EXT_T, 0, s>>>(L, tg, fg, pb, bs, warm, out, rec, redo_list(redo, L, tg));
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

// ------------------------------------------------------------------------------------------------
// Power-Doppler / power-delay profiles (Sec. IV-A, IV-B): incoherent sum of |a|^2 of the valid
// path-steps per (time bin, Doppler or delay bin).  Block x takes PB_ITEMS path-steps of time
// bin x / per_t, adds them into a shared-memory histogram (FP64 shared atomics) and adds its non-zero bins
// into the zeroed output, so a window of any length spreads over the whole GPU.
constexpr int PB_T = 256, PB_ITEMS = 16 * PB_T;

template <class A>
__global__ void __launch_bounds__(PB_T)
k_power_bin(const double *__restrict__ tau, const A *__restrict__ amp, const A *__restrict__ fd,
            const uint8_t *__restrict__ flags, int n_steps, int n_paths, int steps_per_bin, double x0, double dx,
            int n_bins, int kind, unsigned per_t, double *__restrict__ out) {
    extern __shared__ double hist[];
    const int tb = blockIdx.x / per_t;
    const int t0 = tb * steps_per_bin, t1 = min(n_steps, t0 + steps_per_bin);
    const long long n = (long long)(t1 - t0) * n_paths;
    const long long q0 = (long long)(blockIdx.x % per_t) * PB_ITEMS;
    if (q0 >= n) return;
    for (int j = threadIdx.x; j < n_bins; j += PB_T) hist[j] = 0.0;
    __syncthreads();
    const long long q1 = min(n, q0 + PB_ITEMS);
    const size_t base = (size_t)t0 * n_paths;
    for (long long q = q0 + threadIdx.x; q < q1; q += PB_T) {
        const size_t i = base + q;
        if (flags[i]) continue;
        const double x = kind == 0 ? (double)fd[i] : tau[i];
        const double u = floor((x - x0) / dx);
        if (!(u >= 0.0 && u < (double)n_bins)) continue;
        const double ar = (double)amp[2 * i], ai = (double)amp[2 * i + 1];
        atomicAdd(&hist[(int)u], ar * ar + ai * ai);
    }
    __syncthreads();
    double *row = out + (size_t)tb * n_bins;
    for (int j = threadIdx.x; j < n_bins; j += PB_T)
        if (hist[j] != 0.0) atomicAdd(&row[j], hist[j]);
}

cudaError_t launch_power_bin(bool fp64, const OutD &rec, int n_steps, int n_paths, int steps_per_bin, double x0,
                             double dx, int n_bins, int kind, double *out, cudaStream_t s) {
    const int n_t = (n_steps + steps_per_bin - 1) / steps_per_bin;
    if (n_t == 0) return cudaSuccess;
    if (cudaError_t e = cudaMemsetAsync(out, 0, (size_t)n_t * n_bins * sizeof(double), s)) return e;
    const long long per_bin = (long long)std::min(steps_per_bin, n_steps) * n_paths;
    if (per_bin == 0) return cudaSuccess;
    const long long per_t = (per_bin + PB_ITEMS - 1) / PB_ITEMS;
    if (per_t * n_t > 0x7fffffffLL) return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)(per_t * n_t);
    const size_t sh = (size_t)n_bins * sizeof(double);
    if (fp64)
        k_power_bin<double><<<grid, PB_T, sh, s>>>(rec.tau, reinterpret_cast<const double *>(rec.amp),
                                                   reinterpret_cast<const double *>(rec.doppler), rec.flags,
                                                   n_steps, n_paths, steps_per_bin, x0, dx, n_bins, kind, (unsigned)per_t, out);
    else
        k_power_bin<float><<<grid, PB_T, sh, s>>>(rec.tau, reinterpret_cast<const float *>(rec.amp),
                                                  reinterpret_cast<const float *>(rec.doppler), rec.flags,
                                                  n_steps, n_paths, steps_per_bin, x0, dx, n_bins, kind,
                                                  (unsigned)per_t, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Multipath lifetime T_C (Sec. II): the multipath structure expires at an instant where a path with a
// non-negligible share of the power appears or disappears.  k_step_power sums |a|^2 of the valid paths
// of every instant (one warp per instant); k_toggle marks instant n when some path's validity differs
// between n - 1 and n while, at the instant where it is valid, it carries >= `share` of that total.
template <class A>
__global__ void __launch_bounds__(256)
k_step_power(const A *__restrict__ amp, const uint8_t *__restrict__ flags, int n_steps, int n_paths,
             double *__restrict__ tot) {
    const int n = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (n >= n_steps) return;   // warp-uniform
    double acc = 0.0;
    for (int p = lane; p < n_paths; p += 32) {
        const size_t i = (size_t)n * n_paths + p;
        if (flags[i]) continue;
        const double ar = (double)amp[2 * i], ai = (double)amp[2 * i + 1];
        acc += ar * ar + ai * ai;
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) tot[n] = acc;
}

template <class A>
__global__ void __launch_bounds__(256)
k_toggle(const A *__restrict__ amp, const uint8_t *__restrict__ flags, const double *__restrict__ tot, int n_steps,
         int n_paths, double share, uint8_t *__restrict__ major) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)(n_steps - 1) * n_paths) return;
    const int n = 1 + (int)(q / n_paths);
    const size_t i1 = (size_t)n * n_paths + (size_t)(q % n_paths), i0 = i1 - n_paths;
    const bool v1 = flags[i1] == 0, v0 = flags[i0] == 0;
    if (v1 == v0) return;
    const size_t im = v1 ? i1 : i0;
    const double ar = (double)amp[2 * im], ai = (double)amp[2 * im + 1];
    if (ar * ar + ai * ai >= share * tot[v1 ? n : n - 1]) major[n] = 1;
}

cudaError_t launch_lifetime(bool fp64, const OutD &rec, int n_steps, int n_paths, double share, double *tot,
                            uint8_t *major, cudaStream_t s) {
    if (n_steps == 0) return cudaSuccess;
    if (cudaError_t e = cudaMemsetAsync(major, 0, n_steps, s)) return e;
    if (n_paths == 0) return cudaSuccess;
    const unsigned gp = (unsigned)((n_steps + 7) / 8);
    const long long nq = (long long)(n_steps - 1) * n_paths;
    const unsigned gt = (unsigned)((nq + 255) / 256);
    if (fp64) {
        const double *a = reinterpret_cast<const double *>(rec.amp);
        k_step_power<double><<<gp, 256, 0, s>>>(a, rec.flags, n_steps, n_paths, tot);
        if (nq) k_toggle<double><<<gt, 256, 0, s>>>(a, rec.flags, tot, n_steps, n_paths, share, major);
    } else {
        const float *a = reinterpret_cast<const float *>(rec.amp);
        k_step_power<float><<<gp, 256, 0, s>>>(a, rec.flags, n_steps, n_paths, tot);
        if (nq) k_toggle<float><<<gt, 256, 0, s>>>(a, rec.flags, tot, n_steps, n_paths, share, major);
    }
    return cudaGetLastError();
}

// DRT over T_C windows: a path that is not valid at the first instant of its window is outside that
// window's multipath (sel[start][caller index] != 0, its FP64 flags at the window start) and its
// records carry a = 0; the same holds for the FP64 redo contributions of the FP32-bulk form.
// k_select evaluates the FP64 flags of every (window start, path) in one launch (poses computed at the
// instant, multi-diffraction warm starts from the grid's table).
__device__ __forceinline__ int window_of(const int32_t *__restrict__ starts, int n_w, int n) {
    int lo = 0, hi = n_w - 1;   // the last window starting at or before n (starts[0] = 0)
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (starts[mid] <= n) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(32)
k_select(const LinkDev L, const TimeGridD tg, const FreqGridD fg, WinMask wm, const double *__restrict__ warm) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)wm.n_w * L.n_paths) return;
    const int w = (int)(q / L.n_paths), p = (int)(q % L.n_paths);
    OutD o{};
    o.flags = wm.sel;   // written at [starts[w]][caller index]
    const RecD none{nullptr, nullptr};
    path_step_redo(L, tg, fg, p, wm.starts[w], o, none, warm);
}

cudaError_t launch_select(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, const WinMask &wm,
                          const double *warm, cudaStream_t s) {
    const long long n = (long long)wm.n_w * L.n_paths;
    if (n == 0) return cudaSuccess;
    k_select<<<(unsigned)((n + 31) / 32), 32, 0, s>>>(L, tg, fg, wm, warm);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256)
k_window_mask(float4 *__restrict__ rec_a, int n_steps, int n_paths, const int32_t *__restrict__ perm,
              WinMask wm) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)n_steps * n_paths) return;
    const int n = (int)(q / n_paths), p = (int)(q % n_paths);
    const int w = window_of(wm.starts, wm.n_w, n);
    if (wm.sel[(size_t)wm.starts[w] * n_paths + perm[p]])
        reinterpret_cast<float2 *>(rec_a + q)[0] = make_float2(0.f, 0.f);
}

__global__ void __launch_bounds__(128)
k_redo_window_mask(const RedoList redo, const int32_t *__restrict__ perm, int n_paths, WinMask wm,
                   double *__restrict__ in3) {
    const int n = min(*redo.count, redo.cap);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int4 it = redo.items[k];
        const int w = window_of(wm.starts, wm.n_w, it.z);
        if (wm.sel[(size_t)wm.starts[w] * n_paths + perm[it.y]]) in3[3 * (size_t)k] = in3[3 * (size_t)k + 1] = 0.0;
    }
}

cudaError_t launch_window_mask(const LinkDev &L, const TimeGridD &tg, const RecD &rec, const WinMask &wm,
                               cudaStream_t s) {
    const long long n = (long long)tg.n_steps * L.n_paths;
    if (n == 0) return cudaSuccess;
    k_window_mask<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(rec.rec_a, tg.n_steps, L.n_paths, L.perm, wm);
    return cudaGetLastError();
}

cudaError_t launch_redo_window_mask(const LinkDev &L, const TimeGridD &tg, void *redo, const WinMask &wm, double *in3,
                                    cudaStream_t s) {
    if (L.n_paths == 0 || tg.n_steps == 0) return cudaSuccess;
    k_redo_window_mask<<<152 * 2, 128, 0, s>>>(redo_list(redo, L, tg), L.perm, L.n_paths, wm, in3);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// a9: H synthesis.  A block owns SYN_PAIRS consecutive (step, tile of KT bins) pairs; its PG warps
// split the paths of those steps (warp w takes paths w, w + PG, ...), lane l owns pair l, so the
// lanes of a warp that share a step read the same record (broadcast).  Per (pair, path): seed
// exp(-j 2 pi frac(phi0 + k0 step)) by sincospi with the step split so k0 * hi is exact, then a
// complex rotation by exp(-j 2 pi step) per bin; the PG partial sums are added through shared memory.
constexpr int KT = 16, PG = 4, SYN_PAIRS = 32;

__global__ void __launch_bounds__(SYN_PAIRS * PG)
k_synth(const float4 *__restrict__ rec_a, const float *__restrict__ rec_b, int n_paths, int n_steps, int n_bins,
        float2 *__restrict__ H, int ld) {
    __shared__ float2 part[PG][KT][SYN_PAIRS + 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int ntile = (n_bins + KT - 1) / KT;
    const long long pair = (long long)blockIdx.x * SYN_PAIRS + lane;
    const bool live = pair < (long long)n_steps * ntile;
    const int ti = live ? (int)(pair / ntile) : 0, k0 = live ? (int)(pair % ntile) * KT : 0;
    const float kf = (float)k0;
    float2 acc[KT];
#pragma unroll
    for (int j = 0; j < KT; ++j) acc[j] = make_float2(0.f, 0.f);
    if (live) {
        const float4 *ra = rec_a + (size_t)ti * n_paths;
        const float *rb = rec_b + (size_t)ti * n_paths;
        // the next path's record is loaded one iteration ahead (its latency hides behind the terms)
        float4 rn = w < n_paths ? __ldg(ra + w) : make_float4(0.f, 0.f, 0.f, 0.f);
        float lon = w < n_paths ? __ldg(rb + w) : 0.f;
        for (int p = w; p < n_paths; p += PG) {
            const float4 r = rn;
            const float lo = lon;
            if (p + PG < n_paths) {
                rn = __ldg(ra + p + PG);
                lon = __ldg(rb + p + PG);
            }
            if (r.x == 0.f && r.y == 0.f) continue;
            float ph = kf * r.w;   // exact
            ph -= floorf(ph);
            ph += r.z + kf * lo;
            ph -= rintf(ph);       // cycles in [-1/2, 1/2]
            float st = r.w + lo;
            st -= rintf(st);
            // the hardware sine / cosine on [-pi, pi] (absolute error ~4e-7: far below the
            // synthesis tolerance of 1e-4 of the row RMS)
            float sn, cs, ws, wc;
            __sincosf(6.28318530717958648f * ph, &sn, &cs);
            __sincosf(6.28318530717958648f * st, &ws, &wc);
            // z = a exp(-j 2 pi ph), w = exp(-j 2 pi step)
            float zr = fmaf(r.x, cs, r.y * sn), zi = fmaf(r.y, cs, -r.x * sn);
            add_geometric<KT>(acc, zr, zi, wc, -ws);
        }
    }
#pragma unroll
    for (int j = 0; j < KT; ++j) part[w][j][lane] = acc[j];
    __syncthreads();
    // warp w adds and writes bins j = w, w + PG, ... of every pair of the block
    if (!live) return;
    float2 *out = H + (size_t)ti * ld + k0;
#pragma unroll
    for (int j = w; j < KT; j += PG) {
        float2 v = part[0][j][lane];
#pragma unroll
        for (int g = 1; g < PG; ++g) {
            v.x += part[g][j][lane].x;
            v.y += part[g][j][lane].y;
        }
        if (k0 + j < n_bins) out[j] = v;
    }
}

cudaError_t launch_synth(const RecD &rec, int32_t n_paths, const TimeGridD &tg, const FreqGridD &fg, float2 *H,
                         cudaStream_t s, int ld) {
    if (ld < 0) ld = fg.n_bins;
    int ntile = (fg.n_bins + KT - 1) / KT;
    long long pairs = (long long)tg.n_steps * ntile;
    if (pairs == 0) return cudaSuccess;
    k_synth<<<(unsigned)((pairs + SYN_PAIRS - 1) / SYN_PAIRS), SYN_PAIRS * PG, 0, s>>>(rec.rec_a, rec.rec_b, n_paths,
                                                                                     tg.n_steps, fg.n_bins, H, ld);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// FMA issue-rate probe: 8 independent chains per thread, 4096 iterations
template <class T>
__global__ void k_probe(T *sink, int iters) {
    T a[8];
    T x = T(threadIdx.x) * T(1e-3), y = T(0.999999);
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = x + T(j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = fma(a[j], y, x);
    }
    T s = T(0);
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == T(-1)) sink[0] = s;   // never true; keeps the loop alive
}

cudaError_t launch_probe(int kind, int blocks, double *sink, cudaStream_t s, float *ms) {
    const int iters = kind == 0 ? 2048 : 65536;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int rep = 0; rep < 2; ++rep) {   // first launch warms up
        cudaEventRecord(e0, s);
        if (kind == 0) k_probe<double><<<blocks, 256, 0, s>>>(sink, iters);
        else k_probe<float><<<blocks, 256, 0, s>>>(reinterpret_cast<float *>(sink), iters);
        cudaEventRecord(e1, s);
    }
    cudaError_t err = cudaEventSynchronize(e1);
    cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // FLOPs: blocks * 256 threads * iters * 8 chains * 2
    *ms = *ms;
    return err != cudaSuccess ? err : cudaGetLastError();
}

}  // namespace drt
