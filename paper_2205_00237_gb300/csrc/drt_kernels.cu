// drt_kernels.cu -- kernels of the DRT hot path on sm_103a (the per-(path, step) extrapolation
// kernels are in drt_k_fp64.cu and drt_k_bulk.cu):
//   k_pose           a2: per (time-step, body) pose table R(t), O(t), v_O(t), omega(t) (FP64)
//   k_power_bin      power-Doppler / power-delay profiles
//   k_step_power, k_toggle, k_select, k_window_mask
//                    multipath-lifetime expiry and T_C windows
//   k_synth          a9: H(t, f) = sum_p a_p exp(-j 2 pi f tau_p); one thread per (time-step,
//                    16-bin frequency tile, path group), sincos seed per tile and a complex
//                    rotation recurrence inside it, FP32 FMA accumulation, groups added in
//                    shared memory
//   k_probe          FMA issue-rate probe for the roofline denominators
#include <algorithm>
#include "drt_launch.cuh"

namespace drt {

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
    path_step_redo_as<false>(L, tg, fg, p, wm.starts[w], o, none, warm);   // flags only: values suffice
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
