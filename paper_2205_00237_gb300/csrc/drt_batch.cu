// drt_batch.cu -- a10: many resident links in one call, FP32-bulk form.
//
// A batch plan holds, per link, its grids, the caller's H buffer and slices of one scratch
// allocation (base poses, FP64 chunk poses, multi-diffraction warm starts, FP64 chunk anchors).
// Each stage is one persistent launch over a flattened list of (link, item) work units claimed with
// an atomic counter, so links of very different sizes share the GPU without a launch per link:
//   stage 0  FP32 base poses              (link, body or terminal, chunk)
//   stage 1  FP64 chunk-base poses        (link, body, chunk)
//   stage 2  multi-diffraction warm start (link, path with >= 2 D in a segment, chunk base 0..n)
//   stage 3  FP64 chunk anchors           (link, path, chunk)
//   stage 4  fused extrapolation + H      (link, block of 32 time steps)
// Stage 4 never writes per-path-step records to HBM: WARPS warps compute the records of WARPS
// paths for 32 time steps into shared memory, then every thread rotates and accumulates BPT
// frequency bins of one time step in registers.  Links are ordered by decreasing path count so the
// largest units are claimed first.  Steps FP32 cannot resolve go to an FP64 redo kernel, which adds
// their contribution to H with atomics.  The whole sequence can be captured in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <type_traits>
#include <vector>

#include "drt_internal.h"
#include "drt_physics.cuh"

namespace drt {

enum { ST_POSEB = 0, ST_POSE64 = 1, ST_WARM = 2, ST_BASE = 3, ST_FUSED = 4, N_STAGES = 5 };
constexpr int FUSED_T = 32;   // time steps per fused work unit (one warp's lanes)

struct BatchLink {
    LinkDev L;
    TimeGridD tg;
    FreqGridD fg;
    PoseB *poseb;      // [bodies + 2][chunks]
    double *pose64;    // [bodies][chunks]
    double *warm;      // [chunks][n_paths - n_bulk][2 * MAXI]
    BaseRec *base;     // [chunks][paths]
    float2 *H;         // caller's [T][F]
    OutD out;          // caller's optional per-path-step records (FP32 formats), [T][P]
    long long it0[N_STAGES + 1];
};

struct BatchDev {
    int n_links;
    const BatchLink *links;
    long long n_items[N_STAGES];
    unsigned long long *counters;   // [N_STAGES]
    RedoList redo;                  // items (link, path, step)
};

__device__ __forceinline__ int find_link(const BatchDev &B, int stage, long long it) {
    int lo = 0, hi = B.n_links - 1;
    while (lo < hi) {   // last link whose first item is <= it
        int mid = (lo + hi + 1) >> 1;
        if (B.links[mid].it0[stage] <= it) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int chunks_of(const TimeGridD &tg) { return (tg.n_steps + tg.chunk - 1) / tg.chunk; }

// stages 0-3: block-wide claims of blockDim.x consecutive items
template <int STAGE>
__global__ void __launch_bounds__(128) k_stage(const BatchDev B) {
    __shared__ long long s_start;
    const long long total = B.n_items[STAGE];
    for (;;) {
        if (threadIdx.x == 0) s_start = (long long)atomicAdd(&B.counters[STAGE], (unsigned long long)blockDim.x);
        __syncthreads();
        long long it = s_start + threadIdx.x;
        bool done = s_start >= total;
        __syncthreads();
        if (done) break;
        if (it >= total) continue;
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

// stage 4: fused extrapolation + synthesis
template <int WARPS, int BPT>
__global__ void __launch_bounds__(WARPS * 32) k_fused(const BatchDev B) {
    __shared__ Rec5 srec[WARPS][32];
    __shared__ long long s_item;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long total = B.n_items[ST_FUSED];
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(&B.counters[ST_FUSED], 1ull);
        __syncthreads();
        const long long it = s_item;
        __syncthreads();
        if (it >= total) break;
        const int li = find_link(B, ST_FUSED, it);
        const BatchLink &BL = B.links[li];
        const int t = (int)(it - BL.it0[ST_FUSED]) * FUSED_T + lane;
        const int F = BL.fg.n_bins, P = BL.L.n_paths, T = BL.tg.n_steps;
        const OutD none{};
        for (int kp = 0; kp < F; kp += WARPS * BPT) {
            const int k0 = kp + w * BPT;
            RedoList rl = B.redo;
            if (kp > 0) rl.count = nullptr;   // queue and record each step once
            const OutD &out = kp > 0 ? none : BL.out;
            float2 acc[BPT];
#pragma unroll
            for (int j = 0; j < BPT; ++j) acc[j] = make_float2(0.f, 0.f);
            const float kf = (float)k0;
            for (int pb = 0; pb < P; pb += WARPS) {
                const int p = pb + w;
                Rec5 r{0.f, 0.f, 0.f, 0.f, 0.f};
                if (p < P && t < T) bulk_eval(BL.L, BL.tg, BL.fg, BL.poseb, BL.base, BL.warm, p, t, out, r, rl, li);
                srec[w][lane] = r;
                __syncthreads();
                if (t < T && k0 < F) {
                    for (int j = 0; j < WARPS; ++j) {
                        const Rec5 q = srec[j][lane];
                        if (q.ar == 0.f && q.ai == 0.f) continue;
                        float ph = kf * q.hi;   // exact: hi has 12 significant bits, k0 < 4096
                        ph -= floorf(ph);
                        ph += q.ph + kf * q.lo;
                        ph -= floorf(ph);
                        float sn, cs, ws, wc;
                        sincospif(2.f * ph, &sn, &cs);
                        sincospif(2.f * (q.hi + q.lo), &ws, &wc);
                        float zr = fmaf(q.ar, cs, q.ai * sn), zi = fmaf(q.ai, cs, -q.ar * sn);
                        const float wr = wc, wi = -ws;
#pragma unroll
                        for (int m = 0; m < BPT; ++m) {
                            acc[m].x += zr;
                            acc[m].y += zi;
                            float nr = fmaf(zr, wr, -zi * wi);
                            zi = fmaf(zr, wi, zi * wr);
                            zr = nr;
                        }
                    }
                }
                __syncthreads();
            }
            if (t < T) {
                float2 *out = BL.H + (size_t)t * F + k0;
#pragma unroll
                for (int m = 0; m < BPT; ++m)
                    if (k0 + m < F) out[m] = acc[m];
            }
        }
    }
}

// FP64 redo of queued steps; their contribution is added to H (all bins) with atomics
__global__ void __launch_bounds__(32) k_batch_redo(const BatchDev B) {   // one warp per block, spread over SMs
    const int n = min(*B.redo.count, B.redo.cap);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int4 itm = B.redo.items[k];
        const BatchLink &BL = B.links[itm.x];
        const double t = BL.tg.t_start + itm.z * BL.tg.dt;
        double r[3];
        const RecD nor{nullptr, nullptr};
        path_step_fp64_core(
            BL.L, BL.tg, BL.fg, itm.y, itm.z, BL.out, nor, true,
            [&](int ty, int idx) { return load_prim_direct<double>(BL.L, t, ty, idx); }, BL.warm, r);
        if (r[0] == 0.0 && r[1] == 0.0) continue;
        const double f0 = BL.fg.fc - 0.5 * BL.fg.bandwidth, df = BL.fg.bandwidth / BL.fg.n_bins;
        float2 *row = BL.H + (size_t)itm.z * BL.fg.n_bins;
        for (int kb = 0; kb < BL.fg.n_bins; ++kb) {
            double x = (f0 + kb * df) * r[2];
            double s, c;
            sincospi(2.0 * (x - floor(x)), &s, &c);
            atomicAdd(&row[kb].x, (float)(r[0] * c + r[1] * s));
            atomicAdd(&row[kb].y, (float)(r[1] * c - r[0] * s));
        }
    }
}

// ------------------------------------------------------------------------------------------------
// host side
//
// One device block per plan: [counters | link table | redo list | per-link scratch], so that a plan
// can live in memory its owner provides (the serving loop's arena) or in its own allocation.
struct BatchPlan {
    int n_links = 0;
    std::vector<BatchLink> host;
    size_t off_links = 0, off_redo = 0, off_scratch = 0, redo_bytes = 0, bytes = 0;
    char *mem = nullptr;
    bool owns = false;
    long long n_items[N_STAGES] = {};
    int variant = -1;   // fused kernel variant (autotuner or caller)
    cudaGraphExec_t graph = nullptr;
    cudaStream_t capture = nullptr;   // private stream the graph is captured on (any caller stream,
                                      // the legacy default stream included, can then launch it)
};

static const int VARIANTS[4][2] = {{8, 32}, {8, 16}, {4, 32}, {4, 16}};   // (warps, bins per thread)

static BatchDev dev_view(const BatchPlan &P, long long fused_limit = -1) {
    BatchDev B;
    B.n_links = P.n_links;
    B.links = reinterpret_cast<const BatchLink *>(P.mem + P.off_links);
    for (int s = 0; s < N_STAGES; ++s) B.n_items[s] = P.n_items[s];
    if (fused_limit >= 0) B.n_items[ST_FUSED] = std::min(fused_limit, P.n_items[ST_FUSED]);
    B.counters = reinterpret_cast<unsigned long long *>(P.mem);
    B.redo.count = reinterpret_cast<int *>(P.mem + P.off_redo);
    B.redo.items = reinterpret_cast<int4 *>(P.mem + P.off_redo + 256);
    B.redo.cap = (int)std::min<size_t>((P.redo_bytes - 256) / sizeof(int4), 0x7fffffff);
    return B;
}

static int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

static cudaError_t launch_fused(int variant, const BatchDev &B, cudaStream_t s) {
    const int sms = sm_count();
    switch (variant) {
    case 0: k_fused<VARIANTS[0][0], VARIANTS[0][1]><<<sms * 2, VARIANTS[0][0] * 32, 0, s>>>(B); break;
    case 1: k_fused<VARIANTS[1][0], VARIANTS[1][1]><<<sms * 2, VARIANTS[1][0] * 32, 0, s>>>(B); break;
    case 2: k_fused<VARIANTS[2][0], VARIANTS[2][1]><<<sms * 4, VARIANTS[2][0] * 32, 0, s>>>(B); break;
    default: k_fused<VARIANTS[3][0], VARIANTS[3][1]><<<sms * 4, VARIANTS[3][0] * 32, 0, s>>>(B); break;
    }
    return cudaGetLastError();
}

// all stages of one run, on one stream
static cudaError_t run_stages(BatchPlan &P, cudaStream_t s, long long fused_limit = -1) {
    BatchDev B = dev_view(P, fused_limit);
    cudaError_t e = cudaMemsetAsync(P.mem, 0, sizeof(unsigned long long) * N_STAGES, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.mem + P.off_redo, 0, sizeof(int), s);
    const int sms = sm_count();
    if (e == cudaSuccess && P.n_items[ST_POSEB]) k_stage<ST_POSEB><<<sms * 4, 128, 0, s>>>(B);
    if (e == cudaSuccess && P.n_items[ST_POSE64]) k_stage<ST_POSE64><<<sms * 4, 128, 0, s>>>(B);
    if (e == cudaSuccess && P.n_items[ST_WARM]) k_stage<ST_WARM><<<sms * 4, 128, 0, s>>>(B);
    if (e == cudaSuccess && P.n_items[ST_BASE]) k_stage<ST_BASE><<<sms * 4, 128, 0, s>>>(B);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess && B.n_items[ST_FUSED]) e = launch_fused(P.variant < 0 ? 0 : P.variant, B, s);
    if (e == cudaSuccess && B.n_items[ST_FUSED]) k_batch_redo<<<sms * 8, 32, 0, s>>>(B);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

// chunk length from a phase-error model: the FP32 delta error grows with the path-length change
// over a chunk, err ~ K fc rate chunk dt (rate = 4 x the fastest terminal or body point); K is
// calibrated on the canyon workload (7.2e-4 rad at 60 GHz, 16 steps of 0.5 ms); the largest power
// of two in [4, 32] that keeps err <= 8e-4 rad is taken
int choose_chunk(const drt_scene_view &v, const drt_time_grid &tg, const drt_freq_grid &fg) {
    const double K = 9.9e-15, target = 8e-4;
    double T = std::fabs(tg.t_start) + std::fabs(tg.dt) * tg.n_steps;
    double vmax = v.vmax + v.amax * T + v.wmax * 20.0;
    double rate = 4.0 * std::max(vmax, 1e-3);
    double lim = target / (K * fg.fc * rate * std::max(std::fabs(tg.dt), 1e-12));
    int c = 4;
    while (c * 2 <= 32 && c * 2 <= lim) c *= 2;
    return c;
}

cudaError_t batch_free(BatchPlan *P) {
    if (!P) return cudaSuccess;
    if (P->graph) cudaGraphExecDestroy(P->graph);
    if (P->capture) cudaStreamDestroy(P->capture);
    if (P->owns) cudaFree(P->mem);
    delete P;
    return cudaSuccess;
}

static size_t r256(size_t b) { return (b + 255) & ~(size_t)255; }

// plan the batch on the host; *bytes is the size of the device block it needs
cudaError_t batch_build(const std::vector<const LinkDev *> &links, const std::vector<drt_scene_view> &views,
                        const drt_time_grid *tgs, const drt_freq_grid *fgs, void *const *H, const OutD *outs,
                        BatchPlan **out, size_t *bytes) {
    const int n = (int)links.size();
    BatchPlan *P = new BatchPlan();
    P->n_links = n;
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    // largest links first: their fused units are claimed first
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (long long)links[a]->n_paths * tgs[a].n_steps > (long long)links[b]->n_paths * tgs[b].n_steps;
    });
    P->host.resize(n);
    size_t off = 0;   // scratch offsets; made absolute in batch_bind
    auto take = [&](size_t b) {
        size_t o = off;
        off += r256(b);
        return o;
    };
    long long it[N_STAGES] = {};
    size_t redo_items = 0;
    for (int k = 0; k < n; ++k) {
        int i = order[k];
        BatchLink &B = P->host[k];
        std::memset(&B, 0, sizeof(B));
        B.L = *links[i];
        int chunk = choose_chunk(views[i], tgs[i], fgs[i]);
        B.tg = make_tgrid(tgs[i].t_start, tgs[i].dt, tgs[i].n_steps, chunk);
        B.fg = make_fgrid(fgs[i].fc, fgs[i].bandwidth, fgs[i].n_bins);
        B.H = reinterpret_cast<float2 *>(H[i]);
        if (outs) B.out = outs[i];
        long long nch = (tgs[i].n_steps + chunk - 1) / chunk;
        int md = B.L.n_paths - B.L.n_bulk;
        B.poseb = reinterpret_cast<PoseB *>(take((size_t)(B.L.n_bodies + 2) * nch * sizeof(PoseB)));
        B.pose64 = reinterpret_cast<double *>(take((size_t)B.L.n_bodies * nch * POSE_W * sizeof(double)));
        B.warm = reinterpret_cast<double *>(take((size_t)md * (nch + 1) * 2 * MAXI * sizeof(double)));
        B.base = reinterpret_cast<BaseRec *>(take((size_t)B.L.n_paths * nch * sizeof(BaseRec)));
        long long cnt[N_STAGES] = {(B.L.n_bodies + 2) * nch, (long long)B.L.n_bodies * nch, (long long)md * (nch + 1),
                                   (long long)B.L.n_paths * nch,
                                   (tgs[i].n_steps + FUSED_T - 1) / FUSED_T};   // a link without paths gets H = 0
        for (int s = 0; s < N_STAGES; ++s) {
            B.it0[s] = it[s];
            it[s] += cnt[s];
        }
        redo_items += (size_t)B.L.n_paths * tgs[i].n_steps;
    }
    for (int s = 0; s < N_STAGES; ++s) P->n_items[s] = it[s];
    // the redo list is bounded: beyond 2^22 + 1/16 of all steps the surplus is dropped and counted
    P->redo_bytes = 256 + r256(std::min<size_t>(redo_items, ((size_t)1 << 22) + redo_items / 16) * sizeof(int4));
    P->off_links = 256;
    P->off_redo = P->off_links + r256(sizeof(BatchLink) * std::max(n, 1));
    P->off_scratch = P->off_redo + P->redo_bytes;
    P->bytes = P->off_scratch + off;
    *bytes = P->bytes;
    *out = P;
    return cudaSuccess;
}

// place the plan in `mem` (P->bytes, 256-byte aligned) and upload its link table on `s`
cudaError_t batch_bind(BatchPlan *P, void *mem, cudaStream_t s) {
    char *old = P->mem ? P->mem + P->off_scratch : nullptr;
    P->mem = reinterpret_cast<char *>(mem);
    char *base = P->mem + P->off_scratch;
    auto rebase = [&](auto *&ptr) {
        size_t o = old ? (size_t)(reinterpret_cast<char *>(ptr) - old) : reinterpret_cast<size_t>(ptr);
        ptr = reinterpret_cast<std::remove_reference_t<decltype(ptr)>>(base + o);
    };
    for (auto &B : P->host) {
        rebase(B.poseb);
        rebase(B.pose64);
        rebase(B.warm);
        rebase(B.base);
    }
    if (!P->n_links) return cudaSuccess;
    return cudaMemcpyAsync(P->mem + P->off_links, P->host.data(), sizeof(BatchLink) * P->n_links,
                           cudaMemcpyHostToDevice, s);
}

cudaError_t batch_alloc(BatchPlan *P) {
    void *mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, std::max<size_t>(P->bytes, 256));
    if (e != cudaSuccess) return e;
    P->owns = true;
    e = batch_bind(P, mem, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    return e;
}

// autotune: time each fused variant on the first units of the batch (after one run of the
// preparation stages) and keep the fastest
cudaError_t batch_autotune(BatchPlan *P, cudaStream_t s, float *best_ms) {
    const long long sample = std::min<long long>(P->n_items[ST_FUSED], (long long)sm_count() * 4);
    float best = 1e30f;
    int pick = 0;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaError_t e = run_stages(*P, s, 0);   // preparation only
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep)   // first pass warms up
        for (int v = 0; v < 4 && e == cudaSuccess; ++v) {
            BatchDev B = dev_view(*P, sample);
            e = cudaMemsetAsync(P->mem + ST_FUSED * sizeof(unsigned long long), 0, sizeof(unsigned long long), s);
            if (e == cudaSuccess) e = cudaMemsetAsync(P->mem + P->off_redo, 0, sizeof(int), s);
            cudaEventRecord(a, s);
            if (e == cudaSuccess) e = launch_fused(v, B, s);
            cudaEventRecord(b, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (rep == 1 && ms < best) {
                best = ms;
                pick = v;
            }
        }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    P->variant = pick;
    *best_ms = best;
    return e;
}

cudaError_t batch_run(BatchPlan *P, cudaStream_t s, bool use_graph) {
    if (!use_graph) return run_stages(*P, s);
    if (!P->graph) {
        cudaGraph_t g = nullptr;
        cudaError_t e = P->capture ? cudaSuccess : cudaStreamCreateWithFlags(&P->capture, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(P->capture, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        cudaError_t e2 = run_stages(*P, P->capture);
        e = cudaStreamEndCapture(P->capture, &g);
        if (e2 != cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&P->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) return e;
    }
    return cudaGraphLaunch(P->graph, s);
}

int batch_variant(const BatchPlan *P) { return P->variant; }
void batch_set_variant(BatchPlan *P, int v) { P->variant = v; }
int batch_chunk(const BatchPlan *P, int k) { return P->host[k].tg.chunk; }
size_t batch_bytes(const BatchPlan *P) { return P->bytes; }

// queued FP64 redo steps of the last completed run (the count may exceed the list's capacity)
cudaError_t batch_redo_count(const BatchPlan *P, long long *n) {
    int c = 0;
    cudaError_t e = cudaMemcpy(&c, P->mem + P->off_redo, sizeof(int), cudaMemcpyDeviceToHost);
    *n = c;
    return e;
}

}  // namespace drt
