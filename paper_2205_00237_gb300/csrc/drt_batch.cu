// drt_batch.cu -- a10: many resident links in one call, FP32-bulk form.
//
// A batch plan holds, per link, its grids, the caller's H buffer and slices of one scratch
// allocation (base poses, FP64 chunk poses, multi-diffraction warm starts, FP64 chunk anchors,
// synthesis records).  Each stage is one persistent launch over a flattened list of (link, unit)
// work units claimed with an atomic counter, so links of very different sizes share the GPU without
// a launch per link:
//   stage 0  FP32 base poses              (link, body or terminal, chunk)
//   stage 1  FP64 chunk-base poses        (link, body, chunk)
//   stage 2  multi-diffraction warm start (link, path with >= 2 D in a segment, chunk base 0..n)
//   stage 3  FP64 chunk anchors           (link, path, chunk)
//   stage 4  FP32-bulk extrapolation      (link, path, 32 consecutive steps: one warp), one unit
//            range and launch per chain length 0..3, per length 2 and 3 of the multi-diffraction
//            chains, and one for the rest (each path of it running the instance for its length)
//   stage 5  H synthesis                  (link, 32 consecutive (step, bin tile) pairs: one block)
// All stages run in waves of links whose per-path-step records (20 B each) fit one record buffer and
// whose poses, warm starts and anchors fit one scratch region, both reused by the next wave, so a
// batch of any size streams through a bounded scratch.  Links are ordered by decreasing work so the
// largest units are claimed first.  Steps FP32 cannot resolve go to an FP64 redo kernel at the end
// of their wave, which adds their contribution to H with atomics.  The frequency tile
// width of stage 5 (8, 16 or 32 bins per thread) is autotuned on the batch.  The whole sequence can
// be captured in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <numeric>
#include <tuple>
#include <type_traits>
#include <vector>

#include "drt_batch.cuh"

namespace drt {

// stage 5: a block takes (link, SYNTH_U consecutive (step, tile of KT bins) pairs), as in the
// single-link synthesis: lane l owns pair l, the SYNTH_PG warps split the paths and add their
// partial sums in shared memory; exact FP32 seed per (pair, path), complex rotation across the tile
template <int VI>
__global__ void __launch_bounds__(SYNTH_U * SYNTH_PG) k_batch_synth(const BatchDev B) {
    constexpr int KT = SYNTH_KT[VI];
    __shared__ float2 part[SYNTH_PG][KT][SYNTH_U + 1];
    const long long it = blockIdx.x;   // one unit per block (a plain grid: no claim loop needed here)
    if (it >= B.n_items) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int li = find_link(B, ST_SYNTH + VI, it);
    const BatchLink &BL = B.links[li];
    const int F = BL.fg.n_bins, P = BL.L.n_paths, T = BL.tg.n_steps;
    const int ntile = (F + KT - 1) / KT;
    const long long pair = (it - BL.it0[ST_SYNTH + VI]) * SYNTH_U + lane;
    const bool live = pair < (long long)T * ntile;
    const int ti = live ? (int)(pair / ntile) : 0, k0 = live ? (int)(pair % ntile) * KT : 0;
    const float kf = (float)k0;
    float2 acc[KT];
#pragma unroll
    for (int j = 0; j < KT; ++j) acc[j] = make_float2(0.f, 0.f);
    if (live) {
        const float4 *__restrict__ ra = B.rec_a + BL.rec0 + (size_t)ti * P;
        const float *__restrict__ rb = B.rec_b + BL.rec0 + (size_t)ti * P;
        // the next path's record is loaded one iteration ahead (its latency hides behind the terms)
        float4 rn = w < P ? __ldg(ra + w) : make_float4(0.f, 0.f, 0.f, 0.f);
        float lon = w < P ? __ldg(rb + w) : 0.f;
        for (int p = w; p < P; p += SYNTH_PG) {
            const float4 r = rn;
            const float lo = lon;
            if (p + SYNTH_PG < P) {
                rn = __ldg(ra + p + SYNTH_PG);
                lon = __ldg(rb + p + SYNTH_PG);
            }
            if (r.x == 0.f && r.y == 0.f) continue;
            float ph = kf * r.w;   // exact: the step's high part has 12 significant bits, k0 < 4096
            ph -= floorf(ph);
            ph += r.z + kf * lo;
            ph -= rintf(ph);       // cycles in [-1/2, 1/2]
            float st = r.w + lo;
            st -= rintf(st);
            float sn, cs, ws, wc;   // hardware sine / cosine on [-pi, pi] (abs. error ~4e-7)
            __sincosf(6.28318530717958648f * ph, &sn, &cs);
            __sincosf(6.28318530717958648f * st, &ws, &wc);
            const float zr = fmaf(r.x, cs, r.y * sn), zi = fmaf(r.y, cs, -r.x * sn);
            add_geometric<KT>(acc, zr, zi, wc, -ws);
        }
    }
#pragma unroll
    for (int j = 0; j < KT; ++j) part[w][j][lane] = acc[j];
    __syncthreads();
    if (!live) return;
    float2 *out = BL.H + (size_t)ti * F + k0;
#pragma unroll
    for (int j = w; j < KT; j += SYNTH_PG) {
        float2 v = part[0][j][lane];
#pragma unroll
        for (int g = 1; g < SYNTH_PG; ++g) {
            v.x += part[g][j][lane].x;
            v.y += part[g][j][lane].y;
        }
        if (k0 + j < F) out[j] = v;
    }
}

// ------------------------------------------------------------------------------------------------
// host side
//
// One device block per plan: [counters | link table | redo list | records | per-link scratch], so
// that a plan can live in memory its owner provides (the serving loop's arena) or in its own
// allocation.
// a wave: consecutive links whose records and scratch fit their buffers; its preparation items
// [prep0, prep0 + n_prep) per stage 0-3, its bulk units and synthesis units per tile variant
struct Wave { int l0, l1; long long prep0[4], n_prep[4], n_bulk[MAXI], n_bulkm, n_synth[3], n_rec, n_bulkd[2]; };

struct BatchPlan {
    int n_links = 0;
    std::vector<BatchLink> host;
    std::vector<Wave> waves;
    long long n_items[4] = {};   // stages 0-3 over all links
    size_t off_links = 0, off_redo = 0, off_rec = 0, off_scratch = 0, redo_bytes = 0, rec_count = 0, bytes = 0;
    size_t n_counters = 0;
    char *mem = nullptr;
    bool owns = false;
    int variant = -1;   // synthesis tile width index (autotuner or caller)
    bool dual = false;  // some link asks for Doppler outputs: carry the rates
    bool any_out = false;   // some link asks for per-path-step records (all units then run generic code)
    bool any_pair = false;  // some entries form carrier pairs
    cudaGraphExec_t graph = nullptr;
    cudaStream_t capture = nullptr;   // private stream the graph is captured on (any caller stream,
                                      // the legacy default stream included, can then launch it)
};

static int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// the launch description of stage `st` (0-3: all links; 4-5: wave w), counter k
static BatchDev dev_view(const BatchPlan &P, int l0, int l1, long long n_items, size_t k) {
    BatchDev B;
    B.l0 = l0;
    B.l1 = l1;
    B.links = reinterpret_cast<const BatchLink *>(P.mem + P.off_links);
    B.n_items = n_items;
    B.it_base = 0;
    B.counter = reinterpret_cast<unsigned long long *>(P.mem) + k;
    B.rec_a = reinterpret_cast<float4 *>(P.mem + P.off_rec);
    B.rec_b = reinterpret_cast<float *>(P.mem + P.off_rec + P.rec_count * sizeof(float4));
    B.redo.count = reinterpret_cast<int *>(P.mem + P.off_redo);
    B.redo.items = reinterpret_cast<int4 *>(P.mem + P.off_redo + 256);
    B.redo.cap = (int)std::min<size_t>((P.redo_bytes - 256) / sizeof(int4), 0x7fffffff);
    return B;
}

static cudaError_t launch_synth_variant(int v, const BatchDev &B, int grid, cudaStream_t s) {
    switch (v) {
    case 0: k_batch_synth<0><<<grid, SYNTH_U * SYNTH_PG, 0, s>>>(B); break;
    case 2: k_batch_synth<2><<<grid, SYNTH_U * SYNTH_PG, 0, s>>>(B); break;
    default: k_batch_synth<1><<<grid, SYNTH_U * SYNTH_PG, 0, s>>>(B); break;
    }
    return cudaGetLastError();
}

// counters: 12 per wave (stages 0-3, bulk per chain length 0..3, generic bulk, synthesis, bulk of the
// multi-diffraction chains of 2 and 3 vertices)
constexpr int N_COUNTERS = 12;
static size_t counter_of(size_t w, int slot) { return N_COUNTERS * w + slot; }

// stages 0-3 of wave w
static cudaError_t run_prep(BatchPlan &P, size_t w, cudaStream_t s) {
    const int grid = sm_count() * 4;
    const Wave &W = P.waves[w];
    auto view = [&](int st) {
        BatchDev B = dev_view(P, W.l0, W.l1, W.n_prep[st], counter_of(w, st));
        B.it_base = W.prep0[st];
        return B;
    };
    for (int st = ST_POSEB; st <= ST_BASE; ++st)
        if (W.n_prep[st])
            if (cudaError_t e = launch_batch_stage(st, view(st), grid, s)) return e;
    return cudaSuccess;
}

static cudaError_t run_wave_bulk(BatchPlan &P, size_t w, cudaStream_t s) {
    const Wave &W = P.waves[w];
    for (int n = 0; n < MAXI; ++n) {
        if (!W.n_bulk[n]) continue;
        const BatchDev B = dev_view(P, W.l0, W.l1, W.n_bulk[n], counter_of(w, 4 + n));
        if (cudaError_t e = launch_batch_bulk(n, false, P.any_pair, B, sm_count() * batch_bulk_blocks(n), s)) return e;
    }
    for (int k = 0; k < 2; ++k) {   // multi-diffraction chains of 2 and 3 vertices
        if (!W.n_bulkd[k]) continue;
        const BatchDev B = dev_view(P, W.l0, W.l1, W.n_bulkd[k], counter_of(w, 10 + k));
        if (cudaError_t e = launch_batch_bulk_multi(k + 2, P.any_pair, B, sm_count() * batch_bulk_blocks(k + 2, true), s))
            return e;
    }
    if (W.n_bulkm) {
        const BatchDev B = dev_view(P, W.l0, W.l1, W.n_bulkm, counter_of(w, 8));
        return launch_batch_bulk(-1, P.dual, true, B, sm_count() * batch_bulk_blocks(-1), s);
    }
    return cudaSuccess;
}

static cudaError_t run_wave_synth(BatchPlan &P, size_t w, cudaStream_t s, long long limit = -1) {
    const Wave &W = P.waves[w];
    const int v = P.variant < 0 ? 1 : P.variant;
    long long n = limit >= 0 ? std::min(limit, W.n_synth[v]) : W.n_synth[v];
    if (!n) return cudaSuccess;
    return launch_synth_variant(v, dev_view(P, W.l0, W.l1, n, counter_of(w, 9)), (int)n, s);
}

// the wave's queued FP64 steps (before the next wave reuses its scratch), then an empty list
static cudaError_t run_redo(BatchPlan &P, size_t w, cudaStream_t s) {
    const Wave &W = P.waves[w];
    cudaError_t e = launch_batch_redo(P.dual, dev_view(P, W.l0, W.l1, 0, 0), sm_count() * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.mem + P.off_redo, 0, sizeof(int), s);
    return e;
}

// all stages of one run, on one stream: per wave, preparation, extrapolation, synthesis, redo
static cudaError_t run_stages(BatchPlan &P, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(P.mem, 0, sizeof(unsigned long long) * P.n_counters, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.mem + P.off_redo, 0, 24, s);   // count, run total, overflow
    for (size_t w = 0; w < P.waves.size() && e == cudaSuccess; ++w) {
        e = run_prep(P, w, s);
        if (e == cudaSuccess) e = run_wave_bulk(P, w, s);
        if (e == cudaSuccess) e = run_wave_synth(P, w, s);
        if (e == cudaSuccess) e = run_redo(P, w, s);
    }
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
                        BatchPlan **out, size_t *bytes, int chunk_div) {
    const int n = (int)links.size();
    BatchPlan *P = new BatchPlan();
    P->n_links = n;
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    // largest links first: their units are claimed first
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (long long)links[a]->n_paths * tgs[a].n_steps > (long long)links[b]->n_paths * tgs[b].n_steps;
    });
    // carrier pairs: entries of the same link over the same time grid without per-path-step records
    // (different carriers of one prediction) share the geometry; each second entry goes right after its
    // first, in the same wave
    auto no_out = [&](int i) {
        if (!outs) return true;
        const OutD &o = outs[i];
        return !(o.tau || o.amp || o.doppler || o.angles || o.flags || o.points);
    };
    for (int i = 0; i < n; ++i)
        if (!no_out(i)) P->any_out = true;
    std::vector<int> mate(n, -1);
    {
        std::map<std::tuple<const LinkDev *, double, double, int>, int> open;
        for (int k = 0; k < n; ++k) {
            const int i = order[k];
            if (!no_out(i)) continue;
            auto key = std::make_tuple(links[i], tgs[i].t_start, tgs[i].dt, tgs[i].n_steps);
            auto it = open.find(key);
            if (it == open.end()) {
                open.emplace(key, i);
            } else {
                mate[it->second] = i;
                mate[i] = it->second;
                open.erase(it);
            }
        }
        std::vector<int> grouped;
        std::vector<char> placed(n, 0);
        for (int k = 0; k < n; ++k) {
            const int i = order[k];
            if (placed[i]) continue;
            grouped.push_back(i);
            placed[i] = 1;
            if (mate[i] >= 0 && !placed[mate[i]]) {
                grouped.push_back(mate[i]);
                placed[mate[i]] = 1;
            }
        }
        order.swap(grouped);
    }
    std::vector<int> pos(n);
    for (int k = 0; k < n; ++k) pos[order[k]] = k;
    P->host.resize(n);
    size_t off = 0;   // scratch offsets; made absolute in batch_bind
    auto take = [&](size_t b) {
        size_t o = off;
        off += r256(b);
        return o;
    };
    long long it[4] = {};
    size_t rec_max = 0, scratch_max = 0;
    Wave W{0, 0, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}, 0, {0, 0, 0}, 0, {0, 0}};
    size_t wave_rec = 0;
    auto close_wave = [&](int l1) {
        W.l1 = l1;
        W.n_rec = (long long)wave_rec;
        for (int st = 0; st < 4; ++st) W.n_prep[st] = it[st] - W.prep0[st];
        P->waves.push_back(W);
        rec_max = std::max(rec_max, wave_rec);
        scratch_max = std::max(scratch_max, off);
    };
    for (int k = 0; k < n; ++k) {
        int i = order[k];
        BatchLink &B = P->host[k];
        std::memset(&B, 0, sizeof(B));
        B.L = *links[i];
        const bool first = mate[i] >= 0 && pos[mate[i]] > k, second = mate[i] >= 0 && !first;
        B.partner = first ? pos[mate[i]] : -1;
        B.shared = second ? 1 : 0;
        // a pair shares the chunks of its geometry: the shorter of the two carriers' choices
        int chunk = choose_chunk(views[i], tgs[i], fgs[i]);
        if (mate[i] >= 0) chunk = std::min(chunk, choose_chunk(views[i], tgs[i], fgs[mate[i]]));
        chunk = std::max(4, chunk / std::max(1, chunk_div));
        B.tg = make_tgrid(tgs[i].t_start, tgs[i].dt, tgs[i].n_steps, chunk);
        B.fg = make_fgrid(fgs[i].fc, fgs[i].bandwidth, fgs[i].n_bins);
        B.H = reinterpret_cast<float2 *>(H[i]);
        if (outs) B.out = outs[i];
        P->dual = P->dual || B.out.doppler != nullptr;
        P->any_pair = P->any_pair || mate[i] >= 0;
        B.gen_p0 = P->any_out ? 0 : B.L.len_start[MAXI];
        B.skip_p0 = P->any_out ? 0 : B.L.multi_start[0];   // multi-diffraction chains of 2 and 3 vertices
        B.skip_p1 = P->any_out ? 0 : B.L.multi_start[2];   // have unit ranges of their own
        B.pair_p0 = P->any_out ? 0 : B.L.len_start[2];
        const long long T = tgs[i].n_steps, Pn = B.L.n_paths;
        long long nch = (T + chunk - 1) / chunk;
        int md = B.L.n_paths - B.L.n_bulk;
        const size_t sz[4] = {(size_t)(B.L.n_bodies + 2) * nch * sizeof(PoseB),
                              (size_t)B.L.n_bodies * nch * POSE_W * sizeof(double),
                              (size_t)md * (nch + 1) * 2 * MAXI * sizeof(double), (size_t)B.L.n_paths * nch * sizeof(BaseRec)};
        const size_t sbytes = r256(sz[0]) + r256(sz[1]) + r256(sz[2]) + r256(sz[3]);
        // waves: consecutive links whose records fit the record buffer and whose scratch fits its cap
        // (the scratch of a wave is reused by the next one)
        const size_t recs = (size_t)T * Pn;
        if (k > W.l0 && !second && ((wave_rec + recs) * REC_BYTES > REC_CAP || off + sbytes > SCRATCH_CAP)) {
            close_wave(k);
            W = Wave{k, k, {it[0], it[1], it[2], it[3]}, {0, 0, 0, 0}, {0, 0, 0, 0}, 0, {0, 0, 0}, 0, {0, 0}};
            wave_rec = 0;
            off = 0;
        }
        B.poseb = reinterpret_cast<PoseB *>(take(sz[0]));
        B.pose64 = reinterpret_cast<double *>(take(sz[1]));
        B.warm = reinterpret_cast<double *>(take(sz[2]));
        B.base = reinterpret_cast<BaseRec *>(take(sz[3]));
        long long cnt[4] = {(B.L.n_bodies + 2) * nch, (long long)B.L.n_bodies * nch, (long long)md * (nch + 1),
                            Pn * nch};
        for (int st = 0; st < 4; ++st) {
            B.it0[st] = it[st];
            it[st] += cnt[st];
        }
        B.rec0 = wave_rec;
        wave_rec += recs;
        // units of 32 steps per path: a pair's second entry has those of its lengths 0 and 1 only (the
        // others are evaluated by its first entry together with the first's own)
        const long long nbw = (T + BULK_W - 1) / BULK_W;
        for (int nl = 0; nl < MAXI; ++nl) {
            B.it0[ST_BULK + nl] = W.n_bulk[nl];
            if (!P->any_out && !(second && nl >= 2))
                W.n_bulk[nl] += (long long)(B.L.len_start[nl + 1] - B.L.len_start[nl]) * nbw;
        }
        B.it0[ST_BULKM] = W.n_bulkm;
        if (!second) W.n_bulkm += (Pn - B.gen_p0) * nbw;
        for (int k = 0; k < 2; ++k) {
            B.it0[ST_BULKD + k] = W.n_bulkd[k];
            if (!second && !P->any_out) W.n_bulkd[k] += (long long)(B.L.multi_start[k + 1] - B.L.multi_start[k]) * nbw;
        }
        for (int v = 0; v < 3; ++v) {   // a link without paths gets H = 0
            const long long pairs = T * ((fgs[i].n_bins + SYNTH_KT[v] - 1) / SYNTH_KT[v]);
            B.it0[ST_SYNTH + v] = W.n_synth[v];
            W.n_synth[v] += (pairs + SYNTH_U - 1) / SYNTH_U;
        }
    }
    if (n) close_wave(n);
    for (int st = 0; st < 4; ++st) P->n_items[st] = it[st];
    P->rec_count = rec_max;
    P->n_counters = N_COUNTERS * std::max<size_t>(P->waves.size(), 1);
    // the redo list of a wave is bounded: beyond 2^22 + 1/128 of the wave's steps the surplus is
    // dropped and counted (measured redo rates stay below 1e-3 of the steps)
    size_t redo_cap = std::min<size_t>(rec_max, ((size_t)1 << 22) + rec_max / 128);
    if (const char *env = std::getenv("DRT_BATCH_REDO_CAP")) {   // a smaller list, for memory-tight callers
        const long long v = std::atoll(env);
        if (v >= 1) redo_cap = std::min<size_t>(redo_cap, (size_t)v);
    }
    P->redo_bytes = 256 + r256(redo_cap * sizeof(int4));
    P->off_links = r256(sizeof(unsigned long long) * P->n_counters);
    P->off_redo = P->off_links + r256(sizeof(BatchLink) * std::max(n, 1));
    P->off_rec = P->off_redo + P->redo_bytes;
    P->off_scratch = P->off_rec + r256(rec_max * REC_BYTES);
    P->bytes = P->off_scratch + scratch_max;
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

// autotune: after the preparation stages and the first wave's extrapolation, time each synthesis
// tile width on the first units of the first wave and keep the fastest
cudaError_t batch_autotune(BatchPlan *P, cudaStream_t s, float *best_ms) {
    *best_ms = 0.f;
    if (P->waves.empty()) {
        P->variant = 1;
        return cudaSuccess;
    }
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaError_t e = cudaMemsetAsync(P->mem, 0, sizeof(unsigned long long) * P->n_counters, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->mem + P->off_redo, 0, 24, s);
    if (e == cudaSuccess) e = run_prep(*P, 0, s);
    if (e == cudaSuccess) e = run_wave_bulk(*P, 0, s);
    const long long sample = (long long)sm_count() * 256;   // units of each variant timed
    float best = 1e30f;
    int pick = 1;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep)   // first pass warms up
        for (int v = 0; v < 3 && e == cudaSuccess; ++v) {
            P->variant = v;
            e = cudaMemsetAsync(P->mem + counter_of(0, 9) * sizeof(unsigned long long), 0,
                                sizeof(unsigned long long), s);
            cudaEventRecord(a, s);
            if (e == cudaSuccess) e = run_wave_synth(*P, 0, s, sample);
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

cudaError_t batch_time_extrapolation(BatchPlan *P, cudaStream_t s, float *ns) {
    *ns = 0.f;
    if (P->waves.empty() || P->waves[0].n_rec == 0) return cudaSuccess;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    cudaError_t e = cudaSuccess;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first pass warms up
        e = cudaMemsetAsync(P->mem, 0, sizeof(unsigned long long) * P->n_counters, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(P->mem + P->off_redo, 0, 24, s);
        cudaEventRecord(a, s);
        if (e == cudaSuccess) e = run_prep(*P, 0, s);
        if (e == cudaSuccess) e = run_wave_bulk(*P, 0, s);
        cudaEventRecord(b, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float t = 0.f;
        cudaEventElapsedTime(&t, a, b);
        if (rep == 1) best = t;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ns = (float)(best * 1e6 / (double)P->waves[0].n_rec);   // the waves of the plans may differ
    return e;
}

void batch_adopt(BatchPlan *P, void *mem) {
    P->mem = reinterpret_cast<char *>(mem);
    P->owns = true;
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

// device address of the last run's redo overflow word (non-zero when a wave queued more FP64 redo
// steps than its list holds, so that run's H misses their contributions)
const unsigned long long *batch_redo_overflow(const BatchPlan *P) {
    return reinterpret_cast<const unsigned long long *>(P->mem + P->off_redo + 16);
}

// queued FP64 redo steps of the last completed run, all waves (a wave's count may exceed its list's
// capacity; the total counts every queued step)
cudaError_t batch_redo_count(const BatchPlan *P, long long *n, bool *overflow) {
    unsigned long long c[2] = {0, 0};
    cudaError_t e = cudaMemcpy(c, P->mem + P->off_redo + 8, sizeof(c), cudaMemcpyDeviceToHost);
    *n = (long long)c[0];
    if (overflow) *overflow = c[1] != 0;
    return e;
}

}  // namespace drt
