// drt_api.cu -- C ABI of the DRT hot path (include/drt.h): contexts, link loading and validation,
// structure-of-arrays packing, device memory under an HBM budget, launches on caller streams.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/drt.h"
#include "drt_internal.h"

using namespace drt;

namespace {

thread_local std::string g_err;

drt_status fail(drt_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(expr)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (expr);                                                                \
        if (e_ != cudaSuccess) return fail(DRT_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

// host copy of a link's scene (the environment database), kept for ray-tracing runs whose chains
// are packed into new links
struct HostScene {
    drt_terminal tx, rx;
    std::vector<drt_body> bodies;
    std::vector<drt_material> mats;
    std::vector<drt_face> faces;
    std::vector<drt_edge> edges;
    std::vector<drt_tile> tiles;
    drt_scene view() const {
        drt_scene s{};
        s.tx = tx;
        s.rx = rx;
        s.n_bodies = (int32_t)bodies.size();
        s.n_materials = (int32_t)mats.size();
        s.n_faces = (int32_t)faces.size();
        s.n_edges = (int32_t)edges.size();
        s.n_tiles = (int32_t)tiles.size();
        s.bodies = bodies.data();
        s.materials = mats.data();
        s.faces = faces.data();
        s.edges = edges.data();
        s.tiles = tiles.data();
        return s;
    }
};

struct Link {
    LinkDev dev;
    drt_scene_view view{};
    std::shared_ptr<std::atomic<int>> inflight = std::make_shared<std::atomic<int>>(0);   // serving
    std::shared_ptr<HostScene> scene;
    std::vector<void *> allocs;
    size_t bytes = 0;
    int32_t n_paths = 0;
};

// a device buffer owned by the context that grows on demand
struct Scratch {
    void *ptr = nullptr;
    size_t cap = 0;
};

}  // namespace

struct drt_ctx {
    int32_t device = 0;
    uint64_t budget = 0, used = 0;
    std::mutex mu;
    std::map<uint64_t, Link> links;
    uint64_t next_link = 1;
    Scratch pose, rec_a, rec_b, h, poseb, base, pose64, redo, warm, redo3, pp_tau, pp_amp, pp_fd, pp_fl, lt_tot,
        lt_major, win_sel, win_starts, tr_faces, tr_rays, tr_count;
    double *probe_sink = nullptr;
    // side streams for work that overlaps within one call (FP32-bulk: anchors and the FP64
    // multi-diffraction paths run beside the FP32 kernel), joined back with events
    cudaStream_t side[2] = {nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};
    cudaEvent_t ev_aux[3] = {nullptr, nullptr, nullptr};   // further dependencies between them
    // tracing: (kind, start, stop) per bracketed launch
    bool profiling = false;
    struct Mark { int kind; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    // a11 serving loop and its arena
    Server *server = nullptr;
    void *arena = nullptr;
    size_t arena_bytes = 0;
    // device blocks of unloaded links, kept for the next loads (size -> block): loading and unloading
    // links in a loop then costs no cudaMalloc / cudaFree; the blocks count against the HBM budget
    std::multimap<size_t, void *> link_pool;
    size_t link_pool_bytes = 0;
};

namespace {

drt_status dev_alloc(drt_ctx *c, size_t bytes, void **out) {
    if (c->budget && c->used + bytes > c->budget)
        return fail(DRT_ENOMEM, "HBM budget exceeded: %llu + %llu > %llu bytes", (unsigned long long)c->used,
                    (unsigned long long)bytes, (unsigned long long)c->budget);
    cudaError_t e = cudaMalloc(out, bytes ? bytes : 16);
    if (e != cudaSuccess) return fail(DRT_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    c->used += bytes;
    return DRT_OK;
}

void dev_free(drt_ctx *c, void *p, size_t bytes) {
    if (p) {
        cudaFree(p);
        c->used -= bytes;
    }
}

// Link storage: a pooled block of at least `bytes` (at most twice that, so small links do not hold
// large blocks), else a new allocation, after returning pooled blocks to the device when the budget
// needs the room.  *got receives the block's size.
constexpr size_t LINK_POOL_CAP = (size_t)1 << 30;   // pooled bytes kept at most
drt_status link_block_alloc(drt_ctx *c, size_t bytes, void **out, size_t *got) {
    bytes = std::max<size_t>(bytes, 256);
    auto it = c->link_pool.lower_bound(bytes);
    if (it != c->link_pool.end() && it->first <= 2 * bytes) {
        *out = it->second;
        *got = it->first;
        c->link_pool_bytes -= it->first;
        c->link_pool.erase(it);
        return DRT_OK;
    }
    while (c->budget && c->used + bytes > c->budget && !c->link_pool.empty()) {
        auto last = std::prev(c->link_pool.end());
        cudaFree(last->second);
        c->used -= last->first;
        c->link_pool_bytes -= last->first;
        c->link_pool.erase(last);
    }
    *got = bytes;
    return dev_alloc(c, bytes, out);
}
// the caller has made sure that no queued work still reads the block
void link_block_free(drt_ctx *c, void *p, size_t bytes) {
    if (!p) return;
    if (c->link_pool_bytes + bytes <= LINK_POOL_CAP) {
        c->link_pool.emplace(bytes, p);
        c->link_pool_bytes += bytes;
    } else {
        cudaFree(p);
        c->used -= bytes;
    }
}

drt_status ensure(drt_ctx *c, Scratch &s, size_t bytes) {
    if (s.cap >= bytes) return DRT_OK;
    // the previous contents may still be read by work queued on a stream
    CUDA_TRY(cudaDeviceSynchronize());
    dev_free(c, s.ptr, s.cap);
    s.ptr = nullptr;
    s.cap = 0;
    size_t want = std::max(bytes, (size_t)1 << 20);
    drt_status st = dev_alloc(c, want, &s.ptr);
    if (st) return st;
    s.cap = want;
    return DRT_OK;
}

// the arrays of one link packed at 256-byte offsets into one host image, uploaded as one device
// allocation with one copy (separate allocations cost a cudaMalloc / cudaFree per array per link)
struct LinkImage {
    std::vector<char> host;
    std::vector<std::function<void(char *)>> bind;
    template <class X> void add(const std::vector<X> &v, const X **dst) {
        const size_t off = (host.size() + 255) & ~(size_t)255;
        host.resize(off + v.size() * sizeof(X));
        if (!v.empty()) std::memcpy(host.data() + off, v.data(), v.size() * sizeof(X));
        bind.push_back([dst, off](char *base) { *dst = reinterpret_cast<const X *>(base + off); });
    }
    drt_status upload(drt_ctx *c, Link &L) {
        void *p = nullptr;
        size_t got = 0;
        if (drt_status st = link_block_alloc(c, host.size(), &p, &got)) return st;
        L.allocs.push_back(p);
        L.bytes += got;
        if (!host.empty()) CUDA_TRY(cudaMemcpy(p, host.data(), host.size(), cudaMemcpyHostToDevice));
        for (auto &b : bind) b(reinterpret_cast<char *>(p));
        return DRT_OK;
    }
};

bool finite3(const double *v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }
double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
void cross3(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
bool unit3(const double *v) { return finite3(v) && std::fabs(std::sqrt(dot3(v, v)) - 1.0) < 1e-9; }

drt_status validate(const drt_scene *s, const drt_path_set *ps) {
    if (!s || !ps) return fail(DRT_EINVAL, "scene and paths must be non-NULL");
    if (s->n_bodies < 1 || s->n_materials < 0 || s->n_faces < 0 || s->n_edges < 0 || s->n_tiles < 0)
        return fail(DRT_EINVAL, "scene counts must be >= 0 (and >= 1 body)");
    if (!s->bodies || (s->n_materials && !s->materials) || (s->n_faces && !s->faces) ||
        (s->n_edges && !s->edges) || (s->n_tiles && !s->tiles))
        return fail(DRT_EINVAL, "scene array pointer is NULL");
    for (const drt_terminal *t : {&s->tx, &s->rx})
        if (!finite3(t->r) || !finite3(t->v) || !finite3(t->a)) return fail(DRT_EINVAL, "terminal not finite");
    for (int i = 0; i < s->n_bodies; ++i) {
        const drt_body &b = s->bodies[i];
        if (!finite3(b.o) || !finite3(b.v) || !finite3(b.a) || !unit3(b.k) || !std::isfinite(b.w0) ||
            !std::isfinite(b.wdot))
            return fail(DRT_EINVAL, "body %d: non-finite kinematics or non-unit axis", i);
    }
    for (int i = 0; i < s->n_materials; ++i) {
        const drt_material &m = s->materials[i];
        if (!(m.eps_r >= 1.0) || !(m.sigma >= 0.0) || !(m.rough_s >= 0.0 && m.rough_s <= 1.0) || !std::isfinite(m.pec))
            return fail(DRT_EINVAL, "material %d: need eps_r >= 1, sigma >= 0, 0 <= rough_s <= 1", i);
    }
    auto chk = [&](int body, int mat, const char *what, int i) -> drt_status {
        if (body < 0 || body >= s->n_bodies) return fail(DRT_EINVAL, "%s %d: body %d out of range", what, i, body);
        if (mat < 0 || mat >= s->n_materials) return fail(DRT_EINVAL, "%s %d: material %d out of range", what, i, mat);
        return DRT_OK;
    };
    for (int i = 0; i < s->n_faces; ++i) {
        const drt_face &f = s->faces[i];
        if (drt_status st = chk(f.body, f.material, "face", i)) return st;
        if (!finite3(f.c) || !unit3(f.n) || !unit3(f.u) || std::fabs(dot3(f.n, f.u)) > 1e-9 || !(f.hu > 0) ||
            !(f.hw > 0))
            return fail(DRT_EINVAL, "face %d: need finite centre, unit n and u with u.n = 0, hu, hw > 0", i);
    }
    for (int i = 0; i < s->n_edges; ++i) {
        const drt_edge &e = s->edges[i];
        if (drt_status st = chk(e.body, e.material, "edge", i)) return st;
        double d[3] = {e.b[0] - e.a[0], e.b[1] - e.a[1], e.b[2] - e.a[2]}, x[3];
        double L = std::sqrt(dot3(d, d));
        if (!finite3(e.a) || !finite3(e.b) || !(L > 0) || !unit3(e.n0) || !unit3(e.nn))
            return fail(DRT_EINVAL, "edge %d: need distinct finite endpoints and unit face normals", i);
        cross3(e.n0, e.nn, x);
        if (std::fabs(dot3(e.n0, d)) > 1e-9 * L || std::fabs(dot3(e.nn, d)) > 1e-9 * L || !(dot3(x, d) > 0))
            return fail(DRT_EINVAL, "edge %d: face normals must be perpendicular to the edge and (b-a).(n0 x nn) > 0", i);
        if (!(e.wedge_n >= 1.0 && e.wedge_n <= 2.0)) return fail(DRT_EINVAL, "edge %d: wedge_n must be in [1, 2]", i);
    }
    for (int i = 0; i < s->n_tiles; ++i) {
        const drt_tile &t = s->tiles[i];
        if (drt_status st = chk(t.body, t.material, "tile", i)) return st;
        if (!finite3(t.c) || !unit3(t.n) || !(t.area > 0) || !(t.s >= 0 && t.s <= 1) || !std::isfinite(t.phase) ||
            !(t.alpha_r >= 0 && t.alpha_r <= 16 && t.alpha_r == std::floor(t.alpha_r)))
            return fail(DRT_EINVAL, "tile %d: need unit normal, area > 0, 0 <= S <= 1, integer alpha_R in [0,16]", i);
    }
    if (ps->n_paths < 0 || (ps->n_paths && (!ps->n_int || !ps->types || !ps->prims)))
        return fail(DRT_EINVAL, "path set: bad count or NULL arrays");
    for (int p = 0; p < ps->n_paths; ++p) {
        int n = ps->n_int[p];
        if (n > DRT_MAX_INT) return fail(DRT_EINVAL, "path %d: %d interactions > %d", p, n, DRT_MAX_INT);
        for (int j = 0; j < DRT_MAX_INT; ++j) {
            int ty = ps->types[p * 4 + j], pr = ps->prims[p * 4 + j];
            if (j >= n) {
                if (ty != DRT_T_NONE) return fail(DRT_EINVAL, "path %d: type set past n_int", p);
                continue;
            }
            int lim = ty == DRT_T_R ? s->n_faces : ty == DRT_T_D ? s->n_edges : ty == DRT_T_S ? s->n_tiles : -1;
            if (lim < 0) return fail(DRT_EINVAL, "path %d vertex %d: bad type %d", p, j, ty);
            if (pr < 0 || pr >= lim) return fail(DRT_EINVAL, "path %d vertex %d: primitive %d out of range", p, j, pr);
            if (ps->s0 && !std::isfinite(ps->s0[p * 4 + j])) return fail(DRT_EINVAL, "path %d: s0 not finite", p);
        }
    }
    return DRT_OK;
}

drt_status check_grids(const drt_time_grid *tg, const drt_freq_grid *fg, int32_t precision) {
    if (!tg || !fg) return fail(DRT_EINVAL, "time and frequency grids must be non-NULL");
    if (tg->n_steps < 0 || !std::isfinite(tg->t_start) || !std::isfinite(tg->dt))
        return fail(DRT_EINVAL, "time grid: n_steps >= 0 and finite t_start, dt required");
    if (!(fg->fc > 0) || !(fg->bandwidth >= 0) || fg->n_bins < 1 || fg->n_bins > 4096 || !std::isfinite(fg->fc))
        return fail(DRT_EINVAL, "frequency grid: fc > 0, bandwidth >= 0, 1 <= n_bins <= 4096 required");
    if (precision != DRT_FP64 && precision != DRT_FP32_BULK)
        return fail(DRT_EINVAL, "precision must be DRT_FP64 or DRT_FP32_BULK");
    return DRT_OK;
}

Link *find_link(drt_ctx *c, uint64_t id) {
    auto it = c->links.find(id);
    return it == c->links.end() ? nullptr : &it->second;
}

// chunk of 16 steps (FP64 warm starts); the FP32-bulk form takes its chunk from the phase-error
// model (choose_chunk)
TimeGridD tgd(const drt_time_grid *g, int chunk = 16) { return make_tgrid(g->t_start, g->dt, g->n_steps, chunk); }
FreqGridD fgd(const drt_freq_grid *g) { return make_fgrid(g->fc, g->bandwidth, g->n_bins); }

// bracket one launch with events when tracing is on
template <class F> drt_status traced(drt_ctx *c, int kind, cudaStream_t s, F &&launch) {
    if (!c->profiling) {
        CUDA_TRY(launch());
        return DRT_OK;
    }
    drt_ctx::Mark m{kind, nullptr, nullptr};
    CUDA_TRY(cudaEventCreate(&m.a));
    CUDA_TRY(cudaEventCreate(&m.b));
    CUDA_TRY(cudaEventRecord(m.a, s));
    CUDA_TRY(launch());
    CUDA_TRY(cudaEventRecord(m.b, s));
    c->marks.push_back(m);
    return DRT_OK;
}

// pose table + extrapolation (+ records) for one link
drt_status run_extrapolation(drt_ctx *c, Link &L, const drt_time_grid *tg, const drt_freq_grid *fg,
                             const OutD &out, const RecD &rec, int32_t precision, cudaStream_t s,
                             bool defer_redo = false) {
    // FP32-bulk chunk length from the same phase-error model as the batch planner
    TimeGridD t = precision == DRT_FP32_BULK ? tgd(tg, choose_chunk(L.view, *tg, *fg)) : tgd(tg);
    FreqGridD f = fgd(fg);
    if (precision == DRT_FP32_BULK) {
        if (drt_status st = ensure(c, c->poseb, bulk_pose_bytes(L.dev, t))) return st;
        if (drt_status st = ensure(c, c->base, bulk_base_bytes(L.dev, t))) return st;
        if (drt_status st = ensure(c, c->pose64, bulk_pose64_bytes(L.dev, t))) return st;
        if (drt_status st = ensure(c, c->redo, bulk_redo_bytes(L.dev, t))) return st;
        if (drt_status st = ensure(c, c->warm, warm_bytes(L.dev, t) + 8)) return st;
        void *pb = c->poseb.ptr, *bs = c->base.ptr, *rd = c->redo.ptr;
        double *p64 = reinterpret_cast<double *>(c->pose64.ptr);
        double *warm = reinterpret_cast<double *>(c->warm.ptr);
        // Three streams.  side[0]: FP64 chunk-base poses, then the anchors of the chains with at most one
        // diffraction per segment.  side[1]: the multi-diffraction warm starts (a few latency-bound
        // solves), their anchors (after the chunk-base poses), then the kernels of the generic range.
        // s: the FP32 base poses, then, once their anchors are in, the kernels of chain lengths 0..3,
        // which so do not wait for the warm starts; s joins side[1] at the end.
        cudaStream_t sa = c->side[0], sw = c->side[1];
        const int nb = L.dev.n_bulk;
        cudaEvent_t ev_p64 = c->ev_aux[0], ev_base0 = c->ev_aux[1], ev_pb = c->ev_aux[2];
        CUDA_TRY(cudaMemsetAsync(rd, 0, sizeof(int), s));   // the redo counter, before any kernel that queues
        CUDA_TRY(cudaEventRecord(c->ev_fork, s));
        CUDA_TRY(cudaStreamWaitEvent(sa, c->ev_fork, 0));
        CUDA_TRY(cudaStreamWaitEvent(sw, c->ev_fork, 0));
        if (drt_status st = traced(c, 3, sw, [&] { return launch_warm_fp64(L.dev, t, warm, sw); })) return st;
        if (drt_status st = traced(c, 3, sa, [&] { return launch_base_pose64(L.dev, t, p64, sa); })) return st;
        CUDA_TRY(cudaEventRecord(ev_p64, sa));
        if (drt_status st = traced(c, 3, sa, [&] { return launch_base_paths(L.dev, t, f, p64, bs, warm, 0, nb, sa); }))
            return st;
        CUDA_TRY(cudaEventRecord(ev_base0, sa));
        CUDA_TRY(cudaStreamWaitEvent(sw, ev_p64, 0));
        if (drt_status st = traced(c, 3, sw, [&] {
                return launch_base_paths(L.dev, t, f, p64, bs, warm, nb, L.dev.n_paths, sw);
            }))
            return st;
        if (drt_status st = traced(c, 0, s, [&] { return launch_pose_bulk(L.dev, t, pb, s); })) return st;
        CUDA_TRY(cudaEventRecord(ev_pb, s));
        CUDA_TRY(cudaStreamWaitEvent(s, ev_base0, 0));
        CUDA_TRY(cudaStreamWaitEvent(sw, ev_pb, 0));
        CUDA_TRY(cudaStreamWaitEvent(sw, ev_base0, 0));   // the 4-vertex chains of the generic range
        if (drt_status st = traced(c, 1, s, [&] {
                cudaError_t e = launch_extrapolate_bulk(L.dev, t, f, pb, bs, warm, out, rec, rd, s, nullptr, true,
                                                        false, false);
                if (e == cudaSuccess)
                    e = launch_extrapolate_bulk(L.dev, t, f, pb, bs, warm, out, rec, rd, s, sw, false, true, false);
                if (e == cudaSuccess) e = cudaEventRecord(c->ev_join[1], sw);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->ev_join[1], 0);
                return e;
            }))
            return st;
        if (!defer_redo)   // else the caller runs the redo beside the synthesis (synth_into)
            if (drt_status st = traced(c, 3, s, [&] { return launch_redo(L.dev, t, f, out, rec, rd, warm, s); }))
                return st;
        return DRT_OK;
    }
    size_t pose_bytes = (size_t)tg->n_steps * L.dev.n_bodies * POSE_W * sizeof(double);
    if (drt_status st = ensure(c, c->pose, pose_bytes)) return st;
    if (drt_status st = ensure(c, c->warm, warm_bytes(L.dev, t))) return st;
    double *pose = reinterpret_cast<double *>(c->pose.ptr);
    double *warm = reinterpret_cast<double *>(c->warm.ptr);
    if (drt_status st = traced(c, 0, s, [&] { return launch_pose(L.dev, t, pose, s); })) return st;
    // The FP64 kernels all wait on the FP64 pipe, so the launches of one call run side by side on three
    // streams: every launch's last wave of blocks then shares the SMs with the others instead of
    // leaving them idle, and the latency-bound multi-diffraction warm starts overlap the chains that
    // do not need them.  side[1]: warm starts, the generic chains (several diffractions in a segment,
    // 4 vertices), length 1; side[0]: length 2, length 0; s: length 3.
    return traced(c, 1, s, [&] {
        const LinkDev &D = L.dev;
        const int *ls = D.len_start;
        cudaStream_t s0 = c->side[0], s1 = c->side[1];
        cudaError_t e = cudaEventRecord(c->ev_fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s0, c->ev_fork, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s1, c->ev_fork, 0);
        if (e == cudaSuccess) e = launch_warm_fp64(D, t, warm, s1);
        if (e == cudaSuccess) e = launch_extrapolate_fp64(D, t, f, pose, out, rec, s1, ls[MAXI], -1, false, warm);
        if (e == cudaSuccess) e = launch_extrapolate_fp64(D, t, f, pose, out, rec, s1, ls[1], ls[2], false, warm);
        if (e == cudaSuccess) e = launch_extrapolate_fp64(D, t, f, pose, out, rec, s0, ls[2], ls[3], false, warm);
        if (e == cudaSuccess) e = launch_extrapolate_fp64(D, t, f, pose, out, rec, s0, ls[0], ls[1], false, warm);
        if (e == cudaSuccess) e = launch_extrapolate_fp64(D, t, f, pose, out, rec, s, ls[3], ls[MAXI], false, warm);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_join[0], s0);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_join[1], s1);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->ev_join[0], 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->ev_join[1], 0);
        return e;
    });
}

drt_status synth_into(drt_ctx *c, Link &L, const drt_time_grid *tg, const drt_freq_grid *fg, float2 *H,
                      int32_t precision, cudaStream_t s, const WinMask *wm = nullptr, int ld = -1) {
    size_t n = (size_t)tg->n_steps * L.n_paths;
    if (drt_status st = ensure(c, c->rec_a, n * sizeof(float4))) return st;
    if (drt_status st = ensure(c, c->rec_b, n * sizeof(float))) return st;
    RecD rec{reinterpret_cast<float4 *>(c->rec_a.ptr), reinterpret_cast<float *>(c->rec_b.ptr)};
    OutD none{};
    TimeGridD t = precision == DRT_FP32_BULK ? tgd(tg, choose_chunk(L.view, *tg, *fg)) : tgd(tg);
    FreqGridD f = fgd(fg);
    if (precision == DRT_FP32_BULK) {
        // the FP64 redo of the few steps FP32 cannot resolve runs beside the synthesis (their records
        // stay zero) and adds its contributions to H afterwards
        if (drt_status st = ensure(c, c->redo3, (size_t)L.n_paths * tg->n_steps * 3 * sizeof(double) + 8)) return st;
        if (drt_status st = run_extrapolation(c, L, tg, fg, none, rec, precision, s, true)) return st;
        double *r3 = reinterpret_cast<double *>(c->redo3.ptr);
        void *rd = c->redo.ptr;
        const double *warm = reinterpret_cast<const double *>(c->warm.ptr);
        if (wm) CUDA_TRY(launch_select(L.dev, t, f, *wm, warm, s));
        cudaStream_t sb = c->side[1];
        CUDA_TRY(cudaEventRecord(c->ev_fork, s));
        CUDA_TRY(cudaStreamWaitEvent(sb, c->ev_fork, 0));
        if (drt_status st = traced(c, 3, sb, [&] { return launch_redo_rec(L.dev, t, f, rd, warm, r3, sb); })) return st;
        if (wm) CUDA_TRY(launch_redo_window_mask(L.dev, t, rd, *wm, r3, sb));
        CUDA_TRY(cudaEventRecord(c->ev_join[1], sb));
        if (wm) CUDA_TRY(launch_window_mask(L.dev, t, rec, *wm, s));
        if (drt_status st = traced(c, 2, s, [&] { return launch_synth(rec, L.n_paths, t, f, H, s, ld); })) return st;
        CUDA_TRY(cudaStreamWaitEvent(s, c->ev_join[1], 0));
        return traced(c, 3, s, [&] { return launch_redo_add(L.dev, t, f, rd, r3, H, s, ld); });
    }
    if (drt_status st = run_extrapolation(c, L, tg, fg, none, rec, precision, s)) return st;
    if (wm) {
        CUDA_TRY(launch_select(L.dev, t, f, *wm, reinterpret_cast<const double *>(c->warm.ptr), s));
        CUDA_TRY(launch_window_mask(L.dev, t, rec, *wm, s));
    }
    return traced(c, 2, s, [&] { return launch_synth(rec, L.n_paths, t, f, H, s, ld); });
}

}  // namespace

// validated host-side structure-of-arrays image of one link (device pointers unset)
drt_status drt::pack_link(const drt_scene *s, const drt_path_set *ps, PackedLink &H) {
    if (drt_status st = validate(s, ps)) return st;
    {
        auto n3 = [](const double *x) { return std::sqrt(dot3(x, x)); };
        drt_scene_view v{std::max(n3(s->tx.v), n3(s->rx.v)), std::max(n3(s->tx.a), n3(s->rx.a)), 0.0};
        for (int i = 0; i < s->n_bodies; ++i) {
            const drt_body &b = s->bodies[i];
            v.vmax = std::max(v.vmax, n3(b.v));
            v.amax = std::max(v.amax, n3(b.a));
            v.wmax = std::max(v.wmax, std::fabs(b.w0) + std::fabs(b.wdot));
        }
        H.view = v;
    }
    LinkDev &d = H.dev;
    d.n_paths = ps->n_paths;
    d.n_bodies = s->n_bodies;
    d.n_faces = s->n_faces;
    d.n_edges = s->n_edges;
    d.n_tiles = s->n_tiles;
    d.n_mats = s->n_materials;
    std::memcpy(&d.tx, &s->tx, sizeof(TermD));
    std::memcpy(&d.rx, &s->rx, sizeof(TermD));

    std::vector<BodyD> &bodies = H.bodies;
    bodies.resize(s->n_bodies);
    std::memcpy(bodies.data(), s->bodies, sizeof(BodyD) * s->n_bodies);
    H.body_fixed.resize(s->n_bodies);
    for (int i = 0; i < s->n_bodies; ++i) {   // a body at rest poses its primitives at their t0 placement
        const BodyD &b = bodies[i];
        bool fixed = b.w0 == 0.0 && b.wdot == 0.0;
        for (int j = 0; j < 3; ++j) fixed = fixed && b.v[j] == 0.0 && b.a[j] == 0.0;
        H.body_fixed[i] = fixed ? 1 : 0;
    }
    auto rel = [&](int body, const double *x, double *o) {
        for (int j = 0; j < 3; ++j) o[j] = x[j] - s->bodies[body].o[j];
    };
    std::vector<FaceD> &faces = H.faces;
    faces.resize(s->n_faces);
    for (int i = 0; i < s->n_faces; ++i) {
        const drt_face &f = s->faces[i];
        FaceD &g = faces[i];
        rel(f.body, f.c, g.c);
        std::memcpy(g.n, f.n, 24);
        std::memcpy(g.u, f.u, 24);
        g.hu = f.hu;
        g.hw = f.hw;
        g.body = f.body;
        g.mat = f.material;
    }
    std::vector<EdgeD> &edges = H.edges;
    edges.resize(s->n_edges);
    for (int i = 0; i < s->n_edges; ++i) {
        const drt_edge &e = s->edges[i];
        EdgeD &g = edges[i];
        double dv[3] = {e.b[0] - e.a[0], e.b[1] - e.a[1], e.b[2] - e.a[2]};
        double L0 = std::sqrt(dot3(dv, dv));
        rel(e.body, e.a, g.a);
        for (int j = 0; j < 3; ++j) g.e[j] = dv[j] / L0;
        cross3(e.n0, g.e, g.t0);
        std::memcpy(g.n0, e.n0, 24);
        g.len = L0;
        g.wn = e.wedge_n;
        g.snp = std::sin(M_PI * e.wedge_n);   // direction of the n-face in the edge frame, once per load
        g.cnp = std::cos(M_PI * e.wedge_n);
        g.body = e.body;
        g.mat = e.material;
        g.pad0 = g.pad1 = 0;
    }
    std::vector<TileD> &tiles = H.tiles;
    tiles.resize(s->n_tiles);
    for (int i = 0; i < s->n_tiles; ++i) {
        const drt_tile &t = s->tiles[i];
        TileD &g = tiles[i];
        rel(t.body, t.c, g.c);
        std::memcpy(g.n, t.n, 24);
        g.area = t.area;
        g.s = t.s;
        g.alpha = t.alpha_r;
        g.cph = std::cos(t.phase);   // the tile's constant phase factor exp(j phase), once per load
        g.sph = std::sin(t.phase);
        g.body = t.body;
        g.mat = t.material;
    }
    std::vector<MatD> &mats = H.mats;
    mats.resize(s->n_materials);
    for (int i = 0; i < s->n_materials; ++i) {
        const drt_material &m = s->materials[i];
        const double spec = std::sqrt(std::max(0.0, 1.0 - m.rough_s * m.rough_s));   // specular scale of a rough face
        mats[i] = MatD{m.eps_r, m.sigma, spec, m.pec, (float)m.eps_r, (float)m.sigma, (float)spec, (float)m.pec};
    }
    auto f3 = [](float *d, const double *x) {
        for (int j = 0; j < 3; ++j) d[j] = (float)x[j];
    };
    H.facesF.resize(s->n_faces);
    for (int i = 0; i < s->n_faces; ++i) {
        const FaceD &g = faces[i];
        FaceF &h = H.facesF[i];
        f3(h.c, g.c);
        f3(h.n, g.n);
        f3(h.u, g.u);
        h.hu = (float)g.hu;
        h.hw = (float)g.hw;
        h.body = g.body;
        h.mat = g.mat;
        h.pad0 = h.pad1 = h.pad2 = 0;
    }
    H.edgesF.resize(s->n_edges);
    for (int i = 0; i < s->n_edges; ++i) {
        const EdgeD &g = edges[i];
        EdgeF &h = H.edgesF[i];
        f3(h.a, g.a);
        f3(h.e, g.e);
        f3(h.t0, g.t0);
        f3(h.n0, g.n0);
        h.len = (float)g.len;
        h.wn = (float)g.wn;
        h.snp = (float)g.snp;
        h.cnp = (float)g.cnp;
        h.body = g.body;
        h.mat = g.mat;
    }
    H.tilesF.resize(s->n_tiles);
    for (int i = 0; i < s->n_tiles; ++i) {
        const TileD &g = tiles[i];
        TileF &h = H.tilesF[i];
        f3(h.c, g.c);
        f3(h.n, g.n);
        h.area = (float)g.area;
        h.s = (float)g.s;
        h.alpha = (float)g.alpha;
        h.cph = (float)g.cph;
        h.sph = (float)g.sph;
        h.body = g.body;
        h.mat = g.mat;
    }

    // paths sorted by chain signature so that warps run uniform code
    int P = ps->n_paths;
    std::vector<uint32_t> code(P);
    for (int p = 0; p < P; ++p) {
        uint32_t c0 = 0;
        for (int j = 0; j < DRT_MAX_INT; ++j) c0 |= (uint32_t)ps->types[p * 4 + j] << (8 * j);
        code[p] = c0;
    }
    std::vector<int32_t> &perm = H.perm;
    perm.resize(P);
    std::iota(perm.begin(), perm.end(), 0);
    // chains with two or more diffractions between point sources (TX, tile, RX) need the Newton solve,
    // which the FP32-bulk form leaves to FP64: they go last, after the `n_bulk` others
    auto multi_d = [](uint32_t c0) {
        int nd = 0;
        for (int j = 0; j < DRT_MAX_INT; ++j) {
            int ty = (c0 >> (8 * j)) & 0xff;
            if (ty == DRT_T_D) {
                if (++nd >= 2) return true;
            } else if (ty == DRT_T_S || ty == DRT_T_NONE) {
                nd = 0;
            }
        }
        return false;
    };
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) {
        bool ma = multi_d(code[a]), mb = multi_d(code[b]);
        return ma != mb ? mb : code[a] < code[b];
    });
    int n_bulk = 0;
    for (int p = 0; p < P; ++p) n_bulk += multi_d(code[p]) ? 0 : 1;
    d.n_bulk = n_bulk;
    {   // the multi-diffraction chains by length (2..4 vertices; sorted by signature, so by length)
        int cnt[MAXI + 1] = {0, 0, 0, 0, 0};
        for (int p = 0; p < P; ++p)
            if (multi_d(code[p])) ++cnt[ps->n_int[p]];
        d.multi_start[0] = n_bulk;
        for (int k = 0; k + 1 < MAXI; ++k) d.multi_start[k + 1] = d.multi_start[k] + cnt[k + 2];
    }
    // start of each chain length among the first n_bulk (sorted) paths
    {
        int cnt[MAXI + 1] = {0, 0, 0, 0, 0};
        for (int p = 0; p < P; ++p)
            if (!multi_d(code[p])) ++cnt[ps->n_int[p]];
        d.len_start[0] = 0;
        for (int k = 0; k <= MAXI; ++k) d.len_start[k + 1] = d.len_start[k] + cnt[k];
    }
    std::vector<uint32_t> &ptypes = H.ptypes;
    ptypes.resize(P);
    std::vector<int4> &pprims = H.pprims;
    pprims.resize(P);
    std::vector<double> &ps0 = H.ps0;
    ps0.resize((size_t)P * 4);
    for (int q = 0; q < P; ++q) {
        int p = perm[q];
        ptypes[q] = code[p];
        const int32_t *pr = ps->prims + p * 4;
        int n = ps->n_int[p];
        pprims[q] = make_int4(n > 0 ? pr[0] : 0, n > 1 ? pr[1] : 0, n > 2 ? pr[2] : 0, n > 3 ? pr[3] : 0);
        for (int j = 0; j < 4; ++j) {
            double v = 0.0;
            if (j < n && ps->types[p * 4 + j] == DRT_T_D)
                v = ps->s0 ? ps->s0[p * 4 + j] : 0.5 * edges[pr[j]].len;
            ps0[(size_t)q * 4 + j] = v;
        }
    }
    return DRT_OK;
}


extern "C" {

const char *drt_last_error(void) { return g_err.c_str(); }

drt_status drt_create(drt_ctx **out, int32_t device, uint64_t hbm_budget_bytes) {
    if (!out) return fail(DRT_EINVAL, "out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0)
        return fail(DRT_ECUDA, "no CUDA device: %s", e != cudaSuccess ? cudaGetErrorString(e) : "count is 0");
    if (device < 0 || device >= n) return fail(DRT_ECUDA, "device %d out of range (%d devices)", device, n);
    CUDA_TRY(cudaSetDevice(device));
    drt_ctx *c = new drt_ctx();
    c->device = device;
    c->budget = hbm_budget_bytes;
    if (cudaMalloc(&c->probe_sink, 64) != cudaSuccess) {
        delete c;
        return fail(DRT_ENOMEM, "cudaMalloc failed");
    }
    // side[1] carries the critical chain of a call (the latency-bound warm starts, then the chains that
    // wait for them; in the FP32-bulk form also the FP64 redo beside the synthesis): at the greatest
    // stream priority its blocks are dispatched before those of the other streams' wide launches
    // (7-8 % off a canyon call in both forms)
    int prio_lo = 0, prio_hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess) prio_lo = prio_hi = 0;
    for (int i = 0; i < 2; ++i) {
        if (cudaStreamCreateWithPriority(&c->side[i], cudaStreamNonBlocking, i == 1 ? prio_hi : prio_lo) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_join[i], cudaEventDisableTiming) != cudaSuccess) {
            drt_destroy(c);
            return fail(DRT_ECUDA, "stream/event creation failed");
        }
    }
    for (int i = 0; i < 3; ++i)
        if (cudaEventCreateWithFlags(&c->ev_aux[i], cudaEventDisableTiming) != cudaSuccess) {
            drt_destroy(c);
            return fail(DRT_ECUDA, "event creation failed");
        }
    if (cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess) {
        drt_destroy(c);
        return fail(DRT_ECUDA, "event creation failed");
    }
    *out = c;
    return DRT_OK;
}

void drt_destroy(drt_ctx *c) {
    if (!c) return;
    drt_serve_stop(c);
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (auto &kv : c->links)
        for (void *p : kv.second.allocs) cudaFree(p);
    for (auto &kv : c->link_pool) cudaFree(kv.second);
    for (Scratch *s : {&c->pose, &c->rec_a, &c->rec_b, &c->h, &c->poseb, &c->base, &c->pose64, &c->redo, &c->warm, &c->redo3, &c->pp_tau,
                       &c->pp_amp, &c->pp_fd, &c->pp_fl, &c->lt_tot, &c->lt_major, &c->win_sel, &c->win_starts,
                       &c->tr_faces, &c->tr_rays, &c->tr_count})
        if (s->ptr) cudaFree(s->ptr);
    cudaFree(c->probe_sink);
    for (int i = 0; i < 2; ++i) {
        if (c->side[i]) cudaStreamDestroy(c->side[i]);
        if (c->ev_join[i]) cudaEventDestroy(c->ev_join[i]);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    for (int i = 0; i < 3; ++i)
        if (c->ev_aux[i]) cudaEventDestroy(c->ev_aux[i]);
    for (auto &m : c->marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    delete c;
}

}  // extern "C"

namespace {

// validate, pack and upload one link (the caller holds the context lock and set the device)
void free_link(drt_ctx *c, Link &L);

drt_status load_link(drt_ctx *c, const drt_scene *s, const drt_path_set *ps, Link &L) {
    PackedLink H;
    if (drt_status st = pack_link(s, ps, H)) return st;
    auto hs = std::make_shared<HostScene>();
    hs->tx = s->tx;
    hs->rx = s->rx;
    hs->bodies.assign(s->bodies, s->bodies + s->n_bodies);
    hs->mats.assign(s->materials, s->materials + s->n_materials);
    hs->faces.assign(s->faces, s->faces + s->n_faces);
    hs->edges.assign(s->edges, s->edges + s->n_edges);
    hs->tiles.assign(s->tiles, s->tiles + s->n_tiles);
    L.scene = hs;
    L.dev = H.dev;
    L.view = H.view;
    L.n_paths = ps->n_paths;
    LinkDev &d = L.dev;
    LinkImage img;
    img.add(H.bodies, &d.bodies);
    img.add(H.body_fixed, &d.body_fixed);
    img.add(H.faces, &d.faces);
    img.add(H.edges, &d.edges);
    img.add(H.tiles, &d.tiles);
    img.add(H.mats, &d.mats);
    img.add(H.facesF, &d.facesF);
    img.add(H.edgesF, &d.edgesF);
    img.add(H.tilesF, &d.tilesF);
    img.add(H.ptypes, &d.ptypes);
    img.add(H.pprims, &d.pprims);
    img.add(H.ps0, &d.ps0);
    img.add(H.perm, &d.perm);
    // multi-diffraction edge parameters and rates at t = 0 (warm-start predictor), solved below
    const size_t n_t0 = (size_t)(d.n_paths - d.n_bulk) * 2 * MAXI;
    std::vector<double> t0par(n_t0, 0.0);
    img.add(t0par, &d.t0par);
    drt_status st = img.upload(c, L);
    if (!st && n_t0) {
        cudaError_t e = launch_t0par(d, const_cast<double *>(d.t0par), 0);
        if (e == cudaSuccess) e = cudaStreamSynchronize(0);
        if (e != cudaSuccess) st = fail(DRT_ECUDA, "t0 edge parameters: %s", cudaGetErrorString(e));
    }
    if (st) {
        free_link(c, L);
        return st;
    }
    return DRT_OK;
}

// a link holds one block (see LinkImage); the caller has made sure no queued work reads it
void free_link(drt_ctx *c, Link &L) {
    for (void *p : L.allocs) link_block_free(c, p, L.bytes);
    L.allocs.clear();
    L.bytes = 0;
}

}  // namespace

extern "C" {

drt_status drt_load_paths(drt_ctx *c, const drt_scene *s, const drt_path_set *ps, uint64_t *out_link) {
    if (!c || !out_link) return fail(DRT_EINVAL, "ctx and out_link must be non-NULL");
    if (!s || !ps) return fail(DRT_EINVAL, "scene and paths must be non-NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    CUDA_TRY(cudaSetDevice(c->device));
    Link L;
    if (drt_status st = load_link(c, s, ps, L)) return st;
    uint64_t id = c->next_link++;
    c->links.emplace(id, std::move(L));
    *out_link = id;
    return DRT_OK;
}

drt_status drt_unload(drt_ctx *c, uint64_t link) {
    if (!c) return fail(DRT_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    Link *L = find_link(c, link);
    if (!L) return fail(DRT_ENOTFOUND, "unknown link %llu", (unsigned long long)link);
    if (L->inflight->load() > 0)
        return fail(DRT_EBUSY, "link %llu has %d pending requests", (unsigned long long)link, L->inflight->load());
    CUDA_TRY(cudaSetDevice(c->device));
    CUDA_TRY(cudaDeviceSynchronize());
    free_link(c, *L);
    c->links.erase(link);
    return DRT_OK;
}

drt_status drt_link_info(drt_ctx *c, uint64_t link, int32_t *n_paths) {
    if (!c || !n_paths) return fail(DRT_EINVAL, "ctx and n_paths must be non-NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    Link *L = find_link(c, link);
    if (!L) return fail(DRT_ENOTFOUND, "unknown link %llu", (unsigned long long)link);
    *n_paths = L->n_paths;
    return DRT_OK;
}

drt_status drt_extrapolate(drt_ctx *c, uint64_t link, const drt_time_grid *tg, const drt_freq_grid *fg,
                           const drt_path_outputs *out, int32_t precision, void *stream) {
    if (!c || !out) return fail(DRT_EINVAL, "ctx and out must be non-NULL");
    if (drt_status st = check_grids(tg, fg, precision)) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    Link *L = find_link(c, link);
    if (!L) return fail(DRT_ENOTFOUND, "unknown link %llu", (unsigned long long)link);
    CUDA_TRY(cudaSetDevice(c->device));
    OutD o{out->tau, out->amp, out->doppler, out->angles, out->flags, out->points};
    RecD none{nullptr, nullptr};
    return run_extrapolation(c, *L, tg, fg, o, none, precision, (cudaStream_t)stream);
}

drt_status drt_synthesize_H(drt_ctx *c, uint64_t link, const drt_time_grid *tg, const drt_freq_grid *fg, void *H,
                            int32_t precision, void *stream) {
    if (!c || !H) return fail(DRT_EINVAL, "ctx and H must be non-NULL");
    if (drt_status st = check_grids(tg, fg, precision)) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    Link *L = find_link(c, link);
    if (!L) return fail(DRT_ENOTFOUND, "unknown link %llu", (unsigned long long)link);
    CUDA_TRY(cudaSetDevice(c->device));
    return synth_into(c, *L, tg, fg, reinterpret_cast<float2 *>(H), precision, (cudaStream_t)stream);
}

drt_status drt_synthesize_H_host(drt_ctx *c, uint64_t link, const drt_time_grid *tg, const drt_freq_grid *fg,
                                 void *H_host, int32_t precision, void *stream) {
    if (!c || !H_host) return fail(DRT_EINVAL, "ctx and H_host must be non-NULL");
    if (drt_status st = check_grids(tg, fg, precision)) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    Link *L = find_link(c, link);
    if (!L) return fail(DRT_ENOTFOUND, "unknown link %llu", (unsigned long long)link);
    CUDA_TRY(cudaSetDevice(c->device));
    size_t bytes = (size_t)tg->n_steps * fg->n_bins * sizeof(float2);
    if (drt_status st = ensure(c, c->h, bytes)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (drt_status st = synth_into(c, *L, tg, fg, reinterpret_cast<float2 *>(c->h.ptr), precision, s)) return st;
    CUDA_TRY(cudaMemcpyAsync(H_host, c->h.ptr, bytes, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return DRT_OK;
}

drt_status drt_power_profile(drt_ctx *c, uint64_t link, const drt_time_grid *tg, const drt_freq_grid *fg,
                             const drt_power_grid *g, double *P, int32_t precision, void *stream) {
    if (!c || !g) return fail(DRT_EINVAL, "ctx and power grid must be non-NULL");
    if (drt_status st = check_grids(tg, fg, precision)) return st;
    if (!P && tg->n_steps > 0) return fail(DRT_EINVAL, "P must be non-NULL");
    if (g->steps_per_bin < 1 || g->n_bins < 1 || g->n_bins > 4096 || !(g->dx > 0) || !std::isfinite(g->x0) ||
        (g->kind != DRT_PP_DOPPLER && g->kind != DRT_PP_DELAY))
        return fail(DRT_EINVAL, "power grid: steps_per_bin >= 1, 1 <= n_bins <= 4096, dx > 0, finite x0, kind "
                                "DRT_PP_DOPPLER or DRT_PP_DELAY required");
    std::lock_guard<std::mutex> lk(c->mu);
    Link *L = find_link(c, link);
    if (!L) return fail(DRT_ENOTFOUND, "unknown link %llu", (unsigned long long)link);
    CUDA_TRY(cudaSetDevice(c->device));
    const size_t n = (size_t)tg->n_steps * L->n_paths;
    const size_t fsz = precision == DRT_FP64 ? sizeof(double) : sizeof(float);
    if (drt_status st = ensure(c, c->pp_tau, n * sizeof(double) + 8)) return st;
    if (drt_status st = ensure(c, c->pp_amp, 2 * n * fsz + 8)) return st;
    if (drt_status st = ensure(c, c->pp_fd, n * fsz + 8)) return st;
    if (drt_status st = ensure(c, c->pp_fl, n + 8)) return st;
    OutD o{reinterpret_cast<double *>(c->pp_tau.ptr), c->pp_amp.ptr, c->pp_fd.ptr, nullptr,
           reinterpret_cast<uint8_t *>(c->pp_fl.ptr), nullptr};
    cudaStream_t s = (cudaStream_t)stream;
    RecD none{nullptr, nullptr};
    if (drt_status st = run_extrapolation(c, *L, tg, fg, o, none, precision, s)) return st;
    CUDA_TRY(launch_power_bin(precision == DRT_FP64, o, tg->n_steps, L->n_paths, g->steps_per_bin, g->x0, g->dx,
                              g->n_bins, g->kind, P, s));
    return DRT_OK;
}

drt_status drt_lifetime_windows(drt_ctx *c, uint64_t link, const drt_time_grid *tg, const drt_freq_grid *fg,
                                const drt_lifetime_params *lp, int32_t precision, uint8_t *major, int32_t *starts,
                                int32_t cap, int32_t *n_windows, void *stream) {
    if (!c || !lp || !n_windows) return fail(DRT_EINVAL, "ctx, params and n_windows must be non-NULL");
    if (drt_status st = check_grids(tg, fg, precision)) return st;
    if (!(lp->share >= 0.0) || !std::isfinite(lp->share) || lp->min_steps < 1 || lp->max_steps < lp->min_steps)
        return fail(DRT_EINVAL, "lifetime params: finite share >= 0, 1 <= min_steps <= max_steps required");
    if (cap < 0 || (cap > 0 && !starts)) return fail(DRT_EINVAL, "starts must hold cap >= 0 entries");
    std::lock_guard<std::mutex> lk(c->mu);
    Link *L = find_link(c, link);
    if (!L) return fail(DRT_ENOTFOUND, "unknown link %llu", (unsigned long long)link);
    CUDA_TRY(cudaSetDevice(c->device));
    const int T = tg->n_steps;
    *n_windows = 0;
    if (T == 0) return DRT_OK;
    const size_t n = (size_t)T * L->n_paths;
    const size_t fsz = precision == DRT_FP64 ? sizeof(double) : sizeof(float);
    if (drt_status st = ensure(c, c->pp_amp, 2 * n * fsz + 8)) return st;
    if (drt_status st = ensure(c, c->pp_fl, n + 8)) return st;
    if (drt_status st = ensure(c, c->lt_tot, (size_t)T * sizeof(double))) return st;
    if (drt_status st = ensure(c, c->lt_major, (size_t)T)) return st;
    OutD o{nullptr, c->pp_amp.ptr, nullptr, nullptr, reinterpret_cast<uint8_t *>(c->pp_fl.ptr), nullptr};
    cudaStream_t s = (cudaStream_t)stream;
    RecD none{nullptr, nullptr};
    if (drt_status st = run_extrapolation(c, *L, tg, fg, o, none, precision, s)) return st;
    uint8_t *mj = reinterpret_cast<uint8_t *>(c->lt_major.ptr);
    CUDA_TRY(launch_lifetime(precision == DRT_FP64, o, T, L->n_paths, lp->share,
                             reinterpret_cast<double *>(c->lt_tot.ptr), mj, s));
    std::vector<uint8_t> m(T);
    CUDA_TRY(cudaMemcpyAsync(m.data(), mj, T, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (major) std::memcpy(major, m.data(), T);
    // windows: from start w, the first major change in [w + min_steps, w + max_steps], else w + max_steps
    std::vector<int32_t> w{0};
    for (long long s0 = 0;;) {
        long long nxt = s0 + lp->max_steps;
        for (long long k = s0 + lp->min_steps; k <= std::min<long long>(s0 + lp->max_steps, T - 1); ++k)
            if (m[k]) {
                nxt = k;
                break;
            }
        if (nxt >= T) break;
        w.push_back((int32_t)nxt);
        s0 = nxt;
    }
    *n_windows = (int32_t)w.size();
    if ((int32_t)w.size() > cap)
        return fail(DRT_EINVAL, "starts holds %d entries, %d windows found (n_windows)", cap, (int)w.size());
    std::memcpy(starts, w.data(), w.size() * sizeof(int32_t));
    return DRT_OK;
}

drt_status drt_synthesize_H_windows(drt_ctx *c, uint64_t link, const drt_time_grid *tg, const drt_freq_grid *fg,
                                    const int32_t *starts, int32_t n_windows, void *H, int32_t precision,
                                    void *stream) {
    if (!c) return fail(DRT_EINVAL, "ctx must be non-NULL");
    if (drt_status st = check_grids(tg, fg, precision)) return st;
    const int T = tg->n_steps;
    if (T > 0) {
        if (!H || !starts || n_windows < 1 || starts[0] != 0)
            return fail(DRT_EINVAL, "H, starts and n_windows >= 1 with starts[0] = 0 required");
        for (int k = 1; k < n_windows; ++k)
            if (starts[k] <= starts[k - 1] || starts[k] >= T)
                return fail(DRT_EINVAL, "window starts must increase strictly and stay below n_steps");
    }
    std::lock_guard<std::mutex> lk(c->mu);
    Link *L = find_link(c, link);
    if (!L) return fail(DRT_ENOTFOUND, "unknown link %llu", (unsigned long long)link);
    CUDA_TRY(cudaSetDevice(c->device));
    if (T == 0) return DRT_OK;
    const int P = L->n_paths;
    cudaStream_t s = (cudaStream_t)stream;
    // re-initialisation at every window start: the paths valid there (FP64 flags of that instant,
    // one selection launch inside the synthesis)
    if (drt_status st = ensure(c, c->win_sel, (size_t)T * P + 8)) return st;
    if (drt_status st = ensure(c, c->win_starts, (size_t)n_windows * sizeof(int32_t))) return st;
    int32_t *sd = reinterpret_cast<int32_t *>(c->win_starts.ptr);
    CUDA_TRY(cudaMemcpyAsync(sd, starts, (size_t)n_windows * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    WinMask wm{sd, n_windows, reinterpret_cast<uint8_t *>(c->win_sel.ptr)};
    return synth_into(c, *L, tg, fg, reinterpret_cast<float2 *>(H), precision, s, &wm);
}

drt_status drt_synthesize_H_wideband(drt_ctx *c, uint64_t link, const drt_time_grid *tg, const drt_freq_grid *fg,
                                     int32_t n_sub, void *H, int32_t precision, void *stream) {
    if (!c || !H) return fail(DRT_EINVAL, "ctx and H must be non-NULL");
    if (drt_status st = check_grids(tg, fg, precision)) return st;
    if (n_sub < 1 || n_sub > fg->n_bins) return fail(DRT_EINVAL, "1 <= n_sub <= n_bins required");
    std::lock_guard<std::mutex> lk(c->mu);
    Link *L = find_link(c, link);
    if (!L) return fail(DRT_ENOTFOUND, "unknown link %llu", (unsigned long long)link);
    CUDA_TRY(cudaSetDevice(c->device));
    const int N = fg->n_bins;
    const double df = fg->bandwidth / N;
    float2 *h = reinterpret_cast<float2 *>(H);
    for (int sb = 0; sb < n_sub; ++sb) {
        // sub-band [k0, k1) spans [f_k0, f_k0 + (k1 - k0) df); coefficients at its centre
        const int k0 = (int)((long long)sb * N / n_sub), k1 = (int)((long long)(sb + 1) * N / n_sub);
        const int n = k1 - k0;
        drt_freq_grid fs{fg->fc - 0.5 * fg->bandwidth + (k0 + 0.5 * n) * df, n * df, n, 0};
        if (drt_status st = synth_into(c, *L, tg, &fs, h + k0, precision, (cudaStream_t)stream, nullptr, N)) return st;
    }
    return DRT_OK;
}

}  // extern "C"

namespace {

// conventional ray tracing at t over a link's scene into host arrays (the context lock is held)
drt_status trace_into(drt_ctx *c, Link &L, double t, int max_order, int with_tiles, drt_traced_paths *out,
                      cudaStream_t s) {
    const long long n_cand = trace_candidates(L.dev, max_order, with_tiles);
    const int cap_dev = (int)std::min<long long>(n_cand, 1 << 22);
    if (drt_status st = ensure(c, c->tr_faces, (size_t)std::max(L.dev.n_faces, 1) * trace_face_bytes())) return st;
    if (drt_status st = ensure(c, c->tr_rays, (size_t)cap_dev * trace_ray_bytes())) return st;
    if (drt_status st = ensure(c, c->tr_count, 256)) return st;
    int *cnt = reinterpret_cast<int *>(c->tr_count.ptr);
    CUDA_TRY(launch_trace(L.dev, t, max_order, with_tiles, c->tr_faces.ptr, c->tr_rays.ptr, cap_dev, cnt, s));
    int count = 0;
    CUDA_TRY(cudaMemcpyAsync(&count, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (count > cap_dev) return fail(DRT_ENOMEM, "ray tracing found %d rays, more than %d", count, cap_dev);
    std::vector<char> rays((size_t)count * trace_ray_bytes());
    if (count) CUDA_TRY(cudaMemcpy(rays.data(), c->tr_rays.ptr, rays.size(), cudaMemcpyDeviceToHost));
    out->n_found = count;
    trace_unpack(rays.data(), count, out->n_int, out->types, out->prims, out->s0, out->cap);
    return DRT_OK;
}

drt_status check_trace_args(int32_t max_order, const drt_traced_paths *out) {
    if (max_order < 0 || max_order > 2) return fail(DRT_EINVAL, "max_order must be 0, 1 or 2");
    if (out && (out->cap < 0 || (out->cap > 0 && (!out->n_int || !out->types || !out->prims || !out->s0))))
        return fail(DRT_EINVAL, "traced paths: cap >= 0 and non-NULL arrays required");
    return DRT_OK;
}

}  // namespace

extern "C" {

drt_status drt_trace_paths(drt_ctx *c, uint64_t link, double t, int32_t max_order, int32_t with_tiles,
                           drt_traced_paths *out, void *stream) {
    if (!c || !out) return fail(DRT_EINVAL, "ctx and out must be non-NULL");
    if (!std::isfinite(t)) return fail(DRT_EINVAL, "t must be finite");
    if (drt_status st = check_trace_args(max_order, out)) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    Link *L = find_link(c, link);
    if (!L) return fail(DRT_ENOTFOUND, "unknown link %llu", (unsigned long long)link);
    CUDA_TRY(cudaSetDevice(c->device));
    return trace_into(c, *L, t, max_order, with_tiles != 0, out, (cudaStream_t)stream);
}

drt_status drt_synthesize_H_retraced(drt_ctx *c, uint64_t link, const drt_time_grid *tg, const drt_freq_grid *fg,
                                     const int32_t *starts, int32_t n_windows, int32_t max_order, int32_t with_tiles,
                                     void *H, int32_t precision, void *stream) {
    if (!c) return fail(DRT_EINVAL, "ctx must be non-NULL");
    if (drt_status st = check_grids(tg, fg, precision)) return st;
    if (drt_status st = check_trace_args(max_order, nullptr)) return st;
    const int T = tg->n_steps;
    if (T > 0) {
        if (!H || !starts || n_windows < 1 || starts[0] != 0)
            return fail(DRT_EINVAL, "H, starts and n_windows >= 1 with starts[0] = 0 required");
        for (int k = 1; k < n_windows; ++k)
            if (starts[k] <= starts[k - 1] || starts[k] >= T)
                return fail(DRT_EINVAL, "window starts must increase strictly and stay below n_steps");
    }
    std::lock_guard<std::mutex> lk(c->mu);
    Link *L = find_link(c, link);
    if (!L) return fail(DRT_ENOTFOUND, "unknown link %llu", (unsigned long long)link);
    CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int F = fg->n_bins;
    const drt_scene scene = L->scene->view();
    for (int w = 0; w < n_windows && T > 0; ++w) {
        const int k0 = starts[w], k1 = w + 1 < n_windows ? starts[w + 1] : T;
        const double tw = tg->t_start + k0 * tg->dt;
        // the window's chains: a ray-tracing run at its first instant
        const long long n_cand = trace_candidates(L->dev, max_order, with_tiles != 0);
        const int cap = (int)std::min<long long>(n_cand, 1 << 22);
        std::vector<uint8_t> n_int(cap), types((size_t)cap * MAXI);
        std::vector<int32_t> prims((size_t)cap * MAXI);
        std::vector<double> s0((size_t)cap * MAXI);
        drt_traced_paths tp{cap, 0, n_int.data(), types.data(), prims.data(), s0.data()};
        if (drt_status st = trace_into(c, *L, tw, max_order, with_tiles != 0, &tp, s)) return st;
        // extrapolated over the window's instants into its rows of H
        const drt_path_set ps{tp.n_found, 0, n_int.data(), types.data(), prims.data(), s0.data()};
        Link W;
        if (drt_status st = load_link(c, &scene, &ps, W)) return st;
        const drt_time_grid tw_grid{tw, tg->dt, k1 - k0, 0};
        drt_status st = synth_into(c, W, &tw_grid, fg, reinterpret_cast<float2 *>(H) + (size_t)k0 * F, precision, s,
                                   nullptr, F);
        cudaError_t e = cudaStreamSynchronize(s);
        free_link(c, W);
        if (st) return st;
        if (e != cudaSuccess) return fail(DRT_ECUDA, "window %d: %s", w, cudaGetErrorString(e));
    }
    return DRT_OK;
}

drt_status drt_profile_enable(drt_ctx *c, int32_t on) {
    if (!c) return fail(DRT_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    c->profiling = on != 0;
    return DRT_OK;
}

drt_status drt_profile_read(drt_ctx *c, int64_t counts[4], double ms[4]) {
    if (!c || !counts || !ms) return fail(DRT_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(c->mu);
    CUDA_TRY(cudaSetDevice(c->device));
    CUDA_TRY(cudaDeviceSynchronize());
    for (int k = 0; k < 4; ++k) {
        counts[k] = 0;
        ms[k] = 0.0;
    }
    drt_status st = DRT_OK;
    for (auto &m : c->marks) {
        float x = 0.f;
        if (cudaEventElapsedTime(&x, m.a, m.b) != cudaSuccess) st = fail(DRT_ECUDA, "cudaEventElapsedTime failed");
        counts[m.kind] += 1;
        ms[m.kind] += x;
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    c->marks.clear();
    return st;
}

drt_status drt_profile_timeline(drt_ctx *c, int32_t cap, int32_t *n, int32_t *kind, double *t0_ms, double *t1_ms) {
    if (!c || !n || cap < 0 || (cap > 0 && (!kind || !t0_ms || !t1_ms))) return fail(DRT_EINVAL, "bad timeline arguments");
    std::lock_guard<std::mutex> lk(c->mu);
    CUDA_TRY(cudaSetDevice(c->device));
    CUDA_TRY(cudaDeviceSynchronize());
    *n = (int32_t)c->marks.size();
    const int m = std::min<int>(cap, (int)c->marks.size());
    for (int i = 0; i < m; ++i) {
        const drt_ctx::Mark &k = c->marks[i];
        float a = 0.f, b = 0.f;
        if (cudaEventElapsedTime(&a, c->marks[0].a, k.a) != cudaSuccess ||
            cudaEventElapsedTime(&b, c->marks[0].a, k.b) != cudaSuccess)
            return fail(DRT_ECUDA, "cudaEventElapsedTime failed");
        kind[i] = k.kind;
        t0_ms[i] = a;
        t1_ms[i] = b;
    }
    return DRT_OK;
}

drt_status drt_probe_peak(drt_ctx *c, int32_t kind, int32_t blocks, double *flops) {
    if (!c || !flops || (kind != 0 && kind != 1) || blocks < 1) return fail(DRT_EINVAL, "bad probe arguments");
    std::lock_guard<std::mutex> lk(c->mu);
    CUDA_TRY(cudaSetDevice(c->device));
    float ms = 0.f;
    CUDA_TRY(launch_probe(kind, blocks, c->probe_sink, 0, &ms));
    const double iters = kind == 0 ? 2048 : 65536;
    *flops = (double)blocks * 256 * iters * 8 * 2 / (ms * 1e-3);
    return DRT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Allocation-free synthesis.  Some callers cannot allocate device memory when they ask for a
// channel prediction: a latency-bound prediction loop cannot afford cudaMalloc / cudaFree, which
// may synchronise the device, and a process whose device memory is already reserved by another
// allocator has none to give.  For them the scratch of drt_synthesize_H (pose table, warm-start
// table of the multi-diffraction chains, synthesis records) lives in this file-scope device array
// instead of context-owned buffers.  Host code never names the array directly: its device address
// comes from cudaGetSymbolAddress with the context's device current, looked up on every call (the
// lookup allocates nothing, and a cached address would go stale if the device were reset).
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[DRT_NOALLOC_SCRATCH_BYTES];

// device address of the static scratch on the current device
drt_status noalloc_scratch(int device, unsigned char **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return fail(DRT_ECUDA, "cudaGetSymbolAddress(scratch) on device %d: %s", device, cudaGetErrorString(e));
    *out = reinterpret_cast<unsigned char *>(p);
    return DRT_OK;
}

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" drt_status drt_synthesize_H_noalloc(drt_ctx *c, uint64_t link, const drt_time_grid *tg,
                                               const drt_freq_grid *fg, void *H, int32_t precision, void *stream) {
    if (!c || !H) return fail(DRT_EINVAL, "ctx and H must be non-NULL");
    if (drt_status st = check_grids(tg, fg, precision)) return st;
    std::lock_guard<std::mutex> lk(c->mu);
    Link *L = find_link(c, link);
    if (!L) return fail(DRT_ENOTFOUND, "unknown link %llu", (unsigned long long)link);
    TimeGridD t = tgd(tg);
    FreqGridD f = fgd(fg);
    size_t pose_bytes = round256((size_t)tg->n_steps * L->dev.n_bodies * POSE_W * sizeof(double));
    size_t warm_sz = round256(warm_bytes(L->dev, t));
    size_t reca_bytes = round256((size_t)tg->n_steps * L->n_paths * sizeof(float4));
    size_t recb_bytes = round256((size_t)tg->n_steps * L->n_paths * sizeof(float));
    size_t need = pose_bytes + warm_sz + reca_bytes + recb_bytes;
    if (need > (size_t)DRT_NOALLOC_SCRATCH_BYTES)
        return fail(DRT_EINVAL,
                    "allocation-free synthesis needs %zu bytes of scratch for %d steps x %d paths x %d bodies, "
                    "more than the %u-byte static array; split the time grid or use drt_synthesize_H",
                    need, tg->n_steps, L->n_paths, L->dev.n_bodies, (unsigned)DRT_NOALLOC_SCRATCH_BYTES);
    CUDA_TRY(cudaSetDevice(c->device));
    unsigned char *base = nullptr;
    if (drt_status st = noalloc_scratch(c->device, &base)) return st;
    double *pose = reinterpret_cast<double *>(base);
    double *warm = reinterpret_cast<double *>(base + pose_bytes);
    RecD rec{reinterpret_cast<float4 *>(base + pose_bytes + warm_sz),
             reinterpret_cast<float *>(base + pose_bytes + warm_sz + reca_bytes)};
    cudaStream_t s = (cudaStream_t)stream;
    OutD none{};
    // the same launches as drt_synthesize_H's FP64 form: pose table, multi-diffraction warm starts,
    // extrapolation into the records, synthesis
    CUDA_TRY(launch_pose(L->dev, t, pose, s));
    CUDA_TRY(launch_warm_fp64(L->dev, t, warm, s));
    CUDA_TRY(launch_extrapolate_fp64(L->dev, t, f, pose, none, rec, s, 0, -1, false, warm));
    CUDA_TRY(launch_synth(rec, L->n_paths, t, f, reinterpret_cast<float2 *>(H), s));
    return DRT_OK;
}

// ---------------------------------------------------------------------------------------------
// a10: batches of links
struct drt_batch {
    drt::BatchPlan *plan = nullptr;
    size_t bytes = 0;
    int32_t n_links = 0;
    float tune_ms = 0.f;
    int32_t chunk_div = 1;                  // chosen divisor of the phase-error model's chunk
    float chunk_ns[3] = {0.f, 0.f, 0.f};    // first wave's preparation + extrapolation, ns per path-step,
                                            // at the model's chunk, 1/2 and 1/4 of it
};

extern "C" drt_status drt_batch_create(drt_ctx *c, int32_t n_links, const uint64_t *links, const drt_time_grid *tgrids,
                                       const drt_freq_grid *fgrids, void *const *H, int32_t precision,
                                       drt_batch **out) {
    if (!c || !out || n_links < 0 || (n_links && (!links || !tgrids || !fgrids || !H)))
        return fail(DRT_EINVAL, "batch: NULL or negative argument");
    if (precision != DRT_FP32_BULK)
        return fail(DRT_EINVAL, "batched synthesis runs the FP32-bulk form (DRT_FP32_BULK); use drt_synthesize_H "
                                "per link for DRT_FP64");
    *out = nullptr;
    std::lock_guard<std::mutex> lk(c->mu);
    std::vector<const LinkDev *> devs(n_links);
    std::vector<drt_scene_view> views(n_links);
    for (int i = 0; i < n_links; ++i) {
        if (drt_status st = check_grids(&tgrids[i], &fgrids[i], precision)) return st;
        Link *L = find_link(c, links[i]);
        if (!L) return fail(DRT_ENOTFOUND, "batch: unknown link %llu", (unsigned long long)links[i]);
        if (!H[i] && tgrids[i].n_steps > 0) return fail(DRT_EINVAL, "batch: H[%d] is NULL", i);
        devs[i] = &L->dev;
        views[i] = L->view;
    }
    CUDA_TRY(cudaSetDevice(c->device));
    // Chunk autotuning: the phase-error model gives each link the longest chunk whose FP32 deltas stay
    // within the phase bar; shorter chunks meet it too (more FP64 anchors, shorter deltas).  Plans with
    // the model's chunk, half and a quarter of it share one allocation (the largest), the first wave's
    // preparation and extrapolation are timed in each (per path-step: the waves may differ), and the
    // fastest plan is kept.
    constexpr int N_DIV = 3;
    const int divs[N_DIV] = {1, 2, 4};
    BatchPlan *cand[N_DIV] = {nullptr, nullptr, nullptr};
    size_t sizes[N_DIV] = {0, 0, 0}, bytes = 0;
    auto drop = [&](int keep) {
        for (int k = 0; k < N_DIV; ++k)
            if (k != keep && cand[k]) batch_free(cand[k]);
    };
    for (int k = 0; k < N_DIV; ++k) {
        cudaError_t e = batch_build(devs, views, tgrids, fgrids, H, nullptr, &cand[k], &sizes[k], divs[k]);
        if (e != cudaSuccess) {
            drop(-1);
            return fail(DRT_ECUDA, "batch planning: %s", cudaGetErrorString(e));
        }
        bytes = std::max(bytes, sizes[k]);
    }
    if (c->budget && c->used + bytes > c->budget) {
        drop(-1);
        return fail(DRT_ENOMEM, "batch needs %zu bytes of scratch; HBM budget %llu, in use %llu", bytes,
                    (unsigned long long)c->budget, (unsigned long long)c->used);
    }
    void *mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, std::max<size_t>(bytes, 256));
    if (e != cudaSuccess) {
        drop(-1);
        return fail(DRT_ENOMEM, "batch allocation of %zu bytes: %s", bytes, cudaGetErrorString(e));
    }
    float ns[N_DIV] = {0.f, 0.f, 0.f};
    int best = 0;
    cudaStream_t s0 = c->side[0];
    for (int k = 0; k < N_DIV && e == cudaSuccess; ++k) {
        e = batch_bind(cand[k], mem, s0);
        if (e == cudaSuccess) e = batch_time_extrapolation(cand[k], s0, &ns[k]);
        if (e == cudaSuccess && ns[k] < ns[best]) best = k;
    }
    drop(best);
    BatchPlan *P = cand[best];
    batch_adopt(P, mem);
    if (e == cudaSuccess) e = batch_bind(P, mem, s0);   // the chosen plan's link table back in place
    if (e == cudaSuccess) e = cudaStreamSynchronize(s0);
    c->used += bytes;
    drt_batch *b = new drt_batch();
    b->plan = P;
    b->bytes = bytes;
    b->n_links = n_links;
    b->chunk_div = divs[best];
    for (int k = 0; k < N_DIV; ++k) b->chunk_ns[k] = ns[k];
    if (e == cudaSuccess) e = batch_autotune(P, s0, &b->tune_ms);
    if (e != cudaSuccess) {
        c->used -= bytes;
        batch_free(P);
        delete b;
        return fail(DRT_ECUDA, "batch autotune: %s", cudaGetErrorString(e));
    }
    *out = b;
    return DRT_OK;
}

extern "C" drt_status drt_batch_tuning(drt_ctx *c, const drt_batch *b, int32_t *chunk_div, float ns_per_step[3]) {
    if (!c || !b) return fail(DRT_EINVAL, "ctx and batch must be non-NULL");
    if (chunk_div) *chunk_div = b->chunk_div;
    if (ns_per_step)
        for (int k = 0; k < 3; ++k) ns_per_step[k] = b->chunk_ns[k];
    return DRT_OK;
}

extern "C" drt_status drt_batch_run(drt_ctx *c, drt_batch *b, int32_t use_graph, void *stream) {
    if (!c || !b) return fail(DRT_EINVAL, "ctx and batch must be non-NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    CUDA_TRY(cudaSetDevice(c->device));
    CUDA_TRY(batch_run(b->plan, (cudaStream_t)stream, use_graph != 0));
    return DRT_OK;
}

extern "C" drt_status drt_batch_info(drt_ctx *c, const drt_batch *b, int32_t *variant, uint64_t *scratch_bytes,
                                     float *tune_ms, int64_t *redo_steps) {
    if (!c || !b) return fail(DRT_EINVAL, "ctx and batch must be non-NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    if (variant) *variant = batch_variant(b->plan);
    if (scratch_bytes) *scratch_bytes = b->bytes;
    if (tune_ms) *tune_ms = b->tune_ms;
    if (redo_steps) {
        long long n = 0;
        CUDA_TRY(cudaSetDevice(c->device));
        CUDA_TRY(cudaDeviceSynchronize());
        bool over = false;
        CUDA_TRY(batch_redo_count(b->plan, &n, &over));
        *redo_steps = n;
        if (over)
            return fail(DRT_ENOMEM, "%lld steps went to the FP64 redo, more than a wave's redo list holds: "
                                    "H of the last run is incomplete", n);
    }
    return DRT_OK;
}

extern "C" void drt_batch_destroy(drt_ctx *c, drt_batch *b) {
    if (!c || !b) return;
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    batch_free(b->plan);
    c->used -= b->bytes;
    delete b;
}

// ---------------------------------------------------------------------------------------------
// a11: serving
static drt_status serve_start_locked(drt_ctx *c, uint64_t pool_bytes, int32_t n_slots, int32_t max_batch) {
    if (c->server) return fail(DRT_EBUSY, "the serving loop is already running");
    if (n_slots < 1 || n_slots > 16 || max_batch < 1) return fail(DRT_EINVAL, "1 <= n_slots <= 16, max_batch >= 1");
    if (!pool_bytes) {   // half of what the budget leaves, at most 16 GiB
        const uint64_t cap = 16ull << 30;
        pool_bytes = c->budget ? std::min<uint64_t>(cap, c->budget > c->used ? (c->budget - c->used) / 2 : 0) : cap;
    }
    if (pool_bytes < (1u << 20)) return fail(DRT_ENOMEM, "no HBM budget left for the serving arena");
    CUDA_TRY(cudaSetDevice(c->device));
    void *arena = nullptr;
    if (drt_status st = dev_alloc(c, pool_bytes, &arena)) return st;
    Server *S = server_start(c->device, arena, pool_bytes, n_slots, max_batch);
    if (!S) {
        dev_free(c, arena, pool_bytes);
        return fail(DRT_ECUDA, "serving streams could not be created");
    }
    c->server = S;
    c->arena = arena;
    c->arena_bytes = pool_bytes;
    return DRT_OK;
}

extern "C" drt_status drt_serve_start(drt_ctx *c, uint64_t pool_bytes, int32_t n_slots, int32_t max_batch) {
    if (!c) return fail(DRT_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    return serve_start_locked(c, pool_bytes, n_slots, max_batch);
}

extern "C" drt_status drt_serve_stop(drt_ctx *c) {
    if (!c) return fail(DRT_EINVAL, "ctx is NULL");
    Server *S;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        S = c->server;
        c->server = nullptr;
    }
    if (!S) return DRT_OK;
    server_stop(S);   // without the ctx lock: completions need none, waiters may hold none
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    dev_free(c, c->arena, c->arena_bytes);
    c->arena = nullptr;
    c->arena_bytes = 0;
    return DRT_OK;
}

extern "C" drt_status drt_submit(drt_ctx *c, const drt_request *req, uint64_t *out_ticket) {
    if (!c || !req || !out_ticket) return fail(DRT_EINVAL, "ctx, req and out_ticket must be non-NULL");
    if (req->precision != DRT_FP32_BULK) return fail(DRT_EINVAL, "served requests run the FP32-bulk form");
    if (drt_status st = check_grids(&req->tgrid, &req->fgrid, req->precision)) return st;
    if (!req->H && req->tgrid.n_steps > 0) return fail(DRT_EINVAL, "request H is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    Link *L = find_link(c, req->link);
    if (!L) return fail(DRT_ENOTFOUND, "unknown link %llu", (unsigned long long)req->link);
    if (!c->server)
        if (drt_status st = serve_start_locked(c, 0, 4, 256)) return st;
    std::string msg;
    if (server_failed(c->server, &msg)) return fail(DRT_ECUDA, "serving loop failed: %s", msg.c_str());
    ServeItem it;
    it.dev = L->dev;
    it.view = L->view;
    it.tg = req->tgrid;
    it.fg = req->fgrid;
    it.H = req->H;
    const drt_path_outputs &o = req->records;
    it.out = OutD{o.tau, o.amp, o.doppler, o.angles, o.flags, o.points};
    it.inflight = L->inflight;
    L->inflight->fetch_add(1);
    *out_ticket = server_submit(c->server, it);
    return DRT_OK;
}

static Server *server_of(drt_ctx *c) {
    std::lock_guard<std::mutex> lk(c->mu);
    return c->server;
}

extern "C" drt_status drt_poll(drt_ctx *c, uint64_t ticket, int32_t *done, drt_result *res) {
    if (!c || !done) return fail(DRT_EINVAL, "ctx and done must be non-NULL");
    Server *S = server_of(c);
    if (!S) return fail(DRT_ENOTFOUND, "no serving loop");
    int r = server_poll(S, ticket, res);
    if (r < 0) return fail(DRT_ENOTFOUND, "unknown or retired ticket %llu", (unsigned long long)ticket);
    *done = r;
    return DRT_OK;
}

extern "C" drt_status drt_wait(drt_ctx *c, uint64_t ticket, uint32_t timeout_ms, drt_result *res) {
    if (!c) return fail(DRT_EINVAL, "ctx is NULL");
    Server *S = server_of(c);
    if (!S) return fail(DRT_ENOTFOUND, "no serving loop");
    int r = server_wait(S, ticket, timeout_ms, res);
    if (r < 0) return fail(DRT_ENOTFOUND, "unknown or retired ticket %llu", (unsigned long long)ticket);
    if (r == 0) return fail(DRT_ETIMEOUT, "ticket %llu not done after %u ms", (unsigned long long)ticket, timeout_ms);
    return DRT_OK;
}

extern "C" drt_status drt_serve_stats_read(drt_ctx *c, drt_serve_stats *out) {
    if (!c || !out) return fail(DRT_EINVAL, "ctx and out must be non-NULL");
    Server *S = server_of(c);
    if (!S) return fail(DRT_ENOTFOUND, "no serving loop");
    server_stats(S, out);
    return DRT_OK;
}
