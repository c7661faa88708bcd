// drt_internal.h -- device-side data layout of a loaded link and the launch interface between the
// C-ABI host code (drt_api.cu) and the kernels (drt_kernels.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <memory>
#include <string>
#include <vector>

#include "../../include/drt.h"

namespace drt {

constexpr int MAXI = 4;
constexpr int POSE_W = 18;   // doubles per (time, body) pose record: R (3x3 row-major), O, v_O, omega

// primitives, positions relative to the owning body's rotation centre o (world axes at t0), so a
// posed position is O(t) + R(t) rel
struct FaceD { double c[3], n[3], u[3], hu, hw; int32_t body, mat; };                       // 96 B
struct EdgeD { double a[3], e[3], t0[3], n0[3], len, wn, snp, cnp; int32_t body, mat, pad0, pad1; };  // 144 B: snp, cnp = sin, cos(wn pi)
struct TileD { double c[3], n[3], area, s, alpha, cph, sph; int32_t body, mat; };          // 96 B: cph + j sph = exp(j phase)
struct MatD { double eps_r, sigma, spec, pec; float eps_rf, sigmaf, specf, pecf; };         // 48 B: spec = sqrt(1 - S^2)
// FP32 copies for the FP32-bulk form (same meaning, no FP64 conversions in its kernels)
struct FaceF { float c[3], n[3], u[3], hu, hw; int32_t body, mat, pad0, pad1, pad2; };          // 64 B
struct EdgeF { float a[3], e[3], t0[3], n0[3], len, wn, snp, cnp; int32_t body, mat; };      // 72 B
struct TileF { float c[3], n[3], area, s, alpha, cph, sph; int32_t body, mat; };            // 52 B
struct TermD { double r[3], v[3], a[3]; };
struct BodyD { double o[3], v[3], a[3], k[3], w0, wdot; };

// one loaded link, passed to kernels by value
struct LinkDev {
    int32_t n_paths, n_bodies, n_faces, n_edges, n_tiles, n_mats;
    int32_t n_bulk;   // paths [0, n_bulk) have at most one diffraction per segment (FP32-bulk capable)
    // among those, paths [len_start[n], len_start[n + 1]) have n vertices (the signature sort groups
    // them by length); the unrolled kernels take lengths 0..3, paths [len_start[MAXI], n_paths) form
    // the generic range (4-vertex chains, then the multi-diffraction chains)
    int32_t len_start[MAXI + 2];
    // the multi-diffraction chains of k + 2 vertices are [multi_start[k], multi_start[k + 1]), k = 0..2
    // (multi_start[0] = n_bulk, multi_start[3] = n_paths)
    int32_t multi_start[MAXI];
    TermD tx, rx;
    const BodyD *bodies;
    const int32_t *body_fixed;   // per body: 1 when it does not move (no velocity, acceleration or rotation)
    const FaceD *faces;
    const EdgeD *edges;
    const TileD *tiles;
    const MatD *mats;
    const FaceF *facesF;
    const EdgeF *edgesF;
    const TileF *tilesF;
    // paths in internal (signature-sorted) order
    const uint32_t *ptypes;   // byte j = type of vertex j (0 past the chain)
    const int4 *pprims;       // primitive index of vertex j
    const double *ps0;        // [P][4] Newton start for segments with >= 2 diffractions
    const int32_t *perm;      // internal index -> caller index
    // per path with >= 2 diffractions in a segment ([n_bulk, n_paths)): its edge parameters and their
    // rates at the scene's reference instant t = 0, solved once when the link is loaded
    const double *t0par;      // [n_paths - n_bulk][2 * MAXI]
};

// chunk: time steps per chunk (FP32-bulk FP64 anchors and multi-diffraction warm starts are taken
// at the first step of every chunk); a power of two in [4, 64]
// grids as kernels see them, with the FP32 constants of the FP32-bulk form derived once on the host
// (per-step FP64 divisions of grid constants would occupy the FP64 pipe of the FP32 kernels)
struct TimeGridD {
    double t_start, dt;
    int32_t n_steps, chunk;
    float dtf;   // dt
};
struct FreqGridD {
    double fc, bandwidth;
    int32_t n_bins;
    float fcf;        // fc
    float f0c, dfc;   // (fc - B/2) / c and B / (n_bins c): first bin and bin step over c (1/m)
    float disp_lim;   // interaction-point displacement since the chunk base past which a step is redone in FP64 (m)
    double f0, df;    // first bin fc - B/2 and bin step B / n_bins (Hz), so that no kernel divides per step
};
inline TimeGridD make_tgrid(double t_start, double dt, int32_t n_steps, int32_t chunk) {
    return TimeGridD{t_start, dt, n_steps, chunk, (float)dt};
}
inline FreqGridD make_fgrid(double fc, double bandwidth, int32_t n_bins) {
    const double c0 = 299792458.0;
    return FreqGridD{fc, bandwidth, n_bins, (float)fc, (float)((fc - 0.5 * bandwidth) / c0),
                     (float)(bandwidth / n_bins / c0), (float)(0.8 * 60e9 / fc), fc - 0.5 * bandwidth,
                     n_bins > 0 ? bandwidth / n_bins : 0.0};
}

// user-visible outputs (caller order), any may be null
struct OutD {
    double *tau;
    void *amp;
    void *doppler;
    float *angles;
    uint8_t *flags;
    double *points;
};

// record consumed by the H synthesis, internal order [T][P]:
//   rec_a = (Re a, Im a, phi0, dhi) and rec_b = dlo, with a = 0 for a path that does not exist at
//   that instant, phi0 = frac(f_0 tau) (cycles), dhi + dlo = frac(df tau) (cycles), where
//   f_0 = fc - B/2 is the first bin and df = B / n_bins; dhi carries the leading 12 bits of the
//   step so that k * dhi is exact in FP32 for k < 4096.
struct RecD { float4 *rec_a; float *rec_b; };

// kinematic bounds of a link used by the batch planner's chunk model: fastest terminal / body
// translation speed (m/s), largest acceleration (m/s^2), largest angular speed (rad/s)
struct drt_scene_view { double vmax, amax, wmax; };

// a10 batch plans (drt_batch.cu)
struct BatchPlan;
// chunk_div: every link's chunk is the phase-error model's choice divided by chunk_div (at least 4 steps)
cudaError_t batch_build(const std::vector<const LinkDev *> &links, const std::vector<drt_scene_view> &views,
                        const drt_time_grid *tgs, const drt_freq_grid *fgs, void *const *H, const OutD *outs,
                        BatchPlan **out, size_t *bytes, int chunk_div = 1);
// device time of the first wave's preparation and extrapolation stages of a bound plan, in ns per
// path-step of that wave
cudaError_t batch_time_extrapolation(BatchPlan *P, cudaStream_t s, float *ns);
void batch_adopt(BatchPlan *P, void *mem);   // the plan, bound to mem, takes ownership of it
cudaError_t batch_bind(BatchPlan *P, void *mem, cudaStream_t s);
cudaError_t batch_alloc(BatchPlan *P);
cudaError_t batch_autotune(BatchPlan *P, cudaStream_t s, float *best_ms);
cudaError_t batch_run(BatchPlan *P, cudaStream_t s, bool use_graph);
cudaError_t batch_free(BatchPlan *P);
int batch_variant(const BatchPlan *P);
void batch_set_variant(BatchPlan *P, int v);
int batch_chunk(const BatchPlan *P, int k);
size_t batch_bytes(const BatchPlan *P);
cudaError_t batch_redo_count(const BatchPlan *P, long long *n, bool *overflow = nullptr);
const unsigned long long *batch_redo_overflow(const BatchPlan *P);
int choose_chunk(const drt_scene_view &v, const drt_time_grid &tg, const drt_freq_grid &fg);

// a11 serving loop (drt_serve.cu): one request as the serving thread sees it
struct ServeItem {
    LinkDev dev;
    drt_scene_view view;
    drt_time_grid tg;
    drt_freq_grid fg;
    void *H;
    OutD out;
    std::shared_ptr<std::atomic<int>> inflight;   // the link's count of pending requests
};
struct Server;
Server *server_start(int device, void *arena, size_t arena_bytes, int n_slots, int max_batch);
void server_stop(Server *S);
bool server_failed(Server *S, std::string *msg);
uint64_t server_submit(Server *S, const ServeItem &item);
int server_poll(Server *S, uint64_t ticket, drt_result *res);
int server_wait(Server *S, uint64_t ticket, uint32_t timeout_ms, drt_result *res);
void server_stats(Server *S, drt_serve_stats *st);

// validated host image of one link, ready for upload (drt_api.cu)
struct PackedLink {
    LinkDev dev{};
    drt_scene_view view{};
    std::vector<BodyD> bodies;
    std::vector<int32_t> body_fixed;
    std::vector<FaceD> faces;
    std::vector<EdgeD> edges;
    std::vector<TileD> tiles;
    std::vector<MatD> mats;
    std::vector<FaceF> facesF;
    std::vector<EdgeF> edgesF;
    std::vector<TileF> tilesF;
    std::vector<uint32_t> ptypes;
    std::vector<int4> pprims;
    std::vector<double> ps0;
    std::vector<int32_t> perm;
};
drt_status pack_link(const drt_scene *s, const drt_path_set *ps, PackedLink &out);

// launchers (drt_kernels.cu); all return cudaError_t of the launch
cudaError_t launch_pose(const LinkDev &L, const TimeGridD &tg, double *pose, cudaStream_t s);
// FP64 per-(path, step) kernel over paths [p0, p1); f32out selects the FP32-bulk output formats
// warm != nullptr: a pre-pass fills warm (warm_bytes) with per-chunk Newton starts for the paths
// [n_bulk, n_paths) first
// multi-diffraction chains [n_bulk, n_paths) run in a launch of their own on s_multi (null: on s; the
// caller orders s_multi after the warm starts and joins it back)
cudaError_t launch_extrapolate_fp64(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg,
                                    const double *pose, const OutD &out, const RecD &rec,
                                    cudaStream_t s, int p0 = 0, int p1 = -1, bool f32out = false,
                                    double *warm = nullptr, cudaStream_t s_multi = nullptr);
size_t warm_bytes(const LinkDev &L, const TimeGridD &tg);
// the warm-start table of the multi-diffraction chains (FP64 dual-number solves at the chunk bases)
// edge parameters and rates at t = 0 of the multi-diffraction paths (LinkDev::t0par), at load
cudaError_t launch_t0par(const LinkDev &L, double *t0par, cudaStream_t s);
cudaError_t launch_warm_fp64(const LinkDev &L, const TimeGridD &tg, double *warm, cudaStream_t s);
// FP32-bulk form (CHUNK consecutive steps share FP64 anchors); see drt_physics.cuh.  Scratch:
// per-(body or terminal, chunk) FP32 base poses and per-(path, chunk) FP64 anchors.
size_t bulk_pose_bytes(const LinkDev &L, const TimeGridD &tg);
size_t bulk_base_bytes(const LinkDev &L, const TimeGridD &tg);
cudaError_t launch_pose_bulk(const LinkDev &L, const TimeGridD &tg, void *poseb, cudaStream_t s);
size_t bulk_pose64_bytes(const LinkDev &L, const TimeGridD &tg);
size_t bulk_redo_bytes(const LinkDev &L, const TimeGridD &tg);
// FP32-bulk anchors in parts: FP64 poses at the chunk bases, then the anchors of paths [p0, p1) (the
// multi-diffraction paths [n_bulk, n_paths) need their warm starts, launch_warm_fp64, first)
cudaError_t launch_base_pose64(const LinkDev &L, const TimeGridD &tg, double *pose64, cudaStream_t s);
cudaError_t launch_base_paths(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, const double *pose64,
                              void *base, const double *warm, int p0, int p1, cudaStream_t s);
// the redo scratch holds an int counter (zeroed here, on s, when zero is set) followed by the
// (path, step) list; lengths / generic select the launches of chain lengths 0..3 (on s) and of the
// generic range (on s_multi, else s)
cudaError_t launch_extrapolate_bulk(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, const void *poseb,
                                    const void *base, const double *warm, const OutD &out, const RecD &rec,
                                    void *redo, cudaStream_t s, cudaStream_t s_multi = nullptr, bool lengths = true,
                                    bool generic = true, bool zero = true);
cudaError_t launch_redo(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, const OutD &out, const RecD &rec,
                        void *redo, const double *warm, cudaStream_t s);
// the redo for an H synthesis: (Re a, Im a, tau) per queued step into out3 ([cap][3] doubles), then
// added into H after the synthesis
cudaError_t launch_redo_rec(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, void *redo, const double *warm,
                            double *out3, cudaStream_t s);
cudaError_t launch_redo_add(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, void *redo, const double *in3,
                            float2 *H, cudaStream_t s, int ld = -1);
// multipath lifetime: per-instant total |a|^2 of the valid paths (tot[T]) and major validity changes
// (major[T], 1 at instant n when a path with >= share of the power at its valid side changes validity)
cudaError_t launch_lifetime(bool fp64, const OutD &rec, int n_steps, int n_paths, double share, double *tot,
                            uint8_t *major, cudaStream_t s);
// T_C windows: window w starts at step starts[w] (starts[0] = 0, increasing); sel is [T][P] (caller
// path order) and holds, in the rows of the window starts, the path's FP64 flags at that instant
// (0: in the window's multipath); launch_select writes those rows
struct WinMask {
    const int32_t *starts;
    int32_t n_w;
    uint8_t *sel;
};
cudaError_t launch_select(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, const WinMask &wm,
                          const double *warm, cudaStream_t s);
cudaError_t launch_window_mask(const LinkDev &L, const TimeGridD &tg, const RecD &rec, const WinMask &wm,
                               cudaStream_t s);
cudaError_t launch_redo_window_mask(const LinkDev &L, const TimeGridD &tg, void *redo, const WinMask &wm, double *in3,
                                    cudaStream_t s);
// histogram of |a|^2 over (time bin, Doppler (kind 0) or delay (kind 1) bin) from [T][P] records;
// out[n_time_bins][n_bins] is written whole (FP64)
cudaError_t launch_power_bin(bool fp64, const OutD &rec, int n_steps, int n_paths, int steps_per_bin, double x0,
                             double dx, int n_bins, int kind, double *out, cudaStream_t s);
// H rows of ld elements (ld < 0: n_bins), bins written at H[t * ld + k]
cudaError_t launch_synth(const RecD &rec, int32_t n_paths, const TimeGridD &tg, const FreqGridD &fg,
                         float2 *H, cudaStream_t s, int ld = -1);
cudaError_t launch_probe(int kind, int blocks, double *sink, cudaStream_t s, float *ms);
// conventional ray tracing at an instant (drt_trace.cu): candidates of the enumeration, sizes of the
// scratch records (faces posed at the instant, rays found), the launch, and the host-side unpacking of
// `count` rays into path-set arrays in enumeration order
long long trace_candidates(const LinkDev &L, int max_order, int with_tiles);
size_t trace_ray_bytes();
size_t trace_face_bytes();
cudaError_t launch_trace(const LinkDev &L, double t, int max_order, int with_tiles, void *faces, void *rays, int cap,
                         int *count, cudaStream_t s);
void trace_unpack(const void *rays_host, int count, uint8_t *n_int, uint8_t *types, int32_t *prims, double *s0,
                  int cap);

}  // namespace drt
