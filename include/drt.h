/*
 * drt.h -- C ABI of the GB300 Dynamic Ray Tracing (DRT) hot path.
 *
 * Method: Bilibashi, Vitucci, Degli-Esposti, "On Dynamic Ray Tracing and Anticipative Channel
 * Prediction for Dynamic Environments".  Given the multipath geometry of one ray-tracing run at t0
 * (Sec. II: chains of specular reflections, edge diffractions and diffuse-scattering tiles) and the
 * kinematics of terminals and rigid bodies (Eq. Taylor, Sec. III-A), the library extrapolates every
 * path to t0 + dt (Sec. III) and synthesises the time-varying channel
 *     H(t, f) = sum_p a_p(t) exp(-j 2 pi f tau_p(t))
 * from the per-path complex amplitudes a_p and delays tau_p ("time-variant channel's transfer
 * function", Sec. II).
 *
 * Conventions
 *   - SI units; time-harmonic convention exp(+j w t); c = 299792458 m/s.
 *   - Times are seconds after t0: t_n = t_start + n dt, n = 0 .. n_steps-1.
 *   - Frequencies f_k = fc - bandwidth/2 + k bandwidth/n_bins; coefficients are evaluated at fc.
 *   - Per-(time-step, path) outputs are row-major [n_steps][n_paths] (path index fastest) in the
 *     caller's path order.
 *   - Antennas are isotropic and vertically polarised (vertical projected transverse to the ray,
 *     x if the ray is vertical); line of sight gives a = lambda / (4 pi d).
 *   - Every call returns a drt_status; the message of the last failure on the calling thread is
 *     available from drt_last_error().  Per-result conditions (a point left its face or edge, a
 *     Newton solve did not converge, ...) are reported as flag bits in the outputs, never as call
 *     errors.
 *   - Device pointers are CUDA global-memory pointers on the context's device; `stream` is a
 *     cudaStream_t (NULL = legacy default stream).  Calls on one context are serialised internally;
 *     device work is ordered on the given stream and the call returns without synchronising unless
 *     stated otherwise.
 *   - No CPU fallback: without a usable device, drt_create fails with DRT_ECUDA.
 */
#ifndef DRT_H
#define DRT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct drt_ctx drt_ctx;
typedef int32_t drt_status;

#define DRT_OK 0
#define DRT_EINVAL (-1)     /* malformed argument (message says which)                        */
#define DRT_ENOMEM (-2)     /* device allocation failed or the HBM budget would be exceeded   */
#define DRT_ECUDA (-3)      /* a CUDA runtime call failed                                     */
#define DRT_EBUSY (-4)      /* no serving slot / budget free right now                        */
#define DRT_ETIMEOUT (-5)   /* a bounded wait expired                                         */
#define DRT_ENOTFOUND (-6)  /* unknown link or ticket                                         */

/* interaction types of a chain vertex (Sec. II, Fig. ray_path) */
#define DRT_T_NONE 0
#define DRT_T_R 1   /* specular reflection on a face (Sec. III-A)              */
#define DRT_T_D 2   /* UTD edge diffraction (Sec. III-B)                        */
#define DRT_T_S 3   /* diffuse scattering from a tile centroid (Sec. III-C)     */
#define DRT_MAX_INT 4

/* per-(time-step, path) flag bits; 0 means the path exists at that instant (the multipath
 * structure of the t0 run still holds, Sec. II "multipath lifetime") */
#define DRT_F_FACE 1     /* a reflection point lies outside its face rectangle                    */
#define DRT_F_EDGE 2     /* a diffraction point lies outside its edge segment                     */
#define DRT_F_SIDE 4     /* a neighbour of a vertex is behind its face / inside its wedge / behind its tile */
#define DRT_F_NOCONV 8   /* the Newton solve of a segment with >= 2 diffractions did not converge */
#define DRT_F_DEGEN 16   /* a zero-length segment or a degenerate diffraction geometry            */

/* precision of a call */
#define DRT_FP64 0        /* all per-path-step geometry, field and Doppler work in FP64           */
#define DRT_FP32_BULK 1   /* FP32 work on deltas from per-chunk FP64 bases (delay, phase anchors) */

/* ---- dynamic environment database (Sec. II); all positions in world coordinates at t0 ---- */
typedef struct { double o[3], v[3], a[3], k[3], w0, wdot; } drt_body;      /* 112 B: rotation centre o,
    its velocity v and constant acceleration a (Eq. Taylor), fixed unit rotation axis k, angular
    speed w0 at t0 and constant angular acceleration wdot (theta(t) = w0 dt + wdot dt^2 / 2).
    Body 0 is conventionally the static world. */
typedef struct { double r[3], v[3], a[3]; } drt_terminal;                 /* 72 B, Eq. Taylor */
typedef struct { double eps_r, sigma, rough_s, pec; } drt_material;       /* 32 B: relative
    permittivity, conductivity (S/m), ER roughness of the face (specular term scaled by
    sqrt(1 - S^2)), perfect conductor if pec != 0 */
typedef struct { int32_t body, material; double c[3], n[3], u[3], hu, hw; } drt_face;  /* 96 B:
    rectangle centred at c with unit outward normal n, in-plane unit axis u and half-extents hu
    along u and hw along u x n; hu = hw = +inf for an unbounded plane */
typedef struct { int32_t body, material; double a[3], b[3], n0[3], nn[3], wedge_n; } drt_edge; /*
    112 B: wedge edge from a to b; n0 / nn are the outward normals of the 0-face and the n-face,
    ordered so that (b - a) is parallel to n0 x nn; exterior wedge angle wedge_n * pi */
typedef struct { int32_t body, material; double c[3], n[3], area, s, alpha_r, phase; } drt_tile; /*
    88 B: ER scattering tile (centroid c, unit normal n, area, scattering parameter S, integer lobe
    exponent alpha_R in 0..16, constant phase (rad)) */

typedef struct {
    drt_terminal tx, rx;
    int32_t n_bodies, n_materials, n_faces, n_edges, n_tiles, reserved;
    const drt_body *bodies;
    const drt_material *materials;
    const drt_face *faces;
    const drt_edge *edges;
    const drt_tile *tiles;
} drt_scene;   /* host pointers; copied by drt_load_paths */

/* ray chains of one link (the t0 ray-tracing result): vertex j of path p has type types[p*4+j]
 * and primitive prims[p*4+j] (face / edge / tile index); s0[p*4+j] is the t0 edge parameter (m
 * from edge point a) of a diffraction vertex, used as the starting point of the Newton solve of a
 * segment with two or more diffractions (may be NULL: edge midpoints). */
typedef struct {
    int32_t n_paths, reserved;
    const uint8_t *n_int;     /* [P] number of interactions, 0..4 */
    const uint8_t *types;     /* [P][4]                            */
    const int32_t *prims;     /* [P][4]                            */
    const double *s0;         /* [P][4] or NULL                    */
} drt_path_set;   /* host pointers; copied by drt_load_paths */

typedef struct { double t_start, dt; int32_t n_steps, reserved; } drt_time_grid;
typedef struct { double fc, bandwidth; int32_t n_bins, reserved; } drt_freq_grid;

/* caller-owned DEVICE buffers, [n_steps][n_paths] unless stated; any member may be NULL */
typedef struct {
    double *tau;     /* delay (s), path length / c                                            */
    void *amp;       /* complex amplitude a_p (re, im): double[2] for DRT_FP64, float[2] for   */
                     /* DRT_FP32_BULK; excludes the propagation phase exp(-j 2 pi f tau)      */
    void *doppler;   /* Doppler shift f' - fc (Hz), App. A Eq. doppler_freq: double / float    */
    float *angles;   /* [T][P][4]: AoD azimuth, AoD elevation, AoA azimuth, AoA elevation (rad) */
    uint8_t *flags;  /* DRT_F_* bits                                                           */
    double *points;  /* [T][P][4][3] interaction points (m), NaN past the chain's length        */
} drt_path_outputs;

/* ---------------------------------------------------------------------------------------------
 * Context.  drt_create binds `device`, creates the context's streams and sets the HBM budget
 * (bytes of device memory the context may hold for links and scratch; 0 = no limit).
 * Errors: DRT_EINVAL (out == NULL), DRT_ECUDA (no such device / CUDA failure).
 * drt_destroy frees everything the context owns; NULL is ignored.  drt_last_error returns the
 * message of the last failing call on this thread (valid until the next call on this thread). */
drt_status drt_create(drt_ctx **out, int32_t device, uint64_t hbm_budget_bytes);
void drt_destroy(drt_ctx *ctx);
const char *drt_last_error(void);

/* ---------------------------------------------------------------------------------------------
 * a1 load / stage (Sec. II: dynamic environment database + t0 ray-tracing result).  Validates the
 * scene and paths (indices in range, unit normals and axes, edge ordering, finite values, integer
 * alpha_R), packs them into the device's structure-of-arrays layout (paths reordered by chain
 * signature internally; outputs keep the caller's order) and copies them to the device.  Inputs
 * are copied, so the caller may free them on return.  *out_link receives a handle valid until
 * drt_unload.  Synchronous.  Errors: DRT_EINVAL, DRT_ENOMEM (budget or cudaMalloc), DRT_ECUDA. */
drt_status drt_load_paths(drt_ctx *ctx, const drt_scene *scene, const drt_path_set *paths,
                          uint64_t *out_link);
drt_status drt_unload(drt_ctx *ctx, uint64_t link);

/* ---------------------------------------------------------------------------------------------
 * a2-a8: extrapolate every path of `link` over the time grid (Sec. III-A reflection points by the
 * image method and back-tracking, Eq. ref_point; Sec. III-B diffraction points on the Keller cone,
 * Eq. diff_point; Sec. III-C rigid scattering tiles), with delay, departure / arrival angles,
 * Doppler (App. A Eq. doppler_freq, interaction-point velocities), validity flags and the complex
 * amplitude (Fresnel, UTD, ER and ray spreading at fgrid->fc; only fgrid->fc is used).  Writes the
 * non-NULL members of *out (device buffers sized for [tgrid->n_steps][n_paths]).
 * Errors: DRT_EINVAL (bad grid / precision), DRT_ENOTFOUND (link), DRT_ECUDA. */
drt_status drt_extrapolate(drt_ctx *ctx, uint64_t link, const drt_time_grid *tgrid,
                           const drt_freq_grid *fgrid, const drt_path_outputs *out,
                           int32_t precision, void *stream);

/* ---------------------------------------------------------------------------------------------
 * a2-a9: the whole hot path: extrapolation as above into context-owned scratch, then
 * H[t][k] = sum over valid paths of a_p(t) exp(-j 2 pi f_k tau_p(t)).  H is a caller-owned DEVICE
 * buffer of [tgrid->n_steps][fgrid->n_bins] complex64 (float re, im), in both precisions (the
 * synthesis accumulates in FP32 from phases reduced in FP64).  Scratch grows on demand within the
 * HBM budget.  Errors: DRT_EINVAL, DRT_ENOTFOUND, DRT_ENOMEM, DRT_ECUDA. */
drt_status drt_synthesize_H(drt_ctx *ctx, uint64_t link, const drt_time_grid *tgrid,
                            const drt_freq_grid *fgrid, void *H, int32_t precision, void *stream);

/* Same as drt_synthesize_H with H in HOST memory (pinned or pageable): the result is copied to
 * the host on `stream` and the call synchronises the stream before returning. */
drt_status drt_synthesize_H_host(drt_ctx *ctx, uint64_t link, const drt_time_grid *tgrid,
                                 const drt_freq_grid *fgrid, void *H_host, int32_t precision,
                                 void *stream);

/* Allocation-free variant of drt_synthesize_H (no counterpart in the paper; it exists for callers
 * that cannot allocate device memory at call time: latency-bound anticipative-prediction loops,
 * where cudaMalloc / cudaFree may synchronise the device and stall for milliseconds, and processes
 * whose device memory is already fully reserved by another allocator).  Same inputs, output and
 * result as drt_synthesize_H's FP64 form (the same launches), but the pose table, the warm-start
 * table of the chains with several diffractions in one segment and the synthesis records live in one
 * static device array of DRT_NOALLOC_SCRATCH_BYTES (32 MiB) that the library reserves on every
 * device that loads it, until the process exits; the call makes no cudaMalloc, cudaFree or other
 * allocating call.  `precision` is checked, and the synthesis runs the FP64 form, whose result
 * meets the tolerances of both forms.  It needs 144 n_steps n_bodies + 64 n_multi (ceil(n_steps / 16)
 * + 1) + 20 n_steps n_paths bytes (n_multi = chains with two or more diffractions in a segment;
 * each part rounded up to 256 B) and fails with DRT_EINVAL when that exceeds the array.  Every call
 * looks up the array's device address (cudaGetSymbolAddress) with the context's device current,
 * which allocates nothing; make the first call on a device before any stream capture, since the
 * runtime may load the library's device code there.  Every call on a device shares the array and
 * nothing in it needs to start at zero (each call writes the pose table, warm starts and records
 * before reading them); calls whose device work overlaps (different streams, or different contexts
 * on the same device) race on it, so order them on one stream or serialise them.
 * Errors: DRT_EINVAL, DRT_ENOTFOUND, DRT_ECUDA. */
#define DRT_NOALLOC_SCRATCH_BYTES (32u << 20)
drt_status drt_synthesize_H_noalloc(drt_ctx *ctx, uint64_t link, const drt_time_grid *tgrid,
                                    const drt_freq_grid *fgrid, void *H, int32_t precision,
                                    void *stream);

/* ---------------------------------------------------------------------------------------------
 * Power-Doppler profile (PDfP, Sec. IV-A) and power-delay profile (PDP, Sec. IV-B) of a link:
 * P[i][j] = sum of |a_p(t)|^2 over the valid path-steps whose instant t_n falls in time bin
 * i = n / steps_per_bin (the last bin may be ragged) and whose Doppler shift f' - fc (Hz, App. A
 * Eq. doppler_freq; kind DRT_PP_DOPPLER) or delay tau (s; kind DRT_PP_DELAY) falls in bin
 * j = floor((x - x0) / dx), 0 <= j < n_bins (the paper bins 200 ms x 14.34 Hz).  The whole path
 * runs on the device: extrapolation with records into context scratch, then one block per time bin
 * adds its path-steps into a shared-memory histogram.  P is a caller-owned DEVICE buffer of
 * ceil(n_steps / steps_per_bin) x n_bins doubles, written whole (may be NULL when n_steps is 0);
 * 1 <= n_bins <= 4096, dx > 0.
 * Errors: DRT_EINVAL (grids), DRT_ENOTFOUND, DRT_ENOMEM, DRT_ECUDA. */
#define DRT_PP_DOPPLER 0
#define DRT_PP_DELAY 1
typedef struct { int32_t steps_per_bin, n_bins; double x0, dx; int32_t kind, reserved; } drt_power_grid;
drt_status drt_power_profile(drt_ctx *ctx, uint64_t link, const drt_time_grid *tgrid,
                             const drt_freq_grid *fgrid, const drt_power_grid *grid, double *P,
                             int32_t precision, void *stream);

/* ---------------------------------------------------------------------------------------------
 * Wideband coefficients: H(t, f) with the field coefficients (Fresnel with eps_c(f), UTD with k(f),
 * ER, lambda / 4 pi; Sec. III-A to III-C) evaluated per sub-band instead of once at fc.  The n_bins
 * bins split into n_sub sub-bands of near-equal size, [k0, k1) with k0 = s n_bins / n_sub (integer
 * division); sub-band s spans [f_k0, f_k0 + (k1 - k0) df) of the grid f_k = fc - B/2 + k B/n_bins,
 * df = B / n_bins, and its coefficients are taken at the centre of that span (n_sub = 1 is
 * drt_synthesize_H).  Each sub-band runs its own extrapolation (the geometry is repeated) and
 * synthesis into its columns of H.  H: caller-owned DEVICE buffer [n_steps][n_bins] complex64.
 * Asynchronous on `stream`.  Errors: DRT_EINVAL (grids, 1 <= n_sub <= n_bins), DRT_ENOTFOUND,
 * DRT_ENOMEM, DRT_ECUDA. */
drt_status drt_synthesize_H_wideband(drt_ctx *ctx, uint64_t link, const drt_time_grid *tgrid,
                                     const drt_freq_grid *fgrid, int32_t n_sub, void *H,
                                     int32_t precision, void *stream);

/* ---------------------------------------------------------------------------------------------
 * Multipath lifetime T_C management (Sec. II: extrapolation holds while no major path appears or
 * disappears; Sec. IV-B divides a span into T_C windows, long where the multipath is stable and short
 * near LoS/NLoS transitions, and re-initialises the multipath at every window start).
 *
 * drt_lifetime_windows: expiry criterion and window plan of `link` over the time grid.  Step n >= 1
 * is a major change when some path is valid at one of the instants n - 1, n and not at the other
 * while, at the instant where it is valid, its |a|^2 is at least params->share of the total |a|^2 of
 * the valid paths of that instant.  A window starting at step w ends at the first major change in
 * [w + min_steps, w + max_steps], else after max_steps steps.  Writes the window starts (steps,
 * starts[0] = 0) to the HOST array `starts` (cap entries), their count to *n_windows (0 when
 * n_steps = 0) and, if `major` is non-NULL, the per-step major flags to the HOST array major[n_steps].
 * Runs the extrapolation (amplitudes and flags, `precision` form) and two reduction kernels on
 * `stream`, then waits for it.  Errors: DRT_EINVAL (params: finite share >= 0,
 * 1 <= min_steps <= max_steps; or cap smaller than the window count, which is then in *n_windows),
 * DRT_ENOTFOUND, DRT_ENOMEM, DRT_ECUDA. */
typedef struct { double share; int32_t min_steps, max_steps; } drt_lifetime_params;
drt_status drt_lifetime_windows(drt_ctx *ctx, uint64_t link, const drt_time_grid *tgrid,
                                const drt_freq_grid *fgrid, const drt_lifetime_params *params,
                                int32_t precision, uint8_t *major, int32_t *starts, int32_t cap,
                                int32_t *n_windows, void *stream);

/* drt_synthesize_H_windows: H(t, f) of DRT over the span divided into T_C windows that start at the
 * HOST steps starts[0..n_windows) (starts[0] = 0, strictly increasing, < n_steps).  Each window's
 * multipath is the set of paths valid at its first instant (FP64 validity at that instant, as a
 * ray-tracing run there would return it); a path outside that set contributes nothing until the next
 * window, even where it becomes valid inside this one.  One window at every step gives
 * drt_synthesize_H.  H: caller-owned DEVICE buffer [n_steps][n_bins] complex64, as drt_synthesize_H.
 * Asynchronous on `stream` (starts is copied before the call returns).
 * Errors: DRT_EINVAL (grids, starts), DRT_ENOTFOUND, DRT_ENOMEM, DRT_ECUDA. */
drt_status drt_synthesize_H_windows(drt_ctx *ctx, uint64_t link, const drt_time_grid *tgrid,
                                    const drt_freq_grid *fgrid, const int32_t *starts,
                                    int32_t n_windows, void *H, int32_t precision, void *stream);

/* ---------------------------------------------------------------------------------------------
 * Conventional ray tracing at one instant (Sec. II: the ray-tracing run DRT starts from at t0; Sec.
 * IV-B: it is run again at the start of every multipath-lifetime window) over the scene of a loaded
 * link, whose own chains are not used.  Brute-force image-tree enumeration on the device: every chain
 * of at most max_order (0, 1 or 2) reflections / diffractions with no primitive twice in a row and,
 * when with_tiles != 0, every single-tile scattering chain, posed at t (seconds after t0), is solved
 * with the extrapolation's FP64 geometry (image method and back-tracking, Keller cone, Newton from the
 * edge midpoints for two diffractions in one segment) and kept when its FP64 validity flags are 0 and
 * no face of the scene blocks any of its segments (a face blocks a segment that crosses its plane
 * strictly between the segment's ends inside its rectangle; a face whose plane holds an end of the
 * segment -- the face a reflection point or a tile lies on, the faces of a diffracting edge -- does
 * not).  Candidates are enumerated as the line of sight, then faces (reflections), edges
 * (diffractions) and tiles (scattering), then ordered pairs of faces and edges; the rays found are
 * written to the caller's HOST arrays in that order, at most cap of them, with the edge parameter
 * (m from edge point a) of each diffraction point at t in s0, so that the result loads as a link's
 * path set (drt_load_paths).  n_found receives the number found (above cap, only the first cap were
 * written).  Runs on `stream` and waits for it.  Errors: DRT_EINVAL, DRT_ENOTFOUND, DRT_ENOMEM (more
 * than 2^22 rays), DRT_ECUDA. */
typedef struct {
    int32_t cap, n_found;
    uint8_t *n_int;      /* [cap]    */
    uint8_t *types;      /* [cap][4] */
    int32_t *prims;      /* [cap][4] */
    double *s0;          /* [cap][4] */
} drt_traced_paths;
drt_status drt_trace_paths(drt_ctx *ctx, uint64_t link, double t, int32_t max_order, int32_t with_tiles,
                           drt_traced_paths *out, void *stream);

/* DRT with a ray-tracing run at every window start, the paper's procedure over a span (Sec. II,
 * Sec. IV-B): the span divides into T_C windows starting at the HOST steps starts[0..n_windows)
 * (starts[0] = 0, strictly increasing, < n_steps); window w takes the chains of drt_trace_paths at its
 * first instant t_start + starts[w] dt (max_order, with_tiles as there), extrapolates them over its
 * instants and synthesises its rows of H (caller-owned DEVICE buffer [n_steps][n_bins] complex64, as
 * drt_synthesize_H; `precision` selects the form).  A ray that appears inside a window is found at the
 * next window start.  Each window's chains go to the host to be packed into a temporary link, so the
 * call is synchronous.  Errors: DRT_EINVAL, DRT_ENOTFOUND, DRT_ENOMEM, DRT_ECUDA. */
drt_status drt_synthesize_H_retraced(drt_ctx *ctx, uint64_t link, const drt_time_grid *tgrid,
                                     const drt_freq_grid *fgrid, const int32_t *starts, int32_t n_windows,
                                     int32_t max_order, int32_t with_tiles, void *H, int32_t precision,
                                     void *stream);

/* ---------------------------------------------------------------------------------------------
 * a10: batched synthesis over many resident links (FP32-bulk form).  drt_batch_create plans one
 * batch: link i is synthesised over tgrids[i] x fgrids[i] into the caller's DEVICE buffer H[i]
 * ([n_steps][n_bins] complex64).  Each stage (base poses, FP64 chunk poses, multi-diffraction warm
 * starts, FP64 chunk anchors, FP32-bulk extrapolation, H synthesis, FP64 redo) is one persistent
 * launch over the (link, work unit) pairs of all links, claimed with atomic counters, largest links
 * first, so uneven links (8 to thousands of paths, 100 to thousands of steps) share one launch per
 * stage.  Extrapolation and synthesis stream through a record buffer of at most 4 GiB in waves of
 * links.  The chunk length per link comes from a phase-error model, shortened by a factor 1, 2 or 4
 * chosen by timing the first wave's preparation and extrapolation (drt_batch_tuning), and the
 * synthesis frequency tile (bins per thread) from timing its variants on the batch (autotuning,
 * done synchronously inside drt_batch_create).  Scratch is allocated once per batch within the HBM budget.  The links
 * must stay loaded and the H buffers valid while the batch exists.
 * drt_batch_run launches the batch on `stream`; with use_graph != 0 the first run is captured into
 * a CUDA graph (captured on a stream of the batch, so any stream can replay it) and later runs
 * replay it.  precision must be DRT_FP32_BULK.
 * Errors: DRT_EINVAL, DRT_ENOTFOUND, DRT_ENOMEM, DRT_ECUDA. */
typedef struct drt_batch drt_batch;
drt_status drt_batch_create(drt_ctx *ctx, int32_t n_links, const uint64_t *links,
                            const drt_time_grid *tgrids, const drt_freq_grid *fgrids, void *const *H,
                            int32_t precision, drt_batch **out);
drt_status drt_batch_run(drt_ctx *ctx, drt_batch *batch, int32_t use_graph, void *stream);
/* chosen synthesis variant (frequency tile of 0: 8, 1: 16, 2: 32 bins per thread), scratch
 * bytes, the autotuner's best sample time (ms) and the path-steps of the last run that FP32 could
 * not resolve and the FP64 redo kernel recomputed (reading it waits for the device); any output
 * may be NULL.  With redo_steps non-NULL the call returns DRT_ENOMEM when a wave of the last run
 * queued more redo steps than its list holds (2^22 + 1/128 of the wave's path-steps, or the value
 * of the environment variable DRT_BATCH_REDO_CAP when that is smaller, read when a plan is built):
 * that run's H is then incomplete. */
drt_status drt_batch_info(drt_ctx *ctx, const drt_batch *batch, int32_t *variant,
                          uint64_t *scratch_bytes, float *tune_ms, int64_t *redo_steps);
/* the chunk length drt_batch_create chose: every link's chunk is the phase-error model's choice
 * divided by *chunk_div (1, 2 or 4; at least 4 steps), the fastest of the three in ns_per_step
 * (device time of the first wave's preparation and extrapolation over its path-steps, with the
 * model's chunk, half and a quarter of it; 0 for a batch without path-steps); either output may be
 * NULL.  Errors: DRT_EINVAL. */
drt_status drt_batch_tuning(drt_ctx *ctx, const drt_batch *batch, int32_t *chunk_div, float ns_per_step[3]);
void drt_batch_destroy(drt_ctx *ctx, drt_batch *batch);

/* ---------------------------------------------------------------------------------------------
 * a11: serving.  The context runs one serving thread that takes anticipative-prediction requests
 * (Sec. II: the multipath of a loaded link predicted over [t_start, t_start + n_steps dt)) from
 * any thread, admits them by HBM footprint into an arena of `pool_bytes` reserved within the
 * context's budget, and batches whatever is queued whenever one of `n_slots` streams is free
 * (continuous batching, at most `max_batch` requests per launch), so requests that arrive while
 * others run start as soon as a slot and arena memory free up and overlap with them on the device.
 * Requests run the FP32-bulk batched form (drt_batch_create); each result depends only on its own
 * request, not on the batch it ran in.  drt_serve_start is optional: the first drt_submit starts
 * the loop with pool_bytes = min(half the free budget, 16 GiB), 4 slots, 256 requests per launch.
 * Errors: DRT_EINVAL, DRT_EBUSY (already started), DRT_ENOMEM (arena beyond the budget),
 * DRT_ECUDA. */
typedef struct {
    uint64_t link;
    drt_time_grid tgrid;
    drt_freq_grid fgrid;
    void *H;                    /* DEVICE [n_steps][n_bins] complex64, caller-owned, required    */
    drt_path_outputs records;   /* optional DEVICE records [n_steps][n_paths] in the FP32-bulk    */
                                /* formats (tau double, amp float[2], doppler float); NULL = skip */
    int32_t precision;          /* DRT_FP32_BULK                                                  */
    int32_t reserved;
} drt_request;
typedef struct {
    drt_status status;          /* DRT_OK; DRT_ENOMEM when the request is larger than the arena, */
                                /* or when its batch queued more FP64 redo steps than the redo    */
                                /* list holds (H then misses them); DRT_EINVAL when the batch     */
                                /* could not be planned; DRT_ECUDA                                */
    int32_t batch_requests;     /* requests in the launch that served this one                    */
    double t_submit, t_launch, t_done;   /* seconds on the library's steady clock                 */
} drt_result;
typedef struct {
    uint64_t submitted, completed, launches, queued, in_flight;
    uint64_t arena_bytes, arena_used, arena_peak;
} drt_serve_stats;
drt_status drt_serve_start(drt_ctx *ctx, uint64_t pool_bytes, int32_t n_slots, int32_t max_batch);
/* finishes every submitted request, then ends the loop and frees the arena (drt_destroy calls it) */
drt_status drt_serve_stop(drt_ctx *ctx);
/* copies the request and returns a ticket at once; the link must stay loaded (drt_unload answers
 * DRT_EBUSY while it has pending requests) and H / records valid until the request is done.
 * Errors: DRT_EINVAL, DRT_ENOTFOUND (link), DRT_ECUDA (the serving loop failed earlier). */
drt_status drt_submit(drt_ctx *ctx, const drt_request *req, uint64_t *out_ticket);
/* *done = 1 and *res filled once the request is finished (the ticket is then retired; res may
 * be NULL); *done = 0 while pending.  Errors: DRT_ENOTFOUND (unknown or retired ticket). */
drt_status drt_poll(drt_ctx *ctx, uint64_t ticket, int32_t *done, drt_result *res);
/* blocks until the request is finished (DRT_OK, ticket retired) or timeout_ms passes
 * (DRT_ETIMEOUT, ticket kept).  Errors: DRT_ENOTFOUND, DRT_ETIMEOUT. */
drt_status drt_wait(drt_ctx *ctx, uint64_t ticket, uint32_t timeout_ms, drt_result *res);
drt_status drt_serve_stats_read(drt_ctx *ctx, drt_serve_stats *out);

/* Number of paths of a link (for sizing outputs).  Errors: DRT_ENOTFOUND. */
drt_status drt_link_info(drt_ctx *ctx, uint64_t link, int32_t *n_paths);

/* ---------------------------------------------------------------------------------------------
 * Tracing.  While enabled, every kernel the context launches is bracketed by CUDA events recorded
 * on the launch stream.  drt_profile_read synchronises the device and returns, per kernel kind
 * (0 = pose table, 1 = extrapolation, 2 = H synthesis, 3 = FP64 chunk anchors and FP64 redo of
 * the FP32-bulk form), the number of launches and
 * their summed device time in ms since the previous read, then clears the record.
 * Errors: DRT_EINVAL (NULL arguments), DRT_ECUDA. */
drt_status drt_profile_enable(drt_ctx *ctx, int32_t on);
drt_status drt_profile_read(drt_ctx *ctx, int64_t counts[4], double ms[4]);

/* The same record as a timeline: for each bracketed launch group since the last drt_profile_read,
 * in the order the groups were issued, its kind (as above) and its start and end in ms after the
 * start of the first group.  A group is one kernel, or one stage whose launches fork onto the
 * context's side streams and join back before its closing event.  Writes min(cap, count) entries
 * into the caller's host arrays kind, t0_ms, t1_ms (each of cap elements) and the count to *n; does
 * not clear the record.  Synchronises the device.  Errors: DRT_EINVAL (NULL arguments, cap < 0),
 * DRT_ECUDA. */
drt_status drt_profile_timeline(drt_ctx *ctx, int32_t cap, int32_t *n, int32_t *kind, double *t0_ms,
                                double *t1_ms);

/* ---------------------------------------------------------------------------------------------
 * Utility: calibrated issue-rate probe of this device's arithmetic pipes, used to quote roofline
 * fractions.  kind 0 = FP64 FMA, 1 = FP32 FMA.  Runs a fixed dependent-chain-free FMA loop over
 * `blocks` x 256 threads and returns the achieved FLOP/s (2 per FMA) in *flops.  Synchronous. */
drt_status drt_probe_peak(drt_ctx *ctx, int32_t kind, int32_t blocks, double *flops);

#ifdef __cplusplus
}
#endif
#endif /* DRT_H */
