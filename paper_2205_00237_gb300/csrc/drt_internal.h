// drt_internal.h -- device-side data layout of a loaded link and the launch interface between the
// C-ABI host code (drt_api.cu) and the kernels (drt_kernels.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/drt.h"

namespace drt {

constexpr int MAXI = 4;
constexpr int POSE_W = 18;   // doubles per (time, body) pose record: R (3x3 row-major), O, v_O, omega

// primitives, positions relative to the owning body's rotation centre o (world axes at t0), so a
// posed position is O(t) + R(t) rel
struct FaceD { double c[3], n[3], u[3], hu, hw; int32_t body, mat; };                       // 96 B
struct EdgeD { double a[3], e[3], t0[3], n0[3], len, wn; int32_t body, mat, pad0, pad1; };  // 128 B
struct TileD { double c[3], n[3], area, s, alpha, phase; int32_t body, mat; };               // 88 B
struct MatD { double eps_r, sigma, rough, pec; float eps_rf, sigmaf, roughf, pecf; };       // 48 B
// FP32 copies for the FP32-bulk form (same meaning, no FP64 conversions in its kernels)
struct FaceF { float c[3], n[3], u[3], hu, hw; int32_t body, mat, pad0, pad1, pad2; };          // 64 B
struct EdgeF { float a[3], e[3], t0[3], n0[3], len, wn; int32_t body, mat; };                 // 64 B
struct TileF { float c[3], n[3], area, s, alpha, phase; int32_t body, mat; };                 // 48 B
struct TermD { double r[3], v[3], a[3]; };
struct BodyD { double o[3], v[3], a[3], k[3], w0, wdot; };

// one loaded link, passed to kernels by value
struct LinkDev {
    int32_t n_paths, n_bodies, n_faces, n_edges, n_tiles, n_mats;
    int32_t n_bulk;   // paths [0, n_bulk) have at most one diffraction per segment (FP32-bulk capable)
    TermD tx, rx;
    const BodyD *bodies;
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
};

struct TimeGridD { double t_start, dt; int32_t n_steps; };
struct FreqGridD { double fc, bandwidth; int32_t n_bins; };

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

// validated host image of one link, ready for upload (drt_api.cu)
struct PackedLink {
    LinkDev dev{};
    std::vector<BodyD> bodies;
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
cudaError_t launch_extrapolate_fp64(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg,
                                    const double *pose, const OutD &out, const RecD &rec,
                                    cudaStream_t s, int p0 = 0, int p1 = -1, bool f32out = false,
                                    double *warm = nullptr);
size_t warm_bytes(const LinkDev &L, const TimeGridD &tg);
// FP32-bulk form (CHUNK consecutive steps share FP64 anchors); see drt_physics.cuh.  Scratch:
// per-(body or terminal, chunk) FP32 base poses and per-(path, chunk) FP64 anchors.
size_t bulk_pose_bytes(const LinkDev &L, const TimeGridD &tg);
size_t bulk_base_bytes(const LinkDev &L, const TimeGridD &tg);
cudaError_t launch_pose_bulk(const LinkDev &L, const TimeGridD &tg, void *poseb, cudaStream_t s);
size_t bulk_pose64_bytes(const LinkDev &L, const TimeGridD &tg);
size_t bulk_redo_bytes(const LinkDev &L, const TimeGridD &tg);
cudaError_t launch_base_fp64(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, double *pose64, void *base,
                             cudaStream_t s);
// the redo scratch holds an int counter (zeroed here, on the stream) followed by the (path, step) list
cudaError_t launch_extrapolate_bulk(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, const void *poseb,
                                    const void *base, const OutD &out, const RecD &rec, void *redo, cudaStream_t s);
cudaError_t launch_redo(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, const OutD &out, const RecD &rec,
                        void *redo, cudaStream_t s);
cudaError_t launch_synth(const RecD &rec, int32_t n_paths, const TimeGridD &tg, const FreqGridD &fg,
                         float2 *H, cudaStream_t s);
cudaError_t launch_probe(int kind, int blocks, double *sink, cudaStream_t s, float *ms);

}  // namespace drt
