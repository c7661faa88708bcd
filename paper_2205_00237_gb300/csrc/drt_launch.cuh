// drt_launch.cuh -- small helpers shared by the kernel translation units (drt_kernels.cu, drt_k_*.cu):
// block shape of the per-(path, step) kernels, chunk counts, the FP32-bulk redo list view, the
// launches of the generic-range kernels.
#pragma once
#include <algorithm>

#include "drt_internal.h"
#include "drt_physics.cuh"

namespace drt {

// a block of the per-(path, step) kernels covers EXT_T consecutive time steps of one path
constexpr int EXT_T = 128;

DRT_HD int n_chunks_of(const TimeGridD &tg) { return (tg.n_steps + tg.chunk - 1) / tg.chunk; }

inline bool any_output(const OutD &o) { return o.tau || o.amp || o.doppler || o.angles || o.flags || o.points; }

// the redo scratch: an int counter, then (link, path, step) items from byte 256
inline RedoList redo_list(void *redo, const LinkDev &L, const TimeGridD &tg) {
    RedoList r;
    r.count = reinterpret_cast<int *>(redo);
    r.items = reinterpret_cast<int4 *>(reinterpret_cast<char *>(redo) + 256);
    r.cap = L.n_paths * tg.n_steps;
    return r;
}

// the FP64 H-synthesis path (values, no user outputs), one chain length N per launch
template <int N>
__global__ void __launch_bounds__(EXT_T)
k_extrapolate_fp64_n(const LinkDev L, const TimeGridD tg, const FreqGridD fg, const double *__restrict__ pose,
                     const OutD out, const RecD rec, int p0, int p1, int f32out, const double *__restrict__ warm) {
    const int p = p0 + blockIdx.x;
    const int ti = blockIdx.y * EXT_T + threadIdx.x;
    if (p >= p1 || ti >= tg.n_steps) return;
    path_step_fp64<false, N, false, false>(L, tg, fg, pose, p, ti, out, rec, f32out != 0, warm);
}

// The FP32-bulk step with the block mapping of the FP64 form (time-major block order: an SM's resident
// blocks are nearby paths, so nearby signatures).  The H-synthesis path runs one launch per chain
// length with the register budget of that length (72, 107 and ~150 registers for 1, 2 and 3 vertices
// unbounded): 1-vertex chains (most of the scattering tiles) get 12 warps per SM more than a bound set
// for the longest chain would give them.
// MULTI: the multi-diffraction chains of that length (Newton in FP32 delta numbers from the FP64
// warm starts), 3 blocks per SM.
template <int N, bool MULTI = false> struct BulkBlocks { static constexpr int v = MULTI ? 3 : N <= 1 ? 6 : 4; };

template <int N, bool MULTI = false>
__global__ void __launch_bounds__(EXT_T, BulkBlocks<N, MULTI>::v)
k_extrapolate_bulk_n(const LinkDev L, const TimeGridD tg, const FreqGridD fg, const PoseB *__restrict__ poseb,
                     const BaseRec *__restrict__ base, const double *__restrict__ warm, const OutD out, const RecD rec,
                     const RedoList redo, int p0, int p1) {
    const int p = p0 + blockIdx.y;
    const int ti = blockIdx.x * EXT_T + threadIdx.x;
    if (p >= p1 || ti >= tg.n_steps) return;
    const BulkRows R = bulk_rows_global(L, poseb, base, nullptr, (tg.n_steps + tg.chunk - 1) / tg.chunk, p);
    path_step_bulk<N, MULTI, false, de>(L, tg, fg, R, warm, p, ti, out, rec, redo);
}

// The generic range [len_start[MAXI], n_paths) in launch classes: the multi-diffraction chains of 2
// and 3 vertices (FP32-bulk H path: kernels of their own, compiled for their length: kind 2, 3) and
// the 4-vertex chains (kind -1: the kernel that selects its instance per path), clipped to [p0, p1).
// With split = false the whole clipped range is one kind -1 launch.
template <class F>
cudaError_t for_generic_ranges(const LinkDev &L, int p0, int p1, bool split, F &&launch) {
    const int g0 = std::max(p0, L.len_start[MAXI]);
    if (p1 <= g0) return cudaSuccess;
    if (!split) return launch(-1, g0, p1);
    const int r[4][3] = {{-1, L.len_start[MAXI], L.n_bulk},
                         {2, L.multi_start[0], L.multi_start[1]},
                         {3, L.multi_start[1], L.multi_start[2]},
                         {-1, L.multi_start[2], L.multi_start[3]}};
    for (const auto &q : r) {
        const int a = std::max(g0, q[1]), b = std::min(p1, q[2]);
        if (b > a)
            if (cudaError_t e = launch(q[0], a, b)) return e;
    }
    return cudaSuccess;
}

// launches of the generic-range kernels (their own translation units)
// the FP64 form over the generic range clipped to [p0, p1)
cudaError_t launch_extrapolate_fp64_generic(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg,
                                            const double *pose, const OutD &out, const RecD &rec, int p0, int p1,
                                            int f32, const double *warm, cudaStream_t s);
// the FP32-bulk form over the generic range
cudaError_t launch_extrapolate_bulk_generic(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, const PoseB *pb,
                                            const BaseRec *bs, const double *warm, const OutD &out, const RecD &rec,
                                            const RedoList &rl, cudaStream_t s);

}  // namespace drt
