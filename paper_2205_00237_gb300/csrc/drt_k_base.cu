// drt_k_base.cu -- the FP32-bulk form's FP64 anchors: body poses at the chunk bases and, per (path,
// chunk), the FP64 path length, segment vectors and phase seeds the FP32 deltas build on.
#include "drt_launch.cuh"

namespace drt {

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

}  // namespace drt
