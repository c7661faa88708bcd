// drt_batch.cuh -- data layout of a batch plan shared by its host code (drt_batch.cu) and its
// extrapolation kernels (drt_k_batch.cu).
#pragma once
#include "drt_internal.h"
#include "drt_physics.cuh"

namespace drt {

// stage slots; the synthesis has one slot per tile variant (its units depend on the tile width)
// (ST_BULK + n: chains of n vertices; ST_BULKD + k: multi-diffraction chains of k + 2 vertices; ST_BULKM:
// the generic code)
enum { ST_POSEB = 0, ST_POSE64 = 1, ST_WARM = 2, ST_BASE = 3, ST_BULK = 4, ST_SYNTH = 8, ST_BULKM = 11, ST_BULKD = 12,
       N_STAGES = 14 };
constexpr int BULK_W = 32;                // time steps per extrapolation unit (one warp's lanes)
constexpr int SYNTH_U = 32;               // (step, tile) pairs per synthesis unit (one block) ...
constexpr int SYNTH_PG = 4;               // ... whose warps split the paths
constexpr int SYNTH_KT[3] = {8, 16, 32};
constexpr size_t REC_BYTES = sizeof(float4) + sizeof(float);   // one synthesis record
constexpr size_t REC_CAP = (size_t)4 << 30;                    // record buffer of one wave (bytes)
constexpr size_t SCRATCH_CAP = (size_t)8 << 30;                // poses, warm starts, anchors of one wave

struct alignas(16) BatchLink {
    LinkDev L;
    TimeGridD tg;
    FreqGridD fg;
    PoseB *poseb;      // [bodies + 2][chunks]
    double *pose64;    // [bodies][chunks]
    double *warm;      // [chunks + 1][n_paths - n_bulk][2 * MAXI]
    BaseRec *base;     // [chunks][paths]
    float2 *H;         // caller's [T][F]
    OutD out;          // caller's optional per-path-step records (FP32 formats), [T][P]
    size_t rec0;       // first record of this link in its wave's record buffer ([T][P])
    long long it0[N_STAGES];   // first item per stage slot (4 on: counted within the link's wave)
    // carrier pairs: two entries of one link over one time grid (different carriers) share the
    // geometry; the first (partner >= 0: the second's index) evaluates it and both carriers' coefficients
    // and records, the second (shared = 1) has no extrapolation units of its own
    int32_t partner, shared;
    int32_t gen_p0;    // first path of the generic-code unit range (len_start[MAXI]; 0 when the batch
                       // writes per-path-step records, which only the generic code does)
    int32_t skip_p0, skip_p1;   // paths of that range with units of their own (the multi-diffraction
                                // chains of 2 and 3 vertices; empty when the batch writes records)
    int32_t pair_p0;   // a pair's first entry also evaluates its partner's paths [pair_p0, n_paths)
};

// one launch: the links [l0, l1) of its stage or wave, its item count and claim counter
struct BatchDev {
    int l0, l1;
    const BatchLink *links;
    long long n_items;
    long long it_base;   // stages 0-3: item of the wave's first link
    unsigned long long *counter;
    float4 *rec_a;
    float *rec_b;
    RedoList redo;   // items (link, path, step)
};

__device__ __forceinline__ int find_link(const BatchDev &B, int stage, long long it) {
    int lo = B.l0, hi = B.l1 - 1;
    while (lo < hi) {   // last link whose first item is <= it
        int mid = (lo + hi + 1) >> 1;
        if (B.links[mid].it0[stage] <= it) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int chunks_of(const TimeGridD &tg) { return (tg.n_steps + tg.chunk - 1) / tg.chunk; }

// the per-chain-length extrapolation launch of one wave (drt_k_batch.cu): N = 0..3 with pair = the
// batch has carrier pairs, N < 0 the generic code (dual: Doppler rates; records allowed)
cudaError_t launch_batch_bulk(int N, bool dual, bool pair, const BatchDev &B, int grid, cudaStream_t s);
// the multi-diffraction chains of N = 2 or 3 vertices (values only)
cudaError_t launch_batch_bulk_multi(int N, bool pair, const BatchDev &B, int grid, cudaStream_t s);
int batch_bulk_blocks(int N, bool multi = false);

// the stage kernels in their own translation units
cudaError_t launch_batch_stage(int stage, const BatchDev &B, int grid, cudaStream_t s);   // stages 0-3
cudaError_t launch_batch_redo(bool dual, const BatchDev &B, int grid, cudaStream_t s);

}  // namespace drt
