// drt_launch.cuh -- small helpers shared by the kernel translation units (drt_kernels.cu,
// drt_k_fp64.cu, drt_k_bulk.cu): block shape of the per-(path, step) kernels, chunk counts, the
// FP32-bulk redo list view.
#pragma once
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

}  // namespace drt
