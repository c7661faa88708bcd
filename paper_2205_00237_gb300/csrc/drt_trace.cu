// drt_trace.cu -- conventional ray tracing at one instant on the GPU (Sec. II: the ray-tracing run DRT
// starts from at t0 and repeats at every multipath-lifetime boundary, Sec. IV-B), by brute-force
// image-tree enumeration: every chain of at most two reflections / diffractions (no primitive twice
// in a row) and every single-tile scattering chain is a candidate; one thread solves a candidate with
// the extrapolation's FP64 geometry at the instant (image method, Keller cone, Newton from the edge
// midpoints for two diffractions in a segment), keeps it when its FP64 validity flags are 0 and no
// face blocks any of its segments, and appends it to the output list.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "drt_launch.cuh"

namespace drt {

// a face posed at the instant: centre, unit normal, in-plane axes, half extents
struct PosedFace { double c[3], n[3], u[3], w[3], hu, hw; };

DRT_HD void pose_face(const LinkDev &L, double t, int f, PosedFace *out_f) {
    const FaceD &F = L.faces[f];
    double P[POSE_W];
    body_pose_row(L.bodies[F.body], t, P);
    const Pose<double> q = load_pose<double>(P);
    const v3<double> c = q.O + rot(q, F.c), n = rot(q, F.n), u = rot(q, F.u), w = cross(u, n);
    PosedFace r;
    r.c[0] = c.x; r.c[1] = c.y; r.c[2] = c.z;
    r.n[0] = n.x; r.n[1] = n.y; r.n[2] = n.z;
    r.u[0] = u.x; r.u[1] = u.y; r.u[2] = u.z;
    r.w[0] = w.x; r.w[1] = w.y; r.w[2] = w.z;
    r.hu = F.hu;
    r.hw = F.hw;
    *out_f = r;
}

__global__ void k_pose_faces(const LinkDev L, double t, PosedFace *__restrict__ out) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < L.n_faces) pose_face(L, t, f, out + f);
}

// Does the face block the segment A -> B?  It does when the segment crosses the face's plane
// strictly between its ends at a point inside the rectangle; a face whose plane holds A or B (within
// 1e-9 m: the face a reflection point or a tile lies on, the faces of a diffracting edge, faces coplanar
// with those) does not.
DRT_HD bool face_blocks(const PosedFace &F, v3<double> A, v3<double> B) {
    const v3<double> c = V3(F.c[0], F.c[1], F.c[2]), n = V3(F.n[0], F.n[1], F.n[2]);
    const double ha = dot(A - c, n), hb = dot(B - c, n);
    if (fabs(ha) < 1e-9 || fabs(hb) < 1e-9) return false;
    if ((ha > 0.0) == (hb > 0.0)) return false;
    const v3<double> r = A + (B - A) * (ha / (ha - hb)) - c;
    return fabs(dot(r, V3(F.u[0], F.u[1], F.u[2]))) <= F.hu && fabs(dot(r, V3(F.w[0], F.w[1], F.w[2]))) <= F.hw;
}

// one ray found: its enumeration index, chain and diffraction parameters at the instant
struct TracedRay { long long index; int32_t n; uint32_t types; int32_t prims[MAXI]; double s[MAXI]; };

constexpr int TRACE_T = 128;

// candidate k of the enumeration (0 = line of sight; single faces (R), edges (D), tiles (S); ordered
// pairs of faces / edges, the same primitive twice excluded) solved at t: true when it is a ray, which
// then fills *r
// the candidate's chain of N interactions (codes c[0..N-1]): solved, checked and, if it is a ray, stored
template <int N>
DRT_HD bool trace_chain(const LinkDev &L, double t, long long k, const int *code, const PosedFace *faces,
                        TracedRay *r) {
    const int NP = L.n_faces + L.n_edges;
    Prim<double> pr[N > 0 ? N : 1];
    double s0[MAXI] = {0.0, 0.0, 0.0, 0.0};
    uint32_t types = 0;
    int prims[MAXI] = {0, 0, 0, 0};
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const int c = code[j];
        int ty, idx;
        if (c < L.n_faces) { ty = T_R; idx = c; }
        else if (c < NP) { ty = T_D; idx = c - L.n_faces; s0[j] = 0.5 * L.edges[idx].len; }
        else { ty = T_S; idx = c - NP; }
        pr[j] = val_prim(load_prim_direct<double>(L, t, ty, idx));
        types |= (uint32_t)ty << (8 * j);
        prims[j] = idx;
    }
    v3<double> V[N + 2];
    V[0] = val(terminal<double>(L.tx, t));
    V[N + 1] = val(terminal<double>(L.rx, t));
    uint32_t fl = 0;
    solve_geometry_any<N>(pr, V, s0, fl);
    fl |= validity<N>(pr, N, V);
#pragma unroll
    for (int i = 1; i <= N; ++i)
        if (!(isfinite(V[i].x) && isfinite(V[i].y) && isfinite(V[i].z))) fl |= F_DEGEN;
    if (fl) return false;
#pragma unroll
    for (int i = 1; i <= N + 1; ++i)
        for (int f = 0; f < L.n_faces; ++f)
            if (face_blocks(faces[f], V[i - 1], V[i])) return false;
    r->index = k;
    r->n = N;
    r->types = types;
#pragma unroll
    for (int j = 0; j < MAXI; ++j) {
        r->prims[j] = prims[j];
        r->s[j] = 0.0;
        if (j < N)
            if (pr[j].type == T_D) r->s[j] = dot(V[j + 1] - pr[j].p, pr[j].a);
    }
    return true;
}

DRT_HD bool trace_eval(const LinkDev &L, double t, long long k, int with_tiles, const PosedFace *faces, TracedRay *r) {
    const int NP = L.n_faces + L.n_edges, NT = with_tiles ? L.n_tiles : 0;
    int n = 0, code[2] = {0, 0};
    if (k > 0) {
        const long long j = k - 1;
        if (j < NP + NT) {
            code[0] = (int)j;
            n = 1;
        } else {
            const long long q = j - NP - NT;
            code[0] = (int)(q / NP);
            code[1] = (int)(q % NP);
            if (code[0] == code[1]) return false;
            n = 2;
        }
    }
    if (n == 0) return trace_chain<0>(L, t, k, code, faces, r);
    if (n == 1) return trace_chain<1>(L, t, k, code, faces, r);
    return trace_chain<2>(L, t, k, code, faces, r);
}

__global__ void __launch_bounds__(TRACE_T)
k_trace(const LinkDev L, double t, long long n_cand, int with_tiles, const PosedFace *__restrict__ faces,
        TracedRay *__restrict__ out, int cap, int *__restrict__ count) {
    const long long k = blockIdx.x * (long long)TRACE_T + threadIdx.x;
    if (k >= n_cand) return;
    TracedRay r;
    if (!trace_eval(L, t, k, with_tiles, faces, &r)) return;
    const int slot = atomicAdd(count, 1);
    if (slot < cap) out[slot] = r;
}

long long trace_candidates(const LinkDev &L, int max_order, int with_tiles) {
    const long long NP = L.n_faces + L.n_edges, NT = with_tiles ? L.n_tiles : 0;
    return 1 + (max_order >= 1 ? NP + NT : 0) + (max_order >= 2 ? NP * NP : 0);
}

size_t trace_ray_bytes() { return sizeof(TracedRay); }
size_t trace_face_bytes() { return sizeof(PosedFace); }

cudaError_t launch_trace(const LinkDev &L, double t, int max_order, int with_tiles, void *faces, void *rays, int cap,
                         int *count, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (L.n_faces > 0) k_pose_faces<<<(L.n_faces + 127) / 128, 128, 0, s>>>(L, t, reinterpret_cast<PosedFace *>(faces));
    const long long n = trace_candidates(L, max_order, with_tiles);
    k_trace<<<(unsigned)((n + TRACE_T - 1) / TRACE_T), TRACE_T, 0, s>>>(
        L, t, n, with_tiles, reinterpret_cast<const PosedFace *>(faces), reinterpret_cast<TracedRay *>(rays), cap, count);
    return cudaGetLastError();
}

// the found rays (count of them, in any order) to host arrays in enumeration order
void trace_unpack(const void *rays_host, int count, uint8_t *n_int, uint8_t *types, int32_t *prims, double *s0,
                  int cap) {
    const TracedRay *R = reinterpret_cast<const TracedRay *>(rays_host);
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return R[a].index < R[b].index; });
    for (int q = 0; q < count && q < cap; ++q) {
        const TracedRay &r = R[order[q]];
        n_int[q] = (uint8_t)r.n;
        for (int j = 0; j < MAXI; ++j) {
            types[q * MAXI + j] = (uint8_t)((r.types >> (8 * j)) & 0xff);
            prims[q * MAXI + j] = j < r.n ? r.prims[j] : -1;
            s0[q * MAXI + j] = r.s[j];
        }
    }
}

}  // namespace drt
