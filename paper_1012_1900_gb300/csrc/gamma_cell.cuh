// Per-cell helpers shared by the search kernels and the paper-design
// ablation: criteria resolution, the near-singular Gram pre-filter, the FP64
// redo of a cell, and the evaluation of every face a cell owns.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "gamma_face.cuh"
#include "gamma_internal.h"

namespace gk {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float resolve_dnorm(const Problem& P)
{
    return P.dose_norm > 0.f ? P.dose_norm : fdec(P.ctr->dnorm_enc);
}

// Pre-filter threshold on D for the near-singular Gram test (see face_core).
__device__ __forceinline__ float ill_dmax(const Problem& P)
{
    return P.tau > 0.f ? 0.99f * rsqrtf(P.tau) : kInf;
}

// The cutoff below which a reference voxel is not evaluated: cutoff_frac *
// D_norm.  Global criteria need a positive dose norm (their Delta D is
// dd_frac * D_norm); without one (a reference with no positive dose and no
// norm given) no voxel is evaluated: the threshold is +inf, every voxel gets
// NaN and the run reports GAMMA_ERR_DOSE_NORM, instead of searching with a
// zero Delta D, whose infinite gamma would walk the whole grid per voxel.
__host__ __device__ __forceinline__ float cutoff_threshold(int local, float cutoff_frac, float dnorm)
{
    return (local || dnorm > 0.f) ? cutoff_frac * dnorm : kInf;
}

__device__ __forceinline__ bool is_evaluated(const Problem& P, float dr, float thr)
{
    return dr >= thr && (!P.local || dr > 0.f);
}

// --------------------------------------------------------------------------
// FP64 redo of one cell whose Gram matrices are near singular
// --------------------------------------------------------------------------

template <int N, typename C = int>
__device__ __noinline__ float cell_redo_f64(const float* __restrict__ ev, long long p, long long sy,
                                            long long sz, uint32_t ok, C cx, C cy, C cz,
                                            double drd, double invd, MetricT<double> mtd,
                                            unsigned int* fp64_counter)
{
    double q[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        q[u] = 0.0;
        if (u < (1 << N) && ((ok >> u) & 1u)) {
            const long long o = p + ((u & 1) ? 1 : 0) + ((u & 2) ? sy : 0) + ((u & 4) ? sz : 0);
            q[u] = ((double)ev[o] - drd) * invd;
        }
    }
    CellGeom<double> g;
    cell_geom<N, double>(cx, cy, cz, mtd, g);
    bool ill = false;
    const double b = cell_min_d2<N, double>(q, ok, g, mtd, (double)kInf, (double)kInf, ill);
    atomicAdd(fp64_counter, 1u);
    return (float)b;
}

// A cell whose FP32 pass raised the near-singular pre-filter (rare): the
// exact test on the same relative doses, reloaded here from the evaluation
// grid as the caller formed them ((D_e - D_r) * inv), then the FP64 redo when
// the test holds.  Out of line, so that the callers keep no registers for it.
template <int N>
__device__ __noinline__ float cell_recheck(const Problem& P, uint32_t ok, int cx, int cy, int cz,
                                           long long p, float dr, float inv, float dnorm, float cb)
{
    const long long sy = P.nx, sz = (long long)P.nx * P.ny;
    float q[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        q[u] = 0.f;
        if (u < (1 << N) && ((ok >> u) & 1u)) {
            const long long o = p + ((u & 1) ? 1 : 0) + ((u & 2) ? sy : 0) + ((u & 4) ? sz : 0);
            q[u] = (__ldg(P.ev + o) - dr) * inv;
        }
    }
    if (!cell_gram_ill<N>(q, ok, P.mt.kappa, P.tau)) return cb;
    const double drd = dr;
    const double invd = 1.0 / ((double)P.dd_frac * (P.local ? drd : (double)dnorm));
    return cell_redo_f64<N>(P.ev, p, sy, sz, ok, cx, cy, cz, drd, invd, P.mtd, &P.ctr->fp64_cells);
}

// Every face of the cell with lower corner (x+cx, y+cy, z+cz) as squared
// gamma, with the FP64 redo when a face's Gram matrix is near singular.  q
// holds (D_e - dr) * inv of the cell's vertices.  Out of line: each kernel
// keeps one copy, and the callers keep their own registers few.
template <int N>
__device__ __noinline__ float cell_all_faces(const Problem& P, float q0, float q1, float q2,
                                             float q3, float q4, float q5, float q6, float q7,
                                             uint32_t ok, int cx, int cy, int cz, long long p,
                                             float dr, float dnorm)
{
    const float q[8] = {q0, q1, q2, q3, q4, q5, q6, q7};
    CellGeom<float> g;
    cell_geom<N, float>(cx, cy, cz, P.mt, g);
    bool ill = false;
    float cb = cell_min_d2<N, float>(q, ok, g, P.mt, ill_dmax(P), kInf, ill);
    if (ill) ill = cell_gram_ill<N>(q, ok, P.mt.kappa, P.tau);
    if (ill) {
        const double drd = dr;
        const double invd = 1.0 / ((double)P.dd_frac * (P.local ? drd : (double)dnorm));
        const long long sy = P.nx, sz = (long long)P.nx * P.ny;
        cb = cell_redo_f64<N>(P.ev, p, sy, sz, ok, cx, cy, cz, drd, invd, P.mtd, &P.ctr->fp64_cells);
    }
    return cb;
}

}  // namespace gk
