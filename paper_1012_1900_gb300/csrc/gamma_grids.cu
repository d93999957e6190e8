// Reference and evaluation doses on different grids (each grid with its own
// shape, spacing and origin; same axes).  Eq. 1 as for coincident grids: the
// evaluation surface is the Freudenthal interpolant of the evaluation grid,
// and each reference voxel searches it from its own position, which is in
// general not an evaluation node.
//
//   k_grid_prepare  max of the reference dose (the global dose norm) and a
//                   finite check of both grids
//   k_grid_walk     a group of lanes per reference voxel (eight by default)
//                   walks the cell table in key order, a cell per lane and
//                   round, from the evaluation cell
//                   that holds the voxel (clamped to the grid), with the exact
//                   stop of A1 step 4b-ii; a cell is skipped when the distance
//                   from the reference point to its box, with its dose gap,
//                   already reaches the running gamma, else every face of it
//                   is evaluated (real-valued cell offsets; FP64 redo when a
//                   Gram matrix is near singular)
//
// The table is keyed by the distance between the box of the voxel's cell and
// the box of the other cell, divided by the DTA: a lower bound on the distance
// from any point of the first box to any face of the second.  It stays a
// lower bound for a voxel outside the evaluation grid, whose clamped cell is
// the grid cell nearest to it: per axis, its distance to any cell is at least
// that cell's gap to the clamped one.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/gamma.h"
#include "gamma_cell.cuh"
#include "gamma_internal.h"

namespace gk {

// --------------------------------------------------------------------------
// Prepare: dose norm over the reference grid, finite checks
// --------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_grid_prepare(const __grid_constant__ GridProblem G)
{
    float m = -kInf;
    bool bad = false;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long first = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long i = first; i < G.nref; i += stride) {
        const float r = __ldg(G.ref + i);
        bad |= !isfinite(r);
        m = fmaxf(m, r);
    }
    for (long long i = first; i < G.neval; i += stride) bad |= !isfinite(__ldg(G.ev + i));
    __shared__ float sh_m[8];                  // one atomic per block
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
    if ((threadIdx.x & 31) == 0) sh_m[threadIdx.x >> 5] = m;
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, sh_m[w]);
        atomicMax(&G.ctr->dnorm_enc, fenc(m));
        if (bad) atomicOr(&G.ctr->flags, kFlagNonFinite);
    }
}

// --------------------------------------------------------------------------
// The walk
// --------------------------------------------------------------------------

// Every face of evaluation cell p (its lower corner, grid coordinates) for a
// reference point at u (evaluation voxel units, real), unless the cell's
// key and dose range already keep it at least sqrt(best) away.
template <int N>
__device__ __forceinline__ float grid_cell(const GridProblem& G, const int (&p)[3],
                                           const double (&u)[3], const float (&cf)[3], float key,
                                           float dr, float inv, float dnorm, float best)
{
    const long long sy = G.en[0], sz = (long long)G.en[0] * G.en[1];
    const long long pidx = (long long)p[2] * sz + (long long)p[1] * sy + p[0];
    const bool ex = p[0] + 1 < G.en[0], ey = p[1] + 1 < G.en[1], ez = N == 3 && p[2] + 1 < G.en[2];
    float q[8];
    uint32_t ok = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        q[w] = 0.f;
        if (w < (1 << N)) {
            const bool present = (!(w & 1) || ex) && (!(w & 2) || ey) && (!(w & 4) || ez);
            if (present) {
                const long long o = pidx + ((w & 1) ? 1 : 0) + ((w & 2) ? sy : 0) + ((w & 4) ? sz : 0);
                q[w] = (__ldg(G.ev + o) - dr) * inv;
                ok |= 1u << w;
            }
        }
    }
    float qmin = kInf, qmax = -kInf;
#pragma unroll
    for (int w = 0; w < 8; ++w)
        if ((ok >> w) & 1u) {
            qmin = fminf(qmin, q[w]);
            qmax = fmaxf(qmax, q[w]);
        }
    const float gap = qmin > 0.f ? qmin : (qmax < 0.f ? -qmax : 0.f);
    if (fmaf(gap, gap, key * key) >= best) return best;
    // the cell's corner relative to the point (voxel units), cf = d - fraction
    CellGeom<float> g;
    cell_geom<N, float>(cf[0], cf[1], N == 3 ? cf[2] : 0.f, G.mt, g);
    bool ill = false;
    const float dmax = G.tau > 0.f ? 0.99f * rsqrtf(G.tau) : kInf;
    float cb = cell_min_d2<N, float>(q, ok, g, G.mt, dmax, kInf, ill);
    if (ill) ill = cell_gram_ill<N>(q, ok, G.mt.kappa, G.tau);
    if (ill) {
        const double drd = dr;
        const double invd = 1.0 / ((double)G.dd_frac * (G.local ? drd : (double)dnorm));
        cb = cell_redo_f64<N, double>(G.ev, pidx, sy, sz, ok, (double)p[0] - u[0],
                                      (double)p[1] - u[1], N == 3 ? (double)p[2] - u[2] : 0.0,
                                      drd, invd, G.mtd, &G.ctr->fp64_cells);
    }
    return fminf(best, cb);
}

// GL lanes per reference voxel (GL-aligned groups of a warp; 2 .. 32).  The
// table starts with the voxel's own cell (offset 0), so the first round of G
// cells gives a finite bound; later cells are skipped when the distance from
// the point itself to the cell's box, with the dose gap, already reaches the
// running gamma.  The exact stop (A1 step 4b-ii) takes the table's key.
template <int N, int GL>
__global__ void __launch_bounds__(256, 2) k_grid_walk(const __grid_constant__ GridProblem G)
{
    const int lane = threadIdx.x & 31, gl = lane & (GL - 1), gbase = lane & ~(GL - 1);
    const unsigned gmask = GL == 32 ? kFull : (((1u << GL) - 1u) << gbase);
    const float dnorm = G.dose_norm > 0.f ? G.dose_norm : fdec(G.ctr->dnorm_enc);
    const float thr = G.cutoff_frac * dnorm;
    const float rc2 = G.r_cover * G.r_cover;
    unsigned my_eval = 0, my_pass = 0, my_over = 0;
    const long long ngroups = ((long long)gridDim.x * blockDim.x) / GL;
    for (long long v = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / GL; v < G.nref;
         v += ngroups) {                                     // group-uniform
        const float dr = __ldg(G.ref + v);
        if (!(dr >= thr && (!G.local || dr > 0.f))) {
            if (gl == 0) G.out[v] = __int_as_float(0x7fc00000);
            continue;
        }
        const long long ix[3] = {v % G.rn[0], (v / G.rn[0]) % G.rn[1], v / ((long long)G.rn[0] * G.rn[1])};
        // the point in evaluation voxel units: its cell c0 (clamped to the
        // grid) and its position fr in that cell (outside [0, 1) beyond the
        // grid), from FP64 on one lane
        double u[3] = {0.0, 0.0, 0.0};
        int c0[3] = {0, 0, 0};
        float fr[3] = {0.f, 0.f, 0.f}, ehf[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a < N; ++a) {
            double ua = 0.0, f = 0.0;
            if (gl == 0) {
                ua = (G.ro[a] + (double)ix[a] * G.rh[a] - G.eo[a]) / G.eh[a];
                f = fmin(fmax(floor(ua), 0.0), (double)(G.en[a] - 2));
            }
            u[a] = __shfl_sync(gmask, ua, gbase);
            c0[a] = (int)__shfl_sync(gmask, f, gbase);
            fr[a] = (float)(u[a] - (double)c0[a]);
            ehf[a] = (float)G.eh[a];
        }
        const float dD = G.dd_frac * (G.local ? dr : dnorm);
        const float inv = 1.0f / dD;
        float best = kInf;
        int t = 0;
        while (t < G.ntable) {
            const int idx = t + gl;
            float key = kInf;
            uint32_t off = 0;
            if (idx < G.ntable) {
                const TableEntry e = G.table[idx];
                key = e.key;
                off = e.off;
            }
            const float k0 = __shfl_sync(gmask, key, gbase);
            if (k0 * k0 >= best) break;                       // A1 step 4b-ii, exact
            float cb = best;
            if (key * key < best) {
                const int d[3] = {unpack10(off, 0), unpack10(off, 10), N == 3 ? unpack10(off, 20) : 0};
                const int p[3] = {c0[0] + d[0], c0[1] + d[1], c0[2] + d[2]};
                bool in = true;
                // the distance from the point to the cell's box: a lower bound
                // in FP32 from the integer offset and the point's fraction,
                // each axis lowered by its rounding (4 ulp of its operands) and
                // the sum by 1e-5
                float k2 = 0.f;
#pragma unroll
                for (int a = 0; a < N; ++a) {
                    in = in && p[a] >= 0 && p[a] < G.en[a];
                    const float lo = (float)d[a] - fr[a], hi = fr[a] - (float)(d[a] + 1);
                    const float slack = 4.8e-7f * (fabsf(fr[a]) + fabsf((float)d[a]) + 2.f);
                    const float gap = fmaxf(fmaxf(lo, hi) - slack, 0.f) * ehf[a];
                    k2 = fmaf(gap, gap, k2);
                }
                k2 *= 0.99999f;
                if (in && k2 < best) {
                    const float cf[3] = {(float)d[0] - fr[0], (float)d[1] - fr[1], (float)d[2] - fr[2]};
                    cb = grid_cell<N>(G, p, u, cf, sqrtf(fmaxf(k2, key * key)), dr, inv, dnorm, best);
                }
            }
#pragma unroll
            for (int o = GL / 2; o > 0; o >>= 1) cb = fminf(cb, __shfl_xor_sync(gmask, cb, o));
            best = cb;
            t += GL;
        }
        if (t >= G.ntable && best > rc2) {
            // past a truncated table: every remaining cell of the search box
            if (gl == 0) ++my_over;
            const float gm = sqrtf(best);
            int dlo[3] = {0, 0, 0}, dhi[3] = {0, 0, 0};
#pragma unroll
            for (int a = 0; a < N; ++a) {
                const float l = gm / (float)G.eh[a] + 2.f;
                const int lim = l < (float)G.en[a] ? (int)ceilf(l) : G.en[a];
                dlo[a] = max(-lim, -c0[a]);
                dhi[a] = min(lim, G.en[a] - 1 - c0[a]);
            }
            const long long wx = dhi[0] - dlo[0] + 1, wy = dhi[1] - dlo[1] + 1, wz = dhi[2] - dlo[2] + 1;
            const long long tot = wx * wy * wz;
            const float cut = rc2 * 0.99999f;
            float lb = best;
            for (long long b = gl; b < tot; b += GL) {
                const int d[3] = {dlo[0] + (int)(b % wx), dlo[1] + (int)((b / wx) % wy), dlo[2] + (int)(b / (wx * wy))};
                const int p[3] = {c0[0] + d[0], c0[1] + d[1], c0[2] + d[2]};
                bool in = true;
                float k2 = 0.f;
#pragma unroll
                for (int a = 0; a < N; ++a) {
                    in = in && p[a] >= 0 && p[a] < G.en[a];
                    const float gap = (float)max(abs(d[a]) - 1, 0) * (float)G.eh[a];
                    k2 = fmaf(gap, gap, k2);
                }
                if (!in || k2 < cut || k2 >= lb) continue;
                const float cf[3] = {(float)d[0] - fr[0], (float)d[1] - fr[1], (float)d[2] - fr[2]};
                lb = grid_cell<N>(G, p, u, cf, sqrtf(k2), dr, inv, dnorm, lb);
            }
#pragma unroll
            for (int o = GL / 2; o > 0; o >>= 1) lb = fminf(lb, __shfl_xor_sync(gmask, lb, o));
            best = lb;
        }
        if (gl == 0) {
            const float gam = sqrtf(best);
            G.out[v] = gam;
            ++my_eval;
            my_pass += gam <= 1.f;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_eval += __shfl_xor_sync(kFull, my_eval, o);
        my_pass += __shfl_xor_sync(kFull, my_pass, o);
        my_over += __shfl_xor_sync(kFull, my_over, o);
    }
    if (lane == 0) {
        if (my_eval) atomicAdd(&G.ctr->n_eval, (unsigned long long)my_eval);
        if (my_pass) atomicAdd(&G.ctr->n_pass, (unsigned long long)my_pass);
        if (my_over) atomicAdd(&G.ctr->overflow_count, my_over);
    }
}

// --------------------------------------------------------------------------
// Host side
// --------------------------------------------------------------------------

int build_grid_table(int nd, const double hn[3], const int en[3], long long cap,
                     std::vector<TableEntry>& table, double& r_cover)
{
    // radius from a ball-volume estimate of about 2 * cap cells
    const double cellvol = hn[0] * hn[1] * (nd == 3 ? hn[2] : 1.0);
    double R = nd == 3 ? std::cbrt(2.0 * (double)cap * cellvol * 3.0 / (4.0 * M_PI))
                       : std::sqrt(2.0 * (double)cap * cellvol / M_PI);
    bool whole = false, packing = false;
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    double diag = 0;
    for (int a = 0; a < nd; ++a) diag += (double)en[a] * en[a] * hn[a] * hn[a];
    diag = std::sqrt(diag) + 1.0;
    if (R > diag) { R = diag; whole = true; }
    for (int a = 0; a < nd; ++a) {
        long long l = (long long)std::ceil(R / hn[a]) + 2;
        l = std::min<long long>(l, en[a]);
        if (l > 511) { l = 511; packing = true; }
        lo[a] = -(int)l;
        hi[a] = (int)l;
    }
    struct Tmp { double key; int x, y, z; };
    std::vector<Tmp> all;
    try {
        for (int z = lo[2]; z <= hi[2]; ++z)
            for (int y = lo[1]; y <= hi[1]; ++y)
                for (int x = lo[0]; x <= hi[0]; ++x) {
                    const int c[3] = {x, y, z};
                    double k2 = 0;
                    for (int a = 0; a < nd; ++a) {
                        const double gap = std::max(std::abs(c[a]) - 1, 0) * hn[a];
                        k2 += gap * gap;
                    }
                    const double key = std::sqrt(k2);
                    if (key < R) all.push_back({key, x, y, z});
                }
    } catch (const std::bad_alloc&) {
        return GAMMA_ERR_OOM;
    }
    std::sort(all.begin(), all.end(), [](const Tmp& a, const Tmp& b) {
        if (a.key != b.key) return a.key < b.key;
        // the voxel's own cell first among the key-0 cells (a finite bound
        // from the walk's first round), then z, y, x
        const bool a0 = (a.x | a.y | a.z) == 0, b0 = (b.x | b.y | b.z) == 0;
        if (a0 != b0) return a0;
        if (a.z != b.z) return a.z < b.z;
        if (a.y != b.y) return a.y < b.y;
        return a.x < b.x;
    });
    double cover = whole ? INFINITY : R;
    if (packing) {
        double m = INFINITY;
        for (int a = 0; a < nd; ++a) m = std::min(m, 509.0 * hn[a]);
        cover = std::min(cover, m);
    }
    size_t keep = all.size();
    if ((long long)keep > cap) {
        keep = (size_t)cap;
        cover = std::min(cover, all[keep].key);
    }
    table.resize(keep);
    for (size_t i = 0; i < keep; ++i) {
        table[i].off = pack10(all[i].x, all[i].y, all[i].z);
        float f = (float)all[i].key;
        if ((double)f > all[i].key) f = std::nextafterf(f, -INFINITY);
        table[i].key = f;
    }
    r_cover = cover;
    return GAMMA_OK;
}

template <int N>
static void launch_grid_walk_n(const GridProblem& G, int gl, int grid, cudaStream_t s)
{
    switch (gl) {
    case 2: k_grid_walk<N, 2><<<grid, 256, 0, s>>>(G); break;
    case 4: k_grid_walk<N, 4><<<grid, 256, 0, s>>>(G); break;
    case 16: k_grid_walk<N, 16><<<grid, 256, 0, s>>>(G); break;
    case 32: k_grid_walk<N, 32><<<grid, 256, 0, s>>>(G); break;
    default: k_grid_walk<N, 8><<<grid, 256, 0, s>>>(G); break;
    }
}

cudaError_t launch_grids(const GridProblem& G, cudaStream_t s)
{
    const int sms = device_sm_count();
    const long long nmax = std::max(G.nref, G.neval);
    const int gp = (int)std::max<long long>(1, std::min<long long>((nmax + 255) / 256, (long long)sms * 8));
    k_grid_prepare<<<gp, 256, 0, s>>>(G);
    const int gl = G.lanes;
    const int gw = (int)std::max<long long>(1, std::min<long long>((G.nref * gl + 255) / 256,
                                                                   (long long)sms * 16));
    if (G.ndim == 3) launch_grid_walk_n<3>(G, gl, gw, s);
    else launch_grid_walk_n<2>(G, gl, gw, s);
    return cudaGetLastError();
}

}  // namespace gk
