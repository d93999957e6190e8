// gamma_run_noalloc: one gamma map with no memory allocation at all.
//
// Some callers cannot allocate device memory on their own.  A host
// application that owns the whole device through its own pool allocator (a
// treatment-planning or QA system, a deep-learning framework operator) must
// not have a library call cudaMalloc/cudaFree behind its back: that bypasses
// its budget, fragments its pool and may implicitly synchronise the device,
// stalling every other stream.  This entry point serves them: the caller
// passes the dose grids and the output, and every scratch buffer of the run
// (counters, the cell table and the queue of voxels that search past the
// key-0 cells) lives in one file-scope device array of fixed size below.
//
// Costs and limits:
//  - every GPU that loads this library holds the array (about 20.3 MB) until
//    the process exits;
//  - grids are limited to GAMMA_NOALLOC_MAX_VOXELS voxels and the cell table
//    to GAMMA_NOALLOC_MAX_TABLE entries (voxels searching past it fall back to
//    the exact box scan);
//  - every call shares the array and leaves the last call's contents in it,
//    so calls whose GPU work overlaps (different streams, or several host
//    threads) race on it and give wrong results; serialise them.
//  - the first call on each device looks up the array's device address
//    (cudaGetSymbolAddress) with that device current; make that first call
//    before any stream capture starts.
// The table is built on the host in static storage (no heap), guarded by a
// mutex.  It reaches the device array as the by-value parameters of small
// copy kernels (at most kChunk entries per launch): a launch takes its own
// copy of its parameters when it is issued, so no device work reads the host
// table after the call has returned, and a later call that rebuilds it for
// another geometry cannot change what an earlier call's work writes.  The
// launch shapes are the defaults a new handle starts with.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "../../include/gamma.h"
#include "gamma_internal.h"

namespace {

constexpr long long kMaxVoxels = GAMMA_NOALLOC_MAX_VOXELS;
constexpr int kMaxTable = GAMMA_NOALLOC_MAX_TABLE;
constexpr int kMaxEnum = 2 * kMaxTable;
constexpr int kMaxDevices = 64;

// Layout of the scratch array (byte offsets, each 256-aligned).
constexpr size_t kOffCounters = 0;
constexpr size_t kOffTable = 4096;
constexpr size_t kOffTail = kOffTable + sizeof(gk::TableEntry) * kMaxTable;
constexpr size_t kOffBucket = kOffTail + sizeof(unsigned) * kMaxVoxels;
constexpr size_t kScratchBytes = kOffBucket + kMaxVoxels;
static_assert(sizeof(gk::Counters) <= kOffTable, "counters overflow their slot");
static_assert(kOffTail % 256 == 0 && kOffBucket % 256 == 0, "misaligned scratch slots");

}  // namespace

// The scratch memory of every gamma_run_noalloc call on this device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_mutex;                        // guards the host tables and set-up
void* g_scratch_dev[kMaxDevices] = {};     // device address of the array, per device

struct EnumCell { double key; int x, y, z; };
EnumCell g_enum[kMaxEnum];
gk::TableEntry g_table_host[kMaxTable];

float round_down_f(double x)
{
    float f = (float)x;
    if ((double)f > x) f = std::nextafterf(f, -INFINITY);
    return f;
}

double gap1(int i) { return i >= 0 ? (double)i : (double)(-i - 1); }

// The radially sorted cell table (Algorithm A1 steps 2-3) in static storage,
// keyed as the allocating handle's table is (key-0 cells by the distance to
// their faces off the voxel).  Returns the entry count; *cover gets the radius
// below which the table is complete, far2 the squared key-0 distances.
int build_static_table(int nd, const int64_t n[3], const double hn[3], double* cover,
                       float far2[8])
{
    double far[8];
    gk::key0_far(hn, nd, far);
    for (int s = 0; s < 8; ++s) far2[s] = round_down_f(far[s] * far[s]);
    double cellvol = hn[0] * hn[1] * (nd == 3 ? hn[2] : 1.0);
    double R = nd == 3 ? std::cbrt(1.5 * kMaxTable * cellvol * 3.0 / (4.0 * M_PI))
                       : std::sqrt(1.5 * kMaxTable * cellvol / M_PI);
    double diag = 0;
    for (int a = 0; a < nd; ++a) diag += (double)(n[a] * n[a]) * hn[a] * hn[a];
    diag = std::sqrt(diag) + 1.0;
    bool whole_grid = false;
    if (R > diag) { R = diag; whole_grid = true; }
    int cnt = 0;
    for (int attempt = 0; attempt < 64; ++attempt) {
        int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int a = 0; a < nd; ++a) {
            int64_t lim = (int64_t)std::ceil(R / hn[a]) + 1;
            lo[a] = std::max<int64_t>(std::max<int64_t>(-(n[a] - 1), -lim - 1), -511);
            hi[a] = std::min<int64_t>(std::min<int64_t>(n[a] - 1, lim), 511);
        }
        cnt = 0;
        bool full = false;
        for (int64_t z = lo[2]; z <= hi[2] && !full; ++z)
            for (int64_t y = lo[1]; y <= hi[1] && !full; ++y)
                for (int64_t x = lo[0]; x <= hi[0]; ++x) {
                    const double ax = gap1((int)x) * hn[0], ay = gap1((int)y) * hn[1];
                    const double az = nd == 3 ? gap1((int)z) * hn[2] : 0.0;
                    double key = std::sqrt(ax * ax + ay * ay + az * az);
                    if (key == 0.0) key = far[(x & 1) | ((y & 1) << 1) | ((z & 1) << 2)];
                    if (!(key < R)) continue;
                    if (cnt == kMaxEnum) { full = true; break; }
                    g_enum[cnt++] = {key, (int)x, (int)y, (int)z};
                }
        if (!full) break;
        R *= 0.8;
        whole_grid = false;
    }
    std::sort(g_enum, g_enum + cnt, [](const EnumCell& a, const EnumCell& b) {
        if (a.key != b.key) return a.key < b.key;
        if (a.z != b.z) return a.z < b.z;
        if (a.y != b.y) return a.y < b.y;
        return a.x < b.x;
    });
    double cov = whole_grid ? INFINITY : R;
    double pack = INFINITY;
    for (int a = 0; a < nd; ++a) pack = std::min(pack, 510.0 * hn[a]);
    cov = std::min(cov, pack);
    if (cnt > kMaxTable) {
        cov = std::min(cov, g_enum[kMaxTable].key);
        cnt = kMaxTable;
    }
    for (int i = 0; i < cnt; ++i) {
        g_table_host[i].off = gk::pack10(g_enum[i].x, g_enum[i].y, g_enum[i].z);
        g_table_host[i].key = round_down_f(g_enum[i].key);
    }
    *cover = cov;
    return cnt;
}

// Table entries carried to the device by value: kChunk entries keep the
// parameter block under the 32,764-byte kernel parameter limit.
constexpr int kChunk = 4000;
struct TableChunk {
    int first;                 // index of e[0] in the table
    int count;                 // entries used
    gk::TableEntry e[kChunk];
};
static_assert(sizeof(TableChunk) + sizeof(void*) <= 32764,
              "table chunk exceeds the kernel parameter limit");

__global__ void __launch_bounds__(256) k_table_fill(gk::TableEntry* __restrict__ dst,
                                                    const __grid_constant__ TableChunk c)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c.count; i += gridDim.x * blockDim.x)
        dst[c.first + i] = c.e[i];
}

}  // namespace

extern "C" int gamma_run_noalloc(const float* ref_dev, const float* eval_dev, float* gamma_out_dev,
                                 int ndim, const int64_t shape[3], const float spacing_mm[3],
                                 const gamma_criteria* crit, void* cuda_stream, int64_t* n_eval,
                                 int64_t* n_pass)
{
    if (!ref_dev || !eval_dev || !gamma_out_dev || !shape || !spacing_mm || !crit)
        return GAMMA_ERR_INVALID_ARG;
    if (!(crit->dd_frac > 0.f) || !std::isfinite(crit->dd_frac) || !(crit->dta_mm > 0.f) ||
        !std::isfinite(crit->dta_mm) || (crit->mode != GAMMA_GLOBAL && crit->mode != GAMMA_LOCAL) ||
        !std::isfinite(crit->cutoff_frac) || !std::isfinite(crit->dose_norm))
        return GAMMA_ERR_INVALID_ARG;
    if (ndim != 2 && ndim != 3) return GAMMA_ERR_SHAPE;
    const int64_t nz = ndim == 3 ? shape[0] : 1, ny = shape[1], nx = shape[2];
    if (ndim == 2 && shape[0] != 1) return GAMMA_ERR_SHAPE;
    if (nx < 2 || ny < 2 || (ndim == 3 && nz < 2)) return GAMMA_ERR_SHAPE;
    if (nx > kMaxVoxels || ny > kMaxVoxels || nz > kMaxVoxels) return GAMMA_ERR_TOO_LARGE;
    const int64_t nvox = nx * ny * nz;
    if (nvox > kMaxVoxels) return GAMMA_ERR_TOO_LARGE;
    for (int a = (ndim == 3 ? 0 : 1); a < 3; ++a)
        if (!(spacing_mm[a] > 0.f) || !std::isfinite(spacing_mm[a])) return GAMMA_ERR_INVALID_ARG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GAMMA_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;

    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GAMMA_ERR_CUDA;
        g_scratch_dev[dev] = p;
    }
    unsigned char* base = (unsigned char*)g_scratch_dev[dev];

    const double dta = crit->dta_mm;
    const double h[3] = {spacing_mm[2], spacing_mm[1], ndim == 3 ? spacing_mm[0] : 1.0};
    const double hn[3] = {h[0] / dta, h[1] / dta, h[2] / dta};
    const int64_t n[3] = {nx, ny, nz};
    double cover = 0;
    float far2[8];
    const int ntable = build_static_table(ndim, n, hn, &cover, far2);

    gk::Problem P{};
    P.ref = ref_dev;
    P.ev = eval_dev;
    P.out = gamma_out_dev;
    P.nvox = nvox;
    P.ndim = ndim;
    P.nx = (int)nx;
    P.ny = (int)ny;
    P.nz = (int)nz;
    double hn2[3];
    for (int a = 0; a < 3; ++a) {
        P.hn[a] = (float)hn[a];
        hn2[a] = hn[a] * hn[a];
        P.mt.hn2[a] = (float)hn2[a];
        P.mtd.hn2[a] = hn2[a];
    }
    for (int A = 1; A < 8; ++A) {
        double sum = 0;
        for (int a = 0; a < 3; ++a)
            if (A & (1 << a)) sum += hn2[a];
        P.mt.kappa[A] = (float)(1.0 / sum);
        P.mtd.kappa[A] = 1.0 / sum;
    }
    P.dd_frac = crit->dd_frac;
    P.cutoff_frac = crit->cutoff_frac;
    P.dose_norm = crit->dose_norm;
    P.local = crit->mode == GAMMA_LOCAL;
    P.tau = 1e-6f;
    P.stats = 0;
    P.table = (const gk::TableEntry*)(base + kOffTable);
    P.ntable = ntable;
    gk::fill_bucket_keys(g_table_host, ntable, P.bucket_key);
    for (int s = 0; s < 8; ++s) P.key0_far2[s] = far2[s];
    P.r_cover = std::isinf(cover) ? INFINITY : round_down_f(cover);
    P.tail_cap = (unsigned)kMaxVoxels;
    P.ctr = (gk::Counters*)(base + kOffCounters);
    P.tail_raw = (unsigned*)(base + kOffTail);
    P.tail_bucket = base + kOffBucket;
    P.tail_sorted = nullptr;
    P.sort_tail = 0;
    P.shell_minblocks = gk::kDefaultShellBlocksPerSm;

    // the table, kChunk entries per launch, each chunk copied into its
    // launch's parameters (static storage: the struct is 32 KB)
    static TableChunk chunk;
    for (int first = 0; first < ntable; first += kChunk) {
        chunk.first = first;
        chunk.count = std::min(kChunk, ntable - first);
        std::copy(g_table_host + first, g_table_host + first + chunk.count, chunk.e);
        k_table_fill<<<(chunk.count + 255) / 256, 256, 0, s>>>(
            (gk::TableEntry*)(base + kOffTable), chunk);
        if (cudaGetLastError() != cudaSuccess) return GAMMA_ERR_CUDA;
    }
    // the counters must start at zero; the rest is written before it is read
    if (cudaMemsetAsync(base + kOffCounters, 0, sizeof(gk::Counters), s) != cudaSuccess)
        return GAMMA_ERR_CUDA;
    if (gk::launch_prepare(P, s, 1) != cudaSuccess) return GAMMA_ERR_CUDA;
    if (gk::launch_shell(P, s) != cudaSuccess) return GAMMA_ERR_CUDA;
    if (gk::launch_tail(P, gk::kDefaultLanesPerVoxel, gk::kDefaultTailBlocksPerSm, s) != cudaSuccess)
        return GAMMA_ERR_CUDA;

    if (n_eval || n_pass) {
        gk::Counters c;
        if (cudaMemcpyAsync(&c, base + kOffCounters, sizeof(c), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return GAMMA_ERR_CUDA;
        if (c.flags & gk::kFlagNonFinite) return GAMMA_ERR_NAN_INPUT;
        if (crit->mode == GAMMA_GLOBAL && !(crit->dose_norm > 0.f) && !(gk::fdec(c.dnorm_enc) > 0.f))
            return GAMMA_ERR_DOSE_NORM;            // no voxel was evaluated
        if (n_eval) *n_eval = (int64_t)c.n_eval;
        if (n_pass) *n_pass = (int64_t)c.n_pass;
    }
    return GAMMA_OK;
}
