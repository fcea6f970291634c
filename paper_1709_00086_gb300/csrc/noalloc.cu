// Allocation-free variant of the zeta contraction + FP64 reduction.
//
// Some callers cannot call cudaMalloc: code that runs with a fixed, reserved
// device-memory footprint (an embedding framework that owns every byte of the
// device heap, or a service with a hard memory budget), and code that must not
// hit cudaMalloc's implicit device-wide synchronisation in the middle of a
// streamed pipeline.  For them g3pcf_zeta_from_alm_noalloc turns per-primary
// multipoles they already hold into zeta without allocating anything: the
// per-segment partial sums and the small tile tables it needs live in
// file-scope device arrays of fixed size that exist, on every GPU that loads
// this library, until the process exits.
//
// The arrays are shared by all calls.  Each call rewrites its tile and segment
// tables on the device (a one-thread kernel, so nothing is copied from host
// memory), and overwrites every partial it reads and every zeta entry it
// writes, so nothing has to start at zero; but two calls whose work overlaps
// on the GPU (on different streams, or from different host threads) race on
// the same arrays and must be ordered by the caller.  The device addresses of
// the arrays are looked up once per device, by the first call made with that
// device current, and kept until the process exits; a cudaDeviceReset()
// invalidates them, so this entry point must not be used on a device after
// that device has been reset.
#include <cstdio>
#include <mutex>

#include "internal.h"

namespace g3 {
namespace {

constexpr size_t kNoAllocPartialDoubles = (size_t)2 << 20;  // 16 MiB of FP64 partials
constexpr int kNoAllocMaxTiles = 1024;
constexpr int kNoAllocMaxSegs = 64;

static __device__ __align__(256) double g_partials[kNoAllocPartialDoubles];
static __device__ __align__(256) Tile g_tiles[kNoAllocMaxTiles];
static __device__ __align__(256) Segment g_segs[kNoAllocMaxSegs];
static __device__ __align__(256) int g_segfirst[2];

// Writes the tile table and the segments of one call straight into the fixed
// arrays (device code may name them), so that no table is copied from host
// memory.  One thread: the tables hold at most a few hundred entries.
__global__ void k_fill_tables(int nbins, int lmax, int T, int64_t np, int64_t seg, int nsegs) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    fill_tiles(nbins, lmax, T, g_tiles, kNoAllocMaxTiles);
    for (int s = 0; s < nsegs; ++s) {
        const int64_t r0 = (int64_t)s * seg;
        g_segs[s].cat = 0;
        g_segs[s].row0 = (int)r0;
        g_segs[s].row1 = (int)(r0 + seg < np ? r0 + seg : np);
    }
    g_segfirst[0] = 0;
    g_segfirst[1] = nsegs;
}

struct SymbolAddrs {
    int device = -1;
    double* partials = nullptr;
    Tile* tiles = nullptr;
    Segment* segs = nullptr;
    int* segfirst = nullptr;
};

// Host-side addresses of the arrays, looked up once per device (with that
// device current) and kept for the life of the process.  In host code the
// array names are host stand-ins, not device addresses; only the addresses
// returned by cudaGetSymbolAddress are passed to kernels.  The mutex makes
// concurrent first calls from several host threads safe.
SymbolAddrs g_addrs[64];
std::mutex g_addrs_mu;

int resolve(int dev, SymbolAddrs& out) {
    if (dev < 0 || dev >= 64) return -1;
    std::lock_guard<std::mutex> lock(g_addrs_mu);
    SymbolAddrs& s = g_addrs[dev];
    if (s.device != dev) {
        SymbolAddrs t;
        if (cudaGetSymbolAddress((void**)&t.partials, g_partials) != cudaSuccess ||
            cudaGetSymbolAddress((void**)&t.tiles, g_tiles) != cudaSuccess ||
            cudaGetSymbolAddress((void**)&t.segs, g_segs) != cudaSuccess ||
            cudaGetSymbolAddress((void**)&t.segfirst, g_segfirst) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        t.device = dev;
        s = t;
    }
    out = s;
    return 0;
}

}  // namespace

int noalloc_zeta_from_alm(int nbins, int lmax, const float* alm, int64_t ld, const float* w,
                          int64_t np, double* zeta, cudaStream_t st, char* err, size_t errlen) {
    const int T = contract_tile_dim_fp32();
    // the table's size only (the table itself is written on the device)
    const int ntiles = count_tiles(nbins, lmax, T);
    const int RL = nbins * (lmax + 1) * (lmax + 1);
    if (ntiles > kNoAllocMaxTiles) {
        snprintf(err, errlen, "nbins*(lmax+1) too large for the static tile table (%d tiles max)",
                 kNoAllocMaxTiles);
        return G3PCF_ERR_ARG;
    }
    if (ld < RL) {
        snprintf(err, errlen, "ld (%lld) must be >= nbins*(lmax+1)^2 (%d)", (long long)ld, RL);
        return G3PCF_ERR_ARG;
    }
    const size_t part_stride = (size_t)ntiles * T * T;
    if (part_stride > kNoAllocPartialDoubles) {
        snprintf(err, errlen, "one segment needs %zu partial doubles, more than the static maximum %zu",
                 part_stride, kNoAllocPartialDoubles);
        return G3PCF_ERR_ARG;
    }
    int nsegs_max = (int)(kNoAllocPartialDoubles / part_stride);
    if (nsegs_max > kNoAllocMaxSegs) nsegs_max = kNoAllocMaxSegs;
    // segments of primaries: at least 4096 rows each, at most nsegs_max of them
    int64_t seg = 4096;
    int nsegs = 0;
    if (np > 0) {
        seg = (np + nsegs_max - 1) / nsegs_max;
        if (seg < 4096) seg = 4096;
        nsegs = (int)((np + seg - 1) / seg);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        snprintf(err, errlen, "cudaGetDevice failed");
        return G3PCF_ERR_CUDA;
    }
    SymbolAddrs sa;
    if (resolve(dev, sa) != 0) {
        snprintf(err, errlen, "cudaGetSymbolAddress failed for the static scratch arrays");
        return G3PCF_ERR_CUDA;
    }
    if (nsegs == 0) {
        const int64_t zs = g3pcf_zeta_size(nbins, lmax);
        if (cudaMemsetAsync(zeta, 0, sizeof(double) * 2 * zs, st) != cudaSuccess) {
            snprintf(err, errlen, "cudaMemsetAsync failed");
            return G3PCF_ERR_CUDA;
        }
        return G3PCF_OK;
    }
    k_fill_tables<<<1, 1, 0, st>>>(nbins, lmax, T, np, seg, nsegs);
    if (cudaGetLastError() != cudaSuccess ||
        launch_contract_fp32(alm, (int)ld, w, sa.tiles, ntiles, sa.segs, nsegs, sa.partials,
                             (int)part_stride, st) != 0 ||
        launch_reduce(sa.partials, (int)part_stride, sa.segfirst, 1, nbins, lmax, sa.tiles, T,
                      zeta, st) != 0) {
        snprintf(err, errlen, "kernel launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        return G3PCF_ERR_CUDA;
    }
    return G3PCF_OK;
}

}  // namespace g3

extern "C" int g3pcf_zeta_from_alm_noalloc(int nbins, int lmax, const float* alm, int64_t ld,
                                           const float* w, int64_t np, double* zeta,
                                           void* stream) {
    char err[256];
    err[0] = 0;
    int rc = G3PCF_OK;
    if (nbins < 1 || nbins > G3PCF_MAX_NBINS || lmax < 0 || lmax > G3PCF_MAX_LMAX) {
        snprintf(err, sizeof(err), "need 1 <= nbins <= %d and 0 <= lmax <= %d", G3PCF_MAX_NBINS,
                 G3PCF_MAX_LMAX);
        rc = G3PCF_ERR_ARG;
    } else if (np < 0 || np >= G3PCF_MAX_POINTS || !zeta || (np > 0 && (!alm || !w))) {
        snprintf(err, sizeof(err), "need 0 <= np < 2^27, non-null zeta, and alm/w when np > 0");
        rc = G3PCF_ERR_ARG;
    } else if (ld >= ((int64_t)1 << 31)) {
        snprintf(err, sizeof(err), "ld too large");
        rc = G3PCF_ERR_ARG;
    } else {
        rc = g3::noalloc_zeta_from_alm(nbins, lmax, alm, ld, w, np, zeta,
                                       static_cast<cudaStream_t>(stream), err, sizeof(err));
    }
    g3::set_last_error(rc == G3PCF_OK ? "" : err);
    return rc;
}
