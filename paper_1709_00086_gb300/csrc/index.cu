// Device spatial index: cell keys, a stable LSD radix sort of (key, index),
// the sorted point arrays and the first-slot table of every cell.
//
// Replaces the paper's node-local k-d tree (Algorithm 1, "search node-local
// k-d tree for neighbors"; Sec. 5.1, FP32 tree search) with a uniform grid of
// side >= rmax/s whose cells are ordered by (catalog, Morton(cy, cz), cx): an
// x-row of cells is one contiguous slot range, so a sphere of radius rmax is
// covered by a few dozen contiguous ranges.  Everything here is HBM-bound
// streaming (a few passes over 8-16 bytes per point).
#include "internal.h"

#include <cstdio>

namespace g3 {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kTile = kSortThreads * kSortItems;  // 4096 keys per tile
constexpr int kScanBlock = 1024;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---- keys ----------------------------------------------------------------

__global__ void k_keys(IndexArgs a, const int64_t* cat_off, int ncat, unsigned* key,
                       int* val, int* status) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    double x[3];
    if (a.pos_f64) {
        const double* p = static_cast<const double*>(a.pos) + 3 * i;
        x[0] = p[0]; x[1] = p[1]; x[2] = p[2];
    } else {
        const float* p = static_cast<const float*>(a.pos) + 3 * i;
        x[0] = p[0]; x[1] = p[1]; x[2] = p[2];
    }
    float w = a.w[i];
    bool bad = !isfinite(w);
    int c[3];
    for (int d = 0; d < 3; ++d) {
        if (!(x[d] >= 0.0 && x[d] < a.g.boxd)) {  // also catches NaN
            bad = true;
            x[d] = 0.0;
        }
        const float xf = (float)x[d];
        const int n = d == 0 ? a.g.ncx : a.g.nc;
        const int cc = (int)(xf * (d == 0 ? a.g.inv_cellx : a.g.inv_cell));
        c[d] = cc < 0 ? 0 : (cc >= n ? n - 1 : cc);
    }
    if (bad) atomicOr(status, kStatusRange);
    long long cat = 0;
    if (cat_off) {
        int lo = 0, hi = ncat - 1;  // last catalog with cat_off[c] <= i
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (cat_off[mid] <= i) lo = mid; else hi = mid - 1;
        }
        cat = lo;
    }
    long long k = cat * a.g.cells_per_cat + (long long)morton2(c[1], c[2]) * a.g.ncx + c[0];
    key[i] = (unsigned)k;
    val[i] = (int)i;
}

// ---- exclusive scan (int32) --------------------------------------------

__device__ int block_scan_excl(int v, int* sh, int& total) {
    // blockDim.x == kScanBlock; warp shuffles then warp totals
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    int pre = (wid > 0 ? sh[wid - 1] : 0) + x - v;
    total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return pre;
}

__global__ void k_scan_reduce(const int* in, int64_t n, int* bsum) {
    __shared__ int sh[32];
    int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    int v = i < n ? in[i] : 0;
    int tot;
    block_scan_excl(v, sh, tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_top(int* bsum, int nb) {
    __shared__ int sh[32];
    int carry = 0;
    for (int base = 0; base < nb; base += kScanBlock) {
        int i = base + threadIdx.x;
        int v = i < nb ? bsum[i] : 0;
        int tot;
        int pre = block_scan_excl(v, sh, tot);
        if (i < nb) bsum[i] = carry + pre;
        carry += tot;
    }
}

__global__ void k_scan_final(const int* in, int64_t n, const int* bsum, int* out) {
    __shared__ int sh[32];
    int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    int v = i < n ? in[i] : 0;
    int tot;
    int pre = block_scan_excl(v, sh, tot);
    if (i < n) out[i] = bsum[blockIdx.x] + pre;
}

// ---- radix sort -----------------------------------------------------------

__global__ void k_radix_hist(const unsigned* key, int64_t n, int shift, int ntiles, int* hist) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll 4
    for (int it = 0; it < kSortItems; ++it) {
        int64_t i = base + it * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(key[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: warp w of a tile owns tile items [w*512, (w+1)*512) and
// ranks them round by round (32 at a time) with per-warp digit counters; the
// warps' counters are then prefix-summed per digit in warp order.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const unsigned* key, const int* val, int64_t n, int shift, int ntiles, const int* offs,
    unsigned* key_out, int* val_out) {
    constexpr int kWarps = kSortThreads / 32;
    constexpr int kPerWarp = kTile / kWarps;    // 512
    constexpr int kRounds = kPerWarp / 32;      // 16
    __shared__ int wcnt[kWarps][257];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kWarps * 257; d += kSortThreads) (&wcnt[0][0])[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile + wid * kPerWarp;
    unsigned kk[kRounds];
    int vv[kRounds];
    int loc[kRounds];
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        int64_t i = base + r * 32 + lane;
        unsigned k = 0;
        int v = 0;
        int dg = 256;  // sentinel digit for items past the end
        if (i < n) {
            k = key[i];
            v = val[i];
            dg = (k >> shift) & 255u;
        }
        kk[r] = k;
        vv[r] = v;
        unsigned peers = __match_any_sync(0xffffffffu, dg);
        int leader = __ffs(peers) - 1;
        int b = 0;
        if (lane == leader) {
            b = wcnt[wid][dg];
            wcnt[wid][dg] = b + __popc(peers);
        }
        b = __shfl_sync(0xffffffffu, b, leader);
        loc[r] = b + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();
    {
        int d = threadIdx.x;  // 256 threads <-> 256 digits
        int run = 0;
        for (int w = 0; w < kWarps; ++w) {
            int t = wcnt[w][d];
            wcnt[w][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        int64_t i = base + r * 32 + lane;
        if (i < n) {
            int dg = (kk[r] >> shift) & 255u;
            int pos = offs[dg * ntiles + blockIdx.x] + wcnt[wid][dg] + loc[r];
            key_out[pos] = kk[r];
            val_out[pos] = vv[r];
        }
    }
}

// ---- sorted arrays, cell starts, primary list -------------------------------

__global__ void k_gather(IndexArgs a, const int* val, float4* pts, double* pts64, int* orig, int* negw) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= a.n) return;
    int i = val[p];
    double x[3];
    if (a.pos_f64) {
        const double* q = static_cast<const double*>(a.pos) + 3 * (int64_t)i;
        x[0] = q[0]; x[1] = q[1]; x[2] = q[2];
    } else {
        const float* q = static_cast<const float*>(a.pos) + 3 * (int64_t)i;
        x[0] = q[0]; x[1] = q[1]; x[2] = q[2];
    }
    for (int d = 0; d < 3; ++d)
        if (!(x[d] >= 0.0 && x[d] < a.g.boxd)) x[d] = 0.0;  // flagged in k_keys
    float w = a.w[i];
    if (!isfinite(w)) w = 0.f;
    if (w < 0.f) *negw = 1;
    pts[p] = make_float4((float)x[0], (float)x[1], (float)x[2], w);
    if (pts64) {
        pts64[3 * p + 0] = x[0];
        pts64[3 * p + 1] = x[1];
        pts64[3 * p + 2] = x[2];
    }
    orig[p] = i;
}

__global__ void k_cell_start(const unsigned* key, int64_t n, long long ncells, int* cstart) {
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c > ncells) return;
    int64_t lo = 0, hi = n;  // first slot with key >= c
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((long long)key[mid] < c) lo = mid + 1; else hi = mid;
    }
    cstart[c] = (int)lo;
}

__global__ void k_prim_flag(const int* orig, int64_t n, int64_t n_primary, int* flag) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < n) flag[p] = orig[p] < n_primary ? 1 : 0;
}

__global__ void k_prim_compact(const int* flag, const int* pos, int64_t n, int* plist) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < n && flag[p]) plist[pos[p]] = (int)p;
}

__global__ void k_iota_ranges(const int* rstart, const int* rlen, const int* rout, int nr,
                              int* plist) {
    // one block per range
    int r = blockIdx.x;
    if (r >= nr) return;
    for (int k = threadIdx.x; k < rlen[r]; k += blockDim.x) plist[rout[r] + k] = rstart[r] + k;
}

inline int grid_of(int64_t n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

int scan_exclusive(const int* in, int* out, int64_t n, int* tmp, cudaStream_t st) {
    if (n <= 0) return 0;
    int nb = grid_of(n, kScanBlock);
    k_scan_reduce<<<nb, kScanBlock, 0, st>>>(in, n, tmp);
    k_scan_top<<<1, kScanBlock, 0, st>>>(tmp, nb);
    k_scan_final<<<nb, kScanBlock, 0, st>>>(in, n, tmp, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

size_t scan_tmp_ints(int64_t n) { return (size_t)grid_of(n, kScanBlock) + 1; }

size_t radix_hist_ints(int64_t n) { return (size_t)256 * grid_of(n, kTile) + 1; }

int build_index(IndexBuffers& b, const IndexArgs& a, const int64_t* cat_off_dev, int ncat,
                long long ncells, int64_t n_primary, const PrimRanges* ranges,
                cudaStream_t st) {
    const int64_t n = a.n;
    if (n <= 0) return 0;
    const int T = 256;
    int launches = 0;
    k_keys<<<grid_of(n, T), T, 0, st>>>(a, cat_off_dev, ncat, b.key_a, b.val_a, b.status);
    // LSD radix sort on the bits in use
    int bits = 1;
    while (bits < 32 && ((unsigned long long)1 << bits) <= (unsigned long long)ncells) ++bits;
    const int ntiles = grid_of(n, kTile);
    unsigned* kin = b.key_a;
    int* vin = b.val_a;
    unsigned* kout = b.key_b;
    int* vout = b.val_b;
    for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<<<ntiles, kSortThreads, 0, st>>>(kin, n, shift, ntiles, b.hist);
        scan_exclusive(b.hist, b.hist_off, (int64_t)256 * ntiles, b.scan_tmp, st);
        k_radix_scatter<<<ntiles, kSortThreads, 0, st>>>(kin, vin, n, shift, ntiles, b.hist_off,
                                                         kout, vout);
        launches += 5;
        unsigned* tk = kin; kin = kout; kout = tk;
        int* tv = vin; vin = vout; vout = tv;
    }
    b.key_sorted = kin;
    k_gather<<<grid_of(n, T), T, 0, st>>>(a, vin, b.pts, b.pts64, b.orig, b.status + kNegWeightSlot);
    k_cell_start<<<(int)((ncells + 1 + T - 1) / T), T, 0, st>>>(kin, n, ncells, b.cstart);
    launches += 3;
    // primary list
    if (ranges) {
        k_iota_ranges<<<ranges->n, 256, 0, st>>>(ranges->start, ranges->len, ranges->out,
                                                 ranges->n, b.plist);
        launches += 1;
    } else if (n_primary < n) {
        k_prim_flag<<<grid_of(n, T), T, 0, st>>>(b.orig, n, n_primary, vout);
        scan_exclusive(vout, b.hist_off, n, b.scan_tmp, st);
        k_prim_compact<<<grid_of(n, T), T, 0, st>>>(vout, b.hist_off, n, b.plist);
        launches += 5;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "g3pcf index: %s\n", cudaGetErrorString(e));
        return -1;
    }
    return launches;
}

}  // namespace g3
