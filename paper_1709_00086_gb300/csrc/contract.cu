// zeta contraction, plain-FP32 form, and the FP64 reduction to zeta.
//
// Paper: Sec. 3.1 -- about one primary the coefficient is a_lm(r1) a*_l'm(r2),
// "repeated for all primaries"; Sec. 3.2/3.3 -- per-thread partial multipoles
// are combined at the end and reduced across nodes.  Here the sum over
// primaries is a per-m Gram matrix over the A rows,
//      C_m = sum_i w_i v_i v_i^T,   v_i = [Re a_m(i) | Im a_m(i)]  (m >= 1),
// from which zeta_m = (C_XX + C_YY) + i (C_YX - C_XY) (and zeta_0 = C_XX).
// Only upper tiles of the symmetric C_m are formed.  Every (segment of
// primaries, tile) pair is one CTA writing its own partial (FP64), and the
// reduction adds the segments of a catalog in a fixed order, so reruns give
// bit-identical zeta.
#include "internal.h"

namespace g3 {

namespace {

constexpr int kT = 64;       // tile edge
constexpr int kKC = 32;      // rows per smem stage
constexpr int kThreads = 256;
constexpr int kFlushRows = 256;  // FP32 run length before a compensated add

__device__ __forceinline__ void two_sum(double& hi, float v) {
    hi += (double)v;  // FP64 add of an FP32 run sum: error far below FP32 rounding
}

__global__ void __launch_bounds__(kThreads) k_contract_fp32(const float* __restrict__ A, int RLP,
                                                          const float* __restrict__ wrow,
                                                          const Tile* tiles, const Segment* segs,
                                                          double* partials, int part_stride) {
    __shared__ __align__(16) float sa[kKC][kT];
    __shared__ __align__(16) float sb[kKC][kT];
    const Tile t = tiles[blockIdx.x];
    const Segment sg = segs[blockIdx.y];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4];
    double tot[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            acc[i][j] = 0.f;
            tot[i][j] = 0.0;
        }
    int since = 0;
    for (int r0 = sg.row0; r0 < sg.row1; r0 += kKC) {
        // stage kKC rows of the two column windows (rows weighted on the left)
        for (int k = threadIdx.x; k < kKC * kT; k += kThreads) {
            const int rr = k / kT, cc = k % kT;
            const int row = r0 + rr;
            float va = 0.f, vb = 0.f;
            if (row < sg.row1) {
                const float* Ar = A + (int64_t)row * RLP + t.col0;
                if (cc < t.rows) va = Ar[t.r0 + cc] * wrow[row];
                if (cc < t.cols) vb = Ar[t.c0 + cc];
            }
            sa[rr][cc] = va;
            sb[rr][cc] = vb;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kKC; ++k) {
            const float4 a4 = *reinterpret_cast<const float4*>(&sa[k][ty * 4]);
            const float4 b4 = *reinterpret_cast<const float4*>(&sb[k][tx * 4]);
            const float av[4] = {a4.x, a4.y, a4.z, a4.w};
            const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
        since += kKC;
        if (since >= kFlushRows) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    two_sum(tot[i][j], acc[i][j]);
                    acc[i][j] = 0.f;
                }
            since = 0;
        }
    }
    double* out = partials + (int64_t)blockIdx.y * part_stride + t.out_off;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) out[(ty * 4 + i) * kT + tx * 4 + j] = tot[i][j] + (double)acc[i][j];
}

struct BlockInfo {
    int tile_base[kMaxL + 1];
    int ntile[kMaxL + 1];
    int width[kMaxL + 1];
    int zoff[kMaxL + 1];  // complex offset of block m inside one catalog's zeta
};

__device__ __forceinline__ double c_lookup(const double* part, const Tile* tiles,
                                           const BlockInfo& bi, int m, int a, int b, int T,
                                           int colmajor) {
    if (a > b) {
        const int t = a;
        a = b;
        b = t;
    }
    const int ti = a / T, tj = b / T, nt = bi.ntile[m];
    const int idx = bi.tile_base[m] + ti * nt - ti * (ti - 1) / 2 + (tj - ti);
    const Tile& tl = tiles[idx];
    return colmajor ? part[tl.out_off + (b - tl.c0) * T + (a - tl.r0)]
                    : part[tl.out_off + (a - tl.r0) * T + (b - tl.c0)];
}

__global__ void k_reduce(const double* partials, int part_stride, const int* seg_first, int ncat,
                         const Tile* tiles, BlockInfo bi, int nbins, int lmax, int T, int cm,
                         int64_t zsize, double* zeta) {
    const int cat = blockIdx.y;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= zsize || cat >= ncat) return;
    int m = 0;
    while (m < lmax && e >= bi.zoff[m + 1]) ++m;
    const int K = nbins * (lmax + 1 - m);
    const int64_t loc = e - bi.zoff[m];
    const int r = (int)(loc / K), c = (int)(loc % K);
    double re = 0.0, im = 0.0;
    for (int s = seg_first[cat]; s < seg_first[cat + 1]; ++s) {
        const double* p = partials + (int64_t)s * part_stride;
        if (m == 0) {
            re += c_lookup(p, tiles, bi, 0, r, c, T, cm);
        } else {
            re += c_lookup(p, tiles, bi, m, r, c, T, cm) + c_lookup(p, tiles, bi, m, K + r, K + c, T, cm);
            im += c_lookup(p, tiles, bi, m, K + r, c, T, cm) - c_lookup(p, tiles, bi, m, r, K + c, T, cm);
        }
    }
    double* z = zeta + 2 * ((int64_t)cat * zsize + e);
    z[0] = re;
    z[1] = im;
}

// Isotropic 3PCF from zeta: out[c][l][b1][b2] = Re zeta^0_ll(b1,b2)
// + 2 sum_{m=1}^{l} Re zeta^m_ll(b1,b2) (the m < 0 blocks folded in by
// zeta^{-m} = conj(zeta^m) for real weights).
__global__ void k_isotropic(const double* zeta, BlockInfo bi, int nbins, int lmax, int64_t zsize,
                            int ncat, double* out) {
    const int64_t per_cat = (int64_t)(lmax + 1) * nbins * nbins;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= per_cat * ncat) return;
    const int cat = (int)(e / per_cat);
    const int64_t r = e - cat * per_cat;
    const int l = (int)(r / ((int64_t)nbins * nbins));
    const int b1 = (int)((r / nbins) % nbins), b2 = (int)(r % nbins);
    const double* z = zeta + 2 * (int64_t)cat * zsize;
    double acc = 0.0;
    for (int m = 0; m <= l; ++m) {
        const int K = nbins * (lmax + 1 - m);
        const int64_t idx = bi.zoff[m] + (int64_t)((l - m) * nbins + b1) * K + (l - m) * nbins + b2;
        acc += (m == 0 ? 1.0 : 2.0) * z[2 * idx];
    }
    out[e] = acc;
}

// out[e] = sum_c coef[c] zeta_c[e] over the 2 zsize doubles of a zeta block,
// catalogs in index order (fixed summation order: reruns are bit-identical).
__global__ void k_combine(const double* zeta, int64_t n2, int ncat, CombineCoef cf, double* out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2; e += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < ncat; ++c) acc = fma(cf.c[c], zeta[(int64_t)c * n2 + e], acc);
        out[e] = acc;
    }
}

}  // namespace

int launch_combine(const double* zeta, int64_t zsize, int ncat, const double* coef, double* out, cudaStream_t st) {
    if (ncat < 1 || ncat > kMaxCombine) return -1;
    CombineCoef cf{};
    for (int c = 0; c < ncat; ++c) cf.c[c] = coef[c];
    const int64_t n2 = 2 * zsize;
    int64_t blocks = (n2 + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_combine<<<(unsigned)blocks, 256, 0, st>>>(zeta, n2, ncat, cf, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int contract_tile_dim_fp32() { return kT; }

// Tiles of edge T over the upper triangle of every C_m (row-major in (ti, tj)).
int make_tiles(int nbins, int lmax, int T, Tile* out, int max_tiles) {
    return fill_tiles(nbins, lmax, T, out, max_tiles);
}

int launch_contract_fp32(const float* A, int RLP, const float* wrow, const Tile* tiles, int ntiles,
                         const Segment* segs, int nsegs, double* partials, int part_stride,
                         cudaStream_t st) {
    if (ntiles <= 0 || nsegs <= 0) return 0;
    dim3 grid(ntiles, nsegs);
    k_contract_fp32<<<grid, kThreads, 0, st>>>(A, RLP, wrow, tiles, segs, partials, part_stride);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_reduce(const double* partials, int part_stride, const int* seg_first, int ncat,
                  int nbins, int lmax, const Tile* tiles, int T, double* zeta, cudaStream_t st,
                  int colmajor) {
    BlockInfo bi;
    int base = 0;
    int64_t zo = 0;
    for (int m = 0; m <= lmax; ++m) {
        const int K = nbins * (lmax + 1 - m);
        const int W = (m == 0) ? K : 2 * K;
        const int nt = (W + T - 1) / T;
        bi.tile_base[m] = base;
        bi.ntile[m] = nt;
        bi.width[m] = W;
        bi.zoff[m] = (int)zo;
        base += nt * (nt + 1) / 2;
        zo += (int64_t)K * K;
    }
    const int64_t zsize = zo;
    dim3 grid((unsigned)((zsize + 255) / 256), ncat);
    k_reduce<<<grid, 256, 0, st>>>(partials, part_stride, seg_first, ncat, tiles, bi, nbins, lmax,
                                   T, colmajor, zsize, zeta);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_isotropic(const double* zeta, int nbins, int lmax, int ncat, double* out, cudaStream_t st) {
    BlockInfo bi{};
    int64_t zo = 0;
    for (int m = 0; m <= lmax; ++m) {
        const int64_t K = (int64_t)nbins * (lmax + 1 - m);
        bi.zoff[m] = (int)zo;
        zo += K * K;
    }
    const int64_t total = (int64_t)(lmax + 1) * nbins * nbins * ncat;
    if (total == 0) return 0;
    k_isotropic<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(zeta, bi, nbins, lmax, zo, ncat, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace g3
