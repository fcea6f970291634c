// Device helpers shared by the pair-stage kernels (pair.cu: the fused
// forward/adjoint kernel; pairlist.cu: the count / scan / accumulate kernels).
// See pair.cu for the harmonics recurrence and the exact binning rule.
#pragma once

#include <type_traits>

#include "internal.h"

namespace g3 {
namespace {


constexpr int kPairWarps = 4;
constexpr int kPairThreads = kPairWarps * 32;
constexpr int kMaxPieces = 96;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kIdxBits = 27;
constexpr int kStashDepth = 4;  // scan iterations in flight per warp
constexpr int kBinTable = G3_BIN_TABLE;  // r^2 cells of the bin lookup table
constexpr unsigned kIdxMask = (1u << kIdxBits) - 1u;
constexpr int kTabReject = 254;  // bin table: 0..253 bin, 254 surely outside, 255 check

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__host__ __device__ constexpr float beta_lm(int l, int m) {
    return float(l * l - m * m) / float(4 * l * l - 1);
}

// Compile-time loop: f(std::integral_constant<int, I>) for I in [Begin, End).
// The accumulator indices below are therefore constants in the source, so the
// register arrays never depend on the loop unroller's cost limits (inside this
// large kernel the unroller gives up and the arrays would go to local memory).
template <int Begin, int End, class F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (Begin < End) {
        f(std::integral_constant<int, Begin>{});
        static_for<Begin + 1, End>(f);
    }
}

template <int L>
struct Shape {
    static constexpr int NR = (L + 1) * (L + 1);
    static constexpr int NRP = ((NR + 31) / 32) * 32;
    static constexpr int Q = NRP / 32;  // values per lane after the butterfly
};

// Accumulate one pair's w * Dt_lm(z) (x + iy)^m into the register partials.
template <int L>
__device__ __forceinline__ void accum_pair(float (&acc)[Shape<L>::NR], float z, float ux, float uy,
                                           float w) {
    // m = 0: real
    acc[0] += w;
    if constexpr (L >= 1) acc[1] = fmaf(w, z, acc[1]);
    float d0 = 1.f, d1 = z;
    static_for<2, L + 1>([&](auto lc) {
        constexpr int l = decltype(lc)::value;
        const float d2 = fmaf(z, d1, -beta_lm(l - 1, 0) * d0);
        acc[l] = fmaf(w, d2, acc[l]);
        d0 = d1;
        d1 = d2;
    });
    float cr = w * ux, ci = w * uy;  // w (x + iy)^m, m = 1
    static_for<1, L + 1>([&](auto mc) {
        constexpr int m = decltype(mc)::value;
        constexpr int b0 = acc_base(L, m);
        acc[b0] += cr;
        acc[b0 + 1] += ci;
        if constexpr (m + 1 <= L) {
            acc[b0 + 2] = fmaf(z, cr, acc[b0 + 2]);
            acc[b0 + 3] = fmaf(z, ci, acc[b0 + 3]);
        }
        float e0 = 1.f, e1 = z;
        static_for<m + 2, L + 1>([&](auto lc) {
            constexpr int l = decltype(lc)::value;
            const float e2 = fmaf(z, e1, -beta_lm(l - 1, m) * e0);
            acc[b0 + 2 * (l - m)] = fmaf(e2, cr, acc[b0 + 2 * (l - m)]);
            acc[b0 + 2 * (l - m) + 1] = fmaf(e2, ci, acc[b0 + 2 * (l - m) + 1]);
            e0 = e1;
            e1 = e2;
        });
        if constexpr (m < L) {
            const float t = fmaf(cr, ux, -ci * uy);
            ci = fmaf(cr, uy, ci * ux);
            cr = t;
        }
    });
}

// Accumulators of the Chebyshev form (pair-list path): for m = 0, acc0[k] +=
// w T_k(z); for m >= 1, accc[cidx(m) + k] += T_k(z) w (x + iy)^m as (Re, Im),
// k = 0..L-m.  The T_k (first kind, T_{k+1} = 2z T_k - T_{k-1}) do not depend
// on m, so one recurrence of L-1 steps serves every m, and each complex term
// costs one packed FMA.  The monic D_lm(z) of the Legendre form are
// non-negative combinations of the T_k (Gegenbauer-to-Chebyshev connection
// coefficients), applied per primary when its row of multipoles is written.
template <int L>
struct Cheb {
    static constexpr int NC = L * (L + 1) / 2;  // (l, m >= 1) terms
    __host__ __device__ static constexpr int cidx(int m) { return (m - 1) * (L + 1) - (m - 1) * m / 2; }
};

template <int L>
__device__ __forceinline__ void accum_pair_cheb(float (&acc0)[L + 1], float2 (&accc)[Cheb<L>::NC > 0 ? Cheb<L>::NC : 1],
                                                float z, float ux, float uy, float w) {
    float T[L + 1];
    T[0] = 1.f;
    acc0[0] += w;
    if constexpr (L >= 1) {
        T[1] = z;
        const float z2 = z + z;
        static_for<2, L + 1>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            T[k] = fmaf(z2, T[k - 1], -T[k - 2]);
        });
        static_for<1, L + 1>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            acc0[k] = fmaf(w, T[k], acc0[k]);
        });
        // w (x + iy)^m as two interleaved chains (odd m from m = 1, even m
        // from m = 2, each stepping by (x + iy)^2) to halve the dependency depth
        const float u2x = fmaf(ux, ux, -uy * uy), u2y = 2.f * ux * uy;
        float2 co = make_float2(w * ux, w * uy);                      // m = 1
        float2 ce = make_float2(fmaf(co.x, ux, -co.y * uy), fmaf(co.x, uy, co.y * ux));  // m = 2
        static_for<1, L + 1>([&](auto mc) {
            constexpr int m = decltype(mc)::value;
            constexpr int b = Cheb<L>::cidx(m);
            float2& c = (m & 1) ? co : ce;
            accc[b] = __fadd2_rn(accc[b], c);
            static_for<1, L - m + 1>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                accc[b + k] = __ffma2_rn(make_float2(T[k], T[k]), c, accc[b + k]);
            });
            if constexpr (m + 2 <= L) {
                const float t = fmaf(c.x, u2x, -c.y * u2y);
                c.y = fmaf(c.x, u2y, c.y * u2x);
                c.x = t;
            }
        });
    }
}

__host__ __device__ constexpr int bf_size(int n, int r) { return r == 0 ? n : (bf_size(n, r - 1) + 1) / 2; }

// Sum acc over the 32 lanes by recursive halving (5 rounds of shuffles; the
// array keeps exactly NR entries so that it stays in registers) and add the
// lane's share of the result to res_b.  Round r splits the current S entries
// into a lower half of h = ceil(S/2) and an upper half; the lane with bit
// (16 >> r) set keeps the upper half.  Each lane tracks the absolute range
// [base, base + size) it owns, so padding slots (always zero) are skipped.
template <int L>
__device__ __forceinline__ void butterfly_add(float (&acc)[Shape<L>::NR], int lane, float* res_b) {
    constexpr int NR = Shape<L>::NR;
    int base = 0, size = NR;
    static_for<0, 5>([&](auto rc) {
        constexpr int r = decltype(rc)::value;
        constexpr int S = bf_size(NR, r);
        constexpr int h = (S + 1) / 2;
        constexpr int o = 16 >> r;
        const bool hi = (lane & o) != 0;
        static_for<0, h>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            const float lo_v = acc[i];
            float hi_v = 0.f;
            if constexpr (i + h < S) hi_v = acc[i + h];
            const float keep = hi ? hi_v : lo_v;
            const float send = hi ? lo_v : hi_v;
            acc[i] = keep + __shfl_xor_sync(kFull, send, o);
        });
        if (hi) {
            base += h;
            size -= h;
        } else {
            size = size < h ? size : h;
        }
    });
    constexpr int Qf = bf_size(NR, 5);
    static_for<0, Qf>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        if (i < size) res_b[base + i] += acc[i];
    });
}

struct Prim {
    float x, y, z;
    double x64, y64, z64;
};

// Exact (FP64) bin of a candidate, with the reference's operation order.  The
// pair is accepted only through the minimum image: the row's image shift must
// equal the one the minimum-image rule picks.
__device__ __forceinline__ int exact_bin(const float4* __restrict__ pts, const double* pts64, int j,
                                      double xi, double yi, double zi, int sx, int sy, int sz,
                                      double L, int periodic, const double* e2, int B) {
    double xj, yj, zj;
    if (pts64) {
        xj = pts64[3 * (int64_t)j];
        yj = pts64[3 * (int64_t)j + 1];
        zj = pts64[3 * (int64_t)j + 2];
    } else {
        const float4 q = pts[j];
        xj = q.x;
        yj = q.y;
        zj = q.z;
    }
    const double half = 0.5 * L;
    double d[3] = {__dsub_rn(xj, xi), __dsub_rn(yj, yi), __dsub_rn(zj, zi)};
    const int want[3] = {sx, sy, sz};
    for (int k = 0; k < 3; ++k) {
        int s = 0;
        if (periodic) {
            if (d[k] > half) {
                d[k] = __dsub_rn(d[k], L);
                s = -1;
            } else if (d[k] < -half) {
                d[k] = __dadd_rn(d[k], L);
                s = 1;
            }
        }
        if (s != want[k]) return -1;
    }
    double r2 = __dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1]));
    r2 = __dadd_rn(r2, __dmul_rn(d[2], d[2]));
    if (r2 == 0.0) return -1;
    if (r2 < e2[0] || !(r2 < e2[B])) return -1;
    int b = 0;
    while (b + 1 < B && e2[b + 1] <= r2) ++b;
    return b;
}


// Slot ranges of row r of the (2K+1)^2 rows of cells around a primary at P0
// whose cell is (cy, cz): the x-range of cells that the sphere of radius
// rmax (+ slack) can reach in that row, split by x image (-L, 0, +L) into at
// most three contiguous ranges {first slot, end slot, image code, 0}; empty
// ranges have end <= first.  code = (sx+1) + 3 (sy+1) + 9 (sz+1).
__device__ __forceinline__ void row_pieces(int r, int W, int K, int cy, int cz, float4 P0,
                                           const Grid& g, float slack, float rmax2, long long kbase,
                                           const int* __restrict__ cstart, int4& pm, int4& p0,
                                           int4& pp) {
    pm = make_int4(0, 0, 0, 0);
    p0 = pm;
    pp = pm;
    const int ycell = cy + (r % W) - K;
    const int zcell = cz + (r / W) - K;
    bool ok;
    int wy = ycell, wz = zcell, sy = 0, sz = 0;
    if (g.periodic) {
        sy = ycell < 0 ? -1 : (ycell >= g.nc ? 1 : 0);
        sz = zcell < 0 ? -1 : (zcell >= g.nc ? 1 : 0);
        wy = ycell - sy * g.nc;
        wz = zcell - sz * g.nc;
        ok = wy >= 0 && wy < g.nc && wz >= 0 && wz < g.nc;
    } else {
        ok = ycell >= 0 && ycell < g.nc && zcell >= 0 && zcell < g.nc;
    }
    if (!ok) return;
    const float ylo = ycell * g.cell, zlo = zcell * g.cell;
    const float ddy = fmaxf(0.f, fmaxf(ylo - P0.y, P0.y - (ylo + g.cell)) - slack);
    const float ddz = fmaxf(0.f, fmaxf(zlo - P0.z, P0.z - (zlo + g.cell)) - slack);
    const float rem = rmax2 - ddy * ddy - ddz * ddz;
    if (rem < 0.f) return;
    const float h = sqrtf(rem) + slack;
    const int nx = g.ncx;
    int xlo = (int)floorf((P0.x - h) * g.inv_cellx);
    int xhi = (int)floorf((P0.x + h) * g.inv_cellx);
    if (!g.periodic) {
        xlo = max(xlo, 0);
        xhi = min(xhi, nx - 1);
    } else {
        xlo = max(xlo, -nx);
        xhi = min(xhi, 2 * nx - 1);
    }
    const long long pk = kbase + (long long)morton2(wy, wz) * nx;
    auto piece = [&](int s) {
        int4 v = make_int4(0, 0, 0, 0);
        const int a0 = max(xlo, s * nx), a1 = min(xhi, s * nx + nx - 1);
        if (a0 <= a1 && (g.periodic || s == 0)) {
            v.x = cstart[pk + (a0 - s * nx)];
            v.y = cstart[pk + (a1 - s * nx) + 1];
            v.z = (s + 1) + 3 * (sy + 1) + 9 * (sz + 1);
        }
        return v;
    };
    pm = piece(-1);
    p0 = piece(0);
    pp = piece(1);
}

// Entry (lane, lane < 9) of the 3x3 rotation, row-major, that takes the line
// of sight (box centre -> primary at x) to +z (radial mode, Sec. 2): with
// n = unit LOS and v = n x z, R = I + [v]x + [v]x^2 / (1 + n.z); the
// antiparallel case is the half turn about x.  A primary at the centre keeps I.
__device__ __forceinline__ double los_rotation_entry_d(int lane, double x0, double x1, double x2,
                                                       double boxd) {
    const int r = lane / 3, s = lane % 3;
    double Rv = (r == s) ? 1.0 : 0.0;
    const double c = 0.5 * boxd;
    double n0 = x0 - c, n1 = x1 - c, n2 = x2 - c;
    const double nn = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
    if (nn > 0.0) {
        n0 /= nn;
        n1 /= nn;
        n2 /= nn;
        if (n2 < -1.0 + 1e-12) {
            Rv = (lane == 0) ? 1.0 : ((lane == 4 || lane == 8) ? -1.0 : 0.0);
        } else {
            const double v0 = n1, v1 = -n0, f = 1.0 / (1.0 + n2);
            // [v]x = [[0, 0, v1], [0, 0, -v0], [-v1, v0, 0]] (v2 = 0)
            auto kx = [&](int i, int k) -> double {
                return (i == 0 && k == 2) ? v1
                       : (i == 1 && k == 2) ? -v0
                       : (i == 2 && k == 0) ? -v1
                       : (i == 2 && k == 1) ? v0
                                            : 0.0;
            };
            const double k2 = kx(r, 0) * kx(0, s) + kx(r, 1) * kx(1, s) + kx(r, 2) * kx(2, s);
            Rv = ((r == s) ? 1.0 : 0.0) + kx(r, s) + k2 * f;
        }
    }
    return Rv;
}
__device__ __forceinline__ float los_rotation_entry(int lane, double x0, double x1, double x2,
                                                    double boxd) {
    return (float)los_rotation_entry_d(lane, x0, x1, x2, boxd);
}

// A float widened to double by its IEEE-754 fields on the integer ALU (sign,
// exponent rebiased from 127 to 1023, 23 mantissa bits moved to the top of
// 52): exact, and no FP64-pipe conversion, which runs at 1/64 of the FP32
// rate here.  Zero keeps its sign; subnormal, infinite and NaN inputs take the
// plain conversion.
__device__ __forceinline__ double f2d_exact(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu;
    if ((u & 0x7fffffffu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
    if (e == 0u || e == 0xffu) return (double)x;
    const unsigned hi = (u & 0x80000000u) | ((e + (1023u - 127u)) << 20) | ((u >> 3) & 0x000fffffu);
    return __hiloint2double((int)hi, (int)(u << 29));
}

// Cell coordinates of a position (the index build's formula).
__device__ __forceinline__ int cell_of(float x, const Grid& g) {
    const int c = (int)(x * g.inv_cell);
    return c < 0 ? 0 : (c >= g.nc ? g.nc - 1 : c);
}

// The bin of a candidate at squared FP32 distance r2 (-1: not a pair), using the
// r^2 table, the guard-widened FP32 edges and, inside a guard band, the exact
// FP64 rule.  tab/dec/e2 are shared-memory copies.
__device__ __forceinline__ int decide_bin(float r2, float hi_rej, float lo_rej, float tscale,
                                          const unsigned char* tab, float guard0,
                                          const float2* dec, float rminf, float invw, int B,
                                          bool exact_inputs, int code, const float4* __restrict__ pts,
                                          const double* pts64, int j, const double* pd, double boxd,
                                          int periodic, const double* e2) {
    if (!(r2 < hi_rej)) return -1;
    int ti = (int)(r2 * tscale);
    ti = ti > kBinTable + 1 ? kBinTable + 1 : ti;
    const int tv = tab[ti];
    if (tv < kTabReject) return tv;
    if (tv == kTabReject) return -1;
    if (r2 < lo_rej) return -1;
    int bin;
    if (!(r2 > guard0)) {
        bin = (exact_inputs && code == 13 && r2 == 0.f) ? -1 : -2;
    } else {
        const float rr = r2 * rsqrtf(r2);
        int bb = (int)((rr - rminf) * invw);
        bb = bb < 0 ? 0 : (bb >= B ? B - 1 : bb);
        const float2 iv = dec[bb];
        bin = (r2 > iv.x && r2 < iv.y) ? bb : -2;
    }
    if (bin == -2)
        bin = exact_bin(pts, pts64, j, pd[0], pd[1], pd[2], code % 3 - 1, (code / 3) % 3 - 1,
                        code / 9 - 1, boxd, periodic, e2, B);
    return bin;
}

// decide_bin split for warp-wide use: bin_fast settles almost every
// candidate with one lookup in the signed r^2 table (bin, -1 = no pair, -3 =
// in a guard band or an ambiguous cell; indices past the table clamp to its
// last entry, which is -1); bin_slow finishes the -3 cases.
__device__ __forceinline__ int bin_fast(float r2, float tscale, const signed char* tab) {
    int ti = (int)(r2 * tscale);
    ti = ti > kBinTable + 1 ? kBinTable + 1 : ti;
    return tab[ti];
}
__device__ __noinline__ int bin_slow(float r2, float lo_rej, float hi_rej, float guard0, const float2* dec,
                                     float rminf, float invw, int B, bool exact_inputs, int code,
                                     const float4* __restrict__ pts, const double* pts64, int j,
                                     const double* pd, double boxd, int periodic, const double* e2) {
    if (r2 < lo_rej || !(r2 < hi_rej)) return -1;
    int bin;
    if (!(r2 > guard0)) {
        bin = (exact_inputs && code == 13 && r2 == 0.f) ? -1 : -2;
    } else {
        const float rr = r2 * rsqrtf(r2);
        int bb = (int)((rr - rminf) * invw);
        bb = bb < 0 ? 0 : (bb >= B ? B - 1 : bb);
        const float2 iv = dec[bb];
        bin = (r2 > iv.x && r2 < iv.y) ? bb : -2;
    }
    if (bin == -2)
        bin = exact_bin(pts, pts64, j, pd[0], pd[1], pd[2], code % 3 - 1, (code / 3) % 3 - 1,
                        code / 9 - 1, boxd, periodic, e2, B);
    return bin;
}

}  // namespace
}  // namespace g3
