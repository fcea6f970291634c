// Pair-stage kernels for multipoles that are differentiated: the forward
// multipoles a_lm of Sec. 3.1 and the adjoint pair pass, both in double-float
// arithmetic (an FP32 head plus an FP32 tail, about 44 significant bits) over
// the same per-bin pair lists as the FP32 kernels of pairlist.cu.
//
// Why: in the Chebyshev form Y_lm = K_lm sum_k c_k T_k(z) (x + iy)^m the
// connection coefficients c_k are non-negative and large where D_lm(1) is much
// larger than D_lm(z) in the bulk, so any per-pair rounding of the terms
// T_k (x + iy)^m (and of the unit vector they come from) reaches the gradient
// amplified by up to two orders of magnitude.  FP32 evaluation leaves the
// gradient near 1e-6 of its largest component at lmax = 10; carrying every
// per-pair quantity and every sum in double-float, and the conversions in
// FP64, brings it to the 1e-8 level, at a fraction of the cost of FP64, which
// runs at 1/58 of the FP32 rate on this part.
//
//   k_accum_df -- per primary (one warp).  Per chunk of 32 list entries each
//                 lane evaluates one pair: the separation from the primary's
//                 image (FP32 head + tail of the FP64 image, so the difference
//                 is exact), r^2, 1/r by one Newton step from rsqrt, the unit
//                 vector, T_k(z) and w (x + iy)^m, all in double-float, into a
//                 shared-memory record.  Then every lane adds the chunk's 32
//                 terms T_k w (x + iy)^m to the accumulator slots it owns, two
//                 slots per packed f32x2 operation (double-float sums, no
//                 cross-lane reduction).  At a change of bin the slots go to
//                 double-float shared memory; at the primary's end the
//                 Chebyshev -> Legendre-form connection (times K_lm, head +
//                 tail coefficients) is applied in double-float and the row
//                 of A is stored.  No FP64 arithmetic: the FP64 pipe runs at
//                 1/58 of the FP32 rate here.
//   k_adj_df   -- per primary (one warp), one pair per lane: the adjoint
//                 coefficients G_{m,k} = w_i sum_l c^(m)_{l-m,k} K_lm V_lm of
//                 the primary (FP64 from the FP64 V = M A, held as head + tail
//                 in shared memory), and per pair F = sum Re(conj(G) T_k
//                 (x + iy)^m) with its gradient in double-float (F with dF/dz,
//                 and the per-m sums against T_k and T_k', as packed f32x2
//                 pairs), rounded once to FP32 per pair; FP64 atomics for the
//                 secondary, a double-float sum for the primary.
#include "pair_common.cuh"

namespace g3 {
namespace {

constexpr int kDWarps = 4;
constexpr int kDThreads = kDWarps * 32;
constexpr unsigned kNoPairD = 0xffffffffu;

// ---- double-float arithmetic (error-free transformations) ----------------
// Every operation uses the _rn intrinsics so that the compiler never fuses a
// product into a later addition: the error terms below rely on each rounding.
struct df {
    float h, l;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
// |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df a, df b) {
    const df s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ df df_neg(df a) { return {-a.h, -a.l}; }
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
    return fast_two_sum(p, e);
}
// product left unnormalised (head, tail with |tail| <~ ulp(head)): for sums
__device__ __forceinline__ df df_mul_u(df a, df b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
    return {p, e};
}
__device__ __forceinline__ df df_mulf(df a, float b) {
    const float p = __fmul_rn(a.h, b);
    float e = __fmaf_rn(a.h, b, -p);
    e = __fmaf_rn(a.l, b, e);
    return fast_two_sum(p, e);
}
// acc += t (t unnormalised): the head's rounding error goes to the tail
__device__ __forceinline__ void df_acc(df& acc, df t) {
    const df s = two_sum(acc.h, t.h);
    acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, t.l));
    acc.h = s.h;
}
__device__ __forceinline__ df df_from(double v) {
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ double df_to(df a) { return (double)a.h + (double)a.l; }

// (a + ib)(c + id) in double-float
__device__ __forceinline__ void df_cmul(df a, df b, df c, df d, df& re, df& im) {
    re = df_add(df_mul_u(a, c), df_neg(df_mul_u(b, d)));
    im = df_add(df_mul_u(a, d), df_mul_u(b, c));
}

// One coordinate of the separation q - (head + tail): exact up to the tail's
// own rounding (|tail| <= half an ulp of the image), renormalised.
__device__ __forceinline__ df sep(float qh, float ql, float h, float t) {
    const df s = two_sum(qh, -h);
    return two_sum(s.h, __fadd_rn(s.l, __fsub_rn(ql, t)));
}

// Unit vector and 1/r of the separation d (double-float), optionally rotated
// by R (radial line of sight).
__device__ __forceinline__ void unit_df(df dx, df dy, df dz, const df* R, bool radial, df& ux, df& uy, df& uz,
                                        df& rinv) {
    if (radial) {
        const df rx = df_add(df_add(df_mul(R[0], dx), df_mul(R[1], dy)), df_mul(R[2], dz));
        const df ry = df_add(df_add(df_mul(R[3], dx), df_mul(R[4], dy)), df_mul(R[5], dz));
        const df rz = df_add(df_add(df_mul(R[6], dx), df_mul(R[7], dy)), df_mul(R[8], dz));
        dx = rx;
        dy = ry;
        dz = rz;
    }
    const df r2 = df_add(df_add(df_mul(dx, dx), df_mul(dy, dy)), df_mul(dz, dz));
    // y0 ~ r2^(-1/2) (a few ulps); y = y0 + y0 (1 - r2 y0^2) / 2 (Newton), with the
    // residual formed in double-float so that y carries ~44 bits
    const float y0 = rsqrtf(r2.h);
    const float q0 = __fmul_rn(y0, y0);
    const df y2 = {q0, __fmaf_rn(y0, y0, -q0)};
    const df t = df_mul(r2, y2);
    const df e = df_add({1.f, 0.f}, df_neg(t));
    rinv = fast_two_sum(y0, __fmul_rn(__fmul_rn(y0, 0.5f), e.h));
    ux = df_mul(dx, rinv);
    uy = df_mul(dy, rinv);
    uz = df_mul(dz, rinv);
}

// Primary image `code` (position minus the code's box shift, FP64 input used
// when given) as head + tail in shared memory: img[code] head, img[27 + code] tail.
// FP32 input: the position is exact and the shift s (box_h + box_l) is added in
// double-float; FP64 input: formed in FP64.
__device__ __forceinline__ void image_df(float4* img, int code, const float4& P0, const double* pts64, int p,
                                         double boxd, df box) {
    const int sx = code % 3 - 1, sy = (code / 3) % 3 - 1, sz = code / 9 - 1;
    if (!pts64) {
        auto shifted = [&](float v, int sh) {
            return sh == 0 ? df{v, 0.f} : df_add({v, 0.f}, {-(float)sh * box.h, -(float)sh * box.l});
        };
        const df x = shifted(P0.x, sx), y = shifted(P0.y, sy), z = shifted(P0.z, sz);
        img[code] = make_float4(x.h, y.h, z.h, 0.f);
        img[27 + code] = make_float4(x.l, y.l, z.l, 0.f);
        return;
    }
    double x = pts64[3 * (int64_t)p], y = pts64[3 * (int64_t)p + 1], z = pts64[3 * (int64_t)p + 2];
    x -= sx * boxd;
    y -= sy * boxd;
    z -= sz * boxd;
    const float hx = (float)x, hy = (float)y, hz = (float)z;
    img[code] = make_float4(hx, hy, hz, 0.f);
    img[27 + code] = make_float4((float)(x - hx), (float)(y - hy), (float)(z - hz), 0.f);
}

// A secondary's position as head + tail (exact for FP32 input).
__device__ __forceinline__ void load_sec(const ListArgs& a, unsigned e, float4& qv, float3& ql) {
    const unsigned j = e & kIdxMask;
    qv = __ldg(a.pts + j);
    ql = make_float3(0.f, 0.f, 0.f);
    if (a.pts64) {
        const double x = a.pts64[3 * (int64_t)j], y = a.pts64[3 * (int64_t)j + 1], z = a.pts64[3 * (int64_t)j + 2];
        qv.x = (float)x;
        qv.y = (float)y;
        qv.z = (float)z;
        ql = make_float3((float)(x - qv.x), (float)(y - qv.y), (float)(z - qv.z));
    }
}

// ---- forward ----------------------------------------------------------------
// The (lmax+1)^2 accumulator slots are handled in pairs, two slots per packed
// (f32x2) operation: the m = 0 slots k, k + 1 (k even), and for m >= 1 the Re
// and Im slots of one (m, k).  Per-pair record in shared memory (floats, every
// group of four 16-byte aligned so that one 128-bit load gives a slot pair's
// head pair and tail pair):
//   TA (m = 0), k even:  T_k.h, T_k+1.h, T_k.l, T_k+1.l      (LE = lmax+1 rounded up to even)
//   TB (m >= 1), k < L:  T_k.h, T_k.h,   T_k.l, T_k.l
//   W:                   w,     w,       0,     0
//   CB, m = 1..L:        Re.h,  Im.h,    Re.l,  Im.l         of w (x + iy)^m
// Row stride RS (floats) a multiple of 4.
template <int L>
struct DfRec {
    static constexpr int LE = (L + 2) & ~1;       // m = 0 slots, padded to even
    static constexpr int TA = 0;
    static constexpr int TB = 2 * LE;
    static constexpr int W = TB + 4 * L;
    static constexpr int CB = W + 4;
    static constexpr int N = CB + 4 * L;
    static constexpr int RS = N;                   // a multiple of 4
    static constexpr int NP = LE / 2 + L * (L + 1) / 2;  // slot pairs
    static constexpr int S2 = (NP + 31) / 32;            // slot pairs per lane
};

__host__ __device__ constexpr size_t accum_df_smem_per_warp(int L, int B, int NRP) {
    return (size_t)B * NRP * 8 + 54 * 16 + 9 * 8 + 8 + (size_t)32 * (2 * ((L + 2) & ~1) + 8 * L + 4) * 4;
}

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
// Two double-float accumulators at once (.x and .y): (H, Lo) += T * C, the
// operations of df_acc(acc, df_mul_u(T, C)) lane for lane.
__device__ __forceinline__ void df_acc_mul2(float2& H, float2& Lo, float4 T, float4 C) {
    const float2 Th = make_float2(T.x, T.y), Tl = make_float2(T.z, T.w);
    const float2 Ch = make_float2(C.x, C.y), Cl = make_float2(C.z, C.w);
    const float2 p = __fmul2_rn(Th, Ch);
    float2 e = __ffma2_rn(Th, Ch, neg2(p));
    e = __ffma2_rn(Th, Cl, __ffma2_rn(Tl, Ch, e));
    const float2 s = __fadd2_rn(H, p);
    const float2 bb = __fadd2_rn(s, neg2(H));
    const float2 err = __fadd2_rn(__fadd2_rn(H, neg2(__fadd2_rn(s, neg2(bb)))), __fadd2_rn(p, neg2(bb)));
    Lo = __fadd2_rn(Lo, __fadd2_rn(err, e));
    H = s;
}

template <int L>
__global__ void __launch_bounds__(kDThreads) k_accum_df(ListArgs a) {
    using R_ = DfRec<L>;
    constexpr int S2 = R_::S2, RS = R_::RS, NP = R_::NP;
    constexpr int U = S2 == 1 ? 8 : 4;  // pairs per round of the accumulation
    constexpr int NRP = Shape<L>::NRP;
    extern __shared__ __align__(16) unsigned char draw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int B = a.bins.nbins;
    unsigned char* base = draw + (size_t)wid * accum_df_smem_per_warp(L, B, NRP);
    float2* res = reinterpret_cast<float2*>(base);                          // [B][NRP] head, tail
    float4* img = reinterpret_cast<float4*>(base + (size_t)B * NRP * 8);    // [54]
    df* Rd = reinterpret_cast<df*>(base + (size_t)B * NRP * 8 + 54 * 16);   // [9]
    float* rec = reinterpret_cast<float*>(base + (size_t)B * NRP * 8 + 54 * 16 + 9 * 8 + 8);  // [32][RS]
    // this lane's slot pairs: record offsets of their T and C operands and their
    // two slots (slot1 < 0: none, e.g. the padding slot of m = 0)
    int offT[S2], offC[S2], slot0[S2], slot1[S2];
#pragma unroll
    for (int s = 0; s < S2; ++s) {
        const int sp = lane + 32 * s;
        offT[s] = 0;
        offC[s] = R_::W;
        slot0[s] = slot1[s] = -1;
        if (sp < R_::LE / 2) {
            offT[s] = R_::TA + 4 * sp;
            slot0[s] = 2 * sp;
            slot1[s] = 2 * sp + 1 <= L ? 2 * sp + 1 : -1;
        } else if (sp < NP) {
            int idx = sp - R_::LE / 2, m = 1;
            while (idx >= L + 1 - m) {
                idx -= L + 1 - m;
                ++m;
            }
            offT[s] = R_::TB + 4 * idx;
            offC[s] = R_::CB + 4 * (m - 1);
            slot0[s] = acc_base(L, m) + 2 * idx;
            slot1[s] = slot0[s] + 1;
        }
    }
    const Grid& g = a.g;
    const df boxdf = df_from(g.boxd);  // the box side as head + tail
    const bool radial = g.radial != 0;
    const int qa = a.qrange ? a.qrange[0] : a.qa, qb = a.qrange ? a.qrange[1] : a.qb;
    for (;;) {
        int q = 0;
        if (lane == 0) q = qa + atomicAdd(a.queue, 1);
        q = __shfl_sync(kFull, q, 0);
        if (q >= qb) break;
        const int p = a.plist ? a.plist[q] : q;
        const float4 P0 = a.pts[p];
        if (lane < 27) image_df(img, lane, P0, a.pts64, p, g.boxd, boxdf);
        if (lane < 9) {
            if (radial) {
                double x0 = P0.x, x1 = P0.y, x2 = P0.z;
                if (a.pts64) {
                    x0 = a.pts64[3 * (int64_t)p];
                    x1 = a.pts64[3 * (int64_t)p + 1];
                    x2 = a.pts64[3 * (int64_t)p + 2];
                }
                Rd[lane] = df_from(los_rotation_entry_d(lane, x0, x1, x2, g.boxd));
            } else {
                Rd[lane] = {(lane % 4 == 0) ? 1.f : 0.f, 0.f};
            }
        }
        for (int k = lane; k < B * NRP; k += 32) res[k] = make_float2(0.f, 0.f);
        const int cb = a.base[q] < 0 ? 0 : a.base[q];
        const int nch = a.nchunks[q];
        const int* chunks = a.chunks + (int64_t)cb * 32;
        const int* ordp = a.ord + cb;
        __syncwarp();
        float2 accH[S2], accL[S2];
#pragma unroll
        for (int s = 0; s < S2; ++s) accH[s] = accL[s] = make_float2(0.f, 0.f);
        auto flush = [&](int b) {
#pragma unroll
            for (int s = 0; s < S2; ++s) {
                if (slot0[s] >= 0) {
                    const float2 o = res[b * NRP + slot0[s]];
                    const df v = df_add({o.x, o.y}, {accH[s].x, accL[s].x});
                    res[b * NRP + slot0[s]] = make_float2(v.h, v.l);
                }
                if (slot1[s] >= 0) {
                    const float2 o = res[b * NRP + slot1[s]];
                    const df v = df_add({o.x, o.y}, {accH[s].y, accL[s].y});
                    res[b * NRP + slot1[s]] = make_float2(v.h, v.l);
                }
                accH[s] = accL[s] = make_float2(0.f, 0.f);
            }
        };
        if (nch > 0) {
            int curb = (int)((unsigned)__ldg(ordp) >> 26);
            // entries and points of chunk i + 1 load while chunk i is evaluated
            unsigned o_n = (unsigned)__ldg(ordp);
            unsigned e_n = (unsigned)__ldg(chunks + (int64_t)(o_n & 0x3ffffffu) * 32 + lane);
            float4 q_n = make_float4(0.f, 0.f, 0.f, 0.f);
            float3 l_n = make_float3(0.f, 0.f, 0.f);
            if (e_n != kNoPairD) load_sec(a, e_n, q_n, l_n);
            for (int i = 0; i < nch; ++i) {
                const unsigned o = o_n, e = e_n;
                const float4 qv = q_n;
                const float3 ql = l_n;
                if (i + 1 < nch) {
                    o_n = (unsigned)__ldg(ordp + i + 1);
                    e_n = (unsigned)__ldg(chunks + (int64_t)(o_n & 0x3ffffffu) * 32 + lane);
                    if (e_n != kNoPairD) load_sec(a, e_n, q_n, l_n);
                }
                const int b = (int)(o >> 26);
                if (b != curb) {
                    flush(curb);
                    curb = b;
                }
                // this lane's pair -> its record (only valid pairs are read back)
                float4* my = reinterpret_cast<float4*>(rec + lane * RS);
                if (e != kNoPairD) {
                    const int code = (int)(e >> kIdxBits);
                    const float4 hh = img[code], tt = img[27 + code];
                    const df dx = sep(qv.x, ql.x, hh.x, tt.x), dy = sep(qv.y, ql.y, hh.y, tt.y),
                             dz = sep(qv.z, ql.z, hh.z, tt.z);
                    df ux, uy, uz, rinv;
                    unit_df(dx, dy, dz, Rd, radial, ux, uy, uz, rinv);
                    const float w = qv.w;
                    df T[R_::LE];
                    T[0] = {1.f, 0.f};
                    if constexpr (L >= 1) T[1] = uz;
                    const df z2 = {2.f * uz.h, 2.f * uz.l};
#pragma unroll
                    for (int k = 2; k <= L; ++k) T[k] = df_add(df_mul(z2, T[k - 1]), df_neg(T[k - 2]));
#pragma unroll
                    for (int k = L + 1; k < R_::LE; ++k) T[k] = {0.f, 0.f};
#pragma unroll
                    for (int k = 0; k < R_::LE; k += 2)
                        my[(R_::TA >> 2) + (k >> 1)] = make_float4(T[k].h, T[k + 1].h, T[k].l, T[k + 1].l);
#pragma unroll
                    for (int k = 0; k < L; ++k) my[(R_::TB >> 2) + k] = make_float4(T[k].h, T[k].h, T[k].l, T[k].l);
                    my[R_::W >> 2] = make_float4(w, w, 0.f, 0.f);
                    if constexpr (L >= 1) {
                        df cr = df_mulf(ux, w), ci = df_mulf(uy, w);
#pragma unroll
                        for (int m = 1; m <= L; ++m) {
                            my[(R_::CB >> 2) + (m - 1)] = make_float4(cr.h, ci.h, cr.l, ci.l);
                            if (m < L) {
                                df nr, ni;
                                df_cmul(cr, ci, ux, uy, nr, ni);
                                cr = nr;
                                ci = ni;
                            }
                        }
                    }
                }
                __syncwarp();
                // every valid pair of the chunk into this lane's slot pairs, U
                // pairs per round (loads and products of later pairs overlap the
                // sums of earlier ones; the sums keep the pairs' order)
                unsigned valid = __ballot_sync(kFull, e != kNoPairD);
                while (valid) {
                    int t[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        t[u] = -1;
                        if (valid) {
                            t[u] = __ffs(valid) - 1;
                            valid &= valid - 1;
                        }
                    }
#pragma unroll
                    for (int s = 0; s < S2; ++s) {
                        if (lane + 32 * s < NP) {
                            float4 T4[U], C4[U];
#pragma unroll
                            for (int u = 0; u < U; ++u) {
                                if (t[u] >= 0) {
                                    const float* rt = rec + t[u] * RS;
                                    T4[u] = *reinterpret_cast<const float4*>(rt + offT[s]);
                                    C4[u] = *reinterpret_cast<const float4*>(rt + offC[s]);
                                }
                            }
#pragma unroll
                            for (int u = 0; u < U; ++u)
                                if (t[u] >= 0) df_acc_mul2(accH[s], accL[s], T4[u], C4[u]);
                        }
                    }
                }
                __syncwarp();
            }
            flush(curb);
        }
        __syncwarp();
        const int row = a.chunked ? q - a.q0 : a.orig[p];
        float* Arow = a.A + (int64_t)row * a.RLP;
        for (int col = lane; col < a.RL; col += 32) {
            const int4 cv = __ldg(a.colconv + col);
            const float2* cf = a.colcoefdf + cv.w;
            df v = {0.f, 0.f};
            for (int k = 0; k < cv.z; ++k) {
                const float2 c = __ldg(cf + k), r = res[cv.x + cv.y * k];
                v = df_add(v, df_mul({c.x, c.y}, {r.x, r.y}));
            }
            Arow[col] = __fadd_rn(v.h, v.l);
        }
        if (lane == 0) a.wrow[row] = P0.w;
        __syncwarp();
    }
}

// ---- adjoint ----------------------------------------------------------------
__host__ __device__ constexpr size_t adj_df_smem_per_warp(int B, int NRP) {
    return (size_t)B * NRP * 8 + 54 * 16;
}
// a double-float value (head, tail) as the duplicated operand (h, h, t, t) of a
// packed product
__device__ __forceinline__ float4 dup2(float2 v) { return make_float4(v.x, v.x, v.y, v.y); }

template <int L>
__global__ void __launch_bounds__(kDThreads) k_adj_df(ListArgs a) {
    constexpr int NR = Shape<L>::NR, NRP = Shape<L>::NRP;
    extern __shared__ __align__(16) unsigned char draw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int B = a.bins.nbins;
    unsigned char* base = draw + (size_t)wid * adj_df_smem_per_warp(B, NRP);
    float2* G = reinterpret_cast<float2*>(base);                           // [B][NRP] head, tail
    float4* img = reinterpret_cast<float4*>(base + (size_t)B * NRP * 8);   // [54]
    const Grid& g = a.g;
    const df boxdf = df_from(g.boxd);  // the box side as head + tail
    const int qa = a.qrange ? a.qrange[0] : a.qa, qb = a.qrange ? a.qrange[1] : a.qb;
    for (;;) {
        int q = 0;
        if (lane == 0) q = qa + atomicAdd(a.queue, 1);
        q = __shfl_sync(kFull, q, 0);
        if (q >= qb) break;
        const int p = a.plist ? a.plist[q] : q;
        const float4 P0 = a.pts[p];
        if (lane < 27) image_df(img, lane, P0, a.pts64, p, g.boxd, boxdf);
        const int row = a.orig[p];
        const float2* Vrow = a.Vdf + (int64_t)(a.chunked ? q - a.q0 : row) * a.RLP;
        for (int idx = lane; idx < B * NR; idx += 32) {
            const int b = idx / NR, sl = idx - b * NR;
            const int4 cv = __ldg(a.slotconv + sl);
            df v = {0.f, 0.f};
            for (int t = 0; t < cv.z; ++t) {
                const float2 c = __ldg(a.slotcoefdf + cv.w + t), x = Vrow[cv.x + b + t * cv.y];
                v = df_add(v, df_mul({c.x, c.y}, {x.x, x.y}));
            }
            const df gv = df_mulf(v, P0.w);
            G[b * NRP + sl] = make_float2(gv.h, gv.l);
        }
        const int cb = a.base[q] < 0 ? 0 : a.base[q];
        const int nch = a.nchunks[q];
        const int* chunks = a.chunks + (int64_t)cb * 32;
        const int* ordp = a.ord + cb;
        __syncwarp();
        df pix = {0.f, 0.f}, piy = {0.f, 0.f}, piz = {0.f, 0.f};  // the primary's share (this lane)
        unsigned o_n = nch > 0 ? (unsigned)__ldg(ordp) : 0u;
        unsigned e_n = nch > 0 ? (unsigned)__ldg(chunks + (int64_t)(o_n & 0x3ffffffu) * 32 + lane) : kNoPairD;
        float4 q_n = make_float4(0.f, 0.f, 0.f, 0.f);
        float3 l_n = make_float3(0.f, 0.f, 0.f);
        if (e_n != kNoPairD) load_sec(a, e_n, q_n, l_n);
        for (int i = 0; i < nch; ++i) {
            const unsigned o = o_n, e = e_n;
            const float4 qv = q_n;
            const float3 ql = l_n;
            if (i + 1 < nch) {
                o_n = (unsigned)__ldg(ordp + i + 1);
                e_n = (unsigned)__ldg(chunks + (int64_t)(o_n & 0x3ffffffu) * 32 + lane);
                if (e_n != kNoPairD) load_sec(a, e_n, q_n, l_n);
            }
            if (e == kNoPairD) continue;
            const int b = (int)(o >> 26);
            const float2* Gb = G + b * NRP;
            const int code = (int)(e >> kIdxBits);
            const float4 hh = img[code], tt = img[27 + code];
            const df dx = sep(qv.x, ql.x, hh.x, tt.x), dy = sep(qv.y, ql.y, hh.y, tt.y), dz = sep(qv.z, ql.z, hh.z, tt.z);
            df ux, uy, z, rinv;
            unit_df(dx, dy, dz, nullptr, false, ux, uy, z, rinv);
            // T_k(z) and T_k'(z) = k U_{k-1}(z)
            df T[L + 1], D[L + 1];
            T[0] = {1.f, 0.f};
            D[0] = {0.f, 0.f};
            if constexpr (L >= 1) {
                T[1] = z;
                D[1] = {1.f, 0.f};
                const df z2 = {2.f * z.h, 2.f * z.l};
                df u0 = {1.f, 0.f}, u1 = z2;  // U_0, U_1
                static_for<2, L + 1>([&](auto kc) {
                    constexpr int k = decltype(kc)::value;
                    T[k] = df_add(df_mul(z2, T[k - 1]), df_neg(T[k - 2]));
                    D[k] = df_mulf(u1, (float)k);
                    const df u2 = df_add(df_mul(z2, u1), df_neg(u0));
                    u0 = u1;
                    u1 = u2;
                });
            }
            // (T_k, T_k') side by side: the second operand of the packed products
            float4 TD[L + 1];
            static_for<0, L + 1>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                TD[k] = make_float4(T[k].h, D[k].h, T[k].l, D[k].l);
            });
            // (F, Fz) in one packed double-float accumulator (.x = F, .y = Fz), and per
            // m the pairs (gmr, gzr) and (gmi, gzi): every component takes the
            // operations and order of its own scalar sum
            float2 FH = make_float2(0.f, 0.f), FL = make_float2(0.f, 0.f);
            df Fx = {0.f, 0.f}, Fy = {0.f, 0.f};
            static_for<0, L + 1>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                df_acc_mul2(FH, FL, dup2(Gb[k]), TD[k]);
            });
            df pr = {1.f, 0.f}, pim = {0.f, 0.f};  // (x + iy)^(m-1)
            static_for<1, L + 1>([&](auto mc) {
                constexpr int m = decltype(mc)::value;
                constexpr int b0 = acc_base(L, m);
                float2 RH = make_float2(0.f, 0.f), RL = make_float2(0.f, 0.f);  // (gmr, gzr)
                float2 IH = make_float2(0.f, 0.f), IL = make_float2(0.f, 0.f);  // (gmi, gzi)
                static_for<0, L - m + 1>([&](auto kc) {
                    constexpr int k = decltype(kc)::value;
                    df_acc_mul2(RH, RL, dup2(Gb[b0 + 2 * k]), TD[k]);
                    df_acc_mul2(IH, IL, dup2(Gb[b0 + 2 * k + 1]), TD[k]);
                });
                df ur, ui;  // (x + iy)^m
                if constexpr (m == 1) {
                    ur = ux;
                    ui = uy;
                } else {
                    df_cmul(pr, pim, ux, uy, ur, ui);
                }
                // F += Re(conj(gm) u^m), Fz likewise with gz, and the derivatives of
                // u^m: d/dx = m u^(m-1), d/dy = i m u^(m-1)
                df_acc_mul2(FH, FL, make_float4(RH.x, RH.y, RL.x, RL.y), make_float4(ur.h, ur.h, ur.l, ur.l));
                df_acc_mul2(FH, FL, make_float4(IH.x, IH.y, IL.x, IL.y), make_float4(ui.h, ui.h, ui.l, ui.l));
                const df gmr = {RH.x, RL.x}, gmi = {IH.x, IL.x};
                const df ax = df_add(df_mul_u(gmr, pr), df_mul_u(gmi, pim));
                const df ay = df_add(df_mul_u(gmi, pr), df_neg(df_mul_u(gmr, pim)));
                df_acc(Fx, df_mulf(ax, (float)m));
                df_acc(Fy, df_mulf(ay, (float)m));
                pr = ur;
                pim = ui;
            });
            const df F = {FH.x, FL.x}, Fz = {FH.y, FL.y};
            // tangential gradient: (2 w_j / r) (grad F - (grad F . u) u), formed in
            // double-float and rounded once: a per-pair relative error of an FP32
            // ulp is not amplified by the sums over pairs
            const df gdr = df_add(df_add(df_mul(Fx, ux), df_mul(Fy, uy)), df_mul(Fz, z));
            const float tx = df_add(Fx, df_neg(df_mul(gdr, ux))).h;
            const float ty = df_add(Fy, df_neg(df_mul(gdr, uy))).h;
            const float tz = df_add(Fz, df_neg(df_mul(gdr, z))).h;
            const float sc = __fmul_rn(2.f * qv.w, __fadd_rn(rinv.h, rinv.l));
            const float gx = __fmul_rn(sc, tx), gy = __fmul_rn(sc, ty), gz3 = __fmul_rn(sc, tz);
            const int jj = __ldg(a.orig + (e & kIdxMask));
            atomicAdd(a.dw + jj, f2d_exact(__fmul_rn(2.f, __fadd_rn(F.h, F.l))));
            atomicAdd(a.dpos + 3 * (int64_t)jj, f2d_exact(gx));
            atomicAdd(a.dpos + 3 * (int64_t)jj + 1, f2d_exact(gy));
            atomicAdd(a.dpos + 3 * (int64_t)jj + 2, f2d_exact(gz3));
            df_acc(pix, {gx, 0.f});
            df_acc(piy, {gy, 0.f});
            df_acc(piz, {gz3, 0.f});
        }
        double di0 = -df_to(pix), di1 = -df_to(piy), di2 = -df_to(piz);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            di0 += __shfl_xor_sync(kFull, di0, o);
            di1 += __shfl_xor_sync(kFull, di1, o);
            di2 += __shfl_xor_sync(kFull, di2, o);
        }
        if (lane == 0) {
            atomicAdd(a.dpos + 3 * (int64_t)row, di0);
            atomicAdd(a.dpos + 3 * (int64_t)row + 1, di1);
            atomicAdd(a.dpos + 3 * (int64_t)row + 2, di2);
        }
        __syncwarp();
    }
}

template <class K>
int launch_persistent(K kern, const ListArgs& a, size_t smem, int nsm, cudaStream_t st) {
    if (smem > 227 * 1024) return -1;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kDThreads, smem) != cudaSuccess || per_sm < 1)
        return -1;
    int blocks = per_sm * nsm;
    const int need = (a.qb - a.qa + kDWarps - 1) / kDWarps;
    if (!a.qrange && blocks > need) blocks = need > 0 ? need : 1;
    kern<<<blocks, kDThreads, smem, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int L>
int launch_accum_df_t(const ListArgs& a, int nsm, cudaStream_t st) {
    return launch_persistent(k_accum_df<L>, a, accum_df_smem_per_warp(L, a.bins.nbins, Shape<L>::NRP) * kDWarps,
                             nsm, st);
}
template <int L>
int launch_adj_df_t(const ListArgs& a, int nsm, cudaStream_t st) {
    return launch_persistent(k_adj_df<L>, a, adj_df_smem_per_warp(a.bins.nbins, Shape<L>::NRP) * kDWarps, nsm, st);
}

}  // namespace

int launch_accum_df(int lmax, const ListArgs& a, int nsm, cudaStream_t st) {
    if (!a.qrange && a.qb <= a.qa) return 0;
    switch (lmax) {
        case 0: return launch_accum_df_t<0>(a, nsm, st);
        case 1: return launch_accum_df_t<1>(a, nsm, st);
        case 2: return launch_accum_df_t<2>(a, nsm, st);
        case 3: return launch_accum_df_t<3>(a, nsm, st);
        case 4: return launch_accum_df_t<4>(a, nsm, st);
        case 5: return launch_accum_df_t<5>(a, nsm, st);
        case 6: return launch_accum_df_t<6>(a, nsm, st);
        case 7: return launch_accum_df_t<7>(a, nsm, st);
        case 8: return launch_accum_df_t<8>(a, nsm, st);
        case 9: return launch_accum_df_t<9>(a, nsm, st);
        case 10: return launch_accum_df_t<10>(a, nsm, st);
        default: return -1;
    }
}

int launch_adj_df(int lmax, const ListArgs& a, int nsm, cudaStream_t st) {
    if (!a.qrange && a.qb <= a.qa) return 0;
    switch (lmax) {
        case 0: return launch_adj_df_t<0>(a, nsm, st);
        case 1: return launch_adj_df_t<1>(a, nsm, st);
        case 2: return launch_adj_df_t<2>(a, nsm, st);
        case 3: return launch_adj_df_t<3>(a, nsm, st);
        case 4: return launch_adj_df_t<4>(a, nsm, st);
        case 5: return launch_adj_df_t<5>(a, nsm, st);
        case 6: return launch_adj_df_t<6>(a, nsm, st);
        case 7: return launch_adj_df_t<7>(a, nsm, st);
        case 8: return launch_adj_df_t<8>(a, nsm, st);
        case 9: return launch_adj_df_t<9>(a, nsm, st);
        case 10: return launch_adj_df_t<10>(a, nsm, st);
        default: return -1;
    }
}

}  // namespace g3
