// Multipoles through the paper's monomial basis (Sec. 3.3.2): per primary and
// radial bin the power sums M_abc(b) = sum_j w_j xhat^a yhat^b zhat^c over
// a + b + c <= lmax ((lmax+1)(lmax+2)(lmax+3)/6 of them, 286 at lmax = 10), then
// a_lm(b) = K_lm sum_{k,j} d^(lm)_k C(m, j) i^j M_{m-j, j, k}(b), where D_lm(z) =
// sum_k d_k z^k is the monic associated-Legendre factor of Y_lm = K_lm D_lm(z)
// (x + iy)^m.  A cross-check of the Chebyshev form (G3PCF_OPT_BASIS = 1): it
// walks the same pair lists, in FP64 throughout, because FP32 power sums would
// lose about three digits to the cancellation in the conversion at l = 10.
//
// Mapping: one warp per primary.  Each lane evaluates the unit vector and the
// powers of one pair of a 32-entry chunk into shared memory; then every lane
// adds the chunk's 32 terms to the monomials it owns (lane + 32 s), so no
// cross-lane reduction is needed.  At the end of a bin the sums go to shared
// memory and the lanes form that bin's columns of the multipole row.
#include "pair_common.cuh"

namespace g3 {
namespace {

constexpr int kMWarps = 4;
constexpr int kMThreads = kMWarps * 32;
constexpr unsigned kFullM = 0xffffffffu;
constexpr unsigned kNoPairM = 0xffffffffu;
constexpr int kIdxBitsM = kIdxBits;
constexpr unsigned kIdxMaskM = kIdxMask;

__host__ __device__ constexpr int n_mono(int L) { return (L + 1) * (L + 2) * (L + 3) / 6; }

// per-warp shared memory: powers [32][3][L+1] double, weights [32] double,
// sums [NM] double, images [27] double3 (padded to 4), LOS rotation [12]
// double, row res [RL] float
__host__ __device__ constexpr size_t mono_smem_per_warp(int L, int RL) {
    return (size_t)32 * 3 * (L + 1) * 8 + 32 * 8 + (size_t)n_mono(L) * 8 + 27 * 32 + 12 * 8 + (size_t)RL * 4;
}

template <int L>
__global__ void __launch_bounds__(kMThreads) k_mono(ListArgs a) {
    constexpr int NM = n_mono(L);
    constexpr int S = (NM + 31) / 32;  // monomials per lane
    extern __shared__ __align__(16) unsigned char mraw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int B = a.bins.nbins;
    unsigned char* base = mraw + (size_t)wid * mono_smem_per_warp(L, a.RL);
    double* pw = reinterpret_cast<double*>(base);                       // [32][3][L+1]
    double* ww = pw + 32 * 3 * (L + 1);                                 // [32]
    double* msum = ww + 32;                                             // [NM]
    double* im = msum + NM;                                             // [27][4]
    double* Rm = im + 27 * 4;                                           // [12]
    float* res = reinterpret_cast<float*>(Rm + 12);                     // [RL]
    // exponents of this lane's monomials (a | b << 8 | c << 16; -1: none)
    int ex[S];
#pragma unroll
    for (int s = 0; s < S; ++s) ex[s] = lane + 32 * s < NM ? a.monoexp[lane + 32 * s] : -1;
    const Grid& g = a.g;
    const int qa = a.qrange ? a.qrange[0] : a.qa, qb = a.qrange ? a.qrange[1] : a.qb;
    for (;;) {
        int q = 0;
        if (lane == 0) q = qa + atomicAdd(a.queue, 1);
        q = __shfl_sync(kFullM, q, 0);
        if (q >= qb) break;
        const int p = a.plist ? a.plist[q] : q;
        const float4 P0 = a.pts[p];
        if (lane < 27) {  // the primary's images in FP64
            double x = P0.x, y = P0.y, z = P0.z;
            if (a.pts64) {
                x = a.pts64[3 * (int64_t)p];
                y = a.pts64[3 * (int64_t)p + 1];
                z = a.pts64[3 * (int64_t)p + 2];
            }
            const int sx = lane % 3 - 1, sy = (lane / 3) % 3 - 1, sz = lane / 9 - 1;
            im[4 * lane] = x - sx * g.boxd;
            im[4 * lane + 1] = y - sy * g.boxd;
            im[4 * lane + 2] = z - sz * g.boxd;
            if (lane < 9) Rm[lane] = g.radial ? los_rotation_entry_d(lane, x, y, z, g.boxd) : ((lane % 4 == 0) ? 1.0 : 0.0);
        }
        for (int k = lane; k < a.RL; k += 32) res[k] = 0.f;
        __syncwarp();
        const int cb = a.base[q] < 0 ? 0 : a.base[q];
        const int nch = a.nchunks[q];
        const int* chunks = a.chunks + (int64_t)cb * 32;
        const int* ordp = a.ord + cb;
        double acc[S];
#pragma unroll
        for (int s = 0; s < S; ++s) acc[s] = 0.0;
        auto finish_bin = [&](int b) {  // power sums -> this bin's multipole columns
#pragma unroll
            for (int s = 0; s < S; ++s)
                if (lane + 32 * s < NM) msum[lane + 32 * s] = acc[s];
            __syncwarp();
            for (int u = lane; u < (L + 1) * (L + 1); u += 32) {
                const int4 cv = __ldg(a.monoconv + u);
                double v = 0.0;
                for (int t = 0; t < cv.y; ++t) v += __ldg(a.monocoef + cv.x + t) * msum[__ldg(a.monoidx + cv.x + t)];
                res[cv.z + b] = (float)v;
            }
            __syncwarp();
#pragma unroll
            for (int s = 0; s < S; ++s) acc[s] = 0.0;
        };
        int curb = nch > 0 ? (int)((unsigned)__ldg(ordp) >> 26) : 0;
        for (int i = 0; i < nch; ++i) {
            const unsigned o = (unsigned)__ldg(ordp + i);
            const int b = (int)(o >> 26);
            if (b != curb) {
                finish_bin(curb);
                curb = b;
            }
            const unsigned e = (unsigned)__ldg(chunks + (int64_t)(o & 0x3ffffffu) * 32 + lane);
            double w = 0.0, ux = 0.0, uy = 0.0, uz = 1.0;
            if (e != kNoPairM) {
                const float4 qv = __ldg(a.pts + (e & kIdxMaskM));
                const double* oi = im + 4 * (e >> kIdxBitsM);
                double qx = qv.x, qy = qv.y, qz = qv.z;
                if (a.pts64) {
                    const int64_t j = (int64_t)(e & kIdxMaskM);
                    qx = a.pts64[3 * j];
                    qy = a.pts64[3 * j + 1];
                    qz = a.pts64[3 * j + 2];
                }
                double dx = qx - oi[0], dy = qy - oi[1], dz = qz - oi[2];
                if (g.radial) {  // into the primary's line-of-sight frame
                    const double rx = Rm[0] * dx + Rm[1] * dy + Rm[2] * dz;
                    const double ry = Rm[3] * dx + Rm[4] * dy + Rm[5] * dz;
                    const double rz = Rm[6] * dx + Rm[7] * dy + Rm[8] * dz;
                    dx = rx;
                    dy = ry;
                    dz = rz;
                }
                const double r = sqrt(dx * dx + dy * dy + dz * dz);
                ux = dx / r;
                uy = dy / r;
                uz = dz / r;
                w = qv.w;
            }
            double* my = pw + lane * 3 * (L + 1);
            double px = 1.0, py = 1.0, pz = 1.0;
#pragma unroll
            for (int k = 0; k <= L; ++k) {
                my[k] = px;
                my[L + 1 + k] = py;
                my[2 * (L + 1) + k] = pz;
                px *= ux;
                py *= uy;
                pz *= uz;
            }
            ww[lane] = w;
            __syncwarp();
            for (int t = 0; t < 32; ++t) {
                const double wt = ww[t];
                const double* pt = pw + t * 3 * (L + 1);
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    const int x = ex[s];
                    if (x >= 0) {
                        const double term = pt[x & 0xff] * pt[L + 1 + ((x >> 8) & 0xff)] * pt[2 * (L + 1) + (x >> 16)];
                        acc[s] = fma(wt, term, acc[s]);
                    }
                }
            }
            __syncwarp();
        }
        if (nch > 0) finish_bin(curb);
        const int row = a.chunked ? q - a.q0 : a.orig[p];
        float* Arow = a.A + (int64_t)row * a.RLP;
        for (int col = lane; col < a.RL; col += 32) Arow[col] = res[col];
        if (lane == 0) a.wrow[row] = P0.w;
        __syncwarp();
    }
}

template <int L>
int launch_mono_t(const ListArgs& a, int nsm, cudaStream_t st) {
    const size_t smem = mono_smem_per_warp(L, a.RL) * kMWarps;
    if (cudaFuncSetAttribute(k_mono<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mono<L>, kMThreads, smem) != cudaSuccess ||
        per_sm < 1)
        return -1;
    int blocks = per_sm * nsm;
    const int need = (a.qb - a.qa + kMWarps - 1) / kMWarps;
    if (!a.qrange && blocks > need) blocks = need > 0 ? need : 1;
    k_mono<L><<<blocks, kMThreads, smem, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

int mono_count(int lmax) { return n_mono(lmax); }

int launch_mono(int lmax, const ListArgs& a, int nsm, cudaStream_t st) {
    if (!a.qrange && a.qb <= a.qa) return 0;
    switch (lmax) {
        case 0: return launch_mono_t<0>(a, nsm, st);
        case 1: return launch_mono_t<1>(a, nsm, st);
        case 2: return launch_mono_t<2>(a, nsm, st);
        case 3: return launch_mono_t<3>(a, nsm, st);
        case 4: return launch_mono_t<4>(a, nsm, st);
        case 5: return launch_mono_t<5>(a, nsm, st);
        case 6: return launch_mono_t<6>(a, nsm, st);
        case 7: return launch_mono_t<7>(a, nsm, st);
        case 8: return launch_mono_t<8>(a, nsm, st);
        case 9: return launch_mono_t<9>(a, nsm, st);
        case 10: return launch_mono_t<10>(a, nsm, st);
        default: return -1;
    }
}

}  // namespace g3
