// Adjoint of zeta with respect to the weights and positions (not in the
// paper; the derivative of its Sec. 3.1 estimator with the pair set and
// radial bins held fixed).
//
// With G_m = dL/dzeta_m / 2 (the caller passes dL/d(Re zeta, Im zeta)),
// M_m = G_m + G_m^H and A_i the primary's multipoles,
//      V_i = M_m A_i                    (k_vgemm, per m block, FP32; k_vgemm_df
//                                        in double-float for the double-float
//                                        pair pass)
//      dL/dw_i (as a primary) = Re(A_i^H V_i)   (fused into k_vgemm)
//      H_i = w_i V_i                    (applied by the adjoint pair pass)
// (per catalog c of a batched forward, M is built from that catalog's dL/dzeta_c)
// and the pair pass (k_adj over the pair lists, or the fused k_pair mode 1)
// adds, for every pair (i, j) in bin b,
// 2 Re(conj(H_i,b) . Y(rhat_ij)) to dL/dw_j and the gradient of the same
// quantity with respect to the separation to dL/dpos_j and -dL/dpos_i.
// In the real form of an A row ([Re | Im] halves for m >= 1) M acts as
// [[Re M, -Im M], [Im M, Re M]]; for m = 0 only Re M enters because a_l0
// and Y_l0 are real.
#include "internal.h"

namespace g3 {

namespace {

constexpr int kRows = 8;         // primaries per CTA in k_vgemm
constexpr int kVThreads = 256;

struct MInfo {
    int K[kMaxL + 1];
    int W[kMaxL + 1];
    int col0[kMaxL + 1];   // first A column of block m
    int moff[kMaxL + 1];   // offset of block m in the M buffer (floats)
    long long zoff[kMaxL + 1];  // complex offset of block m in zeta
};

// M entries as stored: FP32, or head + tail FP32 pairs for the double-float path
template <class TM>
__device__ __forceinline__ TM m_entry(double v);
template <>
__device__ __forceinline__ float m_entry<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ float2 m_entry<float2>(double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

template <class TM>
__global__ void k_build_mreal(const double* dz, MInfo mi, int lmax, int64_t zsize, size_t mfloats,
                              TM* Mr) {
    const int m = blockIdx.y, cat = blockIdx.z;
    if (m > lmax) return;
    const int K = mi.K[m], W = mi.W[m];
    const double* Z = dz + 2 * ((int64_t)cat * zsize + mi.zoff[m]);
    TM* out = Mr + (size_t)cat * mfloats + mi.moff[m];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < W * W; e += gridDim.x * blockDim.x) {
        const int rr = e / W, cc = e % W;
        const int r = rr % K, c = cc % K;
        // M = G + G^H, G = dz / 2
        const double re = 0.5 * (Z[2 * ((int64_t)r * K + c)] + Z[2 * ((int64_t)c * K + r)]);
        const double im = 0.5 * (Z[2 * ((int64_t)r * K + c) + 1] - Z[2 * ((int64_t)c * K + r) + 1]);
        double v;
        if (m == 0) {
            v = re;
        } else {
            const bool rlo = rr < K, clo = cc < K;
            v = (rlo == clo) ? re : (rlo ? -im : im);
        }
        out[e] = m_entry<TM>(v);
    }
}

// One CTA per block of up to kRows rows of one catalog: blk = {catalog, first
// row, rows}; the catalog picks its M.  Without a block table (blks null) block
// b covers rows row_lo + kRows b .. of catalog 0 below row_hi.  The row's
// primary-weight term is added to dw[row], or, for rows of a chunk of
// primaries (rorig non-null), to dw[rorig[rplist ? rplist[q0 + row] : q0 + row]].
// FP32 M, V and sums.
template <class TM>
__global__ void __launch_bounds__(kVThreads) k_vgemm(const float* __restrict__ A, int RLP, int RL,
                                                     const int4* __restrict__ blks, int64_t row_lo,
                                                     int64_t row_hi, const TM* __restrict__ Mall,
                                                     size_t mfloats, MInfo mi, int lmax, TM* V,
                                                     double* dw, const int* rplist, const int* rorig,
                                                     int64_t q0) {
    extern __shared__ float sA[];  // kRows x RL
    __shared__ TM red[kRows][kVThreads / 32];
    int4 blk;
    if (blks) {
        blk = blks[blockIdx.x];
    } else {
        const int64_t b0 = row_lo + (int64_t)blockIdx.x * kRows;
        blk = make_int4(0, (int)b0, (int)(row_hi - b0 < kRows ? row_hi - b0 : kRows), 0);
    }
    const TM* __restrict__ Mr = Mall + (size_t)blk.x * mfloats;
    const int64_t r0 = blk.y;
    const int64_t rows = r0 + blk.z;
    for (int k = threadIdx.x; k < kRows * RL; k += kVThreads) {
        const int rr = k / RL, c = k % RL;
        sA[k] = (r0 + rr < rows) ? A[(r0 + rr) * RLP + c] : 0.f;
    }
    __syncthreads();
    TM dwp[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) dwp[r] = (TM)0;
    for (int col = threadIdx.x; col < RL; col += kVThreads) {
        int m = 0;
        while (m < lmax && col >= mi.col0[m + 1]) ++m;
        const int W = mi.W[m], c = col - mi.col0[m];
        const TM* Mrow = Mr + mi.moff[m] + (int64_t)c * W;
        const float* As = sA + mi.col0[m];
        TM acc[kRows];
#pragma unroll
        for (int r = 0; r < kRows; ++r) acc[r] = (TM)0;
        for (int k = 0; k < W; ++k) {
            const TM mv = __ldg(Mrow + k);
#pragma unroll
            for (int r = 0; r < kRows; ++r) acc[r] = fma(mv, (TM)As[r * RL + k], acc[r]);
        }
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            if (r0 + r < rows) V[(r0 + r) * RLP + col] = acc[r];
            dwp[r] = fma((TM)sA[r * RL + col], acc[r], dwp[r]);
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        TM v = dwp[r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[r][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < kRows && r0 + threadIdx.x < rows) {
        double s = 0.0;
        for (int k = 0; k < kVThreads / 32; ++k) s += (double)red[threadIdx.x][k];
        const int64_t row = r0 + threadIdx.x;
        int64_t idx = row;
        if (rorig) {
            const int64_t q = q0 + row;
            idx = rorig[rplist ? rplist[q] : q];
        }
        dw[idx] += s;  // the primary-weight term (dw starts at zero; pair terms add atomically)
    }
}

// The same product in double-float: M as head + tail pairs, the FP32 A entries
// exact, each product M_h a formed exactly (a multiply and an FMA), the running
// sum's head updated by an error-free two-sum and every rounding error, the
// product's low part and M_l a gathered in the tail; V stored renormalised as
// head + tail.  ~10 FP32 operations per multiply-add instead of one FP64 FMA,
// which runs at 1/58 of the FP32 rate on this part.  The primary-weight term
// Re(A^H V) sums in FP64 (one term per column).
__global__ void __launch_bounds__(kVThreads) k_vgemm_df(const float* __restrict__ A, int RLP, int RL,
                                                        const int4* __restrict__ blks, int64_t row_lo,
                                                        int64_t row_hi, const float2* __restrict__ Mall,
                                                        size_t mfloats, MInfo mi, int lmax, float2* V,
                                                        double* dw, const int* rplist, const int* rorig,
                                                        int64_t q0) {
    extern __shared__ float sA[];  // kRows x RL
    __shared__ double red[kRows][kVThreads / 32];
    int4 blk;
    if (blks) {
        blk = blks[blockIdx.x];
    } else {
        const int64_t b0 = row_lo + (int64_t)blockIdx.x * kRows;
        blk = make_int4(0, (int)b0, (int)(row_hi - b0 < kRows ? row_hi - b0 : kRows), 0);
    }
    const float2* __restrict__ Mr = Mall + (size_t)blk.x * mfloats;
    const int64_t r0 = blk.y;
    const int64_t rows = r0 + blk.z;
    for (int k = threadIdx.x; k < kRows * RL; k += kVThreads) {
        const int rr = k / RL, c = k % RL;
        sA[k] = (r0 + rr < rows) ? A[(r0 + rr) * RLP + c] : 0.f;
    }
    __syncthreads();
    double dwp[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) dwp[r] = 0.0;
    for (int col = threadIdx.x; col < RL; col += kVThreads) {
        int m = 0;
        while (m < lmax && col >= mi.col0[m + 1]) ++m;
        const int W = mi.W[m], c = col - mi.col0[m];
        const float2* Mrow = Mr + mi.moff[m] + (int64_t)c * W;
        const float* As = sA + mi.col0[m];
        float sh[kRows], sl[kRows];
#pragma unroll
        for (int r = 0; r < kRows; ++r) sh[r] = sl[r] = 0.f;
        for (int k = 0; k < W; ++k) {
            const float2 mv = __ldg(Mrow + k);
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                const float x = As[r * RL + k];
                const float p = __fmul_rn(mv.x, x);
                const float pe = __fmaf_rn(mv.x, x, -p);
                const float s = __fadd_rn(sh[r], p);
                const float bb = __fsub_rn(s, sh[r]);
                const float err = __fadd_rn(__fsub_rn(sh[r], __fsub_rn(s, bb)), __fsub_rn(p, bb));
                sh[r] = s;
                sl[r] = __fmaf_rn(mv.y, x, __fadd_rn(sl[r], __fadd_rn(err, pe)));
            }
        }
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const float h = __fadd_rn(sh[r], sl[r]);
            const float l = __fsub_rn(sl[r], __fsub_rn(h, sh[r]));
            if (r0 + r < rows) V[(r0 + r) * RLP + col] = make_float2(h, l);
            dwp[r] = fma((double)sA[r * RL + col], (double)h + (double)l, dwp[r]);
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        double v = dwp[r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[r][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < kRows && r0 + threadIdx.x < rows) {
        double s = 0.0;
        for (int k = 0; k < kVThreads / 32; ++k) s += red[threadIdx.x][k];
        const int64_t row = r0 + threadIdx.x;
        int64_t idx = row;
        if (rorig) {
            const int64_t q = q0 + row;
            idx = rorig[rplist ? rplist[q] : q];
        }
        dw[idx] += s;
    }
}

template <class TM>
struct VgemmKernel;
template <>
struct VgemmKernel<float> {
    static constexpr auto fn = k_vgemm<float>;
};
template <>
struct VgemmKernel<float2> {
    static constexpr auto fn = k_vgemm_df;
};

MInfo make_info(int nbins, int lmax) {
    MInfo mi{};
    int col = 0, moff = 0;
    long long z = 0;
    for (int m = 0; m <= lmax; ++m) {
        const int K = nbins * (lmax + 1 - m);
        const int W = m == 0 ? K : 2 * K;
        mi.K[m] = K;
        mi.W[m] = W;
        mi.col0[m] = col;
        mi.moff[m] = moff;
        mi.zoff[m] = z;
        col += W;
        moff += W * W;
        z += (long long)K * K;
    }
    return mi;
}

}  // namespace

size_t adjoint_m_floats(int nbins, int lmax) {
    size_t s = 0;
    for (int m = 0; m <= lmax; ++m) {
        const size_t K = (size_t)nbins * (lmax + 1 - m);
        const size_t W = m == 0 ? K : 2 * K;
        s += W * W;
    }
    return s;
}

int adjoint_rows_per_block() { return kRows; }

template <class TM>
int adjoint_m_t(const double* dzeta, int nbins, int lmax, int ncat, int64_t zsize, TM* Mr, cudaStream_t st) {
    const MInfo mi = make_info(nbins, lmax);
    dim3 g1(64, lmax + 1, ncat);
    k_build_mreal<TM><<<g1, 256, 0, st>>>(dzeta, mi, lmax, zsize, adjoint_m_floats(nbins, lmax), Mr);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <class TM>
int adjoint_prep_t(const double* dzeta, int nbins, int lmax, int ncat, int64_t zsize, const float* A, int RLP,
                   int RL, const int4* blks, int nblks, TM* Mr, TM* V, double* dw, cudaStream_t st) {
    if (adjoint_m_t<TM>(dzeta, nbins, lmax, ncat, zsize, Mr, st) != 0) return -1;
    if (nblks > 0) {
        const MInfo mi = make_info(nbins, lmax);
        const size_t smem = sizeof(float) * kRows * RL;
        if (cudaFuncSetAttribute(VgemmKernel<TM>::fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return -1;
        VgemmKernel<TM>::fn<<<(unsigned)nblks, kVThreads, smem, st>>>(A, RLP, RL, blks, 0, 0, Mr,
                                                                      adjoint_m_floats(nbins, lmax), mi, lmax, V,
                                                                      dw, nullptr, nullptr, 0);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <class TM>
int vgemm_rows_t(const float* A, int RLP, int RL, int64_t row_lo, int64_t row_hi, const TM* Mr, int nbins,
                 int lmax, TM* V, double* dw, const int* plist, const int* orig, int64_t q0, cudaStream_t st) {
    if (row_hi <= row_lo) return 0;
    const MInfo mi = make_info(nbins, lmax);
    const size_t smem = sizeof(float) * kRows * RL;
    if (cudaFuncSetAttribute(VgemmKernel<TM>::fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return -1;
    const int64_t nb = (row_hi - row_lo + kRows - 1) / kRows;
    VgemmKernel<TM>::fn<<<(unsigned)nb, kVThreads, smem, st>>>(A, RLP, RL, nullptr, row_lo, row_hi, Mr,
                                                                adjoint_m_floats(nbins, lmax), mi, lmax, V, dw,
                                                                plist, orig, q0);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}


int launch_adjoint_prep(const double* dzeta, int nbins, int lmax, int ncat, int64_t zsize, const float* A,
                        int RLP, int RL, const int4* blks, int nblks, float* Mr, float* V, double* dw,
                        cudaStream_t st) {
    return adjoint_prep_t<float>(dzeta, nbins, lmax, ncat, zsize, A, RLP, RL, blks, nblks, Mr, V, dw, st);
}

int launch_adjoint_prep_df(const double* dzeta, int nbins, int lmax, int ncat, int64_t zsize, const float* A,
                           int RLP, int RL, const int4* blks, int nblks, float2* Mr, float2* V, double* dw,
                           cudaStream_t st) {
    return adjoint_prep_t<float2>(dzeta, nbins, lmax, ncat, zsize, A, RLP, RL, blks, nblks, Mr, V, dw, st);
}

int launch_adjoint_m(const double* dzeta, int nbins, int lmax, int ncat, int64_t zsize, float* Mr,
                     cudaStream_t st) {
    return adjoint_m_t<float>(dzeta, nbins, lmax, ncat, zsize, Mr, st);
}

int launch_adjoint_m_df(const double* dzeta, int nbins, int lmax, int ncat, int64_t zsize, float2* Mr,
                        cudaStream_t st) {
    return adjoint_m_t<float2>(dzeta, nbins, lmax, ncat, zsize, Mr, st);
}

int launch_vgemm_rows(const float* A, int RLP, int RL, int64_t row_lo, int64_t row_hi, const float* Mr,
                      int nbins, int lmax, float* V, double* dw, const int* plist, const int* orig,
                      int64_t q0, cudaStream_t st) {
    return vgemm_rows_t<float>(A, RLP, RL, row_lo, row_hi, Mr, nbins, lmax, V, dw, plist, orig, q0, st);
}

int launch_vgemm_rows_df(const float* A, int RLP, int RL, int64_t row_lo, int64_t row_hi, const float2* Mr,
                         int nbins, int lmax, float2* V, double* dw, const int* plist, const int* orig,
                         int64_t q0, cudaStream_t st) {
    return vgemm_rows_t<float2>(A, RLP, RL, row_lo, row_hi, Mr, nbins, lmax, V, dw, plist, orig, q0, st);
}

}  // namespace g3
