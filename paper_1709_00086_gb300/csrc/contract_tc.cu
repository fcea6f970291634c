// zeta contraction on the 5th-generation tensor cores (tcgen05, sm_103a),
// split-BF16 form.
//
// Paper: Sec. 3.1 -- the coefficient about one primary is a_lm(r1) a*_l'm(r2),
// summed over all primaries; per m this is the Gram matrix
//      C_m = sum_i w_i v_i v_i^T        (v_i the A-row block of m),
// a dense GEMM with the primaries as the reduction dimension.
//
// Precision.  Each FP32 operand x is split into x_hi = bf16(x) and
// x_lo = bf16(x - x_hi); C = L_hi R_hi^T + L_hi R_lo^T + L_lo R_hi^T with FP32
// accumulation in tensor memory (the lo*lo product, ~2^-16 relative, is
// dropped).  With no negative weight L = R = sqrt(w) (.) A, so one hi / lo
// pair serves both sides; otherwise L = A (unweighted) and R = w (.) A.
//
// Data flow.  k_split writes the operands K-major (primaries contiguous)
// as bf16 [column][primary].  k_contract_tc: one CTA per (128 x 128 output
// tile, segment of primaries); one thread issues TMA tile loads (128B
// swizzle, 3-stage mbarrier ring) and the tcgen05.mma instructions, the
// accumulator lives in 128 TMEM columns, and four warps read it back with
// tcgen05.ld and write FP64 partials (one per (segment, tile)) that the FP64
// reduction adds in a fixed order.  Every wait is bounded: on expiry the
// kernel records a timeout in the status word, drains its own copies (again
// bounded), frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstdio>

#include "internal.h"

namespace g3 {

namespace {

constexpr int kTT = 128;          // output tile edge (M = N = 128)
constexpr int kKB = 64;           // primaries per k-block (one 128-byte swizzle row of bf16)
constexpr int kStages = 3;
constexpr int kOpBytes = kTT * kKB * 2;          // one operand tile: 16 KB
constexpr int kStageBytes = 4 * kOpBytes;        // L_hi, L_lo, R_hi, R_lo
constexpr unsigned kSpinLimit = 1u << 26;        // bounded waits

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// One non-blocking test of the phase (the error-path test's shortened first wait).
__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false on expiry.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    for (unsigned it = 0; it < kSpinLimit; ++it) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap* map, int x, int y,
                                            unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor, K-major operand with 128-byte swizzle:
// start address >> 4 (bits 0-13), leading byte offset (unused for this
// layout, 1), stride byte offset 1024 B >> 4 between 8-row groups (bits
// 32-45), descriptor version 1 (bits 46-47), swizzle mode 2 = 128B (61-63).
__device__ __forceinline__ unsigned long long make_desc(unsigned saddr) {
    unsigned long long d = 0;
    d |= (unsigned long long)((saddr & 0x3FFFF) >> 4);
    d |= (unsigned long long)1 << 16;
    d |= (unsigned long long)(1024 >> 4) << 32;
    d |= (unsigned long long)1 << 46;
    d |= (unsigned long long)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and B
// BF16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at
// bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr unsigned make_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) |
           ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(unsigned tmem_d, unsigned long long a, unsigned long long b,
                                         unsigned idesc, unsigned accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(unsigned bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

struct TcArgs {
    const Tile* tiles;
    const Segment* segs;   // row ranges in padded primary coordinates (multiples of kKB)
    double* partials;      // per (segment, tile): 128 x 128 doubles, column-major [c][r]
    int part_stride;
    const int* negw;       // 0: the right operands are the left ones (sqrt(w) A both sides)
    int* status;
    int test_timeout;      // 1: the MMA thread's first wait is one non-blocking test (error-path test)
};

constexpr int kSubKB = 32;          // k-blocks per FP32 accumulation run (2048 primaries)
constexpr int kTcWarps = 5;         // warps 0-3: TMEM drain (lanes 0-127); warp 4: TMA + MMA

__device__ __forceinline__ void tmem_ld32(unsigned taddr, unsigned (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// One CTA = one (tile, segment).  The segment's k-blocks are accumulated in
// runs of kSubKB into one of two TMEM buffers (columns [0,128) and
// [128,256)); while the MMA warp fills one buffer the drain warps add the
// other into the FP64 partial, which bounds every FP32 accumulation run to
// 3 * kSubKB * 4 MMA steps whatever the segment length.
__global__ void __launch_bounds__(kTcWarps * 32, 1)
    k_contract_tc(const __grid_constant__ CUtensorMap mLh, const __grid_constant__ CUtensorMap mLl,
                  const __grid_constant__ CUtensorMap mRh, const __grid_constant__ CUtensorMap mRl,
                  TcArgs a) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    __shared__ __align__(8) unsigned long long bars[2 * kStages + 4];
    __shared__ unsigned tmem_slot;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Tile t = a.tiles[blockIdx.x];
    const Segment sg = a.segs[blockIdx.y];
    const int kb0 = sg.row0 / kKB;
    const int nkb = (sg.row1 - sg.row0 + kKB - 1) / kKB;
    const int nsub = (nkb + kSubKB - 1) / kSubKB;
    const unsigned raw = smem_u32(tc_smem_raw);
    const unsigned sbase = (raw + 1023u) & ~1023u;  // 1024-byte aligned stage buffers
    const unsigned full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[kStages]),
                   ready0 = smem_u32(&bars[2 * kStages]), drained0 = smem_u32(&bars[2 * kStages + 2]);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(ready0 + 8 * b, 1);
            mbar_init(drained0 + 8 * b, 4);  // one arrival per drain warp
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(2 * kTT)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_slot;

    if (warp == 4) {
        if (lane == 0 && nkb > 0) {
            const int xrow = t.col0 + t.r0;  // first operand row (A column) of the tile's rows
            const int xcol = t.col0 + t.c0;  // ... of the tile's columns
            const unsigned idesc = make_idesc(kTT, kTT);
            const bool sym = *a.negw == 0;   // no negative weight: R = L = split(sqrt(w) A)
            const CUtensorMap* mrh = sym ? &mLh : &mRh;
            const CUtensorMap* mrl = sym ? &mLl : &mRl;
            bool ok = true;
            int issued = 0;
            auto issue_load = [&](int kb) {
                const int s = kb % kStages;
                const unsigned st = sbase + s * kStageBytes;
                const int x = (kb0 + kb) * kKB;
                mbar_expect_tx(full0 + 8 * s, kStageBytes);
                tma_load_2d(st + 0 * kOpBytes, &mLh, x, xrow, full0 + 8 * s);
                tma_load_2d(st + 1 * kOpBytes, &mLl, x, xrow, full0 + 8 * s);
                tma_load_2d(st + 2 * kOpBytes, mrh, x, xcol, full0 + 8 * s);
                tma_load_2d(st + 3 * kOpBytes, mrl, x, xcol, full0 + 8 * s);
            };
            for (; issued < kStages && issued < nkb; ++issued) issue_load(issued);
            for (int kb = 0; kb < nkb && ok; ++kb) {
                const int sub = kb / kSubKB, buf = sub & 1;
                const bool first = (kb % kSubKB) == 0;
                const bool last = (kb % kSubKB) == kSubKB - 1 || kb == nkb - 1;
                if (first && sub >= 2 && !mbar_wait(drained0 + 8 * buf, ((sub >> 1) - 1) & 1)) {
                    ok = false;
                    break;
                }
                const int s = kb % kStages;
                const bool landed = (kb == 0 && a.test_timeout) ? mbar_test(full0, 0)
                                                                : mbar_wait(full0 + 8 * s, (kb / kStages) & 1);
                if (!landed) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned st = sbase + s * kStageBytes;
                const unsigned Lh = st, Ll = st + kOpBytes, Rh = st + 2 * kOpBytes, Rl = st + 3 * kOpBytes;
                const unsigned d = tmem + (unsigned)(buf * kTT);
#pragma unroll
                for (int k = 0; k < kKB / 16; ++k) {
                    const unsigned off = k * 32;  // 16 bf16 along K inside the swizzled row
                    mma_bf16(d, make_desc(Lh + off), make_desc(Rh + off), idesc,
                             (first && k == 0) ? 0u : 1u);
                    mma_bf16(d, make_desc(Lh + off), make_desc(Rl + off), idesc, 1u);
                    mma_bf16(d, make_desc(Ll + off), make_desc(Rh + off), idesc, 1u);
                }
                mma_commit(empty0 + 8 * s);  // frees stage s when these MMAs have read it
                if (last) mma_commit(ready0 + 8 * buf);
                if (kb >= 1 && issued < nkb) {
                    // refill the stage freed by the previous k-block
                    const int ps = issued % kStages;
                    if (!mbar_wait(empty0 + 8 * ps, ((issued / kStages) - 1) & 1)) {
                        ok = false;
                        break;
                    }
                    issue_load(issued);
                    ++issued;
                }
            }
            if (!ok) {
                abort_flag = 1;
                __threadfence_block();
                atomicOr(a.status, kStatusTimeout);
                // drain this CTA's own copies still in flight (bounded), then
                // release the drain warps
                for (int kb = 0; kb < issued; ++kb)
                    mbar_wait(full0 + 8 * (kb % kStages), (kb / kStages) & 1);
                mma_commit(ready0);
                mma_commit(ready0 + 8);
            }
        }
    } else {
        // drain warps: TMEM lane (= output row) warp*32 + lane
        const int row = warp * 32 + lane;
        double* out = a.partials + (int64_t)blockIdx.y * a.part_stride + t.out_off;
        for (int sub = 0; sub < nsub; ++sub) {
            const int buf = sub & 1;
            const bool ok = mbar_wait(ready0 + 8 * buf, (sub >> 1) & 1);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (!ok || abort_flag) {
                if (lane == 0) atomicOr(a.status, kStatusTimeout);
                break;
            }
#pragma unroll 1
            for (int c0 = 0; c0 < kTT; c0 += 32) {
                unsigned r[32];
                tmem_ld32(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)(buf * kTT + c0), r);
                if (row < t.rows) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        if (c0 + j < t.cols) {
                            double* o = out + (int64_t)(c0 + j) * kTT + row;  // column-major
                            const double v = (double)__uint_as_float(r[j]);
                            *o = (sub == 0) ? v : *o + v;
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(drained0 + 8 * buf) : "memory");
        }
        if (nsub == 0 && row < t.rows)
            for (int c = 0; c < t.cols; ++c) out[(int64_t)c * kTT + row] = 0.0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTT)
                     : "memory");
}

// A (rows x RLP, FP32) -> K-major bf16 operands [col][pr] for the split
// product.  pr is the padded primary position: catalog c occupies
// [cats[c].x, cats[c].x + cats[c].z) with its rows starting at cats[c].y,
// and every catalog starts on a multiple of kKB; the gaps are written as 0.
// One block per kSplitP = 64 padded primaries sweeps all columns in tiles of
// 32 (rows read as 128-byte lines, each column written as one 128-byte line
// of bf16 pairs per operand).
// With no negative weight (*negw == 0) both sides of w_i a a^T are sqrt(w_i) a,
// so only its hi / lo pair is written (Lh, Ll; the contraction reads them for
// both sides); otherwise L = A and R = w A as four arrays.
constexpr int kSplitP = 64;

__global__ void __launch_bounds__(256) k_split(const float* __restrict__ A, int RLP, int RL,
                                               const float* __restrict__ w, const int4* __restrict__ cats,
                                               int ncat, int64_t P_pad, const int* __restrict__ negw,
                                               __nv_bfloat16* Lh, __nv_bfloat16* Ll, __nv_bfloat16* Rh,
                                               __nv_bfloat16* Rl) {
    __shared__ float tl[kSplitP][33];
    __shared__ float tw[kSplitP];
    __shared__ int trow[kSplitP];
    const bool sym = *negw == 0;
    const int64_t p0 = (int64_t)blockIdx.x * kSplitP;  // padded primary positions
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    if (threadIdx.x < kSplitP) {
        const int64_t pr = p0 + threadIdx.x;
        int lo = 0, hi = ncat - 1;  // last catalog starting at or before pr
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (cats[mid].x <= pr) lo = mid; else hi = mid - 1;
        }
        const int4 ct = cats[lo];
        const int64_t k = pr - ct.x;
        const int r = (pr < P_pad && k >= 0 && k < ct.z) ? (int)(ct.y + k) : -1;
        trow[threadIdx.x] = r;
        const float wr = r >= 0 ? w[r] : 0.f;
        tw[threadIdx.x] = sym ? sqrtf(wr) : wr;
    }
    __syncthreads();
    for (int c0 = 0; c0 < RL; c0 += 32) {
        for (int k = ty; k < kSplitP; k += 8) {  // primary k, columns c0 .. c0 + 31
            const int r = trow[k];
            const int c = c0 + tx;
            tl[k][tx] = (r >= 0 && c < RL) ? A[(int64_t)r * RLP + c] : 0.f;
        }
        __syncthreads();
        for (int k = ty; k < 32; k += 8) {  // column c0 + k, primaries 2 tx and 2 tx + 1
            const int c = c0 + k;
            const int64_t pr = p0 + 2 * tx;
            if (c < RL && pr < P_pad && sym) {
                const float y0 = tl[2 * tx][k] * tw[2 * tx], y1 = tl[2 * tx + 1][k] * tw[2 * tx + 1];
                const __nv_bfloat16 yh0 = __float2bfloat16_rn(y0), yh1 = __float2bfloat16_rn(y1);
                const int64_t o = (int64_t)c * P_pad + pr;
                *reinterpret_cast<__nv_bfloat162*>(Lh + o) = __halves2bfloat162(yh0, yh1);
                *reinterpret_cast<__nv_bfloat162*>(Ll + o) =
                    __halves2bfloat162(__float2bfloat16_rn(y0 - __bfloat162float(yh0)),
                                       __float2bfloat16_rn(y1 - __bfloat162float(yh1)));
            } else if (c < RL && pr < P_pad) {
                const float x0 = tl[2 * tx][k], x1 = tl[2 * tx + 1][k];
                const float y0 = x0 * tw[2 * tx], y1 = x1 * tw[2 * tx + 1];
                const __nv_bfloat16 xh0 = __float2bfloat16_rn(x0), xh1 = __float2bfloat16_rn(x1);
                const __nv_bfloat16 yh0 = __float2bfloat16_rn(y0), yh1 = __float2bfloat16_rn(y1);
                const int64_t o = (int64_t)c * P_pad + pr;
                *reinterpret_cast<__nv_bfloat162*>(Lh + o) = __halves2bfloat162(xh0, xh1);
                *reinterpret_cast<__nv_bfloat162*>(Ll + o) =
                    __halves2bfloat162(__float2bfloat16_rn(x0 - __bfloat162float(xh0)),
                                       __float2bfloat16_rn(x1 - __bfloat162float(xh1)));
                *reinterpret_cast<__nv_bfloat162*>(Rh + o) = __halves2bfloat162(yh0, yh1);
                *reinterpret_cast<__nv_bfloat162*>(Rl + o) =
                    __halves2bfloat162(__float2bfloat16_rn(y0 - __bfloat162float(yh0)),
                                       __float2bfloat16_rn(y1 - __bfloat162float(yh1)));
            }
        }
        __syncthreads();
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

int make_map(CUtensorMap* m, void* base, int64_t P_pad, int RL) {
    auto fn = encode_fn();
    if (!fn) return -1;
    cuuint64_t dims[2] = {(cuuint64_t)P_pad, (cuuint64_t)RL};
    cuuint64_t strides[1] = {(cuuint64_t)P_pad * 2};
    cuuint32_t box[2] = {kKB, kTT};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

}  // namespace

int contract_tile_dim_tc() { return kTT; }
int contract_tc_kblock() { return kKB; }

int launch_split(const float* A, int RLP, int RL, const float* w, const int4* cats, int ncat,
                 int64_t P_pad, const int* negw, void* ops, cudaStream_t st) {
    if (P_pad <= 0) return 0;
    __nv_bfloat16* base = static_cast<__nv_bfloat16*>(ops);
    const int64_t n1 = (int64_t)RL * P_pad;
    k_split<<<(unsigned)((P_pad + kSplitP - 1) / kSplitP), 256, 0, st>>>(A, RLP, RL, w, cats, ncat, P_pad, negw,
                                                                         base, base + n1, base + 2 * n1, base + 3 * n1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_contract_tc(const void* ops, int64_t P_pad, int RL, const Tile* tiles, int ntiles,
                       const Segment* segs, int nsegs, double* partials, int part_stride,
                       const int* negw, int* status, cudaStream_t st, int test_timeout) {
    if (ntiles <= 0 || nsegs <= 0) return 0;
    const __nv_bfloat16* base = static_cast<const __nv_bfloat16*>(ops);
    const int64_t n1 = (int64_t)RL * P_pad;
    CUtensorMap m[4];
    for (int k = 0; k < 4; ++k)
        if (make_map(&m[k], const_cast<__nv_bfloat16*>(base + k * n1), P_pad, RL) != 0) return -2;
    const int smem = kStages * kStageBytes + 1024;
    if (cudaFuncSetAttribute(k_contract_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
        return -1;
    TcArgs a{tiles, segs, partials, part_stride, negw, status, test_timeout};
    dim3 grid(ntiles, nsegs);
    k_contract_tc<<<grid, kTcWarps * 32, smem, st>>>(m[0], m[1], m[2], m[3], a);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace g3
