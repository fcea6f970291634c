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
// Data flow.  The operands are formed inside the kernel from the FP32
// multipole rows A (no separate split pass, no operand buffer): one CTA per
// work item = (strip, range of primaries).  A strip is one or two 128 x 128
// output tiles side by side in one row panel of an m block, computed as one
// M = 128, N = 128 or 256 MMA, so the row panel is formed once for both
// tiles; when the strip starts on the diagonal of the symmetric form its row
// panel is the first column panel.  The primaries of every catalog are cut
// into an even number of equal "virtual segments"; a two-tile strip takes one
// per CTA and a one-tile strip two, so that every CTA does the same MMA work
// (its partial goes to the first slot and the second is zeroed).
//   warp 9 (TMA): per k-block of 64 primaries and panel, one 2-D bulk copy of
//     the FP32 rows of A (the columns the panel's MMAs use, from the panel's
//     first column rounded down to a 16-byte boundary) into a staging slot,
//     with the primaries' scales of that side (sqrt(w), or 1 and w) beside it;
//   warps 10-25 (converters): scale the staged rows, split them into bf16 hi
//     and lo and store them K-major in the 128-byte swizzled shared-memory
//     layout of the MMA descriptors, in one operand stage handed to the MMA
//     thread through mbarriers; every converter warp runs on its own, and a
//     warp whose rows no MMA uses forms nothing;
//   warp 8 (one thread): tcgen05.mma of width N (the strip's valid columns
//     rounded up to 16) into a TMEM accumulator, double-buffered per run of
//     kSubKB k-blocks;
//   warps 0-7 (drain): tcgen05.ld of each finished run (two warps per TMEM
//     lane quarter, alternate 32-column groups), added to the FP64 partials
//     (one per (virtual segment, tile), kept in L2 with evict-last priority)
//     that the FP64 reduction adds in a fixed order.
// Every wait is bounded: on expiry the kernel records a timeout in the status
// word, every warp stops at its next wait, the TMA thread lets its own copies
// land, the TMEM is freed and the kernel returns.
#include <algorithm>
#include <vector>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "internal.h"

namespace g3 {

namespace {

constexpr int kTT = 128;          // output tile edge (M = N = 128)
constexpr int kKB = 64;           // primaries per k-block (one 128-byte swizzle row of bf16)
constexpr int kKSteps = kKB / 16;  // MMA k-steps per k-block (K = 16 for kind::f16)
constexpr int kOpBytes = kTT * kKB * 2;          // one operand box (128 rows x 64 primaries): 16 KB
// stage buffers: 2 to 6 operand boxes per stage (R hi / lo of one or two panels,
// L hi / lo unless shared with R).  One operand stage: while the MMAs read it
// the converters only load and split the next k-block, and store it once the
// MMAs are done (measured faster than a ring of stages, where the converters'
// stores and the MMAs' operand reads contend for shared-memory bandwidth:
// 4.37 vs 4.65 ms on the 2M-point workload); the rest holds FP32 staging slots.
constexpr int kBufBytes = 13 * kOpBytes;         // 208 KB: operand stage + FP32 staging slots
constexpr int kMaxStages = 1;
// FP32 staging of one unit (one panel of one k-block): rows of A for the 64
// primaries, 132 columns from the panel's first column rounded down to a
// multiple of 4 (a TMA box must start on a 16-byte boundary)
constexpr int kStgCols = kTT + 4;
constexpr int kStgBytes = kKB * kStgCols * 4;    // 33,792 bytes
// A unit copies only the columns its panel's MMAs use: boxes of 32 w + 4
// columns (w = 1..4, tensor map w - 1), staged with that row pitch.
constexpr int kBoxes = kTT / 32;
__host__ __device__ constexpr int box_cols(int wi) { return 32 * (wi + 1) + 4; }
struct TcMaps {
    CUtensorMap m[kBoxes];
};

constexpr int kMaxStg = 6;
static_assert(kBufBytes + 1024 + 1024 <= 227 * 1024, "stage buffers and barriers fit in shared memory");
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
    const float* A;        // multipole rows (FP32), row pitch RLP (also read through the tensor map)
    int RLP;
    const float* wrow;     // weight of every A row
    const int4* cats;      // per catalog {padded start, first A row, length, 0}
    const Tile* tiles;
    const TcStrip* strips;
    const TcItem* items;
    const Segment* segs;   // virtual segments in padded primary coordinates (multiples of kKB)
    double* partials;      // per (virtual segment, tile): 128 x 128 doubles, column-major [c][r]
    int part_stride;
    const int* negw;       // 0: both operand sides are sqrt(w) A (no negative weight)
    int* status;
    int test_timeout;      // 1: the MMA thread's first wait gives up at once (error-path test)
};

constexpr int kSubKB = 32;          // k-blocks per FP32 accumulation run (2048 primaries)
constexpr int kDrainWarps = 8;      // warps 0-7: TMEM drain (lanes 32 (w % 4) .., column groups of parity w / 4)
constexpr int kDrainBatch = 16;     // partial columns read before they are written back
constexpr int kMmaWarp = 8;         // warp 8: MMA issue
constexpr int kTmaWarp = 9;         // warp 9: TMA loads of the FP32 rows
constexpr int kCvtWarps = 16;       // warps 10-25: operand formation
constexpr int kTcWarps = kDrainWarps + 2 + kCvtWarps;
static_assert(kCvtWarps * 32 == kTT * kKSteps, "one converter thread per (panel row, k-step)");

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

// The FP64 partials are re-read by every accumulation run of their CTA: kept in
// L2 ahead of the streamed rows of A (evict-last priority).
__device__ __forceinline__ unsigned long long l2_keep_policy() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ double ld_keep(const double* ptr, unsigned long long pol) {
    double v;
    asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_keep(double* ptr, double v, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(ptr), "d"(v), "l"(pol) : "memory");
}

// Bounded wait that also gives up when another warp has flagged an abort.
__device__ __forceinline__ bool mbar_wait_or_abort(unsigned bar, unsigned parity, volatile int* abort_flag) {
    for (unsigned it = 0; it < kSpinLimit; ++it) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (*abort_flag) return false;
    }
    return false;
}

// Drain warps of a work item: TMEM lane (= output row) 32 (warp % 4) + lane;
// column c of the accumulator is column c % 128 of the strip's tile c / 128;
// warp w takes the 32-column groups g with g % 2 == w / 4.  Each finished run
// (ready barrier) is added to the item's FP64 partials, then the TMEM buffer is
// released (drained barrier); the item's other segment slots are zeroed.
__device__ __forceinline__ void drain_item(int warp, int lane, unsigned tmem, int N, int Np, int nt, int nsub,
                                           unsigned ready0, unsigned drained0, volatile int* abort_flag,
                                           const Tile* tiles, const TcStrip& sp, const TcItem& it, double* partials,
                                           int part_stride, int* status) {
    const int quarter = warp & 3, half = warp >> 2;
    const int row = quarter * 32 + lane;
    const unsigned long long keep = l2_keep_policy();
    double* outs = partials + (int64_t)it.vseg0 * part_stride;
    for (int sub = 0; sub < nsub; ++sub) {
        const int buf = sub & 1;
        const bool ok = mbar_wait(ready0 + 8 * buf, (sub >> 1) & 1);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!ok || *abort_flag) {
            if (lane == 0) atomicOr(status, kStatusTimeout);
            break;
        }
        // the partial is column-major (a warp's rows of one column are one
        // 256-byte line); a run after the first adds to it, reading a batch
        // of kDrainBatch columns before writing them, so that the batch's
        // loads are in flight together
#pragma unroll 1
        for (int c0 = 32 * half; c0 < N; c0 += 64) {
            unsigned rr[32];
            tmem_ld32(tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)(buf * Np + c0), rr);
            const Tile t = tiles[sp.tile0 + c0 / kTT];
            const int cc = c0 % kTT;
            const int ncol = t.cols - cc;  // valid columns from cc (the tile's width)
            double* out = outs + t.out_off + (int64_t)cc * kTT + row;
            if (row < t.rows) {
                if (sub == 0) {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (j < ncol) st_keep(out + (int64_t)j * kTT, (double)__uint_as_float(rr[j]), keep);
                } else {
#pragma unroll
                    for (int h = 0; h < 32; h += kDrainBatch) {
                        double old[kDrainBatch];
#pragma unroll
                        for (int j = 0; j < kDrainBatch; ++j)
                            old[j] = (h + j < ncol) ? ld_keep(out + (int64_t)(h + j) * kTT, keep) : 0.0;
#pragma unroll
                        for (int j = 0; j < kDrainBatch; ++j)
                            if (h + j < ncol)
                                st_keep(out + (int64_t)(h + j) * kTT, old[j] + (double)__uint_as_float(rr[h + j]), keep);
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(drained0 + 8 * buf) : "memory");
    }
    // an empty range writes zeros; the item's later virtual segments are zeroed
    // (their primaries are in the first slot's sum)
    for (int p = 0; p < nt; ++p) {
        const Tile t = tiles[sp.tile0 + p];
        for (int v = (nsub == 0 ? 0 : 1); v < it.nvseg; ++v) {
            double* out = partials + (int64_t)(it.vseg0 + v) * part_stride + t.out_off;
            for (int c = half; c < kTT; c += 2) out[(int64_t)c * kTT + row] = 0.0;
        }
    }
}

// One CTA = one work item (strip, virtual segments).  The k-blocks are
// accumulated in runs of kSubKB into one of two TMEM buffers (columns [0, Np)
// and [Np, 2 Np)); while the MMA warp fills one buffer the drain warps add the
// other into the FP64 partials, which bounds every FP32 accumulation run to
// 3 * kSubKB * 4 MMA steps whatever the segment length.
//   units: the panels of every k-block in order (u = nb kb + b; panel b < nt
//   is the b-th column panel, b = nt the row panel when it is not shared);
//   the TMA thread stages unit u in slot u % S, the converters turn it into
//   the operand boxes of stage kb % O, the MMA thread consumes the stage.
__global__ void __launch_bounds__(kTcWarps * 32, 1)
    k_contract_tc(const __grid_constant__ TcMaps maps, TcArgs a) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    __shared__ __align__(8) unsigned long long bars[2 * kMaxStages + 2 * kMaxStg + 4];
    __shared__ unsigned tmem_slot;
    __shared__ int abort_flag;
    __shared__ __align__(16) float meta[kMaxStg][kKB];  // per staged unit: its side's scale of each primary
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const TcItem it = a.items[blockIdx.x];
    const TcStrip sp = a.strips[it.strip];
    const Segment sg0 = a.segs[it.vseg0];
    const int row0 = sg0.row0, row1 = a.segs[it.vseg0 + it.nvseg - 1].row1;
    const int kb0 = row0 / kKB;
    const int nkb = (row1 - row0 + kKB - 1) / kKB;
    const int nsub = (nkb + kSubKB - 1) / kSubKB;
    const int nt = sp.ntile;   // tiles side by side (column panels of 128)
    const int N = sp.n;        // MMA width: the strip's valid columns rounded up to 16
    const int Np = kTT * nt;   // TMEM columns of one accumulator buffer
    const unsigned raw = smem_u32(tc_smem_raw);
    const unsigned sbase = (raw + 1023u) & ~1023u;  // 1024-byte aligned stage buffers
    unsigned char* sgen = tc_smem_raw + (sbase - raw);
    // no negative weight: both sides are sqrt(w) A; a strip that starts on the
    // diagonal then finds its row panel as the first column panel
    const bool sym = *a.negw == 0;
    const bool lshare = sym && sp.xrow == sp.xcol;
    const int nb = lshare ? nt : nt + 1;               // units (panels) per k-block
    const unsigned stage_bytes = (unsigned)(2 * nb) * kOpBytes;
    // as many staging slots (copies in flight) as fit beside one operand stage
    int S = (int)((kBufBytes - stage_bytes) / kStgBytes);
    S = S < kMaxStg ? S : kMaxStg;
    S = S > 1 ? S : 1;
    int O = (int)((kBufBytes - S * kStgBytes) / stage_bytes);
    O = O < kMaxStages ? O : kMaxStages;
    const unsigned stg0 = (unsigned)O * stage_bytes;   // staging after the operand stages
    const unsigned ofull0 = smem_u32(&bars[0]), oempty0 = smem_u32(&bars[kMaxStages]);
    const unsigned sfull0 = smem_u32(&bars[2 * kMaxStages]), sempty0 = smem_u32(&bars[2 * kMaxStages + kMaxStg]);
    const unsigned ready0 = smem_u32(&bars[2 * kMaxStages + 2 * kMaxStg]);
    const unsigned drained0 = ready0 + 16;
    const int nunits = nkb * nb;
    const int4 cat = a.cats[sg0.cat];
    if (threadIdx.x == 0) {
        for (int s = 0; s < kMaxStages; ++s) {
            mbar_init(ofull0 + 8 * s, kCvtWarps);  // one arrival per converter warp
            mbar_init(oempty0 + 8 * s, 1);         // the MMA thread's commit
        }
        for (int s = 0; s < kMaxStg; ++s) {
            mbar_init(sfull0 + 8 * s, 1);          // TMA bytes
            mbar_init(sempty0 + 8 * s, kCvtWarps);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(ready0 + 8 * b, 1);
            mbar_init(drained0 + 8 * b, kDrainWarps);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(2 * Np)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_slot;
    auto unit_col = [&](int b) { return b == nt ? sp.xrow : sp.xcol + kTT * b; };
    // operand rows of unit b that the MMAs use: the B operand's N rows of a
    // column panel, and the row panel's valid rows for A (the other rows of D
    // are discarded); its box is the narrowest that holds them from xp & ~3
    const int rowsL = a.tiles[sp.tile0].rows;
    auto unit_need = [&](int b) {
        const bool isL = b == nt;
        const int needB = isL ? 0 : min(kTT, N - kTT * b);
        return (isL || (lshare && b == 0)) ? max(needB, rowsL) : needB;
    };
    auto unit_box = [&](int b) { return (unit_need(b) + 31) / 32 - 1; };

    if (warp == kTmaWarp) {
        // unit u: the scales of its side into meta[u % S] (0 past the catalog),
        // then the FP32 rows into staging slot u % S; the slot's mbarrier phase
        // (the elected lane's arrive, release, and the copy's bytes) publishes both.
        // The weights of k-block kb + 2 are loaded while kb is issued, so that no
        // global load latency sits between two copies.
        int issued = 0;
        bool ok = true;
        auto wload = [&](int kb, int i) -> float {
            const int k = (kb0 + kb) * kKB + i - cat.x;
            return (kb < nkb && k >= 0 && k < cat.z) ? __ldg(a.wrow + cat.y + k) : 0.f;
        };
        auto inrange = [&](int kb, int i) {
            const int k = (kb0 + kb) * kKB + i - cat.x;
            return k >= 0 && k < cat.z;
        };
        float w0a = wload(0, lane), w0b = wload(0, lane + 32);
        float w1a = wload(1, lane), w1b = wload(1, lane + 32);
        float w2a = 0.f, w2b = 0.f;
        for (int u = 0; u < nunits; ++u) {
            const int slot = u % S;
            if (u >= S) {
                const bool freed = mbar_wait_or_abort(sempty0 + 8 * slot, ((u / S) - 1) & 1, &abort_flag);
                if (!__all_sync(0xffffffffu, freed)) {
                    ok = false;
                    break;
                }
            }
            const int kb = u / nb, b = u - kb * nb;
            const bool isL = b == nt;
            if (b == 0 && kb > 0) {
                w0a = w1a;
                w0b = w1b;
                w1a = w2a;
                w1b = w2b;
            }
            if (b == 0) {
                w2a = wload(kb + 2, lane);
                w2b = wload(kb + 2, lane + 32);
            }
            static_assert(kKB == 64, "two weights per lane");
            meta[slot][lane] = sym ? sqrtf(w0a) : (isL ? (inrange(kb, lane) ? 1.f : 0.f) : w0a);
            meta[slot][lane + 32] = sym ? sqrtf(w0b) : (isL ? (inrange(kb, lane + 32) ? 1.f : 0.f) : w0b);
            __syncwarp();
            if (lane == 0) {
                const int xp = unit_col(b);
                const int y = cat.y + (kb0 + kb) * kKB - cat.x;  // A row of the k-block's first primary
                const int wi = unit_box(b);
                mbar_expect_tx(sfull0 + 8 * slot, (unsigned)(box_cols(wi) * kKB * 4));
                tma_load_2d(sbase + stg0 + slot * kStgBytes, &maps.m[wi], xp & ~3, y, sfull0 + 8 * slot);
            }
            ++issued;
        }
        if (lane == 0) {
            if (!ok && !abort_flag) {
                abort_flag = 1;
                atomicOr(a.status, kStatusTimeout);
            }
            if (abort_flag) {
                // this CTA's copies still in flight (the latest one of every slot;
                // earlier ones were consumed) land before it exits (bounded)
                for (int u = issued > S ? issued - S : 0; u < issued; ++u)
                    mbar_wait(sfull0 + 8 * (u % S), (u / S) & 1);
            }
        }
    } else if (warp == kMmaWarp) {
        if (lane == 0 && nkb > 0) {
            const unsigned idesc = make_idesc(kTT, N);
            bool ok = true;
            for (int kb = 0; kb < nkb && ok; ++kb) {
                const int sub = kb / kSubKB, buf = sub & 1;
                const bool first = (kb % kSubKB) == 0;
                const bool last = (kb % kSubKB) == kSubKB - 1 || kb == nkb - 1;
                if (first && sub >= 2 && !mbar_wait(drained0 + 8 * buf, ((sub >> 1) - 1) & 1)) {
                    ok = false;
                    break;
                }
                const int o = kb % O;
                // error-path test: the first wait gives up at once, as if its bound had expired
                const bool formed = (kb == 0 && a.test_timeout)
                                        ? false
                                        : mbar_wait_or_abort(ofull0 + 8 * o, (kb / O) & 1, &abort_flag);
                if (!formed) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned st = sbase + o * stage_bytes;
                const unsigned Rh = st, Rl = st + nt * kOpBytes;
                const unsigned Lh = lshare ? Rh : st + 2 * nt * kOpBytes, Ll = lshare ? Rl : Lh + kOpBytes;
                const unsigned d = tmem + (unsigned)(buf * Np);
#pragma unroll
                for (int k = 0; k < kKB / 16; ++k) {
                    const unsigned off = k * 32;  // 16 bf16 along K inside the swizzled row
                    mma_bf16(d, make_desc(Lh + off), make_desc(Rh + off), idesc,
                             (first && k == 0) ? 0u : 1u);
                    mma_bf16(d, make_desc(Lh + off), make_desc(Rl + off), idesc, 1u);
                    mma_bf16(d, make_desc(Ll + off), make_desc(Rh + off), idesc, 1u);
                }
                mma_commit(oempty0 + 8 * o);  // frees the operand stage when these MMAs have read it
                if (last) mma_commit(ready0 + 8 * buf);
            }
            if (!ok) {
                if (!abort_flag) {
                    abort_flag = 1;
                    atomicOr(a.status, kStatusTimeout);
                }
                // release the drain warps (the commits complete when every MMA
                // already issued has finished)
                mma_commit(ready0);
                mma_commit(ready0 + 8);
            }
        }
    } else if (warp > kTmaWarp) {
        // converters: unit u (staged FP32 rows of one panel) -> bf16 hi / lo of
        // the scaled rows, K-major in the swizzled layout of operand stage
        // kb % O.  Thread ct takes panel row r = ct % 128 (A column xp + r) and
        // primaries [16 q, 16 q + 16) of the k-block, q = ct / 128: a warp reads
        // 32 consecutive words of one staged row (distinct banks), and its
        // 16-byte stores (one chunk of 8 primaries per lane) cover every bank
        // group four times.  No per-element test: a primary past its catalog
        // has scale 0, columns past the m block only feed discarded rows of the
        // tile, and the box reads zeros past the ends of A.  Every converter
        // warp runs on its own: the mbarriers order it against the TMA and MMA
        // threads, and a warp that stops on an expired wait raises the abort
        // flag, which ends the other warps' next wait.
        const int ct = threadIdx.x - (kTmaWarp + 1) * 32;
        const int r = ct & (kTT - 1);
        const int q = ct >> 7;
        const unsigned swz = (unsigned)((r >> 3) * 1024 + (r & 7) * 128);
        // a warp whose 32 rows are all past unit_need forms nothing (the MMAs
        // never read those rows, or read them only into discarded rows of D)
        const int r0w = r & ~31;
        for (int u = 0; u < nunits; ++u) {
            const int kb = u / nb, b = u - kb * nb;
            const int o = kb % O, slot = u % S;
            const bool landed = mbar_wait_or_abort(sfull0 + 8 * slot, (u / S) & 1, &abort_flag);
            if (!__all_sync(0xffffffffu, landed)) {
                if (lane == 0 && !abort_flag) {
                    abort_flag = 1;
                    atomicOr(a.status, kStatusTimeout);
                }
                break;
            }
            const int xp = unit_col(b);
            const bool isL = b == nt;
            const bool active = r0w < unit_need(b);  // warp-uniform
            const int pitch = box_cols(unit_box(b));
            const float* stg = reinterpret_cast<const float*>(sgen + stg0 + slot * kStgBytes) +
                               (16 * q) * pitch + (xp & 3) + r;
            const float4* sc4 = reinterpret_cast<const float4*>(&meta[slot][16 * q]);
            float cur[16];
            if (active) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float4 sc = sc4[c];
                    cur[4 * c] = __fmul_rn(stg[(4 * c) * pitch], sc.x);
                    cur[4 * c + 1] = __fmul_rn(stg[(4 * c + 1) * pitch], sc.y);
                    cur[4 * c + 2] = __fmul_rn(stg[(4 * c + 2) * pitch], sc.z);
                    cur[4 * c + 3] = __fmul_rn(stg[(4 * c + 3) * pitch], sc.w);
                }
            }
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sempty0 + 8 * slot) : "memory");
            unsigned h[8], l[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const float2 y = make_float2(cur[2 * e], cur[2 * e + 1]);
                const __nv_bfloat162 hp = __floats2bfloat162_rn(y.x, y.y);
                const unsigned hu = *reinterpret_cast<const unsigned*>(&hp);
                const float2 hf = make_float2(__uint_as_float(hu << 16), __uint_as_float(hu & 0xffff0000u));
                const float2 dd = __fadd2_rn(y, make_float2(-hf.x, -hf.y));
                const __nv_bfloat162 lp = __floats2bfloat162_rn(dd.x, dd.y);
                h[e] = hu;
                l[e] = *reinterpret_cast<const unsigned*>(&lp);
            }
            // the operand stage must have been read by the MMAs of k-block kb - O
            if (b == 0 && kb >= O) {
                const bool freed = mbar_wait_or_abort(oempty0 + 8 * o, ((kb / O) - 1) & 1, &abort_flag);
                if (!__all_sync(0xffffffffu, freed)) {
                    if (lane == 0 && !abort_flag) {
                        abort_flag = 1;
                        atomicOr(a.status, kStatusTimeout);
                    }
                    break;
                }
            }
            const unsigned st = o * stage_bytes;
            unsigned char* hib = sgen + st + (isL ? 2 * nt : b) * kOpBytes + swz;
            unsigned char* lob = sgen + st + (isL ? 2 * nt + 1 : nt + b) * kOpBytes + swz;
            if (active) {
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const unsigned chunk = (unsigned)(((2 * q + c) ^ (r & 7)) << 4);
                    *reinterpret_cast<uint4*>(hib + chunk) =
                        make_uint4(h[4 * c], h[4 * c + 1], h[4 * c + 2], h[4 * c + 3]);
                    *reinterpret_cast<uint4*>(lob + chunk) =
                        make_uint4(l[4 * c], l[4 * c + 1], l[4 * c + 2], l[4 * c + 3]);
                }
            }
            if (b == nb - 1) {
                // the MMA reads shared memory through the async proxy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(ofull0 + 8 * o) : "memory");
            }
        }
    } else {
        drain_item(warp, lane, tmem, N, Np, nt, nsub, ready0, drained0, &abort_flag, a.tiles, sp, it, a.partials,
                   a.part_stride, a.status);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * Np)
                     : "memory");
}

// ---- the same contraction from bf16 operand rows written by k_accum ----------
// On request (G3PCF_OPT_TC_OPERANDS = 1) and when no weight is negative, k_accum
// writes sqrt(w) A split into bf16 hi and lo rows (the same operations as the
// converter warps, so the operands and the result are bit-identical), each m
// block from a multiple of 64 columns, a row's hi and lo side by side.  The
// operands are then MN-major in the 128-byte swizzle: one 2-D copy of 64 operand
// columns x 64 primaries lands as eight groups of 8 primaries x 128 bytes, the
// descriptors step 8 KB between 64-column boxes (leading byte offset) and 1 KB
// between 8-primary groups (stride byte offset), and an MMA k-step of 16
// primaries advances 2 KB.  No staging, no conversion: warp 9 copies the boxes
// the MMAs use into a ring of operand stages, warp 8 issues the MMAs, warps 0-7
// drain as in k_contract_tc.
constexpr int kOpMmaWarp = kDrainWarps;      // warp 8
constexpr int kOpTmaWarp = kDrainWarps + 1;  // warp 9
constexpr int kOpWarps = kDrainWarps + 2;
constexpr int kOpBox = 64 * kKB * 2;         // one box: 64 columns x 64 primaries of bf16 = 8 KB
constexpr int kOpMaxStages = 8;

__device__ __forceinline__ unsigned long long make_desc_mn(unsigned saddr) {
    unsigned long long d = 0;
    d |= (unsigned long long)((saddr & 0x3FFFF) >> 4);
    d |= (unsigned long long)(kOpBox >> 4) << 16;  // leading byte offset: the next 64 columns
    d |= (unsigned long long)(1024 >> 4) << 32;    // stride byte offset: the next 8 primaries
    d |= (unsigned long long)1 << 46;
    d |= (unsigned long long)2 << 61;
    return d;
}
// as make_idesc, with both operands MN-major (bits 15 and 16)
__host__ __device__ constexpr unsigned make_idesc_mn(int M, int N) {
    return make_idesc(M, N) | (1u << 15) | (1u << 16);
}

struct TcOpMaps {
    CUtensorMap hi, lo;
};
struct TcOpArgs {
    const Tile* tiles;
    const TcStrip* strips;
    const TcItem* items;
    const Segment* segs;  // padded primary coordinates = operand rows
    double* partials;
    int part_stride;
    int* status;
    int test_timeout;
};

__global__ void __launch_bounds__(kOpWarps * 32, 1)
    k_contract_tc_op(const __grid_constant__ TcOpMaps maps, TcOpArgs a) {
    extern __shared__ __align__(1024) unsigned char op_smem_raw[];
    __shared__ __align__(8) unsigned long long bars[2 * kOpMaxStages + 4];
    __shared__ unsigned tmem_slot;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const TcItem it = a.items[blockIdx.x];
    const TcStrip sp = a.strips[it.strip];
    const int row0 = a.segs[it.vseg0].row0, row1 = a.segs[it.vseg0 + it.nvseg - 1].row1;
    const int kb0 = row0 / kKB;
    const int nkb = (row1 - row0 + kKB - 1) / kKB;
    const int nsub = (nkb + kSubKB - 1) / kSubKB;
    const int nt = sp.ntile, N = sp.n, Np = kTT * nt;
    const int rowsL = a.tiles[sp.tile0].rows;
    const unsigned raw = smem_u32(op_smem_raw);
    const unsigned sbase = (raw + 1023u) & ~1023u;
    // stage: panel b's hi boxes from b * 16 KB, its lo boxes from (nt + b) * 16 KB
    const unsigned stage_bytes = (unsigned)(2 * nt) * kOpBytes;
    int O = (int)(kBufBytes / stage_bytes);
    O = O < kOpMaxStages ? O : kOpMaxStages;
    // boxes of panel b that the MMAs read: B's N columns; panel 0 is also A,
    // whose rows past the row panel's valid rows only feed discarded rows of D
    auto nbox = [&](int b) {
        const int needB = min(kTT, N - kTT * b);
        const int need = b == 0 ? max(needB, rowsL) : needB;
        return (need + 63) / 64;
    };
    unsigned kb_bytes = 0;
    for (int b = 0; b < nt; ++b) kb_bytes += (unsigned)(2 * nbox(b) * kOpBox);
    const unsigned full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[kOpMaxStages]);
    const unsigned ready0 = smem_u32(&bars[2 * kOpMaxStages]);
    const unsigned drained0 = ready0 + 16;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kOpMaxStages; ++s) {
            mbar_init(full0 + 8 * s, 1);   // the copying thread's arrival and the bytes
            mbar_init(empty0 + 8 * s, 1);  // the MMA thread's commit
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(ready0 + 8 * b, 1);
            mbar_init(drained0 + 8 * b, kDrainWarps);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(2 * Np)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_slot;

    if (warp == kOpTmaWarp) {
        if (lane == 0 && nkb > 0) {
            int issued = 0;
            bool ok = true;
            for (int kb = 0; kb < nkb; ++kb) {
                const int o = kb % O;
                if (kb >= O && !mbar_wait_or_abort(empty0 + 8 * o, ((kb / O) - 1) & 1, &abort_flag)) {
                    ok = false;
                    break;
                }
                const unsigned st = sbase + o * stage_bytes;
                const int y = (kb0 + kb) * kKB;  // operand row of the k-block's first primary
                mbar_expect_tx(full0 + 8 * o, kb_bytes);
                for (int b = 0; b < nt; ++b)
                    for (int c = 0; c < nbox(b); ++c) {
                        const int x = sp.xb + kTT * b + 64 * c;  // a multiple of 64 columns
                        tma_load_2d(st + b * kOpBytes + c * kOpBox, &maps.hi, x, y, full0 + 8 * o);
                        tma_load_2d(st + (nt + b) * kOpBytes + c * kOpBox, &maps.lo, x, y, full0 + 8 * o);
                    }
                ++issued;
            }
            if (!ok && !abort_flag) {
                abort_flag = 1;
                atomicOr(a.status, kStatusTimeout);
            }
            if (abort_flag) {
                // this CTA's copies still in flight (the latest of every stage) land
                // before it exits (bounded)
                for (int kb = issued > O ? issued - O : 0; kb < issued; ++kb)
                    mbar_wait(full0 + 8 * (kb % O), (kb / O) & 1);
            }
        }
    } else if (warp == kOpMmaWarp) {
        if (lane == 0 && nkb > 0) {
            const unsigned idesc = make_idesc_mn(kTT, N);
            bool ok = true;
            for (int kb = 0; kb < nkb && ok; ++kb) {
                const int sub = kb / kSubKB, buf = sub & 1;
                const bool first = (kb % kSubKB) == 0;
                const bool last = (kb % kSubKB) == kSubKB - 1 || kb == nkb - 1;
                if (first && sub >= 2 && !mbar_wait(drained0 + 8 * buf, ((sub >> 1) - 1) & 1)) {
                    ok = false;
                    break;
                }
                const int o = kb % O;
                // error-path test: the first wait gives up at once, as if its bound had expired
                const bool landed = (kb == 0 && a.test_timeout)
                                        ? false
                                        : mbar_wait_or_abort(full0 + 8 * o, (kb / O) & 1, &abort_flag);
                if (!landed) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned st = sbase + o * stage_bytes;
                const unsigned H = st, Lo = st + nt * kOpBytes;  // hi and lo (A = their panel 0)
                const unsigned d = tmem + (unsigned)(buf * Np);
#pragma unroll
                for (int k = 0; k < kKB / 16; ++k) {
                    const unsigned off = k * 2048;  // 16 primaries = two groups of 8
                    mma_bf16(d, make_desc_mn(H + off), make_desc_mn(H + off), idesc, (first && k == 0) ? 0u : 1u);
                    mma_bf16(d, make_desc_mn(H + off), make_desc_mn(Lo + off), idesc, 1u);
                    mma_bf16(d, make_desc_mn(Lo + off), make_desc_mn(H + off), idesc, 1u);
                }
                mma_commit(empty0 + 8 * o);  // frees the stage when these MMAs have read it
                if (last) mma_commit(ready0 + 8 * buf);
            }
            if (!ok) {
                if (!abort_flag) {
                    abort_flag = 1;
                    atomicOr(a.status, kStatusTimeout);
                }
                mma_commit(ready0);
                mma_commit(ready0 + 8);
            }
        }
    } else if (warp < kDrainWarps) {
        drain_item(warp, lane, tmem, N, Np, nt, nsub, ready0, drained0, &abort_flag, a.tiles, sp, it, a.partials,
                   a.part_stride, a.status);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * Np)
                     : "memory");
}

__global__ void k_zero_pad(__nv_bfloat16* bop, int pitch, const int4* bcat) {
    const int4 c = bcat[blockIdx.x];
    const int64_t r0 = (int64_t)c.x + c.z, r1 = (int64_t)c.x + (int64_t)(c.z + kKB - 1) / kKB * kKB;
    const int64_t n = (r1 - r0) * 2 * pitch;  // hi and lo of every padding row
    unsigned short* h = reinterpret_cast<unsigned short*>(bop) + r0 * 2 * pitch;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) h[i] = 0;
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

// FP32 rows of A as a 2-D tensor: RL columns (inner) x rows, row pitch RLP
// floats; boxes of `cols` x kKB, no swizzle, zeros outside.
int make_map_a(CUtensorMap* m, const float* A, int RLP, int RL, int64_t rows, int cols) {
    auto fn = encode_fn();
    if (!fn) return -1;
    cuuint64_t dims[2] = {(cuuint64_t)RL, (cuuint64_t)(rows > 0 ? rows : 1)};
    cuuint64_t strides[1] = {(cuuint64_t)RLP * 4};
    cuuint32_t box[2] = {(cuuint32_t)cols, kKB};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

// bf16 operand rows as a 2-D tensor: pitch columns (inner) x rows, rows 2 pitch
// apart (hi and lo of a row side by side); boxes of 64 columns x kKB rows in the
// 128-byte swizzle, zeros outside.
int make_map_op(CUtensorMap* m, const __nv_bfloat16* B, int pitch, int64_t rows) {
    auto fn = encode_fn();
    if (!fn) return -1;
    cuuint64_t dims[2] = {(cuuint64_t)pitch, (cuuint64_t)(rows > 0 ? rows : 1)};
    cuuint64_t strides[1] = {(cuuint64_t)pitch * 4};
    cuuint32_t box[2] = {64, kKB};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(B), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

}  // namespace

int contract_tile_dim_tc() { return kTT; }

// Strips of the tile list (tiles in (m, row tile, column tile) order, column
// tiles from the diagonal): consecutive tiles of one row panel, two at a time.
int make_strips(const Tile* tiles, int ntiles, TcStrip* out, int max_strips) {
    int n = 0;
    int bm = -1, b0 = 0, bnext = 0;  // operand column of the current m block, and of the next
    for (int k = 0; k < ntiles;) {
        if (tiles[k].m != bm) {
            bm = tiles[k].m;
            b0 = bnext;
            bnext = b0 + (tiles[k].width + 63) / 64 * 64;
        }
        const bool pair = k + 1 < ntiles && tiles[k + 1].m == tiles[k].m && tiles[k + 1].r0 == tiles[k].r0 &&
                          tiles[k + 1].c0 == tiles[k].c0 + kTT;
        if (n >= max_strips) return -1;
        out[n].tile0 = k;
        out[n].ntile = pair ? 2 : 1;
        const int cols = tiles[k].cols + (pair ? tiles[k + 1].cols : 0);
        out[n].n = (cols + 15) / 16 * 16;  // kind::f16 with M = 128: N a multiple of 16, <= 256
        out[n].xrow = tiles[k].col0 + tiles[k].r0;
        out[n].xcol = tiles[k].col0 + tiles[k].c0;
        out[n].xb = b0 + tiles[k].c0;
        ++n;
        k += pair ? 2 : 1;
    }
    return n;
}

int contract_tc_kblock() { return kKB; }

int tc_operand_blocks(const Tile* tiles, int ntiles, int4* blk, int max_blk) {
    int bm = -1, nb = 0, bnext = 0;
    for (int k = 0; k < ntiles; ++k) {
        if (tiles[k].m == bm) continue;
        bm = tiles[k].m;
        if (bm >= max_blk) return -1;
        blk[bm] = make_int4(tiles[k].col0, tiles[k].width, bnext, 0);
        bnext += (tiles[k].width + 63) / 64 * 64;
        nb = bm + 1;
    }
    (void)nb;
    return bnext;
}

// Every CTA takes the same number of k-blocks: a strip's k-block costs about
// the same whatever its width (the per-k-block copies and hand-offs bound it),
// so a two-tile strip, with twice the operand panels, takes one segment per
// item and a one-tile strip two.
int plan_tc_items(const TcStrip* strips, int nstrips, int vmax, double slots, int* step) {
    double units = 0.0;  // items per virtual segment
    for (int s = 0; s < nstrips; ++s) {
        step[s] = strips[s].ntile == 2 ? 1 : 2;
        units += 1.0 / step[s];
    }
    if (units <= 0.0) units = 1.0;
    int V = 2 * (int)std::llround(slots / (2.0 * units));
    if (V > vmax) V = vmax;
    if (V < 2) V = 2;
    return V;
}

int launch_contract_tc(const float* A, int RLP, int RL, int64_t arows, const float* wrow, const int4* cats,
                       const Tile* tiles, const TcStrip* strips, const TcItem* items, int nitems,
                       const Segment* segs, double* partials, int part_stride, const int* negw, int* status,
                       cudaStream_t st, int test_timeout) {
    if (nitems <= 0) return 0;
    TcMaps m;
    for (int wi = 0; wi < kBoxes; ++wi)
        if (make_map_a(&m.m[wi], A, RLP, RL, arows, box_cols(wi)) != 0) return -2;
    const int smem = kBufBytes + 1024;
    if (cudaFuncSetAttribute(k_contract_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
        return -1;
    TcArgs a{A, RLP, wrow, cats, tiles, strips, items, segs, partials, part_stride, negw, status, test_timeout};
    k_contract_tc<<<(unsigned)nitems, kTcWarps * 32, smem, st>>>(m, a);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_contract_tc_op(const __nv_bfloat16* bop, int pitch, int64_t rows, const Tile* tiles,
                          const TcStrip* strips, const TcItem* items, int nitems, const Segment* segs,
                          double* partials, int part_stride, int* status, cudaStream_t st, int test_timeout) {
    if (nitems <= 0) return 0;
    if (pitch % 64 != 0) return -1;
    TcOpMaps m;
    if (make_map_op(&m.hi, bop, pitch, rows) != 0 || make_map_op(&m.lo, bop + pitch, pitch, rows) != 0) return -2;
    const int smem = kBufBytes + 1024;
    if (cudaFuncSetAttribute(k_contract_tc_op, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return -1;
    TcOpArgs a{tiles, strips, items, segs, partials, part_stride, status, test_timeout};
    k_contract_tc_op<<<(unsigned)nitems, kOpWarps * 32, smem, st>>>(m, a);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_zero_pad(__nv_bfloat16* bop, int pitch, const int4* bcat, int ncat, cudaStream_t st) {
    if (ncat <= 0) return 0;
    k_zero_pad<<<(unsigned)ncat, 256, 0, st>>>(bop, pitch, bcat);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace g3
