// Pair stage split in three kernels (forward): count, scan, accumulate.
//
// Paper: Algorithm 1 and Sec. 3.1 (neighbours within rmax, radial bin,
// rotation, harmonics, multipoles per shell), Sec. 3.3.1 (pre-binning: pairs
// of one primary collected per radial bin before their multipoles are
// computed) and Sec. 3.3.2 (one reduction of the per-lane partials per
// primary and bin instead of one per pair group).
//
//   k_count  -- per primary, the number of candidate secondaries in the
//               sphere's cell rows; the host turns ceil(candidates/32) + B
//               into exact, non-overlapping list offsets and into passes that
//               fit the list pool.
//   k_scan   -- per primary (one warp), streams the candidates of 32 cell rows
//               at a time, slot range by slot range, decides each pair's bin
//               exactly and compacts the accepted pairs into a staging ring in
//               shared memory; every 32 staged pairs are placed into per-bin
//               chunks of 32 entries (128 bytes, tagged with the bin) of this
//               primary.  Few registers: many warps hide the candidate loads.
//   k_accum  -- per primary (one warp), walks its chunks bin by bin: each
//               lane takes one pair of a chunk, evaluates Y_lm (FP32
//               recurrence, pair_common.cuh) into (lmax+1)^2 register
//               partials, and one warp butterfly per (primary, bin) reduces
//               them; the normalised row of multipoles goes to A.
//
// Compared with the fused kernel (pair.cu, G3PCF_OPT_PAIR_KERNELS = 1, kept as
// a cross-check), the accumulation runs without the scan's state in registers
// and reduces across lanes once per bin instead of once per bucket.  Plain,
// batched and graph-captured forwards, and the adjoint pair pass (k_adj), all
// walk these lists.
#include "pair_common.cuh"

namespace g3 {

namespace {

constexpr int kLWarps = 4;
constexpr int kLThreads = kLWarps * 32;
constexpr int kChunk = 32;      // pairs per list chunk
constexpr int kStage = 256;     // compaction stage of k_scan (entries)
constexpr int kTrip = 4;        // candidate sub-iterations per trip in k_scan
constexpr unsigned kNoPair = 0xffffffffu;  // padding entry of a list chunk (image code 31 is unused)

// Per-warp shared memory of k_scan: img[27] float4, pd[4] double,
// pcs[kMaxPieces] int4 (the slot ranges of a row batch: first, end, image
// code), stage[kStage + 32] int2 (accepted pairs: entry, bin; the last 32 are
// scratch), per-bin fill / open chunk / chunk count.
struct ScanSmem {
    float4* img;
    double* pd;
    int4* pcs;
    int2* stage;
    int* bfill;
    int* bcur;
    int* bnbc;
};
__host__ __device__ constexpr size_t scan_smem_per_warp(int) {
    return 27 * 16 + 4 * 8 + kMaxPieces * 16 + (kStage + 32) * 8 + 3 * 32 * 4;
}
__device__ __forceinline__ ScanSmem scan_smem(unsigned char* raw, int wid, int B) {
    unsigned char* b = raw + (size_t)wid * scan_smem_per_warp(B);
    ScanSmem S;
    S.img = reinterpret_cast<float4*>(b);
    S.pd = reinterpret_cast<double*>(b + 27 * 16);
    S.pcs = reinterpret_cast<int4*>(b + 27 * 16 + 32);
    S.stage = reinterpret_cast<int2*>(b + 27 * 16 + 32 + kMaxPieces * 16);
    S.bfill = reinterpret_cast<int*>(b + 27 * 16 + 32 + kMaxPieces * 16 + (kStage + 32) * 8);
    S.bcur = S.bfill + 32;
    S.bnbc = S.bcur + 32;
    return S;
}

__global__ void __launch_bounds__(kLThreads) k_count(ListArgs a) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const Grid& g = a.g;
    const int K = g.reach, W = 2 * K + 1, nrows = W * W;
    for (int q = a.qa + gw; q < a.qb; q += nw) {
        const int p = a.plist ? a.plist[q] : q;
        const float4 P0 = a.pts[p];
        const long long cat = (long long)(a.key[p] / (unsigned long long)g.cells_per_cat);
        const long long kbase = cat * g.cells_per_cat;
        const int cy = cell_of(P0.y, g), cz = cell_of(P0.z, g);
        long long sum = 0;
        for (int r = lane; r < nrows; r += 32) {
            int4 pm, p0, pp;
            row_pieces(r, W, K, cy, cz, P0, g, a.bins.slack, a.bins.rmax2f, kbase, a.cstart, pm, p0,
                       pp);
            sum += max(pm.y - pm.x, 0) + max(p0.y - p0.x, 0) + max(pp.y - pp.x, 0);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
        if (lane == 0) {
            a.need[q] = (int)((sum + kChunk - 1) / kChunk) + a.bins.nbins;
            atomicAdd(a.ncand, (unsigned long long)sum);
        }
    }
}

__global__ void __launch_bounds__(kLThreads, 7) k_scan(ListArgs a) {
    extern __shared__ __align__(16) unsigned char ls_raw[];
    __shared__ double s_e2[kMaxBins + 1];
    __shared__ float2 s_dec[kMaxBins];
    __shared__ signed char s_tab[kBinTable + 2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int B = a.bins.nbins;
    for (int k = threadIdx.x; k <= B; k += blockDim.x) {
        s_e2[k] = a.bins.e2[k];
        if (k < B)
            s_dec[k] = make_float2(a.bins.e2f[k] + a.bins.guard[k], a.bins.e2f[k + 1] - a.bins.guard[k + 1]);
    }
    for (int k = threadIdx.x; k < kBinTable + 2; k += blockDim.x) s_tab[k] = a.bintab[k];
    __syncthreads();
    const ScanSmem S = scan_smem(ls_raw, wid, B);
    const unsigned lt = lanemask_lt();
    const Grid& g = a.g;
    const float Lb = g.box;
    const bool exact_inputs = (a.pts64 == nullptr);
    const float hi_rej = a.bins.hi_rej, lo_rej = a.bins.lo_rej, guard0 = a.bins.guard[0];
    const float rminf = a.bins.rmin, invw = a.bins.invw, tscale = a.bin_tscale;
    const float slack = a.bins.slack, rmax2 = a.bins.rmax2f;
    const int K = g.reach, W = 2 * K + 1, nrows = W * W;
    unsigned long long my_total = 0;
    long long cur_cat = -1;

    const int qa = a.qrange ? a.qrange[0] : a.qa, qb = a.qrange ? a.qrange[1] : a.qb;
    for (;;) {
        int q = 0;
        if (lane == 0) q = qa + atomicAdd(a.queue, 1);
        q = __shfl_sync(kFull, q, 0);
        if (q >= qb) break;
        if (a.base[q] < 0) {  // no room in the planned passes (flagged by the planner)
            if (lane == 0) a.nchunks[q] = 0;
            continue;
        }
        const int p = a.plist ? a.plist[q] : q;
        const long long cat = (long long)(a.key[p] / (unsigned long long)g.cells_per_cat);
        if (cat != cur_cat) {
            if (cur_cat >= 0 && lane < B && my_total) atomicAdd(&a.counts[cur_cat * B + lane], my_total);
            my_total = 0;
            cur_cat = cat;
        }
        const long long kbase = cat * g.cells_per_cat;
        const float4 P0 = a.pts[p];
        if (lane < 27) {
            const int sx = lane % 3 - 1, sy = (lane / 3) % 3 - 1, sz = lane / 9 - 1;
            S.img[lane] = make_float4(P0.x - sx * Lb, P0.y - sy * Lb, P0.z - sz * Lb, 0.f);
        }
        if (lane < 3) {
            const float pv = lane == 0 ? P0.x : (lane == 1 ? P0.y : P0.z);
            S.pd[lane] = a.pts64 ? a.pts64[3 * (int64_t)p + lane] : (double)pv;
        }
        __syncwarp();
        const int cy = cell_of(P0.y, g), cz = cell_of(P0.z, g);
        int* const pool = a.chunks + (int64_t)a.base[q] * kChunk;  // this primary's chunks
        int* const ptag = a.tag + a.base[q];
        int* const pord = a.ord + a.base[q];
        const int cap_ch = a.need[q];  // chunks reserved for it
        int nch = 0;                   // chunks opened so far (warp-uniform)
        // per-bin state in shared memory: fill of the open chunk (kChunk: none
        // open), its index, chunks opened so far
        if (lane < B) {
            S.bfill[lane] = kChunk;
            S.bcur[lane] = 0;
            S.bnbc[lane] = 0;
        }
        __syncwarp();

        // Place one accepted pair per lane (bin < 0: none) into the open chunk of
        // its bin, opening a new chunk where a bin's chunk fills.  Lanes with the
        // same bin form a group (match); its lowest lane updates the bin state.
        auto place = [&](int entry, int bin) {
            const bool v = bin >= 0;
            const unsigned mine = __match_any_sync(kFull, v ? bin : 63);
            const int rank = __popc(mine & lt);
            const int cnt = __popc(mine);
            const int bs = v ? bin : 0;
            const int fill = S.bfill[bs], cur = S.bcur[bs];
            const bool grow = v && fill + cnt > kChunk;  // at most one new chunk per call
            const bool lead = v && rank == 0;
            const unsigned gm = __ballot_sync(kFull, grow && rank == 0);
            const unsigned below_leader = mine & (0u - mine);  // lowest lane of the group
            const int nnew = nch + __popc(gm & (below_leader - 1u));
            nch += __popc(gm);
            const int pos = fill + rank;
            const int c = pos < kChunk ? cur : nnew;
            if (v && c < cap_ch) pool[(int64_t)c * kChunk + (pos & (kChunk - 1))] = entry;
            __syncwarp();
            if (lead) {
                S.bfill[bin] = grow ? fill + cnt - kChunk : fill + cnt;
                if (grow) {
                    const int nb = S.bnbc[bin];
                    if (nnew < cap_ch)
                        ptag[nnew] = (nb << 5) | bin;  // (rank among the bin's chunks, bin)
                    else
                        atomicOr(a.status, kStatusOverflow);
                    S.bnbc[bin] = nb + 1;
                    S.bcur[bin] = nnew;
                }
            }
            __syncwarp();
        };
        // accepted pairs are first compacted into stage (warp-uniform head/count)
        int shead = 0, scnt = 0;
        auto drain = [&]() {
            while (scnt >= kChunk) {
                __syncwarp();
                const int2 v = S.stage[(shead + lane) & (kStage - 1)];
                shead = (shead + kChunk) & (kStage - 1);
                scnt -= kChunk;
                __syncwarp();
                place(v.x, v.y);
            }
        };

        // candidates: batches of 32 cell rows -> slot ranges (pieces) -> up to
        // kTrip x 32 slots per trip, all loads of a trip in flight together
        for (int rb = 0; rb < nrows; rb += 32) {
            int4 pm = make_int4(0, 0, 0, 0), p0 = pm, pp = pm;
            const int r = rb + lane;
            if (r < nrows) row_pieces(r, W, K, cy, cz, P0, g, slack, rmax2, kbase, a.cstart, pm, p0, pp);
            const int npc = (pm.y > pm.x) + (p0.y > p0.x) + (pp.y > pp.x);
            int incl = npc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            const int npcs = __shfl_sync(kFull, incl, 31);
            __syncwarp();
            {
                int k = incl - npc;
                if (pm.y > pm.x) S.pcs[k++] = pm;
                if (p0.y > p0.x) S.pcs[k++] = p0;
                if (pp.y > pp.x) S.pcs[k++] = pp;
            }
            __syncwarp();
            for (int pi = 0; pi < npcs; ++pi) {
                const int4 pc = S.pcs[pi];
                const float4 o = S.img[pc.z];
                const unsigned codebits = (unsigned)pc.z << kIdxBits;
                for (int j0 = pc.x; j0 < pc.y; j0 += kTrip * kChunk) {
                    const int nu = (pc.y - j0 + kChunk - 1) / kChunk;  // sub-iterations with slots
                    // slots past the piece read as a far point (r^2 ~ 1e36: no pair)
                    float4 qv[kTrip];
#pragma unroll
                    for (int u = 0; u < kTrip; ++u) {
                        const int j = j0 + u * kChunk + lane;
                        qv[u] = make_float4(o.x + 1e18f, o.y, o.z, 0.f);
                        if (j < pc.y) qv[u] = __ldg(a.pts + j);
                    }
                    int bn[kTrip];
                    bool chk = false;
#pragma unroll
                    for (int u = 0; u < kTrip; ++u) {
                        const float dx = qv[u].x - o.x, dy = qv[u].y - o.y, dz = qv[u].z - o.z;
                        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        bn[u] = bin_fast(r2, tscale, s_tab);
                        chk |= bn[u] < -1;
                    }
                    if (__any_sync(kFull, chk)) {
#pragma unroll
                        for (int u = 0; u < kTrip; ++u) {
                            if (bn[u] == -3) {
                                const int j = j0 + u * kChunk + lane;
                                const float dx = qv[u].x - o.x, dy = qv[u].y - o.y, dz = qv[u].z - o.z;
                                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                                bn[u] = bin_slow(r2, lo_rej, hi_rej, guard0, s_dec, rminf, invw, B, exact_inputs,
                                                 pc.z, a.pts, a.pts64, j, S.pd, g.boxd, g.periodic, s_e2);
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kTrip; ++u) {
                        if (u < nu) {
                            // accepted lanes append in lane order; the others write a scratch slot
                            const bool acc = bn[u] >= 0;
                            const unsigned vm = __ballot_sync(kFull, acc);
                            const int at = acc ? ((shead + scnt + __popc(vm & lt)) & (kStage - 1)) : kStage + lane;
                            S.stage[at] = make_int2((int)((unsigned)(j0 + u * kChunk + lane) | codebits), bn[u]);
                            scnt += __popc(vm);
                        }
                    }
                    drain();
                }
            }
            __syncwarp();
        }
        if (scnt > 0) {  // the last accepted pairs (fewer than 32)
            __syncwarp();
            const int2 v = lane < scnt ? S.stage[(shead + lane) & (kStage - 1)] : make_int2(0, -1);
            __syncwarp();
            place(v.x, v.y);
        }
        // the bin state back in lane b
        int cfill = kChunk, ccur = 0, nbc = 0;
        if (lane < B) {
            cfill = S.bfill[lane];
            ccur = S.bcur[lane];
            nbc = S.bnbc[lane];
        }
        const unsigned padd = nbc > 0 ? (unsigned)((nbc - 1) * kChunk + cfill) : 0u;  // pairs of bin lane
        // pad the open chunks behind their last entry
        unsigned pmask = __ballot_sync(kFull, lane < B && cfill < kChunk);
        while (pmask) {
            const int b = __ffs(pmask) - 1;
            pmask &= pmask - 1;
            const int c = __shfl_sync(kFull, ccur, b);
            const int f = __shfl_sync(kFull, cfill, b);
            if (lane >= f && c < cap_ch) pool[(int64_t)c * kChunk + lane] = (int)kNoPair;
        }
        // list the chunks grouped by bin (stable): position = chunks of the
        // lower bins + rank inside the bin
        {
            int off = nbc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, off, o);
                if (lane >= o) off += y;
            }
            off -= nbc;
            const int nlist = nch < cap_ch ? nch : cap_ch;
            for (int c0 = 0; c0 < nlist; c0 += 32) {
                const int c = c0 + lane;
                const int t = c < nlist ? ptag[c] : 0;
                const int b = t & 31;
                const int pos = __shfl_sync(kFull, off, b) + (t >> 5);
                if (c < nlist && pos < cap_ch) pord[pos] = c | (b << 26);
            }
        }
        if (lane == 0) a.nchunks[q] = nch < cap_ch ? nch : cap_ch;
        my_total += padd;
        __syncwarp();
    }
    if (cur_cat >= 0 && lane < B && my_total) atomicAdd(&a.counts[cur_cat * B + lane], my_total);
}

__global__ void k_plan_init(int* passq, int npass, int qb) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p <= npass; p += gridDim.x * blockDim.x) passq[p] = qb;
}

// Exclusive prefix sums of need[qa..qb) in 64 bits (the chunks of a large
// batch exceed 2^31): per-block sums, a scan of those, then the blocks.
constexpr int kScan64 = 1024;
__device__ long long block_scan64(long long v, long long* sh, long long& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        long long t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(kFull, t, o);
            if (lane >= o) t += y;
        }
        sh[lane] = t;
    }
    __syncthreads();
    const long long pre = (wid > 0 ? sh[wid - 1] : 0) + x - v;
    total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return pre;
}
__global__ void k_need_sums(const int* need, int64_t n, long long* bsum) {
    __shared__ long long sh[32];
    const int64_t i = blockIdx.x * (int64_t)kScan64 + threadIdx.x;
    long long tot;
    block_scan64(i < n ? need[i] : 0, sh, tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}
__global__ void k_need_top(long long* bsum, int nb) {
    __shared__ long long sh[32];
    long long carry = 0;
    for (int b0 = 0; b0 < nb; b0 += kScan64) {
        const int i = b0 + threadIdx.x;
        long long tot;
        const long long pre = block_scan64(i < nb ? bsum[i] : 0, sh, tot);
        if (i < nb) bsum[i] = carry + pre;
        carry += tot;
    }
}
__global__ void k_need_final(const int* need, int64_t n, const long long* bsum, long long* out) {
    __shared__ long long sh[32];
    const int64_t i = blockIdx.x * (int64_t)kScan64 + threadIdx.x;
    long long tot;
    const long long pre = block_scan64(i < n ? need[i] : 0, sh, tot);
    if (i < n) out[i] = bsum[blockIdx.x] + pre;
}

__global__ void k_plan(const int* need, const long long* gbase, int qa, int qb, long long stride, int slack,
                       int npass, int* base, int* passq, int* status) {
    for (int q = qa + blockIdx.x * blockDim.x + threadIdx.x; q < qb; q += gridDim.x * blockDim.x) {
        const long long gb = gbase[q - qa];
        const long long pql = gb / stride;
        const int pq = pql < npass ? (int)pql : npass;
        const bool ok = pq < npass && need[q] <= slack;
        base[q] = ok ? (int)(gb - pql * stride) : -1;
        if (!ok) atomicOr(status, kStatusOverflow);
        // first primary of every pass that starts here
        const long long pprevl = q == qa ? -1 : gbase[q - 1 - qa] / stride;
        const int pprev = pprevl < npass ? (int)pprevl : npass;
        for (int pp = pprev + 1; pp <= pq && pp < npass; ++pp) passq[pp] = q;
    }
}

// Asynchronous global -> shared copies (one per lane) and their groups.
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
// 16 bytes, or zeros without reading when !valid
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Image `code` of the primary (its position minus the code's box shift) as an
// FP32 head img[code] and tail img[27 + code] of the FP64 value (the primary's
// FP64 position when the input is FP64): the separation (q - head) - tail is
// then as exact as FP32 allows even where the shift is a whole box side.
__device__ __forceinline__ void set_image(float4* img, int code, const float4& P0, const double* pts64, int p,
                                          double boxd) {
    const int sx = code % 3 - 1, sy = (code / 3) % 3 - 1, sz = code / 9 - 1;
    double x = P0.x, y = P0.y, z = P0.z;
    if (pts64) {
        x = pts64[3 * (int64_t)p];
        y = pts64[3 * (int64_t)p + 1];
        z = pts64[3 * (int64_t)p + 2];
    }
    x -= sx * boxd;
    y -= sy * boxd;
    z -= sz * boxd;
    const float hx = (float)x, hy = (float)y, hz = (float)z;
    img[code] = make_float4(hx, hy, hz, 0.f);
    img[27 + code] = make_float4((float)(x - hx), (float)(y - hy), (float)(z - hz), 0.f);
}

// Separation of one list entry from the primary (image img[code]), rotated
// to the primary's line of sight in radial mode, as a unit vector and weight.
template <bool EXACT>
__device__ __forceinline__ void pair_dir(const float4& q, unsigned e, const float4* img, const float* R,
                                         int radial, float& z, float& ux, float& uy, float& w) {
    float dx = 1.f, dy = 0.f, dz = 0.f;
    w = 0.f;
    if (e != kNoPair) {
        const float4 o = img[e >> kIdxBits];
        dx = q.x - o.x;
        dy = q.y - o.y;
        dz = q.z - o.z;
        if constexpr (EXACT) {  // the tail of the image (nonzero across a box face)
            const float4 ol = img[27 + (e >> kIdxBits)];
            dx -= ol.x;
            dy -= ol.y;
            dz -= ol.z;
        }
        w = q.w;
        if (radial) {
            const float rx = fmaf(R[0], dx, fmaf(R[1], dy, R[2] * dz));
            const float ry = fmaf(R[3], dx, fmaf(R[4], dy, R[5] * dz));
            const float rz = fmaf(R[6], dx, fmaf(R[7], dy, R[8] * dz));
            dx = rx;
            dy = ry;
            dz = rz;
        }
    }
    const float rinv = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    z = dz * rinv;
    ux = dx * rinv;
    uy = dy * rinv;
}

// Reduce the Chebyshev-form partials over the warp into res_b (accumulator
// slot layout: m = 0 slot k; m >= 1 slot acc_base(m) + 2k + part).
template <int L>
__device__ __forceinline__ void reduce_cheb(float (&acc0)[L + 1], float2 (&accc)[Cheb<L>::NC > 0 ? Cheb<L>::NC : 1],
                                            int lane, float* res_b) {
    constexpr int NR = Shape<L>::NR;
    float acc[NR];
    static_for<0, L + 1>([&](auto kc) { acc[decltype(kc)::value] = acc0[decltype(kc)::value]; });
    static_for<0, Cheb<L>::NC>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        acc[L + 1 + 2 * i] = accc[i].x;
        acc[L + 2 + 2 * i] = accc[i].y;
    });
    butterfly_add<L>(acc, lane, res_b);
}

// Per-warp shared memory of k_accum / k_adj: img[27] float4 and its low parts
// imglo[27] float4 (below), R[16] float, point ring [kPtRing][32] float4, entry
// ring [kEntRing][32] uint, res[B][NRP] float.
constexpr int kImgBytes = 2 * 27 * 16;
constexpr int kEntRing = 8;
constexpr int kPtRing = 4;
__host__ __device__ constexpr size_t accum_smem_per_warp(int B, int NRP) {
    return (size_t)B * NRP * 4 + kImgBytes + 64 + kEntRing * 32 * 4 + kPtRing * 32 * 16;
}

// Column col of a row of A from the per-bin Chebyshev sums res: the
// Legendre-form connection times K_lm.
__device__ __forceinline__ float connect(const ListArgs& a, const float* res, int col) {
    const int4 cv = __ldg(a.colconv + col);
    const float* cf = a.colcoef + cv.w;
    float v = 0.f;
    for (int k = 0; k < cv.z; ++k) v = fmaf(__ldg(cf + k), res[cv.x + cv.y * k], v);
    return v;
}

// The row of A of one primary, and, when asked for, the tensor-core operands:
// sqrt(w) times the row split into bf16 hi and lo (the operations of the
// contraction's converter warps) at the row's padded position inside its
// catalog, m block by m block.  Out of line, so that the register allocation of
// the pair loop does not see it.
__device__ __noinline__ void emit_row(const ListArgs& a, const float* res, int row, int p, float w, int lane) {
    float* Arow = a.A + (int64_t)row * a.RLP;
    if (!a.bop) {
        // two columns per lane, their coefficient chains interleaved: the warp runs
        // this tail with fewer FMA warps beside it, so its latency is what counts
        // (337 ms per forward against 341 ms one column at a time; four: 340 ms)
        for (int c0 = lane; c0 < a.RL; c0 += 64) {
            const int c1 = c0 + 32;
            const int4 cv0 = __ldg(a.colconv + c0);
            const int4 cv1 = c1 < a.RL ? __ldg(a.colconv + c1) : make_int4(0, 0, 0, 0);
            const float* cf0 = a.colcoef + cv0.w;
            const float* cf1 = a.colcoef + cv1.w;
            float v0 = 0.f, v1 = 0.f;
            const int n = cv0.z > cv1.z ? cv0.z : cv1.z;
            for (int k = 0; k < n; ++k) {
                if (k < cv0.z) v0 = fmaf(__ldg(cf0 + k), res[cv0.x + cv0.y * k], v0);
                if (k < cv1.z) v1 = fmaf(__ldg(cf1 + k), res[cv1.x + cv1.y * k], v1);
            }
            Arow[c0] = v0;
            if (c1 < a.RL) Arow[c1] = v1;
        }
        return;
    }
    const int4 bc = __ldg(a.bcat + (a.nbcat == 1 ? 0 : (int)(a.key[p] / (unsigned long long)a.g.cells_per_cat)));
    __nv_bfloat16* Bh = a.bop + ((int64_t)bc.x + (row - bc.y)) * 2 * a.bop_pitch;
    __nv_bfloat16* Bl = Bh + a.bop_pitch;
    const float sw = sqrtf(w);
    // one column per lane, as the FP32 rows (consecutive lanes read the bins of
    // one (l, m) in turn from res), the operand columns of an m block contiguous
    for (int m = 0; m < a.nblk; ++m) {
        const int4 bb = __ldg(a.bblk + m);  // {first A column, width, first operand column, 0}
        for (int j = lane; j < bb.y; j += 32) {
            const int col = bb.x + j;
            const float v = connect(a, res, col);
            if (!a.skip_a) Arow[col] = v;
            const float y = __fmul_rn(v, sw);
            const __nv_bfloat16 h = __float2bfloat16_rn(y);
            Bh[bb.z + j] = h;
            Bl[bb.z + j] = __float2bfloat16_rn(__fsub_rn(y, __bfloat162float(h)));
        }
    }
}

template <int L, bool EXACT>
__global__ void __launch_bounds__(kLThreads, 3) k_accum(ListArgs a) {
    constexpr int NRP = Shape<L>::NRP;
    extern __shared__ __align__(16) unsigned char la_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int B = a.bins.nbins;
    unsigned char* base = la_raw + (size_t)wid * accum_smem_per_warp(B, NRP);
    float4* img = reinterpret_cast<float4*>(base);
    float* Rs = reinterpret_cast<float*>(base + kImgBytes);
    float4* pring = reinterpret_cast<float4*>(base + kImgBytes + 64);
    unsigned* ering = reinterpret_cast<unsigned*>(base + kImgBytes + 64 + kPtRing * 32 * 16);
    float* res = reinterpret_cast<float*>(base + kImgBytes + 64 + kPtRing * 32 * 16 + kEntRing * 32 * 4);
    const Grid& g = a.g;
    const int qa = a.qrange ? a.qrange[0] : a.qa, qb = a.qrange ? a.qrange[1] : a.qb;
    for (;;) {
        int q = 0;
        if (lane == 0) q = qa + atomicAdd(a.queue, 1);
        q = __shfl_sync(kFull, q, 0);
        if (q >= qb) break;
        const int p = a.plist ? a.plist[q] : q;
        const float4 P0 = a.pts[p];
        if (lane < 27) set_image(img, lane, P0, a.pts64, p, g.boxd);
        if (lane < 9) {
            double x0 = P0.x, x1 = P0.y, x2 = P0.z;
            if (a.pts64) {
                x0 = a.pts64[3 * (int64_t)p];
                x1 = a.pts64[3 * (int64_t)p + 1];
                x2 = a.pts64[3 * (int64_t)p + 2];
            }
            Rs[lane] = g.radial ? los_rotation_entry(lane, x0, x1, x2, g.boxd)
                                : ((lane % 4 == 0) ? 1.f : 0.f);
        }
        const int cb = a.base[q] < 0 ? 0 : a.base[q];
        const int nch = a.nchunks[q];
        const int* chunks = a.chunks + (int64_t)cb * kChunk;
        const int* ordp = a.ord + cb;
        for (int k = lane; k < B * NRP; k += 32) res[k] = 0.f;
        __syncwarp();
        if (nch > 0) {
            // List slot i = chunk (low 26 bits) | bin << 26.  Copies in flight
            // (cp.async groups): entries up to slot i+4, points up to slot i+2.
            auto ent_async = [&](int i, unsigned o) {
                cp_async4(ering + (i & (kEntRing - 1)) * 32 + lane,
                          chunks + (int64_t)(o & 0x3ffffffu) * kChunk + lane);
            };
            auto pt_async = [&](int i) {
                const unsigned e = ering[(i & (kEntRing - 1)) * 32 + lane];
                const bool v = e != kNoPair;
                cp_async16(pring + (i & (kPtRing - 1)) * 32 + lane, a.pts + (v ? (e & kIdxMask) : 0u), v);
            };
            auto slot = [&](int i) -> unsigned { return i < nch ? (unsigned)__ldg(ordp + i) : 0u; };
            unsigned o0 = slot(0), o1 = slot(1), o2 = slot(2), o3 = slot(3);
            ent_async(0, o0);
            if (nch > 1) ent_async(1, o1);
            cp_async_commit();
            cp_async_wait<0>();
            pt_async(0);
            if (nch > 2) ent_async(2, o2);
            cp_async_commit();
            if (nch > 1) pt_async(1);
            if (nch > 3) ent_async(3, o3);
            cp_async_commit();
            // slot words of i .. i+3 in registers, i+4 .. i+6 loading
            unsigned s4 = slot(4), s5 = slot(5), s6 = slot(6);
            unsigned sA = o0, sB = o1, sC = o2, sD = o3;
            constexpr int NC = Cheb<L>::NC > 0 ? Cheb<L>::NC : 1;
            float acc0[L + 1];
            float2 accc[NC];
            auto clear = [&]() {
                static_for<0, L + 1>([&](auto kc) { acc0[decltype(kc)::value] = 0.f; });
                static_for<0, NC>([&](auto ic) { accc[decltype(ic)::value] = make_float2(0.f, 0.f); });
            };
            clear();
            int curb = (int)(sA >> 26);
            for (int i = 0; i < nch; ++i) {
                cp_async_wait<1>();  // entries of i+2 and points of i have landed
                if (i + 2 < nch) pt_async(i + 2);
                if (i + 4 < nch) ent_async(i + 4, s4);
                cp_async_commit();
                const unsigned s7 = slot(i + 7);
                const int bA = (int)(sA >> 26);
                if (bA != curb) {  // the bin changes: reduce the partials of the last one
                    reduce_cheb<L>(acc0, accc, lane, res + curb * NRP);
                    clear();
                    curb = bA;
                }
                {
                    const unsigned e = ering[(i & (kEntRing - 1)) * 32 + lane];
                    const float4 qv = pring[(i & (kPtRing - 1)) * 32 + lane];
                    float z, ux, uy, w;
                    pair_dir<EXACT>(qv, e, img, Rs, g.radial, z, ux, uy, w);
                    accum_pair_cheb<L>(acc0, accc, z, ux, uy, w);
                }
                sA = sB;
                sB = sC;
                sC = sD;
                sD = s4;
                s4 = s5;
                s5 = s6;
                s6 = s7;
            }
            cp_async_wait<0>();
            reduce_cheb<L>(acc0, accc, lane, res + curb * NRP);
        }
        __syncwarp();
        const int row = a.chunked ? q - a.q0 : a.orig[p];
        emit_row(a, res, row, p, P0.w, lane);
        if (lane == 0) a.wrow[row] = P0.w;
        __syncwarp();
    }
}

// Adjoint pair pass over the pair lists (the derivative of Sec. 3.1's a_lm
// with the pair set and bins held fixed).  Per primary i and bin b the adjoint
// multipoles H_lm = w_i K_lm V_i (V = M A, slot layout) are carried to the
// Chebyshev form, G_{m,k} = sum_l c^(m)_{l-m,k} H_lm (the transpose of the
// forward's connection), so that for a pair with unit separation (x, y, z)
//     F = sum_{m,k} Re(conj(G_{m,k}) T_k(z) (x + iy)^m)
// with dF/dz through T_k' = k U_{k-1} and dF/dx, dF/dy through (x + iy)^m.
// Secondary j receives dL/dw_j += 2F and dL/dpos_j += g, primary i gets -g,
// g = (2 w_j / r)(grad F - (grad F . d) d) (FP64 atomics; the primary's share
// is summed per lane and reduced once).
template <int L>
__global__ void __launch_bounds__(kLThreads) k_adj(ListArgs a) {
    constexpr int NR = Shape<L>::NR, NRP = Shape<L>::NRP;
    extern __shared__ __align__(16) unsigned char la_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int B = a.bins.nbins;
    unsigned char* base = la_raw + (size_t)wid * accum_smem_per_warp(B, NRP);
    float4* img = reinterpret_cast<float4*>(base);
    float4* pring = reinterpret_cast<float4*>(base + kImgBytes + 64);
    unsigned* ering = reinterpret_cast<unsigned*>(base + kImgBytes + 64 + kPtRing * 32 * 16);
    float* G = reinterpret_cast<float*>(base + kImgBytes + 64 + kPtRing * 32 * 16 + kEntRing * 32 * 4);
    const Grid& g = a.g;
    const int qa = a.qrange ? a.qrange[0] : a.qa, qb = a.qrange ? a.qrange[1] : a.qb;
    for (;;) {
        int q = 0;
        if (lane == 0) q = qa + atomicAdd(a.queue, 1);
        q = __shfl_sync(kFull, q, 0);
        if (q >= qb) break;
        const int p = a.plist ? a.plist[q] : q;
        const float4 P0 = a.pts[p];
        if (lane < 27) set_image(img, lane, P0, a.pts64, p, g.boxd);
        const int row = a.orig[p];
        const float* Vrow = a.V + (int64_t)(a.chunked ? q - a.q0 : row) * a.RLP;
        for (int idx = lane; idx < B * NR; idx += 32) {
            const int b = idx / NR, sl = idx - b * NR;
            const int4 cv = __ldg(a.slotconv + sl);
            float v = 0.f;
            for (int t = 0; t < cv.z; ++t) v = fmaf(__ldg(a.slotcoef + cv.w + t), __ldg(Vrow + cv.x + b + t * cv.y), v);
            G[b * NRP + sl] = P0.w * v;
        }
        const int cb = a.base[q] < 0 ? 0 : a.base[q];
        const int nch = a.nchunks[q];
        const int* chunks = a.chunks + (int64_t)cb * kChunk;
        const int* ordp = a.ord + cb;
        __syncwarp();
        double di0 = 0.0, di1 = 0.0, di2 = 0.0;  // -dL/dpos_i, this lane's share
        if (nch > 0) {
            auto ent_async = [&](int i, unsigned o) {
                cp_async4(ering + (i & (kEntRing - 1)) * 32 + lane,
                          chunks + (int64_t)(o & 0x3ffffffu) * kChunk + lane);
            };
            auto pt_async = [&](int i) {
                const unsigned e = ering[(i & (kEntRing - 1)) * 32 + lane];
                const bool v = e != kNoPair;
                cp_async16(pring + (i & (kPtRing - 1)) * 32 + lane, a.pts + (v ? (e & kIdxMask) : 0u), v);
            };
            auto slot = [&](int i) -> unsigned { return i < nch ? (unsigned)__ldg(ordp + i) : 0u; };
            unsigned o0 = slot(0), o1 = slot(1), o2 = slot(2), o3 = slot(3);
            ent_async(0, o0);
            if (nch > 1) ent_async(1, o1);
            cp_async_commit();
            cp_async_wait<0>();
            pt_async(0);
            if (nch > 2) ent_async(2, o2);
            cp_async_commit();
            if (nch > 1) pt_async(1);
            if (nch > 3) ent_async(3, o3);
            cp_async_commit();
            unsigned s4 = slot(4), s5 = slot(5), s6 = slot(6);
            unsigned sA = o0, sB = o1, sC = o2, sD = o3;
            float pix = 0.f, piy = 0.f, piz = 0.f;
            int curb = (int)(sA >> 26);
            for (int i = 0; i < nch; ++i) {
                cp_async_wait<1>();
                if (i + 2 < nch) pt_async(i + 2);
                if (i + 4 < nch) ent_async(i + 4, s4);
                cp_async_commit();
                const unsigned s7 = slot(i + 7);
                const int bA = (int)(sA >> 26);
                if (bA != curb) {
                    di0 -= pix;
                    di1 -= piy;
                    di2 -= piz;
                    pix = piy = piz = 0.f;
                    curb = bA;
                }
                const unsigned e = ering[(i & (kEntRing - 1)) * 32 + lane];
                if (e != kNoPair) {
                    const float4 qv = pring[(i & (kPtRing - 1)) * 32 + lane];
                    const float4 o = img[e >> kIdxBits], ol = img[27 + (e >> kIdxBits)];
                    const int jj = __ldg(a.orig + (e & kIdxMask));
                    const float dx = (qv.x - o.x) - ol.x, dy = (qv.y - o.y) - ol.y, dz = (qv.z - o.z) - ol.z;
                    const float rinv = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                    const float z = dz * rinv, ux = dx * rinv, uy = dy * rinv;
                    const float* Gb = G + bA * NRP;
                    // T_k(z) and T_k'(z) = k U_{k-1}(z)
                    float T[L + 1], D[L + 1];
                    T[0] = 1.f;
                    D[0] = 0.f;
                    if constexpr (L >= 1) {
                        T[1] = z;
                        D[1] = 1.f;
                        const float z2 = z + z;
                        float u0 = 1.f, u1 = z2;  // U_0, U_1
                        static_for<2, L + 1>([&](auto kc) {
                            constexpr int k = decltype(kc)::value;
                            T[k] = fmaf(z2, T[k - 1], -T[k - 2]);
                            D[k] = (float)k * u1;  // k U_{k-1}
                            const float u2 = fmaf(z2, u1, -u0);
                            u0 = u1;
                            u1 = u2;
                        });
                    }
                    float F = 0.f, Fz = 0.f, Fx = 0.f, Fy = 0.f;
                    static_for<0, L + 1>([&](auto kc) {
                        constexpr int k = decltype(kc)::value;
                        const float gk = Gb[k];
                        F = fmaf(gk, T[k], F);
                        Fz = fmaf(gk, D[k], Fz);
                    });
                    float pr = 1.f, pim = 0.f;  // (x + iy)^(m-1)
                    static_for<1, L + 1>([&](auto mc) {
                        constexpr int m = decltype(mc)::value;
                        constexpr int b0 = acc_base(L, m);
                        float2 gm = make_float2(0.f, 0.f), gz = make_float2(0.f, 0.f);
                        static_for<0, L - m + 1>([&](auto kc) {
                            constexpr int k = decltype(kc)::value;
                            const float2 gg = *reinterpret_cast<const float2*>(Gb + b0 + 2 * k);
                            gm = __ffma2_rn(make_float2(T[k], T[k]), gg, gm);
                            gz = __ffma2_rn(make_float2(D[k], D[k]), gg, gz);
                        });
                        const float ur = fmaf(pr, ux, -pim * uy), ui = fmaf(pr, uy, pim * ux);  // (x+iy)^m
                        F = fmaf(gm.x, ur, fmaf(gm.y, ui, F));
                        Fz = fmaf(gz.x, ur, fmaf(gz.y, ui, Fz));
                        Fx = fmaf((float)m, fmaf(gm.x, pr, gm.y * pim), Fx);
                        Fy = fmaf((float)m, fmaf(gm.y, pr, -gm.x * pim), Fy);
                        pr = ur;
                        pim = ui;
                    });
                    const float gdr = fmaf(Fx, ux, fmaf(Fy, uy, Fz * z));
                    const float sc = 2.f * qv.w * rinv;
                    const float gx = sc * fmaf(-gdr, ux, Fx), gy = sc * fmaf(-gdr, uy, Fy),
                                gz3 = sc * fmaf(-gdr, z, Fz);
                    atomicAdd(a.dw + jj, f2d_exact(2.f * F));
                    atomicAdd(a.dpos + 3 * (int64_t)jj, f2d_exact(gx));
                    atomicAdd(a.dpos + 3 * (int64_t)jj + 1, f2d_exact(gy));
                    atomicAdd(a.dpos + 3 * (int64_t)jj + 2, f2d_exact(gz3));
                    pix += gx;
                    piy += gy;
                    piz += gz3;
                }
                sA = sB;
                sB = sC;
                sC = sD;
                sD = s4;
                s4 = s5;
                s5 = s6;
                s6 = s7;
            }
            cp_async_wait<0>();
            di0 -= pix;
            di1 -= piy;
            di2 -= piz;
        }
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

template <int L>
int launch_adj_t(const ListArgs& a, int nsm, cudaStream_t st) {
    const size_t smem = accum_smem_per_warp(a.bins.nbins, Shape<L>::NRP) * kLWarps;
    if (cudaFuncSetAttribute(k_adj<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adj<L>, kLThreads, smem) != cudaSuccess ||
        per_sm < 1)
        return -1;
    int blocks = per_sm * nsm;
    const int need = (a.qb - a.qa + kLWarps - 1) / kLWarps;
    if (!a.qrange && blocks > need) blocks = need > 0 ? need : 1;
    k_adj<L><<<blocks, kLThreads, smem, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int L, bool EXACT>
int launch_accum_e(const ListArgs& a, int nsm, cudaStream_t st) {
    const size_t smem = accum_smem_per_warp(a.bins.nbins, Shape<L>::NRP) * kLWarps;
    if (cudaFuncSetAttribute(k_accum<L, EXACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return -1;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_accum<L, EXACT>, kLThreads, smem) !=
            cudaSuccess ||
        per_sm < 1)
        return -1;
    int blocks = per_sm * nsm;
    const int need = (a.qb - a.qa + kLWarps - 1) / kLWarps;
    if (!a.qrange && blocks > need) blocks = need > 0 ? need : 1;
    k_accum<L, EXACT><<<blocks, kLThreads, smem, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int L>
int launch_accum_t(const ListArgs& a, int nsm, cudaStream_t st) {
    return a.exact_img ? launch_accum_e<L, true>(a, nsm, st) : launch_accum_e<L, false>(a, nsm, st);
}

int launch_scan_k(const ListArgs& a, int nsm, cudaStream_t st) {
    const size_t smem = scan_smem_per_warp(a.bins.nbins) * kLWarps;
    if (cudaFuncSetAttribute(k_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan, kLThreads, smem) != cudaSuccess ||
        per_sm < 1)
        return -1;
    int blocks = per_sm * nsm;
    const int need = (a.qb - a.qa + kLWarps - 1) / kLWarps;
    if (!a.qrange && blocks > need) blocks = need;
    k_scan<<<blocks, kLThreads, smem, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

int launch_count(const ListArgs& a, int nsm, cudaStream_t st) {
    if (a.qb <= a.qa) return 0;
    const int warps = a.qb - a.qa;
    int blocks = (warps + kLWarps - 1) / kLWarps;
    if (blocks > nsm * 16) blocks = nsm * 16;
    k_count<<<blocks, kLThreads, 0, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_scan(const ListArgs& a, int nsm, cudaStream_t st) {
    if (!a.qrange && a.qb <= a.qa) return 0;
    return launch_scan_k(a, nsm, st);
}

size_t plan_scan_tmp_bytes(int64_t n) { return 8 * (size_t)((n + kScan64 - 1) / kScan64 + 1); }

int launch_plan(const int* need, long long* gbase, long long* tmp, int qa, int qb, long long stride, int slack,
                int npass, int* base, int* passq, int* status, cudaStream_t st) {
    const int64_t n = (int64_t)qb - qa;
    if (n > 0) {
        const int nb = (int)((n + kScan64 - 1) / kScan64);
        k_need_sums<<<nb, kScan64, 0, st>>>(need + qa, n, tmp);
        k_need_top<<<1, kScan64, 0, st>>>(tmp, nb);
        k_need_final<<<nb, kScan64, 0, st>>>(need + qa, n, tmp, gbase);
    }
    k_plan_init<<<1, 256, 0, st>>>(passq, npass, qb);
    if (qb > qa) {
        int blocks = (qb - qa + 255) / 256;
        if (blocks > 4096) blocks = 4096;
        k_plan<<<blocks, 256, 0, st>>>(need, gbase, qa, qb, stride, slack, npass, base, passq, status);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_adj(int lmax, const ListArgs& a, int nsm, cudaStream_t st) {
    if (!a.qrange && a.qb <= a.qa) return 0;
    if (a.precise) return launch_adj_df(lmax, a, nsm, st);
    switch (lmax) {
        case 0: return launch_adj_t<0>(a, nsm, st);
        case 1: return launch_adj_t<1>(a, nsm, st);
        case 2: return launch_adj_t<2>(a, nsm, st);
        case 3: return launch_adj_t<3>(a, nsm, st);
        case 4: return launch_adj_t<4>(a, nsm, st);
        case 5: return launch_adj_t<5>(a, nsm, st);
        case 6: return launch_adj_t<6>(a, nsm, st);
        case 7: return launch_adj_t<7>(a, nsm, st);
        case 8: return launch_adj_t<8>(a, nsm, st);
        case 9: return launch_adj_t<9>(a, nsm, st);
        case 10: return launch_adj_t<10>(a, nsm, st);
        default: return -1;
    }
}

int launch_accum(int lmax, const ListArgs& a, int nsm, cudaStream_t st) {
    if (!a.qrange && a.qb <= a.qa) return 0;
    if (a.precise) return launch_accum_df(lmax, a, nsm, st);
    switch (lmax) {
        case 0: return launch_accum_t<0>(a, nsm, st);
        case 1: return launch_accum_t<1>(a, nsm, st);
        case 2: return launch_accum_t<2>(a, nsm, st);
        case 3: return launch_accum_t<3>(a, nsm, st);
        case 4: return launch_accum_t<4>(a, nsm, st);
        case 5: return launch_accum_t<5>(a, nsm, st);
        case 6: return launch_accum_t<6>(a, nsm, st);
        case 7: return launch_accum_t<7>(a, nsm, st);
        case 8: return launch_accum_t<8>(a, nsm, st);
        case 9: return launch_accum_t<9>(a, nsm, st);
        case 10: return launch_accum_t<10>(a, nsm, st);
        default: return -1;
    }
}

}  // namespace g3
