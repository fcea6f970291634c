// Internal declarations of libg3pcf (not part of the public ABI).
//
// Data layout in device memory (per compute call, owned by the plan):
//   pts      float4[n]    points sorted by cell key: (x, y, z, w), FP32
//   pts64    double[3n]   sorted FP64 positions (only when the input is FP64)
//   orig     int[n]       sorted slot -> original index
//   key      uint[n]      cell key of each sorted slot
//   cstart   int[ncell+1] first sorted slot of every cell key
//   plist    int[np]      sorted slots of the primaries, in processing order
//   A        float[np_rows][RLP]  per-primary multipoles, row = original index,
//            columns: for m = 0 one block of K_0 reals (Re a_l0(b)), for m >= 1
//            [Re | Im] blocks of K_m each; column (l-m)*B + b inside a block.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "../../include/g3pcf.h"

namespace g3 {

constexpr int kMaxBins = G3PCF_MAX_NBINS;
constexpr int kMaxL = G3PCF_MAX_LMAX;
constexpr int kWarp = 32;
#define G3_BIN_TABLE 2048

// Cell grid of one compute call.  Key of cell (cx, cy, cz) of catalog c:
// c * cells_per_cat + morton2(cy, cz) * ncx + cx, so that an x-row of cells is a
// contiguous range of keys and neighbouring rows are close in memory.  Cells
// are ncx / nc times narrower along x than along y and z: a row's slot range is
// clipped to the sphere's chord at the finer x step at no extra lookup cost.
struct Grid {
    float box;        // L (FP32)
    float cell;       // L / nc (y and z)
    float inv_cell;   // nc / L
    float inv_cellx;  // ncx / L
    int nc;           // cells per dimension along y and z
    int ncx;          // cells along x
    int span;         // next power of two >= nc (Morton span of (cy, cz))
    int reach;        // max |cell offset| in y or z that can hold a neighbour
    int periodic;
    int radial;
    long long cells_per_cat;  // span * span * ncx
    double boxd;
};

// Radial binning: FP64 squared edges for the exact decision, FP32 copies and
// guard half-widths for the fast decision (see pair.cu).
struct Bins {
    int nbins;
    float rmin;
    float invw;       // nbins / (rmax - rmin)
    float rmax2f;
    float lo_rej;     // r2 below this: surely below e_0
    float hi_rej;     // r2 above this: surely >= e_B
    float slack;      // conservative slack for cell pruning
    float rmaxf;
    double e2[kMaxBins + 1];
    float e2f[kMaxBins + 1];
    float guard[kMaxBins + 1];
};

__host__ __device__ constexpr int nr_of(int L) { return (L + 1) * (L + 1); }
// accumulator slot of (l, m, part): m = 0 -> l; m >= 1 -> base(m) + 2 (l - m) + part
__host__ __device__ constexpr int acc_base(int L, int m) {
    return m == 0 ? 0 : (L + 1) + 2 * ((m - 1) * (L + 1) - (m - 1) * m / 2);
}

__host__ __device__ inline unsigned morton2(unsigned y, unsigned z) {
    unsigned r = 0;
    for (int b = 0; b < 10; ++b) r |= (((y >> b) & 1u) << (2 * b)) | (((z >> b) & 1u) << (2 * b + 1));
    return r;
}

// ---- index.cu --------------------------------------------------------------
struct IndexArgs {
    const void* pos;       // n x 3 float or double (original order)
    const float* w;
    int64_t n;
    int pos_f64;
    Grid g;
};
struct IndexBuffers {
    unsigned *key_a, *key_b;
    int *val_a, *val_b;
    int* hist;         // 256 * ntiles
    int* hist_off;     // max(256 * ntiles, n) + 1
    int* scan_tmp;
    float4* pts;
    double* pts64;     // null unless FP64 input
    int* orig;
    int* cstart;
    int* plist;        // may stay unused (identity order)
    int* status;
    unsigned* key_sorted;  // set by build_index (points into key_a or key_b)
};
struct PrimRanges {    // batch mode: plist = concatenated slot ranges
    const int* start;
    const int* len;
    const int* out;
    int n;
};
int build_index(IndexBuffers& b, const IndexArgs& a, const int64_t* cat_off_dev, int ncat,
                long long ncells, int64_t n_primary, const PrimRanges* ranges, cudaStream_t st);
int scan_exclusive(const int* in, int* out, int64_t n, int* tmp, cudaStream_t st);
size_t scan_tmp_ints(int64_t n);
size_t radix_hist_ints(int64_t n);

// ---- pair.cu ---------------------------------------------------------------
struct PairArgs {
    const float4* pts;
    const double* pts64;     // may be null (FP32 input: pts is exact)
    const int* orig;
    const int* cstart;
    const int* plist;        // null = identity (slot q is the q-th primary)
    const unsigned* key;     // sorted cell keys (catalog = key / cells_per_cat)
    int nprim;               // processing-order index one past the last primary of this launch
    int q0;                  // processing-order index of the first primary of this launch
    int chunked;             // 1: A row = q - q0 (chunk-local), 0: A row = original index
    float* wrow;             // per A row: the primary's weight (forward)
    float* A;                // rows x RLP
    int RLP;
    const int* colmap;       // RL entries: res index (b * NRP + c) feeding A column
    const float* colscale;   // RL entries: normalisation K_lm of that column
    int RL;
    unsigned long long* counts;  // ncat x nbins
    int* queue;              // work counter
    int* status;             // error bits
    int kflush;              // pairs per lane per flush
    const unsigned char* bintab;  // G3_BIN_TABLE + 2 entries over r^2 in [0, table_r2max)
    float bin_tscale;        // G3_BIN_TABLE / table_r2max
    // adjoint pass only (mode 1): V rows (M_m A_i, stride RLP, row = original
    // index), outputs dL/dw and dL/dpos (FP64, original order)
    const float* V;
    double* dw;
    double* dpos;
    Grid g;
    Bins bins;
    // forward, list path: the tensor-core operands written with the multipoles
    // (ListArgs::bop ...; null: not written), used only when no weight is negative
    __nv_bfloat16* bop;
    int nbcat;
    int bop_pitch;
    const int4* bblk;
    int nblk;
    const int4* bcat;
};
// mode 0: forward multipoles; mode 1: adjoint pair pass
int launch_pair(int lmax, const PairArgs& a, int nsm, cudaStream_t st, int mode = 0);
size_t pair_smem_per_warp(int lmax, int nbins, int kflush);

// ---- pairlist.cu -----------------------------------------------------------
// Forward pair stage as three kernels over the primaries [qa, qb) (processing
// order): k_count writes need[q] = ceil(candidates / 32) + nbins (an upper
// bound of the list chunks of q); the host sets base[q] (first chunk of q in
// the pool, relative to the pass) so that a pass fits the pool; k_scan writes
// the chunks (32 entries j | code << 27, padding 0xffffffff), the list of them
// ordered by bin (ord: chunk | bin << 26) and nchunks[q]; k_accum walks that
// list and writes A rows.
struct ListArgs {
    const float4* pts;
    const double* pts64;
    const int* orig;
    const int* cstart;
    const int* plist;
    const unsigned* key;
    int qa, qb;              // primaries of this launch (processing order)
    int q0;                  // first primary of the A chunk (row = q - q0 when chunked)
    int chunked;
    float* wrow;
    float* A;
    int RLP;
    const int4* colconv;     // RL entries: {first res slot, slot stride, terms, coefficient offset}
    const float* colcoef;    // Chebyshev -> Legendre-form coefficients (times K_lm)
    int RL;
    unsigned long long* counts;
    int* queue;
    int* status;
    const signed char* bintab;  // G3_BIN_TABLE + 2: bin, -1 no pair, -3 decide per pair
    float bin_tscale;
    int* need;               // [q] (global processing-order index)
    unsigned long long* ncand;  // candidates visited (k_count adds)
    const int* base;         // [q] first chunk of q, relative to the pool arrays
    int* nchunks;            // [q]
    const int* qrange;       // if set: qa = qrange[0], qb = qrange[1] (device-planned pass)
    int exact_img;           // k_accum: separations from the head + tail of the primary's images
    // monomial-basis multipoles (k_mono): exponents a | b << 8 | c << 16 per monomial;
    // per (l, m, part) {first term, terms, A column of bin 0}; terms (monomial, coefficient)
    const int* monoexp;
    const int4* monoconv;
    const int* monoidx;
    const double* monocoef;
    // adjoint pass (k_adj): V rows (row = original index), slot tables of the
    // transposed Chebyshev connection, outputs (FP64, original order)
    const float* V;
    const int4* slotconv;    // NR entries: {first A column (bin 0), column stride, terms, coefficient offset}
    const float* slotcoef;
    double* dw;
    double* dpos;
    // double-float path (multipoles meant for differentiation): FP64 connection
    // tables (same layout as colcoef / slotcoef) and the FP64 V rows
    int precise;
    const float2* colcoefdf;     // colcoef as head + tail FP32 pairs (double-float path)
    const float2* slotcoefdf;    // slotcoef likewise
    const float2* Vdf;           // V rows as head + tail pairs (double-float adjoint)
    // tensor-core operands written by k_accum (forward, no negative weight):
    // sqrt(w) A split into bf16 hi and lo: row r holds hi at bop + 2 r bop_pitch and
    // lo bop_pitch later (one contiguous stretch per row), m blocks from multiples
    // of 64 (bblk[m] = {first A column, width, first operand column, 0}), rows in
    // padded coordinates (bcat per catalog: {first padded row, first A row, rows,
    // 0}; nbcat catalogs); skip_a: the FP32 rows of A are not written
    __nv_bfloat16* bop;
    int nbcat;
    int bop_pitch;
    const int4* bblk;
    int nblk;
    const int4* bcat;
    int skip_a;
    int* chunks;             // pool: 32 ints per chunk
    int* tag;                // pool: (rank among its bin's chunks) << 5 | bin, per chunk
    int* ord;                // pool: the primary's chunks listed by bin (stable), chunk | bin << 26
    Grid g;
    Bins bins;
};
int launch_count(const ListArgs& a, int nsm, cudaStream_t st);
// Device-side pass plan (graph capture): gbase = exclusive prefix of need over
// [qa, qb) (64-bit; tmp holds plan_scan_tmp_bytes); primary q goes to pass
// p = gbase / stride at base gbase - p * stride (base -1 and the overflow bit
// when p >= npass or need > slack); passq[p] = first primary of pass p
// (passq[npass] = qb).
size_t plan_scan_tmp_bytes(int64_t n);
int launch_plan(const int* need, long long* gbase, long long* tmp, int qa, int qb, long long stride, int slack,
                int npass, int* base, int* passq, int* status, cudaStream_t st);
int launch_scan(const ListArgs& a, int nsm, cudaStream_t st);
int launch_accum(int lmax, const ListArgs& a, int nsm, cudaStream_t st);
int launch_adj(int lmax, const ListArgs& a, int nsm, cudaStream_t st);
// precise.cu: the same two passes in double-float (a.precise selects them inside
// launch_accum / launch_adj)
int launch_accum_df(int lmax, const ListArgs& a, int nsm, cudaStream_t st);
int launch_adj_df(int lmax, const ListArgs& a, int nsm, cudaStream_t st);
// monomial.cu: the multipoles through the paper's monomial power sums (FP64)
int mono_count(int lmax);
int launch_mono(int lmax, const ListArgs& a, int nsm, cudaStream_t st);

// ---- contract.cu -----------------------------------------------------------
struct Tile {          // one output tile of one m block of C_m = sum_i w_i v_i v_i^T
    int m, r0, c0, rows, cols, col0;  // col0: first column of block m inside an A row
    int width;         // block width W_m
    int out_off;       // offset (floats) of this tile inside one segment's partials
};
struct Segment { int cat; int row0; int row1; };
// Upper-triangle output tiles of every m block (T x T, ragged at the block
// edge), in (m, row tile, column tile) order; returns the count or -1 when
// more than max_tiles are needed.  Host and device code (the allocation-free
// entry point fills its fixed table on the device).
__host__ __device__ inline int fill_tiles(int nbins, int lmax, int T, Tile* out, int max_tiles) {
    int n = 0, col0 = 0, off = 0;
    for (int m = 0; m <= lmax; ++m) {
        const int K = nbins * (lmax + 1 - m);
        const int W = (m == 0) ? K : 2 * K;
        const int nt = (W + T - 1) / T;
        for (int ti = 0; ti < nt; ++ti)
            for (int tj = ti; tj < nt; ++tj) {
                if (n >= max_tiles) return -1;
                Tile& t = out[n++];
                t.m = m;
                t.r0 = ti * T;
                t.c0 = tj * T;
                t.rows = W - t.r0 < T ? W - t.r0 : T;
                t.cols = W - t.c0 < T ? W - t.c0 : T;
                t.col0 = col0;
                t.width = W;
                t.out_off = off;
                off += T * T;
            }
        col0 += W;
    }
    return n;
}
int make_tiles(int nbins, int lmax, int T, Tile* out, int max_tiles);
// Number of tiles fill_tiles writes for (nbins, lmax, T).
__host__ __device__ inline int count_tiles(int nbins, int lmax, int T) {
    int n = 0;
    for (int m = 0; m <= lmax; ++m) {
        const int W = (m == 0 ? 1 : 2) * nbins * (lmax + 1 - m);
        const int nt = (W + T - 1) / T;
        n += nt * (nt + 1) / 2;
    }
    return n;
}
int contract_tile_dim_fp32();
int launch_contract_fp32(const float* A, int RLP, const float* wrow, const Tile* tiles, int ntiles,
                         const Segment* segs, int nsegs, double* partials, int part_stride,
                         cudaStream_t st);
// colmajor: partial tiles stored [c][r] (tensor-core path) instead of [r][c]
int launch_reduce(const double* partials, int part_stride, const int* seg_first, int ncat,
                  int nbins, int lmax, const Tile* tiles, int T, double* zeta, cudaStream_t st,
                  int colmajor = 0);
int pair_nrp(int lmax);
int launch_isotropic(const double* zeta, int nbins, int lmax, int ncat, double* out, cudaStream_t st);
// out = sum_c coef[c] zeta_c (coef: host, passed by value; ncat <= kMaxCombine)
constexpr int kMaxCombine = 256;
struct CombineCoef { double c[kMaxCombine]; };
int launch_combine(const double* zeta, int64_t zsize, int ncat, const double* coef, double* out, cudaStream_t st);
// contract_tc.cu: split-BF16 tcgen05 contraction
int contract_tile_dim_tc();
int contract_tc_kblock();
// negw: the status block's negative-weight flag (kNegWeightSlot), read on the
// device: 0 -> both operand sides are hi/lo of sqrt(w) A; else the left side is
// hi/lo of A and the right side hi/lo of w A.  The operands are formed inside
// the kernel from the FP32 rows A (row pitch RLP) and the row weights wrow;
// cats: per catalog {padded start, first A row, length, 0}.
// A strip: ntile (1 or 2) output tiles side by side in one row panel, tiles
// tile0.. of the tile list; xrow / xcol = A column of its first row / column.
// A strip: ntile (1 or 2) tiles of one row panel from tile0, computed as one
// M = 128 MMA of width n (the strip's valid columns rounded up to 16); xb: the
// column of its first column panel in the bf16 operand rows (m blocks from
// multiples of 64).
struct TcStrip { int tile0; int ntile; int xrow; int xcol; int n; int xb; };
// A work item of the tensor-core contraction: a strip and nvseg (1 or 2)
// consecutive virtual segments from vseg0 (partials go to slot vseg0).
struct TcItem { int strip; int vseg0; int nvseg; int pad; };
int make_strips(const Tile* tiles, int ntiles, TcStrip* out, int max_strips);
// Work split of one catalog for the tensor-core contraction: returns V, the
// number of equal virtual segments (even, >= 2, <= vmax unless vmax < 2), about
// slots / (items per segment), and step[s], the segments per work item of strip s.
int plan_tc_items(const TcStrip* strips, int nstrips, int vmax, double slots, int* step);
// arows: rows of A in the buffer (the tensor map's extent; rows beyond read as 0)
int launch_contract_tc(const float* A, int RLP, int RL, int64_t arows, const float* wrow, const int4* cats,
                       const Tile* tiles, const TcStrip* strips, const TcItem* items, int nitems,
                       const Segment* segs, double* partials, int part_stride, const int* negw, int* status,
                       cudaStream_t st, int test_timeout = 0);
// Operand columns of the bf16 rows written by k_accum: every m block starts on a
// multiple of 64; blk[m] = {first A column, width, first operand column, 0}
// (m <= lmax < max_blk); returns the row pitch, or -1
int tc_operand_blocks(const Tile* tiles, int ntiles, int4* blk, int max_blk);
// The same contraction from the bf16 hi / lo operand rows (row r: hi at bop +
// 2 r pitch, lo pitch later; rows = padded rows): no conversion in the kernel;
// every weight must be non-negative (the operands are sqrt(w) A).
int launch_contract_tc_op(const __nv_bfloat16* bop, int pitch, int64_t rows, const Tile* tiles,
                          const TcStrip* strips, const TcItem* items, int nitems, const Segment* segs,
                          double* partials, int part_stride, int* status, cudaStream_t st, int test_timeout = 0);
// Zero the padding rows [first + rows, first + padded) of every catalog's operand
// rows (bcat as in ListArgs; padded = rows rounded up to the k-block)
int launch_zero_pad(__nv_bfloat16* bop, int pitch, const int4* bcat, int ncat, cudaStream_t st);

// ---- adjoint.cu ----------------------------------------------------------------
size_t adjoint_m_floats(int nbins, int lmax);
int adjoint_rows_per_block();
// M_c = G_c + G_c^H per catalog c (ncat x adjoint_m_floats), then V = M_c A and
// the primary-weight term of dL/dw per row block blks[] = {catalog, first row, rows}
int launch_adjoint_prep(const double* dzeta, int nbins, int lmax, int ncat, int64_t zsize, const float* A,
                        int RLP, int RL, const int4* blks, int nblks, float* Mr, float* V, double* dw,
                        cudaStream_t st);
// the two halves of it for a chunked backward: M of every catalog, then V and the
// primary-weight term for the A rows [row_lo, row_hi) of the chunk starting at
// processing-order primary q0 (dw indexed through plist/orig)
int launch_adjoint_m(const double* dzeta, int nbins, int lmax, int ncat, int64_t zsize, float* Mr,
                     cudaStream_t st);
int launch_vgemm_rows(const float* A, int RLP, int RL, int64_t row_lo, int64_t row_hi, const float* Mr,
                      int nbins, int lmax, float* V, double* dw, const int* plist, const int* orig,
                      int64_t q0, cudaStream_t st);
// Double-float forms of the three (M and V as head + tail FP32 pairs, ~48 bits;
// for the double-float adjoint pass)
int launch_adjoint_prep_df(const double* dzeta, int nbins, int lmax, int ncat, int64_t zsize, const float* A,
                           int RLP, int RL, const int4* blks, int nblks, float2* Mr, float2* V, double* dw,
                           cudaStream_t st);
int launch_adjoint_m_df(const double* dzeta, int nbins, int lmax, int ncat, int64_t zsize, float2* Mr,
                        cudaStream_t st);
int launch_vgemm_rows_df(const float* A, int RLP, int RL, int64_t row_lo, int64_t row_hi, const float2* Mr,
                         int nbins, int lmax, float2* V, double* dw, const int* plist, const int* orig,
                         int64_t q0, cudaStream_t st);

// ---- api.cu / noalloc.cu -----------------------------------------------------
void set_last_error(const char* msg);
int noalloc_zeta_from_alm(int nbins, int lmax, const float* alm, int64_t ld, const float* w,
                          int64_t np, double* zeta, cudaStream_t st, char* err, size_t errlen);

// Status block of a call (256 bytes, zeroed per call): int [0] status word,
// [16] work counter, [20] set by the index build when a weight is negative,
// [24..25] candidate count (64-bit).
constexpr int kNegWeightSlot = 20;

// status bits written by kernels
enum : int {
    kStatusRange = 1,
    kStatusTimeout = 2,
    kStatusOverflow = 4,
};

}  // namespace g3
