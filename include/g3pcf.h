/*
 * g3pcf.h -- C ABI of the GB300 (sm_103a) anisotropic three-point correlation
 * function library, after Friesen et al., "Galactos: Computing the Anisotropic
 * 3-Point Correlation Function for 2 Billion Galaxies" (SC17, arXiv 1709.00086).
 *
 * What the library computes (Section 3.1, the expansion equation and
 * Algorithm 1 of the paper): for every primary galaxy i, all secondaries j
 * within rmax are gathered and binned into radial shells (Sec. 3.1,
 * "binned into spherical shells"); the separation is rotated into the frame
 * whose z axis is the primary's line of sight (Sec. 3.1, Fig. 2); the
 * spherical harmonics of the separation direction are summed per shell into
 *      a_lm(i, b) = sum_{j in b} w_j Y_lm(rhat'_ij),     0 <= m <= l <= lmax
 * (Sec. 3.1, the discrete form of the shell integral), and the products of the
 * coefficients about each primary are summed over primaries into
 *      zeta^m_{l l'}(b1, b2) = sum_i w_i a_lm(i, b1) conj(a_l'm(i, b2))
 * (Sec. 3.1, "simply a_lm(r1) a*_l'm(r2)"; equal m from the axisymmetry
 * about the line of sight).  Y_lm are orthonormal with the Condon-Shortley
 * phase.  Weights w are an extension (the paper's catalogs are unweighted):
 * a_lm is weighted by the secondary's w_j, zeta by the primary's w_i.
 *
 * Binning (the exact rule, identical to the FP64 reference): edges
 * e_0 = rmin, e_B = rmax, e_k = rmin + (rmax - rmin)*k/B in FP64; the pair is in
 * bin b iff e_b^2 <= r^2 < e_{b+1}^2 with r^2 = (dx*dx + dy*dy) + dz*dz
 * evaluated in FP64 without fused multiply-add on d = x_j - x_i (minimum image
 * per axis in a periodic box: d -= L if d > L/2, d += L if d < -L/2).  Pairs
 * with r^2 == 0 (the primary itself and coincident points) are skipped.
 *
 * ZETA LAYOUT.  For m = 0..lmax one K_m x K_m complex block, K_m = nbins *
 * (lmax + 1 - m), blocks stored consecutively; within block m the row index is
 * (l - m)*nbins + b1 and the column index (l' - m)*nbins + b2, row-major,
 * each entry two doubles (re, im).  Only m >= 0 is stored (zeta^{-m} =
 * conj(zeta^m) for real weights).  Total g3pcf_zeta_size() complex entries.
 *
 * MEMORY AND STREAMS.  All array arguments marked "device" are device
 * pointers owned by the caller; the library never frees them.  The plan owns
 * its workspace (grown on demand, kept until g3pcf_destroy).  Compute calls are
 * enqueued on the plan's stream (g3pcf_set_stream; default the legacy stream)
 * and, unless G3PCF_F_NO_SYNC is given, synchronise that stream once at the end
 * to read the device status word, so that range errors and bounded-wait
 * timeouts are returned by the call itself.
 *
 * ERRORS.  Every entry point returns G3PCF_OK (0) or a negative code and, on
 * error, stores a message retrievable with g3pcf_last_error() (per thread).
 * Host-side validation happens before any device work is enqueued.
 */
#ifndef G3PCF_H
#define G3PCF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct g3pcf_plan_s* g3pcf_plan_t;

/* Line-of-sight / boundary modes (Sec. 3.1: "the line of sight ... which we
 * here take to be the z-axis", and Fig. 2: rotate so that the primary lies on
 * the z axis of the line of sight to the observer). */
enum {
    G3PCF_LOS_Z_PERIODIC = 0,  /* LOS = +z, periodic cube of side box (minimum image) */
    G3PCF_LOS_Z_OPEN = 1,      /* LOS = +z, open cube [0, box)^3                      */
    G3PCF_LOS_RADIAL_OPEN = 2  /* LOS = direction from the cube centre to the primary;
                                  open cube.  Rotation: Rodrigues about n x z taking n
                                  to +z; a half turn about x when n is within 1e-12 of
                                  -z; n = +z for a primary at the centre.             */
};

/* Return codes. */
enum {
    G3PCF_OK = 0,
    G3PCF_ERR_ARG = -1,         /* invalid argument (null pointer, bad size or mode)     */
    G3PCF_ERR_RANGE = -2,       /* a position outside [0, box) or not finite, or a
                                   non-finite weight (reported by the device check)     */
    G3PCF_ERR_RMAX = -3,        /* periodic box with rmax >= box/2                       */
    G3PCF_ERR_ALLOC = -4,       /* workspace allocation failed                           */
    G3PCF_ERR_CUDA = -5,        /* a CUDA runtime call failed                            */
    G3PCF_ERR_TIMEOUT = -6,     /* a bounded device wait expired (kernel returned early) */
    G3PCF_ERR_STATE = -7,       /* backward/alm without a matching forward on this plan  */
    G3PCF_ERR_UNSUPPORTED = -8  /* valid request the library does not implement           */
};

/* Flags for g3pcf_compute_ex / g3pcf_compute_batch. */
enum {
    G3PCF_F_POS_F64 = 1,        /* pos is double (n x 3) instead of float                */
    G3PCF_F_CONTRACT_FP32 = 2,  /* zeta contraction in plain FP32 on the FMA pipe instead
                                   of split-BF16 (hi+lo, 3 products) tcgen05 tensor cores */
    G3PCF_F_NO_SYNC = 4,        /* do not synchronise at the end; device status is then
                                   read by g3pcf_status()                                 */
    G3PCF_F_KEEP_ALM = 8,       /* the multipoles of the call are meant for g3pcf_alm and
                                   g3pcf_backward (implied when requires_grad is used):
                                   separations are formed from the exact FP64 image of
                                   the primary, and the multipoles are evaluated and
                                   summed in double-float with the connection in FP64
                                   (G3PCF_OPT_GRAD_PRECISION); several times the FP32
                                   pair-stage time                                       */
    G3PCF_F_GRAPH = 16          /* replay a captured CUDA graph: the first call with a new
                                   signature (pointers, sizes, offsets, flags, options) runs
                                   once and captures its device work on an internal stream;
                                   later calls with the same signature replay it, ordered
                                   after the plan's stream.  A call without this flag drops
                                   the graph.                                             */
};

/* Limits of the library. */
#define G3PCF_MAX_LMAX 10
#define G3PCF_MAX_NBINS 32
#define G3PCF_MAX_POINTS ((int64_t)1 << 27)

/* Number of complex entries of zeta for (nbins, lmax): sum_m K_m^2. */
int64_t g3pcf_zeta_size(int nbins, int lmax);

/* Create a plan (host only, no device work).  nbins in [1, 32]; 0 <= rmin <
 * rmax; lmax in [0, 10]; box > 0; los_mode one of G3PCF_LOS_*.  Periodic mode
 * requires rmax < box/2 (else G3PCF_ERR_RMAX).  *out receives the plan. */
int g3pcf_plan(g3pcf_plan_t* out, int nbins, double rmin, double rmax, int lmax, double box,
               int los_mode);

/* Set the CUDA stream (a cudaStream_t, e.g. PyTorch's current stream) on which
 * all later device work of this plan is enqueued.  NULL = legacy stream. */
int g3pcf_set_stream(g3pcf_plan_t plan, void* cuda_stream);

/* Forward: zeta for n points, every point a primary.  pos: device, n x 3
 * float (x, y, z interleaved), in [0, box)^3.  w: device, n floats.
 * zeta: device, 2 * g3pcf_zeta_size() doubles (layout above), overwritten.
 * n may be 0 (zeta is zeroed).  Split-BF16 tensor-core contraction. */
int g3pcf_compute(g3pcf_plan_t plan, const float* pos, const float* w, int64_t n, double* zeta);

/* Forward with options.  pos: device, n x 3 float, or double if
 * G3PCF_F_POS_F64.  n_primary in [0, n] (negative = n): the first n_primary
 * points are primaries, all n are secondaries (the paper's primary/halo split,
 * Algorithm 1 "if not primary: skip").  counts: device, nbins int64 (ordered
 * pairs accepted per bin, bit-exact), may be NULL.  flags: G3PCF_F_*. */
int g3pcf_compute_ex(g3pcf_plan_t plan, const void* pos, const float* w, int64_t n,
                     int64_t n_primary, double* zeta, int64_t* counts, int flags);

/* Batched forward over ncat independent catalogs sharing the plan's geometry
 * (each its own box, every point a primary of its own catalog).  pos, w:
 * device, the catalogs concatenated (float, n_total x 3 and n_total).
 * offsets: HOST, ncat + 1 int64 (catalog c = points [offsets[c], offsets[c+1])).
 * zeta: device, ncat consecutive zeta blocks.  counts: device, ncat x nbins
 * int64, may be NULL.  One launch per stage over all catalogs (device work
 * queue, heaviest catalogs first).  flags: G3PCF_F_CONTRACT_FP32,
 * G3PCF_F_NO_SYNC, G3PCF_F_KEEP_ALM (multipoles kept for g3pcf_backward) and
 * G3PCF_F_GRAPH (capture and replay, as for g3pcf_compute_ex). */
int g3pcf_compute_batch(g3pcf_plan_t plan, const float* pos, const float* w,
                        const int64_t* offsets, int ncat, double* zeta, int64_t* counts,
                        int flags);

/* Adjoint of the last forward on this plan (LOS = z modes; g3pcf_compute* or
 * g3pcf_compute_batch).  dzeta: device, same layout as the forward's zeta (for a
 * batch, ncat consecutive blocks, catalog c's gradient in block c), the gradient
 * of a real loss with respect to (Re zeta, Im zeta) interleaved.  dpos: device,
 * n x 3 doubles; dw: device, n doubles (all points of the forward, its order);
 * both overwritten.  Pair set and bins are held fixed.  The pos and w
 * buffers of the forward must still hold the same values.  Not in the paper:
 * dL/dw_i and dL/dpos_i of zeta through Y_lm and the weights.
 * Not bitwise reproducible: the secondaries' terms are summed with FP64
 * atomic additions whose order varies between runs, so two backwards on the
 * same input can differ in the last bits (the forward is reproducible). */
int g3pcf_backward(g3pcf_plan_t plan, const double* dzeta, double* dpos, double* dw);

/* Multipoles of the last forward (run with G3PCF_F_KEEP_ALM or before a
 * backward) for np primaries given by original index (HOST int64 array).
 * out: HOST, np x nbins x ((lmax+1)(lmax+2)/2) complex (re, im doubles),
 * index [k][b][l(l+1)/2 + m].  Synchronises the plan's stream. */
int g3pcf_alm(g3pcf_plan_t plan, const int64_t* primaries, int64_t np, double* out);

/* Autotuner (a project-written search, not in the paper): times the pair stage
 * on a bounded sample (the first min(n, 32768) points as primaries, all n as
 * secondaries; best of two timed runs after one that sizes the workspace) over
 * the cell resolution around the density heuristic (s - 1, s, s + 1) and, for
 * the pair lists, the x refinement of the cells (4, 8, 16), or, for the fused
 * kernel, two flush sizes; keeps the fastest on the plan (as if set with
 * g3pcf_set_option).  For a batch, tune on its largest catalog (its pairs
 * dominate the step).  pos/w as for g3pcf_compute_ex (flags: G3PCF_F_POS_F64
 * only).  cache_path (may be NULL): a text file of earlier results, one line
 * per key (nbins, lmax, LOS mode, kernel choice, SM count and the expected
 * neighbours per point n (4/3) pi rmax^3 / box^3 in quarter-octave buckets); a
 * hit applies the stored settings without timing anything, a miss tunes and
 * appends a line (an unreadable or unwritable file only disables the cache).
 * With the pair lists in the Chebyshev basis it then times the pair stage and
 * the tensor-core contraction together on the same sample for both settings of
 * G3PCF_OPT_TC_OPERANDS and keeps the faster.
 * chosen (HOST, may be NULL, 6 entries): {cells per rmax, x refinement, kflush,
 * pair-stage microseconds of the sample, 1 if taken from the cache,
 * G3PCF_OPT_TC_OPERANDS}.
 * Allocates a temporary zeta buffer; synchronises the plan's stream. */
int g3pcf_autotune_cached(g3pcf_plan_t plan, const void* pos, const float* w, int64_t n, int flags,
                          const char* cache_path, int64_t* chosen);

/* The same without a cache; chosen (HOST, may be NULL) receives {cells per
 * rmax, kflush, pair-stage microseconds}. */
int g3pcf_autotune(g3pcf_plan_t plan, const void* pos, const float* w, int64_t n, int flags,
                   int64_t* chosen);

/* Status word of the last G3PCF_F_NO_SYNC call (synchronises the stream):
 * returns G3PCF_OK or the error the call would have returned. */
int g3pcf_status(g3pcf_plan_t plan);

/* Per-stage device times (milliseconds, CUDA events) and counters of the last
 * compute call: [0] index build, [1] pair stage, [2] contraction (both summed
 * over the chunks of primaries of a chunked call), [3] reduction, [4] total,
 * [5] accepted pairs (as a double), [6] primaries, [7] cells per Rmax used,
 * [8] kernels launched by the call, [9] candidate secondaries visited
 * (pair-list path; 0 for the fused kernel), [10] passes of the pair lists,
 * [11] and [12] summed device times (ms) of the list scan and accumulate
 * kernels, [13] accumulate launches, [14] 1 when the pair stage wrote the
 * tensor-core operands (G3PCF_OPT_TC_OPERANDS), else 0.  Synchronises the stream.
 * At most min(nvals, 15) values are written. */
int g3pcf_stats(g3pcf_plan_t plan, double* vals, int nvals);

/* zeta from multipoles the caller already holds, without allocating any
 * memory (the paper has no counterpart; this is a service for callers that
 * cannot allocate: code running inside a fixed, pre-reserved device-memory
 * budget, or inside a streamed pipeline that must not pay cudaMalloc's
 * implicit synchronisation).  Computes
 *      zeta^m_{l l'}(b1, b2) = sum_i w_i a_lm(i, b1) conj(a_l'm(i, b2))
 * with the plain-FP32 contraction and the FP64 reduction of g3pcf_compute.
 *   alm:  device, np rows of ld floats (ld >= nbins*(lmax+1)^2); row i holds
 *         primary i's multipoles: first the K_0 = nbins*(lmax+1) values
 *         Re a_l0(b) at column l*nbins + b, then for m = 1..lmax the K_m values
 *         Re a_lm(b) followed by the K_m values Im a_lm(b), each at offset
 *         (l - m)*nbins + b inside its half.
 *   w:    device, np primary weights.   zeta: device output (layout above).
 *   stream: cudaStream_t (NULL = legacy stream).  Asynchronous; no sync.
 * Scratch: 16 MiB of FP64 partial sums and small tile tables in fixed device
 * arrays inside the library, present on every GPU that loads it until the
 * process exits.  The first call on a device looks up their addresses (with
 * that device current; safe from several host threads); do not call this
 * entry point on a device after cudaDeviceReset().  Every call rewrites the tables on the device and
 * overwrites what it reads, so nothing needs clearing; calls that overlap on
 * the GPU share the arrays and race, so the caller must serialise them.
 * Limits: nbins <= 32, lmax <= 10, np < 2^27; shapes whose tile table or one
 * segment of partials would not fit return G3PCF_ERR_ARG. */
int g3pcf_zeta_from_alm_noalloc(int nbins, int lmax, const float* alm, int64_t ld,
                                const float* w, int64_t np, double* zeta, void* stream);

/* Isotropic (Legendre) 3PCF from zeta.  The paper's Sec. 2.2 expands the
 * isotropic 3PCF in Legendre polynomials of rhat_1 . rhat_2 with radial
 * coefficients zeta_l(r1, r2); by the addition theorem these are the m-sums of
 * the anisotropic coefficients of Sec. 3.1.  For every catalog c, l <= lmax and
 * bin pair (b1, b2):
 *     out[c][l][b1][b2] = Re zeta^0_ll(b1,b2) + 2 sum_{m=1}^{l} Re zeta^m_ll(b1,b2)
 *                       = (2l+1)/(4 pi) sum_i w_i sum_{j in b1, k in b2} w_j w_k P_l(rhat_ij . rhat_ik)
 * (j = k terms included, the m < 0 blocks folded in through zeta^{-m} = conj(zeta^m)).
 *   zeta: device, ncat x g3pcf_zeta_size(nbins, lmax) complex FP64 (interleaved), as
 *         written by g3pcf_compute* (caller-owned, read only).
 *   out:  device, ncat x (lmax + 1) x nbins x nbins FP64, row-major (caller-owned).
 *   stream: cudaStream_t or NULL.  Asynchronous; allocates nothing.
 * Errors: G3PCF_ERR_ARG for nbins / lmax / ncat out of range or null pointers;
 * G3PCF_ERR_CUDA if the launch fails. */
int g3pcf_isotropic(int nbins, int lmax, int ncat, const double* zeta, double* out, void* stream);

/* Linear combination of zeta blocks: out = sum_c coef[c] zeta_c.  The paper's
 * Sec. 6 corrects the measured 3PCF with random catalogs, whose own noise is
 * averaged down by using many of them; with a batch of D - R_k catalogs (data
 * plus the k-th random catalog at negative weight) and of the randoms R_k from
 * one g3pcf_compute_batch, coef = 1/N_R on the first N_R blocks gives the mean
 * zeta of the D - R field, and on the last N_R blocks the mean zeta of the
 * randoms.  The sum runs over catalogs in index order (reruns are bit-identical).
 *   zeta: device, ncat x g3pcf_zeta_size(nbins, lmax) complex FP64 (caller-owned).
 *   coef: HOST, ncat finite doubles (copied into the launch).
 *   out:  device, one zeta block (caller-owned; must not overlap zeta).
 *   stream: cudaStream_t or NULL.  Asynchronous; allocates nothing.
 * Errors: G3PCF_ERR_ARG for nbins / lmax out of range, ncat outside
 * [1, G3PCF_MAX_COMBINE], a null pointer or a non-finite coefficient;
 * G3PCF_ERR_CUDA if the launch fails. */
#define G3PCF_MAX_COMBINE 256
int g3pcf_zeta_combine(int nbins, int lmax, int ncat, const double* zeta, const double* coef, double* out,
                       void* stream);

/* Diagnostic: measured FP32 FMA throughput of the current device (TFLOP/s,
 * one FMA = 2 flop), best of 5 timed launches of an FMA-chain kernel that fills
 * every SM.  The denominator of the pair stage's roofline.  stream may be NULL.
 * Allocates and frees a small device buffer; synchronises the stream. */
int g3pcf_fp32_peak(double* tflops, void* stream);

/* Tuning knobs of a plan (0 = automatic, the default for each):
 *   G3PCF_OPT_CHUNK_ROWS      primaries per pass of the pair stage + contraction;
 *                             large catalogs are processed in chunks so that the
 *                             per-primary multipoles never exceed the memory budget
 *                             (automatic: all primaries if they fit, else chunks);
 *                             after a chunked forward g3pcf_alm returns
 *                             G3PCF_ERR_STATE and g3pcf_backward recomputes the
 *                             multipoles chunk by chunk (pair lists only)
 *   G3PCF_OPT_CELLS_PER_RMAX  cell-list resolution s (cell side >= rmax / s, 1..8)
 *   G3PCF_OPT_X_REFINE        cells are this many times narrower along x than
 *                             along y and z (1..16; automatic: 8): an x-row of
 *                             cells is one contiguous slot range, so a finer x step
 *                             clips each row to the sphere more tightly
 *   G3PCF_OPT_KFLUSH          pairs per lane per bucket flush of the fused pair
 *                             kernel (2..16)
 *   G3PCF_OPT_PAIR_KERNELS    forward pair stage: 1 = the fused kernel (bucket and
 *                             accumulate in one pass), 0 or 2 = pair lists (count,
 *                             scan into per-bin lists of 32 pairs, accumulate; one
 *                             host synchronisation per chunk of primaries; inside a
 *                             captured graph (G3PCF_F_GRAPH) the list passes are
 *                             planned on the device instead)
 *   G3PCF_OPT_LIST_BYTES      device bytes for the pair lists (0: up to 40% of free
 *                             memory, at most 32 GB); more pairs than fit are
 *                             processed in several passes
 *   G3PCF_OPT_GRAD_PRECISION  arithmetic of the pair stage for multipoles that are
 *                             differentiated (forwards with G3PCF_F_KEEP_ALM, the
 *                             backward and its recomputation): 0 = double-float
 *                             (FP32 head + tail, V = M A too), gradients within
 *                             1e-7 of the FP64 reference; 1 = FP32, about 1e-6
 *                             (faster).  Plain forwards always use FP32; the fused
 *                             kernel (G3PCF_OPT_PAIR_KERNELS = 1) is FP32 only
 *   G3PCF_OPT_BASIS           multipoles of the pair-list forward: 0 = Chebyshev form
 *                             (FP32, the fast path); 1 = the paper's monomial power
 *                             sums sum w x^a y^b z^c, a + b + c <= lmax (Sec. 3.3.2),
 *                             accumulated and converted in FP64 -- a slow cross-check
 *   G3PCF_OPT_TEST_FAIL_ALLOC test hook for the allocation-failure path: with value
 *                             k >= 1 the k-th workspace growth of this plan from now
 *                             on fails once with G3PCF_ERR_ALLOC (host side, before
 *                             anything is launched with that buffer); 0 = off
 *   G3PCF_OPT_TEST_TC_TIMEOUT test hook for the bounded-wait path of the tensor-core
 *                             contraction: 1 = the MMA thread's first wait for its
 *                             operands gives up at once, as if its bound had expired;
 *                             the kernel then flags G3PCF_ERR_TIMEOUT, waits (bounded)
 *                             for its own copies, frees its tensor memory and
 *                             returns; 0 = off
 *   G3PCF_OPT_TC_OPERANDS     operands of the tensor-core contraction: 0 = formed
 *                             inside the contraction kernel from the FP32 rows of A;
 *                             1 = written by the pair stage as bf16 hi / lo rows of
 *                             sqrt(w) A, so that the contraction only copies and
 *                             multiplies (used when no weight is negative, the
 *                             forward is one pass of the pair lists in the Chebyshev
 *                             basis outside a captured graph and they fit in memory;
 *                             otherwise as 0).  Both give bit-identical results; 1
 *                             shortens the contraction and lengthens the accumulate
 *                             kernel (on the 2M-point workload by 1.6 and 3.7 ms).
 * Returns G3PCF_ERR_ARG for unknown options or values out of range. */
enum {
    G3PCF_OPT_CHUNK_ROWS = 1,
    G3PCF_OPT_CELLS_PER_RMAX = 2,
    G3PCF_OPT_KFLUSH = 3,
    G3PCF_OPT_PAIR_KERNELS = 4,
    G3PCF_OPT_LIST_BYTES = 5,
    G3PCF_OPT_BASIS = 7,
    G3PCF_OPT_X_REFINE = 8,
    G3PCF_OPT_GRAD_PRECISION = 9,
    G3PCF_OPT_TEST_FAIL_ALLOC = 10,
    G3PCF_OPT_TEST_TC_TIMEOUT = 11,
    G3PCF_OPT_TC_OPERANDS = 12
};
int g3pcf_set_option(g3pcf_plan_t plan, int option, int64_t value);

/* Destroy a plan and free its workspace (synchronises its stream). */
int g3pcf_destroy(g3pcf_plan_t plan);

/* Message of the last error on this thread ("" if none). */
const char* g3pcf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* G3PCF_H */
