// C ABI of libg3pcf: plans, workspace, host-side validation and the launch
// sequence of one forward call (index -> pair stage -> contraction ->
// reduction), all enqueued on the plan's stream.
//
// The problem statement follows the paper's Sec. 3.1 and Algorithm 1; see
// include/g3pcf.h for the contract of every entry point.
#include <algorithm>
#include <cmath>
#include <new>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

using namespace g3;

namespace {
thread_local std::string g_err;
}  // namespace

void g3::set_last_error(const char* msg) { g_err = msg ? msg : ""; }

namespace {

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(call)                                                                       \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(G3PCF_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));      \
    } while (0)

// Grow-only device buffer.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    int ensure(size_t need) {
        if (need <= bytes && p) return 0;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        size_t b = need < 256 ? 256 : need;
        if (cudaMalloc(&p, b) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        bytes = b;
        return 0;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

double lfact(int k) { return std::lgamma((double)k + 1.0); }

}  // namespace

struct g3pcf_plan_s {
    int nbins, lmax, los_mode;
    double rmin, rmax, box;
    cudaStream_t stream = nullptr;
    int device = -1, nsm = 0;
    Bins bins{};
    int RL = 0, RLP = 0, nrp = 0;
    std::vector<int> colmap;
    std::vector<float> colscale;
    std::vector<int4> colconv;     // Chebyshev-form columns (pair-list path)
    std::vector<float> colcoef;
    std::vector<double> colcoef64;  // the same coefficients in FP64 (double-float path)
    std::vector<float2> colcoefdf;  // ... as head + tail FP32 pairs (uploaded)
    std::vector<int4> slotconv;    // the transposed connection (pair-list adjoint)
    std::vector<float> slotcoef;
    std::vector<double> slotcoef64;
    std::vector<float2> slotcoefdf;
    std::vector<int> monoexp, monoidx;  // monomial-basis tables (k_mono)
    std::vector<int4> monoconv;
    std::vector<double> monocoef;
    int opt_basis = 0;             // G3PCF_OPT_BASIS
    int opt_grad = 0;              // G3PCF_OPT_GRAD_PRECISION (0 double-float, 1 FP32)
    int test_fail_alloc = 0;       // G3PCF_OPT_TEST_FAIL_ALLOC countdown (0: off)
    int test_tc_timeout = 0;       // G3PCF_OPT_TEST_TC_TIMEOUT
    std::vector<Tile> tiles;      // FP32 contraction tiles (edge T)
    std::vector<Tile> tiles_tc;   // tensor-core contraction tiles (edge T_tc)
    std::vector<TcStrip> strips_tc;  // their strips (one or two tiles of a row panel)
    std::vector<int4> bblk;          // per m block: {first A column, width, first bf16 operand column, 0}
    int RLPb = 0;                    // bf16 operand row pitch
    int opt_tc_operands = 0;         // 0: operands formed in the contraction; 1: written by the pair stage when possible
    bool direct_used = false;        // this forward's pair stage wrote the bf16 operands
    int T = 0, T_tc = 0;
    int kflush = 16;
    // device buffers
    DevBuf key_a, key_b, val_a, val_b, hist, hist_off, scan_tmp, pts, pts64, orig, cstart, plist;
    DevBuf small;       // status, queue
    DevBuf counts, A, partials, d_tiles, d_segs, d_segfirst, d_colmap, d_colscale, d_catoff;
    DevBuf d_colconv, d_colcoef, d_bintab_s, d_slotconv, d_slotcoef, d_monoexp, d_monoconv, d_monoidx, d_monocoef;
    DevBuf d_ranges, d_tiles_tc, d_cats, d_mreal, d_V, d_bintab, wrow, d_vblk, d_strips_tc, d_items;
    DevBuf d_bop, d_bblk, d_bcat;
    DevBuf d_slotcoefdf, d_mrealdf, d_Vdf, d_colcoefdf;
    int64_t opt_chunk = 0;   // G3PCF_OPT_CHUNK_ROWS
    // pinned staging for host -> device tables (capturable copies); offset
    // restarts at every forward
    unsigned char* h_stage = nullptr;
    size_t stage_cap = 0, stage_off = 0;
    bool capturing = false;
    int64_t fixed_chunk = -1;  // chunk size frozen for a captured graph
    // CUDA graph of the last G3PCF_F_GRAPH call
    cudaStream_t gstream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<long long> gkey;
    cudaEvent_t gev[2] = {};
    int opt_cells = 0;       // G3PCF_OPT_CELLS_PER_RMAX
    int opt_xref = 0;        // G3PCF_OPT_X_REFINE
    int opt_pair = 0;        // G3PCF_OPT_PAIR_KERNELS
    int64_t opt_list_bytes = 0;  // G3PCF_OPT_LIST_BYTES
    // pair lists (forward, pairlist.cu): per-primary need / base / nchunks,
    // the chunk pool and its bin tags; pinned host copies of need and base
    DevBuf l_need, l_base, l_nch, l_pool, l_tag, l_ord;
    int* h_need = nullptr;
    int* h_base = nullptr;
    size_t h_list_cap = 0;
    // graph capture of the list path: per A-chunk {total chunks, largest need} of
    // the uncaptured warm-up run, consumed in order by the capture run
    std::vector<std::pair<int64_t, int64_t>> gl_warm;
    size_t gl_idx = 0;
    bool warm_for_graph = false;
    bool exact_alm = false;  // this forward runs with G3PCF_F_KEEP_ALM
    int gl_events = 0;  // events the capture run will record
    DevBuf l_gbase, l_scantmp, l_passq;
    // events around every k_scan / k_accum launch of the last forward (4 per pass)
    std::vector<cudaEvent_t> lev;
    int lev_used = 0;
    // per chunk of primaries: pair stage done, contraction done (stats [1], [2])
    std::vector<cudaEvent_t> cev;
    int cev_used = 0;
    bool last_chunked = false;
    std::vector<unsigned char> bintab;  // r^2 -> bin lookup (see compute_bins)
    std::vector<signed char> bintab_s;  // signed form (pair-list scan)
    float bin_tscale = 0.f;
    // index state of the last forward (for the adjoint pair pass)
    bool last_plist = false;
    int* h_status = nullptr;
    cudaEvent_t ev[5] = {};
    bool consts_uploaded = false;
    // state of the last forward
    bool have_forward = false;
    bool have_alm = false;
    int64_t last_n = 0, last_np = 0;
    int last_ncat = 0;
    std::vector<int64_t> last_offs;  // catalog offsets of the last forward
    const void* last_pos = nullptr;
    const float* last_w = nullptr;
    int last_pos_f64 = 0;
    Grid last_grid{};
    unsigned* key_sorted = nullptr;
    double stats[15] = {};
    int launches = 0;
};

namespace {

// FP64 values as head + tail FP32 pairs (head = the nearest float, tail = the
// nearest float to the remainder): ~48 significant bits.
std::vector<float2> to_df(const std::vector<double>& v) {
    std::vector<float2> out(v.size());
    for (size_t k = 0; k < v.size(); ++k) {
        const float h = (float)v[k];
        out[k] = float2{h, (float)(v[k] - (double)h)};
    }
    return out;
}

// Copy a host table to the device through the plan's pinned staging buffer
// so that the copy can be captured into a CUDA graph (replays read the same
// staging bytes, which the capturing call has filled).
int upload(g3pcf_plan_t P, void* dev, const void* host, size_t bytes, cudaStream_t st) {
    if (bytes == 0) return 0;
    const size_t off = (P->stage_off + 255) & ~(size_t)255;
    if (off + bytes > P->stage_cap) {
        if (P->capturing)
            return fail(G3PCF_ERR_CUDA, "staging buffer too small during graph capture");
        // a fresh buffer: the old one may still be read by copies in flight
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(G3PCF_ERR_CUDA, "cudaStreamSynchronize: %s", cudaGetErrorString(e));
        if (P->h_stage) cudaFreeHost(P->h_stage);
        P->h_stage = nullptr;
        size_t cap = (off + bytes) * 2 + 65536;
        if (cudaHostAlloc(reinterpret_cast<void**>(&P->h_stage), cap, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            P->stage_cap = 0;
            return fail(G3PCF_ERR_ALLOC, "pinned staging allocation failed");
        }
        P->stage_cap = cap;
    }
    std::memcpy(P->h_stage + off, host, bytes);
    P->stage_off = off + bytes;
    cudaError_t e = cudaMemcpyAsync(dev, P->h_stage + off, bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(G3PCF_ERR_CUDA, "cudaMemcpyAsync: %s", cudaGetErrorString(e));
    return 0;
}

#define UP(dev, host, bytes)                                     \
    do {                                                         \
        if (int r_ = upload(P, (dev), (host), (bytes), st)) return r_; \
    } while (0)

int setup_device(g3pcf_plan_t P) {
    if (P->device >= 0) return 0;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, dev));
    P->device = dev;
    P->nsm = prop.multiProcessorCount;
    CK(cudaHostAlloc(reinterpret_cast<void**>(&P->h_status), 64, cudaHostAllocDefault));
    for (auto& e : P->ev) CK(cudaEventCreate(&e));
    return 0;
}

int upload_consts(g3pcf_plan_t P) {
    if (P->consts_uploaded) return 0;
    if (P->d_colmap.ensure(P->RL * sizeof(int)) || P->d_colscale.ensure(P->RL * sizeof(float)) ||
        P->d_tiles.ensure(P->tiles.size() * sizeof(Tile)) ||
        P->d_tiles_tc.ensure(P->tiles_tc.size() * sizeof(Tile)))
        return fail(G3PCF_ERR_ALLOC, "workspace allocation failed (constants)");
    CK(cudaMemcpy(P->d_tiles_tc.p, P->tiles_tc.data(), P->tiles_tc.size() * sizeof(Tile),
                  cudaMemcpyHostToDevice));
    if (!P->bblk.empty()) {
        if (P->d_bblk.ensure(P->bblk.size() * sizeof(int4)))
            return fail(G3PCF_ERR_ALLOC, "workspace allocation failed (constants)");
        CK(cudaMemcpy(P->d_bblk.p, P->bblk.data(), P->bblk.size() * sizeof(int4), cudaMemcpyHostToDevice));
    }
    if (P->d_strips_tc.ensure(P->strips_tc.size() * sizeof(TcStrip)))
        return fail(G3PCF_ERR_ALLOC, "workspace allocation failed (constants)");
    CK(cudaMemcpy(P->d_strips_tc.p, P->strips_tc.data(), P->strips_tc.size() * sizeof(TcStrip),
                  cudaMemcpyHostToDevice));
    if (P->d_bintab.ensure(P->bintab.size()) || P->d_bintab_s.ensure(P->bintab_s.size()))
        return fail(G3PCF_ERR_ALLOC, "workspace allocation failed (bin table)");
    CK(cudaMemcpy(P->d_bintab.p, P->bintab.data(), P->bintab.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->d_bintab_s.p, P->bintab_s.data(), P->bintab_s.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->d_colmap.p, P->colmap.data(), P->RL * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->d_colscale.p, P->colscale.data(), P->RL * sizeof(float), cudaMemcpyHostToDevice));
    if (P->d_colconv.ensure(P->colconv.size() * sizeof(int4)) ||
        P->d_colcoef.ensure(P->colcoef.size() * sizeof(float)))
        return fail(G3PCF_ERR_ALLOC, "workspace allocation failed (constants)");
    CK(cudaMemcpy(P->d_colconv.p, P->colconv.data(), P->colconv.size() * sizeof(int4), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->d_colcoef.p, P->colcoef.data(), P->colcoef.size() * sizeof(float), cudaMemcpyHostToDevice));
    if (P->d_slotconv.ensure(P->slotconv.size() * sizeof(int4)) ||
        P->d_slotcoef.ensure(P->slotcoef.size() * sizeof(float)))
        return fail(G3PCF_ERR_ALLOC, "workspace allocation failed (constants)");
    CK(cudaMemcpy(P->d_slotconv.p, P->slotconv.data(), P->slotconv.size() * sizeof(int4), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->d_slotcoef.p, P->slotcoef.data(), P->slotcoef.size() * sizeof(float), cudaMemcpyHostToDevice));
    // the double-float path's coefficients as head + tail FP32 pairs
    P->colcoefdf = to_df(P->colcoef64);
    P->slotcoefdf = to_df(P->slotcoef64);
    if (P->d_colcoefdf.ensure(P->colcoefdf.size() * sizeof(float2)) ||
        P->d_slotcoefdf.ensure(P->slotcoefdf.size() * sizeof(float2)))
        return fail(G3PCF_ERR_ALLOC, "workspace allocation failed (constants)");
    CK(cudaMemcpy(P->d_colcoefdf.p, P->colcoefdf.data(), P->colcoefdf.size() * sizeof(float2), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->d_slotcoefdf.p, P->slotcoefdf.data(), P->slotcoefdf.size() * sizeof(float2),
                  cudaMemcpyHostToDevice));
    if (P->d_monoexp.ensure(P->monoexp.size() * sizeof(int)) || P->d_monoconv.ensure(P->monoconv.size() * sizeof(int4)) ||
        P->d_monoidx.ensure(P->monoidx.size() * sizeof(int)) || P->d_monocoef.ensure(P->monocoef.size() * sizeof(double)))
        return fail(G3PCF_ERR_ALLOC, "workspace allocation failed (constants)");
    CK(cudaMemcpy(P->d_monoexp.p, P->monoexp.data(), P->monoexp.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->d_monoconv.p, P->monoconv.data(), P->monoconv.size() * sizeof(int4), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->d_monoidx.p, P->monoidx.data(), P->monoidx.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->d_monocoef.p, P->monocoef.data(), P->monocoef.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->d_tiles.p, P->tiles.data(), P->tiles.size() * sizeof(Tile),
                  cudaMemcpyHostToDevice));
    P->consts_uploaded = true;
    return 0;
}

// Cell grid for a (pair-weighted) density: cell side >= rmax/s with s chosen
// so that a cell holds a few dozen points.
Grid choose_grid(g3pcf_plan_t P, double density, int ncat) {
    Grid g{};
    const double target = 48.0;
    double cs = std::cbrt(target / (density > 0 ? density : 1e-30));
    int s = (int)std::floor(P->rmax / cs);
    if (s < 1) s = 1;
    if (s > 8) s = 8;
    if (P->opt_cells > 0) s = P->opt_cells;
    int nc = (int)std::floor(P->box * s / P->rmax);
    if (nc < 1) nc = 1;
    if (nc > 256) nc = 256;
    int fx = P->opt_xref > 0 ? P->opt_xref : 8;
    for (;;) {  // keys stay below 2^31: coarsen x first, then the whole grid
        int span = 1;
        while (span < nc) span <<= 1;
        long long cpc = (long long)span * span * nc * fx;
        if ((long long)ncat * cpc < (1ll << 31) || (nc == 1 && fx == 1)) {
            g.span = span;
            g.cells_per_cat = cpc;
            break;
        }
        if (fx > 1)
            fx = fx / 2;
        else
            nc = nc / 2;
    }
    g.nc = nc;
    g.ncx = nc * fx;
    g.boxd = P->box;
    g.box = (float)P->box;
    g.cell = (float)(P->box / nc);
    g.inv_cell = (float)(nc / P->box);
    g.inv_cellx = (float)(g.ncx / P->box);
    g.reach = (int)std::ceil(P->rmax * nc / P->box - 1e-9);
    if (g.reach < 1) g.reach = 1;
    g.periodic = (P->los_mode == G3PCF_LOS_Z_PERIODIC);
    g.radial = (P->los_mode == G3PCF_LOS_RADIAL_OPEN);
    return g;
}

void compute_bins(g3pcf_plan_t P) {
    Bins& b = P->bins;
    const int B = P->nbins;
    b.nbins = B;
    for (int k = 0; k <= B; ++k) {
        double e;
        if (k == 0) e = P->rmin;
        else if (k == B) e = P->rmax;
        else e = P->rmin + ((P->rmax - P->rmin) * (double)k) / (double)B;
        b.e2[k] = e * e;
        b.e2f[k] = (float)(e * e);
    }
    // Bound on |r2_fp32 - r2_exact| near an edge e: separation error per axis
    // dD <= u (4L + rmax) (input rounding to FP32, image shift, subtraction),
    // r2 error <= 2 sqrt(3) e dD + 3 dD^2 + ~6 u e^2 (products, FMA chain,
    // FP32 edge and the comparison); doubled for safety.
    const double u = std::ldexp(1.0, -24);
    const double dD = u * (4.0 * P->box + P->rmax);
    for (int k = 0; k <= B; ++k) {
        const double e = std::sqrt(b.e2[k]);
        b.guard[k] = (float)(2.0 * (2.0 * std::sqrt(3.0) * e * dD + 3.0 * dD * dD + 6.0 * u * e * e));
    }
    b.rmin = (float)P->rmin;
    b.invw = (float)(B / (P->rmax - P->rmin));
    b.rmaxf = (float)P->rmax;
    b.rmax2f = (float)(P->rmax * P->rmax);
    b.hi_rej = b.e2f[B] + b.guard[B];
    b.lo_rej = b.e2f[0] - b.guard[0];
    b.slack = (float)(1e-4 * P->box / 1.0 + 1e-3 * P->rmax);
    // r^2 -> bin table over [0, e_B^2): cell t covers [t D, (t+1) D).  An entry
    // names bin b only if the cell, widened by 1% of a cell on each side (far
    // more than the FP32 error of the kernel's index r2 * T / e_B^2), lies
    // inside b's decided interval (e_b^2 + g_b, e_{b+1}^2 - g_{b+1}); 254 if it
    // lies below e_0^2 - g_0 (surely outside); 255 otherwise (checked per pair).
    const int T = G3_BIN_TABLE;
    P->bintab.assign(T + 2, 255);
    const double r2max = b.e2[B];
    P->bin_tscale = (float)(T / r2max);
    const double D = r2max / T;
    for (int t = 0; t < T + 2; ++t) {
        const double lo = (t - 0.01) * D, hi = (t + 1.01) * D;
        if (hi < b.e2[0] - b.guard[0] && lo >= 0.0) {
            P->bintab[t] = 254;
            continue;
        }
        for (int k = 0; k < B; ++k)
            if (lo > b.e2[k] + b.guard[k] && hi < b.e2[k + 1] - b.guard[k + 1]) {
                P->bintab[t] = (unsigned char)k;
                break;
            }
    }
    // Signed form for the pair-list scan: bin, -1 surely outside (also every
    // cell from e_B^2 + g_B up, so the last entry takes all larger r^2), -3 check.
    P->bintab_s.assign(T + 2, -3);
    for (int t = 0; t < T + 2; ++t) {
        const double lo = (t - 0.01) * D, hi = (t + 1.01) * D;
        const unsigned char v = P->bintab[t];
        if (v == 254 || lo > b.e2[B] + b.guard[B])
            P->bintab_s[t] = -1;
        else if (v < 254)
            P->bintab_s[t] = (signed char)v;
    }
}

// Column map of an A row: block m (m = 0: K_0 reals; m >= 1: Re and Im halves)
// and the normalisation K_lm of Y_lm.
// Coefficients c_k of the monic D_{m+n,m}(z) = sum_k c_k T_k(z) (Chebyshev
// polynomials of the first kind), k = 0..n.  D follows the monic recurrence
// D_{l+1} = z D_l - (l^2 - m^2)/(4 l^2 - 1) D_{l-1}; both sides are expanded in
// powers of z (FP64) and the T_k are peeled off from the top degree down.
// Powers-of-z coefficients of the monic D_{m+n,m}(z) (degree n), from the
// recurrence D_{l+1} = z D_l - (l^2 - m^2)/(4 l^2 - 1) D_{l-1}, FP64.
std::vector<double> monic_poly(int m, int n) {
    std::vector<double> d0(n + 1, 0.0), d1(n + 1, 0.0);
    d0[0] = 1.0;
    if (n >= 1) d1[1] = 1.0;
    std::vector<double> D = n == 0 ? d0 : d1;
    for (int l = m + 1; l < m + n; ++l) {
        const double beta = double(l * l - m * m) / double(4 * l * l - 1);
        std::vector<double> d2(n + 1, 0.0);
        for (int d = 0; d <= n; ++d) d2[d] = (d > 0 ? d1[d - 1] : 0.0) - beta * d0[d];
        d0 = d1;
        d1 = d2;
        D = d2;
    }
    return D;
}

std::vector<double> cheb_coeffs(int m, int n) {
    std::vector<std::vector<double>> T(n + 1, std::vector<double>(n + 1, 0.0));
    T[0][0] = 1.0;
    if (n >= 1) T[1][1] = 1.0;
    for (int k = 1; k < n; ++k)
        for (int d = 0; d <= n; ++d)
            T[k + 1][d] = (d > 0 ? 2.0 * T[k][d - 1] : 0.0) - T[k - 1][d];
    std::vector<double> D = monic_poly(m, n);
    std::vector<double> c(n + 1, 0.0);
    for (int k = n; k >= 0; --k) {
        c[k] = D[k] / T[k][k];
        for (int d = 0; d <= k; ++d) D[d] -= c[k] * T[k][d];
    }
    return c;
}

void compute_columns(g3pcf_plan_t P) {
    const int B = P->nbins, L = P->lmax;
    P->nrp = pair_nrp(L);
    P->RL = B * (L + 1) * (L + 1);
    P->RLP = (P->RL + 7) & ~7;
    P->colmap.assign(P->RL, 0);
    P->colscale.assign(P->RL, 0.f);
    P->colconv.assign(P->RL, int4{0, 0, 0, 0});
    P->colcoef.clear();
    P->colcoef64.clear();
    // coefficient rows (times K_lm) per (l, m), shared by the bins and parts
    std::vector<int> coef_off((L + 1) * (L + 1), 0);
    for (int m = 0; m <= L; ++m)
        for (int l = m; l <= L; ++l) {
            const double lnN = 0.5 * (std::log((2.0 * l + 1.0) / (4.0 * M_PI)) + lfact(l - m) - lfact(l + m));
            const double lnLead = lfact(2 * l) - l * std::log(2.0) - lfact(l) - lfact(l - m);
            double kl = std::exp(lnN + lnLead);
            if (m & 1) kl = -kl;
            coef_off[l * (L + 1) + m] = (int)P->colcoef.size();
            for (double ck : cheb_coeffs(m, l - m)) {
                P->colcoef.push_back((float)(ck * kl));
                P->colcoef64.push_back(ck * kl);
            }
        }
    int col = 0;
    for (int m = 0; m <= L; ++m) {
        const int K = B * (L + 1 - m);
        const int parts = m == 0 ? 1 : 2;
        for (int part = 0; part < parts; ++part)
            for (int idx = 0; idx < K; ++idx) {
                const int l = m + idx / B, b = idx % B;
                const int slot = (m == 0) ? l : acc_base(L, m) + 2 * (l - m) + part;
                // K_lm = (-1)^m sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) (2l)! / (2^l l! (l-m)!)
                const double lnN = 0.5 * (std::log((2.0 * l + 1.0) / (4.0 * M_PI)) + lfact(l - m) - lfact(l + m));
                const double lnLead = lfact(2 * l) - l * std::log(2.0) - lfact(l) - lfact(l - m);
                double kl = std::exp(lnN + lnLead);
                if (m & 1) kl = -kl;
                P->colmap[col] = b * P->nrp + slot;
                P->colscale[col] = (float)kl;
                const int slot0 = (m == 0) ? 0 : acc_base(L, m) + part;
                P->colconv[col] = int4{b * P->nrp + slot0, m == 0 ? 1 : 2, l - m + 1, coef_off[l * (L + 1) + m]};
                ++col;
            }
    }
    // adjoint: per accumulator slot (m, k, part) the A columns (l = m + n, n = k..L-m,
    // stride B from bin 0) and coefficients c^(m)_{n,k} K_lm of the transposed connection
    const int NR = (L + 1) * (L + 1);
    P->slotconv.assign(NR, int4{0, 0, 0, 0});
    P->slotcoef.clear();
    P->slotcoef64.clear();
    int colm = 0;
    for (int m = 0; m <= L; ++m) {
        const int K = B * (L + 1 - m);
        for (int part = 0; part < (m == 0 ? 1 : 2); ++part)
            for (int k = 0; k <= L - m; ++k) {
                const int slot = (m == 0) ? k : acc_base(L, m) + 2 * k + part;
                P->slotconv[slot] = int4{colm + part * K + k * B, B, L - m - k + 1, (int)P->slotcoef.size()};
                for (int nn = k; nn <= L - m; ++nn) {
                    const int l = m + nn;
                    const double lnN = 0.5 * (std::log((2.0 * l + 1.0) / (4.0 * M_PI)) + lfact(l - m) - lfact(l + m));
                    const double lnLead = lfact(2 * l) - l * std::log(2.0) - lfact(l) - lfact(l - m);
                    double kl = std::exp(lnN + lnLead);
                    if (m & 1) kl = -kl;
                    P->slotcoef.push_back((float)(cheb_coeffs(m, nn)[k] * kl));
                    P->slotcoef64.push_back(cheb_coeffs(m, nn)[k] * kl);
                }
            }
        colm += (m == 0) ? K : 2 * K;
    }
    // monomial basis (Sec. 3.3.2): monomial (a, b, c), a + b + c <= L, in a fixed
    // order; per (l, m, part) the terms K_lm d_k C(m, j) Re / Im(i^j) of a_lm on
    // M_{m-j, j, k}
    P->monoexp.clear();
    std::vector<int> mindex((L + 1) * (L + 1) * (L + 1), -1);
    for (int a = 0; a <= L; ++a)
        for (int bb = 0; a + bb <= L; ++bb)
            for (int c = 0; a + bb + c <= L; ++c) {
                mindex[(a * (L + 1) + bb) * (L + 1) + c] = (int)P->monoexp.size();
                P->monoexp.push_back(a | (bb << 8) | (c << 16));
            }
    P->monoconv.assign(NR, int4{0, 0, 0, 0});
    P->monoidx.clear();
    P->monocoef.clear();
    colm = 0;
    int u = 0;
    for (int m = 0; m <= L; ++m) {
        const int K = B * (L + 1 - m);
        for (int part = 0; part < (m == 0 ? 1 : 2); ++part)
            for (int l = m; l <= L; ++l) {
                const double lnN = 0.5 * (std::log((2.0 * l + 1.0) / (4.0 * M_PI)) + lfact(l - m) - lfact(l + m));
                const double lnLead = lfact(2 * l) - l * std::log(2.0) - lfact(l) - lfact(l - m);
                double kl = std::exp(lnN + lnLead);
                if (m & 1) kl = -kl;
                const std::vector<double> d = monic_poly(m, l - m);
                const int first = (int)P->monoidx.size();
                for (int k = 0; k <= l - m; ++k) {
                    if (d[k] == 0.0) continue;
                    double binom = 1.0;  // C(m, j)
                    for (int j = 0; j <= m; ++j) {
                        if (j > 0) binom = binom * (m - j + 1) / j;
                        // i^j: 1, i, -1, -i
                        const int r = j % 4;
                        double f = 0.0;
                        if (part == 0 && (r == 0 || r == 2)) f = r == 0 ? 1.0 : -1.0;
                        if (part == 1 && (r == 1 || r == 3)) f = r == 1 ? 1.0 : -1.0;
                        if (f == 0.0) continue;
                        P->monoidx.push_back(mindex[((m - j) * (L + 1) + j) * (L + 1) + k]);
                        P->monocoef.push_back(kl * d[k] * binom * f);
                    }
                }
                P->monoconv[u++] = int4{first, (int)P->monoidx.size() - first, colm + part * K + (l - m) * B, 0};
            }
        colm += (m == 0) ? K : 2 * K;
    }
}

int64_t zsize_of(int nbins, int lmax) {
    int64_t s = 0;
    for (int m = 0; m <= lmax; ++m) {
        const int64_t K = (int64_t)nbins * (lmax + 1 - m);
        s += K * K;
    }
    return s;
}

struct CallSpec {
    const void* pos;
    const float* w;
    int64_t n;
    int64_t n_primary;
    int pos_f64;
    int ncat;
    std::vector<int64_t> offs;  // ncat + 1 (host)
    double* zeta;
    int64_t* counts;
    int flags;
};

int ensure(g3pcf_plan_t P, DevBuf& b, size_t bytes, const char* what) {
    // test hook (G3PCF_OPT_TEST_FAIL_ALLOC): the k-th workspace growth fails once
    if (P->test_fail_alloc > 0 && !(bytes <= b.bytes && b.p) && --P->test_fail_alloc == 0)
        return fail(G3PCF_ERR_ALLOC, "injected allocation failure (%s, %zu bytes)", what, bytes);
    if (b.ensure(bytes)) return fail(G3PCF_ERR_ALLOC, "cudaMalloc of %zu bytes (%s) failed", bytes, what);
    return 0;
}

int read_status(g3pcf_plan_t P) {
    int s = P->h_status[0];
    if (s & kStatusRange)
        return fail(G3PCF_ERR_RANGE, "a position is outside [0, box) or not finite, or a weight is not finite");
    if (s & kStatusTimeout) return fail(G3PCF_ERR_TIMEOUT, "a bounded device wait expired");
    if (s & kStatusOverflow) return fail(G3PCF_ERR_CUDA, "device-side capacity exceeded");
    return G3PCF_OK;
}

// Device-planned passes of a captured forward over a pool of C chunks, for a
// warm-up run that needed `total` chunks with `most` for one primary: stride
// between pass bases, slack for the primary that straddles a pass end, passes.
void graph_plan_sizes(int64_t C, int64_t total, int64_t most, int nbins, int64_t& slack, int64_t& stride,
                      int& npass) {
    slack = std::min<int64_t>(C / 2, 2 * most + nbins + 64);
    stride = C - slack;
    npass = stride > 0 ? (int)((total + total / 4 + stride - 1) / stride) + 1 : 0;
}

int ensure_events(g3pcf_plan_t P, int n) {
    while ((int)P->lev.size() < n) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        P->lev.push_back(e);
    }
    return 0;
}

// Forward pair stage through pair lists for the primaries [pa.q0, pa.nprim):
// count candidates, bring the per-primary chunk bounds to the host, split the
// range into passes whose lists fit the pool, then scan + accumulate each pass.
int run_pair_lists(g3pcf_plan_t P, const PairArgs& pa, cudaStream_t st, int mode = 0) {
    const int qa = pa.q0, qb = pa.nprim;
    const int64_t nq = (int64_t)qb - qa;
    if (nq <= 0) return G3PCF_OK;
    if (ensure(P, P->l_need, 4 * (size_t)qb, "pair-list bounds") ||
        ensure(P, P->l_base, 4 * (size_t)qb, "pair-list bounds") ||
        ensure(P, P->l_nch, 4 * (size_t)qb, "pair-list bounds"))
        return G3PCF_ERR_ALLOC;
    if ((size_t)nq > P->h_list_cap) {
        if (P->h_need) cudaFreeHost(P->h_need);
        if (P->h_base) cudaFreeHost(P->h_base);
        P->h_need = P->h_base = nullptr;
        P->h_list_cap = 0;
        if (cudaHostAlloc(reinterpret_cast<void**>(&P->h_need), 4 * nq, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc(reinterpret_cast<void**>(&P->h_base), 4 * nq, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return fail(G3PCF_ERR_ALLOC, "pinned host allocation of %lld bytes failed", (long long)(8 * nq));
        }
        P->h_list_cap = (size_t)nq;
    }
    ListArgs la{};
    la.pts = pa.pts;
    la.pts64 = pa.pts64;
    la.orig = pa.orig;
    la.cstart = pa.cstart;
    la.plist = pa.plist;
    la.key = pa.key;
    la.q0 = pa.q0;
    la.chunked = pa.chunked;
    la.wrow = pa.wrow;
    la.A = pa.A;
    la.RLP = pa.RLP;
    la.colconv = P->d_colconv.as<int4>();
    la.colcoef = P->d_colcoef.as<float>();
    la.RL = pa.RL;
    la.counts = pa.counts;
    la.queue = pa.queue;
    la.status = pa.status;
    la.bintab = P->d_bintab_s.as<signed char>();
    la.bin_tscale = pa.bin_tscale;
    la.g = pa.g;
    la.bins = pa.bins;
    // multipoles that will be differentiated take the exact image separations and,
    // unless the FP32 form is asked for, the double-float kernels (precise.cu)
    la.exact_img = (mode >= 1 || P->exact_alm) ? 1 : 0;
    la.precise = (la.exact_img && P->opt_grad == 0) ? 1 : 0;
    la.colcoefdf = P->d_colcoefdf.as<float2>();
    la.slotcoefdf = P->d_slotcoefdf.as<float2>();
    la.monoexp = P->d_monoexp.as<int>();
    la.monoconv = P->d_monoconv.as<int4>();
    la.monoidx = P->d_monoidx.as<int>();
    la.monocoef = P->d_monocoef.as<double>();
    if (mode >= 1) {
        la.V = pa.V;
        la.dw = pa.dw;
        la.dpos = pa.dpos;
        la.slotconv = P->d_slotconv.as<int4>();
        la.slotcoef = P->d_slotcoef.as<float>();
        la.Vdf = P->d_Vdf.as<float2>();
    }
    la.need = P->l_need.as<int>();
    la.base = P->l_base.as<int>();
    la.nchunks = P->l_nch.as<int>();
    la.qa = qa;
    la.qb = qb;
    la.ncand = reinterpret_cast<unsigned long long*>(pa.status + 24);  // zeroed with the status word
    la.bop = nullptr;
    if (mode == 0 && pa.bop && !la.precise && P->opt_basis == 0 && !P->capturing) {
        la.bop = pa.bop;
        la.nbcat = pa.nbcat;
        la.bop_pitch = pa.bop_pitch;
        la.bblk = pa.bblk;
        la.nblk = pa.nblk;
        la.bcat = pa.bcat;
    }
    if (P->capturing) {
        // no host round trip inside a graph: plan the passes on the device from
        // the pool the warm-up run sized (sizes of that run, same A-chunk order)
        if (P->gl_idx >= P->gl_warm.size())
            return fail(G3PCF_ERR_STATE, "graph capture without a matching warm-up forward");
        const std::pair<int64_t, int64_t> wm = P->gl_warm[P->gl_idx++];
        const int64_t C = (int64_t)(P->l_pool.bytes / 128);
        int64_t slack = 0, stride = 0;
        int npass = 0;
        graph_plan_sizes(C, wm.first, wm.second, P->nbins, slack, stride, npass);
        if (stride < 1 || (int64_t)P->l_tag.bytes / 4 < C || (int64_t)P->l_ord.bytes / 4 < C ||
            P->l_gbase.bytes < 8 * (size_t)nq || P->l_passq.bytes < 4 * (size_t)(npass + 1) ||
            P->l_scantmp.bytes < plan_scan_tmp_bytes(nq) || (int)P->lev.size() < P->lev_used + 4 * npass) {
            ++P->launches;  // the warm-up did not size the plan (cannot happen): the fused kernel
            if (launch_pair(P->lmax, pa, P->nsm, st) != 0)
                return fail(G3PCF_ERR_CUDA, "pair kernel launch failed: %s", cudaGetErrorString(cudaGetLastError()));
            return G3PCF_OK;
        }
        la.chunks = P->l_pool.as<int>();
        la.tag = P->l_tag.as<int>();
        la.ord = P->l_ord.as<int>();
        ++P->launches;
        if (launch_count(la, P->nsm, st) != 0)
            return fail(G3PCF_ERR_CUDA, "pair count launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        P->launches += 5;
        if (launch_plan(la.need, P->l_gbase.as<long long>(), P->l_scantmp.as<long long>(), qa, qb, stride,
                        (int)slack, npass, P->l_base.as<int>(), P->l_passq.as<int>(), pa.status, st) != 0)
            return fail(G3PCF_ERR_CUDA, "pair-list plan launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        for (int k = 0; k < npass; ++k) {
            la.qrange = P->l_passq.as<int>() + k;
            cudaEvent_t* ev = P->lev.data() + P->lev_used;
            P->lev_used += 4;
            CK(cudaMemsetAsync(la.queue, 0, sizeof(int), st));
            P->launches += 2;
            CK(cudaEventRecord(ev[0], st));
            if (launch_scan(la, P->nsm, st) != 0)
                return fail(G3PCF_ERR_CUDA, "pair scan launch failed: %s", cudaGetErrorString(cudaGetLastError()));
            CK(cudaEventRecord(ev[1], st));
            CK(cudaMemsetAsync(la.queue, 0, sizeof(int), st));
            CK(cudaEventRecord(ev[2], st));
            if ((P->opt_basis == 1 ? launch_mono(P->lmax, la, P->nsm, st) : launch_accum(P->lmax, la, P->nsm, st)) != 0)
                return fail(G3PCF_ERR_CUDA, "pair accumulate launch failed: %s", cudaGetErrorString(cudaGetLastError()));
            CK(cudaEventRecord(ev[3], st));
        }
        P->stats[10] += (double)npass;
        return G3PCF_OK;
    }
    ++P->launches;
    if (launch_count(la, P->nsm, st) != 0)
        return fail(G3PCF_ERR_CUDA, "pair count launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    CK(cudaMemcpyAsync(P->h_need, la.need + qa, 4 * nq, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(P->h_status + 8, la.ncand, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(P->h_status + 12, pa.status + kNegWeightSlot, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    P->stats[9] = (double)*reinterpret_cast<unsigned long long*>(P->h_status + 8);
    // the bf16 operands are sqrt(w) A: with a negative weight the contraction
    // forms its operands from the FP32 rows instead
    if (la.bop && P->h_status[12] != 0) la.bop = nullptr;
    la.skip_a = (la.bop && !P->exact_alm) ? 1 : 0;
    if (mode == 0) P->direct_used = la.bop != nullptr;
    // pool capacity (per chunk: 128 bytes of entries, a tag and a list int)
    int64_t total = 0, most = 0;
    for (int64_t k = 0; k < nq; ++k) {
        total += P->h_need[k];
        most = std::max<int64_t>(most, P->h_need[k]);
    }
    double budget = (double)P->opt_list_bytes;
    if (budget <= 0) {
        size_t fr = 0, tot = 0;
        CK(cudaMemGetInfo(&fr, &tot));
        budget = 0.4 * (double)(fr + P->l_pool.bytes + P->l_tag.bytes + P->l_ord.bytes);
        if (budget > 32e9) budget = 32e9;
    }
    int64_t cap = (int64_t)(budget / 136.0);
    if (cap > ((int64_t)1 << 30)) cap = (int64_t)1 << 30;
    P->gl_warm.emplace_back(total, most);
    // a warm-up for a graph capture keeps headroom for the device-planned passes
    const int64_t want = P->warm_for_graph ? total + total / 4 + 2 * most + P->nbins + 64 : total;
    if (cap > want) cap = want;
    if (cap < most)
        return fail(G3PCF_ERR_ALLOC, "pair lists of one primary (%lld chunks) exceed the list budget (%lld)",
                    (long long)most, (long long)cap);
    if (cap > 0 && (ensure(P, P->l_pool, 128 * (size_t)cap, "pair lists") ||
                    ensure(P, P->l_tag, 4 * (size_t)cap, "pair lists") ||
                    ensure(P, P->l_ord, 4 * (size_t)cap, "pair lists")))
        return G3PCF_ERR_ALLOC;
    la.chunks = P->l_pool.as<int>();
    la.tag = P->l_tag.as<int>();
    la.ord = P->l_ord.as<int>();
    if (P->warm_for_graph && cap > 0) {  // what the capture run will need (no allocation while capturing)
        int64_t slack = 0, stride = 0;
        int npass = 0;
        graph_plan_sizes(cap, total, most, P->nbins, slack, stride, npass);
        if (ensure(P, P->l_gbase, 8 * (size_t)nq, "pair-list plan") ||
            ensure(P, P->l_scantmp, plan_scan_tmp_bytes(nq), "pair-list plan") ||
            ensure(P, P->l_passq, 4 * (size_t)(npass + 1), "pair-list plan"))
            return G3PCF_ERR_ALLOC;
        P->gl_events += 4 * npass;
        if (int r = ensure_events(P, P->gl_events)) return r;
    }
    std::vector<int> cuts{qa};
    int64_t acc = 0;
    for (int64_t k = 0; k < nq; ++k) {
        if (acc + P->h_need[k] > cap) {
            cuts.push_back(qa + (int)k);
            acc = 0;
        }
        P->h_base[k] = (int)acc;
        acc += P->h_need[k];
    }
    cuts.push_back(qb);
    CK(cudaMemcpyAsync(P->l_base.as<int>() + qa, P->h_base, 4 * nq, cudaMemcpyHostToDevice, st));
    for (size_t k = 0; k + 1 < cuts.size(); ++k) {
        la.qa = cuts[k];
        la.qb = cuts[k + 1];
        if (la.qb <= la.qa) continue;
        if (int r = ensure_events(P, P->lev_used + 4)) return r;
        cudaEvent_t* ev = P->lev.data() + P->lev_used;
        P->lev_used += 4;
        CK(cudaMemsetAsync(la.queue, 0, sizeof(int), st));
        ++P->launches;
        CK(cudaEventRecord(ev[0], st));
        if (launch_scan(la, P->nsm, st) != 0)
            return fail(G3PCF_ERR_CUDA, "pair scan launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        CK(cudaEventRecord(ev[1], st));
        CK(cudaMemsetAsync(la.queue, 0, sizeof(int), st));
        ++P->launches;
        CK(cudaEventRecord(ev[2], st));
        if (mode == 2) {
            // recompute: the chunk-local multipole rows of this pass, their V = M A and
            // primary-weight terms, then the adjoint pair pass over the same lists
            P->launches += 2;
            int vr = launch_accum(P->lmax, la, P->nsm, st);
            if (vr == 0)
                vr = la.precise ? launch_vgemm_rows_df(la.A, la.RLP, la.RL, la.qa - la.q0, la.qb - la.q0,
                                                      P->d_mrealdf.as<float2>(), P->nbins, P->lmax,
                                                      P->d_Vdf.as<float2>(), pa.dw, la.plist, la.orig, la.q0, st)
                                : launch_vgemm_rows(la.A, la.RLP, la.RL, la.qa - la.q0, la.qb - la.q0,
                                                    P->d_mreal.as<float>(), P->nbins, P->lmax, P->d_V.as<float>(),
                                                    pa.dw, la.plist, la.orig, la.q0, st);
            if (vr != 0)
                return fail(G3PCF_ERR_CUDA, "adjoint recompute launch failed: %s", cudaGetErrorString(cudaGetLastError()));
            CK(cudaMemsetAsync(la.queue, 0, sizeof(int), st));
        }
        if ((mode >= 1 ? launch_adj(P->lmax, la, P->nsm, st)
                       : (P->opt_basis == 1 ? launch_mono(P->lmax, la, P->nsm, st)
                                            : launch_accum(P->lmax, la, P->nsm, st))) != 0)
            return fail(G3PCF_ERR_CUDA, "pair accumulate launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        CK(cudaEventRecord(ev[3], st));
    }
    P->stats[10] += (double)(cuts.size() - 1);
    return G3PCF_OK;
}

int run_forward(g3pcf_plan_t P, CallSpec& c) {
    if (int r = setup_device(P)) return r;
    if (int r = upload_consts(P)) return r;
    cudaStream_t st = P->stream;
    const int B = P->nbins;
    const int64_t n = c.n;
    const int64_t zs = zsize_of(B, P->lmax);
    P->have_forward = false;
    P->have_alm = false;
    P->launches = 0;
    P->stats[9] = P->stats[10] = 0.0;
    P->lev_used = 0;
    P->exact_alm = (c.flags & G3PCF_F_KEEP_ALM) != 0;
    if (P->capturing) {
        P->gl_idx = 0;
    } else {
        P->gl_warm.clear();
        P->gl_events = 0;
    }
    P->stage_off = 0;
    P->cev_used = 0;
    CK(cudaEventRecord(P->ev[0], st));
    // zero outputs and counters
    if (ensure(P, P->small, 256, "status")) return G3PCF_ERR_ALLOC;
    int* d_status = P->small.as<int>();
    int* d_queue = d_status + 16;
    CK(cudaMemsetAsync(P->small.p, 0, 256, st));
    if (ensure(P, P->counts, sizeof(unsigned long long) * B * c.ncat + 8, "counts")) return G3PCF_ERR_ALLOC;
    CK(cudaMemsetAsync(P->counts.p, 0, sizeof(unsigned long long) * B * c.ncat, st));
    CK(cudaMemsetAsync(c.zeta, 0, sizeof(double) * 2 * zs * c.ncat, st));
    // density for the grid: pair-weighted over catalogs
    double num = 0, den = 0;
    for (int k = 0; k < c.ncat; ++k) {
        const double nk = (double)(c.offs[k + 1] - c.offs[k]);
        num += nk * nk;
        den += nk;
    }
    const double vol = P->box * P->box * P->box;
    const double density = den > 0 ? num / den / vol : 0.0;
    Grid g = choose_grid(P, density, c.ncat);
    const long long ncells = (long long)c.ncat * g.cells_per_cat;
    P->last_grid = g;
    P->stats[7] = (double)P->rmax / (P->box / g.nc);

    int64_t nprim = 0;
    if (n > 0) {
        // ---- workspace
        const size_t hist_ints = radix_hist_ints(n);
        const size_t off_ints = (hist_ints > (size_t)n ? hist_ints : (size_t)n) + 1;
        if (ensure(P, P->key_a, 4 * n, "keys") || ensure(P, P->key_b, 4 * n, "keys") ||
            ensure(P, P->val_a, 4 * n, "vals") || ensure(P, P->val_b, 4 * n, "vals") ||
            ensure(P, P->hist, 4 * hist_ints, "hist") || ensure(P, P->hist_off, 4 * off_ints, "hist") ||
            ensure(P, P->scan_tmp, 4 * (scan_tmp_ints(off_ints) + 16), "scan") ||
            ensure(P, P->pts, 16 * n, "points") || ensure(P, P->orig, 4 * n, "orig") ||
            ensure(P, P->cstart, 4 * (ncells + 1), "cells") || ensure(P, P->plist, 4 * n, "plist"))
            return G3PCF_ERR_ALLOC;
        if (c.pos_f64 && ensure(P, P->pts64, 24 * n, "points64")) return G3PCF_ERR_ALLOC;
        IndexBuffers ib{};
        ib.key_a = P->key_a.as<unsigned>();
        ib.key_b = P->key_b.as<unsigned>();
        ib.val_a = P->val_a.as<int>();
        ib.val_b = P->val_b.as<int>();
        ib.hist = P->hist.as<int>();
        ib.hist_off = P->hist_off.as<int>();
        ib.scan_tmp = P->scan_tmp.as<int>();
        ib.pts = P->pts.as<float4>();
        ib.pts64 = c.pos_f64 ? P->pts64.as<double>() : nullptr;
        ib.orig = P->orig.as<int>();
        ib.cstart = P->cstart.as<int>();
        ib.plist = P->plist.as<int>();
        ib.status = d_status;
        IndexArgs ia{};
        ia.pos = c.pos;
        ia.w = c.w;
        ia.n = n;
        ia.pos_f64 = c.pos_f64;
        ia.g = g;
        const int64_t* d_catoff = nullptr;
        PrimRanges pr{};
        const PrimRanges* prp = nullptr;
        if (c.ncat > 1) {
            if (ensure(P, P->d_catoff, 8 * (c.ncat + 1), "offsets")) return G3PCF_ERR_ALLOC;
            UP(P->d_catoff.p, c.offs.data(), 8 * (c.ncat + 1));
            d_catoff = P->d_catoff.as<int64_t>();
            // processing order: catalogs by decreasing size (heaviest first)
            std::vector<int> order(c.ncat);
            for (int k = 0; k < c.ncat; ++k) order[k] = k;
            std::sort(order.begin(), order.end(), [&](int a, int b) {
                return (c.offs[a + 1] - c.offs[a]) > (c.offs[b + 1] - c.offs[b]);
            });
            std::vector<int> rs(3 * c.ncat);
            int o = 0;
            for (int k = 0; k < c.ncat; ++k) {
                const int cat = order[k];
                rs[k] = (int)c.offs[cat];
                rs[c.ncat + k] = (int)(c.offs[cat + 1] - c.offs[cat]);
                rs[2 * c.ncat + k] = o;
                o += rs[c.ncat + k];
            }
            if (ensure(P, P->d_ranges, 4 * rs.size(), "ranges")) return G3PCF_ERR_ALLOC;
            UP(P->d_ranges.p, rs.data(), 4 * rs.size());
            pr.start = P->d_ranges.as<int>();
            pr.len = pr.start + c.ncat;
            pr.out = pr.start + 2 * c.ncat;
            pr.n = c.ncat;
            prp = &pr;
            nprim = n;
        } else {
            nprim = c.n_primary;
        }
        const int nl = build_index(ib, ia, d_catoff, c.ncat, ncells, c.n_primary, prp, st);
        if (nl >= 0) P->launches += nl;
        if (nl < 0)
            return fail(G3PCF_ERR_CUDA, "index build launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        P->key_sorted = ib.key_sorted;
        CK(cudaEventRecord(P->ev[1], st));

        // ---- pair stage + contraction, one pass per chunk of primaries
        const bool use_tc = !(c.flags & G3PCF_F_CONTRACT_FP32);
        const int KB = contract_tc_kblock();
        const int64_t rows_all = (c.ncat > 1) ? n : c.n_primary;
        int64_t C = rows_all;
        // the bf16 tensor-core operands (4 bytes per operand column and row) are
        // written by the pair stage only when they fit beside A in the budget
        bool ops_fit = false;
        const bool ops = use_tc && P->opt_tc_operands == 1 && P->opt_pair != 1 && P->opt_basis == 0 && !P->capturing;
        // no memory query inside a capture: a captured forward keeps the warm-up's chunking
        const bool fixed = P->capturing && P->fixed_chunk > 0;
        double budget = 0.0;
        const double per_row = 4.0 * P->RLP + 4.0;
        if (ops || (c.ncat == 1 && P->opt_chunk <= 0 && !fixed)) {
            size_t fr = 0, tot = 0;
            CK(cudaMemGetInfo(&fr, &tot));
            budget = 0.4 * (double)fr;
            if (budget > 48e9) budget = 48e9;
        }
        ops_fit = ops && budget / (per_row + 4.0 * P->RLPb) >= (double)(rows_all + 64 * c.ncat);
        if (c.ncat == 1) {
            if (P->opt_chunk > 0) {
                C = P->opt_chunk;
            } else if (fixed) {
                C = P->fixed_chunk;
            } else {
                C = (int64_t)(budget / per_row) / KB * KB;
                if (C < KB) C = KB;
            }
            if (C > rows_all) C = rows_all;
        }
        const bool chunked = (c.ncat == 1) && C < rows_all;
        P->fixed_chunk = C;
        const int64_t nchunks = chunked ? (rows_all + C - 1) / C : 1;
        const int64_t rows_cap = chunked ? C : rows_all;
        if (ensure(P, P->A, sizeof(float) * (size_t)P->RLP * (rows_cap > 0 ? rows_cap : 1), "multipoles") ||
            ensure(P, P->wrow, sizeof(float) * (size_t)(rows_cap > 0 ? rows_cap : 1), "row weights"))
            return G3PCF_ERR_ALLOC;
        const std::vector<Tile>& tl = use_tc ? P->tiles_tc : P->tiles;
        const int T = use_tc ? P->T_tc : P->T;
        Tile* d_tl = use_tc ? P->d_tiles_tc.as<Tile>() : P->d_tiles.as<Tile>();
        const int ntiles = (int)tl.size();
        const int part_stride = ntiles * T * T;
        // segments of every chunk (partial slots are global across chunks)
        std::vector<std::vector<Segment>> csegs(nchunks);
        // tensor-core work split per (chunk, catalog): segments per item of every strip
        const int nstrips = (int)P->strips_tc.size();
        std::vector<std::vector<int>> csteps(nchunks);
        const int64_t rows_tot = chunked ? std::min<int64_t>(C, rows_all) : rows_all;
        std::vector<int> segfirst(c.ncat + 1, 0);
        std::vector<std::vector<int>> ccats(nchunks);
        std::vector<int64_t> cpad(nchunks, 0);
        int total_segs = 0;
        for (int64_t ch = 0; ch < nchunks; ++ch) {
            const int64_t q0 = ch * C, q1 = chunked ? std::min(rows_all, q0 + C) : rows_all;
            for (int k = 0; k < c.ncat; ++k) {
                if (ch == 0) segfirst[k] = total_segs + (int)csegs[ch].size();
                // rows of catalog k inside this pass (A-row coordinates)
                const int64_t r0 = chunked ? 0 : ((c.ncat > 1) ? c.offs[k] : 0);
                const int64_t r1 = chunked ? q1 - q0 : ((c.ncat > 1) ? c.offs[k + 1] : c.n_primary);
                const int64_t len = r1 - r0;
                if (use_tc) {
                    // padded primary coordinates: every catalog starts on a k-block; an
                    // V equal virtual segments per catalog; every strip's items cover
                    // step[s] of them, balanced over the catalog's share of the SMs
                    const int64_t plen = (len + KB - 1) / KB * KB;
                    ccats[ch].insert(ccats[ch].end(), {(int)cpad[ch], (int)r0, (int)len, 0});
                    const double share = rows_tot > 0 ? (double)plen / (double)rows_tot : 1.0;
                    // at least one full FP32 accumulation run (2048 primaries) per segment
                    const int64_t vmax = 2 * (plen / (2 * 2048));
                    const size_t st0 = csteps[ch].size();
                    csteps[ch].resize(st0 + (size_t)nstrips);
                    const int64_t V = plan_tc_items(P->strips_tc.data(), nstrips, (int)std::min<int64_t>(vmax, 1 << 20),
                                                    share * P->nsm, csteps[ch].data() + st0);
                    const int64_t seg = ((plen + V - 1) / V + KB - 1) / KB * KB;
                    for (int64_t v = 0; v < V; ++v) {
                        Segment sg;
                        sg.cat = k;
                        const int64_t s0 = std::min(plen, v * seg), s1 = std::min(plen, (v + 1) * seg);
                        sg.row0 = (int)(cpad[ch] + s0);
                        sg.row1 = (int)(cpad[ch] + s1);
                        csegs[ch].push_back(sg);
                    }
                    cpad[ch] += plen;
                } else {
                    int64_t seg = len / 32;
                    if (seg < 8192) seg = 8192;
                    for (int64_t s0 = r0; s0 < r1; s0 += seg) {
                        Segment sg;
                        sg.cat = k;
                        sg.row0 = (int)s0;
                        sg.row1 = (int)(s0 + seg < r1 ? s0 + seg : r1);
                        csegs[ch].push_back(sg);
                    }
                }
            }
            total_segs += (int)csegs[ch].size();
        }
        segfirst[c.ncat] = total_segs;
        if (total_segs > 0) {
            size_t max_segs = 0, max_cats = 1;
            for (int64_t ch = 0; ch < nchunks; ++ch) {
                max_segs = std::max(max_segs, csegs[ch].size());
                max_cats = std::max(max_cats, ccats[ch].size());
            }
            if (ensure(P, P->d_segs, sizeof(Segment) * max_segs, "segments") ||
                ensure(P, P->d_segfirst, 4 * (c.ncat + 1), "segments") ||
                ensure(P, P->partials, sizeof(double) * (size_t)part_stride * total_segs, "partials"))
                return G3PCF_ERR_ALLOC;
            if (use_tc && ensure(P, P->d_cats, 4 * max_cats, "catalog table")) return G3PCF_ERR_ALLOC;
            UP(P->d_segfirst.p, segfirst.data(), 4 * (c.ncat + 1));
        }
        // per-chunk stage events (created outside a capture; a capture that finds
        // too few keeps the single-span timing)
        P->cev_used = 0;
        if (!P->capturing)
            while ((int64_t)P->cev.size() < 2 * nchunks) {
                cudaEvent_t e;
                CK(cudaEventCreate(&e));
                P->cev.push_back(e);
            }
        const bool chunk_events = (int64_t)P->cev.size() >= 2 * nchunks;
        // bf16 tensor-core operands written by the pair stage (one pass of the
        // multipoles, list path, Chebyshev basis, outside a capture): rows in the
        // padded catalog coordinates of the contraction, padding rows zeroed
        P->direct_used = false;
        __nv_bfloat16* bop = nullptr;
        int64_t bop_elems = 0;
        if (ops_fit && !chunked && nprim > 0 && !ccats.empty() && cpad[0] > 0) {
            bop_elems = cpad[0] * 2 * (int64_t)P->RLPb;  // hi and lo of every padded row
            if (ensure(P, P->d_bop, sizeof(__nv_bfloat16) * (size_t)bop_elems, "tensor-core operands") ||
                ensure(P, P->d_bcat, sizeof(int4) * (ccats[0].size() / 4), "tensor-core operands"))
                return G3PCF_ERR_ALLOC;
            bop = P->d_bop.as<__nv_bfloat16>();
            UP(P->d_bcat.p, ccats[0].data(), 4 * ccats[0].size());
            P->launches += 1;
            if (launch_zero_pad(bop, P->RLPb, P->d_bcat.as<int4>(), (int)(ccats[0].size() / 4), st) != 0)
                return fail(G3PCF_ERR_CUDA, "operand padding launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        }
        int seg_base = 0;
        for (int64_t ch = 0; ch < nchunks; ++ch) {
            const int64_t q0 = ch * C, q1 = chunked ? std::min(rows_all, q0 + C) : nprim;
            if (ch > 0) CK(cudaMemsetAsync(d_queue, 0, sizeof(int), st));
            if (nprim > 0 && q1 > q0) {
                PairArgs pa{};
                pa.pts = ib.pts;
                pa.pts64 = ib.pts64;
                pa.orig = ib.orig;
                pa.cstart = ib.cstart;
                pa.plist = (c.ncat > 1 || c.n_primary < n) ? ib.plist : nullptr;
                P->last_plist = pa.plist != nullptr;
                pa.key = ib.key_sorted;
                pa.nprim = (int)q1;
                pa.q0 = (int)q0;
                pa.chunked = chunked ? 1 : 0;
                pa.wrow = P->wrow.as<float>();
                pa.A = P->A.as<float>();
                pa.RLP = P->RLP;
                pa.colmap = P->d_colmap.as<int>();
                pa.colscale = P->d_colscale.as<float>();
                pa.RL = P->RL;
                pa.counts = P->counts.as<unsigned long long>();
                pa.queue = d_queue;
                pa.status = d_status;
                pa.kflush = P->kflush;
                pa.g = g;
                pa.bins = P->bins;
                pa.bintab = P->d_bintab.as<unsigned char>();
                pa.bin_tscale = P->bin_tscale;
                pa.bop = bop;
                pa.nbcat = (int)(ccats.empty() ? 0 : ccats[0].size() / 4);
                pa.bop_pitch = P->RLPb;
                pa.bblk = P->d_bblk.as<int4>();
                pa.nblk = (int)P->bblk.size();
                pa.bcat = P->d_bcat.as<int4>();
                const bool use_list = P->opt_pair != 1;
                if (use_list) {
                    if (int r = run_pair_lists(P, pa, st)) return r;
                } else {
                    ++P->launches;
                    if (launch_pair(P->lmax, pa, P->nsm, st) != 0)
                        return fail(G3PCF_ERR_CUDA, "pair kernel launch failed: %s", cudaGetErrorString(cudaGetLastError()));
                }
            }
            if (ch == 0) CK(cudaEventRecord(P->ev[2], st));
            if (chunk_events) CK(cudaEventRecord(P->cev[2 * ch], st));
            const std::vector<Segment>& segs = csegs[ch];
            const int nsegs = (int)segs.size();
            if (nsegs > 0) {
                double* part = P->partials.as<double>() + (size_t)seg_base * part_stride;
                UP(P->d_segs.p, segs.data(), sizeof(Segment) * nsegs);
                if (use_tc) {
                    UP(P->d_cats.p, ccats[ch].data(), 4 * ccats[ch].size());
                    P->launches += 1;
                    // work items: every strip over every virtual segment of every
                    // catalog, step[s] consecutive segments at a time (planned above)
                    std::vector<TcItem> items;
                    int kc = 0;  // catalog index within this chunk
                    for (int s0 = 0; s0 < nsegs; ++kc) {
                        int s1 = s0;
                        while (s1 < nsegs && segs[s1].cat == segs[s0].cat) ++s1;
                        const int* stp = csteps[ch].data() + (size_t)kc * nstrips;
                        for (int k = 0; k < nstrips; ++k) {
                            const int step = stp[k];
                            for (int v = s0; v < s1; v += step)
                                items.push_back(TcItem{k, v, std::min(step, s1 - v), 0});
                        }
                        s0 = s1;
                    }
                    if (ensure(P, P->d_items, sizeof(TcItem) * items.size(), "tensor-core work items"))
                        return G3PCF_ERR_ALLOC;
                    UP(P->d_items.p, items.data(), sizeof(TcItem) * items.size());
                    // the rows of A written by this pass: the map reads zeros past them, so
                    // the padding primaries of the last k-block never meet stale memory
                    const int64_t rows_written = chunked ? q1 - q0 : rows_all;
                    const int rc =
                        P->direct_used
                            ? launch_contract_tc_op(bop, P->RLPb, cpad[ch], d_tl,
                                                    P->d_strips_tc.as<TcStrip>(), P->d_items.as<TcItem>(),
                                                    (int)items.size(), P->d_segs.as<Segment>(), part, part_stride,
                                                    d_status, st, P->test_tc_timeout)
                            : launch_contract_tc(P->A.as<float>(), P->RLP, P->RL, rows_written, P->wrow.as<float>(),
                                                 P->d_cats.as<int4>(), d_tl, P->d_strips_tc.as<TcStrip>(),
                                                 P->d_items.as<TcItem>(), (int)items.size(), P->d_segs.as<Segment>(),
                                                 part, part_stride, d_status + kNegWeightSlot, d_status, st,
                                                 P->test_tc_timeout);
                    if (rc == -2) return fail(G3PCF_ERR_CUDA, "cuTensorMapEncodeTiled unavailable or failed");
                    if (rc != 0)
                        return fail(G3PCF_ERR_CUDA, "tensor-core contraction launch failed: %s", cudaGetErrorString(cudaGetLastError()));
                } else {
                    P->launches += 1;
                    if (launch_contract_fp32(P->A.as<float>(), P->RLP, P->wrow.as<float>(), d_tl, ntiles,
                                             P->d_segs.as<Segment>(), nsegs, part, part_stride, st) != 0)
                        return fail(G3PCF_ERR_CUDA, "contraction launch failed: %s", cudaGetErrorString(cudaGetLastError()));
                }
            }
            seg_base += nsegs;
            if (chunk_events) CK(cudaEventRecord(P->cev[2 * ch + 1], st));
        }
        if (chunk_events) P->cev_used = (int)(2 * nchunks);
        CK(cudaEventRecord(P->ev[3], st));
        if (total_segs > 0) {
            P->launches += 1;
            if (launch_reduce(P->partials.as<double>(), part_stride, P->d_segfirst.as<int>(), c.ncat,
                              B, P->lmax, d_tl, T, c.zeta, st, use_tc ? 1 : 0) != 0)
                return fail(G3PCF_ERR_CUDA, "reduction launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        }
        P->last_chunked = chunked;
    } else {
        CK(cudaEventRecord(P->ev[1], st));
        CK(cudaEventRecord(P->ev[2], st));
        CK(cudaEventRecord(P->ev[3], st));
    }
    CK(cudaEventRecord(P->ev[4], st));
    if (c.counts) {
        CK(cudaMemcpyAsync(c.counts, P->counts.p, sizeof(int64_t) * B * c.ncat, cudaMemcpyDeviceToDevice, st));
    }
    CK(cudaMemcpyAsync(P->h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    P->have_forward = true;
    P->have_alm = true;
    P->last_n = n;
    P->last_np = nprim;
    P->last_ncat = c.ncat;
    P->last_offs = c.offs;
    P->last_pos = c.pos;
    P->last_w = c.w;
    P->last_pos_f64 = c.pos_f64;
    P->stats[6] = (double)nprim;
    if (c.flags & G3PCF_F_NO_SYNC) return G3PCF_OK;
    CK(cudaStreamSynchronize(st));
    return read_status(P);
}

// G3PCF_F_GRAPH: the first call with a new signature runs once normally (all
// allocations, staging sizes and the chunk size settle), then captures the
// same device work into a CUDA graph on an internal stream; calls with the
// same signature replay the graph, ordered after the plan's stream.
int forward_entry(g3pcf_plan_t P, CallSpec& c) {
    if (!(c.flags & G3PCF_F_GRAPH)) {
        if (P->gexec) {  // a plain forward reuses the staging buffer: drop the graph
            cudaGraphExecDestroy(P->gexec);
            P->gexec = nullptr;
        }
        return run_forward(P, c);
    }
    if (int r = setup_device(P)) return r;
    std::vector<long long> key = {(long long)(intptr_t)c.pos, (long long)(intptr_t)c.w,
                                  (long long)(intptr_t)c.zeta, (long long)(intptr_t)c.counts,
                                  (long long)c.n, (long long)c.n_primary, (long long)c.ncat,
                                  (long long)c.pos_f64,
                                  (long long)(c.flags & ~(G3PCF_F_NO_SYNC | G3PCF_F_GRAPH)),
                                  (long long)P->opt_chunk, (long long)P->opt_cells, (long long)P->kflush};
    key.insert(key.end(), c.offs.begin(), c.offs.end());
    if (!P->gstream) {
        CK(cudaStreamCreateWithFlags(&P->gstream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&P->gev[0], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&P->gev[1], cudaEventDisableTiming));
    }
    cudaStream_t user = P->stream;
    if (!(P->gexec && key == P->gkey)) {
        if (P->gexec) {
            cudaGraphExecDestroy(P->gexec);
            P->gexec = nullptr;
        }
        CallSpec warm = c;
        warm.flags &= ~(G3PCF_F_GRAPH | G3PCF_F_NO_SYNC);
        P->warm_for_graph = true;
        const int rw = run_forward(P, warm);
        P->warm_for_graph = false;
        if (rw) return rw;
        CallSpec cap = c;
        cap.flags = (c.flags & ~G3PCF_F_GRAPH) | G3PCF_F_NO_SYNC;
        P->stream = P->gstream;
        P->capturing = true;
        cudaError_t e = cudaStreamBeginCapture(P->gstream, cudaStreamCaptureModeThreadLocal);
        int r = (e == cudaSuccess) ? run_forward(P, cap)
                                   : fail(G3PCF_ERR_CUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
        cudaGraph_t graph = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(P->gstream, &graph);
        P->stream = user;
        P->capturing = false;
        if (r != 0 || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return r != 0 ? r : fail(G3PCF_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e2));
        }
        e = cudaGraphInstantiate(&P->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            P->gexec = nullptr;
            return fail(G3PCF_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
        }
        P->gkey = key;
    }
    CK(cudaEventRecord(P->gev[0], user));
    CK(cudaStreamWaitEvent(P->gstream, P->gev[0], 0));
    CK(cudaGraphLaunch(P->gexec, P->gstream));
    CK(cudaEventRecord(P->gev[1], P->gstream));
    CK(cudaStreamWaitEvent(user, P->gev[1], 0));
    if (c.flags & G3PCF_F_NO_SYNC) return G3PCF_OK;
    CK(cudaStreamSynchronize(user));
    if (P->h_status[0] & kStatusOverflow) {
        // the data outgrew the lists planned at capture: drop the graph (the next
        // graph call captures again) and run this call uncaptured
        cudaGraphExecDestroy(P->gexec);
        P->gexec = nullptr;
        P->gkey.clear();
        CallSpec plain = c;
        plain.flags &= ~G3PCF_F_GRAPH;
        return run_forward(P, plain);
    }
    return read_status(P);
}

int check_plan(g3pcf_plan_t P) {
    if (!P) return fail(G3PCF_ERR_ARG, "plan is NULL");
    return 0;
}

}  // namespace

extern "C" {

int64_t g3pcf_zeta_size(int nbins, int lmax) {
    if (nbins < 1 || lmax < 0) return 0;
    return zsize_of(nbins, lmax);
}

const char* g3pcf_last_error(void) { return g_err.c_str(); }

int g3pcf_plan(g3pcf_plan_t* out, int nbins, double rmin, double rmax, int lmax, double box,
               int los_mode) {
    g_err.clear();
    if (!out) return fail(G3PCF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nbins < 1 || nbins > G3PCF_MAX_NBINS) return fail(G3PCF_ERR_ARG, "nbins must be in [1, %d]", G3PCF_MAX_NBINS);
    if (lmax < 0 || lmax > G3PCF_MAX_LMAX) return fail(G3PCF_ERR_ARG, "lmax must be in [0, %d]", G3PCF_MAX_LMAX);
    if (!std::isfinite(rmin) || !std::isfinite(rmax) || !(rmin >= 0.0) || !(rmax > rmin))
        return fail(G3PCF_ERR_ARG, "need 0 <= rmin < rmax (finite)");
    if (!std::isfinite(box) || !(box > 0.0)) return fail(G3PCF_ERR_ARG, "box must be finite and > 0");
    if (los_mode < 0 || los_mode > 2) return fail(G3PCF_ERR_ARG, "unknown los_mode %d", los_mode);
    if (los_mode == G3PCF_LOS_Z_PERIODIC && !(rmax < 0.5 * box * (1.0 - 1e-6)))
        return fail(G3PCF_ERR_RMAX, "periodic box needs rmax < box/2 (rmax=%g, box=%g)", rmax, box);
    g3pcf_plan_t P = new (std::nothrow) g3pcf_plan_s();
    if (!P) return fail(G3PCF_ERR_ALLOC, "out of host memory");
    P->nbins = nbins;
    P->lmax = lmax;
    P->los_mode = los_mode;
    P->rmin = rmin;
    P->rmax = rmax;
    P->box = box;
    compute_bins(P);
    compute_columns(P);
    // pairs per lane per bucket flush: the largest k <= 16 for which two
    // 4-warp CTAs of the pair kernel fit in 227 KB of shared memory
    // (dynamic per warp x 4 warps + ~2.6 KB static + 1 KB reserved, per CTA)
    P->kflush = 2;
    for (int kf = 16; kf >= 2; --kf)
        if ((pair_smem_per_warp(lmax, nbins, kf) * 4 + 4096) * 2 <= 227 * 1024) {
            P->kflush = kf;
            break;
        }
    P->T = contract_tile_dim_fp32();
    P->tiles.resize(4096);
    int nt = make_tiles(nbins, lmax, P->T, P->tiles.data(), (int)P->tiles.size());
    if (nt < 0) {
        delete P;
        return fail(G3PCF_ERR_ARG, "too many contraction tiles");
    }
    P->tiles.resize(nt);
    P->T_tc = contract_tile_dim_tc();
    P->tiles_tc.resize(4096);
    nt = make_tiles(nbins, lmax, P->T_tc, P->tiles_tc.data(), (int)P->tiles_tc.size());
    if (nt < 0) {
        delete P;
        return fail(G3PCF_ERR_ARG, "too many contraction tiles");
    }
    P->tiles_tc.resize(nt);
    P->strips_tc.resize(nt);
    const int nstrip = make_strips(P->tiles_tc.data(), nt, P->strips_tc.data(), nt);
    P->strips_tc.resize(nstrip > 0 ? nstrip : 0);
    P->bblk.assign(lmax + 1, int4{0, 0, 0, 0});
    P->RLPb = tc_operand_blocks(P->tiles_tc.data(), nt, P->bblk.data(), lmax + 1);
    if (P->RLPb < 0) {
        delete P;
        return fail(G3PCF_ERR_ARG, "operand blocks out of range");
    }
    *out = P;
    return G3PCF_OK;
}

int g3pcf_set_stream(g3pcf_plan_t P, void* s) {
    if (int r = check_plan(P)) return r;
    P->stream = static_cast<cudaStream_t>(s);
    return G3PCF_OK;
}

int g3pcf_compute_ex(g3pcf_plan_t P, const void* pos, const float* w, int64_t n, int64_t n_primary,
                     double* zeta, int64_t* counts, int flags) {
    g_err.clear();
    if (int r = check_plan(P)) return r;
    if (n < 0) return fail(G3PCF_ERR_ARG, "n < 0");
    if (n >= G3PCF_MAX_POINTS) return fail(G3PCF_ERR_ARG, "n must be < 2^27");
    if (!zeta) return fail(G3PCF_ERR_ARG, "zeta is NULL");
    if (n > 0 && (!pos || !w)) return fail(G3PCF_ERR_ARG, "pos or w is NULL");
    if (flags & ~(G3PCF_F_POS_F64 | G3PCF_F_CONTRACT_FP32 | G3PCF_F_NO_SYNC | G3PCF_F_KEEP_ALM |
                  G3PCF_F_GRAPH))
        return fail(G3PCF_ERR_ARG, "unknown flags 0x%x", flags);
    if (n_primary < 0 || n_primary > n) n_primary = n;
    CallSpec c;
    c.pos = pos;
    c.w = w;
    c.n = n;
    c.n_primary = n_primary;
    c.pos_f64 = (flags & G3PCF_F_POS_F64) ? 1 : 0;
    c.ncat = 1;
    c.offs = {0, n};
    c.zeta = zeta;
    c.counts = counts;
    c.flags = flags;
    return forward_entry(P, c);
}

int g3pcf_compute(g3pcf_plan_t P, const float* pos, const float* w, int64_t n, double* zeta) {
    return g3pcf_compute_ex(P, pos, w, n, -1, zeta, nullptr, 0);
}

int g3pcf_compute_batch(g3pcf_plan_t P, const float* pos, const float* w, const int64_t* offsets,
                        int ncat, double* zeta, int64_t* counts, int flags) {
    g_err.clear();
    if (int r = check_plan(P)) return r;
    if (!offsets || ncat < 1) return fail(G3PCF_ERR_ARG, "need ncat >= 1 and offsets");
    if (!zeta) return fail(G3PCF_ERR_ARG, "zeta is NULL");
    if (flags & ~(G3PCF_F_CONTRACT_FP32 | G3PCF_F_NO_SYNC | G3PCF_F_KEEP_ALM | G3PCF_F_GRAPH))
        return fail(G3PCF_ERR_ARG, "unsupported flags 0x%x for batch", flags);
    if (offsets[0] != 0) return fail(G3PCF_ERR_ARG, "offsets[0] must be 0");
    for (int k = 0; k < ncat; ++k)
        if (offsets[k + 1] < offsets[k]) return fail(G3PCF_ERR_ARG, "offsets must be non-decreasing");
    const int64_t n = offsets[ncat];
    if (n >= G3PCF_MAX_POINTS) return fail(G3PCF_ERR_ARG, "total points must be < 2^27");
    if (n > 0 && (!pos || !w)) return fail(G3PCF_ERR_ARG, "pos or w is NULL");
    CallSpec c;
    c.pos = pos;
    c.w = w;
    c.n = n;
    c.n_primary = n;
    c.pos_f64 = 0;
    c.ncat = ncat;
    c.offs.assign(offsets, offsets + ncat + 1);
    c.zeta = zeta;
    c.counts = counts;
    c.flags = flags;
    return forward_entry(P, c);
}

int g3pcf_alm(g3pcf_plan_t P, const int64_t* primaries, int64_t np, double* out) {
    g_err.clear();
    if (int r = check_plan(P)) return r;
    if (!P->have_alm) return fail(G3PCF_ERR_STATE, "no forward with multipoles on this plan");
    if (P->last_chunked)
        return fail(G3PCF_ERR_STATE, "the last forward ran in chunks; its multipoles were not kept");
    if (np < 0 || (np > 0 && (!primaries || !out))) return fail(G3PCF_ERR_ARG, "bad primaries/out");
    const int64_t rows = (P->last_ncat > 1) ? P->last_n : P->last_np;
    const int B = P->nbins, L = P->lmax;
    const int nlm = (L + 1) * (L + 2) / 2;
    std::vector<float> row(P->RLP);
    CK(cudaStreamSynchronize(P->stream));
    for (int64_t k = 0; k < np; ++k) {
        const int64_t i = primaries[k];
        if (i < 0 || i >= rows) return fail(G3PCF_ERR_ARG, "primary index %lld out of range", (long long)i);
        CK(cudaMemcpy(row.data(), P->A.as<float>() + i * P->RLP, sizeof(float) * P->RL, cudaMemcpyDeviceToHost));
        double* o = out + k * (int64_t)B * nlm * 2;
        std::memset(o, 0, sizeof(double) * B * nlm * 2);
        int col = 0;
        for (int m = 0; m <= L; ++m) {
            const int K = B * (L + 1 - m);
            const int parts = m == 0 ? 1 : 2;
            for (int part = 0; part < parts; ++part)
                for (int idx = 0; idx < K; ++idx) {
                    const int l = m + idx / B, b = idx % B;
                    o[2 * ((int64_t)b * nlm + l * (l + 1) / 2 + m) + part] = row[col++];
                }
        }
    }
    return G3PCF_OK;
}

int g3pcf_backward(g3pcf_plan_t P, const double* dzeta, double* dpos, double* dw) {
    g_err.clear();
    if (int r = check_plan(P)) return r;
    if (!P->have_forward) return fail(G3PCF_ERR_STATE, "backward before forward on this plan");
    if (!dzeta || !dpos || !dw) return fail(G3PCF_ERR_ARG, "dzeta, dpos and dw must be non-null");
    if (P->los_mode == G3PCF_LOS_RADIAL_OPEN)
        return fail(G3PCF_ERR_UNSUPPORTED, "the adjoint supports the z line-of-sight modes only");
    if (P->last_chunked && P->opt_pair == 1)
        return fail(G3PCF_ERR_UNSUPPORTED, "a chunked backward recomputes the multipoles through the pair lists");
    cudaStream_t st = P->stream;
    const int64_t n = P->last_n, rows = P->last_np;
    CK(cudaMemsetAsync(dpos, 0, sizeof(double) * 3 * (n > 0 ? n : 1), st));
    CK(cudaMemsetAsync(dw, 0, sizeof(double) * (n > 0 ? n : 1), st));
    if (n == 0 || rows == 0) {
        CK(cudaStreamSynchronize(st));
        return G3PCF_OK;
    }
    const int ncat = P->last_ncat;
    if (P->last_chunked) {
        // the multipoles did not fit: recompute them chunk by chunk (same chunks as the
        // forward) and run each chunk's adjoint on the lists that recomputed them
        const int64_t C = P->fixed_chunk;
        const bool precise = P->opt_grad == 0;
        if (precise ? (ensure(P, P->d_mrealdf, sizeof(float2) * adjoint_m_floats(P->nbins, P->lmax), "adjoint M") ||
                       ensure(P, P->d_Vdf, sizeof(float2) * (size_t)P->RLP * C, "adjoint V"))
                    : (ensure(P, P->d_mreal, sizeof(float) * adjoint_m_floats(P->nbins, P->lmax), "adjoint M") ||
                       ensure(P, P->d_V, sizeof(float) * (size_t)P->RLP * C, "adjoint V")))
            return G3PCF_ERR_ALLOC;
        int* d_status = P->small.as<int>();
        int* d_queue = d_status + 16;
        CK(cudaMemsetAsync(P->small.p, 0, 256, st));
        CK(cudaMemsetAsync(P->counts.p, 0, sizeof(unsigned long long) * P->nbins, st));
        if ((precise ? launch_adjoint_m_df(dzeta, P->nbins, P->lmax, 1, zsize_of(P->nbins, P->lmax),
                                           P->d_mrealdf.as<float2>(), st)
                     : launch_adjoint_m(dzeta, P->nbins, P->lmax, 1, zsize_of(P->nbins, P->lmax),
                                        P->d_mreal.as<float>(), st)) != 0)
            return fail(G3PCF_ERR_CUDA, "adjoint preparation launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        P->lev_used = 0;
        for (int64_t q0 = 0; q0 < rows; q0 += C) {
            PairArgs pa{};
            pa.pts = P->pts.as<float4>();
            pa.pts64 = P->last_pos_f64 ? P->pts64.as<double>() : nullptr;
            pa.orig = P->orig.as<int>();
            pa.cstart = P->cstart.as<int>();
            pa.plist = P->last_plist ? P->plist.as<int>() : nullptr;
            pa.key = P->key_sorted;
            pa.q0 = (int)q0;
            pa.nprim = (int)std::min<int64_t>(rows, q0 + C);
            pa.chunked = 1;
            pa.wrow = P->wrow.as<float>();
            pa.A = P->A.as<float>();
            pa.RLP = P->RLP;
            pa.colmap = P->d_colmap.as<int>();
            pa.colscale = P->d_colscale.as<float>();
            pa.RL = P->RL;
            pa.counts = P->counts.as<unsigned long long>();
            pa.queue = d_queue;
            pa.status = d_status;
            pa.kflush = P->kflush;
            pa.V = P->d_V.as<float>();
            pa.dw = dw;
            pa.dpos = dpos;
            pa.g = P->last_grid;
            pa.bins = P->bins;
            pa.bintab = P->d_bintab.as<unsigned char>();
            pa.bin_tscale = P->bin_tscale;
            CK(cudaMemsetAsync(d_queue, 0, sizeof(int), st));
            if (int r = run_pair_lists(P, pa, st, 2)) return r;
        }
        CK(cudaMemcpyAsync(P->h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        return read_status(P);
    }
    // row blocks of one catalog each (rows are original indices; catalog c holds
    // [offs[c], offs[c+1]) of a batched forward, every row of a single one)
    const int RB = adjoint_rows_per_block();
    std::vector<int4> blks;
    for (int c = 0; c < ncat; ++c) {
        const int64_t r0 = ncat > 1 ? P->last_offs[c] : 0, r1 = ncat > 1 ? P->last_offs[c + 1] : rows;
        for (int64_t r = r0; r < r1; r += RB) blks.push_back(int4{c, (int)r, (int)std::min<int64_t>(RB, r1 - r), 0});
    }
    // the double-float pair pass (list path, G3PCF_OPT_GRAD_PRECISION 0) takes M and V in FP64
    const bool precise = P->opt_grad == 0 && P->opt_pair != 1;
    if ((precise ? (ensure(P, P->d_mrealdf, sizeof(float2) * adjoint_m_floats(P->nbins, P->lmax) * ncat, "adjoint M") ||
                    ensure(P, P->d_Vdf, sizeof(float2) * (size_t)P->RLP * rows, "adjoint V"))
                 : (ensure(P, P->d_mreal, sizeof(float) * adjoint_m_floats(P->nbins, P->lmax) * ncat, "adjoint M") ||
                    ensure(P, P->d_V, sizeof(float) * (size_t)P->RLP * rows, "adjoint V"))) ||
        ensure(P, P->d_vblk, sizeof(int4) * (blks.size() + 1), "adjoint blocks"))
        return G3PCF_ERR_ALLOC;
    CK(cudaMemcpyAsync(P->d_vblk.p, blks.data(), sizeof(int4) * blks.size(), cudaMemcpyHostToDevice, st));
    int* d_status = P->small.as<int>();
    int* d_queue = d_status + 16;
    CK(cudaMemsetAsync(P->small.p, 0, 256, st));
    CK(cudaMemsetAsync(P->counts.p, 0, sizeof(unsigned long long) * P->nbins * ncat, st));
    if ((precise ? launch_adjoint_prep_df(dzeta, P->nbins, P->lmax, ncat, zsize_of(P->nbins, P->lmax),
                                         P->A.as<float>(), P->RLP, P->RL, P->d_vblk.as<int4>(), (int)blks.size(),
                                         P->d_mrealdf.as<float2>(), P->d_Vdf.as<float2>(), dw, st)
                 : launch_adjoint_prep(dzeta, P->nbins, P->lmax, ncat, zsize_of(P->nbins, P->lmax),
                                       P->A.as<float>(), P->RLP, P->RL, P->d_vblk.as<int4>(), (int)blks.size(),
                                       P->d_mreal.as<float>(), P->d_V.as<float>(), dw, st)) != 0)
        return fail(G3PCF_ERR_CUDA, "adjoint preparation launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    PairArgs pa{};
    pa.pts = P->pts.as<float4>();
    pa.pts64 = P->last_pos_f64 ? P->pts64.as<double>() : nullptr;
    pa.orig = P->orig.as<int>();
    pa.cstart = P->cstart.as<int>();
    pa.plist = P->last_plist ? P->plist.as<int>() : nullptr;
    pa.key = P->key_sorted;
    pa.nprim = (int)rows;
    pa.A = P->A.as<float>();
    pa.RLP = P->RLP;
    pa.colmap = P->d_colmap.as<int>();
    pa.colscale = P->d_colscale.as<float>();
    pa.RL = P->RL;
    pa.counts = P->counts.as<unsigned long long>();
    pa.queue = d_queue;
    pa.status = d_status;
    pa.kflush = P->kflush;
    pa.V = P->d_V.as<float>();
    pa.dw = dw;
    pa.dpos = dpos;
    pa.g = P->last_grid;
    pa.bins = P->bins;
    pa.bintab = P->d_bintab.as<unsigned char>();
    pa.bin_tscale = P->bin_tscale;
    if (P->opt_pair != 1) {
        pa.q0 = 0;
        pa.chunked = 0;
        P->lev_used = 0;
        if (int r = run_pair_lists(P, pa, st, 1)) return r;
    } else if (launch_pair(P->lmax, pa, P->nsm, st, 1) != 0) {
        return fail(G3PCF_ERR_CUDA, "adjoint pair kernel launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    }
    CK(cudaMemcpyAsync(P->h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return read_status(P);
}

int g3pcf_set_option(g3pcf_plan_t P, int option, int64_t value) {
    g_err.clear();
    if (int r = check_plan(P)) return r;
    switch (option) {
        case G3PCF_OPT_CHUNK_ROWS:
            if (value < 0) return fail(G3PCF_ERR_ARG, "chunk rows must be >= 0");
            P->opt_chunk = value > 0 ? (value + 63) / 64 * 64 : 0;
            return G3PCF_OK;
        case G3PCF_OPT_CELLS_PER_RMAX:
            if (value < 0 || value > 8) return fail(G3PCF_ERR_ARG, "cells per rmax must be in [0, 8]");
            P->opt_cells = (int)value;
            return G3PCF_OK;
        case G3PCF_OPT_KFLUSH: {
            if (value == 0) return G3PCF_OK;
            if (value < 2 || value > 16) return fail(G3PCF_ERR_ARG, "kflush must be in [2, 16]");
            if ((pair_smem_per_warp(P->lmax, P->nbins, (int)value) * 4 + 4096) > 227 * 1024)
                return fail(G3PCF_ERR_ARG, "kflush %lld does not fit in shared memory", (long long)value);
            P->kflush = (int)value;
            return G3PCF_OK;
        }
        case G3PCF_OPT_PAIR_KERNELS:
            if (value < 0 || value > 2) return fail(G3PCF_ERR_ARG, "pair kernels must be 0, 1 or 2");
            P->opt_pair = (int)value;
            return G3PCF_OK;
        case G3PCF_OPT_X_REFINE:
            if (value < 0 || value > 16) return fail(G3PCF_ERR_ARG, "x refinement must be in [0, 16]");
            P->opt_xref = (int)value;
            return G3PCF_OK;
        case G3PCF_OPT_BASIS:
            if (value < 0 || value > 1) return fail(G3PCF_ERR_ARG, "basis must be 0 (Chebyshev) or 1 (monomials)");
            P->opt_basis = (int)value;
            return G3PCF_OK;
        case G3PCF_OPT_TEST_FAIL_ALLOC:
            if (value < 0 || value > 1000000) return fail(G3PCF_ERR_ARG, "allocation-failure countdown out of range");
            P->test_fail_alloc = (int)value;
            return G3PCF_OK;
        case G3PCF_OPT_TEST_TC_TIMEOUT:
            if (value < 0 || value > 1) return fail(G3PCF_ERR_ARG, "tensor-core timeout test must be 0 or 1");
            P->test_tc_timeout = (int)value;
            return G3PCF_OK;
        case G3PCF_OPT_TC_OPERANDS:
            if (value < 0 || value > 1) return fail(G3PCF_ERR_ARG, "tensor-core operands must be 0 or 1");
            P->opt_tc_operands = (int)value;
            return G3PCF_OK;
        case G3PCF_OPT_GRAD_PRECISION:
            if (value < 0 || value > 1) return fail(G3PCF_ERR_ARG, "gradient precision must be 0 or 1");
            P->opt_grad = (int)value;
            return G3PCF_OK;
        case G3PCF_OPT_LIST_BYTES:
            if (value < 0) return fail(G3PCF_ERR_ARG, "list bytes must be >= 0");
            if (value > 0 && value < (int64_t)1 << 20) return fail(G3PCF_ERR_ARG, "list bytes must be >= 1 MiB");
            P->opt_list_bytes = value;
            return G3PCF_OK;
        default:
            return fail(G3PCF_ERR_ARG, "unknown option %d", option);
    }
}

namespace {

// Tune-cache key: plan shape, line-of-sight mode, kernel choice, SM count and
// the expected neighbours per point (n V / L^3) in quarter-octave buckets.
std::string tune_key(g3pcf_plan_t P, int64_t n) {
    const double V = 4.0 / 3.0 * M_PI * P->rmax * P->rmax * P->rmax;
    const double nb = (double)n * V / (P->box * P->box * P->box);
    const int bucket = (int)std::lround(4.0 * std::log2(nb > 1e-30 ? nb : 1e-30));
    char k[160];
    snprintf(k, sizeof(k), "g3pcf-tune-v2 nbins=%d lmax=%d los=%d pairk=%d sm=%d nbr4=%d", P->nbins, P->lmax,
             P->los_mode, P->opt_pair == 1 ? 1 : 0, P->nsm, bucket);
    return k;
}

// A cache line is "<key> | <cells> <xref> <kflush> <microseconds> <operands>".
bool tune_lookup(const char* path, const std::string& key, int v[5]) {
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        const char* bar = std::strstr(line, " | ");
        if (!bar || (size_t)(bar - line) != key.size() || std::strncmp(line, key.c_str(), key.size()) != 0) continue;
        int a[5];
        if (std::sscanf(bar + 3, "%d %d %d %d %d", &a[0], &a[1], &a[2], &a[3], &a[4]) == 5 && a[0] >= 1 &&
            a[0] <= 8 && a[1] >= 1 && a[1] <= 16 && a[2] >= 2 && a[2] <= 16 && (a[4] == 0 || a[4] == 1)) {
            for (int t = 0; t < 5; ++t) v[t] = a[t];
            found = true;  // the last matching line wins
        }
    }
    std::fclose(f);
    return found;
}

void tune_store(const char* path, const std::string& key, const int v[5]) {
    FILE* f = std::fopen(path, "a");
    if (!f) return;  // an unwritable cache only costs a re-tune
    std::fprintf(f, "%s | %d %d %d %d %d\n", key.c_str(), v[0], v[1], v[2], v[3], v[4]);
    std::fclose(f);
}

}  // namespace

int g3pcf_autotune_cached(g3pcf_plan_t P, const void* pos, const float* w, int64_t n, int flags,
                          const char* cache_path, int64_t* chosen) {
    g_err.clear();
    if (int r = check_plan(P)) return r;
    if (n <= 0 || !pos || !w) return fail(G3PCF_ERR_ARG, "autotune needs n > 0 points");
    if (n >= G3PCF_MAX_POINTS) return fail(G3PCF_ERR_ARG, "n must be < 2^27");
    if (flags & ~G3PCF_F_POS_F64) return fail(G3PCF_ERR_ARG, "autotune accepts G3PCF_F_POS_F64 only");
    if (int r = setup_device(P)) return r;
    const std::string key = tune_key(P, n);
    int hit[5];
    if (cache_path && *cache_path && tune_lookup(cache_path, key, hit)) {
        P->opt_cells = hit[0];
        P->opt_xref = hit[1];
        P->kflush = hit[2];
        P->opt_tc_operands = hit[4];
        if (chosen) {
            for (int t = 0; t < 4; ++t) chosen[t] = hit[t];
            chosen[4] = 1;
            chosen[5] = hit[4];
        }
        return G3PCF_OK;
    }
    const int64_t zs = zsize_of(P->nbins, P->lmax);
    double* ztmp = nullptr;
    if (cudaMalloc(&ztmp, sizeof(double) * 2 * zs) != cudaSuccess) {
        cudaGetLastError();
        return fail(G3PCF_ERR_ALLOC, "autotune scratch allocation failed");
    }
    // the density heuristic's resolution, and the largest flush size that fits
    const double density = (double)n / (P->box * P->box * P->box);
    int s0 = (int)std::floor(P->rmax / std::cbrt(48.0 / density));
    s0 = s0 < 1 ? 1 : (s0 > 8 ? 8 : s0);
    int kmax = 2;
    for (int kf = 16; kf >= 2; --kf)
        if ((pair_smem_per_warp(P->lmax, P->nbins, kf) * 4 + 4096) * 2 <= 227 * 1024) {
            kmax = kf;
            break;
        }
    const int saved_cells = P->opt_cells, saved_xref = P->opt_xref, saved_kf = P->kflush;
    const int saved_ops = P->opt_tc_operands;
    const int64_t saved_chunk = P->opt_chunk;
    double best = 1e300;
    int best_s = s0, best_x = 8, best_kf = saved_kf;
    int rc = G3PCF_OK;
    // pair lists (the default): cell resolution x x refinement; the fused kernel
    // (G3PCF_OPT_PAIR_KERNELS = 1): cell resolution x flush size
    const bool fused = P->opt_pair == 1;
    std::vector<std::pair<int, int>> second;
    if (fused) {
        second = {{8, kmax}, {8, kmax > 6 ? kmax - 4 : kmax}};
    } else {
        second = {{4, saved_kf}, {8, saved_kf}, {16, saved_kf}};
    }
    for (int s = s0 - 1; s <= s0 + 1 && rc == G3PCF_OK; ++s) {
        if (s < 1 || s > 8) continue;
        for (const auto& xk : second) {
            P->opt_cells = s;
            P->opt_xref = xk.first;
            P->kflush = xk.second;
            CallSpec c;
            c.pos = pos;
            c.w = w;
            c.n = n;
            c.n_primary = n < 32768 ? n : 32768;  // a bounded sample of primaries
            c.pos_f64 = (flags & G3PCF_F_POS_F64) ? 1 : 0;
            c.ncat = 1;
            c.offs = {0, n};
            c.zeta = ztmp;
            c.counts = nullptr;
            c.flags = G3PCF_F_CONTRACT_FP32;
            double t = 1e300;
            for (int rep = 0; rep < 3 && rc == G3PCF_OK; ++rep) {
                rc = run_forward(P, c);
                if (rc == G3PCF_OK && rep >= 1) {  // the first run sizes the workspace
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, P->ev[1], P->ev[2]);
                    t = std::min(t, (double)ms);
                }
            }
            if (rc == G3PCF_OK && t < best) {
                best = t;
                best_s = s;
                best_x = xk.first;
                best_kf = xk.second;
            }
        }
    }
    // with those, the contraction's operands (pair-list path, Chebyshev basis):
    // formed in the contraction kernel or written by the pair stage, timed over
    // the pair stage and the tensor-core contraction together
    int best_ops = saved_ops;
    if (rc == G3PCF_OK && !fused && P->opt_basis == 0) {
        P->opt_cells = best_s;
        P->opt_xref = best_x;
        P->kflush = best_kf;
        double best_total = 1e300;
        for (int ops = 0; ops <= 1 && rc == G3PCF_OK; ++ops) {
            P->opt_tc_operands = ops;
            CallSpec c;
            c.pos = pos;
            c.w = w;
            c.n = n;
            c.n_primary = n < 32768 ? n : 32768;
            c.pos_f64 = (flags & G3PCF_F_POS_F64) ? 1 : 0;
            c.ncat = 1;
            c.offs = {0, n};
            c.zeta = ztmp;
            c.counts = nullptr;
            c.flags = 0;
            double t = 1e300;
            for (int rep = 0; rep < 3 && rc == G3PCF_OK; ++rep) {
                rc = run_forward(P, c);
                if (rc == G3PCF_OK && rep >= 1) {
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, P->ev[1], P->ev[3]);
                    t = std::min(t, (double)ms);
                }
            }
            if (rc == G3PCF_OK && t < best_total) {
                best_total = t;
                best_ops = ops;
            }
        }
    }
    cudaFree(ztmp);
    P->have_forward = false;
    P->have_alm = false;
    P->opt_chunk = saved_chunk;
    if (rc != G3PCF_OK) {
        P->opt_cells = saved_cells;
        P->opt_xref = saved_xref;
        P->kflush = saved_kf;
        P->opt_tc_operands = saved_ops;
        return rc;
    }
    P->opt_cells = best_s;
    P->opt_xref = best_x;
    P->kflush = best_kf;
    P->opt_tc_operands = best_ops;
    const int v[5] = {best_s, best_x, best_kf, (int)std::min(best * 1000.0, 2e9), best_ops};
    if (cache_path && *cache_path) tune_store(cache_path, key, v);
    if (chosen) {
        for (int t = 0; t < 4; ++t) chosen[t] = v[t];
        chosen[4] = 0;
        chosen[5] = best_ops;
    }
    return G3PCF_OK;
}

int g3pcf_autotune(g3pcf_plan_t P, const void* pos, const float* w, int64_t n, int flags,
                   int64_t* chosen) {
    int64_t c5[6] = {0, 0, 0, 0, 0, 0};
    const int rc = g3pcf_autotune_cached(P, pos, w, n, flags, nullptr, c5);
    if (rc == G3PCF_OK && chosen) {
        chosen[0] = c5[0];
        chosen[1] = c5[2];
        chosen[2] = c5[3];
    }
    return rc;
}

int g3pcf_status(g3pcf_plan_t P) {
    g_err.clear();
    if (int r = check_plan(P)) return r;
    if (!P->h_status) return G3PCF_OK;
    CK(cudaStreamSynchronize(P->stream));
    if ((P->h_status[0] & kStatusOverflow) && P->gexec) {  // see forward_entry
        cudaGraphExecDestroy(P->gexec);
        P->gexec = nullptr;
        P->gkey.clear();
    }
    return read_status(P);
}

int g3pcf_stats(g3pcf_plan_t P, double* vals, int nvals) {
    g_err.clear();
    if (int r = check_plan(P)) return r;
    if (!vals || nvals < 0) return fail(G3PCF_ERR_ARG, "bad vals");
    if (P->have_forward) {
        CK(cudaStreamSynchronize(P->stream));
        float ms;
        CK(cudaEventElapsedTime(&ms, P->ev[0], P->ev[1]));
        P->stats[0] = ms;
        if (P->cev_used > 0) {  // summed over the chunks of primaries
            double pair = 0.0, con = 0.0;
            for (int k = 0; k + 1 < P->cev_used; k += 2) {
                CK(cudaEventElapsedTime(&ms, k == 0 ? P->ev[1] : P->cev[k - 1], P->cev[k]));
                pair += ms;
                CK(cudaEventElapsedTime(&ms, P->cev[k], P->cev[k + 1]));
                con += ms;
            }
            P->stats[1] = pair;
            P->stats[2] = con;
        } else {
            CK(cudaEventElapsedTime(&ms, P->ev[1], P->ev[2]));
            P->stats[1] = ms;
            CK(cudaEventElapsedTime(&ms, P->ev[2], P->ev[3]));
            P->stats[2] = ms;
        }
        CK(cudaEventElapsedTime(&ms, P->ev[3], P->ev[4]));
        P->stats[3] = ms;
        CK(cudaEventElapsedTime(&ms, P->ev[0], P->ev[4]));
        P->stats[4] = ms;
        std::vector<unsigned long long> cnt((size_t)P->nbins * P->last_ncat);
        CK(cudaMemcpy(cnt.data(), P->counts.p, sizeof(unsigned long long) * cnt.size(), cudaMemcpyDeviceToHost));
        double tot = 0;
        for (auto v : cnt) tot += (double)v;
        P->stats[5] = tot;
    }
    P->stats[8] = (double)P->launches;
    double scan_ms = 0.0, accum_ms = 0.0;
    for (int k = 0; k + 3 < P->lev_used; k += 4) {
        float a = 0.f, b = 0.f;
        CK(cudaEventElapsedTime(&a, P->lev[k], P->lev[k + 1]));
        CK(cudaEventElapsedTime(&b, P->lev[k + 2], P->lev[k + 3]));
        scan_ms += a;
        accum_ms += b;
    }
    P->stats[11] = scan_ms;
    P->stats[12] = accum_ms;
    P->stats[13] = (double)(P->lev_used / 4);
    P->stats[14] = P->direct_used ? 1.0 : 0.0;
    for (int k = 0; k < nvals && k < 15; ++k) vals[k] = P->stats[k];
    return G3PCF_OK;
}

int g3pcf_isotropic(int nbins, int lmax, int ncat, const double* zeta, double* out, void* stream) {
    g_err.clear();
    if (nbins < 1 || nbins > G3PCF_MAX_NBINS || lmax < 0 || lmax > G3PCF_MAX_LMAX || ncat < 0)
        return fail(G3PCF_ERR_ARG, "isotropic: nbins in [1, %d], lmax in [0, %d], ncat >= 0", G3PCF_MAX_NBINS,
                    G3PCF_MAX_LMAX);
    if (ncat == 0) return G3PCF_OK;
    if (!zeta || !out) return fail(G3PCF_ERR_ARG, "isotropic: null pointer");
    if (launch_isotropic(zeta, nbins, lmax, ncat, out, static_cast<cudaStream_t>(stream)) != 0)
        return fail(G3PCF_ERR_CUDA, "isotropic launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return G3PCF_OK;
}

int g3pcf_zeta_combine(int nbins, int lmax, int ncat, const double* zeta, const double* coef, double* out,
                       void* stream) {
    g_err.clear();
    if (nbins < 1 || nbins > G3PCF_MAX_NBINS || lmax < 0 || lmax > G3PCF_MAX_LMAX)
        return fail(G3PCF_ERR_ARG, "combine: nbins in [1, %d], lmax in [0, %d]", G3PCF_MAX_NBINS, G3PCF_MAX_LMAX);
    if (ncat < 1 || ncat > G3PCF_MAX_COMBINE)
        return fail(G3PCF_ERR_ARG, "combine: ncat must be in [1, %d]", G3PCF_MAX_COMBINE);
    if (!zeta || !coef || !out) return fail(G3PCF_ERR_ARG, "combine: null pointer");
    for (int c = 0; c < ncat; ++c)
        if (!std::isfinite(coef[c])) return fail(G3PCF_ERR_ARG, "combine: coefficient %d is not finite", c);
    if (launch_combine(zeta, zsize_of(nbins, lmax), ncat, coef, out, static_cast<cudaStream_t>(stream)) != 0)
        return fail(G3PCF_ERR_CUDA, "combine launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return G3PCF_OK;
}

int g3pcf_destroy(g3pcf_plan_t P) {
    g_err.clear();
    if (!P) return G3PCF_OK;
    if (P->device >= 0) cudaStreamSynchronize(P->stream);
    DevBuf* bufs[] = {&P->key_a, &P->key_b, &P->val_a, &P->val_b, &P->hist, &P->hist_off,
                      &P->scan_tmp, &P->pts, &P->pts64, &P->orig, &P->cstart, &P->plist,
                      &P->small, &P->counts, &P->A, &P->partials, &P->d_tiles, &P->d_segs,
                      &P->d_segfirst, &P->d_colmap, &P->d_colscale, &P->d_colconv, &P->d_colcoef, &P->d_bintab_s, &P->d_slotconv, &P->d_slotcoef, &P->d_monoexp, &P->d_monoconv, &P->d_monoidx, &P->d_monocoef, &P->d_catoff, &P->d_ranges,
                      &P->d_tiles_tc, &P->d_cats, &P->d_mreal, &P->d_V, &P->d_bintab, &P->d_vblk,
                      &P->d_strips_tc, &P->d_items,
                      &P->d_slotcoefdf, &P->d_mrealdf, &P->d_Vdf, &P->d_colcoefdf,
                      &P->wrow, &P->l_need, &P->l_base, &P->l_nch, &P->l_pool, &P->l_tag, &P->l_ord,
                      &P->l_gbase, &P->l_scantmp, &P->l_passq};
    for (DevBuf* b : bufs) b->release();
    if (P->h_need) cudaFreeHost(P->h_need);
    if (P->h_base) cudaFreeHost(P->h_base);
    if (P->h_status) cudaFreeHost(P->h_status);
    if (P->h_stage) cudaFreeHost(P->h_stage);
    if (P->gexec) cudaGraphExecDestroy(P->gexec);
    if (P->gstream) cudaStreamDestroy(P->gstream);
    for (auto& e : P->gev)
        if (e) cudaEventDestroy(e);
    for (auto& e : P->ev)
        if (e) cudaEventDestroy(e);
    for (auto& e : P->lev) cudaEventDestroy(e);
    for (auto& e : P->cev) cudaEventDestroy(e);
    delete P;
    return G3PCF_OK;
}

}  // extern "C"
