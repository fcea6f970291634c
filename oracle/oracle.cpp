// FP64 CPU oracle for the anisotropic three-point correlation function (3PCF)
// of Friesen et al., "Galactos" (SC17, arXiv 1709.00086), Section 3.1.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
// definition that the CUDA path is checked against.  Only the test-suite, the
// smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
// no code, header, table or constant with the CUDA library, and it never calls
// into it.
//
// What is computed (Section 3.1, the expansion equation and Algorithm 1):
//   * edges        e_k = rmin + (rmax-rmin)*k/B, e_0 = rmin, e_B = rmax exactly
//   * pairs        primary i (< n_primary), secondary j (any point, j != i);
//                  separation d = x_j - x_i, minimum image per axis when the
//                  box is periodic ("if d > L/2: d -= L; if d < -L/2: d += L")
//   * bin          r2 = (dx*dx + dy*dy) + dz*dz in FP64 (no fused multiply-add);
//                  pair is in bin b iff e_b^2 <= r2 < e_{b+1}^2; r2 == 0 skipped
//   * frame        LOS = z (modes 0, 1) or the radial direction from the box
//                  centre to the primary (mode 2), the pair separation being
//                  rotated so that the LOS becomes +z (Section 3.1, Fig. 2)
//   * harmonics    Y_lm(theta, phi) = std::sph_legendre(l, m, theta) e^{i m phi}
//                  (orthonormal, Condon-Shortley phase) -- a library routine,
//                  not a recurrence of our own
//   * multipoles   a_lm(i, b) = sum_{j in b} w_j Y_lm(rhat'_ij), m >= 0
//                  (the discrete form of the integral over the shell, Sec 3.1)
//   * zeta         zeta^m_{l l'}(b1, b2) = sum_i w_i a_lm(i,b1) conj(a_l'm(i,b2))
//                  (the product of coefficients about one primary, summed over
//                  primaries, Sec 3.1)
//   * counts       number of ordered (i, j) pairs accepted into each bin
//   * gradient     of L = sum over all stored entries |zeta - zeta_t|^2 with the
//                  pair set and bins frozen (not in the paper; the adjoint's
//                  definition)
//   * monomials    the paper's own route to a_lm (Sec. 3.3.2): per primary and
//                  bin the power sums M_abc = sum_j w_j xhat^a yhat^b zhat^c over
//                  a + b + c <= lmax ((lmax+1)(lmax+2)(lmax+3)/6 of them, 286 at
//                  lmax = 10), then a_lm = sum_abc C^lm_abc M_abc with the
//                  expansion of Y_lm in those monomials
//
// Output layout of zeta: for m = 0..lmax a K_m x K_m complex block, K_m =
// B*(lmax+1-m), row (l-m)*B + b1, column (l'-m)*B + b2, (re, im) interleaved.
//
// Build: g++ -O2 -fopenmp -ffp-contract=off -shared -fPIC (contraction off so
// that r2 is rounded exactly as written above).

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef std::complex<double> cplx;

namespace {

const double kPi = 3.14159265358979323846264338327950288;

struct Geom {
    double box;
    int periodic;   // 1 for LOS mode 0 (periodic, z), 0 otherwise
    int radial;     // 1 for LOS mode 2 (radial from the box centre)
    int nbins;
    int lmax;
    std::vector<double> e2;  // squared edges, nbins+1
};

int make_geom(Geom& g, int nbins, double rmin, double rmax, int lmax, double box,
              int los_mode) {
    if (nbins < 1 || lmax < 0 || !(rmin >= 0.0) || !(rmax > rmin) || !(box > 0.0))
        return -1;
    if (los_mode < 0 || los_mode > 2) return -1;
    g.box = box;
    g.periodic = (los_mode == 0);
    g.radial = (los_mode == 2);
    g.nbins = nbins;
    g.lmax = lmax;
    g.e2.resize(nbins + 1);
    for (int k = 0; k <= nbins; ++k) {
        double e;
        if (k == 0) e = rmin;
        else if (k == nbins) e = rmax;
        else e = rmin + ((rmax - rmin) * (double)k) / (double)nbins;
        g.e2[k] = e * e;
    }
    return 0;
}

// Separation, image shift and radial bin of the pair (i -> j).  Returns the
// bin or -1.  sh[] receives the integer image shift applied per axis.
int pair_bin(const Geom& g, const double* xi, const double* xj, double d[3], int sh[3]) {
    for (int a = 0; a < 3; ++a) {
        double t = xj[a] - xi[a];
        int s = 0;
        if (g.periodic) {
            if (t > 0.5 * g.box) { t -= g.box; s = -1; }
            else if (t < -0.5 * g.box) { t += g.box; s = 1; }
        }
        d[a] = t;
        sh[a] = s;
    }
    double r2 = d[0] * d[0] + d[1] * d[1];
    r2 = r2 + d[2] * d[2];
    if (r2 == 0.0) return -1;
    if (r2 < g.e2[0] || !(r2 < g.e2[g.nbins])) return -1;
    int b = 0;
    while (b + 1 < g.nbins && g.e2[b + 1] <= r2) ++b;
    return b;
}

// Rotation taking the primary's line of sight to +z (identity for z modes).
// Radial mode: n = (x_i - c)/|x_i - c|, c the box centre (n = z if x_i = c);
// Rodrigues rotation about n x z; a half turn about x when n is (nearly) -z.
void los_rotation(const Geom& g, const double* xi, double R[9]) {
    for (int k = 0; k < 9; ++k) R[k] = (k % 4 == 0) ? 1.0 : 0.0;
    if (!g.radial) return;
    double c = 0.5 * g.box;
    double n[3] = {xi[0] - c, xi[1] - c, xi[2] - c};
    double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (nn == 0.0) return;
    for (int a = 0; a < 3; ++a) n[a] /= nn;
    double ct = n[2];
    if (ct < -1.0 + 1e-12) {
        R[4] = -1.0;
        R[8] = -1.0;
        return;
    }
    // v = n x z = (n_y, -n_x, 0); R = I + [v]x + [v]x^2 / (1 + ct)
    double v[3] = {n[1], -n[0], 0.0};
    double K[9] = {0.0, -v[2], v[1], v[2], 0.0, -v[0], -v[1], v[0], 0.0};
    double K2[9];
    for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 3; ++s) {
            double acc = 0.0;
            for (int t = 0; t < 3; ++t) acc += K[3 * r + t] * K[3 * t + s];
            K2[3 * r + s] = acc;
        }
    for (int k = 0; k < 9; ++k) R[k] += K[k] + K2[k] / (1.0 + ct);
}

inline int lm_index(int l, int m) { return l * (l + 1) / 2 + m; }
inline int n_lm(int lmax) { return (lmax + 1) * (lmax + 2) / 2; }

// Y_lm(rhat) for 0 <= m <= l <= lmax, via the library's spherical Legendre
// function.  out[lm_index(l,m)].
void ylm_all(int lmax, const double d[3], cplx* out) {
    double r = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double ct = d[2] / r;
    if (ct > 1.0) ct = 1.0;
    if (ct < -1.0) ct = -1.0;
    double theta = std::acos(ct);
    double phi = std::atan2(d[1], d[0]);
    for (int l = 0; l <= lmax; ++l)
        for (int m = 0; m <= l; ++m) {
            double p = std::sph_legendre((unsigned)l, (unsigned)m, theta);
            out[lm_index(l, m)] = p * cplx(std::cos(m * phi), std::sin(m * phi));
        }
}

// Y_{l,m} for any integer m (Y_{l,-m} = (-1)^m conj(Y_lm)); zero if |m| > l.
cplx ylm_signed(const cplx* Y, int l, int m) {
    if (l < 0 || m > l || -m > l) return cplx(0.0, 0.0);
    if (m >= 0) return Y[lm_index(l, m)];
    cplx v = std::conj(Y[lm_index(l, -m)]);
    return (((-m) & 1) ? -v : v);
}

// Gradient of Y_lm(d/|d|) with respect to the separation d, from the ladder
// relations of the regular solid harmonics R_lm = r^l Y_lm:
//   dz R_lm          =  sqrt((2l+1)/(2l-1) (l-m)(l+m))   R_{l-1,m}
//   (dx + i dy) R_lm =  sqrt((2l+1)/(2l-1) (l-m)(l-m-1)) R_{l-1,m+1}
//   (dx - i dy) R_lm = -sqrt((2l+1)/(2l-1) (l+m)(l+m-1)) R_{l-1,m-1}
// and grad Y_lm = r^-l grad R_lm - l r^-2 Y_lm d.  Y holds Y_{l'm'}(rhat) for
// l' <= lmax (computed by ylm_all); gY receives 3 complex per (l, m >= 0).
void ylm_grad_all(int lmax, const double d[3], const cplx* Y, cplx* gY) {
    double r = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double rhat[3] = {d[0] / r, d[1] / r, d[2] / r};
    for (int l = 0; l <= lmax; ++l)
        for (int m = 0; m <= l; ++m) {
            cplx gx(0.0, 0.0), gy(0.0, 0.0), gz(0.0, 0.0);
            if (l >= 1) {
                double f = (2.0 * l + 1.0) / (2.0 * l - 1.0);
                double cz = std::sqrt(f * (double)(l - m) * (double)(l + m));
                double cp = std::sqrt(f * (double)(l - m) * (double)(l - m - 1));
                double cm = -std::sqrt(f * (double)(l + m) * (double)(l + m - 1));
                cplx up = cp * ylm_signed(Y, l - 1, m + 1);   // (dx + i dy) R / r^(l-1)
                cplx dn = cm * ylm_signed(Y, l - 1, m - 1);   // (dx - i dy) R / r^(l-1)
                gx = 0.5 * (up + dn) / r;
                gy = (up - dn) / (cplx(0.0, 2.0) * r);
                gz = cz * ylm_signed(Y, l - 1, m) / r;
            }
            cplx y = Y[lm_index(l, m)];
            double s = (double)l / r;
            gY[3 * lm_index(l, m) + 0] = gx - s * y * rhat[0];
            gY[3 * lm_index(l, m) + 1] = gy - s * y * rhat[1];
            gY[3 * lm_index(l, m) + 2] = gz - s * y * rhat[2];
        }
}

inline int64_t zeta_block_offset(int nbins, int lmax, int m) {
    int64_t off = 0;
    for (int mm = 0; mm < m; ++mm) {
        int64_t K = (int64_t)nbins * (lmax + 1 - mm);
        off += K * K;
    }
    return off;  // in complex entries
}

inline int64_t zeta_size(int nbins, int lmax) { return zeta_block_offset(nbins, lmax, lmax + 1); }

// a_lm(i, b) for one primary, all n points as secondaries.  alm: nbins*nlm
// complex, zeroed here.  Optional frozen geometry: if pos_bins is given, the
// pair set, bins and image shifts come from pos_bins and only the separation
// vectors come from pos.
void alm_one(const Geom& g, const double* pos, const double* pos_bins, const double* w,
             int64_t n, int64_t i, cplx* alm, int64_t* counts) {
    const int nlm = n_lm(g.lmax);
    std::fill(alm, alm + (int64_t)g.nbins * nlm, cplx(0.0, 0.0));
    std::vector<cplx> Y(nlm);
    const double* P = pos_bins ? pos_bins : pos;
    double R[9];
    los_rotation(g, pos + 3 * i, R);
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        double d[3];
        int sh[3];
        int b = pair_bin(g, P + 3 * i, P + 3 * j, d, sh);
        if (b < 0) continue;
        if (pos_bins) {
            for (int a = 0; a < 3; ++a) d[a] = (pos[3 * j + a] - pos[3 * i + a]) + sh[a] * g.box;
        }
        double dr[3];
        for (int a = 0; a < 3; ++a) dr[a] = R[3 * a] * d[0] + R[3 * a + 1] * d[1] + R[3 * a + 2] * d[2];
        ylm_all(g.lmax, dr, Y.data());
        cplx* ab = alm + (int64_t)b * nlm;
        for (int k = 0; k < nlm; ++k) ab[k] += w[j] * Y[k];
        if (counts) counts[b] += 1;
    }
}

// zeta += wi * a a^H (per m block), alm of one primary in [b][lm] layout.
void zeta_accumulate(int nbins, int lmax, const cplx* alm, double wi, cplx* zeta) {
    const int nlm = n_lm(lmax);
    for (int m = 0; m <= lmax; ++m) {
        const int64_t K = (int64_t)nbins * (lmax + 1 - m);
        cplx* Z = zeta + zeta_block_offset(nbins, lmax, m);
        for (int l = m; l <= lmax; ++l)
            for (int b1 = 0; b1 < nbins; ++b1) {
                const int64_t r = (int64_t)(l - m) * nbins + b1;
                const cplx a1 = wi * alm[(int64_t)b1 * nlm + lm_index(l, m)];
                for (int lp = m; lp <= lmax; ++lp)
                    for (int b2 = 0; b2 < nbins; ++b2) {
                        const int64_t c = (int64_t)(lp - m) * nbins + b2;
                        Z[r * K + c] += a1 * std::conj(alm[(int64_t)b2 * nlm + lm_index(lp, m)]);
                    }
            }
    }
}

// ---- the monomial route (Sec. 3.3.2) -------------------------------------

// Monomials xhat^a yhat^b zhat^c with a + b + c <= lmax, enumerated by degree
// n = a + b + c, then a descending, then b descending.
struct Monomials {
    std::vector<int> a, b, c;
    std::vector<int> index;  // (a * (L+1) + b) * (L+1) + c -> position, -1 if none
    int L;
    explicit Monomials(int lmax) : L(lmax) {
        index.assign((size_t)(L + 1) * (L + 1) * (L + 1), -1);
        for (int n = 0; n <= L; ++n)
            for (int ia = n; ia >= 0; --ia)
                for (int ib = n - ia; ib >= 0; --ib) {
                    const int ic = n - ia - ib;
                    index[((size_t)ia * (L + 1) + ib) * (L + 1) + ic] = (int)a.size();
                    a.push_back(ia);
                    b.push_back(ib);
                    c.push_back(ic);
                }
    }
    int count() const { return (int)a.size(); }
    int at(int ia, int ib, int ic) const { return index[((size_t)ia * (L + 1) + ib) * (L + 1) + ic]; }
};

double binom(int n, int k) {
    double r = 1.0;
    for (int t = 1; t <= k; ++t) r = r * (n - k + t) / t;
    return r;
}

// Y_lm on the unit sphere as a polynomial in (xhat, yhat, zhat):
//   Y_lm = N_lm (-1)^m P_l^(m)(zhat) (xhat + i yhat)^m,
// P_l^(m) the m-th derivative of the Legendre polynomial (so that N_lm (-1)^m
// (1 - z^2)^(m/2) P_l^(m) is the orthonormal associated Legendre function with
// the Condon-Shortley phase, and sin^m(theta) e^(i m phi) = (xhat + i yhat)^m),
// P_l(z) = 2^-l sum_j (-1)^j C(l, j) C(2l - 2j, l) z^(l - 2j).  Returns, per
// (l, m) in lm_index order, the list of (monomial, complex coefficient).
std::vector<std::vector<std::pair<int, cplx>>> ylm_monomial_coefficients(const Monomials& M) {
    const int L = M.L;
    std::vector<std::vector<std::pair<int, cplx>>> out((size_t)n_lm(L));
    for (int l = 0; l <= L; ++l) {
        std::vector<double> p(l + 1, 0.0);  // P_l coefficients by power of z
        for (int j = 0; 2 * j <= l; ++j)
            p[l - 2 * j] = std::ldexp(((j & 1) ? -1.0 : 1.0) * binom(l, j) * binom(2 * l - 2 * j, l), -l);
        for (int m = 0; m <= l; ++m) {
            // m-th derivative: coefficient of z^k is p[k + m] (k + m)! / k!
            std::vector<double> d(l - m + 1, 0.0);
            for (int k = 0; k + m <= l; ++k) {
                double f = 1.0;
                for (int t = k + 1; t <= k + m; ++t) f *= t;
                d[k] = p[k + m] * f;
            }
            double ratio = 1.0;  // (l - m)! / (l + m)!
            for (int t = l - m + 1; t <= l + m; ++t) ratio /= t;
            const double N = std::sqrt((2 * l + 1) / (4.0 * kPi) * ratio) * ((m & 1) ? -1.0 : 1.0);
            auto& terms = out[lm_index(l, m)];
            for (int k = 0; k <= l - m; ++k) {
                if (d[k] == 0.0) continue;
                for (int t = 0; t <= m; ++t) {  // C(m, t) xhat^(m-t) (i yhat)^t
                    static const cplx ipow[4] = {cplx(1, 0), cplx(0, 1), cplx(-1, 0), cplx(0, -1)};
                    terms.push_back({M.at(m - t, t, k), N * d[k] * binom(m, t) * ipow[t & 3]});
                }
            }
        }
    }
    return out;
}

// a_lm(i, b) for one primary through the monomial power sums: the pairs and
// frame are those of alm_one; per pair the unit separation's monomials are
// added (weighted) to the sums of its bin, and the sums are converted at the end.
void alm_one_monomial(const Geom& g, const Monomials& M,
                      const std::vector<std::vector<std::pair<int, cplx>>>& C, const double* pos,
                      const double* w, int64_t n, int64_t i, cplx* alm) {
    const int nlm = n_lm(g.lmax), nm = M.count(), L = g.lmax;
    std::vector<double> S((size_t)g.nbins * nm, 0.0);
    std::vector<double> px(L + 1), py(L + 1), pz(L + 1);
    double R[9];
    los_rotation(g, pos + 3 * i, R);
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        double d[3];
        int sh[3];
        const int b = pair_bin(g, pos + 3 * i, pos + 3 * j, d, sh);
        if (b < 0) continue;
        double dr[3];
        for (int a = 0; a < 3; ++a) dr[a] = R[3 * a] * d[0] + R[3 * a + 1] * d[1] + R[3 * a + 2] * d[2];
        const double r = std::sqrt(dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2]);
        px[0] = py[0] = pz[0] = 1.0;
        for (int k = 1; k <= L; ++k) {
            px[k] = px[k - 1] * (dr[0] / r);
            py[k] = py[k - 1] * (dr[1] / r);
            pz[k] = pz[k - 1] * (dr[2] / r);
        }
        double* Sb = S.data() + (size_t)b * nm;
        for (int t = 0; t < nm; ++t) Sb[t] += w[j] * px[M.a[t]] * py[M.b[t]] * pz[M.c[t]];
    }
    for (int b = 0; b < g.nbins; ++b)
        for (int k = 0; k < nlm; ++k) {
            cplx v(0.0, 0.0);
            for (const auto& tc : C[k]) v += tc.second * S[(size_t)b * nm + tc.first];
            alm[(int64_t)b * nlm + k] = v;
        }
}

int threads_of(int nthreads) {
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

}  // namespace

extern "C" {

// Number of complex entries of the zeta output.
int64_t orc_zeta_size(int nbins, int lmax) { return zeta_size(nbins, lmax); }

int orc_edges(int nbins, double rmin, double rmax, double* edges2) {
    Geom g;
    if (make_geom(g, nbins, rmin, rmax, 0, 1.0, 1) != 0) return -1;
    for (int k = 0; k <= nbins; ++k) edges2[k] = g.e2[k];
    return 0;
}

// Y_lm at n directions d (n x 3, need not be unit): out n x nlm complex.
int orc_ylm(int lmax, const double* d, int64_t n, double* out) {
    const int nlm = n_lm(lmax);
    for (int64_t k = 0; k < n; ++k)
        ylm_all(lmax, d + 3 * k, reinterpret_cast<cplx*>(out) + k * nlm);
    return 0;
}

// grad_d Y_lm(d/|d|): out n x nlm x 3 complex.
int orc_ylm_grad(int lmax, const double* d, int64_t n, double* out) {
    const int nlm = n_lm(lmax + 1);
    std::vector<cplx> Y(nlm);
    for (int64_t k = 0; k < n; ++k) {
        ylm_all(lmax, d + 3 * k, Y.data());
        ylm_grad_all(lmax, d + 3 * k, Y.data(), reinterpret_cast<cplx*>(out) + k * 3 * n_lm(lmax));
    }
    return 0;
}

// Per-primary multipoles for the listed primaries: alm np x nbins x nlm
// complex; counts (nbins int64, may be null) accumulates their pair counts.
int orc_alm(const double* pos, const double* w, int64_t n, const int64_t* prim, int64_t np,
            double box, int los_mode, int nbins, double rmin, double rmax, int lmax,
            double* alm, int64_t* counts, int nthreads) {
    Geom g;
    if (make_geom(g, nbins, rmin, rmax, lmax, box, los_mode) != 0) return -1;
    const int nlm = n_lm(lmax);
    const int nt = threads_of(nthreads);
    std::vector<std::vector<int64_t>> tc(nt, std::vector<int64_t>(nbins, 0));
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int64_t k = 0; k < np; ++k) {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        alm_one(g, pos, nullptr, w, n, prim[k],
                reinterpret_cast<cplx*>(alm) + k * (int64_t)nbins * nlm, tc[t].data());
    }
    if (counts)
        for (int t = 0; t < nt; ++t)
            for (int b = 0; b < nbins; ++b) counts[b] += tc[t][b];
    return 0;
}

// Number of monomials with a + b + c <= lmax (the paper's power sums).
int64_t orc_mono_count(int lmax) { return lmax < 0 ? 0 : Monomials(lmax).count(); }

// Per-primary multipoles through the monomial power sums (Sec. 3.3.2); same
// arguments and output layout as orc_alm.
int orc_alm_monomial(const double* pos, const double* w, int64_t n, const int64_t* prim, int64_t np,
                     double box, int los_mode, int nbins, double rmin, double rmax, int lmax,
                     double* alm, int nthreads) {
    Geom g;
    if (make_geom(g, nbins, rmin, rmax, lmax, box, los_mode) != 0) return -1;
    const Monomials M(lmax);
    const auto C = ylm_monomial_coefficients(M);
    const int nlm = n_lm(lmax);
    const int nt = threads_of(nthreads);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int64_t k = 0; k < np; ++k)
        alm_one_monomial(g, M, C, pos, w, n, prim[k], reinterpret_cast<cplx*>(alm) + k * (int64_t)nbins * nlm);
    return 0;
}

// zeta over primaries 0..n_primary-1 (all n points are secondaries).
// pos_bins: optional frozen pair geometry (see alm_one), may be null.
int orc_zeta(const double* pos, const double* pos_bins, const double* w, int64_t n,
             int64_t n_primary, double box, int los_mode, int nbins, double rmin, double rmax,
             int lmax, double* zeta, int64_t* counts, int nthreads) {
    Geom g;
    if (make_geom(g, nbins, rmin, rmax, lmax, box, los_mode) != 0) return -1;
    const int nlm = n_lm(lmax);
    const int64_t zs = zeta_size(nbins, lmax);
    const int nt = threads_of(nthreads);
    std::vector<std::vector<cplx>> tz(nt, std::vector<cplx>(zs, cplx(0.0, 0.0)));
    std::vector<std::vector<int64_t>> tc(nt, std::vector<int64_t>(nbins, 0));
#pragma omp parallel num_threads(nt)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        std::vector<cplx> alm((int64_t)nbins * nlm);
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < n_primary; ++i) {
            alm_one(g, pos, pos_bins, w, n, i, alm.data(), tc[t].data());
            zeta_accumulate(nbins, lmax, alm.data(), w[i], tz[t].data());
        }
    }
    cplx* Z = reinterpret_cast<cplx*>(zeta);
    std::fill(Z, Z + zs, cplx(0.0, 0.0));
    for (int t = 0; t < nt; ++t)
        for (int64_t k = 0; k < zs; ++k) Z[k] += tz[t][k];
    if (counts)
        for (int t = 0; t < nt; ++t)
            for (int b = 0; b < nbins; ++b) counts[b] += tc[t][b];
    return 0;
}

// zeta from given per-primary multipoles (np x nbins x nlm complex) and weights.
int orc_zeta_from_alm(const double* alm, const double* wprim, int64_t np, int nbins,
                      int lmax, double* zeta) {
    const int nlm = n_lm(lmax);
    const int64_t zs = zeta_size(nbins, lmax);
    cplx* Z = reinterpret_cast<cplx*>(zeta);
    std::fill(Z, Z + zs, cplx(0.0, 0.0));
    for (int64_t i = 0; i < np; ++i)
        zeta_accumulate(nbins, lmax, reinterpret_cast<const cplx*>(alm) + i * (int64_t)nbins * nlm,
                        wprim[i], Z);
    return 0;
}

// O(N^3) triplet sum: zeta^m_{ll'}(b1,b2) = sum_i w_i sum_{j in b1} sum_{k in b2}
// w_j w_k Y_lm(rhat_ij) conj(Y_l'm(rhat_ik)), j = k included.  Tiny N only.
int orc_zeta_triplets(const double* pos, const double* w, int64_t n, double box, int los_mode,
                      int nbins, double rmin, double rmax, int lmax, double* zeta) {
    Geom g;
    if (make_geom(g, nbins, rmin, rmax, lmax, box, los_mode) != 0) return -1;
    const int nlm = n_lm(lmax);
    cplx* Z = reinterpret_cast<cplx*>(zeta);
    std::fill(Z, Z + zeta_size(nbins, lmax), cplx(0.0, 0.0));
    std::vector<cplx> Yj(nlm), Yk(nlm);
    for (int64_t i = 0; i < n; ++i) {
        double R[9];
        los_rotation(g, pos + 3 * i, R);
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dj[3], rj[3];
            int sj[3];
            int bj = pair_bin(g, pos + 3 * i, pos + 3 * j, dj, sj);
            if (bj < 0) continue;
            for (int a = 0; a < 3; ++a) rj[a] = R[3 * a] * dj[0] + R[3 * a + 1] * dj[1] + R[3 * a + 2] * dj[2];
            ylm_all(lmax, rj, Yj.data());
            for (int64_t k = 0; k < n; ++k) {
                if (k == i) continue;
                double dk[3], rk[3];
                int sk[3];
                int bk = pair_bin(g, pos + 3 * i, pos + 3 * k, dk, sk);
                if (bk < 0) continue;
                for (int a = 0; a < 3; ++a) rk[a] = R[3 * a] * dk[0] + R[3 * a + 1] * dk[1] + R[3 * a + 2] * dk[2];
                ylm_all(lmax, rk, Yk.data());
                const double wt = w[i] * w[j] * w[k];
                for (int m = 0; m <= lmax; ++m) {
                    const int64_t K = (int64_t)nbins * (lmax + 1 - m);
                    cplx* Zm = Z + zeta_block_offset(nbins, lmax, m);
                    for (int l = m; l <= lmax; ++l)
                        for (int lp = m; lp <= lmax; ++lp)
                            Zm[((int64_t)(l - m) * nbins + bj) * K + (int64_t)(lp - m) * nbins + bk] +=
                                wt * Yj[lm_index(l, m)] * std::conj(Yk[lm_index(lp, m)]);
                }
            }
        }
    }
    return 0;
}

// Isotropic Legendre 3PCF by brute force over pairs of pairs (Section 2.2):
// iso[l][b1][b2] = (2l+1)/(4 pi) sum_i w_i sum_{j in b1, k in b2} w_j w_k
// P_l(rhat_ij . rhat_ik), j = k included.  Output (lmax+1) x nbins x nbins.
int orc_iso_legendre(const double* pos, const double* w, int64_t n, double box, int los_mode,
                     int nbins, double rmin, double rmax, int lmax, double* iso) {
    Geom g;
    if (make_geom(g, nbins, rmin, rmax, lmax, box, los_mode) != 0) return -1;
    std::fill(iso, iso + (int64_t)(lmax + 1) * nbins * nbins, 0.0);
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dj[3];
            int sj[3];
            int bj = pair_bin(g, pos + 3 * i, pos + 3 * j, dj, sj);
            if (bj < 0) continue;
            double rj = std::sqrt(dj[0] * dj[0] + dj[1] * dj[1] + dj[2] * dj[2]);
            for (int64_t k = 0; k < n; ++k) {
                if (k == i) continue;
                double dk[3];
                int sk[3];
                int bk = pair_bin(g, pos + 3 * i, pos + 3 * k, dk, sk);
                if (bk < 0) continue;
                double rk = std::sqrt(dk[0] * dk[0] + dk[1] * dk[1] + dk[2] * dk[2]);
                double mu = (dj[0] * dk[0] + dj[1] * dk[1] + dj[2] * dk[2]) / (rj * rk);
                if (mu > 1.0) mu = 1.0;
                if (mu < -1.0) mu = -1.0;
                const double wt = w[i] * w[j] * w[k];
                for (int l = 0; l <= lmax; ++l)
                    iso[((int64_t)l * nbins + bj) * nbins + bk] +=
                        (2.0 * l + 1.0) / (4.0 * kPi) * wt * std::legendre((unsigned)l, mu);
            }
        }
    }
    return 0;
}

// Reference gradient of L = sum over all stored entries |zeta - zeta_t|^2,
// given G = zeta - zeta_t (same layout as zeta), LOS = z modes only, every
// point a primary (n_primary = n).  Pair set and bins are held fixed.
//   H_{i,m} = w_i (G_m + G_m^H) A_{i,m}
//   dL/dw_i      += 2 sum_m Re(A_{i,m}^H G_m A_{i,m})
//   dL/dw_j      += sum_i 2 Re sum_lm conj(H_{i,lm,b}) Y_lm(rhat_ij)
//   dL/dd_ij      = 2 w_j Re sum_lm conj(H_{i,lm,b}) grad_d Y_lm(d_ij)
//   dpos_j += dL/dd_ij, dpos_i -= dL/dd_ij
int orc_grad(const double* pos, const double* w, int64_t n, double box, int los_mode, int nbins,
             double rmin, double rmax, int lmax, const double* Gz, double* dpos, double* dw,
             int nthreads) {
    Geom g;
    if (make_geom(g, nbins, rmin, rmax, lmax, box, los_mode) != 0) return -1;
    if (g.radial) return -2;
    const int nlm = n_lm(lmax);
    const cplx* G = reinterpret_cast<const cplx*>(Gz);
    const int nt = threads_of(nthreads);
    std::vector<std::vector<double>> tdpos(nt, std::vector<double>(3 * n, 0.0));
    std::vector<std::vector<double>> tdw(nt, std::vector<double>(n, 0.0));
#pragma omp parallel num_threads(nt)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        std::vector<cplx> alm((int64_t)nbins * nlm), H((int64_t)nbins * nlm);
        std::vector<cplx> Y(n_lm(lmax + 1)), gY(3 * (int64_t)nlm);
        double* mydpos = tdpos[t].data();
        double* mydw = tdw[t].data();
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < n; ++i) {
            alm_one(g, pos, nullptr, w, n, i, alm.data(), nullptr);
            // H and the primary-weight term, block by block.
            std::fill(H.begin(), H.end(), cplx(0.0, 0.0));
            double dwi = 0.0;
            for (int m = 0; m <= lmax; ++m) {
                const int64_t K = (int64_t)nbins * (lmax + 1 - m);
                const cplx* Gm = G + zeta_block_offset(nbins, lmax, m);
                for (int l = m; l <= lmax; ++l)
                    for (int b1 = 0; b1 < nbins; ++b1) {
                        const int64_t r = (int64_t)(l - m) * nbins + b1;
                        cplx acc(0.0, 0.0), accG(0.0, 0.0);
                        for (int lp = m; lp <= lmax; ++lp)
                            for (int b2 = 0; b2 < nbins; ++b2) {
                                const int64_t c = (int64_t)(lp - m) * nbins + b2;
                                const cplx a = alm[(int64_t)b2 * nlm + lm_index(lp, m)];
                                acc += (Gm[r * K + c] + std::conj(Gm[c * K + r])) * a;
                                accG += Gm[r * K + c] * a;
                            }
                        const cplx ar = alm[(int64_t)b1 * nlm + lm_index(l, m)];
                        H[(int64_t)b1 * nlm + lm_index(l, m)] = w[i] * acc;
                        dwi += 2.0 * std::real(std::conj(ar) * accG);
                    }
            }
            mydw[i] += dwi;
            // Pair pass: secondary weights and separations.
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                double d[3];
                int sh[3];
                int b = pair_bin(g, pos + 3 * i, pos + 3 * j, d, sh);
                if (b < 0) continue;
                ylm_all(lmax, d, Y.data());
                ylm_grad_all(lmax, d, Y.data(), gY.data());
                double sw = 0.0, sd[3] = {0.0, 0.0, 0.0};
                for (int l = 0; l <= lmax; ++l)
                    for (int m = 0; m <= l; ++m) {
                        const cplx h = std::conj(H[(int64_t)b * nlm + lm_index(l, m)]);
                        sw += std::real(h * Y[lm_index(l, m)]);
                        for (int a = 0; a < 3; ++a) sd[a] += std::real(h * gY[3 * lm_index(l, m) + a]);
                    }
                mydw[j] += 2.0 * sw;
                for (int a = 0; a < 3; ++a) {
                    const double v = 2.0 * w[j] * sd[a];
                    mydpos[3 * j + a] += v;
                    mydpos[3 * i + a] -= v;
                }
            }
        }
    }
    std::fill(dpos, dpos + 3 * n, 0.0);
    std::fill(dw, dw + n, 0.0);
    for (int t = 0; t < nt; ++t) {
        for (int64_t k = 0; k < 3 * n; ++k) dpos[k] += tdpos[t][k];
        for (int64_t k = 0; k < n; ++k) dw[k] += tdw[t][k];
    }
    return 0;
}

// The reference gradient of orc_grad restricted to nsel chosen galaxies
// sel[k] (each a primary and a secondary, every point a primary): galaxy s
// receives its primary terms (the primary-weight term and -dL/dd over its own
// pairs) and, for every primary i with s among its accepted secondaries, the
// terms of the pair (i, s).  Only the primaries within rmax of a chosen galaxy
// (and the chosen ones) have their multipoles evaluated, so a large catalog
// costs about (number of such primaries) x n pair tests.  dpos: nsel x 3,
// dw: nsel, in the order of sel.
int orc_grad_sel(const double* pos, const double* w, int64_t n, double box, int los_mode, int nbins,
                 double rmin, double rmax, int lmax, const double* Gz, const int64_t* sel, int64_t nsel,
                 double* dpos, double* dw, int nthreads) {
    Geom g;
    if (make_geom(g, nbins, rmin, rmax, lmax, box, los_mode) != 0) return -1;
    if (g.radial) return -2;
    const int nlm = n_lm(lmax);
    const cplx* G = reinterpret_cast<const cplx*>(Gz);
    const int nt = threads_of(nthreads);
    std::vector<int64_t> slot(n, -1);
    for (int64_t k = 0; k < nsel; ++k) {
        if (sel[k] < 0 || sel[k] >= n || slot[sel[k]] >= 0) return -3;
        slot[sel[k]] = k;
    }
    // primaries whose multipoles are needed: the chosen galaxies and every
    // primary that has a chosen galaxy among its accepted secondaries
    std::vector<char> need(n, 0);
    for (int64_t k = 0; k < nsel; ++k) need[sel[k]] = 1;
#pragma omp parallel for schedule(static) num_threads(nt)
    for (int64_t i = 0; i < n; ++i) {
        if (need[i]) continue;
        for (int64_t k = 0; k < nsel; ++k) {
            double d[3];
            int sh[3];
            if (pair_bin(g, pos + 3 * i, pos + 3 * sel[k], d, sh) >= 0) {
                need[i] = 1;
                break;
            }
        }
    }
    std::vector<int64_t> prim;
    for (int64_t i = 0; i < n; ++i)
        if (need[i]) prim.push_back(i);
    std::vector<std::vector<double>> tdpos(nt, std::vector<double>(3 * nsel, 0.0));
    std::vector<std::vector<double>> tdw(nt, std::vector<double>(nsel, 0.0));
#pragma omp parallel num_threads(nt)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        std::vector<cplx> alm((int64_t)nbins * nlm), H((int64_t)nbins * nlm);
        std::vector<cplx> Y(n_lm(lmax + 1)), gY(3 * (int64_t)nlm);
        double* mydpos = tdpos[t].data();
        double* mydw = tdw[t].data();
#pragma omp for schedule(dynamic, 1)
        for (int64_t k = 0; k < (int64_t)prim.size(); ++k) {
            const int64_t i = prim[k];
            const int64_t si = slot[i];
            alm_one(g, pos, nullptr, w, n, i, alm.data(), nullptr);
            // H = w_i (G + G^H) A and the primary-weight term, as in orc_grad
            std::fill(H.begin(), H.end(), cplx(0.0, 0.0));
            double dwi = 0.0;
            for (int m = 0; m <= lmax; ++m) {
                const int64_t K = (int64_t)nbins * (lmax + 1 - m);
                const cplx* Gm = G + zeta_block_offset(nbins, lmax, m);
                for (int l = m; l <= lmax; ++l)
                    for (int b1 = 0; b1 < nbins; ++b1) {
                        const int64_t r = (int64_t)(l - m) * nbins + b1;
                        cplx acc(0.0, 0.0), accG(0.0, 0.0);
                        for (int lp = m; lp <= lmax; ++lp)
                            for (int b2 = 0; b2 < nbins; ++b2) {
                                const int64_t c = (int64_t)(lp - m) * nbins + b2;
                                const cplx a = alm[(int64_t)b2 * nlm + lm_index(lp, m)];
                                acc += (Gm[r * K + c] + std::conj(Gm[c * K + r])) * a;
                                accG += Gm[r * K + c] * a;
                            }
                        const cplx ar = alm[(int64_t)b1 * nlm + lm_index(l, m)];
                        H[(int64_t)b1 * nlm + lm_index(l, m)] = w[i] * acc;
                        dwi += 2.0 * std::real(std::conj(ar) * accG);
                    }
            }
            if (si >= 0) mydw[si] += dwi;
            // pairs (i, j) that touch a chosen galaxy: j chosen, or i chosen
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                const int64_t sj = slot[j];
                if (si < 0 && sj < 0) continue;
                double d[3];
                int sh[3];
                int b = pair_bin(g, pos + 3 * i, pos + 3 * j, d, sh);
                if (b < 0) continue;
                ylm_all(lmax, d, Y.data());
                ylm_grad_all(lmax, d, Y.data(), gY.data());
                double sw = 0.0, sd[3] = {0.0, 0.0, 0.0};
                for (int l = 0; l <= lmax; ++l)
                    for (int m = 0; m <= l; ++m) {
                        const cplx h = std::conj(H[(int64_t)b * nlm + lm_index(l, m)]);
                        sw += std::real(h * Y[lm_index(l, m)]);
                        for (int a = 0; a < 3; ++a) sd[a] += std::real(h * gY[3 * lm_index(l, m) + a]);
                    }
                if (sj >= 0) mydw[sj] += 2.0 * sw;
                for (int a = 0; a < 3; ++a) {
                    const double v = 2.0 * w[j] * sd[a];
                    if (sj >= 0) mydpos[3 * sj + a] += v;
                    if (si >= 0) mydpos[3 * si + a] -= v;
                }
            }
        }
    }
    std::fill(dpos, dpos + 3 * nsel, 0.0);
    std::fill(dw, dw + nsel, 0.0);
    for (int t = 0; t < nt; ++t) {
        for (int64_t k = 0; k < 3 * nsel; ++k) dpos[k] += tdpos[t][k];
        for (int64_t k = 0; k < nsel; ++k) dw[k] += tdw[t][k];
    }
    return 0;
}

}  // extern "C"
