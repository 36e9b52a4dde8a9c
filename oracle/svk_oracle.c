/*
 * svk_oracle.c -- plain, slow FP64 CPU oracle for the spatially-varying kernel
 * convolution of Optimal Image Subtraction (Hartung, Shukla, Miller, Pennypacker,
 * "GPU Acceleration of Image Convolution Using Spatially-Varying Kernel").
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg may load this library.  It shares no code, header or table with the
 * CUDA library under paper_1209_5823_gb300/; the product path never calls it.
 *
 * Every function follows the paper's statement of the problem (Sec. 2):
 *   Eq. 1   D = (R (x) K) - I
 *   Eq. 2   K_{x,y} = sum_i a_i(x,y) B_i          (a different kernel at every pixel)
 *   Eq. 3   a(x,y) = bivariate polynomial of order n (n = 2 written out in the paper)
 * and the cost models of Sec. 3.  Readings of what the paper leaves open:
 *   - (x) is a true convolution: out(x,y) = sum_{u,v} K(u,v) R(x-u, y-v);
 *   - the kernel is evaluated at the OUTPUT pixel (x,y) (gather form, Sec. 4: one
 *     thread and one kernel per output pixel);
 *   - R is zero outside the frame; the output has the size of R;
 *   - polynomial coordinates are normalised to [-1, 1] over the frame,
 *     xt = (2x - (W-1)) / (W-1) (xt = 0 when W == 1), likewise yt;
 *   - monomials m_t = xt^i yt^j for i + j <= d, i outer, j inner, so d = 2 gives
 *     1, yt, yt^2, xt, xt*yt, xt^2 -- the six terms of Eq. 3;
 *   - coefficients c[k][t] with a_k(x,y) = sum_t c[k][t] m_t(xt, yt);
 *   - basis stamps stored basis[k][v+h][u+h] (row = v = y offset, column = u = x
 *     offset), h = (L-1)/2.
 *
 * Pins (tests/test_oracle_pins.py): FFT and direct library convolution for spatially
 * constant a_k, closed forms for delta bases, impulse responses, flux conservation,
 * the printed FLOP-model numbers of Sec. 3, numpy's Cholesky, planted-coefficient
 * recovery.  No function here is "parity unpinned".
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SVKO_OK 0
#define SVKO_ERR_ARG 1
#define SVKO_ERR_NOT_SPD 3
#define SVKO_NORM_NONE 0
#define SVKO_NORM_ALARD 1

/* ---- threads (OpenMP over output rows only; the per-pixel arithmetic is unchanged) */
void svko_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int svko_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- small helpers ------------------------------------------------------------- */
static double ipow(double x, int n) {
    double r = 1.0;
    for (int i = 0; i < n; ++i) r *= x;
    return r;
}

/* Number of monomials of total degree <= d (Eq. 3 generalised to order d). */
int svko_n_terms(int d) { return d < 0 ? 0 : (d + 1) * (d + 2) / 2; }

/* Normalised polynomial coordinate of integer pixel index x in a frame of size W. */
double svko_norm_coord(int x, int W) {
    return W > 1 ? (2.0 * (double)x - (double)(W - 1)) / (double)(W - 1) : 0.0;
}

/* Monomials m_t(xt, yt), t over (i, j), i + j <= d, i (power of xt) outer. */
void svko_monomials(double xt, double yt, int d, double *m) {
    int t = 0;
    for (int i = 0; i <= d; ++i)
        for (int j = 0; j <= d - i; ++j) m[t++] = ipow(xt, i) * ipow(yt, j);
}

/* ---- basis stamps (Sec. 2: Gaussian function basis and Dirac delta basis) -------- */

int svko_gauss_basis_count(int n_gauss, const int *deg) {
    int n = 0;
    for (int g = 0; g < n_gauss; ++g) n += svko_n_terms(deg[g]);
    return n;
}

/*
 * Gaussian function basis (GFB, Alard & Lupton): for each Gaussian g and each
 * (p, q) with p + q <= deg[g] (p outer), B(u,v) = exp(-(u^2+v^2)/(2 sigma_g^2)) u^p v^q.
 * normalize == ALARD: B_0 scaled to unit sum; every other stamp with even p and even q
 * has (its sum) * B_0 subtracted so that it sums to zero (odd ones already do by
 * symmetry); then every stamp k >= 1 is scaled to unit L2 norm.  Returns N or -1.
 */
int svko_gauss_basis(int L, int n_gauss, const double *sigma, const int *deg, int normalize,
                     double *out) {
    if (L < 1 || (L % 2) == 0 || n_gauss < 1) return -1;
    const int h = (L - 1) / 2, LL = L * L;
    int N = svko_gauss_basis_count(n_gauss, deg);
    int *pp = (int *)malloc(sizeof(int) * N), *qq = (int *)malloc(sizeof(int) * N);
    int k = 0;
    for (int g = 0; g < n_gauss; ++g) {
        const double s2 = 2.0 * sigma[g] * sigma[g];
        for (int p = 0; p <= deg[g]; ++p)
            for (int q = 0; q <= deg[g] - p; ++q) {
                for (int v = -h; v <= h; ++v)
                    for (int u = -h; u <= h; ++u)
                        out[(size_t)k * LL + (v + h) * L + (u + h)] =
                            exp(-((double)(u * u + v * v)) / s2) * ipow(u, p) * ipow(v, q);
                pp[k] = p;
                qq[k] = q;
                ++k;
            }
    }
    if (normalize == SVKO_NORM_ALARD) {
        double *b0 = out;
        double s0 = 0.0;
        for (int i = 0; i < LL; ++i) s0 += b0[i];
        for (int i = 0; i < LL; ++i) b0[i] /= s0;
        for (k = 1; k < N; ++k) {
            double *bk = out + (size_t)k * LL;
            if ((pp[k] % 2) == 0 && (qq[k] % 2) == 0) {
                double sk = 0.0;
                for (int i = 0; i < LL; ++i) sk += bk[i];
                for (int i = 0; i < LL; ++i) bk[i] -= sk * b0[i];
            }
            double n2 = 0.0;
            for (int i = 0; i < LL; ++i) n2 += bk[i] * bk[i];
            const double nrm = sqrt(n2);
            if (nrm > 0.0)
                for (int i = 0; i < LL; ++i) bk[i] /= nrm;
        }
    }
    free(pp);
    free(qq);
    return N;
}

/*
 * Dirac delta function basis (DFB, Miller et al.): one stamp per kernel pixel,
 * B_k = delta at tap k (k = (v+h)*L + (u+h)).  normalize == ALARD: every stamp other
 * than the centre tap becomes delta_k - delta_centre (zero sum).  Returns N = L*L.
 */
int svko_delta_basis(int L, int normalize, double *out) {
    if (L < 1 || (L % 2) == 0) return -1;
    const int LL = L * L, c = (LL - 1) / 2;
    memset(out, 0, sizeof(double) * (size_t)LL * LL);
    for (int k = 0; k < LL; ++k) {
        out[(size_t)k * LL + k] = 1.0;
        if (normalize == SVKO_NORM_ALARD && k != c) out[(size_t)k * LL + c] = -1.0;
    }
    return LL;
}

/* ---- the spatially-varying convolution (Eq. 1-3) --------------------------------- */

/* One output pixel: kernel of Eq. 2 formed at (x, y), then a zero-padded convolution. */
static double conv_pixel(const double *R, int W, int H, const double *basis, int N, int L,
                         const double *coeffs, int degree, int x, int y, double *a, double *K) {
    const int T = svko_n_terms(degree), h = (L - 1) / 2, LL = L * L;
    double m[64];
    svko_monomials(svko_norm_coord(x, W), svko_norm_coord(y, H), degree, m);
    for (int k = 0; k < N; ++k) {
        double s = 0.0;
        for (int t = 0; t < T; ++t) s += coeffs[(size_t)k * T + t] * m[t];
        a[k] = s; /* a_k(x, y), Eq. 3 */
    }
    for (int i = 0; i < LL; ++i) {
        double s = 0.0;
        for (int k = 0; k < N; ++k) s += a[k] * basis[(size_t)k * LL + i];
        K[i] = s; /* K_{x,y}(u, v), Eq. 2 */
    }
    double acc = 0.0;
    for (int v = -h; v <= h; ++v) {
        const int yy = y - v;
        if (yy < 0 || yy >= H) continue;
        for (int u = -h; u <= h; ++u) {
            const int xx = x - u;
            if (xx < 0 || xx >= W) continue;
            acc += K[(v + h) * L + (u + h)] * R[(size_t)yy * W + xx];
        }
    }
    return acc;
}

/* Rows [y0, y1) of R (x) K_{x,y}; out holds (y1 - y0) * W values. */
int svko_convolve_rows(const double *R, int W, int H, const double *basis, int N, int L,
                       const double *coeffs, int degree, int y0, int y1, double *out) {
    if (W < 1 || H < 1 || N < 1 || L < 1 || (L % 2) == 0 || degree < 0 || degree > 7) return SVKO_ERR_ARG;
    if (y0 < 0 || y1 > H || y0 > y1) return SVKO_ERR_ARG;
#pragma omp parallel
    {
        double *a = (double *)malloc(sizeof(double) * N);
        double *K = (double *)malloc(sizeof(double) * L * L);
#pragma omp for schedule(dynamic, 1)
        for (int y = y0; y < y1; ++y)
            for (int x = 0; x < W; ++x)
                out[(size_t)(y - y0) * W + x] =
                    conv_pixel(R, W, H, basis, N, L, coeffs, degree, x, y, a, K);
        free(a);
        free(K);
    }
    return SVKO_OK;
}

int svko_convolve(const double *R, int W, int H, const double *basis, int N, int L,
                  const double *coeffs, int degree, double *out) {
    return svko_convolve_rows(R, W, H, basis, N, L, coeffs, degree, 0, H, out);
}

/* Selected output pixels (px[i], py[i]) of R (x) K_{x,y}. */
int svko_convolve_points(const double *R, int W, int H, const double *basis, int N, int L,
                         const double *coeffs, int degree, const int *px, const int *py, int n,
                         double *out) {
    if (W < 1 || H < 1 || N < 1 || L < 1 || (L % 2) == 0 || degree < 0 || degree > 7) return SVKO_ERR_ARG;
#pragma omp parallel
    {
        double *a = (double *)malloc(sizeof(double) * N);
        double *K = (double *)malloc(sizeof(double) * L * L);
#pragma omp for schedule(dynamic, 64)
        for (int i = 0; i < n; ++i)
            out[i] = conv_pixel(R, W, H, basis, N, L, coeffs, degree, px[i], py[i], a, K);
        free(a);
        free(K);
    }
    return SVKO_OK;
}

/* Difference image of Eq. 1: D = (R (x) K) - I. */
int svko_difference(const double *R, const double *I, int W, int H, const double *basis, int N,
                    int L, const double *coeffs, int degree, double *D) {
    int st = svko_convolve(R, W, H, basis, N, L, coeffs, degree, D);
    if (st != SVKO_OK) return st;
    for (size_t i = 0; i < (size_t)W * H; ++i) D[i] -= I[i];
    return SVKO_OK;
}

/* ---- Optimal Image Subtraction least-squares fit (Sec. 2) ------------------------
 * Unknowns: c[k][t] (index k*T + t) followed by n_bg background-polynomial terms.
 * Model at a stamp pixel: sum_k sum_t c[k][t] m_t(xt,yt) C_k(x,y) + sum_j g_j m_j(xt,yt),
 * with C_k = R (x) B_k (plain convolution with stamp k, zero padding).  Minimise
 * sum over stamp pixels of w * (model - I)^2 through the normal equations A c = b,
 * A = sum w v v^T, b = sum w v I, solved by a textbook Cholesky factorisation.
 */

/* In-place Cholesky A = G G^T of an M x M row-major SPD matrix (lower triangle holds G).
 * Returns -1 on success, else the index of the first non-positive pivot. */
int svko_cholesky(double *A, int M) {
    for (int j = 0; j < M; ++j) {
        double d = A[(size_t)j * M + j];
        for (int k = 0; k < j; ++k) d -= A[(size_t)j * M + k] * A[(size_t)j * M + k];
        if (!(d > 0.0)) return j;
        const double gjj = sqrt(d);
        A[(size_t)j * M + j] = gjj;
        for (int i = j + 1; i < M; ++i) {
            double s = A[(size_t)i * M + j];
            for (int k = 0; k < j; ++k) s -= A[(size_t)i * M + k] * A[(size_t)j * M + k];
            A[(size_t)i * M + j] = s / gjj;
        }
    }
    return -1;
}

/* Solve G G^T x = b given the factor from svko_cholesky (x may alias b). */
void svko_cholesky_solve(const double *G, int M, const double *b, double *x) {
    for (int i = 0; i < M; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= G[(size_t)i * M + k] * x[k];
        x[i] = s / G[(size_t)i * M + i];
    }
    for (int i = M - 1; i >= 0; --i) {
        double s = x[i];
        for (int k = i + 1; k < M; ++k) s -= G[(size_t)k * M + i] * x[k];
        x[i] = s / G[(size_t)i * M + i];
    }
}

static double conv_basis_pixel(const double *R, int W, int H, const double *bk, int L, int x, int y) {
    const int h = (L - 1) / 2;
    double acc = 0.0;
    for (int v = -h; v <= h; ++v) {
        const int yy = y - v;
        if (yy < 0 || yy >= H) continue;
        for (int u = -h; u <= h; ++u) {
            const int xx = x - u;
            if (xx < 0 || xx >= W) continue;
            acc += bk[(v + h) * L + (u + h)] * R[(size_t)yy * W + xx];
        }
    }
    return acc;
}

/* Design-vector of one stamp pixel. */
static void design_vector(const double *R, int W, int H, const double *basis, int N, int L,
                          int degree, int bg_degree, int x, int y, double *v) {
    const int T = svko_n_terms(degree), nb = svko_n_terms(bg_degree), LL = L * L;
    double m[64], mb[64];
    const double xt = svko_norm_coord(x, W), yt = svko_norm_coord(y, H);
    svko_monomials(xt, yt, degree, m);
    if (nb > 0) svko_monomials(xt, yt, bg_degree, mb);
    for (int k = 0; k < N; ++k) {
        const double ck = conv_basis_pixel(R, W, H, basis + (size_t)k * LL, L, x, y);
        for (int t = 0; t < T; ++t) v[k * T + t] = m[t] * ck;
    }
    for (int j = 0; j < nb; ++j) v[N * T + j] = mb[j];
}

/* Accumulate the normal equations over all stamp pixels.  Stamps are S x S (S odd)
 * centred on stamp_xy[2s], stamp_xy[2s+1]; pixels outside the frame are skipped.
 * A = sum_p w v v^T and b = sum_p w v I over the stamp pixels p in order (stamp by stamp,
 * rows then columns).  OpenMP only splits the work: a stamp's design vectors are formed
 * pixel by pixel in parallel, then each thread owns whole rows of A and adds the pixels'
 * contributions to them in that same pixel order, so every element is the same sum in
 * the same order as a single-threaded loop. */
int svko_normal_equations(const double *R, const double *I, int W, int H, const int *stamp_xy,
                          int n_stamps, int S, const double *basis, int N, int L, int degree,
                          int bg_degree, const double *weight, double *A, double *b) {
    if (S < 1 || (S % 2) == 0 || N < 1 || L < 1 || (L % 2) == 0 || degree < 0 || degree > 7 ||
        bg_degree < -1 || bg_degree > 7)
        return SVKO_ERR_ARG;
    const int T = svko_n_terms(degree), M = N * T + svko_n_terms(bg_degree), hs = (S - 1) / 2;
    const int P = S * S;
    memset(A, 0, sizeof(double) * (size_t)M * M);
    memset(b, 0, sizeof(double) * (size_t)M);
    double *V = (double *)malloc(sizeof(double) * (size_t)P * M);
    double *wp = (double *)malloc(sizeof(double) * P);
    double *ip = (double *)malloc(sizeof(double) * P);
    int *valid = (int *)malloc(sizeof(int) * P);
    for (int s = 0; s < n_stamps; ++s) {
        const int cx = stamp_xy[2 * s], cy = stamp_xy[2 * s + 1];
#pragma omp parallel for schedule(static)
        for (int p = 0; p < P; ++p) {
            const int y = cy - hs + p / S, x = cx - hs + p % S;
            valid[p] = (y >= 0 && y < H && x >= 0 && x < W);
            if (!valid[p]) continue;
            design_vector(R, W, H, basis, N, L, degree, bg_degree, x, y, V + (size_t)p * M);
            wp[p] = weight ? weight[(size_t)y * W + x] : 1.0;
            ip[p] = I[(size_t)y * W + x];
        }
#pragma omp parallel for schedule(static)
        for (int i = 0; i < M; ++i) {
            double *Ai = A + (size_t)i * M;
            for (int p = 0; p < P; ++p) {
                if (!valid[p]) continue;
                const double *v = V + (size_t)p * M;
                const double wvi = wp[p] * v[i];
                b[i] += wvi * ip[p];
                for (int j = 0; j < M; ++j) Ai[j] += wvi * v[j];
            }
        }
    }
    free(V);
    free(wp);
    free(ip);
    free(valid);
    return SVKO_OK;
}

/* chi^2 = sum over stamp pixels of w * (model(c) - I)^2. */
double svko_chi2(const double *R, const double *I, int W, int H, const int *stamp_xy, int n_stamps,
                 int S, const double *basis, int N, int L, int degree, int bg_degree,
                 const double *weight, const double *c) {
    const int T = svko_n_terms(degree), M = N * T + svko_n_terms(bg_degree), hs = (S - 1) / 2;
    double *v = (double *)malloc(sizeof(double) * M);
    double chi2 = 0.0;
    for (int s = 0; s < n_stamps; ++s) {
        const int cx = stamp_xy[2 * s], cy = stamp_xy[2 * s + 1];
        for (int y = cy - hs; y <= cy + hs; ++y) {
            if (y < 0 || y >= H) continue;
            for (int x = cx - hs; x <= cx + hs; ++x) {
                if (x < 0 || x >= W) continue;
                design_vector(R, W, H, basis, N, L, degree, bg_degree, x, y, v);
                double r = -I[(size_t)y * W + x];
                for (int i = 0; i < M; ++i) r += v[i] * c[i];
                chi2 += (weight ? weight[(size_t)y * W + x] : 1.0) * r * r;
            }
        }
    }
    free(v);
    return chi2;
}

/* Full fit: normal equations, Cholesky, solve, chi^2.  A_out / b_out (nullable) receive
 * the normal equations before factorisation.  *info = -1 on success, else the failing
 * pivot (status SVKO_ERR_NOT_SPD). */
int svko_fit(const double *R, const double *I, int W, int H, const int *stamp_xy, int n_stamps,
             int S, const double *basis, int N, int L, int degree, int bg_degree,
             const double *weight, double *coeffs_out, double *chi2_out, double *A_out,
             double *b_out, int *info) {
    const int M = N * svko_n_terms(degree) + svko_n_terms(bg_degree);
    double *A = (double *)malloc(sizeof(double) * (size_t)M * M);
    double *b = (double *)malloc(sizeof(double) * M);
    int st = svko_normal_equations(R, I, W, H, stamp_xy, n_stamps, S, basis, N, L, degree,
                                   bg_degree, weight, A, b);
    if (st != SVKO_OK) {
        free(A);
        free(b);
        return st;
    }
    if (A_out) memcpy(A_out, A, sizeof(double) * (size_t)M * M);
    if (b_out) memcpy(b_out, b, sizeof(double) * M);
    const int piv = svko_cholesky(A, M);
    if (info) *info = piv;
    if (piv >= 0) {
        free(A);
        free(b);
        return SVKO_ERR_NOT_SPD;
    }
    svko_cholesky_solve(A, M, b, coeffs_out);
    if (chi2_out)
        *chi2_out = svko_chi2(R, I, W, H, stamp_xy, n_stamps, S, basis, N, L, degree, bg_degree,
                              weight, coeffs_out);
    free(A);
    free(b);
    return SVKO_OK;
}

/* ---- cost models of Sec. 3 ------------------------------------------------------- */
/* Delta basis, including the final subtraction: 20 L^2 + 1 FLOP per pixel. */
double svko_flops_dfb_per_pixel(int L) { return 20.0 * L * L + 1.0; }
/* Gaussian basis with N functions: N L^2 + 2 L^2 + 18 N + 1 FLOP per pixel. */
double svko_flops_gfb_per_pixel(int N, int L) {
    return (double)N * L * L + 2.0 * L * L + 18.0 * N + 1.0;
}
