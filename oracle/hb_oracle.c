/*
 * hb_oracle.c -- plain FP64 CPU reference of the haemoglobin estimator of
 * "Fast Estimation of Haemoglobin Concentration in Tissue Via Wavelet
 * Decomposition" (Jones et al.).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load this file.  It shares no code,
 * header, table or constant with the CUDA library; it depends on libc/libm
 * (and pthreads for the row split of the posterior loop) only.
 *
 * Every step is written the slow, literal way, in the paper's order:
 *   1. log-attenuation  y = -ln(max(I, eps))              (Section 2, Eq. 8's -log)
 *   2. edge-replicated padding to a multiple of 2^n       (the paper is silent; reading)
 *   3. n levels of the 2x2 window Haar transform           (Eq. 1-2, Section 2)
 *   4. Tikhonov operator M = (A^T A + gamma I)^-1 A^T on every directional coefficient
 *                                                          (Eq. 5; "only ... on the sparse
 *                                                           directional components")
 *   5. Bayesian posterior mean over a discretised (HbO2, Hb) grid on the low-pass band
 *      (Section 2, Bayesian estimation on the low-pass coefficients, Eq. 8-11: Gaussian
 *       likelihood on -log of the low-pass data, flat prior, posterior mean)
 *   6. n levels of the inverse transform, H being its own inverse (Eq. 4: H = H*)
 *   7. THb = HbO2 + Hb, SO2 = HbO2 / THb                  (Section 3, Fig. 1-2)
 *
 * Readings of silent or garbled passages (listed again in the design notes):
 *   - the transform is applied to log-attenuation, so that y = A c is linear;
 *   - window order (x,y),(x,y+1),(x+1,y),(x+1,y+1) with x = row, y = column (Eq. 1);
 *   - the low-pass coefficient after n levels is 2^n times the block mean; the
 *     likelihood compares ybar = LL / 2^n with A c and the estimate is scaled back by 2^n;
 *   - gamma = lambda * trace(A^T A) / 2 ("relative") unless absolute is requested;
 *   - SO2 := 0 where THb <= 0.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define HBO_FMT_F32 0
#define HBO_FMT_U8 1

/* ---------------------------------------------------------------- step 1 */
/* Log-attenuation of every pixel and channel (the -log of Eq. 8 applied to RGB
 * intensities).  u8 codes k stand for the intensity k / 255.  Intensities
 * below eps are clamped to eps.  y is H*W*3, row-major, channel fastest. */
void hbo_log_atten(const void *frame, int fmt, int H, int W, long row_stride_bytes, double eps,
                   double *y) {
    for (int r = 0; r < H; ++r) {
        const unsigned char *row = (const unsigned char *)frame + (long)r * row_stride_bytes;
        for (int c = 0; c < W; ++c) {
            for (int ch = 0; ch < 3; ++ch) {
                double I;
                if (fmt == HBO_FMT_U8)
                    I = (double)row[c * 3 + ch] / 255.0;
                else
                    I = (double)((const float *)row)[c * 3 + ch];
                if (I < eps) I = eps;
                y[((long)r * W + c) * 3 + ch] = -log(I);
            }
        }
    }
}

/* The floored intensities max(I, eps) themselves (for the intensity-domain low pass of
 * Eq. 3-8, where the transform is applied to I and the logarithm taken after it). */
void hbo_intensity(const void *frame, int fmt, int H, int W, long row_stride_bytes, double eps, double *out) {
    for (int r = 0; r < H; ++r) {
        const unsigned char *row = (const unsigned char *)frame + (long)r * row_stride_bytes;
        for (int c = 0; c < W; ++c)
            for (int ch = 0; ch < 3; ++ch) {
                double I = fmt == HBO_FMT_U8 ? (double)row[c * 3 + ch] / 255.0 : (double)((const float *)row)[c * 3 + ch];
                out[((long)r * W + c) * 3 + ch] = I < eps ? eps : I;
            }
    }
}

/* ---------------------------------------------------------------- step 2 */
/* Edge replication: pixel (r, c) of the padded image is pixel
 * (min(r, H-1), min(c, W-1)) of the input. */
void hbo_pad_edge(const double *in, int H, int W, int C, int Hp, int Wp, double *out) {
    for (int r = 0; r < Hp; ++r)
        for (int c = 0; c < Wp; ++c) {
            int rs = r < H ? r : H - 1, cs = c < W ? c : W - 1;
            for (int ch = 0; ch < C; ++ch) out[((long)r * Wp + c) * C + ch] = in[((long)rs * W + cs) * C + ch];
        }
}

/* ---------------------------------------------------------------- step 3 */
/* The 4x4 Haar matrix of Eq. 2 (0.5 times a +-1 pattern). */
static const double HAAR[4][4] = {
    {0.5, 0.5, 0.5, 0.5},
    {0.5, 0.5, -0.5, -0.5},
    {0.5, -0.5, -0.5, 0.5},
    {0.5, -0.5, 0.5, -0.5},
};

/* One level of the window transform of Eq. 1: for every non-overlapping 2x2
 * window I = {I(x,y), I(x,y+1), I(x+1,y), I(x+1,y+1)} the four coefficients
 * are I * H.  Band b of window (x/2, y/2) receives coefficient b: band 0 is
 * the low pass (Section 2, H_LP = 0.5 [1 1 1 1]), bands 1..3 the three
 * directional components.  in is h*w*C (h, w even); each band is (h/2)*(w/2)*C. */
void hbo_haar_level(const double *in, int h, int w, int C, double *ll, double *d1, double *d2, double *d3) {
    double *bands[4] = {ll, d1, d2, d3};
    int h2 = h / 2, w2 = w / 2;
    for (int r = 0; r < h2; ++r)
        for (int c = 0; c < w2; ++c)
            for (int ch = 0; ch < C; ++ch) {
                double win[4];
                win[0] = in[((long)(2 * r) * w + 2 * c) * C + ch];
                win[1] = in[((long)(2 * r) * w + 2 * c + 1) * C + ch];
                win[2] = in[((long)(2 * r + 1) * w + 2 * c) * C + ch];
                win[3] = in[((long)(2 * r + 1) * w + 2 * c + 1) * C + ch];
                for (int b = 0; b < 4; ++b) {
                    double s = 0.0;
                    for (int i = 0; i < 4; ++i) s += win[i] * HAAR[i][b]; /* row vector times H */
                    bands[b][((long)r * w2 + c) * C + ch] = s;
                }
            }
}

/* ---------------------------------------------------------------- step 6 */
/* Inverse of one level.  The paper uses H = H* (Eq. 4): H is symmetric and
 * orthonormal, so the window is recovered as coefficients * H. */
void hbo_haar_level_inv(const double *ll, const double *d1, const double *d2, const double *d3, int h2, int w2,
                        int C, double *out) {
    const double *bands[4] = {ll, d1, d2, d3};
    int w = 2 * w2;
    for (int r = 0; r < h2; ++r)
        for (int c = 0; c < w2; ++c)
            for (int ch = 0; ch < C; ++ch) {
                double coef[4], win[4];
                for (int b = 0; b < 4; ++b) coef[b] = bands[b][((long)r * w2 + c) * C + ch];
                for (int i = 0; i < 4; ++i) {
                    double s = 0.0;
                    for (int b = 0; b < 4; ++b) s += coef[b] * HAAR[b][i];
                    win[i] = s;
                }
                out[((long)(2 * r) * w + 2 * c) * C + ch] = win[0];
                out[((long)(2 * r) * w + 2 * c + 1) * C + ch] = win[1];
                out[((long)(2 * r + 1) * w + 2 * c) * C + ch] = win[2];
                out[((long)(2 * r + 1) * w + 2 * c + 1) * C + ch] = win[3];
            }
}

/* ---------------------------------------------------------------- step 4 */
/* Tikhonov operator of Eq. 5 for the 3x2 mixing matrix A (row c = R,G,B,
 * column j = HbO2, Hb; A[c*2+j]):  M = (A^T A + gamma I)^-1 A^T, 2x3, M[j*3+c].
 * Gamma is "the identity matrix multiplied by a small constant": gamma =
 * lambda if absolute, else lambda * trace(A^T A) / 2.  Returns gamma. */
double hbo_tikhonov_operator(const double *A, double lambda, int relative, double *M) {
    double G[2][2];
    for (int j = 0; j < 2; ++j)
        for (int k = 0; k < 2; ++k) {
            double s = 0.0;
            for (int c = 0; c < 3; ++c) s += A[c * 2 + j] * A[c * 2 + k];
            G[j][k] = s;
        }
    double gamma = relative ? lambda * (G[0][0] + G[1][1]) / 2.0 : lambda;
    G[0][0] += gamma;
    G[1][1] += gamma;
    double det = G[0][0] * G[1][1] - G[0][1] * G[1][0];
    double Gi[2][2] = {{G[1][1] / det, -G[0][1] / det}, {-G[1][0] / det, G[0][0] / det}};
    for (int j = 0; j < 2; ++j)
        for (int c = 0; c < 3; ++c) M[j * 3 + c] = Gi[j][0] * A[c * 2 + 0] + Gi[j][1] * A[c * 2 + 1];
    return gamma;
}

/* The same operator with the constant column of Eq. 8 ("a constant term ... to account
 * for global illumination changes"): xi = [A | 1] (3x3), M3 = (xi^T xi + gamma I)^-1 xi^T,
 * and M = its HbO2 and Hb rows (the constant's row is dropped).  Gamma follows the same
 * rule as above, from A alone.  The 3x3 inverse is the adjugate over the determinant.
 * Returns gamma. */
double hbo_tikhonov_operator_illum(const double *A, double lambda, int relative, double *M) {
    double xi[3][3];
    for (int c = 0; c < 3; ++c) {
        xi[c][0] = A[c * 2 + 0];
        xi[c][1] = A[c * 2 + 1];
        xi[c][2] = 1.0;
    }
    double R[3][3];
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) {
            double s = 0.0;
            for (int c = 0; c < 3; ++c) s += xi[c][j] * xi[c][k];
            R[j][k] = s;
        }
    double gamma = relative ? lambda * (R[0][0] + R[1][1]) / 2.0 : lambda;
    for (int j = 0; j < 3; ++j) R[j][j] += gamma;
    double adj[3][3];
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) {
            /* cofactor of R[k][j] (transposed into the adjugate) */
            int r0 = (k + 1) % 3, r1 = (k + 2) % 3, c0 = (j + 1) % 3, c1 = (j + 2) % 3;
            adj[j][k] = R[r0][c0] * R[r1][c1] - R[r0][c1] * R[r1][c0];
        }
    double det = R[0][0] * adj[0][0] + R[0][1] * adj[1][0] + R[0][2] * adj[2][0];
    for (int j = 0; j < 2; ++j)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += adj[j][k] * xi[c][k];
            M[j * 3 + c] = s / det;
        }
    return gamma;
}

/* ---------------------------------------------------------------- step 5 */
/* Posterior mean of c = (HbO2, Hb) over the inclusive grid
 *   c_ij = (lo0 + i (hi0-lo0)/(n0-1), lo1 + j (hi1-lo1)/(n1-1)),
 * flat prior, Gaussian likelihood  L_ij = -|ybar - A c_ij|^2 / (2 sigma^2)
 * evaluated as the direct residual.  Weights exp(L_ij - max L).
 * illum: the model carries the constant term of Eq. 8, ybar = A c + kappa (1,1,1), with a
 * flat prior on kappa.  For each node the best kappa is the mean of the residual, and
 * integrating kappa out leaves the likelihood of the residual minus its mean (up to a
 * factor that is the same for every node), which is what is evaluated. */
static double grid_node(int i, int n, double lo, double hi) { return n > 1 ? lo + (hi - lo) * (double)i / (double)(n - 1) : lo; }

static double residual2(const double *ybar, const double *A, double c0, double c1, int illum) {
    double r[3], m = 0.0, r2 = 0.0;
    for (int ch = 0; ch < 3; ++ch) {
        r[ch] = ybar[ch] - A[ch * 2 + 0] * c0 - A[ch * 2 + 1] * c1;
        m += r[ch] / 3.0;
    }
    for (int ch = 0; ch < 3; ++ch) {
        double e = illum ? r[ch] - m : r[ch];
        r2 += e * e;
    }
    return r2;
}

void hbo_posterior_mean(const double *ybar, const double *A, int n0, int n1, double lo0, double hi0, double lo1,
                        double hi1, double sigma, int illum, double *out) {
    double Lmax = -INFINITY;
    for (int i = 0; i < n0; ++i)
        for (int j = 0; j < n1; ++j) {
            double c0 = grid_node(i, n0, lo0, hi0), c1 = grid_node(j, n1, lo1, hi1);
            double r2 = residual2(ybar, A, c0, c1, illum);
            double L = -r2 / (2.0 * sigma * sigma);
            if (L > Lmax) Lmax = L;
        }
    double sw = 0.0, s0 = 0.0, s1 = 0.0;
    for (int i = 0; i < n0; ++i)
        for (int j = 0; j < n1; ++j) {
            double c0 = grid_node(i, n0, lo0, hi0), c1 = grid_node(j, n1, lo1, hi1);
            double r2 = residual2(ybar, A, c0, c1, illum);
            double w = exp(-r2 / (2.0 * sigma * sigma) - Lmax);
            sw += w;
            s0 += w * c0;
            s1 += w * c1;
        }
    out[0] = s0 / sw;
    out[1] = s1 / sw;
}

/* Posterior means of many pixels, split over threads by contiguous ranges. */
typedef struct {
    const double *ybar;
    const double *A;
    int n0, n1;
    double lo0, hi0, lo1, hi1, sigma;
    int illum;
    long begin, end;
    double *out;
} post_job;

static void *post_worker(void *arg) {
    post_job *j = (post_job *)arg;
    for (long p = j->begin; p < j->end; ++p)
        hbo_posterior_mean(j->ybar + 3 * p, j->A, j->n0, j->n1, j->lo0, j->hi0, j->lo1, j->hi1, j->sigma, j->illum,
                           j->out + 2 * p);
    return NULL;
}

void hbo_posterior_mean_many(const double *ybar, long npix, const double *A, int n0, int n1, double lo0,
                             double hi0, double lo1, double hi1, double sigma, int illum, int nthreads, double *out) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    post_job jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (post_job){ybar, A, n0, n1, lo0, hi0, lo1, hi1, sigma, illum,
                             npix * t / nthreads, npix * (t + 1) / nthreads, out};
    }
    if (nthreads == 1) {
        post_worker(&jobs[0]);
        return;
    }
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, post_worker, &jobs[t]);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* ---------------------------------------------------------------- whole estimator */
/* Runs steps 1..7 on one frame.  lowpass_mode 0 = Bayesian on the low pass
 * (the proposed method), 1 = Tikhonov on the low pass as well (the
 * all-Tikhonov comparison of Table 1).  illum = 1 adds the constant
 * (illumination) term of Eq. 8 to both the Tikhonov operator and the posterior.
 * ll_intensity = 1 takes the low pass of Eq. 3-8 literally: -log of the low pass of the
 * intensities (their block mean) instead of the low pass of -log I.
 * levels = 0 means no decomposition:
 * the Bayesian estimate on every pixel (the full-resolution comparison).
 * Outputs (each may be NULL): hbo2, hb, thb, so2 (H*W); ybar_ll ((Hp>>n)*(Wp>>n)*3,
 * the low-pass band divided by 2^n); conc_ll ((Hp>>n)*(Wp>>n)*2, concentration
 * low-pass coefficients 2^n * posterior mean).  Returns 0, or -1 on bad
 * arguments / allocation failure. */
int hbo_estimate(const void *frame, int fmt, int H, int W, long row_stride_bytes, const double *A, double lambda,
                 int lambda_relative, int n0, int n1, double lo0, double hi0, double lo1, double hi1,
                 double sigma, int levels, int lowpass_mode, int illum, int ll_intensity, int nthreads,
                 double *hbo2, double *hb, double *thb, double *so2, double *ybar_ll, double *conc_ll) {
    if (H <= 0 || W <= 0 || levels < 0 || levels > 6 || n0 < 1 || n1 < 1 || sigma <= 0) return -1;
    if (lowpass_mode < 0 || lowpass_mode > 2) return -1;
    if (levels == 0 && lowpass_mode == 1) return -1;
    if (ll_intensity && lowpass_mode == 1) return -1;
    const double eps = fmt == HBO_FMT_U8 ? 1.0 / 255.0 : 1e-6;
    const int blk = 1 << levels;
    const int Hp = (H + blk - 1) / blk * blk, Wp = (W + blk - 1) / blk * blk;
    const int hl = Hp >> levels, wl = Wp >> levels;
    double M[6];
    if (illum)
        hbo_tikhonov_operator_illum(A, lambda, lambda_relative, M);
    else
        hbo_tikhonov_operator(A, lambda, lambda_relative, M);

    double *y = malloc(sizeof(double) * (size_t)H * W * 3);
    double *yp = malloc(sizeof(double) * (size_t)Hp * Wp * 3);
    /* per level: the three directional bands, in concentrations (2 channels) */
    double *cdet[7][3] = {{0}};
    double *cur = NULL, *conc = NULL;
    int ok = y && yp;
    if (ok) {
        hbo_log_atten(frame, fmt, H, W, row_stride_bytes, eps, y);              /* step 1 */
        hbo_pad_edge(y, H, W, 3, Hp, Wp, yp);                                   /* step 2 */
    }
    /* step 3 + 4: analysis; every directional coefficient goes through M */
    cur = yp;
    int h = Hp, w = Wp;
    for (int l = 1; ok && l <= levels; ++l) {
        int h2 = h / 2, w2 = w / 2;
        size_t n = (size_t)h2 * w2;
        double *ll = malloc(sizeof(double) * n * 3), *d[3];
        ok = ll != NULL;
        for (int b = 0; b < 3; ++b) {
            d[b] = malloc(sizeof(double) * n * 3);
            cdet[l][b] = malloc(sizeof(double) * n * 2);
            ok = ok && d[b] && cdet[l][b];
        }
        if (ok) {
            hbo_haar_level(cur, h, w, 3, ll, d[0], d[1], d[2]);
            for (int b = 0; b < 3; ++b)
                for (size_t p = 0; p < n; ++p)
                    for (int j = 0; j < 2; ++j) {
                        double s = 0.0;
                        for (int c = 0; c < 3; ++c) s += M[j * 3 + c] * d[b][p * 3 + c];
                        cdet[l][b][p * 2 + j] = s;
                    }
        }
        for (int b = 0; b < 3; ++b) free(d[b]);
        if (cur != yp) free(cur);
        cur = ll;
        h = h2;
        w = w2;
    }
    /* step 5: the low-pass band (hl x wl x 3) */
    double *cll = ok ? malloc(sizeof(double) * (size_t)hl * wl * 2) : NULL;
    double *yb = ok ? malloc(sizeof(double) * (size_t)hl * wl * 3) : NULL;
    ok = ok && cll && yb;
    if (ok && ll_intensity) {
        /* Eq. 3-8 for the low pass: the n-level low pass of the (floored, padded)
         * intensities, then -log of it divided by 2^n, i.e. of the block mean. */
        double *ii = malloc(sizeof(double) * (size_t)H * W * 3), *ip = malloc(sizeof(double) * (size_t)Hp * Wp * 3);
        ok = ii && ip;
        if (ok) {
            hbo_intensity(frame, fmt, H, W, row_stride_bytes, eps, ii);
            hbo_pad_edge(ii, H, W, 3, Hp, Wp, ip);
            double *icur = ip;
            int ih = Hp, iw = Wp;
            for (int l = 1; ok && l <= levels; ++l) {
                size_t n = (size_t)(ih / 2) * (iw / 2) * 3;
                double *ll = malloc(sizeof(double) * n), *d1 = malloc(sizeof(double) * n),
                       *d2 = malloc(sizeof(double) * n), *d3 = malloc(sizeof(double) * n);
                ok = ll && d1 && d2 && d3;
                if (ok) hbo_haar_level(icur, ih, iw, 3, ll, d1, d2, d3);
                free(d1);
                free(d2);
                free(d3);
                if (icur != ip) free(icur);
                icur = ll;
                ih /= 2;
                iw /= 2;
            }
            if (ok)
                for (size_t p = 0; p < (size_t)hl * wl * 3; ++p) yb[p] = -log(icur[p] / (double)blk);
            if (icur != ip) free(icur);
        }
        free(ii);
        free(ip);
    }
    if (ok) {
        double scale = (double)blk; /* 2^n */
        if (!ll_intensity)
            for (size_t p = 0; p < (size_t)hl * wl * 3; ++p) yb[p] = cur[p] / scale;
        if (lowpass_mode == 0) {
            hbo_posterior_mean_many(yb, (long)hl * wl, A, n0, n1, lo0, hi0, lo1, hi1, sigma, illum, nthreads, cll);
        } else {
            /* 1: the Tikhonov operator M on the low pass too (Eq. 5 on every band);
             * 2: least squares on the low pass (the fit of Section 2's maximisation step,
             *    Eq. 9 read as the ordinary least-squares solution over xi = A, or [A | 1]
             *    with the illumination term): the same operator with no regularisation */
            double L[6];
            if (lowpass_mode == 2) {
                if (illum)
                    hbo_tikhonov_operator_illum(A, 0.0, 0, L);
                else
                    hbo_tikhonov_operator(A, 0.0, 0, L);
            }
            const double *Op = lowpass_mode == 2 ? L : M;
            for (size_t p = 0; p < (size_t)hl * wl; ++p)
                for (int j = 0; j < 2; ++j) {
                    double s = 0.0;
                    for (int c = 0; c < 3; ++c) s += Op[j * 3 + c] * yb[p * 3 + c];
                    cll[p * 2 + j] = s;
                }
        }
        for (size_t p = 0; p < (size_t)hl * wl * 2; ++p) cll[p] *= scale;
        if (ybar_ll) memcpy(ybar_ll, yb, sizeof(double) * (size_t)hl * wl * 3);
        if (conc_ll) memcpy(conc_ll, cll, sizeof(double) * (size_t)hl * wl * 2);
    }
    if (cur != yp) free(cur);
    /* step 6: synthesis, level n down to 1 */
    conc = cll;
    h = hl;
    w = wl;
    for (int l = levels; ok && l >= 1; --l) {
        double *up = malloc(sizeof(double) * (size_t)(2 * h) * (2 * w) * 2);
        ok = up != NULL;
        if (ok) hbo_haar_level_inv(conc, cdet[l][0], cdet[l][1], cdet[l][2], h, w, 2, up);
        if (conc != cll) free(conc);
        conc = up;
        h *= 2;
        w *= 2;
    }
    /* step 7: crop, THb and SO2 */
    if (ok) {
        for (int r = 0; r < H; ++r)
            for (int c = 0; c < W; ++c) {
                double a = conc[((size_t)r * Wp + c) * 2 + 0], b = conc[((size_t)r * Wp + c) * 2 + 1];
                size_t o = (size_t)r * W + c;
                if (hbo2) hbo2[o] = a;
                if (hb) hb[o] = b;
                if (thb) thb[o] = a + b;
                if (so2) so2[o] = (a + b) > 0.0 ? a / (a + b) : 0.0;
            }
    }
    if (conc && conc != cll) free(conc);
    free(cll);
    free(yb);
    for (int l = 0; l < 7; ++l)
        for (int b = 0; b < 3; ++b) free(cdet[l][b]);
    free(y);
    free(yp);
    return ok ? 0 : -1;
}
