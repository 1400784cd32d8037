/*
 * Plain, slow FP64 CPU oracle for the GMM superpixel method of
 * Ban, Liu and Cao, "Superpixel Segmentation Using Gaussian Mixture Model"
 * (arXiv 1612.08792).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker the CUDA path is
 * compared against.  Only the test-suite, the smoke check and the timed CPU
 * baseline of the benchmark may load it; the product library never does.
 * It shares no code, header, table or constant with the CUDA path.
 *
 * Every routine follows the paper's definitions in the order the paper
 * states them, in double precision, with no blocking, fusion or reordering:
 *   - pixel vector z_i = (x_i, y_i, L, a, b)               Sec. III-A
 *   - grid spacing and superpixel count                    Eq. (vxy), Eq. (nxyK)
 *   - pixel sets I_k and candidate sets K_i                Eq. (Ik), Eq. (kxy)
 *   - Gaussian density                                     Eq. (gaussian)
 *   - posteriors R_ik (E-step)                             Eq. (Rik)
 *   - log-likelihood L(theta)                              Eq. (ftheta) and the L that follows it
 *   - mean and block covariance update (M-step)            Eq. (UpdateMu), (UpdateSigS), (UpdateSigC)
 *   - eigenvalue floor and reconstruction                  Eq. (eigdecs)-(eigdecrc), (mlams), (mlamc)
 *   - initialisation                                       Sec. III-C, the paragraph after Eq. (eigdecrc)
 *   - labels by maximum posterior                          Eq. (obtLi)
 *   - the loop                                             Algorithm 1, steps 1-7
 * Three colour models (argument `cmodel`), Sec. III-A and III-C:
 *   0  full: Sigma_c a 3x3 over (L, a, b)                  Eq. (BlockSigma)
 *   1  split: Sigma_c = diag(sigma_l^2, Sigma_(a,b))       Eq. (BlockSigma1)
 *   2  grayscale: c_i a scalar, Sigma_c = sigma^2          Sec. III-A, III-C (Q_k,c = 1)
 * The connectivity post-processing (Algorithm 1, step 8) is not part of the
 * EM loop and is not implemented here.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - CIELAB: sRGB (IEC 61966-2-1) decoding, D65 white, CIE 1976 L*a*b*.
 *   - argmax ties go to the smaller superpixel index k.
 *   - a superpixel whose total responsibility is below 1e-8 keeps its
 *     previous parameters (the paper does not say what happens then).
 *   - the floor epsilon is applied to eigenvalues of the covariance
 *     (variance units).
 *   - grayscale: the scalar colour is the CIE L* of the pixel (the L
 *     channel of a colour input; for a grey-level input g, L* of the
 *     luminance Y = sRGB-decode(g / 255)), so that eps_c and lambda keep
 *     their CIELAB units.
 *   - the split model's M-step is the maximiser of Q over covariances of
 *     the form of Eq. (BlockSigma1): the variance of L and the 2x2 weighted
 *     covariance of (a, b), with no L-(a, b) cross terms; its floor acts on
 *     the eigenvalues of each block (together, the eigenvalues of Sigma_c).
 *
 * Threading: the E-step is parallel over pixels and the M-step over
 * superpixels, the two independent loops the paper's Sec. III-D names.
 * Every output is written by exactly one thread in a fixed order, so results
 * do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_D 5          /* dimension of z: x, y, L, a, b (x, y, L for grayscale) */
#define ORC_FULL 0
#define ORC_SPLIT 1
#define ORC_GRAY 2
#define ORC_MAXC 9       /* |K_i| <= 9, Sec. III-D */
#define ORC_DEAD_W 1e-8  /* reading: below this total weight theta_k is kept */

static const double ORC_PI = 3.14159265358979323846;

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------
 * CIELAB conversion (Sec. IV, first paragraph: the experiments use CIELAB).
 * The paper does not fix the white point or the RGB space; this oracle
 * reads the input as sRGB and uses the D65 white.  Written from the
 * definitions of the sRGB transfer curve, the sRGB-to-XYZ matrix for D65 and
 * the CIE 1976 L*a*b* formulas.
 * ---------------------------------------------------------------------- */
static double srgb_decode(double c)
{
    /* sRGB electro-optical transfer function, c in [0, 1]. */
    if (c <= 0.04045) return c / 12.92;
    return pow((c + 0.055) / 1.055, 2.4);
}

static double cielab_f(double t)
{
    /* CIE 1976: f(t) = t^(1/3) above (6/29)^3, a line below it. */
    const double delta = 6.0 / 29.0;
    if (t > delta * delta * delta) return cbrt(t);
    return t / (3.0 * delta * delta) + 4.0 / 29.0;
}

void orc_rgb2lab(const uint8_t *rgb, long n, double *lab)
{
    /* Linear sRGB -> XYZ for the D65 white point. */
    static const double M[3][3] = {
        {0.4124564, 0.3575761, 0.1804375},
        {0.2126729, 0.7151522, 0.0721750},
        {0.0193339, 0.1191920, 0.9503041},
    };
    const double Xn = 0.95047, Yn = 1.0, Zn = 1.08883;
    long i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) {
        double r = srgb_decode(rgb[3 * i + 0] / 255.0);
        double g = srgb_decode(rgb[3 * i + 1] / 255.0);
        double b = srgb_decode(rgb[3 * i + 2] / 255.0);
        double X = M[0][0] * r + M[0][1] * g + M[0][2] * b;
        double Y = M[1][0] * r + M[1][1] * g + M[1][2] * b;
        double Z = M[2][0] * r + M[2][1] * g + M[2][2] * b;
        double fx = cielab_f(X / Xn), fy = cielab_f(Y / Yn), fz = cielab_f(Z / Zn);
        lab[3 * i + 0] = 116.0 * fy - 16.0;
        lab[3 * i + 1] = 500.0 * (fx - fy);
        lab[3 * i + 2] = 200.0 * (fy - fz);
    }
}

/* Grey levels -> CIE L*: a grey pixel has R = G = B = g, whose luminance
 * relative to the white is Y / Yn = sRGB-decode(g / 255) (the three primaries
 * at equal drive add up to the white point). */
void orc_gray2l(const uint8_t *gray, long n, double *L)
{
    long i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) L[i] = 116.0 * cielab_f(srgb_decode(gray[i] / 255.0)) - 16.0;
}

/* ------------------------------------------------------------------------
 * Grid, Eq. (vxy) and Eq. (nxyK).
 *   v_x = v_y = floor(sqrt(W*H/K)) when K is given, else the given spacing;
 *   n_x = floor(W/v_x), n_y = floor(H/v_y), K = n_x * n_y.
 * The floor of the square root is taken in exact integer arithmetic.
 * out = {v, n_x, n_y, K}.  Returns 0, or -1 when the grid is empty.
 * ---------------------------------------------------------------------- */
int orc_grid(int W, int H, int K_req, int spacing, int *out)
{
    long long v;
    if (W < 1 || H < 1) return -1;
    if (spacing > 0) {
        v = spacing;
    } else {
        long long N = (long long)W * H;
        if (K_req < 1) return -1;
        v = (long long)floor(sqrt((double)N / (double)K_req));
        while ((v + 1) * (v + 1) * (long long)K_req <= N) ++v;  /* v = max{v : v^2 K <= N} */
        while (v > 0 && v * v * (long long)K_req > N) --v;
    }
    if (v < 1) return -1;
    out[0] = (int)v;
    out[1] = (int)(W / v);
    out[2] = (int)(H / v);
    out[3] = out[1] * out[2];
    if (out[1] < 1 || out[2] < 1) return -1;
    return 0;
}

/* ------------------------------------------------------------------------
 * Pixel sets, Eq. (Ik) with Eq. (kxy).  The window of superpixel k is
 *   x_{k,b} = max(0, v(k_x-1)) <= x < x_{k,e} = min(W, v(k_x+2)),
 *   y_{k,b} = max(0, v(k_y-1)) <= y < y_{k,e} = min(H, v(k_y+2)).
 * The condition is a product of a condition on x with one on k_x and a
 * condition on y with one on k_y, so K_i = {k_y n_x + k_x} over the k_x whose
 * x-window holds x_i and the k_y whose y-window holds y_i.  Both lists are
 * found by testing every k_x (every k_y) against the literal bounds.
 * ---------------------------------------------------------------------- */
static void window(int kq, int v, int extent, int *b, int *e)
{
    int lo = v * (kq - 1), hi = v * (kq + 2);
    *b = lo > 0 ? lo : 0;
    *e = hi < extent ? hi : extent;
}

/* lists[p*3 + j], counts[p] for every coordinate p in [0, extent). */
static int axis_lists(int extent, int v, int nq, int *lists, int *counts)
{
    int p, kq;
    for (p = 0; p < extent; ++p) {
        int c = 0;
        for (kq = 0; kq < nq; ++kq) {
            int b, e;
            window(kq, v, extent, &b, &e);
            if (b <= p && p < e) {
                if (c == 3) return -1; /* cannot happen: at most 3 windows overlap */
                lists[p * 3 + c++] = kq;
            }
        }
        counts[p] = c;
    }
    return 0;
}

/* Candidate sets for every pixel: cand[i*9 + j] in ascending k, ncand[i]. */
int orc_candidates(int W, int H, int v, int nx, int ny, int32_t *cand, int32_t *ncand)
{
    int *xl = malloc(sizeof(int) * 3 * W), *xc = malloc(sizeof(int) * W);
    int *yl = malloc(sizeof(int) * 3 * H), *yc = malloc(sizeof(int) * H);
    int x, y, rc = 0;
    if (!xl || !xc || !yl || !yc) { rc = -2; goto done; }
    if (axis_lists(W, v, nx, xl, xc) || axis_lists(H, v, ny, yl, yc)) { rc = -1; goto done; }
    for (y = 0; y < H; ++y)
        for (x = 0; x < W; ++x) {
            long i = (long)y * W + x;
            int jy, jx, c = 0;
            for (jy = 0; jy < yc[y]; ++jy)
                for (jx = 0; jx < xc[x]; ++jx)
                    cand[i * ORC_MAXC + c++] = yl[y * 3 + jy] * nx + xl[x * 3 + jx];
            ncand[i] = c;
        }
done:
    free(xl); free(xc); free(yl); free(yc);
    return rc;
}

/* ------------------------------------------------------------------------
 * Small dense linear algebra in plain loops.
 * Block covariance layout (Eq. BlockSigma):
 *   cs[3] = {S_xx, S_xy, S_yy}           spatial 2x2
 *   cc[6] = {C_LL, C_La, C_Lb, C_aa, C_ab, C_bb}   colour 3x3
 * ---------------------------------------------------------------------- */
static void sym_unpack(int n, const double *p, double A[3][3])
{
    if (n == 1) {
        A[0][0] = p[0];
    } else if (n == 2) {
        A[0][0] = p[0]; A[0][1] = A[1][0] = p[1]; A[1][1] = p[2];
    } else {
        A[0][0] = p[0]; A[0][1] = A[1][0] = p[1]; A[0][2] = A[2][0] = p[2];
        A[1][1] = p[3]; A[1][2] = A[2][1] = p[4]; A[2][2] = p[5];
    }
}

static void sym_pack(int n, double A[3][3], double *p)
{
    if (n == 1) {
        p[0] = A[0][0];
    } else if (n == 2) {
        p[0] = A[0][0]; p[1] = 0.5 * (A[0][1] + A[1][0]); p[2] = A[1][1];
    } else {
        p[0] = A[0][0]; p[1] = 0.5 * (A[0][1] + A[1][0]); p[2] = 0.5 * (A[0][2] + A[2][0]);
        p[3] = A[1][1]; p[4] = 0.5 * (A[1][2] + A[2][1]); p[5] = A[2][2];
    }
}

/* Cholesky factor of an SPD n x n matrix (n <= 3); returns -1 if not SPD. */
static int cholesky(int n, double A[3][3], double L[3][3])
{
    int i, j, k;
    memset(L, 0, sizeof(double) * 9);
    for (j = 0; j < n; ++j) {
        double s = A[j][j];
        for (k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
        if (!(s > 0.0)) return -1;
        L[j][j] = sqrt(s);
        for (i = j + 1; i < n; ++i) {
            double t = A[i][j];
            for (k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
            L[i][j] = t / L[j][j];
        }
    }
    return 0;
}

/* Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix (n <= 3),
 * Golub & Van Loan, "Matrix Computations", the symmetric Schur 2x2 rotation.
 * On return A's diagonal holds the eigenvalues and column j of Q the
 * eigenvector of eigenvalue j. */
static void jacobi_eigen(int n, double A[3][3], double Q[3][3])
{
    int sweep, p, q, r;
    for (p = 0; p < 3; ++p)
        for (q = 0; q < 3; ++q) Q[p][q] = (p == q) ? 1.0 : 0.0;
    for (sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, fro = 0.0;
        for (p = 0; p < n; ++p)
            for (q = 0; q < n; ++q) {
                fro += A[p][q] * A[p][q];
                if (p != q) off += A[p][q] * A[p][q];
            }
        if (off == 0.0 || off <= 1e-36 * fro) break;
        for (p = 0; p < n - 1; ++p)
            for (q = p + 1; q < n; ++q) {
                double apq = A[p][q], tau, t, c, s;
                if (apq == 0.0) continue;
                tau = (A[q][q] - A[p][p]) / (2.0 * apq);
                t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                c = 1.0 / sqrt(1.0 + t * t);
                s = t * c;
                /* A <- J^T A J with J the rotation in the (p, q) plane. */
                for (r = 0; r < n; ++r) {
                    double arp = A[r][p], arq = A[r][q];
                    A[r][p] = c * arp - s * arq;
                    A[r][q] = s * arp + c * arq;
                }
                for (r = 0; r < n; ++r) {
                    double apr = A[p][r], aqr = A[q][r];
                    A[p][r] = c * apr - s * aqr;
                    A[q][r] = s * apr + c * aqr;
                }
                for (r = 0; r < n; ++r) {
                    double qrp = Q[r][p], qrq = Q[r][q];
                    Q[r][p] = c * qrp - s * qrq;
                    Q[r][q] = s * qrp + c * qrq;
                }
            }
    }
}

/* Eigenvalue floor, Eq. (eigdecs)/(eigdecc), (mlams)/(mlamc), (eigdecrs)/(eigdecrc):
 * Sigma = Q Lambda Q^T, lambda~_j = lambda_j if lambda_j >= eps else eps,
 * Sigma~ = Q Lambda~ Q^T.  Returns the number of eigenvalues raised. */
int orc_eig_clamp(int n, const double *packed_in, double eps, double *packed_out)
{
    double A[3][3] = {{0}}, Q[3][3], lam[3], B[3][3] = {{0}};
    int i, j, m, raised = 0;
    sym_unpack(n, packed_in, A);
    jacobi_eigen(n, A, Q);
    for (j = 0; j < n; ++j) {
        lam[j] = A[j][j];
        if (!(lam[j] >= eps)) { lam[j] = eps; ++raised; }
    }
    for (i = 0; i < n; ++i)
        for (m = 0; m < n; ++m) {
            double s = 0.0;
            for (j = 0; j < n; ++j) s += Q[i][j] * lam[j] * Q[m][j];
            B[i][m] = s;
        }
    sym_pack(n, B, packed_out);
    return raised;
}

/* Eigenvalues only (ascending), for tests of the clamp. */
void orc_sym_eigvals(int n, const double *packed, double *lam)
{
    double A[3][3] = {{0}}, Q[3][3];
    int i, j;
    sym_unpack(n, packed, A);
    jacobi_eigen(n, A, Q);
    for (i = 0; i < n; ++i) lam[i] = A[i][i];
    for (i = 0; i < n; ++i)
        for (j = i + 1; j < n; ++j)
            if (lam[j] < lam[i]) { double t = lam[i]; lam[i] = lam[j]; lam[j] = t; }
}

/* ------------------------------------------------------------------------
 * Initialisation, Sec. III-C: mu_k = z_j at the centre pixel
 *   j = k_x v + floor(v/2) + W (k_y v + floor(v/2)),
 * Sigma_s = diag(v^2, v^2), Sigma_c = lambda^2 I (of the colour dimension).
 * lab is N x 3 (L, a, b); mu is K x 5 (x, y, L, a, b).  Grayscale: the
 * colour is L alone; mu's a, b and every Sigma_c entry but LL are 0.
 * ---------------------------------------------------------------------- */
void orc_init(const double *lab, int W, int H, int v, int nx, int ny, double lambda_c,
              double *mu, double *cs, double *cc, int cmodel)
{
    int k, K = nx * ny;
    (void)H;
    for (k = 0; k < K; ++k) {
        int kx = k % nx, ky = k / nx;
        int x = kx * v + v / 2, y = ky * v + v / 2;
        long j = (long)x + (long)W * y;
        mu[5 * k + 0] = x;
        mu[5 * k + 1] = y;
        mu[5 * k + 2] = lab[3 * j + 0];
        mu[5 * k + 3] = lab[3 * j + 1];
        mu[5 * k + 4] = lab[3 * j + 2];
        cs[3 * k + 0] = (double)v * v; cs[3 * k + 1] = 0.0; cs[3 * k + 2] = (double)v * v;
        cc[6 * k + 0] = lambda_c * lambda_c; cc[6 * k + 1] = 0.0; cc[6 * k + 2] = 0.0;
        cc[6 * k + 3] = lambda_c * lambda_c; cc[6 * k + 4] = 0.0; cc[6 * k + 5] = lambda_c * lambda_c;
        if (cmodel == ORC_GRAY) {
            mu[5 * k + 3] = mu[5 * k + 4] = 0.0;
            cc[6 * k + 3] = cc[6 * k + 5] = 0.0;
        }
    }
}

/* ------------------------------------------------------------------------
 * Log of the Gaussian density, Eq. (gaussian), D = 2 + (colour dimension),
 * with the block diagonal covariance of Eq. (BlockSigma):
 *   ln p = -(D/2) ln 2pi - (1/2) ln det Sigma - (1/2) d^T Sigma^{-1} d.
 * Sigma^{-1} d and ln det Sigma come from a Cholesky factor of each block.
 * The colour block is the full 3x3 (model 0), diag(sigma_l^2, Sigma_(a,b))
 * of Eq. (BlockSigma1) (model 1: the L-a and L-b entries are zero, whatever
 * cc holds there), or the 1x1 sigma^2 of a grayscale image (model 2).
 * ---------------------------------------------------------------------- */
typedef struct {
    double Ls[3][3], Lc[3][3];
    double logdet;
    int nc;   /* colour dimension */
    int ok;
} orc_chol;

static void orc_factor(const double *cs, const double *cc, int cmodel, orc_chol *f)
{
    double A[3][3] = {{0}}, B[3][3] = {{0}};
    int j;
    f->nc = (cmodel == ORC_GRAY) ? 1 : 3;
    sym_unpack(2, cs, A);
    sym_unpack(f->nc, cc, B);
    if (cmodel == ORC_SPLIT) B[0][1] = B[1][0] = B[0][2] = B[2][0] = 0.0;
    f->ok = (cholesky(2, A, f->Ls) == 0) && (cholesky(f->nc, B, f->Lc) == 0);
    f->logdet = 0.0;
    if (f->ok) {
        f->logdet = 2.0 * (log(f->Ls[0][0]) + log(f->Ls[1][1]));
        for (j = 0; j < f->nc; ++j) f->logdet += 2.0 * log(f->Lc[j][j]);
    }
}

static double quad_form(int n, const double (*L)[3], const double *d)
{
    /* d^T (L L^T)^{-1} d = |w|^2 with L w = d (forward substitution). */
    double w[3], s = 0.0;
    int i, k;
    for (i = 0; i < n; ++i) {
        double t = d[i];
        for (k = 0; k < i; ++k) t -= L[i][k] * w[k];
        w[i] = t / L[i][i];
        s += w[i] * w[i];
    }
    return s;
}

static double log_gauss(const double *z, const double *mu, const orc_chol *f)
{
    double ds[2] = {z[0] - mu[0], z[1] - mu[1]};
    double dc[3] = {z[2] - mu[2], z[3] - mu[3], z[4] - mu[4]};
    double q = quad_form(2, f->Ls, ds) + quad_form(f->nc, f->Lc, dc);
    return -0.5 * (2 + f->nc) * log(2.0 * ORC_PI) - 0.5 * f->logdet - 0.5 * q;
}

/* Log density of pixel z under theta_k, exposed for tests. */
double orc_log_gauss(const double *z, const double *mu, const double *cs, const double *cc, int cmodel)
{
    orc_chol f;
    orc_factor(cs, cc, cmodel, &f);
    if (!f.ok) return NAN;
    return log_gauss(z, mu, &f);
}

/* ------------------------------------------------------------------------
 * E-step, Eq. (Rik): R_ik = p(z_i; theta_k) / sum_{k' in K_i} p(z_i; theta_k'),
 * and L(theta) = sum_i ln sum_{k in K_i} p(z_i; theta_k) (the L defined after
 * Eq. ftheta).  The sum of exponentials is taken relative to the largest
 * term so that it neither overflows nor underflows.
 *   R[i*9 + j] is the posterior of cand[i*9 + j]; unused slots are 0.
 *   ll[i] (optional) is ln sum_k p(z_i; theta_k).
 * Returns L(theta), or NAN when a covariance is not positive definite.
 * ---------------------------------------------------------------------- */
double orc_estep(const double *lab, int W, int H, int K, const int32_t *cand, const int32_t *ncand,
                 const double *mu, const double *cs, const double *cc, double *R, double *ll, int cmodel)
{
    long N = (long)W * H, i;
    int k, bad = 0;
    double L = 0.0;
    orc_chol *F = malloc(sizeof(orc_chol) * (size_t)K);
    double *lli = malloc(sizeof(double) * (size_t)N);
    if (!F || !lli) { free(F); free(lli); return NAN; }
    for (k = 0; k < K; ++k) {
        orc_factor(cs + 3 * k, cc + 6 * k, cmodel, &F[k]);
        if (!F[k].ok) bad = 1;
    }
    if (bad) { free(F); free(lli); return NAN; }
#pragma omp parallel for schedule(static)
    for (i = 0; i < N; ++i) {
        double z[5], lg[ORC_MAXC], m = -INFINITY, s = 0.0;
        int j, n = ncand[i];
        z[0] = (double)(i % W);
        z[1] = (double)(i / W);
        z[2] = lab[3 * i + 0]; z[3] = lab[3 * i + 1]; z[4] = lab[3 * i + 2];
        for (j = 0; j < n; ++j) {
            int kk = cand[i * ORC_MAXC + j];
            lg[j] = log_gauss(z, mu + 5 * kk, &F[kk]);
            if (lg[j] > m) m = lg[j];
        }
        for (j = 0; j < n; ++j) s += exp(lg[j] - m);
        for (j = 0; j < ORC_MAXC; ++j) R[i * ORC_MAXC + j] = (j < n) ? exp(lg[j] - m) / s : 0.0;
        lli[i] = m + log(s);
    }
    for (i = 0; i < N; ++i) L += lli[i];  /* sequential: fixed order */
    if (ll) memcpy(ll, lli, sizeof(double) * (size_t)N);
    free(F);
    free(lli);
    return L;
}

/* ------------------------------------------------------------------------
 * M-step for every superpixel k, over its pixel set I_k (Eq. Ik):
 *   mu_k      = sum R_ik z_i / sum R_ik                                   Eq. (UpdateMu)
 *   Sigma_k,s = sum R_ik (z_i,s - mu_k,s)(z_i,s - mu_k,s)^T / sum R_ik      Eq. (UpdateSigS)
 *   Sigma_k,c = sum R_ik (z_i,c - mu_k,c)(z_i,c - mu_k,c)^T / sum R_ik      Eq. (UpdateSigC)
 * then the eigenvalue floor (Eq. mlams, mlamc) with eps_s, eps_c.
 * The covariances use the new mean (Algorithm 1, step 4 before step 5) and
 * are formed in two passes: the mean first, then centred products.
 * Split model (Eq. BlockSigma1): sigma_l^2 and the (a, b) block are the
 * same weighted sums with the L-a, L-b entries not formed (zero), and each
 * block is floored on its own.  Grayscale: the colour is L alone (mu's a, b
 * and Sigma_c's entries other than LL are zero).
 * mu, cs, cc hold theta_t on entry and theta_{t+1} on return.
 * cs_raw/cc_raw (optional) receive the covariances before the floor;
 * wsum (optional) receives sum_i R_ik; nraised (optional, [2]) counts the
 * raised spatial and colour eigenvalues.  Returns the number of superpixels
 * kept unchanged because their total weight was below 1e-8.
 * ---------------------------------------------------------------------- */
int orc_mstep(const double *lab, int W, int H, int v, int nx, int ny,
              const int32_t *cand, const int32_t *ncand, const double *R,
              double eps_s, double eps_c, double *mu, double *cs, double *cc,
              double *cs_raw, double *cc_raw, double *wsum, int *nraised, int cmodel)
{
    int K = nx * ny, k, dead = 0, rs = 0, rc = 0;
#pragma omp parallel for schedule(static) reduction(+ : dead, rs, rc)
    for (k = 0; k < K; ++k) {
        int kx = k % nx, ky = k / nx, xb, xe, yb, ye, x, y, j, c;
        double Wk = 0.0, S[5] = {0, 0, 0, 0, 0}, m[5], ps[3] = {0, 0, 0}, pc[6] = {0, 0, 0, 0, 0, 0};
        window(kx, v, W, &xb, &xe);
        window(ky, v, H, &yb, &ye);
        /* pass 1: weights and weighted sums -> mean */
        for (y = yb; y < ye; ++y)
            for (x = xb; x < xe; ++x) {
                long i = (long)y * W + x;
                double r = 0.0, z[5];
                for (j = 0; j < ncand[i]; ++j)
                    if (cand[i * ORC_MAXC + j] == k) r = R[i * ORC_MAXC + j];
                z[0] = x; z[1] = y;
                z[2] = lab[3 * i + 0]; z[3] = lab[3 * i + 1]; z[4] = lab[3 * i + 2];
                Wk += r;
                for (c = 0; c < 5; ++c) S[c] += r * z[c];
            }
        if (wsum) wsum[k] = Wk;
        if (!(Wk >= ORC_DEAD_W)) {
            ++dead;
            if (cs_raw) memcpy(cs_raw + 3 * k, cs + 3 * k, sizeof(double) * 3);
            if (cc_raw) memcpy(cc_raw + 6 * k, cc + 6 * k, sizeof(double) * 6);
            continue;
        }
        for (c = 0; c < 5; ++c) m[c] = S[c] / Wk;
        /* pass 2: centred second moments with the new mean */
        for (y = yb; y < ye; ++y)
            for (x = xb; x < xe; ++x) {
                long i = (long)y * W + x;
                double r = 0.0, d[5];
                for (j = 0; j < ncand[i]; ++j)
                    if (cand[i * ORC_MAXC + j] == k) r = R[i * ORC_MAXC + j];
                d[0] = x - m[0]; d[1] = y - m[1];
                d[2] = lab[3 * i + 0] - m[2]; d[3] = lab[3 * i + 1] - m[3]; d[4] = lab[3 * i + 2] - m[4];
                ps[0] += r * d[0] * d[0]; ps[1] += r * d[0] * d[1]; ps[2] += r * d[1] * d[1];
                pc[0] += r * d[2] * d[2];
                if (cmodel == ORC_FULL) { pc[1] += r * d[2] * d[3]; pc[2] += r * d[2] * d[4]; }
                if (cmodel != ORC_GRAY) {
                    pc[3] += r * d[3] * d[3]; pc[4] += r * d[3] * d[4]; pc[5] += r * d[4] * d[4];
                }
            }
        for (c = 0; c < 3; ++c) ps[c] /= Wk;
        for (c = 0; c < 6; ++c) pc[c] /= Wk;
        if (cs_raw) memcpy(cs_raw + 3 * k, ps, sizeof(double) * 3);
        if (cc_raw) memcpy(cc_raw + 6 * k, pc, sizeof(double) * 6);
        if (cmodel == ORC_GRAY) m[3] = m[4] = 0.0;
        for (c = 0; c < 5; ++c) mu[5 * k + c] = m[c];
        rs += orc_eig_clamp(2, ps, eps_s, cs + 3 * k);
        if (cmodel == ORC_FULL) {
            rc += orc_eig_clamp(3, pc, eps_c, cc + 6 * k);
        } else {
            double ab[3] = {pc[3], pc[4], pc[5]}, ab_out[3] = {0.0, 0.0, 0.0};
            memset(cc + 6 * k, 0, sizeof(double) * 6);
            rc += orc_eig_clamp(1, pc, eps_c, cc + 6 * k);
            if (cmodel == ORC_SPLIT) {
                rc += orc_eig_clamp(2, ab, eps_c, ab_out);
                cc[6 * k + 3] = ab_out[0]; cc[6 * k + 4] = ab_out[1]; cc[6 * k + 5] = ab_out[2];
            }
        }
    }
    if (nraised) { nraised[0] = rs; nraised[1] = rc; }
    return dead;
}

/* ------------------------------------------------------------------------
 * Labels, Eq. (obtLi): L_i = argmax_{k in K_i} R_ik; ties go to the smaller
 * k (candidates are in ascending k, so the first maximum wins).
 * margin[i] (optional) = R_(1) - R_(2), the gap between the two largest
 * posteriors (1 when |K_i| = 1).
 * ---------------------------------------------------------------------- */
void orc_labels(long N, const int32_t *cand, const int32_t *ncand, const double *R,
                int32_t *labels, double *margin)
{
    long i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < N; ++i) {
        int j, best = 0;
        double r1 = -1.0, r2 = -1.0;
        for (j = 0; j < ncand[i]; ++j) {
            double r = R[i * ORC_MAXC + j];
            if (r > r1) { r2 = r1; r1 = r; best = j; }
            else if (r > r2) r2 = r;
        }
        labels[i] = cand[i * ORC_MAXC + best];
        if (margin) margin[i] = (ncand[i] > 1) ? r1 - r2 : 1.0;
    }
}

/* ------------------------------------------------------------------------
 * Algorithm 1, steps 1-7, for T iterations, on a CIELAB image, for the
 * colour model cmodel (grayscale reads only the L column of lab).
 *   step 1   initialise theta (Sec. III-C)
 *   step 2   R from theta_0
 *   loop T:  steps 4-5 (M-step with the floor), step 6 (R from theta_{t+1})
 *   step 7   labels from the last R
 * theta_in (optional): if mu_in is non-null the loop starts from
 * (mu_in, cs_in, cc_in) instead of step 1.
 * loglik[t] = L(theta_t) for t = 0..T (T+1 values).
 * mu/cs/cc receive theta_T.  labels and margin (optional) are N long.
 * post (optional, N x 9) receives the last posteriors, cand/ncand
 * (optional) the candidate sets.  raised (optional, 2*T) the number of
 * raised spatial/colour eigenvalues per iteration.
 * Returns the number of dead-superpixel events, or a negative error code.
 * ---------------------------------------------------------------------- */
int orc_em(const double *lab, int W, int H, int K_req, int spacing, int T,
           double lambda_c, double eps_s, double eps_c,
           const double *mu_in, const double *cs_in, const double *cc_in,
           double *mu, double *cs, double *cc, int32_t *labels, double *margin,
           double *loglik, double *post, int32_t *cand_out, int32_t *ncand_out, int *raised, int cmodel)
{
    int g[4], v, nx, ny, K, t, dead = 0;
    long N = (long)W * H;
    int32_t *cand, *ncand;
    double *R;
    if (orc_grid(W, H, K_req, spacing, g)) return -1;
    v = g[0]; nx = g[1]; ny = g[2]; K = g[3];
    cand = malloc(sizeof(int32_t) * ORC_MAXC * (size_t)N);
    ncand = malloc(sizeof(int32_t) * (size_t)N);
    R = malloc(sizeof(double) * ORC_MAXC * (size_t)N);
    if (!cand || !ncand || !R) { free(cand); free(ncand); free(R); return -2; }
    if (orc_candidates(W, H, v, nx, ny, cand, ncand)) { dead = -3; goto done; }
    if (mu_in) {
        memcpy(mu, mu_in, sizeof(double) * 5 * K);
        memcpy(cs, cs_in, sizeof(double) * 3 * K);
        memcpy(cc, cc_in, sizeof(double) * 6 * K);
    } else {
        orc_init(lab, W, H, v, nx, ny, lambda_c, mu, cs, cc, cmodel);
    }
    {
        double L0 = orc_estep(lab, W, H, K, cand, ncand, mu, cs, cc, R, NULL, cmodel);
        if (loglik) loglik[0] = L0;
    }
    for (t = 0; t < T; ++t) {
        int nr[2];
        double Lt;
        dead += orc_mstep(lab, W, H, v, nx, ny, cand, ncand, R, eps_s, eps_c, mu, cs, cc,
                          NULL, NULL, NULL, nr, cmodel);
        if (raised) { raised[2 * t] = nr[0]; raised[2 * t + 1] = nr[1]; }
        Lt = orc_estep(lab, W, H, K, cand, ncand, mu, cs, cc, R, NULL, cmodel);
        if (loglik) loglik[t + 1] = Lt;
    }
    orc_labels(N, cand, ncand, R, labels, margin);
    if (post) memcpy(post, R, sizeof(double) * ORC_MAXC * (size_t)N);
    if (cand_out) memcpy(cand_out, cand, sizeof(int32_t) * ORC_MAXC * (size_t)N);
    if (ncand_out) memcpy(ncand_out, ncand, sizeof(int32_t) * (size_t)N);
done:
    free(cand); free(ncand); free(R);
    return dead;
}
