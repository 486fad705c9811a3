/*
 * hsc_oracle.c -- plain, slow FP64 CPU oracle of the spatial-spectral
 * classifier's hot path (PCA one-band, OvO SVM + Platt + pairwise coupling,
 * row-window KNN filter).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the bench's
 * CPU-baseline leg may load this library. It shares no code, header, table or
 * helper with the CUDA library; the two only see the same seeded inputs.
 *
 * Every stage follows the paper's description directly, in double precision,
 * with no blocking, fusion or reordering:
 *   PCA  -- Section II.C.2 steps (i)-(iv): band means, covariance of the
 *           centred image (divided by the pixel count, Section III.A.2.b),
 *           classical Jacobi (rotate on the largest off-diagonal element until
 *           all are below the stop threshold), projection on the first
 *           eigenvector, then min-max normalisation of the one-band image
 *           (the "normalized pixel value" of Eq. 1).
 *   SVM  -- Section II.C.1 / III.A.1: distances to the one-vs-one hyperplanes,
 *           sigmoid (Platt) binary probabilities, and the pairwise coupling of
 *           the paper's reference [30] (Wu, Lin, Weng 2004, second method),
 *           whose exact minimiser is the solution of its FP64 KKT system.
 *   KNN  -- Section II.C.3, Eq. 1 and Eq. 2, with the 14-row window of
 *           Section III.A.3: every window candidate's distance, a full sort by
 *           (distance, linear index), the first K kept, their probabilities
 *           averaged, argmax label.
 *
 * Readings where the paper is silent or garbled:
 *   - Eq. 1's third term is printed (r-j)^2; it is read as (c-j)^2.
 *   - lambda scales the spatial coordinates: d = dI^2 + lambda^2 (dr^2 + dc^2).
 *   - the window holds rows r-floor(R/2) .. r+ceil(R/2)-1, truncated at the
 *     image edges, all columns; the pixel itself is a candidate.
 *   - distance ties are broken by the smaller linear index i*W+j; label ties
 *     by the smaller class.
 *   - Platt: r_ij = 1/(1+exp(A f + B)), clipped to [1e-7, 1-1e-7].
 *   - the first eigenvector's sign is fixed so that its largest-magnitude
 *     component is positive (ties: smaller band index).
 *
 * Return codes: 0 ok, 1 invalid argument, 4 Jacobi did not converge.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_INVALID 1
#define ORC_NOT_CONVERGED 4

/* ---------------------------------------------------------------- PCA --- */

/* Step (i): band means, Neumaier-compensated FP64 sums over the N pixels. */
int oracle_band_means(const float *cube, int B, long N, double *mu)
{
    if (!cube || !mu || B <= 0 || N <= 0) return ORC_INVALID;
    for (int b = 0; b < B; ++b) {
        const float *band = cube + (size_t)b * (size_t)N;
        double s = 0.0, comp = 0.0;
        for (long p = 0; p < N; ++p) {
            double x = (double)band[p];
            double t = s + x;
            if (fabs(s) >= fabs(x)) comp += (s - t) + x;
            else comp += (x - t) + s;
            s = t;
        }
        mu[b] = (s + comp) / (double)N;
    }
    return ORC_OK;
}

/* Step (ii): covariance of the centred image, C = Xc Xc^T / N (B x B,
 * symmetric, row-major), second pass over the data after the means. */
int oracle_covariance(const float *cube, int B, long N, const double *mu, double *C)
{
    if (!cube || !mu || !C || B <= 0 || N <= 0) return ORC_INVALID;
    double *y = (double *)malloc(sizeof(double) * (size_t)B);
    if (!y) return ORC_INVALID;
    memset(C, 0, sizeof(double) * (size_t)B * (size_t)B);
    for (long p = 0; p < N; ++p) {
        for (int b = 0; b < B; ++b) y[b] = (double)cube[(size_t)b * (size_t)N + p] - mu[b];
        for (int b = 0; b < B; ++b) {
            double yb = y[b];
            double *row = C + (size_t)b * B;
            for (int c = b; c < B; ++c) row[c] += yb * y[c];
        }
    }
    for (int b = 0; b < B; ++b)
        for (int c = b; c < B; ++c) {
            double v = C[(size_t)b * B + c] / (double)N;
            C[(size_t)b * B + c] = v;
            C[(size_t)c * B + b] = v;
        }
    free(y);
    return ORC_OK;
}

/* Step (iii): classical Jacobi. Each rotation zeroes the off-diagonal entry of
 * largest magnitude (ties: smallest (p,q) in row-major order); the rotation is
 * the symmetric Schur rotation (t = sgn(tau)/(|tau|+sqrt(1+tau^2)) with
 * tau = (a_qq - a_pp)/(2 a_pq)). Stops when every off-diagonal magnitude is
 * <= tol * ||C||_F. A = working copy, V accumulates the rotations, so that on
 * exit C = V diag(evals) V^T. */
int oracle_jacobi(const double *C, int B, double tol, long max_rot,
                  double *evals, double *V, long *n_rot)
{
    if (!C || !evals || !V || B <= 0) return ORC_INVALID;
    size_t n2 = (size_t)B * (size_t)B;
    double *A = (double *)malloc(sizeof(double) * n2);
    if (!A) return ORC_INVALID;
    memcpy(A, C, sizeof(double) * n2);
    memset(V, 0, sizeof(double) * n2);
    for (int i = 0; i < B; ++i) V[(size_t)i * B + i] = 1.0;
    double fro = 0.0;
    for (size_t i = 0; i < n2; ++i) fro += C[i] * C[i];
    fro = sqrt(fro);
    double stop = tol * fro;
    if (max_rot <= 0) max_rot = 100L * B * B;
    long rot = 0;
    int status = ORC_OK;
    for (;;) {
        int p = 0, q = 1;
        double big = -1.0;
        for (int i = 0; i < B; ++i)
            for (int j = i + 1; j < B; ++j) {
                double a = fabs(A[(size_t)i * B + j]);
                if (a > big) { big = a; p = i; q = j; }
            }
        if (B < 2 || big <= stop) break;
        if (rot >= max_rot) { status = ORC_NOT_CONVERGED; break; }
        double app = A[(size_t)p * B + p], aqq = A[(size_t)q * B + q];
        double apq = A[(size_t)p * B + q];
        double tau = (aqq - app) / (2.0 * apq);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = t * c;
        /* A <- A J (columns p, q) */
        for (int i = 0; i < B; ++i) {
            double aip = A[(size_t)i * B + p], aiq = A[(size_t)i * B + q];
            A[(size_t)i * B + p] = c * aip - s * aiq;
            A[(size_t)i * B + q] = s * aip + c * aiq;
        }
        /* A <- J^T A (rows p, q) */
        for (int j = 0; j < B; ++j) {
            double apj = A[(size_t)p * B + j], aqj = A[(size_t)q * B + j];
            A[(size_t)p * B + j] = c * apj - s * aqj;
            A[(size_t)q * B + j] = s * apj + c * aqj;
        }
        /* V <- V J */
        for (int i = 0; i < B; ++i) {
            double vip = V[(size_t)i * B + p], viq = V[(size_t)i * B + q];
            V[(size_t)i * B + p] = c * vip - s * viq;
            V[(size_t)i * B + q] = s * vip + c * viq;
        }
        ++rot;
    }
    for (int i = 0; i < B; ++i) evals[i] = A[(size_t)i * B + i];
    if (n_rot) *n_rot = rot;
    free(A);
    return status;
}

/* Step (iv): projection of the centred pixels on the first eigenvector,
 * I_p = v1^T (x_p - mu), then the min-max normalisation (I - min)/(max - min)
 * (all zeros when I is constant). I_norm is nullable. */
int oracle_project(const float *cube, int B, long N, const double *mu, const double *v1,
                   double *I_raw, double *I_norm)
{
    if (!cube || !mu || !v1 || !I_raw || B <= 0 || N <= 0) return ORC_INVALID;
    double mn = INFINITY, mx = -INFINITY;
    for (long p = 0; p < N; ++p) {
        double acc = 0.0;
        for (int b = 0; b < B; ++b)
            acc += v1[b] * ((double)cube[(size_t)b * (size_t)N + p] - mu[b]);
        I_raw[p] = acc;
        if (acc < mn) mn = acc;
        if (acc > mx) mx = acc;
    }
    if (I_norm)
        for (long p = 0; p < N; ++p)
            I_norm[p] = (mx > mn) ? (I_raw[p] - mn) / (mx - mn) : 0.0;
    return ORC_OK;
}

/* Whole one-band PCA (steps (i)-(iv) plus the min-max normalisation that the
 * KNN's "normalized pixel value" needs). Outputs (all caller-allocated):
 *   mu[B], C[B*B], evals[B], V[B*B], v1[B], *lambda1,
 *   I_raw[N] = v1^T (x_p - mu), I_norm[N] = (I - min)/(max - min) (0 if flat).
 */
int oracle_pca_one_band(const float *cube, int B, int H, int W, double tol,
                        double *mu, double *C, double *evals, double *V,
                        double *v1, double *lambda1, double *I_raw,
                        double *I_norm, long *n_rot)
{
    if (!cube || B <= 0 || H <= 0 || W <= 0) return ORC_INVALID;
    long N = (long)H * (long)W;
    int st = oracle_band_means(cube, B, N, mu);
    if (st) return st;
    st = oracle_covariance(cube, B, N, mu, C);
    if (st) return st;
    st = oracle_jacobi(C, B, tol, 0, evals, V, n_rot);
    int lead = 0;
    for (int i = 1; i < B; ++i) if (evals[i] > evals[lead]) lead = i;
    for (int b = 0; b < B; ++b) v1[b] = V[(size_t)b * B + lead];
    int big = 0;
    for (int b = 1; b < B; ++b) if (fabs(v1[b]) > fabs(v1[big])) big = b;
    if (v1[big] < 0.0) for (int b = 0; b < B; ++b) v1[b] = -v1[b];
    *lambda1 = evals[lead];
    oracle_project(cube, B, N, mu, v1, I_raw, I_norm);
    return st;
}

/* ---------------------------------------------------------------- SVM --- */

/* Pairwise coupling, second method of Wu, Lin and Weng (2004), the paper's
 * reference [30]: p minimises sum_i sum_{j!=i} (r_ji p_i - r_ij p_j)^2 subject
 * to sum p = 1. With Q_ii = sum_{j!=i} r_ji^2 and Q_ij = -r_ji r_ij the
 * objective is p^T Q p; Q is only positive semi-definite (it is singular
 * whenever the r_ij are consistent, e.g. always for k = 2), so the minimiser is
 * taken from the optimality (KKT) system
 *     [ Q   e ] [ p ]   [ 0 ]
 *     [ e^T 0 ] [ b ] = [ 1 ]
 * solved by Gaussian elimination with partial pivoting.
 * r is k x k row-major with r[i*k+j] = r_ij (diagonal ignored). */
int oracle_couple(const double *r, int k, double *p)
{
    if (!r || !p || k < 2 || k > 64) return ORC_INVALID;
    int n = k + 1;
    double A[65 * 66];                       /* n x (n+1) augmented matrix */
    memset(A, 0, sizeof(A));
#define AE(i, j) A[(i) * (n + 1) + (j)]
    for (int i = 0; i < k; ++i) {
        double d = 0.0;
        for (int j = 0; j < k; ++j) {
            if (j == i) continue;
            d += r[j * k + i] * r[j * k + i];
            AE(i, j) = -r[j * k + i] * r[i * k + j];
        }
        AE(i, i) = d;
        AE(i, k) = 1.0;
        AE(k, i) = 1.0;
    }
    AE(k, k) = 0.0;
    AE(k, n) = 1.0;
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int i = col + 1; i < n; ++i)
            if (fabs(AE(i, col)) > fabs(AE(piv, col))) piv = i;
        if (AE(piv, col) == 0.0) return ORC_INVALID;
        if (piv != col)
            for (int j = 0; j <= n; ++j) { double t = AE(col, j); AE(col, j) = AE(piv, j); AE(piv, j) = t; }
        for (int i = col + 1; i < n; ++i) {
            double f = AE(i, col) / AE(col, col);
            for (int j = col; j <= n; ++j) AE(i, j) -= f * AE(col, j);
        }
    }
    double x[65];
    for (int i = n - 1; i >= 0; --i) {
        double t = AE(i, n);
        for (int j = i + 1; j < n; ++j) t -= AE(i, j) * x[j];
        x[i] = t / AE(i, i);
    }
#undef AE
    for (int i = 0; i < k; ++i) p[i] = x[i];
    return ORC_OK;
}

/* Platt binary probability of one hyperplane, clipped. */
static double platt(double f, double A, double Bp)
{
    double r = 1.0 / (1.0 + exp(A * f + Bp));
    if (r < 1e-7) r = 1e-7;
    if (r > 1.0 - 1e-7) r = 1.0 - 1e-7;
    return r;
}

/* Per-pixel SVM classification (Section II.C.1): M = k(k-1)/2 decision values
 * f_m = w_m . x + b_m on the raw (un-centred) spectrum, Platt probabilities
 * r_ij and r_ji = 1 - r_ij, coupling into k class probabilities, argmax.
 * Pairs m run (0,1),(0,2),...,(k-2,k-1). P is k x N (class-major).
 * dec (nullable) receives the M x N decision values. */
int oracle_svm_probs(const float *cube, int B, long N, int k, const float *w,
                     const float *bias, const float *pa, const float *pb,
                     double *P, int *labels, double *dec)
{
    if (!cube || !w || !bias || !pa || !pb || !P || B <= 0 || N <= 0 || k < 2 || k > 64)
        return ORC_INVALID;
    int M = k * (k - 1) / 2;
    double r[64 * 64], p[64];
    for (long px = 0; px < N; ++px) {
        int m = 0;
        for (int i = 0; i < k; ++i)
            for (int j = i + 1; j < k; ++j, ++m) {
                double f = (double)bias[m];
                for (int b = 0; b < B; ++b)
                    f += (double)w[(size_t)m * B + b] * (double)cube[(size_t)b * (size_t)N + px];
                if (dec) dec[(size_t)m * (size_t)N + px] = f;
                double rij = platt(f, (double)pa[m], (double)pb[m]);
                r[i * k + j] = rij;
                r[j * k + i] = 1.0 - rij;
            }
        (void)M;
        int st = oracle_couple(r, k, p);
        if (st) return st;
        int best = 0;
        for (int c = 0; c < k; ++c) {
            P[(size_t)c * (size_t)N + px] = p[c];
            if (p[c] > p[best]) best = c;
        }
        if (labels) labels[px] = best;
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------- KNN --- */

/* A candidate's sort key: (d, lo, q). In the FP64 mode lo = 0 and d is the
 * distance. In the float mode (d, lo) is the exact sum s + e of the float
 * terms as an unevaluated pair (hi = fl(s + e), lo = the rounding error), so
 * ordering by (d, lo) orders the real values s + e. */
typedef struct { double d; double lo; long q; } cand_t;

static int cand_cmp(const void *a, const void *b)
{
    const cand_t *x = (const cand_t *)a, *y = (const cand_t *)b;
    if (x->d < y->d) return -1;
    if (x->d > y->d) return 1;
    if (x->lo < y->lo) return -1;
    if (x->lo > y->lo) return 1;
    return (x->q < y->q) ? -1 : (x->q > y->q);
}

/* Eq. 1 with float terms, as the paper's GPU and manycore KNN compute it in
 * float (Section III.B.3): dI = fl(I_p - I_q), e = fl(dI^2),
 * s = fl(fl(lambda^2) (dr^2 + dc^2)), and the sum s + e taken exactly
 * (Knuth's two-sum) so that comparing two candidates compares the real sums.
 * Each float operation is a separately rounded ISO C float operation
 * (compiled without floating-point contraction). */
static void float_key(float Ip, float Iq, float l2, int dr, int dc, double *hi, double *lo)
{
    volatile float dI = Ip - Iq;
    volatile float e = dI * dI;
    volatile float s = l2 * (float)(dr * dr + dc * dc);
    volatile float h = s + e;
    volatile float bb = h - s;
    volatile float t1 = h - bb;
    volatile float t2 = s - t1;
    volatile float t3 = e - bb;
    volatile float l = t2 + t3;
    *hi = (double)h;
    *lo = (double)l;
}

/* Smallest number of window candidates over all rows: K must not exceed it. */
long oracle_knn_min_candidates(int H, int W, int R)
{
    int up = (R + 1) / 2;               /* rows r .. r+ceil(R/2)-1 */
    int rows = up < H ? up : H;
    return (long)rows * (long)W;
}

/* KNN filter of Section II.C.3 for pixels p0 <= p < p1 (linear index r*W+c).
 * Inputs: I_norm (float, H*W, the normalised one-band image), P (float,
 * k x H*W). For each pixel all candidates q = i*W+j with i in the window rows
 * and any column j get d = (I_p - I_q)^2 + lambda^2 ((r-i)^2 + (c-j)^2)
 * computed in FP64 from the float inputs (Eq. 1); the candidates are sorted by
 * (d, q) and the first K averaged (Eq. 2). Outputs per processed pixel t =
 * p - p0 (all nullable except O): O[c*(p1-p0)+t], labels[t],
 * nbr[t*(K+1)+m] = the first K+1 candidates in sorted order (the last is -1
 * when the window holds only K), dK[t] = K-th distance, dK1[t] = (K+1)-th
 * (inf if none), gapO[t] = largest minus second largest O. */
int oracle_knn(const float *I_norm, const float *P, int H, int W, int k, int K,
               int R, double lambda, int float_keys, long p0, long p1, double *O,
               int *labels, int *nbr, double *dK, double *dK1, double *gapO)
{
    if (!I_norm || !P || !O || H <= 0 || W <= 0 || k < 1 || K < 1 || R < 1 ||
        !(lambda >= 0.0) || p0 < 0 || p1 > (long)H * W || p1 < p0)
        return ORC_INVALID;
    if ((long)K > oracle_knn_min_candidates(H, W, R)) return ORC_INVALID;
    long N = (long)H * W, np = p1 - p0;
    double l2 = lambda * lambda;
    volatile float lamf = (float)lambda;
    volatile float l2f = lamf * lamf;
    cand_t *cand = (cand_t *)malloc(sizeof(cand_t) * (size_t)R * (size_t)W);
    if (!cand) return ORC_INVALID;
    for (long p = p0; p < p1; ++p) {
        long t = p - p0;
        int r = (int)(p / W), c = (int)(p % W);
        int lo = r - R / 2, hi = r + (R + 1) / 2 - 1;
        if (lo < 0) lo = 0;
        if (hi > H - 1) hi = H - 1;
        double Ip = (double)I_norm[p];
        long n = 0;
        for (int i = lo; i <= hi; ++i)
            for (int j = 0; j < W; ++j) {
                long q = (long)i * W + j;
                if (float_keys) {
                    float_key(I_norm[p], I_norm[q], l2f, r - i, c - j, &cand[n].d, &cand[n].lo);
                } else {
                    double dI = Ip - (double)I_norm[q];
                    double dr = (double)(r - i), dc = (double)(c - j);
                    cand[n].d = dI * dI + l2 * (dr * dr + dc * dc);
                    cand[n].lo = 0.0;
                }
                cand[n].q = q;
                ++n;
            }
        qsort(cand, (size_t)n, sizeof(cand_t), cand_cmp);
        int best = 0;
        double top1 = -INFINITY, top2 = -INFINITY;
        for (int cl = 0; cl < k; ++cl) {
            double s = 0.0;
            for (int m = 0; m < K; ++m) s += (double)P[(size_t)cl * (size_t)N + cand[m].q];
            double o = s / (double)K;
            O[(size_t)cl * (size_t)np + t] = o;
            if (o > top1) { top2 = top1; top1 = o; best = cl; }
            else if (o > top2) top2 = o;
        }
        if (labels) labels[t] = best;
        if (nbr)
            for (int m = 0; m <= K; ++m)
                nbr[t * (K + 1) + m] = (m < n) ? (int)cand[m].q : -1;
        if (dK) dK[t] = cand[K - 1].d + cand[K - 1].lo;
        if (dK1) dK1[t] = (n > K) ? cand[K].d + cand[K].lo : INFINITY;
        if (gapO) gapO[t] = (k > 1) ? top1 - top2 : INFINITY;
    }
    free(cand);
    return ORC_OK;
}
