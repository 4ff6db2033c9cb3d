/*
 * bpmf_oracle.c -- plain, slow FP64 reference of one BPMF Gibbs sampler.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * What it follows:
 *   - The Gibbs loop of Algorithm 1 (Sec. 2): per sampling iteration, sample
 *     the movie hyper-parameters from V, update every movie, sample the user
 *     hyper-parameters from U, update every user, then predict every test
 *     point and compute the RMSE.
 *   - The per-item update of Sec. 2 / Sec. 3.1: precision = prior precision
 *     plus alpha times the outer products of the other side's vectors; the
 *     precision is factored by Cholesky instead of being inverted.
 *   - The conditionals the paper takes from its BPMF citation (Salakhutdinov
 *     and Mnih 2008), written out in the comments below.
 *   - Philox4x32-10 as defined by Salmon, Moraes, Dror and Shaw, "Parallel
 *     random numbers: as easy as 1, 2, 3" (SC'11); Box-Muller normals; the
 *     Marsaglia-Tsang (2000) gamma sampler; Bartlett's decomposition of the
 *     Wishart distribution.
 *
 * Everything is double precision, unblocked and in textbook order.  Rows of
 * one side are independent given the other side (Sec. 3.2), so the row loop
 * is split over threads by contiguous ranges; each row's arithmetic does not
 * depend on the thread count.
 *
 * Random-number layout (shared by definition, not by code, with the GPU path):
 *   key     = (seed low 32 bits, seed high 32 bits)
 *   counter = (c0 = call index, c1 = element index, c2 = sweep, c3 = tag | job << 8)
 *   tags    : 0 init U, 1 init V, 2 U row noise, 3 V row noise,
 *             4 U hyper normals, 5 V hyper normals, 6 U gamma, 7 V gamma
 *   a "normal stream" (c1, c2, c3) is the concatenation of the four normals
 *   of calls c0 = 0, 1, 2, ...; normal q comes from call q/4, word pair
 *   (q%4)/2, cosine branch for even q and sine branch for odd q.
 *   uniforms use the top 24 bits of a word: open  u = (w>>8 + 1) 2^-24 in (0,1]
 *                                           angle t = (w>>8)     2^-24 in [0,1)
 *   Box-Muller: rho = sqrt(-2 ln u), z = rho cos(2 pi t), rho sin(2 pi t).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2
#define ORC_ENOTPD -4
#define ORC_EGAMMA -7

#define ORC_FLAG_CLIP 0x2u
#define ORC_FLAG_NO_CENTER 0x8u

#define ORC_GAMMA_MAX_ATTEMPTS 64

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 4.2): ten rounds of the 4x32     */
/* Philox S-box with multipliers 0xD2511F53, 0xCD9E8D57 and the key schedule */
/* (Weyl sequence) 0x9E3779B9, 0xBB67AE85.                                    */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static double u_open(uint32_t w) { return ((double)(w >> 8) + 1.0) * 0x1p-24; }
static double u_angle(uint32_t w) { return (double)(w >> 8) * 0x1p-24; }

static const double ORC_PI = 3.14159265358979323846;

/* Box-Muller transform of two words into two standard normals. */
static void box_muller(uint32_t wa, uint32_t wb, double* zc, double* zs)
{
    double rho = sqrt(-2.0 * log(u_open(wa)));
    double th = 2.0 * ORC_PI * u_angle(wb);
    *zc = rho * cos(th);
    *zs = rho * sin(th);
}

static void make_key(uint64_t seed, uint32_t key[2])
{
    key[0] = (uint32_t)(seed & 0xffffffffu);
    key[1] = (uint32_t)(seed >> 32);
}

/* Normals q = first .. first+count-1 of the stream (c1, c2, c3). */
void orc_normal_stream(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3,
                       int64_t first, int64_t count, double* out)
{
    uint32_t key[2];
    make_key(seed, key);
    for (int64_t i = 0; i < count; ++i) {
        int64_t q = first + i;
        uint32_t ctr[4] = {(uint32_t)(q / 4), c1, c2, c3};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        int pair = (int)((q % 4) / 2);
        double zc, zs;
        box_muller(w[2 * pair], w[2 * pair + 1], &zc, &zs);
        out[i] = (q % 2 == 0) ? zc : zs;
    }
}

/*
 * Gamma(shape a, scale 1), a >= 1, by Marsaglia and Tsang (2000): with
 * d = a - 1/3 and c = 1/sqrt(9d), draw x ~ N(0,1) and u ~ U(0,1]; set
 * v = (1 + c x)^3; accept d*v when 1 + c x > 0 and
 * ln u < x^2/2 + d - d v + d ln v.  Attempt number t uses one Philox call
 * with counter (t, c1, c2, c3): words 0,1 give x (cosine branch), word 2
 * gives u.  Only the exact logarithmic test is used (no squeeze), so the
 * accept decision is the defining inequality itself.
 */
int orc_gamma(uint64_t seed, double a, uint32_t c1, uint32_t c2, uint32_t c3, double* out,
              int* attempts)
{
    uint32_t key[2];
    make_key(seed, key);
    if (!(a >= 1.0)) return ORC_EINVAL;
    double d = a - 1.0 / 3.0;
    double c = 1.0 / sqrt(9.0 * d);
    for (int t = 0; t < ORC_GAMMA_MAX_ATTEMPTS; ++t) {
        uint32_t ctr[4] = {(uint32_t)t, c1, c2, c3};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        double x, unused;
        box_muller(w[0], w[1], &x, &unused);
        double s = 1.0 + c * x;
        if (s <= 0.0) continue;
        double v = s * s * s;
        double u = u_open(w[2]);
        if (log(u) < 0.5 * x * x + d - d * v + d * log(v)) {
            *out = d * v;
            if (attempts) *attempts = t + 1;
            return ORC_OK;
        }
    }
    return ORC_EGAMMA;
}

/* ------------------------------------------------------------------------- */
/* Dense FP64 linear algebra, textbook forms, row-major K x K.               */
/* ------------------------------------------------------------------------- */

/* Cholesky-Banachiewicz: A = L L^T, L lower triangular; upper part zeroed. */
int orc_cholesky(int K, const double* A, double* L)
{
    for (int i = 0; i < K * K; ++i) L[i] = 0.0;
    for (int i = 0; i < K; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = A[i * K + j];
            for (int k = 0; k < j; ++k) s -= L[i * K + k] * L[j * K + k];
            if (i == j) {
                if (!(s > 0.0)) return ORC_ENOTPD;
                L[i * K + i] = sqrt(s);
            } else {
                L[i * K + j] = s / L[j * K + j];
            }
        }
    }
    return ORC_OK;
}

/* Solve L y = b (forward substitution). */
static void solve_lower(int K, const double* L, const double* b, double* y)
{
    for (int i = 0; i < K; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[i * K + k] * y[k];
        y[i] = s / L[i * K + i];
    }
}

/* Solve L^T x = y (back substitution with the transpose of L). */
static void solve_upper_t(int K, const double* L, const double* y, double* x)
{
    for (int i = K - 1; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < K; ++k) s -= L[k * K + i] * x[k];
        x[i] = s / L[i * K + i];
    }
}

/* Inverse of an SPD matrix: columns of A^{-1} from L L^T x = e_c. */
int orc_spd_inverse(int K, const double* A, double* Ainv)
{
    double* L = (double*)malloc(sizeof(double) * (size_t)K * K);
    double* e = (double*)malloc(sizeof(double) * (size_t)K);
    double* y = (double*)malloc(sizeof(double) * (size_t)K);
    double* x = (double*)malloc(sizeof(double) * (size_t)K);
    int rc = (L && e && y && x) ? orc_cholesky(K, A, L) : ORC_ENOMEM;
    if (rc == ORC_OK) {
        for (int c = 0; c < K; ++c) {
            for (int i = 0; i < K; ++i) e[i] = (i == c) ? 1.0 : 0.0;
            solve_lower(K, L, e, y);
            solve_upper_t(K, L, y, x);
            for (int i = 0; i < K; ++i) Ainv[i * K + c] = x[i];
        }
    }
    free(L); free(e); free(y); free(x);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Normal-Wishart hyper-parameter draw (BPMF, Salakhutdinov & Mnih 2008,     */
/* Sec. 3.3, as cited in Sec. 2).  Given n rows with mean xbar and scatter   */
/* S = (1/n) sum (x - xbar)(x - xbar)^T:                                     */
/*   beta* = beta0 + n,  nu* = nu0 + n,                                      */
/*   mu*   = (beta0 mu0 + n xbar) / (beta0 + n),                             */
/*   (W*)^{-1} = W0^{-1} + n S + beta0 n/(beta0 + n) (mu0 - xbar)(mu0 - xbar)^T */
/*   Lambda ~ Wishart(W*, nu*)  (E[Lambda] = nu* W*),                        */
/*   mu ~ N(mu*, (beta* Lambda)^{-1}).                                       */
/* Wishart by Bartlett: Lambda = L_W A A^T L_W^T with L_W = chol(W*), A lower */
/* triangular, A_kk^2 ~ chi^2(nu* - k) = 2 Gamma((nu* - k)/2), A_kl ~ N(0,1)  */
/* for k > l.  Off-diagonal normals: stream (c1 = 0), index k(k-1)/2 + l.     */
/* Mean normals: stream (c1 = 1), index k.  Gamma for diagonal k: c1 = k.    */
/* ------------------------------------------------------------------------- */
int orc_nw_draw(int K, int64_t n, const double* xbar, const double* S, double beta0, double nu0,
                const double* mu0, const double* W0inv, uint64_t seed, uint32_t sweep,
                uint32_t c3_normals, uint32_t c3_gamma, double* Lambda, double* mu)
{
    int rc = ORC_OK;
    size_t KK = (size_t)K * K;
    double* P = (double*)malloc(sizeof(double) * KK);
    double* W = (double*)malloc(sizeof(double) * KK);
    double* LW = (double*)malloc(sizeof(double) * KK);
    double* A = (double*)calloc(KK, sizeof(double));
    double* B = (double*)calloc(KK, sizeof(double));
    double* Lm = (double*)malloc(sizeof(double) * KK);
    double* tmp = (double*)malloc(sizeof(double) * KK);
    double* z = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K * K : 1));
    double* w = (double*)malloc(sizeof(double) * (size_t)K);
    double* mustar = (double*)malloc(sizeof(double) * (size_t)K);
    if (!P || !W || !LW || !A || !B || !Lm || !tmp || !z || !w || !mustar) {
        rc = ORC_ENOMEM;
        goto done;
    }
    double nd = (double)n;
    double beta_s = beta0 + nd, nu_s = nu0 + nd;
    for (int k = 0; k < K; ++k) mustar[k] = (beta0 * mu0[k] + nd * xbar[k]) / (beta0 + nd);
    double cross = beta0 * nd / (beta0 + nd);
    for (int a = 0; a < K; ++a)
        for (int b = 0; b < K; ++b)
            P[a * K + b] = W0inv[a * K + b] + nd * S[a * K + b] +
                           cross * (mu0[a] - xbar[a]) * (mu0[b] - xbar[b]);
    rc = orc_spd_inverse(K, P, W);
    if (rc) goto done;
    rc = orc_cholesky(K, W, LW);
    if (rc) goto done;

    /* Bartlett factor A */
    for (int k = 0; k < K; ++k) {
        double g;
        rc = orc_gamma(seed, 0.5 * (nu_s - (double)k), (uint32_t)k, sweep, c3_gamma, &g, NULL);
        if (rc) goto done;
        A[k * K + k] = sqrt(2.0 * g);
    }
    if (K > 1) {
        int64_t noff = (int64_t)K * (K - 1) / 2;
        orc_normal_stream(seed, 0u, sweep, c3_normals, 0, noff, z);
        for (int k = 1; k < K; ++k)
            for (int l = 0; l < k; ++l) A[k * K + l] = z[(int64_t)k * (k - 1) / 2 + l];
    }
    /* B = L_W A ; Lambda = B B^T */
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) {
            double s = 0.0;
            for (int k = 0; k < K; ++k) s += LW[i * K + k] * A[k * K + j];
            B[i * K + j] = s;
        }
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) {
            double s = 0.0;
            for (int k = 0; k < K; ++k) s += B[i * K + k] * B[j * K + k];
            Lambda[i * K + j] = s;
        }
    /* mu = mu* + chol(beta* Lambda)^{-T} z */
    for (size_t i = 0; i < KK; ++i) tmp[i] = beta_s * Lambda[i];
    rc = orc_cholesky(K, tmp, Lm);
    if (rc) goto done;
    orc_normal_stream(seed, 1u, sweep, c3_normals, 0, K, z);
    solve_upper_t(K, Lm, z, w);
    for (int k = 0; k < K; ++k) mu[k] = mustar[k] + w[k];
done:
    free(P); free(W); free(LW); free(A); free(B); free(Lm); free(tmp); free(z); free(w);
    free(mustar);
    return rc;
}

/* Sufficient statistics of the rows of X (n x K): mean and (1/n) scatter, */
/* by their definitions (two passes).                                      */
void orc_row_stats(int64_t n, int K, const double* X, double* xbar, double* S)
{
    for (int k = 0; k < K; ++k) xbar[k] = 0.0;
    for (int64_t r = 0; r < n; ++r)
        for (int k = 0; k < K; ++k) xbar[k] += X[r * K + k];
    for (int k = 0; k < K; ++k) xbar[k] /= (double)n;
    for (int i = 0; i < K * K; ++i) S[i] = 0.0;
    for (int64_t r = 0; r < n; ++r)
        for (int a = 0; a < K; ++a)
            for (int b = 0; b < K; ++b)
                S[a * K + b] += (X[r * K + a] - xbar[a]) * (X[r * K + b] - xbar[b]);
    for (int i = 0; i < K * K; ++i) S[i] /= (double)n;
}

/*
 * One row's Gaussian conditional (BPMF conditional for u_i, cited in Sec. 2;
 * the per-item update of Alg. 1 and Sec. 3.1):
 *   Lambda_i = Lambda_X + alpha sum_c y_c y_c^T
 *   b_i      = alpha sum_c r_c y_c + Lambda_X mu_X
 *   L = chol(Lambda_i);  mean = L^{-T} L^{-1} b_i;  x = mean + L^{-T} z.
 * `work` holds 3 K*K + 3 K doubles.
 */
int orc_row_conditional(int K, const double* LamX, const double* LamMu, double alpha, int64_t d,
                        const int32_t* idx, const double* val, const double* Y, const double* z,
                        double* mean, double* x, double* work)
{
    double* Lam = work;
    double* L = Lam + (size_t)K * K;
    double* b = L + (size_t)K * K;
    double* y = b + K;
    double* e = y + K;
    for (int i = 0; i < K * K; ++i) Lam[i] = LamX[i];
    for (int k = 0; k < K; ++k) b[k] = LamMu[k];
    for (int64_t t = 0; t < d; ++t) {
        const double* yc = Y + (size_t)idx[t] * K;
        for (int a = 0; a < K; ++a) {
            b[a] += alpha * val[t] * yc[a];
            for (int c = 0; c < K; ++c) Lam[a * K + c] += alpha * yc[a] * yc[c];
        }
    }
    int rc = orc_cholesky(K, Lam, L);
    if (rc) return rc;
    solve_lower(K, L, b, y);
    solve_upper_t(K, L, y, mean);
    solve_upper_t(K, L, z, e);
    for (int k = 0; k < K; ++k) x[k] = mean[k] + e[k];
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Whole sampler state.                                                      */
/* ------------------------------------------------------------------------- */
typedef struct {
    int64_t n_rows;    /* rows of this side */
    int64_t* ptr;      /* n_rows + 1 */
    int32_t* idx;      /* other-side index per rating */
    double* val;       /* centred rating */
    double* X;         /* n_rows x K factors */
    double* mean;      /* n_rows x K last conditional means */
    double* mu;        /* K */
    double* Lambda;    /* K x K */
    double* xbar;      /* K, last statistics */
    double* S;         /* K x K */
} orc_side;

typedef struct orc_state {
    int K;
    double alpha, beta0, nu0;
    double* mu0;
    double* W0inv;
    uint64_t seed;
    uint32_t job;
    int32_t burn_in, order;
    uint32_t flags;
    double clip_lo, clip_hi;
    int32_t nthreads;
    double rbar;
    orc_side side[2]; /* 0 = users (CSR rows), 1 = movies (CSC columns) */
    int64_t T;
    int32_t* ti;
    int32_t* tj;
    double* tr;
    double* psum;
    int64_t n_avg;
    uint32_t sweep;
    int status;
} orc_state;

static uint32_t c3_of(const orc_state* o, uint32_t tag) { return tag | (o->job << 8); }

void orc_destroy(orc_state* o)
{
    if (!o) return;
    for (int s = 0; s < 2; ++s) {
        orc_side* sd = &o->side[s];
        free(sd->ptr); free(sd->idx); free(sd->val); free(sd->X); free(sd->mean);
        free(sd->mu); free(sd->Lambda); free(sd->xbar); free(sd->S);
    }
    free(o->mu0); free(o->W0inv); free(o->ti); free(o->tj); free(o->tr); free(o->psum);
    free(o);
}

orc_state* orc_create(int64_t M, int64_t N, int32_t K, const int64_t* csr_ptr, const int32_t* csr_col,
                      const float* csr_val, int64_t T, const int32_t* ti, const int32_t* tj,
                      const float* tr, double alpha, double beta0, double nu0, const double* mu0,
                      const double* W0, uint64_t seed, uint32_t job, int32_t burn_in, int32_t order,
                      uint32_t flags, double clip_lo, double clip_hi, int32_t nthreads)
{
    if (M <= 0 || N <= 0 || K <= 0 || T < 0) return NULL;
    orc_state* o = (orc_state*)calloc(1, sizeof(orc_state));
    if (!o) return NULL;
    o->K = K; o->alpha = alpha; o->beta0 = beta0; o->nu0 = nu0; o->seed = seed; o->job = job;
    o->burn_in = burn_in; o->order = order; o->flags = flags; o->clip_lo = clip_lo;
    o->clip_hi = clip_hi; o->nthreads = nthreads > 0 ? nthreads : 1;
    o->mu0 = (double*)malloc(sizeof(double) * K);
    o->W0inv = (double*)malloc(sizeof(double) * K * K);
    double* W0d = (double*)malloc(sizeof(double) * K * K);
    for (int k = 0; k < K; ++k) o->mu0[k] = mu0 ? mu0[k] : 0.0;
    for (int i = 0; i < K * K; ++i) W0d[i] = W0 ? W0[i] : ((i / K == i % K) ? 1.0 : 0.0);
    int rc = orc_spd_inverse(K, W0d, o->W0inv);
    free(W0d);
    if (rc) { orc_destroy(o); return NULL; }

    int64_t nnz = csr_ptr[M];
    double total = 0.0;
    for (int64_t t = 0; t < nnz; ++t) total += (double)csr_val[t];
    o->rbar = (flags & ORC_FLAG_NO_CENTER) || nnz == 0 ? 0.0 : total / (double)nnz;

    int64_t nrows[2] = {M, N};
    for (int s = 0; s < 2; ++s) {
        orc_side* sd = &o->side[s];
        sd->n_rows = nrows[s];
        sd->ptr = (int64_t*)calloc((size_t)nrows[s] + 1, sizeof(int64_t));
        sd->idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
        sd->val = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
        sd->X = (double*)calloc((size_t)nrows[s] * K, sizeof(double));
        sd->mean = (double*)calloc((size_t)nrows[s] * K, sizeof(double));
        sd->mu = (double*)calloc(K, sizeof(double));
        sd->Lambda = (double*)calloc((size_t)K * K, sizeof(double));
        sd->xbar = (double*)calloc(K, sizeof(double));
        sd->S = (double*)calloc((size_t)K * K, sizeof(double));
        if (!sd->ptr || !sd->idx || !sd->val || !sd->X || !sd->mean) { orc_destroy(o); return NULL; }
        for (int k = 0; k < K; ++k) sd->Lambda[k * K + k] = 1.0;
    }
    /* users: the CSR as given */
    for (int64_t i = 0; i <= M; ++i) o->side[0].ptr[i] = csr_ptr[i];
    for (int64_t t = 0; t < nnz; ++t) {
        o->side[0].idx[t] = csr_col[t];
        o->side[0].val[t] = (double)csr_val[t] - o->rbar;
    }
    /* movies: the plain transpose (counting by column, rows in increasing order) */
    orc_side* mv = &o->side[1];
    for (int64_t t = 0; t < nnz; ++t) mv->ptr[csr_col[t] + 1] += 1;
    for (int64_t j = 0; j < N; ++j) mv->ptr[j + 1] += mv->ptr[j];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
    for (int64_t j = 0; j < N; ++j) fill[j] = mv->ptr[j];
    for (int64_t i = 0; i < M; ++i)
        for (int64_t t = csr_ptr[i]; t < csr_ptr[i + 1]; ++t) {
            int64_t p = fill[csr_col[t]]++;
            mv->idx[p] = (int32_t)i;
            mv->val[p] = (double)csr_val[t] - o->rbar;
        }
    free(fill);

    o->T = T;
    o->ti = (int32_t*)malloc(sizeof(int32_t) * (size_t)(T > 0 ? T : 1));
    o->tj = (int32_t*)malloc(sizeof(int32_t) * (size_t)(T > 0 ? T : 1));
    o->tr = (double*)malloc(sizeof(double) * (size_t)(T > 0 ? T : 1));
    o->psum = (double*)calloc((size_t)(T > 0 ? T : 1), sizeof(double));
    for (int64_t t = 0; t < T; ++t) { o->ti[t] = ti[t]; o->tj[t] = tj[t]; o->tr[t] = (double)tr[t]; }

    /* initial factors: N(0,1) from the init streams (tags 0 and 1), sweep field 0 */
    for (int s = 0; s < 2; ++s) {
        orc_side* sd = &o->side[s];
        for (int64_t r = 0; r < sd->n_rows; ++r)
            orc_normal_stream(seed, (uint32_t)r, 0u, c3_of(o, (uint32_t)s), 0, K, sd->X + r * K);
    }
    return o;
}

double orc_rbar(const orc_state* o) { return o->rbar; }
uint32_t orc_get_sweep(const orc_state* o) { return o->sweep; }
int64_t orc_get_navg(const orc_state* o) { return o->n_avg; }
void orc_set_counters(orc_state* o, uint32_t sweep, int64_t n_avg)
{
    o->sweep = sweep;
    o->n_avg = n_avg;
}

/* Hyper step for one side: statistics of its rows, then the NW draw. */
int orc_hyper(orc_state* o, int s)
{
    orc_side* sd = &o->side[s];
    int K = o->K;
    orc_row_stats(sd->n_rows, K, sd->X, sd->xbar, sd->S);
    return orc_nw_draw(K, sd->n_rows, sd->xbar, sd->S, o->beta0, o->nu0, o->mu0, o->W0inv,
                       o->seed, o->sweep, c3_of(o, 4u + (uint32_t)s), c3_of(o, 6u + (uint32_t)s),
                       sd->Lambda, sd->mu);
}

/* NW draw from externally supplied statistics, for the hyper parity check. */
int orc_nw_from_stats(const orc_state* o, int s, int64_t n, const double* xbar, const double* S,
                      uint32_t sweep, double* Lambda, double* mu)
{
    return orc_nw_draw(o->K, n, xbar, S, o->beta0, o->nu0, o->mu0, o->W0inv, o->seed, sweep,
                       c3_of(o, 4u + (uint32_t)s), c3_of(o, 6u + (uint32_t)s), Lambda, mu);
}

typedef struct {
    orc_state* o;
    int s;
    const int64_t* rows; /* NULL: contiguous range */
    int64_t begin, end;
    int rc;
} row_job;

static void* row_worker(void* arg)
{
    row_job* jb = (row_job*)arg;
    orc_state* o = jb->o;
    int K = o->K, s = jb->s;
    orc_side* sd = &o->side[s];
    const orc_side* other = &o->side[1 - s];
    double* work = (double*)malloc(sizeof(double) * (3 * (size_t)K * K + 3 * (size_t)K));
    double* lammu = (double*)malloc(sizeof(double) * K);
    double* z = (double*)malloc(sizeof(double) * K);
    if (!work || !lammu || !z) {
        jb->rc = ORC_ENOMEM;
        free(work); free(lammu); free(z);
        return NULL;
    }
    for (int a = 0; a < K; ++a) {
        double acc = 0.0;
        for (int b = 0; b < K; ++b) acc += sd->Lambda[a * K + b] * sd->mu[b];
        lammu[a] = acc;
    }
    uint32_t c3 = c3_of(o, 2u + (uint32_t)s);
    for (int64_t q = jb->begin; q < jb->end; ++q) {
        int64_t r = jb->rows ? jb->rows[q] : q;
        orc_normal_stream(o->seed, (uint32_t)r, o->sweep, c3, 0, K, z);
        int64_t p0 = sd->ptr[r], p1 = sd->ptr[r + 1];
        int rc = orc_row_conditional(K, sd->Lambda, lammu, o->alpha, p1 - p0, sd->idx + p0,
                                     sd->val + p0, other->X, z, sd->mean + r * K, sd->X + r * K,
                                     work);
        if (rc) { jb->rc = rc; break; }
    }
    free(work); free(lammu); free(z);
    return NULL;
}

static int run_rows(orc_state* o, int s, const int64_t* rows, int64_t count)
{
    int nt = o->nthreads;
    if (count < nt) nt = count > 0 ? (int)count : 1;
    row_job* jobs = (row_job*)calloc((size_t)nt, sizeof(row_job));
    pthread_t* th = (pthread_t*)calloc((size_t)nt, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return ORC_ENOMEM; }
    for (int t = 0; t < nt; ++t) {
        jobs[t].o = o; jobs[t].s = s; jobs[t].rows = rows;
        jobs[t].begin = count * t / nt;
        jobs[t].end = count * (t + 1) / nt;
    }
    for (int t = 1; t < nt; ++t) pthread_create(&th[t], NULL, row_worker, &jobs[t]);
    row_worker(&jobs[0]);
    for (int t = 1; t < nt; ++t) pthread_join(th[t], NULL);
    int rc = ORC_OK;
    for (int t = 0; t < nt; ++t) if (jobs[t].rc) rc = jobs[t].rc;
    free(jobs); free(th);
    return rc;
}

/* Update every row of side s given the other side (one inner loop of Alg. 1). */
int orc_rows(orc_state* o, int s) { return run_rows(o, s, NULL, o->side[s].n_rows); }

/* Update only the listed rows of side s (for sampled checks at large sizes). */
int orc_rows_subset(orc_state* o, int s, const int64_t* rows, int64_t count)
{
    return run_rows(o, s, rows, count);
}

/* Update the contiguous rows [begin, end) of side s (timing samples). */
int orc_rows_range(orc_state* o, int s, int64_t begin, int64_t end)
{
    int nt = o->nthreads;
    int64_t count = end - begin;
    if (count <= 0) return ORC_OK;
    int64_t* rows = (int64_t*)malloc(sizeof(int64_t) * (size_t)count);
    if (!rows) return ORC_ENOMEM;
    for (int64_t q = 0; q < count; ++q) rows[q] = begin + q;
    (void)nt;
    int rc = run_rows(o, s, rows, count);
    free(rows);
    return rc;
}

/*
 * Predict every test point (Alg. 1, last inner loop): p = rbar + u_i . v_j,
 * clipped only when the clip flag is set; RMSE of this sample; running sum of
 * predictions once sweep >= burn_in; RMSE of the running-average prediction.
 */
int orc_predict(orc_state* o, double* rmse_sample, double* rmse_avg)
{
    int K = o->K;
    int accumulate = (int64_t)o->sweep >= (int64_t)o->burn_in;
    if (accumulate) o->n_avg += 1;
    double se = 0.0, sa = 0.0;
    for (int64_t t = 0; t < o->T; ++t) {
        const double* u = o->side[0].X + (size_t)o->ti[t] * K;
        const double* v = o->side[1].X + (size_t)o->tj[t] * K;
        double p = o->rbar;
        for (int k = 0; k < K; ++k) p += u[k] * v[k];
        if (o->flags & ORC_FLAG_CLIP) {
            if (p < o->clip_lo) p = o->clip_lo;
            if (p > o->clip_hi) p = o->clip_hi;
        }
        se += (p - o->tr[t]) * (p - o->tr[t]);
        if (accumulate) o->psum[t] += p;
        if (o->n_avg > 0) {
            double pa = o->psum[t] / (double)o->n_avg;
            sa += (pa - o->tr[t]) * (pa - o->tr[t]);
        }
    }
    double Td = o->T > 0 ? (double)o->T : 1.0;
    if (rmse_sample) *rmse_sample = sqrt(se / Td);
    if (rmse_avg) *rmse_avg = o->n_avg > 0 ? sqrt(sa / Td) : NAN;
    return ORC_OK;
}

/* One or more full sweeps in the order of Alg. 1 (order 0: movies first). */
int orc_sweep(orc_state* o, int n, double* rmse_sample, double* rmse_avg)
{
    for (int it = 0; it < n; ++it) {
        int first = o->order == 0 ? 1 : 0;
        int second = 1 - first;
        int rc = orc_hyper(o, first);
        if (!rc) rc = orc_rows(o, first);
        if (!rc) rc = orc_hyper(o, second);
        if (!rc) rc = orc_rows(o, second);
        if (!rc) rc = orc_predict(o, rmse_sample, rmse_avg);
        if (rc) { o->status = rc; return rc; }
        o->sweep += 1;
    }
    return ORC_OK;
}

/* ---- state access (row-major K columns, FP64) ---- */
void orc_get_factors(const orc_state* o, int s, double* out)
{
    memcpy(out, o->side[s].X, sizeof(double) * (size_t)o->side[s].n_rows * o->K);
}
void orc_set_factors(orc_state* o, int s, const double* in)
{
    memcpy(o->side[s].X, in, sizeof(double) * (size_t)o->side[s].n_rows * o->K);
}
void orc_get_means(const orc_state* o, int s, double* out)
{
    memcpy(out, o->side[s].mean, sizeof(double) * (size_t)o->side[s].n_rows * o->K);
}
void orc_get_hyper(const orc_state* o, int s, double* mu, double* Lambda)
{
    memcpy(mu, o->side[s].mu, sizeof(double) * o->K);
    memcpy(Lambda, o->side[s].Lambda, sizeof(double) * o->K * o->K);
}
void orc_set_hyper(orc_state* o, int s, const double* mu, const double* Lambda)
{
    memcpy(o->side[s].mu, mu, sizeof(double) * o->K);
    memcpy(o->side[s].Lambda, Lambda, sizeof(double) * o->K * o->K);
}
void orc_get_stats(const orc_state* o, int s, double* xbar, double* S)
{
    memcpy(xbar, o->side[s].xbar, sizeof(double) * o->K);
    memcpy(S, o->side[s].S, sizeof(double) * o->K * o->K);
}
void orc_get_psum(const orc_state* o, double* out)
{
    memcpy(out, o->psum, sizeof(double) * (size_t)o->T);
}
void orc_set_psum(orc_state* o, const double* in)
{
    memcpy(o->psum, in, sizeof(double) * (size_t)o->T);
}
