/*
 * _gen.c -- fast seeded generator of sparse rating patterns and planted scores.
 *
 * Input generation only: nothing here computes any step of the sampler.  Each
 * row draws its own distinct column set with probability proportional to the
 * column weights, from a private xoshiro256** stream seeded through SplitMix64
 * from (seed, row), so the output does not depend on the thread count.
 *
 *   rows with d <= big * N : Walker/Vose alias draws, duplicates rejected
 *   rows with d >  big * N : the d smallest exponential-race keys E_j / w_j
 *                            (weighted sampling without replacement,
 *                             Efraimidis and Spirakis 2006)
 * Columns inside a row are returned in increasing order.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static uint64_t splitmix64(uint64_t* s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } xo_t;

static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t xo_next(xo_t* r)
{
    uint64_t* s = r->s;
    uint64_t out = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return out;
}

static double xo_unit(xo_t* r) { return (double)(xo_next(r) >> 11) * 0x1p-53; }

static void xo_seed(xo_t* r, uint64_t seed, uint64_t stream)
{
    uint64_t s = seed ^ (stream * 0xD1B54A32D192ED03ull);
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&s);
}

typedef struct {
    int64_t N;
    double* prob;
    int64_t* alias;
} alias_t;

static int alias_build(alias_t* a, const double* w, int64_t N)
{
    a->N = N;
    a->prob = (double*)malloc(sizeof(double) * N);
    a->alias = (int64_t*)malloc(sizeof(int64_t) * N);
    int64_t* small = (int64_t*)malloc(sizeof(int64_t) * N);
    int64_t* large = (int64_t*)malloc(sizeof(int64_t) * N);
    double* q = (double*)malloc(sizeof(double) * N);
    if (!a->prob || !a->alias || !small || !large || !q) return -1;
    double tot = 0.0;
    for (int64_t j = 0; j < N; ++j) tot += w[j];
    int64_t ns = 0, nl = 0;
    for (int64_t j = 0; j < N; ++j) {
        q[j] = w[j] * (double)N / tot;
        if (q[j] < 1.0) small[ns++] = j; else large[nl++] = j;
    }
    while (ns > 0 && nl > 0) {
        int64_t s = small[--ns], l = large[--nl];
        a->prob[s] = q[s];
        a->alias[s] = l;
        q[l] = (q[l] + q[s]) - 1.0;
        if (q[l] < 1.0) small[ns++] = l; else large[nl++] = l;
    }
    while (nl > 0) { int64_t l = large[--nl]; a->prob[l] = 1.0; a->alias[l] = l; }
    while (ns > 0) { int64_t s = small[--ns]; a->prob[s] = 1.0; a->alias[s] = s; }
    free(small); free(large); free(q);
    return 0;
}

static int64_t alias_draw(const alias_t* a, xo_t* r)
{
    double u = xo_unit(r) * (double)a->N;
    int64_t j = (int64_t)u;
    if (j >= a->N) j = a->N - 1;
    return (u - (double)j) < a->prob[j] ? j : a->alias[j];
}

static int cmp_i32(const void* x, const void* y)
{
    int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
    return (a > b) - (a < b);
}

typedef struct { double key; int32_t j; } kj_t;

static int cmp_kj(const void* x, const void* y)
{
    double a = ((const kj_t*)x)->key, b = ((const kj_t*)y)->key;
    return (a > b) - (a < b);
}

/* select the d smallest keys (quickselect on kj[0..n)) */
static void select_smallest(kj_t* v, int64_t n, int64_t d, xo_t* r)
{
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        int64_t pi = lo + (int64_t)(xo_unit(r) * (double)(hi - lo + 1));
        if (pi > hi) pi = hi;
        double pv = v[pi].key;
        int64_t i = lo, j = hi;
        while (i <= j) {
            while (v[i].key < pv) ++i;
            while (v[j].key > pv) --j;
            if (i <= j) { kj_t t = v[i]; v[i] = v[j]; v[j] = t; ++i; --j; }
        }
        if (d - 1 <= j) hi = j;
        else if (d - 1 >= i) lo = i;
        else break;
    }
}

typedef struct {
    int64_t r0, r1, N;
    const int64_t* deg;
    const int64_t* ptr;
    const double* w;
    const alias_t* al;
    double big;
    uint64_t seed;
    int32_t* out;
} gen_job;

static void* gen_worker(void* arg)
{
    gen_job* g = (gen_job*)arg;
    int64_t N = g->N;
    uint8_t* mark = (uint8_t*)calloc((size_t)N, 1);
    kj_t* kj = (kj_t*)malloc(sizeof(kj_t) * (size_t)N);
    for (int64_t i = g->r0; i < g->r1; ++i) {
        xo_t r;
        xo_seed(&r, g->seed, (uint64_t)i);
        int64_t d = g->deg[i] < N ? g->deg[i] : N;
        int32_t* o = g->out + g->ptr[i];
        if (d <= 0) continue;
        if ((double)d > g->big * (double)N) {
            for (int64_t j = 0; j < N; ++j) {
                double u = 1.0 - xo_unit(&r);
                kj[j].key = g->w[j] > 0.0 ? -log(u) / g->w[j] : INFINITY;
                kj[j].j = (int32_t)j;
            }
            if (d < N) select_smallest(kj, N, d, &r);
            for (int64_t t = 0; t < d; ++t) o[t] = kj[t].j;
        } else {
            int64_t have = 0;
            while (have < d) {
                int64_t j = alias_draw(g->al, &r);
                if (!mark[j]) { mark[j] = 1; o[have++] = (int32_t)j; }
            }
            for (int64_t t = 0; t < d; ++t) mark[o[t]] = 0;
        }
        qsort(o, (size_t)d, sizeof(int32_t), cmp_i32);
    }
    free(mark); free(kj);
    (void)cmp_kj;
    return NULL;
}

/* ptr[i+1]-ptr[i] must equal min(deg[i], N).  Returns 0 on success. */
int gen_columns(int64_t M, int64_t N, const int64_t* deg, const int64_t* ptr, const double* w,
                double big, uint64_t seed, int nthreads, int32_t* out)
{
    alias_t al;
    if (alias_build(&al, w, N)) return -1;
    if (nthreads < 1) nthreads = 1;
    gen_job* jobs = (gen_job*)calloc((size_t)nthreads, sizeof(gen_job));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (gen_job){M * t / nthreads, M * (t + 1) / nthreads, N, deg, ptr, w, &al, big,
                            seed, out};
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, gen_worker, &jobs[t]);
    gen_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(jobs); free(th); free(al.prob); free(al.alias);
    return 0;
}

typedef struct {
    int64_t a, b, K;
    const int64_t* ptr;
    const int32_t* col;
    const double* U;
    const double* V;
    double* out;
    int64_t M;
} dot_job;

static void* dot_worker(void* arg)
{
    dot_job* g = (dot_job*)arg;
    for (int64_t i = g->a; i < g->b; ++i) {
        const double* u = g->U + i * g->K;
        for (int64_t t = g->ptr[i]; t < g->ptr[i + 1]; ++t) {
            const double* v = g->V + (int64_t)g->col[t] * g->K;
            double s = 0.0;
            for (int64_t k = 0; k < g->K; ++k) s += u[k] * v[k];
            g->out[t] = s;
        }
    }
    return NULL;
}

/* Planted score u_i . v_j for every stored (i, j) of a CSR pattern. */
void gen_planted_scores(int64_t M, int64_t K, const int64_t* ptr, const int32_t* col,
                        const double* U, const double* V, int nthreads, double* out)
{
    if (nthreads < 1) nthreads = 1;
    dot_job* jobs = (dot_job*)calloc((size_t)nthreads, sizeof(dot_job));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; ++t)
        jobs[t] = (dot_job){M * t / nthreads, M * (t + 1) / nthreads, K, ptr, col, U, V, out, M};
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, dot_worker, &jobs[t]);
    dot_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(jobs); free(th);
}
