/*
 * Plain C99 FP64 oracle for randomized Gram-Schmidt and RGS-GMRES.
 *
 * TEST INFRASTRUCTURE ONLY: built and called by the tests and by the
 * benchmark's CPU-baseline leg.  The CUDA library never links or calls it.
 *
 * Written from Balabanov & Grigori, "Randomized Gram-Schmidt process with
 * application to GMRES":
 *   - the sketches of Sec. 2.1 (Gaussian; P-SRHT = first n columns of
 *     (1/sqrt(k)) P H_s D), drawn from Philox4x32-10 (Salmon et al., SC'11)
 *     with the stream layout of the library header;
 *   - Alg. 2 (RGS) with the least-squares step solved by an incremental
 *     Householder QR of S (the solver of Sec. 5) or by Richardson sweeps on the
 *     normal equations (Sec. 2.3);
 *   - Alg. 3 (RGS-Arnoldi) and the randomized GMRES of Eq. hls, with the
 *     Hessenberg problem reduced by Givens rotations (Sec. 4.2, 5.3);
 *   - restarted FP64 GMRES with a CGS2 Arnoldi basis (Sec. 1.2) as comparator.
 * Loops are plain and unblocked so they can be read against the paper.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

/* ---------------- Philox4x32-10 (published definition) ---------------- */
static void philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void orc_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox(ctr, key, out); }

static double u53(uint32_t hi, uint32_t lo) {
    uint64_t v = (((uint64_t)hi << 32) | lo) >> 11;
    return ((double)v + 0.5) * 0x1p-53;
}

/* ---------------- sketches ---------------- */
typedef struct {
    int kind;            /* 0 Gaussian, 1 SRHT */
    int64_t n, s;
    int k;
    uint64_t seed;
    double* theta;       /* Gaussian: k x n column-major */
    double* signs;       /* SRHT: n */
    int64_t* rows;       /* SRHT: k ascending */
    double* work;        /* SRHT: s */
} orc_sketch;

typedef struct { uint64_t key; int64_t idx; } keyidx;

static int cmp_keyidx(const void* a, const void* b) {
    const keyidx* x = (const keyidx*)a;
    const keyidx* y = (const keyidx*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static int cmp_i64(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return x < y ? -1 : (x > y);
}

orc_sketch* orc_sketch_new(int kind, int64_t n, int k, uint64_t seed) {
    orc_sketch* sk = (orc_sketch*)calloc(1, sizeof(orc_sketch));
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    sk->kind = kind; sk->n = n; sk->k = k; sk->seed = seed;
    sk->s = 1;
    while (sk->s < n) sk->s *= 2;
    if (kind == 0) {
        sk->theta = (double*)malloc(sizeof(double) * (size_t)k * (size_t)n);
        double scale = 1.0 / sqrt((double)k);
        for (int64_t c = 0; c < n; ++c) {
            for (int l = 0; l < k; l += 2) {
                uint32_t ctr[4] = {(uint32_t)c, (uint32_t)(l >> 1), 0u, 0u}, x[4];
                philox(ctr, key, x);
                double u1 = u53(x[0], x[1]), u2 = u53(x[2], x[3]);
                double rad = sqrt(-2.0 * log(u1));
                double ang = 2.0 * M_PI * u2;
                sk->theta[(size_t)c * k + l] = rad * cos(ang) * scale;
                if (l + 1 < k) sk->theta[(size_t)c * k + l + 1] = rad * sin(ang) * scale;
            }
        }
    } else {
        if (k > sk->s) { free(sk); return NULL; }
        sk->signs = (double*)malloc(sizeof(double) * (size_t)n);
        for (int64_t c = 0; c < n; ++c) {
            uint32_t ctr[4] = {(uint32_t)(c >> 7), 0u, 0u, 1u}, x[4];
            philox(ctr, key, x);
            uint32_t word = x[(c & 127) >> 5];
            sk->signs[c] = ((word >> (c & 31)) & 1u) ? -1.0 : 1.0;
        }
        keyidx* all = (keyidx*)malloc(sizeof(keyidx) * (size_t)sk->s);
        for (int64_t c = 0; c < sk->s; ++c) {
            uint32_t ctr[4] = {(uint32_t)c, 0u, 0u, 2u}, x[4];
            philox(ctr, key, x);
            all[c].key = ((uint64_t)x[0] << 32) | x[1];
            all[c].idx = c;
        }
        qsort(all, (size_t)sk->s, sizeof(keyidx), cmp_keyidx);
        sk->rows = (int64_t*)malloc(sizeof(int64_t) * (size_t)k);
        for (int j = 0; j < k; ++j) sk->rows[j] = all[j].idx;
        qsort(sk->rows, (size_t)k, sizeof(int64_t), cmp_i64);
        free(all);
        sk->work = (double*)malloc(sizeof(double) * (size_t)sk->s);
    }
    return sk;
}

void orc_sketch_free(orc_sketch* sk) {
    if (!sk) return;
    free(sk->theta); free(sk->signs); free(sk->rows); free(sk->work); free(sk);
}

const int64_t* orc_sketch_rows(const orc_sketch* sk) { return sk->rows; }
const double* orc_sketch_signs(const orc_sketch* sk) { return sk->signs; }
const double* orc_sketch_theta(const orc_sketch* sk) { return sk->theta; }

/* y (k) = Theta x (n) */
void orc_sketch_apply(orc_sketch* sk, const double* x, double* y) {
    if (sk->kind == 0) {
        for (int l = 0; l < sk->k; ++l) y[l] = 0.0;
        for (int64_t c = 0; c < sk->n; ++c) {
            const double* col = sk->theta + (size_t)c * sk->k;
            double xc = x[c];
            for (int l = 0; l < sk->k; ++l) y[l] += col[l] * xc;
        }
        return;
    }
    double* z = sk->work;
    const int64_t s = sk->s;
#pragma omp parallel for schedule(static) if (s >= 65536)
    for (int64_t c = 0; c < s; ++c) z[c] = c < sk->n ? sk->signs[c] * x[c] : 0.0;
    /* stage h: the butterflies (b, b + h) for b with bit h clear; they are independent, so a
     * stage may be split across threads without changing any sum */
    for (int64_t h = 1; h < s; h *= 2) {
#pragma omp parallel for schedule(static) if (s >= 65536)
        for (int64_t t = 0; t < s / 2; ++t) {
            const int64_t b = (t / h) * 2 * h + t % h;
            double u = z[b], v = z[b + h];
            z[b] = u + v;
            z[b + h] = u - v;
        }
    }
    double scale = 1.0 / sqrt((double)sk->k);
    for (int j = 0; j < sk->k; ++j) y[j] = z[sk->rows[j]] * scale;
}

/* Threads of the parallel loops (0 or less: leave the OpenMP default); returns the count in use,
 * 1 without OpenMP.  Only loops over independent rows or butterflies run in parallel, so every
 * result is the same for any thread count. */
int orc_set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* ---------------- precision emulation ---------------- */
static double round_bf16(double v) {
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    uint32_t lsb = (u >> 16) & 1u;
    u = (u + 0x7FFFu + lsb) & 0xFFFF0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

static double round_storage(double v, int storage) {
    if (storage == 0) return v;
    if (storage == 1) return (double)(float)v;
    return round_bf16(v);
}

/* acc - c q for FP32 values acc, c, q, rounded once to FP32 as one fused multiply-add does.
 * c q is exact in FP64 (48 significant bits at most).  s = fl64(acc - c q) and its rounding
 * error e (Knuth's TwoSum) hold the exact difference s + e.  Every FP32 rounding boundary is
 * an FP64 number, so none lies strictly between s + e and s: s rounds to the right FP32 value
 * unless s sits exactly on a boundary (halfway between two FP32 neighbours), where e decides;
 * e = 0 there is a true tie, which the conversion resolves to even. */
static double fma32_once(double acc, double c, double q) {
    double prod = c * q;
    double s = acc - prod;
    double bb = s - acc;
    double e = (acc - (s - bb)) + (-prod - bb);
    float r = (float)s;
    if (e != 0.0 && (double)r != s) {
        float other = nextafterf(r, s > (double)r ? INFINITY : -INFINITY);
        if (0.5 * ((double)r + (double)other) == s && ((e > 0.0) == ((double)other > (double)r))) r = other;
    }
    return (double)r;
}

/* Step 3 in FP32 for rows [0, n): out = fl32(w) - sum_j fl32(c_j) Qp(:, j), one fused
 * multiply-add per term in column order.  Exported for the tests of the emulation. */
void orc_update_fp32(int64_t n, int ncols, const double* w, const double* Qp, int64_t ldq, const double* c,
                     double* out) {
    for (int64_t r = 0; r < n; ++r) {
        double acc = (double)(float)w[r];
        for (int j = 0; j < ncols; ++j) acc = fma32_once(acc, (double)(float)c[j], Qp[(size_t)j * ldq + r]);
        out[r] = acc;
    }
}

/* ---------------- incremental Householder QR of S (k x cols) ---------------- */
typedef struct {
    int k, mmax, cols;
    double* V;    /* k x mmax, reflector j has V[j] = 1 implied, entries l > j stored */
    double* tau;  /* mmax */
    double* Rs;   /* mmax x mmax upper triangular */
} householder;

static void hh_init(householder* h, int k, int mmax) {
    h->k = k; h->mmax = mmax; h->cols = 0;
    h->V = (double*)calloc((size_t)k * mmax, sizeof(double));
    h->tau = (double*)calloc((size_t)mmax, sizeof(double));
    h->Rs = (double*)calloc((size_t)mmax * mmax, sizeof(double));
}

static void hh_free(householder* h) { free(h->V); free(h->tau); free(h->Rs); }

/* y <- H_{cols-1} ... H_0 y */
static void hh_apply(const householder* h, double* y) {
    for (int j = 0; j < h->cols; ++j) {
        const double* v = h->V + (size_t)j * h->k;
        double t = y[j];
        for (int l = j + 1; l < h->k; ++l) t += v[l] * y[l];
        t *= h->tau[j];
        y[j] -= t;
        for (int l = j + 1; l < h->k; ++l) y[l] -= t * v[l];
    }
}

/* x (cols) = argmin || S x - p ||, using work (k) */
static void hh_solve(const householder* h, const double* p, double* x, double* work) {
    memcpy(work, p, sizeof(double) * (size_t)h->k);
    hh_apply(h, work);
    for (int r = h->cols - 1; r >= 0; --r) {
        double t = work[r];
        for (int c = r + 1; c < h->cols; ++c) t -= h->Rs[(size_t)c * h->mmax + r] * x[c];
        x[r] = t / h->Rs[(size_t)r * h->mmax + r];
    }
}

/* append column s (k) to the factorisation */
static void hh_append(householder* h, const double* s, double* work) {
    int i = h->cols, k = h->k;
    memcpy(work, s, sizeof(double) * (size_t)k);
    hh_apply(h, work);
    double alpha = work[i], sig = 0.0;
    for (int l = i + 1; l < k; ++l) sig += work[l] * work[l];
    double* v = h->V + (size_t)i * k;
    double beta, tau;
    if (sig == 0.0) {
        beta = alpha; tau = 0.0;
    } else {
        double nrm = sqrt(alpha * alpha + sig);
        beta = alpha >= 0.0 ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        double sc = 1.0 / (alpha - beta);
        for (int l = i + 1; l < k; ++l) v[l] = work[l] * sc;
    }
    v[i] = 1.0;
    h->tau[i] = tau;
    for (int r = 0; r < i; ++r) h->Rs[(size_t)i * h->mmax + r] = work[r];
    h->Rs[(size_t)i * h->mmax + i] = beta;
    h->cols = i + 1;
}

/* Richardson sweeps on the normal equations: x <- x + S^T (p - S x), x0 = 0 */
static void richardson_solve(const double* S, int k, int cols, const double* p, int sweeps,
                             double* x, double* work) {
    for (int c = 0; c < cols; ++c) x[c] = 0.0;
    for (int it = 0; it < sweeps; ++it) {
        for (int l = 0; l < k; ++l) work[l] = p[l];
        for (int c = 0; c < cols; ++c)
            for (int l = 0; l < k; ++l) work[l] -= S[(size_t)c * k + l] * x[c];
        for (int c = 0; c < cols; ++c) {
            double t = 0.0;
            for (int l = 0; l < k; ++l) t += S[(size_t)c * k + l] * work[l];
            x[c] += t;
        }
    }
}

/* ---------------- one RGS iteration (Alg. 2, steps 2-7) ---------------- */
typedef struct {
    int64_t n;
    int k, mmax, ls, sweeps, storage;
    double* Qp;      /* n x mmax stored q' */
    double* sigma;   /* 1 / r_ii */
    double* S;       /* k x mmax */
    householder hh;
    double* work;    /* k */
    double* x;       /* mmax */
    double* sp;      /* k */
    double* qp;      /* n */
} rgs_state;

static void rgs_init(rgs_state* st, int64_t n, int k, int mmax, int ls, int sweeps, int storage,
                     double* Qp, double* sigma, double* S) {
    st->n = n; st->k = k; st->mmax = mmax; st->ls = ls; st->sweeps = sweeps; st->storage = storage;
    st->Qp = Qp; st->sigma = sigma; st->S = S;
    hh_init(&st->hh, k, mmax);
    st->work = (double*)malloc(sizeof(double) * (size_t)k);
    st->x = (double*)malloc(sizeof(double) * (size_t)mmax);
    st->sp = (double*)malloc(sizeof(double) * (size_t)k);
    st->qp = (double*)malloc(sizeof(double) * (size_t)n);
}

static void rgs_free(rgs_state* st) {
    hh_free(&st->hh); free(st->work); free(st->x); free(st->sp); free(st->qp);
}

/* Iteration i (0-based) on column w with sketch p = Theta w.  Writes R column i
 * (i+1 entries) into rcol.  Returns 0, or 1 on breakdown (column not appended). */
static int rgs_step(rgs_state* st, orc_sketch* sk, int i, const double* w, const double* p, double* rcol) {
    int64_t n = st->n;
    int k = st->k;
    /* step 2 */
    if (i > 0) {
        if (st->ls == 0) hh_solve(&st->hh, p, st->x, st->work);
        else richardson_solve(st->S, k, i, p, st->sweeps, st->x, st->work);
    }
    /* step 3 (rows are independent) */
    if (st->storage == 0) {
#pragma omp parallel for schedule(static) if (n >= 65536)
        for (int64_t r = 0; r < n; ++r) {
            double acc = w[r];
            for (int j = 0; j < i; ++j) acc -= st->Qp[(size_t)j * n + r] * (st->x[j] * st->sigma[j]);
            st->qp[r] = acc;
        }
    } else {
#pragma omp parallel for schedule(static) if (n >= 65536)
        for (int64_t r = 0; r < n; ++r) {
            double acc = (double)(float)w[r];
            for (int j = 0; j < i; ++j) {
                double c = (double)(float)(st->x[j] * st->sigma[j]);
                acc = fma32_once(acc, c, st->Qp[(size_t)j * n + r]);
            }
            st->qp[r] = round_storage(acc, st->storage);
        }
    }
    /* step 4, 5 */
    orc_sketch_apply(sk, st->qp, st->sp);
    double rr = 0.0, pp = 0.0;
    for (int l = 0; l < k; ++l) { rr += st->sp[l] * st->sp[l]; pp += p[l] * p[l]; }
    rr = sqrt(rr);
    for (int j = 0; j < i; ++j) rcol[j] = st->x[j];
    rcol[i] = rr;
    if (!(rr > 16.0 * 0x1p-53 * sqrt(pp))) return 1;
    /* steps 6, 7 */
    double* s = st->S + (size_t)i * k;
    for (int l = 0; l < k; ++l) s[l] = st->sp[l] / rr;
    memcpy(st->Qp + (size_t)i * n, st->qp, sizeof(double) * (size_t)n);
    st->sigma[i] = 1.0 / rr;
    if (st->ls == 0) hh_append(&st->hh, s, st->work);
    return 0;
}

/* Alg. 2.  W n x m column-major (ldw).  Outputs: Qp (n x m), sigma (m), R (m x m, col-major),
 * S (k x m), P (k x m), certs[2] = {Delta_m, Delta~_m}.  Returns 0, or 1 + column on breakdown. */
int orc_rgs_qr(orc_sketch* sk, int64_t n, int m, const double* W, int64_t ldw, int ls, int sweeps,
               int storage, double* Qp, double* sigma, double* R, double* S, double* P, double* certs) {
    int k = sk->k;
    if (m > k || n != sk->n) return -1;
    rgs_state st;
    rgs_init(&st, n, k, m, ls, sweeps, storage, Qp, sigma, S);
    memset(R, 0, sizeof(double) * (size_t)m * m);
    int status = 0;
    for (int i = 0; i < m; ++i) {
        const double* w = W + (size_t)i * ldw;
        orc_sketch_apply(sk, w, P + (size_t)i * k);                 /* step 1 */
        if (rgs_step(&st, sk, i, w, P + (size_t)i * k, R + (size_t)i * m)) { status = 1 + i; break; }
    }
    if (status == 0) {
        double d = 0.0, dt = 0.0, pn = 0.0;
        for (int a = 0; a < m; ++a)
            for (int b = 0; b < m; ++b) {
                double g = 0.0;
                for (int l = 0; l < k; ++l) g += S[(size_t)a * k + l] * S[(size_t)b * k + l];
                double e = (a == b ? 1.0 : 0.0) - g;
                d += e * e;
            }
        for (int c = 0; c < m; ++c)
            for (int l = 0; l < k; ++l) {
                double v = P[(size_t)c * k + l];
                for (int j = 0; j <= c; ++j) v -= S[(size_t)j * k + l] * R[(size_t)c * m + j];
                dt += v * v;
                pn += P[(size_t)c * k + l] * P[(size_t)c * k + l];
            }
        certs[0] = sqrt(d);
        certs[1] = sqrt(dt / pn);
    }
    rgs_free(&st);
    return status;
}

/* ---------------- CSR product y = A x (FP64) ---------------- */
static void csr_mv(int64_t n, const int32_t* rowptr, const int32_t* colind, const double* val,
                   const double* x, double* y) {
    for (int64_t r = 0; r < n; ++r) {
        double t = 0.0;
        for (int32_t e = rowptr[r]; e < rowptr[r + 1]; ++e) t += val[e] * x[colind[e]];
        y[r] = t;
    }
}

/* Givens rotation zeroing b in (a, b) */
static void givens(double a, double b, double* c, double* s, double* r) {
    double d = hypot(a, b);
    if (d == 0.0) { *c = 1.0; *s = 0.0; *r = 0.0; return; }
    *c = a / d; *s = b / d; *r = d;
}

/* Apply rotations 0..j-1 to column h (j+2 entries), then a new rotation j; update g. */
static double hess_column(double* h, int j, double* cs, double* sn, double* g) {
    for (int t = 0; t < j; ++t) {
        double a = h[t], b = h[t + 1];
        h[t] = cs[t] * a + sn[t] * b;
        h[t + 1] = -sn[t] * a + cs[t] * b;
    }
    double r;
    givens(h[j], h[j + 1], &cs[j], &sn[j], &r);
    h[j] = r;
    h[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    return fabs(g[j + 1]);
}

/* Upper-triangular solve of the rotated Hessenberg (column-major, ld) for y (j entries). */
static void hess_solve(const double* Hr, int ld, int j, const double* g, double* y) {
    for (int r = j - 1; r >= 0; --r) {
        double t = g[r];
        for (int c = r + 1; c < j; ++c) t -= Hr[(size_t)c * ld + r] * y[c];
        y[r] = t / Hr[(size_t)r * ld + r];
    }
}

static double nrm2(int64_t n, const double* v) {
    double t = 0.0;
    for (int64_t r = 0; r < n; ++r) t += v[r] * v[r];
    return sqrt(t);
}

/* Restarted RGS-GMRES (Alg. 3 + Eq. hls + FP64 restart residual).
 * info[0] = cycles, info[1] = total Arnoldi steps; res_hist receives the relative
 * true residual after each cycle (max_cycles + 1 entries).  Returns 0 if converged. */
int orc_rgmres(orc_sketch* sk, int64_t n, const int32_t* rowptr, const int32_t* colind,
               const double* val, const double* b, double* x, int restart, double tol,
               int max_cycles, int ls, int sweeps, int storage, int fixed_steps,
               double inner_factor, int* info, double* res_hist) {
    int k = sk->k, mcols = restart + 1;
    double* Qp = (double*)malloc(sizeof(double) * (size_t)n * mcols);
    double* sigma = (double*)malloc(sizeof(double) * (size_t)mcols);
    double* S = (double*)malloc(sizeof(double) * (size_t)k * mcols);
    double* Rcol = (double*)malloc(sizeof(double) * (size_t)mcols);
    double* H = (double*)calloc((size_t)(mcols + 1) * mcols, sizeof(double));
    double* cs = (double*)malloc(sizeof(double) * (size_t)mcols);
    double* sn = (double*)malloc(sizeof(double) * (size_t)mcols);
    double* g = (double*)malloc(sizeof(double) * (size_t)(mcols + 1));
    double* y = (double*)malloc(sizeof(double) * (size_t)mcols);
    double* w = (double*)malloc(sizeof(double) * (size_t)n);
    double* q = (double*)malloc(sizeof(double) * (size_t)n);
    double* p = (double*)malloc(sizeof(double) * (size_t)k);
    double bn = nrm2(n, b);
    orc_sketch_apply(sk, b, p);
    double sb = nrm2(k, p);
    csr_mv(n, rowptr, colind, val, x, w);
    for (int64_t r = 0; r < n; ++r) w[r] = b[r] - w[r];
    double rel = nrm2(n, w) / bn;
    res_hist[0] = rel;
    int cycles = 0, total = 0;
    double thr = inner_factor * tol * sb;   /* inner threshold, tightened after a short cycle */
    while (!(rel <= tol) && cycles < max_cycles) {
        rgs_state st;
        rgs_init(&st, n, k, mcols, ls, sweeps, storage, Qp, sigma, S);
        int j = 0;
        for (int i = 0; i < mcols; ++i) {
            if (i > 0) {
                const double* qp = Qp + (size_t)(i - 1) * n;
                for (int64_t r = 0; r < n; ++r) q[r] = qp[r] * sigma[i - 1];
                csr_mv(n, rowptr, colind, val, q, w);          /* Alg. 3 step 3 */
            }
            orc_sketch_apply(sk, w, p);                         /* Alg. 2 step 1 */
            int bd = rgs_step(&st, sk, i, w, p, Rcol);
            if (i == 0) {
                if (bd) break;
                g[0] = Rcol[0];
                continue;
            }
            double* h = H + (size_t)(i - 1) * (mcols + 1);
            for (int r = 0; r <= i; ++r) h[r] = Rcol[r];     /* H(:, i-1) = R(1:i+1, i+1) */
            double rho = hess_column(h, i - 1, cs, sn, g);
            j = i;
            if (bd) break;                                     /* invariant subspace */
            if (!fixed_steps && rho <= thr) break;
        }
        rgs_free(&st);
        if (j == 0) break;
        hess_solve(H, mcols + 1, j, g, y);
        for (int64_t r = 0; r < n; ++r) {
            double t = 0.0;
            for (int c = 0; c < j; ++c) t += Qp[(size_t)c * n + r] * (sigma[c] * y[c]);
            x[r] += t;
        }
        csr_mv(n, rowptr, colind, val, x, w);
        for (int64_t r = 0; r < n; ++r) w[r] = b[r] - w[r];
        rel = nrm2(n, w) / bn;
        cycles++;
        total += j;
        res_hist[cycles] = rel;
        if (!(rel <= tol) && j < restart) thr *= fmin(1.0, inner_factor * tol / rel);
    }
    info[0] = cycles;
    info[1] = total;
    free(Qp); free(sigma); free(S); free(Rcol); free(H); free(cs); free(sn); free(g); free(y);
    free(w); free(q); free(p);
    return rel <= tol ? 0 : 1;
}

/* Restarted FP64 GMRES with a CGS2 Arnoldi basis (projector (I - V V^T)^2). */
int orc_cgs2_gmres(int64_t n, const int32_t* rowptr, const int32_t* colind, const double* val,
                   const double* b, double* x, int restart, double tol, int max_cycles,
                   int fixed_steps, double inner_factor, int* info, double* res_hist) {
    int mcols = restart + 1;
    double* V = (double*)malloc(sizeof(double) * (size_t)n * mcols);
    double* H = (double*)calloc((size_t)(mcols + 1) * mcols, sizeof(double));
    double* cs = (double*)malloc(sizeof(double) * (size_t)mcols);
    double* sn = (double*)malloc(sizeof(double) * (size_t)mcols);
    double* g = (double*)malloc(sizeof(double) * (size_t)(mcols + 1));
    double* y = (double*)malloc(sizeof(double) * (size_t)mcols);
    double* h2 = (double*)malloc(sizeof(double) * (size_t)mcols);
    double* w = (double*)malloc(sizeof(double) * (size_t)n);
    double bn = nrm2(n, b);
    csr_mv(n, rowptr, colind, val, x, w);
    for (int64_t r = 0; r < n; ++r) w[r] = b[r] - w[r];
    double rel = nrm2(n, w) / bn;
    res_hist[0] = rel;
    int cycles = 0, total = 0;
    double thr = inner_factor * tol * bn;   /* inner threshold, tightened after a short cycle */
    while (!(rel <= tol) && cycles < max_cycles) {
        double beta = nrm2(n, w);
        for (int64_t r = 0; r < n; ++r) V[r] = w[r] / beta;
        g[0] = beta;
        int j = 0;
        for (int i = 0; i < restart; ++i) {
            csr_mv(n, rowptr, colind, val, V + (size_t)i * n, w);
            double* h = H + (size_t)i * (mcols + 1);
            for (int pass = 0; pass < 2; ++pass) {
                for (int c = 0; c <= i; ++c) {
                    double t = 0.0;
                    const double* v = V + (size_t)c * n;
                    for (int64_t r = 0; r < n; ++r) t += v[r] * w[r];
                    h2[c] = t;
                }
                for (int c = 0; c <= i; ++c) {
                    const double* v = V + (size_t)c * n;
                    for (int64_t r = 0; r < n; ++r) w[r] -= h2[c] * v[r];
                    h[c] = pass == 0 ? h2[c] : h[c] + h2[c];
                }
            }
            double hn = nrm2(n, w);
            h[i + 1] = hn;
            double hmax = 0.0;
            for (int c = 0; c <= i; ++c) hmax = fmax(hmax, fabs(h[c]));
            double rho = hess_column(h, i, cs, sn, g);
            j = i + 1;
            if (!(hn > 16.0 * 0x1p-53 * hmax)) break;
            for (int64_t r = 0; r < n; ++r) V[(size_t)(i + 1) * n + r] = w[r] / hn;
            if (!fixed_steps && rho <= thr) break;
        }
        hess_solve(H, mcols + 1, j, g, y);
        for (int64_t r = 0; r < n; ++r) {
            double t = 0.0;
            for (int c = 0; c < j; ++c) t += V[(size_t)c * n + r] * y[c];
            x[r] += t;
        }
        csr_mv(n, rowptr, colind, val, x, w);
        for (int64_t r = 0; r < n; ++r) w[r] = b[r] - w[r];
        rel = nrm2(n, w) / bn;
        cycles++;
        total += j;
        res_hist[cycles] = rel;
        if (!(rel <= tol) && j < restart) thr *= fmin(1.0, inner_factor * tol / rel);
    }
    info[0] = cycles;
    info[1] = total;
    free(V); free(H); free(cs); free(sn); free(g); free(y); free(h2); free(w);
    return rel <= tol ? 0 : 1;
}
