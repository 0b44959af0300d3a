/*
 * CPU oracle for the k-mismatch FM-index search of MICA's BWT phase.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA library and is deliberately plain and slow.
 *
 * What it computes (MICA, Section 2: each read is first placed with "few
 * mismatches" by searching a BWT index of the reference genome; indels are
 * left to a later dynamic-programming phase and are not modelled here):
 *
 *   H(R) = { (p, +, d) : d = Ham(R,     G[p, p+m)) <= k }
 *        u { (p, -, d) : d = Ham(rc(R), G[p, p+m)) <= k },   0 <= p <= N-m
 *
 * computed two independent ways:
 *   - oracle_align: suffix array of T = G$ ($ smallest), BWT, C[] and Occ as
 *     plain arrays, and the textbook recursive backward search that allows a
 *     substitution at each step while the budget lasts; positions read from
 *     the full suffix array;
 *   - oracle_bruteforce: the Hamming scan of every window of both strands.
 *
 * Hit cap (a reading: the paper has no cap; the workloads ask for an exact
 * total with at most `cap` reported positions): when the total exceeds cap,
 * the reported rows are the first `cap` in the order (mismatches ascending,
 * + strand before -, suffix-array row ascending); the reported hits are then
 * sorted by (position, strand, mismatches).
 *
 * Parity pins for every function live in tests/test_oracle_*.py.
 */
#define _GNU_SOURCE   /* qsort_r */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define EMPTY UINT32_MAX

/* ------------------------------------------------------------------------ */
/* Suffix array of T = G$ by sorting suffixes (the definition).             */
/* ------------------------------------------------------------------------ */

typedef struct { const uint8_t *t; uint64_t len; } suffix_ctx;

/* Compare two suffixes of t (symbols 0 = $, 1..4 = A..T); $ appears once,
   at the end, so two distinct suffixes always differ within the shorter. */
static int cmp_suffix(const void *pa, const void *pb, void *vctx)
{
    const suffix_ctx *c = (const suffix_ctx *)vctx;
    uint64_t a = *(const uint32_t *)pa, b = *(const uint32_t *)pb;
    uint64_t la = c->len - a, lb = c->len - b;
    uint64_t l = la < lb ? la : lb;
    int r = memcmp(c->t + a, c->t + b, l);
    if (r) return r;
    return la < lb ? -1 : (la > lb ? 1 : 0);
}

/* genome codes 0..3 -> text symbols 1..4 with $ = 0 appended */
static uint8_t *make_text(const uint8_t *g, uint64_t n)
{
    uint8_t *t = (uint8_t *)malloc(n + 1);
    if (!t) return NULL;
    for (uint64_t i = 0; i < n; i++) t[i] = (uint8_t)(g[i] + 1);
    t[n] = 0;
    return t;
}

int oracle_sa_sort(const uint8_t *g, uint64_t n, uint32_t *sa)
{
    uint8_t *t = make_text(g, n);
    if (!t) return -1;
    for (uint64_t i = 0; i <= n; i++) sa[i] = (uint32_t)i;
    suffix_ctx c = { t, n + 1 };
    qsort_r(sa, n + 1, sizeof(uint32_t), cmp_suffix, &c);
    free(t);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* SA-IS (Nong, Zhang and Chan, "Two efficient algorithms for linear time   */
/* suffix array construction", 2009/2011), written from the description:   */
/* classify L/S suffixes, sort the LMS substrings by induced sorting, name  */
/* them, solve the reduced string (recursively if names repeat), and induce */
/* the full order from the sorted LMS suffixes.                             */
/* The input ends with a unique smallest symbol 0.                          */
/* ------------------------------------------------------------------------ */

static inline uint32_t sym(const void *s, int w, uint64_t i)
{
    return w == 1 ? ((const uint8_t *)s)[i] : ((const uint32_t *)s)[i];
}

static void bucket_bounds(const void *s, int w, uint64_t n, uint32_t K,
                          uint64_t *bkt, int ends)
{
    memset(bkt, 0, sizeof(uint64_t) * K);
    for (uint64_t i = 0; i < n; i++) bkt[sym(s, w, i)]++;
    uint64_t sum = 0;
    for (uint32_t c = 0; c < K; c++) {
        sum += bkt[c];
        bkt[c] = ends ? sum : sum - bkt[c];
    }
}

#define IS_LMS(tt, i) ((i) > 0 && (tt)[i] && !(tt)[(i) - 1])

static void induce(const void *s, int w, uint64_t n, uint32_t K,
                   const uint8_t *t, uint32_t *sa, uint64_t *bkt)
{
    /* L-type: left to right, each placed suffix i puts i-1 at its bucket head */
    bucket_bounds(s, w, n, K, bkt, 0);
    for (uint64_t j = 0; j < n; j++) {
        uint32_t v = sa[j];
        if (v != EMPTY && v > 0 && !t[v - 1]) sa[bkt[sym(s, w, v - 1)]++] = v - 1;
    }
    /* S-type: right to left, at bucket ends */
    bucket_bounds(s, w, n, K, bkt, 1);
    for (uint64_t j = n; j-- > 0;) {
        uint32_t v = sa[j];
        if (v != EMPTY && v > 0 && t[v - 1]) sa[--bkt[sym(s, w, v - 1)]] = v - 1;
    }
}

static int lms_equal(const void *s, int w, uint64_t n, const uint8_t *t,
                     uint64_t a, uint64_t b)
{
    for (uint64_t d = 0;; d++) {
        if (a + d >= n || b + d >= n) return 0;
        if (sym(s, w, a + d) != sym(s, w, b + d) || t[a + d] != t[b + d]) return 0;
        if (d > 0) {
            int ea = IS_LMS(t, a + d), eb = IS_LMS(t, b + d);
            if (ea || eb) return ea && eb;
        }
    }
}

static int sais(const void *s, int w, uint64_t n, uint32_t K, uint32_t *sa)
{
    if (n == 1) { sa[0] = 0; return 0; }
    uint8_t *t = (uint8_t *)malloc(n);
    uint64_t *bkt = (uint64_t *)malloc(sizeof(uint64_t) * K);
    if (!t || !bkt) { free(t); free(bkt); return -1; }
    /* 1. types: S if smaller than the next suffix */
    t[n - 1] = 1;
    for (uint64_t i = n - 1; i-- > 0;) {
        uint32_t a = sym(s, w, i), b = sym(s, w, i + 1);
        t[i] = (a < b) || (a == b && t[i + 1]);
    }
    /* 2. sort LMS substrings: seed LMS positions at bucket ends, induce */
    for (uint64_t j = 0; j < n; j++) sa[j] = EMPTY;
    bucket_bounds(s, w, n, K, bkt, 1);
    for (uint64_t i = 1; i < n; i++)
        if (IS_LMS(t, i)) sa[--bkt[sym(s, w, i)]] = (uint32_t)i;
    induce(s, w, n, K, t, sa, bkt);
    /* 3. name LMS substrings in sorted order */
    uint64_t nlms = 0;
    for (uint64_t i = 1; i < n; i++) nlms += IS_LMS(t, i);
    uint32_t *sorted = (uint32_t *)malloc(sizeof(uint32_t) * nlms);
    uint32_t *name = (uint32_t *)malloc(sizeof(uint32_t) * (n / 2 + 1));
    if (!sorted || !name) { free(t); free(bkt); free(sorted); free(name); return -1; }
    uint64_t q = 0;
    for (uint64_t j = 0; j < n; j++)
        if (sa[j] != EMPTY && IS_LMS(t, sa[j])) sorted[q++] = sa[j];
    uint32_t names = 0;
    for (uint64_t j = 0; j < nlms; j++) {
        if (j == 0 || !lms_equal(s, w, n, t, sorted[j - 1], sorted[j])) names++;
        name[sorted[j] / 2] = names - 1;
    }
    free(sorted);
    /* 4. reduced string in text order of LMS positions; solve it */
    uint32_t *pos = (uint32_t *)malloc(sizeof(uint32_t) * nlms);
    uint32_t *s1 = (uint32_t *)malloc(sizeof(uint32_t) * nlms);
    uint32_t *sa1 = (uint32_t *)malloc(sizeof(uint32_t) * nlms);
    if (!pos || !s1 || !sa1) { free(t); free(bkt); free(name); free(pos); free(s1); free(sa1); return -1; }
    q = 0;
    for (uint64_t i = 1; i < n; i++)
        if (IS_LMS(t, i)) { pos[q] = (uint32_t)i; s1[q] = name[i / 2]; q++; }
    free(name);
    int rc = 0;
    if (names == nlms) {
        for (uint64_t i = 0; i < nlms; i++) sa1[s1[i]] = (uint32_t)i;
    } else {
        rc = sais(s1, 4, nlms, names, sa1);
    }
    free(s1);
    if (rc == 0) {
        /* 5. place LMS suffixes in sorted order at bucket ends, then induce */
        for (uint64_t j = 0; j < n; j++) sa[j] = EMPTY;
        bucket_bounds(s, w, n, K, bkt, 1);
        for (uint64_t i = nlms; i-- > 0;) {
            uint32_t p = pos[sa1[i]];
            sa[--bkt[sym(s, w, p)]] = p;
        }
        induce(s, w, n, K, t, sa, bkt);
    }
    free(pos); free(sa1); free(t); free(bkt);
    return rc;
}

int oracle_sa_is(const uint8_t *g, uint64_t n, uint32_t *sa)
{
    if (n + 1 > (uint64_t)UINT32_MAX) return -2;
    uint8_t *t = make_text(g, n);
    if (!t) return -1;
    int rc = sais(t, 1, n + 1, 5, sa);
    free(t);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Plain FM index over T = G$: BWT[j] = T[SA[j]-1] ($ where SA[j] = 0),     */
/* C[c] = number of symbols of T smaller than c, Occ(c, i) = number of c in */
/* BWT[0, i) from a checkpoint every 64 rows plus a scan.                    */
/* ------------------------------------------------------------------------ */

#define CP 64
#define DOLLAR 4

typedef struct {
    uint64_t n;        /* genome length N; T has N+1 rows */
    uint8_t *g;        /* genome codes 0..3 */
    uint8_t *bwt;      /* 0..3 = A..T, 4 = $ */
    uint32_t *sa;      /* full suffix array, N+1 entries */
    uint32_t *cp;      /* Occ(c, 64*b), 4 per checkpoint */
    uint64_t C[5];
} oracle_fm;

void oracle_fm_free(oracle_fm *f)
{
    if (!f) return;
    free(f->g); free(f->bwt); free(f->sa); free(f->cp); free(f);
}

/* sa_method: 0 = sort (small genomes), 1 = SA-IS; or pass a precomputed SA */
oracle_fm *oracle_fm_new(const uint8_t *g, uint64_t n, int sa_method, const uint32_t *sa_in)
{
    if (n + 1 > (uint64_t)UINT32_MAX) return NULL;
    oracle_fm *f = (oracle_fm *)calloc(1, sizeof(oracle_fm));
    if (!f) return NULL;
    uint64_t rows = n + 1, ncp = rows / CP + 1;
    f->n = n;
    f->g = (uint8_t *)malloc(n ? n : 1);
    f->bwt = (uint8_t *)malloc(rows);
    f->sa = (uint32_t *)malloc(sizeof(uint32_t) * rows);
    f->cp = (uint32_t *)malloc(sizeof(uint32_t) * 4 * ncp);
    if (!f->g || !f->bwt || !f->sa || !f->cp) { oracle_fm_free(f); return NULL; }
    memcpy(f->g, g, n);
    int rc = 0;
    if (sa_in) memcpy(f->sa, sa_in, sizeof(uint32_t) * rows);
    else if (sa_method == 0) rc = oracle_sa_sort(g, n, f->sa);
    else rc = oracle_sa_is(g, n, f->sa);
    if (rc) { oracle_fm_free(f); return NULL; }
    for (uint64_t j = 0; j < rows; j++)
        f->bwt[j] = f->sa[j] == 0 ? DOLLAR : g[f->sa[j] - 1];
    uint64_t cnt[4] = {0, 0, 0, 0};
    for (uint64_t j = 0; j < rows; j++) {
        if (j % CP == 0)
            for (int c = 0; c < 4; c++) f->cp[4 * (j / CP) + c] = (uint32_t)cnt[c];
        if (f->bwt[j] != DOLLAR) cnt[f->bwt[j]]++;
    }
    if (rows % CP == 0)
        for (int c = 0; c < 4; c++) f->cp[4 * (rows / CP) + c] = (uint32_t)cnt[c];
    /* C[A] = 1 (only $ is smaller), C[c+1] = C[c] + count of c */
    f->C[0] = 1;
    for (int c = 0; c < 4; c++) f->C[c + 1] = f->C[c] + cnt[c];
    return f;
}

uint64_t oracle_occ(const oracle_fm *f, int c, uint64_t i)
{
    uint64_t b = i / CP, v = f->cp[4 * b + c];
    for (uint64_t j = b * CP; j < i; j++) v += (f->bwt[j] == c);
    return v;
}

uint64_t oracle_C(const oracle_fm *f, int c) { return f->C[c]; }
uint64_t oracle_rows(const oracle_fm *f) { return f->n + 1; }
void oracle_copy_sa(const oracle_fm *f, uint32_t *out) { memcpy(out, f->sa, sizeof(uint32_t) * (f->n + 1)); }
void oracle_copy_bwt(const oracle_fm *f, uint8_t *out) { memcpy(out, f->bwt, f->n + 1); }

/* Exact backward search of pattern p[0..m) (codes 0..3): SA interval [l, r). */
void oracle_exact_interval(const oracle_fm *f, const uint8_t *p, uint32_t m,
                           uint64_t *l_out, uint64_t *r_out)
{
    uint64_t l = 0, r = f->n + 1;
    for (uint32_t i = m; i-- > 0 && l < r;) {
        int c = p[i];
        l = f->C[c] + oracle_occ(f, c, l);
        r = f->C[c] + oracle_occ(f, c, r);
    }
    *l_out = l; *r_out = l < r ? r : l;
}

/* ------------------------------------------------------------------------ */
/* Backtracking search (Section 2's "align with few mismatches" by the BWT  */
/* index): from the whole interval, extend right-to-left with every symbol; */
/* a symbol other than the read's costs one mismatch while the budget lasts. */
/* ------------------------------------------------------------------------ */

typedef struct { uint64_t l, r; uint8_t strand, d; } interval;
typedef struct { interval *v; uint64_t n, cap; uint64_t nodes; int oom; } ivec;

static void ivec_push(ivec *a, uint64_t l, uint64_t r, int strand, int d)
{
    if (a->n == a->cap) {
        uint64_t nc = a->cap ? 2 * a->cap : 16;
        interval *nv = (interval *)realloc(a->v, nc * sizeof(interval));
        if (!nv) { a->oom = 1; return; }
        a->v = nv; a->cap = nc;
    }
    a->v[a->n].l = l; a->v[a->n].r = r;
    a->v[a->n].strand = (uint8_t)strand; a->v[a->n].d = (uint8_t)d;
    a->n++;
}

static void backtrack(const oracle_fm *f, const uint8_t *P, uint32_t i,
                      uint64_t l, uint64_t r, int d, int k, int strand, ivec *out)
{
    out->nodes++;
    if (i == 0) { ivec_push(out, l, r, strand, d); return; }
    for (int c = 0; c < 4; c++) {
        int dd = d + (c != P[i - 1]);
        if (dd > k) continue;
        uint64_t l2 = f->C[c] + oracle_occ(f, c, l);
        uint64_t r2 = f->C[c] + oracle_occ(f, c, r);
        if (l2 < r2) backtrack(f, P, i - 1, l2, r2, dd, k, strand, out);
    }
}

typedef struct { uint32_t pos; uint8_t strand, mm; uint16_t pad; } oracle_hit;

typedef struct {
    uint64_t n_reads;
    uint64_t *total;     /* exact number of hits per read (sum of interval sizes) */
    uint64_t *offsets;   /* n_reads + 1 */
    oracle_hit *hits;
    uint64_t nodes;      /* backtracking nodes visited, all reads */
    int status;
} oracle_result;

void oracle_result_free(oracle_result *r)
{
    if (!r) return;
    free(r->total); free(r->offsets); free(r->hits); free(r);
}

static int cmp_interval(const void *a, const void *b)
{
    const interval *x = (const interval *)a, *y = (const interval *)b;
    if (x->d != y->d) return x->d < y->d ? -1 : 1;
    if (x->strand != y->strand) return x->strand < y->strand ? -1 : 1;
    if (x->l != y->l) return x->l < y->l ? -1 : 1;
    return 0;
}

static int cmp_hit(const void *a, const void *b)
{
    const oracle_hit *x = (const oracle_hit *)a, *y = (const oracle_hit *)b;
    if (x->pos != y->pos) return x->pos < y->pos ? -1 : 1;
    if (x->strand != y->strand) return x->strand < y->strand ? -1 : 1;
    if (x->mm != y->mm) return x->mm < y->mm ? -1 : 1;
    return 0;
}

static void unpack_read(const uint32_t *words, uint64_t off, uint32_t m, uint8_t *out)
{
    for (uint32_t t = 0; t < m; t++) out[t] = (uint8_t)((words[off + t / 16] >> (2 * (t % 16))) & 3);
}

static void reverse_complement(const uint8_t *r, uint32_t m, uint8_t *out)
{
    for (uint32_t t = 0; t < m; t++) out[t] = (uint8_t)(3 - r[m - 1 - t]);
}

/*
 * Align every read: both strands, all hits with at most k[i] mismatches.
 * cap == 0 means no cap.  Returns NULL on allocation failure or bad input
 * (k > 3, length 0, length > N).
 */
oracle_result *oracle_align(const oracle_fm *f, const uint32_t *words, const uint64_t *word_off,
                            const uint16_t *lengths, const uint8_t *kk, uint64_t n_reads,
                            uint32_t cap, int threads)
{
    for (uint64_t i = 0; i < n_reads; i++)
        if (kk[i] > 3 || lengths[i] == 0 || lengths[i] > f->n) return NULL;
    oracle_result *res = (oracle_result *)calloc(1, sizeof(oracle_result));
    oracle_hit **per = (oracle_hit **)calloc(n_reads ? n_reads : 1, sizeof(oracle_hit *));
    uint64_t *cnt = (uint64_t *)calloc(n_reads ? n_reads : 1, sizeof(uint64_t));
    res->n_reads = n_reads;
    res->total = (uint64_t *)calloc(n_reads ? n_reads : 1, sizeof(uint64_t));
    res->offsets = (uint64_t *)calloc(n_reads + 1, sizeof(uint64_t));
    if (!res->total || !res->offsets || !per || !cnt) { free(per); free(cnt); oracle_result_free(res); return NULL; }
    uint64_t nodes = 0;
    int fail = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
    #pragma omp parallel for schedule(dynamic, 16) reduction(+:nodes) reduction(|:fail)
    for (uint64_t i = 0; i < n_reads; i++) {
        uint32_t m = lengths[i];
        uint8_t *R = (uint8_t *)malloc(m), *Q = (uint8_t *)malloc(m);
        ivec iv = {0};
        unpack_read(words, word_off[i], m, R);
        reverse_complement(R, m, Q);
        backtrack(f, R, m, 0, f->n + 1, 0, kk[i], 0, &iv);
        backtrack(f, Q, m, 0, f->n + 1, 0, kk[i], 1, &iv);
        nodes += iv.nodes;
        uint64_t total = 0;
        for (uint64_t j = 0; j < iv.n; j++) total += iv.v[j].r - iv.v[j].l;
        uint64_t keep = (cap && total > cap) ? cap : total;
        /* rows in the order (d, strand, row): sort intervals, walk rows */
        qsort(iv.v, iv.n, sizeof(interval), cmp_interval);
        oracle_hit *h = (oracle_hit *)malloc(sizeof(oracle_hit) * (keep ? keep : 1));
        uint64_t q = 0;
        for (uint64_t j = 0; j < iv.n && q < keep; j++)
            for (uint64_t row = iv.v[j].l; row < iv.v[j].r && q < keep; row++) {
                h[q].pos = f->sa[row];
                h[q].strand = iv.v[j].strand;
                h[q].mm = iv.v[j].d;
                h[q].pad = 0;
                q++;
            }
        qsort(h, keep, sizeof(oracle_hit), cmp_hit);
        res->total[i] = total;
        cnt[i] = keep;
        per[i] = h;
        if (iv.oom || !R || !Q || !h) fail = 1;
        free(iv.v); free(R); free(Q);
    }
    for (uint64_t i = 0; i < n_reads; i++) res->offsets[i + 1] = res->offsets[i] + cnt[i];
    res->hits = (oracle_hit *)malloc(sizeof(oracle_hit) * (res->offsets[n_reads] ? res->offsets[n_reads] : 1));
    if (res->hits)
        for (uint64_t i = 0; i < n_reads; i++)
            if (cnt[i]) memcpy(res->hits + res->offsets[i], per[i], sizeof(oracle_hit) * cnt[i]);
    for (uint64_t i = 0; i < n_reads; i++) free(per[i]);
    free(per); free(cnt);
    res->nodes = nodes;
    res->status = (fail || !res->hits) ? -1 : 0;
    return res;
}

/* ------------------------------------------------------------------------ */
/* Brute force: Hamming distance of R and rc(R) to every window of G.        */
/* Uncapped; hits come out in (position, strand) order.                      */
/* ------------------------------------------------------------------------ */

oracle_result *oracle_bruteforce(const uint8_t *g, uint64_t n, const uint32_t *words,
                                 const uint64_t *word_off, const uint16_t *lengths,
                                 const uint8_t *kk, uint64_t n_reads, int threads)
{
    for (uint64_t i = 0; i < n_reads; i++)
        if (kk[i] > 3 || lengths[i] == 0 || lengths[i] > n) return NULL;
    oracle_result *res = (oracle_result *)calloc(1, sizeof(oracle_result));
    oracle_hit **per = (oracle_hit **)calloc(n_reads ? n_reads : 1, sizeof(oracle_hit *));
    uint64_t *cnt = (uint64_t *)calloc(n_reads ? n_reads : 1, sizeof(uint64_t));
    res->n_reads = n_reads;
    res->total = (uint64_t *)calloc(n_reads ? n_reads : 1, sizeof(uint64_t));
    res->offsets = (uint64_t *)calloc(n_reads + 1, sizeof(uint64_t));
    if (!res->total || !res->offsets || !per || !cnt) { free(per); free(cnt); oracle_result_free(res); return NULL; }
    int fail = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
    /* one read per chunk: a scan of a large genome per read is long enough
       that even a handful of reads should spread over every thread */
    #pragma omp parallel for schedule(dynamic, 1) reduction(|:fail)
    for (uint64_t i = 0; i < n_reads; i++) {
        uint32_t m = lengths[i];
        int k = kk[i];
        uint8_t *R = (uint8_t *)malloc(m), *Q = (uint8_t *)malloc(m);
        unpack_read(words, word_off[i], m, R);
        reverse_complement(R, m, Q);
        uint64_t cap = 16, q = 0;
        oracle_hit *h = (oracle_hit *)malloc(sizeof(oracle_hit) * cap);
        for (uint64_t p = 0; p + m <= n && h; p++) {
            for (int s = 0; s < 2; s++) {
                const uint8_t *P = s ? Q : R;
                int d = 0;
                for (uint32_t t = 0; t < m && d <= k; t++) d += (P[t] != g[p + t]);
                if (d > k) continue;
                if (q == cap) {
                    cap *= 2;
                    oracle_hit *nh = (oracle_hit *)realloc(h, sizeof(oracle_hit) * cap);
                    if (!nh) { free(h); h = NULL; break; }
                    h = nh;
                }
                h[q].pos = (uint32_t)p; h[q].strand = (uint8_t)s; h[q].mm = (uint8_t)d; h[q].pad = 0;
                q++;
            }
        }
        if (!h) fail = 1;
        per[i] = h; cnt[i] = h ? q : 0; res->total[i] = cnt[i];
        free(R); free(Q);
    }
    for (uint64_t i = 0; i < n_reads; i++) res->offsets[i + 1] = res->offsets[i] + cnt[i];
    res->hits = (oracle_hit *)malloc(sizeof(oracle_hit) * (res->offsets[n_reads] ? res->offsets[n_reads] : 1));
    if (res->hits)
        for (uint64_t i = 0; i < n_reads; i++)
            if (cnt[i]) memcpy(res->hits + res->offsets[i], per[i], sizeof(oracle_hit) * cnt[i]);
    for (uint64_t i = 0; i < n_reads; i++) free(per[i]);
    free(per); free(cnt);
    res->status = (fail || !res->hits) ? -1 : 0;
    return res;
}

/* field accessors for foreign-function callers */
uint64_t oracle_result_n(const oracle_result *r) { return r->n_reads; }
int oracle_result_status(const oracle_result *r) { return r->status; }
uint64_t oracle_result_nodes(const oracle_result *r) { return r->nodes; }
void oracle_result_copy(const oracle_result *r, uint64_t *total, uint64_t *offsets, oracle_hit *hits)
{
    memcpy(total, r->total, sizeof(uint64_t) * r->n_reads);
    memcpy(offsets, r->offsets, sizeof(uint64_t) * (r->n_reads + 1));
    memcpy(hits, r->hits, sizeof(oracle_hit) * r->offsets[r->n_reads]);
}
uint64_t oracle_result_n_hits(const oracle_result *r) { return r->offsets[r->n_reads]; }
