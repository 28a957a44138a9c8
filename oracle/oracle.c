/*
 * CPU oracle for factorization sets Z(n, (g_1..g_d)) in numerical semigroups.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant with
 * the CUDA library, and it never reads a value the CUDA library produced.
 *
 * Everything here is plain, slow and single-threaded on purpose, so that each
 * function can be checked against the paper by eye:
 *
 *   oracle_enumerate_range  the paper's bounded lexicographic stream: the first
 *                           candidate of Sec. 3.2.1 and Algorithm 3.1
 *                           (nextCandidate), consumed by "save if wasValid"
 *                           (Sec. 2, Sec. 3.3).  Lex-DECREASING, as in the paper.
 *   oracle_range_stats      the same stream with the count / length consumers
 *                           (Sec. 2 lists save, count and predicate consumers).
 *   oracle_any              the same stream with the predicate consumer (Sec. 2).
 *   oracle_brute            brute force over the box a_i <= n/g_i (Thm 3.3 bound),
 *                           lex-ascending; the definition of Z (Sec. 1) written out.
 *   oracle_count_dp         |Z| as the coefficient of x^n in prod 1/(1-x^{g_i}),
 *                           the plain definition of the count.
 *   oracle_length_dp        histogram of sum a_i as the coefficients of x^n y^l in
 *                           prod 1/(1-y x^{g_i}).
 *   oracle_minmax_dp        min / max of sum a_i by unbounded-knapsack recurrences.
 *
 * Readings of the paper taken here:
 *   - decrementAndSolve divides by g_{i+1}; the "/g_1" in Sec. 3.2.2 is a typo.
 *   - the pivot of nextCandidate (Algorithm 3.1) is searched among the first
 *     d-1 coordinates only: the text excludes the final one, although the
 *     printed loop bound reads "dim".
 *   - the residual decrementAndSolve divides is n minus phi of the candidate
 *     after the pivot is lowered and everything right of it cleared.
 *   - bounds are half-open: a stream for the slice [lo, hi) starts from hi
 *     (not emitted) or from the first candidate when hi is +infinity, and ends
 *     as soon as a candidate is lex-smaller than lo.  The paper's end test
 *     "candidate <=_lex bound" is the same test with the bound itself excluded
 *     from the lower worker; here the lower bound belongs to its own slice.
 *   - the first candidate (x,0..0) is valid iff x*g_1 == n (Sec. 3.2.1).
 *
 * Mutation hooks: oracle_set_mutation(k) switches on ONE deliberately wrong
 * variant of a single step, so that the pin tests can show each pin catches a
 * plausible mistake.  The default (0) is the faithful oracle.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int oracle_mutation = 0;

void oracle_set_mutation(int k) { oracle_mutation = k; }
int oracle_get_mutation(void) { return oracle_mutation; }

/* lexicographic comparison of two d-vectors: -1, 0, +1 */
static int lex_cmp(const int64_t* a, const int64_t* b, int d)
{
    for (int j = 0; j < d; j++) {
        if (a[j] < b[j]) return -1;
        if (a[j] > b[j]) return 1;
    }
    return 0;
}

/* phi(a) = sum_i a_i g_i  (Sec. 3.2.2) */
static int64_t phi(const int64_t* a, const int64_t* g, int d)
{
    int64_t s = 0;
    for (int j = 0; j < d; j++) s += a[j] * g[j];
    return s;
}

/*
 * The first candidate (Sec. 3.2.1): (x, 0, ..., 0) with x = ceil(n / g_1).
 * It is a factorization iff x g_1 == n.
 */
static void first_candidate(int64_t n, const int64_t* g, int d, int64_t* a, int* was_valid)
{
    for (int j = 0; j < d; j++) a[j] = 0;
    int64_t x = (n + g[0] - 1) / g[0];
    if (oracle_mutation == 4) x = n / g[0]; /* mutation: floor instead of ceiling */
    a[0] = x;
    *was_valid = (x * g[0] == n);
}

/*
 * nextCandidate (Sec. 3.2.2, Algorithm 3.1), in place; a[k] holds the
 * coordinate of generator k (0-based here, 1-based in the paper).
 *
 * The stream runs through N^d in decreasing lex order, but only over the
 * candidates: vectors whose last nonzero coordinate is the least value that
 * brings phi up to at least n.  The candidate after a keeps the longest prefix
 * it can: the pivot is the last nonzero coordinate among the first d-1; it
 * drops by one, everything right of it is cleared, and the coordinate just
 * right of it becomes ceil(rest / g), rest = n - phi of what is left and g its
 * generator (decrementAndSolve).  The new candidate is a factorization exactly
 * when that division is exact.  Thm 3.2: no factorization between a and it is
 * skipped.  With no pivot (a = (0,..,0,x)) nothing is left below and the
 * stream ends; it also ends once a candidate falls below `lo`, the slice's
 * inclusive lower bound (NULL for none).
 *
 * rest >= 1 always: a's prefix up to the pivot was itself reached from below
 * n by a least-value solve (or is the first candidate), so lowering the pivot
 * puts phi strictly below n.
 *
 * Returns 0 at the end of the stream, else 1 with *was_valid set for the
 * candidate left in a.
 */
static int next_candidate(int64_t n, const int64_t* g, int d, int64_t* a,
                          const int64_t* lo, int* was_valid)
{
    int scan = (oracle_mutation == 2) ? d : d - 1; /* mutation: the pivot may be the last */
    int piv = -1;
    for (int k = 0; k < scan; k++)
        if (a[k] > 0) piv = k;
    if (piv < 0 || piv == d - 1) return 0; /* piv == d-1 only under mutation 2 */
    a[piv] -= 1;
    for (int k = piv + 1; k < d; k++) a[k] = 0;
    int64_t rest = n - phi(a, g, d);
    int64_t gn = (oracle_mutation == 1) ? g[0] : g[piv + 1]; /* mutation: the "/g_1" typo */
    int64_t q = rest / gn;
    int exact = (q * gn == rest);
    a[piv + 1] = exact ? q : q + 1;
    *was_valid = exact;
    if (oracle_mutation == 5 && exact && piv + 2 < d) *was_valid = 0; /* mutation: drop exact inner solves */
    if (lo && lex_cmp(a, lo, d) < 0) return 0;
    return 1;
}

static void load_gens(const uint32_t* gens, int d, int64_t* g)
{
    for (int j = 0; j < d; j++) g[j] = (int64_t)gens[j];
}

/*
 * The bounded stream for the slice [lo, hi) of the lex order on N^d, consumed
 * by a callback for every valid candidate.  lo == NULL means (0,...,0); hi ==
 * NULL means +infinity (start at the paper's first candidate).  A finite hi
 * must satisfy the hypothesis of Thm 3.2 (its last coordinate is "minimal"),
 * which holds for every vector whose last coordinate is 0 (Remark 4.2).
 * Returns the number of candidates produced (valid or not).
 */
typedef int (*consume_fn)(const int64_t* a, int d, void* ctx); /* nonzero: stop */

static uint64_t run_stream(int64_t n, const uint32_t* gens, int d, const int64_t* lo,
                           const int64_t* hi, consume_fn consume, void* ctx)
{
    int64_t g[64], a[64];
    load_gens(gens, d, g);
    int valid = 0;
    uint64_t candidates = 0;
    if (hi == NULL) {
        first_candidate(n, g, d, a, &valid);
        candidates++;
        if (lo && lex_cmp(a, lo, d) < 0) return candidates;
        if (valid && consume(a, d, ctx)) return candidates;
    } else {
        for (int j = 0; j < d; j++) a[j] = hi[j];
        /* hi itself belongs to the next slice: it is not consumed here */
    }
    if (oracle_mutation == 3) {
        /* mutation: skip one candidate right after the start */
        if (!next_candidate(n, g, d, a, lo, &valid)) return candidates;
        candidates++;
    }
    while (next_candidate(n, g, d, a, lo, &valid)) {
        candidates++;
        if (valid && consume(a, d, ctx)) break;
    }
    return candidates;
}

/* ---- consumer: save ------------------------------------------------------ */
typedef struct {
    int32_t* out;
    int64_t cap;
    int64_t count;
} save_ctx;

static int consume_save(const int64_t* a, int d, void* vctx)
{
    save_ctx* c = (save_ctx*)vctx;
    if (c->out && c->count < c->cap)
        for (int j = 0; j < d; j++) c->out[c->count * d + j] = (int32_t)a[j];
    c->count++;
    return 0;
}

/*
 * Enumerate Z(n,g) restricted to [lo, hi) in the paper's order (lex
 * decreasing).  Writes at most `cap` rows of d int32 into out (row-major) and
 * returns the number of factorizations in the slice.  *candidates (nullable)
 * receives the number of nextCandidate outputs, valid or not.
 */
int64_t oracle_enumerate_range(int64_t n, const uint32_t* gens, int d, const int64_t* lo,
                               const int64_t* hi, int32_t* out, int64_t cap,
                               uint64_t* candidates)
{
    save_ctx c = {out, cap, 0};
    uint64_t k = run_stream(n, gens, d, lo, hi, consume_save, &c);
    if (candidates) *candidates = k;
    return c.count;
}

/* The whole stream (bound (0,...,0), Sec. 3.1.2). */
int64_t oracle_enumerate(int64_t n, const uint32_t* gens, int d, int32_t* out, int64_t cap,
                         uint64_t* candidates)
{
    return oracle_enumerate_range(n, gens, d, NULL, NULL, out, cap, candidates);
}

/* ---- consumer: count and length statistics --------------------------------- */
typedef struct {
    uint64_t count;
    int64_t min_len, max_len;
    uint64_t* hist; /* nullable, hist_len bins */
    int64_t hist_len;
    int overflow;
} stats_ctx;

static int consume_stats(const int64_t* a, int d, void* vctx)
{
    stats_ctx* c = (stats_ctx*)vctx;
    int64_t len = 0;
    for (int j = 0; j < d; j++) len += a[j];
    if (c->count == 0 || len < c->min_len) c->min_len = len;
    if (c->count == 0 || len > c->max_len) c->max_len = len;
    c->count++;
    if (c->hist) {
        if (len < c->hist_len) c->hist[len]++;
        else c->overflow = 1;
    }
    return 0;
}

/*
 * Count, min / max length and (optionally) the length histogram of the
 * factorizations in [lo, hi), from the bounded stream.  Returns 0, or -1 if a
 * length fell outside the histogram.  min / max are 0 when the slice is empty.
 */
int oracle_range_stats(int64_t n, const uint32_t* gens, int d, const int64_t* lo,
                       const int64_t* hi, uint64_t* count, int64_t* min_len, int64_t* max_len,
                       uint64_t* hist, int64_t hist_len, uint64_t* candidates)
{
    stats_ctx c = {0, 0, 0, hist, hist_len, 0};
    if (hist) memset(hist, 0, sizeof(uint64_t) * (size_t)hist_len);
    uint64_t k = run_stream(n, gens, d, lo, hi, consume_stats, &c);
    *count = c.count;
    *min_len = c.count ? c.min_len : 0;
    *max_len = c.count ? c.max_len : 0;
    if (candidates) *candidates = k;
    return c.overflow ? -1 : 0;
}

/* ---- consumer: predicate ----------------------------------------------------- */
/*
 * A linear predicate on a factorization a (Sec. 2: "a predicate's value for
 * each result"): with s = sum_i w_i a_i,
 *   modulus > 0 : s == c (mod modulus), both sides reduced into [0, modulus);
 *   op 0        : s == c;   op 1 : s <= c;   op 2 : s >= c.
 */
typedef struct {
    const int32_t* w;
    int64_t c;
    int op;
    uint32_t modulus;
    int found;
} pred_ctx;

static int pred_holds(const pred_ctx* p, const int64_t* a, int d)
{
    int64_t s = 0;
    for (int j = 0; j < d; j++) s += (int64_t)p->w[j] * a[j];
    if (p->modulus > 0) {
        int64_t m = (int64_t)p->modulus;
        int64_t sl = ((s % m) + m) % m, cl = ((p->c % m) + m) % m;
        return sl == cl;
    }
    if (p->op == 0) return s == p->c;
    if (p->op == 1) return s <= p->c;
    return s >= p->c;
}

static int consume_pred(const int64_t* a, int d, void* vctx)
{
    pred_ctx* p = (pred_ctx*)vctx;
    if (pred_holds(p, a, d)) {
        p->found = 1;
        return 1;
    }
    return 0;
}

int oracle_any(int64_t n, const uint32_t* gens, int d, const int32_t* w, int64_t c, int op,
               uint32_t modulus)
{
    pred_ctx p = {w, c, op, modulus, 0};
    run_stream(n, gens, d, NULL, NULL, consume_pred, &p);
    return p.found;
}

/* ---- brute force -------------------------------------------------------------- */
/*
 * Every a with 0 <= a_i <= n / g_i (Thm 3.3's box), in lex-ASCENDING order, kept
 * iff sum a_i g_i == n: the definition of Z(n, g) (Sec. 1) written out.
 */
int64_t oracle_brute(int64_t n, const uint32_t* gens, int d, int32_t* out, int64_t cap)
{
    int64_t g[64], a[64], top[64];
    load_gens(gens, d, g);
    for (int j = 0; j < d; j++) {
        a[j] = 0;
        top[j] = n / g[j];
    }
    int64_t count = 0;
    for (;;) {
        if (phi(a, g, d) == n) {
            if (out && count < cap)
                for (int j = 0; j < d; j++) out[count * d + j] = (int32_t)a[j];
            count++;
        }
        int j = d - 1; /* odometer increment, last coordinate fastest */
        while (j >= 0 && a[j] == top[j]) {
            a[j] = 0;
            j--;
        }
        if (j < 0) break;
        a[j]++;
    }
    return count;
}

/* ---- dynamic programmes (plain definitions of count and lengths) -------------- */
/*
 * |Z(n,g)| = [x^n] prod_i 1/(1 - x^{g_i}).  Multiplying by 1/(1-x^g) is the
 * running sum c[p] += c[p-g] for p = g..n.  Exact in 128-bit; returns -1 if the
 * result does not fit 64 bits.
 */
int oracle_count_dp(int64_t n, const uint32_t* gens, int d, uint64_t* out)
{
    unsigned __int128* c = (unsigned __int128*)calloc((size_t)n + 1, sizeof(unsigned __int128));
    if (!c) return -2;
    c[0] = 1;
    for (int j = 0; j < d; j++) {
        int64_t gj = gens[j];
        for (int64_t p = gj; p <= n; p++) c[p] += c[p - gj];
    }
    unsigned __int128 r = c[n];
    free(c);
    if (r > (unsigned __int128)UINT64_MAX) return -1;
    *out = (uint64_t)r;
    return 0;
}

/*
 * hist[l] = [x^n y^l] prod_i 1/(1 - y x^{g_i}), the number of factorizations
 * of n of length l = sum a_i, for l = 0..hist_len-1.  The table T[p][l] is
 * stored ragged (l <= p / min g).  Returns 0, -1 on 64-bit overflow, -2 if out
 * of memory.
 */
int oracle_length_dp(int64_t n, const uint32_t* gens, int d, uint64_t* hist, int64_t hist_len)
{
    int64_t gmin = gens[0];
    for (int j = 1; j < d; j++)
        if ((int64_t)gens[j] < gmin) gmin = gens[j];
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 2));
    if (!off) return -2;
    off[0] = 0;
    for (int64_t p = 0; p <= n; p++) off[p + 1] = off[p] + p / gmin + 1;
    uint64_t* T = (uint64_t*)calloc((size_t)off[n + 1], sizeof(uint64_t));
    if (!T) {
        free(off);
        return -2;
    }
    int ovf = 0;
    T[0] = 1; /* the empty factorization of 0 has length 0 */
    for (int j = 0; j < d; j++) {
        int64_t gj = gens[j];
        for (int64_t p = gj; p <= n; p++) {
            int64_t lmax = p / gmin, lprev = (p - gj) / gmin;
            for (int64_t l = 1; l <= lmax && l - 1 <= lprev; l++) {
                uint64_t add = T[off[p - gj] + l - 1];
                if (__builtin_add_overflow(T[off[p] + l], add, &T[off[p] + l])) ovf = 1;
            }
        }
    }
    for (int64_t l = 0; l < hist_len; l++) hist[l] = (l <= n / gmin) ? T[off[n] + l] : 0;
    free(T);
    free(off);
    return ovf ? -1 : 0;
}

/*
 * Minimum and maximum of sum a_i over Z(n,g) by the recurrences
 * m(p) = min_i m(p - g_i) + 1 and M(p) = max_i M(p - g_i) + 1 with m(0) = M(0) = 0.
 * Returns 1 if Z is nonempty (and fills min / max), 0 if empty.
 */
int oracle_minmax_dp(int64_t n, const uint32_t* gens, int d, int64_t* min_len, int64_t* max_len)
{
    int64_t* mn = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int64_t* mx = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!mn || !mx) {
        free(mn);
        free(mx);
        return -2;
    }
    const int64_t NONE = -1;
    mn[0] = mx[0] = 0;
    for (int64_t p = 1; p <= n; p++) {
        mn[p] = mx[p] = NONE;
        for (int j = 0; j < d; j++) {
            int64_t gj = gens[j];
            if (gj <= p && mn[p - gj] != NONE) {
                if (mn[p] == NONE || mn[p - gj] + 1 < mn[p]) mn[p] = mn[p - gj] + 1;
                if (mx[p] == NONE || mx[p - gj] + 1 > mx[p]) mx[p] = mx[p - gj] + 1;
            }
        }
    }
    int ok = (mn[n] != NONE);
    if (ok) {
        *min_len = mn[n];
        *max_len = mx[n];
    }
    free(mn);
    free(mx);
    return ok;
}
