/*
 * oracle.c -- plain, slow, obviously correct CPU oracle for comparator-based
 * K-nearest-neighbour descent with the Kullback-Leibler comparator
 * (Baron & Darling, "Empirical complexity of comparator-based nearest
 * neighbor descent", arXiv:2202.00517).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or helper with the CUDA library: every routine below is written from the
 * paper's definitions (and, for the random draws, from the published
 * definitions of Philox4x32-10 and of Lemire's bounded integers).
 *
 * Arithmetic: IEEE binary64 throughout.  Compile with -ffp-contract=off so
 * that the only fused operations are the explicit fma() calls of the
 * canonical key chain.
 *
 * Readings of the paper fixed here (each one is listed in the design notes):
 *   - comparator direction: x ranks y by D(x||y) = sum_i x_i log(x_i/y_i)
 *     (Sec. 2.2), evaluated as key(x,y) = negH(x) - <x, log y> with
 *     negH(x) = sum_i x_i log x_i; both sums are sequential fma chains from 0
 *     over i = 0..m-1;
 *   - ties: total order by (key ascending, index ascending);
 *   - candidate pool of x in one round (Sec. 3.1 "Meet"/"Update", Sec. 4.2
 *     proposeNewFriendSet): current friends, co-friends, friends of friends
 *     and friends of co-friends, as a set, minus x itself;
 *   - synchronous rounds: all new friend sets are computed from the old
 *     graph (Sec. 4.2);
 *   - random draws: Philox4x32-10 keyed by the 64-bit seed, counter
 *     (c0, c1, c2, block); streams c2 = 0 initial graph (c0 = point),
 *     c2 = 1 friend-clustering sample (c0 = sample index, c1 = round);
 *   - friend clustering rate (Sec. 3.3): sample x uniformly, then two
 *     distinct positions of x's sorted friend list; a hit when z is a friend
 *     of y or y is a friend of z; stop after the first round whose hit count
 *     does not exceed the previous round's (ties stop).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies whose    */
/* high halves are xored with the other counter words and the round key;    */
/* the key is bumped by the Weyl constants between rounds.                  */
/* ------------------------------------------------------------------------ */
#define ORC_PH_M0 0xD2511F53u
#define ORC_PH_M1 0xCD9E8D57u
#define ORC_PH_W0 0x9E3779B9u
#define ORC_PH_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)ORC_PH_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)ORC_PH_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += ORC_PH_W0;
        k1 += ORC_PH_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A word stream: counter (c0, c1, c2, j) for j = 0, 1, ...; the four words
 * of block j are consumed in order before block j+1 is generated. */
typedef struct {
    uint32_t key[2];
    uint32_t ctr[3];
    uint32_t block;
    uint32_t buf[4];
    int pos; /* next unread word of buf; 4 = empty */
} orc_stream;

static void orc_stream_init(orc_stream *s, uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2)
{
    s->key[0] = (uint32_t)(seed & 0xffffffffu);
    s->key[1] = (uint32_t)(seed >> 32);
    s->ctr[0] = c0; s->ctr[1] = c1; s->ctr[2] = c2;
    s->block = 0;
    s->pos = 4;
}

static uint32_t orc_next_word(orc_stream *s)
{
    if (s->pos == 4) {
        uint32_t c[4] = {s->ctr[0], s->ctr[1], s->ctr[2], s->block};
        orc_philox4x32_10(c, s->key, s->buf);
        s->block += 1;
        s->pos = 0;
    }
    return s->buf[s->pos++];
}

/* Uniform integer in [0, N), N >= 1: Lemire's multiply-shift with rejection
 * ("Fast random integer generation in an interval", ACM TOMACS 2019).  A
 * rejected draw consumes the next word of the stream. */
static uint32_t orc_bounded(orc_stream *s, uint32_t N)
{
    uint32_t w = orc_next_word(s);
    uint64_t mprod = (uint64_t)w * (uint64_t)N;
    uint32_t low = (uint32_t)mprod;
    if (low < N) {
        uint32_t thresh = (uint32_t)(-N) % N;
        while (low < thresh) {
            w = orc_next_word(s);
            mprod = (uint64_t)w * (uint64_t)N;
            low = (uint32_t)mprod;
        }
    }
    return (uint32_t)(mprod >> 32);
}

/* Test hook: the first `count` bounded draws of stream (seed, c0, c1, c2). */
void orc_bounded_draws(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t N,
                       int64_t count, uint32_t *out)
{
    orc_stream s;
    orc_stream_init(&s, seed, c0, c1, c2);
    for (int64_t t = 0; t < count; ++t) out[t] = orc_bounded(&s, N);
}

/* Test hook: the first `count` raw words of stream (seed, c0, c1, c2). */
void orc_stream_words(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, int64_t count, uint32_t *out)
{
    orc_stream s;
    orc_stream_init(&s, seed, c0, c1, c2);
    for (int64_t t = 0; t < count; ++t) out[t] = orc_next_word(&s);
}

/* ------------------------------------------------------------------------ */
/* The KL comparator (Sec. 2.2; Sec. 4.4): D(x||y) = sum_i x_i log(x_i/y_i) */
/* = negH(x) - <x, log y>.                                                   */
/* ------------------------------------------------------------------------ */

/* L[y*m + i] = log(y_i); negH[y] = sum_i y_i * log(y_i) (fma chain from 0). */
void orc_logs(const double *pts, int64_t n, int m, double *L, double *negH)
{
    for (int64_t y = 0; y < n; ++y) {
        double acc = 0.0;
        for (int i = 0; i < m; ++i) {
            double l = log(pts[y * m + i]);
            L[y * m + i] = l;
            acc = fma(pts[y * m + i], l, acc);
        }
        negH[y] = acc;
    }
}

/* The comparator of x (Sec. 2 item (a): any function of x that ranks the
 * other points; set before the calls that key pairs):
 *   0  D(x||y) = key(x, y), the paper's (Sec. 2.2, Sec. 4.4);
 *   1  D(y||x) = key(y, x), the KL divergence the other way round;
 *   2  |x - y|^2 = (|x|^2 - 2 <x, y>) + |y|^2, a symmetric metric comparator,
 *      |x|^2 and <x, y> sequential fma chains from 0 (2 <x, y> is exact);
 *   3  0 - <x, y>: the larger the inner product, the closer (maximum inner
 *      product neighbours), <x, y> a sequential fma chain from 0. */
static int orc_cmp = 0;

void orc_set_comparator(int32_t c) { orc_cmp = (c >= 1 && c <= 3) ? c : 0; }

/* Per-point tables of the comparator: KL forms L = log(x), off = negH(x);
 * squared Euclidean L unused, off = |x|^2; inner product L = x, off = 0. */
static void orc_tables(const double *pts, int64_t n, int m, double *L, double *off)
{
    if (orc_cmp == 3) {
        for (int64_t y = 0; y < n; ++y) {
            for (int i = 0; i < m; ++i) L[y * m + i] = pts[y * m + i];
            off[y] = 0.0;
        }
        return;
    }
    if (orc_cmp != 2) {
        orc_logs(pts, n, m, L, off);
        return;
    }
    for (int64_t y = 0; y < n; ++y) {
        double acc = 0.0;
        for (int i = 0; i < m; ++i) acc = fma(pts[y * m + i], pts[y * m + i], acc);
        off[y] = acc;
    }
}

/* key(x, y) for the comparator: KL negH(x) - sum_i x_i * log(y_i) (the inner
 * sum an fma chain from 0 over i = 0..m-1), the roles swapped for 1;
 * squared Euclidean (off(x) - 2 sum_i x_i y_i) + off(y); inner product
 * 0 - sum_i x_i y_i (the KL form's chain with L = x and off = 0). */
static double orc_key_from_tables(const double *pts, const double *L, const double *off,
                                  int m, int64_t x, int64_t y)
{
    double dot = 0.0;
    if (orc_cmp == 2) {
        for (int i = 0; i < m; ++i) dot = fma(pts[x * m + i], pts[y * m + i], dot);
        return (off[x] - 2.0 * dot) + off[y];
    }
    if (orc_cmp == 1) {
        const int64_t t = x;
        x = y;
        y = t;
    }
    for (int i = 0; i < m; ++i) dot = fma(pts[x * m + i], L[y * m + i], dot);
    return off[x] - dot;
}

/* Keys for a list of (x, y) pairs, building its own log table. */
void orc_keys_pairs(const double *pts, int64_t n, int m, const int32_t *xs, const int32_t *ys,
                    int64_t npairs, double *out)
{
    double *L = (double *)malloc(sizeof(double) * (size_t)n * (size_t)m);
    double *negH = (double *)malloc(sizeof(double) * (size_t)n);
    orc_tables(pts, n, m, L, negH);
    for (int64_t p = 0; p < npairs; ++p) out[p] = orc_key_from_tables(pts, L, negH, m, xs[p], ys[p]);
    free(L);
    free(negH);
}

/* ------------------------------------------------------------------------ */
/* Total order on candidates: (key ascending, index ascending).             */
/* ------------------------------------------------------------------------ */
typedef struct {
    double key;
    int32_t idx;
} orc_cand;

static int orc_cand_cmp(const void *a, const void *b)
{
    const orc_cand *p = (const orc_cand *)a, *q = (const orc_cand *)b;
    if (p->key < q->key) return -1;
    if (p->key > q->key) return 1;
    if (p->idx < q->idx) return -1;
    if (p->idx > q->idx) return 1;
    return 0;
}

static int orc_int_cmp(const void *a, const void *b)
{
    int32_t p = *(const int32_t *)a, q = *(const int32_t *)b;
    return (p > q) - (p < q);
}

/* ------------------------------------------------------------------------ */
/* Initial graph (Sec. 3.2; Sec. 4.2): x draws K distinct friends from the   */
/* other n - 1 points, each equally likely, and orders them by its           */
/* comparator.  Draw: y' uniform in [0, n-1), y = y' + (y' >= x); a value    */
/* already chosen is drawn again.                                            */
/* ------------------------------------------------------------------------ */
void orc_init_graph(const double *pts, int64_t n, int m, int K, uint64_t seed,
                    int32_t *idx, double *key)
{
    double *L = (double *)malloc(sizeof(double) * (size_t)n * (size_t)m);
    double *negH = (double *)malloc(sizeof(double) * (size_t)n);
    orc_tables(pts, n, m, L, negH);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t x = 0; x < n; ++x) {
        orc_stream s;
        orc_stream_init(&s, seed, (uint32_t)x, 0u, 0u);
        orc_cand *c = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)K);
        int cnt = 0;
        while (cnt < K) {
            uint32_t yp = orc_bounded(&s, (uint32_t)(n - 1));
            int32_t y = (int32_t)yp + ((int64_t)yp >= x ? 1 : 0);
            int dup = 0;
            for (int t = 0; t < cnt; ++t)
                if (c[t].idx == y) dup = 1;
            if (dup) continue;
            c[cnt].idx = y;
            c[cnt].key = orc_key_from_tables(pts, L, negH, m, x, y);
            cnt += 1;
        }
        qsort(c, (size_t)K, sizeof(orc_cand), orc_cand_cmp);
        for (int t = 0; t < K; ++t) {
            idx[x * K + t] = c[t].idx;
            key[x * K + t] = c[t].key;
        }
        free(c);
    }
    free(L);
    free(negH);
}

/* ------------------------------------------------------------------------ */
/* Co-friends (Sec. 3.1; Sec. 4.2): coF(v) = { x : v is a friend of x }.     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t *off;  /* n+1 */
    int32_t *list; /* n*K */
} orc_cofriends;

static void orc_cofriends_build(const int32_t *idx, int64_t n, int K, orc_cofriends *c)
{
    c->off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    c->list = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (size_t)K + 1);
    for (int64_t e = 0; e < n * K; ++e) c->off[idx[e] + 1] += 1;
    for (int64_t v = 0; v < n; ++v) c->off[v + 1] += c->off[v];
    int64_t *fill = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    for (int64_t x = 0; x < n; ++x)
        for (int t = 0; t < K; ++t) {
            int32_t v = idx[x * K + t];
            c->list[c->off[v] + fill[v]] = (int32_t)x;
            fill[v] += 1;
        }
    free(fill);
}

static void orc_cofriends_free(orc_cofriends *c)
{
    free(c->off);
    free(c->list);
}

/* In-degree of every point (the size of its co-friend set). */
void orc_indegree(const int32_t *idx, int64_t n, int K, int64_t *deg)
{
    memset(deg, 0, sizeof(int64_t) * (size_t)n);
    for (int64_t e = 0; e < n * K; ++e) deg[idx[e]] += 1;
}

/* Candidate pool of x (Sec. 3.1 "Meet"; Sec. 4.2 proposeNewFriendSet):
 * F(x) u coF(x) u F(F(x)) u F(coF(x)), minus {x}, as a sorted set.  Returns
 * its size; `buf` must hold K + |coF(x)| + K*K + K*|coF(x)| entries. */
static int64_t orc_pool(const int32_t *idx, int K, const orc_cofriends *cf, int64_t x, int32_t *buf)
{
    int64_t len = 0;
    for (int t = 0; t < K; ++t) buf[len++] = idx[x * K + t];                     /* friends */
    for (int64_t q = cf->off[x]; q < cf->off[x + 1]; ++q) buf[len++] = cf->list[q]; /* co-friends */
    for (int t = 0; t < K; ++t) { /* friends of friends */
        int32_t v = idx[x * K + t];
        for (int j = 0; j < K; ++j) buf[len++] = idx[(int64_t)v * K + j];
    }
    for (int64_t q = cf->off[x]; q < cf->off[x + 1]; ++q) { /* friends of co-friends */
        int32_t w = cf->list[q];
        for (int j = 0; j < K; ++j) buf[len++] = idx[(int64_t)w * K + j];
    }
    qsort(buf, (size_t)len, sizeof(int32_t), orc_int_cmp);
    int64_t u = 0;
    for (int64_t t = 0; t < len; ++t) {
        if (buf[t] == (int32_t)x) continue;
        if (u > 0 && buf[u - 1] == buf[t]) continue;
        buf[u++] = buf[t];
    }
    return u;
}

/* Test hook: the pool of every x in [x0, x1) as CSR (pool_off has x1-x0+1
 * entries; pool must hold the sum of the bounds). */
void orc_pools(const int32_t *idx, int64_t n, int K, int64_t x0, int64_t x1, int64_t *pool_off, int32_t *pool)
{
    orc_cofriends cf;
    orc_cofriends_build(idx, n, K, &cf);
    int64_t maxdeg = 0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t d = cf.off[v + 1] - cf.off[v];
        if (d > maxdeg) maxdeg = d;
    }
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)((K + maxdeg) * (K + 1)));
    pool_off[0] = 0;
    for (int64_t x = x0; x < x1; ++x) {
        int64_t len = orc_pool(idx, K, &cf, x, buf);
        memcpy(pool + pool_off[x - x0], buf, sizeof(int32_t) * (size_t)len);
        pool_off[x - x0 + 1] = pool_off[x - x0] + len;
    }
    free(buf);
    orc_cofriends_free(&cf);
}

/* ------------------------------------------------------------------------ */
/* One synchronous round of friend set update (Sec. 3.1; Sec. 4.2): the new  */
/* friend set of x is the K best of its pool under (key, index); every new   */
/* set is computed from the old graph.  Rows x in [x0, x1) are computed and  */
/* written at row x of the outputs.  newflag marks entries absent from the  */
/* old list.  Returns the number of new entries (updates) in those rows.     */
/* *proposals receives the size of the candidate multiset of those rows,    */
/* sum over x of K*K + (K+1)*|coF(x)| (the K + 2K^2 proposals per point of   */
/* the footnote in Sec. 4.4, on average).                                   */
/* ------------------------------------------------------------------------ */
int64_t orc_round(const double *pts, int64_t n, int m, int K, const int32_t *idx_in,
                  int64_t x0, int64_t x1, int32_t *idx_out, double *key_out, uint8_t *newflag,
                  int64_t *proposals)
{
    double *L = (double *)malloc(sizeof(double) * (size_t)n * (size_t)m);
    double *negH = (double *)malloc(sizeof(double) * (size_t)n);
    orc_tables(pts, n, m, L, negH);
    orc_cofriends cf;
    orc_cofriends_build(idx_in, n, K, &cf);
    int64_t maxdeg = 0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t d = cf.off[v + 1] - cf.off[v];
        if (d > maxdeg) maxdeg = d;
    }
    int64_t updates = 0, props = 0;
#pragma omp parallel reduction(+ : updates, props)
    {
        int64_t cap = (K + maxdeg) * (K + 1);
        int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
        orc_cand *c = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
        for (int64_t x = x0; x < x1; ++x) {
            int64_t len = orc_pool(idx_in, K, &cf, x, buf);
            for (int64_t t = 0; t < len; ++t) {
                c[t].idx = buf[t];
                c[t].key = orc_key_from_tables(pts, L, negH, m, x, buf[t]);
            }
            qsort(c, (size_t)len, sizeof(orc_cand), orc_cand_cmp);
            for (int t = 0; t < K; ++t) {
                int32_t y = c[t].idx;
                int old = 0;
                for (int j = 0; j < K; ++j)
                    if (idx_in[x * K + j] == y) old = 1;
                idx_out[x * K + t] = y;
                key_out[x * K + t] = c[t].key;
                newflag[x * K + t] = (uint8_t)(old ? 0 : 1);
                updates += old ? 0 : 1;
            }
            props += (int64_t)K * K + (int64_t)(K + 1) * (cf.off[x + 1] - cf.off[x]);
        }
        free(buf);
        free(c);
    }
    if (proposals) *proposals = props;
    orc_cofriends_free(&cf);
    free(L);
    free(negH);
    return updates;
}

/* ------------------------------------------------------------------------ */
/* Friend clustering rate sample (Sec. 3.3): for s = 0..S-1 draw x uniform   */
/* in [0, n), position i uniform in [0, K), position j uniform among the     */
/* other K-1 positions; y = F(x)[i], z = F(x)[j]; a hit when z is a friend   */
/* of y or y is a friend of z.  Returns the hit count.                       */
/* ------------------------------------------------------------------------ */
static int orc_is_friend(const int32_t *idx, int K, int32_t a, int32_t b)
{
    for (int t = 0; t < K; ++t)
        if (idx[(int64_t)a * K + t] == b) return 1;
    return 0;
}

int64_t orc_fcc(const int32_t *idx, int64_t n, int K, uint64_t seed, int32_t round, int32_t S)
{
    int64_t hits = 0;
    for (int32_t s = 0; s < S; ++s) {
        orc_stream st;
        orc_stream_init(&st, seed, (uint32_t)s, (uint32_t)round, 1u);
        int64_t x = orc_bounded(&st, (uint32_t)n);
        int i = (int)orc_bounded(&st, (uint32_t)K);
        int jp = (int)orc_bounded(&st, (uint32_t)(K - 1));
        int j = jp + (jp >= i ? 1 : 0);
        int32_t y = idx[x * K + i], z = idx[x * K + j];
        if (orc_is_friend(idx, K, y, z) || orc_is_friend(idx, K, z, y)) hits += 1;
    }
    return hits;
}

/* ------------------------------------------------------------------------ */
/* The build loop (Sec. 3; Sec. 4.2): initial graph, then rounds until the   */
/* friend clustering hit count does not increase (Sec. 3.3 (iv)), or a round */
/* makes no update (when stop_on_zero), or (stop_delta > 0) a round makes   */
/* fewer than stop_delta * n * K updates, the delta-proportion rule of Dong  */
/* et al. that Sec. 2 (Table 1, item (b)) contrasts with the statistical     */
/* stop, or max_rounds rounds.  Returns the                                  */
/* number of rounds performed; updates[r-1] is round r's update count and    */
/* hits[r] the clustering hits of the graph after round r (hits[0]: initial  */
/* graph).  proposals (optional) receives the total candidate multiset size. */
/* ------------------------------------------------------------------------ */
int32_t orc_build(const double *pts, int64_t n, int m, int K, uint64_t seed, int32_t S,
                  int32_t max_rounds, int32_t stop_on_zero, double stop_delta, int32_t *idx, double *key,
                  int64_t *updates, int64_t *hits, int64_t *proposals)
{
    int32_t *nidx = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (size_t)K);
    double *nkey = (double *)malloc(sizeof(double) * (size_t)n * (size_t)K);
    uint8_t *nflag = (uint8_t *)malloc((size_t)n * (size_t)K);
    orc_init_graph(pts, n, m, K, seed, idx, key);
    hits[0] = orc_fcc(idx, n, K, seed, 0, S);
    int32_t r = 0;
    int64_t props_total = 0;
    while (r < max_rounds) {
        r += 1;
        int64_t props = 0;
        updates[r - 1] = orc_round(pts, n, m, K, idx, 0, n, nidx, nkey, nflag, &props);
        props_total += props;
        memcpy(idx, nidx, sizeof(int32_t) * (size_t)n * (size_t)K);
        memcpy(key, nkey, sizeof(double) * (size_t)n * (size_t)K);
        hits[r] = orc_fcc(idx, n, K, seed, r, S);
        if (hits[r] <= hits[r - 1]) break;
        if (stop_on_zero && updates[r - 1] == 0) break;
        if (stop_delta > 0.0 && (double)updates[r - 1] < stop_delta * (double)n * (double)K) break;
    }
    if (proposals) *proposals = props_total;
    free(nidx);
    free(nkey);
    free(nflag);
    return r;
}

/* ------------------------------------------------------------------------ */
/* Exact K-NN graph by brute force (Sec. 2.3): for each query x, the K best  */
/* of S \ {x} under (key, index).  Every y != x is keyed; a sorted list of   */
/* the K best seen so far takes y when it ranks before the list's last      */
/* entry, by insertion (the list a full sort of all n - 1 candidates would  */
/* start with, without sorting them all).                                   */
/* ------------------------------------------------------------------------ */
void orc_bruteforce(const double *pts, int64_t n, int m, int K, const int32_t *queries, int64_t nq,
                    int32_t *idx, double *key)
{
    double *L = (double *)malloc(sizeof(double) * (size_t)n * (size_t)m);
    double *negH = (double *)malloc(sizeof(double) * (size_t)n);
    orc_tables(pts, n, m, L, negH);
#pragma omp parallel
    {
        orc_cand *c = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)K);
#pragma omp for schedule(dynamic, 4)
        for (int64_t q = 0; q < nq; ++q) {
            int64_t x = queries[q];
            int len = 0; /* c[0 .. len) holds the best so far, sorted; len <= K */
            for (int64_t y = 0; y < n; ++y) {
                if (y == x) continue;
                orc_cand e;
                e.key = orc_key_from_tables(pts, L, negH, m, x, y);
                e.idx = (int32_t)y;
                if (len == K && orc_cand_cmp(&e, &c[K - 1]) >= 0) continue; /* not among the K best */
                int t = len < K ? len++ : K - 1; /* a full list drops its last entry */
                while (t > 0 && orc_cand_cmp(&e, &c[t - 1]) < 0) {
                    c[t] = c[t - 1];
                    --t;
                }
                c[t] = e;
            }
            for (int t = 0; t < K; ++t) {
                idx[q * K + t] = c[t].idx;
                key[q * K + t] = c[t].key;
            }
        }
        free(c);
    }
    free(L);
    free(negH);
}

/* ------------------------------------------------------------------------ */
/* Diameter of a K-out digraph with its arcs read as undirected edges       */
/* (Sec. 3.2; Sec. 4.3), by breadth-first search.                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t *off;
    int32_t *adj;
} orc_undirected;

static void orc_undirected_build(const int32_t *idx, int64_t n, int K, orc_undirected *g)
{
    /* both directions of every arc, then duplicates removed per vertex */
    int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t x = 0; x < n; ++x)
        for (int t = 0; t < K; ++t) {
            deg[x + 1] += 1;
            deg[idx[x * K + t] + 1] += 1;
        }
    for (int64_t v = 0; v < n; ++v) deg[v + 1] += deg[v];
    int32_t *raw = (int32_t *)malloc(sizeof(int32_t) * (size_t)deg[n] + 1);
    int64_t *fill = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    for (int64_t x = 0; x < n; ++x)
        for (int t = 0; t < K; ++t) {
            int32_t y = idx[x * K + t];
            raw[deg[x] + fill[x]++] = y;
            raw[deg[y] + fill[y]++] = (int32_t)x;
        }
    g->off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)deg[n] + 1);
    for (int64_t v = 0; v < n; ++v) {
        int32_t *seg = raw + deg[v];
        int64_t len = deg[v + 1] - deg[v];
        qsort(seg, (size_t)len, sizeof(int32_t), orc_int_cmp);
        int64_t u = 0;
        for (int64_t t = 0; t < len; ++t)
            if (u == 0 || seg[u - 1] != seg[t]) seg[u++] = seg[t];
        memcpy(g->adj + g->off[v], seg, sizeof(int32_t) * (size_t)u);
        g->off[v + 1] = g->off[v] + u;
    }
    free(raw);
    free(fill);
    free(deg);
}

/* Eccentricity of src (the largest BFS distance), or -1 when some vertex is
 * unreachable.  *far receives a vertex at that distance. */
static int32_t orc_bfs_ecc(const orc_undirected *g, int64_t n, int64_t src, int32_t *dist, int32_t *queue,
                           int64_t *far)
{
    for (int64_t v = 0; v < n; ++v) dist[v] = -1;
    int64_t head = 0, tail = 0;
    dist[src] = 0;
    queue[tail++] = (int32_t)src;
    int32_t ecc = 0;
    int64_t last = src;
    while (head < tail) {
        int32_t v = queue[head++];
        for (int64_t q = g->off[v]; q < g->off[v + 1]; ++q) {
            int32_t w = g->adj[q];
            if (dist[w] >= 0) continue;
            dist[w] = dist[v] + 1;
            if (dist[w] > ecc) {
                ecc = dist[w];
                last = w;
            }
            queue[tail++] = w;
        }
    }
    if (far) *far = last;
    return tail == n ? ecc : -1;
}

/* Exact diameter by BFS from every vertex; -1 when disconnected. */
int32_t orc_diameter_exact(const int32_t *idx, int64_t n, int K)
{
    orc_undirected g;
    orc_undirected_build(idx, n, K, &g);
    int32_t diam = 0;
    int disconnected = 0;
#pragma omp parallel reduction(max : diam) reduction(| : disconnected)
    {
        int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
#pragma omp for schedule(dynamic, 16)
        for (int64_t s = 0; s < n; ++s) {
            int32_t e = orc_bfs_ecc(&g, n, s, dist, queue, NULL);
            if (e < 0)
                disconnected = 1;
            else if (e > diam)
                diam = e;
        }
        free(dist);
        free(queue);
    }
    free(g.off);
    free(g.adj);
    return disconnected ? -1 : diam;
}

/* Diameter bracket for large graphs: `sweeps` double sweeps (BFS from a
 * vertex, then from the farthest vertex found) give the lower bound (largest
 * eccentricity seen); the upper bound is 2 x the smallest eccentricity seen
 * (every distance passes within ecc(v) of any vertex v).  Start vertices
 * come from stream (seed, c0 = sweep, c1 = 0, c2 = 3). */
void orc_diameter_bounds(const int32_t *idx, int64_t n, int K, int32_t sweeps, uint64_t seed,
                         int32_t *lo, int32_t *hi)
{
    orc_undirected g;
    orc_undirected_build(idx, n, K, &g);
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t best_lo = 0, best_hi = -1;
    for (int32_t t = 0; t < sweeps; ++t) {
        orc_stream s;
        orc_stream_init(&s, seed, (uint32_t)t, 0u, 3u);
        int64_t src = orc_bounded(&s, (uint32_t)n), far = src;
        for (int rep = 0; rep < 2; ++rep) {
            int32_t e = orc_bfs_ecc(&g, n, src, dist, queue, &far);
            if (e < 0) {
                best_lo = -1;
                best_hi = -1;
                goto done;
            }
            if (e > best_lo) best_lo = e;
            if (best_hi < 0 || 2 * e < best_hi) best_hi = 2 * e;
            src = far;
        }
    }
done:
    *lo = best_lo;
    *hi = best_hi;
    free(dist);
    free(queue);
    free(g.off);
    free(g.adj);
}

int32_t orc_num_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}
