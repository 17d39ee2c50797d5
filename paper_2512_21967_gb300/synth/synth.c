/*
 * Seeded synthetic graph inputs: R-MAT and 4-neighbour grid edge lists, a
 * Fisher-Yates relabel, and the symmetrise / drop-loops / dedup step that turns
 * an edge list into a sorted int32 CSR.
 *
 * This module holds no breadth-first-search arithmetic.  Both the CPU oracle and
 * the CUDA path are fed from what it produces, so the two always see the same
 * graph.
 *
 * Every random draw is SplitMix64 used as a counter-based generator: draw i of a
 * stream with seed S is  mix(S + (i + 1) * 0x9E3779B97F4A7C15),  where mix is the
 * SplitMix64 output finaliser (Steele, Lea and Flood, OOPSLA 2014; constants as
 * published by Vigna).  Indexing draws by a counter makes the multi-threaded
 * generators produce the same bits as a sequential loop.
 *
 * Build: gcc -O3 -shared -fPIC -pthread synth.c -o libsynth.so
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define SM64_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t sm64_draw(uint64_t seed, uint64_t i) {
    return sm64_mix(seed + (i + 1) * SM64_GAMMA);
}

/* uniform double in [0, 1) from the top 53 bits */
static inline double sm64_unit(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

/* value in [0, bound) by the multiply-high map (Lemire); bias < bound / 2^64 */
static inline uint64_t sm64_bounded(uint64_t x, uint64_t bound) {
    return (uint64_t)(((unsigned __int128)x * (unsigned __int128)bound) >> 64);
}

uint64_t synth_draw(uint64_t seed, uint64_t i) { return sm64_draw(seed, i); }

void synth_draw_many(uint64_t seed, uint64_t start, int64_t count, uint64_t* out) {
    for (int64_t k = 0; k < count; ++k) out[k] = sm64_draw(seed, start + (uint64_t)k);
}

/* ------------------------------------------------------------------ threads */

typedef void (*range_fn)(void* ctx, int64_t lo, int64_t hi);
typedef struct { range_fn fn; void* ctx; int64_t lo, hi; } range_job;

static void* range_trampoline(void* p) {
    range_job* j = (range_job*)p;
    j->fn(j->ctx, j->lo, j->hi);
    return NULL;
}

static void parallel_range(int nthreads, int64_t n, range_fn fn, void* ctx) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (n < 4096 || nthreads == 1) { fn(ctx, 0, n); return; }
    pthread_t th[256];
    range_job jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].fn = fn; jobs[t].ctx = ctx;
        jobs[t].lo = n * t / nthreads; jobs[t].hi = n * (t + 1) / nthreads;
        if (pthread_create(&th[t], NULL, range_trampoline, &jobs[t]) != 0) {
            range_trampoline(&jobs[t]);          /* run inline if a thread cannot start */
            jobs[t].fn = NULL;
        }
    }
    for (int t = 0; t < nthreads; ++t) if (jobs[t].fn) pthread_join(th[t], NULL);
}

/* -------------------------------------------------------------------- R-MAT */

typedef struct {
    int scale; double a, ab, abc; uint64_t seed; int32_t* src; int32_t* dst;
} rmat_ctx;

static void rmat_range(void* p, int64_t lo, int64_t hi) {
    rmat_ctx* c = (rmat_ctx*)p;
    for (int64_t e = lo; e < hi; ++e) {
        uint32_t s = 0, d = 0;
        for (int b = 0; b < c->scale; ++b) {
            double u = sm64_unit(sm64_draw(c->seed, (uint64_t)e * (uint64_t)c->scale + (uint64_t)b));
            uint32_t bit = 1u << (c->scale - 1 - b);
            if (u < c->a) {
            } else if (u < c->ab) {
                d |= bit;
            } else if (u < c->abc) {
                s |= bit;
            } else {
                s |= bit; d |= bit;
            }
        }
        c->src[e] = (int32_t)s;
        c->dst[e] = (int32_t)d;
    }
}

/* m edges of a recursive-matrix graph on 2^scale vertices with quadrant
 * probabilities (a, b, c, 1-a-b-c); edge e consumes draws e*scale .. e*scale+scale-1,
 * the first one choosing the most significant bit.  Returns 0, or -1 on bad input. */
int synth_rmat_edges(int scale, int64_t m, double a, double b, double c, uint64_t seed,
                     int32_t* src, int32_t* dst, int nthreads) {
    if (scale < 1 || scale > 30 || m < 0 || a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return -1;
    rmat_ctx ctx = {scale, a, a + b, a + b + c, seed, src, dst};
    parallel_range(nthreads, m, rmat_range, &ctx);
    return 0;
}

/* ---------------------------------------------------------------- relabel */

/* perm[v] = new label of vertex v.  Fisher-Yates from the top: step t (t = 0..n-2)
 * handles i = n-1-t and swaps perm[i] with perm[j], j = bounded(draw t, i+1). */
void synth_permutation(int64_t n, uint64_t seed, int32_t* perm) {
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t t = 0; t + 1 < n; ++t) {
        int64_t i = n - 1 - t;
        int64_t j = (int64_t)sm64_bounded(sm64_draw(seed, (uint64_t)t), (uint64_t)(i + 1));
        int32_t tmp = perm[i]; perm[i] = perm[j]; perm[j] = tmp;
    }
}

/* --------------------------------------------------------------------- grid */

/* Vertex (r, c) of a side x side grid has id r*side + c.  Horizontal edge
 * (r,c)-(r,c+1) has index r*(side-1)+c; vertical edge (r,c)-(r+1,c) has index
 * side*(side-1) + r*side + c.  Edge with index i is kept iff unit(draw i) < p.
 * Writes the kept edges in index order and returns their count. */
int64_t synth_grid_edges(int32_t side, double p, uint64_t seed, int32_t* src, int32_t* dst) {
    if (side < 1) return -1;
    int64_t k = 0, S = side;
    int64_t nh = S * (S - 1);
    for (int64_t r = 0; r < S; ++r)
        for (int64_t c = 0; c + 1 < S; ++c) {
            uint64_t idx = (uint64_t)(r * (S - 1) + c);
            if (sm64_unit(sm64_draw(seed, idx)) < p) { src[k] = (int32_t)(r * S + c); dst[k] = (int32_t)(r * S + c + 1); ++k; }
        }
    for (int64_t r = 0; r + 1 < S; ++r)
        for (int64_t c = 0; c < S; ++c) {
            uint64_t idx = (uint64_t)(nh + r * S + c);
            if (sm64_unit(sm64_draw(seed, idx)) < p) { src[k] = (int32_t)(r * S + c); dst[k] = (int32_t)((r + 1) * S + c); ++k; }
        }
    return k;
}

/* ---------------------------------------------------------------------- CSR */

static void insertion_sort_i32(int32_t* a, int64_t len) {
    for (int64_t i = 1; i < len; ++i) {
        int32_t x = a[i];
        int64_t j = i - 1;
        while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; --j; }
        a[j + 1] = x;
    }
}

/* LSD radix sort of non-negative int32 keys, 3 passes of 11 bits, tmp >= len. */
static void radix_sort_i32(int32_t* a, int64_t len, int32_t* tmp) {
    int32_t* from = a; int32_t* to = tmp;
    for (int pass = 0; pass < 3; ++pass) {
        int64_t cnt[2049];
        memset(cnt, 0, sizeof(cnt));
        int sh = pass * 11;
        for (int64_t i = 0; i < len; ++i) cnt[(((uint32_t)from[i]) >> sh & 2047u) + 1]++;
        for (int b = 0; b < 2048; ++b) cnt[b + 1] += cnt[b];
        for (int64_t i = 0; i < len; ++i) to[cnt[((uint32_t)from[i]) >> sh & 2047u]++] = from[i];
        int32_t* t = from; from = to; to = t;
    }
    if (from != a) memcpy(a, from, (size_t)len * sizeof(int32_t));
}

typedef struct {
    const int64_t* rp; int32_t* col; int64_t* newdeg; int64_t maxlen;
    volatile int64_t next_row; int64_t n; pthread_mutex_t mu;
} sortrows_ctx;

static void sort_rows_range(sortrows_ctx* c, int32_t* tmp) {
    for (;;) {
        int64_t lo;
        pthread_mutex_lock(&c->mu);
        lo = c->next_row; c->next_row += 4096;
        pthread_mutex_unlock(&c->mu);
        if (lo >= c->n) break;
        int64_t hi = lo + 4096 < c->n ? lo + 4096 : c->n;
        for (int64_t u = lo; u < hi; ++u) {
            int32_t* a = c->col + c->rp[u];
            int64_t len = c->rp[u + 1] - c->rp[u];
            if (len <= 48) insertion_sort_i32(a, len); else radix_sort_i32(a, len, tmp);
            int64_t w = 0;
            for (int64_t i = 0; i < len; ++i)
                if (w == 0 || a[w - 1] != a[i]) a[w++] = a[i];
            c->newdeg[u] = w;
        }
    }
}

typedef struct { sortrows_ctx* c; } sortrows_arg;
static void* sort_rows_thread(void* p) {
    sortrows_ctx* c = ((sortrows_arg*)p)->c;
    int32_t* tmp = (int32_t*)malloc((size_t)(c->maxlen > 0 ? c->maxlen : 1) * sizeof(int32_t));
    if (tmp) sort_rows_range(c, tmp);
    free(tmp);
    return NULL;
}

/* Builds the CSR of the undirected simple graph on n vertices given by m edges:
 * each (s, d) with s != d is stored in both directions, self-loops are dropped,
 * duplicates removed, and every row sorted ascending.  If relabel is not NULL,
 * endpoints are first mapped through it.  row_ptr has n+1 entries; *col_out is
 * allocated with malloc (free with synth_free).  Returns 0, -1 on bad input,
 * -2 when out of memory, -3 when the result has 2^31 or more entries. */
int synth_build_csr(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, const int32_t* relabel,
                    int32_t* row_ptr, int32_t** col_out, int64_t* nnz_out, int nthreads) {
    if (n < 0 || m < 0 || !row_ptr || !col_out || !nnz_out) return -1;
    *col_out = NULL; *nnz_out = 0;
    int64_t* deg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!deg) return -2;
    for (int64_t e = 0; e < m; ++e) {
        int64_t s = src[e], d = dst[e];
        if (s < 0 || s >= n || d < 0 || d >= n) { free(deg); return -1; }
        if (relabel) { s = relabel[s]; d = relabel[d]; }
        if (s == d) continue;
        deg[s]++; deg[d]++;
    }
    int64_t* rp = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!rp) { free(deg); return -2; }
    rp[0] = 0;
    int64_t maxlen = 0;
    for (int64_t u = 0; u < n; ++u) { rp[u + 1] = rp[u] + deg[u]; if (deg[u] > maxlen) maxlen = deg[u]; }
    int64_t total = rp[n];
    int32_t* col = (int32_t*)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
    if (!col) { free(deg); free(rp); return -2; }
    for (int64_t u = 0; u < n; ++u) deg[u] = rp[u];
    for (int64_t e = 0; e < m; ++e) {
        int64_t s = src[e], d = dst[e];
        if (relabel) { s = relabel[s]; d = relabel[d]; }
        if (s == d) continue;
        col[deg[s]++] = (int32_t)d;
        col[deg[d]++] = (int32_t)s;
    }
    /* sort + dedup every row; newdeg reuses deg */
    sortrows_ctx ctx;
    ctx.rp = rp; ctx.col = col; ctx.newdeg = deg; ctx.maxlen = maxlen; ctx.next_row = 0; ctx.n = n;
    pthread_mutex_init(&ctx.mu, NULL);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256]; sortrows_arg arg = {&ctx}; int ok[256];
    for (int t = 0; t < nthreads; ++t) ok[t] = pthread_create(&th[t], NULL, sort_rows_thread, &arg) == 0;
    for (int t = 0; t < nthreads; ++t) if (ok[t]) pthread_join(th[t], NULL);
    int any = 0;
    for (int t = 0; t < nthreads; ++t) any |= ok[t];
    if (!any) sort_rows_thread(&arg);
    pthread_mutex_destroy(&ctx.mu);
    /* compact */
    int64_t w = 0;
    for (int64_t u = 0; u < n; ++u) {
        int64_t len = deg[u], base = rp[u];
        if (w != base) memmove(col + w, col + base, (size_t)len * sizeof(int32_t));
        rp[u] = w;
        w += len;
    }
    rp[n] = w;
    free(deg);
    if (w >= ((int64_t)1 << 31)) { free(rp); free(col); return -3; }
    for (int64_t u = 0; u <= n; ++u) row_ptr[u] = (int32_t)rp[u];
    free(rp);
    int32_t* shrunk = (int32_t*)realloc(col, (size_t)(w > 0 ? w : 1) * sizeof(int32_t));
    *col_out = shrunk ? shrunk : col;
    *nnz_out = w;
    return 0;
}

void synth_free(void* p) { free(p); }

/* ------------------------------------------------------------- components */

static int32_t uf_find(int32_t* parent, int32_t x) {
    while (parent[x] != x) { parent[x] = parent[parent[x]]; x = parent[x]; }
    return x;
}

/* comp[v] = smallest vertex id in v's connected component. */
void synth_components(int64_t n, const int32_t* row_ptr, const int32_t* col, int32_t* comp) {
    for (int64_t v = 0; v < n; ++v) comp[v] = (int32_t)v;
    for (int64_t u = 0; u < n; ++u)
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t a = uf_find(comp, (int32_t)u), b = uf_find(comp, col[e]);
            if (a != b) { if (a < b) comp[b] = a; else comp[a] = b; }
        }
    for (int64_t v = 0; v < n; ++v) comp[v] = uf_find(comp, (int32_t)v);
}
