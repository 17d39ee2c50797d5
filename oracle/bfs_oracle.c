/*
 * ORACLE -- test infrastructure only.  Nothing in the product path may link,
 * load or call this file; only the tests, the smoke check and the benchmark's
 * CPU-baseline leg do.
 *
 * Plain FIFO-queue breadth-first search on a CSR graph, on the original vertex
 * order.  level[v] is the length of a shortest src -> v path (the "level array"
 * form of the output in Section 2, Background and Notation), and -1 when v is
 * unreachable.  Shortest-path lengths are unique, so there is exactly one
 * correct level array per (graph, src).
 *
 * Build: gcc -O2 -shared -fPIC -pthread bfs_oracle.c -o liboracle.so
 */
#include <stdint.h>
#include <stdlib.h>
#include <pthread.h>

/* Returns the number of reached vertices (>= 1), or -1 if src is out of range.
 * queue must hold n entries. */
int64_t oracle_bfs(int64_t n, const int32_t* row_ptr, const int32_t* col, int32_t src,
                   int32_t* level, int32_t* queue) {
    if (src < 0 || src >= n) return -1;
    for (int64_t v = 0; v < n; ++v) level[v] = -1;
    int64_t head = 0, tail = 0;
    level[src] = 0;
    queue[tail++] = src;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t v = col[e];
            if (level[v] < 0) {
                level[v] = level[u] + 1;
                queue[tail++] = v;
            }
        }
    }
    return tail;
}

/* k independent runs, levels[i*n + v] for source srcs[i]; sources are handed
 * to nthreads worker threads (one whole BFS per source, no shared state). */
typedef struct {
    int64_t n; const int32_t* rp; const int32_t* col; const int32_t* srcs; int32_t* levels;
    int64_t k; int64_t next; pthread_mutex_t mu; int64_t bad;
} many_ctx;

static void* many_worker(void* p) {
    many_ctx* c = (many_ctx*)p;
    int32_t* q = (int32_t*)malloc((size_t)(c->n > 0 ? c->n : 1) * sizeof(int32_t));
    if (!q) return NULL;
    for (;;) {
        pthread_mutex_lock(&c->mu);
        int64_t i = c->next++;
        pthread_mutex_unlock(&c->mu);
        if (i >= c->k) break;
        if (oracle_bfs(c->n, c->rp, c->col, c->srcs[i], c->levels + i * c->n, q) < 0) {
            pthread_mutex_lock(&c->mu); c->bad++; pthread_mutex_unlock(&c->mu);
        }
    }
    free(q);
    return NULL;
}

int64_t oracle_bfs_many(int64_t n, const int32_t* row_ptr, const int32_t* col, int64_t k,
                        const int32_t* srcs, int32_t* levels, int nthreads) {
    many_ctx c;
    c.n = n; c.rp = row_ptr; c.col = col; c.srcs = srcs; c.levels = levels; c.k = k; c.next = 0; c.bad = 0;
    pthread_mutex_init(&c.mu, NULL);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 512) nthreads = 512;
    pthread_t th[512]; int ok[512];
    for (int t = 0; t < nthreads; ++t) ok[t] = pthread_create(&th[t], NULL, many_worker, &c) == 0;
    int any = 0;
    for (int t = 0; t < nthreads; ++t) if (ok[t]) { pthread_join(th[t], NULL); any = 1; }
    if (!any) many_worker(&c);
    pthread_mutex_destroy(&c.mu);
    return c.bad ? -1 : 0;
}
