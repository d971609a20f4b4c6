/*
 * oracle.c -- plain, serial, obviously-correct CPU reference for the
 * traversal results.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check
 * and the benchmark's CPU-baseline leg call it; the CUDA library never does.
 * It shares no code, header or helper with the CUDA path.
 *
 * What it computes (definitions from the paper):
 *  - oracle_bfs: hop distance from a source (Sec. 2.2, "the output distance
 *    is the hop distance from the source"), computed by the standard
 *    sequential queue-based BFS that the paper uses as its sequential
 *    baseline (Sec. 4, Setup; BFS table, column marked "*").  Unreachable
 *    vertices get 0xFFFFFFFF.
 *  - oracle_reach: reachability search (Sec. 2.1: all vertices reachable
 *    from a given vertex), for up to 64 sources at once as one bit per
 *    source, one plain BFS per source.  The backward search (which sources
 *    reach v) is the same search on the reversed graph.
 *  - oracle_floyd_warshall / oracle_warshall: brute-force all-pairs hop
 *    distances and transitive closure for tiny graphs; they pin the queue
 *    BFS itself (an independent definition of the same quantities).
 *  - oracle_transpose: reversed CSR, written here independently.
 *  - oracle_sssp: single-source shortest paths with non-negative integer
 *    arc weights (Sec. 2.2, the SSSP paragraph: the output is each vertex's
 *    shortest-path distance from the source), by Dijkstra's algorithm with
 *    a binary heap; 64-bit distances, 0xFFFFFFFFFFFFFFFF if unreachable.
 *  - oracle_floyd_warshall_w: brute-force all-pairs weighted distances for
 *    tiny graphs; it pins oracle_sssp by an independent definition.
 *  - oracle_scc: strongly connected components (Sec. 2: a maximal vertex
 *    set in which every vertex reaches every other) by Tarjan's algorithm,
 *    the paper's sequential SCC baseline (Sec. 4, Setup); each vertex is
 *    labelled with the smallest vertex id of its component.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_INF 0xFFFFFFFFu

/* Sequential FIFO-queue BFS.  Returns 0 on success, -1 on bad input. */
int oracle_bfs(uint32_t n, const uint32_t *offsets, const uint32_t *indices, uint32_t src,
               uint32_t *dist) {
    if (n == 0 || src >= n || !offsets || !dist) return -1;
    uint32_t *queue = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    if (!queue) return -2;
    for (uint32_t v = 0; v < n; v++) dist[v] = OR_INF;
    uint32_t head = 0, tail = 0;
    dist[src] = 0;
    queue[tail++] = src;
    while (head < tail) {
        uint32_t u = queue[head++];
        for (uint32_t e = offsets[u]; e < offsets[u + 1]; e++) {
            uint32_t w = indices[e];
            if (dist[w] == OR_INF) {
                dist[w] = dist[u] + 1;
                queue[tail++] = w;
            }
        }
    }
    free(queue);
    return 0;
}

/* k independent BFS runs; dist is k*n, source-major. */
int oracle_bfs_multi(uint32_t n, const uint32_t *offsets, const uint32_t *indices,
                     const uint32_t *srcs, uint32_t k, uint32_t *dist) {
    for (uint32_t j = 0; j < k; j++) {
        int rc = oracle_bfs(n, offsets, indices, srcs[j], dist + (size_t)j * n);
        if (rc) return rc;
    }
    return 0;
}

/* Reversed graph: arc u->w becomes w->u.  Lists come out sorted because
   sources are scanned in ascending order. */
int oracle_transpose(uint32_t n, const uint32_t *offsets, const uint32_t *indices,
                     uint32_t *t_offsets, uint32_t *t_indices) {
    uint32_t m = offsets[n];
    uint32_t *count = (uint32_t *)calloc((size_t)n + 1, sizeof(uint32_t));
    if (!count) return -2;
    for (uint32_t e = 0; e < m; e++) count[indices[e]]++;
    t_offsets[0] = 0;
    for (uint32_t v = 0; v < n; v++) t_offsets[v + 1] = t_offsets[v] + count[v];
    for (uint32_t v = 0; v < n; v++) count[v] = t_offsets[v];
    for (uint32_t u = 0; u < n; u++)
        for (uint32_t e = offsets[u]; e < offsets[u + 1]; e++)
            t_indices[count[indices[e]]++] = u;
    free(count);
    return 0;
}

/*
 * Reachability for k <= 64 sources: bit j of mask[v] is set iff v is
 * reachable from srcs[j] (v = srcs[j] included).  One BFS per source.
 */
int oracle_reach(uint32_t n, const uint32_t *offsets, const uint32_t *indices,
                 const uint32_t *srcs, uint32_t k, uint64_t *mask) {
    if (n == 0 || k == 0 || k > 64) return -1;
    uint32_t *dist = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    if (!dist) return -2;
    memset(mask, 0, (size_t)n * sizeof(uint64_t));
    for (uint32_t j = 0; j < k; j++) {
        int rc = oracle_bfs(n, offsets, indices, srcs[j], dist);
        if (rc) { free(dist); return rc; }
        for (uint32_t v = 0; v < n; v++)
            if (dist[v] != OR_INF) mask[v] |= (uint64_t)1 << j;
    }
    free(dist);
    return 0;
}

/* Backward reachability: bit j of mask[v] set iff srcs[j] is reachable from v. */
int oracle_reach_backward(uint32_t n, const uint32_t *offsets, const uint32_t *indices,
                          const uint32_t *srcs, uint32_t k, uint64_t *mask) {
    uint32_t m = offsets[n];
    uint32_t *toff = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    uint32_t *tidx = (uint32_t *)malloc((size_t)(m ? m : 1) * sizeof(uint32_t));
    if (!toff || !tidx) { free(toff); free(tidx); return -2; }
    oracle_transpose(n, offsets, indices, toff, tidx);
    int rc = oracle_reach(n, toff, tidx, srcs, k, mask);
    free(toff); free(tidx);
    return rc;
}

/*
 * Floyd-Warshall on hop counts (every arc weight 1, self-distance 0):
 * D[i*n+j] = number of arcs on a shortest i->j path, or 0xFFFFFFFF.
 */
int oracle_floyd_warshall(uint32_t n, const uint32_t *offsets, const uint32_t *indices,
                          uint32_t *D) {
    if (n == 0 || n > 4096) return -1;
    for (uint32_t i = 0; i < n; i++)
        for (uint32_t j = 0; j < n; j++) D[(size_t)i * n + j] = (i == j) ? 0 : OR_INF;
    for (uint32_t u = 0; u < n; u++)
        for (uint32_t e = offsets[u]; e < offsets[u + 1]; e++)
            if (indices[e] != u) D[(size_t)u * n + indices[e]] = 1;
    for (uint32_t k = 0; k < n; k++)
        for (uint32_t i = 0; i < n; i++) {
            uint32_t dik = D[(size_t)i * n + k];
            if (dik == OR_INF) continue;
            for (uint32_t j = 0; j < n; j++) {
                uint32_t dkj = D[(size_t)k * n + j];
                if (dkj == OR_INF) continue;
                if (dik + dkj < D[(size_t)i * n + j]) D[(size_t)i * n + j] = dik + dkj;
            }
        }
    return 0;
}

/* Warshall transitive closure with reflexivity: R[i*n+j] = 1 iff j reachable from i. */
int oracle_warshall(uint32_t n, const uint32_t *offsets, const uint32_t *indices, uint8_t *R) {
    if (n == 0 || n > 4096) return -1;
    memset(R, 0, (size_t)n * n);
    for (uint32_t i = 0; i < n; i++) R[(size_t)i * n + i] = 1;
    for (uint32_t u = 0; u < n; u++)
        for (uint32_t e = offsets[u]; e < offsets[u + 1]; e++) R[(size_t)u * n + indices[e]] = 1;
    for (uint32_t k = 0; k < n; k++)
        for (uint32_t i = 0; i < n; i++)
            if (R[(size_t)i * n + k])
                for (uint32_t j = 0; j < n; j++)
                    if (R[(size_t)k * n + j]) R[(size_t)i * n + j] = 1;
    return 0;
}

/*
 * Traversed-edge count used for TEPS: m_r = sum of out-degrees of the
 * vertices the search reached (dist != 0xFFFFFFFF).  n_r is returned too.
 */
void oracle_reached_edges(uint32_t n, const uint32_t *offsets, const uint32_t *dist,
                          uint64_t *n_r, uint64_t *m_r) {
    uint64_t a = 0, b = 0;
    for (uint32_t v = 0; v < n; v++)
        if (dist[v] != OR_INF) { a++; b += offsets[v + 1] - offsets[v]; }
    *n_r = a; *m_r = b;
}

/* Strongly connected components by Tarjan's algorithm (Tarjan 1972), the
 * paper's sequential SCC baseline (Sec. 4, Setup).  Iterative: an explicit
 * DFS stack of (vertex, next arc) frames replaces the recursion.  label[v]
 * is the smallest vertex id in v's component.  Returns 0, or -1/-2 on bad
 * input / no memory. */
int oracle_scc(uint32_t n, const uint32_t *offsets, const uint32_t *indices, uint32_t *label) {
    if (n == 0 || !offsets || !label) return -1;
    uint32_t *index = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint32_t *low = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint8_t *on = (uint8_t *)calloc(n, 1);
    uint32_t *comp = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));   /* Tarjan's stack */
    uint32_t *fv = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));     /* DFS frames: vertex */
    uint32_t *fe = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));     /*             next arc */
    if (!index || !low || !on || !comp || !fv || !fe) {
        free(index); free(low); free(on); free(comp); free(fv); free(fe);
        return -2;
    }
    for (uint32_t v = 0; v < n; v++) index[v] = OR_INF;
    uint32_t counter = 0, sp = 0, depth = 0;
    for (uint32_t s = 0; s < n; s++) {
        if (index[s] != OR_INF) continue;
        index[s] = low[s] = counter++;
        comp[sp++] = s; on[s] = 1;
        fv[0] = s; fe[0] = offsets[s]; depth = 1;
        while (depth) {
            const uint32_t v = fv[depth - 1];
            if (fe[depth - 1] < offsets[v + 1]) {
                const uint32_t w = indices[fe[depth - 1]++];
                if (index[w] == OR_INF) {            /* tree arc: descend */
                    index[w] = low[w] = counter++;
                    comp[sp++] = w; on[w] = 1;
                    fv[depth] = w; fe[depth] = offsets[w]; depth++;
                } else if (on[w] && index[w] < low[v]) {
                    low[v] = index[w];               /* arc back into the open stack */
                }
                continue;
            }
            /* all arcs of v done: v roots a component iff low == index */
            depth--;
            if (low[v] == index[v]) {
                uint32_t top = sp, mn = OR_INF;
                do { top--; if (comp[top] < mn) mn = comp[top]; } while (comp[top] != v);
                for (uint32_t i = top; i < sp; i++) { on[comp[i]] = 0; label[comp[i]] = mn; }
                sp = top;
            }
            if (depth) {
                const uint32_t p = fv[depth - 1];
                if (low[v] < low[p]) low[p] = low[v];
            }
        }
    }
    free(index); free(low); free(on); free(comp); free(fv); free(fe);
    return 0;
}

/* ---------------------------------------------------------------- SSSP -- */
#define OR_INF64 0xFFFFFFFFFFFFFFFFull

typedef struct { uint64_t d; uint32_t v; } or_item;

static int item_less(or_item a, or_item b) { return a.d < b.d || (a.d == b.d && a.v < b.v); }

static void heap_push(or_item *h, size_t *size, or_item x) {
    size_t i = (*size)++;
    while (i > 0) {
        size_t p = (i - 1) / 2;
        if (!item_less(x, h[p])) break;
        h[i] = h[p];
        i = p;
    }
    h[i] = x;
}

static or_item heap_pop(or_item *h, size_t *size) {
    or_item top = h[0];
    or_item last = h[--(*size)];
    size_t i = 0;
    for (;;) {
        size_t c = 2 * i + 1;
        if (c >= *size) break;
        if (c + 1 < *size && item_less(h[c + 1], h[c])) c++;
        if (!item_less(h[c], last)) break;
        h[i] = h[c];
        i = c;
    }
    if (*size > 0) h[i] = last;
    return top;
}

/* Dijkstra: pop the closest unsettled vertex, relax its out-arcs.  Entries
 * whose distance is stale (a shorter one was pushed later) are skipped. */
int oracle_sssp(uint32_t n, const uint32_t *offsets, const uint32_t *indices, const uint32_t *weights,
                uint32_t src, uint64_t *dist) {
    if (n == 0 || src >= n || !offsets || !dist || (offsets[n] && (!indices || !weights))) return -1;
    const size_t cap = (size_t)offsets[n] + 1;
    or_item *heap = (or_item *)malloc(cap * sizeof(or_item));
    if (!heap) return -2;
    for (uint32_t v = 0; v < n; v++) dist[v] = OR_INF64;
    size_t size = 0;
    dist[src] = 0;
    or_item s0 = {0, src};
    heap_push(heap, &size, s0);
    while (size > 0) {
        or_item it = heap_pop(heap, &size);
        if (it.d != dist[it.v]) continue; /* stale */
        for (uint32_t e = offsets[it.v]; e < offsets[it.v + 1]; e++) {
            const uint32_t x = indices[e];
            const uint64_t nd = it.d + weights[e];
            if (nd < dist[x]) {
                dist[x] = nd;
                or_item y = {nd, x};
                heap_push(heap, &size, y); /* at most one push per arc */
            }
        }
    }
    free(heap);
    return 0;
}

/* All-pairs weighted distances, D[i*n + j], by Floyd-Warshall (n <= 64). */
int oracle_floyd_warshall_w(uint32_t n, const uint32_t *offsets, const uint32_t *indices,
                            const uint32_t *weights, uint64_t *D) {
    if (n == 0 || n > 64 || !offsets || !D) return -1;
    for (uint32_t i = 0; i < n; i++)
        for (uint32_t j = 0; j < n; j++) D[(size_t)i * n + j] = (i == j) ? 0 : OR_INF64;
    for (uint32_t u = 0; u < n; u++)
        for (uint32_t e = offsets[u]; e < offsets[u + 1]; e++) {
            uint64_t *d = &D[(size_t)u * n + indices[e]];
            if (weights[e] < *d) *d = weights[e];
        }
    for (uint32_t k = 0; k < n; k++)
        for (uint32_t i = 0; i < n; i++) {
            const uint64_t dik = D[(size_t)i * n + k];
            if (dik == OR_INF64) continue;
            for (uint32_t j = 0; j < n; j++) {
                const uint64_t dkj = D[(size_t)k * n + j];
                if (dkj == OR_INF64) continue;
                if (dik + dkj < D[(size_t)i * n + j]) D[(size_t)i * n + j] = dik + dkj;
            }
        }
    return 0;
}
