/*
 * oracle.c -- plain, slow, serial CPU oracle for exact triangle counting.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this code.  It
 * shares no source, header, helper or table with the CUDA library, and the
 * CUDA library never calls it.
 *
 * Source: D. A. Bader, "Fast Triangle Counting" (arXiv 2309.09064).
 *
 *   oracle_build_csr        input format of the paper (Sec. III: one graph in
 *                           CSR, read-only): symmetric, no self-loops, no
 *                           duplicate edges, each row ascending.
 *   oracle_count_definition the plain definition of the triangle count
 *                           (Sec. I: triples of pairwise adjacent vertices),
 *                           each unordered triple counted once as the
 *                           increasing triple of a fixed total order.
 *   oracle_alg4             Algorithm 4 ("Fast Triangle Counting") step by
 *                           step: optional relabelling by decreasing degree
 *                           (Sec. II, last paragraph: "BaderD"), BFS from every
 *                           unvisited vertex in label order, partition of E
 *                           into E0 (horizontal) and E1, Algorithm 2
 *                           (forward-hashed) on G0, then the hashed G1
 *                           intersections over the G0 edges.
 *   oracle_alg3             Algorithm 3 (cover-edge triangle counting) with
 *                           its level rule, as an independent cross-check.
 *   oracle_vertex_counts    per-vertex triangle counts from the definition.
 *   oracle_list_definition  every triangle once, from the definition.
 *
 * Readings of points the paper leaves open (the same readings bind the CUDA
 * library):
 *   - Relabelling by decreasing degree: ties broken by ascending original id.
 *     The comparisons u < v inside Algorithms 2-4 compare the new labels.
 *   - BFS roots: the outer loop, a BFS from every vertex still unvisited, visits
 *     vertices in label order, so each component's root is its first vertex
 *     in that order (highest degree, then lowest id, in the degree order).
 *   - The Hash[] array is indexed by vertex id, so it has n entries (the text
 *     sizes it by m, which cannot index vertices).
 *   - Isolated vertices are their own BFS roots, at level 0.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define UNVISITED 0xFFFFFFFFu

static int cmp_u32(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x > y) - (x < y);
}

/*
 * Build the CSR of the simple undirected graph spanned by the tuples: every
 * tuple (a, b) with a != b contributes b to row a and a to row b, then each
 * row is sorted and repeated entries dropped.  row_ptr has n+1 entries, col
 * must hold 2*t entries.  Returns the number of CSR slots (2m), or -1 if a
 * tuple names a vertex >= n.
 */
int64_t oracle_build_csr(uint32_t n, uint64_t t, const uint32_t *src, const uint32_t *dst,
                         uint64_t *row_ptr, uint32_t *col)
{
    for (uint64_t i = 0; i < t; ++i)
        if (src[i] >= n || dst[i] >= n) return -1;
    uint64_t *fill = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    memset(row_ptr, 0, sizeof(uint64_t) * ((size_t)n + 1));
    for (uint64_t i = 0; i < t; ++i) {
        if (src[i] == dst[i]) continue;
        row_ptr[src[i] + 1]++;
        row_ptr[dst[i] + 1]++;
    }
    for (uint32_t v = 0; v < n; ++v) row_ptr[v + 1] += row_ptr[v];
    for (uint32_t v = 0; v < n; ++v) fill[v] = row_ptr[v];
    for (uint64_t i = 0; i < t; ++i) {
        uint32_t a = src[i], b = dst[i];
        if (a == b) continue;
        col[fill[a]++] = b;
        col[fill[b]++] = a;
    }
    /* sort each row, drop repeats, and pack the rows to the left */
    uint64_t out = 0;
    for (uint32_t v = 0; v < n; ++v) {
        uint64_t lo = row_ptr[v], hi = row_ptr[v + 1];
        qsort(col + lo, (size_t)(hi - lo), sizeof(uint32_t), cmp_u32);
        uint64_t start = out;
        for (uint64_t j = lo; j < hi; ++j)
            if (j == lo || col[j] != col[j - 1]) col[out++] = col[j];
        row_ptr[v] = start;
    }
    row_ptr[n] = out;
    free(fill);
    return (int64_t)out;
}

/* ---------------------------------------------------------------- total orders */

static const uint64_t *g_rp; /* row pointers of the graph being ordered */

static uint64_t degree_of(uint32_t v) { return g_rp[v + 1] - g_rp[v]; }

/* decreasing degree, ties by ascending id */
static int cmp_degree_desc(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    uint64_t dx = degree_of(x), dy = degree_of(y);
    if (dx != dy) return dx > dy ? -1 : 1;
    return (x > y) - (x < y);
}

/*
 * order[p] = original id of the vertex with new label p.  degree_order != 0:
 * labels by decreasing degree (ties by id); otherwise the identity.
 */
static void make_order(uint32_t n, const uint64_t *rp, int degree_order, uint32_t *order)
{
    for (uint32_t v = 0; v < n; ++v) order[v] = v;
    if (degree_order) {
        g_rp = rp;
        qsort(order, n, sizeof(uint32_t), cmp_degree_desc);
    }
}

/* Relabel the CSR: vertex order[p] becomes p; rows re-sorted by new labels. */
static void relabel_csr(uint32_t n, const uint64_t *rp, const uint32_t *col, const uint32_t *order,
                        const uint32_t *newid, uint64_t *rp2, uint32_t *col2)
{
    rp2[0] = 0;
    for (uint32_t p = 0; p < n; ++p) {
        uint32_t old = order[p];
        uint64_t d = rp[old + 1] - rp[old];
        rp2[p + 1] = rp2[p] + d;
        for (uint64_t j = 0; j < d; ++j) col2[rp2[p] + j] = newid[col[rp[old] + j]];
        qsort(col2 + rp2[p], (size_t)d, sizeof(uint32_t), cmp_u32);
    }
}

/* --------------------------------------------------------------- the definition */

/*
 * Number of unordered triples {a, b, c} of pairwise adjacent vertices.  Each
 * triple is counted once as a < b < c in the total order "decreasing degree,
 * ties by ascending id" (any total order gives the same count; this one keeps
 * the lists short).  P(x) = neighbours of x that come before x.  For every c:
 * mark P(c); for every b in P(c) and every a in P(b), the triple a < b < c is
 * a triangle exactly when a is marked (a ~ c); unmark P(c).
 */
uint64_t oracle_count_definition(uint32_t n, const uint64_t *rp, const uint32_t *col)
{
    uint32_t *order = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    uint32_t *pos = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    make_order(n, rp, 1, order);
    for (uint32_t p = 0; p < n; ++p) pos[order[p]] = p;
    uint64_t *prp = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    prp[0] = 0;
    for (uint32_t x = 0; x < n; ++x) {
        uint64_t k = 0;
        for (uint64_t j = rp[x]; j < rp[x + 1]; ++j)
            if (pos[col[j]] < pos[x]) ++k;
        prp[x + 1] = prp[x] + k;
    }
    uint32_t *pcol = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)prp[n] + 1));
    for (uint32_t x = 0; x < n; ++x) {
        uint64_t k = prp[x];
        for (uint64_t j = rp[x]; j < rp[x + 1]; ++j)
            if (pos[col[j]] < pos[x]) pcol[k++] = col[j];
    }
    unsigned char *mark = (unsigned char *)calloc((size_t)n + 1, 1);
    uint64_t T = 0;
    for (uint32_t c = 0; c < n; ++c) {
        for (uint64_t j = prp[c]; j < prp[c + 1]; ++j) mark[pcol[j]] = 1;
        for (uint64_t j = prp[c]; j < prp[c + 1]; ++j) {
            uint32_t b = pcol[j];
            for (uint64_t i = prp[b]; i < prp[b + 1]; ++i)
                if (mark[pcol[i]]) ++T;
        }
        for (uint64_t j = prp[c]; j < prp[c + 1]; ++j) mark[pcol[j]] = 0;
    }
    free(order);
    free(pos);
    free(prp);
    free(pcol);
    free(mark);
    return T;
}

/*
 * Per-vertex triangle counts t(v) = number of triangles containing v, from the
 * same enumeration as oracle_count_definition (every found triple adds one to
 * each of its three vertices).  Returns T.
 */
uint64_t oracle_vertex_counts(uint32_t n, const uint64_t *rp, const uint32_t *col, uint64_t *tv)
{
    uint32_t *order = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    uint32_t *pos = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    make_order(n, rp, 1, order);
    for (uint32_t p = 0; p < n; ++p) pos[order[p]] = p;
    memset(tv, 0, sizeof(uint64_t) * (size_t)n);
    uint64_t T = 0;
    for (uint32_t b = 0; b < n; ++b)
        for (uint64_t j = rp[b]; j < rp[b + 1]; ++j) {
            uint32_t c = col[j];
            if (!(pos[b] < pos[c])) continue;
            uint64_t i1 = rp[b], e1 = rp[b + 1], i2 = rp[c], e2 = rp[c + 1];
            while (i1 < e1 && i2 < e2) {
                if (col[i1] < col[i2]) ++i1;
                else if (col[i1] > col[i2]) ++i2;
                else {
                    uint32_t a = col[i1];
                    if (pos[a] < pos[b]) { ++T; ++tv[a]; ++tv[b]; ++tv[c]; }
                    ++i1; ++i2;
                }
            }
        }
    free(order);
    free(pos);
    return T;
}

/*
 * Every triangle once, from the definition: the triples a < b < c (vertex
 * ids) of pairwise adjacent vertices, in lexicographic order -- for every a,
 * every neighbour b > a, and every common neighbour c > b of a and b (sorted
 * rows, one merge).  Writes the first min(T, cap) triples to out (3 ids
 * each) and returns T.
 */
uint64_t oracle_list_definition(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t *out, uint64_t cap)
{
    uint64_t T = 0;
    for (uint32_t a = 0; a < n; ++a)
        for (uint64_t j = rp[a]; j < rp[a + 1]; ++j) {
            uint32_t b = col[j];
            if (b <= a) continue;
            uint64_t i1 = rp[a], e1 = rp[a + 1], i2 = rp[b], e2 = rp[b + 1];
            while (i1 < e1 && i2 < e2) {
                if (col[i1] < col[i2]) ++i1;
                else if (col[i1] > col[i2]) ++i2;
                else {
                    uint32_t c = col[i1];
                    if (c > b) {
                        if (T < cap) {
                            out[3 * T] = a;
                            out[3 * T + 1] = b;
                            out[3 * T + 2] = c;
                        }
                        ++T;
                    }
                    ++i1; ++i2;
                }
            }
        }
    return T;
}

/* ------------------------------------------------------------------- BFS levels */

/*
 * A BFS from every vertex still unvisited (Algorithms 3 and 4), with
 * vertices taken in label order 0..n-1 of the (relabelled) CSR.  L[p] = hop
 * distance from the root of p's component.  Returns the number of levels
 * (max L + 1), 0 for an empty graph.
 */
static uint32_t bfs_all(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t *L)
{
    uint32_t *queue = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    uint32_t levels = 0;
    for (uint32_t v = 0; v < n; ++v) L[v] = UNVISITED;
    for (uint32_t s = 0; s < n; ++s) {
        if (L[s] != UNVISITED) continue;
        uint32_t head = 0, tail = 0;
        L[s] = 0;
        queue[tail++] = s;
        while (head < tail) {
            uint32_t x = queue[head++];
            if (L[x] + 1 > levels) levels = L[x] + 1;
            for (uint64_t j = rp[x]; j < rp[x + 1]; ++j) {
                uint32_t y = col[j];
                if (L[y] == UNVISITED) {
                    L[y] = L[x] + 1;
                    queue[tail++] = y;
                }
            }
        }
    }
    free(queue);
    return levels;
}

/* ------------------------------------------------------------------ Algorithm 4 */

/*
 * Algorithm 4.  out[0] = T, out[1] = triangles inside G0 (Algorithm 2 on G0),
 * out[2] = triangles found through the G1 intersections, out[3] = |E0|
 * (undirected horizontal edges), out[4] = number of BFS levels.  If L_out is
 * not NULL it receives the level of every ORIGINAL vertex id.  Returns 0, or
 * -1 on allocation failure.
 */
int oracle_alg4(uint32_t n, const uint64_t *rp_in, const uint32_t *col_in, int degree_order,
                uint32_t *L_out, uint64_t *out)
{
    const uint64_t slots = rp_in[n];
    uint32_t *order = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    uint32_t *newid = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    uint64_t *rp = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    uint32_t *col = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)slots + 1));
    uint32_t *L = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    if (!order || !newid || !rp || !col || !L) return -1;

    /* pre-processing: relabel by decreasing degree (BaderD) or keep ids (Bader) */
    make_order(n, rp_in, degree_order, order);
    for (uint32_t p = 0; p < n; ++p) newid[order[p]] = p;
    relabel_csr(n, rp_in, col_in, order, newid, rp, col);

    /* BFS from every unvisited vertex */
    uint32_t levels = bfs_all(n, rp, col, L);

    /* partition E into G0 (L(u) == L(v)) and G1 (the rest), both kept as CSR */
    uint64_t *rp0 = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    uint64_t *rp1 = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    for (uint32_t u = 0; u < n; ++u) {
        uint64_t k0 = 0, k1 = 0;
        for (uint64_t j = rp[u]; j < rp[u + 1]; ++j) {
            if (L[col[j]] == L[u]) ++k0; else ++k1;
        }
        rp0[u + 1] = rp0[u] + k0;
        rp1[u + 1] = rp1[u] + k1;
    }
    uint32_t *c0 = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)rp0[n] + 1));
    uint32_t *c1 = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)rp1[n] + 1));
    for (uint32_t u = 0; u < n; ++u) {
        uint64_t k0 = rp0[u], k1 = rp1[u];
        for (uint64_t j = rp[u]; j < rp[u + 1]; ++j) {
            if (L[col[j]] == L[u]) c0[k0++] = col[j]; else c1[k1++] = col[j];
        }
    }

    unsigned char *Hash = (unsigned char *)calloc((size_t)n + 1, 1);

    /* T <- TC_forward-hashed(G0): Algorithm 2 over the edges of G0 in CSR order,
     * with the growing sets A(v) stored in per-vertex slices of size deg_G0(v). */
    uint64_t *afill = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    uint32_t *A = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)rp0[n] + 1));
    for (uint32_t v = 0; v < n; ++v) afill[v] = rp0[v];
    uint64_t t_same = 0;
    for (uint32_t u = 0; u < n; ++u) {
        for (uint64_t j = rp0[u]; j < rp0[u + 1]; ++j) {
            uint32_t v = c0[j];
            if (!(u < v)) continue;
            for (uint64_t a = rp0[u]; a < afill[u]; ++a) Hash[A[a]] = 1;
            for (uint64_t a = rp0[v]; a < afill[v]; ++a)
                if (Hash[A[a]]) ++t_same;
            for (uint64_t a = rp0[u]; a < afill[u]; ++a) Hash[A[a]] = 0;
            A[afill[v]++] = u;
        }
    }

    /* triangles not wholly in G0: for every u, hash N_G1(u); for each G0 edge
     * (u, v) with u < v, probe N_G1(v); then clear the hash */
    uint64_t t_cross = 0;
    for (uint32_t u = 0; u < n; ++u) {
        for (uint64_t j = rp1[u]; j < rp1[u + 1]; ++j) Hash[c1[j]] = 1;
        for (uint64_t j = rp0[u]; j < rp0[u + 1]; ++j) {
            uint32_t v = c0[j];
            if (!(u < v)) continue;
            for (uint64_t k = rp1[v]; k < rp1[v + 1]; ++k)
                if (Hash[c1[k]]) ++t_cross;
        }
        for (uint64_t j = rp1[u]; j < rp1[u + 1]; ++j) Hash[c1[j]] = 0;
    }

    out[0] = t_same + t_cross;
    out[1] = t_same;
    out[2] = t_cross;
    out[3] = rp0[n] / 2;
    out[4] = levels;
    if (L_out)
        for (uint32_t v = 0; v < n; ++v) L_out[v] = L[newid[v]];

    free(order); free(newid); free(rp); free(col); free(L);
    free(rp0); free(rp1); free(c0); free(c1); free(Hash); free(afill); free(A);
    return 0;
}

/* ------------------------------------------------------------------ Algorithm 3 */

/*
 * Algorithm 3 (cover-edge triangle counting): BFS as above; for every edge
 * (u, v) with L(u) == L(v) and u < v, every w in N(u) n N(v) is counted when
 * L(u) != L(w), or when L(u) == L(w) and v < w.  Returns T.
 */
uint64_t oracle_alg3(uint32_t n, const uint64_t *rp_in, const uint32_t *col_in, int degree_order)
{
    const uint64_t slots = rp_in[n];
    uint32_t *order = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    uint32_t *newid = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    uint64_t *rp = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    uint32_t *col = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)slots + 1));
    uint32_t *L = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    make_order(n, rp_in, degree_order, order);
    for (uint32_t p = 0; p < n; ++p) newid[order[p]] = p;
    relabel_csr(n, rp_in, col_in, order, newid, rp, col);
    bfs_all(n, rp, col, L);
    unsigned char *Hash = (unsigned char *)calloc((size_t)n + 1, 1);
    uint64_t T = 0;
    for (uint32_t u = 0; u < n; ++u) {
        for (uint64_t j = rp[u]; j < rp[u + 1]; ++j) {
            uint32_t v = col[j];
            if (!(L[u] == L[v] && u < v)) continue;
            for (uint64_t a = rp[u]; a < rp[u + 1]; ++a) Hash[col[a]] = 1;
            for (uint64_t b = rp[v]; b < rp[v + 1]; ++b) {
                uint32_t w = col[b];
                if (!Hash[w]) continue;
                if (L[u] != L[w] || (L[u] == L[w] && v < w)) ++T;
            }
            for (uint64_t a = rp[u]; a < rp[u + 1]; ++a) Hash[col[a]] = 0;
        }
    }
    free(order); free(newid); free(rp); free(col); free(L); free(Hash);
    return T;
}
