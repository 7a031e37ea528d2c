/*
 * oracle.c -- plain, slow, single-threaded CPU oracle for Pruned Landmark
 * Labeling (Akiba, Iwata, Yoshida, SIGMOD 2013).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the two meet only through
 * the graphs and query pairs handed to both by the input generators.
 *
 * What it computes, in the paper's order and notation:
 *   orc_degree_order   -- the Degree strategy of Sec. 4.4.2: vertices by
 *                         descending degree; ties by ascending vertex id.
 *   orc_build          -- Sec. 5.4: t bit-parallel BFSs (Alg. 3) from greedily
 *                         chosen roots r and neighbour sets S_r, then the
 *                         pruned BFSs of Alg. 2 / Alg. 1 in rank order, each
 *                         pruned by the bit-parallel query of Sec. 5.3 and the
 *                         normal label query evaluated with the root array T of
 *                         Sec. 4.5.1; labels store hub ranks (Sec. 4.5.1,
 *                         "Sorting Labels"), so they are sorted by construction.
 *   orc_query          -- Query(s, t, L) of Sec. 3.3 (merge join over sorted
 *                         labels) combined with the bit-parallel query.
 *   orc_query_batch_mt -- the same answers for many pairs, split over POSIX
 *                         threads (a timing aid for the all-core query rate;
 *                         every pair still goes through orc_query).
 *   orc_bfs            -- plain BFS distances (ground truth for queries).
 *   orc_label_of       -- the label L(u) that the method must produce for a
 *                         fixed order, computed directly from its closed form:
 *                         (v_j, d(v_j,u)) is in L(u) iff v_j is not a
 *                         bit-parallel vertex and no bit-parallel vertex and no
 *                         v_i with i < j lies on a shortest v_j-u path. This is
 *                         the content of the correctness proof (Thm 4.1) and the
 *                         minimality proof (Thm 4.2), extended to bit-parallel
 *                         pruning (Sec. 5.4). One BFS from u with a dynamic
 *                         program over shortest-path predecessors.
 *
 *   orc_export_parents -- Sec. 6, "Shortest-Path Queries": each label entry
 *                         (u, d) of L(v) also carries the parent of v in the
 *                         pruned BFS tree rooted at u (the vertex whose
 *                         expansion first reached v; u itself for (u, 0)).
 *   orc_path           -- one shortest s-t path restored from the labels: the
 *                         best common hub h of L(s) and L(t), then the tree of
 *                         h climbed from s and from t through those parents.
 *                         When only the bit-parallel label reaches the
 *                         distance, the path goes through r_i or a member of
 *                         S_{r_i}, whose distance to every vertex the label
 *                         gives exactly (Sec. 5.1); each step moves to the
 *                         first neighbour one hop nearer.
 *
 *   orc_build_directed -- Sec. 6, "Directed Graphs": labels L_IN and L_OUT
 *                         from a forward and a reverse pruned BFS per root;
 *   orc_dquery         -- d(s, t) from L_OUT(s) and L_IN(t).
 *
 *   orc_core_numbers   -- core number of every vertex (the largest k such that
 *                         the vertex lies in a subgraph of minimum degree k),
 *                         one of the vertex features of the learned order; the
 *                         paper has no counterpart. Bucket peeling in the
 *                         manner of Batagelj and Zaversnik (2003): repeatedly
 *                         remove a vertex of least remaining degree.
 *
 * Readings of the paper taken here (each one is listed in the design notes):
 *   - Alg. 1 appends (v_k, P[u]) to L(u) and expands N_G(u) (the printed
 *     algorithm has typos there); the prune test is "<=".
 *   - Roots that are bit-parallel vertices (a root r or a member of some S_r)
 *     get no pruned BFS: the bit-parallel query already returns 0 for them.
 *   - Bit-parallel roots: r = lowest-rank vertex not used yet; S_r = up to 64
 *     lowest-rank unused neighbours of r; bit j of a mask = j-th member of S_r
 *     in rank order. If no unused vertex is left, the slot holds distance 255
 *     and empty masks for every vertex.
 *   - Distances are 8-bit, 255 = unreachable; a finite distance >= 255 is a
 *     range error.
 *   - Stored S^0_r(v) is the set of Sec. 5.1 (difference exactly 0), i.e. the
 *     Alg. 3 result with the members of S^{-1}_r(v) removed.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_E_INVAL 1
#define ORC_E_ORDER 2
#define ORC_E_RANGE 3
#define ORC_E_NOMEM 4

#define INF8 255
#define NONE 0xffffffffu
#define BPW 64 /* bits in one bit-parallel word (b in Sec. 5) */

typedef struct orc_index {
    uint32_t n, t;
    uint32_t *order;  /* rank -> vertex */
    uint32_t *rank;   /* vertex -> rank */
    uint8_t *inX;     /* vertex is a bit-parallel root or neighbour */
    /* bit-parallel labels, vertex-major [n][t] */
    uint32_t *bp_root;  /* [t], NONE for an empty slot */
    uint32_t *bp_cnt;   /* [t] |S_r| */
    uint32_t *bp_S;     /* [t][64] members of S_r, vertex ids */
    uint8_t *bp_d;
    uint64_t *bp_m1;    /* S^{-1}_r(v) */
    uint64_t *bp_m0;    /* S^{0}_r(v) */
    /* normal labels, indexed by vertex id; hubs are ranks */
    uint32_t *len, *cap;
    uint32_t **hub;
    uint8_t **dist;
    uint32_t **par;     /* parent of the vertex in the hub's pruned BFS tree (Sec. 6) */
    /* counters of the work done by the pruned BFSs */
    uint64_t visited, labeled, scanned, labeled_deg;
} orc_index;

/* ------------------------------------------------------------ helpers */
static const uint32_t *g_deg_for_sort;
static int cmp_degree(const void *a, const void *b) {
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    uint32_t dx = g_deg_for_sort[x], dy = g_deg_for_sort[y];
    if (dx != dy) return dx > dy ? -1 : 1;   /* higher degree first */
    return x < y ? -1 : (x > y ? 1 : 0);    /* then smaller id */
}

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

static const uint32_t *g_rank_for_sort;
static int cmp_rank(const void *a, const void *b) {
    uint32_t x = g_rank_for_sort[*(const uint32_t *)a], y = g_rank_for_sort[*(const uint32_t *)b];
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Degree strategy (Sec. 4.4.2). order[rank] = vertex. */
int orc_degree_order(uint32_t n, const uint32_t *off, const uint32_t *col, uint32_t *order) {
    (void)col;
    uint32_t *deg = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    if (!deg) return ORC_E_NOMEM;
    for (uint32_t v = 0; v < n; ++v) { deg[v] = off[v + 1] - off[v]; order[v] = v; }
    g_deg_for_sort = deg;
    qsort(order, n, sizeof(uint32_t), cmp_degree);
    free(deg);
    return ORC_OK;
}

/* Plain BFS from src: dist[v] = d_G(src, v), 255 if unreachable.
 * Returns ORC_E_RANGE if some finite distance is >= 255. */
int orc_bfs(uint32_t n, const uint32_t *off, const uint32_t *col, uint32_t src, uint8_t *dist) {
    uint32_t *q = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    if (!q) return ORC_E_NOMEM;
    memset(dist, INF8, n);
    int st = ORC_OK;
    uint32_t head = 0, tail = 0;
    dist[src] = 0;
    q[tail++] = src;
    while (head < tail) {
        uint32_t v = q[head++];
        for (uint32_t e = off[v]; e < off[v + 1]; ++e) {
            uint32_t w = col[e];
            if (dist[w] != INF8) continue;
            if (dist[v] + 1 >= INF8) { st = ORC_E_RANGE; continue; }
            dist[w] = (uint8_t)(dist[v] + 1);
            q[tail++] = w;
        }
    }
    free(q);
    return st;
}

static int label_push(orc_index *ix, uint32_t u, uint32_t hub_rank, uint8_t d, uint32_t parent) {
    if (ix->len[u] == ix->cap[u]) {
        uint32_t nc = ix->cap[u] ? 2 * ix->cap[u] : 4;
        uint32_t *h = (uint32_t *)realloc(ix->hub[u], (size_t)nc * sizeof(uint32_t));
        if (!h) return ORC_E_NOMEM;
        ix->hub[u] = h;
        uint8_t *dd = (uint8_t *)realloc(ix->dist[u], nc);
        if (!dd) return ORC_E_NOMEM;
        ix->dist[u] = dd;
        uint32_t *pp = (uint32_t *)realloc(ix->par[u], (size_t)nc * sizeof(uint32_t));
        if (!pp) return ORC_E_NOMEM;
        ix->par[u] = pp;
        ix->cap[u] = nc;
    }
    ix->hub[u][ix->len[u]] = hub_rank;
    ix->dist[u][ix->len[u]] = d;
    ix->par[u][ix->len[u]] = parent;
    ix->len[u]++;
    return ORC_OK;
}

/* ------------------------------------------- Sec. 5.4: choosing r, S_r */
static int select_bp_roots(orc_index *ix, const uint32_t *off, const uint32_t *col) {
    uint32_t n = ix->n;
    uint32_t *cand = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    if (!cand) return ORC_E_NOMEM;
    uint32_t next = 0;
    for (uint32_t i = 0; i < ix->t; ++i) {
        while (next < n && ix->inX[ix->order[next]]) ++next;
        if (next == n) { ix->bp_root[i] = NONE; ix->bp_cnt[i] = 0; continue; }
        uint32_t r = ix->order[next];
        ix->bp_root[i] = r;
        ix->inX[r] = 1;
        uint32_t c = 0;
        for (uint32_t e = off[r]; e < off[r + 1]; ++e)
            if (!ix->inX[col[e]]) cand[c++] = col[e];
        g_rank_for_sort = ix->rank;
        qsort(cand, c, sizeof(uint32_t), cmp_rank);
        uint32_t take = c < BPW ? c : BPW;
        for (uint32_t j = 0; j < take; ++j) {
            ix->bp_S[(size_t)i * BPW + j] = cand[j];
            ix->inX[cand[j]] = 1;
        }
        ix->bp_cnt[i] = take;
    }
    free(cand);
    return ORC_OK;
}

/* ------------------------------------------- Alg. 3: Bp-BFS(G, r, S_r) */
static int bp_bfs(orc_index *ix, const uint32_t *off, const uint32_t *col, uint32_t i,
                  int *P, uint64_t *Sm1, uint64_t *S0, uint32_t *Q0, uint32_t *Q1,
                  uint32_t *E0, uint32_t *E1) {
    uint32_t n = ix->n, t = ix->t;
    uint32_t r = ix->bp_root[i];
    for (uint32_t v = 0; v < n; ++v) { P[v] = -1; Sm1[v] = 0; S0[v] = 0; } /* -1 = infinity */
    int st = ORC_OK;
    if (r != NONE) {
        uint32_t nq0 = 0, nq1 = 0;
        P[r] = 0;
        Q0[nq0++] = r;
        for (uint32_t j = 0; j < ix->bp_cnt[i]; ++j) {
            uint32_t v = ix->bp_S[(size_t)i * BPW + j];
            P[v] = 1;
            Sm1[v] = 1ull << j;
            Q1[nq1++] = v;
        }
        while (nq0 > 0) {
            uint64_t ne0 = 0, ne1 = 0; /* E0, E1 as flat (v,u) pair lists */
            for (uint32_t qi = 0; qi < nq0; ++qi) {
                uint32_t v = Q0[qi];
                for (uint32_t e = off[v]; e < off[v + 1]; ++e) {
                    uint32_t u = col[e];
                    if (P[u] == -1 || P[u] == P[v] + 1) {
                        E1[2 * ne1] = v; E1[2 * ne1 + 1] = u; ++ne1;
                        if (P[u] == -1) {
                            if (P[v] + 1 >= INF8) { st = ORC_E_RANGE; goto out; }
                            P[u] = P[v] + 1;
                            Q1[nq1++] = u;
                        }
                    } else if (P[u] == P[v]) {
                        E0[2 * ne0] = v; E0[2 * ne0 + 1] = u; ++ne0;
                    }
                }
            }
            for (uint64_t x = 0; x < ne0; ++x) S0[E0[2 * x + 1]] |= Sm1[E0[2 * x]];
            for (uint64_t x = 0; x < ne1; ++x) {
                Sm1[E1[2 * x + 1]] |= Sm1[E1[2 * x]];
                S0[E1[2 * x + 1]] |= S0[E1[2 * x]];
            }
            memcpy(Q0, Q1, (size_t)nq1 * sizeof(uint32_t));
            nq0 = nq1;
            nq1 = 0;
        }
    }
out:
    for (uint32_t v = 0; v < n; ++v) {
        size_t k = (size_t)v * t + i;
        if (P[v] == -1) { ix->bp_d[k] = INF8; ix->bp_m1[k] = 0; ix->bp_m0[k] = 0; }
        /* The DP above can leave members of S^{-1}_r(v) in S^0_r(v): a member u
         * of S^{-1}(w) for a same-level neighbour w may be one step closer to v
         * than r is. Sec. 5.1 defines the two sets by d(u,v) - d(r,v) = -1 and
         * = 0, so they are disjoint; store the defined S^0 = DP result minus
         * S^{-1}. Query answers are unaffected (an extra bit can only meet an
         * S^{-1} set where the -2 case already applies). */
        else { ix->bp_d[k] = (uint8_t)P[v]; ix->bp_m1[k] = Sm1[v]; ix->bp_m0[k] = S0[v] & ~Sm1[v]; }
    }
    return st;
}

/* ------------------------------------------- Sec. 5.3: bit-parallel query */
static int bp_query(const orc_index *ix, uint32_t s, uint32_t u) {
    int best = 1 << 20;
    for (uint32_t i = 0; i < ix->t; ++i) {
        size_t ks = (size_t)s * ix->t + i, ku = (size_t)u * ix->t + i;
        if (ix->bp_d[ks] == INF8 || ix->bp_d[ku] == INF8) continue;
        int td = ix->bp_d[ks] + ix->bp_d[ku];
        if (ix->bp_m1[ks] & ix->bp_m1[ku]) td -= 2;
        else if ((ix->bp_m0[ks] & ix->bp_m1[ku]) | (ix->bp_m1[ks] & ix->bp_m0[ku])) td -= 1;
        if (td < best) best = td;
    }
    return best;
}

void orc_free(orc_index *ix) {
    if (!ix) return;
    if (ix->hub) for (uint32_t v = 0; v < ix->n; ++v) { free(ix->hub[v]); free(ix->dist[v]); }
    if (ix->par) for (uint32_t v = 0; v < ix->n; ++v) free(ix->par[v]);
    free(ix->hub); free(ix->dist); free(ix->par); free(ix->len); free(ix->cap);
    free(ix->order); free(ix->rank); free(ix->inX);
    free(ix->bp_root); free(ix->bp_cnt); free(ix->bp_S);
    free(ix->bp_d); free(ix->bp_m1); free(ix->bp_m0);
    free(ix);
}

/* ------------------------- Alg. 2 + Alg. 1 with the Sec. 5.4 combination */
/* with_pruned = 0 stops after the bit-parallel stage (order, X and L_BP only),
 * for checks of single labels on graphs too large for the whole Alg. 2. */
orc_index *orc_build_ex(uint32_t n, const uint32_t *off, const uint32_t *col,
                        const uint32_t *order, uint32_t t, int with_pruned, int *status) {
    int st = ORC_OK;
    orc_index *ix = (orc_index *)calloc(1, sizeof(orc_index));
    if (!ix) { *status = ORC_E_NOMEM; return NULL; }
    ix->n = n; ix->t = t;
    size_t nt = (size_t)n * t;
    ix->order = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    ix->rank = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    ix->inX = (uint8_t *)calloc((size_t)n + 1, 1);
    ix->bp_root = (uint32_t *)malloc(((size_t)t + 1) * sizeof(uint32_t));
    ix->bp_cnt = (uint32_t *)calloc((size_t)t + 1, sizeof(uint32_t));
    ix->bp_S = (uint32_t *)calloc((size_t)t * BPW + 1, sizeof(uint32_t));
    ix->bp_d = (uint8_t *)malloc(nt + 1);
    ix->bp_m1 = (uint64_t *)malloc((nt + 1) * sizeof(uint64_t));
    ix->bp_m0 = (uint64_t *)malloc((nt + 1) * sizeof(uint64_t));
    ix->len = (uint32_t *)calloc((size_t)n + 1, sizeof(uint32_t));
    ix->cap = (uint32_t *)calloc((size_t)n + 1, sizeof(uint32_t));
    ix->hub = (uint32_t **)calloc((size_t)n + 1, sizeof(uint32_t *));
    ix->dist = (uint8_t **)calloc((size_t)n + 1, sizeof(uint8_t *));
    ix->par = (uint32_t **)calloc((size_t)n + 1, sizeof(uint32_t *));
    if (!ix->order || !ix->rank || !ix->inX || !ix->bp_root || !ix->bp_cnt || !ix->bp_S ||
        !ix->bp_d || !ix->bp_m1 || !ix->bp_m0 || !ix->len || !ix->cap || !ix->hub || !ix->dist ||
        !ix->par) {
        orc_free(ix); *status = ORC_E_NOMEM; return NULL;
    }
    /* the vertex order v_1..v_n (Sec. 4.4) */
    if (order) {
        for (uint32_t v = 0; v < n; ++v) ix->rank[v] = NONE;
        for (uint32_t k = 0; k < n; ++k) {
            if (order[k] >= n || ix->rank[order[k]] != NONE) { orc_free(ix); *status = ORC_E_ORDER; return NULL; }
            ix->order[k] = order[k];
            ix->rank[order[k]] = k;
        }
    } else {
        if ((st = orc_degree_order(n, off, col, ix->order))) { orc_free(ix); *status = st; return NULL; }
        for (uint32_t k = 0; k < n; ++k) ix->rank[ix->order[k]] = k;
    }

    /* bit-parallel stage: t unpruned Bp-BFSs (Sec. 5.4) */
    int *P = (int *)malloc(((size_t)n + 1) * sizeof(int));
    uint64_t *Sm1 = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    uint64_t *S0 = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    uint32_t *Q0 = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    uint32_t *Q1 = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    uint64_t narcs = off[n];
    uint32_t *E0 = (uint32_t *)malloc((2 * narcs + 2) * sizeof(uint32_t));
    uint32_t *E1 = (uint32_t *)malloc((2 * narcs + 2) * sizeof(uint32_t));
    if (!P || !Sm1 || !S0 || !Q0 || !Q1 || !E0 || !E1) { st = ORC_E_NOMEM; goto done; }
    if ((st = select_bp_roots(ix, off, col))) goto done;
    for (uint32_t i = 0; i < t; ++i)
        if ((st = bp_bfs(ix, off, col, i, P, Sm1, S0, Q0, Q1, E0, E1))) goto done;
    free(Sm1); Sm1 = NULL; free(S0); S0 = NULL; free(E0); E0 = NULL; free(E1); E1 = NULL;

    /* pruned stage: Alg. 2 calls PrunedBFS(G, v_k, L'_{k-1}) for k = 1..n */
    if (with_pruned) {
        uint8_t *T = (uint8_t *)malloc((size_t)n + 1);     /* root array T (Sec. 4.5.1) */
        uint8_t *Pd = (uint8_t *)malloc((size_t)n + 1);    /* tentative distances P */
        uint32_t *Pp = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t)); /* BFS-tree parents */
        uint32_t *visited = Q1;                            /* for the lazy reset */
        if (!T || !Pd || !Pp) { free(T); free(Pd); free(Pp); st = ORC_E_NOMEM; goto done; }
        memset(T, INF8, n);
        memset(Pd, INF8, n);
        for (uint32_t k = 0; k < n && st == ORC_OK; ++k) {
            uint32_t vk = ix->order[k];
            if (ix->inX[vk]) continue;
            for (uint32_t x = 0; x < ix->len[vk]; ++x) T[ix->hub[vk][x]] = ix->dist[vk][x];
            uint32_t head = 0, tail = 0;
            Q0[tail++] = vk;
            Pd[vk] = 0;
            Pp[vk] = vk;
            while (head < tail) {
                uint32_t u = Q0[head++];
                int delta = Pd[u];
                ix->visited++;
                /* line "if Query(v_k, u, L'_{k-1}) <= P[u] then continue":
                 * bit-parallel labels first, then normal labels via T */
                if (bp_query(ix, vk, u) <= delta) continue;
                int pruned = 0;
                ix->scanned += ix->len[u];
                for (uint32_t x = 0; x < ix->len[u]; ++x) {
                    uint8_t tw = T[ix->hub[u][x]];
                    if (tw != INF8 && (int)tw + ix->dist[u][x] <= delta) { pruned = 1; break; }
                }
                if (pruned) continue;
                /* L'_k[u] <- L'_{k-1}[u] U {(v_k, P[u])}, hub stored as rank k */
                if ((st = label_push(ix, u, k, (uint8_t)delta, Pp[u]))) break;
                ix->labeled++;
                ix->labeled_deg += off[u + 1] - off[u];
                for (uint32_t e = off[u]; e < off[u + 1]; ++e) {
                    uint32_t w = col[e];
                    if (Pd[w] != INF8) continue;
                    if (delta + 1 >= INF8) { st = ORC_E_RANGE; break; }
                    Pd[w] = (uint8_t)(delta + 1);
                    Pp[w] = u;
                    Q0[tail++] = w;
                }
                if (st) break;
            }
            /* lazy reset (Sec. 4.5.1, "Initialization") */
            for (uint32_t x = 0; x < tail; ++x) Pd[Q0[x]] = INF8;
            for (uint32_t x = 0; x < ix->len[vk]; ++x) T[ix->hub[vk][x]] = INF8;
        }
        (void)visited;
        free(T);
        free(Pd);
        free(Pp);
    }
done:
    free(P); free(Sm1); free(S0); free(Q0); free(Q1); free(E0); free(E1);
    if (st) { orc_free(ix); *status = st; return NULL; }
    *status = ORC_OK;
    return ix;
}

orc_index *orc_build(uint32_t n, const uint32_t *off, const uint32_t *col,
                     const uint32_t *order, uint32_t t, int *status) {
    return orc_build_ex(n, off, col, order, t, 1, status);
}

/* Query(s, t, L) of Sec. 3.3 by merge join over hub-sorted labels, combined
 * with the bit-parallel query of Sec. 5.3. Returns the distance, 255 if the
 * labels share no hub; -ORC_E_RANGE if the minimum is finite but >= 255. */
int orc_query(const orc_index *ix, uint32_t s, uint32_t u) {
    int best = bp_query(ix, s, u);
    uint32_t i = 0, j = 0;
    while (i < ix->len[s] && j < ix->len[u]) {
        uint32_t hs = ix->hub[s][i], hu = ix->hub[u][j];
        if (hs == hu) {
            int d = ix->dist[s][i] + ix->dist[u][j];
            if (d < best) best = d;
            ++i; ++j;
        } else if (hs < hu) ++i;
        else ++j;
    }
    if (best >= (1 << 20)) return INF8;
    if (best >= INF8) return -ORC_E_RANGE;
    return best;
}

int orc_query_batch(const orc_index *ix, uint64_t q, const uint32_t *s, const uint32_t *u, uint8_t *out) {
    int st = ORC_OK;
    for (uint64_t x = 0; x < q; ++x) {
        if (s[x] >= ix->n || u[x] >= ix->n) return ORC_E_INVAL;
        int d = orc_query(ix, s[x], u[x]);
        if (d < 0) { st = -d; out[x] = INF8; } else out[x] = (uint8_t)d;
    }
    return st;
}

/* The same answers as orc_query_batch, with the pairs split into `threads`
 * contiguous ranges, one POSIX thread each (a timing aid only: each pair is
 * still answered by orc_query, which reads the index and writes nothing). */
typedef struct {
    const orc_index *ix;
    const uint32_t *s, *u;
    uint8_t *out;
    uint64_t lo, hi;
    int st;
} orc_qrange;

static void *orc_qrange_run(void *p) {
    orc_qrange *r = (orc_qrange *)p;
    r->st = orc_query_batch(r->ix, r->hi - r->lo, r->s + r->lo, r->u + r->lo, r->out + r->lo);
    return NULL;
}

int orc_query_batch_mt(const orc_index *ix, uint64_t q, const uint32_t *s, const uint32_t *u,
                       uint8_t *out, uint32_t threads) {
    if (threads < 1) threads = 1;
    if (threads > 1024) threads = 1024;
    if ((uint64_t)threads > q) threads = q ? (uint32_t)q : 1;
    orc_qrange *rs = (orc_qrange *)calloc(threads, sizeof(orc_qrange));
    pthread_t *th = (pthread_t *)calloc(threads, sizeof(pthread_t));
    if (!rs || !th) { free(rs); free(th); return ORC_E_NOMEM; }
    for (uint32_t i = 0; i < threads; ++i) {
        rs[i].ix = ix; rs[i].s = s; rs[i].u = u; rs[i].out = out;
        rs[i].lo = q * i / threads;
        rs[i].hi = q * (i + 1) / threads;
    }
    uint32_t started = 0;
    for (uint32_t i = 1; i < threads; ++i, ++started)
        if (pthread_create(&th[i], NULL, orc_qrange_run, &rs[i]) != 0) break;
    orc_qrange_run(&rs[0]);
    int st = rs[0].st;
    for (uint32_t i = 1; i <= started; ++i) {
        pthread_join(th[i], NULL);
        if (rs[i].st && !st) st = rs[i].st;
    }
    /* ranges whose thread could not start run here */
    for (uint32_t i = started + 1; i < threads; ++i) {
        orc_qrange_run(&rs[i]);
        if (rs[i].st && !st) st = rs[i].st;
    }
    free(rs);
    free(th);
    return st;
}

/* ------------------------------------------------------------- exports */
uint64_t orc_total_entries(const orc_index *ix) {
    uint64_t s = 0;
    for (uint32_t v = 0; v < ix->n; ++v) s += ix->len[v];
    return s;
}

/* offsets[n+1] by vertex id; hubs are ranks, ascending; dists in hops */
void orc_export_labels(const orc_index *ix, uint64_t *offsets, uint32_t *hubs, uint8_t *dists) {
    uint64_t p = 0;
    for (uint32_t v = 0; v < ix->n; ++v) {
        offsets[v] = p;
        if (ix->len[v]) { /* an empty label has no arrays (memcpy wants real pointers) */
            memcpy(hubs + p, ix->hub[v], (size_t)ix->len[v] * sizeof(uint32_t));
            memcpy(dists + p, ix->dist[v], ix->len[v]);
        }
        p += ix->len[v];
    }
    offsets[ix->n] = p;
}

void orc_export_bp(const orc_index *ix, uint8_t *d, uint64_t *m1, uint64_t *m0) {
    size_t nt = (size_t)ix->n * ix->t;
    memcpy(d, ix->bp_d, nt);
    memcpy(m1, ix->bp_m1, nt * sizeof(uint64_t));
    memcpy(m0, ix->bp_m0, nt * sizeof(uint64_t));
}

/* roots[t] (vertex ids, 0xffffffff = empty slot), cnt[t], S[t][64] */
void orc_export_bp_roots(const orc_index *ix, uint32_t *roots, uint32_t *cnt, uint32_t *S) {
    memcpy(roots, ix->bp_root, (size_t)ix->t * sizeof(uint32_t));
    memcpy(cnt, ix->bp_cnt, (size_t)ix->t * sizeof(uint32_t));
    memcpy(S, ix->bp_S, (size_t)ix->t * BPW * sizeof(uint32_t));
}

/* parents[] in the layout of orc_export_labels, vertex ids (Sec. 6) */
void orc_export_parents(const orc_index *ix, uint32_t *parents) {
    uint64_t p = 0;
    for (uint32_t v = 0; v < ix->n; ++v) {
        if (ix->len[v]) memcpy(parents + p, ix->par[v], (size_t)ix->len[v] * sizeof(uint32_t));
        p += ix->len[v];
    }
}

/* ------------------------------------- Sec. 6: shortest-path queries */
/* Exact distance from the bit-parallel vertex x of slot i to v, from the
 * label of v: x = r_i when j < 0, else the j-th member of S_{r_i}, which lies
 * at d(r_i, v) - 1, d(r_i, v) or d(r_i, v) + 1 from v as bit j is in
 * S^{-1}_{r_i}(v), in S^0_{r_i}(v) or in neither (Sec. 5.1). -1: unreachable. */
static int bp_dist_to(const orc_index *ix, uint32_t i, int j, uint32_t v) {
    size_t k = (size_t)v * ix->t + i;
    if (ix->bp_d[k] == INF8) return -1;
    int d = ix->bp_d[k];
    if (j < 0) return d;
    uint64_t b = 1ull << j;
    if (ix->bp_m1[k] & b) return d - 1;
    if (ix->bp_m0[k] & b) return d;
    return d + 1;
}

/* Walks from v to the bit-parallel vertex (i, j), each step to the first
 * neighbour (in the graph's neighbour order) one hop nearer, writing v and
 * every vertex after it at out[pos], out[pos + step], ... Returns 0, or -1 if
 * some vertex has no nearer neighbour (impossible for a correct label). */
static int bp_descend(const orc_index *ix, const uint32_t *off, const uint32_t *col, uint32_t i,
                      int j, uint32_t v, uint32_t *out, long pos, long step) {
    int dv = bp_dist_to(ix, i, j, v);
    if (dv < 0) return -1;
    out[pos] = v;
    while (dv > 0) {
        uint32_t next = NONE;
        for (uint32_t e = off[v]; e < off[v + 1]; ++e)
            if (bp_dist_to(ix, i, j, col[e]) == dv - 1) { next = col[e]; break; }
        if (next == NONE) return -1;
        v = next;
        --dv;
        pos += step;
        out[pos] = v;
    }
    return 0;
}

/* Climbs the pruned BFS tree of hub rank h from v, which holds (h, d) in its
 * label, up to the hub through the stored parents (Sec. 6), writing the d + 1
 * vertices at out[pos], out[pos + step], ... Returns 0, or -1 if a parent does
 * not hold (h, d - 1) (impossible for a correct index). */
static int climb(const orc_index *ix, uint32_t h, uint32_t v, int d, uint32_t *out, long pos,
                 long step) {
    for (int k = d;; --k) {
        out[pos] = v;
        long x = -1;
        for (uint32_t y = 0; y < ix->len[v]; ++y)
            if (ix->hub[v][y] == h) { x = y; break; }
        if (x < 0 || ix->dist[v][x] != k) return -1;
        if (k == 0) return 0;
        v = ix->par[v][x];
        pos += step;
    }
}

/* One shortest s-u path into out[0..d] (d = d_G(s, u), at most 255 vertices):
 * returns the number of vertices, 0 if u is unreachable from s, or minus a
 * status (ORC_E_INVAL for a bad id or a label that cannot be climbed,
 * ORC_E_RANGE as for orc_query). The hub is the lowest-rank common hub of
 * L(s) and L(u) whose distances add up to d; if there is none, the first
 * bit-parallel slot i that reaches d gives the meeting vertex: a member of
 * S_{r_i} in S^{-1} of both ends (d~ - 2), in S^{-1} of one and S^0 of the
 * other (d~ - 1), or r_i itself (d~), lowest bit first. */
long orc_path(const orc_index *ix, const uint32_t *off, const uint32_t *col, uint32_t s,
              uint32_t u, uint32_t *out) {
    if (s >= ix->n || u >= ix->n) return -ORC_E_INVAL;
    int d = orc_query(ix, s, u);
    if (d < 0) return d;
    if (d == INF8) return 0;
    if (s == u) { out[0] = s; return 1; }
    uint32_t i = 0, j = 0;
    while (i < ix->len[s] && j < ix->len[u]) {
        uint32_t hs = ix->hub[s][i], hu = ix->hub[u][j];
        if (hs == hu) {
            int ds = ix->dist[s][i], du = ix->dist[u][j];
            if (ds + du == d) {
                if (climb(ix, hs, s, ds, out, 0, 1) || climb(ix, hs, u, du, out, d, -1))
                    return -ORC_E_INVAL;
                return d + 1;
            }
            ++i; ++j;
        } else if (hs < hu) ++i;
        else ++j;
    }
    for (uint32_t b = 0; b < ix->t; ++b) {
        size_t ks = (size_t)s * ix->t + b, ku = (size_t)u * ix->t + b;
        if (ix->bp_d[ks] == INF8 || ix->bp_d[ku] == INF8) continue;
        int td = ix->bp_d[ks] + ix->bp_d[ku], x = -2;
        uint64_t c;
        if (td - 2 == d && (c = ix->bp_m1[ks] & ix->bp_m1[ku])) x = __builtin_ctzll(c);
        else if (td - 1 == d && (c = (ix->bp_m1[ks] & ix->bp_m0[ku]) | (ix->bp_m0[ks] & ix->bp_m1[ku])))
            x = __builtin_ctzll(c);
        else if (td == d) x = -1;
        if (x == -2) continue;
        if (bp_dist_to(ix, b, x, s) + bp_dist_to(ix, b, x, u) != d) return -ORC_E_INVAL;
        if (bp_descend(ix, off, col, b, x, s, out, 0, 1) || bp_descend(ix, off, col, b, x, u, out, d, -1))
            return -ORC_E_INVAL;
        return d + 1;
    }
    return -ORC_E_INVAL;
}

void orc_export_order(const orc_index *ix, uint32_t *order) {
    memcpy(order, ix->order, (size_t)ix->n * sizeof(uint32_t));
}

/* visited, labeled, label entries scanned by prune tests, sum of degrees of
 * labeled vertices */
void orc_counters(const orc_index *ix, uint64_t *out4) {
    out4[0] = ix->visited; out4[1] = ix->labeled; out4[2] = ix->scanned; out4[3] = ix->labeled_deg;
}

/* -------------------------------------- closed form of one label L(u) */
/* rank[v] for every vertex, inX[v] = 1 for bit-parallel vertices.
 * Writes L(u) as (hub rank, distance) ascending by rank; returns its size,
 * or -ORC_E_NOMEM / -ORC_E_RANGE. hubs/dists must hold n entries. */
int64_t orc_label_of(uint32_t n, const uint32_t *off, const uint32_t *col, const uint32_t *rank,
                     const uint8_t *inX, uint32_t u, uint32_t *hubs, uint8_t *dists) {
    uint8_t *dist = (uint8_t *)malloc((size_t)n + 1);
    uint32_t *minrank = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    uint8_t *hasX = (uint8_t *)malloc((size_t)n + 1);
    uint32_t *q = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    if (!dist || !minrank || !hasX || !q) { free(dist); free(minrank); free(hasX); free(q); return -ORC_E_NOMEM; }
    memset(dist, INF8, n);
    int64_t res = 0;
    uint32_t head = 0, tail = 0;
    dist[u] = 0; minrank[u] = rank[u]; hasX[u] = inX[u];
    q[tail++] = u;
    /* minrank[v] = least rank on P_G(u, v); hasX[v] = P_G(u, v) meets X.
     * P_G(u, v) = {v} U union of P_G(u, w) over neighbours w of v with
     * d(u, w) = d(u, v) - 1, so both follow in BFS order. */
    while (head < tail) {
        uint32_t v = q[head++];
        for (uint32_t e = off[v]; e < off[v + 1]; ++e) {
            uint32_t w = col[e];
            if (dist[w] == INF8) {
                if (dist[v] + 1 >= INF8) { res = -ORC_E_RANGE; goto out; }
                dist[w] = (uint8_t)(dist[v] + 1);
                minrank[w] = rank[w];
                hasX[w] = inX[w];
                q[tail++] = w;
            }
            if (dist[w] == dist[v] + 1) {
                if (minrank[v] < minrank[w]) minrank[w] = minrank[v];
                hasX[w] |= hasX[v];
            }
        }
    }
    {
        /* collect hubs v with minrank[v] == rank[v] and no X vertex on P(u,v);
         * output sorted by rank via a counting pass over the BFS list */
        uint32_t c = 0;
        for (uint32_t x = 0; x < tail; ++x) {
            uint32_t v = q[x];
            if (!hasX[v] && minrank[v] == rank[v]) { hubs[c] = rank[v]; dists[c] = dist[v]; ++c; }
        }
        /* sort by rank: pack (rank, distance) so one integer sort suffices */
        uint64_t *packed = (uint64_t *)malloc(((size_t)c + 1) * sizeof(uint64_t));
        if (!packed) { res = -ORC_E_NOMEM; goto out; }
        for (uint32_t a = 0; a < c; ++a) packed[a] = ((uint64_t)hubs[a] << 8) | dists[a];
        qsort(packed, c, sizeof(uint64_t), cmp_u64);
        for (uint32_t a = 0; a < c; ++a) { hubs[a] = (uint32_t)(packed[a] >> 8); dists[a] = (uint8_t)packed[a]; }
        free(packed);
        res = c;
    }
out:
    free(dist); free(minrank); free(hasX); free(q);
    return res;
}

/* rank and X of a built index, for orc_label_of on the same order */
void orc_export_rank_inX(const orc_index *ix, uint32_t *rank, uint8_t *inX) {
    memcpy(rank, ix->rank, (size_t)ix->n * sizeof(uint32_t));
    memcpy(inX, ix->inX, ix->n);
}

/* Core numbers by bucket peeling: vertices are kept sorted by their current
 * degree in `vert` (bucket d starts at bin[d]); removing the vertex of least
 * degree lowers each neighbour of larger degree by one, moving it to the front
 * of its bucket first so the array stays sorted. The degree a vertex has when
 * it is removed is its core number. */
int orc_core_numbers(uint32_t n, const uint32_t *off, const uint32_t *col, uint32_t *core) {
    if (n == 0) return ORC_OK;
    uint32_t md = 0;
    uint32_t *deg = malloc(sizeof(uint32_t) * n), *pos = malloc(sizeof(uint32_t) * n);
    uint32_t *vert = malloc(sizeof(uint32_t) * n);
    for (uint32_t v = 0; v < n; ++v) {
        deg[v] = off[v + 1] - off[v];
        if (deg[v] > md) md = deg[v];
    }
    uint32_t *bin = calloc((size_t)md + 2, sizeof(uint32_t));
    if (!deg || !pos || !vert || !bin) {
        free(deg); free(pos); free(vert); free(bin);
        return ORC_E_NOMEM;
    }
    for (uint32_t v = 0; v < n; ++v) bin[deg[v]]++;
    uint32_t start = 0;
    for (uint32_t d = 0; d <= md; ++d) {
        uint32_t c = bin[d];
        bin[d] = start;
        start += c;
    }
    for (uint32_t v = 0; v < n; ++v) {
        pos[v] = bin[deg[v]]++;
        vert[pos[v]] = v;
    }
    for (uint32_t d = md; d > 0; --d) bin[d] = bin[d - 1];
    bin[0] = 0;
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t v = vert[i];
        for (uint32_t e = off[v]; e < off[v + 1]; ++e) {
            uint32_t u = col[e];
            if (deg[u] > deg[v]) {
                uint32_t du = deg[u], pu = pos[u], pw = bin[du], w = vert[pw];
                if (u != w) {
                    pos[u] = pw; vert[pu] = w;
                    pos[w] = pu; vert[pw] = u;
                }
                bin[du]++;
                deg[u]--;
            }
        }
    }
    memcpy(core, deg, sizeof(uint32_t) * n);
    free(deg); free(pos); free(vert); free(bin);
    return ORC_OK;
}

/* ------------------------------------------------ Sec. 6: directed graphs */
/* Two label sets per vertex (Sec. 6, "Directed Graphs"): L_IN(v) holds
 * (u, d(u, v)) and L_OUT(v) holds (u, d(v, u)), hubs as ranks. Each root v_k,
 * in rank order, runs a pruned BFS forward along arcs, which fills L_IN and
 * prunes u when L_OUT(v_k) and L_IN(u) already give d(v_k, u), and one in
 * reverse, which fills L_OUT and prunes u when L_OUT(u) and L_IN(v_k) already
 * give d(u, v_k). Readings: the Degree order counts in- plus out-arcs (ties by
 * ascending id); the forward pass runs first (the order of the two passes
 * does not change the labels: a root's own hub enters neither prune test);
 * there are no bit-parallel labels (Sec. 5's masks need |d(s, v) - d(r, v)|
 * <= 1 for neighbours s of r, which arcs one way do not give). */
typedef struct orc_label_set {
    uint32_t *len, *cap;
    uint32_t **hub;
    uint8_t **dist;
} orc_label_set;

typedef struct orc_dindex {
    uint32_t n;
    uint32_t *order, *rank;
    orc_label_set in, out;
} orc_dindex;

static int set_alloc(orc_label_set *L, uint32_t n) {
    L->len = (uint32_t *)calloc((size_t)n + 1, sizeof(uint32_t));
    L->cap = (uint32_t *)calloc((size_t)n + 1, sizeof(uint32_t));
    L->hub = (uint32_t **)calloc((size_t)n + 1, sizeof(uint32_t *));
    L->dist = (uint8_t **)calloc((size_t)n + 1, sizeof(uint8_t *));
    return (L->len && L->cap && L->hub && L->dist) ? ORC_OK : ORC_E_NOMEM;
}

static void set_free(orc_label_set *L, uint32_t n) {
    if (L->hub) for (uint32_t v = 0; v < n; ++v) free(L->hub[v]);
    if (L->dist) for (uint32_t v = 0; v < n; ++v) free(L->dist[v]);
    free(L->len); free(L->cap); free(L->hub); free(L->dist);
}

static int set_push(orc_label_set *L, uint32_t u, uint32_t hub, uint8_t d) {
    if (L->len[u] == L->cap[u]) {
        uint32_t nc = L->cap[u] ? 2 * L->cap[u] : 4;
        uint32_t *h = (uint32_t *)realloc(L->hub[u], (size_t)nc * sizeof(uint32_t));
        if (!h) return ORC_E_NOMEM;
        L->hub[u] = h;
        uint8_t *dd = (uint8_t *)realloc(L->dist[u], nc);
        if (!dd) return ORC_E_NOMEM;
        L->dist[u] = dd;
        L->cap[u] = nc;
    }
    L->hub[u][L->len[u]] = hub;
    L->dist[u][L->len[u]] = d;
    L->len[u]++;
    return ORC_OK;
}

void orc_dfree(orc_dindex *ix) {
    if (!ix) return;
    set_free(&ix->in, ix->n);
    set_free(&ix->out, ix->n);
    free(ix->order); free(ix->rank);
    free(ix);
}

/* Alg. 1 for root v_k in one direction: follow the arcs of (off, col); the
 * root's own labels `from` give T, the visited vertices are tested against and
 * labelled in `to`. */
static int pruned_bfs_dir(uint32_t n, const uint32_t *off, const uint32_t *col, uint32_t k,
                          uint32_t vk, const orc_label_set *from, orc_label_set *to, uint8_t *T,
                          uint8_t *Pd, uint32_t *Q) {
    (void)n;
    int st = ORC_OK;
    for (uint32_t x = 0; x < from->len[vk]; ++x) T[from->hub[vk][x]] = from->dist[vk][x];
    uint32_t head = 0, tail = 0;
    Q[tail++] = vk;
    Pd[vk] = 0;
    while (head < tail && st == ORC_OK) {
        uint32_t u = Q[head++];
        int delta = Pd[u], pruned = 0;
        for (uint32_t x = 0; x < to->len[u]; ++x) {
            uint8_t tw = T[to->hub[u][x]];
            if (tw != INF8 && (int)tw + to->dist[u][x] <= delta) { pruned = 1; break; }
        }
        if (pruned) continue;
        if ((st = set_push(to, u, k, (uint8_t)delta))) break;
        for (uint32_t e = off[u]; e < off[u + 1]; ++e) {
            uint32_t w = col[e];
            if (Pd[w] != INF8) continue;
            if (delta + 1 >= INF8) { st = ORC_E_RANGE; break; }
            Pd[w] = (uint8_t)(delta + 1);
            Q[tail++] = w;
        }
    }
    for (uint32_t x = 0; x < tail; ++x) Pd[Q[x]] = INF8;
    for (uint32_t x = 0; x < from->len[vk]; ++x) T[from->hub[vk][x]] = INF8;
    return st;
}

/* off, col: arcs u -> col[e] for e in [off[u], off[u+1]) (out-neighbours;
 * self-loops and repeated arcs are allowed and change nothing). order: rank
 * -> vertex, or NULL for the Degree order by in- plus out-degree. */
orc_dindex *orc_build_directed(uint32_t n, const uint32_t *off, const uint32_t *col,
                               const uint32_t *order, int *status) {
    int st = ORC_OK;
    orc_dindex *ix = (orc_dindex *)calloc(1, sizeof(orc_dindex));
    if (!ix) { *status = ORC_E_NOMEM; return NULL; }
    ix->n = n;
    uint64_t m = off[n];
    ix->order = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    ix->rank = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    uint32_t *roff = (uint32_t *)calloc((size_t)n + 2, sizeof(uint32_t));
    uint32_t *rcol = (uint32_t *)malloc((m + 1) * sizeof(uint32_t));
    uint32_t *deg = (uint32_t *)calloc((size_t)n + 1, sizeof(uint32_t));
    uint8_t *T = (uint8_t *)malloc((size_t)n + 1), *Pd = (uint8_t *)malloc((size_t)n + 1);
    uint32_t *Q = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    if (!ix->order || !ix->rank || !roff || !rcol || !deg || !T || !Pd || !Q ||
        set_alloc(&ix->in, n) || set_alloc(&ix->out, n)) { st = ORC_E_NOMEM; goto done; }
    for (uint64_t e = 0; e < m; ++e)
        if (col[e] >= n) { st = ORC_E_INVAL; goto done; }
    /* reverse arcs: in-neighbours of each vertex */
    for (uint64_t e = 0; e < m; ++e) roff[col[e] + 1]++;
    for (uint32_t v = 0; v < n; ++v) roff[v + 1] += roff[v];
    {
        uint32_t *fill = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
        if (!fill) { st = ORC_E_NOMEM; goto done; }
        memcpy(fill, roff, (size_t)n * sizeof(uint32_t));
        for (uint32_t u = 0; u < n; ++u)
            for (uint32_t e = off[u]; e < off[u + 1]; ++e) rcol[fill[col[e]]++] = u;
        free(fill);
    }
    if (order) {
        for (uint32_t v = 0; v < n; ++v) ix->rank[v] = NONE;
        for (uint32_t k = 0; k < n; ++k) {
            if (order[k] >= n || ix->rank[order[k]] != NONE) { st = ORC_E_ORDER; goto done; }
            ix->order[k] = order[k];
            ix->rank[order[k]] = k;
        }
    } else {
        for (uint32_t v = 0; v < n; ++v) {
            deg[v] = (off[v + 1] - off[v]) + (roff[v + 1] - roff[v]);
            ix->order[v] = v;
        }
        g_deg_for_sort = deg;
        qsort(ix->order, n, sizeof(uint32_t), cmp_degree);
        for (uint32_t k = 0; k < n; ++k) ix->rank[ix->order[k]] = k;
    }
    memset(T, INF8, n);
    memset(Pd, INF8, n);
    for (uint32_t k = 0; k < n && st == ORC_OK; ++k) {
        uint32_t vk = ix->order[k];
        st = pruned_bfs_dir(n, off, col, k, vk, &ix->out, &ix->in, T, Pd, Q);
        if (st == ORC_OK) st = pruned_bfs_dir(n, roff, rcol, k, vk, &ix->in, &ix->out, T, Pd, Q);
    }
done:
    free(roff); free(rcol); free(deg); free(T); free(Pd); free(Q);
    if (st) { orc_dfree(ix); *status = st; return NULL; }
    *status = ORC_OK;
    return ix;
}

/* d(s, t) from L_OUT(s) and L_IN(t) (merge join over hub ranks); 255 if they
 * share no hub; -ORC_E_RANGE if the minimum is finite but >= 255. */
int orc_dquery(const orc_dindex *ix, uint32_t s, uint32_t t) {
    const orc_label_set *A = &ix->out, *B = &ix->in;
    int best = 1 << 20;
    uint32_t i = 0, j = 0;
    while (i < A->len[s] && j < B->len[t]) {
        uint32_t hs = A->hub[s][i], ht = B->hub[t][j];
        if (hs == ht) {
            int d = A->dist[s][i] + B->dist[t][j];
            if (d < best) best = d;
            ++i; ++j;
        } else if (hs < ht) ++i;
        else ++j;
    }
    if (best >= (1 << 20)) return INF8;
    if (best >= INF8) return -ORC_E_RANGE;
    return best;
}

int orc_dquery_batch(const orc_dindex *ix, uint64_t q, const uint32_t *s, const uint32_t *t,
                     uint8_t *out) {
    int st = ORC_OK;
    for (uint64_t x = 0; x < q; ++x) {
        if (s[x] >= ix->n || t[x] >= ix->n) return ORC_E_INVAL;
        int d = orc_dquery(ix, s[x], t[x]);
        if (d < 0) { st = -d; out[x] = INF8; } else out[x] = (uint8_t)d;
    }
    return st;
}

/* which = 0: L_IN, 1: L_OUT */
uint64_t orc_dtotal(const orc_dindex *ix, int which) {
    const orc_label_set *L = which ? &ix->out : &ix->in;
    uint64_t s = 0;
    for (uint32_t v = 0; v < ix->n; ++v) s += L->len[v];
    return s;
}

void orc_dexport(const orc_dindex *ix, int which, uint64_t *offsets, uint32_t *hubs, uint8_t *dists) {
    const orc_label_set *L = which ? &ix->out : &ix->in;
    uint64_t p = 0;
    for (uint32_t v = 0; v < ix->n; ++v) {
        offsets[v] = p;
        if (L->len[v]) {
            memcpy(hubs + p, L->hub[v], (size_t)L->len[v] * sizeof(uint32_t));
            memcpy(dists + p, L->dist[v], L->len[v]);
        }
        p += L->len[v];
    }
    offsets[ix->n] = p;
}

void orc_dexport_order(const orc_dindex *ix, uint32_t *order) {
    memcpy(order, ix->order, (size_t)ix->n * sizeof(uint32_t));
}
