/*
 * Maximum-flow / minimum-cut ORACLE.  TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this file.  The CUDA library never includes, links or
 * calls it, and this file includes nothing from the CUDA library: the two
 * share no code, no header and no constant.
 *
 * What it computes (paper §2.1, the problem statement): for a directed graph
 * G(V,E) with integer capacities c(u,v), a source s and a sink t, the maximum
 * s-t flow value, which equals the minimum s-t cut capacity.  All arithmetic
 * is exact integer (int64 flows and excesses).
 *
 * Functions (each a plain, slow, textbook routine):
 *   oracle_maxflow_pr      FIFO push-relabel, the sequential form of the
 *                          procedure of §2.2 (push only when h(u)=h(v)+1,
 *                          relabel to 1+min, h(s)=|V|, a vertex stops being
 *                          active once its height reaches |V|), with the
 *                          global-relabel heuristic of §2.2 (backward BFS from
 *                          the sink) and the gap heuristic; then a second
 *                          phase that returns stranded excess to s so that a
 *                          valid flow per input arc and the canonical cut come
 *                          out.  This is the reference the GPU path is
 *                          compared with.
 *   oracle_maxflow_dinic   Dinic's blocking-flow algorithm (§2.1, background):
 *                          an independent cross-check of the value.
 *   oracle_mincut_brute    enumeration of every s-t cut for |V| <= 22:
 *                          the plain definition of the minimum cut, and the
 *                          intersection of all minimum source sides.
 *   oracle_matching_hk     Hopcroft-Karp maximum bipartite matching (an
 *                          independent check of the matching size that the
 *                          unit-capacity flow network of §4.1 computes).
 *   oracle_verify_flow     the optimality certificate: capacity constraints,
 *                          conservation, value, and a residual-reachable cut
 *                          whose capacity equals the value.
 *   oracle_residual_dist   BFS distances to a target over the arcs of a given
 *                          residual arc list (the global-relabel heights of
 *                          §2.2 for a residual snapshot).
 *
 * Input format shared by all entry points: n vertices 0..n-1, m arcs given as
 * three int32 arrays src[m], dst[m], cap[m] (cap >= 0); s != t.  Self-loops
 * are accepted and carry no flow.  Parallel and antiparallel arcs are kept
 * as separate arcs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL -1
#define ORACLE_ENOMEM -2
#define ORACLE_EINTERNAL -3   /* phase 2 left excess outside s and t */

/* ------------------------------------------------------------------------ */
/* Residual graph: every non-loop input arc k gives two residual arcs,       */
/* 2k (tail -> head, residual c) and 2k+1 (head -> tail, residual 0), so     */
/* the reverse of residual arc a is a ^ 1.  out[first[v] .. first[v+1]) are  */
/* the residual arcs leaving v.                                              */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    int64_t narcs;
    int64_t *first;    /* n + 1 */
    int64_t *out;      /* narcs: residual arc ids grouped by tail */
    int32_t *head;     /* narcs */
    int64_t *res;      /* narcs: residual capacity */
    int64_t *pair_of;  /* m: input arc -> pair index k, or -1 for a self-loop */
} rgraph;

static void rg_free(rgraph *g)
{
    free(g->first); free(g->out); free(g->head); free(g->res); free(g->pair_of);
    memset(g, 0, sizeof(*g));
}

static int rg_build(rgraph *g, int64_t n, int64_t m, const int32_t *src,
                    const int32_t *dst, const int32_t *cap)
{
    memset(g, 0, sizeof(*g));
    g->n = n;
    int64_t pairs = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n || cap[i] < 0)
            return ORACLE_EINVAL;
        if (src[i] != dst[i]) ++pairs;
    }
    g->narcs = 2 * pairs;
    g->first = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->out = (int64_t *)malloc(sizeof(int64_t) * (size_t)(g->narcs + 1));
    g->head = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->narcs + 1));
    g->res = (int64_t *)malloc(sizeof(int64_t) * (size_t)(g->narcs + 1));
    g->pair_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    if (!g->first || !g->out || !g->head || !g->res || !g->pair_of) {
        rg_free(g);
        return ORACLE_ENOMEM;
    }
    int64_t k = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (src[i] == dst[i]) { g->pair_of[i] = -1; continue; }
        g->pair_of[i] = k;
        g->head[2 * k] = dst[i];
        g->res[2 * k] = cap[i];
        g->head[2 * k + 1] = src[i];
        g->res[2 * k + 1] = 0;
        g->first[src[i] + 1]++;
        g->first[dst[i] + 1]++;
        ++k;
    }
    for (int64_t v = 0; v < n; ++v) g->first[v + 1] += g->first[v];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!fill) { rg_free(g); return ORACLE_ENOMEM; }
    memcpy(fill, g->first, sizeof(int64_t) * (size_t)n);
    for (int64_t a = 0; a < g->narcs; ++a) {
        int32_t tail = g->head[a ^ 1];
        g->out[fill[tail]++] = a;
    }
    free(fill);
    return ORACLE_OK;
}

/* Heights by backward BFS: h[v] = base + (number of residual arcs on a      */
/* shortest residual path from v to `target`), never passing `excluded`.     */
/* Vertices with no such path get `unreach`.  h[excluded] is left alone.     */
/* This is the global relabel of §2.2 (target t, base 0, unreachable |V|).   */
static void bfs_heights(const rgraph *g, int32_t target, int32_t excluded,
                        int32_t base, int32_t unreach, int32_t *h, int32_t *queue)
{
    const int64_t n = g->n;
    int32_t keep = h[excluded];
    for (int64_t v = 0; v < n; ++v) h[v] = -1;
    h[excluded] = keep;
    h[target] = base;
    int64_t qh = 0, qt = 0;
    queue[qt++] = target;
    while (qh < qt) {
        int32_t w = queue[qh++];
        for (int64_t p = g->first[w]; p < g->first[w + 1]; ++p) {
            int64_t a = g->out[p];          /* arc w -> v */
            int32_t v = g->head[a];
            if (v == excluded || h[v] != -1) continue;
            if (g->res[a ^ 1] > 0) {        /* residual arc v -> w exists */
                h[v] = h[w] + 1;
                queue[qt++] = v;
            }
        }
    }
    for (int64_t v = 0; v < n; ++v)
        if (h[v] == -1 && v != excluded) h[v] = unreach;
}

/* Counters the caller may ask for. */
typedef struct {
    int64_t arcs_scanned;     /* residual arcs examined by discharge + relabel */
    int64_t pushes;
    int64_t relabels;
    int64_t global_relabels;
    int64_t gaps;
} oracle_stats;

/* One FIFO discharge loop (sequential push-relabel, §2.2 rules).           */
/* phase 1: sink t, heights below n are live, h = n deactivates.           */
/* phase 2: sink s, heights below 2n are live.                             */
typedef struct {
    rgraph *g;
    int32_t s, t, sink, other;
    int32_t cap_height;      /* a vertex with h >= cap_height is inactive */
    int32_t *h;
    int64_t *e;
    int64_t *cur;            /* current-arc pointer per vertex */
    int32_t *count;          /* phase 1 gap heuristic: vertices per height < n */
    int use_gap;
    int32_t *fifo;           /* circular queue of capacity n */
    uint8_t *inq;
    int64_t qh, qlen;
    oracle_stats *st;
} pr_state;

static void q_push(pr_state *P, int32_t v)
{
    int64_t n = P->g->n;
    P->fifo[(P->qh + P->qlen) % n] = v;
    P->qlen++;
    P->inq[v] = 1;
}

static int32_t q_pop(pr_state *P)
{
    int64_t n = P->g->n;
    int32_t v = P->fifo[P->qh];
    P->qh = (P->qh + 1) % n;
    P->qlen--;
    P->inq[v] = 0;
    return v;
}

static int is_active(const pr_state *P, int32_t v)
{
    return v != P->s && v != P->t && P->e[v] > 0 && P->h[v] < P->cap_height;
}

/* Relabel u to 1 + the minimum height of its residual neighbours (capped at */
/* cap_height); in phase 1 apply the gap heuristic when u's old height       */
/* level becomes empty.  Returns the number of relabels performed (1).       */
static void relabel(pr_state *P, int32_t u)
{
    rgraph *g = P->g;
    int64_t minh = INT32_MAX;
    for (int64_t p = g->first[u]; p < g->first[u + 1]; ++p) {
        int64_t a = g->out[p];
        P->st->arcs_scanned++;
        if (g->res[a] > 0 && P->h[g->head[a]] < minh) minh = P->h[g->head[a]];
    }
    int32_t old = P->h[u];
    int64_t nh = (minh == INT32_MAX) ? P->cap_height : minh + 1;
    if (nh > P->cap_height) nh = P->cap_height;
    P->h[u] = (int32_t)nh;
    P->cur[u] = g->first[u];
    P->st->relabels++;
    if (P->use_gap) {
        int32_t n = (int32_t)g->n;
        P->count[old]--;
        if (P->h[u] < n) P->count[P->h[u]]++;
        if (P->count[old] == 0) {
            /* Gap: no vertex at height `old` < n, so no vertex above it can   */
            /* reach t along residual arcs (heights drop by at most one per    */
            /* residual arc).  Lift them all to n.                             */
            P->st->gaps++;
            for (int32_t v = 0; v < n; ++v) {
                if (v == P->s) continue;
                if (P->h[v] > old && P->h[v] < n) {
                    P->count[P->h[v]]--;
                    P->h[v] = n;
                }
            }
        }
    }
}

/* Discharge u: push along admissible arcs (h(u) = h(v) + 1) until its excess */
/* is gone, relabelling whenever the arc list is exhausted.                   */
static void discharge(pr_state *P, int32_t u)
{
    rgraph *g = P->g;
    while (P->e[u] > 0 && P->h[u] < P->cap_height) {
        if (P->cur[u] == g->first[u + 1]) {
            relabel(P, u);
            continue;
        }
        int64_t a = g->out[P->cur[u]];
        int32_t v = g->head[a];
        P->st->arcs_scanned++;
        if (g->res[a] > 0 && P->h[u] == P->h[v] + 1) {
            int64_t d = P->e[u] < g->res[a] ? P->e[u] : g->res[a];
            g->res[a] -= d;
            g->res[a ^ 1] += d;
            P->e[u] -= d;
            P->e[v] += d;
            P->st->pushes++;
            if (!P->inq[v] && is_active(P, v)) q_push(P, v);
            if (g->res[a] == 0) P->cur[u]++;
        } else {
            P->cur[u]++;
        }
    }
}

/* Run the FIFO loop: global relabel, queue every active vertex, discharge   */
/* until the queue is empty or `relabel_budget` relabels have been spent,    */
/* then start over with a fresh global relabel.                              */
static void pr_run(pr_state *P, int32_t base, int32_t unreach, int64_t relabel_budget,
                   int32_t *bfsq)
{
    rgraph *g = P->g;
    const int64_t n = g->n;
    for (;;) {
        bfs_heights(g, P->sink, P->other, base, unreach, P->h, bfsq);
        P->st->global_relabels++;
        if (P->use_gap) {
            for (int64_t v = 0; v < n; ++v) P->count[v] = 0;
            for (int64_t v = 0; v < n; ++v)
                if (v != P->s && P->h[v] < n) P->count[P->h[v]]++;
        }
        P->qh = 0;
        P->qlen = 0;
        for (int64_t v = 0; v < n; ++v) {
            P->inq[v] = 0;
            P->cur[v] = g->first[v];
        }
        for (int32_t v = 0; v < n; ++v)
            if (is_active(P, v)) q_push(P, v);
        if (P->qlen == 0) return;
        int64_t start = P->st->relabels;
        while (P->qlen > 0 && P->st->relabels - start < relabel_budget) {
            int32_t u = q_pop(P);
            discharge(P, u);
        }
    }
}

/*
 * Maximum flow by FIFO push-relabel.
 *   value       out: the maximum flow value (= e(t) after phase 1).
 *   flow        out (may be NULL): flow[i] on input arc i, a valid maximum
 *               flow (phase 2 returns all stranded excess to s first).
 *   source_side out (may be NULL): 1 for the vertices reachable from s in the
 *               residual graph of that flow (the minimal minimum-cut source
 *               side, identical for every maximum flow), else 0.
 *   st          out (may be NULL): counters.
 * Returns 0, ORACLE_EINVAL or ORACLE_ENOMEM.
 */
int oracle_maxflow_pr(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                      const int32_t *cap, int32_t s, int32_t t, int64_t *value,
                      int32_t *flow, uint8_t *source_side, oracle_stats *st)
{
    if (n < 2 || m < 0 || s < 0 || t < 0 || s >= n || t >= n || s == t || !value)
        return ORACLE_EINVAL;
    if (n >= (int64_t)1 << 30) return ORACLE_EINVAL;
    rgraph g;
    int rc = rg_build(&g, n, m, src, dst, cap);
    if (rc) return rc;
    oracle_stats local;
    memset(&local, 0, sizeof(local));
    if (!st) st = &local;
    memset(st, 0, sizeof(*st));

    pr_state P;
    memset(&P, 0, sizeof(P));
    P.g = &g;
    P.s = s;
    P.t = t;
    P.st = st;
    P.h = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    P.e = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    P.cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    P.count = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    P.fifo = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    P.inq = (uint8_t *)calloc((size_t)n, 1);
    int32_t *bfsq = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!P.h || !P.e || !P.cur || !P.count || !P.fifo || !P.inq || !bfsq) {
        rc = ORACLE_ENOMEM;
        goto done;
    }

    /* Step 0, preflow (Alg. 1): saturate every residual arc leaving s.     */
    for (int64_t v = 0; v < n; ++v) P.h[v] = 0;
    P.h[s] = (int32_t)n;
    for (int64_t p = g.first[s]; p < g.first[s + 1]; ++p) {
        int64_t a = g.out[p];
        int64_t d = g.res[a];
        if (d <= 0) continue;
        g.res[a] = 0;
        g.res[a ^ 1] += d;
        P.e[g.head[a]] += d;
        P.e[s] -= d;
    }

    /* Phase 1: maximum preflow; the value is e(t).                          */
    P.sink = t;
    P.other = s;
    P.cap_height = (int32_t)n;
    P.use_gap = 1;
    pr_run(&P, 0, (int32_t)n, n, bfsq);
    *value = P.e[t];

    if (flow || source_side) {
        /* Phase 2: every vertex still holding excess cannot reach t; push   */
        /* the excess back to s with heights measured from s (offset n).     */
        P.sink = s;
        P.other = t;
        P.cap_height = (int32_t)(2 * n);
        P.use_gap = 0;
        P.h[s] = (int32_t)n;
        pr_run(&P, (int32_t)n, (int32_t)(2 * n), INT64_MAX, bfsq);
        for (int64_t v = 0; v < n; ++v) {
            if (v != s && v != t && P.e[v] != 0) { rc = ORACLE_EINTERNAL; goto done; }
        }
        if (flow) {
            for (int64_t i = 0; i < m; ++i) {
                int64_t k = g.pair_of[i];
                flow[i] = (k < 0) ? 0 : (int32_t)(cap[i] - g.res[2 * k]);
            }
        }
        if (source_side) {
            /* Forward BFS from s over residual arcs. */
            memset(source_side, 0, (size_t)n);
            int64_t qh = 0, qt = 0;
            bfsq[qt++] = s;
            source_side[s] = 1;
            while (qh < qt) {
                int32_t u = bfsq[qh++];
                for (int64_t p = g.first[u]; p < g.first[u + 1]; ++p) {
                    int64_t a = g.out[p];
                    int32_t v = g.head[a];
                    if (g.res[a] > 0 && !source_side[v]) {
                        source_side[v] = 1;
                        bfsq[qt++] = v;
                    }
                }
            }
        }
    }
done:
    free(P.h); free(P.e); free(P.cur); free(P.count); free(P.fifo); free(P.inq);
    free(bfsq);
    rg_free(&g);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Dinic: BFS level graph from s, then blocking flow by depth-first search   */
/* with current-arc pointers (an explicit stack, no recursion).              */
/* ------------------------------------------------------------------------ */
int oracle_maxflow_dinic(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                         const int32_t *cap, int32_t s, int32_t t, int64_t *value,
                         int32_t *flow)
{
    if (n < 2 || m < 0 || s < 0 || t < 0 || s >= n || t >= n || s == t || !value)
        return ORACLE_EINVAL;
    rgraph g;
    int rc = rg_build(&g, n, m, src, dst, cap);
    if (rc) return rc;
    int32_t *level = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *it = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *path = (int64_t *)malloc(sizeof(int64_t) * (size_t)n); /* arc stack */
    if (!level || !queue || !it || !path) { rc = ORACLE_ENOMEM; goto done; }
    int64_t total = 0;
    for (;;) {
        for (int64_t v = 0; v < n; ++v) level[v] = -1;
        int64_t qh = 0, qt = 0;
        level[s] = 0;
        queue[qt++] = s;
        while (qh < qt) {
            int32_t u = queue[qh++];
            for (int64_t p = g.first[u]; p < g.first[u + 1]; ++p) {
                int64_t a = g.out[p];
                int32_t v = g.head[a];
                if (g.res[a] > 0 && level[v] < 0) {
                    level[v] = level[u] + 1;
                    queue[qt++] = v;
                }
            }
        }
        if (level[t] < 0) break;
        for (int64_t v = 0; v < n; ++v) it[v] = g.first[v];
        /* Blocking flow: grow a path of level-increasing residual arcs from s; */
        /* on reaching t augment by its bottleneck; on a dead end retreat.      */
        int64_t depth = 0;
        int32_t u = s;
        for (;;) {
            if (u == t) {
                int64_t b = INT64_MAX;
                for (int64_t i = 0; i < depth; ++i)
                    if (g.res[path[i]] < b) b = g.res[path[i]];
                for (int64_t i = 0; i < depth; ++i) {
                    g.res[path[i]] -= b;
                    g.res[path[i] ^ 1] += b;
                }
                total += b;
                /* restart from the tail of the first saturated arc */
                int64_t cut = 0;
                while (g.res[path[cut]] > 0) ++cut;
                depth = cut;
                u = g.head[path[cut] ^ 1];
                continue;
            }
            int advanced = 0;
            while (it[u] < g.first[u + 1]) {
                int64_t a = g.out[it[u]];
                int32_t v = g.head[a];
                if (g.res[a] > 0 && level[v] == level[u] + 1) {
                    path[depth++] = a;
                    u = v;
                    advanced = 1;
                    break;
                }
                it[u]++;
            }
            if (advanced) continue;
            /* dead end: u cannot reach t in the level graph */
            level[u] = -1;
            if (depth == 0) break;
            --depth;
            u = g.head[path[depth] ^ 1];
            it[u]++;
        }
    }
    *value = total;
    if (flow) {
        for (int64_t i = 0; i < m; ++i) {
            int64_t k = g.pair_of[i];
            flow[i] = (k < 0) ? 0 : (int32_t)(cap[i] - g.res[2 * k]);
        }
    }
done:
    free(level); free(queue); free(it); free(path);
    rg_free(&g);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Brute force over all 2^(n-2) s-t cuts (the definition of §2.1).           */
/*   min_cut      out: the minimum cut capacity.                             */
/*   source_side  out (may be NULL): the intersection of the source sides of */
/*                all minimum cuts.                                          */
/* ------------------------------------------------------------------------ */
int oracle_mincut_brute(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                        const int32_t *cap, int32_t s, int32_t t, int64_t *min_cut,
                        uint8_t *source_side)
{
    if (n < 2 || n > 22 || m < 0 || s < 0 || t < 0 || s >= n || t >= n || s == t || !min_cut)
        return ORACLE_EINVAL;
    for (int64_t i = 0; i < m; ++i)
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n || cap[i] < 0)
            return ORACLE_EINVAL;
    int32_t others[22];
    int k = 0;
    for (int32_t v = 0; v < n; ++v)
        if (v != s && v != t) others[k++] = v;
    int64_t best = INT64_MAX;
    uint32_t inter = 0;   /* bitmask over vertices */
    for (uint64_t mask = 0; mask < ((uint64_t)1 << k); ++mask) {
        uint32_t S = (uint32_t)1 << s;
        for (int j = 0; j < k; ++j)
            if (mask >> j & 1) S |= (uint32_t)1 << others[j];
        int64_t c = 0;
        for (int64_t i = 0; i < m; ++i)
            if ((S >> src[i] & 1) && !(S >> dst[i] & 1)) c += cap[i];
        if (c < best) { best = c; inter = S; }
        else if (c == best) inter &= S;
    }
    *min_cut = best;
    if (source_side)
        for (int32_t v = 0; v < n; ++v) source_side[v] = (uint8_t)(inter >> v & 1);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Hopcroft-Karp maximum matching on a bipartite graph with nl left and nr   */
/* right vertices; edge i joins left eu[i] to right ev[i].                   */
/* ------------------------------------------------------------------------ */
int oracle_matching_hk(int64_t nl, int64_t nr, int64_t ne, const int32_t *eu,
                       const int32_t *ev, int64_t *size)
{
    if (nl < 0 || nr < 0 || ne < 0 || !size) return ORACLE_EINVAL;
    for (int64_t i = 0; i < ne; ++i)
        if (eu[i] < 0 || eu[i] >= nl || ev[i] < 0 || ev[i] >= nr) return ORACLE_EINVAL;
    int rc = ORACLE_OK;
    int64_t *first = (int64_t *)calloc((size_t)nl + 1, sizeof(int64_t));
    int32_t *adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ne + 1));
    int32_t *matchL = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nl + 1));
    int32_t *matchR = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nr + 1));
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nl + 1));
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nl + 1));
    int64_t *it = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nl + 1));
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nl + 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nl + 1));
    if (!first || !adj || !matchL || !matchR || !dist || !queue || !it || !stack || !fill) {
        rc = ORACLE_ENOMEM;
        goto done;
    }
    for (int64_t i = 0; i < ne; ++i) first[eu[i] + 1]++;
    for (int64_t u = 0; u < nl; ++u) first[u + 1] += first[u];
    memcpy(fill, first, sizeof(int64_t) * (size_t)nl);
    for (int64_t i = 0; i < ne; ++i) adj[fill[eu[i]]++] = ev[i];
    for (int64_t u = 0; u < nl; ++u) matchL[u] = -1;
    for (int64_t r = 0; r < nr; ++r) matchR[r] = -1;
    int64_t matched = 0;
    const int32_t INF = INT32_MAX;
    for (;;) {
        /* BFS from all free left vertices over alternating paths. */
        int64_t qh = 0, qt = 0;
        int32_t found = INF;
        for (int64_t u = 0; u < nl; ++u) {
            if (matchL[u] < 0) { dist[u] = 0; queue[qt++] = (int32_t)u; }
            else dist[u] = INF;
        }
        while (qh < qt) {
            int32_t u = queue[qh++];
            if (dist[u] >= found) continue;
            for (int64_t p = first[u]; p < first[u + 1]; ++p) {
                int32_t w = matchR[adj[p]];
                if (w < 0) { if (found == INF) found = dist[u] + 1; }
                else if (dist[w] == INF) { dist[w] = dist[u] + 1; queue[qt++] = w; }
            }
        }
        if (found == INF) break;
        /* DFS from each free left vertex along dist-increasing edges. */
        for (int64_t u = 0; u < nl; ++u) it[u] = first[u];
        for (int64_t root = 0; root < nl; ++root) {
            if (matchL[root] >= 0) continue;
            int64_t sp = 0;
            stack[sp++] = (int32_t)root;
            while (sp > 0) {
                int32_t u = stack[sp - 1];
                if (it[u] == first[u + 1]) { dist[u] = INF; --sp; continue; }
                int32_t r = adj[it[u]];
                int32_t w = matchR[r];
                if (w < 0 && dist[u] + 1 == found) {
                    /* augment along the stack: stack[j] takes the right vertex */
                    /* its current arc points to                                */
                    for (int64_t j = sp - 1; j >= 0; --j) {
                        int32_t x = stack[j];
                        int32_t rr = adj[it[x]];
                        matchL[x] = rr;
                        matchR[rr] = x;
                    }
                    ++matched;
                    sp = 0;
                    break;
                }
                if (w >= 0 && dist[w] == dist[u] + 1) { stack[sp++] = w; continue; }
                it[u]++;
            }
        }
    }
    *size = matched;
done:
    free(first); free(adj); free(matchL); free(matchR); free(dist); free(queue);
    free(it); free(stack); free(fill);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Optimality certificate for a flow given per input arc.                   */
/* Returns 0 if: 0 <= flow[i] <= cap[i] for every arc; inflow = outflow at  */
/* every v other than s and t; the net outflow of s and the net inflow of t  */
/* both equal `value`; and the set S of vertices reachable from s along     */
/* residual arcs excludes t and has cut capacity equal to `value` (then the */
/* flow is maximum and S is a minimum cut).  Otherwise returns the first    */
/* failed check: 1 capacity, 2 conservation, 3 value, 4 cut.                */
/* cut_out and source_side (may be NULL) receive the cut capacity and S.    */
/* ------------------------------------------------------------------------ */
int oracle_verify_flow(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                       const int32_t *cap, int32_t s, int32_t t, const int32_t *flow,
                       int64_t value, int64_t *cut_out, uint8_t *source_side)
{
    if (n < 2 || m < 0 || s < 0 || t < 0 || s >= n || t >= n || s == t) return ORACLE_EINVAL;
    for (int64_t i = 0; i < m; ++i) {
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n || cap[i] < 0)
            return ORACLE_EINVAL;
        if (flow[i] < 0 || flow[i] > cap[i]) return 1;
    }
    int rc = 0;
    int64_t *bal = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    uint8_t *S = (uint8_t *)calloc((size_t)n, 1);
    rgraph g;
    if (!bal || !S) { free(bal); free(S); return ORACLE_ENOMEM; }
    for (int64_t i = 0; i < m; ++i) {
        bal[src[i]] -= flow[i];
        bal[dst[i]] += flow[i];
    }
    for (int64_t v = 0; v < n; ++v)
        if (v != s && v != t && bal[v] != 0) { rc = 2; goto out; }
    if (-bal[s] != value || bal[t] != value) { rc = 3; goto out; }
    rc = rg_build(&g, n, m, src, dst, cap);
    if (rc) goto out;
    for (int64_t i = 0; i < m; ++i) {
        int64_t k = g.pair_of[i];
        if (k < 0) continue;
        g.res[2 * k] = cap[i] - flow[i];
        g.res[2 * k + 1] = flow[i];
    }
    {
        int32_t *q = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        if (!q) { rg_free(&g); rc = ORACLE_ENOMEM; goto out; }
        int64_t qh = 0, qt = 0;
        q[qt++] = s;
        S[s] = 1;
        while (qh < qt) {
            int32_t u = q[qh++];
            for (int64_t p = g.first[u]; p < g.first[u + 1]; ++p) {
                int64_t a = g.out[p];
                int32_t v = g.head[a];
                if (g.res[a] > 0 && !S[v]) { S[v] = 1; q[qt++] = v; }
            }
        }
        free(q);
    }
    rg_free(&g);
    {
        int64_t c = 0;
        for (int64_t i = 0; i < m; ++i)
            if (S[src[i]] && !S[dst[i]]) c += cap[i];
        if (cut_out) *cut_out = c;
        if (S[t] || c != value) rc = 4;
    }
    if (source_side) memcpy(source_side, S, (size_t)n);
out:
    free(bal);
    free(S);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Global-relabel heights for a residual snapshot given as an arc list      */
/* (tail[a], head[a], rescap[a]): dist[v] = base + length of a shortest path */
/* v -> target over arcs with rescap > 0 that never visits `excluded`;       */
/* unreachable vertices get `unreach`, dist[excluded] gets `excluded_h`.     */
/* ------------------------------------------------------------------------ */
int oracle_residual_dist(int64_t n, int64_t na, const int32_t *tail, const int32_t *head,
                         const int64_t *rescap, int32_t target, int32_t excluded,
                         int32_t base, int32_t unreach, int32_t excluded_h, int32_t *dist)
{
    if (n < 1 || na < 0 || target < 0 || target >= n) return ORACLE_EINVAL;
    int64_t *first = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *in = (int64_t *)malloc(sizeof(int64_t) * (size_t)(na + 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t *q = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int rc = ORACLE_OK;
    if (!first || !in || !fill || !q) { rc = ORACLE_ENOMEM; goto done; }
    for (int64_t a = 0; a < na; ++a) {
        if (tail[a] < 0 || tail[a] >= n || head[a] < 0 || head[a] >= n) { rc = ORACLE_EINVAL; goto done; }
        first[head[a] + 1]++;
    }
    for (int64_t v = 0; v < n; ++v) first[v + 1] += first[v];
    memcpy(fill, first, sizeof(int64_t) * (size_t)n);
    for (int64_t a = 0; a < na; ++a) in[fill[head[a]]++] = a;   /* arcs entering v */
    for (int64_t v = 0; v < n; ++v) dist[v] = -1;
    int64_t qh = 0, qt = 0;
    dist[target] = base;
    q[qt++] = target;
    while (qh < qt) {
        int32_t w = q[qh++];
        for (int64_t p = first[w]; p < first[w + 1]; ++p) {
            int64_t a = in[p];
            int32_t v = tail[a];
            if (v == excluded || dist[v] != -1 || rescap[a] <= 0) continue;
            dist[v] = dist[w] + 1;
            q[qt++] = v;
        }
    }
    for (int64_t v = 0; v < n; ++v)
        if (dist[v] == -1) dist[v] = unreach;
    if (excluded >= 0 && excluded < n) dist[excluded] = excluded_h;
done:
    free(first); free(in); free(fill); free(q);
    return rc;
}
