/*
 * dg_oracle.c -- plain CPU oracle for dyGRASS (Yuan, Aghdaei, Feng,
 * "dyGRASS: Dynamic Spectral Graph Sparsification via Localized Random Walks
 * on GPUs", arXiv:2505.02741).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, single-threaded,
 * obviously-correct statement of what the method computes.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline / reference arm load
 * it.  It shares no code, header, table or helper with the CUDA library.
 *
 * What it follows (section / equation / algorithm of the paper):
 *   - Section II-A:   weighted undirected graph, r_e = 1 / w_e.
 *   - Section III-B:  non-backtracking random walk (NBRW) from p toward q; the
 *                     walker accumulates the resistance of the edges it crosses;
 *                     estimate R~_pq = min over the s walkers that reach q
 *                     (Eq. 12); distortion threshold w_pq * R_cum > K stops an
 *                     insertion walker; step limit T; a leaf stops the walker.
 *                     An insertion is kept (added to H) iff no walker reaches q.
 *   - Section III-C:  deletion of an edge of H: remove it, walk on the updated
 *                     G up to T steps, recover the edges of the minimum-
 *                     resistance path that reaches q; if none reaches q,
 *                     recover a few local edges near p and q.
 *   - Algorithm 1:    the stream loop (insertion / deletion branches).
 *   - Section III-F:  the GPU version defers sparsifier updates to the end of
 *                     a batch (one snapshot per batch).
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   R1  neighbour lists are ordered by ascending neighbour id;
 *   R2  random numbers: Philox4x32-10 (Salmon et al., SC'11), counter
 *       (step, walker, lo32(update id), hi32(update id)), key (lo32(seed),
 *       hi32(seed)), output word 0;
 *   R3  the step picks uniformly among the neighbours other than the previous
 *       vertex: j = floor(x * n_eff / 2^32), take the j-th such neighbour in
 *       ascending id order;
 *   R4  a walker that reaches q with w_pq * R <= K has hit (stop only on > K);
 *   R5  reaching q on step T counts as a hit;
 *   R6  deletion walks use no K;  R7 deletion walks start at the update's u;
 *   R8  insertion early exit: all walkers of one update advance in lock-step;
 *       at the first step index k* where any walker hits, every walker stops
 *       (its path is cut at min(own stop, k*));
 *   R9  the argmin walker is the lowest walker id among exact FP64 ties;
 *   R10 recovered edges are the distinct edges of the argmin walker's walk
 *       that are not already in H';
 *   R11 fallback (no walker reached q): for x in (u, v), the incident G edge of
 *       minimum resistance (ties: smaller neighbour id) not already in H';
 *   R12 batch snapshot: validate in update order against a batch-local view of
 *       G; G_b = G with all valid changes; H' = H minus every deleted edge that
 *       was in H at batch start; insertion walks run on H', deletion walks on
 *       G_b; H_b = H' U {kept insertions whose edge is in G_b} U recovered U
 *       fallback, weights taken from G_b.
 *
 * Floating point: FP64 only, each operation rounded on its own (build with
 * -ffp-contract=off); 1/w is computed once per edge.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* update status and walker stop reasons                                     */
/* ------------------------------------------------------------------------ */
enum {
    ORC_OK = 0,
    ORC_SELF_LOOP = 1,
    ORC_BAD_VERTEX = 2,
    ORC_DUP_INSERT = 3,
    ORC_MISSING_DELETE = 4,
    ORC_BAD_WEIGHT = 5,
    ORC_BAD_OP = 6
};
enum { STOP_NONE = 0, STOP_HIT = 1, STOP_OVER_K = 2, STOP_AT_T = 3, STOP_LEAF = 4, STOP_CUT = 5 };
enum { OP_INS = 0, OP_DEL = 1 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random        */
/* numbers: as easy as 1, 2, 3"): 10 rounds of the 4x32 S-box with           */
/* multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key increments               */
/* 0x9E3779B9 / 0xBB67AE85 applied between rounds.                           */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The random word a walker uses at one step (reading R2). */
static uint32_t step_random(uint64_t seed, uint64_t upd_id, uint32_t walker, uint32_t step)
{
    uint32_t ctr[4] = {step, walker, (uint32_t)upd_id, (uint32_t)(upd_id >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[0];
}

/* ------------------------------------------------------------------------ */
/* graph: per-vertex adjacency arrays sorted by neighbour id (reading R1)    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t nbr;
    double w;
    double r; /* 1.0 / w, computed once when the edge is created */
} orc_adj;

typedef struct {
    int32_t n;
    int32_t *deg;
    int32_t *cap;
    orc_adj **adj;
} orc_graph;

static int graph_init(orc_graph *g, int32_t n)
{
    g->n = n;
    g->deg = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    g->cap = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    g->adj = (orc_adj **)calloc((size_t)(n > 0 ? n : 1), sizeof(orc_adj *));
    return (g->deg && g->cap && g->adj) ? 0 : -1;
}

static void graph_free(orc_graph *g)
{
    if (g->adj)
        for (int32_t x = 0; x < g->n; x++) free(g->adj[x]);
    free(g->adj);
    free(g->deg);
    free(g->cap);
    memset(g, 0, sizeof(*g));
}

/* position of y in x's list, or -1 (binary search over the sorted list) */
static int32_t graph_find(const orc_graph *g, int32_t x, int32_t y)
{
    int32_t lo = 0, hi = g->deg[x] - 1;
    const orc_adj *L = g->adj[x];
    while (lo <= hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (L[mid].nbr == y) return mid;
        if (L[mid].nbr < y) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

static int graph_has(const orc_graph *g, int32_t a, int32_t b)
{
    return graph_find(g, a, b) >= 0;
}

/* insert the half edge x->y keeping the list sorted; the caller checked absence */
static int half_insert(orc_graph *g, int32_t x, int32_t y, double w, double r)
{
    if (g->deg[x] == g->cap[x]) {
        int32_t nc = g->cap[x] ? 2 * g->cap[x] : 4;
        orc_adj *p = (orc_adj *)realloc(g->adj[x], (size_t)nc * sizeof(orc_adj));
        if (!p) return -1;
        g->adj[x] = p;
        g->cap[x] = nc;
    }
    orc_adj *L = g->adj[x];
    int32_t k = 0;
    while (k < g->deg[x] && L[k].nbr < y) k++;
    memmove(L + k + 1, L + k, (size_t)(g->deg[x] - k) * sizeof(orc_adj));
    L[k].nbr = y;
    L[k].w = w;
    L[k].r = r;
    g->deg[x]++;
    return 0;
}

static void half_remove(orc_graph *g, int32_t x, int32_t y)
{
    int32_t k = graph_find(g, x, y);
    if (k < 0) return;
    orc_adj *L = g->adj[x];
    memmove(L + k, L + k + 1, (size_t)(g->deg[x] - k - 1) * sizeof(orc_adj));
    g->deg[x]--;
}

static int edge_insert(orc_graph *g, int32_t a, int32_t b, double w, double r)
{
    if (half_insert(g, a, b, w, r)) return -1;
    if (half_insert(g, b, a, w, r)) return -1;
    return 0;
}

static void edge_remove(orc_graph *g, int32_t a, int32_t b)
{
    half_remove(g, a, b);
    half_remove(g, b, a);
}

/* weight and resistance stored for edge (a, b); the edge must exist */
static void edge_wr(const orc_graph *g, int32_t a, int32_t b, double *w, double *r)
{
    int32_t k = graph_find(g, a, b);
    *w = g->adj[a][k].w;
    *r = g->adj[a][k].r;
}

/* ------------------------------------------------------------------------ */
/* state of one dynamic graph                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    orc_graph G;
    orc_graph H;
    uint64_t next_id; /* sequence number of the next submitted update */
    uint64_t seed;
    double K;
    int32_t T;
    int32_t s;
    int32_t early_exit; /* reading R8 on (1) or off (0) */
} orc_state;

static int weight_ok(double w)
{
    return isfinite(w) && w > 0.0;
}

static int adj_cmp(const void *x, const void *y)
{
    const orc_adj *a = (const orc_adj *)x, *b = (const orc_adj *)y;
    return (a->nbr > b->nbr) - (a->nbr < b->nbr);
}

/* G(0): n vertices, m undirected edges; simple, 0 <= ids < n, w > 0 finite.
 * Built list by list: count degrees, fill, sort each list by neighbour id,
 * reject a repeated pair (two equal neighbours in one list). */
orc_state *orc_create(int32_t n, int64_t m, const int32_t *u, const int32_t *v, const double *w,
                      uint64_t seed, double K, int32_t T, int32_t s, int32_t early_exit)
{
    if (n < 0 || m < 0 || T < 1 || s < 1 || !(K >= 0.0)) return NULL;
    orc_state *st = (orc_state *)calloc(1, sizeof(orc_state));
    if (!st) return NULL;
    if (graph_init(&st->G, n) || graph_init(&st->H, n)) goto fail;
    for (int64_t i = 0; i < m; i++) {
        int32_t a = u[i], b = v[i];
        if (a < 0 || a >= n || b < 0 || b >= n || a == b || !weight_ok(w[i])) goto fail;
        st->G.cap[a]++;
        st->G.cap[b]++;
    }
    for (int32_t x = 0; x < n; x++) {
        if (st->G.cap[x] == 0) continue;
        st->G.adj[x] = (orc_adj *)malloc((size_t)st->G.cap[x] * sizeof(orc_adj));
        if (!st->G.adj[x]) goto fail;
    }
    for (int64_t i = 0; i < m; i++) {
        int32_t a = u[i], b = v[i];
        double r = 1.0 / w[i];
        orc_adj *ea = &st->G.adj[a][st->G.deg[a]++];
        ea->nbr = b;
        ea->w = w[i];
        ea->r = r;
        orc_adj *eb = &st->G.adj[b][st->G.deg[b]++];
        eb->nbr = a;
        eb->w = w[i];
        eb->r = r;
    }
    for (int32_t x = 0; x < n; x++) {
        if (st->G.deg[x] > 1) qsort(st->G.adj[x], (size_t)st->G.deg[x], sizeof(orc_adj), adj_cmp);
        for (int32_t k = 1; k < st->G.deg[x]; k++)
            if (st->G.adj[x][k].nbr == st->G.adj[x][k - 1].nbr) goto fail;
    }
    st->seed = seed;
    st->K = K;
    st->T = T;
    st->s = s;
    st->early_exit = early_exit;
    return st;
fail:
    graph_free(&st->G);
    graph_free(&st->H);
    free(st);
    return NULL;
}

void orc_destroy(orc_state *st)
{
    if (!st) return;
    graph_free(&st->G);
    graph_free(&st->H);
    free(st);
}

/* H(0) = the listed edges of G (weights taken from G). Replaces any previous H. */
int orc_init_sparsifier(orc_state *st, int64_t mh, const int32_t *u, const int32_t *v)
{
    int32_t n = st->G.n;
    for (int64_t i = 0; i < mh; i++) {
        if (u[i] < 0 || u[i] >= n || v[i] < 0 || v[i] >= n || u[i] == v[i]) return -1;
        if (!graph_has(&st->G, u[i], v[i])) return -1;
    }
    graph_free(&st->H);
    if (graph_init(&st->H, n)) return -2;
    orc_graph *H = &st->H;
    for (int64_t i = 0; i < mh; i++) {
        H->cap[u[i]]++;
        H->cap[v[i]]++;
    }
    for (int32_t x = 0; x < n; x++) {
        if (H->cap[x] == 0) continue;
        H->adj[x] = (orc_adj *)malloc((size_t)H->cap[x] * sizeof(orc_adj));
        if (!H->adj[x]) return -2;
    }
    for (int64_t i = 0; i < mh; i++) {
        double w, r;
        edge_wr(&st->G, u[i], v[i], &w, &r); /* weights taken from G */
        orc_adj *ea = &H->adj[u[i]][H->deg[u[i]]++];
        ea->nbr = v[i];
        ea->w = w;
        ea->r = r;
        orc_adj *eb = &H->adj[v[i]][H->deg[v[i]]++];
        eb->nbr = u[i];
        eb->w = w;
        eb->r = r;
    }
    for (int32_t x = 0; x < n; x++) { /* sort, then keep a repeated pair once */
        if (H->deg[x] > 1) qsort(H->adj[x], (size_t)H->deg[x], sizeof(orc_adj), adj_cmp);
        int32_t kept = 0;
        for (int32_t k = 0; k < H->deg[x]; k++)
            if (kept == 0 || H->adj[x][k].nbr != H->adj[x][kept - 1].nbr) H->adj[x][kept++] = H->adj[x][k];
        H->deg[x] = kept;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* one non-backtracking walker (Section III-B, III-C)                        */
/* ------------------------------------------------------------------------ */
/* Walks from p toward q on g.  Returns the stop reason; *steps_out = steps
 * taken, *R_out = accumulated resistance.  path (nullable, room for T+1
 * entries) receives the visited vertices, path[0] = p.  rcut: a deletion
 * walker whose resistance exceeds rcut stops there (STOP_CUT, tested before
 * the hit test); +inf walks the plain Algorithm 1 deletion branch. */
static int walk_one(const orc_graph *g, int32_t p, int32_t q, double wpq, int deletion, double K,
                    int32_t T, uint64_t seed, uint64_t upd_id, uint32_t walker, double rcut,
                    int32_t *steps_out, double *R_out, int32_t *path)
{
    int32_t c = p;     /* current vertex */
    int32_t prev = -1; /* previous vertex, none at the start */
    int32_t steps = 0;
    double R = 0.0;
    int reason = STOP_NONE;
    if (path) path[0] = p;
    for (;;) {
        const orc_adj *L = g->adj[c];
        int32_t d = g->deg[c];
        int32_t n_eff = (prev < 0) ? d : d - 1; /* neighbours other than prev */
        if (n_eff <= 0) {
            reason = STOP_LEAF;
            break;
        }
        uint32_t x = step_random(seed, upd_id, walker, (uint32_t)steps);
        uint32_t j = (uint32_t)(((uint64_t)x * (uint64_t)(uint32_t)n_eff) >> 32);
        /* the j-th neighbour (ascending id) that is not prev */
        int32_t pick = -1;
        uint32_t seen = 0;
        for (int32_t k = 0; k < d; k++) {
            if (L[k].nbr == prev) continue;
            if (seen == j) {
                pick = k;
                break;
            }
            seen++;
        }
        R = R + L[pick].r;
        steps = steps + 1;
        prev = c;
        c = L[pick].nbr;
        if (path) path[steps] = c;
        if (deletion && R > rcut) {
            reason = STOP_CUT;
            break;
        }
        if (c == q && (deletion || wpq * R <= K)) {
            reason = STOP_HIT;
            break;
        }
        if (!deletion && wpq * R > K) {
            reason = STOP_OVER_K;
            break;
        }
        if (steps == T) {
            reason = STOP_AT_T;
            break;
        }
    }
    *steps_out = steps;
    *R_out = R;
    return reason;
}

/* exported single-walk entry (used by the sampler pins) */
int orc_walk(const orc_state *st, int use_h, int32_t p, int32_t q, double wpq, int deletion,
             uint64_t upd_id, uint32_t walker, int32_t *steps_out, double *R_out, int32_t *path)
{
    const orc_graph *g = use_h ? &st->H : &st->G;
    if (p < 0 || p >= g->n || q < 0 || q >= g->n) return -1;
    return walk_one(g, p, q, wpq, deletion, st->K, st->T, st->seed, upd_id, walker, INFINITY, steps_out,
                    R_out, path);
}

/* ------------------------------------------------------------------------ */
/* batch application (Algorithm 1 with the deferred-batch reading R12)       */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t a, b; /* a < b */
} orc_pair;

typedef struct {
    orc_pair *e;
    int64_t n, cap;
} orc_pairs;

static int pairs_push(orc_pairs *P, int32_t x, int32_t y)
{
    if (P->n == P->cap) {
        int64_t nc = P->cap ? 2 * P->cap : 64;
        orc_pair *q = (orc_pair *)realloc(P->e, (size_t)nc * sizeof(orc_pair));
        if (!q) return -1;
        P->e = q;
        P->cap = nc;
    }
    P->e[P->n].a = x < y ? x : y;
    P->e[P->n].b = x < y ? y : x;
    P->n++;
    return 0;
}

/* Per-walker debug record (optional output). */
typedef struct {
    int32_t reason; /* after the early-exit cut */
    int32_t steps;  /* after the early-exit cut */
    double R;       /* accumulated resistance, meaningful for hitting walkers */
} orc_walker_out;

/*
 * The s walkers of walked update i on the batch snapshot and what Eq. 12
 * makes of them (Section III-B/C): every walker's stop (wr, s records), the
 * early-exit cut of reading R8, then hit, nhits, the argmin walker (R9),
 * steps and R~.  When nhits_min is given, a deletion with a hit also gets its
 * pruned counts: each walker re-walked with the cut R > R~ (a walker whose
 * resistance exceeds R~ can no longer give the minimum), the walkers at R~,
 * their steps, and (wlo, nullable) every walker's pruned record.  Reads the
 * graphs only; writes only update i's outputs, so the walks of different
 * updates may run at the same time.
 */
static void walk_update(const orc_state *st, const orc_graph *G, const orc_graph *H, int64_t i,
                        const int32_t *u, const int32_t *v, const double *w, const int32_t *op,
                        uint64_t id0, orc_walker_out *wr, int32_t *paths, uint8_t *hit, int32_t *nhits,
                        int32_t *best, int32_t *steps, double *rest, int32_t *nhits_min, int32_t *steps_lo,
                        orc_walker_out *wlo)
{
    const int32_t s = st->s, T = st->T;
    const int deletion = (op[i] == OP_DEL);
    const orc_graph *g = deletion ? G : H;
    const uint64_t upd_id = id0 + (uint64_t)i;
    const double wpq = deletion ? 0.0 : w[i];
    int32_t first_hit = -1; /* smallest step at which some walker hit */
    for (int32_t k = 0; k < s; k++) {
        int32_t *row = paths ? paths + ((size_t)i * s + k) * (size_t)(T + 1) : NULL;
        wr[k].reason = walk_one(g, u[i], v[i], wpq, deletion, st->K, T, st->seed, upd_id, (uint32_t)k,
                                INFINITY, &wr[k].steps, &wr[k].R, row);
        if (row) /* pad the unused tail of the path with -1 */
            for (int32_t t = wr[k].steps + 1; t <= T; t++) row[t] = -1;
        if (wr[k].reason == STOP_HIT && (first_hit < 0 || wr[k].steps < first_hit)) first_hit = wr[k].steps;
    }
    /* reading R8: insertion walkers are cut at the first hitting step (a walker
     * that stopped exactly there for another reason keeps its reason) */
    if (!deletion && st->early_exit && first_hit >= 0) {
        for (int32_t k = 0; k < s; k++) {
            if (wr[k].steps > first_hit) {
                wr[k].steps = first_hit;
                wr[k].reason = STOP_CUT;
                if (paths)
                    for (int32_t t = first_hit + 1; t <= T; t++)
                        paths[((size_t)i * s + k) * (size_t)(T + 1) + t] = -1;
            }
        }
    }
    /* Eq. 12: minimum over the walkers that reached q; ties -> lowest id (R9) */
    int32_t nh = 0, bw = -1, tot = 0;
    double Rmin = INFINITY;
    for (int32_t k = 0; k < s; k++) {
        tot += wr[k].steps;
        if (wr[k].reason != STOP_HIT) continue;
        nh++;
        if (wr[k].R < Rmin) {
            Rmin = wr[k].R;
            bw = k;
        }
    }
    nhits[i] = nh;
    best[i] = bw;
    steps[i] = tot;
    rest[i] = Rmin;
    hit[i] = (uint8_t)(nh > 0);
    if (!nhits_min) return;
    nhits_min[i] = nh;
    steps_lo[i] = tot;
    if (wlo)
        for (int32_t k = 0; k < s; k++) wlo[k] = wr[k];
    if (!deletion || nh == 0) return;
    int32_t nmin = 0, lo = 0;
    for (int32_t k = 0; k < s; k++) {
        orc_walker_out c;
        c.reason = walk_one(g, u[i], v[i], 0.0, 1, st->K, T, st->seed, upd_id, (uint32_t)k, Rmin, &c.steps,
                            &c.R, NULL);
        if (c.reason == STOP_HIT) nmin++; /* a hit under the cut R > R~ has R = R~ */
        lo += c.steps;
        if (wlo) wlo[k] = c;
    }
    nhits_min[i] = nmin;
    steps_lo[i] = lo;
}

/*
 * Apply one batch of nu updates.  Per-update outputs (each an array of nu):
 *   status, walked, hit, accepted, fallback, nhits, best, nrec, steps, rest.
 * Optional: wout (nu*s records) and paths (nu*s*(T+1) vertices, -1 padded).
 * walk_mask (nullable): when given, only updates with a non-zero entry run
 * their walks (a sampling mode for very large batches: statuses and G are
 * complete, walk results and commits only for the sampled updates).
 * nhits_min, steps_lo (nullable, arrays of nu): for a walked deletion with a
 * hit, the number of walkers whose hit resistance equals R~, and the steps
 * the s walkers take when each stops at its first step whose resistance
 * exceeds R~ (a walker there can no longer give the minimum of Eq. 12);
 * otherwise nhits and steps.  These are the deletion-pruning counterparts of
 * nhits and steps: the minimum walker, R~ and the recovered edges are the
 * same with or without pruning.  wout_lo (nullable, nu*s records, only with
 * nhits_min): every walker's record under that cut (the plain record where
 * no cut applies).
 * Returns 0, or -2 on allocation failure.
 */
int orc_apply_batch(orc_state *st, int64_t nu, const int32_t *u, const int32_t *v, const double *w,
                    const int32_t *op, int32_t *status, uint8_t *walked, uint8_t *hit,
                    uint8_t *accepted, uint8_t *fallback, int32_t *nhits, int32_t *best,
                    int32_t *nrec, int32_t *steps, double *rest, orc_walker_out *wout,
                    int32_t *paths, const uint8_t *walk_mask, int32_t *nhits_min, int32_t *steps_lo,
                    orc_walker_out *wout_lo)
{
    orc_graph *G = &st->G, *H = &st->H;
    const int32_t n = G->n, s = st->s, T = st->T;
    const uint64_t id0 = st->next_id;
    int rc = 0;
    orc_pairs commit = {0}, hdel = {0};
    orc_walker_out *wr = wout ? wout : (orc_walker_out *)malloc((size_t)(nu > 0 ? nu : 1) * s * sizeof(orc_walker_out));
    int32_t *best_path = (int32_t *)malloc((size_t)(T + 1) * sizeof(int32_t));
    if (!wr || !best_path) {
        rc = -2;
        goto done;
    }

    /* (i) validation in update order against a batch-local view of G.  The
     * view is G itself, changed in order; H is not touched here, so the
     * membership test below sees H at batch start. */
    for (int64_t i = 0; i < nu; i++) {
        walked[i] = hit[i] = accepted[i] = fallback[i] = 0;
        nhits[i] = 0;
        best[i] = -1;
        nrec[i] = 0;
        steps[i] = 0;
        rest[i] = INFINITY;
        if (nhits_min) nhits_min[i] = steps_lo[i] = 0;
        for (int32_t k = 0; k < s; k++) {
            wr[(size_t)i * s + k].reason = STOP_NONE;
            wr[(size_t)i * s + k].steps = 0;
            wr[(size_t)i * s + k].R = 0.0;
            if (wout_lo) wout_lo[(size_t)i * s + k] = wr[(size_t)i * s + k];
        }
        int32_t a = u[i], b = v[i];
        if (op[i] != OP_INS && op[i] != OP_DEL) {
            status[i] = ORC_BAD_OP;
            continue;
        }
        if (a < 0 || a >= n || b < 0 || b >= n) {
            status[i] = ORC_BAD_VERTEX;
            continue;
        }
        if (a == b) {
            status[i] = ORC_SELF_LOOP;
            continue;
        }
        if (op[i] == OP_INS) {
            if (!weight_ok(w[i])) {
                status[i] = ORC_BAD_WEIGHT;
                continue;
            }
            if (graph_has(G, a, b)) {
                status[i] = ORC_DUP_INSERT;
                continue;
            }
            if (edge_insert(G, a, b, w[i], 1.0 / w[i])) {
                rc = -2;
                goto done;
            }
            status[i] = ORC_OK;
            walked[i] = 1; /* every valid insertion is tested by walks on H' */
        } else {
            if (!graph_has(G, a, b)) {
                status[i] = ORC_MISSING_DELETE;
                continue;
            }
            edge_remove(G, a, b);
            status[i] = ORC_OK;
            if (graph_has(H, a, b)) { /* in H at batch start: Algorithm 1, deletion branch */
                walked[i] = 1;
                if (pairs_push(&hdel, a, b)) {
                    rc = -2;
                    goto done;
                }
            }
        }
    }

    /* (ii) H' = H minus the deleted sparsifier edges (G is now G_b). */
    for (int64_t k = 0; k < hdel.n; k++) edge_remove(H, hdel.e[k].a, hdel.e[k].b);

    /* (iii) walks from the snapshot (H' for insertions, G_b for deletions).
     * Every update's walks read the same snapshot and fill only its own
     * outputs; the OpenMP build of this file runs them on several host
     * threads (identical results: nothing here depends on their order). */
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < nu; i++) {
        if (!walked[i]) continue;
        if (walk_mask && !walk_mask[i]) continue;
        walk_update(st, G, H, i, u, v, w, op, id0, wr + (size_t)i * s, paths, hit, nhits, best, steps, rest,
                    nhits_min, steps_lo, wout_lo ? wout_lo + (size_t)i * s : NULL);
    }

    /* (iv) the edges each update returns, in update order. */
    for (int64_t i = 0; i < nu; i++) {
        if (!walked[i]) continue;
        if (walk_mask && !walk_mask[i]) continue;
        const int deletion = (op[i] == OP_DEL);
        const int32_t nh = nhits[i], bw = best[i];
        if (!deletion) {
            /* Section III-B: kept iff q was not reached by any walker. */
            accepted[i] = (uint8_t)(nh == 0);
            if (accepted[i] && graph_has(G, u[i], v[i]))
                if (pairs_push(&commit, u[i], v[i])) {
                    rc = -2;
                    goto done;
                }
            continue;
        }

        /* Section III-C: deletion of a sparsifier edge. */
        int32_t emitted = 0;
        if (nh > 0) {
            /* re-run the argmin walker to get its walk (same counters -> same path) */
            int32_t ts;
            double tR;
            walk_one(G, u[i], v[i], 0.0, 1, st->K, T, st->seed, id0 + (uint64_t)i, (uint32_t)bw, INFINITY, &ts,
                     &tR, best_path);
            /* R10: distinct edges of the walk that are not in H' */
            for (int32_t t = 0; t < ts; t++) {
                int32_t x = best_path[t], y = best_path[t + 1];
                int dup = 0;
                for (int32_t t2 = 0; t2 < t; t2++) {
                    int32_t x2 = best_path[t2], y2 = best_path[t2 + 1];
                    if ((x2 == x && y2 == y) || (x2 == y && y2 == x)) {
                        dup = 1;
                        break;
                    }
                }
                if (dup || graph_has(H, x, y)) continue;
                if (pairs_push(&commit, x, y)) {
                    rc = -2;
                    goto done;
                }
                emitted++;
            }
        } else {
            /* R11: fallback -- for each endpoint, its minimum-resistance G_b edge not in H' */
            fallback[i] = 1;
            int32_t pick_x[2] = {-1, -1}, pick_y[2] = {-1, -1};
            const int32_t ends[2] = {u[i], v[i]};
            for (int e = 0; e < 2; e++) {
                int32_t x = ends[e];
                double rmin = INFINITY;
                for (int32_t k = 0; k < G->deg[x]; k++) {
                    const orc_adj *A = &G->adj[x][k];
                    if (graph_has(H, x, A->nbr)) continue;
                    if (A->r < rmin) { /* ascending ids: first minimum = smaller id */
                        rmin = A->r;
                        pick_x[e] = x;
                        pick_y[e] = A->nbr;
                    }
                }
            }
            for (int e = 0; e < 2; e++) {
                if (pick_x[e] < 0) continue;
                if (e == 1 && pick_x[0] >= 0 &&
                    ((pick_x[0] == pick_x[1] && pick_y[0] == pick_y[1]) ||
                     (pick_x[0] == pick_y[1] && pick_y[0] == pick_x[1])))
                    continue;
                if (pairs_push(&commit, pick_x[e], pick_y[e])) {
                    rc = -2;
                    goto done;
                }
                emitted++;
            }
        }
        nrec[i] = emitted;
    }

    /* (v) H_b = H' U committed edges (set union; weights from G_b). */
    for (int64_t k = 0; k < commit.n; k++) {
        int32_t a = commit.e[k].a, b = commit.e[k].b;
        if (graph_has(H, a, b)) continue;
        double ww, rr;
        edge_wr(G, a, b, &ww, &rr);
        if (edge_insert(H, a, b, ww, rr)) {
            rc = -2;
            goto done;
        }
    }
    st->next_id = id0 + (uint64_t)nu;

done:
    free(commit.e);
    free(hdel.e);
    if (wr != wout) free(wr);
    free(best_path);
    return rc;
}

/* Threads the walk phase may use (the OpenMP build; a no-op otherwise). */
#ifdef _OPENMP
#include <omp.h>
#endif
void orc_set_threads(int32_t k)
{
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}

int32_t orc_max_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* queries                                                                   */
/* ------------------------------------------------------------------------ */
/* Edges (a < b) of H (which = 1) or G (which = 0) in lexicographic order.
 * Writes at most cap entries; returns the total count. */
int64_t orc_query(const orc_state *st, int which, int64_t cap, int32_t *a, int32_t *b, double *w)
{
    const orc_graph *g = which ? &st->H : &st->G;
    int64_t cnt = 0;
    for (int32_t x = 0; x < g->n; x++)
        for (int32_t k = 0; k < g->deg[x]; k++) {
            if (g->adj[x][k].nbr <= x) continue;
            if (cnt < cap) {
                a[cnt] = x;
                b[cnt] = g->adj[x][k].nbr;
                w[cnt] = g->adj[x][k].w;
            }
            cnt++;
        }
    return cnt;
}

/* Degree of x in H (which = 1) or G (which = 0). */
int32_t orc_degree(const orc_state *st, int which, int32_t x)
{
    const orc_graph *g = which ? &st->H : &st->G;
    return (x >= 0 && x < g->n) ? g->deg[x] : -1;
}

uint64_t orc_next_id(const orc_state *st)
{
    return st->next_id;
}

void orc_set_next_id(orc_state *st, uint64_t id)
{
    st->next_id = id;
}

/* ------------------------------------------------------------------------ */
/* spanning-forest stretch (the initial sparsifier of Section III-A)         */
/* ------------------------------------------------------------------------ */
/*
 * The paper takes H(0) from GRASS: a spanning tree plus the off-tree edges
 * that are spectrally critical.  Reading R20: an off-tree edge e = (p, q) is
 * ranked by its stretch w_e * R_T(p, q), where R_T is the resistance of the
 * tree path between p and q -- the distortion dyGRASS's own insertion test
 * measures (Section III-B), which on a tree H is exact because the walk
 * between p and q is the tree path.  R_T is formed from root distances:
 * every tree is rooted at its smallest vertex, D[root] = 0 and D[y] =
 * D[x] + r(x, y) for a child y of x (r = 1 / w, one rounding each), and
 * R_T(p, q) = (D[p] - D[l]) + (D[q] - D[l]) with l the lowest common
 * ancestor.  p and q in different trees: R_T = +inf.
 *
 * n vertices; m edges (a[i], b[i], w[i]) of G; in_tree[i] != 0 marks the
 * edges of the spanning forest.  stretch[i] receives w * R_T for off-tree
 * edges and 0 for tree edges.  Returns 0, -1 if the marked edges contain a
 * cycle or a bad vertex, -2 on allocation failure.
 */
int orc_tree_stretch(int32_t n, int64_t m, const int32_t *a, const int32_t *b, const double *w,
                     const uint8_t *in_tree, double *stretch)
{
    int rc = 0;
    int64_t nt = 0;
    for (int64_t i = 0; i < m; i++) nt += in_tree[i] ? 1 : 0;
    int32_t *deg = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    int64_t *start = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *nb = (int32_t *)malloc((size_t)(2 * nt + 1) * sizeof(int32_t));
    double *nr = (double *)malloc((size_t)(2 * nt + 1) * sizeof(double));
    int32_t *parent = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *depth = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *root = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    double *D = (double *)malloc((size_t)n * sizeof(double));
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int64_t *fill = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    if (!deg || !start || !nb || !nr || !parent || !depth || !root || !D || !queue || !fill) {
        rc = -2;
        goto done;
    }
    /* adjacency of the forest */
    for (int64_t i = 0; i < m; i++) {
        if (!in_tree[i]) continue;
        if (a[i] < 0 || a[i] >= n || b[i] < 0 || b[i] >= n || a[i] == b[i]) {
            rc = -1;
            goto done;
        }
        deg[a[i]]++;
        deg[b[i]]++;
    }
    for (int32_t x = 0; x < n; x++) start[x + 1] = start[x] + deg[x];
    for (int32_t x = 0; x <= n; x++) fill[x] = start[x];
    for (int64_t i = 0; i < m; i++) {
        if (!in_tree[i]) continue;
        const double r = 1.0 / w[i];
        nb[fill[a[i]]] = b[i];
        nr[fill[a[i]]++] = r;
        nb[fill[b[i]]] = a[i];
        nr[fill[b[i]]++] = r;
    }
    /* root every tree at its smallest vertex; breadth-first from it */
    for (int32_t x = 0; x < n; x++) root[x] = -1;
    int64_t reached_edges = 0;
    for (int32_t s = 0; s < n; s++) {
        if (root[s] >= 0) continue;
        int32_t head = 0, tail = 0;
        root[s] = s;
        parent[s] = s;
        depth[s] = 0;
        D[s] = 0.0;
        queue[tail++] = s;
        while (head < tail) {
            const int32_t x = queue[head++];
            for (int64_t k = start[x]; k < start[x + 1]; k++) {
                const int32_t y = nb[k];
                if (y == parent[x] && x != s) continue; /* the edge back to the parent */
                if (root[y] >= 0) { /* reached twice: the marked edges close a cycle */
                    rc = -1;
                    goto done;
                }
                root[y] = s;
                parent[y] = x;
                depth[y] = depth[x] + 1;
                D[y] = D[x] + nr[k];
                queue[tail++] = y;
                reached_edges++;
            }
        }
    }
    if (reached_edges != nt) { /* a repeated tree edge */
        rc = -1;
        goto done;
    }
    /* stretch of every off-tree edge through its lowest common ancestor */
    for (int64_t i = 0; i < m; i++) {
        if (in_tree[i]) {
            stretch[i] = 0.0;
            continue;
        }
        int32_t p = a[i], q = b[i];
        if (root[p] != root[q]) {
            stretch[i] = INFINITY;
            continue;
        }
        int32_t x = p, y = q;
        while (depth[x] > depth[y]) x = parent[x];
        while (depth[y] > depth[x]) y = parent[y];
        while (x != y) {
            x = parent[x];
            y = parent[y];
        }
        const double R = (D[p] - D[x]) + (D[q] - D[x]);
        stretch[i] = w[i] * R;
    }
done:
    free(deg);
    free(start);
    free(nb);
    free(nr);
    free(parent);
    free(depth);
    free(root);
    free(D);
    free(queue);
    free(fill);
    return rc;
}
