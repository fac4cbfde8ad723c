/*
 * mapgen.c -- seeded synthetic workloads for MAP accepting-cycle detection.
 *
 * This module only BUILDS inputs: CSR successor lists (row v = the successors
 * of state v in the state graph G), one accepting flag per vertex, batch plans
 * and arrival schedules.  It holds none of MAP's own arithmetic (no value
 * propagation, no cycle test, no elimination), so both the CPU oracle and the
 * GPU path can consume its output without sharing any method code.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded through
 * SplitMix64 (Steele, Lea & Flood, 2014), both written here from their
 * published definitions.  Every draw that shapes a graph is integer-only
 * (bounded integers by 128-bit multiply-high), so a seed gives the same graph
 * on x86_64 and aarch64.  Only the batch-size and arrival-time draws use
 * libm (exp/log/cos/sqrt); those feed schedules, not graph structure.
 *
 * The workloads stand in for the DiVinE models of the paper (Section 4),
 * which are not available: see each generator for the recipe.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "mapgen.h"

/* ------------------------------------------------------------------ RNG -- */

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t *x)
{
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void rng_seed(rng_t *r, uint64_t seed, uint64_t stream)
{
    uint64_t x = seed ^ (stream * 0xD1B54A32D192ED03ull);
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_u64(rng_t *r)
{
    uint64_t *s = r->s;
    const uint64_t out = rotl64(s[1] * 5u, 7) * 9u;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return out;
}

/* uniform integer in [0, k), k >= 1 (multiply-high; bias below 2^-32 for k < 2^32) */
static inline uint32_t rng_below(rng_t *r, uint32_t k)
{
    return (uint32_t)(((unsigned __int128)rng_u64(r) * k) >> 64);
}

/* Bernoulli with probability num / 1e6 */
static inline int rng_ppm(rng_t *r, uint32_t num) { return rng_below(r, 1000000u) < num; }

/* uniform double in [0, 1) with 53 random bits */
static inline double rng_unit(rng_t *r) { return (double)(rng_u64(r) >> 11) * (1.0 / 9007199254740992.0); }

/* ------------------------------------------------------------ utilities -- */

void mg_free(mg_graph *g)
{
    if (!g) return;
    free(g->rowptr);
    free(g->colidx);
    free(g->acc);
    g->rowptr = NULL;
    g->colidx = NULL;
    g->acc = NULL;
    g->n = 0;
    g->m = 0;
}

static int alloc_graph(mg_graph *g, uint32_t n, uint64_t m)
{
    memset(g, 0, sizeof(*g));
    g->n = n;
    g->m = m;
    g->rowptr = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    g->colidx = (uint32_t *)malloc(sizeof(uint32_t) * (m ? (size_t)m : 1));
    g->acc = (uint8_t *)calloc((size_t)n ? (size_t)n : 1, 1);
    if (!g->rowptr || !g->colidx || !g->acc) {
        mg_free(g);
        return MG_ERR_OOM;
    }
    return MG_OK;
}

/* Append extra edges (src[i] -> dst[i]) at the end of their source rows. */
int mg_add_edges(mg_graph *g, uint32_t count, const uint32_t *src, const uint32_t *dst)
{
    if (count == 0) return MG_OK;
    for (uint32_t i = 0; i < count; ++i)
        if (src[i] >= g->n || dst[i] >= g->n) return MG_ERR_ARG;
    if ((uint64_t)g->m + count > 0xFFFFFFFFull) return MG_ERR_ARG;
    uint32_t *extra = (uint32_t *)calloc((size_t)g->n, sizeof(uint32_t));
    if (!extra) return MG_ERR_OOM;
    for (uint32_t i = 0; i < count; ++i) extra[src[i]]++;
    uint64_t m2 = g->m + count;
    uint32_t *rp = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)g->n + 1));
    uint32_t *ci = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)m2);
    if (!rp || !ci) {
        free(extra); free(rp); free(ci);
        return MG_ERR_OOM;
    }
    rp[0] = 0;
    for (uint32_t v = 0; v < g->n; ++v) {
        uint32_t deg = g->rowptr[v + 1] - g->rowptr[v];
        memcpy(ci + rp[v], g->colidx + g->rowptr[v], sizeof(uint32_t) * deg);
        rp[v + 1] = rp[v] + deg + extra[v];
        extra[v] = rp[v] + deg; /* reuse as the insertion cursor */
    }
    for (uint32_t i = 0; i < count; ++i) ci[extra[src[i]]++] = dst[i];
    free(extra);
    free(g->rowptr);
    free(g->colidx);
    g->rowptr = rp;
    g->colidx = ci;
    g->m = m2;
    return MG_OK;
}

/*
 * Kahn peeling: repeatedly remove vertices of in-degree 0.  The removed set is
 * exactly the set of vertices that no cycle reaches, so none of them lies on a
 * cycle.  peeled[v] = 1 for those.  Returns how many were peeled.
 */
uint32_t mg_peel(uint32_t n, const uint32_t *rowptr, const uint32_t *colidx, uint8_t *peeled)
{
    uint32_t *indeg = (uint32_t *)calloc((size_t)n ? n : 1, sizeof(uint32_t));
    uint32_t *queue = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n ? n : 1));
    if (!indeg || !queue) {
        free(indeg); free(queue);
        return 0;
    }
    for (uint64_t e = 0; e < rowptr[n]; ++e) indeg[colidx[e]]++;
    uint32_t head = 0, tail = 0;
    memset(peeled, 0, n);
    for (uint32_t v = 0; v < n; ++v)
        if (indeg[v] == 0) queue[tail++] = v;
    while (head < tail) {
        uint32_t v = queue[head++];
        peeled[v] = 1;
        for (uint32_t e = rowptr[v]; e < rowptr[v + 1]; ++e)
            if (--indeg[colidx[e]] == 0) queue[tail++] = colidx[e];
    }
    free(indeg);
    free(queue);
    return tail;
}

/* ---------------------------------------------------- random graphs -- -- */

/*
 * Uniform random digraph: vertex v gets deg_lo..deg_hi successors (uniform),
 * drawn uniformly without replacement among the other vertices (no self-loop);
 * each vertex is accepting with probability acc_ppm / 1e6.
 *
 * variant 0: as drawn.
 * variant 1 ("no cycle"): the k accepting flags drawn above are moved onto k
 *   vertices drawn uniformly from the peeled set (vertices that no cycle
 *   reaches, hence on no cycle); info[0] = k, info[1] = flags placed.
 * variant 2 ("cycle"): variant 1, then a = the largest accepting id gets a
 *   planted cycle a -> v1 -> ... -> v(len-1) -> a through len-1 distinct
 *   non-accepting vertices; info[2] = a.  With a the largest accepting id,
 *   map(a) = a, so the expected verdict is a cycle with witness a at the
 *   first outer iteration.
 */
int mg_random(uint32_t n, uint32_t deg_lo, uint32_t deg_hi, uint32_t acc_ppm, uint64_t seed,
              int variant, uint32_t cycle_len, mg_graph *g)
{
    if (n < 2 || deg_lo < 1 || deg_hi < deg_lo || deg_hi > n - 1 || variant < 0 || variant > 2)
        return MG_ERR_ARG;
    rng_t rdeg, rtgt, racc, rmove;
    rng_seed(&rdeg, seed, 1);
    rng_seed(&rtgt, seed, 2);
    rng_seed(&racc, seed, 3);
    rng_seed(&rmove, seed, 4);

    uint32_t *deg = (uint32_t *)malloc(sizeof(uint32_t) * n);
    if (!deg) return MG_ERR_OOM;
    uint64_t m = 0;
    for (uint32_t v = 0; v < n; ++v) {
        deg[v] = deg_lo + rng_below(&rdeg, deg_hi - deg_lo + 1);
        m += deg[v];
    }
    int rc = alloc_graph(g, n, m);
    if (rc) {
        free(deg);
        return rc;
    }
    g->rowptr[0] = 0;
    for (uint32_t v = 0; v < n; ++v) {
        uint32_t base = g->rowptr[v];
        for (uint32_t j = 0; j < deg[v]; ++j) {
            uint32_t u;
            for (;;) {
                u = rng_below(&rtgt, n);
                if (u == v) continue;
                int dup = 0;
                for (uint32_t i = 0; i < j; ++i)
                    if (g->colidx[base + i] == u) { dup = 1; break; }
                if (!dup) break;
            }
            g->colidx[base + j] = u;
        }
        g->rowptr[v + 1] = base + deg[v];
    }
    free(deg);
    for (uint32_t v = 0; v < n; ++v) g->acc[v] = (uint8_t)rng_ppm(&racc, acc_ppm);
    if (variant == 0) return MG_OK;

    /* move the accepting flags onto vertices that no cycle reaches */
    uint32_t k = 0;
    for (uint32_t v = 0; v < n; ++v) k += g->acc[v];
    uint8_t *peeled = (uint8_t *)malloc(n);
    uint32_t *pool = (uint32_t *)malloc(sizeof(uint32_t) * n);
    if (!peeled || !pool) {
        free(peeled); free(pool); mg_free(g);
        return MG_ERR_OOM;
    }
    mg_peel(n, g->rowptr, g->colidx, peeled);
    uint32_t np = 0;
    for (uint32_t v = 0; v < n; ++v)
        if (peeled[v]) pool[np++] = v;
    memset(g->acc, 0, n);
    uint32_t placed = k < np ? k : np;
    for (uint32_t i = 0; i < placed; ++i) { /* partial Fisher-Yates */
        uint32_t j = i + rng_below(&rmove, np - i);
        uint32_t t = pool[i]; pool[i] = pool[j]; pool[j] = t;
        g->acc[pool[i]] = 1;
    }
    free(peeled);
    free(pool);
    g->info[0] = k;
    g->info[1] = placed;
    if (variant == 1) return MG_OK;

    /* plant one accepting cycle through the largest accepting id */
    if (placed == 0 || cycle_len < 1 || cycle_len > n) return MG_ERR_ARG;
    uint32_t a = 0;
    for (uint32_t v = 0; v < n; ++v)
        if (g->acc[v]) a = v;
    uint32_t *cyc = (uint32_t *)malloc(sizeof(uint32_t) * (cycle_len + 1));
    uint32_t *src = (uint32_t *)malloc(sizeof(uint32_t) * cycle_len);
    uint32_t *dst = (uint32_t *)malloc(sizeof(uint32_t) * cycle_len);
    if (!cyc || !src || !dst) {
        free(cyc); free(src); free(dst); mg_free(g);
        return MG_ERR_OOM;
    }
    cyc[0] = a;
    for (uint32_t i = 1; i < cycle_len; ++i) {
        uint32_t u;
        for (;;) {
            u = rng_below(&rmove, n);
            if (g->acc[u]) continue;
            int dup = 0;
            for (uint32_t j = 1; j < i; ++j)
                if (cyc[j] == u) { dup = 1; break; }
            if (!dup) break;
        }
        cyc[i] = u;
    }
    cyc[cycle_len] = a;
    for (uint32_t i = 0; i < cycle_len; ++i) {
        src[i] = cyc[i];
        dst[i] = cyc[i + 1];
    }
    rc = mg_add_edges(g, cycle_len, src, dst);
    free(cyc); free(src); free(dst);
    g->info[2] = a;
    return rc;
}

/* ------------------------------------------------- process products -- */

static uint64_t ipow(uint64_t b, uint32_t e)
{
    uint64_t r = 1;
    while (e--) r *= b;
    return r;
}

/*
 * State space of k cyclic processes with s local states each, crossed with a
 * two-state Buchi automaton.
 *
 * A system state is (x_0 .. x_{k-1}); process i is enabled when x_{(i+1) mod k}
 * is even, and a move of process i sets x_i := (x_i + 1) mod s.
 *  interleave = 0 (synchronous / lock-step): every enabled process moves at
 *    once, so each state has exactly one successor (itself when none moves).
 *  interleave = 1: one enabled process moves per step (one successor per
 *    enabled process; a stutter self-loop when none is enabled).
 * The automaton state after a step is b' = [x'_0 == 3]; a product vertex is
 * accepting iff b = 1.  All 2 * s^k pairs (x, b) are enumerated; the id of
 * (x, b) is b * s^k + sum_i x_i * s^i.  Needs s >= 4.
 */
int mg_product(uint32_t k, uint32_t s, int interleave, mg_graph *g)
{
    if (k < 1 || k > 20 || s < 4) return MG_ERR_ARG;
    uint64_t N = ipow(s, k);
    if (2 * N >= 0x7FFFFFFFull) return MG_ERR_ARG;
    uint32_t n = (uint32_t)(2 * N);
    uint32_t x[32], y[32];
    uint64_t pw[32];
    for (uint32_t i = 0; i < k; ++i) pw[i] = ipow(s, i);

    /* count edges */
    uint64_t m = 0;
    if (!interleave) {
        m = n;
    } else {
        for (uint64_t id = 0; id < N; ++id) {
            uint64_t t = id;
            for (uint32_t i = 0; i < k; ++i) { x[i] = (uint32_t)(t % s); t /= s; }
            uint32_t en = 0;
            for (uint32_t i = 0; i < k; ++i) en += (x[(i + 1) % k] % 2 == 0);
            m += en ? en : 1;
        }
        m *= 2;
    }
    if (m > 0xFFFFFFFFull) return MG_ERR_ARG;
    int rc = alloc_graph(g, n, m);
    if (rc) return rc;
    uint64_t e = 0;
    for (uint32_t b = 0; b < 2; ++b) {
        for (uint64_t id = 0; id < N; ++id) {
            uint32_t v = (uint32_t)(b * N + id);
            g->rowptr[v] = (uint32_t)e;
            g->acc[v] = (uint8_t)b;
            uint64_t t = id;
            for (uint32_t i = 0; i < k; ++i) { x[i] = (uint32_t)(t % s); t /= s; }
            if (!interleave) {
                uint64_t to = 0;
                for (uint32_t i = 0; i < k; ++i) {
                    y[i] = (x[(i + 1) % k] % 2 == 0) ? (x[i] + 1) % s : x[i];
                    to += y[i] * pw[i];
                }
                g->colidx[e++] = (uint32_t)((y[0] == 3 ? N : 0) + to);
            } else {
                uint32_t en = 0;
                for (uint32_t i = 0; i < k; ++i) {
                    if (x[(i + 1) % k] % 2 != 0) continue;
                    ++en;
                    uint32_t xi = (x[i] + 1) % s;
                    uint64_t to = id - x[i] * pw[i] + xi * pw[i];
                    uint32_t y0 = (i == 0) ? xi : x[0];
                    g->colidx[e++] = (uint32_t)((y0 == 3 ? N : 0) + to);
                }
                if (!en) g->colidx[e++] = (uint32_t)((x[0] == 3 ? N : 0) + id);
            }
        }
    }
    g->rowptr[n] = (uint32_t)e;
    return MG_OK;
}

/* ------------------------------------------------- layered graphs - -- */

/* first vertex of layer l when n vertices are split into L layers by
 * layer(v) = floor(v * L / n) */
static inline uint32_t layer_start(uint64_t l, uint64_t n, uint64_t L) { return (uint32_t)((l * n + L - 1) / L); }

/*
 * Layered "BFS-shaped" state graph with accepting vertices on no cycle.
 *
 * Vertices are split into L layers of consecutive ids; each vertex is
 * accepting with probability acc_ppm / 1e6.  Every vertex draws its out-degree
 * from a geometric law on {1, 2, ...} with mean 4 (the number of independent
 * trials with success probability 1/4 up to the first success, capped at 64).
 * Each edge is a forward edge (probability fwd_ppm / 1e6, always on layer 0,
 * never on the last layer) to a vertex of the next layer, or else a back edge to
 * a vertex of one of the previous `window` layers.  Duplicate targets within a
 * row are redrawn (up to 64 times).
 *   non-accepting source: targets are uniform NON-accepting vertices of the
 *     chosen layer range, so the non-accepting vertices form one giant
 *     strongly connected component that never points into an accepting vertex.
 *   accepting source: a forward edge targets a uniform accepting vertex of the
 *     next layer with probability accfwd_ppm / 1e6 unless the next layer starts
 *     a new segment of D layers ((l+1) mod D == 0); otherwise it targets a
 *     uniform non-accepting vertex.  Back edges target non-accepting vertices.
 * Accepting-to-accepting edges thus only go forward inside a D-layer segment,
 * and nothing reachable from a non-accepting vertex is accepting, so no
 * accepting vertex lies on a cycle; the accepting vertices form a DAG of depth
 * at most D, which makes MAP need many outer iterations (about D and more).
 *
 * plant = 1 adds one edge w -> a, where a is a uniform accepting vertex that
 * has a non-accepting successor and w is a uniform one of those successors,
 * closing the cycle a -> w -> a through an accepting vertex.  info[0] = a,
 * info[1] = w, info[2] = number of layers.
 */
int mg_layered(uint32_t n, uint32_t L, uint32_t D, uint32_t window, uint32_t acc_ppm, uint32_t fwd_ppm,
               uint32_t accfwd_ppm, uint64_t seed, int plant, mg_graph *g)
{
    if (n < 2 || L < 1 || L > n || D < 1 || window < 1 || n >= 0x7FFFFFFFu) return MG_ERR_ARG;
    rng_t racc, rdeg, rtgt, rplant;
    rng_seed(&racc, seed, 11);
    rng_seed(&rdeg, seed, 12);
    rng_seed(&rtgt, seed, 13);
    rng_seed(&rplant, seed, 14);

    uint8_t *acc = (uint8_t *)malloc(n);
    uint32_t *deg = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    /* ids of accepting / non-accepting vertices in id order; per-layer offsets */
    uint32_t *alist = NULL, *nlist = NULL, *aoff = NULL, *noff = NULL;
    aoff = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)L + 1));
    noff = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)L + 1));
    if (!acc || !deg || !aoff || !noff) goto oom;
    uint32_t na = 0;
    for (uint32_t v = 0; v < n; ++v) {
        acc[v] = (uint8_t)rng_ppm(&racc, acc_ppm);
        na += acc[v];
    }
    alist = (uint32_t *)malloc(sizeof(uint32_t) * (na ? na : 1));
    nlist = (uint32_t *)malloc(sizeof(uint32_t) * ((n - na) ? (n - na) : 1));
    if (!alist || !nlist) goto oom;
    {
        uint32_t ia = 0, in = 0;
        for (uint32_t l = 0; l < L; ++l) {
            aoff[l] = ia;
            noff[l] = in;
            uint32_t lo = layer_start(l, n, L), hi = layer_start(l + 1, n, L);
            for (uint32_t v = lo; v < hi; ++v) {
                if (acc[v]) alist[ia++] = v;
                else nlist[in++] = v;
            }
        }
        aoff[L] = ia;
        noff[L] = in;
    }
    uint64_t m = 0;
    for (uint32_t v = 0; v < n; ++v) {
        uint32_t d = 1;
        while (d < 64 && (rng_u64(&rdeg) & 3u) != 0) ++d;
        deg[v] = d;
        m += d;
    }
    if (m > 0xFFFFFFFFull) goto arg;
    if (alloc_graph(g, n, m)) goto oom;
    memcpy(g->acc, acc, n);
    {
        uint64_t e = 0;
        for (uint32_t l = 0; l < L; ++l) {
            uint32_t lo = layer_start(l, n, L), hi = layer_start(l + 1, n, L);
            uint32_t blo = l > window ? l - window : 0; /* back window [blo, l) */
            for (uint32_t v = lo; v < hi; ++v) {
                g->rowptr[v] = (uint32_t)e;
                uint64_t row0 = e;
                for (uint32_t j = 0; j < deg[v]; ++j) {
                    uint32_t u = 0;
                    int have = 0;
                    for (int tries = 0; tries < 64; ++tries) {
                        int fwd = (l + 1 < L) && (l == 0 || rng_ppm(&rtgt, fwd_ppm));
                        const uint32_t *list;
                        uint32_t a0, a1;
                        if (fwd) {
                            int to_acc = acc[v] && ((l + 1) % D != 0) && aoff[l + 2] > aoff[l + 1] &&
                                         rng_ppm(&rtgt, accfwd_ppm);
                            if (to_acc) { list = alist; a0 = aoff[l + 1]; a1 = aoff[l + 2]; }
                            else        { list = nlist; a0 = noff[l + 1]; a1 = noff[l + 2]; }
                        } else {
                            list = nlist;
                            a0 = noff[blo];
                            a1 = noff[l];
                        }
                        if (a1 <= a0) continue; /* empty range: redraw */
                        u = list[a0 + rng_below(&rtgt, a1 - a0)];
                        have = 1;
                        int dup = 0;
                        for (uint64_t i = row0; i < e; ++i)
                            if (g->colidx[i] == u) { dup = 1; break; }
                        if (!dup) break;
                    }
                    if (have) g->colidx[e++] = u;
                }
            }
        }
        g->rowptr[n] = (uint32_t)e;
        g->m = e;
    }
    g->info[2] = L;
    if (plant) {
        /* accepting vertices with a non-accepting successor */
        uint32_t cnt = 0;
        for (uint32_t i = 0; i < na; ++i) {
            uint32_t a = alist[i];
            for (uint32_t e = g->rowptr[a]; e < g->rowptr[a + 1]; ++e)
                if (!acc[g->colidx[e]]) { cnt++; break; }
        }
        if (cnt == 0) goto arg;
        uint32_t pick = rng_below(&rplant, cnt), a = 0;
        for (uint32_t i = 0; i < na; ++i) {
            uint32_t c = alist[i];
            int ok = 0;
            for (uint32_t e = g->rowptr[c]; e < g->rowptr[c + 1]; ++e)
                if (!acc[g->colidx[e]]) { ok = 1; break; }
            if (ok && pick-- == 0) { a = c; break; }
        }
        uint32_t nn = 0;
        for (uint32_t e = g->rowptr[a]; e < g->rowptr[a + 1]; ++e) nn += !acc[g->colidx[e]];
        uint32_t wpick = rng_below(&rplant, nn), w = 0;
        for (uint32_t e = g->rowptr[a]; e < g->rowptr[a + 1]; ++e)
            if (!acc[g->colidx[e]] && wpick-- == 0) { w = g->colidx[e]; break; }
        int rc = mg_add_edges(g, 1, &w, &a);
        if (rc) goto fail_rc;
        g->info[0] = a;
        g->info[1] = w;
    }
    free(acc); free(deg); free(alist); free(nlist); free(aoff); free(noff);
    return MG_OK;
oom:
    free(acc); free(deg); free(alist); free(nlist); free(aoff); free(noff);
    mg_free(g);
    return MG_ERR_OOM;
arg:
    free(acc); free(deg); free(alist); free(nlist); free(aoff); free(noff);
    mg_free(g);
    return MG_ERR_ARG;
fail_rc:
    free(acc); free(deg); free(alist); free(nlist); free(aoff); free(noff);
    mg_free(g);
    return MG_ERR_OOM;
}

/* ------------------------------------------------ batch plans --- -- */

/*
 * Sizes log-uniform in [lo, hi]; exactly n_cycle of the `count` graphs (chosen
 * by a random permutation) get a planted accepting cycle; every graph gets its
 * own seed.
 */
int mg_batch_plan(uint32_t count, uint32_t lo, uint32_t hi, uint32_t n_cycle, uint64_t seed, uint32_t *sizes,
                  uint8_t *planted, uint64_t *seeds)
{
    if (count == 0 || lo < 2 || hi < lo || n_cycle > count) return MG_ERR_ARG;
    rng_t r;
    rng_seed(&r, seed, 21);
    double llo = log((double)lo), lhi = log((double)hi);
    for (uint32_t i = 0; i < count; ++i) {
        double x = exp(llo + rng_unit(&r) * (lhi - llo));
        uint32_t s = (uint32_t)(x + 0.5);
        sizes[i] = s < lo ? lo : (s > hi ? hi : s);
        seeds[i] = rng_u64(&r);
    }
    uint32_t *perm = (uint32_t *)malloc(sizeof(uint32_t) * count);
    if (!perm) return MG_ERR_OOM;
    for (uint32_t i = 0; i < count; ++i) perm[i] = i;
    for (uint32_t i = 0; i + 1 < count; ++i) {
        uint32_t j = i + rng_below(&r, count - i);
        uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    memset(planted, 0, count);
    for (uint32_t i = 0; i < n_cycle; ++i) planted[perm[i]] = 1;
    free(perm);
    return MG_OK;
}

/* ------------------------------------------- serving arrivals ----- -- */

/*
 * Poisson arrivals at `rate` jobs/s (exponential gaps), sizes lognormal with
 * the given median and sigma clipped to [lo, hi], half layered graphs
 * (kind 0) and half process products (kind 1).  For a product the (k, s) with
 * 2 * s^k closest to the drawn size and at most hi is chosen among
 * k in [4, 9], s in [5, 7]; size then holds 2 * s^k.  seeds[i] seeds job i.
 */
int mg_arrivals(uint32_t count, double rate, double median, double sigma, uint32_t lo, uint32_t hi, uint64_t seed,
                double *t_arrive, uint32_t *sizes, uint8_t *kind, uint8_t *pk, uint8_t *ps, uint64_t *seeds)
{
    if (count == 0 || rate <= 0 || median <= 0 || lo < 2 || hi < lo) return MG_ERR_ARG;
    rng_t r;
    rng_seed(&r, seed, 31);
    double t = 0.0;
    const double two_pi = 6.283185307179586;
    for (uint32_t i = 0; i < count; ++i) {
        double u = rng_unit(&r);
        t += -log(1.0 - u) / rate;
        t_arrive[i] = t;
        double u1 = rng_unit(&r), u2 = rng_unit(&r);
        double z = sqrt(-2.0 * log(1.0 - u1)) * cos(two_pi * u2);
        double x = median * exp(sigma * z);
        if (x < lo) x = lo;
        if (x > hi) x = hi;
        kind[i] = (uint8_t)(rng_u64(&r) & 1u);
        seeds[i] = rng_u64(&r);
        pk[i] = ps[i] = 0;
        if (kind[i] == 1) {
            double best = 1e300;
            uint32_t bk = 4, bs = 5;
            for (uint32_t kk = 4; kk <= 9; ++kk)
                for (uint32_t ss = 5; ss <= 7; ++ss) {
                    double sz = 2.0 * (double)ipow(ss, kk);
                    if (sz > hi) continue;
                    double d = fabs(log(sz) - log(x));
                    if (d < best) { best = d; bk = kk; bs = ss; }
                }
            pk[i] = (uint8_t)bk;
            ps[i] = (uint8_t)bs;
            sizes[i] = (uint32_t)(2 * ipow(bs, bk));
        } else {
            sizes[i] = (uint32_t)(x + 0.5);
        }
    }
    return MG_OK;
}
