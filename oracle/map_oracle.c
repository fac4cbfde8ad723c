/*
 * map_oracle.c -- TEST INFRASTRUCTURE ONLY: the reference statement of MAP.
 *
 * A plain, slow, single-threaded CPU statement of the MAP accepting-cycle
 * detection loop described in Section 2 ("DiVinE CUDA Algorithmics") of
 * Barnat, Brim, Ceska, "DiVinE-CUDA -- A Tool for GPU Accelerated LTL Model
 * Checking" (PDMC 2009).  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load it; the GPU library never does, and the two share
 * no code.
 *
 * What it computes, in the paper's terms (Section 2):
 *   - an ordering is fixed on the accepting vertices; here it is the vertex id
 *     (larger id = larger), with "no value" below every id;
 *   - map(v), the maximal accepting predecessor of v in the transposed graph,
 *     is computed by value propagation: every vertex keeps the largest value
 *     propagated into it, values travel along edges, and the propagation stops
 *     at the fix-point where no value can be improved;
 *   - an accepting vertex that is its own map value lies on an accepting
 *     cycle: stop with a cycle;
 *   - otherwise every accepting vertex that is the map value of some vertex is
 *     made non-accepting, and the procedure restarts;
 *   - it ends when a cycle is found or no accepting vertex is left.
 *
 * Graph convention.  Row v of the CSR lists the successors of state v in the
 * state graph G.  MAP runs on the transposed graph (Section 2), in which the
 * predecessors of v are exactly these successors; so a value "propagated into"
 * v comes from the vertices of row v, and at the fix-point
 *     map(v) = max { u accepting : v reaches u in G by a path of >= 1 edge }.
 *
 * Readings of points the paper leaves open (each is also listed in the
 * project's design notes):
 *   - propagation is synchronous (Jacobi): round k computes every value from
 *     the values of round k-1.  Round 1 relaxes every row; round k+1 relaxes
 *     only the rows that read a vertex whose value changed in round k (the
 *     other rows would compute the same value again).  The round count of an
 *     outer iteration includes the final round in which nothing changed;
 *   - the value offered by u along an edge is max(u if u is accepting, map(u));
 *   - "maximal accepting predecessor" is proper (paths of at least one edge);
 *   - map is reset to "no value" at every restart;
 *   - the self-map test comes before the elimination; the witness is the
 *     smallest v with map(v) = v;
 *   - the eliminated set is { map(v) : v any vertex, map(v) defined };
 *   - when that set is empty while accepting vertices remain, no remaining
 *     accepting vertex is reachable from any vertex, so none is on a cycle:
 *     stop with "no cycle", counting that iteration.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "map_oracle.h"

#define NONE (-1) /* "no value": below every vertex id */

int oracle_map(uint32_t n, const uint32_t *rowptr, const uint32_t *colidx, const uint8_t *acc, uint32_t max_outer,
               oracle_trace_fn trace, void *user, oracle_result *res, uint32_t *rounds, uint32_t rounds_cap,
               uint32_t *map_out)
{
    if (!res || n == 0 || n >= 0x7FFFFFFFu || !rowptr || !acc) return ORACLE_ERR_ARG;
    memset(res, 0, sizeof(*res));
    res->verdict = ORACLE_NO_CYCLE;
    res->witness = ORACLE_NONE;

    /* validate the CSR */
    if (rowptr[0] != 0) return ORACLE_ERR_ARG;
    for (uint32_t v = 0; v < n; ++v)
        if (rowptr[v + 1] < rowptr[v]) return ORACLE_ERR_ARG;
    uint32_t m = rowptr[n];
    if (m > 0 && !colidx) return ORACLE_ERR_ARG;
    for (uint32_t e = 0; e < m; ++e)
        if (colidx[e] >= n) return ORACLE_ERR_ARG;

    int rc = ORACLE_OK;
    uint8_t *A = malloc(n);                 /* current accepting set */
    int64_t *map = malloc(sizeof(int64_t) * n);
    uint32_t *rdeg = calloc((size_t)n + 1, sizeof(uint32_t)); /* readers: reverse adjacency */
    uint32_t *readers = malloc(sizeof(uint32_t) * (m ? m : 1));
    uint32_t *frontier = malloc(sizeof(uint32_t) * n);
    uint32_t *next = malloc(sizeof(uint32_t) * n);
    uint8_t *queued = calloc(n, 1);
    uint32_t *chg_v = malloc(sizeof(uint32_t) * n);  /* vertices changed this round */
    int64_t *chg_val = malloc(sizeof(int64_t) * n);   /* and their new values */
    uint8_t *elim = calloc(n, 1);
    if (!A || !map || !rdeg || !readers || !frontier || !next || !queued || !chg_v || !chg_val || !elim) {
        rc = ORACLE_ERR_OOM;
        goto done;
    }

    /* reverse adjacency: readers of u are the w whose row contains u */
    for (uint32_t e = 0; e < m; ++e) rdeg[colidx[e] + 1]++;
    for (uint32_t u = 0; u < n; ++u) rdeg[u + 1] += rdeg[u];
    {
        uint32_t *fill = malloc(sizeof(uint32_t) * n);
        if (!fill) {
            rc = ORACLE_ERR_OOM;
            goto done;
        }
        memcpy(fill, rdeg, sizeof(uint32_t) * n);
        for (uint32_t w = 0; w < n; ++w)
            for (uint32_t e = rowptr[w]; e < rowptr[w + 1]; ++e) readers[fill[colidx[e]]++] = w;
        free(fill);
    }

    uint32_t nacc = 0;
    for (uint32_t v = 0; v < n; ++v) {
        A[v] = acc[v] ? 1 : 0;
        nacc += A[v];
        map[v] = NONE;
    }

    uint32_t outer = 0;
    while (nacc > 0) {
        if (max_outer && outer >= max_outer) {
            rc = ORACLE_LIMIT;
            break;
        }
        outer += 1;

        /* restart: every vertex has no value; the first round relaxes every row */
        for (uint32_t v = 0; v < n; ++v) map[v] = NONE;
        uint32_t nf = n;
        for (uint32_t v = 0; v < n; ++v) frontier[v] = v;
        uint32_t k = 0;
        for (;;) {
            k += 1;
            /* one synchronous round: new values are computed from the old ones
             * and only applied once the whole round has been computed */
            uint32_t nc = 0;
            for (uint32_t i = 0; i < nf; ++i) {
                uint32_t v = frontier[i];
                int64_t best = map[v];
                for (uint32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
                    uint32_t u = colidx[e];
                    int64_t offered = map[u];
                    if (A[u] && (int64_t)u > offered) offered = (int64_t)u;
                    if (offered > best) best = offered;
                }
                res->relaxations += rowptr[v + 1] - rowptr[v];
                if (best != map[v]) {
                    chg_v[nc] = v;
                    chg_val[nc] = best;
                    nc++;
                }
            }
            for (uint32_t i = 0; i < nc; ++i) map[chg_v[i]] = chg_val[i];
            if (nc == 0) break; /* fix-point: no value can be improved */
            /* next round: the rows that read a changed vertex */
            uint32_t nn = 0;
            for (uint32_t i = 0; i < nc; ++i) {
                uint32_t u = chg_v[i];
                for (uint32_t e = rdeg[u]; e < rdeg[u + 1]; ++e) {
                    uint32_t w = readers[e];
                    if (!queued[w]) {
                        queued[w] = 1;
                        next[nn++] = w;
                    }
                }
            }
            for (uint32_t i = 0; i < nn; ++i) queued[next[i]] = 0;
            memcpy(frontier, next, sizeof(uint32_t) * nn);
            nf = nn;
        }
        if (outer - 1 < rounds_cap && rounds) rounds[outer - 1] = k;
        res->inner_total += k;
        res->outer = outer;

        if (trace) {
            /* hand out the map vector in the external encoding */
            uint32_t *ext = malloc(sizeof(uint32_t) * n);
            if (!ext) {
                rc = ORACLE_ERR_OOM;
                break;
            }
            for (uint32_t v = 0; v < n; ++v) ext[v] = map[v] == NONE ? ORACLE_NONE : (uint32_t)map[v];
            trace(user, outer, ext, n, k);
            free(ext);
        }

        /* self-map test: an accepting vertex that is its own map value */
        uint32_t witness = ORACLE_NONE;
        for (uint32_t v = 0; v < n; ++v)
            if (map[v] == (int64_t)v) {
                witness = v;
                break;
            }
        if (witness != ORACLE_NONE) {
            res->verdict = ORACLE_CYCLE;
            res->witness = witness;
            break;
        }

        /* elimination: every map value stops being accepting */
        uint32_t ne = 0;
        memset(elim, 0, n);
        for (uint32_t v = 0; v < n; ++v)
            if (map[v] != NONE && !elim[map[v]]) {
                elim[map[v]] = 1;
                ne++;
            }
        if (ne == 0) break; /* nothing reaches a remaining accepting vertex */
        for (uint32_t u = 0; u < n; ++u)
            if (elim[u] && A[u]) {
                A[u] = 0;
                nacc--;
            }
    }

    if (map_out)
        for (uint32_t v = 0; v < n; ++v) map_out[v] = map[v] == NONE ? ORACLE_NONE : (uint32_t)map[v];

done:
    free(A);
    free(map);
    free(rdeg);
    free(readers);
    free(frontier);
    free(next);
    free(queued);
    free(chg_v);
    free(chg_val);
    free(elim);
    return rc;
}
