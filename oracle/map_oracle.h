/*
 * map_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU statement of the MAP accepting-cycle
 * detection loop of the paper (Section 2, "DiVinE CUDA Algorithmics").  It
 * exists to check the GPU library; only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code with the GPU
 * path.
 *
 * Graph convention: row v of the CSR lists the successors of state v in the
 * state graph G.  MAP runs on the transposed graph (Section 2), in which the
 * predecessors of v are exactly the successors of v in G; so the maximal
 * accepting predecessor of v in the transposed graph is the largest accepting
 * u reachable from v in G by a path of at least one edge.
 */
#ifndef MAP_ORACLE_H
#define MAP_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_NONE 0xFFFFFFFFu /* "no value" in map vectors and the witness */

enum { ORACLE_OK = 0, ORACLE_ERR_ARG = 1, ORACLE_ERR_OOM = 2, ORACLE_LIMIT = 3 };
enum { ORACLE_NO_CYCLE = 0, ORACLE_CYCLE = 1 };

typedef struct {
    uint32_t verdict;     /* ORACLE_CYCLE or ORACLE_NO_CYCLE */
    uint32_t witness;     /* smallest v with map(v) = v, else ORACLE_NONE */
    uint32_t outer;       /* outer MAP iterations executed */
    uint32_t reserved;
    uint64_t inner_total; /* sum over outer iterations of synchronous rounds */
    uint64_t relaxations; /* edges examined (sum of row lengths relaxed) */
} oracle_result;

/* Called after the fix-point of every outer iteration, before elimination:
 * map[v] is the map value of v (ORACLE_NONE for none), rounds the number of
 * synchronous rounds that outer iteration took (including the final round in
 * which nothing changed). */
typedef void (*oracle_trace_fn)(void *user, uint32_t outer, const uint32_t *map, uint32_t n, uint32_t rounds);

/*
 * Run MAP to its verdict.
 *   n, rowptr[n+1], colidx[m]: successor CSR of G (validated here).
 *   acc[n]: accepting flags (nonzero = accepting).
 *   max_outer: stop with ORACLE_LIMIT after this many outer iterations (0 = none).
 *   trace/user: optional per-outer callback (may be NULL).
 *   rounds[rounds_cap]: per-outer round counts (entries past the cap are dropped).
 *   map_out[n]: the map vector of the last outer iteration (may be NULL);
 *     all ORACLE_NONE when no outer iteration ran (no accepting vertex).
 * Returns ORACLE_OK, ORACLE_LIMIT, ORACLE_ERR_ARG or ORACLE_ERR_OOM.
 */
int oracle_map(uint32_t n, const uint32_t *rowptr, const uint32_t *colidx, const uint8_t *acc, uint32_t max_outer,
               oracle_trace_fn trace, void *user, oracle_result *res, uint32_t *rounds, uint32_t rounds_cap,
               uint32_t *map_out);

#ifdef __cplusplus
}
#endif
#endif
