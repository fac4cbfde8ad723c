/*
 * mapgen.h -- seeded synthetic workloads (graphs, batch plans, arrivals) for
 * MAP accepting-cycle detection.  Inputs only: no MAP arithmetic lives here.
 *
 * A graph is a CSR of SUCCESSOR lists of the state graph G (row v lists the
 * targets of v's out-edges) with one accepting flag byte per vertex.  Memory
 * of an mg_graph is malloc'd by the generator and released by mg_free().
 */
#ifndef MAPGEN_H
#define MAPGEN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { MG_OK = 0, MG_ERR_ARG = -1, MG_ERR_OOM = -2 };

typedef struct {
    uint32_t n;       /* vertices */
    uint64_t m;       /* edges = rowptr[n] */
    uint32_t *rowptr; /* n + 1 */
    uint32_t *colidx; /* m */
    uint8_t *acc;     /* n accepting flags (0/1) */
    uint32_t info[8]; /* generator-specific facts, see each generator */
} mg_graph;

void mg_free(mg_graph *g);
int mg_add_edges(mg_graph *g, uint32_t count, const uint32_t *src, const uint32_t *dst);
uint32_t mg_peel(uint32_t n, const uint32_t *rowptr, const uint32_t *colidx, uint8_t *peeled);

int mg_random(uint32_t n, uint32_t deg_lo, uint32_t deg_hi, uint32_t acc_ppm, uint64_t seed, int variant,
              uint32_t cycle_len, mg_graph *g);
int mg_product(uint32_t k, uint32_t s, int interleave, mg_graph *g);
int mg_layered(uint32_t n, uint32_t L, uint32_t D, uint32_t window, uint32_t acc_ppm, uint32_t fwd_ppm,
               uint32_t accfwd_ppm, uint64_t seed, int plant, mg_graph *g);
int mg_batch_plan(uint32_t count, uint32_t lo, uint32_t hi, uint32_t n_cycle, uint64_t seed, uint32_t *sizes,
                  uint8_t *planted, uint64_t *seeds);
int mg_arrivals(uint32_t count, double rate, double median, double sigma, uint32_t lo, uint32_t hi, uint64_t seed,
                double *t_arrive, uint32_t *sizes, uint8_t *kind, uint8_t *pk, uint8_t *ps, uint64_t *seeds);

#ifdef __cplusplus
}
#endif
#endif
