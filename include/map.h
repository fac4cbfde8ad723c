/*
 * map.h -- C ABI of the GB300 MAP accepting-cycle detection library (libmapgpu.so).
 *
 * MAP (Section 2 of Barnat, Brim, Ceska, "DiVinE-CUDA -- A Tool for GPU
 * Accelerated LTL Model Checking", PDMC 2009) decides whether a directed graph
 * with accepting vertices has a cycle through an accepting vertex.  It fixes an
 * order on the accepting vertices and computes, for every vertex, its maximal
 * accepting predecessor map(v) by propagating values to a fix-point; an
 * accepting vertex that is its own map value lies on an accepting cycle;
 * otherwise every map value is made non-accepting and the procedure restarts,
 * until a cycle is found or no accepting vertex is left.  The propagation is a
 * (max, id) sparse matrix-vector product over a CSR matrix (Section 2),
 * repeated to the fix-point.
 *
 * GRAPH CONVENTION.  The CSR handed in is the pull matrix of the transposed
 * graph on which MAP runs (Section 2): row v lists the successors of state v in
 * the state graph G, i.e. the predecessors of v in the transposed graph.  So
 *     map(v) = max { u accepting : v reaches u along rows by >= 1 edge }.
 * The order on accepting vertices is the vertex id; "no value" is below every
 * id and is reported as MAP_NONE.
 *
 * All entry points return a map_status code; nothing else crosses the ABI (no
 * exceptions, no aborts).  map_last_error() gives a message for the calling
 * host thread's last failure.  A map_graph is used by one host thread at a time.
 */
#ifndef MAPGPU_MAP_H
#define MAPGPU_MAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define MAP_API __attribute__((visibility("default")))
#else
#define MAP_API
#endif

#define MAP_NONE 0xFFFFFFFFu /* "no value" in map vectors; "no witness" */

typedef enum {
    MAP_OK = 0,
    MAP_ERR_ARG = 1,       /* bad argument (NULL handle, n out of range, ...) */
    MAP_ERR_CSR = 2,       /* invalid CSR: rowptr[0] != 0, decreasing rowptr, colidx >= n */
    MAP_ERR_OOM = 3,       /* device or host allocation failed */
    MAP_ERR_CUDA = 4,      /* a CUDA call failed; see map_last_error() */
    MAP_ERR_TIMEOUT = 5,   /* a bounded device-side wait gave up */
    MAP_ERR_LIMIT = 6,     /* max_outer / max_inner reached before the verdict */
    MAP_ERR_NOT_READY = 7, /* (serving) the job has not finished yet */
    MAP_ERR_BUSY = 8       /* (serving) no room for the job now */
} map_status;

enum { MAP_NO_CYCLE = 0, MAP_CYCLE = 1 };

/* Propagation schedule.
 *  MAP_SCHED_SYNC: synchronous rounds -- round k computes every value from the
 *    values of round k-1; round 1 relaxes every row, round k+1 the rows that
 *    read a vertex changed in round k.  Round counts and relaxation counts are
 *    canonical (identical to the CPU reference) and include the final round in
 *    which nothing changed.
 *  MAP_SCHED_ASYNC: in-place sweeps over the same frontiers; values written in
 *    a sweep may be read in the same sweep.  The fix-point (the least one, which
 *    is unique) and therefore every map vector, the verdict, the witness and the
 *    outer count are the same as under SYNC; the sweep count is at most the
 *    SYNC round count.  On a graph whose every row holds at most one entry (the
 *    state graph of a deterministic system; map_create detects it), a single
 *    graph's run with the dense start, without MAP_FLAG_PUSH / MAP_FLAG_PULL,
 *    propagates by pointer doubling instead: each pass takes, for every vertex,
 *    the value found at the end of its jump pointer along its chain of entries
 *    and doubles the pointer.  With D the largest distance from a vertex to
 *    its map value, an outer iteration then takes 2 + ceil(log2 D) rounds (the
 *    dense round and the passes; 1 if no vertex gets a value) instead of the
 *    1 + D synchronous rounds, and its sweep count is that round count. */
enum { MAP_SCHED_SYNC = 0, MAP_SCHED_ASYNC = 1 };

/* opts.flags */
#define MAP_FLAG_PROFILE 1u /* step the loop from the host and time each phase with CUDA events
                               (result.dense_ms, round_ms, check_ms, frontier_rows) */

#define MAP_FLAG_EARLY_EXIT 2u /* stop an outer iteration's propagation as soon as some vertex becomes its own
                                  map value: values only grow and each is a real accepting successor, so that
                                  vertex lies on an accepting cycle.  The verdict is the same; the witness is
                                  an accepting vertex on a cycle (not necessarily the smallest the full
                                  fix-point would give), the outer count may be smaller, and the round
                                  counts are no longer canonical.  Single graphs only. */

#define MAP_FLAG_FRONTIER_START 4u /* round 1 of every outer iteration without the dense round.  Round 1
                                  (Section 2: one product over the whole matrix from "no value" everywhere)
                                  gives row v the largest accepting vertex in it, so only the rows that hold
                                  a currently accepting vertex get a value.  With this flag each accepting
                                  vertex u pushes u to the rows that hold it (its readers) instead of every
                                  row being streamed; later rounds are unchanged.  Every map vector, the
                                  verdict, the witness, the outer count and, under MAP_SCHED_SYNC, the round
                                  and relaxation counts are the same as without it (relaxations stay the
                                  canonical counts of the pull schedule); under MAP_SCHED_ASYNC relaxations
                                  count the pushes actually made.  It pays when the accepting set is small
                                  against the edges.  In a batch, a graph that has finished keeps its
                                  last map vector as with the dense round.  Refused by map_run_static. */

#define MAP_FLAG_DENSE_START 8u /* the dense round, even on a handle that map_autotune set to the frontier
                                   start (without either flag a handle starts the way map_autotune chose,
                                   by default with the dense round).  Both start flags together: MAP_ERR_ARG. */

#define MAP_FLAG_PUSH 64u  /* every round after round 1 pushes from the vertices changed in the round before
                              to their readers (the reverse CSR); also keeps a graph whose rows hold one
                              entry at most on the rounds instead of pointer doubling */
#define MAP_FLAG_PULL 128u /* every round after round 1 pulls: each row takes the largest offer of the
                              vertices in it that changed in the round before (one pass over the whole
                              matrix, like the dense round).  Without either flag a round pulls when its
                              list holds at least a share of the vertices that map_autotune measures per
                              handle (by default none pulls).  Push and pull give the same values in every round,
                              and under MAP_SCHED_SYNC the same canonical round and relaxation counts.
                              Both flags together: MAP_ERR_ARG.  map_run_static always pushes. */

/* Called after the fix-point of every outer iteration, before the cycle test
 * and the elimination: map[v] is map(v) of that iteration (MAP_NONE if none),
 * host memory valid during the call only; rounds is that iteration's round
 * (or sweep) count.  Costs one device-to-host copy of n words per iteration. */
typedef void (*map_trace_fn)(void *user, uint32_t outer, const uint32_t *map, uint32_t n, uint32_t rounds);

typedef struct {
    uint32_t sched;       /* MAP_SCHED_SYNC (0, default) or MAP_SCHED_ASYNC */
    uint32_t max_outer;   /* stop with MAP_ERR_LIMIT after this many outer iterations; 0 = no limit */
    uint32_t max_inner;   /* per outer iteration; 0 = n + 1, which the synchronous schedule never exceeds */
    uint32_t flags;       /* MAP_FLAG_* */
    map_trace_fn trace;   /* optional, see above */
    void *user;           /* passed to trace */
    uint32_t *rounds_out; /* optional host array: round count of outer iteration i at [i] */
    uint32_t rounds_cap;  /* entries of rounds_out; later iterations are not stored */
    uint32_t timeout_ms;  /* the loop stops with MAP_ERR_TIMEOUT after this long; 0 = 120000 */
    uint32_t repeat;      /* map_run only: run the same MAP this many times back to back, queued on the
                             stream with no host step between them (0 or 1: once; for throughput
                             measurements).  res and map_out describe the last run (every run gives the
                             same), device_ms covers all of them.  Refused (MAP_ERR_ARG) with a trace,
                             MAP_FLAG_PROFILE, MAP_FLAG_EARLY_EXIT, max_outer or max_inner, by
                             map_submit and by map_run_static. */
    uint32_t reserved[2]; /* must be zero */
} map_opts;

typedef struct {
    uint32_t verdict;         /* MAP_CYCLE or MAP_NO_CYCLE */
    uint32_t witness;         /* smallest v with map(v) = v, or MAP_NONE */
    uint32_t outer_iters;     /* outer iterations executed (0 if no vertex is accepting) */
    uint32_t inner_canonical; /* 1 if inner_iters counts synchronous rounds (SYNC), 0 for ASYNC sweeps */
    uint64_t inner_iters;     /* rounds (or sweeps) summed over outer iterations */
    uint64_t relaxations;     /* edges examined.  SYNC (canonical): the row lengths of every
                                 round's frontier (round 1: all m); ASYNC: m per outer
                                 iteration plus one per push (batched ASYNC runs: frontier;
                                 pointer doubling: plus one per value taken along a chain) */
    uint64_t edges_total;     /* m x outer_iters: the edges a fix-point must examine at least once */
    double device_ms;         /* stream time of the whole run (CUDA events) */
    double dense_ms;          /* time of the dense rounds summed over the run: CUDA events around each
                                 launch with MAP_FLAG_PROFILE, else the kernels' own %globaltimer stamps
                                 (each phase runs from the end of the one before it) */
    uint32_t dense_launches;  /* dense-round launches */
    uint32_t accepting_left;  /* accepting vertices left at the end */
    uint64_t launches;        /* kernel launches issued by this run */
    double round_ms;          /* time of the fix-point rounds after the dense round (with the frontier
                                 start: all rounds), summed as dense_ms */
    double check_ms;          /* time of the self-map tests and eliminations, summed as dense_ms */
    uint64_t frontier_rows;   /* frontier rows summed over the rounds after the first (single-
                                 graph ASYNC runs: the vertices that pushed) */
    uint32_t status;          /* map_status of this graph's run (batched runs report one per graph) */
    uint32_t batch_jobs;      /* served jobs: how many jobs shared this job's run (1: it ran alone); else 0 */
    double queue_ms;          /* served jobs (map_poll): from map_submit until a worker took the job */
    double setup_ms;          /* served jobs: map_create (copy to the device, validation, readers) */
    double run_ms;            /* served jobs: the run until the map is back in host memory (host clock) */
} map_result;

typedef struct map_graph map_graph; /* opaque: the device-resident graph and its work space */

/*
 * map_create -- copy a graph to the device and prepare it for map_run.
 *   n        vertices, 1 <= n < 2^31 - 1 (bit 31 of a value word is reserved).
 *   rowptr   n + 1 entries (u32), rowptr[0] = 0, non-decreasing; m = rowptr[n].
 *   colidx   m entries (u32), each < n; may be NULL when m = 0.  Self-loops and
 *            duplicate entries are allowed.
 *   acc_bits ceil(n / 32) words: vertex v is accepting iff bit (v & 31) of word
 *            v >> 5 is set (LSB first); bits at or above n are ignored.
 *   cuda_stream  the cudaStream_t all work of this graph is issued on (NULL:
 *            the legacy default stream).
 * Every pointer may be host or device memory (told apart with
 * cudaPointerGetAttributes); the library copies them and the caller keeps
 * ownership.  Validation runs on the device; an invalid CSR returns
 * MAP_ERR_CSR and no handle.  On success *out owns about
 * 4*(2m + 6n) bytes of device memory until map_destroy.
 */
MAP_API int map_create(uint32_t n, const uint32_t *rowptr, const uint32_t *colidx, const uint32_t *acc_bits,
               void *cuda_stream, map_graph **out);

/*
 * map_run -- run MAP to its verdict (Section 2: propagate to the fix-point,
 * self-map test, eliminate, restart).
 *   opts     NULL for defaults (SYNC, no limits, no trace, the dense start
 *            unless map_autotune chose the frontier start for this handle).
 *   res      filled on MAP_OK and on MAP_ERR_LIMIT (with what was computed).
 *   map_out  optional, n entries, host or device memory: the map vector of the
 *            last outer iteration (all MAP_NONE when no vertex is accepting).
 * The graph is not changed: the accepting set is restored at every call, so
 * runs repeat exactly.  Blocks the calling thread until the result is known.
 * Without a trace or MAP_FLAG_PROFILE the whole run is one CUDA-graph launch
 * (its graph is built on the handle's first run with that schedule and start).
 */
MAP_API int map_run(map_graph *g, const map_opts *opts, map_result *res, uint32_t *map_out);

/* map_destroy -- free the graph's device memory. NULL is accepted. */
MAP_API int map_destroy(map_graph *g);

/*
 * Batched runs: many independent graphs solved together in one run.  The
 * graphs are joined into one disjoint union on the device (each graph's ids
 * are offset, which keeps its own order of accepting vertices), and one
 * CUDA-graph launch runs MAP on all of them at once: every outer iteration is
 * one outer iteration of each graph still running; a graph that has reached
 * its verdict is frozen (the dense round skips its rows, the frontier start
 * leaves its values alone).  Every graph gets exactly the result it gets alone.
 *
 * map_batch_create -- count >= 1 graphs; graph c has ns[c] vertices, rowptrs[c]
 *   (ns[c] + 1 entries), colidxs[c] (its own ids, < ns[c]), acc_bits[c] (as for
 *   map_create).  Host or device pointers; the library copies them.  The union
 *   must have < 2^31 - 1 vertices and < 2^32 edges.  Returns a handle for
 *   map_batch_run and map_destroy (map_run refuses it).
 */
MAP_API int map_batch_create(uint32_t count, const uint32_t *ns, const uint32_t *const *rowptrs,
                             const uint32_t *const *colidxs, const uint32_t *const *acc_bits, void *cuda_stream,
                             map_graph **out);

/*
 * map_batch_run -- run all graphs of a batch.
 *   results    count entries: graph c's result (witness in its own ids,
 *              status = its map_status); device_ms and launches are the batch's.
 *   map_out    optional, sum(ns) entries, host or device: the graphs' final map
 *              vectors one after another, each in its own ids (MAP_NONE = none).
 *   rounds_out optional host array of count * rounds_cap entries: round counts
 *              of graph c's outer iterations at [c * rounds_cap + i] (at most
 *              1024 per graph are kept).
 * opts as for map_run (no trace).  Returns MAP_OK, or the first non-OK status
 * of a graph (all results are filled in either case).
 */
MAP_API int map_batch_run(map_graph *g, const map_opts *opts, map_result *results, uint32_t *map_out,
                          uint32_t *rounds_out, uint32_t rounds_cap);

/*
 * Serving: verification jobs submitted over time and run with continuous
 * admission and batching.  The server has max_slots worker threads, each with
 * its own CUDA stream.  A job is copied at submission, into the server's pinned
 * staging memory (a quarter of hbm_budget_bytes, at most 2 GiB; pageable memory
 * when it is full, which only costs speed), and queued; the oldest queued job
 * is started as soon as a worker is free and its device footprint (about
 * 4 * (4m + 17n) bytes at its set-up's peak) fits into what is left of
 * hbm_budget_bytes (a job larger than the whole budget runs when nothing else
 * does).  When no other worker is waiting for work, queued jobs join its run,
 * as one batched run (see map_batch_create), oldest first, while they fit into
 * the budget and may share it: the same schedule, flags and timeout, no early
 * exit, limit or MAP_FLAG_PROFILE, and at most 2^20 vertices each (a batched
 * run lasts as long as its slowest graph, so larger jobs run alone); at most
 * 128 jobs (map_server_batch_limit) and 2^26 vertices per run.  Jobs that
 * cannot join keep their place in the queue.  Jobs that arrive while
 * others are running are admitted as slots and memory free up, and the
 * admitted jobs' work overlaps on the device.  Every job gets exactly the
 * result map_create + map_run give it (map_result.batch_jobs tells how many
 * jobs shared its run); a batch whose set-up or run fails is rerun job by job,
 * so an error is reported by the job that causes it only.
 *
 * map_server_create -- hbm_budget_bytes = 0: half of the free device memory.
 *   The calling thread's current device is used.
 * map_submit   -- host pointers only (copied); opts as for map_run, no trace.
 *   *job_id identifies the job.
 * map_poll     -- MAP_ERR_NOT_READY while the job is queued or running;
 *   otherwise the job's status, with res and (optional) map_out (n entries,
 *   host memory) filled, and the job and its staging memory are released (poll
 *   it once).
 * map_server_batch_limit -- at most max_jobs (1..1024) jobs share one run from
 *   now on (default 128; 1: every job runs alone).
 * map_server_destroy -- finishes the jobs already admitted and queued, then
 *   frees everything; unpolled results are discarded.
 * The server's calls may come from any host threads.  A job that fails (for
 * example MAP_ERR_OOM when its device memory cannot be had) reports its status
 * at map_poll and releases what it held; the other jobs are not affected.
 *
 * Fault injection for tests (host side, off by default): when the environment
 * variable MAPGPU_INJECT_OOM holds "job:k[,job:k...]" at map_server_create,
 * the k-th device allocation of map_create for the job with that id (ids count
 * from 1 in submission order) fails as if the device were out of memory.
 */
typedef struct map_server map_server; /* opaque */
MAP_API int map_server_create(size_t hbm_budget_bytes, uint32_t max_slots, map_server **out);
MAP_API int map_submit(map_server *sv, uint32_t n, const uint32_t *rowptr, const uint32_t *colidx,
                       const uint32_t *acc_bits, const map_opts *opts, uint64_t *job_id);
MAP_API int map_poll(map_server *sv, uint64_t job_id, map_result *res, uint32_t *map_out);
MAP_API int map_server_batch_limit(map_server *sv, uint32_t max_jobs);
MAP_API int map_server_destroy(map_server *sv);

/*
 * map_autotune -- pick how a handle (single graph or batch) runs, by measurement
 * on full runs of this very graph under schedule `sched`, timed with CUDA
 * events; every choice is kept for later runs of the handle and reported:
 *  1. from which list size a round pulls over the whole matrix instead of
 *     pushing through the readers: never, or from 1/256, 1/64, 1/32, 1/16, 1/8
 *     or 1/4 of the vertices (MAP_FLAG_PUSH / MAP_FLAG_PULL still force
 *     either);
 *  2. (MAP_SCHED_ASYNC, single graphs) how many times a block pushes again, in
 *     the same round, the vertices it raised itself (0, 1, 2, 4, 8, 16 or 32; by
 *     default 1), so that values travel several edges per round;
 *  3. up to which list size one block runs a round alone, with block barriers
 *     instead of the grid-wide one (never, 64, 256 or 1024 listed vertices;
 *     by default 256);
 *  4. the launch shapes: resident blocks per SM of the dense-round kernel and
 *     of the fix-point kernel (up to each kernel's occupancy limit), and the
 *     dense round's 16-byte loads in flight per lane (2, 4 or 8);
 *  5. the start of every outer iteration: the dense round or the frontier
 *     start (MAP_FLAG_DENSE_START / MAP_FLAG_FRONTIER_START still force either).
 * It takes about fifty runs (counted in `trials`); results are unaffected
 * (none of these choices changes any map vector, verdict, witness or outer
 * count, nor the counts of the synchronous schedule).
 *
 * The defaults of a new handle (before any map_autotune) can be set from the
 * environment, read by map_create and the other creating calls:
 * MAPGPU_PULL_FRAC (share of the vertices from which a round pulls; 0, the
 * default, = never), MAPGPU_SOLO_MAX (list size up to which one block runs a
 * round alone; 256), MAPGPU_LC_PASSES (block-local passes of asynchronous
 * rounds; 1), MAPGPU_ROUNDS_BLOCKS_PER_SM (resident blocks per SM of the
 * fix-point kernel, below its occupancy limit).
 */
typedef struct {
    uint32_t dense_blocks_per_sm;  /* chosen shape of the dense-round kernel */
    uint32_t rounds_blocks_per_sm; /* chosen shape of the fix-point kernel */
    double dense_ms;               /* its dense-round time per run at that shape */
    double rounds_ms;              /* its fix-point time per run at that shape */
    uint32_t trials;               /* runs made */
    uint32_t frontier_start;       /* 1: the handle now starts with the frontier start */
    double dense_start_ms;         /* run time with the dense start */
    double frontier_start_ms;      /* run time with the frontier start */
    double pull_share;             /* rounds over lists of at least this share of the vertices pull (0: never) */
    double pull_ms;                /* run time with that share (0: not timed) */
    double push_only_ms;           /* run time when no round pulls (0: not timed) */
    uint32_t solo_max;             /* rounds over at most this many listed vertices run in one block (0: never) */
    uint32_t dense_unroll;         /* the dense round's 16-byte loads in flight per lane */
    double solo_ms;                /* run time with that size (0: not timed) */
    uint32_t local_passes;         /* block-local passes per round of asynchronous runs */
    uint32_t reserved;
} map_tune_result;
MAP_API int map_autotune(map_graph *g, uint32_t sched, map_tune_result *out);

/*
 * map_lasso -- a counterexample for a cycle verdict (Section 5 of the paper
 * names counterexample generation as missing from the tool): a lasso that
 * leads from `init` to the accepting witness and around a cycle back to it,
 * found by breadth-first search along rows (successors in G) on the device.
 *   witness  an accepting vertex on a cycle (map_result.witness of a CYCLE run)
 *   init     start of the prefix, or MAP_NONE for the cycle alone
 *   path     host array of cap entries: the prefix init .. (before the witness),
 *            *prefix_len vertices, then the cycle witness .. witness,
 *            *cycle_len vertices (first == last); each step is an edge of G.
 *            Both parts are shortest.
 * Uses the handle's work space (not while a run is in flight on it).
 * MAP_ERR_ARG if the witness is not reachable as asked; MAP_ERR_LIMIT if the
 * path does not fit into cap entries.  Single graphs only.
 */
MAP_API int map_lasso(map_graph *g, uint32_t init, uint32_t witness, uint32_t *path, uint32_t cap,
                      uint32_t *prefix_len, uint32_t *cycle_len);

/*
 * map_create_reduced -- like map_create, over the part of the graph that can
 * hold an accepting cycle (Section 2 of the paper: the matrix lists only the
 * states of components that contain accepting states).
 *   part   NULL, or n component labels (host or device), e.g. the strongly
 *          connected component of the property automaton each product state
 *          projects to; only edges whose ends share a label are kept.  The
 *          caller guarantees that every cycle of the graph lies within one
 *          label (true for automaton components); NULL = one label.
 * Kept: every vertex reachable from an accepting vertex and reaching one (by
 * zero or more kept edges) -- every accepting cycle lies on such vertices, so
 * the verdict is that of the whole graph.  The handle holds the subgraph they
 * induce, renumbered in increasing order (the order on accepting vertices is
 * kept); map_run results (witness, map vector) use the new numbering, and
 * map_graph_vertex_ids gives the original id of each vertex.  With no
 * accepting vertex the handle holds one isolated non-accepting vertex whose
 * original id is MAP_NONE.  The reduction runs on the device; the full graph
 * lives on the device only while the call runs.
 */
MAP_API int map_create_reduced(uint32_t n, const uint32_t *rowptr, const uint32_t *colidx, const uint32_t *acc_bits,
                               const uint32_t *part, void *cuda_stream, map_graph **out);

/* map_graph_vertex_ids -- the original id of each of the graph's n vertices
 * into ids (host or device): the identity except for reduced graphs. */
MAP_API int map_graph_vertex_ids(const map_graph *g, uint32_t *ids);

/* map_graph_csr -- the graph as the handle holds it: rowptr (n + 1 entries),
 * colidx (m), acc_bits (ceil(n / 32) words, the accepting set at the start of
 * every run); each may be NULL, host or device.  Not while a run is in flight. */
MAP_API int map_graph_csr(const map_graph *g, uint32_t *rowptr, uint32_t *colidx, uint32_t *acc_bits);

/*
 * On-the-fly detection (Section 2 of the paper: one thread builds the matrix
 * while another repeatedly runs the detection on the part built so far, so a
 * cycle in that part is found before the state space is complete).
 * Vertices are numbered in the order they become known; their rows are
 * filled in the same order.  A row that is not yet filled is empty, so every
 * run sees a subgraph of the final graph: a cycle it reports is a cycle of
 * the final graph.
 *
 * map_grow_create -- n known vertices (accepting bits acc_bits, host or
 * device), none expanded yet.
 * map_append -- adds n_add vertices (n .. n + n_add - 1, bits acc_bits_add,
 * LSB-first from the first new vertex; host or device) and fills the rows of
 * the next k unexpanded vertices (rowptr_add: k + 1 offsets starting at 0;
 * colidx_add: rowptr_add[k] targets, each below the new vertex count).  The
 * resident graph stays on the device; only the chunk is copied from the
 * host.  On any error the handle is unchanged.  Also works on graphs from
 * map_create (all of their rows count as expanded).  Not for batched or
 * reduced graphs; not while a run is in flight on the handle.
 */
MAP_API int map_grow_create(uint32_t n, const uint32_t *acc_bits, void *cuda_stream, map_graph **out);
MAP_API int map_append(map_graph *g, uint32_t n_add, const uint32_t *acc_bits_add, uint32_t k,
                       const uint32_t *rowptr_add, const uint32_t *colidx_add);

/* map_graph_info -- n and m of a graph (either pointer may be NULL). */
MAP_API int map_graph_info(const map_graph *g, uint32_t *n, uint64_t *m);

/*
 * map_run_static -- one MAP run on a small graph without allocating anything.
 *
 * (The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory while they run -- plug-ins whose host
 * application owns the whole device budget and hands out none of it, and
 * real-time loops that must never enter an allocator.)
 *
 * Computes exactly what map_create + map_run + map_destroy compute on the same
 * arguments, with the same kernels, but every piece of work space lives in one
 * file-scope device array of MAP_STATIC_SCRATCH_BYTES (about 10.3 MiB) that
 * each GPU which loads this library holds until the process exits.  No
 * cudaMalloc, cudaFree, cudaMallocHost or other allocating call is made.
 *   n <= MAP_STATIC_MAX_N vertices and m = rowptr[n] <= MAP_STATIC_MAX_M edges;
 *   larger graphs are rejected with MAP_ERR_ARG and a message naming the limit.
 *   rowptr, colidx, acc_bits, map_out: as for map_create / map_run, host or
 *   device memory; the inputs are copied into the array on every call.
 *   opts: as for map_run (schedules, limits, timeout_ms, rounds_out for every
 *   outer iteration, MAP_FLAG_EARLY_EXIT, MAP_FLAG_DENSE_START), except that
 *   traces, MAP_FLAG_PROFILE, MAP_FLAG_FRONTIER_START and repeat are refused
 *   (MAP_ERR_ARG); res: as for map_run, status included (device_ms stays 0).
 *   cuda_stream: the stream all work is issued on.
 * The call blocks: it waits for cuda_stream several times (it reads rowptr[0]
 * and rowptr[n], then the control block after every step of the loop, into
 * host memory), so it must not be issued on a stream that is being captured
 * into a CUDA graph.  The first call on a device also looks the array's device
 * address up (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture begins in the process.  Every call on a
 * device shares the one array and overwrites what the previous call left
 * there, so calls that overlap on the GPU (from several host threads, or on
 * several streams) race and must be serialised by the caller.
 */
#define MAP_STATIC_MAX_N 65536u
#define MAP_STATIC_MAX_M 524288u
#define MAP_STATIC_SCRATCH_BYTES 10778368u
MAP_API int map_run_static(uint32_t n, const uint32_t *rowptr, const uint32_t *colidx, const uint32_t *acc_bits,
                           const map_opts *opts, map_result *res, uint32_t *map_out, void *cuda_stream);

/* map_last_error -- message of the calling thread's last failed call ("" if none). */
MAP_API const char *map_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
