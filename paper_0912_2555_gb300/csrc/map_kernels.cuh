// map_kernels.cuh -- sm_103a kernels of the MAP hot path (Section 2 of the paper).
//
// Device layout of one graph (all u32 unless noted):
//   rowptr[n+1], colidx[m]   the CSR handed in: row v = successors of v in G, i.e.
//                            the pull matrix of the transposed graph.  The
//                            library's copy of colidx carries the accepting flag
//                            of each target in bit 31 (ids are < 2^31 - 1), so the
//                            dense round streams the matrix without gathers;
//   rrowptr[n+1], rcol[m]    its transpose: rcol[rrowptr[u] ..] are the readers
//                            of u (the rows that contain u), and rpos[..] the
//                            positions in colidx of those entries (to update the
//                            flag of u when u is eliminated);
//   elog[n]                  vertices eliminated in this run (their flags are
//                            restored at the end of the run);
//   acc[W], W = ceil(n/32)   the current accepting set, LSB-first bitmap;
//   mval[n]                  enc(map(v)): 0 = no value, u + 1 = vertex u;
//   list[3][n]               vertices whose value changed in a round, by round mod 3;
//   flist[3][n]              the frontier of a round (rows reading a vertex that
//                            changed in the round before), for the relaxation count;
//   rec[n] (16 bytes)        per-vertex round state, in one sector so that a push
//                            touches two sectors (mval and rec): snap[0..2], the
//                            value a listed vertex ended its round with
//                            (synchronous rounds), and flags: CB(p) = "in list[p]",
//                            FB(p) = "in flist[p]";
//   touched[n]               vertices that got a value in this outer iteration;
//   alist[|A0|]              the initially accepting vertices (frontier start only);
//   Ctl                      the control block below (one per graph).
//
// One outer iteration: the dense round (every row, k_dense), then push rounds
// until a round changes nothing (k_rounds, one persistent cooperative launch
// with a grid barrier between rounds), then the self-map test and the
// elimination over the touched vertices (check_phase: the tail of k_rounds when
// the loop runs as a CUDA graph, the kernel k_check when it is stepped from the
// host).  With the frontier start there is no dense round: k_rounds resets the
// previous iteration's values and pushes round 1 from the accepting vertices.
// Every kernel that ends a step of the loop finishes with a last-block epilogue
// (the last block to retire, found with an atomic ticket) that updates the
// control block and, when the loop runs as a CUDA graph, sets the graph's
// conditional WHILE handles.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace mapk {

namespace cg = cooperative_groups;

constexpr uint32_t NONE = 0xFFFFFFFFu;
constexpr uint32_t CH_CAP = 1024; // rounds recorded per graph in a batched run
constexpr uint32_t ST_OK = 0, ST_TIMEOUT = 5, ST_LIMIT = 6; // map_status values used on the device

// Counters that many blocks update atomically each get a 128-byte line of their
// own: atomics on one line are serialised, so sharing a line would make every
// kernel wait on the others' updates.
struct alignas(128) Cnt32 {
    uint32_t v;
};
struct alignas(128) Cnt64 {
    uint64_t v;
};

struct Ctl {
    // hot counters
    Cnt32 lcnt[3];         // |list| by round mod 3
    Cnt32 fcnt[3];         // |flist| by round mod 3
    Cnt32 tcnt;            // |touched|
    Cnt32 done;            // last-block ticket
    Cnt32 elim;            // accepting vertices eliminated in this outer iteration
    Cnt32 witness;         // smallest self-mapped vertex of the last iteration
    Cnt32 ecnt;            // |elog|
    Cnt64 relax;           // edges examined (canonical count of the synchronous schedule)
    Cnt64 frontier_rows;   // frontier rows summed over the push rounds
    Cnt32 bar_count;       // grid barrier of k_rounds: arrivals
    Cnt32 bar_gen;         // ... and generation
    Cnt32 stop_req;        // k_rounds: block 0 asks every block to stop after the next barrier
    Cnt32 self_seen;       // smallest vertex seen to become its own map value (NONE: none yet)
    Cnt32 solo_gen;        // k_rounds: hand-backs of block 0 after rounds it ran alone (0 at every launch)
    Cnt32 solo_beat;       // ... and its progress in them (rounds and pushes; the waiting blocks' heartbeat)
    // fix-point loop
    uint32_t k;            // rounds completed in the current outer iteration
    // outer loop
    uint32_t outer;        // current outer iteration, 1-based (0: none ran)
    uint32_t outer_go;     // outer loop continues
    uint32_t status;       // ST_OK, ST_LIMIT or ST_TIMEOUT
    uint32_t verdict;      // 1 = accepting cycle
    uint32_t nacc;         // accepting vertices left
    uint32_t nacc0;        // accepting vertices at the start
    uint32_t max_outer;    // 0 = no limit
    uint32_t max_inner;    // rounds per outer iteration
    uint32_t hist_cap;     // entries of rounds_hist
    uint32_t bad;          // set-up: validation failure
    uint64_t m;            // edges
    uint64_t inner_total;  // rounds summed over outer iterations
    uint32_t *rounds_hist; // rounds of each outer iteration
    uint32_t *out;         // map export destination (device)
    uint64_t t0;           // %globaltimer at the start of the run (ns)
    uint64_t timeout_ns;   // the loop stops with ST_TIMEOUT past t0 + timeout_ns
    uint32_t use_graph;    // epilogues set the conditional handles
    uint32_t early_exit;   // stop the fix-point loop at the first self-mapped vertex
    uint32_t early_hit;    // it did (the run's round state is then left dirty)
    uint32_t tprev;        // |touched| of the previous outer iteration (frontier start resets their values)
    uint32_t pull_min;     // a round whose list holds at least this many vertices pulls (0: never)
    uint32_t solo_max;     // a round over at most this many listed vertices (and at most solo_fmax
    uint32_t solo_fmax;    //   frontier rows to clear) runs in block 0 alone (0: never)
    uint32_t solo_r, solo_nl, solo_nf, solo_status; // block 0's state when it hands back
    uint32_t lc_passes;    // asynchronous single graphs: block-local passes per round
    uint32_t gave_up;      // a bounded device wait gave up (ST_TIMEOUT): 1 = grid barrier, 2 = the
                           //   hand-back of one-block rounds; 0 = none (the time limit, if any)
    uint32_t long_rows;    // set-up: some row holds two entries or more (else: pointer doubling applies)
    // %globaltimer stamps of the phases (ns), summed over the run: the end of the last phase
    // (t_mark), the dense rounds, the fix-point rounds, the self-map tests and eliminations.  Each
    // phase runs from the end of the one before it, so gaps between launches count to the next.
    uint64_t t_mark, ph_dense, ph_rounds, ph_check;
};

struct Handles {
    unsigned long long outer; // cudaGraphConditionalHandle of the outer WHILE node
};

// device pointers of one graph, passed by value to the loop kernels
// Batched runs: several graphs as one disjoint union (ids offset per graph,
// which keeps each graph's order), one state record per graph.  A graph whose
// run has ended is frozen: the dense round skips its rows, so its last map
// vector stays in place, and nothing else touches it.
struct CompState {
    uint32_t active;      // still running
    uint32_t outer;       // its outer iterations so far (current one, 1-based)
    uint32_t verdict;     // 1 = accepting cycle
    uint32_t witness;     // smallest self-mapped vertex (union id) of the current iteration
    uint32_t nacc;        // accepting vertices left
    uint32_t nacc0;       // accepting vertices at the start
    uint32_t elim;        // eliminated in the current iteration
    uint32_t touched;     // vertices with a value in the current iteration
    uint32_t last_change; // last round of the current iteration in which one of its values changed
    uint32_t status;      // ST_OK, ST_LIMIT or ST_TIMEOUT
    uint32_t off;         // its first vertex in the union
    uint32_t pad0;
    uint64_t m;           // its edges
    uint64_t relax;       // its edges examined (canonical count)
    uint64_t inner_total; // its rounds, summed
    uint64_t pad1;
};

struct Dev {
    uint32_t n, words;
    // batched runs only (comp == NULL for a single graph)
    const uint32_t *comp; // graph of each union vertex
    CompState *cs;        // one record per graph
    uint32_t *chist;      // rounds per outer iteration, CH_CAP entries per graph
    uint32_t ncomp;
    const uint32_t *rowptr, *colidx, *rrowptr, *rcol, *rpos;
    uint32_t *colidx_w; // the same array as colidx, for the flag updates
    uint32_t *acc, *mval;
    uint32_t *elog;
    uint32_t *list[3], *flist[3];
    uint4 *rec; // .x / .y / .z: snap[0..2]; .w: flags
    uint32_t *cbit[3]; // pull rounds: bit u of cbit[p] = u is in list[p] (set for a pull round, cleared in the next)
    uint32_t *touched;
    uint32_t *stale; // single graphs: bit v = mval[v] holds a value of an earlier outer iteration (NULL: batched)
    Ctl *ctl;
    // frontier start (single graphs): the initially accepting vertices; round 1 is pushed from
    // those still accepting instead of the dense round (NULL: the dense round runs)
    const uint32_t *alist;
    uint32_t na;
};

__device__ __forceinline__ uint32_t CB(uint32_t p) { return 1u << p; } // in list[p]
__device__ __forceinline__ uint32_t FB(uint32_t p) { return 8u << p; } // in flist[p]
__device__ __forceinline__ uint32_t *rec_snap(uint4 *r, uint32_t p) { return p == 0 ? &r->x : p == 1 ? &r->y : &r->z; }
__device__ __forceinline__ uint32_t *rec_flags(uint4 *r) { return &r->w; }
// a parity-indexed pointer picked with selects (a dynamic index into the
// parameter struct would move it to local memory)
__device__ __forceinline__ uint32_t *pick3(uint32_t p, uint32_t *const (&a)[3])
{
    return p == 0 ? a[0] : p == 1 ? a[1] : a[2];
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// asynchronous global -> shared copies (cp.async): 16 bytes (src_bytes < 16: the rest is
// zero-filled), 4 bytes; a commit closes a group, wait<N> leaves at most N groups in flight
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, uint32_t src_bytes)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ bool acc_bit(const uint32_t *__restrict__ acc, uint32_t u)
{
    return (__ldg(acc + (u >> 5)) >> (u & 31u)) & 1u;
}

// warp-aggregated increment: one atomic per converged set of lanes
__device__ __forceinline__ unsigned agg_inc(unsigned int *ctr)
{
    cg::coalesced_group g = cg::coalesced_threads();
    unsigned base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(ctr, (unsigned)g.size());
    return g.shfl(base, 0) + g.thread_rank();
}

// set bit v of a bitmap; true for the one caller that flipped it from 0 to 1
__device__ __forceinline__ bool test_and_set(uint32_t *bits, uint32_t v)
{
    const uint32_t bit = 1u << (v & 31u);
    if (*(volatile uint32_t *)(bits + (v >> 5)) & bit) return false; // read first: most calls stop here
    return !(atomicOr(bits + (v >> 5), bit) & bit);
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long x)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, off);
    return x;
}

// Block-wide sum (or min) of per-thread values, applied to a global counter with
// one atomic per block.  Every thread of the block calls these (__syncthreads); the barrier on
// entry keeps a call from overwriting the partial sums a previous call is still reading.
__device__ __forceinline__ void block_add_u64(unsigned long long x, unsigned long long *dst)
{
    __shared__ unsigned long long part[32];
    __syncthreads();
    x = warp_sum64(x);
    if (lane_id() == 0) part[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (unsigned w = 0; w < (blockDim.x >> 5); ++w) t += part[w];
        if (t) atomicAdd(dst, t);
    }
}

__device__ __forceinline__ void block_add_min_u32(uint32_t add, uint32_t mn, uint32_t *dst_add, uint32_t *dst_min)
{
    __shared__ uint32_t part_add[32], part_min[32];
    __syncthreads();
    add = __reduce_add_sync(0xFFFFFFFFu, add);
    mn = __reduce_min_sync(0xFFFFFFFFu, mn);
    if (lane_id() == 0) {
        part_add[threadIdx.x >> 5] = add;
        part_min[threadIdx.x >> 5] = mn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t a = 0, m = 0xFFFFFFFFu;
        for (unsigned w = 0; w < (blockDim.x >> 5); ++w) {
            a += part_add[w];
            m = min(m, part_min[w]);
        }
        if (a) atomicAdd(dst_add, a);
        if (m != 0xFFFFFFFFu) atomicMin(dst_min, m);
    }
}

// ---- append staging -------------------------------------------------------
//
// Kernels append vertex ids to global lists.  Instead of one atomic on the
// list's counter per append (or per warp and append step), each warp stages its
// appends in shared memory and the block reserves global space once per list
// when it finishes (a warp whose buffer fills up flushes it on its own).
constexpr int SB_ENTRIES = 128; // staged entries per warp and list

template <int NL>
struct Stage {
    uint32_t *buf;   // this warp's NL x SB_ENTRIES shared buffer
    uint32_t cnt[NL]; // warp-uniform fill counts
};

// append w to list l where flag holds; every lane of the warp calls it.
// dst[l][0..1]: global arrays the entry goes to (dst[l][1] may be NULL), ctr[l]: their counter.
template <int NL>
__device__ __forceinline__ void stage_append(Stage<NL> &st, int l, bool flag, uint32_t w, uint32_t *const (*dst)[2],
                                             unsigned int *const *ctr)
{
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, flag);
    if (!mask) return;
    const unsigned lane = lane_id();
    uint32_t *b = st.buf + l * SB_ENTRIES;
    if (st.cnt[l] + 32 > (uint32_t)SB_ENTRIES) { // full: this warp flushes on its own
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(ctr[l], st.cnt[l]);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        __syncwarp();
        for (uint32_t i = lane; i < st.cnt[l]; i += 32) {
            dst[l][0][base + i] = b[i];
            if (dst[l][1]) dst[l][1][base + i] = b[i];
        }
        __syncwarp();
        st.cnt[l] = 0;
    }
    if (flag) b[st.cnt[l] + __popc(mask & ((1u << lane) - 1u))] = w;
    st.cnt[l] += __popc(mask);
    __syncwarp();
}

// end of a kernel: every thread of the block calls it (it contains __syncthreads);
// one global atomic per list and block.  s_cnt: shared [warps][NL], s_base: shared [NL].
template <int NL>
__device__ __forceinline__ void stage_flush_block(Stage<NL> &st, uint32_t (*s_cnt)[NL], uint32_t *s_base,
                                                  uint32_t *const (*dst)[2], unsigned int *const *ctr)
{
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int l = 0; l < NL; ++l) s_cnt[warp][l] = st.cnt[l];
    }
    __syncthreads();
    if (threadIdx.x < (unsigned)NL) {
        uint32_t tot = 0;
        for (unsigned w = 0; w < nwarps; ++w) tot += s_cnt[w][threadIdx.x];
        s_base[threadIdx.x] = tot ? atomicAdd(ctr[threadIdx.x], tot) : 0;
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        uint32_t off = s_base[l];
        for (unsigned w = 0; w < warp; ++w) off += s_cnt[w][l];
        const uint32_t *b = st.buf + l * SB_ENTRIES;
        for (uint32_t i = lane; i < st.cnt[l]; i += 32) {
            dst[l][0][off + i] = b[i];
            if (dst[l][1]) dst[l][1][off + i] = b[i];
        }
    }
}

// True in exactly one thread of the grid: thread 0 of the last block to get here.
// Every thread of every block must call it (it contains __syncthreads).
__device__ __forceinline__ bool last_block(Ctl *ctl)
{
    __shared__ bool is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(&ctl->done.v, 1u);
        is_last = (t == gridDim.x - 1);
        if (is_last) {
            ctl->done.v = 0;
            __threadfence();
        }
    }
    __syncthreads();
    return is_last && threadIdx.x == 0;
}

__device__ __forceinline__ void set_cond(const Ctl *c, unsigned long long h, unsigned v)
{
    if (*(volatile const uint32_t *)&c->use_graph) cudaGraphSetConditional(h, v);
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// A WHILE body's first kernel sets its condition to "stop"; only the body's
// epilogue sets it back to "continue".  A body whose epilogue does not run
// therefore ends its loop.
__device__ __forceinline__ void default_stop(const Ctl *c, unsigned long long h)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(c, h, 0);
}

// (differences of %globaltimer readings are taken signed: a reading on another SM may lag the
// one that set t0 by a little, and that must not wrap to a huge elapsed time)
__device__ __forceinline__ bool timed_out(volatile Ctl *v)
{
    return (int64_t)(global_ns() - v->t0) > (int64_t)v->timeout_ns;
}

// After round 1 (the dense round) of an outer iteration: list[1] holds the
// vertices that got a value, which are also the touched vertices so far.
// the time since the last phase ended goes to *acc; this phase ends now
__device__ __forceinline__ void phase_end(volatile Ctl *v, volatile uint64_t *acc)
{
    const uint64_t now = global_ns();
    const int64_t d = (int64_t)(now - v->t_mark);
    if (d > 0) { // (a lagging reading adds nothing and does not move the mark back)
        *acc = *acc + (uint64_t)d;
        v->t_mark = now;
    }
}

__device__ void epilogue_dense(Ctl *c)
{
    volatile Ctl *v = c;
    phase_end(v, &v->ph_dense);
    v->tcnt.v = v->lcnt[1].v;
    v->k = 1;
    v->relax.v = v->relax.v + v->m;
    __threadfence();
}

// After the self-map test and the elimination of an outer iteration.
__device__ void epilogue_check(Ctl *c, Handles hd)
{
    volatile Ctl *v = c;
    phase_end(v, &v->ph_check);
    const uint32_t outer = v->outer, k = v->k;
    if (outer - 1 < v->hist_cap) c->rounds_hist[outer - 1] = k;
    v->inner_total = v->inner_total + k;
    uint32_t go = 1;
    // early exit: a vertex that received its own value lies on an accepting cycle, even if a
    // later push of the same round raised it past that value (values only grow)
    if (v->early_exit && v->self_seen.v < v->witness.v) v->witness.v = v->self_seen.v;
    if (v->status != ST_OK) {
        go = 0; // a limit was hit inside the fix-point loop
    } else if (v->witness.v != NONE) {
        v->verdict = 1;
        go = 0;
    } else if (v->tcnt.v == 0) {
        go = 0; // no map value is defined: nothing reaches a remaining accepting vertex
    } else {
        const uint32_t left = v->nacc - v->elim.v;
        v->nacc = left;
        if (left == 0) {
            go = 0;
        } else if ((v->max_outer && outer >= v->max_outer) || outer > v->nacc0) {
            // (every non-final iteration removes an accepting vertex, so more
            // than nacc0 iterations cannot happen; the second test is a guard)
            v->status = ST_LIMIT;
            go = 0;
        } else if (timed_out(v)) {
            v->status = ST_TIMEOUT;
            go = 0;
        }
    }
    // every block of the fix-point launch has left its rounds: the next launch counts block 0's
    // hand-backs from 0 (a block that starts late must not take a hand-back already made in
    // its own launch as its starting point)
    v->solo_gen.v = 0;
    if (go) {
        v->outer = outer + 1;
        v->lcnt[0].v = v->lcnt[1].v = v->lcnt[2].v = 0;
        v->fcnt[0].v = v->fcnt[1].v = v->fcnt[2].v = 0;
        v->tprev = v->tcnt.v;
        v->tcnt.v = 0;
        v->elim.v = 0;
        v->k = 0;
    }
    v->outer_go = go;
    __threadfence();
    set_cond(c, hd.outer, go);
}

// True in every thread of the last block to get here (see last_block).
__device__ __forceinline__ bool last_block_all(Ctl *ctl)
{
    __shared__ bool is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(&ctl->done.v, 1u);
        is_last = (t == gridDim.x - 1);
        if (is_last) {
            ctl->done.v = 0;
            __threadfence();
        }
    }
    __syncthreads();
    return is_last;
}

// Batched runs, after the self-map test and the elimination (Section 2, per
// graph): every thread of the last block takes a share of the graphs.
__device__ void epilogue_batch(const Dev &d, Handles hd)
{
    __shared__ uint32_t s_any, s_gst;
    volatile Ctl *v = d.ctl;
    if (threadIdx.x == 0) {
        phase_end(v, &v->ph_check);
        v->solo_gen.v = 0; // (as in epilogue_check: the next fix-point launch counts hand-backs from 0)
        uint32_t gst = v->status; // a limit or timeout inside the fix-point loop
        if (gst == ST_OK && timed_out(v)) gst = ST_TIMEOUT;
        s_gst = gst;
        s_any = 0;
    }
    __syncthreads();
    const uint32_t gst = s_gst, max_outer = v->max_outer;
    for (uint32_t c = threadIdx.x; c < d.ncomp; c += blockDim.x) {
        volatile CompState &S = d.cs[c];
        if (!S.active) continue;
        const uint32_t outer = S.outer, rounds = S.last_change + 1;
        if (outer - 1 < CH_CAP) d.chist[(size_t)c * CH_CAP + outer - 1] = rounds;
        S.inner_total = S.inner_total + rounds;
        S.relax = S.relax + S.m; // its dense round
        bool go = true;
        if (gst != ST_OK) {
            S.status = gst;
            go = false;
        } else if (S.witness != NONE) {
            S.verdict = 1;
            go = false;
        } else if (S.touched == 0) {
            go = false; // no map value: nothing reaches a remaining accepting vertex
        } else {
            const uint32_t left = S.nacc - S.elim;
            S.nacc = left;
            if (left == 0) {
                go = false;
            } else if ((max_outer && outer >= max_outer) || outer > S.nacc0) {
                S.status = ST_LIMIT;
                go = false;
            }
        }
        if (go) {
            S.outer = outer + 1;
            S.witness = NONE;
            S.elim = 0;
            S.touched = 0;
            S.last_change = 0;
            atomicOr(&s_any, 1u);
        } else {
            S.active = 0;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t go = s_any;
        v->inner_total = v->inner_total + v->k;
        if (go) {
            v->outer = v->outer + 1;
            v->lcnt[0].v = v->lcnt[1].v = v->lcnt[2].v = 0;
            v->fcnt[0].v = v->fcnt[1].v = v->fcnt[2].v = 0;
            v->tprev = v->tcnt.v;
            v->tcnt.v = 0;
            v->elim.v = 0;
            v->k = 0;
        }
        v->outer_go = go;
        __threadfence();
        set_cond(d.ctl, hd.outer, go);
    }
}

// Start of a run: fields written by the host (max_outer, max_inner, out,
// hist_cap, m, nacc0, use_graph, timeout_ns) are kept, the rest is reset.
__global__ void k_run_begin(Ctl *c, Handles hd)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    volatile Ctl *v = c;
    v->lcnt[0].v = v->lcnt[1].v = v->lcnt[2].v = 0;
    v->fcnt[0].v = v->fcnt[1].v = v->fcnt[2].v = 0;
    v->tcnt.v = 0;
    v->tprev = 0;
    v->frontier_rows.v = 0;
    v->bar_count.v = 0;
    v->stop_req.v = 0;
    v->self_seen.v = NONE;
    v->early_hit = 0;
    v->k = 0;
    v->status = ST_OK;
    v->verdict = 0;
    v->witness.v = NONE;
    v->elim.v = 0;
    v->nacc = v->nacc0;
    v->done.v = 0;
    v->relax.v = 0;
    v->inner_total = 0;
    v->t0 = global_ns();
    v->t_mark = v->t0;
    v->ph_dense = v->ph_rounds = v->ph_check = 0;
    const uint32_t go = v->nacc0 ? 1u : 0u;
    v->outer = go;
    v->outer_go = go;
    __threadfence();
    set_cond(c, hd.outer, go);
}

// ------------------------------------------------------------ dense round --
//
// Round 1 of an outer iteration relaxes every row from "no value" everywhere,
// so the value u offers is u + 1 if u is accepting and 0 otherwise -- and the
// flag is bit 31 of the matrix entry itself, so the round is a pure stream.
//
// Each warp owns tiles of WT_ROWS consecutive rows, with no block-wide phase:
// the tile's rowptr slice (fetched one tile ahead into registers) goes to a
// warp-private shared slice; the tile's edge span is streamed with 128-bit
// loads (WT_UNROLL per lane in flight); an edge whose target is accepting finds
// its row by binary search in the slice and does a shared-memory atomicMax.
// The first dense round of a run writes the tile's values out coalesced (this
// also resets whatever the previous run left).  Later ones write only the rows
// that got a value or still hold one from the previous outer iteration (bit v
// of the stale bitmap, fetched a tile ahead), so mval costs n / 4 bitmap bytes
// per round instead of 4n.  The round rewrites each tile's bitmap words with
// the rows that got a value; the push rounds add the vertices they raise from
// "no value".  Every row that got a value goes
// to list[1] (with its value in snap[1]) and to the touched list.
constexpr int DT_THREADS = 256;
constexpr int WT_WARPS = DT_THREADS / 32;
constexpr int WT_ROWS = 128;
// 128-bit colidx loads per lane in flight: a template parameter of k_dense (2, 4 or 8;
// map_autotune picks it per handle, 4 by default)
constexpr uint32_t WT_Q = 64; // queued accepting-target entries per warp (more are applied on the spot)
constexpr size_t DT_SMEM = 0; // static shared memory only

// the row of entry e in a tile: the last r < rows with rp[r] <= e (rp[0] <= e < rp[rows])
__device__ __forceinline__ uint32_t tile_row_of(const uint32_t *rp, uint32_t rows, uint32_t e)
{
    uint32_t lo = 0, hi = rows;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (rp[mid] <= e) lo = mid;
        else hi = mid;
    }
    return lo;
}

#ifndef MAPGPU_DENSE_MIN_BLOCKS
#define MAPGPU_DENSE_MIN_BLOCKS 6 // resident blocks per SM the register budget is sized for (measured best)
#endif

template <int WT_UNROLL>
__global__ void __launch_bounds__(DT_THREADS, MAPGPU_DENSE_MIN_BLOCKS) k_dense(const Dev d, Handles hd)
{
    // per warp, two buffers: the tile's rowptr slice [0, WT_ROWS], its stale words at WT_ROWS + 4
    __shared__ __align__(16) uint32_t s_rp[2][WT_WARPS][WT_ROWS + 8];
    __shared__ __align__(16) uint32_t s_best[WT_WARPS][WT_ROWS];
    // entries of the tile whose target is accepting (position, offered value), queued while the
    // span streams and applied afterwards with one lane per entry
    __shared__ uint32_t s_qe[WT_WARPS][WT_Q], s_qv[WT_WARPS][WT_Q], s_qn[WT_WARPS];
    __shared__ uint32_t s_stage[WT_WARPS][SB_ENTRIES];
    __shared__ uint32_t s_cnt[WT_WARPS][1], s_base[1];
    Ctl *ctl = d.ctl;
    // the rows that get a value go to list[1] and to the touched list
    uint32_t *const dst[1][2] = {{d.list[1], d.touched}};
    unsigned int *const ctr[1] = {&ctl->lcnt[1].v};
    Stage<1> st;
    st.buf = s_stage[threadIdx.x >> 5];
    st.cnt[0] = 0;
    default_stop(ctl, hd.outer);
    const uint32_t n = d.n;
    const uint32_t *__restrict__ rowptr = d.rowptr;
    const uint32_t *__restrict__ colidx = d.colidx;
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    uint32_t *best = s_best[warp];
    const uint32_t ntiles = (n + WT_ROWS - 1) / WT_ROWS;
    const uint32_t nw = gridDim.x * WT_WARPS;
    // sparse write-back from the second outer iteration of a run on
    const bool sparse = d.stale && *(volatile uint32_t *)&ctl->outer > 1;
#pragma unroll
    for (int k = 0; k < 4; ++k) best[lane * 4 + k] = 0;
    if (lane == 0) s_qn[warp] = 0;

    // tile t into buffer b by asynchronous copies (nothing held in registers while in flight):
    // rowptr words r0 + 4 lane .. + 3 (lanes past the tile's last row copy nothing and fill
    // zeros), rowptr[r0 + WT_ROWS] of a full tile, and in sparse mode the tile's 4 stale words
    auto issue = [&](uint32_t t, uint32_t b) {
        const uint32_t r0 = t * WT_ROWS, rows = min((uint32_t)WT_ROWS, n - r0);
        uint32_t *dst = s_rp[b][warp];
        const bool in = lane * 4 <= rows;
        cp_async16(dst + 4 * lane, rowptr + r0 + (in ? 4 * lane : 0), in ? 16u : 0u);
        if (lane == 0 && rows == WT_ROWS) cp_async4(dst + WT_ROWS, rowptr + r0 + WT_ROWS);
        if (lane == 1 && sparse) cp_async16(dst + WT_ROWS + 4, d.stale + 4 * (uint64_t)t, 16u);
        cp_async_commit();
    };
    uint32_t t = blockIdx.x * WT_WARPS + warp, buf = 0;
    if (t < ntiles) issue(t, 0);
    for (; t < ntiles; t += nw, buf ^= 1u) {
        const uint32_t r0 = t * WT_ROWS, rows = min((uint32_t)WT_ROWS, n - r0);
        if (t + nw < ntiles) { // the next tile's slice goes in flight; wait for this one's
            issue(t + nw, buf ^ 1u);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncwarp();
        if (d.comp) { // batched: a tile inside one frozen graph is skipped whole
            const uint32_t c0 = __ldg(d.comp + r0), c1 = __ldg(d.comp + r0 + rows - 1);
            if (c0 == c1 && !*(volatile uint32_t *)&d.cs[c0].active) continue;
        }
        const uint32_t *rp = s_rp[buf][warp];
        const uint32_t stale4 = sparse ? (rp[WT_ROWS + 4 + (lane >> 3)] >> ((lane & 7u) * 4)) & 0xFu : 0u;
        const uint32_t E0 = rp[0], E1 = rp[rows];
        for (uint32_t cs = E0 & ~3u; cs < E1; cs += 32 * 4 * WT_UNROLL) {
            uint4 w[WT_UNROLL];
#pragma unroll
            for (int j = 0; j < WT_UNROLL; ++j) {
                const uint32_t idx = cs + (j * 32 + lane) * 4;
                w[j] = idx < E1 ? __ldg(reinterpret_cast<const uint4 *>(colidx + idx)) : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int j = 0; j < WT_UNROLL; ++j) {
                // almost every entry points to a non-accepting vertex: one test per 128-bit load
                if (((w[j].x | w[j].y | w[j].z | w[j].w) >> 31) == 0u) continue;
                const uint32_t ebase = cs + (j * 32 + lane) * 4;
                const uint32_t cs4[4] = {w[j].x, w[j].y, w[j].z, w[j].w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t e = ebase + k, c = cs4[k];
                    if ((c >> 31) && e >= E0 && e < E1) { // the target is accepting: queue the entry
                        const uint32_t q = atomicAdd(&s_qn[warp], 1u);
                        if (q < WT_Q) {
                            s_qe[warp][q] = e;
                            s_qv[warp][q] = (c & 0x7FFFFFFFu) + 1u;
                        } else { // queue full: apply it here
                            atomicMax(&best[tile_row_of(rp, rows, e)], (c & 0x7FFFFFFFu) + 1u);
                        }
                    }
                }
            }
        }
        __syncwarp();
        { // the queued entries, one lane each: find the row, raise its best value
            const uint32_t nq = min(s_qn[warp], WT_Q);
            for (uint32_t i = lane; i < nq; i += 32)
                atomicMax(&best[tile_row_of(rp, rows, s_qe[warp][i])], s_qv[warp][i]);
            __syncwarp();
            if (lane == 0) s_qn[warp] = 0;
        }
        __syncwarp();
        const uint4 b4 = reinterpret_cast<const uint4 *>(best)[lane];
        uint32_t bs[4] = {b4.x, b4.y, b4.z, b4.w};
        // sparse mode: a tile with no value now and none left from the previous iteration (most
        // tiles) has nothing to write, append or mark, and its best[] slice is still zero
        if (sparse && !__any_sync(0xFFFFFFFFu, (b4.x | b4.y | b4.z | b4.w | stale4) != 0u)) {
            __syncwarp(); // every lane is done with this buffer before it is refilled
            continue;
        }
        if (d.comp) { // batched: rows of frozen graphs keep their values; record the change
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (lane * 4 + k >= rows) continue;
                const uint32_t c = __ldg(d.comp + r0 + lane * 4 + k);
                if (!*(volatile uint32_t *)&d.cs[c].active) {
                    best[lane * 4 + k] = 0;
                    bs[k] = 0xFFFFFFFFu; // marker: do not write
                } else if (bs[k] && *(volatile uint32_t *)&d.cs[c].last_change < 1u) {
                    atomicMax(&d.cs[c].last_change, 1u);
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (lane * 4 + k < rows && bs[k] != 0xFFFFFFFFu) d.mval[r0 + lane * 4 + k] = bs[k];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (bs[k] == 0xFFFFFFFFu) bs[k] = 0;
        } else if (sparse) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (lane * 4 + k < rows && (bs[k] || ((stale4 >> k) & 1u))) d.mval[r0 + lane * 4 + k] = bs[k];
        } else if (lane * 4 + 3 < rows) {
            reinterpret_cast<uint4 *>(d.mval + r0)[lane] = b4;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (lane * 4 + k < rows) d.mval[r0 + lane * 4 + k] = bs[k];
        }
        if (d.stale) { // the tile's bitmap words: the rows that hold a value now
            uint32_t got4 = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) got4 |= (bs[k] != 0u) << k;
            uint32_t word = got4 << ((lane & 7u) * 4);
            word |= __shfl_xor_sync(0xFFFFFFFFu, word, 1);
            word |= __shfl_xor_sync(0xFFFFFFFFu, word, 2);
            word |= __shfl_xor_sync(0xFFFFFFFFu, word, 4);
            if ((lane & 7u) == 0 && t * 4 + (lane >> 3) < d.words) d.stale[t * 4 + (lane >> 3)] = word;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool got = bs[k] && lane * 4 + k < rows;
            const uint32_t v = r0 + lane * 4 + k;
            if (got) {
                best[lane * 4 + k] = 0;
                *rec_snap(d.rec + v, 1) = bs[k];
                if (bs[k] == v + 1) atomicMin(&ctl->self_seen.v, v); // v reaches itself: an accepting cycle
            }
            stage_append<1>(st, 0, got, v, dst, ctr);
        }
        __syncwarp();
    }
    stage_flush_block<1>(st, s_cnt, s_base, dst, ctr);
    if (last_block(ctl)) epilogue_dense(ctl);
}

// ------------------------------------------------------------ push rounds --
//
// Round k + 1 >= 2.  In the synchronous schedule a row's new value is
//   m_{k+1}(w) = max(m_k(w), max over u in row w of offer_k(u)),
//   offer_k(u) = max(u + 1 if u accepting, m_k(u)).
// Every row already holds the offers of round k - 1 (round 1 relaxed every row),
// and only the vertices changed in round k (list[q], q = k & 1) offer anything
// new, so each of them pushes offer_k(u) -- taken from its snapshot snap[q][u],
// the value it ended round k with -- to its readers with atomicMax.  A reader
// that is raised joins list[q ^ 1] (once, via cbit) and raises its own
// snapshot; a reader raised from "no value" joins the touched list (this
// happens once per vertex and outer iteration).  Every reader is a frontier row
// of round k + 1 in the pull formulation; the frontier is kept (fbit, flist) and
// its row lengths are added to the relaxation count when it is cleared, at the
// start of the next round (or by k_check after the last one).
//
// The asynchronous schedule (SYNC = false) pushes the live value of u instead
// of its snapshot; values may then travel several edges in one round.
//
// One thread per listed vertex; the reader loop runs warp-uniformly so that the
// appends are aggregated with one atomic per warp and list.

// append w (where flag) to arr, reserving space with one atomic per warp; all lanes call it
__device__ __forceinline__ void warp_append(bool flag, uint32_t w, uint32_t *arr, unsigned int *ctr)
{
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, flag);
    if (!mask) return;
    const unsigned lane = lane_id(), leader = __ffs(mask) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(ctr, (unsigned)__popc(mask));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    if (flag) arr[base + __popc(mask & ((1u << lane) - 1u))] = w;
}

// The initially accepting vertices (v < n with bit v of acc0), for the frontier
// start; at most cap entries are written (cap = their count).
__global__ void k_acc_list(uint32_t n, const uint32_t *__restrict__ acc0, uint32_t *list, uint32_t cap,
                           unsigned int *cnt)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n; base += stride) {
        const uint64_t v = base + lane_id(); // warp-uniform loop
        const bool a = v < n && acc_bit(acc0, (uint32_t)v);
        const unsigned mask = __ballot_sync(0xFFFFFFFFu, a);
        if (!mask) continue;
        const unsigned lane = lane_id(), leader = __ffs(mask) - 1;
        unsigned at = 0;
        if (lane == leader) at = atomicAdd(cnt, (unsigned)__popc(mask));
        at = __shfl_sync(0xFFFFFFFFu, at, leader) + __popc(mask & ((1u << lane) - 1u));
        if (a && at < cap) list[at] = (uint32_t)v;
    }
}

// clear the frontier flag FB(p) of the rows in flist[p] and return their row lengths
__device__ __forceinline__ unsigned long long clear_frontier(const uint32_t *__restrict__ flist, uint32_t nf,
                                                             uint32_t p, uint4 *rec,
                                                             const uint32_t *__restrict__ rowptr,
                                                             const Dev &d, uint32_t nb, uint32_t bid)
{
    unsigned long long relax = 0;
    const uint64_t nthreads = (uint64_t)nb * blockDim.x; // nb blocks share the work (bid: this one)
    // warp-uniform loop: in batched runs the lanes of a warp add their row
    // lengths per graph (one atomic per graph present in the warp)
    for (uint64_t base = (uint64_t)bid * blockDim.x + (threadIdx.x & ~31u); base < nf; base += nthreads) {
        const uint64_t i = base + lane_id();
        unsigned long long len = 0;
        uint32_t w = 0;
        if (i < nf) {
            w = __ldcg(flist + i); // (written in this launch: read at L2)
            atomicAnd(rec_flags(rec + w), ~FB(p));
            len = __ldg(rowptr + w + 1) - __ldg(rowptr + w);
            relax += len;
        }
        if (d.comp) {
            const uint32_t c = i < nf ? __ldg(d.comp + w) : 0xFFFFFFFFu;
            const unsigned same = __match_any_sync(0xFFFFFFFFu, c);
            // 64-bit sum of the group's row lengths from two 32-bit reductions (no overflow)
            const unsigned lo = __reduce_add_sync(same, (unsigned)(len & 0xFFFFu));
            const unsigned hi = __reduce_add_sync(same, (unsigned)(len >> 16));
            const unsigned long long sum = (unsigned long long)lo + ((unsigned long long)hi << 16);
            if (c != 0xFFFFFFFFu && lane_id() == (unsigned)(__ffs(same) - 1) && sum)
                atomicAdd((unsigned long long *)&d.cs[c].relax, sum);
        }
    }
    return relax;
}

// inclusive warp scan
__device__ __forceinline__ uint32_t warp_inclusive_scan(uint32_t x)
{
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, x, off);
        if (lane_id() >= (unsigned)off) x += t;
    }
    return x;
}

// inclusive scan over a 256-thread block (s_warp: 8 shared words)
__device__ __forceinline__ uint32_t block_inclusive_scan(uint32_t x, uint32_t *s_warp)
{
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    x = warp_inclusive_scan(x);
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = lane < 8 ? s_warp[lane] : 0;
#pragma unroll
        for (int off = 1; off < 8; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, off);
            if (lane >= (unsigned)off) t += y;
        }
        if (lane < 8) s_warp[lane] = t;
    }
    __syncthreads();
    return warp ? x + s_warp[warp - 1] : x;
}

// Bounded grid-wide barrier of a cooperative launch (every block resident).
// Returns false if the wait gave up (the caller then stops).  Only thread 0 of
// each block touches the barrier words; with `p` < 3 it also reads the counters
// the next round needs (|list[p]|, |flist[p]|, self_seen, stop_req) into `s_vals`
// before the block is released, so that they cost one L2 read per block instead
// of one per warp.
constexpr uint32_t BAR_SPIN_LIMIT = 1u << 24;
#ifndef MAPGPU_BAR_SLEEP_NS
#define MAPGPU_BAR_SLEEP_NS 32 // back-off between polls of the barrier generation
#endif

// the barrier's fences: release before the arrival, acquire after the release (the block's
// writes, ordered before thread 0's by the block barrier, are covered cumulatively); a
// fence.acq_rel.gpu in their place measured the same
__device__ __forceinline__ void bar_fence() { __threadfence(); }

__device__ __forceinline__ bool grid_barrier(Ctl *ctl, uint32_t p = 3, uint32_t *s_vals = nullptr)
{
    __shared__ uint32_t s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t ok = 1;
        const uint32_t gen = *(volatile uint32_t *)&ctl->bar_gen.v;
        bar_fence();
        if (atomicAdd(&ctl->bar_count.v, 1u) == gridDim.x - 1) {
            atomicExch(&ctl->bar_count.v, 0u);
            bar_fence();
            atomicAdd(&ctl->bar_gen.v, 1u);
        } else {
            for (uint32_t it = 0; *(volatile uint32_t *)&ctl->bar_gen.v == gen; ++it) {
                if (it > BAR_SPIN_LIMIT) {
                    ok = 0;
                    ((volatile Ctl *)ctl)->gave_up = 1;
                    break;
                }
                if (it > 16) __nanosleep(MAPGPU_BAR_SLEEP_NS);
            }
        }
        bar_fence();
        s_ok = ok;
        if (p < 3) {
            volatile Ctl *v = ctl;
            s_vals[0] = v->lcnt[p].v;
            s_vals[1] = v->fcnt[p].v;
            s_vals[2] = v->self_seen.v;
            s_vals[3] = v->stop_req.v;
        }
    }
    __syncthreads();
    return s_ok != 0;
}

#ifndef MAPGPU_RC_E
#define MAPGPU_RC_E 1 // listed vertices per thread and chunk
#endif
#ifndef MAPGPU_RC_P
#define MAPGPU_RC_P 1 // push pairs per thread and step (loads and atomics in flight together)
#endif
constexpr int RC_E = MAPGPU_RC_E;
constexpr int RC_ENTRIES = 256 * RC_E; // per block and chunk
constexpr int RC_P = MAPGPU_RC_P;
// Asynchronous schedule: block-local passes over a block's own raised vertices per round
// (Ctl::lc_passes, per handle; measured on the 2^26 layered graph, ms per run for 0 / 1 / 2 / 4 /
// 8 passes: 18.2 / 17.0 / 17.2 / 17.4 / 17.5 with the dense start, 9.5 / 8.4 / 8.6 / 8.9 / 9.0
// with the frontier start; map_autotune measures it on the handle's graph)
#ifndef MAPGPU_LC_CAP
#define MAPGPU_LC_CAP 1024
#endif
constexpr uint32_t LC_CAP = MAPGPU_LC_CAP; // entries recorded per block and round (the rest only go through the list)

// The fix-point loop of one outer iteration: rounds 2, 3, ... until a round
// changes nothing.  Round r reads list[(r-1) % 3] and appends to list[r % 3];
// the counters of list[(r+1) % 3] (read in round r-1, appended again in round
// r+1) are reset by block 0 during round r, so one barrier per round suffices.
#ifndef MAPGPU_ROUNDS_MIN_BLOCKS
#define MAPGPU_ROUNDS_MIN_BLOCKS 6 // resident blocks per SM the register budget is sized for (measured best)
#endif
#ifndef MAPGPU_ROUNDS_PULL_MIN_BLOCKS
#define MAPGPU_ROUNDS_PULL_MIN_BLOCKS 5 // the same for the variant with pull rounds: 48 registers, fewer spills
                                        // (256-graph batch, ms per synchronous / asynchronous run at its tuned
                                        // choices: 41.0 / 41.7 with 6 blocks, 39.8 / 33.4 with 5, 40.8 / 30.7 with 4)
#endif

// ------------------------------------------------------------- pull rounds --
//
// A round whose list is a large share of the graph pulls instead of pushing: every row w
// streams its entries (as the dense round does, with the same warp tiles), and an entry u
// that changed in the round before (bit u of cbit[p_in], set from the list beforehand) offers
// max(u + 1 if u accepting, m(u)) -- its snapshot of the round before under the synchronous
// schedule, its live value under the asynchronous one.  Row w takes the largest offer if it
// is above its value; only row w's own warp writes w, so no atomics on values are needed and
// the synchronous round is the exact Jacobi step (Section 2: one product over the matrix):
// every value read is one of the round before.  A row holding a changed entry is a frontier
// row of the pull formulation, so the canonical relaxation count adds its length.  The
// snapshots, list flags and bits of the pulled list are cleared in the next round (or after
// the last one), when nobody reads them any more.
constexpr int PT_ROWS = 128;
#ifndef MAPGPU_PT_UNROLL
#define MAPGPU_PT_UNROLL 2 // 128-bit colidx loads per lane in flight in a pull round
#endif
constexpr int PT_UNROLL = MAPGPU_PT_UNROLL;
constexpr uint32_t PT_Q = 64;

struct NoPullSmem {
    uint32_t unused;
};
struct __align__(16) PullSmem {
    uint32_t rp[8][PT_ROWS + 8]; // per warp: the tile's rowptr slice
    uint32_t best[8][PT_ROWS];
    uint32_t qe[8][PT_Q], qu[8][PT_Q], qn[8];
    uint32_t hit[8][PT_ROWS / 32];
};

template <bool SYNC>
__device__ __forceinline__ uint32_t pull_offer(const Dev &d, uint32_t u, uint32_t p_in)
{
    const uint32_t x = SYNC ? *(volatile uint32_t *)rec_snap(d.rec + u, p_in) : *(volatile uint32_t *)(d.mval + u);
    return acc_bit(d.acc, u) ? max(x, u + 1) : x;
}

// the whole round by pull; appends go to list 1 (changed) and 2 (touched) of `st`.  relax
// gets the canonical count (SYNC or batched) or the entries pulled (asynchronous single
// graphs), prow the frontier rows.
template <bool SYNC>
__device__ __forceinline__ void pull_round(const Dev &d, uint32_t rr, uint32_t p_in, uint32_t p_out, PullSmem &ps, Stage<3> &st,
                           uint32_t *(*dst)[2], unsigned int **ctr, unsigned long long &relax,
                           unsigned long long &prow)
{
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const uint32_t n = d.n;
    const uint32_t *__restrict__ rowptr = d.rowptr;
    const uint32_t *__restrict__ colidx = d.colidx;
    const uint32_t *cb = pick3(p_in, d.cbit);
    const bool track = SYNC || d.comp;
    uint32_t *rp = ps.rp[warp], *best = ps.best[warp];
    unsigned long long hits = 0; // changed entries pulled
    const uint32_t ntiles = (n + PT_ROWS - 1) / PT_ROWS;
    const uint32_t nw = gridDim.x * (blockDim.x >> 5);
    if (lane == 0) ps.qn[warp] = 0;
    if (lane < PT_ROWS / 32) ps.hit[warp][lane] = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) best[lane * 4 + k] = 0;
    __syncwarp();
    // entry e of row (found by binary search in the tile's slice) offers the value of u
    auto apply = [&](uint32_t e, uint32_t u, uint32_t rows) {
        const uint32_t row = tile_row_of(rp, rows, e);
        atomicMax(&best[row], pull_offer<SYNC>(d, u, p_in));
        atomicOr(&ps.hit[warp][row >> 5], 1u << (row & 31u));
    };
    // (a double-buffered cp.async prefetch of the next tile's slice, as in the dense round,
    // measured slower here: the extra registers spill at this kernel's budget)
    for (uint32_t t = blockIdx.x * (blockDim.x >> 5) + warp; t < ntiles; t += nw) {
        const uint32_t r0 = t * PT_ROWS, rows = min((uint32_t)PT_ROWS, n - r0);
        if (d.comp) { // a tile inside one finished graph holds no changed vertex
            const uint32_t c0 = __ldg(d.comp + r0), c1 = __ldg(d.comp + r0 + rows - 1);
            if (c0 == c1 && !*(volatile uint32_t *)&d.cs[c0].active) continue;
        }
        for (uint32_t i = lane; i <= rows; i += 32) rp[i] = __ldg(rowptr + r0 + i);
        __syncwarp();
        const uint32_t E0 = rp[0], E1 = rp[rows];
        for (uint32_t cs = E0 & ~3u; cs < E1; cs += 32 * 4 * PT_UNROLL) {
            uint4 w[PT_UNROLL];
#pragma unroll
            for (int j = 0; j < PT_UNROLL; ++j) {
                const uint32_t idx = cs + (j * 32 + lane) * 4;
                w[j] = idx < E1 ? __ldg(reinterpret_cast<const uint4 *>(colidx + idx)) : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int j = 0; j < PT_UNROLL; ++j) {
                const uint32_t ebase = cs + (j * 32 + lane) * 4;
                const uint32_t c4[4] = {w[j].x, w[j].y, w[j].z, w[j].w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t e = ebase + k, u = c4[k] & 0x7FFFFFFFu;
                    if (e < E0 || e >= E1) continue;
                    // (a plain load: the grid barrier before the round's pull is an acquire, so no
                    // line of an earlier round's bits is left in L1)
                    if (!((cb[u >> 5] >> (u & 31u)) & 1u)) continue;
                    ++hits;
                    const uint32_t q = atomicAdd(&ps.qn[warp], 1u);
                    if (q < PT_Q) {
                        ps.qe[warp][q] = e;
                        ps.qu[warp][q] = u;
                    } else {
                        apply(e, u, rows);
                    }
                }
            }
        }
        __syncwarp();
        {
            const uint32_t nq = min(ps.qn[warp], PT_Q);
            for (uint32_t i = lane; i < nq; i += 32) apply(ps.qe[warp][i], ps.qu[warp][i], rows);
            __syncwarp();
            if (lane == 0) ps.qn[warp] = 0;
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t row = lane * 4 + k, w = r0 + row;
            const bool in = row < rows;
            const bool hit = in && ((ps.hit[warp][row >> 5] >> (row & 31u)) & 1u);
            const uint32_t b = in ? best[row] : 0u;
            if (in) best[row] = 0;
            uint32_t old = 0;
            bool raised = false;
            uint64_t len = 0;
            if (hit) {
                len = rp[row + 1] - rp[row];
                prow += 1;
                if (track) relax += len;
                old = *(volatile uint32_t *)(d.mval + w);
                raised = b > old;
                if (raised) {
                    d.mval[w] = b;
                    if (SYNC) *rec_snap(d.rec + w, p_out) = b;
                    atomicOr(rec_flags(d.rec + w), CB(p_out));
                    if (b == w + 1) atomicMin(&d.ctl->self_seen.v, w); // w reaches itself
                    if (old == 0 && d.stale) atomicOr(d.stale + (w >> 5), 1u << (w & 31u));
                }
            }
            if (d.comp) { // batched: per graph, the change and the frontier rows' lengths
                const uint32_t c = hit ? __ldg(d.comp + w) : 0xFFFFFFFFu;
                if (raised && *(volatile uint32_t *)&d.cs[c].last_change < rr) atomicMax(&d.cs[c].last_change, rr);
                const unsigned same = __match_any_sync(0xFFFFFFFFu, c);
                const unsigned lo = __reduce_add_sync(same, (unsigned)(len & 0xFFFFu));
                const unsigned hi = __reduce_add_sync(same, (unsigned)(len >> 16));
                const unsigned long long sum = (unsigned long long)lo + ((unsigned long long)hi << 16);
                if (c != 0xFFFFFFFFu && lane == (unsigned)(__ffs(same) - 1) && sum)
                    atomicAdd((unsigned long long *)&d.cs[c].relax, sum);
            }
            stage_append<3>(st, 1, raised, w, dst, ctr);
            stage_append<3>(st, 2, raised && old == 0, w, dst, ctr);
        }
        __syncwarp();
        if (lane < PT_ROWS / 32) ps.hit[warp][lane] = 0;
        __syncwarp();
    }
    if (!track) relax += hits;
}

// after a pull round: its list's bits, list flags and (SYNC) snapshots back to zero
template <bool SYNC>
__device__ __forceinline__ void pull_cleanup(const Dev &d, const uint32_t *__restrict__ list, uint32_t nl, uint32_t q)
{
    const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
    uint32_t *cb = pick3(q, d.cbit);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nl; i += nthreads) {
        const uint32_t u = __ldcg(list + i);
        if (SYNC) *rec_snap(d.rec + u, q) = 0;
        atomicAnd(rec_flags(d.rec + u), ~CB(q));
        cb[u >> 5] = 0; // every bit set in cbit[q] belongs to this list
    }
}

// ------------------------------------------------- self-map test, elimination --
//
// Over the touched vertices (exactly the vertices with a defined map value),
// Section 2: witness = smallest v with map(v) = v; every map value u is removed
// from the accepting set (exact count of removals).  The map vector is left
// intact (the next dense round overwrites it).  Every thread of the grid calls
// it (it ends with a last-block epilogue).  When the loop runs as a CUDA graph
// it is the tail of the fix-point kernel; stepped from the host it is k_check.
__device__ __forceinline__ void check_phase(const Dev &d, Handles hd, bool work = true)
{
    Ctl *ctl = d.ctl;
    const uint32_t nt = work ? *(volatile uint32_t *)&ctl->tcnt.v : 0u; // without work: only the ticket
    const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
    unsigned elim = 0;
    uint32_t wit = NONE;
    // warp-uniform loop (batched runs aggregate per graph within the warp)
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < nt; base += nthreads) {
        const uint64_t i = base + lane_id();
        uint32_t c = 0xFFFFFFFFu, removed = 0;
        if (i < nt) {
            // (in a CUDA graph this runs in the launch that wrote both arrays: read them at L2)
            const uint32_t v = __ldcg(d.touched + i);
            const uint32_t x = __ldcg(d.mval + v);
            const uint32_t u = x - 1; // x != 0 for a touched vertex (checked all the same below)
            if (d.comp) c = __ldg(d.comp + v);
            if (x != 0 && u == v) {
                wit = min(wit, u);
                if (d.comp) atomicMin(&d.cs[c].witness, u);
            }
            const uint32_t bit = 1u << (u & 31u);
            // a plain load (it may be served by L1 and be stale): it only saves the atomic when
            // the bit is already clear, and the atomic's old value decides who removed u.  Many
            // vertices share a few map values (state graphs), and their reads stay off the L2 line
            if (x != 0 && (d.acc[u >> 5] & bit)) {
                const uint32_t old = atomicAnd(d.acc + (u >> 5), ~bit);
                if (old & bit) { // this thread removed u
                    elim++;
                    removed = 1;
                    if (!d.alist) { // the dense round reads the flag in the matrix entries: clear it, log u
                        d.elog[atomicAdd(&ctl->ecnt.v, 1u)] = u;
                        const uint32_t b = __ldg(d.rrowptr + u), e = __ldg(d.rrowptr + u + 1);
                        for (uint32_t j = b; j < e; ++j) d.colidx_w[__ldg(d.rpos + j)] = u;
                    }
                }
            }
        }
        if (d.comp) { // per graph: touched vertices and removals, one atomic per graph in the warp
            const unsigned same = __match_any_sync(0xFFFFFFFFu, c);
            const unsigned nt_c = __popc(same);
            const unsigned ne_c = __reduce_add_sync(same, removed);
            if (c != 0xFFFFFFFFu && lane_id() == (unsigned)(__ffs(same) - 1)) {
                atomicAdd(&d.cs[c].touched, nt_c);
                if (ne_c) atomicAdd(&d.cs[c].elim, ne_c);
            }
        }
    }
    block_add_min_u32(elim, wit, &ctl->elim.v, &ctl->witness.v);
    if (!d.comp) {
        if (last_block(ctl)) epilogue_check(ctl, hd);
    } else if (last_block_all(ctl)) {
        epilogue_batch(d, hd);
    }
}

__global__ void __launch_bounds__(256) k_check(const Dev d, Handles hd) { check_phase(d, hd); }

// Small lists: a round over few vertices is mostly the fixed cost of the grid barrier, so
// while the list stays small block 0 runs the rounds alone, with block barriers, and the other
// blocks wait for it to hand back (solo_gen).  The wait is bounded: it gives up when block 0's
// heartbeat (solo_beat, bumped at every round and every 64 Ki pushes) has not moved for about a
// second.
constexpr uint32_t SOLO_BEAT_SPINS = 1u << 14; // polls between heartbeat checks
constexpr uint32_t SOLO_BEAT_CHECKS = 1u << 8; // heartbeat checks without progress before giving up

// every thread of a waiting block calls it; returns false if the wait gave up.  s_vals gets
// block 0's r, |list|, |frontier| and status; *seen (shared: the hand-backs this block has seen)
// counts this one
__device__ __forceinline__ bool solo_wait(Ctl *ctl, uint32_t *seen, uint32_t *s_vals)
{
    __shared__ uint32_t s_ok;
    if (threadIdx.x == 0) {
        volatile Ctl *v = ctl;
        uint32_t ok = 1, beat = v->solo_beat.v, still = 0;
        for (uint32_t it = 0; v->solo_gen.v == *seen; ++it) {
            if (it == SOLO_BEAT_SPINS) {
                it = 0;
                const uint32_t b = v->solo_beat.v;
                if (b == beat && ++still > SOLO_BEAT_CHECKS) {
                    ok = 0;
                    v->gave_up = 2;
                    break;
                }
                if (b != beat) still = 0;
                beat = b;
            }
            __nanosleep(256);
        }
        __threadfence();
        s_vals[0] = v->solo_r;
        s_vals[1] = v->solo_nl;
        s_vals[2] = v->solo_nf;
        s_vals[3] = v->solo_status;
        *seen += 1;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// PULL: the variant with pull rounds (launched when some round may pull; the push-only
// variant keeps the register budget of the push path free of the pull path's needs)
template <bool SYNC, bool PULL>
__global__ void __launch_bounds__(256, PULL ? MAPGPU_ROUNDS_PULL_MIN_BLOCKS : MAPGPU_ROUNDS_MIN_BLOCKS)
    k_rounds(const Dev d, Handles hd)
{
    __shared__ uint32_t s_stage[8][3 * SB_ENTRIES];
    __shared__ uint32_t s_cnt[8][3], s_base[3];
    __shared__ uint32_t s_incl[RC_ENTRIES], s_o[RC_ENTRIES], s_b[RC_ENTRIES], s_scan[8];
    __shared__ uint32_t s_loc[LC_CAP], s_ln; // vertices this block listed in this round
    __shared__ uint32_t *s_dst[3][2];
    __shared__ unsigned int *s_ctr[3];
    __shared__ uint32_t s_vals[4]; // after each barrier: |list|, |flist| of the round, self_seen, stop_req
    __shared__ __align__(16) typename std::conditional<PULL, PullSmem, NoPullSmem>::type s_pull;
    Ctl *ctl = d.ctl;
    volatile Ctl *vc = ctl;
    const unsigned lane = lane_id();
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    const uint32_t max_inner = vc->max_inner;
    unsigned long long relax = 0, frows = 0;
    uint32_t status = ST_OK;
    uint32_t nl = vc->lcnt[1].v; // vertices that got a value in the dense round
    uint32_t nf = vc->fcnt[1].v; // frontier rows of the last round (cleared at the start of the next)
    uint32_t r = 1;              // rounds completed
    const bool early = vc->early_exit && !d.comp;
    // Frontier start: no dense round ran.  Round 1 gives every row the largest accepting id in
    // it; only the rows that hold a currently accepting vertex get one, so here each accepting
    // vertex u pushes u + 1 to its readers (the same values, from far fewer edges when the
    // accepting set is small).  This kernel is then the loop body's first: it resets the
    // values of the previous outer iteration (exactly its touched vertices) before round 1.
    const bool fstart = d.alist != nullptr;
    if (fstart) {
        default_stop(ctl, hd.outer);
        const uint32_t tp = vc->tprev;
        const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tp; i += nthreads) {
            const uint32_t v = __ldg(d.touched + i);
            // (batched: a graph that has finished keeps its last map vector)
            if (!d.comp || *(volatile uint32_t *)&d.cs[__ldg(d.comp + v)].active) d.mval[v] = 0;
        }
        if (!grid_barrier(ctl)) status = ST_TIMEOUT; // every reset is visible before any push
        nl = d.na;
        r = 0;
        if (SYNC && lead) relax += vc->m; // canonical count: round 1 of the pull schedule relaxes every row
    }
    if (early && vc->self_seen.v != NONE) nl = 0; // the dense round already found a self-mapped vertex
    if (!fstart && nl && max_inner < 2) status = ST_LIMIT;
    // the frontier (rows reading a changed vertex) gives the canonical relaxation count of the
    // synchronous schedule; a single-graph asynchronous run counts its pushes instead
    const bool track = SYNC || d.comp;
    const bool local = !SYNC && !d.comp;
    const uint32_t pull_min = (PULL && d.cbit[0]) ? vc->pull_min : 0u;
    uint32_t pulled = 0; // > 0: the last round pulled, over a list of that many vertices
    unsigned long long prow = 0; // frontier rows of pull rounds
    // rounds block 0 may run alone: list and frontier limits, hand-backs seen so far (every
    // block counts the same); in shared memory, which keeps registers for the push path
    __shared__ uint32_t s_solo[4];
    if (threadIdx.x == 0) {
        s_solo[0] = vc->solo_max;
        s_solo[1] = vc->solo_fmax;
        s_solo[2] = 0; // hand-backs seen: every launch starts from 0 (the check epilogue resets the count)
        s_solo[3] = vc->lc_passes; // (block-local passes per round, asynchronous single graphs)
    }
    __syncthreads();
    while (nl && status == ST_OK) {
        const uint32_t rr = r + 1; // this round
        const uint32_t p_in = (rr - 1) % 3, p_out = rr % 3, p_free = (rr + 1) % 3;
        const bool first = rr == 1; // round 1 from the accepting vertices (frontier start only)
        // a small list: block 0 runs this round (and the next small ones) alone
        const bool solo = s_solo[0] && !first && !pulled && nl <= s_solo[0] && nf <= s_solo[1];
        if (solo && blockIdx.x != 0) {
            const bool ok = solo_wait(ctl, &s_solo[2], s_vals);
            if (!ok) {
                status = ST_TIMEOUT;
                break;
            }
            r = s_vals[0];
            nl = s_vals[1];
            nf = s_vals[2];
            status = s_vals[3];
            continue;
        }
        const uint32_t nb = solo ? 1u : gridDim.x, bid = solo ? 0u : blockIdx.x; // blocks sharing the round
        if (lead) {
            vc->lcnt[p_free].v = 0;
            vc->fcnt[p_free].v = 0;
        }
        // the list the round before pulled over (list[p_free], which nothing reads any more)
        if (PULL && pulled) pull_cleanup<SYNC>(d, pick3(p_free, d.list), pulled, p_free);
        const bool pull = PULL && !solo && !first && pull_min && nl >= pull_min;
        const uint32_t *__restrict__ list = first ? d.alist : pick3(p_in, d.list);
        uint32_t *const list_out = pick3(p_out, d.list);
        uint32_t *const flist_out = pick3(p_out, d.flist);
        // appends: 0 = this round's frontier, 1 = changed vertices, 2 = newly touched vertices.
        // Their destinations live in shared memory (read only when a buffer is flushed), which
        // keeps registers free for occupancy; the first read comes after a __syncthreads.
        if (threadIdx.x == 0) {
            s_dst[0][0] = flist_out;
            s_dst[1][0] = list_out;
            s_dst[2][0] = d.touched;
            s_dst[0][1] = s_dst[1][1] = s_dst[2][1] = nullptr;
            s_ctr[0] = &ctl->fcnt[p_out].v;
            s_ctr[1] = &ctl->lcnt[p_out].v;
            s_ctr[2] = &ctl->tcnt.v;
        }
        uint32_t *(*const dst)[2] = s_dst;
        unsigned int **const ctr = s_ctr;
        Stage<3> st;
        st.buf = s_stage[threadIdx.x >> 5];
        st.cnt[0] = st.cnt[1] = st.cnt[2] = 0;
        // the previous round's frontier: clear its flags, count its relaxations
        if (track && !first) relax += clear_frontier(pick3(p_in, d.flist), nf, p_in, d.rec, d.rowptr, d, nb, bid);
        // round 1 of a frontier start keeps no frontier: its relaxations are the canonical m
        const bool trk = track && !first;

        // chunks of RC_ENTRIES listed vertices per block (RC_E per thread, loaded
        // together); their (vertex, reader) pairs are spread evenly over the block's
        // threads, RC_P pairs per thread per step with all their loads and atomics
        // in flight before any result is used
        // every block takes an even contiguous share of the list (a pull round: none)
        const uint64_t per = (nl + nb - 1) / nb;
        const uint64_t beg = (uint64_t)bid * per, end = pull ? beg : min((uint64_t)nl, beg + per);
        if constexpr (PULL) if (pull) { // the list's bits, then (once every block has set its share) the pull itself
            uint32_t *cb = pick3(p_in, d.cbit);
            const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
            for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nl; i += nthreads) {
                const uint32_t u = __ldcg(list + i);
                atomicOr(cb + (u >> 5), 1u << (u & 31u));
            }
            if (!grid_barrier(ctl)) {
                status = ST_TIMEOUT;
                break;
            }
            pull_round<SYNC>(d, rr, p_in, p_out, s_pull, st, dst, ctr, relax, prow);
        }
        // asynchronous single graph: once its share of the list is done, the block pushes again
        // the live values of the vertices it listed itself in this round (recorded in s_loc), up
        // to lc_passes passes, so that values travel several edges per round.  These extra pushes
        // touch no list flag: every listed vertex still goes through the list to the next round.
        if (local) {
            if (threadIdx.x == 0) s_ln = 0;
            __syncthreads();
        }
        uint64_t c0 = beg, cend = end;
        bool loc = false; // chunk entries from s_loc instead of the list
        uint32_t lpass = 0, qend = 0;
        for (;;) {
            if (c0 >= cend) {
                if (!local || lpass >= s_solo[3]) break;
                const uint32_t q = min(s_ln, (uint32_t)LC_CAP); // s_ln is final: a barrier ended the last chunk
                if (q == qend) break;
                loc = true;
                c0 = qend;
                cend = q;
                qend = q;
                ++lpass;
            }
            // each thread reads up to RC_E listed vertices and consumes their
            // snapshots and list flags (nothing else reads them in this round)
            uint32_t o[RC_E], b[RC_E], len[RC_E];
#pragma unroll
            for (int k = 0; k < RC_E; ++k) {
                const uint64_t i = c0 + threadIdx.x * RC_E + k;
                o[k] = b[k] = len[k] = 0;
                if (i < cend) {
                    // (lists are rewritten every third round of this launch: read them at L2, never
                    // through the non-coherent path)
                    const uint32_t u = loc ? s_loc[i] : __ldcg(list + i);
                    const bool listed = !loc && !(first && SYNC); // in list[p_in], with a snapshot (SYNC)
                    const uint32_t mu = SYNC ? (listed ? *(volatile uint32_t *)rec_snap(d.rec + u, p_in) : 0u)
                                             : *(volatile uint32_t *)(d.mval + u);
                    const bool acc_u = acc_bit(d.acc, u);
                    o[k] = acc_u ? max(mu, u + 1) : mu;
                    b[k] = __ldg(d.rrowptr + u);
                    // round 1: an eliminated vertex offers nothing new, nor does one of a finished graph
                    const bool idle = first && !loc &&
                                      (!acc_u || (d.comp && !*(volatile uint32_t *)&d.cs[__ldg(d.comp + u)].active));
                    len[k] = idle ? 0u : __ldg(d.rrowptr + u + 1) - b[k];
                    if (SYNC && listed) *rec_snap(d.rec + u, p_in) = 0;
                    if (listed && !first) atomicAnd(rec_flags(d.rec + u), ~CB(p_in));
                }
            }
            uint32_t tot = 0;
#pragma unroll
            for (int k = 0; k < RC_E; ++k) tot += len[k];
            uint32_t run = block_inclusive_scan(tot, s_scan) - tot; // pairs before this thread's entries
#pragma unroll
            for (int k = 0; k < RC_E; ++k) {
                const uint32_t e = threadIdx.x * RC_E + k;
                s_o[e] = o[k];
                s_b[e] = b[k] - run; // reader of pair p is rcol[s_b[owner] + p] (32-bit wrap intended)
                run += len[k];
                s_incl[e] = run;
            }
            __syncthreads();
            const uint32_t total = s_incl[RC_ENTRIES - 1];
            if (!track && threadIdx.x == 0) relax += total; // pushes of this chunk
            for (uint32_t p0 = 0; p0 < total; p0 += 256 * RC_P) {
                // a round block 0 runs alone shows progress every 64 Ki pushes (the waiting blocks'
                // heartbeat), so a round over long reader lists is not taken for a stalled block
                if (solo && threadIdx.x == 0 && (p0 & 0xFFFFu) == 0 && p0) vc->solo_beat.v = vc->solo_beat.v + 1;
                uint32_t w[RC_P], ob[RC_P], fold[RC_P], mold[RC_P];
                bool act[RC_P];
#pragma unroll
                for (int j = 0; j < RC_P; ++j) {
                    const uint32_t p = p0 + j * 256 + threadIdx.x;
                    act[j] = p < total;
                    w[j] = 0;
                    ob[j] = 0;
                    if (act[j]) {
                        uint32_t lo = 0, hi = RC_ENTRIES - 1; // the owner: first entry with s_incl > p
                        while (lo < hi) {
                            const uint32_t mid = (lo + hi) >> 1;
                            if (s_incl[mid] > p) hi = mid;
                            else lo = mid + 1;
                        }
                        ob[j] = s_o[lo];
                        const uint32_t jj = s_b[lo] + p; // 32-bit arithmetic: jj = b + (p - excl)
                        w[j] = __ldg(d.rcol + jj);
                    }
                }
#pragma unroll
                for (int j = 0; j < RC_P; ++j) {
                    fold[j] = FB(p_out);
                    mold[j] = 0xFFFFFFFFu;
                    if (act[j]) {
                        if (trk) fold[j] = atomicOr(rec_flags(d.rec + w[j]), FB(p_out));
                        mold[j] = atomicMax(d.mval + w[j], ob[j]);
                    }
                }
                uint32_t cold[RC_P];
#pragma unroll
                for (int j = 0; j < RC_P; ++j) {
                    cold[j] = CB(p_out);
                    if (act[j] && ob[j] > mold[j]) { // raised; the record's sector is in L2 by now
                        if (SYNC) atomicMax(rec_snap(d.rec + w[j], p_out), ob[j]);
                        cold[j] = atomicOr(rec_flags(d.rec + w[j]), CB(p_out));
                    }
                }
#pragma unroll
                for (int j = 0; j < RC_P; ++j) {
                    const bool raised = act[j] && ob[j] > mold[j];
                    if (raised && ob[j] == w[j] + 1) atomicMin(&ctl->self_seen.v, w[j]); // w reaches itself
                    if (raised && d.comp) { // batched: this graph changed in this round
                        const uint32_t c = __ldg(d.comp + w[j]);
                        if (*(volatile uint32_t *)&d.cs[c].last_change < rr) atomicMax(&d.cs[c].last_change, rr);
                    }
                    stage_append<3>(st, 0, act[j] && !(fold[j] & FB(p_out)), w[j], dst, ctr);
                    stage_append<3>(st, 1, raised && !(cold[j] & CB(p_out)), w[j], dst, ctr);
                    if (local && raised && !(cold[j] & CB(p_out))) { // listed here: push it again in this round
                        const uint32_t q = atomicAdd(&s_ln, 1u);
                        if (q < LC_CAP) s_loc[q] = w[j];
                    }
                    stage_append<3>(st, 2, raised && mold[j] == 0, w[j], dst, ctr);
                    if (raised && mold[j] == 0 && d.stale) // the next dense round resets it
                        atomicOr(d.stale + (w[j] >> 5), 1u << (w[j] & 31u));
                }
            }
            __syncthreads(); // before the shared arrays are refilled
            c0 += RC_ENTRIES;
        }
        stage_flush_block<3>(st, s_cnt, s_base, dst, ctr);
        if (lead && timed_out(vc)) vc->stop_req.v = 1;
        if (solo) { // block 0 alone: its appends are complete after a block barrier
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                s_vals[0] = vc->lcnt[p_out].v;
                s_vals[1] = vc->fcnt[p_out].v;
                s_vals[2] = vc->self_seen.v;
                s_vals[3] = vc->stop_req.v;
                vc->solo_beat.v = vc->solo_beat.v + 1; // progress: one more round
            }
            __syncthreads();
        } else if (!grid_barrier(ctl, p_out, s_vals)) {
            status = ST_TIMEOUT;
            break;
        }
        r = rr;
        pulled = pull ? nl : 0u;
        nf = s_vals[1];
        if (!first) frows += track ? nf : nl; // frontier rows, or the vertices that pushed
        nl = s_vals[0];                       // changed in this round
        if (early && nl && s_vals[2] != NONE) { // stop here: the recorded vertex is the witness
            nl = 0;
            if (lead) vc->early_hit = 1;
        }
        if (s_vals[3]) status = ST_TIMEOUT;
        else if (nl && r + 1 > max_inner) status = ST_LIMIT;
        // block 0 hands back when the next round is not one it runs alone (the same test every
        // block makes at the top of the loop)
        if (solo && !(nl && status == ST_OK && nl <= s_solo[0] && nf <= s_solo[1])) {
            if (threadIdx.x == 0) {
                vc->solo_r = r;
                vc->solo_nl = nl;
                vc->solo_nf = nf;
                vc->solo_status = status;
                __threadfence();
                atomicAdd(&ctl->solo_gen.v, 1u);
                s_solo[2] += 1; // (read by thread 0 only, in solo_wait)
            }
        }
    }
    // the last round's frontier: clear its flags, count its relaxations
    if (r > 1 && track) relax += clear_frontier(pick3(r % 3, d.flist), nf, r % 3, d.rec, d.rowptr, d, gridDim.x, blockIdx.x);
    if (PULL && pulled) pull_cleanup<SYNC>(d, pick3((r + 2) % 3, d.list), pulled, (r + 2) % 3); // list[p_in] of round r
    block_add_u64(relax, (unsigned long long *)&ctl->relax.v);
    block_add_u64(track ? prow : 0ull, (unsigned long long *)&ctl->frontier_rows.v);
    if (threadIdx.x == 0 && status != ST_OK) vc->status = status; // any block that stopped early
    if (lead) {
        vc->k = r;
        vc->frontier_rows.v = vc->frontier_rows.v + frows;
        phase_end(vc, &vc->ph_rounds); // every block has passed the last barrier
        __threadfence();
    }
    // In a CUDA graph the self-map test and the elimination follow in this launch (one kernel
    // boundary less per outer iteration); every block's appends were flushed before the last
    // barrier.  A block whose barrier gave up skips the work but still takes its ticket.
    if (vc->use_graph) check_phase(d, hd, status == ST_OK);
}

// ------------------------------------------------------- pointer doubling --
//
// The fix-point of one outer iteration, asynchronous schedule, on a graph whose every row holds
// at most one entry (the state graph of a deterministic system: each state has one successor,
// and its row is that one entry).  Row v then takes its value from one vertex only, src(v), so
// the map value of v is the largest offer along the chain src(v), src(src(v)), ...  With
// Q_k(v) = src^{2^k}(v) (NONE past the end of the chain) and B_k(v) the largest offer of
// src^j(v) for 1 <= j <= 2^k, the dense round gives B_0, and
//     B_{k+1}(v) = max(B_k(v), B_k(Q_k(v))),   Q_{k+1}(v) = Q_k(Q_k(v)).
// A round is one pass over every vertex: a pure gather of one 8-byte (B_k, Q_k) pair at Q_k(v),
// the pairs double-buffered (v alone writes its own pair, and its value when it rises).  When a
// round raises nothing, B_k covers the
// whole chain (a vertex at distance d in (2^{k+1}, 2^{k+2}] from v lies within 2^{k+1} of
// Q_k(v), whose value B_{k+1}(v) already took), so the loop stops there: about log2 of the
// propagation depth rounds instead of the depth.  The values are the least fix-point's, as the
// oracle's rounds give them; the round count is the number of passes (at most the synchronous
// schedule's rounds).
__global__ void __launch_bounds__(256, MAPGPU_ROUNDS_MIN_BLOCKS) k_func(const Dev d, Handles hd)
{
    __shared__ uint32_t s_stage[8][SB_ENTRIES];
    __shared__ uint32_t s_cnt[8][1], s_base[1];
    __shared__ uint32_t s_vals[4];
    Ctl *ctl = d.ctl;
    volatile Ctl *vc = ctl;
    const unsigned lane = lane_id();
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    const uint32_t n = d.n, max_inner = vc->max_inner;
    const bool early = vc->early_exit != 0;
    const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t status = ST_OK;
    unsigned long long relax = 0;
    uint32_t r = 1;              // rounds completed (round 1: the dense round)
    uint32_t nl = vc->lcnt[1].v; // vertices that got a value in the dense round
    if (early && vc->self_seen.v != NONE) nl = 0; // the dense round already found a self-mapped vertex
    if (nl && max_inner < 2) status = ST_LIMIT;
    // (B_k(v), Q_k(v)) and (B_{k+1}(v), Q_{k+1}(v)), 8n bytes each, in the change-list and
    // frontier-list spaces (12n bytes each, unused by these rounds), so that one gather brings both
    uint2 *pa = reinterpret_cast<uint2 *>(d.list[0]), *pb = reinterpret_cast<uint2 *>(d.flist[0]);
    if (nl && status == ST_OK) {
        // B_0: the dense round's values; Q_0: the one entry of each row (its flag bit cleared), or NONE
        for (uint64_t v = tid; v < n; v += nthreads) {
            const uint32_t b = __ldg(d.rowptr + v), e = __ldg(d.rowptr + v + 1);
            pa[v] = make_uint2(__ldcg(d.mval + v), e > b ? (__ldcg(d.colidx + b) & 0x7FFFFFFFu) : NONE);
        }
        if (!grid_barrier(ctl)) status = ST_TIMEOUT;
    }
    // vertices raised from "no value" join the touched list (and the stale bitmap)
    uint32_t *const dst[1][2] = {{d.touched, nullptr}};
    unsigned int *const ctr[1] = {&ctl->tcnt.v};
    Stage<1> st;
    st.buf = s_stage[threadIdx.x >> 5];
    st.cnt[0] = 0;
    while (nl && status == ST_OK) {
        const uint32_t rr = r + 1, p_out = rr % 3, p_free = (rr + 1) % 3;
        if (lead) vc->lcnt[p_free].v = 0; // (counts the round after this one)
        uint32_t changed = 0, pulls = 0;
        // warp-uniform steps (every lane takes part in the appends)
        for (uint64_t base = tid - lane; base < n; base += nthreads) {
            const uint64_t v = base + lane;
            bool fresh = false;
            if (v < n) {
                // (both buffers are written within this launch: read them at L2)
                const uint2 cur = __ldcg(pa + v);
                uint2 nxt = make_uint2(cur.x, NONE);
                if (cur.y != NONE) {
                    const uint2 at = __ldcg(pa + cur.y); // (B_k, Q_k) at Q_k(v)
                    nxt.y = at.y;
                    if (at.x) {
                        ++pulls;
                        if (at.x > cur.x) {
                            nxt.x = at.x;
                            d.mval[v] = at.x; // (v's own thread is its only writer)
                            ++changed;
                            fresh = cur.x == 0;
                            if (at.x == (uint32_t)v + 1u) atomicMin(&ctl->self_seen.v, (uint32_t)v); // v reaches itself
                            if (fresh && d.stale) atomicOr(d.stale + (v >> 5), 1u << (v & 31u));
                        }
                    }
                }
                pb[v] = nxt;
            }
            stage_append<1>(st, 0, fresh, (uint32_t)v, dst, ctr);
        }
        stage_flush_block<1>(st, s_cnt, s_base, dst, ctr);
        st.cnt[0] = 0;
        const uint32_t wc = __reduce_add_sync(0xFFFFFFFFu, changed);
        if (lane == 0 && wc) atomicAdd(&ctl->lcnt[p_out].v, wc);
        relax += pulls;
        if (lead && timed_out(vc)) vc->stop_req.v = 1;
        if (!grid_barrier(ctl, p_out, s_vals)) {
            status = ST_TIMEOUT;
            break;
        }
        r = rr;
        nl = s_vals[0]; // vertices raised in this round
        if (early && nl && s_vals[2] != NONE) { // stop here: the recorded vertex is the witness
            nl = 0;
            if (lead) vc->early_hit = 1;
        }
        if (s_vals[3]) status = ST_TIMEOUT;
        else if (nl && r + 1 > max_inner) status = ST_LIMIT;
        uint2 *const tmp = pa;
        pa = pb;
        pb = tmp;
    }
    // (relaxations of an asynchronous run: m per outer iteration, plus one per value taken)
    block_add_u64(relax, (unsigned long long *)&ctl->relax.v);
    block_add_u64(relax, (unsigned long long *)&ctl->frontier_rows.v); // (the vertices that took one)
    if (threadIdx.x == 0 && status != ST_OK) vc->status = status;
    if (lead) {
        vc->k = r;
        phase_end(vc, &vc->ph_rounds); // every block has passed the last barrier
        __threadfence();
    }
    if (vc->use_graph) check_phase(d, hd, status == ST_OK);
}

// Batched runs, start of a run: every graph's record (the host keeps off, m, nacc0).
__global__ void k_batch_begin(const Dev d)
{
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < d.ncomp; c += gridDim.x * blockDim.x) {
        CompState &S = d.cs[c];
        S.active = S.nacc0 ? 1u : 0u;
        S.outer = S.active;
        S.verdict = 0;
        S.witness = NONE;
        S.nacc = S.nacc0;
        S.elim = 0;
        S.touched = 0;
        S.last_change = 0;
        S.status = ST_OK;
        S.relax = 0;
        S.inner_total = 0;
    }
}

// External encoding into `dst` (NULL: ctl->out): MAP_NONE for no value, else
// the vertex id; all MAP_NONE when no outer iteration ran.
__global__ void k_export(uint32_t n, const uint32_t *__restrict__ mval, const Ctl *ctl, uint32_t *dst,
                         const uint32_t *__restrict__ comp, const CompState *cs)
{
    uint32_t *out = dst ? dst : ctl->out;
    const bool none = ctl->outer == 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint32_t x = __ldg(mval + v);
        if (comp) { // batched: each graph's own ids, MAP_NONE for a graph that never ran
            const uint32_t c = __ldg(comp + v);
            out[v] = (cs[c].outer == 0 || x == 0) ? NONE : x - 1u - cs[c].off;
        } else {
            out[v] = none ? NONE : x - 1u;
        }
    }
}

// End of a run: give the vertices eliminated in it their accepting flag back
// in the matrix entries (they are all accepting in the initial set).
__global__ void __launch_bounds__(256) k_restore(const Dev d)
{
    Ctl *ctl = d.ctl;
    const uint32_t ne = *(volatile uint32_t *)&ctl->ecnt.v;
    const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ne; i += nthreads) {
        const uint32_t u = __ldg(d.elog + i);
        const uint32_t b = __ldg(d.rrowptr + u), e = __ldg(d.rrowptr + u + 1);
        for (uint32_t j = b; j < e; ++j) d.colidx_w[__ldg(d.rpos + j)] = u | 0x80000000u;
    }
    if (last_block(ctl)) ctl->ecnt.v = 0;
}

// ---------------------------------------------------------- counterexample --
//
// A lasso for a cycle verdict (the paper lists counterexample generation as
// missing): breadth-first search along rows (successors in G) with parent
// pointers, one level per launch.  parent[v] = NONE while v is unreached.

__global__ void k_fill(uint32_t *x, uint64_t len, uint32_t value)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) x[i] = value;
}

// one level: every row u of the frontier offers its successors; the first
// offer to reach an unreached vertex v sets parent[v] = u and queues v
__global__ void k_bfs_level(const uint32_t *__restrict__ front, const uint32_t *cnt_in, const uint32_t *__restrict__ rowptr,
                            const uint32_t *__restrict__ colidx, uint32_t *parent, uint32_t *next, uint32_t *cnt_out,
                            uint32_t target, uint32_t *found)
{
    const uint32_t nf = *(volatile const uint32_t *)cnt_in;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += stride) {
        const uint32_t u = __ldg(front + i);
        const uint32_t b = __ldg(rowptr + u), e = __ldg(rowptr + u + 1);
        for (uint32_t j = b; j < e; ++j) {
            const uint32_t v = __ldg(colidx + j) & 0x7FFFFFFFu; // bit 31 is the accepting flag
            if (*(volatile uint32_t *)(parent + v) != NONE) continue;
            if (atomicCAS(parent + v, NONE, u) == NONE) {
                next[atomicAdd(cnt_out, 1u)] = v;
                if (v == target) *found = 1;
            }
        }
    }
}

// the path source -> ... -> target, walked back from target along parents (one
// thread); out[0..len) holds it reversed; at most cap vertices, at most limit steps
__global__ void k_walk_back(const uint32_t *__restrict__ parent, uint32_t source, uint32_t target, uint32_t *out,
                            uint32_t cap, uint32_t limit, uint32_t *len)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint32_t k = 0, v = target;
    out[k++] = v;
    for (uint32_t steps = 0; steps < limit; ++steps) {
        v = parent[v];
        if (v == NONE || k >= cap) {
            k = 0xFFFFFFFFu; // broken chain or no room
            break;
        }
        out[k++] = v;
        if (v == source) break;
    }
    *len = k;
}

// ------------------------------------------------ accepting-part reduction --
//
// The paper builds its matrix only over the states in components that hold
// accepting states (the property automaton's components, after Lafuente).
// Every accepting cycle lies on a path from an accepting vertex to an
// accepting vertex, inside one component when the caller labels vertices by
// component (part[v]).  Kept = vertices reachable from an accepting vertex
// and reaching one (by >= 0 edges whose ends share a label); the reduced
// graph is the subgraph they induce, renumbered in increasing order.

// seeds: every accepting vertex gets `bit` in mark[] and is queued
__global__ void k_reach_seed(uint32_t n, const uint32_t *__restrict__ acc0, uint32_t *mark, uint32_t bit, uint32_t *q,
                             unsigned int *cnt)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < n; base += stride) { // warp-uniform
        const uint64_t v = base + threadIdx.x;
        const bool a = v < n && ((__ldg(acc0 + (v >> 5)) >> (v & 31u)) & 1u);
        if (a) mark[v] |= bit;
        const unsigned mask = __ballot_sync(0xFFFFFFFFu, a);
        if (!mask) continue;
        unsigned b = 0;
        if (lane_id() == 0) b = atomicAdd(cnt, __popc(mask));
        b = __shfl_sync(0xFFFFFFFFu, b, 0);
        if (a) q[b + __popc(mask & ((1u << lane_id()) - 1u))] = (uint32_t)v;
    }
}

// level-synchronous reachability from the queued seeds, all levels in one
// cooperative launch: lists by level mod 3 (q + (l % 3) * n), counters
// ctl->lcnt[l % 3].  Along rows of (ptr, col) -- successors for the forward
// sweep, readers for the backward one -- masking bit 31 of col.
__global__ void __launch_bounds__(256) k_reach(uint32_t n, const uint32_t *__restrict__ ptr,
                                               const uint32_t *__restrict__ col, const uint32_t *__restrict__ part,
                                               uint32_t *mark, uint32_t bit, uint32_t *q, Ctl *ctl)
{
    __shared__ uint32_t s_buf[8][SB_ENTRIES];
    __shared__ uint32_t s_cnt[8][1];
    __shared__ uint32_t s_base[1];
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint32_t status = ST_OK;
    for (uint32_t l = 0; l <= n; ++l) {
        const uint32_t nf = *(volatile uint32_t *)&ctl->lcnt[l % 3].v;
        if (nf == 0) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) ctl->lcnt[(l + 2) % 3].v = 0; // read in level l - 1
        const uint32_t *qin = q + (uint64_t)(l % 3) * n;
        uint32_t *qout = q + (uint64_t)((l + 1) % 3) * n;
        uint32_t *const dst[1][2] = {{qout, nullptr}};
        unsigned int *const ctr[1] = {&ctl->lcnt[(l + 1) % 3].v};
        Stage<1> st{&s_buf[warp][0], {0}};
        for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + warp * 32; base < nf; base += stride) {
            const uint64_t i = base + lane;
            uint32_t u = 0, b = 0, e = 0;
            if (i < nf) {
                u = qin[i];
                b = __ldg(ptr + u);
                e = __ldg(ptr + u + 1);
            }
            const uint32_t pu = (part && i < nf) ? __ldg(part + u) : 0;
            const uint32_t len = e - b, most = __reduce_max_sync(0xFFFFFFFFu, len);
            for (uint32_t k = 0; k < most; ++k) {
                bool fresh = false;
                uint32_t v = 0;
                if (k < len) {
                    v = __ldg(col + b + k) & 0x7FFFFFFFu;
                    if ((!part || __ldg(part + v) == pu) && !(*(volatile uint32_t *)(mark + v) & bit))
                        fresh = !(atomicOr(mark + v, bit) & bit);
                }
                stage_append<1>(st, 0, fresh, v, dst, ctr);
            }
        }
        stage_flush_block<1>(st, s_cnt, s_base, dst, ctr);
        if (!grid_barrier(ctl)) {
            status = ST_TIMEOUT;
            break;
        }
    }
    if (status != ST_OK && blockIdx.x == 0 && threadIdx.x == 0) ctl->status = status;
}

// keep[v] = both marks (3), as 0/1 words for the scan
__global__ void k_keep(uint32_t n, const uint32_t *__restrict__ mark, uint32_t *keep)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        keep[v] = (mark[v] & 3u) == 3u ? 1u : 0u;
}

// rank = inclusive scan of keep: kept v becomes rank[v] - 1.  pass 0: the row
// lengths of the reduced graph into rp[1 + new id]; pass 1: the rows into col_out
// (in the original order), the original ids and the accepting bits.
template <int PASS>
__global__ void k_reduce_rows(uint32_t n, const uint32_t *__restrict__ rowptr, const uint32_t *__restrict__ col,
                              const uint32_t *__restrict__ part, const uint32_t *__restrict__ mark,
                              const uint32_t *__restrict__ rank, const uint32_t *__restrict__ acc0, uint32_t *rp,
                              uint32_t *col_out, uint32_t *ids, uint32_t *acc_out)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        if ((mark[u] & 3u) != 3u) continue;
        const uint32_t nu = rank[u] - 1, pu = part ? __ldg(part + u) : 0;
        const uint32_t b = __ldg(rowptr + u), e = __ldg(rowptr + u + 1);
        uint32_t k = PASS ? rp[nu] : 0;
        for (uint32_t j = b; j < e; ++j) {
            const uint32_t v = __ldg(col + j) & 0x7FFFFFFFu;
            if ((mark[v] & 3u) != 3u || (part && __ldg(part + v) != pu)) continue;
            if (PASS) col_out[k] = rank[v] - 1;
            ++k;
        }
        if (!PASS) {
            rp[1 + (uint64_t)nu] = k;
        } else {
            ids[nu] = (uint32_t)u;
            if ((__ldg(acc0 + (u >> 5)) >> (u & 31u)) & 1u) atomicOr(acc_out + (nu >> 5), 1u << (nu & 31u));
        }
    }
}

__global__ void k_iota(uint32_t n, uint32_t *x)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) x[v] = (uint32_t)v;
}

// colidx without the accepting flags (export)
__global__ void k_unflag(uint64_t m, const uint32_t *__restrict__ col, uint32_t *out)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride)
        out[j] = __ldg(col + j) & 0x7FFFFFFFu;
}

// ------------------------------------------------------- on-the-fly growth --
//
// A growing graph (the paper's detection on the part of the matrix computed so
// far): rows [0, r) are expanded, rows [r, n) still empty.  An append copies
// the next k rows to rowptr[r .. r + k] (relative to the chunk) and adds n_add
// vertices; these kernels shift the chunk to the end of the edge array and
// assemble the accepting bitmap.

// rowptr[r .. r + k] hold the chunk's offsets: add m0; rows past them are empty
__global__ void k_grow_rowptr(uint32_t *rowptr, uint32_t r, uint32_t k, uint32_t n2, uint32_t m0, uint32_t m2)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)r + blockIdx.x * blockDim.x + threadIdx.x; i <= n2; i += stride)
        rowptr[i] = (k && i - r <= k) ? rowptr[i] + m0 : m2;
}

// out (ceil(n2 / 32) words) = bits [0, n0) of old, then bits [0, n_add) of add
__global__ void k_grow_acc(uint32_t *out, uint32_t words2, const uint32_t *__restrict__ old, uint32_t n0,
                           const uint32_t *__restrict__ add, uint32_t n_add)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t n2 = (uint64_t)n0 + n_add;
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words2; w += stride) {
        uint32_t x = 0;
        for (uint32_t t = 0; t < 32; ++t) {
            const uint64_t b = w * 32 + t;
            uint32_t bit = 0;
            if (b < n0) bit = (__ldg(old + (b >> 5)) >> (b & 31u)) & 1u;
            else if (b < n2) bit = (__ldg(add + ((b - n0) >> 5)) >> ((b - n0) & 31u)) & 1u;
            x |= bit << t;
        }
        out[w] = x;
    }
}

// ---------------------------------------------------------------- set-up --

// CSR validation: rowptr non-decreasing, every colidx < n.
__global__ void k_validate(uint32_t n, const uint32_t *__restrict__ rowptr, uint64_t m,
                           const uint32_t *__restrict__ colidx, uint32_t *bad)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    bool b = false;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        b |= __ldg(rowptr + i) > __ldg(rowptr + i + 1);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
        b |= __ldg(colidx + i) >= n;
    if (__any_sync(0xFFFFFFFFu, b) && lane_id() == 0) *bad = 1;
}

// Set-up in one pass over the CSR (map_create): rowptr must not decrease; every entry u < n is
// counted in the in-degree histogram (cnt[u + 1]) and gets the accepting flag of u (bitmap acc)
// in bit 31; an entry u >= n sets *bad instead (the graph is then refused, and nothing built
// from it is used).  Four entries per thread and step (one 128-bit load and store).
__device__ __forceinline__ uint32_t ingest_one(uint32_t u, uint32_t n, const uint32_t *__restrict__ acc, uint32_t *cnt,
                                               bool &bad, uint32_t &rank)
{
    if (u >= n) {
        bad = true;
        rank = 0;
        return u;
    }
    rank = atomicAdd(cnt + u + 1, 1u);
    return u | (((__ldg(acc + (u >> 5)) >> (u & 31u)) & 1u) << 31);
}

// Reads rowptr_in and colidx_in and, where the _out array is given (not null), writes the
// result there: the ingest pass is then also the copy from the caller's array (device memory, or
// page-locked host memory read over the host link). colidx_in and colidx_out 16-byte aligned
// (they may be the same array); the inputs are read once each. rank[i] = the number of entries
// before entry i that hold the same vertex (the count each one's increment returned: entry i's
// place in that vertex's reader list, in an arbitrary but fixed order); *long_rows is set when
// some row holds two entries or more.
__global__ void k_ingest(uint32_t n, const uint32_t *rowptr_in, uint32_t *rowptr_out, uint64_t m,
                         const uint32_t *colidx_in, uint32_t *colidx_out, const uint32_t *__restrict__ acc,
                         uint32_t *cnt, uint32_t *rank, uint32_t *bad, uint32_t *long_rows)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned lane = lane_id();
    bool b = false, lr = false;
    // rowptr[0..n]: warp-uniform steps of 32 entries; a lane's successor entry comes from the next
    // lane (lane 31 loads it)
    for (uint64_t i0 = tid - lane; i0 <= n; i0 += stride) {
        const uint64_t i = i0 + lane;
        const uint32_t a = i <= n ? rowptr_in[i] : 0u;
        uint32_t next = __shfl_down_sync(0xFFFFFFFFu, a, 1);
        if (lane == 31 && i < n) next = rowptr_in[i + 1];
        if (i < n) {
            b |= a > next;
            lr |= next - a > 1u;
        }
        if (rowptr_out && i <= n) rowptr_out[i] = a;
    }
    const uint64_t m4 = m / 4;
    const uint4 *c4 = reinterpret_cast<const uint4 *>(colidx_in);
    uint4 *o4 = reinterpret_cast<uint4 *>(colidx_out);
    uint4 *r4 = reinterpret_cast<uint4 *>(rank);
    for (uint64_t q = tid; q < m4; q += stride) {
        uint4 w = c4[q], r;
        w.x = ingest_one(w.x, n, acc, cnt, b, r.x);
        w.y = ingest_one(w.y, n, acc, cnt, b, r.y);
        w.z = ingest_one(w.z, n, acc, cnt, b, r.z);
        w.w = ingest_one(w.w, n, acc, cnt, b, r.w);
        o4[q] = w;
        r4[q] = r;
    }
    for (uint64_t i = m4 * 4 + tid; i < m; i += stride) colidx_out[i] = ingest_one(colidx_in[i], n, acc, cnt, b, rank[i]);
    if (__any_sync(0xFFFFFFFFu, b) && lane == 0) *bad = 1;
    if (__any_sync(0xFFFFFFFFu, lr) && lane == 0) *long_rows = 1;
}

// Reverse CSR scatter from the ranks k_ingest recorded: entry i of row w holding u goes to slot
// rrowptr[u] + rank[i] (rrowptr[u] = the start of u's reader list), with no atomics. A block takes a
// tile of TT_ROWS consecutive rows (grid-stride over tiles), puts the tile's row starts in shared
// memory and walks the tile's contiguous entry range with every thread, TT_E entries per thread in
// flight, finding an entry's row by binary search there: every lane has work whatever the
// degrees, and colidx and rank are read coalesced. Requires a validated CSR.
constexpr uint32_t TT_ROWS = 256;
constexpr int TT_E = 4;

__global__ void __launch_bounds__(256) k_transpose_ranked(uint32_t n, const uint32_t *__restrict__ rowptr,
                                                          const uint32_t *__restrict__ colidx,
                                                          const uint32_t *__restrict__ rank,
                                                          const uint32_t *__restrict__ rrowptr, uint32_t *rcol,
                                                          uint32_t *rpos)
{
    __shared__ uint32_t rs[TT_ROWS + 1];
    const uint32_t tiles = (uint32_t)(((uint64_t)n + TT_ROWS - 1) / TT_ROWS);
    for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const uint32_t r0 = t * TT_ROWS;
        const uint32_t nr = min(TT_ROWS, n - r0);
        __syncthreads(); // the previous tile's searches are done
        for (uint32_t k = threadIdx.x; k <= nr; k += blockDim.x) rs[k] = __ldg(rowptr + r0 + k);
        __syncthreads();
        const uint64_t e1 = rs[nr];
        for (uint64_t base = rs[0]; base < e1; base += (uint64_t)blockDim.x * TT_E) {
            uint32_t slot[TT_E];
#pragma unroll
            for (int j = 0; j < TT_E; ++j) {
                const uint64_t i = base + (uint64_t)j * blockDim.x + threadIdx.x;
                slot[j] = i < e1 ? __ldg(rrowptr + (__ldg(colidx + i) & 0x7FFFFFFFu)) + __ldg(rank + i) : 0u;
            }
#pragma unroll
            for (int j = 0; j < TT_E; ++j) {
                const uint64_t i = base + (uint64_t)j * blockDim.x + threadIdx.x;
                if (i >= e1) continue;
                uint32_t lo = 0, hi = nr; // rs[lo] <= i < rs[hi]
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (rs[mid] <= (uint32_t)i) lo = mid;
                    else hi = mid;
                }
                rcol[slot[j]] = r0 + lo;
                rpos[slot[j]] = (uint32_t)i;
            }
        }
    }
}

// in-degree histogram: cnt[u + 1] += 1 for every edge into u
__global__ void k_indegree(uint64_t m, const uint32_t *__restrict__ colidx, uint32_t *cnt)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
        atomicAdd(cnt + __ldg(colidx + i) + 1, 1u);
}

// block-wise inclusive scan of 1024-element tiles; tile totals into `sums`
__global__ void __launch_bounds__(1024) k_scan_tiles(uint32_t *x, uint64_t len, uint32_t *sums)
{
    __shared__ uint32_t warp_tot[32];
    const uint64_t i = (uint64_t)blockIdx.x * 1024 + threadIdx.x;
    uint32_t v = i < len ? x[i] : 0;
    const unsigned lane = lane_id(), w = threadIdx.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, off);
        if (lane >= (unsigned)off) v += t;
    }
    if (lane == 31) warp_tot[w] = v;
    __syncthreads();
    if (w == 0) {
        uint32_t s = warp_tot[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, s, off);
            if (lane >= (unsigned)off) s += t;
        }
        warp_tot[lane] = s;
    }
    __syncthreads();
    if (w > 0) v += warp_tot[w - 1];
    if (i < len) x[i] = v;
    if (threadIdx.x == 1023 && sums) sums[blockIdx.x] = v;
}

// add the scanned total of the preceding tiles
__global__ void k_scan_add(uint32_t *x, uint64_t len, const uint32_t *__restrict__ sums)
{
    const uint64_t i = (uint64_t)blockIdx.x * 1024 + threadIdx.x;
    if (blockIdx.x > 0 && i < len) x[i] += sums[blockIdx.x - 1];
}

// transpose scatter: the group of row w appends w (and the entry's position) to
// the reader list of each u in row w
template <int G>
__global__ void __launch_bounds__(256) k_transpose(uint32_t n, const uint32_t *__restrict__ rowptr,
                                                   const uint32_t *__restrict__ colidx, uint32_t *cursor,
                                                   uint32_t *rcol, uint32_t *rpos)
{
    const unsigned glane = threadIdx.x & (G - 1);
    const uint64_t groups = (uint64_t)gridDim.x * blockDim.x / G;
    for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; w < n; w += groups) {
        const uint32_t b = __ldg(rowptr + w), e = __ldg(rowptr + w + 1);
        for (uint32_t i = b + glane; i < e; i += G) {
            const uint32_t u = __ldg(colidx + i) & 0x7FFFFFFFu; // (bit 31: the accepting flag, when packed already)
            const uint32_t slot = atomicAdd(cursor + u, 1u);
            rcol[slot] = (uint32_t)w;
            rpos[slot] = i;
        }
    }
}

// ---- batched set-up ------------------------------------------------------

// x[i] += delta for i < len
__global__ void k_add(uint32_t *x, uint64_t len, uint32_t delta)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) x[i] += delta;
}

// comp[v] = the graph whose vertex range [off[c], off[c+1]) holds v
__global__ void k_fill_comp(uint32_t n, const uint32_t *__restrict__ off, uint32_t count, uint32_t *comp)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        uint32_t lo = 0, hi = count; // off[lo] <= v < off[hi]
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(off + mid) <= v) lo = mid;
            else hi = mid;
        }
        comp[v] = lo;
    }
}

// the union's accepting bitmap from the graphs' own bitmaps (staged one after
// another at word offsets woff[c]); one thread builds one union word
__global__ void k_gather_acc(uint32_t n, const uint32_t *__restrict__ off, const uint32_t *__restrict__ woff,
                             const uint32_t *__restrict__ staged, const uint32_t *__restrict__ comp, uint32_t *acc)
{
    const uint32_t words = (n + 31) / 32;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t wd = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; wd < words; wd += stride) {
        uint32_t x = 0;
        for (uint32_t b = 0; b < 32; ++b) {
            const uint32_t v = (uint32_t)wd * 32 + b;
            if (v >= n) break;
            const uint32_t c = __ldg(comp + v), i = v - __ldg(off + c);
            x |= ((__ldg(staged + __ldg(woff + c) + (i >> 5)) >> (i & 31u)) & 1u) << b;
        }
        acc[wd] = x;
    }
}

// accepting vertices per graph
__global__ void k_count_acc(uint32_t n, const uint32_t *__restrict__ acc, const uint32_t *__restrict__ comp,
                            CompState *cs)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n; base += stride) {
        const uint64_t v = base + lane_id();
        const bool a = v < n && ((__ldg(acc + (v >> 5)) >> (v & 31u)) & 1u);
        const uint32_t c = a ? __ldg(comp + v) : 0xFFFFFFFFu;
        const unsigned same = __match_any_sync(0xFFFFFFFFu, c);
        if (c != 0xFFFFFFFFu && lane_id() == (unsigned)(__ffs(same) - 1)) atomicAdd(&cs[c].nacc0, (unsigned)__popc(same));
    }
}

// put the accepting flag of each target into bit 31 of its matrix entry
__global__ void k_pack_flags(uint64_t m, uint32_t *colidx, const uint32_t *__restrict__ acc)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const uint32_t u = colidx[i];
        colidx[i] = u | ((__ldg(acc + (u >> 5)) >> (u & 31u)) << 31);
    }
}

// accepting bitmap: copy, clear the bits at or above n, count the set bits
__global__ void k_acc_init(uint32_t n, const uint32_t *__restrict__ in, uint32_t *acc0, unsigned int *count)
{
    const uint32_t words = (n + 31) / 32;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned c = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += stride) {
        uint32_t x = __ldg(in + i);
        if (i == words - 1 && (n & 31u)) x &= (1u << (n & 31u)) - 1u;
        acc0[i] = x;
        c += __popc(x);
    }
    c = __reduce_add_sync(0xFFFFFFFFu, c);
    if (lane_id() == 0 && c) atomicAdd(count, c);
}

} // namespace mapk
