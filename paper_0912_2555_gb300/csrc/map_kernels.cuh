// map_kernels.cuh -- sm_103a kernels of the MAP hot path (Section 2 of the paper).
//
// Device layout of one graph (all u32 unless noted):
//   rowptr[n+1], colidx[m]      the CSR handed in: row v = successors of v in G,
//                               i.e. the pull matrix of the transposed graph;
//   rrowptr[n+1], rcol[m]       its transpose: rcol[rrowptr[u] ..] are the
//                               readers of u (the rows that contain u);
//   acc[W], W = ceil(n/32)      the current accepting set, LSB-first bitmap;
//   mval[n]                     enc(map(v)): 0 = no value, u + 1 = vertex u;
//   fbits[2][W]                 frontier de-duplication, one bitmap per round parity;
//   queue[2][n]                 frontier of a round, by round parity;
//   chv[n], chval[n]            synchronous rounds: (vertex, new value) changes.
//   Ctl                         the control block below (one per graph).
//
// Every kernel that ends a step of the loop finishes with a last-block epilogue
// (the last block to retire, found with an atomic ticket) that updates the
// control block and, when the loop runs as a CUDA graph, sets the graph's
// conditional WHILE handles.  There are no spin-waits anywhere.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mapk {

namespace cg = cooperative_groups;

constexpr uint32_t NONE = 0xFFFFFFFFu;
constexpr uint32_t ST_OK = 0, ST_TIMEOUT = 5, ST_LIMIT = 6; // map_status values used on the device

struct Ctl {
    // fix-point loop
    uint32_t qcnt[2];      // |frontier| by round parity
    uint32_t ccnt;         // changes found in the current round
    uint32_t k;            // rounds completed in the current outer iteration
    // outer loop
    uint32_t outer;        // current outer iteration, 1-based (0: none ran)
    uint32_t inner_go;     // fix-point loop continues
    uint32_t outer_go;     // outer loop continues
    uint32_t status;       // ST_OK or ST_LIMIT
    uint32_t verdict;      // 1 = accepting cycle
    uint32_t witness;      // smallest self-mapped vertex of the last iteration
    uint32_t nonzero;      // some map value is defined (eliminated set not empty)
    uint32_t elim;         // accepting vertices eliminated in this outer iteration
    uint32_t nacc;         // accepting vertices left
    uint32_t nacc0;        // accepting vertices at the start
    uint32_t done;         // last-block ticket
    uint32_t max_outer;    // 0 = no limit
    uint32_t max_inner;    // rounds per outer iteration
    uint32_t hist_cap;     // entries of rounds_hist
    uint64_t m;            // edges
    uint64_t relax;        // edges examined
    uint64_t inner_total;  // rounds summed over outer iterations
    uint32_t *rounds_hist; // rounds of each outer iteration
    uint32_t *out;         // map export destination (device); NULL: the work buffer chv
    uint32_t use_graph;    // epilogues set the conditional handles
    uint32_t pad0;
    uint64_t t0;           // %globaltimer at the start of the run (ns)
    uint64_t timeout_ns;   // the loop stops with ST_TIMEOUT past t0 + timeout_ns
    uint32_t pad[4];
};

struct Handles {
    unsigned long long inner; // cudaGraphConditionalHandle of the fix-point WHILE node
    unsigned long long outer; // ... of the outer WHILE node
};

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

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

template <int G>
__device__ __forceinline__ uint32_t group_max(uint32_t x)
{
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) x = max(x, __shfl_xor_sync(0xFFFFFFFFu, x, off));
    return x;
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long x)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, off);
    return x;
}

// True in exactly one thread of the grid: thread 0 of the last block to get here.
// Every thread of every block must call it (it contains __syncthreads).
__device__ __forceinline__ bool last_block(Ctl *ctl)
{
    __shared__ bool is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(&ctl->done, 1u);
        is_last = (t == gridDim.x - 1);
        if (is_last) {
            ctl->done = 0;
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

__device__ __forceinline__ bool timed_out(volatile Ctl *v)
{
    return global_ns() - v->t0 > v->timeout_ns;
}

// After round 1 (the dense round) of an outer iteration.
__device__ void epilogue_dense(Ctl *c, Handles hd)
{
    volatile Ctl *v = c;
    const uint32_t changed = v->ccnt;
    v->ccnt = 0;
    v->k = 1;
    v->relax = v->relax + v->m;
    uint32_t go = changed ? 1u : 0u;
    if (go && v->max_inner < 2) {
        v->status = ST_LIMIT;
        go = 0;
    }
    if (v->status != ST_OK) go = 0;
    v->inner_go = go;
    __threadfence();
    set_cond(c, hd.inner, go);
}

// After round k + 1 >= 2 (compute + apply, or one asynchronous sweep).
__device__ void epilogue_round(Ctl *c, Handles hd)
{
    volatile Ctl *v = c;
    const uint32_t changed = v->ccnt;
    const uint32_t k = v->k + 1;          // the round just finished
    v->ccnt = 0;
    v->qcnt[k & 1] = 0;                   // its frontier is consumed
    v->k = k;
    uint32_t go = changed ? 1u : 0u;
    if (go && k + 1 > v->max_inner) {
        v->status = ST_LIMIT;
        go = 0;
    }
    if (go && timed_out(v)) {
        v->status = ST_TIMEOUT;
        go = 0;
    }
    v->inner_go = go;
    __threadfence();
    set_cond(c, hd.inner, go);
}

// After the self-map test and the elimination of an outer iteration.
__device__ void epilogue_check(Ctl *c, Handles hd)
{
    volatile Ctl *v = c;
    const uint32_t outer = v->outer, k = v->k;
    if (outer - 1 < v->hist_cap) c->rounds_hist[outer - 1] = k;
    v->inner_total = v->inner_total + k;
    uint32_t go = 1;
    if (v->status != ST_OK) {
        go = 0; // a limit was hit inside the fix-point loop
    } else if (v->witness != NONE) {
        v->verdict = 1;
        go = 0;
    } else if (!v->nonzero) {
        go = 0; // nothing reaches a remaining accepting vertex
    } else {
        const uint32_t left = v->nacc - v->elim;
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
    if (go) {
        v->outer = outer + 1;
        v->qcnt[0] = 0;
        v->qcnt[1] = 0;
        v->nonzero = 0;
        v->elim = 0;
        v->k = 0;
    }
    v->outer_go = go;
    __threadfence();
    set_cond(c, hd.outer, go);
}

// Start of a run: fields written by the host (max_outer, max_inner, out,
// hist_cap, m, nacc0, use_graph) are kept, the rest is reset.
__global__ void k_run_begin(Ctl *c, Handles hd)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    volatile Ctl *v = c;
    v->qcnt[0] = v->qcnt[1] = 0;
    v->ccnt = 0;
    v->k = 0;
    v->status = ST_OK;
    v->verdict = 0;
    v->witness = NONE;
    v->nonzero = 0;
    v->elim = 0;
    v->nacc = v->nacc0;
    v->done = 0;
    v->relax = 0;
    v->inner_total = 0;
    v->t0 = global_ns();
    const uint32_t go = v->nacc0 ? 1u : 0u;
    v->outer = go;
    v->outer_go = go;
    v->inner_go = 0;
    __threadfence();
    set_cond(c, hd.outer, go);
}

// Mark the readers of u for the next round: set their bit in `bits`; the lane
// that flips a bit from 0 to 1 appends the reader to `queue`.  The G lanes of a
// group split u's reader list.
template <int G>
__device__ __forceinline__ void mark_readers(uint32_t u, unsigned glane, const uint32_t *__restrict__ rrowptr,
                                             const uint32_t *__restrict__ rcol, uint32_t *bits, uint32_t *queue,
                                             unsigned int *qcnt)
{
    const uint32_t b = __ldg(rrowptr + u), e = __ldg(rrowptr + u + 1);
    for (uint32_t i = b + glane; i < e; i += G) {
        const uint32_t w = __ldg(rcol + i);
        const uint32_t bit = 1u << (w & 31u);
        if (*(volatile uint32_t *)(bits + (w >> 5)) & bit) continue; // read first: most re-marks stop here
        const uint32_t old = atomicOr(bits + (w >> 5), bit);
        if (!(old & bit)) queue[agg_inc(qcnt)] = w;
    }
}

// ------------------------------------------------------------ dense round --
//
// Round 1 of an outer iteration relaxes every row from "no value" everywhere,
// so the value u offers is u + 1 if u is accepting and 0 otherwise: only the
// accepting bitmap is gathered.
//
// Each warp owns tiles of WT_ROWS consecutive rows, with no block-wide phase:
// the tile's rowptr slice (fetched one tile ahead into registers) goes to a
// warp-private shared slice; the tile's edge span is streamed with 128-bit
// loads (WT_UNROLL per lane, then 4 * WT_UNROLL independent bitmap gathers);
// an edge that offers a value finds its row by binary search in the slice and
// does a shared-memory atomicMax; the tile's values are written out coalesced
// (this also resets the previous iteration's values) and the readers of every
// row that got a value are marked into the round-2 frontier.
constexpr int DT_THREADS = 256;
constexpr int WT_WARPS = DT_THREADS / 32;
constexpr int WT_ROWS = 128;
constexpr int WT_UNROLL = 4;
constexpr size_t DT_SMEM = 0; // static shared memory only

__global__ void __launch_bounds__(DT_THREADS, 4) k_dense(uint32_t n, const uint32_t *__restrict__ rowptr,
                                                         const uint32_t *__restrict__ colidx,
                                                         const uint32_t *__restrict__ acc,
                                                         uint32_t *__restrict__ mval,
                                                         const uint32_t *__restrict__ rrowptr,
                                                         const uint32_t *__restrict__ rcol, uint32_t *bits,
                                                         uint32_t *queue, Ctl *ctl, Handles hd)
{
    __shared__ __align__(16) uint32_t s_rp[WT_WARPS][WT_ROWS + 4];
    __shared__ __align__(16) uint32_t s_best[WT_WARPS][WT_ROWS];
    default_stop(ctl, hd.outer);
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    uint32_t *rp = s_rp[warp], *best = s_best[warp];
    const uint32_t ntiles = (n + WT_ROWS - 1) / WT_ROWS;
    const uint32_t nw = gridDim.x * WT_WARPS;
    unsigned changed = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) best[lane * 4 + k] = 0;

    // rowptr words r0 + 4 lane .. + 3 of tile t (only the words that exist: <= r0 + rows + 3)
    auto load_rp = [&](uint32_t t, uint4 &q, uint32_t &last) {
        const uint32_t r0 = t * WT_ROWS, rows = min((uint32_t)WT_ROWS, n - r0);
        q = lane * 4 <= rows ? __ldg(reinterpret_cast<const uint4 *>(rowptr + r0) + lane) : make_uint4(0, 0, 0, 0);
        last = (lane == 0 && rows == WT_ROWS) ? __ldg(rowptr + r0 + WT_ROWS) : 0;
    };
    uint32_t t = blockIdx.x * WT_WARPS + warp;
    uint4 q = make_uint4(0, 0, 0, 0);
    uint32_t qlast = 0;
    if (t < ntiles) load_rp(t, q, qlast);
    for (; t < ntiles; t += nw) {
        const uint32_t r0 = t * WT_ROWS, rows = min((uint32_t)WT_ROWS, n - r0);
        reinterpret_cast<uint4 *>(rp)[lane] = q;
        if (lane == 0 && rows == WT_ROWS) rp[WT_ROWS] = qlast;
        if (t + nw < ntiles) load_rp(t + nw, q, qlast); // next tile's slice, in flight meanwhile
        __syncwarp();
        const uint32_t E0 = rp[0], E1 = rp[rows];
        for (uint32_t cs = E0 & ~3u; cs < E1; cs += 32 * 4 * WT_UNROLL) {
            uint4 w[WT_UNROLL];
#pragma unroll
            for (int j = 0; j < WT_UNROLL; ++j) {
                const uint32_t idx = cs + (j * 32 + lane) * 4;
                w[j] = idx < E1 ? __ldg(reinterpret_cast<const uint4 *>(colidx + idx)) : make_uint4(0, 0, 0, 0);
            }
            uint32_t aw[WT_UNROLL][4];
#pragma unroll
            for (int j = 0; j < WT_UNROLL; ++j) {
                aw[j][0] = __ldg(acc + (w[j].x >> 5));
                aw[j][1] = __ldg(acc + (w[j].y >> 5));
                aw[j][2] = __ldg(acc + (w[j].z >> 5));
                aw[j][3] = __ldg(acc + (w[j].w >> 5));
            }
#pragma unroll
            for (int j = 0; j < WT_UNROLL; ++j) {
                const uint32_t ebase = cs + (j * 32 + lane) * 4;
                const uint32_t us[4] = {w[j].x, w[j].y, w[j].z, w[j].w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t e = ebase + k, u = us[k];
                    if (e >= E0 && e < E1 && ((aw[j][k] >> (u & 31u)) & 1u)) {
                        uint32_t lo = 0, hi = rows; // rp[lo] <= e < rp[hi]: the row of e is the last such lo
                        while (hi - lo > 1) {
                            const uint32_t mid = (lo + hi) >> 1;
                            if (rp[mid] <= e) lo = mid;
                            else hi = mid;
                        }
                        atomicMax(&best[lo], u + 1);
                    }
                }
            }
        }
        __syncwarp();
        const uint4 b4 = reinterpret_cast<const uint4 *>(best)[lane];
        const uint32_t bs[4] = {b4.x, b4.y, b4.z, b4.w};
        if (lane * 4 + 3 < rows) {
            reinterpret_cast<uint4 *>(mval + r0)[lane] = b4;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (lane * 4 + k < rows) mval[r0 + lane * 4 + k] = bs[k];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (bs[k] && lane * 4 + k < rows) {
                best[lane * 4 + k] = 0;
                changed++;
                mark_readers<1>(r0 + lane * 4 + k, 0, rrowptr, rcol, bits, queue, &ctl->qcnt[0]);
            }
        }
        __syncwarp();
    }
    changed = __reduce_add_sync(0xFFFFFFFFu, changed);
    if (lane == 0 && changed) atomicAdd(&ctl->ccnt, changed);
    if (last_block(ctl)) epilogue_dense(ctl, hd);
}

// ---------------------------------------------------------- frontier rounds --
//
// A frontier row is handled by a group of G consecutive lanes (G = 1 .. 32,
// picked from the mean degree): each lane takes every G-th edge of the row and
// the group reduces with xor-shuffles.  Loops run so that every lane of a warp
// makes the same number of iterations (full-mask shuffles).  The round number
// and the frontier size are read from the control block.

// Synchronous round, compute half: for every frontier row v, the new value
// max(mval[v], max over u in row v of max(u + 1 if u accepting, mval[u])) from
// the values of the previous round (mval is not written here).  Rows whose value
// grows are appended to the change list.  Clears the frontier's bitmap.
template <int G>
__global__ void __launch_bounds__(256, 6) k_sync_compute(const uint32_t *__restrict__ rowptr,
                                                      const uint32_t *__restrict__ colidx,
                                                      const uint32_t *__restrict__ acc,
                                                      const uint32_t *__restrict__ mval, uint32_t *queue,
                                                      uint32_t *fbits, uint32_t n, uint32_t words, uint32_t *chv,
                                                      uint32_t *chval, Ctl *ctl, Handles hd)
{
    default_stop(ctl, hd.inner);
    const uint32_t p = (*(volatile uint32_t *)&ctl->k + 1) & 1u;
    const uint32_t nfront = *(volatile uint32_t *)&ctl->qcnt[p];
    const uint32_t *front = queue + (size_t)p * n;
    uint32_t *front_bits = fbits + (size_t)p * words;
    const unsigned glane = threadIdx.x & (G - 1);
    const uint64_t groups = (uint64_t)gridDim.x * blockDim.x / G;
    const uint64_t gid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const uint64_t warp_first = gid - (lane_id() / G);
    unsigned long long relax = 0;
    for (uint64_t base = warp_first; base < nfront; base += groups) {
        const uint64_t i = base + lane_id() / G;
        uint32_t best = 0, own = 0, v = 0;
        if (i < nfront) {
            v = __ldg(front + i);
            own = __ldg(mval + v);
            const uint32_t b = __ldg(rowptr + v), e = __ldg(rowptr + v + 1);
            if (glane == 0) {
                relax += e - b;
                front_bits[v >> 5] = 0; // every bit of this bitmap belongs to this frontier
            }
            for (uint32_t j = b + glane; j < e; j += G) {
                const uint32_t u = __ldg(colidx + j);
                uint32_t off = __ldg(mval + u);
                if (acc_bit(acc, u)) off = max(off, u + 1);
                best = max(best, off);
            }
        }
        best = group_max<G>(best);
        if (i < nfront && glane == 0 && best > own) {
            const unsigned slot = agg_inc(&ctl->ccnt);
            chv[slot] = v;
            chval[slot] = best;
        }
    }
    relax = warp_sum64(relax);
    if (lane_id() == 0 && relax) atomicAdd((unsigned long long *)&ctl->relax, relax);
}

// Synchronous round, apply half: write the new values and mark the readers of
// every changed vertex into the frontier of the next round.
template <int G>
__global__ void __launch_bounds__(256, 8) k_sync_apply(const uint32_t *__restrict__ chv,
                                                    const uint32_t *__restrict__ chval, uint32_t *mval,
                                                    const uint32_t *__restrict__ rrowptr,
                                                    const uint32_t *__restrict__ rcol, uint32_t *queue, uint32_t *fbits,
                                                    uint32_t n, uint32_t words, Ctl *ctl, Handles hd)
{
    const uint32_t np = *(volatile uint32_t *)&ctl->k & 1u; // parity of the round after this one
    const uint32_t nch = *(volatile uint32_t *)&ctl->ccnt;
    uint32_t *next = queue + (size_t)np * n;
    uint32_t *nbits = fbits + (size_t)np * words;
    const unsigned glane = threadIdx.x & (G - 1);
    const uint64_t groups = (uint64_t)gridDim.x * blockDim.x / G;
    const uint64_t gid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const uint64_t warp_first = gid - (lane_id() / G);
    for (uint64_t base = warp_first; base < nch; base += groups) {
        const uint64_t i = base + lane_id() / G;
        if (i < nch) {
            const uint32_t v = chv[i];
            if (glane == 0) mval[v] = chval[i];
            mark_readers<G>(v, glane, rrowptr, rcol, nbits, next, &ctl->qcnt[np]);
        }
    }
    if (last_block(ctl)) epilogue_round(ctl, hd);
}

// Asynchronous sweep: like a synchronous round, but a new value is written at
// once (values only grow, so a racing reader sees the old or the new value and
// the fix-point is the same), and its readers are marked at once.
template <int G>
__global__ void __launch_bounds__(256, 6) k_async_sweep(const uint32_t *__restrict__ rowptr,
                                                     const uint32_t *__restrict__ colidx,
                                                     const uint32_t *__restrict__ acc, uint32_t *mval,
                                                     const uint32_t *__restrict__ rrowptr,
                                                     const uint32_t *__restrict__ rcol, uint32_t *queue,
                                                     uint32_t *fbits, uint32_t n, uint32_t words, Ctl *ctl,
                                                     Handles hd)
{
    default_stop(ctl, hd.inner);
    const uint32_t p = (*(volatile uint32_t *)&ctl->k + 1) & 1u, np = p ^ 1u;
    const uint32_t nfront = *(volatile uint32_t *)&ctl->qcnt[p];
    const uint32_t *front = queue + (size_t)p * n;
    uint32_t *front_bits = fbits + (size_t)p * words;
    uint32_t *next = queue + (size_t)np * n;
    uint32_t *nbits = fbits + (size_t)np * words;
    const unsigned glane = threadIdx.x & (G - 1);
    const uint64_t groups = (uint64_t)gridDim.x * blockDim.x / G;
    const uint64_t gid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const uint64_t warp_first = gid - (lane_id() / G);
    unsigned long long relax = 0;
    unsigned changed = 0;
    for (uint64_t base = warp_first; base < nfront; base += groups) {
        const uint64_t i = base + lane_id() / G;
        uint32_t best = 0, own = 0, v = 0;
        if (i < nfront) {
            v = __ldg(front + i);
            own = *(volatile uint32_t *)(mval + v);
            const uint32_t b = __ldg(rowptr + v), e = __ldg(rowptr + v + 1);
            if (glane == 0) {
                relax += e - b;
                front_bits[v >> 5] = 0;
            }
            for (uint32_t j = b + glane; j < e; j += G) {
                const uint32_t u = __ldg(colidx + j);
                uint32_t off = *(volatile uint32_t *)(mval + u);
                if (acc_bit(acc, u)) off = max(off, u + 1);
                best = max(best, off);
            }
        }
        best = group_max<G>(best);
        if (i < nfront && best > own) {
            if (glane == 0) {
                atomicMax(mval + v, best);
                changed++;
            }
            mark_readers<G>(v, glane, rrowptr, rcol, nbits, next, &ctl->qcnt[np]);
        }
    }
    relax = warp_sum64(relax);
    changed = __reduce_add_sync(0xFFFFFFFFu, changed);
    if (lane_id() == 0) {
        if (relax) atomicAdd((unsigned long long *)&ctl->relax, relax);
        if (changed) atomicAdd(&ctl->ccnt, changed);
    }
    if (last_block(ctl)) epilogue_round(ctl, hd);
}

// ------------------------------------------------- self-map test, elimination --
//
// One pass over the map vector (Section 2): witness = smallest v with
// map(v) = v; every defined map value u is removed from the accepting set
// (exact count of removals); nonzero = "some value is defined".  The map vector
// is left intact (the next dense round overwrites it).  128-bit loads, four
// words per thread per step.
__global__ void __launch_bounds__(256) k_check_eliminate(uint32_t n, const uint32_t *__restrict__ mval,
                                                         uint32_t *acc, Ctl *ctl, Handles hd)
{
    const uint32_t n4 = (n + 3) / 4;
    const uint32_t stride = gridDim.x * blockDim.x;
    unsigned elim = 0, any = 0;
    uint32_t wit = NONE;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const uint4 x4 = __ldg(reinterpret_cast<const uint4 *>(mval) + i);
        const uint32_t xs[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t v = i * 4 + q;
            const uint32_t x = xs[q];
            if (v >= n || !x) continue;
            any = 1;
            const uint32_t u = x - 1;
            if (u == v) wit = min(wit, u);
            const uint32_t bit = 1u << (u & 31u);
            if (*(volatile uint32_t *)(acc + (u >> 5)) & bit) {
                const uint32_t old = atomicAnd(acc + (u >> 5), ~bit);
                elim += (old & bit) ? 1u : 0u;
            }
        }
    }
    elim = __reduce_add_sync(0xFFFFFFFFu, elim);
    any = __reduce_or_sync(0xFFFFFFFFu, any);
    wit = __reduce_min_sync(0xFFFFFFFFu, wit);
    if (lane_id() == 0) {
        if (elim) atomicAdd(&ctl->elim, elim);
        if (any) atomicOr(&ctl->nonzero, 1u);
        if (wit != NONE) atomicMin(&ctl->witness, wit);
    }
    if (last_block(ctl)) epilogue_check(ctl, hd);
}

// External encoding into `dst` (NULL: ctl->out): MAP_NONE for no value, else
// the vertex id; all MAP_NONE when no outer iteration ran.
__global__ void k_export(uint32_t n, const uint32_t *__restrict__ mval, const Ctl *ctl, uint32_t *dst)
{
    uint32_t *out = dst ? dst : ctl->out;
    const bool none = ctl->outer == 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        out[v] = none ? NONE : __ldg(mval + v) - 1u;
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

// transpose scatter: the group of row w appends w to the reader list of each u in row w
template <int G>
__global__ void __launch_bounds__(256) k_transpose(uint32_t n, const uint32_t *__restrict__ rowptr,
                                                   const uint32_t *__restrict__ colidx, uint32_t *cursor,
                                                   uint32_t *rcol)
{
    const unsigned glane = threadIdx.x & (G - 1);
    const uint64_t groups = (uint64_t)gridDim.x * blockDim.x / G;
    for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; w < n; w += groups) {
        const uint32_t b = __ldg(rowptr + w), e = __ldg(rowptr + w + 1);
        for (uint32_t i = b + glane; i < e; i += G) {
            const uint32_t u = __ldg(colidx + i);
            rcol[atomicAdd(cursor + u, 1u)] = (uint32_t)w;
        }
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
