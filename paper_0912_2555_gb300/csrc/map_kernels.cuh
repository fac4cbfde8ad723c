// map_kernels.cuh -- sm_103a kernels of the MAP hot path (Section 2 of the paper).
//
// Device layout of one graph (all u32):
//   rowptr[n+1], colidx[m]      the CSR handed in: row v = successors of v in G,
//                               i.e. the pull matrix of the transposed graph;
//   rrowptr[n+1], rcol[m]       its transpose: rcol[rrowptr[u] ..] are the
//                               readers of u (the rows that contain u);
//   acc[W], W = ceil(n/32)      the current accepting set, LSB-first bitmap;
//   mval[n]                     enc(map(v)): 0 = no value, u + 1 = vertex u;
//   fbits[2][W]                 frontier de-duplication, one bitmap per round parity;
//   queue[2][n]                 frontier of the next round, by round parity;
//   chv[n], chval[n]            synchronous rounds: (vertex, new value) changes.
//
// A row is handled by a group of G consecutive lanes (G = 1 .. 32, picked from
// the mean degree): each lane takes every G-th edge of the row, and the group
// reduces with xor-shuffles.  All kernels are grid-stride loops in which every
// lane of a warp runs the same number of iterations, so the full-mask shuffles
// are always reached by the whole warp.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mapk {

namespace cg = cooperative_groups;

struct Ctl {                       // device control block of one graph
    unsigned int qcnt[2];          // |frontier| by round parity
    unsigned int ccnt;             // changes found in the current round
    unsigned int witness;          // smallest self-mapped vertex (0xFFFFFFFF: none)
    unsigned int nonzero;          // 1 if some map value is defined
    unsigned int elim;             // accepting vertices eliminated in this outer iteration
    unsigned int bad;              // validation failure
    unsigned int pad0;
    unsigned long long relax;      // edges examined by the frontier rounds
    unsigned long long pad1[3];
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

template <int G>
__device__ __forceinline__ unsigned long long group_sum64(unsigned long long x)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, off);
    return x;
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
        if (bits[w >> 5] & bit) continue; // read first: most re-marks stop here
        const uint32_t old = atomicOr(bits + (w >> 5), bit);
        if (!(old & bit)) queue[agg_inc(qcnt)] = w;
    }
}

// Round 1 of an outer iteration: every row, from "no value" everywhere, so the
// value offered by u is u + 1 if u is accepting and 0 otherwise.  Writes every
// mval[v] (this is also the reset of the previous iteration's values) and marks
// the readers of every vertex that got a value into the round-2 frontier.
template <int G>
__global__ void __launch_bounds__(256) k_dense(uint32_t n, const uint32_t *__restrict__ rowptr,
                                               const uint32_t *__restrict__ colidx, const uint32_t *__restrict__ acc,
                                               uint32_t *__restrict__ mval, const uint32_t *__restrict__ rrowptr,
                                               const uint32_t *__restrict__ rcol, uint32_t *bits, uint32_t *queue,
                                               Ctl *ctl, unsigned int *qcnt)
{
    const unsigned glane = threadIdx.x & (G - 1);
    const uint64_t groups = (uint64_t)gridDim.x * blockDim.x / G;
    const uint64_t gid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    // iterate so that all lanes of a warp run the same number of iterations
    const uint64_t warp_first = gid - (lane_id() / G);
    unsigned changed = 0;
    for (uint64_t base = warp_first; base < n; base += groups) {
        const uint64_t v = base + lane_id() / G;
        uint32_t best = 0;
        if (v < n) {
            const uint32_t b = __ldg(rowptr + v), e = __ldg(rowptr + v + 1);
            for (uint32_t i = b + glane; i < e; i += G) {
                const uint32_t u = __ldg(colidx + i);
                if (acc_bit(acc, u)) best = max(best, u + 1);
            }
        }
        best = group_max<G>(best);
        if (v < n) {
            if (glane == 0) mval[v] = best;
            if (best) {
                changed += (glane == 0);
                mark_readers<G>((uint32_t)v, glane, rrowptr, rcol, bits, queue, qcnt);
            }
        }
    }
    changed = __reduce_add_sync(0xFFFFFFFFu, changed);
    if (lane_id() == 0 && changed) atomicAdd(&ctl->ccnt, changed);
}

// Synchronous round k >= 2, compute half: for every frontier row v, the new
// value max(mval[v], max over u in row v of max(u + 1 if u accepting, mval[u]))
// from the values of round k-1 (mval is not written here).  Rows whose value
// grows are appended to the change list.  Clears the frontier's bitmap.
template <int G>
__global__ void __launch_bounds__(256) k_sync_compute(const uint32_t *__restrict__ front, uint32_t nfront,
                                                      const uint32_t *__restrict__ rowptr,
                                                      const uint32_t *__restrict__ colidx,
                                                      const uint32_t *__restrict__ acc,
                                                      const uint32_t *__restrict__ mval, uint32_t *front_bits,
                                                      uint32_t *chv, uint32_t *chval, Ctl *ctl)
{
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
    relax = group_sum64<G>(relax);
    if (lane_id() == 0 && relax) atomicAdd(&ctl->relax, relax);
}

// Synchronous round k >= 2, apply half: write the new values and mark the
// readers of every changed vertex into the frontier of round k+1.
template <int G>
__global__ void __launch_bounds__(256) k_sync_apply(const uint32_t *__restrict__ chv,
                                                    const uint32_t *__restrict__ chval, const Ctl *ctl_ro,
                                                    uint32_t *mval, const uint32_t *__restrict__ rrowptr,
                                                    const uint32_t *__restrict__ rcol, uint32_t *bits, uint32_t *queue,
                                                    unsigned int *qcnt)
{
    const uint32_t nch = *(volatile const unsigned int *)&ctl_ro->ccnt;
    const unsigned glane = threadIdx.x & (G - 1);
    const uint64_t groups = (uint64_t)gridDim.x * blockDim.x / G;
    const uint64_t gid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const uint64_t warp_first = gid - (lane_id() / G);
    for (uint64_t base = warp_first; base < nch; base += groups) {
        const uint64_t i = base + lane_id() / G;
        if (i < nch) {
            const uint32_t v = chv[i];
            if (glane == 0) mval[v] = chval[i];
            mark_readers<G>(v, glane, rrowptr, rcol, bits, queue, qcnt);
        }
    }
}

// Asynchronous sweep: like a synchronous round, but the new value is written at
// once (values only grow, so a racing reader sees either the old or the new
// value; either way the fix-point is the same), and readers are marked at once.
template <int G>
__global__ void __launch_bounds__(256) k_async_sweep(const uint32_t *__restrict__ front, uint32_t nfront,
                                                     const uint32_t *__restrict__ rowptr,
                                                     const uint32_t *__restrict__ colidx,
                                                     const uint32_t *__restrict__ acc, uint32_t *mval,
                                                     uint32_t *front_bits, const uint32_t *__restrict__ rrowptr,
                                                     const uint32_t *__restrict__ rcol, uint32_t *bits,
                                                     uint32_t *queue, unsigned int *qcnt, Ctl *ctl)
{
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
            mark_readers<G>(v, glane, rrowptr, rcol, bits, queue, qcnt);
        }
    }
    relax = group_sum64<G>(relax);
    changed = __reduce_add_sync(0xFFFFFFFFu, changed);
    if (lane_id() == 0) {
        if (relax) atomicAdd(&ctl->relax, relax);
        if (changed) atomicAdd(&ctl->ccnt, changed);
    }
}

// Self-map test and elimination (Section 2), one pass over the map vector:
// witness = smallest v with map(v) = v; every defined map value u is removed
// from the accepting set (exact count of removals); nonzero = "some value is
// defined".  The map vector itself is left intact (the next dense round
// overwrites it).
__global__ void __launch_bounds__(256) k_check_eliminate(uint32_t n, const uint32_t *__restrict__ mval,
                                                         uint32_t *acc, Ctl *ctl)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned elim = 0, any = 0;
    uint32_t wit = 0xFFFFFFFFu;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint32_t x = __ldg(mval + v);
        if (!x) continue;
        any = 1;
        const uint32_t u = x - 1;
        if (u == v) wit = min(wit, u);
        const uint32_t bit = 1u << (u & 31u);
        if (*(volatile uint32_t *)(acc + (u >> 5)) & bit) {
            const uint32_t old = atomicAnd(acc + (u >> 5), ~bit);
            elim += (old & bit) ? 1u : 0u;
        }
    }
    elim = __reduce_add_sync(0xFFFFFFFFu, elim);
    any = __reduce_or_sync(0xFFFFFFFFu, any);
    wit = __reduce_min_sync(0xFFFFFFFFu, wit);
    if (lane_id() == 0) {
        if (elim) atomicAdd(&ctl->elim, elim);
        if (any) ctl->nonzero = 1;
        if (wit != 0xFFFFFFFFu) atomicMin(&ctl->witness, wit);
    }
}

// external encoding: MAP_NONE (0xFFFFFFFF) for no value, else the vertex id
__global__ void k_export(uint32_t n, const uint32_t *__restrict__ mval, uint32_t *out)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) out[v] = __ldg(mval + v) - 1u;
}

// ---------------------------------------------------------------- set-up --

// CSR validation: rowptr non-decreasing, every colidx < n.
__global__ void k_validate(uint32_t n, const uint32_t *__restrict__ rowptr, uint64_t m,
                           const uint32_t *__restrict__ colidx, Ctl *ctl)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        bad |= __ldg(rowptr + i) > __ldg(rowptr + i + 1);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
        bad |= __ldg(colidx + i) >= n;
    if (__any_sync(0xFFFFFFFFu, bad) && lane_id() == 0) ctl->bad = 1;
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
