// map_api.cu -- host side of the C ABI declared in include/map.h.
//
// The outer loop of MAP (Section 2: propagate to the fix-point, self-map test,
// eliminate, restart) and the fix-point loop are driven from here; every step
// of the arithmetic runs in the kernels of map_kernels.cuh.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

#include "map.h"
#include "map_kernels.cuh"

using mapk::Ctl;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(call)                                                                                                   \
    do {                                                                                                           \
        cudaError_t e_ = (call);                                                                                   \
        if (e_ != cudaSuccess) {                                                                                   \
            cudaGetLastError();                                                                                    \
            return fail(e_ == cudaErrorMemoryAllocation ? MAP_ERR_OOM : MAP_ERR_CUDA, "%s: %s (%s:%d)", #call,   \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                                               \
        }                                                                                                          \
    } while (0)

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int pick_group(uint32_t n, uint64_t m)
{
    const double avg = n ? (double)m / n : 0.0;
    if (avg < 1.5) return 1;
    if (avg < 3.0) return 2;
    if (avg < 6.0) return 4;
    if (avg < 12.0) return 8;
    if (avg < 24.0) return 16;
    return 32;
}

} // namespace

struct map_graph {
    uint32_t n = 0;
    uint64_t m = 0;
    uint32_t words = 0;
    int G = 4;
    int sms = 0;
    cudaStream_t stream = nullptr;
    uint32_t *rowptr = nullptr, *colidx = nullptr, *rrowptr = nullptr, *rcol = nullptr;
    uint32_t *acc0 = nullptr, *acc = nullptr, *mval = nullptr, *fbits = nullptr, *queue = nullptr;
    uint32_t *chv = nullptr, *chval = nullptr;
    Ctl *ctl = nullptr;
    Ctl *h_ctl = nullptr;        // pinned mirror
    uint32_t *h_stage = nullptr; // pinned n words for traces / host output
    uint32_t nacc0 = 0;
    uint64_t export_launches = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace {

void free_graph(map_graph *g)
{
    if (!g) return;
    void *dev[] = {g->rowptr, g->colidx, g->rrowptr, g->rcol, g->acc0, g->acc, g->mval,
                   g->fbits,  g->queue,  g->chv,     g->chval, g->ctl};
    for (void *p : dev)
        if (p) cudaFree(p);
    if (g->h_ctl) cudaFreeHost(g->h_ctl);
    if (g->h_stage) cudaFreeHost(g->h_stage);
    for (auto &e : g->ev)
        if (e) cudaEventDestroy(e);
    cudaGetLastError();
    delete g;
}

int grid_for(const map_graph *g, uint64_t items, int G)
{
    uint64_t blocks = (items * (uint64_t)G + 255) / 256;
    const uint64_t cap = (uint64_t)g->sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

// inclusive scan of x[0..len) in place (multi-level tiles of 1024)
int scan_inclusive(uint32_t *x, uint64_t len, cudaStream_t s)
{
    if (len <= 1) return MAP_OK;
    const uint64_t tiles = (len + 1023) / 1024;
    uint32_t *sums = nullptr;
    if (tiles > 1) CK(cudaMallocAsync((void **)&sums, tiles * sizeof(uint32_t), s));
    mapk::k_scan_tiles<<<(unsigned)tiles, 1024, 0, s>>>(x, len, sums);
    CK(cudaGetLastError());
    if (tiles > 1) {
        int rc = scan_inclusive(sums, tiles, s);
        if (rc) {
            cudaFreeAsync(sums, s);
            return rc;
        }
        mapk::k_scan_add<<<(unsigned)tiles, 1024, 0, s>>>(x, len, sums);
        CK(cudaGetLastError());
        CK(cudaFreeAsync(sums, s));
    }
    return MAP_OK;
}

template <int G>
void launch_transpose(map_graph *g, uint32_t *cursor)
{
    mapk::k_transpose<G><<<grid_for(g, g->n, G), 256, 0, g->stream>>>(g->n, g->rowptr, g->colidx, cursor, g->rcol);
}

#define DISPATCH_G(G, CALL)                                                                                        \
    switch (G) {                                                                                                   \
    case 1: { constexpr int GG = 1; CALL; } break;                                                                 \
    case 2: { constexpr int GG = 2; CALL; } break;                                                                 \
    case 4: { constexpr int GG = 4; CALL; } break;                                                                 \
    case 8: { constexpr int GG = 8; CALL; } break;                                                                 \
    case 16: { constexpr int GG = 16; CALL; } break;                                                               \
    default: { constexpr int GG = 32; CALL; } break;                                                               \
    }

int read_ctl(map_graph *g)
{
    CK(cudaMemcpyAsync(g->h_ctl, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return MAP_OK;
}

int export_map(map_graph *g, uint32_t *dst, bool dst_is_device)
{
    uint32_t *d = dst_is_device ? dst : g->chv; // chv is free between rounds
    mapk::k_export<<<grid_for(g, g->n, 1), 256, 0, g->stream>>>(g->n, g->mval, d);
    CK(cudaGetLastError());
    g->export_launches++;
    if (!dst_is_device) {
        CK(cudaMemcpyAsync(g->h_stage, d, (size_t)g->n * 4, cudaMemcpyDeviceToHost, g->stream));
        CK(cudaStreamSynchronize(g->stream));
        if (dst != g->h_stage) memcpy(dst, g->h_stage, (size_t)g->n * 4);
    }
    return MAP_OK;
}

} // namespace

extern "C" {

const char *map_last_error(void) { return g_err.c_str(); }

int map_graph_info(const map_graph *g, uint32_t *n, uint64_t *m)
{
    if (!g) return fail(MAP_ERR_ARG, "map_graph_info: NULL graph");
    if (n) *n = g->n;
    if (m) *m = g->m;
    return MAP_OK;
}

int map_create(uint32_t n, const uint32_t *rowptr, const uint32_t *colidx, const uint32_t *acc_bits,
               void *cuda_stream, map_graph **out)
{
    g_err.clear();
    if (!out) return fail(MAP_ERR_ARG, "map_create: out is NULL");
    *out = nullptr;
    if (n == 0 || n >= 0x7FFFFFFFu) return fail(MAP_ERR_ARG, "map_create: n = %u out of range [1, 2^31-1)", n);
    if (!rowptr || !acc_bits) return fail(MAP_ERR_ARG, "map_create: rowptr and acc_bits are required");
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // rowptr[0] and rowptr[n] (m) are needed on the host to size the copies
    uint32_t ends[2];
    const bool rp_dev = is_device_ptr(rowptr);
    if (rp_dev) {
        CK(cudaMemcpyAsync(&ends[0], rowptr, 4, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&ends[1], rowptr + n, 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } else {
        ends[0] = rowptr[0];
        ends[1] = rowptr[n];
    }
    if (ends[0] != 0) return fail(MAP_ERR_CSR, "map_create: rowptr[0] = %u, expected 0", ends[0]);
    const uint64_t m = ends[1];
    if (m > 0 && !colidx) return fail(MAP_ERR_ARG, "map_create: colidx is NULL but m = %llu", (unsigned long long)m);

    map_graph *g = new (std::nothrow) map_graph;
    if (!g) return fail(MAP_ERR_OOM, "map_create: host allocation failed");
    g->n = n;
    g->m = m;
    g->words = (n + 31) / 32;
    g->stream = s;
    g->G = pick_group(n, m);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev);
    if (g->sms <= 0) g->sms = 1;

    auto alloc = [&](uint32_t **p, uint64_t words) -> int {
        CK(cudaMalloc((void **)p, (words + 4) * sizeof(uint32_t))); // 16 bytes of slack at the end
        return MAP_OK;
    };
    int rc = MAP_OK;
    const uint64_t W = g->words;
    if ((rc = alloc(&g->rowptr, (uint64_t)n + 1)) || (rc = alloc(&g->colidx, m)) ||
        (rc = alloc(&g->rrowptr, (uint64_t)n + 1)) || (rc = alloc(&g->rcol, m)) || (rc = alloc(&g->acc0, W)) ||
        (rc = alloc(&g->acc, W)) || (rc = alloc(&g->mval, n)) || (rc = alloc(&g->fbits, 2 * W)) ||
        (rc = alloc(&g->queue, 2 * (uint64_t)n)) || (rc = alloc(&g->chv, n)) || (rc = alloc(&g->chval, n))) {
        free_graph(g);
        return rc;
    }
    auto ck = [&](cudaError_t e, const char *what) -> int {
        if (e == cudaSuccess) return MAP_OK;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? MAP_ERR_OOM : MAP_ERR_CUDA, "map_create: %s: %s", what,
                    cudaGetErrorString(e));
    };
    if ((rc = ck(cudaMalloc((void **)&g->ctl, sizeof(Ctl)), "ctl")) ||
        (rc = ck(cudaMallocHost((void **)&g->h_ctl, sizeof(Ctl)), "h_ctl")) ||
        (rc = ck(cudaMallocHost((void **)&g->h_stage, (size_t)n * 4), "h_stage"))) {
        free_graph(g);
        return rc;
    }
    for (auto &e : g->ev)
        if ((rc = ck(cudaEventCreate(&e), "event"))) {
            free_graph(g);
            return rc;
        }

    // copies (host or device sources)
    const auto kind = [](const void *p) { return is_device_ptr(p) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; };
    if ((rc = ck(cudaMemcpyAsync(g->rowptr, rowptr, ((size_t)n + 1) * 4, kind(rowptr), s), "copy rowptr")) ||
        (m && (rc = ck(cudaMemcpyAsync(g->colidx, colidx, m * 4, kind(colidx), s), "copy colidx")))) {
        free_graph(g);
        return rc;
    }
    uint32_t *acc_in = nullptr;
    if (is_device_ptr(acc_bits)) {
        acc_in = const_cast<uint32_t *>(acc_bits);
    } else {
        acc_in = g->acc; // stage through the work bitmap
        if ((rc = ck(cudaMemcpyAsync(acc_in, acc_bits, W * 4, cudaMemcpyHostToDevice, s), "copy acc"))) {
            free_graph(g);
            return rc;
        }
    }
    if ((rc = ck(cudaMemsetAsync(g->ctl, 0, sizeof(Ctl), s), "memset ctl")) ||
        (rc = ck(cudaMemsetAsync(g->colidx + m, 0, 16, s), "pad")) ||
        (rc = ck(cudaMemsetAsync(g->fbits, 0, 2 * W * 4, s), "memset fbits"))) {
        free_graph(g);
        return rc;
    }
    mapk::k_validate<<<grid_for(g, m > n ? m : n, 1), 256, 0, s>>>(n, g->rowptr, m, g->colidx, g->ctl);
    mapk::k_acc_init<<<grid_for(g, W, 1), 256, 0, s>>>(n, acc_in, g->acc0, &g->ctl->elim);
    if ((rc = ck(cudaGetLastError(), "validate")) || (rc = read_ctl(g))) {
        free_graph(g);
        return rc;
    }
    if (g->h_ctl->bad) {
        free_graph(g);
        return fail(MAP_ERR_CSR, "map_create: invalid CSR (decreasing rowptr or colidx >= n)");
    }
    g->nacc0 = g->h_ctl->elim;

    // reverse CSR: in-degree histogram, scan, scatter
    if ((rc = ck(cudaMemsetAsync(g->rrowptr, 0, ((size_t)n + 1) * 4, s), "memset rrowptr"))) {
        free_graph(g);
        return rc;
    }
    mapk::k_indegree<<<grid_for(g, m, 1), 256, 0, s>>>(m, g->colidx, g->rrowptr);
    if ((rc = ck(cudaGetLastError(), "indegree")) || (rc = scan_inclusive(g->rrowptr, (uint64_t)n + 1, s))) {
        free_graph(g);
        return rc;
    }
    // cursor = rrowptr[0..n) (reuse the queue space)
    if ((rc = ck(cudaMemcpyAsync(g->queue, g->rrowptr, (size_t)n * 4, cudaMemcpyDeviceToDevice, s), "cursor"))) {
        free_graph(g);
        return rc;
    }
    DISPATCH_G(g->G, launch_transpose<GG>(g, g->queue));
    if ((rc = ck(cudaGetLastError(), "transpose")) || (rc = ck(cudaStreamSynchronize(s), "create sync"))) {
        free_graph(g);
        return rc;
    }
    *out = g;
    return MAP_OK;
}

int map_destroy(map_graph *g)
{
    free_graph(g);
    return MAP_OK;
}

int map_run(map_graph *g, const map_opts *opts_in, map_result *res, uint32_t *map_out)
{
    g_err.clear();
    if (!g || !res) return fail(MAP_ERR_ARG, "map_run: NULL graph or result");
    map_opts opts;
    memset(&opts, 0, sizeof opts);
    if (opts_in) opts = *opts_in;
    if (opts.sched > MAP_SCHED_ASYNC) return fail(MAP_ERR_ARG, "map_run: unknown schedule %u", opts.sched);
    const bool sync_sched = opts.sched == MAP_SCHED_SYNC;
    const uint64_t max_inner = opts.max_inner ? opts.max_inner : (uint64_t)g->n + 1;
    const bool profile = (opts.flags & MAP_FLAG_PROFILE) != 0;
    memset(res, 0, sizeof *res);
    res->verdict = MAP_NO_CYCLE;
    res->witness = MAP_NONE;
    res->inner_canonical = sync_sched ? 1 : 0;
    cudaStream_t s = g->stream;
    const uint32_t n = g->n;
    const uint32_t W = g->words;
    const int G = g->G;

    g->export_launches = 0;
    CK(cudaEventRecord(g->ev[0], s));
    CK(cudaMemcpyAsync(g->acc, g->acc0, (size_t)W * 4, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(g->fbits, 0, (size_t)2 * W * 4, s));
    uint64_t nacc = g->nacc0;
    uint32_t outer = 0;
    int status = MAP_OK;
    float dense_ms = 0.f;
    bool ran = false;

    while (nacc > 0) {
        if (opts.max_outer && outer >= opts.max_outer) {
            status = fail(MAP_ERR_LIMIT, "map_run: max_outer = %u reached", opts.max_outer);
            break;
        }
        outer++;
        ran = true;
        Ctl init;
        memset(&init, 0, sizeof init);
        init.witness = MAP_NONE;
        *g->h_ctl = init;
        CK(cudaMemcpyAsync(g->ctl, g->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, s));

        // round 1: every row
        if (profile) CK(cudaEventRecord(g->ev[2], s));
        DISPATCH_G(G, (mapk::k_dense<GG><<<grid_for(g, n, GG), 256, 0, s>>>(
                          n, g->rowptr, g->colidx, g->acc, g->mval, g->rrowptr, g->rcol, g->fbits, g->queue, g->ctl,
                          &g->ctl->qcnt[0])));
        CK(cudaGetLastError());
        res->launches++;
        if (profile) CK(cudaEventRecord(g->ev[3], s));
        res->relaxations += g->m;
        uint64_t k = 1;
        int rc = read_ctl(g);
        if (rc) return rc;
        if (profile) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, g->ev[2], g->ev[3]));
            dense_ms += ms;
            res->dense_launches++;
        }
        uint32_t changed = g->h_ctl->ccnt;
        while (changed) {
            k++;
            if (k > max_inner) {
                status = fail(MAP_ERR_LIMIT, "map_run: max_inner = %llu reached", (unsigned long long)max_inner);
                break;
            }
            const int p = (int)(k & 1), np = p ^ 1;
            const uint32_t nfront = g->h_ctl->qcnt[p];
            uint32_t *front = g->queue + (size_t)p * n, *next = g->queue + (size_t)np * n;
            uint32_t *fb = g->fbits + (size_t)p * W, *nb = g->fbits + (size_t)np * W;
            CK(cudaMemsetAsync(&g->ctl->ccnt, 0, 4, s));
            CK(cudaMemsetAsync(&g->ctl->qcnt[np], 0, 4, s));
            if (nfront) {
                if (sync_sched) {
                    DISPATCH_G(G, (mapk::k_sync_compute<GG><<<grid_for(g, nfront, GG), 256, 0, s>>>(
                                      front, nfront, g->rowptr, g->colidx, g->acc, g->mval, fb, g->chv, g->chval,
                                      g->ctl)));
                    DISPATCH_G(G, (mapk::k_sync_apply<GG><<<grid_for(g, nfront, GG), 256, 0, s>>>(
                                      g->chv, g->chval, g->ctl, g->mval, g->rrowptr, g->rcol, nb, next,
                                      &g->ctl->qcnt[np])));
                } else {
                    DISPATCH_G(G, (mapk::k_async_sweep<GG><<<grid_for(g, nfront, GG), 256, 0, s>>>(
                                      front, nfront, g->rowptr, g->colidx, g->acc, g->mval, fb, g->rrowptr,
                                      g->rcol, nb, next, &g->ctl->qcnt[np], g->ctl)));
                }
                CK(cudaGetLastError());
                res->launches += sync_sched ? 2 : 1;
            }
            if ((rc = read_ctl(g))) return rc;
            changed = g->h_ctl->ccnt;
        }
        if (opts.rounds_out && outer - 1 < opts.rounds_cap) opts.rounds_out[outer - 1] = (uint32_t)k;
        res->inner_iters += k;
        if (status != MAP_OK) break;
        if (opts.trace) {
            if ((rc = export_map(g, g->h_stage, false))) return rc;
            opts.trace(opts.user, outer, g->h_stage, n, (uint32_t)k);
        }

        mapk::k_check_eliminate<<<grid_for(g, n, 1), 256, 0, s>>>(n, g->mval, g->acc, g->ctl);
        CK(cudaGetLastError());
        res->launches++;
        if ((rc = read_ctl(g))) return rc;
        res->relaxations += g->h_ctl->relax;
        if (g->h_ctl->witness != MAP_NONE) {
            res->verdict = MAP_CYCLE;
            res->witness = g->h_ctl->witness;
            break;
        }
        if (!g->h_ctl->nonzero) break; // nothing reaches a remaining accepting vertex
        nacc -= g->h_ctl->elim;
    }
    CK(cudaEventRecord(g->ev[1], s));
    CK(cudaEventSynchronize(g->ev[1]));
    float total_ms = 0.f;
    CK(cudaEventElapsedTime(&total_ms, g->ev[0], g->ev[1]));
    res->device_ms = total_ms;
    res->dense_ms = dense_ms;
    res->outer_iters = outer;
    res->edges_total = g->m * (uint64_t)outer;
    res->accepting_left = (uint32_t)nacc;

    if (map_out) {
        const bool dev = is_device_ptr(map_out);
        if (!ran) {
            CK(cudaMemsetAsync(g->mval, 0, (size_t)n * 4, s)); // no iteration: no value anywhere
        }
        int rc = export_map(g, map_out, dev);
        if (rc) return rc;
        if (dev) CK(cudaStreamSynchronize(s));
    }
    res->launches += g->export_launches;
    return status;
}

} // extern "C"
