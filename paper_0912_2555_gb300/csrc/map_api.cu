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

#include <algorithm>
#include <cmath>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "map.h"
#include "map_kernels.cuh"

using mapk::Ctl;

namespace {

thread_local std::string g_err;
// fault injection for tests (served jobs, MAPGPU_INJECT_OOM): when positive, the device
// allocation of create_graph that brings it to zero fails with MAP_ERR_OOM
thread_local int t_inject_alloc = 0;

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

// a pointer the kernels may read p through: device or managed memory as it is, page-locked
// (registered) host memory by its mapped device address; null for pageable host memory
const uint32_t *device_readable(const uint32_t *p)
{
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
    if (a.type == cudaMemoryTypeHost) return static_cast<const uint32_t *>(a.devicePointer);
    return nullptr;
}

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

// Control-block mirrors in page-locked host memory.  A device-to-host copy into
// pageable memory goes through the driver's staging buffer and, measured with
// several host threads each running a graph on its own stream, kept their runs
// from overlapping; copies into page-locked memory do not.  Allocating
// page-locked memory synchronises the device, so the slots come from chunks that
// are allocated once (the first time they run out) and are never given back;
// a freed slot goes to a free list.
class PinnedSlots {
  public:
    static constexpr size_t SLOT = (sizeof(Ctl) + 255) & ~size_t(255);
    static constexpr int PER_CHUNK = 32;
    // a slot, or nullptr if page-locked memory cannot be had (the caller then uses pageable memory)
    void *get()
    {
        std::lock_guard<std::mutex> lk(mu_);
        if (free_.empty()) {
            uint8_t *chunk = nullptr;
            if (cudaHostAlloc((void **)&chunk, SLOT * PER_CHUNK, cudaHostAllocPortable) != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
            for (int i = PER_CHUNK - 1; i >= 0; --i) free_.push_back(chunk + SLOT * i);
        }
        void *p = free_.back();
        free_.pop_back();
        return p;
    }
    void put(void *p)
    {
        std::lock_guard<std::mutex> lk(mu_);
        free_.push_back(p);
    }
    // make sure `k` slots can be handed out without allocating
    void reserve(size_t k)
    {
        std::vector<void *> got;
        for (size_t i = 0; i < k; ++i)
            if (void *p = get()) got.push_back(p);
        for (void *p : got) put(p);
    }

  private:
    std::mutex mu_;
    std::vector<void *> free_;
};

PinnedSlots &ctl_slots()
{
    static PinnedSlots *pool = new PinnedSlots; // process lifetime (page-locked chunks are kept to exit)
    return *pool;
}

// An NVTX range for profilers, popped when the scope ends (a no-op unless a tool is attached):
// map_create, every map_run and served job, and each outer iteration of a host-stepped run.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Rounds over lists of at least this share of the vertices pull instead of pushing (0 = never,
// the default; map_autotune measures the share per handle; MAPGPU_PULL_FRAC sets the default).
double default_pull_frac()
{
    if (const char *e = getenv("MAPGPU_PULL_FRAC")) return atof(e);
    return 0.0;
}

uint32_t pull_min_for(uint32_t n, double frac)
{
    if (!(frac > 0)) return 0;
    const double v = std::ceil(frac * n);
    return (uint32_t)std::max(1.0, std::min(v, 4294967295.0));
}

// resident 256-thread blocks per SM that every variant of the fix-point kernel supports (its
// launch is cooperative, so the grid may not exceed it)
int dense_occupancy()
{
    int occ = 1 << 30, o = 0;
    for (const void *k : {(const void *)mapk::k_dense<2>, (const void *)mapk::k_dense<4>, (const void *)mapk::k_dense<8>}) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, mapk::DT_THREADS, mapk::DT_SMEM) != cudaSuccess) {
            cudaGetLastError();
            o = 1;
        }
        occ = std::min(occ, o);
    }
    return std::max(1, occ);
}

int rounds_occupancy()
{
    int occ = 1 << 30, o = 0;
    auto take = [&](const void *k) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, 256, 0) != cudaSuccess) {
            cudaGetLastError();
            o = 1;
        }
        occ = std::min(occ, o);
    };
    take((const void *)mapk::k_rounds<true, false>);
    take((const void *)mapk::k_rounds<false, false>);
    return std::max(1, occ);
}

// the same for the variant with pull rounds (its grid is the handle's, at most this many blocks per SM)
int func_occupancy()
{
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, mapk::k_func, 256, 0) != cudaSuccess) {
        cudaGetLastError();
        o = 1;
    }
    return std::max(1, o);
}

int pull_occupancy()
{
    int occ = 1 << 30, o = 0;
    for (const void *k : {(const void *)mapk::k_rounds<true, true>, (const void *)mapk::k_rounds<false, true>}) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, 256, 0) != cudaSuccess) {
            cudaGetLastError();
            o = 1;
        }
        occ = std::min(occ, o);
    }
    return std::max(1, occ);
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
    int dense_grid = 0;  // blocks of the dense-round kernel
    int rounds_grid = 0; // blocks of the cooperative fix-point kernel (all resident)
    int check_grid = 0;  // blocks of the self-map / elimination kernel
    int occ_dense = 1, occ_rounds = 1; // resident blocks per SM of the dense-round and fix-point kernels
    cudaStream_t stream = nullptr;
    uint32_t *rowptr = nullptr, *colidx = nullptr, *rrowptr = nullptr, *rcol = nullptr;
    uint32_t *rpos = nullptr; // positions in colidx of the reader entries
    // (set-up only) caller arrays the ingest pass reads and copies into rowptr / colidx itself,
    // instead of a separate copy: device memory, or page-locked host memory the kernels read
    // over the host link; null when the upload copied them already
    const uint32_t *in_rowptr = nullptr, *in_colidx = nullptr;
    uint32_t *elog = nullptr; // vertices eliminated in the current run
    uint32_t *acc0 = nullptr, *acc = nullptr, *mval = nullptr;
    uint32_t *list = nullptr;  // 3n: vertices changed in a round, by round mod 3
    uint32_t *flist = nullptr; // 3n: frontier rows of a round, by round mod 3
    uint4 *rec = nullptr;      // n: per-vertex round state (snapshots, list and frontier flags)
    uint32_t *touched = nullptr, *xbuf = nullptr;
    uint32_t *stale = nullptr; // words: vertices whose mval the next dense round must reset
    uint32_t *cbit = nullptr;  // 3 bitmaps of `words` (+ slack): the list a pull round reads, by round mod 3
    uint32_t pull_min = 0;     // rounds over lists of at least this many vertices pull (0: never)
    uint32_t solo_max = 256;   // rounds over at most this many listed vertices run in one block (0: never)
    int dense_unroll = 4;      // 128-bit loads per lane in flight in the dense round (2, 4 or 8)
    uint32_t lc_passes = 1;    // asynchronous single graphs: block-local passes per round
    uint32_t *ids = nullptr; // reduced graphs: the original id of each vertex (else NULL: identity)
    uint32_t rows = 0;       // rows expanded so far (growing graphs); the rest are empty
    bool dirty = false; // a run stopped early: per-round state may be stale
    uint32_t *hist = nullptr; // rounds per outer iteration
    uint32_t hist_cap = 0;
    Ctl *ctl = nullptr;
    Ctl *h_ctl = nullptr;        // mirror of ctl: a page-locked slot (ctl_slots) or pageable memory
    bool h_ctl_pinned = false;
    uint32_t *h_stage = nullptr; // pinned n words for traces / host output
    uint32_t *h_hist = nullptr;  // pinned mirror of hist
    uint32_t nacc0 = 0;
    cudaEvent_t ev[8] = {};
    // batched graphs (disjoint union of several graphs; see map_batch_create)
    uint32_t ncomp = 0;
    uint32_t *comp = nullptr;        // graph of each union vertex
    mapk::CompState *cs = nullptr;   // one record per graph
    uint32_t *chist = nullptr;       // rounds per outer iteration, CH_CAP per graph
    mapk::CompState *h_cs = nullptr; // pinned mirrors
    uint32_t *h_chist = nullptr;
    // frontier start: the initially accepting vertices (built on first use), and whether the
    // launches being issued use it
    uint32_t *alist = nullptr;
    uint32_t na = 0;
    bool fstart_on = false;
    bool tuned_fstart = false; // map_autotune found the frontier start faster on this graph
    bool pull_on = false;     // the launches being issued may pull (the fix-point kernel's pull variant)
    bool functional = false;  // every row holds at most one entry (set-up): pointer doubling applies
    bool func_on = false;     // the launches being issued propagate by pointer doubling (k_func)
    // the whole run as one CUDA graph, per schedule, start and kernel variant (built on first
    // use): index sched + 2 * frontier start + 4 * pull variant
    // captured runs: slot = schedule + 2 (frontier start) + 4 (pull variant); 8 = pointer doubling
    cudaGraph_t graph[9] = {};
    cudaGraphExec_t exec[9] = {};
    mapk::Handles handles[9] = {};
};

namespace {

void free_graph(map_graph *g)
{
    if (!g) return;
    for (int i = 0; i < 9; ++i) {
        if (g->exec[i]) cudaGraphExecDestroy(g->exec[i]);
        if (g->graph[i]) cudaGraphDestroy(g->graph[i]);
    }
    void *dev[] = {g->rowptr, g->colidx, g->rrowptr, g->rcol,    g->rpos, g->elog, g->acc0, g->acc,
                   g->mval,   g->list,   g->flist,   g->rec,     g->touched, g->xbuf, g->hist, g->ctl,
                   g->alist};
    for (void *p : dev)
        if (p) cudaFreeAsync(p, g->stream); // stream-ordered: no device-wide synchronisation
    if (g->comp) cudaFreeAsync(g->comp, g->stream);
    if (g->ids) cudaFreeAsync(g->ids, g->stream);
    if (g->stale) cudaFreeAsync(g->stale, g->stream);
    if (g->cbit) cudaFreeAsync(g->cbit, g->stream);
    if (g->cs) cudaFreeAsync(g->cs, g->stream);
    if (g->chist) cudaFreeAsync(g->chist, g->stream);
    free(g->h_cs);
    free(g->h_chist);
    if (g->h_ctl_pinned) ctl_slots().put(g->h_ctl);
    else free(g->h_ctl);
    free(g->h_stage);
    free(g->h_hist);
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

// stream-ordered allocation of `words` u32 plus 16 bytes of slack
int ck_alloc(uint32_t **p, uint64_t words, cudaStream_t s)
{
    *p = nullptr;
    CK(cudaMallocAsync((void **)p, (words + 4) * sizeof(uint32_t), s));
    return MAP_OK;
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

// --- the steps of a run, issued on stream s (shared by both drivers) -------

mapk::Dev dev_of(const map_graph *g)
{
    mapk::Dev d;
    d.n = g->n;
    d.words = g->words;
    d.rowptr = g->rowptr;
    d.colidx = g->colidx;
    d.rrowptr = g->rrowptr;
    d.rcol = g->rcol;
    d.rpos = g->rpos;
    d.colidx_w = g->colidx;
    d.elog = g->elog;
    d.acc = g->acc;
    d.mval = g->mval;
    const size_t n = g->n;
    for (int p = 0; p < 3; ++p) {
        d.list[p] = g->list + p * n;
        d.flist[p] = g->flist + p * n;
    }
    d.rec = g->rec;
    for (int p = 0; p < 3; ++p) d.cbit[p] = g->cbit ? g->cbit + p * ((size_t)g->words + 4) : nullptr;
    d.touched = g->touched;
    d.stale = g->comp ? nullptr : g->stale;
    d.ctl = g->ctl;
    d.alist = g->fstart_on ? g->alist : nullptr;
    d.na = g->fstart_on ? g->na : 0;
    d.comp = g->comp;
    d.cs = g->cs;
    d.chist = g->chist;
    d.ncomp = g->ncomp;
    return d;
}

int launch_dense(map_graph *g, cudaStream_t s, mapk::Handles hd)
{
    const mapk::Dev d = dev_of(g);
    if (g->dense_unroll == 2) mapk::k_dense<2><<<g->dense_grid, mapk::DT_THREADS, mapk::DT_SMEM, s>>>(d, hd);
    else if (g->dense_unroll == 8) mapk::k_dense<8><<<g->dense_grid, mapk::DT_THREADS, mapk::DT_SMEM, s>>>(d, hd);
    else mapk::k_dense<4><<<g->dense_grid, mapk::DT_THREADS, mapk::DT_SMEM, s>>>(d, hd);
    CK(cudaGetLastError());
    return MAP_OK;
}

// the fix-point loop: one cooperative launch (its grid barrier needs every block resident)
// the captured run a schedule uses with the launches' current choices
int run_slot(const map_graph *g, int sched)
{
    if (g->func_on && sched == MAP_SCHED_ASYNC) return 8;
    return sched + (g->fstart_on ? 2 : 0) + (g->pull_on ? 4 : 0);
}

int launch_rounds(map_graph *g, cudaStream_t s, bool sync_sched, mapk::Handles hd)
{
    const mapk::Dev d = dev_of(g);
    cudaLaunchConfig_t cfg = {};
    // (the pull variant may fit fewer blocks per SM: its grid is clamped to its own occupancy)
    static const int occ_pull = pull_occupancy();
    const int grid = g->pull_on ? std::min(g->rounds_grid, g->sms * occ_pull) : g->rounds_grid;
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (g->func_on && !sync_sched) { // pointer doubling (its own occupancy)
        static const int occ_func = func_occupancy();
        cfg.gridDim = dim3((unsigned)std::min(g->rounds_grid, g->sms * occ_func));
        CK(cudaLaunchKernelEx(&cfg, mapk::k_func, d, hd));
    } else if (sync_sched && g->pull_on) CK(cudaLaunchKernelEx(&cfg, mapk::k_rounds<true, true>, d, hd));
    else if (sync_sched) CK(cudaLaunchKernelEx(&cfg, mapk::k_rounds<true, false>, d, hd));
    else if (g->pull_on) CK(cudaLaunchKernelEx(&cfg, mapk::k_rounds<false, true>, d, hd));
    else CK(cudaLaunchKernelEx(&cfg, mapk::k_rounds<false, false>, d, hd));
    return MAP_OK;
}

int launch_check(map_graph *g, cudaStream_t s, mapk::Handles hd)
{
    mapk::k_check<<<g->check_grid, 256, 0, s>>>(dev_of(g), hd);
    CK(cudaGetLastError());
    return MAP_OK;
}

// per-run reset: the accepting set (the round state is clean after every run
// that completes; map_run clears it after one that stopped early)
int launch_reset(map_graph *g, cudaStream_t s)
{
    CK(cudaMemcpyAsync(g->acc, g->acc0, (size_t)g->words * 4, cudaMemcpyDeviceToDevice, s));
    return MAP_OK;
}

// end of a run: the eliminated vertices get their flag back in the matrix entries
int launch_restore(map_graph *g, cudaStream_t s)
{
    mapk::k_restore<<<g->check_grid, 256, 0, s>>>(dev_of(g));
    CK(cudaGetLastError());
    return MAP_OK;
}

int launch_export(map_graph *g, cudaStream_t s, uint32_t *override_dst)
{
    mapk::k_export<<<g->check_grid, 256, 0, s>>>(g->n, g->mval, g->ctl, override_dst, g->comp, g->cs);
    CK(cudaGetLastError());
    return MAP_OK;
}

// --- the run as a CUDA graph: outer WHILE { dense; rounds; check } ---------

int add_while(cudaStream_t cs, unsigned long long handle, cudaGraph_t *body)
{
    cudaStreamCaptureStatus st;
    cudaGraph_t cap = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(cs, &st, nullptr, &cap, &deps, nullptr, &nd));
    if (st != cudaStreamCaptureStatusActive) return fail(MAP_ERR_CUDA, "add_while: stream not capturing");
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
    p.conditional.handle = handle;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, cap, deps, nullptr, nd, &p));
    *body = p.conditional.phGraph_out[0];
    CK(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return MAP_OK;
}

int build_run_graph(map_graph *g, int sched)
{
    const int slot = run_slot(g, sched);
    if (g->exec[slot]) return MAP_OK;
    const bool sync_sched = sched == MAP_SCHED_SYNC;
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    int rc = MAP_OK;
    cudaGraph_t top = nullptr, outer_body = nullptr;
    mapk::Handles hd{};
    auto fin = [&](int code) {
        cudaStreamDestroy(cs);
        if (code != MAP_OK && top) cudaGraphDestroy(top);
        cudaGetLastError();
        return code;
    };
#define GK(call)                                                                                                   \
    do {                                                                                                           \
        cudaError_t e_ = (call);                                                                                   \
        if (e_ != cudaSuccess) {                                                                                   \
            cudaGetLastError();                                                                                    \
            return fin(fail(MAP_ERR_CUDA, "graph build: %s: %s", #call, cudaGetErrorString(e_)));                \
        }                                                                                                          \
    } while (0)
    GK(cudaGraphCreate(&top, 0));
    GK(cudaGraphConditionalHandleCreate(&hd.outer, top, 0, cudaGraphCondAssignDefault));
    // top level: reset, run_begin, outer WHILE, export
    GK(cudaStreamBeginCaptureToGraph(cs, top, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    if ((rc = launch_reset(g, cs)) == MAP_OK && g->fstart_on) // no dense round resets the values
        rc = cudaMemsetAsync(g->mval, 0, (size_t)g->n * 4, cs) == cudaSuccess ? MAP_OK : fail(MAP_ERR_CUDA, "memset");
    if (rc == MAP_OK) {
        mapk::k_run_begin<<<1, 32, 0, cs>>>(g->ctl, hd);
        if (g->comp) mapk::k_batch_begin<<<(g->ncomp + 255) / 256, 256, 0, cs>>>(dev_of(g));
        rc = add_while(cs, hd.outer, &outer_body);
        if (rc == MAP_OK) rc = launch_restore(g, cs);
        if (rc == MAP_OK) rc = launch_export(g, cs, nullptr);
    }
    {
        cudaGraph_t got = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &got);
        if (rc) return fin(rc);
        GK(e);
    }
    // outer body: dense round (or, with the frontier start, round 1 inside the fix-point
    // kernel), fix-point loop, self-map test + elimination
    GK(cudaStreamBeginCaptureToGraph(cs, outer_body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    // (in a graph the fix-point kernel ends with the self-map test and the elimination itself)
    rc = g->fstart_on ? MAP_OK : launch_dense(g, cs, hd);
    if (rc == MAP_OK) rc = launch_rounds(g, cs, sync_sched, hd);
    {
        cudaGraph_t got = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &got);
        if (rc) return fin(rc);
        GK(e);
    }
    cudaGraphExec_t exec = nullptr;
    GK(cudaGraphInstantiate(&exec, top, 0));
#undef GK
    g->graph[slot] = top;
    g->exec[slot] = exec;
    g->handles[slot] = hd;
    cudaStreamDestroy(cs);
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

} // extern "C"

namespace {

// Allocate and prepare a graph of n vertices and m edges.  `upload(g, &acc)`
// fills g->rowptr (n + 1 words) and g->colidx (m words) on stream s and sets acc
// to a device bitmap of the accepting vertices; it may also set up the batch
// fields.  Then: validation, accepting set, readers (reverse CSR), flags.
// The stream-ordered allocator returns freed memory to the system at every
// synchronisation unless told otherwise; graphs are created and destroyed
// often (serving), so the device's default pool keeps what it has.
void keep_pool_memory()
{
    static std::atomic<uint64_t> done_mask{0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return;
    }
    if (done_mask.load() & (1ull << dev)) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done_mask.fetch_or(1ull << dev);
}

template <class Upload>
int create_graph(uint32_t n, uint64_t m, cudaStream_t s, const char *who, Upload upload, map_graph **out)
{
    NvtxRange range(who);
    keep_pool_memory();
    map_graph *g = new (std::nothrow) map_graph;
    if (!g) return fail(MAP_ERR_OOM, "%s: host allocation failed", who);
    g->n = n;
    g->m = m;
    g->rows = n;
    g->words = (n + 31) / 32;
    g->stream = s;
    g->G = pick_group(n, m);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev);
    if (g->sms <= 0) g->sms = 1;
    const int occ = dense_occupancy();
    const uint64_t ntiles = ((uint64_t)n + mapk::WT_ROWS - 1) / mapk::WT_ROWS;
    g->dense_grid = (int)std::min<uint64_t>((ntiles + mapk::WT_WARPS - 1) / mapk::WT_WARPS, (uint64_t)g->sms * occ);
    int occ_r = rounds_occupancy();
    // launch shape of the fix-point kernel: MAPGPU_ROUNDS_BLOCKS_PER_SM (1 .. the occupancy
    // limit) overrides the default of every resident slot
    if (const char *e = getenv("MAPGPU_ROUNDS_BLOCKS_PER_SM")) {
        const int v = atoi(e);
        if (v >= 1 && v < occ_r) occ_r = v;
    }
    g->rounds_grid = (int)std::min<uint64_t>(((uint64_t)n + 255) / 256, (uint64_t)g->sms * occ_r);
    g->occ_dense = occ;
    g->occ_rounds = occ_r;
    g->check_grid = (int)std::min<uint64_t>(((uint64_t)n + 255) / 256, (uint64_t)g->sms * 4);
    g->hist_cap = 1u << 16;
    g->pull_min = pull_min_for(n, default_pull_frac());
    if (const char *e = getenv("MAPGPU_SOLO_MAX")) g->solo_max = (uint32_t)strtoul(e, nullptr, 10); // (default 256)
    if (const char *e = getenv("MAPGPU_LC_PASSES")) g->lc_passes = (uint32_t)strtoul(e, nullptr, 10); // (default 1)

    auto alloc = [&](uint32_t **p, uint64_t words) -> int {
        if (t_inject_alloc > 0 && --t_inject_alloc == 0)
            return fail(MAP_ERR_OOM, "%s: injected device allocation failure (MAPGPU_INJECT_OOM)", who);
        // stream-ordered allocation (does not synchronise the device; graphs on other
        // streams keep running); 16 bytes of slack at the end
        CK(cudaMallocAsync((void **)p, (words + 4) * sizeof(uint32_t), s));
        return MAP_OK;
    };
    int rc = MAP_OK;
    const uint64_t W = g->words;
    if ((rc = alloc(&g->rowptr, (uint64_t)n + 1)) || (rc = alloc(&g->colidx, m)) ||
        (rc = alloc(&g->rrowptr, (uint64_t)n + 1)) || (rc = alloc(&g->rcol, m)) || (rc = alloc(&g->rpos, m)) ||
        (rc = alloc(&g->elog, n)) || (rc = alloc(&g->acc0, W)) ||
        (rc = alloc(&g->acc, W)) || (rc = alloc(&g->mval, n)) || (rc = alloc(&g->list, 3 * (uint64_t)n)) ||
        (rc = alloc(&g->flist, 3 * (uint64_t)n)) || (rc = alloc((uint32_t **)&g->rec, 4 * (uint64_t)n)) ||
        (rc = alloc(&g->touched, n)) || (rc = alloc(&g->xbuf, n)) || (rc = alloc(&g->stale, W)) ||
        (rc = alloc(&g->cbit, 3 * (W + 4))) || (rc = alloc(&g->hist, g->hist_cap))) {
        free_graph(g);
        return rc;
    }
    auto ck = [&](cudaError_t e, const char *what) -> int {
        if (e == cudaSuccess) return MAP_OK;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? MAP_ERR_OOM : MAP_ERR_CUDA, "%s: %s: %s", who, what,
                    cudaGetErrorString(e));
    };
    // the control-block mirror in a page-locked slot (see PinnedSlots); the larger mirrors, used by
    // traces and per-iteration round counts only, in pageable memory (pinning or unpinning them
    // per graph would synchronise the device)
    if (void *slot = ctl_slots().get()) {
        g->h_ctl = static_cast<Ctl *>(slot);
        g->h_ctl_pinned = true;
    } else {
        g->h_ctl = static_cast<Ctl *>(aligned_alloc(128, sizeof(Ctl)));
    }
    g->h_stage = static_cast<uint32_t *>(malloc((size_t)n * 4 + 16));
    g->h_hist = static_cast<uint32_t *>(malloc((size_t)g->hist_cap * 4));
    if (!g->h_ctl || !g->h_stage || !g->h_hist) {
        free_graph(g);
        return fail(MAP_ERR_OOM, "%s: host allocation failed", who);
    }
    if ((rc = ck(cudaMallocAsync((void **)&g->ctl, sizeof(Ctl), s), "ctl"))) {
        free_graph(g);
        return rc;
    }
    for (auto &e : g->ev)
        if ((rc = ck(cudaEventCreate(&e), "event"))) {
            free_graph(g);
            return rc;
        }

    // inputs into g->rowptr, g->colidx and an accepting bitmap (host or device sources)
    uint32_t *acc_in = nullptr;
    if ((rc = ck(cudaMemsetAsync(g->ctl, 0, sizeof(Ctl), s), "memset ctl")) || (rc = upload(g, &acc_in))) {
        free_graph(g);
        return rc;
    }
    if ((rc = ck(cudaMemsetAsync(g->colidx + m, 0, 16, s), "pad")) ||
        (rc = ck(cudaMemsetAsync(g->mval, 0, ((size_t)n + 4) * 4, s), "memset mval")) ||
        (rc = ck(cudaMemsetAsync(g->rec, 0, (size_t)n * 16, s), "memset rec")) ||
        (rc = ck(cudaMemsetAsync(g->stale, 0, ((size_t)W + 4) * 4, s), "memset stale")) ||
        (rc = ck(cudaMemsetAsync(g->cbit, 0, 3 * ((size_t)W + 4) * 4, s), "memset cbit"))) {
        free_graph(g);
        return rc;
    }
    // the accepting set, then one pass over the CSR: validation, in-degree histogram of the reverse
    // CSR, and the accepting flag of each target into bit 31 of its entry (restored after every run)
    if ((rc = ck(cudaMemsetAsync(g->rrowptr, 0, ((size_t)n + 1) * 4, s), "memset rrowptr"))) {
        free_graph(g);
        return rc;
    }
    mapk::k_acc_init<<<grid_for(g, W, 1), 256, 0, s>>>(n, acc_in, g->acc0, &g->ctl->elim.v);
    // (each entry's place in its reader list, kept for the scatter; freed at the end of set-up)
    uint32_t *rank = nullptr;
    if ((rc = alloc(&rank, m))) {
        free_graph(g);
        return rc;
    }
    const auto free_rank = [&]() {
        cudaFreeAsync(rank, s);
        rank = nullptr;
    };
    mapk::k_ingest<<<grid_for(g, std::max<uint64_t>(m / 4, n), 1), 256, 0, s>>>(
        n, g->in_rowptr ? g->in_rowptr : g->rowptr, g->in_rowptr ? g->rowptr : nullptr, m,
        g->in_colidx ? g->in_colidx : g->colidx, g->colidx, g->acc0, g->rrowptr, rank, &g->ctl->bad,
        &g->ctl->long_rows);
    g->in_rowptr = g->in_colidx = nullptr;
    if ((rc = ck(cudaGetLastError(), "validate")) || (rc = read_ctl(g))) {
        free_rank();
        free_graph(g);
        return rc;
    }
    if (g->h_ctl->bad) {
        free_rank();
        free_graph(g);
        return fail(MAP_ERR_CSR, "%s: invalid CSR (decreasing rowptr or colidx out of range)", who);
    }
    g->nacc0 = g->h_ctl->elim.v;
    g->functional = m > 0 && g->h_ctl->long_rows == 0;

    // reverse CSR: scan of the histogram, scatter by rank
    if ((rc = scan_inclusive(g->rrowptr, (uint64_t)n + 1, s))) {
        free_rank();
        free_graph(g);
        return rc;
    }
#ifndef MAPGPU_TT_BPS
#define MAPGPU_TT_BPS 4
#endif
    mapk::k_transpose_ranked<<<(unsigned)std::max<uint64_t>(1, std::min<uint64_t>(((uint64_t)n + mapk::TT_ROWS - 1) / mapk::TT_ROWS,
                                                                                 (uint64_t)g->sms * MAPGPU_TT_BPS)),
                               256, 0, s>>>(n, g->rowptr, g->colidx, rank, g->rrowptr, g->rcol, g->rpos);
    rc = ck(cudaGetLastError(), "transpose");
    free_rank();
    if (rc || (rc = ck(cudaStreamSynchronize(s), "create sync"))) {
        free_graph(g);
        return rc;
    }
    *out = g;
    return MAP_OK;
}

} // namespace

extern "C" {

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

    const auto kind = [](const void *p) { return is_device_ptr(p) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; };
    return create_graph(n, m, s, "map_create",
                        [&](map_graph *g, uint32_t **acc) -> int {
                            // arrays the kernels can read are copied by the ingest pass itself (one
                            // pass over the link or HBM instead of two); colidx's 128-bit loads want
                            // it 16-byte aligned
                            if ((g->in_rowptr = device_readable(rowptr)) == nullptr)
                                CK(cudaMemcpyAsync(g->rowptr, rowptr, ((size_t)n + 1) * 4, kind(rowptr), s));
                            const uint32_t *ci = m ? device_readable(colidx) : nullptr;
                            if (ci && ((uintptr_t)ci & 15u) == 0) g->in_colidx = ci;
                            else if (m) CK(cudaMemcpyAsync(g->colidx, colidx, m * 4, kind(colidx), s));
                            if (is_device_ptr(acc_bits)) {
                                *acc = const_cast<uint32_t *>(acc_bits);
                            } else {
                                *acc = g->acc; // stage through the work bitmap
                                CK(cudaMemcpyAsync(g->acc, acc_bits, (size_t)g->words * 4, cudaMemcpyHostToDevice, s));
                            }
                            return MAP_OK;
                        },
                        out);
}

int map_destroy(map_graph *g)
{
    free_graph(g);
    return MAP_OK;
}

static int run_impl(map_graph *g, const map_opts *opts_in, map_result *res, uint32_t *map_out,
                    bool force_stepped = false)
{
    if (!g || !res) return fail(MAP_ERR_ARG, "map_run: NULL graph or result");
    map_opts opts;
    memset(&opts, 0, sizeof opts);
    if (opts_in) opts = *opts_in;
    if (opts.sched > MAP_SCHED_ASYNC) return fail(MAP_ERR_ARG, "map_run: unknown schedule %u", opts.sched);
    const bool sync_sched = opts.sched == MAP_SCHED_SYNC;
    const bool profile = (opts.flags & MAP_FLAG_PROFILE) != 0;
    // the CUDA-graph driver runs the whole loop on the device; per-iteration
    // traces and per-kernel timing need the host-stepped driver (same kernels)
    const bool stepped = opts.trace != nullptr || profile || force_stepped;
    // (a run that stops early leaves round state for the host to clear, so repeated runs must not)
    if (opts.repeat > 1 && (stepped || (opts.flags & MAP_FLAG_EARLY_EXIT) || opts.max_outer || opts.max_inner))
        return fail(MAP_ERR_ARG, "map_run: repeat with a trace, MAP_FLAG_PROFILE, early exit or a limit");
    const uint32_t reps = opts.repeat > 1 ? opts.repeat : 1u;
    if ((opts.flags & MAP_FLAG_FRONTIER_START) && (opts.flags & MAP_FLAG_DENSE_START))
        return fail(MAP_ERR_ARG, "map_run: MAP_FLAG_FRONTIER_START and MAP_FLAG_DENSE_START together");
    // frontier start (round 1 pushed from the accepting vertices): asked for, or chosen by
    // map_autotune and not overridden; with none accepting no iteration runs and the
    // dense-round graph does as well
    NvtxRange range(stepped ? "map_run (stepped)" : "map_run");
    const bool fstart = ((opts.flags & MAP_FLAG_FRONTIER_START) ||
                         (g->tuned_fstart && !(opts.flags & MAP_FLAG_DENSE_START))) &&
                        g->nacc0 > 0;
    if ((opts.flags & MAP_FLAG_PUSH) && (opts.flags & MAP_FLAG_PULL))
        return fail(MAP_ERR_ARG, "map_run: MAP_FLAG_PUSH and MAP_FLAG_PULL together");
    struct FstartOff { // the flags only hold for the launches of this run
        map_graph *g;
        ~FstartOff()
        {
            g->fstart_on = false;
            g->pull_on = false;
            g->func_on = false;
        }
    } fstart_off{g};
    memset(res, 0, sizeof *res);
    cudaStream_t s = g->stream;
    const uint32_t n = g->n;
    const bool out_dev = map_out && is_device_ptr(map_out);

    // run parameters into the control block (the kernels reset the rest)
    Ctl init;
    memset(&init, 0, sizeof init);
    init.max_outer = opts.max_outer;
    init.max_inner = opts.max_inner ? opts.max_inner : (n + 1 > n ? n + 1 : n);
    init.hist_cap = g->hist_cap;
    init.m = g->m;
    init.nacc0 = g->nacc0;
    init.rounds_hist = g->hist;
    init.out = out_dev ? map_out : g->xbuf;
    init.use_graph = stepped ? 0 : 1;
    init.early_exit = (opts.flags & MAP_FLAG_EARLY_EXIT) ? 1 : 0;
    init.timeout_ns = (uint64_t)(opts.timeout_ms ? opts.timeout_ms : 120000u) * 1000000ull;
    init.witness.v = mapk::NONE;
    // an asynchronous single-graph run with the dense start on a graph whose every row holds at
    // most one entry propagates by pointer doubling (MAP_FLAG_PUSH or MAP_FLAG_PULL keep the rounds)
    g->func_on = g->functional && !sync_sched && !fstart && !g->comp && !(opts.flags & (MAP_FLAG_PUSH | MAP_FLAG_PULL));
    init.pull_min = g->func_on ? 0u : (opts.flags & MAP_FLAG_PULL) ? 1u : (opts.flags & MAP_FLAG_PUSH) ? 0u : g->pull_min;
    g->pull_on = init.pull_min != 0;
    init.solo_max = g->solo_max;
    init.lc_passes = g->lc_passes;
    init.solo_fmax = 8 * g->solo_max; // (and at most this many frontier rows to clear)

    int rc = MAP_OK;
    float dense_ms = 0.f, round_ms = 0.f, check_ms = 0.f;
    if (fstart && !g->alist) { // the initially accepting vertices, listed once per graph
        uint32_t *al = nullptr;
        CK(cudaMallocAsync((void **)&al, ((size_t)g->nacc0 + 4) * 4, s));
        CK(cudaMemsetAsync(al + g->nacc0, 0, 4, s));
        mapk::k_acc_list<<<grid_for(g, g->n, 1), 256, 0, s>>>(g->n, g->acc0, al, g->nacc0, al + g->nacc0);
        CK(cudaGetLastError());
        g->alist = al;
        g->na = g->nacc0;
    }
    g->fstart_on = fstart;
    if (g->dirty) { // the previous run stopped early: clear the round state it may have left
        CK(cudaMemsetAsync(g->rec, 0, (size_t)n * 16, s));
        CK(cudaMemsetAsync(g->cbit, 0, 3 * ((size_t)g->words + 4) * 4, s));
    }
    g->dirty = true; // until this run completes normally
    if (!stepped) {
        if ((rc = build_run_graph(g, opts.sched))) return rc;
        *g->h_ctl = init;
        CK(cudaEventRecord(g->ev[0], s));
        for (uint32_t k = 0; k < reps; ++k) { // (the mirror is read back only after the last run)
            CK(cudaMemcpyAsync(g->ctl, g->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, s));
            CK(cudaGraphLaunch(g->exec[run_slot(g, (int)opts.sched)], s));
        }
        CK(cudaEventRecord(g->ev[1], s));
        if ((rc = read_ctl(g))) return rc;
        res->launches = 0; // filled below from the counts
    } else {
        const mapk::Handles none{};
        *g->h_ctl = init;
        CK(cudaEventRecord(g->ev[0], s));
        CK(cudaMemcpyAsync(g->ctl, g->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, s));
        if ((rc = launch_reset(g, s))) return rc;
        if (fstart) CK(cudaMemsetAsync(g->mval, 0, (size_t)n * 4, s)); // no dense round resets the values
        mapk::k_run_begin<<<1, 32, 0, s>>>(g->ctl, none);
        if (g->comp) mapk::k_batch_begin<<<(g->ncomp + 255) / 256, 256, 0, s>>>(dev_of(g));
        CK(cudaGetLastError());
        if ((rc = read_ctl(g))) return rc;
        while (g->h_ctl->outer_go) {
            char label[32];
            snprintf(label, sizeof label, "outer %u", g->h_ctl->outer);
            NvtxRange outer_range(label);
            if (!fstart) {
                if (profile) CK(cudaEventRecord(g->ev[2], s));
                if ((rc = launch_dense(g, s, none))) return rc;
                if (profile) CK(cudaEventRecord(g->ev[3], s));
                if ((rc = read_ctl(g))) return rc;
                if (profile) {
                    float ms = 0.f;
                    CK(cudaEventElapsedTime(&ms, g->ev[2], g->ev[3]));
                    dense_ms += ms;
                    res->dense_launches++;
                }
            }
            if (profile) CK(cudaEventRecord(g->ev[4], s));
            if ((rc = launch_rounds(g, s, sync_sched, none))) return rc;
            if (profile) CK(cudaEventRecord(g->ev[5], s));
            if ((rc = read_ctl(g))) return rc;
            if (profile) {
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, g->ev[4], g->ev[5]));
                round_ms += ms;
            }
            if (opts.trace) {
                const uint32_t outer = g->h_ctl->outer, k = g->h_ctl->k;
                if ((rc = launch_export(g, s, g->xbuf))) return rc;
                CK(cudaMemcpyAsync(g->h_stage, g->xbuf, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                opts.trace(opts.user, outer, g->h_stage, n, k);
            }
            if (profile) CK(cudaEventRecord(g->ev[6], s));
            if ((rc = launch_check(g, s, none))) return rc;
            if (profile) CK(cudaEventRecord(g->ev[7], s));
            if ((rc = read_ctl(g))) return rc;
            if (profile) {
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, g->ev[6], g->ev[7]));
                check_ms += ms;
            }
        }
        if ((rc = launch_restore(g, s))) return rc;
        if ((rc = launch_export(g, s, nullptr))) return rc;
        CK(cudaEventRecord(g->ev[1], s));
        if ((rc = read_ctl(g))) return rc;
    }
    CK(cudaEventSynchronize(g->ev[1]));
    float total_ms = 0.f;
    CK(cudaEventElapsedTime(&total_ms, g->ev[0], g->ev[1]));
    const Ctl &c = *g->h_ctl;
    res->verdict = c.verdict ? MAP_CYCLE : MAP_NO_CYCLE;
    res->witness = c.verdict ? c.witness.v : MAP_NONE;
    res->outer_iters = c.outer;
    res->inner_canonical = (sync_sched && !c.early_hit) ? 1 : 0;
    res->inner_iters = c.inner_total;
    res->relaxations = c.relax.v;
    res->edges_total = g->m * (uint64_t)c.outer;
    res->device_ms = total_ms;
    if (!profile) { // the kernels' own %globaltimer stamps of each phase
        dense_ms = (float)(c.ph_dense * 1e-6);
        round_ms = (float)(c.ph_rounds * 1e-6);
        check_ms = (float)(c.ph_check * 1e-6);
        res->dense_launches = fstart ? 0u : c.outer;
    }
    res->dense_ms = dense_ms;
    res->round_ms = round_ms;
    res->frontier_rows = c.frontier_rows.v;
    res->check_ms = check_ms;
    res->accepting_left = c.nacc;
    // kernel launches: run_begin, restore, export, and per outer iteration dense (not with the
    // frontier start), rounds and (stepped from the host) check
    res->launches = 3 + ((fstart ? 1ull : 2ull) + (stepped ? 1ull : 0ull)) * c.outer;
    const uint32_t nh = std::min<uint32_t>(c.outer, g->hist_cap);
    if (opts.rounds_out && nh) {
        CK(cudaMemcpyAsync(g->h_hist, g->hist, (size_t)nh * 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        memcpy(opts.rounds_out, g->h_hist, (size_t)std::min(nh, opts.rounds_cap) * 4);
    }
    if (map_out && !out_dev) { // straight into the caller's buffer (DMA at full rate when it is pinned)
        CK(cudaMemcpyAsync(map_out, g->xbuf, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    g->dirty = c.status != mapk::ST_OK || c.early_hit;
    if (c.status == mapk::ST_LIMIT) return fail(MAP_ERR_LIMIT, "map_run: max_outer or max_inner reached");
    if (c.status == mapk::ST_TIMEOUT && c.gave_up)
        return fail(MAP_ERR_TIMEOUT, "map_run: a bounded device wait (%s) gave up after seconds without progress",
                    c.gave_up == 1 ? "grid barrier" : "hand-back of one-block rounds");
    if (c.status == mapk::ST_TIMEOUT)
        return fail(MAP_ERR_TIMEOUT, "map_run: stopped after timeout_ms = %u", opts.timeout_ms ? opts.timeout_ms : 120000u);
    return MAP_OK;
}

int map_run(map_graph *g, const map_opts *opts, map_result *res, uint32_t *map_out)
{
    g_err.clear();
    if (!g || !res) return fail(MAP_ERR_ARG, "map_run: NULL graph or result");
    if (g->comp) return fail(MAP_ERR_ARG, "map_run: this handle holds a batch; use map_batch_run");
    const int rc = run_impl(g, opts, res, map_out);
    res->status = (uint32_t)rc;
    return rc;
}

// Launch shapes of a handle: blocks per SM of the dense-round and fix-point kernels.
static void set_shapes(map_graph *g, uint32_t dense_bps, uint32_t rounds_bps)
{
    const uint64_t ntiles = ((uint64_t)g->n + mapk::WT_ROWS - 1) / mapk::WT_ROWS;
    g->dense_grid = (int)std::max<uint64_t>(
        1, std::min<uint64_t>((ntiles + mapk::WT_WARPS - 1) / mapk::WT_WARPS, (uint64_t)g->sms * dense_bps));
    g->rounds_grid = (int)std::max<uint64_t>(
        1, std::min<uint64_t>(((uint64_t)g->n + 255) / 256, (uint64_t)g->sms * rounds_bps));
    for (int i = 0; i < 9; ++i) { // the captured graphs hold the old shapes
        if (g->exec[i]) cudaGraphExecDestroy(g->exec[i]);
        if (g->graph[i]) cudaGraphDestroy(g->graph[i]);
        g->exec[i] = nullptr;
        g->graph[i] = nullptr;
    }
}

int map_autotune(map_graph *g, uint32_t sched, map_tune_result *out)
{
    g_err.clear();
    if (!g || !out) return fail(MAP_ERR_ARG, "map_autotune: NULL handle or result");
    if (sched > MAP_SCHED_ASYNC) return fail(MAP_ERR_ARG, "map_autotune: unknown schedule %u", sched);
    const int occ_d = dense_occupancy();
    const int occ_r = rounds_occupancy();
    memset(out, 0, sizeof *out);
    map_result r;
    // whole runs (one graph launch each) with `flags`, the better of two
    auto whole_run = [&](uint32_t flags, double *best_ms) -> int {
        map_opts q;
        memset(&q, 0, sizeof q);
        q.sched = sched;
        q.flags = flags;
        *best_ms = 1e30;
        for (int rep = 0; rep < 2; ++rep) {
            const int rc = run_impl(g, &q, &r, nullptr);
            if (rc != MAP_OK) return rc;
            out->trials++;
            *best_ms = std::min(*best_ms, r.device_ms);
        }
        return MAP_OK;
    };
    int rc = MAP_OK;
    // 1. when a round pulls instead of pushing (rounds over lists of at least a share of the
    // vertices; 0 = never)
    out->pull_share = 0;
    if (g->nacc0) {
        const double shares[] = {0.0, 1.0 / 256, 1.0 / 64, 1.0 / 32, 1.0 / 16, 1.0 / 8, 1.0 / 4};
        double best = 1e30;
        uint32_t best_min = 0;
        for (double sh : shares) {
            g->pull_min = pull_min_for(g->n, sh);
            double t = 0;
            if ((rc = whole_run(MAP_FLAG_DENSE_START, &t))) return rc;
            if (sh == 0.0) out->push_only_ms = t;
            if (t < best) {
                best = t;
                best_min = g->pull_min;
                out->pull_share = sh;
            }
        }
        g->pull_min = best_min;
        out->pull_ms = best;
    }
    // 2. (asynchronous single graphs) block-local passes per round
    if (g->nacc0 && sched == MAP_SCHED_ASYNC && !g->comp) {
        const uint32_t passes[] = {0, 1, 2, 4, 8, 16, 32};
        double best = 1e30;
        uint32_t best_p = g->lc_passes;
        for (uint32_t pz : passes) {
            g->lc_passes = pz;
            double t = 0;
            if ((rc = whole_run(MAP_FLAG_DENSE_START, &t))) return rc;
            if (t < best) {
                best = t;
                best_p = pz;
            }
        }
        g->lc_passes = best_p;
        out->local_passes = best_p;
    } else {
        out->local_passes = g->lc_passes;
    }
    // 3. up to which list size block 0 runs a round alone (0 = never)
    if (g->nacc0) {
        const uint32_t sizes[] = {0, 64, 256, 1024};
        double best = 1e30;
        uint32_t best_s = g->solo_max;
        for (uint32_t sz : sizes) {
            g->solo_max = sz;
            double t = 0;
            if ((rc = whole_run(MAP_FLAG_DENSE_START, &t))) return rc;
            if (t < best) {
                best = t;
                best_s = sz;
            }
        }
        g->solo_max = best_s;
        out->solo_max = best_s;
        out->solo_ms = best;
    }
    map_opts o;
    memset(&o, 0, sizeof o);
    o.sched = sched;
    o.flags = MAP_FLAG_PROFILE | MAP_FLAG_DENSE_START; // host-stepped run, CUDA events around every phase
    // the dense-round shape first (with the fix-point shape as it is), then the fix-point shape
    const uint32_t cands[] = {1, 2, 3, 4, 6, 8};
    uint32_t best_d = 0, best_r = 0;
    double t_d = 1e30, t_r = 1e30;
    const uint32_t cur_r = (uint32_t)std::max(1, (g->rounds_grid + g->sms - 1) / g->sms);
    for (uint32_t bps : cands) {
        if ((int)bps > occ_d) continue;
        set_shapes(g, bps, cur_r);
        if ((rc = run_impl(g, &o, &r, nullptr)) != MAP_OK) return rc;
        out->trials++;
        if (r.dense_ms < t_d) {
            t_d = r.dense_ms;
            best_d = bps;
        }
    }
    // the dense round's loads in flight per lane, at that shape
    {
        double t_u = 1e30;
        int best_u = g->dense_unroll;
        set_shapes(g, best_d, cur_r);
        for (int u : {2, 4, 8}) {
            g->dense_unroll = u;
            if ((rc = run_impl(g, &o, &r, nullptr)) != MAP_OK) return rc;
            out->trials++;
            if (r.dense_ms < t_u) {
                t_u = r.dense_ms;
                best_u = u;
            }
        }
        g->dense_unroll = best_u;
        out->dense_unroll = (uint32_t)best_u;
        t_d = std::min(t_d, t_u);
    }
    for (uint32_t bps : cands) {
        if ((int)bps > occ_r) continue;
        set_shapes(g, best_d, bps);
        if ((rc = run_impl(g, &o, &r, nullptr)) != MAP_OK) return rc;
        out->trials++;
        if (r.round_ms < t_r) {
            t_r = r.round_ms;
            best_r = bps;
        }
    }
    set_shapes(g, best_d, best_r);
    out->dense_blocks_per_sm = best_d;
    out->rounds_blocks_per_sm = best_r;
    out->dense_ms = t_d;
    out->rounds_ms = t_r;
    // the start of every outer iteration, with those shapes: whole runs as one graph launch each,
    // the better of two per start
    g->tuned_fstart = false;
    if (g->nacc0) {
        double t[2] = {1e30, 1e30};
        for (int f = 0; f < 2; ++f)
            if ((rc = whole_run(f ? MAP_FLAG_FRONTIER_START : MAP_FLAG_DENSE_START, &t[f]))) return rc;
        g->tuned_fstart = t[1] < t[0];
        out->frontier_start = g->tuned_fstart ? 1u : 0u;
        out->dense_start_ms = t[0];
        out->frontier_start_ms = t[1];
    }
    return MAP_OK;
}

// shortest path source -> target along rows (at least one edge) into host path[0..cap); *len = vertices
static int bfs_path(map_graph *g, uint32_t source, uint32_t target, uint32_t *path, uint32_t cap, uint32_t *len)
{
    cudaStream_t s = g->stream;
    const uint32_t n = g->n;
    uint32_t *parent = g->xbuf, *q0 = g->list, *q1 = g->list + n; // list holds 3n entries
    uint32_t *cnt = &g->ctl->lcnt[0].v, *cnt2 = &g->ctl->lcnt[1].v, *found = &g->ctl->lcnt[2].v;
    mapk::k_fill<<<grid_for(g, n, 1), 256, 0, s>>>(parent, n, mapk::NONE);
    CK(cudaGetLastError());
    if (source != target) { // the source is reached from the start
        CK(cudaMemcpyAsync(parent + source, &source, 4, cudaMemcpyHostToDevice, s));
    }
    uint32_t one = 1, zero = 0;
    CK(cudaMemcpyAsync(q0, &source, 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(cnt, &one, 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(found, &zero, 4, cudaMemcpyHostToDevice, s));
    uint32_t h[2] = {1, 0};
    for (uint32_t level = 0; level <= n && h[0]; ++level) {
        CK(cudaMemcpyAsync(cnt2, &zero, 4, cudaMemcpyHostToDevice, s));
        mapk::k_bfs_level<<<grid_for(g, h[0], 1), 256, 0, s>>>(q0, cnt, g->rowptr, g->colidx, parent, q1, cnt2,
                                                                 target, found);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(&h[0], cnt2, 4, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&h[1], found, 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (h[1]) break;
        std::swap(q0, q1);
        std::swap(cnt, cnt2);
    }
    if (!h[1]) return fail(MAP_ERR_ARG, "map_lasso: vertex %u is not reachable from %u", target, source);
    // a parent chain visits distinct vertices (target twice when it is the source): <= n + 1 entries
    uint32_t k = 0, *out = g->list;
    const uint32_t dcap = cap < n + 1 ? cap : n + 1;
    mapk::k_walk_back<<<1, 32, 0, s>>>(parent, source, target, out, dcap, n + 1, found);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&k, found, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (k == 0xFFFFFFFFu || k > cap) return fail(MAP_ERR_LIMIT, "map_lasso: the path does not fit into %u entries", cap);
    std::vector<uint32_t> rev(k);
    CK(cudaMemcpyAsync(rev.data(), out, (size_t)k * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (uint32_t i = 0; i < k; ++i) path[i] = rev[k - 1 - i];
    *len = k;
    return MAP_OK;
}

int map_lasso(map_graph *g, uint32_t init, uint32_t witness, uint32_t *path, uint32_t cap, uint32_t *prefix_len,
              uint32_t *cycle_len)
{
    g_err.clear();
    if (!g || !path || !prefix_len || !cycle_len) return fail(MAP_ERR_ARG, "map_lasso: NULL argument");
    if (g->comp) return fail(MAP_ERR_ARG, "map_lasso: single graphs only");
    if (witness >= g->n || (init != MAP_NONE && init >= g->n)) return fail(MAP_ERR_ARG, "map_lasso: vertex out of range");
    *prefix_len = *cycle_len = 0;
    uint32_t used = 0;
    int rc = MAP_OK;
    if (init != MAP_NONE && init != witness) { // init -> ... -> witness
        uint32_t k = 0;
        if ((rc = bfs_path(g, init, witness, path, cap, &k))) return rc;
        used = k - 1; // the witness opens the cycle part
        *prefix_len = used;
    }
    uint32_t k = 0; // witness -> ... -> witness
    if ((rc = bfs_path(g, witness, witness, path + used, cap - used, &k))) return rc;
    *cycle_len = k;
    return MAP_OK;
}

// ---------------------------------------------------- reduction and export --

namespace {

int launch_reach(map_graph *g, const uint32_t *ptr, const uint32_t *col, const uint32_t *part, uint32_t *mark,
                 uint32_t bit, uint32_t *q)
{
    cudaStream_t s = g->stream;
    Ctl *c = g->ctl;
    // queue counters, barrier and status of this sweep
    for (mapk::Cnt32 *x : {&c->lcnt[0], &c->lcnt[1], &c->lcnt[2], &c->bar_count, &c->bar_gen})
        CK(cudaMemsetAsync(&x->v, 0, 4, s));
    CK(cudaMemsetAsync(&c->status, 0, 4, s));
    mapk::k_reach_seed<<<grid_for(g, g->n, 1), 256, 0, s>>>(g->n, g->acc0, mark, bit, q, &c->lcnt[0].v);
    CK(cudaGetLastError());
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mapk::k_reach, 256, 0));
    if (occ < 1) occ = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::min<uint64_t>(((uint64_t)g->n + 255) / 256, (uint64_t)g->sms * occ));
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, mapk::k_reach, g->n, ptr, col, part, mark, bit, q, c));
    return MAP_OK;
}

// the reduced graph of g (see map_create_reduced); part: device labels or NULL
int reduce_graph(map_graph *g, const uint32_t *part, map_graph **out)
{
    cudaStream_t s = g->stream;
    const uint32_t n = g->n;
    uint32_t *mark = g->xbuf, *rank = g->touched, *q = g->list; // list: 3n entries
    CK(cudaMemsetAsync(mark, 0, (size_t)n * 4, s));
    int rc;
    if ((rc = launch_reach(g, g->rowptr, g->colidx, part, mark, 1u, q)) ||   // reached from an accepting vertex
        (rc = launch_reach(g, g->rrowptr, g->rcol, part, mark, 2u, q)))      // reaching one
        return rc;
    if ((rc = read_ctl(g))) return rc;
    if (g->h_ctl->status) return fail(MAP_ERR_TIMEOUT, "map_create_reduced: a reachability sweep gave up waiting");
    mapk::k_keep<<<grid_for(g, n, 1), 256, 0, s>>>(n, mark, rank);
    CK(cudaGetLastError());
    if ((rc = scan_inclusive(rank, n, s))) return rc;
    uint32_t n2 = 0;
    CK(cudaMemcpyAsync(&n2, rank + n - 1, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (n2 == 0) { // no accepting vertex: one isolated, non-accepting vertex that stands for nothing
        const uint32_t rp0[2] = {0, 0}, acc0 = 0;
        if ((rc = map_create(1, rp0, nullptr, &acc0, s, out))) return rc;
        if ((rc = ck_alloc(&(*out)->ids, 1, s)) == MAP_OK) {
            mapk::k_fill<<<1, 32, 0, s>>>((*out)->ids, 1, MAP_NONE);
            if (cudaGetLastError() != cudaSuccess) rc = fail(MAP_ERR_CUDA, "map_create_reduced: fill");
        }
        if (rc) {
            free_graph(*out);
            *out = nullptr;
        }
        return rc;
    }
    const uint32_t W2 = (n2 + 31) / 32;
    uint32_t *rp = nullptr, *col2 = nullptr, *ids = nullptr, *acc2 = nullptr;
    auto done = [&](int r) {
        for (uint32_t *p : {rp, col2, acc2}) if (p) cudaFreeAsync(p, s);
        if (r != MAP_OK && ids) cudaFreeAsync(ids, s);
        return r;
    };
    if ((rc = ck_alloc(&rp, (uint64_t)n2 + 1, s)) || (rc = ck_alloc(&ids, n2, s)) || (rc = ck_alloc(&acc2, W2, s)))
        return done(rc);
    if (cudaMemsetAsync(rp, 0, 4, s) || cudaMemsetAsync(acc2, 0, (size_t)W2 * 4, s))
        return done(fail(MAP_ERR_CUDA, "map_create_reduced: memset"));
    mapk::k_reduce_rows<0><<<grid_for(g, n, 1), 256, 0, s>>>(n, g->rowptr, g->colidx, part, mark, rank, g->acc0, rp,
                                                             nullptr, nullptr, nullptr);
    if (cudaGetLastError()) return done(fail(MAP_ERR_CUDA, "map_create_reduced: row lengths"));
    if ((rc = scan_inclusive(rp + 1, n2, s))) return done(rc);
    uint32_t m2 = 0;
    if (cudaMemcpyAsync(&m2, rp + n2, 4, cudaMemcpyDeviceToHost, s) || cudaStreamSynchronize(s))
        return done(fail(MAP_ERR_CUDA, "map_create_reduced: edge count"));
    if ((rc = ck_alloc(&col2, m2, s))) return done(rc);
    mapk::k_reduce_rows<1><<<grid_for(g, n, 1), 256, 0, s>>>(n, g->rowptr, g->colidx, part, mark, rank, g->acc0, rp,
                                                             col2, ids, acc2);
    if (cudaGetLastError()) return done(fail(MAP_ERR_CUDA, "map_create_reduced: rows"));
    if ((rc = map_create(n2, rp, col2, acc2, s, out))) return done(rc);
    (*out)->ids = ids;
    return done(MAP_OK);
}

} // namespace

int map_create_reduced(uint32_t n, const uint32_t *rowptr, const uint32_t *colidx, const uint32_t *acc_bits,
                       const uint32_t *part, void *cuda_stream, map_graph **out)
{
    g_err.clear();
    if (!out) return fail(MAP_ERR_ARG, "map_create_reduced: out is NULL");
    *out = nullptr;
    map_graph *full = nullptr;
    int rc = map_create(n, rowptr, colidx, acc_bits, cuda_stream, &full);
    if (rc) return rc;
    cudaStream_t s = full->stream;
    uint32_t *part_dev = nullptr;
    if (part && !is_device_ptr(part)) { // labels to the device
        if ((rc = ck_alloc(&part_dev, n, s)) == MAP_OK &&
            cudaMemcpyAsync(part_dev, part, (size_t)n * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
            rc = fail(MAP_ERR_CUDA, "map_create_reduced: copy of part");
        if (rc) {
            if (part_dev) cudaFreeAsync(part_dev, s);
            free_graph(full);
            return rc;
        }
    }
    rc = reduce_graph(full, part_dev ? part_dev : part, out);
    if (part_dev) cudaFreeAsync(part_dev, s);
    free_graph(full);
    if (rc == MAP_OK && cudaStreamSynchronize(s) != cudaSuccess) {
        free_graph(*out);
        *out = nullptr;
        return fail(MAP_ERR_CUDA, "map_create_reduced: %s", cudaGetErrorString(cudaGetLastError()));
    }
    return rc;
}

int map_grow_create(uint32_t n, const uint32_t *acc_bits, void *cuda_stream, map_graph **out)
{
    g_err.clear();
    if (!out) return fail(MAP_ERR_ARG, "map_grow_create: out is NULL");
    *out = nullptr;
    if (n == 0 || n >= 0x7FFFFFFFu) return fail(MAP_ERR_ARG, "map_grow_create: n = %u out of range [1, 2^31-1)", n);
    if (!acc_bits) return fail(MAP_ERR_ARG, "map_grow_create: acc_bits is required");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int rc = create_graph(n, 0, s, "map_grow_create",
                                [&](map_graph *g, uint32_t **acc) -> int {
                                    CK(cudaMemsetAsync(g->rowptr, 0, ((size_t)n + 1) * 4, s));
                                    *acc = g->acc;
                                    CK(cudaMemcpyAsync(g->acc, acc_bits, (size_t)g->words * 4, cudaMemcpyDefault, s));
                                    return MAP_OK;
                                },
                                out);
    if (rc == MAP_OK) (*out)->rows = 0;
    return rc;
}

int map_append(map_graph *g, uint32_t n_add, const uint32_t *acc_bits_add, uint32_t k, const uint32_t *rowptr_add,
               const uint32_t *colidx_add)
{
    g_err.clear();
    if (!g) return fail(MAP_ERR_ARG, "map_append: NULL graph");
    if (g->comp || g->ids) return fail(MAP_ERR_ARG, "map_append: not for batched or reduced graphs");
    const uint64_t n2 = (uint64_t)g->n + n_add;
    if (n2 >= 0x7FFFFFFFu) return fail(MAP_ERR_ARG, "map_append: %llu vertices out of range", (unsigned long long)n2);
    if ((uint64_t)g->rows + k > n2)
        return fail(MAP_ERR_ARG, "map_append: %u rows for %llu unexpanded vertices", k,
                    (unsigned long long)(n2 - g->rows));
    if ((n_add && !acc_bits_add) || (k && !rowptr_add)) return fail(MAP_ERR_ARG, "map_append: NULL argument");
    cudaStream_t s = g->stream;
    uint32_t ends[2] = {0, 0}; // chunk offsets: first and last
    if (k) {
        if (is_device_ptr(rowptr_add)) {
            CK(cudaMemcpyAsync(&ends[0], rowptr_add, 4, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(&ends[1], rowptr_add + k, 4, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
        } else {
            ends[0] = rowptr_add[0];
            ends[1] = rowptr_add[k];
        }
    }
    if (ends[0] != 0) return fail(MAP_ERR_CSR, "map_append: rowptr_add[0] = %u, expected 0", ends[0]);
    const uint64_t madd = ends[1], m0 = g->m, m2 = m0 + madd;
    if (madd && !colidx_add) return fail(MAP_ERR_ARG, "map_append: colidx_add is NULL but the rows hold %llu edges",
                                         (unsigned long long)madd);
    if (m2 > 0xFFFFFFFFull) return fail(MAP_ERR_ARG, "map_append: %llu edges out of range", (unsigned long long)m2);
    const uint32_t r = g->rows, n0 = g->n;
    const auto kind = [](const void *p) { return is_device_ptr(p) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; };
    map_graph *ng = nullptr;
    int rc = create_graph(
        (uint32_t)n2, m2, s, "map_append",
        [&](map_graph *x, uint32_t **acc) -> int {
            // the resident part stays on the device; only the chunk crosses from the host
            CK(cudaMemcpyAsync(x->rowptr, g->rowptr, ((size_t)r + 1) * 4, cudaMemcpyDeviceToDevice, s));
            if (k) CK(cudaMemcpyAsync(x->rowptr + r, rowptr_add, ((size_t)k + 1) * 4, kind(rowptr_add), s));
            mapk::k_grow_rowptr<<<grid_for(x, n2 - r + 1, 1), 256, 0, s>>>(x->rowptr, r, k, (uint32_t)n2, (uint32_t)m0,
                                                                          (uint32_t)m2);
            CK(cudaGetLastError());
            if (m0) {
                mapk::k_unflag<<<grid_for(x, m0, 1), 256, 0, s>>>(m0, g->colidx, x->colidx);
                CK(cudaGetLastError());
            }
            if (madd) CK(cudaMemcpyAsync(x->colidx + m0, colidx_add, madd * 4, kind(colidx_add), s));
            const uint32_t *add = acc_bits_add;
            uint32_t *tmp = nullptr;
            if (n_add && !is_device_ptr(add)) {
                int rc2 = ck_alloc(&tmp, (n_add + 31) / 32, s);
                if (rc2) return rc2;
                CK(cudaMemcpyAsync(tmp, add, (size_t)((n_add + 31) / 32) * 4, cudaMemcpyHostToDevice, s));
                add = tmp;
            }
            mapk::k_grow_acc<<<grid_for(x, x->words, 1), 256, 0, s>>>(x->acc, x->words, g->acc0, n0, add, n_add);
            const cudaError_t e = cudaGetLastError();
            if (tmp) cudaFreeAsync(tmp, s);
            CK(e);
            *acc = x->acc;
            return MAP_OK;
        },
        &ng);
    if (rc) return rc;
    ng->rows = r + k;
    std::swap(*g, *ng); // the caller's handle now holds the grown graph
    free_graph(ng);
    return MAP_OK;
}

int map_graph_vertex_ids(const map_graph *g, uint32_t *ids)
{
    g_err.clear();
    if (!g || !ids) return fail(MAP_ERR_ARG, "map_graph_vertex_ids: NULL argument");
    cudaStream_t s = g->stream;
    if (g->ids) {
        CK(cudaMemcpyAsync(ids, g->ids, (size_t)g->n * 4, cudaMemcpyDefault, s));
    } else if (is_device_ptr(ids)) {
        mapk::k_iota<<<grid_for(g, g->n, 1), 256, 0, s>>>(g->n, ids);
        CK(cudaGetLastError());
    } else {
        for (uint32_t v = 0; v < g->n; ++v) ids[v] = v;
    }
    CK(cudaStreamSynchronize(s));
    return MAP_OK;
}

int map_graph_csr(const map_graph *g, uint32_t *rowptr, uint32_t *colidx, uint32_t *acc_bits)
{
    g_err.clear();
    if (!g) return fail(MAP_ERR_ARG, "map_graph_csr: NULL graph");
    cudaStream_t s = g->stream;
    if (rowptr) CK(cudaMemcpyAsync(rowptr, g->rowptr, ((size_t)g->n + 1) * 4, cudaMemcpyDefault, s));
    if (acc_bits) CK(cudaMemcpyAsync(acc_bits, g->acc0, (size_t)g->words * 4, cudaMemcpyDefault, s));
    if (colidx && g->m) {
        uint32_t *tmp = nullptr;
        int rc = ck_alloc(&tmp, g->m, s);
        if (rc) return rc;
        mapk::k_unflag<<<grid_for(g, g->m, 1), 256, 0, s>>>(g->m, g->colidx, tmp);
        const cudaError_t e1 = cudaGetLastError();
        const cudaError_t e2 = e1 ? e1 : cudaMemcpyAsync(colidx, tmp, g->m * 4, cudaMemcpyDefault, s);
        cudaFreeAsync(tmp, s);
        CK(e2);
    }
    CK(cudaStreamSynchronize(s));
    return MAP_OK;
}

int map_batch_create(uint32_t count, const uint32_t *ns, const uint32_t *const *rowptrs,
                     const uint32_t *const *colidxs, const uint32_t *const *acc_bits, void *cuda_stream,
                     map_graph **out)
{
    g_err.clear();
    if (!out) return fail(MAP_ERR_ARG, "map_batch_create: out is NULL");
    *out = nullptr;
    if (count == 0 || !ns || !rowptrs || !colidxs || !acc_bits)
        return fail(MAP_ERR_ARG, "map_batch_create: count = 0 or a NULL array");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    std::vector<uint32_t> off(count + 1), woff(count + 1), mc(count);
    std::vector<uint64_t> eoff(count + 1);
    off[0] = 0;
    eoff[0] = 0;
    woff[0] = 0;
    for (uint32_t c = 0; c < count; ++c) {
        if (ns[c] == 0 || !rowptrs[c] || !acc_bits[c])
            return fail(MAP_ERR_ARG, "map_batch_create: graph %u: n = 0 or NULL rowptr / acc_bits", c);
        uint32_t ends[2];
        if (is_device_ptr(rowptrs[c])) {
            CK(cudaMemcpyAsync(&ends[0], rowptrs[c], 4, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(&ends[1], rowptrs[c] + ns[c], 4, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
        } else {
            ends[0] = rowptrs[c][0];
            ends[1] = rowptrs[c][ns[c]];
        }
        if (ends[0] != 0) return fail(MAP_ERR_CSR, "map_batch_create: graph %u: rowptr[0] = %u", c, ends[0]);
        if (ends[1] > 0 && !colidxs[c]) return fail(MAP_ERR_ARG, "map_batch_create: graph %u: colidx is NULL", c);
        mc[c] = ends[1];
        const uint64_t n_next = (uint64_t)off[c] + ns[c];
        if (n_next >= 0x7FFFFFFFu) return fail(MAP_ERR_ARG, "map_batch_create: the union has too many vertices");
        off[c + 1] = (uint32_t)n_next;
        eoff[c + 1] = eoff[c] + mc[c];
        if (eoff[c + 1] > 0xFFFFFFFFull) return fail(MAP_ERR_ARG, "map_batch_create: the union has too many edges");
        woff[c + 1] = woff[c] + (ns[c] + 31) / 32;
    }
    const uint32_t N = off[count];
    const uint64_t M = eoff[count];
    const auto kind = [](const void *p) { return is_device_ptr(p) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; };
    int rc = create_graph(
        N, M, s, "map_batch_create",
        [&](map_graph *g, uint32_t **acc) -> int {
            g->ncomp = count;
            CK(cudaMallocAsync((void **)&g->comp, ((size_t)N + 4) * 4, s));
            CK(cudaMallocAsync((void **)&g->cs, (size_t)count * sizeof(mapk::CompState), s));
            CK(cudaMallocAsync((void **)&g->chist, (size_t)count * mapk::CH_CAP * 4, s));
            g->h_cs = static_cast<mapk::CompState *>(malloc((size_t)count * sizeof(mapk::CompState)));
            g->h_chist = static_cast<uint32_t *>(malloc((size_t)count * mapk::CH_CAP * 4));
            if (!g->h_cs || !g->h_chist) return fail(MAP_ERR_OOM, "map_batch_create: host allocation failed");
            // graph by graph: its rows and edges into the union, checked in its own ids, then offset
            uint32_t *staged = g->xbuf; // accepting bitmaps one after another (sum of words <= N)
            for (uint32_t c = 0; c < count; ++c) {
                const uint32_t n_c = ns[c];
                CK(cudaMemcpyAsync(g->rowptr + off[c], rowptrs[c], ((size_t)n_c + 1) * 4, kind(rowptrs[c]), s));
                if (mc[c]) CK(cudaMemcpyAsync(g->colidx + eoff[c], colidxs[c], (size_t)mc[c] * 4, kind(colidxs[c]), s));
                CK(cudaMemcpyAsync(staged + woff[c], acc_bits[c], (size_t)(woff[c + 1] - woff[c]) * 4, kind(acc_bits[c]),
                                   s));
                mapk::k_validate<<<grid_for(g, std::max<uint64_t>(mc[c], n_c), 1), 256, 0, s>>>(
                    n_c, g->rowptr + off[c], mc[c], g->colidx + eoff[c], &g->ctl->bad);
                mapk::k_add<<<grid_for(g, (uint64_t)n_c + 1, 1), 256, 0, s>>>(g->rowptr + off[c], (uint64_t)n_c + 1,
                                                                              (uint32_t)eoff[c]);
                if (mc[c])
                    mapk::k_add<<<grid_for(g, mc[c], 1), 256, 0, s>>>(g->colidx + eoff[c], mc[c], off[c]);
                CK(cudaGetLastError());
            }
            // per-graph offsets (in the list space, free at this point), graph of each vertex, union bitmap
            uint32_t *d_off = g->list, *d_woff = g->list + (count + 1);
            CK(cudaMemcpyAsync(d_off, off.data(), (size_t)(count + 1) * 4, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(d_woff, woff.data(), (size_t)(count + 1) * 4, cudaMemcpyHostToDevice, s));
            mapk::k_fill_comp<<<grid_for(g, N, 1), 256, 0, s>>>(N, d_off, count, g->comp);
            mapk::k_gather_acc<<<grid_for(g, g->words, 1), 256, 0, s>>>(N, d_off, d_woff, staged, g->comp, g->acc);
            // per-graph records: off, m (host), accepting count (device)
            std::vector<mapk::CompState> init(count);
            memset(init.data(), 0, init.size() * sizeof(mapk::CompState));
            for (uint32_t c = 0; c < count; ++c) {
                init[c].off = off[c];
                init[c].m = mc[c];
            }
            CK(cudaMemcpyAsync(g->cs, init.data(), (size_t)count * sizeof(mapk::CompState), cudaMemcpyHostToDevice, s));
            mapk::k_count_acc<<<grid_for(g, N, 1), 256, 0, s>>>(N, g->acc, g->comp, g->cs);
            CK(cudaGetLastError());
            CK(cudaStreamSynchronize(s)); // `init` and the offset vectors leave scope
            *acc = g->acc;
            return MAP_OK;
        },
        out);
    return rc;
}

int map_batch_run(map_graph *g, const map_opts *opts, map_result *results, uint32_t *map_out, uint32_t *rounds_out,
                  uint32_t rounds_cap)
{
    g_err.clear();
    if (!g || !results) return fail(MAP_ERR_ARG, "map_batch_run: NULL handle or results");
    if (!g->comp) return fail(MAP_ERR_ARG, "map_batch_run: this handle holds a single graph; use map_run");
    if (opts && opts->trace) return fail(MAP_ERR_ARG, "map_batch_run: traces are not offered for batches");
    map_opts o;
    memset(&o, 0, sizeof o);
    if (opts) o = *opts;
    o.rounds_out = nullptr;
    o.rounds_cap = 0;
    map_result all;
    const int rc = run_impl(g, &o, &all, map_out);
    if (rc != MAP_OK && rc != MAP_ERR_LIMIT && rc != MAP_ERR_TIMEOUT) return rc;
    const uint32_t count = g->ncomp;
    CK(cudaMemcpyAsync(g->h_cs, g->cs, (size_t)count * sizeof(mapk::CompState), cudaMemcpyDeviceToHost, g->stream));
    if (rounds_out && rounds_cap)
        CK(cudaMemcpyAsync(g->h_chist, g->chist, (size_t)count * mapk::CH_CAP * 4, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    int first = MAP_OK;
    for (uint32_t c = 0; c < count; ++c) {
        const mapk::CompState &S = g->h_cs[c];
        map_result &r = results[c];
        memset(&r, 0, sizeof r);
        r.verdict = S.verdict ? MAP_CYCLE : MAP_NO_CYCLE;
        r.witness = S.verdict ? S.witness - S.off : MAP_NONE;
        r.outer_iters = S.outer;
        r.inner_canonical = all.inner_canonical;
        r.inner_iters = S.inner_total;
        r.relaxations = S.relax;
        r.edges_total = S.m * (uint64_t)S.outer;
        r.device_ms = all.device_ms;
        r.accepting_left = S.nacc;
        r.launches = all.launches;
        r.status = S.status == mapk::ST_LIMIT ? MAP_ERR_LIMIT : S.status == mapk::ST_TIMEOUT ? MAP_ERR_TIMEOUT : MAP_OK;
        if (r.status != MAP_OK && first == MAP_OK) first = (int)r.status;
        if (rounds_out && rounds_cap) {
            const uint32_t k = std::min(std::min(S.outer, rounds_cap), mapk::CH_CAP);
            memcpy(rounds_out + (size_t)c * rounds_cap, g->h_chist + (size_t)c * mapk::CH_CAP, (size_t)k * 4);
        }
    }
    if (first != MAP_OK) return fail(first, "map_batch_run: a graph stopped at a limit or timeout");
    return MAP_OK;
}

} // extern "C"

// ============================================================================
// map_run_static: a whole MAP run that allocates nothing.
//
// Some callers cannot allocate device memory at run time: plug-ins whose host
// application hands them a fixed device budget and owns every allocation,
// real-time loops that must never enter an allocator, and code running where
// the allocator is off limits for other reasons.  For graphs up to
// MAP_STATIC_MAX_N vertices and MAP_STATIC_MAX_M edges, map_run_static keeps
// all of its work space in the file-scope device array below, which every GPU
// that loads this library holds until the process exits, and it calls no
// cudaMalloc, cudaFree or allocating routine.  It runs the same kernels as
// map_run, stepped from the host: it waits for its stream several times per
// call (to read the CSR's end offsets and the control block between steps), so
// it blocks, and it cannot be issued on a stream that is being captured.
// ============================================================================

namespace {

constexpr uint64_t ST_MAX_N = MAP_STATIC_MAX_N;
constexpr uint64_t ST_MAX_M = MAP_STATIC_MAX_M;
constexpr uint64_t ST_MAX_W = (ST_MAX_N + 31) / 32;
constexpr uint64_t ST_HIST = ST_MAX_N; // rounds per outer iteration: a run has at most n outer iterations
constexpr uint64_t st_pad(uint64_t words) { return (words + 63) & ~uint64_t(63); } // 256-byte pieces
// word offsets of the pieces of the scratch array
constexpr uint64_t ST_CTL = 0;
constexpr uint64_t ST_ROWPTR = ST_CTL + st_pad((sizeof(Ctl) + 3) / 4);
constexpr uint64_t ST_COLIDX = ST_ROWPTR + st_pad(ST_MAX_N + 5);
constexpr uint64_t ST_RROWPTR = ST_COLIDX + st_pad(ST_MAX_M + 4);
constexpr uint64_t ST_RCOL = ST_RROWPTR + st_pad(ST_MAX_N + 5);
constexpr uint64_t ST_RPOS = ST_RCOL + st_pad(ST_MAX_M + 4);
constexpr uint64_t ST_ELOG = ST_RPOS + st_pad(ST_MAX_M + 4);
constexpr uint64_t ST_ACC0 = ST_ELOG + st_pad(ST_MAX_N + 4);
constexpr uint64_t ST_ACC = ST_ACC0 + st_pad(ST_MAX_W + 4);
constexpr uint64_t ST_STALE = ST_ACC + st_pad(ST_MAX_W + 4);
constexpr uint64_t ST_MVAL = ST_STALE + st_pad(ST_MAX_W + 4);
constexpr uint64_t ST_LIST = ST_MVAL + st_pad(ST_MAX_N + 4);
constexpr uint64_t ST_FLIST = ST_LIST + st_pad(3 * ST_MAX_N);
constexpr uint64_t ST_REC = ST_FLIST + st_pad(3 * ST_MAX_N);
constexpr uint64_t ST_TOUCHED = ST_REC + st_pad(4 * ST_MAX_N);
constexpr uint64_t ST_XBUF = ST_TOUCHED + st_pad(ST_MAX_N);
constexpr uint64_t ST_HISTW = ST_XBUF + st_pad(ST_MAX_N);
constexpr uint64_t ST_SUMS = ST_HISTW + st_pad(ST_HIST);
constexpr uint64_t ST_WORDS = ST_SUMS + st_pad((ST_MAX_N + 1 + 1023) / 1024 + 4);
static_assert(ST_WORDS * 4 == MAP_STATIC_SCRATCH_BYTES, "MAP_STATIC_SCRATCH_BYTES in map.h is out of date");

// The work space of map_run_static.  In host code this name is only a host-side
// stand-in: kernels get the device address found by cudaGetSymbolAddress.
static __device__ __align__(256) uint32_t g_static_scratch[ST_WORDS];

constexpr int ST_MAX_DEVICES = 64;
std::atomic<uint32_t *> g_static_ptr[ST_MAX_DEVICES];

// the scratch array's device address on the current device (resolved once per device)
int static_scratch(uint32_t **out)
{
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= ST_MAX_DEVICES) return fail(MAP_ERR_ARG, "map_run_static: device %d not supported", dev);
    uint32_t *p = g_static_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        void *addr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&addr, g_static_scratch);
        if (e != cudaSuccess || !addr) {
            cudaGetLastError();
            return fail(MAP_ERR_CUDA, "map_run_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        }
        p = static_cast<uint32_t *>(addr);
        g_static_ptr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return MAP_OK;
}

// inclusive scan of at most ST_MAX_N + 1 words: two levels, tile sums in the scratch
int static_scan(uint32_t *x, uint64_t len, uint32_t *sums, cudaStream_t s)
{
    if (len <= 1) return MAP_OK;
    const uint64_t tiles = (len + 1023) / 1024;
    mapk::k_scan_tiles<<<(unsigned)tiles, 1024, 0, s>>>(x, len, tiles > 1 ? sums : nullptr);
    CK(cudaGetLastError());
    if (tiles > 1) { // tiles <= 1024: one tile of sums
        mapk::k_scan_tiles<<<1, 1024, 0, s>>>(sums, tiles, nullptr);
        mapk::k_scan_add<<<(unsigned)tiles, 1024, 0, s>>>(x, len, sums);
        CK(cudaGetLastError());
    }
    return MAP_OK;
}

int static_read_ctl(Ctl *h, const Ctl *d, cudaStream_t s)
{
    CK(cudaMemcpyAsync(h, d, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return MAP_OK;
}

} // namespace

static int run_static_impl(uint32_t n, const uint32_t *rowptr, const uint32_t *colidx, const uint32_t *acc_bits,
                           const map_opts *opts_in, map_result *res, uint32_t *map_out, void *cuda_stream)
{
    if (!res) return fail(MAP_ERR_ARG, "map_run_static: result is NULL");
    if (n == 0 || n > ST_MAX_N)
        return fail(MAP_ERR_ARG, "map_run_static: n = %u is outside [1, %llu] (MAP_STATIC_MAX_N); use map_create/map_run",
                    n, (unsigned long long)ST_MAX_N);
    if (!rowptr || !acc_bits) return fail(MAP_ERR_ARG, "map_run_static: rowptr and acc_bits are required");
    map_opts opts;
    memset(&opts, 0, sizeof opts);
    if (opts_in) opts = *opts_in;
    if (opts.sched > MAP_SCHED_ASYNC) return fail(MAP_ERR_ARG, "map_run_static: unknown schedule %u", opts.sched);
    if (opts.trace || (opts.flags & (MAP_FLAG_PROFILE | MAP_FLAG_FRONTIER_START)) || opts.repeat > 1)
        return fail(MAP_ERR_ARG, "map_run_static: traces, profiling, the frontier start and repeat are not offered here");
    const bool sync_sched = opts.sched == MAP_SCHED_SYNC;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    memset(res, 0, sizeof *res);

    uint32_t *base = nullptr;
    int rc = static_scratch(&base);
    if (rc) return rc;
    // m = rowptr[n], from host or device memory
    uint32_t m32 = 0, r0 = 0;
    CK(cudaMemcpyAsync(&m32, rowptr + n, 4, cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(&r0, rowptr, 4, cudaMemcpyDefault, s));
    CK(cudaStreamSynchronize(s));
    const uint64_t m = m32;
    if (r0 != 0) return fail(MAP_ERR_CSR, "map_run_static: rowptr[0] = %u, expected 0", r0);
    if (m > ST_MAX_M)
        return fail(MAP_ERR_ARG, "map_run_static: m = %llu edges exceeds %llu (MAP_STATIC_MAX_M); use map_create/map_run",
                    (unsigned long long)m, (unsigned long long)ST_MAX_M);
    if (m > 0 && !colidx) return fail(MAP_ERR_ARG, "map_run_static: colidx is NULL but m = %llu", (unsigned long long)m);

    // the pieces of the scratch array (every call reuses them)
    Ctl *ctl = reinterpret_cast<Ctl *>(base + ST_CTL);
    map_graph g; // a view of the scratch in the layout the launch helpers expect
    g.n = n;
    g.m = m;
    g.words = (n + 31) / 32;
    g.stream = s;
    g.G = pick_group(n, m);
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&g.sms, cudaDevAttrMultiProcessorCount, dev));
    const int occ = dense_occupancy();
    const int occ_r = rounds_occupancy();
    const uint64_t ntiles = ((uint64_t)n + mapk::WT_ROWS - 1) / mapk::WT_ROWS;
    g.dense_grid = (int)std::min<uint64_t>((ntiles + mapk::WT_WARPS - 1) / mapk::WT_WARPS, (uint64_t)g.sms * occ);
    g.rounds_grid = (int)std::min<uint64_t>(((uint64_t)n + 255) / 256, (uint64_t)g.sms * occ_r);
    g.check_grid = (int)std::min<uint64_t>(((uint64_t)n + 255) / 256, (uint64_t)g.sms * 4);
    g.rowptr = base + ST_ROWPTR;
    g.colidx = base + ST_COLIDX;
    g.rrowptr = base + ST_RROWPTR;
    g.rcol = base + ST_RCOL;
    g.rpos = base + ST_RPOS;
    g.elog = base + ST_ELOG;
    g.acc0 = base + ST_ACC0;
    g.acc = base + ST_ACC;
    g.stale = base + ST_STALE;
    g.mval = base + ST_MVAL;
    g.list = base + ST_LIST;
    g.flist = base + ST_FLIST;
    g.rec = reinterpret_cast<uint4 *>(base + ST_REC);
    g.touched = base + ST_TOUCHED;
    g.xbuf = base + ST_XBUF;
    g.hist = base + ST_HISTW;
    g.hist_cap = (uint32_t)ST_HIST;
    g.ctl = ctl;
    uint32_t *sums = base + ST_SUMS;
    const uint32_t W = g.words;

    // inputs into the scratch; everything that must start at zero is cleared
    // (the array keeps the previous call's contents)
    CK(cudaMemcpyAsync(g.rowptr, rowptr, ((size_t)n + 1) * 4, cudaMemcpyDefault, s));
    if (m) CK(cudaMemcpyAsync(g.colidx, colidx, m * 4, cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(g.acc, acc_bits, (size_t)W * 4, cudaMemcpyDefault, s));
    CK(cudaMemsetAsync(g.colidx + m, 0, 16, s));
    CK(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
    CK(cudaMemsetAsync(g.mval, 0, ((size_t)n + 4) * 4, s));
    CK(cudaMemsetAsync(g.rec, 0, (size_t)n * 16, s));
    CK(cudaMemsetAsync(g.stale, 0, ((size_t)W + 4) * 4, s));
    CK(cudaMemsetAsync(g.rrowptr, 0, ((size_t)n + 1) * 4, s));
    mapk::k_validate<<<grid_for(&g, m > n ? m : n, 1), 256, 0, s>>>(n, g.rowptr, m, g.colidx, &ctl->bad);
    mapk::k_acc_init<<<grid_for(&g, W, 1), 256, 0, s>>>(n, g.acc, g.acc0, &ctl->elim.v);
    CK(cudaGetLastError());
    Ctl h;
    if ((rc = static_read_ctl(&h, ctl, s))) return rc;
    if (h.bad) return fail(MAP_ERR_CSR, "map_run_static: invalid CSR (decreasing rowptr or colidx >= n)");
    const uint32_t nacc0 = h.elim.v;

    // readers (reverse CSR): in-degree histogram, scan, scatter
    mapk::k_indegree<<<grid_for(&g, m, 1), 256, 0, s>>>(m, g.colidx, g.rrowptr);
    CK(cudaGetLastError());
    if ((rc = static_scan(g.rrowptr, (uint64_t)n + 1, sums, s))) return rc;
    CK(cudaMemcpyAsync(g.list, g.rrowptr, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    DISPATCH_G(std::max(g.G, 16), (mapk::k_transpose<GG><<<grid_for(&g, n, GG), 256, 0, s>>>(n, g.rowptr, g.colidx, g.list,
                                                                             g.rcol, g.rpos)));
    mapk::k_pack_flags<<<grid_for(&g, m, 1), 256, 0, s>>>(m, g.colidx, g.acc);
    CK(cudaGetLastError());

    // the run, stepped from the host (no graph: instantiating one would allocate)
    const bool out_dev = map_out && is_device_ptr(map_out);
    memset(&h, 0, sizeof h);
    h.max_outer = opts.max_outer;
    h.max_inner = opts.max_inner ? opts.max_inner : n + 1;
    h.hist_cap = g.hist_cap;
    h.m = m;
    h.nacc0 = nacc0;
    h.rounds_hist = g.hist;
    h.out = out_dev ? map_out : g.xbuf;
    h.use_graph = 0;
    h.early_exit = (opts.flags & MAP_FLAG_EARLY_EXIT) ? 1 : 0;
    h.lc_passes = 1; // (pull rounds and one-block rounds stay off: their thresholds are zero)
    h.timeout_ns = (uint64_t)(opts.timeout_ms ? opts.timeout_ms : 120000u) * 1000000ull;
    h.witness.v = mapk::NONE;
    CK(cudaMemcpyAsync(ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(g.acc, g.acc0, (size_t)W * 4, cudaMemcpyDeviceToDevice, s));
    const mapk::Handles none{};
    mapk::k_run_begin<<<1, 32, 0, s>>>(ctl, none);
    CK(cudaGetLastError());
    if ((rc = static_read_ctl(&h, ctl, s))) return rc;
    uint64_t launches = 1;
    while (h.outer_go) {
        if ((rc = launch_dense(&g, s, none)) || (rc = launch_rounds(&g, s, sync_sched, none)) ||
            (rc = launch_check(&g, s, none)))
            return rc;
        launches += 3;
        if ((rc = static_read_ctl(&h, ctl, s))) return rc;
    }
    if ((rc = launch_restore(&g, s)) || (rc = launch_export(&g, s, nullptr))) return rc;
    launches += 2;
    if ((rc = static_read_ctl(&h, ctl, s))) return rc;
    res->verdict = h.verdict ? MAP_CYCLE : MAP_NO_CYCLE;
    res->witness = h.verdict ? h.witness.v : MAP_NONE;
    res->outer_iters = h.outer;
    res->inner_canonical = (sync_sched && !h.early_hit) ? 1 : 0;
    res->inner_iters = h.inner_total;
    res->relaxations = h.relax.v;
    res->edges_total = m * (uint64_t)h.outer;
    res->accepting_left = h.nacc;
    res->launches = launches;
    res->frontier_rows = h.frontier_rows.v;
    const uint32_t nh = std::min<uint32_t>(h.outer, g.hist_cap);
    if (opts.rounds_out && nh)
        CK(cudaMemcpyAsync(opts.rounds_out, g.hist, (size_t)std::min(nh, opts.rounds_cap) * 4, cudaMemcpyDefault, s));
    if (map_out && !out_dev) CK(cudaMemcpyAsync(map_out, g.xbuf, (size_t)n * 4, cudaMemcpyDefault, s));
    CK(cudaStreamSynchronize(s));
    if (h.status == mapk::ST_LIMIT) return fail(MAP_ERR_LIMIT, "map_run_static: max_outer or max_inner reached");
    if (h.status == mapk::ST_TIMEOUT) return fail(MAP_ERR_TIMEOUT, "map_run_static: stopped after the timeout");
    return MAP_OK;
}

extern "C" int map_run_static(uint32_t n, const uint32_t *rowptr, const uint32_t *colidx, const uint32_t *acc_bits,
                              const map_opts *opts, map_result *res, uint32_t *map_out, void *cuda_stream)
{
    g_err.clear();
    const int rc = run_static_impl(n, rowptr, colidx, acc_bits, opts, res, map_out, cuda_stream);
    if (res) res->status = (uint32_t)rc; // as map_run: the run's status beside what was computed
    return rc;
}

// ============================================================================
// Serving: a request loop with continuous admission and batching (map_server_*).
//
// Jobs are copied at submission and queued.  Each of the server's worker
// threads owns a CUDA stream; a worker takes the oldest queued job as soon as
// the job's device footprint fits into what is left of the memory budget, with
// the jobs queued right behind it that may share its run, and runs them on its
// stream: one job alone (map_create, map_run, map output, map_destroy), several
// as one batched run (map_batch_create, map_batch_run).  Jobs that arrive while
// others are on the GPU are admitted as workers and memory free up, and the work
// of admitted jobs overlaps on the device.  Allocation is stream-ordered, so one
// job's set-up does not stall the others.
// ============================================================================

namespace {

// Pinned host arena of a server: a job's inputs are copied in once at submission
// (into memory that is already mapped and pinned, so the copy to the device is a
// DMA transfer from there) and its map comes back into the same slot.  First fit
// over a free list of 256-byte pieces, used under the server's lock.
struct PinnedArena {
    uint8_t *base = nullptr;
    std::map<size_t, size_t> free; // offset -> bytes
    static size_t round(size_t b) { return (b + 255) & ~size_t(255); }
    void init(size_t bytes)
    {
        if (bytes && cudaMallocHost((void **)&base, bytes) == cudaSuccess) {
            free[0] = bytes;
        } else {
            cudaGetLastError();
            base = nullptr;
        }
    }
    uint32_t *alloc(size_t bytes)
    {
        if (!base) return nullptr;
        bytes = round(bytes);
        for (auto it = free.begin(); it != free.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, rest = it->second - bytes;
            free.erase(it);
            if (rest) free[off + bytes] = rest;
            return reinterpret_cast<uint32_t *>(base + off);
        }
        return nullptr;
    }
    void release(uint32_t *p, size_t bytes)
    {
        const size_t off = reinterpret_cast<uint8_t *>(p) - base;
        auto it = free.emplace(off, round(bytes)).first;
        auto nx = std::next(it);
        if (nx != free.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free.erase(nx);
        }
        if (it != free.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free.erase(it);
            }
        }
    }
    ~PinnedArena()
    {
        if (base) cudaFreeHost(base);
    }
};

struct ServerJob {
    uint64_t id = 0;
    uint32_t n = 0;
    uint64_t m = 0;
    uint32_t *pin = nullptr; // arena slot: rowptr, colidx, accepting words; later the map
    size_t pin_bytes = 0;
    std::vector<uint32_t> rowptr, colidx, acc; // inputs when the arena had no room
    map_opts opts{};
    size_t footprint = 0;
    bool done = false;
    int status = MAP_OK;
    map_result res{};
    std::vector<uint32_t> map;
    std::string err;
    std::chrono::steady_clock::time_point t_submit;
    int inject_alloc = 0; // test hook: the k-th device allocation of its map_create fails
};

// jobs that may share a batched run, and the size of one
constexpr uint32_t kBatchFlags = MAP_FLAG_FRONTIER_START | MAP_FLAG_DENSE_START | MAP_FLAG_PUSH | MAP_FLAG_PULL;
constexpr uint32_t kMaxBatchJobs = 128;
constexpr uint64_t kMaxBatchVertices = 1ull << 26;
// a batched run lasts as long as its slowest graph: larger jobs run alone, so that the small
// ones batched together do not wait for them
constexpr uint32_t kMaxBatchedJobN = 1u << 20;

// device bytes of a graph: the allocations of create_graph
size_t graph_footprint(uint64_t n, uint64_t m)
{
    const uint64_t W = (n + 31) / 32;
    // (colidx, rcol, rpos, and the set-up's rank array: 4 words per entry at the peak)
    const uint64_t words = 2 * (n + 5) + 4 * (m + 4) + 3 * (W + 4) + (n + 4) + 2 * 3 * (n + 4) + 4 * (n + 4) +
                           3 * (n + 4) + (1u << 16);
    // the changed-vertex bitmaps of pull rounds
    return (size_t)(words + 3 * (W + 4)) * 4 + sizeof(Ctl) + (1u << 20);
}

} // namespace

struct map_server {
    std::map<uint64_t, int> inject; // MAPGPU_INJECT_OOM: job id -> allocation that fails
    size_t budget = 0;
    size_t used = 0;
    int device = 0;
    uint32_t slots = 1;
    uint32_t max_batch = kMaxBatchJobs; // jobs per run at most (map_server_batch_limit)
    uint32_t idle = 0;                  // workers waiting for a job
    bool stop = false;
    uint64_t next_id = 1;
    std::mutex mu;
    std::condition_variable cv_work;
    std::deque<ServerJob *> queue;
    std::unordered_map<uint64_t, ServerJob *> jobs;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    PinnedArena arena;
};

namespace {

// a served job's inputs: its arena slot (page-locked), or its own vectors
void job_inputs(const ServerJob *job, const uint32_t *&rp, const uint32_t *&ci, const uint32_t *&ab)
{
    if (job->pin) {
        rp = job->pin;
        ci = job->m ? job->pin + job->n + 1 : nullptr;
        ab = job->pin + job->n + 1 + job->m;
    } else {
        rp = job->rowptr.data();
        ci = job->m ? job->colidx.data() : nullptr;
        ab = job->acc.data();
    }
}

// Jobs that may share a batched run: the batch engine gives every graph exactly its result alone
// under the options it offers (schedule, start, push / pull); early exit, limits, profiling and an
// injected allocation failure keep a job to itself.

bool batchable(const ServerJob *j)
{
    return j->n <= kMaxBatchedJobN && j->inject_alloc == 0 && (j->opts.flags & ~kBatchFlags) == 0 &&
           j->opts.max_outer == 0 && j->opts.max_inner == 0;
}

bool same_run(const map_opts &a, const map_opts &b)
{
    return a.sched == b.sched && a.flags == b.flags && a.timeout_ms == b.timeout_ms;
}

// grow a worker's page-locked staging buffer to at least `words` (allocating page-locked memory
// synchronises the device, so it grows by a quarter more than asked and is kept)
void ensure_stage(uint32_t *&stage, size_t &stage_words, size_t words)
{
    if (words <= stage_words) return;
    if (stage) cudaFreeHost(stage);
    stage = nullptr;
    stage_words = 0;
    if (cudaMallocHost((void **)&stage, words * 4 * 5 / 4) == cudaSuccess) stage_words = words * 5 / 4;
    else cudaGetLastError();
}

// The fix-point kernel is a cooperative launch: with every resident slot of the device (the
// single-graph shape) a job's rounds cannot run beside another job's.  Each worker's run takes an
// even share of the slots, so the rounds of all workers fit side by side.
void share_rounds(map_server *sv, map_graph *g)
{
    if (sv->slots <= 1) return;
    const int share = std::max(1, (int)((int64_t)g->sms * g->occ_rounds / (int64_t)sv->slots));
    g->rounds_grid = std::min(g->rounds_grid, share);
}

using Clock = std::chrono::steady_clock;

void finish_job(map_server *sv, ServerJob *job, int rc, Clock::time_point t_take, Clock::time_point t_created,
                uint32_t batch_jobs)
{
    using ms = std::chrono::duration<double, std::milli>;
    const auto t_end = Clock::now();
    if (rc != MAP_OK && job->err.empty()) job->err = g_err;
    job->res.queue_ms = ms(t_take - job->t_submit).count();
    job->res.setup_ms = ms(t_created - t_take).count();
    job->res.run_ms = ms(t_end - t_created).count();
    job->res.status = (uint32_t)rc;
    job->res.batch_jobs = batch_jobs;
    // the job's inputs are not needed any more
    std::vector<uint32_t>().swap(job->rowptr);
    std::vector<uint32_t>().swap(job->colidx);
    std::vector<uint32_t>().swap(job->acc);
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        job->status = rc;
        job->done = true;
        sv->used -= job->footprint;
    }
    sv->cv_work.notify_all();
}

// one job alone: map_create, map_run, map output, map_destroy
void serve_one(map_server *sv, cudaStream_t stream, ServerJob *job, uint32_t *&stage, size_t &stage_words)
{
    const uint32_t *rp, *ci, *ab;
    job_inputs(job, rp, ci, ab);
    // a job outside the arena: its inputs into this worker's page-locked staging buffer, so that
    // the set-up reads them over the link directly
    if (!job->pin) {
        ensure_stage(stage, stage_words, (size_t)job->n + 1 + job->m + job->acc.size());
        if (stage) {
            uint32_t *p = stage;
            memcpy(p, rp, ((size_t)job->n + 1) * 4);
            rp = p;
            p += job->n + 1;
            if (job->m) {
                memcpy(p, ci, job->m * 4);
                ci = p;
                p += job->m;
            }
            memcpy(p, ab, job->acc.size() * 4);
            ab = p;
        }
    }
    NvtxRange job_range("served job");
    const auto t_take = Clock::now();
    map_graph *g = nullptr;
    t_inject_alloc = job->inject_alloc;
    int rc = map_create(job->n, rp, ci, ab, stream, &g);
    t_inject_alloc = 0;
    const auto t_created = Clock::now();
    if (rc == MAP_OK) {
        share_rounds(sv, g);
        // the whole run as one CUDA graph; the map comes back by DMA into page-locked memory (the
        // job's arena slot, read out by map_poll, or the staging buffer: map_create has consumed
        // the inputs)
        if (job->pin) {
            rc = run_impl(g, &job->opts, &job->res, job->pin);
        } else {
            job->map.resize(job->n);
            rc = run_impl(g, &job->opts, &job->res, stage ? stage : job->map.data());
            if (stage && rc == MAP_OK) memcpy(job->map.data(), stage, (size_t)job->n * 4);
        }
        map_destroy(g);
    }
    finish_job(sv, job, rc, t_take, t_created, 1);
}

// Continuous batching: jobs that were queued together and may share a run are joined into one
// batched run (map_batch_create / map_batch_run), every one with exactly its own result.  If the
// batch cannot be set up (memory, or an invalid graph among them), each job runs alone, so a
// failure is reported by the job that causes it only.
void serve_batch(map_server *sv, cudaStream_t stream, std::vector<ServerJob *> &batch, uint32_t *&stage,
                 size_t &stage_words)
{
    const uint32_t count = (uint32_t)batch.size();
    std::vector<uint32_t> ns(count);
    std::vector<const uint32_t *> rps(count), cis(count), abs(count);
    uint64_t total_n = 0;
    for (uint32_t c = 0; c < count; ++c) {
        ns[c] = batch[c]->n;
        job_inputs(batch[c], rps[c], cis[c], abs[c]);
        total_n += batch[c]->n;
    }
    NvtxRange job_range("served batch");
    const auto t_take = Clock::now();
    map_graph *g = nullptr;
    int rc = map_batch_create(count, ns.data(), rps.data(), cis.data(), abs.data(), stream, &g);
    const auto t_created = Clock::now();
    if (rc != MAP_OK) {
        for (ServerJob *job : batch) serve_one(sv, stream, job, stage, stage_words);
        return;
    }
    share_rounds(sv, g);
    // the union's map vectors, one after another, into page-locked staging (pageable when it
    // cannot grow), then into each job's slot
    ensure_stage(stage, stage_words, total_n);
    std::vector<uint32_t> pageable;
    uint32_t *maps = stage;
    if (!maps) {
        pageable.resize(total_n);
        maps = pageable.data();
    }
    std::vector<map_result> res(count);
    const int brc = map_batch_run(g, &batch[0]->opts, res.data(), maps, nullptr, 0);
    const std::string err = g_err;
    map_destroy(g);
    if (brc != MAP_OK && brc != MAP_ERR_LIMIT && brc != MAP_ERR_TIMEOUT) { // no per-graph result
        for (ServerJob *job : batch) serve_one(sv, stream, job, stage, stage_words);
        return;
    }
    uint64_t off = 0;
    for (uint32_t c = 0; c < count; ++c) {
        ServerJob *job = batch[c];
        const int rc_c = (int)res[c].status; // (a limit or timeout: each graph's own status)
        job->res = res[c];
        if (rc_c == MAP_OK) {
            if (job->pin) {
                memcpy(job->pin, maps + off, (size_t)job->n * 4);
            } else {
                job->map.assign(maps + off, maps + off + job->n);
            }
        } else {
            job->err = err;
        }
        off += job->n;
        finish_job(sv, job, rc_c, t_take, t_created, count);
    }
}

void server_worker(map_server *sv, cudaStream_t stream)
{
    cudaSetDevice(sv->device);
    uint32_t *stage = nullptr; // page-locked staging for inputs and maps
    size_t stage_words = 0;
    struct Release {
        uint32_t *&p;
        ~Release()
        {
            if (p) cudaFreeHost(p);
        }
    } release{stage};
    for (;;) {
        std::vector<ServerJob *> batch;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            ++sv->idle;
            sv->cv_work.wait(lk, [&] {
                if (sv->stop) return true;
                if (sv->queue.empty()) return false;
                const size_t fp = sv->queue.front()->footprint;
                return sv->used + fp <= sv->budget || sv->used == 0; // a job larger than the budget runs alone
            });
            --sv->idle;
            if (sv->stop && sv->queue.empty()) return;
            if (sv->queue.empty()) continue;
            ServerJob *job = sv->queue.front();
            sv->queue.pop_front();
            sv->used += job->footprint;
            batch.push_back(job);
            // the jobs queued right behind it join its run while they may share it and fit, when no
            // other worker is waiting to take them (a load the workers keep up with runs job by
            // job, at the latency of a job alone)
            if (batchable(job) && sv->idle == 0) {
                // (jobs that cannot join stay queued in their order for the next worker)
                uint64_t un = job->n, um = job->m;
                uint32_t looked = 0;
                for (auto it = sv->queue.begin(); it != sv->queue.end() && batch.size() < sv->max_batch &&
                                                  looked < 4 * sv->max_batch;
                     ++looked) {
                    ServerJob *j = *it;
                    if (!batchable(j) || !same_run(j->opts, job->opts) || un + j->n > kMaxBatchVertices ||
                        um + j->m >= 0xFFFFFFFFull) {
                        ++it;
                        continue;
                    }
                    if (sv->used + j->footprint > sv->budget) break; // the budget is full
                    it = sv->queue.erase(it);
                    sv->used += j->footprint;
                    un += j->n;
                    um += j->m;
                    batch.push_back(j);
                }
            }
        }
        if (batch.size() == 1) serve_one(sv, stream, batch[0], stage, stage_words);
        else serve_batch(sv, stream, batch, stage, stage_words);
    }
}

} // namespace

extern "C" {

int map_server_create(size_t hbm_budget_bytes, uint32_t max_slots, map_server **out)
{
    g_err.clear();
    if (!out) return fail(MAP_ERR_ARG, "map_server_create: out is NULL");
    *out = nullptr;
    if (max_slots == 0 || max_slots > 64) return fail(MAP_ERR_ARG, "map_server_create: max_slots must be 1..64");
    map_server *sv = new (std::nothrow) map_server;
    if (!sv) return fail(MAP_ERR_OOM, "map_server_create: host allocation failed");
    CK(cudaGetDevice(&sv->device));
    if (hbm_budget_bytes == 0) {
        size_t free_b = 0, total_b = 0;
        CK(cudaMemGetInfo(&free_b, &total_b));
        hbm_budget_bytes = free_b / 2;
    }
    sv->budget = hbm_budget_bytes;
    sv->slots = max_slots;
    if (const char *e = getenv("MAPGPU_INJECT_OOM")) { // "job:k,job:k" (test hook)
        const char *q = e;
        while (*q) {
            char *end = nullptr;
            const unsigned long long job = strtoull(q, &end, 10);
            if (end == q || *end != ':') break;
            q = end + 1;
            const long k = strtol(q, &end, 10);
            if (end == q) break;
            if (k > 0) sv->inject[job] = (int)k;
            q = end;
            if (*q == ',') ++q;
        }
    }
    ctl_slots().reserve(2 * (size_t)max_slots); // control-block mirrors for the workers' graphs, allocated now
    // pinned staging for queued and finished jobs: a quarter of the device budget, at most 2 GiB
    sv->arena.init(std::min<size_t>(hbm_budget_bytes / 4, (size_t)2 << 30));
    for (uint32_t i = 0; i < max_slots; ++i) {
        cudaStream_t st;
        cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            cudaGetLastError();
            map_server_destroy(sv);
            return fail(MAP_ERR_CUDA, "map_server_create: stream: %s", cudaGetErrorString(e));
        }
        sv->streams.push_back(st);
    }
    for (uint32_t i = 0; i < max_slots; ++i) sv->workers.emplace_back(server_worker, sv, sv->streams[i]);
    *out = sv;
    return MAP_OK;
}

int map_submit(map_server *sv, uint32_t n, const uint32_t *rowptr, const uint32_t *colidx, const uint32_t *acc_bits,
               const map_opts *opts, uint64_t *job_id)
{
    g_err.clear();
    if (!sv || !job_id) return fail(MAP_ERR_ARG, "map_submit: NULL server or job_id");
    if (n == 0 || n >= 0x7FFFFFFFu || !rowptr || !acc_bits) return fail(MAP_ERR_ARG, "map_submit: bad graph");
    if (opts && opts->trace) return fail(MAP_ERR_ARG, "map_submit: traces are not offered for served jobs");
    if (opts && opts->repeat > 1) return fail(MAP_ERR_ARG, "map_submit: repeat is not offered for served jobs");
    if (is_device_ptr(rowptr) || is_device_ptr(colidx) || is_device_ptr(acc_bits))
        return fail(MAP_ERR_ARG, "map_submit: inputs must be host memory (the job is copied at submission)");
    const uint64_t m = rowptr[n];
    if (m > 0 && !colidx) return fail(MAP_ERR_ARG, "map_submit: colidx is NULL");
    ServerJob *job = new (std::nothrow) ServerJob;
    if (!job) return fail(MAP_ERR_OOM, "map_submit: host allocation failed");
    job->n = n;
    job->m = m;
    const size_t W = (n + 31) / 32, bytes = ((size_t)n + 1 + m + W) * 4;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        job->pin = sv->arena.alloc(bytes);
    }
    if (job->pin) { // one copy, into pinned memory
        job->pin_bytes = bytes;
        memcpy(job->pin, rowptr, ((size_t)n + 1) * 4);
        if (m) memcpy(job->pin + n + 1, colidx, m * 4);
        memcpy(job->pin + n + 1 + m, acc_bits, W * 4);
    } else {
        try {
            job->rowptr.assign(rowptr, rowptr + (size_t)n + 1);
            job->colidx.assign(colidx, colidx + m);
            job->acc.assign(acc_bits, acc_bits + W);
        } catch (...) {
            delete job;
            return fail(MAP_ERR_OOM, "map_submit: host allocation failed");
        }
    }
    if (opts) job->opts = *opts;
    job->opts.rounds_out = nullptr;
    job->opts.rounds_cap = 0;
    job->footprint = graph_footprint(n, m);
    job->t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        job->id = sv->next_id++;
        const auto inj = sv->inject.find(job->id);
        if (inj != sv->inject.end()) job->inject_alloc = inj->second;
        sv->jobs[job->id] = job;
        sv->queue.push_back(job);
        *job_id = job->id;
    }
    sv->cv_work.notify_all();
    return MAP_OK;
}

int map_server_batch_limit(map_server *sv, uint32_t max_jobs)
{
    g_err.clear();
    if (!sv || max_jobs == 0 || max_jobs > 1024)
        return fail(MAP_ERR_ARG, "map_server_batch_limit: NULL server or max_jobs outside 1..1024");
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->max_batch = max_jobs;
    return MAP_OK;
}

int map_poll(map_server *sv, uint64_t job_id, map_result *res, uint32_t *map_out)
{
    g_err.clear();
    if (!sv) return fail(MAP_ERR_ARG, "map_poll: NULL server");
    ServerJob *job = nullptr;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->jobs.find(job_id);
        if (it == sv->jobs.end()) return fail(MAP_ERR_ARG, "map_poll: unknown job %llu", (unsigned long long)job_id);
        if (!it->second->done) return MAP_ERR_NOT_READY;
        job = it->second;
        sv->jobs.erase(it);
    }
    if (res) *res = job->res;
    if (map_out && job->status == MAP_OK) memcpy(map_out, job->pin ? job->pin : job->map.data(), (size_t)job->n * 4);
    if (job->pin) {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->arena.release(job->pin, job->pin_bytes);
    }
    const int rc = job->status;
    if (rc != MAP_OK) fail(rc, "%s", job->err.c_str());
    delete job;
    return rc;
}

int map_server_destroy(map_server *sv)
{
    if (!sv) return MAP_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    for (auto &t : sv->workers) t.join();
    for (auto st : sv->streams) cudaStreamDestroy(st);
    for (auto &kv : sv->jobs) delete kv.second;
    for (ServerJob *j : sv->queue)
        if (!sv->jobs.count(j->id)) delete j;
    delete sv;
    return MAP_OK;
}

} // extern "C"
