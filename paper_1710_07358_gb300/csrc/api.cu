// C ABI of libpr.so (declared in include/pr.h): argument validation,
// per-(device, stream) workspaces, launch-configuration lookup and tuning,
// and the host-memory pipeline.  All arithmetic runs in the kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/pr.h"
#include "axis.cuh"
#include "kernels.cuh"
#include "registry.h"
#include "scan.cuh"
#include "search.cuh"

namespace pr {

// ------------------------------------------------------------------------
// Kernel registry
// ------------------------------------------------------------------------

bool KernelKey::operator<(const KernelKey& o) const {
    return std::tie(kind, dtype, op, prec, aux, unroll, vb) <
           std::tie(o.kind, o.dtype, o.op, o.prec, o.aux, o.unroll, o.vb);
}

static std::map<KernelKey, KernelEntry>& table() {
    static std::map<KernelKey, KernelEntry> t;
    return t;
}
void reg_add(const KernelKey& k, const KernelEntry& e) { table()[k] = e; }
const KernelEntry* reg_find(const KernelKey& k) {
    auto it = table().find(k);
    return it == table().end() ? nullptr : &it->second;
}

void ensure_registered() {
    static std::once_flag once;
    std::call_once(once, [] {
        register_f32();
        register_f32_seg();
        register_f16();
        register_bf16();
        register_f64();
        register_i32();
        register_u32();
        register_i64();
        register_backward();
        register_scan();
    });
}

// ------------------------------------------------------------------------
// Errors
// ------------------------------------------------------------------------

static thread_local std::string g_msg;

pr_status fail(pr_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_msg = buf;
    return s;
}

#define PR_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return fail(PR_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// ------------------------------------------------------------------------
// Host-side fault injection (test hook, pr_debug_inject_fault)
// ------------------------------------------------------------------------
//
// An armed fault makes the library's next device allocation (PR_FAULT_ALLOC)
// or next kernel launch (PR_FAULT_LAUNCH), after `after` of them have passed,
// fail as if the CUDA call had failed: the entry point returns the status it
// returns for a real failure, with nothing further enqueued.  One-shot.  The
// injection happens on the host, before the CUDA call, so no GPU is faulted.

static std::atomic<int> g_fault_site{PR_FAULT_NONE};
static std::mutex g_fault_mu;
static int g_fault_after = 0;

static bool inject(int site) {
    if (g_fault_site.load(std::memory_order_relaxed) != site) return false;
    std::lock_guard<std::mutex> lk(g_fault_mu);
    if (g_fault_site.load(std::memory_order_relaxed) != site) return false;
    if (g_fault_after > 0) {
        g_fault_after--;
        return false;
    }
    g_fault_site.store(PR_FAULT_NONE);
    return true;
}

#define PR_INJECT_LAUNCH() \
    do { if (inject(PR_FAULT_LAUNCH)) return fail(PR_ERR_CUDA, "kernel launch failed (injected by the test hook)"); } while (0)
#define PR_INJECT_ALLOC() \
    do { if (inject(PR_FAULT_ALLOC)) return fail(PR_ERR_NOMEM, "device allocation failed (injected by the test hook)"); } while (0)

// ------------------------------------------------------------------------
// Types
// ------------------------------------------------------------------------

static bool valid_dtype(int d) { return d >= PR_F32 && d <= PR_I64; }
static bool valid_op(int o) { return o >= PR_SUM && o <= PR_XOR; }
static bool is_float(int d) { return d == PR_F32 || d == PR_F16 || d == PR_BF16 || d == PR_F64; }
static int elem_size(int d) {
    switch (d) {
    case PR_F16: case PR_BF16: return 2;
    case PR_F64: case PR_I64: return 8;
    default: return 4;
    }
}
static int out_size(int d, int op) { return elem_size((int)pr_out_dtype((pr_dtype)d, (pr_op)op)); }

// ------------------------------------------------------------------------
// Devices and workspaces
// ------------------------------------------------------------------------

struct DevInfo {
    int sms = 0;
    std::string name;
};

static std::mutex g_mu;
static std::map<int, DevInfo> g_dev;
struct WsRec {
    Workspace ws;
    void* base;
    size_t bytes;
    void* axis = nullptr;    // axis-reduction partials, grown on demand
    size_t axis_bytes = 0;
    void* scan = nullptr;    // scan tile states + counters, grown on demand
    size_t scan_tiles = 0;
    void* search = nullptr;  // line-search state + evaluation partials, made on first use
};
static std::map<std::pair<int, cudaStream_t>, WsRec> g_ws;

static pr_status device_info(DevInfo* out, int* dev_out) {
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_dev.find(dev);
    if (it == g_dev.end()) {
        DevInfo d;
        PR_CUDA(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
        cudaDeviceProp p;
        PR_CUDA(cudaGetDeviceProperties(&p, dev));
        d.name = p.name;
        it = g_dev.emplace(dev, d).first;
    }
    *out = it->second;
    if (dev_out) *dev_out = dev;
    return PR_OK;
}

static size_t ws_bytes(int gmax) { return (size_t)3 * gmax * kSlot + (size_t)(gmax + 64) * 4; }

static pr_status get_ws(cudaStream_t st, Workspace* out) {
    DevInfo di;
    int dev;
    pr_status s = device_info(&di, &dev);
    if (s != PR_OK) return s;
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_pair(dev, st);
    auto it = g_ws.find(key);
    if (it != g_ws.end()) {
        *out = it->second.ws;
        return PR_OK;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    PR_CUDA(cudaStreamIsCapturing(st, &cap));
    if (cap != cudaStreamCaptureStatusNone)
        return fail(PR_ERR_INVALID, "no workspace for this stream yet: call pr_prepare(stream) before graph capture");
    const int gmax = di.sms * 32;
    const size_t bytes = ws_bytes(gmax);
    void* base = nullptr;
    PR_INJECT_ALLOC();
    if (cudaMalloc(&base, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(PR_ERR_NOMEM, "workspace allocation of %zu bytes failed", bytes);
    }
    PR_CUDA(cudaMemsetAsync(base, 0, bytes, st));
    Workspace ws;
    char* b = static_cast<char*>(base);
    ws.partials = b;
    ws.head = b + (size_t)gmax * kSlot;
    ws.tail = b + (size_t)2 * gmax * kSlot;
    unsigned* u = reinterpret_cast<unsigned*>(b + (size_t)3 * gmax * kSlot);
    ws.seg_cnt = u;
    ws.counter = u + gmax;
    ws.chunk_ctr = u + gmax + 1;
    ws.blk_done = u + gmax + 2;
    ws.err = reinterpret_cast<int*>(u + gmax + 32);
    ws.gmax = gmax;
    g_ws[key] = WsRec{ws, base, bytes};
    *out = ws;
    return PR_OK;
}

// ------------------------------------------------------------------------
// Launch configurations
// ------------------------------------------------------------------------

static int bucket_of(int64_t n) {
    int b = 0;
    while (b < 62 && ((int64_t)1 << (b + 1)) <= n) b++;
    return n <= 0 ? 0 : b;
}

using CfgKey = std::tuple<int, int, int, int, int>;  // kind, dtype, op, precision, bucket
static std::map<CfgKey, pr_config> g_tuned;

// Built-in defaults (measured on GB300: two 32-byte loads in flight per thread
// at 1024 resident threads per SM streams at the HBM limit for the plain
// reduction); pr_autotune / pr_tune_load refine them per (dtype, op, size).
static pr_config default_cfg(int kind, int dtype, int op, int prec) {
    (void)prec;
    if (kind == PR_KIND_BACKWARD) return pr_config{512, 4, 4, 16};
    if (kind == PR_KIND_ROWS) return pr_config{512, 2, 2, 32};
    if (kind == PR_KIND_AXIS) return pr_config{256, 4, 2, 32};
    // the split fp64 product keeps two accumulators' state per slot: two tiles in flight
    if (kind == PR_KIND_SEGMENTED) return dtype == PR_F64 && op == PR_PROD ? pr_config{256, 2, 2, 32}
                                                                          : pr_config{256, 2, 4, 32};
    return pr_config{512, 2, 2, 32};
}

// The segmented kernel is built for blocks of at most 512 threads (it keeps
// two tiles of vectors per thread in registers).
static bool cfg_valid(const pr_config& c, int kind = PR_KIND_REDUCE) {
    if (c.block < 64 || c.block > (kind == PR_KIND_SEGMENTED ? 512 : 1024) || c.block % 32) return false;
    if (c.blocks_per_sm < 1 || c.blocks_per_sm > 32) return false;
    if (c.unroll != 2 && c.unroll != 4) return false;
    return c.vec_bytes == 16 || c.vec_bytes == 32;
}

static pr_config lookup_cfg(int kind, int dtype, int op, int prec, int64_t n) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_tuned.find(CfgKey{kind, dtype, op, prec, bucket_of(n)});
    return it != g_tuned.end() ? it->second : default_cfg(kind, dtype, op, prec);
}

static std::map<std::tuple<int, const void*, int>, int> g_occ;

// Resident blocks per SM of `fn` at `block` threads and `smem` bytes of
// dynamic shared memory (allowed above the 48 KB default on first use), per
// device.
static pr_status occupancy(const void* fn, int block, int* bps, size_t smem = 0) {
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_tuple(dev, fn, block);
    auto it = g_occ.find(key);
    if (it == g_occ.end()) {
        if (smem > 48 * 1024)
            PR_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int nb = 0;
        PR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, smem));
        it = g_occ.emplace(key, nb).first;
    }
    *bps = it->second;
    return PR_OK;
}

static std::map<const void*, int> g_maxthr;
static std::map<const void*, size_t> g_local;

// Bytes of local memory (register spills) a thread of `fn` uses.
static size_t local_bytes(const void* fn) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_local.find(fn);
    if (it != g_local.end()) return it->second;
    cudaFuncAttributes fa;
    size_t v = 0;
    if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess) v = fa.localSizeBytes;
    else cudaGetLastError();
    g_local.emplace(fn, v);
    return v;
}

// The configuration with its block size clamped to the kernel's compiled limit
// (a trait with a large per-thread state compiles for at most 512 threads).
static pr_config fit_block(const KernelEntry* e, pr_config c) {
    int mt = 1024;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_maxthr.find(e->fn);
        if (it != g_maxthr.end()) {
            mt = it->second;
        } else {
            cudaFuncAttributes fa;
            if (cudaFuncGetAttributes(&fa, e->fn) == cudaSuccess) {
                mt = fa.maxThreadsPerBlock;
                g_maxthr.emplace(e->fn, mt);
            } else {
                cudaGetLastError();
            }
        }
    }
    if (c.block > mt) c.block = mt / 32 * 32;
    return c;
}

// Claimed tail of the plain reduction.  SMs finish equal static shares of a
// grid-stride loop a few microseconds apart (more, the longer the loop), so
// a static split ends when the slowest SM does.  Inputs from kTailMinBytes
// on leave about a tenth of their vectors (past a multiple of the grid's
// stride) to tiles of about kTileBytes that blocks claim.  Measured on
// GB300, fp32 sum, 1024 x 1 blocks, A/B in one process: 1 GiB 153.6 ->
// 151.7 us, 4 GiB 580.2 -> 574.5 us; 512 MiB 82.0 -> 82.0 us and 256 MiB
// 45.9 -> 47.4 us, where the tiles' barriers cost what the balance saves.
// A fifth measured no better than a tenth, a twentieth worse.
constexpr int64_t kTailMinBytes = (int64_t)3 << 28;
constexpr int64_t kTileBytes = (int64_t)128 << 10;
constexpr size_t kTailSpillSlack = 16;   // spill bytes a thread of the tail kernel may add
// A tile is a run of rounds (a block's loads in flight at once); with rounds
// under 32 KiB (256-thread blocks: fp32 max at 256 x 2, int32 sum at 256 x 4)
// a tile's rounds cost more than the balance saves (174 / 167 us against
// 153 / 158 us without), so such shapes keep the grid-stride kernel.
constexpr int64_t kTailMinRound = (int64_t)32 << 10;

static void tail_split(int64_t nafter_head, int64_t ve, const pr_config& c, int grid, int gmax, int slots,
                       int loads, int64_t* stat, int64_t* tile_vec) {
    *stat = 0;
    *tile_vec = 0;
    const int64_t nvec = nafter_head / ve;
    if (nvec * c.vec_bytes < kTailMinBytes) return;
    const int64_t step = (int64_t)c.unroll * grid * c.block;
    const int64_t tv = kTileBytes / c.vec_bytes;
    const int64_t tail = nvec / 10;
    // the kernel's tile: whole rounds of block x `loads` vectors, as many as
    // fit in tv (at least one).  Keep the tile count within the gmax slots
    // and within the blocks' shared partial slots (`slots` a block: every
    // claimed tile is then reduced, since a block stops claiming only with
    // its slots full)
    const int64_t round_vec = (int64_t)c.block * loads;
    const int64_t tile = tv > round_vec ? tv / round_vec * round_vec : round_vec;
    const int64_t max_tiles = gmax < (int64_t)grid * slots ? gmax : (int64_t)grid * slots;
    int64_t s = (nvec - tail) / step * step;
    while (s < nvec && (nvec - s + tile - 1) / tile > max_tiles) s += step;
    if (s <= 0 || s >= nvec) return;
    *stat = s;
    *tile_vec = tv;
}

// Persistent grid: SMs x blocks-per-SM (clamped to what is resident at once).
static pr_status persistent_grid(const KernelEntry* e, const pr_config& c, int sms, int gmax, int* grid) {
    int occ = 0;
    pr_status s = occupancy(e->fn, c.block, &occ);
    if (s != PR_OK) return s;
    if (occ < 1) return fail(PR_ERR_UNSUPPORTED, "kernel cannot run with %d threads per block", c.block);
    const int bps = c.blocks_per_sm < occ ? c.blocks_per_sm : occ;
    int g = sms * bps;
    *grid = g < gmax ? g : gmax;
    return PR_OK;
}

// ------------------------------------------------------------------------
// Internal launches with an explicit configuration
// ------------------------------------------------------------------------

// The launch a plain reduction makes: kernel (grid-stride or claimed tail),
// shape and arguments.
struct ReducePlan {
    const KernelEntry* run = nullptr;
    pr_config c{};
    int grid = 0;
    ReduceArgs a{};
};

// Inputs of at most kOneBlockBytes run as one block of (up to) 1024 threads
// with two 32-byte vectors a thread: one step covers them, and a single block
// finishes without the ticket (measured on GB300, fp32 sum from a CUDA graph:
// 1024 elements 2.5 -> 1.6 us a call, 8192 elements 2.9 -> 2.0 us).
constexpr int64_t kOneBlockBytes = (int64_t)64 << 10;

static pr_status plan_reduce(const void* x, int64_t n, int dtype, int op, int prec, bool out_f64, void* out,
                             void* part_out, cudaStream_t st, const pr_config& cfg_in, int aux, int64_t* argidx,
                             ReducePlan* pl) {
    const pr_config cfg = n * elem_size(dtype) <= kOneBlockBytes ? pr_config{1024, 1, 2, 32} : cfg_in;
    const KernelEntry* e = reg_find(KernelKey{K_REDUCE, (uint8_t)dtype, (uint8_t)op, (uint8_t)prec, (uint8_t)aux,
                                              (uint8_t)cfg.unroll, (uint8_t)cfg.vec_bytes});
    if (!e) return fail(PR_ERR_UNSUPPORTED, "no reduce kernel for dtype %d op %d precision %d", dtype, op, prec);
    const pr_config c = fit_block(e, cfg);
    DevInfo di;
    pr_status s = device_info(&di, nullptr);
    if (s != PR_OK) return s;
    Workspace ws;
    s = get_ws(st, &ws);
    if (s != PR_OK) return s;
    int grid = 0;
    s = persistent_grid(e, c, di.sms, ws.gmax, &grid);
    if (s != PR_OK) return s;
    const int es = elem_size(dtype);
    const int64_t ve = c.vec_bytes / es;
    const int64_t per_block = (int64_t)c.block * ve * c.unroll;
    const int64_t need = (n + per_block - 1) / per_block;
    if (need < grid) grid = need < 1 ? 1 : (int)need;
    if (n * es <= kOneBlockBytes) grid = 1;   // (a kernel built for fewer threads loops twice)
    const uintptr_t addr = reinterpret_cast<uintptr_t>(x);
    int64_t head = (int64_t)(((uintptr_t)c.vec_bytes - addr % (uintptr_t)c.vec_bytes) % (uintptr_t)c.vec_bytes) / es;
    if (head > n) head = n;
    ReduceArgs a{x, n, head, out, part_out, out_f64 ? 1 : 0, ws, argidx};
    // large inputs: the claimed-tail variant, where it keeps the same
    // resident blocks and spills at most a few words more than the
    // grid-stride kernel (its tile loads take registers)
    const KernelEntry* run = e;
    if ((n - head) * es >= kTailMinBytes) {
        const KernelEntry* et = reg_find(KernelKey{K_REDUCE_TAIL, (uint8_t)dtype, (uint8_t)op, (uint8_t)prec,
                                                   (uint8_t)aux, (uint8_t)c.unroll, (uint8_t)c.vec_bytes});
        int occ_s = 0, occ_t = 0;
        if (et) {
            s = occupancy(e->fn, c.block, &occ_s);
            if (s == PR_OK) s = occupancy(et->fn, c.block, &occ_t);
            if (s != PR_OK) return s;
        }
        const int want = c.blocks_per_sm < occ_s ? c.blocks_per_sm : occ_s;
        if (et && occ_t >= want && local_bytes(et->fn) <= local_bytes(e->fn) + kTailSpillSlack &&
            (int64_t)c.block * et->tile_loads * c.vec_bytes >= kTailMinRound) {
            tail_split(n - head, ve, c, grid, ws.gmax, et->tile_slots, et->tile_loads, &a.stat, &a.tile_vec);
            if (a.tile_vec > 0) run = et;
        }
    }
    pl->run = run;
    pl->c = c;
    pl->grid = grid;
    pl->a = a;
    return PR_OK;
}

static pr_status run_reduce(const void* x, int64_t n, int dtype, int op, int prec, bool out_f64, void* out,
                            void* part_out, cudaStream_t st, const pr_config& cfg, int aux = AUX_NONE,
                            int64_t* argidx = nullptr) {
    ReducePlan pl;
    pr_status s = plan_reduce(x, n, dtype, op, prec, out_f64, out, part_out, st, cfg, aux, argidx, &pl);
    if (s != PR_OK) return s;
    PR_INJECT_LAUNCH();
    cudaError_t err = reinterpret_cast<ReduceLaunch>(pl.run->launch)(pl.a, pl.grid, pl.c.block, st);
    if (err != cudaSuccess) return fail(PR_ERR_CUDA, "reduce launch: %s", cudaGetErrorString(err));
    return PR_OK;
}

// Segmented work split, measured on GB300: every chunk switch or segment
// boundary costs a block a combine (~3 us with its loads drained), so with few
// segments per block one static chunk per block is fastest (64 rows of 2^20:
// 49 us vs 58 us with 4 chunks), while many uneven segments want a few chunks
// claimed dynamically (4096 log-uniform segments: 220 us with one static chunk
// per block, 201-204 us with 8 dynamic chunks per block, 196-198 us with 2).
static void seg_split(int64_t nseg, int grid, int gmax, int* chunks_per_block, int* dynamic) {
    if (nseg > 2 * (int64_t)grid) {
        int c = 2;
        while (c > 1 && (int64_t)c * grid > gmax) c >>= 1;
        *chunks_per_block = c;
        *dynamic = 1;
    } else {
        *chunks_per_block = 1;
        *dynamic = 0;
    }
}

static pr_status run_segmented(const void* x, const int64_t* off, int64_t cols, int64_t nseg, int dtype, int op,
                               int prec, int aux, void* out, int64_t* argidx, pr_prod_aux* paux, cudaStream_t st,
                               const pr_config& c) {
    const KernelEntry* e = reg_find(KernelKey{K_SEGMENTED, (uint8_t)dtype, (uint8_t)op, (uint8_t)prec, (uint8_t)aux,
                                              (uint8_t)c.unroll, (uint8_t)c.vec_bytes});
    if (!e) return fail(PR_ERR_UNSUPPORTED, "no segmented kernel for dtype %d op %d precision %d aux %d", dtype, op,
                        prec, aux);
    DevInfo di;
    pr_status s = device_info(&di, nullptr);
    if (s != PR_OK) return s;
    Workspace ws;
    s = get_ws(st, &ws);
    if (s != PR_OK) return s;
    int grid = 0;
    s = persistent_grid(e, c, di.sms, ws.gmax, &grid);
    if (s != PR_OK) return s;
    const int es = elem_size(dtype);
    const int64_t shift = (int64_t)(reinterpret_cast<uintptr_t>(x) % (uintptr_t)c.vec_bytes) / es;
    int cpb = 1, dyn = 0;
    seg_split(nseg, grid, ws.gmax, &cpb, &dyn);
    SegArgs a{x, off, cols, nseg, shift, out, argidx, paux, 0, cpb, dyn, ws};
    PR_INJECT_LAUNCH();
    cudaError_t err = reinterpret_cast<SegLaunch>(e->launch)(a, grid, c.block, st);
    if (err != cudaSuccess) return fail(PR_ERR_CUDA, "segmented launch: %s", cudaGetErrorString(err));
    return PR_OK;
}

// Row kernel for equal rows; PR_ERR_UNSUPPORTED (nothing enqueued, no message
// kept) when the shape or alignment needs the general segmented kernel.
static pr_status run_rows(const void* x, int64_t rows, int64_t cols, int dtype, int op, int prec, int aux, void* out,
                          int64_t* argidx, pr_prod_aux* paux, cudaStream_t st, const pr_config& cfg) {
    const int es = elem_size(dtype);
    const int64_t ve = cfg.vec_bytes / es;
    if (rows < 1 || cols < 1 || cols % ve != 0 || reinterpret_cast<uintptr_t>(x) % (uintptr_t)cfg.vec_bytes != 0)
        return PR_ERR_UNSUPPORTED;
    const KernelEntry* e = reg_find(KernelKey{K_ROWS, (uint8_t)dtype, (uint8_t)op, (uint8_t)prec, (uint8_t)aux,
                                              (uint8_t)cfg.unroll, (uint8_t)cfg.vec_bytes});
    if (!e) return PR_ERR_UNSUPPORTED;
    const pr_config c = fit_block(e, cfg);
    DevInfo di;
    pr_status s = device_info(&di, nullptr);
    if (s != PR_OK) return s;
    Workspace ws;
    s = get_ws(st, &ws);
    if (s != PR_OK) return s;
    int grid = 0;
    s = persistent_grid(e, c, di.sms, ws.gmax, &grid);
    if (s != PR_OK) return s;
    const int64_t tile = (int64_t)c.block * c.unroll;
    const int64_t ntile = (rows * (cols / ve) + tile - 1) / tile;
    if (ntile < grid) grid = (int)ntile;
    RowArgs a{x, rows, cols, out, argidx, paux, 0, ws};
    PR_INJECT_LAUNCH();
    cudaError_t err = reinterpret_cast<RowLaunch>(e->launch)(a, grid, c.block, st);
    if (err != cudaSuccess) return fail(PR_ERR_CUDA, "row launch: %s", cudaGetErrorString(err));
    return PR_OK;
}

constexpr int kBwdWaves = 8;  // backward grid = resident blocks x this (capped at the chunk count)

static pr_status run_backward(int op, int dtype, const void* x, int64_t rows, int64_t cols, const void* g,
                              const int64_t* argidx, const pr_prod_aux* aux, void* gi, cudaStream_t st,
                              const pr_config& c) {
    const KernelEntry* e = reg_find(KernelKey{K_BACKWARD, (uint8_t)dtype, 0, 0, 0, (uint8_t)c.unroll,
                                              (uint8_t)c.vec_bytes});
    if (!e) return fail(PR_ERR_UNSUPPORTED, "no backward kernel for dtype %d", dtype);
    DevInfo di;
    pr_status s = device_info(&di, nullptr);
    if (s != PR_OK) return s;
    int grid = 0;
    s = persistent_grid(e, c, di.sms, 1 << 30, &grid);
    if (s != PR_OK) return s;
    // Writes balance best with the grid oversubscribed (measured on GB300,
    // 64 x 2^20 fp32: 44.5 us resident-only, 40.9 us at three or more waves).
    grid *= kBwdWaves;
    const int es = elem_size(dtype);
    const int64_t ve = c.vec_bytes / es;
    const int64_t cv = (int64_t)c.block * c.unroll;
    const int64_t nvec_max = cols / ve + 1;
    const int64_t chunks = (nvec_max + cv - 1) / cv;
    const int64_t tiles = rows * chunks;
    if (tiles < grid) grid = (int)tiles;
    const int64_t shift = (int64_t)(reinterpret_cast<uintptr_t>(gi) % (uintptr_t)c.vec_bytes) / es;
    BwdArgs a{x, g, argidx, aux, gi, rows, cols, shift, chunks, op};
    PR_INJECT_LAUNCH();
    cudaError_t err = reinterpret_cast<BwdLaunch>(e->launch)(a, grid, c.block, st);
    if (err != cudaSuccess) return fail(PR_ERR_CUDA, "backward launch: %s", cudaGetErrorString(err));
    return PR_OK;
}

// Axis partials for (device, stream): at least `bytes`, grown outside graph
// capture (the first call with a shape needing more must not be captured).
static pr_status axis_scratch(cudaStream_t st, size_t bytes, char** out) {
    Workspace ws;
    pr_status s = get_ws(st, &ws);
    if (s != PR_OK) return s;
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    WsRec& w = g_ws[std::make_pair(dev, st)];
    if (w.axis_bytes < bytes) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        PR_CUDA(cudaStreamIsCapturing(st, &cap));
        if (cap != cudaStreamCaptureStatusNone)
            return fail(PR_ERR_INVALID, "axis partials need %zu bytes: run this shape once before graph capture", bytes);
        PR_CUDA(cudaStreamSynchronize(st));
        if (w.axis) cudaFree(w.axis);
        w.axis = nullptr;
        w.axis_bytes = 0;
        size_t grow = bytes < ((size_t)1 << 20) ? ((size_t)1 << 20) : bytes;
        PR_INJECT_ALLOC();
        if (cudaMalloc(&w.axis, grow) != cudaSuccess) {
            cudaGetLastError();
            return fail(PR_ERR_NOMEM, "axis partials: allocation of %zu bytes failed", grow);
        }
        w.axis_bytes = grow;
    }
    *out = static_cast<char*>(w.axis);
    return PR_OK;
}

// Reduction of the middle axis of [outer, n, inner] (inner > 1, outer > 0).
// The launch: warps per (slab, column group) times row splits, enough warps
// for about two waves of the resident ones; splits > 1 add a finishing pass.
static pr_status run_axis(const void* x, int64_t outer, int64_t n, int64_t inner, int dtype, int op, int prec,
                          int aux, void* out, int64_t* argidx, pr_prod_aux* paux, cudaStream_t st,
                          const pr_config& cfg) {
    const int es = elem_size(dtype);
    DevInfo di;
    pr_status s = device_info(&di, nullptr);
    if (s != PR_OK) return s;
    AxisArgs a{x, outer, n, inner, 0, 1, 0, 1, 0, out, argidx, paux, 0, nullptr};
    if (n == 0) {
        const KernelEntry* e = reg_find(KernelKey{K_AXIS_EMPTY, (uint8_t)dtype, (uint8_t)op, (uint8_t)prec,
                                                  (uint8_t)aux, 0, 0});
        if (!e) return fail(PR_ERR_UNSUPPORTED, "no axis kernel for dtype %d op %d precision %d", dtype, op, prec);
        const int64_t nout = outer * inner;
        int grid = (int)((nout + 255) / 256 < 4096 ? (nout + 255) / 256 : 4096);
        PR_INJECT_LAUNCH();
        cudaError_t err = reinterpret_cast<AxisLaunch>(e->launch)(a, grid, 256, st);
        if (err != cudaSuccess) return fail(PR_ERR_CUDA, "axis launch: %s", cudaGetErrorString(err));
        return PR_OK;
    }
    // vector columns when a row is a whole number of aligned vectors, else one element per lane
    int vb = cfg.vec_bytes;
    if (inner % (vb / es) != 0 || reinterpret_cast<uintptr_t>(x) % (uintptr_t)vb != 0) vb = 0;
    const KernelEntry* e = reg_find(KernelKey{K_AXIS, (uint8_t)dtype, (uint8_t)op, (uint8_t)prec, (uint8_t)aux,
                                              (uint8_t)cfg.unroll, (uint8_t)vb});
    if (!e) return fail(PR_ERR_UNSUPPORTED, "no axis kernel for dtype %d op %d precision %d", dtype, op, prec);
    const pr_config c = fit_block(e, cfg);
    int occ = 0;
    s = occupancy(e->fn, c.block, &occ);
    if (s != PR_OK) return s;
    if (occ < 1) return fail(PR_ERR_UNSUPPORTED, "axis kernel cannot run with %d threads per block", c.block);
    const int bps = c.blocks_per_sm < occ ? c.blocks_per_sm : occ;
    const int ve = vb ? vb / es : 1;
    a.qv = inner / ve;
    int bx = 1;
    while (bx < 32 && bx < a.qv) bx <<= 1;
    a.bx = bx;
    a.groups = (a.qv + bx - 1) / bx;
    const int64_t tiles = outer * a.groups;
    const int64_t want = (int64_t)di.sms * bps * (c.block / 32) * 2;   // two waves of resident warps
    const int64_t ry = 32 / bx;
    int64_t max_split = n / (ry * c.unroll * 4);                        // >= 4 unrolled steps per warp
    if (max_split < 1) max_split = 1;
    if (max_split > 1024) max_split = 1024;
    int64_t splits = (want + tiles - 1) / tiles;
    if (splits > max_split) splits = max_split;
    if (splits < 1) splits = 1;
    // a split holds fewer than 2^31 rows (the float arg-extremum keeps its
    // row as a 32-bit offset within the split)
    const int64_t kMaxSplitRows = (int64_t)1 << 30;
    if ((n + splits - 1) / splits > kMaxSplitRows) splits = (n + kMaxSplitRows - 1) / kMaxSplitRows;
    a.rows_per_split = (n + splits - 1) / splits;
    a.splits = (n + a.rows_per_split - 1) / a.rows_per_split;
    if (a.splits > 1) {
        char* sc = nullptr;
        s = axis_scratch(st, (size_t)(outer * inner) * (size_t)a.splits * (size_t)e->part_bytes, &sc);
        if (s != PR_OK) return s;
        a.scratch = sc;
    }
    const int64_t warps = tiles * a.splits;
    const int wpb = c.block / 32;
    const int64_t grid = (warps + wpb - 1) / wpb;
    if (grid > 0x7fffffff) return fail(PR_ERR_INVALID, "axis reduction too large for one launch");
    PR_INJECT_LAUNCH();
    cudaError_t err = reinterpret_cast<AxisLaunch>(e->launch)(a, (int)grid, c.block, st);
    if (err != cudaSuccess) return fail(PR_ERR_CUDA, "axis launch: %s", cudaGetErrorString(err));
    if (a.splits > 1) {
        const KernelEntry* f = reg_find(KernelKey{K_AXIS_FINISH, (uint8_t)dtype, (uint8_t)op, (uint8_t)prec,
                                                  (uint8_t)aux, 0, 0});
        if (!f) return fail(PR_ERR_UNSUPPORTED, "no axis finishing kernel");
        const int64_t per_out = a.splits <= kAxisThreadFinish ? 1 : 32;   // threads per output
        const int64_t fgrid = (outer * inner * per_out + 255) / 256;
        if (fgrid > 0x7fffffff) return fail(PR_ERR_INVALID, "axis reduction too large for one launch");
        PR_INJECT_LAUNCH();
        err = reinterpret_cast<AxisLaunch>(f->launch)(a, (int)fgrid, 256, st);
        if (err != cudaSuccess) return fail(PR_ERR_CUDA, "axis finish launch: %s", cudaGetErrorString(err));
    }
    return PR_OK;
}

// Scan state for (device, stream): `tiles` tile records and three counters
// (next tile, blocks done, epoch).  Grown outside graph capture, zero-filled,
// epoch 1, so that no stale flag can look current.
static pr_status scan_state(cudaStream_t st, int64_t tiles, ScanTile** recs, unsigned** ctr) {
    Workspace ws;
    pr_status s = get_ws(st, &ws);
    if (s != PR_OK) return s;
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    WsRec& w = g_ws[std::make_pair(dev, st)];
    if ((int64_t)w.scan_tiles < tiles) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        PR_CUDA(cudaStreamIsCapturing(st, &cap));
        if (cap != cudaStreamCaptureStatusNone)
            return fail(PR_ERR_INVALID, "scan state for %lld tiles: run this size once before graph capture",
                        (long long)tiles);
        PR_CUDA(cudaStreamSynchronize(st));
        if (w.scan) cudaFree(w.scan);
        w.scan = nullptr;
        w.scan_tiles = 0;
        const int64_t grow = tiles < 4096 ? 4096 : tiles;
        const size_t bytes = (size_t)grow * sizeof(ScanTile) + 64;
        PR_INJECT_ALLOC();
        if (cudaMalloc(&w.scan, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(PR_ERR_NOMEM, "scan state: allocation of %zu bytes failed", bytes);
        }
        PR_CUDA(cudaMemset(w.scan, 0, bytes));
        const unsigned one = 1u;
        PR_CUDA(cudaMemcpy(static_cast<char*>(w.scan) + (size_t)grow * sizeof(ScanTile) + 8, &one, 4,
                           cudaMemcpyHostToDevice));
        w.scan_tiles = (size_t)grow;
    }
    *recs = static_cast<ScanTile*>(w.scan);
    *ctr = reinterpret_cast<unsigned*>(static_cast<char*>(w.scan) + w.scan_tiles * sizeof(ScanTile));
    return PR_OK;
}

// Line-search state for (device, stream): the LsState, gmax x kLsMaxPts
// evaluation partials and one ticket, made zero-filled on first use (outside
// graph capture).
static pr_status search_state(cudaStream_t st, LsState** state, double** partials, unsigned** ticket) {
    Workspace ws;
    pr_status s = get_ws(st, &ws);
    if (s != PR_OK) return s;
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    WsRec& w = g_ws[std::make_pair(dev, st)];
    const size_t head = (sizeof(LsState) + 255) / 256 * 256;
    const size_t parts = (size_t)ws.gmax * kLsMaxPts * sizeof(double);
    if (!w.search) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        PR_CUDA(cudaStreamIsCapturing(st, &cap));
        if (cap != cudaStreamCaptureStatusNone)
            return fail(PR_ERR_INVALID, "line-search state: run a search on this stream once before graph capture");
        PR_CUDA(cudaStreamSynchronize(st));
        const size_t bytes = head + parts + 256;
        PR_INJECT_ALLOC();
        if (cudaMalloc(&w.search, bytes) != cudaSuccess) {
            cudaGetLastError();
            w.search = nullptr;
            return fail(PR_ERR_NOMEM, "line-search state: allocation of %zu bytes failed", bytes);
        }
        PR_CUDA(cudaMemset(w.search, 0, bytes));
    }
    char* b = static_cast<char*>(w.search);
    *state = reinterpret_cast<LsState*>(b);
    *partials = reinterpret_cast<double*>(b + head);
    *ticket = reinterpret_cast<unsigned*>(b + head + parts);
    return PR_OK;
}

static pr_status run_axis_backward(int op, int dtype, const void* x, int64_t outer, int64_t n, int64_t inner,
                                   const void* g, const int64_t* argidx, const pr_prod_aux* aux, void* gi,
                                   cudaStream_t st) {
    DevInfo di;
    pr_status s = device_info(&di, nullptr);
    if (s != PR_OK) return s;
    const int es = elem_size(dtype);
    int vb = 32;
    // vectors need grad_in and grad_out aligned to them and whole vectors per row
    auto fits = [&](int w) {
        return inner % (w / es) == 0 && reinterpret_cast<uintptr_t>(gi) % (uintptr_t)w == 0 &&
               reinterpret_cast<uintptr_t>(g) % (uintptr_t)w == 0;
    };
    if (!fits(vb)) vb = 16;
    if (!fits(vb)) vb = 0;
    const int opk = op == PR_SUM ? 0 : (op == PR_PROD ? 2 : 1);
    const KernelEntry* e = reg_find(KernelKey{K_AXIS_BACKWARD, (uint8_t)dtype, (uint8_t)opk, 0, 0, 0, (uint8_t)vb});
    if (!e) return fail(PR_ERR_UNSUPPORTED, "no axis backward kernel for dtype %d", dtype);
    const int ve = vb ? vb / es : 1;
    AxisBwdArgs a{x, g, argidx, aux, gi, outer, n, inner, inner / ve, op};
    const int64_t total = outer * n * a.qv;
    int64_t grid = (total + 255) / 256;
    const int64_t cap = (int64_t)di.sms * 64;
    if (grid > cap) grid = cap;
    PR_INJECT_LAUNCH();
    cudaError_t err = reinterpret_cast<AxisBwdLaunch>(e->launch)(a, (int)grid, 256, st);
    if (err != cudaSuccess) return fail(PR_ERR_CUDA, "axis backward launch: %s", cudaGetErrorString(err));
    return PR_OK;
}

// ------------------------------------------------------------------------
// Validation shared by the entry points
// ------------------------------------------------------------------------

static pr_status check_common(int dtype, int op, int prec) {
    if (!valid_dtype(dtype)) return fail(PR_ERR_INVALID, "unknown dtype %d", dtype);
    if (!valid_op(op)) return fail(PR_ERR_INVALID, "unknown op %d", op);
    if (prec < PR_PREC_PLAIN || prec > PR_PREC_FP64_COMBINE) return fail(PR_ERR_INVALID, "unknown precision %d", prec);
    if (is_float(dtype) && op >= PR_AND)
        return fail(PR_ERR_UNSUPPORTED, "bitwise combiner %d is not defined on floating-point dtype %d", op, dtype);
    if (prec != PR_PREC_PLAIN && !(op == PR_SUM && is_float(dtype) && dtype != PR_F64))
        return fail(PR_ERR_UNSUPPORTED, "precision modes apply to fp32/fp16/bf16 SUM only");
    return PR_OK;
}

static pr_status check_aligned(const void* p, int dtype, const char* what) {
    if (p && reinterpret_cast<uintptr_t>(p) % (uintptr_t)elem_size(dtype))
        return fail(PR_ERR_INVALID, "%s is not aligned to its element size", what);
    return PR_OK;
}

}  // namespace pr

using namespace pr;

// ------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------

extern "C" {

pr_dtype pr_out_dtype(pr_dtype dtype, pr_op op) {
    if (dtype == PR_F16 || dtype == PR_BF16) return (op == PR_MAX || op == PR_MIN) ? dtype : PR_F32;
    if (dtype == PR_I32 && op == PR_SUM) return PR_I64;
    return dtype;
}

const char* pr_status_string(pr_status s) {
    switch (s) {
    case PR_OK: return "PR_OK";
    case PR_ERR_INVALID: return "PR_ERR_INVALID";
    case PR_ERR_UNSUPPORTED: return "PR_ERR_UNSUPPORTED";
    case PR_ERR_CUDA: return "PR_ERR_CUDA";
    case PR_ERR_TIMEOUT: return "PR_ERR_TIMEOUT";
    case PR_ERR_NOMEM: return "PR_ERR_NOMEM";
    default: return "PR_ERR_UNKNOWN";
    }
}

const char* pr_last_error_message(void) { return g_msg.c_str(); }

const char* pr_version(void) { return "pr 0.1 (sm_103a)"; }

pr_status pr_reduce_ex(const void* x, int64_t n, pr_dtype dtype, pr_op op, pr_precision precision,
                       pr_dtype out_dtype, void* out, pr_stream_t stream) {
    g_msg.clear();
    pr_status s = check_common(dtype, op, precision);
    if (s != PR_OK) return s;
    if (n < 0) return fail(PR_ERR_INVALID, "n must be >= 0 (got %lld)", (long long)n);
    if (!x && n > 0) return fail(PR_ERR_INVALID, "x is NULL");
    if (!out) return fail(PR_ERR_INVALID, "out is NULL");
    if ((s = check_aligned(x, dtype, "x")) != PR_OK) return s;
    const pr_dtype def = pr_out_dtype(dtype, op);
    const bool f64 = out_dtype != def;
    if (f64 && !(out_dtype == PR_F64 && precision != PR_PREC_PLAIN))
        return fail(PR_ERR_UNSUPPORTED, "out_dtype %d not available for dtype %d op %d", out_dtype, dtype, op);
    ensure_registered();
    const pr_config c = lookup_cfg(PR_KIND_REDUCE, dtype, op, precision, n);
    return run_reduce(x, n, dtype, op, precision, f64, out, nullptr, (cudaStream_t)stream, c);
}

pr_status pr_reduce_arg(const void* x, int64_t n, pr_dtype dtype, pr_op op, void* out, int64_t* idx,
                        pr_stream_t stream) {
    g_msg.clear();
    pr_status s = check_common(dtype, op, PR_PREC_PLAIN);
    if (s != PR_OK) return s;
    if (op != PR_MAX && op != PR_MIN) return fail(PR_ERR_UNSUPPORTED, "arg-extremum needs MAX or MIN");
    if (n < 0) return fail(PR_ERR_INVALID, "n must be >= 0 (got %lld)", (long long)n);
    if (!x && n > 0) return fail(PR_ERR_INVALID, "x is NULL");
    if (!out || !idx) return fail(PR_ERR_INVALID, "out / idx is NULL");
    if ((s = check_aligned(x, dtype, "x")) != PR_OK) return s;
    ensure_registered();
    // The (key, index) accumulator wants more resident threads than plain
    // max/min, whose tuned shapes it would otherwise share: use the default.
    const pr_config c = default_cfg(PR_KIND_REDUCE, dtype, op, PR_PREC_PLAIN);
    return run_reduce(x, n, dtype, op, PR_PREC_PLAIN, false, out, nullptr, (cudaStream_t)stream, c, AUX_ARG, idx);
}

pr_status pr_reduce(const void* x, int64_t n, pr_dtype dtype, pr_op op, void* out, pr_stream_t stream) {
    if (!valid_dtype(dtype) || !valid_op(op)) {
        g_msg.clear();
        return check_common(dtype, op, PR_PREC_PLAIN);
    }
    return pr_reduce_ex(x, n, dtype, op, PR_PREC_PLAIN, pr_out_dtype(dtype, op), out, stream);
}

static pr_status segmented_common(const void* x, const int64_t* offsets, int64_t cols, int64_t nseg, pr_dtype dtype,
                                  pr_op op, pr_precision precision, void* out, int64_t* argidx, pr_prod_aux* aux,
                                  pr_stream_t stream) {
    pr_status s = check_common(dtype, op, precision);
    if (s != PR_OK) return s;
    if (nseg < 0) return fail(PR_ERR_INVALID, "number of segments must be >= 0");
    if (nseg == 0) return PR_OK;
    if (!out) return fail(PR_ERR_INVALID, "out is NULL");
    if (argidx && op != PR_MAX && op != PR_MIN) return fail(PR_ERR_UNSUPPORTED, "argidx needs MAX or MIN");
    if (aux && !(op == PR_PROD && (dtype == PR_F32 || dtype == PR_F64)))
        return fail(PR_ERR_UNSUPPORTED, "product aux needs PROD on F32 or F64");
    if ((s = check_aligned(x, dtype, "x")) != PR_OK) return s;
    const int auxk = argidx ? AUX_ARG : (aux ? AUX_PROD : AUX_NONE);
    ensure_registered();
    const pr_config c = lookup_cfg(PR_KIND_SEGMENTED, dtype, op, precision, nseg);
    return run_segmented(x, offsets, cols, nseg, dtype, op, precision, auxk, out, argidx, aux, (cudaStream_t)stream, c);
}

pr_status pr_segmented_reduce_aux(const void* x, const int64_t* offsets, int64_t nseg, pr_dtype dtype, pr_op op,
                                  pr_precision precision, void* out, int64_t* argidx, pr_prod_aux* aux,
                                  pr_stream_t stream) {
    g_msg.clear();
    if (nseg > 0 && !offsets) return fail(PR_ERR_INVALID, "offsets is NULL");
    if (nseg > 0 && !x) return fail(PR_ERR_INVALID, "x is NULL");
    return segmented_common(x, offsets, 0, nseg, dtype, op, precision, out, argidx, aux, stream);
}

pr_status pr_segmented_reduce(const void* x, const int64_t* offsets, int64_t nseg, pr_dtype dtype, pr_op op,
                              void* out, pr_stream_t stream) {
    return pr_segmented_reduce_aux(x, offsets, nseg, dtype, op, PR_PREC_PLAIN, out, nullptr, nullptr, stream);
}

pr_status pr_reduce_rows(const void* x, int64_t rows, int64_t cols, pr_dtype dtype, pr_op op, pr_precision precision,
                         void* out, int64_t* argidx, pr_prod_aux* aux, pr_stream_t stream) {
    g_msg.clear();
    if (rows < 0 || cols < 0) return fail(PR_ERR_INVALID, "rows and cols must be >= 0");
    if (cols > 0 && rows > ((int64_t)1 << 62) / cols) return fail(PR_ERR_INVALID, "rows*cols overflows");
    if (rows > 0 && cols > 0 && !x) return fail(PR_ERR_INVALID, "x is NULL");
    // Rows whose length is a whole number of vectors, on an aligned x, take
    // the row kernel; anything else the general segmented kernel.
    if (rows > 0 && cols > 0 && out && check_common(dtype, op, precision) == PR_OK &&
        !(argidx && op != PR_MAX && op != PR_MIN) && !(aux && !(op == PR_PROD && (dtype == PR_F32 || dtype == PR_F64)))) {
        ensure_registered();
        const int auxk = argidx ? AUX_ARG : (aux ? AUX_PROD : AUX_NONE);
        const pr_config c = lookup_cfg(PR_KIND_ROWS, dtype, op, precision, rows * cols);
        const pr_status s = run_rows(x, rows, cols, dtype, op, precision, auxk, out, argidx, aux, (cudaStream_t)stream, c);
        if (s != PR_ERR_UNSUPPORTED) return s;
        g_msg.clear();
    }
    return segmented_common(x, nullptr, cols, rows, dtype, op, precision, out, argidx, aux, stream);
}

pr_status pr_reduce_backward(pr_op op, pr_dtype dtype, const void* x, int64_t rows, int64_t cols,
                             const void* grad_out, const int64_t* argidx, const pr_prod_aux* aux, void* grad_in,
                             pr_stream_t stream) {
    g_msg.clear();
    if (dtype != PR_F32 && dtype != PR_F64) return fail(PR_ERR_UNSUPPORTED, "backward supports F32 and F64");
    if (op != PR_SUM && op != PR_MAX && op != PR_MIN && op != PR_PROD)
        return fail(PR_ERR_UNSUPPORTED, "backward supports SUM, MAX, MIN and PROD");
    if (rows < 0 || cols < 0) return fail(PR_ERR_INVALID, "rows and cols must be >= 0");
    if (cols > 0 && rows > ((int64_t)1 << 62) / cols) return fail(PR_ERR_INVALID, "rows*cols overflows");
    if (rows == 0 || cols == 0) return PR_OK;
    if (!grad_out || !grad_in) return fail(PR_ERR_INVALID, "grad_out / grad_in is NULL");
    if ((op == PR_MAX || op == PR_MIN) && !argidx) return fail(PR_ERR_INVALID, "MAX/MIN backward needs argidx");
    if (op == PR_PROD && (!aux || !x)) return fail(PR_ERR_INVALID, "PROD backward needs x and aux");
    pr_status s;
    if ((s = check_aligned(grad_in, dtype, "grad_in")) != PR_OK) return s;
    if ((s = check_aligned(grad_out, dtype, "grad_out")) != PR_OK) return s;
    if ((s = check_aligned(x, dtype, "x")) != PR_OK) return s;
    ensure_registered();
    const pr_config c = lookup_cfg(PR_KIND_BACKWARD, dtype, op, 0, rows * cols);
    return run_backward(op, dtype, x, rows, cols, grad_out, argidx, aux, grad_in, (cudaStream_t)stream, c);
}

pr_status pr_reduce_axis(const void* x, int64_t outer, int64_t n, int64_t inner, pr_dtype dtype, pr_op op,
                         pr_precision precision, void* out, int64_t* argidx, pr_prod_aux* aux, pr_stream_t stream) {
    g_msg.clear();
    if (outer < 0 || n < 0 || inner < 0) return fail(PR_ERR_INVALID, "outer, n and inner must be >= 0");
    const int64_t lim = (int64_t)1 << 62;
    if ((outer > 0 && inner > 0 && (outer > lim / inner || (n > 0 && outer * inner > lim / n))))
        return fail(PR_ERR_INVALID, "outer*n*inner overflows");
    pr_status s = check_common(dtype, op, precision);
    if (s != PR_OK) return s;
    if (argidx && op != PR_MAX && op != PR_MIN) return fail(PR_ERR_UNSUPPORTED, "argidx needs MAX or MIN");
    if (aux && !(op == PR_PROD && (dtype == PR_F32 || dtype == PR_F64)))
        return fail(PR_ERR_UNSUPPORTED, "product aux needs PROD on F32 or F64");
    if (outer == 0 || inner == 0) return PR_OK;
    if (!out) return fail(PR_ERR_INVALID, "out is NULL");
    if (n > 0 && !x) return fail(PR_ERR_INVALID, "x is NULL");
    if ((s = check_aligned(x, dtype, "x")) != PR_OK) return s;
    if (inner == 1) return pr_reduce_rows(x, outer, n, dtype, op, precision, out, argidx, aux, stream);
    ensure_registered();
    const int auxk = argidx ? AUX_ARG : (aux ? AUX_PROD : AUX_NONE);
    const pr_config c = lookup_cfg(PR_KIND_AXIS, dtype, op, precision, outer * n * inner);
    return run_axis(x, outer, n, inner, dtype, op, precision, auxk, out, argidx, aux, (cudaStream_t)stream, c);
}

pr_status pr_reduce_axis_backward(pr_op op, pr_dtype dtype, const void* x, int64_t outer, int64_t n, int64_t inner,
                                  const void* grad_out, const int64_t* argidx, const pr_prod_aux* aux,
                                  void* grad_in, pr_stream_t stream) {
    g_msg.clear();
    if (dtype != PR_F32 && dtype != PR_F64) return fail(PR_ERR_UNSUPPORTED, "backward supports F32 and F64");
    if (op != PR_SUM && op != PR_MAX && op != PR_MIN && op != PR_PROD)
        return fail(PR_ERR_UNSUPPORTED, "backward supports SUM, MAX, MIN and PROD");
    if (outer < 0 || n < 0 || inner < 0) return fail(PR_ERR_INVALID, "outer, n and inner must be >= 0");
    const int64_t lim = (int64_t)1 << 62;
    if ((outer > 0 && inner > 0 && (outer > lim / inner || (n > 0 && outer * inner > lim / n))))
        return fail(PR_ERR_INVALID, "outer*n*inner overflows");
    if (outer == 0 || n == 0 || inner == 0) return PR_OK;
    if (inner == 1) return pr_reduce_backward(op, dtype, x, outer, n, grad_out, argidx, aux, grad_in, stream);
    if (!grad_out || !grad_in) return fail(PR_ERR_INVALID, "grad_out / grad_in is NULL");
    if ((op == PR_MAX || op == PR_MIN) && !argidx) return fail(PR_ERR_INVALID, "MAX/MIN backward needs argidx");
    if (op == PR_PROD && (!aux || !x)) return fail(PR_ERR_INVALID, "PROD backward needs x and aux");
    pr_status s;
    if ((s = check_aligned(grad_in, dtype, "grad_in")) != PR_OK) return s;
    if ((s = check_aligned(grad_out, dtype, "grad_out")) != PR_OK) return s;
    if ((s = check_aligned(x, dtype, "x")) != PR_OK) return s;
    ensure_registered();
    return run_axis_backward(op, dtype, x, outer, n, inner, grad_out, argidx, aux, grad_in, (cudaStream_t)stream);
}

pr_status pr_scan(const void* x, int64_t n, pr_dtype dtype, pr_op op, int32_t exclusive, void* y,
                  pr_stream_t stream) {
    g_msg.clear();
    if (!valid_dtype(dtype)) return fail(PR_ERR_INVALID, "unknown dtype %d", dtype);
    if (!valid_op(op)) return fail(PR_ERR_INVALID, "unknown op %d", op);
    if (is_float(dtype) && op != PR_MAX && op != PR_MIN)
        return fail(PR_ERR_UNSUPPORTED, "float scans cover MAX and MIN (their results are exact)");
    if (n < 0) return fail(PR_ERR_INVALID, "n must be >= 0");
    if (n == 0) return PR_OK;
    if (!x) return fail(PR_ERR_INVALID, "x is NULL");
    if (!y) return fail(PR_ERR_INVALID, "y is NULL");
    pr_status s;
    if ((s = check_aligned(x, dtype, "x")) != PR_OK) return s;
    if ((s = check_aligned(y, (int)pr_out_dtype(dtype, op), "y")) != PR_OK) return s;
    ensure_registered();
    cudaStream_t st = (cudaStream_t)stream;
    const int es = elem_size(dtype);
    const int64_t tile = kScanTileBytes / es;
    const int64_t tiles = (n + tile - 1) / tile;
    if (tiles > (int64_t)1 << 31) return fail(PR_ERR_INVALID, "scan of %lld elements: too many tiles", (long long)n);
    const bool vec = reinterpret_cast<uintptr_t>(x) % 16 == 0 && reinterpret_cast<uintptr_t>(y) % 16 == 0;
    const KernelEntry* e = reg_find(KernelKey{K_SCAN, (uint8_t)dtype, (uint8_t)op, 0, 0, 0, (uint8_t)(vec ? 1 : 0)});
    if (!e) return fail(PR_ERR_UNSUPPORTED, "no scan kernel for dtype %d op %d", dtype, op);
    DevInfo di;
    if ((s = device_info(&di, nullptr)) != PR_OK) return s;
    Workspace ws;
    if ((s = get_ws(st, &ws)) != PR_OK) return s;
    ScanTile* recs = nullptr;
    unsigned* ctr = nullptr;
    if ((s = scan_state(st, tiles, &recs, &ctr)) != PR_OK) return s;
    int occ = 0;
    const size_t smem = (size_t)kScanStages * kScanTileBytes;
    if ((s = occupancy(e->fn, kScanThreads, &occ, smem)) != PR_OK) return s;
    if (occ < 1) return fail(PR_ERR_UNSUPPORTED, "scan kernel cannot run");
    int64_t grid = (int64_t)di.sms * occ;
    if (grid > tiles) grid = tiles;
    ScanArgs a{x, y, n, tiles, exclusive ? 1 : 0, recs, ctr, ws.err};
    PR_INJECT_LAUNCH();
    cudaError_t err = reinterpret_cast<ScanLaunch>(e->launch)(a, (int)grid, kScanThreads, smem, st);
    if (err != cudaSuccess) return fail(PR_ERR_CUDA, "scan launch: %s", cudaGetErrorString(err));
    return PR_OK;
}

pr_status pr_check_bounded_wait(int32_t polls, pr_stream_t stream) {
    g_msg.clear();
    if (polls < 1) return fail(PR_ERR_INVALID, "polls must be >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    Workspace ws;
    pr_status s = get_ws(st, &ws);
    if (s != PR_OK) return s;
    ScanTile* rec = nullptr;
    PR_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&rec), sizeof(ScanTile), st));
    PR_CUDA(cudaMemsetAsync(rec, 0, sizeof(ScanTile), st));
    cudaError_t err = launch_wait_probe(rec, polls, ws.err, st);
    cudaFreeAsync(rec, st);
    if (err != cudaSuccess) return fail(PR_ERR_CUDA, "wait probe launch: %s", cudaGetErrorString(err));
    return PR_OK;
}

// ------------------------------------------------------------------------
// Line search on the reduction
// ------------------------------------------------------------------------

static pr_status check_links(const float* x, const float* d, const float* t0, const float* cap, int64_t n,
                             float beta, int32_t power) {
    if (n < 0) return fail(PR_ERR_INVALID, "n must be >= 0");
    if (n > 0 && (!x || !d || !t0 || !cap)) return fail(PR_ERR_INVALID, "a link array is NULL");
    const float* arr[4] = {x, d, t0, cap};
    for (const float* p : arr)
        if (reinterpret_cast<uintptr_t>(p) % 4) return fail(PR_ERR_INVALID, "link arrays must be 4-byte aligned");
    if (!(beta >= 0.f) || !std::isfinite(beta)) return fail(PR_ERR_INVALID, "beta must be finite and >= 0");
    if (power < 1 || power > 16) return fail(PR_ERR_INVALID, "power must be in [1, 16]");
    return PR_OK;
}

// One evaluation pass: m points of pts, sums into out (all device memory).
static pr_status run_phi(const float* x, const float* d, const float* t0, const float* cap, int64_t n, float beta,
                         int32_t power, const double* pts, int m, double* out, double* partials, unsigned* ticket,
                         cudaStream_t st, LsState* ls = nullptr, double* result = nullptr) {
    const bool vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(d) |
                       reinterpret_cast<uintptr_t>(t0) | reinterpret_cast<uintptr_t>(cap)) % 16) == 0;
    DevInfo di;
    pr_status s = device_info(&di, nullptr);
    if (s != PR_OK) return s;
    // one grid for every point count (that of the up-to-8-point kernel), so
    // that phi(alpha) has the same bits whatever else a pass evaluates
    int occ = 0;
    if ((s = occupancy(phi_kernel(vec, power, 8), kPhiThreads, &occ)) != PR_OK) return s;
    int occ16 = 0;
    if ((s = occupancy(phi_kernel(vec, power, kLsMaxPts), kPhiThreads, &occ16)) != PR_OK) return s;
    if (occ < 1 || occ16 < 1) return fail(PR_ERR_UNSUPPORTED, "evaluation kernel cannot run");
    Workspace ws;
    if ((s = get_ws(st, &ws)) != PR_OK) return s;
    int64_t grid = (int64_t)di.sms * occ;
    const int64_t need = (n + 4LL * kPhiThreads - 1) / (4LL * kPhiThreads);
    if (grid > need) grid = need > 0 ? need : 1;
    if (grid > ws.gmax) grid = ws.gmax;
    PhiArgs a{x, d, t0, cap, n, beta, power, pts, m, out, partials, ticket, ls, result};
    PR_INJECT_LAUNCH();
    cudaError_t err = launch_phi(a, (int)grid, vec, st);
    if (err != cudaSuccess) return fail(PR_ERR_CUDA, "evaluation launch: %s", cudaGetErrorString(err));
    return PR_OK;
}

pr_status pr_beckmann(const float* x, const float* d, const float* t0, const float* cap, int64_t n, float beta,
                      int32_t power, const double* alphas, int32_t m, double* out, pr_stream_t stream) {
    g_msg.clear();
    pr_status s = check_links(x, d, t0, cap, n, beta, power);
    if (s != PR_OK) return s;
    if (m < 1 || m > kLsMaxPts) return fail(PR_ERR_INVALID, "m must be in [1, %d]", kLsMaxPts);
    if (!alphas || !out) return fail(PR_ERR_INVALID, "alphas / out is NULL");
    if (reinterpret_cast<uintptr_t>(alphas) % 8 || reinterpret_cast<uintptr_t>(out) % 8)
        return fail(PR_ERR_INVALID, "alphas / out must be 8-byte aligned");
    ensure_registered();
    cudaStream_t st = (cudaStream_t)stream;
    LsState* ls = nullptr;
    double* parts = nullptr;
    unsigned* ticket = nullptr;
    if ((s = search_state(st, &ls, &parts, &ticket)) != PR_OK) return s;
    return run_phi(x, d, t0, cap, n, beta, power, alphas, m, out, parts, ticket, st);
}

pr_status pr_golden_iterations(double lo, double hi, double tol, int32_t* count) {
    g_msg.clear();
    if (!count) return fail(PR_ERR_INVALID, "count is NULL");
    if (!std::isfinite(lo) || !std::isfinite(hi) || !(lo < hi)) return fail(PR_ERR_INVALID, "need finite lo < hi");
    if (!std::isfinite(tol) || !(tol > 0.0)) return fail(PR_ERR_INVALID, "tol must be finite and > 0");
    const double r = (std::sqrt(5.0) - 1.0) / 2.0;
    const double w = hi - lo;
    int k = 0;
    while (w * std::pow(r, (double)k) > tol) {
        if (++k > 200) return fail(PR_ERR_INVALID, "tolerance %g needs more than 200 iterations", tol);
    }
    *count = k;
    return PR_OK;
}

pr_status pr_line_search(const float* x, const float* d, const float* t0, const float* cap, int64_t n, float beta,
                         int32_t power, double lo, double hi, pr_search method, int32_t count, int32_t depth,
                         double* result, pr_stream_t stream) {
    g_msg.clear();
    pr_status s = check_links(x, d, t0, cap, n, beta, power);
    if (s != PR_OK) return s;
    if (!std::isfinite(lo) || !std::isfinite(hi) || !(lo < hi)) return fail(PR_ERR_INVALID, "need finite lo < hi");
    if (method != PR_SEARCH_GOLDEN && method != PR_SEARCH_FIBONACCI) return fail(PR_ERR_INVALID, "unknown method");
    if (method == PR_SEARCH_GOLDEN && (count < 0 || count > 200))
        return fail(PR_ERR_INVALID, "golden-section iterations must be in [0, 200]");
    if (method == PR_SEARCH_FIBONACCI && (count < 3 || count > 78))
        return fail(PR_ERR_INVALID, "Fibonacci evaluations must be in [3, 78]");
    if (depth < 1 || depth > kLsMaxDepth) return fail(PR_ERR_INVALID, "depth must be in [1, %d]", kLsMaxDepth);
    if (!result || reinterpret_cast<uintptr_t>(result) % 8) return fail(PR_ERR_INVALID, "result must be 8-byte aligned");
    ensure_registered();
    cudaStream_t st = (cudaStream_t)stream;
    LsState* ls = nullptr;
    double* parts = nullptr;
    unsigned* ticket = nullptr;
    if ((s = search_state(st, &ls, &parts, &ticket)) != PR_OK) return s;
    const int total = method == PR_SEARCH_GOLDEN ? count : count - 2;
    PR_INJECT_LAUNCH();
    cudaError_t err = launch_ls_init(ls, lo, hi, (int)method, count, total, depth, st);
    if (err != cudaSuccess) return fail(PR_ERR_CUDA, "search init launch: %s", cudaGetErrorString(err));
    // passes: the first evaluates x1, x2 and the next min(depth, total)
    // iterations' tree, each later one the next min(depth, left) iterations'
    int iter = 0;
    for (bool first = true; first || iter < total; first = false) {
        const int lv = total - iter < depth ? total - iter : depth;
        const int m = (first ? 2 : 0) + (2 << lv) - 2;
        if ((s = run_phi(x, d, t0, cap, n, beta, power, ls->pts, m, ls->vals, parts, ticket, st, ls, result)) !=
            PR_OK)
            return s;
        iter += lv;
    }
    return PR_OK;
}

pr_status pr_debug_inject_fault(int32_t site, int32_t after, int32_t* pending) {
    g_msg.clear();
    if (site < PR_FAULT_NONE || site > PR_FAULT_LAUNCH) return fail(PR_ERR_INVALID, "unknown fault site %d", site);
    if (after < 0) return fail(PR_ERR_INVALID, "after must be >= 0");
    std::lock_guard<std::mutex> lk(g_fault_mu);
    if (pending) *pending = g_fault_site.load() != PR_FAULT_NONE;
    g_fault_after = after;
    g_fault_site.store(site);
    return PR_OK;
}

pr_status pr_debug_reduce_plan(const void* x, int64_t n, pr_dtype dtype, pr_op op, pr_precision precision,
                               int32_t arg, pr_stream_t stream, int32_t* grid, int32_t* block,
                               int64_t* tail_vectors) {
    g_msg.clear();
    pr_status s = check_common(dtype, op, arg ? PR_PREC_PLAIN : precision);
    if (s != PR_OK) return s;
    if (arg && op != PR_MAX && op != PR_MIN) return fail(PR_ERR_UNSUPPORTED, "arg-extremum needs MAX or MIN");
    if (n < 0) return fail(PR_ERR_INVALID, "n must be >= 0 (got %lld)", (long long)n);
    if (!x && n > 0) return fail(PR_ERR_INVALID, "x is NULL");
    if ((s = check_aligned(x, dtype, "x")) != PR_OK) return s;
    ensure_registered();
    const int prec = arg ? PR_PREC_PLAIN : precision;
    const pr_config c = arg ? default_cfg(PR_KIND_REDUCE, dtype, op, prec) : lookup_cfg(PR_KIND_REDUCE, dtype, op, prec, n);
    ReducePlan pl;
    s = plan_reduce(x, n, dtype, op, prec, false, nullptr, nullptr, (cudaStream_t)stream, c,
                    arg ? AUX_ARG : AUX_NONE, nullptr, &pl);
    if (s != PR_OK) return s;
    if (grid) *grid = pl.grid;
    if (block) *block = pl.c.block;
    if (tail_vectors) {
        const int64_t ve = pl.c.vec_bytes / elem_size(dtype);
        *tail_vectors = pl.a.tile_vec > 0 ? (n - pl.a.head) / ve - pl.a.stat : 0;
    }
    return PR_OK;
}

pr_status pr_prepare(pr_stream_t stream) {
    g_msg.clear();
    ensure_registered();
    Workspace ws;
    return get_ws((cudaStream_t)stream, &ws);
}

pr_status pr_last_device_error(pr_stream_t stream, int32_t* code) {
    g_msg.clear();
    if (!code) return fail(PR_ERR_INVALID, "code is NULL");
    *code = PR_OK;
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    Workspace ws;
    bool have = false;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_ws.find(std::make_pair(dev, (cudaStream_t)stream));
        if (it != g_ws.end()) { ws = it->second.ws; have = true; }
    }
    PR_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (!have) return PR_OK;
    int32_t v = 0;
    PR_CUDA(cudaMemcpy(&v, ws.err, sizeof v, cudaMemcpyDeviceToHost));
    if (v != 0) {
        // A launch that saw malformed input may have left tickets armed: re-zero them.
        PR_CUDA(cudaMemset(ws.seg_cnt, 0, (size_t)(ws.gmax + 64) * 4));
        *code = v;
    }
    return PR_OK;
}

// ------------------------------------------------------------------------
// End to end from host memory
// ------------------------------------------------------------------------

namespace {
struct HostPipe {
    char* stage[2] = {nullptr, nullptr};
    char* parts = nullptr;
    size_t parts_cap = 0;
    void* dout = nullptr;
    cudaStream_t copy = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr};
    cudaEvent_t consumed[2] = {nullptr, nullptr};
};
std::map<int, HostPipe> g_pipes;
std::mutex g_pipe_mu;
constexpr size_t kChunkBytes = (size_t)64 << 20;
}  // namespace

pr_status pr_reduce_host(const void* host_x, int64_t n, pr_dtype dtype, pr_op op, void* host_out,
                         pr_stream_t stream) {
    g_msg.clear();
    pr_status s = check_common(dtype, op, PR_PREC_PLAIN);
    if (s != PR_OK) return s;
    if (n < 0) return fail(PR_ERR_INVALID, "n must be >= 0");
    if (!host_x && n > 0) return fail(PR_ERR_INVALID, "host_x is NULL");
    if (!host_out) return fail(PR_ERR_INVALID, "host_out is NULL");
    if ((s = check_aligned(host_x, dtype, "host_x")) != PR_OK) return s;
    ensure_registered();
    const KernelEntry* ce = reg_find(KernelKey{K_COMBINE, (uint8_t)dtype, (uint8_t)op, 0, AUX_NONE, 0, 0});
    if (!ce) return fail(PR_ERR_UNSUPPORTED, "no combine kernel for dtype %d op %d", dtype, op);
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    HostPipe& hp = g_pipes[dev];
    if (!hp.copy) {
        // staging buffers, events and the copy stream: kept only when all were made
        HostPipe fresh;
        auto release = [&fresh]() {
            for (int b = 0; b < 2; b++) {
                if (fresh.stage[b]) cudaFree(fresh.stage[b]);
                if (fresh.copied[b]) cudaEventDestroy(fresh.copied[b]);
                if (fresh.consumed[b]) cudaEventDestroy(fresh.consumed[b]);
            }
            if (fresh.dout) cudaFree(fresh.dout);
            cudaGetLastError();
        };
        bool ok = true;
        for (int b = 0; b < 2 && ok; b++) {
            ok = !inject(PR_FAULT_ALLOC) && cudaMalloc(&fresh.stage[b], kChunkBytes) == cudaSuccess &&
                 cudaEventCreateWithFlags(&fresh.copied[b], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&fresh.consumed[b], cudaEventDisableTiming) == cudaSuccess;
        }
        ok = ok && !inject(PR_FAULT_ALLOC) && cudaMalloc(&fresh.dout, 64) == cudaSuccess &&
             cudaStreamCreateWithFlags(&fresh.copy, cudaStreamNonBlocking) == cudaSuccess;
        if (!ok) {
            release();
            return fail(PR_ERR_NOMEM, "host pipeline: staging allocation failed");
        }
        hp = fresh;
    }
    const int es = elem_size(dtype);
    const int64_t chunk = (int64_t)(kChunkBytes / (size_t)es);
    const int64_t nchunks = n == 0 ? 1 : (n + chunk - 1) / chunk;
    if ((size_t)nchunks * kSlot > hp.parts_cap) {
        PR_CUDA(cudaStreamSynchronize(st));
        if (hp.parts) PR_CUDA(cudaFree(hp.parts));
        hp.parts = nullptr;
        hp.parts_cap = 0;
        PR_INJECT_ALLOC();
        if (cudaMalloc(&hp.parts, (size_t)nchunks * kSlot) != cudaSuccess) {
            cudaGetLastError();
            hp.parts = nullptr;
            return fail(PR_ERR_NOMEM, "host pipeline: chunk partials allocation failed");
        }
        hp.parts_cap = (size_t)nchunks * kSlot;
    }
    const pr_config c = lookup_cfg(PR_KIND_REDUCE, dtype, op, 0, chunk < n ? chunk : n);
    // The copy stream starts after everything already queued on `st`.  On a
    // failure part-way, the copies already queued may still be reading
    // host_x: wait for them (and for st) before returning, so that the caller
    // may free or reuse host_x as soon as the call returns.
    auto drain = [&](pr_status st_fail) {
        cudaStreamSynchronize(hp.copy);
        cudaStreamSynchronize(st);
        cudaGetLastError();
        return st_fail;
    };
#define PR_HOST_CUDA(call)                                                                          \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return drain(fail(PR_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_))); \
    } while (0)
    PR_HOST_CUDA(cudaEventRecord(hp.consumed[0], st));
    PR_HOST_CUDA(cudaStreamWaitEvent(hp.copy, hp.consumed[0], 0));
    PR_HOST_CUDA(cudaEventRecord(hp.consumed[1], st));
    for (int64_t k = 0; k < nchunks; k++) {
        const int b = (int)(k & 1);
        const int64_t lo = k * chunk;
        const int64_t len = n - lo < chunk ? n - lo : chunk;
        PR_HOST_CUDA(cudaStreamWaitEvent(hp.copy, hp.consumed[b], 0));
        if (len > 0)
            PR_HOST_CUDA(cudaMemcpyAsync(hp.stage[b], static_cast<const char*>(host_x) + lo * es, (size_t)len * es,
                                         cudaMemcpyHostToDevice, hp.copy));
        PR_HOST_CUDA(cudaEventRecord(hp.copied[b], hp.copy));
        PR_HOST_CUDA(cudaStreamWaitEvent(st, hp.copied[b], 0));
        s = run_reduce(hp.stage[b], len, dtype, op, 0, false, nullptr, hp.parts + k * kSlot, st, c);
        if (s != PR_OK) return drain(s);
        PR_HOST_CUDA(cudaEventRecord(hp.consumed[b], st));
    }
    if (inject(PR_FAULT_LAUNCH)) return drain(fail(PR_ERR_CUDA, "kernel launch failed (injected by the test hook)"));
    cudaError_t err = reinterpret_cast<CombineLaunch>(ce->launch)(hp.parts, (int)nchunks, hp.dout, 0, st);
    if (err != cudaSuccess) return drain(fail(PR_ERR_CUDA, "combine launch: %s", cudaGetErrorString(err)));
    PR_HOST_CUDA(cudaMemcpyAsync(host_out, hp.dout, (size_t)out_size(dtype, op), cudaMemcpyDeviceToHost, st));
#undef PR_HOST_CUDA
    PR_CUDA(cudaStreamSynchronize(st));
    return PR_OK;
}

// ------------------------------------------------------------------------
// Tuning
// ------------------------------------------------------------------------

pr_status pr_get_config(pr_kind kind, pr_dtype dtype, pr_op op, pr_precision precision, int64_t n, pr_config* cfg) {
    g_msg.clear();
    if (!cfg) return fail(PR_ERR_INVALID, "cfg is NULL");
    if (kind < PR_KIND_REDUCE || kind > PR_KIND_AXIS) return fail(PR_ERR_INVALID, "unknown kind");
    *cfg = lookup_cfg(kind, dtype, op, precision, n);
    return PR_OK;
}

pr_status pr_set_config(pr_kind kind, pr_dtype dtype, pr_op op, pr_precision precision, int64_t n,
                        const pr_config* cfg) {
    g_msg.clear();
    if (kind < PR_KIND_REDUCE || kind > PR_KIND_AXIS) return fail(PR_ERR_INVALID, "unknown kind");
    if (!cfg || !cfg_valid(*cfg, kind)) return fail(PR_ERR_INVALID, "invalid configuration for kind %d", kind);
    std::lock_guard<std::mutex> lk(g_mu);
    g_tuned[CfgKey{kind, dtype, op, precision, bucket_of(n)}] = *cfg;
    return PR_OK;
}

// Time every candidate configuration of `kind` with CUDA events on st (two
// warm-up runs, best of five) and return the fastest; *best_ms stays 1e30
// when no candidate could run.
static pr_status tune_candidates(int kind, cudaStream_t st, const std::function<pr_status(const pr_config&)>& run,
                                 pr_config* best_c, float* best_ms) {
    cudaEvent_t e0, e1;
    PR_CUDA(cudaEventCreate(&e0));
    PR_CUDA(cudaEventCreate(&e1));
    *best_ms = 1e30f;
    const int blocks[] = {64, 128, 256, 512, 1024};
    const int bpss[] = {1, 2, 4, 8};
    pr_status s = PR_OK;
    for (int blk : blocks)
        for (int bps : bpss) {
            if (blk * bps > 2048 || !cfg_valid(pr_config{blk, bps, 2, 16}, kind)) continue;
            if (blk == 64 && kind != PR_KIND_AXIS) continue;
            for (int u : kUnrolls)
                for (int vb : kVecBytes) {
                    const pr_config c{blk, bps, u, vb};
                    bool ok = true;
                    for (int w = 0; w < 2 && ok; w++) ok = run(c) == PR_OK;
                    if (!ok) continue;
                    float t_min = 1e30f;
                    for (int r = 0; r < 5 && ok; r++) {
                        if (cudaEventRecord(e0, st) != cudaSuccess) { s = PR_ERR_CUDA; break; }
                        ok = run(c) == PR_OK;
                        cudaEventRecord(e1, st);
                        cudaEventSynchronize(e1);
                        float ms = 0;
                        cudaEventElapsedTime(&ms, e0, e1);
                        t_min = ms < t_min ? ms : t_min;
                    }
                    if (ok && t_min < *best_ms) {
                        *best_ms = t_min;
                        *best_c = c;
                    }
                }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return s == PR_OK ? PR_OK : fail(s, "autotune: a CUDA event call failed");
}

static void keep_tuned(int kind, int dtype, int op, int prec, int64_t bucket_n, const pr_config& c, float best_ms) {
    std::lock_guard<std::mutex> lk(g_mu);
    const CfgKey key{kind, dtype, op, prec, bucket_of(bucket_n)};
    if (best_ms >= 1e30f) g_tuned.erase(key);   // no candidate ran: keep the default
    else g_tuned[key] = c;
}

pr_status pr_autotune(pr_kind kind, const void* x, int64_t n, const int64_t* offsets, int64_t nseg, pr_dtype dtype,
                      pr_op op, pr_precision precision, pr_stream_t stream, pr_config* best) {
    g_msg.clear();
    pr_status s = check_common(dtype, op, precision);
    if (s != PR_OK) return s;
    if (kind != PR_KIND_REDUCE && kind != PR_KIND_SEGMENTED && kind != PR_KIND_ROWS)
        return fail(PR_ERR_UNSUPPORTED, "autotune covers PR_KIND_REDUCE, PR_KIND_SEGMENTED and PR_KIND_ROWS "
                                        "(pr_autotune_axis for PR_KIND_AXIS)");
    if (kind == PR_KIND_REDUCE && (n <= 0 || !x)) return fail(PR_ERR_INVALID, "autotune needs data (x, n > 0)");
    if (kind == PR_KIND_SEGMENTED && (nseg <= 0 || !offsets || !x))
        return fail(PR_ERR_INVALID, "autotune needs x, offsets and nseg > 0");
    if (kind == PR_KIND_ROWS && (nseg <= 0 || n <= 0 || n % nseg != 0 || !x))
        return fail(PR_ERR_INVALID, "autotune needs x and rows (nseg) > 0 dividing n");
    // rows are tuned with the outputs the differentiation forward asks for
    const int row_aux = (op == PR_MAX || op == PR_MIN) ? AUX_ARG
                        : (op == PR_PROD && (dtype == PR_F32 || dtype == PR_F64)) ? AUX_PROD : AUX_NONE;
    if ((s = check_aligned(x, dtype, "x")) != PR_OK) return s;
    ensure_registered();
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    PR_CUDA(cudaStreamIsCapturing(st, &cap));
    if (cap != cudaStreamCaptureStatusNone) return fail(PR_ERR_INVALID, "autotune cannot run during capture");
    const int64_t nout = kind == PR_KIND_REDUCE ? 1 : nseg;
    void* dout = nullptr;
    PR_CUDA(cudaMalloc(&dout, (size_t)nout * (8 + sizeof(pr_prod_aux))));
    int64_t* dargs = reinterpret_cast<int64_t*>(static_cast<char*>(dout) + nout * 8);
    pr_prod_aux* daux = reinterpret_cast<pr_prod_aux*>(static_cast<char*>(dout) + nout * 8);
    pr_config best_c = default_cfg(kind, dtype, op, precision);
    float best_ms = 1e30f;
    s = tune_candidates(kind, st, [&](const pr_config& c) -> pr_status {
        if (kind == PR_KIND_REDUCE) return run_reduce(x, n, dtype, op, precision, false, dout, nullptr, st, c);
        if (kind == PR_KIND_ROWS)
            return run_rows(x, nseg, n / nseg, dtype, op, precision, row_aux, dout, row_aux == AUX_ARG ? dargs : nullptr,
                            row_aux == AUX_PROD ? daux : nullptr, st, c);
        return run_segmented(x, offsets, 0, nseg, dtype, op, precision, AUX_NONE, dout, nullptr, nullptr, st, c);
    }, &best_c, &best_ms);
    cudaFree(dout);
    if (s != PR_OK) return s;
    g_msg.clear();
    keep_tuned(kind, dtype, op, precision, kind == PR_KIND_SEGMENTED ? nseg : n, best_c, best_ms);
    if (best) *best = best_c;
    return PR_OK;
}

pr_status pr_autotune_axis(const void* x, int64_t outer, int64_t n, int64_t inner, pr_dtype dtype, pr_op op,
                           pr_precision precision, pr_stream_t stream, pr_config* best) {
    g_msg.clear();
    pr_status s = check_common(dtype, op, precision);
    if (s != PR_OK) return s;
    if (outer <= 0 || n <= 0 || inner <= 1 || !x)
        return fail(PR_ERR_INVALID, "axis autotune needs x, outer > 0, n > 0 and inner > 1");
    const int64_t lim = (int64_t)1 << 62;
    if (outer > lim / inner || outer * inner > lim / n) return fail(PR_ERR_INVALID, "outer*n*inner overflows");
    if ((s = check_aligned(x, dtype, "x")) != PR_OK) return s;
    ensure_registered();
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    PR_CUDA(cudaStreamIsCapturing(st, &cap));
    if (cap != cudaStreamCaptureStatusNone) return fail(PR_ERR_INVALID, "autotune cannot run during capture");
    const int aux = (op == PR_MAX || op == PR_MIN) ? AUX_ARG
                    : (op == PR_PROD && (dtype == PR_F32 || dtype == PR_F64)) ? AUX_PROD : AUX_NONE;
    const int64_t nout = outer * inner;
    void* dout = nullptr;
    PR_CUDA(cudaMalloc(&dout, (size_t)nout * (8 + sizeof(pr_prod_aux))));
    int64_t* dargs = reinterpret_cast<int64_t*>(static_cast<char*>(dout) + nout * 8);
    pr_prod_aux* daux = reinterpret_cast<pr_prod_aux*>(static_cast<char*>(dout) + nout * 8);
    pr_config best_c = default_cfg(PR_KIND_AXIS, dtype, op, precision);
    float best_ms = 1e30f;
    s = tune_candidates(PR_KIND_AXIS, st, [&](const pr_config& c) -> pr_status {
        return run_axis(x, outer, n, inner, dtype, op, precision, aux, dout, aux == AUX_ARG ? dargs : nullptr,
                        aux == AUX_PROD ? daux : nullptr, st, c);
    }, &best_c, &best_ms);
    cudaFree(dout);
    if (s != PR_OK) return s;
    g_msg.clear();
    keep_tuned(PR_KIND_AXIS, dtype, op, precision, outer * n * inner, best_c, best_ms);
    if (best) *best = best_c;
    return PR_OK;
}

pr_status pr_tune_save(const char* path) {
    g_msg.clear();
    if (!path) return fail(PR_ERR_INVALID, "path is NULL");
    DevInfo di;
    pr_status s = device_info(&di, nullptr);
    if (s != PR_OK) return s;
    FILE* f = fopen(path, "w");
    if (!f) return fail(PR_ERR_INVALID, "cannot open %s for writing", path);
    std::lock_guard<std::mutex> lk(g_mu);
    fprintf(f, "{\"gpu\": \"%s\", \"entries\": [\n", di.name.c_str());
    bool first = true;
    for (auto& kv : g_tuned) {
        int kind, dtype, op, prec, bucket;
        std::tie(kind, dtype, op, prec, bucket) = kv.first;
        const pr_config& c = kv.second;
        fprintf(f, "%s {\"kind\": %d, \"dtype\": %d, \"op\": %d, \"precision\": %d, \"bucket\": %d, \"block\": %d, "
                   "\"blocks_per_sm\": %d, \"unroll\": %d, \"vec_bytes\": %d}",
                first ? "" : ",\n", kind, dtype, op, prec, bucket, c.block, c.blocks_per_sm, c.unroll, c.vec_bytes);
        first = false;
    }
    fprintf(f, "\n]}\n");
    fclose(f);
    return PR_OK;
}

pr_status pr_tune_load(const char* path) {
    g_msg.clear();
    if (!path) return fail(PR_ERR_INVALID, "path is NULL");
    DevInfo di;
    pr_status s = device_info(&di, nullptr);
    if (s != PR_OK) return s;
    FILE* f = fopen(path, "r");
    if (!f) return fail(PR_ERR_INVALID, "cannot open %s", path);
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
    fclose(f);
    const std::string want = "\"gpu\": \"" + di.name + "\"";
    if (text.find(want) == std::string::npos) return fail(PR_ERR_INVALID, "tuning file is for another GPU");
    size_t pos = 0;
    int loaded = 0;
    std::map<CfgKey, pr_config> fresh;
    while ((pos = text.find("{\"kind\"", pos)) != std::string::npos) {
        int kind, dtype, op, prec, bucket;
        pr_config c;
        if (sscanf(text.c_str() + pos,
                   "{\"kind\": %d, \"dtype\": %d, \"op\": %d, \"precision\": %d, \"bucket\": %d, \"block\": %d, "
                   "\"blocks_per_sm\": %d, \"unroll\": %d, \"vec_bytes\": %d}",
                   &kind, &dtype, &op, &prec, &bucket, &c.block, &c.blocks_per_sm, &c.unroll, &c.vec_bytes) != 9 ||
            !cfg_valid(c, kind))
            return fail(PR_ERR_INVALID, "malformed tuning entry at byte %zu", pos);
        fresh[CfgKey{kind, dtype, op, prec, bucket}] = c;
        loaded++;
        pos++;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& kv : fresh) g_tuned[kv.first] = kv.second;
    return PR_OK;
}

}  // extern "C"
