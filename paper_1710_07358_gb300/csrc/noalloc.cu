// pr_reduce_noalloc: the plain reduction for callers that must not allocate.
//
// Some callers cannot call cudaMalloc at the point where they reduce: code
// running inside a memory pool or arena that owns every device allocation,
// allocation-free real-time paths, and hosts that forbid the implicit
// first-use allocation pr_reduce makes for its per-stream workspace.  This
// entry point needs no library-allocated memory at all: the partials of the
// one-launch reduction and its completion ticket live in the file-scope device
// array below, which exists on every GPU that loads this library until the
// process exits.
//
// Limits and rules (stated for users of this entry point):
//   - the array holds kNoAllocMaxBlocks block partials; a launch that would
//     need more is rejected with PR_ERR_UNSUPPORTED before anything runs
//     (GB300 uses 304);
//   - every call shares the one array: calls whose kernels overlap on the GPU
//     (e.g. on two streams) race and give wrong results; serialise them;
//   - the first call on a device looks up the array's device address there
//     (cudaGetSymbolAddress, with that device current); make that first call
//     before any stream capture;
//   - the ticket that must start at zero is cleared on the stream before every
//     launch; the partial slots are written before they are read in each call.
#include <cstdio>
#include <mutex>

#include "../../include/pr.h"
#include "kernels.cuh"
#include "registry.h"

namespace pr {
pr_status fail(pr_status s, const char* fmt, ...);
}

using namespace pr;

namespace {

constexpr int kNoAllocMaxBlocks = 1024;
constexpr size_t kTicketOffset = (size_t)kNoAllocMaxBlocks * kSlot;
constexpr size_t kNoAllocScratchBytes = kTicketOffset + 256;  // 64 KiB of slots + the ticket
constexpr int kMaxDevices = 64;
// Launch shape of this entry point: 512 threads, at most 2 blocks per SM,
// two 32-byte vectors per thread per step.
constexpr int kNaBlock = 512, kNaBlocksPerSm = 2, kNaUnroll = 2, kNaVecBytes = 32;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
char* g_scratch[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// Once per device, with that device current: the array's device address.
pr_status scratch_for(int dev, char** ptr, int* sms) {
    if (dev < 0 || dev >= kMaxDevices) return fail(PR_ERR_UNSUPPORTED, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return fail(PR_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return fail(PR_ERR_CUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
        g_sms[dev] = n;
        g_scratch[dev] = static_cast<char*>(p);
    }
    *ptr = g_scratch[dev];
    *sms = g_sms[dev];
    return PR_OK;
}

int elem_bytes(int d) { return (d == PR_F16 || d == PR_BF16) ? 2 : ((d == PR_F64 || d == PR_I64) ? 8 : 4); }

}  // namespace

extern "C" pr_status pr_reduce_noalloc(const void* x, int64_t n, pr_dtype dtype, pr_op op, void* out,
                                       pr_stream_t stream) {
    if (dtype < PR_F32 || dtype > PR_I64) return fail(PR_ERR_INVALID, "unknown dtype %d", dtype);
    if (op < PR_SUM || op > PR_XOR) return fail(PR_ERR_INVALID, "unknown op %d", op);
    const bool is_float = dtype == PR_F32 || dtype == PR_F16 || dtype == PR_BF16 || dtype == PR_F64;
    if (is_float && op >= PR_AND)
        return fail(PR_ERR_UNSUPPORTED, "bitwise combiner %d is not defined on floating-point dtype %d", op, dtype);
    if (n < 0) return fail(PR_ERR_INVALID, "n must be >= 0 (got %lld)", (long long)n);
    if (!x && n > 0) return fail(PR_ERR_INVALID, "x is NULL");
    if (!out) return fail(PR_ERR_INVALID, "out is NULL");
    const int es = elem_bytes(dtype);
    if (reinterpret_cast<uintptr_t>(x) % (uintptr_t)es) return fail(PR_ERR_INVALID, "x is not aligned to its element size");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(PR_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    char* scratch = nullptr;
    int sms = 0;
    pr_status s = scratch_for(dev, &scratch, &sms);
    if (s != PR_OK) return s;

    ensure_registered();
    const KernelEntry* k = reg_find(KernelKey{K_REDUCE, (uint8_t)dtype, (uint8_t)op, PR_PREC_PLAIN, AUX_NONE,
                                              (uint8_t)kNaUnroll, (uint8_t)kNaVecBytes});
    if (!k) return fail(PR_ERR_UNSUPPORTED, "no reduce kernel for dtype %d op %d", dtype, op);
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k->fn, kNaBlock, 0);
    if (e != cudaSuccess) return fail(PR_ERR_CUDA, "occupancy query: %s", cudaGetErrorString(e));
    if (occ < 1) return fail(PR_ERR_UNSUPPORTED, "reduce kernel cannot run with %d threads per block", kNaBlock);
    int64_t grid = (int64_t)sms * (occ < kNaBlocksPerSm ? occ : kNaBlocksPerSm);
    const int64_t per_block = (int64_t)kNaBlock * (kNaVecBytes / es) * kNaUnroll;
    const int64_t need = (n + per_block - 1) / per_block;
    if (need < grid) grid = need < 1 ? 1 : need;
    if (grid > kNoAllocMaxBlocks)
        return fail(PR_ERR_UNSUPPORTED, "this launch needs %lld block partials; the static scratch holds %d",
                    (long long)grid, kNoAllocMaxBlocks);

    Workspace ws{};
    ws.partials = scratch;
    ws.counter = reinterpret_cast<unsigned*>(scratch + kTicketOffset);
    ws.gmax = kNoAllocMaxBlocks;
    e = cudaMemsetAsync(ws.counter, 0, sizeof(unsigned), (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(PR_ERR_CUDA, "clearing the ticket: %s", cudaGetErrorString(e));

    const uintptr_t addr = reinterpret_cast<uintptr_t>(x);
    int64_t head = (int64_t)(((uintptr_t)kNaVecBytes - addr % (uintptr_t)kNaVecBytes) % (uintptr_t)kNaVecBytes) / es;
    if (head > n) head = n;
    ReduceArgs a{x, n, head, out, nullptr, 0, ws};
    e = reinterpret_cast<ReduceLaunch>(k->launch)(a, (int)grid, kNaBlock, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(PR_ERR_CUDA, "reduce launch: %s", cudaGetErrorString(e));
    return PR_OK;
}
