// Layout shared by the scan kernel and the host: per-tile status records,
// launch arguments and the tile shape.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pr {

// One tile's status: the flag ((epoch << 2) | state: 1 aggregate, 2 inclusive
// prefix) travels with its value in one word that is written and read whole,
// so a reader never pairs a flag with a value from another state.
// Accumulators of at most 32 bits: the 64-bit word {flag, value}; 64-bit
// accumulators: the 16-byte word {flag, pad, value} (128-bit atomics).
struct alignas(32) ScanTile {
    unsigned flag;
    unsigned value32;
    unsigned long long value64;
    unsigned long long pad[2];
};

struct ScanArgs {
    const void* x;
    void* y;
    int64_t n;
    int64_t ntiles;
    int exclusive;
    ScanTile* tiles;
    unsigned* ctr;              // [0] next tile, [1] blocks done, [2] epoch
    int* err;
};

// Tiles of 32 KB of input, staged in a ring of kScanStages shared-memory
// buffers per block (224 KB: one block per SM).  Warps: one producer,
// kScanLookWarps look-back, kScanRedWarps reduction and kScanScanWarps
// scan-and-store warps; a look-back step reads kScanLookWin x 32 tile states.
constexpr int kScanTileBytes = 32768;
constexpr int kScanStages = 7;
constexpr int kScanLookWarps = 2;
constexpr int kScanRedWarps = 4;
constexpr int kScanScanWarps = 8;
constexpr int kScanLookWin = 1;
constexpr int kScanThreads = 32 * (1 + kScanLookWarps + kScanRedWarps + kScanScanWarps);

// One bounded wait on a tile state nothing publishes (zero-filled, epoch 1).
cudaError_t launch_wait_probe(ScanTile* t, int spin, int* err, cudaStream_t st);

}  // namespace pr
