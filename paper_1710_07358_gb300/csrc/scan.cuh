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

// Tiles of 256 x 128 input bytes (32 KB).  A block serialises claim, load,
// look-back and stores per tile, and the look-back frontier must keep up with
// the tiles HBM streams in, so tiles are large and several blocks share an SM
// (measured on GB300, 2^28 uint32 prefix sums: 16 KB tiles 601 us, 32 KB tiles
// 544 us, 64 KB tiles 661 us).
constexpr int kScanThreads = 256;
constexpr int kScanBytes = 128;         // input bytes per thread and tile

// One bounded wait on a tile state nothing publishes (zero-filled, epoch 1).
cudaError_t launch_wait_probe(ScanTile* t, int spin, int* err, cudaStream_t st);

}  // namespace pr
