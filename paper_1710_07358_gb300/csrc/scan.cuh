// Layout shared by the scan kernel and the host: per-tile status records,
// launch arguments and the tile shape.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pr {

// The aggregate and the inclusive prefix have their own words: a reader that
// saw the aggregate flag must not pick up the inclusive value written later.
// Accumulators of at most 32 bits instead travel with the flag in one 64-bit
// word (flag in the low half, value in the high half).
struct ScanTile {
    unsigned flag;              // (epoch << 2) | state: 1 aggregate, 2 inclusive prefix
    unsigned pad;
    unsigned long long agg;     // the tile's own combination (written before state 1)
    unsigned long long incl;    // everything up to the tile's end (written before state 2)
    unsigned long long pad2;
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
