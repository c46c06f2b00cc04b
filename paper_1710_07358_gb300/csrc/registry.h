// Host-side table of compiled kernel variants.  Every instantiation unit
// registers, per (kind, dtype, combiner, precision, aux output), one entry per
// (unroll, vector width); the API picks the entry named by the launch
// configuration.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pr {

struct ReduceArgs;
struct SegArgs;
struct RowArgs;
struct AxisArgs;
struct AxisBwdArgs;
struct ScanArgs;
struct BwdArgs;

enum Kind : uint8_t {
    K_REDUCE = 0, K_SEGMENTED = 1, K_BACKWARD = 2, K_COMBINE = 3, K_ROWS = 4,
    K_AXIS = 5, K_AXIS_FINISH = 6, K_AXIS_EMPTY = 7, K_AXIS_BACKWARD = 8, K_SCAN = 9,
    K_REDUCE_TAIL = 10  // k_reduce with claimed tail tiles (large inputs)
};
enum Aux : uint8_t { AUX_NONE = 0, AUX_ARG = 1, AUX_PROD = 2 };

struct KernelKey {
    uint8_t kind, dtype, op, prec, aux, unroll, vb;
    bool operator<(const KernelKey& o) const;
};

using ReduceLaunch = cudaError_t (*)(const ReduceArgs&, int grid, int block, cudaStream_t);
using SegLaunch = cudaError_t (*)(const SegArgs&, int grid, int block, cudaStream_t);
using RowLaunch = cudaError_t (*)(const RowArgs&, int grid, int block, cudaStream_t);
using AxisLaunch = cudaError_t (*)(const AxisArgs&, int grid, int block, cudaStream_t);
using AxisBwdLaunch = cudaError_t (*)(const AxisBwdArgs&, int grid, int block, cudaStream_t);
using ScanLaunch = cudaError_t (*)(const ScanArgs&, int grid, int block, size_t smem, cudaStream_t);
using BwdLaunch = cudaError_t (*)(const BwdArgs&, int grid, int block, cudaStream_t);
using CombineLaunch = cudaError_t (*)(const char* parts, int count, void* out, int out_f64, cudaStream_t);

struct KernelEntry {
    const void* fn;      // the __global__ function (occupancy queries)
    void* launch;        // one of the *Launch types above, by kind
    int part_bytes = 0;  // K_AXIS: bytes of one cross-warp partial
    int tile_slots = 0;  // K_REDUCE_TAIL: claimed tiles a block holds partials for
    int tile_loads = 0;  // K_REDUCE_TAIL: vectors a thread loads per round of a tile
};

void reg_add(const KernelKey& k, const KernelEntry& e);
const KernelEntry* reg_find(const KernelKey& k);

// Unroll factors and vector widths compiled for every family.
constexpr int kUnrolls[] = {2, 4};
constexpr int kVecBytes[] = {16, 32};

void register_f32();
void register_f32_seg();
void register_f16();
void register_bf16();
void register_f64();
void register_i32();
void register_u32();
void register_i64();
void register_backward();
void register_scan();

// Registers every family above exactly once (thread-safe).
void ensure_registered();

}  // namespace pr
