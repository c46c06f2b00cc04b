// Launchers and registration helpers, included by the instantiation units.
#pragma once
#include "axis.cuh"
#include "kernels.cuh"
#include "registry.h"

namespace pr {

template <class T, int U, int VB, bool TAIL>
cudaError_t launch_reduce(const ReduceArgs& a, int grid, int block, cudaStream_t st) {
    reduce_kernel<T, U, VB, TAIL>()<<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

template <class T, int U, int VB>
cudaError_t launch_segmented(const SegArgs& a, int grid, int block, cudaStream_t st) {
    k_segmented<T, U, VB><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

template <class T, int U, int VB>
cudaError_t launch_rows(const RowArgs& a, int grid, int block, cudaStream_t st) {
    k_rows<T, U, VB><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

template <class T, int U, int VB>
cudaError_t launch_axis(const AxisArgs& a, int grid, int block, cudaStream_t st) {
    k_axis<T, U, VB><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_axis_finish(const AxisArgs& a, int grid, int block, cudaStream_t st) {
    k_axis_finish<T><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_axis_empty(const AxisArgs& a, int grid, int block, cudaStream_t st) {
    k_axis_empty<T><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_combine(const char* parts, int count, void* out, int out_f64, cudaStream_t st) {
    k_combine_parts<T><<<1, 256, 0, st>>>(parts, count, out, out_f64);
    return cudaGetLastError();
}

template <class T, int U, int VB>
void reg_one(uint8_t dtype, uint8_t op, uint8_t prec, uint8_t aux, bool plain, bool seg) {
    if (plain) {
        reg_add(KernelKey{K_REDUCE, dtype, op, prec, aux, (uint8_t)U, (uint8_t)VB},
                KernelEntry{reinterpret_cast<const void*>(reduce_kernel<T, U, VB, false>()),
                            reinterpret_cast<void*>(&launch_reduce<T, U, VB, false>)});
        KernelEntry et{reinterpret_cast<const void*>(reduce_kernel<T, U, VB, true>()),
                       reinterpret_cast<void*>(&launch_reduce<T, U, VB, true>)};
        et.tile_slots = TileSlots<T>::value;
        et.tile_loads = TileLoads<T, U>::value;
        reg_add(KernelKey{K_REDUCE_TAIL, dtype, op, prec, aux, (uint8_t)U, (uint8_t)VB}, et);
    }
    if (seg) {
        reg_add(KernelKey{K_SEGMENTED, dtype, op, prec, aux, (uint8_t)U, (uint8_t)VB},
                KernelEntry{reinterpret_cast<const void*>(&k_segmented<T, U, VB>),
                            reinterpret_cast<void*>(&launch_segmented<T, U, VB>)});
        // equal rows (the differentiation forwards) get the lighter row kernel
        reg_add(KernelKey{K_ROWS, dtype, op, prec, aux, (uint8_t)U, (uint8_t)VB},
                KernelEntry{reinterpret_cast<const void*>(&k_rows<T, U, VB>),
                            reinterpret_cast<void*>(&launch_rows<T, U, VB>)});
    }
}

template <class T, int U, int VB>
void reg_axis(uint8_t dtype, uint8_t op, uint8_t prec, uint8_t aux) {
    KernelEntry e{reinterpret_cast<const void*>(&k_axis<T, U, VB>), reinterpret_cast<void*>(&launch_axis<T, U, VB>)};
    e.part_bytes = (int)sizeof(typename GridR<T>::Part);
    reg_add(KernelKey{K_AXIS, dtype, op, prec, aux, (uint8_t)U, (uint8_t)VB}, e);
}

// Register every (unroll, vector width) of one trait; plain-reduce traits
// also get the chunk-partial combiner used by the host-memory path, and
// segmented ones the axis kernels (vector widths 16 and 32, and 0 for
// columns that are not a whole number of vectors).
template <class T>
void reg_family(uint8_t dtype, uint8_t op, uint8_t prec, uint8_t aux, bool plain, bool seg) {
    reg_one<T, 2, 16>(dtype, op, prec, aux, plain, seg);
    reg_one<T, 2, 32>(dtype, op, prec, aux, plain, seg);
    reg_one<T, 4, 16>(dtype, op, prec, aux, plain, seg);
    reg_one<T, 4, 32>(dtype, op, prec, aux, plain, seg);
    if (seg) {
        reg_axis<T, 2, 0>(dtype, op, prec, aux);
        reg_axis<T, 2, 16>(dtype, op, prec, aux);
        reg_axis<T, 2, 32>(dtype, op, prec, aux);
        reg_axis<T, 4, 0>(dtype, op, prec, aux);
        reg_axis<T, 4, 16>(dtype, op, prec, aux);
        reg_axis<T, 4, 32>(dtype, op, prec, aux);
        reg_add(KernelKey{K_AXIS_FINISH, dtype, op, prec, aux, 0, 0},
                KernelEntry{reinterpret_cast<const void*>(&k_axis_finish<T>),
                            reinterpret_cast<void*>(&launch_axis_finish<T>)});
        reg_add(KernelKey{K_AXIS_EMPTY, dtype, op, prec, aux, 0, 0},
                KernelEntry{reinterpret_cast<const void*>(&k_axis_empty<T>),
                            reinterpret_cast<void*>(&launch_axis_empty<T>)});
    }
    if (plain) {
        reg_add(KernelKey{K_COMBINE, dtype, op, prec, aux, 0, 0},
                KernelEntry{reinterpret_cast<const void*>(&k_combine_parts<T>),
                            reinterpret_cast<void*>(&launch_combine<T>)});
    }
}

}  // namespace pr
