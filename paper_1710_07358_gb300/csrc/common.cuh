// Device helpers shared by every reduction kernel: vector loads, shuffles of
// arbitrary trivially-copyable values, and the deterministic warp / block
// combines that replace the shared-memory tree of the two-stage scheme
// (Section 2.3, Listing 1's loop over halving offsets) and the shuffle
// reduction of Section 2.2.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_fp16.h>

namespace pr {

constexpr int kMaxWarps = 32;  // blocks of up to 1024 threads

// VB bytes loaded as VB/4 32-bit words.
template <int VB>
struct Words {
    uint32_t w[VB / 4];
};

// Read-only streaming vector load: bypasses L1 allocation (each byte is read
// exactly once), 16 B (v4) or 32 B (v8, sm_100+) per thread.
template <int VB>
__device__ __forceinline__ Words<VB> ldv(const void* p);

template <>
__device__ __forceinline__ Words<16> ldv<16>(const void* p) {
    Words<16> r;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(r.w[0]), "=r"(r.w[1]), "=r"(r.w[2]), "=r"(r.w[3])
        : "l"(p));
    return r;
}

template <>
__device__ __forceinline__ Words<32> ldv<32>(const void* p) {
    Words<32> r;
    asm("ld.global.nc.L1::no_allocate.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r.w[0]), "=r"(r.w[1]), "=r"(r.w[2]), "=r"(r.w[3]), "=r"(r.w[4]), "=r"(r.w[5]),
          "=r"(r.w[6]), "=r"(r.w[7])
        : "l"(p));
    return r;
}

// Shuffle any value whose size is a multiple of 4 bytes, word by word.
template <class T>
__device__ __forceinline__ T shfl_xor_any(const T& v, int mask) {
    static_assert(sizeof(T) % 4 == 0, "shuffled types are whole words");
    constexpr int NW = sizeof(T) / 4;
    uint32_t w[NW];
    memcpy(w, &v, sizeof(T));
#pragma unroll
    for (int i = 0; i < NW; i++) w[i] = __shfl_xor_sync(0xffffffffu, w[i], mask);
    T r;
    memcpy(&r, w, sizeof(T));
    return r;
}

// L2-coherent load of a value written by another block in the same launch.
template <class T>
__device__ __forceinline__ T ld_cg_any(const T* p) {
    static_assert(sizeof(T) % 4 == 0, "loaded types are whole words");
    constexpr int NW = sizeof(T) / 4;
    const uint32_t* q = reinterpret_cast<const uint32_t*>(p);
    uint32_t w[NW];
#pragma unroll
    for (int i = 0; i < NW; i++) w[i] = __ldcg(q + i);
    T r;
    memcpy(&r, w, sizeof(T));
    return r;
}

// Butterfly over the 32 lanes: every lane ends with the same value because
// every trait's combine is commutative bit for bit.  The association order is
// fixed, so the result is run-to-run deterministic.
template <class T>
__device__ __forceinline__ typename T::Part warp_combine(typename T::Part p) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) p = T::combine(p, shfl_xor_any(p, m));
    return p;
}

// Block combine: warp combine (or the trait's redux.sync form), one value per
// warp to shared memory, warp 0 combines those in warp order.  Every thread of
// the block must call it; the result is valid in thread 0.
template <class T>
__device__ __forceinline__ typename T::Part block_combine(typename T::Part p) {
    using Part = typename T::Part;
    __shared__ Part smem[kMaxWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    p = T::warp_reduce(p);
    __syncthreads();  // smem may still be read by a previous call
    if (lane == 0) smem[warp] = p;
    __syncthreads();
    if (warp == 0) {
        Part q = lane < nwarps ? smem[lane] : T::part_init();
        q = T::warp_reduce(q);
        p = q;
    }
    return p;
}

// 64-bit unsigned shift helpers that are defined for every count in [0, 64].
__device__ __forceinline__ uint64_t shl64(uint64_t v, int s) { return s >= 64 ? 0 : v << s; }

}  // namespace pr
