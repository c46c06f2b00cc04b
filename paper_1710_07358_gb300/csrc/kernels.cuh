// Reduction kernels.  Included by the per-dtype instantiation units only.
//
// k_reduce     plain reduction of x[0..n) in ONE launch:
//   Step 1 (Section 2.3 / Section 3, "Unrolling the step 1"): a persistent grid
//     (Section 2.5) strides over the input in VB-byte vectors; each thread keeps
//     U independent accumulators and issues its U loads before accumulating,
//     so U*VB bytes per thread are in flight.  Elements before the first VB
//     boundary and after the last full vector are read as scalars (no access
//     outside [x, x+n); the identity is never needed as a load mask).
//   Step 3: the U accumulators are combined, then the warp (shuffle butterfly
//     or redux.sync), then the block (one value per warp in shared memory).
//   Large inputs (the TAIL variant): the grid-stride part stops at a
//     multiple of the grid's stride near nine tenths of the vectors, and the
//     rest is cut into tiles of whole rounds of blockDim x TL vectors (about
//     128 KiB) that blocks claim from an atomic counter, a claim ahead.  SMs
//     stream at unequal rates (their finishing times spread over a few
//     microseconds), so a static split ends when the slowest SM does;
//     claimed tiles let the fast SMs take the slow ones' share of the end.
//     An exact trait adds the tiles to its accumulators; any other reduces
//     each tile like a block partial, stored in a slot indexed by the tile,
//     so the result does not depend on which block took which tile.
//   Stage 2 (Section 2.3), fused: every block stores its partial; the last
//     block to finish (atomic ticket after a fence) combines all partials in
//     block-index order, then the tile partials in tile order, writes the
//     result and re-arms the ticket and claim counters.  A launch of one
//     block (small inputs) finishes with the same combine and no ticket.
//
// k_segmented  many reductions (segments of a CSR offsets array, or equal rows)
//   in one launch.  The element range [offsets[0], offsets[nseg]) is cut into
//   tiles of blockDim*U*VB bytes, and runs of tiles form chunks.  With many
//   segments per block there are two chunks per block, claimed dynamically
//   from an atomic counter so that blocks delayed by many segment boundaries
//   do not hold up the launch; with few, one static chunk per block.
//   Inside a tile that lies in one segment the block streams exactly like
//   k_reduce; a tile containing segment boundaries emits the finished
//   segment, reduces the segments that lie wholly inside the tile (short ones
//   one per warp, long ones with the whole block) and starts the next one.
//   A segment that crosses chunk boundaries leaves one partial per chunk it
//   touches (its first chunk's "tail" slot, later chunks' "head" slots); the
//   last of those chunks to finish (per-segment ticket) combines them in chunk
//   order.  Partials are indexed by chunk, not by block, so results are
//   deterministic for a fixed launch configuration whatever the claim order.
//
// k_rows       equal rows of `cols` elements (cols a multiple of the vector
//   width, x aligned to it): the flattened vectors are split into one run of
//   whole tiles per block; a block streams its run exactly like k_reduce and
//   finishes a row each time the run crosses a row end.  The first vectors of
//   the next row are loaded before that row's block combine, so loads stay in
//   flight through it.  A row shared by several blocks leaves one partial per
//   block (the first block's "tail" slot, later blocks' "head" slots); the
//   last of them to finish (per-row ticket) combines them in block order, so
//   results are deterministic for a fixed launch configuration.
//
// k_combine_parts  one block combining an array of partials in order.
#pragma once
#include <type_traits>
#include "traits.cuh"

namespace pr {

constexpr int kSlot = 64;      // bytes per partial slot (>= sizeof(Part) of every trait)
constexpr int kSmallSeg = 512; // segments up to this length are reduced by one warp
enum : int { kErrInvalid = 1, kErrTimeout = 4 };

struct Workspace {
    char* partials;      // gmax slots (k_reduce)
    char* head;          // gmax slots (k_segmented: first-segment partial of a block; k_reduce: tile partials)
    char* tail;          // gmax slots (k_segmented: last-segment partial of a block)
    unsigned* seg_cnt;   // gmax tickets (k_segmented), zero between launches
    unsigned* counter;   // 1 ticket (k_reduce), zero between launches
    unsigned* chunk_ctr; // next chunk (k_segmented) or tile (k_reduce) to claim, zero between launches
    unsigned* blk_done;  // blocks finished (k_segmented), zero between launches
    int* err;            // device error word
    int gmax;
};

struct ReduceArgs {
    const void* x;
    int64_t n;
    int64_t head;        // elements before the first VB-aligned element (< VE, <= n)
    void* out;
    void* part_out;      // non-null: store the final Part here instead of a result
    int out_f64;
    Workspace ws;
    int64_t* argidx;     // arg-extremum traits: index of the first extremum (may be null)
    int64_t stat = 0;      // tile_vec > 0: vectors (after the head) of the grid-stride part,
                           // a multiple of U x threads
    int64_t tile_vec = 0;  // > 0: the vectors past `stat` are claimed in tiles of about this
                           // many vectors (partials in ws.head); 0: no claimed tail
};

struct SegArgs {
    const void* x;
    const int64_t* off;  // nseg+1 CSR offsets, or null for equal rows of `cols`
    int64_t cols;
    int64_t nseg;
    int64_t shift;       // x's element offset from the previous VB boundary
    void* out;
    int64_t* argidx;
    pr_prod_aux* aux;
    int out_f64;
    int chunks_per_block;  // chunks (contiguous tile runs) per block
    int dynamic_chunks;    // 1: blocks claim chunks from an atomic counter; 0: chunk c -> block c mod grid
    Workspace ws;
};

struct RowArgs {
    const void* x;       // aligned to the vector width
    int64_t rows, cols;  // cols > 0, a multiple of the elements per vector
    void* out;
    int64_t* argidx;
    pr_prod_aux* aux;
    int out_f64;
    Workspace ws;
};

struct BwdArgs {
    const void* x;
    const void* g;
    const int64_t* argidx;
    const pr_prod_aux* aux;
    void* gi;
    int64_t rows, cols;
    int64_t shift;           // grad_in's element offset from the previous VB boundary
    int64_t chunks_per_row;
    int op;
};


// The value that crosses blocks: the trait's Part, combined with the trait's
// combine (the same one the warp and block stages use).
template <class T>
struct GridR {
    using Part = typename T::Part;
    __device__ __forceinline__ static Part up(const typename T::Part& p) { return p; }
    __device__ __forceinline__ static Part part_init() { return T::part_init(); }
    __device__ __forceinline__ static Part combine(const Part& a, const Part& b) { return T::combine(a, b); }
    __device__ __forceinline__ static Part warp_reduce(Part p) { return T::warp_reduce(p); }
    __device__ __forceinline__ static void store(void* out, int64_t i, const Part& p, bool f64) { T::store(out, i, p, f64); }
    __device__ __forceinline__ static void store_aux(int64_t* ai, pr_prod_aux* ax, int64_t i, const Part& p, int64_t sb) {
        T::store_aux(ai, ax, i, p, sb);
    }
};

// Largest block a trait's kernels are compiled for (a trait with a large
// per-thread state declares kMaxBlock to get more registers per thread); the
// host clamps launch configurations to it.
template <class T, class = void>
struct MaxBlock {
    static constexpr int value = 1024;
};
template <class T>
struct MaxBlock<T, std::void_t<decltype(T::kMaxBlock)>> {
    static constexpr int value = T::kMaxBlock;
};

// Blocks of the plain reduction that must fit on one SM at once (a trait
// declares kMinBlocks to cap its registers per thread; default 1).
template <class T, class = void>
struct MinBlocks {
    static constexpr int value = 1;
};
template <class T>
struct MinBlocks<T, std::void_t<decltype(T::kMinBlocks)>> {
    static constexpr int value = T::kMinBlocks;
};

// A trait whose combine is exact and independent of order (integer,
// bitwise, max / min and arg-extremum) declares kExact: claimed tail tiles
// then join its running accumulators, with no partial per tile.
template <class T, class = void>
struct Exact {
    static constexpr bool value = false;
};
template <class T>
struct Exact<T, std::void_t<decltype(T::kExact)>> {
    static constexpr bool value = T::kExact;
};

// Vectors a thread loads per round of a claimed tile: four for a float trait
// whose accumulator is one or two words and whose registers are not capped,
// U otherwise (exact traits add tiles to their running accumulators).
template <class T, int U, class = void>
struct TileLoads {
    static constexpr int value =
        (!Exact<T>::value && MinBlocks<T>::value == 1 && sizeof(typename T::Acc) <= 8 && U < 4) ? 4 : U;
};
template <class T, int U>
struct TileLoads<T, U, std::void_t<decltype(T::kTileLoads)>> {   // a trait's own choice
    static constexpr int value = T::kTileLoads;
};

// Claimed tail tiles a block of k_reduce holds partials for: one value per
// warp and tile in shared memory, up to 16 KiB (64 tiles of fp32 partials).
// Exact traits keep no tile partials.
template <class T>
struct TileSlots {
    static constexpr int kBytes = (MaxBlock<T>::value / 32) * (int)sizeof(typename T::Part);
    static constexpr int value = Exact<T>::value ? (1 << 20)
                               : (16384 / kBytes > 64 ? 64 : (16384 / kBytes < 4 ? 4 : 16384 / kBytes));
};

template <class T>
__device__ __forceinline__ typename T::Part* slot(char* base, int64_t i) {
    return reinterpret_cast<typename T::Part*>(base + i * kSlot);
}

// Combine a thread's U accumulators into one Part.
template <class T, int U>
__device__ __forceinline__ typename T::Part fold(typename T::Acc (&acc)[U]) {
    typename T::Part p = T::to_part(acc[0]);
#pragma unroll
    for (int u = 1; u < U; u++) p = T::combine(p, T::to_part(acc[u]));
    return p;
}

// ------------------------------------------------------------------------
// Plain reduction
// ------------------------------------------------------------------------

template <class T, int U, int VB, bool TAIL>
__device__ __forceinline__ void reduce_body(const ReduceArgs& a) {
    using Ld = typename T::Ld;
    using In = typename Ld::In;
    using E = typename Ld::E;
    using Part = typename T::Part;
    constexpr int VE = VB / Ld::ES;
    const In* x = static_cast<const In*>(a.x);

    typename T::Acc acc[U];
#pragma unroll
    for (int u = 0; u < U; u++) acc[u] = T::init();

    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t head = a.head;
    const int64_t nvec = (a.n - head) / VE;
    const bool dyn = TAIL && a.tile_vec > 0;
    int64_t nstat = nvec;                           // vectors of the grid-stride part
    if constexpr (TAIL) nstat = dyn ? a.stat : nvec;
    const char* xv = reinterpret_cast<const char*>(x + head);
    using GR = GridR<T>;
    using G = typename GR::Part;
    // claimed tiles: thread 0 makes the block's first two claims while the
    // loads of its last grid-stride step travel (claims made earlier would
    // hand out tiles by start order rather than by progress), keeps them in
    // shared memory, and then at each tile publishes the claim it made a
    // tile earlier and makes the next, so no warp waits for a claim's round
    // trip
    __shared__ unsigned s_claim[2], s_claim1;
    bool claimed = false;
    auto claim_first = [&]() {
        if constexpr (TAIL)
            if (dyn && !claimed && threadIdx.x == 0) {
                s_claim[0] = atomicAdd(a.ws.chunk_ctr, 1u);
                s_claim1 = atomicAdd(a.ws.chunk_ctr, 1u);
                claimed = true;
            }
    };

    int64_t i = tid;
    for (; i + (int64_t)(U - 1) * nth < nstat; i += (int64_t)U * nth) {
        Words<VB> w[U];
#pragma unroll
        for (int u = 0; u < U; u++) w[u] = ldv<VB>(xv + (i + u * nth) * VB);
        if (i + (int64_t)(2 * U - 1) * nth >= nstat) claim_first();   // the last step
#pragma unroll
        for (int u = 0; u < U; u++) {
            E e[VE];
            Ld::template dec<VB>(w[u], e);
            T::add_vec(acc[u], e, head + (i + u * nth) * VE);
        }
    }
    for (; i < nstat; i += nth) {
        Words<VB> w = ldv<VB>(xv + i * VB);
        E e[VE];
        Ld::template dec<VB>(w, e);
        T::add_vec(acc[0], e, head + i * VE);
    }
    if (tid < head) T::add(acc[0], Ld::one(x, tid), tid);
    for (int64_t j = head + nvec * VE + tid; j < a.n; j += nth) T::add(acc[0], Ld::one(x, j), j);
    claim_first();   // (a grid-stride part too short for the loop)
    unsigned c_next = ~0u;

    // claimed tiles: vectors [nstat, nvec) in tiles of R rounds of blockDim x
    // TL vectors (R from the requested tile size), the next claim issued with
    // a tile's first loads.  An exact trait adds them to its accumulators
    // (each still sees its vectors in increasing index order: tiles lie past
    // the grid-stride part and a block's claims increase), with U loads a
    // thread.  Any other trait reduces each tile like a block partial into a
    // slot indexed by the tile, with four loads a thread where its
    // accumulator is one or two words and its registers are not capped (U
    // where four would spill).
    constexpr bool EX = Exact<T>::value;
    constexpr int TL = TileLoads<T, U>::value;
    const int64_t round_vec = (int64_t)blockDim.x * TL;
    const int rounds = dyn && a.tile_vec > round_vec ? (int)(a.tile_vec / round_vec) : 1;
    const int64_t tile = round_vec * rounds;
    const int64_t ntiles = dyn ? (nvec - nstat + tile - 1) / tile : 0;
    // one tile into accumulators ac; with its first loads thread 0 publishes
    // the next tile (claimed a tile earlier) and claims the one after (if
    // `more`: a block of a float trait stops claiming when its TileSlots
    // partial slots are full)
    auto run_tile = [&](typename T::Acc (&ac)[U], unsigned t, int k, bool more) {
        const int64_t v0 = nstat + (int64_t)t * tile + threadIdx.x;   // this thread's first vector
        const char* p0 = xv + v0 * VB;
        const int64_t left = nvec - v0;                               // vectors from v0 to the end
        const bool full = left >= tile;                               // every tile but the last
        for (int r = 0; r < rounds; r++) {
            const int64_t o = (int64_t)r * round_vec;
            Words<VB> w[TL];
#pragma unroll
            for (int q = 0; q < TL; q++)
                if (full || o + q * (int)blockDim.x < left) w[q] = ldv<VB>(p0 + (o + q * (int)blockDim.x) * VB);
            if (r == 0 && threadIdx.x == 0) {
                s_claim[(k + 1) & 1] = c_next;
                c_next = more ? atomicAdd(a.ws.chunk_ctr, 1u) : ~0u;
            }
#pragma unroll
            for (int q = 0; q < TL; q++) {
                const int64_t oq = o + q * (int)blockDim.x;
                if (full || oq < left) {
                    E e[VE];
                    Ld::template dec<VB>(w[q], e);
                    T::add_vec(ac[q % U], e, head + (v0 + oq) * VE);
                }
            }
        }
    };
    if constexpr (TAIL && EX) {
        if (dyn) {
            __syncthreads();   // the first claims, in shared memory
            unsigned t = s_claim[0];
            if (threadIdx.x == 0) c_next = s_claim1;
            for (int k = 0; (int64_t)t < ntiles; k++) {
                run_tile(acc, t, k, true);
                __syncthreads();
                t = s_claim[(k + 1) & 1];
            }
        }
    }

    const Part p = block_combine<T>(fold<T, U>(acc));

    int ktiles = 0;   // tiles this block reduced (float traits)
    if constexpr (TAIL && !EX) if (dyn) {
        // a tile's partial: each warp's value in a shared slot (no combine
        // across warps inside the loop, so no warp falls behind the others
        // between barriers); after the block's last tile, thread j combines
        // its tile j's warp values in warp order and stores them in the
        // tile's slot
        constexpr int NW = MaxBlock<T>::value / 32;
        constexpr int NS = TileSlots<T>::value;
        __shared__ Part s_tp[NS][NW];
        __shared__ unsigned s_tid[NS];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int nwarps = (blockDim.x + 31) >> 5;
        unsigned t = s_claim[0];   // written before block_combine's barriers
        if (threadIdx.x == 0) c_next = s_claim1;
        int k = 0;
        while ((int64_t)t < ntiles) {
            typename T::Acc ta[U];
#pragma unroll
            for (int u = 0; u < U; u++) ta[u] = T::init();
            run_tile(ta, t, k, k + 2 < NS);
            const Part tp = T::warp_reduce(fold<T, U>(ta));
            if (lane == 0) s_tp[k][warp] = tp;
            if (threadIdx.x == 0) s_tid[k] = t;
            __syncthreads();
            t = s_claim[(k + 1) & 1];
            k++;
        }
        if ((int)threadIdx.x < k) {
            Part q = s_tp[threadIdx.x][0];
            for (int w = 1; w < nwarps; w++) q = T::combine(q, s_tp[threadIdx.x][w]);
            *slot<GR>(a.ws.head, s_tid[threadIdx.x]) = GR::up(q);
        }
        ktiles = k;
    }

    // the result (valid in thread 0) to out, or as a Part to part_out
    auto finish = [&](const G& q) {
        if (a.part_out) {
            *static_cast<G*>(a.part_out) = q;
        } else {
            GR::store(a.out, 0, q, a.out_f64 != 0);
            GR::store_aux(a.argidx, nullptr, 0, q, 0);
        }
    };
    // one block (small inputs): its partial is the only one, so it finishes
    // at once, with the same combine the last block would make, and no
    // round trip through memory, fence or ticket
    if constexpr (!TAIL) {
        if (gridDim.x == 1) {
            G q = threadIdx.x == 0 ? GR::combine(GR::part_init(), GR::up(p)) : GR::part_init();
            q = block_combine<GR>(q);
            if (threadIdx.x == 0) finish(q);
            return;
        }
    }

    // every thread that wrote a partial (thread 0 the block's, and with a
    // claimed tail of a float trait the first threads their tiles') fences;
    // a barrier then orders those writes before thread 0's ticket
    __shared__ unsigned s_last;
    if constexpr (TAIL && !EX) {
        if (threadIdx.x == 0) *slot<GR>(a.ws.partials, blockIdx.x) = GR::up(p);
        if (threadIdx.x == 0 || (int)threadIdx.x < ktiles) __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = (atomicAdd(a.ws.counter, 1u) == gridDim.x - 1);
    } else if (threadIdx.x == 0) {
        *slot<GR>(a.ws.partials, blockIdx.x) = GR::up(p);
        __threadfence();
        const unsigned ticket = atomicAdd(a.ws.counter, 1u);
        s_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    G q = GR::part_init();
    if constexpr (TAIL && !EX) {
        // block partials, then tile partials in tile order; the tile loop is
        // unrolled so that a thread's loads of several slots travel together
        for (int j = threadIdx.x; j < (int)gridDim.x; j += blockDim.x)
            q = GR::combine(q, ld_cg_any(slot<GR>(a.ws.partials, j)));
        const int nt = (int)ntiles;
        int j = threadIdx.x;
        for (; j + 3 * (int)blockDim.x < nt; j += 4 * blockDim.x) {
            G v[4];
#pragma unroll
            for (int r = 0; r < 4; r++) v[r] = ld_cg_any(slot<GR>(a.ws.head, j + r * (int)blockDim.x));
#pragma unroll
            for (int r = 0; r < 4; r++) q = GR::combine(q, v[r]);
        }
        for (; j < nt; j += blockDim.x) q = GR::combine(q, ld_cg_any(slot<GR>(a.ws.head, j)));
    } else {
        for (int j = threadIdx.x; j < (int)gridDim.x; j += blockDim.x)
            q = GR::combine(q, ld_cg_any(slot<GR>(a.ws.partials, j)));
    }
    q = block_combine<GR>(q);
    if (threadIdx.x == 0) {
        finish(q);
        *a.ws.counter = 0u;
        if constexpr (TAIL)
            if (dyn) *a.ws.chunk_ctr = 0u;
    }
}

// The plain reduction's kernel.  A trait that declares kMinBlocks gets the
// two-argument launch bound (a register cap); the others keep the one-argument
// bound, with which the compiler chooses their registers freely (an explicit
// minimum of one block makes it take more, and so halves some traits'
// occupancy).
// TAIL: the variant with claimed tail tiles (large inputs; its tile loads
// take registers the grid-stride kernel does not need).
template <class T, int U, int VB, bool TAIL>
__global__ void __launch_bounds__(MaxBlock<T>::value) k_reduce(ReduceArgs a) {
    reduce_body<T, U, VB, TAIL>(a);
}
template <class T, int U, int VB, bool TAIL>
__global__ void __launch_bounds__(MaxBlock<T>::value, MinBlocks<T>::value) k_reduce_occ(ReduceArgs a) {
    reduce_body<T, U, VB, TAIL>(a);
}
template <class T, int U, int VB, bool TAIL = false>
constexpr auto reduce_kernel() {
    if constexpr (MinBlocks<T>::value > 1) return &k_reduce_occ<T, U, VB, TAIL>;
    else return &k_reduce<T, U, VB, TAIL>;
}

// One block: out = parts[0] (x) parts[1] (x) ... in index order (slot stride kSlot).
template <class T>
__global__ void __launch_bounds__(256) k_combine_parts(const char* parts, int count, void* out, int out_f64) {
    using GR = GridR<T>;
    using G = typename GR::Part;
    G q = GR::part_init();
    for (int j = threadIdx.x; j < count; j += blockDim.x)
        q = GR::combine(q, *reinterpret_cast<const G*>(parts + (int64_t)j * kSlot));
    q = block_combine<GR>(q);
    if (threadIdx.x == 0) GR::store(out, 0, q, out_f64 != 0);
}

// ------------------------------------------------------------------------
// Row reduction
// ------------------------------------------------------------------------

template <class T, int U, int VB>
__global__ void __launch_bounds__(MaxBlock<T>::value) k_rows(RowArgs a) {
    using Ld = typename T::Ld;
    using E = typename Ld::E;
    using Acc = typename T::Acc;
    using Part = typename T::Part;
    using GR = GridR<T>;
    using G = typename GR::Part;
    constexpr int VE = VB / Ld::ES;
    const char* xv = static_cast<const char*>(a.x);
    const bool f64 = a.out_f64 != 0;
    const int B = blockDim.x;
    const int64_t cv = a.cols / VE;                 // vectors per row
    const int64_t nv = a.rows * cv;                 // vectors in all
    const int64_t TILE = (int64_t)B * U;            // vectors per tile
    const int64_t ntile = (nv + TILE - 1) / TILE;
    const int64_t R = (ntile + gridDim.x - 1) / gridDim.x * TILE;  // vectors per block run
    const int64_t vlo = (int64_t)blockIdx.x * R < nv ? (int64_t)blockIdx.x * R : nv;
    const int64_t vhi = vlo + R < nv ? vlo + R : nv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    (void)lane;
    (void)warp;
    __shared__ int s_fin;

    Words<VB> pre[U];   // this thread's first U vectors of the next row piece
    bool have = false;
    for (int64_t v = vlo; v < vhi;) {
        const int64_t r = v / cv;
        const int64_t pend = (r + 1) * cv < vhi ? (r + 1) * cv : vhi;
        Acc acc[U];
#pragma unroll
        for (int u = 0; u < U; u++) acc[u] = T::init();
        int64_t i = v + threadIdx.x;
        if (have) {
#pragma unroll
            for (int u = 0; u < U; u++) {
                E e[VE];
                Ld::template dec<VB>(pre[u], e);
                T::add_vec(acc[u], e, (i + (int64_t)u * B) * VE);
            }
            i += TILE;
        }
        for (; i + (int64_t)(U - 1) * B < pend; i += TILE) {
            Words<VB> w[U];
#pragma unroll
            for (int u = 0; u < U; u++) w[u] = ldv<VB>(xv + (i + (int64_t)u * B) * VB);
#pragma unroll
            for (int u = 0; u < U; u++) {
                E e[VE];
                Ld::template dec<VB>(w[u], e);
                T::add_vec(acc[u], e, (i + (int64_t)u * B) * VE);
            }
        }
        for (; i < pend; i += B) {
            const Words<VB> w = ldv<VB>(xv + i * VB);
            E e[VE];
            Ld::template dec<VB>(w, e);
            T::add_vec(acc[0], e, i * VE);
        }
        // load the next piece's first vectors now, so that they arrive during the combine
        have = false;
        if (pend < vhi) {
            const int64_t nend = pend + cv < vhi ? pend + cv : vhi;
            const int64_t j = pend + threadIdx.x;
            if (j + (int64_t)(U - 1) * B < nend) {
#pragma unroll
                for (int u = 0; u < U; u++) pre[u] = ldv<VB>(xv + (j + (int64_t)u * B) * VB);
                have = true;
            }
        }
        // finish this block's piece of row r
        const Part p = block_combine<T>(fold<T, U>(acc));
        const int64_t sb = r * a.cols;
        const int64_t ba = (r * cv) / R, bb = ((r + 1) * cv - 1) / R;
        if (ba == bb) {
            if (threadIdx.x == 0) {
                const G g = GR::up(p);
                GR::store(a.out, r, g, f64);
                GR::store_aux(a.argidx, a.aux, r, g, sb);
            }
        } else {
            if (threadIdx.x == 0) {
                *slot<GR>(v > r * cv ? a.ws.head : a.ws.tail, blockIdx.x) = GR::up(p);
                __threadfence();
                const unsigned old = atomicAdd(a.ws.seg_cnt + ba, 1u);
                s_fin = (old == (unsigned)(bb - ba));
            }
            __syncthreads();
            if (s_fin) {
                __threadfence();
                G q = GR::part_init();
                for (int64_t k = threadIdx.x; k <= bb - ba; k += B)
                    q = GR::combine(q, ld_cg_any(k == 0 ? slot<GR>(a.ws.tail, ba) : slot<GR>(a.ws.head, ba + k)));
                q = block_combine<GR>(q);
                if (threadIdx.x == 0) {
                    GR::store(a.out, r, q, f64);
                    GR::store_aux(a.argidx, a.aux, r, q, sb);
                    a.ws.seg_cnt[ba] = 0u;
                }
            }
        }
        v = pend;
    }
}

// ------------------------------------------------------------------------
// Segmented reduction
// ------------------------------------------------------------------------

struct Segs {
    const int64_t* off;
    int64_t cols, nseg, P0, P1;
    __device__ __forceinline__ int64_t raw(int64_t s) const { return off ? __ldg(off + s) : s * cols; }
    // segment bounds clamped to [P0, P1]: malformed offsets cannot move a read
    // outside the range the caller vouches for
    __device__ __forceinline__ int64_t begin(int64_t s) const {
        const int64_t b = raw(s);
        return b < P0 ? P0 : (b > P1 ? P1 : b);
    }
    __device__ __forceinline__ int64_t end(int64_t s) const { return begin(s + 1); }
    // Largest s in [lo, nseg) with begin(s) <= p (requires begin(lo) <= p),
    // found by one warp (all 32 lanes call; every lane gets the answer).
    // begin() is non-decreasing, so {s : begin(s) <= p} is a prefix of
    // [lo, nseg): one coalesced probe of the next 32 segments settles the
    // common case (the answer is near lo), else a 32-ary search narrows the
    // interval 32-fold per round.
    __device__ int64_t find(int64_t lo, int64_t p, int lane) const {
        if (!off) {
            int64_t s = p / cols;
            s = s < lo ? lo : s;
            return s > nseg - 1 ? nseg - 1 : s;
        }
        int64_t hi = nseg - 1;
        {
            const int64_t q = lo + 1 + lane;
            const unsigned m = __ballot_sync(0xffffffffu, q <= hi && begin(q) <= p);
            if (m != 0xffffffffu) return lo + __popc(m);
            lo += 32;
        }
        while (lo < hi) {
            const int64_t step = (hi - lo + 32) / 32;
            const int64_t q = lo + (int64_t)lane * step;
            const unsigned m = __ballot_sync(0xffffffffu, q <= hi && begin(q) <= p);
            const int last = 31 - __clz(m);
            lo = lo + (int64_t)last * step;
            hi = lo + step - 1 < hi ? lo + step - 1 : hi;
        }
        return lo;
    }
};

template <class T, int U, int VB>
struct SegCtx {
    using Ld = typename T::Ld;
    using In = typename Ld::In;
    using E = typename Ld::E;
    static constexpr int VE = VB / Ld::ES;
    const In* x;
    Segs sg;
    int64_t P0, P1;

    // Accumulate the elements with position in [lo, hi) among the U vectors
    // this thread owns in the tile starting at position tlo.
    __device__ __forceinline__ void masked(typename T::Acc (&acc)[U], int64_t tlo, int64_t lo, int64_t hi) const {
        if (lo >= hi) return;
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int64_t vp = tlo + ((int64_t)u * blockDim.x + threadIdx.x) * VE;
            if (vp + VE <= lo || vp >= hi) continue;
            if (vp >= P0 && vp + VE <= P1) {
                const Words<VB> w = ldv<VB>(x + vp);
                E e[VE];
                Ld::template dec<VB>(w, e);
#pragma unroll
                for (int k = 0; k < VE; k++)
                    if (vp + k >= lo && vp + k < hi) T::add(acc[u], e[k], vp + k);
            } else {
                const int64_t a0 = vp > lo ? vp : lo;
                const int64_t a1 = vp + VE < hi ? vp + VE : hi;
                for (int64_t p = a0; p < a1; p++) T::add(acc[u], Ld::one(x, p), p);
            }
        }
    }
};

// Same as SegCtx::masked, from vectors already loaded for an interior tile.
template <class T, int U, int VB>
__device__ __forceinline__ void masked_words(typename T::Acc (&acc)[U], const Words<VB> (&w)[U], int64_t tlo,
                                             int64_t lo, int64_t hi) {
    using Ld = typename T::Ld;
    using E = typename Ld::E;
    constexpr int VE = VB / Ld::ES;
    if (lo >= hi) return;
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int64_t vp = tlo + ((int64_t)u * blockDim.x + threadIdx.x) * VE;
        if (vp + VE <= lo || vp >= hi) continue;
        E e[VE];
        Ld::template dec<VB>(w[u], e);
#pragma unroll
        for (int k = 0; k < VE; k++)
            if (vp + k >= lo && vp + k < hi) T::add(acc[u], e[k], vp + k);
    }
}

template <class T, int U, int VB>
__global__ void __launch_bounds__(512) k_segmented(SegArgs a) {
    using Ld = typename T::Ld;
    using In = typename Ld::In;
    using E = typename Ld::E;
    using Acc = typename T::Acc;
    using Part = typename T::Part;
    constexpr int VE = VB / Ld::ES;
    const In* x = static_cast<const In*>(a.x);
    const int64_t nseg = a.nseg;
    const bool f64 = a.out_f64 != 0;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    if (nseg <= 0) return;

    Segs sg{a.off, a.cols, nseg, 0, 0};
    const int64_t raw0 = sg.raw(0), rawN = sg.raw(nseg);
    const int64_t P0 = raw0 < 0 ? 0 : raw0;
    const int64_t P1 = rawN < P0 ? P0 : rawN;
    sg.P0 = P0;
    sg.P1 = P1;

    // Empty segments get the identity; malformed offsets raise the error word.
    for (int64_t s = gtid; s < nseg; s += nth) {
        const int64_t rb = sg.raw(s), re = sg.raw(s + 1);
        if (rb > re || rb < 0) atomicOr(a.ws.err, kErrInvalid);
        if (sg.begin(s) == sg.end(s)) T::store_empty(a.out, s, f64, a.argidx, a.aux);
    }
    if (P1 <= P0) return;

    const int B = blockDim.x;
    const int64_t TILE = (int64_t)B * VE * U;
    const int64_t shift = a.shift;
    const int64_t J0 = ((P0 + shift) / VE) * VE;  // first VB boundary at or before P0
    const int64_t ntiles = (P1 + shift - J0 + TILE - 1) / TILE;
    // chunks: a few per block, at most one slot pair per chunk
    int64_t nchunk = (int64_t)a.chunks_per_block * gridDim.x;
    nchunk = nchunk < a.ws.gmax ? nchunk : a.ws.gmax;
    nchunk = nchunk < ntiles ? nchunk : ntiles;
    const int64_t K = (ntiles + nchunk - 1) / nchunk;  // tiles per chunk
    nchunk = (ntiles + K - 1) / K;                      // chunks that hold tiles
    const int64_t CB = K * TILE;

    SegCtx<T, U, VB> ctx{x, sg, P0, P1};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = B >> 5;

    __shared__ int64_t s_i64;
    __shared__ int s_fin;
    __shared__ unsigned s_chunk;
    using GR = GridR<T>;
    using G = typename GR::Part;

    for (int64_t iter = 0;; iter++) {
        int64_t c;
        if (a.dynamic_chunks) {
            __syncthreads();  // s_chunk / s_i64 of the previous chunk are consumed
            if (threadIdx.x == 0) s_chunk = atomicAdd(a.ws.chunk_ctr, 1u);
            __syncthreads();
            c = s_chunk;
        } else {
            c = blockIdx.x + iter * gridDim.x;
        }
        if (c >= nchunk) break;
        const int64_t t0 = c * K;
        const int64_t t1 = t0 + K < ntiles ? t0 + K : ntiles;
        const int64_t blk_lo = (J0 + t0 * TILE - shift) > P0 ? (J0 + t0 * TILE - shift) : P0;
        const int64_t blk_hi = (J0 + t1 * TILE - shift) < P1 ? (J0 + t1 * TILE - shift) : P1;

        // Finish this chunk's piece of segment s (all threads call).
        auto emit = [&](int64_t s, Acc (&acc)[U]) {
            const Part p = block_combine<T>(fold<T, U>(acc));
#pragma unroll
            for (int u = 0; u < U; u++) acc[u] = T::init();
            const int64_t sb = sg.begin(s), se = sg.end(s);
            if (sb >= blk_lo && se <= blk_hi) {
                if (threadIdx.x == 0) {
                    const G g = GR::up(p);
                    GR::store(a.out, s, g, f64);
                    GR::store_aux(a.argidx, a.aux, s, g, sb);
                }
                return;
            }
            const int64_t ba = (sb + shift - J0) / CB, bb = (se - 1 + shift - J0) / CB;
            if (threadIdx.x == 0) {
                *slot<GR>(sb < blk_lo ? a.ws.head : a.ws.tail, c) = GR::up(p);
                __threadfence();
                const unsigned old = atomicAdd(a.ws.seg_cnt + ba, 1u);
                s_fin = (old == (unsigned)(bb - ba));
            }
            __syncthreads();
            if (s_fin) {
                // the whole block combines the segment's chunk partials (a
                // segment can span every chunk of the launch)
                __threadfence();
                G q = GR::part_init();
                for (int64_t k = threadIdx.x; k <= bb - ba; k += B)
                    q = GR::combine(q, ld_cg_any(k == 0 ? slot<GR>(a.ws.tail, ba) : slot<GR>(a.ws.head, ba + k)));
                q = block_combine<GR>(q);
                if (threadIdx.x == 0) {
                    GR::store(a.out, s, q, f64);
                    GR::store_aux(a.argidx, a.aux, s, q, sb);
                    a.ws.seg_cnt[ba] = 0u;
                }
            }
            __syncthreads();
        };

        // Tiles lying wholly inside [P0, P1) are "interior": their vectors are
        // loaded one tile ahead, so loads stay in flight through the block
        // combines at segment boundaries (and through the search below).
        auto interior = [&](int64_t t) {
            const int64_t l = J0 + t * TILE - shift;
            return l >= P0 && l + TILE <= P1;
        };
        auto load_tile = [&](int64_t t, Words<VB> (&w)[U]) {
            const int64_t l = J0 + t * TILE - shift;
#pragma unroll
            for (int u = 0; u < U; u++) w[u] = ldv<VB>(x + l + ((int64_t)u * B + threadIdx.x) * VE);
        };
        Words<VB> wn[U];
        bool have = t0 < t1 && interior(t0);
        if (have) load_tile(t0, wn);

        if (warp == 0) {
            const int64_t r = sg.find(0, blk_lo, lane);
            if (lane == 0) s_i64 = r;
        }
        __syncthreads();
        int64_t cs = s_i64;
        int64_t cend = sg.end(cs);

        Acc acc[U];
#pragma unroll
        for (int u = 0; u < U; u++) acc[u] = T::init();

        for (int64_t t = t0; t < t1; t++) {
            const int64_t tlo = J0 + t * TILE - shift, thi = tlo + TILE;
            Words<VB> w[U];
#pragma unroll
            for (int u = 0; u < U; u++) w[u] = wn[u];
            const bool cur = have;
            have = t + 1 < t1 && interior(t + 1);
            if (have) load_tile(t + 1, wn);
            if (cur && cend >= thi) {
                // the whole tile lies inside segment cs: stream it
#pragma unroll
                for (int u = 0; u < U; u++) {
                    E e[VE];
                    Ld::template dec<VB>(w[u], e);
                    T::add_vec(acc[u], e, tlo + ((int64_t)u * B + threadIdx.x) * VE);
                }
                continue;
            }
            // accumulate positions [p0, p1) of this tile into ac
            auto part = [&](Acc (&ac)[U], int64_t p0, int64_t p1) {
                if (cur) masked_words<T, U, VB>(ac, w, tlo, p0, p1);
                else ctx.masked(ac, tlo, p0, p1);
            };
            const int64_t lo = tlo > P0 ? tlo : P0, hi = thi < P1 ? thi : P1;
            if (cend >= hi) {
                part(acc, lo, hi);
                continue;
            }
            // segment cs ends inside this tile
            part(acc, lo, cend);
            emit(cs, acc);
            __syncthreads();
            if (warp == 0) {
                const int64_t r = sg.find(cs + 1, hi - 1, lane);
                if (lane == 0) s_i64 = r;
            }
            __syncthreads();
            const int64_t ns = s_i64;
            // segments lying wholly inside the tile: short ones one per warp ...
            for (int64_t s = cs + 1 + warp; s < ns; s += nwarps) {
                const int64_t sb = sg.begin(s), se = sg.end(s);
                if (se == sb || se - sb > kSmallSeg) continue;
                Acc wa = T::init();
                int64_t p = sb + lane;
                for (; p + 96 < se; p += 128) {
                    const E v0 = Ld::one(x, p), v1 = Ld::one(x, p + 32), v2 = Ld::one(x, p + 64), v3 = Ld::one(x, p + 96);
                    T::add(wa, v0, p);
                    T::add(wa, v1, p + 32);
                    T::add(wa, v2, p + 64);
                    T::add(wa, v3, p + 96);
                }
                for (; p < se; p += 32) T::add(wa, Ld::one(x, p), p);
                const Part q = T::warp_reduce(T::to_part(wa));
                if (lane == 0) {
                    const G g = GR::up(q);
                    GR::store(a.out, s, g, f64);
                    GR::store_aux(a.argidx, a.aux, s, g, sb);
                }
            }
            // ... long ones with the whole block
            for (int64_t s = cs + 1; s < ns; s++) {
                const int64_t sb = sg.begin(s), se = sg.end(s);
                if (se - sb <= kSmallSeg) continue;
                Acc ba_[U];
#pragma unroll
                for (int u = 0; u < U; u++) ba_[u] = T::init();
                part(ba_, sb, se);
                const Part q = block_combine<T>(fold<T, U>(ba_));
                if (threadIdx.x == 0) {
                    const G g = GR::up(q);
                    GR::store(a.out, s, g, f64);
                    GR::store_aux(a.argidx, a.aux, s, g, sb);
                }
            }
            cs = ns;
            cend = sg.end(cs);
            part(acc, sg.begin(ns), hi);
        }
        emit(cs, acc);
    }
    // the last block out re-arms the chunk counter for the next launch
    if (a.dynamic_chunks && threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(a.ws.blk_done, 1u) == gridDim.x - 1) {
            *a.ws.chunk_ctr = 0u;
            *a.ws.blk_done = 0u;
        }
    }
}

}  // namespace pr
