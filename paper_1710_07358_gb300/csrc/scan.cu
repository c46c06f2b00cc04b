// Prefix scan y_i = x_0 (x) ... (x) x_i (inclusive) or x_0 (x) ... (x) x_{i-1}
// (exclusive) of x[0..n) in one pass, for the combiners whose result is exact
// (integer and bitwise combiners, float max / min): the prefix counterpart of
// the reduction (Section 1.1), whose consumers the paper names (stream
// compaction, counting and radix sort).
//
// k_scan  persistent blocks, one per SM, claim 32 KB tiles in order from an
// atomic counter, so a block only ever waits for tiles that running blocks
// hold.  Inside a block the warps have roles (see the kernel): a producer
// thread stages claimed tiles of an aligned input in a ring of kScanStages
// shared-memory buffers by bulk copies; reduce warps publish each tile's
// aggregate as soon as its bytes land; look-back warps walk back over the
// preceding tiles, 32 at a time: tiles that already know their inclusive
// prefix end the walk, the others contribute their aggregates (decoupled
// look-back), and the tile publishes its inclusive prefix; scan warps then
// scan the tile out of shared memory with that prefix, store it, and free
// the stage.  A tile's aggregate never waits for a look-back, so no
// look-back waits behind another one.  The combiners are exact, associative
// and commutative, so the result does not depend on how far a look-back
// walked or in which order a tile's elements were combined.
//
// Status words carry an epoch (bumped by the last block of every launch), so
// no reset pass runs between launches and graph replays see fresh flags.
// Every wait is bounded: a wait that runs out sets kErrTimeout in the error
// word (read by pr_last_device_error) and the block winds down (every role
// leaves its loop; the copies it started are waited for, bounded).
#include <cstring>
#include <type_traits>
#include "kernels.cuh"
#include "registry.h"
#include "bulk.cuh"
#include "scan.cuh"

namespace pr {

constexpr int kScanSpin = 1 << 18;      // polls of a tile state before giving up (each >= 64 ns)
constexpr unsigned long long kScanWaitNs = 250000000ull;   // longest wait on a shared-memory barrier

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---- combiners -----------------------------------------------------------

// Integer combiners on In, accumulating in A (int64 for an int32 sum), with
// two's-complement wrap-around for sums and products.
template <class In_, class A_, int OP>
struct ScanInt {
    using In = In_;
    using A = A_;
    using Out = A_;
    using U = std::make_unsigned_t<A_>;
    __device__ __forceinline__ static A conv(In v) { return (A)v; }
    __device__ __forceinline__ static A ident() {
        if (OP == PR_SUM || OP == PR_OR || OP == PR_XOR) return (A)0;
        if (OP == PR_PROD) return (A)1;
        if (OP == PR_AND) return (A)~(U)0;
        if (OP == PR_MAX) return std::is_signed<A>::value ? (A)((U)1 << (sizeof(A) * 8 - 1)) : (A)0;
        return std::is_signed<A>::value ? (A)(~(U)0 >> 1) : (A)~(U)0;
    }
    __device__ __forceinline__ static A comb(A a, A b) {
        if (OP == PR_SUM) return (A)((U)a + (U)b);
        if (OP == PR_PROD) return (A)((U)a * (U)b);
        if (OP == PR_MAX) return a > b ? a : b;
        if (OP == PR_MIN) return a < b ? a : b;
        if (OP == PR_AND) return a & b;
        if (OP == PR_OR) return a | b;
        return a ^ b;
    }
    __device__ __forceinline__ static unsigned long long pack(A v) { return (unsigned long long)(U)v; }
    __device__ __forceinline__ static A unpack(unsigned long long b) { return (A)(U)b; }
    __device__ __forceinline__ static Out out(A v) { return v; }
};

// Float max / min of f32 (and bf16 / f16 widened to f32): max.NaN / min.NaN,
// which propagate NaN and order -0 below +0, and the result is one of the
// inputs, so narrowing it back to the input type is exact.
template <class Ld_, int OutK, bool MX>
struct ScanMaxF {
    using Ld = Ld_;
    using In = typename Ld_::In;
    using A = float;
    using Out = std::conditional_t<OutK == 0, float, uint16_t>;
    __device__ __forceinline__ static A conv(In v) {
        if constexpr (OutK == 0) return v;
        else if constexpr (OutK == 1) return __uint_as_float((uint32_t)v << 16);
        else return __half2float(__ushort_as_half(v));
    }
    __device__ __forceinline__ static A ident() { return MX ? -INFINITY : INFINITY; }
    __device__ __forceinline__ static A comb(A a, A b) {
        float r;
        if (MX) asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
        else asm("min.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
        return r;
    }
    __device__ __forceinline__ static unsigned long long pack(A v) { return __float_as_uint(v); }
    __device__ __forceinline__ static A unpack(unsigned long long b) { return __uint_as_float((uint32_t)b); }
    __device__ __forceinline__ static Out out(A v) {
        if constexpr (OutK == 0) return v;
        else if constexpr (OutK == 1) return isnan(v) ? (uint16_t)0x7fc0 : (uint16_t)(__float_as_uint(v) >> 16);
        else return __half_as_ushort(__float2half_rn(v));
    }
};

// fp64 max / min by order-preserving keys (NaN the extreme, -0 < +0).
template <bool MX>
struct ScanMaxD {
    using In = double;
    using A = double;
    using Out = double;
    __device__ __forceinline__ static uint64_t key(double v) {
        const uint64_t b = (uint64_t)__double_as_longlong(v);
        const uint64_t k = b ^ ((uint64_t)((int64_t)b >> 63) | 0x8000000000000000ull);
        const bool nan = (b & 0x7fffffffffffffffull) > 0x7ff0000000000000ull;
        return nan ? (MX ? ~0ull : 0ull) : k;
    }
    __device__ __forceinline__ static A conv(In v) { return v; }
    __device__ __forceinline__ static A ident() { return MX ? -INFINITY : INFINITY; }
    __device__ __forceinline__ static A comb(A a, A b) {
        const uint64_t ka = key(a), kb = key(b);
        return (MX ? kb > ka : kb < ka) ? b : a;
    }
    __device__ __forceinline__ static unsigned long long pack(A v) { return (unsigned long long)__double_as_longlong(v); }
    __device__ __forceinline__ static A unpack(unsigned long long b) { return __longlong_as_double((long long)b); }
    __device__ __forceinline__ static Out out(A v) { return v; }
};

// ---- kernel --------------------------------------------------------------

// Tile status as the look-back sees it (state 1 aggregate, 2 inclusive).
// Accumulators of at most 32 bits share one 64-bit word with the epoch and
// the state, so one load reads a consistent (state, value) pair: a look-back
// step costs one L2 round trip.  Wider accumulators share a 16-byte word with
// them, read and written by 128-bit atomics (also one round trip).  A reader
// issues load() for many tiles at once and settle()s each word only when it
// needs it: settle polls a word that is not yet published (bounded).
template <bool PACKED>
struct TileStatus;

template <>
struct TileStatus<true> {
    struct Raw {
        unsigned long long w;
    };
    __device__ __forceinline__ static unsigned long long* word(ScanTile* t) {
        return reinterpret_cast<unsigned long long*>(&t->flag);
    }
    // low half: the flag in the same format as the two-word layout ((epoch <<
    // 2) | state), so that neither layout mistakes the other's stale words for
    // current ones; high half: the value
    __device__ __forceinline__ static void publish(ScanTile* t, unsigned long long v, unsigned epoch, unsigned state) {
        st_relaxed_u64(word(t), ((v & 0xffffffffull) << 32) | (unsigned long long)((epoch << 2) | state));
    }
    __device__ __forceinline__ static bool valid(const Raw& r, unsigned epoch) {
        const unsigned f = (unsigned)r.w;
        return (f >> 2) == epoch && (f & 3u) != 0u;
    }
    __device__ __forceinline__ static Raw load(ScanTile* t) { return Raw{ld_relaxed_u64(word(t))}; }
    __device__ __forceinline__ static unsigned state(const Raw& r) { return (unsigned)r.w & 3u; }
    __device__ __forceinline__ static unsigned long long value(const Raw& r) { return r.w >> 32; }
};

// 64-bit accumulators: flag and value in one 16-byte word, written and read
// with 128-bit atomics (exchange; compare-and-swap with a comparand that a
// published word never equals, which returns the word unchanged), so a step
// is still one round trip.
__device__ __forceinline__ void exch128(ScanTile* t, unsigned long long lo, unsigned long long hi) {
    asm volatile("{\n\t.reg .b128 d, b;\n\t"
                 "mov.b128 b, {%0, %1};\n\t"
                 "atom.relaxed.gpu.global.exch.b128 d, [%2], b;\n\t}"
                 :: "l"(lo), "l"(hi), "l"(&t->flag) : "memory");
}
__device__ __forceinline__ void read128(ScanTile* t, unsigned long long& lo, unsigned long long& hi) {
    asm volatile("{\n\t.reg .b128 d, z;\n\t"
                 "mov.b128 z, {%2, %2};\n\t"
                 "atom.relaxed.gpu.global.cas.b128 d, [%3], z, z;\n\t"
                 "mov.b128 {%0, %1}, d;\n\t}"
                 : "=l"(lo), "=l"(hi) : "l"(0ull), "l"(&t->flag) : "memory");
}

template <>
struct TileStatus<false> {
    struct Raw {
        unsigned long long lo, hi;
    };
    // low word: the flag ((epoch << 2) | state, as in the other layout); high word: the value
    __device__ __forceinline__ static void publish(ScanTile* t, unsigned long long v, unsigned epoch, unsigned state) {
        exch128(t, (unsigned long long)((epoch << 2) | state), v);
    }
    __device__ __forceinline__ static bool valid(const Raw& r, unsigned epoch) {
        const unsigned f = (unsigned)r.lo;
        return (f >> 2) == epoch && (f & 3u) != 0u;
    }
    __device__ __forceinline__ static Raw load(ScanTile* t) {
        Raw r;
        read128(t, r.lo, r.hi);
        return r;
    }
    __device__ __forceinline__ static unsigned state(const Raw& r) { return (unsigned)r.lo & 3u; }
    __device__ __forceinline__ static unsigned long long value(const Raw& r) { return r.hi; }
};

// Poll tile t's word until it is published in this epoch, at most `spin`
// times; false (and kErrTimeout in the error word) if it never was.
template <class Status>
__device__ __forceinline__ bool settle(ScanTile* t, typename Status::Raw& r, unsigned epoch, int* err, int spin) {
    for (int it = 0; !Status::valid(r, epoch); it++) {
        if (it >= spin) {
            atomicOr(err, kErrTimeout);
            return false;
        }
        if (it >= 16) __nanosleep(64);
        r = Status::load(t);
    }
    return true;
}

template <class Op>
__device__ __forceinline__ typename Op::A warp_all(typename Op::A v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v = Op::comb(v, shfl_xor_any(v, m));
    return v;
}

// The look-back of tile t > 0 (one warp): the words of the W x 32 nearest
// predecessors not yet seen are loaded at once, lane k reading tiles
// base - k - 32 m; windows m are settled and taken nearest first, and the
// walk ends at the first window holding an inclusive prefix, without waiting
// for the farther ones.  Returns the combination of everything before tile t.
template <class Op, class Status, int W>
__device__ __forceinline__ typename Op::A look_back(const ScanArgs& a, int64_t t, unsigned epoch, int lane, int spin,
                                                    bool& timed_out) {
    using A = typename Op::A;
    A pre = Op::ident();
    for (int64_t base = t - 1;; base -= 32 * W) {
        typename Status::Raw raw[W];
#pragma unroll
        for (int m = 0; m < W; m++) {
            const int64_t j = base - lane - 32 * m;
            if (j >= 0) raw[m] = Status::load(a.tiles + j);
        }
#pragma unroll
        for (int m = 0; m < W; m++) {
            const int64_t j = base - lane - 32 * m;
            unsigned st = 2u;                      // before tile 0: the identity, inclusive
            A v = Op::ident();
            if (j >= 0) {
                if (settle<Status>(a.tiles + j, raw[m], epoch, a.err, spin)) {
                    st = Status::state(raw[m]);
                    v = Op::unpack(Status::value(raw[m]));
                } else {
                    timed_out = true;
                }
            }
            const unsigned incl = __ballot_sync(0xffffffffu, st == 2u);
            const int stop = incl ? __ffs(incl) - 1 : 31;
            pre = Op::comb(pre, warp_all<Op>(lane <= stop ? v : Op::ident()));
            if (incl) return pre;
        }
    }
}

__device__ __forceinline__ void bar_sync_named(int id, int threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}
// named barrier that also ORs a predicate over its threads (the same result in all)
__device__ __forceinline__ bool bar_any_named(int id, int threads, bool v) {
    unsigned r;
    asm volatile("{\n\t.reg .pred p, q;\n\t"
                 "setp.ne.u32 q, %1, 0;\n\t"
                 "bar.red.or.pred p, %2, %3, q;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(r) : "r"((unsigned)v), "r"(id), "r"(threads) : "memory");
    return r != 0u;
}

// Warp roles and ring depth of one scan block.
template <int S_, int NL_, int NR_, int NC_, int W_, int TB_ = kScanTileBytes, int B_ = 1, int G_ = 4>
struct ScanShape {
    static constexpr int G = G_;     // chunks a scan warp scans together
    static constexpr int TB = TB_;   // tile bytes (input)
    static constexpr int B = B_;     // most tiles claimed by one atomic
    static constexpr int S = S_;     // shared-memory stages of TB bytes
    static constexpr int NL = NL_;   // look-back warps (tile j: warp j mod NL)
    static constexpr int NR = NR_;   // reduction warps
    static constexpr int NC = NC_;   // scan-and-store warps
    static constexpr int W = W_;     // look-back step: W x 32 tiles
    static constexpr int kThreads = 32 * (1 + NL + NR + NC);
};

// VEC: x and y 16-byte aligned, so whole tiles are staged by bulk copies and
// outputs leave as 16-byte words; other tiles (the ragged last one, or every
// tile of an unaligned input) are read from x directly.
//
// A tile is 64 chunks of 512 bytes; lane l holds the E elements of bytes
// [16 l, 16 l + 16) of a chunk, so shared-memory reads are conflict-free and
// every warp store covers 512 contiguous input bytes.  Warp roles, each
// walking the block's tiles j = 0, 1, ... through stage j mod S:
//   warp 0, lane 0   claims a tile for a free stage and starts its copy
//                    (full[s]: the bytes have landed);
//   NR reduce warps  combine the tile's chunks into one total per scan warp's
//                    slice and publish the tile aggregate (red[s]);
//   NL look-back     look back over the preceding tiles and publish the
//   warps            tile's inclusive prefix (pre[s]);
//   NC scan warps    scan their slice with the prefix, store it, and release
//                    the stage (empty[s]).
// A claimed tile's aggregate therefore depends only on its own copy, never
// on a look-back, so no look-back waits on another one, and the copies of
// the next S - 1 tiles stay in flight while a tile is looked back and stored.
template <class Op, bool VEC, class Sh>
__global__ void __launch_bounds__(Sh::kThreads, 1) k_scan(ScanArgs a) {
    using In = typename Op::In;
    using A = typename Op::A;
    using Out = typename Op::Out;
    constexpr int S = Sh::S, NL = Sh::NL, NR = Sh::NR, NC = Sh::NC, TB = Sh::TB;
    constexpr int E = 16 / (int)sizeof(In);                 // elements per lane and chunk
    constexpr int CH = TB / 512;                 // chunks per tile
    constexpr int CC = CH / NC;                              // chunks per scan slice
    constexpr int SR = NC / NR;                              // scan slices per reduce warp
    constexpr int CE = 32 * E;                               // elements per chunk
    constexpr int64_t TILE = TB / (int)sizeof(In);
    constexpr int OB = E * (int)sizeof(Out);                 // output bytes per lane and chunk
    constexpr int G = CC < Sh::G ? CC : Sh::G;               // chunks scanned together
    static_assert(OB == 16 || OB == 32, "outputs leave as one or two 16-byte words");
    static_assert(CH % NC == 0 && NC % NR == 0 && NL <= S && CC % G == 0 && TB % 64 == 0, "slices split evenly");

    extern __shared__ __align__(128) unsigned char s_buf[];
    __shared__ __align__(8) unsigned long long s_bar[4 * S];  // full, red, pre, empty
    __shared__ int64_t s_tile[S];
    __shared__ A s_part[S][NC];
    __shared__ A s_agg[S];
    __shared__ A s_prefix[S];
    __shared__ int64_t s_stop;
    __shared__ int64_t s_last[S];                             // last tile copied into each stage
    __shared__ int s_abort;
    __shared__ unsigned s_epoch;

    const In* x = static_cast<const In*>(a.x);
    Out* y = static_cast<Out*>(a.y);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    using Status = TileStatus<(sizeof(A) <= 4)>;
    const uint32_t bars = smem_u32(s_bar), buf0 = smem_u32(s_buf);
    auto full = [&](int s) { return bars + 8u * (uint32_t)s; };
    auto red = [&](int s) { return bars + 8u * (uint32_t)(S + s); };
    auto pre = [&](int s) { return bars + 8u * (uint32_t)(2 * S + s); };
    auto empty = [&](int s) { return bars + 8u * (uint32_t)(3 * S + s); };
    volatile int* abort_flag = &s_abort;
    // a wait that runs out, or sees that another warp gave up, returns false
    // and the block winds down (every role leaves its loop)
    auto wait = [&](uint32_t bar, unsigned par) { return bar_wait(bar, par, kScanWaitNs, abort_flag, a.err); };
    auto staged = [&](int64_t t) { return VEC && (t + 1) * TILE <= a.n; };
    // chunk c of tile t for this lane, from stage s or from x
    auto load_chunk = [&](int s, int64_t t, bool st, int c, A (&v)[E]) {
        if (st) {
            const uint4 w = *reinterpret_cast<const uint4*>(s_buf + s * TB + c * 512 + lane * 16);
            In e[E];
            memcpy(e, &w, 16);
#pragma unroll
            for (int j = 0; j < E; j++) v[j] = Op::conv(e[j]);
        } else {
            const int64_t i0 = t * TILE + (int64_t)c * CE + lane * E;
#pragma unroll
            for (int j = 0; j < E; j++) v[j] = i0 + j < a.n ? Op::conv(x[i0 + j]) : Op::ident();
        }
    };

    if (threadIdx.x == 0) {
        s_epoch = ld_acquire_u32(a.ctr + 2) & 0x3fffffffu;
        s_stop = INT64_MAX;
        s_abort = 0;
#pragma unroll
        for (int s = 0; s < S; s++) {
            s_last[s] = -1;
            mbar_init(full(s), 1u);
            mbar_init(red(s), 1u);
            mbar_init(pre(s), 1u);
            mbar_init(empty(s), (unsigned)NC);
        }
        mbar_fence_init();
    }
    __syncthreads();
    const unsigned epoch = s_epoch;

    if (warp == 0) {
        // ---- producer: claim, copy ----
        if (lane == 0) {
            // stage j mod S is free once the scan warps released tile j - S
            auto is_free = [&](int64_t j) {
                return j < S || mbar_test_wait(empty((int)(j % S)), (unsigned)((j / S - 1) & 1));
            };
            bool done = false;
            for (int64_t j = 0; !done;) {
                if (*abort_flag || (j >= S && !wait(empty((int)(j % S)), (unsigned)((j / S - 1) & 1)))) break;
                // one claim covers every stage that is free now (at most B)
                int k = 1;
                while (k < Sh::B && is_free(j + k)) k++;
                const int64_t t0 = (int64_t)atomicAdd(a.ctr, (unsigned)k);
                for (int i = 0; i < k && !done; i++, j++) {
                    const int s = (int)(j % S);
                    const int64_t t = t0 + i;
                    s_tile[s] = t;
                    if (t < a.ntiles && staged(t)) {
                        s_last[s] = j;
                        mbar_expect_tx(full(s), (unsigned)TB);
                        const char* src = reinterpret_cast<const char*>(x) + t * TB;
#pragma unroll
                        for (int c = 0; c < 4; c++)
                            bulk_g2s(buf0 + (uint32_t)(s * TB + c * (TB / 4)), src + c * (TB / 4), (unsigned)(TB / 4),
                                     full(s));
                    } else {
                        mbar_arrive(full(s));
                    }
                    done = t >= a.ntiles;
                }
            }
        }
    } else if (warp <= NL) {
        // ---- look-back: tiles j = l, l + NL, ... ----
        for (int64_t j = warp - 1;; j += NL) {
            const int s = (int)(j % S);
            if (!__all_sync(0xffffffffu, wait(red(s), (unsigned)((j / S) & 1)))) break;
            const int64_t t = s_tile[s];
            if (j >= s_stop) break;                        // past the last tile, woken by the reducers
            if (t >= a.ntiles) {
                if (lane == 0) mbar_arrive(pre(s));
                break;
            }
            A p = Op::ident();
            if (t != 0) {
                bool late = false;
                p = look_back<Op, Status, Sh::W>(a, t, epoch, lane, *abort_flag ? 1 : kScanSpin, late);
                if (__any_sync(0xffffffffu, late)) {
                    *abort_flag = 1;
                    break;
                }
                if (lane == 0) Status::publish(a.tiles + t, Op::pack(Op::comb(p, s_agg[s])), epoch, 2u);
            }
            if (lane == 0) {
                s_prefix[s] = p;
                mbar_arrive(pre(s));
            }
        }
    } else if (warp <= NL + NR) {
        // ---- reduce: slice totals and the tile aggregate ----
        const int r = warp - 1 - NL;
        for (int64_t j = 0;; j++) {
            const int s = (int)(j % S);
            // the reduce warps leave together (they share a named barrier)
            const bool ok = wait(full(s), (unsigned)((j / S) & 1));
            if (bar_any_named(1, 32 * NR, !ok || *abort_flag)) {
                *abort_flag = 1;
                break;
            }
            const int64_t t = s_tile[s];
            if (t >= a.ntiles) {
                if (r == 0 && lane == 0) {
                    s_stop = j + 1;                         // look-back warps waiting on later tiles stop
                    for (int i = 0; i < NL; i++) mbar_arrive(red((int)((j + i) % S)));
                }
                break;
            }
            const bool st = staged(t);
#pragma unroll
            for (int q = 0; q < SR; q++) {
                A tot = Op::ident();
#pragma unroll 4
                for (int c = 0; c < CC; c++) {
                    A v[E];
                    load_chunk(s, t, st, (r * SR + q) * CC + c, v);
#pragma unroll
                    for (int i = 0; i < E; i++) tot = Op::comb(tot, v[i]);
                }
                tot = warp_all<Op>(tot);
                if (lane == 0) s_part[s][r * SR + q] = tot;
            }
            bar_sync_named(1, 32 * NR);
            if (r == 0 && lane == 0) {
                A agg = Op::ident();
#pragma unroll
                for (int c = 0; c < NC; c++) agg = Op::comb(agg, s_part[s][c]);
                s_agg[s] = agg;
                Status::publish(a.tiles + t, Op::pack(agg), epoch, t == 0 ? 2u : 1u);
                mbar_arrive(red(s));
            }
        }
    } else {
        // ---- scan and store one slice ----
        const int c0 = warp - 1 - NL - NR;
        for (int64_t j = 0;; j++) {
            const int s = (int)(j % S);
            const unsigned par = (unsigned)((j / S) & 1);
            if (!__all_sync(0xffffffffu, wait(pre(s), par))) break;
            const int64_t t = s_tile[s];
            if (t >= a.ntiles) break;
            const bool st = staged(t);
            if (st && !__all_sync(0xffffffffu, wait(full(s), par))) break;   // the copied bytes, seen by this warp
            A carry = s_prefix[s];
#pragma unroll
            for (int c = 0; c < NC; c++)
                if (c < c0) carry = Op::comb(carry, s_part[s][c]);
            // G chunks at a time: their warp scans are independent, so the
            // shuffle chains overlap; the carry then runs through them in order
            for (int c = c0 * CC; c < (c0 + 1) * CC; c += G) {
                A v[G][E], inc[G], ex[G], tot[G];
#pragma unroll
                for (int g = 0; g < G; g++) {
                    load_chunk(s, t, st, c + g, v[g]);
#pragma unroll
                    for (int i = 1; i < E; i++) v[g][i] = Op::comb(v[g][i - 1], v[g][i]);
                    inc[g] = v[g][E - 1];
                }
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
                    for (int g = 0; g < G; g++) {
                        const A o = __shfl_up_sync(0xffffffffu, inc[g], d);
                        if (lane >= d) inc[g] = Op::comb(o, inc[g]);
                    }
                }
#pragma unroll
                for (int g = 0; g < G; g++) {
                    ex[g] = __shfl_up_sync(0xffffffffu, inc[g], 1);
                    tot[g] = __shfl_sync(0xffffffffu, inc[g], 31);
                }
#pragma unroll
                for (int g = 0; g < G; g++) {
                    const A cb = lane == 0 ? carry : Op::comb(carry, ex[g]);
                    carry = Op::comb(carry, tot[g]);
                    Out o[E];
#pragma unroll
                    for (int i = 0; i < E; i++)
                        o[i] = Op::out(a.exclusive ? (i == 0 ? cb : Op::comb(cb, v[g][i - 1])) : Op::comb(cb, v[g][i]));
                    const int64_t i0 = t * TILE + (int64_t)(c + g) * CE + lane * E;
                    if (st) {
                        uint32_t w[OB / 4];
                        memcpy(w, o, OB);
                        char* dst = reinterpret_cast<char*>(y + i0);
#pragma unroll
                        for (int h = 0; h < OB / 16; h++)
                            asm volatile("st.global.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(dst + 16 * h), "r"(w[4 * h]),
                                         "r"(w[4 * h + 1]), "r"(w[4 * h + 2]), "r"(w[4 * h + 3]) : "memory");
                    } else {
#pragma unroll
                        for (int i = 0; i < E; i++)
                            if (i0 + i < a.n) y[i0 + i] = o[i];
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty(s));
        }
    }

    __syncthreads();
    // a block that gave up waits (bounded) for the copies it started, so none
    // lands in shared memory after the block has left
    if (threadIdx.x == 0 && s_abort) {
        for (int s = 0; s < S; s++) {
            if (s_last[s] < 0) continue;
            const uint32_t bar = full(s);
            const unsigned par = (unsigned)((s_last[s] / S) & 1);
            const unsigned long long t0 = global_ns();
            while (!mbar_try_wait(bar, par) && global_ns() - t0 < kScanWaitNs) {
            }
        }
    }
    // the last block out re-arms the tile counter and moves to the next epoch
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(a.ctr + 1, 1u) == gridDim.x - 1) {
            a.ctr[0] = 0u;
            a.ctr[1] = 0u;
            unsigned ne = (s_epoch + 1u) & 0x3fffffffu;
            st_release_u32(a.ctr + 2, ne == 0u ? 1u : ne);
        }
    }
}

// Self-check of the bounded waits: one thread waits, with `spin` polls, on a
// tile state that nothing publishes (both layouts), and for spin
// microseconds on a shared-memory barrier phase that nothing completes; each
// wait must give up and set kErrTimeout in the error word.
__global__ void k_wait_probe(ScanTile* t, int spin, int* err) {
    __shared__ __align__(8) unsigned long long s_b;
    __shared__ int s_give_up;
    if (threadIdx.x != 0) return;
    TileStatus<true>::Raw r1 = TileStatus<true>::load(t);
    settle<TileStatus<true>>(t, r1, 1u, err, spin);
    TileStatus<false>::Raw r2 = TileStatus<false>::load(t);
    settle<TileStatus<false>>(t, r2, 1u, err, spin);
    s_give_up = 0;
    const uint32_t bar = smem_u32(&s_b);
    mbar_init(bar, 1u);
    mbar_fence_init();
    bar_wait(bar, 0u, 1000ull * (unsigned long long)spin, &s_give_up, err);
}

cudaError_t launch_wait_probe(ScanTile* t, int spin, int* err, cudaStream_t st) {
    k_wait_probe<<<1, 32, 0, st>>>(t, spin, err);
    return cudaGetLastError();
}

using ScanMain = ScanShape<kScanStages, kScanLookWarps, kScanRedWarps, kScanScanWarps, kScanLookWin>;
static_assert(ScanMain::kThreads == kScanThreads, "block size of the scan");

template <class Op, bool VEC>
cudaError_t launch_scan(const ScanArgs& a, int grid, int block, size_t smem, cudaStream_t st) {
    k_scan<Op, VEC, ScanMain><<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

// Keyed by (dtype, op, vector flag in the vb field).
template <class Op>
static void reg_scan(uint8_t dtype, uint8_t op) {
    reg_add(KernelKey{K_SCAN, dtype, op, 0, 0, 0, 0},
            KernelEntry{reinterpret_cast<const void*>(&k_scan<Op, false, ScanMain>),
                        reinterpret_cast<void*>(&launch_scan<Op, false>)});
    reg_add(KernelKey{K_SCAN, dtype, op, 0, 0, 0, 1},
            KernelEntry{reinterpret_cast<const void*>(&k_scan<Op, true, ScanMain>),
                        reinterpret_cast<void*>(&launch_scan<Op, true>)});
}

template <class In, class ASum, class A>
static void reg_scan_int(uint8_t dtype) {
    reg_scan<ScanInt<In, ASum, PR_SUM>>(dtype, PR_SUM);
    reg_scan<ScanInt<In, A, PR_PROD>>(dtype, PR_PROD);
    reg_scan<ScanInt<In, A, PR_MAX>>(dtype, PR_MAX);
    reg_scan<ScanInt<In, A, PR_MIN>>(dtype, PR_MIN);
    reg_scan<ScanInt<In, A, PR_AND>>(dtype, PR_AND);
    reg_scan<ScanInt<In, A, PR_OR>>(dtype, PR_OR);
    reg_scan<ScanInt<In, A, PR_XOR>>(dtype, PR_XOR);
}

void register_scan() {
    reg_scan_int<int32_t, int64_t, int32_t>(PR_I32);
    reg_scan_int<uint32_t, uint32_t, uint32_t>(PR_U32);
    reg_scan_int<int64_t, int64_t, int64_t>(PR_I64);
    reg_scan<ScanMaxF<LdF32, 0, true>>(PR_F32, PR_MAX);
    reg_scan<ScanMaxF<LdF32, 0, false>>(PR_F32, PR_MIN);
    reg_scan<ScanMaxF<LdBF16, 1, true>>(PR_BF16, PR_MAX);
    reg_scan<ScanMaxF<LdBF16, 1, false>>(PR_BF16, PR_MIN);
    reg_scan<ScanMaxF<LdF16, 2, true>>(PR_F16, PR_MAX);
    reg_scan<ScanMaxF<LdF16, 2, false>>(PR_F16, PR_MIN);
    reg_scan<ScanMaxD<true>>(PR_F64, PR_MAX);
    reg_scan<ScanMaxD<false>>(PR_F64, PR_MIN);
}

}  // namespace pr
