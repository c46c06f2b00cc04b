// Prefix scan y_i = x_0 (x) ... (x) x_i (inclusive) or x_0 (x) ... (x) x_{i-1}
// (exclusive) of x[0..n) in one pass, for the combiners whose result is exact
// (integer and bitwise combiners, float max / min): the prefix counterpart of
// the reduction (Section 1.1), whose consumers the paper names (stream
// compaction, counting and radix sort).
//
// k_scan  persistent blocks claim tiles in order from an atomic counter, so a
// block only ever waits for tiles that running blocks hold.  Per tile: each
// thread scans its 64 bytes of input, the block scans the thread totals
// (shuffles, then one value per warp), the block publishes the tile's
// aggregate, and warp 0 looks back over the preceding tiles, 32 at a time:
// tiles that already know their inclusive prefix end the walk, the others
// contribute their aggregates (decoupled look-back).  The tile then publishes
// its inclusive prefix and writes its outputs.  The combiners are exact,
// associative and commutative, so the result does not depend on how far a
// look-back walked.
//
// Status words carry an epoch (bumped by the last block of every launch), so
// no reset pass runs between launches and graph replays see fresh flags.
// Every wait is bounded: a wait that runs out sets kErrTimeout in the error
// word (read by pr_last_device_error) and the tile goes on with what it has.
#include <cstring>
#include <type_traits>
#include "kernels.cuh"
#include "registry.h"
#include "scan.cuh"

namespace pr {

constexpr int kScanSpin = 1 << 18;      // polls of one flag before giving up (each >= 64 ns)
constexpr int kScanWin = 2;             // look-back step: kScanWin x 32 tiles

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
// them, read and written by 128-bit atomics (also one round trip).
template <bool PACKED>
struct TileStatus;

template <>
struct TileStatus<true> {
    __device__ __forceinline__ static unsigned long long* word(ScanTile* t) {
        return reinterpret_cast<unsigned long long*>(&t->flag);
    }
    // low half: the flag in the same format as the two-word layout ((epoch <<
    // 2) | state), so that neither layout mistakes the other's stale words for
    // current ones; high half: the value
    __device__ __forceinline__ static void publish(ScanTile* t, unsigned long long v, unsigned epoch, unsigned state) {
        st_relaxed_u64(word(t), ((v & 0xffffffffull) << 32) | (unsigned long long)((epoch << 2) | state));
    }
    __device__ __forceinline__ static bool valid(unsigned long long w, unsigned epoch) {
        const unsigned f = (unsigned)w;
        return (f >> 2) == epoch && (f & 3u) != 0u;
    }
    // W tiles at once: the first loads all go out together; only tiles not
    // yet published are polled again (bounded)
    template <int W>
    __device__ __forceinline__ static void read(ScanTile* const (&t)[W], const bool (&use)[W], unsigned epoch, int* err,
                                                unsigned (&st)[W], unsigned long long (&v)[W], int spin = kScanSpin) {
        unsigned long long w[W];
#pragma unroll
        for (int m = 0; m < W; m++) w[m] = use[m] ? ld_relaxed_u64(word(t[m])) : 0ull;
#pragma unroll
        for (int m = 0; m < W; m++) {
            st[m] = 2u;
            v[m] = 0ull;
            if (!use[m]) continue;
            int it = 0;
            while (!valid(w[m], epoch) && it < spin) {
                if (it >= 16) __nanosleep(64);
                w[m] = ld_relaxed_u64(word(t[m]));
                it++;
            }
            if (!valid(w[m], epoch)) atomicOr(err, kErrTimeout);
            else st[m] = (unsigned)w[m] & 3u;
            v[m] = w[m] >> 32;
        }
    }
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
    // low word: the flag ((epoch << 2) | state, as in the other layout); high word: the value
    __device__ __forceinline__ static void publish(ScanTile* t, unsigned long long v, unsigned epoch, unsigned state) {
        exch128(t, (unsigned long long)((epoch << 2) | state), v);
    }
    __device__ __forceinline__ static bool valid(unsigned long long lo, unsigned epoch) {
        const unsigned f = (unsigned)lo;
        return (f >> 2) == epoch && (f & 3u) != 0u;
    }
    template <int W>
    __device__ __forceinline__ static void read(ScanTile* const (&t)[W], const bool (&use)[W], unsigned epoch, int* err,
                                                unsigned (&st)[W], unsigned long long (&v)[W], int spin = kScanSpin) {
        unsigned long long lo[W], hi[W];
#pragma unroll
        for (int m = 0; m < W; m++) {
            lo[m] = 0ull;
            hi[m] = 0ull;
            if (use[m]) read128(t[m], lo[m], hi[m]);
        }
#pragma unroll
        for (int m = 0; m < W; m++) {
            st[m] = 2u;
            v[m] = 0ull;
            if (!use[m]) continue;
            int it = 0;
            while (!valid(lo[m], epoch) && it < spin) {
                if (it >= 16) __nanosleep(64);
                read128(t[m], lo[m], hi[m]);
                it++;
            }
            if (!valid(lo[m], epoch)) atomicOr(err, kErrTimeout);
            else st[m] = (unsigned)lo[m] & 3u;
            v[m] = hi[m];
        }
    }
};


template <class Op>
__device__ __forceinline__ typename Op::A warp_all(typename Op::A v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v = Op::comb(v, shfl_xor_any(v, m));
    return v;
}

// VEC: x and y aligned so that each thread's 64 input bytes and its outputs
// move as whole 16-byte words.
template <class Op, bool VEC>
__global__ void __launch_bounds__(kScanThreads) k_scan(ScanArgs a) {
    using In = typename Op::In;
    using A = typename Op::A;
    using Out = typename Op::Out;
    constexpr int IT = kScanBytes / (int)sizeof(In);          // elements per thread
    constexpr int64_t TILE = (int64_t)kScanThreads * IT;
    constexpr int NW = kScanThreads / 32;
    const In* x = static_cast<const In*>(a.x);
    Out* y = static_cast<Out*>(a.y);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    using Status = TileStatus<(sizeof(A) <= 4)>;

    __shared__ int64_t s_tile;
    __shared__ unsigned s_epoch;
    __shared__ A s_warp[NW];
    __shared__ A s_prefix;
    if (threadIdx.x == 0) s_epoch = ld_acquire_u32(a.ctr + 2) & 0x3fffffffu;

    for (;;) {
        __syncthreads();   // shared values of the previous tile are consumed
        if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(a.ctr, 1u);
        __syncthreads();
        const int64_t t = s_tile;
        const unsigned epoch = s_epoch;
        if (t >= a.ntiles) break;
        const int64_t e0 = t * TILE + (int64_t)threadIdx.x * IT;   // this thread's first element
        const bool full = e0 + IT <= a.n;

        // 1. load and scan this thread's elements
        A r[IT];
        if (VEC && full) {
            uint32_t w[kScanBytes / 4];
#pragma unroll
            for (int q = 0; q < kScanBytes / 32; q++) {
                const Words<32> v = ldv<32>(x + e0 + q * (32 / (int)sizeof(In)));
                memcpy(w + q * 8, v.w, 32);
            }
            In e[IT];
            memcpy(e, w, kScanBytes);
#pragma unroll
            for (int k = 0; k < IT; k++) r[k] = Op::conv(e[k]);
        } else {
#pragma unroll
            for (int k = 0; k < IT; k++) r[k] = e0 + k < a.n ? Op::conv(x[e0 + k]) : Op::ident();
        }
#pragma unroll
        for (int k = 1; k < IT; k++) r[k] = Op::comb(r[k - 1], r[k]);

        // 2. block scan of the thread totals
        A inc = r[IT - 1];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const A o = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc = Op::comb(o, inc);
        }
        if (lane == 31) s_warp[warp] = inc;
        __syncthreads();
        A wpre = Op::ident(), agg = Op::ident();
#pragma unroll
        for (int w = 0; w < NW; w++) {
            if (w < warp) wpre = Op::comb(wpre, s_warp[w]);
            agg = Op::comb(agg, s_warp[w]);
        }
        A texcl = __shfl_up_sync(0xffffffffu, inc, 1);
        texcl = lane == 0 ? wpre : Op::comb(wpre, texcl);   // everything before this thread in the tile

        // 3. publish the aggregate, look back, publish the inclusive prefix
        if (warp == 0) {
            A pre = Op::ident();
            if (t == 0) {
                if (lane == 0) Status::publish(a.tiles, Op::pack(agg), epoch, 2u);
            } else {
                if (lane == 0) Status::publish(a.tiles + t, Op::pack(agg), epoch, 1u);
                // windows of kScanWin x 32 predecessors: lane k reads tiles
                // base - k - 32 m; sub-windows are taken nearest first
                for (int64_t base = t - 1;; base -= 32 * kScanWin) {
                    ScanTile* tp[kScanWin];
                    bool use[kScanWin];
#pragma unroll
                    for (int m = 0; m < kScanWin; m++) {
                        const int64_t j = base - lane - 32 * m;
                        use[m] = j >= 0;
                        tp[m] = a.tiles + (j >= 0 ? j : 0);
                    }
                    unsigned st[kScanWin];
                    unsigned long long vb[kScanWin];
                    Status::template read<kScanWin>(tp, use, epoch, a.err, st, vb);
                    bool found = false;
#pragma unroll
                    for (int m = 0; m < kScanWin; m++) {
                        if (found) break;
                        const A v = use[m] ? Op::unpack(vb[m]) : Op::ident();
                        const unsigned incl = __ballot_sync(0xffffffffu, st[m] == 2u);
                        const int stop = incl ? __ffs(incl) - 1 : 31;
                        pre = Op::comb(pre, warp_all<Op>(lane <= stop ? v : Op::ident()));
                        found = incl != 0u;
                    }
                    if (found) break;
                }
                if (lane == 0) Status::publish(a.tiles + t, Op::pack(Op::comb(pre, agg)), epoch, 2u);
            }
            if (lane == 0) s_prefix = pre;
        }
        __syncthreads();
        const A base = Op::comb(s_prefix, texcl);

        // 4. outputs
        Out o[IT];
#pragma unroll
        for (int k = 0; k < IT; k++) {
            const A v = a.exclusive ? (k == 0 ? base : Op::comb(base, r[k - 1])) : Op::comb(base, r[k]);
            o[k] = Op::out(v);
        }
        if (VEC && full) {
            constexpr int OB = IT * (int)sizeof(Out);
            uint32_t w[OB / 4];
            memcpy(w, o, OB);
            char* dst = reinterpret_cast<char*>(y + e0);
#pragma unroll
            for (int q = 0; q < OB / 16; q++)
                asm volatile("st.global.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(dst + q * 16), "r"(w[4 * q]),
                             "r"(w[4 * q + 1]), "r"(w[4 * q + 2]), "r"(w[4 * q + 3]) : "memory");
        } else {
#pragma unroll
            for (int k = 0; k < IT; k++)
                if (e0 + k < a.n) y[e0 + k] = o[k];
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

// Self-check of the bounded wait: one thread waits, with `spin` polls, on a
// tile state that nothing publishes; the wait must give up and set
// kErrTimeout in the error word.
__global__ void k_wait_probe(ScanTile* t, int spin, int* err) {
    if (threadIdx.x != 0) return;
    ScanTile* tp[1] = {t};
    const bool use[1] = {true};
    unsigned st[1];
    unsigned long long v[1];
    TileStatus<true>::read<1>(tp, use, 1u, err, st, v, spin);
    TileStatus<false>::read<1>(tp, use, 1u, err, st, v, spin);
}

cudaError_t launch_wait_probe(ScanTile* t, int spin, int* err, cudaStream_t st) {
    k_wait_probe<<<1, 32, 0, st>>>(t, spin, err);
    return cudaGetLastError();
}

template <class Op, bool VEC>
cudaError_t launch_scan(const ScanArgs& a, int grid, int block, cudaStream_t st) {
    k_scan<Op, VEC><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

// Keyed by (dtype, op, vector flag in the vb field).
template <class Op>
static void reg_scan(uint8_t dtype, uint8_t op) {
    reg_add(KernelKey{K_SCAN, dtype, op, 0, 0, 0, 0},
            KernelEntry{reinterpret_cast<const void*>(&k_scan<Op, false>), reinterpret_cast<void*>(&launch_scan<Op, false>)});
    reg_add(KernelKey{K_SCAN, dtype, op, 0, 0, 0, 1},
            KernelEntry{reinterpret_cast<const void*>(&k_scan<Op, true>), reinterpret_cast<void*>(&launch_scan<Op, true>)});
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
