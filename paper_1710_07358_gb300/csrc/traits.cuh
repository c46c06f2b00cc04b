// Combiner traits.  A trait describes one (element type, combiner, precision)
// of the reduction x_0 (x) ... (x) x_{n-1} (Section 1.1):
//
//   Ld        element loader: storage type In, compute type E, vector decode
//   Acc       per-thread accumulator (the "private variable" of Section 2.3)
//   Part      value exchanged between threads and blocks
//   init / add / add_vec    identity and accumulation of elements
//   to_part / part_init / combine   the associative (and, bit for bit,
//             commutative) combine used by the warp, block and grid stages
//   warp_reduce               butterfly shuffle or redux.sync
//   store / store_aux         final result (and argidx / product aux)
//
// Every combine is commutative bit for bit, so the butterfly leaves the same
// value in every lane; all association orders are fixed by the launch
// configuration, which makes results run-to-run deterministic.
#pragma once
#include <cstdint>
#include <cuda_fp16.h>
#include "common.cuh"
#include "../../include/pr.h"

namespace pr {

// ------------------------------------------------------------------------
// Element loaders
// ------------------------------------------------------------------------

struct LdF32 {
    using In = float;
    using E = float;
    static constexpr int ES = 4;
    template <int VB>
    __device__ __forceinline__ static void dec(const Words<VB>& w, E (&e)[VB / ES]) {
#pragma unroll
        for (int k = 0; k < VB / 4; k++) e[k] = __uint_as_float(w.w[k]);
    }
    __device__ __forceinline__ static E one(const In* x, int64_t i) { return __ldg(x + i); }
};

// bfloat16 is the high half of a binary32: widening is a shift.
struct LdBF16 {
    using In = uint16_t;
    using E = float;
    static constexpr int ES = 2;
    template <int VB>
    __device__ __forceinline__ static void dec(const Words<VB>& w, E (&e)[VB / ES]) {
#pragma unroll
        for (int k = 0; k < VB / 4; k++) {
            e[2 * k] = __uint_as_float(w.w[k] << 16);
            e[2 * k + 1] = __uint_as_float(w.w[k] & 0xffff0000u);
        }
    }
    __device__ __forceinline__ static E one(const In* x, int64_t i) {
        return __uint_as_float((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(x) + i) << 16);
    }
};

struct LdF16 {
    using In = uint16_t;
    using E = float;
    static constexpr int ES = 2;
    template <int VB>
    __device__ __forceinline__ static void dec(const Words<VB>& w, E (&e)[VB / ES]) {
#pragma unroll
        for (int k = 0; k < VB / 4; k++) {
            __half2 h;
            memcpy(&h, &w.w[k], 4);
            float2 f = __half22float2(h);
            e[2 * k] = f.x;
            e[2 * k + 1] = f.y;
        }
    }
    __device__ __forceinline__ static E one(const In* x, int64_t i) {
        return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(x) + i)));
    }
};

struct LdF64 {
    using In = double;
    using E = double;
    static constexpr int ES = 8;
    template <int VB>
    __device__ __forceinline__ static void dec(const Words<VB>& w, E (&e)[VB / ES]) {
#pragma unroll
        for (int k = 0; k < VB / 8; k++) e[k] = __hiloint2double((int)w.w[2 * k + 1], (int)w.w[2 * k]);
    }
    __device__ __forceinline__ static E one(const In* x, int64_t i) { return __ldg(x + i); }
};

struct LdI32 {
    using In = int32_t;
    using E = int32_t;
    static constexpr int ES = 4;
    template <int VB>
    __device__ __forceinline__ static void dec(const Words<VB>& w, E (&e)[VB / ES]) {
#pragma unroll
        for (int k = 0; k < VB / 4; k++) e[k] = (int32_t)w.w[k];
    }
    __device__ __forceinline__ static E one(const In* x, int64_t i) { return __ldg(x + i); }
};

struct LdU32 {
    using In = uint32_t;
    using E = uint32_t;
    static constexpr int ES = 4;
    template <int VB>
    __device__ __forceinline__ static void dec(const Words<VB>& w, E (&e)[VB / ES]) {
#pragma unroll
        for (int k = 0; k < VB / 4; k++) e[k] = w.w[k];
    }
    __device__ __forceinline__ static E one(const In* x, int64_t i) { return __ldg(x + i); }
};

// int64 is handled as uint64 bit patterns (two's-complement wrap-around).
struct LdI64 {
    using In = int64_t;
    using E = uint64_t;
    static constexpr int ES = 8;
    template <int VB>
    __device__ __forceinline__ static void dec(const Words<VB>& w, E (&e)[VB / ES]) {
#pragma unroll
        for (int k = 0; k < VB / 8; k++) e[k] = ((uint64_t)w.w[2 * k + 1] << 32) | w.w[2 * k];
    }
    __device__ __forceinline__ static E one(const In* x, int64_t i) {
        return (uint64_t)__ldg(reinterpret_cast<const long long*>(x) + i);
    }
};

// Output writers for float-valued results.
__device__ __forceinline__ void put_f32(void* out, int64_t i, float v) { static_cast<float*>(out)[i] = v; }
__device__ __forceinline__ void put_f64(void* out, int64_t i, double v) { static_cast<double*>(out)[i] = v; }

// ------------------------------------------------------------------------
// SUM
// ------------------------------------------------------------------------

// Float sum with an fp32 per-thread accumulator; PartT = float (PLAIN) or
// double (FP64_COMBINE: cross-thread / cross-block combine in fp64).
template <class Ld_, class PartT>
struct SumF {
    using Ld = Ld_;
    using E = typename Ld::E;
    using Acc = float;
    using Part = PartT;
    static constexpr bool kIdx = false;
    __device__ __forceinline__ static Acc init() { return 0.f; }
    template <int K>
    __device__ __forceinline__ static void add_vec(Acc& a, const E (&e)[K], int64_t) {
        float t[K];
#pragma unroll
        for (int k = 0; k < K; k++) t[k] = e[k];
#pragma unroll
        for (int s = 1; s < K; s <<= 1)
#pragma unroll
            for (int k = 0; k + s < K; k += 2 * s) t[k] = t[k] + t[k + s];
        a = a + t[0];
    }
    __device__ __forceinline__ static void add(Acc& a, E v, int64_t) { a = a + v; }
    __device__ __forceinline__ static Part to_part(const Acc& a) { return (Part)a; }
    __device__ __forceinline__ static Part part_init() { return (Part)0; }
    __device__ __forceinline__ static Part combine(const Part& a, const Part& b) { return a + b; }
    __device__ __forceinline__ static Part warp_reduce(Part p) { return warp_combine<SumF>(p); }
    __device__ __forceinline__ static void store(void* out, int64_t i, const Part& p, bool f64) {
        if (f64) put_f64(out, i, (double)p); else put_f32(out, i, (float)p);
    }
    __device__ __forceinline__ static void store_aux(int64_t*, pr_prod_aux*, int64_t, const Part&, int64_t) {}
    __device__ __forceinline__ static void store_empty(void* out, int64_t i, bool f64, int64_t*, pr_prod_aux*) {
        store(out, i, part_init(), f64);
    }
};

// Compensated sum (Section 1.1, second footnote: Kahan-style compensation).
// Per thread: kLanes independent fp32 (sum, compensation) pairs, element k of
// a vector going to lane k mod kLanes (independent dependency chains), each
// element added with TwoSum.  16-bit inputs (twice the elements per byte
// of fp32) take two lanes and a launch bound that keeps six 256-thread
// blocks resident per SM (at most 42 registers a thread): the eight
// operations an element costs are then hidden by more warps rather than by
// more chains per warp (measured on GB300, 2^28 bf16: four lanes at 40
// resident warps 94.9 us, two lanes at 48 warps 88.6 us; fp32, where four
// lanes measured faster, keeps them: 157 vs 160 us).  Lanes, threads, warps
// and blocks combine as fp32 pairs with Neumaier's algorithm, and the final
// s + c is formed in fp64 and rounded once to the output type.  fp64 stays
// off the path: GB300 issues fp64 adds at ~0.5e12/s, and each fp64 operation
// of the finishing block's dependent chain cost ~0.5 us there (an fp64
// Neumaier tree over 760 block partials took 7 us after the last block's
// loop, plain fp64 adds 2.5 us, the fp32 pairs less: 157.5 -> 155.8 us at
// 2^28).  The pairs also keep more bits than one fp64 sum of the block
// partials did (the ill-conditioned set of 2^26: error 5.7e-6 before, 0 now).
template <class Ld_>
struct SumComp {
    using Ld = Ld_;
    using E = typename Ld::E;
    static constexpr bool kHalf = Ld::ES == 2;
    static constexpr int kLanes = kHalf ? 2 : 4;
    struct Acc { float s[kLanes], c[kLanes]; };
    struct Part { float s, c; };
    static constexpr bool kIdx = false;
    static constexpr int kMaxBlock = kHalf ? 256 : 1024;
    static constexpr int kMinBlocks = kHalf ? 6 : 1;
    __device__ __forceinline__ static Acc init() {
        Acc a;
#pragma unroll
        for (int l = 0; l < kLanes; l++) { a.s[l] = 0.f; a.c[l] = 0.f; }
        return a;
    }
    // Per element: s + v with its exact rounding error (Knuth's TwoSum, six
    // adds and no compare -- the same compensation as Neumaier's branch, but
    // on the FMA pipe instead of the ALU pipe, which the compare and selects
    // saturated for 16-bit inputs), the error accumulated in c.
    __device__ __forceinline__ static void two_sum_acc(float& s, float& c, float v) {
        const float t = s + v;
        const float bp = t - s;
        const float ap = t - bp;
        c = c + ((s - ap) + (v - bp));
        s = t;
    }
    __device__ __forceinline__ static void add(Acc& a, E v, int64_t) { two_sum_acc(a.s[0], a.c[0], v); }
    template <int K>
    __device__ __forceinline__ static void add_vec(Acc& a, const E (&e)[K], int64_t) {
#pragma unroll
        for (int k = 0; k < K; k++) two_sum_acc(a.s[k % kLanes], a.c[k % kLanes], e[k]);
    }
    __device__ __forceinline__ static Part part_init() { return {0.f, 0.f}; }
    __device__ __forceinline__ static Part combine(const Part& a, const Part& b) {
        const float t = a.s + b.s;
        const float e = fabsf(a.s) >= fabsf(b.s) ? (a.s - t) + b.s : (b.s - t) + a.s;
        return {t, (a.c + b.c) + e};
    }
    __device__ __forceinline__ static Part to_part(const Acc& a) {
        Part p{a.s[0], a.c[0]};
#pragma unroll
        for (int l = 1; l < kLanes; l++) p = combine(p, Part{a.s[l], a.c[l]});
        return p;
    }
    __device__ __forceinline__ static Part warp_reduce(Part p) { return warp_combine<SumComp>(p); }
    // The final value: s + c in fp64 (its rounding, 2^-53 relative, is far
    // below the final one), rounded once to the output type.
    __device__ __forceinline__ static void store(void* out, int64_t i, const Part& p, bool f64) {
        const double v = value(p);
        if (f64) put_f64(out, i, v); else put_f32(out, i, (float)v);
    }
    __device__ __forceinline__ static void store_aux(int64_t*, pr_prod_aux*, int64_t, const Part&, int64_t) {}
    __device__ __forceinline__ static void store_empty(void* out, int64_t i, bool f64, int64_t*, pr_prod_aux*) {
        store(out, i, part_init(), f64);
    }
    // Once an infinity enters, s stays +-inf or NaN and the compensation turns
    // NaN; the value is then s itself.
    __device__ __forceinline__ static double value(const Part& p) {
        return isfinite(p.s) ? (double)p.s + (double)p.c : (double)p.s;
    }
};

// fp64 input, fp64 sum.
struct SumF64 {
    using Ld = LdF64;
    using E = double;
    using Acc = double;
    using Part = double;
    static constexpr bool kIdx = false;
    __device__ __forceinline__ static Acc init() { return 0.0; }
    template <int K>
    __device__ __forceinline__ static void add_vec(Acc& a, const E (&e)[K], int64_t) {
        double t[K];
#pragma unroll
        for (int k = 0; k < K; k++) t[k] = e[k];
#pragma unroll
        for (int s = 1; s < K; s <<= 1)
#pragma unroll
            for (int k = 0; k + s < K; k += 2 * s) t[k] = t[k] + t[k + s];
        a = a + t[0];
    }
    __device__ __forceinline__ static void add(Acc& a, E v, int64_t) { a = a + v; }
    __device__ __forceinline__ static Part to_part(const Acc& a) { return a; }
    __device__ __forceinline__ static Part part_init() { return 0.0; }
    __device__ __forceinline__ static Part combine(const Part& a, const Part& b) { return a + b; }
    __device__ __forceinline__ static Part warp_reduce(Part p) { return warp_combine<SumF64>(p); }
    __device__ __forceinline__ static void store(void* out, int64_t i, const Part& p, bool) { put_f64(out, i, p); }
    __device__ __forceinline__ static void store_aux(int64_t*, pr_prod_aux*, int64_t, const Part&, int64_t) {}
    __device__ __forceinline__ static void store_empty(void* out, int64_t i, bool f64, int64_t*, pr_prod_aux*) {
        store(out, i, 0.0, f64);
    }
};

// ------------------------------------------------------------------------
// Integer and bitwise combiners (exact).  OpK: 0 sum, 1 prod, 4 and, 5 or, 6 xor
// ------------------------------------------------------------------------

template <class Ld_, class AccT, int OpK>
struct IntOp {
    using Ld = Ld_;
    using E = typename Ld::E;
    using Acc = AccT;   // uint32_t, or uint64_t (int32 sum widened, int64)
    using Part = AccT;
    static constexpr bool kIdx = false;
    static constexpr bool kExact = true;   // combine exact and order free
    __device__ __forceinline__ static AccT ident() {
        return OpK == 1 ? (AccT)1 : (OpK == 4 ? (AccT)~(AccT)0 : (AccT)0);
    }
    __device__ __forceinline__ static AccT widen(E v) {
        // int32 sum: sign-extend into the 64-bit accumulator
        if (sizeof(AccT) == 8 && sizeof(E) == 4) return (AccT)(int64_t)(int32_t)v;
        return (AccT)v;
    }
    __device__ __forceinline__ static AccT op(AccT a, AccT b) {
        switch (OpK) {
        case 0: return a + b;
        case 1: return a * b;
        case 4: return a & b;
        case 5: return a | b;
        default: return a ^ b;
        }
    }
    __device__ __forceinline__ static Acc init() { return ident(); }
    template <int K>
    __device__ __forceinline__ static void add_vec(Acc& a, const E (&e)[K], int64_t) {
        AccT t[K];
#pragma unroll
        for (int k = 0; k < K; k++) t[k] = widen(e[k]);
#pragma unroll
        for (int s = 1; s < K; s <<= 1)
#pragma unroll
            for (int k = 0; k + s < K; k += 2 * s) t[k] = op(t[k], t[k + s]);
        a = op(a, t[0]);
    }
    __device__ __forceinline__ static void add(Acc& a, E v, int64_t) { a = op(a, widen(v)); }
    __device__ __forceinline__ static Part to_part(const Acc& a) { return a; }
    __device__ __forceinline__ static Part part_init() { return ident(); }
    __device__ __forceinline__ static Part combine(const Part& a, const Part& b) { return op(a, b); }
    __device__ __forceinline__ static Part warp_reduce(Part p) {
        if constexpr (sizeof(AccT) == 4 && OpK != 1) {
            // redux.sync: one instruction for 32-bit add / and / or / xor
            if (OpK == 0) return __reduce_add_sync(0xffffffffu, p);
            if (OpK == 4) return __reduce_and_sync(0xffffffffu, p);
            if (OpK == 5) return __reduce_or_sync(0xffffffffu, p);
            return __reduce_xor_sync(0xffffffffu, p);
        } else {
            return warp_combine<IntOp>(p);
        }
    }
    __device__ __forceinline__ static void store(void* out, int64_t i, const Part& p, bool) {
        static_cast<AccT*>(out)[i] = p;
    }
    __device__ __forceinline__ static void store_aux(int64_t*, pr_prod_aux*, int64_t, const Part&, int64_t) {}
    __device__ __forceinline__ static void store_empty(void* out, int64_t i, bool f64, int64_t*, pr_prod_aux*) {
        store(out, i, ident(), f64);
    }
};

// ------------------------------------------------------------------------
// MAX / MIN through order-preserving unsigned keys
// ------------------------------------------------------------------------
//
// Each value maps to an unsigned key whose unsigned order is the value order
// (floats: -inf < ... < -0 < +0 < ... < +inf; NaN maps to the extreme key of
// the combiner, so it propagates).  The combine is then an integer max / min
// (redux.sync for 32-bit keys), exact and order independent.

// binary32-valued elements (f32, and bf16 / f16 widened exactly to f32).
// OutK: 0 -> float, 1 -> bfloat16 bits, 2 -> binary16 bits.
template <class Ld_, int OutK>
struct KeyF32 {
    using Ld = Ld_;
    using E = float;
    using K = uint32_t;
    __device__ __forceinline__ static K key(E v, bool mx) {
        const uint32_t b = __float_as_uint(v);
        const uint32_t k = b ^ ((uint32_t)((int32_t)b >> 31) | 0x80000000u);
        const bool nan = (b & 0x7fffffffu) > 0x7f800000u;
        return nan ? (mx ? 0xffffffffu : 0u) : k;
    }
    __device__ __forceinline__ static K ident(bool mx) { return mx ? 0x007fffffu : 0xff800000u; }
    __device__ __forceinline__ static void put(void* out, int64_t i, K k, bool mx) {
        const bool nan = mx ? (k == 0xffffffffu) : (k == 0u);
        const uint32_t b = nan ? 0x7fc00000u : ((k & 0x80000000u) ? (k ^ 0x80000000u) : ~k);
        if (OutK == 0) static_cast<uint32_t*>(out)[i] = b;
        else if (OutK == 1) static_cast<uint16_t*>(out)[i] = nan ? (uint16_t)0x7fc0 : (uint16_t)(b >> 16);
        else static_cast<__half*>(out)[i] = nan ? __ushort_as_half((unsigned short)0x7e00)
                                                : __float2half_rn(__uint_as_float(b));
    }
};

struct KeyF64 {
    using Ld = LdF64;
    using E = double;
    using K = uint64_t;
    __device__ __forceinline__ static K key(E v, bool mx) {
        const uint64_t b = (uint64_t)__double_as_longlong(v);
        const uint64_t k = b ^ ((uint64_t)((int64_t)b >> 63) | 0x8000000000000000ull);
        const bool nan = (b & 0x7fffffffffffffffull) > 0x7ff0000000000000ull;
        return nan ? (mx ? ~0ull : 0ull) : k;
    }
    __device__ __forceinline__ static K ident(bool mx) {
        return mx ? 0x000fffffffffffffull : 0xfff0000000000000ull;
    }
    __device__ __forceinline__ static void put(void* out, int64_t i, K k, bool mx) {
        const bool nan = mx ? (k == ~0ull) : (k == 0ull);
        const uint64_t b = nan ? 0x7ff8000000000000ull
                               : ((k & 0x8000000000000000ull) ? (k ^ 0x8000000000000000ull) : ~k);
        static_cast<uint64_t*>(out)[i] = b;
    }
};

struct KeyI32 {
    using Ld = LdI32;
    using E = int32_t;
    using K = uint32_t;
    __device__ __forceinline__ static K key(E v, bool) { return (uint32_t)v ^ 0x80000000u; }
    __device__ __forceinline__ static K ident(bool mx) { return mx ? 0u : 0xffffffffu; }
    __device__ __forceinline__ static void put(void* out, int64_t i, K k, bool) {
        static_cast<uint32_t*>(out)[i] = k ^ 0x80000000u;
    }
};

struct KeyU32 {
    using Ld = LdU32;
    using E = uint32_t;
    using K = uint32_t;
    __device__ __forceinline__ static K key(E v, bool) { return v; }
    __device__ __forceinline__ static K ident(bool mx) { return mx ? 0u : 0xffffffffu; }
    __device__ __forceinline__ static void put(void* out, int64_t i, K k, bool) { static_cast<uint32_t*>(out)[i] = k; }
};

struct KeyI64 {
    using Ld = LdI64;
    using E = uint64_t;
    using K = uint64_t;
    __device__ __forceinline__ static K key(E v, bool) { return v ^ 0x8000000000000000ull; }
    __device__ __forceinline__ static K ident(bool mx) { return mx ? 0ull : ~0ull; }
    __device__ __forceinline__ static void put(void* out, int64_t i, K k, bool) {
        static_cast<uint64_t*>(out)[i] = k ^ 0x8000000000000000ull;
    }
};

template <class Key, bool MX>
struct MaxMin {
    using Ld = typename Key::Ld;
    using E = typename Key::E;
    using K = typename Key::K;
    using Acc = K;
    using Part = K;
    static constexpr bool kIdx = false;
    static constexpr bool kExact = true;   // combine exact and order free
    __device__ __forceinline__ static K pick(K a, K b) { return MX ? (a > b ? a : b) : (a < b ? a : b); }
    __device__ __forceinline__ static Acc init() { return Key::ident(MX); }
    template <int N>
    __device__ __forceinline__ static void add_vec(Acc& a, const typename Ld::E (&e)[N], int64_t) {
        K t[N];
#pragma unroll
        for (int k = 0; k < N; k++) t[k] = Key::key((E)e[k], MX);
#pragma unroll
        for (int s = 1; s < N; s <<= 1)
#pragma unroll
            for (int k = 0; k + s < N; k += 2 * s) t[k] = pick(t[k], t[k + s]);
        a = pick(a, t[0]);
    }
    __device__ __forceinline__ static void add(Acc& a, typename Ld::E v, int64_t) { a = pick(a, Key::key((E)v, MX)); }
    __device__ __forceinline__ static Part to_part(const Acc& a) { return a; }
    __device__ __forceinline__ static Part part_init() { return Key::ident(MX); }
    __device__ __forceinline__ static Part combine(const Part& a, const Part& b) { return pick(a, b); }
    __device__ __forceinline__ static Part warp_reduce(Part p) {
        if constexpr (sizeof(K) == 4) {
            return MX ? __reduce_max_sync(0xffffffffu, p) : __reduce_min_sync(0xffffffffu, p);
        } else {
            return warp_combine<MaxMin>(p);
        }
    }
    __device__ __forceinline__ static void store(void* out, int64_t i, const Part& p, bool) { Key::put(out, i, p, MX); }
    __device__ __forceinline__ static void store_aux(int64_t*, pr_prod_aux*, int64_t, const Part&, int64_t) {}
    __device__ __forceinline__ static void store_empty(void* out, int64_t i, bool f64, int64_t*, pr_prod_aux*) {
        store(out, i, part_init(), f64);
    }
};

// binary32-valued MAX / MIN (f32; bf16 / f16 widened exactly to f32): the
// per-thread accumulation uses max.NaN / min.NaN, one instruction per element,
// which propagate NaN and order -0 below +0 in either operand order -- the
// same semantics as the order-preserving keys, to which the accumulator is
// converted for the warp / block / grid combine.
template <class Ld_, int OutK, bool MX>
struct MaxMinF {
    using Ld = Ld_;
    using E = float;
    using Key = KeyF32<Ld_, OutK>;
    using Acc = float;
    using Part = uint32_t;
    static constexpr bool kIdx = false;
    static constexpr bool kExact = true;   // combine exact and order free
    __device__ __forceinline__ static float f(float a, float b) {
        float r;
        if (MX) asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
        else asm("min.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
        return r;
    }
    __device__ __forceinline__ static Acc init() { return MX ? -INFINITY : INFINITY; }
    template <int N>
    __device__ __forceinline__ static void add_vec(Acc& a, const E (&e)[N], int64_t) {
        float t[N];
#pragma unroll
        for (int k = 0; k < N; k++) t[k] = e[k];
#pragma unroll
        for (int s = 1; s < N; s <<= 1)
#pragma unroll
            for (int k = 0; k + s < N; k += 2 * s) t[k] = f(t[k], t[k + s]);
        a = f(a, t[0]);
    }
    __device__ __forceinline__ static void add(Acc& a, E v, int64_t) { a = f(a, v); }
    __device__ __forceinline__ static Part to_part(const Acc& a) { return Key::key(a, MX); }
    __device__ __forceinline__ static Part part_init() { return Key::ident(MX); }
    __device__ __forceinline__ static Part combine(const Part& a, const Part& b) {
        return MX ? (a > b ? a : b) : (a < b ? a : b);
    }
    __device__ __forceinline__ static Part warp_reduce(Part p) {
        return MX ? __reduce_max_sync(0xffffffffu, p) : __reduce_min_sync(0xffffffffu, p);
    }
    __device__ __forceinline__ static void store(void* out, int64_t i, const Part& p, bool) { Key::put(out, i, p, MX); }
    __device__ __forceinline__ static void store_aux(int64_t*, pr_prod_aux*, int64_t, const Part&, int64_t) {}
    __device__ __forceinline__ static void store_empty(void* out, int64_t i, bool f64, int64_t*, pr_prod_aux*) {
        store(out, i, part_init(), f64);
    }
};

// Extremum plus the index of its first occurrence: ties go to the smaller
// index, so the combine is order independent and the result unique.
template <class Key, bool MX>
struct ArgExt {
    using Ld = typename Key::Ld;
    using E = typename Key::E;
    using K = typename Key::K;
    struct Acc { K key; int64_t idx; };
    using Part = Acc;
    static constexpr bool kIdx = true;
    static constexpr bool kExact = true;   // combine exact and order free
    static constexpr int64_t kNone = INT64_MAX;
    __device__ __forceinline__ static bool better(K ka, int64_t ia, K kb, int64_t ib) {
        return (MX ? ka > kb : ka < kb) || (ka == kb && ia < ib);
    }
    __device__ __forceinline__ static Acc init() { Acc a{}; a.key = Key::ident(MX); a.idx = kNone; return a; }
    __device__ __forceinline__ static void add(Acc& a, typename Ld::E v, int64_t i) {
        const K k = Key::key((E)v, MX);
        if (better(k, i, a.key, a.idx)) { a.key = k; a.idx = i; }
    }
    template <int N>
    __device__ __forceinline__ static void add_vec(Acc& a, const typename Ld::E (&e)[N], int64_t i0) {
#pragma unroll
        for (int k = 0; k < N; k++) add(a, e[k], i0 + k);
    }
    __device__ __forceinline__ static Part to_part(const Acc& a) { return a; }
    __device__ __forceinline__ static Part part_init() { return init(); }
    __device__ __forceinline__ static Part combine(const Part& a, const Part& b) {
        return better(b.key, b.idx, a.key, a.idx) ? b : a;
    }
    __device__ __forceinline__ static Part warp_reduce(Part p) { return warp_combine<ArgExt>(p); }
    __device__ __forceinline__ static void store(void* out, int64_t i, const Part& p, bool) { Key::put(out, i, p.key, MX); }
    __device__ __forceinline__ static void store_aux(int64_t* argidx, pr_prod_aux*, int64_t i, const Part& p,
                                                     int64_t seg_begin) {
        if (argidx) argidx[i] = p.idx == kNone ? -1 : p.idx - seg_begin;
    }
    __device__ __forceinline__ static void store_empty(void* out, int64_t i, bool f64, int64_t* argidx, pr_prod_aux*) {
        store(out, i, part_init(), f64);
        if (argidx) argidx[i] = -1;
    }
};

// Float extremum plus first index, for f32 (and bf16 / f16 widened to f32).
// A thread sees only a few dozen vectors per accumulator, so its running best
// changes often, and in a warp some lane almost always changes: a search of
// the vector on every change would run on nearly every vector.  Instead each
// accumulator keeps the best VECTOR so far: its elements, its first index and
// its extremum's key, updated with selects (no branch); the element index
// inside it is found once, in to_part.  A vector's extremum is max.NaN /
// min.NaN over its elements (a NaN yields the canonical NaN, whose raw key is
// already extreme for max; for min the key is shifted by one so that it wraps
// to 0).  Vectors reach add_vec in increasing index order per accumulator, so
// only a strictly better key replaces the best vector.  Scalars (head, tail and
// masked elements), which may arrive out of order, keep their own (key, index)
// best with the full comparison.  Scalars known to arrive in increasing index
// order per accumulator (add_ordered: the columns of an axis reduction) keep a
// running max.NaN / min.NaN value and take the index whenever its bits change:
// max.NaN turns -0 vs +0 and a first NaN into a change of bits, an equal later
// value into none.  Same result as ArgExt<KeyF32>.
template <class Ld_, int OutK, bool MX>
struct ArgExtF {
    using Ld = Ld_;
    using E = float;
    using Key = KeyF32<Ld_, OutK>;
    using Base = ArgExt<Key, MX>;
    using Part = typename Base::Part;
    static constexpr bool kIdx = true;
    static constexpr bool kExact = true;   // combine exact and order free
    static constexpr int kMaxN = 32 / Ld::ES;     // elements of the widest vector
    static constexpr int kMaxBlock = 512;         // the saved vectors need up to 128 registers
    struct Acc {
        float w[kMaxN];   // best vector's elements (the first n are valid)
        uint32_t kv;      // its extremum's key, shifted by one for min
        int n;
        int64_t iv;       // its first element's index (kNone: none yet)
        uint32_t ks;      // best scalar: key and index
        int64_t is;
        float sv;         // best in-order scalar: running extremum and its index
        int64_t so;
    };
    __device__ __forceinline__ static uint32_t raw_key(float v) {
        const uint32_t b = __float_as_uint(v);
        return b ^ ((uint32_t)((int32_t)b >> 31) | 0x80000000u);
    }
    __device__ __forceinline__ static Acc init() {
        Acc a;
#pragma unroll
        for (int k = 0; k < kMaxN; k++) a.w[k] = 0.f;
        a.kv = MX ? 0u : 0xffffffffu;   // below (above) every key a vector can have
        a.n = 0;
        a.iv = Base::kNone;
        a.ks = Key::ident(MX);
        a.is = Base::kNone;
        a.sv = MX ? -INFINITY : INFINITY;
        a.so = Base::kNone;
        return a;
    }
    __device__ __forceinline__ static void add(Acc& a, E v, int64_t i) {
        const uint32_t k = Key::key(v, MX);
        if (Base::better(k, i, a.ks, a.is)) { a.ks = k; a.is = i; }
    }
    __device__ __forceinline__ static void add_ordered(Acc& a, E v, int64_t i) {
        const float m = MaxMinF<Ld_, OutK, MX>::f(a.sv, v);
        const bool up = __float_as_uint(m) != __float_as_uint(a.sv) || a.so == Base::kNone;
        a.so = up ? i : a.so;
        a.sv = m;
    }
    // The same in-order step on a caller's pair of registers (running
    // extremum and its row, the pair started at the first element, so no
    // test for "none yet"): k_axis keeps the row as a 32-bit offset and
    // builds the accumulator once at the end.
    static constexpr bool kOrderedPair = true;
    __device__ __forceinline__ static float ordered_pick(float a, E v) { return MaxMinF<Ld_, OutK, MX>::f(a, v); }
    __device__ __forceinline__ static Acc from_ordered(float sv, int64_t i) {
        Acc a = init();
        a.sv = sv;
        a.so = i;
        return a;
    }
    template <int N>
    __device__ __forceinline__ static void add_vec(Acc& a, const E (&e)[N], int64_t i0) {
        static_assert(N <= kMaxN, "vector wider than the saved copy");
        float t[N];
#pragma unroll
        for (int k = 0; k < N; k++) t[k] = e[k];
#pragma unroll
        for (int s = 1; s < N; s <<= 1)
#pragma unroll
            for (int k = 0; k + s < N; k += 2 * s) t[k] = MaxMinF<Ld_, OutK, MX>::f(t[k], t[k + s]);
        const uint32_t km = MX ? raw_key(t[0]) : raw_key(t[0]) + 1u;
        const bool up = MX ? km > a.kv : km < a.kv;
        a.kv = up ? km : a.kv;
        a.iv = up ? i0 : a.iv;
#pragma unroll
        for (int k = 0; k < N; k++) a.w[k] = up ? e[k] : a.w[k];
        a.n = N;
    }
    __device__ __forceinline__ static Part to_part(const Acc& a) {
        Part p{a.ks, a.is};
        if (a.so != Base::kNone) p = Base::combine(p, Part{Key::key(a.sv, MX), a.so});
        if (a.iv != Base::kNone) {
            const uint32_t kv = MX ? a.kv : (a.kv == 0u ? 0u : a.kv - 1u);   // as Key::key
            int kk = kMaxN - 1;
#pragma unroll
            for (int k = kMaxN - 1; k >= 0; k--)
                if (k < a.n && Key::key(a.w[k], MX) == kv) kk = k;
            p = Base::combine(p, Part{kv, a.iv + kk});
        }
        return p;
    }
    __device__ __forceinline__ static Part part_init() { return Base::part_init(); }
    __device__ __forceinline__ static Part combine(const Part& a, const Part& b) { return Base::combine(a, b); }
    __device__ __forceinline__ static Part warp_reduce(Part p) { return Base::warp_reduce(p); }
    __device__ __forceinline__ static void store(void* out, int64_t i, const Part& p, bool f64) { Base::store(out, i, p, f64); }
    __device__ __forceinline__ static void store_aux(int64_t* argidx, pr_prod_aux* aux, int64_t i, const Part& p,
                                                     int64_t seg_begin) {
        Base::store_aux(argidx, aux, i, p, seg_begin);
    }
    __device__ __forceinline__ static void store_empty(void* out, int64_t i, bool f64, int64_t* argidx, pr_prod_aux* aux) {
        Base::store_empty(out, i, f64, argidx, aux);
    }
};

// ------------------------------------------------------------------------
// PROD
// ------------------------------------------------------------------------

// fp32 product (f32 input; bf16 / f16 widened to fp32).
template <class Ld_>
struct ProdF {
    using Ld = Ld_;
    using E = typename Ld::E;
    using Acc = float;
    using Part = float;
    static constexpr bool kIdx = false;
    static constexpr bool kOutF64 = false;
    __device__ __forceinline__ static Acc init() { return 1.f; }
    template <int K>
    __device__ __forceinline__ static void add_vec(Acc& a, const E (&e)[K], int64_t) {
        float t[K];
#pragma unroll
        for (int k = 0; k < K; k++) t[k] = e[k];
#pragma unroll
        for (int s = 1; s < K; s <<= 1)
#pragma unroll
            for (int k = 0; k + s < K; k += 2 * s) t[k] = t[k] * t[k + s];
        a = a * t[0];
    }
    __device__ __forceinline__ static void add(Acc& a, E v, int64_t) { a = a * v; }
    __device__ __forceinline__ static Part to_part(const Acc& a) { return a; }
    __device__ __forceinline__ static Part part_init() { return 1.f; }
    __device__ __forceinline__ static Part combine(const Part& a, const Part& b) { return a * b; }
    __device__ __forceinline__ static Part warp_reduce(Part p) { return warp_combine<ProdF>(p); }
    __device__ __forceinline__ static double value(const Part& p) { return (double)p; }
    __device__ __forceinline__ static void store(void* out, int64_t i, const Part& p, bool) { put_f32(out, i, p); }
    __device__ __forceinline__ static void store_aux(int64_t*, pr_prod_aux*, int64_t, const Part&, int64_t) {}
    __device__ __forceinline__ static void store_empty(void* out, int64_t i, bool f64, int64_t*, pr_prod_aux*) {
        store(out, i, 1.f, f64);
    }
};

// fp64 product on the integer pipes.  GB300's fp64 units issue ~0.5e12
// multiplies/s, slower than HBM delivers doubles (~0.9e12/s), so the combine
// keeps a 64-bit significand m in [2^63, 2^64) and a 64-bit exponent e
// (value = m * 2^(e-63)) and multiplies significands with three 32x32->64
// integer multiplies (mul_sig).  Each step errs by less than 2^-61 relative,
// toward zero (fp64: 2^-53 either way), so n factors err by less than
// n * 2^-61; there is no intermediate overflow or underflow.  Zeros, infinities and NaNs are flags; the sign is
// the xor of all signs (the IEEE rule for multiplication).
struct ProdExt {
    using Ld = LdF64;
    using E = double;
    enum : uint32_t { kNeg = 1, kZero = 2, kInf = 4, kNan = 8 };
    struct Acc { uint64_t m; int64_t e; uint32_t f; uint32_t pad_; };
    using Part = Acc;
    static constexpr bool kIdx = false;
    static constexpr bool kOutF64 = true;

    // m' = a*b / 2^(63+adj), truncated, for a, b in [2^63, 2^64); m' in [2^63, 2^64).
    // Built from the three high 32x32->64 partial products: the low product
    // a0*b0 (< 2^64) is dropped and the rest truncated, so each step errs by
    // less than 2^-61 relative, toward zero, and is exact whenever the dropped
    // bits are zero (e.g. a factor that is a power of two).  An fp64 multiply
    // errs by up to 2^-53.
    __device__ __forceinline__ static uint64_t mul_sig(uint64_t a, uint64_t b, int& adj) {
        const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32), b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
        const uint64_t p01 = (uint64_t)a0 * b1, p10 = (uint64_t)a1 * b0, p11 = (uint64_t)a1 * b1;
        const uint64_t mid = (uint64_t)(uint32_t)p01 + (uint32_t)p10;
        const uint64_t hi = p11 + (p01 >> 32) + (p10 >> 32) + (mid >> 32);
        const int top = (int)(hi >> 63);
        adj = top;
        return top ? hi : ((hi << 1) | ((uint32_t)mid >> 31));
    }
    __device__ __forceinline__ static Acc init() { Acc a; a.m = 0x8000000000000000ull; a.e = 0; a.f = 0; a.pad_ = 0; return a; }

    // Significand b in [2^63, 2^64) and biased exponent of v (v = b * 2^(ebias - 1023 - 63)),
    // or a neutral factor (2^63, 1023) with the class recorded in f for 0 / inf / NaN.
    __device__ __forceinline__ static void decode(uint64_t bits, uint64_t& b, int32_t& ebias, uint32_t& f) {
        const uint32_t ef = (uint32_t)(bits >> 52) & 0x7ffu;
        const uint64_t mant = bits & 0x000fffffffffffffull;
        b = (mant | 0x0010000000000000ull) << 11;
        ebias = (int32_t)ef;
        if (__builtin_expect(ef - 1u >= 0x7feu, 0)) {
            if (ef == 0x7ffu) { f |= mant ? kNan : kInf; b = 0x8000000000000000ull; ebias = 1023; }
            else if (mant == 0) { f |= kZero; b = 0x8000000000000000ull; ebias = 1023; }
            else { const int s = __clzll((long long)mant); b = mant << s; ebias = 12 - s; }  // subnormal
        }
    }
    __device__ __forceinline__ static void add(Acc& a, E v, int64_t) {
        const uint64_t bits = (uint64_t)__double_as_longlong(v);
        a.f ^= (uint32_t)(bits >> 63);
        uint64_t b;
        int32_t eb;
        decode(bits, b, eb, a.f);
        int adj;
        a.m = mul_sig(a.m, b, adj);
        a.e += (int64_t)eb - 1023 + adj;
    }
    // A vector's factors are multiplied pairwise first, so the accumulator's
    // dependent chain advances once per vector rather than once per element.
    template <int K>
    __device__ __forceinline__ static void add_vec(Acc& a, const E (&e)[K], int64_t) {
        uint64_t b[K];
        int32_t eb[K];
        uint32_t sgn = 0;
#pragma unroll
        for (int k = 0; k < K; k++) {
            const uint64_t bits = (uint64_t)__double_as_longlong(e[k]);
            sgn ^= (uint32_t)(bits >> 32);
            decode(bits, b[k], eb[k], a.f);
        }
        a.f ^= sgn >> 31;
#pragma unroll
        for (int s = 1; s < K; s <<= 1)
#pragma unroll
            for (int k = 0; k + s < K; k += 2 * s) {
                int adj;
                b[k] = mul_sig(b[k], b[k + s], adj);
                eb[k] += eb[k + s] + adj;
            }
        int adj;
        a.m = mul_sig(a.m, b[0], adj);
        a.e += (int64_t)eb[0] - 1023 * K + adj;
    }
    __device__ __forceinline__ static Part to_part(const Acc& a) { return a; }
    __device__ __forceinline__ static Part part_init() { return init(); }
    __device__ __forceinline__ static Part combine(const Part& a, const Part& b) {
        Part r;
        int adj;
        r.m = mul_sig(a.m, b.m, adj);
        r.e = a.e + b.e + adj;
        r.f = ((a.f ^ b.f) & kNeg) | ((a.f | b.f) & (kZero | kInf | kNan));
        r.pad_ = 0;
        return r;
    }
    __device__ __forceinline__ static Part warp_reduce(Part p) { return warp_combine<ProdExt>(p); }
    __device__ __forceinline__ static double value(const Part& p) {
        const bool neg = p.f & kNeg;
        if ((p.f & kNan) || ((p.f & kInf) && (p.f & kZero))) return __longlong_as_double(0x7ff8000000000000ll);
        if (p.f & kInf) return neg ? -INFINITY : INFINITY;
        if (p.f & kZero) return neg ? -0.0 : 0.0;
        const double d = __ull2double_rn(p.m);
        int64_t sh = p.e - 63;
        sh = sh < -4000 ? -4000 : (sh > 4000 ? 4000 : sh);
        const double r = ldexp(d, (int)sh);
        return neg ? -r : r;
    }
    __device__ __forceinline__ static void store(void* out, int64_t i, const Part& p, bool) { put_f64(out, i, value(p)); }
    __device__ __forceinline__ static void store_aux(int64_t*, pr_prod_aux*, int64_t, const Part&, int64_t) {}
    __device__ __forceinline__ static void store_empty(void* out, int64_t i, bool f64, int64_t*, pr_prod_aux*) {
        put_f64(out, i, 1.0);
    }
};

// Product that also records what its gradient needs: the product of the
// non-zero elements, the number of zeros, the first zero's index and the xor
// of the zeros' signs.  The product itself is P_nz * (+-0) when zeros exist.
template <class Base>
struct ProdAux {
    using Ld = typename Base::Ld;
    using E = typename Ld::E;
    // sx: xor of every element's sign word (bit 31 is the sign of the element;
    // with a zero present it is the sign of the whole product)
    struct Acc { typename Base::Acc p; int64_t zi; uint32_t zc; uint32_t sx; };
    struct Part { typename Base::Part p; int64_t zc; int64_t zi; uint32_t sall; uint32_t pad_; };
    static constexpr bool kIdx = true;
    // The zero handling lengthens each vector's dependent chain; compiled for
    // at most 512 threads, the row kernel gets the registers to keep more of
    // it in flight (measured on GB300, [64, 2^20] fp32: 52.8 -> 51.1 us).
    static constexpr int kMaxBlock = 512;
    __device__ __forceinline__ static uint32_t sign_word(E v) {
        if constexpr (sizeof(E) == 8) return (uint32_t)((uint64_t)__double_as_longlong(v) >> 32);
        else return __float_as_uint(v);
    }
    __device__ __forceinline__ static Acc init() { Acc a; a.p = Base::init(); a.zi = INT64_MAX; a.zc = 0; a.sx = 0; return a; }
    __device__ __forceinline__ static void add(Acc& a, E v, int64_t i) {
        a.sx ^= sign_word(v);
        if (v == (E)0) {
            a.zc += 1;
            a.zi = i < a.zi ? i : a.zi;
        } else {
            Base::add(a.p, v, i);
        }
    }
    // Zeros are replaced by 1 for the product (so the vector multiplies as a
    // tree in the base trait); the zero count and first zero come from a bit
    // mask, the sign from an xor of all sign words: no per-element branch.
    template <int K>
    __device__ __forceinline__ static void add_vec(Acc& a, const E (&e)[K], int64_t i0) {
        static_assert(K <= 32, "zero mask is one word");
        E t[K];
        uint32_t mask = 0, sx = 0;
#pragma unroll
        for (int k = 0; k < K; k++) {
            const bool z = e[k] == (E)0;
            t[k] = z ? (E)1 : e[k];
            mask |= (uint32_t)z << k;
            sx ^= sign_word(e[k]);
        }
        Base::add_vec(a.p, t, i0);
        a.zc += __popc(mask);
        a.sx ^= sx;
        if (mask) {
            const int64_t i = i0 + __ffs(mask) - 1;
            a.zi = i < a.zi ? i : a.zi;
        }
    }
    __device__ __forceinline__ static Part to_part(const Acc& a) {
        Part r; r.p = Base::to_part(a.p); r.zc = a.zc; r.zi = a.zi; r.sall = a.sx >> 31; r.pad_ = 0; return r;
    }
    __device__ __forceinline__ static Part part_init() { return to_part(init()); }
    __device__ __forceinline__ static Part combine(const Part& a, const Part& b) {
        Part r;
        r.p = Base::combine(a.p, b.p);
        r.zc = a.zc + b.zc;
        r.zi = a.zi < b.zi ? a.zi : b.zi;
        r.sall = a.sall ^ b.sall;
        r.pad_ = 0;
        return r;
    }
    __device__ __forceinline__ static Part warp_reduce(Part p) { return warp_combine<ProdAux>(p); }
    // With a zero the product is a zero whose sign is the xor of all signs,
    // unless the non-zero part is infinite or NaN (then NaN, as inf * 0).
    __device__ __forceinline__ static void store(void* out, int64_t i, const Part& p, bool f64) {
        const double pnz = Base::value(p.p);
        const double v = p.zc > 0 ? (isfinite(pnz) ? (p.sall ? -0.0 : 0.0) : pnz * 0.0) : pnz;
        if (Base::kOutF64) put_f64(out, i, v); else put_f32(out, i, (float)v);
    }
    __device__ __forceinline__ static void store_aux(int64_t*, pr_prod_aux* aux, int64_t i, const Part& p,
                                                     int64_t seg_begin) {
        if (aux) {
            pr_prod_aux r;
            r.p_nz = Base::value(p.p);
            r.zero_count = p.zc;
            r.first_zero = p.zc > 0 ? p.zi - seg_begin : -1;
            aux[i] = r;
        }
    }
    __device__ __forceinline__ static void store_empty(void* out, int64_t i, bool f64, int64_t*, pr_prod_aux* aux) {
        const Part e = part_init();
        store(out, i, e, f64);
        store_aux(nullptr, aux, i, e, 0);
    }
};

}  // namespace pr
