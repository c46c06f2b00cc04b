// fp64 product split across two pipes.  GB300's fp64 pipe multiplies about
// 0.5e12 doubles per second and the integer-pipe product of ProdExt (three
// 32x32->64 partial products per factor) is bound by the ALU pipe; HBM
// delivers about 0.85e12 doubles per second, more than either alone.  So in
// every vector of K factors the first K/2 multiply on the fp64 pipe, as
// significands in [1, 2) with their exponents summed as integers (no
// intermediate overflow or underflow: the running significand is rescaled
// when it passes 2^512), and the rest on the integer pipes as in ProdExt.
// Zeros, infinities, NaNs and subnormals always take the integer path, which
// records their class.  The two partial products meet in to_part.
//
// Error, every rounding counted (first order, u = 2^-53).  Whatever the order,
// combining n factors takes exactly n - 1 merges of two partial products that
// both hold factors (a merge with the identity -- an untouched accumulator,
// or the 1.0 an fp64-pipe product starts from -- is exact).  A merge on the
// fp64 pipe rounds to nearest (at most u); a merge on the integer pipes
// (mul_sig: per factor, in to_part, fold, and the warp, block and grid
// combines) truncates, under 3 * 2^-63 < u / 256.  At most n / 2 merges run
// on the fp64 pipe, and the final conversion to double rounds once more.  So
// the relative error is below u (n / 2 + 1) + (u / 256) (n - 1), which is at
// most max(n - 1, 2) u for every n (n <= 4 counted case by case: one vector
// of four makes one rounding fp64 merge and two truncations).
#pragma once
#include "traits.cuh"

namespace pr {

struct ProdMix {
    using Ld = LdF64;
    using E = double;
    using Part = ProdExt::Part;
    struct Acc {
        ProdExt::Acc x;   // integer-pipe product, sign and class flags
        double m2;        // fp64-pipe significand product, in [1, 2^513)
        int64_t e2;       // and its exponent
    };
    static constexpr bool kIdx = false;
    static constexpr bool kOutF64 = true;

    __device__ __forceinline__ static Acc init() {
        Acc a;
        a.x = ProdExt::init();
        a.m2 = 1.0;
        a.e2 = 0;
        return a;
    }
    __device__ __forceinline__ static void add(Acc& a, E v, int64_t i) { ProdExt::add(a.x, v, i); }

    // a normal factor on the fp64 pipe; any other class on the integer path
    __device__ __forceinline__ static void add_fp64(Acc& a, E v) {
        const uint64_t bits = (uint64_t)__double_as_longlong(v);
        const uint32_t hi = (uint32_t)(bits >> 32);
        const uint32_t ef = (hi >> 20) & 0x7ffu;
        if (ef - 1u >= 0x7feu) {
            ProdExt::add(a.x, v, 0);
            return;
        }
        a.x.f ^= hi >> 31;
        const double sig = __longlong_as_double((long long)((bits & 0x000fffffffffffffull) | 0x3ff0000000000000ull));
        a.m2 = __dmul_rn(a.m2, sig);
        a.e2 += (int64_t)ef - 1023;
    }
    // m2 back to [1, 2), its exponent moved into e2
    __device__ __forceinline__ static void rescale(Acc& a) {
        const uint64_t b = (uint64_t)__double_as_longlong(a.m2);
        a.e2 += (int64_t)((b >> 52) & 0x7ffu) - 1023;
        a.m2 = __longlong_as_double((long long)((b & 0x000fffffffffffffull) | 0x3ff0000000000000ull));
    }
    template <int K>
    __device__ __forceinline__ static void add_vec(Acc& a, const E (&e)[K], int64_t i0) {
        constexpr int H = K / 2;
#pragma unroll
        for (int k = 0; k < H; k++) add_fp64(a, e[k]);
        if ((uint32_t)(__double_as_longlong(a.m2) >> 52) > 1023u + 512u) rescale(a);
        if constexpr (K - H == 1) {
            ProdExt::add(a.x, e[H], i0);
        } else {
            E t[K - H];
#pragma unroll
            for (int k = 0; k < K - H; k++) t[k] = e[H + k];
            ProdExt::template add_vec<K - H>(a.x, t, i0);
        }
    }
    // the fp64-pipe product joins the integer-pipe one as one more factor
    __device__ __forceinline__ static Part to_part(const Acc& a) {
        Part p = a.x;
        const uint64_t bits = (uint64_t)__double_as_longlong(a.m2);
        const uint64_t b = ((bits & 0x000fffffffffffffull) | 0x0010000000000000ull) << 11;
        int adj;
        p.m = ProdExt::mul_sig(p.m, b, adj);
        p.e += (int64_t)((bits >> 52) & 0x7ffu) - 1023 + adj + a.e2;
        return p;
    }
    __device__ __forceinline__ static Part part_init() { return ProdExt::part_init(); }
    __device__ __forceinline__ static Part combine(const Part& a, const Part& b) { return ProdExt::combine(a, b); }
    __device__ __forceinline__ static Part warp_reduce(Part p) { return warp_combine<ProdExt>(p); }
    __device__ __forceinline__ static double value(const Part& p) { return ProdExt::value(p); }
    __device__ __forceinline__ static void store(void* out, int64_t i, const Part& p, bool f64) {
        ProdExt::store(out, i, p, f64);
    }
    __device__ __forceinline__ static void store_aux(int64_t* ai, pr_prod_aux* ax, int64_t i, const Part& p,
                                                     int64_t sb) {
        ProdExt::store_aux(ai, ax, i, p, sb);
    }
    __device__ __forceinline__ static void store_empty(void* out, int64_t i, bool f64, int64_t* ai,
                                                       pr_prod_aux* ax) {
        ProdExt::store_empty(out, i, f64, ai, ax);
    }
};

}  // namespace pr
