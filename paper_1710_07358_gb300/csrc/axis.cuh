// Reduction along the middle axis of a contiguous row-major [outer, n, inner]
// array: out[p, q] = x[p, 0, q] (x) x[p, 1, q] (x) ... (x) x[p, n-1, q].  With
// outer = the product of the leading sizes and inner = the product of the
// trailing ones this is the reduction of any one axis of a contiguous tensor
// (Section 1.1's reduction, applied to every column of every [n, inner] slab).
//
// k_axis    one warp per (slab p, group of column vectors, split of the rows).
//   A lane owns one column vector (VB bytes; VB = 0: one element) and keeps
//   one accumulator per element of it.  When a row holds fewer than 32 column
//   vectors, a warp covers 32/bx rows per step (bx lanes per row), so every
//   load instruction still touches 32 neighbouring vectors.  Each lane issues
//   U rows' loads before accumulating any of them.  The lanes that share a
//   column then combine by an xor butterfly over the row bits of the lane
//   index, in a fixed order.  With one split the warp writes the outputs; with
//   more, it writes its partials, and k_axis_finish combines each output's
//   partials in a fixed order (one thread per output folding the splits in
//   order, or with many splits one warp per output and a fixed tree), so
//   results are deterministic for a fixed launch shape.
// k_axis_backward  gradient of an axis reduction: grad_in[p, i, q] from
//   grad_out[p, q] and the per-output state, one streaming write.
#pragma once
#include "kernels.cuh"

namespace pr {

struct AxisArgs {
    const void* x;
    int64_t outer, n, inner;
    int64_t qv;               // column vectors per row: inner / VE
    int bx;                   // lanes per row (power of two, <= 32)
    int64_t groups;           // column groups per row: ceil(qv / bx)
    int64_t splits;           // row splits
    int64_t rows_per_split;
    void* out;
    int64_t* argidx;
    pr_prod_aux* aux;
    int out_f64;
    char* scratch;            // splits > 1: partials of GridR<T>::Part, [split][output] when
                              // splits <= kAxisThreadFinish, else [output][split]
};

// Up to this many splits the finishing pass takes one thread per output
// (coalesced over outputs); beyond it, one warp per output.
constexpr int kAxisThreadFinish = 64;

// A column's elements reach its accumulator in increasing index order, so a
// trait may take them with a cheaper in-order step (add_ordered).
template <class T, class = void>
struct HasOrdered : std::false_type {};
template <class T>
struct HasOrdered<T, std::void_t<decltype(&T::add_ordered)>> : std::true_type {};

// A trait whose in-order step runs on a caller's (value, row) register pair
// (kOrderedPair: the arg-extremum of floats).
template <class T, class = void>
struct HasOrderedPair : std::false_type {};
template <class T>
struct HasOrderedPair<T, std::void_t<decltype(T::kOrderedPair)>> : std::true_type {};

template <class T>
__device__ __forceinline__ void add_in_order(typename T::Acc& a, typename T::Ld::E v, int64_t i) {
    if constexpr (HasOrdered<T>::value) T::add_ordered(a, v, i);
    else T::add(a, v, i);
}

template <int VB, class Ld>
__device__ __forceinline__ void axis_load(const typename Ld::In* x, int64_t e0, typename Ld::E (&e)[VB ? VB / Ld::ES : 1]) {
    if constexpr (VB == 0) {
        e[0] = Ld::one(x, e0);
    } else {
        const Words<VB> w = ldv<VB>(x + e0);
        Ld::template dec<VB>(w, e);
    }
}

template <class T, int U, int VB>
__global__ void __launch_bounds__(MaxBlock<T>::value) k_axis(AxisArgs a) {
    using Ld = typename T::Ld;
    using In = typename Ld::In;
    using E = typename Ld::E;
    using Acc = typename T::Acc;
    using Part = typename T::Part;
    using GR = GridR<T>;
    using G = typename GR::Part;
    constexpr int VE = VB ? VB / Ld::ES : 1;
    const In* x = static_cast<const In*>(a.x);
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t tiles = a.outer * a.groups;
    if (wid >= tiles * a.splits) return;  // whole warps (blockDim is a multiple of 32)
    const int64_t tile = wid / a.splits, s = wid - tile * a.splits;
    const int64_t p = tile / a.groups, grp = tile - p * a.groups;
    const int bx = a.bx, ry = 32 / bx;
    const int tx = lane & (bx - 1), ty = lane / bx;
    const int64_t col = grp * bx + tx;
    const bool has = col < a.qv;
    const int64_t r0 = s * a.rows_per_split;
    const int64_t r1 = r0 + a.rows_per_split < a.n ? r0 + a.rows_per_split : a.n;
    const int64_t slab = p * a.n * a.inner + col * VE;  // element offset of (p, row 0, this column)

    Acc acc[VE];
#pragma unroll
    for (int k = 0; k < VE; k++) acc[k] = T::init();
    if constexpr (HasOrderedPair<T>::value) {
        // per element the running extremum and its row relative to r0 (a
        // split holds fewer than 2^31 rows): three operations an element
        // (pick, compare of bits, select) instead of the accumulator's
        // 64-bit index and its "none yet" test; started at this lane's first
        // row, then the same steps as add_ordered
        if (has && r0 + ty < r1) {
            float sv[VE];
            int so[VE];
            int64_t r = r0 + ty;
            {
                E e[VE];
                axis_load<VB, Ld>(x, slab + r * a.inner, e);
#pragma unroll
                for (int k = 0; k < VE; k++) {
                    sv[k] = e[k];
                    so[k] = (int)(r - r0);
                }
            }
            r += ry;
            for (; r + (int64_t)(U - 1) * ry < r1; r += (int64_t)U * ry) {
                E e[U][VE];
#pragma unroll
                for (int u = 0; u < U; u++) axis_load<VB, Ld>(x, slab + (r + (int64_t)u * ry) * a.inner, e[u]);
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int rel = (int)(r + (int64_t)u * ry - r0);
#pragma unroll
                    for (int k = 0; k < VE; k++) {
                        const float m = T::ordered_pick(sv[k], e[u][k]);
                        so[k] = __float_as_uint(m) != __float_as_uint(sv[k]) ? rel : so[k];
                        sv[k] = m;
                    }
                }
            }
            for (; r < r1; r += ry) {
                E e[VE];
                axis_load<VB, Ld>(x, slab + r * a.inner, e);
                const int rel = (int)(r - r0);
#pragma unroll
                for (int k = 0; k < VE; k++) {
                    const float m = T::ordered_pick(sv[k], e[k]);
                    so[k] = __float_as_uint(m) != __float_as_uint(sv[k]) ? rel : so[k];
                    sv[k] = m;
                }
            }
#pragma unroll
            for (int k = 0; k < VE; k++) acc[k] = T::from_ordered(sv[k], r0 + so[k]);
        }
    } else if (has) {
        int64_t r = r0 + ty;
        for (; r + (int64_t)(U - 1) * ry < r1; r += (int64_t)U * ry) {
            E e[U][VE];
#pragma unroll
            for (int u = 0; u < U; u++) axis_load<VB, Ld>(x, slab + (r + (int64_t)u * ry) * a.inner, e[u]);
#pragma unroll
            for (int u = 0; u < U; u++)
#pragma unroll
                for (int k = 0; k < VE; k++) add_in_order<T>(acc[k], e[u][k], r + (int64_t)u * ry);
        }
        for (; r < r1; r += ry) {
            E e[VE];
            axis_load<VB, Ld>(x, slab + r * a.inner, e);
#pragma unroll
            for (int k = 0; k < VE; k++) add_in_order<T>(acc[k], e[k], r);
        }
    }
    const bool f64 = a.out_f64 != 0;
#pragma unroll
    for (int k = 0; k < VE; k++) {
        Part q = T::to_part(acc[k]);
        for (int m = 16; m >= bx; m >>= 1) q = T::combine(q, shfl_xor_any(q, m));
        if (ty == 0 && has) {
            const int64_t o = p * a.inner + col * VE + k;
            const G g = GR::up(q);
            if (a.splits == 1) {
                GR::store(a.out, o, g, f64);
                GR::store_aux(a.argidx, a.aux, o, g, 0);
            } else {
                const int64_t nout = a.outer * a.inner;
                reinterpret_cast<G*>(a.scratch)[a.splits <= kAxisThreadFinish ? s * nout + o : o * a.splits + s] = g;
            }
        }
    }
}

// Few splits: one thread per output folds its splits in order.  Many: one
// warp per output, the lanes taking the splits in order (lane, lane + 32, ...)
// and combining by a fixed butterfly.
template <class T>
__global__ void __launch_bounds__(256) k_axis_finish(AxisArgs a) {
    using GR = GridR<T>;
    using G = typename GR::Part;
    const int64_t nout = a.outer * a.inner;
    const G* part = reinterpret_cast<const G*>(a.scratch);
    if (a.splits <= kAxisThreadFinish) {
        const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (o >= nout) return;
        G q = part[o];
        for (int64_t s = 1; s < a.splits; s++) q = GR::combine(q, part[s * nout + o]);
        GR::store(a.out, o, q, a.out_f64 != 0);
        GR::store_aux(a.argidx, a.aux, o, q, 0);
        return;
    }
    const int lane = threadIdx.x & 31;
    const int64_t o = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (o >= nout) return;
    const G* src = part + o * a.splits;
    G q = GR::part_init();
    for (int64_t s = lane; s < a.splits; s += 32) q = GR::combine(q, src[s]);
    q = GR::warp_reduce(q);
    if (lane == 0) {
        GR::store(a.out, o, q, a.out_f64 != 0);
        GR::store_aux(a.argidx, a.aux, o, q, 0);
    }
}

// Empty axis (n == 0): every output is the identity.
template <class T>
__global__ void __launch_bounds__(256) k_axis_empty(AxisArgs a) {
    const int64_t nout = a.outer * a.inner;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < nout; o += (int64_t)gridDim.x * blockDim.x)
        T::store_empty(a.out, o, a.out_f64 != 0, a.argidx, a.aux);
}

struct AxisBwdArgs {
    const void* x;            // PROD only
    const void* g;            // grad_out [outer, inner]
    const int64_t* argidx;    // MAX / MIN: [outer, inner]
    const pr_prod_aux* aux;   // PROD: [outer, inner]
    void* gi;                 // grad_in [outer, n, inner]
    int64_t outer, n, inner;
    int64_t qv;               // vectors per row: inner / VE
    int op;
};

// grad_in viewed as rows (p, i) of qv vectors; a thread walks the flattened
// vectors with a grid stride, advancing (p, i, column) by carries instead of
// dividing per vector.  OPK: 0 sum (broadcast), 1 max/min (one-hot at argidx),
// 2 prod (zero-count aware).  With VB > 0, grad_out (and argidx) are read as
// vectors of the same columns.
template <class F, int VB, int OPK>
__global__ void __launch_bounds__(256) k_axis_backward(AxisBwdArgs a) {
    constexpr int VE = VB ? VB / (int)sizeof(F) : 1;
    const F* g = static_cast<const F*>(a.g);
    const F* x = static_cast<const F*>(a.x);
    F* gi = static_cast<F*>(a.gi);
    const int64_t total = a.outer * a.n * a.qv;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= total) return;
    int64_t R = v / a.qv, cq = v - R * a.qv;
    int64_t p = R / a.n, i = R - p * a.n;
    const int64_t dR = stride / a.qv, dq = stride - dR * a.qv;
    const int64_t dp = dR / a.n, di = dR - dp * a.n;
    for (; v < total; v += stride) {
        const int64_t o0 = p * a.inner + cq * VE;        // first output of this vector's columns
        const int64_t e0 = (p * a.n + i) * a.inner + cq * VE;
        F gv[VE];
        if constexpr (VB == 0) {
            gv[0] = g[o0];
        } else {
            const Words<VB> w = ldv<VB>(g + o0);
            memcpy(gv, w.w, VB);
        }
        F vals[VE];
        if constexpr (OPK == 0) {
#pragma unroll
            for (int k = 0; k < VE; k++) vals[k] = gv[k];
        } else if constexpr (OPK == 1) {
#pragma unroll
            for (int k = 0; k < VE; k++) vals[k] = __ldg(a.argidx + o0 + k) == i ? gv[k] : (F)0;
        } else {
#pragma unroll
            for (int k = 0; k < VE; k++) {
                const pr_prod_aux ax = a.aux[o0 + k];
                const F gp = (F)((double)gv[k] * ax.p_nz);
                vals[k] = ax.zero_count == 0 ? gp / x[e0 + k]
                          : (ax.zero_count == 1 && ax.first_zero == i ? gp : (F)0);
            }
        }
        if constexpr (VB == 0) {
            gi[e0] = vals[0];
        } else {
            F* dst = gi + e0;
            if constexpr (sizeof(F) == 4 && VB == 16)
                asm volatile("st.global.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(dst), "f"((float)vals[0]), "f"((float)vals[1]),
                             "f"((float)vals[2]), "f"((float)vals[3]) : "memory");
            else if constexpr (sizeof(F) == 4 && VB == 32)
                asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(dst), "f"((float)vals[0]),
                             "f"((float)vals[1]), "f"((float)vals[2]), "f"((float)vals[3]), "f"((float)vals[4]),
                             "f"((float)vals[5]), "f"((float)vals[6]), "f"((float)vals[7]) : "memory");
            else if constexpr (sizeof(F) == 8 && VB == 16)
                asm volatile("st.global.v2.f64 [%0], {%1,%2};" ::"l"(dst), "d"((double)vals[0]), "d"((double)vals[1]) : "memory");
            else
                asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(dst), "d"((double)vals[0]), "d"((double)vals[1]),
                             "d"((double)vals[2]), "d"((double)vals[3]) : "memory");
        }
        // advance by the stride: columns, then rows, then slabs
        cq += dq;
        const int64_t c1 = cq >= a.qv ? 1 : 0;
        cq -= c1 * a.qv;
        i += di + c1;
        const int64_t c2 = i >= a.n ? 1 : 0;
        i -= c2 * a.n;
        p += dp + c2;
    }
}

}  // namespace pr
