// Line search whose inner step is the reduction: golden-section and Fibonacci
// search (Section 1 names them among the reduction's consumers; Section 5 uses
// the golden-ratio method in the traffic assignment step) of the Beckmann
// objective of BPR link costs along a direction,
//
//   phi(alpha) = sum_i t0_i (v_i + beta c_i / (p + 1) (v_i / c_i)^(p + 1)),
//   v_i = x_i + alpha d_i.
//
// k_phi      one pass over the four float32 link arrays evaluates phi at up
//            to kLsMaxPts points: each term in float32, a thread's eight
//            links per point summed pairwise and added to the point's Kahan
//            pair, combined per block in float64 and by the last block in
//            block order (the persistent reduction of Section 3 with a fixed
//            combine order).  Error (u = 2^-24, first order): the linear
//            part t0 v of a term takes three roundings (the fma placing v,
//            the fma or product adding t0, the final product); the power
//            part 24 u at power 4 (B: fourteen, the approximate reciprocal's
//            2 u four times over, its two squarings, beta / 5, t0 kb and the
//            last product; v^4: four on v and three of its own; the fma and
//            the product) and (4 p + 7) u otherwise; the sums five (three
//            pairwise levels, two for Kahan's update), the float64 combines
//            below 2^-45.  So phi is within
//            u (8 sum |t0 v| + (c_p + 5) sum |power part|), c_4 = 24.
// k_ls_init  places the first two points and the speculative tree.
// ls_step    (one thread of a search pass's last block, after the sums) walks
//            depth D decisions with the values of the pass, then places the
//            next pass's tree: the 2^(D+1) - 2 points the next D iterations
//            could need, so that D iterations cost one pass over the links
//            instead of D, and the sequence of points is exactly the
//            sequential search's.
// k_ls_init and ls_step run on one thread, with float64 operations written
// out (no contraction into FMA), so that the points match a float64
// implementation that evaluates the same expressions in the same order.
#include <cstdint>
#include "kernels.cuh"
#include "search.cuh"

namespace pr {

// ---- evaluation pass -------------------------------------------------------

__device__ void ls_step(LsState& s, double* result);

// Kahan's compensated add: c holds the negated low part lost so far, so the
// running sum is s - c
__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// (v / c)^(p + 1) for a power known only at run time
template <int PW>
__device__ __forceinline__ float pow_p1(float q, int power) {
    float r = q;
    for (int k = 0; k < power; k++) r *= q;
    return r;
}

// L links of this thread at the first m points: per point the L terms are
// summed pairwise in float32 and the sum enters the point's Kahan pair (the
// loop over points stops at m, so a pass costs what its points need)
template <int PW, int L, int MP>
__device__ __forceinline__ void phi_group(const float (&X)[L], const float (&D)[L], const float (&T)[L],
                                          const float (&C)[L], float kb, int power, const float (&al)[MP],
                                          int m, float (&s)[MP], float (&e)[MP]) {
    // power 4: term = v (t0 + B v^4) with B = t0 beta / ((p + 1) c^4), five
    // operations per point; other powers: t0 v + t0 beta c / (p + 1) (v / c)^(p + 1)
    float inv[L], bc[L];
#pragma unroll
    for (int l = 0; l < L; l++) {
        if constexpr (PW == 4) {
            // rcp.approx: within one unit in the last place (PTX ISA), one
            // instruction; only B depends on it
            asm("rcp.approx.f32 %0, %1;" : "=f"(inv[l]) : "f"(C[l]));
            const float i2 = inv[l] * inv[l];
            bc[l] = (T[l] * kb) * (i2 * i2);
        } else {
            inv[l] = __frcp_rn(C[l]);
            bc[l] = T[l] * kb * C[l];
        }
    }
#pragma unroll
    for (int k = 0; k < MP; k++) {
        if (k >= m) break;
        float t[L];
#pragma unroll
        for (int l = 0; l < L; l++) {
            const float v = fmaf(al[k], D[l], X[l]);
            if constexpr (PW == 4) {
                const float v2 = v * v;
                t[l] = v * fmaf(bc[l], v2 * v2, T[l]);
            } else {
                t[l] = fmaf(bc[l], pow_p1<PW>(v * inv[l], power), T[l] * v);
            }
        }
#pragma unroll
        for (int st = 1; st < L; st <<= 1)
#pragma unroll
            for (int l = 0; l + st < L; l += 2 * st) t[l] += t[l + st];
        kahan_add(s[k], e[k], t[0]);
    }
}

__device__ __forceinline__ void split4(const float4& v, float (&o)[8], int at) {
    o[at] = v.x;
    o[at + 1] = v.y;
    o[at + 2] = v.z;
    o[at + 3] = v.w;
}

// MP: most points of a launch (8: two blocks per SM fit; 16: one)
template <bool VEC, int PW, int MP>
__global__ void __launch_bounds__(kPhiThreads, MP <= 8 ? 2 : 1) k_phi(PhiArgs a) {
    __shared__ double s_w[kPhiThreads / 32][kLsMaxPts];
    __shared__ bool s_last;
    // A search's passes are launched as programmatic dependents of one
    // another: the next pass may start as this one's blocks finish and issue
    // its first loads of links, which no pass writes; it waits for this pass
    // (griddepcontrol.wait: completed, its writes visible) before it reads
    // the points this pass's last block places, and before it writes the
    // partials and the ticket this pass's last block reads.  Without a
    // programmatic launch both instructions return at once.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int m = a.m;
    float al[MP], s[MP], e[MP];
#pragma unroll
    for (int k = 0; k < MP; k++) {
        al[k] = 0.f;
        s[k] = 0.f;
        e[k] = 0.f;
    }
    auto points = [&]() {
        asm volatile("griddepcontrol.wait;" ::: "memory");
#pragma unroll
        for (int k = 0; k < MP; k++) al[k] = k < m ? (float)a.pts[k] : 0.f;
    };
    const float kb = a.beta / (float)(a.power + 1);
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t done = 0;
    if (VEC) {
        const int64_t n4 = a.n / 4;
        const float4* x4 = reinterpret_cast<const float4*>(a.x);
        const float4* d4 = reinterpret_cast<const float4*>(a.d);
        const float4* t4 = reinterpret_cast<const float4*>(a.t0);
        const float4* c4 = reinterpret_cast<const float4*>(a.c);
        // groups of 8 links (two strides); the next group's loads are issued
        // before the current group's arithmetic, so 256 bytes per thread stay
        // in flight
        auto load8 = [&](int64_t j, float (&X)[8], float (&D)[8], float (&T)[8], float (&C)[8]) {
            split4(__ldcs(x4 + j), X, 0);
            split4(__ldcs(d4 + j), D, 0);
            split4(__ldcs(t4 + j), T, 0);
            split4(__ldcs(c4 + j), C, 0);
            split4(__ldcs(x4 + j + stride), X, 4);
            split4(__ldcs(d4 + j + stride), D, 4);
            split4(__ldcs(t4 + j + stride), T, 4);
            split4(__ldcs(c4 + j + stride), C, 4);
        };
        int64_t i = tid;
        if (i + stride < n4) {
            float X[8], D[8], T[8], C[8];
            load8(i, X, D, T, C);
            points();
            for (;;) {
                const int64_t j = i + 2 * stride;
                const bool more = j + stride < n4;
                float Xn[8], Dn[8], Tn[8], Cn[8];
                if (more) load8(j, Xn, Dn, Tn, Cn);
                phi_group<PW, 8, MP>(X, D, T, C, kb, a.power, al, m, s, e);
                i = j;
                if (!more) break;
#pragma unroll
                for (int l = 0; l < 8; l++) {
                    X[l] = Xn[l];
                    D[l] = Dn[l];
                    T[l] = Tn[l];
                    C[l] = Cn[l];
                }
            }
        }
        else {
            points();
        }
        if (i < n4) {
            const float4 X = __ldcs(x4 + i), D = __ldcs(d4 + i), T = __ldcs(t4 + i), C = __ldcs(c4 + i);
            const float Xa[4] = {X.x, X.y, X.z, X.w}, Da[4] = {D.x, D.y, D.z, D.w}, Ta[4] = {T.x, T.y, T.z, T.w},
                        Ca[4] = {C.x, C.y, C.z, C.w};
            phi_group<PW, 4, MP>(Xa, Da, Ta, Ca, kb, a.power, al, m, s, e);
        }
        done = n4 * 4;
    } else {
        points();
    }
    for (int64_t i = done + tid; i < a.n; i += stride) {
        const float X[1] = {__ldcs(a.x + i)}, D[1] = {__ldcs(a.d + i)}, T[1] = {__ldcs(a.t0 + i)},
                    C[1] = {__ldcs(a.c + i)};
        phi_group<PW, 1, MP>(X, D, T, C, kb, a.power, al, m, s, e);
    }

    // per point: thread pair -> float64, warp butterfly, warps in order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < MP; k++) {
        if (k < m) {
            double v = (double)s[k] - (double)e[k];
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) s_w[warp][k] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x < m) {
        double v = 0.0;
        for (int w = 0; w < kPhiThreads / 32; w++) v += s_w[w][threadIdx.x];
        a.partials[(int64_t)blockIdx.x * kLsMaxPts + threadIdx.x] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the last block: warp w sums points w, w + 8, ... over the blocks, lanes
    // striding the block index, then a butterfly (a fixed order per grid)
    for (int k = warp; k < m; k += kPhiThreads / 32) {
        double v = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) v += __ldcg(a.partials + (int64_t)b * kLsMaxPts + k);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) a.out[k] = v;
    }
    if (threadIdx.x == 0) *a.ticket = 0u;
    if (a.ls) {
        __syncthreads();                           // the sums of this pass are in a.out
        if (threadIdx.x == 0) ls_step(*a.ls, a.result);
    }
}

// ---- search state ----------------------------------------------------------

// F_0 = F_1 = 1, F_k = F_{k-1} + F_{k-2} by float64 additions: exact up to
// F_77; F_78 (above 2^53) is the IEEE rounding of the exact sum, as in any
// float64 evaluation of the same recurrence.  k_ls_init fills the search
// state's table once; the search step reads it (a step that ran the
// recurrence for each point it placed spent about 4 us a pass in the chain
// of dependent float64 additions).
__device__ void fill_fib(double* f) {
    f[0] = 1.0;
    f[1] = 1.0;
    for (int k = 2; k <= kLsMaxFib; k++) f[k] = __dadd_rn(f[k - 1], f[k - 2]);
}

struct LsNode {
    double a, b, x1, x2;
    int j;     // iterations done
};

// The child of n after one comparison: br 0 (x1 better) keeps [a, x2] and
// moves x1 up to x2; br 1 keeps [x1, b] and moves x2 down to x1.  Returns
// the new point the child needs.
__device__ double ls_child(const LsState& s, const LsNode& n, int br, LsNode& c) {
    c = n;
    c.j = n.j + 1;
    if (s.method == 0) {
        if (br == 0) {
            c.b = n.x2;
            c.x2 = n.x1;
            c.x1 = __dsub_rn(c.b, __dmul_rn(s.golden, __dsub_rn(c.b, c.a)));
            return c.x1;
        }
        c.a = n.x1;
        c.x1 = n.x2;
        c.x2 = __dadd_rn(c.a, __dmul_rn(s.golden, __dsub_rn(c.b, c.a)));
        return c.x2;
    }
    const int N = s.count, j = c.j;
    const bool last = j == N - 2;
    if (br == 0) {
        c.b = n.x2;
        c.x2 = n.x1;
        c.x1 = last ? __dsub_rn(c.x2, __dmul_rn(0.1, s.u)) : __dadd_rn(c.a, __dmul_rn(s.fib[N - j - 2], s.u));
        return c.x1;
    }
    c.a = n.x1;
    c.x1 = n.x2;
    c.x2 = last ? __dadd_rn(c.x1, __dmul_rn(0.1, s.u)) : __dadd_rn(c.a, __dmul_rn(s.fib[N - j - 1], s.u));
    return c.x2;
}

// The tree of the next `levels` iterations below root, into pts[base...]
__device__ int ls_tree(LsState& s, const LsNode& root, int levels, int base) {
    LsNode cur[1 << kLsMaxDepth], nxt[1 << kLsMaxDepth];
    cur[0] = root;
    int width = 1, np = 0;
    for (int l = 1; l <= levels; l++) {
        for (int k = 0; k < width; k++)
            for (int br = 0; br < 2; br++) s.pts[base + np++] = ls_child(s, cur[k], br, nxt[2 * k + br]);
        width *= 2;
        for (int k = 0; k < width; k++) cur[k] = nxt[k];
    }
    return np;
}

__global__ void k_ls_init(LsState* sp, double lo, double hi, int method, int count, int total, int depth) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");   // the first pass may start streaming
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    LsState& s = *sp;
    s.method = method;
    s.count = count;
    s.total = total;
    s.depth = depth;
    s.iter = 0;
    s.first = 1;
    s.done = 0;
    s.golden = __ddiv_rn(__dsub_rn(sqrt(5.0), 1.0), 2.0);
    s.a = lo;
    s.b = hi;
    if (method == 0) {
        s.u = 0.0;
        s.x1 = __dsub_rn(hi, __dmul_rn(s.golden, __dsub_rn(hi, lo)));
        s.x2 = __dadd_rn(lo, __dmul_rn(s.golden, __dsub_rn(hi, lo)));
    } else {
        fill_fib(s.fib);
        s.u = __ddiv_rn(__dsub_rn(hi, lo), s.fib[count]);
        s.x1 = __dadd_rn(lo, __dmul_rn(s.fib[count - 2], s.u));
        s.x2 = __dadd_rn(lo, __dmul_rn(s.fib[count - 1], s.u));
    }
    s.pts[0] = s.x1;
    s.pts[1] = s.x2;
    const LsNode root{s.a, s.b, s.x1, s.x2, 0};
    s.npts = 2 + ls_tree(s, root, depth < total ? depth : total, 2);
}

// After a pass: walk its decisions, then place the next pass's points, or
// finish and write result (a, b, the better of the last two points, its
// value).  Run by one thread of the pass's last block.
__device__ void ls_step(LsState& s, double* result) {
    if (s.done) return;
    const int base = s.first ? 2 : 0;
    if (s.first) {
        s.f1 = s.vals[0];
        s.f2 = s.vals[1];
    }
    LsNode n{s.a, s.b, s.x1, s.x2, s.iter};
    int path = 0;
    for (int l = 0; l < s.depth && s.iter < s.total; l++) {
        const int br = s.f1 < s.f2 ? 0 : 1;
        LsNode c;
        ls_child(s, n, br, c);
        path = 2 * path + br;
        const double fnew = s.vals[base + (2 << l) - 2 + path];
        if (br == 0) {
            s.f2 = s.f1;
            s.f1 = fnew;
        } else {
            s.f1 = s.f2;
            s.f2 = fnew;
        }
        n = c;
        s.iter++;
    }
    s.a = n.a;
    s.b = n.b;
    s.x1 = n.x1;
    s.x2 = n.x2;
    s.first = 0;
    if (s.iter < s.total) {
        const int left = s.total - s.iter;
        s.npts = ls_tree(s, n, s.depth < left ? s.depth : left, 0);
        return;
    }
    // finished: Fibonacci's last comparison only shrinks the bracket
    if (s.method == 1) {
        if (s.f1 < s.f2) s.b = s.x2;
        else s.a = s.x1;
    }
    s.done = 1;
    s.npts = 0;
    result[0] = s.a;
    result[1] = s.b;
    result[2] = s.f1 < s.f2 ? s.x1 : s.x2;
    result[3] = s.f1 < s.f2 ? s.f1 : s.f2;
}

// ---- launchers -------------------------------------------------------------

template <bool VEC, int MP>
static const void* phi_fn(int power) {
    return power == 4 ? reinterpret_cast<const void*>(&k_phi<VEC, 4, MP>)
                      : reinterpret_cast<const void*>(&k_phi<VEC, 0, MP>);
}

const void* phi_kernel(bool vec, int power, int m) {
    if (m <= 8) return vec ? phi_fn<true, 8>(power) : phi_fn<false, 8>(power);
    return vec ? phi_fn<true, kLsMaxPts>(power) : phi_fn<false, kLsMaxPts>(power);
}

// A search's pass is launched as a programmatic dependent of the kernel
// before it on the stream, which is always the search's own k_ls_init or
// previous pass: neither writes the link arrays the pass reads before its
// wait.  A lone evaluation (pr_beckmann) may follow a caller's kernel that
// writes them, so it is launched in plain stream order.
template <bool VEC, int MP>
static void phi_go(const PhiArgs& a, int grid, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kPhiThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = a.ls ? 1 : 0;
    if (a.power == 4) cudaLaunchKernelEx(&cfg, k_phi<VEC, 4, MP>, a);
    else cudaLaunchKernelEx(&cfg, k_phi<VEC, 0, MP>, a);
}

cudaError_t launch_phi(const PhiArgs& a, int grid, bool vec, cudaStream_t st) {
    if (a.m <= 8) {
        if (vec) phi_go<true, 8>(a, grid, st);
        else phi_go<false, 8>(a, grid, st);
    } else {
        if (vec) phi_go<true, kLsMaxPts>(a, grid, st);
        else phi_go<false, kLsMaxPts>(a, grid, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_ls_init(LsState* s, double lo, double hi, int method, int count, int total, int depth,
                           cudaStream_t st) {
    k_ls_init<<<1, 32, 0, st>>>(s, lo, hi, method, count, total, depth);
    return cudaGetLastError();
}


}  // namespace pr
