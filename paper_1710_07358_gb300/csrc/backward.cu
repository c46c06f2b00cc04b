// Backward kernels of a row reduction y[r] = (x) over x[r, 0..cols):
//   SUM      dy/dx[r,c] = 1
//   MAX/MIN  1 at the first arg-extremum, 0 elsewhere
//   PROD     prod_{j != c} x[r,j]: with no zero in the row P_nz / x[r,c];
//            with one zero, P_nz at the zero and 0 elsewhere; with two or
//            more zeros, 0 everywhere (P_nz = product of the non-zero elements)
// times grad_out[r].  The work is one streaming write of grad_in (plus a read
// of x for product rows without zeros): rows are cut into chunks of
// blockDim*U vectors, each thread writes U vectors of VB bytes.  The grid is
// several times what is resident and chunk t goes to block t mod grid, so the
// blocks in flight always write one window of neighbouring chunks and the
// hardware hands the remaining blocks to whichever SMs finish first (no tail of
// SMs still writing fixed shares).  Row-uniform values (grad_out, argidx, aux)
// are re-read only when a block's row changes.
#include "registry.h"
#include "kernels.cuh"
#include "axis.cuh"

namespace pr {


template <class F, int VB>
__device__ __forceinline__ void st_vec(F* p, const F (&v)[VB / sizeof(F)]);

template <>
__device__ __forceinline__ void st_vec<float, 16>(float* p, const float (&v)[4]) {
    asm volatile("st.global.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]) : "memory");
}
template <>
__device__ __forceinline__ void st_vec<float, 32>(float* p, const float (&v)[8]) {
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]),
                 "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]) : "memory");
}
template <>
__device__ __forceinline__ void st_vec<double, 16>(double* p, const double (&v)[2]) {
    asm volatile("st.global.v2.f64 [%0], {%1,%2};" ::"l"(p), "d"(v[0]), "d"(v[1]) : "memory");
}
template <>
__device__ __forceinline__ void st_vec<double, 32>(double* p, const double (&v)[4]) {
    asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(v[0]), "d"(v[1]), "d"(v[2]), "d"(v[3]) : "memory");
}

// Row-uniform description of the gradient: value gv at column `hot` (or at
// every column when hot == -2), 0 elsewhere; div: gv / x[c] at every column.
template <class F>
struct RowGrad {
    F gv;
    int64_t hot;
    bool div;
};

template <class F>
__device__ __forceinline__ RowGrad<F> row_grad(const BwdArgs& a, int64_t r) {
    const F g = static_cast<const F*>(a.g)[r];
    RowGrad<F> rg{g, -2, false};
    if (a.op == PR_MAX || a.op == PR_MIN) {
        rg.hot = a.argidx[r];
        if (rg.hot < 0) rg.hot = -1;
    } else if (a.op == PR_PROD) {
        const pr_prod_aux ax = a.aux[r];
        const F gp = (F)((double)g * ax.p_nz);
        if (ax.zero_count == 0) { rg.gv = gp; rg.div = true; }
        else if (ax.zero_count == 1) { rg.gv = gp; rg.hot = ax.first_zero; }
        else { rg.gv = (F)0; rg.hot = -1; }
    }
    return rg;
}

template <class F>
__device__ __forceinline__ F elem_grad(const RowGrad<F>& rg, const F* xrow, int64_t c) {
    if (rg.div) return rg.gv / xrow[c];
    if (rg.hot == -2) return rg.gv;
    return c == rg.hot ? rg.gv : (F)0;
}

template <class F, int U, int VB>
__global__ void __launch_bounds__(1024) k_backward(BwdArgs a) {
    constexpr int VE = VB / sizeof(F);
    F* gi = static_cast<F*>(a.gi);
    const F* x = static_cast<const F*>(a.x);
    const int64_t ntiles = a.rows * a.chunks_per_row;
    const int64_t CV = (int64_t)blockDim.x * U;  // vectors per chunk
    int64_t rc = -1;
    RowGrad<F> rg{};
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t r = t / a.chunks_per_row, c = t - r * a.chunks_per_row;
        if (r != rc) {
            rg = row_grad<F>(a, r);
            rc = r;
        }
        const int64_t base = r * a.cols;
        const int64_t mis = (base + a.shift) % VE;
        int64_t head = (VE - mis) % VE;
        head = head < a.cols ? head : a.cols;
        const int64_t nvec = (a.cols - head) / VE;
        F* grow = gi + base;
        const F* xrow = x ? x + base : nullptr;
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int64_t v = c * CV + (int64_t)u * blockDim.x + threadIdx.x;
            if (v < nvec) {
                const int64_t c0 = head + v * VE;
                F vals[VE];
                // row-uniform branches: the broadcast and one-hot rows cost no
                // per-element arithmetic beyond one compare
                if (rg.div) {
#pragma unroll
                    for (int k = 0; k < VE; k++) vals[k] = rg.gv / xrow[c0 + k];
                } else if (rg.hot == -2) {
#pragma unroll
                    for (int k = 0; k < VE; k++) vals[k] = rg.gv;
                } else {
                    const int64_t h = rg.hot - c0;
                    const int hk = (h >= 0 && h < VE) ? (int)h : -1;
#pragma unroll
                    for (int k = 0; k < VE; k++) vals[k] = hk == k ? rg.gv : (F)0;
                }
                st_vec<F, VB>(grow + c0, vals);
            }
        }
        if (c == 0) {
            // unaligned head and the tail after the last full vector
            const int64_t tail0 = head + nvec * VE;
            const int64_t nscalar = head + (a.cols - tail0);
            for (int64_t j = threadIdx.x; j < nscalar; j += blockDim.x) {
                const int64_t col = j < head ? j : tail0 + (j - head);
                grow[col] = elem_grad(rg, xrow, col);
            }
        }
    }
}

template <class F, int U, int VB>
cudaError_t launch_backward(const BwdArgs& a, int grid, int block, cudaStream_t st) {
    k_backward<F, U, VB><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

template <class F, int U, int VB>
static void reg_bwd(uint8_t dtype) {
    reg_add(KernelKey{K_BACKWARD, dtype, 0, 0, 0, (uint8_t)U, (uint8_t)VB},
            KernelEntry{reinterpret_cast<const void*>(&k_backward<F, U, VB>),
                        reinterpret_cast<void*>(&launch_backward<F, U, VB>)});
}

template <class F, int VB, int OPK>
cudaError_t launch_axis_backward(const AxisBwdArgs& a, int grid, int block, cudaStream_t st) {
    k_axis_backward<F, VB, OPK><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

// Keyed by (dtype, op kind in the op field: 0 sum, 1 max/min, 2 prod, vector width).
template <class F, int VB>
static void reg_axis_bwd(uint8_t dtype) {
    reg_add(KernelKey{K_AXIS_BACKWARD, dtype, 0, 0, 0, 0, (uint8_t)VB},
            KernelEntry{reinterpret_cast<const void*>(&k_axis_backward<F, VB, 0>),
                        reinterpret_cast<void*>(&launch_axis_backward<F, VB, 0>)});
    reg_add(KernelKey{K_AXIS_BACKWARD, dtype, 1, 0, 0, 0, (uint8_t)VB},
            KernelEntry{reinterpret_cast<const void*>(&k_axis_backward<F, VB, 1>),
                        reinterpret_cast<void*>(&launch_axis_backward<F, VB, 1>)});
    reg_add(KernelKey{K_AXIS_BACKWARD, dtype, 2, 0, 0, 0, (uint8_t)VB},
            KernelEntry{reinterpret_cast<const void*>(&k_axis_backward<F, VB, 2>),
                        reinterpret_cast<void*>(&launch_axis_backward<F, VB, 2>)});
}

void register_backward() {
    reg_axis_bwd<float, 0>(PR_F32);
    reg_axis_bwd<float, 16>(PR_F32);
    reg_axis_bwd<float, 32>(PR_F32);
    reg_axis_bwd<double, 0>(PR_F64);
    reg_axis_bwd<double, 16>(PR_F64);
    reg_axis_bwd<double, 32>(PR_F64);
    reg_bwd<float, 2, 16>(PR_F32);
    reg_bwd<float, 2, 32>(PR_F32);
    reg_bwd<float, 4, 16>(PR_F32);
    reg_bwd<float, 4, 32>(PR_F32);
    reg_bwd<double, 2, 16>(PR_F64);
    reg_bwd<double, 2, 32>(PR_F64);
    reg_bwd<double, 4, 16>(PR_F64);
    reg_bwd<double, 4, 32>(PR_F64);
}

}  // namespace pr
