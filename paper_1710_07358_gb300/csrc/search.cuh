// Layout shared by the line-search kernels and the host: the search state
// that lives in device memory between passes, and the arguments of one
// evaluation pass of the Beckmann objective.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pr {

constexpr int kLsMaxDepth = 3;                       // iterations decided per pass, at most
constexpr int kLsMaxFib = 78;                        // Fibonacci search: at most 78 evaluations
constexpr int kLsMaxPts = 2 + (2 << kLsMaxDepth) - 2; // first pass: 2 initial points + the tree
constexpr int kPhiThreads = 256;

// Bracket [a, b] with points x1 < x2 and their values; iter of total
// iterations done.  pts / npts: the points the next pass evaluates (first
// pass: x1, x2, then the speculative tree; later passes: the tree only),
// vals: their values.  Tree order: level l (1-based) holds 2^l nodes at
// offset 2^l - 2, node k's children are 2k (x1 side kept) and 2k + 1.
struct LsState {
    double a, b, x1, x2, f1, f2;
    double u;          // Fibonacci unit (hi - lo) / F_N
    double golden;     // (sqrt(5) - 1) / 2
    double pts[kLsMaxPts];
    double vals[kLsMaxPts];
    double fib[kLsMaxFib + 1];   // F_0 .. F_78 (F_0 = F_1 = 1), filled by k_ls_init
    int32_t method;    // 0 golden-section, 1 Fibonacci
    int32_t count;     // golden: iterations; Fibonacci: evaluations N
    int32_t iter, total, depth, first, npts, done;
};

struct PhiArgs {
    const float* x;
    const float* d;
    const float* t0;
    const float* c;
    int64_t n;
    float beta;
    int power;
    const double* pts;     // m evaluation points (device)
    int m;
    double* out;           // m sums (device)
    double* partials;      // gridDim.x * kLsMaxPts block partials
    unsigned* ticket;      // zero between launches
    LsState* ls;           // a search's state: its step runs after the sums (or null)
    double* result;        // where the search's last step writes its result
};

// The evaluation kernel for (vector path, power, points) and its launcher.
const void* phi_kernel(bool vec, int power, int m);
cudaError_t launch_phi(const PhiArgs& a, int grid, bool vec, cudaStream_t st);
cudaError_t launch_ls_init(LsState* s, double lo, double hi, int method, int count, int total, int depth,
                           cudaStream_t st);

}  // namespace pr
