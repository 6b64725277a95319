// common.cuh -- device-side data structures and helpers of the t-FDP library.
//
// Notation follows arXiv 2303.03964: gamma (repulsion exponent), alpha / beta
// (attraction weights), k (interpolation nodes per box and axis), N_int (boxes
// per axis), h (box side), G = N_int * k grid nodes per axis, P = FFT size.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace tfdp {

// ---------------------------------------------------------------- dependent launch
// Kernels of one iteration run back to back on one stream. Launched with
// launch_pdl, a kernel may be scheduled while its predecessor is still finishing; it
// calls pdl_wait() first, which returns once the predecessor grid has completed and its
// writes are visible (a no-op when the launch had no programmatic predecessor), and
// pdl_trigger() to let its own successor be scheduled early. Only kernels that start
// with pdl_wait() are launched this way.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

constexpr int kMaxK = 3;
constexpr double kLFloor = 1.0 / 1024.0;  // narrowest layout square side

enum : int { GRID_PAPER = 0, GRID_SNAP_H = 1 };
enum : int { REP_EXACT = 0, REP_FFT = 1 };

// Device-side bit flags (DevState::flags).
enum : unsigned {
    FLAG_NONFINITE = 1u,     // a position became NaN / inf
    FLAG_BOX_RANGE = 2u,     // a box index fell outside [0, N_int) (should not happen)
    FLAG_SORT_RANGE = 4u,    // a sorted slot fell outside [0, n)
    FLAG_WAIT_TIMEOUT = 8u   // a bounded device wait gave up
};

// Parameters as the kernels read them (copied from tfdp_params by the host).
struct DevParams {
    double alpha, beta, gamma;
    double step0, step_min;
    int k;           // interpolation nodes per box and axis; 0 = dynamic (k_of_iter)
    int n_int_min;
    int grid_max;
    int policy;
    int total_iters;
    int P;           // FFT size per axis
    int log2P;
    int gamma_int;   // gamma if it is a small integer (2..8), else 0
    int spread_shift; // fixed-point scale of the spread sums is 2^(27 - spread_shift)
    const double* step_table;  // s_t for t = 0 .. total_iters - 1 (host-computed, FP64)
    // failure-detection test hook (0, 0 in normal operation): polls before a look-back
    // wait of the box-count scan gives up (0 = the built-in limit), and whether the first
    // scan tile withholds its status so that the waits of the later tiles run out
    int scan_spin_limit;
    int scan_stall;
};

// Grid of one iteration, Sec. 3.4: square [lo, lo + N_int h]^2, N_int x N_int boxes,
// k x k interior nodes per box at offsets (l + 1/2) h / k.
struct GridDesc {
    double lo;      // FP64 value of the FP32 minimum coordinate
    double h;       // box side
    double L;       // layout square side (after the floor)
    float lo_f;     // lo as FP32 (exact)
    float h_f;      // h rounded to FP32 (used by the box decision)
    float h_lo_f;   // h - h_f rounded to FP32 (h = h_f + h_lo_f to ~2^-48 relative)
    float hk_f;     // h / k rounded to FP32 (grid spacing)
    int n_int;
    int G;
    int k;          // interpolation nodes per box and axis in this iteration
    float q_scale;  // fixed-point scale of the spread sums (2^(27 - spread_shift))
    float q_inv;    // 1 / q_scale
};

// k of iteration t of a T-iteration run (Sec. 3.4 "Choices of k"). k > 0 is fixed;
// k = 0 is the paper's dynamic strategy: 1 while t < floor(0.9 T), 2 while
// t < floor(0.95 T), then 3 (the boundaries are a reading). The host picks the
// iteration graph of each segment with the same function.
__host__ __device__ __forceinline__ int k_of_iter(int k, long long t, long long T) {
    if (k > 0) return k;
    if (t < (9 * T) / 10) return 1;
    if (t < (19 * T) / 20) return 2;
    return 3;
}

// Mutable state of one graph on the device.
struct DevState {
    unsigned int bbox[2][2];  // [slot][0]: ordered min, [1]: ordered max over both coords
    long long iter;           // iterations completed
    long long t_cur;          // index t of the iteration in flight
    double step_cur;          // s_t of the iteration in flight
    GridDesc grid;            // grid of the iteration in flight
    double spec_h;            // box side the cached spectrum was built for
    double spec_gamma;
    int spec_k;
    int spec_P;
    int spec_valid;
    int spec_dirty;           // 1: this iteration rebuilds the spectrum
    int spec_builds;
    unsigned int flags;
    double net_frep[2];       // FP64 sum of frep over nodes (last iteration)
    unsigned int done_blocks; // completion counter of the last kernel of an iteration
    int pad_;
    unsigned long long scan_ticket;  // tickets of the single-pass scan (launch * tiles + tile)
};

// ---------------------------------------------------------------- ordered floats
// Monotone map float -> uint32 so that atomicMin / atomicMax on the image order floats.
__device__ __forceinline__ unsigned f2ord(float f) {
    unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned o) {
    unsigned u = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
    return __uint_as_float(u);
}
constexpr unsigned kOrdMinInit = 0xFFFFFFFFu;  // identity of atomicMin on ordered floats
constexpr unsigned kOrdMaxInit = 0u;           // identity of atomicMax

// ---------------------------------------------------------------- grid policy
// Sec. 3.4 "Choices of k": N_int = max(n_int_min, ceil(L)), capped at floor(grid_max/k).
// All decisions are exact FP64 operations on FP32 extremes, so the CPU oracle, which
// performs the same operations, obtains the same N_int and h.
__device__ __forceinline__ GridDesc make_grid(float lo_f, float hi_f, const DevParams& p, int k) {
    GridDesc g;
    double L = (double)hi_f - (double)lo_f;
    if (!(L >= kLFloor)) L = kLFloor;  // also catches NaN
    double c = ceil(L);
    if (c > 2.0e9) c = 2.0e9;
    int n_int = (c > (double)p.n_int_min) ? (int)c : p.n_int_min;
    // N_int cap: floor(grid_max / k) for a fixed k; one cap, floor(grid_max / 3), for every
    // k under the dynamic strategy (p.k = 0), whose N_int rule does not depend on k
    int cap = p.grid_max / (p.k > 0 ? k : kMaxK);
    if (n_int > cap) n_int = cap;
    if (n_int < 1) n_int = 1;
    double h;
    if (p.policy == GRID_PAPER) {
        h = L / (double)n_int;
    } else {
        int e;
        double t = L / (double)n_int;
        (void)frexp(t, &e);
        double base = ldexp(1.0, e - 1);
        h = ldexp(1.0, e);
        for (int j = 0; j <= 16; ++j) {
            double cand = base * (16.0 + (double)j) * 0.0625;  // exact
            if ((double)n_int * cand >= L) { h = cand; break; }
        }
    }
    g.lo = (double)lo_f;
    g.h = h;
    g.L = L;
    g.lo_f = lo_f;
    g.h_f = __double2float_rn(h);
    g.h_lo_f = __double2float_rn(h - (double)g.h_f);
    g.hk_f = __double2float_rn(h / (double)k);
    g.n_int = n_int;
    g.G = n_int * k;
    g.k = k;
    g.q_scale = ldexpf(1.0f, 27 - p.spread_shift);
    g.q_inv = ldexpf(1.0f, p.spread_shift - 27);
    return g;
}

// Box index along one axis, decided in IEEE FP32: floor((x - lo) / h) clamped to
// [0, N_int - 1]. Returns the FP32 quotient t in *tq (box-relative coordinate u = t - a).
__device__ __forceinline__ int box_of(float x, float lo_f, float h_f, int n_int, float* tq) {
    float t = __fdiv_rn(__fsub_rn(x, lo_f), h_f);
    *tq = t;
    const float a = floorf(t);
    // NaN and negative quotients go to box 0, quotients past the end to the last box
    return (a >= 0.0f) ? ((a <= (float)(n_int - 1)) ? (int)a : n_int - 1) : 0;
}

// Lagrange basis over the K interior nodes t_l = (l + 1/2) / K of a unit box at u.
template <int K>
__device__ __forceinline__ void lagrange(float u, float* w) {
    if (K == 1) {
        w[0] = 1.0f;
    } else if (K == 2) {
        // nodes 1/4, 3/4
        w[0] = 1.5f - 2.0f * u;
        w[1] = 2.0f * u - 0.5f;
    } else {
        // nodes 1/6, 1/2, 5/6 -> v = 3u - 3/2 puts them at -1, 0, 1
        float v = 3.0f * u - 1.5f;
        w[0] = 0.5f * v * (v - 1.0f);
        w[1] = 1.0f - v * v;
        w[2] = 0.5f * v * (v + 1.0f);
    }
}

// Step size of iteration t: s0 (s_min / s0)^(t / (T - 1)) (reading; the paper gives none),
// read from a table the host fills in FP64, clamped at t = T - 1.
__device__ __forceinline__ double step_size(long long t, const DevParams& p) {
    if (t > p.total_iters - 1) t = p.total_iters - 1;
    if (t < 0) t = 0;
    return p.step_table[t];
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ float warp_min(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace tfdp
