// launch.h -- host-side launch interface between the C ABI (tfdp_api.cu) and the
// kernel translation units. Plain structs of device pointers and sizes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace tfdp {

// Buffers and geometry of the FFT stage (fft_kernels.cu).
struct FftLaunch {
    int logP;            // FFT size P = 2^logP per axis (7..13)
    int G_max;           // largest grid G this graph may use
    int Gs;              // row stride (and rows per plane) of gin / gout
    int ystride;         // column stride of T1 / T2 (multiple of 32, >= G_max)
    const float* gin;    // 3 planes of Gs x Gs: rho, m^x, m^y
    float2* T1;          // [3][P/2+1][ystride]
    float2* T2;          // [3][P/2+1][ystride]
    float4* gout;        // [Gs][Gs] (A, O^x, O^y, 0)
    float2* S1;          // [3][P/2+1][P] spectrum build scratch
    float* specK;        // [P/2+1][P]
    float* specHx;       // [P/2+1][P]
    float* specHy;       // [P/2+1][P]
    const float2* tw;    // [P] twiddles exp(-2 pi i t / P)
    DevState* st;
    const DevParams* prm;
};

cudaError_t launch_spectrum(const FftLaunch& a, cudaStream_t s);   // no kernel (rebuilt by the passes below)
cudaError_t launch_rows_fwd(const FftLaunch& a, cudaStream_t s);   // 1 kernel
cudaError_t launch_cols(const FftLaunch& a, cudaStream_t s);       // 1 kernel
cudaError_t launch_rows_inv(const FftLaunch& a, cudaStream_t s);   // 1 kernel
// BF16x3 tensor-core column stage (cols_tc.cu), P = 2048 only: the 96 KB DFT-matrix image
// (build_tc_constants, uploaded once per arena), natural-order kernel spectra
// (3 x (P/2+1) x P floats, rebuilt in place when the spectrum is stale), 1 kernel.
void build_tc_constants(std::vector<unsigned char>& img);
size_t tc_constants_bytes();
size_t tc_spectrum_floats();
cudaError_t prepare_cols_tc();  // shared-memory attribute (call outside stream capture)
cudaError_t launch_cols_tc(const FftLaunch& a, const unsigned char* consts, float* specN, cudaStream_t s);
// Shared-memory attributes of the FFT kernels of size 2^logP (call outside stream capture).
cudaError_t prepare_fft(int logP);

// Buffers of the node stages (node_kernels.cu).
// Degree above which the attraction of a node is summed by a warp instead of a thread
// (scale-free graphs have hubs whose neighbour lists a single thread would walk for
// milliseconds).
constexpr int kHeavyDegree = 32;
// Target nodes per thread of the exact all-pairs kernel (a CTA owns this many times its
// thread count); the host sizes the source chunks by the resulting CTA count.
constexpr int kExactTargets = 2;

struct NodeLaunch {
    int n;
    int k;                 // interpolation nodes per box and axis
    int gamma_int;         // 2, 4, 8 for the fast exact kernel, else 0
    float2* xy[2];         // ping-pong positions; iteration t reads xy[t & 1]
    const int* rowptr;     // n + 1
    const int* col;        // 2m
    // local refinement (per-node weights, caller order); nullptr: every weight is 1
    const float* wrep;     // n, repulsion weight r_i (pair force scaled by r_i r_j)
    const float* watt;     // n, attraction weight a_i (edge force scaled by a_i a_j)
    float* vwr;            // n, r_i in the cell-sorted order (written by the sort) or nullptr
    // nodes of degree > kHeavyDegree, whose attraction one warp sums (the others: a thread)
    const int* heavy;
    int n_heavy;
    DevState* st;
    const DevParams* prm;
    // FFT path
    int nbox_max;          // (G_max / k)^2
    int* cnt;              // nbox_max (zero between iterations)
    int* off;              // nbox_max + 1
    int* bsum;             // scan block sums
    unsigned long long* scan_status;  // one status word per scan tile
    int2* keyslot;         // n, (box, slot in box) per visit slot
    // Visit orders: iteration t visits nodes in order vperm[t & 1] (the cell-sorted order
    // of iteration t - 1) with positions vxy[t & 1]; its sort writes the new order into
    // vperm[t & 1 ^ 1] / vxy[t & 1 ^ 1] (old positions, which the update then overwrites
    // with the new ones).
    int* vperm[2];         // n each
    float2* vxy[2];        // n each
    float* gin;            // spread output
    int Gs;
    const float4* gout;    // grid output
    // exact path
    float2* part;          // [nchunks][n] partial repulsion
    int nchunks;
    // force evaluation outputs (caller order)
    float2* frep_out;
    float2* fatt_out;
};

// Positions -> bbox slot `slot` of the state (min / max over both coordinates).
cudaError_t launch_bbox(const NodeLaunch& a, int slot, cudaStream_t s);
// Visit order `slot` := caller order (identity permutation, positions xy[slot]).
cudaError_t launch_order_reset(const NodeLaunch& a, int slot, cudaStream_t s);
cudaError_t launch_order_refresh(const NodeLaunch& a, int slot, cudaStream_t s);
// FFT path, first kernel of an iteration: grid policy, t_cur = iter, step, spectrum key.
cudaError_t launch_fft_grid(const NodeLaunch& a, int advance, cudaStream_t s);
// FFT path, before the grid interaction: bin + scan + scatter (3 kernels), spread (1).
cudaError_t launch_fft_sort(const NodeLaunch& a, cudaStream_t s);
cudaError_t launch_fft_spread(const NodeLaunch& a, cudaStream_t s);
// FFT path: attraction into fatt_out (caller order; independent of the grid, 1 kernel).
cudaError_t launch_attract(const NodeLaunch& a, cudaStream_t s);
// FFT path, after the grid interaction and launch_attract: gather + update (eval = 0;
// advance != 0 moves the iteration counter on) or gather into frep_out (eval = 1).
cudaError_t launch_fft_back(const NodeLaunch& a, int advance, int eval, cudaStream_t s);
// Exact path: all-pairs repulsion (1 kernel), then attraction + update (eval = 0)
// or outputs (eval = 1) (1 kernel).
cudaError_t launch_exact_pairs(const NodeLaunch& a, int advance, cudaStream_t s);
cudaError_t launch_edge_update(const NodeLaunch& a, int advance, int eval, cudaStream_t s);
int scan_items_per_block();

}  // namespace tfdp
