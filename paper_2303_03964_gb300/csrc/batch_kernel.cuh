// batch_kernel.cuh -- the kernels of a batch of graphs (per-phase and persistent) and the
// data they read. The kernels are instantiated per k in batch_k1.cu, batch_k2.cu and
// batch_k3.cu (which nvcc compiles in parallel); batch.cu holds the host side.
//
// An iteration is nine phases (grid policy; binning + attraction; per-graph scan;
// scatter; spread; row / column / inverse-row FFT stages; back-projection + update), each
// distributing (graph, item) work over CTAs. Two launch shapes run them: one cooperative
// persistent launch for `iters` iterations with a grid-wide barrier between phases, or
// nine ordinary launches per iteration, one CTA per item (the launch-shape autotuner
// keeps the faster). The per-node and per-transform arithmetic is the single-graph code
// (node_dev.cuh, fft_stages.cuh), so every graph evolves as it would alone.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "fft_stages.cuh"
#include "launch.h"
#include "node_dev.cuh"

namespace tfdp {
namespace bk {

namespace cg = cooperative_groups;

constexpr int kBThreads = 256;   // threads per CTA in every phase
constexpr int kBChunk = 256;     // boxes per work item (a thread each)
constexpr int kBNodesPerThread = 2;                      // nodes per thread in the node phases
constexpr int kBNodeChunk = kBThreads * kBNodesPerThread;  // nodes per work item

// Per-graph geometry and buffers (device copy).
struct BGraph {
    int n, node_off, rowptr_off, col_off;
    int G_max, Gs, ystride, nbox_max;
    int* cnt;
    int* off;
    float* gin;
    float2* T1;
    float2* T2;
    float4* gout;
    float2* S1;
    float* specK;
    float* specHx;
    float* specHy;
};

struct BatchArgs {
    int B;
    const BGraph* graphs;
    DevState* st;           // [B]
    const DevParams* prm;   // [B]
    float2* xy[2];          // packed caller-order positions (global node index)
    float2* vxy[2];         // packed visit orders (see launch.h NodeLaunch)
    int* vperm[2];          // global node ids
    int2* keyslot;
    float2* fatt;
    float2* frep;
    const int* rowptr;      // per graph n + 1 entries (local offsets into its col range)
    const int* col;         // global node ids
    const float2* tw;
    const int* pre_nodes;   // [B + 1] prefix of node chunks
    const int* pre_boxes;   // [B + 1] prefix of box chunks (nbox_max)
    const int* pre_rows;    // [B + 1] prefix of row blocks (data + spectrum)
    const int* pre_cols;    // [B + 1] prefix of column blocks
    int iters;
    int advance;
    int eval;
};

// graph owning global item `it` of a phase with prefix table pre[0..B]
__device__ __forceinline__ int owner(const int* __restrict__ pre, int B, int it) {
    int lo = 0, hi = B;  // pre[lo] <= it < pre[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(pre + mid) <= it) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------- phase bodies
// Each phase of an iteration as the work of one CTA on one item, shared by the persistent
// kernel (which walks the items of a phase with a grid-wide barrier after it) and by the
// per-phase kernels (one launch per phase, one CTA per item).

// phase 0: grid policy, step and spectrum key of graph g (one thread)
__device__ __forceinline__ void ph_grid(const BatchArgs& a, int g) { grid_decide(a.st + g, a.prm[g], a.advance); }

// phase 1: binning (visit order) and attraction (caller order) of node chunk `item`, two
// nodes per thread (slots base and base + kBThreads, both position loads in flight)
__device__ __forceinline__ void ph_bin(const BatchArgs& a, int item, int lane) {
    const int g = owner(a.pre_nodes, a.B, item);
    const BGraph G = a.graphs[g];
    const DevState* st = a.st + g;
    const int cur = (int)(st->t_cur & 1);
    const int base = (item - __ldg(a.pre_nodes + g)) * kBNodeChunk + threadIdx.x;
    const float lo = st->grid.lo_f, h = st->grid.h_f;
    const int n_int = st->grid.n_int;
    float2 p[kBNodesPerThread];
#pragma unroll
    for (int u = 0; u < kBNodesPerThread; ++u) {
        const int v = base + u * kBThreads;
        p[u] = (v < G.n) ? a.vxy[cur][G.node_off + v] : make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int u = 0; u < kBNodesPerThread; ++u) {
        const int v = base + u * kBThreads;
        if (v < G.n) {
            float tq;
            const int key = box_of(p[u].y, lo, h, n_int, &tq) * n_int + box_of(p[u].x, lo, h, n_int, &tq);
            const unsigned active = __activemask();
            const unsigned same = __match_any_sync(active, key);
            const int leader = __ffs(same) - 1;
            int b = 0;
            if (lane == leader) b = atomicAdd(G.cnt + key, __popc(same));
            b = __shfl_sync(same, b, leader);
            a.keyslot[G.node_off + v] = make_int2(key, b + __popc(same & ((1u << lane) - 1u)));
        }
    }
    // attraction of caller-order nodes (rowptr holds local offsets): a thread per node,
    // and the whole warp for a node of degree above kHeavyDegree, with the single-graph
    // kernel's two functions (so every node gets its solo-run sum)
    const int* rp = a.rowptr + G.rowptr_off;
    const int* cl = a.col + G.col_off;
    const float alpha = (float)a.prm[g].alpha, beta = (float)a.prm[g].beta;
#pragma unroll
    for (int u = 0; u < kBNodesPerThread; ++u) {
        const int v = base + u * kBThreads;
        const bool mine = v < G.n;
        const int gv = G.node_off + (mine ? v : 0);
        const float2 pi = a.xy[cur][gv];
        const bool heavy = mine && rp[v + 1] - rp[v] > kHeavyDegree;
        if (mine && !heavy) a.fatt[gv] = attraction(v, pi, rp, cl, a.xy[cur], alpha, beta, nullptr);
        for (unsigned hm = __ballot_sync(0xffffffffu, heavy); hm; hm &= hm - 1) {
            const int src = __ffs(hm) - 1;
            const int hv = __shfl_sync(0xffffffffu, v, src);
            const float2 hp = make_float2(__shfl_sync(0xffffffffu, pi.x, src), __shfl_sync(0xffffffffu, pi.y, src));
            const float2 f = attraction_warp<false>(hv, hp, rp, cl, a.xy[cur], alpha, beta, nullptr, lane);
            if (lane == src) a.fatt[gv] = f;
        }
    }
}

// phase 2: exclusive scan of the box counts of graph g (one CTA), counts cleared
__device__ __forceinline__ void ph_scan(const BatchArgs& a, int g, int lane) {
    const BGraph G = a.graphs[g];
    const int nbox = a.st[g].grid.n_int * a.st[g].grid.n_int;
    __shared__ int s_w[32];
    __shared__ int s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < nbox; c0 += kBThreads * 8) {
        const int i0 = c0 + threadIdx.x * 8;
        int v[8], tsum = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            v[q] = (i0 + q < nbox) ? G.cnt[i0 + q] : 0;
            tsum += v[q];
        }
        int incl = tsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int w = threadIdx.x >> 5;
        if (lane == 31) s_w[w] = incl;
        __syncthreads();
        if (w == 0) {
            const int x = lane < (kBThreads >> 5) ? s_w[lane] : 0;
            int xi = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, xi, o);
                if (lane >= o) xi += y;
            }
            if (lane < (kBThreads >> 5)) s_w[lane] = xi - x;
        }
        __syncthreads();
        int run = s_carry + s_w[w] + incl - tsum;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (i0 + q < nbox) {
                G.off[i0 + q] = run;
                G.cnt[i0 + q] = 0;
            }
            run += v[q];
        }
        __syncthreads();
        if (threadIdx.x == kBThreads - 1) s_carry = run;
        __syncthreads();
    }
    if (threadIdx.x == 0) G.off[nbox] = G.n;
    __syncthreads();
}

// phase 3: scatter of node chunk `item` into the new cell-sorted order (two nodes per
// thread, their dependent loads in flight together)
__device__ __forceinline__ void ph_scatter(const BatchArgs& a, int item) {
    const int g = owner(a.pre_nodes, a.B, item);
    const BGraph G = a.graphs[g];
    DevState* st = a.st + g;
    const int cur = (int)(st->t_cur & 1);
    const int base = (item - __ldg(a.pre_nodes + g)) * kBNodeChunk + threadIdx.x;
    int2 ks[kBNodesPerThread];
    int ii[kBNodesPerThread];
    float2 pp[kBNodesPerThread];
#pragma unroll
    for (int u = 0; u < kBNodesPerThread; ++u) {
        const int v = base + u * kBThreads;
        const int gv = G.node_off + (v < G.n ? v : 0);
        ks[u] = a.keyslot[gv];
        ii[u] = a.vperm[cur][gv];
        pp[u] = a.vxy[cur][gv];
    }
#pragma unroll
    for (int u = 0; u < kBNodesPerThread; ++u) {
        const int v = base + u * kBThreads;
        if (v >= G.n) continue;
        const int pos = G.off[ks[u].x] + ks[u].y;
        const int i = ii[u];
        if ((unsigned)pos >= (unsigned)G.n || i < G.node_off || i >= G.node_off + G.n) {
            atomicOr(&st->flags, FLAG_SORT_RANGE);
        } else {
            a.vxy[cur ^ 1][G.node_off + pos] = pp[u];
            a.vperm[cur ^ 1][G.node_off + pos] = i;
        }
    }
}

// phase 4: spread of box chunk `item`, one thread per box
template <int K>
__device__ __forceinline__ void ph_spread(const BatchArgs& a, int item) {
    const int g = owner(a.pre_boxes, a.B, item);
    const BGraph G = a.graphs[g];
    const DevState* st = a.st + g;
    const GridDesc gd = st->grid;
    const int b = (item - __ldg(a.pre_boxes + g)) * kBChunk + threadIdx.x;
    if (b < gd.n_int * gd.n_int) {
        const int by = b / gd.n_int;
        const int bx = b - by * gd.n_int;
        const float2* sxy = a.vxy[(int)(st->t_cur & 1) ^ 1] + G.node_off;
        spread_box<K>(sxy, nullptr, max(G.off[b], 0), min(G.off[b + 1], G.n), bx, by, axis_geom(gd), G.gin, G.Gs);
    }
}

// phase 5: forward row transforms of row-block item `item` (kernel-sample rows on a rebuild)
template <int LOGP>
__device__ __forceinline__ void ph_rows_fwd(const BatchArgs& a, int item, float2* sm) {
    using Rg = RegGeom<LOGP>;
    const int g = owner(a.pre_rows, a.B, item);
    const BGraph G = a.graphs[g];
    const DevState* st = a.st + g;
    const int blk = item - __ldg(a.pre_rows + g);
    const int data_blocks = (G.G_max + 2 * Rg::RG - 1) / (2 * Rg::RG);
    if (blk < data_blocks) {
        GridSource gs;
        gs.gin = G.gin;
        gs.Gs = G.Gs;
        rows_fwd_body<LOGP>(gs, st->grid.G, blk, G.T1, G.ystride, a.tw, sm);
    } else if (st->spec_dirty) {
        KernelSource ks;
        ks.P = 1 << LOGP;
        ks.bind(st, a.prm + g);
        rows_fwd_body<LOGP>(ks, ks.P, blk - data_blocks, G.S1, 1 << LOGP, a.tw, sm);
    }
}

// phase 6: column transforms and spectral product of column-block item `item`
template <int LOGP>
__device__ __forceinline__ void ph_cols(const BatchArgs& a, int item, float2* sm) {
    const int g = owner(a.pre_cols, a.B, item);
    const BGraph G = a.graphs[g];
    const DevState* st = a.st + g;
    cols_body<LOGP>(item - __ldg(a.pre_cols + g), G.T1, G.T2, G.ystride, G.specK, G.specHx, G.specHy, G.S1, a.tw,
                    st->grid.G, st->spec_dirty, sm);
}

// phase 7: inverse row transforms of row-block item `item` into (A, O^x, O^y)
template <int LOGP>
__device__ __forceinline__ void ph_rows_inv(const BatchArgs& a, int item, float2* sm) {
    using Rg = RegGeom<LOGP>;
    const int g = owner(a.pre_rows, a.B, item);
    const BGraph G = a.graphs[g];
    const int blk = item - __ldg(a.pre_rows + g);
    const int data_blocks = (G.G_max + 2 * Rg::RG - 1) / (2 * Rg::RG);
    if (blk < data_blocks) rows_inv_body<LOGP>(blk, G.T2, G.ystride, G.gout, G.Gs, a.tw, a.st[g].grid.G, sm);
}

// phase 8: back-projection + update of node chunk `item` in sorted order, with the
// chunk's bbox and force sums reduced in the CTA (every chunk lies inside one graph)
template <int K>
__device__ __forceinline__ void ph_gather(const BatchArgs& a, int item, int lane) {
    const int g = owner(a.pre_nodes, a.B, item);
    const BGraph G = a.graphs[g];
    DevState* st = a.st + g;
    const int cur = (int)(st->t_cur & 1);
    const int nxt = cur ^ 1;
    const int chunk = item - __ldg(a.pre_nodes + g);
    const int base = chunk * kBNodeChunk + threadIdx.x;
    const AxisGeom ag = axis_geom(st->grid);
    const float step = (float)st->step_cur;
    float mn = INFINITY, mx = -INFINITY, sfx = 0.0f, sfy = 0.0f;
    unsigned bad = 0;
    float2 p[kBNodesPerThread];
    int ii[kBNodesPerThread];
#pragma unroll
    for (int u = 0; u < kBNodesPerThread; ++u) {
        const int s = base + u * kBThreads;
        const int gs = G.node_off + (s < G.n ? s : 0);
        p[u] = a.vxy[nxt][gs];
        ii[u] = a.vperm[nxt][gs];
    }
#pragma unroll
    for (int u = 0; u < kBNodesPerThread; ++u) {
        const int s = base + u * kBThreads;
        const int i = ii[u];
        if (s >= G.n || i < G.node_off || i >= G.node_off + G.n) continue;
        const float2 fr = gather_frep<K>(p[u], ag, G.gout, G.Gs);
        sfx += fr.x;
        sfy += fr.y;
        if (a.eval) {
            a.frep[i] = fr;
        } else {
            const float2 fa = a.fatt[i];
            const float2 q = capped_step(p[u], make_float2(fr.x + fa.x, fr.y + fa.y), step);
            if (!(isfinite(q.x) && isfinite(q.y))) bad = 1;
            a.xy[nxt][i] = q;
            a.vxy[nxt][G.node_off + s] = q;
            mn = fminf(mn, fminf(q.x, q.y));
            mx = fmaxf(mx, fmaxf(q.x, q.y));
        }
    }
    if (bad) atomicOr(&st->flags, FLAG_NONFINITE);
    __shared__ float s_mn[kBThreads / 32], s_mx[kBThreads / 32], s_fx[kBThreads / 32], s_fy[kBThreads / 32];
    mn = warp_min(mn);
    mx = warp_max(mx);
    sfx = warp_sumf(sfx);
    sfy = warp_sumf(sfy);
    const int w = threadIdx.x >> 5;
    if (lane == 0) {
        s_mn[w] = mn;
        s_mx[w] = mx;
        s_fx[w] = sfx;
        s_fy[w] = sfy;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double fx = 0.0, fy = 0.0;
        for (int q = 0; q < kBThreads / 32; ++q) {
            mn = fminf(mn, s_mn[q]);
            mx = fmaxf(mx, s_mx[q]);
            fx += s_fx[q];
            fy += s_fy[q];
        }
        if (!a.eval && mn <= mx) {
            atomicMin(&st->bbox[nxt][0], f2ord(mn));
            atomicMax(&st->bbox[nxt][1], f2ord(mx));
        }
        atomicAdd(&st->net_frep[0], fx);
        atomicAdd(&st->net_frep[1], fy);
        if (chunk == 0 && !a.eval && a.advance) st->iter = st->t_cur + 1;
    }
    __syncthreads();
}

// ---------------------------------------------------------------- persistent kernel
// All `iters` iterations in one cooperative launch: every CTA walks the items of a phase,
// then a grid-wide barrier.
template <int LOGP, int K>
__global__ void __launch_bounds__(kBThreads, 2) k_batch(BatchArgs a) {
    extern __shared__ float2 sm[];
    cg::grid_group grid = cg::this_grid();
    const int lane = threadIdx.x & 31;
    const int n_node_items = __ldg(a.pre_nodes + a.B);
    const int n_box_items = __ldg(a.pre_boxes + a.B);
    const int n_row_items = __ldg(a.pre_rows + a.B);
    const int n_col_items = __ldg(a.pre_cols + a.B);
    for (int it = 0; it < a.iters; ++it) {
        for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.B; g += gridDim.x * blockDim.x) ph_grid(a, g);
        grid.sync();
        for (int item = blockIdx.x; item < n_node_items; item += gridDim.x) ph_bin(a, item, lane);
        grid.sync();
        for (int g = blockIdx.x; g < a.B; g += gridDim.x) ph_scan(a, g, lane);
        grid.sync();
        for (int item = blockIdx.x; item < n_node_items; item += gridDim.x) ph_scatter(a, item);
        grid.sync();
        for (int item = blockIdx.x; item < n_box_items; item += gridDim.x) ph_spread<K>(a, item);
        grid.sync();
        for (int item = blockIdx.x; item < n_row_items; item += gridDim.x) {
            ph_rows_fwd<LOGP>(a, item, sm);
            __syncthreads();
        }
        grid.sync();
        for (int item = blockIdx.x; item < n_col_items; item += gridDim.x) {
            ph_cols<LOGP>(a, item, sm);
            __syncthreads();
        }
        grid.sync();
        for (int item = blockIdx.x; item < n_row_items; item += gridDim.x) {
            ph_rows_inv<LOGP>(a, item, sm);
            __syncthreads();
        }
        grid.sync();
        for (int item = blockIdx.x; item < n_node_items; item += gridDim.x) ph_gather<K>(a, item, lane);
        grid.sync();
    }
}

// ---------------------------------------------------------------- per-phase kernels
// The same phases as nine ordinary launches per iteration, one CTA per item, each kernel
// at its own occupancy (the persistent kernel runs every phase at the two CTAs per SM
// that the FFT phases' registers allow). Programmatic dependent launch overlaps each
// kernel's start with its predecessor's tail.
static __global__ void __launch_bounds__(kBThreads) k_bp_grid(BatchArgs a) {
    pdl_wait();
    pdl_trigger();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < a.B) ph_grid(a, g);
}
static __global__ void __launch_bounds__(kBThreads) k_bp_bin(BatchArgs a) {
    pdl_wait();
    pdl_trigger();
    ph_bin(a, blockIdx.x, threadIdx.x & 31);
}
static __global__ void __launch_bounds__(kBThreads) k_bp_scan(BatchArgs a) {
    pdl_wait();
    pdl_trigger();
    ph_scan(a, blockIdx.x, threadIdx.x & 31);
}
static __global__ void __launch_bounds__(kBThreads) k_bp_scatter(BatchArgs a) {
    pdl_wait();
    pdl_trigger();
    ph_scatter(a, blockIdx.x);
}
template <int K>
__global__ void __launch_bounds__(kBThreads, 3) k_bp_spread(BatchArgs a) {
    pdl_wait();
    pdl_trigger();
    ph_spread<K>(a, blockIdx.x);
}
template <int LOGP>
__global__ void __launch_bounds__(kBThreads, 3) k_bp_rows_fwd(BatchArgs a) {
    extern __shared__ float2 sm[];
    pdl_wait();
    pdl_trigger();
    ph_rows_fwd<LOGP>(a, blockIdx.x, sm);
}
template <int LOGP>
__global__ void __launch_bounds__(kBThreads, 3) k_bp_cols(BatchArgs a) {
    extern __shared__ float2 sm[];
    pdl_wait();
    pdl_trigger();
    ph_cols<LOGP>(a, blockIdx.x, sm);
}
template <int LOGP>
__global__ void __launch_bounds__(kBThreads, 3) k_bp_rows_inv(BatchArgs a) {
    extern __shared__ float2 sm[];
    pdl_wait();
    pdl_trigger();
    ph_rows_inv<LOGP>(a, blockIdx.x, sm);
}
template <int K>
__global__ void __launch_bounds__(kBThreads, 4) k_bp_gather(BatchArgs a) {
    pdl_wait();
    pdl_trigger();
    ph_gather<K>(a, blockIdx.x, threadIdx.x & 31);
}

// Item counts of the phases (host copies of the prefix tables' totals).
struct BatchItems {
    int node, box, row, col;
};

template <int LOGP, int K>
cudaError_t batch_phases_attrs_t() {
    cudaError_t e;
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if ((e = cudaFuncSetAttribute(k_bp_rows_fwd<LOGP>, A, (int)RegGeom<LOGP>::rows_smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_bp_cols<LOGP>, A, (int)RegGeom<LOGP>::cols_smem)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_bp_rows_inv<LOGP>, A, (int)RegGeom<LOGP>::rows_smem);
}

// `a.iters` iterations as 9 launches each (stream-ordered; capturable).
template <int LOGP, int K>
cudaError_t batch_phases_t(const BatchArgs& a, const BatchItems& n, cudaStream_t s) {
    using Rg = RegGeom<LOGP>;
    cudaError_t e = cudaSuccess;
    for (int it = 0; it < a.iters && e == cudaSuccess; ++it) {
        e = launch_pdl(k_bp_grid, (a.B + kBThreads - 1) / kBThreads, kBThreads, 0, s, a);
        if (e == cudaSuccess) e = launch_pdl(k_bp_bin, n.node, kBThreads, 0, s, a);
        if (e == cudaSuccess) e = launch_pdl(k_bp_scan, a.B, kBThreads, 0, s, a);
        if (e == cudaSuccess) e = launch_pdl(k_bp_scatter, n.node, kBThreads, 0, s, a);
        if (e == cudaSuccess) e = launch_pdl(k_bp_spread<K>, n.box, kBThreads, 0, s, a);
        if (e == cudaSuccess) e = launch_pdl(k_bp_rows_fwd<LOGP>, n.row, kBThreads, Rg::rows_smem, s, a);
        if (e == cudaSuccess) e = launch_pdl(k_bp_cols<LOGP>, n.col, kBThreads, Rg::cols_smem, s, a);
        if (e == cudaSuccess) e = launch_pdl(k_bp_rows_inv<LOGP>, n.row, kBThreads, Rg::rows_smem, s, a);
        if (e == cudaSuccess) e = launch_pdl(k_bp_gather<K>, n.node, kBThreads, 0, s, a);
    }
    return e;
}

template <int LOGP, int K>
cudaError_t batch_launch_t(const BatchArgs& a, int blocks, cudaStream_t s) {
    const size_t smem = std::max(RegGeom<LOGP>::rows_smem, RegGeom<LOGP>::cols_smem);  // attribute set at creation
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kBThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch<LOGP, K>, a);
}

template <int LOGP, int K>
cudaError_t batch_occupancy_t(int* blocks_per_sm) {
    const size_t smem = std::max(RegGeom<LOGP>::rows_smem, RegGeom<LOGP>::cols_smem);
    cudaError_t e = cudaFuncSetAttribute(k_batch<LOGP, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch<LOGP, K>, kBThreads, smem);
}

// Launch / occupancy of k_batch<logP, K>, and the per-phase launches, for logP in
// [7, 11] (RegGeom<LOGP>::T * CG equals kBThreads for the FFT phases only there),
// defined in batch_k<K>.cu.
template <int K>
cudaError_t batch_launch_k(int logP, const BatchArgs& a, int blocks, cudaStream_t s);
template <int K>
cudaError_t batch_occupancy_k(int logP, int* blocks_per_sm);
template <int K>
cudaError_t batch_phases_k(int logP, const BatchArgs& a, const BatchItems& n, cudaStream_t s);
template <int K>
cudaError_t batch_phases_attrs_k(int logP);

#define TFDP_BATCH_INSTANTIATE(K)                                                             \
    template <>                                                                               \
    cudaError_t batch_launch_k<K>(int logP, const BatchArgs& a, int blocks, cudaStream_t s) { \
        switch (logP) {                                                                       \
            case 7: return batch_launch_t<7, K>(a, blocks, s);                                \
            case 8: return batch_launch_t<8, K>(a, blocks, s);                                \
            case 9: return batch_launch_t<9, K>(a, blocks, s);                                \
            case 10: return batch_launch_t<10, K>(a, blocks, s);                              \
            case 11: return batch_launch_t<11, K>(a, blocks, s);                              \
            default: return cudaErrorInvalidValue;                                            \
        }                                                                                     \
    }                                                                                         \
    template <>                                                                               \
    cudaError_t batch_occupancy_k<K>(int logP, int* blocks_per_sm) {                          \
        switch (logP) {                                                                       \
            case 7: return batch_occupancy_t<7, K>(blocks_per_sm);                            \
            case 8: return batch_occupancy_t<8, K>(blocks_per_sm);                            \
            case 9: return batch_occupancy_t<9, K>(blocks_per_sm);                            \
            case 10: return batch_occupancy_t<10, K>(blocks_per_sm);                          \
            case 11: return batch_occupancy_t<11, K>(blocks_per_sm);                          \
            default: return cudaErrorInvalidValue;                                            \
        }                                                                                     \
    }                                                                                         \
    template <>                                                                               \
    cudaError_t batch_phases_k<K>(int logP, const BatchArgs& a, const BatchItems& n,          \
                                  cudaStream_t s) {                                           \
        switch (logP) {                                                                       \
            case 7: return batch_phases_t<7, K>(a, n, s);                                     \
            case 8: return batch_phases_t<8, K>(a, n, s);                                     \
            case 9: return batch_phases_t<9, K>(a, n, s);                                     \
            case 10: return batch_phases_t<10, K>(a, n, s);                                   \
            case 11: return batch_phases_t<11, K>(a, n, s);                                   \
            default: return cudaErrorInvalidValue;                                            \
        }                                                                                     \
    }                                                                                         \
    template <>                                                                               \
    cudaError_t batch_phases_attrs_k<K>(int logP) {                                           \
        switch (logP) {                                                                       \
            case 7: return batch_phases_attrs_t<7, K>();                                      \
            case 8: return batch_phases_attrs_t<8, K>();                                      \
            case 9: return batch_phases_attrs_t<9, K>();                                      \
            case 10: return batch_phases_attrs_t<10, K>();                                    \
            case 11: return batch_phases_attrs_t<11, K>();                                    \
            default: return cudaErrorInvalidValue;                                            \
        }                                                                                     \
    }

}  // namespace bk
}  // namespace tfdp
