// node_kernels.cu -- per-node stages of one t-FDP iteration (arXiv 2303.03964).
//
//   k_bbox           layout square extremes (Sec. 3.4: [x_min, x_max]^2 over both axes)
//   k_order_reset /  visit order after a position upload: caller order, or the last
//   k_order_refresh  sorted order with the new positions
//   k_grid           grid policy of the iteration (Sec. 3.4 "Choices of k"), one thread
//   k_bin            box of every node (Sec. 3.4: each point is assigned to the grid
//                    square that contains it) and its slot: counting-sort histogram
//   k_scan_lookback  single-pass exclusive scan of the box counts
//   k_scatter        cell-sorted copy of the positions and the permutation
//   k_spread /       Lagrange projection onto the k x k nodes of each box (Sec. 3.4,
//   k_spread_group   step 1): rho, m^x, m^y; one thread (or one lane group) owns a box,
//                    so no atomics
//   k_attract        attraction over the CSR (Eq. newforce), caller order, on a side
//                    stream; a warp per node of degree > kHeavyDegree
//   k_gather_update  back-projection (step 3) + capped step (update), cell-sorted order
//   k_exact          tiled all-pairs repulsion (Eq. repfK), FP32
//   k_edge_update    attraction + capped step for the exact path
//
// Node coordinates relative to their box origin are formed exactly (TwoSum and an
// FMA-exact product), so that FP32 coordinates of magnitude |x| ~ 10^3 keep the
// precision of the in-box offset.
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "launch.h"
#include "node_dev.cuh"

namespace tfdp {

constexpr int kScanThreads = 256;
constexpr int kScanMaxTiles = 1024;  // tile status words the graph allocates
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;
static_assert(kScanItems == 8, "k_scan_lookback moves its items as two int4");
constexpr int kNodeThreads = 256;

int scan_items_per_block() { return kScanChunk; }

// ---------------------------------------------------------------- reductions
struct BlockAcc {
    float mn, mx;
    double fx, fy;
};


// Reduce (min, max, sum fx, sum fy) over the block; thread 0 publishes with atomics.
// The force sums are FP32 within a warp (one node per thread) and FP64 above.
__device__ void block_publish(float mn, float mx, float fx, float fy, DevState* st, int slot, bool bbox) {
    __shared__ float s_mn[32], s_mx[32];
    __shared__ double s_fx[32], s_fy[32];
    BlockAcc v;
    v.mn = warp_min(mn);
    v.mx = warp_max(mx);
    v.fx = (double)warp_sumf(fx);
    v.fy = (double)warp_sumf(fy);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { s_mn[w] = v.mn; s_mx[w] = v.mx; s_fx[w] = v.fx; s_fy[w] = v.fy; }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        v.mn = lane < nw ? s_mn[lane] : INFINITY;
        v.mx = lane < nw ? s_mx[lane] : -INFINITY;
        v.fx = lane < nw ? s_fx[lane] : 0.0;
        v.fy = lane < nw ? s_fy[lane] : 0.0;
        v.mn = warp_min(v.mn);
        v.mx = warp_max(v.mx);
        v.fx = warp_sum(v.fx);
        v.fy = warp_sum(v.fy);
        if (lane == 0) {
            if (bbox && v.mn <= v.mx) {
                atomicMin(&st->bbox[slot][0], f2ord(v.mn));
                atomicMax(&st->bbox[slot][1], f2ord(v.mx));
            }
            atomicAdd(&st->net_frep[0], v.fx);
            atomicAdd(&st->net_frep[1], v.fy);
        }
    }
}

// ---------------------------------------------------------------- bbox
__global__ void __launch_bounds__(kNodeThreads) k_bbox(const float2* __restrict__ xy, int n, DevState* st,
                                                       int slot) {
    BlockAcc v{INFINITY, -INFINITY, 0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float2 p = xy[i];
        v.mn = fminf(v.mn, fminf(p.x, p.y));
        v.mx = fmaxf(v.mx, fmaxf(p.x, p.y));
    }
    v.mn = warp_min(v.mn);
    v.mx = warp_max(v.mx);
    __shared__ float s_mn[32], s_mx[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { s_mn[w] = v.mn; s_mx[w] = v.mx; }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        float mn = lane < nw ? s_mn[lane] : INFINITY, mx = lane < nw ? s_mx[lane] : -INFINITY;
        mn = warp_min(mn);
        mx = warp_max(mx);
        if (lane == 0 && mn <= mx) {
            atomicMin(&st->bbox[slot][0], f2ord(mn));
            atomicMax(&st->bbox[slot][1], f2ord(mx));
        }
    }
}

// ---------------------------------------------------------------- FFT path: grid
// One thread: the grid of this iteration from the layout extremes (exact FP64
// decisions), the step s_t, the spectrum key, and the bookkeeping of the iteration.
// The first thread of a second warp fetches s_t from the step table while thread 0
// decides the grid: in another warp the table's dependent loads run beside the FP64 work
// instead of taking turns with it as a divergent branch of the same warp.
__global__ void k_grid(NodeLaunch a, int advance) {
    pdl_wait();
    pdl_trigger();
    if (threadIdx.x == 32) {
        a.st->step_cur = step_size(a.st->iter, *a.prm);
        return;
    }
    if (threadIdx.x != 0) return;
    const DevParams prm = *a.prm;
    grid_decide(a.st, prm, advance, false);
}

// Box of every node (the FP32 decision) and its slot in the box (counting-sort
// histogram), visiting nodes in the previous iteration's cell-sorted order: neighbouring
// lanes mostly share a box, so one atomic serves all lanes of a warp with that box.
__global__ void __launch_bounds__(kNodeThreads) k_bin(NodeLaunch a) {
    pdl_wait();
    pdl_trigger();
    const DevState* st = a.st;
    const int cur = (int)(st->t_cur & 1);
    const float2* __restrict__ vxy = a.vxy[cur];
    const float lo = st->grid.lo_f, h = st->grid.h_f;
    const int n_int = st->grid.n_int;
    const int lane = threadIdx.x & 31;
    // two visit slots per thread per round (base and base + blockDim): both position
    // loads are in flight together; each round's lanes still cover consecutive slots
    const int stride = 2 * gridDim.x * blockDim.x;
    for (int base = 2 * blockIdx.x * blockDim.x + threadIdx.x; base < a.n; base += stride) {
        const int v1 = base + (int)blockDim.x;
        const bool has1 = v1 < a.n;
        const float2 p0 = vxy[base];
        const float2 p1 = has1 ? vxy[v1] : p0;
        float tq;
        const int key0 = box_of(p0.y, lo, h, n_int, &tq) * n_int + box_of(p0.x, lo, h, n_int, &tq);
        const int key1 = box_of(p1.y, lo, h, n_int, &tq) * n_int + box_of(p1.x, lo, h, n_int, &tq);
        const unsigned active = __activemask();
        {
            const unsigned same = __match_any_sync(active, key0);
            const int leader = __ffs(same) - 1;
            int b = 0;
            if (lane == leader) b = atomicAdd(a.cnt + key0, __popc(same));
            b = __shfl_sync(same, b, leader);
            a.keyslot[base] = make_int2(key0, b + __popc(same & ((1u << lane) - 1u)));
        }
        const unsigned act1 = __ballot_sync(active, has1);
        if (has1) {
            const unsigned same = __match_any_sync(act1, key1);
            const int leader = __ffs(same) - 1;
            int b = 0;
            if (lane == leader) b = atomicAdd(a.cnt + key1, __popc(same));
            b = __shfl_sync(same, b, leader);
            a.keyslot[v1] = make_int2(key1, b + __popc(same & ((1u << lane) - 1u)));
        }
    }
}

// Visit order `slot` := identity (node v at slot v) with the caller-order positions.
__global__ void __launch_bounds__(kNodeThreads) k_order_reset(NodeLaunch a, int slot) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += gridDim.x * blockDim.x) {
        a.vperm[slot][v] = v;
        a.vxy[slot][v] = a.xy[slot][v];
    }
}

// Keep visit order `slot` (a permutation left by an earlier sort) and refresh its
// positions from the caller-order ones: positions uploaded close to the previous ones
// keep the next sort coherent.
__global__ void __launch_bounds__(kNodeThreads) k_order_refresh(NodeLaunch a, int slot) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += gridDim.x * blockDim.x) {
        const int i = a.vperm[slot][v];
        a.vxy[slot][v] = ((unsigned)i < (unsigned)a.n) ? a.xy[slot][i] : make_float2(0.0f, 0.0f);
    }
}

// ---------------------------------------------------------------- FFT path: scan
// Single-pass exclusive scan of the box counts with decoupled look-back. Each CTA takes
// a ticket; ticket order is launch order, so a CTA only waits for CTAs that are already
// running. Tile status words (flag | epoch | value) carry the launch epoch, so stale
// words of earlier launches read as "not ready" and nothing needs clearing. Waits are
// bounded: on timeout the CTA sets FLAG_WAIT_TIMEOUT and carries on with what it has
// (offsets then fail the scatter's range check instead of faulting).
constexpr unsigned long long kStAggregate = 1ULL << 62;
constexpr unsigned long long kStPrefix = 2ULL << 62;
constexpr int kLookbackSpinLimit = 1 << 20;

__global__ void __launch_bounds__(kScanThreads) k_scan_lookback(NodeLaunch a, int ntiles,
                                                                 unsigned long long* __restrict__ status) {
    pdl_wait();
    pdl_trigger();
    __shared__ unsigned long long s_ticket;
    __shared__ int s_w[32];
    __shared__ int s_prefix;
    DevState* st = a.st;
    if (threadIdx.x == 0) s_ticket = atomicAdd(&st->scan_ticket, 1ULL);
    __syncthreads();
    const unsigned long long tk = s_ticket;
    const int spin_limit = a.prm->scan_spin_limit > 0 ? a.prm->scan_spin_limit : kLookbackSpinLimit;
    const bool stall = a.prm->scan_stall != 0;
    const int tile = (int)(tk % (unsigned long long)ntiles);
    const unsigned long long epoch = (tk / (unsigned long long)ntiles) & 0x3FFFFFFFULL;
    const int n_int = st->grid.n_int;
    const int nbox = n_int * n_int;
    const int i0 = tile * kScanChunk + threadIdx.x * kScanItems;
    int v[kScanItems];
    const int4* src = reinterpret_cast<const int4*>(a.cnt + i0);
    const int4 c0 = src[0], c1 = src[1];
    v[0] = c0.x; v[1] = c0.y; v[2] = c0.z; v[3] = c0.w;
    v[4] = c1.x; v[5] = c1.y; v[6] = c1.z; v[7] = c1.w;
    int tsum = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        if (i0 + q >= nbox) v[q] = 0;
        tsum += v[q];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_w[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int x = lane < kScanThreads / 32 ? s_w[lane] : 0;
        int xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += y;
        }
        s_w[lane] = xi - x;  // exclusive prefix of warp totals
        const int total = __shfl_sync(0xffffffffu, xi, 31);
        const unsigned long long tag = epoch << 32;
        volatile unsigned long long* vs = status;
        int prefix = 0;
        if (tile == 0) {
            if (lane == 0 && !stall) vs[0] = kStPrefix | tag | (unsigned)total;
        } else {
            if (lane == 0) {
                vs[tile] = kStAggregate | tag | (unsigned)total;
                __threadfence();
            }
            __syncwarp();
            // warp-parallel look-back: lane l inspects tile (end - 1 - l) of a window of 32
            int end = tile;
            int spins = 0;
            bool done = false;
            while (!done) {
                const int p = end - 1 - lane;
                unsigned long long sw = 0;
                bool ready = true;
                if (p >= 0) {
                    sw = vs[p];
                    ready = ((sw >> 32) & 0x3FFFFFFFULL) == epoch && (sw >> 62) != 0;
                }
                if (__all_sync(0xffffffffu, ready) == 0) {
                    if (++spins > spin_limit) {
                        if (lane == 0) atomicOr(&st->flags, FLAG_WAIT_TIMEOUT);
                        break;
                    }
                    continue;
                }
                // nearest lane holding an inclusive prefix; sum the values up to it
                const bool is_prefix = (p >= 0) && ((sw >> 62) == (kStPrefix >> 62));
                const unsigned pm = __ballot_sync(0xffffffffu, is_prefix);
                const int first = pm ? (__ffs(pm) - 1) : 31;
                int val = (p >= 0 && lane <= first) ? (int)(unsigned)(sw & 0xFFFFFFFFULL) : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
                prefix += val;
                if (pm || end - 32 <= 0) done = true;
                end -= 32;
            }
            if (lane == 0) {
                __threadfence();
                vs[tile] = kStPrefix | tag | (unsigned)(prefix + total);
            }
        }
        if (lane == 0) s_prefix = prefix;
    }
    __syncthreads();
    int run = s_prefix + s_w[w] + incl - tsum;
    int o[kScanItems];
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        o[q] = run;
        run += v[q];
    }
    // cnt holds ntiles * kScanChunk counters (zero past nbox), off is 256-byte aligned and
    // i0 a multiple of 8: full rows go out as two 16-byte stores
    int4* cz = reinterpret_cast<int4*>(a.cnt + i0);
    cz[0] = make_int4(0, 0, 0, 0);  // ready for the next histogram
    cz[1] = make_int4(0, 0, 0, 0);
    if (i0 + kScanItems <= nbox) {
        int4* od = reinterpret_cast<int4*>(a.off + i0);
        od[0] = make_int4(o[0], o[1], o[2], o[3]);
        od[1] = make_int4(o[4], o[5], o[6], o[7]);
    } else {
#pragma unroll
        for (int q = 0; q < kScanItems; ++q)
            if (i0 + q < nbox) a.off[i0 + q] = o[q];
    }
    // off[nbox] = n, written by the thread whose items end at or contain nbox
    if (i0 <= nbox && (nbox < i0 + kScanItems || (nbox == i0 + kScanItems && i0 + kScanItems == ntiles * kScanChunk)))
        a.off[nbox] = a.n;
}

// ---------------------------------------------------------------- FFT path: scatter
__global__ void __launch_bounds__(kNodeThreads) k_scatter(NodeLaunch a) {
    pdl_wait();
    pdl_trigger();
    const int cur = (int)(a.st->t_cur & 1);
    const int* __restrict__ vperm = a.vperm[cur];
    const float2* __restrict__ vxy = a.vxy[cur];
    int* __restrict__ nperm = a.vperm[cur ^ 1];
    float2* __restrict__ nxy = a.vxy[cur ^ 1];
    // two visit slots per thread per round so that the dependent loads (slot -> box
    // offset) of both are in flight together
    const int stride = 2 * gridDim.x * blockDim.x;
    for (int base = 2 * blockIdx.x * blockDim.x + threadIdx.x; base < a.n; base += stride) {
        const int vv[2] = {base, base + (int)blockDim.x};
        int2 ks[2];
        int ii[2];
        float2 pp[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int v = vv[u] < a.n ? vv[u] : base;
            ks[u] = a.keyslot[v];
            ii[u] = vperm[v];
            pp[u] = vxy[v];
        }
        int pos[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) pos[u] = a.off[ks[u].x] + ks[u].y;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (vv[u] >= a.n) continue;
            if ((unsigned)pos[u] >= (unsigned)a.n || (unsigned)ii[u] >= (unsigned)a.n) {
                atomicOr(&a.st->flags, FLAG_SORT_RANGE);
                continue;
            }
            nxy[pos[u]] = pp[u];
            nperm[pos[u]] = ii[u];
            if (a.vwr) a.vwr[pos[u]] = a.wrep[ii[u]];
        }
    }
}

// ---------------------------------------------------------------- FFT path: spread
// One thread per box: sum over the box's nodes (contiguous after the sort) of the
// Lagrange weights w (rho) and of w times the offset to each grid node (m^x, m^y).
template <int K>
__global__ void __launch_bounds__(kNodeThreads, 3) k_spread(NodeLaunch a) {
    pdl_wait();
    pdl_trigger();
    const GridDesc g = a.st->grid;
    const int nbox = g.n_int * g.n_int;
    const AxisGeom ag = axis_geom(g);
    const float2* __restrict__ sxy = a.vxy[(int)(a.st->t_cur & 1) ^ 1];
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += gridDim.x * blockDim.x) {
        const int by = b / g.n_int;
        const int bx = b - by * g.n_int;
        spread_box<K>(sxy, a.vwr, max(a.off[b], 0), min(a.off[b + 1], a.n), bx, by, ag, a.gin, a.Gs);
    }
}

// L lanes per box (grids with few boxes). blockDim is a multiple of L, so a lane's place
// in its group is fixed across the grid-stride loop and a whole group passes or fails
// the loop test together (same box).
template <int K, int L>
__global__ void __launch_bounds__(kNodeThreads, 3) k_spread_group(NodeLaunch a) {
    pdl_wait();
    pdl_trigger();
    const GridDesc g = a.st->grid;
    const int nbox = g.n_int * g.n_int;
    const AxisGeom ag = axis_geom(g);
    const float2* __restrict__ sxy = a.vxy[(int)(a.st->t_cur & 1) ^ 1];
    const int gl = threadIdx.x & (L - 1);
    const unsigned gmask = ((L == 32) ? 0xffffffffu : ((1u << L) - 1u)) << ((threadIdx.x & 31) & ~(L - 1));
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < L * nbox; q += gridDim.x * blockDim.x) {
        const int b = q / L;
        const int by = b / g.n_int;
        const int bx = b - by * g.n_int;
        spread_box_group<K, L>(sxy, a.vwr, max(a.off[b], 0), min(a.off[b + 1], a.n), bx, by, gl, gmask, ag, a.gin,
                               a.Gs);
    }
}

// ---------------------------------------------------------------- FFT path: attraction
// fatt(i) in caller order (coalesced CSR rows); independent of the grid, so it runs
// on a second stream while the sort, spread and FFT run.
// Blocks [0, heavy_blocks): one warp per node of degree > kHeavyDegree (listed in
// a.heavy), launched first so that the long lists start early. The other blocks: one
// thread per node (two per round), skipping the heavy ones.
template <bool W>
__global__ void __launch_bounds__(kNodeThreads) k_attract(NodeLaunch a, int heavy_blocks) {
    const int cur = (int)(a.st->t_cur & 1);  // set by k_grid, which precedes the fork
    const float2* __restrict__ xin = a.xy[cur];
    const float alpha = (float)a.prm->alpha, beta = (float)a.prm->beta;
    if ((int)blockIdx.x < heavy_blocks) {
        const int w = blockIdx.x * (kNodeThreads / 32) + (threadIdx.x >> 5);
        if (w >= a.n_heavy) return;  // whole warps leave together
        const int i = a.heavy[w];
        const float2 f = attraction_warp<W>(i, xin[i], a.rowptr, a.col, xin, alpha, beta, a.watt, threadIdx.x & 31);
        if ((threadIdx.x & 31) == 0) a.fatt_out[i] = f;
        return;
    }
    const int nb = gridDim.x - heavy_blocks, bx = blockIdx.x - heavy_blocks;
    const int stride = 2 * nb * blockDim.x;
    for (int base = 2 * bx * blockDim.x + threadIdx.x; base < a.n; base += stride) {
        const int ii[2] = {base, base + (int)blockDim.x};
        float2 pp[2], fa[2];
        bool own[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = ii[u] < a.n ? ii[u] : base;
            own[u] = ii[u] < a.n && a.rowptr[i + 1] - a.rowptr[i] <= kHeavyDegree;
            pp[u] = xin[i];
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
            fa[u] = own[u] ? attraction_t<W>(ii[u], pp[u], a.rowptr, a.col, xin, alpha, beta, a.watt)
                           : make_float2(0.0f, 0.0f);
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (own[u]) a.fatt_out[ii[u]] = fa[u];
    }
}

// ---------------------------------------------------------------- FFT path: gather + update
// frep(i) = sum_p w_ip [ (x_i - y_p) A_p + O_p ]  (well-conditioned Eq. Fr1/Fr2), then the
// capped step with fatt(i). Nodes are visited in cell-sorted order, so neighbouring
// threads read the same grid values and the next iteration's visit-order positions are
// written contiguously; caller-order outputs are scattered through perm.
template <int K, bool EVAL>
__global__ void __launch_bounds__(kNodeThreads) k_gather_update(NodeLaunch a, int advance) {
    pdl_wait();
    pdl_trigger();
    DevState* st = a.st;
    const GridDesc g = st->grid;
    const AxisGeom ag = axis_geom(g);
    const int cur = (int)(st->t_cur & 1);
    const int nxt = cur ^ 1;
    float2* __restrict__ sxy = a.vxy[nxt];  // old positions in the new order, then new ones
    const int* __restrict__ perm = a.vperm[nxt];
    float2* __restrict__ xout = a.xy[nxt];
    const float step = (float)st->step_cur;
    float mn = INFINITY, mx = -INFINITY, sfx = 0.0f, sfy = 0.0f;
    unsigned bad = 0;
    // two sorted slots per thread per round (base and base + blockDim) so that the
    // dependent loads of both nodes overlap
    const int stride = 2 * gridDim.x * blockDim.x;
    for (int base = 2 * blockIdx.x * blockDim.x + threadIdx.x; base < a.n; base += stride) {
        const int ss[2] = {base, base + (int)blockDim.x};
        float2 p[2], fa[2];
        int ii[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int s = ss[u] < a.n ? ss[u] : base;
            p[u] = sxy[s];
            ii[u] = perm[s];
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
            fa[u] = ((unsigned)ii[u] < (unsigned)a.n) ? a.fatt_out[ii[u]] : make_float2(0.f, 0.f);
        float2 fr[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) fr[u] = gather_frep<K>(p[u], ag, a.gout, a.Gs);
        if (a.vwr) {  // local refinement: frep(i) = r_i sum_j r_j (...)
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const float r = a.vwr[ss[u] < a.n ? ss[u] : base];
                fr[u].x *= r;
                fr[u].y *= r;
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int s = ss[u], i = ii[u];
            if (s >= a.n || (unsigned)i >= (unsigned)a.n) continue;  // bad ids only after a failed sort
            sfx += fr[u].x;
            sfy += fr[u].y;
            if (EVAL) {
                a.frep_out[i] = fr[u];
            } else {
                const float2 q = capped_step(p[u], make_float2(fr[u].x + fa[u].x, fr[u].y + fa[u].y), step);
                if (!(isfinite(q.x) && isfinite(q.y))) bad = 1;
                xout[i] = q;
                sxy[s] = q;  // next iteration's visit order is this iteration's sorted order
                mn = fminf(mn, fminf(q.x, q.y));
                mx = fmaxf(mx, fmaxf(q.x, q.y));
            }
        }
    }
    if (bad) atomicOr(&st->flags, FLAG_NONFINITE);
    block_publish(mn, mx, sfx, sfy, st, nxt, !EVAL);
    // the last kernel of an iteration advances the counter (the side stream has joined)
    if (!EVAL && advance && blockIdx.x == 0 && threadIdx.x == 0) st->iter = st->t_cur + 1;
}

// ---------------------------------------------------------------- exact path
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// K = (1 + d^2)^-gamma given u = 1 + d^2
template <int GI>
__device__ __forceinline__ float kernel_of(float u, float gamma) {
    if (GI == 0) return ex2_approx(-gamma * lg2_approx(u));
    const float r = rcp_approx(u);
    float k = r;
    if (GI >= 2) k = r * r;
    if (GI >= 4) k = k * k;
    if (GI >= 8) k = k * k;
    return k;
}

// Paired FP32 operations of sm_100-family GPUs on (x, y) pairs held in a 64-bit register:
// each lane rounds exactly like the scalar operation, so a pair op gives the same bits as
// two scalar ones while taking one issue slot.
__device__ __forceinline__ unsigned long long f2_pack(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// One source (qx, qy) with weight wj on target pi2 = (x_i, y_i): (dx, dy) = x_i - x_j,
// K = (1 + d^2)^-gamma (times wj), (fx, fy) += K (dx, dy).
template <int GI, bool W>
__device__ __forceinline__ void exact_pair(unsigned long long pi2, float qx, float qy, float wj, float gamma,
                                           unsigned long long& f2) {
    const unsigned long long d = f2_sub(pi2, f2_pack(qx, qy));
    float dx, dy;
    f2_unpack(d, dx, dy);
    float K = kernel_of<GI>(fmaf(dx, dx, fmaf(dy, dy, 1.0f)), gamma);
    if (W) K *= wj;
    f2 = f2_fma(f2_pack(K, K), d, f2);
}

// Tiled all-pairs repulsion: each CTA owns kExactTargets x kNodeThreads targets (each
// thread kExactTargets of them, kNodeThreads apart) and one chunk of the sources
// (blockIdx.y), staging source tiles in shared memory; every source read from shared
// memory serves all of a thread's targets. Partial sums per chunk go to part[chunk][i];
// k_edge_update adds them in chunk order (deterministic). A full tile is read two sources
// per 16-byte shared load; (dx, dy) and the (fx, fy) sums use the paired operations.
template <int GI, bool W>
__global__ void __launch_bounds__(kNodeThreads) k_exact(NodeLaunch a, int advance) {
    pdl_wait();
    pdl_trigger();
    DevState* st = a.st;
    const long long t = st->iter;
    const int cur = (int)(t & 1);
    const float2* __restrict__ xy = a.xy[cur];
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        st->t_cur = t;
        st->step_cur = step_size(t, *a.prm);
        st->net_frep[0] = 0.0;
        st->net_frep[1] = 0.0;
        if (advance) {
            st->bbox[cur ^ 1][0] = kOrdMinInit;
            st->bbox[cur ^ 1][1] = kOrdMaxInit;
        }
    }
    const float gamma = (float)a.prm->gamma;
    __shared__ __align__(16) float2 tile[kNodeThreads];
    __shared__ __align__(8) float tile_w[W ? kNodeThreads : 2];  // source weights r_j (local refinement)
    int ii[kExactTargets];
    unsigned long long pi2[kExactTargets], f2[kExactTargets];
    float2 pi0 = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < kExactTargets; ++q) {
        ii[q] = blockIdx.x * (kExactTargets * kNodeThreads) + q * kNodeThreads + threadIdx.x;
        const float2 pi = (ii[q] < a.n) ? xy[ii[q]] : make_float2(0.f, 0.f);
        if (q == 0) pi0 = pi;
        pi2[q] = f2_pack(pi.x, pi.y);
        f2[q] = f2_pack(0.0f, 0.0f);
    }
    const int csize = (a.n + a.nchunks - 1) / a.nchunks;
    const int j0 = blockIdx.y * csize;
    const int j1 = min(a.n, j0 + csize);
    for (int s0 = j0; s0 < j1; s0 += kNodeThreads) {
        const int j = s0 + threadIdx.x;
        tile[threadIdx.x] = (j < j1) ? xy[j] : pi0;
        if (W) tile_w[threadIdx.x] = (j < j1) ? a.wrep[j] : 0.0f;
        __syncthreads();
        const int cnt = min(kNodeThreads, j1 - s0);
        if (cnt == kNodeThreads) {
            const float4* t4 = reinterpret_cast<const float4*>(tile);
            const float2* w2 = reinterpret_cast<const float2*>(tile_w);
#pragma unroll 4
            for (int jj = 0; jj < kNodeThreads / 2; ++jj) {
                const float4 q4 = t4[jj];  // sources 2 jj and 2 jj + 1, in that order
                const float2 wq = W ? w2[jj] : make_float2(1.0f, 1.0f);
#pragma unroll
                for (int q = 0; q < kExactTargets; ++q) {
                    exact_pair<GI, W>(pi2[q], q4.x, q4.y, wq.x, gamma, f2[q]);
                    exact_pair<GI, W>(pi2[q], q4.z, q4.w, wq.y, gamma, f2[q]);
                }
            }
        } else {
            for (int jj = 0; jj < cnt; ++jj) {
                const float2 q2 = tile[jj];
#pragma unroll
                for (int q = 0; q < kExactTargets; ++q)
                    exact_pair<GI, W>(pi2[q], q2.x, q2.y, W ? tile_w[jj] : 1.0f, gamma, f2[q]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < kExactTargets; ++q) {
        float fx, fy;
        f2_unpack(f2[q], fx, fy);
        if (ii[q] < a.n) a.part[(size_t)blockIdx.y * a.n + ii[q]] = make_float2(fx, fy);
    }
}

// Attraction + update in caller order, on the repulsion summed over `nchunks` partial
// arrays. Each thread takes two nodes per round so that their dependent loads
// (row pointers, neighbour ids, neighbour positions) overlap.
template <bool EVAL>
__global__ void __launch_bounds__(kNodeThreads) k_edge_update(NodeLaunch a, int advance) {
    pdl_wait();
    pdl_trigger();
    DevState* st = a.st;
    const long long t = st->t_cur;
    const int cur = (int)(t & 1);
    const float2* __restrict__ xin = a.xy[cur];
    float2* __restrict__ xout = a.xy[cur ^ 1];
    const float step = (float)st->step_cur;
    const float alpha = (float)a.prm->alpha, beta = (float)a.prm->beta;
    float mn = INFINITY, mx = -INFINITY, sfx = 0.0f, sfy = 0.0f;
    unsigned bad = 0;
    const int stride = 2 * gridDim.x * blockDim.x;
    for (int base = 2 * blockIdx.x * blockDim.x + threadIdx.x; base < a.n; base += stride) {
        const int ii[2] = {base, base + (int)blockDim.x};
        float2 fr[2], pp[2], fa[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = ii[u] < a.n ? ii[u] : base;
            fr[u] = make_float2(0.0f, 0.0f);
            for (int c = 0; c < a.nchunks; ++c) {
                const float2 v = a.part[(size_t)c * a.n + i];
                fr[u].x += v.x;
                fr[u].y += v.y;
            }
            if (a.wrep) {  // local refinement: frep(i) = r_i sum_j r_j (...)
                fr[u].x *= a.wrep[i];
                fr[u].y *= a.wrep[i];
            }
            pp[u] = xin[i];
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = ii[u] < a.n ? ii[u] : base;
            fa[u] = attraction(i, pp[u], a.rowptr, a.col, xin, alpha, beta, a.watt);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = ii[u];
            if (i >= a.n) continue;
            sfx += fr[u].x;
            sfy += fr[u].y;
            if (EVAL) {
                a.frep_out[i] = fr[u];
                a.fatt_out[i] = fa[u];
            } else {
                const float2 q = capped_step(pp[u], make_float2(fr[u].x + fa[u].x, fr[u].y + fa[u].y), step);
                if (!(isfinite(q.x) && isfinite(q.y))) bad = 1;
                xout[i] = q;
                mn = fminf(mn, fminf(q.x, q.y));
                mx = fmaxf(mx, fmaxf(q.x, q.y));
            }
        }
    }
    if (bad) atomicOr(&st->flags, FLAG_NONFINITE);
    block_publish(mn, mx, sfx, sfy, st, cur ^ 1, !EVAL);
    if (!EVAL && advance && blockIdx.x == 0 && threadIdx.x == 0) st->iter = t + 1;
}

// ---------------------------------------------------------------- launchers
static inline int blocks_for(long long work, int threads) {
    long long b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (1LL << 30)) b = (1LL << 30);
    return (int)b;
}

cudaError_t launch_order_reset(const NodeLaunch& a, int slot, cudaStream_t s) {
    if (a.n == 0 || !a.vperm[slot]) return cudaSuccess;
    k_order_reset<<<blocks_for(a.n, kNodeThreads), kNodeThreads, 0, s>>>(a, slot);
    return cudaGetLastError();
}

cudaError_t launch_order_refresh(const NodeLaunch& a, int slot, cudaStream_t s) {
    if (a.n == 0 || !a.vperm[slot]) return cudaSuccess;
    k_order_refresh<<<blocks_for(a.n, kNodeThreads), kNodeThreads, 0, s>>>(a, slot);
    return cudaGetLastError();
}

cudaError_t launch_bbox(const NodeLaunch& a, int slot, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    int blocks = blocks_for(a.n, kNodeThreads);
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_bbox<<<blocks, kNodeThreads, 0, s>>>(a.xy[slot], a.n, a.st, slot);
    return cudaGetLastError();
}

cudaError_t launch_fft_grid(const NodeLaunch& a, int advance, cudaStream_t s) {
    return launch_pdl(k_grid, 1, 64, 0, s, a, advance);
}

cudaError_t launch_fft_sort(const NodeLaunch& a, cudaStream_t s) {
    const int scan_blocks = blocks_for(a.nbox_max, kScanChunk);
    if (scan_blocks > kScanMaxTiles) return cudaErrorInvalidValue;
    const int nb2 = blocks_for(a.n, 2 * kNodeThreads);  // two visit slots per thread
    cudaError_t e = launch_pdl(k_bin, nb2, kNodeThreads, 0, s, a);
    if (e == cudaSuccess) e = launch_pdl(k_scan_lookback, scan_blocks, kScanThreads, 0, s, a, scan_blocks, a.scan_status);
    if (e == cudaSuccess) e = launch_pdl(k_scatter, nb2, kNodeThreads, 0, s, a);
    return e;
}

// Lanes per box: the smallest power of two (<= 16) that gives half a wave of threads
// (152 SMs x 3 CTAs x 256) over the largest box count; 1 for well-filled grids.
int spread_lanes(int nbox_max) {
    const long long wave = 152LL * 3 * kNodeThreads;
    int L = 1;
    while (L < 16 && 2LL * L * nbox_max < wave) L <<= 1;  // half a wave is enough
    return L;
}

template <int K>
static cudaError_t launch_spread_k(const NodeLaunch& a, cudaStream_t s) {
    const int L = spread_lanes(a.nbox_max);
    const int bb = blocks_for((long long)L * a.nbox_max, kNodeThreads);
    switch (L) {
        case 1: return launch_pdl(k_spread<K>, bb, kNodeThreads, 0, s, a);
        case 2: return launch_pdl(k_spread_group<K, 2>, bb, kNodeThreads, 0, s, a);
        case 4: return launch_pdl(k_spread_group<K, 4>, bb, kNodeThreads, 0, s, a);
        case 8: return launch_pdl(k_spread_group<K, 8>, bb, kNodeThreads, 0, s, a);
        default: return launch_pdl(k_spread_group<K, 16>, bb, kNodeThreads, 0, s, a);
    }
}

cudaError_t launch_fft_spread(const NodeLaunch& a, cudaStream_t s) {
    switch (a.k) {
        case 1: return launch_spread_k<1>(a, s);
        case 2: return launch_spread_k<2>(a, s);
        case 3: return launch_spread_k<3>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_attract(const NodeLaunch& a, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    const int heavy_blocks = (a.n_heavy + kNodeThreads / 32 - 1) / (kNodeThreads / 32);
    const int blocks = heavy_blocks + blocks_for(a.n, 2 * kNodeThreads);
    if (a.watt) k_attract<true><<<blocks, kNodeThreads, 0, s>>>(a, heavy_blocks);
    else k_attract<false><<<blocks, kNodeThreads, 0, s>>>(a, heavy_blocks);
    return cudaGetLastError();
}

cudaError_t launch_fft_back(const NodeLaunch& a, int advance, int eval, cudaStream_t s) {
    const int nb = blocks_for(a.n, 2 * kNodeThreads);
    switch (a.k) {
        case 1: return launch_pdl(eval ? k_gather_update<1, true> : k_gather_update<1, false>, nb, kNodeThreads, 0, s, a, advance);
        case 2: return launch_pdl(eval ? k_gather_update<2, true> : k_gather_update<2, false>, nb, kNodeThreads, 0, s, a, advance);
        case 3: return launch_pdl(eval ? k_gather_update<3, true> : k_gather_update<3, false>, nb, kNodeThreads, 0, s, a, advance);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_exact_pairs(const NodeLaunch& a, int advance, cudaStream_t s) {
    dim3 grid(blocks_for(a.n, kExactTargets * kNodeThreads), a.nchunks);
    switch (a.gamma_int) {
        case 2: return launch_pdl(a.wrep ? k_exact<2, true> : k_exact<2, false>, grid, kNodeThreads, 0, s, a, advance);
        case 4: return launch_pdl(a.wrep ? k_exact<4, true> : k_exact<4, false>, grid, kNodeThreads, 0, s, a, advance);
        case 8: return launch_pdl(a.wrep ? k_exact<8, true> : k_exact<8, false>, grid, kNodeThreads, 0, s, a, advance);
        default: return launch_pdl(a.wrep ? k_exact<0, true> : k_exact<0, false>, grid, kNodeThreads, 0, s, a, advance);
    }
}

cudaError_t launch_edge_update(const NodeLaunch& a, int advance, int eval, cudaStream_t s) {
    const int nb = blocks_for(a.n, 2 * kNodeThreads);
    return launch_pdl(eval ? k_edge_update<true> : k_edge_update<false>, nb, kNodeThreads, 0, s, a, advance);
}

}  // namespace tfdp
