// batch.cu -- many graphs advanced together, by one cooperative persistent kernel or by
// one launch per phase.
//
// A batch holds B independent graphs in packed arenas (positions, CSR, sort buffers)
// with per-graph parameters, state, grids and spectra. An iteration has nine phases
// (grid policy; binning + attraction; per-graph scan; scatter; spread; row / column /
// inverse-row FFT stages; back-projection + update), each distributing (graph, item)
// work over CTAs. An iteration call runs `iters` iterations of every graph either in a
// single cooperative launch, whose CTAs walk the phases with a grid-wide barrier between
// them, or as nine ordinary launches per iteration with one CTA per item, each at its
// own occupancy (captured in a CUDA graph); tfdp_batch_autotune times both. The per-node
// and per-transform arithmetic is the single-graph code (node_dev.cuh, fft_stages.cuh),
// so every graph evolves as it would alone.
//
// A batch is split into parts by (k, FFT size): each part is one such persistent launch
// whose graphs share k and P (P >= 2 G_max - 1 for every graph of the part, so each
// graph's linear convolution is exact), and the parts run one after another on the
// batch's stream. tfdp_batch_plan picks k and the grid cap per graph by measurement, so
// that small graphs run on smaller transforms. The kernel itself is in batch_kernel.cuh.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/tfdp.h"
#include "batch_kernel.cuh"

using namespace tfdp;
using namespace tfdp::bk;

namespace {

// Visit order := caller order for every graph (after a position upload).
__global__ void k_batch_order_reset(int N, const float2* __restrict__ xy, float2* vxy, int* vperm) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
        vperm[v] = v;
        vxy[v] = xy[v];
    }
}

// bbox of each graph into its slot (positions xy, graph of each chunk by prefix table).
__global__ void k_batch_bbox(BatchArgs a, int slot) {
    const int n_node_items = __ldg(a.pre_nodes + a.B);
    for (int item = blockIdx.x; item < n_node_items; item += gridDim.x) {
        const int g = owner(a.pre_nodes, a.B, item);
        const BGraph G = a.graphs[g];
        float mn = INFINITY, mx = -INFINITY;
        for (int u = 0; u < kBNodesPerThread; ++u) {
            const int v = (item - __ldg(a.pre_nodes + g)) * kBNodeChunk + u * kBThreads + threadIdx.x;
            if (v < G.n) {
                const float2 p = a.xy[slot][G.node_off + v];
                mn = fminf(mn, fminf(p.x, p.y));
                mx = fmaxf(mx, fmaxf(p.x, p.y));
            }
        }
        mn = warp_min(mn);
        mx = warp_max(mx);
        if ((threadIdx.x & 31) == 0 && mn <= mx) {
            atomicMin(&a.st[g].bbox[slot][0], f2ord(mn));
            atomicMax(&a.st[g].bbox[slot][1], f2ord(mx));
        }
    }
}

thread_local std::string b_err;

tfdp_status bfail(cudaError_t e, const char* where) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
    b_err = buf;
    return e == cudaErrorMemoryAllocation ? TFDP_ERR_OUT_OF_MEMORY : TFDP_ERR_CUDA;
}

#define BK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return bfail(e_, #call);       \
    } while (0)

size_t up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int log2c(long long v) {
    int l = 0;
    while ((1LL << l) < v) ++l;
    return l;
}

}  // namespace

struct BatchPart {
    int B = 0;
    int64_t N = 0, M = 0;
    int k = 3, logP = 9, P = 512;
    cudaStream_t stream = nullptr;
    std::vector<tfdp_params> params;
    std::vector<int64_t> n, node_off;
    std::vector<BGraph> hg;
    int64_t host_iter = 0;
    void* mem = nullptr;       // node + FFT arena
    BatchArgs args{};
    BGraph* d_graphs = nullptr;
    DevState* d_st = nullptr;
    DevParams* d_prm = nullptr;
    double* d_steps = nullptr;  // per-graph step tables, B x T_max
    int T_max = 0;
    int grid_blocks = 0;       // cooperative grid size
    bool phases = true;        // one launch per phase (false: the cooperative persistent kernel)
    BatchItems items{};        // items of each phase (per-phase launches)
    cudaGraphExec_t exec = nullptr;
    int exec_iters = -1;
    bool no_graph = false;
    std::vector<unsigned> flags_word;  // device flags read back per graph
    std::vector<unsigned> flags_seen;  // every flag reported so far per graph
};

namespace {

// Wait for the batch's stream and report the device flags that graphs [g0, g1) raised
// since the last report (TFDP_ERR_TIMEOUT for a wait that gave up, else
// TFDP_ERR_DEVICE_CHECK); the flags are then cleared on the device and kept per graph
// for the stats call.
tfdp_status batch_sync_checked(BatchPart* b, int g0, int g1) {
    const int cnt = g1 - g0;
    if (cnt > 0) {
        BK(cudaMemcpy2DAsync(b->flags_word.data() + g0, sizeof(unsigned), &b->d_st[g0].flags, sizeof(DevState),
                             sizeof(unsigned), (size_t)cnt, cudaMemcpyDeviceToHost, b->stream));
    }
    BK(cudaStreamSynchronize(b->stream));
    unsigned all = 0;
    for (int q = g0; q < g1; ++q) {
        const unsigned f = b->flags_word[(size_t)q];
        if (!f) continue;
        all |= f;
        b->flags_seen[(size_t)q] |= f;
        BK(cudaMemsetAsync(&b->d_st[q].flags, 0, sizeof(unsigned), b->stream));
    }
    if (!all) return TFDP_OK;
    BK(cudaStreamSynchronize(b->stream));
    return (all & FLAG_WAIT_TIMEOUT) ? TFDP_ERR_TIMEOUT : TFDP_ERR_DEVICE_CHECK;
}

cudaError_t batch_launch(const BatchPart* b, const BatchArgs& a, cudaStream_t s) {
    if (b->phases) {
        switch (b->k) {
            case 1: return batch_phases_k<1>(b->logP, a, b->items, s);
            case 2: return batch_phases_k<2>(b->logP, a, b->items, s);
            case 3: return batch_phases_k<3>(b->logP, a, b->items, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (b->k) {
        case 1: return batch_launch_k<1>(b->logP, a, b->grid_blocks, s);
        case 2: return batch_launch_k<2>(b->logP, a, b->grid_blocks, s);
        case 3: return batch_launch_k<3>(b->logP, a, b->grid_blocks, s);
        default: return cudaErrorInvalidValue;
    }
}
cudaError_t batch_phases_attrs(const BatchPart* b) {
    switch (b->k) {
        case 1: return batch_phases_attrs_k<1>(b->logP);
        case 2: return batch_phases_attrs_k<2>(b->logP);
        case 3: return batch_phases_attrs_k<3>(b->logP);
        default: return cudaErrorInvalidValue;
    }
}
cudaError_t batch_occupancy(const BatchPart* b, int* bps) {
    switch (b->k) {
        case 1: return batch_occupancy_k<1>(b->logP, bps);
        case 2: return batch_occupancy_k<2>(b->logP, bps);
        case 3: return batch_occupancy_k<3>(b->logP, bps);
        default: return cudaErrorInvalidValue;
    }
}

tfdp_status upload_batch_params(BatchPart* b) {
    std::vector<DevParams> dp((size_t)b->B);
    std::vector<double> steps((size_t)b->B * b->T_max, 0.0);
    for (int g = 0; g < b->B; ++g) {
        const tfdp_params& p = b->params[(size_t)g];
        DevParams& d = dp[(size_t)g];
        d.alpha = p.alpha;
        d.beta = p.beta;
        d.gamma = p.gamma;
        d.step0 = p.step0;
        d.step_min = p.step_min;
        d.k = p.k_interp;
        d.n_int_min = p.n_int_min;
        d.grid_max = p.grid_max;
        d.policy = p.grid_policy;
        d.total_iters = p.total_iters;
        d.P = b->P;
        d.log2P = b->logP;
        const double r = std::floor(p.gamma + 0.5);
        d.gamma_int = (p.gamma == r && r >= 2.0 && r <= 8.0) ? (int)r : 0;
        d.spread_shift = 0;  // no local-refinement weights in a batch
        d.step_table = b->d_steps + (size_t)g * b->T_max;
        const int T = p.total_iters;
        for (int t = 0; t < T; ++t)
            steps[(size_t)g * b->T_max + t] =
                (T <= 1) ? p.step0 : p.step0 * std::pow(p.step_min / p.step0, (double)t / (double)(T - 1));
    }
    BK(cudaMemcpyAsync(b->d_prm, dp.data(), sizeof(DevParams) * b->B, cudaMemcpyHostToDevice, b->stream));
    BK(cudaMemcpyAsync(b->d_steps, steps.data(), sizeof(double) * steps.size(), cudaMemcpyHostToDevice, b->stream));
    BK(cudaStreamSynchronize(b->stream));
    return TFDP_OK;
}

tfdp_status batch_refresh(BatchPart* b) {
    const int slot = (int)(b->host_iter & 1);
    for (int g = 0; g < b->B; ++g) {
        const unsigned init[2] = {kOrdMinInit, kOrdMaxInit};
        BK(cudaMemcpyAsync(&b->d_st[g].bbox[slot][0], init, sizeof(init), cudaMemcpyHostToDevice, b->stream));
    }
    BK(cudaStreamSynchronize(b->stream));
    k_batch_bbox<<<1024, kBThreads, 0, b->stream>>>(b->args, slot);
    BK(cudaGetLastError());
    if (b->N > 0) {
        k_batch_order_reset<<<1024, 256, 0, b->stream>>>((int)b->N, b->args.xy[slot], b->args.vxy[slot],
                                                        b->args.vperm[slot]);
        BK(cudaGetLastError());
    }
    return TFDP_OK;
}

}  // namespace

namespace {

tfdp_status part_destroy(BatchPart* b);

tfdp_status part_create(int32_t num_graphs, const int64_t* n, const int64_t* m, const int32_t* const* edges,
                              const float* const* xy0, const tfdp_params* params, void* stream, BatchPart** out) {
    if (!out || num_graphs < 1 || !n || !m || !edges || !xy0) return TFDP_ERR_INVALID_ARG;
    BatchPart* b = new (std::nothrow) BatchPart();
    if (!b) return TFDP_ERR_OUT_OF_MEMORY;
    b->B = num_graphs;
    b->stream = (cudaStream_t)stream;
    b->params.resize((size_t)num_graphs);
    b->flags_word.assign((size_t)num_graphs, 0u);
    b->flags_seen.assign((size_t)num_graphs, 0u);
    int G_need = 0;
    for (int g = 0; g < num_graphs; ++g) {
        tfdp_params p;
        if (params) p = params[g];
        else tfdp_params_default(&p);
        p.rep_mode = TFDP_REP_FFT;
        tfdp_status st = tfdp_params_check(&p, nullptr);
        if (st == TFDP_OK && p.k_interp == TFDP_K_DYNAMIC) st = TFDP_ERR_PARAM_RANGE;  // one fixed k per batch
        if (st == TFDP_OK && p.precision != TFDP_PREC_FP32) st = TFDP_ERR_PARAM_RANGE;  // FP32 kernels only
        if (st != TFDP_OK || (g > 0 && p.k_interp != b->params[0].k_interp) || n[g] < 1 || m[g] < 0 ||
            (m[g] > 0 && !edges[g]) || !xy0[g]) {
            delete b;
            return st != TFDP_OK ? st : TFDP_ERR_INVALID_ARG;
        }
        b->params[(size_t)g] = p;
        G_need = std::max(G_need, (p.grid_max / p.k_interp) * p.k_interp);
        b->T_max = std::max(b->T_max, p.total_iters);
    }
    b->k = b->params[0].k_interp;
    b->logP = std::max(7, log2c(2LL * G_need - 1));
    if (b->logP > 11) {  // one CTA of 256 threads per FFT work item: P <= 2048
        delete b;
        return TFDP_ERR_PARAM_RANGE;
    }
    b->P = 1 << b->logP;

    // host CSR per graph (validated), packed with global column ids
    b->n.assign(n, n + num_graphs);
    b->node_off.resize((size_t)num_graphs + 1);
    b->node_off[0] = 0;
    for (int g = 0; g < num_graphs; ++g) b->node_off[(size_t)g + 1] = b->node_off[(size_t)g] + n[g];
    b->N = b->node_off[(size_t)num_graphs];
    std::vector<int> rowptr, col;
    rowptr.reserve((size_t)(b->N + num_graphs));
    std::vector<int> rowptr_off((size_t)num_graphs), col_off((size_t)num_graphs);
    for (int g = 0; g < num_graphs; ++g) {
        const int64_t ng = n[g], mg = m[g];
        std::vector<int64_t> keys((size_t)mg);
        std::vector<int> deg((size_t)ng, 0);
        for (int64_t q = 0; q < mg; ++q) {
            const int64_t u = edges[g][2 * q], v = edges[g][2 * q + 1];
            if (u < 0 || v < 0 || u >= ng || v >= ng || u == v) {
                delete b;
                return TFDP_ERR_BAD_GRAPH;
            }
            keys[(size_t)q] = std::min(u, v) * ng + std::max(u, v);
            deg[(size_t)u]++;
            deg[(size_t)v]++;
        }
        std::sort(keys.begin(), keys.end());
        for (size_t q = 1; q < keys.size(); ++q)
            if (keys[q] == keys[q - 1]) {
                delete b;
                return TFDP_ERR_BAD_GRAPH;
            }
        rowptr_off[(size_t)g] = (int)rowptr.size();
        col_off[(size_t)g] = (int)col.size();
        const size_t r0 = rowptr.size();
        rowptr.push_back(0);
        for (int64_t i = 0; i < ng; ++i) rowptr.push_back(rowptr.back() + deg[(size_t)i]);
        const size_t c0 = col.size();
        col.resize(c0 + (size_t)(2 * mg));
        std::vector<int> fill(rowptr.begin() + (long)r0, rowptr.end() - 1);
        const int base = (int)b->node_off[(size_t)g];
        for (int64_t q = 0; q < mg; ++q) {
            const int u = edges[g][2 * q], v = edges[g][2 * q + 1];
            col[c0 + (size_t)fill[(size_t)u]++] = base + v;
            col[c0 + (size_t)fill[(size_t)v]++] = base + u;
        }
        for (int64_t i = 0; i < ng; ++i)
            std::sort(col.begin() + (long)c0 + rowptr[r0 + (size_t)i], col.begin() + (long)c0 + rowptr[r0 + (size_t)i + 1]);
        b->M += mg;
    }

    // item prefix tables and per-graph FFT geometry
    const int T_fft = b->P / 8;
    const int RG = (T_fft >= 256) ? 1 : 256 / T_fft;
    const int CG = RG;
    std::vector<int> pre_nodes(1, 0), pre_boxes(1, 0), pre_rows(1, 0), pre_cols(1, 0);
    b->hg.resize((size_t)num_graphs);
    size_t fft_bytes = 0;
    std::vector<size_t> fft_off((size_t)num_graphs);
    const size_t NH = (size_t)b->P / 2 + 1;
    for (int g = 0; g < num_graphs; ++g) {
        const tfdp_params& p = b->params[(size_t)g];
        BGraph& G = b->hg[(size_t)g];
        const int n_int_max = p.grid_max / p.k_interp;
        G.n = (int)n[g];
        G.node_off = (int)b->node_off[(size_t)g];
        G.rowptr_off = rowptr_off[(size_t)g];
        G.col_off = col_off[(size_t)g];
        G.G_max = n_int_max * p.k_interp;
        G.Gs = (int)up((size_t)G.G_max, 4);
        G.ystride = (int)up((size_t)G.G_max, 32);
        G.nbox_max = n_int_max * n_int_max;
        pre_nodes.push_back(pre_nodes.back() + (G.n + kBNodeChunk - 1) / kBNodeChunk);
        pre_boxes.push_back(pre_boxes.back() + (G.nbox_max + kBChunk - 1) / kBChunk);
        pre_rows.push_back(pre_rows.back() + (G.G_max + 2 * RG - 1) / (2 * RG) + (spec_rows(b->P) + 2 * RG - 1) / (2 * RG));
        pre_cols.push_back(pre_cols.back() + (int)((NH + CG - 1) / CG));
        fft_off[(size_t)g] = fft_bytes;
        fft_bytes += up(sizeof(int) * (size_t)G.nbox_max, 256) + up(sizeof(int) * ((size_t)G.nbox_max + 1), 256) +
                     up(sizeof(float) * 3 * (size_t)G.Gs * G.Gs, 256) + 2 * up(sizeof(float2) * 3 * NH * G.ystride, 256) +
                     up(sizeof(float4) * (size_t)G.Gs * G.Gs, 256) + up(sizeof(float2) * 3 * NH * b->P, 256) +
                     3 * up(sizeof(float) * NH * b->P, 256);
    }
    // node arena layout
    const size_t N = (size_t)b->N;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = up(off, 256);
        off = o + up(bytes ? bytes : 1, 256);
        return o;
    };
    const size_t o_xy0 = take(sizeof(float2) * N), o_xy1 = take(sizeof(float2) * N);
    const size_t o_vx0 = take(sizeof(float2) * N), o_vx1 = take(sizeof(float2) * N);
    const size_t o_vp0 = take(sizeof(int) * N), o_vp1 = take(sizeof(int) * N);
    const size_t o_ks = take(sizeof(int2) * N);
    const size_t o_fatt = take(sizeof(float2) * N), o_frep = take(sizeof(float2) * N);
    const size_t o_rp = take(sizeof(int) * rowptr.size()), o_col = take(sizeof(int) * std::max<size_t>(col.size(), 1));
    const size_t o_tw = take(sizeof(float2) * b->P);
    const size_t o_graphs = take(sizeof(BGraph) * num_graphs), o_st = take(sizeof(DevState) * num_graphs);
    const size_t o_prm = take(sizeof(DevParams) * num_graphs);
    const size_t o_steps = take(sizeof(double) * (size_t)num_graphs * b->T_max);
    const size_t o_pn = take(sizeof(int) * (num_graphs + 1)), o_pb = take(sizeof(int) * (num_graphs + 1));
    const size_t o_pr = take(sizeof(int) * (num_graphs + 1)), o_pc = take(sizeof(int) * (num_graphs + 1));
    const size_t o_fft = take(fft_bytes);
    cudaError_t e = cudaMalloc(&b->mem, off);
    if (e != cudaSuccess) {
        delete b;
        return bfail(e, "cudaMalloc(batch arena)");
    }
    char* base = (char*)b->mem;
    BatchArgs& a = b->args;
    a.B = num_graphs;
    a.xy[0] = (float2*)(base + o_xy0);
    a.xy[1] = (float2*)(base + o_xy1);
    a.vxy[0] = (float2*)(base + o_vx0);
    a.vxy[1] = (float2*)(base + o_vx1);
    a.vperm[0] = (int*)(base + o_vp0);
    a.vperm[1] = (int*)(base + o_vp1);
    a.keyslot = (int2*)(base + o_ks);
    a.fatt = (float2*)(base + o_fatt);
    a.frep = (float2*)(base + o_frep);
    a.rowptr = (const int*)(base + o_rp);
    a.col = (const int*)(base + o_col);
    a.tw = (const float2*)(base + o_tw);
    b->d_graphs = (BGraph*)(base + o_graphs);
    b->d_st = (DevState*)(base + o_st);
    b->d_prm = (DevParams*)(base + o_prm);
    b->d_steps = (double*)(base + o_steps);
    a.graphs = b->d_graphs;
    a.st = b->d_st;
    a.prm = b->d_prm;
    a.pre_nodes = (const int*)(base + o_pn);
    a.pre_boxes = (const int*)(base + o_pb);
    a.pre_rows = (const int*)(base + o_pr);
    a.pre_cols = (const int*)(base + o_pc);
    for (int g = 0; g < num_graphs; ++g) {
        BGraph& G = b->hg[(size_t)g];
        char* f = base + o_fft + fft_off[(size_t)g];
        size_t fo = 0;
        auto sub = [&](size_t bytes) {
            char* q = f + fo;
            fo += up(bytes, 256);
            return q;
        };
        G.cnt = (int*)sub(sizeof(int) * (size_t)G.nbox_max);
        G.off = (int*)sub(sizeof(int) * ((size_t)G.nbox_max + 1));
        G.gin = (float*)sub(sizeof(float) * 3 * (size_t)G.Gs * G.Gs);
        G.T1 = (float2*)sub(sizeof(float2) * 3 * NH * G.ystride);
        G.T2 = (float2*)sub(sizeof(float2) * 3 * NH * G.ystride);
        G.gout = (float4*)sub(sizeof(float4) * (size_t)G.Gs * G.Gs);
        G.S1 = (float2*)sub(sizeof(float2) * 3 * NH * b->P);
        G.specK = (float*)sub(sizeof(float) * NH * b->P);
        G.specHx = (float*)sub(sizeof(float) * NH * b->P);
        G.specHy = (float*)sub(sizeof(float) * NH * b->P);
    }
    auto fail = [&](tfdp_status s) {
        part_destroy(b);
        return s;
    };
    std::vector<float2> tw((size_t)b->P);
    for (int t = 0; t < b->P; ++t) {
        const double ang = -2.0 * 3.14159265358979323846 * (double)t / (double)b->P;
        tw[(size_t)t] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    std::vector<float2> xy(N);
    for (int g = 0; g < num_graphs; ++g)
        std::memcpy(xy.data() + b->node_off[(size_t)g], xy0[g], sizeof(float2) * (size_t)n[g]);
    cudaStream_t s = b->stream;
    if ((e = cudaMemsetAsync(b->mem, 0, off, s)) != cudaSuccess) return fail(bfail(e, "memset"));
    if ((e = cudaMemcpyAsync(a.xy[0], xy.data(), sizeof(float2) * N, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync((void*)a.rowptr, rowptr.data(), sizeof(int) * rowptr.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (!col.empty() && (e = cudaMemcpyAsync((void*)a.col, col.data(), sizeof(int) * col.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess) ||
        (e = cudaMemcpyAsync((void*)a.tw, tw.data(), sizeof(float2) * b->P, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(b->d_graphs, b->hg.data(), sizeof(BGraph) * num_graphs, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync((void*)a.pre_nodes, pre_nodes.data(), sizeof(int) * (num_graphs + 1), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync((void*)a.pre_boxes, pre_boxes.data(), sizeof(int) * (num_graphs + 1), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync((void*)a.pre_rows, pre_rows.data(), sizeof(int) * (num_graphs + 1), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync((void*)a.pre_cols, pre_cols.data(), sizeof(int) * (num_graphs + 1), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return fail(bfail(e, "batch upload"));
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(bfail(e, "batch upload sync"));
    tfdp_status st = upload_batch_params(b);
    if (st != TFDP_OK) return fail(st);
    int bps = 0;
    if ((e = batch_occupancy(b, &bps)) != cudaSuccess || bps < 1) return fail(bfail(e, "batch occupancy"));
    if ((e = batch_phases_attrs(b)) != cudaSuccess) return fail(bfail(e, "batch phase kernels"));
    b->items = BatchItems{pre_nodes.back(), pre_boxes.back(), pre_rows.back(), pre_cols.back()};
    int sms = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->grid_blocks = bps * sms;
    st = batch_refresh(b);
    if (st != TFDP_OK) return fail(st);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(bfail(e, "batch init"));
    *out = b;
    return TFDP_OK;
}

tfdp_status part_iterate(BatchPart* b, int32_t iters) {
    if (!b || iters < 0) return TFDP_ERR_INVALID_ARG;
    if (iters == 0) return TFDP_OK;
    if (b->no_graph) {  // the cooperative launch could not be captured: launch directly
        BatchArgs a = b->args;
        a.iters = iters;
        a.advance = 1;
        a.eval = 0;
        BK(batch_launch(b, a, b->stream));
        b->host_iter += iters;
        return TFDP_OK;
    }
    if (!b->exec || b->exec_iters != iters) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
        cudaStream_t cap;
        BK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        BatchArgs a = b->args;
        a.iters = iters;
        a.advance = 1;
        a.eval = 0;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = batch_launch(b, a, cap);
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            cudaGetLastError();  // clear the capture error, fall back to direct launches
            b->no_graph = true;
            return part_iterate(b, iters);
        }
        b->exec_iters = iters;
    }
    BK(cudaGraphLaunch(b->exec, b->stream));
    b->host_iter += iters;
    return TFDP_OK;
}

tfdp_status part_eval_forces(BatchPart* b, int32_t graph, float* frep, float* fatt, int on_device) {
    if (!b || graph < 0 || graph >= b->B) return TFDP_ERR_INVALID_ARG;
    BatchArgs a = b->args;
    a.iters = 1;
    a.advance = 0;
    a.eval = 1;
    BK(batch_launch(b, a, b->stream));
    const size_t o = (size_t)b->node_off[(size_t)graph], ng = (size_t)b->n[(size_t)graph];
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (frep) BK(cudaMemcpyAsync(frep, a.frep + o, sizeof(float2) * ng, kind, b->stream));
    if (fatt) BK(cudaMemcpyAsync(fatt, a.fatt + o, sizeof(float2) * ng, kind, b->stream));
    return batch_sync_checked(b, graph, graph + 1);
}

tfdp_status part_get_positions(BatchPart* b, int32_t graph, float* xy, int on_device) {
    if (!b || !xy || graph < 0 || graph >= b->B) return TFDP_ERR_INVALID_ARG;
    const int slot = (int)(b->host_iter & 1);
    BK(cudaMemcpyAsync(xy, b->args.xy[slot] + b->node_off[(size_t)graph], sizeof(float2) * (size_t)b->n[(size_t)graph],
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
    return batch_sync_checked(b, graph, graph + 1);
}

tfdp_status part_get_stats(BatchPart* b, int32_t graph, tfdp_stats* out) {
    if (!b || !out || graph < 0 || graph >= b->B) return TFDP_ERR_INVALID_ARG;
    DevState s;
    BK(cudaMemcpyAsync(&s, b->d_st + graph, sizeof(DevState), cudaMemcpyDeviceToHost, b->stream));
    BK(cudaStreamSynchronize(b->stream));
    std::memset(out, 0, sizeof(*out));
    out->iteration = s.iter;
    out->net_frep[0] = s.net_frep[0];
    out->net_frep[1] = s.net_frep[1];
    out->grid_lo = s.grid.lo;
    out->grid_h = s.grid.h;
    out->grid_n_int = s.grid.n_int;
    out->grid_G = s.grid.G;
    out->fft_P = b->P;
    out->spectrum_builds = s.spec_builds;
    out->device_flags = (int32_t)(s.flags | b->flags_seen[(size_t)graph]);
    out->kernels_per_iteration = 0;  // all iterations of a call share one launch
    return TFDP_OK;
}

tfdp_status part_synchronize(BatchPart* b) {
    if (!b) return TFDP_ERR_INVALID_ARG;
    return batch_sync_checked(b, 0, b->B);
}

tfdp_status part_destroy(BatchPart* b) {
    if (!b) return TFDP_OK;
    if (b->mem) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->mem) cudaFree(b->mem);
    delete b;
    return TFDP_OK;
}

int32_t part_grid_blocks(const BatchPart* b) { return b ? b->grid_blocks : 0; }

tfdp_status part_autotune(BatchPart* b, int32_t trials, int32_t* chosen_blocks) {
    if (!b || trials < 1) return TFDP_ERR_INVALID_ARG;
    int bps = 0, sms = 0, dev = 0;
    BK(batch_occupancy(b, &bps));
    BK(cudaGetDevice(&dev));
    BK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // candidates: 1 .. bps co-resident CTAs per SM; timed on force evaluations, which
    // run every phase but move no node
    cudaEvent_t e0, e1;
    BK(cudaEventCreate(&e0));
    BK(cudaEventCreate(&e1));
    BatchArgs a = b->args;
    a.iters = 1;
    a.advance = 0;
    a.eval = 1;
    float best = 1e30f;
    int best_blocks = b->grid_blocks;
    auto time_it = [&](float* ms) -> cudaError_t {
        cudaError_t e = batch_launch(b, a, b->stream);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        for (int t = 0; t < trials && e == cudaSuccess; ++t) e = batch_launch(b, a, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
        return e;
    };
    b->phases = false;
    for (int c = 1; c <= bps; ++c) {
        b->grid_blocks = c * sms;
        float ms = 0.0f;
        BK(time_it(&ms));
        if (ms < best) {
            best = ms;
            best_blocks = c * sms;
        }
    }
    // the other launch shape: one launch per phase
    b->phases = true;
    float ms_phases = 0.0f;
    BK(time_it(&ms_phases));
    b->phases = ms_phases < best;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->grid_blocks = best_blocks;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->exec_iters = -1;
    b->no_graph = false;
    if (chosen_blocks) *chosen_blocks = b->phases ? 0 : best_blocks;
    return TFDP_OK;
}

}  // namespace

// ------------------------------------------------------------------ batches of parts
struct tfdp_batch {
    int B = 0;
    cudaStream_t stream = nullptr;
    std::vector<BatchPart*> parts;
    std::vector<int> part_of, local_of;  // graph -> (part, index in the part)
};

namespace {

int batch_log2p(const tfdp_params& p) {
    const int G = (p.grid_max / p.k_interp) * p.k_interp;
    return std::max(7, log2c(2LL * G - 1));
}

}  // namespace

extern "C" {

tfdp_status tfdp_batch_create(int32_t num_graphs, const int64_t* n, const int64_t* m, const int32_t* const* edges,
                              const float* const* xy0, const tfdp_params* params, void* stream, tfdp_batch** out) {
    if (!out || num_graphs < 1 || !n || !m || !edges || !xy0) return TFDP_ERR_INVALID_ARG;
    // parts: graphs grouped by (k, FFT size), in order of first appearance
    std::vector<std::pair<int, int>> keys;
    std::vector<int> part_of((size_t)num_graphs), local_of((size_t)num_graphs);
    std::vector<std::vector<int>> members;
    for (int g = 0; g < num_graphs; ++g) {
        tfdp_params p;
        if (params) p = params[g];
        else tfdp_params_default(&p);
        p.rep_mode = TFDP_REP_FFT;
        tfdp_status st = tfdp_params_check(&p, nullptr);
        if (st != TFDP_OK) return st;
        if (p.k_interp == TFDP_K_DYNAMIC) return TFDP_ERR_PARAM_RANGE;  // one fixed k per graph
        const std::pair<int, int> key(p.k_interp, batch_log2p(p));
        size_t q = 0;
        while (q < keys.size() && keys[q] != key) ++q;
        if (q == keys.size()) {
            keys.push_back(key);
            members.emplace_back();
        }
        part_of[(size_t)g] = (int)q;
        local_of[(size_t)g] = (int)members[q].size();
        members[q].push_back(g);
    }
    tfdp_batch* b = new (std::nothrow) tfdp_batch();
    if (!b) return TFDP_ERR_OUT_OF_MEMORY;
    b->B = num_graphs;
    b->stream = (cudaStream_t)stream;
    b->part_of = part_of;
    b->local_of = local_of;
    for (size_t q = 0; q < members.size(); ++q) {
        const size_t c = members[q].size();
        std::vector<int64_t> pn(c), pm(c);
        std::vector<const int32_t*> pe(c);
        std::vector<const float*> px(c);
        std::vector<tfdp_params> pp(c);
        for (size_t i = 0; i < c; ++i) {
            const int g = members[q][i];
            pn[i] = n[g];
            pm[i] = m[g];
            pe[i] = edges[g];
            px[i] = xy0[g];
            if (params) pp[i] = params[g];
            else tfdp_params_default(&pp[i]);
        }
        BatchPart* part = nullptr;
        const tfdp_status st = part_create((int32_t)c, pn.data(), pm.data(), pe.data(), px.data(), pp.data(), stream,
                                           &part);
        if (st != TFDP_OK) {
            tfdp_batch_destroy(b);
            return st;
        }
        b->parts.push_back(part);
    }
    *out = b;
    return TFDP_OK;
}

tfdp_status tfdp_batch_iterate(tfdp_batch* b, int32_t iters) {
    if (!b || iters < 0) return TFDP_ERR_INVALID_ARG;
    for (BatchPart* part : b->parts) {
        const tfdp_status st = part_iterate(part, iters);
        if (st != TFDP_OK) return st;
    }
    return TFDP_OK;
}

tfdp_status tfdp_batch_eval_forces(tfdp_batch* b, int32_t graph, float* frep, float* fatt, int on_device) {
    if (!b || graph < 0 || graph >= b->B) return TFDP_ERR_INVALID_ARG;
    return part_eval_forces(b->parts[(size_t)b->part_of[(size_t)graph]], b->local_of[(size_t)graph], frep, fatt,
                            on_device);
}

tfdp_status tfdp_batch_get_positions(tfdp_batch* b, int32_t graph, float* xy, int on_device) {
    if (!b || graph < 0 || graph >= b->B) return TFDP_ERR_INVALID_ARG;
    return part_get_positions(b->parts[(size_t)b->part_of[(size_t)graph]], b->local_of[(size_t)graph], xy,
                              on_device);
}

tfdp_status tfdp_batch_get_stats(tfdp_batch* b, int32_t graph, tfdp_stats* out) {
    if (!b || graph < 0 || graph >= b->B) return TFDP_ERR_INVALID_ARG;
    return part_get_stats(b->parts[(size_t)b->part_of[(size_t)graph]], b->local_of[(size_t)graph], out);
}

tfdp_status tfdp_batch_synchronize(tfdp_batch* b) {
    if (!b) return TFDP_ERR_INVALID_ARG;
    tfdp_status first = TFDP_OK;
    for (BatchPart* part : b->parts) {
        const tfdp_status st = part_synchronize(part);
        if (first == TFDP_OK) first = st;
    }
    return first;
}

tfdp_status tfdp_batch_destroy(tfdp_batch* b) {
    if (!b) return TFDP_OK;
    for (BatchPart* part : b->parts) part_destroy(part);
    delete b;
    return TFDP_OK;
}

int32_t tfdp_batch_grid_blocks(const tfdp_batch* b) {
    int32_t best = 0;
    if (b)
        for (const BatchPart* part : b->parts) best = std::max(best, part_grid_blocks(part));
    return best;
}

tfdp_status tfdp_batch_autotune(tfdp_batch* b, int32_t trials, int32_t* chosen_blocks) {
    if (!b || trials < 1) return TFDP_ERR_INVALID_ARG;
    int32_t best = 0;
    for (BatchPart* part : b->parts) {
        int32_t c = 0;
        const tfdp_status st = part_autotune(part, trials, &c);
        if (st != TFDP_OK) return st;
        best = std::max(best, c);
    }
    if (chosen_blocks) *chosen_blocks = best;
    return TFDP_OK;
}

int32_t tfdp_batch_num_parts(const tfdp_batch* b) { return b ? (int32_t)b->parts.size() : 0; }

tfdp_status tfdp_batch_set_phase_launches(tfdp_batch* b, int32_t on) {
    if (!b || (on != 0 && on != 1)) return TFDP_ERR_INVALID_ARG;
    for (BatchPart* part : b->parts) {
        if (part->phases == (on != 0)) continue;
        BK(cudaStreamSynchronize(part->stream));
        part->phases = on != 0;
        if (part->exec) cudaGraphExecDestroy(part->exec);
        part->exec = nullptr;
        part->exec_iters = -1;
        part->no_graph = false;
    }
    return TFDP_OK;
}

int32_t tfdp_batch_phase_parts(const tfdp_batch* b) {
    int32_t c = 0;
    if (b)
        for (const BatchPart* part : b->parts) c += part->phases ? 1 : 0;
    return c;
}

}  // extern "C"

namespace {

// Relative L2 distance of two n x 2 force fields.
double rel_l2(const std::vector<float>& a, const std::vector<float>& ref) {
    double num = 0.0, den = 0.0;
    for (size_t i = 0; i < ref.size(); ++i) {
        const double d = (double)a[i] - (double)ref[i];
        num += d * d;
        den += (double)ref[i] * (double)ref[i];
    }
    return den > 0.0 ? std::sqrt(num / den) : std::sqrt(num);
}

// Force error of the ibFFT at each candidate (k, grid cap) and at the reference
// parameters, against the exact sum of the same positions, for one graph (GPU).
tfdp_status probe_errors(int64_t n, int64_t m, const int32_t* edges, const float* xy, const tfdp_params& base,
                         const std::vector<std::pair<int, int>>& cand, double* err_ref, std::vector<double>& err) {
    tfdp_params p = base;
    p.rep_mode = TFDP_REP_EXACT;
    tfdp_graph* g = nullptr;
    tfdp_status st = tfdp_create_graph(n, m, edges, xy, 0, &p, nullptr, &g);
    if (st != TFDP_OK) return st;
    std::vector<float> exact((size_t)(2 * n)), f((size_t)(2 * n));
    st = tfdp_eval_forces(g, exact.data(), nullptr, 0);
    p.rep_mode = TFDP_REP_FFT;
    if (st == TFDP_OK) st = tfdp_set_params(g, &p);
    if (st == TFDP_OK) st = tfdp_eval_forces(g, f.data(), nullptr, 0);
    if (st == TFDP_OK) *err_ref = rel_l2(f, exact);
    err.assign(cand.size(), 1e300);
    for (size_t c = 0; c < cand.size() && st == TFDP_OK; ++c) {
        tfdp_params q = p;
        q.k_interp = cand[c].first;
        q.grid_max = cand[c].second;
        st = tfdp_set_params(g, &q);
        if (st == TFDP_OK) st = tfdp_eval_forces(g, f.data(), nullptr, 0);
        if (st == TFDP_OK) err[c] = rel_l2(f, exact);
    }
    tfdp_destroy_graph(g);
    return st;
}

}  // namespace

extern "C" tfdp_status tfdp_batch_plan(int32_t num_graphs, const int64_t* n, const int64_t* m,
                                       const int32_t* const* edges, const float* const* xy0,
                                       const tfdp_params* base, double max_error_ratio, double min_error_bound,
                                       int32_t probes, tfdp_params* out_params, double* out_error) {
    if (num_graphs < 1 || !n || !m || !edges || !xy0 || !out_params || probes < 1 || !(max_error_ratio >= 1.0) ||
        !(min_error_bound >= 0.0))
        return TFDP_ERR_INVALID_ARG;
    tfdp_params ref;
    if (base) ref = *base;
    else tfdp_params_default(&ref);
    ref.rep_mode = TFDP_REP_FFT;
    tfdp_status st = tfdp_params_check(&ref, nullptr);
    if (st != TFDP_OK) return st;
    if (ref.k_interp == TFDP_K_DYNAMIC || ref.precision != TFDP_PREC_FP32) return TFDP_ERR_PARAM_RANGE;
    for (int g = 0; g < num_graphs; ++g)
        if (n[g] < 1 || m[g] < 0 || (m[g] > 0 && !edges[g]) || !xy0[g]) return TFDP_ERR_INVALID_ARG;
    // candidates in order of cost: smaller FFT sizes than the reference's (the transforms
    // dominate small graphs), each with k = 1..3 (k^2 grid nodes per node in the spread
    // and gather), then the reference itself; at the reference's FFT size another k would
    // only split the batch into more launches for little saving
    const int ref_log = batch_log2p(ref);
    std::vector<std::pair<int, int>> cand;
    for (int lp = 7; lp < ref_log; ++lp) {
        const int gm = std::min(1 << (lp - 1), ref.grid_max);  // G <= P / 2 keeps 2 G - 1 <= P
        for (int k = 1; k <= kMaxK; ++k) {
            if (gm / k < 1) continue;
            tfdp_params q = ref;
            q.k_interp = k;
            q.grid_max = gm;
            if (tfdp_params_check(&q, nullptr) != TFDP_OK || batch_log2p(q) != lp) continue;
            cand.emplace_back(k, gm);
        }
    }
    cand.emplace_back(ref.k_interp, ref.grid_max);
    // groups: half octaves of n
    std::vector<int> group((size_t)num_graphs);
    int ngroups = 0;
    for (int g = 0; g < num_graphs; ++g) {
        group[(size_t)g] = (int)std::floor(2.0 * std::log2((double)n[g]));
        ngroups = std::max(ngroups, group[(size_t)g] + 1);
    }
    std::vector<int> choice((size_t)ngroups, -1), probed((size_t)ngroups, 0);
    std::vector<double> worst((size_t)ngroups, 0.0);
    std::vector<std::vector<char>> ok((size_t)ngroups, std::vector<char>(cand.size(), 1));
    std::vector<double> worst_c((size_t)ngroups * cand.size(), 0.0);
    std::vector<double> errs;
    double e_ref = 0.0;
    for (int g = 0; g < num_graphs; ++g) {
        const int q = group[(size_t)g];
        if (probed[(size_t)q] >= probes) continue;
        st = probe_errors(n[g], m[g], edges[g], xy0[g], ref, cand, &e_ref, errs);
        if (st != TFDP_OK) return st;
        ++probed[(size_t)q];
        for (size_t c = 0; c < cand.size(); ++c) {
            if (!(errs[c] <= std::max(max_error_ratio * e_ref, min_error_bound))) ok[(size_t)q][c] = 0;
            worst_c[(size_t)q * cand.size() + c] = std::max(worst_c[(size_t)q * cand.size() + c], errs[c]);
        }
        worst[(size_t)q] = std::max(worst[(size_t)q], e_ref);
    }
    for (int q = 0; q < ngroups; ++q) {
        if (!probed[(size_t)q]) continue;
        for (size_t c = 0; c < cand.size(); ++c)
            if (ok[(size_t)q][c]) {
                choice[(size_t)q] = (int)c;
                break;
            }
    }
    for (int g = 0; g < num_graphs; ++g) {
        const int q = group[(size_t)g];
        tfdp_params p = base ? base[0] : ref;
        p.rep_mode = TFDP_REP_FFT;
        double e = worst[(size_t)q];
        if (choice[(size_t)q] >= 0) {
            p.k_interp = cand[(size_t)choice[(size_t)q]].first;
            p.grid_max = cand[(size_t)choice[(size_t)q]].second;
            e = worst_c[(size_t)q * cand.size() + (size_t)choice[(size_t)q]];
        } else {
            p.k_interp = ref.k_interp;
            p.grid_max = ref.grid_max;
        }
        out_params[g] = p;
        if (out_error) out_error[g] = e;
    }
    return TFDP_OK;
}
