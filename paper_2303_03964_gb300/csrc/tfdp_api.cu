// tfdp_api.cu -- C ABI of the t-FDP library (declared in include/tfdp.h).
//
// A graph owns two device arenas: the node arena (positions, CSR, exact-path partial
// sums, force outputs, parameters, state) and the FFT arena (sort buffers, grids,
// transforms, spectrum, twiddles), sized by grid_max and k. Iterations are captured
// once into CUDA graphs on a private stream and replayed on the caller's stream; the
// kernels read the iteration counter, the grid and the step from device state, so
// one captured graph serves every iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/tfdp.h"
#include "common.cuh"
#include "launch.h"

using namespace tfdp;

namespace {

thread_local std::string g_cuda_err;

tfdp_status cuda_fail(cudaError_t e, const char* where) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
    g_cuda_err = buf;
    return e == cudaErrorMemoryAllocation ? TFDP_ERR_OUT_OF_MEMORY : TFDP_ERR_CUDA;
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);        \
    } while (0)

constexpr int kBatchIters = 8;  // iterations per captured multi-iteration graph
constexpr int kMinLogP = 7, kMaxLogP = 13;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Sub-allocation plan inside one cudaMalloc.
struct Arena {
    size_t bytes = 0;
    char* base = nullptr;
    size_t take(size_t n) {
        size_t off = align_up(bytes, 256);
        bytes = off + align_up(n ? n : 1, 256);
        return off;
    }
};

int gamma_int_of(double g) {
    double r = std::floor(g + 0.5);
    if (std::fabs(g - r) == 0.0 && r >= 2.0 && r <= 8.0) return (int)r;
    return 0;
}

int log2_ceil(long long v) {
    int l = 0;
    while ((1LL << l) < v) ++l;
    return l;
}

}  // namespace

struct tfdp_graph {
    int64_t n = 0, m = 0;
    int device = 0;
    cudaStream_t stream = nullptr;      // caller's stream
    cudaStream_t cap_stream = nullptr;  // private, for graph capture
    tfdp_params params{};
    DevParams dp{};
    int64_t host_iter = 0;

    // node arena
    void* node_mem = nullptr;
    float2* xy[2] = {nullptr, nullptr};
    int* rowptr = nullptr;
    int* col = nullptr;
    float2* part = nullptr;
    int nchunks = 1;
    float2* frep_buf = nullptr;
    float2* fatt_buf = nullptr;
    DevParams* dprm = nullptr;
    DevState* dst = nullptr;
    double* step_table = nullptr;  // device, step_capacity entries
    int step_capacity = 0;
    std::vector<double> step_host;  // staging for the table upload

    // FFT arena
    void* fft_mem = nullptr;
    unsigned fft_gen = 0;             // FFT arenas allocated so far (a new one may reuse the old address)
    int fft_k = 0, fft_grid_max = 0;  // what the FFT arena was sized for
    int P = 0, logP = 0, G_max = 0, Gs = 0, ystride = 0, nbox_max = 0;
    int* cnt = nullptr;
    int* off = nullptr;
    int* bsum = nullptr;
    int2* keyslot = nullptr;
    int* vperm[2] = {nullptr, nullptr};
    float2* vxy[2] = {nullptr, nullptr};
    bool last_was_eval = false;  // which visit-order buffer holds the latest sort
    bool order_valid[2] = {false, false};  // vperm[slot] holds a permutation from a sort / reset
    // local refinement: per-node weights (caller order) and r_i in sorted order
    float* wrep = nullptr;
    float* watt = nullptr;
    float* vwr = nullptr;
    bool use_wrep = false, use_watt = false;
    int* heavy = nullptr;  // nodes of degree > kHeavyDegree
    int n_heavy = 0;
    int spread_shift = 0;  // fixed-point scale of the spread: 2^(27 - spread_shift)
    float* gin = nullptr;
    float2* T1 = nullptr;
    float2* T2 = nullptr;
    float4* gout = nullptr;
    float2* S1 = nullptr;
    float* specK = nullptr;
    float* specHx = nullptr;
    float* specHy = nullptr;
    float2* tw = nullptr;
    // per order k (1..3) of the iterations: FFT size, largest grid and twiddle table (all
    // equal to the graph's own for a fixed k; smaller for k < 3 under the dynamic strategy)
    int logP_k[kMaxK + 1] = {};
    int Gmax_k[kMaxK + 1] = {};
    float2* tw_k[kMaxK + 1] = {};
    // BF16x3 tensor-core column stage: DFT-matrix image and natural-order spectra
    unsigned char* tc_consts = nullptr;
    float* specN = nullptr;

    // captured iterations
    // captured iterations, one pair (1 and kBatchIters iterations) per k
    cudaGraphExec_t exec1[kMaxK + 1] = {}, execB[kMaxK + 1] = {};
    long long exec_key[kMaxK + 1] = {-1, -1, -1, -1};

    // stage timing: begin / end events around the stages whose bit is set in timing_mask
    unsigned timing_mask = 0;
    cudaEvent_t ev_b[TFDP_NUM_STAGES] = {}, ev_e[TFDP_NUM_STAGES] = {};
    // the timing events are recorded on their own stream, forked at each stage border and
    // joined at the end of the iteration, so the kernel chain has no event node in it
    cudaStream_t time_stream = nullptr;
    cudaEvent_t time_fork[2 * TFDP_NUM_STAGES] = {};
    cudaEvent_t time_join = nullptr;

    // side stream for the attraction of the FFT path (fork / join events)
    cudaStream_t side_stream = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;

    // failure detection: device flags read back by the synchronising calls (flags_word),
    // every flag reported so far (flags_seen), and the test hooks of tfdp_debug_inject
    unsigned flags_word = 0;
    unsigned flags_seen = 0;
    int inject_alloc_fail = 0;  // FFT-arena allocations still to refuse
    int inject_scan_stall = 0;  // > 0: look-back poll limit with the first tile withheld

    // k of the next iteration (the fixed k, or the dynamic schedule's k at host_iter)
    int k_now() const { return k_of_iter(params.k_interp, host_iter, params.total_iters); }

    NodeLaunch node_launch(int k = 0) const {
        NodeLaunch a{};
        a.n = (int)n;
        a.k = k ? k : k_now();
        a.gamma_int = dp.gamma_int;
        a.xy[0] = xy[0];
        a.xy[1] = xy[1];
        a.rowptr = rowptr;
        a.col = col;
        a.wrep = use_wrep ? wrep : nullptr;
        a.watt = use_watt ? watt : nullptr;
        a.vwr = (use_wrep && params.rep_mode == TFDP_REP_FFT) ? vwr : nullptr;
        a.heavy = heavy;
        a.n_heavy = n_heavy;
        a.st = dst;
        a.prm = dprm;
        a.nbox_max = nbox_max;
        a.cnt = cnt;
        a.off = off;
        a.bsum = bsum;
        a.scan_status = (unsigned long long*)bsum;
        a.keyslot = keyslot;
        a.vperm[0] = vperm[0];
        a.vperm[1] = vperm[1];
        a.vxy[0] = vxy[0];
        a.vxy[1] = vxy[1];
        a.gin = gin;
        a.Gs = Gs;
        a.gout = gout;
        a.part = part;
        a.nchunks = nchunks;
        a.frep_out = frep_buf;
        a.fatt_out = fatt_buf;
        return a;
    }
    FftLaunch fft_launch(int k) const {
        FftLaunch f{};
        f.logP = logP_k[k];
        f.G_max = Gmax_k[k];
        f.Gs = Gs;
        f.ystride = ystride;
        f.gin = gin;
        f.T1 = T1;
        f.T2 = T2;
        f.gout = gout;
        f.S1 = S1;
        f.specK = specK;
        f.specHx = specHx;
        f.specHy = specHy;
        f.tw = tw_k[k];
        f.st = dst;
        f.prm = dprm;
        return f;
    }
};

namespace {

// Source chunks of the exact path for nb target CTAs and n nodes: at least about four
// CTAs per SM in total (nb * chunks >= 4 * 152) while every chunk keeps at least 64
// sources, and among the next few counts the one whose CTAs divide most evenly over the
// 152 SMs (every CTA does the same work).
int exact_chunks(int nb, int64_t n) {
    const int cmax = (int)std::max<int64_t>(1, std::min<int64_t>(1 << 16, (n + 63) / 64));
    const int c0 = std::max(1, std::min(cmax, (4 * 152 + nb - 1) / nb));
    int best = c0;
    double best_imb = 1e30;
    for (int c = c0; c <= std::min(cmax, c0 + 8); ++c) {
        const double per_sm = (double)nb * c / 152.0;
        const double imb = std::ceil(per_sm) / per_sm;
        if (imb < best_imb - 1e-9) {
            best_imb = imb;
            best = c;
        }
    }
    return best;
}

DevParams make_dev_params(const tfdp_params& p, int P, int logP) {
    DevParams d{};
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
    d.P = P;
    d.log2P = logP;
    d.gamma_int = gamma_int_of(p.gamma);
    return d;
}

// FFT geometry implied by the parameters: the largest grid and box count over the k
// the graph can use (all of 1..3 under the dynamic schedule; k = 1 has the most boxes).
bool fft_geometry(const tfdp_params& p, int* P, int* logP, int* G_max, int* nbox_max) {
    // N_int is capped at floor(grid_max / k) for a fixed k; under the dynamic strategy one
    // cap, floor(grid_max / 3), holds for every k (reading R9b), so G = k N_int <= grid_max
    const int kcap = p.k_interp ? p.k_interp : kMaxK;
    const int n_int_max = p.grid_max / kcap;
    if (n_int_max < 1) return false;
    const int G = kcap * n_int_max;
    int l = log2_ceil(2LL * G - 1);
    if (l < kMinLogP) l = kMinLogP;
    if (l > kMaxLogP) return false;
    *logP = l;
    *P = 1 << l;
    *G_max = G;
    *nbox_max = n_int_max * n_int_max;
    return true;
}

// FFT size and largest grid of the iterations of order k (1..3): the graph's own for a
// fixed k; under the dynamic strategy G <= k floor(grid_max / 3), so k = 1 and 2 run
// smaller transforms than k = 3.
bool fft_geometry_k(const tfdp_params& p, int k, int* logP, int* G_max) {
    int P, l, G, nb;
    if (!fft_geometry(p, &P, &l, &G, &nb)) return false;
    if (p.k_interp) {
        *logP = l;
        *G_max = G;
        return true;
    }
    const int Gk = k * (p.grid_max / kMaxK);
    int lk = log2_ceil(2LL * Gk - 1);
    if (lk < kMinLogP) lk = kMinLogP;
    *logP = lk;
    *G_max = Gk;
    return true;
}

void free_execs(tfdp_graph* g) {
    for (int k = 0; k <= kMaxK; ++k) {
        if (g->exec1[k]) cudaGraphExecDestroy(g->exec1[k]);
        if (g->execB[k]) cudaGraphExecDestroy(g->execB[k]);
        g->exec1[k] = g->execB[k] = nullptr;
        g->exec_key[k] = -1;
    }
}

tfdp_status alloc_fft(tfdp_graph* g) {
    int P, logP, G_max, nbox_max;
    if (!fft_geometry(g->params, &P, &logP, &G_max, &nbox_max)) return TFDP_ERR_PARAM_RANGE;
    const int chunk = scan_items_per_block();
    const int scan_blocks = (nbox_max + chunk - 1) / chunk;
    if (scan_blocks > 1024) return TFDP_ERR_PARAM_RANGE;
    const bool tc = g->params.precision == TFDP_PREC_BF16X3;
    if (g->fft_mem && g->P == P && g->nbox_max == nbox_max && g->G_max == G_max && (!tc || g->tc_consts))
        return TFDP_OK;
    if (g->fft_mem) {
        CK(cudaStreamSynchronize(g->stream));
        CK(cudaFree(g->fft_mem));
        g->fft_mem = nullptr;
    }
    free_execs(g);
    const int Gs = (int)align_up((size_t)G_max, 4);
    // column stride of the transposed spectra: the row kernels write whole blocks of up
    // to 32 rows (16 row pairs), so pad to 32
    const int ystride = (int)align_up((size_t)G_max, 32);
    const size_t NH = (size_t)P / 2 + 1;
    const size_t n = (size_t)std::max<int64_t>(g->n, 1);
    Arena A;
    size_t o_cnt = A.take(sizeof(int) * (size_t)scan_blocks * chunk);
    size_t o_off = A.take(sizeof(int) * ((size_t)nbox_max + 1));
    size_t o_bsum = A.take(sizeof(unsigned long long) * 1024);  // scan tile status words
    size_t o_ks = A.take(sizeof(int2) * n);
    size_t o_vp0 = A.take(sizeof(int) * n);
    size_t o_vp1 = A.take(sizeof(int) * n);
    size_t o_vx0 = A.take(sizeof(float2) * n);
    size_t o_vx1 = A.take(sizeof(float2) * n);
    size_t o_gin = A.take(sizeof(float) * 3 * (size_t)Gs * Gs);
    size_t o_T1 = A.take(sizeof(float2) * 3 * NH * ystride);
    size_t o_T2 = A.take(sizeof(float2) * 3 * NH * ystride);
    size_t o_gout = A.take(sizeof(float4) * (size_t)Gs * Gs);
    size_t o_S1 = A.take(sizeof(float2) * 3 * NH * P);
    size_t o_sK = A.take(sizeof(float) * NH * P);
    size_t o_sHx = A.take(sizeof(float) * NH * P);
    size_t o_sHy = A.take(sizeof(float) * NH * P);
    size_t o_tw = A.take(sizeof(float2) * P);
    int lk[kMaxK + 1] = {}, gk[kMaxK + 1] = {};
    size_t o_twk[kMaxK + 1] = {};
    for (int k = 1; k <= kMaxK; ++k) {
        if (!fft_geometry_k(g->params, k, &lk[k], &gk[k])) return TFDP_ERR_PARAM_RANGE;
        o_twk[k] = A.take(sizeof(float2) * ((size_t)1 << lk[k]));
    }
    size_t o_tcc = tc ? A.take(tc_constants_bytes()) : 0;
    size_t o_spn = tc ? A.take(sizeof(float) * tc_spectrum_floats()) : 0;
    void* mem = nullptr;
    CK(prepare_fft(logP));
    for (int k = 1; k <= kMaxK; ++k) CK(prepare_fft(lk[k]));
    if (tc) CK(prepare_cols_tc());
    if (g->inject_alloc_fail > 0) {  // test hook: refused as if the device were full
        --g->inject_alloc_fail;
        return cuda_fail(cudaErrorMemoryAllocation, "cudaMalloc(fft arena) [refused by tfdp_debug_inject]");
    }
    cudaError_t e = cudaMalloc(&mem, A.bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(fft arena)");
    char* b = (char*)mem;
    g->fft_mem = mem;
    ++g->fft_gen;
    g->order_valid[0] = g->order_valid[1] = false;  // the visit orders of a new arena are unset
    g->cnt = (int*)(b + o_cnt);
    g->off = (int*)(b + o_off);
    g->bsum = (int*)(b + o_bsum);
    g->keyslot = (int2*)(b + o_ks);
    g->vperm[0] = (int*)(b + o_vp0);
    g->vperm[1] = (int*)(b + o_vp1);
    g->vxy[0] = (float2*)(b + o_vx0);
    g->vxy[1] = (float2*)(b + o_vx1);
    g->gin = (float*)(b + o_gin);
    g->T1 = (float2*)(b + o_T1);
    g->T2 = (float2*)(b + o_T2);
    g->gout = (float4*)(b + o_gout);
    g->S1 = (float2*)(b + o_S1);
    g->specK = (float*)(b + o_sK);
    g->specHx = (float*)(b + o_sHx);
    g->specHy = (float*)(b + o_sHy);
    g->tw = (float2*)(b + o_tw);
    for (int k = 1; k <= kMaxK; ++k) {
        g->tw_k[k] = (float2*)(b + o_twk[k]);
        g->logP_k[k] = lk[k];
        g->Gmax_k[k] = gk[k];
    }
    g->tc_consts = tc ? (unsigned char*)(b + o_tcc) : nullptr;
    g->specN = tc ? (float*)(b + o_spn) : nullptr;
    g->P = P;
    g->logP = logP;
    g->G_max = G_max;
    g->Gs = Gs;
    g->ystride = ystride;
    g->nbox_max = nbox_max;
    g->fft_k = g->params.k_interp;
    g->fft_grid_max = g->params.grid_max;
    CK(cudaMemsetAsync(g->cnt, 0, sizeof(int) * (size_t)scan_blocks * chunk, g->stream));
    CK(cudaMemsetAsync(g->bsum, 0, sizeof(unsigned long long) * 1024, g->stream));
    CK(cudaMemsetAsync(&g->dst->scan_ticket, 0, sizeof(unsigned long long), g->stream));
    CK(cudaMemsetAsync(g->gin, 0, sizeof(float) * 3 * (size_t)Gs * Gs, g->stream));
    std::vector<float2> tw(P);
    const double pi = 3.14159265358979323846;
    for (int t = 0; t < P; ++t) {
        const double a = -2.0 * pi * (double)t / (double)P;
        tw[t] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    CK(cudaMemcpyAsync(g->tw, tw.data(), sizeof(float2) * P, cudaMemcpyHostToDevice, g->stream));
    std::vector<float2> twk[kMaxK + 1];
    for (int k = 1; k <= kMaxK; ++k) {
        const int Pk = 1 << lk[k];
        twk[k].resize((size_t)Pk);
        for (int t = 0; t < Pk; ++t) {
            const double a = -2.0 * pi * (double)t / (double)Pk;
            twk[k][(size_t)t] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
        CK(cudaMemcpyAsync(g->tw_k[k], twk[k].data(), sizeof(float2) * Pk, cudaMemcpyHostToDevice, g->stream));
    }
    std::vector<unsigned char> tcimg;
    if (tc) {
        build_tc_constants(tcimg);
        CK(cudaMemcpyAsync(g->tc_consts, tcimg.data(), tcimg.size(), cudaMemcpyHostToDevice, g->stream));
    }
    // a new arena has no valid spectrum
    CK(cudaMemsetAsync(&g->dst->spec_valid, 0, sizeof(int), g->stream));
    CK(cudaStreamSynchronize(g->stream));  // keeps `tw`, `twk` and `tcimg` alive until copied
    return TFDP_OK;
}

tfdp_status upload_params(tfdp_graph* g) {
    // step schedule s_t = s0 (s_min / s0)^(t / (T - 1)), computed in FP64 on the host
    const int T = g->params.total_iters;
    if (T > g->step_capacity) {
        CK(cudaStreamSynchronize(g->stream));
        if (g->step_table) CK(cudaFree(g->step_table));
        g->step_table = nullptr;
        g->step_capacity = 0;
        CK(cudaMalloc(&g->step_table, sizeof(double) * (size_t)T));
        g->step_capacity = T;
    }
    CK(cudaStreamSynchronize(g->stream));  // the staging vector is reused below
    g->step_host.resize((size_t)T);
    for (int t = 0; t < T; ++t)
        g->step_host[(size_t)t] = (T <= 1) ? g->params.step0
                                           : g->params.step0 * std::pow(g->params.step_min / g->params.step0,
                                                                        (double)t / (double)(T - 1));
    CK(cudaMemcpyAsync(g->step_table, g->step_host.data(), sizeof(double) * (size_t)T, cudaMemcpyHostToDevice,
                       g->stream));
    g->dp = make_dev_params(g->params, g->P ? g->P : 128, g->logP ? g->logP : 7);
    g->dp.step_table = g->step_table;
    g->dp.spread_shift = g->spread_shift;
    g->dp.scan_spin_limit = g->inject_scan_stall;
    g->dp.scan_stall = g->inject_scan_stall > 0 ? 1 : 0;
    CK(cudaMemcpyAsync(g->dprm, &g->dp, sizeof(DevParams), cudaMemcpyHostToDevice, g->stream));
    // dp lives in the graph object, which outlives the copy; the copy is ordered
    // before any later kernel on the stream.
    return TFDP_OK;
}

// Recompute the bbox slot of the current positions.
tfdp_status refresh_bbox(tfdp_graph* g) {
    const int slot = (int)(g->host_iter & 1);
    static_assert(kOrdMinInit == 0xFFFFFFFFu && kOrdMaxInit == 0u, "bbox identities set by memset");
    CK(cudaMemsetAsync(&g->dst->bbox[slot][0], 0xFF, sizeof(unsigned), g->stream));
    CK(cudaMemsetAsync(&g->dst->bbox[slot][1], 0x00, sizeof(unsigned), g->stream));
    CK(launch_bbox(g->node_launch(), slot, g->stream));
    // visit order after an upload (FFT path): the last sorted order with the new
    // positions when there is one (keeps the next sort coherent), else the caller order
    if (g->fft_mem && g->params.rep_mode == TFDP_REP_FFT) {
        if (g->order_valid[slot]) {
            CK(launch_order_refresh(g->node_launch(), slot, g->stream));
        } else {
            CK(launch_order_reset(g->node_launch(), slot, g->stream));
            g->order_valid[slot] = true;
        }
    }
    return TFDP_OK;
}

// An FFT-mode graph always has its FFT buffers before an FFT kernel runs. A failed
// reallocation (tfdp_set_params asking for a larger grid when device memory is short)
// leaves the graph in FFT mode without them; then retry the allocation, redo what a new
// arena needs (visit order, device parameters), or return the allocation's error.
tfdp_status fft_ready(tfdp_graph* g) {
    if (g->params.rep_mode != TFDP_REP_FFT || g->fft_mem || g->n == 0) return TFDP_OK;
    tfdp_status st = alloc_fft(g);
    if (st != TFDP_OK) return st;
    const int slot = (int)(g->host_iter & 1);
    CK(launch_order_reset(g->node_launch(), slot, g->stream));
    g->order_valid[slot] = true;
    st = upload_params(g);
    if (st != TFDP_OK) return st;
    CK(cudaStreamSynchronize(g->stream));
    return TFDP_OK;
}

// Status of device-side checks: a bounded wait that gave up is TFDP_ERR_TIMEOUT, any
// other flag (a non-finite position, a box or sorted slot out of range) is
// TFDP_ERR_DEVICE_CHECK.
tfdp_status status_of_flags(unsigned f) {
    if (f & FLAG_WAIT_TIMEOUT) return TFDP_ERR_TIMEOUT;
    return f ? TFDP_ERR_DEVICE_CHECK : TFDP_OK;
}

// Wait for the graph's stream and report the device flags raised since the last report.
// The flags are then cleared on the device (tfdp_get_stats keeps showing them); a flag
// of the sort (a wait that ran out, a slot out of range) may have left the visit order
// with repeated or missing nodes, so the order of the next iteration restarts from the
// caller order.
tfdp_status sync_checked(tfdp_graph* g) {
    CK(cudaMemcpyAsync(&g->flags_word, &g->dst->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    const unsigned f = g->flags_word;
    if (!f) return TFDP_OK;
    g->flags_seen |= f;
    CK(cudaMemsetAsync(&g->dst->flags, 0, sizeof(unsigned), g->stream));
    if ((f & (FLAG_WAIT_TIMEOUT | FLAG_SORT_RANGE | FLAG_BOX_RANGE)) && g->fft_mem && g->n > 0) {
        const int slot = (int)(g->host_iter & 1);
        CK(launch_order_reset(g->node_launch(), slot, g->stream));
        g->order_valid[slot] = true;
    }
    CK(cudaStreamSynchronize(g->stream));
    return status_of_flags(f);
}

// Enqueue one iteration (advance = 1) or one force evaluation (advance = 0, eval = 1).
// Stages selected by the timing mask are bracketed by event records. The records sit on
// a branch of their own (forked from the stage's stream at each border, joined at the
// end), so no kernel waits for one; inside a captured graph they become event-record
// nodes off the kernel chain.
tfdp_status enqueue_step(tfdp_graph* g, cudaStream_t s, int advance, int eval, int k) {
    const NodeLaunch a = g->node_launch(k);
    const unsigned tm = g->timing_mask;
    // cudaEventRecordExternal makes the record a node of a captured graph (a plain
    // record inside a capture only orders the capture and is never timed)
    auto stamp = [&](cudaEvent_t ev, cudaEvent_t fork, cudaStream_t st) -> cudaError_t {
        cudaError_t e = cudaEventRecord(fork, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(g->time_stream, fork, 0);
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev, g->time_stream, cudaEventRecordExternal);
        return e;
    };
    // the attraction runs alone on the side stream: its events go on that stream itself,
    // so that the timing branch of the main chain never waits for it
    auto begin = [&](int stage, cudaStream_t st) -> cudaError_t {
        if (!((tm >> stage) & 1u)) return cudaSuccess;
        if (stage == TFDP_STAGE_ATTRACT) return cudaEventRecordWithFlags(g->ev_b[stage], st, cudaEventRecordExternal);
        return stamp(g->ev_b[stage], g->time_fork[2 * stage], st);
    };
    auto end = [&](int stage, cudaStream_t st) -> cudaError_t {
        if (!((tm >> stage) & 1u)) return cudaSuccess;
        if (stage == TFDP_STAGE_ATTRACT) return cudaEventRecordWithFlags(g->ev_e[stage], st, cudaEventRecordExternal);
        return stamp(g->ev_e[stage], g->time_fork[2 * stage + 1], st);
    };
    if (g->params.rep_mode == TFDP_REP_EXACT) {
        CK(begin(TFDP_STAGE_EXACT, s));
        CK(launch_exact_pairs(a, advance, s));
        CK(end(TFDP_STAGE_EXACT, s));
        CK(begin(TFDP_STAGE_EDGE_UPDATE, s));
        CK(launch_edge_update(a, advance, eval, s));
        CK(end(TFDP_STAGE_EDGE_UPDATE, s));
    } else {
        const FftLaunch f = g->fft_launch(k);
        CK(begin(TFDP_STAGE_SORT, s));
        CK(launch_fft_grid(a, advance, s));
        // attraction on the side stream, overlapping sort, spread and FFT
        CK(cudaEventRecord(g->fork_ev, s));
        CK(cudaStreamWaitEvent(g->side_stream, g->fork_ev, 0));
        CK(begin(TFDP_STAGE_ATTRACT, g->side_stream));
        CK(launch_attract(a, g->side_stream));
        CK(end(TFDP_STAGE_ATTRACT, g->side_stream));
        CK(cudaEventRecord(g->join_ev, g->side_stream));
        CK(launch_fft_sort(a, s));
        CK(end(TFDP_STAGE_SORT, s));
        CK(begin(TFDP_STAGE_SPREAD, s));
        CK(launch_fft_spread(a, s));
        CK(end(TFDP_STAGE_SPREAD, s));
        CK(begin(TFDP_STAGE_SPECTRUM, s));
        CK(launch_spectrum(f, s));
        CK(end(TFDP_STAGE_SPECTRUM, s));
        CK(begin(TFDP_STAGE_ROWS_FWD, s));
        CK(launch_rows_fwd(f, s));
        CK(end(TFDP_STAGE_ROWS_FWD, s));
        CK(begin(TFDP_STAGE_COLS, s));
        if (g->params.precision == TFDP_PREC_BF16X3) CK(launch_cols_tc(f, g->tc_consts, g->specN, s));
        else CK(launch_cols(f, s));
        CK(end(TFDP_STAGE_COLS, s));
        CK(begin(TFDP_STAGE_ROWS_INV, s));
        CK(launch_rows_inv(f, s));
        CK(end(TFDP_STAGE_ROWS_INV, s));
        CK(cudaStreamWaitEvent(s, g->join_ev, 0));
        CK(begin(TFDP_STAGE_GATHER_UPDATE, s));
        CK(launch_fft_back(a, advance, eval, s));
        CK(end(TFDP_STAGE_GATHER_UPDATE, s));
    }
    if (tm) {  // the timing branch rejoins the stream at the end of the iteration
        CK(cudaEventRecord(g->time_join, g->time_stream));
        CK(cudaStreamWaitEvent(s, g->time_join, 0));
    }
    return TFDP_OK;
}

// Kernels launched per iteration (count of the launches above).
int kernels_per_iteration(const tfdp_graph* g) {
    // FFT: attraction, grid + bin + scan + scatter, spread, rows, cols, rows, gather +
    // update (every FFT size runs the register-resident kernels, which build the
    // spectrum inside the row and column passes)
    if (g->params.rep_mode == TFDP_REP_EXACT) return 2;
    return 1 + 4 + 1 + 1 + 1 + 1 + 1;
}

long long exec_key_of(const tfdp_graph* g, int k) {
    return ((long long)g->params.rep_mode << 40) | ((long long)k << 32) |
           ((long long)g->dp.gamma_int << 24) | ((long long)g->logP << 16) |
           ((long long)g->timing_mask << 48) | ((long long)g->params.precision << 60) |
           (long long)(g->fft_mem != nullptr);
}

// Capture `iters` iterations with the kernels of interpolation order k.
tfdp_status capture(tfdp_graph* g, int iters, int k, cudaGraphExec_t* out) {
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
    tfdp_status st = TFDP_OK;
    for (int i = 0; i < iters && st == TFDP_OK; ++i) st = enqueue_step(g, g->cap_stream, 1, 0, k);
    cudaError_t e = cudaStreamEndCapture(g->cap_stream, &graph);
    if (st != TFDP_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return TFDP_OK;
}

tfdp_status ensure_execs(tfdp_graph* g, int k) {
    const long long key = exec_key_of(g, k);
    if (g->exec1[k] && g->execB[k] && g->exec_key[k] == key) return TFDP_OK;
    if (g->exec1[k]) cudaGraphExecDestroy(g->exec1[k]);
    if (g->execB[k]) cudaGraphExecDestroy(g->execB[k]);
    g->exec1[k] = g->execB[k] = nullptr;
    g->exec_key[k] = -1;
    tfdp_status st = capture(g, 1, k, &g->exec1[k]);
    if (st != TFDP_OK) return st;
    st = capture(g, kBatchIters, k, &g->execB[k]);
    if (st != TFDP_OK) return st;
    g->exec_key[k] = key;
    return TFDP_OK;
}

uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" {

const char* tfdp_status_str(tfdp_status s) {
    switch (s) {
        case TFDP_OK: return "TFDP_OK";
        case TFDP_ERR_INVALID_ARG: return "TFDP_ERR_INVALID_ARG";
        case TFDP_ERR_BAD_GRAPH: return "TFDP_ERR_BAD_GRAPH";
        case TFDP_ERR_PARAM_RANGE: return "TFDP_ERR_PARAM_RANGE";
        case TFDP_ERR_OUT_OF_MEMORY: return "TFDP_ERR_OUT_OF_MEMORY";
        case TFDP_ERR_CUDA: return "TFDP_ERR_CUDA";
        case TFDP_ERR_TIMEOUT: return "TFDP_ERR_TIMEOUT";
        case TFDP_ERR_BUSY: return "TFDP_ERR_BUSY";
        case TFDP_ERR_DEVICE_CHECK: return "TFDP_ERR_DEVICE_CHECK";
    }
    return "TFDP_ERR_UNKNOWN";
}

const char* tfdp_last_cuda_error(void) { return g_cuda_err.c_str(); }

// TFDP_REP_AUTO -> the mode with the shorter estimated iteration for a graph of n nodes.
// Measured on GB300 (Erdos-Renyi graphs of mean degree 8, n = 500 ... 48,000, FFT sizes
// P = 512 and 2048): an exact iteration takes about 9 us + n^2 / 3.0e12 pairs/s; an FFT
// iteration about 40 us at P <= 512 plus 15 us per doubling of P above 512, nearly
// independent of n at these sizes (its kernel chain, not its work, sets the time). The
// crossover falls near n = 9,600 at P = 512 and 13,500 at P = 2048 (measured: between
// 8,000 and 12,000, and near 16,000).
int resolve_rep_mode(const tfdp_params& p, int64_t n) {
    if (p.rep_mode != TFDP_REP_AUTO) return p.rep_mode;
    int P, logP, G, nb;
    if (!fft_geometry(p, &P, &logP, &G, &nb)) return TFDP_REP_EXACT;
    const double t_fft = 40e-6 + 15e-6 * (double)std::max(0, logP - 9);
    const double t_exact = 9e-6 + (double)n * (double)n / 3.0e12;
    return t_exact <= t_fft ? TFDP_REP_EXACT : TFDP_REP_FFT;
}

tfdp_status tfdp_params_default(tfdp_params* out) {
    if (!out) return TFDP_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    out->alpha = 0.1;
    out->beta = 8.0;
    out->gamma = 2.0;
    out->k_interp = 3;
    out->n_int_min = 50;
    out->grid_max = 1023;
    out->grid_policy = TFDP_GRID_SNAP_H;
    out->rep_mode = TFDP_REP_FFT;
    out->precision = TFDP_PREC_FP32;
    out->step0 = 1.0;
    out->step_min = 0.01;
    out->total_iters = 300;
    return TFDP_OK;
}

tfdp_status tfdp_params_check(const tfdp_params* p, int* weight_ok) {
    if (!p) return TFDP_ERR_INVALID_ARG;
    if (!(p->gamma > 1.0) || !std::isfinite(p->gamma)) return TFDP_ERR_PARAM_RANGE;
    if (!(p->alpha >= 0.0) || !std::isfinite(p->alpha)) return TFDP_ERR_PARAM_RANGE;
    if (!(p->beta >= 0.0) || !std::isfinite(p->beta)) return TFDP_ERR_PARAM_RANGE;
    if (p->k_interp < 0 || p->k_interp > kMaxK) return TFDP_ERR_PARAM_RANGE;  // 0: dynamic
    if (p->n_int_min < 1) return TFDP_ERR_PARAM_RANGE;
    if (p->grid_max < (p->k_interp ? p->k_interp : kMaxK)) return TFDP_ERR_PARAM_RANGE;
    if (p->grid_policy != TFDP_GRID_PAPER && p->grid_policy != TFDP_GRID_SNAP_H) return TFDP_ERR_INVALID_ARG;
    if (p->rep_mode != TFDP_REP_EXACT && p->rep_mode != TFDP_REP_FFT && p->rep_mode != TFDP_REP_AUTO)
        return TFDP_ERR_INVALID_ARG;
    if (p->precision != TFDP_PREC_FP32 && p->precision != TFDP_PREC_BF16X3) return TFDP_ERR_INVALID_ARG;
    if (!(p->step_min > 0.0) || !(p->step0 >= p->step_min) || !std::isfinite(p->step0)) return TFDP_ERR_PARAM_RANGE;
    if (p->total_iters < 1) return TFDP_ERR_PARAM_RANGE;
    for (int i = 0; i < 7; ++i)
        if (p->reserved[i] != 0) return TFDP_ERR_INVALID_ARG;
    if (p->rep_mode != TFDP_REP_EXACT) {  // FFT, or AUTO, which may resolve to FFT
        int P, l, G, nb;
        if (!fft_geometry(*p, &P, &l, &G, &nb)) return TFDP_ERR_PARAM_RANGE;
        if ((nb + scan_items_per_block() - 1) / scan_items_per_block() > 1024) return TFDP_ERR_PARAM_RANGE;
        // the tensor-core column stage is built for the 64 x 32 factorisation of P = 2048
        if (p->precision == TFDP_PREC_BF16X3 && (P != 2048 || p->k_interp == TFDP_K_DYNAMIC))
            return TFDP_ERR_PARAM_RANGE;
    }
    if (weight_ok) *weight_ok = (p->alpha * (1.0 + p->beta) < 1.0) ? 1 : 0;
    return TFDP_OK;
}

tfdp_status tfdp_create_graph(int64_t n, int64_t m, const int32_t* edges, const float* xy0, uint64_t seed,
                              const tfdp_params* params, void* stream, tfdp_graph** out) {
    if (!out || n < 0 || m < 0 || (m > 0 && !edges)) return TFDP_ERR_INVALID_ARG;
    if (n > (int64_t)INT32_MAX / 2 || 2 * m > (int64_t)INT32_MAX) return TFDP_ERR_INVALID_ARG;
    tfdp_params p;
    if (params) p = *params;
    else tfdp_params_default(&p);
    tfdp_status st = tfdp_params_check(&p, nullptr);
    if (st != TFDP_OK) return st;
    p.rep_mode = resolve_rep_mode(p, n);

    // validate edges and build the symmetric CSR (rows sorted by neighbour id)
    std::vector<int64_t> keys((size_t)m);
    std::vector<int> deg((size_t)n + 1, 0);
    for (int64_t q = 0; q < m; ++q) {
        const int64_t a = edges[2 * q], b = edges[2 * q + 1];
        if (a < 0 || b < 0 || a >= n || b >= n || a == b) return TFDP_ERR_BAD_GRAPH;
        keys[(size_t)q] = std::min(a, b) * n + std::max(a, b);
        deg[(size_t)a]++;
        deg[(size_t)b]++;
    }
    std::sort(keys.begin(), keys.end());
    for (size_t q = 1; q < keys.size(); ++q)
        if (keys[q] == keys[q - 1]) return TFDP_ERR_BAD_GRAPH;
    std::vector<int> rowptr((size_t)n + 1, 0);
    for (int64_t i = 0; i < n; ++i) rowptr[(size_t)i + 1] = rowptr[(size_t)i] + deg[(size_t)i];
    std::vector<int> col((size_t)(2 * m));
    std::vector<int> fill(rowptr.begin(), rowptr.end() - 1);
    for (int64_t q = 0; q < m; ++q) {
        const int a = edges[2 * q], b = edges[2 * q + 1];
        col[(size_t)fill[(size_t)a]++] = b;
        col[(size_t)fill[(size_t)b]++] = a;
    }
    for (int64_t i = 0; i < n; ++i) std::sort(col.begin() + rowptr[(size_t)i], col.begin() + rowptr[(size_t)i + 1]);
    std::vector<int> heavy;  // nodes whose attraction a warp sums
    for (int64_t i = 0; i < n; ++i)
        if (deg[(size_t)i] > kHeavyDegree) heavy.push_back((int)i);

    tfdp_graph* g = new (std::nothrow) tfdp_graph();
    if (!g) return TFDP_ERR_OUT_OF_MEMORY;
    g->n = n;
    g->m = m;
    g->params = p;
    g->stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->side_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->fork_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->join_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
        if (g->side_stream) cudaStreamDestroy(g->side_stream);
        if (g->fork_ev) cudaEventDestroy(g->fork_ev);
        if (g->join_ev) cudaEventDestroy(g->join_ev);
        delete g;
        return cuda_fail(e, "create stream");
    }

    // exact-path chunking
    const int nb = (int)std::max<int64_t>(1, (n + 256 * kExactTargets - 1) / (256 * kExactTargets));
    g->nchunks = exact_chunks(nb, n);

    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    Arena A;
    size_t o_xy0 = A.take(sizeof(float2) * nn);
    size_t o_xy1 = A.take(sizeof(float2) * nn);
    size_t o_rp = A.take(sizeof(int) * (nn + 1));
    size_t o_col = A.take(sizeof(int) * (size_t)std::max<int64_t>(2 * m, 1));
    size_t o_heavy = A.take(sizeof(int) * std::max<size_t>(heavy.size(), 1));
    size_t o_part = A.take(sizeof(float2) * nn * (size_t)g->nchunks);
    size_t o_fr = A.take(sizeof(float2) * nn);
    size_t o_fa = A.take(sizeof(float2) * nn);
    size_t o_prm = A.take(sizeof(DevParams));
    size_t o_st = A.take(sizeof(DevState));
    e = cudaMalloc(&g->node_mem, A.bytes);
    if (e != cudaSuccess) {
        cudaStreamDestroy(g->cap_stream);
        cudaStreamDestroy(g->side_stream);
        cudaEventDestroy(g->fork_ev);
        cudaEventDestroy(g->join_ev);
        delete g;
        return cuda_fail(e, "cudaMalloc(node arena)");
    }
    char* b = (char*)g->node_mem;
    g->xy[0] = (float2*)(b + o_xy0);
    g->xy[1] = (float2*)(b + o_xy1);
    g->rowptr = (int*)(b + o_rp);
    g->col = (int*)(b + o_col);
    g->heavy = (int*)(b + o_heavy);
    g->n_heavy = (int)heavy.size();
    g->part = (float2*)(b + o_part);
    g->frep_buf = (float2*)(b + o_fr);
    g->fatt_buf = (float2*)(b + o_fa);
    g->dprm = (DevParams*)(b + o_prm);
    g->dst = (DevState*)(b + o_st);

    auto fail = [&](tfdp_status s) {
        tfdp_destroy_graph(g);
        return s;
    };
    std::vector<float> init;
    const float* src = xy0;
    if (!src && n > 0) {
        init.resize((size_t)(2 * n));
        const double half = 0.5 * std::sqrt((double)n);
        for (int64_t i = 0; i < 2 * n; ++i) {
            const uint64_t z = splitmix64(seed + (uint64_t)i * 0x9E3779B97F4A7C15ULL);
            const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
            init[(size_t)i] = (float)((2.0 * u - 1.0) * half);
        }
        src = init.data();
    }
    if ((e = cudaMemsetAsync(g->dst, 0, sizeof(DevState), g->stream)) != cudaSuccess) return fail(cuda_fail(e, "memset state"));
    if (n > 0) {
        if ((e = cudaMemcpyAsync(g->xy[0], src, sizeof(float2) * (size_t)n, cudaMemcpyHostToDevice, g->stream)) != cudaSuccess)
            return fail(cuda_fail(e, "copy positions"));
        if ((e = cudaMemcpyAsync(g->rowptr, rowptr.data(), sizeof(int) * (size_t)(n + 1), cudaMemcpyHostToDevice, g->stream)) != cudaSuccess)
            return fail(cuda_fail(e, "copy rowptr"));
    }
    if (m > 0 && (e = cudaMemcpyAsync(g->col, col.data(), sizeof(int) * (size_t)(2 * m), cudaMemcpyHostToDevice, g->stream)) != cudaSuccess)
        return fail(cuda_fail(e, "copy col"));
    if (!heavy.empty() && (e = cudaMemcpyAsync(g->heavy, heavy.data(), sizeof(int) * heavy.size(),
                                               cudaMemcpyHostToDevice, g->stream)) != cudaSuccess)
        return fail(cuda_fail(e, "copy heavy list"));
    if (p.rep_mode == TFDP_REP_FFT) {
        st = alloc_fft(g);
        if (st != TFDP_OK) return fail(st);
    }
    st = upload_params(g);
    if (st == TFDP_OK) st = refresh_bbox(g);  // synchronises: host buffers above are consumed
    if (st != TFDP_OK) return fail(st);
    *out = g;
    return TFDP_OK;
}

tfdp_status tfdp_set_params(tfdp_graph* g, const tfdp_params* given) {
    if (!g || !given) return TFDP_ERR_INVALID_ARG;
    tfdp_status st = tfdp_params_check(given, nullptr);
    if (st != TFDP_OK) return st;
    tfdp_params resolved = *given;
    resolved.rep_mode = resolve_rep_mode(resolved, g->n);
    const tfdp_params* p = &resolved;
    const bool to_fft = p->rep_mode == TFDP_REP_FFT && g->params.rep_mode != TFDP_REP_FFT;
    const bool prec_changed = p->precision != g->params.precision;
    g->params = *p;
    if (prec_changed && g->dst)  // each precision mode keeps its own spectrum arrays
        CK(cudaMemsetAsync(&g->dst->spec_valid, 0, sizeof(int), g->stream));
    if (p->rep_mode == TFDP_REP_FFT) {
        // compare generations, not addresses: a new arena can land where the old one was
        const unsigned before = g->fft_gen;
        st = alloc_fft(g);
        if (st != TFDP_OK) return st;
        if ((to_fft || g->fft_gen != before) && g->n > 0) {
            CK(launch_order_reset(g->node_launch(), (int)(g->host_iter & 1), g->stream));
            g->order_valid[g->host_iter & 1] = true;
        }
    }
    st = upload_params(g);
    if (st != TFDP_OK) return st;
    CK(cudaStreamSynchronize(g->stream));  // g->dp may change again before the copy runs
    return TFDP_OK;
}

tfdp_status tfdp_get_params(const tfdp_graph* g, tfdp_params* out) {
    if (!g || !out) return TFDP_ERR_INVALID_ARG;
    *out = g->params;
    return TFDP_OK;
}

tfdp_status tfdp_set_positions(tfdp_graph* g, const float* xy, int on_device) {
    if (!g || (!xy && g->n > 0)) return TFDP_ERR_INVALID_ARG;
    if (g->n == 0) return TFDP_OK;
    const int slot = (int)(g->host_iter & 1);
    CK(cudaMemcpyAsync(g->xy[slot], xy, sizeof(float2) * (size_t)g->n,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->stream));
    return refresh_bbox(g);
}

tfdp_status tfdp_get_positions(tfdp_graph* g, float* xy, int on_device) {
    if (!g || (!xy && g->n > 0)) return TFDP_ERR_INVALID_ARG;
    if (g->n > 0) {
        const int slot = (int)(g->host_iter & 1);
        CK(cudaMemcpyAsync(xy, g->xy[slot], sizeof(float2) * (size_t)g->n,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream));
    }
    return sync_checked(g);
}

tfdp_status tfdp_iterate(tfdp_graph* g, int32_t iters) {
    if (!g || iters < 0) return TFDP_ERR_INVALID_ARG;
    if (iters == 0) return TFDP_OK;
    if (g->n == 0) {
        g->host_iter += iters;
        return tfdp_set_iteration(g, g->host_iter);
    }
    tfdp_status ready = fft_ready(g);
    if (ready != TFDP_OK) return ready;
    // segments of constant k (one segment unless the dynamic schedule switches k); the
    // device derives the same k from its iteration counter
    int left = iters;
    while (left > 0) {
        const int k = g->k_now();
        int seg = 0;
        while (seg < left && k_of_iter(g->params.k_interp, g->host_iter + seg, g->params.total_iters) == k) ++seg;
        tfdp_status st = ensure_execs(g, k);
        if (st != TFDP_OK) return st;
        int todo = seg;
        while (todo >= kBatchIters) {
            CK(cudaGraphLaunch(g->execB[k], g->stream));
            todo -= kBatchIters;
        }
        while (todo-- > 0) CK(cudaGraphLaunch(g->exec1[k], g->stream));
        g->host_iter += seg;
        left -= seg;
    }
    g->last_was_eval = false;
    g->order_valid[0] = g->order_valid[1] = true;  // the sorts wrote both visit orders
    return TFDP_OK;
}

tfdp_status tfdp_run(tfdp_graph* g, const float* xy_in, int32_t iters, float* xy_out) {
    if (!g || (!xy_out && g->n > 0) || iters < 0) return TFDP_ERR_INVALID_ARG;
    if (g->n == 0) return tfdp_iterate(g, iters);
    if (xy_in) {
        const int slot = (int)(g->host_iter & 1);
        CK(cudaMemcpyAsync(g->xy[slot], xy_in, sizeof(float2) * (size_t)g->n, cudaMemcpyHostToDevice, g->stream));
        tfdp_status st = refresh_bbox(g);  // stream-ordered, no synchronisation
        if (st != TFDP_OK) return st;
    }
    tfdp_status st = tfdp_iterate(g, iters);
    if (st != TFDP_OK) return st;
    const int slot = (int)(g->host_iter & 1);
    CK(cudaMemcpyAsync(xy_out, g->xy[slot], sizeof(float2) * (size_t)g->n, cudaMemcpyDeviceToHost, g->stream));
    return sync_checked(g);
}

tfdp_status tfdp_set_iteration(tfdp_graph* g, int64_t t) {
    if (!g || t < 0) return TFDP_ERR_INVALID_ARG;
    const int old_slot = (int)(g->host_iter & 1), new_slot = (int)(t & 1);
    if (old_slot != new_slot && g->n > 0)
        CK(cudaMemcpyAsync(g->xy[new_slot], g->xy[old_slot], sizeof(float2) * (size_t)g->n,
                           cudaMemcpyDeviceToDevice, g->stream));
    g->host_iter = t;
    long long tt = (long long)t;
    CK(cudaMemcpyAsync(&g->dst->iter, &tt, sizeof(tt), cudaMemcpyHostToDevice, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    if (g->n > 0 && old_slot != new_slot) return refresh_bbox(g);
    return TFDP_OK;
}

tfdp_status tfdp_eval_forces(tfdp_graph* g, float* frep, float* fatt, int on_device) {
    if (!g) return TFDP_ERR_INVALID_ARG;
    if (g->n == 0) return TFDP_OK;
    tfdp_status st = fft_ready(g);
    if (st != TFDP_OK) return st;
    st = enqueue_step(g, g->stream, 0, 1, g->k_now());
    if (st != TFDP_OK) return st;
    g->last_was_eval = true;
    g->order_valid[(g->host_iter & 1) ^ 1] = true;  // its sort wrote the other visit order
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (frep) CK(cudaMemcpyAsync(frep, g->frep_buf, sizeof(float2) * (size_t)g->n, kind, g->stream));
    if (fatt) CK(cudaMemcpyAsync(fatt, g->fatt_buf, sizeof(float2) * (size_t)g->n, kind, g->stream));
    return sync_checked(g);
}

tfdp_status tfdp_get_stats(tfdp_graph* g, tfdp_stats* out) {
    if (!g || !out) return TFDP_ERR_INVALID_ARG;
    DevState s;
    CK(cudaMemcpyAsync(&s, g->dst, sizeof(DevState), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    std::memset(out, 0, sizeof(*out));
    out->iteration = s.iter;
    out->net_frep[0] = s.net_frep[0];
    out->net_frep[1] = s.net_frep[1];
    out->grid_lo = s.grid.lo;
    out->grid_h = s.grid.h;
    out->grid_n_int = s.grid.n_int;
    out->grid_G = s.grid.G;
    // the FFT size of the order k of the last iteration or force evaluation
    out->fft_P = (s.grid.k >= 1 && s.grid.k <= kMaxK && g->logP_k[s.grid.k]) ? (1 << g->logP_k[s.grid.k]) : g->P;
    out->spectrum_builds = s.spec_builds;
    out->device_flags = (int32_t)(s.flags | g->flags_seen);
    out->kernels_per_iteration = kernels_per_iteration(g);
    out->grid_k = s.grid.k;
    return TFDP_OK;
}

tfdp_status tfdp_set_node_weights(tfdp_graph* g, const float* w_rep, const float* w_att, int on_device) {
    if (!g) return TFDP_ERR_INVALID_ARG;
    const size_t n = (size_t)g->n;
    if (n == 0) return TFDP_OK;
    // validate both arrays before anything changes
    std::vector<float> h[2];
    float wmax[2] = {0.0f, 0.0f};
    const float* src[2] = {w_rep, w_att};
    for (int q = 0; q < 2; ++q) {
        if (!src[q]) continue;
        h[q].resize(n);
        if (on_device) CK(cudaMemcpy(h[q].data(), src[q], sizeof(float) * n, cudaMemcpyDeviceToHost));
        else std::memcpy(h[q].data(), src[q], sizeof(float) * n);
        for (size_t i = 0; i < n; ++i) {
            const float v = h[q][i];
            if (!(v >= 0.0f && v <= TFDP_WEIGHT_MAX)) return TFDP_ERR_PARAM_RANGE;  // also NaN
            wmax[q] = std::max(wmax[q], v);
        }
    }
    CK(cudaStreamSynchronize(g->stream));  // no queued iteration still reads the old weights
    float** dst[2] = {&g->wrep, &g->watt};
    for (int q = 0; q < 2; ++q) {
        if (!src[q]) continue;
        if (!*dst[q]) CK(cudaMalloc(dst[q], sizeof(float) * n));
        CK(cudaMemcpy(*dst[q], h[q].data(), sizeof(float) * n, cudaMemcpyHostToDevice));
    }
    if (w_rep && !g->vwr) CK(cudaMalloc(&g->vwr, sizeof(float) * n));
    g->use_wrep = w_rep != nullptr;
    g->use_watt = w_att != nullptr;
    // spread terms scale with r <= 2^spread_shift; the fixed-point scale shrinks to match
    int shift = 0;
    while (g->use_wrep && (float)(1 << shift) < wmax[0]) ++shift;
    g->spread_shift = shift;
    free_execs(g);  // the captured kernels carry the weight pointers
    tfdp_status st = upload_params(g);
    if (st != TFDP_OK) return st;
    CK(cudaStreamSynchronize(g->stream));
    return TFDP_OK;
}

tfdp_status tfdp_set_stage_timing_mask(tfdp_graph* g, uint32_t mask) {
    if (!g) return TFDP_ERR_INVALID_ARG;
    mask &= (1u << TFDP_NUM_STAGES) - 1u;
    if (mask && !g->ev_b[0]) {
        for (int i = 0; i < TFDP_NUM_STAGES; ++i) {
            CK(cudaEventCreate(&g->ev_b[i]));
            CK(cudaEventCreate(&g->ev_e[i]));
        }
        for (int i = 0; i < 2 * TFDP_NUM_STAGES; ++i)
            CK(cudaEventCreateWithFlags(&g->time_fork[i], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&g->time_join, cudaEventDisableTiming));
        CK(cudaStreamCreateWithFlags(&g->time_stream, cudaStreamNonBlocking));
    }
    if (mask != g->timing_mask) {
        g->timing_mask = mask;
        free_execs(g);  // recapture with the new set of event nodes
    }
    return TFDP_OK;
}

tfdp_status tfdp_set_stage_timing(tfdp_graph* g, int enable) {
    return tfdp_set_stage_timing_mask(g, enable ? (1u << TFDP_NUM_STAGES) - 1u : 0u);
}

tfdp_status tfdp_get_stage_times(tfdp_graph* g, float* ms, int nstages) {
    if (!g || !ms || nstages < 1) return TFDP_ERR_INVALID_ARG;
    if (!g->timing_mask) return TFDP_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(g->stream));
    const bool exact = g->params.rep_mode == TFDP_REP_EXACT;
    for (int i = 0; i < nstages; ++i) {
        ms[i] = 0.0f;
        if (i >= TFDP_NUM_STAGES || !((g->timing_mask >> i) & 1u)) continue;
        const bool exact_stage = i == TFDP_STAGE_EXACT || i == TFDP_STAGE_EDGE_UPDATE;
        if (exact != exact_stage) continue;  // the stage does not run in this mode
        float t = 0.0f;
        CK(cudaEventElapsedTime(&t, g->ev_b[i], g->ev_e[i]));
        ms[i] = t;
    }
    return TFDP_OK;
}

tfdp_status tfdp_synchronize(tfdp_graph* g) {
    if (!g) return TFDP_ERR_INVALID_ARG;
    return sync_checked(g);
}

tfdp_status tfdp_debug_inject(tfdp_graph* g, int what, int value) {
    if (!g || value < 0) return TFDP_ERR_INVALID_ARG;
    switch (what) {
        case TFDP_INJECT_FFT_ALLOC:
            g->inject_alloc_fail = value;
            return TFDP_OK;
        case TFDP_INJECT_SCAN_STALL: {
            CK(cudaStreamSynchronize(g->stream));  // no queued iteration reads the old parameters
            g->inject_scan_stall = value;
            tfdp_status st = upload_params(g);
            if (st != TFDP_OK) return st;
            CK(cudaStreamSynchronize(g->stream));
            return TFDP_OK;
        }
        default:
            return TFDP_ERR_INVALID_ARG;
    }
}

tfdp_status tfdp_graph_set_stream(tfdp_graph* g, void* stream) {
    if (!g) return TFDP_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(g->stream));  // work queued on the old stream completes first
    g->stream = (cudaStream_t)stream;
    return TFDP_OK;
}

tfdp_status tfdp_graph_footprint(int64_t n, int64_t m, const tfdp_params* params, size_t* bytes) {
    if (!bytes || n < 0 || m < 0) return TFDP_ERR_INVALID_ARG;
    tfdp_params p;
    if (params) p = *params;
    else tfdp_params_default(&p);
    tfdp_status st = tfdp_params_check(&p, nullptr);
    if (st != TFDP_OK) return st;
    p.rep_mode = resolve_rep_mode(p, n);
    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    const int nb = (int)std::max<int64_t>(1, (n + 256 * kExactTargets - 1) / (256 * kExactTargets));
    const int nchunks = exact_chunks(nb, n);
    size_t b = 0;
    b += sizeof(float2) * nn * (4 + (size_t)nchunks) + sizeof(int) * (nn + 1) + sizeof(int) * (size_t)(2 * m);
    b += sizeof(int) * (size_t)std::min<int64_t>((int64_t)nn, 2 * m / (kHeavyDegree + 1) + 1);  // hub list bound
    b += sizeof(DevParams) + sizeof(DevState) + sizeof(double) * (size_t)p.total_iters + 16 * 256;
    if (p.rep_mode == TFDP_REP_FFT) {
        int P, logP, G_max, nbox_max;
        if (!fft_geometry(p, &P, &logP, &G_max, &nbox_max)) return TFDP_ERR_PARAM_RANGE;
        const size_t Gs = align_up((size_t)G_max, 4), ys = align_up((size_t)G_max, 32), NH = (size_t)P / 2 + 1;
        b += sizeof(int) * (align_up((size_t)nbox_max, 8192) + nbox_max + 1) + 8 * 1024;
        b += nn * (sizeof(int2) + 2 * sizeof(int) + 2 * sizeof(float2));
        b += sizeof(float) * 3 * Gs * Gs + 2 * sizeof(float2) * 3 * NH * ys + sizeof(float4) * Gs * Gs;
        b += sizeof(float2) * 3 * NH * P + 3 * sizeof(float) * NH * P + sizeof(float2) * P + 32 * 256;
        b += 3 * sizeof(float2) * P + 3 * 256;  // per-k twiddle tables (each at most P entries)
        if (p.precision == TFDP_PREC_BF16X3)
            b += tc_constants_bytes() + sizeof(float) * tc_spectrum_floats() + 2 * 256;
    }
    *bytes = b;
    return TFDP_OK;
}

tfdp_status tfdp_destroy_graph(tfdp_graph* g) {
    if (!g) return TFDP_OK;
    if (g->stream || g->cap_stream) cudaStreamSynchronize(g->stream);
    free_execs(g);
    for (int i = 0; i < TFDP_NUM_STAGES; ++i) {
        if (g->ev_b[i]) cudaEventDestroy(g->ev_b[i]);
        if (g->ev_e[i]) cudaEventDestroy(g->ev_e[i]);
    }
    for (int i = 0; i < 2 * TFDP_NUM_STAGES; ++i)
        if (g->time_fork[i]) cudaEventDestroy(g->time_fork[i]);
    if (g->time_join) cudaEventDestroy(g->time_join);
    if (g->time_stream) {
        cudaStreamSynchronize(g->time_stream);
        cudaStreamDestroy(g->time_stream);
    }
    if (g->fft_mem) cudaFree(g->fft_mem);
    if (g->node_mem) cudaFree(g->node_mem);
    if (g->wrep) cudaFree(g->wrep);
    if (g->watt) cudaFree(g->watt);
    if (g->vwr) cudaFree(g->vwr);
    if (g->step_table) cudaFree(g->step_table);
    if (g->side_stream) cudaStreamSynchronize(g->side_stream);
    if (g->fork_ev) cudaEventDestroy(g->fork_ev);
    if (g->join_ev) cudaEventDestroy(g->join_ev);
    if (g->side_stream) cudaStreamDestroy(g->side_stream);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    delete g;
    return TFDP_OK;
}

tfdp_status tfdp_debug_fetch(tfdp_graph* g, int what, void* dst, size_t bytes) {
    if (!g || !dst) return TFDP_ERR_INVALID_ARG;
    DevState s;
    CK(cudaMemcpyAsync(&s, g->dst, sizeof(DevState), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    const size_t G = (size_t)s.grid.G;
    if (what == TFDP_DEBUG_SORT_PERM) {
        // the latest sort wrote visit order (t & 1) ^ 1 of its iteration t
        const int slot = g->last_was_eval ? (int)((g->host_iter & 1) ^ 1) : (int)(g->host_iter & 1);
        if (!g->vperm[slot] || bytes < sizeof(int) * (size_t)g->n) return TFDP_ERR_INVALID_ARG;
        CK(cudaMemcpy(dst, g->vperm[slot], sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToHost));
        return TFDP_OK;
    }
    if (what == TFDP_DEBUG_CELL_START) {
        const size_t nb = (size_t)s.grid.n_int * s.grid.n_int + 1;
        if (!g->off || bytes < sizeof(int) * nb) return TFDP_ERR_INVALID_ARG;
        CK(cudaMemcpy(dst, g->off, sizeof(int) * nb, cudaMemcpyDeviceToHost));
        return TFDP_OK;
    }
    if (what == TFDP_DEBUG_GRID_CHARGES) {
        if (!g->gin || bytes < sizeof(float) * 3 * G * G) return TFDP_ERR_INVALID_ARG;
        for (int c = 0; c < 3; ++c)
            CK(cudaMemcpy2D((char*)dst + sizeof(float) * G * G * c, sizeof(float) * G,
                            g->gin + (size_t)c * g->Gs * g->Gs, sizeof(float) * g->Gs, sizeof(float) * G, G,
                            cudaMemcpyDeviceToHost));
        return TFDP_OK;
    }
    if (what == TFDP_DEBUG_GRID_OUTPUT) {
        if (!g->gout || bytes < sizeof(float4) * G * G) return TFDP_ERR_INVALID_ARG;
        CK(cudaMemcpy2D(dst, sizeof(float4) * G, g->gout, sizeof(float4) * g->Gs, sizeof(float4) * G, G,
                        cudaMemcpyDeviceToHost));
        return TFDP_OK;
    }
    return TFDP_ERR_INVALID_ARG;
}

}  // extern "C"
