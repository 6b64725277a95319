// fft_kernels.cu -- grid interaction of the ibFFT repulsion (arXiv 2303.03964, Sec. 3.4,
// second step) as a zero-padded 2D FFT convolution on a P x P circulant, P >= 2G - 1.
//
// The GPU evaluates the well-conditioned form of Eq. (Fr1)/(Fr2):
//   x_i psi_1(i) - psi_x(i) = sum_p w_ip [ (x_i - y_p) A_p + O^x_p ],
//   A = K * rho,   O^x = (Delta_x K) * rho - K * m^x   (and likewise for y),
// with rho_q = sum_j w_jq and m^x_q = sum_j w_jq (x_j - y^x_q). It follows from
// sum_j w_jq x_j = y_q rho_q + m_q and is algebraically identical to the paper's
// three sums; every term is O(h) instead of O(|x|), which keeps FP32 accurate.
// Three transforms in (rho, m^x, m^y), three out (A, O^x, O^y), and three real
// kernel spectra: K (real, even), and Delta_x K, Delta_y K (odd, so their spectra are
// purely imaginary and stored as the imaginary part).
//
// Data flow per iteration (rows = y, columns = x, channels c = 0..2), register-resident
// transforms of fft_reg.cuh for every P = 128 .. 8192:
//   k_rows_fwd_r  one channel of a row block per CTA: real -> half spectrum along x
//                 (P/2+1 bins), two real rows packed in one complex transform; written
//                 column-major T1[c][kx][y] so the column pass reads contiguous data.
//   k_cols_r      per kx: forward along y, spectral product, inverse along y (the
//                 digit-reversed order of the forward output is never undone), keep y < G.
//   k_rows_inv_r  per row pair: complex-to-real along x, keep x < G, write the grid
//                 as float4 (A, O^x, O^y, 0) per node for the gather.
// The kernel spectrum is rebuilt inside the row and column passes (extra blocks of
// k_rows_fwd_r sample the kernels; k_cols_r transforms them along y) only in an
// iteration whose box side, gamma, k or P changed.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "fft.cuh"
#include "fft_reg.cuh"
#include "fft_stages.cuh"
#include "launch.h"

namespace tfdp {

constexpr int kRowsFwdPairs = 2;      // row pairs per thread in the forward row pass at P = 2048
constexpr int kRowsFwdMinBlocks = 4;  // its CTAs per SM then (64 registers)
constexpr int kRowsInvPairs = 2;      // row pairs per thread in the inverse row pass at P = 2048

// Row passes that keep one channel in registers at a time (the *_seq bodies): P = 8192,
// whose sequence fills a CTA. (At P = 2048 the same bodies at four CTAs per SM, one wave
// for the 512 row pairs of a 1023-row grid, measured 4 % slower than three channels at
// three CTAs per SM.)
template <int LOGP>
struct SeqRows {
    static constexpr bool value = RegGeom<LOGP>::T > 512;
    static constexpr int min_blocks = RegGeom<LOGP>::T * RegGeom<LOGP>::RG <= 256 ? 3 : 1;
};

// Forward row pass: one CTA per (row block, channel) below P = 8192, so that a CTA holds
// one sequence of eight values per thread (smaller CTAs, more of them per SM); at
// P = 8192 one CTA per row pair takes its three channels in turn (SeqRows).
template <int LOGP>
struct RowsFwdGeom {
    static constexpr bool seq = SeqRows<LOGP>::value;
    static constexpr int ch = seq ? 1 : 3;  // CTAs per row block
    // row pairs a thread transforms in turn: 2 at P = 2048 (T = 256, one pair per CTA
    // otherwise), so that every block writes 32-byte runs of its output columns
    static constexpr int rp = (!seq && RegGeom<LOGP>::T == 256) ? kRowsFwdPairs : 1;
    static constexpr int rows = 2 * RegGeom<LOGP>::RG * (seq ? 1 : rp);  // rows per block
    static constexpr size_t smem =
        seq ? RegGeom<LOGP>::rows_smem : (size_t)RegGeom<LOGP>::RG * rp * RegGeom<LOGP>::P * sizeof(float2);
    static constexpr int min_blocks = seq ? 1 : (rp > 1 ? kRowsFwdMinBlocks : 5);
};

// Blocks [0, ch data_blocks): channel b % ch of row block b / ch of the spread grid into
// T1. The ch spec_blocks blocks after that: the same for the rows of the sampled kernels
// into S1, each taking every spec_blocks-th row block, only in an iteration that rebuilds
// the spectrum (otherwise they return at once, so they are kept few).
template <int LOGP>
__global__ void __launch_bounds__(RegGeom<LOGP>::T * RegGeom<LOGP>::RG, RowsFwdGeom<LOGP>::min_blocks)
    k_rows_fwd_r(GridSource gsrc, int data_blocks, int spec_blocks, float2* __restrict__ T1, int ystride,
                 float2* __restrict__ S1, const float2* __restrict__ tw, const DevState* __restrict__ st,
                 const DevParams* __restrict__ prm) {
    extern __shared__ float2 sm[];
    pdl_wait();
    pdl_trigger();
    using Fg = RowsFwdGeom<LOGP>;
    constexpr int P = 1 << LOGP;
    const int rb = (int)blockIdx.x / Fg::ch;
    const int c = (int)blockIdx.x - rb * Fg::ch;
    if (rb < data_blocks) {
        if constexpr (Fg::seq) rows_fwd_body_seq<LOGP>(gsrc, st->grid.G, rb, T1, ystride, tw, sm);
        else rows_fwd_body_ch<LOGP, GridSource, Fg::rp>(gsrc, c, st->grid.G, rb, T1, ystride, tw, sm);
    } else {
        if (st->spec_dirty == 0) return;
        KernelSource ks;
        ks.P = P;
        ks.bind(st, prm);
        constexpr int kRowBlocks = (spec_rows(P) + Fg::rows - 1) / Fg::rows;
        for (int sb = rb - data_blocks; sb < kRowBlocks; sb += spec_blocks) {
            if constexpr (Fg::seq) rows_fwd_body_seq<LOGP>(ks, P, sb, S1, P, tw, sm);
            else rows_fwd_body_ch<LOGP, KernelSource, Fg::rp>(ks, c, P, sb, S1, P, tw, sm);
            __syncthreads();  // the next row block's exchanges reuse sm
        }
    }
}

template <int LOGP>
__global__ void __launch_bounds__(RegGeom<LOGP>::T * RegGeom<LOGP>::CG, RegGeom<LOGP>::T * RegGeom<LOGP>::CG <= 256 ? 3 : 1)
    k_cols_r(const float2* __restrict__ T1, float2* __restrict__ T2, int ystride, float* __restrict__ specK,
             float* __restrict__ specHx, float* __restrict__ specHy, const float2* __restrict__ S1,
             const float2* __restrict__ tw, const DevState* __restrict__ st) {
    extern __shared__ float2 sm[];
    pdl_wait();
    pdl_trigger();
    if constexpr (RegGeom<LOGP>::T > 512)
        cols_body_seq<LOGP>(blockIdx.x, T1, T2, ystride, specK, specHx, specHy, S1, tw, st->grid.G, st->spec_dirty,
                            sm);
    else
        cols_body<LOGP>(blockIdx.x, T1, T2, ystride, specK, specHx, specHy, S1, tw, st->grid.G, st->spec_dirty, sm);
}

// Inverse row pass: two row pairs per thread at P = 2048 (as the forward pass), read as
// 32-byte runs of their half-spectrum columns.
template <int LOGP>
struct RowsInvGeom {
    static constexpr int rp = (!SeqRows<LOGP>::value && RegGeom<LOGP>::T == 256) ? kRowsInvPairs : 1;
    static constexpr int rows = 2 * RegGeom<LOGP>::RG * rp;  // rows per block
    static constexpr size_t smem = RegGeom<LOGP>::rows_smem * rp;
};

template <int LOGP>
__global__ void __launch_bounds__(RegGeom<LOGP>::T * RegGeom<LOGP>::RG, SeqRows<LOGP>::min_blocks)
    k_rows_inv_r(const float2* __restrict__ T2, int ystride, float4* __restrict__ gout, int Gs,
                 const float2* __restrict__ tw, const DevState* __restrict__ st) {
    extern __shared__ float2 sm[];
    pdl_wait();
    pdl_trigger();
    if constexpr (SeqRows<LOGP>::value) rows_inv_body_seq<LOGP>(blockIdx.x, T2, ystride, gout, Gs, tw, st->grid.G, sm);
    else rows_inv_body<LOGP, RowsInvGeom<LOGP>::rp>(blockIdx.x, T2, ystride, gout, Gs, tw, st->grid.G, sm);
}

// ---------------------------------------------------------------- launchers
template <int LOGP>
static cudaError_t set_attrs() {
    using Rg = RegGeom<LOGP>;
    cudaError_t e;
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if ((e = cudaFuncSetAttribute(k_rows_fwd_r<LOGP>, A, (int)RowsFwdGeom<LOGP>::smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_cols_r<LOGP>, A, (int)Rg::cols_smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_rows_inv_r<LOGP>, A, (int)RowsInvGeom<LOGP>::smem)) != cudaSuccess) return e;
    return cudaSuccess;
}

template <int LOGP>
static cudaError_t ensure_attrs() {
    static cudaError_t once = set_attrs<LOGP>();
    return once;
}

cudaError_t prepare_fft(int logP) {
    switch (logP) {
        case 7: return set_attrs<7>();
        case 8: return set_attrs<8>();
        case 9: return set_attrs<9>();
        case 10: return set_attrs<10>();
        case 11: return set_attrs<11>();
        case 12: return set_attrs<12>();
        case 13: return set_attrs<13>();
        default: return cudaErrorInvalidValue;
    }
}

// The spectrum needs no launch of its own: the row and column passes rebuild it.
cudaError_t launch_spectrum(const FftLaunch& a, cudaStream_t) {
    return (a.logP >= 7 && a.logP <= 13) ? cudaSuccess : cudaErrorInvalidValue;
}

template <int LOGP>
static cudaError_t launch_rows_fwd_impl(const FftLaunch& a, cudaStream_t s) {
    using Rg = RegGeom<LOGP>;
    using Fg = RowsFwdGeom<LOGP>;
    cudaError_t e = ensure_attrs<LOGP>();
    if (e != cudaSuccess) return e;
    GridSource gs;
    gs.gin = a.gin;
    gs.Gs = a.Gs;
    const int blocks = (a.G_max + Fg::rows - 1) / Fg::rows;
    // spectrum row blocks: about two per SM and channel, each looping over its share
    const int spec_blocks = std::min((spec_rows(Rg::P) + Fg::rows - 1) / Fg::rows, 2 * 152);
    return launch_pdl(k_rows_fwd_r<LOGP>, Fg::ch * (blocks + spec_blocks), Rg::T * Rg::RG, Fg::smem, s, gs, blocks,
                      spec_blocks, a.T1, a.ystride, a.S1, a.tw, (const DevState*)a.st, (const DevParams*)a.prm);
}

template <int LOGP>
static cudaError_t launch_cols_impl(const FftLaunch& a, cudaStream_t s) {
    using Rg = RegGeom<LOGP>;
    cudaError_t e = ensure_attrs<LOGP>();
    if (e != cudaSuccess) return e;
    const int blocks = (Rg::P / 2 + 1 + Rg::CG - 1) / Rg::CG;
    return launch_pdl(k_cols_r<LOGP>, blocks, Rg::T * Rg::CG, Rg::cols_smem, s, (const float2*)a.T1, a.T2, a.ystride,
                      a.specK, a.specHx, a.specHy, (const float2*)a.S1, (const float2*)a.tw, (const DevState*)a.st);
}

template <int LOGP>
static cudaError_t launch_rows_inv_impl(const FftLaunch& a, cudaStream_t s) {
    using Rg = RegGeom<LOGP>;
    cudaError_t e = ensure_attrs<LOGP>();
    if (e != cudaSuccess) return e;
    using Ig = RowsInvGeom<LOGP>;
    const int blocks = (a.G_max + Ig::rows - 1) / Ig::rows;
    return launch_pdl(k_rows_inv_r<LOGP>, blocks, Rg::T * Rg::RG, Ig::smem, s, (const float2*)a.T2, a.ystride,
                      a.gout, a.Gs, (const float2*)a.tw, (const DevState*)a.st);
}

#define TFDP_LOGP_SWITCH(FN)                      \
    switch (a.logP) {                             \
        case 7: return FN<7>(a, s);               \
        case 8: return FN<8>(a, s);               \
        case 9: return FN<9>(a, s);               \
        case 10: return FN<10>(a, s);             \
        case 11: return FN<11>(a, s);             \
        case 12: return FN<12>(a, s);             \
        case 13: return FN<13>(a, s);             \
        default: return cudaErrorInvalidValue;    \
    }

cudaError_t launch_rows_fwd(const FftLaunch& a, cudaStream_t s) { TFDP_LOGP_SWITCH(launch_rows_fwd_impl) }
cudaError_t launch_cols(const FftLaunch& a, cudaStream_t s) { TFDP_LOGP_SWITCH(launch_cols_impl) }
cudaError_t launch_rows_inv(const FftLaunch& a, cudaStream_t s) { TFDP_LOGP_SWITCH(launch_rows_inv_impl) }

}  // namespace tfdp
