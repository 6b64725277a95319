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
// Data flow per iteration (rows = y, columns = x, channels c = 0..2):
//   k_rows_fwd  G rows x 3 channels, real -> half spectrum along x (P/2+1 bins),
//               two real rows packed in one complex transform; written column-major
//               T1[c][kx][y] so the column pass reads contiguous data.
//   k_cols      per kx: forward along y, spectral product, inverse along y (the
//               digit-reversed order of the forward output is never undone), keep y < G.
//   k_rows_inv  per row pair: complex-to-real along x, keep x < G, write the grid
//               as float4 (A, O^x, O^y, 0) per node for the gather.
// The kernel spectrum (k_rows_fwd with a sampling source + k_spec_cols) is rebuilt
// only when the box side, gamma, k or P change.
#include <cuda_runtime.h>

#include "common.cuh"
#include "fft.cuh"
#include "fft_reg.cuh"
#include "fft_stages.cuh"
#include "launch.h"

namespace tfdp {

// ---------------------------------------------------------------- forward rows
// RPC grid rows per CTA (x 3 channels): 3 RPC / 2 complex sequences of length P.
template <int LOGP, int RPC, class Src>
__global__ void __launch_bounds__(256) k_rows_fwd(Src src, float2* __restrict__ T1, int ystride,
                                                  const float2* __restrict__ tw,
                                                  const DevState* __restrict__ st,
                                                  const DevParams* __restrict__ prm) {
    constexpr int P = 1 << LOGP;
    constexpr int PL = padded_len(P);
    constexpr int NSEQ = 3 * RPC / 2;
    constexpr int NH = P / 2 + 1;
    extern __shared__ float2 sm[];
    if (!src.active(st)) return;
    src.bind(st, prm);
    const int nrows = src.rows(st);
    const int y0 = blockIdx.x * RPC;
    if (y0 >= nrows) return;
    const int G = nrows;
    // sequence q: channel c = q / (RPC/2), rows y0 + 2*(q % (RPC/2)) and the next one
    for (int idx = threadIdx.x; idx < NSEQ * P; idx += blockDim.x) {
        const int q = idx / P;
        const int x = idx - q * P;
        const int c = q / (RPC / 2);
        const int y = y0 + 2 * (q % (RPC / 2));
        sm[q * PL + spad(x)] = make_float2(src(c, y, x, G), src(c, y + 1, x, G));
    }
    __syncthreads();
    fft_forward<LOGP>(sm, NSEQ, tw);
    // split each packed transform Z = FFT(a + i b) into A = FFT(a), B = FFT(b):
    // A_k = (Z_k + conj Z_{P-k}) / 2, B_k = (Z_k - conj Z_{P-k}) / (2i)
    for (int idx = threadIdx.x; idx < 3 * NH; idx += blockDim.x) {
        const int c = idx / NH;
        const int kx = idx - c * NH;
        const int pk = spad(pos_of_freq<LOGP>(kx));
        const int pn = spad(pos_of_freq<LOGP>((P - kx) & (P - 1)));
        float2 out[RPC];
#pragma unroll
        for (int s = 0; s < RPC / 2; ++s) {
            const float2* seq = sm + (c * (RPC / 2) + s) * PL;
            const float2 Z = seq[pk], W = seq[pn];
            out[2 * s] = make_float2(0.5f * (Z.x + W.x), 0.5f * (Z.y - W.y));
            out[2 * s + 1] = make_float2(0.5f * (Z.y + W.y), 0.5f * (W.x - Z.x));
        }
        float2* dst = T1 + ((size_t)c * NH + kx) * ystride + y0;
        if (RPC == 4) {
            reinterpret_cast<float4*>(dst)[0] = make_float4(out[0].x, out[0].y, out[1].x, out[1].y);
            reinterpret_cast<float4*>(dst)[1] = make_float4(out[2].x, out[2].y, out[3].x, out[3].y);
        } else {
            reinterpret_cast<float4*>(dst)[0] = make_float4(out[0].x, out[0].y, out[1].x, out[1].y);
        }
    }
}

// ---------------------------------------------------------------- columns
// One CTA per kx in [0, P/2]: forward along y of (rho, m^x, m^y), spectral product
//   A = K rho,  O^x = i hx rho - K m^x,  O^y = i hy rho - K m^y
// (spectra pre-scaled by 1 / P^2 and stored in the digit-reversed order of the
// forward transform), inverse along y, keep y < G.
template <int LOGP>
__global__ void __launch_bounds__(256) k_cols(const float2* __restrict__ T1, float2* __restrict__ T2,
                                              int ystride, const float* __restrict__ specK,
                                              const float* __restrict__ specHx,
                                              const float* __restrict__ specHy,
                                              const float2* __restrict__ tw,
                                              const DevState* __restrict__ st) {
    constexpr int P = 1 << LOGP;
    constexpr int PL = padded_len(P);
    constexpr int NH = P / 2 + 1;
    extern __shared__ float2 sm[];
    const int kx = blockIdx.x;
    const int G = st->grid.G;
    for (int idx = threadIdx.x; idx < 3 * P; idx += blockDim.x) {
        const int c = idx / P;
        const int y = idx - c * P;
        sm[c * PL + spad(y)] = (y < G) ? T1[((size_t)c * NH + kx) * ystride + y] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    fft_forward<LOGP>(sm, 3, tw);
    const size_t so = (size_t)kx * P;
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        const int a = spad(p);
        const float2 r = sm[a], mx = sm[PL + a], my = sm[2 * PL + a];
        const float K = __ldg(specK + so + p), hx = __ldg(specHx + so + p), hy = __ldg(specHy + so + p);
        sm[a] = make_float2(K * r.x, K * r.y);
        sm[PL + a] = make_float2(-hx * r.y - K * mx.x, hx * r.x - K * mx.y);
        sm[2 * PL + a] = make_float2(-hy * r.y - K * my.x, hy * r.x - K * my.y);
    }
    __syncthreads();
    fft_inverse<LOGP>(sm, 3, tw);
    for (int idx = threadIdx.x; idx < 3 * G; idx += blockDim.x) {
        const int c = idx / G;
        const int y = idx - c * G;
        T2[((size_t)c * NH + kx) * ystride + y] = sm[c * PL + spad(y)];
    }
}

// Spectrum columns: forward along y of the three sampled kernels, keep the real part
// of FFT(K) and the imaginary parts of FFT(Delta_x K), FFT(Delta_y K), scaled by 1/P^2.
template <int LOGP>
__global__ void __launch_bounds__(256) k_spec_cols(const float2* __restrict__ S1, float* __restrict__ specK,
                                                   float* __restrict__ specHx, float* __restrict__ specHy,
                                                   const float2* __restrict__ tw,
                                                   const DevState* __restrict__ st) {
    constexpr int P = 1 << LOGP;
    constexpr int PL = padded_len(P);
    constexpr int NH = P / 2 + 1;
    extern __shared__ float2 sm[];
    if (st->spec_dirty == 0) return;
    const int kx = blockIdx.x;
    for (int idx = threadIdx.x; idx < 3 * P; idx += blockDim.x) {
        const int c = idx / P;
        const int y = idx - c * P;
        sm[c * PL + spad(y)] = S1[((size_t)c * NH + kx) * P + y];
    }
    __syncthreads();
    fft_forward<LOGP>(sm, 3, tw);
    const float inv = 1.0f / ((float)P * (float)P);
    const size_t so = (size_t)kx * P;
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        const int a = spad(p);
        specK[so + p] = sm[a].x * inv;
        specHx[so + p] = sm[PL + a].y * inv;
        specHy[so + p] = sm[2 * PL + a].y * inv;
    }
}

// ---------------------------------------------------------------- inverse rows
// RPC rows per CTA: complex-to-real along x, two real rows per complex transform,
// then write (A, O^x, O^y, 0) for x < G.
template <int LOGP, int RPC>
__global__ void __launch_bounds__(256) k_rows_inv(const float2* __restrict__ T2, int ystride,
                                                  float4* __restrict__ gout, int Gs,
                                                  const float2* __restrict__ tw,
                                                  const DevState* __restrict__ st) {
    constexpr int P = 1 << LOGP;
    constexpr int PL = padded_len(P);
    constexpr int NSEQ = 3 * RPC / 2;
    constexpr int NH = P / 2 + 1;
    extern __shared__ float2 sm[];
    const int G = st->grid.G;
    const int y0 = blockIdx.x * RPC;
    if (y0 >= G) return;
    for (int idx = threadIdx.x; idx < 3 * NH; idx += blockDim.x) {
        const int c = idx / NH;
        const int kx = idx - c * NH;
        const float2* src = T2 + ((size_t)c * NH + kx) * ystride + y0;
        float2 X[RPC];
        const float4 v0 = reinterpret_cast<const float4*>(src)[0];
        X[0] = make_float2(v0.x, v0.y);
        X[1] = make_float2(v0.z, v0.w);
        if (RPC == 4) {
            const float4 v1 = reinterpret_cast<const float4*>(src)[1];
            X[2] = make_float2(v1.x, v1.y);
            X[3] = make_float2(v1.z, v1.w);
        }
        const int pk = spad(pos_of_freq<LOGP>(kx));
        const int pn = spad(pos_of_freq<LOGP>((P - kx) & (P - 1)));
#pragma unroll
        for (int s = 0; s < RPC / 2; ++s) {
            float2* seq = sm + (c * (RPC / 2) + s) * PL;
            // rows at or past G were never written by the column pass: use zeros there
            const float2 zero = make_float2(0.0f, 0.0f);
            const float2 a = (y0 + 2 * s < G) ? X[2 * s] : zero;
            const float2 b = (y0 + 2 * s + 1 < G) ? X[2 * s + 1] : zero;
            // Z_k = A_k + i B_k ; Z_{P-k} = conj(A_k) + i conj(B_k)
            seq[pk] = make_float2(a.x - b.y, a.y + b.x);
            if (kx != 0 && kx != P / 2) seq[pn] = make_float2(a.x + b.y, b.x - a.y);
        }
    }
    __syncthreads();
    fft_inverse<LOGP>(sm, NSEQ, tw);
    for (int idx = threadIdx.x; idx < RPC * G; idx += blockDim.x) {
        const int dy = idx / G;
        const int x = idx - dy * G;
        if (y0 + dy >= G) continue;
        const int s = dy >> 1;
        const int a = spad(x);
        float v[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 z = sm[(c * (RPC / 2) + s) * PL + a];
            v[c] = (dy & 1) ? z.y : z.x;
        }
        gout[(size_t)(y0 + dy) * Gs + x] = make_float4(v[0], v[1], v[2], 0.0f);
    }
}

// Row passes that keep one channel in registers at a time (the *_seq bodies): P = 8192,
// whose sequence fills a CTA. (At P = 2048 the same bodies at four CTAs per SM, one wave
// for the 512 row pairs of a 1023-row grid, measured 4 % slower than three channels at
// three CTAs per SM.)
template <int LOGP>
struct SeqRows {
    static constexpr bool value = RegGeom<LOGP>::T > 512;
    static constexpr int min_blocks = RegGeom<LOGP>::T * RegGeom<LOGP>::RG <= 256 ? 3 : 1;
};

// Blocks [0, data_blocks): rows of the spread grid into T1. Blocks after that: rows of
// the sampled kernels into S1, only in an iteration that rebuilds the spectrum.
template <int LOGP>
__global__ void __launch_bounds__(RegGeom<LOGP>::T * RegGeom<LOGP>::RG, SeqRows<LOGP>::min_blocks)
    k_rows_fwd_r(GridSource gsrc, int data_blocks, float2* __restrict__ T1, int ystride, float2* __restrict__ S1,
                 const float2* __restrict__ tw, const DevState* __restrict__ st, const DevParams* __restrict__ prm) {
    extern __shared__ float2 sm[];
    pdl_wait();
    pdl_trigger();
    // sizes whose sequence fills the CTA keep one channel in registers at a time
    constexpr bool kSeq = SeqRows<LOGP>::value;
    if ((int)blockIdx.x < data_blocks) {
        if constexpr (kSeq) rows_fwd_body_seq<LOGP>(gsrc, st->grid.G, blockIdx.x, T1, ystride, tw, sm);
        else rows_fwd_body<LOGP>(gsrc, st->grid.G, blockIdx.x, T1, ystride, tw, sm);
    } else {
        if (st->spec_dirty == 0) return;
        KernelSource ks;
        ks.P = 1 << LOGP;
        ks.bind(st, prm);
        if constexpr (kSeq) rows_fwd_body_seq<LOGP>(ks, ks.P, blockIdx.x - data_blocks, S1, 1 << LOGP, tw, sm);
        else rows_fwd_body<LOGP>(ks, ks.P, blockIdx.x - data_blocks, S1, 1 << LOGP, tw, sm);
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

template <int LOGP>
__global__ void __launch_bounds__(RegGeom<LOGP>::T * RegGeom<LOGP>::RG, SeqRows<LOGP>::min_blocks)
    k_rows_inv_r(const float2* __restrict__ T2, int ystride, float4* __restrict__ gout, int Gs,
                 const float2* __restrict__ tw, const DevState* __restrict__ st) {
    extern __shared__ float2 sm[];
    pdl_wait();
    pdl_trigger();
    if constexpr (SeqRows<LOGP>::value) rows_inv_body_seq<LOGP>(blockIdx.x, T2, ystride, gout, Gs, tw, st->grid.G, sm);
    else rows_inv_body<LOGP>(blockIdx.x, T2, ystride, gout, Gs, tw, st->grid.G, sm);
}

// ---------------------------------------------------------------- launchers
template <int LOGP>
struct FftGeom {
    static constexpr int P = 1 << LOGP;
    // 4 grid rows per CTA while two CTAs fit on an SM, else 2
    static constexpr int RPC = (padded_len(P) * 6 * 8 <= 113 * 1024) ? 4 : 2;
    static constexpr size_t rows_smem = (size_t)3 * RPC / 2 * padded_len(P) * sizeof(float2);
    static constexpr size_t cols_smem = (size_t)3 * padded_len(P) * sizeof(float2);
};

constexpr int kMaxRegLogP = 13;  // register-resident path up to P = 8192 (one channel at a time there)

template <int LOGP>
static cudaError_t set_attrs() {
    using Gm = FftGeom<LOGP>;
    constexpr int RPC = Gm::RPC;
    cudaError_t e;
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if ((e = cudaFuncSetAttribute(k_rows_fwd<LOGP, RPC, GridSource>, A, (int)Gm::rows_smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_rows_fwd<LOGP, RPC, KernelSource>, A, (int)Gm::rows_smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_rows_inv<LOGP, RPC>, A, (int)Gm::rows_smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_cols<LOGP>, A, (int)Gm::cols_smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_spec_cols<LOGP>, A, (int)Gm::cols_smem)) != cudaSuccess) return e;
    if (LOGP <= kMaxRegLogP) {
        using Rg = RegGeom<(LOGP <= kMaxRegLogP ? LOGP : kMaxRegLogP)>;
        constexpr int L = (LOGP <= kMaxRegLogP ? LOGP : kMaxRegLogP);
        if ((e = cudaFuncSetAttribute(k_rows_fwd_r<L>, A, (int)Rg::rows_smem)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_cols_r<L>, A, (int)Rg::cols_smem)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_rows_inv_r<L>, A, (int)Rg::rows_smem)) != cudaSuccess) return e;
    }
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

template <int LOGP>
static cudaError_t launch_spectrum_impl(const FftLaunch& a, cudaStream_t s) {
    using Gm = FftGeom<LOGP>;
    constexpr int P = Gm::P;
    // the register-resident kernels rebuild the spectrum inside the row and column passes
    if (LOGP <= kMaxRegLogP) return cudaSuccess;
    cudaError_t e = ensure_attrs<LOGP>();
    if (e != cudaSuccess) return e;
    KernelSource ks;
    ks.P = P;
    ks.s = 0.0f;
    ks.s2 = 0.0f;
    ks.gamma = 0.0f;
    ks.gamma_int = 0;
    k_rows_fwd<LOGP, Gm::RPC, KernelSource><<<P / Gm::RPC, 256, Gm::rows_smem, s>>>(ks, a.S1, P, a.tw, a.st, a.prm);
    k_spec_cols<LOGP><<<P / 2 + 1, 256, Gm::cols_smem, s>>>(a.S1, a.specK, a.specHx, a.specHy, a.tw, a.st);
    return cudaGetLastError();
}

template <int LOGP>
static cudaError_t launch_rows_fwd_impl(const FftLaunch& a, cudaStream_t s) {
    using Gm = FftGeom<LOGP>;
    cudaError_t e = ensure_attrs<LOGP>();
    if (e != cudaSuccess) return e;
    GridSource gs;
    gs.gin = a.gin;
    gs.Gs = a.Gs;
    if (LOGP <= kMaxRegLogP) {
        constexpr int L = (LOGP <= kMaxRegLogP ? LOGP : kMaxRegLogP);
        using Rg = RegGeom<L>;
        const int blocks = (a.G_max + 2 * Rg::RG - 1) / (2 * Rg::RG);
        const int spec_blocks = Rg::P / (2 * Rg::RG);
        return launch_pdl(k_rows_fwd_r<L>, blocks + spec_blocks, Rg::T * Rg::RG, Rg::rows_smem, s, gs, blocks, a.T1,
                          a.ystride, a.S1, a.tw, (const DevState*)a.st, (const DevParams*)a.prm);
    }
    const int row_blocks = (a.G_max + Gm::RPC - 1) / Gm::RPC;
    k_rows_fwd<LOGP, Gm::RPC, GridSource><<<row_blocks, 256, Gm::rows_smem, s>>>(gs, a.T1, a.ystride, a.tw, a.st, a.prm);
    return cudaGetLastError();
}

template <int LOGP>
static cudaError_t launch_cols_impl(const FftLaunch& a, cudaStream_t s) {
    using Gm = FftGeom<LOGP>;
    constexpr int P = Gm::P;
    cudaError_t e = ensure_attrs<LOGP>();
    if (e != cudaSuccess) return e;
    if (LOGP <= kMaxRegLogP) {
        constexpr int L = (LOGP <= kMaxRegLogP ? LOGP : kMaxRegLogP);
        using Rg = RegGeom<L>;
        const int blocks = (P / 2 + 1 + Rg::CG - 1) / Rg::CG;
        return launch_pdl(k_cols_r<L>, blocks, Rg::T * Rg::CG, Rg::cols_smem, s, (const float2*)a.T1, a.T2,
                          a.ystride, a.specK, a.specHx, a.specHy, (const float2*)a.S1, (const float2*)a.tw,
                          (const DevState*)a.st);
    }
    k_cols<LOGP><<<P / 2 + 1, 256, Gm::cols_smem, s>>>(a.T1, a.T2, a.ystride, a.specK, a.specHx, a.specHy, a.tw, a.st);
    return cudaGetLastError();
}

template <int LOGP>
static cudaError_t launch_rows_inv_impl(const FftLaunch& a, cudaStream_t s) {
    using Gm = FftGeom<LOGP>;
    cudaError_t e = ensure_attrs<LOGP>();
    if (e != cudaSuccess) return e;
    if (LOGP <= kMaxRegLogP) {
        constexpr int L = (LOGP <= kMaxRegLogP ? LOGP : kMaxRegLogP);
        using Rg = RegGeom<L>;
        const int blocks = (a.G_max + 2 * Rg::RG - 1) / (2 * Rg::RG);
        return launch_pdl(k_rows_inv_r<L>, blocks, Rg::T * Rg::RG, Rg::rows_smem, s, (const float2*)a.T2, a.ystride,
                          a.gout, a.Gs, (const float2*)a.tw, (const DevState*)a.st);
    }
    const int row_blocks = (a.G_max + Gm::RPC - 1) / Gm::RPC;
    k_rows_inv<LOGP, Gm::RPC><<<row_blocks, 256, Gm::rows_smem, s>>>(a.T2, a.ystride, a.gout, a.Gs, a.tw, a.st);
    return cudaGetLastError();
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

cudaError_t launch_spectrum(const FftLaunch& a, cudaStream_t s) { TFDP_LOGP_SWITCH(launch_spectrum_impl) }
cudaError_t launch_rows_fwd(const FftLaunch& a, cudaStream_t s) { TFDP_LOGP_SWITCH(launch_rows_fwd_impl) }
cudaError_t launch_cols(const FftLaunch& a, cudaStream_t s) { TFDP_LOGP_SWITCH(launch_cols_impl) }
cudaError_t launch_rows_inv(const FftLaunch& a, cudaStream_t s) { TFDP_LOGP_SWITCH(launch_rows_inv_impl) }

int fft_rows_per_cta(int logP) {
    switch (logP) {
        case 7: return FftGeom<7>::RPC;
        case 8: return FftGeom<8>::RPC;
        case 9: return FftGeom<9>::RPC;
        case 10: return FftGeom<10>::RPC;
        case 11: return FftGeom<11>::RPC;
        case 12: return FftGeom<12>::RPC;
        case 13: return FftGeom<13>::RPC;
        default: return 0;
    }
}

}  // namespace tfdp
