// fft_stages.cuh -- the three register-resident FFT stages of the grid interaction
// (Sec. 3.4, second step) as device functions over one work item, shared by the
// single-graph kernels (fft_kernels.cu) and the batch kernels (batch_kernel.cuh).
//
// The transforms evaluate the well-conditioned form of Eq. (Fr1)/(Fr2):
//   A = K * rho,   O^x = (Delta_x K) * rho - K * m^x,   O^y likewise,
// on a zero-padded P x P circulant (P >= 2G - 1): rows forward (real to half spectrum,
// two real rows per complex transform), then per column forward / spectral product /
// inverse, then rows inverse (half spectrum to real).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"
#include "fft.cuh"
#include "fft_reg.cuh"

namespace tfdp {

// ---------------------------------------------------------------- row sources
// Spread grid: gin[c][y][x] with row stride Gs and plane stride Gs * Gs; zero outside
// the G x G grid of this iteration (the zero padding of the linear convolution).
struct GridSource {
    const float* gin;
    int Gs;
    __device__ __forceinline__ void bind(const DevState*, const DevParams*) {}
    __device__ __forceinline__ int rows(const DevState* st) const { return st->grid.G; }
    __device__ __forceinline__ bool active(const DevState* st) const { return true; }
    __device__ __forceinline__ float operator()(int c, int y, int x, int G) const {
        return (x < G && y < G) ? gin[((size_t)c * Gs + y) * Gs + x] : 0.0f;
    }
};

// Kernel samples on the P x P circulant, wraparound offsets d -> d (d < P/2) or d - P.
//   c = 0: K(D) = (1 + |D|^2 s^2)^-gamma,  c = 1: D_x s K(D),  c = 2: D_y s K(D),
// with s = h / k the grid spacing. Entries with |D_x| = P/2 or |D_y| = P/2 are zero:
// the cropped linear convolution never reads them, and zeroing keeps the odd
// kernels exactly odd (their spectra exactly imaginary).
struct KernelSource {
    int P;
    float s2, s, gamma;  // spacing^2, spacing, exponent (FP32)
    int gamma_int;
    __device__ __forceinline__ void bind(const DevState* st, const DevParams* prm) {
        const double sd = st->grid.h / (double)st->grid.k;
        s = (float)sd;
        s2 = (float)(sd * sd);
        gamma = (float)prm->gamma;
        gamma_int = prm->gamma_int;
    }
    __device__ __forceinline__ int rows(const DevState*) const { return P; }
    __device__ __forceinline__ bool active(const DevState* st) const { return st->spec_dirty != 0; }
    __device__ __forceinline__ float operator()(int c, int y, int x, int) const {
        const int half = P >> 1;
        if (x == half || y == half) return 0.0f;
        const int dx = (x < half) ? x : x - P;
        const int dy = (y < half) ? y : y - P;
        // dx^2 + dy^2 < 2^24 is exact in FP32
        const float u = fmaf((float)(dx * dx + dy * dy), s2, 1.0f);
        float K;
        if (gamma_int > 0) {  // integer gamma: u^-gamma by multiplication
            float ug = u;
            for (int q = 1; q < gamma_int; ++q) ug *= u;
            K = 1.0f / ug;
        } else {
            K = powf(u, -gamma);
        }
        if (c == 0) return K;
        return (float)(c == 1 ? dx : dy) * s * K;
    }
};

// ---------------------------------------------------------------- register-resident path
// Same transforms as k_rows_fwd / k_cols / k_rows_inv, with each thread holding eight
// values of each of its three sequences (fft_reg.cuh). RG row pairs (or columns) per
// CTA, T = P/8 threads each.
template <int LOGP>
struct RegGeom {
    static constexpr int P = 1 << LOGP;
    static constexpr int T = P / 8;
    static constexpr int RG = (T >= 256) ? 1 : 256 / T;   // row pairs per CTA (rows kernels), <= 16
    static constexpr int CG = (T >= 256) ? 1 : 256 / T;   // columns per CTA (column kernel)
    static constexpr size_t rows_smem = (size_t)RG * 3 * P * sizeof(float2);
    static constexpr size_t cols_smem = (size_t)CG * 3 * P * sizeof(float2);
};

// Frequency kx handled by split index j (0 <= j <= P/2) in the half-spectrum passes of
// the row kernels, a bijection chosen so that the digit-reversed positions (pos_of_freq)
// of the frequencies a half-warp touches fall in different shared-memory banks
// (consecutive frequencies would all share one bank pair, since the swizzle only mixes
// the low digits). Two maps: lane l of each half-warp takes kx = l P/32 + j div 16
// (every half-warp access conflict-free at P = 128, 256, 1024, 2048, 8192), or the lanes
// of a warp take frequencies P/64 apart (better at P = 512 and 4096, where the first map
// puts pairs of lanes on one bank pair). A bank model of both maps is in the CPU tests.
template <int LOGP>
__device__ __forceinline__ int split_freq(int j) {
    static_assert(LOGP >= 6, "split_freq needs P / 2 to be a multiple of 32");
    constexpr int H = 1 << (LOGP - 1);  // P / 2
    if (j >= H) return j;               // the Nyquist bin
    if constexpr (LOGP == 9 || LOGP == 12) {
        constexpr int R = H / 32;
        return (j & 31) * R + (j >> 5);
    } else {
        return (j & 15) * (H / 16) + (j >> 4);
    }
}

// Forward row transforms of row block `blk` (2 RG rows x 3 channels) of a source into
// out[c][kx][ystride] (half spectrum along x, column-major).
template <int LOGP, class Src>
__device__ __forceinline__ void rows_fwd_body(const Src& src, int nrows, int blk, float2* __restrict__ out,
                                              int ystride, const float2* __restrict__ tw, float2* sm) {
    using Gm = RegGeom<LOGP>;
    constexpr int P = Gm::P, T = Gm::T, RG = Gm::RG, NH = P / 2 + 1;
    const int G = nrows;
    const int ybase = blk * (2 * RG);
    if (ybase >= G) return;
    const int lr = threadIdx.x / T, t = threadIdx.x - lr * T;
    const int y0 = ybase + 2 * lr;
    float2* smr = sm + (size_t)lr * 3 * P;
    float2 v[3][8];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int x = t + r * T;
            v[c][r] = make_float2(src(c, y0, x, G), src(c, y0 + 1, x, G));
        }
    reg_fft_forward<LOGP, 3>(v, smr, tw, t);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 8; ++r) smr[c * P + swz(8 * t + r)] = v[c][r];
    __syncthreads();
    // split Z = FFT(a + i b) into FFT(a), FFT(b); one thread per (channel, kx) writes
    // 2 RG consecutive rows (RG row pairs) of out[c][kx][.]
    for (int idx = threadIdx.x; idx < 3 * NH; idx += blockDim.x) {
        const int c = idx / NH;
        const int kx = split_freq<LOGP>(idx - c * NH);
        const int pk = swz(pos_of_freq<LOGP>(kx));
        const int pn = swz(pos_of_freq<LOGP>((P - kx) & (P - 1)));
        float4* dst = reinterpret_cast<float4*>(out + ((size_t)c * NH + kx) * ystride + ybase);
#pragma unroll
        for (int q = 0; q < RG; ++q) {
            const float2* seq = sm + ((size_t)q * 3 + c) * P;
            const float2 Z = seq[pk], W = seq[pn];
            dst[q] = make_float4(0.5f * (Z.x + W.x), 0.5f * (Z.y - W.y), 0.5f * (Z.y + W.y), 0.5f * (W.x - Z.x));
        }
    }
}

// One 32-byte global store (a 256-bit access, sm_100 and later) of a then b; p must be
// 32-byte aligned.
__device__ __forceinline__ void st_global_v8(float2* p, float4 a, float4 b) {
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(__cvta_generic_to_global(p)),
                 "f"(a.x), "f"(a.y), "f"(a.z), "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w)
                 : "memory");
}

// Channel c only of row block `blk` (2 RG RP rows): the same transform and split as
// rows_fwd_body computes for that channel, for launches with one CTA per (row block,
// channel); sm holds RG RP sequences of P values. Each thread transforms RP row pairs in
// turn, so that the split pass writes 4 RG RP consecutive
// floats of a column: with RG RP even, as 32-byte stores (half the store instructions of
// 16-byte ones for the strided column-major output).
template <int LOGP, class Src, int RP = 1>
__device__ __forceinline__ void rows_fwd_body_ch(const Src& src, int c, int nrows, int blk, float2* __restrict__ out,
                                                 int ystride, const float2* __restrict__ tw, float2* sm) {
    using Gm = RegGeom<LOGP>;
    constexpr int P = Gm::P, T = Gm::T, RG = Gm::RG, NH = P / 2 + 1;
    constexpr int RB = RG * RP;  // row pairs of the block; pair q is rows ybase + 2q, + 1
    const int G = nrows;
    const int ybase = blk * (2 * RB);
    if (ybase >= G) return;
    const int lr = threadIdx.x / T, t = threadIdx.x - lr * T;
#pragma unroll
    for (int h = 0; h < RP; ++h) {
        const int y0 = ybase + 2 * (h * RG + lr);
        float2 v[1][8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int x = t + r * T;
            v[0][r] = make_float2(src(c, y0, x, G), src(c, y0 + 1, x, G));
        }
        float2* smr = sm + (size_t)(h * RG + lr) * P;
        reg_fft_forward<LOGP, 1>(v, smr, tw, t);
#pragma unroll
        for (int r = 0; r < 8; ++r) smr[swz(8 * t + r)] = v[0][r];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < NH; idx += blockDim.x) {
        const int kx = split_freq<LOGP>(idx);
        const int pk = swz(pos_of_freq<LOGP>(kx));
        const int pn = swz(pos_of_freq<LOGP>((P - kx) & (P - 1)));
        float2* dst = out + ((size_t)c * NH + kx) * ystride + ybase;
        float4 z[RB];
#pragma unroll
        for (int q = 0; q < RB; ++q) {
            const float2* seq = sm + (size_t)q * P;
            const float2 Z = seq[pk], W = seq[pn];
            z[q] = make_float4(0.5f * (Z.x + W.x), 0.5f * (Z.y - W.y), 0.5f * (Z.y + W.y), 0.5f * (W.x - Z.x));
        }
        if constexpr (RB % 2 == 0) {
            // ystride is a multiple of 32 and ybase of 4: dst + 2q (q even) is 32-byte aligned
#pragma unroll
            for (int q = 0; q < RB; q += 2) st_global_v8(dst + 2 * q, z[q], z[q + 1]);
        } else {
#pragma unroll
            for (int q = 0; q < RB; ++q) reinterpret_cast<float4*>(dst)[q] = z[q];
        }
    }
}

// Column block cblk (CG columns kx): forward along y of (rho, m^x, m^y) from T1,
// spectral product A = K rho, O^x = i hx rho - K m^x, O^y = i hy rho - K m^y, inverse along
// y, rows y < G to T2. When spec_dirty, the kernel spectra of these columns are first
// rebuilt from the row-transformed kernel samples in S1 (and stored).
template <int LOGP>
__device__ __forceinline__ void cols_body(int cblk, const float2* __restrict__ T1, float2* __restrict__ T2,
                                          int ystride, float* __restrict__ specK, float* __restrict__ specHx,
                                          float* __restrict__ specHy, const float2* __restrict__ S1,
                                          const float2* __restrict__ tw, int G, int spec_dirty, float2* sm) {
    using Gm = RegGeom<LOGP>;
    constexpr int P = Gm::P, T = Gm::T, NH = P / 2 + 1;
    const int lc = threadIdx.x / T, t = threadIdx.x - lc * T;
    const int kx = cblk * Gm::CG + lc;
    const bool valid = kx < NH;
    float2* smc = sm + (size_t)lc * 3 * P;
    float2 v[3][8];
    // kernel spectra at this thread's output positions 8t .. 8t+7 (digit-reversed order),
    // stored per column as two float4 planes of T entries (positions 8t + 0..3 at t,
    // 8t + 4..7 at T + t), so that a warp's loads are contiguous
    float K[8], hx[8], hy[8];
    const size_t so = (size_t)(valid ? kx : 0) * 2 * T + t;  // in float4 units
    if (spec_dirty) {
        // rebuild: forward transform along y of the row-transformed kernel samples
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int r = 0; r < 8; ++r)
                v[c][r] = valid ? s1_row<P>(S1, c, kx, t + r * T) : make_float2(0.f, 0.f);
        reg_fft_forward<LOGP, 3>(v, smc, tw, t);
        const float inv = 1.0f / ((float)P * (float)P);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            K[r] = v[0][r].x * inv;
            hx[r] = v[1][r].y * inv;
            hy[r] = v[2][r].y * inv;
        }
        if (valid) {
            float4* pK = reinterpret_cast<float4*>(specK) + so;
            float4* pX = reinterpret_cast<float4*>(specHx) + so;
            float4* pY = reinterpret_cast<float4*>(specHy) + so;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                pK[h * T] = make_float4(K[4 * h], K[4 * h + 1], K[4 * h + 2], K[4 * h + 3]);
                pX[h * T] = make_float4(hx[4 * h], hx[4 * h + 1], hx[4 * h + 2], hx[4 * h + 3]);
                pY[h * T] = make_float4(hy[4 * h], hy[4 * h + 1], hy[4 * h + 2], hy[4 * h + 3]);
            }
        }
        __syncthreads();  // shared memory is reused by the data transform
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int y = t + r * T;
            v[c][r] = (valid && y < G) ? T1[((size_t)c * NH + kx) * ystride + y] : make_float2(0.f, 0.f);
        }
    reg_fft_forward<LOGP, 3>(v, smc, tw, t);
    if (valid) {
        // spectra at the output positions; loaded here (not before the transform) to keep
        // them out of the registers the transform needs; after a rebuild this re-reads
        // what this thread just wrote
        const float4* pK = reinterpret_cast<const float4*>(specK) + so;
        const float4* pX = reinterpret_cast<const float4*>(specHx) + so;
        const float4* pY = reinterpret_cast<const float4*>(specHy) + so;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float4 a = pK[h * T], b = pX[h * T], d = pY[h * T];
            K[4 * h] = a.x; K[4 * h + 1] = a.y; K[4 * h + 2] = a.z; K[4 * h + 3] = a.w;
            hx[4 * h] = b.x; hx[4 * h + 1] = b.y; hx[4 * h + 2] = b.z; hx[4 * h + 3] = b.w;
            hy[4 * h] = d.x; hy[4 * h + 1] = d.y; hy[4 * h + 2] = d.z; hy[4 * h + 3] = d.w;
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const float2 rr = v[0][r], mx = v[1][r], my = v[2][r];
            v[0][r] = make_float2(K[r] * rr.x, K[r] * rr.y);
            v[1][r] = make_float2(-hx[r] * rr.y - K[r] * mx.x, hx[r] * rr.x - K[r] * mx.y);
            v[2][r] = make_float2(-hy[r] * rr.y - K[r] * my.x, hy[r] * rr.x - K[r] * my.y);
        }
    }
    reg_fft_inverse<LOGP, 3>(v, smc, tw, t);
    if (valid) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int y = t + r * T;
                if (y < G) T2[((size_t)c * NH + kx) * ystride + y] = v[c][r];
            }
    }
}

// Row block blk (RG row pairs): complex-to-real along x of the three outputs from T2,
// two real rows per complex transform, written as (A, O^x, O^y, 0) for x, y < G.
// One 32-byte global load (a 256-bit access, sm_100 and later) into a then b; p must be
// 32-byte aligned.
__device__ __forceinline__ void ld_global_v8(const float2* p, float4& a, float4& b) {
    asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                 : "l"(__cvta_generic_to_global(p)));
}

// Inverse row transforms of row block `blk` (2 RG RP rows x 3 channels) from T2 into gout.
// The half spectra of the block's RG RP row pairs are gathered into shared memory first
// (with RG RP even, 32 bytes per column and load); each thread then transforms RP row
// pairs in turn.
template <int LOGP, int RP = 1>
__device__ __forceinline__ void rows_inv_body(int blk, const float2* __restrict__ T2, int ystride,
                                              float4* __restrict__ gout, int Gs, const float2* __restrict__ tw,
                                              int G, float2* sm) {
    using Gm = RegGeom<LOGP>;
    constexpr int P = Gm::P, T = Gm::T, RG = Gm::RG, NH = P / 2 + 1;
    constexpr int RB = RG * RP;  // row pairs of the block; pair q is rows ybase + 2q, + 1
    const int ybase = blk * (2 * RB);
    if (ybase >= G) return;
    // Z_k = A_k + i B_k for two real rows (A, B) at row pair q, both halves of the spectrum.
    // NB items per thread and round: all their loads are in flight before the first store
    constexpr int NB = (RB >= 4) ? 1 : 4 / RB;
    for (int i0 = threadIdx.x; i0 < 3 * NH; i0 += NB * blockDim.x) {
        float4 X[NB][RB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int idx = i0 + b * blockDim.x;
            const int c = idx / NH;
            const int kx = split_freq<LOGP>(idx - c * NH);
            const float2* src = T2 + ((size_t)c * NH + kx) * ystride + ybase;
            if constexpr (RB % 2 == 0) {
                // ystride is a multiple of 32 and ybase of 4: src + 2q (q even) is 32-byte aligned;
                // rows up to ybase + 2 RB - 1 < ystride lie inside the column
#pragma unroll
                for (int q = 0; q < RB; q += 2) {
                    if (idx < 3 * NH && ybase + 2 * q < G) {
                        ld_global_v8(src + 2 * q, X[b][q], X[b][q + 1]);
                    } else {
                        X[b][q] = make_float4(0.f, 0.f, 0.f, 0.f);
                        X[b][q + 1] = X[b][q];
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < RB; ++q)
                    X[b][q] = (idx < 3 * NH && ybase + 2 * q < G) ? reinterpret_cast<const float4*>(src)[q]
                                                                   : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int idx = i0 + b * blockDim.x;
            if (idx >= 3 * NH) break;
            const int c = idx / NH;
            const int kx = split_freq<LOGP>(idx - c * NH);
            const int pk = swz(pos_of_freq<LOGP>(kx));
            const int pn = swz(pos_of_freq<LOGP>((P - kx) & (P - 1)));
#pragma unroll
            for (int q = 0; q < RB; ++q) {
                float4 x = X[b][q];
                if (ybase + 2 * q >= G) x = make_float4(0.f, 0.f, 0.f, 0.f);  // rows past G: never written
                if (ybase + 2 * q + 1 >= G) { x.z = 0.f; x.w = 0.f; }
                float2* seq = sm + ((size_t)q * 3 + c) * P;
                seq[pk] = make_float2(x.x - x.w, x.y + x.z);
                if (kx != 0 && kx != P / 2) seq[pn] = make_float2(x.x + x.w, x.z - x.y);
            }
        }
    }
    __syncthreads();
    const int lr = threadIdx.x / T, t = threadIdx.x - lr * T;
#pragma unroll 1
    for (int h = 0; h < RP; ++h) {
        const int pq = h * RG + lr;
        const int y0 = ybase + 2 * pq;
        float2* smr = sm + (size_t)pq * 3 * P;
        float2 v[3][8];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int r = 0; r < 8; ++r) v[c][r] = smr[c * P + swz(8 * t + r)];
        reg_fft_inverse<LOGP, 3>(v, smr, tw, t);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int x = t + r * T;
            if (x >= G) continue;
            if (y0 < G) gout[(size_t)y0 * Gs + x] = make_float4(v[0][r].x, v[1][r].x, v[2][r].x, 0.0f);
            if (y0 + 1 < G) gout[(size_t)(y0 + 1) * Gs + x] = make_float4(v[0][r].y, v[1][r].y, v[2][r].y, 0.0f);
        }
    }
}

// ---------------------------------------------------------------- one channel at a time
// The same three stages for sizes whose T = P/8 threads per sequence fill a whole CTA
// (P = 8192: 1024 threads, at most 64 registers each): each thread keeps the eight values
// of one channel in registers at a time, and the three channels of a row pair or column
// sit in three shared-memory slices of P values. A transform uses its own slice for its
// exchanges, and the last exchange of a forward transform reads (and the first of an
// inverse writes) exactly the MF positions 8t .. 8t+7 of its thread, so the results can
// be parked in, and taken back from, the thread's own MF positions without a barrier.

template <int LOGP, class Src>
__device__ __forceinline__ void rows_fwd_body_seq(const Src& src, int nrows, int blk, float2* __restrict__ out,
                                                  int ystride, const float2* __restrict__ tw, float2* sm) {
    using Gm = RegGeom<LOGP>;
    constexpr int P = Gm::P, T = Gm::T, NH = P / 2 + 1;
    static_assert(Gm::RG == 1, "one row pair per CTA");
    const int G = nrows;
    const int y0 = 2 * blk;
    if (y0 >= G) return;
    const int t = threadIdx.x;
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        float2* sl = sm + (size_t)c * P;
        float2 v[1][8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int x = t + r * T;
            v[0][r] = make_float2(src(c, y0, x, G), src(c, y0 + 1, x, G));
        }
        reg_fft_forward<LOGP, 1>(v, sl, tw, t);
#pragma unroll
        for (int r = 0; r < 8; ++r) sl[swz(8 * t + r)] = v[0][r];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 3 * NH; idx += blockDim.x) {
        const int c = idx / NH;
        const int kx = split_freq<LOGP>(idx - c * NH);
        const float2* seq = sm + (size_t)c * P;
        const float2 Z = seq[swz(pos_of_freq<LOGP>(kx))], W = seq[swz(pos_of_freq<LOGP>((P - kx) & (P - 1)))];
        reinterpret_cast<float4*>(out + ((size_t)c * NH + kx) * ystride + y0)[0] =
            make_float4(0.5f * (Z.x + W.x), 0.5f * (Z.y - W.y), 0.5f * (Z.y + W.y), 0.5f * (W.x - Z.x));
    }
}

template <int LOGP>
__device__ __forceinline__ void cols_body_seq(int kx, const float2* __restrict__ T1, float2* __restrict__ T2,
                                              int ystride, float* __restrict__ specK, float* __restrict__ specHx,
                                              float* __restrict__ specHy, const float2* __restrict__ S1,
                                              const float2* __restrict__ tw, int G, int spec_dirty, float2* sm) {
    using Gm = RegGeom<LOGP>;
    constexpr int P = Gm::P, T = Gm::T, NH = P / 2 + 1;
    static_assert(Gm::CG == 1, "one column per CTA");
    const int t = threadIdx.x;
    const size_t so = (size_t)kx * P + 8 * t;
    if (spec_dirty) {
        // rebuild: forward transforms along y of the row-transformed kernel samples
        const float inv = 1.0f / ((float)P * (float)P);
#pragma unroll 1
        for (int c = 0; c < 3; ++c) {
            float2 v[1][8];
#pragma unroll
            for (int r = 0; r < 8; ++r) v[0][r] = s1_row<P>(S1, c, kx, t + r * T);
            reg_fft_forward<LOGP, 1>(v, sm + (size_t)c * P, tw, t);
            float o[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) o[r] = (c == 0 ? v[0][r].x : v[0][r].y) * inv;
            float* dst = (c == 0 ? specK : (c == 1 ? specHx : specHy)) + so;
            reinterpret_cast<float4*>(dst)[0] = make_float4(o[0], o[1], o[2], o[3]);
            reinterpret_cast<float4*>(dst)[1] = make_float4(o[4], o[5], o[6], o[7]);
        }
        __syncthreads();  // the slices are reused by the data transforms
    }
    // forward transforms of rho, m^x, m^y, each parked at its thread's MF positions
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        float2* sl = sm + (size_t)c * P;
        float2 v[1][8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int y = t + r * T;
            v[0][r] = (y < G) ? T1[((size_t)c * NH + kx) * ystride + y] : make_float2(0.f, 0.f);
        }
        reg_fft_forward<LOGP, 1>(v, sl, tw, t);
#pragma unroll
        for (int r = 0; r < 8; ++r) sl[swz(8 * t + r)] = v[0][r];
    }
    // spectral product at this thread's own positions, four at a time
    float2* s0 = sm;
    float2* s1 = sm + P;
    float2* s2 = sm + 2 * P;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float4 Kq = reinterpret_cast<const float4*>(specK + so)[h];
        const float4 Xq = reinterpret_cast<const float4*>(specHx + so)[h];
        const float4 Yq = reinterpret_cast<const float4*>(specHy + so)[h];
        const float K4[4] = {Kq.x, Kq.y, Kq.z, Kq.w}, X4[4] = {Xq.x, Xq.y, Xq.z, Xq.w},
                    Y4[4] = {Yq.x, Yq.y, Yq.z, Yq.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int a = swz(8 * t + 4 * h + q);
            const float2 rr = s0[a], mx = s1[a], my = s2[a];
            const float K = K4[q], hx = X4[q], hy = Y4[q];
            s0[a] = make_float2(K * rr.x, K * rr.y);
            s1[a] = make_float2(-hx * rr.y - K * mx.x, hx * rr.x - K * mx.y);
            s2[a] = make_float2(-hy * rr.y - K * my.x, hy * rr.x - K * my.y);
        }
    }
    // inverse transforms, rows y < G to T2
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        float2* sl = sm + (size_t)c * P;
        float2 v[1][8];
#pragma unroll
        for (int r = 0; r < 8; ++r) v[0][r] = sl[swz(8 * t + r)];
        reg_fft_inverse<LOGP, 1>(v, sl, tw, t);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int y = t + r * T;
            if (y < G) T2[((size_t)c * NH + kx) * ystride + y] = v[0][r];
        }
    }
}

template <int LOGP>
__device__ __forceinline__ void rows_inv_body_seq(int blk, const float2* __restrict__ T2, int ystride,
                                                  float4* __restrict__ gout, int Gs, const float2* __restrict__ tw,
                                                  int G, float2* sm) {
    using Gm = RegGeom<LOGP>;
    constexpr int P = Gm::P, T = Gm::T, NH = P / 2 + 1;
    static_assert(Gm::RG == 1, "one row pair per CTA");
    const int y0 = 2 * blk;
    if (y0 >= G) return;
    // Z_k = A_k + i B_k for the two real rows of the pair, both halves of the spectrum
    for (int idx = threadIdx.x; idx < 3 * NH; idx += blockDim.x) {
        const int c = idx / NH;
        const int kx = split_freq<LOGP>(idx - c * NH);
        float4 x = reinterpret_cast<const float4*>(T2 + ((size_t)c * NH + kx) * ystride + y0)[0];
        if (y0 + 1 >= G) { x.z = 0.f; x.w = 0.f; }  // row past G: never written
        float2* seq = sm + (size_t)c * P;
        seq[swz(pos_of_freq<LOGP>(kx))] = make_float2(x.x - x.w, x.y + x.z);
        if (kx != 0 && kx != P / 2) seq[swz(pos_of_freq<LOGP>((P - kx) & (P - 1)))] = make_float2(x.x + x.w, x.z - x.y);
    }
    __syncthreads();
    const int t = threadIdx.x;
    // inverse transforms one channel at a time; each result is parked at the thread's
    // natural-order positions t + r T of its slice (read by this thread only)
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        float2* sl = sm + (size_t)c * P;
        float2 v[1][8];
#pragma unroll
        for (int r = 0; r < 8; ++r) v[0][r] = sl[swz(8 * t + r)];
        reg_fft_inverse<LOGP, 1>(v, sl, tw, t);
        __syncthreads();  // the last exchange's reads are done before the slice is overwritten
#pragma unroll
        for (int r = 0; r < 8; ++r) sl[swz(t + r * T)] = v[0][r];
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int x = t + r * T;
        if (x >= G) continue;
        const int a = swz(x);
        const float2 A = sm[a], X = sm[P + a], Y = sm[2 * P + a];
        if (y0 < G) gout[(size_t)y0 * Gs + x] = make_float4(A.x, X.x, Y.x, 0.0f);
        if (y0 + 1 < G) gout[(size_t)(y0 + 1) * Gs + x] = make_float4(A.y, X.y, Y.y, 0.0f);
    }
}

}  // namespace tfdp
