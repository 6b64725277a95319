// cols_tc.cu -- column stage of the grid interaction (Sec. 3.4, second step) on the
// tensor cores: BF16 split-precision products with FP32 accumulation (precision mode
// TFDP_PREC_BF16X3, FFT size P = 2048).
//
// The column stage takes, for every frequency column kx of the row-transformed grids
// T1[c][kx][y] (c = rho, m^x, m^y; y < G <= 1023 non-zero, the rest of the P = 2048
// circulant zero), the forward DFT along y, the spectral product
//     A = K rho,   O^x = i hx rho - K m^x,   O^y = i hy rho - K m^y
// (K, hx, hy: the kernel spectra of the FP32 path, pre-scaled by 1/P^2), and the inverse
// DFT along y, keeping y < G, into T2[c][kx][y]. Here each length-2048 DFT is done as a
// four-step transform, P = 64 x 32, with y = 32 n1 + n2 and k = k1 + 64 k2:
//     X[k1 + 64 k2] = sum_n2 W32^(n2 k2) W2048^(n2 k1) sum_n1 W64^(n1 k1) x[32 n1 + n2]
//     x[32 n1 + n2] = sum_k1 W64^(-n1 k1) W2048^(-n2 k1) sum_k2 W32^(-n2 k2) X[k1 + 64 k2]
// (W_N = exp(-2 pi i / N)). Both sums of each transform are dense complex matrix
// products, written as real GEMMs (re/im doubled) for tcgen05.mma kind::f16:
//   stage A  (n1 -> k1)  D[(k1,re/im)][(seq,n2)]   = FA  x data   (M 128, K 64: n1 < 32 only)
//   stage B  (n2 -> k2)  D[(col,k1)][(k2,re/im)]   = data x FB    (M 128, N 64, one per channel)
//   stage B' (k2 -> n2)  D[(n2,re/im)][(seq,k1)]   = FB' x data   (M 128 with 64 rows used)
//   stage A' (k1 -> n1)  D[(seq,n2)][(n1,re/im)]   = data x FA'   (N 64: n1 < 32 only)
// The twiddles W2048^(+-n2 k1) and the spectral product run in FP32 registers between
// the stages. Every operand x is split into x_hi = bf16(x) and x_lo = bf16(x - x_hi); a
// product is accumulated as A_hi B_hi + A_hi B_lo + A_lo B_hi (the dropped A_lo B_lo term
// and the split residues are about 2^-16 of the product).
//
// One CTA (256 threads, one per SM) loops over tiles of two columns x three channels.
// Operands sit in shared memory in the canonical K-major layout without swizzle (core
// matrices of 8 rows x 16 bytes); the DFT matrices (hi and lo, 96 KB, built on the host
// in FP64) are copied once per CTA with bulk asynchronous copies. Accumulators live in
// tensor memory (512 columns); one thread issues the MMAs and commits them to an
// mbarrier that every thread waits on, with a bounded wait that records a timeout in
// the device flags and ends the kernel cleanly instead of hanging.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "fft.cuh"
#include "launch.h"

namespace tfdp {

namespace {

constexpr int kTcLogP = 11;
constexpr int kTcP = 1 << kTcLogP;       // 2048
constexpr int kTcNH = kTcP / 2 + 1;       // 1025 columns
constexpr int kTcThreads = 256;
constexpr int kTcCols = 2;                // columns per tile
constexpr int kTcSeq = 3 * kTcCols;       // sequences per tile (channel-major: seq = 2 c + j)
constexpr int kTcTiles = (kTcNH + kTcCols - 1) / kTcCols;
constexpr uint32_t kTcTmemCols = 512;

// shared-memory map (bytes from the 1024-aligned base)
constexpr int kData = 49152;              // one split of the data operand: 48 KB
constexpr int kDataHi = 0, kDataLo = kData;
constexpr int kConst = 2 * kData;         // DFT matrices
constexpr int kFaHi = kConst, kFaLo = kFaHi + 16384;      // 128 x 64
constexpr int kFbHi = kFaLo + 16384, kFbLo = kFbHi + 8192;    // 64 x 64
constexpr int kFbpHi = kFbLo + 8192, kFbpLo = kFbpHi + 8192;  // 64 (read as 128) x 64
constexpr int kFapHi = kFbpLo + 8192, kFapLo = kFapHi + 16384;  // 64 x 128
constexpr int kConstBytes = kFapLo + 16384 - kConst;      // 98304
constexpr int kSmemBytes = kConst + kConstBytes + 1024;   // + alignment slack
static_assert(kConstBytes == 98304, "constant image size");

// byte offset of element (row, kc) of a K-major bf16 operand with K columns
__host__ __device__ __forceinline__ int koff(int row, int kc, int K) {
    return (row >> 3) * (K * 16) + (kc >> 3) * 128 + (row & 7) * 16 + (kc & 7) * 2;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle; lbo = K-adjacent core matrices,
// sbo = 8-row-group stride
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) |
           (1ull << 46);
}

// instruction descriptor, kind::f16: BF16 A and B (both K-major), FP32 accumulator, M = 128
__host__ __device__ constexpr uint32_t idesc_bf16(int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// D (+)= A_hi B_hi + A_hi B_lo + A_lo B_hi over K / 16 steps of 16 (256 bytes apart in a
// no-swizzle K-major operand)
__device__ __forceinline__ void mma3(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint32_t a_sbo, uint32_t b_hi,
                                     uint32_t b_lo, uint32_t b_sbo, int K, uint32_t idesc) {
    for (int ks = 0; ks < K / 16; ++ks) {
        const uint32_t o = (uint32_t)ks * 256u;
        mma_bf16(d, sdesc(a_hi + o, a_sbo), sdesc(b_hi + o, b_sbo), idesc, ks > 0 ? 1u : 0u);
        mma_bf16(d, sdesc(a_hi + o, a_sbo), sdesc(b_lo + o, b_sbo), idesc, 1u);
        mma_bf16(d, sdesc(a_lo + o, a_sbo), sdesc(b_hi + o, b_sbo), idesc, 1u);
    }
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Bounded wait for phase `parity` of an mbarrier; false if it never completed.
constexpr int kTcWaitPolls = 1 << 22;
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (int it = 0; it < kTcWaitPolls; ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (thread i: lane base + i)
__device__ __forceinline__ void tmem_ld16(uint32_t addr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Split 8 FP32 values into one 16-byte chunk of bf16 highs and one of bf16 lows.
__device__ __forceinline__ void split8(const float* x, uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __nv_bfloat162 bh = __floats2bfloat162_rn(x[2 * q], x[2 * q + 1]);
        const float2 fh = __bfloat1622float2(bh);
        const __nv_bfloat162 bl = __floats2bfloat162_rn(x[2 * q] - fh.x, x[2 * q + 1] - fh.y);
        h[q] = *reinterpret_cast<const uint32_t*>(&bh);
        l[q] = *reinterpret_cast<const uint32_t*>(&bl);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ void put8(unsigned char* base, int off, const float* x) {
    uint4 hi, lo;
    split8(x, hi, lo);
    *reinterpret_cast<uint4*>(base + kDataHi + off) = hi;
    *reinterpret_cast<uint4*>(base + kDataLo + off) = lo;
}

// Natural-order kernel spectra of columns kx0, kx0 + 1 from the row-transformed kernel
// samples S1 (FP32 shared-memory FFT along y, scaled by 1/P^2), in an iteration that
// rebuilds the spectrum.
__device__ void tc_spectrum(int kx0, const float2* __restrict__ S1, const float2* __restrict__ tw,
                            float* __restrict__ specN, float2* sm) {
    constexpr int P = kTcP, PL = padded_len(P);
    for (int j = 0; j < kTcCols; ++j) {
        const int kx = kx0 + j;
        if (kx >= kTcNH) break;
        for (int idx = threadIdx.x; idx < 3 * P; idx += blockDim.x) {
            const int c = idx / P, y = idx - c * P;
            sm[c * PL + spad(y)] = S1[((size_t)c * kTcNH + kx) * P + y];
        }
        __syncthreads();
        fft_forward<kTcLogP>(sm, 3, tw);
        const float inv = 1.0f / ((float)P * (float)P);
        for (int k = threadIdx.x; k < P; k += blockDim.x) {
            const int a = spad(pos_of_freq<kTcLogP>(k));
            specN[(size_t)kx * P + k] = sm[a].x * inv;
            specN[((size_t)kTcNH + kx) * P + k] = sm[PL + a].y * inv;
            specN[((size_t)2 * kTcNH + kx) * P + k] = sm[2 * PL + a].y * inv;
        }
        __threadfence_block();
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_cols_tc(const float2* __restrict__ T1, float2* __restrict__ T2, int ystride, float* specN,
              const float2* __restrict__ S1, const float2* __restrict__ tw,
              const unsigned char* __restrict__ consts, DevState* __restrict__ st) {
    extern __shared__ unsigned char sm_raw[];
    __shared__ __align__(8) uint64_t mbar_mma, mbar_const;
    __shared__ uint32_t tmem_base_sh;
    unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3;   // TMEM lane quadrant of this warp
    const int hh = warp >> 2; // column half
    const int m = 32 * q + lane;  // TMEM lane (accumulator row) of this thread
    const uint32_t s_base = smem_u32(sm);
    const uint32_t mb = smem_u32(&mbar_mma), mc = smem_u32(&mbar_const);

    // DFT matrices: bulk asynchronous copies of the 96 KB image, issued before waiting on
    // the previous kernel (they do not depend on it)
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mc));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mc), "r"(kConstBytes) : "memory");
        constexpr int kPiece = kConstBytes / 4;
        for (int p = 0; p < 4; ++p)
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    s_base + kConst + p * kPiece),
                "l"(consts + p * kPiece), "r"(kPiece), "r"(mc)
                : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(kTcTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base_sh;
    pdl_wait();
    pdl_trigger();
    const int G = st->grid.G;
    const int dirty = st->spec_dirty;
    bool ok = mbar_wait(mc, 0);
    uint32_t phase = 0;
    if (__syncthreads_or(!ok)) goto out;

    for (int tile = blockIdx.x; tile < kTcTiles; tile += gridDim.x) {
        const int kx0 = tile * kTcCols;
        if (dirty) tc_spectrum(kx0, S1, tw, specN, reinterpret_cast<float2*>(sm));  // uses the data area
        // ---- load: stage A operand, rows (seq, n2), K (n1 < 32, re/im) interleaved
        for (int it = tid; it < 4 * kTcSeq * 32; it += kTcThreads) {
            const int qq = it / (kTcSeq * 32);   // n1 block of 8
            const int r = it - qq * (kTcSeq * 32);
            const int seq = r >> 5, n2 = r & 31;
            const int c = seq >> 1, kx = kx0 + (seq & 1);
            const bool col_ok = kx < kTcNH;
            const float2* src = T1 + ((size_t)c * kTcNH + (col_ok ? kx : 0)) * ystride;
            float x[16];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int y = 32 * (8 * qq + i) + n2;
                const float2 v = (col_ok && y < G) ? src[y] : make_float2(0.f, 0.f);
                x[2 * i] = v.x;
                x[2 * i + 1] = v.y;
            }
            put8(sm, koff(r, 16 * qq, 64), x);
            put8(sm, koff(r, 16 * qq + 8, 64), x + 8);
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        // ---- stage A: D[0, 192) = FA (128 x 64) x data (192 rows)
        if (tid == 0) {
            fence_after();
            mma3(tmem, s_base + kFaHi, s_base + kFaLo, 1024, s_base + kDataHi, s_base + kDataLo, 1024, 64,
                 idesc_bf16(kTcSeq * 32));
            mma_commit(mb);
        }
        ok = mbar_wait(mb, phase);
        phase ^= 1u;
        fence_after();
        if (__syncthreads_or(!ok)) goto out;
        // ---- twiddle W2048^(n2 k1); stage B operands (one per channel): rows (j, k1),
        //      K (re/im, n2) blocked
        {
            const int k1 = m >> 1, ro = m & 1;
            for (int s3 = 0; s3 < 3; ++s3) {
                const int seq = 3 * hh + s3;
                const int c = seq >> 1, j = seq & 1;
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    float v[16], o[16];
                    tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(seq * 32 + 16 * half), v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const float pv = __shfl_xor_sync(0xffffffffu, v[i], 1);
                        const float re = ro ? pv : v[i], im = ro ? v[i] : pv;
                        const int n2 = 16 * half + i;
                        const float2 w = __ldg(tw + ((n2 * k1) & (kTcP - 1)));
                        o[i] = ro ? fmaf(re, w.y, im * w.x) : fmaf(re, w.x, -im * w.y);
                    }
                    const int row = 64 * j + k1;
                    const int base = c * 16384;
                    put8(sm, base + koff(row, 32 * ro + 16 * half, 64), o);
                    put8(sm, base + koff(row, 32 * ro + 16 * half + 8, 64), o + 8);
                }
            }
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        // ---- stage B: per channel c, D[64 c, 64 c + 64) = data_c (128 x 64) x FB^T
        if (tid == 0) {
            fence_after();
            for (int c = 0; c < 3; ++c)
                mma3(tmem + 64u * c, s_base + kDataHi + c * 16384, s_base + kDataLo + c * 16384, 1024, s_base + kFbHi,
                     s_base + kFbLo, 1024, 64, idesc_bf16(64));
            mma_commit(mb);
        }
        ok = mbar_wait(mb, phase);
        phase ^= 1u;
        fence_after();
        if (__syncthreads_or(!ok)) goto out;
        // ---- spectral product at k = k1 + 64 k2; stage B' operand: rows (seq, k1),
        //      K (k2, re/im) interleaved
        {
            const int j = m >> 6, k1 = m & 63;
            const int kx = kx0 + j;
            const bool col_ok = kx < kTcNH;
            // plain loads: in an iteration that rebuilds the spectrum this CTA has just
            // written these values (the non-coherent read-only path could miss them)
            const float* sK = specN + (size_t)(col_ok ? kx : 0) * kTcP;
            const float* sX = specN + ((size_t)kTcNH + (col_ok ? kx : 0)) * kTcP;
            const float* sY = specN + ((size_t)2 * kTcNH + (col_ok ? kx : 0)) * kTcP;
#pragma unroll
            for (int sub = 0; sub < 2; ++sub) {
                const int k2b = 16 * hh + 8 * sub;  // first k2 of these 8
                float r_[16], x_[16], y_[16];
                const uint32_t col = (uint32_t)(2 * k2b);
                const uint32_t la = tmem + ((uint32_t)(32 * q) << 16) + col;
                tmem_ld16(la, r_);
                tmem_ld16(la + 64u, x_);
                tmem_ld16(la + 128u, y_);
                float oa[16], ox[16], oy[16];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int k = k1 + 64 * (k2b + i);
                    const float K = col_ok ? sK[k] : 0.f;
                    const float hx = col_ok ? sX[k] : 0.f;
                    const float hy = col_ok ? sY[k] : 0.f;
                    const float rr = r_[2 * i], ri = r_[2 * i + 1];
                    oa[2 * i] = K * rr;
                    oa[2 * i + 1] = K * ri;
                    ox[2 * i] = -hx * ri - K * x_[2 * i];
                    ox[2 * i + 1] = hx * rr - K * x_[2 * i + 1];
                    oy[2 * i] = -hy * ri - K * y_[2 * i];
                    oy[2 * i + 1] = hy * rr - K * y_[2 * i + 1];
                }
                const int kc = 2 * k2b;
                put8(sm, koff((0 * 2 + j) * 64 + k1, kc, 64), oa);
                put8(sm, koff((0 * 2 + j) * 64 + k1, kc + 8, 64), oa + 8);
                put8(sm, koff((1 * 2 + j) * 64 + k1, kc, 64), ox);
                put8(sm, koff((1 * 2 + j) * 64 + k1, kc + 8, 64), ox + 8);
                put8(sm, koff((2 * 2 + j) * 64 + k1, kc, 64), oy);
                put8(sm, koff((2 * 2 + j) * 64 + k1, kc + 8, 64), oy + 8);
            }
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        // ---- stage B': D[0, 384) = FB' (rows 0..63 used) x data (384 rows: N 256 + 128)
        if (tid == 0) {
            fence_after();
            mma3(tmem, s_base + kFbpHi, s_base + kFbpLo, 1024, s_base + kDataHi, s_base + kDataLo, 1024, 64,
                 idesc_bf16(256));
            mma3(tmem + 256u, s_base + kFbpHi, s_base + kFbpLo, 1024, s_base + kDataHi + 32768,
                 s_base + kDataLo + 32768, 1024, 64, idesc_bf16(128));
            mma_commit(mb);
        }
        ok = mbar_wait(mb, phase);
        phase ^= 1u;
        fence_after();
        if (__syncthreads_or(!ok)) goto out;
        // ---- twiddle W2048^(-n2 k1) (lanes 0..63 hold rows (n2, re/im)); stage A'
        //      operand: rows (seq, n2), K (re/im, k1) blocked, 128 wide
        if (q < 2) {
            const int n2 = m >> 1, ro = m & 1;
            for (int s3 = 0; s3 < 3; ++s3) {
                const int seq = 3 * hh + s3;
#pragma unroll
                for (int blk = 0; blk < 4; ++blk) {
                    float v[16], o[16];
                    tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(seq * 64 + 16 * blk), v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const float pv = __shfl_xor_sync(0xffffffffu, v[i], 1);
                        const float re = ro ? pv : v[i], im = ro ? v[i] : pv;
                        const int k1 = 16 * blk + i;
                        const float2 w = __ldg(tw + ((n2 * k1) & (kTcP - 1)));
                        o[i] = ro ? fmaf(im, w.x, -re * w.y) : fmaf(re, w.x, im * w.y);
                    }
                    const int row = 32 * seq + n2;
                    put8(sm, koff(row, 64 * ro + 16 * blk, 128), o);
                    put8(sm, koff(row, 64 * ro + 16 * blk + 8, 128), o + 8);
                }
            }
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        // ---- stage A': D[0, 64) = data rows 0..127 x FA'^T, D[64, 128) = rows 128..255
        //      (rows 192..255 read whatever follows and are never used)
        if (tid == 0) {
            fence_after();
            mma3(tmem, s_base + kDataHi, s_base + kDataLo, 2048, s_base + kFapHi, s_base + kFapLo, 2048, 128,
                 idesc_bf16(64));
            mma3(tmem + 64u, s_base + kDataHi + 32768, s_base + kDataLo + 32768, 2048, s_base + kFapHi,
                 s_base + kFapLo, 2048, 128, idesc_bf16(64));
            mma_commit(mb);
        }
        ok = mbar_wait(mb, phase);
        phase ^= 1u;
        fence_after();
        if (__syncthreads_or(!ok)) goto out;
        // ---- outputs: lane (seq, n2), columns (n1, re/im) -> T2[c][kx][32 n1 + n2]
#pragma unroll
        for (int part = 0; part < 2; ++part) {
            if (part == 1 && q >= 2) continue;
            const int seq = 4 * part + (m >> 5), n2 = m & 31;
            const int c = seq >> 1, kx = kx0 + (seq & 1);
            float v[16];
            float2* dst = T2 + ((size_t)c * kTcNH + kx) * ystride;
#pragma unroll
            for (int sub = 0; sub < 2; ++sub) {
                tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(64 * part + 32 * hh + 16 * sub), v);
                if (kx < kTcNH) {
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int n1 = 16 * hh + 8 * sub + i;
                        const int y = 32 * n1 + n2;
                        if (y < G) dst[y] = make_float2(v[2 * i], v[2 * i + 1]);
                    }
                }
            }
        }
        fence_before();
        __syncthreads();  // TMEM reads done before the next tile's MMAs overwrite it
        fence_after();
    }
out:
    if (!ok && tid == 0) atomicOr(&st->flags, FLAG_WAIT_TIMEOUT);
    fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols));
}

// ------------------------------------------------------------------ host side
uint16_t bf16_rn(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    const uint32_t r = u + 0x7FFFu + ((u >> 16) & 1u);  // round to nearest even (finite inputs)
    return (uint16_t)(r >> 16);
}
float bf16_to_f(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// Store x as (hi, lo) bf16 at element (row, kc) of the operand at byte offset `base`.
void put_const(std::vector<unsigned char>& img, int base, int row, int kc, int K, double x) {
    const uint16_t hi = bf16_rn((float)x);
    const uint16_t lo = bf16_rn((float)(x - (double)bf16_to_f(hi)));
    const int o = koff(row, kc, K);
    int hb = 0, lb = 0;
    switch (base) {  // hi / lo regions of each matrix
        case kFaHi: hb = kFaHi; lb = kFaLo; break;
        case kFbHi: hb = kFbHi; lb = kFbLo; break;
        case kFbpHi: hb = kFbpHi; lb = kFbpLo; break;
        default: hb = kFapHi; lb = kFapLo; break;
    }
    std::memcpy(&img[(size_t)(hb - kConst + o)], &hi, 2);
    std::memcpy(&img[(size_t)(lb - kConst + o)], &lo, 2);
}

}  // namespace

// The 96 KB shared-memory image of the four DFT matrices (hi and lo splits), built in
// FP64. With c + i s = exp(-2 pi i n k / N):
//   FA  [(k1, ro)][(n1, ri)]  forward 64-point DFT, inputs n1 < 32   (rows 2 k1 + ro, cols 2 n1 + ri)
//   FB  [(k2, ro)][(ri, n2)]  forward 32-point DFT                   (rows 2 k2 + ro, cols 32 ri + n2)
//   FB' [(n2, ro)][(k2, ri)]  inverse 32-point DFT                   (rows 2 n2 + ro, cols 2 k2 + ri)
//   FA' [(n1, ro)][(ri, k1)]  inverse 64-point DFT, outputs n1 < 32  (rows 2 n1 + ro, cols 64 ri + k1)
// Forward entries: Re row (c, -s), Im row (s, c); inverse: Re row (c, s), Im row (-s, c).
void build_tc_constants(std::vector<unsigned char>& img) {
    img.assign((size_t)kConstBytes, 0);
    const double pi = 3.14159265358979323846;
    for (int k1 = 0; k1 < 64; ++k1)
        for (int n1 = 0; n1 < 32; ++n1) {
            const double a = -2.0 * pi * (double)((n1 * k1) % 64) / 64.0, c = std::cos(a), s = std::sin(a);
            put_const(img, kFaHi, 2 * k1, 2 * n1, 64, c);
            put_const(img, kFaHi, 2 * k1, 2 * n1 + 1, 64, -s);
            put_const(img, kFaHi, 2 * k1 + 1, 2 * n1, 64, s);
            put_const(img, kFaHi, 2 * k1 + 1, 2 * n1 + 1, 64, c);
            // inverse, outputs n1 < 32: rows (n1, ro), cols (ri, k1)
            put_const(img, kFapHi, 2 * n1, k1, 128, c);
            put_const(img, kFapHi, 2 * n1, 64 + k1, 128, s);
            put_const(img, kFapHi, 2 * n1 + 1, k1, 128, -s);
            put_const(img, kFapHi, 2 * n1 + 1, 64 + k1, 128, c);
        }
    for (int k2 = 0; k2 < 32; ++k2)
        for (int n2 = 0; n2 < 32; ++n2) {
            const double a = -2.0 * pi * (double)((n2 * k2) % 32) / 32.0, c = std::cos(a), s = std::sin(a);
            put_const(img, kFbHi, 2 * k2, n2, 64, c);
            put_const(img, kFbHi, 2 * k2, 32 + n2, 64, -s);
            put_const(img, kFbHi, 2 * k2 + 1, n2, 64, s);
            put_const(img, kFbHi, 2 * k2 + 1, 32 + n2, 64, c);
            put_const(img, kFbpHi, 2 * n2, 2 * k2, 64, c);
            put_const(img, kFbpHi, 2 * n2, 2 * k2 + 1, 64, s);
            put_const(img, kFbpHi, 2 * n2 + 1, 2 * k2, 64, -s);
            put_const(img, kFbpHi, 2 * n2 + 1, 2 * k2 + 1, 64, c);
        }
}

size_t tc_constants_bytes() { return (size_t)kConstBytes; }
size_t tc_spectrum_floats() { return (size_t)3 * kTcNH * kTcP; }

cudaError_t prepare_cols_tc() {
    return cudaFuncSetAttribute(k_cols_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
}

cudaError_t launch_cols_tc(const FftLaunch& a, const unsigned char* consts, float* specN, cudaStream_t s) {
    if (a.logP != kTcLogP) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int grid = sms < kTcTiles ? sms : kTcTiles;
    return launch_pdl(k_cols_tc, grid, kTcThreads, (size_t)kSmemBytes, s, (const float2*)a.T1, a.T2, a.ystride,
                      specN, (const float2*)a.S1, a.tw, consts, a.st);
}

}  // namespace tfdp
