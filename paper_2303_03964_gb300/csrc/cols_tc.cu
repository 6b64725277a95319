// cols_tc.cu -- column stage of the grid interaction (Sec. 3.4, second step) on the
// tensor cores: BF16 split-precision products with FP32 accumulation (precision mode
// TFDP_PREC_BF16X3, FFT size P = 2048).
//
// The column stage takes, for every frequency column kx of the row-transformed grids
// T1[c][kx][y] (c = rho, m^x, m^y; y < G <= 1023 non-zero, the rest of the P = 2048
// circulant zero), the forward DFT along y, the spectral product
//     A = K rho,   O^x = i hx rho - K m^x,   O^y = i hy rho - K m^y
// (K, hx, hy: the kernel spectra, pre-scaled by 1/P^2), and the inverse DFT along y,
// keeping y < G, into T2[c][kx][y]. Here each length-2048 DFT is done as a four-step
// transform, P = 64 x 32, with y = 32 n1 + n2 and k = k1 + 64 k2:
//     X[k1 + 64 k2] = sum_n2 W32^(n2 k2) W2048^(n2 k1) sum_n1 W64^(n1 k1) x[32 n1 + n2]
//     x[32 n1 + n2] = sum_k1 W64^(-n1 k1) W2048^(-n2 k1) sum_k2 W32^(-n2 k2) X[k1 + 64 k2]
// (W_N = exp(-2 pi i / N)). Both sums of each transform are dense complex matrix
// products, written as real GEMMs (re/im doubled) for tcgen05.mma kind::f16. For one
// column (three sequences, c = 0..2):
//   stage A  (n1 -> k1)  D[(k1,re/im)][(c,n2)]     = FA  x data   (M 128, N 96, K 64: n1 < 32)
//   stage B  (n2 -> k2)  D[k1][(k2,re/im)]         = data_c x FB  (M 128 of which 64 used, N 64)
//   stage B' (k2 -> n2)  D[(n2,re/im)][(c,k1)]     = FB' x data   (M 128 of which 64 used, N 192)
//   stage A' (k1 -> n1)  D[(c,n2)][(n1,re/im)]     = data x FA'   (M 128 of which 96 used, N 64: n1 < 32)
// The twiddles W2048^(+-n2 k1) and the spectral product run in FP32 registers between
// the stages. Every operand x is split into x_hi = bf16(x) and x_lo = bf16(x - x_hi); a
// product is accumulated as A_hi B_hi + A_hi B_lo + A_lo B_hi (the dropped A_lo B_lo term
// and the split residues are about 2^-16 of the product).
//
// A CTA (one per SM) holds the DFT matrices and the twiddle table once (112 KB, copied
// with bulk asynchronous copies) and runs two independent pipelines, one per warpgroup,
// each on its own columns with its own 48 KB operand buffer, 256 tensor-memory columns
// and mbarrier: while one warpgroup converts accumulators the other one's MMAs run.
// Operands sit in shared memory in the canonical K-major layout without swizzle (core
// matrices of 8 rows x 16 bytes). One thread per warpgroup issues that warpgroup's MMAs
// and commits them to its mbarrier; the waits are bounded, record a timeout in the
// device flags and end the pipeline cleanly instead of hanging.
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
constexpr int kTcP = 1 << kTcLogP;        // 2048
constexpr int kTcNH = kTcP / 2 + 1;        // 1025 columns
constexpr int kTcThreads = 256;            // two warpgroups
constexpr int kTcPipe = 128;               // threads per pipeline
constexpr uint32_t kTcTmemCols = 512;      // 256 per pipeline

// shared-memory map (bytes from the 1024-aligned base): per pipeline p a data area of
// 48 KB (hi split at +0, lo split at +24 KB), then the constants
constexpr int kPipeBytes = 49152;
constexpr int kLoOff = 24576;
constexpr int kConst = 2 * kPipeBytes;
constexpr int kFaHi = kConst, kFaLo = kFaHi + 16384;            // 128 x 64
constexpr int kFbHi = kFaLo + 16384, kFbLo = kFbHi + 8192;      // 64 x 64
constexpr int kFbpHi = kFbLo + 8192, kFbpLo = kFbpHi + 8192;    // 64 (read as 128) x 64
constexpr int kFapHi = kFbpLo + 8192, kFapLo = kFapHi + 16384;  // 64 x 128
constexpr int kTw = kFapLo + 16384;                             // float2[2048] twiddles
constexpr int kConstBytes = kTw + 8 * kTcP - kConst;            // 114688
constexpr int kSmemBytes = kConst + kConstBytes + 1024;         // + alignment slack
static_assert(kConstBytes == 114688, "constant image size");
static_assert(kSmemBytes <= 227 * 1024, "shared memory");

// byte offset of element (row, kc) of a K-major bf16 operand with K columns
__host__ __device__ __forceinline__ int koff(int row, int kc, int K) {
    return (row >> 3) * (K * 16) + (kc >> 3) * 128 + (row & 7) * 16 + (kc & 7) * 2;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle; leading byte offset 128 (the
// next 8 K-columns), stride byte offset sbo (the next 8 rows)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
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

// barrier of one pipeline's 128 threads (named barrier 1 + p)
__device__ __forceinline__ void pipe_sync(int p) { asm volatile("bar.sync %0, 128;" ::"r"(1 + p) : "memory"); }
// same barrier, returning whether any of the 128 threads passed a true flag
__device__ __forceinline__ bool pipe_sync_or(int p, bool v) {
    uint32_t r;
    asm volatile(
        "{\n.reg .pred a, b;\nsetp.ne.u32 a, %1, 0;\nbar.red.or.pred b, %2, 128, a;\nselp.u32 %0, 1, 0, b;\n}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(1 + p)
        : "memory");
    return r != 0;
}

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

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes (thread i: lane base + i);
// the caller waits with tmem_wait() before using them
__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(addr));
}
__device__ __forceinline__ void tmem_ld16(uint32_t addr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(addr));
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float f32(uint32_t u) { return __uint_as_float(u); }

// Split 8 FP32 values into one 16-byte chunk of bf16 highs and one of bf16 lows and store
// them at byte offset `off` of the hi split and of the lo split.
__device__ __forceinline__ void put8(unsigned char* hi_base, int off, const float* x) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __nv_bfloat162 bh = __floats2bfloat162_rn(x[2 * q], x[2 * q + 1]);
        const float2 fh = __bfloat1622float2(bh);
        const __nv_bfloat162 bl = __floats2bfloat162_rn(x[2 * q] - fh.x, x[2 * q + 1] - fh.y);
        h[q] = *reinterpret_cast<const uint32_t*>(&bh);
        l[q] = *reinterpret_cast<const uint32_t*>(&bl);
    }
    *reinterpret_cast<uint4*>(hi_base + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(hi_base + kLoOff + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// Natural-order kernel spectra of column kx from the row-transformed kernel samples S1
// (FP32 shared-memory FFT along y, scaled by 1/P^2), in an iteration that rebuilds the
// spectrum. Whole CTA; sm holds 3 padded sequences.
__device__ void tc_spectrum(int kx, const float2* __restrict__ S1, const float2* __restrict__ tw, float* specN,
                            float2* sm) {
    constexpr int P = kTcP, PL = padded_len(P);
    for (int idx = threadIdx.x; idx < 3 * P; idx += blockDim.x) {
        const int c = idx / P, y = idx - c * P;
        sm[c * PL + spad(y)] = s1_row<P>(S1, c, kx, y);
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
    __syncthreads();
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_cols_tc(const float2* __restrict__ T1, float2* __restrict__ T2, int ystride, float* specN,
              const float2* __restrict__ S1, const float2* __restrict__ tw,
              const unsigned char* __restrict__ consts, DevState* __restrict__ st) {
    extern __shared__ unsigned char sm_raw[];
    __shared__ __align__(8) uint64_t mbar_mma[2];
    __shared__ __align__(8) uint64_t mbar_const;
    __shared__ uint32_t tmem_base_sh;
    unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x;
    const int p = tid >> 7;           // pipeline (warpgroup)
    const int t = tid & 127;          // thread in the pipeline = TMEM lane of its accumulator row
    const int q = t >> 5;             // lane quadrant of this warp
    const uint32_t s_base = smem_u32(sm);
    const uint32_t mb = smem_u32(&mbar_mma[p]), mc = smem_u32(&mbar_const);
    unsigned char* pd = sm + p * kPipeBytes;           // this pipeline's data (hi split)
    const uint32_t pd_hi = s_base + p * kPipeBytes, pd_lo = pd_hi + kLoOff;
    const float2* tws = reinterpret_cast<const float2*>(sm + kTw);

    // constants: bulk asynchronous copies of the 112 KB image, issued before waiting on
    // the previous kernel (they do not depend on it)
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar_mma[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar_mma[1])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mc));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mc), "r"(kConstBytes) : "memory");
        constexpr int kPiece = kConstBytes / 4;
        for (int i = 0; i < 4; ++i)
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    s_base + kConst + i * kPiece),
                "l"(consts + i * kPiece), "r"(kPiece), "r"(mc)
                : "memory");
    }
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(kTcTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base_sh + 256u * (uint32_t)p;  // this pipeline's 256 columns
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16);
    pdl_wait();
    pdl_trigger();
    const int G = st->grid.G;
    const int workers = 2 * gridDim.x;
    // a stale spectrum is rebuilt first, for every column this CTA's pipelines will take
    if (st->spec_dirty) {
        for (int w = 0; w < 2; ++w)
            for (int kx = 2 * blockIdx.x + w; kx < kTcNH; kx += workers)
                tc_spectrum(kx, S1, tw, specN, reinterpret_cast<float2*>(sm));
        __threadfence_block();
        __syncthreads();
    }
    bool ok = mbar_wait(mc, 0);
    uint32_t phase = 0;
    if (__syncthreads_or(!ok)) goto out;

    for (int kx = 2 * blockIdx.x + p; kx < kTcNH; kx += workers) {
        // ---- load: stage A operand, rows (c, n2), K (n1 < 32, re/im) interleaved
        {
            float2 v[3][8];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int it = t + kTcPipe * i;
                const int qq = it / 96, r = it - qq * 96;
                const int c = r >> 5, n2 = r & 31;
                const float2* src = T1 + ((size_t)c * kTcNH + kx) * ystride;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int y = 32 * (8 * qq + j) + n2;
                    v[i][j] = (y < G) ? src[y] : make_float2(0.f, 0.f);
                }
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int it = t + kTcPipe * i;
                const int qq = it / 96, r = it - qq * 96;
                float x[16];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    x[2 * j] = v[i][j].x;
                    x[2 * j + 1] = v[i][j].y;
                }
                put8(pd, koff(r, 16 * qq, 64), x);
                put8(pd, koff(r, 16 * qq + 8, 64), x + 8);
            }
        }
        fence_async_smem();
        fence_before();
        pipe_sync(p);
        // ---- stage A: D[0, 96) = FA (128 x 64) x data (96 rows)
        if (t == 0) {
            fence_after();
            mma3(tmem, s_base + kFaHi, s_base + kFaLo, 1024, pd_hi, pd_lo, 1024, 64, idesc_bf16(96));
            mma_commit(mb);
        }
        ok = mbar_wait(mb, phase);
        phase ^= 1u;
        fence_after();
        if (pipe_sync_or(p, !ok)) break;
        // ---- twiddle W2048^(n2 k1); stage B operand of channel c at c * 8 KB: row k1,
        //      K (re/im, n2) blocked
        {
            const int k1 = t >> 1, ro = t & 1;
            uint32_t r[3][32];
            tmem_ld32(lane_addr + 0u, r[0]);
            tmem_ld32(lane_addr + 32u, r[1]);
            tmem_ld32(lane_addr + 64u, r[2]);
            tmem_wait();
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float o[32];
#pragma unroll
                for (int n2 = 0; n2 < 32; ++n2) {
                    const float v = f32(r[c][n2]);
                    const float pv = __shfl_xor_sync(0xffffffffu, v, 1);
                    const float re = ro ? pv : v, im = ro ? v : pv;
                    const float2 w = tws[(n2 * k1) & (kTcP - 1)];
                    o[n2] = ro ? fmaf(re, w.y, im * w.x) : fmaf(re, w.x, -im * w.y);
                }
#pragma unroll
                for (int ch = 0; ch < 4; ++ch) put8(pd, c * 8192 + koff(k1, 32 * ro + 8 * ch, 64), o + 8 * ch);
            }
        }
        fence_async_smem();
        fence_before();
        pipe_sync(p);
        // ---- stage B: per channel c, D[64 c, 64 c + 64) = data_c (rows 0..63 used) x FB^T
        if (t == 0) {
            fence_after();
            for (int c = 0; c < 3; ++c)
                mma3(tmem + 64u * c, pd_hi + c * 8192, pd_lo + c * 8192, 1024, s_base + kFbHi, s_base + kFbLo, 1024,
                     64, idesc_bf16(64));
            mma_commit(mb);
        }
        ok = mbar_wait(mb, phase);
        phase ^= 1u;
        fence_after();
        if (pipe_sync_or(p, !ok)) break;
        // ---- spectral product at k = k1 + 64 k2 (lanes 0..63 = k1); stage B' operand:
        //      rows (c, k1), K (k2, re/im) interleaved
        if (q < 2) {
            const int k1 = t;
            const float* sK = specN + (size_t)kx * kTcP + k1;
            const float* sX = specN + ((size_t)kTcNH + kx) * kTcP + k1;
            const float* sY = specN + ((size_t)2 * kTcNH + kx) * kTcP + k1;
            // plain loads: in an iteration that rebuilds the spectrum this CTA has just
            // written these values (the non-coherent read-only path could miss them)
            float Kn[8], Xn[8], Yn[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                Kn[i] = sK[64 * i];
                Xn[i] = sX[64 * i];
                Yn[i] = sY[64 * i];
            }
#pragma unroll 1
            for (int blk = 0; blk < 4; ++blk) {  // k2 in [8 blk, 8 blk + 8)
                uint32_t rr[16], rx[16], ry[16];
                tmem_ld16(lane_addr + 16u * blk, rr);
                tmem_ld16(lane_addr + 64u + 16u * blk, rx);
                tmem_ld16(lane_addr + 128u + 16u * blk, ry);
                float Kc[8], Xc[8], Yc[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    Kc[i] = Kn[i];
                    Xc[i] = Xn[i];
                    Yc[i] = Yn[i];
                }
                if (blk < 3) {  // next block's spectra in flight during this one
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int k = 64 * (8 * (blk + 1) + i);
                        Kn[i] = sK[k];
                        Xn[i] = sX[k];
                        Yn[i] = sY[k];
                    }
                }
                tmem_wait();
                float oa[16], ox[16], oy[16];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float K = Kc[i], hx = Xc[i], hy = Yc[i];
                    const float rre = f32(rr[2 * i]), rim = f32(rr[2 * i + 1]);
                    oa[2 * i] = K * rre;
                    oa[2 * i + 1] = K * rim;
                    ox[2 * i] = fmaf(-hx, rim, -K * f32(rx[2 * i]));
                    ox[2 * i + 1] = fmaf(hx, rre, -K * f32(rx[2 * i + 1]));
                    oy[2 * i] = fmaf(-hy, rim, -K * f32(ry[2 * i]));
                    oy[2 * i + 1] = fmaf(hy, rre, -K * f32(ry[2 * i + 1]));
                }
                const int kc = 16 * blk;
                put8(pd, koff(k1, kc, 64), oa);
                put8(pd, koff(k1, kc + 8, 64), oa + 8);
                put8(pd, koff(64 + k1, kc, 64), ox);
                put8(pd, koff(64 + k1, kc + 8, 64), ox + 8);
                put8(pd, koff(128 + k1, kc, 64), oy);
                put8(pd, koff(128 + k1, kc + 8, 64), oy + 8);
            }
        }
        fence_async_smem();
        fence_before();
        pipe_sync(p);
        // ---- stage B': D[0, 192) = FB' (rows 0..63 used) x data (192 rows)
        if (t == 0) {
            fence_after();
            mma3(tmem, s_base + kFbpHi, s_base + kFbpLo, 1024, pd_hi, pd_lo, 1024, 64, idesc_bf16(192));
            mma_commit(mb);
        }
        ok = mbar_wait(mb, phase);
        phase ^= 1u;
        fence_after();
        if (pipe_sync_or(p, !ok)) break;
        // ---- twiddle W2048^(-n2 k1) (lanes 0..63 = (n2, re/im)); stage A' operand: rows
        //      (c, n2), K (re/im, k1) blocked, 128 wide
        if (q < 2) {
            const int n2 = t >> 1, ro = t & 1;
#pragma unroll 1
            for (int c = 0; c < 3; ++c) {
                uint32_t r[2][32];
                tmem_ld32(lane_addr + 64u * c, r[0]);
                tmem_ld32(lane_addr + 64u * c + 32u, r[1]);
                tmem_wait();
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float o[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const float v = f32(r[h][i]);
                        const float pv = __shfl_xor_sync(0xffffffffu, v, 1);
                        const float re = ro ? pv : v, im = ro ? v : pv;
                        const float2 w = tws[(n2 * (32 * h + i)) & (kTcP - 1)];
                        o[i] = ro ? fmaf(im, w.x, -re * w.y) : fmaf(re, w.x, im * w.y);
                    }
#pragma unroll
                    for (int ch = 0; ch < 4; ++ch)
                        put8(pd, koff(32 * c + n2, 64 * ro + 32 * h + 8 * ch, 128), o + 8 * ch);
                }
            }
        }
        fence_async_smem();
        fence_before();
        pipe_sync(p);
        // ---- stage A': D[0, 64) = data rows 0..127 (96 used) x FA'^T
        if (t == 0) {
            fence_after();
            mma3(tmem, pd_hi, pd_lo, 2048, s_base + kFapHi, s_base + kFapLo, 2048, 128, idesc_bf16(64));
            mma_commit(mb);
        }
        ok = mbar_wait(mb, phase);
        phase ^= 1u;
        fence_after();
        if (pipe_sync_or(p, !ok)) break;
        // ---- outputs: lane (c, n2), columns (n1, re/im) -> T2[c][kx][32 n1 + n2]
        if (q < 3) {
            const int c = q, n2 = t & 31;
            uint32_t r[2][32];
            tmem_ld32(lane_addr + 0u, r[0]);
            tmem_ld32(lane_addr + 32u, r[1]);
            tmem_wait();
            float2* dst = T2 + ((size_t)c * kTcNH + kx) * ystride;
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int y = 32 * (16 * h + i) + n2;
                    if (y < G) dst[y] = make_float2(f32(r[h][2 * i]), f32(r[h][2 * i + 1]));
                }
        }
        fence_before();
        pipe_sync(p);  // TMEM reads done before this pipeline's next MMAs overwrite it
        fence_after();
    }
out:
    if (!ok && t == 0) atomicOr(&st->flags, FLAG_WAIT_TIMEOUT);
    fence_before();
    __syncthreads();
    if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base_sh),
                               "r"(kTcTmemCols));
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

// Store x as (hi, lo) bf16 at element (row, kc) of the matrix whose hi split starts at
// `hi` and lo split at `lo` (byte offsets in the shared-memory map).
void put_const(std::vector<unsigned char>& img, int hi, int lo, int row, int kc, int K, double x) {
    const uint16_t h = bf16_rn((float)x);
    const uint16_t l = bf16_rn((float)(x - (double)bf16_to_f(h)));
    const int o = koff(row, kc, K);
    std::memcpy(&img[(size_t)(hi - kConst + o)], &h, 2);
    std::memcpy(&img[(size_t)(lo - kConst + o)], &l, 2);
}

}  // namespace

// The 112 KB shared-memory image of the four DFT matrices (hi and lo splits) and the
// FP32 twiddle table, built in FP64. With c + i s = exp(-2 pi i n k / N):
//   FA  [(k1, ro)][(n1, ri)]  forward 64-point DFT, inputs n1 < 32   (rows 2 k1 + ro, cols 2 n1 + ri)
//   FB  [(k2, ro)][(ri, n2)]  forward 32-point DFT                   (rows 2 k2 + ro, cols 32 ri + n2)
//   FB' [(n2, ro)][(k2, ri)]  inverse 32-point DFT                   (rows 2 n2 + ro, cols 2 k2 + ri)
//   FA' [(n1, ro)][(ri, k1)]  inverse 64-point DFT, outputs n1 < 32  (rows 2 n1 + ro, cols 64 ri + k1)
// Forward entries: Re row (c, -s), Im row (s, c); inverse: Re row (c, s), Im row (-s, c).
// Twiddles: tw[t] = exp(-2 pi i t / 2048).
void build_tc_constants(std::vector<unsigned char>& img) {
    img.assign((size_t)kConstBytes, 0);
    const double pi = 3.14159265358979323846;
    for (int k1 = 0; k1 < 64; ++k1)
        for (int n1 = 0; n1 < 32; ++n1) {
            const double a = -2.0 * pi * (double)((n1 * k1) % 64) / 64.0, c = std::cos(a), s = std::sin(a);
            put_const(img, kFaHi, kFaLo, 2 * k1, 2 * n1, 64, c);
            put_const(img, kFaHi, kFaLo, 2 * k1, 2 * n1 + 1, 64, -s);
            put_const(img, kFaHi, kFaLo, 2 * k1 + 1, 2 * n1, 64, s);
            put_const(img, kFaHi, kFaLo, 2 * k1 + 1, 2 * n1 + 1, 64, c);
            put_const(img, kFapHi, kFapLo, 2 * n1, k1, 128, c);
            put_const(img, kFapHi, kFapLo, 2 * n1, 64 + k1, 128, s);
            put_const(img, kFapHi, kFapLo, 2 * n1 + 1, k1, 128, -s);
            put_const(img, kFapHi, kFapLo, 2 * n1 + 1, 64 + k1, 128, c);
        }
    for (int k2 = 0; k2 < 32; ++k2)
        for (int n2 = 0; n2 < 32; ++n2) {
            const double a = -2.0 * pi * (double)((n2 * k2) % 32) / 32.0, c = std::cos(a), s = std::sin(a);
            put_const(img, kFbHi, kFbLo, 2 * k2, n2, 64, c);
            put_const(img, kFbHi, kFbLo, 2 * k2, 32 + n2, 64, -s);
            put_const(img, kFbHi, kFbLo, 2 * k2 + 1, n2, 64, s);
            put_const(img, kFbHi, kFbLo, 2 * k2 + 1, 32 + n2, 64, c);
            put_const(img, kFbpHi, kFbpLo, 2 * n2, 2 * k2, 64, c);
            put_const(img, kFbpHi, kFbpLo, 2 * n2, 2 * k2 + 1, 64, s);
            put_const(img, kFbpHi, kFbpLo, 2 * n2 + 1, 2 * k2, 64, -s);
            put_const(img, kFbpHi, kFbpLo, 2 * n2 + 1, 2 * k2 + 1, 64, c);
        }
    for (int i = 0; i < kTcP; ++i) {
        const double a = -2.0 * pi * (double)i / (double)kTcP;
        const float2 w = make_float2((float)std::cos(a), (float)std::sin(a));
        std::memcpy(&img[(size_t)(kTw - kConst) + 8 * (size_t)i], &w, 8);
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
    const int grid = sms < (kTcNH + 1) / 2 ? sms : (kTcNH + 1) / 2;
    return launch_pdl(k_cols_tc, grid, kTcThreads, (size_t)kSmemBytes, s, (const float2*)a.T1, a.T2, a.ystride,
                      specN, (const float2*)a.S1, a.tw, consts, a.st);
}

}  // namespace tfdp
