// fft.cuh -- in-place power-of-two complex FFTs on shared memory, FP32.
//
// The forward transform is decimation in frequency (DIF): natural-order input,
// output in mixed-radix digit-reversed order. The inverse is the mirrored
// decimation in time (DIT): it takes that digit-reversed order and returns natural
// order. A convolution (forward, pointwise product, inverse) therefore never
// reorders its data; only the real-to-complex / complex-to-real split of the row
// transforms needs the position of a frequency, given by pos_of_freq().
//
// Passes use radix 8 while possible; a last radix-4 or radix-2 pass covers the
// remaining factor. Twiddles come from a table tw[t] = exp(-2 pi i t / N) computed
// on the host in FP64. Shared-memory addresses are padded by one element every
// eight to spread the strided accesses of the short-span passes over the banks.
#pragma once

#include <cuda_runtime.h>

namespace tfdp {

__device__ __forceinline__ int spad(int i) { return i + (i >> 3); }

// Padded length of one sequence of N elements.
__host__ __device__ constexpr int padded_len(int n) { return n + (n >> 3); }

template <int LOGN>
struct FftPlan {
    static constexpr int N = 1 << LOGN;
    static constexpr int N8 = LOGN / 3;          // radix-8 passes
    static constexpr int REM = LOGN % 3;         // 0, 1 (radix 2) or 2 (radix 4)
    static constexpr int NPASS = N8 + (REM ? 1 : 0);
    // log2 radix of pass i (DIF order)
    __host__ __device__ static constexpr int lr(int i) { return (i < N8) ? 3 : REM; }
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// In-register DFT of size R (2, 4, 8): y_q = sum_r v_r w^(rq), w = exp(-+2 pi i / R).
template <int R, bool INV>
__device__ __forceinline__ void dft_small(float2* v) {
    if (R == 2) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if (R == 4) {
        float2 e0 = cadd(v[0], v[2]), e1 = csub(v[0], v[2]);
        float2 o0 = cadd(v[1], v[3]), o1 = mul_mi<INV>(csub(v[1], v[3]));
        v[0] = cadd(e0, o0);
        v[2] = csub(e0, o0);
        v[1] = cadd(e1, o1);
        v[3] = csub(e1, o1);
    } else {  // R == 8
        float2 e[4] = {v[0], v[2], v[4], v[6]};
        float2 o[4] = {v[1], v[3], v[5], v[7]};
        dft_small<4, INV>(e);
        dft_small<4, INV>(o);
        const float s = 0.70710678118654752440f;
        // o[q] *= w8^q
        float2 o1 = o[1], o3 = o[3];
        o[1] = INV ? make_float2(s * (o1.x - o1.y), s * (o1.x + o1.y))
                   : make_float2(s * (o1.x + o1.y), s * (o1.y - o1.x));
        o[2] = mul_mi<INV>(o[2]);
        o[3] = INV ? make_float2(-s * (o3.x + o3.y), s * (o3.x - o3.y))
                   : make_float2(s * (o3.y - o3.x), -s * (o3.x + o3.y));
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            v[q] = cadd(e[q], o[q]);
            v[q + 4] = csub(e[q], o[q]);
        }
    }
}

// One DIF (forward) or DIT (inverse) pass of radix R = 2^LR over span S on NSEQ
// sequences stored at buf + s * padded_len(N). Threads stride over butterflies.
template <int LOGN, int LR, bool INV>
__device__ __forceinline__ void fft_pass(float2* __restrict__ buf, int nseq, int S,
                                         const float2* __restrict__ tw) {
    constexpr int N = 1 << LOGN;
    constexpr int R = 1 << LR;
    constexpr int PL = padded_len(N);
    const int sr = S / R;           // distance between butterfly elements
    const int tws = N / S;          // twiddle index stride
    const int nb = nseq * (N / R);  // butterflies in this pass
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const int s = b / (N / R);
        const int bb = b - s * (N / R);
        const int j = bb % sr;
        const int base = (bb / sr) * S;
        float2* seq = buf + s * PL;
        float2 v[R];
        if (!INV) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = seq[spad(base + j + r * sr)];
            dft_small<R, false>(v);
#pragma unroll
            for (int q = 1; q < R; ++q) v[q] = cmul(v[q], __ldg(tw + j * q * tws));
        } else {
            v[0] = seq[spad(base + j)];
#pragma unroll
            for (int q = 1; q < R; ++q) v[q] = cmulc(seq[spad(base + j + q * sr)], __ldg(tw + j * q * tws));
            dft_small<R, true>(v);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) seq[spad(base + j + r * sr)] = v[r];
    }
}

// Forward transform (DIF) of nseq sequences: natural in, digit-reversed out.
template <int LOGN>
__device__ void fft_forward(float2* buf, int nseq, const float2* tw) {
    using Pl = FftPlan<LOGN>;
    int S = Pl::N;
#pragma unroll
    for (int i = 0; i < Pl::NPASS; ++i) {
        const int lr = Pl::lr(i);
        if (lr == 3) fft_pass<LOGN, 3, false>(buf, nseq, S, tw);
        else if (lr == 2) fft_pass<LOGN, 2, false>(buf, nseq, S, tw);
        else fft_pass<LOGN, 1, false>(buf, nseq, S, tw);
        S >>= lr;
        __syncthreads();
    }
}

// Inverse transform (DIT, no 1/N): digit-reversed in, natural out.
template <int LOGN>
__device__ void fft_inverse(float2* buf, int nseq, const float2* tw) {
    using Pl = FftPlan<LOGN>;
    // spans in DIF order are N, N/R0, N/(R0 R1), ...; the inverse walks them backwards
    int spans[Pl::NPASS];
    int S = Pl::N;
#pragma unroll
    for (int i = 0; i < Pl::NPASS; ++i) { spans[i] = S; S >>= Pl::lr(i); }
#pragma unroll
    for (int i = Pl::NPASS - 1; i >= 0; --i) {
        const int lr = Pl::lr(i);
        if (lr == 3) fft_pass<LOGN, 3, true>(buf, nseq, spans[i], tw);
        else if (lr == 2) fft_pass<LOGN, 2, true>(buf, nseq, spans[i], tw);
        else fft_pass<LOGN, 1, true>(buf, nseq, spans[i], tw);
        __syncthreads();
    }
}

// Storage position (unpadded) of frequency k after fft_forward. With DIF radices
// R_0 .. R_{m-1}, position p = sum_i p_i N / (R_0 .. R_i) holds frequency
// k = sum_i p_i (R_0 .. R_{i-1}): the digit fields appear in reverse order.
template <int LOGN>
__device__ __forceinline__ int pos_of_freq(int k) {
    using Pl = FftPlan<LOGN>;
    int p = 0, kb = 0, pb = LOGN;
#pragma unroll
    for (int i = 0; i < Pl::NPASS; ++i) {
        const int lr = Pl::lr(i);
        const int digit = (k >> kb) & ((1 << lr) - 1);
        pb -= lr;
        p |= digit << pb;
        kb += lr;
    }
    return p;
}

template <int LOGN>
__device__ __forceinline__ int freq_of_pos(int p) {
    using Pl = FftPlan<LOGN>;
    int k = 0, kb = 0, pb = LOGN;
#pragma unroll
    for (int i = 0; i < Pl::NPASS; ++i) {
        const int lr = Pl::lr(i);
        pb -= lr;
        const int digit = (p >> pb) & ((1 << lr) - 1);
        k |= digit << kb;
        kb += lr;
    }
    return k;
}

// ---------------------------------------------------------------- kernel-sample rows
// Rows of the kernel samples that a spectrum rebuild transforms along x: 0 .. P/2. The
// three kernels are even in D_y (K, D_x K) or odd (D_y K), so the row-transformed samples
// of row P - y are those of row y, negated for channel 2; s1_row reads them that way.
__host__ __device__ constexpr int spec_rows(int P) { return P / 2 + 1; }

template <int P>
__device__ __forceinline__ float2 s1_row(const float2* __restrict__ S1, int c, int kx, int y) {
    const bool mirror = y > P / 2;
    float2 w = S1[((size_t)c * (P / 2 + 1) + kx) * P + (mirror ? P - y : y)];
    if (mirror && c == 2) {
        w.x = -w.x;
        w.y = -w.y;
    }
    return w;
}

}  // namespace tfdp
