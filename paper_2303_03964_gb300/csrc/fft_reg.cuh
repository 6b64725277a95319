// fft_reg.cuh -- register-resident power-of-two FFTs (FP32), shared memory only for
// the exchanges between passes.
//
// A sequence of N = 2^LOGN complex values is held by T = N/8 threads, eight values
// each. The forward transform is the same decimation-in-frequency sequence of passes
// as fft.cuh (radix 8, then one radix-2 or radix-4 pass), so it produces the same
// digit-reversed order (pos_of_freq). Mappings of thread t's eight values:
//
//   M_p  (radix-8 pass p, span S = N / 8^p): element g S + j + r S/8,
//        j = t mod S/8, g = t div S/8, r = 0..7
//   MF   (after the last pass): element 8t + r
//
// M_0 is unit stride across threads (natural-order input / output), MF is the
// digit-reversed output. Between passes the values go through shared memory with the
// XOR swizzle i -> i ^ ((i >> 3) & 15): for every M_p and MF pattern the 16 lanes of
// a half-warp then hit 16 different 8-byte bank pairs (no bank conflicts for float2).
//
// A convolution does: load M_0 from global, forward, pointwise product in MF (in
// registers), inverse, store M_0 to global. The inverse is the mirrored
// decimation-in-time sequence without the 1/N factor.
#pragma once

#include "fft.cuh"

namespace tfdp {

__device__ __forceinline__ int swz(int i) { return i ^ ((i >> 3) & 15); }

template <int LOGN>
struct RegPlan {
    static constexpr int N = 1 << LOGN;
    static constexpr int T = N / 8;       // threads per sequence
    static constexpr int NP8 = LOGN / 3;  // radix-8 passes
    static constexpr int REM = LOGN % 3;  // 0, 1 (radix 2) or 2 (radix 4)
    // element of value r of thread t in mapping p (p = NP8 means MF)
    __device__ static __forceinline__ int elem(int p, int t, int r) {
        if (p >= NP8) return 8 * t + r;
        const int lsr = LOGN - 3 * p - 3;  // log2(S / 8)
        const int j = t & ((1 << lsr) - 1);
        const int g = t >> lsr;
        return (g << (lsr + 3)) + j + (r << lsr);
    }
};

// Twiddles w^q, q = 1..7, w = exp(-2 pi i j / S) = tw[j N / S]: three table reads,
// the rest by at most two products.
template <int LOGN>
__device__ __forceinline__ void twiddles8(int p, int t, const float2* __restrict__ tw, float2* w) {
    constexpr int N = 1 << LOGN;
    const int lsr = LOGN - 3 * p - 3;
    const int j = t & ((1 << lsr) - 1);
    const int step = j << (3 * p);  // j * N / S
    w[1] = __ldg(tw + step);
    w[2] = __ldg(tw + ((2 * step) & (N - 1)));
    w[4] = __ldg(tw + ((4 * step) & (N - 1)));
    w[3] = cmul(w[1], w[2]);
    w[5] = cmul(w[1], w[4]);
    w[6] = cmul(w[2], w[4]);
    w[7] = cmul(w[3], w[4]);
}

// Move the NS sequences of values from mapping pa to mapping pb through shared memory.
template <int LOGN, int NS>
__device__ __forceinline__ void reg_exchange(float2 (&v)[NS][8], float2* sm, int t, int pa, int pb) {
    using Pl = RegPlan<LOGN>;
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int r = 0; r < 8; ++r) sm[s * Pl::N + swz(Pl::elem(pa, t, r))] = v[s][r];
    __syncthreads();
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int r = 0; r < 8; ++r) v[s][r] = sm[s * Pl::N + swz(Pl::elem(pb, t, r))];
}

// Forward DIF transform. In: M_0 (natural order). Out: MF (digit-reversed order).
// sm holds NS sequences of N values for the exchanges; the caller must __syncthreads()
// before reusing sm afterwards.
template <int LOGN, int NS>
__device__ __forceinline__ void reg_fft_forward(float2 (&v)[NS][8], float2* sm, const float2* __restrict__ tw,
                                                int t) {
    using Pl = RegPlan<LOGN>;
#pragma unroll
    for (int p = 0; p < Pl::NP8; ++p) {
        if (p > 0) reg_exchange<LOGN, NS>(v, sm, t, p - 1, p);
        float2 w[8];
        twiddles8<LOGN>(p, t, tw, w);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            dft_small<8, false>(v[s]);
#pragma unroll
            for (int q = 1; q < 8; ++q) v[s][q] = cmul(v[s][q], w[q]);
        }
    }
    if (Pl::REM > 0) {
        reg_exchange<LOGN, NS>(v, sm, t, Pl::NP8 - 1, Pl::NP8);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            if (Pl::REM == 2) {
                dft_small<4, false>(v[s]);
                dft_small<4, false>(v[s] + 4);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) dft_small<2, false>(v[s] + 2 * q);
            }
        }
    }
}

// Inverse DIT transform (no 1/N). In: MF (digit-reversed). Out: M_0 (natural order).
template <int LOGN, int NS>
__device__ __forceinline__ void reg_fft_inverse(float2 (&v)[NS][8], float2* sm, const float2* __restrict__ tw,
                                                int t) {
    using Pl = RegPlan<LOGN>;
    if (Pl::REM > 0) {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            if (Pl::REM == 2) {
                dft_small<4, true>(v[s]);
                dft_small<4, true>(v[s] + 4);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) dft_small<2, true>(v[s] + 2 * q);
            }
        }
        reg_exchange<LOGN, NS>(v, sm, t, Pl::NP8, Pl::NP8 - 1);
    }
#pragma unroll
    for (int p = Pl::NP8 - 1; p >= 0; --p) {
        float2 w[8];
        twiddles8<LOGN>(p, t, tw, w);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
#pragma unroll
            for (int q = 1; q < 8; ++q) v[s][q] = cmulc(v[s][q], w[q]);
            dft_small<8, true>(v[s]);
        }
        if (p > 0) reg_exchange<LOGN, NS>(v, sm, t, p, p - 1);
    }
}

}  // namespace tfdp
