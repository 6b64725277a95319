// node_dev.cuh -- per-node device functions of the ibFFT path and the update, shared
// by the single-graph kernels (node_kernels.cu) and the batch kernels
// (batch_kernel.cuh) so that both compute identical per-node arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"

namespace tfdp {

// ---------------------------------------------------------------- box geometry
struct AxisGeom {
    float lo, h_hi, h_lo, hk;  // origin, box side as hi + lo FP32 pair, h / k
    float q_scale, q_inv;      // fixed-point scale of the spread sums and its inverse
    int n_int;
};

__device__ __forceinline__ AxisGeom axis_geom(const GridDesc& g) {
    AxisGeom a;
    a.lo = g.lo_f;
    a.h_hi = g.h_f;
    a.h_lo = g.h_lo_f;
    a.hk = g.hk_f;
    a.q_scale = g.q_scale;
    a.q_inv = g.q_inv;
    a.n_int = g.n_int;
    return a;
}

// Offset of x from the origin lo + b h of box b, accurate to a few ulps of h.
__device__ __forceinline__ float box_offset_at(float x, int b, const AxisGeom& a) {
    // x - lo = s + e exactly (TwoSum)
    const float s = __fsub_rn(x, a.lo);
    const float bb = __fsub_rn(s, x);
    const float e = __fadd_rn(__fsub_rn(x, __fsub_rn(s, bb)), __fsub_rn(-a.lo, bb));
    // b * h_hi = p + pe exactly
    const float fb = (float)b;
    const float p = __fmul_rn(fb, a.h_hi);
    const float pe = __fmaf_rn(fb, a.h_hi, -p);
    return __fadd_rn(__fsub_rn(s, p), __fsub_rn(__fsub_rn(e, pe), __fmul_rn(fb, a.h_lo)));
}

// Box index b (the FP32 decision shared with the oracle) and the offset of x from the
// box origin lo + b h.
__device__ __forceinline__ int box_offset(float x, const AxisGeom& a, float* off) {
    float tq;
    const int b = box_of(x, a.lo, a.h_hi, a.n_int, &tq);
    *off = box_offset_at(x, b, a);
    return b;
}

__device__ __forceinline__ float warp_sumf(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------- attraction + update
// alpha * sum_{j <-> i} (1 + beta / (1 + d^2)) (x_j - x_i), Eq. (newforce).
__device__ __forceinline__ float rcp_fast(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// With local-refinement weights (W, wa) the edge (i, j) is scaled by a_i a_j.
template <bool W>
__device__ __forceinline__ float2 attraction_t(int i, float2 p, const int* __restrict__ rowptr,
                                               const int* __restrict__ col, const float2* __restrict__ xy,
                                               float alpha, float beta, const float* __restrict__ wa) {
    float fx = 0.0f, fy = 0.0f;
    int e = rowptr[i];
    const int e1 = rowptr[i + 1];
    // four neighbours per round so that their loads are in flight together
    for (; e + 4 <= e1; e += 4) {
        int j[4];
        float2 q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) j[u] = __ldg(col + e + u);
#pragma unroll
        for (int u = 0; u < 4; ++u) q[u] = xy[j[u]];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float dx = q[u].x - p.x, dy = q[u].y - p.y;
            float c = fmaf(beta, rcp_fast(1.0f + (dx * dx + dy * dy)), 1.0f);
            if (W) c *= __ldg(wa + j[u]);
            fx = fmaf(c, dx, fx);
            fy = fmaf(c, dy, fy);
        }
    }
    for (; e < e1; ++e) {
        const int j = __ldg(col + e);
        const float2 q = xy[j];
        const float dx = q.x - p.x, dy = q.y - p.y;
        float c = fmaf(beta, rcp_fast(1.0f + (dx * dx + dy * dy)), 1.0f);
        if (W) c *= __ldg(wa + j);
        fx = fmaf(c, dx, fx);
        fy = fmaf(c, dy, fy);
    }
    const float s = W ? alpha * __ldg(wa + i) : alpha;
    return make_float2(s * fx, s * fy);
}

__device__ __forceinline__ float2 attraction(int i, float2 p, const int* __restrict__ rowptr,
                                             const int* __restrict__ col, const float2* __restrict__ xy,
                                             float alpha, float beta, const float* __restrict__ wa) {
    return wa ? attraction_t<true>(i, p, rowptr, col, xy, alpha, beta, wa)
              : attraction_t<false>(i, p, rowptr, col, xy, alpha, beta, nullptr);
}

// The same sum for one node by the 32 lanes of a warp: lane l takes neighbours l, l + 32,
// ... (four per round), then a fixed butterfly adds the lanes, so the result does not
// depend on scheduling. All lanes return the sum.
template <bool W>
__device__ __forceinline__ float2 attraction_warp(int i, float2 p, const int* __restrict__ rowptr,
                                                  const int* __restrict__ col, const float2* __restrict__ xy,
                                                  float alpha, float beta, const float* __restrict__ wa, int lane) {
    float fx = 0.0f, fy = 0.0f;
    int e = rowptr[i] + lane;
    const int e1 = rowptr[i + 1];
    for (; e + 96 < e1; e += 128) {
        int j[4];
        float2 q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) j[u] = __ldg(col + e + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; ++u) q[u] = xy[j[u]];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float dx = q[u].x - p.x, dy = q[u].y - p.y;
            float c = fmaf(beta, rcp_fast(1.0f + (dx * dx + dy * dy)), 1.0f);
            if (W) c *= __ldg(wa + j[u]);
            fx = fmaf(c, dx, fx);
            fy = fmaf(c, dy, fy);
        }
    }
    for (; e < e1; e += 32) {
        const int j = __ldg(col + e);
        const float2 q = xy[j];
        const float dx = q.x - p.x, dy = q.y - p.y;
        float c = fmaf(beta, rcp_fast(1.0f + (dx * dx + dy * dy)), 1.0f);
        if (W) c *= __ldg(wa + j);
        fx = fmaf(c, dx, fx);
        fy = fmaf(c, dy, fy);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
    }
    const float s = W ? alpha * __ldg(wa + i) : alpha;
    return make_float2(s * fx, s * fy);
}

// x + D min(1, s / |D|)
__device__ __forceinline__ float2 capped_step(float2 p, float2 D, float s) {
    const float d2 = D.x * D.x + D.y * D.y;
    const float c = (d2 > s * s) ? s * rsqrtf(d2) : 1.0f;
    return make_float2(fmaf(c, D.x, p.x), fmaf(c, D.y, p.y));
}

// The grid of iteration t = st->iter from the layout extremes (exact FP64 decisions),
// the step s_t, the spectrum key and the bookkeeping of the iteration (one thread).
// with_step = false leaves st->step_cur to the caller (k_grid fetches it on another lane).
__device__ __forceinline__ void grid_decide(DevState* st, const DevParams& prm, int advance, bool with_step = true) {
    // both bbox slots are loaded with the counter, so no load waits on another
    const unsigned b00 = st->bbox[0][0], b01 = st->bbox[0][1], b10 = st->bbox[1][0], b11 = st->bbox[1][1];
    const long long t = st->iter;
    const int cur = (int)(t & 1);
    const int kt = k_of_iter(prm.k, t, prm.total_iters);
    const GridDesc g = make_grid(ord2f(cur ? b10 : b00), ord2f(cur ? b11 : b01), prm, kt);
    st->grid = g;
    st->t_cur = t;
    if (with_step) st->step_cur = step_size(t, prm);
    st->net_frep[0] = 0.0;
    st->net_frep[1] = 0.0;
    if (advance) {
        st->bbox[cur ^ 1][0] = kOrdMinInit;
        st->bbox[cur ^ 1][1] = kOrdMaxInit;
    }
    const bool valid = st->spec_valid && st->spec_h == g.h && st->spec_gamma == prm.gamma &&
                       st->spec_k == kt && st->spec_P == prm.P;
    st->spec_dirty = valid ? 0 : 1;
    if (!valid) {
        st->spec_h = g.h;
        st->spec_gamma = prm.gamma;
        st->spec_k = kt;
        st->spec_P = prm.P;
        st->spec_valid = 1;
        st->spec_builds += 1;
    }
}

// ---------------------------------------------------------------- spread and gather
// Fixed-point spread sums. Each term w (|w| <= 3.52 for k <= 3, since a 1D Lagrange
// weight on [0, 1) is at most 1.875) and w d / h (|d| <= 1.5 h), times the node's
// repulsion weight r <= 2^spread_shift, is rounded to an int32 multiple of
// 2^-(27 - spread_shift) (the grid's q_inv) and summed in int64: the sums are exact, so
// they do not depend on the order of the nodes in a box (which the parallel sort leaves
// open) and every iteration is bitwise reproducible. Without weights the quantum is
// 2^-27 = 7.5e-9, far below the FP32 resolution of the results.

__device__ __forceinline__ long long spread_q(float v) {
    // round to nearest even; a float-to-integer conversion saturates to the int32 range
    // by itself (in-box terms stay below 2^30), so no clamp is needed to keep it defined
    return (long long)__float2int_rn(v);
}

// int64 -> FP32 rounded to nearest even, equal to (float)v, in 32-bit integer and FP32
// operations only. For |v| < 2^48 (every sum a box of fewer than ~10^5 nodes produces)
// v = h 2^24 + lo with h, lo exact in FP32, and one FP32 addition rounds the exact sum
// once; larger values take the library conversion.
__device__ __forceinline__ float ll2f_rn(long long v) {
    const unsigned lo32 = (unsigned)v;
    const int hi32 = (int)((unsigned long long)v >> 32);
    if (hi32 >= -(1 << 16) && hi32 < (1 << 16)) {                  // -2^48 <= v < 2^48
        const int h = (int)__funnelshift_r(lo32, (unsigned)hi32, 24);  // v >> 24
        const int lo = (int)(lo32 & 0xFFFFFFu);                        // v mod 2^24
        return __fadd_rn(__int2float_rn(h) * 16777216.0f, __int2float_rn(lo));
    }
    return __ll2float_rn(v);
}

// Lagrange projection (Sec. 3.4 step 1) of the nodes sxy[s0, s1) of box (bx, by) onto its
// K x K grid nodes: rho = sum w, m^x = sum w (x - y^x), m^y = sum w (y - y^y), written to
// the three planes of gin (row stride Gs, plane stride Gs^2). With local-refinement
// weights vw (sorted order; nullptr: all 1) each node's charge is r w.
template <int K>
__device__ __forceinline__ void spread_box(const float2* __restrict__ sxy, const float* __restrict__ vw, int s0,
                                           int s1, int bx, int by, const AxisGeom& ag, float* __restrict__ gin,
                                           int Gs) {
    const size_t plane = (size_t)Gs * Gs;
    long long rho[K][K], mx[K][K], my[K][K];  // fixed point; moments in units of h
#pragma unroll
    for (int ly = 0; ly < K; ++ly)
#pragma unroll
        for (int lx = 0; lx < K; ++lx) rho[ly][lx] = mx[ly][lx] = my[ly][lx] = 0;
    const float inv_h = 1.0f / ag.h_hi;
    // two nodes per round: both loads are in flight before either is used
    for (int s = s0; s < s1; s += 2) {
        const bool two = s + 1 < s1;
        float2 pp[2];
        float rr[2] = {ag.q_scale, ag.q_scale};  // node weight times the fixed-point scale
        pp[0] = sxy[s];
        pp[1] = two ? sxy[s + 1] : pp[0];
        if (vw) {
            rr[0] *= vw[s];
            rr[1] *= two ? vw[s + 1] : 1.0f;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (u == 1 && !two) break;
            // the node's box is (bx, by): the sort placed it there by the same FP32
            // decision, so only the offsets are formed here
            const float ox = box_offset_at(pp[u].x, bx, ag);
            const float oy = box_offset_at(pp[u].y, by, ag);
            float wx[K], wy[K], dx[K], dy[K];
            lagrange<K>(ox * inv_h, wx);
            lagrange<K>(oy * inv_h, wy);
#pragma unroll
            for (int l = 0; l < K; ++l) {
                dx[l] = (ox - ((float)l + 0.5f) * ag.hk) * inv_h;
                dy[l] = (oy - ((float)l + 0.5f) * ag.hk) * inv_h;
                wy[l] *= rr[u];  // the scale is a power of two: exact without weights
            }
#pragma unroll
            for (int ly = 0; ly < K; ++ly)
#pragma unroll
                for (int lx = 0; lx < K; ++lx) {
                    const float w = wx[lx] * wy[ly];
                    rho[ly][lx] += spread_q(w);
                    mx[ly][lx] += spread_q(w * dx[lx]);
                    my[ly][lx] += spread_q(w * dy[ly]);
                }
        }
    }
    const float hs = ag.h_hi * ag.q_inv;
#pragma unroll
    for (int ly = 0; ly < K; ++ly)
#pragma unroll
        for (int lx = 0; lx < K; ++lx) {
            const size_t q = (size_t)(by * K + ly) * Gs + (bx * K + lx);
            gin[q] = ll2f_rn(rho[ly][lx]) * ag.q_inv;
            gin[plane + q] = ll2f_rn(mx[ly][lx]) * hs;
            gin[2 * plane + q] = ll2f_rn(my[ly][lx]) * hs;
        }
}

// spread_box shared by the L lanes of an aligned lane group (gmask), for grids with few
// boxes (one thread per box would leave most of the GPU idle): lane g takes the nodes
// s0 + g, s0 + g + L, ... and the lanes' int64 sums are combined by an xor butterfly.
// The sums are exact, so the result is bit for bit that of spread_box.
template <int K, int L>
__device__ __forceinline__ void spread_box_group(const float2* __restrict__ sxy, const float* __restrict__ vw,
                                                 int s0, int s1, int bx, int by, int g, unsigned gmask,
                                                 const AxisGeom& ag, float* __restrict__ gin, int Gs) {
    const size_t plane = (size_t)Gs * Gs;
    long long acc[3][K][K];  // rho, m^x, m^y in fixed point; moments in units of h
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int ly = 0; ly < K; ++ly)
#pragma unroll
            for (int lx = 0; lx < K; ++lx) acc[c][ly][lx] = 0;
    const float inv_h = 1.0f / ag.h_hi;
    for (int s = s0 + g; s < s1; s += 2 * L) {
        const bool two = s + L < s1;
        float2 pp[2];
        float rr[2] = {ag.q_scale, ag.q_scale};
        pp[0] = sxy[s];
        pp[1] = two ? sxy[s + L] : pp[0];
        if (vw) {
            rr[0] *= vw[s];
            rr[1] *= two ? vw[s + L] : 1.0f;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (u == 1 && !two) break;
            const float ox = box_offset_at(pp[u].x, bx, ag);
            const float oy = box_offset_at(pp[u].y, by, ag);
            float wx[K], wy[K], dx[K], dy[K];
            lagrange<K>(ox * inv_h, wx);
            lagrange<K>(oy * inv_h, wy);
#pragma unroll
            for (int l = 0; l < K; ++l) {
                dx[l] = (ox - ((float)l + 0.5f) * ag.hk) * inv_h;
                dy[l] = (oy - ((float)l + 0.5f) * ag.hk) * inv_h;
                wy[l] *= rr[u];
            }
#pragma unroll
            for (int ly = 0; ly < K; ++ly)
#pragma unroll
                for (int lx = 0; lx < K; ++lx) {
                    const float w = wx[lx] * wy[ly];
                    acc[0][ly][lx] += spread_q(w);
                    acc[1][ly][lx] += spread_q(w * dx[lx]);
                    acc[2][ly][lx] += spread_q(w * dy[ly]);
                }
        }
    }
#pragma unroll
    for (int o = 1; o < L; o <<= 1)
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int ly = 0; ly < K; ++ly)
#pragma unroll
                for (int lx = 0; lx < K; ++lx) acc[c][ly][lx] += __shfl_xor_sync(gmask, acc[c][ly][lx], o);
    // every lane holds the totals; lane g stores the entries v = g, g + L, ...
    const float hs = ag.h_hi * ag.q_inv;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int ly = 0; ly < K; ++ly)
#pragma unroll
            for (int lx = 0; lx < K; ++lx) {
                if (((c * K + ly) * K + lx) % L != g) continue;
                const size_t q = (size_t)(by * K + ly) * Gs + (bx * K + lx);
                gin[c * plane + q] = ll2f_rn(acc[c][ly][lx]) * (c == 0 ? ag.q_inv : hs);
            }
}

// Back-projection (Sec. 3.4 step 3) at position p from the grid (A, O^x, O^y, 0):
// frep = sum_q w_q [ (p - y_q) A_q + O_q ], the well-conditioned Eq. (Fr1)/(Fr2).
template <int K>
__device__ __forceinline__ float2 gather_frep(float2 p, const AxisGeom& ag, const float4* __restrict__ gout, int Gs) {
    float ox, oy;
    const int bx = box_offset(p.x, ag, &ox);
    const int by = box_offset(p.y, ag, &oy);
    const float inv_h = 1.0f / ag.h_hi;
    float wx[K], wy[K], dx[K], dy[K];
    lagrange<K>(ox * inv_h, wx);
    lagrange<K>(oy * inv_h, wy);
#pragma unroll
    for (int l = 0; l < K; ++l) {
        dx[l] = ox - ((float)l + 0.5f) * ag.hk;
        dy[l] = oy - ((float)l + 0.5f) * ag.hk;
    }
    float frx = 0.0f, fry = 0.0f;
#pragma unroll
    for (int ly = 0; ly < K; ++ly) {
        const float4* row = gout + (size_t)(by * K + ly) * Gs + bx * K;
#pragma unroll
        for (int lx = 0; lx < K; ++lx) {
            const float4 v = __ldg(row + lx);  // (A, O^x, O^y, 0)
            const float w = wx[lx] * wy[ly];
            frx = fmaf(w, fmaf(dx[lx], v.x, v.y), frx);
            fry = fmaf(w, fmaf(dy[ly], v.x, v.z), fry);
        }
    }
    return make_float2(frx, fry);
}

}  // namespace tfdp
