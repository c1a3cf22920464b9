// Definitions shared by the FP64 (far.cu) and FP32 (far32.cu) far-field
// kernels: block-class panel layout, accumulator slots, the per-chunk
// element-pair setup and the scatter of local 3x3 matrices into the FP64
// vertex-pair lag windows.
#pragma once
#include "tdbem_internal.h"

namespace tdbem {

__host__ __device__ constexpr int cls_P(int c) {
    return c == C1 ? 3 : c == C2 ? 4 : c == C3 ? 3 : c == SN0 ? 2 : 1;
}
__host__ __device__ constexpr int cls_panel0(int c) {
    return c == C1 ? 0 : c == C2 ? 3 : c == C3 ? 7 : c == S00 ? 10 : c == S01 ? 11 : c == SN0 ? 12 : c == SNN ? 14 : 15;
}
// accumulator slots of class c: lag classes cover cell in [-OFF, OFF] and
// their P panels; specials keep only lag 0
template <int OFF>
__host__ __device__ constexpr int cls_K(int c) { return c < NLAG ? 2 * OFF + cls_P(c) : 1; }
template <int OFF>
__host__ __device__ constexpr int slot0(int c) {
    int s = 0;
    for (int x = 0; x < c; ++x) s += cls_K<OFF>(x);
    return s;
}
template <int OFF>
__host__ __device__ constexpr int total_slots() { return slot0<OFF>(NCLASS); }

constexpr int FAR_WARPS = 7;
constexpr int KW_MAX = 16;  // largest vertex-pair lag window the scatter handles
constexpr int FAR_THREADS = FAR_WARPS * 32;

template <typename R>
struct FarSetup {
    R scale[32];
    R nn[32];
    int base[32];
    int valid[32];
    float f0[32];
    float D[32][3];
    float R0[32];
};

// 7-point rule weight and barycentric in the working precision
template <typename R>
__device__ __forceinline__ R rule_w(const FarArgs &A, int k) {
    if constexpr (sizeof(R) == 8) return A.rule_w64[k];
    else return A.rule_w[k];
}
template <typename R>
__device__ __forceinline__ R rule_l(const FarArgs &A, int k) {
    if constexpr (sizeof(R) == 8) return A.rule_l64[k];
    else return A.rule_l[k];
}


// Sum the local 3x3 matrices of the triangles of this chunk that share a
// trial vertex (host-built per-chunk plan) and add them, read-modify-write
// without atomics, into the FP64 lag windows of rows F[tau][a]. Lb holds
// [32 sigma][NS slots][9] values; su the element-pair setup of the chunk.
// Lb element types: float or double values, or FP32 pairs (hi, lo) summed
// with an error-free two-sum
struct alignas(8) FF {
    float h, l;
};
__device__ __forceinline__ void lb_add(float &s, float v) { s += v; }
__device__ __forceinline__ void lb_add(double &s, double v) { s += v; }
__device__ __forceinline__ void lb_add(FF &s, FF v) {
    const float t = s.h + v.h;
    const float bb = t - s.h;
    const float e = (s.h - (t - bb)) + (v.h - bb);
    s.l = (s.l + v.l) + e;
    s.h = t;
}
__device__ __forceinline__ double lb_value(float s) { return (double)s; }
__device__ __forceinline__ double lb_value(double s) { return s; }
__device__ __forceinline__ double lb_value(FF s) { return (double)s.h + (double)s.l; }

template <typename R, int OFF, int NTHREADS, typename Setup, bool WITH_SPEC = true>
__device__ __forceinline__ void scatter_chunk(const FarArgs &A, int64_t ch, int32_t Ft0, int32_t Ft1, int32_t Ft2,
                                              const Setup &su, const R *Lb) {
    constexpr int NS = WITH_SPEC ? total_slots<OFF>() : slot0<OFF>(NLAG);
    constexpr int NCL = WITH_SPEC ? NCLASS : NLAG;
    const Geo &g = A.g;
    const int64_t M = g.M, MM = M * M;
    const int v0 = A.chunk_vptr[ch], v1 = A.chunk_vptr[ch + 1];
    const int nv = v1 - v0;
    for (int it = threadIdx.x; it < nv * 3 * NCL; it += NTHREADS) {
        const int v = it / (3 * NCL), rem = it % (3 * NCL);
        const int a = rem / NCL, c = rem % NCL;
        const int64_t j = A.chunk_vert[v0 + v];
        const int64_t l = a == 0 ? Ft0 : (a == 1 ? Ft1 : Ft2);
        const int s0 = A.chunk_sptr[v0 + v], s1 = A.chunk_sptr[v0 + v + 1];
        if (c < NLAG) {
            const int P = cls_P(c), K = 2 * OFF + P;
            const int rho = A.lt.rho[c];
            const int so = c == C1 ? slot0<OFF>(C1) : c == C2 ? slot0<OFF>(C2) : slot0<OFF>(C3);
            int dmn = 1 << 30, dmx = -(1 << 30);
            for (int x = s0; x < s1; ++x) {
                const int sl = A.chunk_src[x] / 3;
                if (!su.valid[sl]) continue;
                const int dv = su.base[sl] - rho - (P - 1) - OFF;
                dmn = min(dmn, dv);
                dmx = max(dmx, dv + K - 1);
            }
            const int wlo = A.dlo[c * MM + l * M + j], whi = A.dhi[c * MM + l * M + j];
            dmn = max(dmn, wlo);
            dmx = min(min(dmx, whi), wlo + A.KW - 1);
            if (dmn > dmx) continue;
            // whole window at once: independent loads, sums from shared
            // memory, then the stores (no load waits behind a store)
            double *dst = A.dense + (c * MM + l * M + j) * A.KW;
            double cur[KW_MAX];
#pragma unroll
            for (int k = 0; k < KW_MAX; ++k) {
                const int d = wlo + k;
                cur[k] = (d >= dmn && d <= dmx) ? dst[k] : 0.0;
            }
#pragma unroll
            for (int k = 0; k < KW_MAX; ++k) {
                const int d = wlo + k;
                if (d < dmn || d > dmx) continue;
                R sum{};
                for (int x = s0; x < s1; ++x) {
                    const int src = A.chunk_src[x], sl = src / 3, b = src % 3;
                    if (!su.valid[sl]) continue;
                    const int slot = d - (su.base[sl] - rho - (P - 1) - OFF);
                    if (slot < 0 || slot >= K) continue;
                    lb_add(sum, Lb[((size_t)sl * NS + so + slot) * 9 + 3 * a + b]);
                }
                dst[k] = cur[k] + lb_value(sum);
            }
        } else {
            const int sbit = c - NLAG;
            if (!((A.smask[l * M + j] >> sbit) & 1u)) continue;
            const int so = slot0<OFF>(C3) + cls_K<OFF>(C3) + sbit;
            R sum{};
            for (int x = s0; x < s1; ++x) {
                const int src = A.chunk_src[x], sl = src / 3, b = src % 3;
                if (!su.valid[sl]) continue;
                lb_add(sum, Lb[((size_t)sl * NS + so) * 9 + 3 * a + b]);
            }
            double *dst = A.dense_spec + (sbit * MM + l * M + j);
            *dst += lb_value(sum);
        }
    }
}

}  // namespace tdbem
