// common.cuh -- lattice constants, storage traits and the per-cell collision
// shared by every kernel of the library.
//
// Populations are stored SHIFTED (the paper's "zero-centred storage", Sec. 4):
// g_i = f_i - w_i, so the rest state is all zeros and rho - 1 = sum g_i is
// summed without cancellation.  All arithmetic is FP32; the FP16/BF16 storage
// forms hold g_i * 2^s (s a per-domain exponent) and convert on load/store.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace slbm {

enum { ST_F32 = 0, ST_F16 = 1, ST_BF16 = 2 };
enum { FLAG_FLUID = 0, FLAG_WALL = 1, FLAG_INLET = 2, FLAG_OUTLET = 3 };

// ---------------------------------------------------------------- lattice
// Direction i and its inverse are adjacent: inverse(i) = i+1 (i odd),
// i-1 (i even, i > 0).  D3Q19 is the first 19 directions of D3Q27.
__host__ __device__ __forceinline__ constexpr int cx(int i) {
    constexpr int t[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1,
                           -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, -1, 1};
    return t[i];
}
__host__ __device__ __forceinline__ constexpr int cy(int i) {
    constexpr int t[27] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0,
                           0, 1, -1, 1, -1, 1, -1, 1, -1, -1, 1, 1, -1};
    return t[i];
}
__host__ __device__ __forceinline__ constexpr int cz(int i) {
    constexpr int t[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1,
                           1, 1, -1, -1, 1, 1, -1, -1, 1, 1, -1, 1, -1};
    return t[i];
}
__host__ __device__ __forceinline__ constexpr int inv(int i) {
    return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
}
// Lattice weights from |c|^2 (D3Q19: 1/3, 1/18, 1/36; D3Q27: 8/27, 2/27,
// 1/54, 1/216).
template <int Q>
__host__ __device__ __forceinline__ constexpr float wgt(int i) {
    return Q == 19 ? (i == 0 ? 1.0f / 3.0f : (i < 7 ? 1.0f / 18.0f : 1.0f / 36.0f))
                   : (i == 0 ? 8.0f / 27.0f
                             : (i < 7 ? 2.0f / 27.0f : (i < 19 ? 1.0f / 54.0f : 1.0f / 216.0f)));
}

// --------------------------------------------------------------- storage
template <int ST> struct Store;
template <> struct Store<ST_F32> {
    using T = float;
    static __device__ __forceinline__ float ld(T v, float) { return v; }
    static __device__ __forceinline__ T st(float g, float) { return g; }
};
template <> struct Store<ST_F16> {
    using T = __half;
    static __device__ __forceinline__ float ld(T v, float inv_scale) { return __half2float(v) * inv_scale; }
    static __device__ __forceinline__ T st(float g, float scale) { return __float2half_rn(g * scale); }
};
template <> struct Store<ST_BF16> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float ld(T v, float inv_scale) { return __bfloat162float(v) * inv_scale; }
    static __device__ __forceinline__ T st(float g, float scale) { return __float2bfloat16_rn(g * scale); }
};

// ------------------------------------------------------------- parameters
struct CollideParams {
    float omega_p;      // omega+ (= 1/tau, Eq. 7)
    float omega_m;      // omega- (TRT); equals omega_p for SRT
    float fx, fy, fz;   // body-force density
    float scale;        // 2^s  (storage scale; 1 for FP32)
    float inv_scale;    // 2^-s
};

// Boundary link map applied to a slot on both its read and its write in the
// odd step: value -> s * value + a (shifted, unscaled units).
//   velocity inlet (moving wall):  s =  1, a = 6 w_i (c_i . u_w)
//   pressure outlet (anti-BB):     s = -1, a = 2 w_i (rho_out - 1)
struct LinkMap {
    float s, a;
};

// Moments of shifted populations: drho = sum g, j = sum c g.
template <int Q>
__device__ __forceinline__ void moments(const float (&g)[Q], float &drho, float &jx, float &jy,
                                        float &jz) {
    drho = 0.f;
    jx = 0.f;
    jy = 0.f;
    jz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += g[i];
        if (cx(i) > 0) jx += g[i];
        if (cx(i) < 0) jx -= g[i];
        if (cy(i) > 0) jy += g[i];
        if (cy(i) < 0) jy -= g[i];
        if (cz(i) > 0) jz += g[i];
        if (cz(i) < 0) jz -= g[i];
    }
}

// Collision in place on shifted populations (Eq. 3).  TRT on each pair
// (i, inverse(i)): the even part relaxes with omega+, the odd part with
// omega-; SRT (Eq. 5) is the case omega- = omega+.  Equilibrium (Eq. 6) in
// shifted form  g_i^eq = w_i [drho + rho (3 cu + 4.5 cu^2 - 1.5 u.u)], and the
// Guo source S_i = w_i [3 (c_i - u) + 9 (c_i.u) c_i] . F split into its even
// part w_i (9 cu cF - 3 u.F) and odd part 3 w_i cF, each weighted by
// (1 - omega/2) of its rate.  u = (j + F/2) / rho.
template <int Q>
__device__ __forceinline__ void collide(float (&g)[Q], const CollideParams &p) {
    float drho, jx, jy, jz;
    moments<Q>(g, drho, jx, jy, jz);
    const float rho = 1.0f + drho;
    const float ir = 1.0f / rho;
    const float ux = (jx + 0.5f * p.fx) * ir;
    const float uy = (jy + 0.5f * p.fy) * ir;
    const float uz = (jz + 0.5f * p.fz) * ir;
    const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
    const float uF3 = 3.0f * (ux * p.fx + uy * p.fy + uz * p.fz);
    const float kp = 1.0f - 0.5f * p.omega_p;
    const float km = 1.0f - 0.5f * p.omega_m;
    // rest population: even only
    {
        const float w = wgt<Q>(0);
        const float eq = w * (drho - rho * usq15);
        g[0] += -p.omega_p * (g[0] - eq) + kp * (-w * uF3);
    }
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const int b = i + 1;
        const float w = wgt<Q>(i);
        const float cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
        const float cF = cx(i) * p.fx + cy(i) * p.fy + cz(i) * p.fz;
        const float eqp = w * (drho + rho * (4.5f * cu * cu - usq15));
        const float eqm = w * rho * 3.0f * cu;
        const float sp = w * (9.0f * cu * cF - uF3);
        const float sm = 3.0f * w * cF;
        const float gp = 0.5f * (g[i] + g[b]);
        const float gm = 0.5f * (g[i] - g[b]);
        const float dp = -p.omega_p * (gp - eqp) + kp * sp;
        const float dm = -p.omega_m * (gm - eqm) + km * sm;
        g[i] += dp + dm;
        g[b] += dp - dm;
    }
}

// Shifted equilibrium of (rho, u) (Eq. 6 minus w_i).
template <int Q>
__device__ __forceinline__ void equilibrium_shifted(float rho, float ux, float uy, float uz,
                                                    float (&g)[Q]) {
    const float drho = rho - 1.0f;
    const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
        g[i] = wgt<Q>(i) * (drho + rho * (3.0f * cu + 4.5f * cu * cu - usq15));
    }
}

// AA odd-step slot of direction i for cell k from its pull entry e >= 0
// (Sec. 5.1): the entry lies in row i (fluid neighbour n: e = i*S + n) or in
// row inverse(i) (wall: e = inverse(i)*S + k).  The odd step reads f_i(x_k)
// from the same column with the row flipped: inverse(i)*S + n, resp. i*S + k.
__device__ __forceinline__ int32_t flip_row(int32_t e, int i, int32_t S) {
    if (i & 1) return e < (i + 1) * S ? e + S : e - S;   // inverse = i+1
    return e >= i * S ? e - S : e + S;                    // inverse = i-1
}

}  // namespace slbm
