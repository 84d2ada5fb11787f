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
// 16-bit link codes of the odd-step slots: cells per tile of one column
// base, and the two reserved codes (own slot; read the int32 slot instead).
constexpr int32_t CODE_TILE = 128;
constexpr uint32_t CODE_WALL = 0xFFFF, CODE_ESCAPE = 0xFFFE;

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
// raw()/pack(): stored value <-> float in stored (scaled) units; ld()/st()
// also remove / apply the storage scale 2^s.
template <int ST> struct Store;
template <> struct Store<ST_F32> {
    using T = float;
    static constexpr bool scaled = false;
    static __device__ __forceinline__ float raw(T v) { return v; }
    static __device__ __forceinline__ T pack(float g) { return g; }
    static __device__ __forceinline__ float ld(T v, float) { return v; }
    static __device__ __forceinline__ T st(float g, float) { return g; }
};
template <> struct Store<ST_F16> {
    using T = __half;
    static constexpr bool scaled = true;
    static __device__ __forceinline__ float raw(T v) { return __half2float(v); }
    static __device__ __forceinline__ T pack(float g) { return __float2half_rn(g); }
    static __device__ __forceinline__ float ld(T v, float inv_scale) { return __half2float(v) * inv_scale; }
    static __device__ __forceinline__ T st(float g, float scale) { return __float2half_rn(g * scale); }
};
template <> struct Store<ST_BF16> {
    using T = __nv_bfloat16;
    static constexpr bool scaled = true;
    static __device__ __forceinline__ float raw(T v) { return __bfloat162float(v); }
    static __device__ __forceinline__ T pack(float g) { return __float2bfloat16_rn(g); }
    static __device__ __forceinline__ float ld(T v, float inv_scale) { return __bfloat162float(v) * inv_scale; }
    static __device__ __forceinline__ T st(float g, float scale) { return __float2bfloat16_rn(g * scale); }
};

// ------------------------------------------------------------- parameters
constexpr int MAX_PAIRS = 13;   // (27 - 1) / 2

struct CollideParams {
    float omega_p;      // omega+ (= 1/tau, Eq. 7)
    float omega_m;      // omega- (TRT); equals omega_p for SRT
    float fx, fy, fz;   // body-force density
    float scale;        // sigma = 2^s  (storage scale; 1 for FP32)
    float inv_scale;    // 2^-s
    float kp;           // 1 - omega+/2
    // per direction pair m (direction i = 2m+1 and its inverse i+1), in
    // stored units: the force terms of the TRT collision that depend on the
    // direction only (uniform body force):
    //   alpha_m = sigma (1 - omega+/2) 9 w_i (c_i . F)
    //   kappa_m = sigma (1 - omega-/2) 3 w_i (c_i . F)
    float alpha[MAX_PAIRS];
    float kappa[MAX_PAIRS];
    // MRT (D3Q19): relaxation rate of each moment of the basis below
    // (conserved moments unused)
    float mrt[19];
    float pad;          // keeps the size a multiple of 8 bytes (zero)
};

// Boundary link of cell k, direction i (the pull neighbour x_k - c_i is an
// inlet or outlet voxel).  When the cell's post-collision value of direction
// inverse(i) is stored into the link's slot i*S + k, it is mapped (shifted,
// unscaled units, u = the cell's velocity at that collision):
//   value -> s * value + a + q2 (4.5 (c_i . u)^2 - 1.5 u . u)
//   velocity inlet (moving wall):  s =  1, a = 6 w_i (c_i . u_w),      q2 = 0
//   pressure outlet (anti-BB):     s = -1, a = 2 w_i (rho_out - 1),    q2 = 2 w_i rho_out
struct LinkMap {
    float s, a, q2;
    float cx, cy, cz;   // c_i
};

__device__ __forceinline__ float apply_link(const LinkMap &m, float v, float ux, float uy, float uz, float scale) {
    const float cu = m.cx * ux + m.cy * uy + m.cz * uz;
    const float uu = ux * ux + uy * uy + uz * uz;
    return m.s * v + scale * (m.a + m.q2 * (4.5f * cu * cu - 1.5f * uu));
}

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

template <class V>
struct VelT {
    V x, y, z;
};
using Vel = VelT<float>;

// Two cells' values in the two FP32 lanes of one register pair.  The paired
// FP32 instructions of sm_100-class GPUs round each lane exactly as the
// scalar instruction does (IEEE round-to-nearest, no flush), so a collision
// evaluated on pairs gives the same bits per cell as the scalar one with
// half the FP instructions.  The pair operations are written as PTX with an
// explicit .rn rounding mode.  On its own that does not stop the assembler
// from fusing a paired multiply and a following paired add (measured: it
// does), while the scalar code is compiled without contraction.  So where
// a product feeds one add alone, the collision below writes the fma itself
// (the rest population's source term); the products that feed additions
// otherwise (the velocity components in c.u) have several uses each, and
// the paired kernels are tested bit for bit against the scalar ones.
struct F2 {
    float2 v;
};
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
    F2 r;
    asm("{\n\t.reg .b64 a, b, r;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "add.rn.f32x2 r, a, b;\n\tmov.b64 {%0, %1}, r;\n\t}"
        : "=f"(r.v.x), "=f"(r.v.y)
        : "f"(a.v.x), "f"(a.v.y), "f"(b.v.x), "f"(b.v.y));
    return r;
}
__device__ __forceinline__ F2 f2_sub(F2 a, F2 b) {
    F2 r;
    asm("{\n\t.reg .b64 a, b, r;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "sub.rn.f32x2 r, a, b;\n\tmov.b64 {%0, %1}, r;\n\t}"
        : "=f"(r.v.x), "=f"(r.v.y)
        : "f"(a.v.x), "f"(a.v.y), "f"(b.v.x), "f"(b.v.y));
    return r;
}
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
    F2 r;
    asm("{\n\t.reg .b64 a, b, r;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "mul.rn.f32x2 r, a, b;\n\tmov.b64 {%0, %1}, r;\n\t}"
        : "=f"(r.v.x), "=f"(r.v.y)
        : "f"(a.v.x), "f"(a.v.y), "f"(b.v.x), "f"(b.v.y));
    return r;
}
__device__ __forceinline__ F2 f2_fma(F2 a, F2 b, F2 c) {
    F2 r;
    asm("{\n\t.reg .b64 a, b, c, r;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "mov.b64 c, {%6, %7};\n\tfma.rn.f32x2 r, a, b, c;\n\tmov.b64 {%0, %1}, r;\n\t}"
        : "=f"(r.v.x), "=f"(r.v.y)
        : "f"(a.v.x), "f"(a.v.y), "f"(b.v.x), "f"(b.v.y), "f"(c.v.x), "f"(c.v.y));
    return r;
}
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return f2_add(a, b); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return f2_sub(a, b); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return f2_mul(a, b); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2{make_float2(-a.v.x, -a.v.y)}; }

// Scalar / pair forms used by the generic collision: broadcast of a per-cell
// constant, fused multiply-add (one rounding), reciprocal 1/x (IEEE division).
template <class V>
__device__ __forceinline__ V bc(float s);
template <>
__device__ __forceinline__ float bc<float>(float s) { return s; }
template <>
__device__ __forceinline__ F2 bc<F2>(float s) { return F2{make_float2(s, s)}; }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ F2 vfma(F2 a, F2 b, F2 c) { return f2_fma(a, b, c); }
__device__ __forceinline__ float vrcp(float x) { return 1.0f / x; }
__device__ __forceinline__ F2 vrcp(F2 x) { return F2{make_float2(1.0f / x.v.x, 1.0f / x.v.y)}; }

// Collision in place (Eq. 3) on shifted populations held in stored units
// (g * sigma; sigma = 1 for FP32).  TRT on each pair (i, inverse(i)) with
// s = g_i + g_inv and d = g_i - g_inv: the even part s/2 relaxes towards
//   g^eq+ = w [drho + rho (4.5 cu^2 - 1.5 u.u)]    with rate omega+,
// the odd part d/2 towards
//   g^eq- = 3 w rho cu                              with rate omega-
// (Eq. 6 in shifted form), plus the Guo source S = w[3(c - u) + 9 (c.u) c].F
// split into its even part w (9 cu cF - 3 u.F) and odd part 3 w cF, each
// weighted by (1 - omega/2) of its rate.  SRT (Eq. 5) is omega- = omega+.
// Moments: rho = 1 + drho, drho = sum g, j = sum c g, u = (j + F/2) / rho.
//
// Written per pair as  g_i' = A + B,  g_inv' = A - B  with
//   A = (1 - omega+)/2 s + omega+ g^eq+ + (1 - omega+/2) S+
//   B = (1 - omega-)/2 d + omega- g^eq- + (1 - omega-/2) S-
// and the terms that depend only on the weight class folded per cell.  Each
// fma is one rounding; compiled without FMA contraction the sequence of
// roundings is fixed, so every kernel gives the same bits for a cell.
// V = float: one cell; V = F2: two cells, the same operations lane-wise.
// Pair sums s_m = g_i + g_inv, d_m = g_i - g_inv (i = 2m + 1), the density
// deviation drho, rho and the Guo velocity u = (j + F/2) / rho of shifted
// populations in stored units, in the order of roundings of the TRT
// collision (which calls it), so that a kernel that needs only u gets the
// collision's bits.
template <int Q, bool SCALED, class V>
__device__ __forceinline__ void pair_moments(const V (&g)[Q], V (&s)[(Q - 1) / 2], V (&d)[(Q - 1) / 2],
                                             const CollideParams &p, V &drho, V &rho, VelT<V> &u) {
    constexpr int NP = (Q - 1) / 2;
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        s[m] = g[2 * m + 1] + g[2 * m + 2];
        d[m] = g[2 * m + 1] - g[2 * m + 2];
    }
    V jx = bc<V>(0.f), jy = bc<V>(0.f), jz = bc<V>(0.f);
    drho = g[0];
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        drho = drho + s[m];
        const int i = 2 * m + 1;
        if (cx(i) > 0) jx = jx + d[m];
        if (cx(i) < 0) jx = jx - d[m];
        if (cy(i) > 0) jy = jy + d[m];
        if (cy(i) < 0) jy = jy - d[m];
        if (cz(i) > 0) jz = jz + d[m];
        if (cz(i) < 0) jz = jz - d[m];
    }
    if (SCALED) {
        const V is = bc<V>(p.inv_scale);
        drho = drho * is;
        jx = jx * is;
        jy = jy * is;
        jz = jz * is;
    }
    rho = bc<V>(1.0f) + drho;
    const V ir = vrcp(rho);
    u.x = vfma(bc<V>(0.5f), bc<V>(p.fx), jx) * ir;
    u.y = vfma(bc<V>(0.5f), bc<V>(p.fy), jy) * ir;
    u.z = vfma(bc<V>(0.5f), bc<V>(p.fz), jz) * ir;
}

// The Guo velocity of one cell with the TRT collision's bits.
template <int Q, bool SCALED>
__device__ __forceinline__ Vel guo_velocity(const float (&g)[Q], const CollideParams &p) {
    float s[(Q - 1) / 2], d[(Q - 1) / 2], drho, rho;
    Vel u;
    pair_moments<Q, SCALED, float>(g, s, d, p, drho, rho, u);
    return u;
}

template <int Q, bool SCALED, class V>
__device__ __forceinline__ VelT<V> collide_v(V (&g)[Q], const CollideParams &p) {
    constexpr int NP = (Q - 1) / 2;
    V s[NP], d[NP], drho, rho;
    VelT<V> u0;
    pair_moments<Q, SCALED, V>(g, s, d, p, drho, rho, u0);
    const V ux = u0.x, uy = u0.y, uz = u0.z;
    const V usq = vfma(uz, uz, vfma(uy, uy, ux * ux));
    const V uF = vfma(uz, bc<V>(p.fz), vfma(uy, bc<V>(p.fy), ux * bc<V>(p.fx)));
    const V E = vfma(bc<V>(-1.5f) * rho, usq, drho);            // drho - 1.5 rho u.u
    const V sr = SCALED ? bc<V>(p.scale) * rho : rho;          // sigma rho
    const V sE = SCALED ? bc<V>(p.scale) * E : E;              // sigma (drho - 1.5 rho u.u)
    const V skF = SCALED ? bc<V>(p.scale) * (bc<V>(p.kp * 3.0f) * uF)
                         : bc<V>(p.kp * 3.0f) * uF;            // sigma kp 3 u.F
    const float wp = p.omega_p, wm = p.omega_m;
    const float hp = 0.5f - 0.5f * wp, hm = 0.5f - 0.5f * wm;   // (1 - omega)/2
    const V pE = bc<V>(wp) * sE, pR = bc<V>(wp) * sr, mR = bc<V>(wm) * sr;
    // rest population: even only.  Its source term enters through one fma:
    // the paired form would otherwise be open to a multiply-add contraction
    // that the scalar form is compiled without, and both must round alike.
    {
        constexpr float w = wgt<Q>(0);
        g[0] = vfma(bc<V>(-w), skF, vfma(bc<V>(w), pE, vfma(bc<V>(-wp), g[0], g[0])));
    }
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        const int i = 2 * m + 1;
        const float w = wgt<Q>(i);
        V cu = bc<V>(0.f);
        if (cx(i) > 0) cu = cu + ux;
        if (cx(i) < 0) cu = cu - ux;
        if (cy(i) > 0) cu = cu + uy;
        if (cy(i) < 0) cu = cu - uy;
        if (cz(i) > 0) cu = cu + uz;
        if (cz(i) < 0) cu = cu - uz;
        // class constants (folded by the compiler per weight class)
        const V Ap = vfma(bc<V>(w), pE, -(bc<V>(w) * skF));     // omega+ w sE - w skF
        const V Bp = bc<V>(4.5f * w) * pR;                       // omega+ 4.5 w sigma rho
        const V Cm = bc<V>(3.0f * w) * mR;                       // omega- 3 w sigma rho
        const V A = vfma(bc<V>(hp), s[m], vfma(Bp, cu * cu, vfma(bc<V>(p.alpha[m]), cu, Ap)));
        const V B = vfma(bc<V>(hm), d[m], vfma(Cm, cu, bc<V>(p.kappa[m])));
        g[i] = A + B;
        g[i + 1] = A - B;
    }
    return VelT<V>{ux, uy, uz};
}

template <int Q, bool SCALED>
__device__ __forceinline__ Vel collide(float (&g)[Q], const CollideParams &p) {
    return collide_v<Q, SCALED, float>(g, p);
}

// ---------------------------------------------------------------- MRT
// D3Q19 moment basis of d'Humieres, Ginzburg, Krafczyk, Lallemand, Luo
// (2002), row a at velocity c = (x, y, z), |c|^2 = n:
//   0 rho 1            1 e 19n - 30         2 eps (21n^2 - 53n + 24)/2
//   3 jx x   4 qx (5n - 9)x   5 jy y   6 qy (5n - 9)y   7 jz z   8 qz (5n - 9)z
//   9 3pxx 3x^2 - n    10 3pixx (3n - 5)(3x^2 - n)
//   11 pww y^2 - z^2   12 piww (3n - 5)(y^2 - z^2)
//   13 pxy xy  14 pyz yz  15 pxz xz
//   16 mx x(y^2 - z^2)  17 my y(z^2 - x^2)  18 mz z(x^2 - y^2)
// All entries are integers; the rows are orthogonal, so M^-1 = M^T / |row|^2.
__host__ __device__ constexpr int mrt_m(int a, int i) {
    const int x = cx(i), y = cy(i), z = cz(i), n = x * x + y * y + z * z;
    switch (a) {
        case 0: return 1;
        case 1: return 19 * n - 30;
        case 2: return (21 * n * n - 53 * n + 24) / 2;
        case 3: return x;
        case 4: return (5 * n - 9) * x;
        case 5: return y;
        case 6: return (5 * n - 9) * y;
        case 7: return z;
        case 8: return (5 * n - 9) * z;
        case 9: return 3 * x * x - n;
        case 10: return (3 * n - 5) * (3 * x * x - n);
        case 11: return y * y - z * z;
        case 12: return (3 * n - 5) * (y * y - z * z);
        case 13: return x * y;
        case 14: return y * z;
        case 15: return x * z;
        case 16: return x * (y * y - z * z);
        case 17: return y * (z * z - x * x);
        default: return z * (x * x - y * y);
    }
}

__host__ __device__ constexpr int mrt_norm(int a) {
    int s = 0;
    for (int i = 0; i < 19; ++i) s += mrt_m(a, i) * mrt_m(a, i);
    return s;
}

__host__ __device__ constexpr bool mrt_odd_row(int a) {
    return (a >= 3 && a <= 8) || a >= 16;     // j, q, m: odd in c
}

// MRT collision in stored (shifted, scaled) units: with the non-equilibrium
// part x_i = g_i - sigma (f_i^eq - w_i) and the Guo source sigma S_i,
//   dm_a = -s_a (M x)_a + (1 - s_a/2) (M sigma S)_a   (non-conserved a)
//   g*_i = g_i + sum_a M_ai dm_a / |row a|^2 + sigma (c_i . F) / 10
// (the last term is the momentum rows' kick, |row jx|^2 = 10; the density
// row changes nothing).  Every row is even or odd under c -> -c, so both
// transforms run on the sums and differences of the 9 inverse pairs: an even
// row sees g_0 and the pair sums, an odd row the pair differences, and the
// back transform yields both members of a pair from one even and one odd sum.
template <bool SCALED, class V>
__device__ __forceinline__ VelT<V> collide_mrt_v(V (&g)[19], const CollideParams &p) {
    constexpr int NP = 9;
    V sg[NP], dg[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        sg[m] = g[2 * m + 1] + g[2 * m + 2];
        dg[m] = g[2 * m + 1] - g[2 * m + 2];
    }
    V drho = g[0], jx = bc<V>(0.f), jy = bc<V>(0.f), jz = bc<V>(0.f);
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        drho = drho + sg[m];
        const int i = 2 * m + 1;
        if (cx(i) > 0) jx = jx + dg[m];
        if (cx(i) < 0) jx = jx - dg[m];
        if (cy(i) > 0) jy = jy + dg[m];
        if (cy(i) < 0) jy = jy - dg[m];
        if (cz(i) > 0) jz = jz + dg[m];
        if (cz(i) < 0) jz = jz - dg[m];
    }
    if (SCALED) {
        const V is = bc<V>(p.inv_scale);
        drho = drho * is;
        jx = jx * is;
        jy = jy * is;
        jz = jz * is;
    }
    const V rho = bc<V>(1.0f) + drho;
    const V ir = vrcp(rho);
    const V ux = vfma(bc<V>(0.5f), bc<V>(p.fx), jx) * ir;
    const V uy = vfma(bc<V>(0.5f), bc<V>(p.fy), jy) * ir;
    const V uz = vfma(bc<V>(0.5f), bc<V>(p.fz), jz) * ir;
    const V usq = vfma(uz, uz, vfma(uy, uy, ux * ux));
    const V uF = vfma(uz, bc<V>(p.fz), vfma(uy, bc<V>(p.fy), ux * bc<V>(p.fx)));
    const float sig = SCALED ? p.scale : 1.0f;
    // non-equilibrium and source, as pair sums (even) and differences (odd):
    //   geq_i +- geq_ib = 2 w (drho + rho (4.5 cu^2 - 1.5 u.u)),  2 w 3 rho cu
    //   S_i +- S_ib     = 2 w (9 cu cF - 3 u.F),                   2 w 3 cF
    const V e0 = vfma(bc<V>(-1.5f) * rho, usq, drho);           // drho - 1.5 rho u.u
    const V x0 = vfma(bc<V>(-sig * wgt<19>(0)), e0, g[0]);
    const V s0 = bc<V>(-3.0f * sig * wgt<19>(0)) * uF;
    V xs[NP], xd[NP], ss[NP];
    float sd[NP];                                                // per-cell constant
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        const int i = 2 * m + 1;
        const float w2 = 2.0f * wgt<19>(i) * sig;
        V cu = bc<V>(0.f);
        float cF = 0.f;
        if (cx(i) > 0) { cu = cu + ux; cF += p.fx; }
        if (cx(i) < 0) { cu = cu - ux; cF -= p.fx; }
        if (cy(i) > 0) { cu = cu + uy; cF += p.fy; }
        if (cy(i) < 0) { cu = cu - uy; cF -= p.fy; }
        if (cz(i) > 0) { cu = cu + uz; cF += p.fz; }
        if (cz(i) < 0) { cu = cu - uz; cF -= p.fz; }
        xs[m] = vfma(bc<V>(-w2), vfma(bc<V>(4.5f) * rho * cu, cu, e0), sg[m]);
        xd[m] = vfma(bc<V>(-w2), bc<V>(3.0f) * rho * cu, dg[m]);
        ss[m] = bc<V>(w2) * vfma(bc<V>(9.0f) * cu, bc<V>(cF), bc<V>(-3.0f) * uF);
        sd[m] = w2 * 3.0f * cF;
    }
    V dm[19];
#pragma unroll
    for (int a = 0; a < 19; ++a) {
        dm[a] = bc<V>(0.f);
        if (a == 0 || a == 3 || a == 5 || a == 7) continue;       // conserved
        V mx = bc<V>(0.f), ms = bc<V>(0.f);
        if (!mrt_odd_row(a)) {
            mx = bc<V>((float)mrt_m(a, 0)) * x0;
            ms = bc<V>((float)mrt_m(a, 0)) * s0;
        }
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            const int i = 2 * m + 1;
            if (mrt_m(a, i) == 0) continue;
            if (mrt_odd_row(a)) {
                mx = vfma(bc<V>((float)mrt_m(a, i)), xd[m], mx);
                ms = vfma(bc<V>((float)mrt_m(a, i)), bc<V>(sd[m]), ms);
            } else {
                mx = vfma(bc<V>((float)mrt_m(a, i)), xs[m], mx);
                ms = vfma(bc<V>((float)mrt_m(a, i)), ss[m], ms);
            }
        }
        const float sa = p.mrt[a];
        dm[a] = vfma(bc<V>(-sa), mx, bc<V>(1.0f - 0.5f * sa) * ms) * bc<V>(1.0f / (float)mrt_norm(a));
    }
    {
        V v = g[0];
#pragma unroll
        for (int a = 0; a < 19; ++a)
            if (!mrt_odd_row(a) && a != 0 && mrt_m(a, 0) != 0) v = vfma(bc<V>((float)mrt_m(a, 0)), dm[a], v);
        g[0] = v;
    }
    const float kx = sig * p.fx * 0.1f, ky = sig * p.fy * 0.1f, kz = sig * p.fz * 0.1f;
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        const int i = 2 * m + 1;
        V E = bc<V>(0.f), O = bc<V>(0.f);
        if (cx(i) > 0) O = O + bc<V>(kx);
        if (cx(i) < 0) O = O - bc<V>(kx);
        if (cy(i) > 0) O = O + bc<V>(ky);
        if (cy(i) < 0) O = O - bc<V>(ky);
        if (cz(i) > 0) O = O + bc<V>(kz);
        if (cz(i) < 0) O = O - bc<V>(kz);
#pragma unroll
        for (int a = 0; a < 19; ++a) {
            if (a == 0 || a == 3 || a == 5 || a == 7 || mrt_m(a, i) == 0) continue;
            if (mrt_odd_row(a)) O = vfma(bc<V>((float)mrt_m(a, i)), dm[a], O);
            else E = vfma(bc<V>((float)mrt_m(a, i)), dm[a], E);
        }
        const V gi = g[i], gb = g[i + 1];
        g[i] = gi + E + O;
        g[i + 1] = gb + E - O;
    }
    return VelT<V>{ux, uy, uz};
}

template <bool SCALED>
__device__ __forceinline__ Vel collide_mrt(float (&g)[19], const CollideParams &p) {
    return collide_mrt_v<SCALED, float>(g, p);
}

enum { OP_TRT = 0, OP_MRT = 1 };

}  // namespace slbm

#include "central.cuh"

namespace slbm {

// The collision of operator OP (SRT is TRT with equal rates; OP_CM and
// OP_CUM are the D3Q27 central-moment and cumulant collisions).
template <int Q, bool SCALED, int OP>
__device__ __forceinline__ Vel collide_op(float (&g)[Q], const CollideParams &p) {
    if constexpr (OP == OP_MRT) {
        static_assert(Q == 19, "MRT is defined for D3Q19");
        return collide_mrt<SCALED>(g, p);
    } else if constexpr (OP == OP_CM || OP == OP_CUM) {
        static_assert(Q == 27, "the central-moment operators are defined for D3Q27");
        return collide_central<SCALED, OP>(g, p);
    } else {
        return collide<Q, SCALED>(g, p);
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

// Row flip between i and inverse(i) of a slot e >= 0 in one of those two rows
// (Sec. 5.1).  A pull entry P(i,k) lies in row i (fluid neighbour n:
// i*S + n) or in row inverse(i) (wall: inverse(i)*S + k); the AA odd step
// reads f_i(x_k) from the same column with the row flipped.  The flip is an
// involution, so it also maps the odd-step slot back to the pull entry.
__device__ __forceinline__ int32_t flip_row(int32_t e, int i, int32_t S) {
    if (i & 1) return e < (i + 1) * S ? e + S : e - S;   // inverse = i+1
    return e >= i * S ? e - S : e + S;                    // inverse = i-1
}

}  // namespace slbm
