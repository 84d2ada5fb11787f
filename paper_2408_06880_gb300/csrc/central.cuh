// central.cuh -- central-moment and cumulant collisions on D3Q27 (two of the
// operators the paper generates and benchmarks, Sec. 4 and Sec. 5.1), on
// shifted populations g = f - w in FP32.
//
// Central moments about the Guo velocity u, kappa_abc = sum_i f_i
// (c_ix - u_x)^a (c_iy - u_y)^b (c_iz - u_z)^c with a, b, c in {0, 1, 2}
// (index a + 3b + 9c), are formed and inverted axis by axis: along one axis
// the three populations of velocity -1, 0, +1 map to the moments of order 0,
// 1, 2 about u and back, so three passes over nine lines each do the full
// 27 x 27 change of basis.
//
// The collision works on deviations from the factorised equilibrium,
// Dk = kappa(f) - kappa_eq with kappa_eq = rho prod m(.), m = (1, 0, 1/3):
// the rest weights of D3Q27 factorise with the same one-dimensional moments
// (1, 0, 1/3) about 0, so kappa(f) = kappa(g) + prod (m + d) with the
// shifts d = (0, -u, u^2), and Dk = kappa(g) + B with
// B = [prod (m + d) - prod m] - (rho - 1) prod m evaluated without
// subtracting nearly equal numbers (see Bq below).  Relaxation (rates: omega+ on the shear
// moments, the bulk rate on the trace of the second ones, the higher rate on
// orders 3..6):
//   order 0: Dk = 0;   order 1: the first central moments become +F/2 (the
//   momentum gains F, the Guo velocity half-step);
//   order 2: trace * (1 - bulk), normal differences and off-diagonal
//   moments * (1 - omega+);
//   central moments (OP_CM): orders 3..6 * (1 - higher);
//   cumulants (OP_CUM, higher rate 1): every cumulant of order 3..6 becomes
//   0, so the post-collision central moments of orders 3 and 5 vanish and
//   those of orders 4 and 6 are the Gaussian (pairing) products of the
//   post-collision second ones -- e.g. kappa_220 = rho (m_200 m_020 + 2
//   m_110^2), kappa_222 = rho (m_200 m_020 m_002 + 2 m_200 m_011^2 + ... +
//   8 m_110 m_101 m_011), m = kappa / rho -- written in deviations.
// Then g* = inverse transform of (Dk* - B), B formed per moment where it is
// used.
#pragma once

namespace slbm {

enum { OP_CM = 2, OP_CUM = 3 };

// Direction of D3Q27 with velocity (x, y, z) in {-1, 0, 1}^3, by grid
// position (x+1) + 3(y+1) + 9(z+1).
__host__ __device__ __forceinline__ constexpr int dir_at(int pos) {
    constexpr int t[27] = {20, 16, 26, 12, 6, 13, 24, 17, 21,   // z = -1
                           8, 4, 9, 2, 0, 1, 10, 3, 7,          // z = 0
                           22, 18, 23, 14, 5, 11, 25, 15, 19};  // z = +1
    return t[pos];
}

// Axis pass of the forward map on the line (k[o], k[o+s], k[o+2s]) holding the
// values of velocity -1, 0, +1 along the axis: to moments 0, 1, 2 about v.
__device__ __forceinline__ void to_central(float &a, float &b, float &c, float v) {
    const float s0 = a + b + c, d = c - a, e = c + a;
    a = s0;
    b = fmaf(-v, s0, d);
    c = fmaf(v * v, s0, fmaf(-2.0f * v, d, e));
}

// Inverse axis pass: moments 0, 1, 2 about v to the values of -1, 0, +1.
__device__ __forceinline__ void from_central(float &k0, float &k1, float &k2, float v) {
    const float vv = v * v;
    const float m = 0.5f * (fmaf(vv - v, k0, fmaf(2.0f * v - 1.0f, k1, k2)));
    const float z = fmaf(1.0f - vv, k0, fmaf(-2.0f * v, k1, -k2));
    const float pl = 0.5f * (fmaf(vv + v, k0, fmaf(2.0f * v + 1.0f, k1, k2)));
    k0 = m;
    k1 = z;
    k2 = pl;
}

template <bool SCALED, int OP>
__device__ __forceinline__ Vel collide_central(float (&g)[27], const CollideParams &p) {
    static_assert(OP == OP_CM || OP == OP_CUM, "central-moment operators");
    if (SCALED) {
#pragma unroll
        for (int i = 0; i < 27; ++i) g[i] *= p.inv_scale;
    }
    float drho, jx, jy, jz;
    moments<27>(g, drho, jx, jy, jz);
    const float rho = 1.0f + drho;
    const float ir = 1.0f / rho;
    const float ux = fmaf(0.5f, p.fx, jx) * ir, uy = fmaf(0.5f, p.fy, jy) * ir, uz = fmaf(0.5f, p.fz, jz) * ir;
    float k[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) k[q] = g[dir_at(q)];
    // forward: x, y, z passes
#pragma unroll
    for (int l = 0; l < 9; ++l) to_central(k[3 * l], k[3 * l + 1], k[3 * l + 2], ux);
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        const int o = (l % 3) + 9 * (l / 3);
        to_central(k[o], k[o + 3], k[o + 6], uy);
    }
#pragma unroll
    for (int l = 0; l < 9; ++l) to_central(k[l], k[l + 9], k[l + 18], uz);
    // B of moment q = (a, b, c), formed where it is used (no array of B is
    // kept).  With an index 1, prod(m) = 0 and B = prod(m + d), a product of
    // the factors 1, -u, 1/3 + u^2.  Otherwise m + d = m (1 + delta) per axis,
    // delta = 0 (index 0) or 3 u^2 (index 2), and B = prod(m) (S - drho) with
    // S = prod(1 + delta) - 1 expanded axis by axis as S' = S + delta +
    // S delta, so that no O(1) terms cancel.
    const float ex2 = fmaf(ux, ux, 1.0f / 3.0f), ey2 = fmaf(uy, uy, 1.0f / 3.0f), ez2 = fmaf(uz, uz, 1.0f / 3.0f);
    const float dx3 = 3.0f * (ux * ux), dy3 = 3.0f * (uy * uy), dz3 = 3.0f * (uz * uz);
    auto Bq = [&](int q) {
        const int a = q % 3, b = (q / 3) % 3, c = q / 9;
        if (a == 1 || b == 1 || c == 1) {
            float r = a == 1 ? -ux : ex2;
            if (a == 0) r = 1.0f;
            if (b == 1) r = r * -uy;
            if (b == 2) r = r * ey2;
            if (c == 1) r = r * -uz;
            if (c == 2) r = r * ez2;
            return r;
        }
        float S = 0.0f;
        bool any = false;
        if (a == 2) {
            S = dx3;
            any = true;
        }
        if (b == 2) {
            S = any ? fmaf(S, dy3, S + dy3) : dy3;
            any = true;
        }
        if (c == 2) S = any ? fmaf(S, dz3, S + dz3) : dz3;
        const int n2 = (a == 2) + (b == 2) + (c == 2);
        const float M = n2 == 0 ? 1.0f : n2 == 1 ? 1.0f / 3.0f : n2 == 2 ? 1.0f / 9.0f : 1.0f / 27.0f;
        return n2 == 0 ? -drho : M * (S - drho);
    };
    constexpr int XX = 2, YY = 6, ZZ = 18, XY = 4, XZ = 10, YZ = 12;
    const float w = p.omega_p, wb = p.mrt[0], wh = p.mrt[1];
    // orders 0 and 1
    k[0] = 0.0f - Bq(0);
    k[1] = 0.5f * p.fx - Bq(1);
    k[3] = 0.5f * p.fy - Bq(3);
    k[9] = 0.5f * p.fz - Bq(9);
    // order 2: trace * (1 - bulk), normal differences and off-diagonals * (1 - omega+)
    const float Bxx = Bq(XX), Byy = Bq(YY), Bzz = Bq(ZZ), Bxy = Bq(XY), Bxz = Bq(XZ), Byz = Bq(YZ);
    float sxx, syy, szz, sxy, sxz, syz;              // relaxed deviations Dk*
    {
        const float dxx = k[XX] + Bxx, dyy = k[YY] + Byy, dzz = k[ZZ] + Bzz;
        const float T = (dxx + dyy + dzz) * (1.0f - wb);
        const float D1 = (dxx - dyy) * (1.0f - w), D2 = (dxx - dzz) * (1.0f - w);
        sxx = (T + D1 + D2) * (1.0f / 3.0f);
        syy = (T - 2.0f * D1 + D2) * (1.0f / 3.0f);
        szz = (T + D1 - 2.0f * D2) * (1.0f / 3.0f);
        sxy = (k[XY] + Bxy) * (1.0f - w);
        sxz = (k[XZ] + Bxz) * (1.0f - w);
        syz = (k[YZ] + Byz) * (1.0f - w);
    }
    k[XX] = sxx - Bxx;
    k[YY] = syy - Byy;
    k[ZZ] = szz - Bzz;
    k[XY] = sxy - Bxy;
    k[XZ] = sxz - Bxz;
    k[YZ] = syz - Byz;
    if constexpr (OP == OP_CM) {
#pragma unroll
        for (int q = 0; q < 27; ++q) {
            const int o = q % 3 + (q / 3) % 3 + q / 9;
            if (o >= 3) {
                const float B = Bq(q);
                k[q] = (k[q] + B) * (1.0f - wh) - B;
            }
        }
    } else {
        // normalised post-collision second moments as deviations: m_aa = 1/3 + a_a
        const float ax = sxx * ir, ay = syy * ir, az = szz * ir;
        const float bxy = sxy * ir, bxz = sxz * ir, byz = syz * ir;
        constexpr float t3 = 1.0f / 3.0f;
#pragma unroll
        for (int q = 0; q < 27; ++q) {
            const int o = q % 3 + (q / 3) % 3 + q / 9;
            if (o == 3 || o == 5) k[q] = 0.0f - Bq(q);
        }
        // order 4: (2,2,0)-type and (2,1,1)-type, each minus its equilibrium
        k[2 + 6] = rho * ((ax + ay) * t3 + ax * ay + 2.0f * bxy * bxy) - Bq(2 + 6);          // 220
        k[2 + 18] = rho * ((ax + az) * t3 + ax * az + 2.0f * bxz * bxz) - Bq(2 + 18);        // 202
        k[6 + 18] = rho * ((ay + az) * t3 + ay * az + 2.0f * byz * byz) - Bq(6 + 18);        // 022
        k[2 + 3 + 9] = rho * ((t3 + ax) * byz + 2.0f * bxy * bxz) - Bq(2 + 3 + 9);           // 211
        k[1 + 6 + 9] = rho * ((t3 + ay) * bxz + 2.0f * bxy * byz) - Bq(1 + 6 + 9);           // 121
        k[1 + 3 + 18] = rho * ((t3 + az) * bxy + 2.0f * bxz * byz) - Bq(1 + 3 + 18);         // 112
        // order 6: 222 minus 1/27
        k[26] = rho * ((ax + ay + az) * (t3 * t3) + (ax * ay + ax * az + ay * az) * t3 + ax * ay * az +
                       2.0f * ((t3 + ax) * byz * byz + (t3 + ay) * bxz * bxz + (t3 + az) * bxy * bxy) +
                       8.0f * bxy * bxz * byz) - Bq(26);
    }
    // back: inverse passes z, y, x
#pragma unroll
    for (int l = 0; l < 9; ++l) from_central(k[l], k[l + 9], k[l + 18], uz);
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        const int o = (l % 3) + 9 * (l / 3);
        from_central(k[o], k[o + 3], k[o + 6], uy);
    }
#pragma unroll
    for (int l = 0; l < 9; ++l) from_central(k[3 * l], k[3 * l + 1], k[3 * l + 2], ux);
#pragma unroll
    for (int q = 0; q < 27; ++q) g[dir_at(q)] = SCALED ? k[q] * p.scale : k[q];
    return Vel{ux, uy, uz};
}

}  // namespace slbm
