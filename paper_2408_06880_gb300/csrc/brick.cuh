// brick.cuh -- the dense part of the hybrid sparse/dense layout (the paper's
// hybrid blocks, Sec. 4.1, at the granularity of 8^3 bricks): the AA odd
// step (Sec. 5.1) of the cells of full bricks.
//
// With the cell order SLBM_ORDER_HYBRID the complete bricks whose 512 voxels
// are all fluid come first: brick j holds cells 512 j .. 512 j + 511 in
// lexicographic order inside the brick.  The pull neighbour x_k - c_i of a
// cell of such a brick that lies inside the same brick is cell
// k - (c_x + 8 c_y + 64 c_z), so its odd-step slot is
// R(i,k) = inverse(i)*S + k - (c_x + 8 c_y + 64 c_z) by arithmetic, as in a
// dense block; only the links that cross the brick's faces need the list.
// Their slots are kept in a compact per-brick face list (about a fifth of
// the brick's index-list entries), so the odd step of a full brick reads
// ~0.8 instead of 4 index bytes per link (D3Q19).  The cells of the other
// bricks, numbered after the full ones, take the sparse odd step.
#pragma once

#include <type_traits>

#include "aa_kernels.cuh"

namespace slbm {

// Face value of a local coordinate for velocity component c (+1: 0, -1: 7).
__host__ __device__ __forceinline__ constexpr int face_of(int c) { return c == 1 ? 0 : 7; }

// Rank of local cell (lx, ly, lz) among the cells of a brick whose pull
// neighbour in direction i lies outside the brick, in local (lexicographic)
// order; -1 when the neighbour is inside.
template <int Q>
__host__ __device__ __forceinline__ int face_rank(int i, int lx, int ly, int lz) {
    const int ax = cx(i), ay = cy(i), az = cz(i);
    const bool fx = ax != 0 && lx == face_of(ax), fy = ay != 0 && ly == face_of(ay), fz = az != 0 && lz == face_of(az);
    if (!(fx || fy || fz)) return -1;
    if (ay == 0 && az == 0) return ly + 8 * lz;
    if (ax == 0 && az == 0) return lx + 8 * lz;
    if (ax == 0 && ay == 0) return lx + 8 * ly;
    if (az == 0) {
        const int by = face_of(ay);
        return 15 * lz + ly + 7 * (ly > by) + (ly == by ? lx : 0);
    }
    if (ay == 0) {
        const int bz = face_of(az);
        return 8 * lz + 56 * (lz > bz) + (lz == bz ? lx + 8 * ly : ly);
    }
    if (ax == 0) {
        const int bz = face_of(az);
        return 8 * lz + 56 * (lz > bz) + (lz == bz ? lx + 8 * ly : lx);
    }
    const int by = face_of(ay), bz = face_of(az);
    return 15 * lz + 49 * (lz > bz) + (lz == bz ? lx + 8 * ly : ly + 7 * (ly > by) + (ly == by ? lx : 0));
}

// Face cells of direction i: 64 (one nonzero velocity component), 120 (two)
// or 169 (three).
__host__ __device__ __forceinline__ constexpr int face_count(int i) {
    return ((cx(i) != 0) + (cy(i) != 0) + (cz(i) != 0)) == 1 ? 64
           : ((cx(i) != 0) + (cy(i) != 0) + (cz(i) != 0)) == 2 ? 120 : 169;
}

// Offset of direction i's face entries in a brick's face block.
__host__ __device__ __forceinline__ constexpr int face_offset(int i) {
    int o = 0;
    for (int j = 1; j < i; ++j) o += face_count(j);
    return o;
}

// Entries of a brick's face block: 1824 (D3Q19), 3176 (D3Q27).
template <int Q>
__host__ __device__ __forceinline__ constexpr int face_block() {
    return face_offset(Q);
}

// f(integral_constant<int, I>) for I = B .. E-1, so that direction-dependent
// offsets are compile-time constants.
template <int B, int E, class F>
__device__ __forceinline__ void for_dirs(F &&f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        for_dirs<B + 1, E>(f);
    }
}

// Face lists of the full bricks from the device slot list: one thread per
// (full brick, local cell); each writes its face entries.
template <int Q>
__global__ void build_face_list(const int32_t *__restrict__ R, int32_t S, int32_t n_full_cells,
                                int32_t *__restrict__ face) {
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_full_cells) return;
    const int32_t j = k >> 9, l = k & 511;
    const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
    constexpr int FB = face_block<Q>();
    int32_t *fb = face + (int64_t)j * FB;
    for_dirs<1, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int off = face_offset(i);
        const int r = face_rank<Q>(i, lx, ly, lz);
        if (r >= 0) fb[off + r] = R[(int64_t)(i - 1) * S + k];
    });
}

// Odd step of the cells of full bricks, [0, n_full_cells): 128 threads, one
// cell each (a brick is four blocks).  Inside-brick links by arithmetic,
// face links from the brick's face block; then the collision and the scatter
// of the plain odd step.  pf_dist > 0: thread 0 first asks the bulk-copy
// engine to prefetch into L2 the face block of the brick pf_dist blocks
// ahead.
template <int Q, int ST, bool HAS_BC>
__global__ void __launch_bounds__(256) aa_odd_brick_kernel(typename Store<ST>::T *__restrict__ pdf,
                                                           const int32_t *__restrict__ face, int32_t S,
                                                           int32_t n_full_cells, const LinkMap *__restrict__ maps,
                                                           CollideParams p, int32_t pf_dist) {
    using St = Store<ST>;
    constexpr int FB = face_block<Q>();
    if (pf_dist > 0 && threadIdx.x == 0) {
        const int64_t c0 = ((int64_t)blockIdx.x + pf_dist) * blockDim.x;
        if (c0 < n_full_cells && (c0 & 511) == 0) bulk_prefetch_l2(face + (c0 >> 9) * FB, FB * 4u);
    }
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_full_cells) return;
    const int32_t j = k >> 9, l = k & 511;
    const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
    const int32_t *fb = face + (int64_t)j * FB;
    int32_t e[Q], R[Q];
    for_dirs<1, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int off = face_offset(i);
        constexpr int shift = cx(i) + 8 * cy(i) + 64 * cz(i);
        const int r = face_rank<Q>(i, lx, ly, lz);
        e[i] = r < 0 ? inv(i) * S + k - shift : __ldg(fb + off + r);
    });
    float g[Q];
    g[0] = St::raw(__ldg(pdf + k));
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        R[i] = (HAS_BC && e[i] < 0) ? i * S + k : e[i];
        g[i] = St::raw(__ldg(pdf + R[i]));
    }
    const Vel u = collide<Q, St::scaled>(g, p);
    pdf[k] = St::pack(g[0]);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        float v = g[inv(i)];
        if (HAS_BC && e[i] < 0) v = apply_link(maps[-(e[i] + 1)], v, u.x, u.y, u.z, p.scale);
        pdf[R[i]] = St::pack(v);
    }
}

}  // namespace slbm
