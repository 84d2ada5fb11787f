// aa_kernels.cuh -- the in-place AA stream-collide kernels (Sec. 5.1) over the
// compacted PDF-list (Sec. 3.1).
//
// State convention: after an even number of steps the field is "natural":
// row i, column k holds f_i(x_k) - w_i.
//   even step (t even, cell-local, no index reads): read row i of column k,
//     collide, write the post-collision value of direction i into row
//     inverse(i) of column k.
//   odd step (t odd): f_i(x_k) is the post-collision value of direction i of
//     the pull neighbour x_k - c_i, which the even step left in row inverse(i)
//     of that neighbour's column; flipping the row of the pull entry gives its
//     slot R(i,k).  Read all R(i,k), collide, and write the post-collision
//     value of direction inverse(i) back into R(i,k).  R(i,k) lies in row
//     inverse(i) of the neighbour x_k - c_i, which is the natural slot of
//     f_inverse(i) at that neighbour for the next time level (or, at a wall,
//     row i of column k: the bounced-back value), so the field is natural
//     again.  Each slot is read and written by one cell only, hence in place
//     without races.
// Boundary links (inlet/outlet) keep the cell's own slot i*S + k and apply
// their affine map on the read and on the write.
#pragma once

#include "common.cuh"

namespace slbm {

template <class T, int N>
struct alignas(sizeof(T) * N) Vec {
    T v[N];
};

template <class T, int N>
__device__ __forceinline__ Vec<T, N> ld_vec(const T *p) {
    return *reinterpret_cast<const Vec<T, N> *>(p);
}

template <class T, int N>
__device__ __forceinline__ void st_vec(T *p, const Vec<T, N> &x) {
    *reinterpret_cast<Vec<T, N> *>(p) = x;
}

// Index entries are read once per odd step: stream them past L2 (evict-first).
template <int N>
__device__ __forceinline__ Vec<int32_t, N> ld_index(const int32_t *p) {
    if constexpr (N == 1) {
        Vec<int32_t, 1> r;
        r.v[0] = __ldcs(p);
        return r;
    } else if constexpr (N == 2) {
        const int2 a = __ldcs(reinterpret_cast<const int2 *>(p));
        Vec<int32_t, 2> r;
        r.v[0] = a.x;
        r.v[1] = a.y;
        return r;
    } else {
        const int4 a = __ldcs(reinterpret_cast<const int4 *>(p));
        Vec<int32_t, 4> r;
        r.v[0] = a.x;
        r.v[1] = a.y;
        r.v[2] = a.z;
        r.v[3] = a.w;
        return r;
    }
}

template <int Q, int ST, int CPT>
__global__ void __launch_bounds__(256) aa_even_kernel(typename Store<ST>::T *__restrict__ pdf, int32_t S,
                                                      int32_t nf, CollideParams p) {
    using St = Store<ST>;
    using T = typename St::T;
    const int32_t k0 = (blockIdx.x * blockDim.x + threadIdx.x) * CPT;
    if (k0 >= nf) return;
    float g[CPT][Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const Vec<T, CPT> x = ld_vec<T, CPT>(pdf + i * S + k0);
#pragma unroll
        for (int c = 0; c < CPT; ++c) g[c][i] = St::ld(x.v[c], p.inv_scale);
    }
#pragma unroll
    for (int c = 0; c < CPT; ++c) collide<Q>(g[c], p);
    const bool full = k0 + CPT <= nf;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        Vec<T, CPT> y;
#pragma unroll
        for (int c = 0; c < CPT; ++c) y.v[c] = St::st(g[c][i], p.scale);
        T *dst = pdf + inv(i) * S + k0;
        if (full) {
            st_vec<T, CPT>(dst, y);
        } else {
#pragma unroll
            for (int c = 0; c < CPT; ++c)
                if (k0 + c < nf) dst[c] = y.v[c];
        }
    }
}

__device__ __forceinline__ void latch(int32_t *err, int32_t code) {
    if (err) atomicCAS(err, 0, code);
}

template <int Q, int ST, int CPT, bool HAS_BC, bool CHECK>
__global__ void __launch_bounds__(256) aa_odd_kernel(typename Store<ST>::T *__restrict__ pdf,
                                                     const int32_t *__restrict__ P, int32_t S, int32_t nf,
                                                     const LinkMap *__restrict__ maps, int32_t n_links,
                                                     CollideParams p, int32_t *err) {
    using St = Store<ST>;
    using T = typename St::T;
    const int32_t k0 = (blockIdx.x * blockDim.x + threadIdx.x) * CPT;
    if (k0 >= nf) return;
    int32_t e[CPT][Q];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const Vec<int32_t, CPT> x = ld_index<CPT>(P + (i - 1) * S + k0);
#pragma unroll
        for (int c = 0; c < CPT; ++c) e[c][i] = x.v[c];
    }
    float g[CPT][Q];
    int32_t R[CPT][Q];
    {
        const Vec<T, CPT> x = ld_vec<T, CPT>(pdf + k0);
#pragma unroll
        for (int c = 0; c < CPT; ++c) g[c][0] = St::ld(x.v[c], p.inv_scale);
    }
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        const int32_t k = k0 + c;
        const bool valid = (CPT == 1) || k < nf;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            int32_t ee = e[c][i];
            int32_t r = ee >= 0 ? flip_row(ee, i, S) : i * S + k;
            if (CHECK) {
                const bool bad = ee >= 0 ? (ee >= Q * S || r < 0 || r >= Q * S || r % S >= nf)
                                         : (-(ee + 1) >= n_links);
                if (bad) {
                    latch(err, 1 + i);
                    r = i * S + k;
                    e[c][i] = ee = i * S + k;   // treat as own slot, no map
                }
            }
            R[c][i] = r;
            if (valid) g[c][i] = St::ld(pdf[r], p.inv_scale);
            else g[c][i] = 0.f;
            if (HAS_BC && valid && ee < 0) {
                const LinkMap m = maps[-(ee + 1)];
                g[c][i] = m.s * g[c][i] + m.a;
            }
        }
    }
#pragma unroll
    for (int c = 0; c < CPT; ++c) collide<Q>(g[c], p);
    {
        Vec<T, CPT> y;
#pragma unroll
        for (int c = 0; c < CPT; ++c) y.v[c] = St::st(g[c][0], p.scale);
        if (k0 + CPT <= nf) {
            st_vec<T, CPT>(pdf + k0, y);
        } else {
#pragma unroll
            for (int c = 0; c < CPT; ++c)
                if (k0 + c < nf) pdf[k0 + c] = y.v[c];
        }
    }
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        if (CPT > 1 && k0 + c >= nf) continue;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            float v = g[c][inv(i)];
            if (HAS_BC && e[c][i] < 0) {
                const LinkMap m = maps[-(e[c][i] + 1)];
                v = m.s * v + m.a;
            }
            pdf[R[c][i]] = St::st(v, p.scale);
        }
    }
}

}  // namespace slbm
