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
//     of that neighbour's column: the slot R(i,k), which is the pull entry
//     P(i,k) with its row flipped between i and inverse(i).  The device
//     index-list stores R(i,k) directly (see lists.cu).  Read all R(i,k), collide, and write the post-collision
//     value of direction inverse(i) back into R(i,k).  R(i,k) lies in row
//     inverse(i) of the neighbour x_k - c_i, which is the natural slot of
//     f_inverse(i) at that neighbour for the next time level (or, at a wall,
//     row i of column k: the bounced-back value), so the field is natural
//     again.  Each slot is read and written by one cell only, hence in place
//     without races.
// Boundary links (inlet/outlet) keep the cell's own slot i*S + k; the value
// stored there is the link's map of the post-collision value, applied when it
// is written (here for the odd step; around the even step by the boundary
// fix-up kernels), so reads are plain.
#pragma once

#include "bulk.cuh"
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

// ld_vec through the read-only data path (2, 4, 8 or 16 bytes).
template <class T, int N>
__device__ __forceinline__ Vec<T, N> ldg_vec(const T *p) {
    constexpr int B = (int)sizeof(Vec<T, N>);
    static_assert(B == 2 || B == 4 || B == 8 || B == 16, "vector of 2, 4, 8 or 16 bytes");
    Vec<T, N> r;
    if constexpr (B == 2) {
        const unsigned short x = __ldg(reinterpret_cast<const unsigned short *>(p));
        memcpy(&r, &x, 2);
    } else if constexpr (B == 4) {
        const unsigned int x = __ldg(reinterpret_cast<const unsigned int *>(p));
        memcpy(&r, &x, 4);
    } else if constexpr (B == 8) {
        const uint2 x = __ldg(reinterpret_cast<const uint2 *>(p));
        memcpy(&r, &x, 8);
    } else {
        const uint4 x = __ldg(reinterpret_cast<const uint4 *>(p));
        memcpy(&r, &x, 16);
    }
    return r;
}

// A row segment of CPT consecutive cells: stored values <-> floats in stored
// units.  load_ro (global memory only) takes the read-only data path: in the
// even step a cell reads its own slots and writes its own slots (rows i and
// inverse(i) of its column), which no other cell touches.  FP16 pairs convert with the packed half2 forms (same rounding as
// element-wise conversion, half the instructions on the store side).
template <int ST, int CPT>
struct RowIO {
    using St = Store<ST>;
    using T = typename St::T;
    static __device__ __forceinline__ void load(const T *p, float (&f)[CPT]) {
        const Vec<T, CPT> x = ld_vec<T, CPT>(p);
#pragma unroll
        for (int c = 0; c < CPT; ++c) f[c] = St::raw(x.v[c]);
    }
    static __device__ __forceinline__ void load_ro(const T *p, float (&f)[CPT]) {   // global memory only
        const Vec<T, CPT> x = ldg_vec<T, CPT>(p);
#pragma unroll
        for (int c = 0; c < CPT; ++c) f[c] = St::raw(x.v[c]);
    }
    static __device__ __forceinline__ Vec<T, CPT> pack(const float (&f)[CPT]) {
        Vec<T, CPT> y;
#pragma unroll
        for (int c = 0; c < CPT; ++c) y.v[c] = St::pack(f[c]);
        return y;
    }
};

template <int CPT>
struct RowIO<ST_F16, CPT> {
    static_assert(CPT == 1 || CPT % 2 == 0, "FP16 rows: 1 or an even number of cells");
    static __device__ __forceinline__ void load(const __half *p, float (&f)[CPT]) {
        if constexpr (CPT == 1) {
            f[0] = __half2float(*p);
        } else {
            const Vec<__half2, CPT / 2> x = ld_vec<__half2, CPT / 2>(reinterpret_cast<const __half2 *>(p));
#pragma unroll
            for (int c = 0; c < CPT / 2; ++c) {
                const float2 v = __half22float2(x.v[c]);
                f[2 * c] = v.x;
                f[2 * c + 1] = v.y;
            }
        }
    }
    static __device__ __forceinline__ void load_ro(const __half *p, float (&f)[CPT]) {   // global memory only
        if constexpr (CPT == 1) {
            f[0] = __half2float(__ldg(p));
        } else {
            const Vec<__half2, CPT / 2> x = ldg_vec<__half2, CPT / 2>(reinterpret_cast<const __half2 *>(p));
#pragma unroll
            for (int c = 0; c < CPT / 2; ++c) {
                const float2 v = __half22float2(x.v[c]);
                f[2 * c] = v.x;
                f[2 * c + 1] = v.y;
            }
        }
    }
    static __device__ __forceinline__ Vec<__half, CPT> pack(const float (&f)[CPT]) {
        Vec<__half, CPT> y;
        if constexpr (CPT == 1) {
            y.v[0] = __float2half_rn(f[0]);
        } else {
#pragma unroll
            for (int c = 0; c < CPT / 2; ++c) {
                const __half2 h = __floats2half2_rn(f[2 * c], f[2 * c + 1]);
                y.v[2 * c] = __low2half(h);
                y.v[2 * c + 1] = __high2half(h);
            }
        }
        return y;
    }
};

// Collision of the CPT cells a thread holds (g[c][i]: cell c, direction i).
// PACK (CPT even): cells c and c + 1 share one pass of the
// collision in the two lanes of the paired FP32 instructions -- the same
// roundings per cell as the scalar pass, half the FP instructions.
template <int Q, bool SCALED, int OP, int CPT, bool PACK>
__device__ __forceinline__ void collide_cells(float (&g)[CPT][Q], const CollideParams &p, Vel (&u)[CPT]) {
    if constexpr (PACK) {
        static_assert(CPT % 2 == 0, "paired collision: an even number of cells");
#pragma unroll
        for (int c = 0; c < CPT; c += 2) {
            F2 h[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) h[i] = F2{make_float2(g[c][i], g[c + 1][i])};
            static_assert(OP == OP_TRT || OP == OP_MRT, "paired collision: TRT and MRT");
            VelT<F2> v;
            if constexpr (OP == OP_MRT) {
                static_assert(Q == 19, "MRT is defined for D3Q19");
                v = collide_mrt_v<SCALED>(h, p);
            } else {
                v = collide_v<Q, SCALED>(h, p);
            }
            u[c] = Vel{v.x.v.x, v.y.v.x, v.z.v.x};
            u[c + 1] = Vel{v.x.v.y, v.y.v.y, v.z.v.y};
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                g[c][i] = h[i].v.x;
                g[c + 1][i] = h[i].v.y;
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c < CPT; ++c) u[c] = collide_op<Q, SCALED, OP>(g[c], p);
    }
}

template <int Q, bool SCALED, int OP, int CPT, bool PACK>
__device__ __forceinline__ void collide_cells(float (&g)[CPT][Q], const CollideParams &p) {
    Vel u[CPT];
    collide_cells<Q, SCALED, OP, CPT, PACK>(g, p, u);
}

// Inlet/outlet links of the even step, applied by the even kernel itself.
// The links are numbered by cell (link_cell ascending) and ltile[t] is the
// first link of a cell at or after cell 32 t, so the links of the cells
// [32 t0, 32 t1) are ltile[t0] .. ltile[t1] - 1.  A block reads its range
// while its populations load; after its stores it writes its cells'
// velocities to shared memory, synchronises, and its threads replace each
// link slot (re-read after the barrier) by its map -- the operations of the
// separate fix-up kernels.
struct EvenLinks {
    const int32_t *ltile, *link_cell, *link_dir;
    const LinkMap *maps;
};
constexpr int EVEN_LINK_TILE = 32;

// Link range [b0, b1) of the cells [kb, ke), kb a multiple of 32 and
// ke <= N_F; empty when kb >= ke (a staged tile of padding columns only),
// without reading the table, whose last entry is tile ceil(N_F / 32).
__device__ __forceinline__ void even_link_range(const EvenLinks &lk, int32_t kb, int32_t ke, int32_t &b0,
                                                int32_t &b1) {
    if (kb >= ke) {
        b0 = b1 = 0;
        return;
    }
    b0 = lk.ltile[kb / EVEN_LINK_TILE];
    b1 = lk.ltile[(ke + EVEN_LINK_TILE - 1) / EVEN_LINK_TILE];
}

template <int ST>
__device__ __forceinline__ void even_links_apply(typename Store<ST>::T *pdf, int32_t S, int32_t kb, int32_t b0,
                                                 int32_t b1, const float *us, int32_t span, const EvenLinks &lk,
                                                 float scale) {
    using St = Store<ST>;
    for (int32_t b = b0 + threadIdx.x; b < b1; b += blockDim.x) {
        const int32_t c = lk.link_cell[b] - kb;
        const LinkMap m = lk.maps[b];
        typename St::T *slot = pdf + lk.link_dir[b] * S + (kb + c);
        *slot = St::pack(apply_link(m, St::raw(*slot), us[c], us[span + c], us[2 * span + c], scale));
    }
}

// Load, collide and store the CPT cells k0 .. k0 + CPT - 1 of the even step.
template <int Q, int ST, int CPT, int OP, bool PACK>
__device__ __forceinline__ void aa_even_cells(typename Store<ST>::T *__restrict__ pdf, int32_t S, int32_t nf,
                                              const CollideParams &p, int32_t k0, Vel (&u)[CPT]) {
    using St = Store<ST>;
    using T = typename St::T;
    float g[CPT][Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float f[CPT];
        RowIO<ST, CPT>::load_ro(pdf + i * S + k0, f);
#pragma unroll
        for (int c = 0; c < CPT; ++c) g[c][i] = f[c];
    }
    collide_cells<Q, St::scaled, OP, CPT, PACK>(g, p, u);
    const bool full = k0 + CPT <= nf;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float f[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) f[c] = g[c][i];
        const Vec<T, CPT> y = RowIO<ST, CPT>::pack(f);
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

// The even step of a block's cells.  BC: the domain has inlet/outlet links;
// the kernel applies their maps to the link slots it stored (EvenLinks;
// dynamic shared memory: 3 x blockDim x CPT floats).
template <int Q, int ST, int CPT, int OP, bool PACK, bool BC>
__device__ __forceinline__ void aa_even_body(typename Store<ST>::T *__restrict__ pdf, int32_t S, int32_t nf,
                                             const CollideParams &p, const EvenLinks &lk) {
    const int32_t k0 = (blockIdx.x * blockDim.x + threadIdx.x) * CPT;
    if constexpr (BC) {
        extern __shared__ float even_us[];
        const int32_t span = blockDim.x * CPT, kb = blockIdx.x * span;
        const int32_t ke = kb + span < nf ? kb + span : nf;
        int32_t b0, b1;
        even_link_range(lk, kb, ke, b0, b1);
        // this thread's first link of the block's range: its cell, direction
        // and map are loaded while the populations load, so that after the
        // barrier only the slot's re-read remains
        const int32_t lb = b0 + threadIdx.x;
        const bool first = lb < b1;
        int32_t lc = 0, ld = 0;
        LinkMap lm{};
        if (first) {
            lc = lk.link_cell[lb] - kb;
            ld = lk.link_dir[lb];
            lm = lk.maps[lb];
        }
        Vel u[CPT] = {};
        if (k0 < nf) aa_even_cells<Q, ST, CPT, OP, PACK>(pdf, S, nf, p, k0, u);
        if (b0 == b1) return;                         // uniform across the block
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int32_t l = threadIdx.x * CPT + c;
            even_us[l] = u[c].x;
            even_us[span + l] = u[c].y;
            even_us[2 * span + l] = u[c].z;
        }
        __syncthreads();
        if (first) {
            using St = Store<ST>;
            typename St::T *slot = pdf + ld * S + (kb + lc);
            *slot = St::pack(apply_link(lm, St::raw(*slot), even_us[lc], even_us[span + lc], even_us[2 * span + lc],
                                        p.scale));
        }
        even_links_apply<ST>(pdf, S, kb, lb + blockDim.x - threadIdx.x, b1, even_us, span, lk, p.scale);
    } else {
        if (k0 >= nf) return;
        Vel u[CPT];
        aa_even_cells<Q, ST, CPT, OP, PACK>(pdf, S, nf, p, k0, u);
    }
}

template <int Q, int ST, int CPT, int OP = OP_TRT, bool PACK = false, bool BC = false>
__global__ void __launch_bounds__(256) aa_even_kernel(typename Store<ST>::T *__restrict__ pdf, int32_t S,
                                                      int32_t nf, CollideParams p, EvenLinks lk = {}) {
    aa_even_body<Q, ST, CPT, OP, PACK, BC>(pdf, S, nf, p, lk);
}

__device__ __forceinline__ void latch(int32_t *err, int32_t code) {
    if (err) atomicCAS(err, 0, code);
}

// CPT cells per thread, strided by the block size (cell c of thread t in block
// b is b*blockDim*CPT + c*blockDim + t), so that every load and store
// instruction of a warp covers consecutive cells.
// pf_dist > 0: thread 0 first asks the bulk-copy engine to prefetch into L2
// the index-list rows of the block pf_dist blocks ahead -- about one residency
// wave later -- so that block's first round trip hits L2.
// RELOAD (CPT = 1, no links): the slots are re-read from the list (an L1
// hit) before the scatter instead of being held in registers through the
// collision, which frees registers for more resident threads.
// The gathers go through the read-only data path (__ldg) although the kernel
// writes the PDF-list: each slot is read by one cell only, once, and written
// afterwards by that same cell, so no thread ever reads a slot after it was
// written in this launch and a line held in the read-only cache can never
// supply a stale value that is used.
// CODE: the slots come from the 16-bit link codes and their per-tile column
// bases (2 bytes per link instead of 4); an escape code reads the slot from
// the int32 list.  The decoded slot equals R(i, k) exactly.
template <int Q, int ST, int CPT, bool HAS_BC, bool CHECK, bool RELOAD, bool CODE, int OP>
__device__ __forceinline__ void aa_odd_body(typename Store<ST>::T *__restrict__ pdf, const int32_t *__restrict__ P,
                                            int32_t S, int32_t nf, const LinkMap *__restrict__ maps,
                                            int32_t n_links, const CollideParams &p, int32_t *err,
                                            int32_t pf_dist, const uint16_t *__restrict__ code,
                                            const int32_t *__restrict__ cbase, int32_t k_first = 0) {
    using St = Store<ST>;
    using T = typename St::T;
    const int32_t span = blockDim.x * CPT;
    if (pf_dist > 0 && threadIdx.x == 0) {
        const int64_t c0 = k_first + ((int64_t)blockIdx.x + pf_dist) * span;
        if (c0 < nf) {
            const int64_t left = (int64_t)S - c0;
            const uint32_t cells = (uint32_t)(left < (int64_t)span ? left : (int64_t)span);
#pragma unroll
            for (int r = 0; r < Q - 1; ++r) {
                if (CODE) bulk_prefetch_l2(code + r * S + c0, cells * 2u);
                else bulk_prefetch_l2(P + r * S + c0, cells * 4u);
            }
        }
    }
    const int32_t kb = k_first + blockIdx.x * span + threadIdx.x;
    // CODE: every lane stays to the end of the decode (warp shuffles)
    if (!CODE && kb >= nf) return;
    int32_t e[CPT][Q];
    bool valid[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) valid[c] = kb + c * (int32_t)blockDim.x < nf;
    if (CODE) {
        // A warp's cells lie in one code tile: lane r holds the tile's base of
        // direction r+1, loaded beside the codes and broadcast by shuffles.
        // Base -1 (a tile-direction of too wide a span): the whole warp reads
        // the int32 slots; an escape code (inlet/outlet link, domains with
        // links only) reads that one slot.
        const int lane = threadIdx.x & 31;
        const int32_t n_tiles = S / CODE_TILE;
        uint32_t cc[CPT][Q];
        int32_t bl[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int32_t tile = (kb + c * (int32_t)blockDim.x) / CODE_TILE;
            bl[c] = (lane < Q - 1 && tile < n_tiles) ? __ldg(cbase + tile * (Q - 1) + lane) : -1;
        }
#pragma unroll
        for (int i = 1; i < Q; ++i) {
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int32_t k = kb + c * blockDim.x;
                cc[c][i] = valid[c] ? __ldg(code + (i - 1) * S + k) : CODE_WALL;
            }
        }
#pragma unroll
        for (int i = 1; i < Q; ++i) {
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int32_t k = kb + c * blockDim.x;
                const int32_t b = __shfl_sync(0xffffffffu, bl[c], i - 1);
                const uint32_t x = cc[c][i];
                if (b >= 0 && !(HAS_BC && x == CODE_ESCAPE)) e[c][i] = x == CODE_WALL ? i * S + k : inv(i) * S + b + (int32_t)x;
                else e[c][i] = valid[c] ? P[(i - 1) * S + k] : i * S + k;
            }
        }
        if (kb >= nf) return;
    } else {
#pragma unroll
        for (int i = 1; i < Q; ++i) {
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int32_t k = kb + c * blockDim.x;
                if (RELOAD) e[c][i] = P[(i - 1) * S + k];
                else e[c][i] = valid[c] ? __ldg(P + (i - 1) * S + k) : 0;
            }
        }
    }
    float g[CPT][Q];
    int32_t R[CPT][Q];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        const int32_t k = kb + c * blockDim.x;
        g[c][0] = valid[c] ? St::raw(__ldg(pdf + k)) : 0.f;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            int32_t ee = e[c][i];
            int32_t r = ee >= 0 ? ee : i * S + k;
            if (CHECK) {
                const bool bad = ee >= 0 ? (ee >= Q * S || r % S >= nf) : (-(ee + 1) >= n_links);
                if (bad) {
                    latch(err, 1 + i);
                    r = i * S + k;
                    e[c][i] = ee = i * S + k;   // treat as own slot, no map
                }
            }
            R[c][i] = r;
            g[c][i] = valid[c] ? St::raw(__ldg(pdf + r)) : 0.f;
        }
    }
    Vel u[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) u[c] = collide_op<Q, St::scaled, OP>(g[c], p);
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        const int32_t k = kb + c * blockDim.x;
        if (!valid[c]) continue;
        pdf[k] = St::pack(g[c][0]);
        if constexpr (RELOAD) {
#pragma unroll
            for (int i = 1; i < Q; ++i) pdf[__ldcs(P + (i - 1) * S + k)] = St::pack(g[c][inv(i)]);
        } else {
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                float v = g[c][inv(i)];
                if (HAS_BC && e[c][i] < 0) v = apply_link(maps[-(e[c][i] + 1)], v, u[c].x, u[c].y, u[c].z, p.scale);
                pdf[R[c][i]] = St::pack(v);
            }
        }
    }
}

template <int Q, int ST, int CPT, bool HAS_BC, bool CHECK, bool RELOAD = false, bool CODE = false,
          int OP = OP_TRT>
__global__ void __launch_bounds__(256) aa_odd_kernel(typename Store<ST>::T *__restrict__ pdf,
                                                     const int32_t *__restrict__ P, int32_t S, int32_t nf,
                                                     const LinkMap *__restrict__ maps, int32_t n_links,
                                                     CollideParams p, int32_t *err, int32_t pf_dist,
                                                     const uint16_t *__restrict__ code = nullptr,
                                                     const int32_t *__restrict__ cbase = nullptr) {
    aa_odd_body<Q, ST, CPT, HAS_BC, CHECK, RELOAD, CODE, OP>(pdf, P, S, nf, maps, n_links, p, err, pf_dist, code,
                                                              cbase);
}

// The plain odd kernel (1 cell per thread, L2 index prefetch) over the cells
// k_first .. nf-1 only (the sparse part of the hybrid cell order).
template <int Q, int ST, bool HAS_BC>
__global__ void __launch_bounds__(256) aa_odd_kernel_from(typename Store<ST>::T *__restrict__ pdf,
                                                          const int32_t *__restrict__ P, int32_t S, int32_t nf,
                                                          const LinkMap *__restrict__ maps, int32_t n_links,
                                                          CollideParams p, int32_t *err, int32_t pf_dist,
                                                          int32_t k_first) {
    aa_odd_body<Q, ST, 1, HAS_BC, false, false, false, OP_TRT>(pdf, P, S, nf, maps, n_links, p, err, pf_dist, nullptr,
                                                                nullptr, k_first);
}

// The plain odd kernel (1 cell per thread, L2 index prefetch) held to 64
// registers a thread -- four resident 256-thread blocks -- so that more warps
// keep gathers in flight, at the cost of some registers spilled to L1.
template <int Q, int ST, bool HAS_BC>
__global__ void __launch_bounds__(256, 4) aa_odd_kernel_r64(typename Store<ST>::T *__restrict__ pdf,
                                                            const int32_t *__restrict__ P, int32_t S, int32_t nf,
                                                            const LinkMap *__restrict__ maps, int32_t n_links,
                                                            CollideParams p, int32_t *err, int32_t pf_dist) {
    aa_odd_body<Q, ST, 1, HAS_BC, false, false, false, OP_TRT>(pdf, P, S, nf, maps, n_links, p, err, pf_dist,
                                                                nullptr, nullptr);
}

// The MRT, central-moment and cumulant collisions hold a cell's moments
// through several hundred instructions; these forms of the plain kernels
// (128 threads, 1 cell each; odd: L2 index prefetch) are held to five
// resident blocks a multiprocessor (at most 102 registers a thread) so that
// more warps keep memory requests in flight.
template <int Q, int ST, int OP, bool BC>
__global__ void __launch_bounds__(128, 5) aa_even_kernel_b5(typename Store<ST>::T *__restrict__ pdf, int32_t S,
                                                            int32_t nf, CollideParams p, EvenLinks lk) {
    aa_even_body<Q, ST, 1, OP, false, BC>(pdf, S, nf, p, lk);
}

template <int Q, int ST, int OP, bool HAS_BC>
__global__ void __launch_bounds__(128, 5) aa_odd_kernel_b5(typename Store<ST>::T *__restrict__ pdf,
                                                           const int32_t *__restrict__ P, int32_t S, int32_t nf,
                                                           const LinkMap *__restrict__ maps, int32_t n_links,
                                                           CollideParams p, int32_t *err, int32_t pf_dist) {
    aa_odd_body<Q, ST, 1, HAS_BC, false, false, false, OP>(pdf, P, S, nf, maps, n_links, p, err, pf_dist, nullptr,
                                                           nullptr);
}


}  // namespace slbm

// ---------------------------------------------------------------------------
// Persistent variants with asynchronous bulk staging (Blackwell bulk-copy
// engine, cp.async.bulk + mbarrier transaction counts).  Each CTA walks tiles
// of TILE cells (tile, tile + gridDim, ...).  One elected thread keeps NSTAGE
// tiles in flight: for the odd step the Q-1 index-list rows of the tile, for
// the even step the Q PDF rows.  Threads read their column from shared
// memory, so the index (or PDF) round trip of the next tiles overlaps the
// gathers, collision and stores of the current one.  Waits are bounded; a
// timeout latches an error code in *err and every thread of the CTA leaves
// the loop together, after the elected thread has waited (bounded) for the
// copies it still has in flight.  TILE divides 128 and the row stride S is a
// multiple of 128, so every tile is whole and every copy is 16-byte aligned.
namespace slbm {

constexpr int32_t ERR_STAGE_TIMEOUT = 100;

// ---------------------------------------------------------------------------
// Boundary fix-up around the even step of a pool member with inlet/outlet
// links (the pool kernels do not apply link maps).  Before the even step each
// boundary cell's Guo velocity at the current time is saved, with the TRT
// collision's bits; after it, the values the even step stored in the cell's
// link slots are replaced by their link maps -- the same operations as the
// even kernels that fold the maps in (EvenLinks), so both give the same bits.
template <int Q, int ST>
__global__ void bc_pre_kernel(const typename Store<ST>::T *__restrict__ pdf, int32_t S,
                              const int32_t *__restrict__ bcell, int32_t n_bcells, CollideParams p,
                              float *__restrict__ ubuf) {
    using St = Store<ST>;
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_bcells) return;
    const int32_t k = bcell[j];
    float g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = St::raw(pdf[i * S + k]);
    const Vel u = guo_velocity<Q, St::scaled>(g, p);
    ubuf[3 * j] = u.x;
    ubuf[3 * j + 1] = u.y;
    ubuf[3 * j + 2] = u.z;
}

template <int ST>
__global__ void bc_post_kernel(typename Store<ST>::T *__restrict__ pdf, int32_t S, const int32_t *__restrict__ bcell,
                               const int32_t *__restrict__ bfirst, int32_t n_bcells,
                               const int32_t *__restrict__ link_dir, const LinkMap *__restrict__ maps,
                               const float *__restrict__ ubuf, float scale) {
    using St = Store<ST>;
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_bcells) return;
    const int32_t k = bcell[j];
    const float ux = ubuf[3 * j], uy = ubuf[3 * j + 1], uz = ubuf[3 * j + 2];
    for (int32_t b = bfirst[j]; b < bfirst[j + 1]; ++b) {
        typename Store<ST>::T *slot = pdf + link_dir[b] * S + k;
        *slot = St::pack(apply_link(maps[b], St::raw(*slot), ux, uy, uz, scale));
    }
}


// The odd-step update of one cell from its Q-1 pull entries.
template <int Q, int ST, bool HAS_BC>
__device__ __forceinline__ void odd_cell(typename Store<ST>::T *__restrict__ pdf, const int32_t (&e)[Q],
                                         int32_t k, int32_t S, const LinkMap *__restrict__ maps,
                                         const CollideParams &p) {
    using St = Store<ST>;
    int32_t R[Q];
    float g[Q];
    g[0] = St::raw(__ldg(pdf + k));
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int32_t ee = e[i];
        R[i] = (HAS_BC && ee < 0) ? i * S + k : ee;
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

// Pipeline bookkeeping kept by the elected thread: which stages have a copy
// in flight and the parity of each stage's next completion.
struct StageState {
    uint32_t pending = 0, phase = 0;
};

template <int NSTAGE>
__device__ __forceinline__ void drain_stages(uint64_t *bar, const StageState &ss) {
#pragma unroll
    for (int s = 0; s < NSTAGE; ++s)
        if (ss.pending >> s & 1u) mbar_wait_bounded(&bar[s], ss.phase >> s & 1u);
}

template <int Q, int ST, bool HAS_BC, int TILE, int NSTAGE>
__global__ void __launch_bounds__(TILE) aa_odd_staged_kernel(typename Store<ST>::T *__restrict__ pdf,
                                                             const int32_t *__restrict__ P, int32_t S,
                                                             int32_t nf, const LinkMap *__restrict__ maps,
                                                             CollideParams p, int32_t *err) {
    constexpr int R1 = Q - 1;
    __shared__ __align__(128) int32_t tile[NSTAGE][R1][TILE];
    __shared__ __align__(8) uint64_t bar[NSTAGE];
    const int tid = threadIdx.x;
    const int32_t n_tiles = S / TILE;
    StageState ss;
    auto issue = [&](int32_t t, int s) {
        mbar_arrive_expect_tx(&bar[s], R1 * TILE * 4);
#pragma unroll
        for (int r = 0; r < R1; ++r) bulk_g2s(&tile[s][r][0], P + r * S + t * TILE, TILE * 4, &bar[s]);
        ss.pending |= 1u << s;
    };
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < NSTAGE; ++s) mbar_init(&bar[s], 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < NSTAGE; ++s) {
            const int32_t t = blockIdx.x + s * gridDim.x;
            if (t < n_tiles) issue(t, s);
        }
    }
    int it = 0;
    for (int32_t t = blockIdx.x; t < n_tiles; t += gridDim.x, ++it) {
        const int s = it % NSTAGE;
        const uint32_t ph = (uint32_t)(it / NSTAGE) & 1u;
        const bool ok = mbar_wait_bounded(&bar[s], ph);
        int32_t e[Q];
        e[0] = 0;
        if (ok) {
#pragma unroll
            for (int r = 0; r < R1; ++r) e[r + 1] = tile[s][r][tid];
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) latch(err, ERR_STAGE_TIMEOUT);
            break;
        }
        if (tid == 0) {
            ss.pending &= ~(1u << s);
            ss.phase ^= 1u << s;
            const int32_t tn = t + NSTAGE * gridDim.x;
            if (tn < n_tiles) issue(tn, s);
        }
        const int32_t k = t * TILE + tid;
        if (k < nf) odd_cell<Q, ST, HAS_BC>(pdf, e, k, S, maps, p);
    }
    if (tid == 0 && ss.pending) drain_stages<NSTAGE>(bar, ss);
    __syncthreads();
}

// TILE cells per tile, CPT consecutive cells per thread (TILE / CPT threads);
// PACK: the cells of a thread collide in pairs (collide_cells).  BC: the
// inlet/outlet link maps of a tile's cells are applied after its stores
// (EvenLinks), behind one barrier.
template <int Q, int ST, int TILE, int NSTAGE, int CPT = 1, bool PACK = false, bool BC = false>
__global__ void __launch_bounds__(TILE / CPT) aa_even_staged_kernel(typename Store<ST>::T *__restrict__ pdf,
                                                                    int32_t S, int32_t nf, CollideParams p,
                                                                    int32_t *err, EvenLinks lk = {}) {
    using St = Store<ST>;
    using T = typename St::T;
    static_assert(TILE % EVEN_LINK_TILE == 0, "tiles of whole link tiles");
    __shared__ __align__(128) T tile[NSTAGE][Q][TILE];
    __shared__ __align__(8) uint64_t bar[NSTAGE];
    __shared__ float us[BC ? 3 * TILE : 1];
    const int tid = threadIdx.x;
    const int32_t n_tiles = S / TILE;
    StageState ss;
    auto issue = [&](int32_t t, int s) {
        mbar_arrive_expect_tx(&bar[s], Q * TILE * (uint32_t)sizeof(T));
#pragma unroll
        for (int i = 0; i < Q; ++i) bulk_g2s(&tile[s][i][0], pdf + i * S + t * TILE, TILE * sizeof(T), &bar[s]);
        ss.pending |= 1u << s;
    };
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < NSTAGE; ++s) mbar_init(&bar[s], 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < NSTAGE; ++s) {
            const int32_t t = blockIdx.x + s * gridDim.x;
            if (t < n_tiles) issue(t, s);
        }
    }
    int it = 0;
    for (int32_t t = blockIdx.x; t < n_tiles; t += gridDim.x, ++it) {
        const int s = it % NSTAGE;
        const uint32_t ph = (uint32_t)(it / NSTAGE) & 1u;
        int32_t b0 = 0, b1 = 0;
        if constexpr (BC) even_link_range(lk, t * TILE, (t + 1) * TILE < nf ? (t + 1) * TILE : nf, b0, b1);
        const bool ok = mbar_wait_bounded(&bar[s], ph);
        float g[CPT][Q];
        if (ok) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                float f[CPT];
                RowIO<ST, CPT>::load(&tile[s][i][CPT * tid], f);
#pragma unroll
                for (int c = 0; c < CPT; ++c) g[c][i] = f[c];
            }
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) latch(err, ERR_STAGE_TIMEOUT);
            break;
        }
        if (tid == 0) {
            ss.pending &= ~(1u << s);
            ss.phase ^= 1u << s;
            const int32_t tn = t + NSTAGE * gridDim.x;
            if (tn < n_tiles) issue(tn, s);
        }
        const int32_t k0 = t * TILE + CPT * tid;
        Vel u[CPT] = {};
        if (k0 < nf) {
            collide_cells<Q, St::scaled, OP_TRT, CPT, PACK>(g, p, u);
            const bool full = k0 + CPT <= nf;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                float f[CPT];
#pragma unroll
                for (int c = 0; c < CPT; ++c) f[c] = g[c][i];
                const Vec<T, CPT> y = RowIO<ST, CPT>::pack(f);
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
        if constexpr (BC) {
            if (b0 != b1) {                    // uniform across the block
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    us[CPT * tid + c] = u[c].x;
                    us[TILE + CPT * tid + c] = u[c].y;
                    us[2 * TILE + CPT * tid + c] = u[c].z;
                }
                __syncthreads();
                // the next write of us follows the next tile's barrier
                even_links_apply<ST>(pdf, S, t * TILE, b0, b1, us, TILE, lk, p.scale);
            }
        }
    }
    if (tid == 0 && ss.pending) drain_stages<NSTAGE>(bar, ss);
    __syncthreads();
}

}  // namespace slbm
