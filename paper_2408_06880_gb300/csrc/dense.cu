// dense.cu -- the dense direct-addressing comparator (Sec. 3, Sec. 4 single
// node results): the same AA update over every voxel of the box, neighbours by
// index arithmetic with periodic wrap, solids skipped after one mask read.
//
// Layout: Q rows of S = round_up(N, 128) stored populations, column = voxel
// id.  A per-voxel 32-bit mask carries bit 31 = fluid and bit i = "the pull
// neighbour x - c_i is a wall (or outside a non-periodic face)".  Inlet and
// outlet voxels are not supported by this comparator.
#include <type_traits>

#include "aa_kernels.cuh"
#include "internal.h"

namespace slbm {

template <int Q>
__global__ void dense_mask_kernel(const uint8_t *flags, int32_t nx, int32_t ny, int32_t nz, uint32_t periodic,
                                  uint32_t *mask) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= nx) return;
    const int64_t v = (int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z);
    if (flags[v] != FLAG_FLUID) {
        mask[v] = 0u;
        return;
    }
    uint32_t m = 1u << 31;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        int xn = x - cx(i), yn = y - cy(i), zn = z - cz(i);
        bool wall = false;
        if (xn < 0 || xn >= nx) {
            if (periodic & 1u) xn = (xn + nx) % nx;
            else wall = true;
        }
        if (yn < 0 || yn >= ny) {
            if (periodic & 2u) yn = (yn + ny) % ny;
            else wall = true;
        }
        if (zn < 0 || zn >= nz) {
            if (periodic & 4u) zn = (zn + nz) % nz;
            else wall = true;
        }
        if (!wall) wall = flags[(int64_t)xn + (int64_t)nx * ((int64_t)yn + (int64_t)ny * zn)] != FLAG_FLUID;
        if (wall) m |= 1u << i;
    }
    mask[v] = m;
}

// Slot arithmetic in 32 bits unless Q * S reaches 2^31 (WIDE).
template <bool WIDE>
using SlotT = typename std::conditional<WIDE, int64_t, int32_t>::type;

// Even step, two consecutive voxels per thread with vector loads and stores.
// A pair with at least one fluid voxel is updated whole: the solid voxel's
// slots are never read by a fluid neighbour (its mask bits send the
// neighbour to its own slots) nor by the read-outs, so writing them is
// harmless and keeps the accesses vectorised.
template <int Q, int ST, bool WIDE>
__global__ void __launch_bounds__(128) dense_even_kernel(typename Store<ST>::T *__restrict__ pdf,
                                                         const uint32_t *__restrict__ mask, int64_t S, int32_t n,
                                                         CollideParams p) {
    using St = Store<ST>;
    using T = typename St::T;
    using I = SlotT<WIDE>;
    const int32_t v0 = (blockIdx.x * blockDim.x + threadIdx.x) * 2;
    if (v0 >= n) return;
    const bool two = v0 + 1 < n;
    const uint32_t m0 = mask[v0], m1 = two ? mask[v0 + 1] : 0u;
    if (!((m0 | m1) >> 31)) return;
    const I s = (I)S;
    float g[2][Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float f[2];
        if (two) {
            RowIO<ST, 2>::load_ro(pdf + (I)i * s + v0, f);
        } else {
            f[0] = St::raw(pdf[(I)i * s + v0]);
            f[1] = 0.f;
        }
        g[0][i] = f[0];
        g[1][i] = f[1];
    }
    collide<Q, St::scaled>(g[0], p);
    collide<Q, St::scaled>(g[1], p);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        T *dst = pdf + (I)inv(i) * s + v0;
        if (two) {
            const float f[2] = {g[0][i], g[1][i]};
            st_vec<T, 2>(dst, RowIO<ST, 2>::pack(f));
        } else {
            dst[0] = St::pack(g[0][i]);
        }
    }
}

// grid (ceil(nx/blockDim), ny, nz): no divisions to find the coordinates.
template <int Q, int ST, bool WIDE>
__global__ void __launch_bounds__(128) dense_odd_kernel(typename Store<ST>::T *__restrict__ pdf,
                                                        const uint32_t *__restrict__ mask, int64_t S, int32_t nx,
                                                        int32_t ny, int32_t nz, CollideParams p) {
    using St = Store<ST>;
    using I = SlotT<WIDE>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= nx) return;
    const int32_t v = x + nx * (y + ny * z);
    const uint32_t m = mask[v];
    if (!(m >> 31)) return;
    const I s = (I)S;
    // rows away from the y and z faces (uniform over the block): the pull
    // neighbour is v minus a per-direction offset, wrapped only in x
    const bool interior = y > 0 && y < ny - 1 && z > 0 && z < nz - 1;
    const int32_t nxy = nx * ny;
    I R[Q];
    float g[Q];
    g[0] = St::raw(__ldg(pdf + v));
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (m >> i & 1u) {
            R[i] = (I)i * s + v;
        } else if (interior) {
            int32_t n = v - cx(i);
            if (cy(i) > 0) n -= nx;
            if (cy(i) < 0) n += nx;
            if (cz(i) > 0) n -= nxy;
            if (cz(i) < 0) n += nxy;
            if (cx(i) > 0 && x == 0) n += nx;
            if (cx(i) < 0 && x == nx - 1) n -= nx;
            R[i] = (I)inv(i) * s + (I)n;
        } else {
            int xn = x - cx(i), yn = y - cy(i), zn = z - cz(i);
            xn = xn < 0 ? xn + nx : (xn >= nx ? xn - nx : xn);
            yn = yn < 0 ? yn + ny : (yn >= ny ? yn - ny : yn);
            zn = zn < 0 ? zn + nz : (zn >= nz ? zn - nz : zn);
            R[i] = (I)inv(i) * s + (I)(xn + nx * (yn + ny * zn));
        }
        g[i] = St::raw(__ldg(pdf + R[i]));
    }
    collide<Q, St::scaled>(g, p);
    pdf[v] = St::pack(g[0]);
#pragma unroll
    for (int i = 1; i < Q; ++i) pdf[R[i]] = St::pack(g[inv(i)]);
}

int build_dense_mask(Ctx &cx, Domain &d, const uint8_t *d_flags) {
    if (cx.alloc(d.mask, std::max<int64_t>(d.n_vox, 1) * sizeof(uint32_t))) return -1;
    const dim3 grid((unsigned)((d.nx + 127) / 128), (unsigned)d.ny, (unsigned)d.nz);
    if (d.q == 19)
        dense_mask_kernel<19><<<grid, 128, 0, cx.stream>>>(d_flags, d.nx, d.ny, d.nz, d.periodic, (uint32_t *)d.mask.p);
    else
        dense_mask_kernel<27><<<grid, 128, 0, cx.stream>>>(d_flags, d.nx, d.ny, d.nz, d.periodic, (uint32_t *)d.mask.p);
    return cx.check(cudaGetLastError(), "dense mask");
}

template <int Q, int ST>
static cudaError_t dense_step_t(const Domain &d, int parity, cudaStream_t st) {
    using T = typename Store<ST>::T;
    const CollideParams p = d.collide_params();
    T *pdf = (T *)d.pdf.p;
    const uint32_t *mask = (const uint32_t *)d.mask.p;
    const bool wide = (int64_t)Q * d.S >= ((int64_t)1 << 31);
    if (parity == 0) {
        const unsigned grid = (unsigned)((d.n_vox + 255) / 256);
        if (wide) dense_even_kernel<Q, ST, true><<<grid, 128, 0, st>>>(pdf, mask, d.S, (int32_t)d.n_vox, p);
        else dense_even_kernel<Q, ST, false><<<grid, 128, 0, st>>>(pdf, mask, d.S, (int32_t)d.n_vox, p);
    } else {
        const dim3 grid((unsigned)((d.nx + 127) / 128), (unsigned)d.ny, (unsigned)d.nz);
        if (wide) dense_odd_kernel<Q, ST, true><<<grid, 128, 0, st>>>(pdf, mask, d.S, d.nx, d.ny, d.nz, p);
        else dense_odd_kernel<Q, ST, false><<<grid, 128, 0, st>>>(pdf, mask, d.S, d.nx, d.ny, d.nz, p);
    }
    return cudaGetLastError();
}

cudaError_t launch_dense_step(const Domain &d, int parity, cudaStream_t st) {
    if (d.n_vox == 0) return cudaSuccess;
    if (d.q == 19) {
        switch (d.storage) {
            case SLBM_FP32: return dense_step_t<19, ST_F32>(d, parity, st);
            case SLBM_FP16: return dense_step_t<19, ST_F16>(d, parity, st);
            default: return dense_step_t<19, ST_BF16>(d, parity, st);
        }
    }
    switch (d.storage) {
        case SLBM_FP32: return dense_step_t<27, ST_F32>(d, parity, st);
        case SLBM_FP16: return dense_step_t<27, ST_F16>(d, parity, st);
        default: return dense_step_t<27, ST_BF16>(d, parity, st);
    }
}

}  // namespace slbm
