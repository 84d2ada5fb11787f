// macro.cu -- macroscopic fields (Eq. 1 with the Guo half-force velocity), the
// deterministic FP64 domain sums, and equilibrium initialisation (Eq. 6).
//
// The state is read at either AA parity: after an even number of steps the
// field is natural (row i of column k); after an odd number the populations
// of cell k sit in the odd-step slots R(i,k) that the device index-list holds,
// so reading them is the gather half of the odd kernel.
//
// The sums are deterministic: cells are cut into fixed chunks of RED_CHUNK
// cells (independent of the device and the launch shape), each chunk is summed
// in a fixed order into FP64 partials, and one block adds the partials in a
// fixed order.  A domain therefore gives the same bits alone or in a pool.
#include "internal.h"
#include "reduce.cuh"

namespace slbm {

// --------------------------------------------------------------- layouts
struct SparseView {
    const int32_t *P;
    const LinkMap *maps;
    const int32_t *cell_voxel;
    int32_t S, n;             // n = cells
    __device__ __forceinline__ bool fluid(int32_t) const { return true; }
    __device__ __forceinline__ int32_t voxel(int32_t k) const { return cell_voxel[k]; }
    template <int Q, class St>
    __device__ __forceinline__ void load(const typename St::T *pdf, int32_t k, bool odd, float inv_scale,
                                         float (&g)[Q]) const {
        g[0] = St::ld(pdf[k], inv_scale);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            if (!odd) {
                g[i] = St::ld(pdf[i * S + k], inv_scale);
            } else {
                const int32_t e = P[(i - 1) * S + k];
                const int32_t r = e >= 0 ? e : i * S + k;   // link slots already hold mapped values
                g[i] = St::ld(pdf[r], inv_scale);
            }
        }
    }
};

// Pull layout: at t > 0 the stored grid holds the post-collision C(t-1), and
// the natural populations are its pull through the canonical entries,
// f_i(k) = C[P(i,k)] (no inlet/outlet links in this layout); at t = 0 the
// grid is natural.
struct PullView {
    const int32_t *P;
    const int32_t *cell_voxel;
    int32_t S, n;
    __device__ __forceinline__ bool fluid(int32_t) const { return true; }
    __device__ __forceinline__ int32_t voxel(int32_t k) const { return cell_voxel[k]; }
    template <int Q, class St>
    __device__ __forceinline__ void load(const typename St::T *pdf, int32_t k, bool pulled, float inv_scale,
                                         float (&g)[Q]) const {
        g[0] = St::ld(pdf[k], inv_scale);
#pragma unroll
        for (int i = 1; i < Q; ++i) g[i] = St::ld(pdf[pulled ? P[(i - 1) * S + k] : i * S + k], inv_scale);
    }
};

// Dense comparator layout: every voxel is a column; the per-voxel mask holds
// bit 31 = fluid and bit i = "pull neighbour of direction i is a wall".
struct DenseView {
    const uint32_t *mask;
    int64_t S;
    int32_t n, nx, ny, nz;
    __device__ __forceinline__ bool fluid(int32_t v) const { return mask[v] >> 31; }
    __device__ __forceinline__ int32_t voxel(int32_t v) const { return v; }
    template <int Q, class St>
    __device__ __forceinline__ void load(const typename St::T *pdf, int32_t v, bool odd, float inv_scale,
                                         float (&g)[Q]) const {
        const uint32_t m = mask[v];
        const int x = v % nx, y = (v / nx) % ny, z = v / (nx * ny);
        g[0] = St::ld(pdf[v], inv_scale);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            int64_t r;
            if (!odd) {
                r = i * S + v;
            } else if (m >> i & 1u) {
                r = i * S + v;
            } else {
                const int xn = (x - cx(i) + nx) % nx, yn = (y - cy(i) + ny) % ny, zn = (z - cz(i) + nz) % nz;
                r = inv(i) * S + xn + nx * (yn + ny * zn);
            }
            g[i] = St::ld(pdf[r], inv_scale);
        }
    }
};

// ------------------------------------------------------------ kernels
// Largest of two values, NaN if either is NaN (fmaxf would drop it).
__device__ __forceinline__ float nan_max(float a, float b) {
    return a != a ? a : (b != b ? b : fmaxf(a, b));
}

// Maximum over the block of two floats (exact, so independent of the order;
// a NaN wins); thread 0 writes them to out[0..1].
__device__ __forceinline__ void block_max2_to(float a, float b, float *out) {
    __shared__ float sm[32][2];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a = nan_max(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = nan_max(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sm[warp][0] = a;
        sm[warp][1] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            a = nan_max(a, sm[w][0]);
            b = nan_max(b, sm[w][1]);
        }
        out[0] = a;
        out[1] = b;
    }
}

// One block per chunk of RED_CHUNK cells; thread t takes cells
// chunk*RED_CHUNK + j*RED_THREADS + t, j = 0..RED_CELLS_PER_THREAD-1, in
// that order.  Writes optional fields and the chunk's five FP64 partials;
// with `maxes`, also the chunk's largest |f_i - w_i| over the populations it
// read (unscaled) and largest speed |u| (a NaN anywhere makes them NaN).
template <int Q, class St, class View>
__global__ void __launch_bounds__(RED_THREADS) macro_reduce_kernel(const typename St::T *pdf, View view,
                                                                   bool odd, CollideParams p, float *rho_out,
                                                                   float *u_out, int64_t u_stride, int order,
                                                                   double *partial, float *maxes = nullptr) {
    double acc[5] = {0, 0, 0, 0, 0};
    float gmax = 0.f, umax = 0.f;
    const int32_t base = blockIdx.x * RED_CHUNK + threadIdx.x;
#pragma unroll 1
    for (int j = 0; j < RED_CELLS_PER_THREAD; ++j) {
        const int32_t k = base + j * RED_THREADS;
        if (k >= view.n || !view.fluid(k)) continue;
        float g[Q];
        view.template load<Q, St>(pdf, k, odd, p.inv_scale, g);
        float drho, jx, jy, jz;
        moments<Q>(g, drho, jx, jy, jz);
        const float rho = 1.0f + drho;
        const float mx = jx + 0.5f * p.fx, my = jy + 0.5f * p.fy, mz = jz + 0.5f * p.fz;
        const float ux = mx / rho, uy = my / rho, uz = mz / rho;
        acc[0] += (double)drho;
        acc[1] += (double)mx;
        acc[2] += (double)my;
        acc[3] += (double)mz;
        acc[4] += (double)ux;
        if (maxes) {
#pragma unroll
            for (int i = 0; i < Q; ++i) gmax = nan_max(gmax, fabsf(g[i]));
            umax = nan_max(umax, sqrtf(ux * ux + uy * uy + uz * uz));
        }
        const int64_t o = order == SLBM_ORDER_VOXELS ? (int64_t)view.voxel(k) : (int64_t)k;
        if (rho_out) rho_out[o] = rho;
        if (u_out) {
            u_out[o] = ux;
            u_out[o + u_stride] = uy;
            u_out[o + 2 * u_stride] = uz;
        }
    }
    if (partial) block_sum5_to(acc, partial + (int64_t)blockIdx.x * 5);
    if (maxes) block_max2_to(gmax, umax, maxes + 2 * (int64_t)blockIdx.x);
}

// One block: out[c] = max over chunks of maxes[2*chunk + c], c = 0, 1 (NaN
// if any is NaN), as doubles.
__global__ void reduce_max_partials_kernel(const float *maxes, int64_t chunks, double *out) {
    float a = 0.f, b = 0.f;
    for (int64_t j = threadIdx.x; j < chunks; j += blockDim.x) {
        a = nan_max(a, maxes[2 * j]);
        b = nan_max(b, maxes[2 * j + 1]);
    }
    __shared__ float r[2];
    block_max2_to(a, b, r);
    __syncthreads();
    if (threadIdx.x == 0) {
        out[0] = (double)r[0];
        out[1] = (double)r[1];
    }
}

template <int Q, class St, class View>
__global__ void init_eq_kernel(typename St::T *pdf, View view, const float *rho, const float *u, int64_t u_stride,
                               int order, float scale) {
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= view.n || !view.fluid(k)) return;
    const int64_t o = order == SLBM_ORDER_VOXELS ? (int64_t)view.voxel(k) : (int64_t)k;
    const float r = rho ? rho[o] : 1.0f;
    const float ux = u ? u[o] : 0.f, uy = u ? u[o + u_stride] : 0.f, uz = u ? u[o + 2 * u_stride] : 0.f;
    float g[Q];
    equilibrium_shifted<Q>(r, ux, uy, uz, g);
#pragma unroll
    for (int i = 0; i < Q; ++i) pdf[(int64_t)i * view.S + k] = St::st(g[i], scale);
}

// ------------------------------------------------------------- dispatch
template <class Fn>
static cudaError_t with_types(const Domain &d, Fn &&fn) {
    auto by_view = [&](auto qtag, auto sttag) -> cudaError_t {
        constexpr int Q = decltype(qtag)::value;
        using St = Store<decltype(sttag)::value>;
        if (d.pull()) {
            PullView v{(const int32_t *)d.P.p, (const int32_t *)d.cell_voxel.p, (int32_t)d.S, (int32_t)d.n_fluid};
            return fn(std::integral_constant<int, Q>{}, St{}, v);
        }
        if (d.layout == SLBM_LAYOUT_SPARSE) {
            SparseView v{(const int32_t *)d.P.p, (const LinkMap *)d.link_map.p, (const int32_t *)d.cell_voxel.p,
                         (int32_t)d.S, (int32_t)d.n_fluid};
            return fn(std::integral_constant<int, Q>{}, St{}, v);
        }
        DenseView v{(const uint32_t *)d.mask.p, d.S, (int32_t)d.n_vox, d.nx, d.ny, d.nz};
        return fn(std::integral_constant<int, Q>{}, St{}, v);
    };
    auto by_st = [&](auto qtag) -> cudaError_t {
        switch (d.storage) {
            case SLBM_FP32: return by_view(qtag, std::integral_constant<int, ST_F32>{});
            case SLBM_FP16: return by_view(qtag, std::integral_constant<int, ST_F16>{});
            default: return by_view(qtag, std::integral_constant<int, ST_BF16>{});
        }
    };
    return d.q == 19 ? by_st(std::integral_constant<int, 19>{}) : by_st(std::integral_constant<int, 27>{});
}

int64_t Domain::red_chunks() const {
    const int64_t n = sparse() ? n_fluid : n_vox;
    return (n + RED_CHUNK - 1) / RED_CHUNK;
}

cudaError_t launch_macroscopic(const Domain &d, float *rho, float *u, int order, cudaStream_t st) {
    const int64_t chunks = d.red_chunks();
    if (chunks == 0) return cudaSuccess;
    const int64_t u_stride = order == SLBM_ORDER_VOXELS ? d.n_vox
                                                        : (d.sparse() ? d.n_fluid : d.n_vox);
    const bool odd = d.pull() ? d.step > 0 : (d.step & 1);
    const CollideParams p = d.collide_params();
    return with_types(d, [&](auto qtag, auto st_t, auto view) -> cudaError_t {
        constexpr int Q = decltype(qtag)::value;
        using St = decltype(st_t);
        macro_reduce_kernel<Q, St><<<(unsigned)chunks, RED_THREADS, 0, st>>>(
            (const typename St::T *)d.cur_pdf(), view, odd, p, rho, u, u_stride, order, nullptr);
        return cudaGetLastError();
    });
}

cudaError_t launch_reduce(const Domain &d, double *out_dev, cudaStream_t st) {
    const int64_t chunks = d.red_chunks();
    if (chunks == 0) return cudaMemsetAsync(out_dev, 0, 5 * sizeof(double), st);
    const bool odd = d.pull() ? d.step > 0 : (d.step & 1);
    const CollideParams p = d.collide_params();
    cudaError_t e = with_types(d, [&](auto qtag, auto st_t, auto view) -> cudaError_t {
        constexpr int Q = decltype(qtag)::value;
        using St = decltype(st_t);
        macro_reduce_kernel<Q, St><<<(unsigned)chunks, RED_THREADS, 0, st>>>(
            (const typename St::T *)d.cur_pdf(), view, odd, p, nullptr, nullptr, 0, 0, (double *)d.red_partial.p);
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
    reduce_partials_kernel<<<1, RED_THREADS, 0, st>>>((const double *)d.red_partial.p, chunks, out_dev);
    return cudaGetLastError();
}

// The five sums into out_dev[0..4] (the same bits as launch_reduce) and the
// two maxima into out_dev[5..6].  The chunk maxima sit behind the sums'
// partials in red_partial.
cudaError_t launch_reduce_ext(const Domain &d, double *out_dev, cudaStream_t st) {
    const int64_t chunks = d.red_chunks();
    if (chunks == 0) return cudaMemsetAsync(out_dev, 0, 7 * sizeof(double), st);
    const bool odd = d.pull() ? d.step > 0 : (d.step & 1);
    const CollideParams p = d.collide_params();
    double *partial = (double *)d.red_partial.p;
    float *maxes = (float *)(partial + 5 * chunks);
    cudaError_t e = with_types(d, [&](auto qtag, auto st_t, auto view) -> cudaError_t {
        constexpr int Q = decltype(qtag)::value;
        using St = decltype(st_t);
        macro_reduce_kernel<Q, St><<<(unsigned)chunks, RED_THREADS, 0, st>>>(
            (const typename St::T *)d.cur_pdf(), view, odd, p, nullptr, nullptr, 0, 0, partial, maxes);
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
    reduce_partials_kernel<<<1, RED_THREADS, 0, st>>>(partial, chunks, out_dev);
    reduce_max_partials_kernel<<<1, RED_THREADS, 0, st>>>(maxes, chunks, out_dev + 5);
    return cudaGetLastError();
}

cudaError_t launch_init_equilibrium(const Domain &d, const float *rho, const float *u, int order,
                                    cudaStream_t st) {
    const int64_t n = d.sparse() ? d.n_fluid : d.n_vox;
    if (n == 0) return cudaSuccess;
    const int64_t u_stride = order == SLBM_ORDER_VOXELS ? d.n_vox : n;
    const float scale = d.collide_params().scale;
    return with_types(d, [&](auto qtag, auto st_t, auto view) -> cudaError_t {
        constexpr int Q = decltype(qtag)::value;
        using St = decltype(st_t);
        init_eq_kernel<Q, St><<<(unsigned)((n + 255) / 256), 256, 0, st>>>((typename St::T *)d.pdf.p, view, rho, u,
                                                                          u_stride, order, scale);
        return cudaGetLastError();
    });
}

}  // namespace slbm

namespace slbm {
__global__ void reduce_partials_kernel(const double *partial, int64_t chunks, double *out) {
    double acc[5] = {0, 0, 0, 0, 0};
    for (int64_t b = threadIdx.x; b < chunks; b += blockDim.x) {
#pragma unroll
        for (int c = 0; c < 5; ++c) acc[c] += partial[b * 5 + c];
    }
    block_sum5_to(acc, out);
}
}  // namespace slbm
