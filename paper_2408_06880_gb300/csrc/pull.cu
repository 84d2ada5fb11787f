// pull.cu -- the sparse two-grid pull step (Sec. 3.1 streaming by the pull
// index-list, Sec. 5.1's comparison scheme for the AA pattern): each cell
// gathers f_i from P(i,k) of the source grid, collides, and stores its
// post-collision populations in its own column of the destination grid.
//
// State convention.  At step 0 the current grid A holds the natural
// populations f(0).  Step 0 -> 1 collides in place (C(0) in A, row i); every
// later step t -> t+1 pulls C(t-1) from the current grid, collides and writes
// C(t) to the other grid.  The current grid is therefore A at t = 0 and at odd
// t, B at even t > 0 -- a function of t alone, so captured graphs stay valid.
// The natural populations at t > 0 are the pull of C(t-1): f_i(x_k, t) =
// C(t-1)[P(i,k)] (fluid neighbour: row i, column n; wall: row inverse(i),
// column k), which the macroscopic read-out gathers.  Bytes per cell update:
// Q B_pdf gathered + Q B_pdf written + (Q-1) index bytes (Table 2's pull row).
#include "aa_launch.cuh"

namespace slbm {

template <int Q, int ST, int OP>
__global__ void __launch_bounds__(256) pull_first_kernel(typename Store<ST>::T *__restrict__ a, int32_t S,
                                                         int32_t nf, CollideParams p) {
    using St = Store<ST>;
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nf) return;
    float g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = St::raw(a[i * S + k]);
    collide_op<Q, St::scaled, OP>(g, p);
#pragma unroll
    for (int i = 0; i < Q; ++i) a[i * S + k] = St::pack(g[i]);
}

// pf_dist > 0: thread 0 asks the bulk-copy engine to prefetch into L2 the
// index rows of the block pf_dist blocks ahead (about one residency wave).
template <int Q, int ST, int OP>
__global__ void __launch_bounds__(256) pull_step_kernel(const typename Store<ST>::T *__restrict__ src,
                                                        typename Store<ST>::T *__restrict__ dst,
                                                        const int32_t *__restrict__ P, int32_t S, int32_t nf,
                                                        CollideParams p, int32_t pf_dist) {
    using St = Store<ST>;
    if (pf_dist > 0 && threadIdx.x == 0) {
        const int64_t c0 = ((int64_t)blockIdx.x + pf_dist) * blockDim.x;
        if (c0 < nf) {
            const int64_t left = (int64_t)S - c0;
            const uint32_t cells = (uint32_t)(left < (int64_t)blockDim.x ? left : (int64_t)blockDim.x);
#pragma unroll
            for (int r = 0; r < Q - 1; ++r) bulk_prefetch_l2(P + r * S + c0, cells * 4u);
        }
    }
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nf) return;
    int32_t e[Q];
#pragma unroll
    for (int i = 1; i < Q; ++i) e[i] = __ldcs(P + (i - 1) * S + k);   // streaming: measured faster here
    float g[Q];
    g[0] = St::raw(src[k]);
#pragma unroll
    for (int i = 1; i < Q; ++i) g[i] = St::raw(src[e[i]]);
    collide_op<Q, St::scaled, OP>(g, p);
#pragma unroll
    for (int i = 0; i < Q; ++i) dst[i * S + k] = St::pack(g[i]);
}

template <int Q, int ST, int OP>
static cudaError_t launch_pull_op(const Domain &d, int64_t t, cudaStream_t st) {
    using T = typename Store<ST>::T;
    const int32_t S = (int32_t)d.S, nf = (int32_t)d.n_fluid;
    if (nf == 0) return cudaSuccess;
    const CollideParams p = d.collide_params();
    constexpr int TH = 128;
    const unsigned grid = (unsigned)((nf + TH - 1) / TH);
    T *a = reinterpret_cast<T *>(d.pdf.p), *b = reinterpret_cast<T *>(d.pdf2.p);
    if (t == 0) {
        pull_first_kernel<Q, ST, OP><<<grid, TH, 0, st>>>(a, S, nf, p);
        return cudaGetLastError();
    }
    // C(t-1) sits in A at odd t, in B at even t
    const bool from_a = t & 1;
    auto k = pull_step_kernel<Q, ST, OP>;
    const int32_t pf = (int32_t)persistent_grid(k, TH, INT32_MAX);
    k<<<grid, TH, 0, st>>>(from_a ? a : b, from_a ? b : a, reinterpret_cast<const int32_t *>(d.P.p), S, nf, p, pf);
    return cudaGetLastError();
}

template <int Q, int ST>
static cudaError_t launch_pull_st(const Domain &d, int64_t t, cudaStream_t st) {
    if constexpr (Q == 19) {
        if (d.op == SLBM_MRT) return launch_pull_op<Q, ST, OP_MRT>(d, t, st);
    }
    if constexpr (Q == 27) {
        if (d.op == SLBM_CM) return launch_pull_op<Q, ST, OP_CM>(d, t, st);
        if (d.op == SLBM_CUMULANT) return launch_pull_op<Q, ST, OP_CUM>(d, t, st);
    }
    return launch_pull_op<Q, ST, OP_TRT>(d, t, st);
}

template <int Q>
static cudaError_t launch_pull_q(const Domain &d, int64_t t, cudaStream_t st) {
    switch (d.storage) {
        case SLBM_FP32: return launch_pull_st<Q, ST_F32>(d, t, st);
        case SLBM_FP16: return launch_pull_st<Q, ST_F16>(d, t, st);
        default: return launch_pull_st<Q, ST_BF16>(d, t, st);
    }
}

// Step t -> t+1 (t = the absolute step index, d.step + the launch's offset).
cudaError_t launch_pull_step(const Domain &d, int64_t t, cudaStream_t st) {
    return d.q == 19 ? launch_pull_q<19>(d, t, st) : launch_pull_q<27>(d, t, st);
}

}  // namespace slbm
