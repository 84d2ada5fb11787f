// aa_dispatch.cu -- dispatch of an AA step and of the pool's boundary fix-ups
// by storage type; the launch paths and kernels are compiled per stencil and
// storage in aa_q19_*.cu and aa_q27_*.cu.
#include "common.cuh"
#include "internal.h"

namespace slbm {

template <int Q, int ST>
cudaError_t launch_aa_storage(const Domain &d, int parity, cudaStream_t st);
template <int Q, int ST>
cudaError_t launch_bc_pre(const Domain &d, cudaStream_t st);
template <int Q, int ST>
cudaError_t launch_bc_post(const Domain &d, cudaStream_t st);
extern template cudaError_t launch_aa_storage<19, ST_F32>(const Domain &, int, cudaStream_t);
extern template cudaError_t launch_bc_pre<19, ST_F32>(const Domain &, cudaStream_t);
extern template cudaError_t launch_bc_post<19, ST_F32>(const Domain &, cudaStream_t);
extern template cudaError_t launch_aa_storage<19, ST_F16>(const Domain &, int, cudaStream_t);
extern template cudaError_t launch_bc_pre<19, ST_F16>(const Domain &, cudaStream_t);
extern template cudaError_t launch_bc_post<19, ST_F16>(const Domain &, cudaStream_t);
extern template cudaError_t launch_aa_storage<19, ST_BF16>(const Domain &, int, cudaStream_t);
extern template cudaError_t launch_bc_pre<19, ST_BF16>(const Domain &, cudaStream_t);
extern template cudaError_t launch_bc_post<19, ST_BF16>(const Domain &, cudaStream_t);
extern template cudaError_t launch_aa_storage<27, ST_F32>(const Domain &, int, cudaStream_t);
extern template cudaError_t launch_bc_pre<27, ST_F32>(const Domain &, cudaStream_t);
extern template cudaError_t launch_bc_post<27, ST_F32>(const Domain &, cudaStream_t);
extern template cudaError_t launch_aa_storage<27, ST_F16>(const Domain &, int, cudaStream_t);
extern template cudaError_t launch_bc_pre<27, ST_F16>(const Domain &, cudaStream_t);
extern template cudaError_t launch_bc_post<27, ST_F16>(const Domain &, cudaStream_t);
extern template cudaError_t launch_aa_storage<27, ST_BF16>(const Domain &, int, cudaStream_t);
extern template cudaError_t launch_bc_pre<27, ST_BF16>(const Domain &, cudaStream_t);
extern template cudaError_t launch_bc_post<27, ST_BF16>(const Domain &, cudaStream_t);

// Fix-ups for the pool's even step (per member with links).
template <int Q>
cudaError_t launch_bc_fixup_q(const Domain &d, int post, cudaStream_t st) {
    switch (d.storage) {
        case SLBM_FP32: return post ? launch_bc_post<Q, ST_F32>(d, st) : launch_bc_pre<Q, ST_F32>(d, st);
        case SLBM_FP16: return post ? launch_bc_post<Q, ST_F16>(d, st) : launch_bc_pre<Q, ST_F16>(d, st);
        default: return post ? launch_bc_post<Q, ST_BF16>(d, st) : launch_bc_pre<Q, ST_BF16>(d, st);
    }
}

template <int Q>
cudaError_t launch_aa_step_q(const Domain &d, int parity, cudaStream_t st) {
    switch (d.storage) {
        case SLBM_FP32: return launch_aa_storage<Q, ST_F32>(d, parity, st);
        case SLBM_FP16: return launch_aa_storage<Q, ST_F16>(d, parity, st);
        case SLBM_BF16: return launch_aa_storage<Q, ST_BF16>(d, parity, st);
    }
    return cudaErrorInvalidValue;
}

template cudaError_t launch_aa_step_q<19>(const Domain &, int, cudaStream_t);
template cudaError_t launch_aa_step_q<27>(const Domain &, int, cudaStream_t);
template cudaError_t launch_bc_fixup_q<19>(const Domain &, int, cudaStream_t);
template cudaError_t launch_bc_fixup_q<27>(const Domain &, int, cudaStream_t);

}  // namespace slbm
