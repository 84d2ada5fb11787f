// aa_q27_bf16.cu -- the AA launch paths and kernels of D3Q27 with BF16 storage
// (one translation unit per stencil and storage, so that they compile in parallel).
#include "aa_launch.cuh"
namespace slbm {
template cudaError_t launch_aa_storage<27, ST_BF16>(const Domain &, int, cudaStream_t);
template cudaError_t launch_bc_pre<27, ST_BF16>(const Domain &, cudaStream_t);
template cudaError_t launch_bc_post<27, ST_BF16>(const Domain &, cudaStream_t);
}  // namespace slbm
