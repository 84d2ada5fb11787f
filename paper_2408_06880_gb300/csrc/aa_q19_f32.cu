// aa_q19_f32.cu -- the AA launch paths and kernels of D3Q19 with FP32 storage
// (one translation unit per stencil and storage, so that they compile in parallel).
#include "aa_launch.cuh"
namespace slbm {
template cudaError_t launch_aa_storage<19, ST_F32>(const Domain &, int, cudaStream_t);
template cudaError_t launch_bc_pre<19, ST_F32>(const Domain &, cudaStream_t);
template cudaError_t launch_bc_post<19, ST_F32>(const Domain &, cudaStream_t);
}  // namespace slbm
