// aa_q19.cu -- D3Q19 instantiation of the AA stream-collide kernels.
#include "aa_launch.cuh"
namespace slbm {
template cudaError_t launch_aa_step_q<19>(const Domain &, int, cudaStream_t);
template cudaError_t launch_bc_fixup_q<19>(const Domain &, int, cudaStream_t);
}
