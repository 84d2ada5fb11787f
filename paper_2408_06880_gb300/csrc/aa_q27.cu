// aa_q27.cu -- D3Q27 instantiation of the AA stream-collide kernels.
#include "aa_launch.cuh"
namespace slbm {
template cudaError_t launch_aa_step_q<27>(const Domain &, int, cudaStream_t);
template cudaError_t launch_bc_fixup_q<27>(const Domain &, int, cudaStream_t);
}
