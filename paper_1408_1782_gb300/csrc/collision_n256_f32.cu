// Instantiation of the collision kernels for the 256 x 256 padded grid (N = 128), FP32 transforms.
#include "collision_kernels.cuh"

namespace qbe {
template cudaError_t collide_batch_n<256, float>(const Tables&, CollisionWork&, const double*, double*, int,
                                              cudaStream_t, long long&, KernelTimer*);
template int i3_blocks_per_sm<256, float>();
}  // namespace qbe
