// Instantiation of the collision kernels for the 256 x 256 padded grid (N = 128), FP32 transforms.
#include "collision_vjp.cuh"

namespace qbe {
template cudaError_t collide_batch_n<256, float>(const Tables&, CollisionWork&, const double*, double*, int,
                                              cudaStream_t, long long&, KernelTimer*);
template int i3_blocks_per_sm<256, float>(int);
template int i3_variant_count<256, float>();
template int i3_default_variant<256, float>();
template int i3_variant_concurrency<256, float>(int, int, int);
template const char* i3_variant_name<256, float>(int);
template cudaError_t collide_vjp_n<256, float>(const Tables&, CollisionWork&, VjpWork&, const double*,
                                              const double* const*, double* const*, int, int, int, cudaStream_t,
                                              long long&, KernelTimer*);
template int i3_vjp_blocks_per_sm<256, float>();
template cudaError_t collide_pre_n<256, float>(const Tables&, CollisionWork&, const double*, int, cudaStream_t,
                                            long long&, KernelTimer*);
template cudaError_t collide_post_n<256, float>(const Tables&, CollisionWork&, double*, int, cudaStream_t, long long&,
                                             KernelTimer*);
template cudaError_t i3_group_n<256, float>(const Tables* const*, const CollisionWork* const*, const int*, int, void*,
                                         int, cudaStream_t, long long&, int);
}  // namespace qbe
