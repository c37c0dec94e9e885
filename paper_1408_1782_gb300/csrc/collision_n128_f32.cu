// Instantiation of the collision kernels for the 128 x 128 padded grid (N = 64), FP32 transforms.
#include "collision_vjp.cuh"

namespace qbe {
template cudaError_t collide_batch_n<128, float>(const Tables&, CollisionWork&, const double*, double*, int,
                                              cudaStream_t, long long&, KernelTimer*);
template int i3_blocks_per_sm<128, float>(int);
template int i3_variant_count<128, float>();
template int i3_default_variant<128, float>();
template int i3_variant_concurrency<128, float>(int, int, int);
template const char* i3_variant_name<128, float>(int);
template cudaError_t collide_vjp_n<128, float>(const Tables&, CollisionWork&, VjpWork&, const double*,
                                              const double* const*, double* const*, int, int, int, cudaStream_t,
                                              long long&, KernelTimer*);
template int i3_vjp_blocks_per_sm<128, float>();
template cudaError_t collide_pre_n<128, float>(const Tables&, CollisionWork&, const double*, int, cudaStream_t,
                                            long long&, KernelTimer*);
template cudaError_t collide_post_n<128, float>(const Tables&, CollisionWork&, double*, int, cudaStream_t, long long&,
                                             KernelTimer*);
template cudaError_t i3_group_n<128, float>(const Tables* const*, const CollisionWork* const*, const int*, int, void*,
                                         int, cudaStream_t, long long&, int);
}  // namespace qbe
