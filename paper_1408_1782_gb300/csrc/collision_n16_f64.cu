// Instantiation of the collision kernels for the 16 x 16 padded grid (N = 8), FP64 transforms.
#include "collision_vjp.cuh"

namespace qbe {
template cudaError_t collide_batch_n<16, double>(const Tables&, CollisionWork&, const double*, double*, int,
                                              cudaStream_t, long long&, KernelTimer*);
template int i3_blocks_per_sm<16, double>(int);
template int i3_variant_count<16, double>();
template int i3_default_variant<16, double>();
template int i3_variant_concurrency<16, double>(int, int, int);
template const char* i3_variant_name<16, double>(int);
template cudaError_t collide_vjp_n<16, double>(const Tables&, CollisionWork&, VjpWork&, const double*,
                                              const double* const*, double* const*, int, int, int, cudaStream_t,
                                              long long&, KernelTimer*);
template int i3_vjp_blocks_per_sm<16, double>();
template cudaError_t collide_pre_n<16, double>(const Tables&, CollisionWork&, const double*, int, cudaStream_t,
                                            long long&, KernelTimer*);
template cudaError_t collide_post_n<16, double>(const Tables&, CollisionWork&, double*, int, cudaStream_t, long long&,
                                             KernelTimer*);
template cudaError_t i3_group_n<16, double>(const Tables* const*, const CollisionWork* const*, const int*, int, void*,
                                         int, cudaStream_t, long long&, int);
}  // namespace qbe
