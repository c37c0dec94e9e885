// Instantiation of the collision kernels for the 192 x 192 padded grid (N = 96), FP64 transforms.
#include "collision_vjp.cuh"

namespace qbe {
template cudaError_t collide_batch_n<192, double>(const Tables&, CollisionWork&, const double*, double*, int,
                                              cudaStream_t, long long&, KernelTimer*);
template int i3_blocks_per_sm<192, double>(int);
template int i3_variant_count<192, double>();
template int i3_default_variant<192, double>();
template int i3_variant_concurrency<192, double>(int, int, int);
template const char* i3_variant_name<192, double>(int);
template cudaError_t collide_vjp_n<192, double>(const Tables&, CollisionWork&, VjpWork&, const double*,
                                              const double* const*, double* const*, int, int, int, cudaStream_t,
                                              long long&, KernelTimer*);
template int i3_vjp_blocks_per_sm<192, double>();
template cudaError_t collide_pre_n<192, double>(const Tables&, CollisionWork&, const double*, int, cudaStream_t,
                                            long long&, KernelTimer*);
template cudaError_t collide_post_n<192, double>(const Tables&, CollisionWork&, double*, int, cudaStream_t, long long&,
                                             KernelTimer*);
template cudaError_t i3_group_n<192, double>(const Tables* const*, const CollisionWork* const*, const int*, int, void*,
                                         int, cudaStream_t, long long&, int);
}  // namespace qbe
