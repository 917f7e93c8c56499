// temporary: entry points not yet implemented
#include "internal.h"
namespace hsmm {
static __device__ uint32_t g_status_ring;
uint32_t status_take_ring() { uint32_t v = 0, z = 0; cudaMemcpyFromSymbol(&v, g_status_ring, 4); cudaMemcpyToSymbol(g_status_ring, &z, 4); return v; }
hsmm_status_t ring_gemm_f64(int, int, int64_t, const double*, int64_t, const double*, int64_t, double*, int64_t, cudaStream_t) { return HSMM_STATUS_NOT_SUPPORTED; }
hsmm_status_t gemm_ozaki_slices(int64_t, int64_t, int64_t, int64_t, int, int, const void*, const void*, const int32_t*, const int32_t*, double, double, double*, int64_t, double*, cudaStream_t) { return HSMM_STATUS_NOT_SUPPORTED; }
struct GroupedPlan { int dummy; };
hsmm_status_t grouped_plan_create(hsmm_dtype_t, hsmm_dtype_t, int64_t, const hsmm_gemm_desc_t*, int, GroupedPlan**) { return HSMM_STATUS_NOT_SUPPORTED; }
hsmm_status_t grouped_plan_launch(GroupedPlan*, float, float, cudaStream_t) { return HSMM_STATUS_NOT_SUPPORTED; }
hsmm_status_t grouped_plan_info(GroupedPlan*, int64_t*, int*) { return HSMM_STATUS_NOT_SUPPORTED; }
void grouped_plan_destroy(GroupedPlan*) {}
}
