// Read-bandwidth probe: the denominator of the walk kernels' roofline.
//
// The walk kernels read node and primitive records of scenes that stay
// resident in L2 (hundreds of kB to tens of MB), so their bandwidth ceiling
// is the L2's, not HBM's.  This kernel streams a caller buffer with 16-byte
// loads that bypass L1 (ld.global.cg), several independent loads in flight
// per thread, over `passes` sweeps: with a buffer well below the L2 size the
// sweeps after the first hit L2, with one well above it they measure HBM.
// The caller times the launch (it allocates nothing and synchronises
// nothing).
#include <cuda_runtime.h>

#include <algorithm>

#include "capi_internal.h"

namespace wost {

__global__ void __launch_bounds__(256) k_read_probe(const float4 *__restrict__ buf, int64_t n4, int passes,
                                                    float *sink) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int p = 0; p < passes; ++p) {
        int64_t i = tid;
        // four independent loads per iteration keep enough bytes in flight
        for (; i + 3 * stride < n4; i += 4 * stride) {
            float4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride), c = __ldcg(buf + i + 2 * stride),
                   d = __ldcg(buf + i + 3 * stride);
            acc.x += a.x + b.x + c.x + d.x;
            acc.y += a.y + b.y + c.y + d.y;
            acc.z += a.z + b.z + c.z + d.z;
            acc.w += a.w + b.w + c.w + d.w;
        }
        for (; i < n4; i += stride) {
            float4 a = __ldcg(buf + i);
            acc.x += a.x;
            acc.y += a.y;
            acc.z += a.z;
            acc.w += a.w;
        }
    }
    // one store per thread, only if the sum is a value no buffer of finite
    // floats below 1e30 produces: the loads cannot be optimised away
    float s = acc.x + acc.y + acc.z + acc.w;
    if (s == 1.2345e38f) sink[0] = s;
}

}  // namespace wost

using namespace wost;

extern "C" wost_status wost_read_probe(const void *buf, int64_t bytes, int32_t passes, float *sink, void *stream) {
    if (!buf || !sink) return fail(WOST_ERR_INVALID_ARG, "null buffer");
    if (bytes < 16 || bytes % 16 || ((uintptr_t)buf & 15u))
        return fail(WOST_ERR_INVALID_ARG, "buffer must be 16-byte aligned and a positive multiple of 16 bytes");
    if (passes < 1) return fail(WOST_ERR_INVALID_ARG, "passes must be >= 1");
    int dev = 0, sms = 0, per_sm = 0;
    CK(cudaGetDevice(&dev), "cudaGetDevice");
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_read_probe, 256, 0), "occupancy");
    const int64_t n4 = bytes / 16;
    int64_t blocks = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    blocks = std::min<int64_t>(blocks, (n4 + 255) / 256);
    k_read_probe<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>((const float4 *)buf, n4, passes, sink);
    CK(cudaGetLastError(), "kernel launch");
    return WOST_OK;
}
