// Masked Adam on the active set (Supp. "3DGS Optimization in Changed
// Regions"): only rows listed in a scene's active_idx are read or written, so
// neither the parameters nor the Adam moments of the frozen Gaussians move.
#include "common.cuh"

namespace cls {

// b^t for t >= 0 by repeated squaring in double (at most 2 x 31 multiplies; a
// general double pow is a long dependent chain of slow double operations).
__device__ __forceinline__ double pow_uint(double b, int t) {
    double r = 1.0;
    while (t > 0) {
        if (t & 1) r *= b;
        b *= b;
        t >>= 1;
    }
    return r;
}

// t += 1 per scene, then the bias corrections 1 - b1^t and 1 - b2^t.
__global__ void adam_advance_kernel(const ClsScene* __restrict__ scenes, int n_scenes, float b1,
                                    float b2, float2* __restrict__ bias) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_scenes) return;
    if (scenes[s].n_active <= 0) return;  // nothing to update: the step count stays
    int32_t* step = scenes[s].adam_step;
    const int t = *step + 1;
    *step = t;
    bias[s] = make_float2((float)(1.0 - pow_uint((double)b1, t)),
                          (float)(1.0 - pow_uint((double)b2, t)));
}

// One thread per float4 of an active row.
__global__ void __launch_bounds__(256)
adam_active_kernel(const ClsScene* __restrict__ scenes, const float* __restrict__ grads,
                   const float2* __restrict__ bias, float lr, float b1, float b2, float eps) {
    const ClsScene& sc = scenes[blockIdx.y];
    const int q = sc.row_stride / 4;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)sc.n_active * q) return;
    const int a = (int)(i / q), c = (int)(i - (int64_t)a * q);
    const int64_t g = sc.active_idx[a];
    const float2 bc = bias[blockIdx.y];
    const float4 gr = reinterpret_cast<const float4*>(grads + (sc.grad_base + a) * sc.row_stride)[c];
    float4* pp = reinterpret_cast<float4*>(sc.params + g * sc.row_stride) + c;
    float4* mp = reinterpret_cast<float4*>(sc.adam_m + g * sc.row_stride) + c;
    float4* vp = reinterpret_cast<float4*>(sc.adam_v + g * sc.row_stride) + c;
    float4 p = *pp, m = *mp, v = *vp;
    const float gg[4] = {gr.x, gr.y, gr.z, gr.w};
    float* P = &p.x;
    float* M = &m.x;
    float* Vv = &v.x;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        M[k] = b1 * M[k] + (1.0f - b1) * gg[k];
        Vv[k] = b2 * Vv[k] + (1.0f - b2) * gg[k] * gg[k];
        const float mh = M[k] / bc.x;
        const float vh = Vv[k] / bc.y;
        P[k] -= lr * mh / (sqrtf(vh) + eps);
    }
    *pp = p;
    *mp = m;
    *vp = v;
}

}  // namespace cls

using namespace cls;

extern "C" size_t cls_adam_workspace_size(int32_t n_scenes) {
    return n_scenes <= 0 ? 0 : ((size_t)n_scenes * sizeof(float2) + 255) / 256 * 256;
}

extern "C" int cls_adam_step_active(const ClsScene* scenes_dev, const ClsBatchInfo* info,
                                    const float* grads, float lr, float beta1, float beta2,
                                    float eps, void* workspace, size_t workspace_bytes,
                                    cls_stream_t stream) {
    if (!scenes_dev || !info || info->n_scenes <= 0 || info->n_scenes > 65535 || !workspace ||
        workspace_bytes < cls_adam_workspace_size(info->n_scenes) ||
        (info->total_grad_rows > 0 && !grads) || !(beta1 >= 0.f && beta1 < 1.f) ||
        !(beta2 >= 0.f && beta2 < 1.f) || !(eps >= 0.f))
        return CLS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    float2* bias = static_cast<float2*>(workspace);
    adam_advance_kernel<<<(info->n_scenes + 127) / 128, 128, 0, s>>>(scenes_dev, info->n_scenes,
                                                                     beta1, beta2, bias);
    const int64_t work = (int64_t)info->max_active * (info->max_row_stride / 4);
    if (work > 0) {
        adam_active_kernel<<<dim3((unsigned)((work + 255) / 256), info->n_scenes), 256, 0, s>>>(
            scenes_dev, grads, bias, lr, beta1, beta2, eps);
    }
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}
