// mg_params.cu -- the parameterisation of the fit (Sec. 3.2) and the
// anisotropy regulariser (Eqs. E12, E13), forward and backward, one launch
// each (plus a one-block FP64 finish for the regulariser's mean).
//
// Optimised variables per Gaussian: mean_c (canonical coordinates, mm =
// centre + half * mean_c), an unnormalised quaternion q_raw, log-scales ls
// and alpha. The renderer takes mean, q = q_raw / |q_raw|, scale = exp(ls).
// L_aniso = (1/N) sum_i max(0, max_a s_ia / min_a s_ia - lambda_r), s = exp(ls)
// (the ratio of the scales; E13 writes it on the log-scales, which has no
// meaning). The backward maps dL/d(mean, q, scale) and lambda_aniso * L_aniso
// to dL/d(mean_c, q_raw, ls); with ties the first index attains the max / min.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mg_internal.cuh"

mg_status mg_set_error(mg_status s, const char *msg);  // mg_api.cu

namespace {

constexpr int PR_NT = 256;
constexpr int PR_MAX_BLOCKS = 148 * 4;

__device__ __forceinline__ void argmaxmin3(const float *v, int &imax, int &imin)
{
    imax = 0;
    imin = 0;
    for (int a = 1; a < 3; ++a) {
        if (v[a] > v[imax]) imax = a;
        if (v[a] < v[imin]) imin = a;
    }
}

__global__ void __launch_bounds__(PR_NT) k_params_fwd(long long n, const float *__restrict__ mean_c,
                                                      const float *__restrict__ quat_raw,
                                                      const float *__restrict__ log_scale, float c0, float c1,
                                                      float c2, float half, float lambda_r, float *__restrict__ mean,
                                                      float *__restrict__ quat, float *__restrict__ scale,
                                                      double *__restrict__ part)
{
    __shared__ double red[PR_NT / 32];
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * PR_NT + threadIdx.x; i < n; i += (long long)gridDim.x * PR_NT) {
        mean[3 * i] = fmaf(half, mean_c[3 * i], c0);
        mean[3 * i + 1] = fmaf(half, mean_c[3 * i + 1], c1);
        mean[3 * i + 2] = fmaf(half, mean_c[3 * i + 2], c2);
        const float4 q = *(const float4 *)(quat_raw + 4 * i);
        const float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
        *(float4 *)(quat + 4 * i) = make_float4(q.x * inv, q.y * inv, q.z * inv, q.w * inv);
        float ls[3] = {log_scale[3 * i], log_scale[3 * i + 1], log_scale[3 * i + 2]};
        for (int a = 0; a < 3; ++a) scale[3 * i + a] = expf(ls[a]);
        int imax, imin;
        argmaxmin3(ls, imax, imin);  // exp is monotone: the same indices as on the scales
        const float ratio = expf(ls[imax] - ls[imin]);
        acc += (double)fmaxf(ratio - lambda_r, 0.f);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (part && threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < PR_NT / 32; ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(256) k_params_finish(const double *__restrict__ part, int nb, double inv_n,
                                                       double *__restrict__ aniso_out)
{
    __shared__ double s[256];
    double a = 0.0;
    for (int i = threadIdx.x; i < nb; i += 256) a += part[i];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *aniso_out = s[0] * inv_n;
}

__global__ void __launch_bounds__(PR_NT) k_params_bwd(long long n, const float *__restrict__ quat_raw,
                                                      const float *__restrict__ log_scale, float half, float lambda_r,
                                                      float w_aniso, const float *__restrict__ g_mean,
                                                      const float *__restrict__ g_quat,
                                                      const float *__restrict__ g_scale, float *__restrict__ g_mean_c,
                                                      float *__restrict__ g_quat_raw,
                                                      float *__restrict__ g_log_scale)
{
    for (long long i = (long long)blockIdx.x * PR_NT + threadIdx.x; i < n; i += (long long)gridDim.x * PR_NT) {
        g_mean_c[3 * i] = half * g_mean[3 * i];
        g_mean_c[3 * i + 1] = half * g_mean[3 * i + 1];
        g_mean_c[3 * i + 2] = half * g_mean[3 * i + 2];
        // q = q_raw / |q_raw|: dL/dq_raw = (g - q (q . g)) / |q_raw|
        const float4 q = *(const float4 *)(quat_raw + 4 * i);
        const float4 g = *(const float4 *)(g_quat + 4 * i);
        const float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
        const float4 u = make_float4(q.x * inv, q.y * inv, q.z * inv, q.w * inv);
        const float ug = u.x * g.x + u.y * g.y + u.z * g.z + u.w * g.w;
        *(float4 *)(g_quat_raw + 4 * i) =
            make_float4((g.x - u.x * ug) * inv, (g.y - u.y * ug) * inv, (g.z - u.z * ug) * inv,
                        (g.w - u.w * ug) * inv);
        // scale = exp(ls), plus the regulariser on the ratio exp(ls_max - ls_min)
        float ls[3] = {log_scale[3 * i], log_scale[3 * i + 1], log_scale[3 * i + 2]};
        float gl[3];
        for (int a = 0; a < 3; ++a) gl[a] = g_scale[3 * i + a] * expf(ls[a]);
        int imax, imin;
        argmaxmin3(ls, imax, imin);
        const float ratio = expf(ls[imax] - ls[imin]);
        if (ratio - lambda_r > 0.f) {
            const float d = w_aniso * ratio;
            gl[imax] += d;
            gl[imin] -= d;
        }
        for (int a = 0; a < 3; ++a) g_log_scale[3 * i + a] = gl[a];
    }
}

int params_blocks(long long n)
{
    long long b = (n + PR_NT - 1) / PR_NT;
    if (b > PR_MAX_BLOCKS) b = PR_MAX_BLOCKS;
    return b < 1 ? 1 : (int)b;
}

bool al16(const void *p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace

extern "C" size_t mg_params_workspace_size(int64_t n) { return (size_t)params_blocks(n) * sizeof(double) + 256; }

extern "C" mg_status mg_params_fwd(int64_t n, const float *mean_c, const float *quat_raw, const float *log_scale,
                                   const float centre[3], float half, float lambda_r, float *mean, float *quat,
                                   float *scale, double *aniso_out, void *ws, size_t ws_bytes, mg_stream_t stream)
{
    if (n < 0 || !centre || !(half > 0.f) || !isfinite(half) || !isfinite(lambda_r))
        return mg_set_error(MG_ERR_INVALID_ARG, "mg_params_fwd: need n >= 0, a centre, half > 0, finite lambda_r");
    if (n == 0) return MG_OK;
    if (!mean_c || !quat_raw || !log_scale || !mean || !quat || !scale || !al16(quat_raw) || !al16(quat))
        return mg_set_error(MG_ERR_INVALID_ARG, "mg_params_fwd: NULL or misaligned (quaternions: 16 B) pointer");
    if (aniso_out && (!ws || ws_bytes < mg_params_workspace_size(n)))
        return mg_set_error(MG_ERR_INVALID_ARG, "mg_params_fwd: workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = params_blocks(n);
    double *part = aniso_out ? (double *)ws : nullptr;  // no regulariser value requested: no partial sums
    k_params_fwd<<<nb, PR_NT, 0, st>>>(n, mean_c, quat_raw, log_scale, centre[0], centre[1], centre[2], half,
                                       lambda_r, mean, quat, scale, part);
    if (aniso_out) k_params_finish<<<1, 256, 0, st>>>(part, nb, 1.0 / (double)n, aniso_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mg_set_error(MG_ERR_CUDA, cudaGetErrorString(e));
    return MG_OK;
}

extern "C" mg_status mg_params_bwd(int64_t n, const float *quat_raw, const float *log_scale, float half,
                                   float lambda_r, float lambda_aniso, const float *g_mean, const float *g_quat,
                                   const float *g_scale, float *g_mean_c, float *g_quat_raw, float *g_log_scale,
                                   mg_stream_t stream)
{
    if (n < 0 || !(half > 0.f) || !isfinite(half) || !isfinite(lambda_r) || !isfinite(lambda_aniso))
        return mg_set_error(MG_ERR_INVALID_ARG, "mg_params_bwd: need n >= 0, half > 0, finite lambdas");
    if (n == 0) return MG_OK;
    if (!quat_raw || !log_scale || !g_mean || !g_quat || !g_scale || !g_mean_c || !g_quat_raw || !g_log_scale ||
        !al16(quat_raw) || !al16(g_quat) || !al16(g_quat_raw))
        return mg_set_error(MG_ERR_INVALID_ARG, "mg_params_bwd: NULL or misaligned (quaternions: 16 B) pointer");
    cudaStream_t st = (cudaStream_t)stream;
    k_params_bwd<<<params_blocks(n), PR_NT, 0, st>>>(n, quat_raw, log_scale, half, lambda_r,
                                                     (float)((double)lambda_aniso / (double)n), g_mean, g_quat,
                                                     g_scale, g_mean_c, g_quat_raw, g_log_scale);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mg_set_error(MG_ERR_CUDA, cudaGetErrorString(e));
    return MG_OK;
}
