// mg_adam.cu -- the optimiser step of the fit (Sec. 4.1.4: Adam with one
// learning rate per parameter group), fused over all groups in one launch.
//
// Adam (Kingma & Ba 2015) with the bias corrections of its Algorithm 1 and
// epsilon added to the bias-corrected root of the second moment:
//   m <- b1 m + (1-b1) g,  v <- b2 v + (1-b2) g^2,
//   p <- p - lr/(1-b1^t) * m / (sqrt(v)/sqrt(1-b2^t) + eps),  t = step + 1,
// then an optional clamp of p to [lo, hi] (the alpha range of Sec. 3.2).
//
// The update is predicated on a device status word: when (*status & mask) is
// nonzero (the forward of this iteration overflowed its bins or met a
// non-finite input) no parameter, moment or step counter changes. A fit
// replayed as a CUDA graph can therefore run without host checks: a failed
// iteration is a no-op, the host sees the step counter lag behind and grows
// the workspace.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mg_internal.cuh"

mg_status mg_set_error(mg_status s, const char *msg);  // mg_api.cu

namespace {

struct AdamGroupDev {
    float *p;
    const float *g;
    float *m;
    float *v;
    long long units;  // float4 units when vec, else floats
    float lr, lo, hi;
    int vec, clamp;
};

struct AdamArgs {
    int ng;
    long long unit_end[MG_ADAM_MAX_GROUPS];  // inclusive prefix of units
    AdamGroupDev g[MG_ADAM_MAX_GROUPS];
};

__device__ __forceinline__ float adam_one(float &p, float g, float &m, float &v, float b1, float b2, float step_size,
                                          float inv_sqrt_bc2, float eps)
{
    m = fmaf(b1, m, (1.f - b1) * g);
    v = fmaf(b2, v, (1.f - b2) * g * g);
    float denom = sqrtf(v) * inv_sqrt_bc2 + eps;
    p = p - step_size * (m / denom);
    return p;
}

__global__ void __launch_bounds__(256) k_adam(AdamArgs A, float b1, float b2, float eps, const int *step,
                                              const unsigned *status, unsigned mask)
{
    __shared__ AdamGroupDev sg[MG_ADAM_MAX_GROUPS];
    __shared__ long long send[MG_ADAM_MAX_GROUPS];
    __shared__ float s_step[MG_ADAM_MAX_GROUPS], s_isb2;
    if (status && (*status & mask)) return;  // uniform over the grid
    if (threadIdx.x < A.ng) {
        sg[threadIdx.x] = A.g[threadIdx.x];
        send[threadIdx.x] = A.unit_end[threadIdx.x];
    }
    if (threadIdx.x == 0) {
        // bias corrections once per block, in double
        const double t = (double)(*step + 1);
        const double bc1 = 1.0 - pow((double)b1, t), bc2 = 1.0 - pow((double)b2, t);
        for (int k = 0; k < A.ng; ++k) s_step[k] = (float)((double)A.g[k].lr / bc1);
        s_isb2 = (float)(1.0 / sqrt(bc2));
    }
    __syncthreads();
    const float inv_sqrt_bc2 = s_isb2;
    const int ng = A.ng;
    const long long total = send[ng - 1];
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < total;
         u += (long long)gridDim.x * blockDim.x) {
        int k = 0;
        while (k < ng - 1 && u >= send[k]) ++k;
        const AdamGroupDev &G = sg[k];
        const long long i = u - (k ? send[k - 1] : 0);
        const float step_size = s_step[k];
        if (G.vec) {
            float4 p = ((float4 *)G.p)[i], g = ((const float4 *)G.g)[i];
            float4 m = ((float4 *)G.m)[i], v = ((float4 *)G.v)[i];
            adam_one(p.x, g.x, m.x, v.x, b1, b2, step_size, inv_sqrt_bc2, eps);
            adam_one(p.y, g.y, m.y, v.y, b1, b2, step_size, inv_sqrt_bc2, eps);
            adam_one(p.z, g.z, m.z, v.z, b1, b2, step_size, inv_sqrt_bc2, eps);
            adam_one(p.w, g.w, m.w, v.w, b1, b2, step_size, inv_sqrt_bc2, eps);
            if (G.clamp) {
                p.x = fminf(fmaxf(p.x, G.lo), G.hi);
                p.y = fminf(fmaxf(p.y, G.lo), G.hi);
                p.z = fminf(fmaxf(p.z, G.lo), G.hi);
                p.w = fminf(fmaxf(p.w, G.lo), G.hi);
            }
            ((float4 *)G.p)[i] = p;
            ((float4 *)G.m)[i] = m;
            ((float4 *)G.v)[i] = v;
        } else {
            float p = G.p[i], m = G.m[i], v = G.v[i];
            adam_one(p, G.g[i], m, v, b1, b2, step_size, inv_sqrt_bc2, eps);
            if (G.clamp) p = fminf(fmaxf(p, G.lo), G.hi);
            G.p[i] = p;
            G.m[i] = m;
            G.v[i] = v;
        }
    }
}

__global__ void k_adam_tick(int *step, const unsigned *status, unsigned mask)
{
    if (status && (*status & mask)) return;
    *step += 1;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace

extern "C" mg_status mg_adam_step(const mg_adam_group *groups, int n_groups, float beta1, float beta2, float eps,
                                  int32_t *step, const uint32_t *status, uint32_t status_mask, mg_stream_t stream)
{
    if (!groups || n_groups < 1 || n_groups > MG_ADAM_MAX_GROUPS || !step)
        return mg_set_error(MG_ERR_INVALID_ARG, "mg_adam_step: groups, n_groups (1..8) and step are required");
    if (!(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f) || !isfinite(eps))
        return mg_set_error(MG_ERR_INVALID_ARG, "mg_adam_step: need 0 <= beta < 1 and eps > 0");
    AdamArgs A;
    A.ng = n_groups;
    long long acc = 0;
    for (int k = 0; k < n_groups; ++k) {
        const mg_adam_group &g = groups[k];
        if (g.n < 0 || (g.n > 0 && (!g.param || !g.grad || !g.m || !g.v)))
            return mg_set_error(MG_ERR_INVALID_ARG, "mg_adam_step: a group has a NULL pointer or n < 0");
        if (!isfinite(g.lr) || g.lr < 0.f)
            return mg_set_error(MG_ERR_INVALID_ARG, "mg_adam_step: lr must be finite and >= 0");
        AdamGroupDev &d = A.g[k];
        d.p = g.param;
        d.g = g.grad;
        d.m = g.m;
        d.v = g.v;
        d.lr = g.lr;
        d.clamp = g.clamp_lo <= g.clamp_hi;
        d.lo = g.clamp_lo;
        d.hi = g.clamp_hi;
        d.vec = (g.n % 4 == 0) && aligned16(g.param) && aligned16(g.grad) && aligned16(g.m) && aligned16(g.v);
        d.units = d.vec ? g.n / 4 : g.n;
        acc += d.units;
        A.unit_end[k] = acc;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (acc > 0) {
        long long want = (acc + 255) / 256;
        int grid = (int)(want < 148 * 8 ? want : 148 * 8);
        k_adam<<<grid, 256, 0, st>>>(A, beta1, beta2, eps, step, status, status_mask);
    }
    k_adam_tick<<<1, 1, 0, st>>>(step, status, status_mask);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mg_set_error(MG_ERR_CUDA, cudaGetErrorString(e));
    return MG_OK;
}
