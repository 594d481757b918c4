// mg_reduce.cu -- deterministic FP64 loss / MSE reductions (K10).
//
// Each thread sums 16 consecutive voxels in FP32 (|r| <= 1 here, so the leaf
// error is below 16 * 2^-24 relative), then accumulates the leaf sums in
// FP64 over a fixed grid-stride order; blocks reduce in FP64 and a final
// single block adds the block partials in index order. The result is the
// same bit pattern on every run. FP64 arithmetic is used only for the
// leaf-sum accumulation because FP64 throughput on this part is a small
// fraction of FP32.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "mg_internal.cuh"

mg_status mg_set_error(mg_status s, const char *msg);  // mg_api.cu

constexpr int RED_NT = 256;
constexpr int RED_LEAF = 16;

int mg_reduce_blocks(long long n)
{
    long long leaves = (n + RED_LEAF - 1) / RED_LEAF;
    long long b = (leaves + RED_NT - 1) / RED_NT;
    if (b > 148 * 8) b = 148 * 8;
    if (b < 1) b = 1;
    return (int)b;
}

__device__ __forceinline__ double block_sum_d(double v)
{
    __shared__ double sh[RED_NT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < RED_NT / 32; ++i) s += sh[i];
    __syncthreads();
    return s;
}

// mode 0: L1 + L2 loss (+ gradient); mode 1: sum of squared differences
template <int MODE>
__global__ void __launch_bounds__(RED_NT) k_reduce_leaf(const float *__restrict__ a, const float *__restrict__ b,
                                                        long long n, float *__restrict__ grad, double inv_n,
                                                        double *__restrict__ part)
{
    long long leaves = (n + RED_LEAF - 1) / RED_LEAF;
    double s1 = 0.0, s2 = 0.0;
    for (long long l = (long long)blockIdx.x * RED_NT + threadIdx.x; l < leaves; l += (long long)gridDim.x * RED_NT) {
        long long i0 = l * RED_LEAF;
        float f1 = 0.f, f2 = 0.f;
        if (i0 + RED_LEAF <= n && ((((uintptr_t)(a + i0)) | ((uintptr_t)(b + i0))) & 15) == 0) {
#pragma unroll
            for (int j = 0; j < RED_LEAF; j += 4) {
                float4 x = *(const float4 *)(a + i0 + j);
                float4 y = *(const float4 *)(b + i0 + j);
                float r[4] = {x.x - y.x, x.y - y.y, x.z - y.z, x.w - y.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    f1 += fabsf(r[u]);
                    f2 = fmaf(r[u], r[u], f2);
                }
                if (MODE == 0 && grad) {
                    float4 g;
                    const float sc = (float)inv_n;
                    g.x = (copysignf(r[0] != 0.f ? 1.f : 0.f, r[0]) + 2.f * r[0]) * sc;
                    g.y = (copysignf(r[1] != 0.f ? 1.f : 0.f, r[1]) + 2.f * r[1]) * sc;
                    g.z = (copysignf(r[2] != 0.f ? 1.f : 0.f, r[2]) + 2.f * r[2]) * sc;
                    g.w = (copysignf(r[3] != 0.f ? 1.f : 0.f, r[3]) + 2.f * r[3]) * sc;
                    if ((((uintptr_t)(grad + i0)) & 15) == 0)
                        *(float4 *)(grad + i0 + j) = g;
                    else {
                        grad[i0 + j] = g.x;
                        grad[i0 + j + 1] = g.y;
                        grad[i0 + j + 2] = g.z;
                        grad[i0 + j + 3] = g.w;
                    }
                }
            }
        } else {
            for (int j = 0; j < RED_LEAF; ++j) {
                long long i = i0 + j;
                if (i >= n) break;
                float r = a[i] - b[i];
                f1 += fabsf(r);
                f2 = fmaf(r, r, f2);
                if (MODE == 0 && grad)
                    grad[i] = (copysignf(r != 0.f ? 1.f : 0.f, r) + 2.f * r) * (float)inv_n;
            }
        }
        s1 += (double)f1;
        s2 += (double)f2;
    }
    double t1 = block_sum_d(s1);
    double t2 = block_sum_d(s2);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = t1;
        part[2 * blockIdx.x + 1] = t2;
    }
}

// one block: thread i adds partials i, i+256, ... in index order, then a
// fixed shuffle tree; the same bits on every run
template <int MODE>
__global__ void __launch_bounds__(RED_NT) k_reduce_final(const double *__restrict__ part, int nb, double inv_n,
                                                         double *__restrict__ out)
{
    double s1 = 0.0, s2 = 0.0;
    for (int i = threadIdx.x; i < nb; i += RED_NT) {
        s1 += part[2 * i];
        s2 += part[2 * i + 1];
    }
    double t1 = block_sum_d(s1);
    double t2 = block_sum_d(s2);
    if (threadIdx.x == 0) {
        if (MODE == 0) {
            out[0] = t1 * inv_n + t2 * inv_n;
            out[1] = t2;
        } else {
            out[0] = t2;
        }
    }
}

void mg_launch_loss_l1l2(const float *pred, const float *target, long long n, float *grad, double *out,
                         double *part, cudaStream_t st)
{
    int nb = mg_reduce_blocks(n);
    double inv_n = n > 0 ? 1.0 / (double)n : 0.0;
    k_reduce_leaf<0><<<nb, RED_NT, 0, st>>>(pred, target, n, grad, inv_n, part);
    k_reduce_final<0><<<1, RED_NT, 0, st>>>(part, nb, inv_n, out);
}

void mg_launch_sq_diff(const float *a, const float *b, long long n, double *out, double *part, cudaStream_t st)
{
    int nb = mg_reduce_blocks(n);
    k_reduce_leaf<1><<<nb, RED_NT, 0, st>>>(a, b, n, nullptr, 0.0, part);
    k_reduce_final<1><<<1, RED_NT, 0, st>>>(part, nb, 0.0, out);
}

// ---------------------------------------------------------------------------
// mg_loss_l1l2_noalloc: the same reduction with its per-block partial sums in
// a fixed array inside the library instead of a caller workspace.
// ---------------------------------------------------------------------------
#define MG_NOALLOC_MAX_BLOCKS 8192  // 2 doubles each: 128 KiB
#define MG_NOALLOC_MAX_N ((long long)MG_NOALLOC_MAX_BLOCKS * RED_NT * RED_LEAF)
#define MG_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) double g_noalloc_part[2 * MG_NOALLOC_MAX_BLOCKS];

static std::mutex g_noalloc_mu;
static double *g_noalloc_ptr[MG_NOALLOC_MAX_DEVICES];

extern "C" mg_status mg_loss_l1l2_noalloc(const float *pred, const float *target, int64_t n, float *grad,
                                          double *loss_out, mg_stream_t stream)
{
    if (n < 0 || (n > 0 && (!pred || !target)) || !loss_out)
        return mg_set_error(MG_ERR_INVALID_ARG, "mg_loss_l1l2_noalloc: bad pointer or size");
    if (n > MG_NOALLOC_MAX_N)
        return mg_set_error(MG_ERR_INVALID_ARG,
                            "mg_loss_l1l2_noalloc: n exceeds the fixed partial-sum array (at most 33554432 "
                            "elements); use mg_loss_l1l2 with a workspace");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MG_NOALLOC_MAX_DEVICES)
        return mg_set_error(MG_ERR_CUDA, "mg_loss_l1l2_noalloc: no usable current device");
    cudaStream_t st = (cudaStream_t)stream;
    // Is the stream being captured into a graph? A query that fails (the
    // legacy stream while another stream captures) counts as capturing.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        (void)cudaGetLastError();
        cap = cudaStreamCaptureStatusActive;
    }
    double *part = nullptr;
    {
        // The device address of the array (its name is only a host-side
        // stand-in), looked up with the device current. Outside a capture it
        // is looked up on every call (no allocation), so it stays right after
        // a cudaDeviceReset reloads the module; inside a capture the address
        // of the last call outside one is used.
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (cap == cudaStreamCaptureStatusNone) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_part);
            if (e != cudaSuccess || !p)
                return mg_set_error(MG_ERR_CUDA, "mg_loss_l1l2_noalloc: cudaGetSymbolAddress failed");
            g_noalloc_ptr[dev] = (double *)p;
        } else if (!g_noalloc_ptr[dev]) {
            return mg_set_error(MG_ERR_INVALID_ARG,
                                "mg_loss_l1l2_noalloc: first call on this device inside a stream capture; make one "
                                "call outside any capture first");
        }
        part = g_noalloc_ptr[dev];
    }
    long long leaves = (n + RED_LEAF - 1) / RED_LEAF;
    int nb = (int)((leaves + RED_NT - 1) / RED_NT);
    if (nb < 1) nb = 1;
    double inv_n = n > 0 ? 1.0 / (double)n : 0.0;
    // every partial slot the final pass reads is written by the first pass,
    // so nothing left in the array by an earlier call is used
    k_reduce_leaf<0><<<nb, RED_NT, 0, st>>>(pred, target, n, grad, inv_n, part);
    k_reduce_final<0><<<1, RED_NT, 0, st>>>(part, nb, inv_n, loss_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mg_set_error(MG_ERR_CUDA, cudaGetErrorString(e));
    return MG_OK;
}
