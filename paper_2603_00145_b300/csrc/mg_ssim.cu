// mg_ssim.cu -- the paper's reconstruction loss (Sec. 3.5.2):
//   L_recon = L_L1 + lambda_SSIM (1 - mean SSIM),
// L_L1 the smooth-L1 mean of Eq. E11, SSIM the structural similarity of Wang
// et al. (2004) of every pixel of every rendered slice against the acquired
// slice (11 x 11 Gaussian window, sigma 1.5 px, zero padding outside the
// slice, C1 = 0.01^2, C2 = 0.03^2), and its gradient with respect to the
// rendered slices, in one fused kernel.
//
// One block per 32 x 32 output tile of a slice. The tile's inputs with a
// 10-pixel halo (52 x 52) are staged in shared memory; the five windowed
// moments (mu_x, mu_y, E_xx, E_yy, E_xy) are formed on the 42 x 42 region
// (tile + 5-pixel halo) by a horizontal then a vertical 11-tap pass; each
// pixel of that region inside the slice gives SSIM_p and the three
// sensitivities dSSIM_p/d(mu_x, E_xx, E_xy) scaled by dL/dSSIM_p; a second
// pair of passes sums them over the window of each output pixel (the
// window is symmetric, so the adjoint of the windowed sum is the same sum),
// and dL/dx_q = u_mu + 2 x_q u_xx + y_q u_xy plus the smooth-L1 term.
// Everything is FP32 except the loss sums: per-block FP64 partials, added in
// block order by a single final block (deterministic).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>

#include "mg_internal.cuh"

mg_status mg_set_error(mg_status s, const char *msg);  // mg_api.cu

namespace {

constexpr int TS = 32;           // output tile edge
constexpr int RAD = 5;           // window radius (11 taps)
constexpr int NTAP = 2 * RAD + 1;
constexpr int MR = TS + 2 * RAD; // moment / sensitivity region edge (42)
constexpr int IR = TS + 4 * RAD; // input region edge (52)
constexpr int SS_NT = 256;
constexpr float C1 = 1e-4f;      // (0.01 * 1)^2
constexpr float C2 = 9e-4f;      // (0.03 * 1)^2

struct SsimStacks {
    int n_stacks;
    int tile_base[MG_MAX_STACKS + 1];
    int TX[MG_MAX_STACKS], TY[MG_MAX_STACKS], W[MG_MAX_STACKS], H[MG_MAX_STACKS];
    long long pix_base[MG_MAX_STACKS];  // offset of slice 0 of the stack
    float g[NTAP];                      // 1-D window, unit sum
    float inv_n;                        // 1 / total pixels
    float lam;                          // lambda_SSIM
};

struct SsimSmem {
    float x[IR][IR], y[IR][IR];
    union {
        float h[5][IR][MR];  // horizontal moment sums
        float t[3][MR][TS];  // horizontal sums of the sensitivities
    } a;
    float s[3][MR][MR];      // sensitivities on the moment region
    double red[2][SS_NT / 32];
};

__global__ void __launch_bounds__(SS_NT) k_loss_recon(const float *__restrict__ pred, const float *__restrict__ target,
                                                      SsimStacks T, float *__restrict__ grad,
                                                      double *__restrict__ part)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SsimSmem &sm = *reinterpret_cast<SsimSmem *>(smem_raw);
    const int tid = threadIdx.x;
    // block -> (stack, slice, tile)
    int st = 0;
    while (st + 1 < T.n_stacks && (int)blockIdx.x >= T.tile_base[st + 1]) ++st;
    const int local = (int)blockIdx.x - T.tile_base[st];
    const int TX = T.TX[st], TY = T.TY[st], W = T.W[st], H = T.H[st];
    const int per_slice = TX * TY;
    const int k = local / per_slice, tl = local - k * per_slice;
    const int ty = tl / TX, tx = tl - ty * TX;
    const long long base = T.pix_base[st] + (long long)k * H * W;
    const int oy = ty * TS, ox = tx * TS;

    // 1. inputs with a 2 * RAD halo, zero outside the slice
    for (int i = tid; i < IR * IR; i += SS_NT) {
        const int r = i / IR, c = i - r * IR;
        const int py = oy - 2 * RAD + r, px = ox - 2 * RAD + c;
        float xv = 0.f, yv = 0.f;
        if (py >= 0 && py < H && px >= 0 && px < W) {
            xv = pred[base + (long long)py * W + px];
            yv = target[base + (long long)py * W + px];
        }
        sm.x[r][c] = xv;
        sm.y[r][c] = yv;
    }
    __syncthreads();
    // 2. horizontal window sums of x, y, x^2, y^2, x y
    for (int i = tid; i < IR * MR; i += SS_NT) {
        const int r = i / MR, c = i - r * MR;
        float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f;
#pragma unroll
        for (int j = 0; j < NTAP; ++j) {
            const float xv = sm.x[r][c + j], yv = sm.y[r][c + j], gj = T.g[j];
            m0 = fmaf(gj, xv, m0);
            m1 = fmaf(gj, yv, m1);
            m2 = fmaf(gj, xv * xv, m2);
            m3 = fmaf(gj, yv * yv, m3);
            m4 = fmaf(gj, xv * yv, m4);
        }
        sm.a.h[0][r][c] = m0;
        sm.a.h[1][r][c] = m1;
        sm.a.h[2][r][c] = m2;
        sm.a.h[3][r][c] = m3;
        sm.a.h[4][r][c] = m4;
    }
    __syncthreads();
    // 3. vertical sums -> SSIM_p and its sensitivities (zero outside the slice)
    const float dlds = -T.lam * T.inv_n;
    float ssum = 0.f;
    for (int i = tid; i < MR * MR; i += SS_NT) {
        const int r = i / MR, c = i - r * MR;
        const int py = oy - RAD + r, px = ox - RAD + c;
        float d0 = 0.f, d1 = 0.f, d2 = 0.f;
        if (py >= 0 && py < H && px >= 0 && px < W) {
            float mx = 0.f, my = 0.f, exx = 0.f, eyy = 0.f, exy = 0.f;
#pragma unroll
            for (int j = 0; j < NTAP; ++j) {
                const float gj = T.g[j];
                mx = fmaf(gj, sm.a.h[0][r + j][c], mx);
                my = fmaf(gj, sm.a.h[1][r + j][c], my);
                exx = fmaf(gj, sm.a.h[2][r + j][c], exx);
                eyy = fmaf(gj, sm.a.h[3][r + j][c], eyy);
                exy = fmaf(gj, sm.a.h[4][r + j][c], exy);
            }
            const float sxx = exx - mx * mx, syy = eyy - my * my, sxy = exy - mx * my;
            const float a1 = 2.f * mx * my + C1, a2 = 2.f * sxy + C2;
            const float b1 = mx * mx + my * my + C1, b2 = sxx + syy + C2;
            const float s = (a1 * a2) / (b1 * b2);
            if (r >= RAD && r < RAD + TS && c >= RAD && c < RAD + TS) ssum += s;
            const float ia1 = 1.f / a1, ia2 = 1.f / a2, ib1 = 1.f / b1, ib2 = 1.f / b2;
            d0 = dlds * s * 2.f * (my * (ia1 - ia2) + mx * (ib2 - ib1));  // dS/dmu_x
            d1 = -dlds * s * ib2;                                          // dS/dE_xx
            d2 = dlds * s * 2.f * ia2;                                     // dS/dE_xy
        }
        sm.s[0][r][c] = d0;
        sm.s[1][r][c] = d1;
        sm.s[2][r][c] = d2;
    }
    __syncthreads();
    // 4. horizontal window sums of the sensitivities (the moment sums are dead)
    for (int i = tid; i < MR * TS; i += SS_NT) {
        const int r = i / TS, c = i - r * TS;
        float u0 = 0.f, u1 = 0.f, u2 = 0.f;
#pragma unroll
        for (int j = 0; j < NTAP; ++j) {
            const float gj = T.g[j];
            u0 = fmaf(gj, sm.s[0][r][c + j], u0);
            u1 = fmaf(gj, sm.s[1][r][c + j], u1);
            u2 = fmaf(gj, sm.s[2][r][c + j], u2);
        }
        sm.a.t[0][r][c] = u0;
        sm.a.t[1][r][c] = u1;
        sm.a.t[2][r][c] = u2;
    }
    __syncthreads();
    // 5. vertical sums, gradient of the tile, smooth-L1 term
    float lsum = 0.f;
    for (int i = tid; i < TS * TS; i += SS_NT) {
        const int r = i / TS, c = i - r * TS;
        const int py = oy + r, px = ox + c;
        if (py >= H || px >= W) continue;
        float u0 = 0.f, u1 = 0.f, u2 = 0.f;
#pragma unroll
        for (int j = 0; j < NTAP; ++j) {
            const float gj = T.g[j];
            u0 = fmaf(gj, sm.a.t[0][r + j][c], u0);
            u1 = fmaf(gj, sm.a.t[1][r + j][c], u1);
            u2 = fmaf(gj, sm.a.t[2][r + j][c], u2);
        }
        const float xv = sm.x[r + 2 * RAD][c + 2 * RAD], yv = sm.y[r + 2 * RAD][c + 2 * RAD];
        const float res = xv - yv, ar = fabsf(res);
        lsum += ar < 1.f ? 0.5f * res * res : ar - 0.5f;
        if (grad) {
            const float gl1 = (ar < 1.f ? res : copysignf(1.f, res)) * T.inv_n;
            grad[base + (long long)py * W + px] = gl1 + u0 + 2.f * xv * u1 + yv * u2;
        }
    }
    // block partials in FP64
    double v0 = (double)lsum, v1 = (double)ssum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    }
    if ((tid & 31) == 0) {
        sm.red[0][tid >> 5] = v0;
        sm.red[1][tid >> 5] = v1;
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < SS_NT / 32; ++w) {
            a += sm.red[0][w];
            b += sm.red[1][w];
        }
        part[2 * (size_t)blockIdx.x] = a;
        part[2 * (size_t)blockIdx.x + 1] = b;
    }
}

// one block: fixed-order FP64 sum of the block partials
__global__ void __launch_bounds__(256) k_loss_recon_final(const double *__restrict__ part, int nb, double inv_n,
                                                          double lam, double *__restrict__ out)
{
    __shared__ double sa[256], sb[256];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nb; i += 256) {
        a += part[2 * (size_t)i];
        b += part[2 * (size_t)i + 1];
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sa[threadIdx.x] += sa[threadIdx.x + s];
            sb[threadIdx.x] += sb[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double l1 = sa[0] * inv_n, ss = sb[0] * inv_n;
        out[0] = l1 + lam * (1.0 - ss);
        out[1] = l1;
        out[2] = ss;
    }
}

bool make_ssim_stacks(const mg_stack *stacks, int n_stacks, SsimStacks &T, long long &blocks, long long &pixels,
                      std::string &why)
{
    if (!stacks || n_stacks < 1 || n_stacks > MG_MAX_STACKS) {
        why = "need 1..32 stacks";
        return false;
    }
    T.n_stacks = n_stacks;
    blocks = 0;
    pixels = 0;
    for (int s = 0; s < n_stacks; ++s) {
        const mg_stack &d = stacks[s];
        if (d.n_slices < 1 || d.H < 1 || d.W < 1 || d.H > 16384 || d.W > 16384) {
            why = "stack " + std::to_string(s) + ": need n_slices >= 1 and 1 <= H, W <= 16384";
            return false;
        }
        T.tile_base[s] = (int)blocks;
        T.TX[s] = (d.W + TS - 1) / TS;
        T.TY[s] = (d.H + TS - 1) / TS;
        T.W[s] = d.W;
        T.H[s] = d.H;
        T.pix_base[s] = pixels;
        blocks += (long long)d.n_slices * T.TX[s] * T.TY[s];
        pixels += (long long)d.n_slices * d.H * d.W;
        if (blocks > 0x7fffffffLL) {
            why = "too many tiles";
            return false;
        }
    }
    T.tile_base[n_stacks] = (int)blocks;
    double g[NTAP], sum = 0.0;
    for (int j = 0; j < NTAP; ++j) {
        const double t = (double)(j - RAD);
        g[j] = exp(-t * t / (2.0 * 1.5 * 1.5));
        sum += g[j];
    }
    for (int j = 0; j < NTAP; ++j) T.g[j] = (float)(g[j] / sum);
    T.inv_n = (float)(1.0 / (double)pixels);
    return true;
}

}  // namespace

extern "C" size_t mg_loss_recon_workspace_size(const mg_stack *stacks, int n_stacks)
{
    SsimStacks T;
    long long blocks = 0, pixels = 0;
    std::string why;
    if (!make_ssim_stacks(stacks, n_stacks, T, blocks, pixels, why)) return 0;
    return (size_t)(16 * blocks + 255) / 256 * 256;
}

extern "C" mg_status mg_loss_recon(const float *pred, const float *target, const mg_stack *stacks, int n_stacks,
                                   float lambda_ssim, float *grad, double *loss_out, void *ws, size_t ws_bytes,
                                   mg_stream_t stream)
{
    SsimStacks T;
    long long blocks = 0, pixels = 0;
    std::string why;
    if (!make_ssim_stacks(stacks, n_stacks, T, blocks, pixels, why))
        return mg_set_error(MG_ERR_INVALID_ARG, ("mg_loss_recon: " + why).c_str());
    if (!pred || !target || !loss_out || !ws)
        return mg_set_error(MG_ERR_INVALID_ARG, "mg_loss_recon: pred, target, loss_out and ws are required");
    if (!(lambda_ssim >= 0.f) || !isfinite(lambda_ssim))
        return mg_set_error(MG_ERR_INVALID_ARG, "mg_loss_recon: lambda_ssim must be finite and >= 0");
    if (ws_bytes < (size_t)(16 * blocks)) return mg_set_error(MG_ERR_INVALID_ARG, "mg_loss_recon: workspace too small");
    T.lam = lambda_ssim;
    cudaStream_t st = (cudaStream_t)stream;
    MG_PROF(MG_ST_LOSS, st);
    const size_t smem = sizeof(SsimSmem);
    cudaFuncSetAttribute(k_loss_recon, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_loss_recon<<<(unsigned)blocks, SS_NT, smem, st>>>(pred, target, T, grad, (double *)ws);
    k_loss_recon_final<<<1, 256, 0, st>>>((const double *)ws, (int)blocks, 1.0 / (double)pixels, (double)lambda_ssim,
                                          loss_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mg_set_error(MG_ERR_CUDA, cudaGetErrorString(e));
    return MG_OK;
}
