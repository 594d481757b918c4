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
// (tile + 5-pixel halo) by a horizontal then a vertical 11-tap pass (each
// thread 4 consecutive outputs from 14 loaded values); each
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
constexpr int SS_NT = 512;
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

constexpr int IRP = IR + 4;   // input row pitch: a 4-wide group reads 14 values from any group start

struct SsimSmem {
    float x[IR][IRP], y[IR][IRP];
    union {
        float h[5][IR + 4][MR];  // horizontal moment sums (4 spare rows for the last 4-row group)
        float t[3][MR][TS];      // horizontal sums of the sensitivities
    } a;
    float s[3][MR][MR];          // sensitivities on the moment region
    double red[2][SS_NT / 32];
};

// Each thread computes 4 consecutive outputs of a window pass from 14 loaded
// values (4 + 10 halo) instead of 4 x 11: the passes are bound by shared-memory
// loads. Every output sums its 11 taps in the same order as a single pass.
__device__ __forceinline__ void taps4(const float (&v)[14], const float *g, float (&o)[4])
{
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float m = 0.f;
#pragma unroll
        for (int j = 0; j < NTAP; ++j) m = fmaf(g[j], v[i + j], m);
        o[i] = m;
    }
}

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

    // 1. inputs with a 2 * RAD halo, zero outside the slice (and in the pitch padding)
    for (int i = tid; i < IR * IRP; i += SS_NT) {
        const int r = i / IRP, c = i - r * IRP;
        const int py = oy - 2 * RAD + r, px = ox - 2 * RAD + c;
        float xv = 0.f, yv = 0.f;
        if (c < IR && py >= 0 && py < H && px >= 0 && px < W) {
            xv = pred[base + (long long)py * W + px];
            yv = target[base + (long long)py * W + px];
        }
        sm.x[r][c] = xv;
        sm.y[r][c] = yv;
    }
    __syncthreads();
    // 2. horizontal window sums of x, y, x^2, y^2, x y: row r, columns c0..c0+3
    constexpr int G2 = (MR + 3) / 4;  // 11 column groups
    for (int i = tid; i < IR * G2; i += SS_NT) {
        const int r = i / G2, c0 = 4 * (i - r * G2);
        float xv[14], yv[14], v[14], o[4];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float4 a4 = *(const float4 *)&sm.x[r][c0 + 4 * q];
            const float4 b4 = *(const float4 *)&sm.y[r][c0 + 4 * q];
            xv[4 * q] = a4.x, xv[4 * q + 1] = a4.y, xv[4 * q + 2] = a4.z, xv[4 * q + 3] = a4.w;
            yv[4 * q] = b4.x, yv[4 * q + 1] = b4.y, yv[4 * q + 2] = b4.z, yv[4 * q + 3] = b4.w;
        }
        {
            const float2 a2 = *(const float2 *)&sm.x[r][c0 + 12];
            const float2 b2 = *(const float2 *)&sm.y[r][c0 + 12];
            xv[12] = a2.x, xv[13] = a2.y, yv[12] = b2.x, yv[13] = b2.y;
        }
        const int nv = min(4, MR - c0);
#pragma unroll
        for (int m = 0; m < 5; ++m) {
#pragma unroll
            for (int j = 0; j < 14; ++j)
                v[j] = m == 0 ? xv[j] : m == 1 ? yv[j] : m == 2 ? xv[j] * xv[j] : m == 3 ? yv[j] * yv[j] : xv[j] * yv[j];
            taps4(v, T.g, o);
            for (int q = 0; q < nv; ++q) sm.a.h[m][r][c0 + q] = o[q];
        }
    }
    __syncthreads();
    // 3. vertical sums -> SSIM_p and its sensitivities (zero outside the slice):
    //    column c, rows r0..r0+3
    const float dlds = -T.lam * T.inv_n;
    float ssum = 0.f;
    for (int i = tid; i < MR * G2; i += SS_NT) {
        const int g3 = i / MR, c = i - g3 * MR, r0 = 4 * g3;
        float mo[5][4];
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            float v[14], o[4];
#pragma unroll
            for (int j = 0; j < 14; ++j) v[j] = sm.a.h[m][r0 + j][c];
            taps4(v, T.g, o);
#pragma unroll
            for (int q = 0; q < 4; ++q) mo[m][q] = o[q];
        }
        const int px = ox - RAD + c;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = r0 + q;
            if (r >= MR) break;
            const int py = oy - RAD + r;
            float d0 = 0.f, d1 = 0.f, d2 = 0.f;
            if (py >= 0 && py < H && px >= 0 && px < W) {
                const float mx = mo[0][q], my = mo[1][q], exx = mo[2][q], eyy = mo[3][q], exy = mo[4][q];
                const float sxx = exx - mx * mx, syy = eyy - my * my, sxy = exy - mx * my;
                const float a1 = 2.f * mx * my + C1, a2 = 2.f * sxy + C2;
                const float b1 = mx * mx + my * my + C1, b2 = sxx + syy + C2;
                // S = N / D, N = a1 a2, D = b1 b2; b1 >= C1 and b2 >= C2, while
                // a1 and a2 vanish for anti-correlated windows: the quotient
                // rule divides by D only
                const float iD = 1.f / (b1 * b2);
                const float sv = (a1 * a2) * iD;
                if (r >= RAD && r < RAD + TS && c >= RAD && c < RAD + TS) ssum += sv;
                const float k2 = 2.f * dlds * iD;
                d0 = k2 * (my * (a2 - a1) - sv * mx * (b2 - b1));  // dS/dmu_x
                d1 = -dlds * sv / b2;                               // dS/dE_xx
                d2 = k2 * a1;                                       // dS/dE_xy
            }
            sm.s[0][r][c] = d0;
            sm.s[1][r][c] = d1;
            sm.s[2][r][c] = d2;
        }
    }
    __syncthreads();
    // 4. horizontal window sums of the sensitivities (the moment sums are dead):
    //    row r, columns c0..c0+3
    constexpr int G4 = TS / 4;  // 8 column groups
    for (int i = tid; i < MR * G4; i += SS_NT) {
        const int g4 = i / MR, r = i - g4 * MR, c0 = 4 * g4;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            float v[14], o[4];
#pragma unroll
            for (int j = 0; j < 14; ++j) v[j] = sm.s[m][r][c0 + j];
            taps4(v, T.g, o);
#pragma unroll
            for (int q = 0; q < 4; ++q) sm.a.t[m][r][c0 + q] = o[q];
        }
    }
    __syncthreads();
    // 5. vertical sums, gradient of the tile, smooth-L1 term: column c, rows r0..r0+3
    float lsum = 0.f;
    for (int i = tid; i < TS * G4; i += SS_NT) {
        const int g5 = i / TS, c = i - g5 * TS, r0 = 4 * g5;
        float u[3][4];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            float v[14], o[4];
#pragma unroll
            for (int j = 0; j < 14; ++j) v[j] = sm.a.t[m][r0 + j][c];
            taps4(v, T.g, o);
#pragma unroll
            for (int q = 0; q < 4; ++q) u[m][q] = o[q];
        }
        const int px = ox + c;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int py = oy + r0 + q;
            if (py >= H || px >= W) continue;
            const float xv = sm.x[r0 + q + 2 * RAD][c + 2 * RAD], yv = sm.y[r0 + q + 2 * RAD][c + 2 * RAD];
            const float res = xv - yv, ar = fabsf(res);
            lsum += ar < 1.f ? 0.5f * res * res : ar - 0.5f;
            if (grad) {
                const float gl1 = (ar < 1.f ? res : copysignf(1.f, res)) * T.inv_n;
                grad[base + (long long)py * W + px] = gl1 + u[0][q] + 2.f * xv * u[1][q] + yv * u[2][q];
            }
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
