// mg_nrf.cu -- the neural residual field (Sec. 3.4, Eq. E8): fused coordinate
// encoding + MLP, forward and backward, r(x) = out_scale * tanh(MLP(enc(x))).
//
// Two encodings (mgauss.h): the paper's Fourier features (6 bands, 39
// features, 4 hidden layers of 64 SiLU units) and a 16-level hash grid with 2
// features per level (2 hidden layers of 64 ReLU units). Two precisions:
//   BF16: activations and weights in BF16 in shared memory, hidden layers as
//         mma.sync m16n8k16 BF16 GEMMs with FP32 accumulation; tiles of 64
//         points, 4 warps, each warp 16 points.
//   FP32: the same data flow with register-blocked SIMT FP32 GEMMs on tiles of
//         16 points.
// A block keeps the weights in shared memory for all its tiles (grid-stride).
// The backward recomputes the forward of a tile (pre-activations kept), then
// walks the layers back: weight gradients dW += delta^T H (one GEMM), input
// deltas delta W (one GEMM), accumulated per block in shared memory and
// flushed with one atomic per parameter per block. Grid-table gradients are
// scattered with one float2 atomic per (point, level, corner): both features
// of a level come out of one register pair of the D W_0 product.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "mg_internal.cuh"

namespace {

typedef __nv_bfloat16 bf16;

constexpr int NRF_NT = 128;  // threads per block (4 warps)
constexpr int WIDTH = 64;    // hidden width
constexpr int GRID_LEVELS = 16;

template <int ENC>
struct Preset;
template <>
struct Preset<MG_NRF_FOURIER> {
    static constexpr int L = 4;     // hidden layers
    static constexpr int K0 = 39;   // encoded features
    static constexpr int K0P = 48;  // padded to a multiple of 16
    static constexpr bool SILU = true;
};
template <>
struct Preset<MG_NRF_GRID> {
    static constexpr int L = 2;
    static constexpr int K0 = 32;
    static constexpr int K0P = 32;
    static constexpr bool SILU = false;
};

// input width of hidden layer l (padded / real)
template <int ENC>
__host__ __device__ constexpr int kin_pad(int l)
{
    return l == 0 ? Preset<ENC>::K0P : WIDTH;
}
template <int ENC>
__host__ __device__ constexpr int kin_real(int l)
{
    return l == 0 ? Preset<ENC>::K0 : WIDTH;
}
// offsets of W_l / b_l / w_out / b_out in the packed FP32 parameter vector
template <int ENC>
__host__ __device__ constexpr int off_w(int l)
{
    return l == 0 ? 0 : off_w<ENC>(l - 1) + WIDTH * kin_real<ENC>(l - 1) + WIDTH;
}
template <int ENC>
__host__ __device__ constexpr int off_b(int l)
{
    return off_w<ENC>(l) + WIDTH * kin_real<ENC>(l);
}
template <int ENC>
__host__ __device__ constexpr int off_wout()
{
    return off_w<ENC>(Preset<ENC>::L);
}
template <int ENC>
__host__ __device__ constexpr int n_params()
{
    return off_wout<ENC>() + WIDTH + 1;
}

struct GridGeom {
    int res[GRID_LEVELS];
    int dense[GRID_LEVELS];
    unsigned tmask;
    int log2T;
};

struct NrfArgs {
    const float *params;
    const float *table;
    float out_scale;
    GridGeom grid;
    const long long *idx;  // point i is row idx[i] of xyz / out / grad_out (NULL: row i)
    long long rows;        // with idx: rows of xyz / out / grad_out; other indices are skipped
    void *enc;             // grid encoding cache [n][32] (element type of the precision)
    int enc_mode;          // MG_NRF_ENC_NONE / _STORE / _LOAD
};

// Row of point i (-1: past the end or an index outside [0, rows)).
__device__ __forceinline__ long long nrf_row(const NrfArgs &A, long long i, long long n)
{
    if (i >= n) return -1;
    if (!A.idx) return i;
    const long long r = A.idx[i];
    return (r >= 0 && r < A.rows) ? r : -1;
}

// ---------------------------------------------------------------------------
// element helpers
// ---------------------------------------------------------------------------
template <typename E>
__device__ __forceinline__ E to_e(float x);
template <>
__device__ __forceinline__ bf16 to_e<bf16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ float to_e<float>(float x) { return x; }
__device__ __forceinline__ float to_f(bf16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float to_f(float x) { return x; }

__device__ __forceinline__ float tanh_approx(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <bool BF16>
__device__ __forceinline__ float sigmoid(float z)
{
    if (BF16) return fmaf(0.5f, tanh_approx(0.5f * z), 0.5f);
    return 1.0f / (1.0f + expf(-z));
}

template <int ENC, bool BF16>
__device__ __forceinline__ float act(float z)
{
    if (Preset<ENC>::SILU) return z * sigmoid<BF16>(z);
    return fmaxf(z, 0.f);
}

template <int ENC, bool BF16>
__device__ __forceinline__ float act_grad(float z)
{
    if (Preset<ENC>::SILU) {
        float s = sigmoid<BF16>(z);
        return s * fmaf(z, 1.f - s, 1.f);
    }
    return z > 0.f ? 1.f : 0.f;
}

// ---------------------------------------------------------------------------
// tensor-core helpers (mma.sync m16n8k16 BF16, FP32 accumulate)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ldsm_x4(unsigned r[4], const void *p)
{
    unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned r[4], const void *p)
{
    unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}
__device__ __forceinline__ void mma16816(float c[4], const unsigned a[4], unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Z[64 x 64] = H[64 x K] W^T (W [64][K]); warp w: rows 16w..16w+15.
// epi(row, col, value) for every output of the warp.
template <int K, class Epi>
__device__ __forceinline__ void gemm_hwT_bf16(const bf16 *H, int ldh, const bf16 *W, int ldw, int w, int lane, Epi epi)
{
    float c[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i) c[i][0] = c[i][1] = c[i][2] = c[i][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < K / 16; ++ks) {
        unsigned a[4];
        ldsm_x4(a, H + (16 * w + (lane & 15)) * ldh + ks * 16 + (lane >> 4) * 8);
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            unsigned b[4];
            ldsm_x4(b, W + (n2 * 16 + (lane & 7) + ((lane >> 4) << 3)) * ldw + ks * 16 + ((lane >> 3) & 1) * 8);
            mma16816(c[2 * n2], a, b[0], b[1]);
            mma16816(c[2 * n2 + 1], a, b[2], b[3]);
        }
    }
    const int g = lane >> 2, q = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        epi(16 * w + g, nt * 8 + 2 * q, c[nt][0]);
        epi(16 * w + g, nt * 8 + 2 * q + 1, c[nt][1]);
        epi(16 * w + g + 8, nt * 8 + 2 * q, c[nt][2]);
        epi(16 * w + g + 8, nt * 8 + 2 * q + 1, c[nt][3]);
    }
}

// G[64 x K] = D^T H, D [64 points][64], H [64 points][K]; warp w: rows
// (outputs) 16w..16w+15; the reduction runs over the 64 points.
template <int K, class Epi>
__device__ __forceinline__ void gemm_dTh_bf16(const bf16 *D, int ldd, const bf16 *H, int ldh, int w, int lane, Epi epi)
{
    float c[K / 8][4];
#pragma unroll
    for (int i = 0; i < K / 8; ++i) c[i][0] = c[i][1] = c[i][2] = c[i][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
        unsigned a[4];
        ldsm_x4_t(a, D + (ks * 16 + (lane & 7) + ((lane >> 4) & 1) * 8) * ldd + 16 * w + ((lane >> 3) & 1) * 8);
#pragma unroll
        for (int n2 = 0; n2 < K / 16; ++n2) {
            unsigned b[4];
            ldsm_x4_t(b, H + (ks * 16 + (lane & 7) + ((lane >> 3) & 1) * 8) * ldh + n2 * 16 + ((lane >> 4) << 3));
            mma16816(c[2 * n2], a, b[0], b[1]);
            mma16816(c[2 * n2 + 1], a, b[2], b[3]);
        }
    }
    const int g = lane >> 2, q = lane & 3;
#pragma unroll
    for (int nt = 0; nt < K / 8; ++nt) {
        epi(16 * w + g, nt * 8 + 2 * q, c[nt][0]);
        epi(16 * w + g, nt * 8 + 2 * q + 1, c[nt][1]);
        epi(16 * w + g + 8, nt * 8 + 2 * q, c[nt][2]);
        epi(16 * w + g + 8, nt * 8 + 2 * q + 1, c[nt][3]);
    }
}

// P[64 x K] = D W, D [64 points][64], W [64][K]; warp w: points 16w..16w+15.
// PAIR: epi(point, even column, value, value of the next column).
template <int K, bool PAIR = false, class Epi>
__device__ __forceinline__ void gemm_dw_bf16(const bf16 *D, int ldd, const bf16 *W, int ldw, int w, int lane, Epi epi)
{
    float c[K / 8][4];
#pragma unroll
    for (int i = 0; i < K / 8; ++i) c[i][0] = c[i][1] = c[i][2] = c[i][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
        unsigned a[4];
        ldsm_x4(a, D + (16 * w + (lane & 15)) * ldd + ks * 16 + (lane >> 4) * 8);
#pragma unroll
        for (int n2 = 0; n2 < K / 16; ++n2) {
            unsigned b[4];
            ldsm_x4_t(b, W + (ks * 16 + (lane & 7) + ((lane >> 3) & 1) * 8) * ldw + n2 * 16 + ((lane >> 4) << 3));
            mma16816(c[2 * n2], a, b[0], b[1]);
            mma16816(c[2 * n2 + 1], a, b[2], b[3]);
        }
    }
    const int g = lane >> 2, q = lane & 3;
#pragma unroll
    for (int nt = 0; nt < K / 8; ++nt) {
        if constexpr (PAIR) {
            epi(16 * w + g, nt * 8 + 2 * q, c[nt][0], c[nt][1]);
            epi(16 * w + g + 8, nt * 8 + 2 * q, c[nt][2], c[nt][3]);
        } else {
            epi(16 * w + g, nt * 8 + 2 * q, c[nt][0]);
            epi(16 * w + g, nt * 8 + 2 * q + 1, c[nt][1]);
            epi(16 * w + g + 8, nt * 8 + 2 * q, c[nt][2]);
            epi(16 * w + g + 8, nt * 8 + 2 * q + 1, c[nt][3]);
        }
    }
}

// ---------------------------------------------------------------------------
// SIMT FP32 GEMMs (tiles of 16 points)
// ---------------------------------------------------------------------------
// Z[16 x 64] = H[16 x K] W^T: warp w rows 4w..4w+3; lane: row 4w + lane/8, 8 columns
template <int K, class Epi>
__device__ __forceinline__ void gemm_hwT_f32(const float *H, int ldh, const float *W, int ldw, int w, int lane, Epi epi)
{
    const int row = 4 * w + (lane >> 3), c0 = (lane & 7) * 8;
    float c[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) c[i] = 0.f;
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
        const float h = H[row * ldh + k];
#pragma unroll
        for (int i = 0; i < 8; ++i) c[i] = fmaf(h, W[(c0 + i) * ldw + k], c[i]);
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 8; ++i) epi(row, c0 + i, c[i]);
}

// G[64 x K] = D^T H over 16 points: warp w rows 16w.., lane: row 16w + lane/2, K/2 columns
template <int K, class Epi>
__device__ __forceinline__ void gemm_dTh_f32(const float *D, int ldd, const float *H, int ldh, int w, int lane, Epi epi)
{
    const int row = 16 * w + (lane >> 1), c0 = (lane & 1) * (K / 2);
    float c[K / 2];
#pragma unroll
    for (int i = 0; i < K / 2; ++i) c[i] = 0.f;
#pragma unroll 2
    for (int p = 0; p < 16; ++p) {
        const float d = D[p * ldd + row];
#pragma unroll
        for (int i = 0; i < K / 2; ++i) c[i] = fmaf(d, H[p * ldh + c0 + i], c[i]);
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < K / 2; ++i) epi(row, c0 + i, c[i]);
}

// P[16 x K] = D W: warp w points 4w.., lane: point 4w + lane/8, K/8 columns
// (PAIR as in gemm_dw_bf16).
template <int K, bool PAIR = false, class Epi>
__device__ __forceinline__ void gemm_dw_f32(const float *D, int ldd, const float *W, int ldw, int w, int lane, Epi epi)
{
    const int row = 4 * w + (lane >> 3), c0 = (lane & 7) * (K / 8);
    float c[K / 8];
#pragma unroll
    for (int i = 0; i < K / 8; ++i) c[i] = 0.f;
#pragma unroll 4
    for (int o = 0; o < WIDTH; ++o) {
        const float d = D[row * ldd + o];
#pragma unroll
        for (int i = 0; i < K / 8; ++i) c[i] = fmaf(d, W[o * ldw + c0 + i], c[i]);
    }
    __syncwarp();
    if constexpr (PAIR) {
        static_assert(K % 16 == 0, "column pairs");
#pragma unroll
        for (int i = 0; i < K / 8; i += 2) epi(row, c0 + i, c[i], c[i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < K / 8; ++i) epi(row, c0 + i, c[i]);
    }
}

// ---------------------------------------------------------------------------
// encodings
// ---------------------------------------------------------------------------
// Fourier: x, then per band j: sin(2^j pi x_c) (c = 0..2), cos(2^j pi x_c)
template <bool BF16, typename E>
__device__ __forceinline__ void encode_fourier(float x, int c, E *h)
{
    h[c] = to_e<E>(x);
    if (BF16) {
        float s, co;
        sincospif(x, &s, &co);
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            h[3 + 6 * j + c] = to_e<E>(s);
            h[3 + 6 * j + 3 + c] = to_e<E>(co);
            const float s2 = 2.f * s * co;  // double-angle step to the next band
            co = fmaf(-2.f * s, s, 1.f);
            s = s2;
        }
    } else {
        float a = x;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            float s, co;
            sincospif(a, &s, &co);
            h[3 + 6 * j + c] = to_e<E>(s);
            h[3 + 6 * j + 3 + c] = to_e<E>(co);
            a *= 2.f;
        }
    }
}

struct Corner8 {
    unsigned idx[8];
    float wt[8];
};

__device__ __forceinline__ void grid_corners(const float x[3], int level, const GridGeom &G, Corner8 &o)
{
    const int N = G.res[level];
    float f[3];
    int i0[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float p = fminf(fmaxf((x[d] + 1.f) * 0.5f, 0.f), 1.f);
        float pos = p * (float)N;
        int ii = (int)floorf(pos);
        if (ii > N - 1) ii = N - 1;
        i0[d] = ii;
        f[d] = pos - (float)ii;
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const unsigned vx = i0[0] + (c & 1), vy = i0[1] + ((c >> 1) & 1), vz = i0[2] + ((c >> 2) & 1);
        unsigned id;
        if (G.dense[level])
            id = vx + vy * (unsigned)(N + 1) + vz * (unsigned)(N + 1) * (unsigned)(N + 1);
        else
            id = (vx * 1u) ^ (vy * 2654435761u) ^ (vz * 805459861u);
        o.idx[c] = id & G.tmask;
        o.wt[c] = ((c & 1) ? f[0] : 1.f - f[0]) * (((c >> 1) & 1) ? f[1] : 1.f - f[1]) *
                  (((c >> 2) & 1) ? f[2] : 1.f - f[2]);
    }
}

// ---------------------------------------------------------------------------
// shared-memory layout of one block
// ---------------------------------------------------------------------------
template <int ENC, bool BF16, bool TRAIN>
struct Layout {
    typedef typename std::conditional<BF16, bf16, float>::type E;
    static constexpr int P = BF16 ? 64 : 16;   // points per tile
    static constexpr int PADE = BF16 ? 8 : 1;  // row padding (elements)
    static constexpr int L = Preset<ENC>::L;
    static constexpr int LDH0 = Preset<ENC>::K0P + PADE;
    static constexpr int LDH = WIDTH + PADE;
    __host__ __device__ static constexpr int ldw(int l) { return kin_pad<ENC>(l) + PADE; }
    __host__ __device__ static constexpr int w_off(int l) { return l == 0 ? 0 : w_off(l - 1) + WIDTH * ldw(l - 1); }
    static constexpr int W_ELEMS = w_off(L);
    static constexpr int DW_FLOATS = n_params<ENC>();
    // byte offsets
    static constexpr size_t o_w = 0;
    static constexpr size_t o_bias = (o_w + sizeof(E) * W_ELEMS + 15) / 16 * 16;
    static constexpr size_t o_wout = o_bias + sizeof(float) * L * WIDTH;
    static constexpr size_t o_h0 = (o_wout + sizeof(float) * (WIDTH + 4) + 15) / 16 * 16;
    static constexpr size_t o_hs = (o_h0 + sizeof(E) * P * LDH0 + 15) / 16 * 16;
    static constexpr size_t o_z = (o_hs + sizeof(E) * P * LDH + 15) / 16 * 16;
    static constexpr size_t o_d = o_z + (TRAIN ? sizeof(E) * L * P * LDH : 0);
    static constexpr size_t o_dw = (o_d + (TRAIN ? sizeof(E) * P * LDH : 0) + 15) / 16 * 16;
    static constexpr size_t o_pt = o_dw + (TRAIN ? sizeof(float) * DW_FLOATS : 0);
    static constexpr size_t bytes = o_pt + sizeof(float) * P * 4;  // per-point scratch: x, y, z, delta_out
};

template <int ENC, bool BF16, bool TRAIN>
__device__ __forceinline__ void nrf_body(const NrfArgs A, const float *__restrict__ xyz, long long n,
                                         const float *__restrict__ grad_out, float *__restrict__ out,
                                         float *__restrict__ g_params, float *__restrict__ g_table)
{
    typedef Layout<ENC, BF16, TRAIN> LY;
    typedef typename LY::E E;
    constexpr int P = LY::P, L = LY::L, K0P = Preset<ENC>::K0P;
    extern __shared__ __align__(16) unsigned char smem[];
    E *sW = (E *)(smem + LY::o_w);
    float *sBias = (float *)(smem + LY::o_bias);
    float *sWout = (float *)(smem + LY::o_wout);
    E *sH0 = (E *)(smem + LY::o_h0);
    E *sH = (E *)(smem + LY::o_hs);  // current activations
    E *sZ = (E *)(smem + LY::o_z);   // pre-activations Z_l of every layer (training)
    E *sD = (E *)(smem + LY::o_d);
    float *sDW = (float *)(smem + LY::o_dw);
    float *sPt = (float *)(smem + LY::o_pt);  // [P][4]
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    // grid geometry in shared memory: levels are indexed at run time
    __shared__ GridGeom sGrid;
    if (tid == 0) sGrid = A.grid;

    // weights -> shared (converted to E, zero padded), biases, output layer
    for (int l = 0; l < L; ++l) {
        const int kr = kin_real<ENC>(l), ld = LY::ldw(l);
        for (int i = tid; i < WIDTH * ld; i += NRF_NT) {
            const int o = i / ld, k = i - o * ld;
            float v = (k < kr) ? A.params[off_w<ENC>(l) + o * kr + k] : 0.f;
            sW[LY::w_off(l) + i] = to_e<E>(v);
        }
        for (int i = tid; i < WIDTH; i += NRF_NT) sBias[l * WIDTH + i] = A.params[off_b<ENC>(l) + i];
    }
    for (int i = tid; i <= WIDTH; i += NRF_NT) sWout[i] = A.params[off_wout<ENC>() + i];
    if (TRAIN)
        for (int i = tid; i < LY::DW_FLOATS; i += NRF_NT) sDW[i] = 0.f;
    __syncthreads();

    const long long n_tiles = (n + P - 1) / P;
    for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const long long p0 = tile * P;
        // ---- encoding -> H0
        for (int i = tid; i < P * 3; i += NRF_NT) {
            const int p = i / 3, c = i - 3 * p;
            const long long row = nrf_row(A, p0 + p, n);
            sPt[p * 4 + c] = row >= 0 ? xyz[row * 3 + c] : 0.f;
        }
        __syncthreads();
        if (ENC == MG_NRF_FOURIER) {
            for (int i = tid; i < P * 3; i += NRF_NT) {
                const int p = i / 3, c = i - 3 * p;
                encode_fourier<BF16, E>(sPt[p * 4 + c], c, sH0 + p * LY::LDH0);
            }
            constexpr int PADK = K0P - Preset<ENC>::K0;
            constexpr int PADD = PADK > 0 ? PADK : 1;
            for (int i = tid; i < P * PADK; i += NRF_NT) {
                const int p = i / PADD, k = Preset<ENC>::K0 + i % PADD;
                sH0[p * LY::LDH0 + k] = to_e<E>(0.f);
            }
        } else if (A.enc_mode == MG_NRF_ENC_LOAD) {
            // the features a forward call stored for these points (coalesced)
            const E *ec = (const E *)A.enc;
            for (int i = tid; i < P * 2 * GRID_LEVELS; i += NRF_NT) {
                const int p = i / (2 * GRID_LEVELS), k = i - p * (2 * GRID_LEVELS);
                sH0[p * LY::LDH0 + k] = (p0 + p < n) ? ec[(p0 + p) * (2 * GRID_LEVELS) + k] : to_e<E>(0.f);
            }
        } else {
            E *ec = A.enc_mode == MG_NRF_ENC_STORE ? (E *)A.enc : nullptr;
            for (int i = tid; i < P * GRID_LEVELS; i += NRF_NT) {
                const int p = i / GRID_LEVELS, lv = i - p * GRID_LEVELS;
                const float x[3] = {sPt[p * 4], sPt[p * 4 + 1], sPt[p * 4 + 2]};
                Corner8 cr;
                grid_corners(x, lv, sGrid, cr);
                const float2 *tb = (const float2 *)A.table + ((size_t)lv << sGrid.log2T);
                float f0 = 0.f, f1 = 0.f;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const float2 v = __ldg(tb + cr.idx[c]);
                    f0 = fmaf(cr.wt[c], v.x, f0);
                    f1 = fmaf(cr.wt[c], v.y, f1);
                }
                const E e0 = to_e<E>(f0), e1 = to_e<E>(f1);
                sH0[p * LY::LDH0 + 2 * lv] = e0;
                sH0[p * LY::LDH0 + 2 * lv + 1] = e1;
                if (ec && p0 + p < n) {
                    ec[(p0 + p) * (2 * GRID_LEVELS) + 2 * lv] = e0;
                    ec[(p0 + p) * (2 * GRID_LEVELS) + 2 * lv + 1] = e1;
                }
            }
        }
        __syncthreads();
        // ---- hidden layers: Z = H W^T + b, H = act(Z) (in place, per warp rows)
#pragma unroll
        for (int l = 0; l < L; ++l) {
            const E *Hin = (l == 0) ? sH0 : sH;
            const int ldin = (l == 0) ? LY::LDH0 : LY::LDH;
            const E *Wl = sW + LY::w_off(l);
            const float *bl = sBias + l * WIDTH;
            E *Zl = sZ + (size_t)l * P * LY::LDH;
            auto epi = [&](int r, int c, float v) {
                const float z = v + bl[c];
                if (TRAIN) Zl[r * LY::LDH + c] = to_e<E>(z);
                sH[r * LY::LDH + c] = to_e<E>(act<ENC, BF16>(z));
            };
            if (BF16) {
                if (l == 0)
                    gemm_hwT_bf16<K0P>((const bf16 *)Hin, ldin, (const bf16 *)Wl, LY::ldw(l), w, lane, epi);
                else
                    gemm_hwT_bf16<WIDTH>((const bf16 *)Hin, ldin, (const bf16 *)Wl, LY::ldw(l), w, lane, epi);
            } else {
                if (l == 0)
                    gemm_hwT_f32<K0P>((const float *)Hin, ldin, (const float *)Wl, LY::ldw(l), w, lane, epi);
                else
                    gemm_hwT_f32<WIDTH>((const float *)Hin, ldin, (const float *)Wl, LY::ldw(l), w, lane, epi);
            }
            __syncthreads();
        }
        const E *HL = sH;
        // ---- output layer: o = H w_out + b_out, r = s tanh(o); two threads per point
        for (int i = tid; i < 2 * P; i += NRF_NT) {
            const int p = i >> 1, half = i & 1;
            float acc = 0.f;
#pragma unroll 8
            for (int k = half * 32; k < half * 32 + 32; ++k) acc = fmaf(to_f(HL[p * LY::LDH + k]), sWout[k], acc);
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            const float o = acc + sWout[WIDTH];
            const float th = tanhf(o);
            if (half == 0) {
                const long long row = nrf_row(A, p0 + p, n);
                if (!TRAIN && row >= 0) {
                    if (A.idx)
                        atomicAdd(&out[row], A.out_scale * th);  // added to the indexed row
                    else
                        out[row] = A.out_scale * th;
                }
                if (TRAIN) {
                    const float go = row >= 0 ? grad_out[row] : 0.f;
                    sPt[p * 4 + 3] = go * A.out_scale * (1.f - th * th);  // dL/do
                }
            }
        }
        if (!TRAIN) {
            __syncthreads();
            continue;
        }
        __syncthreads();
        // ---- backward of the output layer: two threads per output, 32 points each
        float *dWout = sDW + off_wout<ENC>();
        for (int i = tid; i < 2 * WIDTH; i += NRF_NT) {
            const int k = i >> 1, half = i & 1;
            float acc = 0.f;
#pragma unroll 8
            for (int p = half * (P / 2); p < (half + 1) * (P / 2); ++p)
                acc = fmaf(sPt[p * 4 + 3], to_f(HL[p * LY::LDH + k]), acc);
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            if (half == 0) dWout[k] += acc;
        }
        if (tid == 0) {
            float acc = 0.f;
            for (int p = 0; p < P; ++p) acc += sPt[p * 4 + 3];
            dWout[WIDTH] += acc;
        }
        {
            const E *Zl = sZ + (size_t)(L - 1) * P * LY::LDH;
            for (int i = tid; i < P * WIDTH; i += NRF_NT) {
                const int p = i / WIDTH, k = i - p * WIDTH;
                const float ag = act_grad<ENC, BF16>(to_f(Zl[p * LY::LDH + k]));
                sD[p * LY::LDH + k] = to_e<E>(sPt[p * 4 + 3] * sWout[k] * ag);
            }
        }
        __syncthreads();
        // ---- hidden layers backward
#pragma unroll
        for (int l = L - 1; l >= 0; --l) {
            // the layer's input activations
            const E *Hin;
            int ldin;
            if (l == 0) {
                Hin = sH0;
                ldin = LY::LDH0;
            } else {
                const E *Zp = sZ + (size_t)(l - 1) * P * LY::LDH;
                for (int i = tid; i < P * WIDTH; i += NRF_NT) {
                    const int p = i / WIDTH, k = i - p * WIDTH;
                    sH[p * LY::LDH + k] = to_e<E>(act<ENC, BF16>(to_f(Zp[p * LY::LDH + k])));
                }
                Hin = sH;
                ldin = LY::LDH;
                __syncthreads();
            }
            // dW_l += D^T Hin  (rows = outputs owned by the warp)
            float *dWl = sDW + off_w<ENC>(l);
            const int kr = kin_real<ENC>(l);
            auto epi_g = [&](int o, int k, float v) {
                if (k < kr) dWl[o * kr + k] += v;
            };
            if (BF16) {
                if (l == 0)
                    gemm_dTh_bf16<K0P>((const bf16 *)sD, LY::LDH, (const bf16 *)Hin, ldin, w, lane, epi_g);
                else
                    gemm_dTh_bf16<WIDTH>((const bf16 *)sD, LY::LDH, (const bf16 *)Hin, ldin, w, lane, epi_g);
            } else {
                if (l == 0)
                    gemm_dTh_f32<K0P>((const float *)sD, LY::LDH, (const float *)Hin, ldin, w, lane, epi_g);
                else
                    gemm_dTh_f32<WIDTH>((const float *)sD, LY::LDH, (const float *)Hin, ldin, w, lane, epi_g);
            }
            // bias gradients: two threads per output, half of the points each
            float *dbl = sDW + off_b<ENC>(l);
            for (int i = tid; i < 2 * WIDTH; i += NRF_NT) {
                const int o = i >> 1, half = i & 1;
                float acc = 0.f;
#pragma unroll 8
                for (int p = half * (P / 2); p < (half + 1) * (P / 2); ++p) acc += to_f(sD[p * LY::LDH + o]);
                acc += __shfl_xor_sync(0xffffffffu, acc, 1);
                if (half == 0) dbl[o] += acc;
            }
            __syncthreads();
            if (l > 0) {
                // D <- (D W_l) * act'(Z_{l-1}), in place per warp rows
                const E *Zp = sZ + (size_t)(l - 1) * P * LY::LDH;
                const E *Wl = sW + LY::w_off(l);
                auto epi_d = [&](int p, int k, float v) {
                    sD[p * LY::LDH + k] = to_e<E>(v * act_grad<ENC, BF16>(to_f(Zp[p * LY::LDH + k])));
                };
                if (BF16) {
                    __syncwarp();
                    gemm_dw_bf16<WIDTH>((const bf16 *)sD, LY::LDH, (const bf16 *)Wl, LY::ldw(l), w, lane, epi_d);
                } else {
                    gemm_dw_f32<WIDTH>((const float *)sD, LY::LDH, (const float *)Wl, LY::ldw(l), w, lane, epi_d);
                }
                __syncthreads();
            } else if (ENC == MG_NRF_GRID && g_table) {
                // encoding gradient: dL/dfeatures = D W_0, scattered to the grid corners
                const E *W0 = sW + LY::w_off(0);
                auto epi_t = [&](int p, int k, float v0, float v1) {
                    // k = 2 * level: both features of one level, one float2 atomic per corner
                    if (p0 + p >= n) return;
                    const int lv = k >> 1;
                    const float x[3] = {sPt[p * 4], sPt[p * 4 + 1], sPt[p * 4 + 2]};
                    Corner8 cr;
                    grid_corners(x, lv, sGrid, cr);
                    float2 *tg = (float2 *)g_table + ((size_t)lv << sGrid.log2T);
                    // corners x, x + 1 in one 16-byte slot (indices differing in the
                    // lowest bit only) take one float4 atomic, else one float2 each
#pragma unroll
                    for (int c = 0; c < 8; c += 2) {
                        const unsigned ia = cr.idx[c], ib = cr.idx[c + 1];
                        const float2 ga = make_float2(cr.wt[c] * v0, cr.wt[c] * v1);
                        const float2 gb = make_float2(cr.wt[c + 1] * v0, cr.wt[c + 1] * v1);
                        if ((ia ^ ib) == 1u) {
                            atomicAdd((float4 *)&tg[ia & ~1u], (ia & 1u) ? make_float4(gb.x, gb.y, ga.x, ga.y)
                                                                          : make_float4(ga.x, ga.y, gb.x, gb.y));
                        } else {
                            atomicAdd(&tg[ia], ga);
                            atomicAdd(&tg[ib], gb);
                        }
                    }
                };
                if (BF16)
                    gemm_dw_bf16<K0P, true>((const bf16 *)sD, LY::LDH, (const bf16 *)W0, LY::ldw(0), w, lane, epi_t);
                else
                    gemm_dw_f32<K0P, true>((const float *)sD, LY::LDH, (const float *)W0, LY::ldw(0), w, lane, epi_t);
                __syncthreads();
            }
        }
    }
    if (TRAIN) {
        __syncthreads();
        for (int i = tid; i < LY::DW_FLOATS; i += NRF_NT) atomicAdd(&g_params[i], sDW[i]);
    }
}

// Two entry points with the same body: the forward (inference) kernels are
// compiled for 4 resident blocks of 4 warps per SM, which lets the compiler
// keep more grid gathers in flight (measured: 0.39 vs 0.81 ms per 2^20
// points for the grid BF16 forward); the training kernels keep the default
// register allocation (their shared memory limits residency anyway).
template <int ENC, bool BF16, bool TRAIN>
__global__ void __launch_bounds__(NRF_NT) k_nrf(NrfArgs A, const float *__restrict__ xyz, long long n,
                                                const float *__restrict__ grad_out, float *__restrict__ out,
                                                float *__restrict__ g_params, float *__restrict__ g_table)
{
    nrf_body<ENC, BF16, TRAIN>(A, xyz, n, grad_out, out, g_params, g_table);
}

template <int ENC, bool BF16, bool TRAIN>
__global__ void __launch_bounds__(NRF_NT, 4) k_nrf4(NrfArgs A, const float *__restrict__ xyz, long long n,
                                                    const float *__restrict__ grad_out, float *__restrict__ out,
                                                    float *__restrict__ g_params, float *__restrict__ g_table)
{
    nrf_body<ENC, BF16, TRAIN>(A, xyz, n, grad_out, out, g_params, g_table);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
GridGeom make_grid(const mg_nrf *net)
{
    GridGeom G;
    int lt = net->log2_table > 0 ? net->log2_table : 19;
    int nmin = net->n_min > 0 ? net->n_min : 16, nmax = net->n_max > 0 ? net->n_max : 512;
    double b = exp((log((double)nmax) - log((double)nmin)) / (GRID_LEVELS - 1));
    unsigned long long T = 1ull << lt;
    for (int l = 0; l < GRID_LEVELS; ++l) {
        int N = (int)floor((double)nmin * pow(b, (double)l));
        G.res[l] = N;
        unsigned long long v = (unsigned long long)(N + 1);
        G.dense[l] = (v * v * v <= T) ? 1 : 0;
    }
    G.tmask = (unsigned)(T - 1);
    G.log2T = lt;
    return G;
}

template <int ENC, bool BF16, bool TRAIN>
cudaError_t launch_nrf(const mg_nrf *net, const float *xyz, long long n, const float *grad_out, float *out,
                       float *g_params, float *g_table, const long long *idx, long long rows, cudaStream_t st)
{
    typedef Layout<ENC, BF16, TRAIN> LY;
    NrfArgs A;
    A.idx = idx;
    A.rows = rows;
    A.params = net->params;
    A.table = net->table;
    A.out_scale = net->out_scale;
    A.grid = make_grid(net);
    A.enc = ENC == MG_NRF_GRID ? net->enc : nullptr;
    A.enc_mode = (ENC == MG_NRF_GRID && net->enc) ? net->enc_mode : MG_NRF_ENC_NONE;
    auto kern = TRAIN ? k_nrf<ENC, BF16, TRAIN> : k_nrf4<ENC, BF16, TRAIN>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LY::bytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NRF_NT, LY::bytes);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long tiles = (n + LY::P - 1) / LY::P;
    long long grid = (long long)sms * (per_sm > 0 ? per_sm : 1);
    if (grid > tiles) grid = tiles;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, NRF_NT, LY::bytes, st>>>(A, xyz, n, grad_out, out, g_params, g_table);
    return cudaGetLastError();
}

}  // namespace

size_t mg_nrf_enc_bytes_impl(const mg_nrf *net, long long n)
{
    if (!net || n < 0 || net->encoding != MG_NRF_GRID) return 0;
    return (size_t)n * 2 * GRID_LEVELS * (net->precision == MG_NRF_BF16 ? 2 : 4);
}

int64_t mg_nrf_param_count_impl(int32_t encoding)
{
    if (encoding == MG_NRF_FOURIER) return n_params<MG_NRF_FOURIER>();
    if (encoding == MG_NRF_GRID) return n_params<MG_NRF_GRID>();
    return -1;
}

cudaError_t mg_launch_nrf(const mg_nrf *net, const float *xyz, long long n, const float *grad_out, float *out,
                          float *g_params, float *g_table, bool train, cudaStream_t st, const long long *idx,
                          long long rows)
{
    const bool bf = net->precision == MG_NRF_BF16;
    if (net->encoding == MG_NRF_FOURIER) {
        if (train)
            return bf ? launch_nrf<MG_NRF_FOURIER, true, true>(net, xyz, n, grad_out, out, g_params, g_table, idx, rows, st)
                      : launch_nrf<MG_NRF_FOURIER, false, true>(net, xyz, n, grad_out, out, g_params, g_table, idx, rows, st);
        return bf ? launch_nrf<MG_NRF_FOURIER, true, false>(net, xyz, n, grad_out, out, g_params, g_table, idx, rows, st)
                  : launch_nrf<MG_NRF_FOURIER, false, false>(net, xyz, n, grad_out, out, g_params, g_table, idx, rows, st);
    }
    if (train)
        return bf ? launch_nrf<MG_NRF_GRID, true, true>(net, xyz, n, grad_out, out, g_params, g_table, idx, rows, st)
                  : launch_nrf<MG_NRF_GRID, false, true>(net, xyz, n, grad_out, out, g_params, g_table, idx, rows, st);
    return bf ? launch_nrf<MG_NRF_GRID, true, false>(net, xyz, n, grad_out, out, g_params, g_table, idx, rows, st)
              : launch_nrf<MG_NRF_GRID, false, false>(net, xyz, n, grad_out, out, g_params, g_table, idx, rows, st);
}
