// mg_render.cu -- per-tile evaluation of the additive Gaussian mixture
// (Sec. 3.3.2, Eq. E7 with the slice profile) and its adjoint.
//
// K4 k_render_fwd : one warp per 16x16 tile; lane = one pixel column, 8 rows.
//     The tile's records are staged 32 at a time through shared memory and
//     read back by broadcast; per (record, voxel): q = A dx^2 + B2 dx dy +
//     C dy^2 (conic pre-scaled to log2 units), I += amp * 2^q.
// K5 k_render_bwd : the same sweep with dL/dI; per record each lane forms
//     six moments of w = g 2^q (sum w, w dx, w dy, w dx^2, w dx dy, w dy^2),
//     the warp reduce-scatters them with 8 shuffles, and six lanes issue one
//     atomic each into the record's moment slots. Nothing per pair is stored.
// K6 k_chain : per record, moments -> dL/d(centre, conic, amp) -> adjoint of
//     the record geometry -> dL/d(mean, quat, scale, alpha) (atomics).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mg_internal.cuh"

constexpr int RW = 4;     // warps (tiles) per block
constexpr int VPT = 8;    // voxels per thread (a column strip)

struct TileLoc {
    int W, H, px, py0;
    long long pixbase;
};

__device__ __forceinline__ TileLoc locate_tile(const StackTable &tab, int t, int lane)
{
    int s = 0;
    while (s + 1 < tab.n_stacks && t >= tab.tile_base[s + 1]) ++s;
    int local = t - tab.tile_base[s];
    int TX = tab.TX[s];
    int T = TX * tab.TY[s];
    int kk = local / T;
    int within = local - kk * T;
    int ty = within / TX, tx = within - ty * TX;
    TileLoc L;
    L.W = tab.W[s];
    L.H = tab.H[s];
    L.pixbase = tab.pix_base[s] + (long long)kk * L.H * L.W;
    L.px = tx * MG_TILE + (lane & 15);
    L.py0 = ty * MG_TILE + (lane >> 4) * VPT;
    return L;
}

__global__ void __launch_bounds__(32 * RW) k_render_fwd(StackTable tab, const unsigned *__restrict__ tile_off,
                                                        const unsigned *__restrict__ entries, long long cap_entries,
                                                        long long cap_records, const float4 *__restrict__ geo,
                                                        const float2 *__restrict__ geo2, float *__restrict__ out)
{
    __shared__ float4 sg[RW][32];
    __shared__ float2 sg2[RW][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * RW + w;
    if (t >= tab.n_tiles_total) return;  // whole warp
    TileLoc L = locate_tile(tab, t, lane);
    const float fpx = (float)L.px, fpy0 = (float)L.py0;
    unsigned e0 = tile_off[t], e1 = tile_off[t + 1];
    if ((long long)e1 > cap_entries) e1 = (unsigned)cap_entries;
    if (e0 > e1) e0 = e1;
    float acc[VPT];
#pragma unroll
    for (int v = 0; v < VPT; ++v) acc[v] = 0.f;
    // software pipeline: fetch the next chunk's records while evaluating
    float4 na = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 nb = make_float2(0.f, 0.f);
    if (e0 + lane < e1) {
        unsigned r = entries[e0 + lane];
        if ((long long)r < cap_records) {
            na = geo[r];
            nb = geo2[r];
        }
    }
    for (unsigned base = e0; base < e1; base += 32) {
        sg[w][lane] = na;
        sg2[w][lane] = nb;
        __syncwarp();
        unsigned nxt = base + 32 + lane;
        na = make_float4(0.f, 0.f, 0.f, 0.f);
        nb = make_float2(0.f, 0.f);
        if (nxt < e1) {
            unsigned r = entries[nxt];
            if ((long long)r < cap_records) {
                na = geo[r];
                nb = geo2[r];
            }
        }
        const int m = (int)min(32u, e1 - base);
        for (int j = 0; j < m; ++j) {
            const float4 a = sg[w][j];
            const float2 b = sg2[w][j];
            const float dx = fpx - a.x;
            const float dy0 = fpy0 - a.y;
            const float C = b.x, amp = b.y;
            const float cdy = C * dy0;
            const float a1 = fmaf(a.w, dx, cdy + cdy);
            const float a0 = fmaf(fmaf(a.z, dx, a.w * dy0), dx, cdy * dy0);
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                const float q = fmaf(fmaf(C, (float)v, a1), (float)v, a0);
                acc[v] = fmaf(amp, ex2_approx(q), acc[v]);
            }
        }
        __syncwarp();
    }
    if (L.px < L.W) {
#pragma unroll
        for (int v = 0; v < VPT; ++v)
            if (L.py0 + v < L.H) out[L.pixbase + (long long)(L.py0 + v) * L.W + L.px] = acc[v];
    }
}

// reduce-scatter of six per-lane values over the warp (8 shuffles); lanes
// 0,4,8 hold the sums of v0,v1,v2 and lanes 16,20,24 those of v3,v4,v5.
__device__ __forceinline__ float warp_reduce6(const float v[6], int lane, int &idx)
{
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float k[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float send = b4 ? v[i] : v[3 + i];
        float recv = __shfl_xor_sync(0xffffffffu, send, 16);
        k[i] = (b4 ? v[3 + i] : v[i]) + recv;
    }
    float s0 = b3 ? k[0] : k[2];
    float r0 = __shfl_xor_sync(0xffffffffu, s0, 8);
    float s1 = b3 ? k[1] : 0.f;
    float r1 = __shfl_xor_sync(0xffffffffu, s1, 8);
    float m0 = (b3 ? k[2] : k[0]) + r0;
    float m1 = b3 ? 0.f : (k[1] + r1);
    float s2 = b2 ? m0 : m1;
    float r2 = __shfl_xor_sync(0xffffffffu, s2, 4);
    float n = (b2 ? m1 : m0) + r2;
    n += __shfl_xor_sync(0xffffffffu, n, 2);
    n += __shfl_xor_sync(0xffffffffu, n, 1);
    int base = b4 ? 3 : 0;
    idx = b3 ? (b2 ? -1 : base + 2) : base + (b2 ? 1 : 0);
    if (lane & 3) idx = -1;
    return n;
}

__global__ void __launch_bounds__(32 * RW) k_render_bwd(StackTable tab, const unsigned *__restrict__ tile_off,
                                                        const unsigned *__restrict__ entries, long long cap_entries,
                                                        long long cap_records, const float4 *__restrict__ geo,
                                                        const float2 *__restrict__ geo2,
                                                        const float *__restrict__ grad_out, float *__restrict__ mom)
{
    __shared__ float4 sg[RW][32];
    __shared__ float2 sg2[RW][32];
    __shared__ unsigned sr[RW][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * RW + w;
    if (t >= tab.n_tiles_total) return;
    TileLoc L = locate_tile(tab, t, lane);
    const float fpx = (float)L.px, fpy0 = (float)L.py0;
    unsigned e0 = tile_off[t], e1 = tile_off[t + 1];
    if ((long long)e1 > cap_entries) e1 = (unsigned)cap_entries;
    if (e0 > e1) e0 = e1;
    float gv[VPT];
#pragma unroll
    for (int v = 0; v < VPT; ++v)
        gv[v] = (L.px < L.W && L.py0 + v < L.H) ? grad_out[L.pixbase + (long long)(L.py0 + v) * L.W + L.px] : 0.f;
    for (unsigned base = e0; base < e1; base += 32) {
        unsigned e = base + lane;
        unsigned r = 0xffffffffu;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 b = make_float2(0.f, 0.f);
        if (e < e1) {
            r = entries[e];
            if ((long long)r < cap_records) {
                a = geo[r];
                b = geo2[r];
            } else {
                r = 0xffffffffu;
            }
        }
        sg[w][lane] = a;
        sg2[w][lane] = b;
        sr[w][lane] = r;
        __syncwarp();
        const int m = (int)min(32u, e1 - base);
        for (int j = 0; j < m; ++j) {
            const float4 aa = sg[w][j];
            const float2 bb = sg2[w][j];
            const float dx = fpx - aa.x;
            const float dy0 = fpy0 - aa.y;
            const float C = bb.x;
            const float cdy = C * dy0;
            const float a1 = fmaf(aa.w, dx, cdy + cdy);
            const float a0 = fmaf(fmaf(aa.z, dx, aa.w * dy0), dx, cdy * dy0);
            float W0 = 0.f, M1 = 0.f, M2 = 0.f;
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                const float q = fmaf(fmaf(C, (float)v, a1), (float)v, a0);
                const float wv = gv[v] * ex2_approx(q);
                const float jc = (float)v - 0.5f * (VPT - 1);
                W0 += wv;
                M1 = fmaf(jc, wv, M1);
                M2 = fmaf(jc * jc, wv, M2);
            }
            const float dyc = dy0 + 0.5f * (VPT - 1);
            float mv[6];
            mv[0] = W0;
            mv[1] = dx * W0;
            mv[2] = fmaf(dyc, W0, M1);
            mv[3] = dx * mv[1];
            mv[4] = dx * mv[2];
            mv[5] = fmaf(dyc, fmaf(dyc, W0, M1 + M1), M2);
            int idx;
            float s = warp_reduce6(mv, lane, idx);
            const unsigned rr = sr[w][j];
            if (idx >= 0 && rr != 0xffffffffu) atomicAdd(&mom[(size_t)rr * 8 + idx], s);
        }
        __syncwarp();
    }
}

// Pair statistics over the bins: evaluated (record, in-image voxel) pairs and
// those inside the record's K-sigma ellipsoid (q >= thr in log2 units).
__global__ void __launch_bounds__(32 * RW) k_pair_count(StackTable tab, const unsigned *__restrict__ tile_off,
                                                        const unsigned *__restrict__ entries, long long cap_entries,
                                                        long long cap_records, const float4 *__restrict__ geo,
                                                        const float2 *__restrict__ geo2,
                                                        const float *__restrict__ thr, WsHeader *hdr)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * RW + w;
    if (t >= tab.n_tiles_total) return;
    TileLoc L = locate_tile(tab, t, lane);
    const float fpx = (float)L.px, fpy0 = (float)L.py0;
    unsigned e0 = tile_off[t], e1 = tile_off[t + 1];
    if ((long long)e1 > cap_entries) e1 = (unsigned)cap_entries;
    if (e0 > e1) e0 = e1;
    unsigned long long inside = 0, evald = 0;
    int nvalid = 0;
#pragma unroll
    for (int v = 0; v < VPT; ++v) nvalid += (L.px < L.W && L.py0 + v < L.H);
    for (unsigned e = e0; e < e1; ++e) {
        unsigned r = entries[e];
        if ((long long)r >= cap_records) continue;
        const float4 a = geo[r];
        const float C = geo2[r].x;
        const float th = thr[r];
        const float dx = fpx - a.x;
        const float dy0 = fpy0 - a.y;
        const float cdy = C * dy0;
        const float a1 = fmaf(a.w, dx, cdy + cdy);
        const float a0 = fmaf(fmaf(a.z, dx, a.w * dy0), dx, cdy * dy0);
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const float q = fmaf(fmaf(C, (float)v, a1), (float)v, a0);
            inside += (L.px < L.W && L.py0 + v < L.H && q >= th);
        }
        evald += nvalid;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        inside += __shfl_xor_sync(0xffffffffu, inside, o);
        evald += __shfl_xor_sync(0xffffffffu, evald, o);
    }
    if (lane == 0) {
        atomicAdd(&hdr->pairs_inside, inside);
        atomicAdd(&hdr->pairs_evaluated, evald);
    }
}

// ---------------------------------------------------------------------------
// K6: chain the per-record moments to the Gaussian parameters
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T c_exp(T x);
template <>
__device__ __forceinline__ float c_exp<float>(float x) { return expf(x); }
template <>
__device__ __forceinline__ double c_exp<double>(double x) { return exp(x); }

// Adjoint of the record geometry: (centre, conic, amp) of the record of a
// Gaussian on a slice, given dL/d(pcx, pcy, A, B2, C, amp).
template <typename T>
__device__ void geometry_adjoint(const float *mu, const float *q, const float *s, float alpha, const SliceDev &S,
                                 T gA, T gB2, T gC, T gpx, T gpy, T gamp, T gmu[3], T gq[4], T gs[3], T &galpha)
{
    // forward recomputation (same formulas as the record pass)
    T w = q[0], x = q[1], y = q[2], z = q[3];
    T R[3][3];
    R[0][0] = 1 - 2 * (y * y + z * z);
    R[0][1] = 2 * (x * y - w * z);
    R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);
    R[1][1] = 1 - 2 * (x * x + z * z);
    R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);
    R[2][1] = 2 * (y * z + w * x);
    R[2][2] = 1 - 2 * (x * x + y * y);
    T sc[3] = {s[0], s[1], s[2]};
    T P[3][3], g[3][3], Lm[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            P[a][c] = (T)S.Q[a] * R[0][c] + (T)S.Q[3 + a] * R[1][c] + (T)S.Q[6 + a] * R[2][c];
            g[a][c] = P[a][c] / sc[c];
            Lm[a][c] = P[a][c] * sc[c];
        }
    T p0 = (T)mu[0] - (T)S.t[0], p1 = (T)mu[1] - (T)S.t[1], p2 = (T)mu[2] - (T)S.t[2];
    T w0 = (T)S.Q[2] * p0 + (T)S.Q[5] * p1 + (T)S.Q[8] * p2;
    T Huw = g[0][0] * g[2][0] + g[0][1] * g[2][1] + g[0][2] * g[2][2];
    T Hvw = g[1][0] * g[2][0] + g[1][1] * g[2][1] + g[1][2] * g[2][2];
    T Hww = g[2][0] * g[2][0] + g[2][1] * g[2][1] + g[2][2] * g[2][2];
    T Suw = Lm[0][0] * Lm[2][0] + Lm[0][1] * Lm[2][1] + Lm[0][2] * Lm[2][2];
    T Svw = Lm[1][0] * Lm[2][0] + Lm[1][1] * Lm[2][1] + Lm[1][2] * Lm[2][2];
    T sig2 = (T)S.sig2;
    T Sww = Lm[2][0] * Lm[2][0] + Lm[2][1] * Lm[2][1] + Lm[2][2] * Lm[2][2] + sig2;
    T D = 1 + sig2 * Hww;
    T f = sig2 / D;
    T rD = (T)1 / sqrt(D);
    T E = c_exp<T>((T)(-0.5) * w0 * w0 / Sww);
    T amp = (T)alpha * rD * E;
    const T kap = (T)(-0.72134752044448170368);
    T dx = S.dx, dy = S.dy;
    // reverse
    T gKuu = gA * kap * dx * dx;
    T gKuv = gB2 * 2 * kap * dx * dy;
    T gKvv = gC * kap * dy * dy;
    T gcu = gpx / dx, gcv = gpy / dy;
    galpha = gamp * rD * E;
    T gD = gamp * amp * (T)(-0.5) / D;
    T gw0 = -gamp * amp * w0 / Sww;
    T gSww = gamp * amp * (T)0.5 * w0 * w0 / (Sww * Sww);
    T gdu = gcu, gdv = gcv;
    T gSuw = -gcu * w0 / Sww;
    T gSvw = -gcv * w0 / Sww;
    T cs = gcu * Suw + gcv * Svw;
    gw0 -= cs / Sww;
    gSww += cs * w0 / (Sww * Sww);
    T gHuu = gKuu, gHvv = gKvv, gHuv = gKuv;
    T gHuw = -f * (2 * gKuu * Huw + gKuv * Hvw);
    T gHvw = -f * (2 * gKvv * Hvw + gKuv * Huw);
    gD += sig2 / (D * D) * (gKuu * Huw * Huw + gKuv * Huw * Hvw + gKvv * Hvw * Hvw);
    T gHww = sig2 * gD;
    T gR[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) gR[r][c] = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        T gg0 = 2 * gHuu * g[0][c] + gHuv * g[1][c] + gHuw * g[2][c];
        T gg1 = 2 * gHvv * g[1][c] + gHuv * g[0][c] + gHvw * g[2][c];
        T gg2 = 2 * gHww * g[2][c] + gHuw * g[0][c] + gHvw * g[1][c];
        T gL0 = gSuw * Lm[2][c];
        T gL1 = gSvw * Lm[2][c];
        T gL2 = gSuw * Lm[0][c] + gSvw * Lm[1][c] + 2 * gSww * Lm[2][c];
        T gP0 = gg0 / sc[c] + gL0 * sc[c];
        T gP1 = gg1 / sc[c] + gL1 * sc[c];
        T gP2 = gg2 / sc[c] + gL2 * sc[c];
        gs[c] = -(gg0 * P[0][c] + gg1 * P[1][c] + gg2 * P[2][c]) / (sc[c] * sc[c]) +
                (gL0 * P[0][c] + gL1 * P[1][c] + gL2 * P[2][c]);
#pragma unroll
        for (int r = 0; r < 3; ++r) gR[r][c] = (T)S.Q[3 * r] * gP0 + (T)S.Q[3 * r + 1] * gP1 + (T)S.Q[3 * r + 2] * gP2;
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) gmu[r] = (T)S.Q[3 * r] * gdu + (T)S.Q[3 * r + 1] * gdv + (T)S.Q[3 * r + 2] * gw0;
    gq[0] = 2 * (-z * gR[0][1] + y * gR[0][2] + z * gR[1][0] - x * gR[1][2] - y * gR[2][0] + x * gR[2][1]);
    gq[1] = 2 * (y * gR[0][1] + z * gR[0][2] + y * gR[1][0] - 2 * x * gR[1][1] - w * gR[1][2] + z * gR[2][0] +
                 w * gR[2][1] - 2 * x * gR[2][2]);
    gq[2] = 2 * (-2 * y * gR[0][0] + x * gR[0][1] + w * gR[0][2] + x * gR[1][0] + z * gR[1][2] - w * gR[2][0] +
                 z * gR[2][1] - 2 * y * gR[2][2]);
    gq[3] = 2 * (-2 * z * gR[0][0] - w * gR[0][1] + x * gR[0][2] + w * gR[1][0] - 2 * z * gR[1][1] + y * gR[1][2] +
                 x * gR[2][0] + y * gR[2][1]);
}

__global__ void k_zero_mom(float4 *mom, const WsHeader *hdr, long long cap_records)
{
    long long n = (long long)hdr->n_records;
    if (n > cap_records) n = cap_records;
    long long nv = n * 2;  // 8 floats per record
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x)
        mom[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void k_chain(const WsHeader *hdr, long long cap_records, const float4 *__restrict__ geo,
                        const float2 *__restrict__ geo2, const int *__restrict__ gid, const int *__restrict__ rslice,
                        const float *__restrict__ mom, const SliceDev *__restrict__ slices, const float *mean,
                        const float *quat, const float *scale, const float *alpha, float f64_ratio, float *g_mean,
                        float *g_quat, float *g_scale, float *g_alpha)
{
    long long n = (long long)hdr->n_records;
    if (n > cap_records) n = cap_records;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        const float4 m0 = *(const float4 *)(mom + r * 8);
        const float2 m1 = *(const float2 *)(mom + r * 8 + 4);
        const float S0 = m0.x, Sx = m0.y, Sy = m0.z, Sxx = m0.w, Sxy = m1.x, Syy = m1.y;
        const float4 a = geo[r];
        const float2 b = geo2[r];
        const float A = a.z, B2 = a.w, C = b.x, amp = b.y;
        const float la = amp * 0.69314718055994531f;
        const float gA = la * Sxx, gB2 = la * Sxy, gC = la * Syy;
        const float gpx = -la * (2.f * A * Sx + B2 * Sy);
        const float gpy = -la * (B2 * Sx + 2.f * C * Sy);
        const float gamp = S0;
        const long long g = gid[r];
        const SliceDev Sd = slices[rslice[r]];
        float mu[3] = {mean[3 * g], mean[3 * g + 1], mean[3 * g + 2]};
        float qv[4] = {quat[4 * g], quat[4 * g + 1], quat[4 * g + 2], quat[4 * g + 3]};
        float sc[3] = {scale[3 * g], scale[3 * g + 1], scale[3 * g + 2]};
        float al = alpha[g];
        float mx = fmaxf(fmaxf(sc[0], sc[1]), sc[2]), mn = fminf(fminf(sc[0], sc[1]), sc[2]);
        float gm[3], gq[4], gs[3], ga;
        if (f64_ratio > 0.f && mx > f64_ratio * mn) {
            double dm[3], dq[4], ds[3], da;
            geometry_adjoint<double>(mu, qv, sc, al, Sd, gA, gB2, gC, gpx, gpy, gamp, dm, dq, ds, da);
            for (int i = 0; i < 3; ++i) gm[i] = (float)dm[i], gs[i] = (float)ds[i];
            for (int i = 0; i < 4; ++i) gq[i] = (float)dq[i];
            ga = (float)da;
        } else {
            geometry_adjoint<float>(mu, qv, sc, al, Sd, gA, gB2, gC, gpx, gpy, gamp, gm, gq, gs, ga);
        }
        // gradient on the unit sphere: drop the component along q (the
        // normalisation q = q_raw/|q_raw| removes it, and the rotation formula
        // is only a rotation for unit q)
        {
            float qq = qv[0] * qv[0] + qv[1] * qv[1] + qv[2] * qv[2] + qv[3] * qv[3];
            float rad = (gq[0] * qv[0] + gq[1] * qv[1] + gq[2] * qv[2] + gq[3] * qv[3]) / qq;
            for (int i = 0; i < 4; ++i) gq[i] -= rad * qv[i];
        }
        atomicAdd(&g_mean[3 * g], gm[0]);
        atomicAdd(&g_mean[3 * g + 1], gm[1]);
        atomicAdd(&g_mean[3 * g + 2], gm[2]);
        atomicAdd(&g_quat[4 * g], gq[0]);
        atomicAdd(&g_quat[4 * g + 1], gq[1]);
        atomicAdd(&g_quat[4 * g + 2], gq[2]);
        atomicAdd(&g_quat[4 * g + 3], gq[3]);
        atomicAdd(&g_scale[3 * g], gs[0]);
        atomicAdd(&g_scale[3 * g + 1], gs[1]);
        atomicAdd(&g_scale[3 * g + 2], gs[2]);
        atomicAdd(&g_alpha[g], ga);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void mg_launch_pair_count(const WsLayout &L, char *ws, const StackTable &tab, cudaStream_t st)
{
    WsHeader *hdr = (WsHeader *)(ws + L.hdr);
    cudaMemsetAsync(&hdr->pairs_inside, 0, 2 * sizeof(unsigned long long), st);
    int nt = tab.n_tiles_total;
    if (nt <= 0) return;
    MG_PROF(MG_ST_PAIRS, st);
    k_pair_count<<<(nt + RW - 1) / RW, 32 * RW, 0, st>>>(
        tab, (const unsigned *)(ws + L.tile_off), (const unsigned *)(ws + L.entries), L.cap_entries, L.cap_records,
        (const float4 *)(ws + L.rec_geo), (const float2 *)(ws + L.rec_geo2), (const float *)(ws + L.rec_thr), hdr);
}

void mg_launch_render_fwd(const WsLayout &L, char *ws, const StackTable &tab, float *out, cudaStream_t st)
{
    int nt = tab.n_tiles_total;
    if (nt <= 0) return;
    MG_PROF(MG_ST_RENDER_FWD, st);
    k_render_fwd<<<(nt + RW - 1) / RW, 32 * RW, 0, st>>>(
        tab, (const unsigned *)(ws + L.tile_off), (const unsigned *)(ws + L.entries), L.cap_entries, L.cap_records,
        (const float4 *)(ws + L.rec_geo), (const float2 *)(ws + L.rec_geo2), out);
}

void mg_launch_render_bwd(const WsLayout &L, char *ws, const SliceDev *slices, const StackTable &tab,
                          const float *grad_out, const float *mean, const float *quat, const float *scale,
                          const float *alpha, long long n, float f64_ratio, float *g_mean, float *g_quat,
                          float *g_scale, float *g_alpha, cudaStream_t st)
{
    const WsHeader *hdr = (const WsHeader *)(ws + L.hdr);
    cudaMemsetAsync(g_mean, 0, sizeof(float) * 3 * n, st);
    cudaMemsetAsync(g_quat, 0, sizeof(float) * 4 * n, st);
    cudaMemsetAsync(g_scale, 0, sizeof(float) * 3 * n, st);
    cudaMemsetAsync(g_alpha, 0, sizeof(float) * n, st);
    long long capv = L.cap_records * 2;
    int gz = (int)((capv + 255) / 256 < 148 * 16 ? (capv + 255) / 256 : 148 * 16);
    if (gz < 1) gz = 1;
    {
        MG_PROF(MG_ST_ZERO, st);
        k_zero_mom<<<gz, 256, 0, st>>>((float4 *)(ws + L.rec_mom), hdr, L.cap_records);
    }
    int nt = tab.n_tiles_total;
    {
        MG_PROF(MG_ST_RENDER_BWD, st);
        if (nt > 0)
            k_render_bwd<<<(nt + RW - 1) / RW, 32 * RW, 0, st>>>(
                tab, (const unsigned *)(ws + L.tile_off), (const unsigned *)(ws + L.entries), L.cap_entries,
                L.cap_records, (const float4 *)(ws + L.rec_geo), (const float2 *)(ws + L.rec_geo2), grad_out,
                (float *)(ws + L.rec_mom));
    }
    int gc = (int)((L.cap_records + 255) / 256 < 148 * 16 ? (L.cap_records + 255) / 256 : 148 * 16);
    if (gc < 1) gc = 1;
    MG_PROF(MG_ST_CHAIN, st);
    k_chain<<<gc, 256, 0, st>>>(hdr, L.cap_records, (const float4 *)(ws + L.rec_geo), (const float2 *)(ws + L.rec_geo2),
                                (const int *)(ws + L.rec_gid), (const int *)(ws + L.rec_slice),
                                (const float *)(ws + L.rec_mom), slices, mean, quat, scale, alpha, f64_ratio, g_mean,
                                g_quat, g_scale, g_alpha);
}
