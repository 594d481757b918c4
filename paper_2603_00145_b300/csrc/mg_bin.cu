// mg_bin.cu -- record pass and tile binning (count, exclusive scan, stable scatter).
//
// Sec. 3.3.1 of the paper restricts each voxel's sum to a local Gaussian set;
// here that set is decided per (Gaussian, slice) record and per 8x8 tile:
//   K1  k1_count / k1_emit / k_rec_fill : per (Gaussian, slice) K-sigma slab
//       test of the profile-convolved covariance, the tile rectangle of the
//       cut ellipse and its per-row culling (the FP32 record predicate of
//       mgauss.h, bit-exact), then the record's evaluation geometry (2D
//       centre, conic, amplitude).
//   K2  two-phase exclusive scans (no inter-block waiting).
//   K3  bin_hist / bin_colscan / bin_scatter : a counting sort of (record,
//       tile) entries by tile, chunked per slice, with warp-level ranking by
//       __match_any_sync so the order inside each tile list is reproducible.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mg_internal.cuh"

// ---------------------------------------------------------------------------
// slice table
// ---------------------------------------------------------------------------
__global__ void k_build_slices(StackIn in, SliceDev *out, int S)
{
    pdl_entry();
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S) return;
    int s = 0, base = 0, tile_base = 0;
    long long pix = 0;
    while (s < in.n_stacks && k >= base + in.n_slices[s]) {
        int TX = (in.W[s] + MG_TILE - 1) / MG_TILE, TY = (in.H[s] + MG_TILE - 1) / MG_TILE;
        tile_base += in.n_slices[s] * TX * TY;
        pix += (long long)in.n_slices[s] * in.H[s] * in.W[s];
        base += in.n_slices[s];
        ++s;
    }
    int kk = k - base;
    SliceDev d;
    d.W = in.W[s];
    d.H = in.H[s];
    d.TX = (d.W + MG_TILE - 1) / MG_TILE;
    d.TY = (d.H + MG_TILE - 1) / MG_TILE;
    d.tile_base = tile_base + kk * d.TX * d.TY;
    d.pix_base = pix + (long long)kk * d.H * d.W;
    d.stack = s;
    d.dx = in.dx[s];
    d.dy = in.dy[s];
    d.idx = __fdiv_rn(1.0f, d.dx);
    d.idy = __fdiv_rn(1.0f, d.dy);
    d.sig2 = in.sig2[s];
    d.pu2 = in.planes ? 0.f : in.pu2[s];
    d.pv2 = in.planes ? 0.f : in.pv2[s];
    d.hx = 0.5f * (float)(d.W - 1);
    d.hy = 0.5f * (float)(d.H - 1);
    d.same_frame = 0;
    if (in.planes) {
        d.same_frame = kk > 0;
        for (int i = 0; i < 9; ++i) d.Q[i] = (i % 4 == 0) ? 1.0f : 0.0f;
        d.t[0] = in.cx;
        d.t[1] = in.cy;
        // plane height evaluated in double, rounded once to float
        d.t[2] = (float)__dadd_rn((double)in.cz, __dmul_rn((double)in.h, (double)kk - 0.5 * (double)(in.n_slices[0] - 1)));
    } else {
        const float *x = in.xform[s] + (size_t)kk * 12;
        for (int i = 0; i < 9; ++i) d.Q[i] = x[i];
        for (int i = 0; i < 3; ++i) d.t[i] = x[9 + i];
        if (kk > 0) {
            const unsigned *a = (const unsigned *)x, *b = (const unsigned *)(x - 12);
            int same = 1;
            for (int i = 0; i < 9; ++i) same &= (a[i] == b[i]);
            d.same_frame = same;
        }
    }
    d.ent = __fadd_rn(__fadd_rn(__fmul_rn(d.Q[2], d.t[0]), __fmul_rn(d.Q[5], d.t[1])), __fmul_rn(d.Q[8], d.t[2]));
    out[k] = d;
}

void mg_launch_build_slices(const StackIn &in, SliceDev *out, int S, cudaStream_t st)
{
    MG_PROF(MG_ST_SLICES, st);
    launch_pdl(k_build_slices, dim3((S + 127) / 128), dim3(128), 0, st, in, out, S);
}

// ---------------------------------------------------------------------------
// two-phase exclusive scan of uint32 (block totals, then each block sums the
// totals before it and scans its range; totals in uint64, outputs saturate)
// ---------------------------------------------------------------------------
template <int NT>
__device__ unsigned long long block_exclusive_scan(unsigned long long v, unsigned long long *total)
{
    __shared__ unsigned long long wsum[NT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned long long s = (lane < NT / 32) ? wsum[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < NT / 32) wsum[lane] = s;  // inclusive
    }
    __syncthreads();
    unsigned long long pre = (w > 0 ? wsum[w - 1] : 0ull) + x - v;
    if (total) *total = wsum[NT / 32 - 1];
    __syncthreads();
    return pre;
}

constexpr int SCAN_NT = 512;
constexpr int SCAN_ITEMS = 4;

// Two independent scans may share the launches: blockIdx.y selects the array.
struct ScanPair {
    const unsigned *in[2];
    unsigned *out[2];
    long long n[2];
    unsigned long long *total[2];
};

__global__ void __launch_bounds__(SCAN_NT) k_scan_reduce(ScanPair sp, unsigned long long *parts)
{
    pdl_entry();
    const unsigned *in = sp.in[blockIdx.y];
    const long long n = sp.n[blockIdx.y];
    unsigned long long *part = parts + (size_t)blockIdx.y * gridDim.x;
    long long per = (n + gridDim.x - 1) / gridDim.x;
    long long b0 = (long long)blockIdx.x * per;
    long long b1 = b0 + per < n ? b0 + per : n;
    unsigned long long s = 0;
    for (long long i = b0 + threadIdx.x; i < b1; i += SCAN_NT) s += in[i];
    unsigned long long tot;
    block_exclusive_scan<SCAN_NT>(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_NT) k_scan_down(ScanPair sp, const unsigned long long *parts, int write_end)
{
    pdl_entry();
    const unsigned *in = sp.in[blockIdx.y];
    unsigned *out = sp.out[blockIdx.y];
    const long long n = sp.n[blockIdx.y];
    const unsigned long long *part = parts + (size_t)blockIdx.y * gridDim.x;
    long long per = (n + gridDim.x - 1) / gridDim.x;
    long long b0 = (long long)blockIdx.x * per;
    long long b1 = b0 + per < n ? b0 + per : n;
    // this block's offset: the totals of the blocks before it (at most MG_SCAN_BLOCKS)
    unsigned long long run;
    {
        unsigned long long v = 0;
        for (int i = threadIdx.x; i < (int)blockIdx.x; i += SCAN_NT) v += part[i];
        block_exclusive_scan<SCAN_NT>(v, &run);
    }
    for (long long base = b0; base < b1; base += (long long)SCAN_NT * SCAN_ITEMS) {
        unsigned v[SCAN_ITEMS];
        unsigned long long s = 0;
        long long i0 = base + (long long)threadIdx.x * SCAN_ITEMS;
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; ++j) {
            v[j] = (i0 + j < b1) ? in[i0 + j] : 0u;
            s += v[j];
        }
        unsigned long long tot;
        unsigned long long pre = block_exclusive_scan<SCAN_NT>(s, &tot) + run;
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; ++j) {
            if (i0 + j < b1) out[i0 + j] = pre > 0xffffffffull ? 0xffffffffu : (unsigned)pre;
            pre += v[j];
        }
        run += tot;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        if (write_end) out[n] = run > 0xffffffffull ? 0xffffffffu : (unsigned)run;
        if (sp.total[blockIdx.y]) *sp.total[blockIdx.y] = run;
    }
}

void mg_launch_scan_u32(const unsigned *in, unsigned *out, long long n_host, const unsigned long long *n_dev,
                        unsigned long long *part, unsigned long long *total_out, cudaStream_t st)
{
    (void)n_dev;
    ScanPair sp;
    sp.in[0] = sp.in[1] = in;
    sp.out[0] = sp.out[1] = out;
    sp.n[0] = sp.n[1] = n_host;
    sp.total[0] = sp.total[1] = total_out;
    int nb = MG_SCAN_BLOCKS;
    launch_pdl(k_scan_reduce, dim3(nb), dim3(SCAN_NT), 0, st, sp, part);
    launch_pdl(k_scan_down, dim3(nb), dim3(SCAN_NT), 0, st, sp, part, 1);
}

// two independent exclusive scans in the same two launches (part holds
// 2 * MG_SCAN_BLOCKS entries)
void mg_launch_scan2_u32(const unsigned *in0, unsigned *out0, long long n0, unsigned long long *total0,
                         const unsigned *in1, unsigned *out1, long long n1, unsigned long long *total1,
                         unsigned long long *part, cudaStream_t st)
{
    ScanPair sp;
    sp.in[0] = in0;
    sp.out[0] = out0;
    sp.n[0] = n0;
    sp.total[0] = total0;
    sp.in[1] = in1;
    sp.out[1] = out1;
    sp.n[1] = n1;
    sp.total[1] = total1;
    int nb = MG_SCAN_BLOCKS;
    launch_pdl(k_scan_reduce, dim3(nb, 2), dim3(SCAN_NT), 0, st, sp, part);
    launch_pdl(k_scan_down, dim3(nb, 2), dim3(SCAN_NT), 0, st, sp, part, 1);
}

// ---------------------------------------------------------------------------
// the FP32 record predicate (specified operation by operation in mgauss.h)
// ---------------------------------------------------------------------------
struct GaussPred {
    float mu[3];
    float Sg[3][3];  // covariance, FP32 as specified
};

__device__ __forceinline__ float dot3_rn(float a0, float a1, float a2, float b0, float b1, float b2)
{
    return __fadd_rn(__fadd_rn(__fmul_rn(a0, b0), __fmul_rn(a1, b1)), __fmul_rn(a2, b2));
}

__device__ __forceinline__ bool finite_f(float x) { return isfinite(x); }

// loads one Gaussian; false if any value is not finite or a scale is <= 0
__device__ bool load_gauss_pred(const float *mean, const float *quat, const float *scale, const float *alpha,
                                long long g, GaussPred &G)
{
    float m0 = mean[3 * g], m1 = mean[3 * g + 1], m2 = mean[3 * g + 2];
    float w = quat[4 * g], x = quat[4 * g + 1], y = quat[4 * g + 2], z = quat[4 * g + 3];
    float s0 = scale[3 * g], s1 = scale[3 * g + 1], s2 = scale[3 * g + 2];
    float a = alpha[g];
    bool ok = finite_f(m0) && finite_f(m1) && finite_f(m2) && finite_f(w) && finite_f(x) && finite_f(y) &&
              finite_f(z) && finite_f(s0) && finite_f(s1) && finite_f(s2) && finite_f(a) && s0 > 0.f && s1 > 0.f &&
              s2 > 0.f;
    G.mu[0] = m0;
    G.mu[1] = m1;
    G.mu[2] = m2;
    float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
    float xy = __fmul_rn(x, y), xz = __fmul_rn(x, z), yz = __fmul_rn(y, z);
    float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, z);
    float R[3][3];
    R[0][0] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(yy, zz)));
    R[0][1] = __fmul_rn(2.0f, __fsub_rn(xy, wz));
    R[0][2] = __fmul_rn(2.0f, __fadd_rn(xz, wy));
    R[1][0] = __fmul_rn(2.0f, __fadd_rn(xy, wz));
    R[1][1] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, zz)));
    R[1][2] = __fmul_rn(2.0f, __fsub_rn(yz, wx));
    R[2][0] = __fmul_rn(2.0f, __fsub_rn(xz, wy));
    R[2][1] = __fmul_rn(2.0f, __fadd_rn(yz, wx));
    R[2][2] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, yy)));
    float s[3] = {s0, s1, s2};
    float M[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) M[r][c] = __fmul_rn(R[r][c], s[c]);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = r; c < 3; ++c) {
            float v = dot3_rn(M[r][0], M[r][1], M[r][2], M[c][0], M[c][1], M[c][2]);
            G.Sg[r][c] = v;
            G.Sg[c][r] = v;
        }
    return ok;
}

struct PredOut {
    int il, ih, jl, jh;  // clamped pixel box
    float cu, cv, Cuu, Cvv, Cuv, r2, ru;  // the cut ellipse (slice mm) for the row culling
};

// The terms of the predicate that depend on the Gaussian's covariance and the
// slice's rotation only (reused across the slices of a stack without motion).
struct FrameTerms {
    float Lww;
    float wmu;  // e_n . mu
    float k2sww;  // K2 * (Lww + sig2) of the frame's profile (slab test)
    float Luw, Lvw, Luu, Lvv, Luv;
    bool full;  // Luw..Luv computed
};

__device__ __forceinline__ void frame_slab(const GaussPred &G, const float *Q, FrameTerms &f)
{
    float en0 = Q[2], en1 = Q[5], en2 = Q[8];
    float sn0 = dot3_rn(G.Sg[0][0], G.Sg[0][1], G.Sg[0][2], en0, en1, en2);
    float sn1 = dot3_rn(G.Sg[1][0], G.Sg[1][1], G.Sg[1][2], en0, en1, en2);
    float sn2 = dot3_rn(G.Sg[2][0], G.Sg[2][1], G.Sg[2][2], en0, en1, en2);
    f.Lww = dot3_rn(en0, en1, en2, sn0, sn1, sn2);
    f.wmu = dot3_rn(en0, en1, en2, G.mu[0], G.mu[1], G.mu[2]);
    f.full = false;
}

__device__ __forceinline__ void frame_full(const GaussPred &G, const float *Q, FrameTerms &f)
{
    float en0 = Q[2], en1 = Q[5], en2 = Q[8];
    float eu0 = Q[0], eu1 = Q[3], eu2 = Q[6];
    float ev0 = Q[1], ev1 = Q[4], ev2 = Q[7];
    float sn0 = dot3_rn(G.Sg[0][0], G.Sg[0][1], G.Sg[0][2], en0, en1, en2);
    float sn1 = dot3_rn(G.Sg[1][0], G.Sg[1][1], G.Sg[1][2], en0, en1, en2);
    float sn2 = dot3_rn(G.Sg[2][0], G.Sg[2][1], G.Sg[2][2], en0, en1, en2);
    f.Lww = dot3_rn(en0, en1, en2, sn0, sn1, sn2);
    f.wmu = dot3_rn(en0, en1, en2, G.mu[0], G.mu[1], G.mu[2]);
    f.Luw = dot3_rn(eu0, eu1, eu2, sn0, sn1, sn2);
    f.Lvw = dot3_rn(ev0, ev1, ev2, sn0, sn1, sn2);
    float su0 = dot3_rn(G.Sg[0][0], G.Sg[0][1], G.Sg[0][2], eu0, eu1, eu2);
    float su1 = dot3_rn(G.Sg[1][0], G.Sg[1][1], G.Sg[1][2], eu0, eu1, eu2);
    float su2 = dot3_rn(G.Sg[2][0], G.Sg[2][1], G.Sg[2][2], eu0, eu1, eu2);
    f.Luu = dot3_rn(eu0, eu1, eu2, su0, su1, su2);
    float sv0 = dot3_rn(G.Sg[0][0], G.Sg[0][1], G.Sg[0][2], ev0, ev1, ev2);
    float sv1 = dot3_rn(G.Sg[1][0], G.Sg[1][1], G.Sg[1][2], ev0, ev1, ev2);
    float sv2 = dot3_rn(G.Sg[2][0], G.Sg[2][1], G.Sg[2][2], ev0, ev1, ev2);
    f.Lvv = dot3_rn(ev0, ev1, ev2, sv0, sv1, sv2);
    f.Luv = dot3_rn(ev0, ev1, ev2, su0, su1, su2);
    f.full = true;
}

// The record-existence part of the predicate: the K-sigma slab test, with
// the frame's e_n . mu and K2 * Sww (f.k2sww set by the caller).
__device__ __forceinline__ bool slab_test(const FrameTerms &f, const SliceDev &S)
{
    const float w0 = __fsub_rn(f.wmu, S.ent);
    return __fmul_rn(w0, w0) <= f.k2sww;
}

__device__ __forceinline__ void pixel_box(const SliceDev &S, float cu, float cv, float ru, float rv, PredOut &o);

// The record predicate of mgauss.h given the frame terms (computed here when
// missing). Returns existence and the clamped pixel box.
__device__ __forceinline__ bool record_predicate(const GaussPred &G, const SliceDev &S, float K2, FrameTerms &f,
                                                 PredOut &o)
{
    const float *Q = S.Q;
    float p0 = __fsub_rn(G.mu[0], S.t[0]), p1 = __fsub_rn(G.mu[1], S.t[1]), p2 = __fsub_rn(G.mu[2], S.t[2]);
    float w0 = __fsub_rn(f.wmu, S.ent);
    float Sww = __fadd_rn(f.Lww, S.sig2);
    float ww = __fmul_rn(w0, w0);
    if (!(ww <= __fmul_rn(K2, Sww))) return false;
    if (!f.full) frame_full(G, Q, f);
    float u0 = dot3_rn(Q[0], Q[3], Q[6], p0, p1, p2);
    float v0 = dot3_rn(Q[1], Q[4], Q[7], p0, p1, p2);
    const float iSww = __fdiv_rn(1.0f, Sww);
    float r2 = __fsub_rn(K2, __fmul_rn(ww, iSww));
    if (r2 < 0.0f) r2 = 0.0f;
    float Cuu = __fsub_rn(f.Luu, __fmul_rn(__fmul_rn(f.Luw, f.Luw), iSww));
    if (Cuu < 0.0f) Cuu = 0.0f;
    Cuu = __fadd_rn(Cuu, S.pu2);
    float Cvv = __fsub_rn(f.Lvv, __fmul_rn(__fmul_rn(f.Lvw, f.Lvw), iSww));
    if (Cvv < 0.0f) Cvv = 0.0f;
    Cvv = __fadd_rn(Cvv, S.pv2);
    float cu = __fsub_rn(u0, __fmul_rn(__fmul_rn(f.Luw, w0), iSww));
    float cv = __fsub_rn(v0, __fmul_rn(__fmul_rn(f.Lvw, w0), iSww));
    float ru = __fsqrt_rn(__fmul_rn(r2, Cuu));
    float rv = __fsqrt_rn(__fmul_rn(r2, Cvv));
    pixel_box(S, cu, cv, ru, rv, o);
    o.cu = cu;
    o.cv = cv;
    o.Cuu = Cuu;
    o.Cvv = Cvv;
    o.Cuv = __fsub_rn(f.Luv, __fmul_rn(__fmul_rn(f.Luw, f.Lvw), iSww));
    o.r2 = r2;
    o.ru = ru;
    return true;
}

// Per-row culling of the tile rectangle (the FP32 rule of mgauss.h): for each
// of the first eight tile rows, the tile columns that the cut ellipse reaches
// over the row's pixel band. The band's extreme ellipse point on each side is
// the ellipse's own (at v = cv -/+ Cuv ru/Cuu) when it lies in the band, else
// on the band edge nearest to it (the boundary is convex in v), where the
// chord is centred at cu + (Cuv/Cvv) d with half-width
// sqrt((r2 - d^2/Cvv)(Cuu - Cuv^2/Cvv)). Extents grow by ru/256 + dx/1024.
// Rectangles one tile wide are not culled. 8 bits per row: insets from the
// rectangle's left (low nibble) and right edges, each at most 15.
// the chord of the cut ellipse at v (v != the side's extreme): centre and half-width
__device__ __forceinline__ float2 row_chord(float v, const PredOut &o, float g, float h2, float iCvv)
{
    const float d = __fsub_rn(v, o.cv);
    const float t = fmaxf(__fsub_rn(o.r2, __fmul_rn(__fmul_rn(d, d), iCvv)), 0.f);
    return make_float2(__fadd_rn(o.cu, __fmul_rn(g, d)), __fsqrt_rn(__fmul_rn(t, h2)));
}

__device__ __forceinline__ unsigned long long row_insets(const SliceDev &S, const PredOut &o)
{
    if (!(o.r2 > 0.f) || !(o.Cuu > 0.f) || !(o.Cvv > 0.f) || o.il > o.ih) return 0ull;
    const int tx0 = o.il / MG_TILE, tx1 = o.ih / MG_TILE, ty0 = o.jl / MG_TILE, ty1 = o.jh / MG_TILE;
    if (tx1 == tx0) return 0ull;
    const float idx = S.idx;
    const float e = __fdiv_rn(o.ru, o.Cuu);
    const float iCvv = __fdiv_rn(1.0f, o.Cvv);
    const float g = __fmul_rn(o.Cuv, iCvv);
    const float h2 = fmaxf(__fsub_rn(o.Cuu, __fmul_rn(o.Cuv, g)), 0.f);
    const float m = __fadd_rn(__fmul_rn(o.ru, 0.00390625f), __fmul_rn(S.dx, 0.0009765625f));
    const float ce = __fmul_rn(o.Cuv, e);
    const float vL = __fsub_rn(o.cv, ce), vR = __fadd_rn(o.cv, ce);
    const float fil = (float)o.il, fih = (float)o.ih;
    unsigned long long out = 0ull;
    const int last = min(ty1 - ty0, 7);
    for (int n = 0; n <= last; ++n) {
        const int ty = ty0 + n;
        const int a = max(o.jl, MG_TILE * ty), b = min(o.jh, MG_TILE * ty + MG_TILE - 1);
        const float va = __fmul_rn(__fsub_rn((float)a, S.hy), S.dy);
        const float vb = __fmul_rn(__fsub_rn((float)b, S.hy), S.dy);
        // both sides usually clamp to the same band edge: one chord serves both
        const float wl = fminf(fmaxf(vL, va), vb), wr = fminf(fmaxf(vR, va), vb);
        const bool el = wl == vL, er = wr == vR;
        float2 cl = make_float2(0.f, 0.f), cr = make_float2(0.f, 0.f);
        if (!el) cl = row_chord(wl, o, g, h2, iCvv);
        if (!er) cr = (!el && wr == wl) ? cl : row_chord(wr, o, g, h2, iCvv);
        const float left = el ? __fsub_rn(o.cu, o.ru) : __fsub_rn(cl.x, cl.y);
        const float right = er ? __fadd_rn(o.cu, o.ru) : __fadd_rn(cr.x, cr.y);
        const float lo = fmaxf(ceilf(__fadd_rn(__fmul_rn(__fsub_rn(left, m), idx), S.hx)), fil);
        const float hi = fminf(floorf(__fadd_rn(__fmul_rn(__fadd_rn(right, m), idx), S.hx)), fih);
        int l, r;
        if (!(lo <= hi)) {  // no voxel column of the band: the row lists nothing
            l = tx1 - tx0 + 1;
            r = 0;
        } else {
            l = (int)lo / MG_TILE - tx0;
            r = tx1 - (int)hi / MG_TILE;
        }
        l = min(l, 15);
        r = min(r, 15);
        out |= (unsigned long long)(l | (r << 4)) << (8 * n);
    }
    return out;
}

// one 16-byte load of a record's listed tiles
__device__ __forceinline__ RecTiles load_tiles(const RecTiles *p)
{
    const uint4 u = __ldg((const uint4 *)p);
    RecTiles t;
    t.rect = make_ushort4((unsigned short)(u.x & 0xFFFFu), (unsigned short)(u.x >> 16),
                          (unsigned short)(u.y & 0xFFFFu), (unsigned short)(u.y >> 16));
    t.inset = (unsigned long long)u.z | ((unsigned long long)u.w << 32);
    return t;
}

// the tile columns [first, last] that record row n (0-based in its rectangle) lists
__device__ __forceinline__ int2 row_span(const ushort4 &rc, unsigned long long ins, int n)
{
    const unsigned b = n < 8 ? (unsigned)(ins >> (8 * n)) & 0xFFu : 0u;
    return make_int2((int)rc.x + (int)(b & 15u), (int)rc.z - (int)(b >> 4));
}

// The tile (index ty * TX + tx in its slice) of a record's i-th listed tile
// in row-major order (i below the record's listed count): the first eight
// rows by their insets, the rows after them whole.
__device__ __forceinline__ int nth_listed_tile(const ushort4 &rc, unsigned long long ins, unsigned i, int TX)
{
    int n = 0;
    const int h = (int)rc.w - (int)rc.y + 1;
    for (; n < 8 && n < h; ++n) {
        const int2 sp = row_span(rc, ins, n);
        const unsigned w = sp.y >= sp.x ? (unsigned)(sp.y - sp.x + 1) : 0u;
        if (i < w) return ((int)rc.y + n) * TX + sp.x + (int)i;
        i -= w;
    }
    const unsigned W = (unsigned)((int)rc.z - (int)rc.x + 1);
    return ((int)rc.y + n + (int)(i / W)) * TX + (int)rc.x + (int)(i % W);
}

// the number of tiles a record lists (its rectangle less the first eight
// rows' insets)
__device__ __forceinline__ int listed_count(const ushort4 &rc, unsigned long long ins)
{
    if (rc.x > rc.z || rc.y > rc.w) return 0;
    const int h = (int)rc.w - (int)rc.y + 1, W = (int)rc.z - (int)rc.x + 1;
    int a = 0;
#pragma unroll
    for (int n = 0; n < 8; ++n) {
        const unsigned b = (unsigned)(ins >> (8 * n)) & 0xFFu;
        if (n < h) a += max(W - (int)(b & 15u) - (int)(b >> 4), 0);
    }
    return a + max(h - 8, 0) * W;
}

// does the record list tile (tx, ty)?
__device__ __forceinline__ bool lists_tile(const ushort4 &rc, unsigned long long ins, int tx, int ty)
{
    if (ty < (int)rc.y || ty > (int)rc.w) return false;
    const int2 sp = row_span(rc, ins, ty - (int)rc.y);
    return tx >= sp.x && tx <= sp.y;
}

// A batch's records listed apart (large, while the chunk's list has room):
// the same rule in the histogram and the scatter. nbig: the chunk's list
// length so far (updated); returns the lane's slot, or -1.
__device__ __forceinline__ int big_slot(int area, unsigned &nbig, unsigned lt)
{
    const bool big = area > BIG_AREA;
    const unsigned bm = __ballot_sync(0xffffffffu, big);
    const unsigned slot = nbig + __popc(bm & lt);
    nbig = min(nbig + (unsigned)__popc(bm), (unsigned)BIG_MAX);
    return big && slot < (unsigned)BIG_MAX ? (int)slot : -1;
}

// lane j's record tiles, fetched by every lane of the warp
__device__ __forceinline__ void shfl_tiles(const ushort4 &rc, unsigned long long ins, int j, ushort4 &rj,
                                           unsigned long long &ij)
{
    const unsigned a0 = __shfl_sync(0xffffffffu, (unsigned)rc.x | ((unsigned)rc.y << 16), j);
    const unsigned a1 = __shfl_sync(0xffffffffu, (unsigned)rc.z | ((unsigned)rc.w << 16), j);
    const unsigned b0 = __shfl_sync(0xffffffffu, (unsigned)ins, j);
    const unsigned b1 = __shfl_sync(0xffffffffu, (unsigned)(ins >> 32), j);
    rj = make_ushort4((unsigned short)(a0 & 0xFFFFu), (unsigned short)(a0 >> 16), (unsigned short)(a1 & 0xFFFFu),
                      (unsigned short)(a1 >> 16));
    ij = (unsigned long long)b0 | ((unsigned long long)b1 << 32);
}

// A batch of 32 records is flattened (one entry per lane per round, in
// record-major order) when its largest record holds well over the mean: a
// lane walking its own record's tiles would keep the warp for the largest one.
__device__ __forceinline__ bool flatten_batch(int maxa, unsigned total)
{
    const unsigned rounds = (total + 31u) / 32u;
    return (unsigned)maxa > rounds + rounds / 2u + 2u;
}

// The batch lane that owns flattened entry e: the first lane whose inclusive
// prefix of listed-tile counts exceeds e (e below the batch total).
__device__ __forceinline__ int entry_owner(unsigned incl, unsigned e)
{
    int lo = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const unsigned v = __shfl_sync(0xffffffffu, incl, lo + step - 1);
        if (v <= e) lo += step;
    }
    return lo;
}

// The pixel box of [cu - ru, cu + ru] x [cv - rv, cv + rv] (slice mm), clamped
// to the image; an empty box is stored as the tile rectangle (1,1,0,0).
__device__ __forceinline__ void pixel_box(const SliceDev &S, float cu, float cv, float ru, float rv, PredOut &o)
{
    const float idx = S.idx, idy = S.idy;  // the correctly rounded 1/dx, 1/dy
    float il = ceilf(__fadd_rn(__fmul_rn(__fsub_rn(cu, ru), idx), S.hx));
    float ih = floorf(__fadd_rn(__fmul_rn(__fadd_rn(cu, ru), idx), S.hx));
    float jl = ceilf(__fadd_rn(__fmul_rn(__fsub_rn(cv, rv), idy), S.hy));
    float jh = floorf(__fadd_rn(__fmul_rn(__fadd_rn(cv, rv), idy), S.hy));
    float Wm1 = (float)(S.W - 1), Hm1 = (float)(S.H - 1);
    if (!(il <= ih) || !(jl <= jh) || !(il <= Wm1) || !(ih >= 0.0f) || !(jl <= Hm1) || !(jh >= 0.0f)) {
        o.il = o.jl = MG_TILE;  // empty box: tile rectangle (1,1,0,0)
        o.ih = o.jh = 0;
        return;
    }
    if (il < 0.0f) il = 0.0f;
    if (jl < 0.0f) jl = 0.0f;
    if (ih > Wm1) ih = Wm1;
    if (jh > Hm1) jh = Hm1;
    o.il = (int)il;
    o.ih = (int)ih;
    o.jl = (int)jl;
    o.jh = (int)jh;
}

// ---------------------------------------------------------------------------
// record geometry for the evaluation kernels (not bit-specified; FP32, or
// FP64 for near-degenerate Gaussians). Profile-convolved covariance
// Sigma' = Sigma_L + sig2 e_w e_w^T in slice coordinates; its precision block
// on the plane (Sherman-Morrison on Sigma_L^-1 = g g^T, g = Q^T R diag(1/s)),
// conditional centre and amplitude alpha |Sigma_L|^1/2 |Sigma'|^-1/2 e^{-w0^2/2Sww}.
// ---------------------------------------------------------------------------
template <typename T>
struct RecGeomT {
    T pcx, pcy, A, B2, C, amp, thr;
};

template <typename T>
__device__ __forceinline__ T t_exp(T x);
template <>
__device__ __forceinline__ float t_exp<float>(float x) { return expf(x); }
template <>
__device__ __forceinline__ double t_exp<double>(double x) { return exp(x); }

template <typename T>
__device__ __forceinline__ T t_rsqrt(T x);
template <>
__device__ __forceinline__ float t_rsqrt<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double t_rsqrt<double>(double x) { return 1.0 / sqrt(x); }

template <typename T>
__device__ __forceinline__ T t_rcp(T x);
template <>
__device__ __forceinline__ float t_rcp<float>(float x) { return __frcp_rn(x); }
template <>
__device__ __forceinline__ double t_rcp<double>(double x) { return 1.0 / x; }

template <typename T>
__device__ void record_geometry(const float *mu, const float *q, const float *s, float alpha, const SliceDev &S,
                                float K2, RecGeomT<T> &o)
{
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
    T isc[3] = {t_rcp<T>(sc[0]), t_rcp<T>(sc[1]), t_rcp<T>(sc[2])};
    T P[3][3];  // P[a][c] = e_a . R_c,  a in (u, v, w)
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            P[a][c] = (T)S.Q[a] * R[0][c] + (T)S.Q[3 + a] * R[1][c] + (T)S.Q[6 + a] * R[2][c];
    T p0 = (T)mu[0] - (T)S.t[0], p1 = (T)mu[1] - (T)S.t[1], p2 = (T)mu[2] - (T)S.t[2];
    T du = (T)S.Q[0] * p0 + (T)S.Q[3] * p1 + (T)S.Q[6] * p2;
    T dv = (T)S.Q[1] * p0 + (T)S.Q[4] * p1 + (T)S.Q[7] * p2;
    T w0 = (T)S.Q[2] * p0 + (T)S.Q[5] * p1 + (T)S.Q[8] * p2;
    T g[3][3], L[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            g[a][c] = P[a][c] * isc[c];
            L[a][c] = P[a][c] * sc[c];
        }
    T Huu = g[0][0] * g[0][0] + g[0][1] * g[0][1] + g[0][2] * g[0][2];
    T Huv = g[0][0] * g[1][0] + g[0][1] * g[1][1] + g[0][2] * g[1][2];
    T Hvv = g[1][0] * g[1][0] + g[1][1] * g[1][1] + g[1][2] * g[1][2];
    T Huw = g[0][0] * g[2][0] + g[0][1] * g[2][1] + g[0][2] * g[2][2];
    T Hvw = g[1][0] * g[2][0] + g[1][1] * g[2][1] + g[1][2] * g[2][2];
    T Hww = g[2][0] * g[2][0] + g[2][1] * g[2][1] + g[2][2] * g[2][2];
    T Suw = L[0][0] * L[2][0] + L[0][1] * L[2][1] + L[0][2] * L[2][2];
    T Svw = L[1][0] * L[2][0] + L[1][1] * L[2][1] + L[1][2] * L[2][2];
    T Sww = L[2][0] * L[2][0] + L[2][1] * L[2][1] + L[2][2] * L[2][2] + (T)S.sig2;
    T iSww = t_rcp<T>(Sww);
    T sig2 = (T)S.sig2;
    T D = 1 + sig2 * Hww;
    T rD = t_rsqrt<T>(D);
    T f = sig2 * rD * rD;  // sig2 / D
    T Kuu = Huu - f * Huw * Huw;
    T Kuv = Huv - f * Huw * Hvw;
    T Kvv = Hvv - f * Hvw * Hvw;
    T wS = w0 * iSww;
    T cu = du - Suw * wS;
    T cv = dv - Svw * wS;
    const T kap = (T)(-0.72134752044448170368);  // -log2(e)/2
    T dx = S.dx, dy = S.dy;
    // FP32: the slice's correctly rounded reciprocals (what t_rcp gives)
    const T idx = sizeof(T) == 4 ? (T)S.idx : t_rcp<T>(dx), idy = sizeof(T) == 4 ? (T)S.idy : t_rcp<T>(dy);
    o.pcx = cu * idx + (T)S.hx;
    o.pcy = cv * idy + (T)S.hy;
    o.A = kap * Kuu * dx * dx;
    o.B2 = 2 * kap * Kuv * dx * dy;
    o.C = kap * Kvv * dy * dy;
    T amp = (T)alpha * rD * t_exp<T>((T)(-0.5) * w0 * wS);
    if (S.pu2 > 0.f || S.pv2 > 0.f) {
        // in-plane PSF: the conditional covariance C = K^-1 gains diag(pu2, pv2):
        // (K^-1 + P)^-1 = [[Kuu + pv2 |K|, Kuv], [Kuv, Kvv + pu2 |K|]] / m,
        // m = det(I + P K) = 1 + pu2 Kuu + pv2 Kvv + pu2 pv2 |K|; |Sigma'| grows by m
        const T pu2 = (T)S.pu2, pv2 = (T)S.pv2;
        const T dK = Kuu * Kvv - Kuv * Kuv;
        const T m = 1 + pu2 * Kuu + pv2 * Kvv + pu2 * pv2 * dK;
        const T im = t_rcp<T>(m);
        const T nu = (Kuu + pv2 * dK) * im, nv = (Kvv + pu2 * dK) * im;
        Kuv = Kuv * im;
        Kuu = nu;
        Kvv = nv;
        amp = amp * t_rsqrt<T>(m);
        o.A = kap * Kuu * dx * dx;
        o.B2 = 2 * kap * Kuv * dx * dy;
        o.C = kap * Kvv * dy * dy;
    }
    o.amp = amp;
    T r2 = (T)K2 - w0 * wS;  // the cut ellipse is q <= r2 (natural units)
    o.thr = kap * (r2 > 0 ? r2 : (T)0);
}

__device__ __forceinline__ bool is_degenerate(const float *s, float ratio)
{
    if (!(ratio > 0.0f)) return false;
    float mx = fmaxf(fmaxf(s[0], s[1]), s[2]);
    float mn = fminf(fminf(s[0], s[1]), s[2]);
    return mx > ratio * mn;
}

// ---------------------------------------------------------------------------
// K1: count, emit and geometry passes
//   k1_count : one thread per Gaussian sweeps every slice (frame terms reused
//              while the rotation is unchanged); writes a bit per (Gaussian,
//              slice) record, per-(slice, warp) record counts and per-Gaussian
//              counts.
//   k1_emit  : revisits only the set bits; the exclusive scan of the
//              (slice, warp) counts gives slice-major, Gaussian-ascending
//              record positions; writes record identity, tile rectangle and
//              the Gaussian-major record list used by the chain.
//   k_rec_geom : one thread per record, evaluation geometry.
// ---------------------------------------------------------------------------
constexpr int K1_NT = 256;
constexpr int K1_SMEM_SLICES = 256;  // slices staged in shared memory at a time

// One thread per (Gaussian, window of 32 slices): blockIdx.y is the window
// (staged in shared memory), so the tests of one Gaussian run in parallel
// over the windows; the frame terms are formed at the first slice of each run
// of slices sharing a frame. gcnt must be zero on entry (summed over the
// windows with one atomic per thread).
// Within a window, slices form runs that share a frame; along a run whose
// plane offsets e_n . t are monotone, the slab test can only pass on the
// contiguous range of slices whose offset lies within the slab's half-width
// of e_n . mu. Each lane finds that range (grown so that FP32 rounding cannot
// exclude a passing slice) by bisection, and the warp runs the exact test
// over the union of its lanes' ranges only: every slice outside the union
// fails the test, so the bits and counts are the exact test's.
__global__ void __launch_bounds__(K1_NT) k1_count(const SliceDev *__restrict__ slices, int S,
                                                  const float *mean, const float *quat, const float *scale,
                                                  const float *alpha, long long n, float K2, float f64_ratio,
                                                  unsigned *cnt, long long NW, unsigned *gcnt, unsigned *bits,
                                                  WsHeader *hdr)
{
    pdl_entry();
    __shared__ SliceDev ssl[32];
    __shared__ float sent[32];
    __shared__ int run_end[32], run_dir[32];  // at a run's first slice: its last slice, +1/-1 monotone, 0 not
    __shared__ float sig2max;                  // the largest profile variance in the window
    const long long g = (long long)blockIdx.x * K1_NT + threadIdx.x;
    const long long wg = g >> 5;
    const int lane = threadIdx.x & 31;
    const int wd = blockIdx.y, k0 = wd * 32, nk = min(32, S - k0);
    GaussPred G;
    bool valid = false;
    if (g < n) {
        valid = load_gauss_pred(mean, quat, scale, alpha, g, G);
        if (wd == 0) {
            if (!valid) atomicOr(&hdr->flags, MG_FLAG_NOT_FINITE);
            float sc[3] = {scale[3 * g], scale[3 * g + 1], scale[3 * g + 2]};
            if (valid && is_degenerate(sc, f64_ratio)) atomicOr(&hdr->flags, MG_FLAG_DEGENERATE);
        }
    }
    FrameTerms f;
    f.full = false;
    {
        for (int i = threadIdx.x; i < nk; i += K1_NT) {
            ssl[i] = slices[k0 + i];
            sent[i] = slices[k0 + i].ent;
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int l = threadIdx.x;
            const bool in = l < nk;
            const bool first = in && (l == 0 || !ssl[l].same_frame);
            const unsigned starts = __ballot_sync(0xffffffffu, first);
            const unsigned inc = __ballot_sync(0xffffffffu, in && !first && sent[l] > sent[l - 1]);
            const unsigned dec = __ballot_sync(0xffffffffu, in && !first && sent[l] < sent[l - 1]);
            if (first) {
                const unsigned later = l < 31 ? starts & (0xffffffffu << (l + 1)) : 0u;
                const int e = later ? __ffs(later) - 2 : nk - 1;
                const unsigned upto = e >= 31 ? 0xffffffffu : ((1u << (e + 1)) - 1u);
                const unsigned steps = e > l ? upto & ~((1u << (l + 1)) - 1u) : 0u;
                run_end[l] = e;
                run_dir[l] = (inc & steps) == steps ? 1 : ((dec & steps) == steps ? -1 : 0);
            }
            const float m = __reduce_max_sync(0xffffffffu, in ? __float_as_uint(ssl[l].sig2) : 0u);
            if (l == 0) sig2max = __uint_as_float(m);  // variances are >= 0: their bits order as they do
        }
        __syncthreads();
        // cheap screen for slices tested one by one: |e_n . mu - e_n . t| beyond
        // K sqrt(s_max^2 + sig2max), grown by 2^-8 of it plus 2^-18 |mu|_1 (far more
        // than the FP32 rounding of the exact test and of this bound), fails the
        // exact test, since e_n . Sigma e_n <= s_max^2
        float bnd = 0.f;
        if (valid) {
            const float sm = fmaxf(fmaxf(scale[3 * g], scale[3 * g + 1]), scale[3 * g + 2]);
            bnd = sqrtf(K2 * (sm * sm + sig2max)) * 1.00390625f +
                  (fabsf(G.mu[0]) + fabsf(G.mu[1]) + fabsf(G.mu[2])) * 3.814697265625e-6f;
        }
        unsigned word = 0, myc = 0;  // myc: the warp's count at slice k0 + lane
        for (int a = 0; a < nk;) {
            const int e = run_end[a], dir = run_dir[a];
            if (!(dir != 0 && e - a >= 7)) {
                // short runs (moving slices): the screen, then the exact test slice by slice
                bool cand = false;
                if (valid) {
                    const float *Q = ssl[a].Q;
                    const float wm = fmaf(Q[2], G.mu[0], fmaf(Q[5], G.mu[1], Q[8] * G.mu[2]));
                    for (int kk = a; kk <= e; ++kk) cand |= fabsf(wm - sent[kk]) <= bnd;
                    if (cand) {
                        frame_slab(G, Q, f);
                        f.k2sww = __fmul_rn(K2, __fadd_rn(f.Lww, ssl[a].sig2));
                    }
                }
                if (__any_sync(0xffffffffu, cand)) {  // else every lane fails every slice of the run
                    for (int kk = a; kk <= e; ++kk) {
                        const bool ex = cand && slab_test(f, ssl[kk]);  // off the screen: fails the test
                        const unsigned c = __popc(__ballot_sync(0xffffffffu, ex));
                        if (lane == kk) myc = c;
                        word |= (unsigned)ex << kk;
                    }
                }
                a = e + 1;
                continue;
            }
            int lo = e + 1, hi = a - 1;  // this lane's candidate slices in the run (none)
            if (valid) {
                frame_slab(G, ssl[a].Q, f);
                f.k2sww = __fmul_rn(K2, __fadd_rn(f.Lww, ssl[a].sig2));
                // offsets within R of e_n . mu: R exceeds the test's sqrt(K2 Sww) by 2^-9
                // of it plus 2^-20 |e_n . mu|, more than the FP32 rounding of the test
                // and of the bounds below
                const float R = sqrtf(f.k2sww) * 1.001953125f + fabsf(f.wmu) * 9.5367431640625e-7f;
                const float olo = f.wmu - R, ohi = f.wmu + R;
                int b0 = a, b1 = e + 1;
                if (dir > 0) {
                    while (b0 < b1) {  // first offset >= olo
                        const int m = (b0 + b1) >> 1;
                        if (sent[m] < olo) b0 = m + 1; else b1 = m;
                    }
                    lo = b0;
                    b1 = e + 1;
                    while (b0 < b1) {  // first offset > ohi
                        const int m = (b0 + b1) >> 1;
                        if (sent[m] <= ohi) b0 = m + 1; else b1 = m;
                    }
                    hi = b0 - 1;
                } else {
                    while (b0 < b1) {  // first offset <= ohi
                        const int m = (b0 + b1) >> 1;
                        if (sent[m] > ohi) b0 = m + 1; else b1 = m;
                    }
                    lo = b0;
                    b1 = e + 1;
                    while (b0 < b1) {  // first offset < olo
                        const int m = (b0 + b1) >> 1;
                        if (sent[m] >= olo) b0 = m + 1; else b1 = m;
                    }
                    hi = b0 - 1;
                }
                if (lo > hi) {  // nothing to test: neutral in the warp's union
                    lo = e + 1;
                    hi = a - 1;
                }
            }
            const int ulo = __reduce_min_sync(0xffffffffu, lo), uhi = __reduce_max_sync(0xffffffffu, hi);
            for (int kk = ulo; kk <= uhi; ++kk) {
                const bool ex = valid && slab_test(f, ssl[kk]);
                const unsigned c = __popc(__ballot_sync(0xffffffffu, ex));
                if (lane == kk) myc = c;
                word |= (unsigned)ex << kk;
            }
            a = e + 1;
        }
        if (wg < NW && lane < nk) cnt[(long long)(k0 + lane) * NW + wg] = myc;
        if (g < n) {
            bits[(long long)wd * n + g] = word;
            if (word) atomicAdd(&gcnt[g], (unsigned)__popc(word));
        }
    }
}

// ---------------------------------------------------------------------------
// MG_LOCAL_CELLS (Eqs. E4-E6): a Gaussian's cell and the centre of its member
// box; the record test is the slice plane passing within the margin of the box
__device__ __forceinline__ void gauss_cell(const float *mu, const CellGrid &cg, int c[3], float b[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        c[a] = cell_coord(mu[a], cg.C[a], cg.h, cg.hres);
        b[a] = __fadd_rn(cg.C[a], __fmul_rn(cg.h, __fsub_rn(__fdiv_rn(__fadd_rn((float)c[a], 0.5f), cg.hres), 1.0f)));
    }
}

__device__ __forceinline__ float abs_sum3(float a, float b, float c)
{
    return __fadd_rn(__fadd_rn(fabsf(a), fabsf(b)), fabsf(c));
}

__device__ __forceinline__ bool cell_slab(const float b[3], const SliceDev &S, const CellGrid &cg)
{
    const float *Q = S.Q;
    float p0 = __fsub_rn(b[0], S.t[0]), p1 = __fsub_rn(b[1], S.t[1]), p2 = __fsub_rn(b[2], S.t[2]);
    float w = dot3_rn(Q[2], Q[5], Q[8], p0, p1, p2);
    return fabsf(w) <= __fadd_rn(__fmul_rn(cg.e, abs_sum3(Q[2], Q[5], Q[8])), cg.m);
}

__global__ void __launch_bounds__(K1_NT) k1_count_cells(const SliceDev *__restrict__ slices, int S, const float *mean,
                                                        const float *quat, const float *scale, const float *alpha,
                                                        long long n, float f64_ratio, CellGrid cg, unsigned *cnt,
                                                        long long NW, unsigned *gcnt, unsigned *bits, WsHeader *hdr)
{
    pdl_entry();
    __shared__ SliceDev ssl[K1_SMEM_SLICES];
    const long long g = (long long)blockIdx.x * K1_NT + threadIdx.x;
    const long long wg = g >> 5;
    const int lane = threadIdx.x & 31;
    GaussPred G;
    bool valid = false;
    int c[3];
    float b[3];
    if (g < n) {
        valid = load_gauss_pred(mean, quat, scale, alpha, g, G);
        if (!valid) atomicOr(&hdr->flags, MG_FLAG_NOT_FINITE);
        float sc[3] = {scale[3 * g], scale[3 * g + 1], scale[3 * g + 2]};
        if (valid && is_degenerate(sc, f64_ratio)) atomicOr(&hdr->flags, MG_FLAG_DEGENERATE);
        gauss_cell(G.mu, cg, c, b);
    }
    unsigned word = 0, mine = 0;
    for (int k0 = 0; k0 < S; k0 += K1_SMEM_SLICES) {
        const int nk = min(K1_SMEM_SLICES, S - k0);
        __syncthreads();
        for (int i = threadIdx.x; i < nk; i += K1_NT) ssl[i] = slices[k0 + i];
        __syncthreads();
        for (int kk = 0; kk < nk; ++kk) {
            const int k = k0 + kk;
            const bool ex = valid && cell_slab(b, ssl[kk], cg);
            unsigned bal = __ballot_sync(0xffffffffu, ex);
            if (lane == 0 && wg < NW) cnt[(long long)k * NW + wg] = __popc(bal);
            word |= (unsigned)ex << (k & 31);
            mine += ex;
            if ((k & 31) == 31 || k == S - 1) {
                if (g < n) bits[(long long)(k >> 5) * n + g] = word;
                word = 0;
            }
        }
    }
    if (g < n) gcnt[g] = mine;
}

__global__ void __launch_bounds__(K1_NT) k1_emit(int S, long long n, const unsigned *__restrict__ bits,
                                                 const unsigned *__restrict__ off, long long NW,
                                                 const unsigned *__restrict__ goff, Records rec, unsigned *gmap,
                                                 const SliceDev *__restrict__ slices, WsHeader *hdr)
{
    pdl_entry();
    // block 0 also marks the stacks whose slices do not all share one rotation
    if (blockIdx.x == 0)
        for (int k = 1 + threadIdx.x; k < S; k += K1_NT)
            if (slices[k].stack == slices[k - 1].stack && !slices[k].same_frame)
                atomicOr(&hdr->moving, 1u << slices[k].stack);
    const long long g = (long long)blockIdx.x * K1_NT + threadIdx.x;
    const long long wg = g >> 5;
    const bool valid = g < n;
    const unsigned lt = lanemask_lt();
    unsigned long long gpos = valid ? goff[g] : 0;
    const int SW = (S + 31) >> 5;
    for (int wd = 0; wd < SW; ++wd) {
        unsigned word = valid ? bits[(long long)wd * n + g] : 0u;
        unsigned uni = __reduce_or_sync(0xffffffffu, word);
        // lane j loads the warp's output offset for slice 32 wd + j when some
        // lane has a record there (all of the word's loads in flight at once)
        const unsigned offl = (uni >> (threadIdx.x & 31)) & 1u ? off[(long long)(wd * 32 + (threadIdx.x & 31)) * NW + wg] : 0u;
        while (uni) {
            const int b = __ffs(uni) - 1;
            uni &= uni - 1;
            const int k = wd * 32 + b;
            const bool f = (word >> b) & 1u;
            const unsigned bal = __ballot_sync(0xffffffffu, f);
            const unsigned ob = __shfl_sync(0xffffffffu, offl, b);
            if (f) {
                const unsigned long long pos = (unsigned long long)ob + __popc(bal & lt);
                if ((long long)pos < rec.cap) {
                    rec.gid[pos] = (int)g;
                    rec.slice[pos] = k;
                }
                if ((long long)gpos < rec.cap) gmap[gpos] = (unsigned)pos;
                ++gpos;
            }
        }
    }
}

// one thread per record: the tile rectangle (rest of the FP32 predicate; the
// slab test passed in k1_count) and the FP32 evaluation geometry (FP64 for
// near-degenerate Gaussians in k_rec_geom_f64)
template <bool CELLS>
__global__ void __launch_bounds__(256, 4)
    k_rec_fill(const WsHeader *hdr, const SliceDev *__restrict__ slices, const float *mean, const float *quat,
               const float *scale, const float *alpha, float K2, float f64_ratio, CellGrid cg, Records rec)
{
    pdl_entry();
    long long nr = (long long)hdr->n_records;
    if (nr > rec.cap) nr = rec.cap;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += (long long)gridDim.x * blockDim.x) {
        const long long g = rec.gid[r];
        const SliceDev &Sd = slices[rec.slice[r]];
        GaussPred G;
        load_gauss_pred(mean, quat, scale, alpha, g, G);
        PredOut po;
        if (CELLS) {
            // pixel box of the member box's extent along e_u, e_v
            int c[3];
            float b[3];
            gauss_cell(G.mu, cg, c, b);
            const float *Q = Sd.Q;
            float p0 = __fsub_rn(b[0], Sd.t[0]), p1 = __fsub_rn(b[1], Sd.t[1]), p2 = __fsub_rn(b[2], Sd.t[2]);
            float uc = dot3_rn(Q[0], Q[3], Q[6], p0, p1, p2);
            float vc = dot3_rn(Q[1], Q[4], Q[7], p0, p1, p2);
            float ru = __fadd_rn(__fmul_rn(cg.e, abs_sum3(Q[0], Q[3], Q[6])), cg.m);
            float rv = __fadd_rn(__fmul_rn(cg.e, abs_sum3(Q[1], Q[4], Q[7])), cg.m);
            pixel_box(Sd, uc, vc, ru, rv, po);
            rec.cell[r] = make_int4(c[0], c[1], c[2], 0);
        } else {
            FrameTerms ft;
            frame_slab(G, Sd.Q, ft);
            record_predicate(G, Sd, K2, ft, po);  // true: the slab test of k1_count
        }
        RecTiles rt;
        rt.rect = make_ushort4((unsigned short)(po.il / MG_TILE), (unsigned short)(po.jl / MG_TILE),
                               (unsigned short)(po.ih / MG_TILE), (unsigned short)(po.jh / MG_TILE));
        float sc[3] = {scale[3 * g], scale[3 * g + 1], scale[3 * g + 2]};
        // rows are culled for max scale <= 64 min scale only (beyond, FP32
        // cancellation in the conditional covariance can exceed the margin)
        unsigned long long ins = 0ull;
        if (!CELLS && fmaxf(fmaxf(sc[0], sc[1]), sc[2]) <= 64.0f * fminf(fminf(sc[0], sc[1]), sc[2]))
            ins = row_insets(Sd, po);
        rt.inset = ins;
        rec.tiles[r] = rt;
        // the backward's moment slots start at zero (it accumulates into them);
        // near-degenerate Gaussians accumulate in FP64
        ((float4 *)rec.mom)[2 * r] = make_float4(0.f, 0.f, 0.f, 0.f);
        ((float4 *)rec.mom)[2 * r + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        const bool dg = is_degenerate(sc, f64_ratio);
        // bit 0: FP64 geometry; bit 1: elongated (the backward's centre-out moment sums)
        rec.f64[r] = (dg ? 1 : 0) | (dg || is_degenerate(sc, ELONG_RATIO) ? 2 : 0);
        if (dg) {
            double2 *m2 = (double2 *)(rec.mom64 + MOM64_STRIDE * r);
            m2[0] = m2[1] = m2[2] = make_double2(0.0, 0.0);
            continue;
        }
        float qv[4] = {quat[4 * g], quat[4 * g + 1], quat[4 * g + 2], quat[4 * g + 3]};
        RecGeomT<float> o;
        record_geometry<float>(G.mu, qv, sc, alpha[g], Sd, K2, o);
        rec.geo[r] = make_float4(o.pcx, o.pcy, o.A, o.B2);
        rec.geo2[r] = make_float2(o.C, o.amp);
        rec.thr[r] = o.thr;
    }
}

// FP64 record geometry for near-degenerate Gaussians (scale ratio above
// f64_ratio), one thread per Gaussian over its records
__global__ void k_rec_geom_f64(const WsHeader *hdr, long long n, const SliceDev *__restrict__ slices,
                               const float *mean, const float *quat, const float *scale, const float *alpha, float K2,
                               float f64_ratio, const unsigned *__restrict__ goff, const unsigned *__restrict__ gmap,
                               Records rec)
{
    pdl_entry();
    if (!(hdr->flags & MG_FLAG_DEGENERATE)) return;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x) {
        float sc[3] = {scale[3 * g], scale[3 * g + 1], scale[3 * g + 2]};
        if (!is_degenerate(sc, f64_ratio)) continue;
        float mu[3] = {mean[3 * g], mean[3 * g + 1], mean[3 * g + 2]};
        float qv[4] = {quat[4 * g], quat[4 * g + 1], quat[4 * g + 2], quat[4 * g + 3]};
        float av = alpha[g];
        unsigned long long j1 = goff[g + 1];
        if ((long long)j1 > rec.cap) j1 = rec.cap;
        for (unsigned long long j = goff[g]; j < j1; ++j) {
            const unsigned r = gmap[j];
            if ((long long)r >= rec.cap) continue;
            RecGeomT<double> o;
            record_geometry<double>(mu, qv, sc, av, slices[rec.slice[r]], K2, o);
            rec.geo[r] = make_float4((float)o.pcx, (float)o.pcy, (float)o.A, (float)o.B2);
            rec.geo2[r] = make_float2((float)o.C, (float)o.amp);
            rec.thr[r] = (float)o.thr;
            // the FP64 centre and conic: rounded to FP32, the conic of a needle
            // far along its axis moves the exponent by ~ 2^-24 (max/min scale)^2
            double *g64 = rec.mom64 + MOM64_STRIDE * r + MOM64_GEO;
            g64[0] = o.pcx;
            g64[1] = o.pcy;
            g64[2] = o.A;
            g64[3] = o.B2;
            g64[4] = o.C;
        }
    }
}

// ---------------------------------------------------------------------------
// K3: per-slice chunks of records, chunk histograms, column scan, scatter
// ---------------------------------------------------------------------------
// one block: slice record ranges (clamped to capacity) and chunk offsets
__global__ void __launch_bounds__(1024) k_chunk_setup(const unsigned *rec_off, int S, int NB,
                                                      unsigned *slice_rs, unsigned *chunk_base, long long cap_rec,
                                                      long long cap_chunks, WsHeader *hdr)
{
    pdl_entry();
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    unsigned long long total = hdr->n_records;
    for (int base = 0; base < S; base += 1024) {
        int k = base + threadIdx.x;
        unsigned long long nch = 0;
        if (k < S) {
            unsigned long long rs = rec_off[(long long)k * NB];
            unsigned long long re = (k + 1 < S) ? rec_off[(long long)(k + 1) * NB] : total;
            if (rs > (unsigned long long)cap_rec) rs = cap_rec;
            if (re > (unsigned long long)cap_rec) re = cap_rec;
            slice_rs[k] = (unsigned)rs;
            if (k == S - 1) slice_rs[S] = (unsigned)re;
            nch = (re > rs) ? (re - rs + MG_CHUNK - 1) / MG_CHUNK : 0;
        }
        // block scan with 1024 threads
        __shared__ unsigned long long ws[32];
        unsigned long long x = nch;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[w] = x;
        __syncthreads();
        if (w == 0) {
            unsigned long long s = ws[lane];
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            ws[lane] = s;
        }
        __syncthreads();
        unsigned long long pre = carry + (w > 0 ? ws[w - 1] : 0ull) + x - nch;
        if (k < S) chunk_base[k] = (unsigned)pre;
        __syncthreads();
        if (threadIdx.x == 0) carry += ws[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        chunk_base[S] = (unsigned)carry;
        hdr->n_chunks = carry;
        if (carry > (unsigned long long)cap_chunks) atomicOr(&hdr->flags, MG_FLAG_CAP_CHUNKS);
        if (total > (unsigned long long)cap_rec) atomicOr(&hdr->flags, MG_FLAG_CAP_RECORDS);
    }
}

__device__ __forceinline__ int find_slice(const unsigned *chunk_base, int S, unsigned c)
{
    // largest k with chunk_base[k] <= c (chunk_base is non-decreasing, chunk_base[S] = total)
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (chunk_base[mid] <= c)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// warps (chunks) per block of the histogram and scatter passes: each warp
// holds a counter per tile of a slice in shared memory, so large slices get
// fewer warps per block
constexpr int BIN_WARPS = 4;
constexpr size_t BIN_SMEM_MAX = 200 * 1024;

__global__ void __launch_bounds__(32 * BIN_WARPS) k_bin_hist(const SliceDev *slices, int S, const unsigned *slice_rs,
                                                             const unsigned *chunk_base, const RecTiles *tiles,
                                                             unsigned *hist, int Tmax, long long cap_chunks,
                                                             unsigned *big_n, unsigned *big_list, WsHeader *hdr)
{
    pdl_entry();
    extern __shared__ unsigned smem_u[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    unsigned *hs = smem_u + w * Tmax;
    unsigned n_chunks = chunk_base[S];
    if ((long long)n_chunks > cap_chunks) n_chunks = (unsigned)cap_chunks;
    const unsigned nw = blockDim.x >> 5;
    for (unsigned c = blockIdx.x * nw + w; c < n_chunks; c += gridDim.x * nw) {
        int k = find_slice(chunk_base, S, c);
        const int TX = slices[k].TX, Tk = TX * slices[k].TY;
        unsigned r0 = slice_rs[k] + (c - chunk_base[k]) * MG_CHUNK;
        unsigned r1 = min(r0 + MG_CHUNK, slice_rs[k + 1]);
        for (int t = lane; t < Tk; t += 32) hs[t] = 0;
        __syncwarp();
        unsigned nbig = 0;
        for (unsigned base = r0; base < r1; base += 32) {
            const unsigned r = base + lane;
            RecTiles rt;
            rt.rect = make_ushort4(1, 1, 0, 0);
            rt.inset = 0ull;
            if (r < r1) rt = load_tiles(tiles + r);
            const ushort4 rc = rt.rect;
            const unsigned long long ins = rt.inset;
            // a rectangle of at most BIG_AREA tiles lists at most that many
            const bool wide = rc.x <= rc.z && rc.y <= rc.w && ((int)rc.z - rc.x + 1) * ((int)rc.w - rc.y + 1) > BIG_AREA;
            const int area = wide ? listed_count(rc, ins) : 0;
            const int slot = big_slot(area, nbig, lt);
            if (slot >= 0) {
                big_list[(size_t)c * BIG_MAX + slot] = r;  // counted and placed by k_bin_big
                continue;
            }
            for (int ty = rc.y; ty <= rc.w; ++ty) {
                const int2 sp = row_span(rc, ins, ty - rc.y);
                for (int tx = sp.x; tx <= sp.y; ++tx) atomicAdd(&hs[ty * TX + tx], 1u);
            }
        }
        __syncwarp();
        unsigned *hout = hist + (size_t)c * Tmax;
        for (int t = lane; t < Tk; t += 32) hout[t] = hs[t];
        if (lane == 0) {
            big_n[c] = nbig;
            if (nbig) atomicAdd(&hdr->n_big, (unsigned long long)nbig);
        }
        __syncwarp();
    }
}

// per (slice, tile): exclusive prefix over the slice's chunks; tile totals;
// and the tile lists of the render kernels: tiles without records at the back
// of the tile list, tiles with records on the dense (more than SPARSE_MAX
// records) or the sparse list (counts aggregated per block, one atomic per
// block and list; the order within each list is arbitrary and does not change
// any result)
constexpr int COLSCAN_NT = 256;
__global__ void __launch_bounds__(COLSCAN_NT) k_bin_colscan(const SliceDev *slices, int S, const unsigned *chunk_base,
                                                            unsigned *hist, int Tmax, long long cap_chunks,
                                                            unsigned *tile_cnt, unsigned *tile_list,
                                                            long long n_tiles, WsHeader *hdr,
                                                            const unsigned *tile_big, unsigned *tile_small,
                                                            unsigned *dense_list, unsigned *sparse_list)
{
    pdl_entry();
    const bool any_big = hdr->n_big > 0;  // tile_big is written only then
    __shared__ unsigned wi[COLSCAN_NT / 32], wd[COLSCAN_NT / 32], ws_[COLSCAN_NT / 32];
    __shared__ unsigned base_i, base_d, base_s;
    const long long total = (long long)S * Tmax;
    const unsigned lt = lanemask_lt();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (long long blk = (long long)blockIdx.x * COLSCAN_NT; blk < total; blk += (long long)gridDim.x * COLSCAN_NT) {
        const long long idx = blk + threadIdx.x;
        int k = 0, t = 0;
        bool real = false;
        unsigned run = 0;
        if (idx < total) {
            k = (int)(idx / Tmax);
            t = (int)(idx % Tmax);
            real = t < slices[k].TX * slices[k].TY;
        }
        if (real) {
            unsigned c0 = chunk_base[k], c1 = chunk_base[k + 1];
            if ((long long)c1 > cap_chunks) c1 = (unsigned)cap_chunks;
            // sixteen independent (guarded) loads in flight per thread before the
            // dependent stores: a slice's column of chunk counts in one or two rounds
            for (unsigned c = c0; c < c1; c += 16) {
                unsigned v[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) v[u] = (c + u < c1) ? __ldcg(&hist[(size_t)(c + u) * Tmax + t]) : 0u;
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    if (c + u < c1) hist[(size_t)(c + u) * Tmax + t] = run;
                    run += v[u];
                }
            }
            // the large records listed apart follow the tile's other entries
            const int tile = slices[k].tile_base + t;
            tile_small[tile] = run;
            if (any_big) run += tile_big[tile];
            tile_cnt[tile] = run;
        }
        const bool busy = real && run > 0, idle = real && run == 0;
        const bool dense = busy && run > SPARSE_MAX, sparse = busy && run <= SPARSE_MAX;
        const unsigned ib = __ballot_sync(0xffffffffu, idle);
        const unsigned db = __ballot_sync(0xffffffffu, dense), sbm = __ballot_sync(0xffffffffu, sparse);
        if (lane == 0) {
            wi[w] = __popc(ib);
            wd[w] = __popc(db);
            ws_[w] = __popc(sbm);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned si = 0, sd = 0, ss = 0;
            for (int i = 0; i < COLSCAN_NT / 32; ++i) {
                const unsigned b = wi[i], c = wd[i], e = ws_[i];
                wi[i] = si;
                wd[i] = sd;
                ws_[i] = ss;
                si += b;
                sd += c;
                ss += e;
            }
            base_i = si ? atomicAdd(&hdr->n_idle, si) : 0u;
            base_d = sd ? atomicAdd(&hdr->n_dense, sd) : 0u;
            base_s = ss ? atomicAdd(&hdr->n_sparse, ss) : 0u;
        }
        __syncthreads();
        const unsigned tid = (unsigned)(slices[k].tile_base + t);
        if (idle) tile_list[n_tiles - 1 - (long long)(base_i + wi[w] + __popc(ib & lt))] = tid;
        if (dense) dense_list[base_d + wd[w] + __popc(db & lt)] = tid;
        if (sparse) sparse_list[base_s + ws_[w] + __popc(sbm & lt)] = tid;
        __syncthreads();  // the per-warp counts and the bases are rewritten by the next round
    }
}

__global__ void __launch_bounds__(32 * BIN_WARPS, 12) k_bin_scatter(const SliceDev *slices, int S,
                                                                const unsigned *slice_rs, const unsigned *chunk_base,
                                                                const RecTiles *tiles, const unsigned *hist,
                                                                int Tmax,
                                                                long long cap_chunks, const unsigned *tile_off,
                                                                unsigned *entries, long long cap_entries,
                                                                WsHeader *hdr)
{
    pdl_entry();
    extern __shared__ unsigned smem_u[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0 && hdr->n_entries > (unsigned long long)cap_entries)
        atomicOr(&hdr->flags, MG_FLAG_CAP_ENTRIES);
    unsigned *cur = smem_u + w * Tmax;
    unsigned n_chunks = chunk_base[S];
    if ((long long)n_chunks > cap_chunks) n_chunks = (unsigned)cap_chunks;
    const unsigned lt = lanemask_lt();
    const unsigned nw = blockDim.x >> 5;
    for (unsigned c = blockIdx.x * nw + w; c < n_chunks; c += gridDim.x * nw) {
        int k = find_slice(chunk_base, S, c);
        const int TX = slices[k].TX, Tk = TX * slices[k].TY, tb = slices[k].tile_base;
        unsigned r0 = slice_rs[k] + (c - chunk_base[k]) * MG_CHUNK;
        unsigned r1 = min(r0 + MG_CHUNK, slice_rs[k + 1]);
        const unsigned *hin = hist + (size_t)c * Tmax;
        {
            // eight independent load pairs in flight per lane
            int t = lane;
            for (; t + 7 * 32 < Tk; t += 8 * 32) {
                unsigned o[8], h[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) o[u] = tile_off[tb + t + 32 * u], h[u] = hin[t + 32 * u];
#pragma unroll
                for (int u = 0; u < 8; ++u) cur[t + 32 * u] = o[u] + h[u];
            }
            for (; t < Tk; t += 32) cur[t] = tile_off[tb + t] + hin[t];
        }
        __syncwarp();
        unsigned nbig = 0;
        for (unsigned base = r0; base < r1; base += 32) {
            unsigned r = base + lane;
            bool have = r < r1;
            RecTiles rt;
            rt.rect = make_ushort4(1, 1, 0, 0);
            rt.inset = 0ull;
            if (have) rt = load_tiles(tiles + r);
            const ushort4 rc = rt.rect;
            const unsigned long long ins = rt.inset;
            int area = listed_count(rc, ins);
            if (big_slot(area, nbig, lt) >= 0) area = 0;  // listed apart: placed by k_bin_big_place
            int maxa = __reduce_max_sync(0xffffffffu, area);
            unsigned incl = (unsigned)area;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
            if (flatten_batch(maxa, total)) {
                // one entry per lane per round, record-major: the ranks within a tile
                // follow record order. The per-lane loop below orders a tile's entries
                // by (round, lane) instead; both orders are deterministic, but they
                // differ, so a tile's summation order depends on which path its batch took
                for (unsigned eb = 0; eb < total; eb += 32) {
                    const unsigned e = eb + lane;
                    const bool act = e < total;
                    const int j = entry_owner(incl, act ? e : total - 1);
                    ushort4 rj;
                    unsigned long long ij;
                    shfl_tiles(rc, ins, j, rj, ij);
                    const unsigned excl = __shfl_sync(0xffffffffu, incl, j) - __shfl_sync(0xffffffffu, (unsigned)area, j);
                    const unsigned t = act ? (unsigned)nth_listed_tile(rj, ij, e - excl, TX) : 0xffffffffu;
                    const unsigned peers = __match_any_sync(0xffffffffu, t);
                    const unsigned before = peers & lt;
                    unsigned pos = 0;
                    if (act) pos = cur[t] + __popc(before);
                    __syncwarp();
                    if (act) {
                        if ((long long)pos < cap_entries) entries[pos] = base + (unsigned)j;
                        if (before == 0) cur[t] += __popc(peers);
                    }
                    __syncwarp();
                }
                continue;
            }
            // the listed tiles in row-major order: (jx, jy) with the row's last column xe
            int jy = rc.y;
            int2 sp = row_span(rc, ins, 0);
            while (sp.x > sp.y && jy < (int)rc.w) sp = row_span(rc, ins, ++jy - rc.y);
            int jx = sp.x, xe = sp.y;
            for (int j = 0; j < maxa; ++j) {
                bool act = j < area;
                unsigned t = 0xffffffffu;
                if (act) t = (unsigned)(jy * TX + jx);
                if (act && ++jx > xe) {
                    do {
                        if (++jy > (int)rc.w) break;
                        sp = row_span(rc, ins, jy - rc.y);
                    } while (sp.x > sp.y);
                    jx = sp.x;
                    xe = sp.y;
                }
                unsigned peers = __match_any_sync(0xffffffffu, t);
                unsigned before = peers & lt;
                unsigned pos = 0;
                if (act) pos = cur[t] + __popc(before);
                __syncwarp();
                if (act) {
                    if ((long long)pos < cap_entries) entries[pos] = r;
                    if (before == 0) cur[t] += __popc(peers);
                }
                __syncwarp();
            }
        }
        __syncwarp();
    }
}

// The records listed apart (large records), one thread per tile of a slice:
// COUNT writes how many list the tile (tile_big); PLACE writes them after the
// tile's other entries, in chunk order and each chunk's list order. The
// slice's listed records are staged in shared memory (their chunks' list
// lengths scanned, then the records loaded in parallel) and every tile thread
// tests them in order.
constexpr int BIG_NT = 1024;  // a slice's tiles per job (all of a 256x256 slice's)
constexpr int BIG_STAGE = 1024;
template <bool PLACE>
__global__ void __launch_bounds__(BIG_NT) k_bin_big(const SliceDev *__restrict__ slices, int S, int Tmax,
                                                    const unsigned *__restrict__ chunk_base, long long cap_chunks,
                                                    const unsigned *__restrict__ big_n,
                                                    const unsigned *__restrict__ big_list,
                                                    const RecTiles *__restrict__ tiles, unsigned *tile_big,
                                                    const unsigned *__restrict__ tile_off,
                                                    const unsigned *__restrict__ tile_small, unsigned *entries,
                                                    long long cap_entries, const WsHeader *hdr)
{
    pdl_entry();
    __shared__ unsigned offs[BIG_NT + 1];
    __shared__ unsigned wsum[BIG_NT / 32];
    __shared__ uint4 srt[BIG_STAGE];
    __shared__ unsigned srid[BIG_STAGE];
    if (hdr->n_big == 0) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int per = (Tmax + BIG_NT - 1) / BIG_NT;  // blocks of tiles per slice
    for (long long job = blockIdx.x; job < (long long)S * per; job += gridDim.x) {
        const int k = (int)(job / per), t = (int)(job % per) * BIG_NT + threadIdx.x;
        const int TX = slices[k].TX;
        const bool act = t < TX * slices[k].TY;
        const int tile = slices[k].tile_base + (act ? t : 0), tx = t % TX, ty = t / TX;
        unsigned long long pos = PLACE && act ? (unsigned long long)tile_off[tile] + tile_small[tile] : 0ull;
        const unsigned c0 = chunk_base[k];
        unsigned c1 = chunk_base[k + 1];
        if ((long long)c1 > cap_chunks) c1 = (unsigned)cap_chunks;
        for (unsigned cg = c0; cg < c1; cg += BIG_NT) {
            const unsigned nch = min((unsigned)BIG_NT, c1 - cg);
            // exclusive offsets of the group's list lengths
            const unsigned m = threadIdx.x < nch ? big_n[cg + threadIdx.x] : 0u;
            unsigned x = m;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned v = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += v;
            }
            if (lane == 31) wsum[w] = x;
            __syncthreads();
            unsigned before = 0, total = 0;
            for (int i = 0; i < BIG_NT / 32; ++i) {
                before += i < w ? wsum[i] : 0u;
                total += wsum[i];
            }
            offs[threadIdx.x] = before + x - m;
            if (threadIdx.x == 0) offs[BIG_NT] = total;
            __syncthreads();
            for (unsigned s0 = 0; s0 < total; s0 += BIG_STAGE) {
                const unsigned ns = min((unsigned)BIG_STAGE, total - s0);
                for (unsigned i = threadIdx.x; i < ns; i += BIG_NT) {
                    // the chunk of element s0 + i: the last q with offs[q] <= s0 + i
                    const unsigned e = s0 + i;
                    int lo = 0, hi = (int)nch - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (offs[mid] <= e)
                            lo = mid;
                        else
                            hi = mid - 1;
                    }
                    const unsigned r = big_list[(size_t)(cg + lo) * BIG_MAX + (e - offs[lo])];
                    srid[i] = r;
                    srt[i] = __ldg((const uint4 *)(tiles + r));
                }
                __syncthreads();
                if (act) {
                    for (unsigned i = 0; i < ns; ++i) {
                        const uint4 u = srt[i];
                        const ushort4 rc = make_ushort4((unsigned short)(u.x & 0xFFFFu), (unsigned short)(u.x >> 16),
                                                        (unsigned short)(u.y & 0xFFFFu), (unsigned short)(u.y >> 16));
                        if (lists_tile(rc, (unsigned long long)u.z | ((unsigned long long)u.w << 32), tx, ty)) {
                            if (PLACE && (long long)pos < cap_entries) entries[pos] = srid[i];
                            ++pos;
                        }
                    }
                }
                __syncthreads();
            }
        }
        if (!PLACE && act) tile_big[tile] = (unsigned)pos;
    }
}

// ---------------------------------------------------------------------------
// the whole record + binning pass
// ---------------------------------------------------------------------------
void mg_launch_bin(const WsLayout &L, char *ws, const SliceDev *slices, const StackTable &tab, const float *mean,
                   const float *quat, const float *scale, const float *alpha, long long n, float K, float f64_ratio,
                   const CellGrid &cg, cudaStream_t st)
{
    WsHeader *hdr = (WsHeader *)(ws + L.hdr);
    unsigned *cnt = (unsigned *)(ws + L.cnt);
    unsigned long long *part = (unsigned long long *)(ws + L.scan_part);
    Records rec;
    rec.geo = (float4 *)(ws + L.rec_geo);
    rec.geo2 = (float2 *)(ws + L.rec_geo2);
    rec.gid = (int *)(ws + L.rec_gid);
    rec.slice = (int *)(ws + L.rec_slice);
    rec.tiles = (RecTiles *)(ws + L.rec_rect);
    rec.mom = (float *)(ws + L.rec_mom);
    rec.f64 = (unsigned char *)(ws + L.rec_f64);
    rec.mom64 = (double *)(ws + L.rec_mom64);
    rec.thr = (float *)(ws + L.rec_thr);
    rec.cell = cg.on ? (int4 *)(ws + L.rec_cell) : nullptr;
    rec.cap = L.cap_records;
    unsigned *chunk_base = (unsigned *)(ws + L.chunk_base);
    unsigned *slice_rs = chunk_base + (L.S + 1);
    unsigned *hist = (unsigned *)(ws + L.hist);
    unsigned *tile_cnt = (unsigned *)(ws + L.tile_cnt);
    unsigned *tile_off = (unsigned *)(ws + L.tile_off);
    unsigned *entries = (unsigned *)(ws + L.entries);
    unsigned *big_n = (unsigned *)(ws + L.big_n);
    unsigned *big_list = (unsigned *)(ws + L.big_list);
    unsigned *tile_small = (unsigned *)(ws + L.tile_small);
    unsigned *tile_big = (unsigned *)(ws + L.tile_big);
    const int S = (int)L.S;
    const float K2 = K * K;  // one FP32 multiply, rounded once (as in the predicate)

    cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st);
    unsigned *gcnt = (unsigned *)(ws + L.gcnt);
    unsigned *bits = (unsigned *)(ws + L.bits);
    unsigned *gmap = (unsigned *)(ws + L.gmap);
    const long long NW = L.NW;
    const unsigned g1 = (unsigned)L.NB;
    {
        MG_PROF(MG_ST_K1_COUNT, st);
        if (cg.on) {
            launch_pdl(k1_count_cells, dim3(g1), dim3(K1_NT), 0, st,
                slices, S, mean, quat, scale, alpha, n, f64_ratio, cg, cnt, NW, gcnt,
                                                 bits, hdr);
        } else {
            cudaMemsetAsync(gcnt, 0, sizeof(unsigned) * (size_t)n, st);
            launch_pdl(k1_count, dim3(g1, (unsigned)L.SW), dim3(K1_NT), 0, st,
                slices, S, mean, quat, scale, alpha, n, K2, f64_ratio,
                                                                 cnt, NW, gcnt, bits, hdr);
        }
    }
    {
        MG_PROF(MG_ST_SCAN_REC, st);
        mg_launch_scan2_u32(cnt, cnt, (long long)S * NW, &hdr->n_records, gcnt, gcnt, n, &hdr->scan_total, part, st);
    }
    {
        MG_PROF(MG_ST_K1_EMIT, st);
        launch_pdl(k1_emit, dim3(g1), dim3(K1_NT), 0, st, S, n, bits, cnt, NW, gcnt, rec, gmap, slices, hdr);
    }
    {
        MG_PROF(MG_ST_REC_FILL, st);
        long long want_r = (L.cap_records + 255) / 256;
        int gr = (int)(want_r < 148 * 16 ? (want_r > 0 ? want_r : 1) : 148 * 16);
        if (cg.on)
            launch_pdl(k_rec_fill<true>, dim3(gr), dim3(256), 0, st,
                hdr, slices, mean, quat, scale, alpha, K2, f64_ratio, cg, rec);
        else
            launch_pdl(k_rec_fill<false>, dim3(gr), dim3(256), 0, st,
                hdr, slices, mean, quat, scale, alpha, K2, f64_ratio, cg, rec);
    }
    if (f64_ratio > 0.f) {
        MG_PROF(MG_ST_REC_GEOM, st);
        // grid-strided: two blocks per SM; most steps have no near-degenerate Gaussian and every block returns at once
        int gg = (int)((n + 255) / 256 < 148 * 2 ? (n + 255) / 256 : 148 * 2);
        launch_pdl(k_rec_geom_f64, dim3(gg), dim3(256), 0, st,
            hdr, n, slices, mean, quat, scale, alpha, K2, f64_ratio, gcnt, gmap, rec);
    }
    {
        MG_PROF(MG_ST_CHUNKS, st);
        launch_pdl(k_chunk_setup, dim3(1), dim3(1024), 0, st,
            cnt, S, (int)NW, slice_rs, chunk_base, L.cap_records, L.cap_chunks, hdr);
    }
    const int Tmax = (int)L.max_tiles;
    int bw = BIN_WARPS;
    while (bw > 1 && (size_t)bw * Tmax * sizeof(unsigned) > BIN_SMEM_MAX) --bw;
    size_t smem = (size_t)bw * Tmax * sizeof(unsigned);
    if (smem > 48 * 1024) {
        cudaFuncSetAttribute(k_bin_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_bin_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    long long want = (L.cap_chunks + bw - 1) / bw;
    int gb = (int)(want < 148 * 16 ? (want > 0 ? want : 1) : 148 * 16);
    {
        MG_PROF(MG_ST_BIN_HIST, st);
        launch_pdl(k_bin_hist, dim3(gb), dim3(32 * bw), smem, st,
            slices, S, slice_rs, chunk_base, rec.tiles, hist, Tmax,
                                                     L.cap_chunks, big_n, big_list, hdr);
    }
    // the large records' tile counts: jobs of 1024 tiles of a slice (the
    // slice's listed records staged once per job), at most two blocks per SM
    // (every block returns at once when no record was listed apart)
    const long long big_jobs = (long long)S * ((Tmax + BIG_NT - 1) / BIG_NT);
    const int gbig = (int)(big_jobs < 148 * 2 ? (big_jobs > 0 ? big_jobs : 1) : 148 * 2);
    launch_pdl(k_bin_big<false>, dim3(gbig), dim3(BIG_NT), 0, st,
        slices, S, Tmax, chunk_base, L.cap_chunks, big_n, big_list, rec.tiles,
                                              tile_big, tile_off, tile_small, entries, L.cap_entries, hdr);
    long long tot = (long long)S * Tmax;
    int gc = (int)((tot + 255) / 256 < 148 * 32 ? (tot + 255) / 256 : 148 * 32);
    {
        MG_PROF(MG_ST_BIN_COLSCAN, st);
        launch_pdl(k_bin_colscan, dim3(gc), dim3(COLSCAN_NT), 0, st,
            slices, S, chunk_base, hist, Tmax, L.cap_chunks, tile_cnt,
                                          (unsigned *)(ws + L.tile_list), L.n_tiles, hdr, tile_big, tile_small,
                                          (unsigned *)(ws + L.dense_list), (unsigned *)(ws + L.sparse_list));
    }
    {
        MG_PROF(MG_ST_SCAN_TILES, st);
        mg_launch_scan_u32(tile_cnt, tile_off, L.n_tiles, nullptr, part, &hdr->n_entries, st);
    }
    {
        MG_PROF(MG_ST_BIN_SCATTER, st);
        launch_pdl(k_bin_scatter, dim3(gb), dim3(32 * bw), smem, st,
            slices, S, slice_rs, chunk_base, rec.tiles, hist, Tmax,
                                                        L.cap_chunks, tile_off, entries, L.cap_entries, hdr);
    }
    launch_pdl(k_bin_big<true>, dim3(gbig), dim3(BIG_NT), 0, st,
        slices, S, Tmax, chunk_base, L.cap_chunks, big_n, big_list, rec.tiles,
                                             tile_big, tile_off, tile_small, entries, L.cap_entries, hdr);
}
