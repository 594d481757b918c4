// mg_render.cu -- per-tile evaluation of the additive Gaussian mixture
// (Sec. 3.3.2, Eq. E7 with the slice profile) and its adjoint.
//
// K4 k_render_fwd : one warp per 8x8 tile (persistent warps pull tiles);
//     records staged 32 at a time through shared memory, each already in
//     the tile's frame: q(x, y) = A x^2 + B x y + C y^2 + D x + E y + F with
//     (x, y) the voxel's offset from the tile centre (log2 units), and
//     I += amp * 2^q.
// K5 k_render_bwd : lane = record; each lane sweeps the tile's 64 voxels
//     and forms six moments of w = g 2^q (sum w, w dx, w dy, w dx^2, w dx dy,
//     w dy^2); two vector atomics per (record, tile). A batch of <= 16
//     records shares each record's rows among 2-8 lanes. Nothing per pair is
//     stored.
// K6 k_chain_fused : per Gaussian, its records' moments -> dL/d(centre,
//     conic, amp) -> adjoint of the record geometry -> dL/d(mean, quat,
//     scale, alpha), summed in a fixed order (no atomics).
// k_pose_rec / k_pose_sum : the slice-pose gradient from the same moments.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mg_internal.cuh"

static_assert(MG_TILE == 8, "the evaluation kernels are laid out for 8x8 tiles");

constexpr int RW = 4;                           // warps (tiles) per block
constexpr int NV = MG_TILE * MG_TILE;           // voxels per tile (64)
constexpr int VPT = NV / 32;                    // voxels per lane in the pair count (2)
constexpr float TC = 0.5f * (MG_TILE - 1);      // tile-centre offset of the first row / column (3.5)

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
    L.px = tx * MG_TILE + (lane % MG_TILE);
    L.py0 = ty * MG_TILE + (lane / MG_TILE) * VPT;
    return L;
}

struct TileId {
    int s, kk, tx, ty, W, H;
    long long pixbase;
};

__device__ __forceinline__ TileId tile_id(const StackTable &tab, int t)
{
    TileId d;
    int s = 0;
    while (s + 1 < tab.n_stacks && t >= tab.tile_base[s + 1]) ++s;
    const int TX = tab.TX[s], T = TX * tab.TY[s];
    const int local = t - tab.tile_base[s];
    d.s = s;
    d.kk = local / T;
    const int within = local - d.kk * T;
    d.ty = within / TX;
    d.tx = within - d.ty * TX;
    d.W = tab.W[s];
    d.H = tab.H[s];
    d.pixbase = tab.pix_base[s] + (long long)d.kk * d.H * d.W;
    return d;
}

// The exponent of a record about the centre (x0c, y0c) of a tile: with
// dx0 = x0c - cx, dy0 = y0c - cy (the tile centre's offset from the record
// centre) and (x, y) a voxel's offset from the tile centre,
// A (dx0+x)^2 + B (dx0+x)(dy0+y) + C (dy0+y)^2 = A x^2 + B x y + C y^2 + D x + E y + F.
struct TileQuad {
    float D, E, F;
};
__device__ __forceinline__ TileQuad tile_quad(float A, float B, float C, float dx0, float dy0)
{
    TileQuad t;
    const float Bdy = B * dy0;
    t.D = fmaf(2.f * A, dx0, Bdy);
    t.E = fmaf(B, dx0, 2.f * C * dy0);
    t.F = fmaf(fmaf(A, dx0, Bdy), dx0, (C * dy0) * dy0);
    return t;
}

// The same coefficients D, E, F for a near-degenerate record, from its FP64
// centre and conic (g64 = pcx, pcy, A, B2, C), in FP64: for a needle the
// three terms of F are large and cancel, and its FP32 conic alone is off by
// ~ 2^-24 (max/min scale)^2 in the exponent far along its axis.
// (Out of line: the caller tests a warp-uniform flag first, so the FP64 work
// never runs predicated off for ordinary records.)
__device__ __noinline__ TileQuad tile_quad_f64(const double *__restrict__ g64, float x0c, float y0c)
{
    const double dx0 = (double)x0c - g64[0], dy0 = (double)y0c - g64[1];
    const double A = g64[2], B = g64[3], C = g64[4];
    TileQuad t;
    t.D = (float)fma(2.0 * A, dx0, B * dy0);
    t.E = (float)fma(B, dx0, 2.0 * C * dy0);
    t.F = (float)fma(fma(A, dx0, B * dy0), dx0, C * dy0 * dy0);
    return t;
}

// CELLS: the tile's voxel cells packed relative to its smallest cell (one
// word per voxel, row-major), and that smallest cell
__device__ __forceinline__ void tile_cells(const SliceDev &Sd, const CellGrid &cg, int tx, int ty, int lane,
                                           unsigned *srelw, int &cb0, int &cb1, int &cb2)
{
    int m0 = 0x7fffffff, m1 = 0x7fffffff, m2 = 0x7fffffff;
    for (int i = lane; i < NV; i += 32) {
        int c[3];
        voxel_cell(Sd, tx * MG_TILE + (i % MG_TILE), ty * MG_TILE + (i / MG_TILE), cg, c);
        m0 = min(m0, c[0]);
        m1 = min(m1, c[1]);
        m2 = min(m2, c[2]);
    }
    cb0 = __reduce_min_sync(0xffffffffu, m0);
    cb1 = __reduce_min_sync(0xffffffffu, m1);
    cb2 = __reduce_min_sync(0xffffffffu, m2);
    for (int i = lane; i < NV; i += 32) {
        int c[3];
        voxel_cell(Sd, tx * MG_TILE + (i % MG_TILE), ty * MG_TILE + (i / MG_TILE), cg, c);
        srelw[i] = (unsigned)min(c[0] - cb0, 255) | ((unsigned)min(c[1] - cb1, 255) << 8) |
                   ((unsigned)min(c[2] - cb2, 255) << 16);
    }
    __syncwarp();
}

// Staged records of a forward warp, one float4 array per term so that the
// four quarter-warps' broadcast reads of consecutive records are
// conflict-free: (A, A, B, B), (C, C, D, D), (E, E, F, F), (amp, amp, -, -).
struct FwdStage {
    float4 ab[32], cd[32], ef[32], am[32];
};

// K4: one warp per 8x8 tile. Eight lane groups of four take every eighth
// record of the tile's list; lane c of a group owns pixel columns 2c and
// 2c+1 of the tile over its 8 rows, so a record's set-up is shared by 16
// voxels. Per record and lane: the two columns' coefficients
// a1 = B x + E, a0 = (A x + D) x + F as one packed pair each (three FP32x2
// FMAs), then per row q = (C y + a1) y + a0 (two packed FMAs), two ex2 and
// one packed FMA into the row's accumulator. The lane that stages a record
// rewrites it in the tile frame once. At the end the groups reduce-scatter
// their partial sums (14 shuffles, fixed order) and each lane writes one row
// of its two columns.
// CELLS: the paper's cell-grid local set; each (record, voxel) term is kept
// only when the voxel is a member (mgauss.h, MG_LOCAL_CELLS).
// The L1 + L2 slice loss of one voxel (mg_loss_l1l2): r = pred - target,
// dloss/dpred = (sign(r) + 2 r) / n; adds |r| and r^2 to the FP32 partials.
__device__ __forceinline__ void l1l2_voxel(float pred, float tgt, float inv_n, float *grad, float &f1, float &f2)
{
    const float r = pred - tgt;
    f1 += fabsf(r);
    f2 = fmaf(r, r, f2);
    if (grad) *grad = (copysignf(r != 0.f ? 1.f : 0.f, r) + 2.f * r) * inv_n;
}

// The fused loss of the forward (LOSS): per-voxel gradient and the tile's
// FP32 partials of |r| and r^2, written in FP64 to the tile's slot.
struct FwdLoss {
    const float *target;
    float *grad;
    double2 *tile_part;
    float inv_n;
};

template <bool CELLS, bool LOSS>
__device__ __forceinline__ void fwd_tile(const StackTable &tab, int t, int lane, FwdStage &sw, int4 *sgcw,
                                         unsigned *srelw, const unsigned *__restrict__ tile_off,
                                         const unsigned *__restrict__ entries, long long cap_entries,
                                         long long cap_records, const float4 *__restrict__ geo,
                                         const float2 *__restrict__ geo2, const SliceDev *__restrict__ slices,
                                         const CellGrid &cg, const int4 *__restrict__ rcell,
                                         const unsigned char *__restrict__ f64, const double *__restrict__ mom64,
                                         float *__restrict__ out, const FwdLoss &ls)
{
    const TileId d = tile_id(tab, t);
    const int grp = lane >> 2, c4 = lane & 3;
    const float x0c = (float)(d.tx * MG_TILE) + TC, y0c = (float)(d.ty * MG_TILE) + TC;
    unsigned e0 = tile_off[t], e1 = tile_off[t + 1];
    if ((long long)e1 > cap_entries) e1 = (unsigned)cap_entries;
    if (e0 > e1) e0 = e1;
    int cb0 = 0, cb1 = 0, cb2 = 0;
    uint2 rel[MG_TILE];  // CELLS: this lane's two columns of voxel cells, per row
    if (CELLS) {
        tile_cells(slices[tab.slice_base[d.s] + d.kk], cg, d.tx, d.ty, lane, srelw, cb0, cb1, cb2);
#pragma unroll
        for (int r = 0; r < MG_TILE; ++r) rel[r] = *(const uint2 *)&srelw[r * MG_TILE + 2 * c4];
    }
    // lane constants: the two column offsets and each row's offset as a pair
    // (an opaque zero added so that they stay in registers)
    const float rz = __uint_as_float(e1 & 0x80000000u);
    const float2 xo2 = make_float2((float)(2 * c4) - TC + rz, (float)(2 * c4 + 1) - TC + rz);
    float2 yy[MG_TILE];
#pragma unroll
    for (int r = 0; r < MG_TILE; ++r) yy[r] = make_float2((float)r - TC + rz, (float)r - TC + rz);
    float2 acc[MG_TILE];  // per row: (column 2 c4, column 2 c4 + 1)
#pragma unroll
    for (int r = 0; r < MG_TILE; ++r) acc[r] = make_float2(0.f, 0.f);
    // loads run two steps ahead: record ids two batches ahead, their
    // geometry one batch ahead (a zero record past the end)
    float4 na = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 nb = make_float2(0.f, 0.f);
    int4 nc = make_int4(0, 0, 0, 0);
    unsigned nr = 0xffffffffu;  // the staged record's id when it takes the FP64 geometry
    unsigned er = (e0 + lane < e1) ? entries[e0 + lane] : 0xffffffffu;
    if ((long long)er < cap_records) {
        na = geo[er];
        nb = geo2[er];
        if (CELLS) nc = rcell[er];
        if (f64[er] & 1) nr = er;
    }
    er = (e0 + 32 + lane < e1) ? entries[e0 + 32 + lane] : 0xffffffffu;
    for (unsigned base = e0; base < e1; base += 32) {
        {
            // stage this lane's record in the tile frame (a zero record past the end)
            const float A = na.z, B = na.w, C = nb.x;
            TileQuad tq = tile_quad(A, B, C, x0c - na.x, y0c - na.y);
            if (__any_sync(0xffffffffu, nr != 0xffffffffu) && nr != 0xffffffffu)
                tq = tile_quad_f64(mom64 + (size_t)nr * MOM64_STRIDE + MOM64_GEO, x0c, y0c);
            sw.ab[lane] = make_float4(A, A, B, B);
            sw.cd[lane] = make_float4(C, C, tq.D, tq.D);
            sw.ef[lane] = make_float4(tq.E, tq.E, tq.F, tq.F);
            sw.am[lane] = make_float4(nb.y, nb.y, 0.f, 0.f);
            if (CELLS) sgcw[lane] = nc;
        }
        __syncwarp();
        na = make_float4(0.f, 0.f, 0.f, 0.f);
        nb = make_float2(0.f, 0.f);
        nr = 0xffffffffu;
        if ((long long)er < cap_records) {
            na = geo[er];
            nb = geo2[er];
            if (CELLS) nc = rcell[er];
            if (f64[er] & 1) nr = er;
        }
        er = (base + 64 + lane < e1) ? entries[base + 64 + lane] : 0xffffffffu;
        const int m = (int)min(32u, e1 - base);
        for (int j8 = 0; j8 < m; j8 += 8) {
            const int j = j8 + grp;  // this group's record (a zero record past the end)
            const float4 ab = sw.ab[j], cd = sw.cd[j], ef = sw.ef[j], am = sw.am[j];
            const float2 A2 = make_float2(ab.x, ab.y), B2 = make_float2(ab.z, ab.w);
            const float2 C2 = make_float2(cd.x, cd.y), D2 = make_float2(cd.z, cd.w);
            const float2 E2 = make_float2(ef.x, ef.y), F2 = make_float2(ef.z, ef.w);
            float2 amp2 = make_float2(am.x, am.y);
            unsigned clo = 0u, chi = 0u;
            if (CELLS && !cell_range(sgcw[j], cg.R, cb0, cb1, cb2, clo, chi)) amp2 = make_float2(0.f, 0.f);
            const float2 a1 = __ffma2_rn(B2, xo2, E2);
            const float2 a0 = __ffma2_rn(__ffma2_rn(A2, xo2, D2), xo2, F2);
#pragma unroll
            for (int r = 0; r < MG_TILE; ++r) {
                const float2 q = __ffma2_rn(__ffma2_rn(C2, yy[r], a1), yy[r], a0);
                float2 e = make_float2(ex2_approx(q.x), ex2_approx(q.y));
                if (CELLS) {
                    if (!cell_member(rel[r].x, clo, chi)) e.x = 0.f;
                    if (!cell_member(rel[r].y, clo, chi)) e.y = 0.f;
                }
                acc[r] = __ffma2_rn(amp2, e, acc[r]);
            }
        }
        __syncwarp();
    }
    // reduce-scatter over the eight groups (lanes c4 + 4 g): across xor 16
    // the upper groups keep rows 4..7, across xor 8 the upper two of the
    // four, across xor 4 the upper one of the two; group g ends with row g
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int half = 4 >> k;  // rows kept after this step: 4, 2, 1
        const bool up = (lane >> (4 - k)) & 1;
#pragma unroll
        for (int r = 0; r < half; ++r) {
            const float2 send = up ? acc[r] : acc[r + half];
            float2 recv;
            recv.x = __shfl_xor_sync(0xffffffffu, send.x, 16 >> k);
            recv.y = __shfl_xor_sync(0xffffffffu, send.y, 16 >> k);
            const float2 keep = up ? acc[r + half] : acc[r];
            acc[r] = make_float2(keep.x + recv.x, keep.y + recv.y);
        }
    }
    const int px = d.tx * MG_TILE + 2 * c4, py = d.ty * MG_TILE + grp;
    float f1 = 0.f, f2 = 0.f;
    if (py < d.H) {
        const long long o = d.pixbase + (long long)py * d.W;
        float *row = out + o;
        if (px < d.W) {
            row[px] = acc[0].x;
            if (LOSS) l1l2_voxel(acc[0].x, ls.target[o + px], ls.inv_n, ls.grad ? ls.grad + o + px : nullptr, f1, f2);
        }
        if (px + 1 < d.W) {
            row[px + 1] = acc[0].y;
            if (LOSS)
                l1l2_voxel(acc[0].y, ls.target[o + px + 1], ls.inv_n, ls.grad ? ls.grad + o + px + 1 : nullptr, f1, f2);
        }
    }
    if (LOSS) {
        // the tile's partials by a fixed shuffle tree
#pragma unroll
        for (int k = 16; k > 0; k >>= 1) {
            f1 += __shfl_xor_sync(0xffffffffu, f1, k);
            f2 += __shfl_xor_sync(0xffffffffu, f2, k);
        }
        if (lane == 0) ls.tile_part[t] = make_double2((double)f1, (double)f2);
    }
}

// Up to SPARSE_CLAIM_FWD tiles of at most SPARSE_MAX records each (a fitted
// model's background), one claim: their records (at most 64) are staged once,
// each already in its tile's frame (A, B, C, amp | D, E, F), in the warp's
// FwdStage memory; then lane l computes pixels (2 (l mod 4), 2 (l mod 4) + 1)
// of row l / 4 of each tile over that tile's records in list order, with no
// reduce-scatter, writes them and the tile's loss partials. The tiles' loads
// overlap, where one tile at a time would wait on its own chain of loads.
constexpr unsigned SPARSE_CLAIM_FWD = 4;
template <bool LOSS>
__device__ __forceinline__ void fwd_sparse(const StackTable &tab, const unsigned *__restrict__ sparse_list, unsigned i0,
                                           unsigned nt, int lane, FwdStage &sw,
                                           const unsigned *__restrict__ tile_off, long long cap_entries,
                                           const unsigned *__restrict__ entries, long long cap_records,
                                           const float4 *__restrict__ geo, const float2 *__restrict__ geo2,
                                           const unsigned char *__restrict__ f64, const double *__restrict__ mom64,
                                           float *__restrict__ out, const FwdLoss &ls)
{
    // lane k < nt: tile k's entry range and position
    unsigned e0 = 0, e1 = 0;
    int t = 0, tx = 0, ty = 0, W = 0, H = 0;
    long long pb = 0;
    if ((unsigned)lane < nt) {
        t = (int)sparse_list[i0 + lane];
        e0 = tile_off[t];
        e1 = tile_off[t + 1];
        if ((long long)e1 > cap_entries) e1 = (unsigned)cap_entries;
        if (e0 > e1) e0 = e1;
        const TileId d = tile_id(tab, t);
        tx = d.tx;
        ty = d.ty;
        W = d.W;
        H = d.H;
        pb = d.pixbase;
    }
    const unsigned cnt = e1 - e0;
    unsigned incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const unsigned excl = incl - cnt;
    const unsigned total = __shfl_sync(0xffffffffu, incl, 31);  // at most SPARSE_CLAIM_FWD * SPARSE_MAX
    float4 *sab = sw.ab, *sdef = sw.cd;  // 64 records: sw.ab | sw.cd, sw.ef | sw.am
    // stage the claim's records, 32 at a time (record gi of the claim: tile k, entry gi - excl_k)
    for (unsigned base = 0; base < total; base += 32) {
        const unsigned gi = base + lane;
        int k = 0;
#pragma unroll
        for (int kk = 0; kk < (int)SPARSE_CLAIM_FWD; ++kk) k += (kk < (int)nt && gi >= __shfl_sync(0xffffffffu, incl, kk)) ? 1 : 0;
        const unsigned ek = __shfl_sync(0xffffffffu, e0, k), xk = __shfl_sync(0xffffffffu, excl, k);
        const unsigned ck = __shfl_sync(0xffffffffu, cnt, k);
        const int kx = __shfl_sync(0xffffffffu, tx, k), ky = __shfl_sync(0xffffffffu, ty, k);
        const bool act = gi < total && k < (int)nt && gi - xk < ck;
        unsigned r = act ? entries[ek + (gi - xk)] : 0xffffffffu;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 b = make_float2(0.f, 0.f);
        bool dbl = false;
        if ((long long)r < cap_records) {
            a = geo[r];
            b = geo2[r];
            dbl = f64[r] & 1;
        } else {
            r = 0xffffffffu;
        }
        const float x0c = (float)(kx * MG_TILE) + TC, y0c = (float)(ky * MG_TILE) + TC;
        TileQuad tq = tile_quad(a.z, a.w, b.x, x0c - a.x, y0c - a.y);
        if (__any_sync(0xffffffffu, dbl) && dbl) tq = tile_quad_f64(mom64 + (size_t)r * MOM64_STRIDE + MOM64_GEO, x0c, y0c);
        const float amp = r != 0xffffffffu ? b.y : 0.f;
        float4 *d0 = gi < 32 ? sab : sw.ef, *d1 = gi < 32 ? sdef : sw.am;
        if (gi < 64u) {
            d0[gi & 31u] = make_float4(a.z, a.w, b.x, amp);
            d1[gi & 31u] = make_float4(tq.D, tq.E, tq.F, 0.f);
        }
    }
    __syncwarp();
    // lane l: row l / 4, columns 2 (l mod 4), 2 (l mod 4) + 1 of each tile (tile-centred)
    const float y = (float)(lane >> 2) - TC;
    const float2 x2 = make_float2((float)(2 * (lane & 3)) - TC, (float)(2 * (lane & 3) + 1) - TC);
    for (unsigned k = 0; k < nt; ++k) {
        const unsigned lo = __shfl_sync(0xffffffffu, excl, k), hi = __shfl_sync(0xffffffffu, incl, k);
        float2 acc = make_float2(0.f, 0.f);
        for (unsigned i = lo; i < hi; ++i) {
            const float4 c0 = i < 32 ? sab[i] : sw.ef[i - 32], c1 = i < 32 ? sdef[i] : sw.am[i - 32];
            const float b1 = fmaf(c0.y, y, c1.x);                // B y + D
            const float b0 = fmaf(fmaf(c0.z, y, c1.y), y, c1.z);  // (C y + E) y + F
            const float2 q = __ffma2_rn(__ffma2_rn(make_float2(c0.x, c0.x), x2, make_float2(b1, b1)), x2,
                                        make_float2(b0, b0));
            const float2 e = make_float2(ex2_approx(q.x), ex2_approx(q.y));
            acc = __ffma2_rn(make_float2(c0.w, c0.w), e, acc);
        }
        const int kx = __shfl_sync(0xffffffffu, tx, k), ky = __shfl_sync(0xffffffffu, ty, k);
        const int kW = __shfl_sync(0xffffffffu, W, k), kH = __shfl_sync(0xffffffffu, H, k);
        const long long kp = __shfl_sync(0xffffffffu, pb, k);
        const int px = kx * MG_TILE + 2 * (lane & 3), py = ky * MG_TILE + (lane >> 2);
        float f1 = 0.f, f2 = 0.f;
        if (py < kH) {
            const long long o = kp + (long long)py * kW;
            if (px < kW) {
                out[o + px] = acc.x;
                if (LOSS) l1l2_voxel(acc.x, ls.target[o + px], ls.inv_n, ls.grad ? ls.grad + o + px : nullptr, f1, f2);
            }
            if (px + 1 < kW) {
                out[o + px + 1] = acc.y;
                if (LOSS)
                    l1l2_voxel(acc.y, ls.target[o + px + 1], ls.inv_n, ls.grad ? ls.grad + o + px + 1 : nullptr, f1, f2);
            }
        }
        if (LOSS) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                f1 += __shfl_xor_sync(0xffffffffu, f1, o);
                f2 += __shfl_xor_sync(0xffffffffu, f2, o);
            }
            const int tk = __shfl_sync(0xffffffffu, t, k);
            if (lane == 0) ls.tile_part[tk] = make_double2((double)f1, (double)f2);
        }
    }
}

// Persistent warps pull the tiles with records from a counter (tiles carry
// very different numbers of records); a warp that finds none left pulls the
// tiles without records 32 at a time from a second counter and writes their
// zeros (and loss terms) one lane per tile, so that work fills the tail.
// LOSS: the L1 + L2 slice loss and its gradient fused into the writes (the
// empty tiles' zeros included), one FP64 partial pair per tile.
template <bool CELLS, bool LOSS>
__global__ void __launch_bounds__(32 * RW, CELLS ? 4 : 8) k_render_fwd(StackTable tab, const unsigned *__restrict__ tile_off,
                                                          const unsigned *__restrict__ entries, long long cap_entries,
                                                          long long cap_records, const float4 *__restrict__ geo,
                                                          const float2 *__restrict__ geo2,
                                                          const SliceDev *__restrict__ slices, CellGrid cg,
                                                          const int4 *__restrict__ rcell,
                                                          const unsigned *__restrict__ tile_list,
                                                          const unsigned *__restrict__ dense_list,
                                                          const unsigned *__restrict__ sparse_list,
                                                          const WsHeader *__restrict__ hdr,
                                                          const unsigned char *__restrict__ f64,
                                                          const double *__restrict__ mom64, float *__restrict__ out,
                                                          FwdLoss ls, unsigned *counter, unsigned *sparse_ctr)
{
    pdl_entry();
    __shared__ FwdStage sg[RW];
    __shared__ int4 sgc[CELLS ? RW : 1][32];
    __shared__ __align__(16) unsigned srel[CELLS ? RW : 1][CELLS ? NV : 4];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long n_tiles = tab.n_tiles_total;
    const long long n_idle = hdr->n_idle, n_dense = hdr->n_dense, n_sparse = hdr->n_sparse;
    const long long n_bulk = max(0ll, n_dense - (long long)TILE_RESERVE * gridDim.x * RW);
    auto tile = [&](int t) {
        fwd_tile<CELLS, LOSS>(tab, t, lane, sg[w], sgc[CELLS ? w : 0], srel[CELLS ? w : 0], tile_off, entries,
                              cap_entries, cap_records, geo, geo2, slices, cg, rcell, f64, mom64, out, ls);
        __syncwarp();
    };
    // the dense tiles (more than SPARSE_MAX records): claims of two, then a reserve of single tiles
    for (unsigned part = 0; part < 2; ++part) {
        const long long lo = part ? n_bulk : 0, hi = part ? n_dense : n_bulk;
        const unsigned step = part ? 1u : TILE_CLAIM;
        for (;;) {
            unsigned i0 = 0;
            if (lane == 0) i0 = atomicAdd(part ? counter + 5 : counter, step);  // tile_ctr[0], tile_ctr[5]
            i0 = __shfl_sync(0xffffffffu, i0, 0);
            if (lo + (long long)i0 >= hi) break;
            for (long long i = lo + i0; i < lo + i0 + step && i < hi; ++i) tile((int)dense_list[i]);
        }
    }
    // the sparse tiles, SPARSE_CLAIM_FWD at a time (the cell-grid form one at a time)
    for (;;) {
        unsigned i0 = 0;
        if (lane == 0) i0 = atomicAdd(sparse_ctr, CELLS ? 1u : SPARSE_CLAIM_FWD);
        i0 = __shfl_sync(0xffffffffu, i0, 0);
        if ((long long)i0 >= n_sparse) break;
        if (CELLS) {
            tile((int)sparse_list[i0]);
        } else {
            fwd_sparse<LOSS>(tab, sparse_list, i0,
                             (unsigned)min((long long)SPARSE_CLAIM_FWD, n_sparse - (long long)i0), lane, sg[w],
                             tile_off, cap_entries, entries, cap_records, geo, geo2, f64, mom64, out, ls);
            __syncwarp();
        }
    }
    for (;;) {
        unsigned i0 = 0;
        if (lane == 0) i0 = atomicAdd(counter + 2, 32u);
        i0 = __shfl_sync(0xffffffffu, i0, 0);
        if ((long long)i0 >= n_idle) break;
        const long long i = (long long)i0 + lane;
        if (i < n_idle) {
            // one lane per empty tile: its rows as two float4 stores where aligned
            const TileId d = tile_id(tab, (int)tile_list[n_tiles - 1 - i]);
            const int px0 = d.tx * MG_TILE, py0 = d.ty * MG_TILE;
            const int nx = min(MG_TILE, d.W - px0), ny = min(MG_TILE, d.H - py0);
            float f1 = 0.f, f2 = 0.f;
            for (int r = 0; r < ny; ++r) {
                const long long o = d.pixbase + (long long)(py0 + r) * d.W + px0;
                float *row = out + o;
                if (nx == MG_TILE && ((uintptr_t)row & 15) == 0) {
                    ((float4 *)row)[0] = make_float4(0.f, 0.f, 0.f, 0.f);
                    ((float4 *)row)[1] = make_float4(0.f, 0.f, 0.f, 0.f);
                } else {
                    for (int c = 0; c < nx; ++c) row[c] = 0.f;
                }
                if (LOSS) {
                    float r1 = 0.f, r2 = 0.f;  // row partials, then added to the tile's
                    float gv[MG_TILE];
                    if (nx == MG_TILE && ((uintptr_t)(ls.target + o) & 15) == 0) {
                        const float4 t0 = ((const float4 *)(ls.target + o))[0], t1 = ((const float4 *)(ls.target + o))[1];
                        const float tv[MG_TILE] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
#pragma unroll
                        for (int c = 0; c < MG_TILE; ++c) l1l2_voxel(0.f, tv[c], ls.inv_n, &gv[c], r1, r2);
                        if (ls.grad && ((uintptr_t)(ls.grad + o) & 15) == 0) {
                            ((float4 *)(ls.grad + o))[0] = make_float4(gv[0], gv[1], gv[2], gv[3]);
                            ((float4 *)(ls.grad + o))[1] = make_float4(gv[4], gv[5], gv[6], gv[7]);
                        } else if (ls.grad) {
#pragma unroll
                            for (int c = 0; c < MG_TILE; ++c) ls.grad[o + c] = gv[c];
                        }
                    } else {
                        for (int c = 0; c < nx; ++c)
                            l1l2_voxel(0.f, ls.target[o + c], ls.inv_n, ls.grad ? ls.grad + o + c : nullptr, r1, r2);
                    }
                    f1 += r1;
                    f2 += r2;
                }
            }
            if (LOSS) ls.tile_part[tile_list[n_tiles - 1 - i]] = make_double2((double)f1, (double)f2);
        }
    }
}

// One record's six moments over the eight rows of its tile (w = g 2^q, g the
// tile's dL/dI in shared memory). Each half of the tile is swept towards the
// centre (rows 0..3, then rows 7..4) with per column pair running sums over
// the half's rows so far: a += g 2^q (one packed FMA, so w is never formed),
// zz += z, then z += a. At the end of a half, with n = 1..4 a row's distance
// from the half's end (n = 1 next to the centre, y = -/+(n - 1/2)):
// a = sum w, z = sum n w, zz = sum n (n - 1) / 2 w, so that
// sum y w = -/+(z - a/2) and sum y^2 w = 2 zz + a/4 (no cancellation in the
// even moments, at most 3x in the odd ones). Two adds per voxel instead of
// three weighted sums, and no per-row fold.
//
// CENTRE false: one sweep of the eight rows in order, z += a then zz += z, so
// that after row 7 (n = 8 - j, y = 4.5 - n) a = sum w, z = sum n w and
// zz = sum n (n + 1) / 2 w: one closed-form step per record, but the y^2
// moment 20.25 a - 10 z + 2 zz cancels up to ~80x when the weight sits in the
// middle rows. The backward takes the centre-out form for any batch holding a
// record of a Gaussian with a scale ratio above ELONG_RATIO (where the chain
// amplifies such errors), the single sweep otherwise.
template <bool CELLS, bool CENTRE>
__device__ __forceinline__ void record_rows8(const float2 &A2, float B, float C, const TileQuad &tq,
                                             const float *gt, const unsigned *srelw, unsigned clo, unsigned chi,
                                             const float2 *xp, const float2 *xq, float &T0, float &T1, float &T2,
                                             float &Y0, float &Y1, float &Y2)
{
    T0 = T1 = T2 = Y0 = Y1 = Y2 = 0.f;
    if (!CENTRE) {
        float2 ac[MG_TILE / 2], zc[MG_TILE / 2], zzc[MG_TILE / 2];
#pragma unroll
        for (int c = 0; c < MG_TILE / 2; ++c) ac[c] = zc[c] = zzc[c] = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < MG_TILE; ++j) {
            const float y = (float)j - TC;
            const float b1 = fmaf(B, y, tq.D);
            const float b0 = fmaf(fmaf(C, y, tq.E), y, tq.F);
            const float4 *gr = (const float4 *)&gt[j * MG_TILE];
            const uint4 *relr = (const uint4 *)&srelw[CELLS ? j * MG_TILE : 0];
            const float2 b12 = make_float2(b1, b1), b02 = make_float2(b0, b0);
#pragma unroll
            for (int i4 = 0; i4 < MG_TILE / 4; ++i4) {
                const float4 u = gr[i4];
                uint4 rl = make_uint4(0u, 0u, 0u, 0u);
                if (CELLS) rl = relr[i4];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c = i4 * 2 + h;
                    const float2 x = xp[c];
                    const float2 q = __ffma2_rn(__ffma2_rn(A2, x, b12), x, b02);
                    float2 e = make_float2(ex2_approx(q.x), ex2_approx(q.y));
                    if (CELLS) {
                        if (!cell_member(h ? rl.z : rl.x, clo, chi)) e.x = 0.f;
                        if (!cell_member(h ? rl.w : rl.y, clo, chi)) e.y = 0.f;
                    }
                    const float2 g2 = h ? make_float2(u.z, u.w) : make_float2(u.x, u.y);
                    if (j == 0) {  // first row: the three sums start at w
                        ac[c] = __fmul2_rn(g2, e);
                        zc[c] = ac[c];
                        zzc[c] = ac[c];
                    } else {
                        ac[c] = __ffma2_rn(g2, e, ac[c]);
                        zc[c] = __fadd2_rn(zc[c], ac[c]);
                        zzc[c] = __fadd2_rn(zzc[c], zc[c]);
                    }
                }
            }
        }
        float2 sa = ac[0], sxa = __fmul2_rn(xp[0], ac[0]), sxxa = __fmul2_rn(xq[0], ac[0]), sz = zc[0],
               sxz = __fmul2_rn(xp[0], zc[0]), szz = zzc[0];
#pragma unroll
        for (int c = 1; c < MG_TILE / 2; ++c) {
            sa = __fadd2_rn(sa, ac[c]);
            sxa = __ffma2_rn(xp[c], ac[c], sxa);
            sxxa = __ffma2_rn(xq[c], ac[c], sxxa);
            sz = __fadd2_rn(sz, zc[c]);
            sxz = __ffma2_rn(xp[c], zc[c], sxz);
            szz = __fadd2_rn(szz, zzc[c]);
        }
        const float SA = sa.x + sa.y, SXA = sxa.x + sxa.y, SZ = sz.x + sz.y, SXZ = sxz.x + sxz.y;
        const float Yc = (float)MG_TILE - TC;  // y = Yc - n
        T0 = SA;
        T1 = SXA;
        T2 = sxxa.x + sxxa.y;
        Y0 = fmaf(Yc, SA, -SZ);
        Y1 = fmaf(Yc, SXA, -SXZ);
        Y2 = fmaf(Yc * Yc, SA, fmaf(-(2.f * Yc + 1.f), SZ, 2.f * (szz.x + szz.y)));
        return;
    }
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        float2 ac[MG_TILE / 2], zc[MG_TILE / 2], zzc[MG_TILE / 2];
#pragma unroll
        for (int c = 0; c < MG_TILE / 2; ++c) ac[c] = zc[c] = zzc[c] = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < MG_TILE / 2; ++i) {
            const int j = half ? MG_TILE - 1 - i : i;  // towards the centre
            const float y = (float)j - TC;
            const float b1 = fmaf(B, y, tq.D);
            const float b0 = fmaf(fmaf(C, y, tq.E), y, tq.F);
            const float4 *gr = (const float4 *)&gt[j * MG_TILE];
            const uint4 *relr = (const uint4 *)&srelw[CELLS ? j * MG_TILE : 0];
            const float2 b12 = make_float2(b1, b1), b02 = make_float2(b0, b0);
#pragma unroll
            for (int i4 = 0; i4 < MG_TILE / 4; ++i4) {
                const float4 u = gr[i4];
                uint4 rl = make_uint4(0u, 0u, 0u, 0u);
                if (CELLS) rl = relr[i4];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c = i4 * 2 + h;
                    const float2 x = xp[c];
                    const float2 q = __ffma2_rn(__ffma2_rn(A2, x, b12), x, b02);
                    float2 e = make_float2(ex2_approx(q.x), ex2_approx(q.y));
                    if (CELLS) {
                        if (!cell_member(h ? rl.z : rl.x, clo, chi)) e.x = 0.f;
                        if (!cell_member(h ? rl.w : rl.y, clo, chi)) e.y = 0.f;
                    }
                    const float2 g2 = h ? make_float2(u.z, u.w) : make_float2(u.x, u.y);
                    if (i == 0) {  // the half's first row: a = z = w, zz = 0
                        ac[c] = __fmul2_rn(g2, e);
                        zc[c] = ac[c];
                    } else if (i == 1) {  // zz = z of the first row
                        ac[c] = __ffma2_rn(g2, e, ac[c]);
                        zzc[c] = zc[c];
                        zc[c] = __fadd2_rn(zc[c], ac[c]);
                    } else {
                        ac[c] = __ffma2_rn(g2, e, ac[c]);
                        zzc[c] = __fadd2_rn(zzc[c], zc[c]);
                        zc[c] = __fadd2_rn(zc[c], ac[c]);
                    }
                }
            }
        }
        float2 sa = ac[0], sxa = __fmul2_rn(xp[0], ac[0]), sxxa = __fmul2_rn(xq[0], ac[0]), sz = zc[0],
               sxz = __fmul2_rn(xp[0], zc[0]), szz = zzc[0];
#pragma unroll
        for (int c = 1; c < MG_TILE / 2; ++c) {
            sa = __fadd2_rn(sa, ac[c]);
            sxa = __ffma2_rn(xp[c], ac[c], sxa);
            sxxa = __ffma2_rn(xq[c], ac[c], sxxa);
            sz = __fadd2_rn(sz, zc[c]);
            sxz = __ffma2_rn(xp[c], zc[c], sxz);
            szz = __fadd2_rn(szz, zzc[c]);
        }
        const float SA = sa.x + sa.y, SXA = sxa.x + sxa.y, SZ = sz.x + sz.y, SXZ = sxz.x + sxz.y;
        const float sgn = half ? 1.f : -1.f;  // y = sgn (n - 1/2)
        T0 += SA;
        T1 += SXA;
        T2 += sxxa.x + sxxa.y;
        Y0 = fmaf(sgn, fmaf(-0.5f, SA, SZ), Y0);                         // sum y w
        Y1 = fmaf(sgn, fmaf(-0.5f, SXA, SXZ), Y1);                       // sum x y w
        Y2 += fmaf(2.f, szz.x + szz.y, 0.25f * SA);                      // sum y^2 w
    }
}

// A record's moments about the tile centre moved to the record centre and
// added to its slot: a float4 and a float2 atomic; near-degenerate records in
// FP64 (their moments about the centre are small differences of large terms,
// so the shift from the tile centre, by exact offsets, and the sum over tiles
// are in FP64).
__device__ __forceinline__ void record_add(unsigned r, int dbl, const double *g64, float x0c, float y0c, float dx0,
                                           float dy0, float T0, float T1, float T2, float Y0, float Y1, float Y2,
                                           float *__restrict__ mom, double *__restrict__ mom64)
{
    if (dbl) {
        const double X = (double)x0c - g64[MOM64_GEO], Y = (double)y0c - g64[MOM64_GEO + 1];
        const double t0 = T0, t1 = T1, t2 = T2, y0 = Y0, y1 = Y1, y2 = Y2;
        double *mr = mom64 + (size_t)r * MOM64_STRIDE;
        atomicAdd(mr + 0, t0);
        atomicAdd(mr + 1, fma(X, t0, t1));
        atomicAdd(mr + 2, fma(Y, t0, y0));
        atomicAdd(mr + 3, fma(X, fma(X, t0, t1 + t1), t2));
        atomicAdd(mr + 4, fma(X, fma(Y, t0, y0), fma(Y, t1, y1)));
        atomicAdd(mr + 5, fma(Y, fma(Y, t0, y0 + y0), y2));
    } else {
        float *mr = mom + (size_t)r * 8;
        atomicAdd((float4 *)mr, make_float4(T0, fmaf(dx0, T0, T1), fmaf(dy0, T0, Y0),
                                            fmaf(dx0, fmaf(dx0, T0, T1 + T1), T2)));
        atomicAdd((float2 *)(mr + 4), make_float2(fmaf(dx0, fmaf(dy0, T0, Y0), fmaf(dy0, T1, Y1)),
                                                  fmaf(dy0, fmaf(dy0, T0, Y0 + Y0), Y2)));
    }
}

// K5, "one lane per record": lane l takes record l of the tile's next 32
// entries and sweeps all 64 voxels of the tile, reading dL/dI from shared
// memory by broadcast. Per row y: b1 = B y + D, b0 = (C y + E) y + F; per
// column pair q = (A x + b1) x + b0 with packed FP32x2 FMAs, w = g 2^q, and
// three row sums (w, x w, x^2 w) with x and x^2 held in registers (only g is
// read from shared memory: broadcasting g x and g x^2 as well made the
// shared-memory path, at 12 bytes per pair and lane, the limit); per row the
// row sums fold into six moment accumulators with y. Moments are
// taken about the tile centre and moved to the record centre at the end; a
// lane then adds its record's six moments with a float4 and a float2 atomic.
// A batch of at most 16 records (a tile's last, or only, batch) splits each
// record's rows over 2, 4 or 8 lanes and sums their moments by shuffles first.
template <bool CELLS>
__device__ __forceinline__ void bwd_tile(const StackTable &tab, int t, unsigned e0, unsigned e1, int lane, float *sgvw,
                                         unsigned *srelw, const unsigned *__restrict__ entries,
                                         long long cap_records, const float4 *__restrict__ geo,
                                         const float2 *__restrict__ geo2, const SliceDev *__restrict__ slices,
                                         const CellGrid &cg, const int4 *__restrict__ rcell,
                                         const unsigned char *__restrict__ f64, const float *__restrict__ grad_out,
                                         float *__restrict__ mom, double *__restrict__ mom64)
{
    if (e0 >= e1) return;
    const TileId d = tile_id(tab, t);
    // dL/dI of the tile (shared by all records of the tile)
    for (int i = lane; i < NV; i += 32) {
        const int px = d.tx * MG_TILE + (i % MG_TILE), py = d.ty * MG_TILE + (i / MG_TILE);
        sgvw[i] = (px < d.W && py < d.H) ? grad_out[d.pixbase + (long long)py * d.W + px] : 0.f;
    }
    int cb0 = 0, cb1 = 0, cb2 = 0;
    if (CELLS) tile_cells(slices[tab.slice_base[d.s] + d.kk], cg, d.tx, d.ty, lane, srelw, cb0, cb1, cb2);
    __syncwarp();
    const float x0c = (float)(d.tx * MG_TILE) + TC, y0c = (float)(d.ty * MG_TILE) + TC;
    // column offsets as register pairs, formed once per tile (an opaque zero
    // added so that they stay in registers)
    const float rz = __uint_as_float(e1 & 0x80000000u);
    float2 xp[MG_TILE / 2], xq[MG_TILE / 2];
#pragma unroll
    for (int c = 0; c < MG_TILE / 2; ++c) {
        xp[c] = make_float2((float)(2 * c) - TC + rz, (float)(2 * c + 1) - TC + rz);
        xq[c] = make_float2(((float)(2 * c) - TC) * ((float)(2 * c) - TC) + rz,
                            ((float)(2 * c + 1) - TC) * ((float)(2 * c + 1) - TC) + rz);
    }
    // the next batch of 32 records is fetched while the current one is swept
    // loads run two steps ahead: record ids two batches ahead, their
    // geometry one batch ahead
    unsigned nr = 0xffffffffu;
    float4 na = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 nb = make_float2(0.f, 0.f);
    int4 ncl = make_int4(0, 0, 0, 0);
    int nf = 0;
    unsigned er = (e0 + lane < e1) ? entries[e0 + lane] : 0xffffffffu;
    if ((long long)er < cap_records) {
        nr = er;
        na = geo[er];
        nb = geo2[er];
        nf = f64[er];
        if (CELLS) ncl = rcell[er];
    }
    er = (e0 + 32 + lane < e1) ? entries[e0 + 32 + lane] : 0xffffffffu;
    for (unsigned base = e0; base < e1; base += 32) {
        unsigned r = nr;
        float4 a = na;
        float2 b = nb;
        int4 cl = ncl;
        int dbl = nf;
        nr = 0xffffffffu;
        na = make_float4(0.f, 0.f, 0.f, 0.f);
        nb = make_float2(0.f, 0.f);
        nf = 0;
        if ((long long)er < cap_records) {
            nr = er;
            na = geo[er];
            nb = geo2[er];
            nf = f64[er];
            if (CELLS) ncl = rcell[er];
        }
        er = (base + 64 + lane < e1) ? entries[base + 64 + lane] : 0xffffffffu;
        // A batch of m <= 16 records splits each record's 8 rows over L = 2,
        // 4 or 8 lanes (lane l: record l mod 32/L, rows (l div 32/L) 8/L ..),
        // so that a sparse tile does not leave most lanes idle; the L partial
        // moment sets are summed by shuffles before the atomics.
        const unsigned m = min(32u, e1 - base);
        const int lg = m > 16u ? 0 : m > 8u ? 1 : m > 4u ? 2 : 3;  // log2 L (warp-uniform)
        const int P = 32 >> lg;                                 // records per pass
        int j0 = 0;
        if (lg) {
            const int src = lane & (P - 1);
            r = __shfl_sync(0xffffffffu, r, src);
            a.x = __shfl_sync(0xffffffffu, a.x, src);
            a.y = __shfl_sync(0xffffffffu, a.y, src);
            a.z = __shfl_sync(0xffffffffu, a.z, src);
            a.w = __shfl_sync(0xffffffffu, a.w, src);
            b.x = __shfl_sync(0xffffffffu, b.x, src);
            dbl = __shfl_sync(0xffffffffu, dbl, src);
            if (CELLS) {
                cl.x = __shfl_sync(0xffffffffu, cl.x, src);
                cl.y = __shfl_sync(0xffffffffu, cl.y, src);
                cl.z = __shfl_sync(0xffffffffu, cl.z, src);
                cl.w = __shfl_sync(0xffffffffu, cl.w, src);
            }
            j0 = (lane >> (5 - lg)) << (3 - lg);
        }
        const bool elong = dbl != 0;  // bit 1: scale ratio above ELONG_RATIO (bit 0, FP64, implies it)
        dbl &= 1;
        unsigned clo = 0u, chi = 0u;
        if (CELLS && r != 0xffffffffu && !cell_range(cl, cg.R, cb0, cb1, cb2, clo, chi)) r = 0xffffffffu;
        const float A = a.z, B = a.w, C = b.x;
        const float dx0 = x0c - a.x;  // the tile centre's offset from the record centre
        const float dy0 = y0c - a.y;
        TileQuad tq = tile_quad(A, B, C, dx0, dy0);
        const bool tdbl = dbl && r != 0xffffffffu;
        const double *g64 = mom64 + (size_t)(tdbl ? r : 0u) * MOM64_STRIDE;
        if (__any_sync(0xffffffffu, tdbl) && tdbl) tq = tile_quad_f64(g64 + MOM64_GEO, x0c, y0c);
        const float2 A2 = make_float2(A, A);
        float T0 = 0.f, T1 = 0.f, T2 = 0.f, Y0 = 0.f, Y1 = 0.f, Y2 = 0.f;
        // one row y of the record: three row sums, folded into the six moments
        auto row = [&](int j, float y) {
            const float b1 = fmaf(B, y, tq.D);
            const float b0 = fmaf(fmaf(C, y, tq.E), y, tq.F);
            const float4 *gr = (const float4 *)&sgvw[j * MG_TILE];
            const uint4 *relr = (const uint4 *)&srelw[CELLS ? j * MG_TILE : 0];
            // column pairs (i, i+1) with packed FP32x2 arithmetic: w = g e,
            // P0 += w, P1 += x w, P2 += x^2 w
            const float2 b12 = make_float2(b1, b1), b02 = make_float2(b0, b0);
            float2 P0 = make_float2(0.f, 0.f), P1 = P0, P2 = P0;
#pragma unroll
            for (int i4 = 0; i4 < MG_TILE / 4; ++i4) {
                const float4 u = gr[i4];
                uint4 rl = make_uint4(0u, 0u, 0u, 0u);
                if (CELLS) rl = relr[i4];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float2 x = xp[i4 * 2 + h];
                    const float2 q = __ffma2_rn(__ffma2_rn(A2, x, b12), x, b02);
                    float2 e = make_float2(ex2_approx(q.x), ex2_approx(q.y));
                    if (CELLS) {
                        if (!cell_member(h ? rl.z : rl.x, clo, chi)) e.x = 0.f;
                        if (!cell_member(h ? rl.w : rl.y, clo, chi)) e.y = 0.f;
                    }
                    const float2 w = __fmul2_rn(h ? make_float2(u.z, u.w) : make_float2(u.x, u.y), e);
                    P0 = __fadd2_rn(P0, w);
                    P1 = __ffma2_rn(x, w, P1);
                    P2 = __ffma2_rn(xq[i4 * 2 + h], w, P2);
                }
            }
            const float R0 = P0.x + P0.y, R1 = P1.x + P1.y, R2 = P2.x + P2.y;
            T0 += R0;
            T1 += R1;
            T2 += R2;
            Y0 = fmaf(y, R0, Y0);
            Y1 = fmaf(y, R1, Y1);
            Y2 = fmaf(y * y, R0, Y2);
        };
        if (lg == 0) {
            if (__any_sync(0xffffffffu, elong && r != 0xffffffffu))
                record_rows8<CELLS, true>(A2, B, C, tq, sgvw, srelw, clo, chi, xp, xq, T0, T1, T2, Y0, Y1, Y2);
            else
                record_rows8<CELLS, false>(A2, B, C, tq, sgvw, srelw, clo, chi, xp, xq, T0, T1, T2, Y0, Y1, Y2);
        } else {
            const int nrow = MG_TILE >> lg;
            float y = (float)j0 - TC;
            for (int j = j0; j < j0 + nrow; ++j, y += 1.f) row(j, y);
            // the L partial sets of each record, summed over lanes src + k P
            for (int o = P; o < 32; o <<= 1) {
                T0 += __shfl_xor_sync(0xffffffffu, T0, o);
                T1 += __shfl_xor_sync(0xffffffffu, T1, o);
                T2 += __shfl_xor_sync(0xffffffffu, T2, o);
                Y0 += __shfl_xor_sync(0xffffffffu, Y0, o);
                Y1 += __shfl_xor_sync(0xffffffffu, Y1, o);
                Y2 += __shfl_xor_sync(0xffffffffu, Y2, o);
            }
            if (lane >= P) r = 0xffffffffu;  // one lane per record adds it
        }
        if (r != 0xffffffffu) record_add(r, dbl, g64, x0c, y0c, dx0, dy0, T0, T1, T2, Y0, Y1, Y2, mom, mom64);
    }
}

// Up to SPARSE_CLAIM tiles of at most SPARSE_MAX records each (a fitted
// model's background: most tiles hold a handful of records), their records
// packed into batches of up to 32 lanes (tiles whole), each lane over all
// eight rows of its own tile: the tiles' loads overlap and no rows are split
// over lanes. The tiles' dL/dI is staged once, tile k at 68 k words, so that
// the tiles' rows fall in different banks.
constexpr int SG = NV + 4;
__device__ __forceinline__ void bwd_sparse(const StackTable &tab, const unsigned *__restrict__ sparse_list,
                                           unsigned i0, unsigned nt, int lane, float *sgvw,
                                           const unsigned *__restrict__ tile_off, long long cap_entries,
                                           const unsigned *__restrict__ entries, long long cap_records,
                                           const float4 *__restrict__ geo, const float2 *__restrict__ geo2,
                                           const unsigned char *__restrict__ f64, const float *__restrict__ grad_out,
                                           float *__restrict__ mom, double *__restrict__ mom64)
{
    // lane k < nt: tile k's entry range and position
    unsigned e0 = 0, e1 = 0;
    int tx = 0, ty = 0, W = 0, H = 0;
    long long pb = 0;
    if ((unsigned)lane < nt) {
        const int t = (int)sparse_list[i0 + lane];
        e0 = tile_off[t];
        e1 = tile_off[t + 1];
        if ((long long)e1 > cap_entries) e1 = (unsigned)cap_entries;
        if (e0 > e1) e0 = e1;
        const TileId d = tile_id(tab, t);
        tx = d.tx;
        ty = d.ty;
        W = d.W;
        H = d.H;
        pb = d.pixbase;
    }
    // the tiles' dL/dI, all loads in flight before the stores: half-tile j of tile j / 2
    float gv[2 * SPARSE_CLAIM];
#pragma unroll
    for (int j = 0; j < 2 * (int)SPARSE_CLAIM; ++j) {
        const int k = j >> 1, v = (j & 1) * 32 + lane;
        const int kx = __shfl_sync(0xffffffffu, tx, k), ky = __shfl_sync(0xffffffffu, ty, k);
        const int kW = __shfl_sync(0xffffffffu, W, k), kH = __shfl_sync(0xffffffffu, H, k);
        const long long kp = __shfl_sync(0xffffffffu, pb, k);
        const int px = kx * MG_TILE + (v % MG_TILE), py = ky * MG_TILE + (v / MG_TILE);
        gv[j] = (j < 2 * (int)nt && px < kW && py < kH) ? grad_out[kp + (long long)py * kW + px] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < 2 * (int)SPARSE_CLAIM; ++j)
        if (j < 2 * (int)nt) sgvw[(j >> 1) * SG + (j & 1) * 32 + lane] = gv[j];
    __syncwarp();
    // inclusive prefix of the tiles' record counts
    const unsigned cnt = e1 - e0;
    unsigned incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const unsigned excl = incl - cnt;
    const float rz = __uint_as_float(e1 & 0x80000000u);
    float2 xp[MG_TILE / 2], xq[MG_TILE / 2];
#pragma unroll
    for (int c = 0; c < MG_TILE / 2; ++c) {
        xp[c] = make_float2((float)(2 * c) - TC + rz, (float)(2 * c + 1) - TC + rz);
        xq[c] = make_float2(((float)(2 * c) - TC) * ((float)(2 * c) - TC) + rz,
                            ((float)(2 * c + 1) - TC) * ((float)(2 * c + 1) - TC) + rz);
    }
    unsigned lem;
    asm("mov.u32 %0, %%lanemask_le;" : "=r"(lem));
    for (unsigned s = 0; s < nt;) {
        // the batch: tiles s..e whole, at most 32 records (each tile holds at most SPARSE_MAX)
        const unsigned base = __shfl_sync(0xffffffffu, excl, s);
        const bool in = (unsigned)lane >= s && (unsigned)lane < nt && incl - base <= 32u;
        const unsigned fit = __ballot_sync(0xffffffffu, in);
        const unsigned e = 31u - __clz(fit);
        const unsigned end = __shfl_sync(0xffffffffu, incl, e);
        // lane l takes record base + l: its tile is the last tile of the batch starting at or before l
        // (a tile left without entries by a capacity overflow starts where the
        // next does; the count check below keeps every read inside its tile)
        const unsigned starts = __reduce_or_sync(0xffffffffu, in && excl - base < 32u ? 1u << (excl - base) : 0u);
        const unsigned gi = base + lane;
        const int k = (int)s + __popc(starts & lem) - 1;
        const unsigned ek = __shfl_sync(0xffffffffu, e0, k), xk = __shfl_sync(0xffffffffu, excl, k);
        const unsigned ck = __shfl_sync(0xffffffffu, cnt, k);
        const int kx = __shfl_sync(0xffffffffu, tx, k), ky = __shfl_sync(0xffffffffu, ty, k);
        const bool act = gi < end && k >= (int)s && gi - xk < ck;
        unsigned r = act ? entries[ek + (gi - xk)] : 0xffffffffu;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 b = make_float2(0.f, 0.f);
        int dbl = 0;
        if ((long long)r < cap_records) {
            a = geo[r];
            b = geo2[r];
            dbl = f64[r];
        } else {
            r = 0xffffffffu;
        }
        const bool elong = dbl != 0;  // bit 1: scale ratio above ELONG_RATIO (bit 0, FP64, implies it)
        dbl &= 1;
        const float x0c = (float)(kx * MG_TILE) + TC, y0c = (float)(ky * MG_TILE) + TC;
        const float A = a.z, B = a.w, C = b.x;
        const float dx0 = x0c - a.x, dy0 = y0c - a.y;
        TileQuad tq = tile_quad(A, B, C, dx0, dy0);
        const bool tdbl = dbl && r != 0xffffffffu;
        const double *g64 = mom64 + (size_t)(tdbl ? r : 0u) * MOM64_STRIDE;
        if (__any_sync(0xffffffffu, tdbl) && tdbl) tq = tile_quad_f64(g64 + MOM64_GEO, x0c, y0c);
        float T0, T1, T2, Y0, Y1, Y2;
        const float *gk = sgvw + (act ? k : 0) * SG;
        if (__any_sync(0xffffffffu, elong))
            record_rows8<false, true>(make_float2(A, A), B, C, tq, gk, nullptr, 0u, 0u, xp, xq, T0, T1, T2, Y0, Y1, Y2);
        else
            record_rows8<false, false>(make_float2(A, A), B, C, tq, gk, nullptr, 0u, 0u, xp, xq, T0, T1, T2, Y0, Y1, Y2);
        if (r != 0xffffffffu) record_add(r, dbl, g64, x0c, y0c, dx0, dy0, T0, T1, T2, Y0, Y1, Y2, mom, mom64);
        s = e + 1;
    }
}

template <bool CELLS>
__global__ void __launch_bounds__(32 * RW, 5) k_render_bwd(StackTable tab, const unsigned *__restrict__ tile_off,
                                                          const unsigned *__restrict__ entries, long long cap_entries,
                                                          long long cap_records, const float4 *__restrict__ geo,
                                                          const float2 *__restrict__ geo2,
                                                          const SliceDev *__restrict__ slices, CellGrid cg,
                                                          const int4 *__restrict__ rcell,
                                                          const unsigned *__restrict__ dense_list,
                                                          const unsigned *__restrict__ sparse_list,
                                                          const WsHeader *__restrict__ hdr,
                                                          const unsigned char *__restrict__ f64,
                                                          const float *__restrict__ grad_out, float *__restrict__ mom,
                                                          double *__restrict__ mom64, unsigned *counter)
{
    pdl_entry();
    __shared__ __align__(16) float sgv[RW][SPARSE_CLAIM * SG];
    __shared__ __align__(16) unsigned srel[CELLS ? RW : 1][CELLS ? NV : 4];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long n_dense = hdr->n_dense, n_sparse = hdr->n_sparse;
    const long long n_bulk = max(0ll, n_dense - (long long)TILE_RESERVE * gridDim.x * RW);
    auto tile = [&](int t) {
        unsigned e0 = tile_off[t], e1 = tile_off[t + 1];
        if ((long long)e1 > cap_entries) e1 = (unsigned)cap_entries;
        if (e0 > e1) e0 = e1;
        bwd_tile<CELLS>(tab, t, e0, e1, lane, sgv[w], srel[CELLS ? w : 0], entries, cap_records, geo, geo2, slices,
                        cg, rcell, f64, grad_out, mom, mom64);
        __syncwarp();
    };
    // the dense tiles: claims of two, then a reserve of single tiles
    for (unsigned part = 0; part < 2; ++part) {
        const long long lo = part ? n_bulk : 0, hi = part ? n_dense : n_bulk;
        const unsigned step = part ? 1u : TILE_CLAIM;
        for (;;) {
            unsigned i0 = 0;
            if (lane == 0) i0 = atomicAdd(part ? counter + 3 : counter, step);  // tile_ctr[1], tile_ctr[4]
            i0 = __shfl_sync(0xffffffffu, i0, 0);
            if (lo + (long long)i0 >= hi) break;
            for (long long i = lo + i0; i < lo + i0 + step && i < hi; ++i) tile((int)dense_list[i]);
        }
    }
    // the sparse tiles, SPARSE_CLAIM at a time (the cell-grid form one at a time)
    for (;;) {
        unsigned i0 = 0;
        if (lane == 0) i0 = atomicAdd(counter + 1, CELLS ? 1u : SPARSE_CLAIM);  // tile_ctr[2]
        i0 = __shfl_sync(0xffffffffu, i0, 0);
        if ((long long)i0 >= n_sparse) break;
        if (CELLS) {
            tile((int)sparse_list[i0]);
        } else {
            bwd_sparse(tab, sparse_list, i0, (unsigned)min((long long)SPARSE_CLAIM, n_sparse - (long long)i0), lane,
                       sgv[w], tile_off, cap_entries, entries, cap_records, geo, geo2, f64, grad_out, mom, mom64);
            __syncwarp();
        }
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
__device__ __forceinline__ T c_rcp(T x);
template <>
__device__ __forceinline__ float c_rcp<float>(float x) { return __frcp_rn(x); }
template <>
__device__ __forceinline__ double c_rcp<double>(double x) { return 1.0 / x; }
template <typename T>
__device__ __forceinline__ T c_rsqrt(T x);
template <>
__device__ __forceinline__ float c_rsqrt<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double c_rsqrt<double>(double x) { return 1.0 / sqrt(x); }

// Adjoint of the record geometry: (centre, conic, amp) of the record of a
// Gaussian on a slice, given dL/d(pcx, pcy, A, B2, C, amp).
// POSE: also the record's share of the slice-pose gradient, gpose[0..2] =
// dL/dt (world) and gpose[3..5] = dL/domega for the slice rotation perturbed
// as R (I + [omega]x) (omega in the slice frame). With d = R^T (mu - t) and
// P = R^T R_gauss the record geometry's only slice-dependent inputs,
// delta d = -omega x d and delta P = -[omega]x P, so dL/domega =
// g_d x d + axial part of (P gP^T) (dL/dP = gP).
// Per-Gaussian part of the record geometry: the rotation of q and the scales.
template <typename T>
struct GaussFrame {
    T R[3][3], sc[3], isc[3];
};
template <typename T>
__device__ __forceinline__ void gauss_frame(const float *q, const float *s, GaussFrame<T> &F)
{
    const T w = q[0], x = q[1], y = q[2], z = q[3];
    F.R[0][0] = 1 - 2 * (y * y + z * z);
    F.R[0][1] = 2 * (x * y - w * z);
    F.R[0][2] = 2 * (x * z + w * y);
    F.R[1][0] = 2 * (x * y + w * z);
    F.R[1][1] = 1 - 2 * (x * x + z * z);
    F.R[1][2] = 2 * (y * z - w * x);
    F.R[2][0] = 2 * (x * z - w * y);
    F.R[2][1] = 2 * (y * z + w * x);
    F.R[2][2] = 1 - 2 * (x * x + y * y);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        F.sc[c] = s[c];
        F.isc[c] = c_rcp<T>(F.sc[c]);
    }
}

// dL/dq from dL/dR (R the rotation of q; linear in dL/dR, so it may be
// applied once to a sum over records).
template <typename T>
__device__ __forceinline__ void quat_adjoint(const float *q, const T gR[3][3], T gq[4])
{
    const T w = q[0], x = q[1], y = q[2], z = q[3];
    gq[0] = 2 * (-z * gR[0][1] + y * gR[0][2] + z * gR[1][0] - x * gR[1][2] - y * gR[2][0] + x * gR[2][1]);
    gq[1] = 2 * (y * gR[0][1] + z * gR[0][2] + y * gR[1][0] - 2 * x * gR[1][1] - w * gR[1][2] + z * gR[2][0] +
                 w * gR[2][1] - 2 * x * gR[2][2]);
    gq[2] = 2 * (-2 * y * gR[0][0] + x * gR[0][1] + w * gR[0][2] + x * gR[1][0] + z * gR[1][2] - w * gR[2][0] +
                 z * gR[2][1] - 2 * y * gR[2][2]);
    gq[3] = 2 * (-2 * z * gR[0][0] - w * gR[0][1] + x * gR[0][2] + w * gR[1][0] - 2 * z * gR[1][1] + y * gR[1][2] +
                 x * gR[2][0] + y * gR[2][1]);
}

// Adjoint of one record's geometry (the record pass's formulas recomputed):
// dL/d(conic A, B2, C, centre px, py, amp) -> dL/d(mean, R, scale, alpha),
// ADDED to gmu, gR, gs, galpha; POSE: also the record's share of the slice
// pose gradient (dL/dt, dL/domega) written to gpose.
template <typename T, bool POSE = false>
__device__ __forceinline__ void record_adjoint(const GaussFrame<T> &F, const float *mu, float alpha, const SliceDev &S,
                                               T gA, T gB2, T gC, T gpx, T gpy, T gamp, T gmu[3], T gR[3][3],
                                               T gs[3], T &galpha, T *gpose = nullptr)
{
    T Q[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) Q[i] = (T)S.Q[i];
    T P[3][3], g[3][3], Lm[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            P[a][c] = Q[a] * F.R[0][c] + Q[3 + a] * F.R[1][c] + Q[6 + a] * F.R[2][c];
            g[a][c] = P[a][c] * F.isc[c];
            Lm[a][c] = P[a][c] * F.sc[c];
        }
    T p0 = (T)mu[0] - (T)S.t[0], p1 = (T)mu[1] - (T)S.t[1], p2 = (T)mu[2] - (T)S.t[2];
    T w0 = Q[2] * p0 + Q[5] * p1 + Q[8] * p2;
    T Huw = g[0][0] * g[2][0] + g[0][1] * g[2][1] + g[0][2] * g[2][2];
    T Hvw = g[1][0] * g[2][0] + g[1][1] * g[2][1] + g[1][2] * g[2][2];
    T Hww = g[2][0] * g[2][0] + g[2][1] * g[2][1] + g[2][2] * g[2][2];
    T Suw = Lm[0][0] * Lm[2][0] + Lm[0][1] * Lm[2][1] + Lm[0][2] * Lm[2][2];
    T Svw = Lm[1][0] * Lm[2][0] + Lm[1][1] * Lm[2][1] + Lm[1][2] * Lm[2][2];
    T sig2 = (T)S.sig2;
    T Sww = Lm[2][0] * Lm[2][0] + Lm[2][1] * Lm[2][1] + Lm[2][2] * Lm[2][2] + sig2;
    T iSww = c_rcp<T>(Sww);
    T D = 1 + sig2 * Hww;
    T rD = c_rsqrt<T>(D);
    T iD = rD * rD;
    T f = sig2 * iD;
    T wS = w0 * iSww;
    T E = c_exp<T>((T)(-0.5) * w0 * wS);
    T amp = (T)alpha * rD * E;
    const T kap = (T)(-0.72134752044448170368);
    T dx = S.dx, dy = S.dy;
    // reverse
    T gKuu = gA * kap * dx * dx;
    T gKuv = gB2 * 2 * kap * dx * dy;
    T gKvv = gC * kap * dy * dy;
    T gcu = gpx * c_rcp<T>(dx), gcv = gpy * c_rcp<T>(dy);
    if (S.pu2 > 0.f || S.pv2 > 0.f) {
        // adjoint of the in-plane PSF step K -> (K^-1 + P)^-1, amp -> amp m^-1/2
        // (record pass): gradients with respect to the PSF-free K and amp
        T Huu = g[0][0] * g[0][0] + g[0][1] * g[0][1] + g[0][2] * g[0][2];
        T Huv = g[0][0] * g[1][0] + g[0][1] * g[1][1] + g[0][2] * g[1][2];
        T Hvv = g[1][0] * g[1][0] + g[1][1] * g[1][1] + g[1][2] * g[1][2];
        T K0uu = Huu - f * Huw * Huw, K0uv = Huv - f * Huw * Hvw, K0vv = Hvv - f * Hvw * Hvw;
        const T pu2 = (T)S.pu2, pv2 = (T)S.pv2;
        T dK = K0uu * K0vv - K0uv * K0uv;
        T m = 1 + pu2 * K0uu + pv2 * K0vv + pu2 * pv2 * dK;
        T im = c_rcp<T>(m), rm = c_rsqrt<T>(m);
        T Kpuu = (K0uu + pv2 * dK) * im, Kpuv = K0uv * im, Kpvv = (K0vv + pu2 * dK) * im;
        T gm = -(gKuu * Kpuu + gKuv * Kpuv + gKvv * Kpvv) * im - (T)0.5 * gamp * amp * rm * im;
        T gNuu = gKuu * im, gNuv = gKuv * im, gNvv = gKvv * im;
        T gdK = pv2 * gNuu + pu2 * gNvv + gm * pu2 * pv2;
        gKuu = gNuu + gm * pu2 + gdK * K0vv;
        gKvv = gNvv + gm * pv2 + gdK * K0uu;
        gKuv = gNuv - 2 * gdK * K0uv;
        gamp = gamp * rm;
    }
    galpha += gamp * rD * E;
    T ga = gamp * amp;
    T gD = (T)(-0.5) * ga * iD;
    T gw0 = -ga * wS;
    T gSww = (T)0.5 * ga * wS * wS;
    T gdu = gcu, gdv = gcv;
    T gSuw = -gcu * wS;
    T gSvw = -gcv * wS;
    T cs = gcu * Suw + gcv * Svw;
    gw0 -= cs * iSww;
    gSww += cs * wS * iSww;
    T gHuu = gKuu, gHvv = gKvv, gHuv = gKuv;
    T gHuw = -f * (2 * gKuu * Huw + gKuv * Hvw);
    T gHvw = -f * (2 * gKvv * Hvw + gKuv * Huw);
    gD += f * iD * (gKuu * Huw * Huw + gKuv * Huw * Hvw + gKvv * Hvw * Hvw);
    T gHww = sig2 * gD;
    T M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  // P gP^T (POSE)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        T gg0 = 2 * gHuu * g[0][c] + gHuv * g[1][c] + gHuw * g[2][c];
        T gg1 = 2 * gHvv * g[1][c] + gHuv * g[0][c] + gHvw * g[2][c];
        T gg2 = 2 * gHww * g[2][c] + gHuw * g[0][c] + gHvw * g[1][c];
        T gL0 = gSuw * Lm[2][c];
        T gL1 = gSvw * Lm[2][c];
        T gL2 = gSuw * Lm[0][c] + gSvw * Lm[1][c] + 2 * gSww * Lm[2][c];
        T gP0 = gg0 * F.isc[c] + gL0 * F.sc[c];
        T gP1 = gg1 * F.isc[c] + gL1 * F.sc[c];
        T gP2 = gg2 * F.isc[c] + gL2 * F.sc[c];
        gs[c] += -(gg0 * g[0][c] + gg1 * g[1][c] + gg2 * g[2][c]) * F.isc[c] +
                 (gL0 * P[0][c] + gL1 * P[1][c] + gL2 * P[2][c]);
#pragma unroll
        for (int r = 0; r < 3; ++r) gR[r][c] += Q[3 * r] * gP0 + Q[3 * r + 1] * gP1 + Q[3 * r + 2] * gP2;
        if (POSE) {
#pragma unroll
            for (int a2 = 0; a2 < 3; ++a2) {
                M[a2][0] += P[a2][c] * gP0;
                M[a2][1] += P[a2][c] * gP1;
                M[a2][2] += P[a2][c] * gP2;
            }
        }
    }
    T rmu[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        rmu[r] = Q[3 * r] * gdu + Q[3 * r + 1] * gdv + Q[3 * r + 2] * gw0;
        gmu[r] += rmu[r];
    }
    if (POSE) {
        const T u0 = Q[0] * p0 + Q[3] * p1 + Q[6] * p2, v0 = Q[1] * p0 + Q[4] * p1 + Q[7] * p2;
        gpose[0] = -rmu[0];
        gpose[1] = -rmu[1];
        gpose[2] = -rmu[2];
        gpose[3] = (gdv * w0 - gw0 * v0) + (M[2][1] - M[1][2]);
        gpose[4] = (gw0 * u0 - gdu * w0) + (M[0][2] - M[2][0]);
        gpose[5] = (gdu * v0 - gdv * u0) + (M[1][0] - M[0][1]);
    }
}

// The whole adjoint of one record (the Gaussian's frame computed here).
template <typename T, bool POSE = false>
__device__ void geometry_adjoint(const float *mu, const float *q, const float *s, float alpha, const SliceDev &S,
                                 T gA, T gB2, T gC, T gpx, T gpy, T gamp, T gmu[3], T gq[4], T gs[3], T &galpha,
                                 T *gpose = nullptr)
{
    GaussFrame<T> F;
    gauss_frame<T>(q, s, F);
    T gR[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    gmu[0] = gmu[1] = gmu[2] = 0;
    gs[0] = gs[1] = gs[2] = 0;
    galpha = 0;
    record_adjoint<T, POSE>(F, mu, alpha, S, gA, gB2, gC, gpx, gpy, gamp, gmu, gR, gs, galpha, gpose);
    quat_adjoint<T>(q, gR, gq);
}

__global__ void k_zero_mom(float4 *mom, const unsigned char *__restrict__ f64, double2 *mom64, const WsHeader *hdr,
                           long long cap_records)
{
    pdl_entry();
    long long n = (long long)hdr->n_records;
    if (n > cap_records) n = cap_records;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        mom[2 * r] = mom[2 * r + 1] = make_float4(0.f, 0.f, 0.f, 0.f);  // 8 floats per record
        if (f64[r] & 1) {
            double2 *m2 = mom64 + (MOM64_STRIDE / 2) * r;
            m2[0] = m2[1] = m2[2] = make_double2(0.0, 0.0);
        }
    }
}

// Slice-pose shares: one thread per record, moments -> dL/d(centre, conic,
// amp) -> adjoint of the record geometry -> the record's share of dL/dT_k
// (dL/dt, dL/domega), written to its slot (FP32 geometry; DBL: only the
// records of near-degenerate Gaussians, in FP64)
template <bool DBL>
__global__ void k_pose_rec(const WsHeader *hdr, long long cap_records, const float4 *__restrict__ geo,
                           const float2 *__restrict__ geo2, const int *__restrict__ gid, const int *__restrict__ rslice,
                           const float *__restrict__ mom, const double *__restrict__ mom64,
                           const SliceDev *__restrict__ slices,
                           const float *__restrict__ mean, const float *__restrict__ quat,
                           const float *__restrict__ scale, const float *__restrict__ alpha, float f64_ratio,
                           float4 *__restrict__ rg)
{
    if (DBL && !(hdr->flags & MG_FLAG_DEGENERATE)) return;
    long long nr = (long long)hdr->n_records;
    if (nr > cap_records) nr = cap_records;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += (long long)gridDim.x * blockDim.x) {
        const long long g = gid[r];
        float sc[3] = {scale[3 * g], scale[3 * g + 1], scale[3 * g + 2]};
        float mx = fmaxf(fmaxf(sc[0], sc[1]), sc[2]), mn = fminf(fminf(sc[0], sc[1]), sc[2]);
        const bool dbl = f64_ratio > 0.f && mx > f64_ratio * mn;
        if (dbl != DBL) continue;  // the other instance handles this record
        float mu[3] = {mean[3 * g], mean[3 * g + 1], mean[3 * g + 2]};
        float qv[4] = {quat[4 * g], quat[4 * g + 1], quat[4 * g + 2], quat[4 * g + 3]};
        float al = alpha[g];
        const float4 a = geo[r];
        const float2 b = geo2[r];
        const float A = a.z, B2 = a.w, C = b.x, amp = b.y;
        const SliceDev &Sd = slices[rslice[r]];
        float o6[6];
        if (DBL) {
            // the FP64 moments of a near-degenerate Gaussian, chained in FP64
            const double *m = mom64 + (size_t)r * MOM64_STRIDE;
            const double S0 = m[0], Sx = m[1], Sy = m[2], Sxx = m[3], Sxy = m[4], Syy = m[5];
            const double A64 = m[MOM64_GEO + 2], B64 = m[MOM64_GEO + 3], C64 = m[MOM64_GEO + 4];
            const double la = (double)amp * 0.6931471805599453;
            const double gpx = -la * (2.0 * A64 * Sx + B64 * Sy);
            const double gpy = -la * (B64 * Sx + 2.0 * C64 * Sy);
            double dm[3], dq[4], ds[3], da, dp[6];
            geometry_adjoint<double, true>(mu, qv, sc, al, Sd, la * Sxx, la * Sxy, la * Syy, gpx, gpy, S0, dm, dq,
                                           ds, da, dp);
            for (int i = 0; i < 6; ++i) o6[i] = (float)dp[i];
        } else {
            const float4 m0 = *(const float4 *)(mom + (size_t)r * 8);
            const float2 m1 = *(const float2 *)(mom + (size_t)r * 8 + 4);
            const float S0 = m0.x, Sx = m0.y, Sy = m0.z, Sxx = m0.w, Sxy = m1.x, Syy = m1.y;
            const float la = amp * 0.69314718055994531f;
            const float gA = la * Sxx, gB2 = la * Sxy, gC = la * Syy;
            const float gpx = -la * (2.f * A * Sx + B2 * Sy);
            const float gpy = -la * (B2 * Sx + 2.f * C * Sy);
            float gm[3], gq[4], gs[3], ga;
            geometry_adjoint<float, true>(mu, qv, sc, al, Sd, gA, gB2, gC, gpx, gpy, S0, gm, gq, gs, ga, o6);
        }
        rg[2 * r] = make_float4(o6[0], o6[1], o6[2], 0.f);
        rg[2 * r + 1] = make_float4(o6[3], o6[4], o6[5], 0.f);
    }
}

// The chain of a near-degenerate Gaussian, out of line (rare, and inlining
// it would size every thread's registers for it): its records' FP64
// moments through the FP64 record-geometry adjoint, summed in FP64 in the
// order of the Gaussian-major list; o = dL/d(mean[3], quat[4], scale[3], alpha).
__device__ __noinline__ void chain_gaussian_f64(const float *mu, const float *q, const float *s, float alpha,
                                                unsigned long long j0, unsigned long long j1,
                                                const unsigned *__restrict__ gmap, long long cap_records,
                                                const float4 *__restrict__ geo, const float2 *__restrict__ geo2,
                                                const int *__restrict__ rslice, const double *__restrict__ mom64,
                                                const SliceDev *__restrict__ slices, float o[11])
{
    GaussFrame<double> F;
    gauss_frame<double>(q, s, F);
    double gmu[3] = {0, 0, 0}, gR[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, gs[3] = {0, 0, 0}, ga = 0;
    for (unsigned long long j = j0; j < j1; ++j) {
        const unsigned r = gmap[j];
        if ((long long)r >= cap_records) continue;
        const float2 b = geo2[r];
        const double *m = mom64 + (size_t)r * MOM64_STRIDE;
        const double A = m[MOM64_GEO + 2], B2 = m[MOM64_GEO + 3], C = m[MOM64_GEO + 4];
        const double la = (double)b.y * 0.6931471805599453;
        const double gpx = -la * (2.0 * A * m[1] + B2 * m[2]);
        const double gpy = -la * (B2 * m[1] + 2.0 * C * m[2]);
        record_adjoint<double>(F, mu, alpha, slices[rslice[r]], la * m[3], la * m[4], la * m[5], gpx, gpy, m[0], gmu,
                               gR, gs, ga);
    }
    double gq[4];
    quat_adjoint<double>(q, gR, gq);
    for (int i = 0; i < 3; ++i) o[i] = (float)gmu[i], o[7 + i] = (float)gs[i];
    for (int i = 0; i < 4; ++i) o[3 + i] = (float)gq[i];
    o[10] = (float)ga;
}

// One record's moments chained into the Gaussian's dL/d(mean, R, scale, alpha).
__device__ __forceinline__ void chain_record(const GaussFrame<float> &F, const float *mu, float al, const float4 &a,
                                             const float2 &b, const float4 &m0, const float2 &m1, const SliceDev &S,
                                             float *gmu, float (*gR)[3], float *gs, float &ga)
{
    const float A = a.z, B2 = a.w, C = b.x, amp = b.y;
    const float S0 = m0.x, Sx = m0.y, Sy = m0.z, Sxx = m0.w, Sxy = m1.x, Syy = m1.y;
    const float la = amp * 0.69314718055994531f;
    const float gpx = -la * (2.f * A * Sx + B2 * Sy);
    const float gpy = -la * (B2 * Sx + 2.f * C * Sy);
    record_adjoint<float>(F, mu, al, S, la * Sxx, la * Sxy, la * Syy, gpx, gpy, S0, gmu, gR, gs, ga);
}

// The chain of a Gaussian's records, grouped by slice frame. A record's
// conic, determinant factor and the regression of its centre on the slab
// offset depend only on the Gaussian and on the slice's frame (rotation,
// profile, spacing, PSF; the stack's slices share one unless they move), not
// on the slice's offset w0. The adjoint of record_adjoint is linear in nine
// frame-level gradients (of H = Sigma_L^-1 and of Sigma_L's uw, vw, ww entries)
// and in the offset gradients (du, dv, dw0), each record adding terms formed
// from its own w0, exp factor and moments; so a record adds those twelve
// sums, and the 3x3 part (through the frame to R and the scales) runs once per
// run of records in one frame. Same formulas as record_adjoint, summed in a
// different order.
struct ChainFrame {
    // frame constants (rotation, spacing, profile and PSF variances are read from the slice)
    float iSww, rD, iD, f, Suw, Svw, Huw, Hvw;
    float Kpuu, Kpuv, Kpvv, im, rm, K0uu, K0uv, K0vv;
    // sums over the frame's records
    float aHuu, aHuv, aHvv, aHuw, aHvw, aHww, aSuw, aSvw, aSww, adu, adv, adw;
};

__device__ __forceinline__ void chain_frame_begin(const float *qv, const float *sc, const SliceDev &S, ChainFrame &C)
{
    GaussFrame<float> F;
    gauss_frame<float>(qv, sc, F);
    float g[3][3], Lm[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float P = S.Q[a] * F.R[0][c] + S.Q[3 + a] * F.R[1][c] + S.Q[6 + a] * F.R[2][c];
            g[a][c] = P * F.isc[c];
            Lm[a][c] = P * F.sc[c];
        }
    C.Huw = g[0][0] * g[2][0] + g[0][1] * g[2][1] + g[0][2] * g[2][2];
    C.Hvw = g[1][0] * g[2][0] + g[1][1] * g[2][1] + g[1][2] * g[2][2];
    const float Hww = g[2][0] * g[2][0] + g[2][1] * g[2][1] + g[2][2] * g[2][2];
    C.Suw = Lm[0][0] * Lm[2][0] + Lm[0][1] * Lm[2][1] + Lm[0][2] * Lm[2][2];
    C.Svw = Lm[1][0] * Lm[2][0] + Lm[1][1] * Lm[2][1] + Lm[1][2] * Lm[2][2];
    const float Sww = Lm[2][0] * Lm[2][0] + Lm[2][1] * Lm[2][1] + Lm[2][2] * Lm[2][2] + S.sig2;
    C.iSww = c_rcp<float>(Sww);
    const float D = 1.f + S.sig2 * Hww;
    C.rD = c_rsqrt<float>(D);
    C.iD = C.rD * C.rD;
    C.f = S.sig2 * C.iD;
    if (S.pu2 > 0.f || S.pv2 > 0.f) {
        const float Huu = g[0][0] * g[0][0] + g[0][1] * g[0][1] + g[0][2] * g[0][2];
        const float Huv = g[0][0] * g[1][0] + g[0][1] * g[1][1] + g[0][2] * g[1][2];
        const float Hvv = g[1][0] * g[1][0] + g[1][1] * g[1][1] + g[1][2] * g[1][2];
        C.K0uu = Huu - C.f * C.Huw * C.Huw;
        C.K0uv = Huv - C.f * C.Huw * C.Hvw;
        C.K0vv = Hvv - C.f * C.Hvw * C.Hvw;
        const float pu2 = S.pu2, pv2 = S.pv2;
        const float dK = C.K0uu * C.K0vv - C.K0uv * C.K0uv;
        const float m = 1.f + pu2 * C.K0uu + pv2 * C.K0vv + pu2 * pv2 * dK;
        C.im = c_rcp<float>(m);
        C.rm = c_rsqrt<float>(m);
        C.Kpuu = (C.K0uu + pv2 * dK) * C.im;
        C.Kpuv = C.K0uv * C.im;
        C.Kpvv = (C.K0vv + pu2 * dK) * C.im;
    }
    C.aHuu = C.aHuv = C.aHvv = C.aHuw = C.aHvw = C.aHww = 0.f;
    C.aSuw = C.aSvw = C.aSww = C.adu = C.adv = C.adw = 0.f;
}

// One record's terms (its moments a, b, m0, m1 as the backward left them).
__device__ __forceinline__ void chain_frame_record(ChainFrame &C, const float *mu, float alpha, const SliceDev &S,
                                                   const float4 &a, const float2 &b, const float4 &m0,
                                                   const float2 &m1, float &galpha)
{
    const float A = a.z, B2 = a.w, Cc = b.x, ampr = b.y;
    const float S0 = m0.x, Sx = m0.y, Sy = m0.z, Sxx = m0.w, Sxy = m1.x, Syy = m1.y;
    const float la = ampr * 0.69314718055994531f;
    const float gpx = -la * (2.f * A * Sx + B2 * Sy);
    const float gpy = -la * (B2 * Sx + 2.f * Cc * Sy);
    float gamp = S0;
    const float p0 = mu[0] - S.t[0], p1 = mu[1] - S.t[1], p2 = mu[2] - S.t[2];
    const float w0 = S.Q[2] * p0 + S.Q[5] * p1 + S.Q[8] * p2;
    const float wS = w0 * C.iSww;
    const float E = c_exp<float>(-0.5f * w0 * wS);
    const float amp = alpha * C.rD * E;
    const float kap = -0.72134752044448170368f, dx = S.dx, dy = S.dy;
    float gKuu = la * Sxx * (kap * dx * dx), gKuv = la * Sxy * (2.f * kap * dx * dy), gKvv = la * Syy * (kap * dy * dy);
    const float gcu = gpx * c_rcp<float>(dx), gcv = gpy * c_rcp<float>(dy);
    const float pu2 = S.pu2, pv2 = S.pv2;
    if (pu2 > 0.f || pv2 > 0.f) {
        const float gm = -(gKuu * C.Kpuu + gKuv * C.Kpuv + gKvv * C.Kpvv) * C.im - 0.5f * gamp * amp * C.rm * C.im;
        const float gNuu = gKuu * C.im, gNuv = gKuv * C.im, gNvv = gKvv * C.im;
        const float gdK = pv2 * gNuu + pu2 * gNvv + gm * pu2 * pv2;
        gKuu = gNuu + gm * pu2 + gdK * C.K0vv;
        gKvv = gNvv + gm * pv2 + gdK * C.K0uu;
        gKuv = gNuv - 2.f * gdK * C.K0uv;
        gamp = gamp * C.rm;
    }
    galpha += gamp * C.rD * E;
    const float ga = gamp * amp;
    float gD = -0.5f * ga * C.iD;
    float gw0 = -ga * wS;
    float gSww = 0.5f * ga * wS * wS;
    const float cs = gcu * C.Suw + gcv * C.Svw;
    gw0 -= cs * C.iSww;
    gSww += cs * wS * C.iSww;
    gD += C.f * C.iD * (gKuu * C.Huw * C.Huw + gKuv * C.Huw * C.Hvw + gKvv * C.Hvw * C.Hvw);
    C.aHuu += gKuu;
    C.aHvv += gKvv;
    C.aHuv += gKuv;
    C.aHuw += -C.f * (2.f * gKuu * C.Huw + gKuv * C.Hvw);
    C.aHvw += -C.f * (2.f * gKvv * C.Hvw + gKuv * C.Huw);
    C.aHww += S.sig2 * gD;
    C.aSuw += -gcu * wS;
    C.aSvw += -gcv * wS;
    C.aSww += gSww;
    C.adu += gcu;
    C.adv += gcv;
    C.adw += gw0;
}

// The frame's sums through Sigma_L = P diag(s^2) P^T and H = g g^T (P = Q^T R)
// to R and the scales, and the offsets to the mean: added to gmu, gR, gs.
__device__ __forceinline__ void chain_frame_end(const float *qv, const float *sc, const ChainFrame &C,
                                                const float *Q, float gmu[3], float gR[3][3], float gs[3])
{
    GaussFrame<float> F;
    gauss_frame<float>(qv, sc, F);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float P[3], g[3], Lm[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            P[a] = Q[a] * F.R[0][c] + Q[3 + a] * F.R[1][c] + Q[6 + a] * F.R[2][c];
            g[a] = P[a] * F.isc[c];
            Lm[a] = P[a] * F.sc[c];
        }
        const float gg0 = 2.f * C.aHuu * g[0] + C.aHuv * g[1] + C.aHuw * g[2];
        const float gg1 = 2.f * C.aHvv * g[1] + C.aHuv * g[0] + C.aHvw * g[2];
        const float gg2 = 2.f * C.aHww * g[2] + C.aHuw * g[0] + C.aHvw * g[1];
        const float gL0 = C.aSuw * Lm[2];
        const float gL1 = C.aSvw * Lm[2];
        const float gL2 = C.aSuw * Lm[0] + C.aSvw * Lm[1] + 2.f * C.aSww * Lm[2];
        const float gP0 = gg0 * F.isc[c] + gL0 * F.sc[c];
        const float gP1 = gg1 * F.isc[c] + gL1 * F.sc[c];
        const float gP2 = gg2 * F.isc[c] + gL2 * F.sc[c];
        gs[c] += -(gg0 * g[0] + gg1 * g[1] + gg2 * g[2]) * F.isc[c] + (gL0 * P[0] + gL1 * P[1] + gL2 * P[2]);
#pragma unroll
        for (int r = 0; r < 3; ++r) gR[r][c] += Q[3 * r] * gP0 + Q[3 * r + 1] * gP1 + Q[3 * r + 2] * gP2;
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) gmu[r] += Q[3 * r] * C.adu + Q[3 * r + 1] * C.adv + Q[3 * r + 2] * C.adw;
}

// The Gaussian's gradients; the quaternion's on the unit sphere: its component
// along q dropped (the normalisation q = q_raw/|q_raw| removes it, and the
// rotation formula is only a rotation for unit q).
__device__ __forceinline__ void write_gaussian_grads(long long g, const float *o, const float *qv, float *g_mean,
                                                     float *g_quat, float *g_scale, float *g_alpha)
{
    const float qq = qv[0] * qv[0] + qv[1] * qv[1] + qv[2] * qv[2] + qv[3] * qv[3];
    const float rad = qq > 0.f ? (o[3] * qv[0] + o[4] * qv[1] + o[5] * qv[2] + o[6] * qv[3]) / qq : 0.f;
    g_mean[3 * g] = o[0];
    g_mean[3 * g + 1] = o[1];
    g_mean[3 * g + 2] = o[2];
    for (int i = 0; i < 4; ++i) g_quat[4 * g + i] = o[3 + i] - rad * qv[i];
    g_scale[3 * g] = o[7];
    g_scale[3 * g + 1] = o[8];
    g_scale[3 * g + 2] = o[9];
    g_alpha[g] = o[10];
}

// K6 fused: one thread per Gaussian visits its records in slice order (the
// Gaussian-major list), turns each record's moments into dL/d(centre, conic,
// amplitude) and chains them through the record geometry (FP64 for
// near-degenerate Gaussians), summing in that fixed order; the records add to
// dL/d(mean, R, scale, alpha), and dL/dq follows from dL/dR once. The warp
// walks the stacks together: in a stack whose slices share one rotation (no
// motion) a record only adds its terms to the frame sums (ChainFrame) and the
// 3x3 part runs once per (Gaussian, stack); in a moving stack every record is
// chained whole. Walking the stacks in step keeps the lanes' frame set-ups
// aligned (per-lane frame changes would run the set-up divergently on almost
// every record). The next record's data is loaded while the current one is
// chained. A Gaussian with more than 64 records (a fitted model grows a few
// that span many slices) is summed by its whole warp instead, record by record,
// lane l taking records l, l + 32, ..., then a fixed shuffle tree: one thread
// would hold the warp for all of them. Nothing per record is written.
constexpr unsigned CHAIN_WARP_RECORDS = 64;

__global__ void __launch_bounds__(128, 4) k_chain_fused(StackTable tab, const WsHeader *__restrict__ hdr, long long n,
                                                     const unsigned *__restrict__ goff,
                                                     const unsigned *__restrict__ gmap, long long cap_records,
                                                     const float4 *__restrict__ geo, const float2 *__restrict__ geo2,
                                                     const int *__restrict__ rslice, const float *__restrict__ mom,
                                                     const double *__restrict__ mom64,
                                                     const SliceDev *__restrict__ slices,
                                                     const float *__restrict__ mean, const float *__restrict__ quat,
                                                     const float *__restrict__ scale, const float *__restrict__ alpha,
                                                     float f64_ratio, float *g_mean, float *g_quat, float *g_scale,
                                                     float *g_alpha)
{
    pdl_entry();
    const int lane = threadIdx.x & 31;
    const unsigned moving = hdr->moving;  // bit s: the slices of stack s do not share one rotation
    for (long long gb = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); gb < n;
         gb += (long long)gridDim.x * blockDim.x) {
        const long long g = gb + lane;
        const bool valid = g < n;
        const long long gl = valid ? g : gb;  // lanes past n read a valid Gaussian and write nothing
        unsigned long long j0 = goff[gl], j1 = goff[gl + 1];
        if ((long long)j1 > cap_records) j1 = cap_records;
        if (j0 > j1) j0 = j1;
        float sc[3] = {scale[3 * gl], scale[3 * gl + 1], scale[3 * gl + 2]};
        float mu[3] = {mean[3 * gl], mean[3 * gl + 1], mean[3 * gl + 2]};
        float qv[4] = {quat[4 * gl], quat[4 * gl + 1], quat[4 * gl + 2], quat[4 * gl + 3]};
        const float al = alpha[gl];
        const float mx = fmaxf(fmaxf(sc[0], sc[1]), sc[2]), mn = fminf(fminf(sc[0], sc[1]), sc[2]);
        const bool dbl = f64_ratio > 0.f && mx > f64_ratio * mn;
        const bool many = valid && !dbl && j1 - j0 > CHAIN_WARP_RECORDS;
        if (valid && !many) {
            float o[11];
            if (dbl) {
                chain_gaussian_f64(mu, qv, sc, al, j0, j1, gmap, cap_records, geo, geo2, rslice, mom64, slices, o);
            } else {
                float gmu[3] = {0.f, 0.f, 0.f}, gR[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
                float gs[3] = {0.f, 0.f, 0.f}, ga = 0.f;
                // record ids are loaded two records ahead, their data one record
                // ahead (an id past the capacity reads as slice 0 and is skipped)
                unsigned nr = j0 < j1 ? gmap[j0] : 0xffffffffu;
                unsigned nr2 = j0 + 1 < j1 ? gmap[j0 + 1] : 0xffffffffu;
                float4 na = make_float4(0.f, 0.f, 0.f, 0.f), nm0 = na;
                float2 nb = make_float2(0.f, 0.f), nm1 = nb;
                int ns = 0;
                if ((long long)nr < cap_records) {
                    na = geo[nr];
                    nb = geo2[nr];
                    nm0 = *(const float4 *)(mom + (size_t)nr * 8);
                    nm1 = *(const float2 *)(mom + (size_t)nr * 8 + 4);
                    ns = rslice[nr];
                }
                unsigned long long j = j0;
                auto advance = [&](unsigned &r, float4 &a, float2 &b, float4 &m0, float2 &m1, int &sl) {
                    r = nr;
                    a = na;
                    m0 = nm0;
                    b = nb;
                    m1 = nm1;
                    sl = ns;
                    nr = nr2;
                    nr2 = j + 2 < j1 ? gmap[j + 2] : 0xffffffffu;
                    ns = 0;
                    if ((long long)nr < cap_records) {
                        na = geo[nr];
                        nb = geo2[nr];
                        nm0 = *(const float4 *)(mom + (size_t)nr * 8);
                        nm1 = *(const float2 *)(mom + (size_t)nr * 8 + 4);
                        ns = rslice[nr];
                    }
                    ++j;
                };
                // stack by stack (the records are in slice order), the same
                // stack for every lane of the warp at a time
                for (int s = 0; s < tab.n_stacks; ++s) {
                    const int sb = tab.slice_base[s], se = tab.slice_base[s + 1];
                    const bool has = j < j1 && ns < se;
                    if (!(moving >> s & 1u)) {
                        // one rotation for the whole stack: one frame
                        ChainFrame C;
                        if (has) chain_frame_begin(qv, sc, slices[sb], C);
                        while (j < j1 && ns < se) {
                            unsigned r;
                            float4 a, m0;
                            float2 b, m1;
                            int sl;
                            advance(r, a, b, m0, m1, sl);
                            if ((long long)r < cap_records) chain_frame_record(C, mu, al, slices[sl], a, b, m0, m1, ga);
                        }
                        if (has) chain_frame_end(qv, sc, C, slices[sb].Q, gmu, gR, gs);
                    } else if (has) {
                        GaussFrame<float> F;
                        gauss_frame<float>(qv, sc, F);
                        while (j < j1 && ns < se) {
                            unsigned r;
                            float4 a, m0;
                            float2 b, m1;
                            int sl;
                            advance(r, a, b, m0, m1, sl);
                            if ((long long)r < cap_records) chain_record(F, mu, al, a, b, m0, m1, slices[sl], gmu, gR, gs, ga);
                        }
                    }
                }
                float gq[4];
                quat_adjoint<float>(qv, gR, gq);
                for (int i = 0; i < 3; ++i) o[i] = gmu[i], o[7 + i] = gs[i];
                for (int i = 0; i < 4; ++i) o[3 + i] = gq[i];
                o[10] = ga;
            }
            write_gaussian_grads(g, o, qv, g_mean, g_quat, g_scale, g_alpha);
        }
        // the warp's Gaussians with many records, one at a time
        unsigned lm = __ballot_sync(0xffffffffu, many);
        while (lm) {
            const int src = __ffs(lm) - 1;
            lm &= lm - 1;
            const long long gg = gb + src;
            const unsigned long long k0 = __shfl_sync(0xffffffffu, j0, src), k1 = __shfl_sync(0xffffffffu, j1, src);
            const float sg[3] = {scale[3 * gg], scale[3 * gg + 1], scale[3 * gg + 2]};
            const float mg[3] = {mean[3 * gg], mean[3 * gg + 1], mean[3 * gg + 2]};
            const float qg[4] = {quat[4 * gg], quat[4 * gg + 1], quat[4 * gg + 2], quat[4 * gg + 3]};
            const float ag = alpha[gg];
            GaussFrame<float> F;
            gauss_frame<float>(qg, sg, F);
            float acc[16];  // dL/d mean (3), R (9), scale (3), alpha
            for (int i = 0; i < 16; ++i) acc[i] = 0.f;
            for (unsigned long long j = k0 + lane; j < k1; j += 32) {
                const unsigned r = gmap[j];
                if ((long long)r >= cap_records) continue;
                const float4 a = geo[r], m0 = *(const float4 *)(mom + (size_t)r * 8);
                const float2 b = geo2[r], m1 = *(const float2 *)(mom + (size_t)r * 8 + 4);
                chain_record(F, mg, ag, a, b, m0, m1, slices[rslice[r]], acc, (float(*)[3])(acc + 3), acc + 12,
                             acc[15]);
            }
#pragma unroll
            for (int i = 0; i < 16; ++i)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
            if (lane == src) {
                float gq[4], o[11];
                quat_adjoint<float>(qg, (float(*)[3])(acc + 3), gq);
                for (int i = 0; i < 3; ++i) o[i] = acc[i], o[7 + i] = acc[12 + i];
                for (int i = 0; i < 4; ++i) o[3 + i] = gq[i];
                o[10] = acc[15];
                write_gaussian_grads(gg, o, qg, g_mean, g_quat, g_scale, g_alpha);
            }
        }
    }
}

// K6c: one block per slice sums its records' pose shares (records of a slice
// are contiguous) in a fixed order, in FP64
__global__ void __launch_bounds__(256) k_pose_sum(int S, const unsigned *__restrict__ slice_rs,
                                                  const float4 *__restrict__ rg, float *__restrict__ g_pose)
{
    __shared__ double red[6][8];
    const int k = blockIdx.x;
    if (k >= S) return;
    const unsigned r0 = slice_rs[k], r1 = slice_rs[k + 1];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (unsigned r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        const float4 a = rg[2 * (size_t)r], b = rg[2 * (size_t)r + 1];
        acc[0] += a.x, acc[1] += a.y, acc[2] += a.z;
        acc[3] += b.x, acc[4] += b.y, acc[5] += b.z;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double v = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[i][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = 0.0;
        for (int j = 0; j < 8; ++j) v += red[threadIdx.x][j];
        g_pose[6 * (size_t)k + threadIdx.x] = (float)v;
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

static int resident_grid(const void *kern, int threads)
{
    int dev = 0, sms = 148, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, 0);
    return sms * (per > 0 ? per : 1);
}

// The per-tile loss partials summed in two fixed-order levels (FP64): block
// b adds the tiles of its contiguous range (thread i: tiles i, i + 256, ...
// of the range, then a fixed shuffle tree), one block adds the block sums
// in order; the same bits on every run.
constexpr int LT_NT = 256;

__device__ __forceinline__ void lt_block_sum(double &s1, double &s2, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[threadIdx.x >> 5] = s1;
        sh[LT_NT / 32 + (threadIdx.x >> 5)] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        s1 = s2 = 0.0;
        for (int k = 0; k < LT_NT / 32; ++k) s1 += sh[k], s2 += sh[LT_NT / 32 + k];
    }
}

// The per-tile loss partials in two fixed-order FP64 levels, one launch: each
// block sums its range of tiles, and the block that finishes last (a ticket
// counter, no waiting) sums the block sums in block order and writes the loss.
__global__ void __launch_bounds__(LT_NT) k_loss_tiles(const double2 *__restrict__ part, long long n, long long per,
                                                      double2 *__restrict__ bsum, unsigned *ticket, double inv_n,
                                                      double *__restrict__ out)
{
    pdl_entry();
    __shared__ double sh[2 * LT_NT / 32];
    __shared__ bool last;
    const long long i0 = (long long)blockIdx.x * per, i1 = min(n, i0 + per);
    double s1 = 0.0, s2 = 0.0;
    for (long long i = i0 + threadIdx.x; i < i1; i += LT_NT) {
        const double2 p = part[i];
        s1 += p.x;
        s2 += p.y;
    }
    lt_block_sum(s1, s2, sh);
    if (threadIdx.x == 0) {
        bsum[blockIdx.x] = make_double2(s1, s2);
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    s1 = 0.0;
    s2 = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += LT_NT) {
        const double2 b = __ldcg(&bsum[i]);
        s1 += b.x;
        s2 += b.y;
    }
    lt_block_sum(s1, s2, sh);
    if (threadIdx.x == 0) {
        out[0] = s1 * inv_n + s2 * inv_n;
        out[1] = s2;
        *ticket = 0u;  // ready for the next launch
    }
}

template <bool CELLS, bool LOSS>
static void launch_fwd(const WsLayout &L, char *ws, const StackTable &tab, const SliceDev *slices, const CellGrid &cg,
                       float *out, const FwdLoss &ls, cudaStream_t st)
{
    WsHeader *hdr = (WsHeader *)(ws + L.hdr);
    int grid = resident_grid((const void *)k_render_fwd<CELLS, LOSS>, 32 * RW);
    const int nt = tab.n_tiles_total;
    if (grid > (nt + RW - 1) / RW) grid = (nt + RW - 1) / RW;
    launch_pdl(k_render_fwd<CELLS, LOSS>, dim3(grid), dim3(32 * RW), 0,
        st, tab, (const unsigned *)(ws + L.tile_off), (const unsigned *)(ws + L.entries), L.cap_entries, L.cap_records,
        (const float4 *)(ws + L.rec_geo), (const float2 *)(ws + L.rec_geo2), slices, cg,
        cg.on ? (const int4 *)(ws + L.rec_cell) : nullptr, (const unsigned *)(ws + L.tile_list),
        (const unsigned *)(ws + L.dense_list), (const unsigned *)(ws + L.sparse_list), hdr,
        (const unsigned char *)(ws + L.rec_f64), (const double *)(ws + L.rec_mom64), out, ls, &hdr->tile_ctr[0],
        &hdr->fwd_sparse_ctr);
}

// target != NULL: the L1 + L2 slice loss of mg_loss_l1l2 fused into the
// forward (grad may be NULL), loss_out = {loss, sum r^2} (device doubles)
void mg_launch_render_fwd(const WsLayout &L, char *ws, const StackTable &tab, const SliceDev *slices,
                          const CellGrid &cg, float *out, cudaStream_t st, const float *target, float *grad,
                          double *loss_out, long long n_vox)
{
    int nt = tab.n_tiles_total;
    if (nt <= 0) return;
    WsHeader *hdr = (WsHeader *)(ws + L.hdr);
    // the work counters (tile_ctr) start at zero: the bin pass that precedes
    // every forward clears the workspace header
    FwdLoss ls;
    ls.target = target;
    ls.grad = grad;
    ls.tile_part = (double2 *)(ws + L.tile_loss);
    ls.inv_n = n_vox > 0 ? (float)(1.0 / (double)n_vox) : 0.f;
    {
        MG_PROF(MG_ST_RENDER_FWD, st);
        if (target) {
            if (cg.on)
                launch_fwd<true, true>(L, ws, tab, slices, cg, out, ls, st);
            else
                launch_fwd<false, true>(L, ws, tab, slices, cg, out, ls, st);
        } else {
            if (cg.on)
                launch_fwd<true, false>(L, ws, tab, slices, cg, out, ls, st);
            else
                launch_fwd<false, false>(L, ws, tab, slices, cg, out, ls, st);
        }
    }
    if (target) {
        MG_PROF(MG_ST_LOSS, st);
        // block sums after the tile partials (the workspace slot holds both)
        const long long per = 8 * LT_NT;
        const int nb = (int)((nt + per - 1) / per);
        double2 *bsum = ls.tile_part + nt;
        launch_pdl(k_loss_tiles, dim3(nb), dim3(LT_NT), 0, st, ls.tile_part, nt, per, bsum, &hdr->tile_ctr[3],
                                           n_vox > 0 ? 1.0 / (double)n_vox : 0.0, loss_out);
    }
}

// Slice-pose gradient from the moments the last backward left in the workspace.
void mg_launch_pose_grad(const WsLayout &L, char *ws, const SliceDev *slices, const float *mean, const float *quat,
                         const float *scale, const float *alpha, float f64_ratio, float *g_pose, cudaStream_t st)
{
    const WsHeader *hdr = (const WsHeader *)(ws + L.hdr);
    MG_PROF(MG_ST_CHAIN, st);
    float4 *rg = (float4 *)(ws + L.rec_grad);
    long long wr = (L.cap_records + 255) / 256;
    int gr = (int)(wr < 148 * 16 ? (wr > 0 ? wr : 1) : 148 * 16);
    k_pose_rec<false><<<gr, 256, 0, st>>>(hdr, L.cap_records, (const float4 *)(ws + L.rec_geo),
                                                 (const float2 *)(ws + L.rec_geo2), (const int *)(ws + L.rec_gid),
                                                 (const int *)(ws + L.rec_slice), (const float *)(ws + L.rec_mom),
                                                 (const double *)(ws + L.rec_mom64),
                                                 slices, mean, quat, scale, alpha, f64_ratio, rg);
    if (f64_ratio > 0.f)
        k_pose_rec<true><<<gr, 256, 0, st>>>(hdr, L.cap_records, (const float4 *)(ws + L.rec_geo),
                                                    (const float2 *)(ws + L.rec_geo2), (const int *)(ws + L.rec_gid),
                                                    (const int *)(ws + L.rec_slice), (const float *)(ws + L.rec_mom),
                                                 (const double *)(ws + L.rec_mom64),
                                                    slices, mean, quat, scale, alpha, f64_ratio, rg);
    const unsigned *slice_rs = (const unsigned *)(ws + L.chunk_base) + (L.S + 1);
    k_pose_sum<<<(unsigned)L.S, 256, 0, st>>>((int)L.S, slice_rs, rg, g_pose);
}

void mg_launch_render_bwd(const WsLayout &L, char *ws, const SliceDev *slices, const StackTable &tab,
                          const CellGrid &cg, const float *grad_out, const float *mean, const float *quat,
                          const float *scale, const float *alpha, long long n, float f64_ratio, float *g_mean,
                          float *g_quat, float *g_scale, float *g_alpha, bool zero_moments, cudaStream_t st)
{
    const WsHeader *hdr = (const WsHeader *)(ws + L.hdr);
    if (zero_moments) {
        // the record pass zeroes the moments; a second backward on the same forward clears them again
        long long capv = L.cap_records * 2;
        int gz = (int)((capv + 255) / 256 < 148 * 16 ? (capv + 255) / 256 : 148 * 16);
        if (gz < 1) gz = 1;
        MG_PROF(MG_ST_ZERO, st);
        launch_pdl(k_zero_mom, dim3(gz), dim3(256), 0, st,
            (float4 *)(ws + L.rec_mom), (const unsigned char *)(ws + L.rec_f64),
                                       (double2 *)(ws + L.rec_mom64), hdr, L.cap_records);
    }
    int nt = tab.n_tiles_total;
    if (nt > 0) {
        // the backward's work counters: tile_ctr[1] and [4] (dense tiles) and
        // tile_ctr[2] (sparse tiles; the forward's counters [2] and [3] are
        // spent by now)
        cudaMemsetAsync((void *)&hdr->tile_ctr[1], 0, 4 * sizeof(unsigned), st);
        MG_PROF(MG_ST_RENDER_BWD, st);
        const void *kern = cg.on ? (const void *)k_render_bwd<true> : (const void *)k_render_bwd<false>;
        int grid = resident_grid(kern, 32 * RW);
        if (grid > (nt + RW - 1) / RW) grid = (nt + RW - 1) / RW;
        const int4 *rcell = cg.on ? (const int4 *)(ws + L.rec_cell) : nullptr;
        if (cg.on)
            launch_pdl(k_render_bwd<true>, dim3(grid), dim3(32 * RW), 0, st,
                tab, (const unsigned *)(ws + L.tile_off), (const unsigned *)(ws + L.entries), L.cap_entries,
                L.cap_records, (const float4 *)(ws + L.rec_geo), (const float2 *)(ws + L.rec_geo2), slices, cg, rcell,
                (const unsigned *)(ws + L.dense_list), (const unsigned *)(ws + L.sparse_list), hdr,
                (const unsigned char *)(ws + L.rec_f64), grad_out, (float *)(ws + L.rec_mom),
                (double *)(ws + L.rec_mom64), (unsigned *)&hdr->tile_ctr[1]);
        else
            launch_pdl(k_render_bwd<false>, dim3(grid), dim3(32 * RW), 0, st,
                tab, (const unsigned *)(ws + L.tile_off), (const unsigned *)(ws + L.entries), L.cap_entries,
                L.cap_records, (const float4 *)(ws + L.rec_geo), (const float2 *)(ws + L.rec_geo2), slices, cg, rcell,
                (const unsigned *)(ws + L.dense_list), (const unsigned *)(ws + L.sparse_list), hdr,
                (const unsigned char *)(ws + L.rec_f64), grad_out, (float *)(ws + L.rec_mom),
                (double *)(ws + L.rec_mom64), (unsigned *)&hdr->tile_ctr[1]);
    }
    MG_PROF(MG_ST_CHAIN, st);
    long long wg = (n + 127) / 128;
    int gc = (int)(wg < 148 * 32 ? (wg > 0 ? wg : 1) : 148 * 32);
    launch_pdl(k_chain_fused, dim3(gc), dim3(128), 0, st,
        tab, hdr, n, (const unsigned *)(ws + L.gcnt), (const unsigned *)(ws + L.gmap),
                                      L.cap_records, (const float4 *)(ws + L.rec_geo),
                                      (const float2 *)(ws + L.rec_geo2), (const int *)(ws + L.rec_slice),
                                      (const float *)(ws + L.rec_mom), (const double *)(ws + L.rec_mom64), slices,
                                      mean, quat, scale, alpha, f64_ratio,
                                      g_mean, g_quat, g_scale, g_alpha);
}
