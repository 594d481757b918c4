// mg_internal.cuh -- device-side data layout shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "mgauss.h"

#define MG_TILE MG_TILE_EDGE    // tile edge in pixels (record rectangles are in tiles)
#define MG_MAX_STACKS 32
#define MG_MAX_TILES_SLICE 16384 // 1024 x 1024 pixels
#define MG_CHUNK 512           // records per binning chunk (one warp each)
#define MG_SCAN_BLOCKS 256     // blocks of the two-phase scan

// device status flags (workspace header)
#define MG_FLAG_CAP_RECORDS 1u
#define MG_FLAG_CAP_ENTRIES 2u
#define MG_FLAG_CAP_CHUNKS 4u
#define MG_FLAG_NOT_FINITE 8u
#define MG_FLAG_DEGENERATE 16u  // some Gaussian takes the FP64 geometry

// One slice as the kernels see it (built on the device from the stacks).
struct SliceDev {
    float Q[9];  // rotation, row-major (columns e_u, e_v, e_n)
    float t[3];
    float sig2;  // FP32 profile variance (record predicate)
    float ent;   // e_n . t in FP32 (record predicate: w0 = e_n . mu - e_n . t)
    float pu2, pv2;  // FP32 in-plane PSF variances along e_u, e_v (0: none)
    float dx, dy, hx, hy;  // spacing, 0.5*(W-1), 0.5*(H-1)
    float idx, idy;        // 1/dx, 1/dy rounded once (FP32 division)
    int W, H, TX, TY;
    int tile_base;  // global index of tile (0,0)
    int stack;
    int same_frame;  // 1: rotation and profile bitwise equal to the previous slice's
    int pad[2];
    long long pix_base;  // offset of pixel (0,0) in the output
};
// Kernels gather one field of 32 different slices per warp (and stage slices
// in shared memory one per thread): a size that is a multiple of 128 bytes
// would put every lane's word in the same bank.
static_assert(sizeof(SliceDev) % 128 != 0, "the slice table's stride must not be a multiple of 128 bytes");

// Per-stack table passed by value: maps a global tile to its slice.
struct StackTable {
    int n_stacks;
    int n_slices_total;
    int n_tiles_total;
    int max_tiles_slice;
    int tile_base[MG_MAX_STACKS + 1];
    int slice_base[MG_MAX_STACKS + 1];
    int TX[MG_MAX_STACKS], TY[MG_MAX_STACKS], W[MG_MAX_STACKS], H[MG_MAX_STACKS];
    long long pix_base[MG_MAX_STACKS + 1];
};

// Input for the slice-table builder.
struct StackIn {
    int n_stacks;
    int n_slices[MG_MAX_STACKS];
    int H[MG_MAX_STACKS], W[MG_MAX_STACKS];
    float dx[MG_MAX_STACKS], dy[MG_MAX_STACKS], sig2[MG_MAX_STACKS];
    float pu2[MG_MAX_STACKS], pv2[MG_MAX_STACKS];
    const float *xform[MG_MAX_STACKS];
    // volume-plane mode (inference sampling): one stack of G z-planes built
    // from centre / spacing instead of xform
    int planes;
    float cx, cy, cz, h;
};

// The paper's cell-grid local set (MG_LOCAL_CELLS), as the kernels see it.
struct CellGrid {
    int on;       // 0: the K-sigma local set
    int R;        // block radius (cells)
    float hres;   // 0.5 * grid_res
    float h;      // half edge of the normalised cube (mm)
    float C[3];   // its centre (mm)
    float e;      // half-width of a Gaussian's member box (mm)
    float m;      // margin of the record and pixel-box tests (mm)
};

// cell index of one coordinate (mgauss.h, MG_LOCAL_CELLS)
__device__ __forceinline__ int cell_coord(float p, float c, float h, float hres)
{
    float t = __fmul_rn(__fadd_rn(__fdiv_rn(__fsub_rn(p, c), h), 1.0f), hres);
    t = fminf(fmaxf(t, -1048576.0f), 1048576.0f);
    return (int)floorf(t);
}

// cell of voxel (i, j) of a slice (mgauss.h, MG_LOCAL_CELLS)
__device__ __forceinline__ void voxel_cell(const SliceDev &S, int i, int j, const CellGrid &cg, int c[3])
{
    const float u = __fmul_rn(__fsub_rn((float)i, S.hx), S.dx);
    const float v = __fmul_rn(__fsub_rn((float)j, S.hy), S.dy);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float x = __fadd_rn(__fadd_rn(__fmul_rn(S.Q[3 * a], u), __fmul_rn(S.Q[3 * a + 1], v)), S.t[a]);
        c[a] = cell_coord(x, cg.C[a], cg.h, cg.hres);
    }
}

// Tile-relative member test of MG_LOCAL_CELLS: voxel cells are packed as
// bytes (x | y << 8 | z << 16) relative to the tile's smallest cell; a
// record's member range [lo, hi] per axis is packed the same way. Returns
// false when no voxel of the tile can be a member.
__device__ __forceinline__ bool cell_range(int4 c, int R, int b0, int b1, int b2, unsigned &lo, unsigned &hi)
{
    const int l0 = c.x - R - b0, l1 = c.y - R - b1, l2 = c.z - R - b2;
    const int h0 = c.x + R - b0, h1 = c.y + R - b1, h2 = c.z + R - b2;
    if (h0 < 0 || h1 < 0 || h2 < 0 || l0 > 255 || l1 > 255 || l2 > 255) {
        lo = 0xffffffu;
        hi = 0u;
        return false;
    }
    lo = (unsigned)max(l0, 0) | ((unsigned)max(l1, 0) << 8) | ((unsigned)max(l2, 0) << 16);
    hi = (unsigned)min(h0, 255) | ((unsigned)min(h1, 255) << 8) | ((unsigned)min(h2, 255) << 16);
    return true;
}
__device__ __forceinline__ bool cell_member(unsigned rel, unsigned lo, unsigned hi)
{
    return (__vsubus4(lo, rel) | __vsubus4(rel, hi)) == 0u;
}

// Workspace header (device memory, first 256 bytes of the workspace).
struct WsHeader {
    unsigned int flags;
    unsigned int pad0;
    unsigned long long n_records;  // exact total (may exceed capacity)
    unsigned long long n_entries;
    unsigned long long n_chunks;
    unsigned long long scan_total;
    unsigned long long pairs_inside;     // mg_render_pair_count
    unsigned long long pairs_evaluated;
    unsigned int tile_ctr[6];  // work counters: [0] forward busy tiles (bulk), [1] backward dense tiles
                               // (bulk), [2] forward empty tiles, then backward sparse tiles, [3] loss
                               // ticket, [4] backward dense tiles (reserve), [5] forward busy tiles (reserve)
    unsigned int pad2;
    unsigned int n_idle;       // tiles without records (back of the tile list)
    unsigned long long n_big;  // records listed apart from their chunks (large records)
    unsigned int moving;       // bit s: stack s has slices of different rotations (set by k1_emit)
    unsigned int fwd_sparse_ctr;  // forward work counter over the sparse tiles
    unsigned int n_dense;      // tiles with more than SPARSE_MAX records (dense list)
    unsigned int n_sparse;     // tiles with 1..SPARSE_MAX records (sparse list)
    unsigned long long reserved[18];
};

static_assert(sizeof(WsHeader) == 256, "the workspace header is 256 bytes");

// Persistent render warps take the busy tiles in two parts: the bulk of the
// list in claims of TILE_CLAIM consecutive tiles (half the claims; neighbours
// share records, which then hit L1; a fitted model's many light tiles gain
// most: its step 1.52 -> 1.38 ms), and the last TILE_RESERVE tiles per
// resident warp one at a time from a second counter, so that the kernel's
// tail is one tile.
constexpr unsigned TILE_CLAIM = 2;
constexpr unsigned TILE_RESERVE = 2;

// Records are stored as structure-of-arrays.
// a record's listed tiles: the tile rectangle (tx0, ty0, tx1, ty1) and, per
// tile row (first 8), the tile-column insets, left (low nibble) and right
struct __align__(16) RecTiles {
    ushort4 rect;
    unsigned long long inset;
};

struct Records {
    float4 *geo;        // (pcx, pcy, A, B2): centre in pixels, conic (log2 units)
    float2 *geo2;       // (C, amp)
    int *gid;           // Gaussian id
    int *slice;         // global slice id
    RecTiles *tiles;    // listed tiles
    float *mom;         // [cap][8] backward moments (6 used)
    float *thr;         // q threshold of the K-sigma ellipsoid (log2 units), for pair counts
    int4 *cell;         // MG_LOCAL_CELLS: the Gaussian's cell (x, y, z, 0); else unused
    unsigned char *f64; // bit 0: near-degenerate Gaussian (FP64 geometry and FP64 moments);
                        // bit 1: scale ratio above ELONG_RATIO (the backward's centre-out sums)
    double *mom64;      // [cap][12] of the FP64 records: [0..5] backward moments (FP64
                        // accumulation), [6..10] FP64 geometry (pcx, pcy, A, B2, C)
    long long cap;
};

// Workspace layout, computed identically on the host for fwd, bwd and the
// size query.
struct WsLayout {
    size_t hdr, slices, cnt, scan_part, rec_geo, rec_geo2, rec_gid, rec_slice, rec_rect, rec_inset, rec_mom, rec_thr;
    size_t chunk_base, hist, tile_cnt, tile_off, tile_list, tile_loss, entries, gcnt, bits, gmap, rec_grad, rec_cell, rec_f64,
        rec_mom64, big_n, big_list, tile_small, tile_big, dense_list, sparse_list, total;
    long long S, NB, NW, SW, cap_records, cap_entries, cap_chunks, n_tiles, max_tiles;
};

// -------------------------------------------------------------------------
// small device helpers
// -------------------------------------------------------------------------
// The backward takes the tiles with more than SPARSE_MAX records (the dense
// list) with two-tile claims, then the others (the sparse list, a fitted
// model's background) SPARSE_CLAIM at a time, their records packed into
// batches of up to 32 lanes, each lane over all rows of its own tile.
constexpr unsigned SPARSE_MAX = 16;
// Gaussians with a scale ratio above ELONG_RATIO (flag bit 1 of a record) take
// the backward's cancellation-free moment sums. With the default FP64
// threshold (a ratio of 16) the same records also take the FP64 path; the
// flag matters where a caller raises that threshold.
constexpr float ELONG_RATIO = 16.f;
constexpr unsigned SPARSE_CLAIM = 8;

// Binning of large records: a record listing more than BIG_AREA tiles is
// listed apart from its chunk (up to BIG_MAX per chunk, in record order) and
// placed after the tile's other entries by one thread per tile, so that a
// chunk holding a few records that span whole slices does not hold its warp.
constexpr int BIG_AREA = 16;
constexpr int BIG_MAX = 64;

// FP64 slots of a near-degenerate record: moments, then its FP64 geometry
constexpr int MOM64_STRIDE = 12;
constexpr int MOM64_GEO = 6;

// Programmatic dependent launch between the kernels of a step: a kernel
// launched through launch_pdl is set up while its predecessor's last blocks
// finish (no explicit trigger: the predecessor's blocks release it as they
// exit), which hides the launch gap. It starts with pdl_entry(): wait until
// the predecessor grid has completed and its writes are visible, before any
// other statement (early returns included), so that completion stays
// transitive along the stream. Where the preceding stream operation is not a
// kernel the wait returns at once. (Triggering the successor at the start of
// every kernel was slower: its waiting blocks took SM slots from the tail.)
__device__ __forceinline__ void pdl_entry()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... KArgs, typename... Args>
static inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                     Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// per-stage CUDA-event timing (mg_profile_*); no-ops unless enabled
enum MgStage {
    MG_ST_SLICES = 0,
    MG_ST_K1_COUNT,
    MG_ST_SCAN_REC,
    MG_ST_K1_EMIT,
    MG_ST_CHUNKS,
    MG_ST_BIN_HIST,
    MG_ST_BIN_COLSCAN,
    MG_ST_SCAN_TILES,
    MG_ST_BIN_SCATTER,
    MG_ST_RENDER_FWD,
    MG_ST_ZERO,
    MG_ST_RENDER_BWD,
    MG_ST_CHAIN,
    MG_ST_LOSS,
    MG_ST_PAIRS,
    MG_ST_NRF_FWD,
    MG_ST_NRF_BWD,
    MG_ST_REC_GEOM,
    MG_ST_REC_FILL,
    MG_NSTAGES
};
void mg_prof_begin(int stage, cudaStream_t st);
void mg_prof_end(int stage, cudaStream_t st);
struct MgProfScope {
    int s;
    cudaStream_t st;
    MgProfScope(int stage, cudaStream_t stream) : s(stage), st(stream) { mg_prof_begin(s, st); }
    ~MgProfScope() { mg_prof_end(s, st); }
};
#define MG_PROF(stage, stream) MgProfScope mg_prof_scope_##stage(stage, stream)

// host-side launch helpers (defined in the .cu files)
int64_t mg_nrf_param_count_impl(int32_t encoding);
size_t mg_nrf_enc_bytes_impl(const mg_nrf *net, long long n);
cudaError_t mg_launch_nrf(const mg_nrf *net, const float *xyz, long long n, const float *grad_out, float *out,
                          float *g_params, float *g_table, bool train, cudaStream_t st, const long long *idx = nullptr,
                          long long rows = 0);
void mg_launch_pair_count(const WsLayout &L, char *ws, const StackTable &tab, cudaStream_t st);
void mg_launch_build_slices(const StackIn &in, SliceDev *out, int S, cudaStream_t st);
void mg_launch_bin(const WsLayout &L, char *ws, const SliceDev *slices, const StackTable &tab, const float *mean,
                   const float *quat, const float *scale, const float *alpha, long long n, float K, float f64_ratio,
                   const CellGrid &cg, cudaStream_t st);
void mg_launch_render_fwd(const WsLayout &L, char *ws, const StackTable &tab, const SliceDev *slices,
                          const CellGrid &cg, float *out, cudaStream_t st, const float *target = nullptr,
                          float *grad = nullptr, double *loss_out = nullptr, long long n_vox = 0);
void mg_launch_render_bwd(const WsLayout &L, char *ws, const SliceDev *slices, const StackTable &tab,
                          const CellGrid &cg, const float *grad_out, const float *mean, const float *quat,
                          const float *scale, const float *alpha, long long n, float f64_ratio, float *g_mean,
                          float *g_quat, float *g_scale, float *g_alpha, bool zero_moments, cudaStream_t st);
void mg_launch_pose_grad(const WsLayout &L, char *ws, const SliceDev *slices, const float *mean, const float *quat,
                         const float *scale, const float *alpha, float f64_ratio, float *g_pose, cudaStream_t st);
// record geometry pass (one thread per record)
void mg_launch_rec_geom(const WsLayout &L, char *ws, const SliceDev *slices, const float *mean, const float *quat,
                        const float *scale, const float *alpha, float K, float f64_ratio, cudaStream_t st);
void mg_launch_scan_u32(const unsigned *in, unsigned *out, long long n_host, const unsigned long long *n_dev,
                        unsigned long long *part, unsigned long long *total_out, cudaStream_t st);
