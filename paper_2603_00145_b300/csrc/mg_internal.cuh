// mg_internal.cuh -- device-side data layout shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mgauss.h"

#define MG_TILE 16             // tile edge in pixels (record rectangles are in tiles)
#define MG_MAX_STACKS 32
#define MG_MAX_TILES_SLICE 4096  // 1024 x 1024 pixels
#define MG_CHUNK 512           // records per binning chunk (one warp each)
#define MG_SCAN_BLOCKS 256     // blocks of the three-phase scan

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
    float pu2, pv2;  // FP32 in-plane PSF variances along e_u, e_v (0: none)
    float dx, dy, hx, hy;  // spacing, 0.5*(W-1), 0.5*(H-1)
    int W, H, TX, TY;
    int tile_base;  // global index of tile (0,0)
    int stack;
    int same_frame;  // 1: rotation and profile bitwise equal to the previous slice's
    long long pix_base;  // offset of pixel (0,0) in the output
};

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
    unsigned int tile_ctr[2];  // work counters of the persistent render kernels
    unsigned long long reserved[24];
};

// Records are stored as structure-of-arrays.
struct Records {
    float4 *geo;        // (pcx, pcy, A, B2): centre in pixels, conic (log2 units)
    float2 *geo2;       // (C, amp)
    int *gid;           // Gaussian id
    int *slice;         // global slice id
    ushort4 *rect;      // tile rectangle (tx0, ty0, tx1, ty1)
    float *mom;         // [cap][8] backward moments (6 used)
    float *thr;         // q threshold of the K-sigma ellipsoid (log2 units), for pair counts
    long long cap;
};

// Workspace layout, computed identically on the host for fwd, bwd and the
// size query.
struct WsLayout {
    size_t hdr, slices, cnt, scan_part, rec_geo, rec_geo2, rec_gid, rec_slice, rec_rect, rec_mom, rec_thr;
    size_t chunk_base, hist, tile_cnt, tile_off, entries, gcnt, bits, gmap, rec_grad, total;
    long long S, NB, NW, SW, cap_records, cap_entries, cap_chunks, n_tiles, max_tiles;
};

// -------------------------------------------------------------------------
// small device helpers
// -------------------------------------------------------------------------
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
cudaError_t mg_launch_nrf(const mg_nrf *net, const float *xyz, long long n, const float *grad_out, float *out,
                          float *g_params, float *g_table, bool train, cudaStream_t st);
void mg_launch_pair_count(const WsLayout &L, char *ws, const StackTable &tab, cudaStream_t st);
void mg_launch_build_slices(const StackIn &in, SliceDev *out, int S, cudaStream_t st);
void mg_launch_bin(const WsLayout &L, char *ws, const SliceDev *slices, const StackTable &tab, const float *mean,
                   const float *quat, const float *scale, const float *alpha, long long n, float K, float f64_ratio,
                   cudaStream_t st);
void mg_launch_render_fwd(const WsLayout &L, char *ws, const StackTable &tab, float *out, cudaStream_t st);
void mg_launch_render_bwd(const WsLayout &L, char *ws, const SliceDev *slices, const StackTable &tab,
                          const float *grad_out, const float *mean, const float *quat, const float *scale,
                          const float *alpha, long long n, float f64_ratio, float *g_mean, float *g_quat,
                          float *g_scale, float *g_alpha, cudaStream_t st);
void mg_launch_pose_grad(const WsLayout &L, char *ws, const SliceDev *slices, const float *mean, const float *quat,
                         const float *scale, const float *alpha, float f64_ratio, float *g_pose, cudaStream_t st);
// record geometry pass (one thread per record)
void mg_launch_rec_geom(const WsLayout &L, char *ws, const SliceDev *slices, const float *mean, const float *quat,
                        const float *scale, const float *alpha, float K, float f64_ratio, cudaStream_t st);
void mg_launch_scan_u32(const unsigned *in, unsigned *out, long long n_host, const unsigned long long *n_dev,
                        unsigned long long *part, unsigned long long *total_out, cudaStream_t st);
