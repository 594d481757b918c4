/*
 * mgauss.h -- C ABI of the B300 (sm_103a) Magnetic Gaussian slice renderer.
 *
 * The library implements the rendering path of M-Gaussian (arxiv 2603.00145):
 * anisotropic 3D Gaussians G_i = {mu_i, Sigma_i, alpha_i} (Sec. 3.2, Eq. E2),
 * Sigma_i = R_i S_i S_i^T R_i^T with R_i from a unit quaternion and S_i the
 * diagonal of scales (Eq. E3), evaluated as the additive mixture of Eq. E7
 * (Sec. 3.3.2: no compositing, no sort) at the voxels of thick acquired slices
 * after each slice's rigid transform T_k, integrated along the slice normal
 * against a unit-integral Gaussian slice profile of FWHM = slice thickness.
 * Convolving a Gaussian with the profile adds covariances, so the term of
 * Gaussian i at a slice voxel x of slice k is
 *
 *     alpha_i sqrt(|Sigma_i| / |Sigma'_i|) exp(-1/2 (x-mu_i)^T Sigma'_i^-1 (x-mu_i)),
 *     Sigma'_i = Sigma_i + sig_s^2 n_k n_k^T,   sig_s^2 = FWHM^2 / (8 ln 2),
 *
 * which is Eq. E7 exactly when the thickness is 0 (volume sampling, Sec. 3.1).
 * A stack may also carry an in-plane Gaussian PSF (FWHM psf_u, psf_v along
 * the slice axes e_u, e_v; the paper models none): the full 3-D PSF
 * P = diag(psf_u^2, psf_v^2, thickness^2)/(8 ln 2) in the slice frame adds to
 * the covariance the same way, Sigma'_i = Sigma_i + R_k P R_k^T.
 * Like the paper's local Gaussian set G_local (Sec. 3.3.1), the sum is
 * restricted per 8x8 voxel tile (MG_TILE_EDGE): Gaussian i contributes to every voxel
 * of a tile of slice k iff its (i,k) record lists that tile (the record predicate
 * below: a K-sigma slab test plus the tile rectangle of the cut ellipse).
 *
 * CONVENTIONS
 *   Units are mm. Gaussians: mean [n,3], quat [n,4] = (w,x,y,z) with unit norm
 *   (normalise before calling; the rotation formula assumes it), scale [n,3]
 *   = per-axis standard deviations exp(s) > 0, alpha [n] (any real). All are
 *   FP32, C-contiguous, in DEVICE memory unless stated otherwise.
 *   A stack has n_slices slices of H x W pixels at dx x dy mm. xform
 *   [n_slices,12] (device) holds per slice the rotation R (3x3, row-major;
 *   columns e_u, e_v, e_n) and translation t: world = R (u,v,w)^T + t, the slice
 *   plane is w = 0. Pixel (i,j) (column i, row j) lies at u = (i-(W-1)/2) dx,
 *   v = (j-(H-1)/2) dy. Slices are written [n_slices,H,W], stacks concatenated
 *   in call order.
 *
 * RECORD PREDICATE (FP32, round-to-nearest, every operation rounded, no fused
 * multiply-add, in this order). q = (w,x,y,z), xx = x*x, ..., wz = w*z:
 *   R = [[1-2(yy+zz), 2(xy-wz), 2(xz+wy)], [2(xy+wz), 1-2(xx+zz), 2(yz-wx)],
 *        [2(xz-wy), 2(yz+wx), 1-2(xx+yy)]];  M_rc = R_rc s_c;
 *   Sigma_rc = (M_r0 M_c0 + M_r1 M_c1) + M_r2 M_c2;  a.b = (a0 b0 + a1 b1) + a2 b2;
 *   p = mu - t;  w0 = (e_n.mu) - (e_n.t), u0 = e_u.p, v0 = e_v.p;  (Sigma a)_r = Sigma_r . a;
 *   Lww = e_n.(Sigma e_n), Luw = e_u.(Sigma e_n), Lvw = e_v.(Sigma e_n),
 *   Luu = e_u.(Sigma e_u), Lvv = e_v.(Sigma e_v);  Sww = Lww + sig2;  K2 = K*K;
 *   sig2 = (float)(thickness^2 * 0.18033688011112042) (computed in double);
 *   the record exists iff  w0*w0 <= K2*Sww  (the K-sigma slab test); its pixel box:
 *   iSww = 1/Sww;  r2 = max(K2 - (w0*w0)*iSww, 0);  Cuu = max(Luu - (Luw*Luw)*iSww, 0) + pu2;
 *   Cvv = max(Lvv - (Lvw*Lvw)*iSww, 0) + pv2;  cu = u0 - (Luw*w0)*iSww;  cv = v0 - (Lvw*w0)*iSww;
 *   pu2 = (float)(psf_u^2 * 0.18033688011112042), pv2 likewise (computed in double);
 *   ru = sqrt(r2*Cuu), rv = sqrt(r2*Cvv);  hx = 0.5*(W-1), hy = 0.5*(H-1);
 *   idx = 1/dx, idy = 1/dy;  il = ceil((cu-ru)*idx + hx), ih = floor((cu+ru)*idx + hx),
 *   jl = ceil((cv-rv)*idy + hy), jh = floor((cv+rv)*idy + hy);
 *   the box is empty unless il<=ih, jl<=jh, il<=W-1, ih>=0, jl<=H-1, jh>=0 (NaN: empty);
 *   a non-empty box is clamped (il,jl up to 0, ih,jh down to W-1,H-1) and spans the
 *   tile rectangle [tx0, tx1] x [ty0, ty1] = [il/8, ih/8] x [jl/8, jh/8]; an empty box
 *   lists no tile (stored as the tile rectangle (1,1,0,0)).
 *   Row culling: tile row ty0 + n lists the columns [tx0 + l_n, tx1 - r_n]. l_n = r_n = 0
 *   for n >= 8, and for every row unless max(s) <= 64*min(s) (fmaxf/fminf over the
 *   three scales), r2 > 0, Cuu > 0, Cvv > 0 and tx1 > tx0. Otherwise, with
 *   Luv = e_v.(Sigma e_u), Cuv = Luv - (Luw*Lvw)*iSww, e = ru/Cuu, iCvv = 1/Cvv,
 *   g = Cuv*iCvv, h2 = max(Cuu - Cuv*g, 0),
 *   m = ru*(1/256) + dx*(1/1024), vL = cv - Cuv*e, vR = cv + Cuv*e, and per row n <= 7:
 *   a = max(jl, 8ty), b = min(jh, 8ty+7), va = ((float)a - hy)*dy, vb = ((float)b - hy)*dy;
 *   left: v = fminf(fmaxf(vL, va), vb); if v == vL: left = cu - ru, else d = v - cv,
 *     t = max(r2 - (d*d)*iCvv, 0), left = (cu + g*d) - sqrt(t*h2);
 *   right: the same with vR, cu + ru and + sqrt(t*h2);
 *   lo = fmaxf(ceil((left - m)*idx + hx), il), hi = fminf(floor((right + m)*idx + hx), ih);
 *   if !(lo <= hi): l_n = tx1 - tx0 + 1, r_n = 0 (the row lists nothing), else
 *   l_n = (int)lo/8 - tx0, r_n = tx1 - (int)hi/8; both then capped at 15 (a cap only
 *   lists more). The listed tiles hold every voxel of the cut ellipse with a margin.
 *   Tile (tx,ty) of a slice covers pixels 8tx..8tx+7 x 8ty..8ty+7.
 *   The count of records and of (record, tile) entries is therefore exact
 *   and reproducible bit for bit by any IEEE FP32 implementation.
 *
 * OWNERSHIP AND ERRORS
 *   The caller owns every buffer; the library never allocates device memory
 *   in a compute call. Scratch comes from a caller-provided workspace of the
 *   size the matching *_workspace_size query returns (256-byte aligned).
 *   Calls are asynchronous on `stream` (NULL = the legacy default stream),
 *   in stream order with the caller's work: the render kernels are
 *   programmatic dependent launches, each waiting for the completion of the
 *   work before it on the stream as its first action. Host-visible argument
 *   errors return immediately; capacity overflow and
 *   non-finite inputs are detected on the device, recorded in the workspace
 *   and reported by mg_render_stats_get (which synchronises the stream).
 *   On MG_ERR_CUDA the message of the CUDA error is in mg_last_error().
 *   Every function is thread-safe for distinct workspaces; mg_last_error is
 *   per thread.
 */
#ifndef MGAUSS_H
#define MGAUSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *mg_stream_t; /* a cudaStream_t */

#define MG_TILE_EDGE 8 /* edge of the evaluation tiles in pixels (record rectangles are in tiles) */

typedef enum {
    MG_OK = 0,
    MG_ERR_INVALID_ARG = 1,     /* bad pointer, size, shape or option; nothing launched */
    MG_ERR_CUDA = 2,            /* a CUDA runtime call failed; see mg_last_error() */
    MG_ERR_CAPACITY = 3,        /* records/entries did not fit the workspace; grow and retry */
    MG_ERR_DEVICE_TIMEOUT = 4,  /* reserved: no kernel of this library waits on another */
    MG_ERR_NOT_FINITE = 5,      /* a Gaussian or transform had a NaN/Inf or a scale <= 0 */
    MG_ERR_STALE_WORKSPACE = 6  /* backward called without the matching forward on this workspace */
} mg_status;

typedef struct {
    int64_t n;
    const float *mean;  /* [n,3] */
    const float *quat;  /* [n,4] (w,x,y,z), unit */
    const float *scale; /* [n,3] std-devs, > 0 */
    const float *alpha; /* [n] */
} mg_gaussians;

typedef struct {
    int32_t n_slices, H, W; /* 1 <= H, W <= 1024 */
    float dx, dy;           /* pixel spacing (mm), > 0 */
    float thickness;        /* slice-profile FWHM (mm), >= 0; 0 = point sampling (Eq. E7) */
    const float *xform;     /* device [n_slices,12] */
    float psf_u, psf_v;     /* in-plane Gaussian PSF FWHM (mm) along e_u, e_v, >= 0; 0 = none */
} mg_stack;

/*
 * Local set. MG_LOCAL_KSIGMA (the default, above): per (Gaussian, slice)
 * record, every voxel of the listed 8x8 tiles. MG_LOCAL_CELLS: the paper's
 * own rule (Sec. 3.3.1, Eqs. E4-E6): the normalised cube [-1,1]^3 (mapped to
 * grid_centre + grid_half * [-1,1]^3 mm) is cut into grid_res^3 cells; a
 * Gaussian sits in the cell of its mean, and voxel x sums exactly the
 * Gaussians whose cell is within block_radius cells of x's cell along each
 * axis. FP32, every operation rounded, in this order (hres = 0.5 * grid_res):
 *   cell(p)_a = (int) floor(clamp(((p_a - grid_centre_a) / grid_half + 1) * hres,
 *                                 -2^20, 2^20))
 *   voxel (i,j) of a slice: u = ((float)i - hx) * dx, v = ((float)j - hy) * dy,
 *                           x_a = (R_a0 u + R_a1 v) + t_a   (R, t of the slice)
 *   member iff |cell(x)_a - cell(mu)_a| <= block_radius for a = 0, 1, 2.
 * Records and tiles only bound the members: the (Gaussian, slice) record
 * exists iff the slice plane passes within m of the axis-aligned box of the
 * member cells (centre b_a = grid_centre_a + grid_half ((cell(mu)_a + 0.5)/hres - 1),
 * half-width e = (float)(grid_half (block_radius + 0.5) / hres), margin
 * m = (float)(grid_half / (1024 hres)), both in double):
 *   |n.(b - t)| <= e ((|n_0| + |n_1|) + |n_2|) + m,
 * and it lists the tiles of the pixel box of the box's extent along e_u, e_v
 * (centre u_c = e_u.(b - t), radius e ((|e_u0| + |e_u1|) + |e_u2|) + m, the
 * pixel box as in the K-sigma predicate). The sum at each voxel is then
 * restricted to members, per (record, voxel). The grid must be coarse enough
 * that an 8x8 tile spans at most 250 cells per axis (else
 * MG_ERR_INVALID_ARG). mg_render_pair_count is for MG_LOCAL_KSIGMA only.
 */
enum { MG_LOCAL_KSIGMA = 0, MG_LOCAL_CELLS = 1 };

typedef struct {
    float cutoff_k;      /* K of the K-sigma record predicate; default 3 */
    float f64_ratio;     /* record geometry and moments in FP64 when max(scale)/min(scale) > f64_ratio; default 16; <= 0: never */
    int64_t cap_records; /* workspace capacity in records; 0 = n * total slices (upper bound) capped at 2^28 */
    int64_t cap_entries; /* workspace capacity in (record, tile) entries; 0 = 8 * cap_records capped at 2^30 */
    int32_t local_set;   /* MG_LOCAL_KSIGMA (0, default) or MG_LOCAL_CELLS */
    int32_t grid_res;    /* MG_LOCAL_CELLS: cells per axis, 1..4096 */
    int32_t block_radius;   /* MG_LOCAL_CELLS: neighbourhood radius in cells, 0..1024 (the paper's default 5) */
    float grid_centre[3];   /* MG_LOCAL_CELLS: centre of the normalised cube (mm) */
    float grid_half;        /* MG_LOCAL_CELLS: half edge of the normalised cube (mm), > 0 */
} mg_opts;

/* Filled by mg_render_stats_get from the workspace of the last forward call. */
typedef struct {
    int64_t records;         /* (Gaussian, slice) records that exist */
    int64_t entries;         /* (record, tile) entries = evaluated (record, 8x8 tile) pairs */
    int64_t tiles;           /* tiles over all slices */
    int64_t cap_records, cap_entries;
    int32_t status;          /* MG_OK, MG_ERR_CAPACITY or MG_ERR_NOT_FINITE */
    int32_t reserved;
} mg_render_stats;

/* Default options (K = 3, f64_ratio = 16, capacities from the bounds above). */
mg_opts mg_default_opts(void);

/*
 * Workspace bytes for mg_render_fwd / mg_render_bwd with these Gaussians
 * (only n is read), stacks (shapes only) and options. Returns 0 on invalid
 * arguments. The same (n, stacks, opts) must be passed to fwd and bwd.
 */
size_t mg_render_workspace_size(const mg_gaussians *g, const mg_stack *stacks, int n_stacks, const mg_opts *opts);

/*
 * Forward render (Sec. 3.3.2, Eq. E7 with the slice profile; Sec. 3.3.1 local
 * set via records): out[total voxels] (device, FP32) is overwritten with the
 * slice values of all stacks. n_stacks in [1, 32]. Runs the record pass, the
 * tile binning (count, exclusive scan, stable scatter) and the per-tile
 * evaluation. The workspace keeps the records and bins for mg_render_bwd.
 * Capacity overflow leaves `out` undefined and is reported by
 * mg_render_stats_get as MG_ERR_CAPACITY with the required counts.
 */
mg_status mg_render_fwd(const mg_gaussians *g, const mg_stack *stacks, int n_stacks, const mg_opts *opts, float *out,
                        void *ws, size_t ws_bytes, mg_stream_t stream);

/*
 * mg_render_fwd with the L1 + L2 slice loss of mg_loss_l1l2 fused into the
 * writes of the evaluation kernel (Sec. 3.5.2 with the plain fit's loss; an
 * addition of this library): out as mg_render_fwd; with r = out - target,
 * grad[total voxels] (device FP32, may be NULL) receives
 * dloss/dout = (sign(r) + 2 r) / n bit for bit as mg_loss_l1l2 computes it, and
 * loss_out (device double[2]) = {mean|r| + mean r^2, sum r^2}, FP32 partials per
 * 8x8 tile added in FP64 in tile order (deterministic; it differs from
 * mg_loss_l1l2 only by the grouping of the FP32 partial sums, ~1e-8 relative). target: device FP32, same layout as out. The
 * workspace is that of mg_render_fwd and serves mg_render_bwd afterwards.
 * Errors: those of mg_render_fwd; target or loss_out NULL: MG_ERR_INVALID_ARG.
 */
mg_status mg_render_fwd_l1l2(const mg_gaussians *g, const mg_stack *stacks, int n_stacks, const mg_opts *opts,
                             const float *target, float *out, float *grad, double *loss_out, void *ws, size_t ws_bytes,
                             mg_stream_t stream);

/*
 * Adjoint of mg_render_fwd (the paper trains by differentiable rendering,
 * Sec. 3.1): given grad_out = dL/d(out) (device, FP32, total voxels), writes
 * dL/dmean [n,3], dL/dquat [n,4] (derivative of the rotation formula above in
 * the four quaternion components, projected on the tangent space of the unit
 * sphere at quat: the component along quat is removed, as the normalisation
 * quat = q_raw/|q_raw| does; the rotation formula is a rotation only for unit
 * quat), dL/dscale [n,3] and dL/dalpha [n]
 * (device, FP32, overwritten). The records are held fixed (the sum is
 * piecewise constant in them). Must follow mg_render_fwd on the same
 * workspace with the same arguments (else MG_ERR_STALE_WORKSPACE); the
 * per-pair terms are recomputed per tile, nothing per pair is stored.
 */
mg_status mg_render_bwd(const mg_gaussians *g, const mg_stack *stacks, int n_stacks, const mg_opts *opts,
                        const float *grad_out, float *g_mean, float *g_quat, float *g_scale, float *g_alpha, void *ws,
                        size_t ws_bytes, mg_stream_t stream);

/*
 * Gradient with respect to the slice poses T_k (the per-slice rigid
 * transforms of Sec. 3.3.2, 6 degrees of freedom each), for joint motion
 * estimation. Uses the per-record moments of dL/dI that the immediately
 * preceding mg_render_bwd on this workspace accumulated (same arguments as
 * that call's forward), so it returns the pose gradient of the same loss.
 * g_pose: device FP32 [S_total, 6], S_total = the slices of all stacks in
 * order; per slice k, with the slice transform world = R_k (u,v,w)^T + t_k:
 *   g_pose[6k+0..2] = dL/dt_k (world frame),
 *   g_pose[6k+3..5] = dL/domega_k for the rotation perturbed as
 *                     R_k (I + [omega_k]x), omega_k in the slice's own frame
 *                     (axes e_u, e_v, e_n), at omega_k = 0.
 * The bins are those of the forward (piecewise constant in the poses, like
 * the Gaussian gradients). Sums over a slice's records are FP64, fixed order.
 * Errors: MG_ERR_STALE_WORKSPACE when no mg_render_bwd followed the matching
 * forward on this workspace; MG_ERR_INVALID_ARG for NULL pointers.
 */
mg_status mg_render_pose_grad(const mg_gaussians *g, const mg_stack *stacks, int n_stacks, const mg_opts *opts,
                              float *g_pose, void *ws, size_t ws_bytes, mg_stream_t stream);

/*
 * Read-only introspection of a render workspace (for tests and tools): byte
 * offsets, inside the workspace, of the per-record arrays and of the tile
 * bins written by mg_render_fwd / mg_sample_volume. Records are ordered by
 * global slice, then ascending Gaussian id (the first `records` entries of
 * each array are valid): rec_gid int32, rec_slice int32; rec_rect: 16-byte
 * records of uint16x4 (tx0, ty0, tx1, ty1) followed by a uint64 of row insets
 * (byte n: l_n | r_n << 4 of the row culling above), rec_inset = rec_rect + 8
 * (same 16-byte stride). Bins: tile_off uint32 [tiles+1] (exclusive offsets,
 * global tile order = stacks, slices, ty*TX+tx), entries uint32 (record
 * ids). Returns MG_ERR_INVALID_ARG on bad arguments.
 */
typedef struct {
    uint64_t rec_gid, rec_slice, rec_rect, rec_inset, tile_off, entries, total_bytes;
} mg_ws_layout;
mg_status mg_render_ws_layout(const mg_gaussians *g, const mg_stack *stacks, int n_stacks, const mg_opts *opts,
                              mg_ws_layout *out);
mg_status mg_sample_ws_layout(int64_t n, int32_t G, const mg_opts *opts, mg_ws_layout *out);

/* Synchronises `stream`, then reads the counters and status of the last
 * forward on this workspace. Returns that status (or MG_ERR_CUDA/INVALID_ARG). */
mg_status mg_render_stats_get(const void *ws, size_t ws_bytes, mg_render_stats *stats, mg_stream_t stream);

/*
 * Inference sampling (Sec. 3.1 and Fig. 1c): the mixture of Eq. E7 (no slice
 * profile) on the isotropic grid of G^3 voxels, voxel (c,j,i) at
 * (cx + (i-(G-1)/2) h, cy + (j-(G-1)/2) h, float(cz + h (c-(G-1)/2))), the last
 * coordinate evaluated in double and rounded to float. centre is a HOST
 * array of 3 floats. out: device [G,G,G] (z,y,x) FP32, overwritten. Uses the
 * same record/binning/evaluation kernels with G z-planes as one stack.
 */
size_t mg_sample_workspace_size(int64_t n, int32_t G, const mg_opts *opts);
mg_status mg_sample_volume(const mg_gaussians *g, const float centre[3], float spacing, int32_t G, const mg_opts *opts,
                           float *out, void *ws, size_t ws_bytes, mg_stream_t stream);

/*
 * FP64 loss reduction of the plain-fit workload (Sec. 3.5.2 with the L1 + L2
 * slice loss): loss = mean|r| + mean r^2 over n voxels, r = pred - target,
 * accumulated in FP64 in a fixed order (deterministic). loss_out: device
 * double [2] = {loss, sum r^2}. grad (device FP32 [n], may be NULL) receives
 * dloss/dpred = (sign(r) + 2 r) / n.
 */
size_t mg_reduce_workspace_size(int64_t n);
mg_status mg_loss_l1l2(const float *pred, const float *target, int64_t n, float *grad, double *loss_out, void *ws,
                       size_t ws_bytes, mg_stream_t stream);

/*
 * mg_loss_l1l2 without any device allocation (an addition of this library;
 * the paper has no counterpart). Some callers cannot allocate device memory
 * or hand out a workspace: an application that reserves all device memory
 * for its own pool up front, a plugin inside another runtime that owns every
 * device allocation, a real-time loop that must never enter the driver's
 * allocator. This entry point keeps its per-block FP64 partial sums in a
 * fixed 128 KiB array inside the library (a file-scope __device__ array that
 * every GPU which loads the library holds until the process exits) and calls
 * no cudaMalloc, cudaFree or other allocating routine.
 *   Limit: n <= 33554432 (8192 partial blocks of 4096 voxels); larger n
 *   returns MG_ERR_INVALID_ARG with nothing launched.
 *   Set-up: each call made outside a stream capture looks up the array's
 *   device address with the device current (no allocation), so the address
 *   stays right across a cudaDeviceReset; a call inside a capture uses the
 *   address found by the last call outside one. So the first call on each
 *   device, and the first after a reset, must come before any stream
 *   capture (inside one it returns MG_ERR_INVALID_ARG, nothing launched).
 *   Sharing: every call uses the same array. Calls that overlap on the GPU
 *   (other streams, other host threads) race on it; serialise them. Each
 *   call writes every slot it reads, so nothing needs clearing between calls.
 * Arguments and results are those of mg_loss_l1l2 (device pointers; grad
 * may be NULL); the result agrees with mg_loss_l1l2 up to FP64 summation
 * order.
 */
mg_status mg_loss_l1l2_noalloc(const float *pred, const float *target, int64_t n, float *grad, double *loss_out,
                               mg_stream_t stream);

/*
 * The paper's reconstruction loss (Sec. 3.5.2) on rendered slices:
 *   L_recon = L_L1 + lambda_ssim * (1 - mean SSIM),
 * L_L1 = mean over all pixels of smooth_L1(pred - target) (Eq. E11: 0.5 r^2
 * for |r| < 1, else |r| - 0.5), SSIM the structural similarity of Wang et
 * al. (2004) of each pixel of each 2-D slice: 11 x 11 Gaussian window of
 * standard deviation 1.5 pixels (unit sum), zero padding outside the slice,
 * C1 = 0.01^2, C2 = 0.03^2 (intensity range 1); the mean runs over every
 * pixel of every slice. The paper does not write L_SSIM out; 1 - mean SSIM
 * over whole slices is the reading (the paper's lambda_SSIM is 0.5).
 * pred, target: device FP32 slices laid out as mg_render_fwd writes them
 * (stacks concatenated, [n_slices, H, W] each); only n_slices, H and W of the
 * stacks are read (1 <= H, W <= 16384). grad (device FP32, same size, may be
 * NULL) is overwritten with dL_recon/dpred. loss_out: device double[3] =
 * {L_recon, mean smooth-L1, mean SSIM}; the sums are FP64 and fixed-order
 * (the result is the same bit pattern on every run). Evaluation is FP32.
 * ws: device scratch of mg_loss_recon_workspace_size bytes (0 on invalid
 * stacks). Errors: MG_ERR_INVALID_ARG (nothing launched).
 */
size_t mg_loss_recon_workspace_size(const mg_stack *stacks, int n_stacks);
mg_status mg_loss_recon(const float *pred, const float *target, const mg_stack *stacks, int n_stacks,
                        float lambda_ssim, float *grad, double *loss_out, void *ws, size_t ws_bytes,
                        mg_stream_t stream);

/* FP64 sum of squared differences (for MSE / PSNR, Sec. 4.1.3): out: device
 * double [1] = sum (a-b)^2, fixed-order FP64 accumulation. */
mg_status mg_sq_diff_sum(const float *a, const float *b, int64_t n, double *out, void *ws, size_t ws_bytes,
                         mg_stream_t stream);

/*
 * Pair statistics of the last forward on this workspace (same arguments as
 * that forward): counts[0] = (record, in-image voxel) pairs inside the
 * record's K-sigma ellipsoid of the profile-convolved covariance (FP32 test
 * of the voxel's quadratic form against K^2 - w0^2/Sww), counts[1] = all
 * evaluated pairs (records x in-image voxels of their listed tiles).
 * counts: HOST int64[2]. Synchronises `stream`.
 */
mg_status mg_render_pair_count(const mg_gaussians *g, const mg_stack *stacks, int n_stacks, const mg_opts *opts,
                               void *ws, size_t ws_bytes, int64_t counts[2], mg_stream_t stream);

/*
 * Per-stage GPU timing with CUDA events. While enabled, every kernel stage
 * this library launches is bracketed by two events on its stream;
 * mg_profile_read waits for them and returns the accumulated milliseconds
 * and call counts per stage (arrays of mg_profile_stage_count() entries,
 * host memory; either may be NULL), optionally resetting them. Off by
 * default; enabling affects all threads of the process.
 */
mg_status mg_profile_enable(int on);
/* As mg_profile_enable, for the stages whose bit is set in mask only (bit i:
 * stage i of mg_profile_stage_name); the others launch without events. */
mg_status mg_profile_stages(uint32_t mask);
int mg_profile_stage_count(void);
const char *mg_profile_stage_name(int stage);
mg_status mg_profile_read(double *ms, int64_t *calls, int reset);

/*
 * Neural residual field (Sec. 3.4, Eq. E8): r(x) = out_scale * tanh(MLP(enc(x)))
 * for coordinates x in the canonical cube [-1,1]^3, added to the Gaussian
 * intensity (I_final = I + r). Two encodings:
 *   MG_NRF_FOURIER (the paper's): enc(x) = [x, sin(2^j pi x), cos(2^j pi x)],
 *     j = 0..5 (per band: sin of x0,x1,x2 then cos of x0,x1,x2; 39 features),
 *     4 hidden layers of 64 SiLU units;
 *   MG_NRF_GRID: 16-level multiresolution hash grid, 2 features per level
 *     (resolution floor(n_min * b^l), b = exp((ln n_max - ln n_min)/15);
 *     p = clamp((x+1)/2, 0, 1); cell min(floor(p N), N-1); corners looked up
 *     densely when (N+1)^3 <= 2^log2_table, else by the spatial hash
 *     (x * 1) ^ (y * 2654435761) ^ (z * 805459861) mod 2^log2_table;
 *     trilinear weights), 2 hidden layers of 64 ReLU units.
 * Precision MG_NRF_BF16: weights and activations rounded to BF16, hidden
 * layers on the tensor cores (mma.sync BF16, FP32 accumulation);
 * MG_NRF_FP32: FP32 throughout (SIMT).
 * params (device, FP32): for each hidden layer W[64][in] row-major then
 * b[64]; then w_out[64], b_out (mg_nrf_param_count floats).
 */
typedef enum { MG_NRF_FOURIER = 0, MG_NRF_GRID = 1 } mg_nrf_encoding;
typedef enum { MG_NRF_BF16 = 0, MG_NRF_FP32 = 1 } mg_nrf_precision;
typedef struct {
    int32_t encoding;   /* mg_nrf_encoding */
    int32_t precision;  /* mg_nrf_precision */
    const float *params;
    const float *table; /* MG_NRF_GRID: device FP32 [16][2^log2_table][2], 8-byte aligned (an
                           entry's two features are one 8-byte word); else unused */
    int32_t log2_table, n_min, n_max; /* MG_NRF_GRID geometry; 0 = 19, 16, 512 */
    float out_scale;    /* bound of |r|; the paper's 0.1 */
    /* Encoding cache (MG_NRF_GRID; ignored for MG_NRF_FOURIER): a device buffer
     * of mg_nrf_enc_bytes(net, n) bytes holding, for batch position i < n, the
     * 32 encoded features of point i in the precision's element type (BF16 or
     * FP32), caller-owned. enc_mode MG_NRF_ENC_STORE: a forward call (mg_nrf_fwd,
     * mg_nrf_fwd_at) also writes the features; MG_NRF_ENC_LOAD: a backward call
     * reads them instead of gathering the table again (the training step runs
     * the forward and then the backward on the same points: the backward's grid
     * gathers were 82M L2 requests per 2^20 points). The features read back
     * are the bits the gathers would give, so results are unchanged. With
     * LOAD the buffer must hold a STORE call's features for the same points,
     * table and geometry. MG_NRF_ENC_NONE (0): no cache. */
    void *enc;
    int32_t enc_mode;
} mg_nrf;
enum { MG_NRF_ENC_NONE = 0, MG_NRF_ENC_STORE = 1, MG_NRF_ENC_LOAD = 2 };
/* Bytes of the encoding cache for n points (0 for MG_NRF_FOURIER or bad args). */
size_t mg_nrf_enc_bytes(const mg_nrf *net, int64_t n);

/* Number of FP32 parameters of an encoding's MLP (-1 for an unknown one). */
int64_t mg_nrf_param_count(int32_t encoding);
/* out[i] = r(xyz[i]) for n points (device xyz [n,3], out [n]). */
mg_status mg_nrf_fwd(const mg_nrf *net, const float *xyz, int64_t n, float *out, mg_stream_t stream);
/* Gradients of sum_i grad_out[i] r(xyz[i]): g_params (device, param_count
 * floats) and, for MG_NRF_GRID, g_table (device, same shape as table,
 * 16-byte aligned: two neighbouring entries that share a 16-byte word take
 * one atomic; MG_ERR_INVALID_ARG otherwise) are overwritten. Accumulated with
 * atomics (FP32 summation order varies). */
mg_status mg_nrf_bwd(const mg_nrf *net, const float *xyz, int64_t n, const float *grad_out, float *g_params,
                     float *g_table, mg_stream_t stream);
/* The residual at a batch of rows of a coordinate table (the NRF's random
 * voxel batch of a training step, Sec. 3.4, without a gathered copy): for
 * i < n, acc[idx[i]] += r(coords[idx[i]]). Device buffers: coords [rows,3],
 * idx int64 [n], acc [rows]; repeated rows each add (atomic adds, so the
 * summation order of repeats is unspecified). An index outside [0, rows) is
 * skipped: it adds nothing and reads nothing. mg_nrf_bwd_at: gradients of
 * sum_i grad_acc[idx[i]] r(coords[idx[i]]) (grad_acc [rows]), outputs and
 * errors as mg_nrf_bwd. n == 0 is valid (fwd: no work; bwd: zero gradients). */
mg_status mg_nrf_fwd_at(const mg_nrf *net, const float *coords, int64_t rows, const int64_t *idx, int64_t n,
                        float *acc, mg_stream_t stream);
mg_status mg_nrf_bwd_at(const mg_nrf *net, const float *coords, int64_t rows, const int64_t *idx, int64_t n,
                        const float *grad_acc, float *g_params, float *g_table, mg_stream_t stream);

/*
 * Parameterisation of the fit (Sec. 3.2) and the anisotropy regulariser
 * (Eqs. E12, E13), so that a training step needs no framework autograd for
 * them. Per Gaussian i (device FP32 arrays):
 *   mean_i  = centre + half * mean_c_i        (canonical coordinates; centre: HOST float[3], mm)
 *   quat_i  = q_raw_i / |q_raw_i|             ([n,4], 16-byte aligned)
 *   scale_i = exp(ls_i)
 *   L_aniso = (1/n) sum_i max(0, max_a scale_ia / min_a scale_ia - lambda_r)
 * (E13 writes the ratio on the log-scales; the ratio of the scales is the
 * reading). mg_params_fwd writes mean, quat, scale and, when aniso_out
 * (device double[1]) is given, L_aniso in FP64 with a fixed summation order
 * (ws: device scratch of mg_params_workspace_size(n) bytes). mg_params_bwd
 * writes dL/d(mean_c, q_raw, ls) for L = (the loss whose gradients g_mean,
 * g_quat, g_scale are given) + lambda_aniso * L_aniso; a tie for the largest or
 * smallest scale takes the first index. Errors: MG_ERR_INVALID_ARG.
 */
size_t mg_params_workspace_size(int64_t n);
mg_status mg_params_fwd(int64_t n, const float *mean_c, const float *quat_raw, const float *log_scale,
                        const float centre[3], float half, float lambda_r, float *mean, float *quat, float *scale,
                        double *aniso_out, void *ws, size_t ws_bytes, mg_stream_t stream);
mg_status mg_params_bwd(int64_t n, const float *quat_raw, const float *log_scale, float half, float lambda_r,
                        float lambda_aniso, const float *g_mean, const float *g_quat, const float *g_scale,
                        float *g_mean_c, float *g_quat_raw, float *g_log_scale, mg_stream_t stream);

/*
 * Device status word of a render workspace. The first 32-bit word of a
 * workspace filled by mg_render_fwd / mg_sample_volume holds the forward's
 * status bits; a bit of MG_WS_FAIL_BITS set means the forward failed (bins
 * over capacity, or a non-finite input) and its output is incomplete. It is
 * written by the device during the forward, so stream-ordered kernels (such
 * as mg_adam_step below) can read it without a host round trip.
 */
#define MG_WS_FAIL_BITS 0x0Fu

/*
 * Optimiser step of the fit (Sec. 4.1.4: Adam, one learning rate per
 * parameter group), all groups in one launch. Per element, with t = *step + 1:
 *   m <- b1 m + (1-b1) g;  v <- b2 v + (1-b2) g^2;
 *   p <- p - lr/(1-b1^t) * m / (sqrt(v)/sqrt(1-b2^t) + eps)
 * (Kingma & Ba 2015, Algorithm 1, eps added after the bias correction of v),
 * then p is clamped to [clamp_lo, clamp_hi] when clamp_lo <= clamp_hi (the
 * alpha range [0, 1] of Sec. 3.2; pass lo > hi for no clamp). *step (device
 * int32) is incremented after the update.
 * Predication: when `status` (device, may be NULL) is given and
 * (*status & status_mask) != 0 at the time the step runs, nothing is changed:
 * no parameter, moment or step. With status = a render workspace's status word
 * and status_mask = MG_WS_FAIL_BITS, an iteration whose forward failed is a
 * no-op, so a fit can be replayed without host checks and detect failures
 * later from *step. The paper has no counterpart of the predicate.
 * All group pointers are device FP32 arrays of n elements; m and v are the
 * caller's moment buffers (zero before the first step). 1 <= n_groups <= 8.
 * Errors: MG_ERR_INVALID_ARG (NULL pointers, betas outside [0,1), eps <= 0,
 * negative or non-finite lr); nothing is launched then.
 */
#define MG_ADAM_MAX_GROUPS 8
typedef struct {
    float *param;
    const float *grad;
    float *m, *v;
    int64_t n;
    float lr;
    float clamp_lo, clamp_hi;
} mg_adam_group;
mg_status mg_adam_step(const mg_adam_group *groups, int n_groups, float beta1, float beta2, float eps,
                       int32_t *step, const uint32_t *status, uint32_t status_mask, mg_stream_t stream);

const char *mg_status_string(mg_status s);
const char *mg_last_error(void);
/* Library version string. */
const char *mg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MGAUSS_H */
