// mg_api.cu -- the C ABI (include/mgauss.h): argument checks, workspace
// layout and the launch sequence of each entry point.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "mg_internal.cuh"

int mg_reduce_blocks(long long n);
void mg_launch_loss_l1l2(const float *pred, const float *target, long long n, float *grad, double *out,
                         double *part, cudaStream_t st);
void mg_launch_sq_diff(const float *a, const float *b, long long n, double *out, double *part, cudaStream_t st);

// ---------------------------------------------------------------------------
// per-stage CUDA-event timing
// ---------------------------------------------------------------------------
namespace prof {
std::atomic<unsigned> on{0u};  // bit per stage
std::mutex mu;
struct Pending {
    int stage;
    cudaEvent_t a, b;
};
std::vector<Pending> pending;
std::vector<cudaEvent_t> pool;
double ms[MG_NSTAGES];
long long calls[MG_NSTAGES];
thread_local cudaEvent_t open_ev[MG_NSTAGES];
const char *names[MG_NSTAGES] = {"slices",      "k1_count",   "scan_records", "k1_emit",    "chunks",
                                 "bin_hist",    "bin_colscan", "scan_tiles",   "bin_scatter", "render_fwd",
                                 "zero_moments", "render_bwd", "chain",        "loss",       "pair_count",
                                 "nrf_fwd",     "nrf_bwd",     "rec_geom",   "rec_fill"};

cudaEvent_t get_event()
{
    std::lock_guard<std::mutex> lk(mu);
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
}  // namespace prof

void mg_prof_begin(int stage, cudaStream_t st)
{
    if (!((prof::on.load(std::memory_order_relaxed) >> stage) & 1u)) return;
    cudaEvent_t e = prof::get_event();
    cudaEventRecord(e, st);
    prof::open_ev[stage] = e;
}

void mg_prof_end(int stage, cudaStream_t st)
{
    if (!((prof::on.load(std::memory_order_relaxed) >> stage) & 1u) || !prof::open_ev[stage]) return;
    cudaEvent_t e = prof::get_event();
    cudaEventRecord(e, st);
    std::lock_guard<std::mutex> lk(prof::mu);
    prof::pending.push_back({stage, prof::open_ev[stage], e});
    prof::open_ev[stage] = nullptr;
}

namespace {

thread_local std::string g_last_error;

mg_status fail(mg_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

mg_status check_cuda(const char *where)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return MG_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr double FWHM2VAR = 0.18033688011112042;  // 1 / (8 ln 2)

struct StackDesc {
    int n_slices, H, W;
    float dx, dy, thickness;
    const float *xform;
    float psf_u, psf_v;
};

mg_opts resolve_opts(const mg_opts *o, long long n, long long S)
{
    mg_opts r = mg_default_opts();
    if (o) r = *o;
    if (!(r.cutoff_k > 0.f)) r.cutoff_k = 3.0f;
    long long bound = n * S;
    if (r.cap_records <= 0) r.cap_records = bound < (1ll << 28) ? bound : (1ll << 28);
    if (r.cap_records < 1) r.cap_records = 1;
    if (r.cap_entries <= 0) {
        long long e = 8 * r.cap_records;
        r.cap_entries = e < (1ll << 30) ? e : (1ll << 30);
    }
    return r;
}

// The kernels' view of the MG_LOCAL_CELLS options (cg.on = 0 for the K-sigma
// set). max_px: the largest pixel spacing of the stacks (mm), for the check
// that a tile (MG_TILE pixels square) spans at most 250 cells per axis.
bool make_cellgrid(const mg_opts &o, float max_px, CellGrid &cg, std::string &why)
{
    memset(&cg, 0, sizeof(cg));
    if (o.local_set == MG_LOCAL_KSIGMA) return true;
    if (o.local_set != MG_LOCAL_CELLS) {
        why = "local_set must be MG_LOCAL_KSIGMA or MG_LOCAL_CELLS";
        return false;
    }
    if (o.grid_res < 1 || o.grid_res > 4096 || o.block_radius < 0 || o.block_radius > 1024 || !(o.grid_half > 0.f) ||
        !isfinite(o.grid_half) || !isfinite(o.grid_centre[0]) || !isfinite(o.grid_centre[1]) ||
        !isfinite(o.grid_centre[2])) {
        why = "MG_LOCAL_CELLS needs 1 <= grid_res <= 4096, 0 <= block_radius <= 1024, grid_half > 0, finite centre";
        return false;
    }
    const double hres = 0.5 * (double)o.grid_res, h = (double)o.grid_half;
    if (2.0 * MG_TILE * (double)max_px * hres / h + 2.0 > 250.0) {
        why = "MG_LOCAL_CELLS grid too fine: an 8x8 tile would span more than 250 cells";
        return false;
    }
    cg.on = 1;
    cg.R = o.block_radius;
    cg.hres = (float)hres;
    cg.h = o.grid_half;
    for (int a = 0; a < 3; ++a) cg.C[a] = o.grid_centre[a];
    cg.e = (float)(h * ((double)o.block_radius + 0.5) / hres);
    cg.m = (float)(h / (1024.0 * hres));
    return true;
}

float max_pixel(const std::vector<StackDesc> &st)
{
    float m = 0.f;
    for (const StackDesc &d : st) m = fmaxf(m, fmaxf(d.dx, d.dy));
    return m;
}

bool valid_stacks(const std::vector<StackDesc> &st, bool need_xform, std::string &why)
{
    if (st.empty() || st.size() > MG_MAX_STACKS) {
        why = "n_stacks must be in [1, 32]";
        return false;
    }
    for (size_t s = 0; s < st.size(); ++s) {
        const StackDesc &d = st[s];
        if (d.n_slices < 1 || d.H < 1 || d.W < 1 || d.H > 1024 || d.W > 1024) {
            why = "stack " + std::to_string(s) + ": need n_slices >= 1 and 1 <= H, W <= 1024";
            return false;
        }
        if (!(d.dx > 0.f) || !(d.dy > 0.f) || !(d.thickness >= 0.f) || !isfinite(d.dx) || !isfinite(d.dy) ||
            !isfinite(d.thickness)) {
            why = "stack " + std::to_string(s) + ": need dx, dy > 0 and thickness >= 0, finite";
            return false;
        }
        if (!(d.psf_u >= 0.f) || !(d.psf_v >= 0.f) || !isfinite(d.psf_u) || !isfinite(d.psf_v)) {
            why = "stack " + std::to_string(s) + ": need psf_u, psf_v >= 0, finite";
            return false;
        }
        if (need_xform && !d.xform) {
            why = "stack " + std::to_string(s) + ": xform is NULL";
            return false;
        }
    }
    return true;
}

WsLayout make_layout(long long n, const std::vector<StackDesc> &st, const mg_opts &o)
{
    WsLayout L;
    memset(&L, 0, sizeof(L));
    long long S = 0, tiles = 0, tmax = 0;
    for (const StackDesc &d : st) {
        long long TX = (d.W + MG_TILE - 1) / MG_TILE, TY = (d.H + MG_TILE - 1) / MG_TILE;
        S += d.n_slices;
        tiles += (long long)d.n_slices * TX * TY;
        if (TX * TY > tmax) tmax = TX * TY;
    }
    L.S = S;
    L.NB = (n + 255) / 256;
    L.NW = (n + 31) / 32;
    L.SW = (S + 31) / 32;
    L.cap_records = o.cap_records;
    L.cap_entries = o.cap_entries;
    L.cap_chunks = o.cap_records / MG_CHUNK + S + 1;
    L.n_tiles = tiles;
    L.max_tiles = tmax;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align256(off + bytes);
        return at;
    };
    L.hdr = take(sizeof(WsHeader));
    L.slices = take(sizeof(SliceDev) * (size_t)S);
    L.cnt = take(sizeof(unsigned) * (size_t)(S * L.NW + 1));
    L.gcnt = take(sizeof(unsigned) * (size_t)(n + 1));
    L.bits = take(sizeof(unsigned) * (size_t)(L.SW * n + 1));
    L.scan_part = take(sizeof(unsigned long long) * 2 * MG_SCAN_BLOCKS);
    L.rec_geo = take(16 * (size_t)L.cap_records);
    L.rec_geo2 = take(8 * (size_t)L.cap_records);
    L.rec_gid = take(4 * (size_t)L.cap_records);
    L.rec_slice = take(4 * (size_t)L.cap_records);
    L.rec_rect = take(16 * (size_t)L.cap_records);  // RecTiles: rect, then the row insets
    L.rec_inset = L.rec_rect + 8;
    L.rec_mom = take(32 * (size_t)L.cap_records);
    L.rec_thr = take(4 * (size_t)L.cap_records);
    L.chunk_base = take(sizeof(unsigned) * 2 * (size_t)(S + 1));
    L.hist = take(sizeof(unsigned) * (size_t)L.cap_chunks * (size_t)tmax);
    L.tile_cnt = take(sizeof(unsigned) * (size_t)tiles);
    L.tile_off = take(sizeof(unsigned) * (size_t)(tiles + 1));
    L.tile_list = take(sizeof(unsigned) * (size_t)tiles);
    L.dense_list = take(sizeof(unsigned) * (size_t)tiles);
    L.sparse_list = take(sizeof(unsigned) * (size_t)tiles);
    // loss partials: per tile and per block of 2048 tiles (fused forward), or per
    // reduction block (no Gaussians)
    L.tile_loss = take(16 * (size_t)(tiles + tiles / 2048 + 1 > 148 * 8 ? tiles + tiles / 2048 + 1 : 148 * 8));
    L.entries = take(sizeof(unsigned) * (size_t)L.cap_entries);
    L.gmap = take(sizeof(unsigned) * (size_t)L.cap_records);
    L.rec_grad = take(32 * (size_t)L.cap_records);  // slice-pose shares: 2 float4 per record
    L.rec_cell = o.local_set == MG_LOCAL_CELLS ? take(16 * (size_t)L.cap_records) : 0;
    L.rec_f64 = take((size_t)L.cap_records);
    L.rec_mom64 = take(sizeof(double) * MOM64_STRIDE * (size_t)L.cap_records);
    L.big_n = take(sizeof(unsigned) * (size_t)L.cap_chunks);
    L.big_list = take(sizeof(unsigned) * BIG_MAX * (size_t)L.cap_chunks);
    L.tile_small = take(sizeof(unsigned) * (size_t)tiles);
    L.tile_big = take(sizeof(unsigned) * (size_t)tiles);
    L.total = off;
    return L;
}

StackTable make_table(const std::vector<StackDesc> &st)
{
    StackTable t;
    memset(&t, 0, sizeof(t));
    t.n_stacks = (int)st.size();
    int tb = 0, sb = 0;
    long long pb = 0;
    int tmax = 0;
    for (size_t s = 0; s < st.size(); ++s) {
        const StackDesc &d = st[s];
        int TX = (d.W + MG_TILE - 1) / MG_TILE, TY = (d.H + MG_TILE - 1) / MG_TILE;
        t.tile_base[s] = tb;
        t.slice_base[s] = sb;
        t.pix_base[s] = pb;
        t.TX[s] = TX;
        t.TY[s] = TY;
        t.W[s] = d.W;
        t.H[s] = d.H;
        tb += d.n_slices * TX * TY;
        sb += d.n_slices;
        pb += (long long)d.n_slices * d.H * d.W;
        if (TX * TY > tmax) tmax = TX * TY;
    }
    t.tile_base[st.size()] = tb;
    t.slice_base[st.size()] = sb;
    t.pix_base[st.size()] = pb;
    t.n_slices_total = sb;
    t.n_tiles_total = tb;
    t.max_tiles_slice = tmax;
    return t;
}

StackIn make_stack_in(const std::vector<StackDesc> &st)
{
    StackIn in;
    memset(&in, 0, sizeof(in));
    in.n_stacks = (int)st.size();
    for (size_t s = 0; s < st.size(); ++s) {
        in.n_slices[s] = st[s].n_slices;
        in.H[s] = st[s].H;
        in.W[s] = st[s].W;
        in.dx[s] = st[s].dx;
        in.dy[s] = st[s].dy;
        in.sig2[s] = (float)((double)st[s].thickness * (double)st[s].thickness * FWHM2VAR);
        in.pu2[s] = (float)((double)st[s].psf_u * (double)st[s].psf_u * FWHM2VAR);
        in.pv2[s] = (float)((double)st[s].psf_v * (double)st[s].psf_v * FWHM2VAR);
        in.xform[s] = st[s].xform;
    }
    return in;
}

std::vector<StackDesc> to_desc(const mg_stack *stacks, int n_stacks)
{
    std::vector<StackDesc> v;
    if (!stacks || n_stacks < 1 || n_stacks > MG_MAX_STACKS) return v;
    for (int s = 0; s < n_stacks; ++s)
        v.push_back({stacks[s].n_slices, stacks[s].H, stacks[s].W, stacks[s].dx, stacks[s].dy, stacks[s].thickness,
                     stacks[s].xform, stacks[s].psf_u, stacks[s].psf_v});
    return v;
}

bool valid_gauss(const mg_gaussians *g, std::string &why, bool need_ptrs = true)
{
    if (!g) {
        why = "gaussians is NULL";
        return false;
    }
    if (g->n < 0 || g->n > 0x7fffffffll) {
        why = "n must be in [0, 2^31)";
        return false;
    }
    if (need_ptrs && g->n > 0 && (!g->mean || !g->quat || !g->scale || !g->alpha)) {
        why = "a Gaussian parameter pointer is NULL";
        return false;
    }
    return true;
}

// what the backward needs to know about the forward that filled a workspace
struct FwdTag {
    long long n;
    const void *p[4];
    std::vector<float> stack_key;
    std::vector<const void *> xforms;
    float K, f64;
    long long capr, cape;
    int ls, res, R;
    float gc[4];
    bool bwd_done = false;  // an mg_render_bwd has filled the moments since this forward
};

std::mutex g_tag_mu;
std::unordered_map<const void *, FwdTag> g_tags;

FwdTag make_tag(const mg_gaussians *g, const std::vector<StackDesc> &st, const mg_opts &o)
{
    FwdTag t;
    t.n = g->n;
    t.p[0] = g->mean;
    t.p[1] = g->quat;
    t.p[2] = g->scale;
    t.p[3] = g->alpha;
    for (const StackDesc &d : st) {
        t.stack_key.insert(t.stack_key.end(),
                           {(float)d.n_slices, (float)d.H, (float)d.W, d.dx, d.dy, d.thickness, d.psf_u, d.psf_v});
        t.xforms.push_back(d.xform);
    }
    t.K = o.cutoff_k;
    t.f64 = o.f64_ratio;
    t.capr = o.cap_records;
    t.cape = o.cap_entries;
    t.ls = o.local_set;
    t.res = o.grid_res;
    t.R = o.block_radius;
    t.gc[0] = o.grid_centre[0];
    t.gc[1] = o.grid_centre[1];
    t.gc[2] = o.grid_centre[2];
    t.gc[3] = o.grid_half;
    return t;
}

bool same_tag(const FwdTag &a, const FwdTag &b)
{
    return a.n == b.n && memcmp(a.p, b.p, sizeof(a.p)) == 0 && a.stack_key == b.stack_key && a.xforms == b.xforms &&
           a.K == b.K && a.f64 == b.f64 && a.capr == b.capr && a.cape == b.cape && a.ls == b.ls &&
           (a.ls == MG_LOCAL_KSIGMA ||
            (a.res == b.res && a.R == b.R && memcmp(a.gc, b.gc, sizeof(a.gc)) == 0));
}

mg_status render_fwd_impl(const mg_gaussians *g, const std::vector<StackDesc> &st, const StackIn &in,
                          const mg_opts *opts, float *out, void *ws, size_t ws_bytes, cudaStream_t stream,
                          const float *target = nullptr, float *grad = nullptr, double *loss_out = nullptr)
{
    std::string why;
    if (!valid_gauss(g, why)) return fail(MG_ERR_INVALID_ARG, why);
    if (!valid_stacks(st, !in.planes, why)) return fail(MG_ERR_INVALID_ARG, why);
    if (!out || !ws) return fail(MG_ERR_INVALID_ARG, "out or workspace is NULL");
    if (((uintptr_t)ws & 255) != 0) return fail(MG_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    long long S = 0, tiles = 0;
    for (const StackDesc &d : st) {
        S += d.n_slices;
        tiles += (long long)d.n_slices * ((d.W + MG_TILE - 1) / MG_TILE) * ((d.H + MG_TILE - 1) / MG_TILE);
    }
    if (tiles >= (1ll << 31) || S >= (1ll << 20)) return fail(MG_ERR_INVALID_ARG, "too many slices or tiles");
    mg_opts o = resolve_opts(opts, g->n, S);
    if (o.cap_records >= (1ll << 31) || o.cap_entries >= (1ll << 32) - 1)
        return fail(MG_ERR_INVALID_ARG, "capacities must be below 2^31 records and 2^32-1 entries");
    CellGrid cg;
    if (!make_cellgrid(o, in.planes ? in.h : max_pixel(st), cg, why)) return fail(MG_ERR_INVALID_ARG, why);
    WsLayout L = make_layout(g->n, st, o);
    if (ws_bytes < L.total)
        return fail(MG_ERR_INVALID_ARG, "workspace too small: need " + std::to_string(L.total) + " bytes");
    char *w = (char *)ws;
    SliceDev *slices = (SliceDev *)(w + L.slices);
    StackTable tab = make_table(st);
    mg_launch_build_slices(in, slices, (int)S, stream);
    if (g->n > 0) {
        mg_launch_bin(L, w, slices, tab, g->mean, g->quat, g->scale, g->alpha, g->n, o.cutoff_k, o.f64_ratio, cg,
                      stream);
        mg_launch_render_fwd(L, w, tab, slices, cg, out, stream, target, grad, loss_out, tab.pix_base[tab.n_stacks]);
    } else {
        // no Gaussians: empty bins and a zero output
        cudaMemsetAsync(w + L.hdr, 0, sizeof(WsHeader), stream);
        cudaMemsetAsync(w + L.tile_off, 0, sizeof(unsigned) * (size_t)(tiles + 1), stream);
        cudaMemsetAsync(out, 0, sizeof(float) * (size_t)tab.pix_base[tab.n_stacks], stream);
        if (target)
            mg_launch_loss_l1l2(out, target, tab.pix_base[tab.n_stacks], grad, loss_out, (double *)(w + L.tile_loss),
                                stream);
    }
    mg_status s = check_cuda("mg_render_fwd");
    if (s != MG_OK) return s;
    {
        std::lock_guard<std::mutex> lk(g_tag_mu);
        g_tags[ws] = make_tag(g, st, o);
    }
    return MG_OK;
}

}  // namespace

mg_status mg_set_error(mg_status s, const char *msg) { return fail(s, msg); }

extern "C" {

mg_opts mg_default_opts(void)
{
    mg_opts o;
    o.cutoff_k = 3.0f;
    o.f64_ratio = 16.0f;
    o.cap_records = 0;
    o.cap_entries = 0;
    o.local_set = MG_LOCAL_KSIGMA;
    o.grid_res = 0;
    o.block_radius = 5;
    o.grid_centre[0] = o.grid_centre[1] = o.grid_centre[2] = 0.f;
    o.grid_half = 0.f;
    return o;
}

const char *mg_version(void) { return "mgauss 0.1 (sm_103a)"; }

const char *mg_last_error(void) { return g_last_error.c_str(); }

const char *mg_status_string(mg_status s)
{
    switch (s) {
    case MG_OK: return "ok";
    case MG_ERR_INVALID_ARG: return "invalid argument";
    case MG_ERR_CUDA: return "CUDA error";
    case MG_ERR_CAPACITY: return "workspace capacity exceeded";
    case MG_ERR_DEVICE_TIMEOUT: return "device wait timed out";
    case MG_ERR_NOT_FINITE: return "non-finite or non-positive input";
    case MG_ERR_STALE_WORKSPACE: return "workspace does not hold the matching forward";
    }
    return "unknown status";
}

size_t mg_render_workspace_size(const mg_gaussians *g, const mg_stack *stacks, int n_stacks, const mg_opts *opts)
{
    std::string why;
    if (!valid_gauss(g, why, false)) return 0;
    std::vector<StackDesc> st = to_desc(stacks, n_stacks);
    if (!valid_stacks(st, false, why)) return 0;
    long long S = 0;
    for (const StackDesc &d : st) S += d.n_slices;
    mg_opts o = resolve_opts(opts, g->n, S);
    return make_layout(g->n, st, o).total;
}

mg_status mg_render_fwd(const mg_gaussians *g, const mg_stack *stacks, int n_stacks, const mg_opts *opts, float *out,
                        void *ws, size_t ws_bytes, mg_stream_t stream)
{
    std::vector<StackDesc> st = to_desc(stacks, n_stacks);
    if (st.empty()) return fail(MG_ERR_INVALID_ARG, "stacks is NULL or n_stacks not in [1, 32]");
    StackIn in = make_stack_in(st);
    return render_fwd_impl(g, st, in, opts, out, ws, ws_bytes, (cudaStream_t)stream);
}

mg_status mg_render_fwd_l1l2(const mg_gaussians *g, const mg_stack *stacks, int n_stacks, const mg_opts *opts,
                             const float *target, float *out, float *grad, double *loss_out, void *ws, size_t ws_bytes,
                             mg_stream_t stream)
{
    std::vector<StackDesc> st = to_desc(stacks, n_stacks);
    if (st.empty()) return fail(MG_ERR_INVALID_ARG, "stacks is NULL or n_stacks not in [1, 32]");
    if (!target || !loss_out) return fail(MG_ERR_INVALID_ARG, "mg_render_fwd_l1l2: target and loss_out are required");
    StackIn in = make_stack_in(st);
    return render_fwd_impl(g, st, in, opts, out, ws, ws_bytes, (cudaStream_t)stream, target, grad, loss_out);
}

mg_status mg_render_bwd(const mg_gaussians *g, const mg_stack *stacks, int n_stacks, const mg_opts *opts,
                        const float *grad_out, float *g_mean, float *g_quat, float *g_scale, float *g_alpha, void *ws,
                        size_t ws_bytes, mg_stream_t stream)
{
    std::string why;
    if (!valid_gauss(g, why)) return fail(MG_ERR_INVALID_ARG, why);
    std::vector<StackDesc> st = to_desc(stacks, n_stacks);
    if (!valid_stacks(st, true, why)) return fail(MG_ERR_INVALID_ARG, why);
    if (!grad_out || !ws) return fail(MG_ERR_INVALID_ARG, "grad_out or workspace is NULL");
    if (g->n > 0 && (!g_mean || !g_quat || !g_scale || !g_alpha))
        return fail(MG_ERR_INVALID_ARG, "a gradient output pointer is NULL");
    long long S = 0;
    for (const StackDesc &d : st) S += d.n_slices;
    mg_opts o = resolve_opts(opts, g->n, S);
    WsLayout L = make_layout(g->n, st, o);
    if (ws_bytes < L.total) return fail(MG_ERR_INVALID_ARG, "workspace too small");
    bool again = false;  // a backward already ran on this forward: its moments must be cleared
    {
        std::lock_guard<std::mutex> lk(g_tag_mu);
        auto it = g_tags.find(ws);
        if (it == g_tags.end() || !same_tag(it->second, make_tag(g, st, o)))
            return fail(MG_ERR_STALE_WORKSPACE, "mg_render_bwd: no matching mg_render_fwd on this workspace");
        again = it->second.bwd_done;
        it->second.bwd_done = true;
    }
    if (g->n == 0) return MG_OK;
    CellGrid cg;
    if (!make_cellgrid(o, max_pixel(st), cg, why)) return fail(MG_ERR_INVALID_ARG, why);
    char *w = (char *)ws;
    StackTable tab = make_table(st);
    mg_launch_render_bwd(L, w, (const SliceDev *)(w + L.slices), tab, cg, grad_out, g->mean, g->quat, g->scale,
                         g->alpha, g->n, o.f64_ratio, g_mean, g_quat, g_scale, g_alpha, again,
                         (cudaStream_t)stream);
    return check_cuda("mg_render_bwd");
}

mg_status mg_render_pose_grad(const mg_gaussians *g, const mg_stack *stacks, int n_stacks, const mg_opts *opts,
                              float *g_pose, void *ws, size_t ws_bytes, mg_stream_t stream)
{
    std::string why;
    if (!valid_gauss(g, why)) return fail(MG_ERR_INVALID_ARG, why);
    std::vector<StackDesc> st = to_desc(stacks, n_stacks);
    if (!valid_stacks(st, true, why)) return fail(MG_ERR_INVALID_ARG, why);
    if (!g_pose || !ws) return fail(MG_ERR_INVALID_ARG, "g_pose or workspace is NULL");
    long long S = 0;
    for (const StackDesc &d : st) S += d.n_slices;
    mg_opts o = resolve_opts(opts, g->n, S);
    WsLayout L = make_layout(g->n, st, o);
    if (ws_bytes < L.total) return fail(MG_ERR_INVALID_ARG, "workspace too small");
    {
        std::lock_guard<std::mutex> lk(g_tag_mu);
        auto it = g_tags.find(ws);
        if (it == g_tags.end() || !same_tag(it->second, make_tag(g, st, o)) || !it->second.bwd_done)
            return fail(MG_ERR_STALE_WORKSPACE,
                        "mg_render_pose_grad: no mg_render_bwd after the matching mg_render_fwd on this workspace");
    }
    cudaStream_t cs = (cudaStream_t)stream;
    if (g->n == 0) {
        cudaMemsetAsync(g_pose, 0, sizeof(float) * 6 * (size_t)S, cs);
        return check_cuda("mg_render_pose_grad");
    }
    char *w = (char *)ws;
    mg_launch_pose_grad(L, w, (const SliceDev *)(w + L.slices), g->mean, g->quat, g->scale, g->alpha, o.f64_ratio,
                        g_pose, cs);
    return check_cuda("mg_render_pose_grad");
}

static mg_status fill_layout(const WsLayout &L, mg_ws_layout *out)
{
    out->rec_gid = L.rec_gid;
    out->rec_slice = L.rec_slice;
    out->rec_rect = L.rec_rect;
    out->rec_inset = L.rec_inset;
    out->tile_off = L.tile_off;
    out->entries = L.entries;
    out->total_bytes = L.total;
    return MG_OK;
}

mg_status mg_render_ws_layout(const mg_gaussians *g, const mg_stack *stacks, int n_stacks, const mg_opts *opts,
                              mg_ws_layout *out)
{
    std::string why;
    if (!out || !valid_gauss(g, why, false)) return fail(MG_ERR_INVALID_ARG, out ? why : "out is NULL");
    std::vector<StackDesc> st = to_desc(stacks, n_stacks);
    if (!valid_stacks(st, false, why)) return fail(MG_ERR_INVALID_ARG, why);
    long long S = 0;
    for (const StackDesc &d : st) S += d.n_slices;
    return fill_layout(make_layout(g->n, st, resolve_opts(opts, g->n, S)), out);
}

mg_status mg_sample_ws_layout(int64_t n, int32_t G, const mg_opts *opts, mg_ws_layout *out)
{
    if (!out || n < 0 || G < 1 || G > 1024) return fail(MG_ERR_INVALID_ARG, "bad arguments");
    std::vector<StackDesc> st = {{G, G, G, 1.f, 1.f, 0.f, nullptr, 0.f, 0.f}};
    return fill_layout(make_layout(n, st, resolve_opts(opts, n, G)), out);
}

mg_status mg_render_stats_get(const void *ws, size_t ws_bytes, mg_render_stats *stats, mg_stream_t stream)
{
    if (!ws || !stats || ws_bytes < sizeof(WsHeader)) return fail(MG_ERR_INVALID_ARG, "bad workspace or stats");
    FwdTag tag;
    {
        std::lock_guard<std::mutex> lk(g_tag_mu);
        auto it = g_tags.find(ws);
        if (it == g_tags.end()) return fail(MG_ERR_STALE_WORKSPACE, "no forward recorded on this workspace");
        tag = it->second;
    }
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return check_cuda("mg_render_stats_get");
    WsHeader h;
    if (cudaMemcpy(&h, ws, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return check_cuda("mg_render_stats_get");
    memset(stats, 0, sizeof(*stats));
    stats->records = (int64_t)h.n_records;
    stats->entries = (int64_t)h.n_entries;
    long long tiles = 0;
    for (size_t s = 0; s < tag.stack_key.size() / 8; ++s) {
        long long ns = (long long)tag.stack_key[8 * s], H = (long long)tag.stack_key[8 * s + 1],
                  W = (long long)tag.stack_key[8 * s + 2];
        tiles += ns * ((W + MG_TILE - 1) / MG_TILE) * ((H + MG_TILE - 1) / MG_TILE);
    }
    stats->tiles = tiles;
    stats->cap_records = tag.capr;
    stats->cap_entries = tag.cape;
    mg_status st = MG_OK;
    if (h.flags & MG_FLAG_NOT_FINITE) st = MG_ERR_NOT_FINITE;
    if ((long long)h.n_records > tag.capr || (long long)h.n_entries > tag.cape || (h.flags & MG_FLAG_CAP_CHUNKS))
        st = MG_ERR_CAPACITY;
    stats->status = st;
    return st;
}

size_t mg_sample_workspace_size(int64_t n, int32_t G, const mg_opts *opts)
{
    if (n < 0 || G < 1 || G > 1024) return 0;
    std::vector<StackDesc> st = {{G, G, G, 1.f, 1.f, 0.f, nullptr, 0.f, 0.f}};
    mg_opts o = resolve_opts(opts, n, G);
    return make_layout(n, st, o).total;
}

mg_status mg_sample_volume(const mg_gaussians *g, const float centre[3], float spacing, int32_t G, const mg_opts *opts,
                           float *out, void *ws, size_t ws_bytes, mg_stream_t stream)
{
    if (!centre || !(spacing > 0.f) || !isfinite(spacing) || G < 1 || G > 1024)
        return fail(MG_ERR_INVALID_ARG, "need a centre, spacing > 0 and 1 <= G <= 1024");
    if (!isfinite(centre[0]) || !isfinite(centre[1]) || !isfinite(centre[2]))
        return fail(MG_ERR_INVALID_ARG, "centre must be finite");
    std::vector<StackDesc> st = {{G, G, G, spacing, spacing, 0.f, nullptr}};
    StackIn in = make_stack_in(st);
    in.planes = 1;
    in.cx = centre[0];
    in.cy = centre[1];
    in.cz = centre[2];
    in.h = spacing;
    return render_fwd_impl(g, st, in, opts, out, ws, ws_bytes, (cudaStream_t)stream);
}

size_t mg_reduce_workspace_size(int64_t n)
{
    if (n < 0) return 0;
    return align256(sizeof(double) * 2 * (size_t)mg_reduce_blocks(n));
}

mg_status mg_loss_l1l2(const float *pred, const float *target, int64_t n, float *grad, double *loss_out, void *ws,
                       size_t ws_bytes, mg_stream_t stream)
{
    if (n < 0 || (n > 0 && (!pred || !target)) || !loss_out || !ws)
        return fail(MG_ERR_INVALID_ARG, "bad pointer or size");
    if (ws_bytes < mg_reduce_workspace_size(n)) return fail(MG_ERR_INVALID_ARG, "workspace too small");
    {
        MG_PROF(MG_ST_LOSS, (cudaStream_t)stream);
        mg_launch_loss_l1l2(pred, target, n, grad, loss_out, (double *)ws, (cudaStream_t)stream);
    }
    return check_cuda("mg_loss_l1l2");
}

mg_status mg_render_pair_count(const mg_gaussians *g, const mg_stack *stacks, int n_stacks, const mg_opts *opts,
                               void *ws, size_t ws_bytes, int64_t counts[2], mg_stream_t stream)
{
    std::string why;
    if (!counts || !ws || !valid_gauss(g, why, false)) return fail(MG_ERR_INVALID_ARG, "bad arguments");
    std::vector<StackDesc> st = to_desc(stacks, n_stacks);
    if (!valid_stacks(st, false, why)) return fail(MG_ERR_INVALID_ARG, why);
    long long S = 0;
    for (const StackDesc &d : st) S += d.n_slices;
    mg_opts o = resolve_opts(opts, g->n, S);
    if (o.local_set != MG_LOCAL_KSIGMA) return fail(MG_ERR_INVALID_ARG, "pair counts are for MG_LOCAL_KSIGMA only");
    WsLayout L = make_layout(g->n, st, o);
    if (ws_bytes < L.total) return fail(MG_ERR_INVALID_ARG, "workspace too small");
    {
        std::lock_guard<std::mutex> lk(g_tag_mu);
        if (g_tags.find(ws) == g_tags.end()) return fail(MG_ERR_STALE_WORKSPACE, "no forward on this workspace");
    }
    mg_launch_pair_count(L, (char *)ws, make_table(st), (cudaStream_t)stream);
    mg_status s = check_cuda("mg_render_pair_count");
    if (s != MG_OK) return s;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return check_cuda("mg_render_pair_count");
    WsHeader h;
    if (cudaMemcpy(&h, ws, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
        return check_cuda("mg_render_pair_count");
    counts[0] = (int64_t)h.pairs_inside;
    counts[1] = (int64_t)h.pairs_evaluated;
    return MG_OK;
}

int64_t mg_nrf_param_count(int32_t encoding) { return mg_nrf_param_count_impl(encoding); }
size_t mg_nrf_enc_bytes(const mg_nrf *net, int64_t n) { return mg_nrf_enc_bytes_impl(net, n); }

static bool valid_nrf(const mg_nrf *net, std::string &why)
{
    if (!net) {
        why = "net is NULL";
        return false;
    }
    if (net->encoding != MG_NRF_FOURIER && net->encoding != MG_NRF_GRID) {
        why = "unknown encoding";
        return false;
    }
    if (net->precision != MG_NRF_BF16 && net->precision != MG_NRF_FP32) {
        why = "unknown precision";
        return false;
    }
    if (!net->params) {
        why = "params is NULL";
        return false;
    }
    if (net->encoding == MG_NRF_GRID) {
        if (!net->table) {
            why = "grid encoding needs a table";
            return false;
        }
        if ((uintptr_t)net->table & 7u) {
            why = "the grid table must be 8-byte aligned";
            return false;
        }
        if (net->log2_table < 0 || net->log2_table > 24 || net->n_min < 0 || net->n_max < 0 ||
            (net->n_min > 0 && net->n_max > 0 && net->n_max < net->n_min)) {
            why = "bad grid geometry";
            return false;
        }
    }
    if (!(net->out_scale > 0.f) || !isfinite(net->out_scale)) {
        why = "out_scale must be positive";
        return false;
    }
    if (net->enc_mode != MG_NRF_ENC_NONE && net->enc_mode != MG_NRF_ENC_STORE && net->enc_mode != MG_NRF_ENC_LOAD) {
        why = "unknown enc_mode";
        return false;
    }
    if (net->encoding == MG_NRF_GRID && net->enc_mode != MG_NRF_ENC_NONE && !net->enc) {
        why = "enc_mode needs an encoding cache";
        return false;
    }
    return true;
}

mg_status mg_nrf_fwd(const mg_nrf *net, const float *xyz, int64_t n, float *out, mg_stream_t stream)
{
    std::string why;
    if (!valid_nrf(net, why)) return fail(MG_ERR_INVALID_ARG, why);
    if (n < 0 || (n > 0 && (!xyz || !out))) return fail(MG_ERR_INVALID_ARG, "bad xyz/out or n");
    if (n == 0) return MG_OK;
    MG_PROF(MG_ST_NRF_FWD, (cudaStream_t)stream);
    cudaError_t e = mg_launch_nrf(net, xyz, n, nullptr, out, nullptr, nullptr, false, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("mg_nrf_fwd: ") + cudaGetErrorString(e));
    return MG_OK;
}

mg_status mg_nrf_bwd(const mg_nrf *net, const float *xyz, int64_t n, const float *grad_out, float *g_params,
                     float *g_table, mg_stream_t stream)
{
    std::string why;
    if (!valid_nrf(net, why)) return fail(MG_ERR_INVALID_ARG, why);
    if (n < 0 || (n > 0 && (!xyz || !grad_out)) || !g_params) return fail(MG_ERR_INVALID_ARG, "bad pointers or n");
    if (net->encoding == MG_NRF_GRID && (!g_table || ((uintptr_t)g_table & 15u)))
        return fail(MG_ERR_INVALID_ARG, "grid encoding needs a 16-byte aligned g_table");
    cudaStream_t st = (cudaStream_t)stream;
    MG_PROF(MG_ST_NRF_BWD, st);
    cudaMemsetAsync(g_params, 0, sizeof(float) * (size_t)mg_nrf_param_count_impl(net->encoding), st);
    if (net->encoding == MG_NRF_GRID) {
        int lt = net->log2_table > 0 ? net->log2_table : 19;
        cudaMemsetAsync(g_table, 0, sizeof(float) * 2 * 16 * ((size_t)1 << lt), st);
    }
    if (n > 0) {
        cudaError_t e = mg_launch_nrf(net, xyz, n, grad_out, nullptr, g_params, g_table, true, st);
        if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("mg_nrf_bwd: ") + cudaGetErrorString(e));
    }
    return check_cuda("mg_nrf_bwd");
}

mg_status mg_nrf_fwd_at(const mg_nrf *net, const float *coords, int64_t rows, const int64_t *idx, int64_t n,
                        float *acc, mg_stream_t stream)
{
    std::string why;
    if (!valid_nrf(net, why)) return fail(MG_ERR_INVALID_ARG, why);
    if (n < 0 || rows < 0 || (n > 0 && (!coords || !idx || !acc)))
        return fail(MG_ERR_INVALID_ARG, "bad coords/idx/acc, rows or n");
    if (n == 0) return MG_OK;
    MG_PROF(MG_ST_NRF_FWD, (cudaStream_t)stream);
    cudaError_t e = mg_launch_nrf(net, coords, n, nullptr, acc, nullptr, nullptr, false, (cudaStream_t)stream,
                                  (const long long *)idx, rows);
    if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("mg_nrf_fwd_at: ") + cudaGetErrorString(e));
    return MG_OK;
}

mg_status mg_nrf_bwd_at(const mg_nrf *net, const float *coords, int64_t rows, const int64_t *idx, int64_t n,
                        const float *grad_acc, float *g_params, float *g_table, mg_stream_t stream)
{
    std::string why;
    if (!valid_nrf(net, why)) return fail(MG_ERR_INVALID_ARG, why);
    if (n < 0 || rows < 0 || (n > 0 && (!coords || !idx || !grad_acc)) || !g_params)
        return fail(MG_ERR_INVALID_ARG, "bad pointers or n");
    if (net->encoding == MG_NRF_GRID && (!g_table || ((uintptr_t)g_table & 15u)))
        return fail(MG_ERR_INVALID_ARG, "grid encoding needs a 16-byte aligned g_table");
    cudaStream_t st = (cudaStream_t)stream;
    MG_PROF(MG_ST_NRF_BWD, st);
    cudaMemsetAsync(g_params, 0, sizeof(float) * (size_t)mg_nrf_param_count_impl(net->encoding), st);
    if (net->encoding == MG_NRF_GRID) {
        int lt = net->log2_table > 0 ? net->log2_table : 19;
        cudaMemsetAsync(g_table, 0, sizeof(float) * 2 * 16 * ((size_t)1 << lt), st);
    }
    if (n > 0) {
        cudaError_t e = mg_launch_nrf(net, coords, n, grad_acc, nullptr, g_params, g_table, true, st,
                                      (const long long *)idx, rows);
        if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("mg_nrf_bwd_at: ") + cudaGetErrorString(e));
    }
    return check_cuda("mg_nrf_bwd_at");
}

mg_status mg_profile_enable(int on)
{
    prof::on.store(on != 0 ? (MG_NSTAGES >= 32 ? 0xffffffffu : (1u << MG_NSTAGES) - 1u) : 0u);
    return MG_OK;
}

mg_status mg_profile_stages(uint32_t mask)
{
    prof::on.store(mask & (MG_NSTAGES >= 32 ? 0xffffffffu : (1u << MG_NSTAGES) - 1u));
    return MG_OK;
}

int mg_profile_stage_count(void) { return MG_NSTAGES; }

const char *mg_profile_stage_name(int stage)
{
    return (stage >= 0 && stage < MG_NSTAGES) ? prof::names[stage] : "";
}

mg_status mg_profile_read(double *ms, int64_t *calls, int reset)
{
    std::vector<prof::Pending> todo;
    {
        std::lock_guard<std::mutex> lk(prof::mu);
        todo.swap(prof::pending);
    }
    for (const prof::Pending &p : todo) {
        float f = 0.f;
        if (cudaEventSynchronize(p.b) != cudaSuccess) return check_cuda("mg_profile_read");
        cudaEventElapsedTime(&f, p.a, p.b);
        std::lock_guard<std::mutex> lk(prof::mu);
        prof::ms[p.stage] += f;
        prof::calls[p.stage] += 1;
        prof::pool.push_back(p.a);
        prof::pool.push_back(p.b);
    }
    std::lock_guard<std::mutex> lk(prof::mu);
    for (int i = 0; i < MG_NSTAGES; ++i) {
        if (ms) ms[i] = prof::ms[i];
        if (calls) calls[i] = prof::calls[i];
        if (reset) {
            prof::ms[i] = 0.0;
            prof::calls[i] = 0;
        }
    }
    return check_cuda("mg_profile_read");
}

mg_status mg_sq_diff_sum(const float *a, const float *b, int64_t n, double *out, void *ws, size_t ws_bytes,
                         mg_stream_t stream)
{
    if (n < 0 || (n > 0 && (!a || !b)) || !out || !ws) return fail(MG_ERR_INVALID_ARG, "bad pointer or size");
    if (ws_bytes < mg_reduce_workspace_size(n)) return fail(MG_ERR_INVALID_ARG, "workspace too small");
    mg_launch_sq_diff(a, b, n, out, (double *)ws, (cudaStream_t)stream);
    return check_cuda("mg_sq_diff_sum");
}

}  // extern "C"
