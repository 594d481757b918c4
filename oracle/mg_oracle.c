/*
 * mg_oracle.c -- CPU reference ("oracle") for the Magnetic Gaussian slice
 * renderer.
 *
 * TEST INFRASTRUCTURE ONLY. It is called by the tests, by the smoke check and
 * by the benchmark's CPU-baseline leg, never by the product path. It shares no
 * code, header or constant table with the CUDA library; both sides implement
 * the same written definitions.
 *
 * Plain loops, FP64 evaluation, no blocking or fusion, so that it can be read
 * against the paper:
 *
 *   Sec. 3.2, Eq. E3:  Sigma = R S S^T R^T, R from the unit quaternion,
 *                      S = diag(scale) (scale = exp(s), taken as input).
 *   Sec. 3.3.2, E7:    I(x) = sum_i alpha_i exp(-1/2 (x-mu_i)^T Sigma_i^-1 (x-mu_i)),
 *                      an additive mixture, no compositing and no sort.
 *   Slice profile:     a slice voxel integrates I along the slice normal n
 *                      against a unit-integral Gaussian profile of variance
 *                      sig2 = FWHM^2 / (8 ln 2). Convolving a Gaussian with a
 *                      Gaussian adds covariances, so each term becomes
 *                      alpha sqrt(|Sigma| / |Sigma'|) exp(-1/2 y^T Sigma'^-1 y),
 *                      Sigma' = Sigma + sig2 n n^T, y = x - mu. With sig2 = 0
 *                      this is E7 exactly.
 *   In-plane PSF:      a stack may add a Gaussian PSF of FWHM pu, pv along the
 *                      slice axes e_u, e_v (the paper models none): then
 *                      Sigma' = Sigma + R_k diag(pu^2, pv^2, th^2) R_k^T / (8 ln 2)
 *                      with the same form of the term.
 *   Truncation:        the paper already restricts the sum to a local set
 *                      G_local (Sec. 3.3.1). Here the local set of a slice
 *                      voxel is the set of Gaussians whose record for that
 *                      slice lists the voxel's 8x8 tile (record predicate
 *                      below, K-sigma ellipsoid of Sigma').
 *
 * Record predicate (evaluated in FP32, IEEE round-to-nearest, every operation
 * rounded, no fused multiply-add, in the order written; compile with
 * -ffp-contract=off). For Gaussian (mu, q=(w,x,y,z), s) and slice (Q, t):
 *   R    = standard rotation of q (entries as in quat_rot_f below)
 *   M    = R diag(s);  Sigma_rc = (M_r0 M_c0 + M_r1 M_c1) + M_r2 M_c2
 *   p    = mu - t;  e_u, e_v, e_n = columns of Q;  a.b = (a0 b0 + a1 b1) + a2 b2
 *   w0 = (e_n.mu) - (e_n.t), u0 = e_u.p, v0 = e_v.p
 *   Lww = e_n.(Sigma e_n), Luw = e_u.(Sigma e_n), Lvw = e_v.(Sigma e_n),
 *   Luu = e_u.(Sigma e_u), Lvv = e_v.(Sigma e_v), (Sigma a)_r = (S_r0 a0 + S_r1 a1) + S_r2 a2
 *   Sww = Lww + sig2;  K2 = K*K
 *   the record exists iff  w0*w0 <= K2*Sww  (the K-sigma slab test)
 *   iSww = 1/Sww;  r2 = max(K2 - (w0*w0)*iSww, 0)
 *   Cuu = max(Luu - (Luw*Luw)*iSww, 0) + pu2,  Cvv = max(Lvv - (Lvw*Lvw)*iSww, 0) + pv2
 *   cu = u0 - (Luw*w0)*iSww,  cv = v0 - (Lvw*w0)*iSww
 *   ru = sqrt(r2*Cuu),  rv = sqrt(r2*Cvv)
 *   idx = 1/dx, idy = 1/dy
 *   il = ceil((cu-ru)*idx + hx), ih = floor((cu+ru)*idx + hx), hx = 0.5*(W-1)
 *   jl = ceil((cv-rv)*idy + hy), jh = floor((cv+rv)*idy + hy), hy = 0.5*(H-1)
 *   the pixel box is empty unless il<=ih, jl<=jh, il<=W-1, ih>=0, jl<=H-1,
 *   jh>=0 (false for NaN); a non-empty box has il,jl clamped up to 0 and ih,jh
 *   down to W-1,H-1 and lists the tiles [il/8, ih/8] x [jl/8, jh/8]
 *   (integer division); an empty box lists none (rectangle (1,1,0,0))
 *   sig2 = (float)(thickness^2 * 0.18033688011112042) computed in double,
 *   pu2, pv2 likewise from the in-plane PSF FWHM (0 without a PSF).
 * (u,v) bounds of the ellipse {y : y^T Sigma'^-1 y <= K^2} cut by the plane
 * w = 0 are cu +- ru, cv +- rv: the in-plane conditional covariance of Sigma'
 * is C = Sigma'_uv - Sigma'_uv,w Sigma'_w,uv / Sww and the cut ellipse has
 * "radius^2" r2 = K^2 - w0^2/Sww.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_TILE 8
#define OR_FWHM2VAR 0.18033688011112042 /* 1 / (8 ln 2) */

/* ------------------------------------------------------------------ */
/* per-slice table built from the stack descriptors                   */
/* ------------------------------------------------------------------ */
typedef struct {
    int H, W, TX, TY;
    float dx, dy, thk, pu, pv; /* pu, pv: in-plane PSF FWHM along e_u, e_v (0 = none) */
    const float *xf;   /* 12 floats: Q row-major, then t (record predicate) */
    double dxd, dyd, thkd, pud, pvd;
    const double *xfd; /* the same in FP64 (evaluation) */
    int64_t out_base;  /* offset of this slice's [H,W] image in the output */
} or_slice;

static or_slice *or_build_slices(int n_stacks, const int32_t *nsl, const int32_t *H, const int32_t *W,
                                 const float *dx, const float *dy, const float *thk, const float *psf,
                                 const float *xform, const double *dxd, const double *dyd, const double *thkd,
                                 const double *psfd, const double *xformd,
                                 int *S_out)
{
    int S = 0;
    for (int s = 0; s < n_stacks; ++s) S += nsl[s];
    or_slice *sl = (or_slice *)calloc((size_t)(S > 0 ? S : 1), sizeof(or_slice));
    int k = 0;
    int64_t base = 0;
    for (int s = 0; s < n_stacks; ++s) {
        for (int j = 0; j < nsl[s]; ++j, ++k) {
            sl[k].H = H[s];
            sl[k].W = W[s];
            sl[k].TX = (W[s] + OR_TILE - 1) / OR_TILE;
            sl[k].TY = (H[s] + OR_TILE - 1) / OR_TILE;
            if (xform) {
                sl[k].dx = dx[s];
                sl[k].dy = dy[s];
                sl[k].thk = thk[s];
                sl[k].pu = psf[2 * s];
                sl[k].pv = psf[2 * s + 1];
                sl[k].xf = xform + (size_t)k * 12;
            }
            if (xformd) {
                sl[k].dxd = dxd[s];
                sl[k].dyd = dyd[s];
                sl[k].thkd = thkd[s];
                sl[k].pud = psfd[2 * s];
                sl[k].pvd = psfd[2 * s + 1];
                sl[k].xfd = xformd + (size_t)k * 12;
            }
            sl[k].out_base = base;
            base += (int64_t)H[s] * W[s];
        }
    }
    *S_out = S;
    return sl;
}

/* ------------------------------------------------------------------ */
/* FP32 record predicate (the written specification above)             */
/* ------------------------------------------------------------------ */
static void quat_rot_f(const float *q, float R[3][3])
{
    float w = q[0], x = q[1], y = q[2], z = q[3];
    float xx = x * x, yy = y * y, zz = z * z;
    float xy = x * y, xz = x * z, yz = y * z;
    float wx = w * x, wy = w * y, wz = w * z;
    R[0][0] = 1.0f - 2.0f * (yy + zz);
    R[0][1] = 2.0f * (xy - wz);
    R[0][2] = 2.0f * (xz + wy);
    R[1][0] = 2.0f * (xy + wz);
    R[1][1] = 1.0f - 2.0f * (xx + zz);
    R[1][2] = 2.0f * (yz - wx);
    R[2][0] = 2.0f * (xz - wy);
    R[2][1] = 2.0f * (yz + wx);
    R[2][2] = 1.0f - 2.0f * (xx + yy);
}

static float dot3f(const float a[3], const float b[3])
{
    float t = a[0] * b[0] + a[1] * b[1];
    return t + a[2] * b[2];
}

/* Row culling of a record's tile rectangle (FP32, each operation rounded, as
 * the record predicate): for each of the first eight tile rows, the tile
 * columns that the cut ellipse {(u,v): (u-cu, v-cv) C^-1 (u-cu, v-cv)^T <= r2}
 * reaches over the row's pixel band v in [va, vb]. The band's leftmost ellipse
 * point is the ellipse's own leftmost point (cu - ru at v = cv - Cuv ru/Cuu,
 * ru = sqrt(r2 Cuu)) when that v lies in the band; otherwise, the left boundary
 * being convex in v, it lies on the band edge nearest to it, where the chord of
 * the ellipse is centred at cu + (Cuv/Cvv) d with half-width
 * sqrt((r2 - d^2/Cvv)(Cuu - Cuv^2/Cvv)), d = v - cv; the right side mirrors
 * this. A rectangle one tile wide is not culled. The extents grow by
 * ru/256 + dx/1024 so that FP32 rounding never drops a tile that holds a voxel
 * of the ellipse. Returned as 8 bits per row: the tile-column insets from the
 * rectangle's left (low 4 bits) and right edges, each at most 15. */
static uint64_t row_insets(const or_slice *sl, float cu, float cv, float Cuu, float Cvv, float Cuv, float r2,
                           float ru, float il, float ih, float jl, float jh)
{
    int tx0 = (int32_t)il / OR_TILE, tx1 = (int32_t)ih / OR_TILE;
    int ty0 = (int32_t)jl / OR_TILE, ty1 = (int32_t)jh / OR_TILE;
    if (!(r2 > 0.0f) || !(Cuu > 0.0f) || !(Cvv > 0.0f) || tx1 == tx0) return 0;
    float hx = 0.5f * (float)(sl->W - 1), hy = 0.5f * (float)(sl->H - 1);
    float idx = 1.0f / sl->dx;
    float e = ru / Cuu;
    float iCvv = 1.0f / Cvv;
    float g = Cuv * iCvv;
    float h2 = Cuu - Cuv * g;
    if (h2 < 0.0f) h2 = 0.0f;
    float m = ru * 0.00390625f + sl->dx * 0.0009765625f;
    float vL = cv - Cuv * e, vR = cv + Cuv * e;
    uint64_t out = 0;
    int last = ty1 - ty0 < 7 ? ty1 - ty0 : 7;
    for (int n = 0; n <= last; ++n) {
        int ty = ty0 + n;
        int a = (int)jl > OR_TILE * ty ? (int)jl : OR_TILE * ty;
        int b = (int)jh < OR_TILE * ty + OR_TILE - 1 ? (int)jh : OR_TILE * ty + OR_TILE - 1;
        float va = ((float)a - hy) * sl->dy, vb = ((float)b - hy) * sl->dy;
        float left, right;
        float v = fminf(fmaxf(vL, va), vb);
        if (v == vL) {
            left = cu - ru;
        } else {
            float d = v - cv;
            float t = r2 - (d * d) * iCvv;
            if (t < 0.0f) t = 0.0f;
            left = (cu + g * d) - sqrtf(t * h2);
        }
        v = fminf(fmaxf(vR, va), vb);
        if (v == vR) {
            right = cu + ru;
        } else {
            float d = v - cv;
            float t = r2 - (d * d) * iCvv;
            if (t < 0.0f) t = 0.0f;
            right = (cu + g * d) + sqrtf(t * h2);
        }
        float lo = fmaxf(ceilf((left - m) * idx + hx), il);
        float hi = fminf(floorf((right + m) * idx + hx), ih);
        int l, r;
        if (!(lo <= hi)) { /* no voxel column in this band: the row lists nothing */
            l = tx1 - tx0 + 1;
            r = 0;
        } else {
            l = (int32_t)lo / OR_TILE - tx0;
            r = tx1 - (int32_t)hi / OR_TILE;
        }
        if (l > 15) l = 15;
        if (r > 15) r = 15;
        out |= (uint64_t)(l | (r << 4)) << (8 * n);
    }
    return out;
}

/* The pixel columns [*i0, *i1) that record r lists in pixel row j: its
 * rectangle's tiles, narrowed by the row insets (NULL: none). */
static void listed_cols(const int32_t *rc, const uint64_t *rec_inset, int64_t r, int j, int W, int *i0, int *i1)
{
    int n = j / OR_TILE - rc[1];
    int bits = (rec_inset && n < 8) ? (int)((rec_inset[r] >> (8 * n)) & 0xFF) : 0;
    *i0 = (rc[0] + (bits & 15)) * OR_TILE;
    *i1 = (rc[2] - (bits >> 4) + 1) * OR_TILE;
    if (*i1 > W) *i1 = W;
}

/* returns 1 and the tile rectangle (and the row insets, if asked) if the
 * (Gaussian, slice) record exists */
static int record_predicate(const float *mu, const float *q, const float *s, const or_slice *sl, float K,
                            int32_t rect[4], uint64_t *inset)
{
    float R[3][3], M[3][3], Sg[3][3];
    quat_rot_f(q, R);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M[r][c] = R[r][c] * s[c];
    for (int r = 0; r < 3; ++r)
        for (int c = r; c < 3; ++c) {
            float t = M[r][0] * M[c][0] + M[r][1] * M[c][1];
            Sg[r][c] = t + M[r][2] * M[c][2];
            Sg[c][r] = Sg[r][c];
        }
    const float *Q = sl->xf;
    float eu[3] = {Q[0], Q[3], Q[6]};
    float ev[3] = {Q[1], Q[4], Q[7]};
    float en[3] = {Q[2], Q[5], Q[8]};
    float p[3] = {mu[0] - Q[9], mu[1] - Q[10], mu[2] - Q[11]};
    float wm = dot3f(en, mu), wt = dot3f(en, &Q[9]);
    float w0 = wm - wt, u0 = dot3f(eu, p), v0 = dot3f(ev, p);
    float sn[3], su[3], sv[3];
    for (int r = 0; r < 3; ++r) {
        sn[r] = dot3f(Sg[r], en);
        su[r] = dot3f(Sg[r], eu);
        sv[r] = dot3f(Sg[r], ev);
    }
    float Lww = dot3f(en, sn), Luw = dot3f(eu, sn), Lvw = dot3f(ev, sn);
    float Luu = dot3f(eu, su), Lvv = dot3f(ev, sv), Luv = dot3f(ev, su);
    float sig2 = (float)((double)sl->thk * (double)sl->thk * OR_FWHM2VAR);
    float Sww = Lww + sig2;
    float K2 = K * K;
    float ww = w0 * w0;
    if (!(ww <= K2 * Sww)) return 0;
    float iSww = 1.0f / Sww;
    float r2 = K2 - ww * iSww;
    if (r2 < 0.0f) r2 = 0.0f;
    float pu2 = (float)((double)sl->pu * (double)sl->pu * OR_FWHM2VAR);
    float pv2 = (float)((double)sl->pv * (double)sl->pv * OR_FWHM2VAR);
    float Cuu = Luu - (Luw * Luw) * iSww;
    if (Cuu < 0.0f) Cuu = 0.0f;
    Cuu = Cuu + pu2;
    float Cvv = Lvv - (Lvw * Lvw) * iSww;
    if (Cvv < 0.0f) Cvv = 0.0f;
    Cvv = Cvv + pv2;
    float cu = u0 - (Luw * w0) * iSww;
    float cv = v0 - (Lvw * w0) * iSww;
    float ru = sqrtf(r2 * Cuu), rv = sqrtf(r2 * Cvv);
    float hx = 0.5f * (float)(sl->W - 1), hy = 0.5f * (float)(sl->H - 1);
    float idx = 1.0f / sl->dx, idy = 1.0f / sl->dy;
    float il = ceilf((cu - ru) * idx + hx);
    float ih = floorf((cu + ru) * idx + hx);
    float jl = ceilf((cv - rv) * idy + hy);
    float jh = floorf((cv + rv) * idy + hy);
    float Wm1 = (float)(sl->W - 1), Hm1 = (float)(sl->H - 1);
    if (inset) *inset = 0;
    if (!(il <= ih) || !(jl <= jh) || !(il <= Wm1) || !(ih >= 0.0f) || !(jl <= Hm1) || !(jh >= 0.0f)) {
        rect[0] = 1; rect[1] = 1; rect[2] = 0; rect[3] = 0; /* record without tiles */
        return 1;
    }
    if (il < 0.0f) il = 0.0f;
    if (jl < 0.0f) jl = 0.0f;
    if (ih > Wm1) ih = Wm1;
    if (jh > Hm1) jh = Hm1;
    rect[0] = (int32_t)il / OR_TILE;
    rect[1] = (int32_t)jl / OR_TILE;
    rect[2] = (int32_t)ih / OR_TILE;
    rect[3] = (int32_t)jh / OR_TILE;
    /* rows are culled for Gaussians with max scale <= 64 min scale only: beyond
     * that, FP32 cancellation in the conditional covariance can exceed the margin */
    float smax = fmaxf(fmaxf(s[0], s[1]), s[2]), smin = fminf(fminf(s[0], s[1]), s[2]);
    if (inset && smax <= 64.0f * smin) {
        float Cuv = Luv - (Luw * Lvw) * iSww;
        *inset = row_insets(sl, cu, cv, Cuu, Cvv, Cuv, r2, ru, il, ih, jl, jh);
    }
    return 1;
}

/* ------------------------------------------------------------------ */
/* The paper's cell-grid local set (Sec. 3.3.1, Eqs. E4-E6), FP32 in  */
/* the written order: the cube [-1,1]^3 mapped to centre + h [-1,1]^3 */
/* mm is cut into res^3 cells; a Gaussian belongs to the cell of its  */
/* mean; the local set of voxel x is every Gaussian whose cell is     */
/* within R cells of x's cell along each axis.                        */
/* ------------------------------------------------------------------ */
typedef struct {
    int res, R;
    float C[3], h, hres, e, m;
} or_cells;

static void cells_setup(const int32_t *ci, const float *cf, or_cells *c)
{
    c->res = ci[0];
    c->R = ci[1];
    c->C[0] = cf[0];
    c->C[1] = cf[1];
    c->C[2] = cf[2];
    c->h = cf[3];
    double hres = 0.5 * (double)c->res, h = (double)c->h;
    c->hres = (float)hres;
    c->e = (float)(h * ((double)c->R + 0.5) / hres);  /* half-width of the member box */
    c->m = (float)(h / (1024.0 * hres));             /* margin of the record tests */
}

/* cell index of one coordinate: floor(((p - C)/h + 1) hres), clamped to +-2^20 */
static int cell_coord_f(float p, float c, float h, float hres)
{
    float t = (p - c) / h;
    t = t + 1.0f;
    t = t * hres;
    if (!(t >= -1048576.0f)) t = -1048576.0f;
    if (t > 1048576.0f) t = 1048576.0f;
    return (int)floorf(t);
}

static void gauss_cell_f(const float mu[3], const or_cells *c, int cell[3], float b[3])
{
    for (int a = 0; a < 3; ++a) {
        cell[a] = cell_coord_f(mu[a], c->C[a], c->h, c->hres);
        float t = ((float)cell[a] + 0.5f) / c->hres;
        t = t - 1.0f;
        b[a] = c->C[a] + c->h * t; /* centre of the member box */
    }
}

/* FP32 world position of voxel (i, j) of a slice and its cell */
static void voxel_cell_f(const or_slice *sl, int i, int j, const or_cells *c, int cell[3])
{
    float hx = 0.5f * (float)(sl->W - 1), hy = 0.5f * (float)(sl->H - 1);
    float dx = (float)sl->dxd, dy = (float)sl->dyd;
    float u = ((float)i - hx) * dx, v = ((float)j - hy) * dy;
    for (int a = 0; a < 3; ++a) {
        float q0 = (float)sl->xfd[3 * a], q1 = (float)sl->xfd[3 * a + 1], t = (float)sl->xfd[9 + a];
        float x = q0 * u + q1 * v;
        x = x + t;
        cell[a] = cell_coord_f(x, c->C[a], c->h, c->hres);
    }
}

static int cell_member(const int vc[3], const int gc[3], int R)
{
    for (int a = 0; a < 3; ++a)
        if (abs(vc[a] - gc[a]) > R) return 0;
    return 1;
}

static float abs_sum3f(float a, float b, float c)
{
    float t = fabsf(a) + fabsf(b);
    return t + fabsf(c);
}

/* Record test of the cell rule: the slice plane passes within m of the
 * Gaussian's member box; the tiles cover the box's extent along e_u, e_v. */
static int record_predicate_cells(const float *mu, const or_slice *sl, const or_cells *c, int32_t rect[4])
{
    int gc[3];
    float b[3];
    gauss_cell_f(mu, c, gc, b);
    const float *Q = sl->xf;
    float eu[3] = {Q[0], Q[3], Q[6]};
    float ev[3] = {Q[1], Q[4], Q[7]};
    float en[3] = {Q[2], Q[5], Q[8]};
    float p[3] = {b[0] - Q[9], b[1] - Q[10], b[2] - Q[11]};
    float w = dot3f(en, p);
    if (!(fabsf(w) <= c->e * abs_sum3f(en[0], en[1], en[2]) + c->m)) return 0;
    float uc = dot3f(eu, p), vc = dot3f(ev, p);
    float ru = c->e * abs_sum3f(eu[0], eu[1], eu[2]) + c->m;
    float rv = c->e * abs_sum3f(ev[0], ev[1], ev[2]) + c->m;
    float hx = 0.5f * (float)(sl->W - 1), hy = 0.5f * (float)(sl->H - 1);
    float idx = 1.0f / sl->dx, idy = 1.0f / sl->dy;
    float il = ceilf((uc - ru) * idx + hx);
    float ih = floorf((uc + ru) * idx + hx);
    float jl = ceilf((vc - rv) * idy + hy);
    float jh = floorf((vc + rv) * idy + hy);
    float Wm1 = (float)(sl->W - 1), Hm1 = (float)(sl->H - 1);
    if (!(il <= ih) || !(jl <= jh) || !(il <= Wm1) || !(ih >= 0.0f) || !(jl <= Hm1) || !(jh >= 0.0f)) {
        rect[0] = 1; rect[1] = 1; rect[2] = 0; rect[3] = 0;
        return 1;
    }
    if (il < 0.0f) il = 0.0f;
    if (jl < 0.0f) jl = 0.0f;
    if (ih > Wm1) ih = Wm1;
    if (jh > Hm1) jh = Hm1;
    rect[0] = (int32_t)il / OR_TILE;
    rect[1] = (int32_t)jl / OR_TILE;
    rect[2] = (int32_t)ih / OR_TILE;
    rect[3] = (int32_t)jh / OR_TILE;
    return 1;
}

int64_t or_make_records_cells(int64_t n, const float *mean, int n_stacks, const int32_t *nsl, const int32_t *H,
                              const int32_t *W, const float *dx, const float *dy, const float *thk, const float *psf,
                              const float *xform, const int32_t *cells_i, const float *cells_f, int64_t cap,
                              int32_t *rec_slice, int32_t *rec_gid, int32_t *rec_rect)
{
    int S;
    or_slice *sl = or_build_slices(n_stacks, nsl, H, W, dx, dy, thk, psf, xform, NULL, NULL, NULL, NULL, NULL, &S);
    or_cells c;
    cells_setup(cells_i, cells_f, &c);
    int64_t *cnt = (int64_t *)calloc((size_t)S + 1, sizeof(int64_t));
#pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < S; ++k) {
        int64_t m = 0;
        int32_t rect[4];
        for (int64_t g = 0; g < n; ++g) m += record_predicate_cells(mean + 3 * g, &sl[k], &c, rect);
        cnt[k + 1] = m;
    }
    for (int k = 0; k < S; ++k) cnt[k + 1] += cnt[k];
    int64_t total = cnt[S];
    if (rec_slice && cap > 0) {
#pragma omp parallel for schedule(dynamic)
        for (int k = 0; k < S; ++k) {
            int64_t pos = cnt[k];
            int32_t rect[4];
            for (int64_t g = 0; g < n && pos < cap; ++g) {
                if (record_predicate_cells(mean + 3 * g, &sl[k], &c, rect)) {
                    rec_slice[pos] = k;
                    rec_gid[pos] = (int32_t)g;
                    memcpy(rec_rect + 4 * pos, rect, sizeof(rect));
                    ++pos;
                }
            }
        }
    }
    free(cnt);
    free(sl);
    return total;
}

/* Records, slice-major (all stacks' slices in order), ascending Gaussian id
 * within a slice. Returns the total; fills at most cap. */
int64_t or_make_records(int64_t n, const float *mean, const float *quat, const float *scale, int n_stacks,
                        const int32_t *nsl, const int32_t *H, const int32_t *W, const float *dx, const float *dy,
                        const float *thk, const float *psf, const float *xform, float K, int64_t cap,
                        int32_t *rec_slice,
                        int32_t *rec_gid, int32_t *rec_rect, uint64_t *rec_inset)
{
    int S;
    or_slice *sl = or_build_slices(n_stacks, nsl, H, W, dx, dy, thk, psf, xform, NULL, NULL, NULL, NULL, NULL, &S);
    int64_t *cnt = (int64_t *)calloc((size_t)S + 1, sizeof(int64_t));
#pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < S; ++k) {
        int64_t c = 0;
        int32_t rect[4];
        for (int64_t g = 0; g < n; ++g)
            c += record_predicate(mean + 3 * g, quat + 4 * g, scale + 3 * g, &sl[k], K, rect, NULL);
        cnt[k + 1] = c;
    }
    for (int k = 0; k < S; ++k) cnt[k + 1] += cnt[k];
    int64_t total = cnt[S];
    if (rec_slice && cap > 0) {
#pragma omp parallel for schedule(dynamic)
        for (int k = 0; k < S; ++k) {
            int64_t pos = cnt[k];
            int32_t rect[4];
            for (int64_t g = 0; g < n && pos < cap; ++g) {
                uint64_t ins;
                if (record_predicate(mean + 3 * g, quat + 4 * g, scale + 3 * g, &sl[k], K, rect, &ins)) {
                    rec_slice[pos] = k;
                    rec_gid[pos] = (int32_t)g;
                    memcpy(rec_rect + 4 * pos, rect, sizeof(rect));
                    if (rec_inset) rec_inset[pos] = ins;
                    ++pos;
                }
            }
        }
    }
    free(cnt);
    free(sl);
    return total;
}

/* ------------------------------------------------------------------ */
/* FP64 Gaussian algebra                                               */
/* ------------------------------------------------------------------ */
static void quat_rot_d(const double *qf, double R[3][3])
{
    double w = qf[0], x = qf[1], y = qf[2], z = qf[3];
    R[0][0] = 1 - 2 * (y * y + z * z);
    R[0][1] = 2 * (x * y - w * z);
    R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);
    R[1][1] = 1 - 2 * (x * x + z * z);
    R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);
    R[2][1] = 2 * (y * z + w * x);
    R[2][2] = 1 - 2 * (x * x + y * y);
}

/* d R_rc / d q_m for the same formula (m = w,x,y,z) */
static void quat_rot_grad_d(const double *qf, double dR[4][3][3])
{
    double w = qf[0], x = qf[1], y = qf[2], z = qf[3];
    memset(dR, 0, sizeof(double) * 36);
    /* R00 = 1 - 2(y^2 + z^2) */
    dR[2][0][0] = -4 * y; dR[3][0][0] = -4 * z;
    /* R01 = 2(xy - wz) */
    dR[0][0][1] = -2 * z; dR[1][0][1] = 2 * y; dR[2][0][1] = 2 * x; dR[3][0][1] = -2 * w;
    /* R02 = 2(xz + wy) */
    dR[0][0][2] = 2 * y; dR[1][0][2] = 2 * z; dR[2][0][2] = 2 * w; dR[3][0][2] = 2 * x;
    /* R10 = 2(xy + wz) */
    dR[0][1][0] = 2 * z; dR[1][1][0] = 2 * y; dR[2][1][0] = 2 * x; dR[3][1][0] = 2 * w;
    /* R11 = 1 - 2(x^2 + z^2) */
    dR[1][1][1] = -4 * x; dR[3][1][1] = -4 * z;
    /* R12 = 2(yz - wx) */
    dR[0][1][2] = -2 * x; dR[1][1][2] = -2 * w; dR[2][1][2] = 2 * z; dR[3][1][2] = 2 * y;
    /* R20 = 2(xz - wy) */
    dR[0][2][0] = -2 * y; dR[1][2][0] = 2 * z; dR[2][2][0] = -2 * w; dR[3][2][0] = 2 * x;
    /* R21 = 2(yz + wx) */
    dR[0][2][1] = 2 * x; dR[1][2][1] = 2 * w; dR[2][2][1] = 2 * z; dR[3][2][1] = 2 * y;
    /* R22 = 1 - 2(x^2 + y^2) */
    dR[1][2][2] = -4 * x; dR[2][2][2] = -4 * y;
}

/* Sigma = R diag(s^2) R^T */
static void cov_d(const double *qf, const double *sf, double Sg[3][3], double R[3][3])
{
    quat_rot_d(qf, R);
    double s2[3] = {sf[0] * sf[0], sf[1] * sf[1], sf[2] * sf[2]};
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int m = 0; m < 3; ++m) acc += R[r][m] * s2[m] * R[c][m];
            Sg[r][c] = acc;
        }
}

static double det3(const double A[3][3])
{
    return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
           A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

/* inverse by the adjugate */
static void inv3(const double A[3][3], double Ai[3][3], double *det_out)
{
    double d = det3(A);
    Ai[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / d;
    Ai[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / d;
    Ai[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / d;
    Ai[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / d;
    Ai[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / d;
    Ai[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / d;
    Ai[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / d;
    Ai[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / d;
    Ai[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / d;
    if (det_out) *det_out = d;
}

/* Everything one (Gaussian, slice) term needs in FP64. */
typedef struct {
    double mu[3], alpha, R[3][3], Sg[3][3], Sgi[3][3], Sp[3][3], P[3][3], c;
} or_term;

static void term_setup(const double *mu, const double *q, const double *s, double alpha, const or_slice *sl,
                       or_term *T)
{
    cov_d(q, s, T->Sg, T->R);
    double dS;
    inv3(T->Sg, T->Sgi, &dS);
    /* Sigma' = Sigma + R_k diag(pu^2, pv^2, sig^2) R_k^T: the slice's 3-D PSF
     * (in-plane PSF and slice profile) in world coordinates */
    const double *Q = sl->xfd;
    double var[3] = {sl->pud * sl->pud * OR_FWHM2VAR, sl->pvd * sl->pvd * OR_FWHM2VAR,
                     sl->thkd * sl->thkd * OR_FWHM2VAR};
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int a = 0; a < 3; ++a) acc += Q[3 * r + a] * var[a] * Q[3 * c + a];
            T->Sp[r][c] = T->Sg[r][c] + acc;
        }
    double dSp;
    inv3(T->Sp, T->P, &dSp);
    T->c = sqrt(dS / dSp);
    T->alpha = alpha;
    for (int r = 0; r < 3; ++r) T->mu[r] = mu[r];
}

static void pixel_world(const or_slice *sl, int i, int j, double x[3])
{
    const double *Q = sl->xfd;
    double u = (i - 0.5 * (sl->W - 1)) * sl->dxd;
    double v = (j - 0.5 * (sl->H - 1)) * sl->dyd;
    for (int r = 0; r < 3; ++r) x[r] = Q[3 * r + 0] * u + Q[3 * r + 1] * v + Q[9 + r];
}

/* Mahalanobis form y^T P y and P y */
static double quad_form(const or_term *T, const double x[3], double y[3], double Py[3])
{
    for (int r = 0; r < 3; ++r) y[r] = x[r] - T->mu[r];
    double qf = 0;
    for (int r = 0; r < 3; ++r) {
        Py[r] = T->P[r][0] * y[0] + T->P[r][1] * y[1] + T->P[r][2] * y[2];
        qf += y[r] * Py[r];
    }
    return qf;
}

/* ------------------------------------------------------------------ */
/* renders                                                             */
/* ------------------------------------------------------------------ */

/* exact = 0: S^bin from the records; exact = 1: every Gaussian at every pixel. */
void or_render(int64_t n, const double *mean, const double *quat, const double *scale, const double *alpha, int n_stacks,
               const int32_t *nsl, const int32_t *H, const int32_t *W, const double *dx, const double *dy,
               const double *thk, const double *psf, const double *xform, int64_t nrec, const int32_t *rec_slice,
               const int32_t *rec_gid, const int32_t *rec_rect, const uint64_t *rec_inset, int exact, double *out,
               const int32_t *cells_i, const float *cells_f)
{
    int S;
    or_slice *sl = or_build_slices(n_stacks, nsl, H, W, NULL, NULL, NULL, NULL, NULL, dx, dy, thk, psf, xform, &S);
    or_cells cc;
    if (cells_i) cells_setup(cells_i, cells_f, &cc);
    int64_t total = 0;
    for (int k = 0; k < S; ++k) total += (int64_t)sl[k].H * sl[k].W;
    memset(out, 0, sizeof(double) * (size_t)total);
    if (exact) {
#pragma omp parallel for schedule(dynamic)
        for (int k = 0; k < S; ++k) {
            double *img = out + sl[k].out_base;
            for (int64_t g = 0; g < n; ++g) {
                or_term T;
                term_setup(mean + 3 * g, quat + 4 * g, scale + 3 * g, alpha[g], &sl[k], &T);
                for (int j = 0; j < sl[k].H; ++j)
                    for (int i = 0; i < sl[k].W; ++i) {
                        double x[3], y[3], Py[3];
                        pixel_world(&sl[k], i, j, x);
                        double qf = quad_form(&T, x, y, Py);
                        img[(int64_t)j * sl[k].W + i] += T.alpha * T.c * exp(-0.5 * qf);
                    }
            }
        }
    } else {
        /* records are slice-major: find each slice's record range, then one
           thread per slice owns that slice's image */
        int64_t *first = (int64_t *)malloc(sizeof(int64_t) * ((size_t)S + 1));
        for (int k = 0; k <= S; ++k) first[k] = nrec;
        for (int64_t r = nrec - 1; r >= 0; --r) first[rec_slice[r]] = r;
        for (int k = S - 1; k >= 0; --k)
            if (first[k] > first[k + 1]) first[k] = first[k + 1];
#pragma omp parallel for schedule(dynamic)
        for (int k = 0; k < S; ++k) {
            double *img = out + sl[k].out_base;
            for (int64_t r = first[k]; r < first[k + 1]; ++r) {
                int64_t g = rec_gid[r];
                or_term T;
                term_setup(mean + 3 * g, quat + 4 * g, scale + 3 * g, alpha[g], &sl[k], &T);
                const int32_t *rc = rec_rect + 4 * r;
                int j0 = rc[1] * OR_TILE, j1 = (rc[3] + 1) * OR_TILE;
                if (j1 > sl[k].H) j1 = sl[k].H;
                int gcell[3];
                if (cells_i) {
                    float muf[3] = {(float)mean[3 * g], (float)mean[3 * g + 1], (float)mean[3 * g + 2]};
                    float b[3];
                    gauss_cell_f(muf, &cc, gcell, b);
                }
                for (int j = j0; j < j1; ++j) {
                    int i0, i1;
                    listed_cols(rc, rec_inset, r, j, sl[k].W, &i0, &i1);
                    for (int i = i0; i < i1; ++i) {
                        if (cells_i) {
                            int vcell[3];
                            voxel_cell_f(&sl[k], i, j, &cc, vcell);
                            if (!cell_member(vcell, gcell, cc.R)) continue;
                        }
                        double x[3], y[3], Py[3];
                        pixel_world(&sl[k], i, j, x);
                        double qf = quad_form(&T, x, y, Py);
                        img[(int64_t)j * sl[k].W + i] += T.alpha * T.c * exp(-0.5 * qf);
                    }
                }
            }
        }
        free(first);
    }
    free(sl);
}

/*
 * Analytic FP64 gradient of L = sum_pixels gout * S^bin with the records held
 * fixed, w.r.t. mean, quat (the 4 components entering the rotation formula),
 * scale and alpha. Per term f = alpha c e, c = sqrt(|Sigma|/|Sigma'|),
 * e = exp(-1/2 y^T P y), P = Sigma'^-1, y = x - mu:
 *   df/dalpha = c e
 *   df/dmu    = f P y
 *   df/dSigma = f/2 (Sigma^-1 - P + P y y^T P)     (as a symmetric matrix)
 * then Sigma = R diag(s^2) R^T gives
 *   dL/dR = 2 G R diag(s^2),  dL/ds_c = 2 s_c (R^T G R)_cc
 * and dL/dq from dR/dq.
 */
void or_grad(int64_t n, const double *mean, const double *quat, const double *scale, const double *alpha, int n_stacks,
             const int32_t *nsl, const int32_t *H, const int32_t *W, const double *dx, const double *dy, const double *thk,
             const double *psf, const double *xform, int64_t nrec, const int32_t *rec_slice, const int32_t *rec_gid,
             const int32_t *rec_rect, const uint64_t *rec_inset, const double *gout, double *gmean, double *gquat,
             double *gscale, double *galpha, const int32_t *cells_i, const float *cells_f)
{
    int S;
    or_slice *sl = or_build_slices(n_stacks, nsl, H, W, NULL, NULL, NULL, NULL, NULL, dx, dy, thk, psf, xform, &S);
    or_cells cc;
    if (cells_i) cells_setup(cells_i, cells_f, &cc);
    double *rg = (double *)calloc((size_t)(nrec > 0 ? nrec : 1) * 11, sizeof(double));
#pragma omp parallel for schedule(dynamic)
    for (int64_t r = 0; r < nrec; ++r) {
        int k = rec_slice[r];
        int64_t g = rec_gid[r];
        or_term T;
        term_setup(mean + 3 * g, quat + 4 * g, scale + 3 * g, alpha[g], &sl[k], &T);
        const double *go = gout + sl[k].out_base;
        const int32_t *rc = rec_rect + 4 * r;
        int j0 = rc[1] * OR_TILE, j1 = (rc[3] + 1) * OR_TILE;
        if (j1 > sl[k].H) j1 = sl[k].H;
        double ga = 0, gmu[3] = {0, 0, 0}, GS[3][3];
        memset(GS, 0, sizeof(GS));
        int gcell[3];
        if (cells_i) {
            float muf[3] = {(float)mean[3 * g], (float)mean[3 * g + 1], (float)mean[3 * g + 2]};
            float b[3];
            gauss_cell_f(muf, &cc, gcell, b);
        }
        for (int j = j0; j < j1; ++j) {
            int i0, i1;
            listed_cols(rc, rec_inset, r, j, sl[k].W, &i0, &i1);
            for (int i = i0; i < i1; ++i) {
                double G = go[(int64_t)j * sl[k].W + i];
                if (G == 0.0) continue;
                if (cells_i) {
                    int vcell[3];
                    voxel_cell_f(&sl[k], i, j, &cc, vcell);
                    if (!cell_member(vcell, gcell, cc.R)) continue;
                }
                double x[3], y[3], Py[3];
                pixel_world(&sl[k], i, j, x);
                double qf = quad_form(&T, x, y, Py);
                double e = exp(-0.5 * qf);
                double f = T.alpha * T.c * e;
                ga += G * T.c * e;
                for (int a = 0; a < 3; ++a) gmu[a] += G * f * Py[a];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        GS[a][b] += G * f * 0.5 * (T.Sgi[a][b] - T.P[a][b] + Py[a] * Py[b]);
            }
        }
        /* chain Sigma -> R, s -> q */
        const double *s = scale + 3 * g;
        double dLdR[3][3];
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) {
                double acc = 0;
                for (int b = 0; b < 3; ++b) acc += GS[a][b] * T.R[b][c];
                dLdR[a][c] = 2.0 * acc * s[c] * s[c];
            }
        double gs[3];
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) acc += T.R[a][c] * GS[a][b] * T.R[b][c];
            gs[c] = 2.0 * s[c] * acc;
        }
        double dR[4][3][3];
        quat_rot_grad_d(quat + 4 * g, dR);
        double gq[4];
        for (int m = 0; m < 4; ++m) {
            double acc = 0;
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) acc += dLdR[a][c] * dR[m][a][c];
            gq[m] = acc;
        }
        double *o = rg + 11 * r;
        o[0] = gmu[0]; o[1] = gmu[1]; o[2] = gmu[2];
        o[3] = gq[0]; o[4] = gq[1]; o[5] = gq[2]; o[6] = gq[3];
        o[7] = gs[0]; o[8] = gs[1]; o[9] = gs[2];
        o[10] = ga;
    }
    memset(gmean, 0, sizeof(double) * 3 * (size_t)n);
    memset(gquat, 0, sizeof(double) * 4 * (size_t)n);
    memset(gscale, 0, sizeof(double) * 3 * (size_t)n);
    memset(galpha, 0, sizeof(double) * (size_t)n);
    for (int64_t r = 0; r < nrec; ++r) {
        int64_t g = rec_gid[r];
        const double *o = rg + 11 * r;
        for (int a = 0; a < 3; ++a) gmean[3 * g + a] += o[a];
        for (int a = 0; a < 4; ++a) gquat[4 * g + a] += o[3 + a];
        for (int a = 0; a < 3; ++a) gscale[3 * g + a] += o[7 + a];
        galpha[g] += o[10];
    }
    free(rg);
    free(sl);
}

/* counts[0] = pairs (record, pixel in a listed tile) with y^T Sigma'^-1 y <= K^2
 * (FP64), counts[1] = all evaluated pairs (record, pixel in a listed tile). The
 * listed tiles are the rectangle's, culled per row by rec_inset (NULL: none). */
void or_pair_counts(int64_t n_unused, const double *mean, const double *quat, const double *scale, const double *alpha,
                    int n_stacks, const int32_t *nsl, const int32_t *H, const int32_t *W, const double *dx,
                    const double *dy, const double *thk, const double *psf, const double *xform, int64_t nrec,
                    const int32_t *rec_slice,
                    const int32_t *rec_gid, const int32_t *rec_rect, const uint64_t *rec_inset, double K,
                    int64_t *counts)
{
    (void)n_unused;
    int S;
    or_slice *sl = or_build_slices(n_stacks, nsl, H, W, NULL, NULL, NULL, NULL, NULL, dx, dy, thk, psf, xform, &S);
    int64_t inside = 0, evald = 0;
#pragma omp parallel for schedule(dynamic) reduction(+ : inside, evald)
    for (int64_t r = 0; r < nrec; ++r) {
        int k = rec_slice[r];
        int64_t g = rec_gid[r];
        or_term T;
        term_setup(mean + 3 * g, quat + 4 * g, scale + 3 * g, alpha[g], &sl[k], &T);
        const int32_t *rc = rec_rect + 4 * r;
        int j0 = rc[1] * OR_TILE, j1 = (rc[3] + 1) * OR_TILE;
        if (j1 > sl[k].H) j1 = sl[k].H;
        for (int j = j0; j < j1; ++j) {
            int i0, i1;
            listed_cols(rc, rec_inset, r, j, sl[k].W, &i0, &i1);
            for (int i = i0; i < i1; ++i) {
                double x[3], y[3], Py[3];
                pixel_world(&sl[k], i, j, x);
                double qf = quad_form(&T, x, y, Py);
                inside += (qf <= K * K);
                evald += 1;
            }
        }
    }
    counts[0] = inside;
    counts[1] = evald;
    free(sl);
}
