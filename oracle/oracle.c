/*
 * oracle.c -- plain FP64 CPU reference for gradient-aware spline upscaling of
 * 3D Gaussian Splatting images (Niedermayr, Neuhauser, Westermann, ICCV 2025).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg load this library.  It shares no code, no
 * header and no constant with the CUDA library; the two meet only through the
 * seeded inputs of the `scenes` module.
 *
 * Every function is the definition written out in double precision, in the
 * order the paper states it, with no blocking, fusion or reordering:
 *
 *   ora_sh_basis     real spherical harmonics (view-dependent colour, Sec. 4)
 *   ora_project      EWA projection Sigma' = J W Sigma W^T J^T (Sec. 4)
 *   ora_bin          brute-force tile binning, order (tile, depth, id) (Sec. 4:
 *                    Gaussians are blended front to back)
 *   ora_render       per-pixel front-to-back blend with the A/B recurrences and
 *                    their screen-space derivatives (Sec. 5 "3DGS Image
 *                    Gradients"; supplement "Forward pass")
 *   ora_spline_cinv  inverse of the constant Hermite matrix C (supplement
 *                    "Spline Image Interpolation")
 *   ora_upscale      bicubic patch p(x,y) = [1 x x^2 x^3] C^-1 F C^-T [1 y y^2 y^3]^T
 *                    per low-res cell (Sec. 5 "Spline Interpolation")
 *   ora_upscale_adjoint  transpose of the (linear) upscale
 *   ora_render_adjoint   per-pixel tape swept back to front (supplement
 *                    "Backward Pass"): dL/d(mean2D, conic, opacity, colour)
 *   ora_project_adjoint  forward-mode (dual number) derivatives of the
 *                    projection, contracted with the upstream gradient
 *   ora_bicubic      classical bicubic (cubic convolution) comparator
 *
 * Readings of passages the paper leaves open (all inherited from the 3DGS
 * renderer the paper builds on, Sec. 6.2):
 *   - Gaussian exponent g = -1/2 d^T Sigma'^-1 d, d = (x - mu_x, y - mu_y) in pixels
 *     (Sec. 4 prints the exponent without the inverse and the 1/2).
 *   - Sigma' gets +0.3 px^2 on its diagonal; radius = ceil(3 sqrt(lambda_max));
 *     a Gaussian's tiles are those holding a pixel centre inside the 3-sigma
 *     square cut to the bounding box of its alpha >= 1/255 ellipse.
 *   - near plane z <= znear culls; J uses x/z, y/z clamped to 1.3 tan(fov/2).
 *   - mode 0 ("3dgs"): alpha = min(0.99, sigma e^g), pairs with alpha < 1/255 are
 *     skipped, a pixel stops before the Gaussian that would take its
 *     transmittance below 1e-4.  mode 1 ("exact"): none of these, and every
 *     Gaussian is binned into every tile, so the image is smooth.
 *   - colour = max(0, sum_k sh_k Y_k(dir) + 1/2), dir from camera centre to mean.
 *   - pixel (i, j) is evaluated at the continuous point (i, j).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_OK 0
#define ORA_EINVAL 1
#define ORA_ENOMEM 2

#define MODE_3DGS 0
#define MODE_EXACT 1

/* ------------------------------------------------------------------------- */
/* Real spherical harmonics, degree <= 3.                                     */
/* Y_{l,m} for m > 0:  sqrt(2) K_l^m P_l^m(cos t) cos(m p)                    */
/*           m < 0:  sqrt(2) K_l^|m| P_l^|m|(cos t) sin(|m| p)                */
/*           m = 0:  K_l^0 P_l(cos t)                                         */
/* K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), P_l^m with the Condon-Shortley  */
/* phase.  Coefficient index k = l^2 + l + m.                                 */
/* ------------------------------------------------------------------------- */

static double fact(int k)
{
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= (double)i;
    return f;
}

/* associated Legendre function P_l^m(x), 0 <= m <= l, Condon-Shortley phase */
static double legendre_p(int l, int m, double x)
{
    double s = sqrt(fmax(0.0, 1.0 - x * x));
    /* P_m^m = (-1)^m (2m-1)!! s^m */
    double p_mm = 1.0;
    for (int i = 1; i <= m; ++i) p_mm *= -(double)(2 * i - 1) * s;
    if (l == m) return p_mm;
    /* P_{m+1}^m = x (2m+1) P_m^m */
    double p_prev = p_mm;
    double p_cur = x * (double)(2 * m + 1) * p_mm;
    /* (l-m) P_l^m = (2l-1) x P_{l-1}^m - (l+m-1) P_{l-2}^m */
    for (int ll = m + 2; ll <= l; ++ll) {
        double p_next = ((double)(2 * ll - 1) * x * p_cur - (double)(ll + m - 1) * p_prev) / (double)(ll - m);
        p_prev = p_cur;
        p_cur = p_next;
    }
    return p_cur;
}

static void sh_basis_one(int deg, const double dir_in[3], double* out)
{
    double nrm = sqrt(dir_in[0] * dir_in[0] + dir_in[1] * dir_in[1] + dir_in[2] * dir_in[2]);
    double x = dir_in[0] / nrm, y = dir_in[1] / nrm, z = dir_in[2] / nrm;
    double ct = fmin(1.0, fmax(-1.0, z));
    double ph = atan2(y, x);
    for (int l = 0; l <= deg; ++l) {
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * fact(l - am) / fact(l + am));
            double P = legendre_p(l, am, ct);
            double v;
            if (m == 0)
                v = K * P;
            else if (m > 0)
                v = sqrt(2.0) * K * P * cos((double)am * ph);
            else
                v = sqrt(2.0) * K * P * sin((double)am * ph);
            out[l * l + l + m] = v;
        }
    }
}

int ora_sh_basis(int deg, int64_t n, const double* dirs, double* out)
{
    if (deg < 0 || deg > 3 || n < 0) return ORA_EINVAL;
    int K = (deg + 1) * (deg + 1);
    for (int64_t i = 0; i < n; ++i) sh_basis_one(deg, dirs + 3 * i, out + K * i);
    return ORA_OK;
}

/* ------------------------------------------------------------------------- */
/* Projection (Sec. 4): Sigma = R S S^T R^T, Sigma' = J W Sigma W^T J^T.       */
/* ------------------------------------------------------------------------- */

/* Tile span of one axis: the tiles that contain a pixel centre i with
 * |i - m| <= h, for pixels 0..npix-1.  Returns 0 (and t0 > t1) if none. */
static int axis_span(double m, double h, int npix, int tile, int32_t* t0, int32_t* t1)
{
    double lo = ceil(m - h), hi = floor(m + h);
    *t0 = 0;
    *t1 = -1;
    if (!(h >= 0.0) || hi < 0.0 || lo > (double)(npix - 1) || lo > hi) return 0;
    int32_t p0 = lo < 0.0 ? 0 : (int32_t)lo;
    int32_t p1 = hi > (double)(npix - 1) ? npix - 1 : (int32_t)hi;
    *t0 = p0 / tile;
    *t1 = p1 / tile;
    return 1;
}

/* rect = {tx0, ty0, tx1, ty1} inclusive from the two axis spans; returns the
 * tile count (0: none). */
static int64_t rect_of(double mx, double my, double hx, double hy, int W, int H, int tile, int32_t rect[4])
{
    int32_t a0, a1, b0, b1;
    int okx = axis_span(mx, hx, W, tile, &a0, &a1);
    int oky = axis_span(my, hy, H, tile, &b0, &b1);
    rect[0] = 0; rect[1] = 0; rect[2] = -1; rect[3] = -1;
    if (!okx || !oky) return 0;
    rect[0] = a0; rect[1] = b0; rect[2] = a1; rect[3] = b1;
    return (int64_t)(a1 - a0 + 1) * (int64_t)(b1 - b0 + 1);
}

/* Envelope / core of one axis span over perturbed (m, h): returns 1 if any
 * perturbation changes the span or its emptiness. */
static int axis_perturb(double m, double eps_m, const double* hs, int nh, int npix, int tile,
                        int32_t nominal0, int32_t nominal1, int nominal_ok,
                        int32_t* env0, int32_t* env1, int32_t* core0, int32_t* core1, int* core_ok)
{
    int changed = 0;
    *env0 = nominal0; *env1 = nominal1; *core0 = nominal0; *core1 = nominal1;
    *core_ok = nominal_ok;
    for (int a = -1; a <= 1; ++a)
        for (int k = 0; k < nh; ++k) {
            int32_t t0, t1;
            int ok = axis_span(m + a * eps_m, hs[k], npix, tile, &t0, &t1);
            if (ok != nominal_ok || (ok && (t0 != nominal0 || t1 != nominal1))) changed = 1;
            if (!ok) { *core_ok = 0; continue; }
            if (!nominal_ok && *env1 < *env0) { *env0 = t0; *env1 = t1; }
            if (t0 < *env0) *env0 = t0;
            if (t1 > *env1) *env1 = t1;
            if (t0 > *core0) *core0 = t0;
            if (t1 < *core1) *core1 = t1;
        }
    if (*core1 < *core0) *core_ok = 0;
    return changed;
}

int ora_project(int64_t n,
                const double* means, const double* log_scales, const double* quats,
                const double* opacity_logits, const double* sh, int sh_degree,
                const double* rgb_in,
                const double* viewmat, double fx, double fy, double cx, double cy,
                double znear, int W, int H, int tile, int mode,
                double* mean2d, double* cov2d, double* conic, double* rgb,
                double* opacity, double* depth, int32_t* radius, int32_t* rect,
                int64_t* tiles_touched, uint8_t* borderline, int32_t* envelope, int32_t* core)
{
    if (n < 0 || W < 1 || H < 1 || tile < 1 || sh_degree < 0 || sh_degree > 3) return ORA_EINVAL;
    if (sh == NULL && rgb_in == NULL && n > 0) return ORA_EINVAL;
    const int tiles_x = (W + tile - 1) / tile, tiles_y = (H + tile - 1) / tile;
    const int K = (sh_degree + 1) * (sh_degree + 1);

    double Rv[3][3], tv[3];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) Rv[r][c] = viewmat[4 * r + c];
        tv[r] = viewmat[4 * r + 3];
    }
    /* camera centre in world coordinates: -Rv^T t */
    double campos[3];
    for (int c = 0; c < 3; ++c) campos[c] = -(Rv[0][c] * tv[0] + Rv[1][c] * tv[1] + Rv[2][c] * tv[2]);
    const double lim_x = 1.3 * ((double)W / (2.0 * fx));
    const double lim_y = 1.3 * ((double)H / (2.0 * fy));

    for (int64_t i = 0; i < n; ++i) {
        mean2d[2 * i] = mean2d[2 * i + 1] = 0.0;
        for (int k = 0; k < 3; ++k) { cov2d[3 * i + k] = 0.0; conic[3 * i + k] = 0.0; rgb[3 * i + k] = 0.0; }
        opacity[i] = 0.0; depth[i] = 0.0; radius[i] = 0; tiles_touched[i] = 0; borderline[i] = 0;
        rect[4 * i + 0] = 0; rect[4 * i + 1] = 0; rect[4 * i + 2] = -1; rect[4 * i + 3] = -1;
        for (int k = 0; k < 4; ++k) envelope[4 * i + k] = core[4 * i + k] = rect[4 * i + k];

        const double* mu = means + 3 * i;
        double p[3];
        for (int r = 0; r < 3; ++r) p[r] = Rv[r][0] * mu[0] + Rv[r][1] * mu[1] + Rv[r][2] * mu[2] + tv[r];
        if (fabs(p[2] - znear) < 1e-6 * (1.0 + fabs(p[2]))) borderline[i] = 1;
        if (p[2] <= znear) continue;

        /* Sigma = R S S^T R^T, R from the normalised quaternion (w, x, y, z) */
        const double* q = quats + 4 * i;
        double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        if (!(qn > 0.0)) continue;
        double w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
        double R[3][3] = {
            {1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y)},
            {2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x)},
            {2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y)}};
        double s[3];
        for (int k = 0; k < 3; ++k) s[k] = exp(log_scales[3 * i + k]);
        double Sig[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += R[r][k] * s[k] * s[k] * R[c][k];
                Sig[r][c] = acc;
            }

        /* J: Jacobian of the perspective map at the (frustum-clamped) mean */
        double tz = p[2];
        double txz = p[0] / tz, tyz = p[1] / tz;
        txz = fmin(lim_x, fmax(-lim_x, txz));
        tyz = fmin(lim_y, fmax(-lim_y, tyz));
        double J[2][3] = {{fx / tz, 0.0, -fx * txz / tz},
                          {0.0, fy / tz, -fy * tyz / tz}};
        /* M = J W (2x3); Sigma' = M Sigma M^T (2x2) */
        double M[2][3];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) M[r][c] = J[r][0] * Rv[0][c] + J[r][1] * Rv[1][c] + J[r][2] * Rv[2][c];
        double S2[2][2];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) acc += M[r][k] * Sig[k][l] * M[c][l];
                S2[r][c] = acc;
            }
        S2[0][0] += 0.3;
        S2[1][1] += 0.3;
        double det = S2[0][0] * S2[1][1] - S2[0][1] * S2[1][0];
        if (!(det > 0.0)) continue;

        /* largest eigenvalue of the symmetric 2x2 Sigma' */
        double mid = 0.5 * (S2[0][0] + S2[1][1]);
        double half_diff = 0.5 * (S2[0][0] - S2[1][1]);
        double lam = mid + sqrt(half_diff * half_diff + S2[0][1] * S2[0][1]);
        double v = 3.0 * sqrt(lam);
        double r_nom = ceil(v);

        double mx = fx * p[0] / p[2] + cx;
        double my = fy * p[1] / p[2] + cy;

        mean2d[2 * i] = mx;
        mean2d[2 * i + 1] = my;
        cov2d[3 * i + 0] = S2[0][0];
        cov2d[3 * i + 1] = S2[0][1];
        cov2d[3 * i + 2] = S2[1][1];
        conic[3 * i + 0] = S2[1][1] / det;
        conic[3 * i + 1] = -S2[0][1] / det;
        conic[3 * i + 2] = S2[0][0] / det;
        depth[i] = p[2];
        radius[i] = (int32_t)r_nom;
        opacity[i] = 1.0 / (1.0 + exp(-opacity_logits[i]));

        if (sh != NULL) {
            double dir[3] = {mu[0] - campos[0], mu[1] - campos[1], mu[2] - campos[2]};
            double Y[16];
            sh_basis_one(sh_degree, dir, Y);
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int k = 0; k < K; ++k) acc += sh[(i * K + k) * 3 + c] * Y[k];
                rgb[3 * i + c] = fmax(0.0, acc + 0.5);
            }
        } else {
            for (int c = 0; c < 3; ++c) rgb[3 * i + c] = rgb_in[3 * i + c];
        }

        int32_t* rc = rect + 4 * i;
        int32_t* ev = envelope + 4 * i;
        int32_t* co = core + 4 * i;
        if (mode == MODE_EXACT) {
            rc[0] = 0; rc[1] = 0; rc[2] = tiles_x - 1; rc[3] = tiles_y - 1;
            tiles_touched[i] = (int64_t)tiles_x * tiles_y;
            for (int k = 0; k < 4; ++k) ev[k] = co[k] = rc[k];
            continue;
        }
        /* Only pixels with alpha = sigma e^g >= 1/255 can blend: g >= -L with
         * L = ln(255 sigma), the ellipse d^T Sigma'^-1 d <= 2L, whose bounding box
         * has half-widths sqrt(2 L Sigma'_xx), sqrt(2 L Sigma'_yy).  The tile set is
         * the 3-sigma square of the 3DGS renderer cut to that box (no pair
         * outside it can pass the cut-off, so the image is unchanged). */
        const double L = log(255.0 * opacity[i]);
        const double ex = L > 0.0 ? sqrt(2.0 * L * S2[0][0]) : -1.0;
        const double ey = L > 0.0 ? sqrt(2.0 * L * S2[1][1]) : -1.0;
        const double hx = fmin(r_nom, ex), hy = fmin(r_nom, ey);
        tiles_touched[i] = rect_of(mx, my, hx, hy, W, H, tile, rc);
        for (int k = 0; k < 4; ++k) ev[k] = co[k] = rc[k];

        /* Borderline: the rect is not stable under the rounding error an FP32
         * evaluation of the same quantities can make (mean2D within eps_pos;
         * 3 sqrt(lambda), the box half-widths and L within a relative 2e-5). */
        const double eps_pos = 3e-7 * (fabs(mx) + fabs(my) + fabs(fx) + fabs(fy)) + 1e-6;
        const double eps_r = 2e-5 * v;
        const double rc_lo = ceil(v - eps_r), rc_hi = ceil(v + eps_r);
        double hxs[6], hys[6];
        int nh = 0;
        const double Lp[2] = {L * (1.0 - 2e-5) - 1e-6, L * (1.0 + 2e-5) + 1e-6};
        for (int q = 0; q < 2; ++q) {
            const double exq = Lp[q] > 0.0 ? sqrt(2.0 * Lp[q] * S2[0][0]) : -1.0;
            const double eyq = Lp[q] > 0.0 ? sqrt(2.0 * Lp[q] * S2[1][1]) : -1.0;
            hxs[nh] = fmin(rc_lo, exq); hys[nh] = fmin(rc_lo, eyq); ++nh;
            hxs[nh] = fmin(rc_hi, exq); hys[nh] = fmin(rc_hi, eyq); ++nh;
        }
        int32_t nx0, nx1, ny0, ny1;
        const int okx = axis_span(mx, hx, W, tile, &nx0, &nx1);
        const int oky = axis_span(my, hy, H, tile, &ny0, &ny1);
        int32_t ex0, ex1, ey0, ey1, cx0, cx1, cy0, cy1;
        int cokx, coky;
        const int chx = axis_perturb(mx, eps_pos, hxs, nh, W, tile, nx0, nx1, okx, &ex0, &ex1, &cx0, &cx1, &cokx);
        const int chy = axis_perturb(my, eps_pos, hys, nh, H, tile, ny0, ny1, oky, &ey0, &ey1, &cy0, &cy1, &coky);
        if (chx || chy) {
            borderline[i] = 1;
            if (ex1 >= ex0 && ey1 >= ey0) { ev[0] = ex0; ev[1] = ey0; ev[2] = ex1; ev[3] = ey1; }
            if (cokx && coky) { co[0] = cx0; co[1] = cy0; co[2] = cx1; co[3] = cy1; }
            else { co[0] = 0; co[1] = 0; co[2] = -1; co[3] = -1; }
        }
    }
    return ORA_OK;
}

/* ------------------------------------------------------------------------- */
/* Tile binning: every (tile, Gaussian) pair of the rects, ordered by tile,    */
/* then by the FP32 bits of the view depth (front to back), then by id.        */
/* key = tile << 32 | depth bits, value = Gaussian id.                         */
/* ------------------------------------------------------------------------- */

typedef struct { uint64_t key; uint32_t id; } Pair;

static int pair_cmp(const void* a, const void* b)
{
    const Pair* x = (const Pair*)a;
    const Pair* y = (const Pair*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

int ora_bin(int64_t n, const double* depth, const int32_t* rect, int tiles_x, int tiles_y,
            int64_t P, uint64_t* keys, uint32_t* vals, uint32_t* ranges)
{
    if (n < 0 || tiles_x < 1 || tiles_y < 1 || P < 0) return ORA_EINVAL;
    int64_t count = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int32_t* rc = rect + 4 * i;
        if (rc[2] >= rc[0] && rc[3] >= rc[1]) count += (int64_t)(rc[2] - rc[0] + 1) * (rc[3] - rc[1] + 1);
    }
    if (count != P) return ORA_EINVAL;
    Pair* pairs = (Pair*)malloc(sizeof(Pair) * (size_t)(P > 0 ? P : 1));
    if (!pairs) return ORA_ENOMEM;
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int32_t* rc = rect + 4 * i;
        if (!(rc[2] >= rc[0] && rc[3] >= rc[1])) continue;
        float d32 = (float)depth[i];
        uint32_t bits;
        memcpy(&bits, &d32, 4);
        for (int ty = rc[1]; ty <= rc[3]; ++ty)
            for (int tx = rc[0]; tx <= rc[2]; ++tx) {
                uint64_t t = (uint64_t)ty * (uint64_t)tiles_x + (uint64_t)tx;
                pairs[k].key = (t << 32) | (uint64_t)bits;
                pairs[k].id = (uint32_t)i;
                ++k;
            }
    }
    qsort(pairs, (size_t)P, sizeof(Pair), pair_cmp);
    const int64_t T = (int64_t)tiles_x * tiles_y;
    memset(ranges, 0, sizeof(uint32_t) * 2 * (size_t)T);
    for (int64_t j = 0; j < P; ++j) {
        keys[j] = pairs[j].key;
        vals[j] = pairs[j].id;
        uint64_t t = pairs[j].key >> 32;
        if (j == 0 || (pairs[j - 1].key >> 32) != t) ranges[2 * t] = (uint32_t)j;
        if (j == P - 1 || (pairs[j + 1].key >> 32) != t) ranges[2 * t + 1] = (uint32_t)(j + 1);
    }
    free(pairs);
    return ORA_OK;
}

/* ------------------------------------------------------------------------- */
/* Blend with screen-space derivatives (supplement, "Forward pass"):           */
/*   B_i = B_{i-1} + (1 - A_{i-1}) alpha_i c_i,  A_i = A_{i-1} + alpha_i (1 - A_{i-1})
 *   dB_i/dx = dB_{i-1}/dx + c_i ((1 - A_{i-1}) alpha_x - A_{i-1,x} alpha_i)
 *   d2B_i/dxdy = d2B_{i-1}/dxdy + c_i ((1 - A_{i-1}) alpha_xy - A_{i-1,y} alpha_x
 *                - A_{i-1,xy} alpha_i - A_{i-1,x} alpha_y)
 *   A_{i,x} = A_{i-1,x} (1 - alpha_i) + (1 - A_{i-1}) alpha_x
 *   A_{i,xy} = A_{i-1,xy} (1 - alpha_i) + (1 - A_{i-1}) alpha_xy
 *              - A_{i-1,x} alpha_y - A_{i-1,y} alpha_x
 * with alpha = sigma e^g, alpha_x = alpha g_x, alpha_xy = alpha (g_x g_y + g_xy).
 * I = B_N + (1 - A_N) bg; derivatives likewise.                              */
/* ------------------------------------------------------------------------- */

/* A decision the FP32 path may take the other way: its quantity lies within a
 * relative DELTA of its threshold and flipping it moves the outputs by more
 * than EFFECT_MIN.  Types: 0 = alpha cutoff, 1 = 0.99 clamp, 2 = termination. */
#define DEC_DELTA 1e-3
#define DEC_EFFECT_MIN 1e-5
#define MAX_SENS 3
#define MAX_VAR (1 << MAX_SENS)

typedef struct { int32_t j; int32_t type; } Decision;

typedef struct {
    int W, H, tile, tiles_x, mode;
    double bg[3];
    double off_x, off_y;
    const double *mean2d, *conic, *opacity, *rgb;
    const uint32_t *vals, *ranges;
} RenderCtx;

static int is_flipped(const Decision* flips, int nflips, int j, int type)
{
    for (int k = 0; k < nflips; ++k)
        if (flips[k].j == j && flips[k].type == type) return 1;
    return 0;
}

/* out[12] = C rgb, Cx rgb, Cy rgb, Cxy rgb; st[5] = A, A_x, A_y, A_xy, count */
static void blend_pixel(const RenderCtx* c, int ix, int iy, const Decision* flips, int nflips,
                        double out[12], double st[5], Decision* sens, int* nsens,
                        int64_t* n_eval, int64_t* n_acc)
{
    const double px = ix + c->off_x, py = iy + c->off_y;
    const int64_t t = (int64_t)(iy / c->tile) * c->tiles_x + (ix / c->tile);
    const uint32_t start = c->ranges[2 * t], end = c->ranges[2 * t + 1];
    double A = 0.0, Ax = 0.0, Ay = 0.0, Axy = 0.0;
    double B[3] = {0, 0, 0}, Bx[3] = {0, 0, 0}, By[3] = {0, 0, 0}, Bxy[3] = {0, 0, 0};
    int32_t count = 0;
    int ns = 0;
    for (uint32_t j = 0; j < end - start; ++j) {
        const uint32_t id = c->vals[start + j];
        const double dx = px - c->mean2d[2 * id], dy = py - c->mean2d[2 * id + 1];
        const double a = c->conic[3 * id], b = c->conic[3 * id + 1], cc = c->conic[3 * id + 2];
        const double g = -0.5 * (a * dx * dx + 2.0 * b * dx * dy + cc * dy * dy);
        const double gx = -(a * dx + b * dy), gy = -(b * dx + cc * dy), gxy = -b;
        double alpha = c->opacity[id] * exp(g);
        double ax = alpha * gx, ay = alpha * gy, axy = alpha * (gx * gy + gxy);
        ++*n_eval;
        if (c->mode == MODE_3DGS) {
            const double T = 1.0 - A;
            const double dsum = fabs(gx) + fabs(gy) + fabs(gx * gy + gxy);
            int reject = alpha < 1.0 / 255.0;
            if (fabs(alpha * 255.0 - 1.0) < DEC_DELTA && T / 255.0 * (1.0 + dsum) > DEC_EFFECT_MIN) {
                if (sens && ns < MAX_SENS + 1) { sens[ns].j = (int32_t)j; sens[ns].type = 0; }
                ++ns;
            }
            if (is_flipped(flips, nflips, (int)j, 0)) reject = !reject;
            if (reject) continue;
            int clamped = alpha > 0.99;
            if (fabs(alpha / 0.99 - 1.0) < DEC_DELTA && T * dsum > DEC_EFFECT_MIN) {
                if (sens && ns < MAX_SENS + 1) { sens[ns].j = (int32_t)j; sens[ns].type = 1; }
                ++ns;
            }
            if (is_flipped(flips, nflips, (int)j, 1)) clamped = !clamped;
            if (clamped) { alpha = 0.99; ax = 0.0; ay = 0.0; axy = 0.0; }
            const double tnext = T * (1.0 - alpha);
            int stop = tnext < 1e-4;
            if (fabs(tnext / 1e-4 - 1.0) < DEC_DELTA && T * (1.0 + dsum) > DEC_EFFECT_MIN) {
                if (sens && ns < MAX_SENS + 1) { sens[ns].j = (int32_t)j; sens[ns].type = 2; }
                ++ns;
            }
            if (is_flipped(flips, nflips, (int)j, 2)) stop = !stop;
            if (stop) break;
        }
        ++*n_acc;
        const double T = 1.0 - A;
        for (int k = 0; k < 3; ++k) {
            const double col = c->rgb[3 * id + k];
            B[k] += T * alpha * col;
            Bx[k] += col * (T * ax - Ax * alpha);
            By[k] += col * (T * ay - Ay * alpha);
            Bxy[k] += col * (T * axy - Ay * ax - Axy * alpha - Ax * ay);
        }
        const double Axy_n = Axy * (1.0 - alpha) + T * axy - Ax * ay - Ay * ax;
        const double Ax_n = Ax * (1.0 - alpha) + T * ax;
        const double Ay_n = Ay * (1.0 - alpha) + T * ay;
        const double A_n = A + alpha * T;
        A = A_n; Ax = Ax_n; Ay = Ay_n; Axy = Axy_n;
        count = (int32_t)(j + 1);
    }
    for (int k = 0; k < 3; ++k) {
        out[k] = B[k] + (1.0 - A) * c->bg[k];
        out[3 + k] = Bx[k] - Ax * c->bg[k];
        out[6 + k] = By[k] - Ay * c->bg[k];
        out[9 + k] = Bxy[k] - Axy * c->bg[k];
    }
    st[0] = A; st[1] = Ax; st[2] = Ay; st[3] = Axy; st[4] = (double)count;
    if (nsens) *nsens = ns;
}

typedef struct {
    const RenderCtx* c;
    int64_t p0, p1;
    const int32_t* pix;
    double *out, *state, *variants;
    int32_t* nvar;
    int64_t n_eval, n_acc;
} RenderJob;

static void* render_worker(void* arg)
{
    RenderJob* jb = (RenderJob*)arg;
    const RenderCtx* c = jb->c;
    for (int64_t p = jb->p0; p < jb->p1; ++p) {
        int ix, iy;
        if (jb->pix) { ix = jb->pix[2 * p]; iy = jb->pix[2 * p + 1]; }
        else { ix = (int)(p % c->W); iy = (int)(p / c->W); }
        Decision sens[MAX_SENS + 1];
        int ns = 0;
        double st[5];
        blend_pixel(c, ix, iy, NULL, 0, jb->out + 12 * p, st, sens, &ns, &jb->n_eval, &jb->n_acc);
        if (jb->state) for (int k = 0; k < 5; ++k) jb->state[5 * p + k] = st[k];
        if (jb->nvar) jb->nvar[p] = ns <= MAX_SENS ? (1 << ns) : -ns;
        if (jb->variants) {
            double* vv = jb->variants + (size_t)12 * MAX_VAR * p;
            for (int k = 0; k < 12 * MAX_VAR; ++k) vv[k] = 0.0;
            for (int k = 0; k < 12; ++k) vv[k] = jb->out[12 * p + k];
            if (ns <= MAX_SENS) {
                for (int mask = 1; mask < (1 << ns); ++mask) {
                    Decision fl[MAX_SENS];
                    int nf = 0;
                    for (int k = 0; k < ns; ++k)
                        if (mask & (1 << k)) fl[nf++] = sens[k];
                    double st2[5];
                    int64_t e2 = 0, a2 = 0;
                    blend_pixel(c, ix, iy, fl, nf, vv + 12 * mask, st2, NULL, NULL, &e2, &a2);
                }
            }
        }
    }
    return NULL;
}

int ora_render(int W, int H, int tile, int mode, const double* bg, double off_x, double off_y,
               const double* mean2d, const double* conic, const double* opacity, const double* rgb,
               const uint32_t* vals, const uint32_t* ranges,
               int64_t npix, const int32_t* pix,
               double* out, double* state, int32_t* nvar, double* variants,
               int64_t* stats, int nthreads)
{
    if (W < 1 || H < 1 || tile < 1 || npix < 0) return ORA_EINVAL;
    if (pix == NULL && npix != (int64_t)W * H) return ORA_EINVAL;
    if (pix != NULL)
        for (int64_t p = 0; p < npix; ++p)
            if (pix[2 * p] < 0 || pix[2 * p] >= W || pix[2 * p + 1] < 0 || pix[2 * p + 1] >= H) return ORA_EINVAL;
    RenderCtx c;
    c.W = W; c.H = H; c.tile = tile; c.tiles_x = (W + tile - 1) / tile; c.mode = mode;
    for (int k = 0; k < 3; ++k) c.bg[k] = bg ? bg[k] : 0.0;
    c.off_x = off_x; c.off_y = off_y;
    c.mean2d = mean2d; c.conic = conic; c.opacity = opacity; c.rgb = rgb;
    c.vals = vals; c.ranges = ranges;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > npix) nthreads = npix > 0 ? (int)npix : 1;
    RenderJob jobs[256];
    pthread_t th[256];
    for (int k = 0; k < nthreads; ++k) {
        jobs[k].c = &c;
        jobs[k].p0 = npix * k / nthreads;
        jobs[k].p1 = npix * (k + 1) / nthreads;
        jobs[k].pix = pix; jobs[k].out = out; jobs[k].state = state;
        jobs[k].variants = variants; jobs[k].nvar = nvar;
        jobs[k].n_eval = 0; jobs[k].n_acc = 0;
    }
    for (int k = 1; k < nthreads; ++k) pthread_create(&th[k], NULL, render_worker, &jobs[k]);
    render_worker(&jobs[0]);
    for (int k = 1; k < nthreads; ++k) pthread_join(th[k], NULL);
    if (stats) {
        stats[0] = 0; stats[1] = 0;
        for (int k = 0; k < nthreads; ++k) { stats[0] += jobs[k].n_eval; stats[1] += jobs[k].n_acc; }
    }
    return ORA_OK;
}

/* ------------------------------------------------------------------------- */
/* Spline upscale (Sec. 5; supplement "Spline Image Interpolation").           */
/* C maps the cubic's coefficients (a0..a3) to (f(0), f(1), f'(0), f'(1)).     */
/* ------------------------------------------------------------------------- */

static const double SPLINE_C[4][4] = {
    {1.0, 0.0, 0.0, 0.0},
    {1.0, 1.0, 1.0, 1.0},
    {0.0, 1.0, 0.0, 0.0},
    {0.0, 1.0, 2.0, 3.0}};

/* Gauss-Jordan elimination with partial pivoting */
static int invert4(const double Min[4][4], double Inv[4][4])
{
    double a[4][8];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 8; ++c) a[r][c] = c < 4 ? Min[r][c] : (c - 4 == r ? 1.0 : 0.0);
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        for (int r = col + 1; r < 4; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (a[piv][col] == 0.0) return ORA_EINVAL;
        if (piv != col)
            for (int c = 0; c < 8; ++c) { double t = a[col][c]; a[col][c] = a[piv][c]; a[piv][c] = t; }
        double d = a[col][col];
        for (int c = 0; c < 8; ++c) a[col][c] /= d;
        for (int r = 0; r < 4; ++r) {
            if (r == col) continue;
            double f = a[r][col];
            if (f == 0.0) continue;
            for (int c = 0; c < 8; ++c) a[r][c] -= f * a[col][c];
        }
    }
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) Inv[r][c] = a[r][c + 4];
    return ORA_OK;
}

int ora_spline_cinv(double* out16)
{
    double inv[4][4];
    int st = invert4(SPLINE_C, inv);
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) out16[4 * r + c] = inv[r][c];
    return st;
}

/* Low-res sample point of hi-res pixel X: x = (X + 0.5) W / W2 - 0.5 (half-pixel
 * centres); cell i = clamp(floor(x), 0, W - 2), local t = x - i (extrapolated
 * outside [0, 1] in the border half-cells). */
static void cell_of(int X, int W, int W2, int* i, double* t)
{
    double x = ((double)X + 0.5) * (double)W / (double)W2 - 0.5;
    double fl = floor(x);
    int ii = (int)fl;
    if (ii < 0) ii = 0;
    if (ii > W - 2) ii = W - 2;
    *i = ii;
    *t = x - (double)ii;
}

/* C: [3][H][W]; G: [3 (d/dx, d/dy, d2/dxdy)][3][H][W]; out: [npix][3] */
int ora_upscale(int W, int H, int W2, int H2, const double* C, const double* G,
                int64_t npix, const int32_t* pix, double* out)
{
    if (W < 2 || H < 2 || W2 < 1 || H2 < 1 || npix < 0) return ORA_EINVAL;
    if (pix == NULL && npix != (int64_t)W2 * H2) return ORA_EINVAL;
    double Ci[4][4];
    if (invert4(SPLINE_C, Ci) != ORA_OK) return ORA_EINVAL;
    const int64_t plane = (int64_t)W * H;
    for (int64_t p = 0; p < npix; ++p) {
        int X, Y;
        if (pix) { X = pix[2 * p]; Y = pix[2 * p + 1]; }
        else { X = (int)(p % W2); Y = (int)(p / W2); }
        if (X < 0 || X >= W2 || Y < 0 || Y >= H2) return ORA_EINVAL;
        int i, j;
        double t, u;
        cell_of(X, W, W2, &i, &t);
        cell_of(Y, H, H2, &j, &u);
        for (int ch = 0; ch < 3; ++ch) {
            /* f(a, b): value at low-res pixel (x = i + a, y = j + b) */
#define VAL(q, a, b) ((q)[(int64_t)ch * plane + (int64_t)(j + (b)) * W + (i + (a))])
            const double* fx = G;
            const double* fy = G + 3 * plane;
            const double* fxy = G + 6 * plane;
            double F[4][4] = {
                {VAL(C, 0, 0), VAL(C, 0, 1), VAL(fy, 0, 0), VAL(fy, 0, 1)},
                {VAL(C, 1, 0), VAL(C, 1, 1), VAL(fy, 1, 0), VAL(fy, 1, 1)},
                {VAL(fx, 0, 0), VAL(fx, 0, 1), VAL(fxy, 0, 0), VAL(fxy, 0, 1)},
                {VAL(fx, 1, 0), VAL(fx, 1, 1), VAL(fxy, 1, 0), VAL(fxy, 1, 1)}};
#undef VAL
            /* A = C^-1 F C^-T */
            double CF[4][4], A[4][4];
            for (int r = 0; r < 4; ++r)
                for (int cc = 0; cc < 4; ++cc) {
                    double acc = 0.0;
                    for (int k = 0; k < 4; ++k) acc += Ci[r][k] * F[k][cc];
                    CF[r][cc] = acc;
                }
            for (int r = 0; r < 4; ++r)
                for (int cc = 0; cc < 4; ++cc) {
                    double acc = 0.0;
                    for (int k = 0; k < 4; ++k) acc += CF[r][k] * Ci[cc][k];
                    A[r][cc] = acc;
                }
            /* p(t, u) = [1 t t^2 t^3] A [1 u u^2 u^3]^T */
            double tv[4] = {1.0, t, t * t, t * t * t};
            double uv[4] = {1.0, u, u * u, u * u * u};
            double acc = 0.0;
            for (int r = 0; r < 4; ++r)
                for (int cc = 0; cc < 4; ++cc) acc += tv[r] * A[r][cc] * uv[cc];
            out[3 * p + ch] = acc;
        }
    }
    return ORA_OK;
}

/* ========================================================================= */
/* Reverse mode (training with differentiable upscaling; supplement          */
/* "Backward Pass").  Upstream gradients are dL/d(output); every function     */
/* returns the gradient of the same scalar L with respect to its inputs.      */
/* ========================================================================= */

/* ------------------------------------------------------------------------- */
/* Adjoint of ora_upscale.  The upscale is linear in the 12 low-res planes:    */
/* out = [1 t t^2 t^3] C^-1 F C^-T [1 u u^2 u^3]^T, so dL/dF_rc = dL/dout *     */
/* (C^-T tv)_r (C^-T uv)_c, scattered back to the plane entries F was read     */
/* from.  dout: [3][H2][W2]; dC: [3][H][W]; dG: [3][3][H][W] (overwritten).    */
/* ------------------------------------------------------------------------- */
int ora_upscale_adjoint(int W, int H, int W2, int H2, const double* dout, double* dC, double* dG)
{
    if (W < 2 || H < 2 || W2 < 1 || H2 < 1) return ORA_EINVAL;
    double Ci[4][4];
    if (invert4(SPLINE_C, Ci) != ORA_OK) return ORA_EINVAL;
    const int64_t plane = (int64_t)W * H;
    for (int64_t k = 0; k < 3 * plane; ++k) dC[k] = 0.0;
    for (int64_t k = 0; k < 9 * plane; ++k) dG[k] = 0.0;
    double* fx = dG;
    double* fy = dG + 3 * plane;
    double* fxy = dG + 6 * plane;
    for (int Y = 0; Y < H2; ++Y)
        for (int X = 0; X < W2; ++X) {
            int i, j;
            double t, u;
            cell_of(X, W, W2, &i, &t);
            cell_of(Y, H, H2, &j, &u);
            const double tv[4] = {1.0, t, t * t, t * t * t};
            const double uv[4] = {1.0, u, u * u, u * u * u};
            double wt[4], wu[4];
            for (int r = 0; r < 4; ++r) {
                wt[r] = 0.0;
                wu[r] = 0.0;
                for (int k = 0; k < 4; ++k) {
                    wt[r] += tv[k] * Ci[k][r];
                    wu[r] += uv[k] * Ci[k][r];
                }
            }
            for (int ch = 0; ch < 3; ++ch) {
                const double d = dout[(int64_t)ch * W2 * H2 + (int64_t)Y * W2 + X];
                double dF[4][4];
                for (int r = 0; r < 4; ++r)
                    for (int c = 0; c < 4; ++c) dF[r][c] = d * wt[r] * wu[c];
#define ACC(q, a, b, v) ((q)[(int64_t)ch * plane + (int64_t)(j + (b)) * W + (i + (a))] += (v))
                /* the layout of F in ora_upscale: rows (f(0,.), f(1,.), fx(0,.), fx(1,.)),
                 * columns (f(.,0), f(.,1), fy(.,0), fy(.,1)) */
                ACC(dC, 0, 0, dF[0][0]); ACC(dC, 0, 1, dF[0][1]); ACC(fy, 0, 0, dF[0][2]); ACC(fy, 0, 1, dF[0][3]);
                ACC(dC, 1, 0, dF[1][0]); ACC(dC, 1, 1, dF[1][1]); ACC(fy, 1, 0, dF[1][2]); ACC(fy, 1, 1, dF[1][3]);
                ACC(fx, 0, 0, dF[2][0]); ACC(fx, 0, 1, dF[2][1]); ACC(fxy, 0, 0, dF[2][2]); ACC(fxy, 0, 1, dF[2][3]);
                ACC(fx, 1, 0, dF[3][0]); ACC(fx, 1, 1, dF[3][1]); ACC(fxy, 1, 0, dF[3][2]); ACC(fxy, 1, 1, dF[3][3]);
#undef ACC
            }
        }
    return ORA_OK;
}

/* ------------------------------------------------------------------------- */
/* Adjoint of the blend (supplement "Backward Pass").  Per pixel, the forward  */
/* pass is replayed with the same decisions as blend_pixel and every blended   */
/* step is kept on a tape (alpha and its x/y derivatives, the state A_{k-1}    */
/* before the step).  The tape is then swept back to front with                */
/*   B^_k = (1 - alpha_k) B^_{k+1} + alpha_k c_k, B^_{N+1} = background,        */
/* and its x, y, xy derivatives.  With T = 1 - A_{k-1} and D = c_k - B^_{k+1}:  */
/*   P    = dI/dalpha_k           = T D                                         */
/*   P_x  = d2I/(dalpha_k dx)     = T_x D - T B^_x                              */
/*   P_xy = d3I/(dalpha_k dx dy)  = T_xy D - T_x B^_y - T_y B^_x - T B^_xy       */
/* (the passage writes 1 - A_k; the state before step k is meant), and for a  */
/* 2D parameter theta with Q = dalpha_k/dtheta:                                 */
/*   dI/dtheta = P Q,  dI_x/dtheta = P_x Q + P Q_x,                            */
/*   dI_xy/dtheta = P_xy Q + P_x Q_y + P_y Q_x + P Q_xy                         */
/* (the passage's third term pairs d2I/(dalpha dx) with d2alpha/(dsigma dx);   */
/* the y-derivative is meant).  Colour: dI/dc_k = T alpha_k and its x, y, xy    */
/* derivatives.  Q for alpha = sigma e^g, g = -1/2 (a dx^2 + 2 b dx dy + c dy^2):*/
/*   Q = alpha g_t, Q_x = alpha (g_x g_t + g_tx), Q_y = alpha (g_y g_t + g_ty),  */
/*   Q_xy = alpha (g_y (g_x g_t + g_tx) + g_xy g_t + g_x g_ty + g_txy)           */
/* with g_t = dg/dtheta etc.; for sigma, Q = alpha / sigma (and its x, y, xy    */
/* derivatives alike).  A clamped alpha (0.99) is a constant: Q = 0.           */
/* g2d layout per Gaussian: (mean_x, mean_y, conic a, conic b, conic c,        */
/* opacity, r, g, b); b is the off-diagonal entry of the conic.               */
/* ------------------------------------------------------------------------- */

typedef struct {
    uint32_t id;
    int clamped;
    double alpha, ax, ay, axy;
    double A, Ax, Ay, Axy;    /* state before the step */
    double dx, dy, gx, gy;
} TapeStep;

typedef struct {
    const RenderCtx* c;
    int64_t p0, p1;
    const int32_t* pix;
    const double* dout;    /* [npix][12] */
    double* g2d;           /* this worker's accumulator [n][9] */
    double* b2f;           /* [npix][12] back-to-front image, or NULL */
    TapeStep* tape;
    int64_t tape_cap;
} AdjJob;

static void adjoint_pixel(AdjJob* jb, int ix, int iy, const double u[12], double b2f[12])
{
    const RenderCtx* c = jb->c;
    const double px = ix + c->off_x, py = iy + c->off_y;
    const int64_t t = (int64_t)(iy / c->tile) * c->tiles_x + (ix / c->tile);
    const uint32_t start = c->ranges[2 * t], end = c->ranges[2 * t + 1];
    /* forward replay: the decisions of blend_pixel (no flips) */
    double A = 0.0, Ax = 0.0, Ay = 0.0, Axy = 0.0;
    int64_t ns = 0;
    for (uint32_t j = 0; j < end - start; ++j) {
        const uint32_t id = c->vals[start + j];
        const double dx = px - c->mean2d[2 * id], dy = py - c->mean2d[2 * id + 1];
        const double a = c->conic[3 * id], b = c->conic[3 * id + 1], cc = c->conic[3 * id + 2];
        const double g = -0.5 * (a * dx * dx + 2.0 * b * dx * dy + cc * dy * dy);
        const double gx = -(a * dx + b * dy), gy = -(b * dx + cc * dy), gxy = -b;
        double alpha = c->opacity[id] * exp(g);
        double ax = alpha * gx, ay = alpha * gy, axy = alpha * (gx * gy + gxy);
        int clamped = 0;
        if (c->mode == MODE_3DGS) {
            if (alpha < 1.0 / 255.0) continue;
            if (alpha > 0.99) { clamped = 1; alpha = 0.99; ax = 0.0; ay = 0.0; axy = 0.0; }
            if ((1.0 - A) * (1.0 - alpha) < 1e-4) break;
        }
        TapeStep* s = jb->tape + ns++;
        s->id = id; s->clamped = clamped;
        s->alpha = alpha; s->ax = ax; s->ay = ay; s->axy = axy;
        s->A = A; s->Ax = Ax; s->Ay = Ay; s->Axy = Axy;
        s->dx = dx; s->dy = dy; s->gx = gx; s->gy = gy;
        const double T = 1.0 - A;
        const double Axy_n = Axy * (1.0 - alpha) + T * axy - Ax * ay - Ay * ax;
        const double Ax_n = Ax * (1.0 - alpha) + T * ax;
        const double Ay_n = Ay * (1.0 - alpha) + T * ay;
        A = A + alpha * T; Ax = Ax_n; Ay = Ay_n; Axy = Axy_n;
    }
    /* back to front */
    double Bh[3], Bx[3], By[3], Bxy[3];
    for (int k = 0; k < 3; ++k) { Bh[k] = c->bg[k]; Bx[k] = 0.0; By[k] = 0.0; Bxy[k] = 0.0; }
    for (int64_t k = ns - 1; k >= 0; --k) {
        const TapeStep* s = jb->tape + k;
        const uint32_t id = s->id;
        const double T = 1.0 - s->A, Tx = -s->Ax, Ty = -s->Ay, Txy = -s->Axy;
        const double al = s->alpha, ax = s->ax, ay = s->ay, axy = s->axy;
        const double a = c->conic[3 * id], b = c->conic[3 * id + 1], cc = c->conic[3 * id + 2];
        const double dx = s->dx, dy = s->dy, gx = s->gx, gy = s->gy, gxy = -b;
        /* dg/dtheta, d2g/(dtheta dx), d2g/(dtheta dy), d3g/(dtheta dx dy) for
         * theta = mean_x, mean_y, a, b, c */
        const double gt[5] = {a * dx + b * dy, b * dx + cc * dy, -0.5 * dx * dx, -dx * dy, -0.5 * dy * dy};
        const double gtx[5] = {a, b, -dx, -dy, 0.0};
        const double gty[5] = {b, cc, 0.0, -dx, -dy};
        const double gtxy[5] = {0.0, 0.0, 0.0, -1.0, 0.0};
        double Q[6], Qx[6], Qy[6], Qxy[6];
        for (int p = 0; p < 5; ++p) {
            if (s->clamped) { Q[p] = Qx[p] = Qy[p] = Qxy[p] = 0.0; continue; }
            const double hx = gx * gt[p] + gtx[p];
            Q[p] = al * gt[p];
            Qx[p] = al * hx;
            Qy[p] = al * (gy * gt[p] + gty[p]);
            Qxy[p] = al * (gy * hx + gxy * gt[p] + gx * gty[p] + gtxy[p]);
        }
        const double sig = c->opacity[id];
        if (s->clamped || !(sig > 0.0)) { Q[5] = Qx[5] = Qy[5] = Qxy[5] = 0.0; }
        else { Q[5] = al / sig; Qx[5] = ax / sig; Qy[5] = ay / sig; Qxy[5] = axy / sig; }
        double* acc = jb->g2d + 9 * (int64_t)id;
        for (int ch = 0; ch < 3; ++ch) {
            const double col = c->rgb[3 * id + ch];
            const double D = col - Bh[ch];
            const double P = T * D;
            const double Px = Tx * D - T * Bx[ch];
            const double Py = Ty * D - T * By[ch];
            const double Pxy = Txy * D - Tx * By[ch] - Ty * Bx[ch] - T * Bxy[ch];
            const double uC = u[ch], uX = u[3 + ch], uY = u[6 + ch], uZ = u[9 + ch];
            for (int p = 0; p < 6; ++p)
                acc[p] += uC * P * Q[p] + uX * (Px * Q[p] + P * Qx[p]) + uY * (Py * Q[p] + P * Qy[p]) +
                          uZ * (Pxy * Q[p] + Px * Qy[p] + Py * Qx[p] + P * Qxy[p]);
            const double dc = T * al, dcx = Tx * al + T * ax, dcy = Ty * al + T * ay;
            const double dcxy = Txy * al + Tx * ay + Ty * ax + T * axy;
            acc[6 + ch] += uC * dc + uX * dcx + uY * dcy + uZ * dcxy;
            /* B^_k from B^_{k+1} */
            const double nBxy = (1.0 - al) * Bxy[ch] + axy * D - ay * Bx[ch] - ax * By[ch];
            const double nBx = (1.0 - al) * Bx[ch] + ax * D;
            const double nBy = (1.0 - al) * By[ch] + ay * D;
            const double nB = (1.0 - al) * Bh[ch] + al * col;
            Bh[ch] = nB; Bx[ch] = nBx; By[ch] = nBy; Bxy[ch] = nBxy;
        }
    }
    if (b2f)
        for (int k = 0; k < 3; ++k) { b2f[k] = Bh[k]; b2f[3 + k] = Bx[k]; b2f[6 + k] = By[k]; b2f[9 + k] = Bxy[k]; }
}

static void* adjoint_worker(void* arg)
{
    AdjJob* jb = (AdjJob*)arg;
    const RenderCtx* c = jb->c;
    for (int64_t p = jb->p0; p < jb->p1; ++p) {
        int ix, iy;
        if (jb->pix) { ix = jb->pix[2 * p]; iy = jb->pix[2 * p + 1]; }
        else { ix = (int)(p % c->W); iy = (int)(p / c->W); }
        adjoint_pixel(jb, ix, iy, jb->dout + 12 * p, jb->b2f ? jb->b2f + 12 * p : NULL);
    }
    return NULL;
}

int ora_render_adjoint(int W, int H, int tile, int mode, const double* bg,
                       const double* mean2d, const double* conic, const double* opacity, const double* rgb,
                       const uint32_t* vals, const uint32_t* ranges, int64_t n,
                       int64_t npix, const int32_t* pix, const double* dout,
                       double* g2d, double* b2f, int nthreads)
{
    if (W < 1 || H < 1 || tile < 1 || npix < 0 || n < 0) return ORA_EINVAL;
    if (pix == NULL && npix != (int64_t)W * H) return ORA_EINVAL;
    if (pix != NULL)
        for (int64_t p = 0; p < npix; ++p)
            if (pix[2 * p] < 0 || pix[2 * p] >= W || pix[2 * p + 1] < 0 || pix[2 * p + 1] >= H) return ORA_EINVAL;
    RenderCtx c;
    c.W = W; c.H = H; c.tile = tile; c.tiles_x = (W + tile - 1) / tile; c.mode = mode;
    for (int k = 0; k < 3; ++k) c.bg[k] = bg ? bg[k] : 0.0;
    c.off_x = 0.0; c.off_y = 0.0;
    c.mean2d = mean2d; c.conic = conic; c.opacity = opacity; c.rgb = rgb;
    c.vals = vals; c.ranges = ranges;
    /* the longest tile list bounds a pixel's tape */
    const int64_t T = (int64_t)c.tiles_x * ((H + tile - 1) / tile);
    int64_t cap = 1;
    for (int64_t k = 0; k < T; ++k)
        if ((int64_t)(ranges[2 * k + 1] - ranges[2 * k]) > cap) cap = ranges[2 * k + 1] - ranges[2 * k];
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > npix) nthreads = npix > 0 ? (int)npix : 1;
    AdjJob jobs[256];
    pthread_t th[256];
    int st = ORA_OK;
    for (int k = 0; k < nthreads; ++k) {
        jobs[k].c = &c;
        jobs[k].p0 = npix * k / nthreads;
        jobs[k].p1 = npix * (k + 1) / nthreads;
        jobs[k].pix = pix; jobs[k].dout = dout; jobs[k].b2f = b2f;
        jobs[k].g2d = (double*)calloc((size_t)(n > 0 ? n : 1) * 9, sizeof(double));
        jobs[k].tape = (TapeStep*)malloc(sizeof(TapeStep) * (size_t)cap);
        jobs[k].tape_cap = cap;
        if (!jobs[k].g2d || !jobs[k].tape) st = ORA_ENOMEM;
    }
    if (st == ORA_OK) {
        for (int k = 1; k < nthreads; ++k) pthread_create(&th[k], NULL, adjoint_worker, &jobs[k]);
        adjoint_worker(&jobs[0]);
        for (int k = 1; k < nthreads; ++k) pthread_join(th[k], NULL);
        for (int64_t q = 0; q < 9 * n; ++q) {
            double s = 0.0;
            for (int k = 0; k < nthreads; ++k) s += jobs[k].g2d[q];
            g2d[q] = s;
        }
    }
    for (int k = 0; k < nthreads; ++k) { free(jobs[k].g2d); free(jobs[k].tape); }
    return st;
}

/* ------------------------------------------------------------------------- */
/* Adjoint of the projection, by forward-mode differentiation of its          */
/* definition: every input of a Gaussian is seeded in turn with dual numbers   */
/* (value, derivative), the projection of ora_project is evaluated in dual     */
/* arithmetic, and the derivatives of (mean2D, conic, opacity, colour) are     */
/* contracted with the upstream g2d row.  Piecewise functions (the frustum     */
/* clamp of J, max(0, .) of the colour) take the derivative of the branch the  */
/* value takes.                                                                */
/* ------------------------------------------------------------------------- */

typedef struct { double v, d; } Dual;

static Dual dc(double v) { Dual r = {v, 0.0}; return r; }
static Dual dadd(Dual a, Dual b) { Dual r = {a.v + b.v, a.d + b.d}; return r; }
static Dual dsub(Dual a, Dual b) { Dual r = {a.v - b.v, a.d - b.d}; return r; }
static Dual dmul(Dual a, Dual b) { Dual r = {a.v * b.v, a.d * b.v + a.v * b.d}; return r; }
static Dual ddiv(Dual a, Dual b) { Dual r = {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; return r; }
static Dual dscale(Dual a, double s) { Dual r = {a.v * s, a.d * s}; return r; }
static Dual dsqrt(Dual a) { double s = sqrt(a.v); Dual r = {s, a.d / (2.0 * s)}; return r; }
static Dual dexp(Dual a) { double e = exp(a.v); Dual r = {e, a.d * e}; return r; }
static Dual dcos(Dual a) { Dual r = {cos(a.v), -sin(a.v) * a.d}; return r; }
static Dual dsin(Dual a) { Dual r = {sin(a.v), cos(a.v) * a.d}; return r; }
static Dual datan2(Dual y, Dual x)
{
    Dual r = {atan2(y.v, x.v), (x.v * y.d - y.v * x.d) / (x.v * x.v + y.v * y.v)};
    return r;
}
static Dual dclamp(Dual a, double lo, double hi)
{
    if (a.v < lo) return dc(lo);
    if (a.v > hi) return dc(hi);
    return a;
}

/* P_l^m(x) in dual arithmetic (same recurrences as legendre_p) */
static Dual legendre_dual(int l, int m, Dual x)
{
    Dual s = dsqrt(dclamp(dsub(dc(1.0), dmul(x, x)), 0.0, 1.0));
    Dual p_mm = dc(1.0);
    for (int i = 1; i <= m; ++i) p_mm = dmul(p_mm, dscale(s, -(double)(2 * i - 1)));
    if (l == m) return p_mm;
    Dual p_prev = p_mm;
    Dual p_cur = dmul(dscale(x, (double)(2 * m + 1)), p_mm);
    for (int ll = m + 2; ll <= l; ++ll) {
        Dual t1 = dmul(dscale(x, (double)(2 * ll - 1)), p_cur);
        Dual t2 = dscale(p_prev, (double)(ll + m - 1));
        Dual p_next = dscale(dsub(t1, t2), 1.0 / (double)(ll - m));
        p_prev = p_cur;
        p_cur = p_next;
    }
    return p_cur;
}

static void sh_basis_dual(int deg, const Dual dir[3], Dual* out)
{
    Dual nrm = dsqrt(dadd(dadd(dmul(dir[0], dir[0]), dmul(dir[1], dir[1])), dmul(dir[2], dir[2])));
    Dual x = ddiv(dir[0], nrm), y = ddiv(dir[1], nrm), z = ddiv(dir[2], nrm);
    Dual ct = dclamp(z, -1.0, 1.0);
    Dual ph = datan2(y, x);
    for (int l = 0; l <= deg; ++l)
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * fact(l - am) / fact(l + am));
            Dual P = legendre_dual(l, am, ct);
            Dual v;
            if (m == 0) v = dscale(P, K);
            else if (m > 0) v = dmul(dscale(P, sqrt(2.0) * K), dcos(dscale(ph, (double)am)));
            else v = dmul(dscale(P, sqrt(2.0) * K), dsin(dscale(ph, (double)am)));
            out[l * l + l + m] = v;
        }
}

typedef struct {
    double Rv[3][3], tv[3], campos[3];
    double fx, fy, cx, cy, znear, lim_x, lim_y;
} OraCam;

/* out: mean_x, mean_y, conic a, b, c, opacity, r, g, b.  Returns 0 if culled. */
static int project_one_dual(const OraCam* cam, const Dual mu[3], const Dual ls[3], const Dual q[4], Dual ol,
                            const Dual* sh, int deg, const Dual* rgb_in, Dual out[9])
{
    Dual p[3];
    for (int r = 0; r < 3; ++r)
        p[r] = dadd(dadd(dadd(dscale(mu[0], cam->Rv[r][0]), dscale(mu[1], cam->Rv[r][1])),
                         dscale(mu[2], cam->Rv[r][2])), dc(cam->tv[r]));
    if (p[2].v <= cam->znear) return 0;
    Dual qn = dsqrt(dadd(dadd(dmul(q[0], q[0]), dmul(q[1], q[1])), dadd(dmul(q[2], q[2]), dmul(q[3], q[3]))));
    if (!(qn.v > 0.0)) return 0;
    Dual w = ddiv(q[0], qn), x = ddiv(q[1], qn), y = ddiv(q[2], qn), z = ddiv(q[3], qn);
    Dual two = dc(2.0), one = dc(1.0);
    Dual R[3][3] = {
        {dsub(one, dmul(two, dadd(dmul(y, y), dmul(z, z)))), dmul(two, dsub(dmul(x, y), dmul(w, z))),
         dmul(two, dadd(dmul(x, z), dmul(w, y)))},
        {dmul(two, dadd(dmul(x, y), dmul(w, z))), dsub(one, dmul(two, dadd(dmul(x, x), dmul(z, z)))),
         dmul(two, dsub(dmul(y, z), dmul(w, x)))},
        {dmul(two, dsub(dmul(x, z), dmul(w, y))), dmul(two, dadd(dmul(y, z), dmul(w, x))),
         dsub(one, dmul(two, dadd(dmul(x, x), dmul(y, y))))}};
    Dual s2[3];
    for (int k = 0; k < 3; ++k) { Dual s = dexp(ls[k]); s2[k] = dmul(s, s); }
    Dual Sig[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            Dual acc = dc(0.0);
            for (int k = 0; k < 3; ++k) acc = dadd(acc, dmul(dmul(R[r][k], s2[k]), R[c][k]));
            Sig[r][c] = acc;
        }
    Dual tz = p[2];
    Dual txz = dclamp(ddiv(p[0], tz), -cam->lim_x, cam->lim_x);
    Dual tyz = dclamp(ddiv(p[1], tz), -cam->lim_y, cam->lim_y);
    Dual J[2][3] = {{ddiv(dc(cam->fx), tz), dc(0.0), dscale(ddiv(txz, tz), -cam->fx)},
                    {dc(0.0), ddiv(dc(cam->fy), tz), dscale(ddiv(tyz, tz), -cam->fy)}};
    Dual M[2][3];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c)
            M[r][c] = dadd(dadd(dscale(J[r][0], cam->Rv[0][c]), dscale(J[r][1], cam->Rv[1][c])),
                           dscale(J[r][2], cam->Rv[2][c]));
    Dual S2[2][2];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            Dual acc = dc(0.0);
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) acc = dadd(acc, dmul(dmul(M[r][k], Sig[k][l]), M[c][l]));
            S2[r][c] = acc;
        }
    S2[0][0] = dadd(S2[0][0], dc(0.3));
    S2[1][1] = dadd(S2[1][1], dc(0.3));
    Dual det = dsub(dmul(S2[0][0], S2[1][1]), dmul(S2[0][1], S2[1][0]));
    if (!(det.v > 0.0)) return 0;
    out[0] = dadd(dscale(ddiv(p[0], p[2]), cam->fx), dc(cam->cx));
    out[1] = dadd(dscale(ddiv(p[1], p[2]), cam->fy), dc(cam->cy));
    out[2] = ddiv(S2[1][1], det);
    out[3] = dscale(ddiv(S2[0][1], det), -1.0);
    out[4] = ddiv(S2[0][0], det);
    out[5] = ddiv(dc(1.0), dadd(dc(1.0), dexp(dscale(ol, -1.0))));
    if (sh) {
        Dual dir[3];
        for (int k = 0; k < 3; ++k) dir[k] = dsub(mu[k], dc(cam->campos[k]));
        Dual Y[16];
        sh_basis_dual(deg, dir, Y);
        const int K = (deg + 1) * (deg + 1);
        for (int ch = 0; ch < 3; ++ch) {
            Dual acc = dc(0.0);
            for (int k = 0; k < K; ++k) acc = dadd(acc, dmul(sh[3 * k + ch], Y[k]));
            acc = dadd(acc, dc(0.5));
            out[6 + ch] = acc.v > 0.0 ? acc : dc(0.0);
        }
    } else {
        for (int ch = 0; ch < 3; ++ch) out[6 + ch] = rgb_in[ch];
    }
    return 1;
}

/* g2d: [n][9] upstream; outputs (overwritten): g_means [n][3], g_log_scales
 * [n][3], g_quats [n][4], g_opacity_logits [n], g_sh [n][K][3] (if sh) or
 * g_rgb [n][3] (if rgb_in). */
int ora_project_adjoint(int64_t n, const double* means, const double* log_scales, const double* quats,
                        const double* opacity_logits, const double* sh, int sh_degree, const double* rgb_in,
                        const double* viewmat, double fx, double fy, double cx, double cy, double znear,
                        int W, int H, const double* g2d,
                        double* g_means, double* g_log_scales, double* g_quats, double* g_opacity_logits,
                        double* g_sh, double* g_rgb)
{
    if (n < 0 || W < 1 || H < 1 || sh_degree < 0 || sh_degree > 3) return ORA_EINVAL;
    if (sh == NULL && rgb_in == NULL && n > 0) return ORA_EINVAL;
    OraCam cam;
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) cam.Rv[r][c] = viewmat[4 * r + c];
        cam.tv[r] = viewmat[4 * r + 3];
    }
    for (int c = 0; c < 3; ++c)
        cam.campos[c] = -(cam.Rv[0][c] * cam.tv[0] + cam.Rv[1][c] * cam.tv[1] + cam.Rv[2][c] * cam.tv[2]);
    cam.fx = fx; cam.fy = fy; cam.cx = cx; cam.cy = cy; cam.znear = znear;
    cam.lim_x = 1.3 * ((double)W / (2.0 * fx));
    cam.lim_y = 1.3 * ((double)H / (2.0 * fy));
    const int K = (sh_degree + 1) * (sh_degree + 1);
    const int ncol = sh ? 3 * K : 3;
    const int npar = 3 + 3 + 4 + 1 + ncol;
    for (int64_t i = 0; i < n; ++i) {
        double grad[3 + 3 + 4 + 1 + 48];
        for (int j = 0; j < npar; ++j) {
            Dual mu[3], ls[3], q[4], ol, col[48];
            for (int k = 0; k < 3; ++k) { mu[k] = dc(means[3 * i + k]); ls[k] = dc(log_scales[3 * i + k]); }
            for (int k = 0; k < 4; ++k) q[k] = dc(quats[4 * i + k]);
            ol = dc(opacity_logits[i]);
            for (int k = 0; k < ncol; ++k) col[k] = dc(sh ? sh[i * ncol + k] : rgb_in[3 * i + k]);
            if (j < 3) mu[j].d = 1.0;
            else if (j < 6) ls[j - 3].d = 1.0;
            else if (j < 10) q[j - 6].d = 1.0;
            else if (j == 10) ol.d = 1.0;
            else col[j - 11].d = 1.0;
            Dual out[9];
            double gj = 0.0;
            if (project_one_dual(&cam, mu, ls, q, ol, sh ? col : NULL, sh_degree, sh ? NULL : col, out))
                for (int k = 0; k < 9; ++k) gj += g2d[9 * i + k] * out[k].d;
            grad[j] = gj;
        }
        for (int k = 0; k < 3; ++k) { g_means[3 * i + k] = grad[k]; g_log_scales[3 * i + k] = grad[3 + k]; }
        for (int k = 0; k < 4; ++k) g_quats[4 * i + k] = grad[6 + k];
        g_opacity_logits[i] = grad[10];
        for (int k = 0; k < ncol; ++k) {
            if (sh && g_sh) g_sh[i * ncol + k] = grad[11 + k];
            if (!sh && g_rgb) g_rgb[3 * i + k] = grad[11 + k];
        }
    }
    return ORA_OK;
}

/* ------------------------------------------------------------------------- */
/* Classical bicubic upscale, the comparator of Sec. 5 / Sec. 6: cubic         */
/* convolution (Keys) with parameter a on the colour samples alone,           */
/*   W(d) = (a + 2)|d|^3 - (a + 3)|d|^2 + 1            for |d| <= 1             */
/*   W(d) = a|d|^3 - 5a|d|^2 + 8a|d| - 4a              for 1 < |d| < 2          */
/* out(X, Y) = sum_{k,l = -1..2} W(t - k) W(u - l) f(clamp(i + k), clamp(j + l))  */
/* with the half-pixel map x = (X + 0.5) W / W2 - 0.5, i = floor(x), t = x - i,  */
/* sample indices clamped to the image.  a = -0.5 is the Hermite patch with    */
/* central-difference slopes (the finite-difference gradients of Sec. 5);     */
/* a = -0.75 is the kernel of PyTorch's bicubic interpolation used in the     */
/* paper's experiments (Sec. 6).  C: [3][H][W]; out: [npix][3].                */
/* ------------------------------------------------------------------------- */
static double keys_w(double d, double a)
{
    d = fabs(d);
    if (d <= 1.0) return ((a + 2.0) * d - (a + 3.0)) * d * d + 1.0;
    if (d < 2.0) return ((a * d - 5.0 * a) * d + 8.0 * a) * d - 4.0 * a;
    return 0.0;
}

int ora_bicubic(int W, int H, int W2, int H2, const double* C, double a, int64_t npix, const int32_t* pix,
                double* out)
{
    if (W < 1 || H < 1 || W2 < 1 || H2 < 1 || npix < 0) return ORA_EINVAL;
    if (pix == NULL && npix != (int64_t)W2 * H2) return ORA_EINVAL;
    const int64_t plane = (int64_t)W * H;
    for (int64_t p = 0; p < npix; ++p) {
        int X, Y;
        if (pix) { X = pix[2 * p]; Y = pix[2 * p + 1]; }
        else { X = (int)(p % W2); Y = (int)(p / W2); }
        if (X < 0 || X >= W2 || Y < 0 || Y >= H2) return ORA_EINVAL;
        const double x = ((double)X + 0.5) * (double)W / (double)W2 - 0.5;
        const double y = ((double)Y + 0.5) * (double)H / (double)H2 - 0.5;
        const int i = (int)floor(x), j = (int)floor(y);
        const double t = x - (double)i, u = y - (double)j;
        for (int ch = 0; ch < 3; ++ch) {
            double acc = 0.0;
            for (int l = -1; l <= 2; ++l) {
                int jj = j + l;
                jj = jj < 0 ? 0 : (jj > H - 1 ? H - 1 : jj);
                for (int k = -1; k <= 2; ++k) {
                    int ii = i + k;
                    ii = ii < 0 ? 0 : (ii > W - 1 ? W - 1 : ii);
                    acc += keys_w(t - (double)k, a) * keys_w(u - (double)l, a) *
                           C[(int64_t)ch * plane + (int64_t)jj * W + ii];
                }
            }
            out[3 * p + ch] = acc;
        }
    }
    return ORA_OK;
}
