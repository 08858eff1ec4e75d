/*
 * FP64 CPU oracle: front-to-back alpha blending of projected Gaussians, its
 * exact adjoint, and a per-pixel brute-force renderer.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library path links or calls this
 * file; only the tests, the smoke check and the bench's CPU-baseline leg do.
 * It shares no code, header or constant with the CUDA path.
 *
 * What it computes (Sec. 3.1, the compositing the method inherits from 3DGS):
 *   C = sum_i c_i alpha_i prod_{j<i} (1 - alpha_j)  (+ T_final * bg)
 *   alpha_i = min(0.99, o'_i * exp(power_i)),
 *   power_i = -1/2 (A dx^2 + C dy^2) - B dx dy,  d = pixel - centre_i,
 * with the inherited rules: power > 0 skips the pair, alpha < 1/255 skips the
 * pair, and the walk stops, without blending, at the first pair whose
 * transmittance after blending would fall below 1e-4.
 *
 * Pixel (px, py) is evaluated at index coordinates (px, py); the projected
 * centres handed in already carry the -0.5 pixel-centre shift.
 *
 * Ambiguity flags: the GPU decides the same thresholds in binary32, so a pair
 * whose FP64 value lies within a small relative band of a threshold may be
 * decided the other way there. Every pixel that meets such a pair before its
 * walk ends is flagged; the parity tests treat those pixels separately.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TILE 16

static const double ALPHA_MIN = 1.0 / 255.0;
static const double ALPHA_MAX = 0.99;
static const double T_STOP = 1e-4;

/* relative half-width of the ambiguity band around each threshold */
static double g_band_alpha = 2e-5;
static double g_band_T = 5e-5;
static double g_band_power = 1e-6;

void orc_set_bands(double band_alpha, double band_T, double band_power)
{
    g_band_alpha = band_alpha;
    g_band_T = band_T;
    g_band_power = band_power;
}

typedef struct {
    const double *xy;     /* [N][2] */
    const double *conic;  /* [N][3]  A, B, C */
    const double *op;     /* [N]     o' = m_g * o */
    const double *rgb;    /* [N][3] */
} orc_gauss2d;

/* One pixel's front-to-back walk over `n` Gaussians listed in `ids`.
 * Records the contributing pairs when `rec_*` is non-null. */
static int walk_pixel(const orc_gauss2d *g, const int64_t *ids, int64_t n,
                      double px, double py, double *out_c, double *out_T,
                      int64_t *out_last, int *amb,
                      int64_t *rec_k, double *rec_alpha, double *rec_T,
                      double *rec_G, int *rec_clamped, int64_t *n_rec,
                      uint64_t *sig)
{
    double T = 1.0, c[3] = {0.0, 0.0, 0.0};
    int64_t last = 0, nr = 0;
    uint64_t h = 1469598103934665603ull;
    int a = 0;
    for (int64_t k = 0; k < n; ++k) {
        const int64_t id = ids[k];
        const double dx = px - g->xy[2 * id + 0];
        const double dy = py - g->xy[2 * id + 1];
        const double A = g->conic[3 * id + 0];
        const double B = g->conic[3 * id + 1];
        const double C = g->conic[3 * id + 2];
        const double power = -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy;
        if (fabs(power) <= g_band_power) a = 1;
        if (power > 0.0) continue;
        const double G = exp(power);
        const double ag = g->op[id] * G;
        if (fabs(ag - ALPHA_MAX) <= g_band_alpha * ALPHA_MAX) a = 1;
        const int clamped = ag > ALPHA_MAX;
        const double alpha = clamped ? ALPHA_MAX : ag;
        if (fabs(alpha - ALPHA_MIN) <= g_band_alpha * ALPHA_MIN) a = 1;
        if (alpha < ALPHA_MIN) continue;
        const double Tn = T * (1.0 - alpha);
        if (fabs(Tn - T_STOP) <= g_band_T * T_STOP) a = 1;
        if (Tn < T_STOP) break;
        for (int ch = 0; ch < 3; ++ch) c[ch] += g->rgb[3 * id + ch] * alpha * T;
        if (rec_k) {
            rec_k[nr] = k;
            rec_alpha[nr] = alpha;
            rec_T[nr] = T;
            rec_G[nr] = G;
            rec_clamped[nr] = clamped;
        }
        ++nr;
        h = (h ^ (uint64_t)(k + 1)) * 1099511628211ull;
        T = Tn;
        last = k + 1;
    }
    out_c[0] = c[0];
    out_c[1] = c[1];
    out_c[2] = c[2];
    *out_T = T;
    *out_last = last;
    *amb = a;
    if (n_rec) *n_rec = nr;
    if (sig) *sig = h;
    return 0;
}

/*
 * Tiled forward. ranges[2*t], ranges[2*t+1] delimit tile t's list inside ids[].
 * tile_sel (may be null = all tiles) selects which tiles are rendered; pixels
 * of unselected tiles are left untouched.
 * img: [3][H][W], T_final/last/amb/sig: [H][W].
 */
/*
 * Importance (App. A.2, importance-based selection): the sum over rays of a
 * Gaussian's blend weight w = alpha_i T_i. Added into weight[id] when the
 * pointer is non-null.
 */
static void add_weights(const int64_t *ids, const int64_t *rk, const double *ra,
                        const double *rT, int64_t nr, double *weight)
{
    for (int64_t i = 0; i < nr; ++i) {
        const double w = ra[i] * rT[i];
#pragma omp atomic
        weight[ids[rk[i]]] += w;
    }
}

void orc_blend_forward(int W, int H, const int64_t *ranges, const int64_t *ids,
                       const double *xy, const double *conic, const double *op,
                       const double *rgb, const double *bg, const uint8_t *tile_sel,
                       double *img, double *T_final, int64_t *last, uint8_t *amb,
                       uint64_t *sig, double *weight)
{
    const orc_gauss2d g = {xy, conic, op, rgb};
    const int tx_n = (W + ORC_TILE - 1) / ORC_TILE;
    const int ty_n = (H + ORC_TILE - 1) / ORC_TILE;
    const int64_t HW = (int64_t)H * W;
    int64_t max_len = 0;
    for (int t = 0; t < tx_n * ty_n; ++t) {
        const int64_t len = ranges[2 * t + 1] - ranges[2 * t];
        if (len > max_len) max_len = len;
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < tx_n * ty_n; ++t) {
        if (tile_sel && !tile_sel[t]) continue;
        const int tx = t % tx_n, ty = t / tx_n;
        const int64_t s = ranges[2 * t], e = ranges[2 * t + 1];
        int64_t *rk = 0;
        double *ra = 0, *rT = 0, *rG = 0;
        int *rc = 0;
        if (weight) {
            rk = (int64_t *)malloc(sizeof(int64_t) * (size_t)(max_len + 1));
            ra = (double *)malloc(sizeof(double) * (size_t)(max_len + 1));
            rT = (double *)malloc(sizeof(double) * (size_t)(max_len + 1));
            rG = (double *)malloc(sizeof(double) * (size_t)(max_len + 1));
            rc = (int *)malloc(sizeof(int) * (size_t)(max_len + 1));
        }
        for (int py = ty * ORC_TILE; py < (ty + 1) * ORC_TILE && py < H; ++py)
            for (int px = tx * ORC_TILE; px < (tx + 1) * ORC_TILE && px < W; ++px) {
                double c[3], T;
                int64_t l, nr = 0;
                int a;
                uint64_t h;
                walk_pixel(&g, ids + s, e - s, (double)px, (double)py, c, &T, &l, &a,
                           rk, ra, rT, rG, rc, weight ? &nr : 0, &h);
                if (weight) add_weights(ids + s, rk, ra, rT, nr, weight);
                const int64_t p = (int64_t)py * W + px;
                for (int ch = 0; ch < 3; ++ch) img[ch * HW + p] = c[ch] + T * bg[ch];
                T_final[p] = T;
                last[p] = l;
                amb[p] = (uint8_t)a;
                if (sig) sig[p] = h;
            }
        free(rk);
        free(ra);
        free(rT);
        free(rG);
        free(rc);
    }
}

/*
 * Adjoint of orc_blend_forward for the loss L = sum(dimg * img). Accumulates
 * dL/d(xy, conic, o', rgb) per Gaussian (arrays are added to, not cleared);
 * tiles run in parallel, so the FP64 summation order varies from run to run.
 * Exact derivative of the walk as written: zero through the skips, the stop,
 * and on the clamped branch of the 0.99 alpha clamp.
 */
void orc_blend_backward(int W, int H, const int64_t *ranges, const int64_t *ids,
                        const double *xy, const double *conic, const double *op,
                        const double *rgb, const double *bg, const uint8_t *tile_sel,
                        const double *dimg, double *dxy, double *dconic, double *dop,
                        double *drgb)
{
    const orc_gauss2d g = {xy, conic, op, rgb};
    const int tx_n = (W + ORC_TILE - 1) / ORC_TILE;
    const int ty_n = (H + ORC_TILE - 1) / ORC_TILE;
    const int64_t HW = (int64_t)H * W;
    int64_t max_len = 0;
    for (int t = 0; t < tx_n * ty_n; ++t) {
        const int64_t len = ranges[2 * t + 1] - ranges[2 * t];
        if (len > max_len) max_len = len;
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < tx_n * ty_n; ++t) {
        if (tile_sel && !tile_sel[t]) continue;
        const int tx = t % tx_n, ty = t / tx_n;
        const int64_t s = ranges[2 * t], e = ranges[2 * t + 1];
        int64_t *rk = (int64_t *)malloc(sizeof(int64_t) * (size_t)(max_len + 1));
        double *ra = (double *)malloc(sizeof(double) * (size_t)(max_len + 1));
        double *rT = (double *)malloc(sizeof(double) * (size_t)(max_len + 1));
        double *rG = (double *)malloc(sizeof(double) * (size_t)(max_len + 1));
        int *rc = (int *)malloc(sizeof(int) * (size_t)(max_len + 1));
        for (int py = ty * ORC_TILE; py < (ty + 1) * ORC_TILE && py < H; ++py)
            for (int px = tx * ORC_TILE; px < (tx + 1) * ORC_TILE && px < W; ++px) {
                double c[3], Tf;
                int64_t l, nr;
                int a;
                walk_pixel(&g, ids + s, e - s, (double)px, (double)py, c, &Tf, &l, &a,
                           rk, ra, rT, rG, rc, &nr, 0);
                const int64_t p = (int64_t)py * W + px;
                const double gc[3] = {dimg[p], dimg[HW + p], dimg[2 * HW + p]};
                /* suffix S = sum_{k>i} c_k alpha_k T_k, walked from the back */
                double S[3] = {0.0, 0.0, 0.0};
                for (int64_t i = nr - 1; i >= 0; --i) {
                    const int64_t id = ids[s + rk[i]];
                    const double al = ra[i], Ti = rT[i];
                    double dalpha = 0.0;
                    for (int ch = 0; ch < 3; ++ch) {
                        const double ci = rgb[3 * id + ch];
                        {
                        const double v_ = al * Ti * gc[ch];
#pragma omp atomic
                        drgb[3 * id + ch] += v_;
                    }
                        dalpha += gc[ch] * (ci * Ti - (S[ch] + Tf * bg[ch]) / (1.0 - al));
                        S[ch] += ci * al * Ti;
                    }
                    if (rc[i]) continue; /* alpha = 0.99 constant on this branch */
                    const double G = rG[i];
                    {
                        const double v_ = dalpha * G;
#pragma omp atomic
                        dop[id] += v_;
                    }
                    const double dpower = dalpha * op[id] * G;
                    const double dx = (double)px - xy[2 * id + 0];
                    const double dy = (double)py - xy[2 * id + 1];
                    const double A = conic[3 * id + 0], B = conic[3 * id + 1],
                                 C = conic[3 * id + 2];
                    {
                        const double v_ = dpower * (-0.5 * dx * dx);
#pragma omp atomic
                        dconic[3 * id + 0] += v_;
                    }
                    {
                        const double v_ = dpower * (-dx * dy);
#pragma omp atomic
                        dconic[3 * id + 1] += v_;
                    }
                    {
                        const double v_ = dpower * (-0.5 * dy * dy);
#pragma omp atomic
                        dconic[3 * id + 2] += v_;
                    }
                    /* d power / d dx = -(A dx + B dy); d dx / d x_centre = -1 */
                    {
                        const double v_ = dpower * (A * dx + B * dy);
#pragma omp atomic
                        dxy[2 * id + 0] += v_;
                    }
                    {
                        const double v_ = dpower * (C * dy + B * dx);
#pragma omp atomic
                        dxy[2 * id + 1] += v_;
                    }
                }
            }
        free(rk);
        free(ra);
        free(rT);
        free(rG);
        free(rc);
    }
}

/* ------------------------------------------------------------------------ */
/* Brute force: every pixel walks ALL Gaussians in global (depth key, id)    */
/* order, keeping those whose tile rectangle contains the pixel's tile.      */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint32_t depth_bits;
    int64_t id;
} orc_key;

static int cmp_key(const void *a, const void *b)
{
    const orc_key *x = (const orc_key *)a, *y = (const orc_key *)b;
    if (x->depth_bits != y->depth_bits) return x->depth_bits < y->depth_bits ? -1 : 1;
    return (x->id > y->id) - (x->id < y->id);
}

/*
 * rect: [N][4] = x0, y0, x1, y1 in tiles (half-open); visible: [N] (0 = culled).
 * gate = 0 drops the footprint test (every visible Gaussian reaches every
 * pixel), which gives the "full support" image.
 */
void orc_brute_force(int N, int W, int H, const uint32_t *depth_bits,
                     const int32_t *rect, const uint8_t *visible, const double *xy,
                     const double *conic, const double *op, const double *rgb,
                     const double *bg, int gate, double *img, double *T_final,
                     int64_t *last)
{
    const orc_gauss2d g = {xy, conic, op, rgb};
    orc_key *keys = (orc_key *)malloc(sizeof(orc_key) * (size_t)(N > 0 ? N : 1));
    int64_t nv = 0;
    for (int i = 0; i < N; ++i)
        if (visible[i]) {
            keys[nv].depth_bits = depth_bits[i];
            keys[nv].id = i;
            ++nv;
        }
    qsort(keys, (size_t)nv, sizeof(orc_key), cmp_key);
    const int64_t HW = (int64_t)H * W;
#pragma omp parallel
    {
        int64_t *list = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nv > 0 ? nv : 1));
#pragma omp for schedule(dynamic, 16)
        for (int py = 0; py < H; ++py)
            for (int px = 0; px < W; ++px) {
                const int tx = px / ORC_TILE, ty = py / ORC_TILE;
                int64_t n = 0;
                for (int64_t k = 0; k < nv; ++k) {
                    const int64_t id = keys[k].id;
                    const int32_t *r = rect + 4 * id;
                    if (!gate || (tx >= r[0] && tx < r[2] && ty >= r[1] && ty < r[3]))
                        list[n++] = id;
                }
                double c[3], T;
                int64_t l;
                int a;
                walk_pixel(&g, list, n, (double)px, (double)py, c, &T, &l, &a, 0, 0, 0, 0,
                           0, 0, 0);
                const int64_t p = (int64_t)py * W + px;
                for (int ch = 0; ch < 3; ++ch) img[ch * HW + p] = c[ch] + T * bg[ch];
                T_final[p] = T;
                last[p] = l;
            }
        free(list);
    }
    free(keys);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads the blend loops use from now on (n >= 1). */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
