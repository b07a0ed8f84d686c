/*
 * dibr_oracle.c -- reference CPU implementation of the pseudo-stereo (DIBR) pipeline.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct statement of what
 * the GPU path computes.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline may load it.  The product library never links, loads or calls it, and it
 * shares no code, header, table or constant with the CUDA sources.
 *
 * Single-threaded plain C99.  Integer steps are exact; the one floating-point step (the
 * cross-bilateral depth filter) runs in IEEE double precision.  Every function follows
 * the pipeline of the paper "3D Pseudo Stereo Visualization with GPGPU Support"
 * (Al-Oraiqat, Zori; arXiv 2009.09501):
 *
 *   Sec. 3 / Fig. 1 -- six components: depth map, filtered depth map, left frame, right
 *                      frame, post-processed (inpainted) left and right frames;
 *   Sec. 4          -- stage list: depth map, cross-bilateral filtering, left/right frame
 *                      reconstruction, left/right inpainting, stereo-pair formatting;
 *   Fig. 3          -- the per-pixel shift rule (threshold 150 on the filtered depth,
 *                      Base/2 scaling, out-of-range fallback) and the red-cyan channel map.
 *
 * Where the paper is silent the readings below are used (each is also a test pin):
 *   depth      = BT.601 luminance in exact thousandths, rounded half up;
 *   smoothing  = 5x5 binomial with clamp-to-edge (default), plain luminance, or the
 *                cross-bilateral filter of Sec. 3 with an RGB guide and clipped window;
 *   shift      = Fig. 3's expression as an exact rational, floored (forward warp) or
 *                truncated toward zero like Fig. 3's (int) cast (literal gather mode);
 *   occlusion  = larger depth is nearer and wins; equal depth prefers the smaller source
 *                column in the left view and the larger one in the right view;
 *   hole fill  = row-local copy of the nearer-to-background neighbour (Sec. 4 names a
 *                "simplified" inpainting for the GPU); plus the iterative 2-D block
 *                inpainting of Fig. 3's pseudo-code as a separate post-process.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Mode codes understood by the oracle.  They are the oracle's own; the values are chosen
 * to match the public C-ABI so that one parameter record can be handed to both sides. */
enum { OR_DEPTH_LUMA = 0, OR_DEPTH_BINOM5 = 1, OR_DEPTH_XBF = 2 };
enum { OR_DISP_PAPER = 0, OR_DISP_LINEAR = 1 };
enum { OR_WARP_FORWARD = 0, OR_WARP_GATHER_FIG3 = 1 };
/* Hole fill: the row-local copy alone, or followed by the iterative 2-D block inpainting
 * of Fig. 3 (inpaint2d_oracle.c) over the holes of each view. */
enum { OR_FILL_ROW = 0, OR_FILL_INPAINT2D = 1 };

typedef struct {
    int32_t depth_rule;      /* OR_DEPTH_* */
    int32_t disparity_rule;  /* OR_DISP_* */
    int32_t warp_mode;       /* OR_WARP_* */
    int32_t max_parallax;    /* P, the paper's "Base" (Fig. 3), pixels */
    int32_t threshold;       /* T, 150 in Fig. 3 */
    double  xbf_sigma_s;     /* spatial sigma of the cross-bilateral filter, pixels */
    double  xbf_sigma_r;     /* range sigma, RGB units */
    int32_t xbf_radius;      /* half width of the square window */
    int32_t fill_mode;       /* OR_FILL_* */
    int32_t inpaint_block;   /* side of the square blocks of the 2-D inpainting */
} or_params;

int64_t or_inpaint2d(const uint8_t *view, int W, int H, int64_t pitch, const uint8_t *damaged,
                     int64_t dpitch, int bw, int bh, uint8_t *out, int64_t out_pitch);

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* ---------------------------------------------------------------------------------
 * Depth map (Sec. 3 "Depth Map"; Sec. 4 "CPU Map generation").  The paper derives depth
 * from the image with a method of its earlier work that is not given; the depth here is
 * the pixel's luminance Y = 0.299 R + 0.587 G + 0.114 B, evaluated exactly as an integer
 * number of thousandths and rounded half up.
 * ------------------------------------------------------------------------------- */
void or_luma(const uint8_t *rgb, int W, int H, int64_t pitch, uint8_t *Y)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const uint8_t *p = rgb + (int64_t)y * pitch + 3 * (int64_t)x;
            int thousandths = 299 * p[0] + 587 * p[1] + 114 * p[2];
            Y[(int64_t)y * W + x] = (uint8_t)((thousandths + 500) / 1000);
        }
}

/* ---------------------------------------------------------------------------------
 * Filtered depth map (Sec. 3 "Filtered Depth Map", Sec. 4 "GPU Cross Bilateral
 * Filtering").  Default smoothing: separable binomial [1 4 6 4 1] x [1 4 6 4 1] / 256,
 * coordinates clamped to the image, result rounded half up.  Column pass first, then
 * row pass, both in exact integers.
 * ------------------------------------------------------------------------------- */
void or_smooth_binom5(const uint8_t *Y, int W, int H, uint8_t *D)
{
    static const int b[5] = {1, 4, 6, 4, 1};
    int32_t *V = (int32_t *)malloc(sizeof(int32_t) * (size_t)W * (size_t)H);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int s = 0;
            for (int i = -2; i <= 2; ++i)
                s += b[i + 2] * Y[(int64_t)clampi(y + i, 0, H - 1) * W + x];
            V[(int64_t)y * W + x] = s;
        }
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int s = 0;
            for (int j = -2; j <= 2; ++j)
                s += b[j + 2] * V[(int64_t)y * W + clampi(x + j, 0, W - 1)];
            D[(int64_t)y * W + x] = (uint8_t)((s + 128) >> 8);
        }
    free(V);
}

/* Cross-bilateral filtering of the depth map (Sec. 3, Sec. 4; the paper gives no
 * parameters).  Guide = the RGB image.  For output pixel p the window is the square
 * |dx|,|dy| <= r clipped to the image; each sample q is weighted by
 *   w = exp(-(dx^2+dy^2) / (2 sigma_s^2)) * exp(-|RGB(p)-RGB(q)|^2 / (2 sigma_r^2))
 * and D(p) = round-half-up( sum w Y(q) / sum w ).  Double precision throughout. */
void or_smooth_xbf(const uint8_t *rgb, int W, int H, int64_t pitch, const uint8_t *Y,
                   int r, double sigma_s, double sigma_r, uint8_t *D)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const uint8_t *cp = rgb + (int64_t)y * pitch + 3 * (int64_t)x;
            double num = 0.0, den = 0.0;
            for (int dy = -r; dy <= r; ++dy)
                for (int dx = -r; dx <= r; ++dx) {
                    int qy = y + dy, qx = x + dx;
                    if (qy < 0 || qy >= H || qx < 0 || qx >= W) continue;
                    const uint8_t *cq = rgb + (int64_t)qy * pitch + 3 * (int64_t)qx;
                    double dr = (double)cp[0] - cq[0], dg = (double)cp[1] - cq[1],
                           db = (double)cp[2] - cq[2];
                    double ws = exp(-(double)(dx * dx + dy * dy) / (2.0 * sigma_s * sigma_s));
                    double wr = exp(-(dr * dr + dg * dg + db * db) / (2.0 * sigma_r * sigma_r));
                    double w = ws * wr;
                    num += w * Y[(int64_t)qy * W + qx];
                    den += w;
                }
            double v = floor(num / den + 0.5);
            D[(int64_t)y * W + x] = (uint8_t)clampi((int)v, 0, 255);
        }
}

/* ---------------------------------------------------------------------------------
 * Depth -> shift (Fig. 3).  With T the threshold and P = Base the shift applied to the
 * left view's sampling position is
 *     s_L(d) = -(P/2) * d/255          if d > T
 *     s_L(d) =  (P/2) * (1 - d/255)    otherwise
 * and the right view uses s_R = -s_L.  Exact rational arithmetic: s_L = n_L / 510 with
 * n_L = -P d (d > T) or P (255 - d).  The forward warp uses h = floor(s); a source pixel
 * at column x lands on target column t = x - h.
 * Rule LINEAR (a monotone alternative with zero shift at zero depth): s_L = -P d / 510,
 * floored magnitude: h_L = -floor(P d / 510), h_R = +floor(P d / 510).
 * ------------------------------------------------------------------------------- */
static int64_t floor_div(int64_t a, int64_t b) /* b > 0 */
{
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0) q -= 1;
    return q;
}

/* numerator of s_L(d) over the common denominator 510 (Fig. 3 rule) */
static int64_t paper_shift_num(int d, int P, int T)
{
    return d > T ? -(int64_t)P * d : (int64_t)P * (255 - d);
}

void or_disparity_lut(int rule, int P, int T, int16_t *hL, int16_t *hR)
{
    for (int d = 0; d < 256; ++d) {
        if (rule == OR_DISP_PAPER) {
            int64_t n = paper_shift_num(d, P, T);
            hL[d] = (int16_t)floor_div(n, 510);
            hR[d] = (int16_t)floor_div(-n, 510);
        } else {
            int64_t m = ((int64_t)P * d) / 510;
            hL[d] = (int16_t)(-m);
            hR[d] = (int16_t)m;
        }
    }
}

/* ---------------------------------------------------------------------------------
 * Left/right frame reconstruction and row-local inpainting, one row of one view
 * (Sec. 3 "Left Frame", "Right Frame", "Post-Processed ... Frame"; Sec. 4).
 *
 * Forward warp: every source column x with depth d goes to t = x - h[d]; targets outside
 * [0, W) are dropped.  Occlusion: per target keep the source with the largest d; equal d
 * prefers the smaller x in the left view and the larger x in the right view.
 * Hole fill: an empty target t takes the nearest filled target l < t and r > t; when
 * both exist the one whose winning depth is smaller (farther, background side) is used,
 * l on a tie; with one side only that side; with none, the input pixel at t.  The colour
 * is that of the chosen target's winning source (a single-level copy).
 * out_src[t] receives the source column whose colour target t shows.
 * ------------------------------------------------------------------------------- */
static void warp_fill_row(const uint8_t *Drow, int W, const int16_t *h, int is_left,
                          int32_t *win_x, int32_t *win_d, int32_t *out_src)
{
    for (int t = 0; t < W; ++t) { win_x[t] = -1; win_d[t] = -1; }
    for (int x = 0; x < W; ++x) {
        int d = Drow[x];
        int t = x - h[d];
        if (t < 0 || t >= W) continue;
        int better;
        if (win_x[t] < 0) better = 1;
        else if (d != win_d[t]) better = d > win_d[t];
        else better = is_left ? (x < win_x[t]) : (x > win_x[t]);
        if (better) { win_x[t] = x; win_d[t] = d; }
    }
    for (int t = 0; t < W; ++t) {
        if (win_x[t] >= 0) { out_src[t] = win_x[t]; continue; }
        int l = t - 1, r = t + 1;
        while (l >= 0 && win_x[l] < 0) --l;
        while (r < W && win_x[r] < 0) ++r;
        int have_l = l >= 0, have_r = r < W;
        if (have_l && have_r) out_src[t] = (win_d[l] <= win_d[r]) ? win_x[l] : win_x[r];
        else if (have_l) out_src[t] = win_x[l];
        else if (have_r) out_src[t] = win_x[r];
        else out_src[t] = t;
    }
}

/* Literal gather of Fig. 3: target x samples column trunc(x + s(d)) of the source, d
 * being the target pixel's own filtered depth; out of range samples column x itself.
 * trunc is C's conversion toward zero, applied to the exact rational x + n/510. */
static void gather_row(const uint8_t *Drow, int W, int P, int T, int is_left, int32_t *out_src)
{
    for (int x = 0; x < W; ++x) {
        int64_t n = paper_shift_num(Drow[x], P, T);
        if (!is_left) n = -n;
        int64_t num = 510 * (int64_t)x + n;
        int64_t xs = num / 510; /* C99: truncation toward zero */
        out_src[x] = (xs >= 0 && xs < W) ? (int32_t)xs : x;
    }
}

/* Outputs of the stereo-pair formatting stage (Sec. 4 "GPU-Stereo 3D Pair formatting";
 * Figs. 4-5): red-cyan anaglyph (red from the left view, green and blue from the right
 * view, Fig. 3), full left and right views, anamorphic half side-by-side (each view
 * squeezed 2:1 horizontally by pairwise means rounded half up; left view in the left
 * half), the filtered depth map itself and the holes of the forward warp (one byte per
 * pixel: bit 0 a hole of the left view, bit 1 of the right view).  Any pointer may be
 * NULL. */
typedef struct {
    uint8_t *anaglyph, *left, *right, *hsbs, *depth, *holes;
    int64_t pitch;        /* bytes between rows of the RGB outputs */
    int64_t depth_pitch;  /* bytes between rows of the one-byte maps (depth, holes) */
} or_outputs;

/* One row of the formatted outputs from one row of each view. */
static void compose_row(const uint8_t *Lrow, const uint8_t *Rrow, int W, int y, const or_outputs *out)
{
    if (out->left) memcpy(out->left + (int64_t)y * out->pitch, Lrow, 3 * (size_t)W);
    if (out->right) memcpy(out->right + (int64_t)y * out->pitch, Rrow, 3 * (size_t)W);
    if (out->anaglyph) {
        uint8_t *a = out->anaglyph + (int64_t)y * out->pitch;
        for (int t = 0; t < W; ++t) {
            a[3 * t + 0] = Lrow[3 * t + 0];
            a[3 * t + 1] = Rrow[3 * t + 1];
            a[3 * t + 2] = Rrow[3 * t + 2];
        }
    }
    if (out->hsbs) {
        uint8_t *s = out->hsbs + (int64_t)y * out->pitch;
        int half = W / 2;
        for (int x = 0; x < W; ++x) {
            const uint8_t *v = x < half ? Lrow : Rrow;
            int k = x < half ? x : x - half;
            for (int c = 0; c < 3; ++c)
                s[3 * x + c] = (uint8_t)((v[3 * (2 * k) + c] + v[3 * (2 * k + 1) + c] + 1) >> 1);
        }
    }
}

/* The back half of the pipeline (warp, occlusion, fill, formatting) for a given depth
 * map D (W x H, tightly packed).  Returns 0, or -1 for invalid arguments.  The frame is
 * reconstructed whole first (both views and their holes), then -- with the 2-D fill
 * mode -- each view is inpainted, then the outputs are formatted. */
int or_from_depth(const uint8_t *rgb, int W, int H, int64_t pitch, const uint8_t *D,
                  const or_params *prm, const or_outputs *out)
{
    if (W < 1 || H < 1 || pitch < 3 * (int64_t)W) return -1;
    if (out->hsbs && (W & 1)) return -1;
    if (prm->fill_mode != OR_FILL_ROW && prm->fill_mode != OR_FILL_INPAINT2D) return -1;
    if (prm->fill_mode == OR_FILL_INPAINT2D && prm->inpaint_block < 1) return -1;
    int16_t hL[256], hR[256];
    or_disparity_lut(prm->disparity_rule, prm->max_parallax, prm->threshold, hL, hR);
    const size_t npx = (size_t)W * (size_t)H;
    int32_t *wx = (int32_t *)malloc(sizeof(int32_t) * (size_t)W);
    int32_t *wd = (int32_t *)malloc(sizeof(int32_t) * (size_t)W);
    int32_t *sL = (int32_t *)malloc(sizeof(int32_t) * (size_t)W);
    int32_t *sR = (int32_t *)malloc(sizeof(int32_t) * (size_t)W);
    uint8_t *Lv = (uint8_t *)malloc(3 * npx), *Rv = (uint8_t *)malloc(3 * npx);
    uint8_t *holeL = (uint8_t *)calloc(npx, 1), *holeR = (uint8_t *)calloc(npx, 1);
    for (int y = 0; y < H; ++y) {
        const uint8_t *Drow = D + (int64_t)y * W;
        const uint8_t *Irow = rgb + (int64_t)y * pitch;
        if (prm->warp_mode == OR_WARP_GATHER_FIG3) {
            gather_row(Drow, W, prm->max_parallax, prm->threshold, 1, sL);
            gather_row(Drow, W, prm->max_parallax, prm->threshold, 0, sR);
        } else {
            warp_fill_row(Drow, W, hL, 1, wx, wd, sL);
            for (int t = 0; t < W; ++t) holeL[(size_t)y * W + t] = wx[t] < 0;
            warp_fill_row(Drow, W, hR, 0, wx, wd, sR);
            for (int t = 0; t < W; ++t) holeR[(size_t)y * W + t] = wx[t] < 0;
        }
        for (int t = 0; t < W; ++t)
            for (int c = 0; c < 3; ++c) {
                Lv[3 * ((size_t)y * W + t) + c] = Irow[3 * sL[t] + c];
                Rv[3 * ((size_t)y * W + t) + c] = Irow[3 * sR[t] + c];
            }
    }
    if (prm->fill_mode == OR_FILL_INPAINT2D) {
        uint8_t *tmp = (uint8_t *)malloc(3 * npx);
        const int b = prm->inpaint_block;
        or_inpaint2d(Lv, W, H, 3 * (int64_t)W, holeL, W, b, b, tmp, 3 * (int64_t)W);
        memcpy(Lv, tmp, 3 * npx);
        or_inpaint2d(Rv, W, H, 3 * (int64_t)W, holeR, W, b, b, tmp, 3 * (int64_t)W);
        memcpy(Rv, tmp, 3 * npx);
        free(tmp);
    }
    for (int y = 0; y < H; ++y) {
        compose_row(Lv + 3 * (size_t)y * W, Rv + 3 * (size_t)y * W, W, y, out);
        if (out->depth) memcpy(out->depth + (int64_t)y * out->depth_pitch, D + (int64_t)y * W, (size_t)W);
        if (out->holes)
            for (int t = 0; t < W; ++t)
                out->holes[(int64_t)y * out->depth_pitch + t] =
                    (uint8_t)(holeL[(size_t)y * W + t] | (holeR[(size_t)y * W + t] << 1));
    }
    free(wx); free(wd); free(sL); free(sR); free(Lv); free(Rv); free(holeL); free(holeR);
    return 0;
}

/* Front half: depth map and its smoothing.  D receives W x H bytes, tightly packed. */
int or_depth(const uint8_t *rgb, int W, int H, int64_t pitch, const or_params *prm, uint8_t *D)
{
    if (W < 1 || H < 1 || pitch < 3 * (int64_t)W) return -1;
    uint8_t *Y = (uint8_t *)malloc((size_t)W * (size_t)H);
    or_luma(rgb, W, H, pitch, Y);
    if (prm->depth_rule == OR_DEPTH_LUMA) memcpy(D, Y, (size_t)W * (size_t)H);
    else if (prm->depth_rule == OR_DEPTH_BINOM5) or_smooth_binom5(Y, W, H, D);
    else if (prm->depth_rule == OR_DEPTH_XBF)
        or_smooth_xbf(rgb, W, H, pitch, Y, prm->xbf_radius, prm->xbf_sigma_s, prm->xbf_sigma_r, D);
    else { free(Y); return -1; }
    free(Y);
    return 0;
}

/* The whole pipeline for one image. */
int or_dibr(const uint8_t *rgb, int W, int H, int64_t pitch, const or_params *prm,
            const or_outputs *out)
{
    if (W < 1 || H < 1 || pitch < 3 * (int64_t)W) return -1;
    uint8_t *D = (uint8_t *)malloc((size_t)W * (size_t)H);
    int rc = or_depth(rgb, W, H, pitch, prm, D);
    if (rc == 0) rc = or_from_depth(rgb, W, H, pitch, D, prm, out);
    free(D);
    return rc;
}

/* Rows [y0, y1) of the whole pipeline, for a band-parallel CPU driver: the depth of a
 * band needs two rows of context on either side, which this function reads itself.
 * Outputs are written for rows y0..y1-1 only (pointers address row 0 of the image). */
int or_dibr_rows(const uint8_t *rgb, int W, int H, int64_t pitch, const or_params *prm,
                 const or_outputs *out, int y0, int y1)
{
    if (y0 < 0 || y1 > H || y0 >= y1) return -1;
    if (prm->fill_mode != OR_FILL_ROW) return -1; /* the 2-D fill is not row-local */
    int ctx = prm->depth_rule == OR_DEPTH_XBF ? prm->xbf_radius : 2;
    int a = y0 - ctx < 0 ? 0 : y0 - ctx;
    int b = y1 + ctx > H ? H : y1 + ctx;
    /* Rows outside [a, b) never influence rows [y0, y1): the filters reach ctx rows and
     * clamp at the image edge, which the sub-image reproduces only when it touches the
     * edge, so the sub-image is cut at the true image edges. */
    int hb = b - a;
    uint8_t *D = (uint8_t *)malloc((size_t)W * (size_t)hb);
    int rc = or_depth(rgb + (int64_t)a * pitch, W, hb, pitch, prm, D);
    if (rc == 0) {
        or_outputs o = *out;
        int64_t off = (int64_t)y0 * out->pitch, doff = (int64_t)y0 * out->depth_pitch;
        if (o.anaglyph) o.anaglyph += off;
        if (o.left) o.left += off;
        if (o.right) o.right += off;
        if (o.hsbs) o.hsbs += off;
        if (o.depth) o.depth += doff;
        if (o.holes) o.holes += doff;
        rc = or_from_depth(rgb + (int64_t)y0 * pitch, W, y1 - y0, pitch,
                           D + (int64_t)(y0 - a) * W, prm, &o);
    }
    free(D);
    return rc;
}
