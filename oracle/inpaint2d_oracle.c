/*
 * inpaint2d_oracle.c -- the iterative 2-D block inpainting of the paper, as a plain CPU
 * statement.  TEST INFRASTRUCTURE ONLY: only the test suite, the smoke check and the
 * benchmark's CPU baseline may load it; the product library never links or calls it and
 * shares no code with it.
 *
 * Paper: "3D Pseudo Stereo Visualization with GPGPU Support" (arXiv 2009.09501), Sec. 3
 * (post-processed left / right frames remove the holes of the reconstructed frames) and
 * Fig. 3, left column (the inpainting algorithm).  The algorithm as given:
 *
 *   the frame is cut into blocks; for every block, a private matrix of the frame's pixels
 *   is initialised and the block's damaged pixels are listed, the block's columns in the
 *   outer loop and its rows in the inner loop; then, while damaged pixels remain, the
 *   list is walked in order and every still-damaged pixel with at least two undamaged
 *   neighbours is marked undamaged, its count is decremented and its colour is computed
 *   and stored.
 *
 * Readings where the figure is silent (each is pinned by a test):
 *   damaged      = a target of the forward warp on which no source landed (a hole);
 *   neighbours   = the 8-connected neighbourhood, inside the frame;
 *   matrix       = per block, a copy of the whole frame taken before the block is
 *                  processed: pixels outside the block are seen in that initial state
 *                  and never change, so blocks are independent of each other;
 *   in the pass  = a pixel repaired earlier in the same walk of the list already counts
 *                  as undamaged, with its new colour, for the pixels after it;
 *   colour       = per channel, the mean of the undamaged neighbours' colours rounded
 *                  half up: floor((2 * sum + n) / (2 * n));
 *   termination  = the walk repeats while damaged pixels remain and the previous walk
 *                  repaired at least one (without that condition the figure's loop
 *                  would never end for a block whose damaged pixels cannot reach two
 *                  undamaged neighbours); pixels still damaged then keep the colour
 *                  they came with.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Inpaints one view.
 *   view, pitch      : W x H interleaved RGB, the frame as reconstructed (holes carry
 *                      whatever colour the reconstruction left there);
 *   damaged, dpitch  : W x H bytes, non-zero = damaged;
 *   bw, bh           : block width and height (>= 1);
 *   out, out_pitch   : W x H RGB result (may not alias view).
 * Returns the number of pixels left damaged, or -1 for invalid arguments. */
int64_t or_inpaint2d(const uint8_t *view, int W, int H, int64_t pitch, const uint8_t *damaged,
                     int64_t dpitch, int bw, int bh, uint8_t *out, int64_t out_pitch)
{
    if (W < 1 || H < 1 || bw < 1 || bh < 1 || pitch < 3 * (int64_t)W || dpitch < W ||
        out_pitch < 3 * (int64_t)W)
        return -1;
    for (int y = 0; y < H; ++y) memcpy(out + (int64_t)y * out_pitch, view + (int64_t)y * pitch, 3 * (size_t)W);

    /* the block's private matrix: colours and damage flags of the block plus a one-pixel
     * frame around it (the only pixels outside the block a neighbourhood reaches) */
    const int mw = bw + 2, mh = bh + 2;
    uint8_t *mc = (uint8_t *)malloc(3 * (size_t)mw * (size_t)mh);
    uint8_t *md = (uint8_t *)malloc((size_t)mw * (size_t)mh);
    int32_t *list = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)bw * (size_t)bh);
    int64_t left = 0;

    for (int by = 0; by < H; by += bh)
        for (int bx = 0; bx < W; bx += bw) {
            const int ew = bx + bw <= W ? bw : W - bx, eh = by + bh <= H ? bh : H - by;
            /* initialise the matrix: matrix cell (i, j) holds frame pixel (bx - 1 + i, by - 1 + j);
             * cells outside the frame are marked absent (2) */
            for (int j = 0; j < mh; ++j)
                for (int i = 0; i < mw; ++i) {
                    const int x = bx - 1 + i, y = by - 1 + j;
                    uint8_t *c = mc + 3 * ((size_t)j * mw + i);
                    if (x < 0 || y < 0 || x >= W || y >= H) {
                        md[(size_t)j * mw + i] = 2;
                        c[0] = c[1] = c[2] = 0;
                        continue;
                    }
                    md[(size_t)j * mw + i] = damaged[(int64_t)y * dpitch + x] ? 1 : 0;
                    memcpy(c, view + (int64_t)y * pitch + 3 * (int64_t)x, 3);
                }
            /* the list of damaged pixels: block columns outer, rows inner */
            int n = 0;
            for (int i = 0; i < ew; ++i)
                for (int j = 0; j < eh; ++j)
                    if (md[(size_t)(j + 1) * mw + (i + 1)] == 1) {
                        list[2 * n] = i + 1;
                        list[2 * n + 1] = j + 1;
                        ++n;
                    }
            int remaining = n, repaired;
            do {
                repaired = 0;
                for (int k = 0; k < n; ++k) {
                    const int i = list[2 * k], j = list[2 * k + 1];
                    if (md[(size_t)j * mw + i] != 1) continue;
                    int cnt = 0, sum[3] = {0, 0, 0};
                    for (int dj = -1; dj <= 1; ++dj)
                        for (int di = -1; di <= 1; ++di) {
                            if (!di && !dj) continue;
                            const size_t q = (size_t)(j + dj) * mw + (i + di);
                            if (md[q] != 0) continue; /* damaged, or outside the frame */
                            ++cnt;
                            for (int c = 0; c < 3; ++c) sum[c] += mc[3 * q + c];
                        }
                    if (cnt < 2) continue;
                    md[(size_t)j * mw + i] = 0;
                    --remaining;
                    ++repaired;
                    for (int c = 0; c < 3; ++c)
                        mc[3 * ((size_t)j * mw + i) + c] = (uint8_t)((2 * sum[c] + cnt) / (2 * cnt));
                }
            } while (remaining > 0 && repaired > 0);
            left += remaining;
            /* the block's pixels of the matrix are the result */
            for (int j = 0; j < eh; ++j)
                for (int i = 0; i < ew; ++i)
                    memcpy(out + (int64_t)(by + j) * out_pitch + 3 * (int64_t)(bx + i),
                           mc + 3 * ((size_t)(j + 1) * mw + (i + 1)), 3);
        }
    free(mc);
    free(md);
    free(list);
    return left;
}
