/* Oracle (test infrastructure only): the two sequential algorithms of the LIDAR sample
 * update of Section III-B whose results are integers decided by floating point.  They run
 * in FP32 with a fixed operation order, so a second implementation that performs the same
 * FP32 operations reaches the same decisions.  Build with -ffp-contract=off (no fused
 * multiply-add) and without fast-math.
 *
 *  fs_select   Section III-B.1 (Floyd-Steinberg dithering of the belief map, Fig. 1c):
 *              raster order, left to right and top to bottom; value v = min(1, m * fs)
 *              plus the diffused error; selected iff value >= 0.5; the quantisation error
 *              goes 7/16 right, 3/16 down-left, 5/16 down, 1/16 down-right; error that
 *              would leave the grid is dropped.
 *  dda_cells   Expected range of a state for the likelihood P(z | x) of Eq. 9: walk the
 *              grid cells crossed by the ray from the centre of cell (j, i) along the unit
 *              direction (dx, dy) (Amanatides-Woo traversal) until an occupied cell or the
 *              grid edge; a tie between the next x and y crossings steps x first.  Returns
 *              the distance in cells, capped at rmax.
 *  range_table The expected-range table of the dense scan update: dda_cells from every cell
 *              along A fixed directions, quantised to 8 bits with the FP32 operations
 *              q = floor(t * inv_step + 0.5) (the product rounded, then the sum), capped
 *              at 255.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

int fs_select(const float* m, int H, int W, float fs, uint8_t* sel)
{
    float* E = (float*)calloc((size_t)H * (size_t)W, sizeof(float));
    if (!E) return -1;
    int count = 0;
    for (int j = 0; j < H; ++j) {
        for (int i = 0; i < W; ++i) {
            size_t q = (size_t)j * W + i;
            float v = m[q] * fs;
            if (v > 1.0f) v = 1.0f;
            float val = v + E[q];
            int on = val >= 0.5f;
            float err = on ? val - 1.0f : val;
            sel[q] = (uint8_t)on;
            count += on;
            if (i + 1 < W) E[q + 1] += err * 0.4375f;                 /* 7/16 */
            if (j + 1 < H) {
                if (i > 0) E[q + W - 1] += err * 0.1875f;             /* 3/16 */
                E[q + W] += err * 0.3125f;                            /* 5/16 */
                if (i + 1 < W) E[q + W + 1] += err * 0.0625f;         /* 1/16 */
            }
        }
    }
    free(E);
    return count;
}

float dda_cells(const uint8_t* occ, int H, int W, int j, int i, float dx, float dy, float rmax)
{
    if (occ[(size_t)j * W + i]) return 0.0f;
    int sx = dx > 0.0f ? 1 : -1;
    int sy = dy > 0.0f ? 1 : -1;
    float tdx = dx != 0.0f ? 1.0f / fabsf(dx) : INFINITY;
    float tdy = dy != 0.0f ? 1.0f / fabsf(dy) : INFINITY;
    int nx = 0, ny = 0;
    for (;;) {
        float tx = ((float)nx + 0.5f) * tdx;
        float ty = ((float)ny + 0.5f) * tdy;
        float t;
        if (tx <= ty) { i += sx; nx += 1; t = tx; }
        else          { j += sy; ny += 1; t = ty; }
        if (t >= rmax) return rmax;
        if (i < 0 || i >= W || j < 0 || j >= H) return t;
        if (occ[(size_t)j * W + i]) return t;
    }
}

/* Expected ranges in metres for every (sample, ray): out[s * n_rays + r] =
 * dda_cells(cell of sample s, dir r) * cell_m, all in FP32. */
void dda_ranges(const uint8_t* occ, int H, int W, const int32_t* cells, int n_cells,
                const float* dirs, int n_rays, float rmax_cells, float cell_m, float* out)
{
    for (int s = 0; s < n_cells; ++s) {
        int j = cells[s] / W, i = cells[s] % W;
        for (int r = 0; r < n_rays; ++r)
            out[(size_t)s * n_rays + r] =
                dda_cells(occ, H, W, j, i, dirs[2 * r], dirs[2 * r + 1], rmax_cells) * cell_m;
    }
}

/* out[(a * H + j) * W + i] = the 8-bit code of dda_cells(j, i, dirs[a]) (0 on occupied
 * cells, whose walk returns 0). */
void range_table(const uint8_t* occ, int H, int W, const float* dirs, int A, float rmax_cells,
                 float inv_step, uint8_t* out)
{
    for (int a = 0; a < A; ++a)
        for (int j = 0; j < H; ++j)
            for (int i = 0; i < W; ++i) {
                float t = dda_cells(occ, H, W, j, i, dirs[2 * a], dirs[2 * a + 1], rmax_cells);
                float x = t * inv_step;
                float y = x + 0.5f;
                float f = floorf(y);
                out[((size_t)a * H + j) * W + i] = (uint8_t)(f > 255.0f ? 255.0f : f);
            }
}
