/* Oracle (test infrastructure only): Algorithm 1's propagation of every channel in FP64,
 * the direct sums of oracle/filter.py (propagate) written out in plain C so that long
 * trajectories and full-size baselines finish in reasonable time.  Every value is computed
 * with the same double operations in the same order as the numpy version (no contraction,
 * no fast-math), so the two agree bit for bit; a test checks that.
 *
 * For channel k with the per-channel translation s_k = (sx, sy) in cells (Eq. 2):
 *   AF (Eq. 3):   the source point of output cell (j, i) is (i - sx, j - sy); with
 *                 x0 = floor(-sx), y0 = floor(-sy), fx = -sx - x0, fy = -sy - y0 the bilinear
 *                 pull is ((w00 a + w01 b) + w10 c) + w11 d, where a, b, c, d are B at
 *                 (j+y0, i+x0), (j+y0, i+x0+1), (j+y0+1, i+x0), (j+y0+1, i+x0+1), zero off
 *                 the grid, and w00 = (1-fx)(1-fy), w01 = fx(1-fy), w10 = (1-fx)fy, w11 = fx fy.
 *   mask:         S = M * AF.
 *   blur (Eq. 7): T[k][j][i] = sum over dk, dj, di (in that nesting order, each from -r to r)
 *                 of g[dk][dj][di] * S[(k+dk) mod K][j+dj][i+di], zero off the grid.
 *   mask, edge correction (Eq. 8): out = (M * T) * corr.
 * No normalisation: the caller divides by Z (Eq. 9).
 *
 * threads > 1 computes the channels on that many OpenMP threads (when built with OpenMP);
 * every output value is the same sum in the same order whatever the thread count.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static double at(const double* P, int H, int W, int j, int i)
{
    return (j >= 0 && j < H && i >= 0 && i < W) ? P[(size_t)j * W + i] : 0.0;
}

int propagate_direct(const double* B, const double* M, const double* corr, const double* shifts,
                     const double* g, int K, int H, int W, int rk, int r, int threads, double* out)
{
    const size_t hw = (size_t)H * (size_t)W;
    double* S = (double*)malloc(hw * (size_t)K * sizeof(double));
    if (!S) return -1;
    const int nk = 2 * rk + 1, nx = 2 * r + 1;
    if (threads < 1) threads = 1;
#ifdef _OPENMP
#pragma omp parallel for num_threads(threads) schedule(static)
#endif
    for (int k = 0; k < K; ++k) {
        const double sx = shifts[2 * k], sy = shifts[2 * k + 1];
        const double x0d = floor(-sx), y0d = floor(-sy);
        const double fx = -sx - x0d, fy = -sy - y0d;
        const int x0 = (int)x0d, y0 = (int)y0d;
        const double w00 = (1.0 - fx) * (1.0 - fy), w01 = fx * (1.0 - fy);
        const double w10 = (1.0 - fx) * fy, w11 = fx * fy;
        const double* P = B + (size_t)k * hw;
        double* Sk = S + (size_t)k * hw;
        for (int j = 0; j < H; ++j)
            for (int i = 0; i < W; ++i) {
                double v = w00 * at(P, H, W, j + y0, i + x0);
                v = v + w01 * at(P, H, W, j + y0, i + x0 + 1);
                v = v + w10 * at(P, H, W, j + y0 + 1, i + x0);
                v = v + w11 * at(P, H, W, j + y0 + 1, i + x0 + 1);
                Sk[(size_t)j * W + i] = M[(size_t)j * W + i] * v;
            }
    }
#ifdef _OPENMP
#pragma omp parallel for num_threads(threads) schedule(static)
#endif
    for (int k = 0; k < K; ++k) {
        double* T = out + (size_t)k * hw;
        for (size_t q = 0; q < hw; ++q) T[q] = 0.0;
        for (int a = -rk; a <= rk; ++a) {
            const int kk = ((k + a) % K + K) % K;
            const double* Sk = S + (size_t)kk * hw;
            for (int b = -r; b <= r; ++b)
                for (int c = -r; c <= r; ++c) {
                    const double w = g[((size_t)(a + rk) * nx + (b + r)) * nx + (c + r)];
                    const int js = b < 0 ? -b : 0, je = b > 0 ? H - b : H;
                    const int is = c < 0 ? -c : 0, ie = c > 0 ? W - c : W;
                    for (int j = js; j < je; ++j) {
                        double* Tr = T + (size_t)j * W;
                        const double* Sr = Sk + (size_t)(j + b) * W + c;
                        for (int i = is; i < ie; ++i) Tr[i] = Tr[i] + w * Sr[i];
                    }
                }
        }
        (void)nk;
        for (size_t q = 0; q < hw; ++q) T[q] = (M[q] * T[q]) * corr[(size_t)k * hw + q];
    }
    free(S);
    return 0;
}
