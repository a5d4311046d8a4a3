/*
 * FP64 CPU oracle for the dense pyramidal Lucas-Kanade optical flow of
 * Gautier & Aider, "Real-time planar flow velocity measurements using an optical
 * flow algorithm implemented on GPU" (arXiv:1306.2461), Sect. 2.4.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, loads or calls
 * this file; only the tests, the package's smoke check and the benchmark's CPU
 * baseline do. It shares no code, header or constant table with the CUDA path.
 *
 * Plain, slow and direct on purpose: every window sum is the full (2r+1)^2 double
 * loop, every pyramid tap the full 5x5 double loop, all arithmetic in double.
 * Compile without -ffast-math and with -ffp-contract=off so that x86 and Arm hosts
 * give bit-identical results.
 *
 * What the paper fixes (Sect. 2.4): a pyramid whose images shrink by 4 in area per
 * level; zero displacement at the top level; an iterative Gauss-Newton minimisation
 * of a sum of squared differences over a window of radius r, one vector per pixel;
 * each level's result is the initial estimate of the next finer level. What it
 * leaves open is read as follows (the same readings the CUDA path implements):
 *   - pyramid: separable 5-tap binomial [1 4 6 4 1]/16 low-pass with clamp-to-edge
 *     taps, keep the even samples; a level of n pixels has ceil(n/2) at the next;
 *   - warp: bilinear interpolation of I2 at x + u(x), sample position clamped to
 *     [0, W-1] x [0, H-1], right/bottom neighbour index clamped;
 *   - gradient: the gradient of I2 at the displaced position, taken as the central
 *     difference of two bilinear samples one pixel either side of x + u(x) (sample
 *     positions clamped, always divided by 2): the Jacobian of I2(x + u) in u;
 *   - Gauss-Newton step of the window SSD with the image linearised at every pixel's
 *     own current estimate u_k(x): with e = I1 - I2w and e~ = e + gx u_k + gy v_k,
 *     solve [Sa Sb; Sb Sc] u_{k+1} = [Sd; Se] where S* are the (2r+1)^2 box sums of
 *     gx^2, gx gy, gy^2, gx e~, gy e~ (terms outside the image contribute 0), for all
 *     pixels at once (Jacobi). The estimate is kept when tr <= 0 or
 *     det <= 1e-6 tr^2. (Written as an increment u += H^-1 sum(g e) the same step is
 *     unstable under Jacobi updates: the box window's transfer function dips to
 *     -0.22, so some flow-error modes grow by ~22% per iteration.);
 *   - propagation: u_l(x, y) = 2 * bilinear(u_{l+1}; x/2, y/2) (clamped).
 *
 * Parity of this oracle is pinned in the CPU tests against closed forms and library
 * routines (scipy/numpy), not against itself.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OFO_SINGULAR_EPS 1e-6

static int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }
static double clampd(double a, double lo, double hi) { return a < lo ? lo : (a > hi ? hi : a); }

/* Pyramid reduction (Sect. 2.4: images reduced by a factor of 4 per level, i.e. by 2
 * per axis, Fig. 3). out has ceil(H/2) x ceil(W/2) pixels. Direct 25-tap sum. */
void ofo_pyr_down(const double *in, int H, int W, double *out)
{
    static const double w[5] = {1.0, 4.0, 6.0, 4.0, 1.0};
    const int Ho = (H + 1) / 2, Wo = (W + 1) / 2;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < Ho; ++i) {
        for (int j = 0; j < Wo; ++j) {
            double s = 0.0;
            for (int a = 0; a < 5; ++a) {
                const int y = clampi(2 * i + a - 2, 0, H - 1);
                for (int b = 0; b < 5; ++b) {
                    const int x = clampi(2 * j + b - 2, 0, W - 1);
                    s += w[a] * w[b] * in[(size_t)y * W + x];
                }
            }
            out[(size_t)i * Wo + j] = s / 256.0;
        }
    }
}

/* Bilinear interpolation with the sample position clamped to the image. */
double ofo_bilinear(const double *img, int H, int W, double x, double y)
{
    x = clampd(x, 0.0, (double)(W - 1));
    y = clampd(y, 0.0, (double)(H - 1));
    const int x0 = (int)floor(x), y0 = (int)floor(y);
    const int x1 = x0 + 1 < W ? x0 + 1 : W - 1;
    const int y1 = y0 + 1 < H ? y0 + 1 : H - 1;
    const double ax = x - x0, ay = y - y0;
    const double top = (1.0 - ax) * img[(size_t)y0 * W + x0] + ax * img[(size_t)y0 * W + x1];
    const double bot = (1.0 - ax) * img[(size_t)y1 * W + x0] + ax * img[(size_t)y1 * W + x1];
    return (1.0 - ay) * top + ay * bot;
}

/* Coarse-to-fine propagation (Sect. 2.4: a level's displacement is the initial
 * estimate at the next finer level). Displacements double with the resolution. */
void ofo_upsample_flow(const double *fc, int Hc, int Wc, double *f, int H, int W)
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            f[(size_t)y * W + x] = 2.0 * ofo_bilinear(fc, Hc, Wc, 0.5 * x, 0.5 * y);
}

/* I2 warped by the current displacement, I2w(x, y) = I2(x + u, y + v), and the
 * gradient of I2 at that displaced position: central difference of bilinear samples
 * at (x + u +- 1, y + v) and (x + u, y + v +- 1), each sample position clamped. */
void ofo_warp_grad(const double *I2, const double *u, const double *v, int H, int W,
                   double *Iw, double *gx, double *gy)
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const size_t k = (size_t)y * W + x;
            const double px = x + u[k], py = y + v[k];
            Iw[k] = ofo_bilinear(I2, H, W, px, py);
            gx[k] = (ofo_bilinear(I2, H, W, px + 1.0, py) - ofo_bilinear(I2, H, W, px - 1.0, py)) / 2.0;
            gy[k] = (ofo_bilinear(I2, H, W, px, py + 1.0) - ofo_bilinear(I2, H, W, px, py - 1.0)) / 2.0;
        }
}

/* Window sum over the (2r+1)^2 box of radius r (Sect. 2.4), zero outside the image.
 * Brute force: the full double loop for every pixel. */
void ofo_window_sum(const double *c, int H, int W, int r, double *out)
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double s = 0.0;
            for (int dy = -r; dy <= r; ++dy) {
                const int yy = y + dy;
                if (yy < 0 || yy >= H) continue;
                for (int dx = -r; dx <= r; ++dx) {
                    const int xx = x + dx;
                    if (xx < 0 || xx >= W) continue;
                    s += c[(size_t)yy * W + xx];
                }
            }
            out[(size_t)y * W + x] = s;
        }
}

/* The 2x2 normal equations of one window: [a b; b c] x = [d0; e0] by Cramer's rule.
 * Returns 1 and the solution when the system passes the singular guard
 * (tr > 0 and det > 1e-6 tr^2), else 0. *ratio = det/tr^2 (-1 when tr <= 0). */
int ofo_solve2(double a, double b, double c, double d0, double e0, double *xu, double *xv,
               double *ratio)
{
    const double tr = a + c;
    const double det = a * c - b * b;
    if (!(tr > 0.0)) {
        *ratio = -1.0;
        return 0;
    }
    *ratio = det / (tr * tr);
    if (det <= OFO_SINGULAR_EPS * tr * tr) return 0;
    *xu = (c * d0 - b * e0) / det;
    *xv = (a * e0 - b * d0) / det;
    return 1;
}

/* Vector form of ofo_solve2; where the guard fails, xu/xv receive the fallback
 * values fu/fv (the current estimate in the iteration). ok[k] = 1 when solved. */
void ofo_solve(const double *Sa, const double *Sb, const double *Sc, const double *Sd,
               const double *Se, const double *fu, const double *fv, int n,
               double *xu, double *xv, double *ratio, int *ok)
{
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n; ++k) {
        double q, a = fu[k], b = fv[k];
        const int solved = ofo_solve2(Sa[k], Sb[k], Sc[k], Sd[k], Se[k], &a, &b, &q);
        xu[k] = a;
        xv[k] = b;
        if (ratio) ratio[k] = q;
        if (ok) ok[k] = solved;
    }
}

/* One Gauss-Newton iteration at one level (Sect. 2.4), all pixels from the previous
 * iterate (u, v): warp and gradient, residual, the five window sums, solve.
 * ratio (optional) receives det/tr^2 per pixel. */
int ofo_lk_iteration(const double *P1, const double *P2, int H, int W, int r,
                     const double *u, const double *v, double *u_new, double *v_new,
                     double *ratio)
{
    const size_t N = (size_t)H * W;
    double *buf = (double *)malloc(sizeof(double) * N * 13);
    if (!buf) return -1;
    double *Iw = buf, *gx = buf + N, *gy = buf + 2 * N;
    double *p[5], *S[5];
    for (int k = 0; k < 5; ++k) { p[k] = buf + (3 + k) * N; S[k] = buf + (8 + k) * N; }

    ofo_warp_grad(P2, u, v, H, W, Iw, gx, gy);
    for (size_t k = 0; k < N; ++k) {
        const double e = P1[k] - Iw[k] + gx[k] * u[k] + gy[k] * v[k];
        p[0][k] = gx[k] * gx[k];
        p[1][k] = gx[k] * gy[k];
        p[2][k] = gy[k] * gy[k];
        p[3][k] = gx[k] * e;
        p[4][k] = gy[k] * e;
    }
    for (int k = 0; k < 5; ++k) ofo_window_sum(p[k], H, W, r, S[k]);
    ofo_solve(S[0], S[1], S[2], S[3], S[4], u, v, (int)N, u_new, v_new, ratio, NULL);
    free(buf);
    return 0;
}

/* Variant with the window matrix fixed per level (the FOLKI lineage): the image is
 * linearised with the gradient of the FIRST image at integer pixels (central
 * difference, indices clamped, /2) instead of the gradient of I2 at the displaced
 * position, so that [Sa Sb; Sb Sc] depends on I1 only. Per iteration, with
 * e~ = I1 - I2w + g1x u_k + g1y v_k, solve [Sa Sb; Sb Sc] u_{k+1} = [sum g1x e~; sum g1y e~]
 * (same guard as ofo_lk_iteration). */
int ofo_lk_iteration_i1grad(const double *P1, const double *P2, int H, int W, int r,
                            const double *u, const double *v, double *u_new, double *v_new,
                            double *ratio)
{
    const size_t N = (size_t)H * W;
    double *buf = (double *)malloc(sizeof(double) * N * 13);
    if (!buf) return -1;
    double *Iw = buf, *g1x = buf + N, *g1y = buf + 2 * N;
    double *p[5], *S[5];
    for (int k = 0; k < 5; ++k) { p[k] = buf + (3 + k) * N; S[k] = buf + (8 + k) * N; }
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const size_t k = (size_t)y * W + x;
            const int xm = clampi(x - 1, 0, W - 1), xp = clampi(x + 1, 0, W - 1);
            const int ym = clampi(y - 1, 0, H - 1), yp = clampi(y + 1, 0, H - 1);
            g1x[k] = (P1[(size_t)y * W + xp] - P1[(size_t)y * W + xm]) / 2.0;
            g1y[k] = (P1[(size_t)yp * W + x] - P1[(size_t)ym * W + x]) / 2.0;
            Iw[k] = ofo_bilinear(P2, H, W, x + u[k], y + v[k]);
        }
    for (size_t k = 0; k < N; ++k) {
        const double et = P1[k] - Iw[k] + g1x[k] * u[k] + g1y[k] * v[k];
        p[0][k] = g1x[k] * g1x[k];
        p[1][k] = g1x[k] * g1y[k];
        p[2][k] = g1y[k] * g1y[k];
        p[3][k] = g1x[k] * et;
        p[4][k] = g1y[k] * et;
    }
    for (int k = 0; k < 5; ++k) ofo_window_sum(p[k], H, W, r, S[k]);
    ofo_solve(S[0], S[1], S[2], S[3], S[4], u, v, (int)N, u_new, v_new, ratio, NULL);
    free(buf);
    return 0;
}

/* Level sizes of the pyramid: level 0 is H x W, level l+1 is ceil of half of level l. */
void ofo_level_size(int H, int W, int level, int *Hl, int *Wl)
{
    for (int l = 0; l < level; ++l) { H = (H + 1) / 2; W = (W + 1) / 2; }
    *Hl = H; *Wl = W;
}

/* Full coarse-to-fine flow (Sect. 2.4, Fig. 3): build both pyramids, start at zero
 * displacement on the coarsest level, run `iters` iterations per level, propagate.
 * u, v: H x W outputs (level 0). ratio_min (optional, H x W): the smallest det/tr^2
 * each pixel saw over the level-0 iterations, for locating near-singular pixels. */
int ofo_flow_variant(const double *I1, const double *I2, int H, int W, int levels, int r, int iters,
                     double *u, double *v, double *ratio_min, int i1grad)
{
    if (H <= 0 || W <= 0 || levels < 1 || r < 0 || iters < 0) return -1;
    double **P1 = (double **)calloc((size_t)levels, sizeof(double *));
    double **P2 = (double **)calloc((size_t)levels, sizeof(double *));
    int *Hs = (int *)calloc((size_t)levels, sizeof(int));
    int *Ws = (int *)calloc((size_t)levels, sizeof(int));
    const size_t N0 = (size_t)H * W;
    double *fu = (double *)malloc(sizeof(double) * N0), *fv = (double *)malloc(sizeof(double) * N0);
    double *gu = (double *)malloc(sizeof(double) * N0), *gv = (double *)malloc(sizeof(double) * N0);
    double *rt = (double *)malloc(sizeof(double) * N0);
    int rc = 0;
    if (!P1 || !P2 || !Hs || !Ws || !fu || !fv || !gu || !gv || !rt) { rc = -1; goto done; }

    for (int l = 0; l < levels; ++l) {
        ofo_level_size(H, W, l, &Hs[l], &Ws[l]);
        const size_t n = (size_t)Hs[l] * Ws[l];
        P1[l] = (double *)malloc(sizeof(double) * n);
        P2[l] = (double *)malloc(sizeof(double) * n);
        if (!P1[l] || !P2[l]) { rc = -1; goto done; }
    }
    memcpy(P1[0], I1, sizeof(double) * N0);
    memcpy(P2[0], I2, sizeof(double) * N0);
    for (int l = 0; l + 1 < levels; ++l) {
        ofo_pyr_down(P1[l], Hs[l], Ws[l], P1[l + 1]);
        ofo_pyr_down(P2[l], Hs[l], Ws[l], P2[l + 1]);
    }
    if (ratio_min)
        for (size_t k = 0; k < N0; ++k) ratio_min[k] = INFINITY;

    for (int l = levels - 1; l >= 0; --l) {
        const int h = Hs[l], w = Ws[l];
        const size_t n = (size_t)h * w;
        if (l == levels - 1) {
            memset(fu, 0, sizeof(double) * n);
            memset(fv, 0, sizeof(double) * n);
        } else {
            ofo_upsample_flow(fu, Hs[l + 1], Ws[l + 1], gu, h, w);
            ofo_upsample_flow(fv, Hs[l + 1], Ws[l + 1], gv, h, w);
            memcpy(fu, gu, sizeof(double) * n);
            memcpy(fv, gv, sizeof(double) * n);
        }
        for (int it = 0; it < iters; ++it) {
            const int it_rc = i1grad ? ofo_lk_iteration_i1grad(P1[l], P2[l], h, w, r, fu, fv, gu, gv, rt)
                                     : ofo_lk_iteration(P1[l], P2[l], h, w, r, fu, fv, gu, gv, rt);
            if (it_rc) { rc = -1; goto done; }
            memcpy(fu, gu, sizeof(double) * n);
            memcpy(fv, gv, sizeof(double) * n);
            if (l == 0 && ratio_min)
                for (size_t k = 0; k < n; ++k)
                    if (rt[k] < ratio_min[k]) ratio_min[k] = rt[k];
        }
    }
    memcpy(u, fu, sizeof(double) * N0);
    memcpy(v, fv, sizeof(double) * N0);

done:
    if (P1) for (int l = 0; l < levels; ++l) free(P1[l]);
    if (P2) for (int l = 0; l < levels; ++l) free(P2[l]);
    free(P1); free(P2); free(Hs); free(Ws);
    free(fu); free(fv); free(gu); free(gv); free(rt);
    return rc;
}

int ofo_flow(const double *I1, const double *I2, int H, int W, int levels, int r, int iters,
             double *u, double *v, double *ratio_min)
{
    return ofo_flow_variant(I1, I2, H, W, levels, r, iters, u, v, ratio_min, 0);
}

/* Number of OpenMP threads the oracle will use (1 when built without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
int ofo_threads(void) { return omp_get_max_threads(); }
void ofo_set_threads(int n) { if (n > 0) omp_set_num_threads(n); }
#else
int ofo_threads(void) { return 1; }
void ofo_set_threads(int n) { (void)n; }
#endif

/* Recirculation-bubble surface (Sect. 3.2, Eq. 3), read as the number of vectors whose
 * streamwise component u is at most the threshold T_v, over the number of vectors.
 * Returns the count; the fraction is count / (H W). */
long long ofo_sbubble_count(const float *u, int H, int W, float Tv)
{
    long long c = 0;
    for (size_t k = 0; k < (size_t)H * W; ++k)
        if (u[k] <= Tv) ++c;
    return c;
}

/* The threshold of Eq. 3: T_v = (min + max) / 2 of the mean streamwise field. */
double ofo_sbubble_threshold(const float *mean_u, int H, int W)
{
    float lo = mean_u[0], hi = mean_u[0];
    for (size_t k = 1; k < (size_t)H * W; ++k) {
        if (mean_u[k] < lo) lo = mean_u[k];
        if (mean_u[k] > hi) hi = mean_u[k];
    }
    return 0.5 * ((double)lo + (double)hi);
}

/* Local normalisation of an image before the flow (Sect. 2.4, Eq. 2): with I_m the
 * local mean and s the local standard deviation over the (2 rho + 1)^2 window clipped
 * to the image (n pixels), out = (I - I_m) / sqrt(s^2 + eps). The printed radicand
 * (mean^2 - mean of squares) is negative; the variance is read instead. Written with
 * the window sums S1 = sum I, S2 = sum I^2: out = (n I - S1) / sqrt(n S2 - S1^2 + n^2 eps).
 * Direct double loops over every window. */
void ofo_znssd(const double *I, int H, int W, int rho, double eps, double *out)
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double n = 0.0, s1 = 0.0, s2 = 0.0;
            for (int yy = y - rho; yy <= y + rho; ++yy) {
                if (yy < 0 || yy >= H) continue;
                for (int xx = x - rho; xx <= x + rho; ++xx) {
                    if (xx < 0 || xx >= W) continue;
                    const double v = I[(size_t)yy * W + xx];
                    n += 1.0;
                    s1 += v;
                    s2 += v * v;
                }
            }
            const double mean = s1 / n;
            const double var = s2 / n - mean * mean;
            out[(size_t)y * W + x] = (I[(size_t)y * W + x] - mean) / sqrt(var + eps);
        }
}
