/*
 * FP64 CPU oracle for block-wise foveated Gaussian blur.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain restatement of the
 * method that the CUDA path is checked against. Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it. It shares no
 * code, header, table or helper with the CUDA library.
 *
 * What it computes (paper: "CUDA-Optimized real-time rendering of a Foveated
 * Visual System", arXiv 2012.08655):
 *
 *  - Block-wise foveation (Section 2, Algorithm 1): the image is split into
 *    square fragments of side B; every fragment is blurred with ONE Gaussian
 *    whose sigma is set by the distance from the fragment's midpoint to the
 *    fixation point.
 *  - Gaussian filter (Appendix "Methods", Eq. 1 and the paragraph after it):
 *    point samples of exp(-(x^2+y^2)/(2 sigma^2)) at integer offsets with the
 *    centre at (0,0), truncated at 3 sigma, then normalised so the filter sums
 *    to one. Radius r = ceil(3 sigma), i.e. 2r+1 taps per axis, centred.
 *  - Borders clamp to the edge (the paper is silent; clamp-to-edge is the
 *    reading used throughout).
 *  - Sigma law: sigma_b = sigma0 + k * e_b, e_b the Euclidean distance in
 *    pixels from the block centre to the fixation. (The Geisler-Perry law of
 *    Appendix "Choosing the Standard Deviation", Eqs. 2-6, is linear in the
 *    pixel distance, so it is an instance of this form.)
 *
 * The forward map is written as the DIRECT 2D double sum over the
 * (2r+1) x (2r+1) normalised 2D kernel for every output pixel -- no
 * separable pass, no sharing between pixels -- so that it can be checked
 * against the definition by eye:
 *
 *   out(x,y,c) = sum_{j=-r..r} sum_{i=-r..r} K[j][i] * in(clampx(x+i), clampy(y+j), c)
 *   K[j][i]    = w_i * w_j / S^2,  w_i = exp(-i^2/(2 sigma^2)),  S = sum_i w_i
 *
 * The adjoint is the literal transpose of that sum, written as a scatter:
 *
 *   g_in(q,c) += K[j][i] * g_out(p,c)  for every output p and tap (i,j)
 *                                      with clamp(p + (i,j)) = q.
 *
 * Floating-point rules shared with any implementation that wants bit-exact
 * radii: the sigma law is evaluated in IEEE binary64 with no fused
 * multiply-add (this file must be compiled with -ffp-contract=off), sqrt is
 * the correctly rounded IEEE square root, and r = ceil(3 * sigma) is taken on
 * the binary64 product.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Centre of block index b along one axis: B*b + B/2 in continuous pixel
 * coordinates (pixel x covers [x, x+1)); nominal even for a partial edge
 * block (Section 2: "distance from its midpoint to the point of fixation"). */
static double block_centre(int b, int B) { return (double)B * (double)b + 0.5 * (double)B; }

/* Sigma and radius of one block (Section 2; Eq. 5 makes eccentricity linear in
 * pixel distance, and the linear law sigma = sigma0 + k*e follows). */
static void block_sigma(int bx, int by, int B, double fx, double fy, double sigma0, double k,
                        double* sigma, int* radius) {
  double dx = block_centre(bx, B) - fx;
  double dy = block_centre(by, B) - fy;
  double dx2 = dx * dx;
  double dy2 = dy * dy;
  double e = sqrt(dx2 + dy2);
  double ke = k * e;
  double s = sigma0 + ke;
  double three_s = 3.0 * s;
  *sigma = s;
  *radius = (int)ceil(three_s);
}

int oracle_num_blocks(int W, int H, int B) {
  if (W <= 0 || H <= 0 || B <= 0) return 0;
  return ((W + B - 1) / B) * ((H + B - 1) / B);
}

/* Per-block sigma and radius, row-major over the block grid. */
void oracle_sigma_table(int W, int H, int B, double fx, double fy, double sigma0, double k,
                        double* sigma_out, int* radius_out) {
  int nbx = (W + B - 1) / B, nby = (H + B - 1) / B;
  for (int by = 0; by < nby; ++by)
    for (int bx = 0; bx < nbx; ++bx)
      block_sigma(bx, by, B, fx, fy, sigma0, k, &sigma_out[by * nbx + bx], &radius_out[by * nbx + bx]);
}

/* Normalised 1D taps w[0..2r] for offsets -r..r (Eq. 1 sampled at integer
 * offsets, centre at 0, normalised to unit sum). r = 0 gives the single
 * weight 1 (the identity). */
void oracle_taps(double sigma, int r, double* w) {
  if (r <= 0) { w[0] = 1.0; return; }
  double S = 0.0;
  for (int i = -r; i <= r; ++i) {
    double v = (i == 0) ? 1.0 : exp(-((double)i * (double)i) / (2.0 * sigma * sigma));
    w[i + r] = v;
    S += v;
  }
  for (int i = 0; i <= 2 * r; ++i) w[i] /= S;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Forward map over a list of blocks (all blocks when block_list is NULL).
 * Element (x, y, c) lives at base[y*sy + x*sx + c*sc] for both in and out.
 * Only the pixels of the listed blocks are written. */
void oracle_forward(const double* in, double* out, int W, int H, int C, long sy, long sx, long sc,
                    int B, double fx, double fy, double sigma0, double k,
                    const int* block_list, int nlist, int nthreads) {
  int nbx = (W + B - 1) / B, nby = (H + B - 1) / B;
  int nb = block_list ? nlist : nbx * nby;
  int nt = 1;
#ifdef _OPENMP
  nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
#endif
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
    for (int t = 0; t < nb; ++t) {
      int b = block_list ? block_list[t] : t;
      int bx = b % nbx, by = b / nbx;
      double sigma;
      int r;
      block_sigma(bx, by, B, fx, fy, sigma0, k, &sigma, &r);
      size_t n = (size_t)(2 * r + 1);
      double* w = (double*)malloc(n * sizeof(double));
      double* K = (double*)malloc(n * n * sizeof(double));
      oracle_taps(sigma, r, w);
      for (size_t j = 0; j < n; ++j)
        for (size_t i = 0; i < n; ++i) K[j * n + i] = w[i] * w[j];
      int x0 = bx * B, y0 = by * B;
      int x1 = x0 + B < W ? x0 + B : W, y1 = y0 + B < H ? y0 + B : H;
      for (int c = 0; c < C; ++c)
        for (int y = y0; y < y1; ++y)
          for (int x = x0; x < x1; ++x) {
            double acc = 0.0;
            for (int j = -r; j <= r; ++j) {
              int yy = clampi(y + j, 0, H - 1);
              for (int i = -r; i <= r; ++i) {
                int xx = clampi(x + i, 0, W - 1);
                acc += K[(size_t)(j + r) * n + (size_t)(i + r)] * in[yy * sy + xx * sx + c * sc];
              }
            }
            out[y * sy + x * sx + c * sc] = acc;
          }
      free(K);
      free(w);
    }
}

/* Adjoint (transpose) of the forward map: g_in = A^T g_out, written as the
 * scatter of every output pixel's weighted value to the clamped input
 * positions it was computed from. g_in is overwritten. */
void oracle_adjoint(const double* g_out, double* g_in, int W, int H, int C, long sy, long sx, long sc,
                    int B, double fx, double fy, double sigma0, double k, int nthreads) {
  int nbx = (W + B - 1) / B, nby = (H + B - 1) / B;
  size_t total = (size_t)W * H * C;
  int nt = 1;
#ifdef _OPENMP
  nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
#endif
  /* One private accumulation image per thread; summed at the end. Indexing
   * of the private images is dense CHW, independent of (sy, sx, sc). */
  double* priv = (double*)calloc((size_t)nt * total, sizeof(double));
#pragma omp parallel num_threads(nt)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double* acc = priv + (size_t)tid * total;
#pragma omp for schedule(dynamic, 1)
    for (int b = 0; b < nbx * nby; ++b) {
      int bx = b % nbx, by = b / nbx;
      double sigma;
      int r;
      block_sigma(bx, by, B, fx, fy, sigma0, k, &sigma, &r);
      int n = 2 * r + 1;
      double* w = (double*)malloc((size_t)n * sizeof(double));
      oracle_taps(sigma, r, w);
      int x0 = bx * B, y0 = by * B;
      int x1 = x0 + B < W ? x0 + B : W, y1 = y0 + B < H ? y0 + B : H;
      for (int c = 0; c < C; ++c)
        for (int y = y0; y < y1; ++y)
          for (int x = x0; x < x1; ++x) {
            double g = g_out[y * sy + x * sx + c * sc];
            for (int j = -r; j <= r; ++j) {
              int yy = clampi(y + j, 0, H - 1);
              for (int i = -r; i <= r; ++i) {
                int xx = clampi(x + i, 0, W - 1);
                acc[((size_t)c * H + yy) * W + xx] += (w[i + r] * w[j + r]) * g;
              }
            }
          }
      free(w);
    }
  }
  for (int c = 0; c < C; ++c)
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) {
        double s = 0.0;
        for (int t = 0; t < nt; ++t) s += priv[(size_t)t * total + ((size_t)c * H + y) * W + x];
        g_in[y * sy + x * sx + c * sc] = s;
      }
  free(priv);
}

/* uint8 output coding: nearest integer with halves rounded up, clamped to
 * [0, 255] (the paper keeps 8-bit images end to end; "rounded to nearest"). */
void oracle_quantize_u8(const double* v, uint8_t* q, long n) {
  for (long i = 0; i < n; ++i) {
    double f = floor(v[i] + 0.5);
    if (f < 0.0) f = 0.0;
    if (f > 255.0) f = 255.0;
    q[i] = (uint8_t)f;
  }
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
