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
 *    pixel distance, so it is an instance of this form; oracle_gp_sigma
 *    evaluates its chain of equations literally and oracle_gp_linear gives
 *    the two coefficients.) Alternatively a per-block sigma map.
 *  - Block grid: block (bx, by) covers pixels x in [B bx - ox, B bx - ox + B)
 *    clipped to the frame (likewise in y), with an origin offset 0 <= ox < B
 *    (0: the grid starts at the frame corner; Algorithm 1 shifts it so that
 *    a fragment is centred on the fixation, see oracle_centred_origin).
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
 * Two further functions serve the per-pixel workload of Section 3.1: the
 * per-pixel ("perfect") foveation the paper uses as its quality reference
 * (every pixel blurred with the sigma of its own centre), and the SSIM map
 * (Wang et al. 2004, standard window and constants) it is scored with.
 * And the Gaussian-pyramid (mipmap) foveation the paper compares its speed
 * and smoothness against (Section 3.2 and its appendix on previous work).
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

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Centre of block index b along one axis: B*b + B/2 in continuous pixel
 * coordinates (pixel x covers [x, x+1)); nominal even for a partial edge
 * block (Section 2: "distance from its midpoint to the point of fixation"). */
static double block_centre(int b, int B) { return (double)B * (double)b + 0.5 * (double)B; }

/* Sigma and radius of one block (Section 2; Eq. 5 makes eccentricity linear in
 * pixel distance, and the linear law sigma = sigma0 + k*e follows). The
 * block centre is B*b + B/2 - o along each axis for grid origin offset o. */
static void block_sigma_o(int bx, int by, int B, int ox, int oy, double fx, double fy, double sigma0, double k,
                          double* sigma, int* radius) {
  double dx = (block_centre(bx, B) - (double)ox) - fx;
  double dy = (block_centre(by, B) - (double)oy) - fy;
  double dx2 = dx * dx;
  double dy2 = dy * dy;
  double e = sqrt(dx2 + dy2);
  double ke = k * e;
  double s = sigma0 + ke;
  double three_s = 3.0 * s;
  *sigma = s;
  *radius = (int)ceil(three_s);
}

/* Blocks along an axis of n pixels with origin offset o: ceil((n + o) / B). */
static int grid_count(int n, int B, int o) { return (n + o + B - 1) / B; }

/* Pixel range [*a0, *a1) of block index b along an axis of n pixels. */
static void block_span(int b, int B, int o, int n, int* a0, int* a1) {
  int s = B * b - o;
  *a0 = s < 0 ? 0 : s;
  *a1 = s + B < n ? s + B : n;
}

/* Sigma of one block: from the law, or map[by * nbx + bx] when map != NULL
 * (r = ceil(3 sigma) either way). */
static void block_sigma_any(int bx, int by, int nbx, int B, int ox, int oy, double fx, double fy,
                            double sigma0, double k, const double* map, double* sigma, int* radius) {
  if (map) {
    double s = map[by * nbx + bx];
    double three_s = 3.0 * s;
    *sigma = s;
    *radius = (int)ceil(three_s);
  } else {
    block_sigma_o(bx, by, B, ox, oy, fx, fy, sigma0, k, sigma, radius);
  }
}

/* Geisler-Perry chain (Appendix "Choosing the Standard Deviation"), taken
 * step by step for a pixel at distance d from the fixation in a W x H frame
 * whose corner is at eccentricity e_corner degrees:
 *   Eq. 5  e = d / d_corner * e_corner,  d_corner = half the frame diagonal
 *   Eq. 3  f_c_deg = e2 / (alpha (e + e2)) ln(1 / CT0)   (Eq. 2 set to 1)
 *          f_max = f_c_deg at e = 0 (highest acuity, at the fovea)
 *   Eq. 4  f_c_pix = 0.5 f_c_deg / f_max
 *   Eq. 6  sigma = 1 / (2 pi f_c_pix)
 * with alpha = 0.106, e2 = 2.3, CT0 = 1/64. */
double oracle_gp_sigma(double d, int W, int H, double e_corner) {
  const double alpha = 0.106, e2 = 2.3, ct0 = 1.0 / 64.0;
  double d_corner = 0.5 * sqrt((double)W * (double)W + (double)H * (double)H);
  double e = d / d_corner * e_corner;
  double f_c_deg = e2 / (alpha * (e + e2)) * log(1.0 / ct0);
  double f_max = e2 / (alpha * (0.0 + e2)) * log(1.0 / ct0);
  double f_c_pix = 0.5 * f_c_deg / f_max;
  return 1.0 / (2.0 * M_PI * f_c_pix);
}

/* The same law as sigma = sigma0 + k d: the chain above reduces to
 * sigma = (1 + e / e2) / pi, so sigma0 = 1 / pi and
 * k = e_corner / ((pi e2) d_corner). */
void oracle_gp_linear(int W, int H, double e_corner, double* sigma0, double* k) {
  const double e2 = 2.3;
  double d_corner = 0.5 * sqrt((double)W * (double)W + (double)H * (double)H);
  *sigma0 = 1.0 / M_PI;
  *k = e_corner / ((M_PI * e2) * d_corner);
}

/* Grid origin offset that centres a fragment on the fixation (Algorithm 1,
 * Section 3.1), to the nearest pixel: the fragment starting at
 * floor(f + 1/2) - floor(B/2) is a whole block, so
 * o = (floor(B/2) - floor(f + 1/2)) mod B. */
int oracle_centred_origin(double f, int B) {
  long c = (long)floor(f + 0.5);
  long o = ((long)(B / 2) - c) % B;
  if (o < 0) o += B;
  return (int)o;
}

int oracle_num_blocks(int W, int H, int B) {
  if (W <= 0 || H <= 0 || B <= 0) return 0;
  return ((W + B - 1) / B) * ((H + B - 1) / B);
}

/* Per-block sigma and radius, row-major over the block grid. */
void oracle_sigma_table_ex(int W, int H, int B, int ox, int oy, double fx, double fy, double sigma0, double k,
                           const double* map, double* sigma_out, int* radius_out) {
  int nbx = grid_count(W, B, ox), nby = grid_count(H, B, oy);
  for (int by = 0; by < nby; ++by)
    for (int bx = 0; bx < nbx; ++bx)
      block_sigma_any(bx, by, nbx, B, ox, oy, fx, fy, sigma0, k, map, &sigma_out[by * nbx + bx],
                      &radius_out[by * nbx + bx]);
}

void oracle_sigma_table(int W, int H, int B, double fx, double fy, double sigma0, double k,
                        double* sigma_out, int* radius_out) {
  oracle_sigma_table_ex(W, H, B, 0, 0, fx, fy, sigma0, k, NULL, sigma_out, radius_out);
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
void oracle_forward_ex(const double* in, double* out, int W, int H, int C, long sy, long sx, long sc,
                       int B, int ox, int oy, double fx, double fy, double sigma0, double k, const double* map,
                       const int* block_list, int nlist, int nthreads) {
  int nbx = grid_count(W, B, ox), nby = grid_count(H, B, oy);
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
      block_sigma_any(bx, by, nbx, B, ox, oy, fx, fy, sigma0, k, map, &sigma, &r);
      size_t n = (size_t)(2 * r + 1);
      double* w = (double*)malloc(n * sizeof(double));
      double* K = (double*)malloc(n * n * sizeof(double));
      oracle_taps(sigma, r, w);
      for (size_t j = 0; j < n; ++j)
        for (size_t i = 0; i < n; ++i) K[j * n + i] = w[i] * w[j];
      int x0, x1, y0, y1;
      block_span(bx, B, ox, W, &x0, &x1);
      block_span(by, B, oy, H, &y0, &y1);
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

void oracle_forward(const double* in, double* out, int W, int H, int C, long sy, long sx, long sc,
                    int B, double fx, double fy, double sigma0, double k,
                    const int* block_list, int nlist, int nthreads) {
  oracle_forward_ex(in, out, W, H, C, sy, sx, sc, B, 0, 0, fx, fy, sigma0, k, NULL, block_list, nlist, nthreads);
}

/* Adjoint (transpose) of the forward map: g_in = A^T g_out, written as the
 * scatter of every output pixel's weighted value to the clamped input
 * positions it was computed from. g_in is overwritten. */
void oracle_adjoint_ex(const double* g_out, double* g_in, int W, int H, int C, long sy, long sx, long sc,
                       int B, int ox, int oy, double fx, double fy, double sigma0, double k, const double* map,
                       int nthreads) {
  int nbx = grid_count(W, B, ox), nby = grid_count(H, B, oy);
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
      block_sigma_any(bx, by, nbx, B, ox, oy, fx, fy, sigma0, k, map, &sigma, &r);
      int n = 2 * r + 1;
      double* w = (double*)malloc((size_t)n * sizeof(double));
      oracle_taps(sigma, r, w);
      int x0, x1, y0, y1;
      block_span(bx, B, ox, W, &x0, &x1);
      block_span(by, B, oy, H, &y0, &y1);
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

void oracle_adjoint(const double* g_out, double* g_in, int W, int H, int C, long sy, long sx, long sc,
                    int B, double fx, double fy, double sigma0, double k, int nthreads) {
  oracle_adjoint_ex(g_out, g_in, W, H, C, sy, sx, sc, B, 0, 0, fx, fy, sigma0, k, NULL, nthreads);
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

/* ------------------------------------------------------------------------
 * Per-pixel ("perfect") foveation: the reference the paper scores its
 * block-wise output against (Section 3.1, Fig. 3). Every pixel gets its own
 * sigma from the distance between ITS centre (x + 1/2, y + 1/2) and the
 * fixation, with the same law, the same truncated, normalised taps and the
 * same clamp-to-edge border as the block-wise map:
 *
 *   sigma_p = sigma0 + k * |(x + 1/2, y + 1/2) - f|,  r_p = ceil(3 sigma_p)
 *   out(x,y,c) = sum_{|i|,|j| <= r_p} w_i w_j / S^2 * in(clamp(x+i), clamp(y+j), c)
 *
 * (binary64, no FMA, as for the block sigma). Written as the direct 2D sum.
 * ------------------------------------------------------------------------ */

/* Sigma and radius of pixel (x, y). */
void oracle_pixel_sigma(int x, int y, double fx, double fy, double sigma0, double k, double* sigma, int* radius) {
  double dx = ((double)x + 0.5) - fx;
  double dy = ((double)y + 0.5) - fy;
  double dx2 = dx * dx;
  double dy2 = dy * dy;
  double e = sqrt(dx2 + dy2);
  double ke = k * e;
  double s = sigma0 + ke;
  double three_s = 3.0 * s;
  *sigma = s;
  *radius = (int)ceil(three_s);
}

/* Per-pixel foveation of the listed pixels (row-major indices y * W + x; all
 * pixels when pixel_list is NULL), every channel. Layout as oracle_forward_ex.
 * Pixels not listed are left untouched. */
void oracle_forward_pixel(const double* in, double* out, int W, int H, int C, long sy, long sx, long sc,
                          double fx, double fy, double sigma0, double k, const long* pixel_list, long nlist,
                          int nthreads) {
  long np = pixel_list ? nlist : (long)W * (long)H;
  int nt = 1;
#ifdef _OPENMP
  nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
#endif
#pragma omp parallel for num_threads(nt) schedule(dynamic, 64)
  for (long t = 0; t < np; ++t) {
    long p = pixel_list ? pixel_list[t] : t;
    int x = (int)(p % W), y = (int)(p / W);
    double sigma;
    int r;
    oracle_pixel_sigma(x, y, fx, fy, sigma0, k, &sigma, &r);
    double* w = (double*)malloc((size_t)(2 * r + 1) * sizeof(double));
    oracle_taps(sigma, r, w);
    for (int c = 0; c < C; ++c) {
      double acc = 0.0;
      for (int j = -r; j <= r; ++j) {
        int yy = clampi(y + j, 0, H - 1);
        for (int i = -r; i <= r; ++i) {
          int xx = clampi(x + i, 0, W - 1);
          acc += (w[i + r] * w[j + r]) * in[yy * sy + xx * sx + c * sc];
        }
      }
      out[y * sy + x * sx + c * sc] = acc;
    }
    free(w);
  }
}

/* ------------------------------------------------------------------------
 * SSIM map (the image-quality measure of Section 3.1; Wang, Bovik, Sheikh and
 * Simoncelli 2004, with their standard settings): for every pixel and
 * channel, local statistics under an 11 x 11 Gaussian window of standard
 * deviation 1.5 normalised to unit sum (clamp-to-edge at the border),
 *
 *   mu_a = sum w a,  var_a = sum w (a - mu_a)^2,  cov = sum w (a - mu_a)(b - mu_b)
 *   SSIM = (2 mu_a mu_b + C1)(2 cov + C2) / ((mu_a^2 + mu_b^2 + C1)(var_a + var_b + C2))
 *
 * with C1 = (0.01 L)^2, C2 = (0.03 L)^2 for dynamic range L. The map value of
 * a pixel is the mean over its channels. Written out pixel by pixel in
 * binary64, two passes over the window (means first, then the centred
 * moments).
 * ------------------------------------------------------------------------ */
void oracle_ssim_map(const double* a, const double* b, int W, int H, int C, long sy, long sx, long sc,
                     double L, double* map, int nthreads) {
  const int R = 5;
  double g[11], gs = 0.0;
  for (int i = -R; i <= R; ++i) {
    g[i + R] = exp(-((double)i * (double)i) / (2.0 * 1.5 * 1.5));
    gs += g[i + R];
  }
  for (int i = 0; i <= 2 * R; ++i) g[i] /= gs;
  const double C1 = (0.01 * L) * (0.01 * L);
  const double C2 = (0.03 * L) * (0.03 * L);
  int nt = 1;
#ifdef _OPENMP
  nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
#endif
#pragma omp parallel for num_threads(nt) schedule(static)
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      double total = 0.0;
      for (int c = 0; c < C; ++c) {
        double ma = 0.0, mb = 0.0;
        for (int j = -R; j <= R; ++j)
          for (int i = -R; i <= R; ++i) {
            long q = clampi(y + j, 0, H - 1) * sy + clampi(x + i, 0, W - 1) * sx + c * sc;
            double wij = g[i + R] * g[j + R];
            ma += wij * a[q];
            mb += wij * b[q];
          }
        double va = 0.0, vb = 0.0, cv = 0.0;
        for (int j = -R; j <= R; ++j)
          for (int i = -R; i <= R; ++i) {
            long q = clampi(y + j, 0, H - 1) * sy + clampi(x + i, 0, W - 1) * sx + c * sc;
            double wij = g[i + R] * g[j + R];
            double da = a[q] - ma, db = b[q] - mb;
            va += wij * da * da;
            vb += wij * db * db;
            cv += wij * da * db;
          }
        total += ((2.0 * ma * mb + C1) * (2.0 * cv + C2)) / ((ma * ma + mb * mb + C1) * (va + vb + C2));
      }
      map[(long)y * W + x] = total / (double)C;
    }
}

/* ------------------------------------------------------------------------
 * Gaussian-pyramid (mipmap) foveation: the earlier approach the paper
 * compares against (Section 3.2, Fig. 4, and its appendix on previous
 * foveated rendering): a Burt-Adelson pyramid (each level the previous one
 * convolved with a small Gaussian and subsampled by two in each axis), and
 * every output pixel interpolated from the pyramid at a fractional level.
 *
 *  - REDUCE with the 5-tap generating kernel w = (1, 4, 6, 4, 1) / 16,
 *    clamp-to-edge:  g_{l+1}(i, j) = sum_{m,n} w(m) w(n) g_l(2i + m, 2j + n),
 *    level sizes W_{l+1} = (W_l + 1) / 2 (samples at the even indices).
 *  - Sample i of level l sits on original pixel 2^l i. w has unit variance,
 *    so level l is the original blurred with variance (4^l - 1) / 3 (in
 *    original pixels, per axis); the level whose blur matches a pixel's
 *    sigma_p is L = log4(3 sigma_p^2 + 1), clamped to [0, top level].
 *  - out = (1 - f) S_{l0} + f S_{l0+1}, l0 = floor(L), f = L - l0, where S_l
 *    is the bilinear interpolation of level l at u = x / 2^l, v = y / 2^l
 *    (neighbour indices clamped to the level).
 * sigma_p is the per-pixel law at the pixel centre (oracle_pixel_sigma).
 * ------------------------------------------------------------------------ */

/* Number of levels of a W x H pyramid down to 1 x 1 (level 0 included). */
int oracle_pyramid_levels(int W, int H) {
  int n = 1;
  while (W > 1 || H > 1) {
    W = (W + 1) / 2;
    H = (H + 1) / 2;
    ++n;
  }
  return n;
}

/* One REDUCE of a plane (W x H, row-major) into (W+1)/2 x (H+1)/2. */
void oracle_pyramid_reduce(const double* in, int W, int H, double* out) {
  static const double w[5] = {1.0 / 16.0, 4.0 / 16.0, 6.0 / 16.0, 4.0 / 16.0, 1.0 / 16.0};
  int W2 = (W + 1) / 2, H2 = (H + 1) / 2;
  for (int j = 0; j < H2; ++j)
    for (int i = 0; i < W2; ++i) {
      double acc = 0.0;
      for (int n = -2; n <= 2; ++n)
        for (int m = -2; m <= 2; ++m)
          acc += w[n + 2] * w[m + 2] * in[(long)clampi(2 * j + n, 0, H - 1) * W + clampi(2 * i + m, 0, W - 1)];
      out[(long)j * W2 + i] = acc;
    }
}

/* Bilinear sample of a level plane (Wl x Hl) at level coordinates (u, v). */
static double bilinear(const double* g, int Wl, int Hl, double u, double v) {
  int i0 = (int)floor(u), j0 = (int)floor(v);
  double fu = u - (double)i0, fv = v - (double)j0;
  int i1 = clampi(i0 + 1, 0, Wl - 1), j1 = clampi(j0 + 1, 0, Hl - 1);
  i0 = clampi(i0, 0, Wl - 1);
  j0 = clampi(j0, 0, Hl - 1);
  return (1.0 - fu) * (1.0 - fv) * g[(long)j0 * Wl + i0] + fu * (1.0 - fv) * g[(long)j0 * Wl + i1] +
         (1.0 - fu) * fv * g[(long)j1 * Wl + i0] + fu * fv * g[(long)j1 * Wl + i1];
}

/* Pyramid foveation of the listed pixels (all when pixel_list is NULL);
 * layout as oracle_forward_ex. */
void oracle_forward_pyramid(const double* in, double* out, int W, int H, int C, long sy, long sx, long sc,
                            double fx, double fy, double sigma0, double k, const long* pixel_list, long nlist) {
  int NL = oracle_pyramid_levels(W, H);
  double** lev = (double**)malloc((size_t)NL * sizeof(double*));
  int* lw = (int*)malloc((size_t)NL * sizeof(int));
  int* lh = (int*)malloc((size_t)NL * sizeof(int));
  long np = pixel_list ? nlist : (long)W * (long)H;
  for (int c = 0; c < C; ++c) {
    lw[0] = W;
    lh[0] = H;
    lev[0] = (double*)malloc((size_t)W * H * sizeof(double));
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) lev[0][(long)y * W + x] = in[y * sy + x * sx + c * sc];
    for (int l = 1; l < NL; ++l) {
      lw[l] = (lw[l - 1] + 1) / 2;
      lh[l] = (lh[l - 1] + 1) / 2;
      lev[l] = (double*)malloc((size_t)lw[l] * lh[l] * sizeof(double));
      oracle_pyramid_reduce(lev[l - 1], lw[l - 1], lh[l - 1], lev[l]);
    }
    for (long t = 0; t < np; ++t) {
      long p = pixel_list ? pixel_list[t] : t;
      int x = (int)(p % W), y = (int)(p / W);
      double sigma;
      int r;
      oracle_pixel_sigma(x, y, fx, fy, sigma0, k, &sigma, &r);
      double L = log(3.0 * sigma * sigma + 1.0) / log(4.0);
      if (L < 0.0) L = 0.0;
      if (L > (double)(NL - 1)) L = (double)(NL - 1);
      int l0 = (int)floor(L);
      double f = L - (double)l0;
      double s0 = bilinear(lev[l0], lw[l0], lh[l0], (double)x / ldexp(1.0, l0), (double)y / ldexp(1.0, l0));
      double v = s0;
      if (l0 + 1 < NL && f > 0.0) {
        double s1 = bilinear(lev[l0 + 1], lw[l0 + 1], lh[l0 + 1], (double)x / ldexp(1.0, l0 + 1),
                             (double)y / ldexp(1.0, l0 + 1));
        v = (1.0 - f) * s0 + f * s1;
      }
      out[y * sy + x * sx + c * sc] = v;
    }
    for (int l = 0; l < NL; ++l) free(lev[l]);
  }
  free(lh);
  free(lw);
  free(lev);
}
