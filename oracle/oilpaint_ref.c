/*
 * oracle/oilpaint_ref.c -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.
 *
 * A plain, slow, obviously-correct CPU implementation of the histogram
 * oil-paint filter of S. Mukherjee, "Study on performance improvement of oil
 * paint image filter algorithm using Parallel Pattern Library" (arXiv
 * 1405.1020).  Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg may load this library.  It shares no code, header or constant
 * with the CUDA path.
 *
 * What it computes, per output pixel (x, y), in the order of section 4
 * ("Histogram based algorithm for Oil Paint") and its sequential listing:
 *   1. start from an empty histogram of L intensity levels, each level
 *      holding a pixel count and the running sums of R, G and B;
 *   2. visit every neighbour of the square (2r+1) x (2r+1) window centred on
 *      (x, y) (the two nested loops over -radius..radius in section 4);
 *      neighbours outside the image are skipped;
 *   3. give each neighbour the level floor((R+G+B) * L / 765) -- section 4
 *      writes it as ((r+g+b)*intensity_level/3.0)/255 truncated to int, which
 *      equals this integer quotient for every R+G+B in 0..765 and L in 1..256
 *      (tests pin the equality exhaustively) -- clamped to L-1 so that pure
 *      white (R+G+B = 765, the only sum that reaches level L) joins the top
 *      level; a second level mode, floor(floor((R+G+B)/3) * L / 255), also
 *      clamped, is provided for callers that want integer division by 3 first;
 *   4. add one to that level's count and the neighbour's R, G, B to its sums;
 *   5. pick the level with the largest count, scanning levels upward from 0
 *      and replacing the current best only on a strictly larger count, so the
 *      lowest level wins a tie (section 4's "most frequently occurring
 *      intensity");
 *   6. write each colour channel as that level's sum divided by its count,
 *      truncating (section 4, step 3: the channel-wise average of the pixels
 *      holding the most frequent intensity).
 * The centre pixel is always inside the image, so the winning count is >= 1.
 * With 4 bytes per pixel the fourth byte (alpha) is ignored by the filter
 * and copied from the input's centre pixel.  Bytes past width*bpp in a row
 * (row padding) are never written.
 *
 * Literal mode (mode bit ORC_LITERAL) follows the section-4 listing as
 * printed instead of the readings above:
 *   - only pixels with r <= x < w-r and r <= y < h-r are visited (the
 *     listing's loops start at radius and stop radius short of each edge),
 *     so every window lies inside the image; nothing else is written, and
 *     nothing at all when w <= 2r or h <= 2r;
 *   - the level is not clamped: pure white lands on level L, which the
 *     listing counts (its arrays hold 255 levels, so L <= 254) but whose
 *     count its argmax, running over levels 0..L-1, never reads;
 *   - the argmax starts from level 0's count and keeps the first strictly
 *     larger count, as in step 5; when every level below L is empty (a
 *     window of white pixels only) the listing's guard skips the write;
 *   - only the three colour bytes are written.
 * The listing clears only the first 255 bytes of each 255-entry int array
 * per pixel; its prose asks for a fresh histogram per pixel, which both
 * modes use (the two agree whenever L <= 63: levels 0..62 are cleared).
 *
 * Threads: rows are independent, so they are split across worker threads the
 * way section 5 splits them across parallel_for tasks; every thread owns its
 * histogram and the output does not depend on the thread count.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORC_LEVEL_PAPER 0u
#define ORC_LEVEL_INTDIV3 1u
#define ORC_LITERAL 2u /* mode bit: the listing as printed (see above) */

typedef struct {
  const uint8_t *in;
  uint8_t *out;
  uint32_t w, h, stride, bpp;
  int32_t r;
  uint32_t L, mode;
  /* rows handled: y = y_begin + k * y_step for k >= 0 while y < y_end */
  uint32_t y_begin, y_end, y_step;
  int status;
} orc_job_t;

/* Step 3 above (literal mode: not clamped, so white reaches level L). */
static uint32_t orc_level(uint32_t R, uint32_t G, uint32_t B, uint32_t L, uint32_t mode) {
  uint32_t s = R + G + B;
  uint32_t l;
  if (mode & ORC_LEVEL_INTDIV3)
    l = ((s / 3u) * L) / 255u;
  else
    l = (s * L) / 765u;
  if (mode & ORC_LITERAL) return l;
  return l < L ? l : L - 1u;
}

/* Steps 1-6 for one output pixel; writes rgb[0..2] and returns 1, or returns
 * 0 (literal mode, no level below L in the window) without writing.  The
 * arrays hold L + 1 levels. */
static int orc_pixel(const uint8_t *in, uint32_t w, uint32_t h, uint32_t stride, uint32_t bpp,
                     int32_t r, uint32_t L, uint32_t mode, uint32_t x, uint32_t y,
                     uint32_t *count, uint32_t *sumR, uint32_t *sumG, uint32_t *sumB,
                     uint8_t rgb[3]) {
  /* step 1 */
  memset(count, 0, (L + 1u) * sizeof(uint32_t));
  memset(sumR, 0, (L + 1u) * sizeof(uint32_t));
  memset(sumG, 0, (L + 1u) * sizeof(uint32_t));
  memset(sumB, 0, (L + 1u) * sizeof(uint32_t));
  /* step 2 */
  for (int32_t dy = -r; dy <= r; ++dy) {
    for (int32_t dx = -r; dx <= r; ++dx) {
      int64_t yy = (int64_t)y + dy, xx = (int64_t)x + dx;
      if (yy < 0 || yy >= (int64_t)h || xx < 0 || xx >= (int64_t)w) continue;
      const uint8_t *p = in + (size_t)yy * stride + (size_t)xx * bpp;
      uint32_t R = p[0], G = p[1], B = p[2];
      uint32_t l = orc_level(R, G, B, L, mode); /* step 3 */
      count[l] += 1u;                            /* step 4 */
      sumR[l] += R;
      sumG[l] += G;
      sumB[l] += B;
    }
  }
  /* step 5 */
  uint32_t best = 0;
  for (uint32_t l = 1; l < L; ++l)
    if (count[l] > count[best]) best = l;
  if (count[best] == 0) return 0; /* literal mode only: the listing's guard */
  /* step 6 */
  rgb[0] = (uint8_t)(sumR[best] / count[best]);
  rgb[1] = (uint8_t)(sumG[best] / count[best]);
  rgb[2] = (uint8_t)(sumB[best] / count[best]);
  return 1;
}

static void *orc_worker(void *arg) {
  orc_job_t *j = (orc_job_t *)arg;
  const uint32_t n = j->L + 1u;
  uint32_t *bins = (uint32_t *)malloc((size_t)4 * n * sizeof(uint32_t));
  if (!bins) {
    j->status = -3;
    return NULL;
  }
  uint32_t *count = bins, *sumR = bins + n, *sumG = bins + 2 * n, *sumB = bins + 3 * n;
  const int literal = (j->mode & ORC_LITERAL) != 0;
  /* literal mode: the listing's loop bounds, radius .. size-radius-1 */
  const int64_t r = j->r;
  const int64_t x_lo = literal ? r : 0, x_hi = literal ? (int64_t)j->w - r : (int64_t)j->w;
  const int64_t y_lo = literal ? r : 0, y_hi = literal ? (int64_t)j->h - r : (int64_t)j->h;
  for (uint32_t y = j->y_begin; y < j->y_end; y += j->y_step) {
    if ((int64_t)y < y_lo || (int64_t)y >= y_hi) continue;
    for (int64_t xi = x_lo; xi < x_hi; ++xi) {
      const uint32_t x = (uint32_t)xi;
      uint8_t rgb[3];
      if (!orc_pixel(j->in, j->w, j->h, j->stride, j->bpp, j->r, j->L, j->mode, x, y, count,
                     sumR, sumG, sumB, rgb))
        continue;
      uint8_t *o = j->out + (size_t)y * j->stride + (size_t)x * j->bpp;
      o[0] = rgb[0];
      o[1] = rgb[1];
      o[2] = rgb[2];
      if (j->bpp == 4 && !literal) o[3] = j->in[(size_t)y * j->stride + (size_t)x * 4 + 3];
    }
  }
  free(bins);
  return NULL;
}

static int orc_check(uint32_t w, uint32_t h, uint32_t stride, uint32_t bpp, int32_t r,
                     uint32_t L, uint32_t mode) {
  if (w == 0 || h == 0) return -1;
  if (bpp != 3 && bpp != 4) return -1;
  if ((uint64_t)stride < (uint64_t)w * bpp) return -1;
  if (r < 0 || r > 1000) return -1;
  if (L < 1 || L > 256) return -1;
  if (mode & ~(ORC_LEVEL_INTDIV3 | ORC_LITERAL)) return -1;
  if ((mode & ORC_LITERAL) && L > 254) return -1; /* level L must index a 255-entry array */
  return 0;
}

int orc_num_cpus(void) {
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n > 0 ? (int)n : 1;
}

/*
 * Filters rows [y_begin, y_end) of a w x h image (the window still sees every
 * row of the image).  in/out: host buffers of at least h*stride bytes, rows
 * `stride` bytes apart, `bpp` bytes per pixel (R, G, B[, A]).  threads <= 0
 * means one thread per online CPU.  Returns 0, -1 on bad arguments, -3 on
 * allocation failure.
 */
int orc_oilpaint_rows(const uint8_t *in, uint8_t *out, uint32_t w, uint32_t h, uint32_t stride,
                      uint32_t bpp, int32_t r, uint32_t L, uint32_t mode, uint32_t y_begin,
                      uint32_t y_end, int threads) {
  if (!in || !out) return -1;
  if (orc_check(w, h, stride, bpp, r, L, mode)) return -1;
  if (y_end > h || y_begin > y_end) return -1;
  if (y_begin == y_end) return 0;
  int nt = threads > 0 ? threads : orc_num_cpus();
  if ((uint32_t)nt > y_end - y_begin) nt = (int)(y_end - y_begin);
  orc_job_t *jobs = (orc_job_t *)calloc((size_t)nt, sizeof(orc_job_t));
  pthread_t *tids = (pthread_t *)calloc((size_t)nt, sizeof(pthread_t));
  if (!jobs || !tids) {
    free(jobs);
    free(tids);
    return -3;
  }
  int status = 0;
  for (int t = 0; t < nt; ++t) {
    orc_job_t j = {in, out, w, h, stride, bpp, r, L, mode, y_begin + (uint32_t)t, y_end,
                   (uint32_t)nt, 0};
    jobs[t] = j;
  }
  int started = 0;
  for (int t = 1; t < nt; ++t) {
    if (pthread_create(&tids[t], NULL, orc_worker, &jobs[t]) != 0) break;
    started = t;
  }
  orc_worker(&jobs[0]);
  for (int t = 1; t <= started; ++t) pthread_join(tids[t], NULL);
  /* rows of workers that failed to start are done here, serially */
  for (int t = started + 1; t < nt; ++t) orc_worker(&jobs[t]);
  for (int t = 0; t < nt; ++t)
    if (jobs[t].status) status = jobs[t].status;
  free(jobs);
  free(tids);
  return status;
}

/* Whole image. */
int orc_oilpaint(const uint8_t *in, uint8_t *out, uint32_t w, uint32_t h, uint32_t stride,
                 uint32_t bpp, int32_t r, uint32_t L, uint32_t mode, int threads) {
  return orc_oilpaint_rows(in, out, w, h, stride, bpp, r, L, mode, 0, h, threads);
}

/*
 * Individual pixels: for k < n, computes pixel (xs[k], ys[k]) and writes its
 * R, G, B to rgb[3k..3k+2].  Used to check sampled outputs of large images.
 */
int orc_oilpaint_pixels(const uint8_t *in, uint32_t w, uint32_t h, uint32_t stride,
                        uint32_t bpp, int32_t r, uint32_t L, uint32_t mode, const uint32_t *xs,
                        const uint32_t *ys, uint32_t n, uint8_t *rgb) {
  if (!in || (n && (!xs || !ys || !rgb))) return -1;
  if (orc_check(w, h, stride, bpp, r, L, mode)) return -1;
  if (mode & ORC_LITERAL) return -1; /* sampled pixels: the default readings only */
  const uint32_t nb = L + 1u;
  uint32_t *bins = (uint32_t *)malloc((size_t)4 * nb * sizeof(uint32_t));
  if (!bins) return -3;
  for (uint32_t k = 0; k < n; ++k) {
    if (xs[k] >= w || ys[k] >= h) {
      free(bins);
      return -1;
    }
    orc_pixel(in, w, h, stride, bpp, r, L, mode, xs[k], ys[k], bins, bins + nb, bins + 2 * nb,
              bins + 3 * nb, rgb + 3 * (size_t)k);
  }
  free(bins);
  return 0;
}

/* The level of step 3 for one R+G+B sum, exported so tests can pin it. */
uint32_t orc_level_of_sum(uint32_t s, uint32_t L, uint32_t mode) {
  /* split s into channels that add back to s; orc_level only uses the sum */
  uint32_t R = s > 255u ? 255u : s;
  uint32_t rest = s - R;
  uint32_t G = rest > 255u ? 255u : rest;
  uint32_t B = rest - G;
  return orc_level(R, G, B, L, mode);
}
