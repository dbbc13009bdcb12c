/*
 * Köhler contrast-curve ORACLE — test infrastructure, not part of the product.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this code.  It shares nothing with the CUDA library: no header, no table,
 * no helper.  It is deliberately plain and slow so that a reader can check each
 * loop against the paper ("Speeding up the Köhler's method of contrast
 * thresholding", G. Noyel) by eye.
 *
 * What it computes (Section 2.1, Eq. 1-4), for an image f on a W x H grid with
 * integer values in [0, M[ and every integer threshold t in [0, M[:
 *
 *   card(t) = #B(t),  B(t) = { (x0,x1) : x1 in N4(x0), f(x0) <= t < f(x1) }   (Eq. 1)
 *   sumc(t) = sum over B(t) of min(f(x1) - t, t - f(x0))                     (Eq. 2)
 *   C(t)    = sumc(t) / card(t)                                               (Eq. 3)
 *
 * Only pairs with both pixels inside the image exist (Eq. 1 takes (x0,x1) in D^2).
 * card and sumc are exact unsigned 64-bit integers; C(t) is the IEEE double
 * quotient (round to nearest) of the two converted integers, and 0.0 where
 * card(t) = 0 (the normalisation step of Algorithm 1 divides by zero there).
 *
 * Four ways to the same integers are provided, so that the tests can pin them
 * against each other and against a brute-force set construction:
 *   oracle_curve_n4    ordered pairs over the full 4-neighbourhood, literally Eq. 1-2;
 *   oracle_curve       unordered pairs of the half neighbourhood N4* (right, down),
 *                      which Section 3.2 (Eq. 7-9) proves gives the same sums;
 *   oracle_curve_at    the same as oracle_curve, but only at a list of thresholds;
 *   oracle_curve_alg1  Algorithm 1 (per image line, per neighbour of N4*, add the
 *                      contribution of the pair to every t in [min, max-1]),
 *                      with per-thread accumulators summed at the end (Section 3.3).
 * oracle_curve_n8, oracle_curve_n8half and oracle_curve_n8_alg1 are the same three
 * routes with the 8-neighbourhood (ordered N8, half neighbourhood N8* = right,
 * down, down-right, down-left, and Algorithm 1 over the four N8* translations).
 * oracle_curve_n6, oracle_curve_n6half and oracle_curve_n6_alg1 do the same with
 * the 6-neighbourhood of a hexagonal grid (odd rows shifted half a pixel right).
 * oracle_thresholds selects the local maxima of C (Section 2.1, text after Eq. 4
 * and Fig. 1) and the optimal threshold t0 of Eq. 4 with exact rational
 * comparisons.
 *
 * Pixel layout: row-major, `pitch` bytes between row starts, elem_size 1 (uint8)
 * or 2 (uint16, host byte order).  Return value: 0 on success, -1 on a bad
 * argument, -3 if some pixel value is >= M.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ERR_ARG (-1)
#define ORACLE_ERR_RANGE (-3)

static uint32_t pixel(const void* img, int elem_size, int64_t pitch, int64_t x, int64_t y) {
  const unsigned char* row = (const unsigned char*)img + y * pitch;
  if (elem_size == 1) return row[x];
  uint16_t v;
  memcpy(&v, row + 2 * x, 2);
  return v;
}

static int check_args(const void* img, int elem_size, int64_t W, int64_t H, int64_t pitch, int32_t M) {
  if (!img || (elem_size != 1 && elem_size != 2) || W < 1 || H < 1 || pitch < W * elem_size || M < 2)
    return ORACLE_ERR_ARG;
  for (int64_t y = 0; y < H; ++y)
    for (int64_t x = 0; x < W; ++x)
      if (pixel(img, elem_size, pitch, x, y) >= (uint32_t)M) return ORACLE_ERR_RANGE;
  return ORACLE_OK;
}

static uint64_t min_u64(uint64_t a, uint64_t b) { return a < b ? a : b; }

/* Eq. 1-2 literally: every ordered pair (x0, x1) with x1 one of the four
 * neighbours of x0 inside the image; the pair is in B(t) when f(x0) <= t < f(x1). */
int oracle_curve_n4(const void* img, int elem_size, int64_t W, int64_t H, int64_t pitch, int32_t M,
                    uint64_t* card, uint64_t* sumc) {
  int rc = check_args(img, elem_size, W, H, pitch, M);
  if (rc) return rc;
  if (!card || !sumc) return ORACLE_ERR_ARG;
  static const int dx[4] = {1, -1, 0, 0};
  static const int dy[4] = {0, 0, 1, -1};
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t t = 0; t < M; ++t) {
    uint64_t n = 0, s = 0;
    for (int64_t y = 0; y < H; ++y)
      for (int64_t x = 0; x < W; ++x) {
        uint64_t f0 = pixel(img, elem_size, pitch, x, y);
        for (int k = 0; k < 4; ++k) {
          int64_t x1 = x + dx[k], y1 = y + dy[k];
          if (x1 < 0 || x1 >= W || y1 < 0 || y1 >= H) continue;
          uint64_t f1 = pixel(img, elem_size, pitch, x1, y1);
          if (f0 <= (uint64_t)t && (uint64_t)t < f1) {
            n += 1;
            s += min_u64(f1 - (uint64_t)t, (uint64_t)t - f0);
          }
        }
      }
    card[t] = n;
    sumc[t] = s;
  }
  return ORACLE_OK;
}

/* One threshold over the half neighbourhood N4* (right and down neighbours).
 * The pair {x0, x1} is taken without order: with lo/hi the smaller/larger value,
 * it is in the boundary when lo <= t < hi and contributes min(hi - t, t - lo)
 * (Eq. 7 and Eq. 9: of the two ordered pairs at most one is in B(t)). */
static void half_nbhd_at(const void* img, int elem_size, int64_t W, int64_t H, int64_t pitch, uint64_t t,
                         uint64_t* n_out, uint64_t* s_out) {
  uint64_t n = 0, s = 0;
  for (int64_t y = 0; y < H; ++y)
    for (int64_t x = 0; x < W; ++x) {
      uint64_t f0 = pixel(img, elem_size, pitch, x, y);
      for (int k = 0; k < 2; ++k) {
        int64_t x1 = x + (k == 0), y1 = y + (k == 1);
        if (x1 >= W || y1 >= H) continue;
        uint64_t f1 = pixel(img, elem_size, pitch, x1, y1);
        uint64_t lo = f0 < f1 ? f0 : f1, hi = f0 < f1 ? f1 : f0;
        if (lo <= t && t < hi) {
          n += 1;
          s += min_u64(hi - t, t - lo);
        }
      }
    }
  *n_out = n;
  *s_out = s;
}

int oracle_curve(const void* img, int elem_size, int64_t W, int64_t H, int64_t pitch, int32_t M,
                 uint64_t* card, uint64_t* sumc) {
  int rc = check_args(img, elem_size, W, H, pitch, M);
  if (rc) return rc;
  if (!card || !sumc) return ORACLE_ERR_ARG;
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t t = 0; t < M; ++t) half_nbhd_at(img, elem_size, W, H, pitch, (uint64_t)t, &card[t], &sumc[t]);
  return ORACLE_OK;
}

int oracle_curve_at(const void* img, int elem_size, int64_t W, int64_t H, int64_t pitch, int32_t M,
                    const int32_t* ts, int32_t n_t, uint64_t* card, uint64_t* sumc) {
  int rc = check_args(img, elem_size, W, H, pitch, M);
  if (rc) return rc;
  if (!ts || n_t < 0 || !card || !sumc) return ORACLE_ERR_ARG;
  for (int32_t i = 0; i < n_t; ++i)
    if (ts[i] < 0 || ts[i] >= M) return ORACLE_ERR_ARG;
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t i = 0; i < n_t; ++i) half_nbhd_at(img, elem_size, W, H, pitch, (uint64_t)ts[i], &card[i], &sumc[i]);
  return ORACLE_OK;
}

/* Algorithm 1 (Section 3.1) with the parallel organisation of Section 3.3: image
 * lines are shared among threads; each thread keeps its own C_k / Card_k arrays
 * of length M, and the arrays are summed after the parallel loop.  For line i and
 * each translation a of N4* = {right, down}, the neighbour of column j is read
 * directly (a neighbour outside the image gives no pair); mini/maxi are the pair's
 * smaller and larger values and every t in [mini, maxi - 1] receives
 * min(maxi - t, t - mini) in C and 1 in card. */
int oracle_curve_alg1(const void* img, int elem_size, int64_t W, int64_t H, int64_t pitch, int32_t M,
                      uint64_t* card, uint64_t* sumc) {
  int rc = check_args(img, elem_size, W, H, pitch, M);
  if (rc) return rc;
  if (!card || !sumc) return ORACLE_ERR_ARG;
  for (int32_t t = 0; t < M; ++t) card[t] = sumc[t] = 0;
  int failed = 0;
#pragma omp parallel
  {
    uint64_t* Ck = (uint64_t*)calloc((size_t)M, sizeof(uint64_t));
    uint64_t* Cardk = (uint64_t*)calloc((size_t)M, sizeof(uint64_t));
    int ok = Ck && Cardk;
#pragma omp for schedule(static)
    for (int64_t i = 0; i < H; ++i) {
      if (!ok) continue;
      for (int a = 0; a < 2; ++a) {       /* a = 0: right neighbour, a = 1: lower neighbour */
        int64_t ay = (a == 1), ax = (a == 0);
        if (i + ay >= H) continue;
        for (int64_t j = 0; j + ax < W; ++j) {
          uint64_t cur = pixel(img, elem_size, pitch, j, i);
          uint64_t nb = pixel(img, elem_size, pitch, j + ax, i + ay);
          uint64_t mini = cur < nb ? cur : nb, maxi = cur < nb ? nb : cur;
          for (uint64_t t = mini; t < maxi; ++t) {
            Ck[t] += min_u64(maxi - t, t - mini);
            Cardk[t] += 1;
          }
        }
      }
    }
#pragma omp critical
    {
      if (ok) {
        for (int32_t t = 0; t < M; ++t) {
          sumc[t] += Ck[t];
          card[t] += Cardk[t];
        }
      } else {
        failed = 1;
      }
    }
    free(Ck);
    free(Cardk);
  }
  return failed ? ORACLE_ERR_ARG : ORACLE_OK;
}

/* The 8-neighbourhood (Section 2: the method is stated for the 4-neighbourhood
 * and the text notes that the 8- (or 6-) neighbourhood gives insignificant
 * differences).  The definitions are the same with N8 in place of N4 in Eq. 1:
 * x1 one of the eight neighbours of x0, the diagonals included. */
static const int n8_dx[8] = {1, -1, 0, 0, 1, -1, 1, -1};
static const int n8_dy[8] = {0, 0, 1, -1, 1, -1, -1, 1};

/* Eq. 1-2 literally over ordered pairs of the full 8-neighbourhood. */
int oracle_curve_n8(const void* img, int elem_size, int64_t W, int64_t H, int64_t pitch, int32_t M,
                    uint64_t* card, uint64_t* sumc) {
  int rc = check_args(img, elem_size, W, H, pitch, M);
  if (rc) return rc;
  if (!card || !sumc) return ORACLE_ERR_ARG;
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t t = 0; t < M; ++t) {
    uint64_t n = 0, s = 0;
    for (int64_t y = 0; y < H; ++y)
      for (int64_t x = 0; x < W; ++x) {
        uint64_t f0 = pixel(img, elem_size, pitch, x, y);
        for (int k = 0; k < 8; ++k) {
          int64_t x1 = x + n8_dx[k], y1 = y + n8_dy[k];
          if (x1 < 0 || x1 >= W || y1 < 0 || y1 >= H) continue;
          uint64_t f1 = pixel(img, elem_size, pitch, x1, y1);
          if (f0 <= (uint64_t)t && (uint64_t)t < f1) {
            n += 1;
            s += min_u64(f1 - (uint64_t)t, (uint64_t)t - f0);
          }
        }
      }
    card[t] = n;
    sumc[t] = s;
  }
  return ORACLE_OK;
}

/* The half 8-neighbourhood N8* = {right, down, down-right, down-left}: every
 * unordered 8-neighbour pair exactly once (the argument of Section 3.2, Eq. 7-9,
 * holds for any symmetric neighbourhood); per threshold, per pair, as
 * oracle_curve does for N4*. */
int oracle_curve_n8half(const void* img, int elem_size, int64_t W, int64_t H, int64_t pitch, int32_t M,
                        uint64_t* card, uint64_t* sumc) {
  int rc = check_args(img, elem_size, W, H, pitch, M);
  if (rc) return rc;
  if (!card || !sumc) return ORACLE_ERR_ARG;
  static const int hdx[4] = {1, 0, 1, -1};
  static const int hdy[4] = {0, 1, 1, 1};
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t t = 0; t < M; ++t) {
    uint64_t n = 0, s = 0;
    for (int64_t y = 0; y < H; ++y)
      for (int64_t x = 0; x < W; ++x) {
        uint64_t f0 = pixel(img, elem_size, pitch, x, y);
        for (int k = 0; k < 4; ++k) {
          int64_t x1 = x + hdx[k], y1 = y + hdy[k];
          if (x1 < 0 || x1 >= W || y1 >= H) continue;
          uint64_t f1 = pixel(img, elem_size, pitch, x1, y1);
          uint64_t lo = f0 < f1 ? f0 : f1, hi = f0 < f1 ? f1 : f0;
          if (lo <= (uint64_t)t && (uint64_t)t < hi) {
            n += 1;
            s += min_u64(hi - (uint64_t)t, (uint64_t)t - lo);
          }
        }
      }
    card[t] = n;
    sumc[t] = s;
  }
  return ORACLE_OK;
}

/* Algorithm 1 with the four translations of N8* instead of the two of N4*
 * (same per-thread accumulators, Section 3.3). */
int oracle_curve_n8_alg1(const void* img, int elem_size, int64_t W, int64_t H, int64_t pitch, int32_t M,
                         uint64_t* card, uint64_t* sumc) {
  int rc = check_args(img, elem_size, W, H, pitch, M);
  if (rc) return rc;
  if (!card || !sumc) return ORACLE_ERR_ARG;
  static const int hdx[4] = {1, 0, 1, -1};
  static const int hdy[4] = {0, 1, 1, 1};
  for (int32_t t = 0; t < M; ++t) card[t] = sumc[t] = 0;
  int failed = 0;
#pragma omp parallel
  {
    uint64_t* Ck = (uint64_t*)calloc((size_t)M, sizeof(uint64_t));
    uint64_t* Cardk = (uint64_t*)calloc((size_t)M, sizeof(uint64_t));
    int ok = Ck && Cardk;
#pragma omp for schedule(static)
    for (int64_t i = 0; i < H; ++i) {
      if (!ok) continue;
      for (int a = 0; a < 4; ++a) {
        if (i + hdy[a] >= H) continue;
        for (int64_t j = 0; j < W; ++j) {
          int64_t j1 = j + hdx[a];
          if (j1 < 0 || j1 >= W) continue;
          uint64_t cur = pixel(img, elem_size, pitch, j, i);
          uint64_t nb = pixel(img, elem_size, pitch, j1, i + hdy[a]);
          uint64_t mini = cur < nb ? cur : nb, maxi = cur < nb ? nb : cur;
          for (uint64_t t = mini; t < maxi; ++t) {
            Ck[t] += min_u64(maxi - t, t - mini);
            Cardk[t] += 1;
          }
        }
      }
    }
#pragma omp critical
    {
      if (ok) {
        for (int32_t t = 0; t < M; ++t) {
          sumc[t] += Ck[t];
          card[t] += Cardk[t];
        }
      } else {
        failed = 1;
      }
    }
    free(Ck);
    free(Cardk);
  }
  return failed ? ORACLE_ERR_ARG : ORACLE_OK;
}

/* The 6-neighbourhood of a hexagonal grid (Section 2 names it beside the 8-
 * neighbourhood).  The grid is stored row by row with every odd row (0-based)
 * shifted half a pixel to the right, so that the pixel (x, y) touches:
 *   (x - 1, y), (x + 1, y), and in the rows y - 1 and y + 1
 *   columns x - 1 and x when y is even, columns x and x + 1 when y is odd.
 * The relation is symmetric: an even-row pixel's lower-left neighbour has it as
 * its upper-right one.  Eq. 1-3 are unchanged with N6 in place of N4. */
static void n6_neighbour(int64_t x, int64_t y, int k, int64_t* x1, int64_t* y1) {
  /* k = 0..5: right, left, up (same column), down (same column), up-shifted,
   * down-shifted; the shifted column is x - 1 on even rows, x + 1 on odd rows */
  int64_t shift = (y % 2 == 0) ? -1 : 1;
  static const int dx0[6] = {1, -1, 0, 0, 0, 0};
  static const int dy0[6] = {0, 0, -1, 1, -1, 1};
  *x1 = x + dx0[k] + (k >= 4 ? shift : 0);
  *y1 = y + dy0[k];
}

/* Eq. 1-2 literally over ordered pairs of the full 6-neighbourhood. */
int oracle_curve_n6(const void* img, int elem_size, int64_t W, int64_t H, int64_t pitch, int32_t M,
                    uint64_t* card, uint64_t* sumc) {
  int rc = check_args(img, elem_size, W, H, pitch, M);
  if (rc) return rc;
  if (!card || !sumc) return ORACLE_ERR_ARG;
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t t = 0; t < M; ++t) {
    uint64_t n = 0, s = 0;
    for (int64_t y = 0; y < H; ++y)
      for (int64_t x = 0; x < W; ++x) {
        uint64_t f0 = pixel(img, elem_size, pitch, x, y);
        for (int k = 0; k < 6; ++k) {
          int64_t x1, y1;
          n6_neighbour(x, y, k, &x1, &y1);
          if (x1 < 0 || x1 >= W || y1 < 0 || y1 >= H) continue;
          uint64_t f1 = pixel(img, elem_size, pitch, x1, y1);
          if (f0 <= (uint64_t)t && (uint64_t)t < f1) {
            n += 1;
            s += min_u64(f1 - (uint64_t)t, (uint64_t)t - f0);
          }
        }
      }
    card[t] = n;
    sumc[t] = s;
  }
  return ORACLE_OK;
}

/* The half 6-neighbourhood N6* = {right, down, down-shifted}: every unordered
 * 6-neighbour pair once (Section 3.2's argument, Eq. 7-9, for a symmetric
 * neighbourhood); per threshold, per pair. */
int oracle_curve_n6half(const void* img, int elem_size, int64_t W, int64_t H, int64_t pitch, int32_t M,
                        uint64_t* card, uint64_t* sumc) {
  int rc = check_args(img, elem_size, W, H, pitch, M);
  if (rc) return rc;
  if (!card || !sumc) return ORACLE_ERR_ARG;
  static const int half[3] = {0, 3, 5};  /* right, down, down-shifted in n6_neighbour */
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t t = 0; t < M; ++t) {
    uint64_t n = 0, s = 0;
    for (int64_t y = 0; y < H; ++y)
      for (int64_t x = 0; x < W; ++x) {
        uint64_t f0 = pixel(img, elem_size, pitch, x, y);
        for (int k = 0; k < 3; ++k) {
          int64_t x1, y1;
          n6_neighbour(x, y, half[k], &x1, &y1);
          if (x1 < 0 || x1 >= W || y1 >= H) continue;
          uint64_t f1 = pixel(img, elem_size, pitch, x1, y1);
          uint64_t lo = f0 < f1 ? f0 : f1, hi = f0 < f1 ? f1 : f0;
          if (lo <= (uint64_t)t && (uint64_t)t < hi) {
            n += 1;
            s += min_u64(hi - (uint64_t)t, (uint64_t)t - lo);
          }
        }
      }
    card[t] = n;
    sumc[t] = s;
  }
  return ORACLE_OK;
}

/* Algorithm 1 over the three translations of N6*: line i against itself moved
 * one column (right pairs), against line i + 1 (down pairs) and against line
 * i + 1 moved one column left (i even) or right (i odd) (Section 3.3 accumulators). */
int oracle_curve_n6_alg1(const void* img, int elem_size, int64_t W, int64_t H, int64_t pitch, int32_t M,
                         uint64_t* card, uint64_t* sumc) {
  int rc = check_args(img, elem_size, W, H, pitch, M);
  if (rc) return rc;
  if (!card || !sumc) return ORACLE_ERR_ARG;
  for (int32_t t = 0; t < M; ++t) card[t] = sumc[t] = 0;
  int failed = 0;
#pragma omp parallel
  {
    uint64_t* Ck = (uint64_t*)calloc((size_t)M, sizeof(uint64_t));
    uint64_t* Cardk = (uint64_t*)calloc((size_t)M, sizeof(uint64_t));
    int ok = Ck && Cardk;
#pragma omp for schedule(static)
    for (int64_t i = 0; i < H; ++i) {
      if (!ok) continue;
      int64_t shift = (i % 2 == 0) ? -1 : 1;
      const int64_t adx[3] = {1, 0, shift};
      const int64_t ady[3] = {0, 1, 1};
      for (int a = 0; a < 3; ++a) {
        if (i + ady[a] >= H) continue;
        for (int64_t j = 0; j < W; ++j) {
          int64_t j1 = j + adx[a];
          if (j1 < 0 || j1 >= W) continue;
          uint64_t cur = pixel(img, elem_size, pitch, j, i);
          uint64_t nb = pixel(img, elem_size, pitch, j1, i + ady[a]);
          uint64_t mini = cur < nb ? cur : nb, maxi = cur < nb ? nb : cur;
          for (uint64_t t = mini; t < maxi; ++t) {
            Ck[t] += min_u64(maxi - t, t - mini);
            Cardk[t] += 1;
          }
        }
      }
    }
#pragma omp critical
    {
      if (ok) {
        for (int32_t t = 0; t < M; ++t) {
          sumc[t] += Ck[t];
          card[t] += Cardk[t];
        }
      } else {
        failed = 1;
      }
    }
    free(Ck);
    free(Cardk);
  }
  return failed ? ORACLE_ERR_ARG : ORACLE_OK;
}

/* Normalisation step of Algorithm 1 (C(t) <- C(t) / card(t)); C(t) = 0 where the
 * boundary is empty. */
void oracle_normalise(const uint64_t* card, const uint64_t* sumc, int32_t M, double* curve) {
  for (int32_t t = 0; t < M; ++t) curve[t] = card[t] ? (double)sumc[t] / (double)card[t] : 0.0;
}

/* Sign of C(a) - C(b) for two thresholds with non-empty boundaries, exactly:
 * sumc(a)/card(a) vs sumc(b)/card(b)  <=>  sumc(a)*card(b) vs sumc(b)*card(a). */
static int compare_contrast(const uint64_t* card, const uint64_t* sumc, int32_t a, int32_t b) {
  unsigned __int128 l = (unsigned __int128)sumc[a] * card[b];
  unsigned __int128 r = (unsigned __int128)sumc[b] * card[a];
  return (l > r) - (l < r);
}

/* Local maxima of the contrast curve (Section 2.1, text after Eq. 4) and t0 (Eq. 4).
 *  - Only thresholds with a non-empty boundary (card > 0) take part.
 *  - A plateau is a maximal run of consecutive such thresholds with equal C.
 *  - A plateau is a local maximum when each of its two outside neighbours is
 *    either absent (card = 0 or outside [0, M[) or has a strictly smaller C;
 *    it is reported by its smallest threshold.
 *  - The maxima are ranked by C descending, then by t ascending; the first
 *    min(count, max_k) go to out_t, the rest of out_t is filled with -1.
 *  - *out_count is the total number of local maxima; *out_t0 is the smallest t
 *    reaching the largest C (Eq. 4), -1 when every boundary is empty. */
int oracle_thresholds(const uint64_t* card, const uint64_t* sumc, int32_t M, int32_t max_k,
                      int32_t* out_t, int32_t* out_count, int32_t* out_t0) {
  if (!card || !sumc || M < 1 || max_k < 0 || (max_k > 0 && !out_t) || !out_count || !out_t0) return ORACLE_ERR_ARG;
  int32_t* maxima = (int32_t*)malloc(sizeof(int32_t) * (size_t)M);
  if (!maxima) return ORACLE_ERR_ARG;
  int32_t count = 0;
  int32_t t = 0;
  while (t < M) {
    if (card[t] == 0) { ++t; continue; }
    int32_t a = t, b = t;
    while (b + 1 < M && card[b + 1] > 0 && compare_contrast(card, sumc, b + 1, a) == 0) ++b;
    int left_lower = (a == 0) || card[a - 1] == 0 || compare_contrast(card, sumc, a - 1, a) < 0;
    int right_lower = (b + 1 >= M) || card[b + 1] == 0 || compare_contrast(card, sumc, b + 1, b) < 0;
    if (left_lower && right_lower) maxima[count++] = a;
    t = b + 1;
  }
  /* rank: insertion sort by (C descending, t ascending) */
  for (int32_t i = 1; i < count; ++i) {
    int32_t v = maxima[i];
    int32_t j = i - 1;
    while (j >= 0) {
      int c = compare_contrast(card, sumc, maxima[j], v);
      if (c < 0 || (c == 0 && maxima[j] > v)) {
        maxima[j + 1] = maxima[j];
        --j;
      } else {
        break;
      }
    }
    maxima[j + 1] = v;
  }
  for (int32_t i = 0; i < max_k; ++i) out_t[i] = i < count ? maxima[i] : -1;
  *out_count = count;
  /* Eq. 4: the first threshold reaching the largest contrast */
  int32_t t0 = -1;
  for (int32_t u = 0; u < M; ++u)
    if (card[u] > 0 && (t0 < 0 || compare_contrast(card, sumc, u, t0) > 0)) t0 = u;
  *out_t0 = t0;
  free(maxima);
  return ORACLE_OK;
}
