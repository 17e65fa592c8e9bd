/*
 * DDHF oracle: a plain, slow, single-threaded restatement in FP64 of the
 * per-pixel frequency-analysis pipeline of "Real-Time Drone Detection in Event
 * Cameras via Per-Pixel Frequency Analysis" (arXiv 2603.08386).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library. The CUDA library never calls it
 * and shares no code, header, table or constant with it.
 *
 * Each function follows the definition it cites, step by step, with no
 * blocking, fusion or reordering beyond what that definition states. Where the
 * paper is silent, the reading taken is stated at the function.
 *
 * Build: cc -O2 -std=c11 -ffp-contract=off -fPIC -shared (contraction of
 * a*b+c into one FMA is switched off so that the FP32 restatement of the
 * comb score rounds every operation on its own, on x86-64 and on aarch64).
 *
 * Conventions shared with the pins in tests/:
 *   events  (x, y, t_us, p) with p in {-1, +1} (or {0, 1}, 0 meaning -1),
 *   window  [t0, t0 + window_us), tau = t - t0 in microseconds,
 *   grid    a_j = a0 + j*da in units of 1/denom cycles per microsecond
 *           (Hz grid: a_j in mHz, denom = 1e9; mode grid: a_j = k, denom =
 *           window_us), so the phase of event k at bin j is the exact integer
 *           residue r = (a_j * tau_k) mod denom, i.e. r/denom cycles.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Windowing, validation and stable binning into a per-pixel list.           */
/* Sec. 3.1 (event tuple), Sec. 3.5 "Event processing": events of a window   */
/* are sorted by pixel index and pixels with fewer than n_min events are     */
/* dropped. Reading: the sort is stable (input order kept within a pixel),   */
/* the key is y*W + x, an event is kept iff t0 <= t < t0+window_us,          */
/* 0 <= x < W, 0 <= y < H and p is a valid polarity.                         */
/* Written as a counting sort: count per key, prefix sum, then place events  */
/* in input order, which is stable by construction.                          */
/* Returns the number of kept events; *n_dropped gets the others.            */
/* ------------------------------------------------------------------------ */
int64_t oracle_bin_events(int32_t W, int32_t H, int64_t n, const int16_t *x,
                          const int16_t *y, const int64_t *t, const int8_t *p,
                          int64_t t0, int64_t window_us, int32_t polarity_01,
                          int64_t *counts,  /* [W*H]   out */
                          int64_t *offsets, /* [W*H+1] out */
                          int64_t *tau,     /* [n]     out, CSR order */
                          int8_t *pol,      /* [n]     out, CSR order, +-1 */
                          int64_t *n_dropped) {
  int64_t npx = (int64_t)W * (int64_t)H;
  int64_t kept = 0;
  for (int64_t k = 0; k < npx; ++k) counts[k] = 0;
  for (int64_t i = 0; i < n; ++i) {
    int valid_p = polarity_01 ? (p[i] == 0 || p[i] == 1) : (p[i] == -1 || p[i] == 1);
    if (!valid_p) continue;
    if (x[i] < 0 || x[i] >= W || y[i] < 0 || y[i] >= H) continue;
    if (t[i] < t0 || t[i] - t0 >= window_us) continue;
    counts[(int64_t)y[i] * W + x[i]] += 1;
    kept += 1;
  }
  offsets[0] = 0;
  for (int64_t k = 0; k < npx; ++k) offsets[k + 1] = offsets[k] + counts[k];
  int64_t *cursor = (int64_t *)malloc(sizeof(int64_t) * (size_t)(npx > 0 ? npx : 1));
  for (int64_t k = 0; k < npx; ++k) cursor[k] = offsets[k];
  for (int64_t i = 0; i < n; ++i) {
    int valid_p = polarity_01 ? (p[i] == 0 || p[i] == 1) : (p[i] == -1 || p[i] == 1);
    if (!valid_p) continue;
    if (x[i] < 0 || x[i] >= W || y[i] < 0 || y[i] >= H) continue;
    if (t[i] < t0 || t[i] - t0 >= window_us) continue;
    int64_t key = (int64_t)y[i] * W + x[i];
    int64_t at = cursor[key]++;
    tau[at] = t[i] - t0;
    pol[at] = polarity_01 ? (p[i] == 1 ? 1 : -1) : p[i];
  }
  free(cursor);
  *n_dropped = n - kept;
  return kept;
}

/* Exact residue (a * tau) mod denom for a >= 0, tau >= 0, denom > 0. */
static int64_t phase_residue(int64_t a, int64_t tau, int64_t denom) {
  unsigned __int128 prod = (unsigned __int128)(uint64_t)a * (unsigned __int128)(uint64_t)tau;
  return (int64_t)(prod % (unsigned __int128)(uint64_t)denom);
}

/* ------------------------------------------------------------------------ */
/* Non-uniform DFT and power, Sec. 3.3 Eq. 6 and P_k = |F_k|^2.              */
/* F_j = sum_k p_k exp(-2 pi i f_j tau_k), f_j tau_k = r_jk / denom cycles   */
/* with r_jk = (a_j tau_k) mod denom exact. The paper writes exp(+i k t)     */
/* over timestamps mapped to [-pi, pi); that is the conjugate of the same sum */
/* times a phase common to all events, so the power is the same.             */
/* Output: P[j] for j = 0..n_bins-1, and optionally F (re, im interleaved).   */
/* ------------------------------------------------------------------------ */
void oracle_ndft(int64_t n, const int64_t *tau, const int8_t *pol, int64_t a0,
                 int64_t da, int64_t denom, int32_t n_bins, double *P,
                 double *F /* nullable, [2*n_bins] */) {
  for (int32_t j = 0; j < n_bins; ++j) {
    int64_t a = a0 + (int64_t)j * da;
    double re = 0.0, im = 0.0;
    for (int64_t k = 0; k < n; ++k) {
      int64_t r = phase_residue(a, tau[k], denom);
      double theta = 2.0 * M_PI * ((double)r / (double)denom);
      re += (double)pol[k] * cos(theta);
      im -= (double)pol[k] * sin(theta);
    }
    P[j] = re * re + im * im;
    if (F) {
      F[2 * j] = re;
      F[2 * j + 1] = im;
    }
  }
}

/* The same sum in single precision, for the FP32 CPU baseline of the      */
/* benchmark (not a reference: the parity tests use the FP64 version): the */
/* exact integer residue, its phase rounded once to float, float sin/cos   */
/* and float accumulation in event order.                                   */
void oracle_ndft_f32(int64_t n, const int64_t *tau, const int8_t *pol, int64_t a0,
                     int64_t da, int64_t denom, int32_t n_bins, float *P) {
  for (int32_t j = 0; j < n_bins; ++j) {
    int64_t a = a0 + (int64_t)j * da;
    float re = 0.0f, im = 0.0f;
    for (int64_t k = 0; k < n; ++k) {
      int64_t r = phase_residue(a, tau[k], denom);
      float theta = (float)(2.0 * M_PI * ((double)r / (double)denom));
      re += (float)pol[k] * cosf(theta);
      im -= (float)pol[k] * sinf(theta);
    }
    P[j] = re * re + im * im;
  }
}

/* Same sum at arbitrary real frequencies f (Hz) with tau in microseconds,   */
/* evaluated in FP64 with the frequency split as f = fi/1000 + fr where fi   */
/* is an integer number of mHz (exact residue) and fr the remainder; used by */
/* the soft comb of the differentiation pattern. Also returns                */
/* D = dF/df = sum_k (-2 pi i tau_k 1e-6) p_k exp(-2 pi i f tau_k).           */
/* tau_c is subtracted from tau before use (window-centre reference).        */
void oracle_ndft_at(int64_t n, const int64_t *tau, const int8_t *pol,
                    double tau_c, int32_t n_f, const double *f_hz,
                    double *F /* [2*n_f] */, double *D /* [2*n_f], nullable */) {
  for (int32_t j = 0; j < n_f; ++j) {
    double f = f_hz[j];
    double fi_mhz = floor(f * 1000.0);
    double fr = f - fi_mhz / 1000.0; /* Hz, in [0, 1e-3) up to rounding */
    int64_t a = (int64_t)fi_mhz;
    double re = 0.0, im = 0.0, dre = 0.0, dim = 0.0;
    for (int64_t k = 0; k < n; ++k) {
      /* cycles = f * (tau - tau_c) * 1e-6, split into the exact integer part
         a*tau mod 1e9 (in 1e-9 cycles) and the small remainders. */
      int64_t am = a % 1000000000LL; /* residue of any sign, into [0, 1e9) */
      if (am < 0) am += 1000000000LL;
      int64_t r = phase_residue(am, tau[k], 1000000000LL);
      double cyc = (double)r * 1e-9 + fr * (double)tau[k] * 1e-6 - f * tau_c * 1e-6;
      double theta = 2.0 * M_PI * cyc;
      double c = cos(theta), s = sin(theta);
      double pk = (double)pol[k];
      re += pk * c;
      im -= pk * s;
      /* d/df of exp(-i 2 pi f (tau-tau_c)1e-6) = -i 2 pi (tau-tau_c)1e-6 exp(.) */
      double w = 2.0 * M_PI * ((double)tau[k] - tau_c) * 1e-6;
      /* -i w (c - i s) = -w s - i w c */
      dre += pk * (-w * s);
      dim += pk * (-w * c);
    }
    F[2 * j] = re;
    F[2 * j + 1] = im;
    if (D) {
      D[2 * j] = dre;
      D[2 * j + 1] = dim;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Spectral flatness, Sec. 3.4 Eq. 7: geometric mean over arithmetic mean of */
/* the N evaluated bins. Readings: the N bins are the grid j = 0..N-1, a bin */
/* with P = 0 enters the log as ln(1e-30), and a spectrum whose arithmetic   */
/* mean is 0 is called flat (SF = 1). Returns ln SF.                         */
/* ------------------------------------------------------------------------ */
double oracle_log_sf(int32_t N, const double *P) {
  double slog = 0.0, sum = 0.0;
  for (int32_t j = 0; j < N; ++j) {
    double v = P[j] > 1e-30 ? P[j] : 1e-30;
    slog += log(v);
    sum += P[j];
  }
  if (!(sum > 0.0)) return 0.0;
  return slog / (double)N - log(sum / (double)N);
}

static int cmp_double(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return (x > y) - (x < y);
}
static int cmp_float(const void *a, const void *b) {
  float x = *(const float *)a, y = *(const float *)b;
  return (x > y) - (x < y);
}

/* Number of harmonics m = 1..M whose window [m w - d, m w + d] lies inside   */
/* 0..N-1 (Eq. 8, M_valid). For w >= max(1, d) the in-band windows form a     */
/* prefix m = 1..M_valid. Returns 0 for candidates outside that range.       */
static int32_t comb_m_valid(int32_t N, int32_t w, int32_t M, int32_t d) {
  int32_t lo = d > 1 ? d : 1;
  if (w < lo) return 0;
  int32_t mv = 0;
  for (int32_t m = 1; m <= M; ++m) {
    if ((int64_t)m * w + d <= N - 1) mv = m;
    else break;
  }
  return mv;
}

/* ------------------------------------------------------------------------ */
/* Median-normalised harmonic comb, Sec. 3.4 Eq. 8-11, in FP64.              */
/* For each candidate fundamental w (integer bin, w >= max(1,d), M_valid(w)  */
/* >= h_min):                                                                */
/*   N(w)  = (1/M_valid) sum_{m=1..M_valid} max_{|k - m w| <= d} P_k   Eq. 8 */
/*   H(w)  = union of those windows; B(w) = median of P over the rest  Eq. 9 */
/*   SNR(w)= N(w) / B(w)                                              Eq. 10 */
/* Readings: median of an even count is the mean of the two middle values; */
/* B <= 0 gives SNR = +inf if N > 0 else 0; a candidate whose complement is  */
/* empty is skipped; the best SNR is the maximum over w and its first        */
/* attaining w is the dominant bin (Eq. 11 compares it with tau_comb).       */
/* Returns the best SNR (0 and *best_w = -1 when no candidate is valid).     */
/* ------------------------------------------------------------------------ */
double oracle_comb(int32_t N, const double *P, int32_t M, int32_t d, int32_t h_min,
                   int32_t *best_w) {
  double best = 0.0;
  int32_t bw = -1;
  unsigned char *in_h = (unsigned char *)malloc((size_t)N);
  double *rest = (double *)malloc(sizeof(double) * (size_t)N);
  for (int32_t w = 1; w < N; ++w) {
    int32_t mv = comb_m_valid(N, w, M, d);
    if (mv < 1 || mv < h_min) continue;
    double s = 0.0;
    memset(in_h, 0, (size_t)N);
    for (int32_t m = 1; m <= mv; ++m) {
      double mx = -INFINITY;
      for (int32_t k = m * w - d; k <= m * w + d; ++k) {
        if (P[k] > mx) mx = P[k];
        in_h[k] = 1;
      }
      s += mx;
    }
    double nw = s / (double)mv;
    int32_t c = 0;
    for (int32_t k = 0; k < N; ++k)
      if (!in_h[k]) rest[c++] = P[k];
    if (c == 0) continue;
    qsort(rest, (size_t)c, sizeof(double), cmp_double);
    double b = (c % 2) ? rest[(c - 1) / 2] : 0.5 * (rest[c / 2 - 1] + rest[c / 2]);
    double snr = b > 0.0 ? nw / b : (nw > 0.0 ? INFINITY : 0.0);
    if (bw < 0 || snr > best) {
      best = snr;
      bw = w;
    }
  }
  free(in_h);
  free(rest);
  *best_w = bw;
  return bw < 0 ? 0.0 : best;
}

/* The same Eq. 8-11 in FP32 with every operation rounded on its own, in this */
/* order: s = 0; s = s + max_m for m = 1..M_valid; N = s / (float)M_valid;    */
/* even-count median = (a + b) * 0.5f; SNR = N / B. This fixes one FP32       */
/* evaluation of the definition so that a GPU spectrum can be scored on the   */
/* CPU and on the GPU with the same bits.                                     */
float oracle_comb_f32(int32_t N, const float *P, int32_t M, int32_t d, int32_t h_min,
                      int32_t *best_w) {
  float best = 0.0f;
  int32_t bw = -1;
  unsigned char *in_h = (unsigned char *)malloc((size_t)N);
  float *rest = (float *)malloc(sizeof(float) * (size_t)N);
  for (int32_t w = 1; w < N; ++w) {
    int32_t mv = comb_m_valid(N, w, M, d);
    if (mv < 1 || mv < h_min) continue;
    float s = 0.0f;
    memset(in_h, 0, (size_t)N);
    for (int32_t m = 1; m <= mv; ++m) {
      float mx = -INFINITY;
      for (int32_t k = m * w - d; k <= m * w + d; ++k) {
        if (P[k] > mx) mx = P[k];
        in_h[k] = 1;
      }
      s = s + mx;
    }
    float nw = s / (float)mv;
    int32_t c = 0;
    for (int32_t k = 0; k < N; ++k)
      if (!in_h[k]) rest[c++] = P[k];
    if (c == 0) continue;
    qsort(rest, (size_t)c, sizeof(float), cmp_float);
    float b;
    if (c % 2) {
      b = rest[(c - 1) / 2];
    } else {
      float sum2 = rest[c / 2 - 1] + rest[c / 2];
      b = sum2 * 0.5f;
    }
    float snr = b > 0.0f ? nw / b : (nw > 0.0f ? INFINITY : 0.0f);
    if (bw < 0 || snr > best) {
      best = snr;
      bw = w;
    }
  }
  free(in_h);
  free(rest);
  *best_w = bw;
  return bw < 0 ? 0.0f : best;
}

/* ------------------------------------------------------------------------ */
/* 8-connected component labelling of the rotor mask, Sec. 3.5 "Segmentation */
/* mask processing". Breadth-first flood fill started from each unlabelled   */
/* mask pixel in raster order, so every component is labelled with the      */
/* smallest linear index y*W + x of its pixels. Background gets -1.          */
/* Returns the number of components.                                          */
/* ------------------------------------------------------------------------ */
int32_t oracle_ccl8(int32_t W, int32_t H, const uint8_t *mask, int32_t *labels) {
  int64_t npx = (int64_t)W * H;
  int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)(npx > 0 ? npx : 1));
  int32_t ncomp = 0;
  for (int64_t i = 0; i < npx; ++i) labels[i] = -1;
  for (int64_t s = 0; s < npx; ++s) {
    if (!mask[s] || labels[s] >= 0) continue;
    int64_t head = 0, tail = 0;
    queue[tail++] = s;
    labels[s] = (int32_t)s;
    while (head < tail) {
      int64_t q = queue[head++];
      int32_t qx = (int32_t)(q % W), qy = (int32_t)(q / W);
      for (int32_t dy = -1; dy <= 1; ++dy)
        for (int32_t dx = -1; dx <= 1; ++dx) {
          int32_t nx = qx + dx, ny = qy + dy;
          if (nx < 0 || nx >= W || ny < 0 || ny >= H) continue;
          int64_t nb = (int64_t)ny * W + nx;
          if (mask[nb] && labels[nb] < 0) {
            labels[nb] = (int32_t)s;
            queue[tail++] = nb;
          }
        }
    }
    ncomp += 1;
  }
  free(queue);
  return ncomp;
}

typedef struct {
  int64_t x0, y0, x1, y1, n;
} obox;

static int cmp_box(const void *a, const void *b) {
  const obox *p = (const obox *)a, *q = (const obox *)b;
  if (p->y0 != q->y0) return p->y0 < q->y0 ? -1 : 1;
  if (p->x0 != q->x0) return p->x0 < q->x0 ? -1 : 1;
  if (p->y1 != q->y1) return p->y1 < q->y1 ? -1 : 1;
  if (p->x1 != q->x1) return p->x1 < q->x1 ? -1 : 1;
  if (p->n != q->n) return p->n < q->n ? -1 : 1;
  return 0;
}

/* Eq. 12 test in FP64: dist(c1, c2) < alpha * max(w1, h1, w2, h2) with      */
/* c = ((x0+x1)/2, (y0+y1)/2) and w = x1-x0+1, h = y1-y0+1, squared and      */
/* doubled so the left side is an exact integer:                             */
/*   (2dx)^2 + (2dy)^2 < (2 alpha m)^2, with s = (2*alpha)*m, rhs = s*s.      */
static int eq12_close(const obox *a, const obox *b, double alpha) {
  int64_t dx2 = (a->x0 + a->x1) - (b->x0 + b->x1);
  int64_t dy2 = (a->y0 + a->y1) - (b->y0 + b->y1);
  int64_t m = a->x1 - a->x0 + 1;
  if (a->y1 - a->y0 + 1 > m) m = a->y1 - a->y0 + 1;
  if (b->x1 - b->x0 + 1 > m) m = b->x1 - b->x0 + 1;
  if (b->y1 - b->y0 + 1 > m) m = b->y1 - b->y0 + 1;
  double lhs = (double)(dx2 * dx2 + dy2 * dy2);
  double s = (2.0 * alpha) * (double)m;
  double rhs = s * s;
  return lhs < rhs;
}

static int64_t uf_find(int64_t *par, int64_t i) {
  while (par[i] != i) i = par[i];
  return i;
}

/* ------------------------------------------------------------------------ */
/* Bounding boxes, area filter and centroid merge, Sec. 3.5 and Eq. 12.      */
/* 1. one box per component (inclusive x0,y0,x1,y1) with its pixel count;   */
/* 2. drop boxes whose area (x1-x0+1)(y1-y0+1) < A_min;                      */
/* 3. repeat: join every pair of current boxes that satisfies Eq. 12, take   */
/*    the transitive groups, replace each group by its union box (counts     */
/*    summed), until no pair satisfies Eq. 12;                               */
/* 4. sort by (y0, x0, y1, x1, n).                                           */
/* Readings: area filter before merging; union box as the merged box.        */
/* Writes min(count, cap) boxes as int32 quintuples; returns the count.      */
/* ------------------------------------------------------------------------ */
int32_t oracle_boxes(int32_t W, int32_t H, const int32_t *labels, int32_t A_min,
                     double alpha, int32_t cap, int32_t *out) {
  int64_t npx = (int64_t)W * H;
  int64_t nb = 0;
  for (int64_t i = 0; i < npx; ++i)
    if (labels[i] == (int32_t)i) nb += 1;
  obox *bx = (obox *)malloc(sizeof(obox) * (size_t)(nb > 0 ? nb : 1));
  int64_t *slot = (int64_t *)malloc(sizeof(int64_t) * (size_t)(npx > 0 ? npx : 1));
  int64_t c = 0;
  for (int64_t i = 0; i < npx; ++i) {
    slot[i] = -1;
    if (labels[i] == (int32_t)i) {
      slot[i] = c;
      bx[c].x0 = bx[c].x1 = i % W;
      bx[c].y0 = bx[c].y1 = i / W;
      bx[c].n = 0;
      c += 1;
    }
  }
  for (int64_t i = 0; i < npx; ++i) {
    if (labels[i] < 0) continue;
    obox *b = &bx[slot[labels[i]]];
    int64_t xx = i % W, yy = i / W;
    if (xx < b->x0) b->x0 = xx;
    if (xx > b->x1) b->x1 = xx;
    if (yy < b->y0) b->y0 = yy;
    if (yy > b->y1) b->y1 = yy;
    b->n += 1;
  }
  free(slot);
  int64_t m = 0;
  for (int64_t i = 0; i < nb; ++i) {
    int64_t area = (bx[i].x1 - bx[i].x0 + 1) * (bx[i].y1 - bx[i].y0 + 1);
    if (area >= A_min) bx[m++] = bx[i];
  }
  int64_t *par = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
  obox *nxt = (obox *)malloc(sizeof(obox) * (size_t)(m > 0 ? m : 1));
  for (;;) {
    int any = 0;
    for (int64_t i = 0; i < m; ++i) par[i] = i;
    for (int64_t i = 0; i < m; ++i)
      for (int64_t j = i + 1; j < m; ++j)
        if (eq12_close(&bx[i], &bx[j], alpha)) {
          any = 1;
          int64_t ri = uf_find(par, i), rj = uf_find(par, j);
          if (ri != rj) par[ri > rj ? ri : rj] = ri < rj ? ri : rj;
        }
    if (!any) break;
    int64_t k = 0;
    for (int64_t i = 0; i < m; ++i) {
      if (uf_find(par, i) != i) continue;
      obox u = bx[i];
      u.n = 0;
      for (int64_t j = 0; j < m; ++j) {
        if (uf_find(par, j) != i) continue;
        if (bx[j].x0 < u.x0) u.x0 = bx[j].x0;
        if (bx[j].y0 < u.y0) u.y0 = bx[j].y0;
        if (bx[j].x1 > u.x1) u.x1 = bx[j].x1;
        if (bx[j].y1 > u.y1) u.y1 = bx[j].y1;
        u.n += bx[j].n;
      }
      nxt[k++] = u;
    }
    memcpy(bx, nxt, sizeof(obox) * (size_t)k);
    m = k;
  }
  qsort(bx, (size_t)m, sizeof(obox), cmp_box);
  for (int64_t i = 0; i < m && i < cap; ++i) {
    out[5 * i + 0] = (int32_t)bx[i].x0;
    out[5 * i + 1] = (int32_t)bx[i].y0;
    out[5 * i + 2] = (int32_t)bx[i].x1;
    out[5 * i + 3] = (int32_t)bx[i].y1;
    out[5 * i + 4] = (int32_t)bx[i].n;
  }
  free(par);
  free(nxt);
  free(bx);
  return (int32_t)m;
}

/* ------------------------------------------------------------------------ */
/* Per-pixel classification of one window, Sec. 3.5: for every active pixel  */
/* (count >= n_min, in pixel order) the NDFT power (Eq. 6), ln SF (Eq. 7),    */
/* and, when SF <= tau_sf, the comb score and dominant bin (Eq. 8-11); the    */
/* rotor mask bit is set when SF <= tau_sf and best SNR >= tau_comb.          */
/* snr = 0 and w = -1 for pixels rejected by SF. Mask is [W*H].               */
/* Returns the number of active pixels. pix_list restricts the work to the    */
/* listed pixels when n_list >= 0 (used for sampled parity at large sizes).   */
/* ------------------------------------------------------------------------ */
int64_t oracle_classify(int32_t W, int32_t H, const int64_t *offsets, const int64_t *tau,
                        const int8_t *pol, int64_t a0, int64_t da, int64_t denom,
                        int32_t n_bins, double tau_sf, double tau_comb, int32_t M,
                        int32_t d, int32_t h_min, int32_t n_min, int64_t n_list,
                        const int64_t *pix_list, int64_t *active, double *log_sf,
                        double *snr, int32_t *best_w, uint8_t *mask) {
  int64_t npx = (int64_t)W * H;
  double *P = (double *)malloc(sizeof(double) * (size_t)n_bins);
  double ln_tau_sf = log(tau_sf);
  int64_t na = 0;
  int64_t total = n_list >= 0 ? n_list : npx;
  if (mask && n_list < 0) memset(mask, 0, (size_t)npx);
  for (int64_t q = 0; q < total; ++q) {
    int64_t k = n_list >= 0 ? pix_list[q] : q;
    int64_t cnt = offsets[k + 1] - offsets[k];
    if (cnt < n_min) continue;
    oracle_ndft(cnt, tau + offsets[k], pol + offsets[k], a0, da, denom, n_bins, P, NULL);
    double lsf = oracle_log_sf(n_bins, P);
    double s = 0.0;
    int32_t w = -1;
    uint8_t bit = 0;
    if (lsf <= ln_tau_sf) {
      s = oracle_comb(n_bins, P, M, d, h_min, &w);
      bit = (w >= 0 && s >= tau_comb) ? 1 : 0;
    }
    if (active) active[na] = k;
    if (log_sf) log_sf[na] = lsf;
    if (snr) snr[na] = s;
    if (best_w) best_w[na] = w;
    if (mask) mask[k] = bit;
    na += 1;
  }
  free(P);
  return na;
}

/* ------------------------------------------------------------------------ */
/* Soft comb score (differentiation pattern; the paper has no soft score,   */
/* it is built on Eq. 6 and the comb idea of Eq. 8-10):                     */
/*   f_hq = h f0 + q delta,  h = 1..n_h, q = -Q..Q                           */
/*   G_hq = exp(-(q delta)^2 / (2 sigma_h^2)),  Z_h = sum_q G_hq             */
/*   S    = sum_h w_h (sum_q G_hq P(f_hq) / Z_h) / B                         */
/* with P(f) = |F(f)|^2 of Eq. 6 at real frequency f and B a given positive */
/* background (the median of the plain-grid spectrum, held constant).        */
/* Gradients, from dP/df = 2 Re(conj(F) dF/df):                              */
/*   dS/dw_h     = (sum_q G P / Z_h) / B                                     */
/*   dS/df0      = sum_h w_h h (sum_q G P' / Z_h) / B                        */
/*   dS/dsigma_h = w_h / (B sigma_h^3) [sum_q G P q^2d^2 / Z - (sum_q G P/Z) */
/*                 (sum_q G q^2 d^2 / Z)]                                    */
/*   dS/df_hq    = w_h G_hq P'(f_hq) / (Z_h B)   (written to dS_df, [n_h][2Q+1]) */
/* Returns S.                                                                */
/* ------------------------------------------------------------------------ */
double oracle_softcomb(int64_t n, const int64_t *tau, const int8_t *pol, double tau_c,
                       double f0, int32_t n_h, const double *w, const double *sigma,
                       double delta, int32_t Q, double B, double *dS_df0, double *dS_dw,
                       double *dS_dsigma, double *dS_df) {
  double S = 0.0, g0 = 0.0;
  int32_t nq = 2 * Q + 1;
  double *fq = (double *)malloc(sizeof(double) * (size_t)nq);
  double *F = (double *)malloc(sizeof(double) * 2 * (size_t)nq);
  double *D = (double *)malloc(sizeof(double) * 2 * (size_t)nq);
  for (int32_t h = 1; h <= n_h; ++h) {
    for (int32_t q = -Q; q <= Q; ++q) fq[q + Q] = (double)h * f0 + (double)q * delta;
    oracle_ndft_at(n, tau, pol, tau_c, nq, fq, F, D);
    double sg = sigma[h - 1];
    double Z = 0.0, A = 0.0, Ad = 0.0, C = 0.0, E = 0.0;
    for (int32_t q = -Q; q <= Q; ++q) {
      double qd = (double)q * delta;
      double G = exp(-(qd * qd) / (2.0 * sg * sg));
      double fr = F[2 * (q + Q)], fi = F[2 * (q + Q) + 1];
      double dr = D[2 * (q + Q)], di = D[2 * (q + Q) + 1];
      double P = fr * fr + fi * fi;
      double Pd = 2.0 * (fr * dr + fi * di);
      Z += G;
      A += G * P;
      Ad += G * Pd;
      C += G * P * qd * qd;
      E += G * qd * qd;
    }
    double wh = w[h - 1];
    S += wh * (A / Z) / B;
    if (dS_dw) dS_dw[h - 1] = (A / Z) / B;
    g0 += wh * (double)h * (Ad / Z) / B;
    if (dS_dsigma)
      dS_dsigma[h - 1] = wh / (B * sg * sg * sg) * (C / Z - (A / Z) * (E / Z));
    if (dS_df) {
      for (int32_t q = -Q; q <= Q; ++q) {
        double qd = (double)q * delta;
        double G = exp(-(qd * qd) / (2.0 * sg * sg));
        double fr = F[2 * (q + Q)], fi = F[2 * (q + Q) + 1];
        double dr = D[2 * (q + Q)], di = D[2 * (q + Q) + 1];
        dS_df[(h - 1) * nq + (q + Q)] = wh * G * 2.0 * (fr * dr + fi * di) / (Z * B);
      }
    }
  }
  if (dS_df0) *dS_df0 = g0;
  free(fq);
  free(F);
  free(D);
  return S;
}
