/*
 * xc_oracle.c -- plain, slow, obviously-correct CPU oracle for the X-engine.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file; only the tests, the smoke check and the bench's CPU
 * baseline leg do.  It shares no source, header or build step with the CUDA
 * path (the seeded input generators are the only thing both sides use).
 *
 * What it computes (Clark, La Plante & Greenhill, "Accelerating Radio
 * Astronomy Cross-Correlation with GPUs"):
 *
 *   Sec. 2.1, Eq. (outer): for every frequency channel f the correlation
 *   matrix is the time-integrated sum of self outer products of the
 *   station signal vector,   S_f = sum_{t<I} X_t(f) (x) X_t(f).
 *   Sec. 2.1 (dual polarisation): each station contributes two
 *   polarisations, so the vector has length N*P; only the lower triangle of
 *   station pairs (N(N+1)/2 baselines, autocorrelations included) is kept.
 *   Sec. 4.1: input ordering has station fastest, then frequency, then time;
 *   each sample holds the polarisations of one station as complex numbers.
 *
 * Readings taken where the paper is silent or garbled:
 *   - Conjugation: V_ab = sum_t x_a(t) * conj(x_b(t)) (row index a is not
 *     conjugated).  Eq. (XF) prints both a star and a dagger, Eq. (outer) none.
 *   - Triangle and order: baseline k(s1,s2) = s1(s1+1)/2 + s2 with s2 <= s1
 *     (row >= column, the lower triangle of Sec. 4.2's block map); the four
 *     polarisation products of one baseline are stored as p1*P + p2, each
 *     as {re, im}.  Diagonal baselines keep all P*P products.
 *   - 8-bit input (Sec. 5) is integrated as raw integers, without the
 *     texture unit's normalisation; accumulation here is int64.
 *   - Float input is accumulated in FP64.  Complex gains g (one per
 *     station and polarisation) are applied to the voltages before
 *     correlating: y = g*x.
 *
 * Adjoint (not in the paper; the differentiable form of the engine): for a
 * real loss L of the stored visibilities, with grad_out_ab = dL/dReV_ab +
 * i dL/dImV_ab scattered into a dense matrix G (zero off the stored set) and
 * H = G + G^H:  grad_y = H y,  grad_x = conj(g) grad_y,
 * grad_g = sum_{f,t} conj(x) grad_y.
 *
 * F-engine (Sec. 2, the FX correlator): each station's signal is Fourier
 * transformed in blocks of F consecutive complex samples, giving F channels
 * per block,  X_t(f) = sum_{m<F} x(t F + m) exp(-2 pi i f m / F), and the
 * corner turn reorders the result from station-major to the X-engine's order
 * (station fastest, then channel, then block; Sec. 4.1).  Readings: the
 * transform carries a caller-given real factor `scale` (the paper leaves the
 * normalisation open); channel f is the f-th DFT bin (DC first), not
 * re-centred.  The optional polyphase front end (not in the paper; the usual
 * F-engine filter) weights ntaps consecutive blocks with caller-given taps
 * h[p][m] and sums them before the DFT:
 *   y_t(m) = sum_{p<ntaps} h[p][m] x((t + p) F + m),   t < T - ntaps + 1.
 *
 * Every function follows the definition with plain loops in the order
 * channel -> baseline -> polarisation pair -> time; OpenMP only splits the
 * independent channels (blocks for the F-engine) across threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Sec. 4.2 / lower triangle: packed index of station pair (s1 >= s2). */
int64_t xco_baseline_index(int64_t s1, int64_t s2) { return s1 * (s1 + 1) / 2 + s2; }

int64_t xco_num_baselines(int64_t nstation) { return nstation * (nstation + 1) / 2; }

int xco_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void xco_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Offset (in scalars) of the real part of x[t][f][s][p] in [T][F][N][P][2]. */
static inline int64_t in_off(int64_t t, int64_t f, int64_t s, int64_t p, int64_t F, int64_t N,
                             int64_t P) {
  return ((((t * F + f) * N + s) * P + p) * 2);
}

/*
 * Integer X-engine, Eq. (outer) with 8-bit two's-complement input.
 *   in   : int8  [T][F][N][P][2]   (re, im)
 *   chans: list of nchans channel indices to compute (NULL = all F, in order)
 *   out  : int64 [nchans][N(N+1)/2][P*P][2]
 * Returns 0, or -1 on a bad argument.
 */
int xco_correlate_i8(const int8_t* in, int N, int P, int F, int T, const int32_t* chans,
                     int nchans, int64_t* out) {
  if (!in || !out || N <= 0 || P <= 0 || F <= 0 || T < 0) return -1;
  if (!chans) nchans = F;
  const int64_t nb = xco_num_baselines(N);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int ci = 0; ci < nchans; ++ci) {
    const int64_t f = chans ? chans[ci] : ci;
    if (f < 0 || f >= F) {
      bad = 1;
      continue;
    }
    for (int64_t s1 = 0; s1 < N; ++s1) {
      for (int64_t s2 = 0; s2 <= s1; ++s2) {
        const int64_t k = xco_baseline_index(s1, s2);
        for (int64_t p1 = 0; p1 < P; ++p1) {
          for (int64_t p2 = 0; p2 < P; ++p2) {
            int64_t re = 0, im = 0;
            for (int64_t t = 0; t < T; ++t) {
              const int8_t* a = in + in_off(t, f, s1, p1, F, N, P);
              const int8_t* b = in + in_off(t, f, s2, p2, F, N, P);
              const int64_t ar = a[0], ai = a[1], br = b[0], bi = b[1];
              /* a * conj(b) */
              re += ar * br + ai * bi;
              im += ai * br - ar * bi;
            }
            int64_t* o = out + (((int64_t)ci * nb + k) * P * P + p1 * P + p2) * 2;
            o[0] = re;
            o[1] = im;
          }
        }
      }
    }
  }
  return bad ? -1 : 0;
}

/*
 * Float X-engine in FP64, Eq. (outer), with optional per-(station, pol)
 * complex gains applied to the voltages first (y = g x).
 *   in   : double [T][F][N][P][2]
 *   gains: double [N][P][2] or NULL (unit gains)
 *   out  : double [nchans][N(N+1)/2][P*P][2]
 */
int xco_correlate_f64(const double* in, const double* gains, int N, int P, int F, int T,
                      const int32_t* chans, int nchans, double* out) {
  if (!in || !out || N <= 0 || P <= 0 || F <= 0 || T < 0) return -1;
  if (!chans) nchans = F;
  const int64_t nb = xco_num_baselines(N);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int ci = 0; ci < nchans; ++ci) {
    const int64_t f = chans ? chans[ci] : ci;
    if (f < 0 || f >= F) {
      bad = 1;
      continue;
    }
    for (int64_t s1 = 0; s1 < N; ++s1) {
      for (int64_t s2 = 0; s2 <= s1; ++s2) {
        const int64_t k = xco_baseline_index(s1, s2);
        for (int64_t p1 = 0; p1 < P; ++p1) {
          for (int64_t p2 = 0; p2 < P; ++p2) {
            double gar = 1.0, gai = 0.0, gbr = 1.0, gbi = 0.0;
            if (gains) {
              gar = gains[(s1 * P + p1) * 2];
              gai = gains[(s1 * P + p1) * 2 + 1];
              gbr = gains[(s2 * P + p2) * 2];
              gbi = gains[(s2 * P + p2) * 2 + 1];
            }
            double re = 0.0, im = 0.0;
            for (int64_t t = 0; t < T; ++t) {
              const double* a = in + in_off(t, f, s1, p1, F, N, P);
              const double* b = in + in_off(t, f, s2, p2, F, N, P);
              /* y = g x */
              const double ar = gar * a[0] - gai * a[1], ai = gar * a[1] + gai * a[0];
              const double br = gbr * b[0] - gbi * b[1], bi = gbr * b[1] + gbi * b[0];
              re += ar * br + ai * bi;
              im += ai * br - ar * bi;
            }
            double* o = out + (((int64_t)ci * nb + k) * P * P + p1 * P + p2) * 2;
            o[0] = re;
            o[1] = im;
          }
        }
      }
    }
  }
  return bad ? -1 : 0;
}

/*
 * FP64 adjoint of xco_correlate_f64 (all channels).
 *   grad_out: double [F][N(N+1)/2][P*P][2], dL/dReV + i dL/dImV per stored entry
 *   grad_in : double [T][F][N][P][2]   (written)
 *   grad_g  : double [N][P][2]         (written; may be NULL)
 * With n = N*P inputs per channel, G[a][b] = grad_out entry of (a, b) when
 * station(a) >= station(b), else 0; H = G + G^H; for every t:
 *   y = g x_t,  grad_y = H y,  grad_x_t = conj(g) grad_y,
 *   grad_g += conj(x_t) grad_y.
 */
int xco_backward_f64(const double* in, const double* gains, const double* grad_out, int N, int P,
                     int F, int T, double* grad_in, double* grad_g) {
  if (!in || !grad_out || !grad_in || N <= 0 || P <= 0 || F <= 0 || T < 0) return -1;
  const int64_t n = (int64_t)N * P;
  const int64_t nb = xco_num_baselines(N);
  double* gg_all = (double*)calloc((size_t)F * n * 2, sizeof(double));
  if (!gg_all) return -1;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int f = 0; f < F; ++f) {
    double* H = (double*)calloc((size_t)n * n * 2, sizeof(double)); /* H[a][b] re, im */
    double* y = (double*)malloc((size_t)n * 2 * sizeof(double));
    if (!H || !y) {
      bad = 1;
      free(H);
      free(y);
      continue;
    }
    /* H = G + G^H, G from the stored lower triangle. */
    for (int64_t s1 = 0; s1 < N; ++s1) {
      for (int64_t s2 = 0; s2 <= s1; ++s2) {
        const int64_t k = xco_baseline_index(s1, s2);
        for (int64_t p1 = 0; p1 < P; ++p1) {
          for (int64_t p2 = 0; p2 < P; ++p2) {
            const double* go = grad_out + (((int64_t)f * nb + k) * P * P + p1 * P + p2) * 2;
            const int64_t a = s1 * P + p1, b = s2 * P + p2;
            /* G[a][b] */
            H[(a * n + b) * 2] += go[0];
            H[(a * n + b) * 2 + 1] += go[1];
            /* (G^H)[b][a] = conj(G[a][b]) */
            H[(b * n + a) * 2] += go[0];
            H[(b * n + a) * 2 + 1] -= go[1];
          }
        }
      }
    }
    for (int64_t t = 0; t < T; ++t) {
      for (int64_t a = 0; a < n; ++a) {
        const double* x = in + in_off(t, f, a / P, a % P, F, N, P);
        double gr = 1.0, gi = 0.0;
        if (gains) {
          gr = gains[a * 2];
          gi = gains[a * 2 + 1];
        }
        y[a * 2] = gr * x[0] - gi * x[1];
        y[a * 2 + 1] = gr * x[1] + gi * x[0];
      }
      for (int64_t a = 0; a < n; ++a) {
        double gyr = 0.0, gyi = 0.0; /* (H y)_a */
        for (int64_t b = 0; b < n; ++b) {
          const double hr = H[(a * n + b) * 2], hi = H[(a * n + b) * 2 + 1];
          gyr += hr * y[b * 2] - hi * y[b * 2 + 1];
          gyi += hr * y[b * 2 + 1] + hi * y[b * 2];
        }
        double gr = 1.0, gi = 0.0;
        if (gains) {
          gr = gains[a * 2];
          gi = gains[a * 2 + 1];
        }
        double* gx = grad_in + in_off(t, f, a / P, a % P, F, N, P);
        /* conj(g) * grad_y */
        gx[0] = gr * gyr + gi * gyi;
        gx[1] = gr * gyi - gi * gyr;
        /* conj(x) * grad_y, summed over t (per channel, reduced below) */
        const double* x = in + in_off(t, f, a / P, a % P, F, N, P);
        gg_all[((int64_t)f * n + a) * 2] += x[0] * gyr + x[1] * gyi;
        gg_all[((int64_t)f * n + a) * 2 + 1] += x[0] * gyi - x[1] * gyr;
      }
    }
    free(H);
    free(y);
  }
  if (grad_g) {
    memset(grad_g, 0, (size_t)n * 2 * sizeof(double));
    for (int f = 0; f < F; ++f)
      for (int64_t a = 0; a < n; ++a) {
        grad_g[a * 2] += gg_all[((int64_t)f * n + a) * 2];
        grad_g[a * 2 + 1] += gg_all[((int64_t)f * n + a) * 2 + 1];
      }
  }
  free(gg_all);
  return bad ? -1 : 0;
}

/*
 * F-engine, Sec. 2: the DFT definition over each block of F samples of each
 * station and polarisation, written in the corner-turned order.
 *   in  [N][P][T*F][2]  (station-major streams)
 *   out [T][F][N][P][2] when sel is NULL, else [nsel][N][P][2] for the
 *       (block, channel) pairs sel[2 i], sel[2 i + 1].
 * The phase index f*m is reduced mod F before the cosine and sine, so every
 * twiddle is one of the F exact roots of unity.
 */
int xco_channelize_f64(const double* in, int N, int P, int F, int T, double scale,
                       const int32_t* sel, int nsel, double* out) {
  if (N <= 0 || P <= 0 || F <= 0 || T <= 0 || (sel && nsel <= 0)) return -1;
  const int64_t n = (int64_t)N * P;
  const int64_t nout = sel ? nsel : (int64_t)T * F;
  double* wr = (double*)malloc((size_t)F * sizeof(double));
  double* wi = (double*)malloc((size_t)F * sizeof(double));
  if (!wr || !wi) {
    free(wr);
    free(wi);
    return -1;
  }
  const double two_pi = 6.283185307179586476925286766559;
  for (int j = 0; j < F; ++j) {
    wr[j] = cos(two_pi * (double)j / (double)F);
    wi[j] = -sin(two_pi * (double)j / (double)F);
  }
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int64_t o = 0; o < nout; ++o) {
    const int64_t t = sel ? sel[2 * o] : o / F;
    const int64_t f = sel ? sel[2 * o + 1] : o % F;
    if (t < 0 || t >= T || f < 0 || f >= F) {
      bad = 1;
      continue;
    }
    for (int64_t a = 0; a < n; ++a) {
      const double* x = in + (a * T * F + t * F) * 2;
      double re = 0.0, im = 0.0;
      for (int64_t m = 0; m < F; ++m) {
        const int64_t j = (f * m) % F;
        re += x[2 * m] * wr[j] - x[2 * m + 1] * wi[j];
        im += x[2 * m] * wi[j] + x[2 * m + 1] * wr[j];
      }
      out[(o * n + a) * 2] = scale * re;
      out[(o * n + a) * 2 + 1] = scale * im;
    }
  }
  free(wr);
  free(wi);
  return bad ? -1 : 0;
}

/*
 * Polyphase F-engine: the DFT definition applied to the tap-weighted sum of
 * ntaps consecutive blocks, y_t(m) = sum_p h[p F + m] x((t + p) F + m), for
 * the T - ntaps + 1 output blocks; h is [ntaps][F] real.  Same layouts as
 * xco_channelize_f64, out [T - ntaps + 1][F][N][P][2].
 */
int xco_channelize_pfb_f64(const double* in, int N, int P, int F, int T, const double* h,
                           int ntaps, double scale, double* out) {
  if (N <= 0 || P <= 0 || F <= 0 || ntaps <= 0 || T < ntaps || !h) return -1;
  const int64_t n = (int64_t)N * P;
  const int64_t Tout = (int64_t)T - ntaps + 1;
  double* wr = (double*)malloc((size_t)F * sizeof(double));
  double* wi = (double*)malloc((size_t)F * sizeof(double));
  if (!wr || !wi) {
    free(wr);
    free(wi);
    return -1;
  }
  const double two_pi = 6.283185307179586476925286766559;
  for (int j = 0; j < F; ++j) {
    wr[j] = cos(two_pi * (double)j / (double)F);
    wi[j] = -sin(two_pi * (double)j / (double)F);
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t o = 0; o < Tout * F; ++o) {
    const int64_t t = o / F, f = o % F;
    for (int64_t a = 0; a < n; ++a) {
      double re = 0.0, im = 0.0;
      for (int64_t m = 0; m < F; ++m) {
        double yr = 0.0, yi = 0.0;
        for (int p = 0; p < ntaps; ++p) {
          const double* x = in + (a * T * F + (t + p) * F + m) * 2;
          yr += h[(int64_t)p * F + m] * x[0];
          yi += h[(int64_t)p * F + m] * x[1];
        }
        const int64_t j = (f * m) % F;
        re += yr * wr[j] - yi * wi[j];
        im += yr * wi[j] + yi * wr[j];
      }
      out[(o * n + a) * 2] = scale * re;
      out[(o * n + a) * 2 + 1] = scale * im;
    }
  }
  free(wr);
  free(wi);
  return 0;
}
