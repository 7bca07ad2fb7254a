/*
 * X-engine oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct CPU restatement of what the correlator's
 * X-engine computes (Niu et al., "The Design and Implementation of a
 * ROACH2+GPU based Correlator on the Tianlai Dish Array", arXiv:1904.07778).
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this library.  It shares no code, header, table or
 * helper with the CUDA path, and the CUDA path never calls it.
 *
 * What it computes (Sec. 2, System Design; Sec. 2.2, X-engine): for every
 * frequency channel c and every input pair j <= i, the integrated visibility
 *     V[c][i][j] = sum_t x_i(c,t) * conj(x_j(c,t))
 * over all spectra t, as exact int64 (the CMAC "multiply and accumulation"
 * process of Sec. 2; "integrated for some pre-specified duration", Sec. 2).
 * Storage: lower triangle incl. autos, baseline b(i,j) = i(i+1)/2 + j,
 * vis[c][b][0] = Re, vis[c][b][1] = Im.
 *
 * Input encodings (Sec. 2.1, F-engine, equaliser): a 4-bit complex sample is
 * one byte holding two 4-bit two's-complement numbers (real and imaginary).
 * Reading: the real part is the high nibble unless hi_is_real == 0.  Code 0x8
 * decodes to -8 (plain two's complement) although the equaliser never emits
 * it.  An 8-bit complex sample is two bytes (re, im) of int8; the value -128
 * is outside the symmetric [-127, 127] quantiser and is reported as an error.
 *
 * Layouts (sample order in the packed block):
 *   0 = [t][c][i]  -- the payload order of Sec. 2.3 (time, channel, input)
 *   1 = [t][i][c]  -- input-major, channel-minor spectra (needs a corner turn,
 *                     Sec. 2.1 "Transpose")
 *   2 = [c][i][t]  -- already corner-turned
 *
 * Parity status: every function here is pinned by tests under tests/ that
 * check it against hand-evaluated products, closed forms, invariants, the
 * FX == XF identity of Sec. 2 and the delay test of Sec. 3 (Eq. 5).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ERANGE (-4)
#define OR_ENOMEM (-2)

static size_t sample_offset(int layout, int N, int C, int T, int c, int i, int t) {
  (void)T;
  switch (layout) {
    case 0: return ((size_t)t * C + c) * N + i;
    case 1: return ((size_t)t * N + i) * C + c;
    default: return ((size_t)c * N + i) * T + t;
  }
}

static int nibble_value(int n) { return n >= 8 ? n - 16 : n; }

/* Decode sample (c, i, t).  Returns 0, or OR_ERANGE for an 8-bit -128. */
static int decode(const uint8_t* in, int layout, int bits, int hi_is_real, int N, int C, int T, int c,
                  int i, int t, int* re, int* im) {
  size_t s = sample_offset(layout, N, C, T, c, i, t);
  if (bits == 4) {
    int byte = in[s];
    int hi = nibble_value(byte >> 4), lo = nibble_value(byte & 15);
    *re = hi_is_real ? hi : lo;
    *im = hi_is_real ? lo : hi;
    return OR_OK;
  }
  int r = (int)(int8_t)in[2 * s], m = (int)(int8_t)in[2 * s + 1];
  *re = r;
  *im = m;
  return (r == -128 || m == -128) ? OR_ERANGE : OR_OK;
}

typedef struct {
  const uint8_t* in;
  int layout, bits, hi_is_real, N, C, T;
  const int* chans;
  int nchan;
  int64_t* vis;
  int stride, offset;
  int status;
} corr_job;

/* One channel: decode all of it, then the textbook triple loop, t innermost. */
static int correlate_channel(const corr_job* jb, int c, int64_t* out) {
  int N = jb->N, T = jb->T;
  int* re = (int*)malloc(sizeof(int) * (size_t)N * T);
  int* im = (int*)malloc(sizeof(int) * (size_t)N * T);
  if (!re || !im) {
    free(re);
    free(im);
    return OR_ENOMEM;
  }
  int status = OR_OK;
  for (int i = 0; i < N; ++i)
    for (int t = 0; t < T; ++t) {
      int st = decode(jb->in, jb->layout, jb->bits, jb->hi_is_real, N, jb->C, T, c, i, t,
                      &re[(size_t)i * T + t], &im[(size_t)i * T + t]);
      if (st != OR_OK) status = st;
    }
  for (int i = 0; i < N; ++i) {
    for (int j = 0; j <= i; ++j) {
      int64_t sre = 0, sim = 0;
      const int* ai = re + (size_t)i * T;
      const int* bi = im + (size_t)i * T;
      const int* aj = re + (size_t)j * T;
      const int* bj = im + (size_t)j * T;
      for (int t = 0; t < T; ++t) {
        /* (a_i + i b_i) * (a_j - i b_j) = (a_i a_j + b_i b_j) + i (b_i a_j - a_i b_j) */
        sre += (int64_t)ai[t] * aj[t] + (int64_t)bi[t] * bj[t];
        sim += (int64_t)bi[t] * aj[t] - (int64_t)ai[t] * bj[t];
      }
      size_t b = (size_t)i * (i + 1) / 2 + j;
      out[2 * b] += sre;
      out[2 * b + 1] += sim;
    }
  }
  free(re);
  free(im);
  return status;
}

static void* corr_worker(void* arg) {
  corr_job* jb = (corr_job*)arg;
  size_t nb = (size_t)jb->N * (jb->N + 1) / 2;
  for (int k = jb->offset; k < jb->nchan; k += jb->stride) {
    int c = jb->chans ? jb->chans[k] : k;
    int st = correlate_channel(jb, c, jb->vis + (size_t)k * nb * 2);
    if (st != OR_OK) jb->status = st;
  }
  return NULL;
}

/*
 * Accumulate (+=) visibilities of one packed block into vis.
 * chans: optional list of nchan channel indices (vis then has nchan rows, in
 * list order); NULL means all C channels.  nthreads <= 1 runs serially.
 * Returns OR_ERANGE if an 8-bit sample equals -128 (the sum is still formed).
 */
int oracle_correlate(const uint8_t* in, int layout, int bits, int hi_is_real, int N, int C, int T,
                     const int* chans, int nchan, int64_t* vis, int nthreads) {
  if (!in || !vis || N < 1 || C < 1 || T < 0 || (bits != 4 && bits != 8) || layout < 0 ||
      layout > 2)
    return OR_EINVAL;
  if (!chans) nchan = C;
  for (int k = 0; chans && k < nchan; ++k)
    if (chans[k] < 0 || chans[k] >= C) return OR_EINVAL;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > nchan) nthreads = nchan > 0 ? nchan : 1;
  corr_job* jobs = (corr_job*)calloc((size_t)nthreads, sizeof(corr_job));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !th) {
    free(jobs);
    free(th);
    return OR_ENOMEM;
  }
  for (int w = 0; w < nthreads; ++w) {
    corr_job jb = {in, layout, bits, hi_is_real, N, C, T, chans, nchan, vis, nthreads, w, OR_OK};
    jobs[w] = jb;
  }
  int status = OR_OK;
  if (nthreads == 1) {
    corr_worker(&jobs[0]);
  } else {
    for (int w = 0; w < nthreads; ++w) pthread_create(&th[w], NULL, corr_worker, &jobs[w]);
    for (int w = 0; w < nthreads; ++w) pthread_join(th[w], NULL);
  }
  for (int w = 0; w < nthreads; ++w)
    if (jobs[w].status != OR_OK) status = jobs[w].status;
  free(jobs);
  free(th);
  return status;
}

/*
 * Decode a packed block into separate int32 planes re[c][i][t], im[c][i][t]
 * (all channels).  Used by tests to evaluate definitions independently.
 */
int oracle_decode(const uint8_t* in, int layout, int bits, int hi_is_real, int N, int C, int T,
                  int32_t* re, int32_t* im) {
  if (!in || !re || !im || (bits != 4 && bits != 8)) return OR_EINVAL;
  int status = OR_OK;
  for (int c = 0; c < C; ++c)
    for (int i = 0; i < N; ++i)
      for (int t = 0; t < T; ++t) {
        int a, b;
        int st = decode(in, layout, bits, hi_is_real, N, C, T, c, i, t, &a, &b);
        if (st != OR_OK) status = st;
        size_t k = ((size_t)c * N + i) * T + t;
        re[k] = a;
        im[k] = b;
      }
  return status;
}

/*
 * The same visibility definition over complex double samples
 * x[c][i][t][2] (re, im), used for the FX == XF identity of Sec. 2:
 * vis[c][b][2] += sum_t x_i conj(x_j).
 */
int oracle_correlate_cd(const double* x, int N, int C, int T, double* vis) {
  if (!x || !vis) return OR_EINVAL;
  size_t nb = (size_t)N * (N + 1) / 2;
  for (int c = 0; c < C; ++c)
    for (int i = 0; i < N; ++i)
      for (int j = 0; j <= i; ++j) {
        double sre = 0, sim = 0;
        const double* xi = x + (((size_t)c * N + i) * T) * 2;
        const double* xj = x + (((size_t)c * N + j) * T) * 2;
        for (int t = 0; t < T; ++t) {
          double ai = xi[2 * t], bi = xi[2 * t + 1], aj = xj[2 * t], bj = xj[2 * t + 1];
          sre += ai * aj + bi * bj;
          sim += bi * aj - ai * bj;
        }
        size_t b = (size_t)i * (i + 1) / 2 + j;
        vis[((size_t)c * nb + b) * 2] += sre;
        vis[((size_t)c * nb + b) * 2 + 1] += sim;
      }
  return OR_OK;
}

/*
 * Correlation coefficients rho_ij = V_ij / sqrt(V_ii V_jj) in FP64, written
 * as double(V) / sqrt(double(V_ii) * double(V_jj)).  The paper does not
 * define a normalisation; this is the standard one.  Where V_ii * V_jj == 0,
 * rho = 0 and zero_flag[c][b] = 1.
 */
int oracle_normalise(const int64_t* vis, int N, int C, double* rho, uint8_t* zero_flag) {
  if (!vis || !rho) return OR_EINVAL;
  size_t nb = (size_t)N * (N + 1) / 2;
  for (int c = 0; c < C; ++c)
    for (int i = 0; i < N; ++i)
      for (int j = 0; j <= i; ++j) {
        const int64_t* v = vis + (size_t)c * nb * 2;
        size_t b = (size_t)i * (i + 1) / 2 + j;
        size_t bii = (size_t)i * (i + 1) / 2 + i, bjj = (size_t)j * (j + 1) / 2 + j;
        double pii = (double)v[2 * bii], pjj = (double)v[2 * bjj];
        double den2 = pii * pjj;
        double* r = rho + ((size_t)c * nb + b) * 2;
        if (den2 == 0.0) {
          r[0] = 0.0;
          r[1] = 0.0;
          if (zero_flag) zero_flag[(size_t)c * nb + b] = 1;
        } else {
          double den = sqrt(den2);
          r[0] = (double)v[2 * b] / den;
          r[1] = (double)v[2 * b + 1] / den;
          if (zero_flag) zero_flag[(size_t)c * nb + b] = 0;
        }
      }
  return OR_OK;
}

/*
 * Projected power P[k][v] = sum_t | sum_i conj(w_v,i) x_i(c_k, t) |^2 for
 * complex integer weight vectors w[v][i][2].  For the Hermitian matrix V of
 * a channel, P equals w^H V w, which gives a full-coverage check of a
 * visibility matrix at sizes where the full oracle is too slow.  Each
 * channel's samples are decoded once (as in correlate_channel); channels are
 * spread over nthreads threads (<= 1: serial).
 */
typedef struct {
  const uint8_t* in;
  int layout, bits, hi_is_real, N, C, T;
  const int* chans;
  int nchan;
  const int32_t* w;
  int nvec;
  int64_t* out;
  int stride, offset;
  int status;
} power_job;

static int power_channel(const power_job* jb, int c, int64_t* out) {
  int N = jb->N, T = jb->T;
  int* re = (int*)malloc(sizeof(int) * (size_t)N * (T > 0 ? T : 1));
  int* im = (int*)malloc(sizeof(int) * (size_t)N * (T > 0 ? T : 1));
  if (!re || !im) {
    free(re);
    free(im);
    return OR_ENOMEM;
  }
  int status = OR_OK;
  for (int i = 0; i < N; ++i)
    for (int t = 0; t < T; ++t) {
      int st = decode(jb->in, jb->layout, jb->bits, jb->hi_is_real, N, jb->C, T, c, i, t,
                      &re[(size_t)i * T + t], &im[(size_t)i * T + t]);
      if (st != OR_OK) status = st;
    }
  for (int v = 0; v < jb->nvec; ++v) {
    const int32_t* wv = jb->w + (size_t)v * N * 2;
    int64_t acc = 0;
    for (int t = 0; t < T; ++t) {
      int64_t pre = 0, pim = 0;
      for (int i = 0; i < N; ++i) {
        int64_t a = re[(size_t)i * T + t], b = im[(size_t)i * T + t];
        int64_t wr = wv[2 * i], wi = wv[2 * i + 1];
        /* conj(w) * x = (wr - i wi)(a + i b) = (wr a + wi b) + i (wr b - wi a) */
        pre += wr * a + wi * b;
        pim += wr * b - wi * a;
      }
      acc += pre * pre + pim * pim;
    }
    out[v] = acc;
  }
  free(re);
  free(im);
  return status;
}

static void* power_worker(void* arg) {
  power_job* jb = (power_job*)arg;
  for (int k = jb->offset; k < jb->nchan; k += jb->stride) {
    int c = jb->chans ? jb->chans[k] : k;
    int st = power_channel(jb, c, jb->out + (size_t)k * jb->nvec);
    if (st != OR_OK) jb->status = st;
  }
  return NULL;
}

int oracle_projected_power(const uint8_t* in, int layout, int bits, int hi_is_real, int N, int C,
                           int T, const int* chans, int nchan, const int32_t* w, int nvec,
                           int64_t* out, int nthreads) {
  if (!in || !w || !out || N < 1 || C < 1 || T < 0 || nvec < 0 || (bits != 4 && bits != 8) ||
      layout < 0 || layout > 2)
    return OR_EINVAL;
  if (!chans) nchan = C;
  for (int k = 0; chans && k < nchan; ++k)
    if (chans[k] < 0 || chans[k] >= C) return OR_EINVAL;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > nchan) nthreads = nchan > 0 ? nchan : 1;
  power_job* jobs = (power_job*)calloc((size_t)nthreads, sizeof(power_job));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !th) {
    free(jobs);
    free(th);
    return OR_ENOMEM;
  }
  for (int k = 0; k < nthreads; ++k) {
    power_job jb = {in, layout, bits, hi_is_real, N, C, T, chans, nchan, w, nvec, out, nthreads, k,
                    OR_OK};
    jobs[k] = jb;
  }
  if (nthreads == 1) {
    power_worker(&jobs[0]);
  } else {
    for (int k = 0; k < nthreads; ++k) pthread_create(&th[k], NULL, power_worker, &jobs[k]);
    for (int k = 0; k < nthreads; ++k) pthread_join(th[k], NULL);
  }
  int status = OR_OK;
  for (int k = 0; k < nthreads; ++k)
    if (jobs[k].status != OR_OK) status = jobs[k].status;
  free(jobs);
  free(th);
  return status;
}
