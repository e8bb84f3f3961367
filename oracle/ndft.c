/*
 * Direct nonequispaced DFT, the CPU oracle of this repository.
 *
 * TEST INFRASTRUCTURE ONLY: this file is the slow, plain FP64 reference
 * against which the CUDA library is checked.  It shares no code with the
 * CUDA path, and no product code may link or call it.
 *
 * Definitions (HP-NFFT paper, Section 1):
 *   I_N   = { k in Z^d : -N_t/2 <= k_t < N_t/2 }            (N_t even)
 *   Eq. 5 = adjoint:  fhat(k) = sum_{j<M} f(x_j) exp(-2 pi i k.x_j),  k in I_N
 *   Eq. 6 = forward:  f(x_j)  = sum_{k in I_N} fhat(k) exp(+2 pi i k.x_j)
 *
 * Layouts: x is M*d doubles, point-major (x[j*d+t] pairs with N_t).  Complex
 * values are interleaved (re, im) doubles.  A full fhat is stored in C order
 * over (k_0, ..., k_{d-1}), each k_t ascending from -N_t/2.
 *
 * Every exponential is evaluated directly with sin/cos of a reduced phase;
 * there is no recurrence, no FFT and no window.  The phase k*x is reduced to
 * [-1/2, 1/2] turns using the exact product (p plus its FMA residual) so the
 * error in the angle stays near 1e-16 turns for any |k|, |x|.
 *
 * Threads: a fixed partition of the outputs over POSIX threads; each output
 * is summed over its inputs in one fixed order, so results do not depend on
 * the thread count.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define TWO_PI 6.283185307179586476925286766559

/* frac(k*x) in [-1/2, 1/2] turns, from the exact product p + e. */
static double reduced_turns(double k, double x) {
  double p = k * x;
  double e = fma(k, x, -p); /* p + e == k*x exactly */
  double r = (p - nearbyint(p)) + e;
  return r - nearbyint(r);
}

/* exp(sign * 2 pi i * turns) */
static void cis_turns(double turns, int sign, double* re, double* im) {
  double a = TWO_PI * turns;
  *re = cos(a);
  *im = sign * sin(a);
}

/* d <= 3 is embedded in three dimensions: missing leading dimensions have
 * N = 1 (only k = 0) and x = 0, so they contribute a factor exp(0) = 1. */
typedef struct {
  int64_t n3[3];   /* bandwidths, leading dims padded with 1 */
  int off;         /* 3 - d: position of the first real dimension */
  int d;
} shape3;

static int make_shape(int d, const int64_t* N, shape3* s) {
  if (d < 1 || d > 3) return -1;
  s->d = d;
  s->off = 3 - d;
  for (int t = 0; t < 3; ++t) s->n3[t] = 1;
  for (int t = 0; t < d; ++t) {
    if (N[t] < 2 || (N[t] & 1)) return -1;
    s->n3[s->off + t] = N[t];
  }
  return 0;
}

static double coord3(const shape3* s, const double* x, int64_t j, int t3) {
  int t = t3 - s->off;
  return t < 0 ? 0.0 : x[j * s->d + t];
}

static int resolve_threads(int nthreads) {
  if (nthreads > 0) return nthreads;
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  return c > 0 ? (int)c : 1;
}

typedef void* (*worker_fn)(void*);

typedef struct {
  const shape3* s;
  int64_t M;
  const double* x;
  const double* in;        /* f (adjoint) or fhat (forward), interleaved */
  const int64_t* sel;      /* selected k (K*d) or j (J), or NULL */
  int64_t nsel;            /* number of outputs */
  double* out;
  int64_t lo, hi;          /* this worker's output range */
  int status;
} job;

static int run_pool(worker_fn fn, job* proto, int64_t nout, int nthreads) {
  int T = resolve_threads(nthreads);
  if (T > nout && nout > 0) T = (int)nout;
  if (T < 1) T = 1;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * T);
  job* jobs = (job*)malloc(sizeof(job) * T);
  if (!th || !jobs) { free(th); free(jobs); return -3; }
  int64_t chunk = (nout + T - 1) / T;
  int started = 0, rc = 0;
  for (int i = 0; i < T; ++i) {
    jobs[i] = *proto;
    jobs[i].lo = i * chunk < nout ? i * chunk : nout;
    jobs[i].hi = (i + 1) * chunk < nout ? (i + 1) * chunk : nout;
    jobs[i].status = 0;
    if (pthread_create(&th[i], NULL, fn, &jobs[i]) != 0) { rc = -4; break; }
    ++started;
  }
  for (int i = 0; i < started; ++i) {
    pthread_join(th[i], NULL);
    if (jobs[i].status) rc = jobs[i].status;
  }
  free(th);
  free(jobs);
  return rc;
}

/* ---- Eq. 5 over all of I_N: worker owns a range of flat C-order k ------- */
static void* adjoint_full_worker(void* arg) {
  job* J = (job*)arg;
  const shape3* s = J->s;
  const int64_t n0 = s->n3[0], n1 = s->n3[1], n2 = s->n3[2];
  double* e0 = (double*)malloc(sizeof(double) * 2 * n0);
  double* e1 = (double*)malloc(sizeof(double) * 2 * n1);
  double* e2 = (double*)malloc(sizeof(double) * 2 * n2);
  if (!e0 || !e1 || !e2) { J->status = -3; free(e0); free(e1); free(e2); return NULL; }
  for (int64_t j = 0; j < J->M; ++j) {
    const double fr = J->in[2 * j], fi = J->in[2 * j + 1];
    const double x0 = coord3(s, J->x, j, 0), x1 = coord3(s, J->x, j, 1), x2 = coord3(s, J->x, j, 2);
    /* E_t(k_t) = exp(-2 pi i k_t x_t) for every k_t = i - N_t/2 of dimension t */
    for (int64_t a = 0; a < n0; ++a) cis_turns(reduced_turns((double)(a - n0 / 2), x0), -1, &e0[2 * a], &e0[2 * a + 1]);
    for (int64_t b = 0; b < n1; ++b) cis_turns(reduced_turns((double)(b - n1 / 2), x1), -1, &e1[2 * b], &e1[2 * b + 1]);
    for (int64_t c = 0; c < n2; ++c) cis_turns(reduced_turns((double)(c - n2 / 2), x2), -1, &e2[2 * c], &e2[2 * c + 1]);
    /* fhat(k) += f_j E_0(k_0) E_1(k_1) E_2(k_2) over this worker's flat k */
    for (int64_t k = J->lo; k < J->hi;) {
      const int64_t row = k / n2, c_lo = k % n2;
      const int64_t c_hi = (n2 - c_lo < J->hi - k) ? n2 : c_lo + (J->hi - k);
      const int64_t a = row / n1, b = row % n1;
      const double ar = fr * e0[2 * a] - fi * e0[2 * a + 1];
      const double ai = fr * e0[2 * a + 1] + fi * e0[2 * a];
      const double br = ar * e1[2 * b] - ai * e1[2 * b + 1];
      const double bi = ar * e1[2 * b + 1] + ai * e1[2 * b];
      double* o = J->out + 2 * (row * n2);
      for (int64_t c = c_lo; c < c_hi; ++c) {
        o[2 * c] += br * e2[2 * c] - bi * e2[2 * c + 1];
        o[2 * c + 1] += br * e2[2 * c + 1] + bi * e2[2 * c];
      }
      k += c_hi - c_lo;
    }
  }
  free(e0); free(e1); free(e2);
  return NULL;
}

/* ---- Eq. 5 at a list of frequencies k (sampled mode) -------------------- */
static void* adjoint_sel_worker(void* arg) {
  job* J = (job*)arg;
  const shape3* s = J->s;
  for (int64_t q = J->lo; q < J->hi; ++q) {
    const int64_t* k = J->sel + q * s->d;
    double sr = 0.0, si = 0.0;
    for (int64_t j = 0; j < J->M; ++j) {
      double r = 0.0;
      for (int t = 0; t < s->d; ++t) r += reduced_turns((double)k[t], J->x[j * s->d + t]);
      double cr, ci;
      cis_turns(r - nearbyint(r), -1, &cr, &ci);
      const double fr = J->in[2 * j], fi = J->in[2 * j + 1];
      sr += fr * cr - fi * ci;
      si += fr * ci + fi * cr;
    }
    J->out[2 * q] = sr;
    J->out[2 * q + 1] = si;
  }
  return NULL;
}

/* ---- Eq. 6 at points j (all points, or a list) -------------------------- */
static void* forward_worker(void* arg) {
  job* J = (job*)arg;
  const shape3* s = J->s;
  const int64_t n0 = s->n3[0], n1 = s->n3[1], n2 = s->n3[2];
  double* e0 = (double*)malloc(sizeof(double) * 2 * n0);
  double* e1 = (double*)malloc(sizeof(double) * 2 * n1);
  double* e2 = (double*)malloc(sizeof(double) * 2 * n2);
  if (!e0 || !e1 || !e2) { J->status = -3; free(e0); free(e1); free(e2); return NULL; }
  for (int64_t q = J->lo; q < J->hi; ++q) {
    const int64_t j = J->sel ? J->sel[q] : q;
    if (j < 0 || j >= J->M) { J->status = -1; break; }
    const double x0 = coord3(s, J->x, j, 0), x1 = coord3(s, J->x, j, 1), x2 = coord3(s, J->x, j, 2);
    /* E_t(k_t) = exp(+2 pi i k_t x_t) */
    for (int64_t a = 0; a < n0; ++a)
      cis_turns(reduced_turns((double)(a - n0 / 2), x0), +1, &e0[2 * a], &e0[2 * a + 1]);
    for (int64_t b = 0; b < n1; ++b)
      cis_turns(reduced_turns((double)(b - n1 / 2), x1), +1, &e1[2 * b], &e1[2 * b + 1]);
    for (int64_t c = 0; c < n2; ++c)
      cis_turns(reduced_turns((double)(c - n2 / 2), x2), +1, &e2[2 * c], &e2[2 * c + 1]);
    double sr = 0.0, si = 0.0;
    for (int64_t a = 0; a < n0; ++a) {
      for (int64_t b = 0; b < n1; ++b) {
        const double abr = e0[2 * a] * e1[2 * b] - e0[2 * a + 1] * e1[2 * b + 1];
        const double abi = e0[2 * a] * e1[2 * b + 1] + e0[2 * a + 1] * e1[2 * b];
        const double* h = J->in + 2 * ((a * n1 + b) * n2);
        for (int64_t c = 0; c < n2; ++c) {
          /* E(k) = E_0 E_1 E_2 */
          const double er = abr * e2[2 * c] - abi * e2[2 * c + 1];
          const double ei = abr * e2[2 * c + 1] + abi * e2[2 * c];
          sr += h[2 * c] * er - h[2 * c + 1] * ei;
          si += h[2 * c] * ei + h[2 * c + 1] * er;
        }
      }
    }
    J->out[2 * q] = sr;
    J->out[2 * q + 1] = si;
  }
  free(e0); free(e1); free(e2);
  return NULL;
}

/* Eq. 5.  ksel == NULL: out holds all of I_N (C order), else out[q] is
 * fhat(ksel[q*d .. q*d+d-1]) for q < nsel.  Returns 0 or a negative code. */
int oracle_ndft_adjoint(int d, const int64_t* N, int64_t M, const double* x, const double* f,
                        int64_t nsel, const int64_t* ksel, double* out, int nthreads) {
  shape3 s;
  if (make_shape(d, N, &s) || M < 0 || !out) return -1;
  if (M > 0 && (!x || !f)) return -1;
  job proto;
  memset(&proto, 0, sizeof proto);
  proto.s = &s; proto.M = M; proto.x = x; proto.in = f; proto.sel = ksel; proto.nsel = nsel; proto.out = out;
  if (ksel) {
    memset(out, 0, sizeof(double) * 2 * (size_t)nsel);
    if (nsel == 0) return 0;
    return run_pool(adjoint_sel_worker, &proto, nsel, nthreads);
  }
  const int64_t total = s.n3[0] * s.n3[1] * s.n3[2];
  memset(out, 0, sizeof(double) * 2 * (size_t)total);
  return run_pool(adjoint_full_worker, &proto, total, nthreads);
}

/* Eq. 6.  jsel == NULL: out[j] for every j < M (nsel ignored), else out[q]
 * is f(x_{jsel[q]}) for q < nsel.  fhat holds all of I_N in C order. */
int oracle_ndft_forward(int d, const int64_t* N, int64_t M, const double* x, const double* fhat,
                        int64_t nsel, const int64_t* jsel, double* out, int nthreads) {
  shape3 s;
  if (make_shape(d, N, &s) || M < 0 || !fhat || !out) return -1;
  if (M > 0 && !x) return -1;
  job proto;
  memset(&proto, 0, sizeof proto);
  proto.s = &s; proto.M = M; proto.x = x; proto.in = fhat; proto.sel = jsel; proto.out = out;
  const int64_t nout = jsel ? nsel : M;
  proto.nsel = nout;
  if (nout == 0) return 0;
  return run_pool(forward_worker, &proto, nout, nthreads);
}

int oracle_threads(int nthreads) { return resolve_threads(nthreads); }
