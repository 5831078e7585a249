/*
 * Jacobi-preconditioned CG on an assembled CSR matrix, on POSIX threads
 * (oracle; test infrastructure only -- only the tests and the benchmark's CPU
 * baseline call it).
 *
 * It is the textbook Hestenes-Stiefel PCG of oracle/pcg.py (Sec. 3: diagonally
 * preconditioned CG; Saad, Iterative Methods for Sparse Linear Systems,
 * Alg. 9.1, with M = diag(A) and x0 = 0), written so that one solve uses every
 * host core:
 *
 *   r = b, z = r / d, p = z, rz = (r, z)
 *   repeat `iters` times:
 *     w = A p;  alpha = rz / (p, w)
 *     x += alpha p;  r -= alpha w;  z = r / d
 *     rz' = (r, z);  beta = rz' / rz;  rz = rz';  p = z + beta p
 *
 * Rows (and vector entries) are split into one contiguous range per thread.
 * Each thread sums its part of every inner product in index order; the parts
 * are added in thread order, so a given thread count always gives the same
 * bits.  Every row of A p is summed in the CSR order, like a sequential loop.
 * The arithmetic is plain C doubles (built with -ffp-contract=off: no fused
 * multiply-adds).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct {
  int64_t n;
  const int64_t* indptr;
  const int32_t* indices;
  const double* data;
  const double* diag;
  double *x, *r, *z, *p, *w;
  int nthreads, iters;
  pthread_barrier_t bar;
  double* part; /* [nthreads][3] partial inner products */
  double rz, alpha, beta;
  double* hist; /* [iters + 1] residual 2-norms */
  int done;     /* iterations completed */
  int breakdown;
} shared_t;

typedef struct {
  shared_t* S;
  int t;
} arg_t;

static void rows_of(int64_t n, int nt, int t, int64_t* a, int64_t* b) {
  *a = n * t / nt;
  *b = n * (t + 1) / nt;
}

static void* worker(void* vp) {
  arg_t* A = (arg_t*)vp;
  shared_t* S = A->S;
  const int t = A->t;
  int64_t i0, i1;
  rows_of(S->n, S->nthreads, t, &i0, &i1);
  for (int it = 0; it < S->iters; ++it) {
    double pw = 0.0;
    for (int64_t i = i0; i < i1; ++i) {
      double s = 0.0;
      for (int64_t k = S->indptr[i]; k < S->indptr[i + 1]; ++k) s += S->data[k] * S->p[S->indices[k]];
      S->w[i] = s;
      pw += S->p[i] * s;
    }
    S->part[3 * t] = pw;
    pthread_barrier_wait(&S->bar);
    if (t == 0) {
      double pAp = 0.0;
      for (int u = 0; u < S->nthreads; ++u) pAp += S->part[3 * u];
      if (!(pAp > 0.0)) S->breakdown = 1;
      else S->alpha = S->rz / pAp;
    }
    pthread_barrier_wait(&S->bar);
    if (S->breakdown) break;
    const double alpha = S->alpha;
    double rz = 0.0, rr = 0.0;
    for (int64_t i = i0; i < i1; ++i) {
      S->x[i] += alpha * S->p[i];
      S->r[i] -= alpha * S->w[i];
      S->z[i] = S->r[i] / S->diag[i];
      rz += S->r[i] * S->z[i];
      rr += S->r[i] * S->r[i];
    }
    S->part[3 * t + 1] = rz;
    S->part[3 * t + 2] = rr;
    pthread_barrier_wait(&S->bar);
    if (t == 0) {
      double rzn = 0.0, rrn = 0.0;
      for (int u = 0; u < S->nthreads; ++u) {
        rzn += S->part[3 * u + 1];
        rrn += S->part[3 * u + 2];
      }
      S->beta = rzn / S->rz;
      S->rz = rzn;
      S->hist[it + 1] = sqrt(rrn);
      S->done = it + 1;
    }
    pthread_barrier_wait(&S->bar);
    const double beta = S->beta;
    for (int64_t i = i0; i < i1; ++i) S->p[i] = S->z[i] + beta * S->p[i];
    pthread_barrier_wait(&S->bar); /* the next product reads p of every range */
  }
  return NULL;
}

/*
 * x (length n, output) after `iters` iterations from x0 = 0; hist (length
 * iters + 1, output) the residual norms ||r_k||_2.  Returns the number of
 * iterations done (fewer than iters after a breakdown, (p, A p) <= 0), or -1
 * if memory or threads could not be had.
 */
int oracle_pcg_threads(int64_t n, const int64_t* indptr, const int32_t* indices, const double* data,
                       const double* diag, const double* b, double* x, int iters, int nthreads, double* hist) {
  if (nthreads < 1) nthreads = 1;
  shared_t S;
  S.n = n;
  S.indptr = indptr;
  S.indices = indices;
  S.data = data;
  S.diag = diag;
  S.x = x;
  S.nthreads = nthreads;
  S.iters = iters;
  S.hist = hist;
  S.done = 0;
  S.breakdown = 0;
  S.r = (double*)malloc(sizeof(double) * (size_t)n);
  S.z = (double*)malloc(sizeof(double) * (size_t)n);
  S.p = (double*)malloc(sizeof(double) * (size_t)n);
  S.w = (double*)malloc(sizeof(double) * (size_t)n);
  S.part = (double*)calloc((size_t)nthreads * 3, sizeof(double));
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
  arg_t* args = (arg_t*)malloc(sizeof(arg_t) * (size_t)nthreads);
  int result = -1;
  if (S.r && S.z && S.p && S.w && S.part && th && args) {
    double rz = 0.0, rr = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      x[i] = 0.0;
      S.r[i] = b[i];
      S.z[i] = b[i] / diag[i];
      S.p[i] = S.z[i];
      rz += S.r[i] * S.z[i];
      rr += S.r[i] * S.r[i];
    }
    S.rz = rz;
    hist[0] = sqrt(rr);
    if (pthread_barrier_init(&S.bar, NULL, (unsigned)nthreads) == 0) {
      int started = 0;
      for (int t = 0; t < nthreads; ++t) {
        args[t].S = &S;
        args[t].t = t;
        if (pthread_create(&th[t], NULL, worker, &args[t]) != 0) break;
        ++started;
      }
      if (started == nthreads) {
        for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
        result = S.done;
      } else {
        /* threads that did start would wait at the barrier forever: not recoverable here */
        abort();
      }
      pthread_barrier_destroy(&S.bar);
    }
  }
  free(S.r);
  free(S.z);
  free(S.p);
  free(S.w);
  free(S.part);
  free(th);
  free(args);
  return result;
}
