/* FP64 direct-sum N-body oracle — test infrastructure only (see oracle/__init__.py).
 *
 * Section 4 of the paper (N-Body on the Loop skeleton): every body interacts with
 * every other one (direct sum); positions are needed whole by every partition
 * (COPY transfer mode) and the bodies synchronise between iterations.
 * The paper gives neither the force law's constants nor the integrator; the
 * executor reads them as:
 *   a_i = G * sum_j m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^(3/2)   (Plummer softening,
 *         the j = i term is exactly zero and is not skipped),
 *   kick-drift-kick leapfrog:  v += dt/2 a;  x += dt v;  a = a(x);  v += dt/2 a.
 * The sum over j runs in index order, in double precision. Threads split the
 * bodies i only, so the result does not depend on the thread count.
 *
 * Pins (tests/test_oracle_nbody.py): the two-body closed form, momentum
 * conservation, a symmetric 8-body configuration, a pure-Python brute force for
 * N <= 16 and the second-order convergence of the integrator on a circular orbit.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct {
  int64_t n, i0, i1;
  const double *x; /* [n][4] = (x, y, z, m) */
  double g, eps2;
  double *a;       /* [n][3] */
} accel_job;

static void *accel_range(void *p) {
  accel_job *job = (accel_job *)p;
  for (int64_t i = job->i0; i < job->i1; ++i) {
    const double xi = job->x[4 * i + 0], yi = job->x[4 * i + 1], zi = job->x[4 * i + 2];
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int64_t j = 0; j < job->n; ++j) {
      const double dx = job->x[4 * j + 0] - xi;
      const double dy = job->x[4 * j + 1] - yi;
      const double dz = job->x[4 * j + 2] - zi;
      const double r2 = dx * dx + dy * dy + dz * dz + job->eps2;
      const double inv_r3 = 1.0 / (r2 * sqrt(r2));
      const double s = job->x[4 * j + 3] * inv_r3;
      ax += s * dx;
      ay += s * dy;
      az += s * dz;
    }
    job->a[3 * i + 0] = job->g * ax;
    job->a[3 * i + 1] = job->g * ay;
    job->a[3 * i + 2] = job->g * az;
  }
  return NULL;
}

/* a[i] = acceleration of body i; returns 0 on success. */
int oracle_nbody_accel(int64_t n, const double *x, double g, double eps, double *a, int nthreads) {
  if (n < 0 || nthreads < 1) return 1;
  if (nthreads > 256) nthreads = 256;
  pthread_t tid[256];
  accel_job jobs[256];
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].n = n;
    jobs[t].i0 = n * t / nthreads;
    jobs[t].i1 = n * (t + 1) / nthreads;
    jobs[t].x = x;
    jobs[t].g = g;
    jobs[t].eps2 = eps * eps;
    jobs[t].a = a;
  }
  int started = 0;
  for (int t = 1; t < nthreads; ++t) {
    if (pthread_create(&tid[t], NULL, accel_range, &jobs[t]) != 0) break;
    started = t;
  }
  accel_range(&jobs[0]);
  for (int t = 1; t <= started; ++t) pthread_join(tid[t], NULL);
  /* threads that failed to start: run their share here */
  for (int t = started + 1; t < nthreads; ++t) accel_range(&jobs[t]);
  return 0;
}

/* `steps` kick-drift-kick steps in place. x: [n][4] (mass in slot 3), v, a: [n][3].
 * `a` must hold a(x) on entry and holds a(x) on exit. */
int oracle_nbody_kdk(int64_t n, double *x, double *v, double *a, double g, double eps, double dt,
                     int64_t steps, int nthreads) {
  for (int64_t s = 0; s < steps; ++s) {
    for (int64_t i = 0; i < n; ++i) {
      for (int k = 0; k < 3; ++k) {
        v[3 * i + k] += 0.5 * dt * a[3 * i + k];
        x[4 * i + k] += dt * v[3 * i + k];
      }
    }
    int rc = oracle_nbody_accel(n, x, g, eps, a, nthreads);
    if (rc) return rc;
    for (int64_t i = 0; i < n; ++i)
      for (int k = 0; k < 3; ++k) v[3 * i + k] += 0.5 * dt * a[3 * i + k];
  }
  return 0;
}
