/*
 * FP64 CPU oracle for the PDMP sample-morphing path (arXiv 2108.11775).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  It shares no code,
 * header, table or constant with the CUDA library under
 * paper_2108_11775_gb300/csrc, and the CUDA library never calls it.
 *
 * Everything here is the plain definition in double precision with libm
 * exp/sin/cos/log, written for a reader to check against the paper by eye:
 * no blocking, no fused or reordered sums.  Threads split independent
 * samples (or, for the fit's transposed sums, independent centres) and never
 * change the order of any sum.
 *
 * What each function follows:
 *   features, cost, gradient, Hessian  -- Sec. 3.1 (occupancy p(y=1|x) with a
 *       sigmoid output; its input derivatives); the feature map is the
 *       continuous "Hilbert map" family Sec. 3.1 cites: RBF
 *       phi_m = exp(-gamma |x-mu_m|^2) or random Fourier phi_m = cos(w_m.x+b_m).
 *   morph                              -- Eq. (1) integrated by Euler's method
 *       (Sec. 3.2, last sentence of "Constructing Diffeomorphisms"):
 *       x_{t+1} = x_t - eta * grad c(x_t), t = 0..T-1.
 *   inverse                            -- Eq. (2): each Euler step undone by
 *       the fixed point y = z + eta * grad c(y).
 *   vjp / parameter gradient           -- chain rule through the Euler steps
 *       of Eq. (1).
 *   log-det                            -- the Jacobian determinant of the map
 *       that Sec. 3.2 ("Drawing Samples") says sampling does not need; here it
 *       is computed because density evaluation does.
 *   Lipschitz bound                    -- Sec. 3.2: the gradient of the cost
 *       must be Lipschitz for the flow to be a diffeomorphism; a certified
 *       bound L on |Hessian| sets the Euler step eta < 1/L.
 *   fit                                -- Sec. 3.1: binary cross entropy
 *       minimised by gradient descent (here Nesterov-accelerated, preceded by a
 *       power-iteration step-size estimate).
 *   box labels                         -- ground-truth occupancy of the
 *       dataset D of Sec. 3.1, from axis-aligned boxes.
 *   MLP forward/backward               -- the surrogate network (no
 *       counterpart in the paper): dense layers with SiLU, MSE loss.
 *   C-space pull-back                  -- Sec. 3.2, Eq. (3): a planar serial
 *       chain's body points, the task-space gradient pulled back through the
 *       kinematic Jacobians, the morph in joint space, a certified bound.
 *   Philox4x32-10, uniform batch       -- the base samples a device-side
 *       sampler draws (Sec. 3.3's prior), from the generator's published
 *       definition, so the oracle can regenerate them.
 *   tanh network cost                  -- Sec. 3.1's own occupancy model: a
 *       fully connected network, tanh between hidden layers, sigmoid output;
 *       its input gradient / Hessian, the morph of Eq. (1) through it, and a
 *       certified Lipschitz bound from spectral norms.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define KIND_RBF 0
#define KIND_RFF 1
#define MAXD 8

/* ------------------------------------------------------------------ */
/* threading over independent items                                   */
/* ------------------------------------------------------------------ */
static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
int orc_get_threads(void) { return g_threads; }

typedef void (*range_fn)(void* ctx, long lo, long hi);
typedef struct { range_fn fn; void* ctx; long lo, hi; } range_job;

static void* range_trampoline(void* p) {
  range_job* j = (range_job*)p;
  j->fn(j->ctx, j->lo, j->hi);
  return NULL;
}

/* Calls fn(ctx, lo, hi) on disjoint contiguous ranges that cover [0, n),
 * on at most nt threads.  Items are independent, so the results do not depend
 * on the split. */
static void parallel_range_nt(long n, int nt, range_fn fn, void* ctx) {
  if (n <= 0) return;
  if (nt > n) nt = (int)n;
  if (nt <= 1) { fn(ctx, 0, n); return; }
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nt);
  range_job* jobs = (range_job*)malloc(sizeof(range_job) * nt);
  long chunk = (n + nt - 1) / nt;
  int started = 0;
  for (int t = 0; t < nt; ++t) {
    long lo = t * chunk, hi = lo + chunk;
    if (lo >= n) break;
    if (hi > n) hi = n;
    jobs[t].fn = fn; jobs[t].ctx = ctx; jobs[t].lo = lo; jobs[t].hi = hi;
    if (pthread_create(&th[t], NULL, range_trampoline, &jobs[t]) != 0) {
      fn(ctx, lo, hi);            /* could not start a thread: do it here */
      jobs[t].fn = NULL;
    }
    started = t + 1;
  }
  for (int t = 0; t < started; ++t)
    if (jobs[t].fn) pthread_join(th[t], NULL);
  free(th); free(jobs);
}

static void parallel_range(long n, range_fn fn, void* ctx) { parallel_range_nt(n, g_threads, fn, ctx); }

/* As parallel_range, with no more threads than give each about a million
 * feature evaluations (item_cost per item): the fit's per-iteration passes
 * are small, and a thread per pass would cost more than the pass. */
static void parallel_range_sized(long n, double item_cost, range_fn fn, void* ctx) {
  double want = (double)n * item_cost / 1.0e6;
  int nt = want < 1.0 ? 1 : (want < (double)g_threads ? (int)want : g_threads);
  parallel_range_nt(n, nt, fn, ctx);
}

/* ------------------------------------------------------------------ */
/* the occupancy field                                                 */
/* ------------------------------------------------------------------ */
typedef struct {
  int kind;              /* KIND_RBF or KIND_RFF */
  int d;                 /* dimension of x */
  long M;                /* number of features */
  const double* centres; /* RBF: mu, M x d.  RFF: omega, M x d */
  const double* phase;   /* RFF: b, M.  RBF: unused */
  double gamma;          /* RBF width */
  const double* w;       /* M weights */
  double bias;           /* logit bias */
} field_t;

/* logistic sigmoid and its first two derivatives, from exp(-|s|) so that no
 * intermediate overflows:  sigma' = sigma (1 - sigma),
 * sigma'' = sigma (1 - sigma) (1 - 2 sigma). */
void orc_sigmoid3(double s, double out[3]) {
  double e = exp(-fabs(s));
  double sig = s >= 0 ? 1.0 / (1.0 + e) : e / (1.0 + e);
  double one_minus = s >= 0 ? e / (1.0 + e) : 1.0 / (1.0 + e);
  out[0] = sig;
  out[1] = sig * one_minus;
  out[2] = sig * one_minus * (one_minus - sig);
}

/* One feature and its derivatives at x.
 *   RBF: phi = exp(-gamma r^2), r = x - mu,
 *        dphi = -2 gamma r phi,
 *        d2phi = phi (4 gamma^2 r r^T - 2 gamma I).
 *   RFF: theta = omega.x + b, phi = cos(theta),
 *        dphi = -sin(theta) omega,
 *        d2phi = -cos(theta) omega omega^T.
 * dphi / d2phi may be NULL. */
static double feature(const field_t* f, long m, const double* x, double* dphi, double* d2phi) {
  int d = f->d;
  const double* c = f->centres + m * d;
  if (f->kind == KIND_RBF) {
    double r[MAXD], r2 = 0.0;
    for (int i = 0; i < d; ++i) { r[i] = x[i] - c[i]; r2 += r[i] * r[i]; }
    double phi = exp(-f->gamma * r2);
    if (dphi)
      for (int i = 0; i < d; ++i) dphi[i] = -2.0 * f->gamma * r[i] * phi;
    if (d2phi)
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j)
          d2phi[i * d + j] = phi * (4.0 * f->gamma * f->gamma * r[i] * r[j] - (i == j ? 2.0 * f->gamma : 0.0));
    return phi;
  } else {
    double theta = f->phase[m];
    for (int i = 0; i < d; ++i) theta += c[i] * x[i];
    double cs = cos(theta), sn = sin(theta);
    if (dphi)
      for (int i = 0; i < d; ++i) dphi[i] = -sn * c[i];
    if (d2phi)
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) d2phi[i * d + j] = -cs * c[i] * c[j];
    return cs;
  }
}

/* Logit s = sum_m w_m phi_m(x) + bias with gradient and (optional) Hessian of s,
 * and the absolute sum  sum_m |w_m| |grad phi_m(x)|_2  (optional). */
static double logit_derivs(const field_t* f, const double* x, double* gs, double* hs, double* abs_grad_sum) {
  int d = f->d;
  double s = f->bias;
  double dphi[MAXD], d2phi[MAXD * MAXD];
  for (int i = 0; i < d; ++i) gs[i] = 0.0;
  if (hs) for (int i = 0; i < d * d; ++i) hs[i] = 0.0;
  if (abs_grad_sum) *abs_grad_sum = 0.0;
  for (long m = 0; m < f->M; ++m) {
    double phi = feature(f, m, x, dphi, hs ? d2phi : NULL);
    double wm = f->w[m];
    s += wm * phi;
    for (int i = 0; i < d; ++i) gs[i] += wm * dphi[i];
    if (hs) for (int i = 0; i < d * d; ++i) hs[i] += wm * d2phi[i];
    if (abs_grad_sum) {
      double nrm = 0.0;
      for (int i = 0; i < d; ++i) nrm += dphi[i] * dphi[i];
      *abs_grad_sum += fabs(wm) * sqrt(nrm);
    }
  }
  return s;
}

/* Cost c = sigma(s), grad c = sigma'(s) grad s,
 * Hess c = sigma'(s) Hess s + sigma''(s) grad s grad s^T. */
static double cost_derivs(const field_t* f, const double* x, double* gc, double* hc, double* s_out, double* scale_out) {
  int d = f->d;
  double gs[MAXD], hs[MAXD * MAXD], sg[3], abs_sum;
  double s = logit_derivs(f, x, gs, hc ? hs : NULL, scale_out ? &abs_sum : NULL);
  orc_sigmoid3(s, sg);
  for (int i = 0; i < d; ++i) gc[i] = sg[1] * gs[i];
  if (hc)
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) hc[i * d + j] = sg[1] * hs[i * d + j] + sg[2] * gs[i] * gs[j];
  if (s_out) *s_out = s;
  if (scale_out) *scale_out = sg[1] * abs_sum;
  return sg[0];
}

static field_t make_field(int kind, int d, long M, const double* centres, const double* phase, double gamma,
                          const double* w, double bias) {
  field_t f;
  f.kind = kind; f.d = d; f.M = M; f.centres = centres; f.phase = phase;
  f.gamma = gamma; f.w = w; f.bias = bias;
  return f;
}

/* ------------------------------------------------------------------ */
/* point evaluation                                                    */
/* ------------------------------------------------------------------ */
typedef struct {
  const field_t* f; const double* x;
  double *c, *s, *g, *h, *scale;
} eval_ctx;

static void eval_range(void* p, long lo, long hi) {
  eval_ctx* e = (eval_ctx*)p;
  int d = e->f->d;
  for (long n = lo; n < hi; ++n) {
    double gc[MAXD], hc[MAXD * MAXD], s, sc;
    double c = cost_derivs(e->f, e->x + n * d, gc, e->h ? hc : NULL, &s, e->scale ? &sc : NULL);
    if (e->c) e->c[n] = c;
    if (e->s) e->s[n] = s;
    if (e->g) for (int i = 0; i < d; ++i) e->g[n * d + i] = gc[i];
    if (e->h) for (int i = 0; i < d * d; ++i) e->h[n * d * d + i] = hc[i];
    if (e->scale) e->scale[n] = sc;
  }
}

/* Evaluates, at n points x (n x d): c, s, grad c (n x d), Hess c (n x d x d)
 * and sigma'(s) * sum_m |w_m| |grad phi_m| (n).  Any output may be NULL. */
int orc_eval(int kind, int d, long M, const double* centres, const double* phase, double gamma,
             const double* w, double bias, const double* x, long n,
             double* c, double* s, double* grad, double* hess, double* scale) {
  if (d < 1 || d > MAXD || M < 0 || n < 0) return 1;
  field_t f = make_field(kind, d, M, centres, phase, gamma, w, bias);
  eval_ctx e = { &f, x, c, s, grad, hess, scale };
  parallel_range(n, eval_range, &e);
  return 0;
}

/* ------------------------------------------------------------------ */
/* morph: Euler integration of Eq. (1)                                 */
/* ------------------------------------------------------------------ */
typedef struct {
  const field_t* f; const double* x0; long N; int T; double eta;
  double* xT; double* traj;
} morph_ctx;

static void morph_range(void* p, long lo, long hi) {
  morph_ctx* m = (morph_ctx*)p;
  int d = m->f->d;
  for (long n = lo; n < hi; ++n) {
    double x[MAXD], gc[MAXD];
    for (int i = 0; i < d; ++i) x[i] = m->x0[n * d + i];
    if (m->traj) for (int i = 0; i < d; ++i) m->traj[(n * (m->T + 1)) * d + i] = x[i];
    for (int t = 0; t < m->T; ++t) {
      cost_derivs(m->f, x, gc, NULL, NULL, NULL);
      for (int i = 0; i < d; ++i) x[i] = x[i] - m->eta * gc[i];
      if (m->traj) for (int i = 0; i < d; ++i) m->traj[(n * (m->T + 1) + t + 1) * d + i] = x[i];
    }
    if (m->xT) for (int i = 0; i < d; ++i) m->xT[n * d + i] = x[i];
  }
}

/* x_T of every sample (N x d), and optionally the whole trajectory
 * traj (N x (T+1) x d, traj[n][0] = x_0). */
int orc_morph(int kind, int d, long M, const double* centres, const double* phase, double gamma,
              const double* w, double bias, const double* x0, long N, int T, double eta,
              double* xT, double* traj) {
  if (d < 1 || d > MAXD || M < 0 || N < 0 || T < 0) return 1;
  field_t f = make_field(kind, d, M, centres, phase, gamma, w, bias);
  morph_ctx c = { &f, x0, N, T, eta, xT, traj };
  parallel_range(N, morph_range, &c);
  return 0;
}

/* ------------------------------------------------------------------ */
/* inverse: Eq. (2), each Euler step undone by fixed-point iteration   */
/* ------------------------------------------------------------------ */
typedef struct {
  const field_t* f; const double* z; long N; int T; double eta; double tol; int maxit;
  double* y; int* iters_used;
} inv_ctx;

static void inverse_range(void* p, long lo, long hi) {
  inv_ctx* c = (inv_ctx*)p;
  int d = c->f->d;
  for (long n = lo; n < hi; ++n) {
    double z[MAXD], y[MAXD], gc[MAXD];
    int worst = 0;
    for (int i = 0; i < d; ++i) z[i] = c->z[n * d + i];
    /* steps are undone last-first; the field does not depend on t, so each
     * undo solves y = z + eta grad c(y) for the current z */
    for (int t = c->T - 1; t >= 0; --t) {
      for (int i = 0; i < d; ++i) y[i] = z[i];
      int it;
      for (it = 0; it < c->maxit; ++it) {
        cost_derivs(c->f, y, gc, NULL, NULL, NULL);
        double delta = 0.0;
        for (int i = 0; i < d; ++i) {
          double ynew = z[i] + c->eta * gc[i];
          double a = fabs(ynew - y[i]);
          if (a > delta) delta = a;
          y[i] = ynew;
        }
        if (delta < c->tol) { ++it; break; }
      }
      if (it > worst) worst = it;
      for (int i = 0; i < d; ++i) z[i] = y[i];
    }
    for (int i = 0; i < d; ++i) c->y[n * d + i] = z[i];
    if (c->iters_used) c->iters_used[n] = worst;
  }
}

int orc_morph_inverse(int kind, int d, long M, const double* centres, const double* phase, double gamma,
                      const double* w, double bias, const double* z, long N, int T, double eta,
                      double tol, int maxit, double* y, int* iters_used) {
  if (d < 1 || d > MAXD || M < 0 || N < 0 || T < 0) return 1;
  field_t f = make_field(kind, d, M, centres, phase, gamma, w, bias);
  inv_ctx c = { &f, z, N, T, eta, tol, maxit, y, iters_used };
  parallel_range(N, inverse_range, &c);
  return 0;
}

/* ------------------------------------------------------------------ */
/* VJP through the Euler chain                                         */
/* ------------------------------------------------------------------ */
typedef struct {
  const field_t* f; const double* x0; long N; int T; double eta;
  const double* gT; double* g0; double* gw_rows; double* gb_rows;
} vjp_ctx;

/* For one sample: g_t = (I - eta H(x_t))^T g_{t+1} = (I - eta H(x_t)) g_{t+1}
 * (H symmetric), and the derivative of <g_T, x_T> with respect to w_m and the
 * bias:  sum_t g_{t+1}^T (-eta d grad c(x_t) / d w_m), with
 * d grad c / d w_m = sigma''(s) phi_m grad s + sigma'(s) grad phi_m and
 * d grad c / d bias = sigma''(s) grad s.  gw_row (M) accumulates this sample's
 * share; it may be NULL. */
static void vjp_one(const field_t* f, const double* x0, int T, double eta, const double* gT, double* g0,
                    double* gw_row, double* gb) {
  int d = f->d;
  double* xs = (double*)malloc(sizeof(double) * (size_t)(T + 1) * d);
  double gc[MAXD], hc[MAXD * MAXD], g[MAXD], gnew[MAXD];
  for (int i = 0; i < d; ++i) xs[i] = x0[i];
  for (int t = 0; t < T; ++t) {
    cost_derivs(f, xs + t * d, gc, NULL, NULL, NULL);
    for (int i = 0; i < d; ++i) xs[(t + 1) * d + i] = xs[t * d + i] - eta * gc[i];
  }
  for (int i = 0; i < d; ++i) g[i] = gT[i];
  if (gb) *gb = 0.0;
  for (int t = T - 1; t >= 0; --t) {
    const double* x = xs + t * d;
    /* g currently holds g_{t+1} */
    if (gw_row || gb) {
      double gs[MAXD], sg[3], dphi[MAXD];
      double s = logit_derivs(f, x, gs, NULL, NULL);
      orc_sigmoid3(s, sg);
      double g_dot_gs = 0.0;
      for (int i = 0; i < d; ++i) g_dot_gs += g[i] * gs[i];
      if (gb) *gb += -eta * sg[2] * g_dot_gs;
      if (gw_row)
        for (long m = 0; m < f->M; ++m) {
          double phi = feature(f, m, x, dphi, NULL);
          double g_dot_dphi = 0.0;
          for (int i = 0; i < d; ++i) g_dot_dphi += g[i] * dphi[i];
          gw_row[m] += -eta * (sg[2] * phi * g_dot_gs + sg[1] * g_dot_dphi);
        }
    }
    cost_derivs(f, x, gc, hc, NULL, NULL);
    for (int i = 0; i < d; ++i) {
      double hv = 0.0;
      for (int j = 0; j < d; ++j) hv += hc[i * d + j] * g[j];
      gnew[i] = g[i] - eta * hv;
    }
    for (int i = 0; i < d; ++i) g[i] = gnew[i];
  }
  for (int i = 0; i < d; ++i) g0[i] = g[i];
  free(xs);
}

static void vjp_range(void* p, long lo, long hi) {
  vjp_ctx* c = (vjp_ctx*)p;
  int d = c->f->d;
  for (long n = lo; n < hi; ++n)
    vjp_one(c->f, c->x0 + n * d, c->T, c->eta, c->gT + n * d, c->g0 + n * d,
            c->gw_rows ? c->gw_rows + n * c->f->M : NULL, c->gb_rows ? c->gb_rows + n : NULL);
}

/* g0 (N x d) = (d x_T / d x_0)^T g_T per sample.  If gw (M) is given it
 * receives d/dw of sum_n <g_T[n], x_T[n]>; gbias (1) likewise for the bias.
 * The per-sample parameter rows are summed over n in sample order. */
int orc_morph_vjp(int kind, int d, long M, const double* centres, const double* phase, double gamma,
                  const double* w, double bias, const double* x0, long N, int T, double eta,
                  const double* gT, double* g0, double* gw, double* gbias) {
  if (d < 1 || d > MAXD || M < 0 || N < 0 || T < 0) return 1;
  field_t f = make_field(kind, d, M, centres, phase, gamma, w, bias);
  double* rows = gw ? (double*)calloc((size_t)N * (size_t)(M > 0 ? M : 1), sizeof(double)) : NULL;
  double* brow = gbias ? (double*)calloc((size_t)(N > 0 ? N : 1), sizeof(double)) : NULL;
  if ((gw && !rows) || (gbias && !brow)) { free(rows); free(brow); return 2; }
  vjp_ctx c = { &f, x0, N, T, eta, gT, g0, rows, brow };
  parallel_range(N, vjp_range, &c);
  if (gw) {
    for (long m = 0; m < M; ++m) gw[m] = 0.0;
    for (long n = 0; n < N; ++n)
      for (long m = 0; m < M; ++m) gw[m] += rows[n * M + m];
  }
  if (gbias) {
    *gbias = 0.0;
    for (long n = 0; n < N; ++n) *gbias += brow[n];
  }
  free(rows); free(brow);
  return 0;
}

/* ------------------------------------------------------------------ */
/* log-det of the Jacobian of the T-step map                            */
/* ------------------------------------------------------------------ */
/* log|det A| and sign(det A) of a d x d matrix by Gaussian elimination with
 * partial pivoting (A is overwritten). */
static double logabsdet(double* a, int d, int* sign) {
  int sg = 1;
  double acc = 0.0;
  for (int k = 0; k < d; ++k) {
    int piv = k;
    for (int i = k + 1; i < d; ++i)
      if (fabs(a[i * d + k]) > fabs(a[piv * d + k])) piv = i;
    if (a[piv * d + k] == 0.0) { *sign = 0; return -INFINITY; }
    if (piv != k) {
      for (int j = 0; j < d; ++j) { double t = a[k * d + j]; a[k * d + j] = a[piv * d + j]; a[piv * d + j] = t; }
      sg = -sg;
    }
    double p = a[k * d + k];
    if (p < 0) sg = -sg;
    acc += log(fabs(p));
    for (int i = k + 1; i < d; ++i) {
      double l = a[i * d + k] / p;
      for (int j = k; j < d; ++j) a[i * d + j] -= l * a[k * d + j];
    }
  }
  *sign = sg;
  return acc;
}

typedef struct {
  const field_t* f; const double* x0; long N; int T; double eta;
  double* logdet; double* xT; double* min_det;
} logdet_ctx;

static void logdet_range(void* p, long lo, long hi) {
  logdet_ctx* c = (logdet_ctx*)p;
  int d = c->f->d;
  for (long n = lo; n < hi; ++n) {
    double x[MAXD], gc[MAXD], hc[MAXD * MAXD], a[MAXD * MAXD];
    double total = 0.0, mindet = INFINITY;
    for (int i = 0; i < d; ++i) x[i] = c->x0[n * d + i];
    for (int t = 0; t < c->T; ++t) {
      cost_derivs(c->f, x, gc, hc, NULL, NULL);
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) a[i * d + j] = (i == j ? 1.0 : 0.0) - c->eta * hc[i * d + j];
      int sg;
      double la = logabsdet(a, d, &sg);
      total += la;
      double det = sg * exp(la);
      if (det < mindet) mindet = det;
      for (int i = 0; i < d; ++i) x[i] = x[i] - c->eta * gc[i];
    }
    c->logdet[n] = total;
    if (c->xT) for (int i = 0; i < d; ++i) c->xT[n * d + i] = x[i];
    if (c->min_det) c->min_det[n] = mindet;
  }
}

/* logdet[n] = sum_t log|det(I - eta Hess c(x_t))|; min_det[n] = smallest
 * signed det over the steps (positive for a diffeomorphic chain). */
int orc_logdet(int kind, int d, long M, const double* centres, const double* phase, double gamma,
               const double* w, double bias, const double* x0, long N, int T, double eta,
               double* logdet, double* xT, double* min_det) {
  if (d < 1 || d > MAXD || M < 0 || N < 0 || T < 0) return 1;
  field_t f = make_field(kind, d, M, centres, phase, gamma, w, bias);
  logdet_ctx c = { &f, x0, N, T, eta, logdet, xT, min_det };
  parallel_range(N, logdet_range, &c);
  return 0;
}

/* ------------------------------------------------------------------ */
/* certified Lipschitz bound of grad c                                 */
/* ------------------------------------------------------------------ */
/* |Hess c| <= |sigma'| |Hess s| + |sigma''| |grad s|^2
 *          <= (1/4) |Hess s| + (1/(6 sqrt 3)) |grad s|^2,
 * the two constants being the maxima of sigma(1-sigma) and
 * |sigma(1-sigma)(1-2 sigma)|.  For RBF features, with r = |x - mu_m|:
 *   |grad phi_m| = h1(r) = 2 gamma r exp(-gamma r^2),
 *   |Hess phi_m|_2 = h2(r) = max(2 gamma, |4 gamma^2 r^2 - 2 gamma|) exp(-gamma r^2).
 * Over an axis-aligned cell, r lies in [rmin, rmax] and each h is replaced by
 * its maximum over that interval; the bound is the maximum over cells. */
static double h1(double gamma, double r) { return 2.0 * gamma * r * exp(-gamma * r * r); }
static double h2(double gamma, double r) {
  double a = fabs(4.0 * gamma * gamma * r * r - 2.0 * gamma);
  double b = 2.0 * gamma;
  return (a > b ? a : b) * exp(-gamma * r * r);
}
/* h1 rises on [0, 1/sqrt(2 gamma)] and falls after. */
static double h1_max(double gamma, double rmin, double rmax) {
  double rs = 1.0 / sqrt(2.0 * gamma);
  if (rmax <= rs) return h1(gamma, rmax);
  if (rmin >= rs) return h1(gamma, rmin);
  return h1(gamma, rs);
}
/* In u = gamma r^2, h2 = 2 gamma e^{-u} max(1, |2u - 1|) falls on [0,1], rises
 * on [1, 3/2] and falls after; its only interior maximum is at u = 3/2. */
static double h2_max(double gamma, double rmin, double rmax) {
  double a = h2(gamma, rmin), b = h2(gamma, rmax);
  double m = a > b ? a : b;
  double rpk = sqrt(1.5 / gamma);
  if (rmin <= rpk && rpk <= rmax) {
    double c = h2(gamma, rpk);
    if (c > m) m = c;
  }
  return m;
}

typedef struct {
  const double* centres; const double* w; long M; int d; double gamma;
  const double* lo; const double* hi; int cells; long ncells;
  double* cellL; double* cellG;
} lip_ctx;

static void lip_range(void* p, long clo, long chi) {
  lip_ctx* c = (lip_ctx*)p;
  int d = c->d;
  for (long cell = clo; cell < chi; ++cell) {
    double blo[MAXD], bhi[MAXD];
    long rem = cell;
    for (int i = 0; i < d; ++i) {
      long k = rem % c->cells; rem /= c->cells;
      double wdt = (c->hi[i] - c->lo[i]) / c->cells;
      blo[i] = c->lo[i] + wdt * k;
      bhi[i] = (k == c->cells - 1) ? c->hi[i] : c->lo[i] + wdt * (k + 1);
    }
    double sum_h1 = 0.0, sum_h2 = 0.0;
    for (long m = 0; m < c->M; ++m) {
      const double* mu = c->centres + m * d;
      double dmin2 = 0.0, dmax2 = 0.0;
      for (int i = 0; i < d; ++i) {
        double near = mu[i] < blo[i] ? blo[i] : (mu[i] > bhi[i] ? bhi[i] : mu[i]);
        double far = fabs(mu[i] - blo[i]) > fabs(mu[i] - bhi[i]) ? blo[i] : bhi[i];
        dmin2 += (mu[i] - near) * (mu[i] - near);
        dmax2 += (mu[i] - far) * (mu[i] - far);
      }
      double rmin = sqrt(dmin2), rmax = sqrt(dmax2);
      sum_h1 += fabs(c->w[m]) * h1_max(c->gamma, rmin, rmax);
      sum_h2 += fabs(c->w[m]) * h2_max(c->gamma, rmin, rmax);
    }
    c->cellL[cell] = 0.25 * sum_h2 + sum_h1 * sum_h1 / (6.0 * sqrt(3.0));
    c->cellG[cell] = 0.25 * sum_h1;
  }
}

/* RBF: L >= sup |Hess c|_2 and G >= sup |grad c|_2 over the box [lo, hi],
 * from cells^d cells. */
int orc_lipschitz_rbf(int d, long M, const double* centres, double gamma, const double* w,
                      const double* lo, const double* hi, int cells, double* L, double* G) {
  if (d < 1 || d > MAXD || M < 0 || cells < 1) return 1;
  long ncells = 1;
  for (int i = 0; i < d; ++i) ncells *= cells;
  double* cl = (double*)malloc(sizeof(double) * ncells);
  double* cg = (double*)malloc(sizeof(double) * ncells);
  lip_ctx c = { centres, w, M, d, gamma, lo, hi, cells, ncells, cl, cg };
  parallel_range(ncells, lip_range, &c);
  double bl = 0.0, bg = 0.0;
  for (long i = 0; i < ncells; ++i) { if (cl[i] > bl) bl = cl[i]; if (cg[i] > bg) bg = cg[i]; }
  free(cl); free(cg);
  *L = bl; *G = bg;
  return 0;
}

/* RFF: |grad phi_m| <= |omega_m|, |Hess phi_m|_2 <= |omega_m|^2 everywhere. */
int orc_lipschitz_rff(int d, long M, const double* omega, const double* w, double* L, double* G) {
  if (d < 1 || d > MAXD || M < 0) return 1;
  double s1 = 0.0, s2 = 0.0;
  for (long m = 0; m < M; ++m) {
    double n2 = 0.0;
    for (int i = 0; i < d; ++i) n2 += omega[m * d + i] * omega[m * d + i];
    s1 += fabs(w[m]) * sqrt(n2);
    s2 += fabs(w[m]) * n2;
  }
  *L = 0.25 * s2 + s1 * s1 / (6.0 * sqrt(3.0));
  *G = 0.25 * s1;
  return 0;
}

/* ------------------------------------------------------------------ */
/* occupancy fit: BCE + (l2/2)|w|^2 by Nesterov gradient descent        */
/* ------------------------------------------------------------------ */
typedef struct {
  const field_t* f; const double* X; const uint8_t* y; long n;
  const double* vin; double vbias; double* out_n;   /* per sample */
  const double* r; double* out_m;                    /* per centre */
} fit_ctx;

/* out_n[i] = sum_m v_m phi_m(x_i) + vbias */
static void fit_forward_range(void* p, long lo, long hi) {
  fit_ctx* c = (fit_ctx*)p;
  int d = c->f->d;
  for (long i = lo; i < hi; ++i) {
    double acc = c->vbias;
    for (long m = 0; m < c->f->M; ++m) acc += c->vin[m] * feature(c->f, m, c->X + i * d, NULL, NULL);
    c->out_n[i] = acc;
  }
}
/* out_m[m] = sum_i r_i phi_m(x_i) */
static void fit_backward_range(void* p, long lo, long hi) {
  fit_ctx* c = (fit_ctx*)p;
  int d = c->f->d;
  for (long m = lo; m < hi; ++m) {
    double acc = 0.0;
    for (long i = 0; i < c->n; ++i) acc += c->r[i] * feature(c->f, m, c->X + i * d, NULL, NULL);
    c->out_m[m] = acc;
  }
}

static double softplus(double a) { return a > 0 ? a + log1p(exp(-a)) : log1p(exp(a)); }
static double sigmoid(double a) { double s3[3]; orc_sigmoid3(a, s3); return s3[0]; }

/* mean BCE + (l2/2)|w|^2 at (w, b); gw (M), gb receive its gradient when non-NULL */
static double fit_objective(const field_t* f, const double* X, const uint8_t* y, long n, double l2,
                            const double* w, double b, double* logits, double* r, double* gw, double* gb) {
  fit_ctx c; memset(&c, 0, sizeof c);
  c.f = f; c.X = X; c.y = y; c.n = n; c.vin = w; c.vbias = b; c.out_n = logits;
  parallel_range_sized(n, (double)f->M, fit_forward_range, &c);
  double loss = 0.0, rsum = 0.0;
  for (long i = 0; i < n; ++i) {
    loss += softplus(logits[i]) - (y[i] ? logits[i] : 0.0);
    r[i] = sigmoid(logits[i]) - (y[i] ? 1.0 : 0.0);
    rsum += r[i];
  }
  double reg = 0.0;
  for (long m = 0; m < f->M; ++m) reg += w[m] * w[m];
  loss = loss / n + 0.5 * l2 * reg;
  if (gw) {
    c.r = r; c.out_m = gw;
    parallel_range_sized(f->M, (double)n, fit_backward_range, &c);
    for (long m = 0; m < f->M; ++m) gw[m] = gw[m] / n + l2 * w[m];
  }
  if (gb) *gb = rsum / n;
  return loss;
}

/* Step size: lambda_hat = largest eigenvalue of (1/n) [Phi 1]^T [Phi 1] by
 * `power_iters` power iterations from the normalised all-ones vector; the
 * logistic loss has curvature at most lambda_hat / 4 (+ l2), so the step is
 * alpha = 1 / (lambda_hat / 4 + l2).  Then `iters` Nesterov iterations from
 * w = 0, b = 0:  v = w_k + (k-1)/(k+2) (w_k - w_{k-1}),  w_{k+1} = v - alpha grad(v). */
int orc_fit(int kind, int d, long M, const double* centres, const double* phase, double gamma,
            const double* X, const uint8_t* y, long n, double l2, int power_iters, int iters,
            double* w_out, double* bias_out, double* loss_out, double* alpha_out) {
  if (d < 1 || d > MAXD || M < 1 || n < 1 || iters < 0 || power_iters < 1) return 1;
  field_t f = make_field(kind, d, M, centres, phase, gamma, NULL, 0.0);
  double* v = (double*)malloc(sizeof(double) * M);
  double* av = (double*)malloc(sizeof(double) * M);
  double* tn = (double*)malloc(sizeof(double) * n);
  double* r = (double*)malloc(sizeof(double) * n);
  double* w = (double*)calloc(M, sizeof(double));
  double* wprev = (double*)calloc(M, sizeof(double));
  double* vw = (double*)malloc(sizeof(double) * M);
  double* g = (double*)malloc(sizeof(double) * M);

  /* power iteration on A = (1/n) [Phi 1]^T [Phi 1]; v = (v_w, v_b) */
  double vb = 1.0 / sqrt((double)(M + 1)), lam = 0.0;
  for (long m = 0; m < M; ++m) v[m] = 1.0 / sqrt((double)(M + 1));
  for (int it = 0; it < power_iters; ++it) {
    fit_ctx c; memset(&c, 0, sizeof c);
    c.f = &f; c.X = X; c.y = y; c.n = n; c.vin = v; c.vbias = vb; c.out_n = tn;
    parallel_range_sized(n, (double)M, fit_forward_range, &c);   /* tn = [Phi 1] v */
    c.r = tn; c.out_m = av;
    parallel_range_sized(M, (double)n, fit_backward_range, &c);  /* av = Phi^T tn */
    double avb = 0.0;                                  /* bias row: 1^T tn */
    for (long i = 0; i < n; ++i) avb += tn[i];
    avb /= n;
    for (long m = 0; m < M; ++m) av[m] /= n;
    double nrm = avb * avb;
    for (long m = 0; m < M; ++m) nrm += av[m] * av[m];
    nrm = sqrt(nrm);
    lam = nrm;                                         /* |A v| with |v| = 1 */
    if (nrm == 0.0) break;
    for (long m = 0; m < M; ++m) v[m] = av[m] / nrm;
    vb = avb / nrm;
  }
  double alpha = 1.0 / (0.25 * lam + l2);

  double b = 0.0, bprev = 0.0, gb = 0.0;
  for (int k = 1; k <= iters; ++k) {
    double beta = (double)(k - 1) / (double)(k + 2);
    for (long m = 0; m < M; ++m) vw[m] = w[m] + beta * (w[m] - wprev[m]);
    double vbias = b + beta * (b - bprev);
    fit_objective(&f, X, y, n, l2, vw, vbias, tn, r, g, &gb);
    for (long m = 0; m < M; ++m) { wprev[m] = w[m]; w[m] = vw[m] - alpha * g[m]; }
    bprev = b; b = vbias - alpha * gb;
  }
  double loss = fit_objective(&f, X, y, n, l2, w, b, tn, r, NULL, NULL);
  for (long m = 0; m < M; ++m) w_out[m] = w[m];
  *bias_out = b;
  *loss_out = loss;
  if (alpha_out) *alpha_out = alpha;
  free(v); free(av); free(tn); free(r); free(w); free(wprev); free(vw); free(g);
  return 0;
}

/* loss and gradient of the fit objective at a given (w, b) -- for tests */
int orc_fit_objective(int kind, int d, long M, const double* centres, const double* phase, double gamma,
                      const double* X, const uint8_t* y, long n, double l2, const double* w, double b,
                      double* loss, double* gw, double* gb) {
  if (d < 1 || d > MAXD || M < 1 || n < 1) return 1;
  field_t f = make_field(kind, d, M, centres, phase, gamma, NULL, 0.0);
  double* tn = (double*)malloc(sizeof(double) * n);
  double* r = (double*)malloc(sizeof(double) * n);
  *loss = fit_objective(&f, X, y, n, l2, w, b, tn, r, gw, gb);
  free(tn); free(r);
  return 0;
}

/* ------------------------------------------------------------------ */
/* ground-truth occupancy from axis-aligned boxes                      */
/* ------------------------------------------------------------------ */
/* label[i] = 1 iff some box k has lo_k <= x_i <= hi_k on every axis (closed
 * boxes).  boxes: nb x 2d floats (lo_0..lo_{d-1}, hi_0..hi_{d-1}); the
 * comparisons are done on the float values themselves. */
int orc_box_labels(int d, const float* boxes, long nb, const float* x, long n, uint8_t* label) {
  if (d < 1 || d > MAXD || nb < 0 || n < 0) return 1;
  for (long i = 0; i < n; ++i) {
    int inside_any = 0;
    for (long k = 0; k < nb && !inside_any; ++k) {
      int inside = 1;
      for (int j = 0; j < d; ++j) {
        float v = x[i * d + j];
        if (!(boxes[k * 2 * d + j] <= v && v <= boxes[k * 2 * d + d + j])) inside = 0;
      }
      inside_any = inside;
    }
    label[i] = (uint8_t)inside_any;
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* surrogate MLP (no counterpart in the paper)                          */
/* ------------------------------------------------------------------ */
/* nl linear layers with widths[0..nl]; W_l is widths[l+1] x widths[l]
 * row-major, all layers concatenated in W; biases likewise in B.
 * a_0 = x;  z_l = W_l a_{l-1} + b_l;  a_l = silu(z_l) = z_l sigmoid(z_l)
 * for every layer but the last, whose z is the output. */
static double silu(double z) { return z * sigmoid(z); }
static double silu_grad(double z) { double s = sigmoid(z); return s * (1.0 + z * (1.0 - s)); }

static void mlp_forward_one(int nl, const int* widths, const double* W, const double* B, const double* x,
                            double** z, double** a) {
  long ow = 0, ob = 0;
  for (int i = 0; i < widths[0]; ++i) a[0][i] = x[i];
  for (int l = 0; l < nl; ++l) {
    int in = widths[l], out = widths[l + 1];
    for (int o = 0; o < out; ++o) {
      double acc = B[ob + o];
      for (int i = 0; i < in; ++i) acc += W[ow + (long)o * in + i] * a[l][i];
      z[l + 1][o] = acc;
      a[l + 1][o] = (l + 1 < nl) ? silu(acc) : acc;
    }
    ow += (long)in * out; ob += out;
  }
}

static double** alloc_layers(int nl, const int* widths) {
  double** p = (double**)malloc(sizeof(double*) * (nl + 1));
  for (int l = 0; l <= nl; ++l) p[l] = (double*)calloc(widths[l], sizeof(double));
  return p;
}
static void free_layers(double** p, int nl) { for (int l = 0; l <= nl; ++l) free(p[l]); free(p); }

int orc_mlp_forward(int nl, const int* widths, const double* W, const double* B, const double* X, long n,
                    double* out, double* unused) {
  (void)unused;
  if (nl < 1 || n < 0) return 1;
  double** z = alloc_layers(nl, widths);
  double** a = alloc_layers(nl, widths);
  for (long s = 0; s < n; ++s) {
    mlp_forward_one(nl, widths, W, B, X + s * widths[0], z, a);
    for (int o = 0; o < widths[nl]; ++o) out[s * widths[nl] + o] = a[nl][o];
  }
  free_layers(z, nl); free_layers(a, nl);
  return 0;
}

/* loss = (1/(n * d_out)) sum (f(x) - y)^2 and its gradient w.r.t. every W, B */
int orc_mlp_loss_backward(int nl, const int* widths, const double* W, const double* B, const double* X,
                          const double* Y, long n, double* loss, double* gW, double* gB) {
  if (nl < 1 || n < 1) return 1;
  long nw = 0, nb = 0;
  for (int l = 0; l < nl; ++l) { nw += (long)widths[l] * widths[l + 1]; nb += widths[l + 1]; }
  for (long i = 0; i < nw; ++i) gW[i] = 0.0;
  for (long i = 0; i < nb; ++i) gB[i] = 0.0;
  double** z = alloc_layers(nl, widths);
  double** a = alloc_layers(nl, widths);
  double** dz = alloc_layers(nl, widths);
  long* offw = (long*)malloc(sizeof(long) * nl);
  long* offb = (long*)malloc(sizeof(long) * nl);
  { long ow = 0, ob = 0;
    for (int l = 0; l < nl; ++l) { offw[l] = ow; offb[l] = ob; ow += (long)widths[l] * widths[l + 1]; ob += widths[l + 1]; } }
  int dout = widths[nl];
  double total = 0.0, scale = 1.0 / ((double)n * dout);
  for (long s = 0; s < n; ++s) {
    mlp_forward_one(nl, widths, W, B, X + s * widths[0], z, a);
    for (int o = 0; o < dout; ++o) {
      double r = a[nl][o] - Y[s * dout + o];
      total += r * r;
      dz[nl][o] = 2.0 * r * scale;
    }
    for (int l = nl - 1; l >= 0; --l) {
      int in = widths[l], out = widths[l + 1];
      /* dz[l+1] holds dLoss/dz_{l+1} */
      for (int o = 0; o < out; ++o) {
        gB[offb[l] + o] += dz[l + 1][o];
        for (int i = 0; i < in; ++i) gW[offw[l] + (long)o * in + i] += dz[l + 1][o] * a[l][i];
      }
      if (l > 0)
        for (int i = 0; i < in; ++i) {
          double acc = 0.0;
          for (int o = 0; o < out; ++o) acc += W[offw[l] + (long)o * in + i] * dz[l + 1][o];
          dz[l][i] = acc * silu_grad(z[l][i]);
        }
    }
  }
  *loss = total * scale;
  free_layers(z, nl); free_layers(a, nl); free_layers(dz, nl); free(offw); free(offb);
  return 0;
}

/* Fourier encoding of the surrogate's normalised input u (n x 3):
 * out (n x (3 + 6 nf)) = [u_0..u_2, then for k = 0..nf-1:
 * sin(2^k pi u_0..u_2), cos(2^k pi u_0..u_2)]. */
int orc_mlp_encode(const double* u, long n, int nf, double* out) {
  if (n < 0 || nf < 0) return 1;
  const int w = 3 + 6 * nf;
  const double pi = 3.14159265358979323846;
  for (long s = 0; s < n; ++s) {
    for (int j = 0; j < 3; ++j) out[s * w + j] = u[s * 3 + j];
    double f = pi;
    for (int k = 0; k < nf; ++k) {
      for (int j = 0; j < 3; ++j) {
        out[s * w + 3 + 6 * k + j] = sin(f * u[s * 3 + j]);
        out[s * w + 3 + 6 * k + 3 + j] = cos(f * u[s * 3 + j]);
      }
      f *= 2.0;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* The paper's own occupancy network (Sec. 3.1): a fully connected       */
/* network with tanh between the hidden layers and a sigmoid output.    */
/* Two hidden layers of width H:                                        */
/*   a1 = W1 x + b1, h1 = tanh(a1), a2 = W2 h1 + b2, h2 = tanh(a2),     */
/*   s = w3 . h2 + b3,  c = sigma(s).                                   */
/* W1 is H x d and W2 is H x H, row-major (row = output unit).          */
/* ------------------------------------------------------------------ */
#define TNET_HMAX 128

typedef struct {
  int d, H;
  const double *W1, *b1, *W2, *b2, *w3;
  double b3;
} tnet_t;

/* s, grad s and (optional) Hess s at x by the chain rule:
 *   v2 = w3 (.) tanh'(a2),  u1 = W2^T v2,  g1 = u1 (.) tanh'(a1),  grad s = W1^T g1,
 *   Hess s = W1^T diag(u1 (.) tanh''(a1)) W1 + P^T diag(w3 (.) tanh''(a2)) P,
 *   P = W2 diag(tanh'(a1)) W1,
 * with tanh' = 1 - tanh^2 and tanh'' = -2 tanh (1 - tanh^2). */
static double tnet_logit(const tnet_t* n, const double* x, double* gs, double* hs) {
  const int d = n->d, H = n->H;
  double h1[TNET_HMAX], t1[TNET_HMAX], h2[TNET_HMAX], t2[TNET_HMAX], u1[TNET_HMAX];
  for (int i = 0; i < H; ++i) {
    double a = n->b1[i];
    for (int k = 0; k < d; ++k) a += n->W1[i * d + k] * x[k];
    h1[i] = tanh(a);
    t1[i] = 1.0 - h1[i] * h1[i];
  }
  double s = n->b3;
  for (int i = 0; i < H; ++i) {
    double a = n->b2[i];
    for (int j = 0; j < H; ++j) a += n->W2[i * H + j] * h1[j];
    h2[i] = tanh(a);
    t2[i] = 1.0 - h2[i] * h2[i];
    s += n->w3[i] * h2[i];
  }
  for (int j = 0; j < H; ++j) {
    double u = 0.0;
    for (int i = 0; i < H; ++i) u += n->W2[i * H + j] * n->w3[i] * t2[i];
    u1[j] = u;
  }
  for (int k = 0; k < d; ++k) {
    double g = 0.0;
    for (int j = 0; j < H; ++j) g += n->W1[j * d + k] * u1[j] * t1[j];
    gs[k] = g;
  }
  if (hs) {
    double P[TNET_HMAX * MAXD];
    for (int i = 0; i < H; ++i)
      for (int k = 0; k < d; ++k) {
        double p = 0.0;
        for (int j = 0; j < H; ++j) p += n->W2[i * H + j] * t1[j] * n->W1[j * d + k];
        P[i * d + k] = p;
      }
    for (int k = 0; k < d; ++k)
      for (int l = 0; l < d; ++l) {
        double acc = 0.0;
        for (int j = 0; j < H; ++j) acc += n->W1[j * d + k] * (u1[j] * (-2.0 * h1[j] * t1[j])) * n->W1[j * d + l];
        for (int i = 0; i < H; ++i) acc += P[i * d + k] * (n->w3[i] * (-2.0 * h2[i] * t2[i])) * P[i * d + l];
        hs[k * d + l] = acc;
      }
  }
  return s;
}

static double tnet_cost(const tnet_t* n, const double* x, double* gc, double* hc, double* s_out) {
  const int d = n->d;
  double gs[MAXD], hs[MAXD * MAXD], sg[3];
  double s = tnet_logit(n, x, gs, hc ? hs : NULL);
  orc_sigmoid3(s, sg);
  for (int i = 0; i < d; ++i) gc[i] = sg[1] * gs[i];
  if (hc)
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) hc[i * d + j] = sg[1] * hs[i * d + j] + sg[2] * gs[i] * gs[j];
  if (s_out) *s_out = s;
  return sg[0];
}

static int tnet_ok(int d, int H) { return d >= 1 && d <= MAXD && H >= 1 && H <= TNET_HMAX; }

typedef struct { const tnet_t* n; const double* X; double *c, *s, *gc, *hc; } tnet_eval_ctx;
static void tnet_eval_range(void* p, long lo, long hi) {
  tnet_eval_ctx* q = (tnet_eval_ctx*)p;
  const int d = q->n->d;
  for (long i = lo; i < hi; ++i) {
    double s;
    double c = tnet_cost(q->n, q->X + i * d, q->gc + i * d, q->hc ? q->hc + i * d * d : NULL, &s);
    if (q->c) q->c[i] = c;
    if (q->s) q->s[i] = s;
  }
}

int orc_tnet_eval(int d, int H, const double* W1, const double* b1, const double* W2, const double* b2,
                  const double* w3, double b3, const double* X, long n, double* c, double* s, double* gc,
                  double* hc) {
  if (!tnet_ok(d, H) || n < 0) return 1;
  tnet_t net = {d, H, W1, b1, W2, b2, w3, b3};
  tnet_eval_ctx q = {&net, X, c, s, gc, hc};
  parallel_range(n, tnet_eval_range, &q);
  return 0;
}

/* Eq. (1) by Euler's method with c the network's occupancy. */
typedef struct { const tnet_t* n; const double* X0; int T; double eta; double* XT; } tnet_morph_ctx;
static void tnet_morph_range(void* p, long lo, long hi) {
  tnet_morph_ctx* q = (tnet_morph_ctx*)p;
  const int d = q->n->d;
  for (long i = lo; i < hi; ++i) {
    double x[MAXD], g[MAXD];
    for (int k = 0; k < d; ++k) x[k] = q->X0[i * d + k];
    for (int t = 0; t < q->T; ++t) {
      tnet_cost(q->n, x, g, NULL, NULL);
      for (int k = 0; k < d; ++k) x[k] -= q->eta * g[k];
    }
    for (int k = 0; k < d; ++k) q->XT[i * d + k] = x[k];
  }
}

int orc_tnet_morph(int d, int H, const double* W1, const double* b1, const double* W2, const double* b2,
                   const double* w3, double b3, const double* X0, long n, int T, double eta, double* XT) {
  if (!tnet_ok(d, H) || n < 0 || T < 0) return 1;
  tnet_t net = {d, H, W1, b1, W2, b2, w3, b3};
  tnet_morph_ctx q = {&net, X0, T, eta, XT};
  parallel_range(n, tnet_morph_range, &q);
  return 0;
}

/* Largest eigenvalue of a symmetric n x n matrix (cyclic Jacobi rotations
 * until the off-diagonal mass is negligible); A is overwritten. */
static double sym_max_eigenvalue(double* A, int n) {
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += A[i * n + j] * A[i * n + j];
        if (i != j) off += A[i * n + j] * A[i * n + j];
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (apq == 0.0) continue;
        const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < n; ++k) {  /* columns p, q */
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = cs * akp - sn * akq;
          A[k * n + q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < n; ++k) {  /* rows p, q */
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = cs * apk - sn * aqk;
          A[q * n + k] = sn * apk + cs * aqk;
        }
      }
  }
  double m = A[0];
  for (int i = 1; i < n; ++i) m = A[i * n + i] > m ? A[i * n + i] : m;
  return m;
}

/* spectral norm of the r x k matrix W from the largest eigenvalue of W^T W,
 * with a relative margin for the eigenvalue's rounding */
static double spectral_norm(const double* W, int r, int k) {
  double* G = (double*)calloc((size_t)k * k, sizeof(double));
  for (int a = 0; a < k; ++a)
    for (int b = 0; b < k; ++b) {
      double acc = 0.0;
      for (int i = 0; i < r; ++i) acc += W[i * k + a] * W[i * k + b];
      G[a * k + b] = acc;
    }
  double lam = sym_max_eigenvalue(G, k);
  free(G);
  return sqrt(fmax(lam, 0.0) * (1.0 + 1e-12));
}

/* Certified bounds over all of R^d (|tanh'| <= 1, |tanh''| <= 4/(3 sqrt 3)):
 *   |grad s| <= G = |W1| |W2| |w3|_2,
 *   |Hess s| <= |W1|^2 (k max_j sum_i |W2_ij| |w3_i| + k |W2|^2 max_i |w3_i|),
 *   L = |Hess s| / 4 + G^2 / (6 sqrt 3)   (the sigmoid's |sigma'| <= 1/4, |sigma''| <= 1/(6 sqrt 3)),
 * with |.| the spectral norm. */
int orc_tnet_lipschitz(int d, int H, const double* W1, const double* W2, const double* w3, double* L, double* G) {
  if (!tnet_ok(d, H)) return 1;
  const double kappa = 4.0 / (3.0 * sqrt(3.0));
  const double n1 = spectral_norm(W1, H, d), n2 = spectral_norm(W2, H, H);
  double w3n = 0.0, w3max = 0.0, colmax = 0.0;
  for (int i = 0; i < H; ++i) {
    w3n += w3[i] * w3[i];
    w3max = fmax(w3max, fabs(w3[i]));
  }
  for (int j = 0; j < H; ++j) {
    double col = 0.0;
    for (int i = 0; i < H; ++i) col += fabs(W2[i * H + j]) * fabs(w3[i]);
    colmax = fmax(colmax, col);
  }
  const double g = n1 * n2 * sqrt(w3n);
  const double hs = n1 * n1 * (kappa * colmax + kappa * n2 * n2 * w3max);
  *G = g;
  *L = 0.25 * hs + g * g / (6.0 * sqrt(3.0));
  return 0;
}

/* ------------------------------------------------------------------ */
/* Configuration space (Sec. 3.2, "Bringing Diffeomorphisms into        */
/* Configuration Space", Eq. (3)).  A planar serial chain with n         */
/* revolute joints: joint angles q, absolute link angles                */
/* theta_k = q_1 + .. + q_k, joint positions o_1 = base,                */
/* o_{k+1} = o_k + l_k (cos theta_k, sin theta_k).  Link k carries p     */
/* body points psi = o_k + (r/p) l_k (cos theta_k, sin theta_k),         */
/* r = 1..p, so b = n p.  The cost on the body points is                 */
/* f_c(q) = sum_i c(psi_i(q)); its C-space gradient pulls the            */
/* task-space gradients back through the kinematic Jacobians,            */
/* grad_q f_c = sum_i J_i^T grad_x c(psi_i(q))  (Eq. (3) with the        */
/* transpose the chain rule needs), where column j of J_i is             */
/* z x (psi_i - o_j) for the joints j that move point i, else 0.         */
/* ------------------------------------------------------------------ */
#define CHAIN_MAX 16

typedef struct {
  int n, p;
  double base[2];
  const double* len;
} chain_t;

/* joint positions o[0..n] (o[n] the tip) and body points psi[0..n p) */
static void chain_fk(const chain_t* ch, const double* q, double* o, double* psi) {
  double th = 0.0;
  o[0] = ch->base[0];
  o[1] = ch->base[1];
  for (int k = 0; k < ch->n; ++k) {
    th += q[k];
    const double cx = cos(th), sy = sin(th);
    for (int r = 1; r <= ch->p; ++r) {
      const double f = (double)r / ch->p;
      psi[2 * (k * ch->p + r - 1)] = o[2 * k] + f * ch->len[k] * cx;
      psi[2 * (k * ch->p + r - 1) + 1] = o[2 * k + 1] + f * ch->len[k] * sy;
    }
    o[2 * (k + 1)] = o[2 * k] + ch->len[k] * cx;
    o[2 * (k + 1) + 1] = o[2 * k + 1] + ch->len[k] * sy;
  }
}

/* f_c(q) and grad_q f_c by Eq. (3) */
static double chain_cost(const field_t* f, const chain_t* ch, const double* q, double* gq) {
  double o[2 * (CHAIN_MAX + 1)], psi[2 * CHAIN_MAX * 8];
  chain_fk(ch, q, o, psi);
  for (int j = 0; j < ch->n; ++j) gq[j] = 0.0;
  double fc = 0.0;
  for (int i = 0; i < ch->n * ch->p; ++i) {
    const int link = i / ch->p;
    double gx[2];
    fc += cost_derivs(f, psi + 2 * i, gx, NULL, NULL, NULL);
    for (int j = 0; j <= link; ++j) {
      const double vx = psi[2 * i] - o[2 * j], vy = psi[2 * i + 1] - o[2 * j + 1];
      gq[j] += -vy * gx[0] + vx * gx[1];     /* (z x v) . g */
    }
  }
  return fc;
}

static int chain_ok(int n, int p) { return n >= 1 && n <= CHAIN_MAX && p >= 1 && p <= 8; }

typedef struct { const field_t* f; const chain_t* ch; const double* Q; double *fc, *gq; } cs_eval_ctx;
static void cs_eval_range(void* p, long lo, long hi) {
  cs_eval_ctx* c = (cs_eval_ctx*)p;
  const int n = c->ch->n;
  for (long i = lo; i < hi; ++i) {
    const double v = chain_cost(c->f, c->ch, c->Q + i * n, c->gq + i * n);
    if (c->fc) c->fc[i] = v;
  }
}

int orc_cspace_eval(int kind, int d, long M, const double* centres, const double* phase, double gamma,
                    const double* w, double bias, int n, int p, const double* base, const double* len,
                    const double* Q, long N, double* fc, double* gq) {
  if (d != 2 || !chain_ok(n, p) || N < 0) return 1;
  field_t f = make_field(kind, d, M, centres, phase, gamma, w, bias);
  chain_t ch = {n, p, {base[0], base[1]}, len};
  cs_eval_ctx c = {&f, &ch, Q, fc, gq};
  parallel_range(N, cs_eval_range, &c);
  return 0;
}

/* the body points themselves (for tests of the forward kinematics) */
int orc_cspace_points(int n, int p, const double* base, const double* len, const double* Q, long N, double* P) {
  if (!chain_ok(n, p) || N < 0) return 1;
  chain_t ch = {n, p, {base[0], base[1]}, len};
  double o[2 * (CHAIN_MAX + 1)];
  for (long i = 0; i < N; ++i) chain_fk(&ch, Q + i * n, o, P + i * 2 * n * p);
  return 0;
}

/* Eq. (1) in C-space: q_{t+1} = q_t - eta grad_q f_c(q_t) */
typedef struct { const field_t* f; const chain_t* ch; const double* Q0; int T; double eta; double* QT; } cs_morph_ctx;
static void cs_morph_range(void* p, long lo, long hi) {
  cs_morph_ctx* c = (cs_morph_ctx*)p;
  const int n = c->ch->n;
  for (long i = lo; i < hi; ++i) {
    double q[CHAIN_MAX], g[CHAIN_MAX];
    for (int j = 0; j < n; ++j) q[j] = c->Q0[i * n + j];
    for (int t = 0; t < c->T; ++t) {
      chain_cost(c->f, c->ch, q, g);
      for (int j = 0; j < n; ++j) q[j] -= c->eta * g[j];
    }
    for (int j = 0; j < n; ++j) c->QT[i * n + j] = q[j];
  }
}

int orc_cspace_morph(int kind, int d, long M, const double* centres, const double* phase, double gamma,
                     const double* w, double bias, int n, int p, const double* base, const double* len,
                     const double* Q0, long N, int T, double eta, double* QT) {
  if (d != 2 || !chain_ok(n, p) || N < 0 || T < 0) return 1;
  field_t f = make_field(kind, d, M, centres, phase, gamma, w, bias);
  chain_t ch = {n, p, {base[0], base[1]}, len};
  cs_morph_ctx c = {&f, &ch, Q0, T, eta, QT};
  parallel_range(N, cs_morph_range, &c);
  return 0;
}

/* Certified bound on sup |Hess_q f_c|_2 from bounds Lx >= sup |Hess c|_2 and
 * Gx >= sup |grad c| in the task space:
 *   Hess_q f_c = sum_i [ J_i^T Hess c J_i + sum_a (dc/dx_a) Hess_q psi_{i,a} ],
 * |J_i|_2^2 <= sum_{j <= k} |psi_i - o_j|^2 <= sum_{j <= k} R_{j,i}^2 and the
 * entries of Hess_q psi_i (the second derivative about joints j, m is
 * z x (z x (psi_i - o_max(j,m)))) have norm <= R_{max(j,m),i}, where R_{j,i}
 * is the chain length from joint j to point i. */
int orc_cspace_lipschitz(int n, int p, const double* len, double Lx, double Gx, double* Lq) {
  if (!chain_ok(n, p)) return 1;
  double total = 0.0;
  for (int k = 0; k < n; ++k)
    for (int r = 1; r <= p; ++r) {
      double R[CHAIN_MAX];              /* R[j]: chain length from joint j to the point */
      for (int j = 0; j <= k; ++j) {
        double s = (double)r / p * len[k];
        for (int m = j; m < k; ++m) s += len[m];
        R[j] = s;
      }
      double jf = 0.0, hf = 0.0;
      for (int j = 0; j <= k; ++j) {
        jf += R[j] * R[j];
        for (int m = 0; m <= k; ++m) {
          const double rr = R[j > m ? j : m];
          hf += rr * rr;
        }
      }
      total += jf * Lx + Gx * sqrt(hf);
    }
  *Lq = total;
  return 0;
}

/* ------------------------------------------------------------------ */
/* Counter-based generator for base samples drawn on the device          */
/* (the planner's prior, Sec. 3.3): Philox4x32 with 10 rounds (Salmon,   */
/* Moraes, Dror, Shaw, SC'11), written from its published definition.    */
/* Sample i, coordinate j of batch b is word (i d + j) mod 4 of block    */
/* (i d + j) / 4 with counter (block, 0-hi, b, b-hi) and key (seed lo,    */
/* seed hi); its top 24 bits u give the coordinate fmaf(u 2^-24,         */
/* hi - lo, lo) in float32.                                              */
/* ------------------------------------------------------------------ */
static void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

int orc_philox4x32(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  philox4x32_10(ctr, key, out);
  return 0;
}

int orc_uniform_batch(uint64_t seed, uint64_t batch, long n, int d, const float* lo, const float* hi, float* x) {
  if (d < 1 || d > MAXD || n < 0) return 1;
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (long e = 0; e < n * d; ++e) {
    const uint64_t blk = (uint64_t)e / 4;
    const uint32_t ctr[4] = {(uint32_t)blk, (uint32_t)(blk >> 32), (uint32_t)batch, (uint32_t)(batch >> 32)};
    uint32_t o[4];
    philox4x32_10(ctr, key, o);
    const int j = (int)(e % d);
    const float u = (float)(o[e % 4] >> 8) * (1.0f / 16777216.0f);
    x[e] = fmaf(u, hi[j] - lo[j], lo[j]);
  }
  return 0;
}
