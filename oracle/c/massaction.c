/*
 * Plain C float64 oracle for mass-action kinetics (test infrastructure only; nothing in
 * the product path links or calls it). It computes, one trajectory at a time and one time
 * step after another, what the numpy oracle in oracle/dynamics.py, oracle/newton.py and
 * oracle/adjoint.py computes, at sizes the numpy loops cannot reach in seconds:
 *
 *   - the right-hand side g(c) of mass-action kinetics (reaction r has rate
 *     k_r c_i1 c_i2, c_i2 -> 1 when unimolecular, consumes i1, i2 and produces p1, p2);
 *   - one explicit Euler or classical RK4 step f(s) and its exact Jacobian
 *     A = df/ds by the chain rule through the stages (the step Jacobian A_t of Eq. lil_j);
 *   - d f / d k through the stages (k enters every stage);
 *   - the sequential rollout s_t = f(s_{t-1}) from s_0 (Sec. 2.1: the plain definition
 *     of the answer the parallel iteration converges to);
 *   - the adjoint of the loss by the reverse recursion of Eq. bptt / unrolled_bwds:
 *     lambda_T = g_T, lambda_{t-1} = g_{t-1} + A_t^T lambda_t (A_t at s_{t-1}),
 *     dl/dk = sum_t lambda_t^T df/dk (s_{t-1}), dl/ds_0 = A_1^T lambda_1.
 *
 * Compiled with -ffp-contract=off (round to nearest, no fused multiply-add). Every entry
 * point works on the trajectories [b_lo, b_hi) so that callers can split a batch over host
 * threads.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int d, R;
  const int32_t* topo; /* [R][4] */
  const double* k;     /* [R] */
} Net;

/* monomial of reaction r without its rate constant */
static double monomial(const Net* n, int r, const double* c) {
  const int32_t* tp = n->topo + 4 * r;
  double v = c[tp[0]];
  if (tp[1] >= 0) v *= c[tp[1]];
  return v;
}

/* out[i * stride + col] += nu_r[i] * val for the species i that reaction r changes */
static void stoich_add(const Net* n, int r, double* out, int stride, int col, double val) {
  const int32_t* tp = n->topo + 4 * r;
  out[tp[0] * stride + col] -= val;
  if (tp[1] >= 0) out[tp[1] * stride + col] -= val;
  out[tp[2] * stride + col] += val;
  if (tp[3] >= 0) out[tp[3] * stride + col] += val;
}

/* g(c) [d] */
static void rhs(const Net* n, const double* c, double* g) {
  memset(g, 0, sizeof(double) * n->d);
  for (int r = 0; r < n->R; ++r) stoich_add(n, r, g, 1, 0, n->k[r] * monomial(n, r, c));
}

/* G = dg/dc [d][d] */
static void rhs_jac(const Net* n, const double* c, double* G) {
  const int d = n->d;
  memset(G, 0, sizeof(double) * d * d);
  for (int r = 0; r < n->R; ++r) {
    const int32_t* tp = n->topo + 4 * r;
    const double kr = n->k[r];
    /* d(rate)/dc_j for the reactants j: k c_i2 for i1, k c_i1 for i2 (adds up when equal) */
    for (int j = 0; j < d; ++j) {
      double dr = 0.0;
      if (j == tp[0]) dr += tp[1] >= 0 ? kr * c[tp[1]] : kr;
      if (tp[1] >= 0 && j == tp[1]) dr += kr * c[tp[0]];
      if (dr != 0.0) stoich_add(n, r, G, d, j, dr);
    }
  }
}

/* dg/dk [d][R] */
static void rhs_dk(const Net* n, const double* c, double* P) {
  memset(P, 0, sizeof(double) * n->d * n->R);
  for (int r = 0; r < n->R; ++r) stoich_add(n, r, P, n->R, r, monomial(n, r, c));
}

/* C[m][p] = A[m][q] B[q][p] */
static void matmul(int m, int q, int p, const double* A, const double* B, double* C) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < p; ++j) {
      double acc = 0.0;
      for (int l = 0; l < q; ++l) acc += A[i * q + l] * B[l * p + j];
      C[i * p + j] = acc;
    }
}

/* the four RK4 stage points and slopes of one step from s */
typedef struct {
  double *s2, *s3, *s4, *k1, *k2, *k3, *k4;
} Stages;

static void stages(const Net* n, double h, const double* s, Stages* st) {
  const int d = n->d;
  rhs(n, s, st->k1);
  for (int i = 0; i < d; ++i) st->s2[i] = s[i] + 0.5 * h * st->k1[i];
  rhs(n, st->s2, st->k2);
  for (int i = 0; i < d; ++i) st->s3[i] = s[i] + 0.5 * h * st->k2[i];
  rhs(n, st->s3, st->k3);
  for (int i = 0; i < d; ++i) st->s4[i] = s[i] + h * st->k3[i];
  rhs(n, st->s4, st->k4);
}

/* workspace for one trajectory */
typedef struct {
  Stages st;
  double *G, *K1, *K2, *K3, *K4, *M, *P1, *P2, *P3, *P4, *Pt, *A, *Pk, *lam, *back, *gk;
} Work;

static int work_alloc(Work* w, int d, int R) {
  const size_t dd = (size_t)d * d, dr = (size_t)d * R;
  const size_t total = 7 * (size_t)d + 7 * dd + 6 * dr + 3 * (size_t)d + dd;
  double* p = (double*)calloc(total, sizeof(double));
  if (!p) return -1;
  w->st.s2 = p; p += d; w->st.s3 = p; p += d; w->st.s4 = p; p += d;
  w->st.k1 = p; p += d; w->st.k2 = p; p += d; w->st.k3 = p; p += d; w->st.k4 = p; p += d;
  w->G = p; p += dd; w->K1 = p; p += dd; w->K2 = p; p += dd; w->K3 = p; p += dd;
  w->K4 = p; p += dd; w->M = p; p += dd; w->A = p; p += dd;
  w->P1 = p; p += dr; w->P2 = p; p += dr; w->P3 = p; p += dr; w->P4 = p; p += dr;
  w->Pt = p; p += dr; w->Pk = p; p += dr;
  w->lam = p; p += d; w->back = p; p += d; w->gk = p; p += d;
  return 0;
}

static void work_free(Work* w) { free(w->st.s2); }

/* one step s -> out = f(s) */
static void step(const Net* n, int rk4, double h, const double* s, double* out, Work* w) {
  const int d = n->d;
  if (!rk4) {
    rhs(n, s, w->st.k1);
    for (int i = 0; i < d; ++i) out[i] = s[i] + h * w->st.k1[i];
    return;
  }
  stages(n, h, s, &w->st);
  for (int i = 0; i < d; ++i)
    out[i] = s[i] + (h / 6.0) * (w->st.k1[i] + 2.0 * w->st.k2[i] + 2.0 * w->st.k3[i] +
                                 w->st.k4[i]);
}

/* M = I + a K */
static void eye_plus(int d, double a, const double* K, double* M) {
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) M[i * d + j] = (i == j ? 1.0 : 0.0) + a * K[i * d + j];
}

/* A = df/ds at s (exact: RK4 stage slopes K_m = G(s_m) dS_m/ds by the chain rule) */
static void step_jac(const Net* n, int rk4, double h, const double* s, Work* w) {
  const int d = n->d;
  if (!rk4) {
    rhs_jac(n, s, w->G);
    eye_plus(d, h, w->G, w->A);
    return;
  }
  stages(n, h, s, &w->st);
  rhs_jac(n, s, w->K1);
  rhs_jac(n, w->st.s2, w->G);
  eye_plus(d, 0.5 * h, w->K1, w->M);
  matmul(d, d, d, w->G, w->M, w->K2);
  rhs_jac(n, w->st.s3, w->G);
  eye_plus(d, 0.5 * h, w->K2, w->M);
  matmul(d, d, d, w->G, w->M, w->K3);
  rhs_jac(n, w->st.s4, w->G);
  eye_plus(d, h, w->K3, w->M);
  matmul(d, d, d, w->G, w->M, w->K4);
  for (int i = 0; i < d * d; ++i)
    w->A[i] = (i % (d + 1) == 0 ? 1.0 : 0.0) +
              (h / 6.0) * (w->K1[i] + 2.0 * w->K2[i] + 2.0 * w->K3[i] + w->K4[i]);
}

/* Pk = df/dk at s [d][R]: P_m = dg/dk(s_m) + G(s_m) dS_m/dk through the stages */
static void step_dk(const Net* n, int rk4, double h, const double* s, Work* w) {
  const int d = n->d, R = n->R;
  if (!rk4) {
    rhs_dk(n, s, w->P1);
    for (int i = 0; i < d * R; ++i) w->Pk[i] = h * w->P1[i];
    return;
  }
  stages(n, h, s, &w->st);
  rhs_dk(n, s, w->P1);
  const double* pts[3] = {w->st.s2, w->st.s3, w->st.s4};
  const double cs[3] = {0.5 * h, 0.5 * h, h};
  double* prev = w->P1;
  double* outs[3] = {w->P2, w->P3, w->P4};
  for (int m = 0; m < 3; ++m) {
    rhs_dk(n, pts[m], outs[m]);
    rhs_jac(n, pts[m], w->G);
    matmul(d, d, R, w->G, prev, w->Pt);
    for (int i = 0; i < d * R; ++i) outs[m][i] += cs[m] * w->Pt[i];
    prev = outs[m];
  }
  for (int i = 0; i < d * R; ++i)
    w->Pk[i] = (h / 6.0) * (w->P1[i] + 2.0 * w->P2[i] + 2.0 * w->P3[i] + w->P4[i]);
}

static Net net_of(int d, int R, const int32_t* topo, int64_t tstride, const double* k,
                  int64_t kstride, int64_t b) {
  Net n = {d, R, topo + b * tstride, k + b * kstride};
  return n;
}

/* Sequential rollout of the trajectories b in [b_lo, b_hi): sequence b owns rows
   offsets[b] .. offsets[b+1]-1 of out [N][d] (row offsets[b] + t - 1 holds s_t). */
int ora_ma_rollout(int d, int R, int rk4, double dt, const int64_t* offsets,
                   const int32_t* topo, int64_t tstride, const double* k, int64_t kstride,
                   const double* s0, double* out, int64_t b_lo, int64_t b_hi) {
  Work w;
  if (work_alloc(&w, d, R)) return -1;
  for (int64_t b = b_lo; b < b_hi; ++b) {
    const Net n = net_of(d, R, topo, tstride, k, kstride, b);
    const double* prev = s0 + b * d;
    for (int64_t row = offsets[b]; row < offsets[b + 1]; ++row) {
      step(&n, rk4, dt, prev, out + row * d, &w);
      prev = out + row * d;
    }
  }
  work_free(&w);
  return 0;
}

/* Step Jacobians A_t = df/ds (s_{t-1}) of the rows of the trajectories in [b_lo, b_hi)
   (s_0 for the first row of each): A [N][d][d]. */
int ora_ma_step_jacobians(int d, int R, int rk4, double dt, const int64_t* offsets,
                          const int32_t* topo, int64_t tstride, const double* k,
                          int64_t kstride, const double* s0, const double* s, double* A,
                          int64_t b_lo, int64_t b_hi) {
  Work w;
  if (work_alloc(&w, d, R)) return -1;
  for (int64_t b = b_lo; b < b_hi; ++b) {
    const Net n = net_of(d, R, topo, tstride, k, kstride, b);
    for (int64_t row = offsets[b]; row < offsets[b + 1]; ++row) {
      const double* prev = row == offsets[b] ? s0 + b * d : s + (row - 1) * d;
      step_jac(&n, rk4, dt, prev, &w);
      memcpy(A + row * d * d, w.A, sizeof(double) * d * d);
    }
  }
  work_free(&w);
  return 0;
}

/* Adjoint of a loss with cotangents g [N][d] at the trajectories s [N][d]: dk [B][R]
   (row b at dk + b * R) and ds0 [B][d], for the trajectories in [b_lo, b_hi). */
int ora_ma_adjoint(int d, int R, int rk4, double dt, const int64_t* offsets,
                   const int32_t* topo, int64_t tstride, const double* k, int64_t kstride,
                   const double* s0, const double* s, const double* g, double* dk,
                   double* ds0, int64_t b_lo, int64_t b_hi) {
  Work w;
  if (work_alloc(&w, d, R)) return -1;
  for (int64_t b = b_lo; b < b_hi; ++b) {
    const Net n = net_of(d, R, topo, tstride, k, kstride, b);
    const int64_t r0 = offsets[b], r1 = offsets[b + 1];
    for (int r = 0; r < R; ++r) dk[b * R + r] = 0.0;
    for (int i = 0; i < d; ++i) ds0[b * d + i] = 0.0;
    if (r1 == r0) continue;
    for (int i = 0; i < d; ++i) w.lam[i] = g[(r1 - 1) * d + i];
    for (int64_t row = r1 - 1; row >= r0; --row) {
      const double* prev = row == r0 ? s0 + b * d : s + (row - 1) * d;
      /* dl/dk += lambda_t^T df/dk (s_{t-1}) */
      step_dk(&n, rk4, dt, prev, &w);
      for (int r = 0; r < R; ++r) {
        double acc = 0.0;
        for (int i = 0; i < d; ++i) acc += w.lam[i] * w.Pk[i * R + r];
        dk[b * R + r] += acc;
      }
      /* A_t^T lambda_t */
      step_jac(&n, rk4, dt, prev, &w);
      for (int j = 0; j < d; ++j) {
        double acc = 0.0;
        for (int i = 0; i < d; ++i) acc += w.A[i * d + j] * w.lam[i];
        w.back[j] = acc;
      }
      if (row > r0)
        for (int i = 0; i < d; ++i) w.lam[i] = w.back[i] + g[(row - 1) * d + i];
    }
    for (int i = 0; i < d; ++i) ds0[b * d + i] = w.back[i];
  }
  work_free(&w);
  return 0;
}
