// Device implementations of the built-in recurrences f_t and their Jacobians
// A_t = df_t/ds_{t-1} (Eq. lil_j). One thread evaluates one row (one time step).
//
// Mass-action kinetics are evaluated through per-sequence tensors built once per solve
// (see k_ma_setup): with L the linear (unimolecular) part and B_m[i][j] the symmetrised
// bimolecular coefficients, the rate Jacobian is G(c) = L + sum_m c_m B_m and the rate
// itself is g(c) = (L c + G(c) c) / 2 (no zeroth-order reactions exist in the registry).
// Dense register arithmetic replaces the data-dependent gathers of a per-reaction loop.
#pragma once

#include "common.cuh"

namespace deer {

template <int D>
struct Unroll { static constexpr int n = D <= 8 ? D : 1; };

// ----------------------------------------------------------------------------
// Brusselator, explicit Euler (d = 2)
// ----------------------------------------------------------------------------
template <class real>
__device__ __forceinline__ void bruss_eval(const DynView<real>& dv, int64_t seq,
                                           const real* s, real* F, real (*A)[2], bool wantA) {
  const real* p = dv.params + seq * dv.pstride;
  real a = p[0], b = p[1], dt = dv.dt;
  real x = s[0], y = s[1];
  real x2 = x * x, xy = x * y;
  F[0] = x + dt * (a - (b + real(1)) * x + x2 * y);
  F[1] = y + dt * (b * x - x2 * y);
  if (wantA) {
    A[0][0] = real(1) + dt * (real(2) * xy - (b + real(1)));
    A[0][1] = dt * x2;
    A[1][0] = dt * (b - real(2) * xy);
    A[1][1] = real(1) - dt * x2;
  }
}

// ----------------------------------------------------------------------------
// Mass action
// ----------------------------------------------------------------------------

// One RK4/Euler stage at state c: slope g = (L c + G c) / 2 with G built row by row.
// If wantA: Knew = G (I + cK * Kold)  (or Knew = G when Kold == nullptr), and
// Kacc += w * Knew.
template <class real, int D>
__device__ __forceinline__ void ma_stage(const real* __restrict__ Lm,
                                         const real* __restrict__ Bm, const real* c, real* g,
                                         const real (*Kold)[D], real cK, real (*Knew)[D],
                                         real (*Kacc)[D], real w, bool wantA) {
#pragma unroll Unroll<D>::n
  for (int i = 0; i < D; ++i) {
    real Gi[D];
    real lc = real(0);
#pragma unroll Unroll<D>::n
    for (int j = 0; j < D; ++j) {
      real l = __ldg(Lm + i * D + j);
      Gi[j] = l;
      lc += l * c[j];
    }
#pragma unroll Unroll<D>::n
    for (int m = 0; m < D; ++m) {
      real cm = c[m];
      const real* row = Bm + ((int64_t)m * D + i) * D;
#pragma unroll Unroll<D>::n
      for (int j = 0; j < D; ++j) Gi[j] += cm * __ldg(row + j);
    }
    real gc = real(0);
#pragma unroll Unroll<D>::n
    for (int j = 0; j < D; ++j) gc += Gi[j] * c[j];
    g[i] = real(0.5) * (lc + gc);
    if (wantA) {
#pragma unroll Unroll<D>::n
      for (int j = 0; j < D; ++j) {
        real v = Gi[j];
        if (Kold != nullptr) {
          real acc = real(0);
#pragma unroll Unroll<D>::n
          for (int m = 0; m < D; ++m) acc += Gi[m] * Kold[m][j];
          v += cK * acc;
        }
        Knew[i][j] = v;
        Kacc[i][j] += w * v;
      }
    }
  }
}

template <class real, int D>
__device__ __forceinline__ void ma_eval(const DynView<real>& dv, int64_t seq, bool rk4,
                                        const real* s, real* F, real (*A)[D], bool wantA) {
  const real* T = dv.ma + seq * dv.ma_stride;
  const real* Lm = T;
  const real* Bm = T + D * D;
  const real h = dv.dt;
  real Kacc[D][D];
  if (wantA) {
#pragma unroll Unroll<D>::n
    for (int i = 0; i < D; ++i)
#pragma unroll Unroll<D>::n
      for (int j = 0; j < D; ++j) Kacc[i][j] = real(0);
  }
  real g[D];
  if (!rk4) {
    real K[D][D];
    ma_stage<real, D>(Lm, Bm, s, g, nullptr, real(0), K, Kacc, real(1), wantA);
#pragma unroll Unroll<D>::n
    for (int i = 0; i < D; ++i) F[i] = s[i] + h * g[i];
    if (wantA) {
#pragma unroll Unroll<D>::n
      for (int i = 0; i < D; ++i)
#pragma unroll Unroll<D>::n
        for (int j = 0; j < D; ++j) A[i][j] = (i == j ? real(1) : real(0)) + h * Kacc[i][j];
    }
    return;
  }
  real acc[D], st[D];
  real Ka[D][D], Kb[D][D];
  // stage 1: k1 = g(s), K1 = G(s)
  ma_stage<real, D>(Lm, Bm, s, g, nullptr, real(0), Ka, Kacc, real(1), wantA);
#pragma unroll Unroll<D>::n
  for (int i = 0; i < D; ++i) { acc[i] = g[i]; st[i] = s[i] + real(0.5) * h * g[i]; }
  // stage 2: k2 = g(s + h/2 k1), K2 = G(.) (I + h/2 K1)
  ma_stage<real, D>(Lm, Bm, st, g, Ka, real(0.5) * h, Kb, Kacc, real(2), wantA);
#pragma unroll Unroll<D>::n
  for (int i = 0; i < D; ++i) { acc[i] += real(2) * g[i]; st[i] = s[i] + real(0.5) * h * g[i]; }
  // stage 3
  ma_stage<real, D>(Lm, Bm, st, g, Kb, real(0.5) * h, Ka, Kacc, real(2), wantA);
#pragma unroll Unroll<D>::n
  for (int i = 0; i < D; ++i) { acc[i] += real(2) * g[i]; st[i] = s[i] + h * g[i]; }
  // stage 4
  ma_stage<real, D>(Lm, Bm, st, g, Ka, h, Kb, Kacc, real(1), wantA);
  const real h6 = h / real(6);
#pragma unroll Unroll<D>::n
  for (int i = 0; i < D; ++i) F[i] = s[i] + h6 * (acc[i] + g[i]);
  if (wantA) {
#pragma unroll Unroll<D>::n
    for (int i = 0; i < D; ++i)
#pragma unroll Unroll<D>::n
      for (int j = 0; j < D; ++j) A[i][j] = (i == j ? real(1) : real(0)) + h6 * Kacc[i][j];
  }
}

// ----------------------------------------------------------------------------
// GRU (generic thread-per-row form)
// ----------------------------------------------------------------------------
template <class real>
__device__ __forceinline__ real sigm(real v) { return real(1) / (real(1) + exp(-v)); }

// jmode: 0 = no Jacobian, 1 = full (A [D][D]), 2 = diagonal only (Ad[i] = A_ii)
template <class real, int D>
__device__ __forceinline__ void gru_eval(const DynView<real>& dv, int64_t row, const real* h,
                                         real* F, real (*A)[D], real* Ad, int jmode) {
  const int din = dv.d_in;
  const real* Wz = dv.params;
  const real* Wr = Wz + D * din;
  const real* Wh = Wr + D * din;
  const real* Uz = Wh + D * din;
  const real* Ur = Uz + D * D;
  const real* Uh = Ur + D * D;
  const real* x = dv.x + row * din;
  real z[D], r[D], ht[D];
#pragma unroll Unroll<D>::n
  for (int i = 0; i < D; ++i) {
    real az = real(0), ar = real(0), ah = real(0);
    for (int k = 0; k < din; ++k) {
      real xk = __ldg(x + k);
      az += __ldg(Wz + i * din + k) * xk;
      ar += __ldg(Wr + i * din + k) * xk;
      ah += __ldg(Wh + i * din + k) * xk;
    }
#pragma unroll Unroll<D>::n
    for (int j = 0; j < D; ++j) {
      az += __ldg(Uz + i * D + j) * h[j];
      ar += __ldg(Ur + i * D + j) * h[j];
    }
    z[i] = sigm(az);
    r[i] = sigm(ar);
    ht[i] = ah;  // input part of the candidate pre-activation
  }
#pragma unroll Unroll<D>::n
  for (int i = 0; i < D; ++i) {
    real ah = ht[i];
#pragma unroll Unroll<D>::n
    for (int j = 0; j < D; ++j) ah += __ldg(Uh + i * D + j) * (r[j] * h[j]);
    ht[i] = tanh(ah);
  }
#pragma unroll Unroll<D>::n
  for (int i = 0; i < D; ++i) F[i] = (real(1) - z[i]) * h[i] + z[i] * ht[i];
  if (jmode == 0) return;
  if (jmode == 2) {
    // A_ii = (1 - z_i) + (h~_i - h_i) z_i (1 - z_i) Uz_ii
    //        + z_i (1 - h~_i^2) (Uh_ii r_i + sum_j M_ij h_j r_j (1 - r_j)),  M_ij = Uh_ij Ur_ji
#pragma unroll Unroll<D>::n
    for (int i = 0; i < D; ++i) {
      real sum = real(0);
#pragma unroll Unroll<D>::n
      for (int j = 0; j < D; ++j) sum += __ldg(dv.gru_M + i * D + j) * (h[j] * r[j] * (real(1) - r[j]));
      real zi = z[i];
      Ad[i] = (real(1) - zi) + (ht[i] - h[i]) * zi * (real(1) - zi) * __ldg(Uz + i * D + i) +
                zi * (real(1) - ht[i] * ht[i]) * (__ldg(Uh + i * D + i) * r[i] + sum);
    }
    return;
  }
  // full Jacobian
  real c[D];
#pragma unroll Unroll<D>::n
  for (int m = 0; m < D; ++m) c[m] = h[m] * r[m] * (real(1) - r[m]);
#pragma unroll Unroll<D>::n
  for (int i = 0; i < D; ++i) {
    real zi = z[i];
    real e1 = (ht[i] - h[i]) * zi * (real(1) - zi);
    real e2 = zi * (real(1) - ht[i] * ht[i]);
#pragma unroll Unroll<D>::n
    for (int j = 0; j < D; ++j) {
      real da = __ldg(Uh + i * D + j) * r[j];
      for (int m = 0; m < D; ++m) da += __ldg(Uh + i * D + m) * c[m] * __ldg(Ur + m * D + j);
      A[i][j] = (i == j ? real(1) - zi : real(0)) + e1 * __ldg(Uz + i * D + j) + e2 * da;
    }
  }
}

// ----------------------------------------------------------------------------
// Linear: f(s) = A s + x_t
// ----------------------------------------------------------------------------
template <class real, int D>
__device__ __forceinline__ void lin_eval(const DynView<real>& dv, int64_t row, const real* s,
                                         real* F, real (*A)[D], bool wantA) {
  const real* M = dv.params;
#pragma unroll Unroll<D>::n
  for (int i = 0; i < D; ++i) {
    real v = dv.x ? __ldg(dv.x + row * D + i) : real(0);
#pragma unroll Unroll<D>::n
    for (int j = 0; j < D; ++j) {
      real a = __ldg(M + i * D + j);
      v += a * s[j];
      if (wantA) A[i][j] = a;
    }
    F[i] = v;
  }
}

// ----------------------------------------------------------------------------
// Mean-field RNN: f(s) = W tanh(s) + u_t, A = W diag(1 - tanh(s)^2) (Sec. ssc:exp_thresh).
// JM: 0 = value, 1 = full Jacobian into A, 2 = diagonal into Ad.
// ----------------------------------------------------------------------------
template <class real, int D, int JM>
__device__ __forceinline__ void rnn_eval(const DynView<real>& dv, int64_t seq, int64_t row,
                                         const real* s, real* F, real (*A)[D], real* Ad) {
  const real* W = dv.params + seq * dv.pstride;
  real th[D];
#pragma unroll Unroll<D>::n
  for (int j = 0; j < D; ++j) th[j] = tanh(s[j]);
#pragma unroll Unroll<D>::n
  for (int i = 0; i < D; ++i) {
    real v = dv.x ? __ldg(dv.x + row * D + i) : real(0);
#pragma unroll Unroll<D>::n
    for (int j = 0; j < D; ++j) {
      const real w = __ldg(W + i * D + j);
      v += w * th[j];
      if constexpr (JM == 1) A[i][j] = w * (real(1) - th[j] * th[j]);
    }
    F[i] = v;
    if constexpr (JM == 2) Ad[i] = __ldg(W + i * D + i) * (real(1) - th[i] * th[i]);
  }
}

// ----------------------------------------------------------------------------
// Langevin step in a two-component Gaussian-mixture potential (Eq. langevin):
//   f(s) = s - dt grad phi(s) + sqrt(2 dt) w_t,  phi = -log(w1 N1 + w2 N2),
// with responsibilities g_k = w_k N_k / (w1 N1 + w2 N2) taken from the log-densities
// l_k = log w_k - (1/2) sum_i [log v_ki + (s_i - m_ki)^2 / v_ki] (the 2 pi terms cancel).
//   grad phi = g1 (s - m1)/v1 + g2 (s - m2)/v2
//   Hess phi = diag(g1/v1 + g2/v2) - g1 g2 e e^T,  e = (s - m2)/v2 - (s - m1)/v1
// (the covariance of the component scores under the responsibilities), A = I - dt Hess.
// ----------------------------------------------------------------------------
template <class real, int D, int JM>
__device__ __forceinline__ void langevin_eval(const DynView<real>& dv, int64_t seq,
                                              int64_t row, const real* s, real* F,
                                              real (*A)[D], real* Ad) {
  const real* p = dv.params + seq * dv.pstride;
  const real* m1 = p;
  const real* m2 = p + D;
  const real* v1 = p + 2 * D;
  const real* v2 = p + 3 * D;
  real q1 = real(0), q2 = real(0);
  real z1[D], z2[D];  // (s - m_k) / v_k
#pragma unroll Unroll<D>::n
  for (int i = 0; i < D; ++i) {
    const real a1 = s[i] - __ldg(m1 + i), a2 = s[i] - __ldg(m2 + i);
    const real iv1 = real(1) / __ldg(v1 + i), iv2 = real(1) / __ldg(v2 + i);
    z1[i] = a1 * iv1;
    z2[i] = a2 * iv2;
    q1 += log(__ldg(v1 + i)) + a1 * z1[i];
    q2 += log(__ldg(v2 + i)) + a2 * z2[i];
  }
  const real l1 = log(__ldg(p + 4 * D)) - real(0.5) * q1;
  const real l2 = log(__ldg(p + 4 * D + 1)) - real(0.5) * q2;
  const real g1 = real(1) / (real(1) + exp(l2 - l1));
  const real g2 = real(1) / (real(1) + exp(l1 - l2));
  const real dt = dv.dt;
  const real amp = sqrt(real(2) * dt);
#pragma unroll Unroll<D>::n
  for (int i = 0; i < D; ++i) {
    const real grad = g1 * z1[i] + g2 * z2[i];
    const real w = dv.x ? __ldg(dv.x + row * D + i) : real(0);
    F[i] = s[i] - dt * grad + amp * w;
  }
  if constexpr (JM != 0) {
    const real g12 = g1 * g2;
#pragma unroll Unroll<D>::n
    for (int i = 0; i < D; ++i) {
      const real ei = z2[i] - z1[i];
      const real hii = g1 / __ldg(v1 + i) + g2 / __ldg(v2 + i);
      if constexpr (JM == 2) {
        Ad[i] = real(1) - dt * (hii - g12 * ei * ei);
      } else {
#pragma unroll Unroll<D>::n
        for (int j = 0; j < D; ++j) {
          const real h = (i == j ? hii : real(0)) - g12 * ei * (z2[j] - z1[j]);
          A[i][j] = (i == j ? real(1) : real(0)) - dt * h;
        }
      }
    }
  }
}

// ----------------------------------------------------------------------------
// Lorenz-96, one fixed step of the fifth-order Dormand-Prince solution. Stages
//   Y_k = s + h sum_{j<k} a_kj k_j,  k_k = g(Y_k),  f(s) = s + h sum_k b_k k_k,
// and the step Jacobian column by column in forward mode: for the tangent e_c,
//   dY_k = e_c + h sum_{j<k} a_kj dk_j,  dk_k = g'(Y_k) dY_k,  A e_c = e_c + h sum_k b_k dk_k,
// where g'(x) v = (v_{i+1} - v_{i-2}) x_{i-1} + (x_{i+1} - x_{i-2}) v_{i-1} - v_i.
// Coefficients: the published Dormand-Prince (1980) tableau; the seventh stage carries no
// weight in the fifth-order solution and is not evaluated.
// ----------------------------------------------------------------------------
struct DP5 {
  static constexpr int S = 6;
  __device__ static constexpr double a(int k, int j) {
    return k == 1 ? (j == 0 ? 1.0 / 5 : 0.0)
         : k == 2 ? (j == 0 ? 3.0 / 40 : j == 1 ? 9.0 / 40 : 0.0)
         : k == 3 ? (j == 0 ? 44.0 / 45 : j == 1 ? -56.0 / 15 : j == 2 ? 32.0 / 9 : 0.0)
         : k == 4 ? (j == 0 ? 19372.0 / 6561 : j == 1 ? -25360.0 / 2187
                    : j == 2 ? 64448.0 / 6561 : j == 3 ? -212.0 / 729 : 0.0)
         : k == 5 ? (j == 0 ? 9017.0 / 3168 : j == 1 ? -355.0 / 33 : j == 2 ? 46732.0 / 5247
                    : j == 3 ? 49.0 / 176 : j == 4 ? -5103.0 / 18656 : 0.0)
         : 0.0;
  }
  __device__ static constexpr double b(int k) {
    return k == 0 ? 35.0 / 384 : k == 1 ? 0.0 : k == 2 ? 500.0 / 1113 : k == 3 ? 125.0 / 192
         : k == 4 ? -2187.0 / 6784 : k == 5 ? 11.0 / 84 : 0.0;
  }
};

template <class real, int D>
__device__ __forceinline__ void l96_rhs(const real* x, real F, real* g) {
#pragma unroll
  for (int i = 0; i < D; ++i)
    g[i] = (x[(i + 1) % D] - x[(i + D - 2) % D]) * x[(i + D - 1) % D] - x[i] + F;
}

template <class real, int D>
__device__ __forceinline__ void l96_jvp(const real* x, const real* v, real* out) {
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const int ip = (i + 1) % D, im = (i + D - 1) % D, im2 = (i + D - 2) % D;
    out[i] = (v[ip] - v[im2]) * x[im] + (x[ip] - x[im2]) * v[im] - v[i];
  }
}

template <class real, int D, int JM>
__device__ __forceinline__ void l96_eval(const DynView<real>& dv, int64_t seq, const real* s,
                                         real* F, real (*A)[D], real* Ad) {
  static_assert(D >= 4, "Lorenz-96 needs at least four coordinates");
  const real Fc = __ldg(dv.params + seq * dv.pstride);
  const real h = dv.dt;
  real Y[DP5::S][D], k[DP5::S][D];
#pragma unroll
  for (int st = 0; st < DP5::S; ++st) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
      real y = s[i];
#pragma unroll
      for (int j = 0; j < st; ++j) y += h * real(DP5::a(st, j)) * k[j][i];
      Y[st][i] = y;
    }
    l96_rhs<real, D>(Y[st], Fc, k[st]);
  }
#pragma unroll
  for (int i = 0; i < D; ++i) {
    real acc = real(0);
#pragma unroll
    for (int st = 0; st < DP5::S; ++st) acc += real(DP5::b(st)) * k[st][i];
    F[i] = s[i] + h * acc;
  }
  if constexpr (JM != 0) {
#pragma unroll 1
    for (int c = 0; c < D; ++c) {
      real dk[DP5::S][D];
#pragma unroll
      for (int st = 0; st < DP5::S; ++st) {
        real dy[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          real v = i == c ? real(1) : real(0);
#pragma unroll
          for (int j = 0; j < st; ++j) v += h * real(DP5::a(st, j)) * dk[j][i];
          dy[i] = v;
        }
        l96_jvp<real, D>(Y[st], dy, dk[st]);
      }
#pragma unroll
      for (int i = 0; i < D; ++i) {
        real acc = real(0);
#pragma unroll
        for (int st = 0; st < DP5::S; ++st) acc += real(DP5::b(st)) * dk[st][i];
        const real v = (i == c ? real(1) : real(0)) + h * acc;
        if constexpr (JM == 1) A[i][c] = v;
        if constexpr (JM == 2) if (i == c) Ad[c] = v;
      }
    }
  }
}

// ----------------------------------------------------------------------------
// Input-selected permutation (Prop. cayley): F_i = s[x_t[i]], A_t[i][j] = [j == x_t[i]].
// An index that is not an integer in [0, D) yields NaN for that entry.
// ----------------------------------------------------------------------------
template <class real, int D, int JM>
__device__ __forceinline__ void perm_eval(const DynView<real>& dv, int64_t row, const real* s,
                                          real* F, real (*A)[D], real* Ad) {
#pragma unroll Unroll<D>::n
  for (int i = 0; i < D; ++i) {
    const real xv = __ldg(dv.x + row * D + i);
    const bool ok = xv >= real(0) && xv < real(D) && xv == real((int)xv);
    const int src = ok ? (int)xv : -1;
    real v = ok ? real(0) : real(NAN);
#pragma unroll Unroll<D>::n
    for (int j = 0; j < D; ++j) {
      if (j == src) v = s[j];
      if constexpr (JM == 1) A[i][j] = j == src ? real(1) : real(0);
    }
    F[i] = v;
    if constexpr (JM == 2) Ad[i] = src == i ? real(1) : real(0);
  }
}

// ----------------------------------------------------------------------------
// Input vector-Jacobian product out_k = sum_i lam_i d f_i / d x_k at s_{t-1} = h, for the
// kinds whose inputs x_t enter f_t (Sec. 2.1): additive inputs (affine, mean-field RNN),
// scaled noise draws (Langevin: sqrt(2 dt)), and the GRU through its three gates:
//   dz~_i = lam_i (h~_i - h_i) z_i (1 - z_i),   da_i = lam_i z_i (1 - h~_i^2),
//   dr~_m = h_m r_m (1 - r_m) sum_i Uh_im da_i,
//   out_k = sum_i (Wz_ik dz~_i + Wr_ik dr~_i + Wh_ik da_i).
// ----------------------------------------------------------------------------
template <class real, int D, int KIND>
__device__ __forceinline__ void input_vjp(const DynView<real>& dv, int64_t row, const real* h,
                                          const real* lam, real* __restrict__ out) {
  if constexpr (KIND == DEER_F_GRU) {
    const int din = dv.d_in;
    const real* Wz = dv.params;
    const real* Wr = Wz + D * din;
    const real* Wh = Wr + D * din;
    const real* Uz = Wh + D * din;
    const real* Ur = Uz + D * D;
    const real* Uh = Ur + D * D;
    const real* x = dv.x + row * din;
    real z[D], r[D], ht[D];
#pragma unroll Unroll<D>::n
    for (int i = 0; i < D; ++i) {
      real az = real(0), ar = real(0), ah = real(0);
      for (int k = 0; k < din; ++k) {
        const real xk = __ldg(x + k);
        az += __ldg(Wz + i * din + k) * xk;
        ar += __ldg(Wr + i * din + k) * xk;
        ah += __ldg(Wh + i * din + k) * xk;
      }
#pragma unroll Unroll<D>::n
      for (int j = 0; j < D; ++j) {
        az += __ldg(Uz + i * D + j) * h[j];
        ar += __ldg(Ur + i * D + j) * h[j];
      }
      z[i] = sigm(az);
      r[i] = sigm(ar);
      ht[i] = ah;
    }
#pragma unroll Unroll<D>::n
    for (int i = 0; i < D; ++i) {
      real ah = ht[i];
#pragma unroll Unroll<D>::n
      for (int j = 0; j < D; ++j) ah += __ldg(Uh + i * D + j) * (r[j] * h[j]);
      ht[i] = tanh(ah);
    }
    real dz[D], da[D], dr[D];
#pragma unroll Unroll<D>::n
    for (int i = 0; i < D; ++i) {
      dz[i] = lam[i] * (ht[i] - h[i]) * z[i] * (real(1) - z[i]);
      da[i] = lam[i] * z[i] * (real(1) - ht[i] * ht[i]);
    }
#pragma unroll Unroll<D>::n
    for (int m = 0; m < D; ++m) {
      real q = real(0);
#pragma unroll Unroll<D>::n
      for (int i = 0; i < D; ++i) q += __ldg(Uh + i * D + m) * da[i];
      dr[m] = q * h[m] * r[m] * (real(1) - r[m]);
    }
    for (int k = 0; k < din; ++k) {
      real v = real(0);
#pragma unroll Unroll<D>::n
      for (int i = 0; i < D; ++i)
        v += __ldg(Wz + i * din + k) * dz[i] + __ldg(Wr + i * din + k) * dr[i] +
             __ldg(Wh + i * din + k) * da[i];
      out[k] = v;
    }
  } else {
    const real scale = KIND == DEER_F_LANGEVIN_2WELL ? sqrt(real(2) * dv.dt) : real(1);
#pragma unroll Unroll<D>::n
    for (int i = 0; i < D; ++i) out[i] = scale * lam[i];
  }
}

// Dispatch on the dynamics kind (compile time). JM: 0 = value only, 1 = full Jacobian
// into A, 2 = diagonal of the Jacobian into Ad.
template <class real, int D, int KIND, int JM>
__device__ __forceinline__ void eval_f(const DynView<real>& dv, int64_t seq, int64_t row,
                                       const real* s, real* F, real (*A)[D], real* Ad) {
  if constexpr (KIND == DEER_F_GRU) {
    gru_eval<real, D>(dv, row, s, F, A, Ad, JM);
  } else if constexpr (KIND == DEER_F_RNN_TANH) {
    rnn_eval<real, D, JM>(dv, seq, row, s, F, A, Ad);
  } else if constexpr (KIND == DEER_F_LANGEVIN_2WELL) {
    langevin_eval<real, D, JM>(dv, seq, row, s, F, A, Ad);
  } else if constexpr (KIND == DEER_F_LORENZ96_DP5) {
    if constexpr (D >= 4) l96_eval<real, D, JM>(dv, seq, s, F, A, Ad);
  } else if constexpr (KIND == DEER_F_PERMUTE) {
    perm_eval<real, D, JM>(dv, row, s, F, A, Ad);
  } else {
    real Af[JM == 2 ? D : 1][JM == 2 ? D : 1];
    real (*Aw)[D] = nullptr;
    if constexpr (JM == 1) Aw = A;
    if constexpr (JM == 2) Aw = reinterpret_cast<real (*)[D]>(&Af[0][0]);
    if constexpr (KIND == DEER_F_BRUSSELATOR_EULER) {
      if constexpr (D == 2) bruss_eval<real>(dv, seq, s, F, Aw, JM != 0);
    } else if constexpr (KIND == DEER_F_MASSACTION_EULER) {
      ma_eval<real, D>(dv, seq, false, s, F, Aw, JM != 0);
    } else if constexpr (KIND == DEER_F_MASSACTION_RK4) {
      ma_eval<real, D>(dv, seq, true, s, F, Aw, JM != 0);
    } else {
      lin_eval<real, D>(dv, row, s, F, Aw, JM != 0);
    }
    if constexpr (JM == 2) {
#pragma unroll Unroll<D>::n
      for (int i = 0; i < D; ++i) Ad[i] = Af[i][i];
    }
  }
}

}  // namespace deer

namespace deer {

// ----------------------------------------------------------------------------
// Mass action, register path for d <= 8. One row per LPR lanes; every lane builds the full
// rate Jacobian G of a stage and advances its own JC = D/LPR columns of the stage Jacobian
// K_j = G_j (I + c_j K_{j-1}) in place (column j of K_j depends on column j of K_{j-1}
// only), so no values are exchanged between lanes. The RK4 stage loop is kept rolled:
// fully unrolled, the four stages exceed what the register allocator handles without
// spilling.
// ----------------------------------------------------------------------------
template <class real, int D>
__device__ __forceinline__ void ldrow(const real* __restrict__ p, real (&v)[D]) {
  constexpr int bytes = D * (int)sizeof(real);
  if constexpr (bytes % 16 == 0) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int i = 0; i < bytes / 16; ++i) reinterpret_cast<float4*>(v)[i] = __ldg(q + i);
  } else if constexpr (bytes % 8 == 0) {
    const float2* q = reinterpret_cast<const float2*>(p);
#pragma unroll
    for (int i = 0; i < bytes / 8; ++i) reinterpret_cast<float2*>(v)[i] = __ldg(q + i);
  } else {
#pragma unroll
    for (int i = 0; i < D; ++i) v[i] = __ldg(p + i);
  }
}

// G(c) = L + sum_m c_m B_m and g(c) = (L c + G c) / 2.
template <class real, int D>
__device__ __forceinline__ void ma_build_G(const real* __restrict__ Lm,
                                           const real* __restrict__ Bm, const real (&c)[D],
                                           real (&G)[D][D], real (&g)[D]) {
  real lc[D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    ldrow<real, D>(Lm + i * D, G[i]);
    lc[i] = real(0);
#pragma unroll
    for (int j = 0; j < D; ++j) lc[i] += G[i][j] * c[j];
  }
#pragma unroll
  for (int m = 0; m < D; ++m) {
    const real cm = c[m];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      real br[D];
      ldrow<real, D>(Bm + (m * D + i) * D, br);
#pragma unroll
      for (int j = 0; j < D; ++j) G[i][j] += cm * br[j];
    }
  }
#pragma unroll
  for (int i = 0; i < D; ++i) {
    real gc = real(0);
#pragma unroll
    for (int j = 0; j < D; ++j) gc += G[i][j] * c[j];
    g[i] = real(0.5) * (lc[i] + gc);
  }
}

// One integrator step: F (all rows) and, if WANTA, the columns h*JC .. h*JC+JC-1 of
// A = I + h/6 (K1 + 2 K2 + 2 K3 + K4) (RK4) or I + h G (Euler).
// Entry h * RPL + ii of a full register vector without a run-time register index.
template <class real, int D, int RPL>
__device__ __forceinline__ real own_row(const real (&v)[D], int h, int ii) {
  if constexpr (RPL == D) return v[ii];
  else return h == 0 ? v[ii] : v[RPL + ii];
}

template <class real, int D, int LPR, bool RK4, bool WANTA>
__device__ __forceinline__ void ma_step_cols(const real* __restrict__ T, real hstep, int h,
                                             const real (&s)[D], real (&F)[D],
                                             real (&Aown)[D][D / LPR]) {
  static_assert(LPR == 1 || LPR == 2, "one or two lanes per row");
  constexpr int JC = D / LPR;
  const real* Lm = T;
  const real* Bm = T + D * D;
  real G[D][D], g[D], st[D], acc[D];
  real K[D][JC], Kacc[D][JC];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    st[i] = s[i];
    acc[i] = real(0);
#pragma unroll
    for (int j = 0; j < JC; ++j) { K[i][j] = real(0); Kacc[i][j] = real(0); }
  }
  constexpr int NST = RK4 ? 4 : 1;
#pragma unroll 1
  for (int stage = 0; stage < NST; ++stage) {
    // RK4 tableau: stage derivative weights (1, 2, 2, 1), stage offsets (h/2, h/2, h)
    const real cK = stage == 0 ? real(0) : (stage == 3 ? hstep : real(0.5) * hstep);
    const real w = (stage == 1 || stage == 2) ? real(2) : real(1);
    ma_build_G<real, D>(Lm, Bm, st, G, g);
    if constexpr (WANTA) {
#pragma unroll
      for (int jj = 0; jj < JC; ++jj) {
        real col[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          real v = own_row<real, D, JC>(G[i], h, jj);
          real pr = real(0);
#pragma unroll
          for (int m = 0; m < D; ++m) pr += G[i][m] * K[m][jj];
          col[i] = v + cK * pr;
        }
#pragma unroll
        for (int i = 0; i < D; ++i) { K[i][jj] = col[i]; Kacc[i][jj] += w * col[i]; }
      }
    }
    const real cs = stage == 2 ? hstep : real(0.5) * hstep;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      acc[i] += w * g[i];
      st[i] = s[i] + cs * g[i];
    }
  }
  const real hw = RK4 ? hstep / real(6) : hstep;
#pragma unroll
  for (int i = 0; i < D; ++i) F[i] = s[i] + hw * acc[i];
  if constexpr (WANTA) {
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int jj = 0; jj < JC; ++jj)
        Aown[i][jj] = hw * Kacc[i][jj] + ((h * JC + jj) == i ? real(1) : real(0));
  }
}

}  // namespace deer
