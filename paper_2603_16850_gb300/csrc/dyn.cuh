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

// Dispatch on the dynamics kind (compile time). JM: 0 = value only, 1 = full Jacobian
// into A, 2 = diagonal of the Jacobian into Ad.
template <class real, int D, int KIND, int JM>
__device__ __forceinline__ void eval_f(const DynView<real>& dv, int64_t seq, int64_t row,
                                       const real* s, real* F, real (*A)[D], real* Ad) {
  if constexpr (KIND == DEER_F_GRU) {
    gru_eval<real, D>(dv, row, s, F, A, Ad, JM);
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
