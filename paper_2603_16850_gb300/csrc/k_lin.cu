// Linearisation / residual kernels, initial guesses, mass-action tensor set-up and the
// sequential GPU rollout (comparison baseline).
#include <cstdio>

#include "lin_generic.cuh"
#include "tc.cuh"

namespace deer {

// ----------------------------------------------------------------------------
// Mass-action tensors: L (unimolecular) and B_m (symmetrised bimolecular), per sequence.
// ----------------------------------------------------------------------------
template <class real>
__global__ void k_ma_setup(int64_t n_seq, int d, int R, const real* __restrict__ k,
                           int64_t kstride, const int32_t* __restrict__ topo, int64_t tstride,
                           real* __restrict__ out, int64_t ostride, int32_t* bad) {
  const int64_t seq = blockIdx.x;
  if (seq >= n_seq) return;
  real* L = out + seq * ostride;
  real* Bm = L + d * d;
  const int64_t n = (int64_t)d * d + (int64_t)d * d * d;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) L[i] = real(0);
  __syncthreads();
  if (threadIdx.x != 0) return;
  const real* kk = k + seq * kstride;
  const int32_t* tt = topo + seq * tstride;
  for (int r = 0; r < R; ++r) {
    const int i1 = tt[4 * r + 0], i2 = tt[4 * r + 1], p1 = tt[4 * r + 2], p2 = tt[4 * r + 3];
    // species indices must lie in [0, d) (second slots may be -1); a bad reaction is
    // skipped and reported instead of being written out of bounds
    if (i1 < 0 || i1 >= d || p1 < 0 || p1 >= d || i2 < -1 || i2 >= d || p2 < -1 || p2 >= d) {
      *bad = 1;
      continue;
    }
    const real kr = kk[r];
    int sp[4] = {i1, i2, p1, p2};
    real nu[4] = {real(-1), real(-1), real(1), real(1)};
    for (int q = 0; q < 4; ++q) {
      const int i = sp[q];
      if (i < 0) continue;
      const real v = nu[q] * kr;
      if (i2 < 0) {
        L[i * d + i1] += v;  // rate k c_i1
      } else {
        Bm[((int64_t)i2 * d + i) * d + i1] += v;  // d/dc_i1 of k c_i1 c_i2 = k c_i2
        Bm[((int64_t)i1 * d + i) * d + i2] += v;  // d/dc_i2 = k c_i1
      }
    }
  }
}

// ----------------------------------------------------------------------------
// Mass action, d <= 8: LPR lanes per row, each owning JC = D/LPR columns of A_t and the
// rows h*JC .. h*JC+JC-1 of F_t, r_t and b_t (see ma_step_cols).
// ----------------------------------------------------------------------------
template <class real, int D, int LPR, bool RK4, int JAC>
__global__ void __launch_bounds__(128) k_lin_ma(LinArgs<real> a) {
  constexpr int JC = D / LPR;
  constexpr bool WANTA = JAC == DEER_JAC_FULL || JAC == DEER_JAC_DIAG;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t ar = tid / LPR;
  const int h = LPR == 2 ? (int)(tid & 1) : 0;
  const bool valid = ar < a.bt.act_rows();
  int64_t seq = 0, row = 0;
  if (valid) act_row(a.bt, ar, seq, row);
  real mx = real(0), sq = real(0);
  unsigned long long key = 0ull;  // first failing row (sliding window)
  if (valid) {
    real sp[D], sc[JC];
    if (row == __ldg(a.bt.offsets + seq)) {
#pragma unroll
      for (int i = 0; i < D; ++i) sp[i] = __ldg(a.s0 + seq * D + i);
    } else {
      load_row<real, D>(a.s + (row - 1) * D, sp);
    }
    load_row<real, JC>(a.s + row * D + h * JC, sc);
    const real* T = a.dv.ma + seq * a.dv.ma_stride;
    real F[D], A[D][JC];
    ma_step_cols<real, D, LPR, RK4, WANTA>(T, a.dv.dt, h, sp, F, A);
    const real k = a.dparam;
    real b[JC];
#pragma unroll
    for (int ii = 0; ii < JC; ++ii) {
      const real Fi = own_row<real, D, JC>(F, h, ii);
      const real r = sc[ii] - Fi;
      const real sabs = rabs(sc[ii]);
      const real sr = rabs(r) / (sabs > real(1) ? sabs : real(1));
      mx = (sr > mx || sr != sr) ? sr : mx;
      if (!(sr <= a.tol)) key = bad_key(true, row - __ldg(a.bt.offsets + seq));
      sq += r * r;
      b[ii] = -r;
    }
    if constexpr (JAC == DEER_JAC_FULL) {
      const real scale = (a.damp == DEER_DAMP_SCALE) ? real(1) - k : real(1);
      real* Ao = a.A + row * (int64_t)(D * D) + h * JC;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        real v[JC];
#pragma unroll
        for (int jj = 0; jj < JC; ++jj) v[jj] = scale * A[i][jj];
        store_row<real, JC>(Ao + i * D, v);
      }
    } else {
      real ad[JC];
#pragma unroll
      for (int ii = 0; ii < JC; ++ii) {
        real ai;
        if constexpr (JAC == DEER_JAC_DIAG) {
          // diagonal entry (h*JC + ii, h*JC + ii) lives in own column ii
          if constexpr (LPR == 1) ai = A[ii][ii];
          else ai = h == 0 ? A[ii][ii] : A[JC + ii][ii];
        } else if constexpr (JAC == DEER_JAC_IDENTITY) {
          ai = real(1);
        } else {
          ai = real(0);
        }
        if (a.damp == DEER_DAMP_SCALE) ai *= (real(1) - k);
        else if (a.damp == DEER_DAMP_CLIP) ai = ai > k ? k : (ai < -k ? -k : ai);
        ad[ii] = ai;
        // standard form: b = F - a s_{t-1}
        b[ii] = own_row<real, D, JC>(F, h, ii) - ai * own_row<real, D, JC>(sp, h, ii);
      }
      if constexpr (JAC == DEER_JAC_DIAG) store_row<real, JC>(a.A + row * D + h * JC, ad);
    }
    store_row<real, JC>(a.b + row * D + h * JC, b);
  }
  acc_resid_t(a.acc, seq, valid, mx, sq, key);
}

// ----------------------------------------------------------------------------
// Sequential rollout (baseline). Mass action: D lanes per trajectory, lane i owns species
// i, one pass over the reactions per stage with shuffles for the reactant values (no
// Jacobian). Other kinds: one thread per trajectory.
// ----------------------------------------------------------------------------
template <class real, int D>
__device__ __forceinline__ real ma_lane_rate(const real* __restrict__ kk,
                                             const int4* __restrict__ tt, int R, real c,
                                             int lane, unsigned mask) {
  real g = real(0);
  for (int r = 0; r < R; ++r) {
    const int4 q = __ldg(tt + r);
    const real kr = __ldg(kk + r);
    const real c1 = __shfl_sync(mask, c, q.x, D);
    const real c2 = __shfl_sync(mask, c, q.y < 0 ? 0 : q.y, D);
    const real rate = kr * c1 * (q.y < 0 ? real(1) : c2);
    const real nu = real((lane == q.z) + (lane == q.w) - (lane == q.x) - (lane == q.y));
    g += nu * rate;
  }
  return g;
}

template <class real, int D>
__global__ void __launch_bounds__(128) k_rollout_ma(RolloutArgs<real> a, int rk4) {
  constexpr int G = D;  // lanes per trajectory (D divides 32)
  const int64_t gid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
  const int lane = threadIdx.x % G;
  const int64_t seq = gid < a.B ? gid : a.B - 1;
  const bool live = gid < a.B;
  const unsigned mask = 0xffffffffu;
  int64_t r0, r1;
  rollout_rows(a, seq, r0, r1);
  const real* kk = a.dv.params + seq * a.dv.pstride;
  const int4* tt = reinterpret_cast<const int4*>(a.dv.topo + seq * a.dv.tstride);
  const int R = a.dv.R;
  const real h = a.dv.dt;
  real c = a.s0[seq * D + lane];
  const int64_t n = live ? r1 - r0 : 0;
  // all groups of a warp iterate the warp maximum so that shuffles stay converged
  int64_t nmax = n;
  for (int o = 16; o > 0; o >>= 1) {
    int64_t v = __shfl_xor_sync(mask, nmax, o);
    nmax = v > nmax ? v : nmax;
  }
  for (int64_t t = 0; t < nmax; ++t) {
    real cn;
    if (!rk4) {
      cn = c + h * ma_lane_rate<real, D>(kk, tt, R, c, lane, mask);
    } else {
      const real k1 = ma_lane_rate<real, D>(kk, tt, R, c, lane, mask);
      const real k2 = ma_lane_rate<real, D>(kk, tt, R, c + real(0.5) * h * k1, lane, mask);
      const real k3 = ma_lane_rate<real, D>(kk, tt, R, c + real(0.5) * h * k2, lane, mask);
      const real k4 = ma_lane_rate<real, D>(kk, tt, R, c + h * k3, lane, mask);
      cn = c + (h / real(6)) * (k1 + real(2) * k2 + real(2) * k3 + k4);
    }
    if (t < n) {
      c = cn;
      a.s[(r0 + t) * D + lane] = c;
    }
  }
}


// GRU set-up: M[i][j] = Uh[i][j] * Ur[j][i], the matrix of the off-diagonal term of the
// closed-form Jacobian diagonal.
template <class real>
__global__ void k_gru_setup(int d, const real* __restrict__ params, int d_in, real* M) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= d * d) return;
  const int i = id / d, j = id % d;
  const real* Ur = params + 3 * d * d_in + d * d;
  const real* Uh = Ur + d * d;
  M[id] = Uh[i * d + j] * Ur[j * d + i];
}


// ----------------------------------------------------------------------------
// Adjoint parameter gradient (one thread per row): the vector-Jacobian product
// lambda_t^T df_t/dtheta (s_{t-1}) by reverse-mode through the integrator stages, summed
// over the rows of each sequence (warp reduction, then one atomic per warp and
// parameter), and dl/ds0 = A_1^T lambda_1. Mass action: theta = rate constants k;
// Brusselator: theta = (a, b).
// ----------------------------------------------------------------------------
constexpr int kMaxD = 32;

template <class real>
__device__ __forceinline__ void ma_rate_vec(const real* kk, const int4* tt, int R, int d,
                                            const real* c, real* g) {
  for (int i = 0; i < d; ++i) g[i] = real(0);
  for (int r = 0; r < R; ++r) {
    const int4 q = __ldg(tt + r);
    const real rate = __ldg(kk + r) * c[q.x] * (q.y >= 0 ? c[q.y] : real(1));
    g[q.x] -= rate;
    if (q.y >= 0) g[q.y] -= rate;
    g[q.z] += rate;
    if (q.w >= 0) g[q.w] += rate;
  }
}

// out += G(c)^T u for the mass-action rate Jacobian G
template <class real>
__device__ __forceinline__ void ma_rate_vjp(const real* kk, const int4* tt, int R,
                                            const real* c, const real* u, real* out) {
  for (int r = 0; r < R; ++r) {
    const int4 q = __ldg(tt + r);
    real nu_u = u[q.z] - u[q.x];
    if (q.y >= 0) nu_u -= u[q.y];
    if (q.w >= 0) nu_u += u[q.w];
    const real w = __ldg(kk + r) * nu_u;
    if (q.y >= 0) {
      out[q.x] += w * c[q.y];
      out[q.y] += w * c[q.x];
    } else {
      out[q.x] += w;
    }
  }
}

template <class real>
__global__ void __launch_bounds__(128) k_param_grad(ParamGradArgs<real> a, int rk4) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool valid = row < a.bt.N;
  const int d = a.dv.d;
  int64_t seq = 0;
  if (valid) seq = find_seq(a.bt.offsets, a.bt.B, row);
  const int64_t first = valid ? a.bt.offsets[seq] : 0;
  const real* sp = valid ? (row == first ? a.s0 + seq * d : a.s + (row - 1) * d) : a.s0;
  const real* lam = a.lam + (valid ? row : 0) * d;
  if (valid && a.ds0 && row == first) {
    const real* A1 = a.A + row * (int64_t)d * d;
    for (int j = 0; j < d; ++j) {
      real acc = real(0);
      for (int i = 0; i < d; ++i) acc += A1[i * d + j] * lam[i];
      a.ds0[seq * d + j] = acc;
    }
  }
  if (!a.dparams) return;
  const unsigned full = 0xffffffffu;
  const unsigned vm = __ballot_sync(full, valid);
  if (vm == 0) return;
  const long long sseq = __shfl_sync(full, (long long)seq, __ffs(vm) - 1);
  const bool uniform = __all_sync(full, !valid || seq == sseq);
  auto put = [&](int j, real v) {
    if (uniform) {
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(full, v, o);
      if ((threadIdx.x & 31) == 0) atomicAdd(a.dparams + sseq * a.pstride + j, v);
    } else if (valid) {
      atomicAdd(a.dparams + seq * a.pstride + j, v);
    }
  };
  if (a.dv.kind == DEER_F_BRUSSELATOR_EULER) {
    const real dt = a.dv.dt;
    const real ga = valid ? dt * lam[0] : real(0);
    const real gb = valid ? dt * sp[0] * (lam[1] - lam[0]) : real(0);
    put(0, ga);
    put(1, gb);
    return;
  }
  // mass action
  const int R = a.dv.R;
  const real* kk = a.dv.params + seq * a.dv.pstride;
  const int4* tt = reinterpret_cast<const int4*>(a.dv.topo + seq * a.dv.tstride);
  const real h = a.dv.dt;
  real c[4][kMaxD], u[4][kMaxD], tmp[kMaxD];
  const int nst = rk4 ? 4 : 1;
  if (valid) {
    for (int i = 0; i < d; ++i) c[0][i] = sp[i];
    if (rk4) {
      ma_rate_vec(kk, tt, R, d, c[0], tmp);
      for (int i = 0; i < d; ++i) c[1][i] = sp[i] + real(0.5) * h * tmp[i];
      ma_rate_vec(kk, tt, R, d, c[1], tmp);
      for (int i = 0; i < d; ++i) c[2][i] = sp[i] + real(0.5) * h * tmp[i];
      ma_rate_vec(kk, tt, R, d, c[2], tmp);
      for (int i = 0; i < d; ++i) c[3][i] = sp[i] + h * tmp[i];
      // cotangents of the stage slopes, from the last stage back
      for (int i = 0; i < d; ++i) u[3][i] = h / real(6) * lam[i];
      for (int i = 0; i < d; ++i) tmp[i] = real(0);
      ma_rate_vjp(kk, tt, R, c[3], u[3], tmp);
      for (int i = 0; i < d; ++i) u[2][i] = h / real(3) * lam[i] + h * tmp[i];
      for (int i = 0; i < d; ++i) tmp[i] = real(0);
      ma_rate_vjp(kk, tt, R, c[2], u[2], tmp);
      for (int i = 0; i < d; ++i) u[1][i] = h / real(3) * lam[i] + real(0.5) * h * tmp[i];
      for (int i = 0; i < d; ++i) tmp[i] = real(0);
      ma_rate_vjp(kk, tt, R, c[1], u[1], tmp);
      for (int i = 0; i < d; ++i) u[0][i] = h / real(6) * lam[i] + real(0.5) * h * tmp[i];
    } else {
      for (int i = 0; i < d; ++i) u[0][i] = h * lam[i];
    }
  }
  // d f / d k_r contracted with lambda: sum over stages of phi_r(c_s) (nu_r . u_s)
  for (int r = 0; r < R; ++r) {
    real v = real(0);
    if (valid) {
      const int4 q = __ldg(tt + r);
      for (int st = 0; st < nst; ++st) {
        const real phi = c[st][q.x] * (q.y >= 0 ? c[st][q.y] : real(1));
        real nu_u = u[st][q.z] - u[st][q.x];
        if (q.y >= 0) nu_u -= u[st][q.y];
        if (q.w >= 0) nu_u += u[st][q.w];
        v += phi * nu_u;
      }
    }
    put(r, v);
  }
}

template <class real>
cudaError_t launch_param_grad(const ParamGradArgs<real>& a, cudaStream_t st) {
  if (a.bt.N == 0) return cudaSuccess;
  if (a.dv.d > kMaxD) return cudaErrorInvalidValue;
  const int rk4 = a.dv.kind == DEER_F_MASSACTION_RK4;
  k_param_grad<real><<<grid_for(a.bt.N, 128), 128, 0, st>>>(a, rk4);
  note_launch();
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Host-side dispatch
// ----------------------------------------------------------------------------
template <class real>
cudaError_t launch_gru_setup(int d, const real* params, int d_in, real* M, cudaStream_t st) {
  k_gru_setup<real><<<grid_for(d * d, 128), 128, 0, st>>>(d, params, d_in, M);
  note_launch();
  return cudaGetLastError();
}

template <class real>
cudaError_t launch_ma_setup(int64_t n_seq, int d, int R, const real* k, int64_t kstride,
                            const int32_t* topo, int64_t tstride, real* out, int64_t ostride,
                            int32_t* bad, cudaStream_t st) {
  k_ma_setup<real><<<(unsigned)n_seq, 128, 0, st>>>(n_seq, d, R, k, kstride, topo, tstride, out,
                                                    ostride, bad);
  note_launch();
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Kind dispatch. Mass action runs its own kernels here; the kinds evaluated through the
// generic kernels are launched from their own translation units.
// ----------------------------------------------------------------------------
// DEER_INIT_RANDN: iid standard normal entries (Sec. 3.3.3 draws the guess from N(0, I)).
// Entry e of the packed state takes outputs 2e+1 and 2e+2 of the SplitMix64 stream
// started at the seed (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", 2014: output n is the mix of seed + n * golden gamma), so any thread can
// draw any entry, and turns them into one normal by the Box-Muller transform in float64.
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed,
                                                            unsigned long long n) {
  unsigned long long z = seed + n * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <class real>
__global__ void __launch_bounds__(256) k_init_randn(real* __restrict__ s, int64_t n,
                                                    unsigned long long seed) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += stride) {
    const unsigned long long z1 = splitmix64_at(seed, 2ull * (unsigned long long)e + 1ull);
    const unsigned long long z2 = splitmix64_at(seed, 2ull * (unsigned long long)e + 2ull);
    const double u1 = (double)((z1 >> 11) + 1ull) * 0x1.0p-53;  // (0, 1]
    const double u2 = (double)(z2 >> 11) * 0x1.0p-53;           // [0, 1)
    s[e] = (real)(sqrt(-2.0 * log(u1)) * cospi(2.0 * u2));
  }
}

template <class real>
cudaError_t launch_init(const InitArgs<real>& a, cudaStream_t st) {
  if (a.bt.N == 0) return cudaSuccess;
  if (a.init == DEER_INIT_RANDN) {
    const int64_t n = a.bt.N * a.dv.d;
    int64_t g = (n + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    k_init_randn<real><<<(unsigned)g, 256, 0, st>>>(a.s, n, a.seed);
    note_launch();
    return cudaGetLastError();
  }
  switch (a.dv.kind) {
    case DEER_F_MASSACTION_EULER: return generic_init<real, DEER_F_MASSACTION_EULER>(a, st);
    case DEER_F_MASSACTION_RK4: return generic_init<real, DEER_F_MASSACTION_RK4>(a, st);
    case DEER_F_BRUSSELATOR_EULER:
    case DEER_F_GRU:
    case DEER_F_LINEAR: return launch_init_basic<real>(a, st);
    default: return launch_init_models<real>(a, st);
  }
}

template <class real, int JAC>
cudaError_t launch_lin_ma_wide(const LinArgs<real>& a, cudaStream_t st);

template <class real, bool RK4, int JAC>
static cudaError_t lin_ma_jac(const LinArgs<real>& a, cudaStream_t st) {
  const unsigned g = grid_for(a.bt.act_rows(), 128);
  switch (a.dv.d) {
    case 2: k_lin_ma<real, 2, 1, RK4, JAC><<<g, 128, 0, st>>>(a); break;
    case 4: k_lin_ma<real, 4, 1, RK4, JAC><<<g, 128, 0, st>>>(a); break;
    case 8:
      if constexpr (sizeof(real) == 4) {
        k_lin_ma<real, 8, 1, RK4, JAC><<<g, 128, 0, st>>>(a);
      } else {
        k_lin_ma<real, 8, 2, RK4, JAC><<<grid_for(a.bt.act_rows() * 2, 128), 128, 0, st>>>(a);
      }
      break;
    case 16:
    case 32: return launch_lin_ma_wide<real, JAC>(a, st);
    default: return cudaErrorInvalidValue;
  }
  note_launch();
  return cudaGetLastError();
}

template <class real, bool RK4>
static cudaError_t lin_ma(const LinArgs<real>& a, cudaStream_t st) {
  switch (a.jac) {
    case DEER_JAC_FULL: return lin_ma_jac<real, RK4, DEER_JAC_FULL>(a, st);
    case DEER_JAC_DIAG: return lin_ma_jac<real, RK4, DEER_JAC_DIAG>(a, st);
    case DEER_JAC_IDENTITY: return lin_ma_jac<real, RK4, DEER_JAC_IDENTITY>(a, st);
    default: return lin_ma_jac<real, RK4, DEER_JAC_ZERO>(a, st);
  }
}

template <class real>
cudaError_t launch_linearize(const LinArgs<real>& a, cudaStream_t st) {
  if (a.bt.act_rows() == 0) return cudaSuccess;
  switch (a.dv.kind) {
    case DEER_F_MASSACTION_EULER: return lin_ma<real, false>(a, st);
    case DEER_F_MASSACTION_RK4: return lin_ma<real, true>(a, st);
    case DEER_F_BRUSSELATOR_EULER:
    case DEER_F_GRU:
    case DEER_F_LINEAR: return launch_linearize_basic<real>(a, st);
    default: return launch_linearize_models<real>(a, st);
  }
}

template <class real>
cudaError_t launch_rollout(const RolloutArgs<real>& a, cudaStream_t st) {
  if (a.B == 0) return cudaSuccess;
  const int kind = a.dv.kind;
  if (kind == DEER_F_MASSACTION_EULER || kind == DEER_F_MASSACTION_RK4) {
    const int rk4 = kind == DEER_F_MASSACTION_RK4;
    const int d = a.dv.d;
    const int64_t threads = a.B * (int64_t)d;
    const unsigned g = grid_for(threads, 128);
    switch (d) {
      case 2: k_rollout_ma<real, 2><<<g, 128, 0, st>>>(a, rk4); break;
      case 4: k_rollout_ma<real, 4><<<g, 128, 0, st>>>(a, rk4); break;
      case 8: k_rollout_ma<real, 8><<<g, 128, 0, st>>>(a, rk4); break;
      case 16: k_rollout_ma<real, 16><<<g, 128, 0, st>>>(a, rk4); break;
      case 32: k_rollout_ma<real, 32><<<g, 128, 0, st>>>(a, rk4); break;
      default: return cudaErrorInvalidValue;
    }
    note_launch();
    return cudaGetLastError();
  }
  if (kind == DEER_F_BRUSSELATOR_EULER || kind == DEER_F_GRU || kind == DEER_F_LINEAR)
    return launch_rollout_basic<real>(a, st);
  return launch_rollout_models<real>(a, st);
}

template <class real>
cudaError_t launch_input_grad(const InputGradArgs<real>& a, cudaStream_t st) {
  if (a.bt.N == 0) return cudaSuccess;
  switch (a.dv.kind) {
    case DEER_F_GRU:
    case DEER_F_LINEAR: return launch_input_grad_basic<real>(a, st);
    case DEER_F_RNN_TANH:
    case DEER_F_LANGEVIN_2WELL: return launch_input_grad_models<real>(a, st);
    default: return cudaErrorInvalidValue;  // no differentiable inputs
  }
}

#define DEER_INST(real)                                                                         \
  template cudaError_t launch_input_grad<real>(const InputGradArgs<real>&, cudaStream_t);     \
  template cudaError_t launch_ma_setup<real>(int64_t, int, int, const real*, int64_t,          \
                                             const int32_t*, int64_t, real*, int64_t,          \
                                             int32_t*, cudaStream_t);                          \
  template cudaError_t launch_init<real>(const InitArgs<real>&, cudaStream_t);                 \
  template cudaError_t launch_linearize<real>(const LinArgs<real>&, cudaStream_t);             \
  template cudaError_t launch_rollout<real>(const RolloutArgs<real>&, cudaStream_t);          \
  template cudaError_t launch_gru_setup<real>(int, const real*, int, real*, cudaStream_t);   \
  template cudaError_t launch_param_grad<real>(const ParamGradArgs<real>&, cudaStream_t);
DEER_INST(float)
DEER_INST(double)
#undef DEER_INST

}  // namespace deer

namespace deer {

constexpr int kMaRows = 4;  // consecutive rows per lane group in k_lin_ma_wide

// ----------------------------------------------------------------------------
// Mass action, d = 16 / 32: D lanes per row, lane i owns species i (its state, slope and
// row i of the stage Jacobians). Rates come from one pass over the reactions with
// shuffles for the reactant concentrations; the sparse rate Jacobian G is scattered into
// shared memory by the (at most four) lanes each reaction touches; the chain
// K_j = G_j (I + c_j K_{j-1}) reads the previous K rows from shared memory as broadcasts.
// ----------------------------------------------------------------------------
template <class real, int D, bool RK4, int JAC>
__global__ void __launch_bounds__(128, (D == 32 && sizeof(real) == 4) ? 4 : 1)
    k_lin_ma_wide(LinArgs<real> a) {
  constexpr int GROUPS = 128 / D;          // rows per block
  constexpr bool WANTA = JAC == DEER_JAC_FULL || JAC == DEER_JAC_DIAG;
  // d = 32 float32: the stage-Jacobian products G_j K_{j-1} run on the tensor cores as
  // warp-level tf32 MMAs with the three-term split (float32 accuracy); the rate-Jacobian
  // rows are then padded to 36 floats (conflict-free fragment and 16-byte row reads)
  constexpr bool TCW = D == 32 && sizeof(real) == 4;
  // full Jacobian on that path: the stage Jacobians stay in the MMA accumulator layout
  // from stage to stage (written to shared memory only as the next product's operand), and
  // A_t leaves through a shared-memory tile in 16-byte pieces
  constexpr bool FRAG = TCW && JAC == DEER_JAC_FULL;
  constexpr int GS = TCW ? D + 4 : D + 1;
  __shared__ __align__(16) real sG[GROUPS][D][GS];
  // rows padded by 16 bytes (the d lanes' 16-byte row writes fall in distinct banks) and
  // the group stride by another 16 (the groups of a warp read their K rows from different
  // banks)
  // (the accumulator-layout path pads its stage rows to 40 floats instead: its fragment
  // loads and two-float stores then fall in distinct banks)
  constexpr int RSK = FRAG ? D + 8 : D + 16 / (int)sizeof(real);
  __shared__ __align__(16) real sK[GROUPS][D * RSK + 16 / sizeof(real)];
  // per reaction of the group's row: rate constant, first reactant concentration and the
  // second factor (the second reactant's concentration, or 1): written by lane r mod d,
  // read by the lanes of the species the reaction changes
  constexpr int RMAX = 4 * D;
  __shared__ real sKr[GROUPS][RMAX], sC1[GROUPS][RMAX], sF2[GROUPS][RMAX];
  const int grp = threadIdx.x / D, lane = threadIdx.x % D;
  const unsigned gmask = D == 32 ? 0xffffffffu : (0xffffu << (16 * ((threadIdx.x >> 4) & 1)));
  const bool use_adj = a.adj_off != nullptr && a.dv.R <= RMAX;
  // each group walks kMaRows consecutive active rows and flushes the residual statistics
  // once per sequence it meets (not once per row): fewer atomics on the accumulator of a
  // long sequence
  const int64_t ar0 = (blockIdx.x * (int64_t)GROUPS + grp) * kMaRows;
  int64_t cur = -1;
  real mx = real(0), sq = real(0);
  unsigned long long key = 0ull;  // first failing row (sliding window)
  for (int ri = 0; ri < kMaRows; ++ri) {
    const int64_t ar = ar0 + ri;
    if (ar >= a.bt.act_rows()) break;  // uniform over the group
    int64_t seq, row;
    act_row(a.bt, ar, seq, row);
    if (seq != cur) {
      if (cur >= 0) acc_resid_group<D>(a.acc, cur, mx, sq, key, lane, gmask);
      cur = seq;
      mx = real(0);
      sq = real(0);
      key = 0ull;
    }
    const bool row_first = row == __ldg(a.bt.offsets + seq);
    const real s_prev = row_first ? a.s0[seq * D + lane] : a.s[(row - 1) * D + lane];
    // compensated state (float32 path): the parts below the half ulp of s_{t-1} and s_t
    const real p_lo = (a.slo && !row_first) ? a.slo[(row - 1) * D + lane] : real(0);
    const real* kk = a.dv.params + seq * a.dv.pstride;
    const int4* tt = reinterpret_cast<const int4*>(a.dv.topo + seq * a.dv.tstride);
    const int R = a.dv.R;
    const real h = a.dv.dt;
    real c = s_prev, acc = real(0), g = real(0);
    float KaccF[2][4][4];  // FRAG: sum of w K_j, accumulator layout
    if constexpr (FRAG) {
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
          for (int e = 0; e < 4; ++e) KaccF[mt][nt][e] = 0.f;
    }
    real Kacc[D];
#pragma unroll
    for (int j = 0; j < D; ++j) Kacc[j] = real(0);
    const int nst = RK4 ? 4 : 1;
    for (int stage = 0; stage < nst; ++stage) {
      const real cK = stage == 0 ? real(0) : (stage == 3 ? h : real(0.5) * h);
      const real w = (stage == 1 || stage == 2) ? real(2) : real(1);
      if (WANTA) {
        if constexpr (TCW) {
#pragma unroll
          for (int j = 0; j < D; j += 4)
            *reinterpret_cast<float4*>(&sG[grp][lane][j]) = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
#pragma unroll
          for (int j = 0; j < D; ++j) sG[grp][lane][j] = real(0);
        }
      }
      __syncwarp(gmask);
      g = real(0);
      if (use_adj) {
        // each reaction's factors once (reaction r on lane r mod d), then each lane walks
        // the reactions that change its species, in reaction order (the same products and
        // sums as the walk over every reaction below)
        for (int k0 = 0; k0 < R; k0 += D) {  // uniform over the group
          const int r = k0 + lane;
          const int4 q = r < R ? __ldg(tt + r) : make_int4(0, -1, 0, 0);
          const real c1 = __shfl_sync(gmask, c, q.x, D);
          const real c2 = __shfl_sync(gmask, c, q.y < 0 ? 0 : q.y, D);
          if (r < R) {
            sKr[grp][r] = __ldg(kk + r);
            sC1[grp][r] = c1;
            sF2[grp][r] = q.y < 0 ? real(1) : c2;
          }
        }
        __syncwarp(gmask);
        const int32_t* aoff = a.adj_off + (a.adj_stride ? seq : 0) * (D + 1);
        const int32_t* ae = a.adj_e + (a.adj_stride ? seq : 0) * a.adj_stride;
        const int e1 = __ldg(aoff + lane + 1);
        for (int e = __ldg(aoff + lane); e < e1; ++e) {
          const int code = __ldg(ae + e);
          const int r = code & 0xffff;
          const real nu = real((code >> 16) - 4);
          const real kr = sKr[grp][r], c1 = sC1[grp][r], f2 = sF2[grp][r];
          g += nu * (kr * c1 * f2);
          if (WANTA) {
            const int4 q = __ldg(tt + r);
            sG[grp][lane][q.x] += nu * kr * f2;                  // d rate / d c_i1
            if (q.y >= 0) sG[grp][lane][q.y] += nu * kr * c1;    // d rate / d c_i2
          }
        }
      } else {
        for (int r = 0; r < R; ++r) {
          const int4 q = __ldg(tt + r);
          const real kr = __ldg(kk + r);
          const real c1 = __shfl_sync(gmask, c, q.x, D);
          const real c2 = __shfl_sync(gmask, c, q.y < 0 ? 0 : q.y, D);
          const real f2 = q.y < 0 ? real(1) : c2;
          const real nu = real((lane == q.z) + (lane == q.w) - (lane == q.x) - (lane == q.y));
          g += nu * (kr * c1 * f2);
          if (WANTA && nu != real(0)) {
            sG[grp][lane][q.x] += nu * kr * f2;                  // d rate / d c_i1
            if (q.y >= 0) sG[grp][lane][q.y] += nu * kr * c1;    // d rate / d c_i2
          }
        }
      }
      if constexpr (FRAG) {
        __syncwarp(gmask);
        const int g8 = lane >> 2, tq = lane & 3;
        float Kf[2][4][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
          for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) Kf[mt][nt][e] = 0.f;
        if (stage > 0) {
          // P = G_j K_{j-1} (32 x 32 x 32) on the tensor cores, three-term tf32 split
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            uint32_t ah[2][4], al[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
              const float* r0 = &sG[grp][16 * mt + g8][8 * kk];
              const float* r1 = &sG[grp][16 * mt + g8 + 8][8 * kk];
              const float av[4] = {r0[tq], r1[tq], r0[tq + 4], r1[tq + 4]};
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                ah[mt][e] = tc::tf32_rna(av[e]);
                al[mt][e] = tc::tf32_rna(av[e] - __uint_as_float(ah[mt][e]));
              }
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
              const float bx0 = sK[grp][(8 * kk + tq) * RSK + 8 * nt + g8];
              const float bx1 = sK[grp][(8 * kk + tq + 4) * RSK + 8 * nt + g8];
              const uint32_t bh0 = tc::tf32_rna(bx0), bh1 = tc::tf32_rna(bx1);
              const uint32_t bl0 = tc::tf32_rna(bx0 - __uint_as_float(bh0));
              const uint32_t bl1 = tc::tf32_rna(bx1 - __uint_as_float(bh1));
#pragma unroll
              for (int mt = 0; mt < 2; ++mt) {
                tc::mma_1688_tf32(Kf[mt][nt], al[mt], bh0, bh1);
                tc::mma_1688_tf32(Kf[mt][nt], ah[mt], bl0, bl1);
                tc::mma_1688_tf32(Kf[mt][nt], ah[mt], bh0, bh1);
              }
            }
          }
        }
        // K_j = G_j + cK P in the accumulator layout (rows 16 mt + g, + 8; columns
        // 8 nt + 2 t, + 1)
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            const float2 g0 =
                *reinterpret_cast<const float2*>(&sG[grp][16 * mt + g8][8 * nt + 2 * tq]);
            const float2 g1 =
                *reinterpret_cast<const float2*>(&sG[grp][16 * mt + g8 + 8][8 * nt + 2 * tq]);
            Kf[mt][nt][0] = g0.x + cK * Kf[mt][nt][0];
            Kf[mt][nt][1] = g0.y + cK * Kf[mt][nt][1];
            Kf[mt][nt][2] = g1.x + cK * Kf[mt][nt][2];
            Kf[mt][nt][3] = g1.y + cK * Kf[mt][nt][3];
          }
        __syncwarp(gmask);  // every read of K_{j-1} done
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            *reinterpret_cast<float2*>(&sK[grp][(16 * mt + g8) * RSK + 8 * nt + 2 * tq]) =
                make_float2(Kf[mt][nt][0], Kf[mt][nt][1]);
            *reinterpret_cast<float2*>(&sK[grp][(16 * mt + g8 + 8) * RSK + 8 * nt + 2 * tq]) =
                make_float2(Kf[mt][nt][2], Kf[mt][nt][3]);
#pragma unroll
            for (int e = 0; e < 4; ++e) KaccF[mt][nt][e] += (float)w * Kf[mt][nt][e];
          }
        __syncwarp(gmask);
      } else if (WANTA) {
        __syncwarp(gmask);
        real Gi[D], Kn[D];
        if constexpr (TCW) {
          // (the rate-Jacobian row is read after the product, so that it is not held in
          // registers across the MMAs)
          if (stage == 0) {
#pragma unroll
            for (int j = 0; j < D; j += 4) {
              const float4 q = *reinterpret_cast<const float4*>(&sG[grp][lane][j]);
              Kn[j] = q.x; Kn[j + 1] = q.y; Kn[j + 2] = q.z; Kn[j + 3] = q.w;
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < D; ++j) Gi[j] = sG[grp][lane][j];
#pragma unroll
          for (int j = 0; j < D; ++j) Kn[j] = Gi[j];
        }
        if constexpr (TCW) {
          if (stage > 0) {
            // P = G_j K_{j-1} (32 x 32 x 32): 2 x 4 output tiles, 4 k-steps, three MMAs
            // each (lo*hi, hi*lo, hi*hi); A from the rate-Jacobian rows, B from the
            // previous stage's rows
            const int g = lane >> 2, tq = lane & 3;
            float P[2][4][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
              for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) P[mt][nt][e] = 0.f;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              uint32_t ah[2][4], al[2][4];
#pragma unroll
              for (int mt = 0; mt < 2; ++mt) {
                const float* r0 = &sG[grp][16 * mt + g][8 * kk];
                const float* r1 = &sG[grp][16 * mt + g + 8][8 * kk];
                const float av[4] = {r0[tq], r1[tq], r0[tq + 4], r1[tq + 4]};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                  ah[mt][e] = tc::tf32_rna(av[e]);
                  al[mt][e] = tc::tf32_rna(av[e] - __uint_as_float(ah[mt][e]));
                }
              }
#pragma unroll
              for (int nt = 0; nt < 4; ++nt) {
                const float bx0 = sK[grp][(8 * kk + tq) * RSK + 8 * nt + g];
                const float bx1 = sK[grp][(8 * kk + tq + 4) * RSK + 8 * nt + g];
                const uint32_t bh0 = tc::tf32_rna(bx0), bh1 = tc::tf32_rna(bx1);
                const uint32_t bl0 = tc::tf32_rna(bx0 - __uint_as_float(bh0));
                const uint32_t bl1 = tc::tf32_rna(bx1 - __uint_as_float(bh1));
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                  tc::mma_1688_tf32(P[mt][nt], al[mt], bh0, bh1);
                  tc::mma_1688_tf32(P[mt][nt], ah[mt], bl0, bl1);
                  tc::mma_1688_tf32(P[mt][nt], ah[mt], bh0, bh1);
                }
              }
            }
            // the previous stage's rows are no longer needed: P goes there, then each lane
            // takes its row, K_j = G_j + cK P
            __syncwarp(gmask);
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
              for (int nt = 0; nt < 4; ++nt) {
                float* q0 = &sK[grp][(16 * mt + g) * RSK + 8 * nt + 2 * tq];
                float* q1 = &sK[grp][(16 * mt + g + 8) * RSK + 8 * nt + 2 * tq];
                *reinterpret_cast<float2*>(q0) = make_float2(P[mt][nt][0], P[mt][nt][1]);
                *reinterpret_cast<float2*>(q1) = make_float2(P[mt][nt][2], P[mt][nt][3]);
              }
            __syncwarp(gmask);
#pragma unroll
            for (int j = 0; j < D; j += 4) {
              const float4 q = *reinterpret_cast<const float4*>(&sK[grp][lane * RSK + j]);
              const float4 gq = *reinterpret_cast<const float4*>(&sG[grp][lane][j]);
              Kn[j] = gq.x + cK * q.x;
              Kn[j + 1] = gq.y + cK * q.y;
              Kn[j + 2] = gq.z + cK * q.z;
              Kn[j + 3] = gq.w + cK * q.w;
            }
          }
        } else if (stage > 0) {
          // row m of the previous stage Jacobian (the same for every lane of the group) in
          // 16-byte pieces, folded in with the packed FMA row update
          constexpr int VW = 16 / (int)sizeof(real);
#pragma unroll
          for (int m = 0; m < D; ++m) {
            const real gm = cK * Gi[m];
            const real* km = &sK[grp][m * RSK];
#pragma unroll
            for (int j = 0; j < D; j += VW) {
              real kv[VW], acc[VW];
              if constexpr (sizeof(real) == 4) {
                const float4 q = *reinterpret_cast<const float4*>(km + j);
                kv[0] = q.x; kv[1] = q.y; kv[2] = q.z; kv[3] = q.w;
              } else {
                const double2 q = *reinterpret_cast<const double2*>(km + j);
                kv[0] = q.x; kv[1] = q.y;
              }
#pragma unroll
              for (int e = 0; e < VW; ++e) acc[e] = Kn[j + e];
              axpy_row<VW>(gm, kv, acc);
#pragma unroll
              for (int e = 0; e < VW; ++e) Kn[j + e] = acc[e];
            }
          }
        }
        __syncwarp(gmask);
#pragma unroll
        for (int j = 0; j < D; j += 16 / (int)sizeof(real)) {
          if constexpr (sizeof(real) == 4) {
            *reinterpret_cast<float4*>(&sK[grp][lane * RSK + j]) =
                make_float4(Kn[j], Kn[j + 1], Kn[j + 2], Kn[j + 3]);
          } else {
            *reinterpret_cast<double2*>(&sK[grp][lane * RSK + j]) =
                make_double2(Kn[j], Kn[j + 1]);
          }
        }
        axpy_row<D>(w, Kn, Kacc);
        __syncwarp(gmask);
      }
      acc += w * g;
      const real cs = stage == 2 ? h : real(0.5) * h;
      c = s_prev + cs * g;
    }
    const real hw = RK4 ? h / real(6) : h;
    const real F = s_prev + hw * acc;
    {
      const real sc = a.s[row * D + lane];
      const real rr = a.slo ? cs_residual(sc, a.slo[row * D + lane], s_prev, p_lo, hw * acc)
                            : sc - F;
      const real sabs = rabs(sc);
      real m1 = rabs(rr) / (sabs > real(1) ? sabs : real(1));
      if (rr != rr) m1 = rr;  // keep NaN
      mx = (m1 > mx || m1 != m1) ? m1 : mx;
      sq += rr * rr;
      if (!(m1 <= a.tol) && key == 0ull) key = bad_key(true, row - __ldg(a.bt.offsets + seq));
      const real k = a.dparam;
      if constexpr (JAC == DEER_JAC_FULL) {
        const real scale = a.damp == DEER_DAMP_SCALE ? real(1) - k : real(1);
        // the rate-Jacobian buffer is free after the last stage
        __syncwarp(gmask);
        if constexpr (FRAG) {
          // A = s (I + hw Kacc) from the accumulator layout into the tile, then out in
          // 16-byte pieces (row p / 8, columns 4 (p % 8) .. + 3 of piece p)
          const int g8 = lane >> 2, tq = lane & 3;
          float* tile = &sG[grp][0][0];
#pragma unroll
          for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
              const int r0 = 16 * mt + g8, c0 = 8 * nt + 2 * tq;
              const float sc = (float)scale, hf = (float)hw;
              *reinterpret_cast<float2*>(tile + r0 * GS + c0) =
                  make_float2(sc * (hf * KaccF[mt][nt][0] + (r0 == c0 ? 1.f : 0.f)),
                              sc * (hf * KaccF[mt][nt][1] + (r0 == c0 + 1 ? 1.f : 0.f)));
              *reinterpret_cast<float2*>(tile + (r0 + 8) * GS + c0) =
                  make_float2(sc * (hf * KaccF[mt][nt][2] + (r0 + 8 == c0 ? 1.f : 0.f)),
                              sc * (hf * KaccF[mt][nt][3] + (r0 + 8 == c0 + 1 ? 1.f : 0.f)));
            }
          __syncwarp(gmask);
          float4* dst = reinterpret_cast<float4*>(a.A + row * (int64_t)(D * D));
#pragma unroll
          for (int q = 0; q < D * D / 4 / 32; ++q) {
            const int pc = q * 32 + lane;
            dst[pc] = *reinterpret_cast<const float4*>(tile + (pc >> 3) * GS + (pc & 7) * 4);
          }
          __syncwarp(gmask);
        } else {
          real An[D];
#pragma unroll
          for (int j = 0; j < D; ++j)
            An[j] = scale * (hw * Kacc[j] + (j == lane ? real(1) : real(0)));
          store_block_rows<real, D>(&sG[grp][0][0], a.A + row * (int64_t)(D * D), An, lane,
                                    gmask);
        }
        a.b[row * D + lane] = -rr;
      } else {
        real ai;
        if constexpr (JAC == DEER_JAC_DIAG) {
          ai = real(0);
#pragma unroll
          for (int j = 0; j < D; ++j)
            if (j == lane) ai = real(1) + hw * Kacc[j];
        } else if constexpr (JAC == DEER_JAC_IDENTITY) {
          ai = real(1);
        } else {
          ai = real(0);
        }
        if (a.damp == DEER_DAMP_SCALE) ai *= (real(1) - k);
        else if (a.damp == DEER_DAMP_CLIP) ai = ai > k ? k : (ai < -k ? -k : ai);
        if constexpr (JAC == DEER_JAC_DIAG) a.A[row * D + lane] = ai;
        a.b[row * D + lane] = F - ai * s_prev;
      }
    }
  }
  if (cur >= 0) acc_resid_group<D>(a.acc, cur, mx, sq, key, lane, gmask);
}

template <class real, int JAC>
cudaError_t launch_lin_ma_wide(const LinArgs<real>& a, cudaStream_t st) {
  const bool rk4 = a.dv.kind == DEER_F_MASSACTION_RK4;
  const int d = a.dv.d;
  const int64_t rows_per_block = 128 / d * kMaRows;
  const unsigned g = grid_for(a.bt.act_rows(), (int)rows_per_block);
  if (d == 16) {
    if (rk4) k_lin_ma_wide<real, 16, true, JAC><<<g, 128, 0, st>>>(a);
    else k_lin_ma_wide<real, 16, false, JAC><<<g, 128, 0, st>>>(a);
  } else if (d == 32) {
    if (rk4) k_lin_ma_wide<real, 32, true, JAC><<<g, 128, 0, st>>>(a);
    else k_lin_ma_wide<real, 32, false, JAC><<<g, 128, 0, st>>>(a);
  } else {
    return cudaErrorInvalidValue;
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace deer

namespace deer {
template cudaError_t launch_lin_ma_wide<float, DEER_JAC_FULL>(const LinArgs<float>&, cudaStream_t);
template cudaError_t launch_lin_ma_wide<float, DEER_JAC_DIAG>(const LinArgs<float>&, cudaStream_t);
template cudaError_t launch_lin_ma_wide<float, DEER_JAC_IDENTITY>(const LinArgs<float>&, cudaStream_t);
template cudaError_t launch_lin_ma_wide<float, DEER_JAC_ZERO>(const LinArgs<float>&, cudaStream_t);
template cudaError_t launch_lin_ma_wide<double, DEER_JAC_FULL>(const LinArgs<double>&, cudaStream_t);
template cudaError_t launch_lin_ma_wide<double, DEER_JAC_DIAG>(const LinArgs<double>&, cudaStream_t);
template cudaError_t launch_lin_ma_wide<double, DEER_JAC_IDENTITY>(const LinArgs<double>&, cudaStream_t);
template cudaError_t launch_lin_ma_wide<double, DEER_JAC_ZERO>(const LinArgs<double>&, cudaStream_t);
}  // namespace deer
