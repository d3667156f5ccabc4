// Whole Newton solve of a short sequence inside one thread block (Algorithm 1 with the
// full Jacobian): one block per sequence runs every iteration itself, linearisation,
// convergence test and the scan of Eq. bin_op_affine, with the iterate kept in registers.
// There is no launch and no host round trip per iteration, and a batch of short
// sequences is one launch in which every block stops on its own convergence.
//
// Thread q owns the contiguous rows [q R, q R + R) of its block's sequence (R = rows per
// thread for this T). One iteration:
//   1. each thread evaluates F_t = f_t(s_{t-1}) and A_t on its rows (the row before its
//      first comes from the previous thread through shared memory, s_0 for thread 0),
//      forms the residual r_t = s_t - F_t and composes its rows' affine steps
//      Delta -> A_t Delta - r_t into one element (P, v);
//   2. a block reduction gives the largest scaled residual max |r| / max(1, |s|) and
//      sum r^2; the test and the iteration count follow the library's convergence check;
//   3. a block-wide exclusive scan of the elements (warp shuffles, then the warp totals)
//      gives the correction Delta entering each thread's rows, which the thread then
//      propagates through its rows (evaluating A_t again rather than keeping it) and adds
//      to the iterate, with the reset heuristic.
#include <cfloat>

#include "dyn.cuh"
#include "kernels.h"

namespace deer {

template <class real, int D>
struct Aff {  // the affine map Delta -> P Delta + v
  real P[D][D];
  real v[D];
};

// later o earlier
template <class real, int D>
__device__ __forceinline__ Aff<real, D> compose(const Aff<real, D>& l, const Aff<real, D>& e) {
  Aff<real, D> o;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    real x = l.v[i];
#pragma unroll
    for (int k = 0; k < D; ++k) x += l.P[i][k] * e.v[k];
    o.v[i] = x;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      real y = real(0);
#pragma unroll
      for (int k = 0; k < D; ++k) y += l.P[i][k] * e.P[k][j];
      o.P[i][j] = y;
    }
  }
  return o;
}

template <class real, int D>
__device__ __forceinline__ Aff<real, D> shfl_up_aff(const Aff<real, D>& a, int off) {
  Aff<real, D> o;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    o.v[i] = __shfl_up_sync(0xffffffffu, a.v[i], off);
#pragma unroll
    for (int j = 0; j < D; ++j) o.P[i][j] = __shfl_up_sync(0xffffffffu, a.P[i][j], off);
  }
  return o;
}

template <class real, int D>
__device__ __forceinline__ Aff<real, D> aff_identity() {
  Aff<real, D> o;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    o.v[i] = real(0);
#pragma unroll
    for (int j = 0; j < D; ++j) o.P[i][j] = i == j ? real(1) : real(0);
  }
  return o;
}

// inclusive scan over the lanes of a warp (lane order = time order)
template <class real, int D>
__device__ __forceinline__ Aff<real, D> warp_scan_aff(Aff<real, D> x, int lane) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const Aff<real, D> y = shfl_up_aff<real, D>(x, off);
    if (lane >= off) x = compose<real, D>(x, y);
  }
  return x;
}

template <class real, int D, int KIND, int NT, int RPT>
__global__ void __launch_bounds__(NT) k_block_solve(BlockSolveArgs<real> a) {
  constexpr int NW = NT / 32;
  __shared__ real s_last[NT][D];       // each thread's last row of the iterate
  __shared__ Aff<real, D> s_warp[NW];  // inclusive warp totals, then their prefixes
  __shared__ real s_mx[NW];
  __shared__ double s_sq[NW];
  const int64_t seq = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r0 = a.offsets[seq];
  const int64_t T = a.offsets[seq + 1] - r0;
  const int rpt = (int)((T + NT - 1) / NT);  // rows per thread (<= RPT, checked by the host)
  const int64_t k0 = (int64_t)tid * rpt;
  const int nmine = T - k0 <= 0 ? 0 : (T - k0 < rpt ? (int)(T - k0) : rpt);
  const real scale = a.damp == DEER_DAMP_SCALE ? real(1) - a.dparam : real(1);
  real s[RPT][D];
  real s0[D];
#pragma unroll
  for (int i = 0; i < D; ++i) s0[i] = a.s0[seq * D + i];
#pragma unroll
  for (int k = 0; k < RPT; ++k)
#pragma unroll
    for (int i = 0; i < D; ++i) s[k][i] = k < nmine ? a.s[(r0 + k0 + k) * D + i] : real(0);
  SeqInfo inf = a.info[seq];
  int passes = 0;
  bool done = false, nonfinite = false;
  double merit = 0.0, mres = 0.0;
  int iters = 0;
  for (int it = 0;; ++it) {
    // the row before this thread's first is the previous thread's last (a thread without
    // rows is followed only by threads without rows)
#pragma unroll
    for (int k = 0; k < RPT; ++k)
      if (k == nmine - 1) {
#pragma unroll
        for (int i = 0; i < D; ++i) s_last[tid][i] = s[k][i];
      }
    __syncthreads();
    real prev[D];
#pragma unroll
    for (int i = 0; i < D; ++i) prev[i] = tid == 0 ? s0[i] : s_last[tid - 1][i];
    // 1. linearise, residual statistics, this thread's element
    Aff<real, D> e = aff_identity<real, D>();
    real mx = real(0);
    double sq = 0.0;
    {
      real sp[D];
#pragma unroll
      for (int i = 0; i < D; ++i) sp[i] = prev[i];
#pragma unroll
      for (int k = 0; k < RPT; ++k) {
        if (k < nmine) {
          real F[D], A[D][D];
          eval_f<real, D, KIND, 1>(a.dv, seq, r0 + k0 + k, sp, F, A, nullptr);
          real b[D];
#pragma unroll
          for (int i = 0; i < D; ++i) {
            const real r = s[k][i] - F[i];
            b[i] = -r;
            const real sabs = rabs(s[k][i]);
            const real sr = rabs(r) / (sabs > real(1) ? sabs : real(1));
            mx = (sr > mx || sr != sr) ? sr : mx;
            sq += (double)r * (double)r;
          }
          Aff<real, D> st;
#pragma unroll
          for (int i = 0; i < D; ++i) {
            st.v[i] = b[i];
#pragma unroll
            for (int j = 0; j < D; ++j) st.P[i][j] = scale * A[i][j];
          }
          e = compose<real, D>(st, e);
#pragma unroll
          for (int i = 0; i < D; ++i) sp[i] = s[k][i];
        }
      }
    }
    // 2. block reduction and the convergence test
    {
      double m = (double)mx;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        m = nanmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        sq += __shfl_xor_sync(0xffffffffu, sq, o);
      }
      if (lane == 0) {
        s_mx[warp] = (real)m;
        s_sq[warp] = sq;
      }
    }
    __syncthreads();
    double bm = 0.0, bs = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      bm = nanmax(bm, (double)s_mx[w]);
      bs += s_sq[w];
    }
    merit = 0.5 * bs;
    mres = bm;
    nonfinite = !(bm <= DBL_MAX);
    passes = bm <= a.tol ? passes + 1 : 0;
    if (passes >= a.confirm) {
      done = true;
      iters = it;
      break;
    }
    iters = it < a.max_iters ? it + 1 : it;
    if ((nonfinite && !a.reset) || it >= a.max_iters) break;
    // 3. block-wide exclusive scan of the elements, then this thread's rows
    const Aff<real, D> inc = warp_scan_aff<real, D>(e, lane);
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      Aff<real, D> wt = lane < NW ? s_warp[lane] : aff_identity<real, D>();
      wt = warp_scan_aff<real, D>(wt, lane);
      if (lane < NW) s_warp[lane] = wt;
    }
    __syncthreads();
    real din[D];
    {
      // Delta entering this thread: the warps before, then the lanes before in this warp
      Aff<real, D> ex = shfl_up_aff<real, D>(inc, 1);
      if (lane == 0) ex = aff_identity<real, D>();
      real dw[D];
#pragma unroll
      for (int i = 0; i < D; ++i) dw[i] = warp > 0 ? s_warp[warp - 1].v[i] : real(0);
#pragma unroll
      for (int i = 0; i < D; ++i) {
        real x = ex.v[i];
#pragma unroll
        for (int k = 0; k < D; ++k) x += ex.P[i][k] * dw[k];
        din[i] = x;
      }
    }
    {
      real sp[D];
#pragma unroll
      for (int i = 0; i < D; ++i) sp[i] = prev[i];
#pragma unroll
      for (int k = 0; k < RPT; ++k) {
        if (k < nmine) {
          real F[D], A[D][D];
          eval_f<real, D, KIND, 1>(a.dv, seq, r0 + k0 + k, sp, F, A, nullptr);
          real dn[D];
#pragma unroll
          for (int i = 0; i < D; ++i) {
            real x = F[i] - s[k][i];
#pragma unroll
            for (int j = 0; j < D; ++j) x += scale * A[i][j] * din[j];
            dn[i] = x;
          }
#pragma unroll
          for (int i = 0; i < D; ++i) {
            sp[i] = s[k][i];
            const real y = s[k][i] + dn[i];
            s[k][i] = (a.reset && !(y <= a.reset_thr && y >= -a.reset_thr)) ? real(0) : y;
            din[i] = dn[i];
          }
        }
      }
    }
    __syncthreads();  // s_last and s_warp are rewritten by the next iteration
  }
#pragma unroll
  for (int k = 0; k < RPT; ++k)
    if (k < nmine)
#pragma unroll
      for (int i = 0; i < D; ++i) a.s[(r0 + k0 + k) * D + i] = s[k][i];
  if (tid == 0) {
    inf.iters = iters;
    inf.done = done ? 1 : 0;
    inf.passes = passes;
    inf.merit = merit;
    inf.max_resid = mres;
    a.info[seq] = inf;
    if (nonfinite) atomicAdd(&a.flags->n_nonfinite, 1);
    if (!done) atomicAdd(&a.flags->n_active, 1);
  }
}

// rows per thread and threads per block by state size: every row's iterate stays in
// registers (D <= 2: 512 threads x 8 rows; D = 4: 256 x 4)
template <int D>
struct BlockCfg {
  static constexpr int NT = D <= 2 ? 512 : 256;
  static constexpr int RPT = D <= 2 ? 8 : 4;
};

int64_t block_solve_max_T(int kind, int d) {
  const bool kind_ok = kind == DEER_F_BRUSSELATOR_EULER || kind == DEER_F_MASSACTION_EULER ||
                       kind == DEER_F_MASSACTION_RK4 || kind == DEER_F_LINEAR ||
                       kind == DEER_F_RNN_TANH || kind == DEER_F_LANGEVIN_2WELL;
  if (!kind_ok) return 0;
  switch (d) {
    case 1: return (int64_t)BlockCfg<1>::NT * BlockCfg<1>::RPT;
    case 2: return (int64_t)BlockCfg<2>::NT * BlockCfg<2>::RPT;
    case 4: return (int64_t)BlockCfg<4>::NT * BlockCfg<4>::RPT;
    default: return 0;
  }
}

template <class real, int D, int KIND>
static void block_launch(const BlockSolveArgs<real>& a, cudaStream_t st) {
  using C = BlockCfg<D>;
  k_block_solve<real, D, KIND, C::NT, C::RPT><<<(unsigned)a.B, C::NT, 0, st>>>(a);
  note_launch();
}

template <class real, int D>
static cudaError_t block_kind(const BlockSolveArgs<real>& a, cudaStream_t st) {
  switch (a.dv.kind) {
    case DEER_F_BRUSSELATOR_EULER:
      if constexpr (D == 2) { block_launch<real, D, DEER_F_BRUSSELATOR_EULER>(a, st); break; }
      return cudaErrorInvalidValue;
    case DEER_F_MASSACTION_EULER:
      if constexpr (D >= 2) { block_launch<real, D, DEER_F_MASSACTION_EULER>(a, st); break; }
      return cudaErrorInvalidValue;
    case DEER_F_MASSACTION_RK4:
      if constexpr (D >= 2) { block_launch<real, D, DEER_F_MASSACTION_RK4>(a, st); break; }
      return cudaErrorInvalidValue;
    case DEER_F_LINEAR: block_launch<real, D, DEER_F_LINEAR>(a, st); break;
    case DEER_F_RNN_TANH: block_launch<real, D, DEER_F_RNN_TANH>(a, st); break;
    case DEER_F_LANGEVIN_2WELL: block_launch<real, D, DEER_F_LANGEVIN_2WELL>(a, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class real>
cudaError_t launch_block_solve(const BlockSolveArgs<real>& a, cudaStream_t st) {
  if (a.B == 0) return cudaSuccess;
  switch (a.dv.d) {
    case 1: return block_kind<real, 1>(a, st);
    case 2: return block_kind<real, 2>(a, st);
    case 4: return block_kind<real, 4>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_block_solve<float>(const BlockSolveArgs<float>&, cudaStream_t);
template cudaError_t launch_block_solve<double>(const BlockSolveArgs<double>&, cudaStream_t);

}  // namespace deer
