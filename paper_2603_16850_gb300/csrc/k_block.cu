// Whole Newton solve of a short sequence inside one thread-block cluster (Algorithm 1 with
// the full Jacobian): one cluster per sequence runs every iteration itself,
// linearisation, convergence test and the scan of Eq. bin_op_affine, with the iterate
// kept in registers. There is no launch and no host round trip per iteration, and a
// batch of short sequences is one launch in which every cluster stops on its own
// convergence.
//
// The cluster's threads own contiguous rows of the sequence in (block rank, thread)
// order, R rows each. One iteration:
//   1. each thread evaluates F_t = f_t(s_{t-1}) and A_t on its rows (the row before its
//      first comes from the previous thread through shared memory, from the previous
//      block's shared memory for thread 0, s_0 at the start), forms the residual
//      r_t = s_t - F_t and composes its rows' affine steps Delta -> A_t Delta - r_t into
//      one element (P, v);
//   2. a reduction over the cluster gives the largest scaled residual max |r| / max(1, |s|)
//      and sum r^2, and, behind the same cluster barrier, an exclusive scan of the
//      elements (warp shuffles, the warp totals, then the blocks' totals read across the
//      cluster) gives the correction Delta entering each thread's rows;
//   3. the test and the iteration count follow the library's convergence check, taken
//      identically by every block; unless it stops, each thread propagates Delta through
//      its rows with the A_t and F_t it kept, adding it to the iterate with the reset
//      heuristic.
// Two cluster barriers per iteration: the boundary rows, then statistics and scan totals.
#include <cooperative_groups.h>

#include <cfloat>

#include "dyn.cuh"
#include "kernels.h"

namespace deer {

template <class real>
constexpr real kRealMax = sizeof(real) == 8 ? real(DBL_MAX) : real(FLT_MAX);

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

// inclusive scan over the first n lanes of a warp (lane order = time order; n <= 32, the
// steps stop at the first power of two >= n: every float64 product counts on this GPU)
template <class real, int D>
__device__ __forceinline__ Aff<real, D> warp_scan_aff(Aff<real, D> x, int lane, int n = 32) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    if (off >= n) break;  // uniform over the warp
    const Aff<real, D> y = shfl_up_aff<real, D>(x, off);
    if (lane >= off) x = compose<real, D>(x, y);
  }
  return x;
}

template <class real, int D, int KIND, int NT, int RPT>
__global__ void __launch_bounds__(NT) k_block_solve(BlockSolveArgs<real> a) {
  namespace cg = cooperative_groups;
  constexpr int NW = NT / 32;
  __shared__ real s_last[NT][D];       // each thread's last row of the iterate
  __shared__ Aff<real, D> s_warp[NW];  // inclusive warp totals, then their prefixes
  __shared__ Aff<real, D> s_tot;       // this block's element (read by later blocks)
  __shared__ real s_mx[NW];
  __shared__ double s_sq[NW];
  __shared__ double s_part[2];         // this block's max scaled residual and sum r^2
  __shared__ double s_stat[2];         // the cluster's
  __shared__ real s_din[D];            // Delta entering this block's rows
  cg::cluster_group cl = cg::this_cluster();
  const int CL = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int64_t seq = blockIdx.x / CL;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r0 = a.offsets[seq];
  const int64_t T = a.offsets[seq + 1] - r0;
  // rows spread evenly over the cluster's blocks (rpc each, in rank order), then over a
  // block's threads (rpt each, <= RPT: the host sizes the cluster); the threads with rows
  // are a prefix of each block, and whole warps without rows skip the float64 scans
  const int64_t rpc = (T + CL - 1) / CL;
  const int rpt = (int)((rpc + NT - 1) / NT);
  const int64_t cbeg = (int64_t)rank * rpc;
  const int64_t cend = cbeg + rpc < T ? cbeg + rpc : T;
  const int64_t k0 = cbeg + (int64_t)tid * rpt;
  const int nmine = cend - k0 <= 0 ? 0 : (cend - k0 < rpt ? (int)(cend - k0) : rpt);
  const bool warp_rows = cbeg + (int64_t)(warp * 32) * rpt < cend;  // uniform over the warp
  // the previous block (full whenever this one has rows) ends with thread (rpc - 1) / rpt
  // (an empty sequence has rpt = 0 and no thread with rows: nothing is read)
  const int prev_last = rpt > 0 ? (int)((rpc - 1) / rpt) : 0;
  const real scale = a.damp == DEER_DAMP_SCALE ? real(1) - a.dparam : real(1);
  real s[RPT][D];
  real s0[D];
#pragma unroll
  for (int i = 0; i < D; ++i) s0[i] = a.s0[seq * D + i];
#pragma unroll
  for (int k = 0; k < RPT; ++k)
#pragma unroll
    for (int i = 0; i < D; ++i) s[k][i] = k < nmine ? a.s[(r0 + k0 + k) * D + i] : real(0);
  int passes = 0;
  bool done = false, nonfinite = false;
  double merit = 0.0, mres = 0.0;
  int iters = 0;
  for (int it = 0;; ++it) {
    // the row before this thread's first is the previous thread's last, in this block or
    // (thread 0) in the previous block of the cluster; a thread without rows is followed
    // only by threads without rows
#pragma unroll
    for (int k = 0; k < RPT; ++k)
      if (k == nmine - 1) {
#pragma unroll
        for (int i = 0; i < D; ++i) s_last[tid][i] = s[k][i];
      }
    cl.sync();
    real prev[D];
    if (nmine == 0) {
#pragma unroll
      for (int i = 0; i < D; ++i) prev[i] = real(0);  // unused: no rows
    } else if (tid > 0) {
#pragma unroll
      for (int i = 0; i < D; ++i) prev[i] = s_last[tid - 1][i];
    } else if (rank > 0) {
      const real* pl = cl.map_shared_rank(&s_last[prev_last][0], rank - 1);
#pragma unroll
      for (int i = 0; i < D; ++i) prev[i] = pl[i];
    } else {
#pragma unroll
      for (int i = 0; i < D; ++i) prev[i] = s0[i];
    }
    // 1. linearise, residual statistics, this thread's element; F and A are kept for the
    //    apply pass
    Aff<real, D> e = aff_identity<real, D>();
    real Fk[RPT][D], Ak[RPT][D][D];
    // largest scaled residual |r| / max(1, |s|) kept as a fraction (fn / fd, compared by
    // cross-multiplication), so that one division per warp replaces one per entry (the
    // float64 divide is a long sequence on this GPU); non-finite entries raise fnan
    real fn = real(0), fd = real(1);
    bool fnan = false;
    double sq = 0.0;
    {
      real sp[D];
#pragma unroll
      for (int i = 0; i < D; ++i) sp[i] = prev[i];
#pragma unroll
      for (int k = 0; k < RPT; ++k) {
        if (k < nmine) {
          eval_f<real, D, KIND, 1>(a.dv, seq, r0 + k0 + k, sp, Fk[k], Ak[k], nullptr);
          Aff<real, D> st;
#pragma unroll
          for (int i = 0; i < D; ++i) {
            const real r = s[k][i] - Fk[k][i];
            st.v[i] = -r;
            const real sabs = rabs(s[k][i]);
            const real num = rabs(r), den = sabs > real(1) ? sabs : real(1);
            if (!(num <= kRealMax<real>) || !(den <= kRealMax<real>)) {
              fnan = true;
            } else if (num * fd > fn * den) {
              fn = num;
              fd = den;
            }
            sq += (double)r * (double)r;
#pragma unroll
            for (int j = 0; j < D; ++j) {
              Ak[k][i][j] *= scale;
              st.P[i][j] = Ak[k][i][j];
            }
          }
          e = compose<real, D>(st, e);
#pragma unroll
          for (int i = 0; i < D; ++i) sp[i] = s[k][i];
        }
      }
    }
    // 2. statistics and scan totals: per warp, per block, then across the cluster with one
    //    barrier. Every block reduces the blocks' partials in the same order, so all take
    //    the same decision; the scan is formed before the test and unused if it stops.
    if (warp_rows) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const real on = __shfl_xor_sync(0xffffffffu, fn, o);
        const real od = __shfl_xor_sync(0xffffffffu, fd, o);
        fnan |= __shfl_xor_sync(0xffffffffu, (int)fnan, o) != 0;
        if (on * fd > fn * od) {
          fn = on;
          fd = od;
        }
        sq += __shfl_xor_sync(0xffffffffu, sq, o);
      }
      if (lane == 0) {
        s_mx[warp] = fnan ? real(NAN) : fn / fd;
        s_sq[warp] = sq;
      }
    } else if (lane == 0) {
      s_mx[warp] = real(0);
      s_sq[warp] = 0.0;
    }
    // 3. scan of the elements: lanes, warps, then the blocks of the cluster
    const Aff<real, D> inc = warp_rows ? warp_scan_aff<real, D>(e, lane) : e;  // e = I
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      Aff<real, D> wt = lane < NW ? s_warp[lane] : aff_identity<real, D>();
      wt = warp_scan_aff<real, D>(wt, lane, NW);
      if (lane < NW) s_warp[lane] = wt;
      if (lane == NW - 1) s_tot = wt;
      double bm = lane < NW ? (double)s_mx[lane] : 0.0;
      double bs = lane < NW ? s_sq[lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        bm = nanmax(bm, __shfl_xor_sync(0xffffffffu, bm, o));
        bs += __shfl_xor_sync(0xffffffffu, bs, o);
      }
      if (lane == 0) {
        s_part[0] = bm;
        s_part[1] = bs;
      }
    }
    cl.sync();
    if (warp == 0) {
      double bm = 0.0, bs = 0.0;
      if (lane < CL) {
        const double* pp = cl.map_shared_rank(&s_part[0], lane);
        bm = pp[0];
        bs = pp[1];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        bm = nanmax(bm, __shfl_xor_sync(0xffffffffu, bm, o));
        bs += __shfl_xor_sync(0xffffffffu, bs, o);
      }
      if (lane == 0) {
        s_stat[0] = bm;
        s_stat[1] = bs;
      }
      // the blocks before this one, composed in order: Delta entering this block
      Aff<real, D> bt = lane < CL ? *cl.map_shared_rank(&s_tot, lane) : aff_identity<real, D>();
      bt = warp_scan_aff<real, D>(bt, lane, CL);
      const Aff<real, D> ex = shfl_up_aff<real, D>(bt, 1);
      if (lane == rank) {
#pragma unroll
        for (int i = 0; i < D; ++i) s_din[i] = rank > 0 ? ex.v[i] : real(0);
      }
    }
    __syncthreads();
    const double bm = s_stat[0], bs = s_stat[1];
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
    real din[D] = {};
    if (warp_rows) {
      // then the warps before in this block, then the lanes before in this warp
      real db[D], dw[D];
#pragma unroll
      for (int i = 0; i < D; ++i) db[i] = s_din[i];
      if (warp > 0) {
        const Aff<real, D>& wp = s_warp[warp - 1];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          real x = wp.v[i];
#pragma unroll
          for (int k = 0; k < D; ++k) x += wp.P[i][k] * db[k];
          dw[i] = x;
        }
      } else {
#pragma unroll
        for (int i = 0; i < D; ++i) dw[i] = db[i];
      }
      Aff<real, D> ex = shfl_up_aff<real, D>(inc, 1);
      if (lane == 0) ex = aff_identity<real, D>();
#pragma unroll
      for (int i = 0; i < D; ++i) {
        real x = ex.v[i];
#pragma unroll
        for (int k = 0; k < D; ++k) x += ex.P[i][k] * dw[k];
        din[i] = x;
      }
    }
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      if (k < nmine) {
        real dn[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          real x = Fk[k][i] - s[k][i];
#pragma unroll
          for (int j = 0; j < D; ++j) x += Ak[k][i][j] * din[j];
          dn[i] = x;
        }
#pragma unroll
        for (int i = 0; i < D; ++i) {
          const real y = s[k][i] + dn[i];
          s[k][i] = (a.reset && !(y <= a.reset_thr && y >= -a.reset_thr)) ? real(0) : y;
          din[i] = dn[i];
        }
      }
    }
    // (the next iteration's first cluster barrier orders the rewrites of the shared
    // buffers after every block's reads of them)
  }
  cl.sync();  // no block leaves while another may still read its shared memory
#pragma unroll
  for (int k = 0; k < RPT; ++k)
    if (k < nmine)
#pragma unroll
      for (int i = 0; i < D; ++i) a.s[(r0 + k0 + k) * D + i] = s[k][i];
  if (tid == 0 && rank == 0) {
    SeqInfo inf = a.info[seq];
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

// Threads per block and the most rows per thread by state size (each thread keeps its
// rows' iterate, F_t and A_t in registers). A sequence is spread over a cluster of up to
// 16 blocks (one row per thread where it fits), whose shared memory the blocks read from
// each other: the more SMs, the more of the GPU's float64 units (a small fraction of its
// float32 rate) a single sequence gets.
constexpr int kBlockThreads = 128;
constexpr int kMaxCluster = 8;    // portable cluster size: sets the longest sequence taken
constexpr int kWideCluster = 16;  // non-portable, used when the GPU schedules it
template <int D>
struct BlockRows { static constexpr int n = D <= 2 ? 8 : 2; };

int64_t block_solve_max_T(int kind, int d) {
  const bool kind_ok = kind == DEER_F_BRUSSELATOR_EULER || kind == DEER_F_MASSACTION_EULER ||
                       kind == DEER_F_MASSACTION_RK4 || kind == DEER_F_LINEAR ||
                       kind == DEER_F_RNN_TANH || kind == DEER_F_LANGEVIN_2WELL;
  if (!kind_ok) return 0;
  const int64_t per = (int64_t)kMaxCluster * kBlockThreads;
  switch (d) {
    case 1: return per * BlockRows<1>::n;
    case 2: return per * BlockRows<2>::n;
    case 4: return per * BlockRows<4>::n;
    default: return 0;
  }
}

template <class real, int D, int KIND>
static cudaError_t block_launch(const BlockSolveArgs<real>& a, cudaStream_t st) {
  auto kern = k_block_solve<real, D, KIND, kBlockThreads, BlockRows<D>::n>;
  // cluster size: 64 rows per block where the longest sequence allows it (the float64
  // pipe is the SM's, shared by its warps), up to 16 blocks when the GPU can schedule
  // that, else 8
  int64_t cl = (a.max_T + kBlockThreads / 2 - 1) / (kBlockThreads / 2);
  cl = cl < 1 ? 1 : (cl > kWideCluster ? kWideCluster : cl);
  if (cl > kMaxCluster) {
    static thread_local int wide_ok = -1;  // per host thread: 1 if the attribute took
    if (wide_ok < 0)
      wide_ok = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                     1) == cudaSuccess ? 1 : 0;
    if (!wide_ok) cl = kMaxCluster;
    (void)cudaGetLastError();
  }
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg{};
  cfg.blockDim = dim3(kBlockThreads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  for (;;) {
    attr[0].val.clusterDim.x = (unsigned)cl;
    cfg.gridDim = dim3((unsigned)(a.B * cl), 1, 1);
    // a cluster of 16 that cannot be placed: take 8 instead (the longest sequence taken
    // fits 8)
    if (cl > kMaxCluster) {
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess ||
          nclusters < 1) {
        (void)cudaGetLastError();
        cl = kMaxCluster;
        continue;
      }
    }
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, a);
    if (e != cudaSuccess && cl > kMaxCluster) {
      (void)cudaGetLastError();
      cl = kMaxCluster;
      continue;
    }
    if (e == cudaSuccess) note_launch();
    return e;
  }
}

template <class real, int D>
static cudaError_t block_kind(const BlockSolveArgs<real>& a, cudaStream_t st) {
  switch (a.dv.kind) {
    case DEER_F_BRUSSELATOR_EULER:
      if constexpr (D == 2) return block_launch<real, D, DEER_F_BRUSSELATOR_EULER>(a, st);
      return cudaErrorInvalidValue;
    case DEER_F_MASSACTION_EULER:
      if constexpr (D >= 2) return block_launch<real, D, DEER_F_MASSACTION_EULER>(a, st);
      return cudaErrorInvalidValue;
    case DEER_F_MASSACTION_RK4:
      if constexpr (D >= 2) return block_launch<real, D, DEER_F_MASSACTION_RK4>(a, st);
      return cudaErrorInvalidValue;
    case DEER_F_LINEAR: return block_launch<real, D, DEER_F_LINEAR>(a, st);
    case DEER_F_RNN_TANH: return block_launch<real, D, DEER_F_RNN_TANH>(a, st);
    case DEER_F_LANGEVIN_2WELL: return block_launch<real, D, DEER_F_LANGEVIN_2WELL>(a, st);
    default: return cudaErrorInvalidValue;
  }
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
