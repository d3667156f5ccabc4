// Fused full-Jacobian Newton iteration for state sizes d <= 8 (see FusedArgs in
// kernels.h). One pass over HBM per iteration: read A_t, b_t and s_t, write s_t and the new
// A_t, b_t; the chunk aggregates for the next scan are formed on the fly, so the scan's
// separate aggregate pass (another full read of the Jacobians) disappears.
#include "dyn.cuh"
#include "kernels.h"

namespace deer {

template <class real, int D>
__device__ __forceinline__ void ld_vec(const real* __restrict__ p, real (&v)[D]) {
  ldrow<real, D>(p, v);
}

template <class real, int D>
__device__ __forceinline__ void st_vec(real* __restrict__ p, const real (&v)[D]) {
  constexpr int bytes = D * (int)sizeof(real);
  if constexpr (bytes % 16 == 0) {
#pragma unroll
    for (int i = 0; i < bytes / 16; ++i)
      reinterpret_cast<float4*>(p)[i] = reinterpret_cast<const float4*>(v)[i];
  } else if constexpr (bytes % 8 == 0) {
#pragma unroll
    for (int i = 0; i < bytes / 8; ++i)
      reinterpret_cast<float2*>(p)[i] = reinterpret_cast<const float2*>(v)[i];
  } else {
#pragma unroll
    for (int i = 0; i < D; ++i) p[i] = v[i];
  }
}

// F = f_t(prev), A = df_t/ds at prev
template <class real, int D, int KIND>
__device__ __forceinline__ void lin_eval(const DynView<real>& dv, int64_t seq, int64_t row,
                                         const real (&prev)[D], real (&F)[D],
                                         real (&A)[D][D]) {
  if constexpr (KIND == DEER_F_MASSACTION_EULER || KIND == DEER_F_MASSACTION_RK4) {
    const real* T = dv.ma + seq * dv.ma_stride;
    ma_step_cols<real, D, 1, KIND == DEER_F_MASSACTION_RK4, true>(T, dv.dt, 0, prev, F, A);
  } else {
    eval_f<real, D, KIND, 1>(dv, seq, row, prev, F, A, nullptr);
  }
}

constexpr int kFusedBlock = 128;

template <class real, int D, int KIND, int MODE>
__global__ void __launch_bounds__(kFusedBlock) k_dense_fused(FusedArgs<real> a) {
  constexpr int E = D * D;
  // thread-private scratch: chunk aggregate P, v and the values that must survive the
  // register-heavy linearisation (Delta and the new state of the current row)
  __shared__ real sP[E][kFusedBlock];
  __shared__ real sV[D][kFusedBlock];
  __shared__ real sD[D][kFusedBlock];
  __shared__ real sN[D][kFusedBlock];
  const int tid = threadIdx.x;
  const int64_t ac = blockIdx.x * (int64_t)blockDim.x + tid;
  const bool valid = ac < a.bt.act_chunks();
  int64_t seq = 0;
  real mx = real(0), sq = real(0);  // residual statistics in the path's own precision
  unsigned long long key = 0ull;     // first failing row (sliding window)
  // the largest scaled residual |r| / max(1, |s|) is kept as the pair (|r|, max(1, |s|))
  // and divided out once per chunk: no division on the per-row dependent chain (float64
  // division is long on this GPU); the test |r| <= tol max(1, |s|) needs none either
  real mnum = real(0), mden = real(1);
  bool nan_seen = false;
  if (valid) {
    int64_t c, r0;
    int n;
    act_chunk(a.bt, ac, seq, c, r0, n);
    const int64_t base = __ldg(a.bt.offsets + seq);
    const int64_t gi = c >> 5;
    const int lane = (int)(c & 31);
    const int L = a.bt.L;
    // first chunk of the sequence (starts from s_0) / first solved chunk (starts from
    // Delta = 0; with a sliding window the rows before it are frozen)
    const bool seq_first = c == __ldg(a.bt.chunk_first + seq);
    const bool first = c == win_first(a.bt, seq);
    const bool need_P = !first;
    const real k = a.dparam;
    const real scale = a.damp == DEER_DAMP_SCALE ? real(1) - k : real(1);
    real prev[D];
    if (seq_first) {
#pragma unroll
      for (int i = 0; i < D; ++i) prev[i] = a.s0[seq * D + i];
    } else if (MODE == 0 || first) {
      ld_vec<real, D>(a.s + (r0 - 1) * D, prev);
    } else {
#pragma unroll
      for (int i = 0; i < D; ++i) prev[i] = a.sprev[c * D + i];
    }
#pragma unroll
    for (int i = 0; i < D; ++i) {
      sD[i][tid] = MODE == 1 ? a.cin[c * D + i] : real(0);
      sV[i][tid] = real(0);
#pragma unroll
      for (int j = 0; j < D; ++j) sP[i * D + j][tid] = i == j ? real(1) : real(0);
    }
    // small states: the next row's pending (A, b) and state are loaded one row ahead, so
    // their memory latency overlaps the current row's dependent arithmetic
    constexpr bool PF = D <= 4;
    constexpr int PE = MODE == 1 ? E : 1, PD = MODE == 1 ? D : 1;
    real fA[PF ? PE : 1], fb[PF ? PD : 1], fs[PF ? D : 1];
    auto fetch = [&](int t) {
      if constexpr (PF) {
        const real* Ar = a.Ai + ((gi * L + t) * E) * 32 + lane;
        const real* br = a.bi + ((gi * L + t) * D) * 32 + lane;
        if constexpr (MODE == 1) {
#pragma unroll
          for (int e = 0; e < E; ++e) fA[e] = Ar[e * 32];
#pragma unroll
          for (int i = 0; i < D; ++i) fb[i] = br[i * 32];
        }
#pragma unroll
        for (int i = 0; i < D; ++i) fs[i] = a.s[(r0 + t) * D + i];
      }
    };
    if (PF && n > 0) fetch(0);
    for (int t = 0; t < n; ++t) {
      const int64_t row = r0 + t;
      real* Arow = a.Ai + ((gi * L + t) * E) * 32 + lane;
      real* brow = a.bi + ((gi * L + t) * D) * 32 + lane;
      real sn[D], pA[PE], pb[PD];
      if constexpr (PF) {
#pragma unroll
        for (int i = 0; i < D; ++i) sn[i] = fs[i];
        if constexpr (MODE == 1) {
#pragma unroll
          for (int e = 0; e < E; ++e) pA[e] = fA[e];
#pragma unroll
          for (int i = 0; i < D; ++i) pb[i] = fb[i];
        }
        if (t + 1 < n) fetch(t + 1);
      } else {
        ld_vec<real, D>(a.s + row * D, sn);
        if constexpr (MODE == 1) {
#pragma unroll
          for (int e = 0; e < E; ++e) pA[e] = Arow[e * 32];
#pragma unroll
          for (int i = 0; i < D; ++i) pb[i] = brow[i * 32];
        }
      }
      if constexpr (MODE == 1) {
        // apply the pending scan step: Delta_t = A_t Delta_{t-1} + b_t, s_t += Delta_t
        real dl[D], nd[D];
#pragma unroll
        for (int i = 0; i < D; ++i) dl[i] = sD[i][tid];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          real v = pb[i];
#pragma unroll
          for (int j = 0; j < D; ++j) v += pA[i * D + j] * dl[j];
          nd[i] = v;
        }
#pragma unroll
        for (int i = 0; i < D; ++i) {
          sD[i][tid] = nd[i];
          real x = sn[i] + nd[i];
          if (a.reset && !(x <= a.reset_thr && x >= -a.reset_thr)) x = real(0);
          sn[i] = x;
        }
        st_vec<real, D>(a.s + row * D, sn);
      }
#pragma unroll
      for (int i = 0; i < D; ++i) sN[i][tid] = sn[i];
      // linearise at the new state of the previous row
      real F[D], A[D][D];
      lin_eval<real, D, KIND>(a.dv, seq, row, prev, F, A);
      real r[D];
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const real x = sN[i][tid];
        prev[i] = x;
        r[i] = x - F[i];
        const real sabs = rabs(x);
        const real m = sabs > real(1) ? sabs : real(1);
        const real ra = rabs(r[i]);
        if (ra * mden > mnum * m) { mnum = ra; mden = m; }
        nan_seen |= ra != ra;
        sq += r[i] * r[i];
        if (!(ra <= a.tol * m) && key == 0ull) key = bad_key(true, row - base);
      }
#pragma unroll
      for (int i = 0; i < D; ++i) {
        brow[i * 32] = -r[i];
#pragma unroll
        for (int j = 0; j < D; ++j) {
          A[i][j] *= scale;
          Arow[(i * D + j) * 32] = A[i][j];
        }
      }
      // chunk aggregate for the next scan: v <- A v - r, P <- A P (column by column)
      {
        real vv[D], nv[D];
#pragma unroll
        for (int i = 0; i < D; ++i) vv[i] = sV[i][tid];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          real x = -r[i];
#pragma unroll
          for (int j = 0; j < D; ++j) x += A[i][j] * vv[j];
          nv[i] = x;
        }
#pragma unroll
        for (int i = 0; i < D; ++i) sV[i][tid] = nv[i];
      }
      if (need_P) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
          real col[D], nc[D];
#pragma unroll
          for (int i = 0; i < D; ++i) col[i] = sP[i * D + j][tid];
#pragma unroll
          for (int i = 0; i < D; ++i) {
            real x = real(0);
#pragma unroll
            for (int m = 0; m < D; ++m) x += A[i][m] * col[m];
            nc[i] = x;
          }
#pragma unroll
          for (int i = 0; i < D; ++i) sP[i * D + j][tid] = nc[i];
        }
      }
    }
    real* Po = a.aggP + c * (int64_t)E;
    real* vo = a.aggv + c * D;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      vo[i] = sV[i][tid];
#pragma unroll
      for (int j = 0; j < D; ++j) Po[i * D + j] = sP[i * D + j][tid];
    }
  }
  mx = nan_seen ? real(NAN) : mnum / mden;
  acc_resid_t(a.acc, seq, valid, mx, sq, key);
}

// Row loads / stores through plain (coherent) accesses, for shared memory and for global
// data the same kernel also writes.
template <class real, int D>
__device__ __forceinline__ void ldrow_p(const real* p, real (&v)[D]) {
  if constexpr (sizeof(real) == 4 && D % 4 == 0) {
#pragma unroll
    for (int k = 0; k < D / 4; ++k) {
      const float4 q = reinterpret_cast<const float4*>(p)[k];
      v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
    }
  } else if constexpr (sizeof(real) == 8 && D % 2 == 0) {
#pragma unroll
    for (int k = 0; k < D / 2; ++k) {
      const double2 q = reinterpret_cast<const double2*>(p)[k];
      v[2 * k] = q.x; v[2 * k + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] = p[k];
  }
}

template <class real, int D>
__device__ __forceinline__ void strow_p(real* p, const real (&v)[D]) {
  if constexpr (sizeof(real) == 4 && D % 4 == 0) {
#pragma unroll
    for (int k = 0; k < D / 4; ++k)
      reinterpret_cast<float4*>(p)[k] =
          make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
  } else if constexpr (sizeof(real) == 8 && D % 2 == 0) {
#pragma unroll
    for (int k = 0; k < D / 2; ++k)
      reinterpret_cast<double2*>(p)[k] = make_double2(v[2 * k], v[2 * k + 1]);
  } else {
#pragma unroll
    for (int k = 0; k < D; ++k) p[k] = v[k];
  }
}
// Read-only row load (the per-sequence kinetics tensors) through the non-coherent path.
template <class real, int D>
__device__ __forceinline__ void ldrow_ro(const real* __restrict__ p, real (&v)[D]) {
  if constexpr (sizeof(real) == 4 && D % 4 == 0) {
#pragma unroll
    for (int k = 0; k < D / 4; ++k) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(p) + k);
      v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
    }
  } else if constexpr (sizeof(real) == 8 && D % 2 == 0) {
#pragma unroll
    for (int k = 0; k < D / 2; ++k) {
      const double2 q = __ldg(reinterpret_cast<const double2*>(p) + k);
      v[2 * k] = q.x; v[2 * k + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] = __ldg(p + k);
  }
}

// ---------------------------------------------------------------------------
// Lane-per-species variant for mass-action kinetics (d = 4, 8): a group of d lanes owns
// one chunk and lane i owns species i, i.e. row i of every d x d matrix of the row being
// processed (the rate Jacobian G, the stage Jacobian K, the accumulated sum of K, the new
// A_t and the chunk aggregate P). Values a lane needs from other species travel by
// shuffles (vectors) or through a small padded shared-memory buffer per group (matrix
// rows: K of the previous stage, P of the previous row). The work per row is the same as
// in the thread-per-chunk kernel, but each thread holds about a tenth of the registers,
// so far more warps are resident to hide latency. The pending (A_t, b_t) of a chunk are
// stored chunk-major: A at ((c L + t) d + i) d + j, b at (c L + t) d + i.
// ---------------------------------------------------------------------------
template <class real, int D, bool RK4, int MODE, bool CS>
__global__ void __launch_bounds__(kFusedBlock, 4) k_fused_ma_lps(FusedArgs<real> a) {
  constexpr int GPB = kFusedBlock / D;                  // chunks per block
  constexpr int E = D * D;
  // Exchange buffers: row stride D + 16 B and group stride + 16 B, so that the d lanes of a
  // group storing their rows, and the groups of a warp reading one row each, hit distinct
  // banks.
  constexpr int RS = D + 16 / (int)sizeof(real);
  constexpr int GS = D * RS + 16 / (int)sizeof(real);
  // B_m[i][:] for all m held in registers (float32), else re-read through L1 per stage
  constexpr bool BREG = sizeof(real) == 4;
  __shared__ __align__(16) real sK[GPB][GS];
  __shared__ __align__(16) real sP[GPB][GS];
  // per-lane prefetch ring (two rows): the pending row A_t[i][:] (mode 1), b_t[i] (mode 1),
  // s_t[i] and its compensation term, copied one row ahead with cp.async so that their
  // DRAM latency overlaps the previous row's work; each lane reads back only its own slot
  constexpr int PF = D + 4;
  __shared__ __align__(16) real sPF[2][kFusedBlock][PF];
  // the group's stage states (all species), exchanged through shared memory: written with
  // the stage Jacobian's rows, read back as two 16-byte pieces (instead of d shuffles)
  __shared__ __align__(16) real sC[GPB][D];
  const int grp = threadIdx.x / D, i = threadIdx.x % D;
  const unsigned gm = ((1u << D) - 1u) << ((threadIdx.x & 31) & ~(D - 1));
  const int64_t ac = blockIdx.x * (int64_t)GPB + grp;
  const bool valid = ac < a.bt.act_chunks();
  int64_t seq = 0;
  real mx = real(0), sq = real(0);  // residual statistics in the path's own precision
  unsigned long long key = 0ull;     // first failing row (sliding window)
  if (valid) {
    int64_t c, r0;
    int n;
    act_chunk(a.bt, ac, seq, c, r0, n);
    const int64_t base = __ldg(a.bt.offsets + seq);
    const int L = a.bt.L;
    // first chunk of the sequence (starts from s_0) / first solved chunk (starts from
    // Delta = 0; with a sliding window the rows before it are frozen)
    const bool seq_first = c == __ldg(a.bt.chunk_first + seq);
    const bool first = c == win_first(a.bt, seq);
    const real scale = a.damp == DEER_DAMP_SCALE ? real(1) - a.dparam : real(1);
    const real h = a.dv.dt;
    const real hw = RK4 ? h / real(6) : h;
    real* Kx = sK[grp];
    real* Px = sP[grp];
    real* Cx = sC[grp];
    const real* T = a.dv.ma + seq * a.dv.ma_stride;
    real Lrow[D];
    ldrow_ro<real, D>(T + i * D, Lrow);
    const real* Brow = T + E + i * D;  // B_m[i][:] at Brow + m E
    real Breg[BREG ? D : 1][BREG ? D : 1];
    if constexpr (BREG) {
#pragma unroll
      for (int m = 0; m < D; ++m) ldrow_ro<real, D>(Brow + m * E, Breg[m]);
    }
    // CS: the state is the pair (s, slo) (compensated float32 state, see cs_add)
    real prev, prev_lo = real(0);
    if (seq_first) {
      prev = a.s0[seq * D + i];
    } else if (MODE == 0 || first) {
      prev = a.s[(r0 - 1) * D + i];
      if constexpr (CS) prev_lo = a.slo[(r0 - 1) * D + i];
    } else {
      prev = a.sprev[c * D + i];
      if constexpr (CS) prev_lo = a.sprev_lo[c * D + i];
    }
    real dl = MODE == 1 ? a.cin[c * D + i] : real(0);
    real v = real(0);
#pragma unroll
    for (int j = 0; j < D; ++j) Px[i * RS + j] = i == j ? real(1) : real(0);
    Cx[i] = prev;  // the first row's first-stage states
    __syncwarp(gm);
    auto prefetch = [&](int slot, int t) {
      if (t < n) {
        real* q = sPF[slot][threadIdx.x];
        const int64_t row = r0 + t;
        if constexpr (MODE == 1) {
          const real* src = a.Ai + (c * L + t) * E + i * D;
#pragma unroll
          for (int k = 0; k < D * (int)sizeof(real) / 16; ++k)
            cp_async16(q + k * 16 / (int)sizeof(real), src + k * 16 / (int)sizeof(real));
          cp_async_small<sizeof(real)>(q + D, a.bi + (c * L + t) * D + i);
        }
        cp_async_small<sizeof(real)>(q + D + 1, a.s + row * D + i);
        if constexpr (CS) cp_async_small<sizeof(real)>(q + D + 2, a.slo + row * D + i);
      }
      cp_async_commit();
    };
    prefetch(0, 0);
    for (int t = 0; t < n; ++t) {
      const int64_t row = r0 + t;
      const int64_t pr = (c * L + t);
      real* Arow = a.Ai + pr * E + i * D;
      real* bp = a.bi + pr * D + i;
      prefetch((t + 1) & 1, t + 1);
      cp_async_wait<1>();  // this lane's copies of row t have landed
      const real* q = sPF[t & 1][threadIdx.x];
      real sn = q[D + 1];
      real sn_lo = real(0);
      if constexpr (CS) sn_lo = q[D + 2];
      if constexpr (MODE == 1) {
        // pending scan step: Delta_t = A_t Delta_{t-1} + b_t, s_t += Delta_t
        real Ar[D];
        ldrow_p<real, D>(q, Ar);
        real nd = q[D];
#pragma unroll
        for (int j = 0; j < D; ++j) nd += Ar[j] * __shfl_sync(gm, dl, j, D);
        dl = nd;
        if constexpr (CS) {
          cs_add(sn, sn_lo, nd);
          if (a.reset && !(sn <= a.reset_thr && sn >= -a.reset_thr)) {
            sn = real(0);
            sn_lo = real(0);
          }
          a.slo[row * D + i] = sn_lo;
        } else {
          real x = sn + nd;
          if (a.reset && !(x <= a.reset_thr && x >= -a.reset_thr)) x = real(0);
          sn = x;
        }
        a.s[row * D + i] = sn;
      }
      // linearise at the new state of the previous row
      real accg = real(0);
      real Kacc[D], Kown[D];
#pragma unroll
      for (int j = 0; j < D; ++j) Kacc[j] = real(0);
      constexpr int NST = RK4 ? 4 : 1;
#pragma unroll 1
      for (int stage = 0; stage < NST; ++stage) {
        // RK4 tableau: stage derivative weights (1, 2, 2, 1), stage offsets (h/2, h/2, h)
        const real cK = stage == 0 ? real(0) : (stage == 3 ? h : real(0.5) * h);
        const real w = (stage == 1 || stage == 2) ? real(2) : real(1);
        real cj[D], Gr[D];
        ldrow_p<real, D>(Cx, cj);  // this stage's states of every species
#pragma unroll
        for (int j = 0; j < D; ++j) Gr[j] = Lrow[j];
        if constexpr (BREG && D % 2 == 0) {
          // G row i = L_i + H c with H[m][j] = B_m[i][j] symmetric in (m, j) (second
          // derivatives of the rates): only H's 2 x 2 blocks on and above the diagonal are
          // read, so the compiler keeps 40 of its 64 entries in registers. A block below the
          // diagonal enters as the dot product of c's pair with a row of its mirror block,
          // accumulated in pairs and folded in at the end; the two-wide FMA count is the
          // dense one.
          float2 Tl[D / 2][2];
#pragma unroll
          for (int q = 0; q < D / 2; ++q) Tl[q][0] = Tl[q][1] = make_float2(0.f, 0.f);
#pragma unroll
          for (int p = 0; p < D / 2; ++p) {
            const float2 c2 = make_float2(cj[2 * p], cj[2 * p + 1]);
#pragma unroll
            for (int q = p; q < D / 2; ++q) {
              float2 y = make_float2(Gr[2 * q], Gr[2 * q + 1]);
              y = __ffma2_rn(make_float2(cj[2 * p], cj[2 * p]),
                             make_float2(Breg[2 * p][2 * q], Breg[2 * p][2 * q + 1]), y);
              y = __ffma2_rn(make_float2(cj[2 * p + 1], cj[2 * p + 1]),
                             make_float2(Breg[2 * p + 1][2 * q], Breg[2 * p + 1][2 * q + 1]), y);
              Gr[2 * q] = y.x;
              Gr[2 * q + 1] = y.y;
            }
#pragma unroll
            for (int q = 0; q < p; ++q) {
              Tl[q][0] = __ffma2_rn(c2, make_float2(Breg[2 * q][2 * p], Breg[2 * q][2 * p + 1]),
                                    Tl[q][0]);
              Tl[q][1] = __ffma2_rn(
                  c2, make_float2(Breg[2 * q + 1][2 * p], Breg[2 * q + 1][2 * p + 1]), Tl[q][1]);
            }
          }
#pragma unroll
          for (int q = 0; q < D / 2 - 1; ++q) {
            Gr[2 * q] += Tl[q][0].x + Tl[q][0].y;
            Gr[2 * q + 1] += Tl[q][1].x + Tl[q][1].y;
          }
        } else {
#pragma unroll
          for (int m = 0; m < D; ++m) {
            if constexpr (BREG) {
              axpy_row<D>(cj[m], Breg[m], Gr);
            } else {
              real bm[D];
              ldrow_ro<real, D>(Brow + m * E, bm);
              axpy_row<D>(cj[m], bm, Gr);
            }
          }
        }
        real g = real(0);
#pragma unroll
        for (int j = 0; j < D; ++j) g += (Lrow[j] + Gr[j]) * cj[j];
        g *= real(0.5);
        // K_s = G_s (I + cK K_{s-1}), row i; K_{s-1} rows come from the group buffer
#pragma unroll
        for (int j = 0; j < D; ++j) Kown[j] = Gr[j];
        if (stage > 0) {
#pragma unroll
          for (int m = 0; m < D; ++m) {
            real km[D];
            ldrow_p<real, D>(Kx + m * RS, km);
            axpy_row<D>(cK * Gr[m], km, Kown);
          }
        }
        // the next stage's state of this species (after the last stage: the row's new
        // state, the next row's first-stage state)
        const real cs = stage == 2 ? h : real(0.5) * h;
        const real st_next = stage == NST - 1 ? sn : prev + cs * g;
        __syncwarp(gm);
        strow_p<real, D>(Kx + i * RS, Kown);
        Cx[i] = st_next;
        __syncwarp(gm);
        axpy_row<D>(w, Kown, Kacc);
        accg += w * g;
      }
      real r;
      if constexpr (CS) {
        r = cs_residual(sn, sn_lo, prev, prev_lo, hw * accg);
      } else {
        const real F = prev + hw * accg;
        r = sn - F;
      }
      const real sabs = rabs(sn);
      const real sr = rabs(r) / (sabs > real(1) ? sabs : real(1));
      mx = (sr > mx || sr != sr) ? sr : mx;
      sq += r * r;
      if (!(sr <= a.tol) && key == 0ull) key = bad_key(true, row - base);
      real An[D];
#pragma unroll
      for (int j = 0; j < D; ++j) An[j] = scale * (hw * Kacc[j] + (j == i ? real(1) : real(0)));
      strow_p<real, D>(Arow, An);
      *bp = -r;
      // chunk aggregate for the next scan: v <- A v - r, P <- A P
      real nv = -r;
#pragma unroll
      for (int j = 0; j < D; ++j) nv += An[j] * __shfl_sync(gm, v, j, D);
      v = nv;
      if (!first) {
        real np[D];
#pragma unroll
        for (int j = 0; j < D; ++j) np[j] = real(0);
#pragma unroll
        for (int m = 0; m < D; ++m) {
          real pm[D];
          ldrow_p<real, D>(Px + m * RS, pm);
          axpy_row<D>(An[m], pm, np);
        }
        __syncwarp(gm);
        strow_p<real, D>(Px + i * RS, np);
        __syncwarp(gm);
      }
      prev = sn;
      prev_lo = sn_lo;
    }
    cp_async_wait<0>();
    real pf[D];
    ldrow_p<real, D>(Px + i * RS, pf);
    strow_p<real, D>(a.aggP + c * (int64_t)E + i * D, pf);
    a.aggv[c * D + i] = v;
  }
  // one accumulator update per chunk: reduce over the group's species first
#pragma unroll
  for (int o = D / 2; o > 0; o >>= 1) {
    const real om = __shfl_xor_sync(0xffffffffu, mx, o, D);
    mx = (om > mx || om != om) ? om : mx;
    sq += __shfl_xor_sync(0xffffffffu, sq, o, D);
    const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, o, D);
    key = ok > key ? ok : key;
  }
  acc_resid_t(a.acc, seq, valid && i == 0, mx, sq, key);
}

// Per active sequence: compose the chunk aggregates in order; record the Delta entering
// each chunk and the new state at the row before it (read from the old iterate before the
// fused pass overwrites it).
template <class real, int D>
__global__ void __launch_bounds__(128) k_dense_fused_carry(FusedArgs<real> a) {
  constexpr int E = D * D;
  // aggregates and state rows loaded K chunks ahead (register ring of about 64 32-bit
  // registers: deep for d <= 2, one chunk ahead for d = 8, whose aggregate is 64 values)
  constexpr int V = (E + 2 * D) * (int)(sizeof(real) / 4);
  constexpr int K = V >= 64 ? 1 : (64 / V > 8 ? 8 : 64 / V);
  const int64_t kq = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (kq >= a.bt.n_act()) return;
  const int64_t seq = a.bt.act_seq[kq];
  const int64_t cf = a.bt.chunk_first[seq], c0 = win_first(a.bt, seq);
  const int64_t c1 = a.bt.chunk_first[seq + 1];
  const int64_t base = a.bt.offsets[seq];
  real x[D];
#pragma unroll
  for (int i = 0; i < D; ++i) x[i] = real(0);
  real Pr[K][E], vr[K][D], sr[K][D];
  auto fetch = [&](int slot, int64_t c) {
    if (c < c1) {
#pragma unroll
      for (int e = 0; e < E; ++e) Pr[slot][e] = a.aggP[c * E + e];
#pragma unroll
      for (int i = 0; i < D; ++i) vr[slot][i] = a.aggv[c * D + i];
      if (c > c0) {
        const int64_t r0 = base + ((c - cf) << a.bt.log2L);
#pragma unroll
        for (int i = 0; i < D; ++i) sr[slot][i] = a.s[(r0 - 1) * D + i];
      }
    }
  };
#pragma unroll
  for (int slot = 0; slot < K; ++slot) fetch(slot, c0 + slot);
  for (int64_t cb = c0; cb < c1; cb += K) {
#pragma unroll
    for (int slot = 0; slot < K; ++slot) {
      const int64_t c = cb + slot;
      if (c >= c1) break;
      real Pc[E], vc[D], so[D];
#pragma unroll
      for (int e = 0; e < E; ++e) Pc[e] = Pr[slot][e];
#pragma unroll
      for (int i = 0; i < D; ++i) { vc[i] = vr[slot][i]; so[i] = sr[slot][i]; }
      fetch(slot, c + K);
#pragma unroll
      for (int i = 0; i < D; ++i) a.cin[c * D + i] = x[i];
      if (c > c0) {
#pragma unroll
        for (int i = 0; i < D; ++i) {
          real y = so[i] + x[i];
          if (a.reset && !(y <= a.reset_thr && y >= -a.reset_thr)) y = real(0);
          a.sprev[c * D + i] = y;
        }
      }
      real nx[D];
#pragma unroll
      for (int i = 0; i < D; ++i) {
        real y = vc[i];
        if (c > c0) {
#pragma unroll
          for (int j = 0; j < D; ++j) y += Pc[i * D + j] * x[j];
        }
        nx[i] = y;
      }
#pragma unroll
      for (int i = 0; i < D; ++i) x[i] = nx[i];
    }
  }
}

// Lane-per-species carry pass (d = 4, 8): d lanes per sequence, lane i owns row i of every
// chunk aggregate and entry i of the carried Delta; the other entries arrive by shuffles.
// The next chunk's aggregate row is loaded before the current one is applied.
template <class real, int D, bool CS>
__global__ void __launch_bounds__(128) k_fused_carry_lps(FusedArgs<real> a) {
  constexpr int E = D * D;
  constexpr int GPB = 128 / D;
  // the chunk aggregates and the state rows before the chunks do not depend on the carry:
  // they are loaded K chunks ahead (a register ring), so the dependent chain costs one
  // matrix-vector product per chunk instead of one memory round trip
  constexpr int K = sizeof(real) == 4 ? 8 : 4;
  const int grp = threadIdx.x / D, i = threadIdx.x % D;
  const unsigned gm = ((1u << D) - 1u) << ((threadIdx.x & 31) & ~(D - 1));
  const int64_t kq = blockIdx.x * (int64_t)GPB + grp;
  if (kq >= a.bt.n_act()) return;  // whole groups
  const int64_t seq = a.bt.act_seq[kq];
  const int64_t cf = a.bt.chunk_first[seq], c0 = win_first(a.bt, seq);
  const int64_t c1 = a.bt.chunk_first[seq + 1];
  const int64_t base = a.bt.offsets[seq];
  real Pr[K][D], vr[K], sr[K], sl[CS ? K : 1];
  auto fetch = [&](int slot, int64_t c) {
    if (c < c1) {
      ldrow_p<real, D>(a.aggP + c * E + i * D, Pr[slot]);
      vr[slot] = a.aggv[c * D + i];
      const int64_t rb = base + ((c - cf) << a.bt.log2L) - 1;
      sr[slot] = c > c0 ? a.s[rb * D + i] : real(0);
      if constexpr (CS) sl[slot] = c > c0 ? a.slo[rb * D + i] : real(0);
    }
  };
#pragma unroll
  for (int slot = 0; slot < K; ++slot) fetch(slot, c0 + slot);
  real x = real(0);
  for (int64_t cb = c0; cb < c1; cb += K) {
#pragma unroll
    for (int slot = 0; slot < K; ++slot) {
      const int64_t c = cb + slot;
      if (c < c1) {  // uniform over the group
        real Pc[D];
#pragma unroll
        for (int j = 0; j < D; ++j) Pc[j] = Pr[slot][j];
        const real vc = vr[slot], so = sr[slot];
        real so_lo = real(0);
        if constexpr (CS) so_lo = sl[slot];
        fetch(slot, c + K);
        a.cin[c * D + i] = x;
        real nx = vc;
        if (c > c0) {
          if constexpr (CS) {
            real y = so, ylo = so_lo;
            cs_add(y, ylo, x);
            if (a.reset && !(y <= a.reset_thr && y >= -a.reset_thr)) {
              y = real(0);
              ylo = real(0);
            }
            a.sprev[c * D + i] = y;
            a.sprev_lo[c * D + i] = ylo;
          } else {
            real y = so + x;
            if (a.reset && !(y <= a.reset_thr && y >= -a.reset_thr)) y = real(0);
            a.sprev[c * D + i] = y;
          }
#pragma unroll
          for (int j = 0; j < D; ++j) nx += Pc[j] * __shfl_sync(gm, x, j, D);
        }
        x = nx;
      }
    }
  }
}

template <class real, int D, int KIND>
static void fused_launch(const FusedArgs<real>& a, cudaStream_t st) {
  constexpr bool MA = KIND == DEER_F_MASSACTION_EULER || KIND == DEER_F_MASSACTION_RK4;
  if constexpr (MA && (D == 4 || D == 8)) {
    constexpr bool RK4 = KIND == DEER_F_MASSACTION_RK4;
    const unsigned g = grid_for(a.bt.act_chunks(), kFusedBlock / D);
    if (a.slo) {
      if (a.mode == 0) k_fused_ma_lps<real, D, RK4, 0, true><<<g, kFusedBlock, 0, st>>>(a);
      else k_fused_ma_lps<real, D, RK4, 1, true><<<g, kFusedBlock, 0, st>>>(a);
    } else {
      if (a.mode == 0) k_fused_ma_lps<real, D, RK4, 0, false><<<g, kFusedBlock, 0, st>>>(a);
      else k_fused_ma_lps<real, D, RK4, 1, false><<<g, kFusedBlock, 0, st>>>(a);
    }
  } else {
    const unsigned g = grid_for(a.bt.act_chunks(), kFusedBlock);
    if (a.mode == 0) k_dense_fused<real, D, KIND, 0><<<g, kFusedBlock, 0, st>>>(a);
    else k_dense_fused<real, D, KIND, 1><<<g, kFusedBlock, 0, st>>>(a);
  }
}

template <class real, int KIND>
static cudaError_t fused_kind(const FusedArgs<real>& a, cudaStream_t st) {
  switch (a.dv.d) {
    case 1: if constexpr (KIND != DEER_F_BRUSSELATOR_EULER) { fused_launch<real, 1, KIND>(a, st); break; }
            return cudaErrorInvalidValue;
    case 2: fused_launch<real, 2, KIND>(a, st); break;
    case 4: if constexpr (KIND != DEER_F_BRUSSELATOR_EULER) { fused_launch<real, 4, KIND>(a, st); break; }
            return cudaErrorInvalidValue;
    case 8: if constexpr (KIND != DEER_F_BRUSSELATOR_EULER) { fused_launch<real, 8, KIND>(a, st); break; }
            return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
  note_launch();
  return cudaGetLastError();
}

template <class real>
cudaError_t launch_dense_fused(const FusedArgs<real>& a, cudaStream_t st) {
  if (a.bt.act_chunks() == 0) return cudaSuccess;
  switch (a.dv.kind) {
    case DEER_F_BRUSSELATOR_EULER: return fused_kind<real, DEER_F_BRUSSELATOR_EULER>(a, st);
    case DEER_F_MASSACTION_EULER: return fused_kind<real, DEER_F_MASSACTION_EULER>(a, st);
    case DEER_F_MASSACTION_RK4: return fused_kind<real, DEER_F_MASSACTION_RK4>(a, st);
    case DEER_F_GRU: return fused_kind<real, DEER_F_GRU>(a, st);
    default: return fused_kind<real, DEER_F_LINEAR>(a, st);
  }
}

template <class real>
cudaError_t launch_dense_fused_carry(const FusedArgs<real>& a, cudaStream_t st) {
  if (a.bt.n_act() == 0) return cudaSuccess;
  const bool ma = a.dv.kind == DEER_F_MASSACTION_EULER || a.dv.kind == DEER_F_MASSACTION_RK4;
  if (ma && (a.dv.d == 4 || a.dv.d == 8)) {
    // same kernels as the fused pass selects (lane-per-species layout of the aggregates is
    // row-major either way)
    if (a.slo) {
      if (a.dv.d == 4) k_fused_carry_lps<real, 4, true><<<grid_for(a.bt.n_act(), 32), 128, 0, st>>>(a);
      else k_fused_carry_lps<real, 8, true><<<grid_for(a.bt.n_act(), 16), 128, 0, st>>>(a);
    } else {
      if (a.dv.d == 4) k_fused_carry_lps<real, 4, false><<<grid_for(a.bt.n_act(), 32), 128, 0, st>>>(a);
      else k_fused_carry_lps<real, 8, false><<<grid_for(a.bt.n_act(), 16), 128, 0, st>>>(a);
    }
    note_launch();
    return cudaGetLastError();
  }
  const unsigned g = grid_for(a.bt.n_act(), 128);
  switch (a.dv.d) {
    case 1: k_dense_fused_carry<real, 1><<<g, 128, 0, st>>>(a); break;
    case 2: k_dense_fused_carry<real, 2><<<g, 128, 0, st>>>(a); break;
    case 4: k_dense_fused_carry<real, 4><<<g, 128, 0, st>>>(a); break;
    case 8: k_dense_fused_carry<real, 8><<<g, 128, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  note_launch();
  return cudaGetLastError();
}

template cudaError_t launch_dense_fused<float>(const FusedArgs<float>&, cudaStream_t);
template cudaError_t launch_dense_fused<double>(const FusedArgs<double>&, cudaStream_t);
template cudaError_t launch_dense_fused_carry<float>(const FusedArgs<float>&, cudaStream_t);
template cudaError_t launch_dense_fused_carry<double>(const FusedArgs<double>&, cudaStream_t);

}  // namespace deer
