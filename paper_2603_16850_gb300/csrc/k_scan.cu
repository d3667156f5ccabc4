// Convergence check and the chunked parallel scans (dense and diagonal families).
//
// Scan structure (three phases, no host involvement): every chunk of L consecutive rows
// of one sequence is reduced to its aggregate under the affine composition of Eq.
// bin_op_affine, (A_j, b_j) o (A_i, b_i) = (A_j A_i, b_j + A_j b_i); a per-sequence pass
// composes the chunk aggregates in order (the operation does not commute) to obtain the
// state entering every chunk; a final pass re-runs each chunk from its carry.
#include <cfloat>

#include "kernels.h"
#include "tc.cuh"

namespace deer {

// ----------------------------------------------------------------------------
// Convergence / merit (one block): per sequence max |r| / max(1, |s|) vs tol, merit
// 1/2 |r|^2; then the sequences still iterating are compacted (in order) into the active
// lists that size and index every later launch. Thread t owns a contiguous range of
// sequences so that a block-wide exclusive scan gives each its output offsets.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void block_excl_scan3(long long& a, long long& b, long long& c,
                                                 long long& ta, long long& tb, long long& tc) {
  __shared__ long long sa[32], sb[32], sc[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned full = 0xffffffffu;
  long long ia = a, ib = b, ic = c;  // inclusive warp scan
  for (int o = 1; o < 32; o <<= 1) {
    long long xa = __shfl_up_sync(full, ia, o), xb = __shfl_up_sync(full, ib, o),
              xc = __shfl_up_sync(full, ic, o);
    if (lane >= o) { ia += xa; ib += xb; ic += xc; }
  }
  if (lane == 31) { sa[warp] = ia; sb[warp] = ib; sc[warp] = ic; }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    long long va = lane < nw ? sa[lane] : 0, vb = lane < nw ? sb[lane] : 0,
              vc = lane < nw ? sc[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      long long xa = __shfl_up_sync(full, va, o), xb = __shfl_up_sync(full, vb, o),
                xc = __shfl_up_sync(full, vc, o);
      if (lane >= o) { va += xa; vb += xb; vc += xc; }
    }
    if (lane < nw) { sa[lane] = va; sb[lane] = vb; sc[lane] = vc; }
  }
  __syncthreads();
  const int nw = blockDim.x >> 5;
  const long long wa = warp > 0 ? sa[warp - 1] : 0, wb = warp > 0 ? sb[warp - 1] : 0,
                  wc = warp > 0 ? sc[warp - 1] : 0;
  ta = sa[nw - 1]; tb = sb[nw - 1]; tc = sc[nw - 1];
  a = wa + ia - a; b = wb + ib - b; c = wc + ic - c;
}

// whether the Newton loop goes on after the check of iteration `it` (the host loop's
// stopping rules, evaluated on the device)
__device__ __forceinline__ bool loop_goes_on(const Flags* f, int it, int max_iters,
                                             int reset) {
  if (f->bad_input || f->timeout) return false;
  if (f->n_nonfinite > 0 && !reset) return false;
  if (f->n_active == 0) return false;
  return it < max_iters;
}

__global__ void k_loop_gate(Flags* f, int max_iters, int reset,
                            cudaGraphConditionalHandle cond) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    cudaGraphSetConditional(cond, loop_goes_on(f, f->iter - 1, max_iters, reset) ? 1u : 0u);
}

cudaError_t launch_loop_gate(Flags* flags, int max_iters, int reset,
                             cudaGraphConditionalHandle cond, cudaStream_t st) {
  k_loop_gate<<<1, 32, 0, st>>>(flags, max_iters, reset, cond);
  note_launch();
  return cudaGetLastError();
}

__global__ void __launch_bounds__(1024) k_check(CheckArgs a) {
  // iteration index: the host's, or the device loop's counter (read by every thread
  // before thread 0 advances it at the end)
  const int it_now = a.device_it ? a.flags->iter : a.it;
  a.it = it_now;
  const int64_t per = (a.B + blockDim.x - 1) / blockDim.x;
  const int64_t lo = threadIdx.x * per;
  const int64_t hi = lo + per < a.B ? lo + per : a.B;
  int nonfinite = 0;
  long long n_act = 0, rows = 0, chunks = 0;
  double h_merit = 0.0, h_max = 0.0;  // history: over the sequences tested here
  for (int64_t seq = lo; seq < hi; ++seq) {
    SeqInfo inf = a.info[seq];
    if (!inf.done && !a.compact_only) {
      SeqAcc acc = a.acc[seq];
      a.acc[seq] = SeqAcc{0ull, 0.0, 0ull};
      const double mr = __longlong_as_double((long long)acc.max_bits);
      inf.max_resid = mr;
      inf.merit = 0.5 * acc.sumsq;
      h_merit += inf.merit;
      h_max = nanmax(h_max, mr);
      if (!(mr <= DBL_MAX)) ++nonfinite;  // NaN or Inf
      inf.passes = mr <= a.tol ? inf.passes + 1 : 0;
      if (inf.passes >= a.confirm) {
        inf.done = 1;
        inf.iters = a.it;
      } else {
        inf.iters = a.it < a.max_iters ? a.it + 1 : a.it;
        if (a.window) {
          // rows that passed in one more consecutive iterate than the convergence test asks
          // for (so every frozen row has had one further Newton step after it first
          // qualified) are frozen, in whole chunks
          const int64_t len = a.offsets[seq + 1] - a.offsets[seq];
          const int64_t nch = a.chunk_first[seq + 1] - a.chunk_first[seq];
          const int64_t fb = acc.badkey ? (int64_t)(~acc.badkey) : len;
          int64_t fbw = fb < inf.fb_prev ? fb : (int64_t)inf.fb_prev;
          if (a.confirm >= 2 && inf.fb_prev2 < fbw) fbw = inf.fb_prev2;
          inf.fb_prev2 = inf.fb_prev;
          inf.fb_prev = (int32_t)fb;
          int64_t j0 = fbw >> a.log2L;
          if (j0 < inf.j0) j0 = inf.j0;
          if (j0 > nch - 1) j0 = nch - 1 > 0 ? nch - 1 : 0;
          inf.j0 = (int32_t)j0;
          a.win_chunk[seq] = a.chunk_first[seq] + j0;
        }
      }
      a.info[seq] = inf;
    }
    if (!inf.done) {
      ++n_act;
      rows += a.offsets[seq + 1] - a.offsets[seq] - ((int64_t)inf.j0 << a.log2L);
      chunks += a.chunk_first[seq + 1] - a.chunk_first[seq] - inf.j0;
    }
  }
  long long tn, tr, tc;
  long long pn = n_act, pr = rows, pc = chunks;
  block_excl_scan3(pn, pr, pc, tn, tr, tc);
  for (int64_t seq = lo; seq < hi; ++seq) {
    const SeqInfo inf = a.info[seq];
    if (inf.done) continue;
    a.act_seq[pn] = seq;
    a.act_row_off[pn] = pr;
    a.act_chunk_off[pn] = pc;
    ++pn;
    pr += a.offsets[seq + 1] - a.offsets[seq] - ((int64_t)inf.j0 << a.log2L);
    pc += a.chunk_first[seq + 1] - a.chunk_first[seq] - inf.j0;
  }
  __shared__ int s_nonfinite;
  if (threadIdx.x == 0) s_nonfinite = 0;
  __syncthreads();
  if (nonfinite) atomicAdd(&s_nonfinite, nonfinite);
  __syncthreads();
  if (threadIdx.x == 0) {
    a.act_row_off[tn] = tr;
    a.act_chunk_off[tn] = tc;
    a.flags->n_active = (int32_t)tn;
    a.flags->n_nonfinite = s_nonfinite;
    a.flags->active_rows = tr;
    a.flags->active_chunks = tc;
  }
  if (a.device_it) {
    __syncthreads();  // every thread has read the counter
    if (threadIdx.x == 0) {
      a.flags->iter = it_now + 1;
      if (a.set_cond)
        cudaGraphSetConditional(
            a.cond, loop_goes_on(a.flags, it_now, a.max_iters, a.reset) ? 1u : 0u);
    }
  }
  if (a.history && !a.compact_only && a.it < a.history_len) {
    // block reduction of the tested sequences' merit sum and largest scaled residual
    __shared__ double s_sum[32], s_max[32];
    const unsigned full = 0xffffffffu;
    for (int o = 16; o > 0; o >>= 1) {
      h_merit += __shfl_xor_sync(full, h_merit, o);
      h_max = nanmax(h_max, __shfl_xor_sync(full, h_max, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { s_sum[warp] = h_merit; s_max[warp] = h_max; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0, mx = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        sum += s_sum[w];
        mx = nanmax(mx, s_max[w]);
      }
      double* h = a.history + 4 * (int64_t)a.it;
      h[0] = (double)a.it;
      h[1] = sum;
      h[2] = mx;
      h[3] = (double)tn;
    }
  }
}

__global__ void k_uniform_tables(int64_t* off, int64_t* cf, int64_t B, int64_t T,
                                 int64_t cps) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b <= B;
       b += (int64_t)gridDim.x * blockDim.x) {
    off[b] = b * T;
    cf[b] = b * cps;
  }
}

cudaError_t launch_uniform_tables(int64_t* offsets, int64_t* chunk_first, int64_t B,
                                  int64_t T, int64_t chunks_per_seq, cudaStream_t st) {
  const int64_t n = B + 1;
  const unsigned g = (unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
  k_uniform_tables<<<g, 256, 0, st>>>(offsets, chunk_first, B, T, chunks_per_seq);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_check(const CheckArgs& a, cudaStream_t st) {
  k_check<<<1, 1024, 0, st>>>(a);
  note_launch();
  return cudaGetLastError();
}

template <int D>
struct U { static constexpr int n = D <= 8 ? D : 1; };

template <class real>
__device__ __forceinline__ real reset_val(real v, real thr, int reset) {
  if (reset && !(v <= thr && v >= -thr)) return real(0);
  return v;
}

// ----------------------------------------------------------------------------
// Dense scan (one thread per chunk)
// ----------------------------------------------------------------------------
template <class real, int D>
__global__ void __launch_bounds__(128) k_dense_chunk(DenseScanArgs<real> a) {
  const int64_t ac = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (ac >= a.bt.act_chunks()) return;
  int64_t seq, c, r0;
  int n;
  act_chunk(a.bt, ac, seq, c, r0, n);
  // the first solved chunk of a sequence starts from Delta = 0: its carry never
  // multiplies P (the rows before it are the initial state or frozen)
  const bool need_P = c != win_first(a.bt, seq);
  real P[D][D], v[D];
#pragma unroll U<D>::n
  for (int i = 0; i < D; ++i) {
    v[i] = real(0);
#pragma unroll U<D>::n
    for (int j = 0; j < D; ++j) P[i][j] = (i == j) ? real(1) : real(0);
  }
  for (int t = 0; t < n; ++t) {
    const real* At = a.A + (r0 + t) * (int64_t)(D * D);
    const real* bt = a.b + (r0 + t) * D;
    real nv[D];
#pragma unroll U<D>::n
    for (int i = 0; i < D; ++i) {
      real acc = __ldg(bt + i);
#pragma unroll U<D>::n
      for (int k = 0; k < D; ++k) acc += __ldg(At + i * D + k) * v[k];
      nv[i] = acc;
    }
#pragma unroll U<D>::n
    for (int i = 0; i < D; ++i) v[i] = nv[i];
    if (need_P) {
      real NP[D][D];
#pragma unroll U<D>::n
      for (int i = 0; i < D; ++i)
#pragma unroll U<D>::n
        for (int j = 0; j < D; ++j) {
          real acc = real(0);
#pragma unroll U<D>::n
          for (int k = 0; k < D; ++k) acc += __ldg(At + i * D + k) * P[k][j];
          NP[i][j] = acc;
        }
#pragma unroll U<D>::n
      for (int i = 0; i < D; ++i)
#pragma unroll U<D>::n
        for (int j = 0; j < D; ++j) P[i][j] = NP[i][j];
    }
  }
  real* Po = a.aggP + c * (int64_t)(D * D);
  real* vo = a.aggv + c * D;
#pragma unroll U<D>::n
  for (int i = 0; i < D; ++i) {
    vo[i] = v[i];
#pragma unroll U<D>::n
    for (int j = 0; j < D; ++j) Po[i * D + j] = P[i][j];
  }
}

template <class real, int D>
__global__ void __launch_bounds__(128) k_dense_carry(DenseScanArgs<real> a) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= a.bt.n_act()) return;
  const int64_t seq = a.bt.act_seq[k];
  const int64_t c0 = win_first(a.bt, seq), c1 = a.bt.chunk_first[seq + 1];
  real x[D];
#pragma unroll U<D>::n
  for (int i = 0; i < D; ++i) x[i] = real(0);
  for (int64_t c = c0; c < c1; ++c) {
    real* ci = a.cin + c * D;
#pragma unroll U<D>::n
    for (int i = 0; i < D; ++i) ci[i] = x[i];
    if (c == c1 - 1) break;
    const real* P = a.aggP + c * (int64_t)(D * D);
    const real* v = a.aggv + c * D;
    real nx[D];
    if (c == c0) {
#pragma unroll U<D>::n
      for (int i = 0; i < D; ++i) nx[i] = v[i];
    } else {
#pragma unroll U<D>::n
      for (int i = 0; i < D; ++i) {
        real acc = v[i];
#pragma unroll U<D>::n
        for (int k = 0; k < D; ++k) acc += P[i * D + k] * x[k];
        nx[i] = acc;
      }
    }
#pragma unroll U<D>::n
    for (int i = 0; i < D; ++i) x[i] = nx[i];
  }
}

template <class real, int D>
__global__ void __launch_bounds__(128) k_dense_apply(DenseScanArgs<real> a) {
  const int64_t ac = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (ac >= a.bt.act_chunks()) return;
  int64_t seq, c, r0;
  int n;
  act_chunk(a.bt, ac, seq, c, r0, n);
  real x[D];
#pragma unroll U<D>::n
  for (int i = 0; i < D; ++i) x[i] = a.cin[c * D + i];
  for (int t = 0; t < n; ++t) {
    const int64_t row = r0 + t;
    const real* At = a.A + row * (int64_t)(D * D);
    const real* bt = a.b + row * D;
    real nx[D];
#pragma unroll U<D>::n
    for (int i = 0; i < D; ++i) {
      real acc = __ldg(bt + i);
#pragma unroll U<D>::n
      for (int k = 0; k < D; ++k) acc += __ldg(At + i * D + k) * x[k];
      nx[i] = acc;
    }
    real* sr = a.s + row * D;
#pragma unroll U<D>::n
    for (int i = 0; i < D; ++i) {
      x[i] = nx[i];
      sr[i] = reset_val(sr[i] + nx[i], a.reset_thr, a.reset);
    }
  }
}

template <class real, int D>
static void dense_launch(const DenseScanArgs<real>& a, cudaStream_t st) {
  const unsigned gc = grid_for(a.bt.act_chunks(), 128);
  const unsigned gs = grid_for(a.bt.n_act(), 128);
  k_dense_chunk<real, D><<<gc, 128, 0, st>>>(a);
  k_dense_carry<real, D><<<gs, 128, 0, st>>>(a);
  k_dense_apply<real, D><<<gc, 128, 0, st>>>(a);
  note_launch(3);
}

template <class real, int D>
void dense_launch_wide(const DenseScanArgs<real>& a, cudaStream_t st);

template <class real>
cudaError_t launch_dense_scan(const DenseScanArgs<real>& a, cudaStream_t st) {
  if (a.bt.act_rows() == 0) return cudaSuccess;
  switch (a.d) {
    case 1: dense_launch<real, 1>(a, st); break;
    case 2: dense_launch<real, 2>(a, st); break;
    case 4: dense_launch<real, 4>(a, st); break;
    case 5: dense_launch<real, 5>(a, st); break;
    case 8: dense_launch<real, 8>(a, st); break;
    case 16: dense_launch_wide<real, 16>(a, st); break;
    case 32: dense_launch_wide<real, 32>(a, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Diagonal family (one thread per (chunk, coordinate))
// ----------------------------------------------------------------------------
template <class real>
__device__ __forceinline__ void diag_elem(const DiagScanArgs<real>& a, int64_t row, int j,
                                          real& at, real& bt) {
  at = a.amode == 0 ? __ldg(a.a + row * a.d + j) : a.aconst;
  bt = __ldg(a.b + row * a.d + j);
}

template <class real>
__global__ void __launch_bounds__(128) k_diag_chunk(DiagScanArgs<real> a) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= a.bt.act_chunks() * a.d) return;
  const int64_t ac = id / a.d;
  const int j = (int)(id - ac * a.d);
  int64_t seq, c, r0;
  int n;
  act_chunk(a.bt, ac, seq, c, r0, n);
  real A = real(1), Bv = real(0);
  for (int t = 0; t < n; ++t) {
    real at, bt;
    diag_elem(a, r0 + t, j, at, bt);
    Bv = at * Bv + bt;
    A = at * A;
  }
  a.aggA[c * a.d + j] = A;
  a.aggB[c * a.d + j] = Bv;
}

template <class real>
__global__ void __launch_bounds__(128) k_diag_carry(DiagScanArgs<real> a) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= a.bt.n_act() * a.d) return;
  const int64_t k = id / a.d;
  const int j = (int)(id - k * a.d);
  const int64_t seq = a.bt.act_seq[k];
  const int64_t cf = a.bt.chunk_first[seq], c0 = win_first(a.bt, seq);
  const int64_t c1 = a.bt.chunk_first[seq + 1];
  real x = c0 == cf ? a.s0[seq * a.d + j]
                   : a.s[(a.bt.offsets[seq] + ((c0 - cf) << a.bt.log2L) - 1) * a.d + j];
  for (int64_t c = c0; c < c1; ++c) {
    a.cin[c * a.d + j] = x;
    x = a.aggA[c * a.d + j] * x + a.aggB[c * a.d + j];
  }
}

template <class real>
__global__ void __launch_bounds__(128) k_diag_apply(DiagScanArgs<real> a) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= a.bt.act_chunks() * a.d) return;
  const int64_t ac = id / a.d;
  const int j = (int)(id - ac * a.d);
  int64_t seq, c, r0;
  int n;
  act_chunk(a.bt, ac, seq, c, r0, n);
  real x = a.cin[c * a.d + j];
  for (int t = 0; t < n; ++t) {
    real at, bt;
    diag_elem(a, r0 + t, j, at, bt);
    x = at * x + bt;
    a.s[(r0 + t) * a.d + j] = reset_val(x, a.reset_thr, a.reset);
  }
}

// --- Kalman-filter damping (quasi-ELK), per coordinate -----------------------
// The filtered variance obeys P_t = sigma2 (a_t^2 P_{t-1} + 1) / (a_t^2 P_{t-1} + 1 + sigma2),
// a linear-fractional (Moebius) map of P_{t-1} with matrix
// [[sigma2 a^2, sigma2], [a^2, 1 + sigma2]]; maps compose by matrix product, scaled by
// their largest entry to stay finite (a Moebius map is invariant under scaling).
template <class real>
__device__ __forceinline__ void mob_elem(real at, real s2, real& m00, real& m01, real& m10,
                                         real& m11) {
  const real a2 = at * at;
  m00 = s2 * a2; m01 = s2; m10 = a2; m11 = real(1) + s2;
}

template <class real>
__global__ void __launch_bounds__(128) k_elk_chunk(DiagScanArgs<real> a) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= a.bt.act_chunks() * a.d) return;
  const int64_t ac = id / a.d;
  const int j = (int)(id - ac * a.d);
  int64_t seq, c, r0;
  int n;
  act_chunk(a.bt, ac, seq, c, r0, n);
  real p00 = 1, p01 = 0, p10 = 0, p11 = 1;
  for (int t = 0; t < n; ++t) {
    const int64_t row = r0 + t;
    const real at = a.amode == 0 ? __ldg(a.a + row * a.d + j) : a.aconst;
    real m00, m01, m10, m11;
    mob_elem(at, a.sigma2, m00, m01, m10, m11);
    real q00 = m00 * p00 + m01 * p10, q01 = m00 * p01 + m01 * p11;
    real q10 = m10 * p00 + m11 * p10, q11 = m10 * p01 + m11 * p11;
    real mx = fmax(fmax(fabs(q00), fabs(q01)), fmax(fabs(q10), fabs(q11)));
    real inv = mx > real(0) ? real(1) / mx : real(1);
    p00 = q00 * inv; p01 = q01 * inv; p10 = q10 * inv; p11 = q11 * inv;
  }
  real* o = a.mob + (c * a.d + j) * 4;
  o[0] = p00; o[1] = p01; o[2] = p10; o[3] = p11;
}

template <class real>
__global__ void __launch_bounds__(128) k_elk_carry(DiagScanArgs<real> a) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= a.bt.n_act() * a.d) return;
  const int64_t k = id / a.d;
  const int j = (int)(id - k * a.d);
  const int64_t seq = a.bt.act_seq[k];
  real P = real(0);  // the state before the first solved row (s_0 or frozen) is known exactly
  const int64_t c0 = win_first(a.bt, seq), c1 = a.bt.chunk_first[seq + 1];
  for (int64_t c = c0; c < c1; ++c) {
    a.pin[c * a.d + j] = P;
    const real* m = a.mob + (c * a.d + j) * 4;
    P = (m[0] * P + m[1]) / (m[2] * P + m[3]);
  }
}

// The filtered mean's transition of a row, with the attenuation recomputed from the
// variance carried along the chunk: P^-_t = a_t^2 P_{t-1} + 1, Gamma_t = sigma2 / (P^-_t +
// sigma2), P_t = Gamma_t P^-_t; mu_t = Gamma_t a_t mu_{t-1} + Gamma_t b_t + (1 - Gamma_t) y_t.
template <class real>
__device__ __forceinline__ void elk_row(const DiagScanArgs<real>& a, int64_t row, int j,
                                        real& P, real& at, real& bt) {
  const real a0 = a.amode == 0 ? __ldg(a.a + row * a.d + j) : a.aconst;
  const real Pm = a0 * a0 * P + real(1);
  const real g = a.sigma2 / (Pm + a.sigma2);
  P = g * Pm;
  at = g * a0;
  bt = g * __ldg(a.b + row * a.d + j) + (real(1) - g) * a.s[row * a.d + j];
}

// Mean aggregates of the chunks (quasi-ELK): the variance entering the chunk (pin) is known
// from the Moebius carry, so the attenuations are formed on the fly instead of being
// stored and read back.
template <class real>
__global__ void __launch_bounds__(128) k_elk_mean_chunk(DiagScanArgs<real> a) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= a.bt.act_chunks() * a.d) return;
  const int64_t ac = id / a.d;
  const int j = (int)(id - ac * a.d);
  int64_t seq, c, r0;
  int n;
  act_chunk(a.bt, ac, seq, c, r0, n);
  real P = a.pin[c * a.d + j];
  real A = real(1), Bv = real(0);
  for (int t = 0; t < n; ++t) {
    real at, bt;
    elk_row(a, r0 + t, j, P, at, bt);
    Bv = at * Bv + bt;
    A = at * A;
  }
  a.aggA[c * a.d + j] = A;
  a.aggB[c * a.d + j] = Bv;
}

template <class real>
__global__ void __launch_bounds__(128) k_elk_apply(DiagScanArgs<real> a) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= a.bt.act_chunks() * a.d) return;
  const int64_t ac = id / a.d;
  const int j = (int)(id - ac * a.d);
  int64_t seq, c, r0;
  int n;
  act_chunk(a.bt, ac, seq, c, r0, n);
  real P = a.pin[c * a.d + j];
  real x = a.cin[c * a.d + j];
  for (int t = 0; t < n; ++t) {
    real at, bt;
    elk_row(a, r0 + t, j, P, at, bt);  // reads y_t = s_t before it is overwritten
    x = at * x + bt;
    a.s[(r0 + t) * a.d + j] = reset_val(x, a.reset_thr, a.reset);
  }
}

template <class real>
cudaError_t launch_diag_scan(const DiagScanArgs<real>& a, cudaStream_t st) {
  if (a.bt.act_rows() == 0) return cudaSuccess;
  const unsigned gc = grid_for(a.bt.act_chunks() * a.d, 128);
  const unsigned gs = grid_for(a.bt.n_act() * a.d, 128);
  if (a.elk) {
    // variance: Moebius chunk aggregates and their carry; mean: aggregates, carry and
    // apply with the attenuations recomputed from the carried variance
    k_elk_chunk<real><<<gc, 128, 0, st>>>(a);
    k_elk_carry<real><<<gs, 128, 0, st>>>(a);
    k_elk_mean_chunk<real><<<gc, 128, 0, st>>>(a);
    k_diag_carry<real><<<gs, 128, 0, st>>>(a);
    k_elk_apply<real><<<gc, 128, 0, st>>>(a);
    note_launch(5);
    return cudaGetLastError();
  }
  k_diag_chunk<real><<<gc, 128, 0, st>>>(a);
  k_diag_carry<real><<<gs, 128, 0, st>>>(a);
  k_diag_apply<real><<<gc, 128, 0, st>>>(a);
  note_launch(3);
  return cudaGetLastError();
}

template cudaError_t launch_dense_scan<float>(const DenseScanArgs<float>&, cudaStream_t);
template cudaError_t launch_dense_scan<double>(const DenseScanArgs<double>&, cudaStream_t);
template cudaError_t launch_diag_scan<float>(const DiagScanArgs<float>&, cudaStream_t);
template cudaError_t launch_diag_scan<double>(const DiagScanArgs<double>&, cudaStream_t);

}  // namespace deer

namespace deer {

// ----------------------------------------------------------------------------
// Reverse dense scan for the adjoint (one thread per chunk / per sequence), rows visited
// from the end of the sequence: lambda_t = M_t lambda_{t+1} + g_t with M_t = A_{t+1}^T and
// lambda_{T+1} = 0. Chunk aggregates compose in reverse row order.
// ----------------------------------------------------------------------------
template <class real, int D>
__global__ void __launch_bounds__(128) k_adj_chunk(AdjScanArgs<real> a) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= a.bt.n_chunks) return;
  int64_t seq, r0;
  int n;
  chunk_rows(a.bt, c, seq, r0, n);
  const int64_t rend = __ldg(a.bt.offsets + seq + 1);  // one past the last row
  const bool need_P = c != __ldg(a.bt.chunk_first + seq + 1) - 1;  // last chunk: carry 0
  real P[D][D], v[D];
#pragma unroll U<D>::n
  for (int i = 0; i < D; ++i) {
    v[i] = real(0);
#pragma unroll U<D>::n
    for (int j = 0; j < D; ++j) P[i][j] = (i == j) ? real(1) : real(0);
  }
  for (int t = n - 1; t >= 0; --t) {
    const int64_t row = r0 + t;
    const real* gt = a.g + row * D;
    if (row + 1 < rend) {
      const real* An = a.A + (row + 1) * (int64_t)(D * D);  // M_t = A_{t+1}^T
      real nv[D];
#pragma unroll U<D>::n
      for (int i = 0; i < D; ++i) {
        real acc = __ldg(gt + i);
#pragma unroll U<D>::n
        for (int k = 0; k < D; ++k) acc += __ldg(An + k * D + i) * v[k];
        nv[i] = acc;
      }
#pragma unroll U<D>::n
      for (int i = 0; i < D; ++i) v[i] = nv[i];
      if (need_P) {
        real NP[D][D];
#pragma unroll U<D>::n
        for (int i = 0; i < D; ++i)
#pragma unroll U<D>::n
          for (int j = 0; j < D; ++j) {
            real acc = real(0);
#pragma unroll U<D>::n
            for (int k = 0; k < D; ++k) acc += __ldg(An + k * D + i) * P[k][j];
            NP[i][j] = acc;
          }
#pragma unroll U<D>::n
        for (int i = 0; i < D; ++i)
#pragma unroll U<D>::n
          for (int j = 0; j < D; ++j) P[i][j] = NP[i][j];
      }
    } else {
      // last row of the sequence: lambda_T = g_T, the carry (lambda_{T+1} = 0) is dropped
#pragma unroll U<D>::n
      for (int i = 0; i < D; ++i) {
        v[i] = __ldg(gt + i);
#pragma unroll U<D>::n
        for (int j = 0; j < D; ++j) P[i][j] = real(0);
      }
    }
  }
  real* Po = a.aggP + c * (int64_t)(D * D);
  real* vo = a.aggv + c * D;
#pragma unroll U<D>::n
  for (int i = 0; i < D; ++i) {
    vo[i] = v[i];
#pragma unroll U<D>::n
    for (int j = 0; j < D; ++j) Po[i * D + j] = P[i][j];
  }
}

template <class real, int D>
__global__ void __launch_bounds__(128) k_adj_carry(AdjScanArgs<real> a) {
  const int64_t seq = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (seq >= a.bt.B) return;
  const int64_t c0 = a.bt.chunk_first[seq], c1 = a.bt.chunk_first[seq + 1];
  real x[D];
#pragma unroll U<D>::n
  for (int i = 0; i < D; ++i) x[i] = real(0);
  for (int64_t c = c1 - 1; c >= c0; --c) {
    real* ci = a.cin + c * D;
#pragma unroll U<D>::n
    for (int i = 0; i < D; ++i) ci[i] = x[i];
    const real* P = a.aggP + c * (int64_t)(D * D);
    const real* v = a.aggv + c * D;
    real nx[D];
#pragma unroll U<D>::n
    for (int i = 0; i < D; ++i) {
      real acc = v[i];
#pragma unroll U<D>::n
      for (int k = 0; k < D; ++k) acc += P[i * D + k] * x[k];
      nx[i] = acc;
    }
#pragma unroll U<D>::n
    for (int i = 0; i < D; ++i) x[i] = nx[i];
  }
}

template <class real, int D>
__global__ void __launch_bounds__(128) k_adj_apply(AdjScanArgs<real> a) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= a.bt.n_chunks) return;
  int64_t seq, r0;
  int n;
  chunk_rows(a.bt, c, seq, r0, n);
  const int64_t rend = __ldg(a.bt.offsets + seq + 1);
  real x[D];
#pragma unroll U<D>::n
  for (int i = 0; i < D; ++i) x[i] = a.cin[c * D + i];
  for (int t = n - 1; t >= 0; --t) {
    const int64_t row = r0 + t;
    const real* gt = a.g + row * D;
    real nx[D];
    if (row + 1 < rend) {
      const real* An = a.A + (row + 1) * (int64_t)(D * D);
#pragma unroll U<D>::n
      for (int i = 0; i < D; ++i) {
        real acc = __ldg(gt + i);
#pragma unroll U<D>::n
        for (int k = 0; k < D; ++k) acc += __ldg(An + k * D + i) * x[k];
        nx[i] = acc;
      }
    } else {
#pragma unroll U<D>::n
      for (int i = 0; i < D; ++i) nx[i] = __ldg(gt + i);
    }
    real* lr = a.lam + row * D;
#pragma unroll U<D>::n
    for (int i = 0; i < D; ++i) {
      x[i] = nx[i];
      lr[i] = nx[i];
    }
  }
}

template <class real, int D>
static void adj_launch(const AdjScanArgs<real>& a, cudaStream_t st) {
  const unsigned gc = grid_for(a.bt.n_chunks, 128);
  const unsigned gs = grid_for(a.bt.B, 128);
  k_adj_chunk<real, D><<<gc, 128, 0, st>>>(a);
  k_adj_carry<real, D><<<gs, 128, 0, st>>>(a);
  k_adj_apply<real, D><<<gc, 128, 0, st>>>(a);
  note_launch(3);
}

template <class real, int D>
void adj_launch_wide(const AdjScanArgs<real>& a, cudaStream_t st);

template <class real>
cudaError_t launch_adjoint_scan(const AdjScanArgs<real>& a, cudaStream_t st) {
  if (a.bt.N == 0) return cudaSuccess;
  switch (a.d) {
    case 1: adj_launch<real, 1>(a, st); break;
    case 2: adj_launch<real, 2>(a, st); break;
    case 4: adj_launch<real, 4>(a, st); break;
    case 5: adj_launch<real, 5>(a, st); break;
    case 8: adj_launch<real, 8>(a, st); break;
    case 16: adj_launch_wide<real, 16>(a, st); break;
    case 32: adj_launch_wide<real, 32>(a, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template cudaError_t launch_adjoint_scan<float>(const AdjScanArgs<float>&, cudaStream_t);
template cudaError_t launch_adjoint_scan<double>(const AdjScanArgs<double>&, cudaStream_t);

}  // namespace deer

namespace deer {

// ----------------------------------------------------------------------------
// Dense scan, d = 16 / 32: D lanes per chunk (per sequence in the carry pass; four warps
// per chunk in the d = 32 chunk pass). Lane j owns column j of the chunk product P and
// entry j of the vectors; the Jacobian rows and chunk aggregates are staged in a
// shared-memory ring ahead of use, vector entries travel by shuffles.
// ----------------------------------------------------------------------------
// 16 bytes (four floats or two doubles) from a 16-byte aligned address. Plain (coherent)
// load: used for data the same launch never writes, and for data written by earlier
// launches.
template <class real>
__device__ __forceinline__ void ld16(const real* p, real* v) {
  if constexpr (sizeof(real) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
    const double2 q = *reinterpret_cast<const double2*>(p);
    v[0] = q.x; v[1] = q.y;
  }
}

template <int D>
__device__ __forceinline__ unsigned group_mask() {
  return D == 32 ? 0xffffffffu : (0xffffu << (16 * ((threadIdx.x >> 4) & 1)));
}

// ----------------------------------------------------------------------------
// Asynchronous row staging for the wide dense scans. Lane i of a group copies its own row
// (D values, 16-byte pieces) of a d x d block, and one entry of a vector, from global
// memory into a slot of a shared-memory ring with cp.async; the ring runs kRing slots
// ahead of the rows being consumed, so the DRAM latency of a row is hidden behind the
// dependent work on the rows before it. Rows are padded to D + 16 B so that 128-bit
// reads of eight lanes' rows hit distinct banks. Every stage commits one (possibly empty)
// group, and cp.async.wait_group(kRing - 1) before a slot is read guarantees that the
// slot's copies (issued kRing commits earlier) have landed: the wait ends when the copies
// do, with no spin loop of our own.
// ----------------------------------------------------------------------------
template <class real>
constexpr int ring_depth() { return sizeof(real) == 4 ? 8 : 4; }

template <class real, int D>
struct RowRing {
  static constexpr int K = ring_depth<real>();
  static constexpr int RS = D + 16 / (int)sizeof(real);
  real m[K][D][RS];  // row `lane` of a d x d block per slot
  real v[K][D];      // one vector entry per lane per slot

  // copy row `lane` of the block at `blk` (16-byte aligned) and vec[lane] into `slot`
  __device__ __forceinline__ void issue(int slot, int lane, const real* blk, const real* vec) {
    constexpr int PIECES = D * (int)sizeof(real) / 16;
#pragma unroll
    for (int q = 0; q < PIECES; ++q)
      cp_async16(&m[slot][lane][q * 16 / (int)sizeof(real)],
                 blk + lane * D + q * 16 / (int)sizeof(real));
    cp_async_small<sizeof(real)>(&v[slot][lane], vec + lane);
  }
  __device__ __forceinline__ void row(int slot, int r, real (&out)[D]) const {
#pragma unroll
    for (int k = 0; k < D; k += 16 / (int)sizeof(real)) {
      if constexpr (sizeof(real) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(&m[slot][r][k]);
        out[k] = q.x; out[k + 1] = q.y; out[k + 2] = q.z; out[k + 3] = q.w;
      } else {
        const double2 q = *reinterpret_cast<const double2*>(&m[slot][r][k]);
        out[k] = q.x; out[k + 1] = q.y;
      }
    }
  }
};

// Chunk pass, d = 16 / 32: one group of D lanes per chunk (one warp per block), lane j owns
// column j of the chunk product P and entry j of the vector part. Row t's Jacobian is
// staged in the ring; every lane reads all of its rows (broadcast) for P <- A_t P and
// its own row for v <- A_t v + b_t.
template <class real, int D>
__global__ void __launch_bounds__(32) k_dense_chunk_ring(DenseScanArgs<real> a) {
  constexpr int G = 32 / D;
  using Ring = RowRing<real, D>;
  constexpr int K = Ring::K;
  __shared__ __align__(16) Ring ring[G];
  const int grp = threadIdx.x / D, lane = threadIdx.x % D;
  const unsigned gm = group_mask<D>();
  const int64_t ac = blockIdx.x * (int64_t)G + grp;
  if (ac >= a.bt.act_chunks()) return;  // whole groups; groups never synchronise with each other
  int64_t seq, c, r0;
  int n;
  act_chunk(a.bt, ac, seq, c, r0, n);
  const bool need_P = c != win_first(a.bt, seq);
  Ring& R = ring[grp];
  const real* A0 = a.A + r0 * (int64_t)(D * D);
  const real* b0 = a.b + r0 * D;
#pragma unroll
  for (int s = 0; s < K; ++s) {
    if (s < n) R.issue(s, lane, A0 + s * (int64_t)(D * D), b0 + s * D);
    cp_async_commit();
  }
  real Pc[D];  // column `lane` of P
  real v = real(0);
#pragma unroll
  for (int i = 0; i < D; ++i) Pc[i] = i == lane ? real(1) : real(0);
  for (int t0 = 0; t0 < n; t0 += K) {
#pragma unroll
    for (int s = 0; s < K; ++s) {
      const int t = t0 + s;
      cp_async_wait<K - 1>();
      __syncwarp(gm);  // the other lanes' rows of this slot have landed
      if (t < n) {
        real own[D];
        R.row(s, lane, own);
        real nv = R.v[s][lane];
#pragma unroll
        for (int k = 0; k < D; ++k) nv += own[k] * __shfl_sync(gm, v, k, D);
        v = nv;
        if (need_P) {
          real np[D];
#pragma unroll
          for (int i = 0; i < D; ++i) {
            real ar[D];
            R.row(s, i, ar);
            real x = real(0);
#pragma unroll
            for (int k = 0; k < D; ++k) x += ar[k] * Pc[k];
            np[i] = x;
          }
#pragma unroll
          for (int i = 0; i < D; ++i) Pc[i] = np[i];
        }
      }
      __syncwarp(gm);  // every lane is done with the slot before it is refilled
      if (t + K < n) R.issue(s, lane, A0 + (t + K) * (int64_t)(D * D), b0 + (t + K) * D);
      cp_async_commit();
    }
  }
  cp_async_wait<0>();
  real* Po = a.aggP + c * (int64_t)(D * D);
#pragma unroll
  for (int i = 0; i < D; ++i) Po[i * D + lane] = Pc[i];
  a.aggv[c * D + lane] = v;
}

// Chunk pass, d = 32: one chunk per block of four warps. The staged rows of A_t are shared
// by the block (its 128 threads copy the 4 KB block together); warp w forms rows
// 8w .. 8w+7 of P <- A_t P for all 32 columns (lane j owns column j), the new rows meet
// in shared memory and every warp reloads its full column. The vector part
// v <- A_t v + b_t is formed redundantly by every warp (lane i, row i). A quarter of the
// dependent work per warp compared with one warp per chunk, and four times the warps:
// the single long sequences that leave few chunks stay busy.
template <class real>
__global__ void __launch_bounds__(128) k_dense_chunk_ring4(DenseScanArgs<real> a) {
  constexpr int D = 32;
  constexpr int W = 4;                       // warps per chunk
  constexpr int RW = D / W;                  // rows of P per warp
  constexpr int K = ring_depth<real>();
  constexpr int RS = D + 16 / (int)sizeof(real);
  constexpr int VW = 16 / (int)sizeof(real);
  constexpr int PIECES = D * D / VW;         // 16-byte pieces of one A_t
  __shared__ __align__(16) real sA[K][D][RS];
  __shared__ __align__(16) real sB[K][D];
  __shared__ real sP[D][D + 1];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ac = blockIdx.x;
  if (ac >= a.bt.act_chunks()) return;  // uniform over the block
  int64_t seq, c, r0;
  int n;
  act_chunk(a.bt, ac, seq, c, r0, n);
  const bool need_P = c != win_first(a.bt, seq);
  const real* A0 = a.A + r0 * (int64_t)(D * D);
  const real* b0 = a.b + r0 * D;
  auto issue = [&](int slot, int t) {
    if (t < n) {
      const real* src = A0 + t * (int64_t)(D * D);
      for (int p = tid; p < PIECES; p += 128)
        cp_async16(&sA[slot][p / (D / VW)][(p % (D / VW)) * VW], src + p * VW);
      if (tid < D / VW) cp_async16(&sB[slot][tid * VW], b0 + t * D + tid * VW);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int s = 0; s < K; ++s) issue(s, s);
  real Pc[D];  // column `lane` of P (the same in every warp)
  real v = real(0);
#pragma unroll
  for (int i = 0; i < D; ++i) Pc[i] = i == lane ? real(1) : real(0);
  for (int t0 = 0; t0 < n; t0 += K) {
#pragma unroll
    for (int s = 0; s < K; ++s) {
      const int t = t0 + s;
      cp_async_wait<K - 1>();
      __syncthreads();  // slot s complete for the block; last row's column reloads done
      if (t < n) {
        real own[D];
#pragma unroll
        for (int k = 0; k < D; k += VW) ld16<real>(&sA[s][lane][k], own + k);
        real nv = sB[s][lane];
#pragma unroll
        for (int k = 0; k < D; ++k) nv += own[k] * __shfl_sync(0xffffffffu, v, k);
        v = nv;
        if (need_P) {
#pragma unroll
          for (int ii = 0; ii < RW; ++ii) {
            const int i = warp * RW + ii;
            real x = real(0);
#pragma unroll
            for (int k = 0; k < D; k += VW) {
              real ar[VW];
              ld16<real>(&sA[s][i][k], ar);
#pragma unroll
              for (int q = 0; q < VW; ++q) x += ar[q] * Pc[k + q];
            }
            sP[i][lane] = x;
          }
        }
      }
      __syncthreads();  // new rows of P complete; every read of slot s done
      if (need_P && t < n) {
#pragma unroll
        for (int k = 0; k < D; ++k) Pc[k] = sP[k][lane];
      }
      issue(s, t + K);
    }
  }
  cp_async_wait<0>();
  if (warp == 0) {
    real* Po = a.aggP + c * (int64_t)(D * D);
#pragma unroll
    for (int i = 0; i < D; ++i) Po[i * D + lane] = Pc[i];
    a.aggv[c * D + lane] = v;
  }
}

// Chunk pass, d = 32, float32, on the tensor cores. P <- A_t P acts on every column of P
// independently, so the chunk product is carried transposed, P^T <- P^T A_t^T, and split
// by rows of P^T (columns of P) over two warps: warp w owns rows 16w .. 16w + 15 of P^T and
// never exchanges data with the other warp. Each row step is a 16 x 32 x 32 product per
// warp as warp-level tf32 MMAs (m16n8k8, float32 accumulation) with the three-term split
// x = x_hi + x_lo (x_hi = x rounded to tf32): A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi, a
// relative error of about 2^-21, so the aggregates keep float32 accuracy. The A operand is
// the previous accumulator re-laid by shuffles within each quad of lanes (the accumulator
// holds columns 2t, 2t+1 of a row where the operand wants t, t + 4); the B operand
// A_t^T[k][n] = A_t[n][k] is read from the row-major staged A_t (rows padded to 36 floats:
// the 32 lanes' words fall in distinct banks). The vector part v <- A_t v + b_t is formed
// by lane i (row i) of warp 0. Rows are staged through the same cp.async ring as
// k_dense_chunk_ring4.
__global__ void __launch_bounds__(64) k_dense_chunk_mma32(DenseScanArgs<float> a) {
  constexpr int D = 32;
  constexpr int K = ring_depth<float>();
  constexpr int RS = D + 4;
  constexpr int PIECES = D * D / 4;  // 16-byte pieces of one A_t
  __shared__ __align__(16) float sA[K][D][RS];
  __shared__ __align__(16) float sB[K][D];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, tq = lane & 3;
  const int64_t ac = blockIdx.x;
  if (ac >= a.bt.act_chunks()) return;  // uniform over the block
  int64_t seq, c, r0;
  int n;
  act_chunk(a.bt, ac, seq, c, r0, n);
  const bool need_P = c != win_first(a.bt, seq);
  const float* A0 = a.A + r0 * (int64_t)(D * D);
  const float* b0 = a.b + r0 * D;
  auto issue = [&](int slot, int t) {
    if (t < n) {
      const float* src = A0 + t * (int64_t)(D * D);
      for (int p = tid; p < PIECES; p += 64)
        cp_async16(&sA[slot][p / (D / 4)][(p % (D / 4)) * 4], src + p * 4);
      if (tid < D / 4) cp_async16(&sB[slot][tid * 4], b0 + t * D + tid * 4);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int s = 0; s < K; ++s) issue(s, s);
  // accumulator of this warp's 16 rows of P^T: n-tile j holds P^T[m][8j + 2tq (+1)] for
  // m = 16 warp + g (entries 0, 1) and m + 8 (entries 2, 3); P^T starts as I
  float acc[4][4];
  const int m0 = 16 * warp + g;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int n0 = 8 * j + 2 * tq;
    acc[j][0] = m0 == n0 ? 1.f : 0.f;
    acc[j][1] = m0 == n0 + 1 ? 1.f : 0.f;
    acc[j][2] = m0 + 8 == n0 ? 1.f : 0.f;
    acc[j][3] = m0 + 8 == n0 + 1 ? 1.f : 0.f;
  }
  float v = 0.f;
  const int qsrc = (lane & ~3) + (tq >> 1);  // quad lane holding column tq of a tile
  const bool odd = tq & 1;
  for (int t0 = 0; t0 < n; t0 += K) {
#pragma unroll
    for (int s = 0; s < K; ++s) {
      const int t = t0 + s;
      cp_async_wait<K - 1>();
      __syncthreads();  // slot s complete for the block
      if (t < n) {
        if (warp == 0) {
          float nv = sB[s][lane];
#pragma unroll
          for (int k = 0; k < D; k += 4) {
            const float4 q = *reinterpret_cast<const float4*>(&sA[s][lane][k]);
            nv += q.x * __shfl_sync(0xffffffffu, v, k) + q.y * __shfl_sync(0xffffffffu, v, k + 1) +
                  q.z * __shfl_sync(0xffffffffu, v, k + 2) + q.w * __shfl_sync(0xffffffffu, v, k + 3);
          }
          v = nv;
        }
        if (need_P) {
          // A operand (P^T rows, K = columns of P^T) from the accumulator, split
          uint32_t ah[4][4], al[4][4];
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const float x0 = __shfl_sync(0xffffffffu, acc[kk][0], qsrc);
            const float x1 = __shfl_sync(0xffffffffu, acc[kk][1], qsrc);
            const float x2 = __shfl_sync(0xffffffffu, acc[kk][2], qsrc);
            const float x3 = __shfl_sync(0xffffffffu, acc[kk][3], qsrc);
            const float y0 = __shfl_sync(0xffffffffu, acc[kk][0], qsrc + 2);
            const float y1 = __shfl_sync(0xffffffffu, acc[kk][1], qsrc + 2);
            const float y2 = __shfl_sync(0xffffffffu, acc[kk][2], qsrc + 2);
            const float y3 = __shfl_sync(0xffffffffu, acc[kk][3], qsrc + 2);
            const float av[4] = {odd ? x1 : x0, odd ? x3 : x2, odd ? y1 : y0, odd ? y3 : y2};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              ah[kk][e] = tc::tf32_rna(av[e]);
              al[kk][e] = tc::tf32_rna(av[e] - __uint_as_float(ah[kk][e]));
            }
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float dn[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              // B[k][n] = A_t[n][k]: n = 8j + g, k = 8kk + tq (+ 4)
              const float bx0 = sA[s][8 * j + g][8 * kk + tq];
              const float bx1 = sA[s][8 * j + g][8 * kk + tq + 4];
              const uint32_t bh0 = tc::tf32_rna(bx0), bh1 = tc::tf32_rna(bx1);
              const uint32_t bl0 = tc::tf32_rna(bx0 - __uint_as_float(bh0));
              const uint32_t bl1 = tc::tf32_rna(bx1 - __uint_as_float(bh1));
              tc::mma_1688_tf32(dn, al[kk], bh0, bh1);
              tc::mma_1688_tf32(dn, ah[kk], bl0, bl1);
              tc::mma_1688_tf32(dn, ah[kk], bh0, bh1);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[j][e] = dn[e];
          }
        }
      }
      __syncthreads();  // every read of slot s done before it is refilled
      issue(s, t + K);
    }
  }
  cp_async_wait<0>();
  // P[i][j] = P^T[j][i]
  float* Po = a.aggP + c * (int64_t)(D * D);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int n0 = 8 * j + 2 * tq;
    Po[n0 * D + m0] = acc[j][0];
    Po[(n0 + 1) * D + m0] = acc[j][1];
    Po[n0 * D + m0 + 8] = acc[j][2];
    Po[(n0 + 1) * D + m0 + 8] = acc[j][3];
  }
  if (warp == 0) a.aggv[c * D + lane] = v;
}

// Carry pass: x_c = P_c x_{c-1} + v_c along each active sequence's chunks (one group per
// sequence); the aggregates do not depend on x and stream through the ring.
template <class real, int D>
__global__ void __launch_bounds__(32) k_dense_carry_ring(DenseScanArgs<real> a) {
  constexpr int G = 32 / D;
  using Ring = RowRing<real, D>;
  constexpr int K = Ring::K;
  __shared__ __align__(16) Ring ring[G];
  const int grp = threadIdx.x / D, lane = threadIdx.x % D;
  const unsigned gm = group_mask<D>();
  const int64_t kq = blockIdx.x * (int64_t)G + grp;
  if (kq >= a.bt.n_act()) return;
  const int64_t seq = a.bt.act_seq[kq];
  const int64_t c0 = win_first(a.bt, seq), c1 = a.bt.chunk_first[seq + 1];
  Ring& R = ring[grp];
#pragma unroll
  for (int s = 0; s < K; ++s) {
    if (c0 + s < c1) R.issue(s, lane, a.aggP + (c0 + s) * (int64_t)(D * D), a.aggv + (c0 + s) * D);
    cp_async_commit();
  }
  real x = real(0);
  for (int64_t cb = c0; cb < c1; cb += K) {
#pragma unroll
    for (int s = 0; s < K; ++s) {
      const int64_t c = cb + s;
      cp_async_wait<K - 1>();  // each lane reads only its own row: no exchange needed
      if (c < c1) {
        a.cin[c * D + lane] = x;
        real y = R.v[s][lane];
        if (c > c0) {
          real pr[D];
          R.row(s, lane, pr);
#pragma unroll
          for (int k = 0; k < D; ++k) y += pr[k] * __shfl_sync(gm, x, k, D);
        }
        x = y;
      }
      if (c + K < c1) R.issue(s, lane, a.aggP + (c + K) * (int64_t)(D * D), a.aggv + (c + K) * D);
      cp_async_commit();
    }
  }
  cp_async_wait<0>();
}

// Apply pass: Delta_t = A_t Delta_{t-1} + b_t from the chunk's carry, s_t += Delta_t; lane
// i reads its own row of each staged A_t.
template <class real, int D>
__global__ void __launch_bounds__(32) k_dense_apply_ring(DenseScanArgs<real> a) {
  constexpr int G = 32 / D;
  using Ring = RowRing<real, D>;
  constexpr int K = Ring::K;
  __shared__ __align__(16) Ring ring[G];
  const int grp = threadIdx.x / D, lane = threadIdx.x % D;
  const unsigned gm = group_mask<D>();
  const int64_t ac = blockIdx.x * (int64_t)G + grp;
  if (ac >= a.bt.act_chunks()) return;
  int64_t seq, c, r0;
  int n;
  act_chunk(a.bt, ac, seq, c, r0, n);
  const real* A0 = a.A + r0 * (int64_t)(D * D);
  const real* b0 = a.b + r0 * D;
  Ring& R = ring[grp];
#pragma unroll
  for (int s = 0; s < K; ++s) {
    if (s < n) R.issue(s, lane, A0 + s * (int64_t)(D * D), b0 + s * D);
    cp_async_commit();
  }
  real x = a.cin[c * D + lane];
  for (int t0 = 0; t0 < n; t0 += K) {
#pragma unroll
    for (int s = 0; s < K; ++s) {
      const int t = t0 + s;
      cp_async_wait<K - 1>();
      if (t < n) {
        real ar[D];
        R.row(s, lane, ar);
        real y = R.v[s][lane];
#pragma unroll
        for (int k = 0; k < D; ++k) y += ar[k] * __shfl_sync(gm, x, k, D);
        x = y;
        real* sp = a.s + (r0 + t) * D + lane;
        if (a.slo) {
          // compensated state: (s, slo) += Delta with error-free transformations
          real hi = *sp, lo = a.slo[(r0 + t) * D + lane];
          cs_add(hi, lo, y);
          if (a.reset && !(hi <= a.reset_thr && hi >= -a.reset_thr)) {
            hi = real(0);
            lo = real(0);
          }
          *sp = hi;
          a.slo[(r0 + t) * D + lane] = lo;
        } else {
          *sp = reset_val(*sp + y, a.reset_thr, a.reset);
        }
      }
      if (t + K < n) R.issue(s, lane, A0 + (t + K) * (int64_t)(D * D), b0 + (t + K) * D);
      cp_async_commit();
    }
  }
  cp_async_wait<0>();
}

template <class real, int D>
void dense_launch_wide(const DenseScanArgs<real>& a, cudaStream_t st) {
  constexpr int G = 32 / D;
  const unsigned gc = grid_for(a.bt.act_chunks(), G);
  const unsigned gs = grid_for(a.bt.n_act(), G);
  if constexpr (D == 32) {
    if constexpr (sizeof(real) == 4) {
      if (a.tensor_cores)
        k_dense_chunk_mma32<<<grid_for(a.bt.act_chunks(), 1), 64, 0, st>>>(a);
      else
        k_dense_chunk_ring4<real><<<grid_for(a.bt.act_chunks(), 1), 128, 0, st>>>(a);
    } else {
      k_dense_chunk_ring4<real><<<grid_for(a.bt.act_chunks(), 1), 128, 0, st>>>(a);
    }
  } else {
    k_dense_chunk_ring<real, D><<<gc, 32, 0, st>>>(a);
  }
  k_dense_carry_ring<real, D><<<gs, 32, 0, st>>>(a);
  k_dense_apply_ring<real, D><<<gc, 32, 0, st>>>(a);
  note_launch(3);
}

template void dense_launch_wide<float, 16>(const DenseScanArgs<float>&, cudaStream_t);
template void dense_launch_wide<float, 32>(const DenseScanArgs<float>&, cudaStream_t);
template void dense_launch_wide<double, 16>(const DenseScanArgs<double>&, cudaStream_t);
template void dense_launch_wide<double, 32>(const DenseScanArgs<double>&, cudaStream_t);

}  // namespace deer

namespace deer {

// ----------------------------------------------------------------------------
// Reverse (adjoint) dense scan, d = 16 / 32: D lanes per chunk / sequence; lane i owns
// entry i of the vectors and column i of the reversed chunk product. M_t = A_{t+1}^T is
// read column-wise (entry (k, i) of A_{t+1} for lane i), i.e. coalesced across lanes.
// ----------------------------------------------------------------------------
template <class real, int D>
__global__ void __launch_bounds__(128) k_adj_chunk_wide(AdjScanArgs<real> a) {
  constexpr int G = 128 / D;
  const int grp = threadIdx.x / D, lane = threadIdx.x % D;
  const unsigned gm = group_mask<D>();
  const int64_t c = blockIdx.x * (int64_t)G + grp;
  const bool valid = c < a.bt.n_chunks;
  int64_t seq = 0, r0 = 0;
  int n = 0;
  if (valid) chunk_rows(a.bt, c, seq, r0, n);
  const int64_t rend = valid ? __ldg(a.bt.offsets + seq + 1) : 0;
  const bool need_P = valid && c != __ldg(a.bt.chunk_first + seq + 1) - 1;
  real Pc[D];
  real v = real(0);
#pragma unroll
  for (int i = 0; i < D; ++i) Pc[i] = i == lane ? real(1) : real(0);
  for (int t = n - 1; t >= 0; --t) {
    const int64_t row = r0 + t;
    const real gt = __ldg(a.g + row * D + lane);
    if (row + 1 < rend) {
      const real* An = a.A + (row + 1) * (int64_t)(D * D);
      real nv = gt;
#pragma unroll
      for (int k = 0; k < D; ++k) nv += __ldg(An + k * D + lane) * __shfl_sync(gm, v, k, D);
      v = nv;
      if (need_P) {
        real np[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          real x = real(0);
#pragma unroll
          for (int k = 0; k < D; ++k) x += __ldg(An + k * D + i) * Pc[k];
          np[i] = x;
        }
#pragma unroll
        for (int i = 0; i < D; ++i) Pc[i] = np[i];
      }
    } else {
      v = gt;
#pragma unroll
      for (int i = 0; i < D; ++i) Pc[i] = real(0);
    }
  }
  if (valid) {
    real* Po = a.aggP + c * (int64_t)(D * D);
#pragma unroll
    for (int i = 0; i < D; ++i) Po[i * D + lane] = Pc[i];
    a.aggv[c * D + lane] = v;
  }
}

template <class real, int D>
__global__ void __launch_bounds__(128) k_adj_carry_wide(AdjScanArgs<real> a) {
  constexpr int G = 128 / D;
  const int grp = threadIdx.x / D, lane = threadIdx.x % D;
  const unsigned gm = group_mask<D>();
  const int64_t seq = blockIdx.x * (int64_t)G + grp;
  const bool valid = seq < a.bt.B;
  const int64_t c0 = valid ? a.bt.chunk_first[seq] : 0;
  const int64_t c1 = valid ? a.bt.chunk_first[seq + 1] : 0;
  real x = real(0);
  for (int64_t c = c1 - 1; c >= c0; --c) {
    a.cin[c * D + lane] = x;
    const real* P = a.aggP + c * (int64_t)(D * D);
    real y = a.aggv[c * D + lane];
#pragma unroll
    for (int k = 0; k < D; ++k) y += P[lane * D + k] * __shfl_sync(gm, x, k, D);
    x = y;
  }
}

template <class real, int D>
__global__ void __launch_bounds__(128) k_adj_apply_wide(AdjScanArgs<real> a) {
  constexpr int G = 128 / D;
  const int grp = threadIdx.x / D, lane = threadIdx.x % D;
  const unsigned gm = group_mask<D>();
  const int64_t c = blockIdx.x * (int64_t)G + grp;
  const bool valid = c < a.bt.n_chunks;
  int64_t seq = 0, r0 = 0;
  int n = 0;
  if (valid) chunk_rows(a.bt, c, seq, r0, n);
  const int64_t rend = valid ? __ldg(a.bt.offsets + seq + 1) : 0;
  real x = valid ? a.cin[c * D + lane] : real(0);
  for (int t = n - 1; t >= 0; --t) {
    const int64_t row = r0 + t;
    real y = __ldg(a.g + row * D + lane);
    if (row + 1 < rend) {
      const real* An = a.A + (row + 1) * (int64_t)(D * D);
#pragma unroll
      for (int k = 0; k < D; ++k) y += __ldg(An + k * D + lane) * __shfl_sync(gm, x, k, D);
    }
    x = y;
    a.lam[row * D + lane] = y;
  }
}

template <class real, int D>
void adj_launch_wide(const AdjScanArgs<real>& a, cudaStream_t st) {
  constexpr int G = 128 / D;
  const unsigned gc = grid_for(a.bt.n_chunks, G);
  const unsigned gs = grid_for(a.bt.B, G);
  k_adj_chunk_wide<real, D><<<gc, 128, 0, st>>>(a);
  k_adj_carry_wide<real, D><<<gs, 128, 0, st>>>(a);
  k_adj_apply_wide<real, D><<<gc, 128, 0, st>>>(a);
  note_launch(3);
}

template void adj_launch_wide<float, 16>(const AdjScanArgs<float>&, cudaStream_t);
template void adj_launch_wide<float, 32>(const AdjScanArgs<float>&, cudaStream_t);
template void adj_launch_wide<double, 16>(const AdjScanArgs<double>&, cudaStream_t);
template void adj_launch_wide<double, 32>(const AdjScanArgs<double>&, cudaStream_t);

}  // namespace deer
