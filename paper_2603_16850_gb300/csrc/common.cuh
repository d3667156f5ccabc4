// Shared device/host definitions of the parallel-Newton library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "deer.h"

namespace deer {

// ---------------------------------------------------------------------------
// Per-sequence solver state kept in the workspace.
// ---------------------------------------------------------------------------
struct SeqAcc {                 // reset every iteration
  unsigned long long max_bits;  // bit pattern of max_t ||r_t||_inf (non-negative double)
  double sumsq;                 // sum_t ||r_t||^2
  unsigned long long badkey;    // max over rows failing the test of ~(row - first row);
                                // 0 = every evaluated row passed
};

struct SeqInfo {                // persistent during one solve
  int32_t iters;
  int32_t done;                 // 1 once converged (masked out of later iterations)
  double merit;
  double max_resid;
  int32_t passes;               // consecutive iterates that passed the test
  int32_t j0;                   // sliding window: first chunk (from the sequence's first)
                                // still solved; rows before it are frozen
  int32_t fb_prev;              // first failing row of the previous iterate
  int32_t fb_prev2;             // ... and of the one before
};

struct Flags {                  // read back by the host once per iteration
  int32_t n_active;
  int32_t n_nonfinite;
  int32_t timeout;
  int32_t bad_input;            // set by set-up kernels that reject their inputs
  long long active_rows;        // rows of the sequences still active after the check
  long long active_chunks;      // scan chunks of those sequences
  int32_t iter;                 // convergence checks done (device-resident loop)
  int32_t pad_;
};

// Everything a kernel needs to evaluate f_t for a row of the packed batch.
template <class real>
struct DynView {
  int32_t kind, d, d_in, R;
  real dt;
  const real* params;
  int64_t pstride;
  const int32_t* topo;
  int64_t tstride;
  const real* x;          // packed inputs [N][d_in] or nullptr
  const real* ma;         // mass-action tensors per sequence: [Lm d*d | Bm d*d*d]
  int64_t ma_stride;      // 0 when shared
  const real* gru_M;      // GRU: M[i][j] = Uh[i][j] * Ur[j][i]
};

// Row-to-sequence maps of a packed ragged batch, and the compacted list of the sequences
// that are still iterating (converged sequences drop out of every later launch, so the
// work of an iteration scales with the rows still active).
struct Batch {
  int64_t B;
  int64_t N;
  const int64_t* offsets;        // [B+1]
  const int64_t* chunk_first;    // [B+1]: first chunk index of each sequence
  int64_t n_chunks;
  int32_t L;                     // chunk length (power of two)
  int32_t log2L;
  const int64_t* act_seq;        // [n_act] active sequence ids, ascending
  const int64_t* act_row_off;    // [n_act+1] exclusive prefix of their lengths
  const int64_t* act_chunk_off;  // [n_act+1] exclusive prefix of their chunk counts
  // sizes of the active set for the current launch, read through n_act() / act_rows() /
  // act_chunks(): the host's values, or, when `live` is set (the Newton loop running on
  // the device as a CUDA graph), the ones the last convergence check wrote to device
  // memory. The host's values are then upper bounds that size the grids.
  int64_t n_act_, act_rows_, act_chunks_;
  const Flags* live = nullptr;
  // sliding window: [B] first chunk still solved per sequence (>= chunk_first); nullptr =
  // whole sequences. Active rows / chunks of a sequence start at its window.
  const int64_t* win_chunk = nullptr;

  __host__ __device__ __forceinline__ int64_t n_act() const {
#ifdef __CUDA_ARCH__
    if (live) return (int64_t)live->n_active;
#endif
    return n_act_;
  }
  __host__ __device__ __forceinline__ int64_t act_rows() const {
#ifdef __CUDA_ARCH__
    if (live) return (int64_t)live->active_rows;
#endif
    return act_rows_;
  }
  __host__ __device__ __forceinline__ int64_t act_chunks() const {
#ifdef __CUDA_ARCH__
    if (live) return (int64_t)live->active_chunks;
#endif
    return act_chunks_;
  }
  void set_counts(int64_t n, int64_t rows, int64_t chunks) {
    n_act_ = n;
    act_rows_ = rows;
    act_chunks_ = chunks;
  }
};

__device__ __forceinline__ int64_t win_first(const Batch& bt, int64_t seq) {
  return bt.win_chunk ? __ldg(bt.win_chunk + seq) : __ldg(bt.chunk_first + seq);
}

__device__ __forceinline__ int64_t find_seq(const int64_t* __restrict__ off, int64_t B,
                                            int64_t row) {
  // largest b with off[b] <= row (off[B] = N > row). Empty sequences are skipped
  // because equal offsets resolve to the last of them.
  int64_t lo = 0, hi = B - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= row) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// largest k < n with off[k] <= x (off ascending; ties resolve to the last, which skips
// empty sequences)
__device__ __forceinline__ int64_t find_k(const int64_t* __restrict__ off, int64_t n,
                                          int64_t x) {
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// active row index -> (sequence, packed row)
__device__ __forceinline__ void act_row(const Batch& bt, int64_t ar, int64_t& seq,
                                        int64_t& row) {
  const int64_t k = find_k(bt.act_row_off, bt.n_act(), ar);
  seq = __ldg(bt.act_seq + k);
  const int64_t j0 = win_first(bt, seq) - __ldg(bt.chunk_first + seq);
  row = __ldg(bt.offsets + seq) + (j0 << bt.log2L) + (ar - __ldg(bt.act_row_off + k));
}

// active chunk index -> (sequence, global chunk index, first row, row count)
__device__ __forceinline__ void act_chunk(const Batch& bt, int64_t ac, int64_t& seq,
                                          int64_t& c, int64_t& r0, int32_t& n) {
  const int64_t k = find_k(bt.act_chunk_off, bt.n_act(), ac);
  seq = __ldg(bt.act_seq + k);
  const int64_t cf = __ldg(bt.chunk_first + seq);
  const int64_t j = (win_first(bt, seq) - cf) + (ac - __ldg(bt.act_chunk_off + k));
  c = cf + j;
  const int64_t s0 = __ldg(bt.offsets + seq), s1 = __ldg(bt.offsets + seq + 1);
  r0 = s0 + (j << bt.log2L);
  const int64_t e = r0 + bt.L;
  n = (int32_t)((e < s1 ? e : s1) - r0);
}

// chunk c -> (sequence, first row, row count)
__device__ __forceinline__ void chunk_rows(const Batch& bt, int64_t c, int64_t& seq,
                                           int64_t& r0, int32_t& n) {
  seq = find_seq(bt.chunk_first, bt.B, c);
  int64_t j = c - __ldg(bt.chunk_first + seq);
  int64_t s0 = __ldg(bt.offsets + seq), s1 = __ldg(bt.offsets + seq + 1);
  r0 = s0 + (j << bt.log2L);
  int64_t e = r0 + bt.L;
  n = (int32_t)((e < s1 ? e : s1) - r0);
}

__device__ __forceinline__ unsigned long long dbits(double v) {
  return (unsigned long long)__double_as_longlong(v);
}

template <class real>
__device__ __forceinline__ real rabs(real v) { return v < real(0) ? -v : v; }

// NaN-propagating maximum of two non-negative doubles.
__device__ __forceinline__ double nanmax(double a, double b) {
  return (b > a || b != b) ? b : a;
}

// Accumulate |r| max and r^2 sum of one row into its sequence's accumulator. Must be
// called by all 32 lanes of the warp. Lanes of a warp whose valid rows all belong to one
// sequence reduce first and issue one atomic; otherwise each valid lane issues its own.
// Non-negative doubles order like their bit patterns, and NaN sorts above +Inf, so the
// integer atomicMax both takes the maximum and flags non-finite residuals.
__device__ __forceinline__ void acc_resid(SeqAcc* acc, int64_t seq, bool valid, double mx,
                                          double sq, unsigned long long badkey = 0ull) {
  const unsigned full = 0xffffffffu;
  unsigned vm = __ballot_sync(full, valid);
  if (vm == 0) return;
  int src = __ffs(vm) - 1;
  long long sseq = __shfl_sync(full, (long long)seq, src);
  bool uniform = __all_sync(full, (!valid) || (seq == sseq));
  if (uniform) {
    if (!valid) { mx = 0.0; sq = 0.0; badkey = 0ull; }
    for (int o = 16; o > 0; o >>= 1) {
      mx = nanmax(mx, __shfl_xor_sync(full, mx, o));
      sq += __shfl_xor_sync(full, sq, o);
      const unsigned long long ok = __shfl_xor_sync(full, badkey, o);
      badkey = ok > badkey ? ok : badkey;
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMax(&acc[sseq].max_bits, dbits(mx));
      atomicAdd(&acc[sseq].sumsq, sq);
      if (badkey) atomicMax(&acc[sseq].badkey, badkey);
    }
  } else if (valid) {
    atomicMax(&acc[seq].max_bits, dbits(mx));
    atomicAdd(&acc[seq].sumsq, sq);
    if (badkey) atomicMax(&acc[seq].badkey, badkey);
  }
}

// Key of a row for the sliding window: rows failing the test map to ~(row - first row of
// the sequence), so the largest key over a sequence names its first failing row.
__device__ __forceinline__ unsigned long long bad_key(bool bad, int64_t rel) {
  return bad ? ~(unsigned long long)rel : 0ull;
}

// Float32 statistics variant of acc_resid for the float32 paths: the warp reduction runs
// in float32 and only the final atomics touch float64, since every float64 instruction
// costs the FP64 pipe (a small fraction of the FP32 rate on this GPU).
__device__ __forceinline__ float nanmaxf(float a, float b) {
  return (b > a || b != b) ? b : a;
}

__device__ __forceinline__ void acc_resid_f(SeqAcc* acc, int64_t seq, bool valid, float mx,
                                            float sq, unsigned long long badkey = 0ull) {
  const unsigned full = 0xffffffffu;
  unsigned vm = __ballot_sync(full, valid);
  if (vm == 0) return;
  int src = __ffs(vm) - 1;
  long long sseq = __shfl_sync(full, (long long)seq, src);
  bool uniform = __all_sync(full, (!valid) || (seq == sseq));
  if (uniform) {
    if (!valid) { mx = 0.f; sq = 0.f; badkey = 0ull; }
    for (int o = 16; o > 0; o >>= 1) {
      mx = nanmaxf(mx, __shfl_xor_sync(full, mx, o));
      sq += __shfl_xor_sync(full, sq, o);
      const unsigned long long ok = __shfl_xor_sync(full, badkey, o);
      badkey = ok > badkey ? ok : badkey;
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMax(&acc[sseq].max_bits, dbits((double)mx));
      atomicAdd(&acc[sseq].sumsq, (double)sq);
      if (badkey) atomicMax(&acc[sseq].badkey, badkey);
    }
  } else if (valid) {
    atomicMax(&acc[seq].max_bits, dbits((double)mx));
    atomicAdd(&acc[seq].sumsq, (double)sq);
    if (badkey) atomicMax(&acc[seq].badkey, badkey);
  }
}

// Dispatch on the precision of the per-thread statistics.
__device__ __forceinline__ void acc_resid_t(SeqAcc* acc, int64_t seq, bool valid, float mx,
                                            float sq, unsigned long long badkey = 0ull) {
  acc_resid_f(acc, seq, valid, mx, sq, badkey);
}
__device__ __forceinline__ void acc_resid_t(SeqAcc* acc, int64_t seq, bool valid, double mx,
                                            double sq, unsigned long long badkey = 0ull) {
  acc_resid(acc, seq, valid, mx, sq, badkey);
}

// Group-local variant for kernels whose D-lane groups walk several rows each: the lanes of
// one group reduce their per-lane statistics (shuffles within the group mask only, so
// the groups of a warp need not flush together) and lane 0 issues the atomics.
template <int D, class real>
__device__ __forceinline__ void acc_resid_group(SeqAcc* acc, int64_t seq, real mx, real sq,
                                                unsigned long long badkey, int lane,
                                                unsigned gm) {
#pragma unroll
  for (int o = D / 2; o > 0; o >>= 1) {
    const real om = __shfl_xor_sync(gm, mx, o, D);
    mx = (om > mx || om != om) ? om : mx;
    sq += __shfl_xor_sync(gm, sq, o, D);
    const unsigned long long ok = __shfl_xor_sync(gm, badkey, o, D);
    badkey = ok > badkey ? ok : badkey;
  }
  if (lane == 0) {
    atomicMax(&acc[seq].max_bits, dbits((double)mx));
    atomicAdd(&acc[seq].sumsq, (double)sq);
    if (badkey) atomicMax(&acc[seq].badkey, badkey);
  }
}

// y += a x for a register row. Float32 rows go through the packed two-wide FMA (one
// instruction for two lanes of the FP32 pipe; each half rounds like a scalar FMA, so the
// results are the same as the scalar loop's): the kinetics kernel below is bound by
// instruction issue, not by the FMA pipe.
template <int D>
__device__ __forceinline__ void axpy_row(double a, const double (&x)[D], double (&y)[D]) {
#pragma unroll
  for (int j = 0; j < D; ++j) y[j] += a * x[j];
}

template <int D>
__device__ __forceinline__ void axpy_row(float a, const float (&x)[D], float (&y)[D]) {
  if constexpr (D % 2 == 0) {
    const float2 a2 = make_float2(a, a);
#pragma unroll
    for (int q = 0; q < D / 2; ++q) {
      const float2 r = __ffma2_rn(a2, make_float2(x[2 * q], x[2 * q + 1]),
                                  make_float2(y[2 * q], y[2 * q + 1]));
      y[2 * q] = r.x;
      y[2 * q + 1] = r.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < D; ++j) y[j] += a * x[j];
  }
}

// Writes a D x D block held one row per lane of a D-lane group (row `lane` in registers)
// to `dst` (16-byte aligned) with contiguous 16-byte stores across the group: the rows go
// through `tile` ([D][D + 1] per group; the odd stride keeps both the row writes and the
// strided reads free of bank conflicts for float).
template <class real, int D>
__device__ __forceinline__ void store_block_rows(real* tile, real* dst, const real (&row)[D],
                                                 int lane, unsigned gm) {
  constexpr int VW = 16 / (int)sizeof(real);
  static_assert(D % VW == 0, "rows of whole 16-byte pieces");
#pragma unroll
  for (int j = 0; j < D; ++j) tile[lane * (D + 1) + j] = row[j];
  __syncwarp(gm);
#pragma unroll
  for (int q = 0; q < D / VW; ++q) {
    const int e = (q * D + lane) * VW;
    const real* src = tile + (e / D) * (D + 1) + e % D;
    if constexpr (sizeof(real) == 4) {
      reinterpret_cast<float4*>(dst)[q * D + lane] = make_float4(src[0], src[1], src[2], src[3]);
    } else {
      reinterpret_cast<double2*>(dst)[q * D + lane] = make_double2(src[0], src[1]);
    }
  }
  __syncwarp(gm);
}

// ---------------------------------------------------------------------------
// Compensated state (float32 paths of the mass-action kinetics): the state entry is the
// unevaluated sum hi + lo of two floats, hi the stored float32 value and lo the part below
// its half ulp (kept in the workspace). Near equilibrium the per-step increments of a
// trajectory fall below half an ulp of the state and a plain float32 state loses them
// (the drift then adds up along the conserved directions of the kinetics); the pair keeps
// them.
// ---------------------------------------------------------------------------
// (hi, lo) += d exactly up to the rounding of lo: Knuth's two-sum of hi and d gives the
// rounded sum and its exact error, which joins lo; a fast two-sum renormalises the pair so
// that |lo| <= ulp(hi) / 2.
template <class real>
__device__ __forceinline__ void cs_add(real& hi, real& lo, real d) {
  const real s = hi + d;
  const real bb = s - hi;
  const real err = (hi - (s - bb)) + (d - bb);
  const real l = lo + err;
  const real h2 = s + l;
  lo = l - (h2 - s);
  hi = h2;
}

// Residual r_t = s_t - f(s_{t-1}) of an explicit integrator step f(s) = s + inc(s) from
// compensated states: (s_t - s_{t-1}) - inc + (lo_t - lo_{t-1}). The difference of the two
// high parts is exact when they lie within a factor of two (Sterbenz) and otherwise rounds
// relative to the increment, so the residual is accurate to the rounding of the increment.
template <class real>
__device__ __forceinline__ real cs_residual(real hi_t, real lo_t, real hi_p, real lo_p,
                                            real inc) {
  return ((hi_t - hi_p) - inc) + (lo_t - lo_p);
}

// ---------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async): 16 bytes through L2 only, or 4 / 8
// bytes; every commit closes a group, and wait_group<N> returns when all but the N most
// recent groups of this thread have landed (the data is then visible to this thread).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

template <int BYTES>
__device__ __forceinline__ void cp_async_small(void* smem, const void* gmem) {
  static_assert(BYTES == 4 || BYTES == 8, "cp.async.ca copies 4, 8 or 16 bytes");
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(BYTES)
               : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------
// Launch bookkeeping (counted for deer_kernel_launch_count).
// ---------------------------------------------------------------------------
void note_launch(int n = 1);

inline unsigned grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace deer
