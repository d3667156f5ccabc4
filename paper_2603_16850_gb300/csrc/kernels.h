// Argument blocks and launchers shared between the kernel translation units and the
// host API. Internal to the library (not part of the C ABI).
#pragma once

#include "common.cuh"

namespace deer {

template <class real>
struct InitArgs {
  DynView<real> dv;
  Batch bt;
  const real* s0;
  real* s;
  int init;
  unsigned long long seed = 0ull;  // DEER_INIT_RANDN
};

template <class real>
struct LinArgs {
  DynView<real> dv;
  Batch bt;
  const real* s0;
  const real* s;   // current iterate [N][d]
  real* A;         // FULL: [N][d][d]; DIAG: [N][d]; unused otherwise
  real* b;         // [N][d]
  SeqAcc* acc;
  const SeqInfo* info;
  int jac, damp;
  real dparam;
  real tol = real(0);  // convergence test in this precision: rows with a scaled residual
                       // above it are reported (first failing row, for the sliding window)
  const real* slo = nullptr;  // compensation of s ([N][d], the state is s + slo); nullptr =
                              // plain state (mass-action kinetics only)
  // mass action, d = 16 / 32: per-species lists of the reactions that change the species
  // (launch_ma_adjacency; entry = r | (nu + 4) << 16), so that each lane walks its own
  // reactions rather than all of them; nullptr = walk every reaction
  const int32_t* adj_off = nullptr;  // [nseq][d+1]
  const int32_t* adj_e = nullptr;    // [nseq][adj_stride]
  int64_t adj_stride = 0;            // 0: one list shared by every sequence
};

template <class real>
struct RolloutArgs {
  DynView<real> dv;
  int64_t B;
  int64_t T;               // uniform length when offsets == nullptr
  const int64_t* offsets;  // device [B+1] or nullptr
  const real* s0;
  real* s;
};

template <class real>
__device__ __forceinline__ void rollout_rows(const RolloutArgs<real>& a, int64_t seq,
                                             int64_t& r0, int64_t& r1) {
  if (a.offsets) { r0 = a.offsets[seq]; r1 = a.offsets[seq + 1]; }
  else { r0 = seq * a.T; r1 = r0 + a.T; }
}

struct CheckArgs {
  int64_t B;
  const int64_t* offsets;
  const int64_t* chunk_first;
  SeqAcc* acc;
  SeqInfo* info;
  Flags* flags;
  int64_t* act_seq;        // outputs: compacted active set
  int64_t* act_row_off;
  int64_t* act_chunk_off;
  double tol;
  int it, max_iters;
  int compact_only;        // 1: rebuild the active set from info without testing
  int confirm;             // consecutive passing iterates needed
  // sliding window (Sec. 3.2): advance each sequence's first solved chunk past the rows
  // that passed the test (in the last `confirm` iterates); nullptr / 0 = off
  int64_t* win_chunk = nullptr;
  int window = 0;
  int log2L = 0;
  // optional per-iteration record [history_len][4] (iteration, merit sum, max scaled
  // residual, active sequences after the test); nullptr = off
  double* history = nullptr;
  int history_len = 0;
  // device-resident Newton loop: the iteration index comes from flags->iter, which the
  // check advances; with set_cond the check also sets the graph's while condition (go on
  // unless the loop must stop: converged, cap reached, bad input, timeout, or non-finite
  // residuals without the reset heuristic)
  int device_it = 0;
  int set_cond = 0;
  int reset = 0;
  cudaGraphConditionalHandle cond = 0;
};

// Whole solve of short sequences, one thread-block cluster per sequence (full Jacobian,
// no damping or scale damping; the kinds and state sizes block_solve_max_T accepts).
template <class real>
struct BlockSolveArgs {
  DynView<real> dv;
  int64_t B;
  int64_t max_T;           // longest sequence (sets the cluster size)
  const int64_t* offsets;  // [B+1]
  const real* s0;          // [B][d]
  real* s;                 // [N][d]: the initial guess in, the last iterate out
  SeqInfo* info;           // [B]
  Flags* flags;            // n_active += unconverged sequences, n_nonfinite += ...
  double tol;
  int max_iters, confirm, reset, damp;
  real dparam, reset_thr;
};
// longest sequence the block solve takes for this kind and state size (0: not built)
int64_t block_solve_max_T(int kind, int d);
template <class real>
cudaError_t launch_block_solve(const BlockSolveArgs<real>& a, cudaStream_t st);

// offsets[b] = b T and chunk_first[b] = b ceil(T / L) for b = 0..B (B + 1 entries each)
cudaError_t launch_uniform_tables(int64_t* offsets, int64_t* chunk_first, int64_t B,
                                  int64_t T, int64_t chunks_per_seq, cudaStream_t st);

// first node of the device-resident loop's graph: sets the while condition from the flags
// of the check that ran before the graph
cudaError_t launch_loop_gate(Flags* flags, int max_iters, int reset,
                             cudaGraphConditionalHandle cond, cudaStream_t st);

// Dense (FULL) correction-form scan: Delta_t = A_t Delta_{t-1} + b_t, Delta_0 = 0,
// then s_t += Delta_t. Chunk aggregates hold (P, v) = (A_n...A_1, local Delta).
template <class real>
struct DenseScanArgs {
  Batch bt;
  int d;
  const real* A;   // [N][d][d]
  const real* b;   // [N][d]
  real* s;         // [N][d] updated in place
  real* aggP;      // [n_chunks][d][d]
  real* aggv;      // [n_chunks][d]
  real* cin;       // [n_chunks][d] carry into each chunk
  const SeqInfo* info;
  int reset;
  real reset_thr;
  real* slo = nullptr;  // compensation of s ([N][d]): s + slo += Delta exactly; nullptr = off
  int tensor_cores = 0;  // d = 32 float32: chunk products on the tensor cores
};

// Diagonal-family scan in standard form: s_t = a_t s_{t-1} + b_t from s_0, where a_t is
// read (DIAG), a constant (IDENTITY / ZERO, after damping), or the Kalman-damped
// transition Gamma_t a_t with offset Gamma_t b_t + (1 - Gamma_t) y_t (ELK).
template <class real>
struct DiagScanArgs {
  Batch bt;
  int d;
  int amode;        // 0 = read a, 1 = constant aconst
  real aconst;
  const real* a;    // [N][d]
  const real* b;    // [N][d]
  const real* s0;   // [B][d]
  real* s;          // [N][d]: input y (ELK emissions) and output
  real* aggA;       // [n_chunks][d]
  real* aggB;       // [n_chunks][d]
  real* cin;        // [n_chunks][d]
  const SeqInfo* info;
  int elk;          // 1: Kalman-filter damping with sigma2 = 1/lambda
  real sigma2;
  real* mob;        // [n_chunks][d][4] Moebius aggregates (ELK)
  real* pin;        // [n_chunks][d] filtered variance entering each chunk (ELK)
  int reset;
  real reset_thr;
};

template <class real>
cudaError_t launch_ma_setup(int64_t n_seq, int d, int R, const real* k, int64_t kstride,
                            const int32_t* topo, int64_t tstride, real* out, int64_t ostride,
                            int32_t* bad, cudaStream_t st);
template <class real>
cudaError_t launch_init(const InitArgs<real>& a, cudaStream_t st);
template <class real>
cudaError_t launch_linearize(const LinArgs<real>& a, cudaStream_t st);
template <class real>
cudaError_t launch_rollout(const RolloutArgs<real>& a, cudaStream_t st);
template <class real>
cudaError_t launch_gru_setup(int d, const real* params, int d_in, real* M, cudaStream_t st);
// Input gradient of the adjoint: dx[row] = lambda_row^T d f_row / d x_row at s_{row-1}.
template <class real>
struct InputGradArgs {
  DynView<real> dv;
  Batch bt;           // offsets of the packed batch (rows of every sequence)
  const real* s0;     // [B][d]
  const real* s;      // [N][d] trajectory
  const real* lam;    // [N][d] adjoint states
  real* dx;           // [N][d_in]
};

template <class real>
cudaError_t launch_input_grad(const InputGradArgs<real>& a, cudaStream_t st);
template <class real>
cudaError_t launch_input_grad_basic(const InputGradArgs<real>& a, cudaStream_t st);
template <class real>
cudaError_t launch_input_grad_models(const InputGradArgs<real>& a, cudaStream_t st);

// Generic-kernel launchers per group of kinds (each group in its own translation unit):
// Brusselator, GRU and affine ("basic"); mean-field RNN, Langevin, Lorenz-96 and
// permutation ("models").
template <class real>
cudaError_t launch_init_basic(const InitArgs<real>& a, cudaStream_t st);
template <class real>
cudaError_t launch_linearize_basic(const LinArgs<real>& a, cudaStream_t st);
template <class real>
cudaError_t launch_rollout_basic(const RolloutArgs<real>& a, cudaStream_t st);
template <class real>
cudaError_t launch_init_models(const InitArgs<real>& a, cudaStream_t st);
template <class real>
cudaError_t launch_linearize_models(const LinArgs<real>& a, cudaStream_t st);
template <class real>
cudaError_t launch_rollout_models(const RolloutArgs<real>& a, cudaStream_t st);

cudaError_t launch_check(const CheckArgs& a, cudaStream_t st);

template <class real>
cudaError_t launch_dense_scan(const DenseScanArgs<real>& a, cudaStream_t st);
template <class real>
cudaError_t launch_diag_scan(const DiagScanArgs<real>& a, cudaStream_t st);

}  // namespace deer

namespace deer {

// Reverse (adjoint) dense scan: lambda_t = A_{t+1}^T lambda_{t+1} + g_t within each
// sequence, lambda_{T+1} = 0 (Eq. bptt_lds run backwards in time).
template <class real>
struct AdjScanArgs {
  Batch bt;
  int d;
  const real* A;    // [N][d][d] Jacobians A_t at the fixed point
  const real* g;    // [N][d] cotangents dl/ds_t
  real* lam;        // [N][d] output adjoints
  real* aggP;       // [n_chunks][d][d]
  real* aggv;       // [n_chunks][d]
  real* cin;        // [n_chunks][d]
};

template <class real>
cudaError_t launch_adjoint_scan(const AdjScanArgs<real>& a, cudaStream_t st);

// Parameter gradient sum_t lambda_t^T df_t/dtheta (s_{t-1}) and dl/ds0 = A_1^T lambda_1.
template <class real>
struct ParamGradArgs {
  DynView<real> dv;
  Batch bt;
  const real* s0;
  const real* s;       // fixed point [N][d]
  const real* lam;     // [N][d]
  const real* A;       // [N][d][d]
  real* dparams;       // [B][P] or nullptr (accumulated with atomics: zero it first)
  int64_t pstride;     // P
  real* ds0;           // [B][d] or nullptr
};

template <class real>
cudaError_t launch_param_grad(const ParamGradArgs<real>& a, cudaStream_t st);

}  // namespace deer

namespace deer {

// Single-pass diagonal scan with decoupled look-back (standard form, no damping):
// one CTA per active chunk (tile), tiles taken in order from a ticket counter.
template <class real>
struct DiagLBArgs {
  Batch bt;
  int d;
  int amode;            // 0 = read a, 1 = constant aconst
  real aconst;
  const real* a;        // [N][d]
  const real* b;        // [N][d]
  const real* s0;       // [B][d]
  real* s;              // [N][d] output
  unsigned* ticket;     // tile counter, zeroed before the launch
  unsigned* flags;      // [n_chunks] (epoch << 2) | state, state 1 = aggregate, 2 = prefix
  real* agg;            // [n_chunks][d][2] tile aggregates (A, B)
  real* pre;            // [n_chunks][d] state at the end of the tile
  unsigned epoch;       // distinct per launch within one solve (starts at 1)
  // device-resident loop: the epoch is read from epoch_from->iter, the count of checks
  // done, which grows by one per launch; nullptr = `epoch`
  const Flags* epoch_from = nullptr;
  int64_t cps;          // > 0: every active sequence has this many chunks and tickets
                        // are dealt round-robin over the sequences (tile k of every
                        // sequence before tile k+1 of any), which keeps look-back short
  Flags* status;        // timeout reporting
  int reset;
  real reset_thr;
};

// chunk length used by the look-back kernel for state size d (d % 4 == 0)
inline int diag_lb_chunk(int d) { return d >= 8 ? 8192 / d : 1024; }

template <class real>
cudaError_t launch_diag_lookback(const DiagLBArgs<real>& a, cudaStream_t st,
                                 unsigned first_ticket = 0);

}  // namespace deer

namespace deer {

// Fused dense (full-Jacobian) iteration for d <= 8:
//   mode 0: linearise at the current iterate and reduce every chunk to its aggregate;
//   mode 1: first apply the pending scan (Delta_t = A_t Delta_{t-1} - r_t from the chunk's
//           carry, s_t += Delta_t), then linearise at the new iterate in the same pass.
// Mass-action kinetics with d = 4, 8 run lane-per-species (d lanes per chunk) and keep
// A_t, b_t = -r_t chunk-major: A at ((c L + t) d + i) d + j, b at (c L + t) d + i, so a
// group's d lanes touch d*d contiguous values per row. The other dynamics run one thread
// per chunk with a chunk-interleaved layout (element e of row t of chunk c at
// ((c/32 * L + t) * E + e) * 32 + c%32, E = d*d or d) so that the 32 lanes of a warp, which
// walk 32 chunks in step, touch 128 contiguous bytes per access.
template <class real>
struct FusedArgs {
  DynView<real> dv;
  Batch bt;
  const real* s0;
  real* s;
  real* Ai;          // pending Jacobians (layout above)
  real* bi;          // pending offsets -r_t
  real* aggP;        // [n_chunks][d][d]
  real* aggv;        // [n_chunks][d]
  real* cin;         // [n_chunks][d]  Delta entering each chunk
  real* sprev;       // [n_chunks][d]  new state at the row before each chunk
  SeqAcc* acc;
  int damp;
  real dparam;
  int reset;
  real reset_thr;
  int mode;
  real tol = real(0);  // see LinArgs::tol
  // compensated state (mass-action kinetics, lane-per-species kernels): slo [N][d] is the
  // part of the state below the half ulp of s, sprev_lo [n_chunks][d] that of sprev;
  // nullptr = plain state
  real* slo = nullptr;
  real* sprev_lo = nullptr;
};

template <class real>
cudaError_t launch_dense_fused(const FusedArgs<real>& a, cudaStream_t st);
template <class real>
cudaError_t launch_dense_fused_carry(const FusedArgs<real>& a, cudaStream_t st);

inline bool dense_fused_supported(int kind, int d) {
  // the kinds of the thesis's second workloads (RNN, Langevin, Lorenz-96, permutation)
  // take the unfused linearise + dense scan path
  return kind <= DEER_F_LINEAR && (d == 1 || d == 2 || d == 4 || d == 8);
}

}  // namespace deer

namespace deer {

// GRU linearisation for d = d_in = 64 in float32 (quasi-DEER family): rows are processed in
// tiles of 64 time steps by persistent CTAs holding U_z^T, U_r^T, U_h^T and M^T (M_ij =
// U_h,ij U_r,ji) in shared memory; the input projections W x_t are computed once per solve.
struct GruTileArgs {
  DynView<float> dv;
  Batch bt;
  const float* s0;
  const float* s;
  const float* xproj;   // [N][3][64] = W_z x_t, W_r x_t, W_h x_t
  float* A;             // [N][64] diag A~_t (DIAG only)
  float* b;             // [N][64]
  SeqAcc* acc;
  Flags* status;        // timeout flag of the bounded waits (tensor-core variant)
  int jac, damp;
  float dparam;
  float tol_f = 0.f;    // see LinArgs::tol
};

cudaError_t launch_gru_xproj(const float* W, const float* x, int64_t N, float* out,
                             cudaStream_t st);
cudaError_t launch_gru_lin_tiled(const GruTileArgs& a, cudaStream_t st);
// the same linearisation with the three products on tcgen05 (kind::tf32, split to float32
// accuracy); one persistent CTA per SM
cudaError_t launch_gru_lin_tc(const GruTileArgs& a, cudaStream_t st);

inline bool gru_tiled_supported(int kind, int d, int d_in, int jac, int prec) {
  return kind == DEER_F_GRU && d == 64 && d_in == 64 && jac != DEER_JAC_FULL &&
         prec == DEER_FP32;
}

}  // namespace deer

#include <cuda_bf16.h>

namespace deer {

// Mixed precision (DEER_MIXED_BF16), mass action with d = 16 / 32, full Jacobian:
// float64 state, dynamics value and residual; float32 Jacobian arithmetic stored as
// E_t = A_t - I in bfloat16; the correction-form scan Delta_t = (I + E_t) Delta_{t-1} - r_t
// accumulates in float32 and the update s += Delta is applied in float64.
struct MixedLinArgs {
  DynView<double> dv;
  Batch bt;
  const int32_t* adj_off;  // [n_seq][d+1] per-species offsets into adj_e
  const int32_t* adj_e;    // [n_seq][4R] (reaction | (nu + 4) << 16)
  int64_t adj_stride;      // 0 when the topology is shared
  const double* s0;
  const double* s;
  __nv_bfloat16* E;   // [N][d][d]
  float* b;           // [N][d]  (-r_t)
  SeqAcc* acc;
  const SeqInfo* info;  // previous check's max scaled residual selects the value path
  int it;               // iteration (0: no previous residual yet)
  int damp;
  double dparam;
  float scale_f;        // (1 - k) under scale damping, else 1
  float dt_f;
  float tol_f = 0.f;    // see LinArgs::tol
};

struct MixedScanArgs {
  Batch bt;
  int d;
  const __nv_bfloat16* E;
  const float* b;
  double* s;
  float* aggP;  // [n_chunks][d][d]
  float* aggv;  // [n_chunks][d]
  float* cin;   // [n_chunks][d]
  int reset;
  double reset_thr;
  int tc_mode = 1;          // d = 16 chunk pass: 1 warp-level bf16 MMAs, 2 tcgen05
                            // block-diagonal MMAs (8 chunks per CTA)
  Flags* status = nullptr;  // timeout flag of the bounded waits (tcgen05 variant)
};

// Mixed-precision iteration without stored Jacobians (d = 16): the linearisation of each
// chunk forms the chunk's aggregate as it goes (no E, no b in HBM), and the scan's final
// pass linearises the chunk again from the same old iterate to apply the correction.
// The two passes take the same value path per sequence (fastsel, decided by the first),
// so the recomputed E_t and r_t equal the ones the aggregates were formed from.
struct MixedRcArgs {
  MixedLinArgs lin;     // E and b unused
  float* aggP;          // [n_chunks][16][16]
  float* aggv;          // [n_chunks][16]
  const float* cin;     // [n_chunks][16] Delta entering each chunk (carry pass)
  double* sbound;       // [n_chunks][16] old state at the row before each chunk
  uint8_t* fastsel;     // [B] value path of the sequence in this iteration (1 = float32)
  int reset;
  double reset_thr;
};

cudaError_t launch_lin_ma_mixed(const MixedLinArgs& a, cudaStream_t st);
cudaError_t launch_mixed_lin_agg(const MixedRcArgs& a, cudaStream_t st);
cudaError_t launch_mixed_apply_rc(const MixedRcArgs& a, const MixedScanArgs& carry,
                                  cudaStream_t st);
// per-sequence species -> (reaction, stoichiometric coefficient) lists for the mixed kernel
cudaError_t launch_ma_adjacency(int64_t n_seq, int d, int R, const int32_t* topo,
                                int64_t tstride, int32_t* adj_off, int32_t* adj_e,
                                cudaStream_t st);
cudaError_t launch_dense_scan_mixed(const MixedScanArgs& a, cudaStream_t st);
cudaError_t launch_mixed_chunk_tcgen05(const MixedScanArgs& a, cudaStream_t st);

inline bool mixed_supported(int kind, int d, int jac) {
  return (kind == DEER_F_MASSACTION_RK4 || kind == DEER_F_MASSACTION_EULER) &&
         (d == 16 || d == 32) && jac == DEER_JAC_FULL;
}

}  // namespace deer

namespace deer {

// Largest Lyapunov exponent of each of B sequences of T steps from the stored step
// Jacobians (A [B*T][d][d], row-major, J_t at row b*T + t - 1) and unit start vectors
// u0 [B][d]; out [B] (float64).
template <class real>
struct LleArgs {
  int64_t B, T;
  int d;
  const real* A;
  const real* u0;
  double* out;
};

template <class real>
cudaError_t launch_lle(const LleArgs<real>& a, cudaStream_t st);

}  // namespace deer

namespace deer {

// Dense ELK (Kalman-filter damping of the full-Jacobian step): rewrites the linearised
// A [N][d][d] and b [N][d] of the active rows in place as Gamma_t A_t, Gamma_t b_t.
template <class real>
struct ElkDenseArgs {
  Batch bt;
  int d;
  real* A;
  real* b;
  real lambda;
  // parallel-in-time covariance (nullptr = one dependent chain per sequence): the chunks'
  // covariance elements (A, C, J) [n_chunks][3][d][d] and the filtered covariance entering
  // each chunk [n_chunks][d][d]
  real* cov_agg = nullptr;
  real* cov_in = nullptr;
};

template <class real>
cudaError_t launch_elk_dense(const ElkDenseArgs<real>& a, cudaStream_t st);

}  // namespace deer
