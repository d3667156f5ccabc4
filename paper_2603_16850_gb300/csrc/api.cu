// Host side of the C ABI: argument checks, workspace layout and the Newton loop of
// Algorithm alg:deer (linearise -> convergence test -> parallel scan, repeated).
#include <atomic>
#include <cmath>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <vector>

#include "kernels.h"

namespace deer {

static std::atomic<int64_t> g_launches{0};
static thread_local char g_err[256] = "";

void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Optional per-phase timing with CUDA events on the solver's stream (deer_profile_*).
enum { PH_SETUP = 0, PH_LIN = 1, PH_CHECK = 2, PH_SCAN = 3, PH_N = 4 };
static std::atomic<int> g_prof_on{0};
static std::atomic<int> g_tensor_cores{1};
static std::mutex g_prof_mu;
static deer_profile g_prof{};

struct PhaseTimer {
  bool on;
  cudaStream_t st;
  cudaEvent_t ev[PH_N][2];
  bool used[PH_N];
  explicit PhaseTimer(cudaStream_t s) : on(g_prof_on.load() != 0), st(s) {
    for (int p = 0; p < PH_N; ++p) {
      used[p] = false;
      if (on) { cudaEventCreate(&ev[p][0]); cudaEventCreate(&ev[p][1]); }
    }
  }
  ~PhaseTimer() {
    if (!on) return;
    for (int p = 0; p < PH_N; ++p) { cudaEventDestroy(ev[p][0]); cudaEventDestroy(ev[p][1]); }
  }
  void begin(int p) { if (on) cudaEventRecord(ev[p][0], st); }
  void end(int p) { if (on) { cudaEventRecord(ev[p][1], st); used[p] = true; } }
  // call after the stream has been synchronised
  void collect(const int64_t* launches, const int64_t* rows) {
    if (!on) return;
    std::lock_guard<std::mutex> g(g_prof_mu);
    for (int p = 0; p < PH_N; ++p) {
      if (!used[p]) continue;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[p][0], ev[p][1]) == cudaSuccess) g_prof.ms[p] += ms;
      g_prof.launches[p] += launches[p];
      g_prof.rows[p] += rows[p];
      used[p] = false;
    }
  }
};

static deer_status cuda_fail(cudaError_t e, const char* where) {
  snprintf(g_err, sizeof(g_err), "%s: %s", where, cudaGetErrorString(e));
  return DEER_ERR_CUDA;
}

#define DEER_CK(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

static bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

static int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

static size_t align_up(size_t v, size_t a = 256) { return (v + a - 1) / a * a; }

// Supported state sizes per kind (the kernels are instantiated for these).
static bool d_supported(int kind, int d, int jac) {
  if (kind == DEER_F_BRUSSELATOR_EULER) return d == 2;
  const bool p2 = d == 1 || d == 2 || d == 4 || d == 8 || d == 16 || d == 32;
  if (kind == DEER_F_GRU) return p2 || (d == 64 && jac != DEER_JAC_FULL);
  if (kind == DEER_F_MASSACTION_EULER || kind == DEER_F_MASSACTION_RK4) return p2 && d >= 2;
  if (kind == DEER_F_LORENZ96_DP5) return d == 4 || d == 5 || d == 8;
  if (kind == DEER_F_PERMUTE) return (p2 && d >= 2) || d == 5;
  return p2;
}

// Kinds whose input rows have d entries (the GRU's have d_in).
static bool input_is_d(int kind) {
  return kind == DEER_F_LINEAR || kind == DEER_F_RNN_TANH || kind == DEER_F_LANGEVIN_2WELL ||
         kind == DEER_F_PERMUTE;
}

// Kinds whose f_t cannot be evaluated without inputs.
static bool needs_x(int kind) { return kind == DEER_F_GRU || kind == DEER_F_PERMUTE; }

// Smallest per-sequence parameter stride of a kind (0: no parameters read).
static int64_t min_param_stride(const deer_dynamics* f) {
  switch (f->kind) {
    case DEER_F_BRUSSELATOR_EULER: return 2;
    case DEER_F_MASSACTION_EULER:
    case DEER_F_MASSACTION_RK4: return f->n_reactions;
    case DEER_F_RNN_TANH: return (int64_t)f->d * f->d;
    case DEER_F_LANGEVIN_2WELL: return 4 * (int64_t)f->d + 2;
    case DEER_F_LORENZ96_DP5: return 1;
    default: return 0;
  }
}

// Everything the solver carves out of the caller's workspace.
struct Layout {
  size_t offsets, chunk_first, win_chunk, act_seq, act_row_off, act_chunk_off, acc, info, flags,
      ma, gru_M,
      A, b, aggP, aggv, cin, mob, pin, sprev, lb_ticket, lb_flags, lb_agg, lb_pre, xproj,
      adj_off, adj_e, slo, sprev_lo, sbound, fastsel, cov_agg, cov_in, total;
  bool cs;         // compensated float32 state
  bool mixed_rc;   // mixed precision without stored Jacobians
  int64_t n_chunks_max;
  int64_t ma_stride, n_ma;
  int L;
};

// Diagonal-family solves without Kalman damping run the single-pass look-back scan when
// d is a multiple of 4; its tile length is fixed by d.
static bool use_diag_lookback(const deer_options* o, int d) {
  return o->jac != DEER_JAC_FULL && o->damp != DEER_DAMP_ELK && d % 4 == 0 && d >= 4 &&
         d <= 64;
}

// Compensated float32 state: the mass-action kinetics with the full Jacobian on the
// lane-per-species fused path (d = 4, 8) and the wide path (d = 16, 32).
static bool use_compensated(const deer_dynamics* f, const deer_options* o) {
  const bool ma = f->kind == DEER_F_MASSACTION_EULER || f->kind == DEER_F_MASSACTION_RK4;
  return o->prec == DEER_FP32 && o->compensate && ma && o->jac == DEER_JAC_FULL &&
         o->damp != DEER_DAMP_ELK && (f->d == 4 || f->d == 8 || f->d == 16 || f->d == 32);
}

static int choose_chunk(const deer_options* o, int d) {
  if (use_diag_lookback(o, d)) return diag_lb_chunk(d);
  if (o->chunk > 0) return o->chunk;
  if (o->jac == DEER_JAC_FULL) return d >= 16 ? 32 : 64;
  return 128;
}

// Largest row count any layout accepts: keeps every size product below (N + C) d^2 * 8
// far from overflowing 64 bits (d <= 64).
constexpr int64_t kMaxRows = int64_t(1) << 44;

static bool make_layout(const deer_dynamics* f, int64_t B, int64_t N, const deer_options* o,
                        Layout& ly) {
  if (!f || !o || B < 0 || N < 0) return false;
  if (N > kMaxRows || B > kMaxRows || f->d <= 0 || f->d > 64) return false;
  if (o->prec != DEER_FP64 && o->prec != DEER_FP32 && o->prec != DEER_MIXED_BF16) return false;
  const size_t rs = o->prec == DEER_FP32 ? 4 : 8;
  const bool mixed = o->prec == DEER_MIXED_BF16;
  const int d = f->d;
  const int L = choose_chunk(o, d);
  if (!pow2(L) || L < 8 || L > 1024) return false;
  ly.L = L;
  ly.n_chunks_max = N / L + B + 1;
  const int64_t C = ly.n_chunks_max;
  size_t p = 0;
  auto take = [&](size_t bytes) { size_t at = p; p = align_up(p + bytes); return at; };
  ly.offsets = take((size_t)(B + 1) * 8);
  ly.chunk_first = take((size_t)(B + 1) * 8);
  ly.win_chunk = take((size_t)(B + 1) * 8);
  ly.act_seq = take((size_t)(B + 1) * 8);
  ly.act_row_off = take((size_t)(B + 1) * 8);
  ly.act_chunk_off = take((size_t)(B + 1) * 8);
  ly.acc = take((size_t)(B > 0 ? B : 1) * sizeof(SeqAcc));
  ly.info = take((size_t)(B > 0 ? B : 1) * sizeof(SeqInfo));
  ly.flags = take(sizeof(Flags));
  ly.ma = ly.gru_M = ly.A = ly.aggP = ly.mob = ly.pin = ly.cov_agg = ly.cov_in = p;
  ly.ma_stride = 0;
  ly.n_ma = 0;
  if (f->kind == DEER_F_MASSACTION_EULER || f->kind == DEER_F_MASSACTION_RK4) {
    ly.ma_stride = (int64_t)d * d + (int64_t)d * d * d;
    ly.ma_stride = (ly.ma_stride + 3) / 4 * 4;
    const bool shared = f->params_stride == 0 && f->topology_stride == 0;
    ly.n_ma = shared ? 1 : B;
    ly.ma = take((size_t)(ly.n_ma > 0 ? ly.n_ma : 1) * ly.ma_stride * rs);
  }
  if (f->kind == DEER_F_GRU) ly.gru_M = take((size_t)d * d * rs);
  // mixed precision, d = 16: the Jacobians are not stored when they would exceed the bound
  ly.mixed_rc = mixed && d == 16 && o->jac_bytes_max > 0 &&
                (double)N * d * d * 2 > (double)o->jac_bytes_max;
  ly.sbound = ly.fastsel = p;
  if (ly.mixed_rc) {
    ly.sbound = take((size_t)C * d * 8);
    ly.fastsel = take((size_t)(B > 0 ? B : 1));
  } else if (mixed) {
    // bfloat16 E = A - I, float32 offsets and aggregates
    ly.A = take((size_t)N * d * d * 2);
    ly.b = take((size_t)N * d * 4);
  } else if (o->jac == DEER_JAC_FULL && o->damp != DEER_DAMP_ELK &&
             dense_fused_supported(f->kind, d)) {
    // pending Jacobians / offsets of the fused path (chunk-major or chunk-interleaved),
    // padded to whole chunks and to groups of 32 chunks
    const size_t rows = (size_t)((C + 31) / 32 * 32) * L;
    ly.A = take(rows * d * d * rs);
    ly.b = take(rows * d * rs);
  } else {
    if (o->jac == DEER_JAC_FULL) ly.A = take((size_t)N * d * d * rs);
    else if (o->jac == DEER_JAC_DIAG) ly.A = take((size_t)N * d * rs);
    ly.b = take((size_t)N * d * rs);
  }
  const size_t ars = mixed ? 4 : rs;
  if (o->jac == DEER_JAC_FULL) ly.aggP = take((size_t)C * d * d * ars);
  ly.aggv = take((size_t)C * d * ars);
  ly.cin = take((size_t)C * d * ars);
  // diag family also needs a second aggregate array; reuse aggP slot for it
  if (o->jac != DEER_JAC_FULL) ly.aggP = take((size_t)C * d * rs);
  if (o->damp == DEER_DAMP_ELK) {
    ly.mob = take((size_t)C * d * 4 * rs);
    ly.pin = take((size_t)C * d * rs);
    if (o->jac == DEER_JAC_FULL) {
      // dense ELK's covariance in parallel over time: chunk elements and carried covariances
      ly.cov_agg = take((size_t)C * 3 * d * d * rs);
      ly.cov_in = take((size_t)C * d * d * rs);
    }
  }
  ly.adj_off = ly.adj_e = p;
  const bool ma_kind = f->kind == DEER_F_MASSACTION_EULER || f->kind == DEER_F_MASSACTION_RK4;
  if (mixed || (ma_kind && (d == 16 || d == 32))) {
    // per-species reaction lists (the mixed path's and the wide linearisation's)
    const int64_t nseq = f->topology_stride ? (B > 0 ? B : 1) : 1;
    ly.adj_off = take((size_t)nseq * (d + 1) * 4);
    ly.adj_e = take((size_t)nseq * 4 * f->n_reactions * 4);
  }
  ly.xproj = p;
  if (gru_tiled_supported(f->kind, d, f->d_in, o->jac, o->prec))
    ly.xproj = take((size_t)N * 3 * d * rs);
  ly.sprev = p;
  if (!mixed && o->jac == DEER_JAC_FULL && o->damp != DEER_DAMP_ELK &&
      dense_fused_supported(f->kind, d))
    ly.sprev = take((size_t)C * d * rs);
  ly.cs = use_compensated(f, o);
  ly.slo = ly.sprev_lo = p;
  if (ly.cs) {
    ly.slo = take((size_t)N * d * 4);
    if (d <= 8) ly.sprev_lo = take((size_t)C * d * 4);
  }
  ly.lb_ticket = ly.lb_flags = ly.lb_agg = ly.lb_pre = p;
  if (use_diag_lookback(o, d)) {
    ly.lb_ticket = take(256);
    ly.lb_flags = take((size_t)C * 4);
    ly.lb_agg = take((size_t)C * d * 2 * rs);
    ly.lb_pre = take((size_t)C * d * rs);
  }
  ly.total = p;
  return true;
}

// Rows per time window of the memory-bounded adjoint: the step Jacobians of all B sequences
// over W rows take B W d^2 values; 0 = no bound (every Jacobian stored at once).
static int64_t grad_window_rows(const deer_dynamics* f, int64_t B, int64_t T,
                                const deer_options* o) {
  if (o->jac_bytes_max <= 0 || B <= 0) return T;
  const size_t rs = o->prec == DEER_FP32 ? 4 : 8;
  const int64_t per_row = B * (int64_t)f->d * f->d * (int64_t)rs;
  int64_t W = o->jac_bytes_max / per_row;
  if (W < 1) W = 1;
  return W < T ? W : T;
}

// Workspace of the windowed adjoint: the layout of a problem of B sequences of W rows, and
// per window the adjoints, the gathered trajectory, cotangents and inputs, the states
// before the window and two carries [B][d].
struct GradWinLayout {
  Layout ly;
  size_t lam, s, g, x, dx, s0, carry0, carry1, total;
};

static bool grad_win_layout(const deer_dynamics* f, int64_t B, int64_t W, const deer_options* o,
                            bool has_x, bool want_dx, GradWinLayout& gl) {
  if (!make_layout(f, B, B * W, o, gl.ly)) return false;
  const size_t rs = o->prec == DEER_FP32 ? 4 : 8;
  const int din = input_is_d(f->kind) ? f->d : f->d_in;
  size_t p = gl.ly.total;
  auto take = [&](size_t bytes) { size_t at = p; p = align_up(p + bytes); return at; };
  gl.lam = take((size_t)B * W * f->d * rs);
  gl.s = take((size_t)B * W * f->d * rs);
  gl.g = take((size_t)B * W * f->d * rs);
  gl.x = has_x ? take((size_t)B * W * din * rs) : p;
  gl.dx = want_dx ? take((size_t)B * W * din * rs) : p;
  gl.s0 = take((size_t)B * f->d * rs);
  gl.carry0 = take((size_t)B * f->d * rs);
  gl.carry1 = take((size_t)B * f->d * rs);
  gl.total = p;
  return true;
}

template <class real>
static DynView<real> make_view(const deer_dynamics* f, const void* x, char* ws,
                               const Layout& ly) {
  DynView<real> v;
  v.kind = f->kind;
  v.d = f->d;
  v.d_in = input_is_d(f->kind) ? f->d : f->d_in;
  v.R = f->n_reactions;
  v.dt = (real)f->dt;
  v.params = static_cast<const real*>(f->params);
  v.pstride = f->params_stride;
  v.topo = f->topology;
  v.tstride = f->topology_stride;
  v.x = static_cast<const real*>(x);
  v.ma = ws ? reinterpret_cast<const real*>(ws + ly.ma) : nullptr;
  v.ma_stride = ly.n_ma == 1 ? 0 : ly.ma_stride;
  v.gru_M = ws ? reinterpret_cast<const real*>(ws + ly.gru_M) : nullptr;
  return v;
}

static deer_status check_common(const deer_dynamics* f, const deer_options* o) {
  if (!f || !o) return DEER_ERR_INVALID;
  if (f->kind < 0 || f->kind > DEER_F_PERMUTE) return DEER_ERR_INVALID;
  if (o->jac < 0 || o->jac > DEER_JAC_ZERO) return DEER_ERR_INVALID;
  if (o->damp < 0 || o->damp > DEER_DAMP_CLIP) return DEER_ERR_INVALID;
  if (o->init < 0 || o->init > DEER_INIT_RANDN) return DEER_ERR_INVALID;
  if (o->history_len < 0 || (o->history_len > 0 && !o->history)) return DEER_ERR_INVALID;
  if (o->jac_bytes_max < 0) return DEER_ERR_INVALID;
  if (o->prec != DEER_FP64 && o->prec != DEER_FP32 && o->prec != DEER_MIXED_BF16)
    return DEER_ERR_INVALID;
  if (o->prec == DEER_MIXED_BF16 &&
      (!mixed_supported(f->kind, f->d, o->jac) || f->n_reactions > 64 ||
       (o->damp != DEER_DAMP_NONE && o->damp != DEER_DAMP_SCALE)))
    return DEER_ERR_UNSUPPORTED;
  if (!d_supported(f->kind, f->d, o->jac)) return DEER_ERR_UNSUPPORTED;
  // dense ELK: the covariance recursion is built for d <= 16
  if (o->damp == DEER_DAMP_ELK && o->jac == DEER_JAC_FULL &&
      !(f->d == 1 || f->d == 2 || f->d == 4 || f->d == 8 || f->d == 16))
    return DEER_ERR_UNSUPPORTED;
  if (o->damp == DEER_DAMP_CLIP && o->jac == DEER_JAC_FULL) return DEER_ERR_INVALID;
  if (o->damp == DEER_DAMP_ELK && !(o->damp_param >= 0.0)) return DEER_ERR_INVALID;
  if (o->window != 0 && o->window != 1) return DEER_ERR_INVALID;
  if (!f->params) return DEER_ERR_INVALID;
  if (f->kind == DEER_F_MASSACTION_EULER || f->kind == DEER_F_MASSACTION_RK4) {
    if (!f->topology || f->n_reactions <= 0) return DEER_ERR_INVALID;
    if (f->params_stride != 0 && f->params_stride < f->n_reactions) return DEER_ERR_INVALID;
    if (f->topology_stride != 0 && f->topology_stride < 4 * (int64_t)f->n_reactions)
      return DEER_ERR_INVALID;
    if (f->topology_stride % 4 != 0) return DEER_ERR_INVALID;
  }
  if (f->kind == DEER_F_GRU && f->d_in <= 0) return DEER_ERR_INVALID;
  if (f->params_stride < 0 || (f->params_stride != 0 && f->params_stride < min_param_stride(f)))
    return DEER_ERR_INVALID;
  if ((f->kind == DEER_F_LANGEVIN_2WELL || f->kind == DEER_F_LORENZ96_DP5) && !(f->dt > 0.0))
    return DEER_ERR_INVALID;
  return DEER_OK;
}

template <class real>
static deer_status solve_impl(const deer_dynamics* f, int64_t B, const int64_t* offsets_h,
                              const void* s0_, const void* x_, void* s_, const deer_options* o,
                              void* ws_, size_t ws_bytes, cudaStream_t st, deer_info* info_h) {
  const int64_t N = offsets_h[B];
  Layout ly;
  if (!make_layout(f, B, N, o, ly)) return DEER_ERR_INVALID;
  if (!ws_ || ws_bytes < ly.total || (reinterpret_cast<uintptr_t>(ws_) & 255u))
    return DEER_ERR_WORKSPACE;
  char* ws = static_cast<char*>(ws_);
  const int d = f->d;
  const real* s0 = static_cast<const real*>(s0_);
  real* s = static_cast<real*>(s_);

  // sequence / chunk tables
  std::vector<int64_t> chunk_first(B + 1);
  int64_t maxT = 0, nc = 0;
  for (int64_t b = 0; b < B; ++b) {
    const int64_t len = offsets_h[b + 1] - offsets_h[b];
    if (len < 0) return DEER_ERR_INVALID;
    chunk_first[b] = nc;
    nc += (len + ly.L - 1) / ly.L;
    if (len > maxT) maxT = len;
  }
  chunk_first[B] = nc;
  if (offsets_h[0] != 0) return DEER_ERR_INVALID;
  int64_t* d_off = reinterpret_cast<int64_t*>(ws + ly.offsets);
  int64_t* d_cf = reinterpret_cast<int64_t*>(ws + ly.chunk_first);
  // sequences of one length (deer_solve): the tables are written on the device, which
  // spares two copies from pageable host memory per call (they dominate small solves)
  bool uniform = B > 0;
  const int64_t T0 = B > 0 ? offsets_h[1] : 0;
  for (int64_t b = 1; b <= B && uniform; ++b) uniform = offsets_h[b] == b * T0;
  if (uniform) {
    DEER_CK(launch_uniform_tables(d_off, d_cf, B, T0, (T0 + ly.L - 1) / ly.L, st));
  } else {
    DEER_CK(cudaMemcpyAsync(d_off, offsets_h, (B + 1) * 8, cudaMemcpyHostToDevice, st));
    DEER_CK(cudaMemcpyAsync(d_cf, chunk_first.data(), (B + 1) * 8, cudaMemcpyHostToDevice,
                            st));
  }
  SeqAcc* acc = reinterpret_cast<SeqAcc*>(ws + ly.acc);
  SeqInfo* info = reinterpret_cast<SeqInfo*>(ws + ly.info);
  Flags* flags = reinterpret_cast<Flags*>(ws + ly.flags);
  if (B > 0) {
    DEER_CK(cudaMemsetAsync(acc, 0, B * sizeof(SeqAcc), st));
    DEER_CK(cudaMemsetAsync(info, 0, B * sizeof(SeqInfo), st));
  }
  DEER_CK(cudaMemsetAsync(flags, 0, sizeof(Flags), st));

  Batch bt;
  bt.B = B;
  bt.N = N;
  bt.offsets = d_off;
  bt.chunk_first = d_cf;
  bt.n_chunks = nc;
  bt.L = ly.L;
  bt.log2L = ilog2(ly.L);
  bt.act_seq = reinterpret_cast<int64_t*>(ws + ly.act_seq);
  bt.act_row_off = reinterpret_cast<int64_t*>(ws + ly.act_row_off);
  bt.act_chunk_off = reinterpret_cast<int64_t*>(ws + ly.act_chunk_off);
  bt.set_counts(B, N, nc);
  int64_t* d_win = reinterpret_cast<int64_t*>(ws + ly.win_chunk);
  // the window freezes rows one iterate after they qualify, which relies on the fast
  // (quadratic) convergence of undamped steps; damped steps converge linearly and run whole
  const bool window = o->window && o->damp == DEER_DAMP_NONE;
  if (window) {
    // sliding window: every sequence starts solved from its first chunk
    DEER_CK(uniform ? cudaMemcpyAsync(d_win, d_cf, (B + 1) * 8, cudaMemcpyDeviceToDevice, st)
                    : cudaMemcpyAsync(d_win, chunk_first.data(), (B + 1) * 8,
                                      cudaMemcpyHostToDevice, st));
    bt.win_chunk = d_win;
  }
  // the convergence test in the kernels' precision: the largest value of that type not
  // above tol, so that a row passes exactly when the float64 test on its value would
  real tol_r = (real)o->tol;
  if ((double)tol_r > o->tol) tol_r = std::nextafter(tol_r, real(0));
  float tol_f = (float)o->tol;
  if ((double)tol_f > o->tol) tol_f = std::nextafter(tol_f, 0.f);

  DynView<real> dv = make_view<real>(f, x_, ws, ly);
  if (ly.n_ma > 0) {
    DEER_CK(launch_ma_setup<real>(ly.n_ma, d, f->n_reactions, static_cast<const real*>(f->params),
                                  f->params_stride, f->topology, f->topology_stride,
                                  reinterpret_cast<real*>(ws + ly.ma), ly.ma_stride,
                                  &flags->bad_input, st));
  }
  if (f->kind == DEER_F_GRU) {
    DEER_CK(launch_gru_setup<real>(d, static_cast<const real*>(f->params), f->d_in,
                                   reinterpret_cast<real*>(ws + ly.gru_M), st));
  }
  const bool gru_tiled = gru_tiled_supported(f->kind, d, f->d_in, o->jac, o->prec);
  GruTileArgs gta;
  if constexpr (sizeof(real) == 4) {
    if (gru_tiled) {
      // input projections W x_t, once per solve
      DEER_CK(launch_gru_xproj(static_cast<const float*>(f->params),
                               static_cast<const float*>(x_), N,
                               reinterpret_cast<float*>(ws + ly.xproj), st));
      gta.dv = dv;
      gta.bt = bt;
      gta.s0 = s0;
      gta.s = s;
      gta.xproj = reinterpret_cast<const float*>(ws + ly.xproj);
      gta.A = reinterpret_cast<float*>(ws + ly.A);
      gta.b = reinterpret_cast<float*>(ws + ly.b);
      gta.acc = acc;
      gta.status = flags;
      gta.jac = o->jac;
      gta.damp = o->damp;
      gta.dparam = (float)o->damp_param;
      gta.tol_f = tol_f;
    }
  }
  if (o->init != DEER_INIT_USER) {
    InitArgs<real> ia{dv, bt, s0, s, o->init};
    ia.seed = o->seed;
    DEER_CK(launch_init<real>(ia, st));
  }

  const int max_iters = o->max_iters > 0 ? o->max_iters : (int)(maxT > 0 ? maxT : 1);
  const real reset_thr = sizeof(real) == 8 ? real(1e30) : real(1e18);

  LinArgs<real> la;
  la.dv = dv;
  la.bt = bt;
  la.s0 = s0;
  la.s = s;
  la.A = reinterpret_cast<real*>(ws + ly.A);
  la.b = reinterpret_cast<real*>(ws + ly.b);
  la.acc = acc;
  la.info = info;
  la.jac = o->jac;
  la.damp = o->damp;
  la.dparam = (real)o->damp_param;
  la.tol = tol_r;
  if (!(o->prec == DEER_MIXED_BF16) && ly.adj_off != ly.adj_e) {
    // mass action, d = 16 / 32: each lane of the wide linearisation walks its species'
    // reactions
    const int64_t nseq = f->topology_stride ? B : 1;
    DEER_CK(launch_ma_adjacency(nseq, d, f->n_reactions, f->topology, f->topology_stride,
                                reinterpret_cast<int32_t*>(ws + ly.adj_off),
                                reinterpret_cast<int32_t*>(ws + ly.adj_e), st));
    la.adj_off = reinterpret_cast<const int32_t*>(ws + ly.adj_off);
    la.adj_e = reinterpret_cast<const int32_t*>(ws + ly.adj_e);
    la.adj_stride = f->topology_stride ? 4 * (int64_t)f->n_reactions : 0;
  }
  real* slo = ly.cs ? reinterpret_cast<real*>(ws + ly.slo) : nullptr;
  if (slo) {
    // the compensation terms start at zero (the initial guess is a plain float32 state)
    DEER_CK(cudaMemsetAsync(slo, 0, (size_t)N * d * sizeof(real), st));
    la.slo = slo;
  }

  CheckArgs ca{B, d_off, d_cf, acc, info, flags,
               reinterpret_cast<int64_t*>(ws + ly.act_seq),
               reinterpret_cast<int64_t*>(ws + ly.act_row_off),
               reinterpret_cast<int64_t*>(ws + ly.act_chunk_off), o->tol, 0, max_iters, 1,
               o->confirm > 1 ? o->confirm : 1};
  ca.win_chunk = window ? d_win : nullptr;
  ca.window = window ? 1 : 0;
  ca.log2L = bt.log2L;
  DEER_CK(launch_check(ca, st));  // every sequence starts active
  ca.compact_only = 0;
  ca.history = o->history;
  ca.history_len = o->history_len;

  DenseScanArgs<real> dsa;
  DiagScanArgs<real> gsa;
  if (o->jac == DEER_JAC_FULL) {
    dsa.bt = bt;
    dsa.d = d;
    dsa.A = la.A;
    dsa.b = la.b;
    dsa.s = s;
    dsa.aggP = reinterpret_cast<real*>(ws + ly.aggP);
    dsa.aggv = reinterpret_cast<real*>(ws + ly.aggv);
    dsa.cin = reinterpret_cast<real*>(ws + ly.cin);
    dsa.info = info;
    dsa.reset = o->reset;
    dsa.reset_thr = reset_thr;
    dsa.slo = slo;
    dsa.tensor_cores = g_tensor_cores.load();
  } else {
    gsa.bt = bt;
    gsa.d = d;
    gsa.amode = o->jac == DEER_JAC_DIAG ? 0 : 1;
    real ac = o->jac == DEER_JAC_IDENTITY ? real(1) : real(0);
    if (o->damp == DEER_DAMP_SCALE) ac *= real(1) - (real)o->damp_param;
    if (o->damp == DEER_DAMP_CLIP) {
      const real rho = (real)o->damp_param;
      ac = ac > rho ? rho : (ac < -rho ? -rho : ac);
    }
    gsa.aconst = ac;
    gsa.a = la.A;
    gsa.b = la.b;
    gsa.s0 = s0;
    gsa.s = s;
    gsa.aggA = reinterpret_cast<real*>(ws + ly.aggP);
    gsa.aggB = reinterpret_cast<real*>(ws + ly.aggv);
    gsa.cin = reinterpret_cast<real*>(ws + ly.cin);
    gsa.info = info;
    gsa.elk = (o->damp == DEER_DAMP_ELK && o->damp_param > 0.0) ? 1 : 0;
    gsa.sigma2 = gsa.elk ? real(1.0 / o->damp_param) : real(0);
    gsa.mob = reinterpret_cast<real*>(ws + ly.mob);
    gsa.pin = reinterpret_cast<real*>(ws + ly.pin);
    gsa.reset = o->reset;
    gsa.reset_thr = reset_thr;
  }

  const bool mixed = o->prec == DEER_MIXED_BF16;
  MixedLinArgs mla;
  MixedScanArgs msa;
  MixedRcArgs rca{};
  if constexpr (sizeof(real) == 8) {
    if (mixed) {
      const int64_t nseq = f->topology_stride ? B : 1;
      DEER_CK(launch_ma_adjacency(nseq, d, f->n_reactions, f->topology, f->topology_stride,
                                  reinterpret_cast<int32_t*>(ws + ly.adj_off),
                                  reinterpret_cast<int32_t*>(ws + ly.adj_e), st));
      mla.adj_off = reinterpret_cast<const int32_t*>(ws + ly.adj_off);
      mla.adj_e = reinterpret_cast<const int32_t*>(ws + ly.adj_e);
      mla.adj_stride = f->topology_stride ? 4 * (int64_t)f->n_reactions : 0;
      mla.dv = dv;
      mla.bt = bt;
      mla.s0 = s0;
      mla.s = s;
      mla.E = reinterpret_cast<__nv_bfloat16*>(ws + ly.A);
      mla.b = reinterpret_cast<float*>(ws + ly.b);
      mla.acc = acc;
      mla.info = info;
      mla.it = 0;
      mla.damp = o->damp;
      mla.dparam = o->damp_param;
      mla.scale_f = o->damp == DEER_DAMP_SCALE ? (float)(1.0 - o->damp_param) : 1.f;
      mla.dt_f = (float)f->dt;
      mla.tol_f = tol_f;
      msa.bt = bt;
      msa.d = d;
      msa.E = mla.E;
      msa.b = mla.b;
      msa.s = s;
      msa.aggP = reinterpret_cast<float*>(ws + ly.aggP);
      msa.aggv = reinterpret_cast<float*>(ws + ly.aggv);
      msa.cin = reinterpret_cast<float*>(ws + ly.cin);
      msa.reset = o->reset;
      msa.reset_thr = 1e18;  // the scan and the Jacobians are float32
      msa.tc_mode = g_tensor_cores.load() >= 2 ? 2 : 1;
      msa.status = flags;
      if (ly.mixed_rc) {
        rca.lin = mla;
        rca.lin.E = nullptr;
        rca.lin.b = nullptr;
        rca.aggP = msa.aggP;
        rca.aggv = msa.aggv;
        rca.cin = msa.cin;
        rca.sbound = reinterpret_cast<double*>(ws + ly.sbound);
        rca.fastsel = reinterpret_cast<uint8_t*>(ws + ly.fastsel);
        rca.reset = o->reset;
        rca.reset_thr = 1e18;
      }
    }
  }
  const bool fused = !mixed && o->jac == DEER_JAC_FULL && o->damp != DEER_DAMP_ELK &&
                     dense_fused_supported(f->kind, d);
  FusedArgs<real> fa;
  if (fused) {
    fa.dv = dv;
    fa.bt = bt;
    fa.s0 = s0;
    fa.s = s;
    fa.Ai = la.A;
    fa.bi = la.b;
    fa.aggP = reinterpret_cast<real*>(ws + ly.aggP);
    fa.aggv = reinterpret_cast<real*>(ws + ly.aggv);
    fa.cin = reinterpret_cast<real*>(ws + ly.cin);
    fa.sprev = reinterpret_cast<real*>(ws + ly.sprev);
    fa.acc = acc;
    fa.damp = o->damp;
    fa.dparam = (real)o->damp_param;
    fa.reset = o->reset;
    fa.reset_thr = reset_thr;
    fa.mode = 0;
    fa.tol = tol_r;
    fa.slo = slo;
    fa.sprev_lo = slo ? reinterpret_cast<real*>(ws + ly.sprev_lo) : nullptr;
  }

  const bool lookback = use_diag_lookback(o, d);
  // all sequences of equal length: round-robin tile order for the look-back scan
  int64_t uniform_chunks = B > 0 ? chunk_first[1] - chunk_first[0] : 0;
  for (int64_t b = 1; b < B && uniform_chunks > 0; ++b)
    if (chunk_first[b + 1] - chunk_first[b] != uniform_chunks) uniform_chunks = 0;
  DiagLBArgs<real> lba;
  if (lookback) {
    lba.bt = bt;
    lba.d = d;
    lba.amode = gsa.amode;
    lba.aconst = gsa.aconst;
    lba.a = gsa.a;
    lba.b = gsa.b;
    lba.s0 = s0;
    lba.s = s;
    lba.ticket = reinterpret_cast<unsigned*>(ws + ly.lb_ticket);
    lba.flags = reinterpret_cast<unsigned*>(ws + ly.lb_flags);
    lba.agg = reinterpret_cast<real*>(ws + ly.lb_agg);
    lba.pre = reinterpret_cast<real*>(ws + ly.lb_pre);
    lba.epoch = 0;
    lba.status = flags;
    lba.reset = o->reset;
    lba.reset_thr = reset_thr;
    DEER_CK(cudaMemsetAsync(lba.flags, 0, (size_t)ly.n_chunks_max * 4, st));
  }

  deer_status status = DEER_OK;
  Flags hf;
  PhaseTimer pt(st);

  // The steps of one iteration, shared by the host-driven loop and the graph of the
  // device-resident one, enqueued on `lst`. `b` carries the active-set sizes (host values,
  // or upper bounds with live counts).
  cudaStream_t lst = st;
  // fused path, iterations after the first: compose the previous pass's aggregates
  auto carry_step = [&](const Batch& b) -> cudaError_t {
    fa.bt = b;
    return launch_dense_fused_carry<real>(fa, lst);
  };
  auto lin_step = [&](const Batch& b, int it) -> cudaError_t {
    la.bt = b;
    if (fused) {
      fa.bt = b;
      fa.mode = it > 0 ? 1 : 0;
      return launch_dense_fused<real>(fa, lst);
    }
    if (gru_tiled) {
      if constexpr (sizeof(real) == 4) {
        gta.bt = b;
        return g_tensor_cores.load() != 0 ? launch_gru_lin_tc(gta, lst)
                                          : launch_gru_lin_tiled(gta, lst);
      }
    }
    if (mixed) {
      if constexpr (sizeof(real) == 8) {
        mla.bt = b;
        mla.it = it;
        if (ly.mixed_rc) {
          rca.lin.bt = b;
          rca.lin.it = it;
          return launch_mixed_lin_agg(rca, lst);
        }
        return launch_lin_ma_mixed(mla, lst);
      }
    }
    return launch_linearize<real>(la, lst);
  };
  // non-fused paths: solve the linearised recurrence of the last linearisation
  auto scan_step = [&](const Batch& b, bool host_loop) -> cudaError_t {
    dsa.bt = b;
    gsa.bt = b;
    if (mixed) {
      if constexpr (sizeof(real) == 8) {
        msa.bt = b;
        if (ly.mixed_rc) {
          rca.lin.bt = b;
          return launch_mixed_apply_rc(rca, msa, lst);
        }
        return launch_dense_scan_mixed(msa, lst);
      }
    }
    if (o->jac == DEER_JAC_FULL) {
      if (o->damp == DEER_DAMP_ELK && o->damp_param > 0.0) {
        // dense ELK: Kalman-filter damping of the linearised step (A, b rewritten). The
        // covariance recursion runs in parallel over time (chunk elements, carry) when
        // the sequences are long (8 or more chunks each on average) and too few to fill
        // the GPU on their own (under 1024), as one chain per sequence otherwise
        ElkDenseArgs<real> ea{b, d, la.A, la.b, (real)o->damp_param};
        if (b.n_act() < 1024 && b.act_chunks() >= 8 * b.n_act()) {
          ea.cov_agg = reinterpret_cast<real*>(ws + ly.cov_agg);
          ea.cov_in = reinterpret_cast<real*>(ws + ly.cov_in);
        }
        const cudaError_t e = launch_elk_dense<real>(ea, lst);
        if (e != cudaSuccess) return e;
      }
      return launch_dense_scan<real>(dsa, lst);
    }
    if (lookback) {
      lba.bt = b;
      lba.epoch += 1;
      // device-resident loop: the epoch comes from the check counter instead
      lba.epoch_from = host_loop ? nullptr : flags;
      // round-robin tile order assumes every sequence has the same chunks to solve,
      // which a sliding window breaks
      lba.cps = window ? 0 : uniform_chunks;
      return launch_diag_lookback<real>(lba, lst);
    }
    return launch_diag_scan<real>(gsa, lst);
  };

  // Short sequences (every one within what a thread-block cluster holds in registers)
  // with the full Jacobian: the whole loop runs inside one kernel, one cluster per
  // sequence
  const bool block_solve = !o->no_block_solve && o->jac == DEER_JAC_FULL &&
                           (o->damp == DEER_DAMP_NONE || o->damp == DEER_DAMP_SCALE) &&
                           !mixed && !ly.cs && !o->history && maxT >= 1 &&
                           maxT <= block_solve_max_T(f->kind, d) && B <= INT32_MAX;
  if (block_solve) {
    // the initial active-set pass counted every sequence; the block solve counts the
    // unconverged ones itself
    DEER_CK(cudaMemsetAsync(&flags->n_active, 0, sizeof(int32_t), st));
    BlockSolveArgs<real> ba{dv, B, maxT, d_off, s0, s, info, flags, o->tol, max_iters,
                            o->confirm > 1 ? o->confirm : 1, o->reset, o->damp,
                            (real)o->damp_param, reset_thr};
    pt.begin(PH_LIN);  // the whole loop is one launch: its time goes to linearisation
    DEER_CK(launch_block_solve<real>(ba, st));
    pt.end(PH_LIN);
    DEER_CK(cudaMemcpyAsync(&hf, flags, sizeof(Flags), cudaMemcpyDeviceToHost, st));
    DEER_CK(cudaStreamSynchronize(st));
    if (pt.on) {
      const int64_t launches[PH_N] = {0, 1, 0, 0};
      const int64_t rows[PH_N] = {0, N, 0, 0};
      pt.collect(launches, rows);
    }
    if (hf.bad_input) status = DEER_ERR_INVALID;
    else if (hf.n_nonfinite > 0 && !o->reset) status = DEER_ERR_NONFINITE;
    else if (hf.n_active > 0) status = DEER_NOT_CONVERGED;
  } else if (o->device_loop && !pt.on) {
    // Device-resident loop (opt-in): iteration 0 runs on the stream as usual; the rest is
    // one CUDA graph, a gate node and a conditional while node whose body is one iteration
    // (scan or carry, linearise, check), the check setting the condition for the next. No
    // host synchronisation between iterations; every kernel reads the active-set sizes the
    // last check wrote, and grids are sized for the whole problem (the look-back scan's
    // surplus CTAs draw tickets past the active tiles and leave). Per-phase timing keeps
    // the host loop.
    ca.it = 0;
    ca.device_it = 1;
    ca.set_cond = 0;
    ca.reset = o->reset;
    DEER_CK(lin_step(bt, 0));
    DEER_CK(launch_check(ca, st));
    Batch gb = bt;  // upper bounds: the sizes of the whole problem
    gb.live = flags;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // the graph is recorded on a private stream (the caller's may be the legacy default
    // stream, which cannot capture) and launched on the caller's
    cudaStream_t cs = nullptr;
    cudaError_t ge = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (ge == cudaSuccess) ge = cudaGraphCreate(&graph, 0);
    cudaGraphConditionalHandle cond = 0;
    int64_t body_launches = 0;
    const int64_t lg0 = g_launches.load();
    if (ge == cudaSuccess)
      ge = cudaGraphConditionalHandleCreate(&cond, graph, 0, cudaGraphCondAssignDefault);
    cudaGraphNode_t gate_node = nullptr, while_node = nullptr;
    if (ge == cudaSuccess) {
      // the gate: one kernel node
      ge = cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal);
      if (ge == cudaSuccess) {
        const cudaError_t le = launch_loop_gate(flags, max_iters, o->reset, cond, cs);
        cudaGraph_t g2 = nullptr;
        ge = cudaStreamEndCapture(cs, &g2);
        if (ge == cudaSuccess) ge = le;
      }
    }
    if (ge == cudaSuccess) {
      size_t nn = 0;
      ge = cudaGraphGetNodes(graph, nullptr, &nn);
      if (ge == cudaSuccess && nn == 1) ge = cudaGraphGetNodes(graph, &gate_node, &nn);
      else if (ge == cudaSuccess) ge = cudaErrorInvalidValue;
    }
    cudaGraph_t body = nullptr;
    if (ge == cudaSuccess) {
      cudaGraphNodeParams cp{};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = cond;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      ge = cudaGraphAddNode(&while_node, graph, &gate_node, nullptr, 1, &cp);
      if (ge == cudaSuccess) body = cp.conditional.phGraph_out[0];
    }
    if (ge == cudaSuccess) {
      ge = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal);
      if (ge == cudaSuccess) {
        const int64_t lb0 = g_launches.load();
        lst = cs;
        cudaError_t le = fused ? carry_step(gb) : scan_step(gb, false);
        if (le == cudaSuccess) le = lin_step(gb, 1);
        CheckArgs cb = ca;
        cb.set_cond = 1;
        cb.cond = cond;
        if (le == cudaSuccess) le = launch_check(cb, cs);
        lst = st;
        body_launches = g_launches.load() - lb0;
        cudaGraph_t g2 = nullptr;
        ge = cudaStreamEndCapture(cs, &g2);
        if (ge == cudaSuccess) ge = le;
      }
    }
    if (ge == cudaSuccess) ge = cudaGraphInstantiate(&exec, graph, 0);
    // the launches recorded while capturing are counted as they run (below)
    g_launches.store(lg0);
    if (ge == cudaSuccess) ge = cudaGraphLaunch(exec, st);
    if (ge == cudaSuccess)
      ge = cudaMemcpyAsync(&hf, flags, sizeof(Flags), cudaMemcpyDeviceToHost, st);
    if (ge == cudaSuccess) ge = cudaStreamSynchronize(st);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
    if (ge != cudaSuccess) return cuda_fail(ge, "device-resident Newton loop");
    // gate, then one body per check after the first
    note_launch((int)(1 + body_launches * (int64_t)(hf.iter - 1)));
    const int last = hf.iter - 1;  // index of the last check
    if (hf.bad_input) status = DEER_ERR_INVALID;
    else if (hf.timeout) status = DEER_ERR_TIMEOUT;
    else if (hf.n_nonfinite > 0 && !o->reset) status = DEER_ERR_NONFINITE;
    else if (hf.n_active == 0) status = DEER_OK;
    else if (last >= max_iters) status = DEER_NOT_CONVERGED;
  } else {
    int64_t lin_rows = N;  // rows linearised in the current iteration
    for (int it = 0;; ++it) {
      int64_t carry_launches = 0;
      if (fused && it > 0) {
        const int64_t c0l = g_launches.load();
        pt.begin(PH_SCAN);
        DEER_CK(carry_step(bt));
        pt.end(PH_SCAN);
        carry_launches = g_launches.load() - c0l;
      }
      const int64_t l0 = g_launches.load();
      pt.begin(PH_LIN);
      DEER_CK(lin_step(bt, it));
      pt.end(PH_LIN);
      const int64_t l1 = g_launches.load();
      ca.it = it;
      pt.begin(PH_CHECK);
      DEER_CK(launch_check(ca, st));
      pt.end(PH_CHECK);
      DEER_CK(cudaMemcpyAsync(&hf, flags, sizeof(Flags), cudaMemcpyDeviceToHost, st));
      DEER_CK(cudaStreamSynchronize(st));
      bool stop = false;
      if (hf.bad_input) { status = DEER_ERR_INVALID; stop = true; }
      else if (hf.timeout) { status = DEER_ERR_TIMEOUT; stop = true; }
      else if (hf.n_nonfinite > 0 && !o->reset) { status = DEER_ERR_NONFINITE; stop = true; }
      else if (hf.n_active == 0) stop = true;
      else if (it >= max_iters) { status = DEER_NOT_CONVERGED; stop = true; }
      int64_t scan_launches = carry_launches;
      bt.set_counts(hf.n_active, hf.active_rows, hf.active_chunks);
      if (!stop && !fused) {
        const int64_t s0c = g_launches.load();
        pt.begin(PH_SCAN);
        DEER_CK(scan_step(bt, true));
        pt.end(PH_SCAN);
        scan_launches = g_launches.load() - s0c;
      }
      if (pt.on) {
        DEER_CK(cudaStreamSynchronize(st));
        const int64_t launches[PH_N] = {0, l1 - l0, 1, scan_launches};
        const int64_t rows[PH_N] = {0, lin_rows, (int64_t)B,
                                    fused ? (carry_launches ? lin_rows : 0)
                                          : (stop ? 0 : (int64_t)hf.active_rows)};
        pt.collect(launches, rows);
      }
      lin_rows = hf.active_rows;
      if (stop) break;
    }
  }

  if (info_h && B > 0) {
    std::vector<SeqInfo> hi(B);
    DEER_CK(cudaMemcpyAsync(hi.data(), info, B * sizeof(SeqInfo), cudaMemcpyDeviceToHost, st));
    DEER_CK(cudaStreamSynchronize(st));
    for (int64_t b = 0; b < B; ++b) {
      info_h[b].iters = hi[b].iters;
      info_h[b].converged = hi[b].done;
      info_h[b].merit = hi[b].merit;
      info_h[b].max_resid = hi[b].max_resid;
    }
  } else {
    DEER_CK(cudaStreamSynchronize(st));
  }
  return status;
}

}  // namespace deer

using namespace deer;

extern "C" {

void deer_default_options(deer_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->max_iters = 0;
  o->tol = 1e-10;
  o->jac = DEER_JAC_FULL;
  o->damp = DEER_DAMP_NONE;
  o->damp_param = 0.0;
  o->init = DEER_INIT_S0;
  o->prec = DEER_FP64;
  o->reset = 0;
  o->chunk = 0;
  o->confirm = 1;
  o->window = 0;
  o->compensate = 1;
}

size_t deer_workspace_bytes(const deer_dynamics* f, int64_t batch, int64_t total_steps,
                            const deer_options* opt) {
  if (check_common(f, opt) != DEER_OK) return 0;
  Layout ly;
  if (!make_layout(f, batch, total_steps, opt, ly)) return 0;
  return ly.total;
}

static deer_status solve_dispatch(const deer_dynamics* f, int64_t batch, const int64_t* off,
                                  const void* s0, const void* x, void* s_out,
                                  const deer_options* opt, void* ws, size_t wsb,
                                  deer_stream_t stream, deer_info* info) {
  deer_status c = check_common(f, opt);
  if (c != DEER_OK) return c;
  if (batch < 0) return DEER_ERR_INVALID;
  if (batch == 0) return DEER_OK;
  if (!s0 || !s_out) return DEER_ERR_INVALID;
  if (needs_x(f->kind) && !x) return DEER_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (opt->prec == DEER_FP32)
    return solve_impl<float>(f, batch, off, s0, x, s_out, opt, ws, wsb, st, info);
  return solve_impl<double>(f, batch, off, s0, x, s_out, opt, ws, wsb, st, info);
}

deer_status deer_solve(const deer_dynamics* f, int64_t batch, int64_t T, const void* s0,
                       const void* x, void* s_out, const deer_options* opt, void* workspace,
                       size_t workspace_bytes, deer_stream_t stream, deer_info* info) {
  if (batch < 0 || T < 0) return DEER_ERR_INVALID;
  if (batch > 0 && T > kMaxRows / batch) return DEER_ERR_INVALID;
  std::vector<int64_t> off(batch + 1);
  for (int64_t b = 0; b <= batch; ++b) off[b] = b * T;
  return solve_dispatch(f, batch, off.data(), s0, x, s_out, opt, workspace, workspace_bytes,
                        stream, info);
}

deer_status deer_solve_batched(const deer_dynamics* f, int64_t batch, const int64_t* offsets,
                               const void* s0, const void* x, void* s_out,
                               const deer_options* opt, void* workspace, size_t workspace_bytes,
                               deer_stream_t stream, deer_info* info) {
  if (!offsets || batch < 0) return DEER_ERR_INVALID;
  for (int64_t b = 0; b < batch; ++b)
    if (offsets[b + 1] < offsets[b]) return DEER_ERR_INVALID;
  if (offsets[0] != 0) return DEER_ERR_INVALID;
  return solve_dispatch(f, batch, offsets, s0, x, s_out, opt, workspace, workspace_bytes,
                        stream, info);
}

deer_status deer_rollout(const deer_dynamics* f, int64_t batch, int64_t T,
                         const int64_t* offsets, const void* s0, const void* x, void* s_out,
                         int32_t prec, deer_stream_t stream) {
  deer_options o;
  deer_default_options(&o);
  o.prec = prec;
  o.jac = DEER_JAC_ZERO;
  deer_status c = check_common(f, &o);
  if (c != DEER_OK) return c;
  if (batch < 0 || (!offsets && T < 0)) return DEER_ERR_INVALID;
  if (batch == 0) return DEER_OK;
  if (!s0 || !s_out) return DEER_ERR_INVALID;
  if (needs_x(f->kind) && !x) return DEER_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Layout ly{};
  cudaError_t e;
  if (prec == DEER_FP32) {
    RolloutArgs<float> a{make_view<float>(f, x, nullptr, ly), batch, T, offsets,
                         static_cast<const float*>(s0), static_cast<float*>(s_out)};
    e = launch_rollout<float>(a, st);
  } else {
    RolloutArgs<double> a{make_view<double>(f, x, nullptr, ly), batch, T, offsets,
                          static_cast<const double*>(s0), static_cast<double*>(s_out)};
    e = launch_rollout<double>(a, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "deer_rollout");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "deer_rollout sync");
  return DEER_OK;
}

size_t deer_grad_workspace_bytes(const deer_dynamics* f, int64_t batch, int64_t T,
                                 const deer_options* opt) {
  if (!opt || batch < 0 || T < 0 || opt->prec == DEER_MIXED_BF16) return 0;
  if (batch > 0 && T > kMaxRows / batch) return 0;
  deer_options o = *opt;
  o.jac = DEER_JAC_FULL;
  o.damp = DEER_DAMP_NONE;
  o.compensate = 0;
  if (check_common(f, &o) != DEER_OK) return 0;
  const int64_t W = grad_window_rows(f, batch, T, &o);
  if (W < T) {
    // the windowed adjoint (inputs and their gradient included where the kind has them)
    GradWinLayout gl;
    const bool has_x = needs_x(f->kind) || input_is_d(f->kind) || f->d_in > 0;
    if (!grad_win_layout(f, batch, W, &o, has_x, has_x, gl)) return 0;
    return gl.total;
  }
  Layout ly;
  if (!make_layout(f, batch, batch * T, &o, ly)) return 0;
  const size_t rs = o.prec == DEER_FP32 ? 4 : 8;
  return ly.total + align_up((size_t)batch * T * f->d * rs);
}

}  // extern "C"

namespace deer {
// Step Jacobians A_t = df_t/ds at s_{t-1} (Eq. lil_j) for every row of B sequences of T
// steps of the trajectory s, written row-major to ws + ly.A (shared by the adjoint and the
// Lyapunov-exponent entry points).
template <class real>
static deer_status jacobians_at(const deer_dynamics* f, int64_t B, int64_t T, const void* s0_,
                                const void* x_, const void* s_, const Layout& ly, char* ws,
                                cudaStream_t st, Batch& bt, DynView<real>& dv, Flags*& flags,
                                LinArgs<real>& la) {
  const int64_t N = B * T;
  const int d = f->d;
  std::vector<int64_t> off(B + 1), cf(B + 1);
  int64_t nc = 0;
  for (int64_t b = 0; b <= B; ++b) {
    off[b] = b * T;
    cf[b] = nc;
    if (b < B) nc += (T + ly.L - 1) / ly.L;
  }
  int64_t* d_off = reinterpret_cast<int64_t*>(ws + ly.offsets);
  int64_t* d_cf = reinterpret_cast<int64_t*>(ws + ly.chunk_first);
  DEER_CK(cudaMemcpyAsync(d_off, off.data(), (B + 1) * 8, cudaMemcpyHostToDevice, st));
  DEER_CK(cudaMemcpyAsync(d_cf, cf.data(), (B + 1) * 8, cudaMemcpyHostToDevice, st));
  SeqAcc* acc = reinterpret_cast<SeqAcc*>(ws + ly.acc);
  SeqInfo* info = reinterpret_cast<SeqInfo*>(ws + ly.info);
  flags = reinterpret_cast<Flags*>(ws + ly.flags);
  DEER_CK(cudaMemsetAsync(acc, 0, B * sizeof(SeqAcc), st));
  DEER_CK(cudaMemsetAsync(info, 0, B * sizeof(SeqInfo), st));
  DEER_CK(cudaMemsetAsync(flags, 0, sizeof(Flags), st));
  bt = Batch{B, N, d_off, d_cf, nc, ly.L, ilog2(ly.L),
             reinterpret_cast<int64_t*>(ws + ly.act_seq),
             reinterpret_cast<int64_t*>(ws + ly.act_row_off),
             reinterpret_cast<int64_t*>(ws + ly.act_chunk_off), B, N, nc};
  {
    CheckArgs ca{B, d_off, d_cf, acc, info, flags,
                 reinterpret_cast<int64_t*>(ws + ly.act_seq),
                 reinterpret_cast<int64_t*>(ws + ly.act_row_off),
                 reinterpret_cast<int64_t*>(ws + ly.act_chunk_off), 0.0, 0, 0, 1, 1};
    DEER_CK(launch_check(ca, st));
  }
  dv = make_view<real>(f, x_, ws, ly);
  if (ly.n_ma > 0) {
    DEER_CK(launch_ma_setup<real>(ly.n_ma, d, f->n_reactions, static_cast<const real*>(f->params),
                                  f->params_stride, f->topology, f->topology_stride,
                                  reinterpret_cast<real*>(ws + ly.ma), ly.ma_stride,
                                  &flags->bad_input, st));
  }
  if (f->kind == DEER_F_GRU) {
    DEER_CK(launch_gru_setup<real>(d, static_cast<const real*>(f->params), f->d_in,
                                   reinterpret_cast<real*>(ws + ly.gru_M), st));
  }
  la.dv = dv;
  la.bt = bt;
  la.s0 = static_cast<const real*>(s0_);
  la.s = static_cast<const real*>(s_);
  la.A = reinterpret_cast<real*>(ws + ly.A);
  la.b = reinterpret_cast<real*>(ws + ly.b);
  la.acc = acc;
  la.info = info;
  la.jac = DEER_JAC_FULL;
  la.damp = DEER_DAMP_NONE;
  la.dparam = real(0);
  DEER_CK(launch_linearize<real>(la, st));
  return DEER_OK;
}

// One adjoint solve over B sequences of T rows whose step Jacobians all fit the workspace:
// Jacobians at the trajectory, the reverse scan, the parameter VJP (accumulated into dp,
// which is zeroed first when zero_dp), dl/ds0 (the sensitivity to the state before the
// first row) and the input gradient.
template <class real>
static deer_status grad_core(const deer_dynamics* f, int64_t B, int64_t T, const void* s0_,
                             const void* x_, const void* sstar_, const void* g_, void* dp_,
                             void* ds0_, void* dx_, const Layout& ly, char* ws, size_t lam_off,
                             bool zero_dp, cudaStream_t st, Flags** flags_out) {
  const int d = f->d;
  const size_t rs = sizeof(real);
  Batch bt;
  DynView<real> dv;
  Flags* flags = nullptr;
  LinArgs<real> la;
  deer_status js = jacobians_at<real>(f, B, T, s0_, x_, sstar_, ly, ws, st, bt, dv, flags, la);
  if (js != DEER_OK) return js;
  *flags_out = flags;
  // reverse scan lambda_t = A_{t+1}^T lambda_{t+1} + g_t
  AdjScanArgs<real> sa;
  sa.bt = bt;
  sa.d = d;
  sa.A = la.A;
  sa.g = static_cast<const real*>(g_);
  sa.lam = reinterpret_cast<real*>(ws + lam_off);
  sa.aggP = reinterpret_cast<real*>(ws + ly.aggP);
  sa.aggv = reinterpret_cast<real*>(ws + ly.aggv);
  sa.cin = reinterpret_cast<real*>(ws + ly.cin);
  DEER_CK(launch_adjoint_scan<real>(sa, st));
  ParamGradArgs<real> pa;
  pa.dv = dv;
  pa.bt = bt;
  pa.s0 = la.s0;
  pa.s = la.s;
  pa.lam = sa.lam;
  pa.A = la.A;
  pa.dparams = static_cast<real*>(dp_);
  pa.pstride = f->kind == DEER_F_BRUSSELATOR_EULER ? 2 : f->n_reactions;
  pa.ds0 = static_cast<real*>(ds0_);
  if (pa.dparams && zero_dp) DEER_CK(cudaMemsetAsync(pa.dparams, 0, B * pa.pstride * rs, st));
  DEER_CK(launch_param_grad<real>(pa, st));
  if (dx_) {
    InputGradArgs<real> ia{dv, bt, la.s0, la.s, sa.lam, static_cast<real*>(dx_)};
    DEER_CK(launch_input_grad<real>(ia, st));
  }
  return DEER_OK;
}

// rows [t][d] of every sequence b: dst[b * dst_stride + (n - 1) * d + i] += add[b * d + i]
template <class real>
__global__ void k_add_last_rows(int64_t B, int d, const real* add, real* dst,
                                int64_t dst_stride) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= B * d) return;
  const int64_t b = e / d;
  dst[b * dst_stride + e % d] += add[e];
}

template <class real>
static deer_status grad_impl(const deer_dynamics* f, int64_t B, int64_t T, const void* s0_,
                             const void* x_, const void* sstar_, const void* g_, void* dp_,
                             void* ds0_, void* dx_, const deer_options* o, void* ws_,
                             size_t ws_bytes, cudaStream_t st) {
  const int64_t N = B * T;
  const size_t rs = sizeof(real);
  const int d = f->d;
  const int64_t W = grad_window_rows(f, B, T, o);
  Flags* flags = nullptr;
  if (W >= T) {
    Layout ly;
    if (!make_layout(f, B, N, o, ly)) return DEER_ERR_INVALID;
    const size_t lam_off = ly.total;
    const size_t need = ly.total + align_up((size_t)N * d * rs);
    if (!ws_ || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws_) & 255u))
      return DEER_ERR_WORKSPACE;
    deer_status c = grad_core<real>(f, B, T, s0_, x_, sstar_, g_, dp_, ds0_, dx_, ly,
                                    static_cast<char*>(ws_), lam_off, true, st, &flags);
    if (c != DEER_OK) return c;
  } else {
    // Memory-bounded adjoint: the reverse recursion of Eq. bptt runs over time windows of
    // W rows from the end of the sequences. Each window's Jacobians are formed when it is
    // reached (never all T of them at once); the adjoint entering a window from the later
    // one, A_{t_hi}^T lambda_{t_hi}, is the later window's sensitivity to the state before
    // its first row, and joins the cotangent of the window's last row.
    GradWinLayout gl;
    if (!grad_win_layout(f, B, W, o, x_ != nullptr, dx_ != nullptr, gl)) return DEER_ERR_INVALID;
    if (!ws_ || ws_bytes < gl.total || (reinterpret_cast<uintptr_t>(ws_) & 255u))
      return DEER_ERR_WORKSPACE;
    char* ws = static_cast<char*>(ws_);
    const int din = input_is_d(f->kind) ? f->d : f->d_in;
    const char* s_all = static_cast<const char*>(sstar_);
    const char* g_all = static_cast<const char*>(g_);
    const char* x_all = static_cast<const char*>(x_);
    char* carry_in = ws + gl.carry0;
    char* carry_out = ws + gl.carry1;
    bool first_window = true;
    for (int64_t t_hi = T; t_hi > 0; t_hi -= W) {
      const int64_t t_lo = t_hi > W ? t_hi - W : 0;
      const int64_t Wk = t_hi - t_lo;
      const size_t row_b = (size_t)d * rs, xrow_b = (size_t)din * rs;
      // gather the window's rows of every sequence (strided by the full length T)
      DEER_CK(cudaMemcpy2DAsync(ws + gl.s, Wk * row_b, s_all + t_lo * row_b, T * row_b,
                                Wk * row_b, B, cudaMemcpyDeviceToDevice, st));
      DEER_CK(cudaMemcpy2DAsync(ws + gl.g, Wk * row_b, g_all + t_lo * row_b, T * row_b,
                                Wk * row_b, B, cudaMemcpyDeviceToDevice, st));
      if (x_all)
        DEER_CK(cudaMemcpy2DAsync(ws + gl.x, Wk * xrow_b, x_all + t_lo * xrow_b, T * xrow_b,
                                  Wk * xrow_b, B, cudaMemcpyDeviceToDevice, st));
      // the state before the window: s_0, or row t_lo - 1 of the trajectory
      if (t_lo == 0)
        DEER_CK(cudaMemcpyAsync(ws + gl.s0, s0_, B * row_b, cudaMemcpyDeviceToDevice, st));
      else
        DEER_CK(cudaMemcpy2DAsync(ws + gl.s0, row_b, s_all + (t_lo - 1) * row_b, T * row_b,
                                  row_b, B, cudaMemcpyDeviceToDevice, st));
      if (!first_window) {
        k_add_last_rows<real><<<grid_for(B * d, 128), 128, 0, st>>>(
            B, d, reinterpret_cast<const real*>(carry_in),
            reinterpret_cast<real*>(ws + gl.g) + (Wk - 1) * d, Wk * d);
        note_launch();
        DEER_CK(cudaGetLastError());
      }
      deer_status c = grad_core<real>(f, B, Wk, ws + gl.s0, x_all ? ws + gl.x : nullptr,
                                      ws + gl.s, ws + gl.g, dp_, carry_out,
                                      dx_ ? ws + gl.dx : nullptr, gl.ly, ws, gl.lam,
                                      first_window, st, &flags);
      if (c != DEER_OK) return c;
      if (dx_)
        DEER_CK(cudaMemcpy2DAsync(static_cast<char*>(dx_) + t_lo * xrow_b, T * xrow_b,
                                  ws + gl.dx, Wk * xrow_b, Wk * xrow_b, B,
                                  cudaMemcpyDeviceToDevice, st));
      char* tmp = carry_in;
      carry_in = carry_out;
      carry_out = tmp;
      first_window = false;
    }
    // the earliest window's sensitivity to its initial state is dl/ds_0
    if (ds0_)
      DEER_CK(cudaMemcpyAsync(ds0_, carry_in, B * (size_t)d * rs, cudaMemcpyDeviceToDevice, st));
  }
  Flags hf;
  DEER_CK(cudaMemcpyAsync(&hf, flags, sizeof(Flags), cudaMemcpyDeviceToHost, st));
  DEER_CK(cudaStreamSynchronize(st));
  if (hf.bad_input) return DEER_ERR_INVALID;
  return DEER_OK;
}
template <class real>
static deer_status lle_impl(const deer_dynamics* f, int64_t B, int64_t T, const void* s0_,
                            const void* x_, const void* s_, const void* u0_, double* out,
                            const deer_options* o, void* ws_, size_t ws_bytes,
                            cudaStream_t st) {
  Layout ly;
  if (!make_layout(f, B, B * T, o, ly)) return DEER_ERR_INVALID;
  if (!ws_ || ws_bytes < ly.total || (reinterpret_cast<uintptr_t>(ws_) & 255u))
    return DEER_ERR_WORKSPACE;
  char* ws = static_cast<char*>(ws_);
  Batch bt;
  DynView<real> dv;
  Flags* flags = nullptr;
  LinArgs<real> la;
  deer_status js = jacobians_at<real>(f, B, T, s0_, x_, s_, ly, ws, st, bt, dv, flags, la);
  if (js != DEER_OK) return js;
  LleArgs<real> a{B, T, f->d, la.A, static_cast<const real*>(u0_), out};
  DEER_CK(launch_lle<real>(a, st));
  Flags hf;
  DEER_CK(cudaMemcpyAsync(&hf, flags, sizeof(Flags), cudaMemcpyDeviceToHost, st));
  DEER_CK(cudaStreamSynchronize(st));
  if (hf.bad_input) return DEER_ERR_INVALID;
  return DEER_OK;
}
}  // namespace deer

extern "C" {

size_t deer_lle_workspace_bytes(const deer_dynamics* f, int64_t batch, int64_t T,
                                int32_t prec) {
  if (batch < 0 || T < 0 || (prec != DEER_FP64 && prec != DEER_FP32) || !f || f->d > 32)
    return 0;
  deer_options o;
  deer_default_options(&o);
  o.prec = prec;
  if (check_common(f, &o) != DEER_OK) return 0;
  Layout ly;
  if (!make_layout(f, batch, batch * T, &o, ly)) return 0;
  return ly.total;
}

deer_status deer_lle(const deer_dynamics* f, int64_t batch, int64_t T, const void* s0,
                     const void* x, const void* s, const void* u0, double* lle_out,
                     int32_t prec, void* workspace, size_t workspace_bytes,
                     deer_stream_t stream) {
  if (!f || batch < 0 || T < 0) return DEER_ERR_INVALID;
  if (prec != DEER_FP64 && prec != DEER_FP32) return DEER_ERR_UNSUPPORTED;
  if (f->d > 32) return DEER_ERR_UNSUPPORTED;
  if (batch > 0 && T > kMaxRows / batch) return DEER_ERR_INVALID;
  deer_options o;
  deer_default_options(&o);
  o.prec = prec;
  deer_status c = check_common(f, &o);
  if (c != DEER_OK) return c;
  if (batch == 0 || T == 0) return DEER_OK;
  if (!s0 || !s || !u0 || !lle_out) return DEER_ERR_INVALID;
  if (needs_x(f->kind) && !x) return DEER_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (prec == DEER_FP32)
    return lle_impl<float>(f, batch, T, s0, x, s, u0, lle_out, &o, workspace, workspace_bytes,
                           st);
  return lle_impl<double>(f, batch, T, s0, x, s, u0, lle_out, &o, workspace, workspace_bytes,
                          st);
}

deer_status deer_grad(const deer_dynamics* f, int64_t batch, int64_t T, const void* s0,
                      const void* x, const void* s_star, const void* dl_ds, void* dl_dparams,
                      void* dl_ds0, const deer_options* opt, void* workspace,
                      size_t workspace_bytes, deer_stream_t stream) {
  return deer_grad_ex(f, batch, T, s0, x, s_star, dl_ds, dl_dparams, dl_ds0, nullptr, opt,
                      workspace, workspace_bytes, stream);
}

deer_status deer_grad_ex(const deer_dynamics* f, int64_t batch, int64_t T, const void* s0,
                         const void* x, const void* s_star, const void* dl_ds,
                         void* dl_dparams, void* dl_ds0, void* dl_dx,
                         const deer_options* opt, void* workspace, size_t workspace_bytes,
                         deer_stream_t stream) {
  if (!opt || !f) return DEER_ERR_INVALID;
  deer_options o = *opt;
  o.jac = DEER_JAC_FULL;
  o.damp = DEER_DAMP_NONE;
  o.compensate = 0;
  if (o.prec == DEER_MIXED_BF16) return DEER_ERR_UNSUPPORTED;
  deer_status c = check_common(f, &o);
  if (c != DEER_OK) return c;
  if (batch < 0 || T < 0) return DEER_ERR_INVALID;
  if (batch == 0 || T == 0) return DEER_OK;
  if (T > kMaxRows / batch) return DEER_ERR_INVALID;
  if (!s0 || !s_star || !dl_ds) return DEER_ERR_INVALID;
  if (needs_x(f->kind) && !x) return DEER_ERR_INVALID;
  const bool per_seq = f->kind == DEER_F_BRUSSELATOR_EULER ||
                       f->kind == DEER_F_MASSACTION_EULER || f->kind == DEER_F_MASSACTION_RK4;
  if (dl_dparams && !per_seq) return DEER_ERR_UNSUPPORTED;
  const bool has_inputs = f->kind == DEER_F_GRU || f->kind == DEER_F_LINEAR ||
                          f->kind == DEER_F_RNN_TANH || f->kind == DEER_F_LANGEVIN_2WELL;
  if (dl_dx && (!has_inputs || !x)) return DEER_ERR_UNSUPPORTED;
  if (dl_dparams && f->params_stride == 0 && batch > 1) return DEER_ERR_UNSUPPORTED;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (o.prec == DEER_FP32)
    return grad_impl<float>(f, batch, T, s0, x, s_star, dl_ds, dl_dparams, dl_ds0, dl_dx, &o,
                            workspace, workspace_bytes, st);
  return grad_impl<double>(f, batch, T, s0, x, s_star, dl_ds, dl_dparams, dl_ds0, dl_dx, &o,
                           workspace, workspace_bytes, st);
}

deer_status deer_selftest_wait_timeout(deer_stream_t stream) {
  // one sequence of two look-back tiles (d = 4, 1024 rows each) whose first tile is never
  // dealt: the CTA scanning tile 1 waits for tile 0's flag, which nothing sets, until its
  // spin limit, then reports through the status word and finishes
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  constexpr int D = 4;
  const int L = diag_lb_chunk(D);
  const int64_t N = 2 * (int64_t)L;
  struct Host {
    int64_t offsets[2], chunk_first[2], act_seq[1], act_row_off[2], act_chunk_off[2];
  } h{{0, N}, {0, 2}, {0}, {0, N}, {0, 2}};
  size_t p = 0;
  auto take = [&](size_t bytes) { size_t at = p; p = align_up(p + bytes); return at; };
  const size_t o_host = take(sizeof(Host)), o_b = take(N * D * 4),
               o_s = take(N * D * 4), o_s0 = take(D * 4), o_ticket = take(4),
               o_flags = take(2 * 4), o_agg = take(2 * 2 * D * 4), o_pre = take(2 * D * 4),
               o_status = take(sizeof(Flags));
  char* ws = nullptr;
  DEER_CK(cudaMalloc(&ws, p));
  deer_status ret = DEER_OK;
  do {
    if (cudaMemsetAsync(ws, 0, p, st) != cudaSuccess ||
        cudaMemcpyAsync(ws + o_host, &h, sizeof(Host), cudaMemcpyHostToDevice, st) !=
            cudaSuccess) {
      ret = DEER_ERR_CUDA;
      break;
    }
    const Host* dh = reinterpret_cast<const Host*>(ws + o_host);
    Batch bt{1, N, dh->offsets, dh->chunk_first, 2, L, ilog2(L), dh->act_seq, dh->act_row_off,
             dh->act_chunk_off, 1, N, 2};
    // constant transition 0.5 (a is not read), offsets b and s0 zero
    DiagLBArgs<float> la{bt, D, 1, 0.5f, nullptr, reinterpret_cast<const float*>(ws + o_b),
                         reinterpret_cast<const float*>(ws + o_s0),
                         reinterpret_cast<float*>(ws + o_s),
                         reinterpret_cast<unsigned*>(ws + o_ticket),
                         reinterpret_cast<unsigned*>(ws + o_flags),
                         reinterpret_cast<float*>(ws + o_agg),
                         reinterpret_cast<float*>(ws + o_pre), 1u, nullptr, 0,
                         reinterpret_cast<Flags*>(ws + o_status), 0, 0.f};
    if (launch_diag_lookback<float>(la, st, 1u) != cudaSuccess) {
      ret = DEER_ERR_CUDA;
      break;
    }
    Flags hf{};
    if (cudaMemcpyAsync(&hf, ws + o_status, sizeof(Flags), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      ret = DEER_ERR_CUDA;
      break;
    }
    ret = hf.timeout ? DEER_ERR_TIMEOUT : DEER_OK;
  } while (false);
  if (cudaStreamSynchronize(st) != cudaSuccess) ret = DEER_ERR_CUDA;
  if (cudaFree(ws) != cudaSuccess) ret = DEER_ERR_CUDA;
  return ret;
}

int64_t deer_kernel_launch_count(void) { return g_launches.load(); }

void deer_profile_enable(int32_t on) { g_prof_on.store(on ? 1 : 0); }
void deer_set_tensor_cores(int32_t on) { g_tensor_cores.store(on <= 0 ? 0 : (on >= 2 ? 2 : 1)); }
int32_t deer_get_tensor_cores(void) { return g_tensor_cores.load(); }

void deer_profile_reset(void) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  g_prof = deer_profile{};
}

void deer_profile_read(deer_profile* out) {
  if (!out) return;
  std::lock_guard<std::mutex> g(g_prof_mu);
  *out = g_prof;
}

const char* deer_status_string(int32_t s) {
  switch (s) {
    case DEER_OK: return "ok";
    case DEER_NOT_CONVERGED: return "not converged (iteration cap reached)";
    case DEER_ERR_INVALID: return "invalid argument";
    case DEER_ERR_CUDA: return "CUDA error";
    case DEER_ERR_NONFINITE: return "non-finite residual";
    case DEER_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case DEER_ERR_TIMEOUT: return "bounded device wait timed out";
    case DEER_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

const char* deer_last_cuda_error(void) { return g_err; }

int32_t deer_version(void) { return 1; }

}  // extern "C"

// ---------------------------------------------------------------------------
// No-allocation entry point (deer_solve_noalloc).
//
// Some callers cannot allocate device memory when they solve: code that runs while other
// work holds the allocator (a cudaMalloc synchronises the device), real-time loops whose
// latency budget forbids allocation, and embedders whose memory pool is fixed up front.
// For them the library carries one fixed scratch area per device in a file-scope
// __device__ array and solves small problems inside it. The array exists on every GPU
// that loads the library until the process exits; calls share it, so calls that overlap
// on the GPU (two streams, two host threads) race and must be serialised by the caller.
// Everything that must start at zero is cleared by each call.
// ---------------------------------------------------------------------------
namespace deer {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array on the current device. In host code the array's
// name is only a host-side stand-in, so every call asks the runtime for the address that
// belongs to the current device and context (cudaGetSymbolAddress allocates nothing).
// Looking it up per call rather than caching it keeps the address right when the
// caller's primary context was reset and recreated since an earlier call (the module is
// then loaded again and the array may sit elsewhere).
static cudaError_t noalloc_scratch(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  if (!p || (reinterpret_cast<uintptr_t>(p) & 255u)) return cudaErrorInvalidDevicePointer;
  *out = p;
  return cudaSuccess;
}

// offsets[b] = b T and chunk_first[b] = b ceil(T / L) for a batch of equal lengths
__global__ void k_uniform_tables(int64_t B, int64_t T, int64_t cps, int64_t* off,
                                 int64_t* cf) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b > B) return;
  off[b] = b * T;
  cf[b] = b * cps;
}

__global__ void k_info_out(int64_t B, const SeqInfo* in, deer_info* out) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= B) return;
  const SeqInfo s = in[b];
  out[b] = deer_info{s.iters, s.done, s.merit, s.max_resid};
}

template <class real>
static deer_status solve_noalloc_impl(const deer_dynamics* f, int64_t B, int64_t T,
                                      const void* s0_, const void* x_, void* s_,
                                      const deer_options* o, char* ws, cudaStream_t st,
                                      deer_info* info_h) {
  if (B > 0 && T > kMaxRows / B) return DEER_ERR_INVALID;
  const int64_t N = B * T;
  Layout ly;
  if (!make_layout(f, B, N, o, ly)) return DEER_ERR_INVALID;
  const size_t info_bytes = align_up((size_t)B * sizeof(deer_info));
  if (ly.total + info_bytes > kNoAllocScratchBytes) {
    snprintf(g_err, sizeof(g_err),
             "deer_solve_noalloc: problem needs %zu bytes of scratch, the fixed area holds %zu",
             ly.total + info_bytes, kNoAllocScratchBytes);
    return DEER_ERR_WORKSPACE;
  }
  const int d = f->d;
  const real* s0 = static_cast<const real*>(s0_);
  real* s = static_cast<real*>(s_);
  const int64_t cps = (T + ly.L - 1) / ly.L;
  const int64_t nc = B * cps;
  int64_t* d_off = reinterpret_cast<int64_t*>(ws + ly.offsets);
  int64_t* d_cf = reinterpret_cast<int64_t*>(ws + ly.chunk_first);
  k_uniform_tables<<<grid_for(B + 1, 128), 128, 0, st>>>(B, T, cps, d_off, d_cf);
  note_launch();
  DEER_CK(cudaGetLastError());
  SeqAcc* acc = reinterpret_cast<SeqAcc*>(ws + ly.acc);
  SeqInfo* info = reinterpret_cast<SeqInfo*>(ws + ly.info);
  Flags* flags = reinterpret_cast<Flags*>(ws + ly.flags);
  DEER_CK(cudaMemsetAsync(acc, 0, B * sizeof(SeqAcc), st));
  DEER_CK(cudaMemsetAsync(info, 0, B * sizeof(SeqInfo), st));
  DEER_CK(cudaMemsetAsync(flags, 0, sizeof(Flags), st));

  Batch bt{B, N, d_off, d_cf, nc, ly.L, ilog2(ly.L),
           reinterpret_cast<int64_t*>(ws + ly.act_seq),
           reinterpret_cast<int64_t*>(ws + ly.act_row_off),
           reinterpret_cast<int64_t*>(ws + ly.act_chunk_off), B, N, nc};
  DynView<real> dv = make_view<real>(f, x_, ws, ly);
  if (ly.n_ma > 0) {
    DEER_CK(launch_ma_setup<real>(ly.n_ma, d, f->n_reactions, static_cast<const real*>(f->params),
                                  f->params_stride, f->topology, f->topology_stride,
                                  reinterpret_cast<real*>(ws + ly.ma), ly.ma_stride,
                                  &flags->bad_input, st));
  }
  if (f->kind == DEER_F_GRU) {
    DEER_CK(launch_gru_setup<real>(d, static_cast<const real*>(f->params), f->d_in,
                                   reinterpret_cast<real*>(ws + ly.gru_M), st));
  }
  if (o->init != DEER_INIT_USER) {
    InitArgs<real> ia{};
    ia.dv = dv;
    ia.bt = bt;
    ia.s0 = s0;
    ia.s = s;
    ia.init = o->init;
    ia.seed = o->seed;
    DEER_CK(launch_init<real>(ia, st));
  }
  const int max_iters = o->max_iters > 0 ? o->max_iters : (int)(T > 0 ? T : 1);
  const real reset_thr = sizeof(real) == 8 ? real(1e30) : real(1e18);
  // the convergence test in the kernels' precision (see solve_impl)
  real tol_r = (real)o->tol;
  if ((double)tol_r > o->tol) tol_r = std::nextafter(tol_r, real(0));

  // every argument block is filled field by field, as in solve_impl
  LinArgs<real> la{};
  la.dv = dv;
  la.bt = bt;
  la.s0 = s0;
  la.s = s;
  la.A = reinterpret_cast<real*>(ws + ly.A);
  la.b = reinterpret_cast<real*>(ws + ly.b);
  la.acc = acc;
  la.info = info;
  la.jac = o->jac;
  la.damp = o->damp;
  la.dparam = (real)o->damp_param;
  la.tol = tol_r;

  CheckArgs ca{};
  ca.B = B;
  ca.offsets = d_off;
  ca.chunk_first = d_cf;
  ca.acc = acc;
  ca.info = info;
  ca.flags = flags;
  ca.act_seq = reinterpret_cast<int64_t*>(ws + ly.act_seq);
  ca.act_row_off = reinterpret_cast<int64_t*>(ws + ly.act_row_off);
  ca.act_chunk_off = reinterpret_cast<int64_t*>(ws + ly.act_chunk_off);
  ca.tol = o->tol;
  ca.it = 0;
  ca.max_iters = max_iters;
  ca.compact_only = 1;
  ca.confirm = o->confirm > 1 ? o->confirm : 1;
  ca.log2L = bt.log2L;
  DEER_CK(launch_check(ca, st));  // every sequence starts active
  ca.compact_only = 0;
  ca.history = o->history;
  ca.history_len = o->history_len;

  DenseScanArgs<real> dsa{};
  dsa.bt = bt;
  dsa.d = d;
  dsa.A = la.A;
  dsa.b = la.b;
  dsa.s = s;
  dsa.aggP = reinterpret_cast<real*>(ws + ly.aggP);
  dsa.aggv = reinterpret_cast<real*>(ws + ly.aggv);
  dsa.cin = reinterpret_cast<real*>(ws + ly.cin);
  dsa.info = info;
  dsa.reset = o->reset;
  dsa.reset_thr = reset_thr;

  real ac = o->jac == DEER_JAC_IDENTITY ? real(1) : real(0);
  if (o->damp == DEER_DAMP_SCALE) ac *= real(1) - (real)o->damp_param;
  if (o->damp == DEER_DAMP_CLIP) {
    const real rho = (real)o->damp_param;
    ac = ac > rho ? rho : (ac < -rho ? -rho : ac);
  }
  const int elk = (o->damp == DEER_DAMP_ELK && o->damp_param > 0.0) ? 1 : 0;
  DiagScanArgs<real> gsa{};
  gsa.bt = bt;
  gsa.d = d;
  gsa.amode = o->jac == DEER_JAC_DIAG ? 0 : 1;
  gsa.aconst = ac;
  gsa.a = la.A;
  gsa.b = la.b;
  gsa.s0 = s0;
  gsa.s = s;
  gsa.aggA = reinterpret_cast<real*>(ws + ly.aggP);
  gsa.aggB = reinterpret_cast<real*>(ws + ly.aggv);
  gsa.cin = reinterpret_cast<real*>(ws + ly.cin);
  gsa.info = info;
  gsa.elk = elk;
  gsa.sigma2 = elk ? real(1.0 / o->damp_param) : real(0);
  gsa.mob = reinterpret_cast<real*>(ws + ly.mob);
  gsa.pin = reinterpret_cast<real*>(ws + ly.pin);
  gsa.reset = o->reset;
  gsa.reset_thr = reset_thr;

  const bool lookback = use_diag_lookback(o, d);
  DiagLBArgs<real> lba{};
  lba.bt = bt;
  lba.d = d;
  lba.amode = gsa.amode;
  lba.aconst = gsa.aconst;
  lba.a = la.A;
  lba.b = la.b;
  lba.s0 = s0;
  lba.s = s;
  lba.ticket = reinterpret_cast<unsigned*>(ws + ly.lb_ticket);
  lba.flags = reinterpret_cast<unsigned*>(ws + ly.lb_flags);
  lba.agg = reinterpret_cast<real*>(ws + ly.lb_agg);
  lba.pre = reinterpret_cast<real*>(ws + ly.lb_pre);
  lba.epoch = 0u;
  lba.cps = 0;
  lba.status = flags;
  lba.reset = o->reset;
  lba.reset_thr = reset_thr;
  // the look-back flags carry the epoch of their launch; the scratch keeps the last call's
  // flags, so they are cleared before this call's first launch
  if (lookback) DEER_CK(cudaMemsetAsync(lba.flags, 0, (size_t)ly.n_chunks_max * 4, st));

  deer_status status = DEER_OK;
  Flags hf;
  for (int it = 0;; ++it) {
    la.bt = bt;
    DEER_CK(launch_linearize<real>(la, st));
    ca.it = it;
    DEER_CK(launch_check(ca, st));
    DEER_CK(cudaMemcpyAsync(&hf, flags, sizeof(Flags), cudaMemcpyDeviceToHost, st));
    DEER_CK(cudaStreamSynchronize(st));
    bool stop = false;
    if (hf.bad_input) { status = DEER_ERR_INVALID; stop = true; }
    else if (hf.timeout) { status = DEER_ERR_TIMEOUT; stop = true; }
    else if (hf.n_nonfinite > 0 && !o->reset) { status = DEER_ERR_NONFINITE; stop = true; }
    else if (hf.n_active == 0) stop = true;
    else if (it >= max_iters) { status = DEER_NOT_CONVERGED; stop = true; }
    bt.set_counts(hf.n_active, hf.active_rows, hf.active_chunks);
    if (stop) break;
    if (o->jac == DEER_JAC_FULL) {
      dsa.bt = bt;
      DEER_CK(launch_dense_scan<real>(dsa, st));
    } else if (lookback) {
      lba.bt = bt;
      lba.epoch += 1;
      DEER_CK(launch_diag_lookback<real>(lba, st));
    } else {
      gsa.bt = bt;
      DEER_CK(launch_diag_scan<real>(gsa, st));
    }
  }
  if (info_h) {
    deer_info* dinfo = reinterpret_cast<deer_info*>(ws + ly.total);
    k_info_out<<<grid_for(B, 128), 128, 0, st>>>(B, info, dinfo);
    note_launch();
    DEER_CK(cudaGetLastError());
    DEER_CK(cudaMemcpyAsync(info_h, dinfo, B * sizeof(deer_info), cudaMemcpyDeviceToHost, st));
  }
  DEER_CK(cudaStreamSynchronize(st));
  return status;
}

}  // namespace deer

extern "C" {

deer_status deer_solve_noalloc(const deer_dynamics* f, int64_t batch, int64_t T,
                               const void* s0, const void* x, void* s_out,
                               const deer_options* opt, deer_stream_t stream,
                               deer_info* info) {
  deer_status c = check_common(f, opt);
  if (c != DEER_OK) return c;
  if (opt->prec == DEER_MIXED_BF16) return DEER_ERR_UNSUPPORTED;
  if (opt->damp == DEER_DAMP_ELK && opt->jac == DEER_JAC_FULL) return DEER_ERR_UNSUPPORTED;
  if (opt->window) return DEER_ERR_UNSUPPORTED;
  // the fixed scratch solves with a plain float32 state (no compensation terms)
  deer_options plain = *opt;
  plain.compensate = 0;
  opt = &plain;
  if (batch < 0 || T < 0) return DEER_ERR_INVALID;
  if (batch == 0 || T == 0) return DEER_OK;
  if (T > kMaxRows / batch) return DEER_ERR_INVALID;
  if (!s0 || !s_out) return DEER_ERR_INVALID;
  if (needs_x(f->kind) && !x) return DEER_ERR_INVALID;
  void* scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess) return cuda_fail(e, "deer_solve_noalloc scratch lookup");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(scratch);
  if (opt->prec == DEER_FP32)
    return solve_noalloc_impl<float>(f, batch, T, s0, x, s_out, opt, ws, st, info);
  return solve_noalloc_impl<double>(f, batch, T, s0, x, s_out, opt, ws, st, info);
}

size_t deer_noalloc_scratch_bytes(void) { return kNoAllocScratchBytes; }

}  // extern "C"
