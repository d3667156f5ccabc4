// Single-pass diagonal scan with decoupled look-back (quasi-DEER / Picard / Jacobi LDS,
// Eq. quasi_lds in standard form): s_t = a_t * s_{t-1} + b_t, coordinate-wise, s_0 given.
//
// One CTA per tile = one chunk of L rows of one sequence, all d coordinates. Each thread
// owns RPT consecutive rows of 4 coordinates (16-byte vector accesses). The tile scans its
// rows in registers and shared memory (Kogge-Stone over the row sub-ranges), publishes its
// aggregate, resolves the state entering the tile by looking back over the published
// aggregates / prefixes of the preceding tiles of the same sequence, and writes s. a, b are
// read from DRAM once (the second read hits L2) and s written once: 12 bytes of DRAM
// traffic per coordinate-step in float32.
#include "kernels.h"

namespace deer {

template <class real>
struct V4 { real x, y, z, w; };

// L2 eviction-priority policies: a and b are read twice (for the tile aggregate, then after
// the look-back for the output); the first read marks them evict-last so that the second
// read finds them in L2, and the second read and the stores of s mark their lines
// evict-first so that streaming data does not push the pending tiles out.
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

template <class real>
__device__ __forceinline__ V4<real> ld4_hint(const real* p, uint64_t pol) {
  if constexpr (sizeof(real) == 4) {
    float4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p), "l"(pol));
    return {v.x, v.y, v.z, v.w};
  } else {
    double2 u, v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;"
                 : "=d"(u.x), "=d"(u.y)
                 : "l"(p), "l"(pol));
    asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;"
                 : "=d"(v.x), "=d"(v.y)
                 : "l"(p + 2), "l"(pol));
    return {u.x, u.y, v.x, v.y};
  }
}

template <class real>
__device__ __forceinline__ void st4_hint(real* p, const real (&v)[4], uint64_t pol) {
  if constexpr (sizeof(real) == 4) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1,%2,%3,%4}, %5;" ::"l"(p),
                 "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "l"(pol)
                 : "memory");
  } else {
    asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1,%2}, %3;" ::"l"(p), "d"(v[0]),
                 "d"(v[1]), "l"(pol)
                 : "memory");
    asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1,%2}, %3;" ::"l"(p + 2),
                 "d"(v[2]), "d"(v[3]), "l"(pol)
                 : "memory");
  }
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int D>
struct LBShape {
  static constexpr int G = D / 4;                       // 4-coordinate groups
  static constexpr int Q = 256 / G;                     // row sub-ranges per tile
  static constexpr int L = D >= 8 ? 8192 / D : 1024;    // rows per tile
  static constexpr int RPT = L / Q;                     // rows per thread
};

constexpr unsigned kSpinLimit = 1u << 22;  // bounded wait (about 0.3 s with backoff)

// Tile-level part shared by both variants: the inclusive scan over the row sub-ranges of
// the tile (per coordinate, Kogge-Stone through shared memory), publication of the tile's
// aggregate, and the look-back that resolves the state entering the tile into s_in. On
// return sA[q] / sB[q] hold the composition of sub-ranges 0..q and s_in the incoming state.
template <class real, int D>
__device__ __forceinline__ void block_scan_and_lookback(const DiagLBArgs<real>& a,
                                                        int64_t seq, int64_t c, real (&A)[4],
                                                        real (&Bv)[4], int q, int k0,
                                                        real (*sA)[D], real (*sB)[D],
                                                        real* s_in) {
  constexpr int Q = LBShape<D>::Q;
#pragma unroll
  for (int k = 0; k < 4; ++k) { sA[q][k0 + k] = A[k]; sB[q][k0 + k] = Bv[k]; }
  __syncthreads();
  // inclusive Kogge-Stone scan over the sub-ranges, per coordinate
#pragma unroll
  for (int off = 1; off < Q; off <<= 1) {
    real pa[4], pb[4];
    const bool has = q >= off;
    if (has) {
#pragma unroll
      for (int k = 0; k < 4; ++k) { pa[k] = sA[q - off][k0 + k]; pb[k] = sB[q - off][k0 + k]; }
    }
    __syncthreads();
    if (has) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        Bv[k] = A[k] * pb[k] + Bv[k];
        A[k] = A[k] * pa[k];
        sA[q][k0 + k] = A[k];
        sB[q][k0 + k] = Bv[k];
      }
    }
    __syncthreads();
  }

  // publish the tile aggregate and resolve the incoming state (first warp)
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    // the first solved tile starts from s_0 or, under a sliding window, from the frozen
    // state of the row before it
    const int64_t cf = __ldg(a.bt.chunk_first + seq);
    const bool first = c == win_first(a.bt, seq);
    const unsigned ep = a.epoch << 2;
    real* agg = a.agg + c * (int64_t)(2 * D);
    real* pre = a.pre + c * (int64_t)D;
    if (first) {
      const real* sp = c == cf ? a.s0 + seq * D
                               : a.s + (__ldg(a.bt.offsets + seq) + ((c - cf) << a.bt.log2L) - 1) * D;
      for (int k = lane; k < D; k += 32) {
        const real sin = sp[k];
        s_in[k] = sin;
        __stcg(pre + k, sA[Q - 1][k] * sin + sB[Q - 1][k]);
      }
      __threadfence();
      __syncwarp();
      if (lane == 0) st_release(a.flags + c, ep | 2u);
    } else {
      for (int k = lane; k < D; k += 32) {
        __stcg(agg + 2 * k, sA[Q - 1][k]);
        __stcg(agg + 2 * k + 1, sB[Q - 1][k]);
      }
      __threadfence();
      __syncwarp();
      if (lane == 0) st_release(a.flags + c, ep | 1u);
      // look back over the predecessors of this sequence, 32 tiles per round: lane j
      // reads the status of tile base - j; the run of published tiles nearest to this
      // one is folded in (their aggregates are fetched together, so a round costs about
      // two memory latencies however many tiles it folds), and the walk ends at the
      // nearest tile whose inclusive prefix is published.
      constexpr int NJ = (D + 31) / 32;
      real XA[NJ], XB[NJ];
#pragma unroll
      for (int j = 0; j < NJ; ++j) { XA[j] = real(1); XB[j] = real(0); }
      const int64_t cfirst = win_first(a.bt, seq);
      int64_t base = c - 1;
      unsigned spins = 0;
      bool timed_out = false;
      while (true) {
        const int64_t p = base - lane;
        unsigned f = p >= cfirst ? ld_acquire(a.flags + p) : 0u;
        const bool ok = (f >> 2) == a.epoch && (f & 3u) != 0u;
        const unsigned ready = __ballot_sync(0xffffffffu, ok);
        const unsigned haspre = __ballot_sync(0xffffffffu, ok && (f & 3u) == 2u);
        const int run = ready == 0xffffffffu ? 32 : __ffs(~ready) - 1;  // ready from lane 0
        const int kp = haspre ? __ffs(haspre) - 1 : 32;                   // nearest prefix
        const int nfold = kp < run ? kp : run;  // aggregates to fold in this pass of the look-back
        if (nfold == 0 && kp != 0) {
          if (++spins > kSpinLimit) { timed_out = true; break; }
          __nanosleep(64);
          continue;
        }
        // the statuses above were read by other lanes: order this lane's reads after them
        __threadfence();
        // fold the aggregates of tiles base .. base - nfold + 1 (nearest first), four
        // tiles' loads in flight at a time
        for (int j0 = 0; j0 < nfold; j0 += 4) {
          real Ap[4][NJ], Bp[4][NJ];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const real* ap = a.agg + (base - j0 - u) * (int64_t)(2 * D);
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
              const int k = lane + 32 * j;
              if (j0 + u < nfold && k < D) {
                Ap[u][j] = __ldcg(ap + 2 * k);
                Bp[u][j] = __ldcg(ap + 2 * k + 1);
              } else {
                Ap[u][j] = real(1);
                Bp[u][j] = real(0);
              }
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
              XB[j] = XA[j] * Bp[u][j] + XB[j];
              XA[j] = XA[j] * Ap[u][j];
            }
        }
        if (kp <= run && kp < 32) {
          // the tile at base - kp has its inclusive prefix: the state entering this tile
          const real* pp = a.pre + (base - kp) * (int64_t)D;
#pragma unroll
          for (int j = 0; j < NJ; ++j) {
            const int k = lane + 32 * j;
            if (k < D) s_in[k] = XA[j] * __ldcg(pp + k) + XB[j];
          }
          break;
        }
        base -= nfold;
        spins = 0;
      }
      if (timed_out) {
        if (lane == 0) atomicExch(&a.status->timeout, 1);
        for (int k = lane; k < D; k += 32) s_in[k] = real(0);
      }
      for (int k = lane; k < D; k += 32) __stcg(pre + k, sA[Q - 1][k] * s_in[k] + sB[Q - 1][k]);
      __threadfence();
      __syncwarp();
      if (lane == 0) st_release(a.flags + c, ep | 2u);
    }
  }
  __syncthreads();
}

template <class real, int D>
__global__ void __launch_bounds__(256, sizeof(real) == 4 ? 8 : 4) k_diag_lb(DiagLBArgs<real> a) {
  using S = LBShape<D>;
  constexpr int Q = S::Q, G = S::G, RPT = S::RPT;
  __shared__ real sA[Q][D];
  __shared__ real sB[Q][D];
  __shared__ real s_in[D];
  __shared__ unsigned s_tile;
  if (a.epoch_from) a.epoch = (unsigned)a.epoch_from->iter;
  if (threadIdx.x == 0) s_tile = atomicAdd(a.ticket, 1u);
  __syncthreads();
  const int64_t tk = s_tile;
  if (tk >= a.bt.act_chunks()) return;  // uniform over the CTA
  // ticket -> active chunk index: sequence-major, or round-robin over the sequences when
  // they all have cps chunks (a predecessor tile always holds a smaller ticket either way)
  const int64_t ac = a.cps > 0 ? (tk % a.bt.n_act()) * a.cps + tk / a.bt.n_act() : tk;
  int64_t seq, c, r0;
  int n;
  act_chunk(a.bt, ac, seq, c, r0, n);
  const int g = threadIdx.x % G, q = threadIdx.x / G;
  const int k0 = 4 * g;

  // this thread's rows (identity elements past the end of a ragged tile); the values are
  // read twice: here for the aggregate, and after the look-back (from L2) for the output,
  // which keeps few registers live and many CTAs resident
  const uint64_t keep = l2_policy_evict_last(), stream = l2_policy_evict_first();
  auto load_row = [&](int i, real (&av)[4], real (&bv)[4], uint64_t pol) {
    const int lr = q * RPT + i;
    if (lr < n) {
      const int64_t off = (r0 + lr) * D + k0;
      const V4<real> bb = ld4_hint(a.b + off, pol);
      bv[0] = bb.x; bv[1] = bb.y; bv[2] = bb.z; bv[3] = bb.w;
      if (a.amode == 0) {
        const V4<real> aa = ld4_hint(a.a + off, pol);
        av[0] = aa.x; av[1] = aa.y; av[2] = aa.z; av[3] = aa.w;
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) av[k] = a.aconst;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) { av[k] = real(1); bv[k] = real(0); }
    }
  };
  // thread aggregate (composition in row order)
  real A[4], Bv[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) { A[k] = real(1); Bv[k] = real(0); }
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    real av[4], bv[4];
    load_row(i, av, bv, keep);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      Bv[k] = av[k] * Bv[k] + bv[k];
      A[k] = av[k] * A[k];
    }
  }
  block_scan_and_lookback<real, D>(a, seq, c, A, Bv, q, k0, sA, sB, s_in);

  // state entering this thread's rows = exclusive prefix applied to the tile's input
  real x[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const real sin = s_in[k0 + k];
    x[k] = q > 0 ? sA[q - 1][k0 + k] * sin + sB[q - 1][k0 + k] : sin;
  }
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int lr = q * RPT + i;
    if (lr < n) {
      real av[4], bv[4], o[4];
      load_row(i, av, bv, stream);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        x[k] = av[k] * x[k] + bv[k];
        o[k] = (a.reset && !(x[k] <= a.reset_thr && x[k] >= -a.reset_thr)) ? real(0) : x[k];
      }
      st4_hint(a.s + (r0 + lr) * D + k0, o, stream);
    }
  }
}

template <class real>
cudaError_t launch_diag_lookback(const DiagLBArgs<real>& a, cudaStream_t st,
                                 unsigned first_ticket) {
  if (a.bt.act_chunks() == 0) return cudaSuccess;
  // tiles are dealt from first_ticket on (0 in every solve; the wait self-test starts at 1,
  // so that no CTA ever publishes tile 0)
  static const unsigned kOne = 1u;
  cudaError_t e = first_ticket == 0
                      ? cudaMemsetAsync(a.ticket, 0, sizeof(unsigned), st)
                      : (first_ticket == 1 ? cudaMemcpyAsync(a.ticket, &kOne, sizeof(unsigned),
                                                             cudaMemcpyHostToDevice, st)
                                           : cudaErrorInvalidValue);
  if (e != cudaSuccess) return e;
  if ((int64_t)first_ticket >= a.bt.act_chunks()) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)(a.bt.act_chunks() - first_ticket);
  switch (a.d) {
    case 4: k_diag_lb<real, 4><<<grid, 256, 0, st>>>(a); break;
    case 8: k_diag_lb<real, 8><<<grid, 256, 0, st>>>(a); break;
    case 16: k_diag_lb<real, 16><<<grid, 256, 0, st>>>(a); break;
    case 32: k_diag_lb<real, 32><<<grid, 256, 0, st>>>(a); break;
    case 64: k_diag_lb<real, 64><<<grid, 256, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  note_launch();
  return cudaGetLastError();
}

template cudaError_t launch_diag_lookback<float>(const DiagLBArgs<float>&, cudaStream_t,
                                                 unsigned);
template cudaError_t launch_diag_lookback<double>(const DiagLBArgs<double>&, cudaStream_t,
                                                  unsigned);

}  // namespace deer
