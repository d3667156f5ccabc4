// GRU (d = d_in = 64, float32) linearisation as shared-memory-tiled SIMT matrix products.
// For every row t (time step) with h = s_{t-1}:
//   z = sig(Wz x + Uz h), r = sig(Wr x + Ur h), h~ = tanh(Wh x + Uh (r*h)),
//   F = (1 - z) h + z h~,
//   A_ii = (1 - z_i) + (h~_i - h_i) z_i (1 - z_i) Uz_ii
//          + z_i (1 - h~_i^2) (Uh_ii r_i + sum_j M_ij h_j r_j (1 - r_j)),  M_ij = Uh_ij Ur_ji,
// i.e. four 64x64 products per row (Uz h, Ur h, Uh (r*h), M (h*r*(1-r))), done for 64 rows
// at a time. Thread t of 256 owns rows 4(t%16)..+3 and outputs 4(t/16)..+3, so that the
// transposed tiles it writes for the second product are contiguous across a half-warp.
#include "kernels.h"

namespace deer {

constexpr int kGD = 64;       // state size
constexpr int kGT = 64;       // rows per tile
constexpr int kGThreads = 256;

struct GruSmem {
  float UT[4][kGD][kGD];      // Uz^T, Ur^T, Uh^T, M^T as [k][out]  (64 KB)
  float HT[kGD][kGT];         // h transposed [k][row]; reused for r*h after the first product
  float CT[kGD][kGT];         // h*r*(1-r) transposed
  float diag_z[kGD], diag_h[kGD];
  float rmx[kGT];
  float rsq[kGT];
  long long rseq[kGT];
  int rvalid[kGT];
};

__device__ __forceinline__ float fsig(float v) { return 1.f / (1.f + __expf(-v)); }

__device__ __forceinline__ float4 lds4(const float* p) {
  return *reinterpret_cast<const float4*>(p);
}

__global__ void __launch_bounds__(kGThreads) k_gru_lin_tiled(GruTileArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GruSmem& S = *reinterpret_cast<GruSmem*>(smem_raw);
  const int tid = threadIdx.x;
  const int ty = tid & 15, tx = tid >> 4;  // ty: row group, tx: output group
  const float* Uz = a.dv.params + 3 * kGD * a.dv.d_in;
  const float* Ur = Uz + kGD * kGD;
  const float* Uh = Ur + kGD * kGD;
  // stage the transposed recurrent matrices once per CTA
  for (int e = tid; e < kGD * kGD; e += kGThreads) {
    const int i = e / kGD, k = e % kGD;  // U[i][k] -> UT[k][i]
    const float uz = Uz[e], ur = Ur[e], uh = Uh[e];
    S.UT[0][k][i] = uz;
    S.UT[1][k][i] = ur;
    S.UT[2][k][i] = uh;
    S.UT[3][k][i] = a.dv.gru_M[e];
  }
  if (tid < kGD) {
    S.diag_z[tid] = Uz[tid * kGD + tid];
    S.diag_h[tid] = Uh[tid * kGD + tid];
  }
  __syncthreads();
  const int64_t n_tiles = (a.bt.act_rows() + kGT - 1) / kGT;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    // load h (previous states) of the tile's 64 rows, transposed
    if (tid < kGT) {
      const int64_t ar = tile * kGT + tid;
      const bool v = ar < a.bt.act_rows();
      int64_t seq = 0, row = 0;
      if (v) act_row(a.bt, ar, seq, row);
      S.rseq[tid] = seq;
      S.rvalid[tid] = v;
      S.rmx[tid] = 0.f;
      S.rsq[tid] = 0.f;
    }
    __syncthreads();
    for (int e = tid; e < kGT * (kGD / 4); e += kGThreads) {
      const int rl = e % kGT, q = e / kGT;
      const int64_t ar = tile * kGT + rl;
      float4 hv = make_float4(0.f, 0.f, 0.f, 0.f);
      if (S.rvalid[rl]) {
        int64_t seq, row;
        act_row(a.bt, ar, seq, row);
        const float* hp = row == __ldg(a.bt.offsets + seq) ? a.s0 + seq * kGD : a.s + (row - 1) * kGD;
        hv = *reinterpret_cast<const float4*>(hp + 4 * q);
      }
      S.HT[4 * q + 0][rl] = hv.x;
      S.HT[4 * q + 1][rl] = hv.y;
      S.HT[4 * q + 2][rl] = hv.z;
      S.HT[4 * q + 3][rl] = hv.w;
    }
    __syncthreads();
    // phase 1: z and r pre-activations for rows 4ty.., outputs 4tx..
    int64_t rows[4];
    bool rv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int rl = 4 * ty + i;
      rv[i] = S.rvalid[rl];
      rows[i] = 0;
      if (rv[i]) {
        int64_t seq;
        act_row(a.bt, tile * kGT + rl, seq, rows[i]);
      }
    }
    float az[4][4], ar_[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float4 pz = make_float4(0.f, 0.f, 0.f, 0.f), pr = pz;
      if (rv[i]) {
        const float* xp = a.xproj + rows[i] * (3 * kGD);
        pz = *reinterpret_cast<const float4*>(xp + 4 * tx);
        pr = *reinterpret_cast<const float4*>(xp + kGD + 4 * tx);
      }
      az[i][0] = pz.x; az[i][1] = pz.y; az[i][2] = pz.z; az[i][3] = pz.w;
      ar_[i][0] = pr.x; ar_[i][1] = pr.y; ar_[i][2] = pr.z; ar_[i][3] = pr.w;
    }
#pragma unroll 8
    for (int k = 0; k < kGD; ++k) {
      const float4 h4 = lds4(&S.HT[k][4 * ty]);
      const float4 uz = lds4(&S.UT[0][k][4 * tx]);
      const float4 ur = lds4(&S.UT[1][k][4 * tx]);
      const float hh[4] = {h4.x, h4.y, h4.z, h4.w};
      const float zz[4] = {uz.x, uz.y, uz.z, uz.w};
      const float rr[4] = {ur.x, ur.y, ur.z, ur.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          az[i][j] += hh[i] * zz[j];
          ar_[i][j] += hh[i] * rr[j];
        }
    }
    float z[4][4], r[4][4], hreg[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float4 h4 = lds4(&S.HT[4 * tx + j][4 * ty]);
      hreg[0][j] = h4.x; hreg[1][j] = h4.y; hreg[2][j] = h4.z; hreg[3][j] = h4.w;
    }
    __syncthreads();  // every thread is done reading h: its space now takes r*h
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float q[4], cc[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        z[i][j] = fsig(az[i][j]);
        r[i][j] = fsig(ar_[i][j]);
        q[i] = r[i][j] * hreg[i][j];
        cc[i] = hreg[i][j] * r[i][j] * (1.f - r[i][j]);
      }
      *reinterpret_cast<float4*>(&S.HT[4 * tx + j][4 * ty]) = make_float4(q[0], q[1], q[2], q[3]);
      *reinterpret_cast<float4*>(&S.CT[4 * tx + j][4 * ty]) = make_float4(cc[0], cc[1], cc[2], cc[3]);
    }
    __syncthreads();
    // phase 2: candidate pre-activation and the off-diagonal Jacobian term
    float ah[4][4], am[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float4 ph = make_float4(0.f, 0.f, 0.f, 0.f);
      if (rv[i]) ph = *reinterpret_cast<const float4*>(a.xproj + rows[i] * (3 * kGD) + 2 * kGD + 4 * tx);
      ah[i][0] = ph.x; ah[i][1] = ph.y; ah[i][2] = ph.z; ah[i][3] = ph.w;
#pragma unroll
      for (int j = 0; j < 4; ++j) am[i][j] = 0.f;
    }
#pragma unroll 8
    for (int k = 0; k < kGD; ++k) {
      const float4 q4 = lds4(&S.HT[k][4 * ty]);
      const float4 c4 = lds4(&S.CT[k][4 * ty]);
      const float4 uh = lds4(&S.UT[2][k][4 * tx]);
      const float4 mm = lds4(&S.UT[3][k][4 * tx]);
      const float qq[4] = {q4.x, q4.y, q4.z, q4.w};
      const float cc[4] = {c4.x, c4.y, c4.z, c4.w};
      const float hh[4] = {uh.x, uh.y, uh.z, uh.w};
      const float mv[4] = {mm.x, mm.y, mm.z, mm.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          ah[i][j] += qq[i] * hh[j];
          am[i][j] += cc[i] * mv[j];
        }
    }
    // elementwise: F, diag A, residual, outputs
    const float kk = a.dparam;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int rl = 4 * ty + i;
      float bo[4], ao[4];
      float mx = 0.f;
      float sq = 0.f;
      float4 sc4 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (rv[i]) sc4 = *reinterpret_cast<const float4*>(a.s + rows[i] * kGD + 4 * tx);
      const float sc[4] = {sc4.x, sc4.y, sc4.z, sc4.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int o = 4 * tx + j;
        const float h = hreg[i][j];
        const float ht = tanhf(ah[i][j]);
        const float zi = z[i][j], ri = r[i][j];
        const float F = (1.f - zi) * h + zi * ht;
        float ai;
        if (a.jac == DEER_JAC_DIAG) {
          ai = (1.f - zi) + (ht - h) * zi * (1.f - zi) * S.diag_z[o] +
               zi * (1.f - ht * ht) * (S.diag_h[o] * ri + am[i][j]);
        } else {
          ai = a.jac == DEER_JAC_IDENTITY ? 1.f : 0.f;
        }
        if (a.damp == DEER_DAMP_SCALE) ai *= (1.f - kk);
        else if (a.damp == DEER_DAMP_CLIP) ai = fminf(fmaxf(ai, -kk), kk);
        ao[j] = ai;
        bo[j] = F - ai * h;
        const float res = sc[j] - F;
        const float sa = fabsf(sc[j]);
        const float m = fabsf(res) / (sa > 1.f ? sa : 1.f);
        mx = (m > mx || m != m) ? m : mx;
        sq += res * res;
      }
      if (rv[i]) {
        *reinterpret_cast<float4*>(a.b + rows[i] * kGD + 4 * tx) = make_float4(bo[0], bo[1], bo[2], bo[3]);
        if (a.jac == DEER_JAC_DIAG)
          *reinterpret_cast<float4*>(a.A + rows[i] * kGD + 4 * tx) = make_float4(ao[0], ao[1], ao[2], ao[3]);
        // per-row partial residual statistics (non-negative floats order like their bits)
        atomicMax(reinterpret_cast<int*>(&S.rmx[rl]), __float_as_int(mx));
        atomicAdd(&S.rsq[rl], sq);
      }
    }
    __syncthreads();
    if (tid < kGT) {
      const int64_t sq_ = S.rseq[tid];
      int64_t rrow = 0;
      if (S.rvalid[tid]) {
        int64_t sq2;
        act_row(a.bt, tile * kGT + tid, sq2, rrow);
        rrow -= __ldg(a.bt.offsets + sq_);
      }
      acc_resid_f(a.acc, sq_, S.rvalid[tid] != 0, S.rmx[tid], S.rsq[tid],
                  bad_key(!(S.rmx[tid] <= a.tol_f), rrow));
    }
    __syncthreads();
  }
}

// W x_t for the three gates: out[row][g][i] = sum_k W_g[i][k] x_t[k]
__global__ void __launch_bounds__(kGThreads) k_gru_xproj(const float* __restrict__ W,
                                                         const float* __restrict__ x, int64_t N,
                                                         float* __restrict__ out) {
  __shared__ __align__(16) float WT[kGD][kGD];
  __shared__ __align__(16) float XT[kGD][kGT];
  const int tid = threadIdx.x, ty = tid & 15, tx = tid >> 4;
  const int64_t n_tiles = (N + kGT - 1) / kGT;
  for (int g = 0; g < 3; ++g) {
    __syncthreads();
    for (int e = tid; e < kGD * kGD; e += kGThreads) WT[e % kGD][e / kGD] = W[g * kGD * kGD + e];
    __syncthreads();
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
      for (int e = tid; e < kGT * kGD; e += kGThreads) {
        const int rl = e % kGT, k = e / kGT;
        const int64_t row = tile * kGT + rl;
        XT[k][rl] = row < N ? x[row * kGD + k] : 0.f;
      }
      __syncthreads();
      float acc[4][4] = {};
#pragma unroll 8
      for (int k = 0; k < kGD; ++k) {
        const float4 x4 = lds4(&XT[k][4 * ty]);
        const float4 w4 = lds4(&WT[k][4 * tx]);
        const float xx[4] = {x4.x, x4.y, x4.z, x4.w};
        const float ww[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] += xx[i] * ww[j];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int64_t row = tile * kGT + 4 * ty + i;
        if (row < N)
          *reinterpret_cast<float4*>(out + row * (3 * kGD) + g * kGD + 4 * tx) =
              make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      }
      __syncthreads();
    }
  }
}

static int persistent_grid(const void* kernel, int threads, size_t smem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
  return (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
}

cudaError_t launch_gru_xproj(const float* W, const float* x, int64_t N, float* out,
                             cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  const int g = persistent_grid((const void*)k_gru_xproj, kGThreads, 0);
  const int64_t tiles = (N + kGT - 1) / kGT;
  k_gru_xproj<<<(unsigned)(tiles < g ? tiles : g), kGThreads, 0, st>>>(W, x, N, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gru_lin_tiled(const GruTileArgs& a, cudaStream_t st) {
  if (a.bt.act_rows() == 0) return cudaSuccess;
  const size_t smem = sizeof(GruSmem);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_gru_lin_tiled,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int g = persistent_grid((const void*)k_gru_lin_tiled, kGThreads, smem);
  const int64_t tiles = (a.bt.act_rows() + kGT - 1) / kGT;
  k_gru_lin_tiled<<<(unsigned)(tiles < g ? tiles : g), kGThreads, smem, st>>>(a);
  note_launch();
  return cudaGetLastError();
}

}  // namespace deer
