// Per-iteration hot path of the PDF solver: loss of Eq. (13)-(19) and its adjoint.
//
// Data flow of one pdf_loss_grad (p = incidence, n = pixel):
//   k_synth_rowfft     J_p = F*_T(alpha_p) (Eq. 9), padded row DFT of J_p -> A
//   k_colconv          column DFT, x G_D spectrum, inverse column DFT (zero-padded convolution, Eq. 3)
//   k_rowifft_state    inverse row DFT -> G_D J; s = beta J + E_inc + G_D J; per-pixel least squares
//                      R = sum beta J conj(s) / sum |s|^2 over incidences (Eq. 6); chi = R/(beta(1-R))
//                      (Eq. 7); r = R s - beta J and ||r||^2 (Eq. 15)
//   k_gs_partial/reduce  G_S J - E_sca and ||.||^2 (Eq. 16)
//   k_reg              L_Bound, L_TV, L_Bridge (Eq. 17-19) and their cotangent on chi -> on R -> w
//   k_adj_rowfft       u = 2/||Einc||^2 conj(R) r + c_s (goes through G_D^H), v = pointwise part
//   k_colconv(conj)    G_D^H = convolution with the conjugated spectrum (G_D is symmetric)
//   k_gsh              2/||Esca||^2 G_S^H r_d
//   k_adj_rowifft_ana  dL/dJ = v + G_D^H u + G_S^H term, then analysis along x
//   k_ana_y            analysis along y -> dL/d alpha;  k_finalize sums the loss partials
//
// FP32 arithmetic with compensated FP32 per-thread sums and FP64 cross-thread/cross-block
// reductions (FP64 is a small fraction of FP32 throughput on this part, so it is kept out of
// per-element loops).
#include <algorithm>

#include "fft.cuh"
#include "problem.cuh"
#include "tc.cuh"

// Kahan-compensated accumulation in FP32; as a float-float value s - c.
struct KSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ FF ff() const { return ff_add(FF{s, 0.f}, -c); }
  __device__ __forceinline__ float f() const { return s - c; }
};

__device__ __forceinline__ float2 cmulf_(float2 a, float2 b) { return cmul(a, b); }

// ---------------------------------------------------------------------------
// synthesis (+ padded row DFT)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(ROW_THREADS) k_synth_rowfft(Dev d, const float2* __restrict__ alpha,
                                                              float2* __restrict__ Jout, int do_fft) {
  extern __shared__ float2 sm[];
  const int p = blockIdx.y, y0 = blockIdx.x * ROWS_PER_CTA;
  const int nrow = min(ROWS_PER_CTA, d.ny - y0);
  const int kx = d.kx, ky = d.ky;
  float2* sa = sm;                              // [ky][kx]
  float2* ty = sa + ky * kx;                    // [ROWS][kx]
  float2* b0 = ty + ROWS_PER_CTA * kx;          // [ROWS][Px]
  float2* b1 = b0 + ROWS_PER_CTA * d.Px;
  const float2* ap = alpha + (size_t)p * ky * kx;
  for (int i = threadIdx.x; i < ky * kx; i += blockDim.x) sa[i] = ap[i];
  __syncthreads();
  for (int i = threadIdx.x; i < ROWS_PER_CTA * kx; i += blockDim.x) {
    const int rr = i / kx, jx = i - rr * kx;
    float2 acc = make_float2(0.f, 0.f);
    if (rr < nrow) {
      const int y = y0 + rr;
      for (int jy = 0; jy < ky; ++jy) acc = acc + cmul(__ldg(&d.wy[jy * d.ny + y]), sa[jy * kx + jx]);
    }
    ty[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ROWS_PER_CTA * d.Px; i += blockDim.x) {
    const int rr = i / d.Px, x = i - rr * d.Px;
    float2 v = make_float2(0.f, 0.f);
    if (rr < nrow && x < d.nx) {
      for (int jx = 0; jx < kx; ++jx) v = v + cmul(ty[rr * kx + jx], __ldg(&d.wx[jx * d.nx + x]));
      Jout[((size_t)p * d.ny + y0 + rr) * d.nx + x] = v;
    }
    b0[i] = v;
  }
  if (!do_fft) return;
  __syncthreads();
  float2* res = fft_lines(b0, b1, ROWS_PER_CTA, d.Px, d.plx, d.twx, false);
  for (int i = threadIdx.x; i < ROWS_PER_CTA * d.Px; i += blockDim.x) {
    const int rr = i / d.Px, x = i - rr * d.Px;
    if (rr < nrow) d.A[((size_t)p * d.ny + y0 + rr) * d.Px + x] = res[i];
  }
}

// Padded row DFT of an arbitrary field [ni][ny][nx] -> A.
__global__ void __launch_bounds__(ROW_THREADS) k_rowfft_field(Dev d, const float2* __restrict__ in) {
  extern __shared__ float2 sm[];
  const int p = blockIdx.y, y0 = blockIdx.x * ROWS_PER_CTA;
  const int nrow = min(ROWS_PER_CTA, d.ny - y0);
  float2* b0 = sm;
  float2* b1 = sm + ROWS_PER_CTA * d.Px;
  for (int i = threadIdx.x; i < ROWS_PER_CTA * d.Px; i += blockDim.x) {
    const int rr = i / d.Px, x = i - rr * d.Px;
    b0[i] = (rr < nrow && x < d.nx) ? in[((size_t)p * d.ny + y0 + rr) * d.nx + x] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float2* res = fft_lines(b0, b1, ROWS_PER_CTA, d.Px, d.plx, d.twx, false);
  for (int i = threadIdx.x; i < ROWS_PER_CTA * d.Px; i += blockDim.x) {
    const int rr = i / d.Px, x = i - rr * d.Px;
    if (rr < nrow) d.A[((size_t)p * d.ny + y0 + rr) * d.Px + x] = res[i];
  }
}

// Inverse padded row DFT of A, cropped to nx -> out [ni][ny][nx].
__global__ void __launch_bounds__(ROW_THREADS) k_rowifft_field(Dev d, float2* __restrict__ out) {
  extern __shared__ float2 sm[];
  const int p = blockIdx.y, y0 = blockIdx.x * ROWS_PER_CTA;
  const int nrow = min(ROWS_PER_CTA, d.ny - y0);
  float2* b0 = sm;
  float2* b1 = sm + ROWS_PER_CTA * d.Px;
  for (int i = threadIdx.x; i < ROWS_PER_CTA * d.Px; i += blockDim.x) {
    const int rr = i / d.Px, x = i - rr * d.Px;
    b0[i] = rr < nrow ? d.A[((size_t)p * d.ny + y0 + rr) * d.Px + x] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float2* res = fft_lines(b0, b1, ROWS_PER_CTA, d.Px, d.plx, d.twx, true);
  for (int i = threadIdx.x; i < ROWS_PER_CTA * d.nx; i += blockDim.x) {
    const int rr = i / d.nx, x = i - rr * d.nx;
    if (rr < nrow) out[((size_t)p * d.ny + y0 + rr) * d.nx + x] = res[rr * d.Px + x];
  }
}

// ---------------------------------------------------------------------------
// column DFT -> x spectrum -> inverse column DFT (in place on A, rows >= ny dropped)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(COL_THREADS) k_colconv(Dev d, int conj) {
  extern __shared__ float2 sm[];
  const int p = blockIdx.y, c0 = blockIdx.x * COL_CW;
  const int ls = d.Py + 1;
  float2* b0 = sm;
  float2* b1 = sm + COL_CW * ls;
  const int ncol = min(COL_CW, d.Px - c0);
  float2* Ap = d.A + (size_t)p * d.ny * d.Px;
  for (int i = threadIdx.x; i < COL_CW * d.Py; i += blockDim.x) {
    const int y = i / COL_CW, c = i - y * COL_CW;
    float2 v = make_float2(0.f, 0.f);
    if (y < d.ny && c < ncol) v = Ap[(size_t)y * d.Px + c0 + c];
    b0[c * ls + y] = v;
  }
  __syncthreads();
  float2* res = fft_lines(b0, b1, COL_CW, ls, d.ply, d.twy, false);
  float2* oth = (res == b0) ? b1 : b0;
  for (int i = threadIdx.x; i < COL_CW * d.Py; i += blockDim.x) {
    const int k = i / COL_CW, c = i - k * COL_CW;
    if (c < ncol) {
      float2 g = __ldg(&d.ghat[(size_t)k * d.Px + c0 + c]);
      if (conj) g.y = -g.y;
      res[c * ls + k] = cmul(res[c * ls + k], g);
    }
  }
  __syncthreads();
  float2* res2 = fft_lines(res, oth, COL_CW, ls, d.ply, d.twy, true);
  for (int i = threadIdx.x; i < COL_CW * d.ny; i += blockDim.x) {
    const int y = i / COL_CW, c = i - y * COL_CW;
    if (c < ncol) Ap[(size_t)y * d.Px + c0 + c] = res2[c * ls + y];
  }
}

// ---------------------------------------------------------------------------
// inverse row DFT + CIE update + state residual, one CTA per grid row y over all incidences
// ---------------------------------------------------------------------------
#define XPT 2   // pixels per thread (nx <= 256 = XPT * ROW_THREADS)

__device__ __forceinline__ float2 chi_of_R(float2 R, float2 beta, float qmin, bool* clamped) {
  float2 q = make_float2(1.f - R.x, -R.y);
  float aq = sqrtf(cabs2(q));
  *clamped = aq < qmin;
  if (*clamped) q = aq > 0.f ? (qmin / aq) * q : make_float2(qmin, 0.f);
  return cdivf(R, cmul(beta, q));
}

__global__ void __launch_bounds__(ROW_THREADS) k_rowifft_state(Dev d) {
  extern __shared__ float2 sm[];
  __shared__ FF red[32];
  const int y = blockIdx.x;
  float2* b0 = sm;
  float2* b1 = sm + ROWS_PER_CTA * d.Px;
  KSum Nr[XPT], Ni[XPT], Dd[XPT];
  for (int p0 = 0; p0 < d.ni; p0 += ROWS_PER_CTA) {
    const int nb = min(ROWS_PER_CTA, d.ni - p0);
    for (int i = threadIdx.x; i < ROWS_PER_CTA * d.Px; i += blockDim.x) {
      const int b = i / d.Px, k = i - b * d.Px;
      b0[i] = b < nb ? d.A[((size_t)(p0 + b) * d.ny + y) * d.Px + k] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* res = fft_lines(b0, b1, ROWS_PER_CTA, d.Px, d.plx, d.twx, true);
    for (int b = 0; b < nb; ++b) {
#pragma unroll
      for (int k = 0; k < XPT; ++k) {
        const int x = threadIdx.x + k * blockDim.x;
        if (x < d.nx) {
          const size_t idx = ((size_t)(p0 + b) * d.ny + y) * d.nx + x;
          const float2 gj = res[b * d.Px + x];
          const float2 J = d.J[idx];
          const float2 s = cmul(d.beta, J) + d.einc[idx] + gj;
          d.s[idx] = s;
          const float2 n = cmul(d.beta, cmulc(J, s));
          Nr[k].add(n.x);
          Ni[k].add(n.y);
          Dd[k].add(cabs2(s));
        }
      }
    }
    __syncthreads();
  }
  float2 Rv[XPT];
#pragma unroll
  for (int k = 0; k < XPT; ++k) {
    const int x = threadIdx.x + k * blockDim.x;
    Rv[k] = make_float2(0.f, 0.f);
    if (x < d.nx) {
      const float D = Dd[k].f();
      const float2 R = make_float2(Nr[k].f() / D, Ni[k].f() / D);
      bool cl;
      const float2 chi = chi_of_R(R, d.beta, d.q_min, &cl);
      const int n = y * d.nx + x;
      d.R[n] = R;
      d.chi[n] = chi;
      d.D[n] = D;
      d.clamp[n] = cl ? 1 : 0;
      Rv[k] = R;
    }
  }
  KSum acc;
  for (int p = 0; p < d.ni; ++p) {
#pragma unroll
    for (int k = 0; k < XPT; ++k) {
      const int x = threadIdx.x + k * blockDim.x;
      if (x < d.nx) {
        const size_t idx = ((size_t)p * d.ny + y) * d.nx + x;
        const float2 r = cmul(Rv[k], d.s[idx]) - cmul(d.beta, d.J[idx]);
        d.r[idx] = r;
        acc.add(cabs2(r));
      }
    }
  }
  const FF t = ff_block_sum(acc.ff(), red);
  if (threadIdx.x == 0) d.lpart[LP_STATE * PDF_LP_STRIDE + y] = t;
}

// ---------------------------------------------------------------------------
// G_S x over all incidences: per-chunk partial products, then a deterministic reduction
// ---------------------------------------------------------------------------
#define GS_SUB 32
#define GS_TP 2
#define GS_TR 4

__global__ void __launch_bounds__(256) k_gs_partial(Dev d, const float2* __restrict__ X, float2* __restrict__ part) {
  extern __shared__ float2 sm[];
  const int ls = GS_SUB + 1;
  float2* sX = sm;                     // [ni][ls]
  float2* sG = sX + d.ni * ls;         // [nr][ls]
  float2* sR = sG + d.nr * ls;         // reduction scratch [256][GS_TP*GS_TR]
  const int n0 = blockIdx.x * d.gs_chunk;
  const int n1 = min(n0 + d.gs_chunk, d.M);
  const int tpn = (d.ni + GS_TP - 1) / GS_TP, trn = (d.nr + GS_TR - 1) / GS_TR;
  const int ntiles = tpn * trn;
  int kgroups = 1;
  while (kgroups * 2 * ntiles <= (int)blockDim.x && kgroups < GS_SUB) kgroups *= 2;
  const int npass = (ntiles * kgroups + blockDim.x - 1) / blockDim.x;
  for (int pass = 0; pass < npass; ++pass) {
    const int slot = pass * blockDim.x + threadIdx.x;
    const int tile = slot / kgroups, kg = slot - tile * kgroups;
    const bool active = tile < ntiles;
    const int tp = active ? tile / trn : 0, tr = active ? tile - (tile / trn) * trn : 0;
    float2 acc[GS_TP][GS_TR];
#pragma unroll
    for (int a = 0; a < GS_TP; ++a)
#pragma unroll
      for (int b = 0; b < GS_TR; ++b) acc[a][b] = make_float2(0.f, 0.f);
    for (int t0 = n0; t0 < n1; t0 += GS_SUB) {
      const int nt = min(GS_SUB, n1 - t0);
      __syncthreads();
      for (int i = threadIdx.x; i < d.ni * GS_SUB; i += blockDim.x) {
        const int p = i / GS_SUB, t = i - p * GS_SUB;
        sX[p * ls + t] = t < nt ? X[(size_t)p * d.M + t0 + t] : make_float2(0.f, 0.f);
      }
      for (int i = threadIdx.x; i < d.nr * GS_SUB; i += blockDim.x) {
        const int r = i / GS_SUB, t = i - r * GS_SUB;
        sG[r * ls + t] = t < nt ? d.gs[(size_t)r * d.M + t0 + t] : make_float2(0.f, 0.f);
      }
      __syncthreads();
      if (active) {
        for (int t = kg; t < GS_SUB; t += kgroups) {
          float2 xv[GS_TP], gv[GS_TR];
#pragma unroll
          for (int a = 0; a < GS_TP; ++a) {
            const int p = tp * GS_TP + a;
            xv[a] = p < d.ni ? sX[p * ls + t] : make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int b = 0; b < GS_TR; ++b) {
            const int r = tr * GS_TR + b;
            gv[b] = r < d.nr ? sG[r * ls + t] : make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int a = 0; a < GS_TP; ++a)
#pragma unroll
            for (int b = 0; b < GS_TR; ++b) acc[a][b] = acc[a][b] + cmul(gv[b], xv[a]);
        }
      }
    }
    // reduce over k-groups (consecutive threads of one tile) via shared memory
    __syncthreads();
#pragma unroll
    for (int a = 0; a < GS_TP; ++a)
#pragma unroll
      for (int b = 0; b < GS_TR; ++b) sR[threadIdx.x * GS_TP * GS_TR + a * GS_TR + b] = acc[a][b];
    __syncthreads();
    if (active && kg == 0) {
      for (int g = 1; g < kgroups; ++g)
#pragma unroll
        for (int a = 0; a < GS_TP; ++a)
#pragma unroll
          for (int b = 0; b < GS_TR; ++b) acc[a][b] = acc[a][b] + sR[(threadIdx.x + g) * GS_TP * GS_TR + a * GS_TR + b];
#pragma unroll
      for (int a = 0; a < GS_TP; ++a)
#pragma unroll
        for (int b = 0; b < GS_TR; ++b) {
          const int p = tp * GS_TP + a, r = tr * GS_TR + b;
          if (p < d.ni && r < d.nr) part[((size_t)blockIdx.x * d.ni + p) * d.nr + r] = acc[a][b];
        }
    }
  }
}

// out[p][r] = sum over chunks (FP64) [- sub]; ||out||^2 partial per block -> lp (may be NULL)
__global__ void k_gs_reduce(Dev d, const float2* __restrict__ part, int nchunk, const float2* __restrict__ sub,
                            float2* __restrict__ out, FF* __restrict__ lp) {
  __shared__ FF red[32];
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const int nout = d.ni * d.nr;
  FF a2 = FF{0.f, 0.f};
  if (o < nout) {
    FF sx = FF{0.f, 0.f}, sy = FF{0.f, 0.f};
    for (int c = 0; c < nchunk; ++c) {
      const float2 v = part[(size_t)c * nout + o];
      sx = ff_add(sx, v.x);
      sy = ff_add(sy, v.y);
    }
    if (sub) {
      sx = ff_add(sx, -sub[o].x);
      sy = ff_add(sy, -sub[o].y);
    }
    const float2 v = make_float2(sx.hi + sx.lo, sy.hi + sy.lo);
    out[o] = v;
    a2 = ff_make(cabs2(v));
  }
  if (lp) {
    const FF t = ff_block_sum(a2, red);
    if (threadIdx.x == 0) lp[blockIdx.x] = t;
  }
}

// ---------------------------------------------------------------------------
// G_S^H: out[p][n] = scale * sum_r conj(G[r][n]) in[p][r]
// ---------------------------------------------------------------------------
#define GSH_RT 32
#define GSH_TP 4
#define GSH_TN 4

__global__ void __launch_bounds__(256) k_gsh(Dev d, const float2* __restrict__ in, float2* __restrict__ out,
                                             float scale, int data_scale) {
  if (data_scale) scale = d.invn[1];     // 2 / ||E_sca||^2 of Eq. (16)'s gradient
  extern __shared__ float2 sm[];
  float2* sD = sm;                              // [ni][GSH_RT]
  float2* sG = sD + d.ni * GSH_RT;              // [GSH_RT][GSH_CHUNK + 1]
  float2* sR = sG + GSH_RT * (GSH_CHUNK + 1);   // [256][GSH_TP*GSH_TN]
  const int n0 = blockIdx.x * GSH_CHUNK;
  const int nn = min(GSH_CHUNK, d.M - n0);
  const int tpn = (d.ni + GSH_TP - 1) / GSH_TP, tnn = GSH_CHUNK / GSH_TN;
  const int ntiles = tpn * tnn;
  int kgroups = 1;
  while (kgroups * 2 * ntiles <= (int)blockDim.x && kgroups < GSH_RT) kgroups *= 2;
  const int npass = (ntiles * kgroups + blockDim.x - 1) / blockDim.x;
  for (int pass = 0; pass < npass; ++pass) {
    const int slot = pass * blockDim.x + threadIdx.x;
    const int tile = slot / kgroups, kg = slot - tile * kgroups;
    const bool active = tile < ntiles;
    const int tp = active ? tile / tnn : 0, tn = active ? tile - (tile / tnn) * tnn : 0;
    float2 acc[GSH_TP][GSH_TN];
#pragma unroll
    for (int a = 0; a < GSH_TP; ++a)
#pragma unroll
      for (int b = 0; b < GSH_TN; ++b) acc[a][b] = make_float2(0.f, 0.f);
    for (int r0 = 0; r0 < d.nr; r0 += GSH_RT) {
      const int nrt = min(GSH_RT, d.nr - r0);
      __syncthreads();
      for (int i = threadIdx.x; i < d.ni * GSH_RT; i += blockDim.x) {
        const int p = i / GSH_RT, r = i - p * GSH_RT;
        sD[i] = r < nrt ? in[(size_t)p * d.nr + r0 + r] : make_float2(0.f, 0.f);
      }
      for (int i = threadIdx.x; i < GSH_RT * GSH_CHUNK; i += blockDim.x) {
        const int r = i / GSH_CHUNK, t = i - r * GSH_CHUNK;
        sG[r * (GSH_CHUNK + 1) + t] = (r < nrt && t < nn) ? d.gs[(size_t)(r0 + r) * d.M + n0 + t] : make_float2(0.f, 0.f);
      }
      __syncthreads();
      if (active) {
        for (int r = kg; r < GSH_RT; r += kgroups) {
          float2 dv[GSH_TP], gv[GSH_TN];
#pragma unroll
          for (int a = 0; a < GSH_TP; ++a) {
            const int p = tp * GSH_TP + a;
            dv[a] = p < d.ni ? sD[p * GSH_RT + r] : make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int b = 0; b < GSH_TN; ++b) gv[b] = sG[r * (GSH_CHUNK + 1) + tn * GSH_TN + b];
#pragma unroll
          for (int a = 0; a < GSH_TP; ++a)
#pragma unroll
            for (int b = 0; b < GSH_TN; ++b) acc[a][b] = acc[a][b] + cmulc(dv[a], gv[b]);
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < GSH_TP; ++a)
#pragma unroll
      for (int b = 0; b < GSH_TN; ++b) sR[threadIdx.x * GSH_TP * GSH_TN + a * GSH_TN + b] = acc[a][b];
    __syncthreads();
    if (active && kg == 0) {
      for (int g = 1; g < kgroups; ++g)
#pragma unroll
        for (int a = 0; a < GSH_TP; ++a)
#pragma unroll
          for (int b = 0; b < GSH_TN; ++b)
            acc[a][b] = acc[a][b] + sR[(threadIdx.x + g) * GSH_TP * GSH_TN + a * GSH_TN + b];
#pragma unroll
      for (int a = 0; a < GSH_TP; ++a)
#pragma unroll
        for (int b = 0; b < GSH_TN; ++b) {
          const int p = tp * GSH_TP + a, t = tn * GSH_TN + b;
          if (p < d.ni && t < nn) out[(size_t)p * d.M + n0 + t] = scale * acc[a][b];
        }
    }
  }
}

// ---------------------------------------------------------------------------
// regularisers (Eq. 17-19) and their cotangent pulled back to w = c_R / D
// ---------------------------------------------------------------------------
struct TVB {  // per-pixel pieces of the TV and bridge terms at one pixel
  float2 dx, dy;
  float t;          // TV magnitude
  float gx, gy;     // |chi| forward differences
  float sg, e;      // sigmoid and exp factors
};

__device__ __forceinline__ float mag_at(const float2* chi, int nx, int y, int x, float eps) {
  const float2 c = chi[y * nx + x];
  return sqrtf(cabs2(c) + eps);
}

__device__ __forceinline__ TVB tvb_at(const Dev& d, int y, int x) {
  TVB o;
  const float2 c = d.chi[y * d.nx + x];
  const bool hx = x + 1 < d.nx, hy = y + 1 < d.ny;
  o.dx = hx ? d.chi[y * d.nx + x + 1] - c : make_float2(0.f, 0.f);
  o.dy = hy ? d.chi[(y + 1) * d.nx + x] - c : make_float2(0.f, 0.f);
  o.t = sqrtf(cabs2(o.dx) + cabs2(o.dy) + d.eps_tv);
  const float m = sqrtf(cabs2(c) + d.eps_abs);
  o.gx = hx ? mag_at(d.chi, d.nx, y, x + 1, d.eps_abs) - m : 0.f;
  o.gy = hy ? mag_at(d.chi, d.nx, y + 1, x, d.eps_abs) - m : 0.f;
  o.sg = 1.f / (1.f + expf(-(m - d.tau_b) / d.tau_b));
  o.e = expf(-(o.gx * o.gx + o.gy * o.gy));
  return o;
}

__global__ void __launch_bounds__(256) k_reg(Dev d) {
  __shared__ FF red[32];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  float lb = 0.f, ltv = 0.f, lbr = 0.f;
  if (n < d.M) {
    const int y = n / d.nx, x = n - y * d.nx;
    const float2 c = d.chi[n];
    const float neg = fmaxf(-c.x, 0.f);
    lb = neg * neg;
    const TVB o = tvb_at(d, y, x);
    ltv = o.t;
    lbr = o.sg * o.e;
    // TV cotangent: -(dx + dy)/t at the own term, + dx/t of the left term, + dy/t of the upper term
    float2 ctv = (-1.f / o.t) * (o.dx + o.dy);
    // bridge cotangent on |chi|: own sigmoid term, own differences (-1), left / upper differences (+1)
    float dm = o.sg * (1.f - o.sg) / d.tau_b * o.e + 2.f * (o.gx + o.gy) * o.sg * o.e;
    if (x > 0) {
      const TVB l = tvb_at(d, y, x - 1);
      ctv = ctv + (1.f / l.t) * l.dx;
      dm += -2.f * l.gx * l.sg * l.e;
    }
    if (y > 0) {
      const TVB u = tvb_at(d, y - 1, x);
      ctv = ctv + (1.f / u.t) * u.dy;
      dm += -2.f * u.gy * u.sg * u.e;
    }
    const float m = sqrtf(cabs2(c) + d.eps_abs);
    float2 cchi = d.lam_tv * ctv + (d.lam_bridge * dm / m) * c;
    cchi.x += d.lam_bound * (-2.f * neg);
    // chi = R / (beta (1 - R)):  d chi / d R = 1 / (beta (1 - R)^2), zero where clamped
    float2 w = make_float2(0.f, 0.f);
    if (!d.clamp[n]) {
      const float2 R = d.R[n];
      const float2 q = make_float2(1.f - R.x, -R.y);
      const float2 dchi = cdivf(make_float2(1.f, 0.f), cmul(d.beta, cmul(q, q)));
      const float2 cR = cmul(cconj(dchi), cchi);
      w = (1.f / d.D[n]) * cR;
    }
    d.w[n] = w;
  }
  const FF tb = ff_block_sum(ff_make(lb), red);
  const FF tt = ff_block_sum(ff_make(ltv), red);
  const FF tr = ff_block_sum(ff_make(lbr), red);
  if (threadIdx.x == 0) {
    d.lpart[LP_BOUND * PDF_LP_STRIDE + blockIdx.x] = tb;
    d.lpart[LP_TV * PDF_LP_STRIDE + blockIdx.x] = tt;
    d.lpart[LP_BRIDGE * PDF_LP_STRIDE + blockIdx.x] = tr;
  }
}

// ---------------------------------------------------------------------------
// adjoint: u (through G_D^H) and v (pointwise), then padded row DFT of u
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(ROW_THREADS) k_adj_rowfft(Dev d) {
  extern __shared__ float2 sm[];
  const int p = blockIdx.y, y0 = blockIdx.x * ROWS_PER_CTA;
  const int nrow = min(ROWS_PER_CTA, d.ny - y0);
  float2* b0 = sm;
  float2* b1 = sm + ROWS_PER_CTA * d.Px;
  const float ke = d.invn[0];
  const float2 bc = cconj(d.beta);
  for (int i = threadIdx.x; i < ROWS_PER_CTA * d.Px; i += blockDim.x) {
    const int rr = i / d.Px, x = i - rr * d.Px;
    float2 u = make_float2(0.f, 0.f);
    if (rr < nrow && x < d.nx) {
      const int n = (y0 + rr) * d.nx + x;
      const size_t idx = (size_t)p * d.M + n;
      const float2 w = d.w[n], R = d.R[n];
      const float2 J = d.J[idx], s = d.s[idx], r = d.r[idx];
      const float2 wc = cconj(w);
      const float2 cs = cmul(cmul(wc, d.beta), J) - (2.f * cmul(wc, R).x) * s;
      u = ke * cmulc(r, R) + cs;
      const float2 omr = make_float2(1.f - R.x, R.y);                  // 1 - conj(R)
      const float2 v = ke * cmul(cmul(make_float2(-bc.x, -bc.y), omr), r) + cmul(bc, cmul(w, s) + cs);
      d.v[idx] = v;
    }
    b0[i] = u;
  }
  __syncthreads();
  float2* res = fft_lines(b0, b1, ROWS_PER_CTA, d.Px, d.plx, d.twx, false);
  for (int i = threadIdx.x; i < ROWS_PER_CTA * d.Px; i += blockDim.x) {
    const int rr = i / d.Px, x = i - rr * d.Px;
    if (rr < nrow) d.A[((size_t)p * d.ny + y0 + rr) * d.Px + x] = res[i];
  }
}

// inverse row DFT of A (-> G_D^H u), add v and the G_S^H term, then analysis along x -> T2.
// mode 0: full adjoint; mode 1: plain analysis of the field `in` (no DFT, no additions).
__global__ void __launch_bounds__(ROW_THREADS) k_adj_rowifft_ana(Dev d, const float2* __restrict__ in, int mode) {
  extern __shared__ float2 sm[];
  const int p = blockIdx.y, y0 = blockIdx.x * ROWS_PER_CTA;
  const int nrow = min(ROWS_PER_CTA, d.ny - y0);
  float2* b0 = sm;
  float2* b1 = sm + ROWS_PER_CTA * d.Px;
  float2* g;
  if (mode == 0) {
    for (int i = threadIdx.x; i < ROWS_PER_CTA * d.Px; i += blockDim.x) {
      const int rr = i / d.Px, x = i - rr * d.Px;
      b0[i] = rr < nrow ? d.A[((size_t)p * d.ny + y0 + rr) * d.Px + x] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    g = fft_lines(b0, b1, ROWS_PER_CTA, d.Px, d.plx, d.twx, true);
    for (int i = threadIdx.x; i < ROWS_PER_CTA * d.nx; i += blockDim.x) {
      const int rr = i / d.nx, x = i - rr * d.nx;
      if (rr < nrow) {
        const size_t idx = (size_t)p * d.M + (y0 + rr) * d.nx + x;
        g[rr * d.Px + x] = g[rr * d.Px + x] + d.v[idx] + d.gsh[idx];
      }
    }
  } else {
    g = b0;
    for (int i = threadIdx.x; i < ROWS_PER_CTA * d.nx; i += blockDim.x) {
      const int rr = i / d.nx, x = i - rr * d.nx;
      g[rr * d.Px + x] = rr < nrow ? in[(size_t)p * d.M + (y0 + rr) * d.nx + x] : make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ROWS_PER_CTA * d.kx; i += blockDim.x) {
    const int rr = i / d.kx, jx = i - rr * d.kx;
    if (rr < nrow) {
      float2 acc = make_float2(0.f, 0.f);
      for (int x = 0; x < d.nx; ++x) acc = acc + cmulc(g[rr * d.Px + x], __ldg(&d.wx[jx * d.nx + x]));
      d.T2[((size_t)p * d.ny + y0 + rr) * d.kx + jx] = acc;
    }
  }
}

// analysis along y: out[p][jy][jx] = sum_y conj(wy[jy][y]) T2[p][y][jx]; one CTA per (jy, p),
// eight warps over interleaved y, lanes over jx (kx <= 64)
__global__ void __launch_bounds__(256) k_ana_y(Dev d, const float2* __restrict__ T2, float2* __restrict__ out) {
  __shared__ float2 part[8][64];
  const int jy = blockIdx.x, p = blockIdx.y, g = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float2* T = T2 + (size_t)p * d.ny * d.kx;
  float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
  for (int y = g; y < d.ny; y += 8) {
    const float2 w = __ldg(&d.wy[jy * d.ny + y]);
    if (lane < d.kx) a0 = a0 + cmulc(T[(size_t)y * d.kx + lane], w);
    if (lane + 32 < d.kx) a1 = a1 + cmulc(T[(size_t)y * d.kx + lane + 32], w);
  }
  part[g][lane] = a0;
  part[g][lane + 32] = a1;
  __syncthreads();
  if (threadIdx.x < d.kx) {
    float2 s = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 8; ++k) s = s + part[k][threadIdx.x];
    out[((size_t)p * d.ky + jy) * d.kx + threadIdx.x] = s;
  }
}

// terms[6] = L, State, Data, Bound, TV, Bridge from the partial sums
__global__ void k_finalize(Dev d, double* __restrict__ terms, int n_state, int n_data, int n_reg, int* step_inc) {
  __shared__ FF red[32];
  const int cnt[5] = {n_state, n_data, n_reg, n_reg, n_reg};
  double tot[5];
  for (int s = 0; s < 5; ++s) {
    FF a = FF{0.f, 0.f};
    for (int i = threadIdx.x; i < cnt[s]; i += blockDim.x) a = ff_add(a, d.lpart[s * PDF_LP_STRIDE + i]);
    tot[s] = ff_to_d(ff_block_sum(a, red));
  }
  if (threadIdx.x == 0) {
    const double st = tot[0] / d.norms[0], da = tot[1] / d.norms[1];
    terms[1] = st;
    terms[2] = da;
    terms[3] = tot[2];
    terms[4] = tot[3];
    terms[5] = tot[4];
    terms[0] = st + da + (double)d.lam_bound * tot[2] + (double)d.lam_tv * tot[3] + (double)d.lam_bridge * tot[4];
    if (step_inc) *step_inc += 1;
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static size_t sm_row(const Dev& d) { return 2 * ROWS_PER_CTA * (size_t)d.Px * sizeof(float2); }
static size_t sm_synth(const Dev& d) {
  return ((size_t)d.ky * d.kx + ROWS_PER_CTA * d.kx) * sizeof(float2) + sm_row(d);
}
static size_t sm_col(const Dev& d) { return 2 * COL_CW * (size_t)(d.Py + 1) * sizeof(float2); }
static size_t sm_gs(const Dev& d) {
  return ((size_t)(d.ni + d.nr) * (GS_SUB + 1) + 256 * GS_TP * GS_TR) * sizeof(float2);
}
static size_t sm_gsh(const Dev& d) {
  return ((size_t)d.ni * GSH_RT + GSH_RT * (GSH_CHUNK + 1) + 256 * GSH_TP * GSH_TN) * sizeof(float2);
}

pdf_status hp_configure_kernels() {
  const int big = 200 * 1024;
  cudaFuncSetAttribute(k_synth_rowfft, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_rowfft_field, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_rowifft_field, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_colconv, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_rowifft_state, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_gs_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_gsh, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_adj_rowfft, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_adj_rowifft_ana, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(e, "cudaFuncSetAttribute");
  return PDF_OK;
}

static inline dim3 row_grid(const Dev& d) { return dim3((d.ny + ROWS_PER_CTA - 1) / ROWS_PER_CTA, d.ni); }
static inline dim3 col_grid(const Dev& d) { return dim3((d.Px + COL_CW - 1) / COL_CW, d.ni); }

int hp_kernels_per_loss_grad(const pdf_problem* h) { return h->tc ? 11 : 12; }

pdf_status hp_check_limits(const Dev& d) {
  const size_t lim = 200 * 1024;
  if (d.fast && (fp_smem_synth(d) > 100 * 1024 || fp_smem_col(d) > 100 * 1024 || fp_smem_state(d) > 100 * 1024 ||
                 fp_smem_ana(d) > 100 * 1024))
    return set_err(PDF_EUNSUPPORTED, "problem too large for the register-FFT tiling");
  if (sm_row(d) > lim || sm_synth(d) > lim || sm_col(d) > lim || sm_gs(d) > lim || sm_gsh(d) > lim)
    return set_err(PDF_EUNSUPPORTED, "problem too large for the shared-memory tiling (reduce ni, nr or kx*ky)");
  if ((d.ni * d.nr + 255) / 256 > PDF_LP_STRIDE || d.n_reg_blocks > PDF_LP_STRIDE || d.ny > PDF_LP_STRIDE)
    return set_err(PDF_EUNSUPPORTED, "problem too large for the loss-partial buffer");
  return PDF_OK;
}

static const char* kLossGradKernels[] = {
    "k_synth_rowfft", "k_colconv", "k_rowifft_state", "k_gs_partial", "k_gs_reduce", "k_reg",
    "k_adj_rowfft",   "k_colconv(conj)", "k_gsh",     "k_adj_rowifft_ana", "k_ana_y", "k_finalize"};
static const char* kLossGradStagesTC[] = {
    "tc_synth(synth1+gemm+post)", "k_colconv", "k_rowifft_state", "tc_gs(gemm+reduce)", "k_reg",
    "k_adj_rowfft", "k_colconv(conj)", "tc_gsh(gemm)", "tc_adj(rowifft+gemm)", "k_ana_y", "k_finalize"};

const char* hp_kernel_name(int k, int precision) {
  if (precision == 1) return (k >= 0 && k < 11) ? kLossGradStagesTC[k] : "";
  return (k >= 0 && k < 12) ? kLossGradKernels[k] : "";
}

pdf_status hp_loss_grad(pdf_problem* h, const float2* alpha, float2* grad, double* terms, cudaStream_t st,
                        int* step_inc, cudaEvent_t* ev) {
  Dev& d = h->d;
  const int nout = d.ni * d.nr;
  const int n_data_blocks = (nout + 255) / 256;
  const bool tc = h->tc != nullptr;
  pdf_status s;
  int k = 0;
  auto mark = [&]() {
    if (ev) cudaEventRecord(ev[k++], st);
  };
  mark();
  // forward
  if (tc) {
    if ((s = tc_synth(h, alpha, d.J, 1, st)) != PDF_OK) return s;
  } else if (d.fast) {
    if ((s = fp_synth_rowfft(d, alpha, d.J, 1, st)) != PDF_OK) return s;
  } else {
    k_synth_rowfft<<<row_grid(d), ROW_THREADS, sm_synth(d), st>>>(d, alpha, d.J, 1);
  }
  mark();
  if (d.fast) {
    if ((s = fp_colconv(d, 0, st)) != PDF_OK) return s;
  } else {
    k_colconv<<<col_grid(d), COL_THREADS, sm_col(d), st>>>(d, 0);
  }
  mark();
  if (d.fast) {
    if ((s = fp_rowifft_state(d, st)) != PDF_OK) return s;
  } else {
    k_rowifft_state<<<d.ny, ROW_THREADS, sm_row(d), st>>>(d);
  }
  mark();
  if (tc) {
    if ((s = tc_gs_fwd(h, nullptr, d.esca, d.rd, d.lpart + LP_DATA * PDF_LP_STRIDE, 1, st)) != PDF_OK) return s;
  } else {
    k_gs_partial<<<d.n_gs_chunks, 256, sm_gs(d), st>>>(d, d.J, d.gspart);
    mark();
    k_gs_reduce<<<n_data_blocks, 256, 0, st>>>(d, d.gspart, d.n_gs_chunks, d.esca, d.rd,
                                                d.lpart + LP_DATA * PDF_LP_STRIDE);
  }
  mark();
  k_reg<<<d.n_reg_blocks, 256, 0, st>>>(d);
  mark();
  // adjoint
  if (d.fast) {
    if ((s = fp_adj_rowfft(d, st)) != PDF_OK) return s;
  } else {
    k_adj_rowfft<<<row_grid(d), ROW_THREADS, sm_row(d), st>>>(d);
  }
  mark();
  if (d.fast) {
    if ((s = fp_colconv(d, 1, st)) != PDF_OK) return s;
  } else {
    k_colconv<<<col_grid(d), COL_THREADS, sm_col(d), st>>>(d, 1);
  }
  mark();
  const float2* T2 = d.T2;
  if (tc) {
    if ((s = tc_gsh(h, nullptr, 1, st)) != PDF_OK) return s;
    mark();
    if ((s = tc_adj_ana(h, st)) != PDF_OK) return s;
    T2 = (const float2*)h->tc->c_ana;
  } else {
    k_gsh<<<(d.M + GSH_CHUNK - 1) / GSH_CHUNK, 256, sm_gsh(d), st>>>(d, d.rd, d.gsh, 0.f, 1);
    mark();
    if (d.fast) {
      if ((s = fp_adj_rowifft_ana(d, nullptr, 0, st)) != PDF_OK) return s;
    } else {
      k_adj_rowifft_ana<<<row_grid(d), ROW_THREADS, sm_row(d), st>>>(d, nullptr, 0);
    }
  }
  mark();
  float2* g = grad ? grad : h->grad;
  k_ana_y<<<dim3(d.ky, d.ni), 256, 0, st>>>(d, T2, g);
  mark();
  k_finalize<<<1, 256, 0, st>>>(d, terms ? terms : h->terms, d.ny, n_data_blocks, d.n_reg_blocks, step_inc);
  mark();
  pdf_count_launch(tc ? 7 : 12);
  PDF_LAUNCHED("pdf_loss_grad");
  return PDF_OK;
}

pdf_status hp_gd(pdf_problem* h, const float2* in, float2* out, int adjoint, cudaStream_t st) {
  Dev& d = h->d;
  if (d.fast) {
    pdf_status s;
    if ((s = fp_rowfft_field(d, in, st)) != PDF_OK) return s;
    if ((s = fp_colconv(d, adjoint, st)) != PDF_OK) return s;
    if ((s = fp_rowifft_field(d, out, st)) != PDF_OK) return s;
    pdf_count_launch(3);
    PDF_LAUNCHED("G_D apply");
    return PDF_OK;
  }
  k_rowfft_field<<<row_grid(d), ROW_THREADS, sm_row(d), st>>>(d, in);
  k_colconv<<<col_grid(d), COL_THREADS, sm_col(d), st>>>(d, adjoint);
  k_rowifft_field<<<row_grid(d), ROW_THREADS, sm_row(d), st>>>(d, out);
  pdf_count_launch(3);
  PDF_LAUNCHED("G_D apply");
  return PDF_OK;
}

pdf_status hp_gs(pdf_problem* h, const float2* in, float2* out, const float2* subtract, FF* sumsq,
                 cudaStream_t st) {
  if (h->tc) return tc_gs_fwd(h, in, subtract, out, sumsq, 0, st);
  Dev& d = h->d;
  const int nout = d.ni * d.nr;
  k_gs_partial<<<d.n_gs_chunks, 256, sm_gs(d), st>>>(d, in, d.gspart);
  k_gs_reduce<<<(nout + 255) / 256, 256, 0, st>>>(d, d.gspart, d.n_gs_chunks, subtract, out, sumsq);
  pdf_count_launch(2);
  PDF_LAUNCHED("G_S apply");
  return PDF_OK;
}

pdf_status hp_gsh(pdf_problem* h, const float2* in, float2* out, float scale, cudaStream_t st) {
  if (h->tc) return tc_gsh_field(h, in, out, scale, st);
  Dev& d = h->d;
  k_gsh<<<(d.M + GSH_CHUNK - 1) / GSH_CHUNK, 256, sm_gsh(d), st>>>(d, in, out, scale, 0);
  pdf_count_launch(1);
  PDF_LAUNCHED("G_S^H apply");
  return PDF_OK;
}

pdf_status hp_synth(pdf_problem* h, const float2* alpha, float2* out, cudaStream_t st) {
  if (h->tc) return tc_synth(h, alpha, out, 0, st);
  Dev& d = h->d;
  if (d.fast) {
    pdf_status s = fp_synth_rowfft(d, alpha, out, 0, st);
    pdf_count_launch(1);
    return s;
  }
  k_synth_rowfft<<<row_grid(d), ROW_THREADS, sm_synth(d), st>>>(d, alpha, out, 0);
  pdf_count_launch(1);
  PDF_LAUNCHED("synthesis");
  return PDF_OK;
}

pdf_status hp_analysis(pdf_problem* h, const float2* in, float2* out, cudaStream_t st) {
  Dev& d = h->d;
  const float2* T2 = d.T2;
  if (h->tc) {
    pdf_status s = tc_analysis_field(h, in, st);
    if (s != PDF_OK) return s;
    T2 = (const float2*)h->tc->c_ana;
  } else if (d.fast) {
    pdf_status s = fp_adj_rowifft_ana(d, in, 1, st);
    if (s != PDF_OK) return s;
  } else {
    k_adj_rowifft_ana<<<row_grid(d), ROW_THREADS, sm_row(d), st>>>(d, in, 1);
  }
  k_ana_y<<<dim3(d.ky, d.ni), 256, 0, st>>>(d, T2, out);
  pdf_count_launch(2);
  PDF_LAUNCHED("analysis");
  return PDF_OK;
}

pdf_status hp_chi(pdf_problem* h, const float2* alpha, float2* chi_out, cudaStream_t st) {
  Dev& d = h->d;
  if (h->tc) {
    pdf_status s = tc_synth(h, alpha, d.J, 1, st);
    if (s != PDF_OK) return s;
  } else if (d.fast) {
    pdf_status s = fp_synth_rowfft(d, alpha, d.J, 1, st);
    if (s != PDF_OK) return s;
  } else {
    k_synth_rowfft<<<row_grid(d), ROW_THREADS, sm_synth(d), st>>>(d, alpha, d.J, 1);
  }
  if (d.fast) {
    pdf_status s;
    if ((s = fp_colconv(d, 0, st)) != PDF_OK) return s;
    if ((s = fp_rowifft_state(d, st)) != PDF_OK) return s;
  } else {
    k_colconv<<<col_grid(d), COL_THREADS, sm_col(d), st>>>(d, 0);
    k_rowifft_state<<<d.ny, ROW_THREADS, sm_row(d), st>>>(d);
  }
  pdf_count_launch(3);
  PDF_LAUNCHED("chi");
  if (chi_out) PDF_CUDA(cudaMemcpyAsync(chi_out, d.chi, sizeof(float2) * d.M, cudaMemcpyDeviceToDevice, st));
  return PDF_OK;
}
