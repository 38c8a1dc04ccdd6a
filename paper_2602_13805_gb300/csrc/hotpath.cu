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
//                      (with the CCO inside the loss: the six kernels of ccoloss.cu instead)
//   k_adj_rowfft       u = 2/||Einc||^2 conj(R) r + c_s (goes through G_D^H), v = pointwise part
//   k_colconv(conj)    G_D^H = convolution with the conjugated spectrum (G_D is symmetric)
//   k_gsh              2/||Esca||^2 G_S^H r_d
//   k_adj_rowifft_ana  dL/dJ = v + G_D^H u + G_S^H term, then analysis along x
//   k_ana_y            analysis along y -> dL/d alpha;  k_finalize sums the loss partials
//   (with the folded data term and coefficients that fit, the data residual is k_gsf_fwd_p: a
//   warp per receiver, alpha_p in shared memory, no separate reduction)
//
// FP32 arithmetic with compensated FP32 per-thread sums and FP64 cross-thread/cross-block
// reductions (FP64 is a small fraction of FP32 throughput on this part, so it is kept out of
// per-element loops).
#include <algorithm>

#include "fft.cuh"
#include "phases.cuh"
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
      for (int jy = 0; jy < ky; ++jy) acc = cmac(acc, __ldg(&d.wy[jy * d.ny + y]), sa[jy * kx + jx]);
    }
    ty[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ROWS_PER_CTA * d.Px; i += blockDim.x) {
    const int rr = i / d.Px, x = i - rr * d.Px;
    float2 v = make_float2(0.f, 0.f);
    if (rr < nrow && x < d.nx) {
      for (int jx = 0; jx < kx; ++jx) v = cmac(v, ty[rr * kx + jx], __ldg(&d.wx[jx * d.nx + x]));
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
__global__ void __launch_bounds__(256) k_gs_partial(Dev d, const float2* X, float2* part) {
  extern __shared__ float2 sm[];
  ph_gs_partial(d, blockIdx.x, sm, X, part);
}

// out[p][r] = sum over chunks (FP64) [- sub]; ||out||^2 partial per block -> lp (may be NULL)
__global__ void k_gs_reduce(Dev d, const float2* part, int nchunk, const float2* sub, float2* out, FF* lp) {
  ph_gs_reduce(d, blockIdx.x, part, nchunk, sub, out, lp);
}

// ---------------------------------------------------------------------------
// G_S^H: out[p][n] = scale * sum_r conj(G[r][n]) in[p][r]
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gsh(Dev d, const float2* in, float2* out, float scale, int data_scale) {
  extern __shared__ float2 sm[];
  ph_gsh(d, blockIdx.x, sm, in, out, scale, data_scale);
}

// ---------------------------------------------------------------------------
// regularisers (Eq. 17-19) and their cotangent pulled back to w = c_R / D
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_reg(Dev d) {
  pdl_wait();
  ph_reg(d, blockIdx.x, d.chi, nullptr);
}

// The regularisers (Eq. 17-19) by 2-D tiles of RT_Y x RT_X pixels in two phases: chi-hat of the
// tile with a one-pixel halo staged in shared memory; each pixel's TV / bridge pieces evaluated
// once (the tile plus its left column and upper row, one thread each); then at each pixel its own
// pieces combined with its left and upper neighbours', carried to w.  One loss partial per tile
// (slot blockIdx.y gridDim.x + blockIdx.x).
#define RT_X 32
#define RT_Y 8
#define RT_PX ((RT_Y + 1) * (RT_X + 1))
#define RT_THREADS ((RT_PX + 31) / 32 * 32)
__global__ void __launch_bounds__(RT_THREADS) k_reg_tile(Dev d) {
  __shared__ float2 cs[RT_Y + 2][RT_X + 2];
  __shared__ RegPiece pc[RT_Y + 1][RT_X + 1];
  __shared__ FF red_rt[3 * 32];
  pdl_wait();
  const int x0 = blockIdx.x * RT_X, y0 = blockIdx.y * RT_Y;
  const int ty = threadIdx.x / RT_X, y = y0 + ty, x = x0 + threadIdx.x % RT_X, n = y * d.nx + x;
  const bool own = threadIdx.x < RT_X * RT_Y && y < d.ny && x < d.nx;
  // this pixel's operands for carrying the cotangent to w, fetched before the staging waits
  bool clamped = true;
  float2 Rn = make_float2(0.f, 0.f);
  float Dn = 1.f;
  if (own) {
    clamped = d.clamp[n] != 0;
    Rn = d.R[n];
    Dn = d.D[n];
  }
  for (int i = threadIdx.x; i < (RT_Y + 2) * (RT_X + 2); i += blockDim.x) {
    const int ly = i / (RT_X + 2), lx = i - ly * (RT_X + 2), y = y0 - 1 + ly, x = x0 - 1 + lx;
    cs[ly][lx] = (y >= 0 && y < d.ny && x >= 0 && x < d.nx) ? d.chi[y * d.nx + x] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  if (threadIdx.x < RT_PX) {  // region pixel (y0 - 1 + ly, x0 - 1 + lx)
    const int ly = threadIdx.x / (RT_X + 1), lx = threadIdx.x - ly * (RT_X + 1);
    const int y = y0 - 1 + ly, x = x0 - 1 + lx;
    if (y >= 0 && y < d.ny && x >= 0 && x < d.nx) {
      const float2* c = &cs[ly][lx];
      pc[ly][lx] = reg_piece(d, tvb_at(d, [=](int oy, int ox) { return c[oy * (RT_X + 2) + ox]; }, y, x, 0, 0));
    }
  }
  __syncthreads();
  float lb = 0.f, ltv = 0.f, lbr = 0.f;
  if (own) {
    const int tx = x - x0;
    const float2 cchi = reg_combine(d, cs[ty + 1][tx + 1], pc[ty + 1][tx + 1], x > 0 ? &pc[ty + 1][tx] : nullptr,
                                    y > 0 ? &pc[ty][tx + 1] : nullptr, lb, ltv, lbr);
    d.w[n] = reg_w_at(d, clamped, Rn, Dn, cchi);
  }
  FF t3[3] = {ff_make(lb), ff_make(ltv), ff_make(lbr)};
  ff_block_sum_multi<3>(t3, red_rt);
  if (threadIdx.x == 0) {
    const int b = blockIdx.y * gridDim.x + blockIdx.x;
    d.lpart[LP_BOUND * PDF_LP_STRIDE + b] = t3[0];
    d.lpart[LP_TV * PDF_LP_STRIDE + b] = t3[1];
    d.lpart[LP_BRIDGE * PDF_LP_STRIDE + b] = t3[2];
  }
}
static dim3 reg_tile_grid(const Dev& d) { return dim3((d.nx + RT_X - 1) / RT_X, (d.ny + RT_Y - 1) / RT_Y); }
static bool reg_tile_ok(const Dev& d) {
  const dim3 g = reg_tile_grid(d);
  return (size_t)g.x * g.y <= PDF_LP_STRIDE;
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
        g[rr * d.Px + x] = d.fold ? g[rr * d.Px + x] + d.v[idx] : g[rr * d.Px + x] + d.v[idx] + d.gsh[idx];
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
      for (int x = 0; x < d.nx; ++x) acc = cmacc(acc, g[rr * d.Px + x], __ldg(&d.wx[jx * d.nx + x]));
      d.T2[((size_t)p * d.ny + y0 + rr) * d.kx + jx] = acc;
    }
  }
}

// analysis along y: out[p][jy][jx] = sum_y conj(wy[jy][y]) T2[p][y][jx]; one CTA per (jy, p),
// eight warps over interleaved y, lanes over jx (kx <= 64)
__global__ void __launch_bounds__(256) k_ana_y(Dev d, const float2* T2, float2* out, int* step_inc) {
  ph_ana_y(d, blockIdx.x, blockIdx.y, T2, out);
  if (step_inc && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *step_inc += 1;
}

// terms[6] = L, State, Data, Bound, TV, Bridge from the partial sums
// Data residual through the folded operator (Eq. 16 with J = Phi alpha, Eq. 9) as a tiled
// product: block (rb, pb, s) computes the partial sums over coefficients j in chunk s of
// sum_j gsf[r][j] alpha[p][j] for 32 receivers x 8 incidences (one output per thread), staging
// 64-coefficient slices of both operands in shared memory; k_gsf_reduce adds the chunks in order.
__global__ void __launch_bounds__(256) k_gsf_fwd(Dev d, const float2* __restrict__ alpha, float2* __restrict__ part,
                                                 int kc) {
  __shared__ float2 sG[32][65];
  __shared__ float2 sA[8][64];
  const int NA = d.ky * d.kx;
  const int ri = threadIdx.x & 31, pi = threadIdx.x >> 5;
  const int r = blockIdx.x * 32 + ri, p = blockIdx.y * 8 + pi;
  const int j0 = blockIdx.z * kc, j1 = min(j0 + kc, NA);
  float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
  for (int c0 = j0; c0 < j1; c0 += 64) {
    __syncthreads();
    for (int i = threadIdx.x; i < 32 * 64; i += 256) {
      const int rr = i >> 6, jj = i & 63, rg = blockIdx.x * 32 + rr, jg = c0 + jj;
      sG[rr][jj] = (rg < d.nr && jg < j1) ? __ldg(&d.gsf[(size_t)rg * NA + jg]) : make_float2(0.f, 0.f);
    }
    for (int i = threadIdx.x; i < 8 * 64; i += 256) {
      const int pp = i >> 6, jj = i & 63, pg = blockIdx.y * 8 + pp, jg = c0 + jj;
      sA[pp][jj] = (pg < d.ni && jg < j1) ? __ldg(&alpha[(size_t)pg * NA + jg]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 8
    for (int jj = 0; jj < 64; jj += 2) {
      a0 = cmac(a0, sG[ri][jj], sA[pi][jj]);
      a1 = cmac(a1, sG[ri][jj + 1], sA[pi][jj + 1]);
    }
  }
  if (r < d.nr && p < d.ni) part[((size_t)blockIdx.z * d.ni + p) * d.nr + r] = a0 + a1;
}

// r_d[o] = sum of the nsplit chunk partials (float-float, chunk order) - E_sca[o]; per-block
// float-float sums of |r_d|^2 to lp[block].
__global__ void __launch_bounds__(256) k_gsf_reduce(Dev d, const float2* __restrict__ part, int nsplit,
                                                    const float2* __restrict__ esca, float2* __restrict__ rd, FF* lp) {
  __shared__ FF red_gf[32];
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const int nout = d.ni * d.nr;
  FF a2 = FF{0.f, 0.f};
  if (o < nout) {
    FF sx = FF{0.f, 0.f}, sy = FF{0.f, 0.f};
    for (int s = 0; s < nsplit; ++s) {
      const float2 v = part[(size_t)s * nout + o];
      sx = ff_add(sx, v.x);
      sy = ff_add(sy, v.y);
    }
    sx = ff_add(sx, -esca[o].x);
    sy = ff_add(sy, -esca[o].y);
    const float2 v = make_float2(sx.hi + sx.lo, sy.hi + sy.lo);
    rd[o] = v;
    a2 = ff_make(cabs2(v));
  }
  const FF t = ff_block_sum(a2, red_gf);
  if (lp && threadIdx.x == 0) lp[blockIdx.x] = t;
}

// Adjoint data term on the coefficients: g[p][j] += (2 / ||E_sca||^2) sum_r conj(gsf[r][j]) r_d[p][r],
// tiled as 32 coefficients x 8 incidences per block with 32-receiver slices in shared memory.
__global__ void __launch_bounds__(256) k_gsf_adj(Dev d, const float2* __restrict__ rd, float2* __restrict__ g) {
  __shared__ float2 sG[32][33];
  __shared__ float2 sR[8][32];
  const int NA = d.ky * d.kx;
  const int ji = threadIdx.x & 31, pi = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + ji, p = blockIdx.y * 8 + pi;
  float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
  for (int r0 = 0; r0 < d.nr; r0 += 32) {
    __syncthreads();
    for (int i = threadIdx.x; i < 32 * 32; i += 256) {
      const int rr = i >> 5, jj = i & 31, rg = r0 + rr, jg = blockIdx.x * 32 + jj;
      sG[rr][jj] = (rg < d.nr && jg < NA) ? __ldg(&d.gsf[(size_t)rg * NA + jg]) : make_float2(0.f, 0.f);
    }
    {
      const int pp = threadIdx.x >> 5, rr = threadIdx.x & 31, pg = blockIdx.y * 8 + pp, rg = r0 + rr;
      sR[pp][rr] = (pg < d.ni && rg < d.nr) ? rd[(size_t)pg * d.nr + rg] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < 32; rr += 2) {
      a0 = cmacc(a0, sR[pi][rr], sG[rr][ji]);
      a1 = cmacc(a1, sR[pi][rr + 1], sG[rr + 1][ji]);
    }
  }
  if (j < NA && p < d.ni) {
    const size_t i = (size_t)p * NA + j;
    g[i] = g[i] + d.invn[1] * (a0 + a1);
  }
}

// coefficient chunk length and count of the tiled forward product (the partials reuse the
// split-K buffer of the unfolded G_S product, [n_gs_chunks][ni][nr])
static int gsf_kc(const Dev& d) {
  const int NA = d.ky * d.kx;
  const int s = std::max(1, std::min((NA + 63) / 64, d.n_gs_chunks));
  return ((NA + s - 1) / s + 63) / 64 * 64;
}
static int gsf_nsplit(const Dev& d) { return (d.ky * d.kx + gsf_kc(d) - 1) / gsf_kc(d); }

// Analysis along y (second half of Phi^H): out[p][jy][jx] = sum_y T2[p][y][jx] conj(Wy[jy][y]).
// Block (p, jy group of 8) stages T2[p] and the 8 rows of Wy in shared memory; warp jl owns
// coefficient row jy = 8 blockIdx.y + jl, its lanes the jx (kx <= 64).
__global__ void __launch_bounds__(256) k_ana_y_sm(Dev d, const float2* __restrict__ T2, float2* __restrict__ out,
                                                  int* step_inc) {
  extern __shared__ float2 smy[];
  const int p = blockIdx.x, jl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the Adam step counter of a solve-loop evaluation (no k_finalize there); nothing before the
  // Adam step that follows reads it
  if (step_inc && p == 0 && blockIdx.y == 0 && threadIdx.x == 0) *step_inc += 1;
  const int ny = d.ny, kx = d.kx, jy0 = blockIdx.y * 8;
  float2* Ts = smy;                 // [ny][kx]
  float2* Ws = smy + ny * kx;       // [8][ny]
  const float2* T = T2 + (size_t)p * ny * kx;
  for (int i = threadIdx.x; i < ny * kx; i += blockDim.x) Ts[i] = T[i];
  for (int i = threadIdx.x; i < 8 * ny; i += blockDim.x) {
    const int a = i / ny, y = i - a * ny;
    Ws[i] = jy0 + a < d.ky ? d.wy[(size_t)(jy0 + a) * ny + y] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int jy = jy0 + jl;
  if (jy >= d.ky) return;
  float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
  const float2* w = Ws + jl * ny;
  if (kx <= 32) {                                   // four chains over y mod 4, then combined
    float2 b[4] = {a0, a0, a0, a0};
    int y = 0;
    for (; y + 3 < ny; y += 4)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (lane < kx) b[q] = cmacc(b[q], Ts[(y + q) * kx + lane], w[y + q]);
    for (; y < ny; ++y)
      if (lane < kx) b[0] = cmacc(b[0], Ts[y * kx + lane], w[y]);
    a0 = (b[0] + b[1]) + (b[2] + b[3]);
  } else {
#pragma unroll 4
    for (int y = 0; y < ny; ++y) {
      const float2 wv = w[y];
      if (lane < kx) a0 = cmacc(a0, Ts[y * kx + lane], wv);
      if (lane + 32 < kx) a1 = cmacc(a1, Ts[y * kx + lane + 32], wv);
    }
  }
  float2* o = out + ((size_t)p * d.ky + jy) * kx;
  if (lane < kx) o[lane] = a0;
  if (lane + 32 < kx) o[lane + 32] = a1;
}

__device__ __forceinline__ void cp_async8_g(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit_g() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_g() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// y-analysis with its operands staged in one round (cp.async): CTA (p, coefficient rows jy0 ..
// jy0 + 7) copies T2[p] [ny][kx] and the 8 rows of Wy into shared memory, then warp w accumulates,
// lanes over jx (kx <= 32), out[p][jy][jx] = sum_y T2[p][y][jx] conj(Wy[jy][y]) over y = w, w + 8,
// ...; the eight warps' partial sums are added in warp order.  Advances the Adam step counter
// inside the solve loop, as k_ana_y_sm does.
__global__ void __launch_bounds__(256) k_ana_y_cp(Dev d, const float2* __restrict__ T2, float2* __restrict__ out,
                                                  int* step_inc) {
  extern __shared__ float2 smg[];
  const int p = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ny = d.ny, kx = d.kx, jy0 = blockIdx.y * 8;
  const int nj = min(8, d.ky - jy0);
  float2* ts = smg;                        // [ny][kx] T2[p]
  float2* ws = ts + ny * kx;               // [8][ny]  Wy rows jy0 ..
  float2* part = ws + 8 * ny;              // [8 warps][8 rows][32]
  if (step_inc && p == 0 && blockIdx.y == 0 && threadIdx.x == 0) *step_inc += 1;
  const float2* T = T2 + (size_t)p * ny * kx;
  for (int i = threadIdx.x; i < ny * kx; i += blockDim.x) cp_async8_g(&ts[i], &T[i]);
  const float2* W = d.wy + (size_t)jy0 * ny;
  for (int i = threadIdx.x; i < nj * ny; i += blockDim.x) cp_async8_g(&ws[i], &W[i]);
  cp_async_commit_g();
  cp_async_wait_all_g();
  __syncthreads();
  float2 acc[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) acc[a] = make_float2(0.f, 0.f);
  if (lane < kx) {
#pragma unroll 4
    for (int y = warp; y < ny; y += 8) {
      const float2 t = ts[y * kx + lane];
#pragma unroll
      for (int a = 0; a < 8; ++a)
        if (a < nj) acc[a] = cmacc(acc[a], t, ws[a * ny + y]);
    }
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) part[(warp * 8 + a) * 32 + lane] = acc[a];
  __syncthreads();
  const int a = warp, jx = lane;
  if (a < nj && jx < kx) {
    float2 sum = part[a * 32 + jx];
    for (int w = 1; w < 8; ++w) sum = sum + part[(w * 8 + a) * 32 + jx];
    out[(size_t)p * d.ky * kx + (size_t)(jy0 + a) * kx + jx] = sum;
  }
}
static size_t sm_ana_y_cp(const Dev& d) { return ((size_t)d.ny * d.kx + 8 * (size_t)d.ny + 8 * 8 * 32) * sizeof(float2); }
static bool ana_y_cp_ok(const Dev& d) { return d.kx <= 32 && sm_ana_y_cp(d) <= 100 * 1024; }

// Adjoint data term on the coefficients with its operands staged in one round (cp.async): CTA
// (32 coefficients j0 .., 16 incidences p0 ..) copies gsf[r][j0 .. j0 + 31] for every receiver and
// r_d[p0 .. p0 + 15][r] (rows padded to an even length), then thread (j, q), q < 8, adds
// g[p][j] += (2 / ||E_sca||^2) sum_r r_d[p][r] conj(gsf[r][j]) for p = p0 + q and p0 + q + 8 (two
// chains each, over even and odd r, one 16-byte broadcast load per receiver pair and incidence).
#define GSA_P 16
__global__ void __launch_bounds__(GSA_P * 16) k_gsf_adj_cp(Dev d, const float2* __restrict__ rd, float2* __restrict__ g) {
  pdl_wait();
  extern __shared__ float4 sma4[];
  const int NA = d.ky * d.kx, nr = d.nr, nre = (nr + 1) & ~1;
  const int j0 = blockIdx.x * 32, p0 = blockIdx.y * GSA_P;
  const int nj = min(32, NA - j0), np = min(GSA_P, d.ni - p0);
  float2* rs = reinterpret_cast<float2*>(sma4);  // [GSA_P][nre]
  float2* gs = rs + GSA_P * nre;                 // [nre][32]
  for (int i = threadIdx.x; i < nre * 32; i += blockDim.x) {
    const int r = i >> 5, jj = i & 31;
    if (jj < nj && r < nr) cp_async8_g(&gs[i], &d.gsf[(size_t)r * NA + j0 + jj]);
    else gs[i] = make_float2(0.f, 0.f);
  }
  for (int i = threadIdx.x; i < GSA_P * nre; i += blockDim.x) {
    const int pp = i / nre, r = i - pp * nre;
    if (pp < np && r < nr) cp_async8_g(&rs[i], &rd[(size_t)(p0 + pp) * nr + r]);
    else rs[i] = make_float2(0.f, 0.f);
  }
  cp_async_commit_g();
  cp_async_wait_all_g();
  __syncthreads();
  const int jj = threadIdx.x & 31, q = threadIdx.x >> 5;
  float2 a0 = make_float2(0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
  const float4* ra = reinterpret_cast<const float4*>(rs + q * nre);
  const float4* rb = reinterpret_cast<const float4*>(rs + (q + GSA_P / 2) * nre);
#pragma unroll 4
  for (int r2 = 0; r2 < nre / 2; ++r2) {
    const float4 u = ra[r2], v = rb[r2];
    const float2 g0 = gs[(2 * r2) * 32 + jj], g1 = gs[(2 * r2 + 1) * 32 + jj];
    a0 = cmacc(a0, make_float2(u.x, u.y), g0);
    a1 = cmacc(a1, make_float2(u.z, u.w), g1);
    b0 = cmacc(b0, make_float2(v.x, v.y), g0);
    b1 = cmacc(b1, make_float2(v.z, v.w), g1);
  }
  if (jj < nj) {
    if (q < np) {
      const size_t i = (size_t)(p0 + q) * NA + j0 + jj;
      g[i] = g[i] + d.invn[1] * (a0 + a1);
    }
    if (q + GSA_P / 2 < np) {
      const size_t i = (size_t)(p0 + q + GSA_P / 2) * NA + j0 + jj;
      g[i] = g[i] + d.invn[1] * (b0 + b1);
    }
  }
}
static size_t sm_gsf_adj_cp(const Dev& d) {
  const size_t nre = (size_t)((d.nr + 1) & ~1);
  return (nre * 32 + GSA_P * nre) * sizeof(float2);
}
static bool gsf_adj_cp_ok(const Dev& d) { return sm_gsf_adj_cp(d) <= 100 * 1024; }


// Data residual through the folded operator: CTA (p, block of 8 receivers), alpha_p in shared
// memory, a warp per receiver (lanes split the coefficients, four independent partial sums, a
// fixed-order warp sum), r_d[p][r] = sum_j gsf[r][j] alpha[p][j] - E_sca[p][r], and the CTA's
// ||r_d||^2 (float-float, warp order) -> lp[p nrb + block].  Replaces k_gsf_fwd + k_gsf_reduce
// where the partials fit (d.rdwarp).
__global__ void __launch_bounds__(256) k_gsf_fwd_p(Dev d, const float2* __restrict__ alpha, float2* __restrict__ rd,
                                                   FF* __restrict__ lp) {
  extern __shared__ float2 sap[];
  __shared__ FF wpart[8];
  const int p = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int NA = d.ky * d.kx, r = blockIdx.y * 8 + warp;
  for (int i = threadIdx.x; i < NA; i += blockDim.x) sap[i] = alpha[(size_t)p * NA + i];
  __syncthreads();
  FF part = FF{0.f, 0.f};
  if (r < d.nr) {
    const float2* gr = d.gsf + (size_t)r * NA;
    float2 a[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    int j = lane;
    for (; j + 96 < NA; j += 128)
#pragma unroll
      for (int q = 0; q < 4; ++q) a[q] = cmac(a[q], __ldg(&gr[j + 32 * q]), sap[j + 32 * q]);
    for (; j < NA; j += 32) a[0] = cmac(a[0], __ldg(&gr[j]), sap[j]);
    float2 acc = (a[0] + a[1]) + (a[2] + a[3]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = acc + make_float2(__shfl_xor_sync(0xffffffffu, acc.x, o),
                                                         __shfl_xor_sync(0xffffffffu, acc.y, o));
    if (lane == 0) {
      const size_t o = (size_t)p * d.nr + r;
      const float2 v = acc - d.esca[o];
      rd[o] = v;
      part = ff_make(cabs2(v));
    }
  }
  if (lane == 0) wpart[warp] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    FF t = FF{0.f, 0.f};
    for (int w = 0; w < 8; ++w) t = ff_add(t, wpart[w]);
    lp[(size_t)p * gridDim.y + blockIdx.y] = t;
  }
}

// the per-receiver-block data residual kernel: folded data term, coefficients that fit in shared
// memory, and one loss partial per (incidence, receiver block) within the partial buffer
bool hp_rdwarp_ok(const Dev& d) {
  return d.fold && d.ky * d.kx <= 4096 && (size_t)d.ni * ((d.nr + 7) / 8) <= PDF_LP_STRIDE;
}

static size_t sm_ana_y(const Dev& d) { return ((size_t)d.ny * d.kx + 8 * (size_t)d.ny) * sizeof(float2); }
static bool ana_y_sm_ok(const Dev& d) { return d.kx <= 64 && sm_ana_y(d) <= 100 * 1024; }


__global__ void k_finalize(Dev d, double* terms, int n_state, int n_data, int n_reg, int* step_inc) {
  ph_finalize(d, terms, n_state, n_data, n_reg, step_inc);
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
size_t sm_gs_bytes(const Dev& d);
size_t sm_gsh_bytes(const Dev& d);
static size_t sm_gsh(const Dev& d) {
  return ((size_t)d.ni * GSH_RT + GSH_RT * (GSH_CHUNK + 1) + 256 * GSH_TP * GSH_TN) * sizeof(float2);
}

size_t sm_gs_bytes(const Dev& d) { return sm_gs(d); }
size_t sm_gsh_bytes(const Dev& d) { return sm_gsh(d); }

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
  cudaFuncSetAttribute(k_ana_y_sm, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  cudaFuncSetAttribute(k_gsf_fwd_p, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  cudaFuncSetAttribute(k_ana_y_cp, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  cudaFuncSetAttribute(k_gsf_adj_cp, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(e, "cudaFuncSetAttribute");
  return PDF_OK;
}

static inline dim3 row_grid(const Dev& d) { return dim3((d.ny + ROWS_PER_CTA - 1) / ROWS_PER_CTA, d.ni); }
static inline dim3 col_grid(const Dev& d) { return dim3((d.Px + COL_CW - 1) / COL_CW, d.ni); }


pdf_status hp_check_limits(const Dev& d) {
  const size_t lim = 200 * 1024;
  if (d.fast && (fp_smem_synth(d) > 100 * 1024 || fp_smem_col(d) > 100 * 1024 || fp_smem_state(d) > 100 * 1024 ||
                 fp_smem_ana(d) > 100 * 1024 || fp_smem_sums(d) > 100 * 1024))
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

static const char* kLossGradKernelsFold[] = {
    "k_synth_rowfft", "k_colconv", "k_rowifft_state", "k_gsf_fwd", "k_reg", "k_adj_rowfft",
    "k_colconv(conj)", "k_adj_rowifft_ana", "k_ana_y", "k_gsf_adj", "k_finalize"};
static const char* kLossGradStagesTCFold[] = {
    "tc_synth(synth1+gemm+post)", "k_colconv", "k_rowifft_state", "k_gsf_fwd", "k_reg", "k_adj_rowfft",
    "k_colconv(conj)", "tc_adj(rowifft+gemm)", "k_ana_y", "k_gsf_adj", "k_finalize"};
// folded data term with the residual inside the tiled synthesis
static const char* kLossGradKernelsFused[] = {
    "k_synth_rowfft+k_gsf_fwd", "k_colconv", "k_rowifft_state", "k_reg", "k_adj_rowfft",
    "k_colconv(conj)", "k_adj_rowifft_ana", "k_ana_y", "k_gsf_adj", "k_finalize"};

int hp_kernels_per_loss_grad(const pdf_problem* h) {
  const Dev& d = h->d;
  if (!d.fold) return h->tc ? 11 : 12;
  return d.rd_synth ? 10 : 11;
}

const char* hp_kernel_name(int k, int precision, int fold, int rd_synth) {
  if (fold && rd_synth) return (k >= 0 && k < 10) ? kLossGradKernelsFused[k] : "";
  if (fold) {
    if (k < 0 || k >= 11) return "";
    return precision == 1 ? kLossGradStagesTCFold[k] : kLossGradKernelsFold[k];
  }
  if (precision == 1) return (k >= 0 && k < 11) ? kLossGradStagesTC[k] : "";
  return (k >= 0 && k < 12) ? kLossGradKernels[k] : "";
}

pdf_status hp_loss_grad(pdf_problem* h, const float2* alpha, float2* grad, double* terms, cudaStream_t st,
                        int* step_inc, cudaEvent_t* ev) {
  Dev& d = h->d;
  const int nout = d.ni * d.nr;
  const int n_data_blocks = (nout + 255) / 256;
  const bool tc = h->tc != nullptr;
  // an evaluation inside the solve loop (an Adam step counter, no loss terms wanted): the loss
  // partials are not summed (no k_finalize) and the y-analysis advances the step counter
  const bool loop_eval = step_inc != nullptr && terms == nullptr && ev == nullptr;
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
    if ((s = fp_synth_rowfft(d, alpha, d.J, 1, st, d.rd_synth)) != PDF_OK) return s;
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
  if (d.rd_synth) {
    // formed by the synthesis tiles
  } else if (d.rdwarp) {
    k_gsf_fwd_p<<<dim3(d.ni, (d.nr + 7) / 8), 256, sizeof(float2) * d.ky * d.kx, st>>>(d, alpha, d.rd,
                                                                                       d.lpart + LP_DATA * PDF_LP_STRIDE);
  } else if (d.fold) {
    k_gsf_fwd<<<dim3((d.nr + 31) / 32, (d.ni + 7) / 8, gsf_nsplit(d)), 256, 0, st>>>(d, alpha, d.gspart, gsf_kc(d));
    k_gsf_reduce<<<n_data_blocks, 256, 0, st>>>(d, d.gspart, gsf_nsplit(d), d.esca, d.rd,
                                                 d.lpart + LP_DATA * PDF_LP_STRIDE);
  } else if (tc) {
    if ((s = tc_gs_fwd(h, nullptr, d.esca, d.rd, d.lpart + LP_DATA * PDF_LP_STRIDE, 1, st)) != PDF_OK) return s;
  } else {
    k_gs_partial<<<d.n_gs_chunks, 256, sm_gs(d), st>>>(d, d.J, d.gspart);
    mark();
    k_gs_reduce<<<n_data_blocks, 256, 0, st>>>(d, d.gspart, d.n_gs_chunks, d.esca, d.rd,
                                                d.lpart + LP_DATA * PDF_LP_STRIDE);
  }
  if (!d.rd_synth) mark();
  if (d.cco_loss) {
    if ((s = cc_reg(d, st)) != PDF_OK) return s;
    pdf_count_launch(CCO_LOSS_KERNELS - 1);
  } else {
    if (reg_tile_ok(d))
      launch_pdl(k_reg_tile, reg_tile_grid(d), RT_THREADS, 0, st, d);
    else
      launch_pdl(k_reg, d.n_reg_blocks, 128, 0, st, d);
  }
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
    if (!d.fold) {
      if ((s = tc_gsh(h, nullptr, 1, st)) != PDF_OK) return s;
      mark();
    }
    if ((s = tc_adj_ana(h, st)) != PDF_OK) return s;
    T2 = (const float2*)h->tc->c_ana;
  } else {
    if (!d.fold) {
      k_gsh<<<(d.M + GSH_CHUNK - 1) / GSH_CHUNK, 256, sm_gsh(d), st>>>(d, d.rd, d.gsh, 0.f, 1);
      mark();
    }
    if (d.fast) {
      if ((s = fp_adj_rowifft_ana(d, nullptr, 0, st)) != PDF_OK) return s;
    } else {
      k_adj_rowifft_ana<<<row_grid(d), ROW_THREADS, sm_row(d), st>>>(d, nullptr, 0);
    }
  }
  mark();
  float2* g = grad ? grad : h->grad;
  if (fp_ana_y_fft(d, T2, g, loop_eval ? step_inc : nullptr, st)) {
  } else if (ana_y_cp_ok(d))
    k_ana_y_cp<<<dim3(d.ni, (d.ky + 7) / 8), 256, sm_ana_y_cp(d), st>>>(d, T2, g, loop_eval ? step_inc : nullptr);
  else if (ana_y_sm_ok(d))
    k_ana_y_sm<<<dim3(d.ni, (d.ky + 7) / 8), 256, sm_ana_y(d), st>>>(d, T2, g, loop_eval ? step_inc : nullptr);
  else
    k_ana_y<<<dim3(d.ky, d.ni), 256, 0, st>>>(d, T2, g, loop_eval ? step_inc : nullptr);
  mark();
  if (d.fold) {
    if (gsf_adj_cp_ok(d))
      launch_pdl(k_gsf_adj_cp, dim3((d.ky * d.kx + 31) / 32, (d.ni + GSA_P - 1) / GSA_P), GSA_P * 16, sm_gsf_adj_cp(d), st, d,
                 (const float2*)d.rd, g);
    else
      k_gsf_adj<<<dim3((d.ky * d.kx + 31) / 32, (d.ni + 7) / 8), 256, 0, st>>>(d, d.rd, g);
    mark();
  }
  if (!loop_eval) {
    const int n_data = d.rd_synth ? d.ni * fp_synth2p_tpi(d) : d.rdwarp ? d.ni * ((d.nr + 7) / 8) : n_data_blocks;
    k_finalize<<<1, 1024, 0, st>>>(d, terms ? terms : h->terms, d.fast ? fp_n_state(d) : d.ny, n_data,
                                  reg_tile_ok(d) && !d.cco_loss ? (int)(reg_tile_grid(d).x * reg_tile_grid(d).y)
                                                                 : d.n_reg_blocks,
                                  step_inc);
    mark();
  }
  pdf_count_launch((d.fold ? (tc ? 10 : 12) : (tc ? 7 : 12)) - (loop_eval ? 1 : 0) - (d.rdwarp ? 1 : 0) -
                   (d.rd_synth ? 1 : 0));
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
  if (ana_y_sm_ok(d))
    k_ana_y_sm<<<dim3(d.ni, (d.ky + 7) / 8), 256, sm_ana_y(d), st>>>(d, T2, out, nullptr);
  else
    k_ana_y<<<dim3(d.ky, d.ni), 256, 0, st>>>(d, T2, out, nullptr);
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
