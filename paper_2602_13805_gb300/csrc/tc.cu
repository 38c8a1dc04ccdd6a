// Split-BF16 tensor-core contractions of the hot path (precision = 1): operand packing,
// GEMM launches and the consumers of their fp32 outputs.  See tc.cuh for the embeddings.
#include <algorithm>

#include "fft.cuh"
#include "phases.cuh"
#include "problem.cuh"
#include "tc.cuh"

__device__ __forceinline__ void put_split(__nv_bfloat16* hi, __nv_bfloat16* lo, size_t i, float x) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  hi[i] = h;
  lo[i] = __float2bfloat16_rn(x - __bfloat162float(h));
}

static int round64(int k) { return (k + 63) / 64 * 64; }

// ---------------------------------------------------------------------------
// setup-time operand packing
// ---------------------------------------------------------------------------
// GSA[r][2n + c] and GST[n][2r + c] from G_S [nr][M] (c = 0: Re, 1: Im)
__global__ void k_tc_pack_gs(Dev d, TC t) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (n >= d.M) return;
  const float2 g = d.gs[(size_t)r * d.M + n];
  put_split(t.gsa_hi, t.gsa_lo, (size_t)r * t.K2M + 2 * n, g.x);
  put_split(t.gsa_hi, t.gsa_lo, (size_t)r * t.K2M + 2 * n + 1, g.y);
  put_split(t.gst_hi, t.gst_lo, (size_t)n * t.K2R + 2 * r, g.x);
  put_split(t.gst_hi, t.gst_lo, (size_t)n * t.K2R + 2 * r + 1, g.y);
}

// WYA[y][2 jy + c] = Wy[jy][y];  WXB[2 jx][2x + c] = (Re, Im) Wx[jx][x], WXB[2 jx + 1][2x + c] = (-Im, Re)
__global__ void k_tc_pack_w(Dev d, TC t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < d.ky * d.ny) {
    const int jy = i / d.ny, y = i - jy * d.ny;
    const float2 w = d.wy[(size_t)jy * d.ny + y];
    put_split(t.wya_hi, t.wya_lo, (size_t)y * t.KYP + 2 * jy, w.x);
    put_split(t.wya_hi, t.wya_lo, (size_t)y * t.KYP + 2 * jy + 1, w.y);
  }
  if (i < d.kx * d.nx) {
    const int jx = i / d.nx, x = i - jx * d.nx;
    const float2 w = d.wx[(size_t)jx * d.nx + x];
    put_split(t.wxb_hi, t.wxb_lo, (size_t)(2 * jx) * t.KXP + 2 * x, w.x);
    put_split(t.wxb_hi, t.wxb_lo, (size_t)(2 * jx) * t.KXP + 2 * x + 1, w.y);
    put_split(t.wxb_hi, t.wxb_lo, (size_t)(2 * jx + 1) * t.KXP + 2 * x, -w.y);
    put_split(t.wxb_hi, t.wxb_lo, (size_t)(2 * jx + 1) * t.KXP + 2 * x + 1, w.x);
  }
}

// ---------------------------------------------------------------------------
// per-iteration packing and consumers
// ---------------------------------------------------------------------------
// T[p][jy][x] = sum_jx alpha[p][jy][jx] Wx[jx][x] -> TB rows 2(p nx + x) (Re T, -Im T) and +1 (Im T, Re T);
// one thread per (x, jy), grid (x blocks, ky, ni)
__global__ void __launch_bounds__(128) k_tc_synth1(Dev d, TC t, const float2* __restrict__ alpha) {
  const int p = blockIdx.z, jy = blockIdx.y;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= d.nx) return;
  const float2* a = alpha + ((size_t)p * d.ky + jy) * d.kx;
  float2 acc = make_float2(0.f, 0.f);
  for (int jx = 0; jx < d.kx; ++jx) acc = cmac(acc, __ldg(&a[jx]), __ldg(&d.wx[(size_t)jx * d.nx + x]));
  const size_t r0 = (size_t)(2 * (p * d.nx + x)) * t.KYP, r1 = r0 + t.KYP;
  put_split(t.tb_hi, t.tb_lo, r0 + 2 * jy, acc.x);
  put_split(t.tb_hi, t.tb_lo, r0 + 2 * jy + 1, -acc.y);
  put_split(t.tb_hi, t.tb_lo, r1 + 2 * jy, acc.y);
  put_split(t.tb_hi, t.tb_lo, r1 + 2 * jy + 1, acc.x);
}

__device__ __forceinline__ void put_jb(const TC& t, int p, int n, float2 J) {
  const size_t r0 = (size_t)(2 * p) * t.K2M, r1 = r0 + t.K2M;
  put_split(t.jb_hi, t.jb_lo, r0 + 2 * n, J.x);
  put_split(t.jb_hi, t.jb_lo, r0 + 2 * n + 1, -J.y);
  put_split(t.jb_hi, t.jb_lo, r1 + 2 * n, J.y);
  put_split(t.jb_hi, t.jb_lo, r1 + 2 * n + 1, J.x);
}

// J from the synthesis GEMM output C_syn[y][2(p nx + x) + c]; writes J, JB and (optionally) the
// padded row DFT of J into A.
__global__ void __launch_bounds__(ROW_THREADS) k_tc_synth_post(Dev d, TC t, float2* __restrict__ Jout, int do_fft) {
  extern __shared__ float2 sm[];
  const int p = blockIdx.y, y0 = blockIdx.x * ROWS_PER_CTA;
  const int nrow = min(ROWS_PER_CTA, d.ny - y0);
  float2* b0 = sm;
  float2* b1 = sm + ROWS_PER_CTA * d.Px;
  const float2* cs = (const float2*)t.c_syn;
  const int ncs = d.ni * d.nx;                       // complex columns of C_syn
  for (int i = threadIdx.x; i < ROWS_PER_CTA * d.Px; i += blockDim.x) {
    const int rr = i / d.Px, x = i - rr * d.Px;
    float2 v = make_float2(0.f, 0.f);
    if (rr < nrow && x < d.nx) {
      const int y = y0 + rr;
      v = cs[(size_t)y * ncs + p * d.nx + x];
      Jout[((size_t)p * d.ny + y) * d.nx + x] = v;
      if (!d.fold) put_jb(t, p, y * d.nx + x, v);       // G_S GEMM operand (unfolded data term)
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

// Register-FFT form of the synthesis epilogue: one warp per row of C_syn -> J (and JB when the
// data term is unfolded), then the padded row DFT straight into A (no J round trip).
template <int PX>
__global__ void __launch_bounds__(FT) k_tc_synth_post_fast(Dev d, TC t, float2* __restrict__ Jout) {
  constexpr int R = PX / 32;
  __shared__ float2 tw[PX];
  const int p = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int y = blockIdx.x * FW + warp;
  load_tw<PX>(tw, d.twx);
  __syncthreads();
  if (y >= d.ny) return;
  const float2* cs = (const float2*)t.c_syn + (size_t)y * d.ni * d.nx + (size_t)p * d.nx;
  const size_t row = (size_t)p * d.ny + y;
  float2 v[R];
#pragma unroll
  for (int m = 0; m < R; ++m) {
    const int x = lane + 32 * m;
    v[m] = make_float2(0.f, 0.f);
    if (2 * m < R && x < d.nx) {                       // slots m >= R/2 are padding (P >= 2 nx)
      v[m] = cs[x];
      Jout[row * d.nx + x] = v[m];
      if (!d.fold) put_jb(t, p, y * d.nx + x, v[m]);
    }
  }
  WarpFFT<PX>::forward(v, tw, lane);
#pragma unroll
  for (int k = 0; k < R; ++k) d.A[row * PX + k * 32 + lane] = v[k];
}

__global__ void k_tc_field_to_jb(Dev d, TC t, const float2* __restrict__ X) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)d.ni * d.M) return;
  const int p = (int)(i / d.M), n = (int)(i - (size_t)p * d.M);
  put_jb(t, p, n, X[i]);
}

__device__ __forceinline__ void put_rdb(const TC& t, int p, int r, float2 v) {
  const size_t r0 = (size_t)(2 * p) * t.K2R, r1 = r0 + t.K2R;
  put_split(t.rdb_hi, t.rdb_lo, r0 + 2 * r, v.x);
  put_split(t.rdb_hi, t.rdb_lo, r0 + 2 * r + 1, v.y);
  put_split(t.rdb_hi, t.rdb_lo, r1 + 2 * r, v.y);
  put_split(t.rdb_hi, t.rdb_lo, r1 + 2 * r + 1, -v.x);
}

// out[p][r] = sum over splits (FP64) of C_fwd - sub; ||out||^2 per block -> lp; optional RDB packing
__global__ void k_tc_gs_reduce(Dev d, TC t, int nsplit, const float2* __restrict__ sub, float2* __restrict__ out,
                               FF* __restrict__ lp, int write_rdb) {
  __shared__ FF red[32];
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  FF a2 = FF{0.f, 0.f};
  if (o < d.ni * d.nr) {
    const int p = o / d.nr, r = o - p * d.nr;
    const size_t stride = (size_t)d.nr * 2 * d.ni;
    FF sx = FF{0.f, 0.f}, sy = FF{0.f, 0.f};
    for (int s = 0; s < nsplit; ++s) {
      const float* c = t.c_fwd + s * stride + (size_t)r * 2 * d.ni + 2 * p;
      sx = ff_add(sx, c[0]);
      sy = ff_add(sy, c[1]);
    }
    if (sub) {
      sx = ff_add(sx, -sub[o].x);
      sy = ff_add(sy, -sub[o].y);
    }
    const float2 v = make_float2(sx.hi + sx.lo, sy.hi + sy.lo);
    out[o] = v;
    if (write_rdb) put_rdb(t, p, r, v);
    a2 = ff_make(cabs2(v));
  }
  if (lp) {
    const FF tt = ff_block_sum(a2, red);
    if (threadIdx.x == 0) lp[blockIdx.x] = tt;
  }
}

__global__ void k_tc_d_to_rdb(Dev d, TC t, const float2* __restrict__ D) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= d.ni * d.nr) return;
  put_rdb(t, o / d.nr, o % d.nr, D[o]);
}

// out[p][n] = scale * (C_adj[n][2p], C_adj[n][2p + 1])
__global__ void k_tc_cadj_to_field(Dev d, TC t, float2* __restrict__ out, float scale) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)d.ni * d.M) return;
  const int p = (int)(i / d.M), n = (int)(i - (size_t)p * d.M);
  const float* c = t.c_adj + (size_t)n * 2 * d.ni + 2 * p;
  out[i] = make_float2(scale * c[0], scale * c[1]);
}

__device__ __forceinline__ void put_gja(const TC& t, int row, int x, float2 g) {
  const size_t r0 = (size_t)row * t.KXP;
  put_split(t.gja_hi, t.gja_lo, r0 + 2 * x, g.x);
  put_split(t.gja_hi, t.gja_lo, r0 + 2 * x + 1, g.y);
}

// inverse row DFT of A (G_D^H u), + v + (2/||E_sca||^2) G_S^H r_d from C_adj, packed as the
// analysis GEMM's A operand (rows p ny + y).
__global__ void __launch_bounds__(ROW_THREADS) k_tc_adj_rowifft(Dev d, TC t) {
  extern __shared__ float2 sm[];
  const int p = blockIdx.y, y0 = blockIdx.x * ROWS_PER_CTA;
  const int nrow = min(ROWS_PER_CTA, d.ny - y0);
  float2* b0 = sm;
  float2* b1 = sm + ROWS_PER_CTA * d.Px;
  const float ks = d.invn[1];
  for (int i = threadIdx.x; i < ROWS_PER_CTA * d.Px; i += blockDim.x) {
    const int rr = i / d.Px, x = i - rr * d.Px;
    b0[i] = rr < nrow ? d.A[((size_t)p * d.ny + y0 + rr) * d.Px + x] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float2* g = fft_lines(b0, b1, ROWS_PER_CTA, d.Px, d.plx, d.twx, true);
  for (int i = threadIdx.x; i < ROWS_PER_CTA * d.nx; i += blockDim.x) {
    const int rr = i / d.nx, x = i - rr * d.nx;
    if (rr < nrow) {
      const int n = (y0 + rr) * d.nx + x;
      const size_t idx = (size_t)p * d.M + n;
      const float* c = t.c_adj + (size_t)n * 2 * d.ni + 2 * p;
      const float2 v = d.fold ? g[rr * d.Px + x] + d.v[idx] : g[rr * d.Px + x] + d.v[idx] + make_float2(ks * c[0], ks * c[1]);
      put_gja(t, p * d.ny + y0 + rr, x, v);
    }
  }
}

// fast-path form: g = G_D^H u (already inverse-transformed into gdh) + v + G_S^H term -> GJA
__global__ void k_tc_gja_combine(Dev d, TC t, const float2* __restrict__ gdh) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)d.ni * d.M) return;
  const int p = (int)(i / d.M), n = (int)(i - (size_t)p * d.M);
  const int y = n / d.nx, x = n - y * d.nx;
  const float ks = d.invn[1];
  const float* c = t.c_adj + (size_t)n * 2 * d.ni + 2 * p;
  put_gja(t, p * d.ny + y, x, d.fold ? gdh[i] + d.v[i] : gdh[i] + d.v[i] + make_float2(ks * c[0], ks * c[1]));
}

// Register-FFT form of the adjoint packing: inverse row DFT of A (G_D^H u) + v (+ the G_S^H
// term when unfolded), packed straight into the analysis GEMM's A operand.
template <int PX>
__global__ void __launch_bounds__(FT) k_tc_adj_fast(Dev d, TC t) {
  constexpr int R = PX / 32;
  __shared__ float2 tw[PX];
  const int p = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int y = blockIdx.x * FW + warp;
  load_tw<PX>(tw, d.twx);
  __syncthreads();
  if (y >= d.ny) return;
  const size_t row = (size_t)p * d.ny + y;
  const float ks = d.invn[1];
  float2 v[R];
#pragma unroll
  for (int k = 0; k < R; ++k) v[k] = d.A[row * PX + k * 32 + lane];
  WarpFFT<PX>::inverse(v, tw, lane);
#pragma unroll
  for (int m = 0; m < R; ++m) {
    const int x = lane + 32 * m;
    if (2 * m < R && x < d.nx) {
      const int n = y * d.nx + x;
      const size_t idx = row * d.nx + x;
      float2 g = v[m] + d.v[idx];
      if (!d.fold) {
        const float* c = t.c_adj + (size_t)n * 2 * d.ni + 2 * p;
        g = g + make_float2(ks * c[0], ks * c[1]);
      }
      put_gja(t, p * d.ny + y, x, g);
    }
  }
}

__global__ void k_tc_field_to_gja(Dev d, TC t, const float2* __restrict__ X) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)d.ni * d.M) return;
  const int p = (int)(i / d.M), n = (int)(i - (size_t)p * d.M);
  const int y = n / d.nx, x = n - y * d.nx;
  put_gja(t, p * d.ny + y, x, X[i]);
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
static size_t sm_row_tc(const Dev& d) { return 2 * ROWS_PER_CTA * (size_t)d.Px * sizeof(float2); }

pdf_status tc_setup(pdf_problem* h, cudaStream_t st) {
  Dev& d = h->d;
  TC* t = new TC();
  h->tc = t;
  t->K2M = round64(2 * d.M);
  t->K2R = round64(2 * d.nr);
  t->KYP = round64(2 * d.ky);
  t->KXP = round64(2 * d.nx);
  const int kb = umma_kblocks(t->K2M);
  t->nsplit_fwd = std::max(1, std::min(148, kb / 4));
  {
    const int per = (kb + t->nsplit_fwd - 1) / t->nsplit_fwd;
    t->nsplit_fwd = (kb + per - 1) / per;
  }
  pdf_status s;
#define WS(ptr, n) \
  if ((s = ws_alloc(h, (void**)&(ptr), (size_t)(n) * sizeof(*(ptr)))) != PDF_OK) return s
  WS(t->gsa_hi, (size_t)d.nr * t->K2M);
  WS(t->gsa_lo, (size_t)d.nr * t->K2M);
  WS(t->gst_hi, (size_t)d.M * t->K2R);
  WS(t->gst_lo, (size_t)d.M * t->K2R);
  WS(t->wya_hi, (size_t)d.ny * t->KYP);
  WS(t->wya_lo, (size_t)d.ny * t->KYP);
  WS(t->wxb_hi, (size_t)2 * d.kx * t->KXP);
  WS(t->wxb_lo, (size_t)2 * d.kx * t->KXP);
  WS(t->jb_hi, (size_t)2 * d.ni * t->K2M);
  WS(t->jb_lo, (size_t)2 * d.ni * t->K2M);
  WS(t->rdb_hi, (size_t)2 * d.ni * t->K2R);
  WS(t->rdb_lo, (size_t)2 * d.ni * t->K2R);
  WS(t->tb_hi, (size_t)2 * d.ni * d.nx * t->KYP);
  WS(t->tb_lo, (size_t)2 * d.ni * d.nx * t->KYP);
  WS(t->gja_hi, (size_t)d.ni * d.ny * t->KXP);
  WS(t->gja_lo, (size_t)d.ni * d.ny * t->KXP);
  WS(t->c_fwd, (size_t)t->nsplit_fwd * d.nr * 2 * d.ni);
  WS(t->c_adj, (size_t)d.M * 2 * d.ni);
  WS(t->c_syn, (size_t)d.ny * 2 * d.ni * d.nx);
  WS(t->c_ana, (size_t)d.ni * d.ny * 2 * d.kx);
  WS(t->err, 1);
#undef WS
  // zero everything once so that the K padding stays zero
  auto z = [&](void* p, size_t bytes) { return cudaMemsetAsync(p, 0, bytes, st); };
  z(t->gsa_hi, (size_t)d.nr * t->K2M * 2);
  z(t->gsa_lo, (size_t)d.nr * t->K2M * 2);
  z(t->gst_hi, (size_t)d.M * t->K2R * 2);
  z(t->gst_lo, (size_t)d.M * t->K2R * 2);
  z(t->wya_hi, (size_t)d.ny * t->KYP * 2);
  z(t->wya_lo, (size_t)d.ny * t->KYP * 2);
  z(t->wxb_hi, (size_t)2 * d.kx * t->KXP * 2);
  z(t->wxb_lo, (size_t)2 * d.kx * t->KXP * 2);
  z(t->jb_hi, (size_t)2 * d.ni * t->K2M * 2);
  z(t->jb_lo, (size_t)2 * d.ni * t->K2M * 2);
  z(t->rdb_hi, (size_t)2 * d.ni * t->K2R * 2);
  z(t->rdb_lo, (size_t)2 * d.ni * t->K2R * 2);
  z(t->tb_hi, (size_t)2 * d.ni * d.nx * t->KYP * 2);
  z(t->tb_lo, (size_t)2 * d.ni * d.nx * t->KYP * 2);
  z(t->gja_hi, (size_t)d.ni * d.ny * t->KXP * 2);
  z(t->gja_lo, (size_t)d.ni * d.ny * t->KXP * 2);
  z(t->err, sizeof(int));
  PDF_LAUNCHED("tensor-core workspace memset");
  k_tc_pack_gs<<<dim3((d.M + 255) / 256, d.nr), 256, 0, st>>>(d, *t);
  const int nw = std::max(d.ky * d.ny, d.kx * d.nx);
  k_tc_pack_w<<<(nw + 255) / 256, 256, 0, st>>>(d, *t);
  pdf_count_launch(2);
  PDF_LAUNCHED("tensor-core operand packing");
  if ((s = umma_operand(&t->gsa, t->gsa_hi, t->gsa_lo, d.nr, t->K2M)) != PDF_OK) return s;
  if ((s = umma_operand(&t->gst, t->gst_hi, t->gst_lo, d.M, t->K2R)) != PDF_OK) return s;
  if ((s = umma_operand(&t->wya, t->wya_hi, t->wya_lo, d.ny, t->KYP)) != PDF_OK) return s;
  if ((s = umma_operand(&t->wxb, t->wxb_hi, t->wxb_lo, 2 * d.kx, t->KXP)) != PDF_OK) return s;
  if ((s = umma_operand(&t->jb, t->jb_hi, t->jb_lo, 2 * d.ni, t->K2M)) != PDF_OK) return s;
  if ((s = umma_operand(&t->rdb, t->rdb_hi, t->rdb_lo, 2 * d.ni, t->K2R)) != PDF_OK) return s;
  if ((s = umma_operand(&t->tb, t->tb_hi, t->tb_lo, 2 * d.ni * d.nx, t->KYP)) != PDF_OK) return s;
  if ((s = umma_operand(&t->gja, t->gja_hi, t->gja_lo, d.ni * d.ny, t->KXP)) != PDF_OK) return s;
  cudaFuncSetAttribute(k_tc_synth_post, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_tc_adj_rowifft, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  return PDF_OK;
}

pdf_status tc_synth(pdf_problem* h, const float2* alpha, float2* Jout, int do_fft, cudaStream_t st) {
  Dev& d = h->d;
  TC& t = *h->tc;
  k_tc_synth1<<<dim3((d.nx + 127) / 128, d.ky, d.ni), 128, 0, st>>>(d, t, alpha);
  pdf_count_launch(1);
  pdf_status s = umma_gemm(t.wya, t.tb, 1, 1, t.c_syn, 2 * d.ni * d.nx, 0, t.err, st);
  if (s != PDF_OK) return s;
  if (do_fft && d.fast) {
    const dim3 g((d.ny + FW - 1) / FW, d.ni);
    switch (d.Px) {
      case 64: k_tc_synth_post_fast<64><<<g, FT, 0, st>>>(d, t, Jout); break;
      case 128: k_tc_synth_post_fast<128><<<g, FT, 0, st>>>(d, t, Jout); break;
      case 256: k_tc_synth_post_fast<256><<<g, FT, 0, st>>>(d, t, Jout); break;
      case 384: k_tc_synth_post_fast<384><<<g, FT, 0, st>>>(d, t, Jout); break;
      case 512: k_tc_synth_post_fast<512><<<g, FT, 0, st>>>(d, t, Jout); break;
      default: return set_err(PDF_EUNSUPPORTED, "register FFT length");
    }
    pdf_count_launch(1);
    PDF_LAUNCHED("tensor-core synthesis epilogue + row DFT");
    return PDF_OK;
  }
  k_tc_synth_post<<<dim3((d.ny + ROWS_PER_CTA - 1) / ROWS_PER_CTA, d.ni), ROW_THREADS, sm_row_tc(d), st>>>(
      d, t, Jout, do_fft);
  pdf_count_launch(1);
  PDF_LAUNCHED("tensor-core synthesis");
  return PDF_OK;
}

pdf_status tc_gs_fwd(pdf_problem* h, const float2* X, const float2* sub, float2* out, FF* lp, int write_rdb,
                     cudaStream_t st) {
  Dev& d = h->d;
  TC& t = *h->tc;
  if (X) {
    k_tc_field_to_jb<<<(unsigned)(((size_t)d.ni * d.M + 255) / 256), 256, 0, st>>>(d, t, X);
    pdf_count_launch(1);
  }
  pdf_status s = umma_gemm(t.gsa, t.jb, 1, t.nsplit_fwd, t.c_fwd, 2 * d.ni, (long long)d.nr * 2 * d.ni, t.err, st);
  if (s != PDF_OK) return s;
  k_tc_gs_reduce<<<(d.ni * d.nr + 255) / 256, 256, 0, st>>>(d, t, t.nsplit_fwd, sub, out, lp, write_rdb);
  pdf_count_launch(1);
  PDF_LAUNCHED("tensor-core G_S");
  return PDF_OK;
}

pdf_status tc_gsh(pdf_problem* h, const float2* D, int from_rdb, cudaStream_t st) {
  Dev& d = h->d;
  TC& t = *h->tc;
  if (!from_rdb) {
    k_tc_d_to_rdb<<<(d.ni * d.nr + 255) / 256, 256, 0, st>>>(d, t, D);
    pdf_count_launch(1);
  }
  return umma_gemm(t.gst, t.rdb, 1, 1, t.c_adj, 2 * d.ni, 0, t.err, st);
}

pdf_status tc_gsh_field(pdf_problem* h, const float2* D, float2* out, float scale, cudaStream_t st) {
  pdf_status s = tc_gsh(h, D, 0, st);
  if (s != PDF_OK) return s;
  Dev& d = h->d;
  k_tc_cadj_to_field<<<(unsigned)(((size_t)d.ni * d.M + 255) / 256), 256, 0, st>>>(d, *h->tc, out, scale);
  pdf_count_launch(1);
  PDF_LAUNCHED("tensor-core G_S^H");
  return PDF_OK;
}

pdf_status tc_adj_ana(pdf_problem* h, cudaStream_t st) {
  Dev& d = h->d;
  TC& t = *h->tc;
  if (d.fast) {
    const dim3 g((d.ny + FW - 1) / FW, d.ni);
    switch (d.Px) {
      case 64: k_tc_adj_fast<64><<<g, FT, 0, st>>>(d, t); break;
      case 128: k_tc_adj_fast<128><<<g, FT, 0, st>>>(d, t); break;
      case 256: k_tc_adj_fast<256><<<g, FT, 0, st>>>(d, t); break;
      case 384: k_tc_adj_fast<384><<<g, FT, 0, st>>>(d, t); break;
      case 512: k_tc_adj_fast<512><<<g, FT, 0, st>>>(d, t); break;
      default: return set_err(PDF_EUNSUPPORTED, "register FFT length");
    }
    pdf_count_launch(1);
    PDF_LAUNCHED("tensor-core adjoint row IFFT + packing");
    return umma_gemm(t.gja, t.wxb, 1, 1, t.c_ana, 2 * d.kx, 0, t.err, st);
  }
  k_tc_adj_rowifft<<<dim3((d.ny + ROWS_PER_CTA - 1) / ROWS_PER_CTA, d.ni), ROW_THREADS, sm_row_tc(d), st>>>(d, t);
  pdf_count_launch(1);
  PDF_LAUNCHED("tensor-core adjoint row IFFT");
  return umma_gemm(t.gja, t.wxb, 1, 1, t.c_ana, 2 * d.kx, 0, t.err, st);
}

pdf_status tc_analysis_field(pdf_problem* h, const float2* in, cudaStream_t st) {
  Dev& d = h->d;
  TC& t = *h->tc;
  k_tc_field_to_gja<<<(unsigned)(((size_t)d.ni * d.M + 255) / 256), 256, 0, st>>>(d, t, in);
  pdf_count_launch(1);
  PDF_LAUNCHED("tensor-core analysis packing");
  return umma_gemm(t.gja, t.wxb, 1, 1, t.c_ana, 2 * d.kx, 0, t.err, st);
}
