// Register-FFT form of the hot path's FFT stages (padded lengths Px, Py in {64, 128, 256, 384,
// 512}).  One warp owns one padded line; rows of the row-transformed planes A are stored in the
// warp FFT's digit-reversed order, columns are processed in that order too, and the G_D
// spectrum is stored pre-permuted ([Px][Py], column-major), so no data are ever reordered.
// Kernel roles and fused epilogues are those of hotpath.cu (same Eq. references).
#include "fftreg.cuh"
#include "problem.cuh"

#define FW 8            // warps per CTA
#define FT (FW * 32)
#define FCOLS 16        // columns per CTA of the column convolution

struct KS {             // compensated FP32 sum
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c, t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

template <int P>
__device__ __forceinline__ void load_tw(float2* tw, const float2* __restrict__ g) {
  for (int i = threadIdx.x; i < P; i += blockDim.x) tw[i] = g[i];
}

// J rows of plane p by synthesis (Eq. 9) and the padded row DFT -> A (permuted order)
template <int PX>
__global__ void __launch_bounds__(FT) kf_synth_rowfft(Dev d, const float2* __restrict__ alpha, float2* __restrict__ Jout,
                                                    int do_fft) {
  constexpr int R = PX / 32;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* sa = sm + PX;
  const int p = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int y = blockIdx.x * FW + warp;
  load_tw<PX>(tw, d.twx);
  for (int i = threadIdx.x; i < d.ky * d.kx; i += blockDim.x) sa[i] = alpha[(size_t)p * d.ky * d.kx + i];
  __syncthreads();
  if (y >= d.ny) return;
  float2 t0 = make_float2(0.f, 0.f), t1 = make_float2(0.f, 0.f);
  for (int jy = 0; jy < d.ky; ++jy) {
    const float2 w = __ldg(&d.wy[jy * d.ny + y]);
    if (lane < d.kx) t0 = t0 + cmul(w, sa[jy * d.kx + lane]);
    if (lane + 32 < d.kx) t1 = t1 + cmul(w, sa[jy * d.kx + lane + 32]);
  }
  float2 v[R];
#pragma unroll
  for (int m = 0; m < R; ++m) v[m] = make_float2(0.f, 0.f);
  for (int jx = 0; jx < d.kx; ++jx) {
    const float2 src = jx < 32 ? t0 : t1;
    const float2 T = make_float2(__shfl_sync(0xffffffffu, src.x, jx & 31), __shfl_sync(0xffffffffu, src.y, jx & 31));
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int x = lane + 32 * m;
      if (x < d.nx) v[m] = v[m] + cmul(T, __ldg(&d.wx[jx * d.nx + x]));
    }
  }
  const size_t row = (size_t)p * d.ny + y;
#pragma unroll
  for (int m = 0; m < R; ++m) {
    const int x = lane + 32 * m;
    if (x < d.nx) Jout[row * d.nx + x] = v[m];
  }
  if (!do_fft) return;
  WarpFFT<PX>::forward(v, tw, lane);
#pragma unroll
  for (int k = 0; k < R; ++k) d.A[row * PX + k * 32 + lane] = v[k];
}

template <int PX>
__global__ void __launch_bounds__(FT) kf_rowfft_field(Dev d, const float2* __restrict__ in) {
  constexpr int R = PX / 32;
  __shared__ float2 tw[PX];
  const int p = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int y = blockIdx.x * FW + warp;
  load_tw<PX>(tw, d.twx);
  __syncthreads();
  if (y >= d.ny) return;
  const size_t row = (size_t)p * d.ny + y;
  float2 v[R];
#pragma unroll
  for (int m = 0; m < R; ++m) {
    const int x = lane + 32 * m;
    v[m] = x < d.nx ? in[row * d.nx + x] : make_float2(0.f, 0.f);
  }
  WarpFFT<PX>::forward(v, tw, lane);
#pragma unroll
  for (int k = 0; k < R; ++k) d.A[row * PX + k * 32 + lane] = v[k];
}

template <int PX>
__global__ void __launch_bounds__(FT) kf_rowifft_field(Dev d, float2* __restrict__ out) {
  constexpr int R = PX / 32;
  __shared__ float2 tw[PX];
  const int p = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int y = blockIdx.x * FW + warp;
  load_tw<PX>(tw, d.twx);
  __syncthreads();
  if (y >= d.ny) return;
  const size_t row = (size_t)p * d.ny + y;
  float2 v[R];
#pragma unroll
  for (int k = 0; k < R; ++k) v[k] = d.A[row * PX + k * 32 + lane];
  WarpFFT<PX>::inverse(v, tw, lane);
#pragma unroll
  for (int m = 0; m < R; ++m) {
    const int x = lane + 32 * m;
    if (x < d.nx) out[row * d.nx + x] = v[m];
  }
}

// column DFT, x (conjugated) permuted spectrum, inverse column DFT, on FCOLS columns of plane p
template <int PY>
__global__ void __launch_bounds__(FT, 2) kf_colconv(Dev d, int conj) {
  constexpr int R = PY / 32;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* tile = sm + PY;
  const int LS = d.ny + 1;
  const int p = blockIdx.y, c0 = blockIdx.x * FCOLS;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* Ap = d.A + (size_t)p * d.ny * d.Px;
  load_tw<PY>(tw, d.twy);
  for (int i = threadIdx.x; i < FCOLS * d.ny; i += blockDim.x) {
    const int y = i / FCOLS, c = i - y * FCOLS;
    tile[c * LS + y] = Ap[(size_t)y * d.Px + c0 + c];
  }
  __syncthreads();
  for (int c = warp; c < FCOLS; c += FW) {
    const int cx = c0 + c;
    float2 v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int y = lane + 32 * m;
      v[m] = y < d.ny ? tile[c * LS + y] : make_float2(0.f, 0.f);
    }
    WarpFFT<PY>::forward(v, tw, lane);
    const float2* g = d.ghat_perm + (size_t)cx * PY;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      float2 s = __ldg(&g[k * 32 + lane]);
      if (conj) s.y = -s.y;
      v[k] = cmul(v[k], s);
    }
    WarpFFT<PY>::inverse(v, tw, lane);
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int y = lane + 32 * m;
      if (y < d.ny) tile[c * LS + y] = v[m];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < FCOLS * d.ny; i += blockDim.x) {
    const int y = i / FCOLS, c = i - y * FCOLS;
    Ap[(size_t)y * d.Px + c0 + c] = tile[c * LS + y];
  }
}

__device__ __forceinline__ float2 chi_of_R_f(float2 R, float2 beta, float qmin, bool* clamped) {
  float2 q = make_float2(1.f - R.x, -R.y);
  const float aq = sqrtf(cabs2(q));
  *clamped = aq < qmin;
  if (*clamped) q = aq > 0.f ? (qmin / aq) * q : make_float2(qmin, 0.f);
  return cdivf(R, cmul(beta, q));
}

// inverse row DFT -> G_D J, s = beta J + E_inc + G_D J, per-pixel least-squares R over all
// incidences (Eq. 6), chi (Eq. 7), state residual r and ||r||^2 (Eq. 15); one CTA per grid row
template <int PX>
__global__ void __launch_bounds__(FT) kf_rowifft_state(Dev d) {
  constexpr int R = PX / 32;
  extern __shared__ float2 sm[];
  __shared__ FF red[32];
  float2* tw = sm;
  float* part = (float*)(sm + PX);             // [3][FW][PX]
  float2* sR = (float2*)(part + 3 * FW * PX);  // [PX]
  const int y = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  load_tw<PX>(tw, d.twx);
  __syncthreads();
  KS nr[R], ni[R], dd[R];
  for (int p = warp; p < d.ni; p += FW) {
    const size_t row = (size_t)p * d.ny + y;
    float2 v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = d.A[row * PX + k * 32 + lane];
    WarpFFT<PX>::inverse(v, tw, lane);
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int x = lane + 32 * m;
      if (x < d.nx) {
        const size_t idx = row * d.nx + x;
        const float2 J = d.J[idx];
        const float2 s = cmul(d.beta, J) + d.einc[idx] + v[m];
        d.s[idx] = s;
        const float2 n = cmul(d.beta, cmulc(J, s));
        nr[m].add(n.x);
        ni[m].add(n.y);
        dd[m].add(cabs2(s));
      }
    }
  }
#pragma unroll
  for (int m = 0; m < R; ++m) {
    const int x = lane + 32 * m;
    part[(0 * FW + warp) * PX + x] = nr[m].s - nr[m].c;
    part[(1 * FW + warp) * PX + x] = ni[m].s - ni[m].c;
    part[(2 * FW + warp) * PX + x] = dd[m].s - dd[m].c;
  }
  __syncthreads();
  for (int x = threadIdx.x; x < d.nx; x += blockDim.x) {
    FF a = FF{0.f, 0.f}, b = FF{0.f, 0.f}, c = FF{0.f, 0.f};
    for (int w = 0; w < FW; ++w) {
      a = ff_add(a, part[(0 * FW + w) * PX + x]);
      b = ff_add(b, part[(1 * FW + w) * PX + x]);
      c = ff_add(c, part[(2 * FW + w) * PX + x]);
    }
    const float cf = c.hi + c.lo;
    const float2 Rv = make_float2((a.hi + a.lo) / cf, (b.hi + b.lo) / cf);
    bool cl;
    const float2 chi = chi_of_R_f(Rv, d.beta, d.q_min, &cl);
    const int n = y * d.nx + x;
    d.R[n] = Rv;
    d.chi[n] = chi;
    d.D[n] = cf;
    d.clamp[n] = cl ? 1 : 0;
    sR[x] = Rv;
  }
  __syncthreads();
  KS acc;
  for (int p = warp; p < d.ni; p += FW) {
    const size_t row = (size_t)p * d.ny + y;
    for (int x = lane; x < d.nx; x += 32) {
      const size_t idx = row * d.nx + x;
      const float2 r = cmul(sR[x], d.s[idx]) - cmul(d.beta, d.J[idx]);
      d.r[idx] = r;
      acc.add(cabs2(r));
    }
  }
  const FF t = ff_block_sum(ff_add(FF{acc.s, 0.f}, -acc.c), red);
  if (threadIdx.x == 0) d.lpart[LP_STATE * PDF_LP_STRIDE + y] = t;
}

// adjoint inputs: u (through G_D^H) and v (pointwise), then the padded row DFT of u
template <int PX>
__global__ void __launch_bounds__(FT) kf_adj_rowfft(Dev d) {
  constexpr int R = PX / 32;
  __shared__ float2 tw[PX];
  const int p = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int y = blockIdx.x * FW + warp;
  load_tw<PX>(tw, d.twx);
  __syncthreads();
  if (y >= d.ny) return;
  const float ke = d.invn[0];
  const float2 bc = cconj(d.beta);
  const size_t row = (size_t)p * d.ny + y;
  float2 v[R];
#pragma unroll
  for (int m = 0; m < R; ++m) {
    const int x = lane + 32 * m;
    v[m] = make_float2(0.f, 0.f);
    if (x < d.nx) {
      const int n = y * d.nx + x;
      const size_t idx = row * d.nx + x;
      const float2 w = d.w[n], Rr = d.R[n];
      const float2 J = d.J[idx], s = d.s[idx], r = d.r[idx];
      const float2 wc = cconj(w);
      const float2 cs = cmul(cmul(wc, d.beta), J) - (2.f * cmul(wc, Rr).x) * s;
      v[m] = ke * cmulc(r, Rr) + cs;
      const float2 omr = make_float2(1.f - Rr.x, Rr.y);
      d.v[idx] = ke * cmul(cmul(make_float2(-bc.x, -bc.y), omr), r) + cmul(bc, cmul(w, s) + cs);
    }
  }
  WarpFFT<PX>::forward(v, tw, lane);
#pragma unroll
  for (int k = 0; k < R; ++k) d.A[row * PX + k * 32 + lane] = v[k];
}

// mode 0: dL/dJ = G_D^H u (inverse row DFT of A) + v + G_S^H term; mode 1: the field `in`.
// Then analysis along x -> T2[p][y][jx] = sum_x g conj(Wx[jx][x]).
template <int PX>
__global__ void __launch_bounds__(FT) kf_adj_rowifft_ana(Dev d, const float2* __restrict__ in, int mode) {
  constexpr int R = PX / 32;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* g = sm + PX;                   // [FW][nx]
  const int p = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int y0 = blockIdx.x * FW;
  const int y = y0 + warp;
  load_tw<PX>(tw, d.twx);
  __syncthreads();
  if (y < d.ny) {
    const size_t row = (size_t)p * d.ny + y;
    if (mode == 0) {
      float2 v[R];
#pragma unroll
      for (int k = 0; k < R; ++k) v[k] = d.A[row * PX + k * 32 + lane];
      WarpFFT<PX>::inverse(v, tw, lane);
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int x = lane + 32 * m;
        if (x < d.nx) {
          const size_t idx = row * d.nx + x;
          g[warp * d.nx + x] = v[m] + d.v[idx] + d.gsh[idx];
        }
      }
    } else {
      for (int x = lane; x < d.nx; x += 32) g[warp * d.nx + x] = in[row * d.nx + x];
    }
  }
  __syncthreads();
  const int nrow = min(FW, d.ny - y0);
  for (int i = threadIdx.x; i < nrow * d.kx; i += blockDim.x) {
    const int rr = i / d.kx, jx = i - rr * d.kx;
    float2 acc = make_float2(0.f, 0.f);
    for (int x = 0; x < d.nx; ++x) acc = acc + cmulc(g[rr * d.nx + x], __ldg(&d.wx[jx * d.nx + x]));
    d.T2[((size_t)p * d.ny + y0 + rr) * d.kx + jx] = acc;
  }
}

// ---------------------------------------------------------------------------
// host dispatch
// ---------------------------------------------------------------------------
#define FAST_SWITCH(P, CALL) \
  switch (P) {               \
    case 64: CALL(64); break;   \
    case 128: CALL(128); break; \
    case 256: CALL(256); break; \
    case 384: CALL(384); break; \
    case 512: CALL(512); break; \
    default: return set_err(PDF_EUNSUPPORTED, "register FFT length"); \
  }

static dim3 frow_grid(const Dev& d) { return dim3((d.ny + FW - 1) / FW, d.ni); }

pdf_status fp_configure() {
#define CFG(P)                                                                                        \
  cudaFuncSetAttribute(kf_synth_rowfft<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);  \
  cudaFuncSetAttribute(kf_colconv<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);       \
  cudaFuncSetAttribute(kf_rowifft_state<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024); \
  cudaFuncSetAttribute(kf_adj_rowifft_ana<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  CFG(64) CFG(128) CFG(256) CFG(384) CFG(512)
#undef CFG
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(e, "cudaFuncSetAttribute(register FFT)");
  return PDF_OK;
}

size_t fp_smem_synth(const Dev& d) { return ((size_t)d.Px + (size_t)d.ky * d.kx) * sizeof(float2); }
size_t fp_smem_col(const Dev& d) { return ((size_t)d.Py + (size_t)FCOLS * (d.ny + 1)) * sizeof(float2); }
size_t fp_smem_state(const Dev& d) { return (size_t)d.Px * sizeof(float2) * 2 + 3 * FW * (size_t)d.Px * sizeof(float); }
size_t fp_smem_ana(const Dev& d) { return ((size_t)d.Px + (size_t)FW * d.nx) * sizeof(float2); }

pdf_status fp_synth_rowfft(const Dev& d, const float2* alpha, float2* Jout, int do_fft, cudaStream_t st) {
#define L(P) kf_synth_rowfft<P><<<frow_grid(d), FT, fp_smem_synth(d), st>>>(d, alpha, Jout, do_fft)
  FAST_SWITCH(d.Px, L)
#undef L
  return PDF_OK;
}
pdf_status fp_rowfft_field(const Dev& d, const float2* in, cudaStream_t st) {
#define L(P) kf_rowfft_field<P><<<frow_grid(d), FT, 0, st>>>(d, in)
  FAST_SWITCH(d.Px, L)
#undef L
  return PDF_OK;
}
pdf_status fp_rowifft_field(const Dev& d, float2* out, cudaStream_t st) {
#define L(P) kf_rowifft_field<P><<<frow_grid(d), FT, 0, st>>>(d, out)
  FAST_SWITCH(d.Px, L)
#undef L
  return PDF_OK;
}
pdf_status fp_colconv(const Dev& d, int conj, cudaStream_t st) {
#define L(P) kf_colconv<P><<<dim3(d.Px / FCOLS, d.ni), FT, fp_smem_col(d), st>>>(d, conj)
  FAST_SWITCH(d.Py, L)
#undef L
  return PDF_OK;
}
pdf_status fp_rowifft_state(const Dev& d, cudaStream_t st) {
#define L(P) kf_rowifft_state<P><<<d.ny, FT, fp_smem_state(d), st>>>(d)
  FAST_SWITCH(d.Px, L)
#undef L
  return PDF_OK;
}
pdf_status fp_adj_rowfft(const Dev& d, cudaStream_t st) {
#define L(P) kf_adj_rowfft<P><<<frow_grid(d), FT, 0, st>>>(d)
  FAST_SWITCH(d.Px, L)
#undef L
  return PDF_OK;
}
pdf_status fp_adj_rowifft_ana(const Dev& d, const float2* in, int mode, cudaStream_t st) {
#define L(P) kf_adj_rowifft_ana<P><<<frow_grid(d), FT, fp_smem_ana(d), st>>>(d, in, mode)
  FAST_SWITCH(d.Px, L)
#undef L
  return PDF_OK;
}

// permuted spectrum: ghat_perm[cx][cy] = ghat[ky(cy)][kx(cx)]
__global__ void k_perm_ghat(const float2* __restrict__ ghat, float2* __restrict__ gp, int Px, int Py) {
  const int cy = blockIdx.x * blockDim.x + threadIdx.x;
  const int cx = blockIdx.y;
  if (cy >= Py) return;
  const int ky = perm_to_freq(cy, Py / 32), kx = perm_to_freq(cx, Px / 32);
  gp[(size_t)cx * Py + cy] = ghat[(size_t)ky * Px + kx];
}

pdf_status fp_perm_ghat(const Dev& d, float2* gp, cudaStream_t st) {
  k_perm_ghat<<<dim3((d.Py + 127) / 128, d.Px), 128, 0, st>>>(d.ghat, gp, d.Px, d.Py);
  pdf_count_launch(1);
  PDF_LAUNCHED("permuted spectrum");
  return PDF_OK;
}
