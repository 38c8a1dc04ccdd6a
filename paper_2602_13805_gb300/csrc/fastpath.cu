// Register-FFT form of the hot path's FFT stages (padded lengths Px, Py in {64, 128, 256, 384,
// 512}).  One warp owns one padded line; rows of the row-transformed planes A are stored in the
// warp FFT's digit-reversed order, columns are processed in that order too, and the G_D
// spectrum is stored pre-permuted ([Px][Py], column-major), so no data are ever reordered.
// Kernel roles and fused epilogues are those of hotpath.cu (same Eq. references).
#include <algorithm>

#include "phases.cuh"

template <int PX>
__global__ void __launch_bounds__(FT) kf_synth_rowfft(Dev d, const float2* alpha, float2* Jout, int do_fft) {
  extern __shared__ float2 sm[];
  ph_synth_rowfft<PX>(d, blockIdx.x, blockIdx.y, sm, alpha, Jout, do_fft);
}
template <int PX>
__global__ void __launch_bounds__(FT) kf_rowfft_field(Dev d, const float2* in) {
  __shared__ float2 sm[PX];
  ph_rowfft_field<PX>(d, blockIdx.x, blockIdx.y, sm, in);
}
template <int PX>
__global__ void __launch_bounds__(FT) kf_rowifft_field(Dev d, float2* out) {
  __shared__ float2 sm[PX];
  ph_rowifft_field<PX>(d, blockIdx.x, blockIdx.y, sm, out);
}
template <int PY>
__global__ void __launch_bounds__(FT, (PY <= 384 ? 3 : 2)) kf_colconv(Dev d, int conj) {
  extern __shared__ float2 sm[];
  ph_colconv<PY>(d, blockIdx.x, blockIdx.y, sm, conj);
}
template <int PX>
__global__ void __launch_bounds__(FT) kf_rowifft_state(Dev d) {
  extern __shared__ float2 sm[];
  ph_rowifft_state<PX>(d, blockIdx.x, sm);
}
template <int PX, bool FUSED_R>
__global__ void __launch_bounds__(FT) kf_adj_rowfft(Dev d) {
  __shared__ float2 sm[PX];
  ph_adj_rowfft<PX, FUSED_R>(d, blockIdx.x, blockIdx.y, sm);
}
template <int PX>
__global__ void __launch_bounds__(FT) kf_rowifft_sums(Dev d) {
  extern __shared__ float2 sm[];
  ph_rowifft_sums<PX>(d, blockIdx.x, blockIdx.y, sm);
}
__global__ void __launch_bounds__(128) k_state_combine(Dev d) {
  ph_state_combine(d, blockIdx.x * blockDim.x + threadIdx.x);
}
template <int PX>
__global__ void __launch_bounds__(FT, (PX <= 384 ? 3 : 2)) kf_adj_rowifft_ana(Dev d, const float2* in, int mode) {
  extern __shared__ float2 sm[];
  ph_adj_rowifft_ana<PX>(d, blockIdx.x, blockIdx.y, sm, in, mode);
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
  cudaFuncSetAttribute(kf_adj_rowifft_ana<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024); \
  cudaFuncSetAttribute(kf_rowifft_sums<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  CFG(64) CFG(128) CFG(256) CFG(384) CFG(512)
#undef CFG
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(e, "cudaFuncSetAttribute(register FFT)");
  return PDF_OK;
}

size_t fp_smem_synth(const Dev& d) { return ((size_t)d.Px + (size_t)d.ky * d.kx) * sizeof(float2); }
size_t fp_smem_col(const Dev& d) { return ((size_t)d.Py + (size_t)FCOLS * (d.ny + 1)) * sizeof(float2); }
size_t fp_smem_state(const Dev& d) { return (size_t)d.Px * sizeof(float2) * 2 + 3 * FW * (size_t)d.Px * sizeof(float); }
size_t fp_smem_ana(const Dev& d) { return (size_t)d.Px * sizeof(float2); }
size_t fp_smem_sums(const Dev& d) { return (size_t)d.Px * sizeof(float2) + 3 * FW * (size_t)(d.Px / 2) * sizeof(float); }

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
// State pass: split over incidence groups (d.nsg > 0: row IFFT + group sums, then a per-pixel
// combine; r and L_State come with the adjoint row DFT) or one CTA per row over all incidences.
pdf_status fp_rowifft_state(const Dev& d, cudaStream_t st) {
  if (d.nsg > 0) {
#define L(P) kf_rowifft_sums<P><<<dim3(d.ny, d.nsg), FT, fp_smem_sums(d), st>>>(d)
    FAST_SWITCH(d.Px, L)
#undef L
    k_state_combine<<<(d.M + 127) / 128, 128, 0, st>>>(d);
    pdf_count_launch(1);
    return PDF_OK;
  }
#define L(P) kf_rowifft_state<P><<<d.ny, FT, fp_smem_state(d), st>>>(d)
  FAST_SWITCH(d.Px, L)
#undef L
  return PDF_OK;
}
pdf_status fp_adj_rowfft(const Dev& d, cudaStream_t st) {
  if (d.nsg > 0) {
#define L(P) kf_adj_rowfft<P, true><<<frow_grid(d), FT, 0, st>>>(d)
    FAST_SWITCH(d.Px, L)
#undef L
    return PDF_OK;
  }
#define L(P) kf_adj_rowfft<P, false><<<frow_grid(d), FT, 0, st>>>(d)
  FAST_SWITCH(d.Px, L)
#undef L
  return PDF_OK;
}

// Incidence groups of the split state pass: FW incidences per group (one per warp), as long as
// the adjoint's L_State partials (one per CTA) fit the partial strip; 0 keeps the
// one-CTA-per-row pass.
int fp_choose_nsg(const Dev& d, int sms) {
  (void)sms;
  const dim3 g = frow_grid(d);
  if ((size_t)g.x * g.y > PDF_LP_STRIDE) return 0;
  return (d.ni + FW - 1) / FW;
}

// number of L_State partials written per loss-and-gradient evaluation on this path
int fp_n_state(const Dev& d) { return d.nsg > 0 ? (int)(frow_grid(d).x * frow_grid(d).y) : d.ny; }
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

// Row DFT of the x synthesis basis: what[jx][c] = sum_{x < nx} Wx[jx][x] exp(-2 pi i f(c) x / Px),
// f(c) the frequency at position c of the register FFT's output order, so that the padded row DFT
// of J = T' Wx (Eq. 9) is T' what and the x-analysis of an inverse row DFT is a product with
// conj(what).  FP64, exact angle reduction (integer numerators modulo nx Px).
__global__ void k_row_dft_table(float2* __restrict__ what, int kx, int nx, int Px) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x, jx = blockIdx.y;
  if (c >= Px) return;
  const long f = perm_to_freq(c, Px / 32);
  const long fj = jx < (kx + 1) / 2 ? jx : nx - kx + jx;
  const long den = (long)nx * Px;
  double re = 0.0, im = 0.0;
  for (int x = 0; x < nx; ++x) {
    const long num = ((fj * x * Px - f * x * nx) % den + den) % den;
    double s, co;
    sincospi(2.0 * (double)num / (double)den, &s, &co);
    re += co;
    im += s;
  }
  const double sc = 1.0 / sqrt((double)nx);
  what[(size_t)jx * Px + c] = make_float2((float)(re * sc), (float)(im * sc));
}

pdf_status fp_row_dft_table(const Dev& d, float2* what, cudaStream_t st) {
  k_row_dft_table<<<dim3((d.Px + 127) / 128, d.kx), 128, 0, st>>>(what, d.kx, d.nx, d.Px);
  pdf_count_launch(1);
  PDF_LAUNCHED("row DFT table of the x basis");
  return PDF_OK;
}

pdf_status fp_perm_ghat(const Dev& d, float2* gp, cudaStream_t st) {
  k_perm_ghat<<<dim3((d.Py + 127) / 128, d.Px), 128, 0, st>>>(d.ghat, gp, d.Px, d.Py);
  pdf_count_launch(1);
  PDF_LAUNCHED("permuted spectrum");
  return PDF_OK;
}
