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
// ---------------------------------------------------------------------------
// Column convolution, pipelined: persistent CTAs walk tiles of PCOLS padded columns of one
// incidence; the next tile's column data are copied into the second shared-memory buffer with
// cp.async while the warps transform the current one (one column per warp: forward register FFT,
// x G_D spectrum or its conjugate, inverse, in place), so the global-load latency of the tile
// overlaps the FFT work instead of stalling every warp of the CTA at the start.
// ---------------------------------------------------------------------------
#define PCOLS 8            // columns per tile of the pipelined column convolution

// Column stride of a tile, the first >= ny that is 2 mod 16 (in complex64 words): a warp's copies
// and stores walk 4 rows x 8 columns, and with this stride each 16-thread half touches 16 distinct
// 8-byte banks; the FFT's reads of one column (lanes along y) are contiguous whatever the stride.
__host__ __device__ __forceinline__ int colpipe_ls(int ny) { return ny + ((18 - ny % 16) % 16); }

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int PY>
__global__ void __launch_bounds__(FT, (PY <= 384 ? 3 : 2)) kf_colconv_pipe(Dev d, int conj, int ntiles) {
  constexpr int R = PY / 32;
  extern __shared__ float2 sm[];
  float2* tw = sm;                                     // [PY]
  const int LS = colpipe_ls(d.ny);
  float2* bufs = sm + PY;                              // [2][PCOLS][LS]
  const int ngrp = d.Px / PCOLS;                       // tiles per incidence
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nel = PCOLS * d.ny;
  auto issue = [&](int t, float2* tile) {
    const int p = t / ngrp, c0 = (t - p * ngrp) * PCOLS;
    const float2* Ap = d.A + (size_t)p * d.ny * d.Px + c0;
    for (int i = threadIdx.x; i < nel; i += FT) {
      const int y = i / PCOLS, c = i - y * PCOLS;
      cp_async8(&tile[c * LS + y], &Ap[(size_t)y * d.Px + c]);
    }
  };
  load_tw<PY>(tw, d.twy);
  int t = blockIdx.x, cur = 0;
  if (t < ntiles) issue(t, bufs);
  cp_async_commit();
  for (; t < ntiles; t += gridDim.x) {
    float2* tile = bufs + cur * PCOLS * LS;
    const int tn = t + gridDim.x;
    if (tn < ntiles) issue(tn, bufs + (cur ^ 1) * PCOLS * LS);
    cp_async_commit();
    cp_async_wait<1>();                                // this tile's copies have landed (own thread)
    __syncthreads();                                   // ... and every thread's
    const int p = t / ngrp, c0 = (t - p * ngrp) * PCOLS;
    for (int c = warp; c < PCOLS; c += FW) {
      const int cx = c0 + c;
      float2 v[R];
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int y = lane + 32 * m;
        v[m] = (2 * m < R && y < d.ny) ? tile[c * LS + y] : make_float2(0.f, 0.f);
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
        if (2 * m < R && y < d.ny) tile[c * LS + y] = v[m];
      }
    }
    __syncthreads();
    float2* Ap = d.A + (size_t)p * d.ny * d.Px + c0;
    for (int i = threadIdx.x; i < nel; i += FT) {
      const int y = i / PCOLS, c = i - y * PCOLS;
      Ap[(size_t)y * d.Px + c] = tile[c * LS + y];
    }
    __syncthreads();                                   // the buffer is refilled two tiles on
    cur ^= 1;
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Adjoint row IFFT + x-analysis, persistent: each CTA stages the twiddles and the x basis
// Wx [kx][nx] in shared memory once and its warps then walk rows (p, y) independently: inverse
// row DFT of dL/dJ's row spectrum, + v (+ the G_S^H term when unfolded), and
// T2[p][y][jx] = sum_x g[x] conj(Wx[jx][x]) in blocks of 8 coefficients (per-lane partial sums
// over the lane's x, then an 8-way warp reduce-scatter), all basis reads from shared memory.
// ---------------------------------------------------------------------------
// Warp reduce-scatter of 8 complex values: on return lane l holds in a[0] the warp-wide sum of
// the values with index l >> 2.
__device__ __forceinline__ void warp_reduce_scatter8(float2 (&a)[8], int lane) {
#pragma unroll
  for (int st = 0; st < 3; ++st) {
    const int h = 16 >> st, n = 4 >> st;
    const bool up = (lane & h) != 0;
#pragma unroll
    for (int i = 0; i < n; ++i) {
      const float2 send = up ? a[i] : a[i + n];
      const float2 keep = up ? a[i + n] : a[i];
      a[i] = keep + shfl_xor2(send, h);
    }
  }
  a[0] = a[0] + shfl_xor2(a[0], 2);
  a[0] = a[0] + shfl_xor2(a[0], 1);
}

// FULL: nx = PX / 2, so every one of the first R/2 slots of a row holds a grid column and no
// per-slot bound checks are needed.  The x basis is staged with its rows padded to a multiple of 8
// (zeros), so the last coefficient block needs no check either.
template <int PX, bool FULL>
__global__ void __launch_bounds__(FT, 3) kf_adj_ana_p(Dev d, const float2* in, int mode) {
  constexpr int R = PX / 32;
  extern __shared__ float2 sm[];
  float2* tw = sm;                       // [PX]
  float2* wxs = sm + PX;                 // [kx8][nx]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kx8 = (d.kx + 7) & ~7;
  load_tw<PX>(tw, d.twx);
  for (int i = threadIdx.x; i < kx8 * d.nx; i += FT) wxs[i] = i < d.kx * d.nx ? d.wx[i] : make_float2(0.f, 0.f);
  __syncthreads();
  const int nrows = d.ni * d.ny;
  for (int row = blockIdx.x * FW + warp; row < nrows; row += gridDim.x * FW) {
    float2 g[R];
    if (mode == 0) {
#pragma unroll
      for (int k = 0; k < R; ++k) g[k] = d.A[(size_t)row * PX + k * 32 + lane];
      WarpFFT<PX>::inverse(g, tw, lane);
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int x = lane + 32 * m;
        if (2 * m < R && (FULL || x < d.nx)) {
          const size_t idx = (size_t)row * d.nx + x;
          g[m] = d.fold ? g[m] + d.v[idx] : g[m] + d.v[idx] + d.gsh[idx];
        } else {
          g[m] = make_float2(0.f, 0.f);
        }
      }
    } else {
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int x = lane + 32 * m;
        g[m] = (2 * m < R && (FULL || x < d.nx)) ? in[(size_t)row * d.nx + x] : make_float2(0.f, 0.f);
      }
    }
    for (int j0 = 0; j0 < d.kx; j0 += 8) {
      float2 acc[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] = make_float2(0.f, 0.f);
      const float2* wb = wxs + j0 * d.nx + lane;
#pragma unroll
      for (int m = 0; m < R / 2; ++m) {
        if (FULL || lane + 32 * m < d.nx) {
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[j] = acc[j] + cmulc(g[m], wb[j * d.nx + 32 * m]);
        }
      }
      warp_reduce_scatter8(acc, lane);
      const int jx = j0 + (lane >> 2);
      if ((lane & 3) == 0 && jx < d.kx) d.T2[(size_t)row * d.kx + jx] = acc[0];
    }
  }
}

// ---------------------------------------------------------------------------
// Synthesis + padded row DFT, persistent: each CTA stages the twiddles and the x basis Wx [kx][nx]
// in shared memory once; its warps then walk rows (p, y): T'[jx] = sum_jy Wy[jy][y] alpha_p[jy][jx]
// (lanes over jx), J[y][x] = sum_jx T'[jx] Wx[jx][x] (Eq. 9) with the basis read from shared
// memory, then the forward register FFT of the row into A.
// ---------------------------------------------------------------------------
// FULL: nx = PX / 2 (no per-slot bound checks).  T' of the warp's row goes through a per-warp
// shared-memory line and is read back as a broadcast, one load per coefficient.
template <int PX, bool FULL>
__global__ void __launch_bounds__(FT, 3) kf_synth_p(Dev d, const float2* __restrict__ alpha, float2* __restrict__ Jout,
                                                    int do_fft) {
  constexpr int R = PX / 32;
  extern __shared__ float2 sm[];
  float2* tw = sm;                       // [PX]
  float2* wxs = sm + PX;                 // [kx][nx]
  float2* tl = wxs + d.kx * d.nx;        // [FW][64] T' of each warp's current row
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  load_tw<PX>(tw, d.twx);
  for (int i = threadIdx.x; i < d.kx * d.nx; i += FT) wxs[i] = d.wx[i];
  __syncthreads();
  float2* tr = tl + warp * 64;
  const int nrows = d.ni * d.ny, NA = d.ky * d.kx;
  for (int row = blockIdx.x * FW + warp; row < nrows; row += gridDim.x * FW) {
    const int p = row / d.ny, y = row - p * d.ny;
    const float2* ap = alpha + (size_t)p * NA;
    float2 t0 = make_float2(0.f, 0.f), t1 = make_float2(0.f, 0.f);
    for (int jy = 0; jy < d.ky; ++jy) {
      const float2 w = __ldg(&d.wy[jy * d.ny + y]);
      if (lane < d.kx) t0 = t0 + cmul(w, __ldg(&ap[jy * d.kx + lane]));
      if (lane + 32 < d.kx) t1 = t1 + cmul(w, __ldg(&ap[jy * d.kx + lane + 32]));
    }
    __syncwarp();
    tr[lane] = t0;
    tr[lane + 32] = t1;
    __syncwarp();
    float2 v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = make_float2(0.f, 0.f);
    const float2* wb = wxs + lane;
#pragma unroll 4
    for (int jx = 0; jx < d.kx; ++jx) {
      const float2 T = tr[jx];
#pragma unroll
      for (int m = 0; m < R / 2; ++m)
        if (FULL || lane + 32 * m < d.nx) v[m] = v[m] + cmul(T, wb[jx * d.nx + 32 * m]);
    }
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int x = lane + 32 * m;
      if (2 * m < R && (FULL || x < d.nx)) Jout[(size_t)row * d.nx + x] = v[m];
    }
    if (do_fft) {
      WarpFFT<PX>::forward(v, tw, lane);
#pragma unroll
      for (int k = 0; k < R; ++k) d.A[(size_t)row * PX + k * 32 + lane] = v[k];
    }
  }
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
  cudaFuncSetAttribute(kf_colconv_pipe<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);  \
  cudaFuncSetAttribute(kf_adj_ana_p<P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024); \
  cudaFuncSetAttribute(kf_adj_ana_p<P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024); \
  cudaFuncSetAttribute(kf_synth_p<P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);   \
  cudaFuncSetAttribute(kf_synth_p<P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);  \
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

size_t fp_smem_ana_p(const Dev& d);
size_t fp_smem_synth_p(const Dev& d);
template <class K>
static int persistent_slots(K kernel, size_t smem);

pdf_status fp_synth_rowfft(const Dev& d, const float2* alpha, float2* Jout, int do_fft, cudaStream_t st) {
  if (fp_smem_synth_p(d) <= 64 * 1024) {               // twiddles + Wx + the warps' T' lines
    const int nrows = d.ni * d.ny, nb = (nrows + FW - 1) / FW;
#define L(P)                                                                                     \
  {                                                                                              \
    static size_t sm_ = 0;                                                                       \
    static int slots_ = 0;                                                                       \
    if (sm_ != fp_smem_synth_p(d)) {                                                             \
      sm_ = fp_smem_synth_p(d);                                                                  \
      slots_ = persistent_slots(kf_synth_p<P, true>, sm_);                                       \
    }                                                                                            \
    if (2 * d.nx == P)                                                                           \
      kf_synth_p<P, true><<<std::min(nb, slots_), FT, sm_, st>>>(d, alpha, Jout, do_fft);        \
    else                                                                                         \
      kf_synth_p<P, false><<<std::min(nb, slots_), FT, sm_, st>>>(d, alpha, Jout, do_fft);       \
  }
    FAST_SWITCH(d.Px, L)
#undef L
    return PDF_OK;
  }
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
size_t fp_smem_colpipe(const Dev& d) { return ((size_t)d.Py + 2 * (size_t)PCOLS * colpipe_ls(d.ny)) * sizeof(float2); }

// resident CTAs of the pipelined column convolution on this device (grid = that many, at most the
// tile count)
template <int P>
static int colpipe_slots(const Dev& d) {
  static size_t smem = 0;
  static int slots = 0;
  const size_t need = fp_smem_colpipe(d);
  if (need != smem) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kf_colconv_pipe<P>, FT, need);
    cudaGetLastError();
    slots = std::max(1, sms * std::max(1, occ));
    smem = need;
  }
  return slots;
}

pdf_status fp_colconv(const Dev& d, int conj, cudaStream_t st) {
  if (d.Px % PCOLS == 0) {
    const int ntiles = d.ni * (d.Px / PCOLS);
#define L(P) kf_colconv_pipe<P><<<std::min(ntiles, colpipe_slots<P>(d)), FT, fp_smem_colpipe(d), st>>>(d, conj, ntiles)
    FAST_SWITCH(d.Py, L)
#undef L
    return PDF_OK;
  }
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
size_t fp_smem_ana_p(const Dev& d) { return ((size_t)d.Px + (size_t)((d.kx + 7) & ~7) * d.nx) * sizeof(float2); }
size_t fp_smem_synth_p(const Dev& d) { return ((size_t)d.Px + (size_t)d.kx * d.nx + FW * 64) * sizeof(float2); }

// resident CTAs of a persistent row kernel with `smem` bytes of dynamic shared memory
template <class K>
static int persistent_slots(K kernel, size_t smem) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, FT, smem);
  cudaGetLastError();
  return std::max(1, sms * std::max(1, occ));
}

pdf_status fp_adj_rowifft_ana(const Dev& d, const float2* in, int mode, cudaStream_t st) {
  if (fp_smem_ana_p(d) <= 64 * 1024) {
    const int nrows = d.ni * d.ny, nb = (nrows + FW - 1) / FW;
#define L(P)                                                                                     \
  {                                                                                              \
    static size_t sm_ = 0;                                                                       \
    static int slots_ = 0;                                                                       \
    if (sm_ != fp_smem_ana_p(d)) {                                                               \
      sm_ = fp_smem_ana_p(d);                                                                    \
      slots_ = persistent_slots(kf_adj_ana_p<P, true>, sm_);                                     \
    }                                                                                            \
    if (2 * d.nx == P)                                                                           \
      kf_adj_ana_p<P, true><<<std::min(nb, slots_), FT, sm_, st>>>(d, in, mode);                 \
    else                                                                                         \
      kf_adj_ana_p<P, false><<<std::min(nb, slots_), FT, sm_, st>>>(d, in, mode);                \
  }
    FAST_SWITCH(d.Px, L)
#undef L
    return PDF_OK;
  }
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
