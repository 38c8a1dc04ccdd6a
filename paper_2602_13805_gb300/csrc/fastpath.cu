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
// Column convolution in two passes through shared memory, for P = 16 Q (Q = 8, 16, 24) and
// ny <= P / 2.  With n = n1 + Q n2 and k = 16 k1 + k2 (n1, k1 < Q; n2, k2 < 16),
//   X[16 k1 + k2] = sum_n1 W_Q^{n1 k1} W_P^{n1 k2} sum_n2 x[n1 + Q n2] W_16^{n2 k2}.
// Pass A, one thread per (column, n1): the 16-point DFT over n2, of which only n2 < 8 can be
// non-zero (the column is zero-padded from ny <= P/2 rows), as two 8-point DFTs, and the twiddle.
// Pass B, one thread per (column, k2): the Q-point DFT over n1, the product with the G_D
// spectrum (or its conjugate), and the inverse Q-point DFT.  Pass A^-1, one thread per (column,
// n1): the conjugate twiddle, the inverse 16-point DFT evaluated only at the rows n2 < 8 that are
// kept, and the store.  Lines stay in registers; the two exchanges go through a padded
// [n1][column][k2] array in shared memory, so no cross-lane shuffles are needed.  Persistent CTAs
// walk tiles of C2P_COLS columns of one incidence; the next tile's column data are copied with
// cp.async during passes B and A^-1 of the current one, and the spectrum of the next tile's
// columns during pass A^-1 (skipped when the columns are the same).
// ---------------------------------------------------------------------------
#define C2P_COLS 8
template <int Q> struct Col2p {
  static constexpr int P = 16 * Q;
  static constexpr int NT = C2P_COLS * (Q > 16 ? Q : 16);   // threads per CTA
  static constexpr int MINB = Q > 16 ? 3 : 4;
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

template <int Q, bool CONJ>
__global__ void __launch_bounds__(Col2p<Q>::NT, Col2p<Q>::MINB) kf_colconv_2p(Dev d, int ntiles) {
  pdl_wait();
  constexpr int P = 16 * Q, NT = Col2p<Q>::NT, C = C2P_COLS, SL = 17;
  extern __shared__ float2 sm[];
  float2* twA = sm;                      // [16][Q]  W_P^{n1 k2} at k2 * Q + n1
  float2* gsp = twA + 16 * Q;            // [C][P]   spectrum of the tile's columns, natural order
  float2* S = gsp + C * P;               // [Q][C][SL]
  float2* tile = S + Q * C * SL;         // [C][LS]  column data, rows < ny
  const int LS = colpipe_ls(d.ny);
  const int ngrp = d.Px / C;
  const int tid = threadIdx.x;
  for (int i = tid; i < 16 * Q; i += NT) {
    const int k2 = i / Q, n1 = i - k2 * Q;
    twA[i] = d.twy[n1 * k2];
  }
  auto issue_cols = [&](int t) {
    const int p = t / ngrp, c0 = (t - p * ngrp) * C;
    const float2* Ap = d.A + (size_t)p * d.ny * d.Px + c0;
    for (int i = tid; i < C * d.ny; i += NT) {
      const int y = i / C, c = i - y * C;
      cp_async8(&tile[c * LS + y], &Ap[(size_t)y * d.Px + c]);
    }
  };
  auto issue_spec = [&](int t) {
    const float2* src = d.ghat_col + (size_t)(t % ngrp) * C * P;
    for (int i = tid; i < C * P / 2; i += NT) cp_async16(&gsp[2 * i], &src[2 * i]);
  };
  int t = blockIdx.x;
  if (t < ntiles) issue_cols(t);
  cp_async_commit();
  if (t < ntiles) issue_spec(t);
  cp_async_commit();
  for (; t < ntiles; t += gridDim.x) {
    const int p = t / ngrp, c0 = (t - p * ngrp) * C;
    const int tn = t + gridDim.x;
    cp_async_wait<1>();                  // this tile's column data (the spectrum may still fly)
    __syncthreads();
    if (tid < C * Q) {                   // pass A
      const int c = tid % C, n1 = tid / C;
      float2 e[8], o[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int n = n1 + Q * j;
        const float2 x = n < d.ny ? tile[c * LS + n] : make_float2(0.f, 0.f);
        e[j] = x;
        o[j] = tw_mul<16, false>(x, j);
      }
      SmallDFT<8, false>::run(e);
      SmallDFT<8, false>::run(o);
      float2* s = S + (n1 * C + c) * SL;
      s[0] = e[0];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (k > 0) s[2 * k] = cmul(e[k], twA[2 * k * Q + n1]);
        s[2 * k + 1] = cmul(o[k], twA[(2 * k + 1) * Q + n1]);
      }
    }
    cp_async_wait<0>();                  // the spectrum of this tile's columns
    __syncthreads();
    if (tn < ntiles) issue_cols(tn);
    cp_async_commit();
    if (tid < C * 16) {                  // pass B
      const int k2 = tid & 15, c = tid >> 4;
      float2* s = S + c * SL + k2;
      float2 v[Q];
#pragma unroll
      for (int n1 = 0; n1 < Q; ++n1) v[n1] = s[n1 * C * SL];
      SmallDFT<Q, false>::run(v);
      const float2* g = gsp + c * P + k2;
#pragma unroll
      for (int k1 = 0; k1 < Q; ++k1) v[k1] = CONJ ? cmulc(v[k1], g[16 * k1]) : cmul(v[k1], g[16 * k1]);
      SmallDFT<Q, true>::run(v);
#pragma unroll
      for (int n1 = 0; n1 < Q; ++n1) s[n1 * C * SL] = v[n1];
    }
    __syncthreads();
    if (tn < ntiles && (tn % ngrp) != (t % ngrp)) issue_spec(tn);
    cp_async_commit();
    if (tid < C * Q) {                   // pass A^-1
      const int c = tid % C, n1 = tid / C;
      const float2* s = S + (n1 * C + c) * SL;
      float2 e[8], o[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {              // conjugate twiddle W_P^{-n1 k2}, k2 = 2k, 2k + 1
        e[k] = k == 0 ? s[0] : cmul(s[2 * k], cconj(twA[2 * k * Q + n1]));
        o[k] = cmul(s[2 * k + 1], cconj(twA[(2 * k + 1) * Q + n1]));
      }
      SmallDFT<8, true>::run(e);
      SmallDFT<8, true>::run(o);
      float2* Ap = d.A + (size_t)p * d.ny * d.Px + c0 + c;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int n = n1 + Q * j;
        if (n < d.ny) Ap[(size_t)n * d.Px] = e[j] + tw_mul<16, true>(o[j], j);
      }
    }
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
          for (int j = 0; j < 8; ++j) acc[j] = cmacc(acc[j], g[m], wb[j * d.nx + 32 * m]);
        }
      }
      warp_reduce_scatter8(acc, lane);
      const int jx = j0 + (lane >> 2);
      if ((lane & 3) == 0 && jx < d.kx) d.T2[(size_t)row * d.kx + jx] = acc[0];
    }
  }
}

// Adjoint row IFFT + x-analysis with the analysis as a DFT (nx = PX / 2): the x basis is the
// truncated unitary DFT (Eq. 9), Wx[jx][x] = exp(2 pi i f_jx x / nx) / sqrt(nx), so
// T2[p][y][jx] = sum_x g[x] conj(Wx[jx][x]) is the forward nx-point DFT of the row g at the retained
// frequencies f_jx, / sqrt(nx).  After the inverse PX-point row DFT the row's columns x < nx sit in
// the warp FFT's natural input layout for nx = 32 (R / 2) points (lane l, slot m: x = l + 32 m), so a
// forward (R/2)-slot warp FFT (nx-entry twiddle table tw2[e] = tw[2 e]) replaces the nx x kx product;
// lane l, slot k1 then holds frequency k1 + (R/2) brev5(l), written out where it is retained.
template <int PX>
__global__ void __launch_bounds__(FT, 3) kf_adj_fft_p(Dev d, const float2* in, int mode) {
  pdl_wait();
  constexpr int R = PX / 32, H = R / 2, NX = PX / 2;
  extern __shared__ float2 sm[];
  float2* tw = sm;                       // [PX]
  float2* tw2 = sm + PX;                 // [NX]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  load_tw<PX>(tw, d.twx);
  for (int i = threadIdx.x; i < NX; i += FT) tw2[i] = d.twx[2 * i];
  __syncthreads();
  const int kx = d.kx, hx = (kx + 1) / 2, fneg = NX - kx;     // f >= NX - kx + hx: jx = f - fneg
  const float sc = 1.f / sqrtf((float)NX);
  const int nrows = d.ni * d.ny;
  for (int row = blockIdx.x * FW + warp; row < nrows; row += gridDim.x * FW) {
    float2 h[H];
    if (mode == 0) {
      float2 g[R];
#pragma unroll
      for (int k = 0; k < R; ++k) g[k] = d.A[(size_t)row * PX + k * 32 + lane];
      WarpFFT<PX>::inverse(g, tw, lane);
#pragma unroll
      for (int m = 0; m < H; ++m) {
        const size_t idx = (size_t)row * NX + lane + 32 * m;
        h[m] = d.fold ? g[m] + d.v[idx] : g[m] + d.v[idx] + d.gsh[idx];
      }
    } else {
#pragma unroll
      for (int m = 0; m < H; ++m) h[m] = in[(size_t)row * NX + lane + 32 * m];
    }
    WarpFFT<NX>::forward(h, tw2, lane);
    const int fb = H * brev5(lane);
#pragma unroll
    for (int k1 = 0; k1 < H; ++k1) {
      const int f = k1 + fb;
      const int jx = f < hx ? f : (f >= fneg + hx ? f - fneg : -1);
      if (jx >= 0) d.T2[(size_t)row * kx + jx] = sc * h[k1];
    }
  }
}
// y-analysis (second half of Phi^H, Eq. 9) as a warp FFT: out[p][jy][jx] = sum_y T2[p][y][jx]
// conj(Wy[jy][y]) is the forward ny-point DFT of column jx of T2[p] at the retained frequencies f_jy,
// / sqrt(ny).  CTA (p, 8 columns jx0 ..): the columns are copied by cp.async into shared memory,
// warp w transforms column jx0 + w (lane l, slot m: y = l + 32 m; twiddles tw_ny[e] = tw_Py[2 e]) and
// writes the retained outputs.  Advances the Adam step counter inside the solve loop, as the other
// y-analysis kernels do.
template <int NY>
__global__ void __launch_bounds__(FT) kf_ana_y_fft(Dev d, const float2* __restrict__ T2, float2* __restrict__ out,
                                                   int* step_inc) {
  pdl_wait();
  constexpr int H = NY / 32;
  __shared__ float2 tws[NY];
  __shared__ float2 cs[NY * 9];            // [y][8 columns], stride 9
  const int p = blockIdx.x, jx0 = blockIdx.y * 8, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kx = d.kx, ky = d.ky, nc = min(8, kx - jx0);
  if (step_inc && p == 0 && blockIdx.y == 0 && threadIdx.x == 0) *step_inc += 1;
  for (int i = threadIdx.x; i < NY; i += FT) tws[i] = d.twy[2 * i];
  const float2* T = T2 + (size_t)p * NY * kx + jx0;
  for (int i = threadIdx.x; i < NY * 8; i += FT) {
    const int y = i >> 3, c = i & 7;
    if (c < nc) cp_async8(&cs[y * 9 + c], &T[(size_t)y * kx + c]);
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  if (warp >= nc) return;
  float2 h[H];
#pragma unroll
  for (int m = 0; m < H; ++m) h[m] = cs[(lane + 32 * m) * 9 + warp];
  WarpFFT<NY>::forward(h, tws, lane);
  const int hy = (ky + 1) / 2, fneg = NY - ky, fb = H * brev5(lane);
  const float sc = 1.f / sqrtf((float)NY);
  float2* o = out + (size_t)p * ky * kx + jx0 + warp;
#pragma unroll
  for (int k1 = 0; k1 < H; ++k1) {
    const int f = k1 + fb;
    const int jy = f < hy ? f : (f >= fneg + hy ? f - fneg : -1);
    if (jy >= 0) o[(size_t)jy * kx] = sc * h[k1];
  }
}

// the FFT y-analysis: ny = Py / 2 in {64, 128, 192, 256}
bool fp_ana_y_fft(const Dev& d, const float2* T2, float2* out, int* step_inc, cudaStream_t st) {
  if (!(d.fast && 2 * d.ny == d.Py && d.ky <= d.ny)) return false;
  const dim3 grid(d.ni, (d.kx + 7) / 8);
  switch (d.ny) {
    case 64: launch_pdl(kf_ana_y_fft<64>, grid, FT, 0, st, d, T2, out, step_inc); break;
    case 128: launch_pdl(kf_ana_y_fft<128>, grid, FT, 0, st, d, T2, out, step_inc); break;
    case 192: launch_pdl(kf_ana_y_fft<192>, grid, FT, 0, st, d, T2, out, step_inc); break;
    case 256: launch_pdl(kf_ana_y_fft<256>, grid, FT, 0, st, d, T2, out, step_inc); break;
    default: return false;
  }
  return true;
}

size_t fp_smem_adjfft(const Dev& d) { return (size_t)(d.Px + d.Px / 2) * sizeof(float2); }
static bool adjfft_ok(const Dev& d) { return 2 * d.nx == d.Px && d.Px >= 128 && d.kx <= d.nx; }

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
      if (lane < d.kx) t0 = cmac(t0, w, __ldg(&ap[jy * d.kx + lane]));
      if (lane + 32 < d.kx) t1 = cmac(t1, w, __ldg(&ap[jy * d.kx + lane + 32]));
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
        if (FULL || lane + 32 * m < d.nx) v[m] = cmac(v[m], T, wb[jx * d.nx + 32 * m]);
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

// ---------------------------------------------------------------------------
// Synthesis (Eq. 9) and padded row DFT by tiles of 8 rows of one incidence, for P = Px = 16 Q
// (Q = 8, 16, 24) and nx <= P / 2.  Per tile: T'[r][jx] = sum_jy Wy[jy][y0 + r] alpha_p[jy][jx]
// (alpha_p and the tile's Wy entries staged in shared memory by cp.async); the J rows
// J[r][x] = sum_jx T'[r][jx] Wx[jx][x]: at full width (nx = P / 2) a warp per row takes the inverse
// nx-point warp FFT of the retained modes (Wx is the truncated unitary DFT, so J is that transform
// / sqrt(nx)), otherwise a thread per x accumulates all 8 rows; then the
// row DFT in two passes through shared memory as in kf_colconv_2p (16-point DFTs over n2 from
// the nx <= P/2 non-zero points, twiddle, Q-point DFTs over n1).  The spectra are staged in the
// register FFT's digit-reversed order (position (f mod R) 32 + brev5(f / R) holds frequency f,
// R = P / 32; rows padded to 33 per 32) and stored as whole rows, so the row-spectrum plane A
// keeps the layout the other kernels read.  With `dterm` each tile also forms the data residual
// r_d[p][r] = sum_j (G_S Phi)[r][j] alpha_p[j] - E_sca[p][r] of its share of the receivers (a warp
// per receiver, alpha_p already in shared memory) and its ||r_d||^2 partial (slot: tile index).
// The next tile's alpha and Wy entries are copied by cp.async from the end of T' on.
// ---------------------------------------------------------------------------
#define S2P_ROWS 8
template <int Q>
__global__ void __launch_bounds__(Col2p<Q>::NT, Col2p<Q>::MINB)
    kf_synth_2p(Dev d, const float2* __restrict__ alpha, float2* __restrict__ Jout, int do_fft, int ntiles,
                int dterm) {
  pdl_wait();
  constexpr int P = 16 * Q, NT = Col2p<Q>::NT, C = S2P_ROWS, SL = 17, R = P / 32, YS = R * 33;
  extern __shared__ float2 sm[];
  const int NA = d.ky * d.kx;
  const int LS = colpipe_ls(d.nx);
  float2* twA = sm;                        // [16][Q]  W_P^{n1 k2} at k2 * Q + n1
  float2* as = twA + 16 * Q;               // [na2]    alpha of the tile's incidence
  float2* wys = as + ((NA + 1) & ~1);      // [ky][C]  Wy entries of the tile's rows
  float2* ts = wys + d.ky * C;             // [kx][C]  T'
  float2* xt = ts + d.kx * C;              // [C][LS]  J rows (pass A input), then the staged spectra [C][YS]
  float2* S = xt + (C * LS > C * YS ? C * LS : C * YS);   // [Q][C][SL] exchange array
  float2* ux = S + Q * C * SL;             // [nx] exp(2 pi i m / nx) / sqrt(nx): Wx[jx][x] = ux[f_jx x mod nx]
  int* posf = reinterpret_cast<int*>(ux + d.nx);          // [P] staging position of frequency f
  __shared__ FF wsum[NT / 32];             // per-warp ||r_d||^2 of the tile's receivers
  const int tid = threadIdx.x;
  const int tpi = (d.ny + C - 1) / C;      // tiles per incidence
  const int hx = (d.kx + 1) / 2;           // modes jx < hx have frequency jx, the others nx - kx + jx
  for (int i = tid; i < 16 * Q; i += NT) {
    const int k2 = i / Q, n1 = i - k2 * Q;
    twA[i] = d.twx[n1 * k2];
  }
  for (int f = tid; f < P; f += NT) posf[f] = (f % R) * 33 + brev5(f / R);
  // full width (nx = P / 2): J rows by an inverse nx-point warp FFT, ux holds its twiddles
  // exp(-2 pi i e / nx) = tw_P[2 e]; otherwise ux is the unit-circle table of the product
  const bool jfft = 2 * d.nx == P;
  for (int m = tid; m < d.nx; m += NT) ux[m] = jfft ? d.twx[2 * m] : d.ux[m];
  auto issue = [&](int t) {
    const int p = t / tpi, y0 = (t - p * tpi) * C;
    const float2* ap = alpha + (size_t)p * NA;
    for (int i = tid; i < NA; i += NT) cp_async8(&as[i], &ap[i]);
    for (int i = tid; i < d.ky * C; i += NT) {
      const int jy = i / C, r = i - jy * C;
      if (y0 + r < d.ny) cp_async8(&wys[i], &d.wy[(size_t)jy * d.ny + y0 + r]);
      else wys[i] = make_float2(0.f, 0.f);
    }
  };
  int t = blockIdx.x;
  if (t < ntiles) issue(t);
  cp_async_commit();
  for (; t < ntiles; t += gridDim.x) {
    const int p = t / tpi, y0 = (t - p * tpi) * C;
    cp_async_wait<0>();
    __syncthreads();
    for (int i = tid; i < d.kx * C; i += NT) {   // T' = Wy^T alpha_p on the tile's rows
      const int r = i / d.kx, jx = i - r * d.kx;
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
      for (int jy = 0; jy < d.ky; ++jy) acc = cmac(acc, wys[jy * C + r], as[jy * d.kx + jx]);
      ts[jx * C + r] = acc;
    }
    if (dterm) {                           // data residual (Eq. 16) of this tile's share of the receivers
      const int ti = t - p * tpi, warp = tid >> 5, lane = tid & 31;
      const int r0 = (int)((long)ti * d.nr / tpi), r1 = (int)((long)(ti + 1) * d.nr / tpi);
      FF e2 = FF{0.f, 0.f};
      for (int rr = r0 + warp; rr < r1; rr += NT / 32) {
        const float2* gr = d.gsf + (size_t)rr * NA;
        float2 a4[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        if (NA <= 1024) {                  // the lane's whole row slice in flight at once (one L2 round trip)
          float2 gv[32];
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const int j = lane + 32 * q;
            gv[q] = j < NA ? __ldg(&gr[j]) : make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const int j = lane + 32 * q;
            if (j < NA) a4[q & 3] = cmac(a4[q & 3], gv[q], as[j]);
          }
        } else {
          int j = lane;
          for (; j + 96 < NA; j += 128)
#pragma unroll
            for (int q = 0; q < 4; ++q) a4[q] = cmac(a4[q], __ldg(&gr[j + 32 * q]), as[j + 32 * q]);
          for (; j < NA; j += 32) a4[0] = cmac(a4[0], __ldg(&gr[j]), as[j]);
        }
        float2 a = (a4[0] + a4[1]) + (a4[2] + a4[3]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
          a = a + make_float2(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o));
        if (lane == 0) {
          const size_t o = (size_t)p * d.nr + rr;
          const float2 v = a - d.esca[o];
          d.rd[o] = v;
          e2 = ff_add(e2, cabs2(v));
        }
      }
      if (lane == 0) wsum[warp] = e2;
    }
    __syncthreads();
    if (dterm && tid == 0) {
      FF e2 = FF{0.f, 0.f};
      for (int w = 0; w < NT / 32; ++w) e2 = ff_add(e2, wsum[w]);
      d.lpart[LP_DATA * PDF_LP_STRIDE + t] = e2;
    }
    if (t + (int)gridDim.x < ntiles) issue(t + gridDim.x);   // alpha and Wy are free until the next tile
    cp_async_commit();
    if (jfft) {                            // J rows: J[r][x] = (1 / sqrt(nx)) sum_f T'(f) e^{2 pi i f x / nx}
      constexpr int H = P / 64;            // slots per lane of the nx = 32 H point warp FFT
      const int warp = tid >> 5, lane = tid & 31, fneg = d.nx - d.kx;
      const float sc = 1.f / sqrtf((float)d.nx);
      for (int r = warp; r < C; r += NT / 32) {
        float2 h[H];
#pragma unroll
        for (int k1 = 0; k1 < H; ++k1) {   // digit-reversed input: lane l, slot k1 has frequency k1 + H brev5(l)
          const int f = k1 + H * brev5(lane);
          const int jx = f < hx ? f : (f >= fneg + hx ? f - fneg : -1);
          h[k1] = jx >= 0 ? ts[jx * C + r] : make_float2(0.f, 0.f);
        }
        WarpFFT<P / 2>::inverse(h, ux, lane);
#pragma unroll
        for (int m = 0; m < H; ++m) {
          const int x = lane + 32 * m;
          const float2 jv = sc * h[m];
          if (y0 + r < d.ny) Jout[((size_t)p * d.ny + y0 + r) * d.nx + x] = jv;
          xt[r * LS + x] = jv;
        }
      }
    } else if (tid < d.nx) {               // J rows: thread x, all C rows
      const int x = tid;
      float2 acc[C];
#pragma unroll
      for (int r = 0; r < C; ++r) acc[r] = make_float2(0.f, 0.f);
      int m = 0;                           // f_jx x mod nx, stepped by x as f_jx steps by 1
#pragma unroll 2
      for (int jx = 0; jx < d.kx; ++jx) {
        if (jx == hx) m = (int)(((long)(d.nx - d.kx + hx) * x) % d.nx);
        const float2 w = ux[m];
        m += x;
        if (m >= d.nx) m -= d.nx;
        const float4* tp = reinterpret_cast<const float4*>(ts + jx * C);
#pragma unroll
        for (int h = 0; h < C / 2; ++h) {
          const float4 tt = tp[h];
          acc[2 * h] = cmac(acc[2 * h], make_float2(tt.x, tt.y), w);
          acc[2 * h + 1] = cmac(acc[2 * h + 1], make_float2(tt.z, tt.w), w);
        }
      }
#pragma unroll
      for (int r = 0; r < C; ++r) {
        if (y0 + r < d.ny) Jout[((size_t)p * d.ny + y0 + r) * d.nx + x] = acc[r];
        xt[r * LS + x] = acc[r];
      }
    }
    if (!do_fft) continue;
    __syncthreads();
    if (tid < C * Q) {                     // pass A: 16-point DFTs over n2 (n2 < 8 non-zero), twiddle
      const int r = tid % C, n1 = tid / C;
      float2 e[8], o[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int n = n1 + Q * j;
        const float2 x = n < d.nx ? xt[r * LS + n] : make_float2(0.f, 0.f);
        e[j] = x;
        o[j] = tw_mul<16, false>(x, j);
      }
      SmallDFT<8, false>::run(e);
      SmallDFT<8, false>::run(o);
      float2* s = S + (n1 * C + r) * SL;
      s[0] = e[0];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (k > 0) s[2 * k] = cmul(e[k], twA[2 * k * Q + n1]);
        s[2 * k + 1] = cmul(o[k], twA[(2 * k + 1) * Q + n1]);
      }
    }
    __syncthreads();
    if (tid < C * 16) {                    // pass B: Q-point DFTs over n1, staged in storage order
      const int k2 = tid & 15, rb = tid >> 4;
      float2 v[Q];
#pragma unroll
      for (int n1 = 0; n1 < Q; ++n1) v[n1] = S[(n1 * C + rb) * SL + k2];
      SmallDFT<Q, false>::run(v);
      float2* yr = xt + rb * YS;
#pragma unroll
      for (int k1 = 0; k1 < Q; ++k1) yr[posf[16 * k1 + k2]] = v[k1];
    }
    __syncthreads();
    const int nr = min(C, d.ny - y0);
    float2* Ar = d.A + ((size_t)p * d.ny + y0) * P;
    for (int c = tid; c < P; c += NT) {
      const float2* yc = xt + (c >> 5) * 33 + (c & 31);
      for (int r = 0; r < nr; ++r) Ar[(size_t)r * P + c] = yc[r * YS];
    }
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Adjoint row IFFT + x-analysis by tiles of 8 rows of one incidence (the tiled counterpart of
// kf_adj_ana_p; P = Px = 16 Q, nx <= P / 2).  The tile's row spectra are copied (cp.async, one
// tile ahead) into the staging layout of kf_synth_2p; pass B^-1, one thread per (row, k2), takes
// the inverse Q-point DFTs over k1; pass A^-1, one thread per (row, n1), the conjugate twiddle and
// the inverse 16-point DFT evaluated at the columns n2 < 8, then adds v (and the unfolded data
// term's G_S^H r_d): the rows g of dL/dJ (mode 0), or the rows of `in` (mode 1).  The x-analysis
// T2[r][jx] = sum_x g[r][x] conj(Wx[jx][x]) runs with lanes over jx, warps over chunks of x, all 8
// rows per thread (the rows of g broadcast from shared memory), then a fixed-order sum over the
// chunks; Wx[jx][x] = u[f_jx x mod nx] is read from the nx-entry table u in shared memory.
// ---------------------------------------------------------------------------
#define YPAD 34        // staged spectrum rows: 32 positions + 2 pad (16-byte aligned pairs)
template <int Q>
__global__ void __launch_bounds__(Col2p<Q>::NT, Col2p<Q>::MINB)
    kf_adj_ana_2p(Dev d, const float2* __restrict__ in, int mode, int ntiles) {
  constexpr int P = 16 * Q, NT = Col2p<Q>::NT, C = S2P_ROWS, SL = 17, R = P / 32, YS = R * YPAD;
  constexpr int NCH = NT / 32;             // x chunks of the analysis
  extern __shared__ float2 sm[];
  float2* twA = sm;                        // [16][Q]
  float2* ys = twA + 16 * Q;               // [C][YS]  staged row spectra
  float2* S = ys + C * YS;                 // [Q][C][SL] exchange array, then the analysis partials
  float2* G = S + Q * C * SL;              // [nx][C]  rows of g by column
  float2* ux = G + d.nx * C;               // [nx] exp(2 pi i m / nx) / sqrt(nx): Wx[jx][x] = ux[f_jx x mod nx]
  int* posf = reinterpret_cast<int*>(ux + d.nx);      // [P]
  const int tid = threadIdx.x;
  const int tpi = (d.ny + C - 1) / C;
  for (int i = tid; i < 16 * Q; i += NT) {
    const int k2 = i / Q, n1 = i - k2 * Q;
    twA[i] = d.twx[n1 * k2];
  }
  for (int f = tid; f < P; f += NT) posf[f] = (f % R) * YPAD + brev5(f / R);
  for (int m = tid; m < d.nx; m += NT) ux[m] = d.ux[m];
  auto issue = [&](int t) {
    const int p = t / tpi, y0 = (t - p * tpi) * C;
    const int nr = min(C, d.ny - y0);
    const float2* Ar = d.A + ((size_t)p * d.ny + y0) * P;
    for (int i = tid; i < nr * (P / 2); i += NT) {
      const int r = i / (P / 2), c = 2 * (i - r * (P / 2));
      cp_async16(&ys[r * YS + (c >> 5) * YPAD + (c & 31)], &Ar[(size_t)r * P + c]);
    }
  };
  const int xc = (d.nx + NCH - 1) / NCH;   // columns per analysis chunk
  int t = blockIdx.x;
  if (mode == 0 && t < ntiles) issue(t);
  cp_async_commit();
  for (; t < ntiles; t += gridDim.x) {
    const int p = t / tpi, y0 = (t - p * tpi) * C;
    const size_t rowbase = (size_t)p * d.ny + y0;
    cp_async_wait<0>();
    __syncthreads();
    if (mode == 0) {
      if (tid < C * 16) {                  // pass B^-1: inverse Q-point DFTs over k1
        const int k2 = tid & 15, rb = tid >> 4;
        const float2* yr = ys + rb * YS;
        float2 v[Q];
#pragma unroll
        for (int k1 = 0; k1 < Q; ++k1) v[k1] = yr[posf[16 * k1 + k2]];
        SmallDFT<Q, true>::run(v);
#pragma unroll
        for (int n1 = 0; n1 < Q; ++n1) S[(n1 * C + rb) * SL + k2] = v[n1];
      }
      __syncthreads();
      if (t + (int)gridDim.x < ntiles) issue(t + gridDim.x);
      cp_async_commit();
      if (tid < C * Q) {                   // pass A^-1: twiddle, inverse 16-point DFTs, + v
        const int r = tid % C, n1 = tid / C;
        const bool live = y0 + r < d.ny;
        const size_t pix = (rowbase + r) * d.nx;
        float2 vp[8];                      // v (+ G_S^H r_d) at this thread's columns, loaded ahead
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int x = n1 + Q * j;
          vp[j] = make_float2(0.f, 0.f);
          if (live && x < d.nx) vp[j] = d.fold ? d.v[pix + x] : d.v[pix + x] + d.gsh[pix + x];
        }
        const float2* s = S + (n1 * C + r) * SL;
        float2 e[8], o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          e[k] = k == 0 ? s[0] : cmul(s[2 * k], cconj(twA[2 * k * Q + n1]));
          o[k] = cmul(s[2 * k + 1], cconj(twA[(2 * k + 1) * Q + n1]));
        }
        SmallDFT<8, true>::run(e);
        SmallDFT<8, true>::run(o);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int x = n1 + Q * j;
          if (x < d.nx) {
            const float2 g = e[j] + tw_mul<16, true>(o[j], j);
            G[x * C + r] = live ? g + vp[j] : make_float2(0.f, 0.f);
          }
        }
      }
    } else {
      for (int i = tid; i < C * d.nx; i += NT) {
        const int r = i / d.nx, x = i - r * d.nx;
        G[x * C + r] = y0 + r < d.ny ? in[(rowbase + r) * d.nx + x] : make_float2(0.f, 0.f);
      }
    }
    __syncthreads();
    {                                      // x-analysis partials over chunk `ch`
      const int jx = tid & 31, ch = tid >> 5;
      float2 acc[C];
#pragma unroll
      for (int r = 0; r < C; ++r) acc[r] = make_float2(0.f, 0.f);
      if (jx < d.kx) {
        const int x0 = ch * xc, xe = min(d.nx, x0 + xc);
        const int f = jx < (d.kx + 1) / 2 ? jx : d.nx - d.kx + jx;
        int m = (int)(((long)f * x0) % d.nx);   // f x mod nx, stepped by f as x steps by 1
#pragma unroll 2
        for (int x = x0; x < xe; ++x) {
          const float2 w = ux[m];
          m += f;
          if (m >= d.nx) m -= d.nx;
          const float4* gp = reinterpret_cast<const float4*>(G + x * C);
#pragma unroll
          for (int h = 0; h < C / 2; ++h) {
            const float4 gg = gp[h];
            acc[2 * h] = cmacc(acc[2 * h], make_float2(gg.x, gg.y), w);
            acc[2 * h + 1] = cmacc(acc[2 * h + 1], make_float2(gg.z, gg.w), w);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < C; ++r) S[(ch * C + r) * 32 + jx] = acc[r];
    }
    __syncthreads();
    for (int i = tid; i < C * d.kx; i += NT) {
      const int r = i / d.kx, jx = i - r * d.kx;
      if (y0 + r < d.ny) {
        float2 a = S[r * 32 + jx];
        for (int ch = 1; ch < NCH; ++ch) a = a + S[(ch * C + r) * 32 + jx];
        d.T2[(rowbase + r) * d.kx + jx] = a;
      }
    }
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Split state pass by tiles of one row y and one incidence group g (the FW = 8 incidences
// p = 8 g + r), P = Px = 16 Q, nx <= P / 2: the inverse row DFT of the convolved plane in two passes
// through shared memory (as kf_colconv_2p; rows by (r, k2) for pass B^-1, by (r, n1) for pass A^-1,
// the exchange array [r][n1][k2]) -> G_D J, s = beta J + E_inc + G_D J (Eq. 6) stored, and the
// group's per-pixel float-float sums of beta J conj(s) and |s|^2 (incidences in increasing order),
// as kf_rowifft_sums.  Persistent CTAs walk the tiles t = y nsg + g and copy the next tile's row
// spectra with cp.async during the current one.  (The same tiling for the adjoint row DFT,
// kf_adj_rowfft, measured slower: 38.9 against 26.6 us at c5, its 8 row groups re-reading the
// per-pixel w and R-hat.)
// ---------------------------------------------------------------------------
template <int Q>
__global__ void __launch_bounds__(Col2p<Q>::NT, Col2p<Q>::MINB) kf_state_2p(Dev d, int ntiles) {
  pdl_wait();
  constexpr int P = 16 * Q, NT = Col2p<Q>::NT, C = FW, SL = 17, R = P / 32, YS = R * YPAD;
  extern __shared__ float2 sm[];
  float2* twA = sm;                        // [16][Q]
  float2* ys = twA + 16 * Q;               // [C][YS]  staged row spectra
  float2* S = ys + C * YS;                 // [C][Q][SL]
  float* part = reinterpret_cast<float*>(S + C * Q * SL);   // [3][C][nx]
  int* posf = reinterpret_cast<int*>(part + 3 * C * d.nx);  // [P]
  const int tid = threadIdx.x;
  for (int i = tid; i < 16 * Q; i += NT) {
    const int k2 = i / Q, n1 = i - k2 * Q;
    twA[i] = d.twx[n1 * k2];
  }
  for (int f = tid; f < P; f += NT) posf[f] = (f % R) * YPAD + brev5(f / R);
  auto issue = [&](int t) {
    const int y = t / d.nsg, g = t - y * d.nsg;
    const int nr = min(C, d.ni - g * C);
    for (int i = tid; i < nr * (P / 2); i += NT) {
      const int r = i / (P / 2), c = 2 * (i - r * (P / 2));
      cp_async16(&ys[r * YS + (c >> 5) * YPAD + (c & 31)], &d.A[((size_t)(g * C + r) * d.ny + y) * P + c]);
    }
  };
  int t = blockIdx.x;
  if (t < ntiles) issue(t);
  cp_async_commit();
  for (; t < ntiles; t += gridDim.x) {
    const int y = t / d.nsg, g = t - y * d.nsg;
    cp_async_wait<0>();
    __syncthreads();
    if (tid < C * 16) {                    // pass B^-1
      const int k2 = tid & 15, r = tid >> 4;
      const float2* yr = ys + r * YS;
      float2 v[Q];
#pragma unroll
      for (int k1 = 0; k1 < Q; ++k1) v[k1] = yr[posf[16 * k1 + k2]];
      SmallDFT<Q, true>::run(v);
#pragma unroll
      for (int n1 = 0; n1 < Q; ++n1) S[(r * Q + n1) * SL + k2] = v[n1];
    }
    __syncthreads();
    if (t + (int)gridDim.x < ntiles) issue(t + gridDim.x);
    cp_async_commit();
    if (tid < C * Q) {                     // pass A^-1 and the state at this thread's pixels
      const int r = tid / Q, n1 = tid - r * Q, p = g * C + r;
      const bool live = p < d.ni;
      const size_t rowpix = ((size_t)p * d.ny + y) * d.nx;
      float2 Jv[8], Ev[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int x = n1 + Q * j;
        Jv[j] = Ev[j] = make_float2(0.f, 0.f);
        if (live && x < d.nx) {
          Jv[j] = d.J[rowpix + x];
          Ev[j] = d.einc[rowpix + x];
        }
      }
      const float2* sr = S + (r * Q + n1) * SL;
      float2 e[8], o[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        e[k] = k == 0 ? sr[0] : cmul(sr[2 * k], cconj(twA[2 * k * Q + n1]));
        o[k] = cmul(sr[2 * k + 1], cconj(twA[(2 * k + 1) * Q + n1]));
      }
      SmallDFT<8, true>::run(e);
      SmallDFT<8, true>::run(o);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int x = n1 + Q * j;
        if (x < d.nx) {
          float3 c = make_float3(0.f, 0.f, 0.f);
          if (live) {
            const float2 gd = e[j] + tw_mul<16, true>(o[j], j);
            const float2 sv = cmul(d.beta, Jv[j]) + Ev[j] + gd;
            d.s[rowpix + x] = sv;
            const float2 nv = cmul(d.beta, cmulc(Jv[j], sv));
            c = make_float3(nv.x, nv.y, cabs2(sv));
          }
          part[(0 * C + r) * d.nx + x] = c.x;
          part[(1 * C + r) * d.nx + x] = c.y;
          part[(2 * C + r) * d.nx + x] = c.z;
        }
      }
    }
    __syncthreads();
    for (int x = tid; x < d.nx; x += NT) {
      FF a = FF{0.f, 0.f}, b = FF{0.f, 0.f}, c = FF{0.f, 0.f};
      for (int r = 0; r < C; ++r) {
        a = ff_add(a, part[(0 * C + r) * d.nx + x]);
        b = ff_add(b, part[(1 * C + r) * d.nx + x]);
        c = ff_add(c, part[(2 * C + r) * d.nx + x]);
      }
      const size_t o = (size_t)g * d.M + (size_t)y * d.nx + x;
      d.sgA[o] = make_float4(a.hi, a.lo, b.hi, b.lo);
      d.sgB[o] = make_float2(c.hi, c.lo);
    }
  }
  cp_async_wait<0>();
}

// u[m] = exp(+2 pi i m / n) / sqrt(n), assembled exactly as the synthesis tables (FP64, the same
// reduced numerator), so that Wx[jx][x] = u[f_jx x mod nx] holds bit for bit
__global__ void k_unit_table(float2* __restrict__ u, int n) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  double s, c;
  sincospi(2.0 * (double)m / (double)n, &s, &c);
  const double sc = 1.0 / sqrt((double)n);
  u[m] = make_float2((float)(c * sc), (float)(s * sc));
}
pdf_status fp_unit_table(int n, float2* u, cudaStream_t st) {
  k_unit_table<<<(n + 127) / 128, 128, 0, st>>>(u, n);
  pdf_count_launch(1);
  PDF_LAUNCHED("unit-circle table of the x basis");
  return PDF_OK;
}

template <int PX>
__global__ void __launch_bounds__(FT) kf_rowifft_state(Dev d) {
  extern __shared__ float2 sm[];
  ph_rowifft_state<PX>(d, blockIdx.x, sm);
}
template <int PX, bool FUSED_R>
__global__ void __launch_bounds__(FT) kf_adj_rowfft(Dev d) {
  pdl_wait();
  __shared__ float2 sm[PX];
  ph_adj_rowfft<PX, FUSED_R>(d, blockIdx.x, blockIdx.y, sm);
}
template <int PX>
__global__ void __launch_bounds__(FT) kf_rowifft_sums(Dev d) {
  extern __shared__ float2 sm[];
  ph_rowifft_sums<PX>(d, blockIdx.x, blockIdx.y, sm);
}
__global__ void __launch_bounds__(128) k_state_combine(Dev d) {
  pdl_wait();
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
#define CFG2(Q)                                                                                        \
  cudaFuncSetAttribute(kf_colconv_2p<Q, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024); \
  cudaFuncSetAttribute(kf_colconv_2p<Q, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  CFG2(8) CFG2(16) CFG2(24)
#undef CFG2
  cudaFuncSetAttribute(kf_synth_2p<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  cudaFuncSetAttribute(kf_synth_2p<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  cudaFuncSetAttribute(kf_synth_2p<24>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  cudaFuncSetAttribute(kf_adj_ana_2p<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  cudaFuncSetAttribute(kf_adj_ana_2p<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  cudaFuncSetAttribute(kf_adj_ana_2p<24>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
#define CFG3(Q) cudaFuncSetAttribute(kf_state_2p<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  CFG3(8) CFG3(16) CFG3(24)
#undef CFG3
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

size_t fp_smem_synth2p(const Dev& d) {
  const int Q = d.Px / 16, NA = d.ky * d.kx;
  const size_t stage = std::max((size_t)colpipe_ls(d.nx), (size_t)(d.Px / 32) * 33) * S2P_ROWS;
  return ((size_t)16 * Q + (size_t)((NA + 1) & ~1) + (size_t)d.ky * S2P_ROWS + (size_t)d.kx * S2P_ROWS + stage +
          (size_t)Q * S2P_ROWS * 17 + d.nx) *
             sizeof(float2) +
         (size_t)d.Px * sizeof(int);
}
// the tiled synthesis covers Px = 128, 256, 384 with nx <= Px / 2, kx <= 32
static bool synth2p_ok(const Dev& d) {
  return (d.Px == 128 || d.Px == 256 || d.Px == 384) && 2 * d.nx <= d.Px && d.kx <= 32 && d.ux &&
         fp_smem_synth2p(d) <= 96 * 1024;
}
template <int Q>
static int synth2p_slots(const Dev& d) {
  static size_t smem = 0;
  static int slots = 0;
  const size_t need = fp_smem_synth2p(d);
  if (need != smem) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kf_synth_2p<Q>, Col2p<Q>::NT, need);
    cudaGetLastError();
    slots = std::max(1, sms * std::max(1, occ));
    smem = need;
  }
  return slots;
}

bool fp_synth2p_ok(const Dev& d) { return synth2p_ok(d); }
int fp_synth2p_tpi(const Dev& d) { return (d.ny + S2P_ROWS - 1) / S2P_ROWS; }

pdf_status fp_synth_rowfft(const Dev& d, const float2* alpha, float2* Jout, int do_fft, cudaStream_t st,
                           int dterm) {
  if (synth2p_ok(d)) {
    const int ntiles = d.ni * ((d.ny + S2P_ROWS - 1) / S2P_ROWS);
#define L(Q)                                                                                     \
  launch_pdl(kf_synth_2p<Q>, std::min(ntiles, synth2p_slots<Q>(d)), Col2p<Q>::NT, fp_smem_synth2p(d), st, d, \
             alpha, Jout, do_fft, ntiles, dterm)
    switch (d.Px / 16) {
      case 8: L(8); break;
      case 16: L(16); break;
      default: L(24); break;
    }
#undef L
    return PDF_OK;
  }
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

size_t fp_smem_col2p(const Dev& d) {
  const int Q = d.Py / 16;
  return ((size_t)16 * Q + (size_t)C2P_COLS * d.Py + (size_t)Q * C2P_COLS * 17 + (size_t)C2P_COLS * colpipe_ls(d.ny)) *
         sizeof(float2);
}
// the two-pass column convolution covers P = 128, 256, 384 with ny <= P / 2
static bool col2p_ok(const Dev& d) {
  return (d.Py == 128 || d.Py == 256 || d.Py == 384) && 2 * d.ny <= d.Py && d.Px % C2P_COLS == 0 && d.ghat_col;
}
template <int Q>
static int col2p_slots(const Dev& d) {
  static size_t smem = 0;
  static int slots = 0;
  const size_t need = fp_smem_col2p(d);
  if (need != smem) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kf_colconv_2p<Q, false>, Col2p<Q>::NT, need);
    cudaGetLastError();
    slots = std::max(1, sms * std::max(1, occ));
    smem = need;
  }
  return slots;
}

pdf_status fp_colconv(const Dev& d, int conj, cudaStream_t st) {
  if (col2p_ok(d)) {
    const int ntiles = d.ni * (d.Px / C2P_COLS);
#define L(Q)                                                                                              \
  {                                                                                                       \
    const int g_ = std::min(ntiles, col2p_slots<Q>(d));                                                   \
    if (conj)                                                                                             \
      launch_pdl(kf_colconv_2p<Q, true>, g_, Col2p<Q>::NT, fp_smem_col2p(d), st, d, ntiles);              \
    else                                                                                                  \
      launch_pdl(kf_colconv_2p<Q, false>, g_, Col2p<Q>::NT, fp_smem_col2p(d), st, d, ntiles);             \
  }
    switch (d.Py / 16) {
      case 8: L(8); break;
      case 16: L(16); break;
      default: L(24); break;
    }
#undef L
    return PDF_OK;
  }
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
size_t fp_smem_state2p(const Dev& d) {
  const int Q = d.Px / 16;
  return ((size_t)16 * Q + (size_t)FW * (d.Px / 32) * YPAD + (size_t)FW * Q * 17) * sizeof(float2) +
         3 * (size_t)FW * d.nx * sizeof(float) + (size_t)d.Px * sizeof(int);
}
// the tiled state pass: split state pass (nsg > 0), Px = 128, 256, 384, nx <= Px / 2
bool fp_row2p_ok(const Dev& d) {
  return d.nsg > 0 && (d.Px == 128 || d.Px == 256 || d.Px == 384) && 2 * d.nx <= d.Px &&
         (size_t)d.ny * d.nsg <= PDF_LP_STRIDE && fp_smem_state2p(d) <= 96 * 1024;
}
template <class K>
static int slots_of(K kernel, int nt, size_t smem) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, nt, smem);
  cudaGetLastError();
  return std::max(1, sms * std::max(1, occ));
}

pdf_status fp_rowifft_state(const Dev& d, cudaStream_t st) {
  if (d.row2p) {
    const int ntiles = d.ny * d.nsg;
#define L(Q)                                                                                \
  {                                                                                         \
    static size_t sm_ = 0;                                                                  \
    static int slots_ = 0;                                                                  \
    if (sm_ != fp_smem_state2p(d)) {                                                        \
      sm_ = fp_smem_state2p(d);                                                             \
      slots_ = slots_of(kf_state_2p<Q>, Col2p<Q>::NT, sm_);                                 \
    }                                                                                       \
    launch_pdl(kf_state_2p<Q>, std::min(ntiles, slots_), Col2p<Q>::NT, sm_, st, d, ntiles);  \
  }
    switch (d.Px / 16) {
      case 8: L(8); break;
      case 16: L(16); break;
      default: L(24); break;
    }
#undef L
    launch_pdl(k_state_combine, (d.M + 127) / 128, 128, 0, st, d);
    pdf_count_launch(1);
    return PDF_OK;
  }
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
#define L(P) launch_pdl(kf_adj_rowfft<P, true>, frow_grid(d), FT, 0, st, d)
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

size_t fp_smem_ana2p(const Dev& d) {
  const int Q = d.Px / 16;
  return ((size_t)16 * Q + (size_t)S2P_ROWS * (d.Px / 32) * YPAD + (size_t)Q * S2P_ROWS * 17 +
          (size_t)d.nx * S2P_ROWS + d.nx) *
             sizeof(float2) +
         (size_t)d.Px * sizeof(int);
}
// the tiled adjoint analysis covers Px = 128, 256 (384 compiles too) with nx <= Px / 2 and kx <= 32
// (the chunk partials, NT / 32 chunks x 8 rows x 32, fit the exchange array); at Px = 384 the
// warp-per-row kf_adj_ana_p measured faster (38.9 against 45 us a launch at c5), at Px = 256 the
// tiles (14.3 against 15.2 us at c3)
static bool ana2p_ok(const Dev& d) {
  return (d.Px == 128 || d.Px == 256) && 2 * d.nx <= d.Px && d.kx <= 32 && d.ux && fp_smem_ana2p(d) <= 96 * 1024;
}
template <int Q>
static int ana2p_slots(const Dev& d) {
  static size_t smem = 0;
  static int slots = 0;
  const size_t need = fp_smem_ana2p(d);
  if (need != smem) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kf_adj_ana_2p<Q>, Col2p<Q>::NT, need);
    cudaGetLastError();
    slots = std::max(1, sms * std::max(1, occ));
    smem = need;
  }
  return slots;
}

pdf_status fp_adj_rowifft_ana(const Dev& d, const float2* in, int mode, cudaStream_t st) {
  if (adjfft_ok(d)) {
    const int nrows = d.ni * d.ny, nb = (nrows + FW - 1) / FW;
#define L(P)                                                                                     \
  {                                                                                              \
    static int slots_ = 0;                                                                       \
    if (!slots_) slots_ = persistent_slots(kf_adj_fft_p<P>, fp_smem_adjfft(d));                  \
    launch_pdl(kf_adj_fft_p<P>, std::min(nb, slots_), FT, fp_smem_adjfft(d), st, d, in, mode);    \
  }
    switch (d.Px) {
      case 128: L(128); break;
      case 256: L(256); break;
      case 384: L(384); break;
      default: L(512); break;
    }
#undef L
    return PDF_OK;
  }
  if (ana2p_ok(d)) {
    const int ntiles = d.ni * ((d.ny + S2P_ROWS - 1) / S2P_ROWS);
#define L(Q)                                                                                          \
  kf_adj_ana_2p<Q><<<std::min(ntiles, ana2p_slots<Q>(d)), Col2p<Q>::NT, fp_smem_ana2p(d), st>>>(d, in, mode, \
                                                                                                  ntiles)
    switch (d.Px / 16) {
      case 8: L(8); break;
      case 16: L(16); break;
      default: L(24); break;
    }
#undef L
    return PDF_OK;
  }
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

// spectrum by column, natural frequency order: gc[cx][ky] = ghat[ky][kx(cx)]
__global__ void k_col_ghat(const float2* __restrict__ ghat, float2* __restrict__ gc, int Px, int Py) {
  const int ky = blockIdx.x * blockDim.x + threadIdx.x;
  const int cx = blockIdx.y;
  if (ky >= Py) return;
  gc[(size_t)cx * Py + ky] = ghat[(size_t)ky * Px + perm_to_freq(cx, Px / 32)];
}

pdf_status fp_col_ghat(const Dev& d, float2* gc, cudaStream_t st) {
  k_col_ghat<<<dim3((d.Py + 127) / 128, d.Px), 128, 0, st>>>(d.ghat, gc, d.Px, d.Py);
  pdf_count_launch(1);
  PDF_LAUNCHED("spectrum by column");
  return PDF_OK;
}

pdf_status fp_perm_ghat(const Dev& d, float2* gp, cudaStream_t st) {
  k_perm_ghat<<<dim3((d.Py + 127) / 128, d.Px), 128, 0, st>>>(d.ghat, gp, d.Px, d.Py);
  pdf_count_launch(1);
  PDF_LAUNCHED("permuted spectrum");
  return PDF_OK;
}
