// Bodies of the hot-path kernels as device functions over virtual block indices (bx, by).
// The stand-alone kernels in hotpath.cu / fastpath.cu call them with their blockIdx; the
// persistent solve kernel (persist.cu) calls them in a loop over virtual blocks between grid
// barriers.  Pointers are plain (no __restrict__, no __ldg on data that change during a
// persistent launch) so that every read of data written by other CTAs goes through the
// coherent path.  Equation references are those of the kernels' original comments.
#pragma once

#include "fftreg.cuh"
#include "problem.cuh"

#define FW 8            // warps per CTA of the register-FFT phases
#define FT (FW * 32)
#define FCOLS 16        // columns per CTA of the column convolution
#define GS_SUB 32
#define GS_TP 2
#define GS_TR 4
#define GSH_RT 32
#define GSH_TP 4
#define GSH_TN 4

struct KS {             // compensated FP32 sum
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c, t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

template <int P>
__device__ __forceinline__ void load_tw(float2* tw, const float2* g) {
  for (int i = threadIdx.x; i < P; i += blockDim.x) tw[i] = g[i];
}

template <int PX>
__device__ __forceinline__ void ph_synth_rowfft(const Dev& d, int bx, int by, float2* sm, const float2* alpha,
                                                float2* Jout, int do_fft) {
  constexpr int R = PX / 32;
    float2* tw = sm;
  float2* sa = sm + PX;
  const int p = by, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int y = bx * FW + warp;
  load_tw<PX>(tw, d.twx);
  for (int i = threadIdx.x; i < d.ky * d.kx; i += blockDim.x) sa[i] = alpha[(size_t)p * d.ky * d.kx + i];
  __syncthreads();
  if (y >= d.ny) return;
  float2 t0 = make_float2(0.f, 0.f), t1 = make_float2(0.f, 0.f);
  for (int jy = 0; jy < d.ky; ++jy) {
    const float2 w = __ldg(&d.wy[jy * d.ny + y]);
    if (lane < d.kx) t0 = cmac(t0, w, sa[jy * d.kx + lane]);
    if (lane + 32 < d.kx) t1 = cmac(t1, w, sa[jy * d.kx + lane + 32]);
  }
  float2 v[R];
#pragma unroll
  for (int m = 0; m < R; ++m) v[m] = make_float2(0.f, 0.f);
#pragma unroll 4
  for (int jx = 0; jx < d.kx; ++jx) {
    const float2 src = jx < 32 ? t0 : t1;
    const float2 T = make_float2(__shfl_sync(0xffffffffu, src.x, jx & 31), __shfl_sync(0xffffffffu, src.y, jx & 31));
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int x = lane + 32 * m;
      if (2 * m < R && x < d.nx) v[m] = cmac(v[m], T, __ldg(&d.wx[jx * d.nx + x]));
    }
  }
  const size_t row = (size_t)p * d.ny + y;
#pragma unroll
  for (int m = 0; m < R; ++m) {
    const int x = lane + 32 * m;
    if (2 * m < R && x < d.nx) Jout[row * d.nx + x] = v[m];
  }
  if (!do_fft) return;
  WarpFFT<PX>::forward(v, tw, lane);
#pragma unroll
  for (int k = 0; k < R; ++k) d.A[row * PX + k * 32 + lane] = v[k];
}


template <int PX>
__device__ __forceinline__ void ph_rowfft_field(const Dev& d, int bx, int by, float2* sm, const float2* in) {
  constexpr int R = PX / 32;
  float2* tw = sm;
  const int p = by, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int y = bx * FW + warp;
  load_tw<PX>(tw, d.twx);
  __syncthreads();
  if (y >= d.ny) return;
  const size_t row = (size_t)p * d.ny + y;
  float2 v[R];
#pragma unroll
  for (int m = 0; m < R; ++m) {
    const int x = lane + 32 * m;
    v[m] = (2 * m < R && x < d.nx) ? in[row * d.nx + x] : make_float2(0.f, 0.f);
  }
  WarpFFT<PX>::forward(v, tw, lane);
#pragma unroll
  for (int k = 0; k < R; ++k) d.A[row * PX + k * 32 + lane] = v[k];
}


template <int PX>
__device__ __forceinline__ void ph_rowifft_field(const Dev& d, int bx, int by, float2* sm, float2* out) {
  constexpr int R = PX / 32;
  float2* tw = sm;
  const int p = by, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int y = bx * FW + warp;
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
    if (2 * m < R && x < d.nx) out[row * d.nx + x] = v[m];
  }
}


template <int PY>
__device__ __forceinline__ void ph_colconv(const Dev& d, int bx, int by, float2* sm, int conj) {
  constexpr int R = PY / 32;
    float2* tw = sm;
  float2* tile = sm + PY;
  const int LS = d.ny + 1;
  const int p = by, c0 = bx * FCOLS;
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


template <int PX>
__device__ __forceinline__ void ph_rowifft_state(const Dev& d, int bx, float2* sm) {
  constexpr int R = PX / 32;
    __shared__ FF red_st[32];
  float2* tw = sm;
  float* part = (float*)(sm + PX);             // [3][FW][PX]
  float2* sR = (float2*)(part + 3 * FW * PX);  // [PX]
  const int y = bx, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
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
      if (2 * m < R && x < d.nx) {
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
  for (int m = 0; m < R / 2; ++m) {                    // slots m >= R/2 are padding (P >= 2 nx)
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
  const FF t = ff_block_sum(ff_add(FF{acc.s, 0.f}, -acc.c), red_st);
  if (threadIdx.x == 0) d.lpart[LP_STATE * PDF_LP_STRIDE + y] = t;
}


// Split state pass, part 1 (block = row y, incidence group g of at most FW incidences, one per
// warp): inverse row DFT -> G_D J, s = beta J + E_inc + G_D J (Eq. 6), and the group's per-pixel
// float-float sums of beta J conj(s) and |s|^2.
template <int PX>
__device__ __forceinline__ void ph_rowifft_sums(const Dev& d, int y, int g, float2* sm) {
  constexpr int R = PX / 32, H = PX / 2;
  float2* tw = sm;
  float* part = (float*)(sm + PX);             // [3][FW][PX / 2]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  load_tw<PX>(tw, d.twx);
  __syncthreads();
  const int p = g * FW + warp;
  if (p < d.ni) {
    const size_t row = (size_t)p * d.ny + y;
    float2 v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = d.A[row * PX + k * 32 + lane];
    WarpFFT<PX>::inverse(v, tw, lane);
#pragma unroll
    for (int m = 0; m < R / 2; ++m) {                  // slots m >= R/2 are padding (P >= 2 nx)
      const int x = lane + 32 * m;
      float3 c = make_float3(0.f, 0.f, 0.f);
      if (x < d.nx) {
        const size_t idx = row * d.nx + x;
        const float2 J = d.J[idx];
        const float2 s = cmul(d.beta, J) + d.einc[idx] + v[m];
        d.s[idx] = s;
        const float2 n = cmul(d.beta, cmulc(J, s));
        c = make_float3(n.x, n.y, cabs2(s));
      }
      part[(0 * FW + warp) * H + x] = c.x;
      part[(1 * FW + warp) * H + x] = c.y;
      part[(2 * FW + warp) * H + x] = c.z;
    }
  } else {
    for (int x = lane; x < H; x += 32)
      part[(0 * FW + warp) * H + x] = part[(1 * FW + warp) * H + x] = part[(2 * FW + warp) * H + x] = 0.f;
  }
  __syncthreads();
  for (int x = threadIdx.x; x < d.nx; x += blockDim.x) {
    FF a = FF{0.f, 0.f}, b = FF{0.f, 0.f}, c = FF{0.f, 0.f};
    for (int w = 0; w < FW; ++w) {
      a = ff_add(a, part[(0 * FW + w) * H + x]);
      b = ff_add(b, part[(1 * FW + w) * H + x]);
      c = ff_add(c, part[(2 * FW + w) * H + x]);
    }
    const size_t o = (size_t)g * d.M + (size_t)y * d.nx + x;
    d.sgA[o] = make_float4(a.hi, a.lo, b.hi, b.lo);
    d.sgB[o] = make_float2(c.hi, c.lo);
  }
}

// Split state pass, part 2 (thread per pixel): the group sums in group order -> R-hat (Eq. 6),
// chi-hat (Eq. 7), D and the clamp flag.
struct StatePix {
  float2 R, chi;
  float D;
  bool cl;
};
__device__ __forceinline__ StatePix state_combine_at(const Dev& d, int n) {
  FF a = FF{0.f, 0.f}, b = FF{0.f, 0.f}, c = FF{0.f, 0.f};
#pragma unroll 8
  for (int g = 0; g < d.nsg; ++g) {
    const float4 A = d.sgA[(size_t)g * d.M + n];
    const float2 B = d.sgB[(size_t)g * d.M + n];
    a = ff_add(a, FF{A.x, A.y});
    b = ff_add(b, FF{A.z, A.w});
    c = ff_add(c, FF{B.x, B.y});
  }
  StatePix o;
  o.D = c.hi + c.lo;
  o.R = make_float2((a.hi + a.lo) / o.D, (b.hi + b.lo) / o.D);
  o.chi = chi_of_R_f(o.R, d.beta, d.q_min, &o.cl);
  return o;
}
__device__ __forceinline__ void ph_state_combine(const Dev& d, int n) {
  if (n >= d.M) return;
  const StatePix o = state_combine_at(d, n);
  d.R[n] = o.R;
  d.chi[n] = o.chi;
  d.D[n] = o.D;
  d.clamp[n] = o.cl ? 1 : 0;
}

// Adjoint inputs and the row DFT of u.  FUSED_R: the state residual r = R-hat s - beta J (Eq. 15)
// is formed here rather than read back, and this block's float-float sum of |r|^2 goes to the
// L_State partials (slot by * gridDim.x + bx).
template <int PX, bool FUSED_R>
__device__ __forceinline__ void ph_adj_rowfft(const Dev& d, int bx, int by, float2* sm) {
  constexpr int R = PX / 32;
  __shared__ FF red_ar[32];
  float2* tw = sm;
  const int p = by, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int y = bx * FW + warp;
  load_tw<PX>(tw, d.twx);
  __syncthreads();
  KS acc;
  if (y < d.ny) {
    const float ke = d.invn[0];
    const float2 bc = cconj(d.beta);
    const size_t row = (size_t)p * d.ny + y;
    float2 v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int x = lane + 32 * m;
      v[m] = make_float2(0.f, 0.f);
      if (2 * m < R && x < d.nx) {
        const int n = y * d.nx + x;
        const size_t idx = row * d.nx + x;
        const float2 w = d.w[n], Rr = d.R[n];
        const float2 J = d.J[idx], s = d.s[idx];
        float2 r;
        if (FUSED_R) {
          r = cmul(Rr, s) - cmul(d.beta, J);
          acc.add(cabs2(r));
        } else {
          r = d.r[idx];
        }
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
  if (FUSED_R) {
    const FF t = ff_block_sum(ff_add(FF{acc.s, 0.f}, -acc.c), red_ar);
    if (threadIdx.x == 0) d.lpart[LP_STATE * PDF_LP_STRIDE + by * gridDim.x + bx] = t;
  }
}


template <int PX>
__device__ __forceinline__ void ph_adj_rowifft_ana(const Dev& d, int bx, int by, float2* sm, const float2* in,
                                                   int mode) {
  constexpr int R = PX / 32;
  float2* tw = sm;
  const int p = by, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int y = bx * FW + warp;
  load_tw<PX>(tw, d.twx);
  __syncthreads();
  if (y < d.ny) {
    const size_t row = (size_t)p * d.ny + y;
    float2 g[R];
    if (mode == 0) {
#pragma unroll
      for (int k = 0; k < R; ++k) g[k] = d.A[row * PX + k * 32 + lane];
      WarpFFT<PX>::inverse(g, tw, lane);
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int x = lane + 32 * m;
        if (2 * m < R && x < d.nx) {
          const size_t idx = row * d.nx + x;
          g[m] = d.fold ? g[m] + d.v[idx] : g[m] + d.v[idx] + d.gsh[idx];
        } else {
          g[m] = make_float2(0.f, 0.f);
        }
      }
    } else {
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int x = lane + 32 * m;
        g[m] = (2 * m < R && x < d.nx) ? in[row * d.nx + x] : make_float2(0.f, 0.f);
      }
    }
    // analysis along x: T2[p][y][jx] = sum_x g[x] conj(Wx[jx][x]), 16 coefficients per warp
    // reduce-scatter (lanes read Wx rows contiguously)
    for (int j0 = 0; j0 < d.kx; j0 += 16) {
      float2 acc[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] = make_float2(0.f, 0.f);
#pragma unroll
      for (int m = 0; m < R; ++m) {
        if (2 * m >= R || 32 * m >= d.nx) break;  // slots m >= R/2 are padding (P >= 2 nx)
        const int x = lane + 32 * m;
        if (2 * m < R && x < d.nx) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (j0 + j < d.kx) acc[j] = cmacc(acc[j], g[m], __ldg(&d.wx[(size_t)(j0 + j) * d.nx + x]));
        }
      }
      warp_reduce_scatter16(acc, lane);
      const int jx = j0 + (lane >> 1);
      if ((lane & 1) == 0 && jx < d.kx) d.T2[row * d.kx + jx] = acc[0];
    }
  }
  __syncthreads();
}


__device__ __forceinline__ void ph_gs_partial(const Dev& d, int bx, float2* sm, const float2* X, float2* part) {
    const int ls = GS_SUB + 1;
  float2* sX = sm;                     // [ni][ls]
  float2* sG = sX + d.ni * ls;         // [nr][ls]
  float2* sR = sG + d.nr * ls;         // reduction scratch [256][GS_TP*GS_TR]
  const int n0 = bx * d.gs_chunk;
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
            for (int b = 0; b < GS_TR; ++b) acc[a][b] = cmac(acc[a][b], gv[b], xv[a]);
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
          if (p < d.ni && r < d.nr) part[((size_t)bx * d.ni + p) * d.nr + r] = acc[a][b];
        }
    }
  }
}


__device__ __forceinline__ void ph_gs_reduce(const Dev& d, int bx, const float2* part, int nchunk, const float2* sub,
                                             float2* out, FF* lp) {
  __shared__ FF red_gr[32];
  const int o = bx * blockDim.x + threadIdx.x;
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
    const FF t = ff_block_sum(a2, red_gr);
    if (threadIdx.x == 0) lp[bx] = t;
  }
}


__device__ __forceinline__ void ph_gsh(const Dev& d, int bx, float2* sm, const float2* in, float2* out, float scale,
                                       int data_scale) {
  if (data_scale) scale = d.invn[1];     // 2 / ||E_sca||^2 of Eq. (16)'s gradient
    float2* sD = sm;                              // [ni][GSH_RT]
  float2* sG = sD + d.ni * GSH_RT;              // [GSH_RT][GSH_CHUNK + 1]
  float2* sR = sG + GSH_RT * (GSH_CHUNK + 1);   // [256][GSH_TP*GSH_TN]
  const int n0 = bx * GSH_CHUNK;
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
            for (int b = 0; b < GSH_TN; ++b) acc[a][b] = cmacc(acc[a][b], dv[a], gv[b]);
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


// The regularisers' cotangent c_chi on chi-hat carried to w = conj(d chi / d R) c_chi / D:
// chi = R / (beta (1 - R)) gives d chi / d R = 1 / (beta (1 - R)^2), zero where the clamp is active.
__device__ __forceinline__ float2 reg_w_at(const Dev& d, bool clamped, float2 R, float Dn, float2 cchi) {
  if (clamped) return make_float2(0.f, 0.f);
  const float2 q = make_float2(1.f - R.x, -R.y);
  const float2 dchi = cdivf(make_float2(1.f, 0.f), cmul(d.beta, cmul(q, q)));
  return (1.f / Dn) * cmul(cconj(dchi), cchi);
}
__device__ __forceinline__ float2 reg_w(const Dev& d, int n, float2 cchi) {
  if (d.clamp[n]) return make_float2(0.f, 0.f);
  return reg_w_at(d, false, d.R[n], d.D[n], cchi);
}

struct TVB {  // per-pixel pieces of the TV and bridge terms at one pixel
  float2 dx, dy;
  float t;          // TV magnitude
  float gx, gy;     // |chi| forward differences
  float sg, e;      // sigmoid and exp factors
};

// The TV and bridge pieces at pixel (y + oy, x + ox); `at(oy, ox)` reads chi there (global memory or
// a staged tile), so every caller shares one arithmetic.
template <class At>
__device__ __forceinline__ TVB tvb_at(const Dev& d, At at, int y, int x, int oy, int ox) {
  TVB o;
  const float2 c = at(oy, ox);
  const bool hx = x + ox + 1 < d.nx, hy = y + oy + 1 < d.ny;
  const float2 cx = hx ? at(oy, ox + 1) : c, cy = hy ? at(oy + 1, ox) : c;
  o.dx = hx ? cx - c : make_float2(0.f, 0.f);
  o.dy = hy ? cy - c : make_float2(0.f, 0.f);
  o.t = sqrtf(cabs2(o.dx) + cabs2(o.dy) + d.eps_tv);
  const float m = sqrtf(cabs2(c) + d.eps_abs);
  o.gx = hx ? sqrtf(cabs2(cx) + d.eps_abs) - m : 0.f;
  o.gy = hy ? sqrtf(cabs2(cy) + d.eps_abs) - m : 0.f;
  o.sg = 1.f / (1.f + expf(-(m - d.tau_b) / d.tau_b));
  o.e = expf(-(o.gx * o.gx + o.gy * o.gy));
  return o;
}

// What one pixel's TV and bridge terms give: their loss values, the cotangent pieces they put on
// the pixel itself (own) and on its right / lower neighbours' cotangents as seen from there (the
// neighbour's "left" / "upper" term).
struct RegPiece {
  float2 tv_own, tv_l, tv_u;  // -(dx + dy)/t;  dx/t;  dy/t
  float dm_own, dm_l, dm_u;   // bridge cotangent on |chi|: own;  -2 gx sg e;  -2 gy sg e
  float t, b;                 // TV and bridge loss values
};
__device__ __forceinline__ RegPiece reg_piece(const Dev& d, const TVB& o) {
  RegPiece r;
  r.tv_own = (-1.f / o.t) * (o.dx + o.dy);
  r.tv_l = (1.f / o.t) * o.dx;
  r.tv_u = (1.f / o.t) * o.dy;
  r.dm_own = o.sg * (1.f - o.sg) / d.tau_b * o.e + 2.f * (o.gx + o.gy) * o.sg * o.e;
  r.dm_l = -2.f * o.gx * o.sg * o.e;
  r.dm_u = -2.f * o.gy * o.sg * o.e;
  r.t = o.t;
  r.b = o.sg * o.e;
  return r;
}

// Regularisers of Eq. (17)-(19) at pixel value c from the pieces of its own, left (x > 0) and upper
// (y > 0) TV / bridge terms: sets lb, ltv, lbr and returns the cotangent on chi there.
__device__ __forceinline__ float2 reg_combine(const Dev& d, float2 c, const RegPiece& o, const RegPiece* l,
                                             const RegPiece* u, float& lb, float& ltv, float& lbr) {
  const float neg = fmaxf(-c.x, 0.f);
  lb = neg * neg;
  ltv = o.t;
  lbr = o.b;
  float2 ctv = o.tv_own;
  float dm = o.dm_own;
  if (l) {
    ctv = ctv + l->tv_l;
    dm += l->dm_l;
  }
  if (u) {
    ctv = ctv + u->tv_u;
    dm += u->dm_u;
  }
  const float m = sqrtf(cabs2(c) + d.eps_abs);
  float2 cchi = d.lam_tv * ctv + (d.lam_bridge * dm / m) * c;
  cchi.x += d.lam_bound * (-2.f * neg);
  return cchi;
}

// Regularisers at pixel (y, x) with every piece evaluated here (own, left, upper).
template <class At>
__device__ __forceinline__ float2 reg_pixel(const Dev& d, At at, int y, int x, float& lb, float& ltv, float& lbr) {
  const RegPiece o = reg_piece(d, tvb_at(d, at, y, x, 0, 0));
  RegPiece l, u;
  if (x > 0) l = reg_piece(d, tvb_at(d, at, y, x, 0, -1));
  if (y > 0) u = reg_piece(d, tvb_at(d, at, y, x, -1, 0));
  return reg_combine(d, at(0, 0), o, x > 0 ? &l : nullptr, y > 0 ? &u : nullptr, lb, ltv, lbr);
}


// Regularisers of Eq. (17)-(19) on the image `img` (chi-hat, or chi_CCO when the CCO is inside the
// loss) and their cotangent on it: written to `cot` when given, else carried on through
// chi = R / (beta (1 - R)) and R = N / D to w.
__device__ __forceinline__ void ph_reg(const Dev& d, int bx, const float2* img, float2* cot) {
  __shared__ FF red_rg[3 * 32];
  const int n = bx * blockDim.x + threadIdx.x;
  float lb = 0.f, ltv = 0.f, lbr = 0.f;
  if (n < d.M) {
    const int y = n / d.nx, x = n - y * d.nx;
    const float2* p = img + n;
    const int nx = d.nx;
    const float2 cchi = reg_pixel(d, [=](int oy, int ox) { return p[oy * nx + ox]; }, y, x, lb, ltv, lbr);
    if (cot) {
      cot[n] = cchi;
    } else {
      d.w[n] = reg_w(d, n, cchi);
    }
  }
  FF t3[3] = {ff_make(lb), ff_make(ltv), ff_make(lbr)};
  ff_block_sum_multi<3>(t3, red_rg);
  if (threadIdx.x == 0) {
    d.lpart[LP_BOUND * PDF_LP_STRIDE + bx] = t3[0];
    d.lpart[LP_TV * PDF_LP_STRIDE + bx] = t3[1];
    d.lpart[LP_BRIDGE * PDF_LP_STRIDE + bx] = t3[2];
  }
}


__device__ __forceinline__ void ph_ana_y(const Dev& d, int bx, int by, const float2* T2, float2* out) {
  __shared__ float2 part_ay[8][64];
  const int jy = bx, p = by, g = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float2* T = T2 + (size_t)p * d.ny * d.kx;
  float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
  for (int y = g; y < d.ny; y += 8) {
    const float2 w = __ldg(&d.wy[jy * d.ny + y]);
    if (lane < d.kx) a0 = cmacc(a0, T[(size_t)y * d.kx + lane], w);
    if (lane + 32 < d.kx) a1 = cmacc(a1, T[(size_t)y * d.kx + lane + 32], w);
  }
  part_ay[g][lane] = a0;
  part_ay[g][lane + 32] = a1;
  __syncthreads();
  if (threadIdx.x < d.kx) {
    float2 s = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 8; ++k) s = s + part_ay[k][threadIdx.x];
    out[((size_t)p * d.ky + jy) * d.kx + threadIdx.x] = s;
  }
}


__device__ __forceinline__ void ph_finalize(const Dev& d, double* terms, int n_state, int n_data, int n_reg, int* step_inc) {
  __shared__ FF red_fn[5 * 32];
  const int cnt[5] = {n_state, n_data, n_reg, n_reg, n_reg};
  FF a[5];
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    a[s] = FF{0.f, 0.f};
    for (int i = threadIdx.x; i < cnt[s]; i += blockDim.x) a[s] = ff_add(a[s], d.lpart[s * PDF_LP_STRIDE + i]);
  }
  ff_block_sum_multi<5>(a, red_fn);
  double tot[5];
#pragma unroll
  for (int s = 0; s < 5; ++s) tot[s] = ff_to_d(a[s]);
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


// Adam (torch.optim.Adam arithmetic, FP32) on element i of the real view, step t >= 1 given
// one element: parameter p, gradient g, moments m, v; sc = tab[t - 1] of the step
__device__ __forceinline__ void ph_adam_at(float& p, float g, float& m, float& v, float2 sc, float b1, float b2,
                                           float eps) {
  m = m + (1.f - b1) * (g - m);
  v = v * b2;
  v = v + ((1.f - b2) * g) * g;
  const float denom = sqrtf(v) / sc.y + eps;
  p = p + (-sc.x) * (m / denom);
}
// the step's table entry: lr / (1 - b1^t), sqrt(1 - b2^t), evaluated in FP64 on the host
__device__ __forceinline__ float2 ph_adam_sc(const float2* tab, int cap, int t) { return tab[min(max(t, 1), cap) - 1]; }
__device__ __forceinline__ void ph_adam(int i, float* p, const float* g, float* m, float* v, int n, int t,
                                        const float2* tab, int cap, float b1, float b2, float eps) {
  if (i >= n) return;
  const float2 sc = ph_adam_sc(tab, cap, t);
  float pi = p[i], mi = m[i], vi = v[i];
  ph_adam_at(pi, g[i], mi, vi, sc, b1, b2, eps);
  m[i] = mi;
  v[i] = vi;
  p[i] = pi;
}
