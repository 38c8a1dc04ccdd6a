// Cluster form of the whole Adam loop for small grids (padded length P = Px = Py <= 128).
//
// One thread-block cluster per incidence p; CTA k of the cluster owns grid rows
// [k RB, (k+1) RB) and padded columns [k CB, (k+1) CB).  Per iteration:
//   1. synthesis (Eq. 9): T' = Wy^T alpha_p for all rows, J on its rows, and the padded row DFT
//      of J at its own columns directly as T' what (what = the row DFT of the x basis), so the
//      forward transform needs no exchange; r_d,p = (G_S Phi) alpha_p - E_sca,p (Eq. 16)
//   2. column DFT, x G_D spectrum, inverse column DFT on its columns; rows < ny go to their row
//      owners' shared memory (DSMEM)                                                   | cluster barrier
//   3. inverse row DFT -> G_D J, s = beta J + E_inc + G_D J; this incidence's per-pixel
//      contributions beta J conj(s), |s|^2 to a global array (double-buffered by iteration) | GRID barrier
//   4. R-hat, chi-hat (Eq. 6, 7) for its rows and one halo row each side from the sums over all
//      incidences (when those sums are large, each CTA of the grid sums one slice of pixels and
//      writes R-hat, chi-hat there, and the CTAs read their rows after a second GRID barrier);
//      the TV / bridge pieces of Eq. 18-19 once per pixel; state residual (Eq. 15),
//      regulariser cotangent -> w; adjoint inputs u, v; row DFTs of u and v / Px -> column owners
//                                                                                     | cluster barrier
//   5. column convolution of u's data with the conjugated spectrum (G_D^H), plus v's data: the row
//      spectrum of dL/dJ = v + G_D^H u, kept at the column owner
//   6. analysis (Phi^H) of dL/dJ: the column data times conj(what) (the x-analysis of an inverse
//      row DFT) over its columns and all rows, then the y-analysis -> partial dL/d alpha_p to
//      every CTA of the cluster                                                        | cluster barrier
//   7. dL/d alpha_p = sum of the partials (same order in every CTA), Adam step on each CTA's copy
//      of alpha_p (identical in all CTAs of the cluster)
// With the coefficient-correcting network (Sec. 3, network architecture) the Adam variable is the
// network's weight vector theta instead: alpha_p = alpha_(0),p + Delta alpha(theta; x_p) is formed at
// the top of each iteration by the cluster (each CTA a slice of the first layer's and the output
// layer's rows, broadcast to every CTA of the cluster through DSMEM; the second layer likewise
// unless the CTA holds a shared-memory copy of W2), step 7 keeps dL/d alpha_p, and the chain rule
// runs per incidence (dL/dy_p, dz2_p from per-CTA partials over the output rows, dz1_p, from
// partials over the CTAs' rows of W2 without the copy) into a global array; after a GRID barrier
// every CTA of the grid forms a slice of dL/d theta as sums over the incidences (increasing p) and
// takes the Adam step on it, and a second GRID barrier publishes theta before the next forward pass.
// The data term goes through the folded operator G_S Phi, its receivers split over the cluster:
// CTA k holds rows r = k + C t, forms r_d,p there in phase 1 and adds (2/||E_sca||^2)(G_S Phi)^H r_d,p
// over those rows to its phase-6 partial.
// The loss value itself is not formed in the loop (the solver evaluates it once at the final
// iterate); the folded operator, the G_D spectrum slice, the bases and the row-DFT table stay in
// shared memory.  The formulas are those of the stand-alone kernels (FP32 with compensated sums);
// the data movement and the summation order differ.  Every wait is bounded: a grid barrier that
// runs out of time sets the error flag, after which no CTA waits at a grid barrier again; the loop
// runs to its end (cluster barriers need no timeout: a cluster is always co-scheduled) and the
// host reports the flag.  Co-residency of all clusters comes from the cooperative launch.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include <cooperative_groups.h>

#include "phases.cuh"

namespace cg = cooperative_groups;

constexpr int CL_NT = 512;                 // threads per CTA
constexpr int CL_NW = CL_NT / 32;

struct ClusterArgs {
  int iters, C, RB, CB;
  float2* alpha;          // [ni][ky][kx] in / out
  const float2* tab;
  int cap;
  float b1, b2, eps;
  float4* nd;             // [2][ni][M] per-incidence (Re N, Im N, D, unused)
  float4* rc;             // [M] (R-hat, chi-hat) when the sums are split over the grid
  float* dsg;             // [M] D, sign = clamp flag, likewise
  int sl, sg;             // pixels per CTA slice (0: every CTA sums its own rows), lanes per pixel
  unsigned* bar;
  int* err;               // 1: a grid barrier timed out; 2: launched with the wrong cluster shape
  long long wait_cap;     // clock cycles a grid-barrier wait may last
  // network form (H > 0): theta = W1 [H][D], b1 [H], W2 [H][H], b2 [H], W3 [D][H], b3 [D], D = 2 ky kx
  int H;
  float* theta;           // [np] in / out
  float* tm;              // [np] Adam moments of theta
  float* tv;
  const float* X;         // [ni][D] scaled network input
  const float* xs;        // [1] input scale s
  const float2* alpha0;   // [ni][ky][kx] alpha_(0)
  float* nvec;            // [ni][D + 4H] per incidence: dL/dy, h2, dz2, h1, dz1
  int wc;                 // 1: W2, b2 and each CTA's output rows of W3, b3 copied to shared memory
};

// Shared floats of the network form's weight copy (W2, b2, a CTA's output rows of W3 and b3).
static inline size_t cl_net_cache_floats(int H, int D, int C) {
  const size_t nsl = (size_t)((D + C - 1) / C);
  return H > 0 ? (size_t)H * H + H + nsl * H + nsl : 0;
}

// Shared floats of the network form: x_p [D], h1, h2, dz2, dz1 [H each], the cluster's dz2 and dz1
// partials [C][H] each, a reduction scratch [CL_NT], alpha_(0),p [D].
static inline size_t cl_net_floats(int H, int D, int C) {
  return H > 0 ? 2 * (size_t)D + 4 * (size_t)H + 2 * (size_t)C * H + CL_NT : 0;
}

__device__ __forceinline__ unsigned cl_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int cl_ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier on a monotonic counter: thread 0 adds one with release semantics and polls
// with acquire loads; bar.sync on both sides extends the ordering to the whole CTA.  Warps 1.. run
// idle_work (work that needs nothing from other CTAs) meanwhile.  Bounded: after `cap` clock
// cycles (checked on the first unsuccessful poll and every 32nd after it), or once any CTA has
// flagged a timeout, it stops waiting.
template <class F>
__device__ __forceinline__ void cl_grid_barrier(unsigned* bar, unsigned target, int* err, long long cap,
                                                F&& idle_work) {
  __syncthreads();
  if (threadIdx.x >= 32) idle_work();                                  // warps 1.. while thread 0 waits
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" : : "l"(bar) : "memory");
    if (cl_ld_relaxed(err) == 0) {
      const long long t0 = clock64();
      unsigned spins = 0;
      while (cl_ld_acquire(bar) < target) {
        if ((spins++ & 31u) == 0) {
          if (cl_ld_relaxed(err) != 0) break;
          if (clock64() - t0 >= cap) {
            atomicExch(err, 1);
            break;
          }
        }
      }
    }
  }
  __syncthreads();
}

// Phase timestamps (instrumented builds, -DPDF_PHASE_STAMPS): thread 0 of CTA 0 records the
// global timer right after each barrier of iterations CL_STAMP_IT0 .. CL_STAMP_IT0 + 3 (marks 0-14
// the loss and gradient steps; with the network also 16 after its forward pass, 15 after the chain
// rule's grid barrier and 17 after the Adam step on theta).  Other builds compile the marks to
// nothing.
#define CL_STAMP_IT0 5
#ifdef PDF_PHASE_STAMPS
__device__ unsigned long long g_cl_stamps[4][20];
#define CL_STAMP(i)                                                                             \
  do {                                                                                          \
    if (blockIdx.x == 0 && threadIdx.x == 0 && it >= CL_STAMP_IT0 && it < CL_STAMP_IT0 + 4) {   \
      unsigned long long t_;                                                                    \
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_));                                    \
      g_cl_stamps[it - CL_STAMP_IT0][i] = t_;                                                   \
    }                                                                                           \
  } while (0)
#else
#define CL_STAMP(i) \
  do {              \
  } while (0)
#endif


// One padded line per warp through the register FFT.  The transforms are called out of line (one
// copy of each in the kernel): the loop body then stays small enough for the instruction cache.
template <int P> struct Line {
  float2 v[P / 32];
};
// Every padded length here satisfies P >= 2n, so register slots m >= R/2 (points P/2 .. P-1) are
// zero on input and unused on output; stating that as constants lets the compiler drop that part
// of the first and last small DFTs.
template <int P>
__device__ __forceinline__ void zero_upper(float2 (&v)[P / 32]) {
#pragma unroll
  for (int m = P / 64; m < P / 32; ++m) v[m] = make_float2(0.f, 0.f);
}
// inverse transform of a line whose outputs are used for n <= P/2 points only
template <int P>
__device__ __noinline__ Line<P> line_inv(Line<P> x, const float2* __restrict__ tw, int lane) {
  WarpFFT<P>::inverse(x.v, tw, lane);
  zero_upper<P>(x.v);
  return x;
}
// circular convolution of a padded line (n <= P/2 points in and out) with the spectrum g (stored in
// the forward transform's order)
template <int P>
__device__ __noinline__ Line<P> line_conv(Line<P> x, Line<P> g, const float2* __restrict__ tw, int lane) {
  zero_upper<P>(x.v);
  WarpFFT<P>::forward(x.v, tw, lane);
#pragma unroll
  for (int k = 0; k < P / 32; ++k) x.v[k] = cmul(x.v[k], g.v[k]);
  WarpFFT<P>::inverse(x.v, tw, lane);
  zero_upper<P>(x.v);
  return x;
}

// two columns convolved together, or two lines transformed together (interleaved butterflies)
template <int P> struct Line2 {
  float2 v[2][P / 32];
};
template <int P>
__device__ __noinline__ Line2<P> line_conv2(Line2<P> x, Line2<P> g, const float2* __restrict__ tw, int lane) {
  zero_upper<P>(x.v[0]);
  zero_upper<P>(x.v[1]);
  WarpFFTn<P, 2>::forward(x.v, tw, lane);
#pragma unroll
  for (int l = 0; l < 2; ++l)
#pragma unroll
    for (int k = 0; k < P / 32; ++k) x.v[l][k] = cmul(x.v[l][k], g.v[l][k]);
  WarpFFTn<P, 2>::inverse(x.v, tw, lane);
  zero_upper<P>(x.v[0]);
  zero_upper<P>(x.v[1]);
  return x;
}
// forward transforms of two padded lines (n <= P/2 points in)
template <int P>
__device__ __noinline__ Line2<P> line_fwd2(Line2<P> x, const float2* __restrict__ tw, int lane) {
  zero_upper<P>(x.v[0]);
  zero_upper<P>(x.v[1]);
  WarpFFTn<P, 2>::forward(x.v, tw, lane);
  return x;
}

// Small complex product on shared-memory operands, C(m, n) = sum_k a(m, k) b(k, n), with
// a(m, k) = A[m sam + k sak] and b(k, n) = B[k sbk + n sbn] (conjugated when CA / CB).  Each output
// tile is held by KS adjacent lanes, lane s summing k = s, s + KS, ... in increasing k, and the KS
// partial sums are added across the lanes.  A tile is TM x TN outputs in registers: rows
// m = m0 + i tm, columns n = n0 + j tn (tm = ceil(M/TM), tn = ceil(N/TN)) for tile index
// m0 tn + n0, so a warp reads few distinct m and consecutive n, and every loaded a(m, k) or b(k, n)
// feeds TN or TM multiply-adds.  epi(m, n, value) receives each output once.
template <int TM, int TN, int KS, bool CA, bool CB, class Epi>
__device__ __forceinline__ void cl_cgemm(int M, int N, int K, const float2* __restrict__ A, int sam, int sak,
                                         const float2* __restrict__ B, int sbk, int sbn, Epi epi) {
  const int tm = (M + TM - 1) / TM, tn = (N + TN - 1) / TN, total = tm * tn * KS;
#pragma unroll 1
  for (int t0 = 0; t0 < total; t0 += CL_NT) {                         // same trip count in every warp
    if (t0 + (int)(threadIdx.x & ~31u) >= total) break;                 // whole warp past the end
    const int t = t0 + threadIdx.x, s = t % KS, tile = min(t / KS, tm * tn - 1);
    const int m0 = tile / tn, n0 = tile - m0 * tn;
    const float2* a[TM];
    const float2* b[TN];
#pragma unroll
    for (int i = 0; i < TM; ++i) a[i] = A + min(m0 + i * tm, M - 1) * sam;   // clamped: computed, not kept
#pragma unroll
    for (int j = 0; j < TN; ++j) b[j] = B + min(n0 + j * tn, N - 1) * sbn;
    float2 acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int k = s; k < K; k += KS) {
      float2 av[TM], bv[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) av[i] = CA ? cconj(a[i][k * sak]) : a[i][k * sak];
#pragma unroll
      for (int j = 0; j < TN; ++j) bv[j] = CB ? cconj(b[j][k * sbk]) : b[j][k * sbk];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = cmac(acc[i][j], av[i], bv[j]);
    }
#pragma unroll
    for (int o = 1; o < KS; o <<= 1)
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = acc[i][j] + shfl_xor2(acc[i][j], o);
    if (t < total && s == 0)
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j)
          if (m0 + i * tm < M && n0 + j * tn < N) epi(m0 + i * tm, n0 + j * tn, acc[i][j]);
  }
}

// Sums over the ni incidences of one pixel's contributions N = beta J conj(s), D = |s|^2 (stride
// M float4): compensated, eight loads in flight, pairwise within a batch.  Returns (Re N, Im N, D, 0).
__device__ __noinline__ float4 cl_pixel_sums(const float4* __restrict__ o, int ni, int M) {
  float nr_ = 0.f, ni_ = 0.f, dd = 0.f, cr = 0.f, ci = 0.f, cd = 0.f;
#pragma unroll 1
  for (int q0 = 0; q0 < ni; q0 += 8) {
    float4 b[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      b[j] = q0 + j < ni ? __ldcg(o + (size_t)(q0 + j) * M) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float sx = ((b[0].x + b[1].x) + (b[2].x + b[3].x)) + ((b[4].x + b[5].x) + (b[6].x + b[7].x));
    const float sy = ((b[0].y + b[1].y) + (b[2].y + b[3].y)) + ((b[4].y + b[5].y) + (b[6].y + b[7].y));
    const float sz = ((b[0].z + b[1].z) + (b[2].z + b[3].z)) + ((b[4].z + b[5].z) + (b[6].z + b[7].z));
    float t, yv;
    yv = sx - cr; t = nr_ + yv; cr = (t - nr_) - yv; nr_ = t;
    yv = sy - ci; t = ni_ + yv; ci = (t - ni_) - yv; ni_ = t;
    yv = sz - cd; t = dd + yv; cd = (t - dd) - yv; dd = t;
  }
  return make_float4(nr_ - cr, ni_ - ci, dd - cd, 0.f);
}

// Network weights are read through L2 (GLB: theta changes between iterations) or from this CTA's
// shared-memory copy of them.
template <bool GLB>
__device__ __forceinline__ float cl_net_ld(const float* p) {
  if (GLB) return __ldcg(p);
  return *p;
}
__device__ __forceinline__ void cl_cp_async4(float* smem, const float* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}

// Network form: out[r0 + i] = sum_c W[i cols + c] v[c] + bias[i] for i < nrow (W, bias: from row r0
// on), a warp per row (lanes over c, c = lane + 32 u in increasing u, a butterfly warp sum);
// epi(r0 + i, value) on lane 0.  Each warp takes NR of its rows at once and issues all their loads
// (CPL per lane and row, in chunks of 32 CPL columns) before the multiply-adds, so the round trips
// overlap.
template <bool GLB, int CPL, int NR, class Epi>
__device__ __forceinline__ void cl_net_rows(const float* __restrict__ W, const float* __restrict__ bias, int cols,
                                            const float* v, int r0, int nrow, Epi epi) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll 1
  for (int ib = warp; ib < nrow; ib += CL_NW * NR) {
    float acc[NR], bv[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      acc[j] = 0.f;
      bv[j] = ib + CL_NW * j < nrow ? cl_net_ld<GLB>(&bias[ib + CL_NW * j]) : 0.f;
    }
#pragma unroll 1
    for (int c0 = 0; c0 < cols; c0 += 32 * CPL) {
      float w[NR][CPL];
#pragma unroll
      for (int j = 0; j < NR; ++j)
#pragma unroll
        for (int u = 0; u < CPL; ++u) {
          const int i = ib + CL_NW * j, c = c0 + lane + 32 * u;
          w[j][u] = i < nrow && c < cols ? cl_net_ld<GLB>(&W[(size_t)i * cols + c]) : 0.f;
        }
#pragma unroll
      for (int j = 0; j < NR; ++j)
#pragma unroll
        for (int u = 0; u < CPL; ++u) {
          const int c = c0 + lane + 32 * u;
          if (c < cols) acc[j] = fmaf(w[j][u], v[c], acc[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      float t = acc[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      const int i = ib + CL_NW * j;
      if (lane == 0 && i < nrow) epi(r0 + i, t + bv[j]);
    }
  }
}
// Network form: out[c] = sum over i < nrow of W[i cols + c] v[i] for c < cols <= CL_NT (W, v: from
// row r0 on): thread (grp, c) sums i = grp, grp + G, ... in increasing i (G = CL_NT / cols), 16
// loads in flight at a time, the G partials are added in group order and epi(c, value) runs on the
// threads c < cols.  Ends with a CTA barrier.
template <bool GLB, class Epi>
__device__ __forceinline__ void cl_net_cols(const float* __restrict__ W, int cols, const float* v, int nrow,
                                            float* red, Epi epi) {
  const int G = CL_NT / cols, t = threadIdx.x, c = t % cols, grp = t / cols;
  if (grp < G) {
    float acc = 0.f;
#pragma unroll 1
    for (int ib = grp; ib < nrow; ib += 16 * G) {
      float w[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int i = ib + u * G;
        w[u] = i < nrow ? cl_net_ld<GLB>(&W[(size_t)i * cols + c]) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int i = ib + u * G;
        if (i < nrow) acc = fmaf(w[u], v[i], acc);
      }
    }
    red[grp * cols + c] = acc;
  }
  __syncthreads();
  if (t < cols) {
    float sum = red[c];
#pragma unroll 1
    for (int q = 1; q < G; ++q) sum += red[q * cols + c];
    epi(c, sum);
  }
  __syncthreads();
}

template <int P>
__global__ void __launch_bounds__(CL_NT, 1) k_cluster_solve(Dev d, ClusterArgs a) {
  constexpr int R = P / 32;
  cg::cluster_group cl = cg::this_cluster();
  const int C = a.C, RB = a.RB, CB = a.CB;
  // a launch without the cluster shape this kernel was built for must not touch peer memory
  if ((int)cl.num_blocks() != C || (int)gridDim.x != d.ni * C || (int)blockDim.x != CL_NT) {
    if (threadIdx.x == 0) atomicExch(a.err, 2);
    return;
  }
  const int k = (int)cl.block_rank();
  const int p = blockIdx.x / C;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nx = d.nx, ny = d.ny, kx = d.kx, ky = d.ky, nr = d.nr, M = d.M, ni = d.ni;
  const int y0 = k * RB, c0 = k * CB;
  // RB, CB: rows and padded columns per CTA (array strides; the last CTA may own fewer when C does
  // not divide ny or P): this CTA owns nrow rows and ncol columns
  const int nrow = min(RB, ny - y0), ncol = min(CB, P - c0);
  const int LS = ny + 1;
  const int NA = ky * kx;
  const int GP = RB * nx;                    // pixel capacity per CTA
  const int HP = (RB + 2) * nx;              // with one halo row above and below
  const int TP = (RB + 1) * nx;              // rows y0-1 .. y0+RB-1
  const int GPk = nrow * nx, HPk = (nrow + 2) * nx, TPk = (nrow + 1) * nx;   // this CTA's counts
  // ---- shared memory carve-up ----
  extern __shared__ float2 sm[];
  float2* tw = sm;                           // [P]
  // The two exchanges write into buffers laid out as the sender's warp holds the data, so that
  // each warp's remote stores are contiguous: a column owner's warp holds one column (lanes along
  // y) and writes into the row owners' rowT[c][yl]; a row owner's warp holds one row (lanes along
  // c) and writes into the column owners' colT[y][lc].  Odd strides keep local reads of the other
  // direction on distinct banks.
  const int RS = (RB + 1) | 1, SC = CB | 1;   // odd strides (RB + 1 or RB + 2, CB or CB + 1)
  float2* rowT = tw + P;                     // [P][RS] row spectra of own rows, column by column
  float2* colb = rowT + P * RS;              // [CB][LS] row DFT of J at own columns (phases 1-2)
  float2* colT = colb + CB * LS;             // [ny][SC] row DFT of u at own columns, then of dL/dJ (4-6)
  float2* colV = colT + ny * SC;             // [ny][SC] row DFT of v / Px at own columns (4-5)
  float2* Js = colV + ny * SC;               // [GP]
  float2* ss = Js + GP;                      // [GP] s
  float2* Es = ss + GP;                      // [GP]
  float2* vs = Es + GP;                      // [GP] v + G_S^H term
  float2* Rh = vs + GP;                      // [HP] R-hat, rows y0-1 .. y0+RB
  float2* Ch = Rh + HP;                      // [HP] chi-hat
  float2* al = Ch + HP;                      // [NA] alpha_p
  const int nscr = 2 * GP + HP + 2 * TP;     // phase-4 scratch (floats), shares space with gpart
  const int NU = max(C * NA, (nscr + 1) / 2);
  float2* gpart = al + NA;                   // [C][NA] partial y-analyses of all ranks (phases 6-7)
  float* Dl = (float*)gpart;                 // [GP] D, sign = clamp flag                 (phase 4)
  float* mgs = Dl + GP;                      // [HP] sqrt(|chi|^2 + eps_abs)              (phase 4)
  float* itv = mgs + HP;                     // [TP] 1 / t (TV magnitude)                 (phase 4)
  float* sge = itv + TP;                     // [TP] sigmoid * exp (bridge term)          (phase 4)
  float* sgs = sge + TP;                     // [GP] sigmoid, own rows                    (phase 4)
  const int NRK = (nr - k + C - 1) / C;      // receivers r = k + C t owned by this CTA
  float2* rd = gpart + NU;                   // [NRK] data residual r_d,p at own receivers
  float2* es = rd + nr;                      // [NRK]
  float2* Tall = es + nr;                    // [ny][kx] T' of all rows (phase 1), x-analysis (phase 6)
  float2* wyf = Tall + ny * kx;              // [ky][ny] y basis
  float2* whs = wyf + ky * ny;               // [CB][kx] row DFT of the x basis at this CTA's columns
  float2* ghs = whs + kx * CB;               // [CB][P] this CTA's columns of the G_D spectrum
  float2* wxs = ghs + CB * P;                // [kx][nx] x basis
  float2* gdv = wxs + kx * nx;               // [NA] (G_S Phi)^H r_d at own receivers
  float* am = (float*)(gdv + NA);            // [2 NA]
  float* av = am + 2 * NA;                   // [2 NA]
  float2* gsf = (float2*)(av + 2 * NA);      // [NRK][NA] folded receiver operator, own receivers
  // network form (the same offset in every CTA: after the largest receiver share)
  const int H = a.H, D = 2 * NA;
  float* xsn = (float*)(gsf + (size_t)((nr + C - 1) / C) * NA);   // [D] x_p
  float* h1s = xsn + D;                      // [H]
  float* h2s = h1s + H;                      // [H]
  float* dz2s = h2s + H;                     // [H]
  float* dz1s = dz2s + H;                    // [H]
  float* npart = dz1s + H;                   // [C][H] dz2 partials of the cluster's CTAs
  float* npart2 = npart + C * H;             // [C][H] dz1 partials (without the weight copy)
  float* nred = npart2 + C * H;              // [CL_NT]
  float* a0n = nred + CL_NT;                 // [D] alpha_(0),p: real parts, then imaginary parts
  // with a.wc: this CTA's copy of W2, b2 and of its output rows' W3, b3 (read in the forward pass and
  // again in the chain rule of the same iteration)
  const int nsl = (D + C - 1) / C, n0 = min(D, k * nsl), nrw = min(D, n0 + nsl) - n0;
  float* cW2 = a0n + D;                      // [H][H]
  float* cb2 = cW2 + H * H;                  // [H]
  float* cW3 = cb2 + H;                      // [nsl][H] rows n0 ..
  float* cb3 = cW3 + nsl * H;                // [nsl]
  float* dys = av;                           // [D] dL/dy_p (av is Adam state of alpha only)

  // ---- one-time loads ----
#pragma unroll 1
  for (int i = threadIdx.x; i < P; i += CL_NT) tw[i] = d.twx[i];
#pragma unroll 1
  for (int i = threadIdx.x; i < NA; i += CL_NT) {
    al[i] = a.alpha[(size_t)p * NA + i];
    am[2 * i] = am[2 * i + 1] = 0.f;
    av[2 * i] = av[2 * i + 1] = 0.f;
  }
#pragma unroll 1
  for (int i = threadIdx.x; i < GPk; i += CL_NT) Es[i] = d.einc[(size_t)p * M + y0 * nx + i];
#pragma unroll 1
  for (int t = threadIdx.x; t < NRK; t += CL_NT) es[t] = d.esca[(size_t)p * nr + k + C * t];
#pragma unroll 1
  for (int i = threadIdx.x; i < ky * ny; i += CL_NT) wyf[i] = d.wy[i];
#pragma unroll 1
  for (int i = threadIdx.x; i < kx * CB; i += CL_NT) {
    const int lc = i / kx, jx = i - lc * kx;
    whs[i] = lc < ncol ? d.what[(size_t)jx * P + c0 + lc] : make_float2(0.f, 0.f);
  }
#pragma unroll 1
  for (int i = threadIdx.x; i < ncol * P; i += CL_NT) ghs[i] = d.ghat_perm[(size_t)c0 * P + i];
#pragma unroll 1
  for (int i = threadIdx.x; i < kx * nx; i += CL_NT) wxs[i] = d.wx[i];
#pragma unroll 1
  for (int i = threadIdx.x; i < NRK * NA; i += CL_NT) {
    const int t = i / NA, j = i - t * NA;
    gsf[i] = d.gsf[(size_t)(k + C * t) * NA + j];
  }
  float net_s = 1.f;
  if (H > 0) {
#pragma unroll 1
    for (int i = threadIdx.x; i < D; i += CL_NT) {
      xsn[i] = a.X[(size_t)p * D + i];
      const int re = i < NA ? 0 : 1, j = i - re * NA;
      a0n[i] = reinterpret_cast<const float*>(a.alpha0)[((size_t)p * NA + j) * 2 + re];
    }
    net_s = a.xs[0];
  }
  const float ke = d.invn[0], ks = d.invn[1];
  const float2 beta = d.beta, bc = cconj(d.beta);
  const unsigned nblocks = gridDim.x;
  unsigned nbar = 0;                         // grid barriers passed (targets nbar * nblocks)
  // theta's offsets in the flat vector
  const size_t oW1 = 0, ob1 = (size_t)H * D, oW2 = ob1 + H, ob2 = oW2 + (size_t)H * H, oW3 = ob2 + H,
               ob3 = oW3 + (size_t)D * H, npar = ob3 + D;
  cl.sync();

  for (int it = 0; it < a.iters; ++it) {
    CL_STAMP(0);
    float4* nd = a.nd + (size_t)(it & 1) * ni * M;
    if (H > 0) {
      // ===== 0. alpha_p = alpha_(0),p + Delta alpha(theta; x_p) =====
      const float* th = a.theta;
      if (a.wc) {                            // W2, b2 and the output rows' W3, b3 in one round of copies
#pragma unroll 1
        for (int i = threadIdx.x; i < H * H; i += CL_NT) cl_cp_async4(cW2 + i, th + oW2 + i);
#pragma unroll 1
        for (int i = threadIdx.x; i < nrw * H; i += CL_NT) cl_cp_async4(cW3 + i, th + oW3 + (size_t)n0 * H + i);
        if ((int)threadIdx.x < H) cl_cp_async4(cb2 + threadIdx.x, th + ob2 + threadIdx.x);
#pragma unroll 1
        for (int i = threadIdx.x; i < nrw; i += CL_NT) cl_cp_async4(cb3 + i, th + ob3 + n0 + i);
        asm volatile("cp.async.commit_group;" ::: "memory");
      }
      const int hs = (H + C - 1) / C, h0 = min(H, k * hs), nh = min(H, h0 + hs) - h0;
      cl_net_rows<true, 16, 1>(th + oW1 + (size_t)h0 * D, th + ob1 + h0, D, xsn, h0, nh, [&](int h, float v) {
        v = fmaxf(v, 0.f);
#pragma unroll 1
        for (int q = 0; q < C; ++q) cl.map_shared_rank(h1s, q)[h] = v;
      });
      if (a.wc) asm volatile("cp.async.wait_group 0;" ::: "memory");
      cl.sync();
      auto out_alpha = [&](int n, float v) {
        const int re = n < NA ? 0 : 1, j = n - re * NA;
        const float o = a0n[n] + v / net_s;
#pragma unroll 1
        for (int q = 0; q < C; ++q) reinterpret_cast<float*>(cl.map_shared_rank(al, q))[2 * j + re] = o;
      };
      if (a.wc) {
        cl_net_rows<false, 2, 4>(cW2, cb2, H, h1s, 0, H, [&](int h, float v) { h2s[h] = fmaxf(v, 0.f); });
        __syncthreads();
        cl_net_rows<false, 2, 8>(cW3, cb3, H, h2s, n0, nrw, out_alpha);
      } else {
        // without the copy, h2 is split over the cluster as h1 is (each CTA reads its rows of W2 once)
        cl_net_rows<true, 2, 4>(th + oW2 + (size_t)h0 * H, th + ob2 + h0, H, h1s, h0, nh, [&](int h, float v) {
          v = fmaxf(v, 0.f);
#pragma unroll 1
          for (int q = 0; q < C; ++q) cl.map_shared_rank(h2s, q)[h] = v;
        });
        cl.sync();
        cl_net_rows<true, 2, 8>(th + oW3 + (size_t)n0 * H, th + ob3 + n0, H, h2s, n0, nrw, out_alpha);
      }
      cl.sync();
      CL_STAMP(16);
    }
    // ===== 1. synthesis (Eq. 9): T' of all rows, J on own rows, the padded row DFT of J on own columns =====
    // T'[y][jx] = sum_jy Wy[jy][y] al[jy][jx] (low threads) while the top warps form r_d
    cl_cgemm<2, 2, 1, false, false>(ny, kx, ky, wyf, 1, ny, al, kx, 1,
                                 [&](int y, int jx, float2 v) { Tall[y * kx + jx] = v; });
#pragma unroll 1
    for (int t = CL_NW - 1 - warp; t < NRK; t += CL_NW) {               // r_d,p = (G_S Phi) alpha_p - E_sca,p, own receivers
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
      for (int j = lane; j < NA; j += 32) acc = cmac(acc, gsf[t * NA + j], al[j]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc = acc + shfl_xor2(acc, o);
      if (lane == 0) rd[t] = acc - es[t];
    }
    __syncthreads();
    CL_STAMP(1);
    CL_STAMP(2);
    cl_cgemm<2, 2, 1, false, false>(ny, ncol, kx, Tall, kx, 1, whs, 1, kx,            // row DFT of J at own columns: T' what
                                 [&](int y, int lc, float2 v) { colb[lc * LS + y] = v; });
    __syncthreads();
    CL_STAMP(3);
    // ===== 2. column convolution, results back to row owners =====
#pragma unroll 1
    for (int lc = warp; lc < ncol; lc += 2 * CL_NW) {                  // columns lc and lc + NW together
      const int lc2 = lc + CL_NW;
      if (lc2 < ncol) {
        Line2<P> G, L;
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          const int c = l ? lc2 : lc;
#pragma unroll
          for (int kk = 0; kk < R; ++kk) G.v[l][kk] = ghs[c * P + kk * 32 + lane];
#pragma unroll
          for (int m = 0; m < R; ++m) {
            const int y = lane + 32 * m;
            L.v[l][m] = y < ny ? colb[c * LS + y] : make_float2(0.f, 0.f);
          }
        }
        L = line_conv2<P>(L, G, tw, lane);
#pragma unroll
        for (int m = 0; m < R; ++m) {                                    // to the row owners
          const int y = lane + 32 * m;
          if (y < ny) {
            float2* dst = cl.map_shared_rank(rowT, y / RB) + y % RB;
            dst[(c0 + lc) * RS] = L.v[0][m];
            dst[(c0 + lc2) * RS] = L.v[1][m];
          }
        }
      } else {
        const float2* g = ghs + lc * P;
        Line<P> G, L;
#pragma unroll
        for (int kk = 0; kk < R; ++kk) G.v[kk] = g[kk * 32 + lane];
#pragma unroll
        for (int m = 0; m < R; ++m) {
          const int y = lane + 32 * m;
          L.v[m] = y < ny ? colb[lc * LS + y] : make_float2(0.f, 0.f);
        }
        L = line_conv<P>(L, G, tw, lane);
#pragma unroll
        for (int m = 0; m < R; ++m) {
          const int y = lane + 32 * m;
          if (y < ny) cl.map_shared_rank(rowT, y / RB)[(c0 + lc) * RS + y % RB] = L.v[m];
        }
      }
    }
    // J on own pixels is needed only after the exchange: it runs between this CTA's arrival at the
    // cluster barrier and its wait
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    cl_cgemm<2, 2, 1, false, false>(nrow, nx, kx, Tall + y0 * kx, kx, 1, wxs, nx, 1, // J = T' Wx on own pixels
                                    [&](int yl, int x, float2 v) { Js[yl * nx + x] = v; });
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
    CL_STAMP(4);
    // ===== 3. inverse row DFT, s, per-incidence contributions, partial G_S J_p =====
#pragma unroll 1
    for (int yl = warp; yl < nrow; yl += CL_NW) {
      Line<P> L;
#pragma unroll
      for (int kk = 0; kk < R; ++kk) L.v[kk] = rowT[(kk * 32 + lane) * RS + yl];
      L = line_inv<P>(L, tw, lane);
#pragma unroll
      for (int m = 0; m < R; ++m) {                                      // G_D J back in place (x < nx)
        const int x = lane + 32 * m;
        if (x < nx) rowT[x * RS + yl] = L.v[m];
      }
    }
    __syncthreads();
    CL_STAMP(5);
#pragma unroll 1
    for (int i = threadIdx.x; i < GPk; i += CL_NT) {
      const int yl = i / nx, x = i - yl * nx;
      const float2 J = Js[i];
      const float2 s = cmul(beta, J) + Es[i] + rowT[x * RS + yl];
      ss[i] = s;
      const float2 n = cmul(beta, cmulc(J, s));
      __stcg(&nd[(size_t)p * M + y0 * nx + i], make_float4(n.x, n.y, cabs2(s), 0.f));
    }
    cl_grid_barrier(a.bar, ++nbar * nblocks, a.err, a.wait_cap, [&] {
#pragma unroll 1
      for (int i = threadIdx.x - 32; i < NA; i += CL_NT - 32) {            // (G_S Phi)^H r_d, own receivers (Eq. 16)
        float2 g = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int t = 0; t < NRK; ++t) g = cmacc(g, rd[t], gsf[t * NA + i]);
        gdv[i] = g;
      }
    });
    CL_STAMP(6);
    // ===== 4. R-hat, chi-hat (own rows + halo), residuals, regulariser cotangent, adjoint inputs =====
    if (a.sl > 0) {
      // Sums over incidences split over the grid: CTA b sums pixels [b sl, (b+1) sl), each pixel
      // over sg adjacent lanes (lane g: incidences 8g .. 8g+7, all loads in flight at once, pairwise
      // sum) whose partial sums are added in float-float across the lanes, and writes R-hat,
      // chi-hat and the signed D there; after a second grid barrier every CTA reads its rows + halo.
      const int G = a.sg, gl = threadIdx.x & (G - 1), pix0 = blockIdx.x * a.sl;
      const int pix1 = min(pix0 + a.sl, M);
#pragma unroll 1
      for (int j0 = pix0; j0 < pix1; j0 += CL_NT / G) {
        if (j0 + (int)(threadIdx.x & ~31u) / G >= pix1) break;           // whole warp past the end
        const int j = j0 + (int)threadIdx.x / G;
        const bool on = j < pix1;
        float4 b[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          const int q = gl * 8 + jj;
          b[jj] = on && q < ni ? __ldcg(nd + (size_t)q * M + j) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        FF f[3] = {ff_make(((b[0].x + b[1].x) + (b[2].x + b[3].x)) + ((b[4].x + b[5].x) + (b[6].x + b[7].x))),
                   ff_make(((b[0].y + b[1].y) + (b[2].y + b[3].y)) + ((b[4].y + b[5].y) + (b[6].y + b[7].y))),
                   ff_make(((b[0].z + b[1].z) + (b[2].z + b[3].z)) + ((b[4].z + b[5].z) + (b[6].z + b[7].z)))};
#pragma unroll 1
        for (int o = 1; o < G; o <<= 1)
#pragma unroll
          for (int c = 0; c < 3; ++c) f[c] = ff_add(f[c], ff_shfl_xor(f[c], o));
        if (on && gl == 0) {
          const float Df = f[2].hi + f[2].lo;
          const float2 Rv = make_float2((f[0].hi + f[0].lo) / Df, (f[1].hi + f[1].lo) / Df);
          bool clamped;
          const float2 chi = chi_of_R_f(Rv, beta, d.q_min, &clamped);
          __stcg(a.rc + j, make_float4(Rv.x, Rv.y, chi.x, chi.y));
          __stcg(a.dsg + j, clamped ? -Df : Df);
        }
      }
      cl_grid_barrier(a.bar, ++nbar * nblocks, a.err, a.wait_cap, [] {});
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
      for (int i0 = threadIdx.x; i0 < HPk; i0 += 4 * CL_NT) {            // own rows + halo, four loads in flight
        float4 v[4];
        float dv[4];
        bool ok[4], own[4];
        int ix[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + u * CL_NT, hy = i / nx, x = i - hy * nx, y = y0 + hy - 1;
          ok[u] = i < HPk && y >= 0 && y < ny;
          own[u] = ok[u] && hy >= 1 && hy <= nrow;
          ix[u] = y * nx + x;
          v[u] = ok[u] ? __ldcg(a.rc + ix[u]) : z4;
          dv[u] = own[u] ? __ldcg(a.dsg + ix[u]) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (ok[u]) {
            const int i = i0 + u * CL_NT;
            const float2 chi = make_float2(v[u].z, v[u].w);
            Rh[i] = make_float2(v[u].x, v[u].y);
            Ch[i] = chi;
            mgs[i] = sqrtf(cabs2(chi) + d.eps_abs);
            if (own[u]) Dl[i - nx] = dv[u];
          }
      }
    } else {
#pragma unroll 1
      for (int i = threadIdx.x; i < HPk; i += CL_NT) {
        const int hy = i / nx, x = i - hy * nx, y = y0 + hy - 1;
        if (y < 0 || y >= ny) continue;
        const float4 sm4 = cl_pixel_sums(nd + (size_t)y * nx + x, ni, M);
        const float Df = sm4.z;
        const float2 Rv = make_float2(sm4.x / Df, sm4.y / Df);
        bool clamped;
        const float2 chi = chi_of_R_f(Rv, beta, d.q_min, &clamped);
        Rh[i] = Rv;
        Ch[i] = chi;
        mgs[i] = sqrtf(cabs2(chi) + d.eps_abs);
        if (hy >= 1 && hy <= nrow) Dl[(hy - 1) * nx + x] = clamped ? -Df : Df;
      }
    }
    __syncthreads();
    CL_STAMP(7);
    // TV and bridge pieces at (y, x) for rows y0-1 .. y0+RB-1, each computed once (Eq. 18, 19)
#pragma unroll 1
    for (int i = threadIdx.x; i < TPk; i += CL_NT) {
      const int hy = i / nx, x = i - hy * nx, y = y0 + hy - 1;
      if (y < 0) continue;
      const float2 c = Ch[i];
      const bool hx = x + 1 < nx, hyn = y + 1 < ny;
      const float2 dx = hx ? Ch[i + 1] - c : make_float2(0.f, 0.f);
      const float2 dy = hyn ? Ch[i + nx] - c : make_float2(0.f, 0.f);
      const float t = sqrtf(cabs2(dx) + cabs2(dy) + d.eps_tv);
      const float m = mgs[i];
      const float gx = hx ? mgs[i + 1] - m : 0.f;
      const float gy = hyn ? mgs[i + nx] - m : 0.f;
      const float sg = 1.f / (1.f + expf(-(m - d.tau_b) / d.tau_b));
      const float e = expf(-(gx * gx + gy * gy));
      itv[i] = 1.f / t;
      sge[i] = sg * e;
      if (hy >= 1) sgs[i - nx] = sg;
    }
    __syncthreads();
    CL_STAMP(8);
    // state residual, cotangent on chi -> w, u (into rowT) and v (into vs)
#pragma unroll 1
    for (int li = threadIdx.x; li < GPk; li += CL_NT) {
      const int yl = li / nx, x = li - yl * nx, y = y0 + yl;
      const int hc = li + nx;                                            // index in the halo-row arrays
      const float2 Rv = Rh[hc], c = Ch[hc];
      const float2 J = Js[li], s = ss[li];
      const float2 r = cmul(Rv, s) - cmul(beta, J);
      const float neg = fmaxf(-c.x, 0.f);
      const bool hx = x + 1 < nx, hyn = y + 1 < ny;
      const float mv = mgs[hc];
      const float2 dxo = hx ? Ch[hc + 1] - c : make_float2(0.f, 0.f);
      const float2 dyo = hyn ? Ch[hc + nx] - c : make_float2(0.f, 0.f);
      const float gxo = hx ? mgs[hc + 1] - mv : 0.f;
      const float gyo = hyn ? mgs[hc + nx] - mv : 0.f;
      const float sg = sgs[li], sgev = sge[hc];
      float2 ctv = (-itv[hc]) * (dxo + dyo);
      float dm = sgev * (1.f - sg) / d.tau_b + 2.f * (gxo + gyo) * sgev;
      if (x > 0) {
        ctv = ctv + itv[hc - 1] * (c - Ch[hc - 1]);
        dm -= 2.f * (mv - mgs[hc - 1]) * sge[hc - 1];
      }
      if (y > 0) {
        ctv = ctv + itv[hc - nx] * (c - Ch[hc - nx]);
        dm -= 2.f * (mv - mgs[hc - nx]) * sge[hc - nx];
      }
      float2 cchi = d.lam_tv * ctv + (d.lam_bridge * dm / mv) * c;
      cchi.x += d.lam_bound * (-2.f * neg);
      const float Dv = Dl[li];
      float2 w = make_float2(0.f, 0.f);
      if (Dv > 0.f) {
        const float2 q = make_float2(1.f - Rv.x, -Rv.y);
        const float2 dchi = cdivf(make_float2(1.f, 0.f), cmul(beta, cmul(q, q)));
        w = (1.f / Dv) * cmul(cconj(dchi), cchi);
      }
      const float2 wc = cconj(w);
      const float2 cs = cmul(cmul(wc, beta), J) - (2.f * cmul(wc, Rv).x) * s;
      rowT[x * RS + yl] = ke * cmulc(r, Rv) + cs;                        // u
      const float2 omr = make_float2(1.f - Rv.x, Rv.y);
      vs[li] = ke * cmul(cmul(make_float2(-bc.x, -bc.y), omr), r) + cmul(bc, cmul(w, s) + cs);   // v
    }
    __syncthreads();
    CL_STAMP(9);
#pragma unroll 1
    for (int yl = warp; yl < nrow; yl += CL_NW) {                        // row DFTs of u and v / Px -> column owners
      Line2<P> L;
      const float sP = 1.f / (float)P;                                   // exact: P is a power of two
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int x = lane + 32 * m;
        L.v[0][m] = x < nx ? rowT[x * RS + yl] : make_float2(0.f, 0.f);
        L.v[1][m] = x < nx ? sP * vs[yl * nx + x] : make_float2(0.f, 0.f);
      }
      L = line_fwd2<P>(L, tw, lane);
#pragma unroll
      for (int kk = 0; kk < R; ++kk) {                                   // to the column owners
        const int c = kk * 32 + lane, o = (y0 + yl) * SC + c % CB;
        cl.map_shared_rank(colT, c / CB)[o] = L.v[0][kk];
        cl.map_shared_rank(colV, c / CB)[o] = L.v[1][kk];
      }
    }
    cl.sync();
    CL_STAMP(10);
    // ===== 5. column convolution with the conjugated spectrum, kept at the column owner =====
#pragma unroll 1
    for (int lc = warp; lc < ncol; lc += 2 * CL_NW) {                  // columns lc and lc + NW together
      const int lc2 = lc + CL_NW;
      if (lc2 < ncol) {
        Line2<P> G, L;
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          const int c = l ? lc2 : lc;
#pragma unroll
          for (int kk = 0; kk < R; ++kk) G.v[l][kk] = cconj(ghs[c * P + kk * 32 + lane]);
#pragma unroll
          for (int m = 0; m < R; ++m) {
            const int y = lane + 32 * m;
            L.v[l][m] = y < ny ? colT[y * SC + c] : make_float2(0.f, 0.f);
          }
        }
        L = line_conv2<P>(L, G, tw, lane);
#pragma unroll
        for (int m = 0; m < R; ++m) {
          const int y = lane + 32 * m;
          if (y < ny) {                                                   // row-spectral v + G_D^H u, own columns
            colT[y * SC + lc] = L.v[0][m] + colV[y * SC + lc];
            colT[y * SC + lc2] = L.v[1][m] + colV[y * SC + lc2];
          }
        }
      } else {
        const float2* g = ghs + lc * P;
        Line<P> G, L;
#pragma unroll
        for (int kk = 0; kk < R; ++kk) G.v[kk] = cconj(g[kk * 32 + lane]);
#pragma unroll
        for (int m = 0; m < R; ++m) {
          const int y = lane + 32 * m;
          L.v[m] = y < ny ? colT[y * SC + lc] : make_float2(0.f, 0.f);
        }
        L = line_conv<P>(L, G, tw, lane);
#pragma unroll
        for (int m = 0; m < R; ++m) {
          const int y = lane + 32 * m;
          if (y < ny) colT[y * SC + lc] = L.v[m] + colV[y * SC + lc];
        }
      }
    }
    __syncthreads();
    CL_STAMP(11);
    // ===== 6. analysis (Phi^H) of dL/dJ = v + G_D^H u, partial over this CTA's columns =====
    // dL/dJ = inverse row DFT of B (B = the row-spectral v + G_D^H u at the column owners), so its
    // x-analysis is B conj(what) summed over the columns (each CTA: all rows, its columns).
    cl_cgemm<2, 2, 1, false, true>(ny, kx, ncol, colT, SC, 1, whs, kx, 1,
                                [&](int y, int jx, float2 v) { Tall[y * kx + jx] = v; });
    __syncthreads();
    CL_STAMP(12);
    // analysis along y, plus the data term (Eq. 16) at own receivers (formed during the grid
    // barrier); to every CTA
    cl_cgemm<1, 2, 1, true, false>(ky, kx, ny, wyf, ny, 1, Tall, kx, 1, [&](int jy, int jx, float2 v) {
      const int i = jy * kx + jx;
      const float2 acc = v + ks * gdv[i];
#pragma unroll 1
      for (int q = 0; q < C; ++q) {
        float2* dst = cl.map_shared_rank(gpart, q);
        dst[k * NA + i] = acc;
      }
    });
    cl.sync();
    CL_STAMP(13);
    // ===== 7. gradient and Adam step on this CTA's copy of alpha_p (network form: dL/dy_p) =====
#pragma unroll 1
    for (int i = threadIdx.x; i < NA; i += CL_NT) {
      float2 g = make_float2(0.f, 0.f);
#pragma unroll 1
      for (int q = 0; q < C; ++q) g = g + gpart[q * NA + i];
      if (H > 0) {
        dys[i] = g.x / net_s;
        dys[NA + i] = g.y / net_s;
        continue;
      }
      float2 ap = al[i];
      ph_adam(0, &ap.x, &g.x, &am[2 * i], &av[2 * i], 1, it + 1, a.tab, a.cap, a.b1, a.b2, a.eps);
      ph_adam(0, &ap.y, &g.y, &am[2 * i + 1], &av[2 * i + 1], 1, it + 1, a.tab, a.cap, a.b1, a.b2, a.eps);
      al[i] = ap;
    }
    __syncthreads();
    CL_STAMP(14);
    if (H > 0) {
      // ===== 8. chain rule to theta, per incidence =====
      const float* th = a.theta;
      // dz2 = (W3^T dL/dy) 1[h2 > 0]: this CTA's output rows, partials to every CTA, summed in rank order
      auto put_part = [&](int h, float v) {
#pragma unroll 1
        for (int q = 0; q < C; ++q) cl.map_shared_rank(npart, q)[k * H + h] = v;
      };
      if (a.wc) cl_net_cols<false>(cW3, H, dys + n0, nrw, nred, put_part);
      else cl_net_cols<true>(th + oW3 + (size_t)n0 * H, H, dys + n0, nrw, nred, put_part);
      cl.sync();
      if ((int)threadIdx.x < H) {
        const int h = threadIdx.x;
        float v = npart[h];
#pragma unroll 1
        for (int q = 1; q < C; ++q) v += npart[q * H + h];
        dz2s[h] = h2s[h] > 0.f ? v : 0.f;
      }
      __syncthreads();
      // dz1 = (W2^T dz2) 1[h1 > 0]; without the copy from partials over this CTA's rows of W2 (the
      // slice of h1 and h2), exchanged and summed in rank order
      if (a.wc) {
        cl_net_cols<false>(cW2, H, dz2s, H, nred, [&](int h, float v) { dz1s[h] = h1s[h] > 0.f ? v : 0.f; });
      } else {
        const int hs = (H + C - 1) / C, h0 = min(H, k * hs), nh = min(H, h0 + hs) - h0;
        cl_net_cols<true>(th + oW2 + (size_t)h0 * H, H, dz2s + h0, nh, nred, [&](int h, float v) {
#pragma unroll 1
          for (int q = 0; q < C; ++q) cl.map_shared_rank(npart2, q)[k * H + h] = v;
        });
        cl.sync();
        if ((int)threadIdx.x < H) {
          const int h = threadIdx.x;
          float v = npart2[h];
#pragma unroll 1
          for (int q = 1; q < C; ++q) v += npart2[q * H + h];
          dz1s[h] = h1s[h] > 0.f ? v : 0.f;
        }
        __syncthreads();
      }
      const int NV = D + 4 * H;
      if (k == 0) {
        float* nv = a.nvec + (size_t)p * NV;
#pragma unroll 1
        for (int i = threadIdx.x; i < NV; i += CL_NT) {
          const float v = i < D ? dys[i] : i < D + H ? h2s[i - D] : i < D + 2 * H ? dz2s[i - D - H]
                          : i < D + 3 * H ? h1s[i - D - 2 * H] : dz1s[i - D - 3 * H];
          __stcg(nv + i, v);
        }
      }
      cl_grid_barrier(a.bar, ++nbar * nblocks, a.err, a.wait_cap, [] {});
      CL_STAMP(15);
      // ===== 9. dL/d theta on this CTA's slice of theta (sums over incidences, increasing p) and Adam =====
      const size_t ps = (npar + nblocks - 1) / nblocks, i0 = (size_t)blockIdx.x * ps, i1 = min(npar, i0 + ps);
      const float2 asc = ph_adam_sc(a.tab, a.cap, it + 1);
#pragma unroll 1
      for (size_t i = i0 + threadIdx.x; i < i1; i += CL_NT) {
        // dW = dZ^T U over the incidences (U = X, h1 or h2), the bias gradients the sums of dZ
        int zo, uo = -1, zi, ui = 0;
        bool ux = false;
        if (i < ob1) {
          zo = D + 3 * H; zi = (int)((i - oW1) / D); ui = (int)((i - oW1) % D); ux = true;
        } else if (i < oW2) {
          zo = D + 3 * H; zi = (int)(i - ob1);
        } else if (i < ob2) {
          zo = D + H; zi = (int)((i - oW2) / H); uo = D + 2 * H; ui = (int)((i - oW2) % H);
        } else if (i < oW3) {
          zo = D + H; zi = (int)(i - ob2);
        } else if (i < ob3) {
          zo = 0; zi = (int)((i - oW3) / H); uo = D; ui = (int)((i - oW3) % H);
        } else {
          zo = 0; zi = (int)(i - ob3);
        }
        float tp = __ldcg(a.theta + i), mi = a.tm[i], vi = a.tv[i];
        // (a bias term is z times 1: fmaf(z, 1, g) rounds z + g once, as the plain sum does)
        float g = 0.f;
#pragma unroll 1
        for (int q0 = 0; q0 < ni; q0 += 16) {
          float z[16], u[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int q = q0 + j;
            const float* nv = a.nvec + (size_t)q * NV;
            z[j] = q < ni ? __ldcg(nv + zo + zi) : 0.f;
            u[j] = q >= ni ? 0.f : ux ? __ldg(a.X + (size_t)q * D + ui) : uo >= 0 ? __ldcg(nv + uo + ui) : 1.f;
          }
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (q0 + j < ni) g = fmaf(z[j], u[j], g);
        }
        ph_adam_at(tp, g, mi, vi, asc, a.b1, a.b2, a.eps);
        __stcg(a.theta + i, tp);
        a.tm[i] = mi;
        a.tv[i] = vi;
      }
      __syncthreads();
      CL_STAMP(17);
      if (it + 1 < a.iters) cl_grid_barrier(a.bar, ++nbar * nblocks, a.err, a.wait_cap, [] {});
    }
  }
  if (k == 0 && H == 0)
#pragma unroll 1
    for (int i = threadIdx.x; i < NA; i += CL_NT) a.alpha[(size_t)p * NA + i] = al[i];
  cl.sync();
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
static size_t cluster_smem(const Dev& d, int C, int RB, int CB, int P, int H) {
  const size_t NA = (size_t)d.ky * d.kx, GP = (size_t)RB * d.nx, HP = (size_t)(RB + 2) * d.nx,
               TP = (size_t)(RB + 1) * d.nx;
  const size_t nscr = 2 * GP + HP + 2 * TP;
  const size_t NU = std::max((size_t)C * NA, (nscr + 1) / 2);
  const size_t RS = (size_t)((RB + 1) | 1), SC = (size_t)(CB | 1);
  const size_t f2 = P + (size_t)P * RS + (size_t)CB * (d.ny + 1) + 2 * (size_t)d.ny * SC + 4 * GP + 2 * HP +
                    NA + NU + 2 * (size_t)d.nr +
                    (size_t)d.ny * d.kx + (size_t)d.ky * d.ny + (size_t)d.kx * CB +
                    (size_t)CB * P + (size_t)d.kx * d.nx + NA + (size_t)((d.nr + C - 1) / C) * NA;
  return f2 * sizeof(float2) + 4 * NA * sizeof(float) + cl_net_floats(H, 2 * (int)NA, C) * sizeof(float);
}

// dynamic shared memory limit of the cluster kernel (227 KB per block; no static use)
static const size_t CL_SMEM_MAX = 226 * 1024;

// Rows and padded columns per CTA for cluster size c (the last CTA may own fewer).
static int cl_rb(const Dev& d, int c) { return (d.ny + c - 1) / c; }
static int cl_cb(const Dev& d, int c) { return (d.Px + c - 1) / c; }

// Whether cluster size c gives every CTA at least one row and one padded column, with ni * c CTAs
// resident.
static bool cluster_ok(const Dev& d, int sms, int c) {
  const int rb = cl_rb(d, c), cb = cl_cb(d, c);
  return d.ni * c <= sms && (c - 1) * rb < d.ny && (c - 1) * cb < d.Px && rb <= 64 && d.nr <= 1024;
}

template <int P>
static cudaLaunchConfig_t cluster_config(int ni, int C, size_t smem, cudaStream_t st, cudaLaunchAttribute* at) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_cluster_solve<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CL_SMEM_MAX);
    cudaFuncSetAttribute(k_cluster_solve<P>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaGetLastError();
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ni * C);
  cfg.blockDim = dim3(CL_NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeCooperative;
  at[1].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  return cfg;
}

// clusters of size C that can be co-resident on this device (-1: the query failed)
template <int P>
static int max_active_clusters(int ni, int C, size_t smem) {
  cudaLaunchAttribute at[2];
  cudaLaunchConfig_t cfg = cluster_config<P>(ni, C, smem, 0, at);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (void*)k_cluster_solve<P>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return n;
}

struct ClPlanRow {
  int C, smem, clusters, usable;
};

// The cluster sizes cl_run considers, in order, with their shared-memory plan and the number of
// such clusters the device can hold at once; a row is usable when all ni clusters fit.
static int cl_plan(const pdf_problem* h, ClPlanRow* rows, int nmax) {
  const Dev& d = h->d;
  if (!d.fast || h->tc || !d.fold || !d.what || d.cco_loss || d.Px != d.Py || d.Px > 128 || d.kx > 64) return 0;
  const int H = h->fc_active ? h->fc.H : 0;
  if (H > CL_NT) return 0;
  int dev = 0, sms = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) {
    cudaGetLastError();
    return 0;
  }
  static const int sizes[] = {16, 8, 6, 4, 2};
  int n = 0;
  for (int c : sizes) {
    if (n >= nmax) break;
    if (!cluster_ok(d, sms, c)) continue;
    const size_t smem = cluster_smem(d, c, cl_rb(d, c), cl_cb(d, c), d.Px, H);
    ClPlanRow r = {c, (int)smem, -1, 0};
    if (smem <= CL_SMEM_MAX) {
      r.clusters = d.Px == 64 ? max_active_clusters<64>(d.ni, c, smem) : max_active_clusters<128>(d.ni, c, smem);
      r.usable = r.clusters >= d.ni;
    }
    rows[n++] = r;
  }
  return n;
}

extern "C" int32_t pdf_cluster_plan(pdf_problem* h, int32_t* out, int32_t nmax) {
  if (!h || !out || nmax < 1) {
    set_err(PDF_EINVAL, "pdf_cluster_plan: bad arguments");
    return PDF_EINVAL;
  }
  ClPlanRow rows[5];
  const int n = cl_plan(h, rows, std::min(5, (int)nmax));
  for (int i = 0; i < n; ++i) {
    out[4 * i + 0] = rows[i].C;
    out[4 * i + 1] = rows[i].smem;
    out[4 * i + 2] = rows[i].clusters;
    out[4 * i + 3] = rows[i].usable;
  }
  return n;
}

extern "C" pdf_status pdf_phase_stamps(uint64_t* out) {
#ifdef PDF_PHASE_STAMPS
  cudaError_t e = cudaMemcpyFromSymbol(out, g_cl_stamps, sizeof(g_cl_stamps));
  if (e != cudaSuccess) return cuda_err(e, "cudaMemcpyFromSymbol(phase stamps)");
  return PDF_OK;
#else
  (void)out;
  return set_err(PDF_EUNSUPPORTED, "phase stamps need a library built with PDF_PHASE_STAMPS");
#endif
}

// Runs `iters` Adam iterations of h->alpha with the cluster kernel.  *done = false (nothing
// launched) when not eligible.
pdf_status cl_run(pdf_problem* h, const pdf_solve_opts* o, int iters, cudaStream_t st, bool* done) {
  *done = false;
  const Dev& d = h->d;
  if (iters < 1) return PDF_OK;
  ClPlanRow rows[5];
  const int n = cl_plan(h, rows, 5);
  int pick = -1;
  for (int i = 0; i < n && pick < 0; ++i)
    if (rows[i].usable) pick = i;
  if (pick < 0) return PDF_OK;
  ClusterArgs a;
  a.iters = iters;
  a.C = rows[pick].C;
  a.RB = cl_rb(d, a.C);
  a.CB = cl_cb(d, a.C);
  // Sums over incidences: each CTA reads ni x (RB + 2) x nx float4 when it forms R-hat on its own
  // rows, all CTAs at once, and the phase is bound by L2 bandwidth; the split form costs a second
  // grid barrier and two more L2 round trips instead.  Measured on GB300 (per iteration): 32x32,
  // Ni = 8, 8-CTA clusters (24 KB per CTA) 10.5 us per CTA vs 12.3 us split; 64x64, Ni = 16, 4-CTA
  // clusters (295 KB) 31.6 vs 29.6 us; 64x64, Ni = 36 (663 KB) 35.6 vs 30.7 us.  With 6-CTA
  // clusters at 64x64, Ni = 16 (213 KB per CTA) a 256 KB threshold, i.e. the unsplit form, timed
  // the same as the split one, so 128 KB stays.
  const int nb = d.ni * a.C;
  const size_t rep_bytes = (size_t)d.ni * (a.RB + 2) * d.nx * sizeof(float4);
  a.sl = rep_bytes > 128 * 1024 ? (d.M + nb - 1) / nb : 0;
  for (a.sg = 1; 8 * a.sg < d.ni; a.sg *= 2) {
  }
  a.H = h->fc_active ? h->fc.H : 0;
  if ((uint64_t)iters * (a.H > 0 ? 4 : 2) * nb >= 0xffffffffull) return PDF_OK;  // barrier counter range
  if (!h->cl_nd) {
    pdf_status s;
    const size_t bytes = sizeof(float4) * (2 * (size_t)d.ni + 1) * d.M + sizeof(float) * (size_t)d.M;
    if ((s = ws_alloc(h, (void**)&h->cl_nd, bytes)) != PDF_OK) return s;
  }
  a.alpha = h->alpha;
  a.tab = h->adam_tab;
  a.cap = h->adam_cap;
  a.b1 = (float)o->adam_b1;
  a.b2 = (float)o->adam_b2;
  a.eps = (float)o->adam_eps;
  a.nd = h->cl_nd;
  a.rc = h->cl_nd + 2 * (size_t)d.ni * d.M;
  a.dsg = (float*)(a.rc + d.M);
  a.bar = h->bar;
  a.err = h->perr;
  a.wait_cap = o->barrier_wait_cycles > 0 ? (long long)o->barrier_wait_cycles : (1ll << 31);
  a.theta = a.tm = a.tv = a.nvec = nullptr;
  a.X = a.xs = nullptr;
  a.alpha0 = nullptr;
  if (a.H > 0) {
    FcState& f = h->fc;
    if (!f.nvec) {
      pdf_status s;
      if ((s = ws_alloc(h, (void**)&f.nvec, sizeof(float) * (size_t)d.ni * (f.D + 4 * f.H))) != PDF_OK) return s;
    }
    a.theta = f.theta;
    a.tm = f.m;
    a.tv = f.v;
    a.X = f.X;
    a.xs = f.s;
    a.alpha0 = f.alpha0;
    a.nvec = f.nvec;
  }
  // Test hook for the solve's recovery path: with PDF_TEST_CLUSTER_SHAPE=mismatch in the environment
  // the kernel is told to expect a cluster size no launch has, so every CTA takes the entry check's
  // early return (error flag 2) exactly as when a tool launches it without its cluster shape.
  if (const char* t = getenv("PDF_TEST_CLUSTER_SHAPE"))
    if (strcmp(t, "mismatch") == 0) a.C = 0;
  PDF_CUDA(cudaMemsetAsync(h->bar, 0, sizeof(unsigned), st));
  cudaLaunchAttribute at[2];
  size_t smem = (size_t)rows[pick].smem;
  // the network weights' shared copy, where it fits beside the plan with all clusters still resident
  a.wc = 0;
  if (a.H > 0) {
    const size_t wc = smem + cl_net_cache_floats(a.H, 2 * d.ky * d.kx, rows[pick].C) * sizeof(float);
    const int fit = wc > CL_SMEM_MAX ? -1
                    : d.Px == 64 ? max_active_clusters<64>(d.ni, rows[pick].C, wc)
                                 : max_active_clusters<128>(d.ni, rows[pick].C, wc);
    if (fit >= d.ni) {
      a.wc = 1;
      smem = wc;
    }
  }
  cudaError_t e;
  if (d.Px == 64) {
    cudaLaunchConfig_t cfg = cluster_config<64>(d.ni, rows[pick].C, smem, st, at);
    e = cudaLaunchKernelEx(&cfg, k_cluster_solve<64>, h->d, a);
  } else {
    cudaLaunchConfig_t cfg = cluster_config<128>(d.ni, rows[pick].C, smem, st, at);
    e = cudaLaunchKernelEx(&cfg, k_cluster_solve<128>, h->d, a);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return PDF_OK;                                   // launch form unsupported: the caller falls back
  }
  pdf_count_launch(1);
  *done = true;
  return PDF_OK;
}
