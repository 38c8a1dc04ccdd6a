// Cluster form of the whole Adam loop for small grids (padded length P = Px = Py <= 128).
//
// One thread-block cluster per incidence p; CTA k of the cluster owns grid rows
// [k RB, (k+1) RB) and padded columns [k CB, (k+1) CB).  Per iteration:
//   1. synthesis of its rows (Eq. 9) and their padded row DFT (register warp FFT); each row's
//      spectrum is stored straight into the column owners' shared memory (DSMEM)      | cluster barrier
//   2. column DFT, x G_D spectrum, inverse column DFT on its columns; rows < ny go back
//      to their row owners over DSMEM                                                  | cluster barrier
//   3. inverse row DFT -> G_D J, s = beta J + E_inc + G_D J; this incidence's per-pixel
//      contributions beta J conj(s), |s|^2 to a global array (double-buffered by iteration);
//      partial G_S J_p over its pixels sent to every CTA of the cluster                  | GRID barrier
//   4. R-hat, chi-hat (Eq. 6, 7) for its rows and one halo row each side from the sums over all
//      incidences; state residual (Eq. 15); data residual r_d,p (Eq. 16); regulariser cotangent
//      (Eq. 17-19) -> w; adjoint inputs u, v; G_S^H r_d,p; row DFT of u -> column owners  | cluster barrier
//   5. column convolution with the conjugated spectrum (G_D^H) -> row owners             | cluster barrier
//   6. inverse row DFT, dL/dJ = v + G_D^H u + G_S^H term, analysis along x and the partial
//      analysis along y over its rows -> every CTA of the cluster                         | cluster barrier
//   7. dL/d alpha_p = sum of the partials (same order in every CTA), Adam step on each CTA's copy
//      of alpha_p (identical in all CTAs of the cluster)
// The arithmetic is that of the stand-alone kernels (same formulas, FP32 with compensated sums);
// only the data movement differs.  The grid barrier is the bounded one of persist.cu (timeout ->
// error flag, every CTA returns); co-residency comes from the cooperative launch.
#include <cooperative_groups.h>

#include "phases.cuh"

namespace cg = cooperative_groups;

struct ClusterArgs {
  int iters, C, RB, CB;
  int gs_smem;            // 1: this CTA's G_S columns [nr][RB nx] are staged in shared memory
  float2* alpha;          // [ni][ky][kx] in / out
  const float2* tab;
  int cap;
  float b1, b2, eps;
  float* nd;              // [2][ni][M][3] per-incidence (Re N, Im N, D)
  FF* lpart;              // [ni * C][5] loss partials of the last iteration
  unsigned* bar;
  int* err;
};

__device__ __forceinline__ unsigned cl_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool cl_grid_barrier(unsigned* bar, unsigned target, int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    atomicAdd(bar, 1u);
    if (cl_ld_acquire(bar) < target) {
      const long long t0 = clock64();
      while (cl_ld_acquire(bar) < target) {
        if (clock64() - t0 > (1ll << 31)) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

struct TVBs {
  float2 dx, dy;
  float t, gx, gy, sg, e;
};

// TV / bridge pieces at grid pixel (y, x) from chi rows held in `ch` (row y at index y - y0 + 1)
__device__ __forceinline__ TVBs tvb_local(const Dev& d, const float2* ch, int y0, int y, int x) {
  TVBs o;
  const int ly = y - y0 + 1;
  const float2 c = ch[ly * d.nx + x];
  const bool hx = x + 1 < d.nx, hy = y + 1 < d.ny;
  o.dx = hx ? ch[ly * d.nx + x + 1] - c : make_float2(0.f, 0.f);
  o.dy = hy ? ch[(ly + 1) * d.nx + x] - c : make_float2(0.f, 0.f);
  o.t = sqrtf(cabs2(o.dx) + cabs2(o.dy) + d.eps_tv);
  const float m = sqrtf(cabs2(c) + d.eps_abs);
  o.gx = hx ? sqrtf(cabs2(ch[ly * d.nx + x + 1]) + d.eps_abs) - m : 0.f;
  o.gy = hy ? sqrtf(cabs2(ch[(ly + 1) * d.nx + x]) + d.eps_abs) - m : 0.f;
  o.sg = 1.f / (1.f + expf(-(m - d.tau_b) / d.tau_b));
  o.e = expf(-(o.gx * o.gx + o.gy * o.gy));
  return o;
}

template <int P>
__global__ void __launch_bounds__(256, 1) k_cluster_solve(Dev d, ClusterArgs a) {
  constexpr int R = P / 32;
  cg::cluster_group cl = cg::this_cluster();
  const int C = a.C, RB = a.RB, CB = a.CB;
  const int k = (int)cl.block_rank();
  const int p = blockIdx.x / C;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  const int nx = d.nx, ny = d.ny, kx = d.kx, ky = d.ky, nr = d.nr, M = d.M;
  const int y0 = k * RB, c0 = k * CB;
  const int LS = ny + 1;
  const int NA = ky * kx;
  // ---- shared memory carve-up ----
  extern __shared__ float2 sm[];
  float2* tw = sm;                           // [P]
  float2* rowb = tw + P;                     // [RB][P]
  float2* colb = rowb + RB * P;              // [CB][LS]
  float2* Js = colb + CB * LS;               // [RB][nx]
  float2* ss = Js + RB * nx;                 // [RB][nx]
  float2* rs = ss + RB * nx;                 // [RB][nx]
  float2* Es = rs + RB * nx;                 // [RB][nx]
  float2* vs = Es + RB * nx;                 // [RB][nx]
  float2* ws = vs + RB * nx;                 // [RB][nx] w
  float2* Rh = ws + RB * nx;                 // [RB + 2][nx] R-hat with halo rows
  float2* Ch = Rh + (RB + 2) * nx;           // [RB + 2][nx] chi-hat with halo rows
  float2* al = Ch + (RB + 2) * nx;           // [NA] alpha_p
  float2* gr = al + NA;                      // [NA] gradient
  float2* gpart = gr + NA;                   // [C][NA] partial y-analyses of all ranks
  float2* dpart = gpart + C * NA;            // [C][nr] partial G_S J_p of all ranks
  float2* rd = dpart + C * nr;               // [nr]
  float2* es = rd + nr;                      // [nr]
  float2* T2 = es + nr;                      // [RB][kx] (also the synthesis temporary)
  float* am = (float*)(T2 + RB * kx);        // [2 NA]
  float* av = am + 2 * NA;                   // [2 NA]
  float* Dl = av + 2 * NA;                   // [RB][nx]
  float2* Gs = (float2*)(Dl + RB * nx + (RB * nx & 1));  // [nr][RB nx] when a.gs_smem
  const int GP = RB * nx;                    // pixels owned by this CTA
  __shared__ FF red[32];
  __shared__ int okflags[16];

  // ---- one-time loads ----
  for (int i = threadIdx.x; i < P; i += blockDim.x) tw[i] = d.twx[i];
  for (int i = threadIdx.x; i < NA; i += blockDim.x) {
    al[i] = a.alpha[(size_t)p * NA + i];
    am[2 * i] = am[2 * i + 1] = 0.f;
    av[2 * i] = av[2 * i + 1] = 0.f;
  }
  for (int i = threadIdx.x; i < RB * nx; i += blockDim.x) Es[i] = d.einc[(size_t)p * M + y0 * nx + i];
  for (int i = threadIdx.x; i < nr; i += blockDim.x) es[i] = d.esca[(size_t)p * nr + i];
  if (a.gs_smem)
    for (int i = threadIdx.x; i < nr * GP; i += blockDim.x) {
      const int r = i / GP, j = i - r * GP;
      Gs[i] = d.gs[(size_t)r * M + y0 * nx + j];
    }
  // G_S entry of receiver r at own pixel j (j = local row * nx + x)
  auto gsv = [&](int r, int j) -> float2 { return a.gs_smem ? Gs[r * GP + j] : d.gs[(size_t)r * M + y0 * nx + j]; };
  const float ke = d.invn[0], ks = d.invn[1];
  const float2 beta = d.beta, bc = cconj(d.beta);
  unsigned gen = 0;
  const unsigned nblocks = gridDim.x;
  cl.sync();

  for (int it = 0; it < a.iters; ++it) {
    float* nd = a.nd + (size_t)(it & 1) * d.ni * M * 3;
    // ===== 1. synthesis of own rows, row DFT, scatter to column owners =====
    for (int i = threadIdx.x; i < RB * kx; i += blockDim.x) {           // T'[yl][jx] = sum_jy Wy[jy][y] al[jy][jx]
      const int yl = i / kx, jx = i - yl * kx;
      float2 acc = make_float2(0.f, 0.f);
      for (int jy = 0; jy < ky; ++jy) acc = acc + cmul(__ldg(&d.wy[jy * ny + y0 + yl]), al[jy * kx + jx]);
      T2[i] = acc;
    }
    __syncthreads();
    for (int yl = warp; yl < RB; yl += nwarp) {
      float2 v[R];
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int x = lane + 32 * m;
        float2 s = make_float2(0.f, 0.f);
        if (x < nx) {
          for (int jx = 0; jx < kx; ++jx) s = s + cmul(T2[yl * kx + jx], __ldg(&d.wx[jx * nx + x]));
          Js[yl * nx + x] = s;
        }
        v[m] = s;
      }
      WarpFFT<P>::forward(v, tw, lane);
#pragma unroll
      for (int kk = 0; kk < R; ++kk) {
        const int c = kk * 32 + lane;
        float2* dst = cl.map_shared_rank(colb, c / CB);
        dst[(c % CB) * LS + y0 + yl] = v[kk];
      }
    }
    cl.sync();
    // ===== 2. column convolution, results back to row owners =====
    for (int lc = warp; lc < CB; lc += nwarp) {
      float2 v[R];
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int y = lane + 32 * m;
        v[m] = y < ny ? colb[lc * LS + y] : make_float2(0.f, 0.f);
      }
      WarpFFT<P>::forward(v, tw, lane);
      const float2* g = d.ghat_perm + (size_t)(c0 + lc) * P;
#pragma unroll
      for (int kk = 0; kk < R; ++kk) v[kk] = cmul(v[kk], __ldg(&g[kk * 32 + lane]));
      WarpFFT<P>::inverse(v, tw, lane);
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int y = lane + 32 * m;
        if (y < ny) {
          float2* dst = cl.map_shared_rank(rowb, y / RB);
          dst[(y % RB) * P + c0 + lc] = v[m];
        }
      }
    }
    cl.sync();
    // ===== 3. inverse row DFT, s, per-incidence contributions, partial G_S J_p =====
    for (int yl = warp; yl < RB; yl += nwarp) {
      float2 v[R];
#pragma unroll
      for (int kk = 0; kk < R; ++kk) v[kk] = rowb[yl * P + kk * 32 + lane];
      WarpFFT<P>::inverse(v, tw, lane);
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int x = lane + 32 * m;
        if (x < nx) {
          const int li = yl * nx + x;
          const float2 J = Js[li];
          const float2 s = cmul(beta, J) + Es[li] + v[m];
          ss[li] = s;
          const float2 n = cmul(beta, cmulc(J, s));
          float* o = nd + ((size_t)p * M + (y0 + yl) * nx + x) * 3;
          o[0] = n.x;
          o[1] = n.y;
          o[2] = cabs2(s);
        }
      }
    }
    for (int r = warp; r < nr; r += nwarp) {                             // partial (G_S J_p)[r] over own pixels
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
      for (int i = lane; i < GP; i += 32) acc = acc + cmul(gsv(r, i), Js[i]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (lane < C) {
        float2* dst = cl.map_shared_rank(dpart, lane);
        dst[k * nr + r] = acc;
      }
    }
    ++gen;
    {
      // the cluster decides together whether to stop (a CTA never leaves while peers may still
      // address its shared memory)
      const bool ok = cl_grid_barrier(a.bar, gen * nblocks, a.err);
      if (threadIdx.x == 0) *cl.map_shared_rank(&okflags[k], 0) = ok ? 1 : 0;
      cl.sync();
      int all = 1;
      if (threadIdx.x == 0)
        for (int q = 0; q < C; ++q) all &= *cl.map_shared_rank(&okflags[q], 0);
      all = __syncthreads_and(all);
      cl.sync();
      if (!all) return;
    }
    // ===== 4. R-hat, chi-hat (own rows + halo), residuals, regulariser cotangent, adjoint inputs =====
    for (int i = threadIdx.x; i < (RB + 2) * nx; i += blockDim.x) {
      const int hy = i / nx, x = i - hy * nx, y = y0 + hy - 1;
      if (y < 0 || y >= ny) continue;
      float nr_ = 0.f, ni_ = 0.f, dd = 0.f, cr = 0.f, ci = 0.f, cd = 0.f;
#pragma unroll 4
      for (int q = 0; q < d.ni; ++q) {
        const float* o = nd + ((size_t)q * M + y * nx + x) * 3;
        float t, yv;
        yv = o[0] - cr; t = nr_ + yv; cr = (t - nr_) - yv; nr_ = t;
        yv = o[1] - ci; t = ni_ + yv; ci = (t - ni_) - yv; ni_ = t;
        yv = o[2] - cd; t = dd + yv; cd = (t - dd) - yv; dd = t;
      }
      const float Df = dd - cd;
      const float2 Rv = make_float2((nr_ - cr) / Df, (ni_ - ci) / Df);
      bool clamped;
      const float2 chi = chi_of_R_f(Rv, beta, d.q_min, &clamped);
      Rh[i] = Rv;
      Ch[i] = chi;
      if (hy >= 1 && hy <= RB) {
        Dl[(hy - 1) * nx + x] = clamped ? -Df : Df;                      // sign carries the clamp flag
      }
    }
    __syncthreads();
    FF l_state = FF{0.f, 0.f}, l_bound = FF{0.f, 0.f}, l_tv = FF{0.f, 0.f}, l_br = FF{0.f, 0.f};
    for (int li = threadIdx.x; li < RB * nx; li += blockDim.x) {
      const int yl = li / nx, x = li - yl * nx, y = y0 + yl;
      const float2 Rv = Rh[(yl + 1) * nx + x];
      const float2 J = Js[li], s = ss[li];
      const float2 r = cmul(Rv, s) - cmul(beta, J);
      rs[li] = r;
      l_state = ff_add(l_state, cabs2(r));
      // regulariser terms at (y, x) and their cotangent on chi (same formulas as k_reg)
      const float2 c = Ch[(yl + 1) * nx + x];
      const float neg = fmaxf(-c.x, 0.f);
      const TVBs o = tvb_local(d, Ch, y0, y, x);
      l_bound = ff_add(l_bound, neg * neg);
      l_tv = ff_add(l_tv, o.t);
      l_br = ff_add(l_br, o.sg * o.e);
      float2 ctv = (-1.f / o.t) * (o.dx + o.dy);
      float dm = o.sg * (1.f - o.sg) / d.tau_b * o.e + 2.f * (o.gx + o.gy) * o.sg * o.e;
      if (x > 0) {
        const TVBs l = tvb_local(d, Ch, y0, y, x - 1);
        ctv = ctv + (1.f / l.t) * l.dx;
        dm += -2.f * l.gx * l.sg * l.e;
      }
      if (y > 0) {
        const TVBs u = tvb_local(d, Ch, y0, y - 1, x);
        ctv = ctv + (1.f / u.t) * u.dy;
        dm += -2.f * u.gy * u.sg * u.e;
      }
      const float mg = sqrtf(cabs2(c) + d.eps_abs);
      float2 cchi = d.lam_tv * ctv + (d.lam_bridge * dm / mg) * c;
      cchi.x += d.lam_bound * (-2.f * neg);
      const float Dv = Dl[li];
      float2 w = make_float2(0.f, 0.f);
      if (Dv > 0.f) {
        const float2 q = make_float2(1.f - Rv.x, -Rv.y);
        const float2 dchi = cdivf(make_float2(1.f, 0.f), cmul(beta, cmul(q, q)));
        w = (1.f / Dv) * cmul(cconj(dchi), cchi);
      }
      ws[li] = w;
    }
    // data residual of this incidence (every rank sums the partials in the same order)
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
      float2 acc = make_float2(0.f, 0.f);
      for (int q = 0; q < C; ++q) acc = acc + dpart[q * nr + r];
      rd[r] = acc - es[r];
    }
    {
      const FF t = ff_block_sum(l_state, red);
      if (threadIdx.x == 0) a.lpart[(size_t)blockIdx.x * 5 + 0] = t;
      const FF tb = ff_block_sum(l_bound, red);
      if (threadIdx.x == 0) a.lpart[(size_t)blockIdx.x * 5 + 2] = p == 0 ? tb : FF{0.f, 0.f};
      const FF tt = ff_block_sum(l_tv, red);
      if (threadIdx.x == 0) a.lpart[(size_t)blockIdx.x * 5 + 3] = p == 0 ? tt : FF{0.f, 0.f};
      const FF tr = ff_block_sum(l_br, red);
      if (threadIdx.x == 0) a.lpart[(size_t)blockIdx.x * 5 + 4] = p == 0 ? tr : FF{0.f, 0.f};
    }
    __syncthreads();
    {
      FF ld = FF{0.f, 0.f};
      if (k == 0)
        for (int r = threadIdx.x; r < nr; r += blockDim.x) ld = ff_add(ld, cabs2(rd[r]));
      const FF t = ff_block_sum(ld, red);
      if (threadIdx.x == 0) a.lpart[(size_t)blockIdx.x * 5 + 1] = t;
    }
    // u (row DFT -> column owners) and v, G_S^H r_d folded into v
    for (int yl = warp; yl < RB; yl += nwarp) {
      float2 v[R];
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int x = lane + 32 * m;
        v[m] = make_float2(0.f, 0.f);
        if (x < nx) {
          const int li = yl * nx + x;
          const float2 Rv = Rh[(yl + 1) * nx + x];
          const float2 w = ws[li], J = Js[li], s = ss[li], r = rs[li];
          const float2 wc = cconj(w);
          const float2 cs = cmul(cmul(wc, beta), J) - (2.f * cmul(wc, Rv).x) * s;
          v[m] = ke * cmulc(r, Rv) + cs;
          const float2 omr = make_float2(1.f - Rv.x, Rv.y);
          float2 vv = ke * cmul(cmul(make_float2(-bc.x, -bc.y), omr), r) + cmul(bc, cmul(w, s) + cs);
          float2 gh = make_float2(0.f, 0.f);
#pragma unroll 8
          for (int q = 0; q < nr; ++q) gh = gh + cmulc(rd[q], gsv(q, li));
          vs[li] = vv + ks * gh;
        }
      }
      WarpFFT<P>::forward(v, tw, lane);
#pragma unroll
      for (int kk = 0; kk < R; ++kk) {
        const int c = kk * 32 + lane;
        float2* dst = cl.map_shared_rank(colb, c / CB);
        dst[(c % CB) * LS + y0 + yl] = v[kk];
      }
    }
    cl.sync();
    // ===== 5. column convolution with the conjugated spectrum =====
    for (int lc = warp; lc < CB; lc += nwarp) {
      float2 v[R];
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int y = lane + 32 * m;
        v[m] = y < ny ? colb[lc * LS + y] : make_float2(0.f, 0.f);
      }
      WarpFFT<P>::forward(v, tw, lane);
      const float2* g = d.ghat_perm + (size_t)(c0 + lc) * P;
#pragma unroll
      for (int kk = 0; kk < R; ++kk) v[kk] = cmul(v[kk], cconj(__ldg(&g[kk * 32 + lane])));
      WarpFFT<P>::inverse(v, tw, lane);
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int y = lane + 32 * m;
        if (y < ny) {
          float2* dst = cl.map_shared_rank(rowb, y / RB);
          dst[(y % RB) * P + c0 + lc] = v[m];
        }
      }
    }
    cl.sync();
    // ===== 6. inverse row DFT, dL/dJ, analysis along x and partial analysis along y =====
    for (int yl = warp; yl < RB; yl += nwarp) {
      float2 v[R];
#pragma unroll
      for (int kk = 0; kk < R; ++kk) v[kk] = rowb[yl * P + kk * 32 + lane];
      WarpFFT<P>::inverse(v, tw, lane);
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int x = lane + 32 * m;
        if (x < nx) rs[yl * nx + x] = v[m] + vs[yl * nx + x];          // g_J (reuses rs)
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < RB * kx; i += blockDim.x) {
      const int yl = i / kx, jx = i - yl * kx;
      float2 acc = make_float2(0.f, 0.f);
      for (int x = 0; x < nx; ++x) acc = acc + cmulc(rs[yl * nx + x], __ldg(&d.wx[jx * nx + x]));
      T2[i] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NA; i += blockDim.x) {
      const int jy = i / kx, jx = i - jy * kx;
      float2 acc = make_float2(0.f, 0.f);
      for (int yl = 0; yl < RB; ++yl) acc = acc + cmulc(T2[yl * kx + jx], __ldg(&d.wy[jy * ny + y0 + yl]));
      for (int q = 0; q < C; ++q) {
        float2* dst = cl.map_shared_rank(gpart, q);
        dst[k * NA + i] = acc;
      }
    }
    cl.sync();
    // ===== 7. gradient and Adam step on this CTA's copy of alpha_p =====
    for (int i = threadIdx.x; i < NA; i += blockDim.x) {
      float2 g = make_float2(0.f, 0.f);
      for (int q = 0; q < C; ++q) g = g + gpart[q * NA + i];
      gr[i] = g;
      float2 ap = al[i];
      ph_adam(0, &ap.x, &g.x, &am[2 * i], &av[2 * i], 1, it + 1, a.tab, a.cap, a.b1, a.b2, a.eps);
      ph_adam(0, &ap.y, &g.y, &am[2 * i + 1], &av[2 * i + 1], 1, it + 1, a.tab, a.cap, a.b1, a.b2, a.eps);
      al[i] = ap;
    }
    __syncthreads();
  }
  if (k == 0)
    for (int i = threadIdx.x; i < NA; i += blockDim.x) a.alpha[(size_t)p * NA + i] = al[i];
  cl.sync();
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
static size_t cluster_smem(const Dev& d, int C, int RB, int CB, int P, bool gs) {
  const size_t NA = (size_t)d.ky * d.kx;
  size_t f2 = P + (size_t)RB * P + (size_t)CB * (d.ny + 1) + 6 * (size_t)RB * d.nx + 2 * (size_t)(RB + 2) * d.nx + 2 * NA +
              (size_t)C * NA + (size_t)C * d.nr + 2 * (size_t)d.nr + (size_t)RB * d.kx;
  size_t fl = 4 * NA + (size_t)RB * d.nx + 1;
  size_t b = f2 * sizeof(float2) + fl * sizeof(float);
  if (gs) b += (size_t)d.nr * RB * d.nx * sizeof(float2);
  return b;
}

// Whether cluster size c splits rows and padded columns evenly with ni * c CTAs resident.
static bool cluster_ok(const Dev& d, int sms, int c) {
  return d.ni * c <= sms && d.ny % c == 0 && d.Px % c == 0 && d.ny / c <= 64 && d.nr <= 1024;
}

__global__ void k_cluster_finalize(Dev d, const FF* lp, int nblocks, double* terms) {
  __shared__ FF red[32];
  double tot[5];
  for (int s = 0; s < 5; ++s) {
    FF acc = FF{0.f, 0.f};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) acc = ff_add(acc, lp[(size_t)b * 5 + s]);
    tot[s] = ff_to_d(ff_block_sum(acc, red));
  }
  if (threadIdx.x == 0) {
    const double st = tot[0] / d.norms[0], da = tot[1] / d.norms[1];
    terms[1] = st;
    terms[2] = da;
    terms[3] = tot[2];
    terms[4] = tot[3];
    terms[5] = tot[4];
    terms[0] = st + da + (double)d.lam_bound * tot[2] + (double)d.lam_tv * tot[3] + (double)d.lam_bridge * tot[4];
  }
}

template <int P>
static pdf_status launch_cluster(pdf_problem* h, ClusterArgs a, size_t smem, cudaStream_t st, bool* done) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_cluster_solve<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
    cudaFuncSetAttribute(k_cluster_solve<P>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaGetLastError();
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(h->d.ni * a.C);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = a.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeCooperative;
  at[1].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, (void*)k_cluster_solve<P>, &cfg) != cudaSuccess ||
      nclusters < h->d.ni) {
    cudaGetLastError();
    return PDF_OK;                                  // does not fit co-resident: caller falls back
  }
  Dev d = h->d;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_cluster_solve<P>, d, a);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return PDF_OK;                                  // launch form unsupported: caller falls back
  }
  pdf_count_launch(1);
  *done = true;
  return PDF_OK;
}

// Runs `iters` Adam iterations of h->alpha with the cluster kernel and writes the last
// iteration's loss terms to h->terms.  *done = false (nothing launched) when not eligible.
pdf_status cl_run(pdf_problem* h, const pdf_solve_opts* o, int iters, cudaStream_t st, bool* done) {
  *done = false;
  const Dev& d = h->d;
  if (!d.fast || h->tc || d.Px != d.Py || d.Px > 128 || iters < 1 || d.kx > 64) return PDF_OK;
  int dev = 0, sms = 0, coop = 0;
  PDF_CUDA(cudaGetDevice(&dev));
  PDF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PDF_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return PDF_OK;
  if (!h->cl_nd) {
    pdf_status s;
    if ((s = ws_alloc(h, (void**)&h->cl_nd, sizeof(float) * 2 * 3 * (size_t)d.ni * d.M)) != PDF_OK) return s;
    if ((s = ws_alloc(h, (void**)&h->cl_lp, sizeof(FF) * 5 * (size_t)d.ni * 16)) != PDF_OK) return s;
  }
  ClusterArgs a;
  a.iters = iters;
  a.alpha = h->alpha;
  a.tab = h->adam_tab;
  a.cap = h->adam_cap;
  a.b1 = (float)o->adam_b1;
  a.b2 = (float)o->adam_b2;
  a.eps = (float)o->adam_eps;
  a.nd = h->cl_nd;
  a.lpart = h->cl_lp;
  a.bar = h->bar;
  a.err = h->perr;
  PDF_CUDA(cudaMemsetAsync(h->bar, 0, sizeof(unsigned), st));
  pdf_status s = PDF_OK;
  int C = 0;
  for (int c = 16; c >= 2 && !*done; c >>= 1) {
    if (!cluster_ok(d, sms, c)) continue;
    a.C = c;
    a.RB = d.ny / c;
    a.CB = d.Px / c;
    size_t smem = cluster_smem(d, c, a.RB, a.CB, d.Px, true);
    a.gs_smem = 1;
    if (smem > 210 * 1024) {
      smem = cluster_smem(d, c, a.RB, a.CB, d.Px, false);
      a.gs_smem = 0;
    }
    if (smem > 210 * 1024) continue;
    if (d.Px == 64) s = launch_cluster<64>(h, a, smem, st, done);
    else if (d.Px == 128) s = launch_cluster<128>(h, a, smem, st, done);
    if (s != PDF_OK) return s;
    C = c;
  }
  if (!*done) return PDF_OK;
  k_cluster_finalize<<<1, 256, 0, st>>>(h->d, h->cl_lp, d.ni * C, h->terms);
  pdf_count_launch(1);
  PDF_LAUNCHED("cluster loss terms");
  return PDF_OK;
}
