// Whole reconstruction around the hot path (Sec. 3): BP + one-step CSI initialisation
// (Sec. 3.1, Eq. 12), the Adam loop on alpha (Sec. 3.3) captured as a CUDA graph, the final
// chi-hat, the contrast-compensated operator (Sec. 2.4, Eq. 10-11), the relative error,
// and the forward scattering solve used to synthesise measured data (Eq. 3-5).
//
// Readings (the paper cites but does not print them):
//   BP       J_p = gamma_p G_S^H E_p with gamma_p = ||G_S^H E_p||^2 / ||G_S G_S^H E_p||^2;
//            E_tot = E_inc + G_D J; chi_0 = per-pixel least squares of J = chi E_tot; R_0 by Eq. (7).
//   CSI step alpha_0 = -t g, g = grad L^CSI(0) at fixed R_0, t the exact line-search minimiser
//            ||g||^2 / (2 (||G_S F* g||^2/||E_sca||^2 + ||A F* g||^2/||E_inc||^2)),
//            A = R_0 (beta I + G_D) - beta I.
//   CCO      self-guided filter (box radius r, clipped windows, Re and Im separately),
//            eta = eta_max sigmoid((|chi| - tau)/delta), out = (1 + eta) G + eta chi.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <vector>

#include "fft.cuh"
#include "phases.cuh"
#include "problem.cuh"

// ---------------------------------------------------------------------------
// Adam on the real view of alpha (torch.optim.Adam arithmetic, FP32)
// ---------------------------------------------------------------------------
__global__ void k_adam(float* p, const float* g, float* m, float* v, int n, const int* tdev, const float2* tab,
                       int cap, float b1, float b2, float eps) {
  pdl_wait();
  ph_adam(blockIdx.x * blockDim.x + threadIdx.x, p, g, m, v, n, *tdev, tab, cap, b1, b2, eps);
}

// Bias-correction table of torch.optim.Adam for steps 1..iters (rebuilt when lr, betas or the
// iteration count change; the solve's CUDA graph holds its address, so it is reset too).
static pdf_status ensure_adam_table(pdf_problem* h, const pdf_solve_opts* o) {
  const int need = std::max(o->iters, 1);
  if (h->adam_tab && h->adam_cap >= need && h->adam_key[0] == o->lr && h->adam_key[1] == o->adam_b1 &&
      h->adam_key[2] == o->adam_b2)
    return PDF_OK;
  const int cap = std::max(need, 1024);
  std::vector<float2> tab(cap);
  for (int t = 1; t <= cap; ++t) {
    const double bc1 = 1.0 - std::pow(o->adam_b1, t), bc2 = 1.0 - std::pow(o->adam_b2, t);
    tab[t - 1] = make_float2((float)(o->lr / bc1), (float)std::sqrt(bc2));
  }
  if (!h->adam_tab || h->adam_cap < cap) {
    if (h->graph_exec) {
      cudaGraphExecDestroy(h->graph_exec);
      h->graph_exec = nullptr;
    }
    float2* p = nullptr;
    pdf_status s = ws_alloc(h, (void**)&p, sizeof(float2) * cap);
    if (s != PDF_OK) return s;
    h->adam_tab = p;
    h->adam_cap = cap;
  }
  PDF_CUDA(cudaMemcpy(h->adam_tab, tab.data(), sizeof(float2) * cap, cudaMemcpyHostToDevice));
  h->adam_key[0] = o->lr;
  h->adam_key[1] = o->adam_b1;
  h->adam_key[2] = o->adam_b2;
  h->d.adam_tab = h->adam_tab;
  return PDF_OK;
}

// ---------------------------------------------------------------------------
// CCO: guided-filter coefficients, then the combination
// ---------------------------------------------------------------------------
__global__ void k_cco_ab(const float2* __restrict__ chi, float4* __restrict__ ab, int nx, int ny, int rad, float eps) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nx * ny) return;
  const int y = n / nx, x = n - y * nx;
  const int y0 = max(0, y - rad), y1 = min(ny - 1, y + rad), x0 = max(0, x - rad), x1 = min(nx - 1, x + rad);
  float sr = 0.f, si = 0.f, srr = 0.f, sii = 0.f;
  for (int yy = y0; yy <= y1; ++yy)
    for (int xx = x0; xx <= x1; ++xx) {
      const float2 c = chi[yy * nx + xx];
      sr += c.x;
      si += c.y;
      srr += c.x * c.x;
      sii += c.y * c.y;
    }
  const float inv = 1.f / (float)((y1 - y0 + 1) * (x1 - x0 + 1));
  const float mr = sr * inv, mi = si * inv;
  const float vr = srr * inv - mr * mr, vi = sii * inv - mi * mi;
  const float ar = vr / (vr + eps), ai = vi / (vi + eps);
  ab[n] = make_float4(ar, mr - ar * mr, ai, mi - ai * mi);
}

__global__ void k_cco_out(const float2* __restrict__ chi, const float4* __restrict__ ab, float2* __restrict__ out,
                          int nx, int ny, int rad, float eta_max, float tau, float delta, float sign) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nx * ny) return;
  const int y = n / nx, x = n - y * nx;
  const int y0 = max(0, y - rad), y1 = min(ny - 1, y + rad), x0 = max(0, x - rad), x1 = min(nx - 1, x + rad);
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int yy = y0; yy <= y1; ++yy)
    for (int xx = x0; xx <= x1; ++xx) {
      const float4 q = ab[yy * nx + xx];
      s.x += q.x;
      s.y += q.y;
      s.z += q.z;
      s.w += q.w;
    }
  const float inv = 1.f / (float)((y1 - y0 + 1) * (x1 - x0 + 1));
  const float2 c = chi[n];
  const float2 gq = make_float2(s.x * inv * c.x + s.y * inv, s.z * inv * c.y + s.w * inv);
  const float eta = eta_max / (1.f + expf(-(sqrtf(cabs2(c)) - tau) / delta));
  out[n] = (1.f + eta) * gq + (sign * eta) * c;
}

// ---------------------------------------------------------------------------
// per-incidence reductions and small pointwise kernels of the initialisation
// ---------------------------------------------------------------------------
// out[p] = sum_i |x[p][i]|^2 (Kahan FP32 per thread, FP64 across threads); grid = ni blocks
__global__ void k_sumsq_per_p(const float2* __restrict__ x, int L, double* __restrict__ out) {
  __shared__ double red[32];
  const int p = blockIdx.x;
  float s = 0.f, c = 0.f;
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    const float v = cabs2(x[(size_t)p * L + i]);
    const float y = v - c, t = s + y;
    c = (t - s) - y;
    s = t;
  }
  const double r = block_sum((double)s - (double)c, red);
  if (threadIdx.x == 0) out[p] = r;
}

// out[p] = sum_i conj(a[p][i]) b[p][i] (complex); grid = ni blocks
__global__ void k_dot_per_p(const float2* __restrict__ a, const float2* __restrict__ b, int L, double2* __restrict__ out) {
  __shared__ double red[32];
  const int p = blockIdx.x;
  float sr = 0.f, si = 0.f;
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    const float2 z = cmulc(b[(size_t)p * L + i], a[(size_t)p * L + i]);
    sr += z.x;
    si += z.y;
  }
  const double rr = block_sum((double)sr, red);
  const double ri = block_sum((double)si, red);
  if (threadIdx.x == 0) out[p] = make_double2(rr, ri);
}

// x[i] *= factor / *norm
__global__ void k_scale_by_norm(float2* __restrict__ x, size_t n, const double* __restrict__ norm, double factor) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[i] = (float)(factor / *norm) * x[i];
}

// x[p][i] *= num[p] / den[p]
__global__ void k_scale_per_p(float2* __restrict__ x, int L, const double* __restrict__ num,
                              const double* __restrict__ den) {
  const int p = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L) return;
  const float s = (float)(num[p] / den[p]);
  x[(size_t)p * L + i] = s * x[(size_t)p * L + i];
}

// E_tot = E_inc + G_D J (in place into gdj); chi_0 per pixel; R_0 = beta chi_0 / (beta chi_0 + 1)
__global__ void k_init_chi0(Dev d, const float2* __restrict__ J, float2* __restrict__ gdj, float2* __restrict__ R0) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= d.M) return;
  float nr = 0.f, ni = 0.f, dd = 0.f;
  for (int p = 0; p < d.ni; ++p) {
    const size_t idx = (size_t)p * d.M + n;
    const float2 e = d.einc[idx] + gdj[idx];
    gdj[idx] = e;
    const float2 z = cmulc(J[idx], e);
    nr += z.x;
    ni += z.y;
    dd += cabs2(e);
  }
  const float2 chi0 = make_float2(nr / dd, ni / dd);
  const float2 bc = cmul(d.beta, chi0);
  R0[n] = cdivf(bc, make_float2(bc.x + 1.f, bc.y));
}

// x = conj(R0) R0 E_inc (the G_D^H input of the CSI gradient at alpha = 0)
__global__ void k_init_x(Dev d, const float2* __restrict__ R0, float2* __restrict__ x) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)d.ni * d.M) return;
  const int n = (int)(i % d.M);
  const float2 R = R0[n];
  x[i] = cabs2(R) * d.einc[i];
}

// gJ = gsh_term + (2/||Einc||^2) (conj(beta) (x - r0) + G_D^H x),  r0 = R0 E_inc
__global__ void k_init_gj(Dev d, const float2* __restrict__ R0, const float2* __restrict__ gdhx,
                          float2* __restrict__ gJ) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)d.ni * d.M) return;
  const int n = (int)(i % d.M);
  const float ke = d.invn[0];
  const float2 R = R0[n];
  const float2 e = d.einc[i];
  const float2 r0 = cmul(R, e);
  const float2 x = cabs2(R) * e;
  gJ[i] = gJ[i] + ke * (cmul(cconj(d.beta), x - r0) + gdhx[i]);
}

// m2 = R0 (beta Jg + G_D Jg) - beta Jg; per-block partial sums of |m2|^2 -> part[block]
__global__ void k_init_m2(Dev d, const float2* __restrict__ R0, const float2* __restrict__ Jg,
                          const float2* __restrict__ gdJg, double* __restrict__ part) {
  __shared__ double red[32];
  float a = 0.f, c = 0.f;
  const size_t n_all = (size_t)d.ni * d.M;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_all; i += (size_t)gridDim.x * blockDim.x) {
    const int n = (int)(i % d.M);
    const float2 bj = cmul(d.beta, Jg[i]);
    const float2 m2 = cmul(R0[n], bj + gdJg[i]) - bj;
    const float y = cabs2(m2) - c, t = a + y;
    c = (t - a) - y;
    a = t;
  }
  const double t = block_sum((double)a - (double)c, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// sc layout: [0] ||g||^2, [1] ||m1||^2, [2] ||m2||^2 ; alpha = -t g
__global__ void k_init_alpha(Dev d, const float2* __restrict__ g, float2* __restrict__ alpha, const double* sc, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double den = sc[1] / d.norms[1] + sc[2] / d.norms[0];
  const float t = (float)(sc[0] / (2.0 * den));
  alpha[i] = (-t) * g[i];
}

// dst = ||a - b|| / ||b|| (single block, double accumulation)
__global__ void k_relerr_to(const float2* __restrict__ a, const float2* __restrict__ b, int n, double* dst) {
  __shared__ double red[32];
  double e = 0.0, t = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double2 bd = to_d(b[i]);
    e += cabs2(to_d(a[i]) - bd);
    t += cabs2(bd);
  }
  const double se = block_sum(e, red);
  const double st = block_sum(t, red);
  if (threadIdx.x == 0) *dst = sqrt(se / st);
}

// warm start with fallback: keep alpha (BP + CSI) unless the candidate's loss is not larger
__global__ void k_pick_warm(float2* __restrict__ alpha, const float2* __restrict__ cand, const double* la,
                            const double* lb, int n, int* used) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool take = isfinite(lb[0]) && lb[0] <= la[0];
  if (i < n && take) alpha[i] = cand[i];
  if (i == 0) *used = take ? 1 : 0;
}

__global__ void k_sum_d(const double* in, int n, double* out) {
  __shared__ double red[32];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += in[i];
  const double t = block_sum(a, red);
  if (threadIdx.x == 0) *out = t;
}

// ---------------------------------------------------------------------------
// host pieces
// ---------------------------------------------------------------------------
pdf_status sv_cco(pdf_problem* h, const float2* chi, float2* out, int radius, double eps, double eta_max,
                  double tau, double delta, cudaStream_t st) {
  const Dev& d = h->d;
  const int nb = (d.M + 255) / 256;
  k_cco_ab<<<nb, 256, 0, st>>>(chi, h->cco_ab, d.nx, d.ny, radius, (float)eps);
  k_cco_out<<<nb, 256, 0, st>>>(chi, h->cco_ab, out, d.nx, d.ny, radius, (float)eta_max, (float)tau, (float)delta,
                                1.f);
  pdf_count_launch(2);
  PDF_LAUNCHED("CCO");
  return PDF_OK;
}

// BP + one exact-line-search CSI step; writes h->alpha.
static pdf_status init_bp_csi(pdf_problem* h, cudaStream_t st) {
  Dev& d = h->d;
  const int L = d.M;
  const size_t NF = (size_t)d.ni * d.M;
  const int NA = d.ni * d.ky * d.kx;
  double* sc = h->scratch_d;            // [0..2] line-search scalars
  double* num = (double*)d.lpart + PDF_LP_STRIDE;            // [ni] per-incidence sums (lpart as scratch)
  double* den = num + d.ni;
  pdf_status s;
  // BP: gh = G_S^H E_sca (tmpA); ggh = G_S gh (small1); gamma_p
  if ((s = hp_gsh(h, d.esca, h->tmpA, 1.0f, st)) != PDF_OK) return s;
  if ((s = hp_gs(h, h->tmpA, h->small1, nullptr, nullptr, st)) != PDF_OK) return s;
  k_sumsq_per_p<<<d.ni, 256, 0, st>>>(h->tmpA, L, num);
  k_sumsq_per_p<<<d.ni, 256, 0, st>>>(h->small1, d.nr, den);
  k_scale_per_p<<<dim3((L + 255) / 256, d.ni), 256, 0, st>>>(h->tmpA, L, num, den);  // J_bp
  pdf_count_launch(3);
  if ((s = hp_gd(h, h->tmpA, h->tmpB, 0, st)) != PDF_OK) return s;                   // G_D J_bp
  k_init_chi0<<<(L + 255) / 256, 256, 0, st>>>(d, h->tmpA, h->tmpB, h->field1);       // R_0
  // CSI gradient at alpha = 0: data part (2/||E||^2) G_S^H(-E) into tmpC
  k_init_x<<<(unsigned)((NF + 255) / 256), 256, 0, st>>>(d, h->field1, h->tmpA);
  pdf_count_launch(2);
  if ((s = hp_gd(h, h->tmpA, h->tmpB, 1, st)) != PDF_OK) return s;                   // G_D^H x
  // data part of the CSI gradient: -(2/||E_sca||^2) G_S^H E_sca into tmpC
  if ((s = hp_gsh(h, d.esca, h->tmpC, 1.0f, st)) != PDF_OK) return s;
  k_scale_by_norm<<<(unsigned)((NF + 255) / 256), 256, 0, st>>>(h->tmpC, NF, d.norms + 1, -2.0);
  k_init_gj<<<(unsigned)((NF + 255) / 256), 256, 0, st>>>(d, h->field1, h->tmpB, h->tmpC);
  pdf_count_launch(2);
  if ((s = hp_analysis(h, h->tmpC, h->grad, st)) != PDF_OK) return s;                // g
  // line search
  if ((s = hp_synth(h, h->grad, h->tmpA, st)) != PDF_OK) return s;                   // Jg = F* g
  if ((s = hp_gs(h, h->tmpA, h->small1, nullptr, nullptr, st)) != PDF_OK) return s;  // m1
  if ((s = hp_gd(h, h->tmpA, h->tmpB, 0, st)) != PDF_OK) return s;                   // G_D Jg
  const int nb = (int)std::min<size_t>((NF + 255) / 256, PDF_LP_STRIDE);
  k_init_m2<<<nb, 256, 0, st>>>(d, h->field1, h->tmpA, h->tmpB, (double*)d.lpart);
  k_sum_d<<<1, 256, 0, st>>>((double*)d.lpart, nb, sc + 2);
  k_sumsq<<<1, 1024, 0, st>>>(h->small1, d.ni * d.nr, sc + 1);
  k_sumsq<<<1, 1024, 0, st>>>(h->grad, NA, sc + 0);
  k_init_alpha<<<(NA + 255) / 256, 256, 0, st>>>(d, h->grad, h->alpha, sc, NA);
  pdf_count_launch(5);
  PDF_LAUNCHED("BP/CSI initialisation");
  return PDF_OK;
}

static pdf_status adam_step(pdf_problem* h, const pdf_solve_opts* o, cudaStream_t st) {
  const int n = 2 * h->d.ni * h->d.ky * h->d.kx;
  launch_pdl(k_adam, (n + 255) / 256, 256, 0, st, (float*)h->alpha, (const float*)h->grad, h->adam_m, h->adam_v, n,
             (const int*)h->adam_t, (const float2*)h->adam_tab, h->adam_cap, (float)o->adam_b1, (float)o->adam_b2,
             (float)o->adam_eps);
  pdf_count_launch(1);
  PDF_LAUNCHED("Adam");
  return PDF_OK;
}

static pdf_status iteration(pdf_problem* h, const pdf_solve_opts* o, cudaStream_t st) {
  // the loss terms are summed only when a history row wants them
  double* terms = o->history_every > 0 ? h->terms : nullptr;
  if (h->fc_active) {
    // alpha = alpha0 + Delta alpha(theta); loss gradient; chain rule to theta; Adam on theta
    pdf_status s = fc_forward(h, st);
    if (s != PDF_OK) return s;
    if ((s = hp_loss_grad(h, h->alpha, h->grad, terms, st, h->adam_t)) != PDF_OK) return s;
    if ((s = fc_backward(h, st)) != PDF_OK) return s;
    const int n = (int)h->fc.np;
    launch_pdl(k_adam, (n + 255) / 256, 256, 0, st, h->fc.theta, (const float*)h->fc.gtheta, h->fc.m, h->fc.v, n,
               (const int*)h->adam_t, (const float2*)h->adam_tab, h->adam_cap, (float)o->adam_b1, (float)o->adam_b2,
               (float)o->adam_eps);
    pdf_count_launch(1);
    PDF_LAUNCHED("Adam on the network weights");
    return PDF_OK;
  }
  pdf_status s = hp_loss_grad(h, h->alpha, h->grad, terms, st, h->adam_t);
  if (s != PDF_OK) return s;
  return adam_step(h, o, st);
}

#define GRAPH_UNROLL 10

static pdf_status build_graph(pdf_problem* h, const pdf_solve_opts* o) {
  const double width = h->fc_active ? (double)h->fc.H : 0.0;
  if (h->graph_exec && h->graph_key[0] == o->lr && h->graph_key[1] == o->adam_b1 && h->graph_key[2] == o->adam_b2 &&
      h->graph_key[3] == o->adam_eps && h->graph_key[4] == width)
    return PDF_OK;
  if (h->graph_exec) {
    cudaGraphExecDestroy(h->graph_exec);
    h->graph_exec = nullptr;
  }
  cudaStream_t cs = h->cap_stream;
  PDF_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  const uint64_t before = pdf_launch_count();
  pdf_status s = PDF_OK;
  for (int k = 0; k < GRAPH_UNROLL && s == PDF_OK; ++k) s = iteration(h, o, cs);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &g);
  const uint64_t nk = pdf_launch_count() - before;
  pdf_count_launch((uint64_t)0 - nk);   // capture does not launch anything
  if (s != PDF_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return cuda_err(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&h->graph_exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_err(e, "cudaGraphInstantiate");
  h->graph_iters = GRAPH_UNROLL;
  h->graph_kernels = (int)nk;
  h->graph_key[0] = o->lr;
  h->graph_key[1] = o->adam_b1;
  h->graph_key[2] = o->adam_b2;
  h->graph_key[3] = o->adam_eps;
  h->graph_key[4] = width;
  return PDF_OK;
}

// The CCO of a solve's output: with the CCO inside the loss, the parameters the loss used.
static pdf_status final_cco(pdf_problem* h, const pdf_solve_opts* o, const float2* chi, float2* out,
                            cudaStream_t st) {
  const pdf_config& c = h->cfg;
  if (c.cco_in_loss) return sv_cco(h, chi, out, c.cco_radius, c.cco_eps, c.cco_eta_max, c.cco_tau, c.cco_delta, st);
  return sv_cco(h, chi, out, o->cco_radius, o->cco_eps, o->cco_eta_max, o->cco_tau, o->cco_delta, st);
}

// Resets the Adam state of alpha (or of the network's weights) to step 0.
static pdf_status reset_adam(pdf_problem* h, cudaStream_t st) {
  const int NA = h->d.ni * h->d.ky * h->d.kx;
  PDF_CUDA(cudaMemsetAsync(h->adam_m, 0, sizeof(float) * 2 * NA, st));
  PDF_CUDA(cudaMemsetAsync(h->adam_v, 0, sizeof(float) * 2 * NA, st));
  PDF_CUDA(cudaMemsetAsync(h->adam_t, 0, sizeof(int), st));
  return PDF_OK;
}

// Runs the Adam iterations of a solve from the current alpha.  fused = 0 forbids the one-launch
// loop forms (the fallback after a cluster launch that came up without its shape).
static pdf_status run_loop(pdf_problem* h, const pdf_solve_opts* o, int fused, int* loop_mode, cudaStream_t st) {
  const Dev& d = h->d;
  pdf_status s;
  int it = 0;
  *loop_mode = 0;
  if (o->history_every > 0) {
    for (; it < o->iters; ++it) {
      if ((s = iteration(h, o, st)) != PDF_OK) return s;
      if (it % o->history_every == 0) {
        double* row = o->history + 8 * (it / o->history_every);
        PDF_CUDA(cudaMemcpyAsync(row, h->terms, 6 * sizeof(double), cudaMemcpyDeviceToDevice, st));
        if (o->chi_true) {
          // chi-hat of this iteration's alpha (before its Adam step) and its CCO image
          k_relerr_to<<<1, 1024, 0, st>>>(d.chi, (const float2*)o->chi_true, d.M, row + 6);
          pdf_count_launch(1);
          if (o->apply_cco) {
            if ((s = final_cco(h, o, d.chi, h->field3, st)) != PDF_OK) return s;
            k_relerr_to<<<1, 1024, 0, st>>>(h->field3, (const float2*)o->chi_true, d.M, row + 7);
            pdf_count_launch(1);
          }
          PDF_LAUNCHED("history relerr");
        }
      }
    }
    return PDF_OK;
  }
  bool persisted = false;
  if (fused && o->use_graph == 3) {
    if ((s = cl_run(h, o, o->iters, st, &persisted)) != PDF_OK) return s;
    if (persisted) {
      it = o->iters;
      *loop_mode = 3;
    }
  }
  if (fused && !persisted && o->use_graph == 2 && !h->fc_active) {
    if ((s = ps_run(h, o, o->iters, h->bar, h->perr, st, &persisted)) != PDF_OK) return s;
    if (persisted) {
      it = o->iters;
      *loop_mode = 2;
    }
  }
  if (!persisted && o->use_graph && o->iters >= GRAPH_UNROLL) {
    if ((s = build_graph(h, o)) != PDF_OK) return s;
    *loop_mode = 1;
    for (; it + h->graph_iters <= o->iters; it += h->graph_iters) {
      PDF_CUDA(cudaGraphLaunch(h->graph_exec, st));
      pdf_count_launch(h->graph_kernels);
    }
  }
  for (; it < o->iters; ++it)
    if ((s = iteration(h, o, st)) != PDF_OK) return s;
  return PDF_OK;
}

// flag[0] |= any element of x not finite
__global__ void k_nonfinite(const float2* __restrict__ x, int n, int* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const float2 v = x[i];
    if (!isfinite(v.x) || !isfinite(v.y)) *flag = 1;
  }
}

// ||a1 - b||^2, ||b||^2, ||a2 - b||^2 (a2 may be NULL) over n elements -> out[0], out[1], out[2],
// out[3] = out[1]: FP32 Kahan sums per thread, FP64 sums per block into part[block][3], and the last
// block to finish sums the partials in block order (deterministic).
__global__ void __launch_bounds__(256) k_relerr2(const float2* __restrict__ a1, const float2* __restrict__ a2,
                                                 const float2* __restrict__ b, int n, double* __restrict__ part,
                                                 unsigned* __restrict__ count, double* __restrict__ out) {
  __shared__ double red[32];
  __shared__ bool last;
  float s[3] = {0.f, 0.f, 0.f}, c[3] = {0.f, 0.f, 0.f};
  auto kahan = [&](int k, float v) {
    const float y = v - c[k], t = s[k] + y;
    c[k] = (t - s[k]) - y;
    s[k] = t;
  };
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float2 bv = b[i];
    kahan(0, cabs2(a1[i] - bv));
    kahan(1, cabs2(bv));
    if (a2) kahan(2, cabs2(a2[i] - bv));
  }
  for (int k = 0; k < 3; ++k) {
    const double t = block_sum((double)s[k] - (double)c[k], red);
    if (threadIdx.x == 0) part[3 * blockIdx.x + k] = t;
  }
  __threadfence();
  if (threadIdx.x == 0) last = atomicAdd(count, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t[3] = {0.0, 0.0, 0.0};
  for (int j = threadIdx.x; j < (int)gridDim.x; j += blockDim.x)
    for (int k = 0; k < 3; ++k) t[k] += __ldcg(&part[3 * j + k]);
  for (int k = 0; k < 3; ++k) t[k] = block_sum(t[k], red);
  if (threadIdx.x == 0) {
    out[0] = t[0];
    out[1] = t[1];
    out[2] = t[2];
    out[3] = t[1];
    *count = 0u;
  }
}

// Final chi-hat, CCO, outputs and (with a truth) the two RelErr sums; then the status check.
static pdf_status finish(pdf_problem* h, const pdf_solve_opts* o, float2* chi_out, float2* chi_raw_out,
                         float2* alpha_out, bool terms, cudaStream_t st) {
  Dev& d = h->d;
  const int NA = d.ni * d.ky * d.kx;
  pdf_status s;
  if (h->fc_active) {                                                  // alpha-hat at the final weights
    if ((s = fc_forward(h, st)) != PDF_OK) return s;
  }
  // final chi-hat (and loss terms when a report is requested)
  if (terms) {
    if ((s = hp_loss_grad(h, h->alpha, h->grad, h->terms, st)) != PDF_OK) return s;
  } else {
    if ((s = hp_chi(h, h->alpha, nullptr, st)) != PDF_OK) return s;
  }
  if (chi_raw_out) PDF_CUDA(cudaMemcpyAsync(chi_raw_out, d.chi, sizeof(float2) * d.M, cudaMemcpyDeviceToDevice, st));
  PDF_CUDA(cudaMemcpyAsync(h->field2, d.chi, sizeof(float2) * d.M, cudaMemcpyDeviceToDevice, st));
  if (o->apply_cco) {
    if ((s = final_cco(h, o, h->field2, h->field3, st)) != PDF_OK) return s;
  } else {
    PDF_CUDA(cudaMemcpyAsync(h->field3, h->field2, sizeof(float2) * d.M, cudaMemcpyDeviceToDevice, st));
  }
  if (chi_out) PDF_CUDA(cudaMemcpyAsync(chi_out, h->field3, sizeof(float2) * d.M, cudaMemcpyDeviceToDevice, st));
  if (alpha_out) PDF_CUDA(cudaMemcpyAsync(alpha_out, h->alpha, sizeof(float2) * NA, cudaMemcpyDeviceToDevice, st));
  const int nb = (d.M + 255) / 256;
  k_nonfinite<<<nb, 256, 0, st>>>(h->field3, d.M, h->perr + 1);
  pdf_count_launch(1);
  if (o->chi_true) {
    const int g = std::min(nb, RELERR_BLOCKS);
    k_relerr2<<<g, 256, 0, st>>>(h->field2, h->field3, (const float2*)o->chi_true, d.M, h->relerr_part,
                                 (unsigned*)(h->perr + 2), h->scratch_d + 40);
    pdf_count_launch(1);
  }
  PDF_LAUNCHED("final contrast");
  return PDF_OK;
}

pdf_status sv_solve(pdf_problem* h, const pdf_solve_opts* o, float2* chi_out, float2* chi_raw_out,
                    float2* alpha_out, pdf_solve_report* rep, cudaStream_t st) {
  Dev& d = h->d;
  const int NA = d.ni * d.ky * d.kx;
  pdf_status s;
  if ((s = ensure_adam_table(h, o)) != PDF_OK) return s;
  PDF_CUDA(cudaMemsetAsync(h->used_warm, 0, sizeof(int), st));
  PDF_CUDA(cudaMemsetAsync(h->perr, 0, 2 * sizeof(int), st));      // loop error, non-finite output
  if (o->init == 0) {
    if ((s = init_bp_csi(h, st)) != PDF_OK) return s;
  } else if (o->init == 3) {
    // warm start with fallback: L at the BP + CSI start vs L at the given alpha0
    if ((s = init_bp_csi(h, st)) != PDF_OK) return s;
    if ((s = hp_loss_grad(h, h->alpha, h->grad, h->scratch_d + 48, st)) != PDF_OK) return s;
    PDF_CUDA(cudaMemcpyAsync(h->alpha_alt, o->alpha0, sizeof(float2) * NA, cudaMemcpyDeviceToDevice, st));
    if ((s = hp_loss_grad(h, h->alpha_alt, h->grad, h->scratch_d + 56, st)) != PDF_OK) return s;
    k_pick_warm<<<(NA + 255) / 256, 256, 0, st>>>(h->alpha, h->alpha_alt, h->scratch_d + 48, h->scratch_d + 56, NA,
                                                  h->used_warm);
    pdf_count_launch(1);
    PDF_LAUNCHED("warm-start selection");
  } else if (o->init == 1) {
    PDF_CUDA(cudaMemcpyAsync(h->alpha, o->alpha0, sizeof(float2) * NA, cudaMemcpyDeviceToDevice, st));
  } else {
    PDF_CUDA(cudaMemsetAsync(h->alpha, 0, sizeof(float2) * NA, st));
  }
  if ((s = reset_adam(h, st)) != PDF_OK) return s;
  h->fc_active = 0;
  if (o->fcnn_hidden > 0) {                                           // the network's input is this alpha
    if (h->fc.H != o->fcnn_hidden && h->graph_exec) {                  // the graph holds the old buffers
      cudaGraphExecDestroy(h->graph_exec);
      h->graph_exec = nullptr;
    }
    if ((s = fc_prepare(h, o->fcnn_hidden, o->fcnn_params0, st)) != PDF_OK) return s;
    h->fc_active = 1;
  }
  int loop_mode = 0;                  // which loop form ran (reported)
  if ((s = run_loop(h, o, 1, &loop_mode, st)) != PDF_OK) return s;
  if ((s = finish(h, o, chi_out, chi_raw_out, alpha_out, rep != nullptr, st)) != PDF_OK) return s;
  // device-side status: the one-launch loops' error flag and the finiteness of the output
  int flag[2] = {0, 0};
  PDF_CUDA(cudaMemcpyAsync(flag, h->perr, sizeof(flag), cudaMemcpyDeviceToHost, st));
  PDF_CUDA(cudaStreamSynchronize(st));
  if (flag[0] == 2 && loop_mode == 3) {
    // the cluster kernel returned on entry without touching alpha or the Adam state: run the same
    // iterations as the CUDA graph of the stand-alone kernels and finish again
    PDF_CUDA(cudaMemsetAsync(h->perr, 0, 2 * sizeof(int), st));
    if ((s = reset_adam(h, st)) != PDF_OK) return s;
    if ((s = run_loop(h, o, 0, &loop_mode, st)) != PDF_OK) return s;
    if ((s = finish(h, o, chi_out, chi_raw_out, alpha_out, rep != nullptr, st)) != PDF_OK) return s;
    PDF_CUDA(cudaMemcpyAsync(flag, h->perr, sizeof(flag), cudaMemcpyDeviceToHost, st));
    PDF_CUDA(cudaStreamSynchronize(st));
  }
  if (flag[0] != 0) {
    PDF_CUDA(cudaMemset(h->perr, 0, 2 * sizeof(int)));
    if (flag[0] == 1)
      return set_err(PDF_ETIMEOUT, loop_mode == 3 ? "a grid barrier of the cluster solve loop timed out"
                                                  : "a grid barrier of the persistent solve loop timed out");
    return set_err(PDF_EUNSUPPORTED, "the one-launch solve loop was not launched in the form it needs");
  }
  if (rep) {
    memset(rep, 0, sizeof(*rep));
    rep->iters_run = o->iters;
    rep->loop_mode = loop_mode;
    double re[4] = {NAN, NAN, NAN, NAN};
    int used = 0;
    PDF_CUDA(cudaMemcpy(rep->terms, h->terms, 6 * sizeof(double), cudaMemcpyDeviceToHost));
    if (o->chi_true) PDF_CUDA(cudaMemcpy(re, h->scratch_d + 40, 4 * sizeof(double), cudaMemcpyDeviceToHost));
    PDF_CUDA(cudaMemcpy(&used, h->used_warm, sizeof(int), cudaMemcpyDeviceToHost));
    rep->relerr = o->chi_true ? sqrt(re[0] / re[1]) : NAN;
    rep->relerr_cco = o->chi_true ? sqrt(re[2] / re[3]) : NAN;
    rep->used_warm_start = used;
    for (int k = 0; k < 6; ++k)
      if (!std::isfinite(rep->terms[k])) rep->nonfinite = 1;
    if (flag[1]) rep->nonfinite = 1;
  }
  if (flag[1]) return set_err(PDF_ENONFINITE, "the reconstructed contrast is not finite");
  if (rep && rep->nonfinite) return set_err(PDF_ENONFINITE, "a loss term is not finite");
  return PDF_OK;
}

// ---------------------------------------------------------------------------
// forward solve: batched BiCGSTAB on (I - G_D diag(chi)) E = E_inc, one system per incidence
// ---------------------------------------------------------------------------
__global__ void k_mul_chi(const float2* __restrict__ chi, const float2* __restrict__ x, float2* __restrict__ y,
                          int M, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  y[i] = cmul(chi[i % M], x[i]);
}

// y = x - y  (A x = x - G_D(chi x), y holds G_D(chi x) on entry)
__global__ void k_xmy(const float2* __restrict__ x, float2* __restrict__ y, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  y[i] = x[i] - y[i];
}

// BiCGSTAB state per incidence: sc[p] = {rho, alpha, omega} (double2 each) in a packed array
struct BiState { double2 rho, alpha, omega; };

// p = r + beta (p - omega v), beta = (rho_new / rho)(alpha / omega); rho <- rho_new
__global__ void k_bi_p(float2* __restrict__ P, const float2* __restrict__ R, const float2* __restrict__ V,
                       BiState* st, const double2* __restrict__ rho_new, int M, int first) {
  const int p = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const BiState s = st[p];
  const double2 rn = rho_new[p];
  float2 beta = make_float2(0.f, 0.f);
  if (!first) beta = to_f(cmul(cdiv(rn, s.rho), cdiv(s.alpha, s.omega)));
  if (i < M) {
    const size_t k = (size_t)p * M + i;
    P[k] = first ? R[k] : R[k] + cmul(beta, P[k] - cmul(to_f(s.omega), V[k]));
  }
}

__global__ void k_bi_rho_commit(BiState* st, const double2* rho_new, int ni) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < ni) st[p].rho = rho_new[p];
}

// alpha = rho / <rhat, v>;  s = r - alpha v (into R)
__global__ void k_bi_s(float2* __restrict__ R, const float2* __restrict__ V, BiState* st,
                       const double2* __restrict__ rv, int M) {
  const int p = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double2 al = cdiv(st[p].rho, rv[p]);
  if (i < M) {
    const size_t k = (size_t)p * M + i;
    R[k] = R[k] - cmul(to_f(al), V[k]);
  }
  if (i == 0) st[p].alpha = al;
}

// omega = <t, s> / <t, t>;  x += alpha p + omega s;  r = s - omega t
__global__ void k_bi_x(float2* __restrict__ X, float2* __restrict__ R, const float2* __restrict__ P,
                       const float2* __restrict__ T, BiState* st, const double2* __restrict__ ts,
                       const double* __restrict__ tt, int M) {
  const int p = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double2 om = make_double2(ts[p].x / tt[p], ts[p].y / tt[p]);
  if (i < M) {
    const size_t k = (size_t)p * M + i;
    const float2 s = R[k];
    X[k] = X[k] + cmul(to_f(st[p].alpha), P[k]) + cmul(to_f(om), s);
    R[k] = s - cmul(to_f(om), T[k]);
  }
  if (i == 0) st[p].omega = om;
}

pdf_status sv_forward(pdf_problem* h, const float2* chi, float2* esca_out, float2* j_out, double tol,
                      int max_iter, int* iters_out, cudaStream_t st) {
  Dev& d = h->d;
  const int M = d.M;
  const size_t NF = (size_t)d.ni * M;
  const unsigned nbf = (unsigned)((NF + 255) / 256);
  const dim3 gp((M + 255) / 256, d.ni);
  // buffers: X = tmpA, R = tmpB, P = tmpC, V = d.v, T = d.gsh, RHAT = d.s (einc copy), tmp = d.r
  float2 *X = h->tmpA, *R = h->tmpB, *P = h->tmpC, *V = d.v, *T = d.gsh, *RH = d.s, *TMP = d.r;
  // device state in the loss-partial buffer: 16-byte types first, then doubles
  double2* rho_new = (double2*)(void*)d.lpart;          // [ni]
  double2* rv = rho_new + d.ni;                         // [ni]
  double2* ts = rv + d.ni;                              // [ni]
  BiState* bst = (BiState*)(ts + d.ni);                 // [ni]
  double* tt = (double*)(bst + d.ni);                   // [ni]
  double* rr = tt + d.ni;                               // [ni]
  double* bb = rr + d.ni;                               // [ni]
  if ((size_t)15 * d.ni > (size_t)LP_NSLOT * PDF_LP_STRIDE)
    return set_err(PDF_EUNSUPPORTED, "too many incidences for the forward solver state");
  pdf_status s;
  auto apply_A = [&](const float2* x, float2* y) -> pdf_status {
    k_mul_chi<<<nbf, 256, 0, st>>>(chi, x, TMP, M, NF);
    pdf_count_launch(1);
    pdf_status q = hp_gd(h, TMP, y, 0, st);
    if (q != PDF_OK) return q;
    k_xmy<<<nbf, 256, 0, st>>>(x, y, NF);
    pdf_count_launch(1);
    return PDF_OK;
  };
  // x0 = E_inc, r0 = b - A x0, rhat = r0
  PDF_CUDA(cudaMemcpyAsync(X, d.einc, NF * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  if ((s = apply_A(X, V)) != PDF_OK) return s;
  // R = E_inc - V
  PDF_CUDA(cudaMemcpyAsync(R, d.einc, NF * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  k_xmy<<<nbf, 256, 0, st>>>(R, V, NF);   // V = R - V  -> r0 in V
  PDF_CUDA(cudaMemcpyAsync(R, V, NF * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  PDF_CUDA(cudaMemcpyAsync(RH, R, NF * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  PDF_CUDA(cudaMemsetAsync(V, 0, NF * sizeof(float2), st));
  k_sumsq_per_p<<<d.ni, 256, 0, st>>>(d.einc, M, bb);
  pdf_count_launch(2);
  std::vector<double> hr(d.ni), hb(d.ni);
  PDF_CUDA(cudaMemcpyAsync(hb.data(), bb, d.ni * sizeof(double), cudaMemcpyDeviceToHost, st));
  int it = 0;
  bool conv = false;
  for (; it < max_iter; ++it) {
    k_dot_per_p<<<d.ni, 256, 0, st>>>(RH, R, M, rho_new);
    k_bi_p<<<gp, 256, 0, st>>>(P, R, V, bst, rho_new, M, it == 0);
    k_bi_rho_commit<<<(d.ni + 127) / 128, 128, 0, st>>>(bst, rho_new, d.ni);
    pdf_count_launch(3);
    if ((s = apply_A(P, V)) != PDF_OK) return s;
    k_dot_per_p<<<d.ni, 256, 0, st>>>(RH, V, M, rv);
    k_bi_s<<<gp, 256, 0, st>>>(R, V, bst, rv, M);
    pdf_count_launch(2);
    if ((s = apply_A(R, T)) != PDF_OK) return s;
    k_dot_per_p<<<d.ni, 256, 0, st>>>(T, R, M, ts);
    k_sumsq_per_p<<<d.ni, 256, 0, st>>>(T, M, tt);
    k_bi_x<<<gp, 256, 0, st>>>(X, R, P, T, bst, ts, tt, M);
    pdf_count_launch(3);
    PDF_LAUNCHED("BiCGSTAB");
    if ((it + 1) % 5 == 0 || it + 1 == max_iter) {
      k_sumsq_per_p<<<d.ni, 256, 0, st>>>(R, M, rr);
      pdf_count_launch(1);
      PDF_CUDA(cudaMemcpyAsync(hr.data(), rr, d.ni * sizeof(double), cudaMemcpyDeviceToHost, st));
      PDF_CUDA(cudaStreamSynchronize(st));
      double worst = 0.0;
      for (int p = 0; p < d.ni; ++p) worst = std::max(worst, sqrt(hr[p] / hb[p]));
      if (!std::isfinite(worst)) return set_err(PDF_ENONFINITE, "forward solve diverged");
      if (worst < tol) {
        conv = true;
        ++it;
        break;
      }
    }
  }
  if (iters_out) *iters_out = it;
  // J = chi E_tot, E_sca = G_S J
  k_mul_chi<<<nbf, 256, 0, st>>>(chi, X, TMP, M, NF);
  pdf_count_launch(1);
  if (j_out) PDF_CUDA(cudaMemcpyAsync(j_out, TMP, NF * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  if ((s = hp_gs(h, TMP, esca_out, nullptr, nullptr, st)) != PDF_OK) return s;
  PDF_CUDA(cudaStreamSynchronize(st));
  if (!conv) return set_err(PDF_ETIMEOUT, "forward solve reached max_iter before tol");
  return PDF_OK;
}
