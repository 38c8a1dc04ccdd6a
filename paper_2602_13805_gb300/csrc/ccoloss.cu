// The contrast-compensated operator inside the loss (Sec. 2.4, Eq. 10-11; pdf_config.cco_in_loss):
// the regularisers of Eq. (17)-(19) act on chi_CCO = (1 + eta) G(chi|chi) + eta chi instead of on
// chi-hat, and their cotangent returns to chi-hat through the CCO's adjoint before it continues to
// R-hat and w as in the plain loss.
//
// Per real channel I (Re and Im of chi-hat are filtered separately), windows w(k) of the (2r+1)^2
// pixels around k clipped to the grid, n_k pixels each:
//   mu_k = mean over w(k) of I, var_k = mean of (I - mu_k)^2, a_k = var_k / (var_k + eps),
//   b_k = mu_k (1 - a_k),  G_i = abar_i I_i + bbar_i  (abar, bbar: means of a, b over w(i)),
//   eta_i = eta_max sigmoid((|chi_i| - tau) / delta),  chi_CCO,i = (1 + eta_i) G_i + eta_i chi_i.
// Adjoint, for the cotangent c on chi_CCO (c_G = (1 + eta) c per channel):
//   on chi directly:  abar c_G + eta c + Re(conj(c) (G + chi)) eta' chi / |chi|
//   on a_k and b_k:   c_a = sum over i in w(k) of c_G,i I_i / n_i - c_b mu_k,  c_b = sum of c_G,i / n_i
//   on var_k:         c_var = c_a eps / (var_k + eps)^2 = c_a (1 - a_k)^2 / eps
//   on I_i:           sum over k in w(i) of [c_b,k (1 - a_k) + 2 (I_i - mu_k) c_var,k] / n_k
// (w(k) holds i exactly when w(i) holds k, so every sum is a gather over the pixel's own window.)
// Five one-thread-per-pixel stencil kernels; the variance is formed in two passes (centred).
#include "phases.cuh"
#include "problem.cuh"

namespace {

struct Win {
  int y0, y1, x0, x1;
  float inv;  // 1 / count
};

__device__ __forceinline__ Win window(const Dev& d, int n) {
  const int y = n / d.nx, x = n - y * d.nx, r = d.cco_r;
  Win w;
  w.y0 = max(0, y - r);
  w.y1 = min(d.ny - 1, y + r);
  w.x0 = max(0, x - r);
  w.x1 = min(d.nx - 1, x + r);
  w.inv = 1.f / (float)((w.y1 - w.y0 + 1) * (w.x1 - w.x0 + 1));
  return w;
}

__device__ __forceinline__ float sigmoidf_(float z) { return 1.f / (1.f + expf(-z)); }

// per window k: (1 - a, mean) of Re and Im
__global__ void __launch_bounds__(256) k_cc_coef(Dev d) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= d.M) return;
  const Win w = window(d, n);
  float2 m = make_float2(0.f, 0.f);
  for (int yy = w.y0; yy <= w.y1; ++yy)
    for (int xx = w.x0; xx <= w.x1; ++xx) m = m + d.chi[yy * d.nx + xx];
  m = w.inv * m;
  float vr = 0.f, vi = 0.f;
  for (int yy = w.y0; yy <= w.y1; ++yy)
    for (int xx = w.x0; xx <= w.x1; ++xx) {
      const float2 e = d.chi[yy * d.nx + xx] - m;
      vr += e.x * e.x;
      vi += e.y * e.y;
    }
  vr *= w.inv;
  vi *= w.inv;
  d.cca[n] = make_float4(d.cco_eps / (vr + d.cco_eps), m.x, d.cco_eps / (vi + d.cco_eps), m.y);
}

// abar, bbar of pixel n (means over its window of a = 1 - (1 - a) and b = mu (1 - a)), Re and Im
__device__ __forceinline__ float4 cc_means(const Dev& d, const Win& w) {
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int yy = w.y0; yy <= w.y1; ++yy)
    for (int xx = w.x0; xx <= w.x1; ++xx) {
      const float4 q = d.cca[yy * d.nx + xx];
      s.x += 1.f - q.x;
      s.y += q.y * q.x;
      s.z += 1.f - q.z;
      s.w += q.w * q.z;
    }
  return make_float4(s.x * w.inv, s.y * w.inv, s.z * w.inv, s.w * w.inv);
}

// chi_CCO
__global__ void __launch_bounds__(256) k_cc_out(Dev d) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= d.M) return;
  const Win w = window(d, n);
  const float4 ab = cc_means(d, w);
  const float2 c = d.chi[n];
  const float2 g = make_float2(ab.x * c.x + ab.y, ab.z * c.y + ab.w);
  const float eta = d.cco_eta_max * sigmoidf_((sqrtf(cabs2(c)) - d.cco_tau) / d.cco_delta);
  d.chic[n] = (1.f + eta) * g + eta * c;
}

__global__ void __launch_bounds__(128) k_cc_reg(Dev d) { ph_reg(d, blockIdx.x, d.chic, d.ccc); }

// per pixel i: the direct part of the cotangent on chi-hat, and c_G I / n, c_G / n for the windows
__global__ void __launch_bounds__(256) k_cc_adj_pix(Dev d) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= d.M) return;
  const Win w = window(d, n);
  const float4 ab = cc_means(d, w);
  const float2 c = d.chi[n], co = d.ccc[n];
  const float2 g = make_float2(ab.x * c.x + ab.y, ab.z * c.y + ab.w);
  const float mag = sqrtf(cabs2(c));
  const float sg = sigmoidf_((mag - d.cco_tau) / d.cco_delta);
  const float eta = d.cco_eta_max * sg, deta = d.cco_eta_max * sg * (1.f - sg) / d.cco_delta;
  const float2 cg = (1.f + eta) * co;
  float2 dir = make_float2(ab.x * cg.x, ab.z * cg.y) + eta * co;
  const float ceta = co.x * (g.x + c.x) + co.y * (g.y + c.y);
  if (mag > 0.f) dir = dir + (ceta * deta / mag) * c;
  d.ccd[n] = dir;
  d.ccu[n] = make_float4(cg.x * c.x * w.inv, cg.x * w.inv, cg.y * c.y * w.inv, cg.y * w.inv);
}

// per window k: [c_b (1 - a), c_var] / n_k, Re and Im
__global__ void __launch_bounds__(256) k_cc_adj_win(Dev d) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= d.M) return;
  const Win w = window(d, n);
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int yy = w.y0; yy <= w.y1; ++yy)
    for (int xx = w.x0; xx <= w.x1; ++xx) {
      const float4 u = d.ccu[yy * d.nx + xx];
      s.x += u.x;
      s.y += u.y;
      s.z += u.z;
      s.w += u.w;
    }
  const float4 q = d.cca[n];                    // (1 - a, mu) Re, Im
  const float car = s.x - s.y * q.y, cai = s.z - s.w * q.w;
  const float cvr = car * q.x * q.x / d.cco_eps, cvi = cai * q.z * q.z / d.cco_eps;
  d.ccp[n] = make_float4(s.y * q.x * w.inv, cvr * w.inv, s.w * q.z * w.inv, cvi * w.inv);
}

// per pixel i: the cotangent on chi-hat, then on to w (the plain loss's regulariser path)
__global__ void __launch_bounds__(256) k_cc_adj_out(Dev d) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= d.M) return;
  const Win w = window(d, n);
  const float2 c = d.chi[n];
  float2 acc = d.ccd[n];
  for (int yy = w.y0; yy <= w.y1; ++yy)
    for (int xx = w.x0; xx <= w.x1; ++xx) {
      const int k = yy * d.nx + xx;
      const float4 p = d.ccp[k], q = d.cca[k];
      acc.x += p.x + 2.f * (c.x - q.y) * p.y;
      acc.y += p.z + 2.f * (c.y - q.w) * p.w;
    }
  d.w[n] = reg_w(d, n, acc);
}

}  // namespace

pdf_status cc_reg(const Dev& d, cudaStream_t st) {
  const int nb = (d.M + 255) / 256;
  k_cc_coef<<<nb, 256, 0, st>>>(d);
  k_cc_out<<<nb, 256, 0, st>>>(d);
  k_cc_reg<<<d.n_reg_blocks, 128, 0, st>>>(d);
  k_cc_adj_pix<<<nb, 256, 0, st>>>(d);
  k_cc_adj_win<<<nb, 256, 0, st>>>(d);
  k_cc_adj_out<<<nb, 256, 0, st>>>(d);
  return PDF_OK;
}
