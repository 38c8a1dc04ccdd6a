// Learned warm start: a fully connected network (BF16 operands, FP32 master weights) mapping
// the normalised measured field to initial Fourier coefficients, trained and evaluated by this
// library's kernels.  Not part of the paper's method (its FCNN is untrained and re-fitted per
// scene); it supplies alpha_(0) for the solve, with the paper's BP + CSI start as fallback.
//
// Layer l: z_l = W_l a_{l-1} + b_l, a_l = ReLU(z_l) for hidden layers, linear output.
// All matrix products run on the tcgen05 GEMM (umma.cu) with BF16 operands and FP32
// accumulation; K-major operand copies (W and W^T, activations and their transposes) are
// written by the element-wise kernels that produce them.  Loss: mean squared error over the
// batch and outputs.  Optimiser: Adam on the FP32 master weights (torch.optim.Adam arithmetic).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "problem.cuh"
#include "umma.cuh"

#define MLP_MAX_LAYERS 8

static int r64(int k) { return (k + 63) / 64 * 64; }

struct MlpLayer {
  int in, out, inp, outp;           // sizes and 64-padded sizes
  float *W, *mW, *vW, *b, *mb, *vb; // FP32 master [out][in], [out]
  float *dW, *db;                   // gradients
  __nv_bfloat16 *Wb, *WbT;          // [out][inp], [in][outp]
  __nv_bfloat16 *Xb, *XbT;          // input activations [B][inp], [in][Bp]
  __nv_bfloat16 *dYb, *dYbT;        // output cotangent [B][outp], [out][Bp]
  float* Z;                         // pre-activation / output [B][out]
  float* dX;                        // [B][in]
  UmmaOperand oWb, oWbT, oXb, oXbT, odYb, odYbT;
};

struct pdf_mlp {
  int nl, bmax, bp;
  MlpLayer L[MLP_MAX_LAYERS];
  std::vector<void*> allocs;
  double* loss;                     // [8] device
  double* parts;                    // loss partial sums [ceil(bmax * out_last / 256)]
  int* err;
  int step;
};

static pdf_status malloc_track(pdf_mlp* m, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 256);
  if (e != cudaSuccess) return cuda_err(e, "cudaMalloc(mlp)");
  m->allocs.push_back(*p);
  return cudaMemset(*p, 0, bytes ? bytes : 256) == cudaSuccess ? PDF_OK : set_err(PDF_ECUDA, "memset(mlp)");
}

static void mlp_free(pdf_mlp* m) {
  if (!m) return;
  for (void* p : m->allocs) cudaFree(p);
  delete m;
}

__device__ __forceinline__ __nv_bfloat16 bf(float x) { return __float2bfloat16_rn(x); }

// BF16 copies of W in both orientations: Wb[o][i] and WbT[i][o]
__global__ void k_mlp_wcast(const float* __restrict__ W, __nv_bfloat16* Wb, __nv_bfloat16* WbT, int out, int in,
                            int inp, int outp) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (size_t)out * in) return;
  const int o = (int)(k / in), i = (int)(k - (size_t)o * in);
  const __nv_bfloat16 v = bf(W[k]);
  Wb[(size_t)o * inp + i] = v;
  WbT[(size_t)i * outp + o] = v;
}

// network input: X fp32 [B][in] -> Xb [B][inp], XbT [in][Bp]
__global__ void k_mlp_xcast(const float* __restrict__ X, __nv_bfloat16* Xb, __nv_bfloat16* XbT, int B, int in, int inp,
                            int bp) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (size_t)B * in) return;
  const int r = (int)(k / in), i = (int)(k - (size_t)r * in);
  const __nv_bfloat16 v = bf(X[k]);
  Xb[(size_t)r * inp + i] = v;
  XbT[(size_t)i * bp + r] = v;
}

// hidden epilogue: z = C + b, a = ReLU(z) -> next layer's Xb / XbT; keeps z in place of C
__global__ void k_mlp_bias_relu(float* __restrict__ Z, const float* __restrict__ b, __nv_bfloat16* Xn,
                                __nv_bfloat16* XnT, int B, int out, int outp, int bp) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (size_t)B * out) return;
  const int r = (int)(k / out), o = (int)(k - (size_t)r * out);
  const float z = Z[k] + b[o];
  Z[k] = z;
  const __nv_bfloat16 a = bf(fmaxf(z, 0.f));
  Xn[(size_t)r * outp + o] = a;
  XnT[(size_t)o * bp + r] = a;
}

// output epilogue: y = C + b (in place), optionally copied to `yout`
__global__ void k_mlp_bias_out(float* __restrict__ Z, const float* __restrict__ b, float* yout, int B, int out) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (size_t)B * out) return;
  const float y = Z[k] + b[k % out];
  Z[k] = y;
  if (yout) yout[k] = y;
}

// MSE: dY = 2 (y - t) / (B out) -> dYb / dYbT (bf16) and into Z (fp32, reused for db); loss partials
__global__ void k_mlp_mse(float* __restrict__ Z, const float* __restrict__ T, __nv_bfloat16* dYb,
                          __nv_bfloat16* dYbT, int B, int out, int outp, int bp, double* part) {
  __shared__ double red[32];
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (k < (size_t)B * out) {
    const int r = (int)(k / out), o = (int)(k - (size_t)r * out);
    const float e = Z[k] - T[k];
    l = (double)e * e;
    const float g = 2.f * e / (float)((double)B * out);
    Z[k] = g;
    const __nv_bfloat16 gb = bf(g);
    dYb[(size_t)r * outp + o] = gb;
    dYbT[(size_t)o * bp + r] = gb;
  }
  const double t = block_sum(l, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// hidden cotangent: dz = dX * 1[z > 0] -> dYb / dYbT of that layer, and into Z (fp32)
__global__ void k_mlp_drelu(const float* __restrict__ dX, float* __restrict__ Z, __nv_bfloat16* dYb,
                            __nv_bfloat16* dYbT, int B, int out, int outp, int bp) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (size_t)B * out) return;
  const int r = (int)(k / out), o = (int)(k - (size_t)r * out);
  const float g = Z[k] > 0.f ? dX[k] : 0.f;
  Z[k] = g;
  const __nv_bfloat16 gb = bf(g);
  dYb[(size_t)r * outp + o] = gb;
  dYbT[(size_t)o * bp + r] = gb;
}

// db[o] = sum_r dz[r][o]  (fp32 cotangent kept in Z)
__global__ void k_mlp_db(const float* __restrict__ G, float* __restrict__ db, int B, int out) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= out) return;
  float s = 0.f;
  for (int r = 0; r < B; ++r) s += G[(size_t)r * out + o];
  db[o] = s;
}

__global__ void k_mlp_sum(const double* in, int n, double* out, double scale) {
  __shared__ double red[32];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += in[i];
  const double t = block_sum(a, red);
  if (threadIdx.x == 0) *out = t * scale;
}

// Adam (torch.optim.Adam arithmetic) on an FP32 array
__global__ void k_mlp_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps, float step_size,
                           float bc2s) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  float mi = m[i];
  mi = mi + (1.f - b1) * (gi - mi);
  float vi = v[i] * b2;
  vi = vi + ((1.f - b2) * gi) * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] = p[i] + (-step_size) * (mi / (sqrtf(vi) / bc2s + eps));
}

static unsigned nb(size_t n) { return (unsigned)((n + 255) / 256); }

extern "C" pdf_status pdf_mlp_create(int32_t nlayers, const int32_t* sizes, int32_t batch_max, pdf_mlp** out) {
  if (!out || !sizes) return set_err(PDF_EINVAL, "pdf_mlp_create: NULL argument");
  *out = nullptr;
  if (nlayers < 1 || nlayers > MLP_MAX_LAYERS) return set_err(PDF_EINVAL, "pdf_mlp_create: 1..8 layers");
  if (batch_max < 1 || batch_max > 4096) return set_err(PDF_EINVAL, "pdf_mlp_create: batch in [1, 4096]");
  for (int l = 0; l <= nlayers; ++l) {
    if (sizes[l] < 1 || sizes[l] > (1 << 20)) return set_err(PDF_EINVAL, "pdf_mlp_create: layer sizes in [1, 2^20]");
    if ((size_t)batch_max * sizes[l] >= ((size_t)1 << 31) ||
        (l < nlayers && (size_t)sizes[l] * sizes[l + 1] >= ((size_t)1 << 31)))
      return set_err(PDF_EINVAL, "pdf_mlp_create: a weight matrix or activation exceeds 2^31 elements");
  }
  pdf_mlp* m = new pdf_mlp();
  m->nl = nlayers;
  m->bmax = batch_max;
  m->bp = r64(batch_max);
  m->step = 0;
  pdf_status s;
#define MA(ptr, bytes)                                                  \
  do {                                                                  \
    if ((s = malloc_track(m, (void**)&(ptr), (bytes))) != PDF_OK) {     \
      mlp_free(m);                                                      \
      return s;                                                         \
    }                                                                   \
  } while (0)
  MA(m->loss, sizeof(double) * 8);
  MA(m->err, sizeof(int));
  MA(m->parts, sizeof(double) * (((size_t)batch_max * sizes[nlayers] + 255) / 256));
  for (int l = 0; l < nlayers; ++l) {
    MlpLayer& L = m->L[l];
    L.in = sizes[l];
    L.out = sizes[l + 1];
    L.inp = r64(L.in);
    L.outp = r64(L.out);
    const size_t nw = (size_t)L.in * L.out;
    MA(L.W, nw * 4);
    MA(L.mW, nw * 4);
    MA(L.vW, nw * 4);
    MA(L.dW, nw * 4);
    MA(L.b, L.out * 4);
    MA(L.mb, L.out * 4);
    MA(L.vb, L.out * 4);
    MA(L.db, L.out * 4);
    MA(L.Wb, (size_t)L.out * L.inp * 2);
    MA(L.WbT, (size_t)L.in * L.outp * 2);
    MA(L.Xb, (size_t)batch_max * L.inp * 2);
    MA(L.XbT, (size_t)L.in * m->bp * 2);
    MA(L.dYb, (size_t)batch_max * L.outp * 2);
    MA(L.dYbT, (size_t)L.out * m->bp * 2);
    MA(L.Z, (size_t)batch_max * L.out * 4);
    MA(L.dX, (size_t)batch_max * L.in * 4);
  }
#undef MA
  *out = m;
  return PDF_OK;
}

extern "C" void pdf_mlp_destroy(pdf_mlp* m) {
  if (!m) return;
  cudaDeviceSynchronize();
  mlp_free(m);
}

// Operand tensor maps depend on the batch size (rows of activations): encoded per call.
static pdf_status encode_layer(pdf_mlp* m, MlpLayer& L, int B) {
  pdf_status s;
  if ((s = umma_operand(&L.oWb, L.Wb, nullptr, L.out, L.inp)) != PDF_OK) return s;
  if ((s = umma_operand(&L.oWbT, L.WbT, nullptr, L.in, L.outp)) != PDF_OK) return s;
  if ((s = umma_operand(&L.oXb, L.Xb, nullptr, B, L.inp)) != PDF_OK) return s;
  if ((s = umma_operand(&L.oXbT, L.XbT, nullptr, L.in, m->bp)) != PDF_OK) return s;
  if ((s = umma_operand(&L.odYb, L.dYb, nullptr, B, L.outp)) != PDF_OK) return s;
  if ((s = umma_operand(&L.odYbT, L.dYbT, nullptr, L.out, m->bp)) != PDF_OK) return s;
  return PDF_OK;
}

extern "C" pdf_status pdf_mlp_set_params(pdf_mlp* m, int32_t layer, const float* W, const float* b, void* stream) {
  if (!m || !W || !b || layer < 0 || layer >= m->nl) return set_err(PDF_EINVAL, "pdf_mlp_set_params: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  MlpLayer& L = m->L[layer];
  PDF_CUDA(cudaMemcpyAsync(L.W, W, sizeof(float) * L.in * L.out, cudaMemcpyHostToDevice, s));
  PDF_CUDA(cudaMemcpyAsync(L.b, b, sizeof(float) * L.out, cudaMemcpyHostToDevice, s));
  PDF_CUDA(cudaMemsetAsync(L.mW, 0, sizeof(float) * L.in * L.out, s));
  PDF_CUDA(cudaMemsetAsync(L.vW, 0, sizeof(float) * L.in * L.out, s));
  PDF_CUDA(cudaMemsetAsync(L.mb, 0, sizeof(float) * L.out, s));
  PDF_CUDA(cudaMemsetAsync(L.vb, 0, sizeof(float) * L.out, s));
  k_mlp_wcast<<<nb((size_t)L.in * L.out), 256, 0, s>>>(L.W, L.Wb, L.WbT, L.out, L.in, L.inp, L.outp);
  pdf_count_launch(1);
  m->step = 0;
  PDF_CUDA(cudaStreamSynchronize(s));
  return PDF_OK;
}

extern "C" pdf_status pdf_mlp_get_params(pdf_mlp* m, int32_t layer, float* W, float* b, float* dW, float* db,
                                         void* stream) {
  if (!m || layer < 0 || layer >= m->nl) return set_err(PDF_EINVAL, "pdf_mlp_get_params: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  MlpLayer& L = m->L[layer];
  if (W) PDF_CUDA(cudaMemcpyAsync(W, L.W, sizeof(float) * L.in * L.out, cudaMemcpyDeviceToHost, s));
  if (b) PDF_CUDA(cudaMemcpyAsync(b, L.b, sizeof(float) * L.out, cudaMemcpyDeviceToHost, s));
  if (dW) PDF_CUDA(cudaMemcpyAsync(dW, L.dW, sizeof(float) * L.in * L.out, cudaMemcpyDeviceToHost, s));
  if (db) PDF_CUDA(cudaMemcpyAsync(db, L.db, sizeof(float) * L.out, cudaMemcpyDeviceToHost, s));
  PDF_CUDA(cudaStreamSynchronize(s));
  return PDF_OK;
}

// Columns [B, Bp) of the transposed activation/cotangent copies are the padded K range of the
// weight-gradient GEMM: keep them zero when B is below the padded batch.
static pdf_status clear_batch_pad(pdf_mlp* m, int B, cudaStream_t s) {
  if (B == m->bp) return PDF_OK;
  for (int l = 0; l < m->nl; ++l) {
    MlpLayer& L = m->L[l];
    PDF_CUDA(cudaMemset2DAsync(L.XbT + B, (size_t)m->bp * 2, 0, (size_t)(m->bp - B) * 2, L.in, s));
    PDF_CUDA(cudaMemset2DAsync(L.dYbT + B, (size_t)m->bp * 2, 0, (size_t)(m->bp - B) * 2, L.out, s));
  }
  return PDF_OK;
}

static pdf_status forward(pdf_mlp* m, const float* X, int B, float* Y, cudaStream_t s) {
  pdf_status st;
  if ((st = clear_batch_pad(m, B, s)) != PDF_OK) return st;
  MlpLayer& L0 = m->L[0];
  k_mlp_xcast<<<nb((size_t)B * L0.in), 256, 0, s>>>(X, L0.Xb, L0.XbT, B, L0.in, L0.inp, m->bp);
  pdf_count_launch(1);
  for (int l = 0; l < m->nl; ++l) {
    MlpLayer& L = m->L[l];
    if ((st = encode_layer(m, L, B)) != PDF_OK) return st;
    if ((st = umma_gemm(L.oXb, L.oWb, 0, 1, L.Z, L.out, 0, m->err, s)) != PDF_OK) return st;
    if (l + 1 < m->nl) {
      MlpLayer& N = m->L[l + 1];
      k_mlp_bias_relu<<<nb((size_t)B * L.out), 256, 0, s>>>(L.Z, L.b, N.Xb, N.XbT, B, L.out, N.inp, m->bp);
    } else {
      k_mlp_bias_out<<<nb((size_t)B * L.out), 256, 0, s>>>(L.Z, L.b, Y, B, L.out);
    }
    pdf_count_launch(1);
  }
  PDF_LAUNCHED("mlp forward");
  return PDF_OK;
}

extern "C" pdf_status pdf_mlp_forward(pdf_mlp* m, const float* X, float* Y, int32_t B, void* stream) {
  if (!m || !X || !Y || B < 1 || B > m->bmax) return set_err(PDF_EINVAL, "pdf_mlp_forward: bad arguments");
  return forward(m, X, B, Y, (cudaStream_t)stream);
}

// Gradients of the mean squared error 1/(B out) sum (y - t)^2 into the layers' dW, db; *loss
// (device double, may be NULL) receives the loss value.
static pdf_status loss_grad(pdf_mlp* m, const float* X, const float* T, int B, double* loss, cudaStream_t s) {
  pdf_status st = forward(m, X, B, nullptr, s);
  if (st != PDF_OK) return st;
  MlpLayer& Lz = m->L[m->nl - 1];
  const size_t n = (size_t)B * Lz.out;
  double* parts = m->parts;
  k_mlp_mse<<<nb(n), 256, 0, s>>>(Lz.Z, T, Lz.dYb, Lz.dYbT, B, Lz.out, Lz.outp, m->bp, parts);
  k_mlp_sum<<<1, 256, 0, s>>>(parts, (int)nb(n), loss ? loss : m->loss, 1.0 / (double)n);
  pdf_count_launch(2);
  for (int l = m->nl - 1; l >= 0; --l) {
    MlpLayer& L = m->L[l];
    // dW[out][in] = dY^T X  (A = dYbT [out][Bp], B = XbT [in][Bp])
    if ((st = umma_gemm(L.odYbT, L.oXbT, 0, 1, L.dW, L.in, 0, m->err, s)) != PDF_OK) return st;
    k_mlp_db<<<nb(L.out), 256, 0, s>>>(L.Z, L.db, B, L.out);
    pdf_count_launch(1);
    if (l > 0) {
      // dX[B][in] = dY W  (A = dYb [B][outp], B = WbT [in][outp])
      if ((st = umma_gemm(L.odYb, L.oWbT, 0, 1, L.dX, L.in, 0, m->err, s)) != PDF_OK) return st;
      MlpLayer& P = m->L[l - 1];
      k_mlp_drelu<<<nb((size_t)B * P.out), 256, 0, s>>>(L.dX, P.Z, P.dYb, P.dYbT, B, P.out, P.outp, m->bp);
      pdf_count_launch(1);
    }
  }
  PDF_LAUNCHED("mlp backward");
  return PDF_OK;
}

extern "C" pdf_status pdf_mlp_loss_grad(pdf_mlp* m, const float* X, const float* T, int32_t B, double* loss,
                                        void* stream) {
  if (!m || !X || !T || B < 1 || B > m->bmax) return set_err(PDF_EINVAL, "pdf_mlp_loss_grad: bad arguments");
  return loss_grad(m, X, T, B, loss, (cudaStream_t)stream);
}

extern "C" pdf_status pdf_mlp_train_step(pdf_mlp* m, const float* X, const float* T, int32_t B, double lr,
                                         double* loss, void* stream) {
  if (!m || !X || !T || B < 1 || B > m->bmax || !(lr >= 0)) return set_err(PDF_EINVAL, "pdf_mlp_train_step: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  pdf_status st = loss_grad(m, X, T, B, loss, s);
  if (st != PDF_OK) return st;
  m->step += 1;
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  const double bc1 = 1.0 - pow(b1, m->step), bc2 = 1.0 - pow(b2, m->step);
  const float step_size = (float)(lr / bc1), bc2s = (float)sqrt(bc2);
  for (int l = 0; l < m->nl; ++l) {
    MlpLayer& L = m->L[l];
    const size_t nw = (size_t)L.in * L.out;
    k_mlp_adam<<<nb(nw), 256, 0, s>>>(L.W, L.dW, L.mW, L.vW, nw, (float)lr, (float)b1, (float)b2, (float)eps,
                                      step_size, bc2s);
    k_mlp_adam<<<nb(L.out), 256, 0, s>>>(L.b, L.db, L.mb, L.vb, L.out, (float)lr, (float)b1, (float)b2, (float)eps,
                                         step_size, bc2s);
    k_mlp_wcast<<<nb(nw), 256, 0, s>>>(L.W, L.Wb, L.WbT, L.out, L.in, L.inp, L.outp);
    pdf_count_launch(3);
  }
  PDF_LAUNCHED("mlp Adam");
  return PDF_OK;
}

extern "C" int32_t pdf_mlp_error_flag(pdf_mlp* m) {
  if (!m) return -1;
  int v = 0;
  cudaMemcpy(&v, m->err, sizeof(int), cudaMemcpyDeviceToHost);
  return v;
}

// Warm-start network input: X[b][2 i + c] = (Re, Im) of E[b][i] / (||E[b]|| / sqrt(n)), one CTA per
// scene (FP32 Kahan partial sums per thread, FP64 across threads).
__global__ void __launch_bounds__(256) k_mlp_features(const float2* __restrict__ E, int n, float* __restrict__ X) {
  __shared__ double red[32];
  __shared__ float inv;
  const int b = blockIdx.x;
  const float2* e = E + (size_t)b * n;
  float s = 0.f, c = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float2 v = e[i];
    const float y = (v.x * v.x + v.y * v.y) - c, t = s + y;
    c = (t - s) - y;
    s = t;
  }
  const double tot = block_sum((double)s - (double)c, red);
  if (threadIdx.x == 0) inv = tot > 0.0 ? (float)(1.0 / sqrt(tot / n)) : 1.f;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float2 v = e[i];
    X[(size_t)b * 2 * n + 2 * i] = v.x * inv;
    X[(size_t)b * 2 * n + 2 * i + 1] = v.y * inv;
  }
}

extern "C" pdf_status pdf_mlp_features(const void* esca, int32_t B, int32_t n, float* X, void* stream) {
  if (!esca || !X || B < 1 || n < 1) return set_err(PDF_EINVAL, "pdf_mlp_features: NULL pointer or size < 1");
  k_mlp_features<<<B, 256, 0, (cudaStream_t)stream>>>((const float2*)esca, n, X);
  pdf_count_launch(1);
  PDF_LAUNCHED("pdf_mlp_features");
  return PDF_OK;
}
