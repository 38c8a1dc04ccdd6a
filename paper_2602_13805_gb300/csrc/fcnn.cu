// Coefficient-correcting network of the solve (Sec. 3, network architecture; training settings).
//
// The solver's variable is the weight vector theta of a fully connected network that maps each
// incidence's initial Fourier coefficients (real and imaginary parts as two channels) to a
// correction: alpha-hat = alpha_(0) + Delta alpha(theta); Adam acts on theta.  The paper does not
// print the architecture; the form built here (also in include/pdf.h): one network for all
// incidences, input x_p = s [Re alpha_(0),p, Im alpha_(0),p] (D = 2 ky kx, s = 1 / RMS of
// alpha_(0)'s real components), two hidden layers of width H with ReLU, a linear output y_p of D
// reals, Delta alpha_p = (y_p[:ky kx] + i y_p[ky kx:]) / s.  The chain rule to theta takes the
// loss gradient g = dL/dRe alpha + i dL/dIm alpha as dL/dy_p = [Re g_p, Im g_p] / s.
//
// All products are FP32 with FP32 accumulation, on a 32 x 32 output tile per 256-thread block
// staged through shared memory; the ones with a long k and only ni <= 64 rows split k into chunks
// of 64 over blocks and add the partial sums in a fixed order (deterministic).
#include <algorithm>

#include "problem.cuh"

constexpr int FCT = 32;   // output tile side and k chunk

// The network output written straight into the coefficients: v = y[m][n] (bias added) goes to
// alpha[m][n mod k2] (real part for n < k2, imaginary part otherwise) as alpha0 + v / s, where
// C = (float*)alpha, ldc = k2, mask = (const float*)alpha0 and sc = s.
__device__ __forceinline__ void fc_store_alpha(float* alpha, const float* a0, const float* sc, int k2, int m, int n,
                                               float v) {
  const int re = n < k2 ? 0 : 1, j = n - re * k2;
  const size_t i = ((size_t)m * k2 + j) * 2 + re;
  alpha[i] = a0[i] + v / sc[0];
}

// C(m, n) = sum_k A(m, k) B(k, n) for m < M, n < N, with A(m, k) = TA ? A[k lda + m] : A[m lda + k]
// and B(k, n) = TB ? B[n ldb + k] : B[k ldb + n].  Epilogue EPI: 0 store; 1 add bias[n], ReLU;
// 2 add bias[n]; 3 multiply by (mask[m ldc + n] > 0), the ReLU derivative of a stored activation;
// 4 add bias[n] and write the coefficients (fc_store_alpha).  With gridDim.z = S > 1 block z covers
// k in [z kc, (z+1) kc) and stores its partial sums to C + z M N (row-major [M][N], no epilogue);
// k_fc_reduce adds the S partials in order.  With `tick` (S > 1) the partials go to `work` instead
// and the last block of each output tile to arrive adds them itself (see the end of the kernel), so
// no reduction launch is needed.  With `colsum` (single k split only) the blocks of the first column
// tile also write colsum[m] = sum_k A(m, k), summed in increasing k (the bias gradient of a weight
// gradient dW = dZ^T X).
template <int EPI>
__device__ __forceinline__ void fc_epilogue(float* C, int ldc, int m, int n, float v, const float* bias,
                                            const float* mask, const float* sc) {
  if (EPI == 1) v = fmaxf(v + bias[n], 0.f);
  if (EPI == 2 || EPI == 4) v = v + bias[n];
  if (EPI == 3) v = mask[(size_t)m * ldc + n] > 0.f ? v : 0.f;
  if (EPI == 4) fc_store_alpha(C, mask, sc, ldc, m, n, v);
  else C[(size_t)m * ldc + n] = v;
}

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256) k_fc_gemm(const float* __restrict__ A, int lda, const float* __restrict__ B,
                                                 int ldb, float* __restrict__ C, int ldc, int M, int N, int K,
                                                 int kc, const float* __restrict__ bias, const float* __restrict__ mask,
                                                 const float* __restrict__ sc, float* __restrict__ colsum,
                                                 float* __restrict__ work, unsigned* __restrict__ tick) {
  pdl_wait();
  __shared__ float As[FCT][FCT + 1];   // [m][k]
  __shared__ float Bs[FCT][FCT + 1];   // [k][n]
  __shared__ int last;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * FCT, n0 = blockIdx.x * FCT;
  const int kb = blockIdx.z * kc, ke = min(K, kb + kc);
  const bool partial = gridDim.z > 1;
  const bool csum = colsum && !partial && blockIdx.x == 0 && tx == 0;
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  float cs0 = 0.f, cs1 = 0.f;
  for (int k0 = kb; k0 < ke; k0 += FCT) {
    for (int e = threadIdx.x; e < FCT * FCT; e += blockDim.x) {
      const int a = e / FCT, b = e - a * FCT;                            // b runs along the contiguous index
      if (TA) {
        const int m = m0 + b, k = k0 + a;
        As[b][a] = (m < M && k < ke) ? A[(size_t)k * lda + m] : 0.f;
      } else {
        const int m = m0 + a, k = k0 + b;
        As[a][b] = (m < M && k < ke) ? A[(size_t)m * lda + k] : 0.f;
      }
      if (TB) {
        const int k = k0 + b, n = n0 + a;
        Bs[b][a] = (k < ke && n < N) ? B[(size_t)n * ldb + k] : 0.f;
      } else {
        const int k = k0 + a, n = n0 + b;
        Bs[a][b] = (k < ke && n < N) ? B[(size_t)k * ldb + n] : 0.f;
      }
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < FCT; ++kk) {
      const float a0 = As[ty][kk], a1 = As[ty + 16][kk];
      const float b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      acc[0][0] = fmaf(a0, b0, acc[0][0]);
      acc[0][1] = fmaf(a0, b1, acc[0][1]);
      acc[1][0] = fmaf(a1, b0, acc[1][0]);
      acc[1][1] = fmaf(a1, b1, acc[1][1]);
    }
    if (csum)
      for (int kk = 0; kk < FCT && k0 + kk < ke; ++kk) {
        cs0 += As[ty][kk];
        cs1 += As[ty + 16][kk];
      }
    __syncthreads();
  }
  if (csum) {
    if (m0 + ty < M) colsum[m0 + ty] = cs0;
    if (m0 + ty + 16 < M) colsum[m0 + ty + 16] = cs1;
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m >= M || n >= N) continue;
      const float v = acc[i][j];
      if (partial) {
        (tick ? work : C)[((size_t)blockIdx.z * M + m) * N + n] = v;
        continue;
      }
      fc_epilogue<EPI>(C, ldc, m, n, v, bias, mask, sc);
    }
  if (!partial || !tick) return;
  // the last block of this output tile to arrive adds the S partials in increasing z (the order of
  // k_fc_reduce), applies the epilogue and re-arms the counter for the next product
  __threadfence();
  __syncthreads();
  const unsigned t = blockIdx.y * gridDim.x + blockIdx.x;
  if (threadIdx.x == 0) last = atomicAdd(&tick[t], 1u) == gridDim.z - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the four outputs of this thread summed together, z unrolled, so many loads are in flight;
  // each output still adds its partials in increasing z
  float v[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  int mi[2], nj[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    mi[i] = min(m0 + ty + 16 * i, M - 1);
    nj[i] = min(n0 + tx + 16 * i, N - 1);
  }
  const int S = gridDim.z;
#pragma unroll 6
  for (int z = 0; z < S; ++z)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) v[i][j] += __ldcg(&work[((size_t)z * M + mi[i]) * N + nj[j]]);
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m < M && n < N) fc_epilogue<EPI>(C, ldc, m, n, v[i][j], bias, mask, sc);
    }
  if (threadIdx.x == 0) tick[t] = 0u;
}

// C[m][n] = epilogue(sum over z (increasing) of part[z][m][n]) for the split-k form
template <int EPI>
__global__ void k_fc_reduce(const float* __restrict__ part, int S, float* __restrict__ C, int ldc, int M, int N,
                            const float* __restrict__ bias, const float* __restrict__ mask,
                            const float* __restrict__ sc) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * N) return;
  const int m = i / N, n = i - m * N;
  float v = 0.f;
  for (int z = 0; z < S; ++z) v += part[(size_t)z * M * N + i];
  fc_epilogue<EPI>(C, ldc, m, n, v, bias, mask, sc);
}

// out[c] = sum over r (increasing) of A[r cols + c]: bias gradients
__global__ void k_fc_colsum(const float* __restrict__ A, int rows, int cols, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += A[(size_t)r * cols + c];
  out[c] = s;
}

// X = s [Re alpha0, Im alpha0] per incidence, s = 1 / RMS of the real components (one block)
__global__ void k_fc_input(const float2* __restrict__ a0, int ni, int k2, float* __restrict__ X,
                           float* __restrict__ s_out) {
  __shared__ double red[32];
  __shared__ float s_sh;
  double acc = 0.0;
  const int n = ni * k2;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float2 v = a0[i];
    acc += (double)v.x * v.x + (double)v.y * v.y;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) tot += red[w];
    const double ms = tot / (2.0 * n);
    s_sh = ms > 0.0 ? (float)(1.0 / sqrt(ms)) : 1.f;                   // all-zero start: unscaled
    s_out[0] = s_sh;
  }
  __syncthreads();
  const float s = s_sh;
  const int D = 2 * k2;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int b = i / k2, j = i - b * k2;
    const float2 v = a0[i];
    X[(size_t)b * D + j] = s * v.x;
    X[(size_t)b * D + k2 + j] = s * v.y;
  }
}

// dL/dy = [Re g, Im g] / s
__global__ void k_fc_dy(const float2* __restrict__ g, const float* __restrict__ s, int ni, int k2,
                        float* __restrict__ dY) {
  pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ni * k2) return;
  const int b = i / k2, j = i - b * k2, D = 2 * k2;
  const float sc = s[0];
  const float2 v = g[i];
  dY[(size_t)b * D + j] = v.x / sc;
  dY[(size_t)b * D + k2 + j] = v.y / sc;
}

// k chunk per split (two 32-wide steps): the batch is small, so a long k runs as many blocks of two
// steps each instead of one block walking k with a round trip to L2 per step
constexpr int FC_KC = 2 * FCT;
constexpr int FC_TICKS = 4096;       // output tiles of a split-k product reduced by their last block
constexpr int FC_SMAX = 32;
static int fc_splits(int K) { return std::min(FC_SMAX, (K + FC_KC - 1) / FC_KC); }

// returns the number of kernels launched; `colsum` (TA products with lda = M): also the sums over
// k of A(m, k)
template <bool TA, bool TB, int EPI>
static int gemm(const float* A, int lda, const float* B, int ldb, float* C, int ldc, int M, int N, int K,
                const float* bias, const float* mask, float* work, cudaStream_t st, const float* sc = nullptr,
                float* colsum = nullptr, unsigned* tick = nullptr) {
  const int S = fc_splits(K), kc = (K + S - 1) / S;
  const dim3 grid((N + FCT - 1) / FCT, (M + FCT - 1) / FCT, S);
  if (S == 1) {
    launch_pdl(k_fc_gemm<TA, TB, EPI>, grid, 256, 0, st, A, lda, B, ldb, C, ldc, M, N, K, K, bias, mask, sc, colsum,
               (float*)nullptr, (unsigned*)nullptr);
    return 1;
  }
  // reduction by the last block where the splits are few (with many, the separate reduction's
  // M N threads add them faster than the blocks of one tile)
  if (tick && !colsum && S <= 8 && grid.x * grid.y <= FC_TICKS) {
    launch_pdl(k_fc_gemm<TA, TB, EPI>, grid, 256, 0, st, A, lda, B, ldb, C, ldc, M, N, K, kc, bias, mask, sc,
               (float*)nullptr, work, tick);
    return 1;
  }
  launch_pdl(k_fc_gemm<TA, TB, EPI>, grid, 256, 0, st, A, lda, B, ldb, work, N, M, N, K, kc, (const float*)nullptr,
             (const float*)nullptr, (const float*)nullptr, (float*)nullptr, (float*)nullptr, (unsigned*)nullptr);
  launch_pdl(k_fc_reduce<EPI>, (M * N + 255) / 256, 256, 0, st, (const float*)work, S, C, ldc, M, N, bias, mask, sc);
  int n = 2;
  if (colsum) {                                                          // A(m, k) = A[k lda + m] here
    k_fc_colsum<<<(M + 255) / 256, 256, 0, st>>>(A, K, M, colsum);
    ++n;
  }
  return n;
}

// parameter offsets in the flat vector
struct FcOff {
  size_t W1, b1, W2, b2, W3, b3;
};
static FcOff fc_off(int D, int H) {
  FcOff o;
  o.W1 = 0;
  o.b1 = (size_t)H * D;
  o.W2 = o.b1 + H;
  o.b2 = o.W2 + (size_t)H * H;
  o.W3 = o.b2 + H;
  o.b3 = o.W3 + (size_t)D * H;
  return o;
}

pdf_status fc_prepare(pdf_problem* h, int hidden, const void* params0, cudaStream_t st) {
  FcState& f = h->fc;
  const Dev& d = h->d;
  const int D = 2 * d.ky * d.kx, B = d.ni, H = hidden;
  const size_t np = (size_t)H * D + H + (size_t)H * H + H + (size_t)D * H + D;
  if (f.H != H || f.D != D || f.B != B) {                              // (re)allocate; old blocks stay owned
    pdf_status s;
    void** bufs[] = {(void**)&f.theta, (void**)&f.gtheta, (void**)&f.m, (void**)&f.v};
    for (void** b : bufs)
      if ((s = ws_alloc(h, b, sizeof(float) * np)) != PDF_OK) return s;
    if ((s = ws_alloc(h, (void**)&f.X, sizeof(float) * B * D)) != PDF_OK) return s;
    if ((s = ws_alloc(h, (void**)&f.y, sizeof(float) * B * D)) != PDF_OK) return s;
    if ((s = ws_alloc(h, (void**)&f.s, sizeof(float))) != PDF_OK) return s;
    float** hb[] = {&f.h1, &f.h2, &f.dz1, &f.dz2};
    for (float** b : hb)
      if ((s = ws_alloc(h, (void**)b, sizeof(float) * B * H)) != PDF_OK) return s;
    if ((s = ws_alloc(h, (void**)&f.alpha0, sizeof(float2) * d.ni * d.ky * d.kx)) != PDF_OK) return s;
    // split-k partials: the products with M = B rows and a long k (D or H)
    const size_t wn = (size_t)std::max(fc_splits(D) * std::max(H, D), fc_splits(H) * std::max(H, D)) * B;
    if ((s = ws_alloc(h, (void**)&f.work, sizeof(float) * wn)) != PDF_OK) return s;
    if ((s = ws_alloc(h, (void**)&f.tick, sizeof(unsigned) * FC_TICKS)) != PDF_OK) return s;
    PDF_CUDA(cudaMemsetAsync(f.tick, 0, sizeof(unsigned) * FC_TICKS, st));
    f.nvec = nullptr;                                                    // sized by the cluster loop on use
    f.H = H;
    f.D = D;
    f.B = B;
    f.np = np;
  }
  PDF_CUDA(cudaMemcpyAsync(f.theta, params0, sizeof(float) * np, cudaMemcpyDeviceToDevice, st));
  PDF_CUDA(cudaMemsetAsync(f.m, 0, sizeof(float) * np, st));
  PDF_CUDA(cudaMemsetAsync(f.v, 0, sizeof(float) * np, st));
  PDF_CUDA(cudaMemcpyAsync(f.alpha0, h->alpha, sizeof(float2) * d.ni * d.ky * d.kx, cudaMemcpyDeviceToDevice, st));
  k_fc_input<<<1, 1024, 0, st>>>(f.alpha0, d.ni, d.ky * d.kx, f.X, f.s);
  pdf_count_launch(1);
  PDF_LAUNCHED("network input");
  return PDF_OK;
}

pdf_status fc_forward(pdf_problem* h, cudaStream_t st) {
  FcState& f = h->fc;
  const Dev& d = h->d;
  const int D = f.D, B = f.B, H = f.H, k2 = d.ky * d.kx;
  const FcOff o = fc_off(D, H);
  const float* th = f.theta;
  int n = 1;
  n += gemm<false, true, 1>(f.X, D, th + o.W1, D, f.h1, H, B, H, D, th + o.b1, nullptr, f.work, st, nullptr, nullptr,
                            f.tick);                                                                 // h1 = relu(X W1^T + b1)
  n += gemm<false, true, 1>(f.h1, H, th + o.W2, H, f.h2, H, B, H, H, th + o.b2, nullptr, f.work, st);  // h2 = relu(h1 W2^T + b2)
  // alpha = alpha0 + (y[:k2] + i y[k2:]) / s with y = h2 W3^T + b3, written by the product's epilogue
  n += gemm<false, true, 4>(f.h2, H, th + o.W3, H, reinterpret_cast<float*>(h->alpha), k2, B, D, H, th + o.b3,
                            reinterpret_cast<const float*>(f.alpha0), f.work, st, f.s);
  pdf_count_launch(n - 1);
  PDF_LAUNCHED("network forward");
  return PDF_OK;
}

pdf_status fc_backward(pdf_problem* h, cudaStream_t st) {
  FcState& f = h->fc;
  const Dev& d = h->d;
  const int D = f.D, B = f.B, H = f.H, k2 = d.ky * d.kx;
  const FcOff o = fc_off(D, H);
  const float* th = f.theta;
  float* g = f.gtheta;
  float* dY = f.y;                                                       // y is not needed any more
  launch_pdl(k_fc_dy, (B * k2 + 255) / 256, 256, 0, st, (const float2*)h->grad, (const float*)f.s, d.ni, k2, dY);
  int n = 1;
  // dW3 = dY^T h2, db3 = column sums of dY
  n += gemm<true, false, 0>(dY, D, f.h2, H, g + o.W3, H, D, H, B, nullptr, nullptr, f.work, st, nullptr, g + o.b3);
  n += gemm<false, false, 3>(dY, D, th + o.W3, H, f.dz2, H, B, H, D, nullptr, f.h2, f.work, st, nullptr, nullptr,
                             f.tick);                                                                // dz2 = (dY W3) 1[h2 > 0]
  // dW2 = dz2^T h1, db2 = column sums of dz2
  n += gemm<true, false, 0>(f.dz2, H, f.h1, H, g + o.W2, H, H, H, B, nullptr, nullptr, f.work, st, nullptr, g + o.b2);
  n += gemm<false, false, 3>(f.dz2, H, th + o.W2, H, f.dz1, H, B, H, H, nullptr, f.h1, f.work, st);   // dz1 = (dz2 W2) 1[h1 > 0]
  // dW1 = dz1^T X, db1 = column sums of dz1
  n += gemm<true, false, 0>(f.dz1, H, f.X, D, g + o.W1, D, H, D, B, nullptr, nullptr, f.work, st, nullptr, g + o.b1);
  pdf_count_launch(n);
  PDF_LAUNCHED("network backward");
  return PDF_OK;
}
