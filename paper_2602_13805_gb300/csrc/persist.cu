// Persistent form of the Adam loop: one cooperative launch runs every iteration of a solve.
//
// Each iteration is the sequence of hot-path phases of pdf_loss_grad followed by the Adam step;
// a CTA executes the virtual blocks of a phase in a grid-stride loop, and phases are separated by
// a grid-wide barrier.  The phases are the same device functions the stand-alone kernels run
// (phases.cuh), in the same order, so the result is identical to the graph-launched loop; what
// changes is that ten barriers per iteration replace thirteen kernel launches.  Used for
// register-FFT problems with square padding (Px == Py) on the FP32 path.
//
// The barrier is a monotonic arrival counter in global memory (release by the arriving CTA,
// acquire by the waiting one).  Every wait is bounded (2^31 clock cycles unless the solve options
// give a shorter cap); on timeout the CTA raises the error flag and returns, so a launch that cannot complete ends in bounded time and the
// host reports PDF_ETIMEOUT.  Co-residency of all CTAs is guaranteed by the cooperative launch.
#include "phases.cuh"

struct PersistArgs {
  int iters;
  float2* alpha;
  float2* grad;
  float* m;
  float* v;
  int nparam;                  // real entries of alpha
  const float2* tab;
  int cap;
  float b1, b2, eps;
  double* terms;
  unsigned* bar;
  int* err;
  long long wait_cap;          // clock cycles a grid-barrier wait may last
  int n_data_blocks;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Returns false (and the CTA leaves the loop) when the wait lasted `cap` clock cycles or another CTA
// has already flagged a timeout.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned target, int* err, long long cap) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    atomicAdd(bar, 1u);
    if (ld_acquire_u32(bar) < target) {
      const long long t0 = clock64();
      unsigned spins = 0;
      while (ld_acquire_u32(bar) < target) {
        if ((spins++ & 31u) == 0 && (ld_relaxed_s32(err) != 0 || clock64() - t0 >= cap)) {
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

template <int P>
__global__ void __launch_bounds__(FT) k_persist(Dev d, PersistArgs a) {
  extern __shared__ float2 sm[];
  const int G = gridDim.x;
  unsigned gen = 0;
  const int rgx = (d.ny + FW - 1) / FW, nrow = rgx * d.ni;
  const int ncgx = d.Px / FCOLS, ncol = ncgx * d.ni;
  const int n_reg = d.n_reg_blocks, n_dat = a.n_data_blocks;
  const int n_gsh = (d.M + 63) / 64;
  const int n_ana = d.ky * d.ni;
  const int n_adam = (a.nparam + FT - 1) / FT;
  const int b0 = blockIdx.x;
#define PDF_BARRIER()                                                  \
  do {                                                                 \
    ++gen;                                                             \
    if (!grid_barrier(a.bar, gen * (unsigned)G, a.err, a.wait_cap)) return;        \
  } while (0)
  for (int it = 0; it < a.iters; ++it) {
    // forward: synthesis + row DFT, column convolution, row IDFT + CIE update + state residual
    for (int vb = b0; vb < nrow; vb += G) {
      ph_synth_rowfft<P>(d, vb % rgx, vb / rgx, sm, a.alpha, d.J, 1);
      __syncthreads();
    }
    PDF_BARRIER();
    for (int vb = b0; vb < ncol; vb += G) {
      ph_colconv<P>(d, vb % ncgx, vb / ncgx, sm, 0);
      __syncthreads();
    }
    PDF_BARRIER();
    for (int vb = b0; vb < d.ny; vb += G) {
      ph_rowifft_state<P>(d, vb, sm);
      __syncthreads();
    }
    PDF_BARRIER();
    // data term and regularisers
    for (int vb = b0; vb < d.n_gs_chunks; vb += G) {
      ph_gs_partial(d, vb, sm, d.J, d.gspart);
      __syncthreads();
    }
    PDF_BARRIER();
    for (int vb = b0; vb < n_dat + n_reg; vb += G) {
      if (vb < n_dat) ph_gs_reduce(d, vb, d.gspart, d.n_gs_chunks, d.esca, d.rd, d.lpart + LP_DATA * PDF_LP_STRIDE);
      else ph_reg(d, vb - n_dat, d.chi, nullptr);
      __syncthreads();
    }
    PDF_BARRIER();
    // adjoint
    for (int vb = b0; vb < nrow + n_gsh; vb += G) {
      if (vb < nrow) ph_adj_rowfft<P, false>(d, vb % rgx, vb / rgx, sm);
      else ph_gsh(d, vb - nrow, sm, d.rd, d.gsh, 0.f, 1);
      __syncthreads();
    }
    PDF_BARRIER();
    for (int vb = b0; vb < ncol; vb += G) {
      ph_colconv<P>(d, vb % ncgx, vb / ncgx, sm, 1);
      __syncthreads();
    }
    PDF_BARRIER();
    for (int vb = b0; vb < nrow; vb += G) {
      ph_adj_rowifft_ana<P>(d, vb % rgx, vb / rgx, sm, nullptr, 0);
      __syncthreads();
    }
    PDF_BARRIER();
    for (int vb = b0; vb < n_ana; vb += G) {
      ph_ana_y(d, vb % d.ky, vb / d.ky, d.T2, a.grad);
      __syncthreads();
    }
    PDF_BARRIER();
    // Adam step t = it + 1 and the loss terms of this iteration
    for (int vb = b0; vb < n_adam + 1; vb += G) {
      if (vb < n_adam) {
        ph_adam(vb * FT + threadIdx.x, (float*)a.alpha, (const float*)a.grad, a.m, a.v, a.nparam, it + 1, a.tab, a.cap,
                a.b1, a.b2, a.eps);
      } else {
        ph_finalize(d, a.terms, d.ny, n_dat, n_reg, nullptr);
      }
      __syncthreads();
    }
    PDF_BARRIER();
  }
#undef PDF_BARRIER
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
size_t sm_gs_bytes(const Dev& d);
size_t sm_gsh_bytes(const Dev& d);

static size_t persist_smem(const Dev& d) {
  size_t s = fp_smem_synth(d);
  s = std::max(s, fp_smem_col(d));
  s = std::max(s, fp_smem_state(d));
  s = std::max(s, fp_smem_ana(d));
  s = std::max(s, (size_t)d.Px * sizeof(float2));
  s = std::max(s, sm_gs_bytes(d));
  s = std::max(s, sm_gsh_bytes(d));
  return s;
}

template <int P>
static pdf_status launch_persist(pdf_problem* h, PersistArgs a, size_t smem, cudaStream_t st, bool* launched) {
  *launched = false;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_persist<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  int dev = 0, sms = 0, coop = 0, occ = 0;
  PDF_CUDA(cudaGetDevice(&dev));
  PDF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PDF_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  PDF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_persist<P>, FT, smem));
  if (!coop || occ < 1) return PDF_OK;                       // caller falls back to the graph loop
  dim3 grid(sms * std::min(occ, 2)), block(FT);
  Dev d = h->d;
  void* args[] = {(void*)&d, (void*)&a};
  PDF_CUDA(cudaLaunchCooperativeKernel((const void*)k_persist<P>, grid, block, args, smem, st));
  pdf_count_launch(1);
  *launched = true;
  return PDF_OK;
}

// Runs `iters` Adam iterations of h->alpha in one persistent launch.  *done = false (and nothing
// launched) when the problem does not qualify; the caller then uses the graph loop.
pdf_status ps_run(pdf_problem* h, const pdf_solve_opts* o, int iters, unsigned* bar, int* err, cudaStream_t st,
                  bool* done) {
  *done = false;
  const Dev& d = h->d;
  if (!d.fast || h->tc || d.fold || d.cco_loss || d.Px != d.Py || iters < 1) return PDF_OK;   // unfolded data term only
  PersistArgs a;
  a.iters = iters;
  a.alpha = h->alpha;
  a.grad = h->grad;
  a.m = h->adam_m;
  a.v = h->adam_v;
  a.nparam = 2 * d.ni * d.ky * d.kx;
  a.tab = h->adam_tab;
  a.cap = h->adam_cap;
  a.b1 = (float)o->adam_b1;
  a.b2 = (float)o->adam_b2;
  a.eps = (float)o->adam_eps;
  a.terms = h->terms;
  a.bar = bar;
  a.err = err;
  a.wait_cap = o->barrier_wait_cycles > 0 ? (long long)o->barrier_wait_cycles : (1ll << 31);
  a.n_data_blocks = (d.ni * d.nr + 255) / 256;
  PDF_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned), st));
  const size_t smem = persist_smem(d);
  if (smem > 200 * 1024) return PDF_OK;
  switch (d.Px) {
    case 64: return launch_persist<64>(h, a, smem, st, done);
    case 128: return launch_persist<128>(h, a, smem, st, done);
    case 256: return launch_persist<256>(h, a, smem, st, done);
    case 384: return launch_persist<384>(h, a, smem, st, done);
    case 512: return launch_persist<512>(h, a, smem, st, done);
    default: return PDF_OK;
  }
}
