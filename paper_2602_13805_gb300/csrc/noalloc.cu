// pdf_gs_apply_static: the receiver-operator product G_S x over all incidences, computed
// without allocating any device memory.
//
// Who needs this: callers whose device memory is owned by someone else -- a host framework
// whose caching allocator has already reserved the GPU's memory, or a latency-critical loop
// in which a cudaMalloc/cudaFree (which can synchronise the device) is not acceptable.  Such
// callers cannot use pdf_setup, which allocates the handle's workspace.
//
// The split-K partial products that the handle-based path keeps in its workspace live here
// in a file-scope __device__ array of fixed size (PDF_STATIC_SCRATCH_BYTES).  Every GPU that
// loads this library holds that array until the process exits.  Its device address is looked
// up with cudaGetSymbolAddress once per device, by the first call made on that device (so make
// that first call before any stream capture).  All calls share the array: calls that overlap
// on the GPU (different streams, or different host threads without ordering) race on it.
// Nothing in it has to start at zero: each call writes every partial slot it later reads.
#include <mutex>
#include <string>

#include "common.cuh"

#define PDF_STATIC_SCRATCH_BYTES (4u << 20)                       // 4 MiB
#define PDF_STATIC_SCRATCH_ELEMS (PDF_STATIC_SCRATCH_BYTES / 8u)  // complex64 slots
#define PDF_STATIC_MAX_DEVICES 64

static __device__ __align__(256) float2 g_gs_scratch[PDF_STATIC_SCRATCH_ELEMS];

// part[c][p][r] = sum over pixels n of chunk c of gs[r][n] x[p][n]
__global__ void __launch_bounds__(256) k_gs_partial_static(const float2* __restrict__ gs, const float2* __restrict__ x,
                                                           float2* __restrict__ part, int ni, int nr, int m, int chunk) {
  const int c = blockIdx.x;
  const int n0 = c * chunk;
  const int n1 = min(n0 + chunk, m);
  const int nout = ni * nr;
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    const int p = o / nr, r = o - p * nr;
    const float2* gr = gs + (size_t)r * m;
    const float2* xp = x + (size_t)p * m;
    float2 acc = make_float2(0.f, 0.f);
    for (int n = n0; n < n1; ++n) acc = cmac(acc, __ldg(&gr[n]), __ldg(&xp[n]));
    part[(size_t)c * nout + o] = acc;
  }
}

// out[p][r] = sum over chunks (FP64)
__global__ void k_gs_reduce_static(const float2* __restrict__ part, int nchunk, int nout, float2* __restrict__ out) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nout) return;
  double sx = 0.0, sy = 0.0;
  for (int c = 0; c < nchunk; ++c) {
    const float2 v = part[(size_t)c * nout + o];
    sx += v.x;
    sy += v.y;
  }
  out[o] = make_float2((float)sx, (float)sy);
}

static std::mutex g_scratch_mu;
static float2* g_scratch_ptr[PDF_STATIC_MAX_DEVICES];

pdf_status set_err(pdf_status st, const std::string& msg);

static pdf_status scratch_for_current_device(float2** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_err(PDF_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= PDF_STATIC_MAX_DEVICES) return set_err(PDF_EUNSUPPORTED, "device index above 63");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_gs_scratch);
    if (e != cudaSuccess || !p)
      return set_err(PDF_ECUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = (float2*)p;
  }
  *out = g_scratch_ptr[dev];
  return PDF_OK;
}

extern "C" pdf_status pdf_gs_apply_static(const void* gs, const void* x, void* out, int32_t ni, int32_t nr,
                                          int32_t m, void* stream) {
  if (!gs || !x || !out) return set_err(PDF_EINVAL, "pdf_gs_apply_static: gs, x or out is NULL");
  if (ni < 1 || nr < 1 || m < 1) return set_err(PDF_EINVAL, "pdf_gs_apply_static: ni, nr, m must be >= 1");
  const long long nout = (long long)ni * nr;
  if (nout > (long long)PDF_STATIC_SCRATCH_ELEMS)
    return set_err(PDF_EINVAL, "pdf_gs_apply_static: ni * nr exceeds the static scratch (4 MiB = 524288 complex64)");
  // as many pixel chunks as fit in the scratch, at most one per 256 pixels
  long long nchunk = ((long long)m + 255) / 256;
  const long long fit = (long long)PDF_STATIC_SCRATCH_ELEMS / nout;
  if (nchunk > fit) nchunk = fit;
  if (nchunk > 65535) nchunk = 65535;
  const int chunk = (int)(((long long)m + nchunk - 1) / nchunk);
  nchunk = ((long long)m + chunk - 1) / chunk;
  float2* scratch = nullptr;
  pdf_status st = scratch_for_current_device(&scratch);
  if (st != PDF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  k_gs_partial_static<<<(unsigned)nchunk, 256, 0, s>>>((const float2*)gs, (const float2*)x, scratch, ni, nr, m, chunk);
  k_gs_reduce_static<<<(unsigned)((nout + 255) / 256), 256, 0, s>>>(scratch, (int)nchunk, (int)nout, (float2*)out);
  pdf_count_launch(2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_err(PDF_ECUDA, std::string("pdf_gs_apply_static: ") + cudaGetErrorString(e));
  return PDF_OK;
}
