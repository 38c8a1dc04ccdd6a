// Batched 1-D FFTs on lines held in shared memory (Stockham auto-sort, radix 4/2/3).
//
// A CTA transforms `nlines` lines of length P at once; line l occupies
// buf[l * ls .. l * ls + P).  Each stage reads from one buffer and writes the
// other, so the caller provides two buffers of nlines * ls elements and gets
// back the pointer holding the result.  All threads of the block must call the
// routine (it synchronises between stages).  Twiddles come from a table of P
// entries tw[e] = exp(-2 pi i e / P) assembled once in FP64 on the device; the
// inverse uses conjugated twiddles and is not normalised.
#pragma once

#include "common.cuh"

template <typename C>
__device__ __forceinline__ C imul(C a) { return mk(-a.y, a.x); }   // i * a

template <typename C, int R> struct Butterfly;

template <typename C> struct Butterfly<C, 2> {
  static __device__ __forceinline__ void run(C* v, bool) {
    C t = v[0] - v[1];
    v[0] = v[0] + v[1];
    v[1] = t;
  }
};

template <typename C> struct Butterfly<C, 4> {
  static __device__ __forceinline__ void run(C* v, bool inv) {
    C t0 = v[0] + v[2], t1 = v[0] - v[2], t2 = v[1] + v[3], t3 = v[1] - v[3];
    C it3 = imul(t3);
    v[0] = t0 + t2;
    v[2] = t0 - t2;
    if (!inv) { v[1] = t1 - it3; v[3] = t1 + it3; }
    else      { v[1] = t1 + it3; v[3] = t1 - it3; }
  }
};

template <typename C> struct Butterfly<C, 3> {
  static __device__ __forceinline__ void run(C* v, bool inv) {
    typedef decltype(v[0].x) T;
    const T h = (T)0.8660254037844386467637231707529362;   // sin(2 pi / 3)
    C s = v[1] + v[2], d = v[1] - v[2];
    C m = v[0] - (T)0.5 * s;
    C id = imul(d);
    v[0] = v[0] + s;
    if (!inv) { v[1] = m - h * id; v[2] = m + h * id; }
    else      { v[1] = m + h * id; v[2] = m - h * id; }
  }
};

template <typename C, int R>
__device__ __forceinline__ void fft_stage(const C* __restrict__ in, C* __restrict__ out, int P, int Ns,
                                          int nlines, int ls, const C* __restrict__ tw, bool inv) {
  const int nb = P / R;
  const int total = nb * nlines;
  const int tstride = P / (Ns * R);
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int line = idx / nb;
    const int j = idx - line * nb;
    const C* src = in + line * ls;
    C* dst = out + line * ls;
    const int k = j % Ns;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[j + r * nb];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C w = __ldg(&tw[k * r * tstride]);
        if (inv) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    Butterfly<C, R>::run(v, inv);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[base + r * Ns] = v[r];
  }
}

// Transforms all lines; returns the buffer (a or b) that holds the result.
template <typename C>
__device__ C* fft_lines(C* a, C* b, int nlines, int ls, const FFTPlan& pl, const C* __restrict__ tw, bool inv) {
  int Ns = 1;
  for (int s = 0; s < pl.nst; ++s) {
    const int R = pl.radix[s];
    if (R == 4) fft_stage<C, 4>(a, b, pl.P, Ns, nlines, ls, tw, inv);
    else if (R == 2) fft_stage<C, 2>(a, b, pl.P, Ns, nlines, ls, tw, inv);
    else fft_stage<C, 3>(a, b, pl.P, Ns, nlines, ls, tw, inv);
    __syncthreads();
    Ns *= R;
    C* t = a; a = b; b = t;
  }
  return a;
}

// Host: plan for P = 2^a 3^b (radix 4 first, then 2, then 3).  Returns false otherwise.
static inline bool make_fft_plan(int P, FFTPlan* pl) {
  pl->P = P;
  pl->nst = 0;
  int q = P;
  while (q % 4 == 0) { pl->radix[pl->nst++] = 4; q /= 4; }
  while (q % 2 == 0) { pl->radix[pl->nst++] = 2; q /= 2; }
  while (q % 3 == 0) { pl->radix[pl->nst++] = 3; q /= 3; }
  return q == 1 && pl->nst <= PDF_MAX_RADICES;
}

// Host: smallest 2^a 3^b >= n.
static inline int next_smooth(int n) {
  int best = 1 << 30;
  for (long p2 = 1; p2 < (1L << 20); p2 *= 2)
    for (long p = p2; p < (1L << 20); p *= 3)
      if (p >= n && p < best) best = (int)p;
  return best;
}
