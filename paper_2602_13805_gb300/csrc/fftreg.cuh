// Register-resident FFT of one line of length P = 32 R per warp (R = 2, 4, 8, 12 or 16).
//
// Lane l holds the R points x[l + 32 m] (m = 0 .. R-1).  With k = k1 + R k2,
//   X[k1 + R k2] = sum_l W32^{l k2} ( W_P^{l k1} sum_m x[l + 32 m] W_R^{m k1} ),
// so the forward transform is an R-point DFT in registers, a twiddle, and a 32-point
// decimation-in-frequency FFT across lanes with shuffles.  Its output is in digit-reversed
// order: lane l, slot k1 holds X[k1 + R brev5(l)].  The inverse (decimation in time) takes that
// order back to natural order, so a convolution (forward, pointwise product with a spectrum
// stored in the same permuted order, inverse) never reorders data.  Neither direction is
// normalised.  The twiddle table tw[e] = exp(-2 pi i e / P) is assembled in FP64 at setup.
#pragma once

#include "fft.cuh"

// W_R^e = exp(-2 pi i e / R) for the in-register R = 8, 12, 16 transforms (cos, -sin pairs)
static __constant__ float2 c_tw8[8] = {{1.000000000f, 0.000000000f},  {0.707106781f, -0.707106781f},
                                       {0.000000000f, -1.000000000f}, {-0.707106781f, -0.707106781f},
                                       {-1.000000000f, 0.000000000f}, {-0.707106781f, 0.707106781f},
                                       {0.000000000f, 1.000000000f},  {0.707106781f, 0.707106781f}};
static __constant__ float2 c_tw12[12] = {{1.000000000f, 0.000000000f},  {0.866025404f, -0.500000000f},
                                         {0.500000000f, -0.866025404f}, {0.000000000f, -1.000000000f},
                                         {-0.500000000f, -0.866025404f}, {-0.866025404f, -0.500000000f},
                                         {-1.000000000f, 0.000000000f}, {-0.866025404f, 0.500000000f},
                                         {-0.500000000f, 0.866025404f}, {0.000000000f, 1.000000000f},
                                         {0.500000000f, 0.866025404f},  {0.866025404f, 0.500000000f}};
static __constant__ float2 c_tw16[16] = {{1.000000000f, 0.000000000f},  {0.923879533f, -0.382683432f},
                                         {0.707106781f, -0.707106781f}, {0.382683432f, -0.923879533f},
                                         {0.000000000f, -1.000000000f}, {-0.382683432f, -0.923879533f},
                                         {-0.707106781f, -0.707106781f}, {-0.923879533f, -0.382683432f},
                                         {-1.000000000f, 0.000000000f}, {-0.923879533f, 0.382683432f},
                                         {-0.707106781f, 0.707106781f}, {-0.382683432f, 0.923879533f},
                                         {0.000000000f, 1.000000000f},  {0.382683432f, 0.923879533f},
                                         {0.707106781f, 0.707106781f},  {0.923879533f, 0.382683432f}};

// W_24^e (cos 15 e degrees, -sin 15 e degrees)
static __constant__ float2 c_tw24[24] = {
    {1.000000000f, 0.000000000f},   {0.965925826f, -0.258819045f},  {0.866025404f, -0.500000000f},
    {0.707106781f, -0.707106781f},  {0.500000000f, -0.866025404f},  {0.258819045f, -0.965925826f},
    {0.000000000f, -1.000000000f},  {-0.258819045f, -0.965925826f}, {-0.500000000f, -0.866025404f},
    {-0.707106781f, -0.707106781f}, {-0.866025404f, -0.500000000f}, {-0.965925826f, -0.258819045f},
    {-1.000000000f, 0.000000000f},  {-0.965925826f, 0.258819045f},  {-0.866025404f, 0.500000000f},
    {-0.707106781f, 0.707106781f},  {-0.500000000f, 0.866025404f},  {-0.258819045f, 0.965925826f},
    {0.000000000f, 1.000000000f},   {0.258819045f, 0.965925826f},   {0.500000000f, 0.866025404f},
    {0.707106781f, 0.707106781f},   {0.866025404f, 0.500000000f},   {0.965925826f, 0.258819045f}};

template <int R>
__device__ __forceinline__ float2 tw_small(int e) {
  return R == 8 ? c_tw8[e] : (R == 12 ? c_tw12[e] : (R == 16 ? c_tw16[e] : c_tw24[e]));
}

// t W_R^e (conjugated twiddle when INV) for an exponent that is a compile-time constant once the
// caller's loops are unrolled: quarter turns (W^{R/4} = -i, W^{R/2} = -1, W^{3R/4} = i) are exact
// swaps and sign changes, the other exponents a complex product with the table entry
template <int R, bool INV>
__device__ __forceinline__ float2 tw_mul(float2 t, int e) {
  e %= R;
  if (e == 0) return t;
  if (4 * e == R) return INV ? make_float2(-t.y, t.x) : make_float2(t.y, -t.x);
  if (2 * e == R) return make_float2(-t.x, -t.y);
  if (4 * e == 3 * R) return INV ? make_float2(t.y, -t.x) : make_float2(-t.y, t.x);
  float2 w = tw_small<R>(e);
  if (INV) w.y = -w.y;
  return cmul(t, w);
}

// R = 4 Q points, m = Q a + b:  X[k1 + 4 k2] = DFT_Q over b of ( W_R^{b k1} DFT_4 over a of x[Q a + b] )
template <int Q, bool INV>
__device__ __forceinline__ void dft_4xq(float2* v) {
  constexpr int R = 4 * Q;
  float2 F[Q][4];
#pragma unroll
  for (int b = 0; b < Q; ++b) {
    float2 t[4] = {v[b], v[Q + b], v[2 * Q + b], v[3 * Q + b]};
    Butterfly<float2, 4>::run(t, INV);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) F[b][k1] = tw_mul<R, INV>(t[k1], b * k1);
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 t[Q];
#pragma unroll
    for (int b = 0; b < Q; ++b) t[b] = F[b][k1];
    Butterfly<float2, Q>::run(t, INV);
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) v[k1 + 4 * k2] = t[k2];
  }
}

template <int R, bool INV> struct SmallDFT;
template <bool INV> struct SmallDFT<2, INV> {
  static __device__ __forceinline__ void run(float2* v) { Butterfly<float2, 2>::run(v, INV); }
};
template <bool INV> struct SmallDFT<4, INV> {
  static __device__ __forceinline__ void run(float2* v) { Butterfly<float2, 4>::run(v, INV); }
};
template <bool INV> struct SmallDFT<8, INV> {
  static __device__ __forceinline__ void run(float2* v) { dft_4xq<2, INV>(v); }
};
template <bool INV> struct SmallDFT<12, INV> {
  static __device__ __forceinline__ void run(float2* v) { dft_4xq<3, INV>(v); }
};
template <bool INV> struct SmallDFT<16, INV> {
  static __device__ __forceinline__ void run(float2* v) { dft_4xq<4, INV>(v); }
};

// R = 2 * 3 points, m = 3 a + b:  X[k1 + 2 k2] = DFT_3 over b of ( W_6^{b k1} DFT_2 over a of x[3 a + b] )
// (W_6^e = W_12^{2e})
template <bool INV> struct SmallDFT<6, INV> {
  static __device__ __forceinline__ void run(float2* v) {
    float2 F[3][2];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      F[b][0] = v[b] + v[3 + b];
      F[b][1] = v[b] - v[3 + b];
      if (b > 0) {
        float2 w = tw_small<12>(2 * b);
        if (INV) w.y = -w.y;
        F[b][1] = cmul(F[b][1], w);
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < 2; ++k1) {
      float2 t[3] = {F[0][k1], F[1][k1], F[2][k1]};
      Butterfly<float2, 3>::run(t, INV);
#pragma unroll
      for (int k2 = 0; k2 < 3; ++k2) v[k1 + 2 * k2] = t[k2];
    }
  }
};

// R = 8 * 3 points, m = 3 a + b:  X[k1 + 8 k2] = DFT_3 over b of ( W_24^{b k1} DFT_8 over a of x[3 a + b] )
template <bool INV> struct SmallDFT<24, INV> {
  static __device__ __forceinline__ void run(float2* v) {
    float2 F[3][8];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      float2 t[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) t[a] = v[3 * a + b];
      dft_4xq<2, INV>(t);
#pragma unroll
      for (int k1 = 0; k1 < 8; ++k1) F[b][k1] = tw_mul<24, INV>(t[k1], b * k1);
    }
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) {
      float2 t[3] = {F[0][k1], F[1][k1], F[2][k1]};
      Butterfly<float2, 3>::run(t, INV);
#pragma unroll
      for (int k2 = 0; k2 < 3; ++k2) v[k1 + 8 * k2] = t[k2];
    }
  }
};

__device__ __forceinline__ float2 shfl_xor2(float2 v, int m) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// Warp reduce-scatter of 16 complex values: on return lane l holds in a[0] the sum over the
// warp of the values with index l >> 1 (each halving step keeps the half selected by one lane bit).
__device__ __forceinline__ void warp_reduce_scatter16(float2 (&a)[16], int lane) {
#pragma unroll
  for (int st = 0; st < 4; ++st) {
    const int h = 16 >> st, n = 8 >> st;
    const bool up = (lane & h) != 0;
#pragma unroll
    for (int i = 0; i < n; ++i) {
      const float2 send = up ? a[i] : a[i + n];
      const float2 keep = up ? a[i + n] : a[i];
      a[i] = keep + shfl_xor2(send, h);
    }
  }
  a[0] = a[0] + shfl_xor2(a[0], 1);
}

template <int P> struct WarpFFT {
  static constexpr int R = P / 32;

  // natural order in (v[m] = x[lane + 32 m]) -> digit-reversed out (v[k1] = X[k1 + R brev5(lane)])
  // Each butterfly is branch-free: the upper lane of a pair computes (p - v) w, the lower one
  // (v + p) 1, i.e. (s v + p) w' with s = -1 / +1 and w' = w / 1 per lane; the last stage has w = 1.
  static __device__ __forceinline__ void forward(float2 (&v)[R], const float2* __restrict__ tw, int lane) {
    SmallDFT<R, false>::run(v);
#pragma unroll
    for (int k1 = 1; k1 < R; ++k1) v[k1] = cmul(v[k1], tw[lane * k1]);
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
      const bool hi = lane & h;
      const float s = hi ? -1.f : 1.f;
      if (h > 1) {
        const float2 wt = tw[(lane & (h - 1)) * (16 / h) * R];
        const float2 w = hi ? wt : make_float2(1.f, 0.f);
#pragma unroll
        for (int k = 0; k < R; ++k) {
          const float2 p = shfl_xor2(v[k], h);
          v[k] = cmul(make_float2(fmaf(s, v[k].x, p.x), fmaf(s, v[k].y, p.y)), w);
        }
      } else {
#pragma unroll
        for (int k = 0; k < R; ++k) {
          const float2 p = shfl_xor2(v[k], h);
          v[k] = make_float2(fmaf(s, v[k].x, p.x), fmaf(s, v[k].y, p.y));
        }
      }
    }
  }

  // digit-reversed in -> natural order out, unnormalised inverse (same branch-free butterflies)
  static __device__ __forceinline__ void inverse(float2 (&v)[R], const float2* __restrict__ tw, int lane) {
#pragma unroll
    for (int h = 1; h <= 16; h <<= 1) {
      const bool hi = lane & h;
      const float s = hi ? -1.f : 1.f;
      if (h > 1) {
        const float2 wt = cconj(tw[(lane & (h - 1)) * (16 / h) * R]);
        const float2 w = hi ? wt : make_float2(1.f, 0.f);
#pragma unroll
        for (int k = 0; k < R; ++k) {
          const float2 t = cmul(v[k], w);
          const float2 p = shfl_xor2(t, h);
          v[k] = make_float2(fmaf(s, t.x, p.x), fmaf(s, t.y, p.y));
        }
      } else {
#pragma unroll
        for (int k = 0; k < R; ++k) {
          const float2 p = shfl_xor2(v[k], h);
          v[k] = make_float2(fmaf(s, v[k].x, p.x), fmaf(s, v[k].y, p.y));
        }
      }
    }
#pragma unroll
    for (int k1 = 1; k1 < R; ++k1) v[k1] = cmul(v[k1], cconj(tw[lane * k1]));
    SmallDFT<R, true>::run(v);
  }
};

// L independent lines per warp, transformed together: the butterflies of WarpFFT applied stage by
// stage to every line, so the lines' shuffles and multiplies overlap (same results line by line).
template <int P, int L> struct WarpFFTn {
  static constexpr int R = P / 32;

  static __device__ __forceinline__ void forward(float2 (&v)[L][R], const float2* __restrict__ tw, int lane) {
#pragma unroll
    for (int l = 0; l < L; ++l) SmallDFT<R, false>::run(v[l]);
#pragma unroll
    for (int k1 = 1; k1 < R; ++k1) {
      const float2 w = tw[lane * k1];
#pragma unroll
      for (int l = 0; l < L; ++l) v[l][k1] = cmul(v[l][k1], w);
    }
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
      const bool hi = lane & h;
      const float s = hi ? -1.f : 1.f;
      if (h > 1) {
        const float2 wt = tw[(lane & (h - 1)) * (16 / h) * R];
        const float2 w = hi ? wt : make_float2(1.f, 0.f);
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
          for (int l = 0; l < L; ++l) {
            const float2 p = shfl_xor2(v[l][k], h);
            v[l][k] = cmul(make_float2(fmaf(s, v[l][k].x, p.x), fmaf(s, v[l][k].y, p.y)), w);
          }
      } else {
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
          for (int l = 0; l < L; ++l) {
            const float2 p = shfl_xor2(v[l][k], h);
            v[l][k] = make_float2(fmaf(s, v[l][k].x, p.x), fmaf(s, v[l][k].y, p.y));
          }
      }
    }
  }

  static __device__ __forceinline__ void inverse(float2 (&v)[L][R], const float2* __restrict__ tw, int lane) {
#pragma unroll
    for (int h = 1; h <= 16; h <<= 1) {
      const bool hi = lane & h;
      const float s = hi ? -1.f : 1.f;
      if (h > 1) {
        const float2 wt = cconj(tw[(lane & (h - 1)) * (16 / h) * R]);
        const float2 w = hi ? wt : make_float2(1.f, 0.f);
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
          for (int l = 0; l < L; ++l) {
            const float2 t = cmul(v[l][k], w);
            const float2 p = shfl_xor2(t, h);
            v[l][k] = make_float2(fmaf(s, t.x, p.x), fmaf(s, t.y, p.y));
          }
      } else {
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
          for (int l = 0; l < L; ++l) {
            const float2 p = shfl_xor2(v[l][k], h);
            v[l][k] = make_float2(fmaf(s, v[l][k].x, p.x), fmaf(s, v[l][k].y, p.y));
          }
      }
    }
#pragma unroll
    for (int k1 = 1; k1 < R; ++k1) {
      const float2 w = cconj(tw[lane * k1]);
#pragma unroll
      for (int l = 0; l < L; ++l) v[l][k1] = cmul(v[l][k1], w);
    }
#pragma unroll
    for (int l = 0; l < L; ++l) SmallDFT<R, true>::run(v[l]);
  }
};

// digit-reversal of the lane index (5 bits)
__host__ __device__ __forceinline__ int brev5(int l) {
  return ((l & 1) << 4) | ((l & 2) << 2) | (l & 4) | ((l & 8) >> 2) | ((l & 16) >> 4);
}

// true DFT index of permuted position c = k1 * 32 + lane for length P = 32 R
__host__ __device__ __forceinline__ int perm_to_freq(int c, int R) { return (c >> 5) + R * brev5(c & 31); }

// supported line lengths of the register path
__host__ __device__ __forceinline__ bool fast_len(int P) {
  return P == 64 || P == 128 || P == 256 || P == 384 || P == 512;
}
