// Split-BF16 tensor-core form of the dense contractions (precision = 1):
//   synthesis     J[p][y][x]  = sum_jy Wy[y][jy] T[p][jy][x],  T = alpha_p Wx^T  (Eq. 9)
//   analysis      T2[p][y][jx] = sum_x gJ[p][y][x] conj(Wx[jx][x])               (Eq. 9 adjoint)
//   data          (G_S J)[p][r] = sum_n G_S[r][n] J[p][n]                          (Eq. 16)
//   data adjoint  (G_S^H r_d)[p][n] = sum_r conj(G_S[r][n]) r_d[p][r]
// Complex products are embedded as real GEMMs with interleaved (re, im) K and two output
// columns per complex result; every operand is stored as a bf16 hi/lo pair.
#pragma once

#include <cuda_bf16.h>

#include "umma.cuh"

struct TC {
  int K2M, K2R, KYP, KXP;        // padded K extents (multiples of 64)
  int nsplit_fwd;
  // setup-time operands
  __nv_bfloat16 *gsa_hi, *gsa_lo;     // [nr][K2M]   G_S interleaved
  __nv_bfloat16 *gst_hi, *gst_lo;     // [M][K2R]    G_S^T interleaved
  __nv_bfloat16 *wya_hi, *wya_lo;     // [ny][KYP]   Wy interleaved over jy
  __nv_bfloat16 *wxb_hi, *wxb_lo;     // [2 kx][KXP] conj(Wx) embedding
  // per-iteration operands
  __nv_bfloat16 *jb_hi, *jb_lo;       // [2 ni][K2M]
  __nv_bfloat16 *rdb_hi, *rdb_lo;     // [2 ni][K2R]
  __nv_bfloat16 *tb_hi, *tb_lo;       // [2 ni nx][KYP]
  __nv_bfloat16 *gja_hi, *gja_lo;     // [ni ny][KXP]
  float *c_fwd;                       // [nsplit][nr][2 ni]
  float *c_adj;                       // [M][2 ni]
  float *c_syn;                       // [ny][2 ni nx]
  float *c_ana;                       // [ni ny][2 kx]
  int* err;
  UmmaOperand gsa, gst, wya, wxb, jb, rdb, tb, gja;
};

struct pdf_problem;
pdf_status tc_setup(pdf_problem* h, cudaStream_t st);
pdf_status tc_synth(pdf_problem* h, const float2* alpha, float2* Jout, int do_fft, cudaStream_t st);
pdf_status tc_gs_fwd(pdf_problem* h, const float2* X, const float2* sub, float2* out, FF* lp, int write_rdb,
                     cudaStream_t st);
pdf_status tc_gsh(pdf_problem* h, const float2* D, int from_rdb, cudaStream_t st);
pdf_status tc_adj_ana(pdf_problem* h, cudaStream_t st);
pdf_status tc_analysis_field(pdf_problem* h, const float2* in, cudaStream_t st);
pdf_status tc_gsh_field(pdf_problem* h, const float2* D, float2* out, float scale, cudaStream_t st);
