// Internal state of a pdf_problem handle and the by-value kernel parameter block.
#pragma once

#include <string>
#include <vector>

#include "common.cuh"

// Loss-partial slots (each a strip of PDF_LP_STRIDE doubles in Dev::lpart).
enum { LP_STATE = 0, LP_DATA = 1, LP_BOUND = 2, LP_TV = 3, LP_BRIDGE = 4, LP_NSLOT = 5 };
#define PDF_LP_STRIDE 4096

#define ROWS_PER_CTA 4        // rows handled by one CTA of the row-FFT kernels
#define ROW_THREADS 128
#define COL_CW 16             // columns per CTA of the column-convolution kernel
#define COL_THREADS 256
#define GS_CHUNK 256          // pixels per CTA of the G_S partial-product kernel
#define GSH_CHUNK 64          // pixels per CTA of the G_S^H kernel

// Everything a kernel needs, passed by value.
struct Dev {
  int nx, ny, ni, nr, kx, ky, M, Px, Py;
  FFTPlan plx, ply;
  float2 beta;
  double2 betad;
  float lam_bound, lam_tv, lam_bridge, tau_b, eps_tv, eps_abs, q_min;
  int n_gs_chunks, n_reg_blocks;
  int fast;              // 1: register-FFT kernels (fastpath.cu), A rows/columns in permuted order

  // geometry (assembled once)
  const float2* twx;     // [Px] exp(-2 pi i e / Px)
  const float2* twy;     // [Py]
  const float2* ghat;    // [Py][Px] spectrum of the circulant G_D kernel / (Px Py)
  const float2* ghat_perm; // [Px][Py] the same in the register FFT's digit-reversed order (fast path)
  const float2* ghat_col;  // [Px][Py] by column (register FFT's order), natural y-frequency order
  const float2* what;    // [kx][Px] row DFT of the x basis, columns in that order (cluster loop)
  const float2* einc;    // [ni][M]
  const float2* gs;      // [nr][M]
  const float2* gsf;     // [nr][ky*kx] folded receiver operator G_S Phi (when fold)
  int fold;              // 1: data term through gsf on the coefficients
  const float2* wx;      // [kx][nx] exp(+2 pi i f_k x / nx) / sqrt(nx)
  const float2* wy;      // [ky][ny]
  const float2* ux;      // [nx] exp(2 pi i m / nx) / sqrt(nx), Wx[jx][x] = ux[f_jx x mod nx] (register-FFT path)
  const float2* esca;    // [ni][nr]
  const double* norms;   // [2] ||E_inc||^2, ||E_sca||^2

  // per-iteration workspace
  float2* J;             // [ni][M]
  float2* A;             // [ni][ny][Px] row-transformed padded planes
  float2* s;             // [ni][M] beta J + E_inc + G_D J
  float2* r;             // [ni][M] state residual
  int nsg;               // > 0: state pass split over nsg incidence groups (register-FFT path)
  float4* sgA;           // [nsg][M] per-group float-float sums of beta J conj(s) (re hi, re lo, im hi, im lo)
  float2* sgB;           // [nsg][M] per-group float-float sums of |s|^2
  float2* v;             // [ni][M] pointwise part of dL/dJ
  float2* gsh;           // [ni][M] scaled G_S^H r_d
  float2* R;             // [M]
  float2* chi;           // [M]
  float2* w;             // [M] regulariser cotangent on R divided by D
  float* D;              // [M] sum_p |s|^2
  unsigned char* clamp;  // [M]
  float2* T2;            // [ni][ny][kx] partial analysis
  float2* gspart;        // [n_gs_chunks][ni][nr]
  float2* rd;            // [ni][nr] data residual
  FF* lpart;             // [LP_NSLOT][PDF_LP_STRIDE] float-float loss partials (also scratch)
  const float* invn;     // [2] 2 / ||E_inc||^2, 2 / ||E_sca||^2 (float)
  const float2* adam_tab;  // [cap] Adam step size lr / (1 - b1^t) and sqrt(1 - b2^t), t = 1..cap
  int gs_chunk;          // pixels per CTA of the SIMT G_S product
  int rdwarp;             // 1: the data residual runs as k_gsf_fwd_p (a warp per receiver, no reduction)
  int rd_synth;           // 1: the data residual is formed inside the tiled synthesis (kf_synth_2p)
  int row2p;              // 1: split state pass by tiles (kf_state_2p)

  // CCO inside the loss (pdf_config.cco_in_loss): the regularisers act on chi_CCO (ccoloss.cu)
  int cco_loss;
  int cco_r;             // guided-filter box radius
  float cco_eps, cco_eta_max, cco_tau, cco_delta;
  float2* chic;          // [M] chi_CCO
  float4* cca;           // [M] per window: 1 - a and the mean, Re then Im (guided-filter coefficients)
  float2* ccc;           // [M] regulariser cotangent on chi_CCO
  float2* ccd;           // [M] the part of the cotangent on chi-hat that needs no window sum
  float4* ccu;           // [M] per pixel: cotangents headed for the window coefficients / count
  float4* ccp;           // [M] per window: cotangents headed for the pixels / count
};

struct TC;

// State of the coefficient-correcting network (fcnn.cu), allocated on the first solve that uses it.
struct FcState {
  int H, D, B;           // hidden width, 2 ky kx, ni
  size_t np;             // parameter count
  float* theta;          // [np] W1 [H][D], b1 [H], W2 [H][H], b2 [H], W3 [D][H], b3 [D]
  float* gtheta;         // [np]
  float* m;              // [np] Adam moments
  float* v;
  float* X;              // [B][D] scaled input
  float* s;              // [1] input scale
  float* h1;             // [B][H]
  float* h2;             // [B][H]
  float* y;              // [B][D] output, then dL/dy
  float* dz1;            // [B][H]
  float* dz2;            // [B][H]
  float2* alpha0;        // [ni][ky][kx] the network's input coefficients
  float* work;           // split-k partial sums
  unsigned* tick;        // [FC_TICKS] per-output-tile arrival counters of the split-k products (zero between uses)
  float* nvec;           // [B][D + 4H] per-incidence chain-rule vectors of the cluster loop (allocated on first use)
};

struct pdf_problem {
  pdf_config cfg;
  FcState fc;
  TC* tc;                // split-BF16 tensor-core state (precision = 1), else NULL
  std::vector<double> tx, rx;
  Dev d;
  int dev_id;
  // owned device memory
  std::vector<void*> allocs;
  // solve state
  float2* alpha;         // [ni][ky][kx]
  float2* grad;
  float* adam_m;         // [2 * ni * ky * kx]
  float* adam_v;
  int* adam_t;           // device step counter
  double* terms;         // [6] device
  double* scratch_d;     // [64] device doubles for init/solve scalars
  float2* tmpA;          // [ni][M] scratch fields for init / ops
  float2* tmpB;
  float2* tmpC;
  float2* field1;        // [M]
  float2* field2;
  float2* field3;
  float2* esca_host_pinned;  // pinned staging [ni][nr]
  float4* cco_ab;        // [M] guided-filter coefficients
  float2* alpha_alt;     // [ni][ky][kx] warm-start candidate
  int* used_warm;        // device flag
  unsigned* bar;         // grid-barrier counter of the persistent and cluster loops
  float4* cl_nd;         // cluster loop: per-incidence pixel sums (lazily allocated)
  int* perr;             // [4]: loop error flag (1 barrier timeout, 2 wrong cluster shape), non-finite
                         // output flag, the RelErr reduction's block counter, unused
  double* relerr_part;   // [3 * RELERR_BLOCKS] per-block partial sums of the final RelErr
  float2* small1;        // [ni][nr] scratch
  float2* small2;
  cudaStream_t cap_stream;   // private stream used only for graph capture
  cudaGraphExec_t graph_exec;
  int graph_iters;       // iterations per graph launch (0 = none)
  int graph_kernels;     // kernel nodes in the graph
  double graph_key[5];   // lr, b1, b2, eps, network width used when captured
  int fc_active;         // the current solve optimises the network's weights (fcnn.cu)
  float2* adam_tab;      // device table (see Dev::adam_tab)
  int adam_cap;
  double adam_key[3];    // lr, b1, b2 of the table
  float* invn;
};

// blocks of the final RelErr reduction (solve.cu)
#define RELERR_BLOCKS 148

// coefficient-correcting network (fcnn.cu)
pdf_status fc_prepare(pdf_problem* h, int hidden, const void* params0, cudaStream_t st);
pdf_status fc_forward(pdf_problem* h, cudaStream_t st);    // h->alpha = alpha0 + Delta alpha(theta)
pdf_status fc_backward(pdf_problem* h, cudaStream_t st);   // fc.gtheta from h->grad

// error helpers (api.cu)
pdf_status set_err(pdf_status st, const std::string& msg);
pdf_status cuda_err(cudaError_t e, const char* where);
#define PDF_CUDA(call)                                  \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) return cuda_err(_e, #call);  \
  } while (0)
#define PDF_LAUNCHED(where)                                         \
  do {                                                              \
    cudaError_t _e = cudaGetLastError();                            \
    if (_e != cudaSuccess) return cuda_err(_e, where);              \
  } while (0)

// workspace allocation owned by the handle (api.cu)
pdf_status ws_alloc(pdf_problem* h, void** p, size_t bytes);

// reductions defined in api.cu
__global__ void k_sumsq(const float2* x, int n, double* out);
__global__ void k_set_invn(const double* norms, float* invn);

// CCO inside the loss (ccoloss.cu): chi_CCO from d.chi, the regularisers on it, and their
// cotangent carried back through the CCO to chi-hat and on to w (replaces k_reg)
pdf_status cc_reg(const Dev& d, cudaStream_t st);
constexpr int CCO_LOSS_KERNELS = 6;

// launchers (hotpath.cu)
pdf_status hp_configure_kernels();
pdf_status hp_check_limits(const Dev& d);
pdf_status hp_loss_grad(pdf_problem* h, const float2* alpha, float2* grad, double* terms, cudaStream_t st,
                        int* step_inc = nullptr, cudaEvent_t* ev = nullptr);
const char* hp_kernel_name(int k, int precision, int fold, int rd_synth);
bool hp_rdwarp_ok(const Dev& d);
__global__ void k_ana_y(Dev d, const float2* T2, float2* out, int* step_inc);
pdf_status hp_gd(pdf_problem* h, const float2* in, float2* out, int adjoint, cudaStream_t st);
pdf_status hp_gs(pdf_problem* h, const float2* in, float2* out, const float2* subtract, FF* sumsq, cudaStream_t st);
pdf_status hp_gsh(pdf_problem* h, const float2* in, float2* out, float scale, cudaStream_t st);
pdf_status hp_synth(pdf_problem* h, const float2* alpha, float2* out, cudaStream_t st);
pdf_status hp_analysis(pdf_problem* h, const float2* in, float2* out, cudaStream_t st);
pdf_status hp_chi(pdf_problem* h, const float2* alpha, float2* chi_out, cudaStream_t st);
int hp_kernels_per_loss_grad(const pdf_problem* h);

// register-FFT path (fastpath.cu)
pdf_status fp_configure();
pdf_status fp_synth_rowfft(const Dev& d, const float2* alpha, float2* Jout, int do_fft, cudaStream_t st,
                           int dterm = 0);
bool fp_synth2p_ok(const Dev& d);
bool fp_row2p_ok(const Dev& d);
bool fp_ana_y_fft(const Dev& d, const float2* T2, float2* out, int* step_inc, cudaStream_t st);
int fp_synth2p_tpi(const Dev& d);
pdf_status fp_rowfft_field(const Dev& d, const float2* in, cudaStream_t st);
pdf_status fp_rowifft_field(const Dev& d, float2* out, cudaStream_t st);
pdf_status fp_colconv(const Dev& d, int conj, cudaStream_t st);
pdf_status fp_rowifft_state(const Dev& d, cudaStream_t st);
pdf_status fp_adj_rowfft(const Dev& d, cudaStream_t st);
pdf_status fp_adj_rowifft_ana(const Dev& d, const float2* in, int mode, cudaStream_t st);
pdf_status fp_perm_ghat(const Dev& d, float2* gp, cudaStream_t st);
pdf_status fp_col_ghat(const Dev& d, float2* gc, cudaStream_t st);
pdf_status fp_unit_table(int n, float2* u, cudaStream_t st);
size_t fp_smem_synth(const Dev& d);
size_t fp_smem_col(const Dev& d);
size_t fp_smem_state(const Dev& d);
size_t fp_smem_ana(const Dev& d);
size_t fp_smem_sums(const Dev& d);
int fp_n_state(const Dev& d);
int fp_choose_nsg(const Dev& d, int sms);
pdf_status fp_row_dft_table(const Dev& d, float2* what, cudaStream_t st);

// persistent solve loop (persist.cu)
pdf_status ps_run(pdf_problem* h, const pdf_solve_opts* o, int iters, unsigned* bar, int* err, cudaStream_t st,
                  bool* done);

// cluster solve loop (cluster.cu)
pdf_status cl_run(pdf_problem* h, const pdf_solve_opts* o, int iters, cudaStream_t st, bool* done);

// solve pieces (solve.cu)
pdf_status sv_cco(pdf_problem* h, const float2* chi, float2* out, int radius, double eps, double eta_max,
                  double tau, double delta, cudaStream_t st);
pdf_status sv_solve(pdf_problem* h, const pdf_solve_opts* o, float2* chi_out, float2* chi_raw_out,
                    float2* alpha_out, pdf_solve_report* rep, cudaStream_t st);
pdf_status sv_forward(pdf_problem* h, const float2* chi, float2* esca_out, float2* j_out, double tol,
                      int max_iter, int* iters_out, cudaStream_t st);
