/*
 * pdf.h -- C ABI of the GB300 (sm_103a) implementation of the per-iteration loss and
 * gradient of the physics-driven Fourier-spectral (PDF) inverse-scattering solver
 * (arXiv 2602.13805), with its initialisation, outer Adam loop and post-processing.
 *
 * Conventions shared by every entry point
 *   - Complex arrays are interleaved complex64 (float re, float im), row-major, x fastest.
 *     Grid arrays are [ny][nx] (M2 rows of M1 pixels, Sec. 2); per-incidence arrays are
 *     [ni][ny][nx]; Fourier coefficients are [ni][ky][kx]; measured data are [ni][nr].
 *   - Retained Fourier indices per axis of length M (Sec. 2.3, Eq. 9): storage slot j holds
 *     DFT index j for j < ceil(K/2) and M - K + j otherwise (K = 2 M_F gives the paper's four
 *     M_F x M_F corner blocks; odd K gives the symmetric set).  The DFT is unitary.
 *   - Gradients of the real loss L with respect to complex z follow PyTorch's convention
 *     dL/dRe z + i dL/dIm z.
 *   - Every call is asynchronous on the CUDA stream it is given (NULL = legacy default
 *     stream) unless its comment says it synchronises.  Device pointers are caller-owned and
 *     are not retained after the call returns.  The problem handle owns its workspace.
 *   - Every call returns a pdf_status; nothing aborts or throws.  On failure
 *     pdf_last_error() returns a message for the calling thread.
 *   - A handle may be used by one stream at a time (its workspace is not duplicated).
 */
#ifndef PDF_H
#define PDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pdf_status {
  PDF_OK = 0,
  PDF_EINVAL = -1,        /* invalid argument (sizes, pointers, parameters)            */
  PDF_ENOMEM = -2,        /* device allocation failed                                  */
  PDF_ECUDA = -3,         /* a CUDA runtime call or kernel launch failed               */
  PDF_ENONFINITE = -4,    /* a loss term became NaN/Inf (only detected when synchronising) */
  PDF_ETIMEOUT = -5,      /* a bounded device-side wait ran out                        */
  PDF_EUNSUPPORTED = -6   /* a size or mode this build does not support                */
} pdf_status;

typedef struct pdf_problem pdf_problem;   /* opaque, owned by the library */

/* Problem statement (Sec. 2 and Sec. 3.2).  Lengths are in the same unit as 2*pi/k0. */
typedef struct pdf_config {
  int32_t nx, ny;            /* M1 x M2 pulse grid over the DOI, 2 <= nx, ny <= 256          */
  double side_x, side_y;     /* DOI side lengths; the DOI is centred on the origin           */
  double k0;                 /* free-space wavenumber (real, > 0)                            */
  int32_t ni, nr;            /* incidences (transmitters) and receivers, 1..1024 each         */
  const double* tx_xy;       /* host [ni][2]: line-source positions, or plane-wave directions */
  const double* rx_xy;       /* host [nr][2]: receiver positions (outside the DOI)           */
  int32_t inc_kind;          /* 0 = line source H0(k0|r - r_p|)/|H0(k0|r_p|)|, 1 = plane wave  */
  int32_t kx, ky;            /* Fourier truncation, 1 <= kx <= nx, 1 <= ky <= ny (Eq. 9)      */
  double beta_re, beta_im;   /* CIE parameter beta of Eq. (6)-(7); Re beta > 0 required      */
  double lambda_bound;       /* lambda_1 of Eq. (13), paper 1e-3                             */
  double lambda_tv;          /* lambda_2, paper 1e-5                                         */
  double lambda_bridge;      /* lambda_3, paper 1e-5                                         */
  double tau_b;              /* bridge threshold tau_B of Eq. (19), paper 0.5                */
  double eps_tv;             /* smoothing inside the TV square root of Eq. (18)              */
  double eps_abs;            /* smoothing inside |chi| of Eq. (19)                           */
  double q_min;              /* clamp of |1 - R| when forming chi = R / (beta (1 - R))       */
  int32_t precision;         /* 0 = FP32 contractions, 1 = split-BF16 tensor-core contractions */
  int32_t fft_path;          /* 0 = register-resident warp FFTs (padded lengths 64..512),
                                1 = generic shared-memory FFT (any padded length 2^a 3^b)      */
  int32_t fold_gs;           /* 1 (default) = data term through the folded receiver operator
                                G_S Phi [nr][ky*kx], assembled once at setup with compensated
                                sums: r_d = (G_S Phi) alpha - E_sca and its adjoint act on the
                                Fourier coefficients (Eq. 9 and 16 composed); 0 = G_S applied to
                                the synthesised currents J every iteration (tensor cores at
                                precision 1).  Same result up to rounding.                      */
  /* Contrast-compensated operator (Sec. 2.4, Eq. 10-11): chi_CCO = (1 + eta) G(chi|chi) + eta chi,
   * G the self-guided filter (box radius cco_radius, windows clipped to the grid, regulariser
   * cco_eps, Re and Im filtered separately), eta = cco_eta_max sigmoid((|chi| - cco_tau)/cco_delta).
   * cco_in_loss = 1: L_Bound, L_TV and L_Bridge (Eq. 17-19) act on chi_CCO of the current chi-hat
   * instead of on chi-hat, and the gradient runs through the CCO's adjoint; pdf_solve's final CCO
   * then uses these parameters too.  0 (default): the CCO only post-processes a solve's output, as
   * Sec. 4.3 describes it, with the pdf_solve_opts parameters.  With cco_in_loss = 1 the solve's
   * loop runs as the CUDA graph (use_graph 2 and 3 fall back to it).  Defaults 0, 2, 1e-2, 0.1, 3,
   * 0.5; 0 <= cco_radius <= 16, cco_eps > 0, cco_delta > 0. */
  int32_t cco_in_loss;
  int32_t cco_radius;
  double cco_eps, cco_eta_max, cco_tau, cco_delta;
} pdf_config;

/* Fills the paper's defaults (beta = 6, lambdas 1e-3/1e-5/1e-5, tau_B = 0.5, k0 = 2 pi, the CCO
 * parameters of Eq. 11) and zero sizes/pointers.  Never fails. */
void pdf_config_default(pdf_config* cfg);

/* Assembles the operators of one geometry on the device: the Richmond G_D kernel spectrum
 * (FP64 Bessel evaluation and FP64 DFT, Eq. 1 and 3), G_S (Eq. 2 and 4), the incident fields,
 * the Fourier synthesis tables (Eq. 9), and allocates the workspace.  esca (may be NULL, then
 * set it with pdf_set_data before use): measured scattered field [ni][nr] complex64, on the
 * host when esca_on_device == 0 (copied synchronously) or on the device.  Synchronises `stream`
 * before returning.  Errors: PDF_EINVAL for out-of-range sizes/parameters or NULL antenna
 * arrays, PDF_EUNSUPPORTED for sizes above the limits stated in pdf_config, PDF_ENOMEM. */
pdf_status pdf_setup(const pdf_config* cfg, const void* esca, int esca_on_device, void* stream,
                     pdf_problem** out);

/* Replaces the measured data E_sca [ni][nr] complex64 (host when on_device == 0: the copy is
 * staged through the handle's pinned buffer and is asynchronous on `stream`; device otherwise)
 * and recomputes ||E_sca||^2 on the device (Eq. 16 denominator). */
pdf_status pdf_set_data(pdf_problem* h, const void* esca, int on_device, void* stream);

/* One evaluation of the composite loss of Eq. (13)-(19) and its gradient.
 *   alpha [ni][ky][kx] complex64, device, read only.
 *   grad  [ni][ky][kx] complex64, device, overwritten with dL/d alpha (may be NULL).
 *   terms [6] float64, device, overwritten with L, L_State, L_Data, L_Bound, L_TV, L_Bridge
 *         (may be NULL).
 * R-hat is the per-pixel least-squares solution of Eq. (6) over the incidences and
 * chi-hat = R / (beta (1 - R)) (Eq. 7); the gradient differentiates through both. */
pdf_status pdf_loss_grad(pdf_problem* h, const void* alpha, void* grad, double* terms, void* stream);

/* Operator application for testing and for callers composing their own solvers.
 * in/out are device complex64 arrays of the shapes below (ni batched where marked). */
enum pdf_op {
  PDF_OP_GD = 0,    /* [ni][ny][nx] -> [ni][ny][nx]   G_D x (zero-padded FFT convolution) */
  PDF_OP_GDH = 1,   /* [ni][ny][nx] -> [ni][ny][nx]   G_D^H x                             */
  PDF_OP_GS = 2,    /* [ni][ny][nx] -> [ni][nr]       G_S x                               */
  PDF_OP_GSH = 3,   /* [ni][nr]     -> [ni][ny][nx]   G_S^H d                             */
  PDF_OP_SYN = 4,   /* [ni][ky][kx] -> [ni][ny][nx]   F*_T (synthesis, Eq. 9)             */
  PDF_OP_ANA = 5,   /* [ni][ny][nx] -> [ni][ky][kx]   F_T restricted to retained modes    */
  PDF_OP_CCO = 6,   /* [ny][nx]     -> [ny][nx]       contrast-compensated operator (Eq. 10-11) */
  PDF_OP_CHI = 7,   /* [ni][ky][kx] -> [ny][nx]       chi-hat of the CIE update (Eq. 6-7) */
  PDF_OP_EINC = 8   /* (ignored)    -> [ni][ny][nx]   the assembled incident fields        */
};
pdf_status pdf_apply_op(pdf_problem* h, int op, const void* in, void* out, void* stream);

/* Options of a whole reconstruction (Sec. 3): initialisation, Adam on alpha viewed as
 * (Re, Im) pairs with torch.optim.Adam semantics, final chi-hat, CCO post-processing. */
typedef struct pdf_solve_opts {
  int32_t iters;             /* Adam iterations (>= 0)                                        */
  int32_t init;              /* 0 = BP + one exact-line-search CSI step (Sec. 3.1, Eq. 12),
                                1 = alpha0 given, 2 = zeros, 3 = alpha0 (a learned warm start)
                                unless its loss exceeds the loss at the BP + CSI start        */
  double lr, adam_b1, adam_b2, adam_eps;   /* paper: lr 1e-2; torch defaults 0.9, 0.999, 1e-8 */
  const void* alpha0;        /* device [ni][ky][kx] complex64 when init == 1 or 3              */
  const void* chi_true;      /* optional device [ny][nx] complex64: enables RelErr             */
  int32_t apply_cco;         /* 1 = post-process chi-hat with the CCO (Sec. 2.4)               */
  int32_t cco_radius;        /* guided-filter box radius (default 2)                           */
  double cco_eps;            /* guided-filter regulariser (default 1e-2)                       */
  double cco_eta_max, cco_tau, cco_delta;  /* Eq. (11): 0.1, 3, 0.5                            */
  int32_t use_graph;         /* how the iteration loop runs (results agree to FP32 rounding):
                                0 = one launch per kernel; 1 = a CUDA graph of the kernels;
                                2 = one persistent cooperative launch for the whole loop;
                                3 = one cooperative launch of thread-block clusters, one cluster
                                per incidence, for the whole loop (default).  2 and 3 need the
                                register-FFT path in FP32 with square padding (3: padding <= 128
                                and Ni * cluster size <= SM count); otherwise the graph runs     */
  int32_t history_every;     /* > 0: every n iterations write a row of 8 doubles to history: the
                                6 loss terms, RelErr of chi-hat and of its CCO image (NaN-free
                                only with chi_true; the loop then runs without a CUDA graph)    */
  double* history;           /* device [ceil(iters / history_every)][8] when history_every > 0 */
  /* Coefficient-correcting network (Sec. 3, network architecture; training settings): with
   * fcnn_hidden = H > 0 the solve optimises the weights theta of a fully connected network that maps
   * each incidence's initial coefficients to a correction, alpha = alpha_(0) + Delta alpha(theta),
   * with Adam (lr, betas, eps above) on theta instead of on alpha.  Per incidence p the input is
   * x_p = s [Re alpha_(0),p, Im alpha_(0),p] (D = 2 ky kx reals, s = 1 / RMS of alpha_(0)'s real
   * components), two hidden layers of width H with ReLU, a linear output y_p of D reals, and
   * Delta alpha_p = (y_p[0 .. ky kx) + i y_p[ky kx .. D)) / s; one network for all incidences.
   * fcnn_params0: device float32, caller-owned, read at the start of the solve: W1 [H][D], b1 [H],
   * W2 [H][H], b2 [H], W3 [D][H], b3 [D], row-major, concatenated.  1 <= H <= 4096.  With
   * use_graph 3 and H <= 512 the loop runs inside the cluster launch where the grid qualifies for
   * it (forward pass and chain rule per incidence in each cluster, the weight gradient and Adam in
   * slices over the grid between two grid barriers per iteration); otherwise as the CUDA graph
   * (use_graph 1..3) or one launch per kernel (0).  alpha_out receives alpha-hat at the final
   * weights. */
  int32_t fcnn_hidden;       /* 0 = off (Adam on alpha) */
  const void* fcnn_params0;
  /* Cap, in SM clock cycles, on each grid-barrier wait of the one-launch loop forms (use_graph 2
   * and 3); 0 = the default 2^31 (about one second).  A wait that reaches the cap makes the solve
   * return PDF_ETIMEOUT instead of waiting on.  A small positive value exists for testing that
   * path: the first CTA to reach a barrier then gives up at once. */
  int64_t barrier_wait_cycles;
} pdf_solve_opts;

typedef struct pdf_solve_report {
  int32_t iters_run;
  int32_t nonfinite;         /* 1 if a loss term was NaN/Inf at the end                        */
  double terms[6];           /* loss terms at the final alpha                                  */
  double relerr;             /* ||chi - chi_true|| / ||chi_true|| before CCO (NaN without truth) */
  double relerr_cco;         /* same after CCO                                                 */
  int32_t used_warm_start;   /* init == 3: 1 if alpha0 was kept, 0 if BP + CSI was used        */
  int32_t loop_mode;         /* the loop form that ran (see use_graph): 0, 1, 2 or 3           */
} pdf_solve_report;

void pdf_solve_opts_default(pdf_solve_opts* o);

/* Whole reconstruction on `stream`.  chi_out [ny][nx] (device, may be NULL) receives chi-hat
 * after the CCO when apply_cco, else chi-hat; chi_raw_out the chi-hat before CCO (may be NULL);
 * alpha_out [ni][ky][kx] the final coefficients (may be NULL); report (host, may be NULL) is
 * filled when given.  The call synchronises `stream` before it returns, to read the solve's
 * device-side status:
 *   PDF_ETIMEOUT      a grid barrier of the one-launch loop (use_graph 2 or 3) ran out of time
 *                     (see barrier_wait_cycles); the outputs are not meaningful;
 *   PDF_ENONFINITE    the reconstructed contrast, or with a report a final loss term, is NaN/Inf
 *                     (for example from a non-finite alpha0); the outputs are written as computed.
 * When the cluster loop (use_graph 3) is launched but its thread-block clusters do not come up
 * with the shape it was launched with (a tool that serialises or replays launches can do this),
 * the kernel returns without touching any state, and the same iterations run again as the CUDA
 * graph of the stand-alone kernels; report->loop_mode then says 1. */
pdf_status pdf_solve(pdf_problem* h, const pdf_solve_opts* opts, void* chi_out, void* chi_raw_out,
                     void* alpha_out, pdf_solve_report* report, void* stream);

/* Forward scattering solve on the device (Eq. 3-5): (I - G_D diag(chi)) E_tot = E_inc by
 * BiCGSTAB with the FFT-applied G_D, then E_sca = G_S chi E_tot.  chi [ny][nx] device
 * complex64, esca_out [ni][nr] device complex64, j_out [ni][ny][nx] (may be NULL).  Synchronises
 * `stream` (convergence is checked on the host).  tol: relative residual; max_iter: cap.
 * Returns PDF_ETIMEOUT if the iteration cap is reached before tol. */
pdf_status pdf_forward(pdf_problem* h, const void* chi, void* esca_out, void* j_out, double tol,
                       int32_t max_iter, int32_t* iters_out, void* stream);

/* Profiling: runs pdf_loss_grad once to warm up, then `reps` times with a CUDA event between
 * consecutive kernels on `stream`, and writes the mean milliseconds of kernel k (in launch
 * order) to ms[k].  Returns the number of kernels K (ms needs n >= K entries) or a negative
 * pdf_status.  Synchronises `stream`.  Does not write a gradient or loss terms for the caller. */
int32_t pdf_profile_loss_grad(pdf_problem* h, const void* alpha, int32_t reps, float* ms, int32_t n,
                              void* stream);

/* Measured FP32 FMA throughput of the current device, the denominator of the "alu" roofline of
 * the cluster loop: a kernel of independent fmaf chains filling every SM (occupancy-sized grid,
 * ~1 ms a launch) runs once to warm up and then `reps` times between two CUDA events on
 * `stream`; *tflops = 2 x FMAs / elapsed time, in TFLOP/s.  Synchronises `stream`.  Errors:
 * PDF_EINVAL (reps < 1 or tflops NULL), PDF_ECUDA. */
pdf_status pdf_fp32_fma_peak(int32_t reps, double* tflops, void* stream);

/* Name of kernel k of pdf_loss_grad in launch order ("" when out of range), FP32 path with the
 * folded data term (fold_gs = 1) as separate kernels; pdf_stage_name gives a handle's actual
 * stages (where the tiled synthesis applies, the data residual is formed inside it). */
const char* pdf_kernel_name(int32_t k);

/* Name of profiled stage k of pdf_loss_grad for this handle's precision (with precision = 1
 * some stages group a tensor-core GEMM with its operand packing). */
const char* pdf_stage_name(pdf_problem* h, int32_t k);

/* Phase timestamps of the cluster loop (use_graph = 3), for libraries built with the compile
 * definition PDF_PHASE_STAMPS only: out[4][20] receives the global-timer readings (ns) that
 * thread 0 of the first CTA took after each barrier of iterations 5..8 of the last cluster
 * solve (marks 0-14 the loss and gradient steps; with the coefficient-correcting network also
 * 16 after its forward pass, 15 after the chain rule's grid barrier and 17 after the Adam step
 * on its weights; unused marks hold stale values).  Synchronises the device.  PDF_EUNSUPPORTED
 * in ordinary builds, whose kernels carry no marks. */
pdf_status pdf_phase_stamps(uint64_t* out);

/* The cluster sizes the cluster loop (use_graph = 3) would consider for this handle (16, 8, 6, 4, 2:
 * at most 5 rows; C need not divide the grid, the last CTA then owns fewer rows or columns), in
 * order of preference: for each, out[4 i + 0..3] = cluster size C, shared-memory bytes per CTA, how many
 * such clusters the device can hold at once (-1 when the plan exceeds the shared-memory limit or
 * the query failed), and 1 when all ni clusters fit (the solve takes the first such row).
 * Returns the number of rows (0: the problem does not qualify; the graph loop runs) or a
 * negative pdf_status.  Makes no launch. */
int32_t pdf_cluster_plan(pdf_problem* h, int32_t* out, int32_t nmax);

/* G_S x without any device allocation, for callers that cannot call cudaMalloc: code whose
 * device memory is already owned by another allocator (a host framework's caching allocator
 * that has reserved the GPU), or latency-critical loops where an allocation, which can
 * synchronise the device, is not acceptable.  The paper has no counterpart: this is the
 * handle-free form of PDF_OP_GS.
 *   gs  [nr][m] complex64, device: the receiver operator (for example conj of PDF_OP_GSH applied
 *       to an identity);  x [ni][m] complex64, device;  out [ni][nr] complex64, device, overwritten
 *       with out[p][r] = sum_n gs[r][n] x[p][n].
 * Its split-K partial sums live in a 4 MiB file-scope device array that every GPU loading the
 * library holds until exit.  The first call on a device looks the array's address up
 * (cudaGetSymbolAddress) with that device current; make that first call before any stream
 * capture.  All calls share the array, so calls that overlap on the GPU race.  Nothing is
 * allocated or freed.  Errors: PDF_EINVAL for NULL pointers, sizes < 1, or ni * nr above 524288
 * (the array's capacity in complex64); PDF_ECUDA if the address look-up or a launch fails.
 * Asynchronous on `stream`. */
pdf_status pdf_gs_apply_static(const void* gs, const void* x, void* out, int32_t ni, int32_t nr, int32_t m,
                               void* stream);

/* ---------------------------------------------------------------------------------------------
 * Learned warm start (not in the paper): a fully connected network with ReLU hidden layers,
 * BF16 tensor-core products with FP32 accumulation and FP32 master weights, trained with the
 * mean squared error and Adam (torch.optim.Adam arithmetic, betas 0.9/0.999, eps 1e-8).
 * Arrays are device float32, row-major: X [B][sizes[0]], T and Y [B][sizes[nlayers]],
 * W [out][in] and b [out] of each layer (host float32 for set/get).  Every call is
 * asynchronous on `stream` except set/get_params, which synchronise.
 * --------------------------------------------------------------------------------------------- */
typedef struct pdf_mlp pdf_mlp;

/* nlayers (1..8) linear layers, sizes[0..nlayers] the widths (1..2^20, each weight matrix and each
 * batch_max x width activation below 2^31 elements); batch_max <= 4096.  Weights start at 0:
 * set them with pdf_mlp_set_params.  PDF_EINVAL on bad sizes, PDF_ENOMEM. */
pdf_status pdf_mlp_create(int32_t nlayers, const int32_t* sizes, int32_t batch_max, pdf_mlp** out);
void pdf_mlp_destroy(pdf_mlp* m);
/* Copies host W [out][in] and b [out] of `layer` in and resets its Adam state and the step count. */
pdf_status pdf_mlp_set_params(pdf_mlp* m, int32_t layer, const float* W, const float* b, void* stream);
/* Copies the master weights and the last gradients of `layer` to host arrays (any may be NULL). */
pdf_status pdf_mlp_get_params(pdf_mlp* m, int32_t layer, float* W, float* b, float* dW, float* db, void* stream);
/* Y = network(X) for B <= batch_max rows. */
pdf_status pdf_mlp_forward(pdf_mlp* m, const float* X, float* Y, int32_t B, void* stream);
/* Gradients of mean((Y - T)^2) with respect to all weights (kept in the handle, see get_params);
 * loss: device double (may be NULL). */
pdf_status pdf_mlp_loss_grad(pdf_mlp* m, const float* X, const float* T, int32_t B, double* loss, void* stream);
/* pdf_mlp_loss_grad followed by one Adam step with learning rate lr on every layer. */
pdf_status pdf_mlp_train_step(pdf_mlp* m, const float* X, const float* T, int32_t B, double lr, double* loss,
                              void* stream);
/* 1 if a tensor-core wait timed out in an earlier call, 0 otherwise (synchronises). */
int32_t pdf_mlp_error_flag(pdf_mlp* m);
/* The network's input for B scenes: esca [B][n] complex64 (n = ni nr, each scene's measured field,
 * device) -> X [B][2 n] float32 (device), X[b][2 i + c] = (Re, Im) of esca[b][i] divided by the
 * scene's RMS magnitude ||esca[b]|| / sqrt(n) (unscaled when the field is zero).  Errors:
 * PDF_EINVAL for NULL pointers or sizes < 1. */
pdf_status pdf_mlp_features(const void* esca, int32_t B, int32_t n, float* X, void* stream);

/* Number of kernels this library has launched in the calling process (graph launches count
 * every kernel node they execute).  For benchmarking evidence. */
uint64_t pdf_launch_count(void);

/* Frees the handle and its workspace (synchronises the device work of the handle first). */
void pdf_destroy(pdf_problem* h);

/* Message of the last failed call on this thread ("" if none). */
const char* pdf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PDF_H */
