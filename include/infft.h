/*
 * infft.h -- C ABI of the GB300 direct inverse NFFT (overdetermined case).
 *
 * Method: Kircheis & Potts, "Direct inversion of the nonequispaced fast Fourier
 * transform", Sec. 3.2.2.  Given N nodes x_j in [-1/2, 1/2) and samples
 * f_j = f(x_j) of a trigonometric polynomial of degree M (eq:trig_polynomial),
 * the Fourier coefficients are approximated by a modified adjoint NFFT
 *
 *     fhat ~ D^* F^* B_opt^* f                               (eq:approx_ansatz2)
 *
 * where B_opt is the (2m+1)-sparse real matrix whose column l solves the
 * least-squares problem min ||L_l b - e_l|| (eq:opt_ansatz2 .. eq:solution_ansatz2)
 * with the Dirichlet choice of Remark remark:Dirichlet_ansatz2.
 *
 * Conventions used by every entry point:
 *   - Frequencies k = -M/2 .. M/2-1 are stored at index k + M/2.
 *   - Grid points l = -M_sigma/2 .. M_sigma/2-1 (M_sigma = sigma*M) at l + M_sigma/2.
 *   - Complex arrays are interleaved (re, im) float pairs (complex64), i.e. a
 *     length-n complex array is 2n floats; double-complex arrays likewise.
 *   - Array pointers may be host or device memory unless stated otherwise; the
 *     library detects which (cudaPointerGetAttributes) and stages host data
 *     through plan-owned device buffers.  Device pointers must be on the plan's
 *     device and 8-byte aligned (16 for double complex).
 *   - `stream` is a CUDA stream handle (cudaStream_t); NULL means the legacy
 *     default stream.  All device work is enqueued on it; calls return before
 *     it finishes unless stated otherwise.  Results in device memory are valid
 *     once the stream has reached the call; results written to HOST memory are
 *     valid when the call returns.
 *   - Every entry point returns an infft_status.  On failure nothing further
 *     is enqueued and infft_last_error() describes the failure (thread-local).
 *   - A plan is not thread-safe: calls on one plan must be serialised by the
 *     caller, and at most one stream should use a plan at a time.
 *
 * There is no CPU fallback: every step runs in CUDA kernels for sm_103a.
 */
#ifndef INFFT_GB300_H
#define INFFT_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque plan: owns a copy of the nodes, the sparsity pattern, the weights
 * of B_opt and every work buffer.  Created by infft_plan / infft_plan_create,
 * released by plan_destroy. */
typedef struct infft_plan_s* infft_plan_t;

/* Same layout as cudaStream_t (a pointer to the driver's stream object). */
typedef struct CUstream_st* infft_stream_t;

typedef enum {
    INFFT_OK = 0,
    INFFT_EINVAL = 1,        /* invalid argument (sizes, sigma, m, nodes, NULL pointers) */
    INFFT_ENOMEM = 2,        /* device or pinned-host allocation failed */
    INFFT_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    INFFT_ENOTREADY = 4,     /* apply before set_nodes/precompute */
    INFFT_EUNSUPPORTED = 5,  /* valid by the paper but not built here (e.g. a column too large) */
    INFFT_ENUMERIC = 6       /* precompute finished but some columns needed the fallback */
} infft_status;

/* Kernel choice of Remark remark:Dirichlet_ansatz2 (w_hat(k) = 1 on the kept
 * frequencies, D = diag(c_k / M_sigma), eq:matrix_D):
 *   INFFT_KERNEL_FULL: all k = -M/2 .. M/2-1 kept (default);
 *   INFFT_KERNEL_SYM : the remark's literal choice, D's k = -M/2 entry set to 0. */
enum { INFFT_KERNEL_FULL = 0, INFFT_KERNEL_SYM = 1 };

/* Which optimisation fills B (Sec. 3.2): the overdetermined case (Sec. 3.2.2, one
 * least-squares problem per grid point l, fhat = D^* F^* B_opt^* f, the default) or the
 * underdetermined case (Sec. 3.2.1, one problem per node x_j,
 * min ||K_j b - M e_j|| with K_j = A D^* T_j (eq:matrix_Kj), fhat = (1/M) D^* F^* B_opt^* f,
 * eq:approx_ansatz1). */
enum { INFFT_ANSATZ_UNDERDETERMINED = 1, INFFT_ANSATZ_OVERDETERMINED = 2 };

/* Diagnostic counters of a plan (infft_get_info synchronises the plan's last stream). */
typedef struct {
    int64_t M, N, M_sigma;
    int32_t m, kernel;
    double sigma, tau;
    int64_t nnz;             /* sum over l of |I(l)|, eq:set_l */
    int32_t max_column;      /* max |I(l)| */
    int32_t empty_columns;   /* columns with I(l) empty (b_l empty, J_l = 1) */
    int32_t bad_nodes;       /* device-checked nodes that were not finite or not in [-1/2, 1/2) */
    int32_t fallback_columns;/* columns whose Cholesky needed a larger regularisation */
    int32_t unsupported_columns; /* columns larger than the largest solver tier */
    int32_t nodes_set;       /* 1 once infft_set_nodes ran */
    int32_t precomputed;     /* 1 once infft_precompute ran after the last set_nodes */
    double objective;        /* overdetermined: sum_l J_l = ||F D A^* B_opt - I||_F^2 (eq:matrixnorm_opt_ansatz2
                              * squared); underdetermined: sum_j J_j = ||A D^* F^* B_opt^* - M I_N||_F^2
                              * (eq:matrixnorm_opt_ansatz1 squared) */
    int32_t grad_failed_columns; /* columns the last infft_grad_nodes could not factor (terms set to 0) */
    int32_t ansatz;          /* INFFT_ANSATZ_OVERDETERMINED or INFFT_ANSATZ_UNDERDETERMINED */
} infft_info;

/* ---- the five calls of the method ------------------------------------- */

/* Creates a plan for M coefficients (M even, >= 2), N >= 1 nodes x (fp64,
 * length N, host or device, each in [-1/2, 1/2), eq:trig_polynomial), oversampling
 * sigma >= 1 with M_sigma = sigma*M an even integer (Sec. 2.1) and cut-off m >= 1
 * with 2m < M_sigma (eq:set_l); kernel FULL, tau = 1e-12.  Runs the pattern step
 * (infft_set_nodes) and waits for it.  *out receives the plan (NULL on failure).
 * The caller keeps ownership of x; the plan copies it. */
infft_status infft_plan(int64_t M, int64_t N, const double* x, double sigma, int m,
                        infft_plan_t* out);

/* Fills B_opt: for every grid point l, the Tikhonov-regularised normal
 * equations (Re G_l + mu I) b_l = Re r_l of min ||L_l b - e_l||^2 over real b
 * (eq:opt_ansatz2, eq:matrix_Ll, eq:solution_ansatz2), with G_l = L_l^* L_l and
 * r_l = L_l^* e_l in closed form and mu = tau * (Re G_l)_{jj}, solved in fp64.
 * Requires infft_set_nodes.  Asynchronous on `stream`; columns that needed the
 * fallback (a larger mu) or exceed the largest solver are reported by infft_get_info. */
infft_status infft_precompute(infft_plan_t plan, infft_stream_t stream);

/* The inverse NFFT (eq:approx_ansatz2): fhat = D^* F^* B_opt^* f.
 *   f    : N complex64 samples in the caller's node order (host or device), read only;
 *   fhat : M complex64 coefficients, k = -M/2 .. M/2-1 at k + M/2 (host or device), written.
 * Steps: spreading g = B_opt^* f onto the M_sigma grid (Sec. 3.2.2), a length-M_sigma
 * FFT F^* (eq:matrix_F) keeping the M central frequencies, and the diagonal D^*
 * (eq:matrix_D) fused into the FFT's last pass.  fp32 arithmetic, fp32 accumulation.
 * Requires infft_precompute. */
infft_status infft_apply(infft_plan_t plan, const float* f, float* fhat, infft_stream_t stream);

/* infft_apply with the samples given in the plan's sorted node order: f_sorted[i] =
 * f[perm[i]] (infft_sort_values forms it; infft_copy_plan_data exports perm).  The
 * spreading then reads the samples without the permutation.  Device pointers only
 * (host pointers: INFFT_EINVAL); result as infft_apply's (the same arithmetic in the same
 * order).  Requires infft_precompute. */
infft_status infft_apply_sorted(infft_plan_t plan, const float* f_sorted, float* fhat, infft_stream_t stream);

/* f_sorted[i] = f[perm[i]], i = 0 .. N-1 (complex64, device pointers, distinct buffers):
 * the samples in the order of the plan's sorted nodes.  Requires infft_set_nodes. */
infft_status infft_sort_values(infft_plan_t plan, const float* f, float* f_sorted, infft_stream_t stream);

/* Tile shapes of the fp32 apply for 2^12 <= M_sigma <= 2^21 (two launches: the spreading
 * fused with pass A of the four-step FFT M_sigma = N1 N2, then pass B with D^*).  Shape
 * `id` spreads, per CTA, runs of `columns_per_run` consecutive grid points at N1 =
 * 2^log2_N1 positions.  All shapes compute the same fhat up to fp32 rounding.
 * infft_set_apply_config(plan, -1) restores the default rule (512 grid points per CTA
 * for m <= 6, 256 beyond); an id whose N2 = M_sigma / N1 lies outside [2^6, 2^12] returns
 * INFFT_EINVAL.  infft_get_apply_config returns the shape the next apply uses (-1 when the
 * plan's M_sigma takes the three-launch path: spreading, pass A, pass B). */
int32_t infft_apply_config_count(void);
infft_status infft_apply_config_shape(int32_t id, int32_t* log2_N1, int32_t* columns_per_run);
infft_status infft_set_apply_config(infft_plan_t plan, int32_t id);
int32_t infft_get_apply_config(infft_plan_t plan);

/* Autotuning of the tile shape: times `repeats` applies (after two untimed ones) of every
 * valid shape on the plan's own B_opt with CUDA events on `stream` (the data vector is
 * the plan's zeroed staging buffer), keeps the fastest for the plan and returns it.
 * ms_out, when not NULL, receives infft_apply_config_count() average times in ms (-1
 * for shapes not valid at this M_sigma).  Synchronises `stream`; allocates nothing.
 * Requires infft_precompute; plans on the three-launch path return INFFT_EUNSUPPORTED. */
infft_status infft_tune_apply(infft_plan_t plan, int32_t repeats, float* ms_out, int32_t* best,
                              infft_stream_t stream);

/* infft_apply for K data vectors sampled at the plan's nodes (the "fixed nodes, several
 * problems" use of the precomputed B_opt, Sec. 1 and Sec. 3.2.2), in one launch per step:
 *   f    : K x N complex64 on the device, vector k at k N (caller's node order), read only;
 *   fhat : K x M complex64 on the device, vector k at k M (k + M/2 layout), written;
 *   workspace : device memory of at least infft_apply_many_workspace(plan, K) bytes,
 *               owned by the caller (the call allocates nothing), overwritten.
 * Each vector's result agrees with infft_apply's for it to fp32 rounding (the same
 * arithmetic, in a different order: spreading tile and FFT split differ).  1 <= K <= 65535; M_sigma > 2048
 * (smaller plans: INFFT_EUNSUPPORTED); host pointers: INFFT_EINVAL.  Requires
 * infft_precompute. */
int64_t infft_apply_many_workspace(infft_plan_t plan, int64_t K);
infft_status infft_apply_many(infft_plan_t plan, int64_t K, const float* f, float* fhat, void* workspace,
                              int64_t workspace_bytes, infft_stream_t stream);

/* The modified NFFT f = B_opt F D fhat (Remark remark:ansatz2_adj), the exact
 * adjoint of infft_apply: <infft_apply(f), g> = <f, nfft_apply(g)>.
 *   fhat : M complex64 (k + M/2 layout), read;  f : N complex64 in node order, written.
 * Requires infft_precompute. */
infft_status nfft_apply(infft_plan_t plan, const float* fhat, float* f, infft_stream_t stream);

/* Releases the plan and every buffer it owns (waits for the device to finish
 * work that uses them).  NULL is accepted. */
infft_status plan_destroy(infft_plan_t plan);

/* ---- finer-grained control ------------------------------------------- */

/* Creates a plan without nodes: validates the sizes (as infft_plan), picks the
 * kernel (INFFT_KERNEL_FULL or INFFT_KERNEL_SYM) and the Tikhonov factor tau
 * (0 <= tau < 1; 1e-12 is the default reading) and allocates every device
 * buffer for the worst case nnz <= (2m+1) N, so later calls allocate nothing.
 * Requires N * (2m+1) < 2^31 and M_sigma <= 2^24.  M_sigma a power of two: every call
 * below.  Any other even M_sigma = 2M with sigma = 2 and M <= 8192 (Sec. 2.1 allows any
 * even sigma M): the plan is a batch of one problem (infft_batch_*), whose FFT is a chirp
 * convolution of power-of-two length; it supports infft_set_nodes, infft_precompute,
 * infft_apply, infft_get_info and infft_copy_plan_data, and every other call returns
 * INFFT_EUNSUPPORTED.  Other non-power-of-two sizes return INFFT_EUNSUPPORTED. */
infft_status infft_plan_create(int64_t M, int64_t N, double sigma, int m, int kernel,
                               double tau, infft_plan_t* out);

/* As infft_plan_create, with the choice of optimisation (INFFT_ANSATZ_OVERDETERMINED,
 * which infft_plan_create makes, or INFFT_ANSATZ_UNDERDETERMINED).  For the
 * underdetermined case (Sec. 3.2.1), infft_precompute solves, per node x_j, the
 * Tikhonov-regularised normal equations
 *   (Re K_j^* K_j + mu_j I) b_j = M Re(K_j^* e_j),   mu_j = tau * mean diagonal entry,
 * of min ||K_j b - M e_j||_2^2 over real b (eq:opt_ansatz1, eq:solution_ansatz1), b_j on
 * the 2m or 2m+1 grid points of I(x_j) (eq:set_xj).  Re K_j^* K_j sums over all N nodes;
 * it is formed from the node moments sum_h exp(2 pi i n x_h), |n| < M (fp64, O(N M)), and
 * one fp64 FFT of length M_sigma per offset of two grid points (2m+1 of them).  The plan
 * stores B_opt / M, so infft_apply returns (1/M) D^* F^* B_opt^* f (eq:approx_ansatz1) and
 * nfft_apply returns (1/M) B_opt F D fhat, the inverse adjoint estimate of Remark
 * remark:ansatz1_adj when fhat = A^* f.  The underdetermined case requires 2m+1 <= 17
 * (INFFT_EUNSUPPORTED otherwise) and has no infft_grad_nodes (INFFT_EUNSUPPORTED). */
infft_status infft_plan_create_ansatz(int64_t M, int64_t N, double sigma, int m, int kernel,
                                      int ansatz, double tau, infft_plan_t* out);

/* The pattern step (eq:set_l): copies x (N fp64, host or device), sorts the
 * nodes by grid cell and derives, for every grid point l, I(l) as a contiguous
 * (wrapping) range of sorted nodes.  A node belongs to I(l) iff
 * ceil(u) - m <= l <= floor(u) + m (mod M_sigma), decided exactly on
 * u = fl(M_sigma x).  Host x is validated on the host (INFFT_EINVAL); device x is
 * validated on the device and reported by infft_get_info (bad_nodes).
 * Invalidates an earlier precompute. */
infft_status infft_set_nodes(infft_plan_t plan, const double* x, infft_stream_t stream);

/* fp64 variants of the two applies (weights, spreading, FFT and accumulation in
 * fp64; double-complex arrays).  For accuracy checks against the oracle. */
infft_status infft_apply_z(infft_plan_t plan, const double* f, double* fhat, infft_stream_t stream);
infft_status nfft_apply_z(infft_plan_t plan, const double* fhat, double* f, infft_stream_t stream);

/* Gradient of a real loss L through the inverse NFFT with respect to the nodes (the
 * differentiable form; the paper has no gradient, this follows from eq:approx_ansatz2 and
 * the column problems eq:opt_ansatz2 .. eq:solution_ansatz2 by implicit differentiation,
 * with the pattern I(l) held fixed, which it is except on a set of measure zero):
 *   f      : N complex64, the data the forward infft_apply used (caller order, device);
 *   w      : M complex64, dL/dRe fhat + i dL/dIm fhat (device);
 *   grad_x : N fp64, dL/dx_j (caller order, device), written.
 * With gamma = F D w, beta_{l,i} = Re(conj(gamma_l) f_i), lambda_l = (Re G_l + mu I)^{-1} beta_l:
 *   dL/dx_j = sum_{l: j in I(l)} [-lambda_{l,j} kappa'(l/M_sigma - x_j)
 *              - lambda_{l,j} sum_k kappa'(x_j - x_k) b_{l,k} - b_{l,j} sum_i kappa'(x_j - x_i) lambda_{l,i}].
 * The gradient with respect to f is nfft_apply(w) (the exact adjoint).  Columns larger
 * than 64 nodes are not handled (their terms are 0; infft_get_info reports them).
 * Requires infft_precompute; device pointers only. */
infft_status infft_grad_nodes(infft_plan_t plan, const float* f, const float* w, double* grad_x,
                              infft_stream_t stream);

/* Synchronises the plan's last stream and fills *info. */
infft_status infft_get_info(infft_plan_t plan, infft_info* info);

/* Copies the pattern and B_opt to HOST arrays (synchronous).  Any pointer may
 * be NULL to skip it.  perm[i] = caller index of the i-th sorted node (N);
 * col_start[p] = first sorted position of I(l), col_count[p] = |I(l)| (M_sigma
 * each, p = l + M_sigma/2; the range wraps modulo N); col_offset[p] = offset of
 * column p's weights (M_sigma + 1); weights[col_offset[p] + i] = b_{l, perm[(col_start[p] + i) mod N]}
 * in fp64 (nnz); objective[p] = J_l = ||L_l b_l - e_l||^2 (M_sigma).  Underdetermined
 * plans: the weights are B_opt / M and objective[j] = J_j = ||K_j b_j - M e_j||^2 in the
 * caller's node order (N). */
infft_status infft_copy_plan_data(infft_plan_t plan, int32_t* perm, int32_t* col_start,
                                  int32_t* col_count, int32_t* col_offset, double* weights,
                                  double* objective);

/* Per-kernel device timing.  infft_profile(plan, 1) makes every later launch of
 * this plan record a CUDA event pair on its stream; infft_profile_read
 * synchronises and returns, per internal kernel, its name, launch count and
 * summed milliseconds (up to `cap` entries; *n receives the number written),
 * then clears the record.  infft_profile(plan, 0) stops recording. */
infft_status infft_profile(infft_plan_t plan, int enable);
infft_status infft_profile_read(infft_plan_t plan, int cap, const char** names,
                                int64_t* launches, double* milliseconds, int* n);

/* ---- batched problems -------------------------------------------------------
 * Many independent inversions of uneven size in one plan (the paper's "fixed
 * nodes, several problems" use of the precomputed B_opt, Sec. 1 and Sec. 3.2.2):
 * problem p has M_p coefficients and N_p nodes and is solved exactly as a plan
 * of its own would solve it (eq:approx_ansatz2, same pattern, same B_opt, same
 * D^* F^*), with sigma = 2 (M_sigma,p = 2 M_p, any even M_p in [4, 8192]; the
 * length-M_sigma DFT is evaluated by a chirp convolution, so M_p need not be a
 * power of two).  Columns with more than 224 nodes (clustered nodes) are solved
 * by a large-column solver up to 1024 nodes; larger columns are counted as
 * unsupported (b_l = 0).
 * Layout: problems back to back in the order given.  x: sum N_p fp64 nodes;
 * f: sum N_p complex64 values; fhat: sum M_p complex64 coefficients, problem p's
 * block at offset sum_{q<p} M_q in the k + M_p/2 layout.
 * The batch owns all device buffers (one arena for the members' patterns and
 * weights, staging for host f/fhat); every step runs on the caller's stream, one
 * launch per stage over all problems. */
typedef struct infft_batch_s* infft_batch_t;

typedef struct {
    int64_t P, sum_N, sum_M;
    int32_t m, nodes_set, precomputed, max_column;
    int64_t nnz;                 /* sum over problems of sum_l |I(l)| */
    int64_t empty_columns, bad_nodes;
    int64_t fallback_columns;    /* columns solved with a raised regulariser */
    int64_t unsupported_columns; /* columns above 1024 nodes (b_l = 0) */
    int64_t large_columns;       /* columns solved by the large-column solver */
    double objective;            /* sum over problems of sum_l J_l (eq:matrixnorm_opt_ansatz2) */
} infft_batch_info;

/* Creates a batch of P >= 1 problems with sizes M[p], N[p] (host arrays, P each),
 * sigma = 2 (others: INFFT_EUNSUPPORTED), cut-off m, kernel FULL or SYM and
 * regulariser tau (as infft_plan_create).  Blocks while it fills the chirp
 * transforms of the problems' DFT lengths. */
infft_status infft_batch_create(int64_t P, const int64_t* M, const int64_t* N, double sigma, int m,
                                int kernel, double tau, infft_batch_t* out);

/* The pattern step (eq:set_l) of every problem: x holds sum N_p nodes (host or
 * device, each in [-1/2, 1/2)); the batch copies them. */
infft_status infft_batch_set_nodes(infft_batch_t batch, const double* x, infft_stream_t stream);

/* B_opt of every problem (as infft_precompute, eq:opt_ansatz2 .. eq:solution_ansatz2). */
infft_status infft_batch_precompute(infft_batch_t batch, infft_stream_t stream);

/* fhat_p = D^* F^* B_opt,p^* f_p for every problem p (eq:approx_ansatz2), fp32:
 * f (sum N_p complex64) -> fhat (sum M_p complex64), host or device. */
infft_status infft_batch_apply(infft_batch_t batch, const float* f, float* fhat, infft_stream_t stream);

/* Tile shapes of the batched apply's spreading (the autotuned part).  Shape `id` cuts
 * each problem's grid into tiles of at most `cols` grid points (one thread each) whose
 * weights start within one block of `weights` entries (both powers of two).  Every
 * shape computes bit-identical fhat: each column is summed in one fixed order that
 * depends on its grid point only.  infft_batch_set_tile_shape(batch, -1) restores the
 * default (the fixed rule: 128 grid points, 2048 weights); on a precomputed batch it
 * re-cuts the tiles on `stream` (three launches), otherwise the precompute uses it.
 * Ids outside [-1, count): INFFT_EINVAL.  infft_batch_get_tile_shape returns the shape
 * the next apply uses (-1 for a NULL batch). */
int32_t infft_batch_tile_shape_count(void);
infft_status infft_batch_tile_shape(int32_t id, int32_t* cols, int32_t* weights);
infft_status infft_batch_set_tile_shape(infft_batch_t batch, int32_t id, infft_stream_t stream);
int32_t infft_batch_get_tile_shape(infft_batch_t batch);

/* Autotuning of the tile shape: times `repeats` batched applies (after two untimed ones)
 * of every shape on the batch's own B_opt with CUDA events on `stream` (the data vector
 * is the batch's zeroed staging buffer), keeps the fastest and returns its id in *best.
 * ms_out, when not NULL, receives infft_batch_tile_shape_count() average times in ms.
 * Synchronises `stream`; allocates nothing.  Requires infft_batch_precompute. */
infft_status infft_batch_tune_apply(infft_batch_t batch, int32_t repeats, float* ms_out, int32_t* best,
                                    infft_stream_t stream);

/* Synchronises the batch's last stream and fills *info (sums over problems). */
infft_status infft_batch_get_info(infft_batch_t batch, infft_batch_info* info);

/* infft_copy_plan_data for problem p of the batch (HOST arrays, synchronous). */
infft_status infft_batch_copy_problem(infft_batch_t batch, int64_t p, int32_t* perm, int32_t* col_start,
                                      int32_t* col_count, int32_t* col_offset, double* weights,
                                      double* objective);

/* Frees the batch (synchronises its device first). */
infft_status infft_batch_destroy(infft_batch_t batch);

/* ---- allocation-free entry point ------------------------------------------
 * The paper has no counterpart of this call; it exists for callers that cannot
 * allocate device memory when they call: processes whose device memory belongs
 * to their own pool allocator, or code that must not call cudaMalloc while
 * another component is recording work on the device.
 *
 * Computes the last two steps of infft_apply on a caller-provided grid:
 *   fhat_k = conj(d_k) sum_{l} grid_l exp(-2 pi i k l / M_sigma),  k = -M/2 .. M/2-1,
 * with d_k = 1/M_sigma (kernel FULL) or the same with d_{-M/2} = 0 (kernel SYM).
 *   grid : M_sigma complex64 on the device, l = -M_sigma/2 .. M_sigma/2-1 at l + M_sigma/2 (read);
 *   fhat : M complex64 on the device, k + M/2 layout (written);
 *   M even >= 2; M_sigma a power of two with max(M, 4) <= M_sigma <= 2^20 (larger sizes
 *   return INFFT_EUNSUPPORTED; host pointers return INFFT_EINVAL).
 * Allocates nothing: its scratch is one static device array of 2^20 complex64
 * (8 MiB) that every GPU loading the library holds until the process exits.  The
 * first call on a device looks up that array's device address (with the device
 * current) and later calls reuse it; make that first call before any stream
 * capture.  A call that finds a different context current on the device than the
 * one the address was taken in (after cudaDeviceReset) looks the address up again,
 * so that call, too, belongs outside a capture.
 * Every call shares the array, so calls that may overlap on the GPU (different
 * streams, or different host threads) race: serialise them.  The array needs no
 * clearing: each call overwrites every element it reads. */
infft_status infft_fft_deconv_noalloc(const float* grid, int64_t M, int64_t M_sigma, int kernel,
                                      float* fhat, infft_stream_t stream);

/* ---- diagnostics -------------------------------------------------------------
 * The paper has no counterpart of these calls.  infft_fp64_fma_probe measures what the
 * fp64-bound precompute is compared against: it launches 8 CTAs per SM of 256 threads,
 * each advancing 8 independent fp64 FMA recurrences for `iters` steps, on `stream`, and
 * stores one double per thread into `sink` (device memory, at least
 * infft_fp64_fma_probe_sink_len() doubles, owned by the caller).  *flops receives the
 * flop count of the launch (2 per FMA); time the launch with events on `stream` to get the
 * rate.  infft_fp64_fma_probe_sink_len returns -1 when no device is usable. */
infft_status infft_fp64_fma_probe(int64_t iters, double* sink, int64_t sink_len, double* flops,
                                  infft_stream_t stream);
int64_t infft_fp64_fma_probe_sink_len(void);

/* ---- two-dimensional tensor-product form ----------------------------------
 * The paper treats one dimension and leaves higher dimensions open (Sec. 5).
 * This form takes every object of Sec. 3.2.2 as the tensor product of its 1-D
 * counterpart: frequencies k = (k1, k2), k_t = -M_t/2 .. M_t/2-1; nodes
 * x_j = (x_j1, x_j2) in [-1/2, 1/2)^2; grid points l = (l1, l2) on the
 * M_sigma,1 x M_sigma,2 grid (M_sigma,t = sigma M_t); D = diag(c_k1 c_k2/(M_sigma,1 M_sigma,2))
 * with the 1-D Dirichlet choices (eq:matrix_D, Remark remark:Dirichlet_ansatz2);
 * the pattern I(l) = { j : l_t in I_t(x_jt), t = 1, 2 } (eq:set_xj per dimension, a
 * box); and per grid point the regularised real least-squares problem of
 * eq:opt_ansatz2 .. eq:solution_ansatz2, whose Gram entries are the real part of the
 * product of the two complex 1-D kernels.  fhat = D^* F^* B_opt^* f (eq:approx_ansatz2).
 * Layout: x is N (x1, x2) fp64 pairs (2N doubles); f is N complex64 (or complex128
 * for the _z call) in the caller's node order; fhat is M1 x M2 complex, k1-major:
 * (k1, k2) at (k1 + M1/2) M2 + k2 + M2/2.  Grid column p = (l1 + M_sigma,1/2) M_sigma,2 +
 * l2 + M_sigma,2/2.
 * Sizes: M_t even, M_sigma,t = sigma M_t a power of two in [4, 2048]; 1 <= m and
 * 2m < M_sigma,t; N (2m+1)^2 < 2^31.  Columns of more than 8192 nodes are
 * counted as unsupported (b_l = 0). */
typedef struct infft2d_plan_s* infft2d_plan_t;

typedef struct {
    int64_t M1, M2, M_sigma1, M_sigma2, N;
    int32_t m, kernel;
    double sigma, tau;
    int64_t nnz;                  /* sum over l of |I(l)| */
    int32_t max_column;           /* max |I(l)| */
    int32_t empty_columns;        /* columns with I(l) empty (J_l = 1) */
    int32_t bad_nodes;            /* nodes not finite or outside [-1/2, 1/2)^2 */
    int32_t fallback_columns;     /* columns whose Cholesky needed a larger regulariser */
    int32_t unsupported_columns;  /* columns above 8192 nodes (b_l = 0) */
    int32_t large_columns;        /* columns solved by the blocked solver (above 128 nodes) */
    int32_t wide_columns;         /* columns spread in float-float (||b_l||_1 > 32) */
    int32_t nodes_set, precomputed;
    double objective;             /* sum_l J_l = ||F D A^* B_opt - I||_F^2 */
    int32_t indexed_columns;      /* columns the fp32 spread reads through node indices (a node on
                                     a grid line); the others as 2m cell-row runs of sorted nodes */
} infft2d_info;

/* Creates a 2-D plan (sizes as above; kernel FULL or SYM; tau >= 0 the regulariser
 * factor).  Allocates the plan's device buffers; *out is NULL on failure. */
infft_status infft2d_plan_create(int64_t M1, int64_t M2, int64_t N, double sigma, int m, int kernel,
                                 double tau, infft2d_plan_t* out);

/* The pattern step: copies the 2N doubles of x (host or device), sorts the nodes
 * by grid cell and builds I(l) for every grid point.  Synchronises `stream` before
 * it returns (the column sizes are read back); INFFT_EINVAL if a node is not finite
 * or outside [-1/2, 1/2)^2. */
infft_status infft2d_set_nodes(infft2d_plan_t plan, const double* x, infft_stream_t stream);

/* Fills B_opt in fp64 (Cholesky of Re G_l + mu I, mu = tau Re kappa(0); a column whose
 * factorisation fails is retried with mu raised 1000-fold, twice, then set to 0 and
 * counted).  Synchronous: it reads the column-size lists back to plan its launches and
 * returns when B_opt is complete; the scratch of the columns above 128 nodes (about
 * 4 n^2 bytes per column being factored) is allocated for the call and released. */
infft_status infft2d_precompute(infft2d_plan_t plan, infft_stream_t stream);

/* fhat = D^* F^* B_opt^* f: spreading onto the grid, the 2-D FFT pruned to the
 * M1 x M2 central frequencies with D^* fused into its last pass.  fp32 arithmetic
 * and accumulation (columns with ||b_l||_1 > 32 spread in float-float on the fp32 pipe).
 * The data is first copied into sorted node order, so the spread reads each column as
 * 2m cell-row runs of consecutive nodes (no node index per entry).  f and fhat host or
 * device; with a host fhat the call returns after the result is copied. */
infft_status infft2d_apply(infft2d_plan_t plan, const float* f, float* fhat, infft_stream_t stream);
/* The same in fp64 throughout (complex128 f and fhat). */
infft_status infft2d_apply_z(infft2d_plan_t plan, const double* f, double* fhat, infft_stream_t stream);

/* Synchronises the plan's last stream and fills *info. */
infft_status infft2d_get_info(infft2d_plan_t plan, infft2d_info* info);

/* Copies the pattern and B_opt to HOST arrays (any may be NULL): col_offset
 * (P + 1 int32, P = M_sigma,1 M_sigma,2), col_node (nnz int32, caller node index of each
 * entry, column by column), weights (nnz fp64), objective (P fp64, J_l).  Synchronous. */
infft_status infft2d_copy_plan_data(infft2d_plan_t plan, int32_t* col_offset, int32_t* col_node,
                                    double* weights, double* objective);

/* Frees the plan (synchronises its device first). */
infft_status infft2d_plan_destroy(infft2d_plan_t plan);

/* ---- fp64 direct sum and residual correction ---------------------------------
 * The trigonometric polynomial at the plan's nodes by its defining sum (eq:nfft),
 *   f_j = sum_{k=-M/2}^{M/2-1} fhat_k e^{2 pi i k x_j},
 * in fp64 (exponentials by complex rotation, restarted every 32 frequencies from an exactly
 * reduced sincospi), O(N M) work.  fhat: M complex128, f: N complex128 in the caller's node
 * order, both device pointers.  Requires infft_set_nodes. */
infft_status infft_ndft_z(infft_plan_t plan, const double* fhat, double* f, infft_stream_t stream);

/* The same trigonometric polynomial by the NFFT of Sec. 2.1 (f ~ B F D fhat with a window w,
 * D = diag(1/(M_sigma w^(k)))), in fp64 with a Kaiser-Bessel window truncated to 12 grid
 * points on either side: error of order exp(-2 pi 12 sqrt(1 - 1/sigma)), below fp64 rounding for
 * sigma = 2 (measured <= 1e-13 relative against the direct sum).  O(M_sigma log M_sigma + 25 N).
 * Needs sigma >= 2 and M_sigma >= 96 (else INFFT_EUNSUPPORTED); device pointers; uses the plan's
 * grid, FFT and output-staging buffers.  Requires infft_set_nodes. */
infft_status infft_nfft_kb_z(infft_plan_t plan, const double* fhat, double* f, infft_stream_t stream);

/* Residual correction of an estimate fhat (in place), `sweeps` times (0 .. 64):
 *   fhat <- fhat + D^* F^* B_opt^* (f - A fhat)
 * with A fhat by infft_nfft_kb_z where it is supported (by infft_ndft_z otherwise) and
 * D^* F^* B_opt^* by infft_apply_z: the modified adjoint NFFT
 * (eq:approx_ansatz2) as an approximate inverse of A in a Richardson iteration for A fhat = f
 * (eq:problem_infft).  For data f = A fhat_true each sweep maps the error e to
 * (I - D^* F^* B_opt^* A) e: on jittered nodes with N = 4M an estimate accurate to ~1e-7
 * reaches ~1e-14 in one sweep.  f: N complex128, fhat: M complex128, device pointers; the
 * plan's staging buffers hold the residual and the correction (no other call on the plan
 * may run meanwhile).  Requires infft_precompute. */
infft_status infft_refine_z(infft_plan_t plan, const double* f, double* fhat, int sweeps, infft_stream_t stream);

/* Number of kernels this library has launched in the process so far. */
int64_t infft_launch_count(void);

/* Thread-local description of the last failure on this thread ("" if none). */
const char* infft_last_error(void);

/* Library version string. */
const char* infft_version(void);

#ifdef __cplusplus
}
#endif
#endif /* INFFT_GB300_H */
