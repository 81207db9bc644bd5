/*
 * chem.h -- C ABI of the GB300 per-cell chemistry library (libchem.so).
 *
 * The hot path of the reactive-flow framework of the paper: advancing every cell's
 * constant-pressure reactor over one CFD time step (§2: finite-rate chemistry, integrated on the
 * CPU with CVODE in the paper; §3.1: the chemistry step of the GPU solver's time loop), an MLP
 * surrogate of that step (§2, §3.1: DNN inference on the GPU), and a serving loop that batches
 * chemistry requests from many flow solvers.
 *
 * Conventions (every entry point):
 *   - Return CHEM_OK (0) on success, a negative CHEM_E* code on failure; chem_last_error()
 *     returns a thread-local message describing the last failure.  No C++ exception crosses
 *     this boundary.
 *   - State arrays are DEVICE pointers owned by the caller, FP64, species-major SoA:
 *       T[ncells], p[ncells] (dyn/cm^2), Y[k * ld + i] for species k and cell i, ld >= ncells.
 *     Units are CHEMKIN cgs (K, dyn/cm^2, s).
 *   - Work is enqueued on `stream` (a cudaStream_t passed as void*, NULL = legacy default
 *     stream) and runs asynchronously; pointers must stay valid until the stream reaches it.
 *     Per-cell outcomes are written to the optional status array (CHEM_CELL_* codes).
 *   - The library owns the device copies of mechanisms and models, and draws per-call
 *     temporaries from the CUDA stream-ordered allocator (cudaMallocAsync / cudaFreeAsync on
 *     `stream`), the allocation strategy of §3.2.
 */
#ifndef CHEM_H
#define CHEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  CHEM_OK = 0,
  CHEM_WCELLS = 1,      /* some cells finished with a non-OK status (synchronous calls only) */
  CHEM_EINVAL = -1,     /* invalid argument */
  CHEM_ENOMEM = -2,     /* device or host allocation failed */
  CHEM_ECUDA = -3,      /* a CUDA runtime call failed */
  CHEM_EBUSY = -4,      /* request can never be admitted (larger than the memory budget) */
  CHEM_ETIMEOUT = -5,   /* a wait ran out of time */
  CHEM_ENOTFOUND = -6   /* unknown handle or id */
};

/* per-cell status written by the integrator */
enum {
  CHEM_CELL_OK = 0,
  CHEM_CELL_MAX_STEPS = 1,    /* step-attempt limit reached; last accepted state kept */
  CHEM_CELL_H_UNDERFLOW = 2,  /* step size fell below 1e-12 dt; last accepted state kept */
  CHEM_CELL_NONFINITE = 3,    /* non-finite input (or T <= 0, p <= 0); cell left unchanged */
  CHEM_CELL_SINGULAR_LU = 4   /* exactly zero pivot in the iteration matrix */
};

typedef void* chem_stream_t;                 /* cudaStream_t */
typedef struct chem_mech_s* chem_mech_t;
typedef struct chem_model_s* chem_model_t;
typedef struct chem_server_s* chem_server_t;

/* ---------------------------------------------------------------------------------------
 * Mechanisms (NASA-7 thermo, Arrhenius / third-body / Troe kinetics; §2 names Cantera as the
 * source of these models).
 * ------------------------------------------------------------------------------------- */

/* Host-side description of a mechanism.  All arrays are host pointers, row-major, read during
 * the call only.  Reactions list up to three species per side (-1 padded; a species appearing
 * twice is listed twice).  rtype: 0 plain, 1 third-body, 2 Troe fall-off.  Ea and Ea0 in
 * cal/mol, A in cgs units.  troe[j] = (A0, b0, Ea0, a, T3, T1, T2), has_t2[j] selects the T2
 * term.  eff[j * ns + k] is the collision efficiency of species k in reaction j (types 1, 2). */
typedef struct chem_mech_desc {
  int32_t n_species, n_elements, n_reactions;
  const double* elem_mass;   /* [ne]  g/mol */
  const int32_t* comp;       /* [ns * ne] atoms of each element in each species */
  const double* nasa_lo;     /* [ns * 7] coefficients for T < 1000 K */
  const double* nasa_hi;     /* [ns * 7] coefficients for T >= 1000 K */
  const int32_t* rtype;      /* [nr] */
  const int32_t* reac;       /* [nr * 3] */
  const int32_t* prod;       /* [nr * 3] */
  const double* A;           /* [nr] */
  const double* b;           /* [nr] */
  const double* Ea;          /* [nr] */
  const double* troe;        /* [nr * 7] */
  const int32_t* has_t2;     /* [nr] */
  const double* eff;         /* [nr * ns] */
} chem_mech_desc;

/* Parse a CHEMMECH text file (format written by synth.mechanism.Mechanism.to_text) and upload
 * it to the current device.  *out receives a handle owned by the caller (chem_free_mechanism).
 * CHEM_ENOTFOUND if the file cannot be opened; CHEM_EINVAL if it does not parse or fails the checks
 * of chem_load_mechanism_desc; CHEM_ECUDA / CHEM_ENOMEM if the upload fails. */
int chem_load_mechanism(const char* path, chem_mech_t* out);
/* Same from an in-memory description.  The description is checked on the host before any device
 * work; CHEM_EINVAL (with the offending species or reaction in chem_last_error) for sizes out of
 * range (1 <= ns <= 4096, 1 <= ne <= 64, 0 <= nr <= 30000), a NULL array, a non-positive or
 * non-finite atomic mass, a negative element count, a species of non-positive molar mass,
 * non-finite NASA coefficients, a reaction type outside 0..2, a species index outside [-1, ns),
 * an empty side, A < 0 or non-finite b / Ea, a negative or non-finite third-body efficiency, or
 * Troe parameters that are non-finite, have A0 < 0, T3 <= 0 or T1 <= 0, or has_t2 outside
 * {0, 1}.  CHEM_ECUDA / CHEM_ENOMEM if the upload fails. */
int chem_load_mechanism_desc(const chem_mech_desc* desc, chem_mech_t* out);
/* Release a mechanism's device copy (cudaFree, which waits for device work still using it); the
 * handle is invalid afterwards.  CHEM_EINVAL for NULL. */
int chem_free_mechanism(chem_mech_t m);
/* Species, reaction and element counts of a loaded mechanism (host ints, each nullable).
 * CHEM_EINVAL for a NULL handle; no device work. */
int chem_mechanism_info(chem_mech_t m, int* n_species, int* n_reactions, int* n_elements);

/* ---------------------------------------------------------------------------------------
 * FP64 integrator: each cell is an adiabatic constant-pressure reactor, dY_k/dt =
 * W_k wdot_k / rho, dT/dt = -sum_k h_k wdot_k / (rho cp), advanced over [0, dt] with the
 * L-stable Rosenbrock method Rodas4 (Hairer & Wanner §IV.7), an analytic Jacobian and a dense
 * LU with partial pivoting per sub-step; adaptive sub-steps from h0 = dt with the weighted RMS
 * error norm sc_i = atol + rtol max(|y_i|, |y_new_i|) over (T, Y).
 * ------------------------------------------------------------------------------------- */

typedef struct chem_options {
  int32_t max_steps;      /* step attempts per cell before CHEM_CELL_MAX_STEPS; 0 -> 100000 */
  int32_t group_threads;  /* threads per cell: 0 auto (2 if ns+1 <= 16 else 128); 2, 4, 8, 16, 32, 64, 128, 256 */
  int32_t groups_per_cta; /* 0 auto (as many as shared memory holds) */
  int32_t max_ctas;       /* 0 auto (SM count x resident CTAs per SM) */
} chem_options;
/* With groups_per_cta and max_ctas both 0, a launch whose cells fill fewer groups than the grid
 * holds is spread over every SM with fewer groups per CTA.  A cell's result does not depend on
 * the launch shape (bitwise); it does depend on group_threads (the order of the group's sums). */

/* Advance ncells cells in place over dt.  ld = ncells.  Asynchronous on stream.
 * CHEM_EINVAL if ncells < 0, dt <= 0, rtol <= 0, atol <= 0 or a required pointer is NULL;
 * ncells == 0 is a no-op.  CHEM_ENOMEM / CHEM_ECUDA if the stream-ordered allocator cannot provide
 * the 8-byte work-queue counter or the launch fails; per-cell failures go to the status codes of
 * chem_advance_ex, not to the return value. */
int chem_advance(chem_mech_t m, double* T, const double* p, double* Y, double dt,
                 int64_t ncells, double rtol, double atol, chem_stream_t stream);

/* Extended form.  idx (device, nullable): advance only cells idx[0..ncells) of arrays whose
 * leading dimension is ld (indexed mode, used for surrogate fallback); otherwise cells
 * [0, ncells).  The indices must be distinct and lie in [0, ld): they live on the device and are
 * not checked (an index outside is an out-of-bounds device access, a repeated one a data race).
 * status (int8), nsub (accepted sub-steps), nrej (rejected attempts): device arrays indexed like
 * the cells they describe (by idx[c] in indexed mode), each nullable.  opt nullable
 * (defaults).
 * The errors of chem_advance (ld < ncells only without idx), and CHEM_EINVAL for options the
 * integrator cannot run: group_threads other than 0, 2, 4, ..., 256, or a mechanism too large for
 * the launch's shared memory. */
int chem_advance_ex(chem_mech_t m, double* T, const double* p, double* Y, int64_t ld,
                    double dt, int64_t ncells, double rtol, double atol, const int32_t* idx,
                    int8_t* status, int32_t* nsub, int32_t* nrej, const chem_options* opt,
                    chem_stream_t stream);

/* One set of cells for chem_advance_batch: device state arrays (as for chem_advance_ex), its
 * own step and tolerances, optional index list and outputs. */
typedef struct chem_segment {
  double* T;
  const double* p;
  double* Y;
  int64_t ld, ncells;
  const int32_t* idx;        /* nullable: cells idx[0..ncells), distinct and in [0, ld) (unchecked) */
  int8_t* status;            /* nullable outputs, as for chem_advance_ex */
  int32_t* nsub;
  int32_t* nrej;
  double dt, rtol, atol;
} chem_segment;

/* Advance several independent segments (different solvers' states, steps and tolerances) in one
 * persistent launch: their 8-cell chunks share one work queue, so small requests fill the GPU
 * together (iteration-level batching, used by the serving loop).  segs is a host array read
 * during the call; the call returns once the descriptors are on the device (it synchronises
 * the stream).
 * CHEM_EINVAL for a NULL mechanism or segment list, nseg < 1, or a segment with arguments
 * chem_advance rejects. */
int chem_advance_batch(chem_mech_t m, const chem_segment* segs, int nseg, chem_stream_t stream);

/* Allocation-free form of chem_advance_ex (cells [0, ncells), default options).  It calls no
 * device allocator: the only scratch a launch needs, the 8-byte counter of the kernel's work
 * queue, lives in a 256-byte file-scope __device__ array inside the library (held by every GPU
 * that loads the library until the process exits), so callers that may not allocate device
 * memory -- a flow solver that already owns the device memory through its own pools, code under
 * a hard allocation budget, a latency-critical loop that must not enter the allocator -- can
 * still advance their cells.  The caller passes all inputs and outputs as for chem_advance_ex.
 * The first call on each device (and the first after a context reset, which moves the array)
 * looks up the array's device address (cudaGetSymbolAddress) and must therefore happen outside
 * any stream capture; the look-up is safe from several host threads.  All calls share the array
 * and the counter is reset at the start of each call: calls whose work overlaps on the GPU race
 * and must be serialised by the caller (one stream, or events).  What such a race does: the
 * later call resets the counter while the earlier call's kernel is still claiming chunks, so the
 * earlier call claims chunks again; its cells are then advanced twice (over 2 dt) or written
 * twice and still report CHEM_CELL_OK.  Nothing detects or reports it: the results are silently
 * wrong.  The scratch does not grow with ncells.
 * The paper has no counterpart of this entry point.
 * The errors of chem_advance_ex. */
int chem_advance_noalloc(chem_mech_t m, double* T, const double* p, double* Y, int64_t ld,
                         double dt, int64_t ncells, double rtol, double atol, int8_t* status,
                         int32_t* nsub, int32_t* nrej, chem_stream_t stream);

/* Right-hand side f[i * ld + c] (i = 0 is dT/dt, i = 1 + k is dY_k/dt) and, if J is non-NULL,
 * the analytic Jacobian J[(i * N + j) * ld + c] = df_i/dy_j (N = ns + 1) of every cell, computed
 * by the same device code the integrator uses.  Device pointers; asynchronous.
 * CHEM_EINVAL for a NULL mechanism, ncells < 0, ld < ncells, or (ncells > 0) a NULL T, p, Y or f. */
int chem_eval_rhs_jac(chem_mech_t m, const double* T, const double* p, const double* Y,
                      int64_t ld, int64_t ncells, double* f, double* J, chem_stream_t stream);

/* ---------------------------------------------------------------------------------------
 * BF16 MLP surrogate of the chemistry step (§2: the paper replaces CVODE by per-species DNNs
 * run on the GPU; here one network maps the state to the step's composition change).
 * Inputs x = [T, ln p, BC(Y_k)] with BC(y) = (y^0.1 - 1)/0.1, z-scored; outputs the z-scored
 * increment of BC(Y_k) over the training step dt; hidden width 512, 4 GELU layers, BF16
 * weights and activations, FP32 accumulation on tcgen05 tensor cores.
 * ------------------------------------------------------------------------------------- */
typedef struct chem_surrogate_desc {
  int32_t n_species;         /* ns (<= 16); inputs nin = ns + 2 */
  int32_t hidden;            /* must be 512 */
  double dt;                 /* step the network was trained for (s) */
  const float* W[5];         /* host, row-major [out x in]: [512 x nin], 3 x [512 x 512], [ns x 512] */
  const float* b[5];         /* host: [512] x 4, [ns] */
  const float* x_mean;       /* [nin] feature mean and standard deviation */
  const float* x_std;
  const float* y_mean;       /* [ns] output mean and standard deviation; y_std = 0 marks a species
                                the step leaves unchanged (an inert one): its increment is 0 */
  const float* y_std;
  const float* box_lo;       /* [nin] training box of the raw features (trust region) */
  const float* box_hi;
} chem_surrogate_desc;

/* Upload a surrogate for use with mechanism m on the current device.  Hidden and output weights
 * are rounded to BF16; the first layer is compensated: its weights and input features are each
 * split into a BF16 pair (hi + lo) and the product keeps the hi*hi, hi*lo and lo*hi terms, about
 * 16 significant bits, because the rates depend exponentially on the temperature feature.
 * CHEM_EINVAL for NULL arguments, weights, biases or statistics, ns different from the mechanism's
 * or above 16, hidden other than 512, or dt <= 0; CHEM_ENOMEM / CHEM_ECUDA if the upload fails. */
int chem_surrogate_create(const chem_surrogate_desc* desc, chem_mech_t m, chem_model_t* out);
/* The paper's own surrogate variant (§2): one network per species, each nin -> h1 -> h2 -> h3 -> 1
 * with GELU (the paper's widths are 1600, 800, 400), on the same features, normalisation and
 * trust box as the single network.  A species with W[k][0..3] all NULL has no network and keeps
 * its mass fraction through the network pass (an inert species, y_std[k] = 0); the others need
 * all four layers.  Weights are host row-major [out x in]: W[k][0] [h1 x nin], W[k][1] [h2 x h1],
 * W[k][2] [h3 x h2], W[k][3] [1 x h3]; biases b[k][l] of the layer's output width.  The first
 * layer is compensated as in the single network; the others are rounded to BF16.  The networks
 * run layer by layer on the tcgen05 GEMM (bias, GELU and BF16 rounding in its epilogue);
 * chem_surrogate_forward and chem_surrogate_advance accept either kind of model. */
typedef struct chem_surrogate_ps_desc {
  int32_t n_species;         /* ns (<= 16) */
  int32_t hidden[3];         /* h1, h2, h3: multiples of 8 in [128, 8192] */
  double dt;                 /* step the networks were trained for (s) */
  const float* W[16][4];     /* per species k < ns, see above */
  const float* b[16][4];
  const float* x_mean;       /* as chem_surrogate_desc */
  const float* x_std;
  const float* y_mean;
  const float* y_std;
  const float* box_lo;
  const float* box_hi;
} chem_surrogate_ps_desc;
/* Copy the per-species networks (host arrays, read during the call) to the device, bound to
 * mechanism m.  *out receives a handle owned by the caller (chem_surrogate_free).  CHEM_EINVAL
 * for NULL arguments or statistics, ns different from the mechanism's or above 16, widths outside
 * the stated range, dt <= 0, or a species given some but not all of its four layers;
 * CHEM_ENOMEM / CHEM_ECUDA if the upload fails. */
int chem_surrogate_create_per_species(const chem_surrogate_ps_desc* desc, chem_mech_t m,
                                      chem_model_t* out);

/* Same from a binary file.  CHEMSUR1 (one network): magic, int32 ns, int32 hidden, double dt,
 * then W[l], b[l] (l = 0..4), x_mean, x_std, y_mean, y_std, box_lo, box_hi as little-endian
 * float32.  CHEMSUR2 (per-species networks): magic, int32 ns, int32 h1, h2, h3, double dt,
 * int32 nnet, int32 species[nnet], then for each network W1, b1, W2, b2, W3, b3, W4, b4, then
 * the statistics as in CHEMSUR1.
 * CHEM_ENOTFOUND if the file cannot be opened; CHEM_EINVAL if it is not a CHEMSUR1 or CHEMSUR2 file
 * of a supported shape; otherwise the errors of the matching create call. */
int chem_surrogate_load(const char* path, chem_mech_t m, chem_model_t* out);
/* Release a model's device memory (cudaFree, which waits for device work still using it); the
 * handle is invalid afterwards.  CHEM_EINVAL for NULL. */
int chem_surrogate_free(chem_model_t model);

/* Network pass only (features, MLP, inverse transform): ynet[k * ncells + c] = predicted Y_k
 * (FP32), zout[k * ncells + c] (nullable) = raw network output, and out_of_box[c] = 1 where the
 * features leave the training box.  Device pointers.  Synchronises the stream to report a
 * pipeline timeout (CHEM_ECUDA). */
int chem_surrogate_forward(chem_model_t model, const double* T, const double* p, const double* Y,
                           int64_t ld, int64_t ncells, float* ynet, float* zout,
                           uint8_t* out_of_box, chem_stream_t stream);

/* Surrogate chemistry step in place: network, element-conservation projection, clipping,
 * temperature from enthalpy conservation (Newton), acceptance tests; cells outside the training
 * box or failing a test are advanced by the FP64 integrator instead (indexed, same call,
 * asynchronous).  dt must equal the model's training step.  route_out[c] (nullable, int8):
 * 0 = network, 1 = FP64 fallback.
 * CHEM_EINVAL for a NULL model or mechanism, a species count that differs between them, ncells < 0,
 * ld < ncells, rtol or atol <= 0, a dt other than the model's, or (ncells > 0) a NULL state
 * pointer; CHEM_ENOMEM / CHEM_ECUDA from the stream-ordered allocator, a launch, or a pipeline wait
 * that timed out. */
int chem_surrogate_advance(chem_model_t model, chem_mech_t m, double* T, const double* p,
                           double* Y, int64_t ld, double dt, int64_t ncells, double rtol,
                           double atol, int8_t* route_out, chem_stream_t stream);

/* Several solvers' states advanced by the surrogate in one pass (iteration-level batching of the
 * serving loop): the segments' cells are gathered into one contiguous state (stream-ordered
 * temporary), advanced by one chem_surrogate_advance (one forward launch, one post-processing
 * launch, one FP64 fallback launch) and scattered back.  Per segment: T, p, Y, ld, ncells as for
 * chem_surrogate_advance, status (nullable) receives the route of each cell (0 network, 1 FP64),
 * idx must be NULL, nsub and nrej are ignored; every segment's dt must be the model's and all
 * segments share the first one's rtol and atol.  Segments beyond kMaxSegsPerLaunch (32) make
 * consecutive passes.  Asynchronous on stream.
 * CHEM_EINVAL for NULL arguments, nseg < 1, or a segment that breaks these rules; the errors of
 * chem_surrogate_advance. */
int chem_surrogate_advance_batch(chem_model_t model, chem_mech_t m, const chem_segment* segs, int nseg,
                                 chem_stream_t stream);

/* Heat-release rate of a step (the accuracy measure of the surrogate):
 * q[c] = -rho0 sum_k h_k(T0) (Y1_k - Y0_k) / (W_k dt) with h_k molar (formation included),
 * rho0 from (T0, p, Y0).  erg / (cm^3 s).  Device pointers, asynchronous.
 * CHEM_EINVAL for a NULL argument, ncells < 0, ld < ncells or dt <= 0. */
int chem_heat_release(chem_mech_t m, const double* T0, const double* p, const double* Y0,
                      const double* Y1, int64_t ld, int64_t ncells, double dt, double* q,
                      chem_stream_t stream);

/* BF16 tensor-core GEMM used by training: C[M x N] (FP32, row pitch ldc) = A[M x K] B[N x K]^T
 * (+ bias[N], nullable); A, B device BF16 with K contiguous, row pitches lda/ldb (elements,
 * 16-byte multiples), M >= 128 and N >= 128 (ragged edges are zero-filled by TMA).  *err
 * (device int) is set to 1 if a pipeline wait times out.
 * CHEM_EINVAL for M or N below 128, K <= 0, a NULL A, B, C or err, or A or B not 16-byte aligned or
 * with a row pitch that is not a multiple of 16 bytes; CHEM_ECUDA if a tensor map cannot be
 * encoded. */
int chem_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc,
                   const float* bias, int M, int N, int K, int* err, chem_stream_t stream);
/* The same product with the activation epilogue of the per-species networks: Cb[M x N] (BF16, row
 * pitch ldc) = bf16(act(A B^T + bias)) with act = exact-erf GELU if gelu != 0, else identity.
 * The errors of chem_gemm_bf16 (with Cb for C). */
int chem_gemm_bf16_act(const void* A, int64_t lda, const void* B, int64_t ldb, void* Cb, int64_t ldc,
                       const float* bias, int gelu, int M, int N, int K, int* err, chem_stream_t stream);

/* ---------------------------------------------------------------------------------------
 * Surrogate training on the GPU (§2: GELU networks trained with Adam).  A trainer holds FP32
 * master weights, Adam moments and BF16 copies of a n_in -> 512 x 4 -> n_out GELU network;
 * every product runs on the tcgen05 GEMM.  Layout: X is BF16 [batch x 128], each row the
 * compensated split of the n_in features [x_hi | x_lo | x_hi | 0] (chem_train_normalize writes
 * it; n_in <= 42); the first layer's BF16 weights are [W_hi | W_hi | W_lo | 0] and its master
 * gradient is dZ^T (x_hi + x_lo).  Targets FP32 [batch x n_out], all device pointers.
 * ------------------------------------------------------------------------------------- */
typedef struct chem_trainer_s* chem_trainer_t;

/* W_init / b_init: host arrays [5] of row-major [out x in] weights and [out] biases, or NULL for
 * a seeded Gaussian initialisation (std 1/sqrt(fan_in), zero biases).  batch: multiple of 128.
 * The errors of chem_mlp_trainer_create_layers. */
int chem_mlp_trainer_create(int n_in, int n_out, int batch, const float* const* W_init,
                            const float* const* b_init, uint64_t seed, chem_trainer_t* out);
/* Same with the caller's hidden widths: n_in -> hidden[0] -> ... -> hidden[n_hidden - 1] -> n_out
 * (1 <= n_hidden <= 7, widths in [1, 8192]; the per-species networks use 1600, 800, 400);
 * W_init / b_init hold n_hidden + 1 layers.
 * CHEM_EINVAL for NULL out or hidden, n_in outside [1, 42], n_out outside [1, 128], n_hidden
 * outside [1, 7], a width outside [1, 8192], or a batch that is not a positive multiple of 128;
 * CHEM_ENOMEM / CHEM_ECUDA if the device buffers cannot be made. */
int chem_mlp_trainer_create_layers(int n_in, int n_out, int n_hidden, const int* hidden, int batch,
                                   const float* const* W_init, const float* const* b_init,
                                   uint64_t seed, chem_trainer_t* out);
/* Release a trainer's parameters, optimiser state and activations (cudaFree, which waits for
 * device work still using them).  CHEM_EINVAL for NULL. */
int chem_mlp_trainer_free(chem_trainer_t t);
/* forward pass of one batch, keeping the activations; out (nullable) receives [batch x n_out].
 * X is read again by chem_mlp_backward: it must stay valid until that call's work is done.
 * CHEM_EINVAL for a NULL trainer or X. */
int chem_mlp_forward(chem_trainer_t t, const void* X, float* out, chem_stream_t stream);
/* mean-squared-error gradients of the last forward pass; loss (device double, nullable).
 * CHEM_EINVAL for a NULL trainer or target. */
int chem_mlp_backward(chem_trainer_t t, const float* target, double* loss, chem_stream_t stream);
/* one Adam update (bias-corrected) of all parameters with the last gradients.  The step counter
 * and the bias corrections 1 - beta^step live in device memory and are advanced by the first
 * kernel of the update, so the whole update can be captured in a CUDA graph and replayed.
 * CHEM_EINVAL for a NULL trainer or lr <= 0. */
int chem_mlp_adam_step(chem_trainer_t t, float lr, float beta1, float beta2, float eps,
                       chem_stream_t stream);
/* the same update with the learning rate read from device memory (*lr, FP32) when the update
 * runs: a training step captured once in a CUDA graph takes each step's scheduled rate from a
 * buffer the host rewrites between replays.  The result is bitwise that of chem_mlp_adam_step
 * with the same rate.  CHEM_EINVAL for a NULL trainer or lr. */
int chem_mlp_adam_step_dev(chem_trainer_t t, const float* lr, float beta1, float beta2, float eps,
                           chem_stream_t stream);
/* host copy of the parameters (which = 0) or of the last gradients (which = 1); W[l], b[l] are
 * host arrays of the unpadded shapes (any may be NULL); synchronises the device.
 * CHEM_EINVAL for a NULL trainer, W or b; CHEM_ECUDA if a copy fails. */
int chem_mlp_trainer_get(chem_trainer_t t, int which, float* const* W, float* const* b);

/* Data-parallel training (each rank of a job holds a trainer with the same weights and computes
 * the gradients of its own share of the global batch; one sum over the ranks, e.g. an NCCL
 * all-reduce of the flat buffer, then every rank takes the same Adam step).  The flat layout of
 * the real (unpadded) gradients is, layer by layer, dW_l [out x in] row-major then db_l [out];
 * chem_mlp_grad_count gives its length in floats (0.80 M for the 11 -> 512 x 4 -> 9 network).
 * pack copies the last gradients into the caller's device buffer flat; unpack writes scale * flat
 * back as the gradients the next chem_mlp_adam_step uses (scale = 1 / ranks turns a sum of the
 * ranks' batch means into the mean over the global batch when every rank's batch has the same
 * size).  Asynchronous on stream.  CHEM_EINVAL for a NULL trainer, count or flat pointer, or a
 * non-finite scale. */
int chem_mlp_grad_count(chem_trainer_t t, int64_t* n);
int chem_mlp_grad_pack(chem_trainer_t t, float* flat, chem_stream_t stream);
int chem_mlp_grad_unpack(chem_trainer_t t, const float* flat, float scale, chem_stream_t stream);

/* Checkpoint and resume of training (Adam, §2): save writes the FP32 master weights and biases,
 * both Adam moments of every parameter and the Adam step counter to the file path (format
 * CHEMTRN1: magic, int32 layers, n_in, n_out, the real input and output widths of every layer,
 * int64 step, then per layer W, b, m_W, m_b, v_W, v_b as little-endian FP32 of the unpadded
 * shapes); load reads such a file into a trainer of the same shape (the batch may differ),
 * rebuilds the BF16 copies and sets the step counter, so that the next steps continue the saved
 * run exactly.  Both synchronise the device.  chem_mlp_trainer_step returns the number of Adam
 * steps taken.  CHEM_EINVAL for NULL arguments, a file of another shape, a truncated file (the
 * trainer is then unchanged) or a write error; CHEM_ENOTFOUND when the file cannot be opened. */
int chem_mlp_trainer_save(chem_trainer_t t, const char* path);
int chem_mlp_trainer_load(chem_trainer_t t, const char* path);
int chem_mlp_trainer_step(chem_trainer_t t, int64_t* step);

/* Training data: raw features x [n x (ns + 2)] = [T, ln p, BC(Y0)] and targets
 * t [n x ns] = BC(Y1) - BC(Y0) (difference formed in FP64) from states before (T0, p, Y0) and
 * after (Y1) a step.  Device arrays; CHEM_EINVAL for a NULL array, n < 0, ld < n or ns outside
 * [1, 62].  Asynchronous on stream. */
int chem_train_features(const double* T0, const double* p, const double* Y0, const double* Y1,
                        int64_t ld, int64_t n, int ns, float* x_raw, float* t_raw,
                        chem_stream_t stream);
/* stats[4 x c] (device doubles): column sums, sums of squares, minima, maxima of A [n x c].
 * CHEM_EINVAL for a NULL array, n < 1 or c outside [1, 64].  Asynchronous on stream. */
int chem_column_stats(const float* A, int64_t n, int c, double* stats, chem_stream_t stream);
/* v = (x - mean) / sd;  X row = [bf16(v) | bf16(v - bf16(v)) | bf16(v) | 0] (c columns each, zero
 * padded to ldx >= 3 c); Tn = (t - tmean) / tsd (t nullable).  CHEM_EINVAL for a NULL array,
 * n < 0, c < 1, ldx < 3 c, or t without tmean, tsd and Tn.  Asynchronous on stream. */
int chem_train_normalize(const float* x, int64_t n, int c, const float* mean, const float* sd,
                         void* X, int ldx, const float* t, int ct, const float* tmean,
                         const float* tsd, float* Tn, chem_stream_t stream);

/* ---------------------------------------------------------------------------------------
 * Serving: chemistry sub-steps from many concurrent flow solvers on one GPU.  Solvers register
 * their resident device states once and submit one request per sub-step; a server thread admits
 * requests under a device-memory budget (resident states + per-request workspace), batches the
 * admitted FP64 requests of a mechanism into one job of the persistent integrator and overlaps
 * launches on a small stream pool (continuous batching).  An FP64 job runs as time slices of
 * slice_ms: each slice stops claiming cells after that time and the next continues the same work
 * queue, so launches on other streams get the SMs in between; issuing a surrogate pass also ends
 * the running slices early (once they have run 2 ms), so that the pass does not wait for the
 * rest of a slice.  Results do not depend on where slices end.  A request completes when the
 * queue passes its last cell.  Latency = submission to completion.  No counterpart in the paper,
 * whose solver owns the GPU alone (§3.1). 
 * ------------------------------------------------------------------------------------- */
enum { CHEM_ROUTE_FP64 = 0, CHEM_ROUTE_SURROGATE = 1 };
enum { CHEM_REQ_QUEUED = 0, CHEM_REQ_RUNNING = 1, CHEM_REQ_DONE = 2, CHEM_REQ_FAILED = 3 };

typedef struct chem_serve_options {
  int32_t n_streams;         /* concurrent FP64 jobs and, on as many high-priority streams,
                                concurrent surrogate launches (0 -> 4 each) */
  double idle_poll_us;       /* polling interval while launches are in flight (0 -> 20 us) */
  double slice_ms;           /* FP64 time slice (0 -> 20 ms; negative: no slicing) */
  double max_pause_ms;       /* a time-sliced FP64 job whose slice ends while surrogate passes run
                                waits up to this long before its next slice, so that the passes'
                                kernels find the SMs free (0 -> 20 ms; negative: never waits) */
} chem_serve_options;

/* Start a server on the current device: its streams (half low-priority FP64, half high-priority
 * surrogate), its device work-queue counters and one host thread that admits, batches and
 * launches requests.  hbm_budget_bytes (> 0) bounds the device memory of registered states plus
 * running requests' workspaces; opt nullable (defaults).  *out receives a handle owned by the
 * caller (chem_serve_destroy).  CHEM_EINVAL for a zero budget or NULL out; CHEM_ECUDA if a
 * stream or the counters cannot be created. */
int chem_serve_create(size_t hbm_budget_bytes, const chem_serve_options* opt, chem_server_t* out);
/* Register a solver's resident state (device arrays owned by the caller, valid until the server
 * is destroyed); model (nullable) enables the surrogate route.  CHEM_EBUSY if the state alone
 * exceeds what is left of the budget. */
int chem_serve_register_state(chem_server_t s, chem_mech_t m, chem_model_t model, double* T,
                              double* p, double* Y, int64_t ld, int64_t ncells, int* state_id);
/* Queue one sub-step of a registered state.  CHEM_EBUSY if the request could never be admitted
 * (its workspace exceeds the budget left by the resident states).  A queued request that stops
 * fitting because states registered after it took the budget fails (CHEM_REQ_FAILED) as soon as
 * nothing else is running, instead of waiting forever. */
int chem_serve_submit(chem_server_t s, int state_id, int route, double dt, double rtol,
                      double atol, uint64_t* req_id);
/* Non-blocking: *state = CHEM_REQ_*, *latency_s (nullable) = seconds from submission to
 * completion once done, else -1.
 * CHEM_EINVAL for a NULL server or state; CHEM_ENOTFOUND for an unknown request. For a failed
 * request its message is left in chem_last_error. */
int chem_serve_poll(chem_server_t s, uint64_t req_id, int* state, double* latency_s);
/* Block until the request is done or timeout_s passes (CHEM_ETIMEOUT); never hangs. */
int chem_serve_wait(chem_server_t s, uint64_t req_id, double timeout_s);
/* out[8]: completed, failed, launches (jobs and surrogate launches), requests launched (those
 * that joined a running job included), max concurrent launches, bytes in use, FP64 time slices
 * issued, FP64 requests that joined a running time-sliced job.
 * CHEM_EINVAL for NULL arguments. */
int chem_serve_stats(chem_server_t s, int64_t* out);
/* Stops the server after its launches finish; queued requests fail and callers blocked in
 * chem_serve_wait on them return.  No call on the server may start once this is entered.
 * CHEM_EINVAL for NULL. */
int chem_serve_destroy(chem_server_t s);

/* ---------------------------------------------------------------------------------------
 * Thermophysical and transport properties per cell (§3.1: the paper's Thermo class computes
 * them with Newton's method and high-order temperature polynomials on the GPU).  SoA state as
 * for chem_advance; device pointers; asynchronous on stream.
 * ------------------------------------------------------------------------------------- */
/* Mixture enthalpy h (erg/g, formation included) and cp (erg/(g K)) from the NASA-7 fits;
 * either output may be NULL.
 * CHEM_EINVAL for a NULL mechanism, ncells < 0, ld < ncells, or (ncells > 0) a NULL T or Y or both
 * outputs NULL. */
int chem_mixture_thermo(chem_mech_t m, const double* T, const double* Y, int64_t ld, int64_t ncells,
                        double* h, double* cp, chem_stream_t stream);
/* Temperature from enthalpy: Newton T <- T - (h(T, Y) - h0) / cp(T, Y) from the initial guess in
 * T, until |dT| < 1e-9 T (at most 50 iterations, T kept in [200, 6000] K).  T is updated only
 * where it converged; status[c] (nullable, int8) = 0 converged, 1 not.
 * CHEM_EINVAL for a NULL mechanism, ncells < 0, ld < ncells, or (ncells > 0) a NULL h0, Y or T. */
int chem_temperature_from_enthalpy(chem_mech_t m, const double* h0, const double* Y, int64_t ld,
                                   int64_t ncells, double* T, int8_t* status, chem_stream_t stream);

typedef struct chem_transport_s* chem_transport_t;
/* Transport data of a mechanism: cubic fits in ln T (T in K) of ln mu_k (g/(cm s)),
 * ln lambda_k (erg/(cm s K)) and ln D_jk (cm^2/s at p_atm; D_jk(p) = D_jk(p_atm) p_atm / p),
 * coefficients in ascending powers; host arrays, copied. */
typedef struct chem_transport_desc {
  int32_t n_species;
  const double* mu_poly;       /* [ns][4] */
  const double* lambda_poly;   /* [ns][4] */
  const double* diff_poly;     /* [ns][ns][4], symmetric */
} chem_transport_desc;
/* Copy a mechanism's transport fits to the device.  *out receives a handle owned by the caller
 * (chem_transport_free).  CHEM_EINVAL for NULL arguments, a NULL table or n_species different from
 * the mechanism's; CHEM_ENOMEM / CHEM_ECUDA if the upload fails. */
int chem_transport_create(chem_mech_t m, const chem_transport_desc* desc, chem_transport_t* out);
/* Release the device copy (cudaFree, which waits for device work still using it).  CHEM_EINVAL
 * for NULL. */
int chem_transport_free(chem_transport_t t);
/* Mixture-averaged properties: viscosity by Wilke's rule, conductivity by the Mathur-Saxena
 * average, D_km = (1 - Y_k) / sum_{j != k} X_j / D_jk (the self-diffusion fit for a cell holding
 * species k alone).  mu [n], lambda [n], Dmix [ns][ld]: device outputs, each nullable.
 * CHEM_EINVAL for a NULL handle, ncells < 0, ld < ncells, or (ncells > 0) a NULL T, p or Y or all
 * three outputs NULL. */
int chem_transport_eval(chem_transport_t t, const double* T, const double* p, const double* Y,
                        int64_t ld, int64_t ncells, double* mu, double* lambda, double* Dmix,
                        chem_stream_t stream);

/* The FP64 exponential the integrator's rate evaluation uses (table-driven, after Tang, ACM TOMS
 * 15(2), 1989: a 64-entry table of 2^(j/64) and a degree-5 polynomial; within a few units in the
 * last place of exp; |x| >= 700 and NaN take the library exp), applied elementwise:
 * y[i] = exp(x[i]) for i < n.  x, y: device arrays of n doubles (may alias).  Asynchronous on
 * stream.  Exposed for testing and measurement.
 * CHEM_EINVAL for n < 0 or (n > 0) a NULL x or y. */
int chem_fast_exp(const double* x, double* y, int64_t n, chem_stream_t stream);

/* Measured FP64 FMA throughput of the current device (TFLOP/s, 2 flops per FMA) from a
 * register-resident FMA chain kernel; synchronous.
 * CHEM_EINVAL for a NULL output; CHEM_ECUDA if the probe fails. */
int chem_fp64_fma_peak(double* tflops);

/* ---------------------------------------------------------------------------------------
 * One "chemistry + thermo" step of the reactive-flow time loop (§3.1, Fig. 1: chemical source,
 * Thermo, transport properties), optionally captured once into a CUDA graph and replayed (§3.2).
 * Stages, on the caller's stream: (0) the start state (T, Y) is copied into buffers of the step
 * and its mixture enthalpy h0 and cp0 are evaluated; (1) chemistry over dt: the BF16 surrogate with
 * FP64 fallback (model given) or the FP64 integrator; (2) the heat-release rate q of the step
 * (nullable) and T from h(T, Y1) = h0 by Newton, written into T (the adiabatic constant-pressure
 * step conserves h, so the Thermo stage recovers T from it); (3) transport properties of the new
 * state (transport given).  All arrays are the caller's device arrays and must stay valid while
 * the step object lives: a captured graph replays on the same pointers.
 * ------------------------------------------------------------------------------------- */
typedef struct chem_step_s* chem_step_t;
typedef struct chem_step_desc {
  chem_mech_t mech;
  chem_model_t model;          /* nullable: FP64 integrator when NULL */
  chem_transport_t transport;  /* nullable: no transport stage when NULL */
  double* T;                   /* [ncells] in/out */
  const double* p;             /* [ncells] */
  double* Y;                   /* [ns][ld] in/out */
  int64_t ld, ncells;
  double dt, rtol, atol;
  double* h0;                  /* [ncells] out: mixture enthalpy of the start state (required) */
  double* cp0;                 /* [ncells] out, nullable */
  double* q;                   /* [ncells] out, nullable: heat-release rate of the step */
  int8_t* route;               /* [ncells] out, nullable: surrogate route (0 network, 1 FP64) */
  int8_t* status;              /* [ncells] out, nullable: FP64 integrator status */
  int32_t* nsub;               /* [ncells] out, nullable: FP64 accepted sub-steps */
  int8_t* thermo_status;       /* [ncells] out, nullable: 0 when the Newton on T converged */
  double* mu;                  /* [ncells] out, nullable */
  double* lambda;              /* [ncells] out, nullable */
  double* Dmix;                /* [ns][ld] out, nullable */
} chem_step_desc;
/* Create a step over the caller's arrays (allocates the start-state copies, stage events and a
 * private capture stream).  CHEM_EINVAL for NULL arguments, ncells < 1, ld < ncells, a NULL T, p,
 * Y or h0, non-positive dt, rtol or atol, a model whose species count differs from the
 * mechanism's, or a transport handle without any transport output; CHEM_ENOMEM / CHEM_ECUDA if
 * the buffers cannot be made. */
int chem_step_create(const chem_step_desc* desc, chem_step_t* out);
/* Issue one step on stream.  use_graph = 0: the stages directly, with events between them
 * (chem_step_stage_ms reads their times); use_graph != 0: the first such call captures the
 * stage sequence into a CUDA graph (a private stream ordered after stream) and every such call
 * launches the graph on stream.  Errors of the stage entry points, or CHEM_ECUDA from capture,
 * instantiation or launch. */
int chem_step_run(chem_step_t s, int use_graph, chem_stream_t stream);
/* Device time of stages 0-3 of the last direct run, in ms (ms[4]); synchronises on its end.
 * CHEM_EINVAL for NULL arguments or when no direct run has been issued. */
int chem_step_stage_ms(chem_step_t s, float* ms);
/* Release the step (the caller's arrays are untouched).  CHEM_EINVAL for NULL. */
int chem_step_free(chem_step_t s);

/* ---------------------------------------------------------------------------------------
 * Finite-volume species equation (the paper's species PDE, §3.1, with the Laplacian term of
 * Alg. 1) and the PaSR factor of its LES closure (§2).
 *
 * A mesh is face-addressed as in the paper's ldu format: internal faces with owner < neighbour,
 * per face the owner's linear-interpolation weight w, the delta coefficient (1 / centre
 * distance) and the area |S|; boundary faces with their cell, patch type (0 zero-gradient,
 * 1 fixed-value), delta coefficient (1 / face-to-centre distance) and area; cell volumes.
 * ------------------------------------------------------------------------------------- */
typedef struct chem_fvmesh_s* chem_fvmesh_t;
typedef struct chem_fvmesh_desc {
  int64_t n_cells, n_faces, n_bfaces;
  const int32_t* owner;      /* [n_faces] host arrays, copied */
  const int32_t* neighbour;  /* [n_faces], owner < neighbour */
  const double* weight;      /* [n_faces] owner interpolation weight */
  const double* delta;       /* [n_faces] */
  const double* mag_sf;      /* [n_faces] */
  const int32_t* b_cell;     /* [n_bfaces] */
  const int8_t* b_type;      /* [n_bfaces] 0 zero-gradient, 1 fixed-value */
  const double* b_delta;     /* [n_bfaces] */
  const double* b_mag_sf;    /* [n_bfaces] */
  const double* volume;      /* [n_cells] */
} chem_fvmesh_desc;
/* Upload a mesh; builds the cell-to-face index and the CSR pattern of its matrices.  At most
 * 2^31 - 1 cells and 2^29 - 1 faces of each kind, and n_cells + 2 n_faces (the matrix entries)
 * at most 2^31 - 1.  Checked on the host before any device work: CHEM_EINVAL for sizes out of
 * range, a NULL array, a face whose owner is not below its neighbour or whose cells are outside
 * the mesh, or a boundary face with a cell outside the mesh or a patch type other than 0 or 1. */
int chem_fvmesh_create(const chem_fvmesh_desc* desc, chem_fvmesh_t* out);
/* Release the mesh's device arrays, the CSR pattern included (cudaFree, which waits for device
 * work still using them).  CHEM_EINVAL for NULL. */
int chem_fvmesh_free(chem_fvmesh_t mesh);
/* The CSR pattern (device arrays owned by the mesh): row_ptr [n_cells + 1], col_idx [nnz],
 * columns ascending within a row; the diagonal is always stored.
 * CHEM_EINVAL for NULL arguments. */
int chem_fvmesh_csr(chem_fvmesh_t mesh, int64_t* nnz, const int32_t** row_ptr, const int32_t** col_idx);

/* Terms of one species equation over one step (device arrays; a NULL input leaves its term out):
 *   (rho Y - rho_old Y_old) V / dt                                    if dt > 0
 *   + sum_f F_f(Y)            upwind convection by the face mass flux phi (owner -> neighbour)
 *                             and the outward boundary flux phi_b (inflow takes Y_b)
 *   - sum_f a_f (Y_N - Y_P) - sum_{fixed-value b} a_b (Y_b - Y_P)      if gamma (= rho D)
 *     with a_f = (w gamma_owner + (1 - w) gamma_neighbour) |S_f| delta_f  (Alg. 1) and
 *     a_b = gamma_b |S_b| delta_b
 *   = V kappa S               if S (kappa NULL: 1) */
typedef struct chem_fvm_terms {
  double dt;
  const double* rho;         /* [n_cells] */
  const double* rho_old;     /* [n_cells] */
  const double* Y_old;       /* [n_cells] */
  const double* phi;         /* [n_faces] */
  const double* phi_b;       /* [n_bfaces] */
  const double* gamma;       /* [n_cells] */
  const double* gamma_b;     /* [n_bfaces] */
  const double* Y_b;         /* [n_bfaces] boundary values (fixed-value faces, inflow) */
  const double* S;           /* [n_cells] source per unit volume */
  const double* kappa;       /* [n_cells] PaSR factor of S */
} chem_fvm_terms;
/* Assemble the matrix in ldu form: upper[f] = A[owner, neighbour], lower[f] = A[neighbour,
 * owner], diag[c], and the right-hand side source[c] (nullable).  One kernel, no atomics;
 * bitwise reproducible.  Asynchronous on stream.
 * CHEM_EINVAL for a NULL mesh, terms or output, and for incomplete terms: the time term (dt > 0)
 * without rho, rho_old and Y_old, boundary fluxes without boundary values, or the Laplacian on a
 * mesh with boundary faces without gamma_b and Y_b. */
int chem_fvm_assemble(chem_fvmesh_t mesh, const chem_fvm_terms* terms, double* lower, double* upper,
                      double* diag, double* source, chem_stream_t stream);
/* The same matrix as CSR values vals [nnz] on the mesh's pattern (for a linear solver).
 * CHEM_EINVAL for NULL arguments. */
int chem_fvm_to_csr(chem_fvmesh_t mesh, const double* lower, const double* upper, const double* diag,
                    double* vals, chem_stream_t stream);
/* PaSR factor per cell: kappa = tau_c / (tau_c + tau_mix), tau_mix = c_mix sqrt(mu_eff / (rho eps)),
 * with the Smagorinsky sub-grid viscosity nu = (c_s Delta)^2 |S|, mu_eff = mu + rho nu and
 * eps = nu |S|^2; kappa = 1 where eps = 0.  tau_c (the chemical time scale), rho, mu, strain
 * (|S|) and delta (filter width): device arrays of n doubles.  Asynchronous on stream.
 * CHEM_EINVAL for n < 0, (n > 0) a NULL array, or c_s or c_mix negative or NaN. */
int chem_pasr_kappa(int64_t n, const double* tau_c, const double* rho, const double* mu,
                    const double* strain, const double* delta, double c_s, double c_mix,
                    double* kappa, chem_stream_t stream);

/* Message of the last failure on the calling thread (empty if none); the string stays valid
 * until the thread's next failing call.  Never fails. */
const char* chem_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CHEM_H */
