/*
 * tami.h -- C ABI of libtami, a GB300 (sm_103a) implementation of the batched evaluation of
 * algorithmic Matsubara integration (AMI) solutions.
 *
 * Method: M. D. Burke and J. P. F. LeBlanc, "TorchAmi: Generalized CPU/GPU Implementation of
 * Algorithmic Matsubara Integration", arXiv:2311.17189.  Section, equation and figure names
 * below are the paper's.
 *
 * Conventions (all calls):
 *   - Status: every int-returning call returns TAMI_OK (0) or one of the TAMI_E* codes below;
 *     tami_last_error() then gives a message (per host thread).  Nothing throws across the ABI.
 *   - Complex numbers are two adjacent doubles (re, im).  Arrays are C-contiguous.
 *   - "device" pointers are CUDA global-memory pointers on the device the diagram was uploaded
 *     to; they are owned by the caller and must stay valid until the stream has run the work.
 *     "host" pointers are ordinary CPU memory read before the call returns.
 *   - stream: a cudaStream_t (NULL = legacy default stream).  Device work is asynchronous on it;
 *     outputs are valid once the stream is synchronised.
 *   - A diagram is library-owned: created by tami_construct, freed by tami_destroy.  Its device
 *     term table is created by tami_upload and freed by tami_destroy.
 *   - Variables: n_vars = m + n_ext frequency/momentum labels, the m internal (summed) ones first
 *     and the n_ext external ones last (Sec. 2.3: a frequency_t row holds m + n_nu entries, "the
 *     external frequency(s) are the last elements").  tami_construct has n_ext = 1; the momentum
 *     calls (tami_sample_energies, tami_forward*, tami_backward, tami_batch_plan) need n_ext = 1,
 *     since the momentum integrand of Sec. 5.2 appends one external momentum, and refuse others
 *     with TAMI_EUNSUPPORTED; energy input (tami_eval_energies) takes any n_ext.
 *   - Lines: n_lines = N Green's functions G_j = 1/(X_j + E_j) (Eq. Green_Function) with
 *     X_j = sum_l i alpha_jl nu_l and E_j = sum_k eps_jk E_k (base energies E_k).
 */
#ifndef TAMI_H
#define TAMI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st* tami_stream_t; /* identical to cudaStream_t */

enum {
  TAMI_OK = 0,
  TAMI_EINVAL = 1,       /* bad argument (sizes, NULL, malformed labels)                  */
  TAMI_ENOMEM = 2,       /* host or device allocation failed                               */
  TAMI_ECUDA = 3,        /* a CUDA runtime call failed                                     */
  TAMI_ETIMEOUT = 4,     /* a bounded device wait gave up                                  */
  TAMI_EUNSUPPORTED = 5  /* valid input outside what the library handles (see message)   */
};

enum { TAMI_MAX_LINES = 16, TAMI_MAX_VARS = 8, TAMI_MAX_EXT = 4 };

typedef struct tami_diagram tami_diagram;

/* Square-lattice Hubbard dispersion eps(k) = -2t(cos kx + cos ky) - 4t' cos kx cos ky and the
 * external momentum; the line energy is E = mu - eps(k) (Sec. 5.2: per-line dispersion of the
 * composed momenta K = k A^T; Eq. Green_Function: epsilon^j is minus the dispersion). */
typedef struct {
  double t, tp, mu;
  double kx_ext, ky_ext;
} tami_lattice;

/* Sizes of a constructed solution and of its device table. */
typedef struct {
  int n_lines, n_vars;
  int64_t n_terms;          /* flat terms A * FT * R (FACTORIZE=false form, Sec. 2.2)        */
  int64_t n_fermi_factors;  /* Fermi/Bose factors over all terms                              */
  int64_t n_g_factors;      /* Green's functions over all terms, powers counted               */
  int max_der;              /* highest derivative order of a Fermi/Bose factor (Eq. Res_mul)  */
  int max_g;                /* most Green's functions in one term                             */
  int64_t unique_poles;     /* distinct (energy combination up to sign, sigma) of FT factors  */
  int64_t unique_dens;      /* distinct (energy combination, external coefficient) of R       */
  /* device table */
  int n_combos;             /* distinct energy combinations c.E evaluated per sample          */
  int n_fermi_values;       /* distinct Fermi/Bose values per sample                          */
  int n_real_dens;          /* frequency-independent denominators                            */
  int n_cplx_dens;          /* denominators carrying the external frequency                   */
  int n_groups_fixed;       /* groups of terms with one denominator signature                 */
  int n_groups_freq;        /* groups sharing one frequency-dependent signature               */
  int table_bytes;
  /* FP64 flops of the kernels' arithmetic (fma = 2, mul/add = 1; exponential, reciprocal and
   * trig by their own operation counts): per sample (frequency independent part) and per
   * (sample, frequency) */
  double flops_per_sample;
  double flops_per_sample_freq;
  /* the same for tami_backward (recomputation + adjoint sweep) */
  double bwd_flops_per_sample;
  double bwd_flops_per_sample_freq;
  /* rows of tami_forward's `saved` output: computed lines + 2 per line carrying k_ext */
  int saved_rows;
  /* per-sample flops of tami_forward when it writes `saved`, and of tami_backward reading it */
  double fwd_save_flops_per_sample;
  double bwd_saved_flops_per_sample;
  /* per (sample, frequency) flops of tami_forward_backward (per sample: bwd_flops_per_sample) */
  double fused_flops_per_sample_freq;
  int n_ext;                /* external variables (the last n_ext of the n_vars labels)       */
  /* per-row flops of tami_eval_energies (flops_per_sample without the momentum sampling and the
   * dispersion) and per (row, frequency) (flops_per_sample_freq without the Monte Carlo sums,
   * which energy input does not return) */
  double energy_in_flops_per_sample;
  double energy_in_flops_per_sample_freq;
  /* pole DAG of the factorised FT (Sec. 2.1): edges (one fma each) and nodes; phase-2 factors:
   * the complex-denominator powers over the frequency-dependent groups */
  int n_dag_ops, n_dag_nodes, n_phase2_factors;
} tami_info;

const char* tami_last_error(void);

/* Build the AMI solution (Sec. 2.2) of beta^-m sum_{nu_1..nu_m} prod_j G_j (Eq. goal) by summing
 * nu_1..nu_m with the residue theorem (Eq. Res_Th), multipole residues (Eq. Res_mul) for
 * coinciding poles.
 *   alpha        host int8 [n_lines][n_vars], entries in {-1,0,1}, external column last.
 *   eps          host int8 [n_lines][n_lines] energy coefficients, or NULL for the identity
 *                (Sec. 5.1: the starting point; rows of lines with equal alpha may be equal).
 *   var_is_boson host uint8 [n_vars] or NULL (all fermionic, as in the paper).  A bosonic
 *                internal variable is summed with weight -n_B.
 *   order        host int32 [n_vars-1] summation order or NULL for 0,1,..,m-1 (Sec. 5.1).
 *   prefactor    constant multiplying the whole integrand (e.g. (-U)^m (-1)^F).
 * Errors: TAMI_EINVAL for bad sizes/labels, TAMI_EUNSUPPORTED if a summed variable appears with
 * |coefficient| > 1, a term decays slower than 1/z^2, or a Bose factor sits at zero energy. */
int tami_construct(int n_lines, int n_vars, const int8_t* alpha, const int8_t* eps,
                   const uint8_t* var_is_boson, const int32_t* order, double prefactor,
                   tami_diagram** out);

/* tami_construct with n_ext external frequencies (Sec. 2.3: n_nu external frequencies, the last
 * n_nu of the m + n_nu labels): the first m = n_vars - n_ext variables are summed, the last n_ext
 * stay free; a denominator then carries sum_q a_q X_q.  var_is_boson covers the externals too (a
 * Fermi/Bose factor whose pole carries an odd number of fermionic frequencies, external ones
 * included, turns f into -n_B and back).  order: host int32 [m] or NULL.
 * Errors: those of tami_construct; TAMI_EINVAL unless 1 <= n_ext <= TAMI_MAX_EXT and n_ext < n_vars. */
int tami_construct_ext(int n_lines, int n_vars, int n_ext, const int8_t* alpha, const int8_t* eps,
                       const uint8_t* var_is_boson, const int32_t* order, double prefactor,
                       tami_diagram** out);

/* Momentum labels of a self-energy graph (Sec. 2.5: label_graph and graph_to_R0 on the 4-column
 * "source target B/F spin" format).
 *   edges  host int32 [n_edges][4]: source vertex, target vertex, 1 = fermionic / 0 = bosonic,
 *          spin (carried, unused).  Fermionic lines are directed along the particle flow; bosonic
 *          lines are instantaneous interactions (no propagator).  One vertex (the external one)
 *          has one outgoing and one incoming fermionic line -- the amputated external legs -- and
 *          no bosonic line; every other vertex has one fermionic line in, one out and one bosonic.
 *   Outputs: the internal fermionic lines, in file order, are the n_lines rows: alpha int8
 *   [n_lines][n_vars] (loop variables on the non-tree lines of a breadth-first spanning tree from
 *   the node the incoming leg enters, external last), eps int8 [n_lines][n_lines] (equal labels
 *   share an energy), row_line int32 [n_lines] (input line of each row), loops = closed fermion
 *   loops F.  With capacity_lines < n_lines only the sizes are written.
 * Errors: TAMI_EINVAL for a malformed or disconnected graph, TAMI_EUNSUPPORTED beyond 16 lines,
 * 7 loops or labels outside {-1,0,1}. */
int tami_label_graph(const int32_t* edges, int n_edges, int capacity_lines, int8_t* alpha, int8_t* eps,
                     int32_t* row_line, int* n_lines, int* n_vars, int* loops);

/* tami_label_graph followed by tami_construct (all variables fermionic, summed in label order). */
int tami_construct_from_graph(const int32_t* edges, int n_edges, double prefactor, tami_diagram** out);

int tami_diagram_info(const tami_diagram* d, tami_info* info);

/* Copy the flattened term table to `device` (cudaMalloc + cudaMemcpyAsync on `stream`).
 * Must precede every evaluation call.  Re-uploading to another device moves the table. */
int tami_upload(tami_diagram* d, int device, tami_stream_t stream);

/* Per-sample momenta and line energies exactly as tami_forward forms them (Sec. 5.2): internal
 * momenta from Philox4x32-10, counter (s_lo, s_hi, l, 0), key (seed_lo, seed_hi), sample
 * s = offset + i; line momenta K_j = sum_l alpha_jl k_l + alpha_j,ext k_ext; E_j = mu - eps(K_j).
 *   E  device double [n][n_lines] (row i = sample offset+i). */
int tami_sample_energies(const tami_diagram* d, const tami_lattice* lat, uint64_t seed, uint64_t offset,
                         int64_t n, double* E, tami_stream_t stream);

/* Errors common to the evaluating calls (tami_eval_energies, tami_forward, tami_forward_noalloc,
 * tami_backward, tami_batch_launch): TAMI_EINVAL, with nothing launched, for beta not finite and
 * positive, n_f outside the call's range, a required pointer NULL, a sample count below 1 (0 rows
 * is allowed in energy input and launches nothing), or a diagram that is not uploaded or was
 * uploaded to another device than the current one.  The library stays usable after an error. */

/* Energy-input evaluation (Sec. 2.3, energy_t / frequency_t): for each configuration i and
 * external frequency row f, the sum over terms of A * FT(E_i) * R(E_i, X_f).
 *   E    device double [n_e][n_lines] base energies.
 *   X    device double [n_f][n_ext][2]: row f holds the diagram's n_ext external frequencies
 *        (i nu_n, or omega + i Gamma after analytic continuation), in label order; n_ext = 1 is
 *        [n_f][2].
 *   out  device double [n_f][n_e][2] (rows are frequencies, Sec. 2.3).
 * n_e = 0 launches nothing (E and out may then be NULL). */
int tami_eval_energies(const tami_diagram* d, const double* E, int64_t n_e, const double* X, int n_f,
                       double beta, double* out, tami_stream_t stream);

/* Scratch needed by tami_forward for n samples and n_f frequencies (per-block partial sums). */
int tami_forward_workspace(const tami_diagram* d, int64_t n_samples, int n_f, size_t* bytes);

/* Monte Carlo evaluation over momenta (Sec. 5.2; samples and their energies as in
 * tami_sample_energies), reduced over samples (Sec. 2.3, "summing the rows"):
 *   X           device double [n_f][2]
 *   mean        device double [n_f][2]  sample mean of the integrand
 *   var         device double [n_f][2]  unbiased sample variances of Re and Im (may be NULL)
 *   per_sample  device double [n_f][n][2] every sample's value, or NULL
 *   saved       device double [saved_rows][n] (tami_info.saved_rows), or NULL: each sample's line
 *               energies (one row per computed line) and, for the lines carrying k_ext, the
 *               factors G_x, G_y of dE/dK = -G; tami_backward reads them instead of recomputing
 *               momenta, energies and trig (term products are still recomputed).  Row-major,
 *               sample index fastest.
 *   workspace   device, at least tami_forward_workspace() bytes, 256-byte aligned.
 * The reduction is deterministic for fixed (n, n_f, device). */
int tami_forward(const tami_diagram* d, const tami_lattice* lat, uint64_t seed, uint64_t offset,
                 int64_t n_samples, const double* X, int n_f, double beta, double* mean, double* var,
                 double* per_sample, double* saved, void* workspace, size_t workspace_bytes,
                 tami_stream_t stream);

/* Scratch needed by tami_backward for n samples and n_f frequencies. */
int tami_backward_workspace(const tami_diagram* d, int64_t n_samples, int n_f, size_t* bytes);

/* Adjoint of tami_forward's mean (the paper defines only the forward evaluation, Sec. 2.3 and
 * Sec. 5.2).  For an upstream gradient g_f = dL/dSigma_f (PyTorch's convention for a real loss
 * L of complex outputs: g = dL/dRe + i dL/dIm) over the same samples:
 *   dsigma_dX   device double [n_f][2] or NULL: dSigma_f/dX_f, the derivative of the mean along
 *               its external frequency (X = omega + i Gamma: dSigma/domega; its real part gives
 *               the quasiparticle weight Z = 1/(1 - dRe Sigma/domega)).
 *   grad_X_re   device double [n_f] or NULL: dL/domega_f = Re(conj(g_f) dSigma_f/dX_f).
 *   grad_params device double [3] or NULL: dL/dmu, dL/dkx_ext, dL/dky_ext
 *               = Re sum_f conj(g_f) dSigma_f/dtheta, through E = mu - eps(K), K = ... + alpha_ext k_ext.
 *   per_sample_dX    device double [n_f][n][2] or NULL: each sample's dv/dX.
 *   per_sample_grads device double [n][3] or NULL: each sample's
 *               Re sum_f conj(g_f) dv/dtheta (theta = mu, kx, ky; not divided by n).
 *   saved       device double [saved_rows][n] written by tami_forward over the same diagram,
 *               lattice, seed, offset and n, or NULL: the line energies and dE/dK factors are
 *               then read instead of recomputed from the momenta (results identical bit for bit;
 *               the caller owns the buffer and its consistency with the forward).
 *   gout        device double [n_f][2]; workspace as tami_backward_workspace, 256-byte aligned.
 * Term products are recomputed, not stored.  Limits: n_f <= 256, derivative order <= 4.
 * Deterministic for fixed (n, n_f, device). */
int tami_backward(const tami_diagram* d, const tami_lattice* lat, uint64_t seed, uint64_t offset,
                  int64_t n_samples, const double* X, int n_f, double beta, const double* gout,
                  double* dsigma_dX, double* grad_X_re, double* grad_params, double* per_sample_dX,
                  double* per_sample_grads, const double* saved, void* workspace, size_t workspace_bytes,
                  tami_stream_t stream);

/* Scratch needed by tami_forward_backward (per-block partial sums of the adjoint and the forward). */
int tami_forward_backward_workspace(const tami_diagram* d, int64_t n_samples, int n_f, size_t* bytes);

/* Forward and adjoint in one pass over the samples, for an upstream gradient known beforehand
 * (no counterpart in the paper, which has no adjoint): the adjoint kernel already recomputes
 * every energy, Fermi value, term product and denominator product of the forward, so it also
 * forms each sample's value and the forward's sums.  Outputs as tami_forward (mean, var,
 * per_sample) and tami_backward (dsigma_dX, grad_X_re, grad_params, per_sample_dX,
 * per_sample_grads), each optional as there except mean.  dsigma_dX does not depend on gout
 * (e.g. Sigma and dSigma/domega for the quasiparticle weight in one pass).  Per-sample outputs
 * equal the separate calls' bit for bit; the reduced ones agree up to the grouping of the sums.
 * Same limits as tami_backward. */
int tami_forward_backward(const tami_diagram* d, const tami_lattice* lat, uint64_t seed, uint64_t offset,
                          int64_t n_samples, const double* X, int n_f, double beta, const double* gout, double* mean,
                          double* var, double* per_sample, double* dsigma_dX, double* grad_X_re, double* grad_params,
                          double* per_sample_dX, double* per_sample_grads, void* workspace, size_t workspace_bytes,
                          tami_stream_t stream);

/* tami_forward without a workspace argument: the same Monte Carlo evaluation and outputs, with
 * its scratch (a status word and the per-block partial sums) taken from a fixed 4 MiB array
 * inside libtami instead of memory the caller allocates.  The paper has no counterpart; this
 * entry exists for callers that cannot allocate device memory, e.g. code whose device memory
 * is all owned by a pool fixed at start-up, or loops that must not let cudaMalloc/cudaFree
 * synchronise the device.
 *   - It allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 *   - The array is part of the loaded library, so every GPU that loads libtami holds its 4 MiB
 *     until the process exits.
 *   - Limit: 256 + 32 * n_f * grid bytes must fit in 4 MiB, grid being the launch's block count
 *     (SM count x resident blocks per SM, at most the number of 128-sample tiles); with 1216
 *     blocks that is n_f <= 107.  Larger requests return TAMI_EINVAL with the sizes in the
 *     message; use tami_forward with a workspace for them.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress, with
 *     that device current); make that first call before any stream capture.
 *   - Every call shares the one array and it keeps the last call's contents; the call clears the
 *     status word itself.  Calls whose work overlaps on the GPU (other streams, other host
 *     threads) race on the array: serialise them.
 *   - The looked-up address is kept for the life of the process: a device reset
 *     (cudaDeviceReset) while libtami is loaded is not supported with this call.
 *   - It always runs the generic kernel (never a specialised one, whose grid it does not size
 *     for); a table the generic kernel cannot stage returns TAMI_EUNSUPPORTED.
 * Arguments, layouts and errors are otherwise those of tami_forward. */
int tami_forward_noalloc(const tami_diagram* d, const tami_lattice* lat, uint64_t seed, uint64_t offset,
                         int64_t n_samples, const double* X, int n_f, double beta, double* mean,
                         double* var, double* per_sample, tami_stream_t stream);

/* Specialised kernels (no counterpart in the paper: how this library runs its evaluating calls).
 * tami_forward, tami_backward, tami_forward_backward and tami_eval_energies can each run a kernel
 * written out for the diagram's own table -- every table index a constant, every per-sample array a set of registers
 * -- instead of the generic kernel, which reads the table from shared memory and keeps per-sample
 * arrays in local memory.  Each is generated as CUDA C++ on the first call that takes it, compiled
 * for sm_103a with NVRTC (loaded at run time: libnvrtc.so.13, or the path in $TAMI_NVRTC; "none"
 * disables it) and cached with the diagram until tami_destroy.  Values agree with the generic kernels to rounding; workspaces and
 * outputs are those of the generic calls.  Part of their double products run on the integer
 * pipes, bit for bit the FP64 unit's for normal values; for tables of at most 256 pole-DAG ops the
 * per-sample products among them flush results below 2^-1022 (and subnormal operands) to zero.
 * The Monte Carlo kinds run 512-thread blocks, two per SM, whose warps meet at barriers in the
 * straight-line per-sample code.  tami_forward_noalloc always runs the generic kernel;
 * batches take the specialised forward kernels of their large diagrams (tami_batch_plan).
 * Compiled kernels are also kept on disk, one file per compilation, in $TAMI_JIT_CACHE (default
 * $HOME/.cache/libtami_jit; "none": no disk cache): an entry records the NVRTC version, options,
 * device arithmetic and source it was built from and a checksum, is loaded only when all of them
 * match the compilation at hand (and NVRTC loads), and is written through a temporary file and a
 * rename.  A missing, damaged or unwritable cache only costs a compilation.
 *   mode TAMI_JIT_NEVER   the generic kernel always;
 *        TAMI_JIT_AUTO    (default; $TAMI_JIT = never | auto | always sets the initial mode) the
 *                         specialised kernel for Monte Carlo launches of at least 2^21 samples and
 *                         energy input of at least 2^25 (row, frequency) values, when the table and
 *                         frequencies are within the generator's limits (Monte Carlo: n_f <= 256)
 *                         and NVRTC is there, else the generic one;
 *        TAMI_JIT_ALWAYS  the specialised kernel for every launch; a call whose kernel cannot be
 *                         built fails with TAMI_EUNSUPPORTED (message from NVRTC), nothing launched.
 * The mode is process-wide.  Compilation takes about a second and happens on the host inside the
 * first call that needs it (or in tami_jit_prepare). */
enum { TAMI_JIT_NEVER = 0, TAMI_JIT_AUTO = 1, TAMI_JIT_ALWAYS = 2 };
int tami_set_jit(int mode);

/* Build the specialised kernels that apply to an uploaded diagram now (for its upload device;
 * several external frequencies: the energy-input one only).
 * TAMI_EUNSUPPORTED when the table is outside the generator's limits or NVRTC is missing or fails. */
int tami_jit_prepare(tami_diagram* d);

/* ready: bit mask of the built kernels (1 fused, 2 forward, 4 adjoint, 8 energy input); last_used:
 * the diagram's last evaluating call ran a specialised kernel (1) or a generic one (0); compile_ms:
 * host time of their generation and compilation. */
int tami_jit_status(const tami_diagram* d, int* ready, int* last_used, double* compile_ms);

/* from_cache: bit mask (as tami_jit_status's ready) of the built kernels that were loaded from the
 * disk cache instead of compiled. */
int tami_jit_cached(const tami_diagram* d, int* from_cache);

/* The generated CUDA C++ source of one kind (0 fused, 1 forward, 2 adjoint, 3 energy input), in host memory,
 * NUL-terminated, truncated to cap bytes; *len is the full size including the NUL.  For inspection
 * and tests. */
int tami_jit_source(const tami_diagram* d, int kind, char* buf, size_t cap, size_t* len);

/* Many diagrams in one persistent launch (the paper evaluates one diagram per call; this batches
 * them).  Each diagram d gets samples[d] Philox samples with key seeds[d] (counter offset 0), the
 * lattice and the n_f external frequencies are shared.
 * tami_batch_plan packs the diagrams' tables into one device buffer, cuts every sample stream into
 * work items of chunk_tiles x 128 samples, orders the items by estimated cost (largest first) and
 * captures [queue reset, persistent kernel, reduction] into a CUDA graph on the current device.
 * chunk_tiles = 0 lets an autotuner pick the chunk size by timing graph replays with typical
 * inputs; the choice is cached per (GPU, batch signature) in memory and in a text file
 * ($TAMI_TUNE_CACHE, default $HOME/.cache/libtami_autotune.txt); $TAMI_TUNE_LOG names a file that
 * each timed candidate (chunk, grid, items, milliseconds per replay) is appended to.
 * Specialised diagrams (see tami_set_jit): in mode "always" every diagram, in "auto" each diagram
 * with at least 2^20 samples whose kernel builds, runs its own generated forward kernel instead of
 * being cut into items: the plan compiles those kernels (on parallel host threads, cached with the
 * diagrams) and the graph launches each over its diagram's whole sample stream after the
 * persistent kernel; the same reduction finishes them.  "always" refuses the plan
 * (TAMI_EUNSUPPORTED) when a diagram's kernel cannot be built.  The diagrams must outlive the plan
 * only until tami_batch_plan returns (their tables are copied, the plan holds its own reference
 * to their compiled kernels).  Allocates device memory. */
typedef struct tami_batch tami_batch;
int tami_batch_plan(const tami_diagram* const* ds, int n_d, const int64_t* samples, const uint64_t* seeds, int n_f,
                    int chunk_tiles, tami_batch** out);

/* Work items, grid size and chunk size (tiles of 128 samples per item) of a plan's persistent
 * kernel (n_items = grid = 0 when every diagram is specialised). */
int tami_batch_info(const tami_batch* b, int* n_items, int* grid, int* chunk_tiles);

/* Which diagrams of a plan run their specialised kernel: flags [n_d] (may be NULL) gets 1 for
 * those, 0 for the persistent kernel's; n_specialised (may be NULL) their count. */
int tami_batch_specialised(const tami_batch* b, int* flags, int* n_specialised);

/* Replay the plan: X device double [n_f][2]; mean and var device double [n_d][n_f][2] (var may be
 * NULL), as tami_forward's mean and variances for each diagram.  Launches asynchronously on
 * `stream`; the per-item reduction is in tile order, so results are deterministic for a plan. */
int tami_batch_launch(tami_batch* b, const tami_lattice* lat, const double* X, double beta, double* mean,
                      double* var, tami_stream_t stream);

void tami_batch_destroy(tami_batch* b);

/* Diagnostic for testing the persistent launch's failure detection (no counterpart in the paper):
 * overwrite entry `item` (0 <= item < the plan's item count) of the plan's device work queue with
 * (diagram d, tiles [tile0, tile1)) and return the previous entry as {d, tile0, tile1} in prev
 * (may be NULL).  The kernel checks every entry it pops against the plan (0 <= d < n_d,
 * 0 <= tile0 < tile1 <= the diagram's tiles); a malformed one is skipped without any access it
 * describes, the plan's status word is set, and that launch's means and variances are NaN.  The
 * next launch resets the status.  Synchronous; the plan must be idle. */
int tami_batch_debug_set_item(tami_batch* b, int item, int d, int64_t tile0, int64_t tile1, int64_t* prev);

/* Hubbard (U n_up n_down) self-energy diagrams of the given order (2..6), one-particle
 * irreducible, without tadpoles, in canonical order, labelled with momentum-conserving alpha
 * (Sec. 2.5: graph representation and labelling).  With capacity 0 only *n_out is set.
 *   alpha  host int8  [capacity][2m-1][m+1]
 *   eps    host int8  [capacity][2m-1][2m-1]  (lines with equal labels share a base energy)
 *   code   host int32 [capacity][1+2m]        canonical contraction code
 *   loops  host int32 [capacity]              closed fermion loops F (sign (-1)^F)
 * Any output pointer may be NULL. */
int tami_enumerate_sigma(int order, int capacity, int8_t* alpha, int8_t* eps, int32_t* code,
                         int32_t* loops, int* n_out);

/* Staging of the term table by the generic forward kernels (tami_eval_energies, tami_forward,
 * tami_forward_noalloc and the persistent kernel of a batch plan; the paper's tables are data
 * read by every evaluation, Sec. 2.3).  Each block copies the table into shared memory with bulk
 * (TMA) copies.  TAMI_STAGING_AUTO (the default) keeps the whole forward pole-DAG program of the
 * factorised FT (Sec. 2.1) resident when it fits beside the tiles and otherwise streams it
 * through two shared-memory buffers of chunk_ops ops each, a bulk copy per chunk, double
 * buffered; TAMI_STAGING_STREAMED always streams (same results bit for bit).  chunk_ops: even,
 * in [16, 4096]; 0 keeps the current value (default 512).  Process-wide; a batch plan takes the
 * setting at planning time.  TAMI_EINVAL for other values. */
#define TAMI_STAGING_AUTO 0
#define TAMI_STAGING_STREAMED 1
int tami_set_table_staging(int mode, int chunk_ops);

/* Test hook (not a term of the paper): bound the first stage of every mbarrier wait of the generic
 * kernels' table staging to `first_stage_spins` polls (0 .. 2^24; -1 restores the default 2^24).
 * A wait that runs out sets the call's status word (TAMI_ETIMEOUT in the device status; the
 * reduced outputs of that launch become NaN) and then waits again, bounded by 2^24 polls, for the
 * copy to land, so a completed copy is still used safely.  With 0 every staging wait "runs out"
 * on a valid copy, which lets a test drive that path without any fault.  Plans (tami_batch_plan)
 * take the value at planning time; the other calls at each launch.  Process-wide. */
int tami_debug_set_wait_limit(int64_t first_stage_spins);

/* Diagnostic: the kernels' exponential for t <= 0 (table-driven after Tang, ACM TOMS 1989), applied
 * elementwise: y = e^t, em = e^t - 1, and y_plain = e^t from the variant that does not form
 * e^t - 1 (the kernels use it where only e^t is needed; it must equal y bit for bit).
 * t, y, em, y_plain: device double [n]; y_plain may be NULL.  Used by the tests to check them
 * against CUDA's exp/expm1. */
int tami_selftest_exp(const double* t, int64_t n, double* y, double* em, double* y_plain, tami_stream_t stream);

/* Diagnostic: the kernels' cos and sin (Cody-Waite reduction by pi and Taylor series, the
 * dispersion of Sec. 5.2's lattice samples; the paper leaves eps(k) to the user) applied
 * elementwise: s = sin k, c = cos k.  k, s, c: device double [n].  c holds NaN where the
 * cosine-only path that the energies use differs from the sin/cos path in any bit.  Used by the
 * tests to bound them against the C library's sin and cos. */
int tami_selftest_sincos(const double* k, int64_t n, double* s, double* c, tami_stream_t stream);

/* Diagnostic: the kernels' double-precision product on the integer pipes (no term of the paper:
 * how the specialised kernels move FP64 work off the FP64 unit), applied elementwise: mul = a * b
 * rounded to nearest even, bit for bit what the FP64 unit gives for every input, the integer path
 * taken for normal operands with a normal result.  a, b, mul: device double [n]. */
int tami_selftest_imul(const double* a, const double* b, int64_t n, double* mul, tami_stream_t stream);

/* Diagnostic: the call-free variant of that product (imul_ftz), which large tables' specialised
 * kernels use for their per-sample products, applied elementwise: for normal operands with a
 * normal result the IEEE product, bit for bit; otherwise flush to zero — a zero or subnormal
 * operand, or a result below 2^-1022, gives a signed zero, a result above the range a signed
 * infinity, an infinite operand a signed infinity (a NaN against a zero or subnormal operand), a
 * NaN operand a NaN.  a, b, mul: device double [n]. */
int tami_selftest_imul_ftz(const double* a, const double* b, int64_t n, double* mul, tami_stream_t stream);

/* Diagnostic: a probe of the FP64 fma issue rate (not a term of the paper; it measures the
 * ceiling that the evaluation kernels are held against).  Launches `blocks` blocks of 256
 * threads, each running independent fma recurrences, a_k <- m_k a_k + c_k (or the running sum
 * a_k <- m_k c_k + a_k), for `trips` trips; `variant` in [0, TAMI_FP64_RATE_VARIANTS) picks the
 * operand pattern, on which the FP64 unit's rate depends (register-file placement), so a caller
 * measuring the ceiling takes the fastest:
 *   0: 8 recurrences x 8 steps per trip, one multiplier and addend for all (m = 0.9999999,
 *      c = 1e-3);
 *   1: 4 x 8, recurrence k with its own m_k = m - 1e-9 k, c_k = c + 1e-9 k;
 *   2: 4 x 16, the running sums a_k <- m_k c_k + a_k;
 *   3: 3 x 16, as 1.
 * Recurrence k of thread t starts at 1e-3 ((t + k) mod 1024).  `out` (device double
 * [blocks * 256]) receives each thread's sum of its recurrences, and `flops` (host, may be NULL)
 * the flops of the launch (2 per fma).  The caller times the launch on `stream`.  TAMI_EINVAL for a
 * bad variant, blocks < 1, trips < 1 or a NULL `out`. */
#define TAMI_FP64_RATE_VARIANTS 4
int tami_selftest_fp64_rate(int variant, int blocks, int64_t trips, double* out, double* flops, tami_stream_t stream);

void tami_destroy(tami_diagram* d);

#ifdef __cplusplus
}
#endif
#endif /* TAMI_H */
