/*
 * pbits.h -- C ABI of the GB300 p-bit Feynman-path sampler.
 *
 * Method: arXiv 2007.07379, "Emulating Quantum Interference with Generalized
 * Ising Machines".  A circuit of d gate layers on n qubits becomes a layered
 * network of p-bits; a configuration s_1..s_d of the layers is a Feynman path
 * beta -> s_1 -> ... -> s_d = alpha whose weight is the product of the layer
 * matrix elements (Eq. U, Eq. path).  Paths are drawn by Gibbs sampling on the
 * real part of the complex energy E = -ln U (Eq. UE), with zero matrix
 * elements replaced by e^{-J} (Appendix), and each sampled valid path adds its
 * phase exp(-i Im E) to the bin of its end state (Fig. 2, Steps 1-3).
 *
 * Conventions for every call:
 *  - Returns a pb_status (0 = PB_OK, negative = error); nothing throws across
 *    the ABI.  pb_strerror() names a code.
 *  - Inputs are copied: the caller keeps ownership of every pointer it passes.
 *  - Device memory is the caller's: pb_run_create() takes a device workspace
 *    (pointer + byte count; size from pb_workspace_bytes()).  The library
 *    performs no device allocation on these paths.
 *  - Streams are CUDA stream handles cast to uintptr_t (0 = legacy default).
 *  - pb_model and trained pb_mlp objects are immutable after creation and may
 *    be shared; a pb_run belongs to one host thread at a time.
 *  - Host arrays passed for results are caller-owned and sized as stated.
 */
#ifndef PBITS_H
#define PBITS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define PB_API __attribute__((visibility("default")))
#else
#define PB_API
#endif

typedef enum {
  PB_OK = 0,
  PB_EINVAL = -1,   /* malformed argument (bad gate, bad pointer, bad enum) */
  PB_ERANGE = -2,   /* size out of range (n > 32, d > 64, buffer too small) */
  PB_ENOMEM = -3,   /* host allocation failed                               */
  PB_ECUDA = -4,    /* a CUDA runtime call failed                           */
  PB_ETIMEOUT = -5, /* a device-side bounded wait expired (status word)     */
  PB_ESTATE = -6    /* call not valid in the object's current state         */
} pb_status;

/* Gate kinds.  Matrices (rows = output, columns = input, Sec. 2):
 *   H  = (1/sqrt2)[[1,1],[1,-1]]  (Eq. Had)
 *   S  = diag(1, i), T = diag(1, e^{i pi/4})  (diagonal Rz family, Appendix,
 *        with the global phase fixed so that <0|G|0> = 1)
 *   CNOT: control q0, target q1, x_t -> x_t XOR x_c  (Appendix, "CNOT Gate")
 *   CZ  = diag(1,1,1,-1) on (q0, q1)  (diagonal two-qubit gate, Appendix)   */
typedef enum { PB_H = 0, PB_S = 1, PB_T = 2, PB_CNOT = 3, PB_CZ = 4, PB_U = 5, PB_X = 6,
               PB_U2 = 7, PB_CCX = 8 } pb_op;
/* PB_CCX: the Toffoli gate (Appendix, "CCNOT"): controls q0, q1, target q2,
 * s_{q2} -> s_{q2} XOR (s_{q0} AND s_{q1}); every output bit is J-linked to
 * its deterministic value.  The target's link holds an AND, and through it
 * a control's demanded value depends on the other control, so the p-bits
 * around a Toffoli take the general-gate kernels (per-lane link counts);
 * the four bits of the target's factor need four distinct colour classes
 * (PB_ERANGE when the colouring needs more than four).  Not with
 * PB_ELIM_CLAMP (the wires are not affine), the learned proposal or the
 * no-allocation run (PB_EINVAL); pb_model_info's rank reads -1. */
/* PB_X: Pauli X, a deterministic NOT (Appendix, "Pauli-X"): the output is
 * J-linked to the complement of the input; no phase.  A plain gate (no
 * matrix; the model stays a Clifford+T-type model).
 * PB_U2: a two-qubit gate on (q0, q1) with a caller-given 4x4 complex matrix
 * (pb_compile_g), basis index x = x_{q0} + 2 x_{q1} (the order 00, 10, 01, 11
 * of Eq. ET2), rows = outputs.  It must be unitary within 1e-9 with exactly
 * one nonzero entry per column: a permutation of the two bits with phases
 * (SWAP, iSWAP, controlled phases, the Appendix's exchange operator J12,
 * CNOT either way).  Every such permutation is affine over GF(2), so each
 * output bit is J-linked to a copy, a complement, or the XOR of the two
 * inputs; an output equal to the complement of the XOR is rejected
 * (PB_EINVAL).  The phase arg U(pi(x), x) of the column taken is added to
 * the path.
 * A unitary PB_U2 with a column of more than one nonzero is a table gate
 * (Eq. ET2): both outputs are free; the real energy of the entry taken,
 * -ln |U(y, x)| (J for a zero entry, the Appendix's e^{-J}), enters through
 * a second Metropolis factor after the heat-bath proposal (and after the
 * coupling factor of PB_U neighbours): a flip of chain c with energy change
 * dE > 0 is kept when u < floor(2^32 e^{-dE}), u = word (c mod 4) of
 * Philox4x32-10 at (c / 32, t, p | 7 << 16, (c mod 32) / 4).  A path
 * through a zero entry is invalid; the phase arg U(y, x) is recorded.  The
 * columns of |U| need not share a sum, so the amplitude scale has no closed
 * form: pb_model_info's log2z is NaN and pb_run_amplitudes needs
 * l2_normalize (PB_ESTATE otherwise; Fig. 2 Step 4).  Gibbs runs only
 * (PB_EINVAL for the exact samplers). */
/* PB_U: a general one-qubit gate with a caller-given 2x2 complex matrix U
 * (pb_compile_u; Sec. 2 Eq. EB, e.g. the rotated Hadamard of Eq. HadT).  U
 * must be unitary within 1e-9 (max |(U^dagger U - I)_ij|).  Kinds:
 *   diagonal      (U01 = U10 = 0 exactly): the output copies the input, a
 *                 different output bit costs J (a J-linked copy);
 *   anti-diagonal (U00 = U11 = 0 exactly): the output is NOT the input
 *                 (a J-linked NOT);
 *   coupled       (all four entries nonzero): a free output bit with the real
 *                 energy K [s_out != s_in], K = ln(a / b), a = (|U00| + |U11|)/2,
 *                 b = (|U01| + |U10|)/2, |z| = hypot(Re z, Im z) (Eq. EB for a
 *                 unitary: the one-body terms cancel into this two-body term);
 *   one zero entry only: rejected (PB_EINVAL).
 * Every PB_U gate adds the phase arg U(s_out, s_in) to the path. */

/* One gate: layer in [0, d) maps s_layer to s_{layer+1}; 1-qubit gates set
 * q1 = -1, gates on fewer than three qubits q2 = -1.  Each qubit appears at
 * most once per layer. */
typedef struct {
  int32_t op, layer, q0, q1, q2;
} pb_gate;

typedef struct pb_model pb_model;
typedef struct pb_run pb_run;
typedef struct pb_mlp pb_mlp;
typedef struct pb_mh pb_mh;

/* ---- A1: compile (Eqs. UE, EB, ET2; Appendix) ---------------------------
 * Builds the layered J-penalty network of a gate list: p-bit (k, q) is bit q
 * of s_k, k = 1..d, s_0 = input_bits (clamped).  Every output bit of a non-H
 * gate whose value differs from the gate's deterministic map of its inputs
 * costs J; H outputs are free.  Computes the sweep's colour classes, the
 * heat-bath thresholds floor(2^32 / (1 + e^{J v})), v = 0..3, h (H count),
 * M = n d - h and the GF(2) rank of H outputs -> s_d.
 *   n_qubits in [1, 32], n_layers in [1, 64], J >= 0 (finite).
 *   Errors: PB_EINVAL (bad op, qubit, duplicate use in a layer, NULL),
 *           PB_ERANGE (n or d out of range).  *out is NULL on error.
 * Host only; the model is freed with pb_model_free(). */
PB_API int pb_compile(int n_qubits, int n_layers, const pb_gate* gates,
                      int n_gates, uint32_t input_bits, double J,
                      pb_model** out);

/* pb_compile with general one-qubit gates (op PB_U).  mats: 8 doubles per
 * gate row (host, caller-owned; rows of other ops are ignored, NULL allowed
 * when no row is PB_U): Re U00, Im U00, Re U01, Im U01, Re U10, Im U10,
 * Re U11, Im U11 with U_yx = <y|U|x> (row = output bit).  A model with a
 * PB_U gate records complex phase sums instead of the 8 phase classes
 * (pb_run_phase_sums; pb_run_histogram returns PB_ESTATE for it), and a
 * model with a coupled gate samples p_C ~ |U_C| (Eq. weightedS):
 *   Gibbs (PB_GIBBS): the heat-bath draw on the J-penalty energy proposes
 *     x' for p-bit x = (k, q); if x' != x, the flip is accepted when
 *     dK = K_in (1 - 2 e_in) + K_out (1 - 2 e_out) <= 0, else when
 *     u' < min(floor(2^32 e^{-dK}), 2^32 - 1), with K_in, e_in = x XOR
 *     s_{k-1,q} for a coupled gate in layer k-1 on q (else 0, 0), K_out,
 *     e_out = x XOR s_{k+1,q} for a coupled gate in layer k on q (else 0, 0),
 *     and u' the uniform of the tag-6 stream (Metropolis-Hastings with the
 *     heat-bath as proposal, Fig. 2 Steps 1-2).
 *   Exact sampler (PB_ELIM): a coupled output is s_in XOR [u < floor(2^32
 *     b / (a + b))], u the tag-4 uniform of that p-bit (planes j = 0..31 as
 *     for the sweep's draws).
 * The amplitude estimate is 2^{log2z} (sum of phases) / valid, log2z =
 * h/2 + sum over coupled gates of log2(a + b).  Such models may not use
 * PB_ELIM_CLAMP when a gate is coupled, the learned proposal or
 * pb_gibbs_run_noalloc (PB_EINVAL).  Errors as pb_compile, plus PB_EINVAL
 * for a matrix that is not unitary or has a single zero entry. */
PB_API int pb_compile_u(int n_qubits, int n_layers, const pb_gate* gates,
                        int n_gates, const double* mats, uint32_t input_bits,
                        double J, pb_model** out);

/* pb_compile_u with a row stride: mats holds mat_stride doubles per gate
 * row (8: one-qubit matrices only; 32: room for PB_U2's 4x4 matrix,
 * mats[32 i + 2 (4 y + x)] = Re <y|U|x>, + 1 = Im; a PB_U row uses its first
 * 8 as in pb_compile_u).  PB_U2 rows need mat_stride >= 32 (PB_EINVAL). */
PB_API int pb_compile_g(int n_qubits, int n_layers, const pb_gate* gates,
                        int n_gates, const double* mats, int mat_stride,
                        uint32_t input_bits, double J, pb_model** out);

typedef struct {
  int32_t n, d;        /* qubits, gate layers                          */
  int32_t n_pbits;     /* n (d + 1), input layer included              */
  int32_t h;           /* H gates = free p-bits of a valid path        */
  int32_t M;           /* linked (non-H) p-bits                        */
  int32_t rank;        /* GF(2) rank of the map H outputs -> s_d       */
  double J;
  uint32_t input_bits;
  uint32_t thr[4];     /* heat-bath thresholds for |v| = 0..3         */
  int32_t colour_size[4];
  int32_t n_u;         /* PB_U gates                                   */
  int32_t n_coupled;   /* coupled PB_U gates (free outputs)            */
  double log2z;        /* log2 of the estimator scale (h/2 + ...)      */
} pb_model_info_t;

PB_API int pb_model_info(const pb_model* m, pb_model_info_t* info);
/* Colour class (0..3) of every p-bit, row-major [d][n] (row k-1 = layer k). */
PB_API int pb_model_colours(const pb_model* m, int32_t* colour);
PB_API void pb_model_free(pb_model* m);

/* ---- runs ---------------------------------------------------------------
 * A run holds the chains of one or more models ("batched" when more than
 * one).  Chains are bit-sliced: 32 chains form a group and share one 32-bit
 * word per p-bit (bit c = chain 32 g + c).  The random numbers of chain c at
 * sweep t for p-bit p = (k-1) n + q are Philox4x32-10 outputs under key =
 * seed at counter (c / 32, t, p | tag << 16, j / 4), word j % 4, j = 0..31:
 * bit c % 32 of word j is bit 31-j of the chain's uniform u (tag 0 = sweep,
 * tag 1 = initial H and coupled-PB_U outputs, tag 6 = the Metropolis
 * acceptance of coupled p-bits).  A p-bit whose violation count changes by v
 * when it goes 0 -> 1 is redrawn as [v < 0] XOR [u < thr[|v|]]  (heat-bath,
 * Fig. 2 Steps 1-2).  One sweep visits the model's colour classes in
 * increasing order (pb_model_colours: a DSATUR colouring of the p-bits'
 * interaction graph, two to four classes; p-bits of one class share no
 * link, so a class is redrawn in parallel). */
enum { PB_GIBBS = 0, PB_LEARNED = 1, PB_ELIM = 2, PB_ELIM_CLAMP = 3 };
/* PB_ELIM: the exact sampler on the eliminated network (Appendix: without
 * the link constraints every non-H bit is a function of the previous layer
 * and each H output a fair coin).  A "sweep" of such a run draws, for every
 * chain, a fresh path from the clamped input: H output p = (k-1) n + q of
 * chain c at sample t is bit c % 32 of word 0 of Philox4x32-10 at counter
 * (c / 32, t, p | 4 << 16, 0), every other bit its deterministic value; each
 * recorded sample is valid and is binned like a Gibbs sample.  The samples
 * are i.i.d. and uniform over the 2^h valid paths (the comparator for the
 * Gibbs and learned samplers).  All models of a run use one sampler;
 * pb_run_set_shape / pb_run_tune have no effect on a PB_ELIM run and the
 * learned-proposal calls reject it.
 * PB_ELIM_CLAMP: the exact sampler with the end state fixed to one output
 * (cfg.alphas = {alpha}, n_alphas = 1; "for a given input beta and output
 * alpha", Sec. 3).  Every wire bit is affine over GF(2) in the H outputs x
 * (in p order), s_d = A x + c; the paths to alpha solve A x = alpha + c.  With
 * the reduced row echelon form of [A | alpha + c] the free variables
 * (non-pivot columns, increasing) take the draws z_b -- bit c % 32 of word
 * b % 4 of Philox4x32-10 at (c / 32, t, (b / 4) | 5 << 16, 0) -- and each
 * pivot variable its row's right-hand side XOR the free variables in that
 * row.  The amplitude is 2^{h/2 - r} sum_phi cnt[phi] w^phi / T (SE smaller
 * than the unclamped estimator's by 2^{r/2}); an unreachable alpha draws
 * nothing and reads 0.  PB_ELIM and PB_ELIM_CLAMP models may share a run. */

typedef struct {
  uint64_t seed;          /* Philox key                                        */
  uint32_t chains;        /* >= 1 (any count; groups of 32, the last ragged)    */
  uint32_t burn_in;       /* first recorded sweep (absolute index)             */
  uint32_t record_every;  /* >= 1: record after sweep t when t >= burn_in and
                             (t - burn_in) % record_every == 0                  */
  uint32_t n_batches;     /* SE batches over chain groups (0 = automatic)      */
  const uint32_t* alphas; /* bins to record; NULL = full 2^n histogram (n<=22)  */
  int32_t n_alphas;
  int32_t sampler;        /* PB_GIBBS, PB_LEARNED, PB_ELIM or PB_ELIM_CLAMP      */
  const pb_mlp* proposal; /* PB_LEARNED: the network (must outlive the run)      */
  uint32_t mh_every;      /* PB_LEARNED: sweeps per move period (>= 1)           */
  uint32_t group0;        /* global index of the first chain group: the chains
                             here are 32*group0 ... (multi-rank sharding; the
                             draws depend on the global index only)             */
} pb_run_cfg;

/* PB_LEARNED: Gibbs sweeps with the learned proposal as a run mode (Fig. 2
 * Step 1 with the network q as the proposal, Steps 2-3 unchanged).  Every
 * call pb_run_sweeps(n) runs n / mh_every periods, each one suffix move of
 * every PB_LEARNED model of the run (the move of pb_mh_moves: k* from
 * SplitMix64 of the seed and the model's move count, proposal drawn layer by
 * layer from `proposal`, Metropolis-Hastings acceptance on the J energy;
 * the move count starts at 0 with the run) followed by mh_every sweeps,
 * then n mod mh_every sweeps without a move.  The whole sequence is one
 * CUDA graph whose periods are counted down on the device (a while node),
 * so no host step runs between moves.  The records of the sweeps are the
 * samples; the moves keep the sampled law whatever the network.  The
 * network's weights are read at every move (training between calls takes
 * effect).  Requirements (PB_EINVAL otherwise): proposal != NULL with the
 * model's n and d and k_in <= 96, n <= 32 (the fused inference kernel), a
 * plain model (no PB_U, PB_U2 or PB_CCX gate), mh_every >= 1, and the same
 * mh_every for all PB_LEARNED models of a run (which may hold PB_GIBBS models
 * too; all draw from their own streams).  pb_run_moves reads the moves done
 * and accepted; pb_run_wait also returns PB_ETIMEOUT from a network's
 * status word; checkpoints hold the move counters. */

/* Bytes of device workspace that pb_run_create() needs for these models. */
PB_API int pb_workspace_bytes(pb_model* const* models, const pb_run_cfg* cfgs,
                              int n_models, size_t* bytes);

/* Lays out the caller's device workspace (>= pb_workspace_bytes, 256-byte
 * aligned), uploads the tables, zeroes the counters and initialises every
 * chain to a valid path with random H outputs (tag-1 stream).  Asynchronous
 * on `stream`.  Errors: PB_EINVAL, PB_ERANGE (workspace too small), PB_ECUDA. */
PB_API int pb_run_create(pb_model* const* models, const pb_run_cfg* cfgs,
                         int n_models, void* d_workspace, size_t workspace_bytes,
                         uintptr_t stream, pb_run** out);

/* Enqueues n_sweeps further sweeps of every chain of every model (one
 * launch, replayed from a CUDA graph cached per n_sweeps; asynchronous).
 * Sweep indices continue from the previous call.  n_sweeps <= 2^26 per call
 * (PB_ERANGE otherwise); the total over a run stays below 2^32. */
PB_API int pb_run_sweeps(pb_run* run, uint32_t n_sweeps);

/* Waits for the run's stream; returns PB_OK, PB_ECUDA or the device status
 * word (PB_ETIMEOUT when a bounded device wait expired, in the run's kernels
 * or, for PB_LEARNED models, in their networks' kernels). */
PB_API int pb_run_wait(pb_run* run);

/* Moves done and proposals accepted (one per chain and move) of a
 * PB_LEARNED model (synchronous).  PB_ESTATE for another sampler; moves /
 * accepted may be NULL. */
PB_API int pb_run_moves(pb_run* run, int model, uint64_t* moves, uint64_t* accepted);

/* Histogram of model `model` (synchronous): counts[bin*8 + b] = valid samples
 * that ended in bin with phase w^b (w = e^{i pi/4}) summed over batches;
 * bins = n_alphas or 2^n.  Any of the three pointers may be NULL. */
PB_API int pb_run_histogram(const pb_run* run, int model, uint64_t* counts,
                            uint64_t* valid_total, uint64_t* samples_total);

/* Phase sums of model `model` (synchronous), any model: per bin, summed over
 * batches, re + i im = sum over the valid recorded samples ending there of
 * e^{i arg U_C} (FP64 sums of the device's per-sample phasors: fixed-point
 * angles of 2^-32 turn per PB_U gate, the phasor by sincospif in FP32, each
 * term within 3e-7 of the exact one), counts = their
 * number.  For a model without PB_U gates the sums are formed from the
 * exact phase classes.  Any pointer may be NULL. */
PB_API int pb_run_phase_sums(const pb_run* run, int model, double* re, double* im,
                             uint64_t* counts, uint64_t* valid_total, uint64_t* samples_total);

/* Amplitude estimates (Eq. U23, uniform valid paths; computed on the device):
 * psi[bin] = 2^{h/2} sum_b counts[bin][b] w^b / valid_total (with PB_U gates
 * 2^{log2z} times the phase sum / valid_total), and its standard
 * error from batch means over chain groups (Eq. U26).  l2_normalize != 0
 * divides by the L2 norm over the recorded bins (Fig. 2 Step 4).
 * re, im, se: host arrays of `bins` doubles (se may be NULL). */
PB_API int pb_run_amplitudes(const pb_run* run, int model, int l2_normalize,
                             double* re, double* im, double* se);

/* Chain words of model `model` (synchronous copy): layout
 * [group][k-1][q] u32, groups = ceil(chains/32); `bytes` must be >=
 * groups * d * n * 4. */
PB_API int pb_run_get_state(const pb_run* run, int model, uint32_t* words,
                            size_t bytes);
PB_API int pb_run_set_state(pb_run* run, int model, const uint32_t* words,
                            size_t bytes);

typedef struct {
  uint64_t sweeps_done;   /* sweeps enqueued so far (per chain)            */
  double flips;           /* p-bit updates enqueued: chains * sweeps * n d */
  double last_ms;         /* device time of the last pb_run_sweeps call    */
  double flips_per_s;     /* flips of that call / its device time          */
} pb_run_stats_t;
PB_API int pb_run_stats(pb_run* run, pb_run_stats_t* stats);

/* CTA shape of the sweep launches: consumer threads (redraw one colour
 * class, 32..224), producer threads (the Philox planes the consumers
 * compare against, made one or two colour steps ahead, 32..352), both
 * multiples of 32, plus one recorder warp; blocks_per_sm
 * caps the persistent grid of batched runs (0 = as many as fit).  A run
 * with PB_U models takes at most 512 threads (consumers + producers + 32;
 * PB_ERANGE otherwise).  The results do not depend on the shape. */
PB_API int pb_run_set_shape(pb_run* run, int consumers, int producers, int blocks_per_sm);
PB_API int pb_run_get_shape(const pb_run* run, int* consumers, int* producers, int* blocks_per_sm,
                            int* grid);
/* Autotuner: times trial_sweeps sweeps of each candidate shape on the run
 * itself (the run's state, counters and sweep index are restored after
 * every trial, so the run is unchanged) and keeps the fastest.  cache_path
 * (may be NULL): a text file of earlier results keyed by the run's (n, d,
 * chains) list; a hit applies the cached shape without trials.  *best_ms
 * (may be NULL) receives the time of trial_sweeps sweeps with that shape. */
PB_API int pb_run_tune(pb_run* run, uint32_t trial_sweeps, const char* cache_path, double* best_ms);

/* Checkpoint: chain words, counters and the sweep index of every model (and
 * the move counters of PB_LEARNED models).
 * bytes_needed is written when host_buf is NULL.  Restore puts them back;
 * since the draws are counter-based the resumed run is bit-identical to an
 * uninterrupted one. */
PB_API int pb_run_checkpoint(const pb_run* run, void* host_buf, size_t bytes,
                             size_t* bytes_needed);
PB_API int pb_run_restore(pb_run* run, const void* host_buf, size_t bytes);
PB_API void pb_run_free(pb_run* run);

/* Test hook: fills out[i*4 .. i*4+3] with Philox4x32-10 of counters
 * ctr[i*4..] under key (k0, k1) on the device (d_ctr, d_out are device
 * pointers, count counters). */
PB_API int pb_philox_fill(const uint32_t* d_ctr, uint32_t k0, uint32_t k1,
                          uint32_t count, uint32_t* d_out, uintptr_t stream);

/* ---- a run that allocates nothing ------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory where they call the library (a plug-in
 * whose host application owns every device allocation, or code that runs
 * while a memory budget is frozen).  It is one complete plain Gibbs run (the
 * same kernels and results as pb_run_create + pb_run_sweeps + the histogram)
 * whose scratch -- run header, tables, chain state, counters -- lives in a
 * fixed 16 MiB array in device memory that every GPU loading the library
 * holds until the process exits.  It calls no allocator.
 *   m        compiled model, n <= 16 (the full 2^n histogram is recorded).
 *   cfg      as for pb_run_create; alphas must be NULL, sampler PB_GIBBS.
 *            The run starts at sweep 0 from freshly drawn valid paths.
 *   n_sweeps sweeps to run (<= 2^26).
 *   d_counts device buffer of 2^n * 8 u64: counts[alpha*8 + b] of valid
 *            samples ending in alpha with phase w^b (the histogram).
 *   d_totals device buffer of 2 u64: valid samples, all samples.
 * Asynchronous on `stream`; the outputs are complete when the stream
 * reaches them.  Returns PB_ERANGE when the run does not fit the array
 * (groups * n * d * 4 + 2^n * 64 bytes plus tables must stay below 16 MiB,
 * e.g. 4096 chains of n=12, d=20), PB_EINVAL for bad arguments.
 * The first call on a device looks up the array's device address and opts
 * the sweep kernels into their shared memory (once per device, with that
 * device current; the lookup assumes the device's context is not reset
 * afterwards).  The call copies its tables from host memory, so it cannot be
 * recorded into a CUDA graph: on a stream that is capturing it returns
 * PB_ESTATE and enqueues nothing.  All calls share the one array and each
 * leaves its contents behind: every call clears what must start at zero, and
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race on it. */
PB_API int pb_gibbs_run_noalloc(const pb_model* m, const pb_run_cfg* cfg, uint32_t n_sweeps,
                                unsigned long long* d_counts, unsigned long long* d_totals,
                                uintptr_t stream);

/* ---- learned proposal network (the paper trains nothing; this is the
 * proposal q(s_j | s_{j-1}, j) of the Metropolis-Hastings suffix move) -----
 * q(s_j | s_{j-1}, j) = prod_q sigma(l_q)^{s_j[q]} sigma(-l_q)^{1-s_j[q]},
 * l = W3 relu(W2 relu(W1 x + b1) + b2) + b3, x = [2 s_{j-1} - 1 (n),
 * onehot(j-1) (d), zeros] (k_in = n + d rounded up to 16).  BF16 tensor-core
 * GEMMs with fp32 accumulation, fp32 master weights, Adam (0.9, 0.999, 1e-8).
 * The caller owns the device workspace (pb_mlp_workspace_bytes); hidden in
 * [16, 256] (multiple of 16), batch a multiple of 128 (the largest number of
 * rows one call processes).  Calls are asynchronous on the creation stream
 * unless stated. */
PB_API int pb_mlp_workspace_bytes(int n, int d, int hidden, int batch, size_t* bytes);
/* Weights uniform(+-1/sqrt(fan_in)) from SplitMix64(seed), biases 0. */
PB_API int pb_mlp_create(int n, int d, int hidden, int batch, uint64_t seed, void* d_workspace,
                         size_t workspace_bytes, uintptr_t stream, pb_mlp** out);
/* dims[6] = n, d, hidden, k_in, batch, number of fp32 parameters. */
PB_API int pb_mlp_info(const pb_mlp* mlp, int* dims);
/* Failure detection of the network's kernels.  Every wait in them for the
 * tensor cores or a bulk copy is bounded; a wait that runs out leaves the
 * kernel (after draining what it started) and sets PB_ETIMEOUT in a status
 * word of the network's workspace.  *status receives that word (PB_OK = 0,
 * else PB_ETIMEOUT); clear != 0 resets it.  Synchronizes the network's
 * stream; call it after the launches that used the network (forward,
 * backward, training, MH moves on a run's stream) have completed.
 * Errors: PB_EINVAL (NULL), PB_ECUDA. */
PB_API int pb_mlp_status(pb_mlp* mlp, int clear, int* status);
/* Self-test of that bounded wait, with nothing else in flight: one thread
 * initialises a one-arrival mbarrier, arrives on it (arrive != 0) or not,
 * and waits for its first phase for at most max_iters tries (1 .. 2^20).
 * *status receives PB_OK when the wait completed, PB_ETIMEOUT when it ran
 * out (arrive == 0).  Runs on the default stream and synchronizes the
 * device; calls must not overlap (one status word in the library).
 * Errors: PB_EINVAL (NULL status, max_iters out of range), PB_ECUDA. */
PB_API int pb_selftest_wait(int arrive, uint32_t max_iters, int* status);
/* Flat fp32 parameters W1 [h x k_in], b1, W2 [h x h], b2, W3 [npad x h]
 * (npad = n rounded up to 16; rows >= n are zero), b3 [npad].  get != 0
 * reads them to host, get == 0 loads them.  Synchronous. */
PB_API int pb_mlp_params(pb_mlp* mlp, float* host, int get);
/* Gradients from the last pb_mlp_backward, same flat layout.  Synchronous. */
PB_API int pb_mlp_grads(pb_mlp* mlp, float* host);
/* d_x: device bf16 [rows x k_in]; d_logits: device fp32 [rows x n]. */
PB_API int pb_mlp_forward(pb_mlp* mlp, const void* d_x, int rows, float* d_logits);
/* Same output from the fused inference kernel (one tcgen05 kernel for the
 * three layers; k_in <= 96, n <= 32); the MH move uses this path. */
PB_API int pb_mlp_forward_fused(pb_mlp* mlp, const void* d_x, int rows, float* d_logits);
/* Gradients of the mean binary cross-entropy against d_target (device fp32
 * 0/1, [rows x n]); rows a multiple of 8; d_loss (device fp32) may be NULL. */
PB_API int pb_mlp_backward(pb_mlp* mlp, const void* d_x, const float* d_target, int rows,
                           float* d_loss);
/* One Adam step with the gradients of the last pb_mlp_backward. */
PB_API int pb_mlp_adam(pb_mlp* mlp, float lr);
PB_API void pb_mlp_free(pb_mlp* mlp);

/* ---- learned proposal: Metropolis-Hastings suffix move (Fig. 2 Steps 1-2,
 * "Metropolis-Hastings" acceptance on |e^{-E}|) -------------------------------
 * One move per call per move index: k* in 1..d is drawn from the seed and
 * the move index; every chain of model `model` proposes s'_{k*}..s'_d layer
 * by layer from the network and accepts with
 *   min(1, e^{-J (v(s') - v(s))} q(s_{k*..d} | s_{k*-1}) / q(s'_{k*..d} | s_{k*-1})),
 * v = violated links of layers k*..d (Re E = J v).  The move keeps the
 * sampled distribution (the J-penalty Boltzmann law of the Gibbs sweeps), so
 * it is interleaved with pb_run_sweeps, whose records count the samples.
 * A pb_mh object ties a run's model to a network and a caller device
 * workspace of pb_mh_workspace_bytes (256-byte aligned); the run and the
 * network must outlive it.  pb_mh_moves enqueues moves on the run's stream
 * (each replayed from a CUDA graph captured once per k*); pb_mh_stats
 * returns the moves done and proposals accepted (synchronous), and returns
 * PB_ETIMEOUT when a bounded wait in the network's kernels has run out
 * (pb_mlp_status; the moves since then are not valid). */
PB_API int pb_mh_workspace_bytes(const pb_run* run, int model, size_t* bytes);
PB_API int pb_mh_create(pb_run* run, int model, pb_mlp* mlp, void* d_workspace,
                        size_t workspace_bytes, pb_mh** out);
PB_API int pb_mh_moves(pb_mh* mh, uint32_t n_moves);
PB_API int pb_mh_stats(pb_mh* mh, uint64_t* moves, uint64_t* accepted);
PB_API void pb_mh_free(pb_mh* mh);
/* Appends the valid paths among the chains of `model` (per-chain layer
 * words s_1..s_d, d u32 each) to d_paths at the device counter *d_count
 * (u64, caller-initialised), up to `capacity` paths.  Workspace as for
 * pb_mh_moves.  Synchronous. */
PB_API int pb_run_collect_paths(pb_run* run, int model, void* d_workspace, size_t workspace_bytes,
                                uint32_t* d_paths, uint64_t capacity, uint64_t* d_count);
/* `steps` Adam steps of the network on batches of `rows` (input s_{j-1}, j;
 * target s_j) drawn uniformly from the n_paths collected paths (Philox,
 * key = seed); the loss of each step goes to d_losses[step] (device fp32,
 * may be NULL).  Asynchronous on the network's stream. */
PB_API int pb_mlp_train_paths(pb_mlp* mlp, const uint32_t* d_paths, uint64_t n_paths, uint32_t beta,
                              int steps, int rows, float lr, uint64_t seed, float* d_losses);

/* ---- BF16 tensor-core GEMM (tcgen05), used by the learned proposal ----------
 * D[M x N] = epilogue(alpha * A[M x K] * B[N x K]^T); A, B bf16 row-major
 * with K contiguous (leading dimensions lda, ldb in elements, multiples of 8,
 * 16-byte aligned rows), fp32 accumulation.  flags: 1 ReLU, 2 store bf16
 * (else fp32), 4 accumulate into fp32 D, 8 multiply by [mask(row,col) > 0]
 * (mask bf16, leading dimension ldm).  dbias (fp32, N) may be NULL.  All
 * pointers are device pointers; asynchronous on `stream`.  Errors: PB_EINVAL
 * (shapes, alignment), PB_ECUDA. */
PB_API int pb_gemm_bf16(const void* dA, int lda, const void* dB, int ldb, void* dD, int ldd,
                        const float* dbias, const void* dmask, int ldm, int M, int N, int K,
                        int flags, float alpha, uintptr_t stream);

/* ---- column sampling of the period-finding circuit (Sec. 5.2 and its
 * column-sampling figure) ------------------------------------------------
 * Sample i is a column x_i (0 <= x_i < 2^n) of the inverse QFT on the first
 * register (t = n bits, Sec. 5.2); its entries 2^{-n/2} e^{2 pi i k x_i / 2^n}
 * are added to column y_i = a^{x_i} mod N of psi, and
 *   prob[k] = sum_y |psi[k, y]|^2 / T,  k = 0 .. 2^n - 1
 * (sums to 1 when the drawn columns are distinct; every column once gives
 * the exact distribution of the first register).  The order r of a mod N
 * shows as r peaks near multiples of 2^n / r (Sec. 5.2: T = gamma r
 * samples, 2 <= gamma <= 4).
 * Device computation: modular exponentiation, a sort of the samples by
 * (y, x), then per k a walk over the sorted samples (FP32 phasors: the
 * exact integer phase k0 x mod 2^n of a 32-k block times the sample's table
 * of e^{2 pi i j x / 2^n}, j < 32; each term within about 5e-7 of the exact
 * one; FP64 output).
 *   N in [2, 2^32), n in [1, 32], 1 <= T <= 2^26, x: host array of T column
 *   indices < 2^n (caller-owned; the draws are the caller's, so that they
 *   can be shared and reproduced).  d_workspace: device, 256-byte aligned,
 *   >= pb_shor_workspace_bytes(n, T).  d_prob: device, 2^n doubles (written).
 *   y_out: optional host array of T u64 receiving y_i (synchronous when
 *   given).  Asynchronous on `stream` otherwise.
 *   Errors: PB_EINVAL (NULL, misaligned, x_i >= 2^n), PB_ERANGE (sizes),
 *   PB_ECUDA. */
PB_API int pb_shor_workspace_bytes(int n, uint32_t T, size_t* bytes);
PB_API int pb_shor_columns(uint64_t N, uint64_t a, int n, const uint32_t* x, uint32_t T,
                           void* d_workspace, size_t workspace_bytes, double* d_prob,
                           uint64_t* y_out, uintptr_t stream);
/* Peaks of prob (2^n doubles on the device): the local maxima in k (cyclic;
 * >= the left neighbour and > the right one) with prob >= threshold.
 * *count = their number; positions (optional host array) receives the first
 * max_positions of them in increasing k; *max_prob (optional) the largest
 * prob.  d_workspace: device, 256-byte aligned, >= 256 + 8 max_positions
 * bytes (a column-sampling workspace may be reused).  Synchronous. */
PB_API int pb_shor_peaks(const double* d_prob, int n, double threshold, void* d_workspace,
                         size_t workspace_bytes, uint64_t* positions, uint32_t max_positions,
                         uint32_t* count, double* max_prob, uintptr_t stream);

PB_API const char* pb_strerror(int status);
PB_API int pb_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PBITS_H */
