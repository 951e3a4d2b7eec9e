/*
 * hs.h -- C ABI of libhs: diagonal-budgeted Trotterization on one GB300 GPU.
 *
 * The library builds the per-step Trotter factors of a Pauli-sum Hamiltonian
 * (Eq. 3, Eq. 4) grouped under a diagonal budget (Sec. 3.1, Eq. 5), stores each
 * factor in the compact diagonal layout of Eq. 6 / Tab. 1 (an offset list plus
 * dense complex diagonals of length N - |d|), and applies the factors to
 * 2^n-amplitude state vectors for many steps (the evolution loop of Alg. 3,
 * with the diagonal-times-vector product of Alg. 1 as the unit of work).
 *
 * Conventions used by every entry point:
 *   - Pauli labels are strings over {I,X,Y,Z}, all of length n_qubits; the
 *     rightmost character acts on qubit 0, which is bit 0 of the basis index.
 *     A term's masks are x (X or Y present) and z (Z or Y present); its action
 *     is P|b> = i^popcount(x&z) (-1)^popcount(z&b) |b xor x>.
 *   - Coefficients are real (H is Hermitian).  theta_j = c_j * (t / n_steps);
 *     term j's rotation is R_j = cos(theta_j) I - i sin(theta_j) P_j, and term 0
 *     acts first, within a factor and within a step.
 *   - Grouping: terms are taken in input order; a term joins the open factor
 *     iff the factor is empty, or the factor's structural offset count after
 *     adding it stays <= diag_budget, or adding it leaves the offset set
 *     unchanged.  A single term above the budget still forms its own factor.
 *   - Offsets are d = col - row; a factor's offsets are listed 0 first, then by
 *     |d| ascending, negative before positive (Tab. 1 gives [0, -3, 3]).
 *     Element i of diagonal d holds entry (row, col) with i = min(row, col).
 *   - State vectors are caller-owned DEVICE buffers of interleaved complex
 *     numbers (float2 for HS_C64, double2 for HS_C128), n_rhs states of 2^n
 *     amplitudes each, rhs-major and contiguous, 16-byte aligned.
 *   - cuda_stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Unless stated otherwise a call only enqueues work on it.
 *   - Every entry point returns HS_OK (0) or a negative code; on failure
 *     hs_last_error() returns a message (thread-local), no output object is
 *     created, and a call rejected before any launch leaves caller buffers
 *     untouched.
 *   - The library never frees caller memory.  hs_factors objects are owned
 *     by the library (device-resident, immutable after the build except for
 *     the values of a time-dependent set, which hs_evolve_td and
 *     hs_factors_set_drive rebuild) and freed only by hs_free_factors.
 */
#ifndef HS_H
#define HS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  HS_OK = 0,
  HS_EINVAL = -1,   /* bad argument: label, length, n_qubits, t, steps, budget, coefficient */
  HS_ENOMEM = -2,   /* device allocation failed */
  HS_ECUDA = -3,    /* a CUDA runtime call or kernel launch failed */
  HS_ETIMEOUT = -4, /* reserved for a bounded device-side wait that ran out; no kernel of this
                       library waits on a flag, a peer or an mbarrier (dependent launches
                       are ordered by the stream), so no call returns it */
  HS_EDTYPE = -5    /* dtype mismatch between arguments */
};

typedef enum { HS_C64 = 1, HS_C128 = 2 } hs_dtype;

#define HS_MAX_QUBITS 30

/* Opaque factor set: G factors for one (H, t, n_steps, diag_budget, dtype). */
typedef struct hs_factors hs_factors;

/* Build the per-step factors of H = sum_j coeffs[j] P_j for time step
 * t / n_steps (Eq. 4) under diag_budget (Eq. 5 read as a cap on each factor's
 * diagonal count), in the compact layout of Eq. 6.
 *   pauli_terms : n_terms NUL-terminated labels (see conventions); host memory.
 *   coeffs      : n_terms finite real coefficients; host memory.
 *   t > 0 and finite; n_steps >= 1; diag_budget >= 1.
 *   dtype       : storage precision of the factor values.  Values are always
 *                 computed in FP64 on the GPU (cos/sin of the angles and the
 *                 group products) and rounded once to FP32 for HS_C64.
 *   out         : receives the new object; set to NULL on failure.
 * The grouping and offsets are planned on the host; the values are computed
 * by kernels enqueued on cuda_stream, into device memory allocated in stream
 * order on cuda_stream (use the factors on that stream, or after it).  Errors: HS_EINVAL (invalid label,
 * labels of different lengths, n_qubits outside 1..HS_MAX_QUBITS, non-finite
 * or non-positive t, n_steps < 1, diag_budget < 1, non-finite coefficient,
 * a factor with more than 4096 diagonals or an x-mask set above 64 elements),
 * HS_ENOMEM, HS_ECUDA. */
int hs_build_factors(const char* const* pauli_terms, const double* coeffs, size_t n_terms, double t,
                     int n_steps, int diag_budget, hs_dtype dtype, void* cuda_stream, hs_factors** out);

/* Term canonicalisation alone (the HamLib Pauli strings of Sec. 4.4 turned
 * into the masks every other entry point takes): label j becomes x[j] (bit q
 * set where character n_qubits-1-q is X or Y) and z[j] (Z or Y), so that
 * P_j|b> = i^popcount(x&z) (-1)^popcount(z&b) |b xor x>.  labels: n_terms
 * NUL-terminated host strings of equal length 1..HS_MAX_QUBITS; x, z: host
 * arrays of n_terms entries, written only on success; *n_qubits receives the
 * label length.  Host only, no GPU call.  Errors: HS_EINVAL (NULL argument,
 * no terms, invalid character, labels of different lengths). */
int hs_parse_terms(const char* const* labels, size_t n_terms, uint64_t* x, uint64_t* z, int* n_qubits);

/* Same as hs_build_factors with pre-parsed terms: x[j], z[j] are the flip and
 * phase masks of term j (bits >= n_qubits must be zero). */
int hs_build_factors_masks(const uint64_t* x, const uint64_t* z, const double* coeffs, size_t n_terms,
                           int n_qubits, double t, int n_steps, int diag_budget, hs_dtype dtype,
                           void* cuda_stream, hs_factors** out);

/* Same with a product formula of the given order (the higher-order formulas
 * the paper names as future work; readings of this library): 1 = the
 * first-order step above; 2 = symmetric Strang splitting, one step applying
 * every term with angle c_j dt/2 in input order and then in reverse order;
 * 4 = Suzuki's fourth-order recursion S2(p dt) S2(p dt) S2((1-4p) dt) S2(p dt)
 * S2(p dt), p = 1/(4 - 4^(1/3)), of that Strang step S2.  The grouping is the
 * first-order one; for order 2 each group is stored twice (forward factor
 * F_g = R_last ... R_first and reversed factor R_first ... R_last, both at
 * dt/2), for order 4 twice per angle (p dt/2 and (1-4p) dt/2).  One step
 * applies the factors hs_factors_sequence lists.  Errors as hs_build_factors,
 * and HS_EINVAL for another order. */
int hs_build_factors_ex(const uint64_t* x, const uint64_t* z, const double* coeffs, size_t n_terms,
                        int n_qubits, double t, int n_steps, int diag_budget, int order, hs_dtype dtype,
                        void* cuda_stream, hs_factors** out);

/* Build options (flags of hs_build_factors_flags). */
enum {
  HS_BUILD_DEFER_DIAGONALS = 1 /* build the planned structure, the per-term records and the value
                                  tables now, and the stored diagonals only when a call first needs
                                  them (plain or staged evolution, hs_apply_factor, hs_factor_get,
                                  a staged batch), on that call's stream; the register sweeps
                                  generate the factors from the records and never need them.
                                  Static sets only (time-dependent builds ignore the flag). */
};

/* hs_build_factors_ex with build options (flags: a combination of the
 * HS_BUILD_* values above, 0 = hs_build_factors_ex).  The device memory of
 * the diagonals is allocated at build time either way.  A deferred set's
 * first use that needs the diagonals builds them on its own stream; uses on
 * other streams must be ordered after it by the caller.  Errors as
 * hs_build_factors_ex, and HS_EINVAL for an unknown flag. */
int hs_build_factors_flags(const uint64_t* x, const uint64_t* z, const double* coeffs, size_t n_terms,
                           int n_qubits, double t, int n_steps, int diag_budget, int order, hs_dtype dtype,
                           int flags, void* cuda_stream, hs_factors** out);

/* The product-formula order of a factor set and the factors one step applies
 * (indices for hs_factor_get, in application order).  seq may be NULL (then
 * only the length is returned); otherwise it holds capacity ints.  Errors:
 * HS_EINVAL (NULL f, capacity too small). */
int hs_factors_sequence(const hs_factors* f, int* order, int* seq, int capacity, int* seq_len);

/* Structural dry run on the host only (no GPU call): the grouping, each
 * factor's offsets in canonical order and the device bytes of the padded
 * factor values -- what the diagonal-set estimation paragraph (Sec. 3.2)
 * computes before any numeric work so that storage is allocated once.
 * Same grouping rule and limits as hs_build_factors (coefficients are not
 * needed).  *n_factors and *n_offsets are always set on success; the arrays
 * (group_first/group_last/n_diags: capacity_factors entries, offsets:
 * capacity_offsets entries) are filled only if they are non-NULL and large
 * enough, otherwise left untouched.  value_bytes may be NULL.
 * Errors: HS_EINVAL, HS_EDTYPE. */
int hs_plan_factors(const uint64_t* x, const uint64_t* z, size_t n_terms, int n_qubits, int diag_budget,
                    hs_dtype dtype, int* n_factors, int* n_offsets, int* group_first, int* group_last, int* n_diags,
                    int64_t* offsets, int64_t* value_bytes, int capacity_factors, int capacity_offsets);

/* Host-only launch schedule of n_steps steps (no GPU call): the factor
 * applications in the order the sweeps apply them, with the factors grouped
 * and stored as hs_build_factors_ex(order) would, tiles of tile_bits local
 * qubits keeping the low_bits lowest ones, at most max_fuse (0 = 64)
 * applications per sweep.  commuting = 0: the formula's order, each sweep a
 * run of consecutive applications (the staged sweep's schedule); 1: the
 * register sweep's schedule, in which a sweep may also take a later
 * application that commutes with every application it passes over (each
 * Pauli term of the one commutes with each term of the other), so that the
 * product is the formula's up to the order of commuting factors (the
 * product formula of Sec. 2 applies the same factors; only their rounding
 * differs).  A factor that does not fit a tile is a sweep of its own.
 * Outputs: *n_apps (= n_steps x step length) and *n_sweeps always; if the
 * three arrays are non-NULL and capacity >= *n_apps, application k is factor
 * app_factor[k] (an index for hs_factor_get; it holds the terms of group
 * app_factor[k] mod G, G the count hs_plan_factors gives) of step
 * app_step[k], applied by sweep sweep_of[k] (nondecreasing).  Errors:
 * HS_EINVAL, HS_EDTYPE. */
int hs_plan_schedule(const uint64_t* x, const uint64_t* z, size_t n_terms, int n_qubits, int diag_budget, int order,
                     hs_dtype dtype, int n_steps, int tile_bits, int low_bits, int max_fuse, int commuting,
                     int* n_apps, int* n_sweeps, int* app_factor, int* app_step, int* sweep_of, int capacity);

/* Evolve psi in place by n_steps Trotter steps: for each step, apply the
 * factors F_0, ..., F_{G-1} in order (Alg. 3's loop, x <- U x, with U the
 * ordered product of the grouped factors).  psi: device buffer of n_rhs
 * states (see conventions), dtype equal to the factors'.  n_steps >= 0
 * (0 is a no-op), n_rhs >= 1.  Work is enqueued on cuda_stream; the call may
 * allocate a temporary device buffer of one state set when a factor cannot be
 * applied tile-locally, and frees it stream-ordered.  Errors: HS_EINVAL,
 * HS_ENOMEM, HS_ECUDA. */
int hs_evolve(const hs_factors* f, void* psi, int n_rhs, int n_steps, void* cuda_stream);

/* Evolution method selector for hs_evolve_ex. */
typedef enum {
  HS_METHOD_AUTO = 0,  /* fused tile sweeps where possible (same as hs_evolve) */
  HS_METHOD_PLAIN = 1, /* one row-parallel diagonal-times-vector launch per factor application */
  HS_METHOD_FUSED = 2, /* tile sweeps; factors that do not fit a tile fall back to PLAIN */
  HS_METHOD_REG = 3    /* register-blocked tile sweeps, one state per tile: each thread keeps 2^reg_bits
                          rows in registers; a factor with a value table of at most two slots is read from
                          it, any other factor is applied term by term (exact rotations from the build's
                          FP64 cos/sin, runs of diagonal terms as phases generated from (z_j, theta_j) per
                          row, the future-work fusion of the factor values into the apply), so no stored
                          diagonal is read.  A sweep may apply a factor ahead of earlier ones whose terms
                          all commute with its terms (hs_plan_schedule, commuting = 1): the same product
                          up to rounding, with fewer sweeps.  A sweep with a term that flips more than two
                          qubits falls back to PLAIN launches.  Needs n_qubits >= reg_bits + 5; smaller
                          states use FUSED. */
} hs_method;

typedef struct {
  hs_method method;
  int tile_bits;  /* log2 amplitudes per tile for FUSED; 0 = library choice */
  int rhs_block;  /* states per tile for FUSED; 0 = library choice */
  int use_graph;  /* 1: replay the launch sequence as a cached CUDA graph; 0: direct launches */
  int low_bits;   /* FUSED: contiguous low bits every tile keeps (coalescing run of 2^low_bits
                     amplitudes); 0 = library choice (32-byte runs) */
  int max_fuse;   /* FUSED: most factor applications one sweep launch applies (step-fusion
                     depth, 1..64); 0 = 64 */
  int smem_kb;    /* FUSED: shared memory per CTA for the tile and factor staging, in KiB
                     (0 = 112); a smaller budget stages fewer factors ahead but fits more CTAs
                     on an SM.  A tile that needs more for one stage gets what it needs. */
  int no_tables;  /* FUSED: 0 (default): factors whose terms touch at most 8 qubits are read from
                     their value tables (entries indexed by the row's bits on those qubits; same
                     values as the stored diagonals); 1: every factor is staged from its diagonals */
  int reg_bits;   /* REG: rows per thread 2^reg_bits, 4 or 5 (complex128: 4); 0 = library choice
                     (5 for complex64, 4 for complex128).  REG tiles: tile_bits 0 = min(13, n_qubits)
                     for complex64, min(12, n_qubits) for complex128; at least reg_bits + 5, at most
                     13, or 14 for complex64 with reg_bits 5 (512 threads per CTA, one CTA per SM) */
} hs_evolve_opts;

/* hs_evolve with an explicit method and tiling (opts may be NULL = AUTO). */
int hs_evolve_ex(const hs_factors* f, void* psi, int n_rhs, int n_steps, const hs_evolve_opts* opts,
                 void* cuda_stream);

/* Time-dependent Hamiltonians H(t) = H0 + f(t) H1 (the paper's outlook on
 * time-dependent Hamiltonians: the grouping and layout are fixed once and
 * serve every time step).  Term j has coefficient coeffs0[j] in H0 and
 * coeffs1[j] in H1 (host arrays of n_terms finite FP64 values; zero where the
 * term belongs to one of them only).  Step k of an evolution freezes the drive
 * at a caller-given sample f_k and applies the product formula of `order`
 * (as hs_build_factors_ex) with coefficients c_j = coeffs0[j] + f_k coeffs1[j]
 * (the product rounded before the sum), dt = t / n_steps.  The structure
 * depends only on the masks, so it is the one hs_build_factors_ex gives; the
 * values are built for f = 0 (H0).  Errors as hs_build_factors_ex; HS_EINVAL
 * if coeffs1 is NULL or holds a non-finite value. */
int hs_build_factors_td(const uint64_t* x, const uint64_t* z, const double* coeffs0, const double* coeffs1,
                        size_t n_terms, int n_qubits, double t, int n_steps, int diag_budget, int order,
                        hs_dtype dtype, void* cuda_stream, hs_factors** out);

/* Evolve psi in place by n_steps steps of a time-dependent factor set (each
 * of length dt = t / n_steps of the build), step k with the drive sample
 * drive[k] (host array of n_steps finite values, copied
 * before the call returns; sampling f at the step midpoints gives the
 * exponential midpoint rule).  Each step first rebuilds, on the device in
 * FP64, the values of the factors that hold a term with coeffs1[j] != 0 (their
 * value tables, and the stored diagonals of factors that have no table or that
 * the chosen method reads from diagonals), then applies the step as
 * hs_evolve_ex would, with no sweep spanning two steps.  Exception: with
 * HS_METHOD_REG, when every factor application of the n_steps (2 to 65535)
 * steps fits a register sweep (no value-table factor, no plain launch), the
 * term records of every step are computed first (one kernel, 48 bytes per
 * term, angle kind and step, held by the factor set) and the register sweeps
 * span steps as in hs_evolve_ex.  After an evolution of register sweeps alone
 * the stored diagonals are rebuilt when something first reads them
 * (hs_factor_get, hs_apply_factor, an evolution that reads them).  The factor
 * values are those of drive[n_steps - 1] afterwards, so calls on one factor
 * set must be ordered (one stream).  opts as hs_evolve_ex (NULL = AUTO); use_graph
 * captures the whole evolution once per (psi, n_rhs, n_steps, options) and
 * replays it with the new drive samples.  Errors: HS_EINVAL (static factor
 * set, NULL or non-finite drive, bad psi / n_rhs / options), HS_ENOMEM,
 * HS_ECUDA. */
int hs_evolve_td(hs_factors* f, void* psi, int n_rhs, const double* drive, int n_steps, const hs_evolve_opts* opts,
                 void* cuda_stream);

/* Rebuild the values of a time-dependent factor set for one frozen drive
 * value (every dependent factor: value tables and stored diagonals), enqueued
 * on cuda_stream; hs_evolve / hs_factor_get then see H0 + drive H1.
 * Errors: HS_EINVAL (static factor set, non-finite drive), HS_ECUDA. */
int hs_factors_set_drive(hs_factors* f, double drive, void* cuda_stream);

/* Launch plan of hs_evolve_ex for these arguments, computed on the host
 * without launching anything: the number of fused tile-sweep launches, of
 * plain one-factor launches, and the tile_bits / rhs_block that would be
 * used.  Output pointers may be NULL.  Errors: HS_EINVAL. */
int hs_evolve_plan(const hs_factors* f, int n_rhs, int n_steps, const hs_evolve_opts* opts, int* n_sweeps,
                   int* n_plain, int* tile_bits, int* rhs_block);

/* Launch plan of hs_evolve_td for these arguments (a time-dependent set),
 * as hs_evolve_plan: the sweep and plain launches of the whole n_steps-step
 * evolution (register sweeps that span steps counted once; a per-step
 * schedule n_steps times), without the per-step record and rebuild kernels.
 * Errors: HS_EINVAL (also for a static factor set). */
int hs_evolve_td_plan(const hs_factors* f, int n_rhs, int n_steps, const hs_evolve_opts* opts, int* n_sweeps,
                      int* n_plain, int* tile_bits, int* rhs_block);

/* Measure candidate launch parameters for evolving these n_rhs states by
 * n_steps steps (plain, and fused with several tile_bits / low_bits /
 * rhs_block values) on a temporary copy of psi (psi itself is not modified),
 * return the fastest in *best, and remember it for every factor set of the
 * same shape (qubits, dtype, n_rhs, and each factor's flip span and slot
 * count): later hs_evolve / hs_evolve_ex calls with default options use it.
 * Allocates one temporary state set, synchronises cuda_stream; do not call
 * during stream capture.  Errors: HS_EINVAL, HS_ENOMEM, HS_ECUDA. */
int hs_autotune(const hs_factors* f, const void* psi, int n_rhs, int n_steps, void* cuda_stream,
                hs_evolve_opts* best);

/* ---- Batched evolution of many independent jobs (one graph launch) ---- */

typedef struct hs_batch hs_batch;

typedef struct {
  const hs_factors* factors; /* the job's factor set */
  void* psi;                 /* its states: device buffer of n_rhs states, the factors' dtype */
  int n_rhs;                 /* >= 1 */
  int n_steps;               /* >= 0 */
} hs_batch_job;

typedef struct {
  int tile_bits; /* log2 amplitudes per tile, 8..11 (0 = 10); jobs with fewer qubits, or whose
                    factors do not fit a tile, are evolved with their own launches */
  int low_bits;  /* contiguous low bits of a tile (0 = library choice) */
  int use_graph; /* 1 (default): capture the launch sequence once and replay it as a CUDA graph */
  int smem_kb;   /* shared memory per CTA for the state tile and factor staging, in KiB (0 = 24);
                    a smaller budget stages fewer factors ahead but fits more CTAs on an SM */
  int no_tables; /* as in hs_evolve_opts: 1 stages every factor from its diagonals */
  int tiles_per_cta; /* tiles one CTA evolves back to back, loading its sweep's tables once
                        (0 = library choice, at most 64) */
  int method;        /* HS_METHOD_REG: register-blocked sweeps (as hs_evolve_ex's REG; tile_bits
                        0 = 13 for complex64, 12 for complex128, at most 13; a job below tile_bits
                        qubits gets tiles of its own size, one below reg_bits + 5 qubits or whose
                        sweeps cannot be expressed as register ops runs with its own launches);
                        any other value: the staged tile sweeps described above */
  int reg_bits;      /* REG: rows per thread 2^reg_bits, 4 or 5 (0 = 5 for complex64, 4 for complex128) */
} hs_batch_opts;

/* Plan a batch (host only; device tables are uploaded on the first launch's
 * stream): every job is scheduled exactly as hs_evolve_ex schedules it
 * (same sweeps, same arithmetic, so results are bitwise those of evolving each
 * job alone with the same tile_bits/low_bits and rhs_block 1), and launch k
 * applies the k-th sweep of every job that has one.  All jobs must share one
 * dtype.  The jobs' factor sets and state buffers must outlive the batch.
 * Errors: HS_EINVAL, HS_EDTYPE. */
int hs_batch_create(const hs_batch_job* jobs, size_t n_jobs, const hs_batch_opts* opts, hs_batch** out);

/* Evolve every job of the batch in place by its n_steps (enqueued on
 * cuda_stream; with use_graph the first call captures the launch sequence).
 * Launching twice evolves twice.  Errors: HS_EINVAL, HS_ECUDA. */
int hs_batch_launch(hs_batch* b, void* cuda_stream);

/* Number of launches (levels), CTAs over all levels, amplitude updates per
 * launch of the batch (sum over jobs of n_steps * factors * 2^n * n_rhs), and
 * jobs evolved with their own launches.  Pointers may be NULL. */
int hs_batch_info(const hs_batch* b, int* n_levels, int64_t* n_ctas, int64_t* n_updates, int* n_separate);

/* Free a batch (NULL is a no-op).  Synchronises the device first. */
void hs_batch_free(hs_batch* b);

/* Measure candidate batch options (staged sweeps over several tile sizes,
 * shared-memory budgets and tiles per CTA; register-blocked sweeps over tile
 * sizes, contiguous low bits and register widths) for these jobs, each timed
 * on a scratch copy of every job's states (the jobs' own states are not
 * modified), and return the fastest in *best (use_graph as given in
 * best->use_graph on entry, 0 if best holds garbage).  Allocates one scratch
 * buffer of all the jobs' states, synchronises cuda_stream; do not call
 * during stream capture.  Errors as hs_batch_create, HS_ENOMEM, HS_ECUDA. */
int hs_batch_autotune(const hs_batch_job* jobs, size_t n_jobs, void* cuda_stream, hs_batch_opts* best);

/* One call over job arrays (the batched form of hs_evolve): job k evolves
 * psi[k] (n_rhs[k] states, device buffer of the factors' dtype) in place by
 * n_steps[k] steps of f[k].  Plans a batch of register-blocked sweeps
 * (hs_batch_opts method HS_METHOD_REG, every other option the library's
 * choice), enqueues its launches on cuda_stream (directly, no graph) and frees the
 * batch's tables in stream order; the same work as hs_batch_create +
 * hs_batch_launch + hs_batch_free_async.  All arrays are host arrays of
 * n_jobs entries.  Errors as hs_batch_create and hs_batch_launch. */
int hs_evolve_batch(const hs_factors* const* f, void* const* psi, const int* n_rhs, const int* n_steps,
                    size_t n_jobs, void* cuda_stream);

/* Free a batch in stream order without synchronising (its tables return to the
 * pool after the work already enqueued on cuda_stream); every launch of b must
 * be ordered before that.  Always HS_OK. */
int hs_batch_free_async(hs_batch* b, void* cuda_stream);

/* y = F_g x for one factor (Alg. 1: the sum over diagonals of the shifted
 * element-wise products), out of place.  x and y are device buffers of n_rhs
 * states of the factors' dtype and must not overlap.  Errors: HS_EINVAL. */
int hs_apply_factor(const hs_factors* f, int g, const void* x, void* y, int n_rhs, void* cuda_stream);

/* State fidelity (evaluation section, Metrics): |<a|b>|^2 / (|a|^2 |b|^2),
 * accumulated in FP64 whatever the storage dtype.  a, b: device buffers of one
 * state each (2^n_qubits amplitudes).  fid, norm_a2, norm_b2: host outputs;
 * norm pointers may be NULL.  Synchronises cuda_stream.  Errors: HS_EINVAL,
 * HS_ECUDA. */
int hs_fidelity(const void* a, const void* b, int n_qubits, hs_dtype dtype, void* cuda_stream, double* fid,
                double* norm_a2, double* norm_b2);

/* <a|b> = sum conj(a_i) b_i and |a|^2, |b|^2 in FP64, written to a DEVICE
 * buffer out[4] = {re, im, |a|^2, |b|^2} without synchronising (usable inside
 * stream capture).  Errors: HS_EINVAL, HS_ECUDA. */
int hs_inner_device(const void* a, const void* b, int n_qubits, hs_dtype dtype, double* out_device,
                    void* cuda_stream);

/* Batched <a_i|b_i>, |a_i|^2, |b_i|^2 (FP64, i = 0 .. n_states-1) that
 * allocates no device memory.  The paper has no counterpart of this call.
 * It exists for callers that cannot allocate: a serving loop that keeps all
 * device memory reserved for resident states and factors, or an application
 * whose device memory belongs to its own allocator.  a, b: device buffers of
 * n_states states each (rhs-major, 2^n_qubits amplitudes per state).
 * out_device: DEVICE buffer of 4 * n_states doubles, written as
 * {re, im, |a_i|^2, |b_i|^2} per state; the values equal hs_inner_device's
 * for each pair.  Scratch is a static per-device array of 4864 partial sums
 * (152 KiB, held by every GPU that loads the library until exit): a call
 * needs n_states * min(ceil(2^n_qubits / 256), 608) of them and is rejected
 * with HS_EINVAL above that (at least 8 states of any size per call).  Every
 * call looks up the array's device address on the current device (a host-side
 * lookup, valid after a context is re-created); the first call on a device
 * also loads the module there, so make it before any stream capture.  Calls
 * that overlap on the GPU race on the array.  Its two kernels are counted by
 * hs_kernel_launches.
 * Does not synchronise.  Errors: HS_EINVAL, HS_EDTYPE, HS_ECUDA. */
int hs_inner_batch_noalloc(const void* a, const void* b, int n_qubits, int n_states, hs_dtype dtype,
                           double* out_device, void* cuda_stream);

/* Introspection.  hs_factors_info: number of factors, qubits, steps the
 * object was built for, dtype, and total device bytes of factor values. */
int hs_factors_info(const hs_factors* f, int* n_factors, int* n_qubits, int* n_steps, hs_dtype* dtype,
                    int64_t* value_bytes);

/* Factor g's term range [term_first, term_last), diagonal count, offsets in
 * canonical order and values as the Eq. 6 view: FP64 interleaved complex,
 * diagonal after diagonal, N - |d| entries each, no padding (2 * S_g doubles,
 * S_g = sum_k (N - |d_k|)).  offsets / values may be NULL to skip them.
 * Copies from the device; synchronises with the device. */
int hs_factor_get(const hs_factors* f, int g, int* term_first, int* term_last, int* n_diags, int64_t* offsets,
                  double* values);

/* Free a factor set (NULL is a no-op).  Synchronises the device first. */
void hs_free_factors(hs_factors* f);

/* Free a factor set in stream order without synchronising: its device memory
 * returns to the stream-ordered pool once the work already enqueued on
 * cuda_stream completes.  All work that uses f must be enqueued on cuda_stream
 * or ordered before it.  Always HS_OK. */
int hs_free_factors_async(hs_factors* f, void* cuda_stream);

/* Message for the last failing call on this thread ("" if none). */
const char* hs_last_error(void);

/* Number of kernels this process has launched through libhs so far (every
 * entry point; a replayed CUDA graph adds the kernels it holds).  Telemetry:
 * the difference across a region counts that region's launches.  Not part of
 * the paper's method. */
uint64_t hs_kernel_launches(void);

/* Index checks (not part of the paper's method).  A library compiled with
 * -DHS_DEBUG_BOUNDS tests every state row, diagonal element, slot and
 * row-base table entry, value-table entry and per-term record a kernel
 * addresses against its array's extent; a failed test counts, records the
 * first failure and redirects the access to element 0 (no trap, the context
 * stays usable, the launch's results are void).  out4 (host, 4 words)
 * receives the number of failures, then the first failure's site, index and
 * extent (sites are listed in csrc/bounds.cuh); reset != 0 clears the counts.
 * Call it after the checked work has completed (e.g. after a device
 * synchronise).  Returns 1 in a checking build, 0 in the ordinary build (out4
 * zeroed), HS_EINVAL for a null out4, HS_ECUDA if a read fails. */
int hs_debug_bounds(uint64_t* out4, int reset);

#ifdef __cplusplus
}
#endif

#endif /* HS_H */
