/*
 * hs_dia.h -- C ABI of libhs, single-factor Taylor mode: the paper's original
 * pipeline (Alg. 3) on one GB300 GPU.
 *
 *   H (Pauli sum) --hs_dia_from_terms--> H in the compact diagonal layout
 *   r = hs_estimate_timesteps(H, T, D_max)         (Eq. 5, Sec. 3.1 flowchart)
 *   U = hs_spme(H, T / r)                           (Alg. 2, SpME paragraph)
 *   psi <- U^r psi  via hs_dia_evolve               (Alg. 3 loop of Alg. 1 SpMV)
 *
 * An hs_dia is a square 2^n x 2^n complex matrix in the layout of Eq. 6 /
 * Tab. 1: an offset list (d = col - row, canonical order 0, then |d|
 * ascending, negative before positive) and one dense diagonal of N - |d|
 * entries per offset, element i of diagonal d holding entry (row, col) with
 * i = min(row, col).  It is device-resident, owned by the library, immutable
 * after creation and freed only by hs_dia_free.  Matrices built by this
 * library compute and store FP64 complex (HS_C128); hs_dia_convert makes a
 * complex64 copy for a complex64 bulk SpMV.
 *
 * Zero diagonals (readings of the paper, which is silent on them):
 *   - hs_dia_from_terms / hs_dia_from_masks keep exactly the diagonals of H
 *     that hold a nonzero entry (the numeric counts of Tab. 3: a Heisenberg
 *     bond keeps 0 and +-2^i, its XX and YY entries on +-3*2^i cancel);
 *   - hs_spgemm keeps the diagonals its diagonal pairs reach, minus those whose
 *     every entry has magnitude <= 2^-46 times the largest entry magnitude of
 *     the product (cancellation residue).
 *
 * The codes, hs_dtype, the Pauli label convention, the state layout and the
 * stream and error conventions are those of hs.h.  Calls that must decide on
 * the host from device results (which diagonals to keep, when the Taylor loop
 * stops) synchronise cuda_stream; the others only enqueue.
 */
#ifndef HS_DIA_H
#define HS_DIA_H

#include "hs.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hs_dia hs_dia;

/* H = sum_j coeffs[j] * P_j (Sec. 3: the Hamiltonian as a Pauli sum) in the
 * compact layout, FP64, exactly-zero diagonals dropped.  pauli_terms: n_terms
 * labels of equal length n_qubits (1..HS_MAX_QUBITS); coeffs: real, finite.
 * Terms sharing an x mask are summed in input order.  Errors: HS_EINVAL (bad
 * label or coefficient, n_terms == 0, more than 65536 candidate diagonals),
 * HS_ENOMEM, HS_ECUDA.  Synchronises cuda_stream. */
int hs_dia_from_terms(const char* const* pauli_terms, const double* coeffs, size_t n_terms, void* cuda_stream,
                      hs_dia** out);
/* Same from pre-parsed masks (x: X or Y present, z: Z or Y present). */
int hs_dia_from_masks(const uint64_t* x, const uint64_t* z, const double* coeffs, size_t n_terms, int n_qubits,
                      void* cuda_stream, hs_dia** out);

/* A matrix from host data: offsets[n_diags] (distinct, |d| < 2^n_qubits, any
 * order; stored in canonical order) and values: FP64 interleaved complex,
 * diagonal after diagonal in the order given, N - |offsets[k]| entries each.
 * dtype: storage precision (HS_C64 rounds once).  All diagonals are kept,
 * zero or not.  Errors: HS_EINVAL, HS_EDTYPE, HS_ENOMEM, HS_ECUDA.
 * Synchronises cuda_stream (values are staged through host memory). */
int hs_dia_create(int n_qubits, const int64_t* offsets, size_t n_diags, const double* values, hs_dtype dtype,
                  void* cuda_stream, hs_dia** out);

/* C = A * B (SpGEMM paragraph, Sec. 3.3): result diagonal dc collects every
 * pair (da, db) of A's and B's diagonals with da + db = dc; entry (i, i+dc) =
 * sum over pairs, in A-major canonical order, of A(i, i+da) * B(i+da, i+dc)
 * over the rows where both entries exist, accumulated in FP64.  A and B are
 * HS_C128 of the same size.  fro_norm (may be NULL): Frobenius norm of C.
 * Errors: HS_EINVAL, HS_EDTYPE, HS_ENOMEM, HS_ECUDA.  Synchronises. */
int hs_spgemm(const hs_dia* a, const hs_dia* b, void* cuda_stream, hs_dia** out, double* fro_norm);

/* U = exp(-i t A) (SpME paragraph).  A diagonal-only A (offset 0 alone) is
 * exponentiated exactly entry by entry; otherwise the truncated Taylor series
 * of Alg. 2: X = -i t A, U = T = I, and for k = 1..max_iter: T = (T X) / k; if
 * ||T||_F < tol stop, else U += T (no scaling and squaring).  tol > 0
 * (the paper uses 1e-6), max_iter >= 1.  n_terms (may be NULL): the k at
 * which the loop stopped (0 for the exact diagonal path); converged (may be
 * NULL): 1 if the tolerance was met.  A is HS_C128; U is HS_C128.  Errors:
 * HS_EINVAL, HS_EDTYPE, HS_ENOMEM, HS_ECUDA.  Synchronises. */
int hs_spme(const hs_dia* a, double t, double tol, int max_iter, void* cuda_stream, hs_dia** out, int* n_terms,
            int* converged);

/* Diagonal-budgeted step count (Eq. 5 and the adaptive timestep flowchart of
 * Sec. 3.1): the smallest r such that the Taylor loop of hs_spme at time t/r
 * converges within max_iter terms and U(t/r) holds <= diag_budget diagonals.
 * A diagonal-only A gives r = 1.  Search: r = 1 is tried; otherwise the upper
 * bound doubles until it passes, then a binary search between the last
 * failing and the first passing count.  Errors: HS_EINVAL (bad argument, or
 * no r <= max_steps passes), HS_EDTYPE, HS_ENOMEM, HS_ECUDA.  Synchronises. */
int hs_estimate_timesteps(const hs_dia* a, double t, int diag_budget, double tol, int max_iter, int max_steps,
                          void* cuda_stream, int* n_steps);

/* y = A x (Alg. 1) for n_rhs states: y[i] = sum_k A(i, i+d_k) x[i+d_k].  x and
 * y are caller-owned device buffers of A's dtype (n_rhs x 2^n, rhs-major) and
 * must not overlap.  HS_C64 accumulates in FP32, HS_C128 in FP64.  Errors:
 * HS_EINVAL, HS_ECUDA.  Enqueues only. */
int hs_spmv(const hs_dia* a, const void* x, void* y, int n_rhs, void* cuda_stream);

/* Expectation values <psi_r|A|psi_r> for n_rhs states (an observable on the
 * compact-layout H; the paper itself evaluates state fidelities only).  psi: device buffer of A's dtype (n_rhs x 2^n, rhs-major).  Each row's
 * (A psi)_i = sum_k A(i, i+d_k) psi[i+d_k] and conj(psi_i) (A psi)_i are
 * formed and summed in FP64 (fixed-order tree, deterministic).  values: host
 * array of 2 * n_rhs doubles (Re, Im per state); norms (may be NULL): host
 * array of n_rhs doubles, <psi_r|psi_r>.  Errors: HS_EINVAL, HS_ENOMEM,
 * HS_ECUDA.  Synchronises cuda_stream. */
int hs_expectation(const hs_dia* a, const void* psi, int n_rhs, void* cuda_stream, double* values, double* norms);

/* psi <- U^n_steps psi (the loop of Alg. 3), psi in U's dtype, updated in
 * place (n_rhs x 2^n).  A one-diagonal U (offset 0) is applied in place; a
 * general U ping-pongs with a stream-ordered scratch state.  Errors:
 * HS_EINVAL, HS_ENOMEM, HS_ECUDA.  Enqueues only. */
int hs_dia_evolve(const hs_dia* u, void* psi, int n_rhs, int n_steps, void* cuda_stream);

/* Time-dependent H(t) = H0 + f(t) H1 in the single-factor mode (the outlook
 * on time-dependent Hamiltonians, Future Work): for step k = 0..n_steps-1 the
 * drive is frozen at drive[k]; H(f_k) = sum_j c_j P_j with c_j = coeffs0[j] +
 * drive[k] * coeffs1[j] (the product rounded before the sum) is formed as by
 * hs_dia_from_masks, U_k = exp(-i dt H(f_k)) by hs_spme (tol, max_iter),
 * dt = t / n_steps, stored as dtype, and psi <- U_k psi (hs_dia_evolve, one
 * step).  x, z, coeffs0, coeffs1: n_terms host entries (masks as
 * hs_dia_from_masks; coefficients finite); drive: n_steps finite host values
 * (step midpoints give the exponential midpoint rule); psi: device buffer of
 * n_rhs states of dtype, updated in place.  The caller chooses n_steps (for
 * example the largest hs_estimate_timesteps over the distinct samples).
 * Errors: HS_EINVAL (bad argument, non-finite value, a step whose Taylor loop
 * does not converge: psi then holds the steps before it), HS_EDTYPE,
 * HS_ENOMEM, HS_ECUDA.  Each step synchronises cuda_stream once (hs_spme
 * decides on the host when the Taylor loop stops); the step's matrices are
 * freed in stream order on cuda_stream, so other streams are not waited for. */
int hs_dia_evolve_td(const uint64_t* x, const uint64_t* z, const double* coeffs0, const double* coeffs1,
                     size_t n_terms, int n_qubits, double t, const double* drive, int n_steps, double tol,
                     int max_iter, void* psi, int n_rhs, hs_dtype dtype, void* cuda_stream);

/* A copy of A stored as dtype (HS_C64 rounds each FP64 part once).  Enqueues only. */
int hs_dia_convert(const hs_dia* a, hs_dtype dtype, void* cuda_stream, hs_dia** out);

/* Size and structure: any pointer may be NULL.  nnz counts entries that are not
 * exactly zero (computed when the matrix was made by this library; -1 for
 * hs_dia_create and hs_dia_convert results). */
int hs_dia_info(const hs_dia* a, int* n_qubits, int* n_diags, int64_t* nnz, hs_dtype* dtype);

/* Host copy: offsets[n_diags] in canonical order and/or values as FP64
 * interleaved complex in the Eq. 6 order (diagonal after diagonal, N - |d|
 * entries each, no padding).  Either pointer may be NULL.  Synchronises. */
int hs_dia_get(const hs_dia* a, int64_t* offsets, double* values);

/* Frees a matrix (NULL is a no-op).  Synchronises the device first. */
void hs_dia_free(hs_dia* a);

#ifdef __cplusplus
}
#endif

#endif /* HS_DIA_H */
