/*
 * Oracle for diagonal-budgeted Trotterization -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-threaded FP64 C.  Only the test suite, the smoke check
 * and the benchmark's CPU-baseline leg may load this file's library; the
 * product path (the CUDA library under paper_2606_16959_gb300/) never does,
 * and the two share no code, header, table or helper.
 *
 * What it computes (paper sections cited per function):
 *   - the action of a Pauli string on a basis state,
 *   - the first-order Trotter product of Eq. 4 applied term by term
 *     ("direct evolution", the reference result),
 *   - the numeric values of one grouped factor F = R_last ... R_first written
 *     into the compact diagonal layout of Eq. 6 / Tab. 1,
 *   - the diagonal-times-vector product of Alg. 1 / the DiagonalTimesVector
 *     figure (y[k] += v[i] x[j] with the affine (j,k) mapping per sign of d),
 *   - squared norms and inner products with pairwise summation (the state
 *     fidelity metric of the evaluation section).
 *
 * Conventions (readings of the paper, all shared with the Python half):
 *   P|b> = i^y (-1)^popcount(z & b) |b xor x>,  y = popcount(x & z);
 *   R_j = cos(theta_j) I - i sin(theta_j) P_j = exp(-i theta_j P_j);
 *   theta_j = c_j * dt,  dt = t / n_steps (each one FP64 rounding);
 *   term 1 acts first, within a step and within a factor;
 *   diagonal offset d = col - row; element index along a diagonal = min(row, col).
 *
 * Complex numbers are C99 `double complex`, layout-compatible with
 * interleaved (re, im) double pairs.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static int parity64(uint64_t v) { return __builtin_popcountll(v) & 1; }

/* i^k for integer k */
static cplx i_pow(int k) {
  switch (k & 3) {
    case 0: return 1.0;
    case 1: return I;
    case 2: return -1.0;
    default: return -I;
  }
}

/* Phase of P acting on |b>: i^y (-1)^popcount(z & b). */
static cplx pauli_phase(uint64_t x, uint64_t z, uint64_t b) {
  int y = __builtin_popcountll(x & z);
  cplx ph = i_pow(y);
  return parity64(z & b) ? -ph : ph;
}

/* out = P psi for one Pauli string (x, z) on N = 2^n amplitudes. */
void orc_pauli_apply(int64_t N, uint64_t x, uint64_t z, const cplx* psi, cplx* out) {
  for (int64_t b = 0; b < N; ++b) out[(int64_t)((uint64_t)b ^ x)] = pauli_phase(x, z, (uint64_t)b) * psi[b];
}

/* psi <- exp(-i theta P) psi = cos(theta) psi - i sin(theta) P psi   (Eq. 4 factor,
 * exact because P^2 = I). */
void orc_rotate(int64_t N, uint64_t x, uint64_t z, double theta, cplx* psi) {
  cplx* tmp = (cplx*)malloc(sizeof(cplx) * (size_t)N);
  orc_pauli_apply(N, x, z, psi, tmp);
  double c = cos(theta), s = sin(theta);
  for (int64_t b = 0; b < N; ++b) psi[b] = c * psi[b] - I * s * tmp[b];
  free(tmp);
}

/* Direct first-order Trotter evolution (Eq. 4; loop shape of Alg. 3):
 * for each of n_steps steps, for j = 0..m-1 in input order, psi <- R_j psi.
 * psi holds n_rhs states of N amplitudes each, rhs-major. */
void orc_evolve_direct(int64_t N, int n_rhs, int m, const uint64_t* x, const uint64_t* z,
                       const double* coeff, double t, int n_steps, cplx* psi) {
  double dt = t / (double)n_steps;
  for (int r = 0; r < n_rhs; ++r)
    for (int s = 0; s < n_steps; ++s)
      for (int j = 0; j < m; ++j) orc_rotate(N, x[j], z[j], coeff[j] * dt, psi + (int64_t)r * N);
}

/* Slot of x-mask u in the group's x-mask list X (linear search; -1 if absent). */
static int slot_of(int nX, const uint64_t* X, uint64_t u) {
  for (int k = 0; k < nX; ++k)
    if (X[k] == u) return k;
  return -1;
}

/* Index of diagonal offset d in the factor's offset list (linear search; -1 if absent). */
static int diag_of(int D, const int64_t* offs, int64_t d) {
  for (int k = 0; k < D; ++k)
    if (offs[k] == d) return k;
  return -1;
}

/* Numeric values of one grouped factor F = R_last ... R_first (term `first`
 * acts first), materialised column by column into the compact diagonal layout
 * (Eq. 6): diagonal k (offset offs[k]) holds N - |offs[k]| entries starting
 * at vals[starts[k]]; entry (row, col) sits at element min(row, col).
 *
 * Column b of F is F e_b.  Every basis state reached from e_b by the group's
 * Paulis is b xor u with u in X (the group's x-mask set, closed under xor),
 * so the column is kept as a sparse vector over the slots of X.
 * theta[j] is the rotation angle of the group's j-th term.
 * Returns 0, or -1 if a structural entry falls outside the given offsets. */
int orc_build_factor(int64_t N, int n_terms, const uint64_t* x, const uint64_t* z,
                     const double* theta, int nX, const uint64_t* X, int D, const int64_t* offs,
                     const int64_t* starts, cplx* vals) {
  int64_t total = starts[D - 1] + (N - llabs(offs[D - 1]));
  for (int64_t e = 0; e < total; ++e) vals[e] = 0.0;
  cplx* col = (cplx*)malloc(sizeof(cplx) * (size_t)nX);
  cplx* pcol = (cplx*)malloc(sizeof(cplx) * (size_t)nX);
  for (int64_t b = 0; b < N; ++b) {
    for (int k = 0; k < nX; ++k) col[k] = 0.0;
    col[slot_of(nX, X, 0)] = 1.0;
    for (int j = 0; j < n_terms; ++j) {
      /* pcol = P_j col */
      for (int k = 0; k < nX; ++k) pcol[k] = 0.0;
      for (int k = 0; k < nX; ++k) {
        uint64_t basis = (uint64_t)b ^ X[k];
        int dst = slot_of(nX, X, X[k] ^ x[j]);
        if (dst < 0) { free(col); free(pcol); return -1; }
        pcol[dst] += pauli_phase(x[j], z[j], basis) * col[k];
      }
      double c = cos(theta[j]), s = sin(theta[j]);
      for (int k = 0; k < nX; ++k) col[k] = c * col[k] - I * s * pcol[k];
    }
    for (int k = 0; k < nX; ++k) {
      int64_t row = (int64_t)((uint64_t)b ^ X[k]);
      int64_t d = b - row;
      int q = diag_of(D, offs, d);
      if (q < 0) { free(col); free(pcol); return -1; }
      vals[starts[q] + (row < b ? row : b)] = col[k];
    }
  }
  free(col);
  free(pcol);
  return 0;
}

/* Diagonal-times-vector product over all diagonals (Alg. 1 with the
 * DiagonalTimesVector mapping): for diagonal offset d and element i,
 *   d < 0: j = i, k = i - d;   d = 0: j = k = i;   d > 0: j = i + d, k = i;
 *   y[k] += v[i] * x[j].
 * y is overwritten (y = A x). */
void orc_dia_apply(int64_t N, int D, const int64_t* offs, const int64_t* starts, const cplx* vals,
                   const cplx* xv, cplx* y) {
  for (int64_t i = 0; i < N; ++i) y[i] = 0.0;
  for (int q = 0; q < D; ++q) {
    int64_t d = offs[q];
    int64_t len = N - llabs(d);
    const cplx* v = vals + starts[q];
    for (int64_t i = 0; i < len; ++i) {
      int64_t j, k;
      if (d < 0) { j = i; k = i - d; }
      else if (d == 0) { j = i; k = i; }
      else { j = i + d; k = i; }
      y[k] += v[i] * xv[j];
    }
  }
}

/* Pairwise (cascade) summation of n doubles. */
static double pairwise_sum(const double* a, int64_t n) {
  if (n <= 8) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i];
    return s;
  }
  int64_t h = n / 2;
  return pairwise_sum(a, h) + pairwise_sum(a + h, n - h);
}

/* ||a||^2 with pairwise summation. */
double orc_norm2(int64_t N, const cplx* a) {
  double* t = (double*)malloc(sizeof(double) * (size_t)N);
  for (int64_t i = 0; i < N; ++i) t[i] = creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
  double s = pairwise_sum(t, N);
  free(t);
  return s;
}

/* <a|b> = sum conj(a_i) b_i with pairwise summation of each part. */
void orc_inner(int64_t N, const cplx* a, const cplx* b, double* re, double* im) {
  double* tr = (double*)malloc(sizeof(double) * (size_t)N);
  double* ti = (double*)malloc(sizeof(double) * (size_t)N);
  for (int64_t i = 0; i < N; ++i) {
    cplx p = conj(a[i]) * b[i];
    tr[i] = creal(p);
    ti[i] = cimag(p);
  }
  *re = pairwise_sum(tr, N);
  *im = pairwise_sum(ti, N);
  free(tr);
  free(ti);
}
