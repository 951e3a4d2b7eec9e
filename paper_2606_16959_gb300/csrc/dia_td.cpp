// Time-dependent H(t) = H0 + f(t) H1 in the single-factor Taylor mode (the
// outlook on time-dependent Hamiltonians), composed from the compact-layout
// calls of hs_dia.h: per step, H(f_k) from the terms, U_k = SpME(H(f_k), dt)
// (Alg. 2, exact for a diagonal H), and one diagonal-times-vector step (Alg. 1).
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/hs.h"
#include "../../include/hs_dia.h"

namespace hs {
int report_error(int code, const std::string& msg);
void dia_free_async(hs_dia* m, cudaStream_t s);
}  // namespace hs

extern "C" int hs_dia_evolve_td(const uint64_t* x, const uint64_t* z, const double* coeffs0, const double* coeffs1,
                                size_t n_terms, int n_qubits, double t, const double* drive, int n_steps, double tol,
                                int max_iter, void* psi, int n_rhs, hs_dtype dtype, void* cuda_stream) {
  if (!x || !z || !coeffs0 || !coeffs1) return hs::report_error(HS_EINVAL, "null term arrays");
  if (!psi) return hs::report_error(HS_EINVAL, "psi is NULL");
  if (n_rhs < 1) return hs::report_error(HS_EINVAL, "n_rhs must be >= 1");
  if (n_steps < 0) return hs::report_error(HS_EINVAL, "n_steps must be >= 0");
  if (n_steps > 0 && !drive) return hs::report_error(HS_EINVAL, "drive is NULL");
  if (!(std::isfinite(t) && t > 0)) return hs::report_error(HS_EINVAL, "t must be finite and > 0");
  if (!(tol > 0) || max_iter < 1) return hs::report_error(HS_EINVAL, "tol must be > 0 and max_iter >= 1");
  if (dtype != HS_C64 && dtype != HS_C128) return hs::report_error(HS_EDTYPE, "dtype must be HS_C64 or HS_C128");
  for (int k = 0; k < n_steps; ++k)
    if (!std::isfinite(drive[k])) return hs::report_error(HS_EINVAL, "non-finite drive value at step " + std::to_string(k));
  for (size_t j = 0; j < n_terms; ++j)
    if (!std::isfinite(coeffs1[j])) return hs::report_error(HS_EINVAL, "non-finite H1 coefficient at term " + std::to_string(j));
  if (n_steps == 0) return HS_OK;
  // Every matrix of a step is freed in stream order on this stream, so a step
  // waits for nothing but its own stream (hs_spme synchronises it to decide
  // when the Taylor loop stops); other streams keep running.
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  const double dt = t / double(n_steps);
  std::vector<double> c(n_terms);
  for (int k = 0; k < n_steps; ++k) {
    const double f = drive[k];
    for (size_t j = 0; j < n_terms; ++j) {
      // The product is rounded before the sum (no fused multiply-add).
      volatile double p = f * coeffs1[j];
      c[j] = coeffs0[j] + p;
    }
    hs_dia* H = nullptr;
    int rc = hs_dia_from_masks(x, z, c.data(), n_terms, n_qubits, cuda_stream, &H);
    if (rc != HS_OK) return rc;
    hs_dia* U = nullptr;
    int n_taylor = 0, converged = 0;
    rc = hs_spme(H, dt, tol, max_iter, cuda_stream, &U, &n_taylor, &converged);
    hs::dia_free_async(H, s);
    if (rc != HS_OK) return rc;
    if (!converged) {
      hs::dia_free_async(U, s);
      return hs::report_error(HS_EINVAL, "Taylor series did not converge within max_iter terms at step " +
                                             std::to_string(k));
    }
    if (dtype == HS_C64) {
      hs_dia* U32 = nullptr;
      rc = hs_dia_convert(U, HS_C64, cuda_stream, &U32);
      hs::dia_free_async(U, s);
      if (rc != HS_OK) return rc;
      U = U32;
    }
    rc = hs_dia_evolve(U, psi, n_rhs, 1, cuda_stream);
    hs::dia_free_async(U, s);  // after the step, in stream order
    if (rc != HS_OK) return rc;
  }
  return HS_OK;
}
