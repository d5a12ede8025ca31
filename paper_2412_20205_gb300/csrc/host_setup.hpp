// Host-side set-up of the tensor-product B-spline multigrid hierarchy.
// Internal header (not part of the C ABI).
#pragma once
#include <vector>

namespace igamg {

// Breakpoints of a uniform mesh of [0, 1] with n elements.
std::vector<double> uniform_breaks(int n);
// Coarse breakpoints (mesh 2h, Sec. 2): every other breakpoint plus the last
// one when the element count is odd, so the coarse space nests in the fine one.
std::vector<double> coarsen_breaks(const std::vector<double>& breaks);
// Open knot vector (Sec. 2.3): end breakpoints repeated p+1 times.
std::vector<double> open_knots(const std::vector<double>& breaks, int p);

// n-point Gauss-Legendre rule on [-1, 1] (Golub-Welsch: eigenvalues of the
// symmetric Jacobi matrix of the Legendre recurrence).
void gauss_legendre(int n, double* x, double* w);

// Symmetric eigen-decomposition A = W diag(lam) W^T by cyclic Jacobi rotations
// (A is n x n row-major, overwritten; W row-major, column j = eigenvector j).
void jacobi_eigen(int n, std::vector<double>& A, std::vector<double>& W, std::vector<double>& lam);

// Banded interior 1D Galerkin factors: rows m = n + p - 2, band 2p+1,
// F[i*(2p+1) + k] = F(i, i+k-p); zero where i+k-p is outside [0, m).
struct Factor1D {
    int m = 0, p = 0;
    std::vector<double> M, K;
};
Factor1D assemble_1d(const std::vector<double>& breaks, int p);

// Interior prolongation by knot insertion (Boehm), dense m_f x m_c row-major:
// coarse B-spline J equals sum_i P(i, J) fine B-spline i.
std::vector<double> prolongation_1d(const std::vector<double>& fine_breaks,
                                    const std::vector<double>& coarse_breaks, int p,
                                    int* m_f, int* m_c);

// Generalised eigenpairs K V = M V diag(lam), V^T M V = I (m x m, from the
// banded factor), used by the exact coarsest-grid solve.
void generalized_eigen(const Factor1D& f, std::vector<double>& V, std::vector<double>& lam);

// Load-vector integrals g_k(i) = int_0^1 sin((k+1) pi x) N_i(x) dx for the
// interior basis, k = 0..modes-1, (p+1) Gauss points per element;
// g[k*m + i].
std::vector<double> sine_moments(const std::vector<double>& breaks, int p, int modes);

}  // namespace igamg
