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

// The p+1 B-splines N_{s-p}..N_s non-zero on knot span s and their
// derivatives at x (U: open knot vector).
void basis_and_derivative(const std::vector<double>& U, int p, int s, double x, double* N, double* dN);

// ---------------------------------------------------------------- general operator (Sec. 4.3)
// (p+1)-point Gauss rule per element of one direction: point q = e (p+1) + g
// (ascending), its weight, and the values / derivatives of the p+1 full-basis
// functions e .. e+p non-zero there: N[q (p+1) + r], dN[q (p+1) + r].
struct Quad1D {
    int n = 0, p = 0, nq = 0;
    std::vector<double> x, w, N, dN;
};
Quad1D quadrature_1d(const std::vector<double>& breaks, int p);

// Operator of a 2D level in stencil form: S[k N + I] = A(I, I + dx + mx dy)
// with k = (dy + p)(2p+1) + (dx + p), |dx|, |dy| <= p (zero where the column
// is outside the grid); I = ix + mx iy over the interior unknowns.
struct Stencil2D {
    int mx = 0, my = 0, p = 0;
    std::vector<double> S;
    size_t N() const { return (size_t)mx * my; }
};
// Galerkin matrix of a(u, v) = int grad v . Ah grad u + (Bh . grad u) v + ch u v
// over the unit square, with coef[k nq + q] (k = 0..5: ah11, ah12, ah22, bh1,
// bh2, ch) at the tensor quadrature points q = qy nqx + qx of qx, qy.
Stencil2D assemble_general(const Quad1D& qx, const Quad1D& qy, const double* coef);
// Galerkin coarse operator P^T A P (Eq. (4)), P = Py (x) Px (dense 1D interior
// prolongations, m_f x m_c row-major).
Stencil2D galerkin_coarse(const Stencil2D& A, const std::vector<double>& Px, int mcx,
                          const std::vector<double>& Py, int mcy);
// Dense inverse (Gauss-Jordan, partial pivoting) of the stencil operator; false when singular.
bool dense_inverse(const Stencil2D& A, std::vector<double>& inv);
// l_I = sum_q w_q fq[q] phi_I(q) at the tensor quadrature points.
std::vector<double> load_general(const Quad1D& qx, const Quad1D& qy, const double* fq);

// Load-vector integrals g_k(i) = int_0^1 sin((k+1) pi x) N_i(x) dx for the
// interior basis, k = 0..modes-1, (p+1) Gauss points per element;
// g[k*m + i].
std::vector<double> sine_moments(const std::vector<double>& breaks, int p, int modes);

}  // namespace igamg
