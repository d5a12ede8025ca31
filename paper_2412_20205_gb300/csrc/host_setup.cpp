// Host-side set-up: knots, B-spline evaluation, Gauss rules, banded 1D
// Galerkin factors, knot-insertion prolongation and the generalised eigenpairs
// of the coarsest grid.  Runs once per problem; nothing here is timed.
#include "host_setup.hpp"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace igamg {

std::vector<double> uniform_breaks(int n) {
    std::vector<double> b(n + 1);
    for (int i = 0; i <= n; ++i) b[i] = (double)i / (double)n;
    b[n] = 1.0;
    return b;
}

std::vector<double> coarsen_breaks(const std::vector<double>& breaks) {
    std::vector<double> c;
    const int n = (int)breaks.size() - 1;
    for (int i = 0; i <= n; i += 2) c.push_back(breaks[i]);
    if (n % 2 == 1) c.push_back(breaks[n]);
    return c;
}

std::vector<double> open_knots(const std::vector<double>& breaks, int p) {
    std::vector<double> U;
    for (int i = 0; i < p; ++i) U.push_back(breaks.front());
    U.insert(U.end(), breaks.begin(), breaks.end());
    for (int i = 0; i < p; ++i) U.push_back(breaks.back());
    return U;
}

void jacobi_eigen(int n, std::vector<double>& A, std::vector<double>& W, std::vector<double>& lam) {
    W.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) W[(size_t)i * n + i] = 1.0;
    auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
    double scale = 0.0;
    for (int i = 0; i < n * n; ++i) scale = std::max(scale, std::fabs(A[i]));
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off = std::max(off, std::fabs(a(i, j)));
        if (off <= 1e-300 || off <= 1e-17 * scale) break;
        for (int p = 0; p < n; ++p) {
            for (int q = p + 1; q < n; ++q) {
                const double apq = a(p, q);
                if (std::fabs(apq) <= 1e-300) continue;
                // rotation angle that annihilates a(p,q): tan(2 phi) = 2 a_pq / (a_qq - a_pp)
                const double theta = (a(q, q) - a(p, p)) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {          // A <- A J (columns p, q)
                    const double akp = a(k, p), akq = a(k, q);
                    a(k, p) = c * akp - s * akq;
                    a(k, q) = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {          // A <- J^T A (rows p, q)
                    const double apk = a(p, k), aqk = a(q, k);
                    a(p, k) = c * apk - s * aqk;
                    a(q, k) = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {          // W <- W J
                    const double wkp = W[(size_t)k * n + p], wkq = W[(size_t)k * n + q];
                    W[(size_t)k * n + p] = c * wkp - s * wkq;
                    W[(size_t)k * n + q] = s * wkp + c * wkq;
                }
            }
        }
    }
    lam.resize(n);
    for (int i = 0; i < n; ++i) lam[i] = a(i, i);
}

void gauss_legendre(int n, double* x, double* w) {
    // Jacobi matrix of the monic Legendre recurrence: zero diagonal and
    // off-diagonal k / sqrt(4k^2 - 1); nodes are its eigenvalues and the
    // weights 2 v_0^2 (mu_0 = int_{-1}^{1} 1 = 2).
    std::vector<double> J((size_t)n * n, 0.0), W, lam;
    for (int k = 1; k < n; ++k) {
        const double b = k / std::sqrt(4.0 * k * k - 1.0);
        J[(size_t)(k - 1) * n + k] = b;
        J[(size_t)k * n + (k - 1)] = b;
    }
    jacobi_eigen(n, J, W, lam);
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return lam[a] < lam[b]; });
    for (int i = 0; i < n; ++i) {
        x[i] = lam[idx[i]];
        const double v0 = W[idx[i]];            // first component of eigenvector idx[i]
        w[i] = 2.0 * v0 * v0;
    }
    for (int i = 0; i < n / 2; ++i) {           // exact symmetry of the rule
        const double xs = 0.5 * (x[n - 1 - i] - x[i]), ws = 0.5 * (w[i] + w[n - 1 - i]);
        x[i] = -xs; x[n - 1 - i] = xs; w[i] = ws; w[n - 1 - i] = ws;
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
}

// Values N_{s-p..s}(x) of the degree-p B-splines on knot span s
// (U[s] <= x < U[s+1]), by the Cox-de Boor recurrence (Eq. moneq) organised
// as a triangular table with the left/right knot distances.
static void basis_on_span(const std::vector<double>& U, int p, int s, double x, double* N) {
    double left[16], right[16];
    N[0] = 1.0;
    for (int q = 1; q <= p; ++q) {
        left[q] = x - U[s + 1 - q];
        right[q] = U[s + q] - x;
        double saved = 0.0;
        for (int r = 0; r < q; ++r) {
            const double tmp = N[r] / (right[r + 1] + left[q - r]);
            N[r] = saved + right[r + 1] * tmp;
            saved = left[q - r] * tmp;
        }
        N[q] = saved;
    }
}

// Values and first derivatives of N_{s-p+r}, r = 0..p, at x in span s.
void basis_and_derivative(const std::vector<double>& U, int p, int s, double x,
                                 double* N, double* dN) {
    basis_on_span(U, p, s, x, N);
    if (p == 0) { dN[0] = 0.0; return; }
    double Nm[16];
    basis_on_span(U, p - 1, s, x, Nm);           // N^{p-1}_{s-p+1..s}
    for (int r = 0; r <= p; ++r) {
        const int j = s - p + r;
        const double a = (r >= 1) ? Nm[r - 1] : 0.0;   // N^{p-1}_j
        const double b = (r <= p - 1) ? Nm[r] : 0.0;   // N^{p-1}_{j+1}
        const double d1 = U[j + p] - U[j], d2 = U[j + p + 1] - U[j + 1];
        dN[r] = p * ((d1 > 0 ? a / d1 : 0.0) - (d2 > 0 ? b / d2 : 0.0));
    }
}

Factor1D assemble_1d(const std::vector<double>& breaks, int p) {
    const int n = (int)breaks.size() - 1;
    const int nb = n + p, m = nb - 2, bw = 2 * p + 1;
    const std::vector<double> U = open_knots(breaks, p);
    std::vector<double> Mf((size_t)nb * bw, 0.0), Kf((size_t)nb * bw, 0.0);
    double xg[16], wg[16], N[16], dN[16];
    gauss_legendre(p + 1, xg, wg);
    for (int e = 0; e < n; ++e) {
        const double a = breaks[e], h = breaks[e + 1] - breaks[e];
        const int s = p + e;                      // knot span of element e
        for (int q = 0; q <= p; ++q) {
            const double x = a + 0.5 * (xg[q] + 1.0) * h, w = 0.5 * wg[q] * h;
            basis_and_derivative(U, p, s, x, N, dN);
            for (int r = 0; r <= p; ++r)
                for (int c = 0; c <= p; ++c) {
                    const int row = e + r, off = c - r + p;
                    Mf[(size_t)row * bw + off] += w * N[r] * N[c];
                    Kf[(size_t)row * bw + off] += w * dN[r] * dN[c];
                }
        }
    }
    Factor1D f;
    f.m = m; f.p = p;
    f.M.assign((size_t)m * bw, 0.0);
    f.K.assign((size_t)m * bw, 0.0);
    for (int i = 0; i < m; ++i)
        for (int k = 0; k < bw; ++k) {
            const int col = i + k - p;
            if (col < 0 || col >= m) continue;
            f.M[(size_t)i * bw + k] = Mf[(size_t)(i + 1) * bw + k];
            f.K[(size_t)i * bw + k] = Kf[(size_t)(i + 1) * bw + k];
        }
    return f;
}

namespace {
struct SparseRow {       // contiguous non-zero range [lo, lo + v.size()) of coarse columns
    int lo = 0;
    std::vector<double> v;
};
SparseRow blend(const SparseRow& a, double alpha, const SparseRow& b, double beta) {
    SparseRow r;
    const int lo = std::min(a.lo, b.lo);
    const int hi = std::max(a.lo + (int)a.v.size(), b.lo + (int)b.v.size());
    r.lo = lo;
    r.v.assign(hi - lo, 0.0);
    for (size_t i = 0; i < a.v.size(); ++i) r.v[a.lo - lo + i] += alpha * a.v[i];
    for (size_t i = 0; i < b.v.size(); ++i) r.v[b.lo - lo + i] += beta * b.v[i];
    return r;
}
}  // namespace

std::vector<double> prolongation_1d(const std::vector<double>& fine_breaks,
                                    const std::vector<double>& coarse_breaks, int p,
                                    int* m_f, int* m_c) {
    // Start from the identity on the coarse basis and insert, one at a time,
    // every fine breakpoint missing from the coarse knot vector (Boehm): with
    // x in [tau_k, tau_{k+1}), new coefficient i is alpha_i c_i + (1 - alpha_i)
    // c_{i-1}, alpha_i = 1 (i <= k-p), (x - tau_i)/(tau_{i+p} - tau_i)
    // (k-p < i <= k), 0 (i > k).  Each row is a coarse-basis combination.
    std::vector<double> tau = open_knots(coarse_breaks, p);
    const int nc = (int)tau.size() - p - 1;
    std::vector<SparseRow> rows(nc);
    for (int i = 0; i < nc; ++i) { rows[i].lo = i; rows[i].v = {1.0}; }
    for (size_t e = 1; e + 1 < fine_breaks.size(); ++e) {
        const double x = fine_breaks[e];
        if (std::binary_search(coarse_breaks.begin(), coarse_breaks.end(), x)) continue;
        int k = (int)(std::upper_bound(tau.begin(), tau.end(), x) - tau.begin()) - 1;
        const int nb = (int)rows.size();
        std::vector<SparseRow> nr(nb + 1);
        for (int i = 0; i <= nb; ++i) {
            if (i <= k - p) nr[i] = rows[i];
            else if (i >= k + 1) nr[i] = rows[i - 1];
            else {
                const double alpha = (x - tau[i]) / (tau[i + p] - tau[i]);
                nr[i] = blend(rows[i], alpha, rows[i - 1], 1.0 - alpha);
            }
        }
        rows.swap(nr);
        tau.insert(tau.begin() + k + 1, x);
    }
    const int nf = (int)rows.size();
    if (nf != (int)fine_breaks.size() - 1 + p) throw std::runtime_error("knot insertion size mismatch");
    const int mf = nf - 2, mc = nc - 2;
    std::vector<double> P((size_t)mf * mc, 0.0);
    for (int i = 1; i <= mf; ++i)
        for (size_t s = 0; s < rows[i].v.size(); ++s) {
            const int J = rows[i].lo + (int)s;
            if (J >= 1 && J <= mc) P[(size_t)(i - 1) * mc + (J - 1)] = rows[i].v[s];
        }
    *m_f = mf;
    *m_c = mc;
    return P;
}

void generalized_eigen(const Factor1D& f, std::vector<double>& V, std::vector<double>& lam) {
    const int m = f.m, p = f.p, bw = 2 * p + 1;
    std::vector<double> M((size_t)m * m, 0.0), K((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i)
        for (int k = 0; k < bw; ++k) {
            const int j = i + k - p;
            if (j < 0 || j >= m) continue;
            M[(size_t)i * m + j] = f.M[(size_t)i * bw + k];
            K[(size_t)i * m + j] = f.K[(size_t)i * bw + k];
        }
    // M = L L^T (Cholesky), C = L^{-1} K L^{-T}, C = W diag(lam) W^T, V = L^{-T} W.
    std::vector<double> L((size_t)m * m, 0.0);
    for (int j = 0; j < m; ++j) {
        double d = M[(size_t)j * m + j];
        for (int k = 0; k < j; ++k) d -= L[(size_t)j * m + k] * L[(size_t)j * m + k];
        if (!(d > 0)) throw std::runtime_error("mass matrix not positive definite");
        L[(size_t)j * m + j] = std::sqrt(d);
        for (int i = j + 1; i < m; ++i) {
            double s = M[(size_t)i * m + j];
            for (int k = 0; k < j; ++k) s -= L[(size_t)i * m + k] * L[(size_t)j * m + k];
            L[(size_t)i * m + j] = s / L[(size_t)j * m + j];
        }
    }
    auto lower_solve = [&](std::vector<double>& B) {   // B <- L^{-1} B, B m x m
        for (int c = 0; c < m; ++c)
            for (int i = 0; i < m; ++i) {
                double s = B[(size_t)i * m + c];
                for (int k = 0; k < i; ++k) s -= L[(size_t)i * m + k] * B[(size_t)k * m + c];
                B[(size_t)i * m + c] = s / L[(size_t)i * m + i];
            }
    };
    std::vector<double> Y = K;
    lower_solve(Y);                                     // Y = L^{-1} K
    std::vector<double> C((size_t)m * m);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) C[(size_t)i * m + j] = Y[(size_t)j * m + i];   // Y^T = K L^{-T}
    lower_solve(C);                                     // C = L^{-1} K L^{-T}
    for (int i = 0; i < m; ++i)
        for (int j = i + 1; j < m; ++j) {
            const double s = 0.5 * (C[(size_t)i * m + j] + C[(size_t)j * m + i]);
            C[(size_t)i * m + j] = s;
            C[(size_t)j * m + i] = s;
        }
    std::vector<double> W;
    jacobi_eigen(m, C, W, lam);
    V = W;                                              // V <- L^{-T} W (back substitution)
    for (int c = 0; c < m; ++c)
        for (int i = m - 1; i >= 0; --i) {
            double s = V[(size_t)i * m + c];
            for (int k = i + 1; k < m; ++k) s -= L[(size_t)k * m + i] * V[(size_t)k * m + c];
            V[(size_t)i * m + c] = s / L[(size_t)i * m + i];
        }
}

std::vector<double> sine_moments(const std::vector<double>& breaks, int p, int modes) {
    const int n = (int)breaks.size() - 1, m = n + p - 2;
    const std::vector<double> U = open_knots(breaks, p);
    std::vector<double> g((size_t)modes * m, 0.0);
    double xg[16], wg[16], N[16];
    gauss_legendre(p + 1, xg, wg);
    const double pi = 3.14159265358979323846;
    for (int e = 0; e < n; ++e) {
        const double a = breaks[e], h = breaks[e + 1] - breaks[e];
        for (int q = 0; q <= p; ++q) {
            const double x = a + 0.5 * (xg[q] + 1.0) * h, w = 0.5 * wg[q] * h;
            basis_on_span(U, p, p + e, x, N);
            for (int r = 0; r <= p; ++r) {
                const int i = e + r - 1;                  // interior index
                if (i < 0 || i >= m) continue;
                for (int k = 0; k < modes; ++k) g[(size_t)k * m + i] += w * std::sin((k + 1) * pi * x) * N[r];
            }
        }
    }
    return g;
}

}  // namespace igamg
