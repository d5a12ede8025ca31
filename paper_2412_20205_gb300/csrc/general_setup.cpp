// Host set-up of the general operator of Sec. 4.3 (Eq. fullelliptic):
// quadrature data, stencil assembly by Gauss quadrature, Galerkin coarse
// operators (Eq. (4)), the coarsest level's dense inverse and the load vector.
#include "host_setup.hpp"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <stdexcept>

namespace igamg {

Quad1D quadrature_1d(const std::vector<double>& breaks, int p) {
    Quad1D Q;
    Q.n = (int)breaks.size() - 1;
    Q.p = p;
    Q.nq = Q.n * (p + 1);
    const std::vector<double> U = open_knots(breaks, p);
    double xg[16], wg[16];
    gauss_legendre(p + 1, xg, wg);
    int ord[16];
    std::iota(ord, ord + p + 1, 0);
    std::sort(ord, ord + p + 1, [&](int a, int b) { return xg[a] < xg[b]; });
    Q.x.resize(Q.nq);
    Q.w.resize(Q.nq);
    Q.N.resize((size_t)Q.nq * (p + 1));
    Q.dN.resize((size_t)Q.nq * (p + 1));
    for (int e = 0; e < Q.n; ++e) {
        const double a = breaks[e], h = breaks[e + 1] - breaks[e];
        for (int g = 0; g <= p; ++g) {
            const int q = e * (p + 1) + g;
            Q.x[q] = a + 0.5 * (xg[ord[g]] + 1.0) * h;
            Q.w[q] = 0.5 * wg[ord[g]] * h;
            basis_and_derivative(U, p, p + e, Q.x[q], &Q.N[(size_t)q * (p + 1)], &Q.dN[(size_t)q * (p + 1)]);
        }
    }
    return Q;
}

Stencil2D assemble_general(const Quad1D& qx, const Quad1D& qy, const double* coef) {
    const int p = qx.p, P1 = p + 1, W = 2 * p + 1;
    Stencil2D A;
    A.p = p;
    A.mx = qx.n + p - 2;
    A.my = qy.n + p - 2;
    const size_t N = A.N(), nq = (size_t)qx.nq * qy.nq;
    A.S.assign((size_t)W * W * N, 0.0);
    for (int ey = 0; ey < qy.n; ++ey)
        for (int gy = 0; gy < P1; ++gy) {
            const int qyi = ey * P1 + gy;
            const double* Ny = &qy.N[(size_t)qyi * P1];
            const double* dNy = &qy.dN[(size_t)qyi * P1];
            for (int ex = 0; ex < qx.n; ++ex)
                for (int gx = 0; gx < P1; ++gx) {
                    const int qxi = ex * P1 + gx;
                    const size_t q = (size_t)qyi * qx.nq + qxi;
                    const double w = qx.w[qxi] * qy.w[qyi];
                    const double a11 = coef[q], a12 = coef[nq + q], a22 = coef[2 * nq + q];
                    const double b1 = coef[3 * nq + q], b2 = coef[4 * nq + q], cc = coef[5 * nq + q];
                    const double* Nx = &qx.N[(size_t)qxi * P1];
                    const double* dNx = &qx.dN[(size_t)qxi * P1];
                    for (int ry = 0; ry < P1; ++ry) {
                        const int iy = ey + ry - 1;                       // interior index of the test function
                        if (iy < 0 || iy >= A.my) continue;
                        for (int rx = 0; rx < P1; ++rx) {
                            const int ix = ex + rx - 1;
                            if (ix < 0 || ix >= A.mx) continue;
                            const double v = Nx[rx] * Ny[ry], gx_ = dNx[rx] * Ny[ry], gy_ = Nx[rx] * dNy[ry];
                            const size_t I = (size_t)iy * A.mx + ix;
                            for (int sy = 0; sy < P1; ++sy) {
                                const int jy = ey + sy - 1;               // trial function
                                if (jy < 0 || jy >= A.my) continue;
                                for (int sx = 0; sx < P1; ++sx) {
                                    const int jx = ex + sx - 1;
                                    if (jx < 0 || jx >= A.mx) continue;
                                    const double u = Nx[sx] * Ny[sy], ux = dNx[sx] * Ny[sy], uy = Nx[sx] * dNy[sy];
                                    const double val = gx_ * (a11 * ux + a12 * uy) + gy_ * (a12 * ux + a22 * uy) +
                                                       (b1 * ux + b2 * uy) * v + cc * u * v;
                                    const int k = (jy - iy + p) * W + (jx - ix + p);
                                    A.S[(size_t)k * N + I] += w * val;
                                }
                            }
                        }
                    }
                }
        }
    return A;
}

Stencil2D galerkin_coarse(const Stencil2D& A, const std::vector<double>& Px, int mcx, const std::vector<double>& Py,
                          int mcy) {
    const int p = A.p, W = 2 * p + 1;
    const int mfx = A.mx, mfy = A.my;
    // non-zero column range of every fine row of the 1D prolongations
    auto ranges = [](const std::vector<double>& P, int mf, int mc, std::vector<int>& lo, std::vector<int>& hi) {
        lo.assign(mf, 0);
        hi.assign(mf, -1);
        for (int i = 0; i < mf; ++i) {
            int l = -1, h = -2;
            for (int J = 0; J < mc; ++J)
                if (P[(size_t)i * mc + J] != 0.0) { if (l < 0) l = J; h = J; }
            lo[i] = l < 0 ? 0 : l;
            hi[i] = l < 0 ? -1 : h;
        }
    };
    std::vector<int> lx, hx, ly, hy;
    ranges(Px, mfx, mcx, lx, hx);
    ranges(Py, mfy, mcy, ly, hy);
    Stencil2D C;
    C.p = p;
    C.mx = mcx;
    C.my = mcy;
    const size_t Nc = C.N(), Nf = A.N();
    C.S.assign((size_t)W * W * Nc, 0.0);
    for (int ky = 0; ky < mfy; ++ky)
        for (int kx = 0; kx < mfx; ++kx) {
            const size_t K = (size_t)ky * mfx + kx;
            for (int dy = -p; dy <= p; ++dy)
                for (int dx = -p; dx <= p; ++dx) {
                    const double a = A.S[(size_t)((dy + p) * W + dx + p) * Nf + K];
                    if (a == 0.0) continue;
                    const int lxx = kx + dx, lyy = ky + dy;                // fine column L
                    if (lxx < 0 || lxx >= mfx || lyy < 0 || lyy >= mfy) continue;
                    for (int iy = ly[ky]; iy <= hy[ky]; ++iy)
                        for (int ix = lx[kx]; ix <= hx[kx]; ++ix) {
                            const double pk = Px[(size_t)kx * mcx + ix] * Py[(size_t)ky * mcy + iy];
                            if (pk == 0.0) continue;
                            for (int jy = ly[lyy]; jy <= hy[lyy]; ++jy)
                                for (int jx = lx[lxx]; jx <= hx[lxx]; ++jx) {
                                    const double pl = Px[(size_t)lxx * mcx + jx] * Py[(size_t)lyy * mcy + jy];
                                    if (pl == 0.0) continue;
                                    const int ox = jx - ix, oy = jy - iy;
                                    if (ox < -p || ox > p || oy < -p || oy > p)
                                        throw std::runtime_error("Galerkin coarse operator outside the stencil");
                                    C.S[(size_t)((oy + p) * W + ox + p) * Nc + (size_t)iy * mcx + ix] += pk * a * pl;
                                }
                        }
                }
        }
    return C;
}

bool dense_inverse(const Stencil2D& A, std::vector<double>& inv) {
    const int p = A.p, W = 2 * p + 1;
    const int n = (int)A.N();
    std::vector<double> M((size_t)n * n, 0.0);
    for (int I = 0; I < n; ++I) {
        const int ix = I % A.mx, iy = I / A.mx;
        for (int dy = -p; dy <= p; ++dy)
            for (int dx = -p; dx <= p; ++dx) {
                const int jx = ix + dx, jy = iy + dy;
                if (jx < 0 || jx >= A.mx || jy < 0 || jy >= A.my) continue;
                M[(size_t)I * n + jy * A.mx + jx] = A.S[(size_t)((dy + p) * W + dx + p) * n + I];
            }
    }
    inv.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(M[(size_t)r * n + c]) > std::fabs(M[(size_t)piv * n + c])) piv = r;
        if (M[(size_t)piv * n + c] == 0.0) return false;
        if (piv != c)
            for (int k = 0; k < n; ++k) {
                std::swap(M[(size_t)c * n + k], M[(size_t)piv * n + k]);
                std::swap(inv[(size_t)c * n + k], inv[(size_t)piv * n + k]);
            }
        const double d = 1.0 / M[(size_t)c * n + c];
        for (int k = 0; k < n; ++k) {
            M[(size_t)c * n + k] *= d;
            inv[(size_t)c * n + k] *= d;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = M[(size_t)r * n + c];
            if (f == 0.0) continue;
            for (int k = 0; k < n; ++k) {
                M[(size_t)r * n + k] -= f * M[(size_t)c * n + k];
                inv[(size_t)r * n + k] -= f * inv[(size_t)c * n + k];
            }
        }
    }
    return true;
}

std::vector<double> load_general(const Quad1D& qx, const Quad1D& qy, const double* fq) {
    const int p = qx.p, P1 = p + 1;
    const int mx = qx.n + p - 2, my = qy.n + p - 2;
    std::vector<double> b((size_t)mx * my, 0.0);
    for (int ey = 0; ey < qy.n; ++ey)
        for (int gy = 0; gy < P1; ++gy) {
            const int qyi = ey * P1 + gy;
            for (int ex = 0; ex < qx.n; ++ex)
                for (int gx = 0; gx < P1; ++gx) {
                    const int qxi = ex * P1 + gx;
                    const double wf = qx.w[qxi] * qy.w[qyi] * fq[(size_t)qyi * qx.nq + qxi];
                    for (int ry = 0; ry < P1; ++ry) {
                        const int iy = ey + ry - 1;
                        if (iy < 0 || iy >= my) continue;
                        for (int rx = 0; rx < P1; ++rx) {
                            const int ix = ex + rx - 1;
                            if (ix < 0 || ix >= mx) continue;
                            b[(size_t)iy * mx + ix] += wf * qx.N[(size_t)qxi * P1 + rx] * qy.N[(size_t)qyi * P1 + ry];
                        }
                    }
                }
        }
    return b;
}

}  // namespace igamg
