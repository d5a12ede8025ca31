// Coarse-level tail of the 2D V-cycle in one CTA.
//
// Below a few thousand unknowns per level, the per-level kernels of
// Algorithm 2 do almost no work per launch: a V-cycle spends most of its
// coarse-level time in launch latency (one launch per GS row phase, residual
// and transfer pass).  Here one CTA runs the whole coarse part of the cycle:
// - pre-smoothing, residual and restriction from level lc down to level 1;
// - the direct coarsest solve;
// - prolongation and post-smoothing back up to level lc.
// Every level's x and b stay in shared memory, with barriers between the
// dependent steps.  The arithmetic is that of the per-level kernels: the same
// colours in the same order, the same transfer operators and fast
// diagonalisation.  Only A x is evaluated directly from the two 1D band pairs
// instead of from row partial sums.
#include "device.hpp"
#include "bands.cuh"

#include <algorithm>

namespace igamg {
namespace dev {

constexpr int kTailThreads = 512;

// One level's operator data as staged in shared memory: band-major 1D factors
// (Mx[b * mx + i] = M_x(i, i + b - p), zero outside the matrix) and 1 / A_qq.
// Iterates x are stored with a zero halo of p nodes on every side (row
// stride mx + 2p), so that stencil loads need no bounds tests.
template <typename T>
struct TailLevel {
    int mx, my;
    const T *Mx, *Kx, *My, *Ky, *inv;
};

template <int P>
__device__ __forceinline__ int padded(int i, int j, int mx) {
    return (j + P) * (mx + 2 * P) + i + P;
}

// (A x)_(i, j) for A = K_y (x) M_x + M_y (x) K_x (Sec. 2, Eq. (2)); xp is the
// padded iterate.
template <typename T, int P>
__device__ __forceinline__ T tail_Ax(const TailLevel<T>& S, const T* xp, int i, int j) {
    const int mx = S.mx, my = S.my, W = mx + 2 * P;
    T cm[2 * P + 1], ck[2 * P + 1];
#pragma unroll
    for (int b = 0; b <= 2 * P; ++b) {
        cm[b] = S.Mx[b * mx + i];
        ck[b] = S.Kx[b * mx + i];
    }
    const T* base = xp + j * W + i;                     // padded (i - p, j - p)
    T acc = 0;
#pragma unroll
    for (int bj = 0; bj <= 2 * P; ++bj) {
        const T* xr = base + bj * W;
        T sM = 0, sK = 0;
#pragma unroll
        for (int bi = 0; bi <= 2 * P; ++bi) {
            const T v = xr[bi];
            sM += cm[bi] * v;
            sK += ck[bi] * v;
        }
        acc += S.Ky[bj * my + j] * sM + S.My[bj * my + j] * sK;
    }
    return acc;
}

// One multicolour GS sweep: colour c = cx + (p+1) cy, ascending (pre) or
// descending (post); x_q += (b_q - (A x)_q) / A_qq on every node of colour c.
template <typename T, int P>
__device__ void tail_gs(const TailLevel<T>& S, T* xp, const T* b, bool descending) {
    constexpr int NC = P + 1;
    const int mx = S.mx, my = S.my;
    for (int cc = 0; cc < NC * NC; ++cc) {
        const int c = descending ? NC * NC - 1 - cc : cc;
        const int cx = c % NC, cy = c / NC;
        const int nx = (mx - cx + NC - 1) / NC, ny = (my - cy + NC - 1) / NC;
        for (int t = threadIdx.x; t < nx * ny; t += blockDim.x) {
            const int jt = t / nx;
            const int i = cx + NC * (t - jt * nx), j = cy + NC * jt;
            const int q = j * mx + i;
            xp[padded<P>(i, j, mx)] += (b[q] - tail_Ax<T, P>(S, xp, i, j)) * S.inv[q];
        }
        __syncthreads();
    }
}

// bc = P^T (b - A x): the residual, then the x and y axes of the restriction.
template <typename T, int P>
__device__ void tail_restrict(const TailLevel<T>& S, const TransferView<T>& X, const T* xp, const T* b, T* r, T* t,
                              T* bc) {
    const int mx = S.mx, my = S.my;
    for (int q = threadIdx.x; q < mx * my; q += blockDim.x) {
        const int j = q / mx;
        r[q] = b[q] - tail_Ax<T, P>(S, xp, q - j * mx, j);
    }
    __syncthreads();
    const int mcx = X.mc[0], mcy = X.mc[1];
    for (int q = threadIdx.x; q < mcx * my; q += blockDim.x) {
        const int I = q % mcx, j = q / mcx, lo = X.rlo[0][I];
        T acc = 0;
        for (int s = 0; s < X.rw[0]; ++s) {
            const int f = lo + s;
            if (f < 0 || f >= mx) continue;
            acc += X.rv[0][I * X.rw[0] + s] * r[j * mx + f];
        }
        t[q] = acc;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < mcx * mcy; q += blockDim.x) {
        const int I = q % mcx, J = q / mcx, lo = X.rlo[1][J];
        T acc = 0;
        for (int s = 0; s < X.rw[1]; ++s) {
            const int f = lo + s;
            if (f < 0 || f >= my) continue;
            acc += X.rv[1][J * X.rw[1] + s] * t[f * mcx + I];
        }
        bc[q] = acc;
    }
    __syncthreads();
}

// x += P e (both padded): the x axis into t, then the y axis added to x.
template <typename T, int P>
__device__ void tail_prolong(const TransferView<T>& X, const T* ep, T* t, T* xp) {
    const int mfx = X.mf[0], mfy = X.mf[1], mcx = X.mc[0], mcy = X.mc[1];
    for (int q = threadIdx.x; q < mfx * mcy; q += blockDim.x) {
        const int i = q % mfx, J = q / mfx, lo = X.plo[0][i];
        T acc = 0;
        for (int s = 0; s < X.pw[0]; ++s) {
            const int f = lo + s;
            if (f < 0 || f >= mcx) continue;
            acc += X.pv[0][i * X.pw[0] + s] * ep[padded<P>(f, J, mcx)];
        }
        t[q] = acc;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < mfx * mfy; q += blockDim.x) {
        const int i = q % mfx, j = q / mfx, lo = X.plo[1][j];
        T acc = 0;
        for (int s = 0; s < X.pw[1]; ++s) {
            const int f = lo + s;
            if (f < 0 || f >= mcy) continue;
            acc += X.pv[1][j * X.pw[1] + s] * t[f * mfx + i];
        }
        xp[padded<P>(i, j, mfx)] += acc;
    }
    __syncthreads();
}

// e = (V_y (x) V_x) diag(laminv) (V_y (x) V_x)^T r (fast diagonalisation),
// written into the padded coarsest iterate.
template <typename T, int P>
__device__ void tail_coarse(const CoarseView<T>& C, const T* r, T* a, T* bb, T* ep) {
    const int m0 = C.m[0], m1 = C.m[1], N = m0 * m1;
    auto pass = [&](const T* in, T* out, int axis, bool transpose, bool pad) {
        const int md = C.m[axis], stride = axis == 0 ? 1 : m0;
        const T* V = C.V[axis];
        for (int idx = threadIdx.x; idx < N; idx += blockDim.x) {
            const int I = axis == 0 ? idx % m0 : idx / m0;
            const int base = idx - I * stride;
            T acc = 0;
            for (int s = 0; s < md; ++s) acc += (transpose ? V[s * md + I] : V[I * md + s]) * in[base + s * stride];
            out[pad ? padded<P>(idx % m0, idx / m0, m0) : idx] = acc;
        }
        __syncthreads();
    };
    pass(r, a, 0, true, false);
    pass(a, bb, 1, true, false);
    for (int i = threadIdx.x; i < N; i += blockDim.x) bb[i] *= C.laminv[i];
    __syncthreads();
    pass(bb, a, 1, false, false);
    pass(a, ep, 0, false, true);
}

// X[l] with its tables in shared memory at off_tr[l] (plo, pv, rlo, rv of the
// x axis, then of the y axis); the sizes add up to tail_transfer_elems(X[l]).
template <typename T>
__device__ __forceinline__ TransferView<T> staged_transfer(const TailView<T>& V, int l, T* sm) {
    TransferView<T> Y = V.X[l];
    T* f = sm + V.off_tr[l];
    for (int d = 0; d < 2; ++d) {
        Y.plo[d] = reinterpret_cast<const int*>(f);
        f += Y.mf[d];
        Y.pv[d] = f;
        f += Y.mf[d] * Y.pw[d];
        Y.rlo[d] = reinterpret_cast<const int*>(f);
        f += Y.mc[d];
        Y.rv[d] = f;
        f += Y.mc[d] * Y.rw[d];
    }
    return Y;
}

template <typename T, int P>
__global__ void __launch_bounds__(kTailThreads, 1) k_coarse_tail(TailView<T> V, const T* __restrict__ b_in,
                                                                 T* __restrict__ x_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int lc = V.lc;
    T* r = sm + V.off_r;
    T* t = sm + V.off_t;
    {
        const int N = V.L[lc].m[0] * V.L[lc].m[1];
        T* b = sm + V.off_b[lc];
        for (int q = threadIdx.x; q < N; q += blockDim.x) b[q] = b_in[q];
    }
    for (int l = 0; l <= lc; ++l) {                     // coarse e^0 = 0 on every level, zero halos
        const int NP = (V.L[l].m[0] + 2 * P) * (V.L[l].m[1] + 2 * P);
        T* x = sm + V.off_x[l];
        for (int q = threadIdx.x; q < NP; q += blockDim.x) x[q] = 0;
    }
    for (int l = 1; l <= lc; ++l) {                     // stage the operator data
        const LevelView<T>& L = V.L[l];
        const int mx = L.m[0], my = L.m[1], N = mx * my;
        T* inv = sm + V.off_inv[l];
        for (int q = threadIdx.x; q < N; q += blockDim.x) inv[q] = L.invdiag[q];
        T* band = sm + V.off_band[l];
        for (int q = threadIdx.x; q < (2 * P + 1) * mx; q += blockDim.x) {
            const int b = q / mx, i = q % mx;
            band[q] = band_m(L, i, b);
            band[(2 * P + 1) * mx + q] = band_k(L, i, b);
        }
        band += 2 * (2 * P + 1) * mx;
        for (int q = threadIdx.x; q < (2 * P + 1) * my; q += blockDim.x) {
            const int b = q / my, j = q % my;
            band[q] = band_md(L, 1, j, b);
            band[(2 * P + 1) * my + q] = band_kd(L, 1, j, b);
        }
    }
    // transfer tables and the coarsest eigenbasis, read by one pass each
    for (int l = 1; l <= lc; ++l) {
        const TransferView<T>& X = V.X[l];
        const TransferView<T> Y = staged_transfer(V, l, sm);
        for (int d = 0; d < 2; ++d) {
            int* plo = const_cast<int*>(Y.plo[d]);
            int* rlo = const_cast<int*>(Y.rlo[d]);
            T* pv = const_cast<T*>(Y.pv[d]);
            T* rv = const_cast<T*>(Y.rv[d]);
            for (int q = threadIdx.x; q < X.mf[d]; q += blockDim.x) plo[q] = X.plo[d][q];
            for (int q = threadIdx.x; q < X.mf[d] * X.pw[d]; q += blockDim.x) pv[q] = X.pv[d][q];
            for (int q = threadIdx.x; q < X.mc[d]; q += blockDim.x) rlo[q] = X.rlo[d][q];
            for (int q = threadIdx.x; q < X.mc[d] * X.rw[d]; q += blockDim.x) rv[q] = X.rv[d][q];
        }
    }
    CoarseView<T> Cs = V.C;
    {
        T* f = sm + V.off_cv;
        const int m0 = V.C.m[0], m1 = V.C.m[1];
        for (int q = threadIdx.x; q < m0 * m0; q += blockDim.x) f[q] = V.C.V[0][q];
        for (int q = threadIdx.x; q < m1 * m1; q += blockDim.x) f[m0 * m0 + q] = V.C.V[1][q];
        for (int q = threadIdx.x; q < m0 * m1; q += blockDim.x) f[m0 * m0 + m1 * m1 + q] = V.C.laminv[q];
        Cs.V[0] = f;
        Cs.V[1] = f + m0 * m0;
        Cs.laminv = f + m0 * m0 + m1 * m1;
    }
    __syncthreads();
    auto level = [&](int l) {
        const int mx = V.L[l].m[0], my = V.L[l].m[1];
        const T* band = sm + V.off_band[l];
        return TailLevel<T>{mx, my, band, band + (2 * P + 1) * mx, band + 2 * (2 * P + 1) * mx,
                            band + 2 * (2 * P + 1) * mx + (2 * P + 1) * my, sm + V.off_inv[l]};
    };
    for (int l = lc; l >= 1; --l) {
        T* x = sm + V.off_x[l];
        const T* b = sm + V.off_b[l];
        const TailLevel<T> S = level(l);
        tail_gs<T, P>(S, x, b, false);                                           // pre-smooth
        tail_restrict<T, P>(S, staged_transfer(V, l, sm), x, b, r, t, sm + V.off_b[l - 1]);   // R (b - A x)
    }
    tail_coarse<T, P>(Cs, sm + V.off_b[0], r, t, sm + V.off_x[0]);              // direct
    for (int l = 1; l <= lc; ++l) {
        T* x = sm + V.off_x[l];
        tail_prolong<T, P>(staged_transfer(V, l, sm), sm + V.off_x[l - 1], t, x);              // x += P e
        tail_gs<T, P>(level(l), x, sm + V.off_b[l], true);                       // post-smooth
    }
    const int mx = V.L[lc].m[0], N = mx * V.L[lc].m[1];
    const T* x = sm + V.off_x[lc];
    for (int q = threadIdx.x; q < N; q += blockDim.x) x_out[q] = x[padded<P>(q % mx, q / mx, mx)];
}

template <typename F>
static void tail_with_p(int p, F&& f) {
    switch (p) {
        case 1: f(std::integral_constant<int, 1>()); break;
        case 2: f(std::integral_constant<int, 2>()); break;
        case 3: f(std::integral_constant<int, 3>()); break;
        case 4: f(std::integral_constant<int, 4>()); break;
        case 5: f(std::integral_constant<int, 5>()); break;
        case 6: f(std::integral_constant<int, 6>()); break;
        case 7: f(std::integral_constant<int, 7>()); break;
        default: break;
    }
}

namespace {
size_t g_tail_limit[64] = {};
}

void prepare_tail_kernels(int optin) {
    int dev = 0;
    cudaGetDevice(&dev);
    for (int p = 1; p <= kMaxP; ++p)
        tail_with_p(p, [&](auto PC) {
            constexpr int P = decltype(PC)::value;
            cudaFuncSetAttribute(k_coarse_tail<float, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        });
    if (dev >= 0 && dev < 64) g_tail_limit[dev] = (size_t)optin;
}

size_t tail_smem_limit() {
    int dev = 0;
    cudaGetDevice(&dev);
    return (dev >= 0 && dev < 64) ? g_tail_limit[dev] : 0;
}

template <typename T>
void coarse_tail(cudaStream_t s, const TailView<T>& V, const T* b, T* x) {
    tail_with_p(V.L[V.lc].p, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        k_coarse_tail<T, P><<<1, kTailThreads, V.smem, s>>>(V, b, x);
    });
    count_launch();
}

template void coarse_tail<float>(cudaStream_t, const TailView<float>&, const float*, float*);

}  // namespace dev
}  // namespace igamg
