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

// Staging copies global -> shared with cp.async (4-byte elements): every
// thread issues all of its copies before waiting once, so the operator data
// of all tail levels arrives in about one memory round trip.
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename E>
__device__ __forceinline__ void stage(E* dst, const E* src, int n) {
    static_assert(sizeof(E) == 4, "4-byte elements");
    for (int q = threadIdx.x; q < n; q += blockDim.x) cp_async4(dst + q, src + q);
}

// One level as the tail sees it, all in shared memory:
// - band-major 1D factors (Mx[b * mx + i] = M_x(i, i + b - p), zero outside
//   the matrix) and 1 / A_qq;
// - the iterate x with a zero halo of p nodes on every side (row stride
//   mx + 2p), so that x-window loads need no bounds tests;
// - the row partial sums T_M = (I (x) M_x) x and T_K = (I (x) K_x) x with p
//   zero rows above and below (row j at (j + p) mx).
// In the uniform interior of x the x-band comes from the level view's
// Toeplitz constants (uniform loads), at the p boundary columns from Mx/Kx.
template <typename T>
struct TailLevel {
    int mx, my, tlo, thi;
    const T *Mx, *Kx, *My, *Ky, *inv;
    T *TM, *TK;
    const T* Mc;                          // Toeplitz interior of M_x, K_x (2p+1 each)
    const T* Kc;
};

template <int P>
__device__ __forceinline__ int padded(int i, int j, int mx) {
    return (j + P) * (mx + 2 * P) + i + P;
}

// sum_b M_x(i, b) x(i + b - p, j) and the K_x sum, from the padded iterate
template <typename T, int P>
__device__ __forceinline__ void tail_xsums(const TailLevel<T>& S, const T* xp, int i, int j, T& sM, T& sK) {
    const T* xr = xp + (j + P) * (S.mx + 2 * P) + i;          // padded (i - p, j)
    sM = 0;
    sK = 0;
    if (i >= S.tlo && i < S.thi) {
#pragma unroll
        for (int b = 0; b <= 2 * P; ++b) {
            const T v = xr[b];
            sM += S.Mc[b] * v;
            sK += S.Kc[b] * v;
        }
    } else {
#pragma unroll
        for (int b = 0; b <= 2 * P; ++b) {
            const T v = xr[b];
            sM += S.Mx[b * S.mx + i] * v;
            sK += S.Kx[b * S.mx + i] * v;
        }
    }
}

// (A x)_(i, j) = sum_bj K_y(j, bj) T_M(i, j + bj - p) + M_y(j, bj) T_K(...),
// A = K_y (x) M_x + M_y (x) K_x (Sec. 2, Eq. (2)); rows bj != skip only.
template <typename T, int P>
__device__ __forceinline__ T tail_couple(const TailLevel<T>& S, int i, int j, int skip) {
    T acc = 0;
#pragma unroll
    for (int bj = 0; bj <= 2 * P; ++bj) {
        if (bj == skip) continue;
        const int row = (j + bj) * S.mx + i;                      // padded row j + bj - p
        acc += S.Ky[bj * S.my + j] * S.TM[row] + S.My[bj * S.my + j] * S.TK[row];
    }
    return acc;
}

// T_M, T_K of every row from x.
template <typename T, int P>
__device__ void tail_xpass(const TailLevel<T>& S, const T* xp) {
    for (int q = threadIdx.x; q < S.mx * S.my; q += blockDim.x) {
        const int j = q / S.mx, i = q - j * S.mx;
        T sM, sK;
        tail_xsums<T, P>(S, xp, i, j, sM, sK);
        S.TM[(j + P) * S.mx + i] = sM;
        S.TK[(j + P) * S.mx + i] = sK;
    }
    __syncthreads();
}

// One multicolour GS sweep: colour c = cx + (p+1) cy, ascending (pre) or
// descending (post); x_q += (b_q - (A x)_q) / A_qq on every node of colour c.
// Row phases: for fixed cy the rows j = cy mod (p+1) never couple, so each
// warp takes whole rows and runs their p+1 x-colours with warp barriers only;
// the CTA synchronises once per row phase.  During a row's colours the other
// rows' T_M, T_K are frozen and the row's own part is summed from x; the row's
// T_M, T_K are refreshed when its colours are done.
template <typename T, int P>
__device__ void tail_gs(const TailLevel<T>& S, T* xp, const T* b, bool descending) {
    constexpr int NC = P + 1;
    const int mx = S.mx, my = S.my, W = mx + 2 * P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    T mc[2 * P + 1], kc[2 * P + 1];                     // interior x-band, in registers
#pragma unroll
    for (int bb = 0; bb <= 2 * P; ++bb) {
        mc[bb] = S.Mc[bb];
        kc[bb] = S.Kc[bb];
    }
    for (int pc = 0; pc < NC; ++pc) {
        const int cy = descending ? P - pc : pc;
        const int nrows = (my - cy + NC - 1) / NC;
        for (int rr = warp; rr < nrows; rr += nwarps) {
            const int j = cy + NC * rr;
            T ky[2 * P + 1], mY[2 * P + 1];             // the row's y-band, in registers
#pragma unroll
            for (int bj = 0; bj <= 2 * P; ++bj) {
                ky[bj] = S.Ky[bj * my + j];
                mY[bj] = S.My[bj * my + j];
            }
            const T* xr0 = xp + (j + P) * W;
            for (int c = 0; c < NC; ++c) {
                const int cx = descending ? P - c : c;
                const int nx = (mx - cx + NC - 1) / NC;
                for (int s0 = 0; s0 < nx; s0 += 32) {
                    if (s0 + lane < nx) {
                        const int i = cx + NC * (s0 + lane);
                        const int q = j * mx + i;
                        const T* xr = xr0 + i;                      // padded (i - p, j)
                        T sM = 0, sK = 0;
                        if (i >= S.tlo && i < S.thi) {
#pragma unroll
                            for (int bb = 0; bb <= 2 * P; ++bb) {
                                const T v = xr[bb];
                                sM += mc[bb] * v;
                                sK += kc[bb] * v;
                            }
                        } else {
#pragma unroll
                            for (int bb = 0; bb <= 2 * P; ++bb) {
                                const T v = xr[bb];
                                sM += S.Mx[bb * mx + i] * v;
                                sK += S.Kx[bb * mx + i] * v;
                            }
                        }
                        T ax = ky[P] * sM + mY[P] * sK;
#pragma unroll
                        for (int bj = 0; bj <= 2 * P; ++bj) {
                            if (bj == P) continue;
                            const int row = (j + bj) * mx + i;          // padded T row j + bj - p
                            ax += ky[bj] * S.TM[row] + mY[bj] * S.TK[row];
                        }
                        xp[(j + P) * W + i + P] += (b[q] - ax) * S.inv[q];
                    }
                }
                __syncwarp();
            }
            for (int i = lane; i < mx; i += 32) {       // refresh the row's T_M, T_K
                const T* xr = xr0 + i;
                T sM = 0, sK = 0;
                if (i >= S.tlo && i < S.thi) {
#pragma unroll
                    for (int bb = 0; bb <= 2 * P; ++bb) {
                        const T v = xr[bb];
                        sM += mc[bb] * v;
                        sK += kc[bb] * v;
                    }
                } else {
#pragma unroll
                    for (int bb = 0; bb <= 2 * P; ++bb) {
                        const T v = xr[bb];
                        sM += S.Mx[bb * mx + i] * v;
                        sK += S.Kx[bb * mx + i] * v;
                    }
                }
                S.TM[(j + P) * mx + i] = sM;
                S.TK[(j + P) * mx + i] = sK;
            }
        }
        __syncthreads();
    }
}

// One weighted-Jacobi sweep x += omega D^{-1} (b - A x) (Sec. 4) with every
// node from the same x (A x from T_M, T_K), using the scratch vector d; then
// T_M, T_K of the new x.
template <typename T, int P>
__device__ void tail_jacobi(const TailLevel<T>& S, T* xp, const T* b, T omega, T* d) {
    const int mx = S.mx, my = S.my;
    for (int q = threadIdx.x; q < mx * my; q += blockDim.x) {
        const int j = q / mx, i = q - j * mx;
        d[q] = omega * (b[q] - tail_couple<T, P>(S, i, j, -1)) * S.inv[q];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < mx * my; q += blockDim.x) {
        const int j = q / mx, i = q - j * mx;
        xp[padded<P>(i, j, mx)] += d[q];
    }
    __syncthreads();
    tail_xpass<T, P>(S, xp);
}

// bc = P^T (b - A x): the residual, then the x and y axes of the restriction.
template <typename T, int P>
__device__ void tail_restrict(const TailLevel<T>& S, const TransferView<T>& X, const T* b, T* r, T* t, T* bc) {
    const int mx = S.mx, my = S.my;
    for (int q = threadIdx.x; q < mx * my; q += blockDim.x) {
        const int j = q / mx;
        r[q] = b[q] - tail_couple<T, P>(S, q - j * mx, j, -1);
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
                                                                 T* __restrict__ x_out, int jacobi, T omega) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int lc = V.lc;
    T* r = sm + V.off_r;
    T* t = sm + V.off_t;
    // Operator data (uploaded at assembly, written by no kernel) is staged
    // before the wait on the previous kernel; the right side b after it.
    for (int l = 1; l <= lc; ++l) {                     // operator data of the smoothed levels
        const LevelView<T>& L = V.L[l];
        const int mx = L.m[0], my = L.m[1];
        stage(sm + V.off_inv[l], L.invdiag, mx * my);
        T* band = sm + V.off_band[l];
        stage(band, L.Mb[0], (2 * P + 1) * mx);
        stage(band + (2 * P + 1) * mx, L.Kb[0], (2 * P + 1) * mx);
        stage(band + 2 * (2 * P + 1) * mx, L.Mb[1], (2 * P + 1) * my);
        stage(band + 2 * (2 * P + 1) * mx + (2 * P + 1) * my, L.Kb[1], (2 * P + 1) * my);
        const TransferView<T>& X = V.X[l];                // transfer tables
        const TransferView<T> Y = staged_transfer(V, l, sm);
        for (int d = 0; d < 2; ++d) {
            stage(const_cast<int*>(Y.plo[d]), X.plo[d], X.mf[d]);
            stage(const_cast<T*>(Y.pv[d]), X.pv[d], X.mf[d] * X.pw[d]);
            stage(const_cast<int*>(Y.rlo[d]), X.rlo[d], X.mc[d]);
            stage(const_cast<T*>(Y.rv[d]), X.rv[d], X.mc[d] * X.rw[d]);
        }
    }
    CoarseView<T> Cs = V.C;                             // coarsest eigenbasis
    {
        T* f = sm + V.off_cv;
        const int m0 = V.C.m[0], m1 = V.C.m[1];
        stage(f, V.C.V[0], m0 * m0);
        stage(f + m0 * m0, V.C.V[1], m1 * m1);
        stage(f + m0 * m0 + m1 * m1, V.C.laminv, m0 * m1);
        Cs.V[0] = f;
        Cs.V[1] = f + m0 * m0;
        Cs.laminv = f + m0 * m0 + m1 * m1;
    }
    for (int l = 0; l <= lc; ++l) {                     // coarse e^0 = 0 on every level, zero halos
        const int mx = V.L[l].m[0], my = V.L[l].m[1];
        T* x = sm + V.off_x[l];
        for (int q = threadIdx.x; q < (mx + 2 * P) * (my + 2 * P); q += blockDim.x) x[q] = 0;
        if (l == 0) continue;
        T* tmk = sm + V.off_tm[l];                      // T_M = T_K = 0 for x = 0
        for (int q = threadIdx.x; q < 2 * (my + 2 * P) * mx; q += blockDim.x) tmk[q] = 0;
        T* tc = sm + V.off_tc[l];
        for (int b = threadIdx.x; b <= 2 * P; b += blockDim.x) {
            tc[b] = V.L[l].Mc[0][b];
            tc[2 * P + 1 + b] = V.L[l].Kc[0][b];
        }
    }
    pdl_enter();
    stage(sm + V.off_b[lc], b_in, V.L[lc].m[0] * V.L[lc].m[1]);
    cp_async_wait_all();
    __syncthreads();
    auto level = [&](int l) {
        const int mx = V.L[l].m[0], my = V.L[l].m[1];
        const T* band = sm + V.off_band[l];
        T* tmk = sm + V.off_tm[l];
        const T* tc = sm + V.off_tc[l];
        return TailLevel<T>{mx, my, V.L[l].tlo[0], V.L[l].thi[0], band, band + (2 * P + 1) * mx,
                            band + 2 * (2 * P + 1) * mx, band + 2 * (2 * P + 1) * mx + (2 * P + 1) * my,
                            sm + V.off_inv[l], tmk, tmk + (my + 2 * P) * mx, tc, tc + 2 * P + 1};
    };
    for (int l = lc; l >= 1; --l) {
        T* x = sm + V.off_x[l];
        const T* b = sm + V.off_b[l];
        const TailLevel<T> S = level(l);
        if (jacobi) tail_jacobi<T, P>(S, x, b, omega, r);                       // pre-smooth
        else tail_gs<T, P>(S, x, b, false);
        tail_restrict<T, P>(S, staged_transfer(V, l, sm), b, r, t, sm + V.off_b[l - 1]);   // R (b - A x)
    }
    tail_coarse<T, P>(Cs, sm + V.off_b[0], r, t, sm + V.off_x[0]);              // direct
    for (int l = 1; l <= lc; ++l) {
        T* x = sm + V.off_x[l];
        const TailLevel<T> S = level(l);
        tail_prolong<T, P>(staged_transfer(V, l, sm), sm + V.off_x[l - 1], t, x);              // x += P e
        tail_xpass<T, P>(S, x);
        if (jacobi) tail_jacobi<T, P>(S, x, sm + V.off_b[l], omega, r);        // post-smooth
        else tail_gs<T, P>(S, x, sm + V.off_b[l], true);
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
void coarse_tail(cudaStream_t s, const TailView<T>& V, const T* b, T* x, int jacobi, T omega) {
    tail_with_p(V.L[V.lc].p, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        launch_chained(k_coarse_tail<T, P>, 1, kTailThreads, V.smem, s, V, b, x, jacobi, omega);
    });
    count_launch();
}

template void coarse_tail<float>(cudaStream_t, const TailView<float>&, const float*, float*, int, float);

}  // namespace dev
}  // namespace igamg
