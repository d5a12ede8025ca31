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
#include <cooperative_groups.h>

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
// 16 bytes, both addresses 16-byte aligned, through L2 only
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

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

// ---------------------------------------------------------------- cluster tail
// The same coarse part of the 2D V-cycle on one thread-block cluster of C CTAs
// (up to 16).  One SM stops paying off once a level has more than a few
// thousand unknowns, while up to about 10^5 unknowns per level the per-level
// kernels still spend most of their time in launch latency.  Here every CTA
// owns a band of grid rows of each level (ClusterTailView) and keeps all of
// its data in shared memory; the few rows a step needs from a neighbouring
// band (the 2p rows within reach of the y-band, the rows a transfer combines)
// are read from that CTA's shared memory through distributed shared memory,
// and cluster barriers separate the dependent steps.  The arithmetic is that
// of the one-CTA tail: the same colours in the same order, the same transfer
// operators and fast diagonalisation; the off-row part of a row is summed
// once per row phase.
//
// Which CTA holds a row is fixed for the launch, so every row a CTA reads is
// resolved once, before the wait on the previous kernel, into a table of
// generic pointers (its own shared memory or a neighbour's): the inner loops
// do no row-owner arithmetic.  (Measured on GB300: reading the neighbours'
// rows where they are is faster than having their owners push copies into
// halo rows, 144 against 154 us per V-cycle tail at 1024^2, p = 3.)
namespace cg = cooperative_groups;

// Level q as CTA `rank` sees it.
template <typename T>
struct CLevel {
    int mx, my, R, lo, hi, tlo, thi, nbc;
    T* x;            // own rows, zero-padded: row lr at lr (mx + 2p), column i at + i + p
    T* b;            // own rows, mx each
    const T* inv;    // 1 / A_qq of the own rows
    T* TM;           // T_M of the own rows, then T_K (at + R mx)
    T* TK;
    const T* yM;     // M_y(j, j + bb - p) of own row lr at yM[bb R + lr]
    const T* yK;
    const T* xM;     // M_x(i, i + bb - p) at xM[s W + bb]: slots 0..nbc-1 the boundary columns, slot nbc the interior
    const T* xK;
    const T* const* rp;   // T_M row of grid row j + bb - p for own row lr at rp[lr W + bb]
};

// Transfer X[q] (levels q - 1, q): x-axis tables in full; for the own coarse
// rows of level q - 1 the fine rows their restriction combines (pointers to
// the t rows, a zero row outside the grid) and weights, for the own fine rows
// the coarse rows their prolongation combines and weights.
template <typename T>
struct CTransfer {
    int pwx, rwx, pwy, rwy;
    const int* plox;
    const T* pvx;
    const int* rlox;
    const T* rvx;
    const T* pvy;            // own fine rows x pw_y
    const T* rvy;            // own coarse rows x rw_y
    const int* ploy;         // own fine rows: first coarse row of the prolongation
    const int* rloy;         // own coarse rows: first fine row of the restriction
    const T* const* rr;      // own coarse rows x rw_y
    const T* const* pr;      // own fine rows x pw_y
};

template <typename T, int P>
__device__ __forceinline__ CLevel<T> clevel(const ClusterTailView<T>& V, unsigned char* raw, int q, int rank) {
    constexpr int W = 2 * P + 1;
    T* sm = reinterpret_cast<T*>(raw);
    CLevel<T> S;
    S.mx = V.L[q].m[0];
    S.my = V.L[q].m[1];
    S.R = V.R[q];
    S.lo = min(rank * S.R, S.my);
    S.hi = min(S.lo + S.R, S.my);
    S.tlo = V.L[q].tlo[0];
    S.thi = V.L[q].thi[0];
    S.nbc = V.nbc[q];
    S.x = sm + V.off_x[q];
    S.b = sm + V.off_b[q];
    S.inv = sm + V.off_inv[q];
    S.TM = sm + V.off_tm[q];
    S.TK = S.TM + S.R * S.mx;
    S.yM = sm + V.off_yb[q];
    S.yK = S.yM + W * S.R;
    S.xM = sm + V.off_xb[q];
    S.xK = S.xM + (S.nbc + 1) * W;
    S.rp = reinterpret_cast<const T* const*>(raw + (size_t)V.off_rp[q] * sizeof(T));
    return S;
}

template <typename T>
__device__ __forceinline__ CTransfer<T> ctransfer(const ClusterTailView<T>& V, unsigned char* raw, int q) {
    const TransferView<T>& X = V.X[q];
    T* sm = reinterpret_cast<T*>(raw);
    CTransfer<T> Y;
    Y.pwx = X.pw[0];
    Y.rwx = X.rw[0];
    Y.pwy = X.pw[1];
    Y.rwy = X.rw[1];
    T* f = sm + V.off_tx[q];
    Y.plox = reinterpret_cast<const int*>(f);
    f += X.mf[0];
    Y.pvx = f;
    f += X.mf[0] * X.pw[0];
    Y.rlox = reinterpret_cast<const int*>(f);
    f += X.mc[0];
    Y.rvx = f;
    const int Rf = V.R[q], Rc = V.R[q - 1];
    T* g = sm + V.off_ty[q];
    Y.pvy = g;
    Y.rvy = g + Rf * X.pw[1];
    Y.ploy = reinterpret_cast<const int*>(Y.rvy + Rc * X.rw[1]);
    Y.rloy = Y.ploy + Rf;
    const T* const* rpq = reinterpret_cast<const T* const*>(raw + (size_t)V.off_rp[q] * sizeof(T));
    Y.rr = rpq + Rf * (2 * V.L[q].p + 1);
    Y.pr = Y.rr + Rc * X.rw[1];
    return Y;
}

// f(k, i) for every (k, i) in [0, n) x [0, m), the CTA's threads striding
// over k m + i without a division per element.
template <typename F>
__device__ __forceinline__ void grid_for(int n, int m, F&& f) {
    const int NT = blockDim.x, dk = NT / m, di = NT - dk * m;
    int k = (int)threadIdx.x / m, i = (int)threadIdx.x - k * m;
    while (k < n) {
        f(k, i);
        i += di;
        k += dk;
        if (i >= m) {
            i -= m;
            ++k;
        }
    }
}

// sum_b M_x(i, b) x(i + b - p) and the K_x sum of an own row (xr: padded
// column i - p).  The band comes from the slot of column i (the interior
// slot in the uniform interior), without a branch: lanes of one warp take
// boundary and interior columns in the same pass.
template <typename T, int P, typename LV>
__device__ __forceinline__ void cwin(const LV& S, const T* xr, int i, T& sM, T& sK) {
    constexpr int W = 2 * P + 1;
    const int slot = i < S.tlo ? i : (i < S.thi ? S.nbc : S.tlo + (i - S.thi));
    const T* cm = S.xM + slot * W;
    const T* ck = S.xK + slot * W;
    sM = 0;
    sK = 0;
#pragma unroll
    for (int bb = 0; bb < W; ++bb) {
        const T v = xr[bb];
        sM += cm[bb] * v;
        sK += ck[bb] * v;
    }
}

// sum over the y-band rows bj (all, or all but the own row) of
// K_y(j, bj) T_M(j + bj - p, i) + M_y(j, bj) T_K(j + bj - p, i) for own row
// lr; band entries outside the matrix are zero (their pointer is the own row).
template <typename T, int P, bool SKIP_OWN>
__device__ __forceinline__ T ccouple(const CLevel<T>& S, int lr, int i) {
    constexpr int W = 2 * P + 1;
    const T* const* rp = S.rp + lr * W;
    const int tko = S.R * S.mx;
    T acc = 0;
#pragma unroll
    for (int bj = 0; bj < W; ++bj) {
        if (SKIP_OWN && bj == P) continue;
        const T* row = rp[bj];
        acc += S.yK[bj * S.R + lr] * row[i] + S.yM[bj * S.R + lr] * row[tko + i];
    }
    return acc;
}

// T_M, T_K of the own rows from x (local only).
template <typename T, int P>
__device__ void cxpass(const CLevel<T>& S) {
    const int PW = S.mx + 2 * P;
    grid_for(S.hi - S.lo, S.mx, [&](int lr, int i) {
        T sM, sK;
        cwin<T, P>(S, S.x + lr * PW + i, i, sM, sK);
        S.TM[lr * S.mx + i] = sM;
        S.TK[lr * S.mx + i] = sK;
    });
}

// Barrier of row group g (G warps: warps g G .. g G + G - 1); named barrier
// 1 + g, one warp: a warp barrier.
__device__ __forceinline__ void group_sync(int g, int G) {
    if (G == 1) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(32 * G) : "memory");
}

// One multicolour GS sweep.  Row phase cy: the own rows j = cy mod (p+1)
// (no two of them couple, across the cluster too) are shared out to groups
// of warps; a group takes its row's frozen off-row part once, runs the row's
// p+1 x-colours and refreshes its T_M, T_K with group barriers only.  A
// cluster barrier then publishes the phase's rows to the next phase.
template <typename T, int P>
__device__ void cgs(const CLevel<T>& S, T* rhs, bool descending) {
    constexpr int P1 = P + 1;
    const int own = S.hi - S.lo, PW = S.mx + 2 * P;
    const int NW = (int)blockDim.x >> 5, warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    const int want = (S.mx + 31) >> 5;                          // warps a row keeps busy
    for (int pc = 0; pc < P1; ++pc) {
        const int cy = descending ? P - pc : pc;
        const int lr0 = ((cy - S.lo) % P1 + P1) % P1;          // first own row of the phase
        const int nr = lr0 < own ? (own - 1 - lr0) / P1 + 1 : 0;
        if (nr > 0) {
            const int G = max(1, min(NW / nr, want)), ng = min(NW / G, 15);
            const int g = warp / G, gl = (warp - g * G) * 32 + lane, gt = 32 * G;
            if (g < ng)
                for (int k = g; k < nr; k += ng) {
                    const int lr = lr0 + k * P1;
                    T* rr = rhs + k * S.mx;
                    for (int i = gl; i < S.mx; i += gt) rr[i] = S.b[lr * S.mx + i] - ccouple<T, P, true>(S, lr, i);
                    group_sync(g, G);
                    const T ky = S.yK[P * S.R + lr], my = S.yM[P * S.R + lr];
                    T* xrow = S.x + lr * PW;
                    const T* inv = S.inv + lr * S.mx;
                    for (int c = 0; c < P1; ++c) {
                        const int cx = descending ? P - c : c;
                        const int nx = (S.mx - cx + P) / P1;
                        for (int sx = gl; sx < nx; sx += gt) {
                            const int i = cx + P1 * sx;
                            T sM, sK;
                            cwin<T, P>(S, xrow + i, i, sM, sK);            // padded column i - p
                            xrow[i + P] += (rr[i] - (ky * sM + my * sK)) * inv[i];
                        }
                        group_sync(g, G);
                    }
                    for (int i = gl; i < S.mx; i += gt) {
                        T sM, sK;
                        cwin<T, P>(S, xrow + i, i, sM, sK);
                        S.TM[lr * S.mx + i] = sM;
                        S.TK[lr * S.mx + i] = sK;
                    }
                }
        }
        cg::this_cluster().sync();
    }
}

// One weighted-Jacobi sweep x += omega D^{-1} (b - A x) from the same x on
// every node; the own T rows change only after every CTA has read them.
template <typename T, int P>
__device__ void cjacobi(const CLevel<T>& S, T* d, T omega) {
    const int own = S.hi - S.lo, PW = S.mx + 2 * P;
    grid_for(own, S.mx, [&](int lr, int i) {
        const int q = lr * S.mx + i;
        d[q] = omega * (S.b[q] - ccouple<T, P, false>(S, lr, i)) * S.inv[q];
    });
    cg::this_cluster().sync();
    grid_for(own, S.mx, [&](int lr, int i) { S.x[lr * PW + i + P] += d[lr * S.mx + i]; });
    __syncthreads();
    cxpass<T, P>(S);
    cg::this_cluster().sync();
}

// b_c = P^T (b - A x): the own rows' residual and x-axis restriction (t),
// then the own coarse rows from the fine rows' t across the cluster.
template <typename T, int P>
__device__ void crestrict(const CLevel<T>& S, const CLevel<T>& Sc, const CTransfer<T>& X, T* r, T* t) {
    const int own = S.hi - S.lo, mcx = Sc.mx;
    grid_for(own, S.mx, [&](int lr, int i) {
        const int q = lr * S.mx + i;
        r[q] = S.b[q] - ccouple<T, P, false>(S, lr, i);
    });
    __syncthreads();
    grid_for(own, mcx, [&](int lr, int I) {
        const int lo = X.rlox[I];
        T acc = 0;
        for (int s = 0; s < X.rwx; ++s) {
            const int f = lo + s;
            if (f < 0 || f >= S.mx) continue;
            acc += X.rvx[I * X.rwx + s] * r[lr * S.mx + f];
        }
        t[lr * mcx + I] = acc;
    });
    cg::this_cluster().sync();
    grid_for(Sc.hi - Sc.lo, mcx, [&](int Jl, int I) {
        const T* const* rows = X.rr + Jl * X.rwy;
        T acc = 0;
        for (int s = 0; s < X.rwy; ++s) acc += X.rvy[Jl * X.rwy + s] * rows[s][I];
        Sc.b[Jl * mcx + I] = acc;
    });
    __syncthreads();
}

// x += P e: the own coarse rows' x-axis prolongation (t), then the own fine
// rows from the coarse rows' t across the cluster, and the new T_M, T_K.
template <typename T, int P>
__device__ void cprolong(const CLevel<T>& S, const CLevel<T>& Sc, const CTransfer<T>& X, T* t) {
    const int mfx = S.mx, PWc = Sc.mx + 2 * P;
    grid_for(Sc.hi - Sc.lo, mfx, [&](int Jl, int i) {
        const int lo = X.plox[i];
        T acc = 0;
        for (int s = 0; s < X.pwx; ++s) {
            const int f = lo + s;
            if (f < 0 || f >= Sc.mx) continue;
            acc += X.pvx[i * X.pwx + s] * Sc.x[Jl * PWc + f + P];
        }
        t[Jl * mfx + i] = acc;
    });
    cg::this_cluster().sync();
    const int PW = S.mx + 2 * P;
    grid_for(S.hi - S.lo, mfx, [&](int jl, int i) {
        const T* const* rows = X.pr + jl * X.pwy;
        T acc = 0;
        for (int s = 0; s < X.pwy; ++s) acc += X.pvy[jl * X.pwy + s] * rows[s][i];
        S.x[jl * PW + i + P] += acc;
    });
    __syncthreads();
    cxpass<T, P>(S);
    cg::this_cluster().sync();
}

// Generic pointer to `local`'s counterpart in CTA o's shared memory.
template <typename T>
__device__ __forceinline__ const T* cptr(T* local, int o, int rank) {
    return o == rank ? local : cg::this_cluster().map_shared_rank(local, o);
}

constexpr int kCTailThreads = 512;

// Every CTA's static shared memory, built once per context (cluster_tail_image):
// the operator data, transfer tables and coarsest eigenbasis staged as the
// tail uses them, the zero row, and each neighbour-row pointer as its
// (owner CTA, element offset) pair, copied out to img[rank * img16 ..].
template <typename T, int P>
__global__ void __launch_bounds__(kCTailThreads, 1) k_cluster_tail_image(ClusterTailView<T> V, uint4* img) {
    static_assert(sizeof(T) == 4, "4-byte elements (staging, integer tables)");
    constexpr int W = 2 * P + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int rank = (int)cg::this_cluster().block_rank();
    const int lc = V.lc;
    T* t = sm + V.off_t;
    T* zrow = sm + V.off_z;
    uint4* s16 = reinterpret_cast<uint4*>(smem_raw);
    for (int e = threadIdx.x; e < V.img16; e += blockDim.x) s16[e] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    auto pair_of = [&](const T* p, int o) { return make_int2(o, (int)(p - sm)); };
    for (int q = 1; q <= lc; ++q) {
        const LevelView<T>& L = V.L[q];
        const CLevel<T> S = clevel<T, P>(V, smem_raw, q, rank);
        const int own = S.hi - S.lo;
        stage(const_cast<T*>(S.inv), L.invdiag + (size_t)S.lo * S.mx, own * S.mx);
        for (int e = threadIdx.x; e < W * own; e += blockDim.x) {
            const int bb = e / own, jl = e - bb * own;
            cp_async4(const_cast<T*>(S.yM) + bb * S.R + jl, L.Mb[1] + bb * S.my + S.lo + jl);
            cp_async4(const_cast<T*>(S.yK) + bb * S.R + jl, L.Kb[1] + bb * S.my + S.lo + jl);
        }
        for (int e = threadIdx.x; e < S.nbc * W; e += blockDim.x) {
            const int sl = e / W, bb = e - sl * W;
            const int i = sl < S.tlo ? sl : S.thi + (sl - S.tlo);
            cp_async4(const_cast<T*>(S.xM) + e, L.Mb[0] + bb * S.mx + i);
            cp_async4(const_cast<T*>(S.xK) + e, L.Kb[0] + bb * S.mx + i);
        }
        for (int bb = threadIdx.x; bb < W; bb += blockDim.x) {      // the interior slot
            const_cast<T*>(S.xM)[S.nbc * W + bb] = L.Mc[0][bb];
            const_cast<T*>(S.xK)[S.nbc * W + bb] = L.Kc[0][bb];
        }
        const TransferView<T>& X = V.X[q];
        const CTransfer<T> Y = ctransfer(V, smem_raw, q);
        stage(const_cast<int*>(Y.plox), X.plo[0], X.mf[0]);
        stage(const_cast<T*>(Y.pvx), X.pv[0], X.mf[0] * X.pw[0]);
        stage(const_cast<int*>(Y.rlox), X.rlo[0], X.mc[0]);
        stage(const_cast<T*>(Y.rvx), X.rv[0], X.mc[0] * X.rw[0]);
        const int Rc = V.R[q - 1], myc = V.L[q - 1].m[1];
        const int loc = min(rank * Rc, myc), ownc = min(loc + Rc, myc) - loc;
        stage(const_cast<T*>(Y.pvy), X.pv[1] + (size_t)S.lo * X.pw[1], own * X.pw[1]);
        stage(const_cast<T*>(Y.rvy), X.rv[1] + (size_t)loc * X.rw[1], ownc * X.rw[1]);
        stage(const_cast<int*>(Y.ploy), X.plo[1] + S.lo, own);
        stage(const_cast<int*>(Y.rloy), X.rlo[1] + loc, ownc);
        // y-band neighbours of the own rows
        int2* rp = reinterpret_cast<int2*>(const_cast<T**>(S.rp));
        for (int e = threadIdx.x; e < own * W; e += blockDim.x) {
            const int lr = e / W, bb = e - lr * W, jj = S.lo + lr + bb - P;
            if (jj < 0 || jj >= S.my) {
                rp[e] = pair_of(S.TM + lr * S.mx, rank);    // zero band entry
            } else {
                const int o = jj / S.R;
                rp[e] = pair_of(S.TM + (jj - o * S.R) * S.mx, o);
            }
        }
    }
    if (rank == 0) {                                    // coarsest eigenbasis
        T* f = sm + V.off_cv;
        const int m0 = V.C.m[0], m1 = V.C.m[1];
        stage(f, V.C.V[0], m0 * m0);
        stage(f + m0 * m0, V.C.V[1], m1 * m1);
        stage(f + m0 * m0 + m1 * m1, V.C.laminv, m0 * m1);
    }
    cp_async_wait_all();
    __syncthreads();
    for (int q = 1; q <= lc; ++q) {                     // the t rows the y-axis transfer passes combine
        const CLevel<T> S = clevel<T, P>(V, smem_raw, q, rank);
        const TransferView<T>& X = V.X[q];
        const CTransfer<T> Y = ctransfer(V, smem_raw, q);
        const int Rc = V.R[q - 1], myc = V.L[q - 1].m[1];
        const int loc = min(rank * Rc, myc), ownc = min(loc + Rc, myc) - loc, own = S.hi - S.lo;
        int2* rr = reinterpret_cast<int2*>(const_cast<T**>(Y.rr));
        for (int e = threadIdx.x; e < ownc * X.rw[1]; e += blockDim.x) {
            const int Jl = e / X.rw[1], s2 = e - Jl * X.rw[1], f = Y.rloy[Jl] + s2;
            if (f < 0 || f >= S.my) {
                rr[e] = pair_of(zrow, rank);
            } else {
                const int o = f / S.R;
                rr[e] = pair_of(t + (f - o * S.R) * X.mc[0], o);
            }
        }
        int2* pr = reinterpret_cast<int2*>(const_cast<T**>(Y.pr));
        for (int e = threadIdx.x; e < own * X.pw[1]; e += blockDim.x) {
            const int jl = e / X.pw[1], s2 = e - jl * X.pw[1], F = Y.ploy[jl] + s2;
            if (F < 0 || F >= myc) {
                pr[e] = pair_of(zrow, rank);
            } else {
                const int o = F / Rc;
                pr[e] = pair_of(t + (F - o * Rc) * X.mf[0], o);
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < V.img16; e += blockDim.x) img[(size_t)rank * V.img16 + e] = s16[e];
}

template <typename T, int P>
__global__ void __launch_bounds__(kCTailThreads, 1) k_cluster_tail(ClusterTailView<T> V, const T* __restrict__ b_in,
                                                                  T* __restrict__ x_out, int jacobi, T omega) {
    static_assert(sizeof(T) == 4, "4-byte elements (staging, integer tables)");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int rank = (int)cg::this_cluster().block_rank();
    const int lc = V.lc;
    T* r = sm + V.off_r;
    T* t = sm + V.off_t;
    // this CTA's static shared memory from its image (operator data only,
    // before the wait on the previous kernel), the dynamic part zeroed, the
    // right side b after the wait; then the neighbour-row pairs become pointers
    {
        const uint4* src = V.img + (size_t)rank * V.img16;
        uint4* dst = reinterpret_cast<uint4*>(smem_raw);
        for (int e = threadIdx.x; e < V.img16; e += blockDim.x) cp_async16(dst + e, src + e);
    }
    CoarseView<T> Cs = V.C;                             // coarsest eigenbasis (CTA 0 only)
    {
        T* f = sm + V.off_cv;
        const int m0 = V.C.m[0], m1 = V.C.m[1];
        Cs.V[0] = f;
        Cs.V[1] = f + m0 * m0;
        Cs.laminv = f + m0 * m0 + m1 * m1;
    }
    for (int q = 0; q <= lc; ++q) {                     // coarse e^0 = 0 on every level, zero pads
        const CLevel<T> S = clevel<T, P>(V, smem_raw, q, rank);
        for (int e = threadIdx.x; e < S.R * (S.mx + 2 * P); e += blockDim.x) S.x[e] = 0;
        if (q > 0)
            for (int e = threadIdx.x; e < 2 * S.R * S.mx; e += blockDim.x) S.TM[e] = 0;
    }
    pdl_enter();
    {
        const CLevel<T> S = clevel<T, P>(V, smem_raw, lc, rank);
        stage(S.b, b_in + (size_t)S.lo * S.mx, (S.hi - S.lo) * S.mx);
    }
    cp_async_wait_all();
    __syncthreads();
    {
        const int2* pairs = reinterpret_cast<const int2*>(smem_raw);
        const T** ptrs = reinterpret_cast<const T**>(smem_raw);
        for (int e = threadIdx.x; e < V.npair; e += blockDim.x) {
            const int2 pq = pairs[e];
            ptrs[e] = cptr(sm + pq.y, pq.x, rank);
        }
    }
    __syncthreads();
    cg::this_cluster().sync();                          // every CTA's zero T rows in place
    for (int l = lc; l >= 1; --l) {
        const CLevel<T> S = clevel<T, P>(V, smem_raw, l, rank);
        if (jacobi) cjacobi<T, P>(S, r, omega);                                // pre-smooth
        else cgs<T, P>(S, r, false);
        crestrict<T, P>(S, clevel<T, P>(V, smem_raw, l - 1, rank), ctransfer(V, smem_raw, l), r, t);
    }
    if (rank == 0) {                                    // direct solve, into the padded rows of x_0
        const int m0 = Cs.m[0], m1 = Cs.m[1], N = m0 * m1;
        const T* b0 = sm + V.off_b[0];
        T* x0 = sm + V.off_x[0];
        auto pass = [&](const T* in, T* out, int axis, bool transpose, bool pad) {
            const int md = Cs.m[axis], stride = axis == 0 ? 1 : m0;
            const T* Vm = Cs.V[axis];
            for (int idx = threadIdx.x; idx < N; idx += blockDim.x) {
                const int I = axis == 0 ? idx % m0 : idx / m0;
                const int base = idx - I * stride;
                T acc = 0;
                for (int s = 0; s < md; ++s) acc += (transpose ? Vm[s * md + I] : Vm[I * md + s]) * in[base + s * stride];
                out[pad ? (idx / m0) * (m0 + 2 * P) + idx % m0 + P : idx] = acc;
            }
            __syncthreads();
        };
        pass(b0, r, 0, true, false);
        pass(r, t, 1, true, false);
        for (int i = threadIdx.x; i < N; i += blockDim.x) t[i] *= Cs.laminv[i];
        __syncthreads();
        pass(t, r, 1, false, false);
        pass(r, x0, 0, false, true);
    }
    cg::this_cluster().sync();
    for (int l = 1; l <= lc; ++l) {
        const CLevel<T> S = clevel<T, P>(V, smem_raw, l, rank);
        cprolong<T, P>(S, clevel<T, P>(V, smem_raw, l - 1, rank), ctransfer(V, smem_raw, l), t);   // x += P e
        if (jacobi) cjacobi<T, P>(S, r, omega);                                // post-smooth
        else cgs<T, P>(S, r, true);
    }
    const CLevel<T> S = clevel<T, P>(V, smem_raw, lc, rank);
    const int PW = S.mx + 2 * P;
    grid_for(S.hi - S.lo, S.mx, [&](int lr, int i) { x_out[(size_t)(S.lo + lr) * S.mx + i] = S.x[lr * PW + i + P]; });
}

// ---------------------------------------------------------------- 3D cluster tail
// The coarse part of the 3D V-cycle on one thread-block cluster, in the form
// of the 2D cluster tail above: every CTA owns a range of grid rows (j, k)
// (numbered r = k m_y + j) of each level in its shared memory, and cluster
// barriers order the steps.  Unlike 2D, most of a row's (2p+1)^2 neighbour
// rows belong to other CTAs, so every CTA keeps halo copies of T_M, T_K for
// the rows within reach of its range (H = p m_y + p rows on each side, a
// contiguous range in row order), and the owner of a row writes its new
// T_M, T_K into every halo that holds it (distributed shared memory stores)
// when it refreshes them; the smoothing steps and the residual read only
// local memory.  (Reading the neighbours' rows in place made the 3D tail
// bound by distributed-shared-memory bandwidth.)  The transfers read the
// neighbours' rows of their scratch through pointers resolved once per launch.
// A row couples to the (2p+1)^2 rows (j + dj, k + dk) with the weights
// K_z M_y + M_z K_y on T_M and M_z M_y on T_K (A = K_z (x) M_y (x) M_x +
// M_z (x) K_y (x) M_x + M_z (x) M_y (x) K_x); they are formed once per launch
// from the staged y- and z-bands.  GS runs the (p+1)^2 row phases of the
// per-level kernels, the row's x-colours inside a phase, and the restriction
// and prolongation apply the x axis to a CTA's own rows and the y and z axes
// together across the cluster.

template <typename T>
struct CLevel3 {
    int mx, my, mz, R, lo, hi, tlo, thi, nbc;
    T* x;            // own rows, zero-padded: row lr at lr (mx + 2p), column i at + i + p
    T* b;
    const T* inv;
    int H;           // halo rows on each side
    T* TM;           // rows lo - H .. hi + H - 1 (own row lr at (lr + H) mx), then T_K at + (R + 2H) mx
    T* TK;
    const T* xM;     // boundary slots 0..nbc-1, interior slot nbc
    const T* xK;
    const T* cc;     // own row lr, neighbour q = (dk + p) W + dj + p: weights at cc[2 (lr W^2 + q)], + 1
};

template <typename T, int P>
__device__ __forceinline__ CLevel3<T> clevel3(const ClusterTail3View<T>& V, unsigned char* raw, int q, int rank) {
    constexpr int W = 2 * P + 1;
    T* sm = reinterpret_cast<T*>(raw);
    CLevel3<T> S;
    S.mx = V.L[q].m[0];
    S.my = V.L[q].m[1];
    S.mz = V.L[q].m[2];
    S.R = V.R[q];
    const int rows = S.my * S.mz;
    S.lo = min(rank * S.R, rows);
    S.hi = min(S.lo + S.R, rows);
    S.tlo = V.L[q].tlo[0];
    S.thi = V.L[q].thi[0];
    S.nbc = V.nbc[q];
    S.x = sm + V.off_x[q];
    S.b = sm + V.off_b[q];
    S.inv = sm + V.off_inv[q];
    S.H = P * S.my + P;
    S.TM = sm + V.off_tm[q];
    S.TK = S.TM + (S.R + 2 * S.H) * S.mx;
    S.xM = sm + V.off_xb[q];
    S.xK = S.xM + (S.nbc + 1) * W;
    S.cc = sm + V.off_cc[q];
    return S;
}

// Transfer X[q] in 3D: staged tables of the three axes (plo, pv, rlo, rv),
// and the pointer tables of the y-z passes (after the neighbour pointers of
// level q in the off_rp region).
template <typename T>
struct CTransfer3 {
    int pw[3], rw[3];
    const int* plo[3];
    const T* pv[3];
    const int* rlo[3];
    const T* rv[3];
    const T* const* rr;      // own coarse rows x (rw_y rw_z): fine t rows, (s_z, s_y) with s_y fastest
    const T* const* pr;      // own fine rows x (pw_y pw_z): coarse t rows
};

template <typename T>
__device__ __forceinline__ CTransfer3<T> ctransfer3(const ClusterTail3View<T>& V, unsigned char* raw, int q) {
    const TransferView<T>& X = V.X[q];
    T* f = reinterpret_cast<T*>(raw) + V.off_tx[q];
    CTransfer3<T> Y;
    for (int d = 0; d < 3; ++d) {
        Y.pw[d] = X.pw[d];
        Y.rw[d] = X.rw[d];
        Y.plo[d] = reinterpret_cast<const int*>(f);
        f += X.mf[d];
        Y.pv[d] = f;
        f += X.mf[d] * X.pw[d];
        Y.rlo[d] = reinterpret_cast<const int*>(f);
        f += X.mc[d];
        Y.rv[d] = f;
        f += X.mc[d] * X.rw[d];
    }
    Y.rr = reinterpret_cast<const T* const*>(raw + (size_t)V.off_rp[q] * sizeof(T));
    Y.pr = Y.rr + V.R[q - 1] * X.rw[1] * X.rw[2];
    return Y;
}

// Own rows [lo, hi) with j = cy and k = cz (mod p+1): with idx < 0 their
// number, else the local index of the idx-th of them (in row order).
template <int P>
__device__ __forceinline__ int phase_rows3(int lo, int hi, int my, int cy, int cz, int idx) {
    constexpr int P1 = P + 1;
    int cnt = 0;
    if (lo >= hi) return idx < 0 ? 0 : -1;
    const int k0 = lo / my, k1 = (hi - 1) / my;
    for (int k = k0; k <= k1; ++k) {
        if (k % P1 != cz) continue;
        const int jlo = k == k0 ? lo - k * my : 0, jhi = k == k1 ? hi - k * my : my;
        const int j0 = jlo + ((cy - jlo) % P1 + P1) % P1;
        const int n = j0 < jhi ? (jhi - 1 - j0) / P1 + 1 : 0;
        if (idx >= 0 && idx < cnt + n) return k * my + j0 + (idx - cnt) * P1 - lo;
        cnt += n;
    }
    return idx < 0 ? cnt : -1;
}

// sum over the (2p+1)^2 neighbour rows (all, or all but the own row) of
// cM T_M + cK T_K at column i of own row lr, from the own and halo rows (a
// neighbour outside the grid has zero weights; its slot holds another row's
// finite values or zeros).
template <typename T, int P, bool SKIP_OWN>
__device__ __forceinline__ T ccouple3(const CLevel3<T>& S, int lr, int i) {
    constexpr int W = 2 * P + 1, W2 = W * W, OWN = P * W + P;
    const T* cc = S.cc + 2 * lr * W2;
    const T* tm = S.TM + (lr + S.H) * S.mx + i;         // the own row's slot
    const int tko = (S.R + 2 * S.H) * S.mx;
    T acc = 0;
    constexpr int U = W2 > 49 ? 9 : W2;
#pragma unroll U
    for (int q = 0; q < W2; ++q) {
        if (SKIP_OWN && q == OWN) continue;
        const int dr = (q / W - P) * S.my + (q % W - P);
        const T* row = tm + dr * S.mx;
        acc += cc[2 * q] * row[0] + cc[2 * q + 1] * row[tko];
    }
    return acc;
}

// T_M, T_K of own row lr at column i: stored in the own slot and written into
// the halo of every other CTA whose range of rows within reach holds it.
template <typename T, int P>
__device__ __forceinline__ void store_t3(const CLevel3<T>& S, int lr, int i, T sM, T sK, int rank, int C) {
    const int tko = (S.R + 2 * S.H) * S.mx;
    T* own = S.TM + (lr + S.H) * S.mx + i;
    own[0] = sM;
    own[tko] = sK;
    const int r = S.lo + lr, rows = S.my * S.mz;
    const int o0 = max(0, (r - S.H) / S.R - 1), o1 = min(C - 1, (r + S.H) / S.R + 1);
    for (int o = o0; o <= o1; ++o) {
        const int lo_o = o * S.R;
        if (o == rank || lo_o >= rows) continue;
        const int hi_o = min(lo_o + S.R, rows);
        if (r < lo_o - S.H || r >= hi_o + S.H) continue;
        T* dst = cg::this_cluster().map_shared_rank(S.TM + (r - lo_o + S.H) * S.mx + i, o);
        dst[0] = sM;
        dst[tko] = sK;
    }
}

template <typename T, int P>
__device__ void cxpass3(const CLevel3<T>& S, int rank, int C) {
    const int PW = S.mx + 2 * P;
    grid_for(S.hi - S.lo, S.mx, [&](int lr, int i) {
        T sM, sK;
        cwin<T, P>(S, S.x + lr * PW + i, i, sM, sK);
        store_t3<T, P>(S, lr, i, sM, sK, rank, C);
    });
}

// One multicolour GS sweep: (p+1)^2 row phases (cz slowest), each over the
// own rows of the phase shared out to groups of warps, then a cluster barrier.
template <typename T, int P>
__device__ void cgs3(const CLevel3<T>& S, T* rhs, bool descending, int rank, int C) {
    constexpr int P1 = P + 1, NPH = P1 * P1, W2 = (2 * P + 1) * (2 * P + 1), OWN = P * (2 * P + 1) + P;
    const int PW = S.mx + 2 * P;
    const int NW = (int)blockDim.x >> 5, warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    const int want = (S.mx + 31) >> 5;
    for (int ph = 0; ph < NPH; ++ph) {
        const int c = descending ? NPH - 1 - ph : ph;
        const int cy = c % P1, cz = c / P1;
        const int nr = phase_rows3<P>(S.lo, S.hi, S.my, cy, cz, -1);
        if (nr > 0) {
            const int G = max(1, min(NW / nr, want)), ng = min(NW / G, 15);
            const int g = warp / G, gl = (warp - g * G) * 32 + lane, gt = 32 * G;
            if (g < ng)
                for (int k = g; k < nr; k += ng) {
                    const int lr = phase_rows3<P>(S.lo, S.hi, S.my, cy, cz, k);
                    T* rr = rhs + k * S.mx;
                    for (int i = gl; i < S.mx; i += gt) rr[i] = S.b[lr * S.mx + i] - ccouple3<T, P, true>(S, lr, i);
                    group_sync(g, G);
                    const T cm = S.cc[2 * (lr * W2 + OWN)], ck = S.cc[2 * (lr * W2 + OWN) + 1];
                    T* xrow = S.x + lr * PW;
                    const T* inv = S.inv + lr * S.mx;
                    for (int cx_ = 0; cx_ < P1; ++cx_) {
                        const int cx = descending ? P - cx_ : cx_;
                        const int nx = (S.mx - cx + P) / P1;
                        for (int sx = gl; sx < nx; sx += gt) {
                            const int i = cx + P1 * sx;
                            T sM, sK;
                            cwin<T, P>(S, xrow + i, i, sM, sK);
                            xrow[i + P] += (rr[i] - (cm * sM + ck * sK)) * inv[i];
                        }
                        group_sync(g, G);
                    }
                    for (int i = gl; i < S.mx; i += gt) {
                        T sM, sK;
                        cwin<T, P>(S, xrow + i, i, sM, sK);
                        store_t3<T, P>(S, lr, i, sM, sK, rank, C);
                    }
                }
        }
        cg::this_cluster().sync();
    }
}

template <typename T, int P>
__device__ void cjacobi3(const CLevel3<T>& S, T* d, T omega, int rank, int C) {
    const int own = S.hi - S.lo, PW = S.mx + 2 * P;
    grid_for(own, S.mx, [&](int lr, int i) {
        const int q = lr * S.mx + i;
        d[q] = omega * (S.b[q] - ccouple3<T, P, false>(S, lr, i)) * S.inv[q];
    });
    cg::this_cluster().sync();
    grid_for(own, S.mx, [&](int lr, int i) { S.x[lr * PW + i + P] += d[lr * S.mx + i]; });
    __syncthreads();
    cxpass3<T, P>(S, rank, C);
    cg::this_cluster().sync();
}

// b_c = P^T (b - A x): residual and x-axis restriction of the own rows (t),
// then the own coarse rows from the fine rows' t (y and z axes together).
template <typename T, int P>
__device__ void crestrict3(const CLevel3<T>& S, const CLevel3<T>& Sc, const CTransfer3<T>& X, T* r, T* t) {
    const int own = S.hi - S.lo, mcx = Sc.mx;
    grid_for(own, S.mx, [&](int lr, int i) {
        const int q = lr * S.mx + i;
        r[q] = S.b[q] - ccouple3<T, P, false>(S, lr, i);
    });
    __syncthreads();
    grid_for(own, mcx, [&](int lr, int I) {
        const int lo = X.rlo[0][I];
        T acc = 0;
        for (int s = 0; s < X.rw[0]; ++s) {
            const int f = lo + s;
            if (f < 0 || f >= S.mx) continue;
            acc += X.rv[0][I * X.rw[0] + s] * r[lr * S.mx + f];
        }
        t[lr * mcx + I] = acc;
    });
    cg::this_cluster().sync();
    const int ryz = X.rw[1] * X.rw[2];
    grid_for(Sc.hi - Sc.lo, mcx, [&](int Jl, int I) {
        const int rc = Sc.lo + Jl, J = rc % Sc.my, K = rc / Sc.my;
        const T* const* rows = X.rr + Jl * ryz;
        T acc = 0;
        for (int sz = 0; sz < X.rw[2]; ++sz) {
            const T wz = X.rv[2][K * X.rw[2] + sz];
            T a2 = 0;
            for (int sy = 0; sy < X.rw[1]; ++sy) a2 += X.rv[1][J * X.rw[1] + sy] * rows[sz * X.rw[1] + sy][I];
            acc += wz * a2;
        }
        Sc.b[Jl * mcx + I] = acc;
    });
    __syncthreads();
}

// x += P e: x-axis prolongation of the own coarse rows (t), then the own fine
// rows from the coarse rows' t (y and z axes together), and the new T_M, T_K.
template <typename T, int P>
__device__ void cprolong3(const CLevel3<T>& S, const CLevel3<T>& Sc, const CTransfer3<T>& X, T* t, int rank, int C) {
    const int mfx = S.mx, PWc = Sc.mx + 2 * P;
    grid_for(Sc.hi - Sc.lo, mfx, [&](int Jl, int i) {
        const int lo = X.plo[0][i];
        T acc = 0;
        for (int s = 0; s < X.pw[0]; ++s) {
            const int f = lo + s;
            if (f < 0 || f >= Sc.mx) continue;
            acc += X.pv[0][i * X.pw[0] + s] * Sc.x[Jl * PWc + f + P];
        }
        t[Jl * mfx + i] = acc;
    });
    cg::this_cluster().sync();
    const int PW = S.mx + 2 * P, pyz = X.pw[1] * X.pw[2];
    grid_for(S.hi - S.lo, mfx, [&](int jl, int i) {
        const int r = S.lo + jl, j = r % S.my, k = r / S.my;
        const T* const* rows = X.pr + jl * pyz;
        T acc = 0;
        for (int sz = 0; sz < X.pw[2]; ++sz) {
            const T wz = X.pv[2][k * X.pw[2] + sz];
            T a2 = 0;
            for (int sy = 0; sy < X.pw[1]; ++sy) a2 += X.pv[1][j * X.pw[1] + sy] * rows[sz * X.pw[1] + sy][i];
            acc += wz * a2;
        }
        S.x[jl * PW + i + P] += acc;
    });
    __syncthreads();
    cxpass3<T, P>(S, rank, C);
    cg::this_cluster().sync();
}

// Every CTA's static shared memory of the 3D tail, built once per context
// (cluster_tail3_image), as k_cluster_tail_image does in 2D; here it also
// holds the row weights cc.
template <typename T, int P>
__global__ void __launch_bounds__(kCTailThreads, 1) k_cluster_tail3_image(ClusterTail3View<T> V, uint4* img) {
    static_assert(sizeof(T) == 4, "4-byte elements (staging, integer tables)");
    constexpr int W = 2 * P + 1, W2 = W * W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int rank = (int)cg::this_cluster().block_rank();
    const int lc = V.lc;
    T* t = sm + V.off_t;
    T* zrow = sm + V.off_z;
    uint4* s16 = reinterpret_cast<uint4*>(smem_raw);
    for (int e = threadIdx.x; e < V.img16; e += blockDim.x) s16[e] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    auto pair_of = [&](const T* p, int o) { return make_int2(o, (int)(p - sm)); };
    for (int q = 1; q <= lc; ++q) {
        const LevelView<T>& L = V.L[q];
        const CLevel3<T> S = clevel3<T, P>(V, smem_raw, q, rank);
        const int own = S.hi - S.lo;
        stage(const_cast<T*>(S.inv), L.invdiag + (size_t)S.lo * S.mx, own * S.mx);
        T* yb = sm + V.off_yb[q];
        T* zb = sm + V.off_zb[q];
        stage(yb, L.Mb[1], W * S.my);
        stage(yb + W * S.my, L.Kb[1], W * S.my);
        stage(zb, L.Mb[2], W * S.mz);
        stage(zb + W * S.mz, L.Kb[2], W * S.mz);
        for (int e = threadIdx.x; e < S.nbc * W; e += blockDim.x) {
            const int sl = e / W, bb = e - sl * W;
            const int i = sl < S.tlo ? sl : S.thi + (sl - S.tlo);
            cp_async4(const_cast<T*>(S.xM) + e, L.Mb[0] + bb * S.mx + i);
            cp_async4(const_cast<T*>(S.xK) + e, L.Kb[0] + bb * S.mx + i);
        }
        for (int bb = threadIdx.x; bb < W; bb += blockDim.x) {      // the interior slot
            const_cast<T*>(S.xM)[S.nbc * W + bb] = L.Mc[0][bb];
            const_cast<T*>(S.xK)[S.nbc * W + bb] = L.Kc[0][bb];
        }
        const TransferView<T>& X = V.X[q];
        const CTransfer3<T> Y = ctransfer3(V, smem_raw, q);
        for (int d = 0; d < 3; ++d) {
            stage(const_cast<int*>(Y.plo[d]), X.plo[d], X.mf[d]);
            stage(const_cast<T*>(Y.pv[d]), X.pv[d], X.mf[d] * X.pw[d]);
            stage(const_cast<int*>(Y.rlo[d]), X.rlo[d], X.mc[d]);
            stage(const_cast<T*>(Y.rv[d]), X.rv[d], X.mc[d] * X.rw[d]);
        }
    }
    if (rank == 0) {                                    // coarsest eigenbasis
        T* f = sm + V.off_cv;
        const int m0 = V.C.m[0], m1 = V.C.m[1], m2 = V.C.m[2];
        stage(f, V.C.V[0], m0 * m0);
        stage(f + m0 * m0, V.C.V[1], m1 * m1);
        stage(f + m0 * m0 + m1 * m1, V.C.V[2], m2 * m2);
        stage(f + m0 * m0 + m1 * m1 + m2 * m2, V.C.laminv, m0 * m1 * m2);
    }
    cp_async_wait_all();
    __syncthreads();
    for (int q = 1; q <= lc; ++q) {                     // row weights, transfer row pointers
        const CLevel3<T> S = clevel3<T, P>(V, smem_raw, q, rank);
        const T* yb = sm + V.off_yb[q];
        const T* zb = sm + V.off_zb[q];
        const int own = S.hi - S.lo;
        T* cc = const_cast<T*>(S.cc);
        for (int e = threadIdx.x; e < own * W2; e += blockDim.x) {
            const int lr = e / W2, qq = e - lr * W2, row = S.lo + lr;
            const int j = row % S.my, k = row / S.my, bj = qq % W, bk = qq / W;
            const T myv = yb[bj * S.my + j], kyv = yb[W * S.my + bj * S.my + j];
            const T mzv = zb[bk * S.mz + k], kzv = zb[W * S.mz + bk * S.mz + k];
            cc[2 * e] = kzv * myv + mzv * kyv;
            cc[2 * e + 1] = mzv * myv;
        }
        const TransferView<T>& X = V.X[q];
        const CTransfer3<T> Y = ctransfer3(V, smem_raw, q);
        const int Rc = V.R[q - 1], myc = V.L[q - 1].m[1], mzc = V.L[q - 1].m[2];
        const int loc = min(rank * Rc, myc * mzc), ownc = min(loc + Rc, myc * mzc) - loc;
        const int ryz = X.rw[1] * X.rw[2], pyz = X.pw[1] * X.pw[2];
        int2* rr = reinterpret_cast<int2*>(const_cast<T**>(Y.rr));
        for (int e = threadIdx.x; e < ownc * ryz; e += blockDim.x) {
            const int Jl = e / ryz, s2 = e - Jl * ryz, sy = s2 % X.rw[1], sz = s2 / X.rw[1];
            const int rc = loc + Jl, J = rc % myc, K = rc / myc;
            const int fj = Y.rlo[1][J] + sy, fk = Y.rlo[2][K] + sz;
            if (fj < 0 || fj >= S.my || fk < 0 || fk >= S.mz) {
                rr[e] = pair_of(zrow, rank);
            } else {
                const int rn = fk * S.my + fj, o = rn / S.R;
                rr[e] = pair_of(t + (rn - o * S.R) * X.mc[0], o);
            }
        }
        int2* pr = reinterpret_cast<int2*>(const_cast<T**>(Y.pr));
        for (int e = threadIdx.x; e < own * pyz; e += blockDim.x) {
            const int jl = e / pyz, s2 = e - jl * pyz, sy = s2 % X.pw[1], sz = s2 / X.pw[1];
            const int row = S.lo + jl, j = row % S.my, k = row / S.my;
            const int Fj = Y.plo[1][j] + sy, Fk = Y.plo[2][k] + sz;
            if (Fj < 0 || Fj >= myc || Fk < 0 || Fk >= mzc) {
                pr[e] = pair_of(zrow, rank);
            } else {
                const int rn = Fk * myc + Fj, o = rn / Rc;
                pr[e] = pair_of(t + (rn - o * Rc) * X.mf[0], o);
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < V.img16; e += blockDim.x) img[(size_t)rank * V.img16 + e] = s16[e];
}

template <typename T, int P>
__global__ void __launch_bounds__(kCTailThreads, 1) k_cluster_tail3(ClusterTail3View<T> V, const T* __restrict__ b_in,
                                                                   T* __restrict__ x_out, int jacobi, T omega) {
    static_assert(sizeof(T) == 4, "4-byte elements (staging, integer tables)");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int rank = (int)cg::this_cluster().block_rank(), C = V.ctas;
    const int lc = V.lc;
    T* r = sm + V.off_r;
    T* t = sm + V.off_t;
    // this CTA's static shared memory from its image before the wait, the
    // dynamic part zeroed, b after it; then the pairs become pointers
    {
        const uint4* src = V.img + (size_t)rank * V.img16;
        uint4* dst = reinterpret_cast<uint4*>(smem_raw);
        for (int e = threadIdx.x; e < V.img16; e += blockDim.x) cp_async16(dst + e, src + e);
    }
    CoarseView<T> Cs = V.C;                             // coarsest eigenbasis (CTA 0 only)
    {
        T* f = sm + V.off_cv;
        const int m0 = V.C.m[0], m1 = V.C.m[1], m2 = V.C.m[2];
        Cs.V[0] = f;
        Cs.V[1] = f + m0 * m0;
        Cs.V[2] = f + m0 * m0 + m1 * m1;
        Cs.laminv = f + m0 * m0 + m1 * m1 + m2 * m2;
    }
    for (int q = 0; q <= lc; ++q) {                     // coarse e^0 = 0 on every level, zero pads
        const CLevel3<T> S = clevel3<T, P>(V, smem_raw, q, rank);
        for (int e = threadIdx.x; e < S.R * (S.mx + 2 * P); e += blockDim.x) S.x[e] = 0;
        if (q > 0)
            for (int e = threadIdx.x; e < 2 * (S.R + 2 * S.H) * S.mx; e += blockDim.x) S.TM[e] = 0;
    }
    pdl_enter();
    {
        const CLevel3<T> S = clevel3<T, P>(V, smem_raw, lc, rank);
        stage(S.b, b_in + (size_t)S.lo * S.mx, (S.hi - S.lo) * S.mx);
    }
    cp_async_wait_all();
    __syncthreads();
    {
        const int2* pairs = reinterpret_cast<const int2*>(smem_raw);
        const T** ptrs = reinterpret_cast<const T**>(smem_raw);
        for (int e = threadIdx.x; e < V.npair; e += blockDim.x) {
            const int2 pq = pairs[e];
            ptrs[e] = cptr(sm + pq.y, pq.x, rank);
        }
    }
    __syncthreads();
    cg::this_cluster().sync();
    for (int l = lc; l >= 1; --l) {
        const CLevel3<T> S = clevel3<T, P>(V, smem_raw, l, rank);
        if (jacobi) cjacobi3<T, P>(S, r, omega, rank, C);                      // pre-smooth
        else cgs3<T, P>(S, r, false, rank, C);
        crestrict3<T, P>(S, clevel3<T, P>(V, smem_raw, l - 1, rank), ctransfer3(V, smem_raw, l), r, t);
    }
    if (rank == 0) {                                    // direct solve, into the padded rows of x_0
        const int m0 = Cs.m[0], m1 = Cs.m[1], m2 = Cs.m[2], N = m0 * m1 * m2;
        const T* b0 = sm + V.off_b[0];
        T* x0 = sm + V.off_x[0];
        auto pass = [&](const T* in, T* out, int axis, bool transpose, bool pad) {
            const int md = Cs.m[axis], stride = axis == 0 ? 1 : (axis == 1 ? m0 : m0 * m1);
            const T* Vm = Cs.V[axis];
            for (int idx = threadIdx.x; idx < N; idx += blockDim.x) {
                const int i0 = idx % m0, tt = idx / m0, i1 = tt % m1, i2 = tt / m1;
                const int I = axis == 0 ? i0 : (axis == 1 ? i1 : i2);
                const int base = idx - I * stride;
                T acc = 0;
                for (int s = 0; s < md; ++s) acc += (transpose ? Vm[s * md + I] : Vm[I * md + s]) * in[base + s * stride];
                out[pad ? tt * (m0 + 2 * P) + i0 + P : idx] = acc;
            }
            __syncthreads();
        };
        pass(b0, r, 0, true, false);
        pass(r, t, 1, true, false);
        pass(t, r, 2, true, false);
        for (int i = threadIdx.x; i < N; i += blockDim.x) r[i] *= Cs.laminv[i];
        __syncthreads();
        pass(r, t, 2, false, false);
        pass(t, r, 1, false, false);
        pass(r, x0, 0, false, true);
    }
    cg::this_cluster().sync();
    for (int l = 1; l <= lc; ++l) {
        const CLevel3<T> S = clevel3<T, P>(V, smem_raw, l, rank);
        cprolong3<T, P>(S, clevel3<T, P>(V, smem_raw, l - 1, rank), ctransfer3(V, smem_raw, l), t, rank, C);
        if (jacobi) cjacobi3<T, P>(S, r, omega, rank, C);                      // post-smooth
        else cgs3<T, P>(S, r, true, rank, C);
    }
    const CLevel3<T> S = clevel3<T, P>(V, smem_raw, lc, rank);
    const int PW = S.mx + 2 * P;
    grid_for(S.hi - S.lo, S.mx, [&](int lr, int i) { x_out[(size_t)(S.lo + lr) * S.mx + i] = S.x[lr * PW + i + P]; });
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
            cudaFuncSetAttribute(k_cluster_tail<float, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
            cudaFuncSetAttribute(k_cluster_tail<float, P>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            cudaFuncSetAttribute(k_cluster_tail_image<float, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
            cudaFuncSetAttribute(k_cluster_tail_image<float, P>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            cudaFuncSetAttribute(k_cluster_tail3<float, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
            cudaFuncSetAttribute(k_cluster_tail3<float, P>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            cudaFuncSetAttribute(k_cluster_tail3_image<float, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
            cudaFuncSetAttribute(k_cluster_tail3_image<float, P>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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

template <typename T>
static cudaLaunchConfig_t cluster_config(const ClusterTailView<T>& V, cudaStream_t s, cudaLaunchAttribute* at,
                                         bool overlap) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(V.ctas);
    cfg.blockDim = dim3(kCTailThreads);
    cfg.dynamicSmemBytes = V.smem;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = V.ctas;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = overlap ? 2 : 1;
    return cfg;
}

template <typename T>
bool cluster_tail_fits(const ClusterTailView<T>& V) {
    if (V.lc < 1 || V.ctas < 2 || V.ctas > 16 || V.smem > tail_smem_limit()) return false;
    int n = 0;
    tail_with_p(V.L[V.lc].p, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        cudaLaunchAttribute at[2];
        const cudaLaunchConfig_t cfg = cluster_config(V, nullptr, at, false);
        if (cudaOccupancyMaxActiveClusters(&n, k_cluster_tail<T, P>, &cfg) != cudaSuccess) n = 0;
    });
    cudaGetLastError();
    return n >= 1;
}

template <typename T>
void cluster_tail(cudaStream_t s, const ClusterTailView<T>& V, const T* b, T* x, int jacobi, T omega) {
    tail_with_p(V.L[V.lc].p, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        cudaLaunchAttribute at[2];
        const cudaLaunchConfig_t cfg = cluster_config(V, s, at, launch_overlap());
        cudaEvent_t e0 = profiling() ? profile_before(s) : nullptr;
        cudaLaunchKernelEx(&cfg, k_cluster_tail<T, P>, V, b, x, jacobi, omega);
        if (e0) profile_after(s, (const void*)k_cluster_tail<T, P>, dim3(V.ctas), e0);
    });
    count_launch();
}

template <typename T>
static cudaLaunchConfig_t cluster3_config(const ClusterTail3View<T>& V, cudaStream_t s, cudaLaunchAttribute* at,
                                          bool overlap) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(V.ctas);
    cfg.blockDim = dim3(kCTailThreads);
    cfg.dynamicSmemBytes = V.smem;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = V.ctas;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = overlap ? 2 : 1;
    return cfg;
}

template <typename T>
bool cluster_tail3_fits(const ClusterTail3View<T>& V) {
    if (V.lc < 1 || V.ctas < 2 || V.ctas > 16 || V.smem > tail_smem_limit()) return false;
    int n = 0;
    tail_with_p(V.L[V.lc].p, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        cudaLaunchAttribute at[2];
        const cudaLaunchConfig_t cfg = cluster3_config(V, nullptr, at, false);
        if (cudaOccupancyMaxActiveClusters(&n, k_cluster_tail3<T, P>, &cfg) != cudaSuccess) n = 0;
    });
    cudaGetLastError();
    return n >= 1;
}

template <typename T>
void cluster_tail3(cudaStream_t s, const ClusterTail3View<T>& V, const T* b, T* x, int jacobi, T omega) {
    tail_with_p(V.L[V.lc].p, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        cudaLaunchAttribute at[2];
        const cudaLaunchConfig_t cfg = cluster3_config(V, s, at, launch_overlap());
        cudaEvent_t e0 = profiling() ? profile_before(s) : nullptr;
        cudaLaunchKernelEx(&cfg, k_cluster_tail3<T, P>, V, b, x, jacobi, omega);
        if (e0) profile_after(s, (const void*)k_cluster_tail3<T, P>, dim3(V.ctas), e0);
    });
    count_launch();
}

template <typename T>
cudaError_t cluster_tail3_image(const ClusterTail3View<T>& V, uint4* img) {
    cudaError_t err = cudaSuccess;
    tail_with_p(V.L[V.lc].p, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        cudaLaunchAttribute at[2];
        const cudaLaunchConfig_t cfg = cluster3_config(V, nullptr, at, false);
        err = cudaLaunchKernelEx(&cfg, k_cluster_tail3_image<T, P>, V, img);
        if (err == cudaSuccess) err = cudaStreamSynchronize(nullptr);
    });
    return err;
}

template cudaError_t cluster_tail3_image<float>(const ClusterTail3View<float>&, uint4*);
template bool cluster_tail3_fits<float>(const ClusterTail3View<float>&);
template void cluster_tail3<float>(cudaStream_t, const ClusterTail3View<float>&, const float*, float*, int, float);
template <typename T>
cudaError_t cluster_tail_image(const ClusterTailView<T>& V, uint4* img) {
    cudaError_t err = cudaSuccess;
    tail_with_p(V.L[V.lc].p, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        cudaLaunchAttribute at[2];
        const cudaLaunchConfig_t cfg = cluster_config(V, nullptr, at, false);
        err = cudaLaunchKernelEx(&cfg, k_cluster_tail_image<T, P>, V, img);
        if (err == cudaSuccess) err = cudaStreamSynchronize(nullptr);
    });
    return err;
}

template cudaError_t cluster_tail_image<float>(const ClusterTailView<float>&, uint4*);
template bool cluster_tail_fits<float>(const ClusterTailView<float>&);
template void cluster_tail<float>(cudaStream_t, const ClusterTailView<float>&, const float*, float*, int, float);

}  // namespace dev
}  // namespace igamg
