// Kernels of the general operator of Sec. 4.3 (Eq. fullelliptic) on 2D
// levels in stencil form (one row of (2p+1)^2 coefficients per unknown,
// band-major so that consecutive unknowns read consecutive words): the
// operator application / residual, the multicolour Gauss-Seidel colours, the
// weighted-Jacobi update, the 2D prolongation with correction and the dense
// coarsest solve.  Restriction reuses the transfer kernels of kernels.cu.
// FP64 throughout (the stencil's variable coefficients have no Kronecker
// structure to exploit).
#include "device.hpp"

namespace igamg {
namespace dev {

namespace {
constexpr int kGenThreads = 256;

template <typename T>
__device__ __forceinline__ T gen_warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// (A x)_I over the stencil of unknown (ix, iy)
template <int P>
__device__ __forceinline__ double stencil_row(const StencilView& V, const double* __restrict__ x, int ix, int iy) {
    constexpr int W = 2 * P + 1;
    const int mx = V.m[0], my = V.m[1];
    const size_t N = V.n(), I = (size_t)iy * mx + ix;
    double acc = 0.0;
#pragma unroll
    for (int dy = -P; dy <= P; ++dy) {
        const int jy = iy + dy;
        if (jy < 0 || jy >= my) continue;
#pragma unroll
        for (int dx = -P; dx <= P; ++dx) {
            const int jx = ix + dx;
            if (jx < 0 || jx >= mx) continue;
            acc += V.S[(size_t)((dy + P) * W + dx + P) * N + I] * x[(size_t)jy * mx + jx];
        }
    }
    return acc;
}
}  // namespace

template <int P>
__global__ void __launch_bounds__(kGenThreads) k_gen_residual(StencilView V, const double* __restrict__ x,
                                                              const double* __restrict__ b, double* __restrict__ r,
                                                              double* __restrict__ partial) {
    pdl_enter();
    __shared__ double red[kGenThreads / 32];
    const size_t N = V.n();
    double ss = 0.0;
    for (size_t I = (size_t)blockIdx.x * blockDim.x + threadIdx.x; I < N; I += (size_t)gridDim.x * blockDim.x) {
        const int ix = (int)(I % V.m[0]), iy = (int)(I / V.m[0]);
        const double ax = stencil_row<P>(V, x, ix, iy);
        const double v = b ? b[I] - ax : ax;
        r[I] = v;
        ss += v * v;
    }
    if (partial) {
        ss = gen_warp_sum(ss);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kGenThreads / 32; ++w) t += red[w];
            partial[blockIdx.x] = t;
        }
    }
}

// one colour (cx, cy): x_I += (b_I - (A x)_I) / A_II for ix = cx mod (p+1), iy = cy mod (p+1)
template <int P>
__global__ void __launch_bounds__(kGenThreads) k_gen_gs_colour(StencilView V, int cx, int cy, double* __restrict__ x,
                                                               const double* __restrict__ b) {
    pdl_enter();
    constexpr int P1 = P + 1;
    const int ncx = (V.m[0] - cx + P) / P1, ncy = (V.m[1] - cy + P) / P1;
    const size_t cnt = (size_t)(ncx > 0 ? ncx : 0) * (ncy > 0 ? ncy : 0);
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += (size_t)gridDim.x * blockDim.x) {
        const int ix = cx + P1 * (int)(t % ncx), iy = cy + P1 * (int)(t / ncx);
        const size_t I = (size_t)iy * V.m[0] + ix;
        const double ax = stencil_row<P>(V, x, ix, iy);
        x[I] += (b[I] - ax) * V.inv[I];
    }
}

__global__ void __launch_bounds__(kGenThreads) k_gen_jacobi(size_t n, double omega, const double* __restrict__ inv,
                                                            const double* __restrict__ r, double* __restrict__ x) {
    pdl_enter();
    for (size_t I = (size_t)blockIdx.x * blockDim.x + threadIdx.x; I < n; I += (size_t)gridDim.x * blockDim.x)
        x[I] += omega * inv[I] * r[I];
}

// x[j][i] += sum_b Py(j, b) sum_a Px(i, a) e[b][a] (row form of both 1D P)
__global__ void __launch_bounds__(kGenThreads) k_gen_prolong(TransferView<double> X, const double* __restrict__ e,
                                                             double* __restrict__ x) {
    pdl_enter();
    const int mfx = X.mf[0], mfy = X.mf[1], mcx = X.mc[0], mcy = X.mc[1];
    const size_t N = (size_t)mfx * mfy;
    for (size_t I = (size_t)blockIdx.x * blockDim.x + threadIdx.x; I < N; I += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(I % mfx), j = (int)(I / mfx);
        double acc = 0.0;
        for (int sb = 0; sb < X.pw[1]; ++sb) {
            const int bb = X.plo[1][j] + sb;
            const double py = X.pv[1][(size_t)j * X.pw[1] + sb];
            if (bb >= mcy || py == 0.0) continue;
            double t = 0.0;
            for (int sa = 0; sa < X.pw[0]; ++sa) {
                const int a = X.plo[0][i] + sa;
                if (a >= mcx) continue;
                t += X.pv[0][(size_t)i * X.pw[0] + sa] * e[(size_t)bb * mcx + a];
            }
            acc += py * t;
        }
        x[I] += acc;
    }
}

__global__ void __launch_bounds__(kGenThreads) k_gen_dense(const double* __restrict__ A, int n, const double* __restrict__ r,
                                                           double* __restrict__ e) {
    pdl_enter();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc += A[(size_t)i * n + j] * r[j];
        e[i] = acc;
    }
}

int gen_blocks(size_t n) {
    size_t g = (n + kGenThreads - 1) / kGenThreads;
    if (g > 152 * 8) g = 152 * 8;
    return (int)(g < 1 ? 1 : g);
}

template <typename F>
static void with_p_gen(int p, F&& f) {
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

void gen_residual(cudaStream_t s, const StencilView& V, const double* x, const double* b, double* r, double* partial) {
    with_p_gen(V.p, [&](auto PC) {
        launch_chained(k_gen_residual<decltype(PC)::value>, gen_blocks(V.n()), kGenThreads, 0, s, V, x, b, r, partial);
    });
    count_launch();
}

void gen_gs_sweep(cudaStream_t s, const StencilView& V, bool descending, double* x, const double* b) {
    const int P1 = V.p + 1;
    for (int c = 0; c < P1 * P1; ++c) {
        const int cc = descending ? P1 * P1 - 1 - c : c;
        const int cx = cc % P1, cy = cc / P1;
        const size_t cnt = (size_t)((V.m[0] - cx + V.p) / P1) * ((V.m[1] - cy + V.p) / P1);
        if (cnt == 0 || V.m[0] <= cx || V.m[1] <= cy) continue;
        with_p_gen(V.p, [&](auto PC) {
            launch_chained(k_gen_gs_colour<decltype(PC)::value>, gen_blocks(cnt), kGenThreads, 0, s, V, cx, cy, x, b);
        });
        count_launch();
    }
}

void gen_jacobi_update(cudaStream_t s, const StencilView& V, double omega, const double* r, double* x) {
    launch_chained(k_gen_jacobi, gen_blocks(V.n()), kGenThreads, 0, s, V.n(), omega, V.inv, r, x);
    count_launch();
}

void gen_prolong_add(cudaStream_t s, const TransferView<double>& X, const double* e, double* x) {
    launch_chained(k_gen_prolong, gen_blocks((size_t)X.mf[0] * X.mf[1]), kGenThreads, 0, s, X, e, x);
    count_launch();
}

void gen_dense_apply(cudaStream_t s, const double* Ainv, int n, const double* r, double* e) {
    launch_chained(k_gen_dense, 1, kGenThreads, 0, s, Ainv, n, r, e);
    count_launch();
}

}  // namespace dev
}  // namespace igamg
