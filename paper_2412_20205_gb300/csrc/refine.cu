// Residual update of the FP32-IR form in double-FP32 arithmetic (2D and 3D).
//
// Within a restart cycle the FP64 residual of the iterate is carried by the
// recurrence r_{i+1} = r_i - A e_i, where e_i is the FP32 correction of the
// i-th V-cycle (x_{i+1} = x_i + e_i).  A e_i is of the size of r_i, so unlike
// b - A x_{i+1} it involves no cancellation against b; it is evaluated with
// every FP64 operator entry held as a float pair (hi + lo) and float-pair
// accumulation (exact products by FMA, two-sum additions), about 2^-46
// relative per entry of A e, on the FP32 pipe (58x the FP64 rate on GB300).
// r itself stays in FP64 and every restart starts from a freshly computed
// FP64 residual b - A x, which is also what the stopping test measures.
#include "device.hpp"

namespace igamg {
namespace dev {

constexpr int kRefThreads = 256;
// 3D passes: one CTA per block of kRowsPerCta3 consecutive rows (the y and z
// passes: rows j of one plane k), its threads striding over rows x columns.
constexpr int kRowsPerCta3 = 8;

// (sh, sl) += (ch + cl) * (vh + vl), float-pair accumulation
__device__ __forceinline__ void df_acc(float& sh, float& sl, float ch, float cl, float vh, float vl) {
    const float p = ch * vh;
    float pe = fmaf(ch, vh, -p);                  // exact low part of ch * vh
    pe = fmaf(ch, vl, fmaf(cl, vh, pe));
    const float t = sh + p;                       // two-sum of the high parts
    const float bv = t - sh;
    const float err = (sh - (t - bv)) + (p - bv);
    sh = t;
    sl += err + pe;
}

__device__ __forceinline__ void df_norm(float& sh, float& sl) {
    const float t = sh + sl;
    sl = sl - (t - sh);
    sh = t;
}

// One CTA per block of rb consecutive rows (2D: rb = 1): S_out = S_in + e;
// float-pair x-band sums of e.
template <int P>
__global__ void __launch_bounds__(kRefThreads) k_xpass_df(DFView D, int rb, const double* __restrict__ S_in,
                                                          double* __restrict__ S_out, const float* __restrict__ e,
                                                          float* __restrict__ tmh, float* __restrict__ tml,
                                                          float* __restrict__ tkh, float* __restrict__ tkl) {
    pdl_enter();
    extern __shared__ float es[];                 // the rows of e, each with a zero halo of p
    const int mx = D.m[0], rows = D.m[1] * D.m[2], PW = mx + 2 * P;
    const int r0 = blockIdx.x * rb, nr = min(rb, rows - r0);
    const size_t base = (size_t)r0 * mx;
    for (int q = threadIdx.x; q < nr * PW; q += blockDim.x) {
        const int rr = q / PW, ii = q - rr * PW, i = ii - P;
        float v = 0.f;
        if (i >= 0 && i < mx) {
            const size_t o = base + (size_t)rr * mx + i;
            v = e[o];
            S_out[o] = S_in[o] + (double)v;
        }
        es[q] = v;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nr * mx; q += blockDim.x) {
        const int rr = q / mx, i = q - rr * mx;
        const float* er = es + rr * PW;
        float mh = 0.f, ml = 0.f, kh = 0.f, kl = 0.f;
        if (i >= D.tlo[0] && i < D.thi[0]) {
#pragma unroll
            for (int b = 0; b <= 2 * P; ++b) {
                const float v = er[i + b];
                df_acc(mh, ml, D.Mch[0][b], D.Mcl[0][b], v, 0.f);
                df_acc(kh, kl, D.Kch[0][b], D.Kcl[0][b], v, 0.f);
            }
        } else {
#pragma unroll
            for (int b = 0; b <= 2 * P; ++b) {
                const float v = er[i + b];
                const int qq = b * mx + i;
                df_acc(mh, ml, D.Mh[0][qq], D.Ml[0][qq], v, 0.f);
                df_acc(kh, kl, D.Kh[0][qq], D.Kl[0][qq], v, 0.f);
            }
        }
        df_norm(mh, ml);
        df_norm(kh, kl);
        const size_t o = base + q;
        tmh[o] = mh;
        tml[o] = ml;
        tkh[o] = kh;
        tkl[o] = kl;
    }
}

// One CTA per row j: r -= sum_dj K_y(j, dj) T_M(e)(j + dj - p) + M_y(j, dj) T_K(e)(...).
template <int P>
__global__ void __launch_bounds__(kRefThreads) k_residual_df(DFView D, const float* __restrict__ tmh,
                                                             const float* __restrict__ tml,
                                                             const float* __restrict__ tkh,
                                                             const float* __restrict__ tkl, double* __restrict__ r,
                                                             float* __restrict__ rf) {
    const int mx = D.m[0], my = D.m[1], j = blockIdx.x;
    const bool uni = j >= D.tlo[1] && j < D.thi[1];
    float kyh[2 * P + 1], kyl[2 * P + 1], myh[2 * P + 1], myl[2 * P + 1];
#pragma unroll
    for (int dj = 0; dj <= 2 * P; ++dj) {
        const int q = dj * my + j;
        kyh[dj] = uni ? D.Kch[1][dj] : D.Kh[1][q];
        kyl[dj] = uni ? D.Kcl[1][dj] : D.Kl[1][q];
        myh[dj] = uni ? D.Mch[1][dj] : D.Mh[1][q];
        myl[dj] = uni ? D.Mcl[1][dj] : D.Ml[1][q];
    }
    pdl_enter();                                  // above: operator data only
    const size_t base = (size_t)j * mx;
    for (int i = threadIdx.x; i < mx; i += blockDim.x) {
        float ah = 0.f, al = 0.f;
#pragma unroll
        for (int dj = 0; dj <= 2 * P; ++dj) {
            const int jj = j + dj - P;
            if (jj < 0 || jj >= my) continue;
            const size_t q = (size_t)jj * mx + i;
            df_acc(ah, al, kyh[dj], kyl[dj], tmh[q], tml[q]);
            df_acc(ah, al, myh[dj], myl[dj], tkh[q], tkl[q]);
        }
        const double v = r[base + i] - ((double)ah + (double)al);
        r[base + i] = v;
        rf[base + i] = (float)v;
    }
}

// 3D, y pass: U = sum_dj M_y(j, dj) T_M(j + dj, k), V = sum_dj K_y(j, dj)
// T_M(j + dj, k) + M_y(j, dj) T_K(j + dj, k), float pairs.  The block's rows'
// y-band pairs are staged in shared memory.
template <int P>
__global__ void __launch_bounds__(kRefThreads) k_yfactor_df3(DFView D, const float* __restrict__ tmh,
                                                             const float* __restrict__ tml,
                                                             const float* __restrict__ tkh,
                                                             const float* __restrict__ tkl, float* __restrict__ uh,
                                                             float* __restrict__ ul, float* __restrict__ vh,
                                                             float* __restrict__ vl) {
    constexpr int W = 2 * P + 1;
    __shared__ float cy[4][kRowsPerCta3][W];        // K_y hi, K_y lo, M_y hi, M_y lo
    const int mx = D.m[0], my = D.m[1];
    const int nbj = (my + kRowsPerCta3 - 1) / kRowsPerCta3;
    const int k = blockIdx.x / nbj, j0 = (blockIdx.x - k * nbj) * kRowsPerCta3;
    const int nr = min(kRowsPerCta3, my - j0);
    for (int e = threadIdx.x; e < nr * W; e += blockDim.x) {
        const int jr = e / W, dj = e - jr * W, j = j0 + jr, q = dj * my + j;
        const bool uni = j >= D.tlo[1] && j < D.thi[1];
        cy[0][jr][dj] = uni ? D.Kch[1][dj] : D.Kh[1][q];
        cy[1][jr][dj] = uni ? D.Kcl[1][dj] : D.Kl[1][q];
        cy[2][jr][dj] = uni ? D.Mch[1][dj] : D.Mh[1][q];
        cy[3][jr][dj] = uni ? D.Mcl[1][dj] : D.Ml[1][q];
    }
    __syncthreads();
    pdl_enter();                                  // above: operator data only
    for (int e = threadIdx.x; e < nr * mx; e += blockDim.x) {
        const int jr = e / mx, i = e - jr * mx, j = j0 + jr;
        float Uh = 0.f, Ul = 0.f, Vh = 0.f, Vl = 0.f;
#pragma unroll
        for (int dj = 0; dj < W; ++dj) {
            const int jj = j + dj - P;
            if (jj < 0 || jj >= my) continue;
            const size_t q = ((size_t)k * my + jj) * mx + i;
            const float ah = tmh[q], al = tml[q];
            df_acc(Uh, Ul, cy[2][jr][dj], cy[3][jr][dj], ah, al);
            df_acc(Vh, Vl, cy[0][jr][dj], cy[1][jr][dj], ah, al);
            df_acc(Vh, Vl, cy[2][jr][dj], cy[3][jr][dj], tkh[q], tkl[q]);
        }
        df_norm(Uh, Ul);
        df_norm(Vh, Vl);
        const size_t o = ((size_t)k * my + j) * mx + i;
        uh[o] = Uh;
        ul[o] = Ul;
        vh[o] = Vh;
        vl[o] = Vl;
    }
}

// 3D, z pass: r -= sum_dk K_z(k, dk) U(j, k + dk) + M_z(k, dk) V(j, k + dk) in
// float pairs; rf = float(r).  The plane's z-band pairs are the CTA's.
template <int P>
__global__ void __launch_bounds__(kRefThreads) k_zresidual_df3(DFView D, const float* __restrict__ uh,
                                                               const float* __restrict__ ul,
                                                               const float* __restrict__ vh,
                                                               const float* __restrict__ vl, double* __restrict__ r,
                                                               float* __restrict__ rf) {
    const int mx = D.m[0], my = D.m[1], mz = D.m[2];
    const int nbj = (my + kRowsPerCta3 - 1) / kRowsPerCta3;
    const int k = blockIdx.x / nbj, j0 = (blockIdx.x - k * nbj) * kRowsPerCta3;
    const int nr = min(kRowsPerCta3, my - j0);
    const bool uni = k >= D.tlo[2] && k < D.thi[2];
    float kzh[2 * P + 1], kzl[2 * P + 1], mzh[2 * P + 1], mzl[2 * P + 1];
#pragma unroll
    for (int dk = 0; dk <= 2 * P; ++dk) {
        const int q = dk * mz + k;
        kzh[dk] = uni ? D.Kch[2][dk] : D.Kh[2][q];
        kzl[dk] = uni ? D.Kcl[2][dk] : D.Kl[2][q];
        mzh[dk] = uni ? D.Mch[2][dk] : D.Mh[2][q];
        mzl[dk] = uni ? D.Mcl[2][dk] : D.Ml[2][q];
    }
    pdl_enter();                                  // above: operator data only
    for (int e = threadIdx.x; e < nr * mx; e += blockDim.x) {
        const int jr = e / mx, i = e - jr * mx, j = j0 + jr;
        float ah = 0.f, al = 0.f;
#pragma unroll
        for (int dk = 0; dk <= 2 * P; ++dk) {
            const int kk = k + dk - P;
            if (kk < 0 || kk >= mz) continue;
            const size_t q = ((size_t)kk * my + j) * mx + i;
            df_acc(ah, al, kzh[dk], kzl[dk], uh[q], ul[q]);
            df_acc(ah, al, mzh[dk], mzl[dk], vh[q], vl[q]);
        }
        const size_t o = ((size_t)k * my + j) * mx + i;
        const double v = r[o] - ((double)ah + (double)al);
        r[o] = v;
        rf[o] = (float)v;
    }
}

template <typename F>
static void ref_with_p(int p, F&& f) {
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

static int ref_threads(int mx) {
    const int t = ((mx + 31) / 32) * 32;
    return t < 64 ? 64 : (t > kRefThreads ? kRefThreads : t);
}

void refine_xpass_df(cudaStream_t s, const DFView& D, const double* S_in, double* S_out, const float* e,
                     float* tm_h, float* tm_l, float* tk_h, float* tk_l) {
    // 2D rows (1025 nodes at 1024^2) fill a CTA; short 3D rows go kRowsPerCta3 to a CTA
    const int rows = D.m[1] * D.m[2], rb = D.m[2] > 1 ? kRowsPerCta3 : 1;
    const size_t smem = (size_t)rb * (D.m[0] + 2 * D.p) * sizeof(float);
    ref_with_p(D.p, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        launch_chained(k_xpass_df<P>, (rows + rb - 1) / rb, ref_threads(D.m[0] * rb), smem, s, D, rb, S_in, S_out, e,
                       tm_h, tm_l, tk_h, tk_l);
    });
    count_launch();
}

void refine_residual_df(cudaStream_t s, const DFView& D, const float* tm_h, const float* tm_l, const float* tk_h,
                        const float* tk_l, double* r, float* rf) {
    ref_with_p(D.p, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        launch_chained(k_residual_df<P>, D.m[1], ref_threads(D.m[0]), 0, s, D, tm_h, tm_l, tk_h, tk_l, r, rf);
    });
    count_launch();
}

void refine_residual_df3(cudaStream_t s, const DFView& D, const float* tm_h, const float* tm_l, const float* tk_h,
                         const float* tk_l, float* u, float* v, double* r, float* rf) {
    const size_t N = (size_t)D.m[0] * D.m[1] * D.m[2];
    const int blocks = D.m[2] * ((D.m[1] + kRowsPerCta3 - 1) / kRowsPerCta3);
    const int threads = ref_threads(D.m[0] * kRowsPerCta3);
    ref_with_p(D.p, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        launch_chained(k_yfactor_df3<P>, blocks, threads, 0, s, D, tm_h, tm_l, tk_h, tk_l, u, u + N, v, v + N);
        launch_chained(k_zresidual_df3<P>, blocks, threads, 0, s, D, u, u + N, v, v + N, r, rf);
    });
    count_launch(2);
}

}  // namespace dev
}  // namespace igamg
