// CUDA kernels of the extrapolated multigrid solver (sm_103a).
//
// Precision: every kernel is templated on the working type T (double for the
// FP64 path, float inside the FP32 V-cycles of iterative refinement).  On
// GB300 the FP64 pipe delivers about 1/58 of the FP32 rate, so the FP64
// kernels are bound by FP64 instruction count: the layouts below are chosen to
// minimise FP64 arithmetic (row partial sums are kept, not recomputed).
//
// Operator (Sec. 2, Eq. (2)): A = sum_d K_d (x) prod_{e!=d} M_e on interior
// unknowns, x fastest.  Writing T_M = (I (x) M_x) x and T_K = (I (x) K_x) x
// ("row partial sums", one x-direction contraction per row), the product
// splits into row couplings:
//   2D: (A x)_row = sum_{dj} Ky(j, j+dj) T_M(row+dj) + My(j, j+dj) T_K(row+dj)
//   3D: coefficients Kz My + Mz Ky on T_M and Mz My on T_K, over (dj, dk).
#include "device.hpp"
#include "bands.cuh"

#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cxxabi.h>
#include <string>
#include <type_traits>
#include <vector>

namespace igamg {

namespace {
thread_local long long g_launches = 0;
std::atomic<bool> g_overlap{true};
thread_local int g_no_overlap = 0;
std::atomic<long long> g_wait_ns{1000000000LL};      // one second
std::atomic<int> g_wait_test{0};
std::atomic<int> g_sync_gen{0};
}
namespace {
struct ProfRecord {
    const void* func;
    unsigned grid;
    cudaEvent_t e0, e1;
};
thread_local bool g_prof = false;
thread_local std::vector<ProfRecord>* g_records = nullptr;
}  // namespace

bool profiling() { return g_prof; }

cudaEvent_t profile_before(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    cudaEventRecord(e, s);
    return e;
}

void profile_after(cudaStream_t s, const void* func, dim3 grid, cudaEvent_t e0) {
    cudaEvent_t e1 = nullptr;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return; }
    cudaEventRecord(e1, s);
    if (!g_records) g_records = new std::vector<ProfRecord>();
    g_records->push_back({func, grid.x * grid.y * grid.z, e0, e1});
}

void profile_start() {
    g_prof = true;
    if (!g_records) g_records = new std::vector<ProfRecord>();
}

long profile_stop(int cap, char* names, int name_len, double* us, int* grid) {
    g_prof = false;
    if (!g_records) return 0;
    const long n = (long)g_records->size();
    for (long i = 0; i < n; ++i) {
        ProfRecord& r = (*g_records)[i];
        cudaEventSynchronize(r.e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.e0, r.e1);
        if (i < cap) {
            if (us) us[i] = 1e3 * (double)ms;
            if (grid) grid[i] = (int)r.grid;
            if (names && name_len > 0) {
                const char* nm = nullptr;
                if (cudaFuncGetName(&nm, r.func) != cudaSuccess || !nm) nm = "?";
                // "void igamg::dev::k_name<args>(params)" -> "k_name<args>"
                int st = 0;
                char* dm = abi::__cxa_demangle(nm, nullptr, nullptr, &st);
                std::string full = (st == 0 && dm) ? dm : nm;
                std::free(dm);
                size_t depth = 0, end = full.size();
                for (size_t c = 0; c < full.size(); ++c) {
                    if (full[c] == '<') ++depth;
                    else if (full[c] == '>') --depth;
                    else if (full[c] == '(' && depth == 0) { end = c; break; }
                }
                std::string shortn = full.substr(0, end);
                const size_t sp = shortn.rfind("::", shortn.find('<') == std::string::npos ? std::string::npos
                                                                                           : shortn.find('<'));
                if (sp != std::string::npos) shortn = shortn.substr(sp + 2);
                if (shortn.rfind("void ", 0) == 0) shortn = shortn.substr(5);
                std::snprintf(names + (size_t)i * name_len, name_len, "%s", shortn.c_str());
            }
        }
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    g_records->clear();
    cudaGetLastError();
    return n;
}

void set_wait_limit(long long ns, int test_unset) {
    g_wait_ns.store(ns < 0 ? 0 : ns);
    g_wait_test.store(test_unset ? 1 : 0);
    g_sync_gen.fetch_add(1);
}
long long wait_limit_ns() { return g_wait_ns.load(); }
int wait_test_unset() { return g_wait_test.load(); }
int sync_generation() { return g_sync_gen.load(); }
void count_launch(long long n) { g_launches += n; }
long long launch_count() { return g_launches; }
bool launch_overlap() { return g_no_overlap == 0 && g_overlap.load(std::memory_order_relaxed); }
void set_launch_overlap(bool on) { g_overlap.store(on, std::memory_order_relaxed); }
NoOverlapScope::NoOverlapScope() { ++g_no_overlap; }
NoOverlapScope::~NoOverlapScope() { --g_no_overlap; }

namespace dev {

constexpr int kThreads = 256;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum (deterministic order); result valid in thread 0.
template <typename T>
__device__ T block_sum(T v, T* red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    T s = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) s += red[i];
    __syncthreads();
    return s;
}

// Row-coupling coefficients of row (j, k): for neighbour q = (dj, dk) the
// weights on T_M and T_K and the neighbour's row index; neighbours outside
// the grid get weight 0 and the row's own index (loads stay in bounds).
template <typename T, int DIM, int P>
__device__ void row_couplings(const LevelView<T>& L, int j, int k, T* cM, T* cK, int* nrow) {
    constexpr int W = 2 * P + 1;
    constexpr int NNB = (DIM == 3) ? W * W : W;
    const int my = L.m[1], mz = L.m[2];
    for (int q = threadIdx.x; q < NNB; q += blockDim.x) {
        const int dj = (q % W) - P, dk = (DIM == 3) ? (q / W) - P : 0;
        const int jj = j + dj, kk = k + dk;
        const bool ok = jj >= 0 && jj < my && kk >= 0 && kk < mz;
        T a = 0, c = 0;
        if (ok) {
            const T myv = band_md(L, 1, j, dj + P), kyv = band_kd(L, 1, j, dj + P);
            if (DIM == 2) {
                a = kyv;
                c = myv;
            } else {
                const T mzv = band_md(L, 2, k, dk + P), kzv = band_kd(L, 2, k, dk + P);
                a = kzv * myv + mzv * kyv;
                c = mzv * myv;
            }
        }
        cM[q] = a;
        cK[q] = c;
        nrow[q] = ok ? (kk * my + jj) : (k * my + j);
    }
}

// Global load of data that other CTAs of the same grid write (CG = true):
// through L2 only (.cg), never from a stale L1 line.  CG = false: a plain load.
template <bool CG, typename T>
__device__ __forceinline__ T ldv(const T* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// sum over neighbour rows q (all, or all but the own row) of cM T_M + cK T_K at column i
template <typename T, int NNB, int SKIP, bool CG = false>
__device__ __forceinline__ T couple(const T* cM, const T* cK, const int* nrow, const T* __restrict__ TM,
                                    const T* __restrict__ TK, int mx, int i) {
    T acc = 0;
    constexpr int U = NNB > 49 ? 9 : NNB;       // bound the loads kept in flight (3D, p >= 4)
#pragma unroll U
    for (int q = 0; q < NNB; ++q) {
        if (q == SKIP) continue;
        const size_t o = (size_t)nrow[q] * mx + i;
        acc += cM[q] * ldv<CG>(TM + o) + cK[q] * ldv<CG>(TK + o);
    }
    return acc;
}

// ---------------------------------------------------------------- x-pass
// One CTA per row.  Source row: x, or x + add (iterative-refinement update),
// or sum_j gamma_j S_j (extrapolated combination); written to x_out when it
// differs from x.  Then T_M, T_K of the row.
template <typename T, typename A, int P>
__global__ void __launch_bounds__(kThreads) k_xpass(LevelView<T> L, const T* __restrict__ x,
                                                     T* __restrict__ x_out, const A* __restrict__ add,
                                                     int nS, const double* __restrict__ gamma,
                                                     const T* __restrict__ S, size_t ldS,
                                                     T* __restrict__ TM, T* __restrict__ TK) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* xs = reinterpret_cast<T*>(smem_raw);
    const int mx = L.m[0];
    const size_t base = (size_t)blockIdx.x * mx;
    __shared__ double g[kMaxQ + 2];
    if (nS > 0) {
        for (int j = threadIdx.x; j < nS; j += blockDim.x) g[j] = gamma[j];
        __syncthreads();
    }
    for (int ii = threadIdx.x; ii < mx + 2 * P; ii += blockDim.x) {
        const int i = ii - P;
        T v = 0;
        if (i >= 0 && i < mx) {
            if (nS > 0) {
                double s = 0.0;
                for (int j = 0; j < nS; ++j)
                    if (g[j] != 0.0) s += g[j] * (double)S[(size_t)j * ldS + base + i];
                v = (T)s;
                x_out[base + i] = v;
            } else if (add != nullptr) {
                v = x[base + i] + (T)add[base + i];
                x_out[base + i] = v;
            } else {
                v = x[base + i];
            }
        }
        xs[ii] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < mx; i += blockDim.x) {
        T am = 0, ak = 0;
#pragma unroll
        for (int b = 0; b <= 2 * P; ++b) {
            const T xv = xs[i + b];
            am += band_m(L, i, b) * xv;
            ak += band_k(L, i, b) * xv;
        }
        TM[base + i] = am;
        TK[base + i] = ak;
    }
}

// ---------------------------------------------------------------- GS phase
// Multicolour Gauss-Seidel, colour c = cx + (p+1) cy (+ (p+1)^2 cz).  For a
// fixed (cy, cz) the rows j = cy mod (p+1) (k = cz mod (p+1)) are updated; no
// two of them couple, and within a row the colours cx = 0..p form a 1D
// multicolour sweep with the frozen off-row part F = sum_{row' != row}
// (cM T_M + cK T_K).  The row's own T_M, T_K at a node are their values at
// the start of the phase plus the x-band applied to this sweep's corrections,
// so a full sweep costs about one apply plus 2(2p+1) FMA per node.
//
// Latency layout: one CTA per target row with enough threads to cover the row
// in one pass; every global load of the phase (neighbour T rows, own T, x, b,
// inverse diagonal, boundary band entries) is issued in one round, and the
// p+1 colour steps then touch shared memory only.  Row couplings and the
// interior x-band come from kernel parameters.
constexpr int kBandCols = 8 * kMaxP;            // staged non-uniform x-band columns

template <typename T, int P>
struct RowBand {
    // x-band entry (row i, band b): parameters in the uniform interior, the
    // staged table for up to kBandCols boundary columns, memory otherwise
    const LevelView<T>& L;
    const T* bm;
    const T* bk;
    int nb;
    __device__ __forceinline__ int slot(int i) const {
        if (i < L.tlo[0]) return i;
        return L.tlo[0] + (i - L.thi[0]);
    }
    __device__ __forceinline__ T m(int i, int b) const {
        if (i >= L.tlo[0] && i < L.thi[0]) return L.Mc[0][b];
        if (nb <= kBandCols) return bm[slot(i) * (2 * P + 1) + b];
        return L.Mb[0][b * L.m[0] + i];
    }
    __device__ __forceinline__ T k(int i, int b) const {
        if (i >= L.tlo[0] && i < L.thi[0]) return L.Kc[0][b];
        if (nb <= kBandCols) return bk[slot(i) * (2 * P + 1) + b];
        return L.Kb[0][b * L.m[0] + i];
    }
};

// largest CTA of the row kernels: 3D rows couple to (2p+1)^2 - 1 neighbour
// rows whose loads are kept in flight together; 2D rows take 512 threads
// (FP32 at 1024^2: 1024-thread CTAs ran 4% slower, 256 and 128 slower still)
template <typename T, int DIM>
constexpr int row_cta_max() { return DIM == 3 ? 256 : 512; }


// The p+1 colour steps of one row in the incremental form.  For the partial-
// sum update the CTA's warps are split into p+1 groups, one per node residue
// rho = i mod (p+1); with the colours unrolled (DESC fixed) the offsets of the
// same-colour nodes within reach of a node, r = (cx - rho) mod (p+1) and
// r - (p+1), are compile-time constants, so in the uniform interior the band
// entries are kernel parameters at fixed offsets (the group branch is
// warp-uniform).  CTAs with fewer than p+1 warps take the generic loop.
template <typename T, int P, bool DESC, bool GROUPS>
__device__ __forceinline__ void gs_colours_incremental(const LevelView<T>& L, const RowBand<T, P>& band, int mx,
                                                       T am, T ak, const T* rhs, T* tm, T* tk, T* dl, T* xs,
                                                       const T* dv) {
    constexpr int P1 = P + 1;
    const int per = GROUPS ? ((int)blockDim.x / 32 / P1) * 32 : 0;   // threads per residue group
    const int rho = per > 0 ? (int)threadIdx.x / per : 0;
    const int k0 = per > 0 ? (int)threadIdx.x - rho * per : 0;
    const int tlo = L.tlo[0], thi = L.thi[0];
#pragma unroll
    for (int c = 0; c < P1; ++c) {
        const int cx = DESC ? P - c : c;
        for (int i = cx + P1 * (int)threadIdx.x; i < mx; i += P1 * (int)blockDim.x) {
            const T d = (rhs[i] - (am * tm[i] + ak * tk[i])) * dv[i];
            xs[i] += d;
            dl[i] = d;
        }
        __syncthreads();
        if (per > 0) {
#pragma unroll
            for (int rr = 0; rr < P1; ++rr) {
                if (rr != rho) continue;
                const int r = ((cx - rr) % P1 + P1) % P1;
                for (int i = rr + P1 * k0; i < mx; i += P1 * per) {
                    T sm = 0, sk = 0;
                    const int i1 = i + r;                       // same-colour node at offset r
                    const int i2 = i1 - P1;                     // and at offset r - (p+1)
                    if (i >= tlo && i < thi) {
                        const T d1 = dl[i1];
                        sm = L.Mc[0][r + P] * d1;
                        sk = L.Kc[0][r + P] * d1;
                        if (r >= 1) {
                            const T d2 = dl[i2];
                            sm += L.Mc[0][r - 1] * d2;
                            sk += L.Kc[0][r - 1] * d2;
                        }
                    } else {
                        if (i1 < mx) {
                            const T d1 = dl[i1];
                            sm += band.m(i, r + P) * d1;
                            sk += band.k(i, r + P) * d1;
                        }
                        if (r >= 1 && i2 >= 0) {
                            const T d2 = dl[i2];
                            sm += band.m(i, r - 1) * d2;
                            sk += band.k(i, r - 1) * d2;
                        }
                    }
                    tm[i] += sm;
                    tk[i] += sk;
                }
            }
        } else {
            for (int i = threadIdx.x; i < mx; i += blockDim.x) {
                int r = (cx - i) % P1;
                if (r < 0) r += P1;
                T sm = 0, sk = 0;
                const int i1 = i + r;
                if (i1 < mx) {
                    const T d1 = dl[i1];
                    sm += band.m(i, r + P) * d1;
                    sk += band.k(i, r + P) * d1;
                }
                const int i2 = i1 - P1;
                if (r >= 1 && i2 >= 0) {
                    const T d2 = dl[i2];
                    sm += band.m(i, r - 1) * d2;
                    sk += band.k(i, r - 1) * d2;
                }
                tm[i] += sm;
                tk[i] += sk;
            }
        }
        __syncthreads();
    }
}

// Which of the two in-row formulations a GS phase uses, by measurement on
// GB300 (2D 1024^2 and 3D 128^3 RRE solves): the window form (one barrier per
// colour, 2(2p+1) FMA per node) won for FP32 2D at p = 2, 4, 5 (by 5-18%)
// and lost at p = 3 to the grouped incremental form; for FP32 3D at p = 3 it
// won by 6% (332 -> 313 ms; other p not measured, window form); in FP64 its
// extra FMAs cost more than the barriers it saves (2D p = 5: 278 ms against
// 226 ms).
template <typename T, int DIM, int P>
constexpr bool gs_window() { return sizeof(T) == 4 && (DIM == 3 || P != 3); }

// Shared-memory rows of one GS row update: right side minus the frozen
// off-row part, the row's own partial sums, this sweep's corrections, x and
// the inverse diagonal (6 rows of m_x), then the row couplings and the staged
// boundary x-band columns.
template <typename T, int DIM, int P>
struct GsSmem {
    static constexpr int W = 2 * P + 1;
    static constexpr int NNB = (DIM == 3) ? W * W : W;
    T *rhs, *tm, *tk, *dl, *xs, *dv;
    T* cM;
    T* cK;
    int* nrow;
    T* bm;
    T* bk;
};

template <typename T, int DIM, int P>
__device__ __forceinline__ GsSmem<T, DIM, P> gs_smem(int mx) {
    using S = GsSmem<T, DIM, P>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T cM[S::NNB], cK[S::NNB];
    __shared__ int nrow[S::NNB];
    __shared__ T bm[kBandCols * S::W], bk[kBandCols * S::W];
    S g;
    g.rhs = reinterpret_cast<T*>(smem_raw);
    g.tm = g.rhs + mx;
    g.tk = g.tm + mx;
    g.dl = g.tk + mx;
    g.xs = g.dl + mx;
    g.dv = g.xs + mx;
    g.cM = cM;
    g.cK = cK;
    g.nrow = nrow;
    g.bm = bm;
    g.bk = bk;
    return g;
}

// The x-band's boundary columns (row independent) into shared memory; returns
// their count (the RowBand falls back to memory above kBandCols).
template <typename T, int P>
__device__ __forceinline__ int gs_stage_band(const LevelView<T>& L, T* bm, T* bk) {
    constexpr int W = 2 * P + 1;
    const int mx = L.m[0];
    const int nb = L.tlo[0] + (mx - L.thi[0]);
    if (nb <= kBandCols)
        for (int t = threadIdx.x; t < nb * W; t += blockDim.x) {
            const int sl = t / W, bb = t % W;
            const int i = sl < L.tlo[0] ? sl : L.thi[0] + (sl - L.tlo[0]);
            bm[t] = L.Mb[0][bb * mx + i];
            bk[t] = L.Kb[0][bb * mx + i];
        }
    return nb;
}

// One target row's p+1 colour steps from its loads to its stores, after the
// row couplings (cM, cK, nrow) and, in 2D, the inverse diagonal (dv) are in
// shared memory and a barrier has made them visible.  CG: x, T_M and T_K are
// read through L2 (they are written by other CTAs of the same launch).
template <typename T, int DIM, int P, bool WINDOW, bool CG>
__device__ __forceinline__ void gs_row(const LevelView<T>& L, const GsSmem<T, DIM, P>& g, const RowBand<T, P>& band,
                                       size_t base, int descending, T* __restrict__ x, const T* __restrict__ b,
                                       T* __restrict__ TM, T* __restrict__ TK) {
    constexpr int P1 = P + 1, W = 2 * P + 1;
    constexpr int NNB = (DIM == 3) ? W * W : W;
    constexpr int OWN = (DIM == 3) ? P * W + P : P;
    const int mx = L.m[0];
    T* rhs = g.rhs;
    T* tm = g.tm;
    T* tk = g.tk;
    T* dl = g.dl;
    T* xs = g.xs;
    T* dv = g.dv;
    for (int i = threadIdx.x; i < mx; i += blockDim.x) {
        rhs[i] = b[base + i] - couple<T, NNB, OWN, CG>(g.cM, g.cK, g.nrow, TM, TK, mx, i);
        tm[i] = ldv<CG>(TM + base + i);
        tk[i] = ldv<CG>(TK + base + i);
        xs[i] = ldv<CG>(x + base + i);
        if constexpr (DIM == 3) dv[i] = L.invdiag[base + i];
        if constexpr (WINDOW) dl[i] = 0;
    }
    __syncthreads();
    const T am = g.cM[OWN], ak = g.cK[OWN];
    if constexpr (WINDOW) {
        const int tlo = L.tlo[0], thi = L.thi[0];
        // sum_b M_x(i, b) dl[i + b - p] (and K_x): the x-band applied to this
        // sweep's corrections so far (zero for colours not yet done).  In the
        // uniform interior (where every neighbour exists: p <= i < m - p, see
        // LevelView) the band comes from the kernel parameters at
        // compile-time offsets.
        auto xband_dl = [&](int i, bool skip_own, T& sm, T& sk) {
            if (i >= tlo && i < thi) {
#pragma unroll
                for (int bb = 0; bb <= 2 * P; ++bb) {
                    if (skip_own && bb == P) continue;
                    const T dn = dl[i + bb - P];
                    sm += L.Mc[0][bb] * dn;
                    sk += L.Kc[0][bb] * dn;
                }
            } else {
#pragma unroll
                for (int bb = 0; bb <= 2 * P; ++bb) {
                    const int n = i + bb - P;
                    if ((skip_own && bb == P) || n < 0 || n >= mx) continue;
                    const T dn = dl[n];
                    sm += band.m(i, bb) * dn;
                    sk += band.k(i, bb) * dn;
                }
            }
        };
        // Colour by colour along the row; the row's own partial sums at node i
        // are tm[i] + xband_dl(i) (its own correction is still zero), so one
        // barrier per colour suffices.
#pragma unroll
        for (int c = 0; c < P1; ++c) {
            const int cx = descending ? P - c : c;
            for (int i = cx + P1 * (int)threadIdx.x; i < mx; i += P1 * (int)blockDim.x) {
                T sm = tm[i], sk = tk[i];
                xband_dl(i, true, sm, sk);
                const T d = (rhs[i] - (am * sm + ak * sk)) * dv[i];
                xs[i] += d;
                dl[i] = d;
            }
            __syncthreads();
        }
        for (int i = threadIdx.x; i < mx; i += blockDim.x) {
            T sm = tm[i], sk = tk[i];
            xband_dl(i, false, sm, sk);
            x[base + i] = xs[i];
            TM[base + i] = sm;
            TK[base + i] = sk;
        }
    } else {
        // Incremental form: after each colour the row's T_M, T_K take the
        // corrections of that colour (a gather of the <= 2 same-colour nodes
        // within reach), two barriers per colour but 4 FMA per node.
        // residue groups measured faster for FP32 2D rows (1024^2 p = 3: 11.75 -> 11.25 ms);
        // FP64 and 3D rows keep the generic update
        constexpr bool G = DIM == 2 && sizeof(T) == 4;
        if (descending) gs_colours_incremental<T, P, true, G>(L, band, mx, am, ak, rhs, tm, tk, dl, xs, dv);
        else gs_colours_incremental<T, P, false, G>(L, band, mx, am, ak, rhs, tm, tk, dl, xs, dv);
        for (int i = threadIdx.x; i < mx; i += blockDim.x) {
            x[base + i] = xs[i];
            TM[base + i] = tm[i];
            TK[base + i] = tk[i];
        }
    }
}

template <typename T, int DIM, int P, bool WINDOW>
__device__ __forceinline__ void gs_phase_body(const LevelView<T>& L, int cy, int cz, int descending,
                                              T* __restrict__ x, const T* __restrict__ b,
                                              T* __restrict__ TM, T* __restrict__ TK) {
    constexpr int P1 = P + 1;
    const int mx = L.m[0], my = L.m[1];
    const int nty = (my - cy + P) / P1;
    const int j = cy + P1 * (blockIdx.x % nty);
    const int k = (DIM == 3) ? cz + P1 * (blockIdx.x / nty) : 0;
    const size_t base = ((size_t)k * my + j) * mx;
    const GsSmem<T, DIM, P> g = gs_smem<T, DIM, P>(mx);
    if constexpr (DIM == 3) pdl_enter();
    row_couplings<T, DIM, P>(L, j, k, g.cM, g.cK, g.nrow);
    const int nb = gs_stage_band<T, P>(L, g.bm, g.bk);
    // 2D rows: everything up to the wait reads operator data that no kernel
    // writes, so under launch overlap it runs during the previous kernel's
    // tail (measured 2-9% per solve).  3D rows wait at entry: this order cost
    // them 27% (128^3, p = 3), with or without overlap.
    if constexpr (DIM == 2) {
        for (int i = threadIdx.x; i < mx; i += blockDim.x) g.dv[i] = L.invdiag[base + i];
        pdl_enter();
    }
    __syncthreads();
    const RowBand<T, P> band{L, g.bm, g.bk, nb};
    gs_row<T, DIM, P, WINDOW, false>(L, g, band, base, descending, x, b, TM, TK);
}

// ---------------------------------------------------------------- single-launch sweep
// Cross-CTA waits of a single-launch sweep.  ld.acquire / st.release at GPU
// scope order a row's published data before and after its flag.
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Waits until *f != 0; false when limit_ns has passed, or at once when an
// earlier wait already gave up (*err != 0), so that a sweep whose waits run
// out ends within about one limit in all.
__device__ __noinline__ bool wait_flag(const unsigned* f, long long limit_ns, const unsigned* err) {
    if (ld_acquire_gpu(f)) return true;
    const long long t0 = global_ns();
    for (;;) {
        if (*(volatile const unsigned*)err) return false;
        __nanosleep(32);
        if (ld_acquire_gpu(f)) return true;
        if (global_ns() - t0 >= limit_ns) return false;
    }
}

// One whole multicolour Gauss-Seidel sweep ((p+1)^dim colours) in ONE launch.
// The colour order is the row-phase order of gs_phase_body: for 2D phases
// ph = 0..p over rows j = cy mod (p+1), cy = ph (descending: p - ph); in 3D
// ph runs over (cy, cz) with cz slowest.  Within a phase no two rows couple,
// and a row reads the T rows of the 2p (3D: (2p+1)^2 - 1) rows within reach.
// Those of earlier phases must hold this sweep's values and those of later
// phases the previous ones; so a row may start as soon as its earlier-phase
// neighbours are done, and a later-phase neighbour cannot overwrite what it
// reads because that neighbour waits for it in turn.  The result is exactly
// that of the phase-by-phase launches (same arithmetic, same order per row).
//
// Work distribution: persistent CTAs claim rows from a counter in phase
// order, so every row a CTA waits on was claimed earlier by a CTA that is
// running; the unfinished row of smallest claim index never waits, which
// rules out deadlock whatever the number of resident CTAs.  Each CTA
// prefetches its next claim.  Every wait is bounded (SweepSync::limit_ns):
// on expiry the kernel records it in *err, goes on and returns normally (the
// host reports IGAMG_ETIMEOUT).  The last CTA to finish clears the row flags
// and counters for the next sweep.
template <typename T, int DIM, int P, bool WINDOW>
__device__ __forceinline__ void gs_sweep_body(const LevelView<T>& L, int descending, T* x, const T* __restrict__ b,
                                              T* TM, T* TK, const SweepSync& sy) {
    constexpr int P1 = P + 1, W = 2 * P + 1;
    constexpr int NPH = (DIM == 3) ? P1 * P1 : P1;
    const int mx = L.m[0], my = L.m[1], mz = (DIM == 3) ? L.m[2] : 1;
    const int rows = my * mz;
    const GsSmem<T, DIM, P> g = gs_smem<T, DIM, P>(mx);
    __shared__ int s_task[2];
    __shared__ int s_last;
    const int nb = gs_stage_band<T, P>(L, g.bm, g.bk);      // operator data: before the wait
    const RowBand<T, P> band{L, g.bm, g.bk, nb};
    pdl_enter();
    if (threadIdx.x == 0) {
        s_task[0] = (int)atomicAdd(&sy.ctr[0], 1u);
        if (sy.test_unset && !wait_flag(sy.never, sy.limit_ns, sy.err)) atomicOr(sy.err, 1u);
    }
    __syncthreads();
    for (int it = 0;; ++it) {
        const int t = s_task[it & 1];
        if (t >= rows) break;
        if (threadIdx.x == 0) s_task[(it + 1) & 1] = (int)atomicAdd(&sy.ctr[0], 1u);
        // claim index -> phase and row, phases in sweep order
        int ph = 0, rem = t, cy = 0, cz = 0, nty = 0;
        for (; ph < NPH; ++ph) {
            const int c = descending ? NPH - 1 - ph : ph;
            cy = c % P1;
            cz = c / P1;
            nty = (my - cy + P) / P1;
            const int ntz = (DIM == 3) ? (mz - cz + P) / P1 : 1;
            const int cnt = (nty > 0 && ntz > 0) ? nty * ntz : 0;
            if (rem < cnt) break;
            rem -= cnt;
        }
        const int j = cy + P1 * (rem % nty);
        const int k = (DIM == 3) ? cz + P1 * (rem / nty) : 0;
        const int row = k * my + j;
        const size_t base = (size_t)row * mx;
        row_couplings<T, DIM, P>(L, j, k, g.cM, g.cK, g.nrow);
        if constexpr (DIM == 2)
            for (int i = threadIdx.x; i < mx; i += blockDim.x) g.dv[i] = L.invdiag[base + i];
        // wait for the neighbours of earlier phases (one thread each)
        constexpr int NQ = (DIM == 3) ? W * W : W;
        for (int q = threadIdx.x; q < NQ; q += blockDim.x) {
            const int dj = (q % W) - P, dk = (DIM == 3) ? (q / W) - P : 0;
            const int jj = j + dj, kk = k + dk;
            if ((dj == 0 && dk == 0) || jj < 0 || jj >= my || kk < 0 || kk >= mz) continue;
            const int c = (jj % P1) + P1 * (kk % P1);
            const int phn = descending ? NPH - 1 - c : c;
            if (phn < ph && !wait_flag(&sy.done[kk * my + jj], sy.limit_ns, sy.err)) atomicOr(sy.err, 1u);
        }
        __syncthreads();
        gs_row<T, DIM, P, WINDOW, true>(L, g, band, base, descending, x, b, TM, TK);
        __syncthreads();                            // every store of the row issued
        if (threadIdx.x == 0) {
            __threadfence();
            st_release_gpu(&sy.done[row], 1u);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&sy.ctr[1], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {                                   // every row is done: reset for the next sweep
        __threadfence();
        for (int r = threadIdx.x; r < rows; r += blockDim.x) sy.done[r] = 0u;
        if (threadIdx.x == 0) {
            sy.ctr[0] = 0u;
            sy.ctr[1] = 0u;
        }
    }
}

// Kernels: one CTA per target row of the phase.  2D rows are compiled for two
// resident 512-thread CTAs per SM (up to 64 registers; without that hint
// ptxas settled on 32-40 registers and spilled, and one CTA per SM with 128
// registers ran slower in FP64); 3D rows keep the compiler's default.
template <typename T, int P, bool WINDOW>
__global__ void __launch_bounds__(row_cta_max<T, 2>(), 2)
    k_gs_phase2(LevelView<T> L, int cy, int cz, int descending, T* __restrict__ x, const T* __restrict__ b,
                T* __restrict__ TM, T* __restrict__ TK) {
    gs_phase_body<T, 2, P, WINDOW>(L, cy, cz, descending, x, b, TM, TK);
}
template <typename T, int P, bool WINDOW>
__global__ void __launch_bounds__(row_cta_max<T, 3>())
    k_gs_phase3(LevelView<T> L, int cy, int cz, int descending, T* __restrict__ x, const T* __restrict__ b,
                T* __restrict__ TM, T* __restrict__ TK) {
    gs_phase_body<T, 3, P, WINDOW>(L, cy, cz, descending, x, b, TM, TK);
}
template <typename T, int P, bool WINDOW>
__global__ void __launch_bounds__(row_cta_max<T, 2>(), 2)
    k_gs_sweep2(LevelView<T> L, int descending, T* x, const T* __restrict__ b, T* TM, T* TK, SweepSync sy) {
    gs_sweep_body<T, 2, P, WINDOW>(L, descending, x, b, TM, TK, sy);
}
template <typename T, int P, bool WINDOW>
__global__ void __launch_bounds__(row_cta_max<T, 3>())
    k_gs_sweep3(LevelView<T> L, int descending, T* x, const T* __restrict__ b, T* TM, T* TK, SweepSync sy) {
    gs_sweep_body<T, 3, P, WINDOW>(L, descending, x, b, TM, TK, sy);
}

// ---------------------------------------------------------------- residual
// r = b - A x (or A x without b) from T_M, T_K; optional per-row ||r||^2 and
// an FP64 copy of r.
template <typename T, typename R, int DIM, int P>
__global__ void __launch_bounds__(kThreads) k_residual(LevelView<T> L, const T* __restrict__ b,
                                                        const T* __restrict__ TM, const T* __restrict__ TK,
                                                        R* __restrict__ r, double* __restrict__ partial,
                                                        double* __restrict__ r64) {
    constexpr int W = 2 * P + 1;
    constexpr int NNB = (DIM == 3) ? W * W : W;
    const int mx = L.m[0], my = L.m[1];
    const int row = blockIdx.x, j = row % my, k = row / my;
    const size_t base = (size_t)row * mx;
    __shared__ T cM[NNB], cK[NNB];
    __shared__ int nrow[NNB];
    __shared__ double red[kThreads / 32];
    row_couplings<T, DIM, P>(L, j, k, cM, cK, nrow);     // operator data only
    pdl_enter();
    __syncthreads();
    double ss = 0.0;
    for (int i = threadIdx.x; i < mx; i += blockDim.x) {
        const T ax = couple<T, NNB, -1>(cM, cK, nrow, TM, TK, mx, i);
        const T v = b ? b[base + i] - ax : ax;
        r[base + i] = (R)v;
        if (r64) r64[base + i] = (double)v;
        ss += (double)v * (double)v;
    }
    if (partial) {
        const double s = block_sum(ss, red);
        if (threadIdx.x == 0) partial[row] = s;
    }
}

// 3D residual by sum factorisation across y and z.  With the row partial
// sums T_M = (I (x) I (x) M_x) x and T_K = (I (x) I (x) K_x) x,
//   A x = sum_dk K_z(k, k+dk) U(j, k+dk) + M_z(k, k+dk) V(j, k+dk),
//   U(j, k') = sum_dj M_y(j, j+dj) T_M(j+dj, k'),
//   V(j, k') = sum_dj K_y(j, j+dj) T_M(j+dj, k') + M_y(j, j+dj) T_K(j+dj, k'),
// so a y pass (U, V: 3(2p+1) FMA per unknown) and a z pass (2(2p+1) FMA)
// replace the (2p+1)^2-row coupling of k_residual (4(2p+1)^2 FMA).  One CTA
// per row (j, k) in both passes.
template <typename T, int P>
__global__ void __launch_bounds__(kThreads) k_yfactor3(LevelView<T> L, const T* __restrict__ TM,
                                                        const T* __restrict__ TK, T* __restrict__ U,
                                                        T* __restrict__ V) {
    constexpr int W = 2 * P + 1;
    const int mx = L.m[0], my = L.m[1];
    const int row = blockIdx.x, j = row % my;
    const size_t base = (size_t)row * mx;
    __shared__ T cm[W], ck[W];
    __shared__ int ok[W];
    if (threadIdx.x < W) {                           // operator data only
        const int jj = j + (int)threadIdx.x - P;
        ok[threadIdx.x] = jj >= 0 && jj < my;
        cm[threadIdx.x] = ok[threadIdx.x] ? band_md(L, 1, j, threadIdx.x) : T(0);
        ck[threadIdx.x] = ok[threadIdx.x] ? band_kd(L, 1, j, threadIdx.x) : T(0);
    }
    pdl_enter();
    __syncthreads();
    for (int i = threadIdx.x; i < mx; i += blockDim.x) {
        T u = 0, v = 0;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            if (!ok[q]) continue;
            const long long o = (long long)base + (long long)(q - P) * mx + i;
            const T tm = TM[o], tk = TK[o];
            u += cm[q] * tm;
            v += ck[q] * tm + cm[q] * tk;
        }
        U[base + i] = u;
        V[base + i] = v;
    }
}

template <typename T, typename R, int P>
__global__ void __launch_bounds__(kThreads) k_zresidual3(LevelView<T> L, const T* __restrict__ b,
                                                          const T* __restrict__ U, const T* __restrict__ V,
                                                          R* __restrict__ r, double* __restrict__ partial,
                                                          double* __restrict__ r64) {
    constexpr int W = 2 * P + 1;
    const int mx = L.m[0], my = L.m[1], mz = L.m[2];
    const int row = blockIdx.x, k = row / my;
    const size_t base = (size_t)row * mx, plane = (size_t)mx * my;
    __shared__ T cz[W], mzc[W];
    __shared__ int ok[W];
    __shared__ double red[kThreads / 32];
    if (threadIdx.x < W) {                           // operator data only
        const int kk = k + (int)threadIdx.x - P;
        ok[threadIdx.x] = kk >= 0 && kk < mz;
        cz[threadIdx.x] = ok[threadIdx.x] ? band_kd(L, 2, k, threadIdx.x) : T(0);
        mzc[threadIdx.x] = ok[threadIdx.x] ? band_md(L, 2, k, threadIdx.x) : T(0);
    }
    pdl_enter();
    __syncthreads();
    double ss = 0.0;
    for (int i = threadIdx.x; i < mx; i += blockDim.x) {
        T ax = 0;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            if (!ok[q]) continue;
            const long long o = (long long)base + (long long)(q - P) * (long long)plane + i;
            ax += cz[q] * U[o] + mzc[q] * V[o];
        }
        const T v = b ? b[base + i] - ax : ax;
        r[base + i] = (R)v;
        if (r64) r64[base + i] = (double)v;
        ss += (double)v * (double)v;
    }
    if (partial) {
        const double t = block_sum(ss, red);
        if (threadIdx.x == 0) partial[row] = t;
    }
}

// Weighted Jacobi (Sec. 4: the paper's smoother, omega = 2/3):
// x += omega D^{-1} (b - A x), every node from the same x.  A x comes from
// the row partial sums, which this kernel only reads, so each CTA may
// overwrite its own row of x; the caller refreshes T_M, T_K afterwards.
template <typename T, int DIM, int P>
__global__ void __launch_bounds__(kThreads) k_jacobi(LevelView<T> L, T omega, const T* __restrict__ b,
                                                      const T* __restrict__ TM, const T* __restrict__ TK,
                                                      T* __restrict__ x) {
    constexpr int W = 2 * P + 1;
    constexpr int NNB = (DIM == 3) ? W * W : W;
    const int mx = L.m[0], my = L.m[1];
    const int row = blockIdx.x, j = row % my, k = row / my;
    const size_t base = (size_t)row * mx;
    __shared__ T cM[NNB], cK[NNB];
    __shared__ int nrow[NNB];
    row_couplings<T, DIM, P>(L, j, k, cM, cK, nrow);     // operator data only
    pdl_enter();
    __syncthreads();
    for (int i = threadIdx.x; i < mx; i += blockDim.x) {
        const T v = b[base + i] - couple<T, NNB, -1>(cM, cK, nrow, TM, TK, mx, i);
        x[base + i] += omega * L.invdiag[base + i] * v;
    }
}

// 2D weighted Jacobi with the row partial sums of the new x in one kernel:
// a CTA updates its row (b - A x from the old sums T_M, T_K of the 2p+1
// coupled rows), keeps it in shared memory with a zero halo of p, and writes
// that row's new sums to TMo, TKo.  The old and new sums live in different
// buffers, so no CTA reads a row sum another CTA writes.
template <typename T, int P>
__global__ void __launch_bounds__(kThreads) k_jacobi2(LevelView<T> L, T omega, const T* __restrict__ b,
                                                       const T* __restrict__ TM, const T* __restrict__ TK,
                                                       T* __restrict__ x, T* __restrict__ TMo,
                                                       T* __restrict__ TKo) {
    constexpr int W = 2 * P + 1;
    const int mx = L.m[0], j = blockIdx.x;
    const size_t base = (size_t)j * mx;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* xs = reinterpret_cast<T*>(smem_raw);
    __shared__ T cM[W], cK[W];
    __shared__ int nrow[W];
    row_couplings<T, 2, P>(L, j, 0, cM, cK, nrow);       // operator data only
    pdl_enter();
    __syncthreads();
    for (int ii = threadIdx.x; ii < mx + 2 * P; ii += blockDim.x) {
        const int i = ii - P;
        T v = 0;
        if (i >= 0 && i < mx) {
            const T rv = b[base + i] - couple<T, W, -1>(cM, cK, nrow, TM, TK, mx, i);
            v = x[base + i] + omega * L.invdiag[base + i] * rv;
            x[base + i] = v;
        }
        xs[ii] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < mx; i += blockDim.x) {
        T am = 0, ak = 0;
#pragma unroll
        for (int bb = 0; bb <= 2 * P; ++bb) {
            const T xv = xs[i + bb];
            am += band_m(L, i, bb) * xv;
            ak += band_k(L, i, bb) * xv;
        }
        TMo[base + i] = am;
        TKo[base + i] = ak;
    }
}

// 2D: r = b - A x of one row (from T_M, T_K) followed by the x-axis pass of
// the restriction on that row, t[j][I] = sum_s rv[I rw + s] r[j][rlo[I] + s];
// r itself never goes to memory.
template <typename T, int P>
__global__ void __launch_bounds__(kThreads) k_residual_restrict_x(LevelView<T> L, const T* __restrict__ b,
                                                                   const T* __restrict__ TM,
                                                                   const T* __restrict__ TK, int mcx,
                                                                   const int* __restrict__ rlo,
                                                                   const T* __restrict__ rv, int rw,
                                                                   T* __restrict__ t) {
    constexpr int W = 2 * P + 1;
    const int mx = L.m[0], j = blockIdx.x;
    const size_t base = (size_t)j * mx;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* rr = reinterpret_cast<T*>(smem_raw);
    __shared__ T cM[W], cK[W];
    __shared__ int nrow[W];
    row_couplings<T, 2, P>(L, j, 0, cM, cK, nrow);       // operator data only
    pdl_enter();
    __syncthreads();
    for (int i = threadIdx.x; i < mx; i += blockDim.x)
        rr[i] = b[base + i] - couple<T, W, -1>(cM, cK, nrow, TM, TK, mx, i);
    __syncthreads();
    for (int I = threadIdx.x; I < mcx; I += blockDim.x) {
        const int lo = rlo[I];
        T acc = 0;
        for (int q = 0; q < rw; ++q) {
            const int f = lo + q;
            if (f < 0 || f >= mx) continue;
            acc += rv[(size_t)I * rw + q] * rr[f];
        }
        t[(size_t)j * mcx + I] = acc;
    }
}

// 2D: x += P e on one fine row with both prolongation axes in one kernel
// (the x-axis values of the <= pw1 coarse rows that reach the row are formed
// on the fly), then the row's T_M, T_K.  Same sums in the same order as the
// two-pass form.  With `staged`, the pw1 coarse rows are first copied to
// shared memory with coalesced loads (same values, same sums).
template <typename T, int P>
__global__ void __launch_bounds__(kThreads) k_prolong_fused2(LevelView<T> L, const T* __restrict__ e, int mcx,
                                                              int mcy, const int* __restrict__ plo0,
                                                              const T* __restrict__ pv0, int pw0,
                                                              const int* __restrict__ plo1,
                                                              const T* __restrict__ pv1, int pw1,
                                                              T* __restrict__ x, T* __restrict__ TM,
                                                              T* __restrict__ TK, int staged) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* xs = reinterpret_cast<T*>(smem_raw);
    const int mx = L.m[0], j = blockIdx.x;
    T* es = xs + mx + 2 * P;                        // staged coarse rows l1 .. l1 + pw1 - 1
    const size_t base = (size_t)j * mx;
    const int l1 = plo1[j];                         // operator data only
    pdl_enter();
    if (staged) {
        for (int t = threadIdx.x; t < pw1 * mcx; t += blockDim.x) {
            const int q1 = t / mcx, f = t - q1 * mcx;
            const int J = l1 + q1;
            es[t] = (J >= 0 && J < mcy) ? e[(size_t)J * mcx + f] : (T)0;
        }
        __syncthreads();
    }
    for (int ii = threadIdx.x; ii < mx + 2 * P; ii += blockDim.x) {
        const int i = ii - P;
        T v = 0;
        if (i >= 0 && i < mx) {
            const int l0 = plo0[i];
            T cor = 0;
            for (int q1 = 0; q1 < pw1; ++q1) {
                const int J = l1 + q1;
                if (J < 0 || J >= mcy) continue;
                T tJ = 0;                               // (P_x e)(i, J)
                for (int q0 = 0; q0 < pw0; ++q0) {
                    const int f = l0 + q0;
                    if (f < 0 || f >= mcx) continue;
                    tJ += pv0[(size_t)i * pw0 + q0] * (staged ? es[q1 * mcx + f] : e[(size_t)J * mcx + f]);
                }
                cor += pv1[(size_t)j * pw1 + q1] * tJ;
            }
            v = x[base + i] + cor;
            x[base + i] = v;
        }
        xs[ii] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < mx; i += blockDim.x) {
        T am = 0, ak = 0;
#pragma unroll
        for (int bb = 0; bb <= 2 * P; ++bb) {
            const T xv = xs[i + bb];
            am += band_m(L, i, bb) * xv;
            ak += band_k(L, i, bb) * xv;
        }
        TM[base + i] = am;
        TK[base + i] = ak;
    }
}

// ---------------------------------------------------------------- transfer
// out (dims d0 x d1 x d2, x fastest) along `axis`: out[.., I, ..] =
// sum_s val[I*width + s] in[.., lo[I] + s, ..], in having n_in along axis.
template <typename T>
__global__ void k_transfer_axis(const T* __restrict__ in, T* __restrict__ out, int d0, int d1, int d2,
                                int axis, int n_in, const int* __restrict__ lo,
                                const T* __restrict__ val, int width, T* __restrict__ zero, size_t nzero) {
    pdl_enter();
    // optionally also clear `zero` (the next level's x | T_M | T_K)
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < nzero; q += (size_t)gridDim.x * blockDim.x)
        zero[q] = 0;
    const size_t total = (size_t)d0 * d1 * d2;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i0 = (int)(idx % d0);
        const size_t t = idx / d0;
        const int i1 = (int)(t % d1), i2 = (int)(t / d1);
        const int I = axis == 0 ? i0 : (axis == 1 ? i1 : i2);
        const int l = lo[I];
        T acc = 0;
        for (int s = 0; s < width; ++s) {
            const int f = l + s;
            if (f < 0 || f >= n_in) continue;
            size_t src;
            if (axis == 0) src = ((size_t)i2 * d1 + i1) * n_in + f;
            else if (axis == 1) src = ((size_t)i2 * n_in + f) * d0 + i0;
            else src = ((size_t)f * d1 + i1) * d0 + i0;
            acc += val[(size_t)I * width + s] * in[src];
        }
        out[idx] = acc;
    }
}

// Last prolongation axis fused with the correction x += P e and the x-pass:
// one CTA per fine row; tmp holds the correction with the last axis coarse.
template <typename T, int DIM, int P>
__global__ void __launch_bounds__(kThreads) k_prolong_last(LevelView<T> L, const T* __restrict__ tmp,
                                                            int n_in, const int* __restrict__ lo,
                                                            const T* __restrict__ val, int width,
                                                            T* __restrict__ x, T* __restrict__ TM,
                                                            T* __restrict__ TK) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* xs = reinterpret_cast<T*>(smem_raw);
    const int mx = L.m[0], my = L.m[1];
    const int row = blockIdx.x, j = row % my, k = row / my;
    const int I = (DIM == 2) ? j : k;
    const size_t base = (size_t)row * mx;
    const int l = lo[I];
    for (int ii = threadIdx.x; ii < mx + 2 * P; ii += blockDim.x) {
        const int i = ii - P;
        T v = 0;
        if (i >= 0 && i < mx) {
            T cor = 0;
            for (int s = 0; s < width; ++s) {
                const int f = l + s;
                if (f < 0 || f >= n_in) continue;
                const size_t src = (DIM == 2) ? (size_t)f * mx + i : ((size_t)f * my + j) * mx + i;
                cor += val[(size_t)I * width + s] * tmp[src];
            }
            v = x[base + i] + cor;
            x[base + i] = v;
        }
        xs[ii] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < mx; i += blockDim.x) {
        T am = 0, ak = 0;
#pragma unroll
        for (int b = 0; b <= 2 * P; ++b) {
            const T xv = xs[i + b];
            am += band_m(L, i, b) * xv;
            ak += band_k(L, i, b) * xv;
        }
        TM[base + i] = am;
        TK[base + i] = ak;
    }
}

// ---------------------------------------------------------------- coarse solve
// Fast diagonalisation in one CTA: e = V diag(laminv) V^T r, V = (x) V_d.
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) k_coarse_fd(CoarseView<T> C, const T* __restrict__ r,
                                                         T* __restrict__ e) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m0 = C.m[0], m1 = C.m[1], m2 = (DIM == 3) ? C.m[2] : 1;
    const int N = m0 * m1 * m2;
    T* a = reinterpret_cast<T*>(smem_raw);
    T* bb = a + N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) a[i] = r[i];
    __syncthreads();
    auto pass = [&](const T* in, T* out, int axis, bool transpose) {
        const int md = C.m[axis];
        const T* V = C.V[axis];
        for (int idx = threadIdx.x; idx < N; idx += blockDim.x) {
            const int i0 = idx % m0, t = idx / m0, i1 = t % m1, i2 = t / m1;
            const int I = axis == 0 ? i0 : (axis == 1 ? i1 : i2);
            const int stride = axis == 0 ? 1 : (axis == 1 ? m0 : m0 * m1);
            const int base = idx - I * stride;
            T acc = 0;
            for (int s = 0; s < md; ++s)
                acc += (transpose ? V[s * md + I] : V[I * md + s]) * in[base + s * stride];
            out[idx] = acc;
        }
        __syncthreads();
    };
    T* cur = a;
    T* nxt = bb;
    for (int d = 0; d < DIM; ++d) {                 // V^T r
        pass(cur, nxt, d, true);
        T* t = cur; cur = nxt; nxt = t;
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) cur[i] *= C.laminv[i];
    __syncthreads();
    for (int d = DIM - 1; d >= 0; --d) {            // V (...)
        pass(cur, nxt, d, false);
        T* t = cur; cur = nxt; nxt = t;
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) e[i] = cur[i];
}

// ---------------------------------------------------------------- norms
__global__ void __launch_bounds__(kThreads) k_sumsq(const double* __restrict__ v, size_t n,
                                                     double* __restrict__ partial) {
    pdl_enter();
    __shared__ double red[kThreads / 32];
    double s = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        s += v[i] * v[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// e = u - v (written to e) with per-block partial sums of e^2.
__global__ void __launch_bounds__(kThreads) k_diff_sumsq(const double* __restrict__ u, const double* __restrict__ v,
                                                         size_t n, double* __restrict__ e, double* __restrict__ partial) {
    pdl_enter();
    __shared__ double red[kThreads / 32];
    double s = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double d = u[i] - v[i];
        e[i] = d;
        s += d * d;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// R = float(c r), E = float(c e) with c = sqrt(n) / enorm[0] (unit RMS of E).
__global__ void __launch_bounds__(kThreads) k_scale_pair(const double* __restrict__ r, const double* __restrict__ e,
                                                         const double* __restrict__ enorm, size_t n,
                                                         float* __restrict__ R, float* __restrict__ E) {
    pdl_enter();
    const double c = sqrt((double)n) / fmax(enorm[0], 1e-300);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        R[i] = (float)(c * r[i]);
        E[i] = (float)(c * e[i]);
    }
}

__global__ void __launch_bounds__(1024) k_norm_final(const double* __restrict__ partial, int nparts,
                                                      const double* __restrict__ denom,
                                                      double* __restrict__ out, int slot) {
    pdl_enter();
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += partial[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
        double v = sqrt(s);
        if (denom) v = v / *denom;
        out[slot] = v;
    }
}

// ---------------------------------------------------------------- device-side restart loop
__global__ void k_loop_step(cudaGraphConditionalHandle h, LoopState* st, const double* __restrict__ res,
                            const unsigned* __restrict__ err, double* __restrict__ hist) {
    pdl_enter();
    if (threadIdx.x != 0) return;
    const int cyc = st->cyc + 1;
    const double r = res[0];
    st->cyc = cyc;
    st->res = r;
    if (hist && cyc < kLoopHist) hist[cyc] = r;
    int code = kLoopRunning;
    if (!isfinite(r)) code = kLoopBreakdown;
    else if (*err) code = kLoopTimeout;
    else if (r <= st->tol) code = kLoopConverged;
    else if (cyc >= st->max_cycles) code = kLoopMaxCycles;
    st->code = code;
    cudaGraphSetConditional(h, code == kLoopRunning ? 1u : 0u);
}

__global__ void k_loop_init(cudaGraphConditionalHandle h, const LoopState* st) {
    pdl_enter();
    if (threadIdx.x == 0) cudaGraphSetConditional(h, st->code == kLoopRunning ? 1u : 0u);
}

// ---------------------------------------------------------------- extrapolation
// Gram partials of Delta s_a = s_{a+1} - s_a (a = 0..Q), upper triangle.
template <int Q>
__global__ void __launch_bounds__(kThreads) k_gram_partial(const double* __restrict__ S, size_t ld,
                                                            size_t n, double* __restrict__ partial) {
    pdl_enter();
    constexpr int NP = (Q + 1) * (Q + 2) / 2;
    double acc[NP];
#pragma unroll
    for (int c = 0; c < NP; ++c) acc[c] = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double s[Q + 2];
#pragma unroll
        for (int j = 0; j < Q + 2; ++j) s[j] = S[(size_t)j * ld + i];
        double d[Q + 1];
#pragma unroll
        for (int j = 0; j <= Q; ++j) d[j] = s[j + 1] - s[j];
        int c = 0;
#pragma unroll
        for (int a = 0; a <= Q; ++a)
#pragma unroll
            for (int bb = a; bb <= Q; ++bb) acc[c++] += d[a] * d[bb];
    }
    __shared__ double red[kThreads / 32][NP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < NP; ++c) {
        const double v = warp_sum(acc[c]);
        if (lane == 0) red[w][c] = v;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < NP; c += blockDim.x) {
        double s = 0.0;
        for (int ww = 0; ww < (int)blockDim.x / 32; ++ww) s += red[ww][c];
        partial[(size_t)blockIdx.x * NP + c] = s;
    }
}

// Extrapolation coefficients by CholeskyQR2 (Fukaya et al., 2014) on the
// difference matrix Delta S = [Delta s_0 .. Delta s_q]: the R of Algorithms 3-4
// is obtained from two Gram passes instead of a Householder QR.
//   pass 1: G = Delta S^T Delta S; D = sqrt(diag G); Cholesky of the
//           equilibrated G^ = D^-1 G D^-1 = R1^T R1, truncated at the first
//           column whose pivot is numerically zero (or whose difference is 0).
//   pass 2: W = Delta S_a (R1 D)^-1 for the a retained columns, plus the raw
//           next column if any; G2 = Z^T Z = R2^T R2; R^ = R2 R1 is the
//           column-normalised R of Delta S to QR accuracy.
// The breakdown guard reads the accurate R^: the first column i >= 1 with
// R^_ii < 1e-6 is dependent on the previous ones (Krylov space exhausted,
// q' = i).  Then RRE: R^T R d = e; MPE or a dependent column: R_q d = -r_q,
// d_q = 1; gamma = d / sum d (with the lambda guard).
__device__ void reduce_gram(int nz, const double* __restrict__ partial, int nblocks, int np, double* G) {
    // one warp per Gram entry; lanes stride over the block partials in a fixed
    // order, then a fixed shuffle tree: deterministic.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int stride = np * (np + 1) / 2;
    for (int c = warp; c < nz * (nz + 1) / 2; c += nw) {
        int a = 0, cc = c;
        while (cc >= nz - a) { cc -= nz - a; ++a; }
        const int bcol = a + cc;
        int idx = 0;                                        // position in the np-column triangle
        for (int r = 0; r < a; ++r) idx += (np - r);
        idx += bcol - a;
        double s = 0.0;
        for (int blk = lane; blk < nblocks; blk += 32) s += partial[(size_t)blk * stride + idx];
        s = warp_sum(s);
        if (lane == 0) {
            G[a * nz + bcol] = s;
            G[bcol * nz + a] = s;
        }
    }
}

__device__ void set_fallback(int q, double* gamma, int* qused) {
    for (int i = 0; i < q + 2; ++i) gamma[i] = 0.0;
    gamma[q + 1] = 1.0;                                     // the last iterate
    *qused = -1;
}

__global__ void __launch_bounds__(kThreads) k_chol1(int q, const double* __restrict__ partial, int nblocks,
                                                     ExtrapInfo* __restrict__ info, double* __restrict__ gamma,
                                                     int* __restrict__ qused) {
    pdl_enter();
    const int n = q + 1;
    __shared__ double G[(kMaxQ + 1) * (kMaxQ + 1)];
    reduce_gram(n, partial, nblocks, n, G);
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double floor2 = 1e-15;                            // numerically zero pivot of G^
    double* D = info->D;
    double* R = info->R1h;
    for (int i = 0; i < q + 2; ++i) gamma[i] = 0.0;
    double Dinv[kMaxQ + 1], Rinv[kMaxQ + 1];
    for (int i = 0; i < n; ++i) {
        const double g = G[i * n + i];
        Dinv[i] = g > 0.0 ? rsqrt(g) : 0.0;
        D[i] = g * Dinv[i];
    }
    info->done = 1;
    if (!(D[0] > 0.0)) {                                    // Delta s_0 = 0: s_0 is a fixed point
        gamma[0] = 1.0;
        *qused = 0;
        return;
    }
    int a = n;
    for (int jc = 0; jc < n && a == n; ++jc) {
        if (!(D[jc] > 0.0)) { a = jc; break; }
        for (int i = 0; i < jc; ++i) {
            double s = G[i * n + jc] * Dinv[i] * Dinv[jc];
            for (int kk = 0; kk < i; ++kk) s -= R[kk * n + i] * R[kk * n + jc];
            R[i * n + jc] = s * Rinv[i];
        }
        double piv = 1.0;
        for (int kk = 0; kk < jc; ++kk) piv -= R[kk * n + jc] * R[kk * n + jc];
        if (jc >= 1 && piv < floor2) {
            a = jc;
        } else {
            Rinv[jc] = rsqrt(piv);
            R[jc * n + jc] = piv * Rinv[jc];
        }
    }
    for (int i = 0; i < a; ++i)
        for (int j = i; j < a; ++j) info->R1p[i * n + j] = R[i * n + j] * D[j];
    for (int j = 0; j < a; ++j) info->R1pinv[j] = Rinv[j] * Dinv[j];
    info->a = a;
    info->dep = a;                                          // pass 2 adds raw column a when a < n
    info->done = 0;
}

// Pass 2: Gram of Z = [Delta S_a (R1 D)^-1, Delta s_dep] formed element by element.
template <int Q>
__global__ void __launch_bounds__(kThreads) k_gram2_partial(const double* __restrict__ S, size_t ld, size_t n,
                                                             const ExtrapInfo* __restrict__ info,
                                                             double* __restrict__ partial) {
    pdl_enter();
    constexpr int NC = Q + 1, NP = NC * (NC + 1) / 2;
    if (info->done) return;
    __shared__ double Rp[NC * NC], Rinv[NC];
    const int a = info->a, dep = info->dep;
    for (int i = threadIdx.x; i < NC * NC; i += blockDim.x) Rp[i] = info->R1p[i];
    for (int i = threadIdx.x; i < NC; i += blockDim.x) Rinv[i] = info->R1pinv[i];
    __syncthreads();
    double acc[NP];
#pragma unroll
    for (int c = 0; c < NP; ++c) acc[c] = 0.0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double s[Q + 2];
#pragma unroll
        for (int j = 0; j < Q + 2; ++j) s[j] = S[(size_t)j * ld + e];
        double z[NC];
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            const double dj = s[j + 1] - s[j];
            double v = dj;
#pragma unroll
            for (int i = 0; i < j; ++i) v -= z[i] * Rp[i * NC + j];
            z[j] = (j < a) ? v * Rinv[j] : (j == dep ? dj : 0.0);   // dep == a here
        }
        int c = 0;
#pragma unroll
        for (int i = 0; i < NC; ++i)
#pragma unroll
            for (int j = i; j < NC; ++j) acc[c++] += z[i] * z[j];
    }
    __shared__ double red[kThreads / 32][NP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < NP; ++c) {
        const double v = warp_sum(acc[c]);
        if (lane == 0) red[w][c] = v;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < NP; c += blockDim.x) {
        double t = 0.0;
        for (int ww = 0; ww < (int)blockDim.x / 32; ++ww) t += red[ww][c];
        partial[(size_t)blockIdx.x * NP + c] = t;
    }
}

__global__ void __launch_bounds__(kThreads) k_gamma2(int q, int method, const double* __restrict__ partial,
                                                      int nblocks, const ExtrapInfo* __restrict__ info,
                                                      double* __restrict__ gamma, int* __restrict__ qused) {
    pdl_enter();
    if (info->done) return;
    const int n = q + 1;
    const int a = info->a, nz = a + (a < n ? 1 : 0);
    __shared__ double G2[(kMaxQ + 1) * (kMaxQ + 1)];
    reduce_gram(nz, partial, nblocks, n, G2);
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double tol = 1e-6;                                // breakdown guard on R^_ii
    const double* D = info->D;
    const double* R1 = info->R1h;
    double R2[(kMaxQ + 1) * (kMaxQ + 1)], Rh[(kMaxQ + 1) * (kMaxQ + 1)], d[kMaxQ + 2], y[kMaxQ + 1];
    double R2inv[kMaxQ + 1], Rhinv[kMaxQ + 1], Dinv[kMaxQ + 1];
    for (int i = 0; i < q + 2; ++i) gamma[i] = 0.0;
    for (int i = 0; i < n; ++i) Dinv[i] = D[i] > 0.0 ? 1.0 / D[i] : 0.0;
    // R2 = chol(G2[0:a, 0:a]) (upper, R2^T R2 = G2)
    for (int j = 0; j < a; ++j) {
        for (int i = 0; i < j; ++i) {
            double s = G2[i * nz + j];
            for (int kk = 0; kk < i; ++kk) s -= R2[kk * n + i] * R2[kk * n + j];
            R2[i * n + j] = s * R2inv[i];
        }
        double piv = G2[j * nz + j];
        for (int kk = 0; kk < j; ++kk) piv -= R2[kk * n + j] * R2[kk * n + j];
        if (!(piv > 0.0)) { set_fallback(q, gamma, qused); return; }
        R2inv[j] = rsqrt(piv);
        R2[j * n + j] = piv * R2inv[j];
    }
    // R^ = R2 R1 (upper triangular product, a x a)
    for (int i = 0; i < a; ++i)
        for (int j = i; j < a; ++j) {
            double s = 0.0;
            for (int kk = i; kk <= j; ++kk) s += R2[i * n + kk] * R1[kk * n + j];
            Rh[i * n + j] = s;
        }
    for (int i = 0; i < a; ++i) Rhinv[i] = 1.0 / Rh[i * n + i];
    int dep = n;
    for (int j = 1; j < a && dep == n; ++j)
        if (Rh[j * n + j] < tol) dep = j;
    if (dep == n && a < n) {
        dep = a;
        if (!(D[a] > 0.0)) {                                // zero difference: s_a is a fixed point
            gamma[a] = 1.0;
            *qused = a;
            return;
        }
    }
    int qq;
    if (dep < n || method == 2) {
        double r[kMaxQ + 1];
        qq = dep < n ? dep : q;
        if (dep < n && dep == a) {                          // raw column: r = R2^-T (W^T Delta s_a) / D_a
            for (int i = 0; i < a; ++i) {
                double s = G2[i * nz + a];
                for (int kk = 0; kk < i; ++kk) s -= R2[kk * n + i] * r[kk];
                r[i] = s * R2inv[i];
            }
            for (int i = 0; i < a; ++i) r[i] *= Dinv[a];
        } else {                                            // r_qq = R^[0:qq, qq]
            for (int i = 0; i < qq; ++i) r[i] = Rh[i * n + qq];
        }
        for (int i = qq - 1; i >= 0; --i) {                 // R^_qq y = -r
            double s = -r[i];
            for (int kk = i + 1; kk < qq; ++kk) s -= Rh[i * n + kk] * y[kk];
            y[i] = s * Rhinv[i];
        }
        for (int i = 0; i < qq; ++i) d[i] = y[i] * Dinv[i];
        d[qq] = Dinv[qq];
    } else {                                                // RRE: R^T R^ z = D^-1 e, d = z / D
        qq = q;
        double z[kMaxQ + 1];
        for (int i = 0; i < n; ++i) {
            double s = Dinv[i];
            for (int kk = 0; kk < i; ++kk) s -= Rh[kk * n + i] * z[kk];
            z[i] = s * Rhinv[i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = z[i];
            for (int kk = i + 1; kk < n; ++kk) s -= Rh[i * n + kk] * z[kk];
            z[i] = s * Rhinv[i];
        }
        for (int i = 0; i < n; ++i) d[i] = z[i] * Dinv[i];
    }
    double lam = 0.0, asum = 0.0;
    for (int i = 0; i <= qq; ++i) { lam += d[i]; asum += fabs(d[i]); }
    bool ok = isfinite(lam) && fabs(lam) > 1e-12 * asum;
    const double laminv = ok ? 1.0 / lam : 0.0;
    for (int i = 0; i <= qq && ok; ++i) {
        gamma[i] = d[i] * laminv;
        ok = isfinite(gamma[i]);
    }
    if (!ok) { set_fallback(q, gamma, qused); return; }
    *qused = qq;
}

__global__ void k_combine(int nS, const double* __restrict__ gamma, const double* __restrict__ S,
                          size_t ld, size_t n, double* __restrict__ t) {
    pdl_enter();
    __shared__ double g[kMaxQ + 2];
    for (int j = threadIdx.x; j < nS; j += blockDim.x) g[j] = gamma[j];
    __syncthreads();
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < nS; ++j)
            if (g[j] != 0.0) s += g[j] * S[(size_t)j * ld + i];
        t[i] = s;
    }
}

// ---------------------------------------------------------------- load vector
// b[k][j][i] = sum_{kz} gz[kz][k] sum_{ky} gy[ky][j] H[kz][ky][i] (2D: no kz),
// H = sum_kx c gx precomputed on the host (separable per sine mode).
__global__ void k_rhs_sine(int dim, int mx, int my, int mz, int modes, const double* __restrict__ H,
                           const double* __restrict__ gy, const double* __restrict__ gz,
                           double* __restrict__ b) {
    const size_t total = (size_t)mx * my * mz;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx % mx);
        const size_t t = idx / mx;
        const int j = (int)(t % my), k = (int)(t / my);
        double s = 0.0;
        if (dim == 2) {
            for (int ky = 0; ky < modes; ++ky) s += gy[(size_t)ky * my + j] * H[(size_t)ky * mx + i];
        } else {
            for (int kz = 0; kz < modes; ++kz) {
                double sy = 0.0;
                for (int ky = 0; ky < modes; ++ky)
                    sy += gy[(size_t)ky * my + j] * H[((size_t)kz * modes + ky) * mx + i];
                s += gz[(size_t)kz * mz + k] * sy;
            }
        }
        b[idx] = s;
    }
}

template <typename T>
__global__ void k_fill_zero(T* p, size_t n) {
    pdl_enter();
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p[i] = (T)0;
}

// ================================================================ launchers
static int grid_for(size_t n, int per = kThreads) {
    size_t g = (n + per - 1) / per;
    if (g > 152 * 16) g = 152 * 16;
    return (int)(g < 1 ? 1 : g);
}

// threads for a CTA that owns one row of length mx: the whole row in one pass
// where the kernel's register budget allows
static int row_threads(int mx, int cap) {
    int t = ((mx + 31) / 32) * 32;
    return t < 64 ? 64 : (t > cap ? cap : t);
}

// run f(integral_constant<int, P>) for the runtime degree p in [1, kMaxP]
template <typename F>
static void with_p(int p, F&& f) {
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

// Dynamic shared-memory limits are raised once per device by prepare_kernels()
// (cudaFuncSetAttribute is not allowed while a stream is being captured).
template <typename K>
static void set_smem(K, size_t) {}

template <typename K>
static void raise_smem(K kernel, int optin) {
    // the opt-in limit covers static plus dynamic shared memory
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

void prepare_kernels() {
    int dev = 0, optin = 48 * 1024;
    cudaGetDevice(&dev);
    static bool done[64] = {};
    if (dev < 0 || dev >= 64 || done[dev]) return;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    auto all_p = [&](auto T_tag) {
        using T = decltype(T_tag);
        for (int p = 1; p <= kMaxP; ++p)
            with_p(p, [&](auto PC) {
                constexpr int P = decltype(PC)::value;
                raise_smem(k_xpass<T, T, P>, optin);
                raise_smem(k_gs_phase2<T, P, gs_window<T, 2, P>()>, optin);
                raise_smem(k_gs_phase3<T, P, gs_window<T, 3, P>()>, optin);
                raise_smem(k_gs_sweep2<T, P, gs_window<T, 2, P>()>, optin);
                raise_smem(k_gs_sweep3<T, P, gs_window<T, 3, P>()>, optin);
                raise_smem(k_prolong_last<T, 2, P>, optin);
                raise_smem(k_prolong_last<T, 3, P>, optin);
                raise_smem(k_residual_restrict_x<T, P>, optin);
                raise_smem(k_prolong_fused2<T, P>, optin);
                raise_smem(k_jacobi2<T, P>, optin);
            });
        raise_smem(k_coarse_fd<T, 2>, optin);
        raise_smem(k_coarse_fd<T, 3>, optin);
    };
    all_p(0.0);
    all_p(0.0f);
    prepare_tail_kernels(optin);
    cnn_prepare();
    for (int p = 1; p <= kMaxP; ++p)
        with_p(p, [&](auto PC) { raise_smem(k_xpass<double, float, decltype(PC)::value>, optin); });
    cudaGetLastError();
    done[dev] = true;
}

template <typename T, typename A>
void xpass(cudaStream_t s, const LevelView<T>& L, const T* x, T* x_out, const A* add, int nS,
           const double* gamma, const T* S, size_t ldS, T* TM, T* TK) {
    const size_t smem = (size_t)(L.m[0] + 2 * L.p) * sizeof(T);
    with_p(L.p, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        set_smem(k_xpass<T, A, P>, smem);
        launch_chained(k_xpass<T, A, P>, L.rows(), kThreads, smem, s, L, x, x_out, add, nS, gamma, S, ldS, TM, TK);
    });
    count_launch();
}

// CTAs of a single-launch sweep: as many as fit on the device at once (more
// would only claim nothing and exit), at most one per row.
template <typename K>
static int resident_grid(K kernel, int threads, size_t smem, int rows) {
    int dev = 0, nsm = 1, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess || per < 1) per = 1;
    const long long g = (long long)per * nsm;
    return (int)(g < rows ? g : rows);
}

template <typename T>
void gs_sweep(cudaStream_t s, int dim, const LevelView<T>& L, bool descending, T* x, const T* b,
              T* TM, T* TK, int cap, const SweepSync* sy) {
    const int p = L.p, P1 = p + 1;
    const size_t smem = (size_t)6 * L.m[0] * sizeof(T);
    const int most = dim == 3 ? row_cta_max<T, 3>() : row_cta_max<T, 2>();
    const int threads = row_threads(L.m[0], (cap >= 64 && cap < most) ? cap : most);
    if (sy) {
        const int rows = L.rows();
        with_p(p, [&](auto PC) {
            constexpr int P = decltype(PC)::value;
            if (dim == 2) {
                constexpr bool WIN = gs_window<T, 2, P>();
                const int grid = resident_grid(k_gs_sweep2<T, P, WIN>, threads, smem, rows);
                launch_chained(k_gs_sweep2<T, P, WIN>, grid, threads, smem, s, L, (int)descending, x, b, TM, TK, *sy);
            } else {
                constexpr bool WIN = gs_window<T, 3, P>();
                const int grid = resident_grid(k_gs_sweep3<T, P, WIN>, threads, smem, rows);
                launch_chained(k_gs_sweep3<T, P, WIN>, grid, threads, smem, s, L, (int)descending, x, b, TM, TK, *sy);
            }
        });
        count_launch();
        return;
    }
    auto launch = [&](int cy, int cz) {
        const int nty = (L.m[1] - cy + p) / P1;
        const int ntz = (dim == 3) ? (L.m[2] - cz + p) / P1 : 1;
        if (nty <= 0 || ntz <= 0) return;
        with_p(p, [&](auto PC) {
            constexpr int P = decltype(PC)::value;
            if (dim == 2) {
                constexpr bool WIN = gs_window<T, 2, P>();
                set_smem(k_gs_phase2<T, P, WIN>, smem);
                launch_chained(k_gs_phase2<T, P, WIN>, nty * ntz, threads, smem, s, L, cy, cz, descending, x, b, TM, TK);
            } else {
                constexpr bool WIN = gs_window<T, 3, P>();
                set_smem(k_gs_phase3<T, P, WIN>, smem);
                launch_chained(k_gs_phase3<T, P, WIN>, nty * ntz, threads, smem, s, L, cy, cz, descending, x, b, TM, TK);
            }
        });
        count_launch();
    };
    const int ncz = (dim == 3) ? P1 : 1;
    for (int c = 0; c < P1 * ncz; ++c) {
        const int cc = descending ? P1 * ncz - 1 - c : c;
        launch(cc % P1, cc / P1);
    }
}

template <typename T, typename R>
void residual(cudaStream_t s, int dim, const LevelView<T>& L, const T* b, const T* TM, const T* TK,
              R* r, double* partial, double* r64, T* u, T* v) {
    with_p(L.p, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        if (dim == 2) {
            launch_chained(k_residual<T, R, 2, P>, L.rows(), kThreads, 0, s, L, b, TM, TK, r, partial, r64);
        } else if (u && v) {                         // sum-factorised across y and z
            launch_chained(k_yfactor3<T, P>, L.rows(), kThreads, 0, s, L, TM, TK, u, v);
            launch_chained(k_zresidual3<T, R, P>, L.rows(), kThreads, 0, s, L, b, (const T*)u, (const T*)v, r,
                           partial, r64);
            count_launch();
        } else {
            launch_chained(k_residual<T, R, 3, P>, L.rows(), kThreads, 0, s, L, b, TM, TK, r, partial, r64);
        }
    });
    count_launch();
}

template <typename T>
void jacobi_sweep(cudaStream_t s, int dim, const LevelView<T>& L, T omega, T* x, const T* b, T* TM, T* TK,
                  T* TMo, T* TKo) {
    if (dim == 2) {
        const size_t smem = (size_t)(L.m[0] + 2 * L.p) * sizeof(T);
        with_p(L.p, [&](auto PC) {
            constexpr int P = decltype(PC)::value;
            set_smem(k_jacobi2<T, P>, smem);
            launch_chained(k_jacobi2<T, P>, L.m[1], kThreads, smem, s, L, omega, b, TM, TK, x, TMo, TKo);
        });
        count_launch();
        return;
    }
    with_p(L.p, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        launch_chained(k_jacobi<T, 3, P>, L.rows(), kThreads, 0, s, L, omega, b, TM, TK, x);
    });
    count_launch();
    xpass<T, T>(s, L, x, x, nullptr, 0, nullptr, nullptr, 0, TM, TK);
}

template <typename T>
void restrict_(cudaStream_t s, int dim, const TransferView<T>& X, const T* fine, T* coarse, T* tmp1,
               T* tmp2, T* zero, size_t nzero) {
    // axis by axis: x, then y (then z); dims shrink one axis at a time
    int d[3] = {X.mf[0], X.mf[1], dim == 3 ? X.mf[2] : 1};
    const T* in = fine;
    for (int a = 0; a < dim; ++a) {
        const int n_in = d[a];
        d[a] = X.mc[a];
        T* out = (a == dim - 1) ? coarse : (a == 0 ? tmp1 : tmp2);
        const size_t total = (size_t)d[0] * d[1] * d[2];
        launch_chained(k_transfer_axis<T>, grid_for(total), kThreads, 0, s, in, out, d[0], d[1], d[2], a, n_in,
                                                                X.rlo[a], X.rv[a], X.rw[a],
                                                                a == dim - 1 ? zero : nullptr,
                                                                a == dim - 1 ? nzero : 0);
        count_launch();
        in = out;
    }
}

template <typename T>
void residual_restrict(cudaStream_t s, int dim, const LevelView<T>& L, const TransferView<T>& X, const T* b,
                       const T* TM, const T* TK, T* r, T* coarse, T* tmp1, T* tmp2, T* zero, size_t nzero) {
    if (dim != 2) {
        residual<T, T>(s, dim, L, b, TM, TK, r, nullptr, nullptr, tmp1, tmp2);
        restrict_<T>(s, dim, X, r, coarse, tmp1, tmp2, zero, nzero);
        return;
    }
    const size_t smem = (size_t)L.m[0] * sizeof(T);
    with_p(L.p, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        launch_chained(k_residual_restrict_x<T, P>, L.m[1], kThreads, smem, s, L, b, TM, TK, X.mc[0], X.rlo[0], X.rv[0],
                                                                   X.rw[0], tmp1);
    });
    count_launch();
    const size_t total = (size_t)X.mc[0] * X.mc[1];
    launch_chained(k_transfer_axis<T>, grid_for(total), kThreads, 0, s, tmp1, coarse, X.mc[0], X.mc[1], 1, 1, X.mf[1],
                                                            X.rlo[1], X.rv[1], X.rw[1], zero, nzero);
    count_launch();
}

template <typename T>
void prolong_add(cudaStream_t s, int dim, const TransferView<T>& X, const LevelView<T>& Lf, const T* e,
                 T* x, T* TM, T* TK, T* tmp1, T* tmp2) {
    if (dim == 2) {
        // FP32 cycles stage the coarse rows when they fit comfortably next to
        // the fine row (1024^2, p = 3: 10.79 -> 10.65 ms per FP32-IR solve);
        // in FP64 the larger CTA footprint cost 1% (22.33 -> 22.57 ms)
        const size_t row = (size_t)(Lf.m[0] + 2 * Lf.p) * sizeof(T);
        const size_t rows_c = (size_t)X.pw[1] * X.mc[0] * sizeof(T);
        const int staged = sizeof(T) == 4 && row + rows_c <= 96 * 1024;
        const size_t smem = staged ? row + rows_c : row;
        with_p(Lf.p, [&](auto PC) {
            constexpr int P = decltype(PC)::value;
            launch_chained(k_prolong_fused2<T, P>, Lf.m[1], kThreads, smem, s, Lf, e, X.mc[0], X.mc[1], X.plo[0], X.pv[0],
                           X.pw[0], X.plo[1], X.pv[1], X.pw[1], x, TM, TK, staged);
        });
        count_launch();
        return;
    }
    int d[3] = {X.mc[0], X.mc[1], dim == 3 ? X.mc[2] : 1};
    const T* in = e;
    for (int a = 0; a < dim - 1; ++a) {
        const int n_in = d[a];
        d[a] = X.mf[a];
        T* out = (a == 0) ? tmp1 : tmp2;
        const size_t total = (size_t)d[0] * d[1] * d[2];
        launch_chained(k_transfer_axis<T>, grid_for(total), kThreads, 0, s, in, out, d[0], d[1], d[2], a, n_in,
                                                                X.plo[a], X.pv[a], X.pw[a], nullptr, 0);
        count_launch();
        in = out;
    }
    const int a = dim - 1;
    const size_t smem = (size_t)(Lf.m[0] + 2 * Lf.p) * sizeof(T);
    with_p(Lf.p, [&](auto PC) {
        constexpr int P = decltype(PC)::value;
        if (dim == 2) {
            set_smem(k_prolong_last<T, 2, P>, smem);
            launch_chained(k_prolong_last<T, 2, P>, Lf.rows(), kThreads, smem, s, Lf, in, X.mc[a], X.plo[a], X.pv[a], X.pw[a], x, TM, TK);
        } else {
            set_smem(k_prolong_last<T, 3, P>, smem);
            launch_chained(k_prolong_last<T, 3, P>, Lf.rows(), kThreads, smem, s, Lf, in, X.mc[a], X.plo[a], X.pv[a], X.pw[a], x, TM, TK);
        }
    });
    count_launch();
}

template <typename T>
void coarse_solve(cudaStream_t s, int dim, const CoarseView<T>& C, const T* r, T* e) {
    const int N = C.m[0] * C.m[1] * (dim == 3 ? C.m[2] : 1);
    const size_t smem = (size_t)2 * N * sizeof(T);
    if (dim == 2) {
        set_smem(k_coarse_fd<T, 2>, smem);
        launch_chained(k_coarse_fd<T, 2>, 1, kThreads, smem, s, C, r, e);
    } else {
        set_smem(k_coarse_fd<T, 3>, smem);
        launch_chained(k_coarse_fd<T, 3>, 1, kThreads, smem, s, C, r, e);
    }
    count_launch();
}

void sumsq_partial(cudaStream_t s, const double* v, size_t n, double* partial, int nblocks) {
    launch_chained(k_sumsq, nblocks, kThreads, 0, s, v, n, partial);
    count_launch();
}

void diff_sumsq(cudaStream_t s, const double* u, const double* v, size_t n, double* e, double* partial,
                int nblocks) {
    launch_chained(k_diff_sumsq, nblocks, kThreads, 0, s, u, v, n, e, partial);
    count_launch();
}

void scale_pair(cudaStream_t s, const double* r, const double* e, const double* enorm, size_t n, float* R, float* E) {
    launch_chained(k_scale_pair, grid_for(n), kThreads, 0, s, r, e, enorm, n, R, E);
    count_launch();
}

void loop_step(cudaStream_t s, cudaGraphConditionalHandle h, LoopState* st, const double* res,
               const unsigned* err, double* hist) {
    launch_chained(k_loop_step, 1, 32, 0, s, h, st, res, err, hist);
    count_launch();
}

void loop_init(cudaStream_t s, cudaGraphConditionalHandle h, const LoopState* st) {
    launch_chained(k_loop_init, 1, 32, 0, s, h, st);
    count_launch();
}

cudaError_t add_loop_init_node(cudaGraph_t g, cudaGraphConditionalHandle h, const LoopState* st,
                               cudaGraphNode_t* node) {
    void* args[2] = {&h, &st};
    cudaKernelNodeParams kp = {};
    kp.func = (void*)k_loop_init;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(32);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    kp.extra = nullptr;
    return cudaGraphAddKernelNode(node, g, nullptr, 0, &kp);
}

void norm_final(cudaStream_t s, const double* partial, int nparts, const double* denom, double* out,
                int slot) {
    launch_chained(k_norm_final, 1, 1024, 0, s, partial, nparts, denom, out, slot);
    count_launch();
}

int gram_blocks(size_t n) {
    size_t g = (n + kThreads - 1) / kThreads;
    if (g > 2 * 152) g = 2 * 152;
    return (int)(g < 1 ? 1 : g);
}

void gram_partial(cudaStream_t s, int q, const double* S, size_t ld, size_t n, double* partial, int nblocks) {
    switch (q) {
#define IGAMG_GRAM_CASE(Q) \
    case Q: launch_chained(k_gram_partial<Q>, nblocks, kThreads, 0, s, S, ld, n, partial); break;
        IGAMG_GRAM_CASE(1) IGAMG_GRAM_CASE(2) IGAMG_GRAM_CASE(3) IGAMG_GRAM_CASE(4)
        IGAMG_GRAM_CASE(5) IGAMG_GRAM_CASE(6) IGAMG_GRAM_CASE(7) IGAMG_GRAM_CASE(8)
        IGAMG_GRAM_CASE(9) IGAMG_GRAM_CASE(10) IGAMG_GRAM_CASE(11) IGAMG_GRAM_CASE(12)
#undef IGAMG_GRAM_CASE
        default: return;
    }
    count_launch();
}

void extrap_gammas(cudaStream_t s, int q, int method, const double* S, size_t ld, size_t n,
                   double* partial, int nblocks, ExtrapInfo* info, double* gamma, int* qused) {
    gram_partial(s, q, S, ld, n, partial, nblocks);
    launch_chained(k_chol1, 1, kThreads, 0, s, q, partial, nblocks, info, gamma, qused);
    count_launch();
    switch (q) {
#define IGAMG_GRAM2_CASE(Q) \
    case Q: launch_chained(k_gram2_partial<Q>, nblocks, kThreads, 0, s, S, ld, n, info, partial); break;
        IGAMG_GRAM2_CASE(1) IGAMG_GRAM2_CASE(2) IGAMG_GRAM2_CASE(3) IGAMG_GRAM2_CASE(4)
        IGAMG_GRAM2_CASE(5) IGAMG_GRAM2_CASE(6) IGAMG_GRAM2_CASE(7) IGAMG_GRAM2_CASE(8)
        IGAMG_GRAM2_CASE(9) IGAMG_GRAM2_CASE(10) IGAMG_GRAM2_CASE(11) IGAMG_GRAM2_CASE(12)
#undef IGAMG_GRAM2_CASE
        default: return;
    }
    count_launch();
    launch_chained(k_gamma2, 1, kThreads, 0, s, q, method, partial, nblocks, info, gamma, qused);
    count_launch();
}

void combine(cudaStream_t s, int q, const double* gamma, const double* S, size_t ld, size_t n, double* t) {
    launch_chained(k_combine, grid_for(n), kThreads, 0, s, q + 2, gamma, S, ld, n, t);
    count_launch();
}

void rhs_sine(cudaStream_t s, int dim, const int* m, int modes, const double* H, const double* gy,
              const double* gz, double* b) {
    const size_t total = (size_t)m[0] * m[1] * (dim == 3 ? m[2] : 1);
    k_rhs_sine<<<grid_for(total), kThreads, 0, s>>>(dim, m[0], m[1], dim == 3 ? m[2] : 1, modes, H, gy, gz, b);
    count_launch();
}

template <typename T>
void fill_zero(cudaStream_t s, T* p, size_t n) {
    launch_chained(k_fill_zero<T>, grid_for(n), kThreads, 0, s, p, n);
    count_launch();
}

// explicit instantiations
#define IGAMG_INST(T)                                                                               \
    template void xpass<T, T>(cudaStream_t, const LevelView<T>&, const T*, T*, const T*, int,       \
                              const double*, const T*, size_t, T*, T*);                             \
    template void gs_sweep<T>(cudaStream_t, int, const LevelView<T>&, bool, T*, const T*, T*, T*, int,   \
                              const SweepSync*);                                                     \
    template void jacobi_sweep<T>(cudaStream_t, int, const LevelView<T>&, T, T*, const T*, T*, T*, T*, T*);  \
    template void restrict_<T>(cudaStream_t, int, const TransferView<T>&, const T*, T*, T*, T*, T*, size_t);  \
    template void residual_restrict<T>(cudaStream_t, int, const LevelView<T>&, const TransferView<T>&,    \
                                       const T*, const T*, const T*, T*, T*, T*, T*, T*, size_t);         \
    template void prolong_add<T>(cudaStream_t, int, const TransferView<T>&, const LevelView<T>&,    \
                                 const T*, T*, T*, T*, T*, T*);                                     \
    template void coarse_solve<T>(cudaStream_t, int, const CoarseView<T>&, const T*, T*);          \
    template void fill_zero<T>(cudaStream_t, T*, size_t);
IGAMG_INST(double)
IGAMG_INST(float)
#undef IGAMG_INST
template void xpass<double, float>(cudaStream_t, const LevelView<double>&, const double*, double*,
                                   const float*, int, const double*, const double*, size_t, double*,
                                   double*);
template void residual<double, double>(cudaStream_t, int, const LevelView<double>&, const double*,
                                       const double*, const double*, double*, double*, double*, double*,
                                       double*);
template void residual<double, float>(cudaStream_t, int, const LevelView<double>&, const double*,
                                      const double*, const double*, float*, double*, double*, double*,
                                      double*);
template void residual<float, float>(cudaStream_t, int, const LevelView<float>&, const float*,
                                     const float*, const float*, float*, double*, double*, float*, float*);

}  // namespace dev
}  // namespace igamg
