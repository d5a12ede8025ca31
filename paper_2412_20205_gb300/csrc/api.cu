// C ABI of the solver: context, set-up/upload, workspace layout, the V-cycle
// sequencer (Algorithm 2, mu = 1) and the restarted extrapolation loop
// (Algorithm 5 with Algorithms 3-4), replayed as a CUDA graph per restart.
#include "../../include/igamg.h"
#include "device.hpp"
#include "host_setup.hpp"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

using namespace igamg;

namespace {

thread_local std::string g_err;

igamg_status fail(igamg_status st, const std::string& msg) {
    g_err = msg;
    return st;
}

#define CUDA_TRY(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(IGAMG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

struct HostLevel {
    int m[3] = {1, 1, 1};
    std::vector<double> breaks[3];
    Factor1D f[3];
    // prolongation from the next coarser level (empty on level 0)
    std::vector<double> P[3];
    int pmf[3] = {0, 0, 0}, pmc[3] = {0, 0, 0};
    std::vector<int> plo[3], rlo[3];
    std::vector<double> pv[3], rv[3];
    int pw[3] = {0, 0, 0}, rw[3] = {0, 0, 0};
    size_t N() const { return (size_t)m[0] * m[1] * m[2]; }
};

// Bump allocator over a device buffer (base == nullptr: size query only).
struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base((char*)b) {}
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? (T*)(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

template <typename T>
struct LevelBuf {
    T* x = nullptr;   // x, TM, TK contiguous (zeroed together)
    T* TM = nullptr;
    T* TK = nullptr;
    T* b = nullptr;
    T* r = nullptr;
    T* tmp1 = nullptr;
    T* tmp2 = nullptr;
};

struct Workspace {
    std::vector<LevelBuf<double>> d;
    std::vector<LevelBuf<float>> f;
    double* S = nullptr;      // k+2 iterates, stride ld
    size_t ld = 0;
    double* partial = nullptr;
    size_t npartial = 0;
    double* gamma = nullptr;
    int* qused = nullptr;
    ExtrapInfo* info = nullptr;
    double* scal = nullptr;   // [0] ||b||, [1] last residual norm, [2..] spare
    void* cnn = nullptr;      // network workspace (learned post-smoother)
    // synchronisation words of the single-launch GS sweeps: per level the row
    // flags and two counters, then the error word and a word nothing sets;
    // cleared when a call takes the workspace into use (every sweep leaves
    // them zero)
    unsigned* sync = nullptr;
    size_t nsync = 0;
    std::vector<unsigned*> done, ctr;
    unsigned* err = nullptr;
    unsigned* never = nullptr;
    LoopState* loop = nullptr;   // device-side restart loop: state and residual history
    double* hist = nullptr;
    size_t bytes = 0;
};

}  // namespace

void igamg::set_last_error(const char* msg) { g_err = msg; }

// Default row threshold of one-launch GS sweeps on 3D levels (igamg_ctx::flow32).
constexpr int kFlowRows3D = 8192;

struct igamg_ctx {
    int dim = 2, p = 1, L = 1;
    std::vector<HostLevel> hl;
    std::vector<double> cV[3], claminv;     // coarsest fast diagonalisation (host)
    bool assembled = false;
    void* dmem = nullptr;
    std::vector<LevelView<double>> lv64;
    std::vector<LevelView<float>> lv32;
    std::vector<TransferView<double>> tv64;
    std::vector<TransferView<float>> tv32;
    CoarseView<double> cv64{};
    CoarseView<float> cv32{};
    // coarse levels of the FP32 2D V-cycle in one CTA (tail32.lc = 0: none);
    // tails[l] covers levels 0..l for every feasible l (tails[0] unused)
    TailView<float> tail32{};
    std::vector<TailView<float>> tails;
    bool tail_on = true;
    // the same on a thread-block cluster (ctail32, when tail_ctas > 1);
    // ctails[k][l] covers levels 0..l on kTailCtas[k] CTAs
    int tail_ctas = 1;
    bool tune_clusters = true;              // igamg_autotune tries the cluster tails
    ClusterTailView<float> ctail32{};
    std::vector<ClusterTailView<float>> ctails[2];
    // 3D: the cluster tail of FP32 cycles (ClusterTail3View)
    ClusterTail3View<float> ctail3{};
    std::vector<ClusterTail3View<float>> ctails3[2];
    int gs_cap32 = 0;                       // row-CTA thread cap of FP32 GS (0: default)
    // GS sweep form per precision: levels with at least this many rows run a
    // sweep in one launch (rows wait on their earlier-phase neighbours), the
    // others one launch per row phase.  Measured on GB300: one launch won
    // where a sweep has many rows per phase (3D 128^3 finest level, 16641
    // rows: 185 us against 828 us per FP32 sweep) and lost where the phase
    // chain's latency dominates (2D 1024^2: 49 against 34 us; 3D 64^3, 4225
    // rows: 185 against 142 us).  kNever: never.
    static constexpr int kNever = 1 << 30;
    int flow32 = kNever, flow64 = kNever;
    // cycle of Algorithm 2: smoother (IGAMG_SMOOTH_GS / IGAMG_SMOOTH_JACOBI),
    // mu = 1 (V-cycle) or 2 (W-cycle), Jacobi weight
    int smoother = 0, mu = 1;
    double omega = 2.0 / 3.0;
    DFView dfv{};                           // finest 2D factors as float pairs
    // sine-moment tables for the load vector (finest level)
    cudaStream_t cap = nullptr;             // capture stream
    double* h_pin = nullptr;                // pinned host scalars
    // restart-cycle graphs, one slot per precision form (igamg_prec), so that
    // alternating forms do not recapture
    cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};
    long long exec_launches[3] = {0, 0, 0};
    struct Key {
        const void* b = nullptr;
        const void* ws = nullptr;
        int k = -1, extrap = -1, prec = -1, abs_tol = -1, overlap = -1, sync = -1;
        const void* w = nullptr;
        bool operator==(const Key& o) const {
            return b == o.b && ws == o.ws && k == o.k && extrap == o.extrap && prec == o.prec &&
                   abs_tol == o.abs_tol && overlap == o.overlap && sync == o.sync && w == o.w;
        }
    } key[3];
    // device-side restart loops (a conditional WHILE node around one restart
    // cycle), one per precision form, keyed like exec[]; body_launches =
    // kernels per cycle; h_loop / h_hist: pinned staging of state and history
    cudaGraphExec_t loop_exec[3] = {nullptr, nullptr, nullptr};
    long long loop_body_launches[3] = {0, 0, 0};
    Key loop_key[3];
    LoopState* h_loop = nullptr;
    double* h_hist = nullptr;
    // general operator of Sec. 4.3 (igamg_setup_general): quadrature data of
    // the finest level, |J| at its points, and per level the stencil
    // operator (device memory gmem, views sv) and the coarsest dense inverse
    bool general = false, gen_ready = false;
    Quad1D gqx, gqy;
    std::vector<double> gdet;
    void* gmem = nullptr;
    std::vector<StencilView> sv;
    double* A0inv = nullptr;
    int n0 = 0;
    // learned post-smoother: caller-owned device weights, stall ratio, outcome
    const float* cnn_w = nullptr;
    double stall = 0.9;
    int fell_back = 0;
};

namespace {

size_t finestN(const igamg_ctx* c) { return c->hl.back().N(); }
size_t lv64_n(const igamg_ctx* c, int l) { return c->hl[l].N(); }

Workspace carve(const igamg_ctx* c, void* base, int k, int prec) {
    Workspace w;
    Carver cv(base);
    const int L = c->L;
    w.d.resize(L);
    for (int l = 0; l < L; ++l) {
        const size_t N = c->hl[l].N();
        LevelBuf<double>& B = w.d[l];
        B.x = cv.take<double>(3 * N);
        if (B.x) { B.TM = B.x + N; B.TK = B.x + 2 * N; }
        B.b = cv.take<double>(N);
        B.r = cv.take<double>(N);
        B.tmp1 = cv.take<double>(N);
        B.tmp2 = cv.take<double>(N);
    }
    if (prec == IGAMG_FP32_IR || prec == IGAMG_FP32_IR_LEARNED) {
        w.f.resize(L);
        for (int l = 0; l < L; ++l) {
            const size_t N = c->hl[l].N();
            LevelBuf<float>& B = w.f[l];
            B.x = cv.take<float>(3 * N);
            if (B.x) { B.TM = B.x + N; B.TK = B.x + 2 * N; }
            B.b = cv.take<float>(N);
            B.r = cv.take<float>(N);
            B.tmp1 = cv.take<float>(N);
            B.tmp2 = cv.take<float>(N);
        }
    }
    const size_t N = finestN(c);
    w.ld = (N + 31) & ~(size_t)31;
    w.S = cv.take<double>(w.ld * (size_t)(k + 2));
    const size_t rows = (size_t)c->hl.back().m[1] * c->hl.back().m[2];
    const size_t np = (size_t)(kMaxQ + 1) * (kMaxQ + 2) / 2;
    w.npartial = std::max(rows, (size_t)dev::gram_blocks(N) * np);
    w.npartial = std::max(w.npartial, (size_t)1024);
    w.partial = cv.take<double>(w.npartial);
    w.gamma = cv.take<double>(kMaxQ + 2);
    w.qused = cv.take<int>(4);
    w.info = cv.take<ExtrapInfo>(1);
    w.scal = cv.take<double>(8);
    w.loop = cv.take<LoopState>(1);
    w.hist = cv.take<double>(kLoopHist);
    w.nsync = 2;
    for (int l = 0; l < L; ++l) w.nsync += 2 + (size_t)c->hl[l].m[1] * c->hl[l].m[2];
    w.sync = cv.take<unsigned>(w.nsync);
    w.done.resize(L);
    w.ctr.resize(L);
    if (w.sync) {
        unsigned* q = w.sync;
        w.err = q++;
        w.never = q++;
        for (int l = 0; l < L; ++l) {
            w.ctr[l] = q;
            w.done[l] = q + 2;
            q += 2 + (size_t)c->hl[l].m[1] * c->hl[l].m[2];
        }
    }
    if (prec == IGAMG_FP32_IR_LEARNED)
        w.cnn = cv.take<unsigned char>(cnn_workspace_bytes((long long)finestN(c)));
    w.bytes = cv.off + 256;
    return w;
}

void compact_transfer(HostLevel& H, int d) {
    const int mf = H.pmf[d], mc = H.pmc[d];
    const std::vector<double>& P = H.P[d];
    H.plo[d].assign(mf, 0);
    H.rlo[d].assign(mc, 0);
    int pw = 1, rw = 1;
    std::vector<int> phi(mf, 0), rhi(mc, 0);
    for (int i = 0; i < mf; ++i) {
        int lo = -1, hi = -1;
        for (int J = 0; J < mc; ++J)
            if (P[(size_t)i * mc + J] != 0.0) { if (lo < 0) lo = J; hi = J; }
        if (lo < 0) { lo = 0; hi = 0; }
        H.plo[d][i] = lo;
        phi[i] = hi;
        pw = std::max(pw, hi - lo + 1);
    }
    for (int J = 0; J < mc; ++J) {
        int lo = -1, hi = -1;
        for (int i = 0; i < mf; ++i)
            if (P[(size_t)i * mc + J] != 0.0) { if (lo < 0) lo = i; hi = i; }
        if (lo < 0) { lo = 0; hi = 0; }
        H.rlo[d][J] = lo;
        rhi[J] = hi;
        rw = std::max(rw, hi - lo + 1);
    }
    H.pw[d] = pw;
    H.rw[d] = rw;
    H.pv[d].assign((size_t)mf * pw, 0.0);
    H.rv[d].assign((size_t)mc * rw, 0.0);
    for (int i = 0; i < mf; ++i)
        for (int s = 0; s < pw; ++s) {
            const int J = H.plo[d][i] + s;
            if (J < mc) H.pv[d][(size_t)i * pw + s] = P[(size_t)i * mc + J];
        }
    for (int J = 0; J < mc; ++J)
        for (int s = 0; s < rw; ++s) {
            const int i = H.rlo[d][J] + s;
            if (i < mf) H.rv[d][(size_t)J * rw + s] = P[(size_t)i * mc + J];
        }
}

// Rows of the x-band equal (to 1e-14 relative) to the middle row's band form
// the Toeplitz interior [lo, hi); returns the middle row index.
int toeplitz_range(const Factor1D& f, int* lo, int* hi) {
    const int m = f.m, bw = 2 * f.p + 1, mid = m / 2;
    double scale = 0.0;
    for (int b = 0; b < bw; ++b)
        scale = std::max(scale, std::max(std::fabs(f.M[(size_t)mid * bw + b]), std::fabs(f.K[(size_t)mid * bw + b])));
    auto same = [&](int i) {
        for (int b = 0; b < bw; ++b) {
            if (std::fabs(f.M[(size_t)i * bw + b] - f.M[(size_t)mid * bw + b]) > 1e-14 * scale) return false;
            if (std::fabs(f.K[(size_t)i * bw + b] - f.K[(size_t)mid * bw + b]) > 1e-14 * scale) return false;
        }
        return true;
    };
    int l = mid, h = mid + 1;
    while (l > 0 && same(l - 1)) --l;
    while (h < m && same(h)) ++h;
    *lo = l;
    *hi = h;
    return mid;
}

template <typename T>
std::vector<T> band_major(const Factor1D& f, bool stiff) {
    const int m = f.m, bw = 2 * f.p + 1;
    std::vector<T> out((size_t)bw * m);
    const std::vector<double>& src = stiff ? f.K : f.M;
    for (int i = 0; i < m; ++i)
        for (int b = 0; b < bw; ++b) out[(size_t)b * m + i] = (T)src[(size_t)i * bw + b];
    return out;
}

// ------------------------------------------------------------ V-cycle sequencer
template <typename T>
struct Views;
template <>
struct Views<double> {
    static const std::vector<LevelView<double>>& lv(const igamg_ctx* c) { return c->lv64; }
    static const std::vector<TransferView<double>>& tv(const igamg_ctx* c) { return c->tv64; }
    static const CoarseView<double>& cv(const igamg_ctx* c) { return c->cv64; }
    static std::vector<LevelBuf<double>>& buf(Workspace& w) { return w.d; }
};
template <>
struct Views<float> {
    static const std::vector<LevelView<float>>& lv(const igamg_ctx* c) { return c->lv32; }
    static const std::vector<TransferView<float>>& tv(const igamg_ctx* c) { return c->tv32; }
    static const CoarseView<float>& cv(const igamg_ctx* c) { return c->cv32; }
    static std::vector<LevelBuf<float>>& buf(Workspace& w) { return w.f; }
};

// CTAs of the cluster-tail variants built at assembly.
constexpr int kTailCtas[2] = {8, 16};

// Highest level of the active coarse tail of FP32 2D cycles (0: none).
int tail_level(const igamg_ctx* c) {
    if (!c->tail_on) return 0;
    if (c->dim == 3) return c->tail_ctas > 1 ? c->ctail3.lc : 0;
    return c->tail_ctas > 1 ? c->ctail32.lc : c->tail32.lc;
}

// Highest tail level available with `ctas` CTAs (1: the one-CTA tail).
int tail_most(const igamg_ctx* c, int ctas) {
    if (ctas == 1) return c->dim == 3 ? 0 : std::max(0, (int)c->tails.size() - 1);
    for (int k = 0; k < 2; ++k)
        if (kTailCtas[k] == ctas)
            return std::max(0, (int)(c->dim == 3 ? c->ctails3[k].size() : c->ctails[k].size()) - 1);
    return 0;
}

// The static shared-memory image of a 2D cluster-tail view, built on first
// use into device memory the context owns; false if it could not be.
template <typename View>
bool ensure_tail_image(View& v) {
    if (v.img) return true;
    uint4* img = nullptr;
    if (cudaMalloc(&img, (size_t)v.ctas * v.img16 * sizeof(uint4)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaError_t err;
    if constexpr (std::is_same_v<View, ClusterTail3View<float>>) err = dev::cluster_tail3_image(v, img);
    else err = dev::cluster_tail_image(v, img);
    if (err != cudaSuccess) {
        cudaGetLastError();
        cudaFree(img);
        return false;
    }
    v.img = img;
    return true;
}

void free_tail_images(igamg_ctx* c) {
    auto drop = [](auto& v) {
        if (v.img) cudaFree(const_cast<uint4*>(v.img));
        v.img = nullptr;
    };
    for (auto& vs : c->ctails)
        for (auto& v : vs) drop(v);
    for (auto& vs : c->ctails3)
        for (auto& v : vs) drop(v);
}

// Selects the tail on `ctas` CTAs over levels 0..lc (lc = 0: no tail).
void select_tail(igamg_ctx* c, int ctas, int lc) {
    lc = std::max(0, std::min(lc, tail_most(c, ctas)));
    c->tail_ctas = ctas;
    c->tail_on = lc > 0;
    if (lc == 0) return;
    if (ctas == 1) c->tail32 = c->tails[lc];
    else
        for (int k = 0; k < 2; ++k)
            if (kTailCtas[k] == ctas) {
                if (c->dim == 3 ? ensure_tail_image(c->ctails3[k][lc]) : ensure_tail_image(c->ctails[k][lc])) {
                    if (c->dim == 3) c->ctail3 = c->ctails3[k][lc];
                    else c->ctail32 = c->ctails[k][lc];
                } else {                                 // no image: the one-CTA tail (2D), else none
                    c->tail_ctas = 1;
                    lc = tail_most(c, 1);
                    c->tail_on = lc > 0;
                    if (c->tail_on) c->tail32 = c->tails[lc];
                }
            }
}

// Levels tail_level(c)..0 of an FP32 2D V-cycle from x = 0 in the active tail.
void run_tail(const igamg_ctx* c, cudaStream_t s, const float* b, float* x, int jacobi = 0, float omega = 0.f) {
    if (c->dim == 3) dev::cluster_tail3<float>(s, c->ctail3, b, x, jacobi, omega);
    else if (c->tail_ctas > 1) dev::cluster_tail<float>(s, c->ctail32, b, x, jacobi, omega);
    else dev::coarse_tail<float>(s, c->tail32, b, x, jacobi, omega);
}

// Cluster-tail views of a 3D hierarchy (ClusterTail3View): out[k][l] covers
// levels 0..l on kTailCtas[k] CTAs (out[k][0] unused).  Offsets in floats;
// integer tables take one element each, pointers two (the pointer tables come
// first, 8-byte aligned).
void build_cluster_tails3(const igamg_ctx* c, std::vector<ClusterTail3View<float>>* out) {
    const int p = c->p, W = 2 * p + 1, W2 = W * W, L = c->L;
    const int N0 = (int)c->hl[0].N();
    for (int k = 0; k < 2; ++k) {
        out[k].assign(1, ClusterTail3View<float>{});
        const int C = kTailCtas[k];
        for (int l = 1; l <= std::min(L - 2, kCTailLevels - 1); ++l) {
            ClusterTail3View<float> v{};
            v.ctas = C;
            v.lc = l;
            for (int q = 0; q <= l; ++q) {
                const int rows = c->hl[q].m[1] * c->hl[q].m[2];
                v.R[q] = q == 0 ? rows : (rows + C - 1) / C;
            }
            int off = 0, rmax = N0, tmax = N0;
            for (int q = 1; q <= l; ++q) {
                const TransferView<float>& X = c->tv32[q];
                v.off_rp[q] = off;
                off += 2 * (v.R[q - 1] * X.rw[1] * X.rw[2] + v.R[q] * X.pw[1] * X.pw[2]);
            }
            v.npair = off / 2;
            for (int q = 1; q <= l; ++q) {                     // static: operator data and tables
                const int mx = c->hl[q].m[0], my = c->hl[q].m[1], mz = c->hl[q].m[2], R = v.R[q];
                const LevelView<float>& Lq = c->lv32[q];
                const TransferView<float>& X = c->tv32[q];
                v.nbc[q] = Lq.tlo[0] + (mx - Lq.thi[0]);
                v.off_inv[q] = off; off += R * mx;
                v.off_cc[q] = off; off += 2 * W2 * R;
                v.off_yb[q] = off; off += 2 * W * my;
                v.off_zb[q] = off; off += 2 * W * mz;
                v.off_xb[q] = off; off += 2 * W * (v.nbc[q] + 1);
                v.off_tx[q] = off;
                for (int d = 0; d < 3; ++d) off += X.mf[d] * (1 + X.pw[d]) + X.mc[d] * (1 + X.rw[d]);
                rmax = std::max(rmax, R * mx);
                tmax = std::max({tmax, R * X.mc[0], v.R[q - 1] * X.mf[0]});
            }
            const int m0 = c->hl[0].m[0], m1 = c->hl[0].m[1], m2 = c->hl[0].m[2];
            v.off_cv = off; off += m0 * m0 + m1 * m1 + m2 * m2 + N0;
            v.off_z = off; off += c->hl[l].m[0];
            off = (off + 3) / 4 * 4;                           // the image: whole 16-byte units
            v.img16 = off / 4;
            for (int q = 0; q <= l; ++q) {                     // dynamic: iterates, right sides, T rows
                const int mx = c->hl[q].m[0], my = c->hl[q].m[1], R = v.R[q];
                v.off_x[q] = off; off += R * (mx + 2 * p);
                v.off_b[q] = off; off += R * mx;
                if (q > 0) { v.off_tm[q] = off; off += 2 * (R + 2 * (p * my + p)) * mx; }   // own rows, halos
            }
            v.off_r = off; off += rmax;
            v.off_t = off; off += tmax;
            v.smem = (size_t)off * sizeof(float);
            for (int q = 0; q <= l; ++q) {
                v.L[q] = c->lv32[q];
                v.X[q] = c->tv32[q];
            }
            v.C = c->cv32;
            if (!dev::cluster_tail3_fits(v)) break;
            out[k].push_back(v);
        }
    }
}

// Row-CTA thread cap of the GS sweeps in cycles of type T (autotuned for FP32).
template <typename T>
int gs_cap(const igamg_ctx* c) { return std::is_same<T, float>::value ? c->gs_cap32 : 0; }

// One GS sweep on level l in the context's form for precision T.
template <typename T>
void sweep(const igamg_ctx* c, cudaStream_t s, const Workspace& w, int l, bool descending, T* x, const T* b,
           T* TM, T* TK) {
    const auto& lv = Views<T>::lv(c);
    const bool flow = lv[l].rows() >= (std::is_same<T, float>::value ? c->flow32 : c->flow64);
    if (flow && w.sync) {
        const SweepSync sy{w.done[l], w.ctr[l], w.err, w.never, wait_limit_ns(), wait_test_unset()};
        dev::gs_sweep<T>(s, c->dim, lv[l], descending, x, b, TM, TK, gs_cap<T>(c), &sy);
    } else {
        dev::gs_sweep<T>(s, c->dim, lv[l], descending, x, b, TM, TK, gs_cap<T>(c));
    }
}

// Clears the workspace's synchronisation words (the first use of a workspace
// in a call; sweeps leave them zero).
cudaError_t clear_sync(const Workspace& w, cudaStream_t s) {
    return cudaMemsetAsync(w.sync, 0, w.nsync * sizeof(unsigned), s);
}

// Algorithm 2 for any mu and either smoother (nu1 = nu2 = 1), recursively:
// level l pre-smooths, restricts its residual, runs mu cycles on level l - 1
// from a zero coarse error (one direct solve on the coarsest level: a second
// one would return the same e), adds the prolonged correction and
// post-smooths.  Gauss-Seidel colours run ascending before and descending
// after the coarse correction, as in the V-cycle below.
template <typename T>
void mu_cycle(const igamg_ctx* c, cudaStream_t s, Workspace& w, int top, int l, T* x_top, const T* b_top,
              bool zero) {
    const auto& lv = Views<T>::lv(c);
    const auto& tv = Views<T>::tv(c);
    auto& B = Views<T>::buf(w);
    const int dim = c->dim;
    T* x = (l == top) ? x_top : B[l].x;
    const T* b = (l == top) ? b_top : B[l].b;
    if (l == 0) {
        dev::coarse_solve<T>(s, dim, Views<T>::cv(c), b, x);                           // direct
        return;
    }
    if constexpr (std::is_same<T, float>::value) {
        // FP32 2D V-cycles (Jacobi smoothing here) hand levels lc..0 to one
        // CTA, as the Gauss-Seidel V-cycle does; W-cycles revisit coarse
        // levels from nonzero iterates, which the tail does not take
        if (c->mu == 1 && tail_level(c) > 0 && l == tail_level(c) && l < top) {
            run_tail(c, s, b, x, c->smoother == IGAMG_SMOOTH_JACOBI, (float)c->omega);
            return;
        }
    }
    const size_t N = lv[l].n();
    if (zero) {
        if (x == B[l].x) dev::fill_zero<T>(s, B[l].x, 3 * N);
        else {
            dev::fill_zero<T>(s, x, N);
            dev::fill_zero<T>(s, B[l].TM, 2 * N);
        }
    }
    // 2D Jacobi sweeps write the new row sums to a second buffer (the level's
    // r and tmp2, which the 2D residual-restriction and prolongation kernels
    // leave untouched): between the two sweeps the sums live there, and the
    // post-smoothing sweep writes them back to T_M, T_K.
    const bool alt = c->smoother == IGAMG_SMOOTH_JACOBI && dim == 2;
    T* tm = alt ? B[l].r : B[l].TM;
    T* tk = alt ? B[l].tmp2 : B[l].TK;
    if (c->smoother == IGAMG_SMOOTH_JACOBI)
        dev::jacobi_sweep<T>(s, dim, lv[l], (T)c->omega, x, b, B[l].TM, B[l].TK, tm, tk);
    else
        sweep<T>(c, s, w, l, false, x, b, B[l].TM, B[l].TK);
    const bool clear = l - 1 >= 1;                  // coarse e^0 = 0: x | T_M | T_K of level l - 1
    dev::residual_restrict<T>(s, dim, lv[l], tv[l], b, tm, tk, B[l].r, B[l - 1].b, B[l].tmp1, B[l].tmp2,
                              clear ? B[l - 1].x : nullptr, clear ? 3 * lv[l - 1].n() : 0);
    const int reps = (l - 1 == 0) ? 1 : c->mu;
    for (int i = 0; i < reps; ++i) mu_cycle<T>(c, s, w, top, l - 1, x_top, b_top, false);
    T* e = (l - 1 == top) ? x_top : B[l - 1].x;
    dev::prolong_add<T>(s, dim, tv[l], lv[l], e, x, tm, tk, B[l].tmp1, B[l].tmp2);
    if (c->smoother == IGAMG_SMOOTH_JACOBI)
        dev::jacobi_sweep<T>(s, dim, lv[l], (T)c->omega, x, b, tm, tk, B[l].TM, B[l].TK);
    else
        sweep<T>(c, s, w, l, true, x, b, B[l].TM, B[l].TK);
}

bool default_cycle(const igamg_ctx* c) { return c->smoother == IGAMG_SMOOTH_GS && c->mu == 1; }

// Algorithm 2 (mu = 1, nu1 = nu2 = 1) from level `top` down to the coarsest
// and back.  x_top / b_top are the top level's iterate and right side; the
// top level's TM/TK must match x_top unless top_zero (then x_top = 0 is set).
template <typename T>
void vcycle(const igamg_ctx* c, cudaStream_t s, Workspace& w, int top, T* x_top, const T* b_top,
            bool top_zero, bool learned_top = false, T* capture_mid = nullptr) {
    if (!default_cycle(c)) {                        // W-cycle or Jacobi smoothing (callers reject the
        mu_cycle<T>(c, s, w, top, top, x_top, b_top, top_zero);    // learned form and the probe there)
        return;
    }
    const auto& lv = Views<T>::lv(c);
    const auto& tv = Views<T>::tv(c);
    auto& B = Views<T>::buf(w);
    const int dim = c->dim;
    // FP32 2D cycles hand levels lc..0 to one CTA or cluster when the hierarchy has a tail
    int lc = 0;
    if constexpr (std::is_same<T, float>::value)
        if (tail_level(c) > 0 && tail_level(c) < top) lc = tail_level(c);
    const int lowest = lc > 0 ? lc + 1 : 1;
    for (int l = top; l >= lowest; --l) {
        T* x = (l == top) ? x_top : B[l].x;
        const T* b = (l == top) ? b_top : B[l].b;
        const size_t N = lv[l].n();
        if (l == top && top_zero) {                     // coarser levels were cleared by the restriction
            if (x == B[l].x) dev::fill_zero<T>(s, B[l].x, 3 * N);
            else {
                dev::fill_zero<T>(s, x, N);
                dev::fill_zero<T>(s, B[l].TM, 2 * N);
            }
        }
        sweep<T>(c, s, w, l, false, x, b, B[l].TM, B[l].TK);                            // pre-smooth
        // b_{l-1} = R (b - A u), R = P^T; the next per-level level's x | T_M | T_K
        // (coarse e^0 = 0) are cleared in the same pass
        const bool clear = l - 1 >= lowest;
        dev::residual_restrict<T>(s, dim, lv[l], tv[l], b, B[l].TM, B[l].TK, B[l].r, B[l - 1].b, B[l].tmp1,
                                  B[l].tmp2, clear ? B[l - 1].x : nullptr, clear ? 3 * lv[l - 1].n() : 0);
    }
    if (lc > 0) {
        if constexpr (std::is_same<T, float>::value)
            run_tail(c, s, B[lc].b, B[lc].x);                                            // levels lc..0
    } else {
        T* x0 = (top == 0) ? x_top : B[0].x;
        const T* b0 = (top == 0) ? b_top : B[0].b;
        dev::coarse_solve<T>(s, dim, Views<T>::cv(c), b0, x0);                          // direct
    }
    for (int l = lc + 1; l <= top; ++l) {
        T* x = (l == top) ? x_top : B[l].x;
        const T* b = (l == top) ? b_top : B[l].b;
        T* e = (l - 1 == top) ? x_top : B[l - 1].x;
        dev::prolong_add<T>(s, dim, tv[l], lv[l], e, x, B[l].TM, B[l].TK, B[l].tmp1, B[l].tmp2);
        if (l == top && capture_mid)                                                    // state before post-smoothing
            cudaMemcpyAsync(capture_mid, x, lv[l].n() * sizeof(T), cudaMemcpyDeviceToDevice, s);
        if constexpr (std::is_same<T, float>::value) {
            if (l == top && learned_top) {                  // learned post-smoother: x += CNN(b - A x)
                dev::residual<float, float>(s, dim, lv[l], b, B[l].TM, B[l].TK, B[l].r, nullptr);
                cnn_forward(s, 1, lv[l].m[1] * lv[l].m[2], lv[l].m[0], B[l].r, c->cnn_w, x, 1, w.cnn);
                continue;
            }
        }
        sweep<T>(c, s, w, l, true, x, b, B[l].TM, B[l].TK);                             // post-smooth
    }
}

// ---------------------------------------------------------------- general operator
// Algorithm 2 (any mu; nu1 = nu2 = 1) on the stencil levels of a general
// context: multicolour Gauss-Seidel (ascending before, descending after the
// coarse correction) or weighted Jacobi, residual on the stencil, restriction
// R = P^T and prolongation P of the Poisson path, Galerkin coarse operators,
// dense coarsest solve.  Level l's r holds its residual; x | TM of a coarse
// level are its iterate.
void gen_mu_cycle(const igamg_ctx* c, cudaStream_t s, Workspace& w, int top, int l, double* x_top,
                  const double* b_top, bool zero) {
    auto& B = w.d;
    double* x = (l == top) ? x_top : B[l].x;
    const double* b = (l == top) ? b_top : B[l].b;
    const StencilView& V = c->sv[l];
    if (l == 0) {
        dev::gen_dense_apply(s, c->A0inv, c->n0, b, x);
        return;
    }
    if (zero) dev::fill_zero<double>(s, x, V.n());
    auto smooth = [&](bool descending) {
        if (c->smoother == IGAMG_SMOOTH_JACOBI) {
            dev::gen_residual(s, V, x, b, B[l].r, nullptr);
            dev::gen_jacobi_update(s, V, c->omega, B[l].r, x);
        } else {
            dev::gen_gs_sweep(s, V, descending, x, b);
        }
    };
    smooth(false);
    dev::gen_residual(s, V, x, b, B[l].r, nullptr);
    dev::restrict_<double>(s, 2, c->tv64[l], B[l].r, B[l - 1].b, B[l].tmp1, B[l].tmp2);
    const int reps = (l - 1 == 0) ? 1 : c->mu;
    for (int i = 0; i < reps; ++i) gen_mu_cycle(c, s, w, top, l - 1, x_top, b_top, i == 0);
    dev::gen_prolong_add(s, c->tv64[l], B[l - 1].x, x);
    smooth(true);
}

// One V-cycle (fixed-point step s_{i+1} = G(s_i), Eq. fixedpoint) from S_in to
// S_out on the finest level; the finest FP64 TM/TK match S_in on entry and
// S_out on exit.
void fixed_point_step(const igamg_ctx* c, cudaStream_t s, Workspace& w, int prec, const double* d_b,
                      double* S_in, double* S_out) {
    const int top = c->L - 1;
    const size_t N = finestN(c);
    LevelBuf<double>& F = w.d[top];
    if (c->general) {                               // FP64 only (checked by the callers)
        if (S_out != S_in) cudaMemcpyAsync(S_out, S_in, N * sizeof(double), cudaMemcpyDeviceToDevice, s);
        gen_mu_cycle(c, s, w, top, top, S_out, d_b, false);
        return;
    }
    if (prec == IGAMG_FP64) {
        if (S_out != S_in) cudaMemcpyAsync(S_out, S_in, N * sizeof(double), cudaMemcpyDeviceToDevice, s);
        vcycle<double>(c, s, w, top, S_out, d_b, false);
        if (top == 0)   // single grid: the direct solve changed x without refreshing its row sums
            dev::xpass<double, double>(s, c->lv64[0], S_out, nullptr, nullptr, 0, nullptr, nullptr, 0, F.TM, F.TK);
    } else {
        LevelBuf<float>& G = w.f[top];
        // r = b - A s in FP64, rounded to FP32; e = V32(0; r); s_out = s_in + e (FP64)
        dev::residual<double, float>(s, c->dim, c->lv64[top], d_b, F.TM, F.TK, G.b, nullptr, nullptr, F.tmp1,
                                     F.tmp2);
        vcycle<float>(c, s, w, top, G.x, G.b, true, prec == IGAMG_FP32_IR_LEARNED);
        dev::xpass<double, float>(s, c->lv64[top], S_in, S_out, G.x, 0, nullptr, nullptr, 0, F.TM, F.TK);
    }
}

// ||b - A x|| / denom into scal[1] using the finest TM/TK (which match x).
void residual_norm(const igamg_ctx* c, cudaStream_t s, Workspace& w, const double* d_b,
                   const double* denom) {
    const int top = c->L - 1;
    LevelBuf<double>& F = w.d[top];
    if (c->general) {
        dev::gen_residual(s, c->sv[top], w.S, d_b, F.r, w.partial);
        dev::norm_final(s, w.partial, dev::gen_blocks(c->sv[top].n()), denom, w.scal, 1);
        return;
    }
    if (!w.f.empty())           // FP32-IR workspace: also leave r in FP32 for the next V-cycle
        dev::residual<double, float>(s, c->dim, c->lv64[top], d_b, F.TM, F.TK, w.f[top].b, w.partial, F.r,
                                     F.tmp1, F.tmp2);
    else
        dev::residual<double, double>(s, c->dim, c->lv64[top], d_b, F.TM, F.TK, F.r, w.partial, nullptr, F.tmp1,
                                      F.tmp2);
    dev::norm_final(s, w.partial, c->lv64[top].rows(), denom, w.scal, 1);
}

// One restart cycle of Algorithm 5 (or one plain V-cycle for extrap = NONE).
void restart_body(const igamg_ctx* c, cudaStream_t s, Workspace& w, int extrap, int k, int prec,
                  const double* d_b, const double* denom) {
    const size_t N = finestN(c);
    const int top = c->L - 1;
    if (extrap == IGAMG_EXTRAP_NONE) {
        fixed_point_step(c, s, w, prec, d_b, w.S, w.S);
    } else if (c->general) {
        // general operator: FP64 cycles; t = sum_j gamma_j s_j -> S_0 (no row sums)
        for (int i = 0; i <= k; ++i)
            fixed_point_step(c, s, w, prec, d_b, w.S + (size_t)i * w.ld, w.S + (size_t)(i + 1) * w.ld);
        const int nb = dev::gram_blocks(N);
        dev::extrap_gammas(s, k, extrap, w.S, w.ld, N, w.partial, nb, w.info, w.gamma, w.qused);
        dev::combine(s, k, w.gamma, w.S, w.ld, N, w.S);
    } else if (prec != IGAMG_FP64) {
        // FP32 V-cycles with the FP64 residual carried by r <- r - A e in
        // double-FP32 arithmetic (refine.cu); the restart's first residual and
        // the one after extrapolation are computed from scratch in FP64.
        // r = b - A S_0 in FP64 (F.r) and FP32 (G.b) was left by the residual
        // norm of the previous restart, or of the solve's start
        LevelBuf<double>& F = w.d[top];
        LevelBuf<float>& G = w.f[top];
        double* r64 = F.r;
        float* tmh = reinterpret_cast<float*>(F.tmp1);
        float* tml = tmh + N;
        float* tkh = reinterpret_cast<float*>(F.tmp2);
        float* tkl = tkh + N;
        for (int i = 0; i <= k; ++i) {
            vcycle<float>(c, s, w, top, G.x, G.b, true, prec == IGAMG_FP32_IR_LEARNED);
            dev::refine_xpass_df(s, c->dfv, w.S + (size_t)i * w.ld, w.S + (size_t)(i + 1) * w.ld, G.x, tmh, tml,
                                 tkh, tkl);
            if (i == k) continue;
            if (c->dim == 2) {
                dev::refine_residual_df(s, c->dfv, tmh, tml, tkh, tkl, r64, G.b);
            } else {                                // 3D: y pass into F.TM | F.TK (free until the x-pass below)
                dev::refine_residual_df3(s, c->dfv, tmh, tml, tkh, tkl, reinterpret_cast<float*>(F.TM),
                                         reinterpret_cast<float*>(F.TK), r64, G.b);
            }
        }
        const int nb = dev::gram_blocks(N);
        dev::extrap_gammas(s, k, extrap, w.S, w.ld, N, w.partial, nb, w.info, w.gamma, w.qused);
        dev::xpass<double, double>(s, c->lv64[top], nullptr, w.S, nullptr, k + 2, w.gamma, w.S, w.ld,
                                   w.d[top].TM, w.d[top].TK);
    } else {
        for (int i = 0; i <= k; ++i)
            fixed_point_step(c, s, w, prec, d_b, w.S + (size_t)i * w.ld, w.S + (size_t)(i + 1) * w.ld);
        const int nb = dev::gram_blocks(N);
        dev::extrap_gammas(s, k, extrap, w.S, w.ld, N, w.partial, nb, w.info, w.gamma, w.qused);
        // t = sum_j gamma_j s_j -> S_0, with fresh FP64 row sums for the residual
        dev::xpass<double, double>(s, c->lv64[top], nullptr, w.S, nullptr, k + 2, w.gamma, w.S, w.ld,
                                   w.d[top].TM, w.d[top].TK);
    }
    residual_norm(c, s, w, d_b, denom);
}

igamg_status check_ctx(const igamg_ctx* c, bool need_assembled = true) {
    if (!c) return fail(IGAMG_EINVAL, "null context");
    if (need_assembled && !c->assembled) return fail(IGAMG_EINVAL, "context not assembled");
    return IGAMG_OK;
}

igamg_status check_ws(const igamg_ctx* c, void* ws, size_t bytes, int k, int prec) {
    const size_t need = carve(c, nullptr, k, prec).bytes;
    if (!ws) return fail(IGAMG_EINVAL, "null workspace");
    if (((uintptr_t)ws & 255) != 0) return fail(IGAMG_EINVAL, "workspace must be 256-byte aligned");
    if (bytes < need) return fail(IGAMG_ENOMEM, "workspace too small: need " + std::to_string(need));
    return IGAMG_OK;
}

// Capture one restart cycle of this context into its CUDA graph (cached per
// right-hand side, workspace, k, method, precision and test).
igamg_status ensure_graph(igamg_ctx* c, Workspace& w, const double* d_b, void* d_ws, int kk, int extrap,
                          int prec, const double* denom) {
    const int slot = prec;
    igamg_ctx::Key key;
    key.b = d_b; key.ws = d_ws; key.k = kk; key.extrap = extrap; key.prec = prec;
    key.abs_tol = denom == nullptr;
    key.overlap = launch_overlap() ? 1 : 0;
    key.sync = sync_generation();
    key.w = prec == IGAMG_FP32_IR_LEARNED ? c->cnn_w : nullptr;
    if (c->exec[slot] && c->key[slot] == key) return IGAMG_OK;
    if (c->exec[slot]) { cudaGraphExecDestroy(c->exec[slot]); c->exec[slot] = nullptr; }
    cudaGraph_t g = nullptr;
    const long long before = launch_count();
    CUDA_TRY(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    restart_body(c, c->cap, w, extrap, kk, prec, d_b, denom);
    cudaError_t ce = cudaStreamEndCapture(c->cap, &g);
    if (ce != cudaSuccess) return fail(IGAMG_ECUDA, std::string("capture: ") + cudaGetErrorString(ce));
    c->exec_launches[slot] = launch_count() - before;
    count_launch(-c->exec_launches[slot]);
    ce = cudaGraphInstantiate(&c->exec[slot], g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
        c->exec[slot] = nullptr;
        return fail(IGAMG_ECUDA, std::string("instantiate: ") + cudaGetErrorString(ce));
    }
    c->key[slot] = key;
    return IGAMG_OK;
}

// Capture the device-side restart loop of this context: a graph holding one
// conditional WHILE node (condition 1 at launch) whose body is one restart
// cycle followed by loop_step, which records the residual and clears the
// condition once the accuracy test passes, max_cycles is reached, the
// residual is not finite or a device wait gave up.  Cached like ensure_graph.
igamg_status ensure_loop_graph(igamg_ctx* c, Workspace& w, const double* d_b, void* d_ws, int kk, int extrap,
                               int prec, const double* denom) {
    const int slot = prec;
    igamg_ctx::Key key;
    key.b = d_b; key.ws = d_ws; key.k = kk; key.extrap = extrap; key.prec = prec;
    key.abs_tol = denom == nullptr;
    key.overlap = launch_overlap() ? 1 : 0;
    key.sync = sync_generation();
    if (c->loop_exec[slot] && c->loop_key[slot] == key) return IGAMG_OK;
    if (c->loop_exec[slot]) { cudaGraphExecDestroy(c->loop_exec[slot]); c->loop_exec[slot] = nullptr; }
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaGraphCreate(&g, 0));
    struct GraphGuard { cudaGraph_t g; ~GraphGuard() { if (g) cudaGraphDestroy(g); } } guard{g};
    cudaGraphConditionalHandle h;
    CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CUDA_TRY(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    const long long before = launch_count();
    CUDA_TRY(cudaStreamBeginCaptureToGraph(c->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    restart_body(c, c->cap, w, extrap, kk, prec, d_b, denom);
    dev::loop_step(c->cap, h, w.loop, w.scal + 1, w.err, w.hist);
    cudaGraph_t got = nullptr;
    cudaError_t ce = cudaStreamEndCapture(c->cap, &got);
    const long long body_launches = launch_count() - before;
    count_launch(-body_launches);
    if (ce != cudaSuccess) return fail(IGAMG_ECUDA, std::string("loop capture: ") + cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&c->loop_exec[slot], g, 0);
    if (ce != cudaSuccess) {
        c->loop_exec[slot] = nullptr;
        return fail(IGAMG_ECUDA, std::string("loop instantiate: ") + cudaGetErrorString(ce));
    }
    c->loop_body_launches[slot] = body_launches;
    c->loop_key[slot] = key;
    return IGAMG_OK;
}

}  // namespace

// ======================================================================= C ABI
extern "C" {

const char* igamg_status_str(int st) {
    switch (st) {
        case IGAMG_OK: return "ok";
        case IGAMG_EINVAL: return "invalid argument";
        case IGAMG_ENOMEM: return "out of memory";
        case IGAMG_ECUDA: return "CUDA error";
        case IGAMG_ENOTCONV: return "not converged";
        case IGAMG_EBREAKDOWN: return "breakdown (non-finite residual)";
        case IGAMG_ETIMEOUT: return "device wait timed out";
        default: return "unknown status";
    }
}

const char* igamg_last_error(void) { return g_err.c_str(); }

long long igamg_launch_count(void) { return launch_count(); }

igamg_status igamg_setup(int dim, int p, const int* n_elems, int n_levels, igamg_ctx** out) {
    if (!out || !n_elems) return fail(IGAMG_EINVAL, "null pointer");
    *out = nullptr;
    if (dim != 2 && dim != 3) return fail(IGAMG_EINVAL, "dim must be 2 or 3");
    if (p < 1 || p > kMaxP) return fail(IGAMG_EINVAL, "p must be in [1, 7]");
    for (int d = 0; d < dim; ++d)
        if (n_elems[d] < 2 || n_elems[d] > 4096) return fail(IGAMG_EINVAL, "n_elems must be in [2, 4096]");
    if (n_levels < 0 || n_levels > 16) return fail(IGAMG_EINVAL, "n_levels must be in [0, 16]");
    igamg_ctx* c = new (std::nothrow) igamg_ctx();
    if (!c) return fail(IGAMG_ENOMEM, "host allocation");
    c->dim = dim;
    c->p = p;
    try {
        std::vector<std::vector<std::vector<double>>> chain;
        std::vector<std::vector<double>> br(3);
        for (int d = 0; d < dim; ++d) br[d] = uniform_breaks(n_elems[d]);
        chain.push_back(br);
        auto nel = [&](const std::vector<std::vector<double>>& b) {
            int mx = 0;
            for (int d = 0; d < dim; ++d) mx = std::max(mx, (int)b[d].size() - 1);
            return mx;
        };
        if (n_levels == 0) {
            while (nel(chain.back()) > 8) {
                std::vector<std::vector<double>> nb(3);
                for (int d = 0; d < dim; ++d) nb[d] = coarsen_breaks(chain.back()[d]);
                chain.push_back(nb);
            }
        } else {
            for (int l = 1; l < n_levels; ++l) {
                std::vector<std::vector<double>> nb(3);
                for (int d = 0; d < dim; ++d) {
                    if ((int)chain.back()[d].size() - 1 < 2) { delete c; return fail(IGAMG_EINVAL, "too many levels"); }
                    nb[d] = coarsen_breaks(chain.back()[d]);
                }
                chain.push_back(nb);
            }
        }
        std::reverse(chain.begin(), chain.end());       // level 0 = coarsest
        c->L = (int)chain.size();
        c->hl.resize(c->L);
        for (int l = 0; l < c->L; ++l) {
            HostLevel& H = c->hl[l];
            for (int d = 0; d < dim; ++d) {
                H.breaks[d] = chain[l][d];
                H.f[d] = assemble_1d(H.breaks[d], p);
                H.m[d] = H.f[d].m;
                if (H.m[d] < 1) { delete c; return fail(IGAMG_EINVAL, "a level has no interior unknowns"); }
                if (l > 0) {
                    H.P[d] = prolongation_1d(H.breaks[d], chain[l - 1][d], p, &H.pmf[d], &H.pmc[d]);
                    compact_transfer(H, d);
                }
            }
        }
        if (c->hl.back().m[0] > 4500) { delete c; return fail(IGAMG_EINVAL, "row length above 4500"); }
        const HostLevel& H0 = c->hl[0];
        const size_t N0 = H0.N();
        if (N0 > 12000) { delete c; return fail(IGAMG_EINVAL, "coarsest grid too large for the direct solve"); }
        std::vector<double> lam[3];
        for (int d = 0; d < dim; ++d) generalized_eigen(H0.f[d], c->cV[d], lam[d]);
        c->claminv.resize(N0);
        for (int k = 0; k < H0.m[2]; ++k)
            for (int j = 0; j < H0.m[1]; ++j)
                for (int i = 0; i < H0.m[0]; ++i) {
                    double s = lam[0][i] + lam[1][j] + (dim == 3 ? lam[2][k] : 0.0);
                    c->claminv[((size_t)k * H0.m[1] + j) * H0.m[0] + i] = 1.0 / s;
                }
    } catch (const std::exception& e) {
        delete c;
        return fail(IGAMG_EINVAL, std::string("setup: ") + e.what());
    }
    // one-launch sweeps on 3D levels with many rows (see igamg_ctx::flow32)
    if (dim == 3) c->flow32 = c->flow64 = kFlowRows3D;
    *out = c;
    return IGAMG_OK;
}

igamg_status igamg_info(const igamg_ctx* c, int* n_levels, int* h_m) {
    if (igamg_status st = check_ctx(c, false)) return st;
    if (n_levels) *n_levels = c->L;
    if (h_m)
        for (int l = 0; l < c->L; ++l)
            for (int d = 0; d < 3; ++d) h_m[3 * l + d] = c->hl[l].m[d];
    return IGAMG_OK;
}

igamg_status igamg_get_factor(const igamg_ctx* c, int level, int d, int which, double* h_out, int* rows,
                              int* cols) {
    if (igamg_status st = check_ctx(c, false)) return st;
    if (level < 0 || level >= c->L || d < 0 || d >= c->dim || which < 0 || which > 2)
        return fail(IGAMG_EINVAL, "bad level/direction/which");
    const HostLevel& H = c->hl[level];
    if (which < 2) {
        const std::vector<double>& F = which == 0 ? H.f[d].M : H.f[d].K;
        if (rows) *rows = H.f[d].m;
        if (cols) *cols = 2 * c->p + 1;
        if (h_out) std::memcpy(h_out, F.data(), F.size() * sizeof(double));
    } else {
        if (level == 0) return fail(IGAMG_EINVAL, "level 0 has no prolongation");
        if (rows) *rows = H.pmf[d];
        if (cols) *cols = H.pmc[d];
        if (h_out) std::memcpy(h_out, H.P[d].data(), H.P[d].size() * sizeof(double));
    }
    return IGAMG_OK;
}

igamg_status igamg_assemble(igamg_ctx* c) {
    if (igamg_status st = check_ctx(c, false)) return st;
    if (c->assembled) return IGAMG_OK;
    const int dim = c->dim, p = c->p, L = c->L;
    // host staging of every device array, then one allocation and copies
    struct Blob {
        std::vector<char> bytes;
        size_t off = 0;
    };
    std::vector<std::pair<size_t, std::vector<char>>> pieces;
    size_t total = 0;
    auto add = [&](const void* src, size_t bytes) -> size_t {
        total = (total + 255) & ~(size_t)255;
        const size_t off = total;
        std::vector<char> v((const char*)src, (const char*)src + bytes);
        pieces.emplace_back(off, std::move(v));
        total += bytes;
        return off;
    };
    struct LevelOff {
        size_t Mb[3][2], Kb[3][2], inv[2];
        size_t plo[3], rlo[3], pv[3][2], rv[3][2];
    };
    std::vector<LevelOff> lo(L);
    for (int l = 0; l < L; ++l) {
        const HostLevel& H = c->hl[l];
        for (int d = 0; d < dim; ++d) {
            auto m64 = band_major<double>(H.f[d], false), k64 = band_major<double>(H.f[d], true);
            auto m32 = band_major<float>(H.f[d], false), k32 = band_major<float>(H.f[d], true);
            lo[l].Mb[d][0] = add(m64.data(), m64.size() * 8);
            lo[l].Kb[d][0] = add(k64.data(), k64.size() * 8);
            lo[l].Mb[d][1] = add(m32.data(), m32.size() * 4);
            lo[l].Kb[d][1] = add(k32.data(), k32.size() * 4);
            if (l > 0) {
                lo[l].plo[d] = add(H.plo[d].data(), H.plo[d].size() * 4);
                lo[l].rlo[d] = add(H.rlo[d].data(), H.rlo[d].size() * 4);
                std::vector<float> pf(H.pv[d].begin(), H.pv[d].end()), rf(H.rv[d].begin(), H.rv[d].end());
                lo[l].pv[d][0] = add(H.pv[d].data(), H.pv[d].size() * 8);
                lo[l].rv[d][0] = add(H.rv[d].data(), H.rv[d].size() * 8);
                lo[l].pv[d][1] = add(pf.data(), pf.size() * 4);
                lo[l].rv[d][1] = add(rf.data(), rf.size() * 4);
            }
        }
        // inverse diagonal of A: 1 / sum_d K_d(i_d,i_d) prod_{e!=d} M_e(i_e,i_e)
        const size_t N = H.N();
        std::vector<double> inv(N);
        std::vector<float> inv32(N);
        const int bw = 2 * p + 1;
        for (int k = 0; k < H.m[2]; ++k)
            for (int j = 0; j < H.m[1]; ++j)
                for (int i = 0; i < H.m[0]; ++i) {
                    const int idx[3] = {i, j, k};
                    double s = 0.0;
                    for (int d = 0; d < dim; ++d) {
                        double t = H.f[d].K[(size_t)idx[d] * bw + p];
                        for (int e = 0; e < dim; ++e)
                            if (e != d) t *= H.f[e].M[(size_t)idx[e] * bw + p];
                        s += t;
                    }
                    const size_t o = ((size_t)k * H.m[1] + j) * H.m[0] + i;
                    inv[o] = 1.0 / s;
                    inv32[o] = (float)(1.0 / s);
                }
        lo[l].inv[0] = add(inv.data(), N * 8);
        lo[l].inv[1] = add(inv32.data(), N * 4);
    }
    // float-pair split of the finest 2D level's factors (double-FP32 refinement update)
    size_t dfo[3][4] = {};
    if (dim >= 2) {
        const HostLevel& H = c->hl[L - 1];
        for (int d = 0; d < dim; ++d)
            for (int which = 0; which < 2; ++which) {
                const std::vector<double> v = band_major<double>(H.f[d], which == 1);
                std::vector<float> hi(v.size()), lw(v.size());
                for (size_t q = 0; q < v.size(); ++q) {
                    hi[q] = (float)v[q];
                    lw[q] = (float)(v[q] - (double)hi[q]);
                }
                dfo[d][2 * which] = add(hi.data(), hi.size() * 4);
                dfo[d][2 * which + 1] = add(lw.data(), lw.size() * 4);
            }
    }
    size_t cVo[3][2], cLo[2];
    for (int d = 0; d < dim; ++d) {
        std::vector<float> f(c->cV[d].begin(), c->cV[d].end());
        cVo[d][0] = add(c->cV[d].data(), c->cV[d].size() * 8);
        cVo[d][1] = add(f.data(), f.size() * 4);
    }
    {
        std::vector<float> f(c->claminv.begin(), c->claminv.end());
        cLo[0] = add(c->claminv.data(), c->claminv.size() * 8);
        cLo[1] = add(f.data(), f.size() * 4);
    }
    dev::prepare_kernels();
    void* dm = nullptr;
    if (cudaMalloc(&dm, total) != cudaSuccess) {
        cudaGetLastError();
        return fail(IGAMG_ENOMEM, "device allocation of the operator data");
    }
    for (auto& pc : pieces) {
        cudaError_t e = cudaMemcpy((char*)dm + pc.first, pc.second.data(), pc.second.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(dm);
            return fail(IGAMG_ECUDA, std::string("upload: ") + cudaGetErrorString(e));
        }
    }
    c->dmem = dm;
    char* base = (char*)dm;
    c->lv64.resize(L);
    c->lv32.resize(L);
    c->tv64.resize(L);
    c->tv32.resize(L);
    for (int l = 0; l < L; ++l) {
        const HostLevel& H = c->hl[l];
        LevelView<double>& a = c->lv64[l];
        LevelView<float>& f = c->lv32[l];
        for (int d = 0; d < 3; ++d) {
            a.m[d] = f.m[d] = H.m[d];
            a.Mb[d] = a.Kb[d] = nullptr;
            f.Mb[d] = f.Kb[d] = nullptr;
        }
        a.p = f.p = p;
        for (int d = 0; d < dim; ++d) {
            a.Mb[d] = (const double*)(base + lo[l].Mb[d][0]);
            a.Kb[d] = (const double*)(base + lo[l].Kb[d][0]);
            f.Mb[d] = (const float*)(base + lo[l].Mb[d][1]);
            f.Kb[d] = (const float*)(base + lo[l].Kb[d][1]);
        }
        a.invdiag = (const double*)(base + lo[l].inv[0]);
        f.invdiag = (const float*)(base + lo[l].inv[1]);
        for (int d = 0; d < 3; ++d) {
            a.tlo[d] = f.tlo[d] = 0;
            a.thi[d] = f.thi[d] = 0;
            for (int b = 0; b < 2 * kMaxP + 1; ++b) a.Mc[d][b] = a.Kc[d][b] = f.Mc[d][b] = f.Kc[d][b] = 0;
            if (d >= dim) continue;
            int tl = 0, th = 0;
            const int mid = toeplitz_range(H.f[d], &tl, &th), bw = 2 * p + 1;
            tl = std::max(tl, p);                    // every band neighbour inside the grid
            th = std::max(tl, std::min(th, H.m[d] - p));
            a.tlo[d] = f.tlo[d] = tl;
            a.thi[d] = f.thi[d] = th;
            for (int b = 0; b < bw; ++b) {
                const double mv = H.f[d].M[(size_t)mid * bw + b], kv = H.f[d].K[(size_t)mid * bw + b];
                a.Mc[d][b] = mv; a.Kc[d][b] = kv;
                f.Mc[d][b] = (float)mv; f.Kc[d][b] = (float)kv;
            }
        }
        TransferView<double>& t = c->tv64[l];
        TransferView<float>& tf = c->tv32[l];
        std::memset(&t, 0, sizeof(t));
        std::memset(&tf, 0, sizeof(tf));
        if (l > 0)
            for (int d = 0; d < 3; ++d) {
                const int mf = (d < dim) ? H.m[d] : 1, mc = (d < dim) ? c->hl[l - 1].m[d] : 1;
                t.mf[d] = tf.mf[d] = mf;
                t.mc[d] = tf.mc[d] = mc;
                if (d >= dim) continue;
                t.pw[d] = tf.pw[d] = H.pw[d];
                t.rw[d] = tf.rw[d] = H.rw[d];
                t.plo[d] = tf.plo[d] = (const int*)(base + lo[l].plo[d]);
                t.rlo[d] = tf.rlo[d] = (const int*)(base + lo[l].rlo[d]);
                t.pv[d] = (const double*)(base + lo[l].pv[d][0]);
                t.rv[d] = (const double*)(base + lo[l].rv[d][0]);
                tf.pv[d] = (const float*)(base + lo[l].pv[d][1]);
                tf.rv[d] = (const float*)(base + lo[l].rv[d][1]);
            }
    }
    for (int d = 0; d < 3; ++d) {
        c->cv64.m[d] = c->cv32.m[d] = c->hl[0].m[d];
        c->cv64.V[d] = (d < dim) ? (const double*)(base + cVo[d][0]) : nullptr;
        c->cv32.V[d] = (d < dim) ? (const float*)(base + cVo[d][1]) : nullptr;
    }
    c->cv64.laminv = (const double*)(base + cLo[0]);
    c->cv32.laminv = (const float*)(base + cLo[1]);
    // Coarse tail of the FP32 2D cycle: the highest level below the finest
    // whose levels 0..lc fit one CTA's shared memory and that one SM handles
    // faster than a launch per step (kTailMaxN unknowns at most).
    constexpr size_t kTailMaxN = 6000;
    c->tail32.lc = 0;
    c->tails.assign(1, TailView<float>{});
    if (dim == 2 && L >= 3) {
        const size_t limit = dev::tail_smem_limit();
        for (int l = 1; l <= std::min(L - 2, kTailLevels - 1); ++l) {
            TailView<float> v{};
            int off = 0;
            for (int q = 0; q <= l; ++q) {
                const int n = (int)c->hl[q].N();
                v.off_x[q] = off; off += (c->hl[q].m[0] + 2 * p) * (c->hl[q].m[1] + 2 * p);   // zero halo of p
                v.off_b[q] = off; off += n;
                v.off_inv[q] = off; off += q > 0 ? n : 0;
                v.off_band[q] = off; off += q > 0 ? 2 * (2 * p + 1) * (c->hl[q].m[0] + c->hl[q].m[1]) : 0;
                v.off_tm[q] = off; off += q > 0 ? 2 * (c->hl[q].m[1] + 2 * p) * c->hl[q].m[0] : 0;
                v.off_tc[q] = off; off += q > 0 ? 2 * (2 * p + 1) : 0;
            }
            for (int q = 1; q <= l; ++q) {
                v.off_tr[q] = off;
                off += tail_transfer_elems(c->tv32[q]);
            }
            v.off_cv = off;
            off += c->hl[0].m[0] * c->hl[0].m[0] + c->hl[0].m[1] * c->hl[0].m[1] + (int)c->hl[0].N();
            const int nl = (int)c->hl[l].N();
            v.off_r = off; off += nl;
            v.off_t = off; off += nl;
            v.smem = (size_t)off * sizeof(float);
            if ((size_t)nl > kTailMaxN || v.smem > limit) break;
            v.lc = l;
            for (int q = 0; q <= l; ++q) {
                v.L[q] = c->lv32[q];
                v.X[q] = c->tv32[q];
            }
            v.C = c->cv32;
            c->tail32 = v;
            c->tails.push_back(v);
        }
    }
    // Cluster tails of the FP32 2D cycle: on kTailCtas[k] CTAs, every lc
    // whose levels fit a CTA's shared memory (ClusterTailView) and whose
    // cluster the device can hold.
    free_tail_images(c);
    for (int k = 0; k < 2; ++k) {
        c->ctails[k].assign(1, ClusterTailView<float>{});
        c->ctails3[k].assign(1, ClusterTail3View<float>{});
    }
    if (dim == 3 && L >= 3) {
        build_cluster_tails3(c, c->ctails3);
        select_tail(c, kTailCtas[1], tail_most(c, kTailCtas[1]));    // 3D: the deepest 16-CTA tail
    }
    if (dim == 2 && L >= 3) {
        const int W = 2 * p + 1;
        const int N0 = (int)c->hl[0].N(), m00 = c->hl[0].m[0], m01 = c->hl[0].m[1];
        for (int k = 0; k < 2; ++k) {
            const int C = kTailCtas[k];
            for (int l = 1; l <= std::min(L - 2, kCTailLevels - 1); ++l) {
                ClusterTailView<float> v{};
                v.ctas = C;
                v.lc = l;
                int off = 0, rmax = N0, tmax = N0;
                for (int q = 0; q <= l; ++q) v.R[q] = q == 0 ? c->hl[0].m[1] : (c->hl[q].m[1] + C - 1) / C;
                for (int q = 1; q <= l; ++q) {                 // row pointers first: 8-byte aligned
                    const TransferView<float>& X = c->tv32[q];
                    v.off_rp[q] = off;
                    off += 2 * (v.R[q] * W + v.R[q - 1] * X.rw[1] + v.R[q] * X.pw[1]);
                }
                v.npair = off / 2;
                for (int q = 1; q <= l; ++q) {                 // static: operator data and tables
                    const int mx = c->hl[q].m[0], R = v.R[q];
                    const LevelView<float>& Lq = c->lv32[q];
                    const TransferView<float>& X = c->tv32[q];
                    v.nbc[q] = Lq.tlo[0] + (mx - Lq.thi[0]);
                    v.off_inv[q] = off; off += R * mx;
                    v.off_yb[q] = off; off += 2 * W * R;
                    v.off_xb[q] = off; off += 2 * W * (v.nbc[q] + 1);      // boundary columns and the interior
                    v.off_tx[q] = off; off += X.mf[0] * (1 + X.pw[0]) + X.mc[0] * (1 + X.rw[0]);
                    v.off_ty[q] = off; off += R * X.pw[1] + v.R[q - 1] * X.rw[1] + R + v.R[q - 1];
                    rmax = std::max(rmax, R * mx);
                    tmax = std::max({tmax, R * X.mc[0], v.R[q - 1] * X.mf[0]});
                }
                v.off_cv = off; off += m00 * m00 + m01 * m01 + N0;
                v.off_z = off; off += c->hl[l].m[0];
                off = (off + 3) / 4 * 4;                       // the image: whole 16-byte units
                v.img16 = off / 4;
                for (int q = 0; q <= l; ++q) {                 // dynamic: iterates, right sides, row sums
                    const int mx = c->hl[q].m[0], R = v.R[q];
                    v.off_x[q] = off; off += R * (mx + 2 * p);
                    v.off_b[q] = off; off += R * mx;
                    if (q > 0) { v.off_tm[q] = off; off += 2 * R * mx; }
                }
                v.off_r = off; off += rmax;
                v.off_t = off; off += tmax;
                v.smem = (size_t)off * sizeof(float);
                for (int q = 0; q <= l; ++q) {
                    v.L[q] = c->lv32[q];
                    v.X[q] = c->tv32[q];
                }
                v.C = c->cv32;
                if (!dev::cluster_tail_fits(v)) break;
                c->ctails[k].push_back(v);
            }
        }
    }
    if (dim >= 2) {
        DFView& D = c->dfv;
        const LevelView<double>& a = c->lv64[L - 1];
        D.p = p;
        D.m[2] = 1;
        for (int d = 0; d < dim; ++d) {
            D.m[d] = a.m[d];
            D.tlo[d] = a.tlo[d];
            D.thi[d] = a.thi[d];
            D.Mh[d] = (const float*)(base + dfo[d][0]);
            D.Ml[d] = (const float*)(base + dfo[d][1]);
            D.Kh[d] = (const float*)(base + dfo[d][2]);
            D.Kl[d] = (const float*)(base + dfo[d][3]);
            for (int b = 0; b < 2 * kMaxP + 1; ++b) {
                const double mv = a.Mc[d][b], kv = a.Kc[d][b];
                D.Mch[d][b] = (float)mv;
                D.Mcl[d][b] = (float)(mv - (double)D.Mch[d][b]);
                D.Kch[d][b] = (float)kv;
                D.Kcl[d][b] = (float)(kv - (double)D.Kch[d][b]);
            }
        }
    }
    CUDA_TRY(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
    CUDA_TRY(cudaMallocHost(&c->h_pin, 64));
    CUDA_TRY(cudaMallocHost(&c->h_loop, sizeof(LoopState)));
    CUDA_TRY(cudaMallocHost(&c->h_hist, sizeof(double) * kLoopHist));
    c->assembled = true;
    return IGAMG_OK;
}

size_t igamg_workspace_bytes(const igamg_ctx* c, int k, int prec) {
    if (!c || k < 0 || k > kMaxQ) return 0;
    return carve(c, nullptr, std::max(k, 1), prec).bytes;
}

static void drop_graphs(igamg_ctx* c);

igamg_status igamg_setup_general(int p, const int* n_elems, int n_levels, igamg_ctx** out) {
    if (igamg_status st = igamg_setup(2, p, n_elems, n_levels, out)) return st;
    igamg_ctx* c = *out;
    if (n_elems[0] > 1024 || n_elems[1] > 1024) {
        igamg_destroy(c);
        *out = nullptr;
        return fail(IGAMG_EINVAL, "general operator: at most 1024 elements per direction");
    }
    c->general = true;
    c->gqx = quadrature_1d(c->hl.back().breaks[0], p);
    c->gqy = quadrature_1d(c->hl.back().breaks[1], p);
    return IGAMG_OK;
}

long igamg_quadrature_count(const igamg_ctx* c) {
    return (c && c->general) ? (long)c->gqx.nq * c->gqy.nq : 0;
}

igamg_status igamg_quadrature_points(const igamg_ctx* c, double* h_xi, double* h_eta) {
    if (!c || !c->general || !h_xi || !h_eta) return fail(IGAMG_EINVAL, "general context and two arrays needed");
    for (int qy = 0; qy < c->gqy.nq; ++qy)
        for (int qx = 0; qx < c->gqx.nq; ++qx) {
            const size_t q = (size_t)qy * c->gqx.nq + qx;
            h_xi[q] = c->gqx.x[qx];
            h_eta[q] = c->gqy.x[qy];
        }
    return IGAMG_OK;
}

igamg_status igamg_assemble_general(igamg_ctx* c, const double* h_coef, const double* h_jac) {
    if (!c || !c->general || !h_coef) return fail(IGAMG_EINVAL, "general context and coefficients needed");
    if (!c->assembled)
        if (igamg_status st = igamg_assemble(c)) return st;
    const size_t nq = (size_t)c->gqx.nq * c->gqy.nq;
    // transformed coefficients on the unit square: |J| J^{-1} A J^{-T}, |J| J^{-1} B, |J| c
    std::vector<double> co(6 * nq);
    c->gdet.assign(nq, 1.0);
    for (size_t q = 0; q < nq; ++q) {
        const double a11 = h_coef[q], a12 = h_coef[nq + q], a22 = h_coef[2 * nq + q];
        const double b1 = h_coef[3 * nq + q], b2 = h_coef[4 * nq + q], cc = h_coef[5 * nq + q];
        double j11 = 1, j12 = 0, j21 = 0, j22 = 1;
        if (h_jac) { j11 = h_jac[q]; j12 = h_jac[nq + q]; j21 = h_jac[2 * nq + q]; j22 = h_jac[3 * nq + q]; }
        const double det = j11 * j22 - j12 * j21;
        if (!(det > 0.0) || !std::isfinite(det)) return fail(IGAMG_EINVAL, "geometry Jacobian not positive");
        // K = J^{-1} = adj(J) / det
        const double k11 = j22 / det, k12 = -j12 / det, k21 = -j21 / det, k22 = j11 / det;
        // K A K^T
        const double t11 = k11 * a11 + k12 * a12, t12 = k11 * a12 + k12 * a22;
        const double t21 = k21 * a11 + k22 * a12, t22 = k21 * a12 + k22 * a22;
        co[q] = det * (t11 * k11 + t12 * k12);
        co[nq + q] = det * (t11 * k21 + t12 * k22);
        co[2 * nq + q] = det * (t21 * k21 + t22 * k22);
        co[3 * nq + q] = det * (k11 * b1 + k12 * b2);
        co[4 * nq + q] = det * (k21 * b1 + k22 * b2);
        co[5 * nq + q] = det * cc;
        c->gdet[q] = det;
    }
    const int L = c->L, p = c->p, W = 2 * p + 1;
    std::vector<Stencil2D> ops(L);
    std::vector<double> A0inv;
    try {
        ops[L - 1] = assemble_general(c->gqx, c->gqy, co.data());
        for (int l = L - 1; l >= 1; --l)
            ops[l - 1] = galerkin_coarse(ops[l], c->hl[l].P[0], c->hl[l - 1].m[0], c->hl[l].P[1], c->hl[l - 1].m[1]);
        if (!dense_inverse(ops[0], A0inv)) return fail(IGAMG_EINVAL, "singular coarsest operator");
    } catch (const std::exception& e) {
        return fail(IGAMG_EINVAL, std::string("general assembly: ") + e.what());
    }
    // one device allocation: per level the stencil and the inverse diagonal, then the coarsest inverse
    std::vector<size_t> off(2 * L + 1);
    size_t total = 0;
    for (int l = 0; l < L; ++l) {
        off[2 * l] = total;
        total = (total + ops[l].S.size() * 8 + 255) & ~(size_t)255;
        off[2 * l + 1] = total;
        total = (total + ops[l].N() * 8 + 255) & ~(size_t)255;
    }
    off[2 * L] = total;
    total += A0inv.size() * 8;
    if (c->gmem) { cudaFree(c->gmem); c->gmem = nullptr; }
    c->gen_ready = false;
    CUDA_TRY(cudaMalloc(&c->gmem, total));
    char* base = (char*)c->gmem;
    c->sv.assign(L, StencilView{});
    for (int l = 0; l < L; ++l) {
        const size_t N = ops[l].N();
        std::vector<double> inv(N);
        for (size_t I = 0; I < N; ++I) {
            const double d = ops[l].S[(size_t)(p * W + p) * N + I];
            if (!(d != 0.0)) return fail(IGAMG_EINVAL, "zero diagonal in the general operator");
            inv[I] = 1.0 / d;
        }
        CUDA_TRY(cudaMemcpy(base + off[2 * l], ops[l].S.data(), ops[l].S.size() * 8, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(base + off[2 * l + 1], inv.data(), N * 8, cudaMemcpyHostToDevice));
        StencilView& V = c->sv[l];
        V.m[0] = ops[l].mx;
        V.m[1] = ops[l].my;
        V.p = p;
        V.S = (const double*)(base + off[2 * l]);
        V.inv = (const double*)(base + off[2 * l + 1]);
    }
    CUDA_TRY(cudaMemcpy(base + off[2 * L], A0inv.data(), A0inv.size() * 8, cudaMemcpyHostToDevice));
    c->A0inv = (double*)(base + off[2 * L]);
    c->n0 = (int)ops[0].N();
    c->gen_ready = true;
    drop_graphs(c);
    return IGAMG_OK;
}

igamg_status igamg_rhs_points(igamg_ctx* c, const double* h_f, double* d_b, void* stream) {
    if (!c || !c->general || !h_f || !d_b) return fail(IGAMG_EINVAL, "general context, f and d_b needed");
    if (c->gdet.empty()) return fail(IGAMG_EINVAL, "call igamg_assemble_general first");
    const size_t nq = (size_t)c->gqx.nq * c->gqy.nq;
    std::vector<double> fq(nq);
    for (size_t q = 0; q < nq; ++q) fq[q] = c->gdet[q] * h_f[q];
    const std::vector<double> b = load_general(c->gqx, c->gqy, fq.data());
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(d_b, b.data(), b.size() * 8, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return IGAMG_OK;
}

igamg_status igamg_rhs_sine(igamg_ctx* c, int modes, const double* h_coeffs, double* d_b, void* stream) {
    if (c && c->general) return fail(IGAMG_EINVAL, "not available for a general-operator context");
    if (igamg_status st = check_ctx(c)) return st;
    if (modes < 1 || modes > 64 || !h_coeffs || !d_b) return fail(IGAMG_EINVAL, "bad rhs arguments");
    const HostLevel& H = c->hl.back();
    const int dim = c->dim;
    std::vector<double> g[3];
    for (int d = 0; d < dim; ++d) g[d] = sine_moments(H.breaks[d], c->p, modes);
    // H[(kz*modes + ky) * m_x + i] = sum_kx c[kz][ky][kx] gx[kx][i]
    const int mx = H.m[0];
    const int outer = (dim == 3) ? modes * modes : modes;
    std::vector<double> Hx((size_t)outer * mx, 0.0);
    for (int o = 0; o < outer; ++o)
        for (int kx = 0; kx < modes; ++kx) {
            const double cc = h_coeffs[(size_t)o * modes + kx];
            if (cc == 0.0) continue;
            for (int i = 0; i < mx; ++i) Hx[(size_t)o * mx + i] += cc * g[0][(size_t)kx * mx + i];
        }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nH = Hx.size(), nY = g[1].size(), nZ = (dim == 3) ? g[2].size() : 0;
    double* tmp = nullptr;
    CUDA_TRY(cudaMallocAsync((void**)&tmp, (nH + nY + nZ + 1) * sizeof(double), s));
    CUDA_TRY(cudaMemcpyAsync(tmp, Hx.data(), nH * 8, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(tmp + nH, g[1].data(), nY * 8, cudaMemcpyHostToDevice, s));
    if (nZ) CUDA_TRY(cudaMemcpyAsync(tmp + nH + nY, g[2].data(), nZ * 8, cudaMemcpyHostToDevice, s));
    dev::rhs_sine(s, dim, H.m, modes, tmp, tmp + nH, nZ ? tmp + nH + nY : nullptr, d_b);
    CUDA_TRY(cudaFreeAsync(tmp, s));
    CUDA_TRY(cudaStreamSynchronize(s));       // host staging vectors go out of scope
    CUDA_TRY(cudaGetLastError());
    return IGAMG_OK;
}

igamg_status igamg_solve(igamg_ctx* c, const double* d_b, double* d_x, double tol, int extrap, int k,
                         int max_cycles, int prec, unsigned flags, void* d_ws, size_t ws_bytes,
                         void* stream, double* h_hist, int* h_cycles, int* h_vcycles) {
    if (igamg_status st = check_ctx(c)) return st;
    if (!d_b || !d_x) return fail(IGAMG_EINVAL, "null vector");
    if (extrap < 0 || extrap > 2 || prec < 0 || prec > 2) return fail(IGAMG_EINVAL, "bad extrap/prec");
    if (prec == IGAMG_FP32_IR_LEARNED && !c->cnn_w) return fail(IGAMG_EINVAL, "no learned smoother set");
    if (prec == IGAMG_FP32_IR_LEARNED && !default_cycle(c))
        return fail(IGAMG_EINVAL, "the learned post-smoother replaces Gauss-Seidel in the V-cycle (igamg_set_cycle)");
    c->fell_back = 0;
    if (c->general && (!c->gen_ready || prec != IGAMG_FP64))
        return fail(IGAMG_EINVAL, "general operator: call igamg_assemble_general first; FP64 cycles only");
    if (extrap != IGAMG_EXTRAP_NONE && (k < 1 || k > kMaxQ)) return fail(IGAMG_EINVAL, "k must be in [1, 12]");
    if (max_cycles < 0 || !(tol >= 0.0)) return fail(IGAMG_EINVAL, "bad max_cycles/tol");
    const int kk = (extrap == IGAMG_EXTRAP_NONE) ? 1 : k;
    if (igamg_status st = check_ws(c, d_ws, ws_bytes, kk, prec)) return st;
    Workspace w = carve(c, d_ws, kk, prec);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t N = finestN(c);
    const int top = c->L - 1;
    CUDA_TRY(clear_sync(w, s));
    if (h_cycles) *h_cycles = 0;
    if (h_vcycles) *h_vcycles = 0;
    // ||b|| (denominator of the relative test)
    dev::sumsq_partial(s, d_b, N, w.partial, 256);
    dev::norm_final(s, w.partial, 256, nullptr, w.scal, 0);
    if (flags & IGAMG_FLAG_X0_GIVEN)
        CUDA_TRY(cudaMemcpyAsync(w.S, d_x, N * 8, cudaMemcpyDeviceToDevice, s));
    else
        dev::fill_zero<double>(s, w.S, N);
    if (!c->general)
        dev::xpass<double, double>(s, c->lv64[top], w.S, w.S, nullptr, 0, nullptr, nullptr, 0,
                                   w.d[top].TM, w.d[top].TK);
    const double* denom = (flags & IGAMG_FLAG_ABS_TOL) ? nullptr : w.scal;
    CUDA_TRY(cudaMemcpyAsync(c->h_pin, w.scal, 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    const double bnorm = c->h_pin[0];
    if (!std::isfinite(bnorm)) return fail(IGAMG_EBREAKDOWN, "non-finite right-hand side");
    if (bnorm == 0.0 && !(flags & IGAMG_FLAG_ABS_TOL)) {           // b = 0: x = 0 is exact
        CUDA_TRY(cudaMemsetAsync(d_x, 0, N * 8, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        if (h_hist) h_hist[0] = 0.0;
        return IGAMG_OK;
    }
    residual_norm(c, s, w, d_b, denom);
    CUDA_TRY(cudaMemcpyAsync(c->h_pin, w.scal + 1, 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    CUDA_TRY(cudaGetLastError());
    double res = c->h_pin[0];
    if (h_hist) h_hist[0] = res;
    igamg_status result = IGAMG_ENOTCONV;
    if (res <= tol) result = IGAMG_OK;
    const bool use_graph = !(flags & IGAMG_FLAG_NO_GRAPH);
    // The restart loop of Algorithm 5 runs on the GPU (one graph launch and one
    // synchronisation per solve) unless the caller asks for the host loop, the
    // graph is off, or the learned form may switch smoothers between cycles.
    const bool device_loop = use_graph && !(flags & IGAMG_FLAG_HOST_LOOP) && prec != IGAMG_FP32_IR_LEARNED &&
                             max_cycles < kLoopHist;
    if (device_loop && result != IGAMG_OK && max_cycles > 0) {
        if (igamg_status st = ensure_loop_graph(c, w, d_b, d_ws, kk, extrap, prec, denom)) return st;
        LoopState* hs = c->h_loop;
        hs->cyc = 0;
        hs->max_cycles = max_cycles;
        hs->code = kLoopRunning;
        hs->pad = 0;
        hs->tol = tol;
        hs->res = res;
        CUDA_TRY(cudaMemcpyAsync(w.loop, hs, sizeof(LoopState), cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaGraphLaunch(c->loop_exec[prec], s));
        CUDA_TRY(cudaMemcpyAsync(hs, w.loop, sizeof(LoopState), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaMemcpyAsync(c->h_hist, w.hist, sizeof(double) * (max_cycles + 1), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        const int n = hs->cyc;
        count_launch((long long)n * c->loop_body_launches[prec]);
        if (h_hist)
            for (int i = 1; i <= n; ++i) h_hist[i] = c->h_hist[i];
        if (h_cycles) *h_cycles = n;
        if (h_vcycles) *h_vcycles = n * (extrap == IGAMG_EXTRAP_NONE ? 1 : kk + 1);
        switch (hs->code) {
            case kLoopConverged: result = IGAMG_OK; break;
            case kLoopBreakdown: result = fail(IGAMG_EBREAKDOWN, "non-finite residual"); break;
            case kLoopTimeout:
                result = fail(IGAMG_ETIMEOUT, "a bounded device-side wait of a Gauss-Seidel sweep gave up");
                break;
            default: result = IGAMG_ENOTCONV; break;
        }
        max_cycles = 0;                                // the host loop below has nothing left to do
    }
    int cur = prec;                                    // the learned form may fall back to plain smoothing
    if (use_graph && result != IGAMG_OK && max_cycles > 0)
        if (igamg_status st = ensure_graph(c, w, d_b, d_ws, kk, extrap, cur, denom)) return st;
    int cyc = 0;
    for (cyc = 1; cyc <= max_cycles && result != IGAMG_OK; ++cyc) {
        const int slot = cur;
        if (use_graph) {
            CUDA_TRY(cudaGraphLaunch(c->exec[slot], s));
            count_launch(c->exec_launches[slot]);
        } else {
            restart_body(c, s, w, extrap, kk, cur, d_b, denom);
        }
        CUDA_TRY(cudaMemcpyAsync(c->h_pin, w.scal + 1, 8, cudaMemcpyDeviceToHost, s));
        unsigned* h_err = reinterpret_cast<unsigned*>(c->h_pin + 2);
        CUDA_TRY(cudaMemcpyAsync(h_err, w.err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        const double prev = res;
        res = c->h_pin[0];
        if (*h_err) {
            result = IGAMG_ETIMEOUT;
            fail(result, "a bounded device-side wait of a Gauss-Seidel sweep gave up");
            break;
        }
        if (h_hist) h_hist[cyc] = res;
        if (h_cycles) *h_cycles = cyc;
        if (h_vcycles) *h_vcycles = cyc * (extrap == IGAMG_EXTRAP_NONE ? 1 : kk + 1);
        if (!std::isfinite(res)) { result = IGAMG_EBREAKDOWN; fail(result, "non-finite residual"); break; }
        if (res <= tol) { result = IGAMG_OK; break; }
        if (cur == IGAMG_FP32_IR_LEARNED && res > c->stall * prev) {
            // the network stalled: plain multicolour Gauss-Seidel post-smoothing from here on
            cur = IGAMG_FP32_IR;
            c->fell_back = 1;
            if (use_graph)
                if (igamg_status st = ensure_graph(c, w, d_b, d_ws, kk, extrap, cur, denom)) return st;
        }
    }
    CUDA_TRY(cudaMemcpyAsync(d_x, w.S, N * 8, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    CUDA_TRY(cudaGetLastError());
    if (result == IGAMG_ENOTCONV) fail(result, "max_cycles reached");
    return result;
}

igamg_status igamg_device_status(const igamg_ctx* c, void* d_ws, size_t ws_bytes, void* stream) {
    if (igamg_status st = check_ctx(c)) return st;
    if (!d_ws || ((uintptr_t)d_ws & 255)) return fail(IGAMG_EINVAL, "bad workspace");
    const Workspace w = carve(c, d_ws, 1, IGAMG_FP64);
    if (ws_bytes < (size_t)((char*)(w.sync + w.nsync) - (char*)d_ws)) return fail(IGAMG_EINVAL, "workspace too small");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned* h_err = reinterpret_cast<unsigned*>(c->h_pin + 2);
    CUDA_TRY(cudaMemcpyAsync(h_err, w.err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (*h_err) {
        CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(unsigned), s));
        CUDA_TRY(cudaStreamSynchronize(s));
        return fail(IGAMG_ETIMEOUT, "a bounded device-side wait of a Gauss-Seidel sweep gave up");
    }
    return IGAMG_OK;
}

void igamg_profile_start(void) { profile_start(); }

long igamg_profile_stop(int cap, char* h_names, int name_len, double* h_us, int* h_grid) {
    return profile_stop(cap, h_names, name_len, h_us, h_grid);
}

void igamg_set_wait_limit(double seconds, int test_unset_flag) {
    set_wait_limit(seconds > 0 ? (long long)(seconds * 1e9) : 0, test_unset_flag);
}

igamg_status igamg_set_sweep_form(igamg_ctx* c, int single_launch_fp32, int single_launch_fp64) {
    if (igamg_status st = check_ctx(c, false)) return st;
    if (single_launch_fp32 < -1 || single_launch_fp64 < -1)
        return fail(IGAMG_EINVAL, "sweep form: -1 unchanged, 0 never, 1 always, N >= 2 on levels of >= N rows");
    auto rows = [](int v) { return v == 0 ? igamg_ctx::kNever : v; };
    if (single_launch_fp32 >= 0) c->flow32 = rows(single_launch_fp32);
    if (single_launch_fp64 >= 0) c->flow64 = rows(single_launch_fp64);
    drop_graphs(c);
    return IGAMG_OK;
}

void igamg_get_sweep_form(const igamg_ctx* c, int* single_launch_fp32, int* single_launch_fp64) {
    auto v = [](int r) { return r >= igamg_ctx::kNever ? 0 : r; };
    if (single_launch_fp32) *single_launch_fp32 = c ? v(c->flow32) : 0;
    if (single_launch_fp64) *single_launch_fp64 = c ? v(c->flow64) : 0;
}

igamg_status igamg_apply(igamg_ctx* c, int level, const double* d_x, double* d_y, void* d_ws,
                         size_t ws_bytes, void* stream) {
    if (igamg_status st = check_ctx(c)) return st;
    if (level < 0 || level >= c->L || !d_x || !d_y) return fail(IGAMG_EINVAL, "bad apply arguments");
    if (igamg_status st = check_ws(c, d_ws, ws_bytes, 1, IGAMG_FP64)) return st;
    Workspace w = carve(c, d_ws, 1, IGAMG_FP64);
    cudaStream_t s = (cudaStream_t)stream;
    LevelBuf<double>& B = w.d[level];
    if (c->general) {
        if (!c->gen_ready) return fail(IGAMG_EINVAL, "call igamg_assemble_general first");
        dev::gen_residual(s, c->sv[level], d_x, nullptr, d_y, nullptr);
        CUDA_TRY(cudaGetLastError());
        return IGAMG_OK;
    }
    dev::xpass<double, double>(s, c->lv64[level], d_x, nullptr, nullptr, 0, nullptr, nullptr, 0, B.TM, B.TK);
    dev::residual<double, double>(s, c->dim, c->lv64[level], nullptr, B.TM, B.TK, d_y, nullptr, nullptr, B.tmp1,
                                  B.tmp2);
    CUDA_TRY(cudaGetLastError());
    return IGAMG_OK;
}

igamg_status igamg_smooth(igamg_ctx* c, int level, double* d_x, const double* d_b, int descending,
                          void* d_ws, size_t ws_bytes, void* stream) {
    if (igamg_status st = check_ctx(c)) return st;
    if (level < 0 || level >= c->L || !d_x || !d_b) return fail(IGAMG_EINVAL, "bad smooth arguments");
    if (igamg_status st = check_ws(c, d_ws, ws_bytes, 1, IGAMG_FP64)) return st;
    Workspace w = carve(c, d_ws, 1, IGAMG_FP64);
    cudaStream_t s = (cudaStream_t)stream;
    LevelBuf<double>& B = w.d[level];
    if (c->general) {
        if (!c->gen_ready) return fail(IGAMG_EINVAL, "call igamg_assemble_general first");
        dev::gen_gs_sweep(s, c->sv[level], descending != 0, d_x, d_b);
        CUDA_TRY(cudaGetLastError());
        return IGAMG_OK;
    }
    dev::xpass<double, double>(s, c->lv64[level], d_x, nullptr, nullptr, 0, nullptr, nullptr, 0, B.TM, B.TK);
    CUDA_TRY(clear_sync(w, s));
    sweep<double>(c, s, w, level, descending != 0, d_x, d_b, B.TM, B.TK);
    CUDA_TRY(cudaGetLastError());
    return IGAMG_OK;
}

igamg_status igamg_smooth_f32(igamg_ctx* c, int level, float* d_x, const float* d_b, int descending,
                              int sums_current, void* d_ws, size_t ws_bytes, void* stream) {
    if (igamg_status st = check_ctx(c)) return st;
    if (c && c->general) return fail(IGAMG_EINVAL, "not available for a general-operator context");
    if (level < 0 || level >= c->L || !d_x || !d_b) return fail(IGAMG_EINVAL, "bad smooth arguments");
    if (igamg_status st = check_ws(c, d_ws, ws_bytes, 1, IGAMG_FP32_IR)) return st;
    Workspace w = carve(c, d_ws, 1, IGAMG_FP32_IR);
    cudaStream_t s = (cudaStream_t)stream;
    LevelBuf<float>& B = w.f[level];
    if (!sums_current) {
        CUDA_TRY(clear_sync(w, s));
        dev::xpass<float, float>(s, c->lv32[level], d_x, nullptr, nullptr, 0, nullptr, nullptr, 0, B.TM, B.TK);
    }
    sweep<float>(c, s, w, level, descending != 0, d_x, d_b, B.TM, B.TK);
    CUDA_TRY(cudaGetLastError());
    return IGAMG_OK;
}

igamg_status igamg_restrict(igamg_ctx* c, int level, const double* d_fine, double* d_coarse, void* d_ws,
                            size_t ws_bytes, void* stream) {
    if (igamg_status st = check_ctx(c)) return st;
    if (level < 1 || level >= c->L || !d_fine || !d_coarse) return fail(IGAMG_EINVAL, "bad restrict arguments");
    if (igamg_status st = check_ws(c, d_ws, ws_bytes, 1, IGAMG_FP64)) return st;
    Workspace w = carve(c, d_ws, 1, IGAMG_FP64);
    dev::restrict_<double>((cudaStream_t)stream, c->dim, c->tv64[level], d_fine, d_coarse, w.d[level].tmp1,
                           w.d[level].tmp2);
    CUDA_TRY(cudaGetLastError());
    return IGAMG_OK;
}

igamg_status igamg_prolong(igamg_ctx* c, int level, const double* d_coarse, double* d_fine, void* d_ws,
                           size_t ws_bytes, void* stream) {
    if (igamg_status st = check_ctx(c)) return st;
    if (level < 1 || level >= c->L || !d_fine || !d_coarse) return fail(IGAMG_EINVAL, "bad prolong arguments");
    if (igamg_status st = check_ws(c, d_ws, ws_bytes, 1, IGAMG_FP64)) return st;
    Workspace w = carve(c, d_ws, 1, IGAMG_FP64);
    LevelBuf<double>& B = w.d[level];
    dev::prolong_add<double>((cudaStream_t)stream, c->dim, c->tv64[level], c->lv64[level], d_coarse, d_fine,
                             B.TM, B.TK, B.tmp1, B.tmp2);
    CUDA_TRY(cudaGetLastError());
    return IGAMG_OK;
}

igamg_status igamg_coarse_solve(igamg_ctx* c, const double* d_r, double* d_e, void* stream) {
    if (igamg_status st = check_ctx(c)) return st;
    if (!d_r || !d_e) return fail(IGAMG_EINVAL, "null vector");
    dev::coarse_solve<double>((cudaStream_t)stream, c->dim, c->cv64, d_r, d_e);
    CUDA_TRY(cudaGetLastError());
    return IGAMG_OK;
}

igamg_status igamg_vcycle(igamg_ctx* c, double* d_x, const double* d_b, int prec, void* d_ws, size_t ws_bytes,
                          void* stream) {
    if (igamg_status st = check_ctx(c)) return st;
    if (!d_x || !d_b || prec < 0 || prec > 2) return fail(IGAMG_EINVAL, "bad vcycle arguments");
    if (c->general && (!c->gen_ready || prec != IGAMG_FP64))
        return fail(IGAMG_EINVAL, "general operator: call igamg_assemble_general first; FP64 cycles only");
    if (prec == IGAMG_FP32_IR_LEARNED && !c->cnn_w) return fail(IGAMG_EINVAL, "no learned smoother set");
    if (prec == IGAMG_FP32_IR_LEARNED && !default_cycle(c))
        return fail(IGAMG_EINVAL, "the learned post-smoother replaces Gauss-Seidel in the V-cycle (igamg_set_cycle)");
    if (igamg_status st = check_ws(c, d_ws, ws_bytes, 1, prec)) return st;
    Workspace w = carve(c, d_ws, 1, prec);
    cudaStream_t s = (cudaStream_t)stream;
    const int top = c->L - 1;
    CUDA_TRY(clear_sync(w, s));
    if (!c->general)
        dev::xpass<double, double>(s, c->lv64[top], d_x, nullptr, nullptr, 0, nullptr, nullptr, 0, w.d[top].TM,
                                   w.d[top].TK);
    fixed_point_step(c, s, w, prec, d_b, d_x, d_x);
    CUDA_TRY(cudaGetLastError());
    return IGAMG_OK;
}

size_t igamg_extrap_workspace_bytes(long n, int q) {
    if (n <= 0 || q < 1 || q > kMaxQ) return 0;
    const size_t np = (size_t)(q + 1) * (q + 2) / 2;
    return ((size_t)dev::gram_blocks((size_t)n) * np * 8 + 255) / 256 * 256 + 512 +
           (sizeof(ExtrapInfo) + 255) / 256 * 256;
}

igamg_status igamg_extrapolate(long n, int q, int method, const double* d_S, long ld, double* d_t,
                               double* h_gamma, int* h_qused, void* d_ws, size_t ws_bytes, void* stream) {
    if (n <= 0 || q < 1 || q > kMaxQ || (method != IGAMG_RRE && method != IGAMG_MPE) || !d_S || !d_t || ld < n)
        return fail(IGAMG_EINVAL, "bad extrapolation arguments");
    if (!d_ws || ws_bytes < igamg_extrap_workspace_bytes(n, q) || ((uintptr_t)d_ws & 255))
        return fail(IGAMG_EINVAL, "workspace missing, unaligned or too small");
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = dev::gram_blocks((size_t)n);
    const size_t np = (size_t)(q + 1) * (q + 2) / 2;
    double* partial = (double*)d_ws;
    char* tail = (char*)d_ws + ((size_t)nb * np * 8 + 255) / 256 * 256;
    double* gamma = (double*)tail;
    int* qused = (int*)(tail + 256);
    ExtrapInfo* info = (ExtrapInfo*)(tail + 512);
    dev::extrap_gammas(s, q, method, d_S, (size_t)ld, (size_t)n, partial, nb, info, gamma, qused);
    dev::combine(s, q, gamma, d_S, (size_t)ld, (size_t)n, d_t);
    double hg[kMaxQ + 2];
    int hq = 0;
    CUDA_TRY(cudaMemcpyAsync(hg, gamma, (q + 2) * 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(&hq, qused, 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    CUDA_TRY(cudaGetLastError());
    if (h_gamma) std::memcpy(h_gamma, hg, (q + 2) * 8);
    if (h_qused) *h_qused = hq;
    return IGAMG_OK;
}

igamg_status igamg_set_smoother(igamg_ctx* c, const float* d_w, double stall_ratio) {
    if (c && c->general) return fail(IGAMG_EINVAL, "not available for a general-operator context");
    if (igamg_status st = check_ctx(c)) return st;
    if (!(stall_ratio > 0.0)) return fail(IGAMG_EINVAL, "stall ratio must be positive");
    if (d_w && c->dim != 2) return fail(IGAMG_EINVAL, "the learned smoother is a 2D network");
    c->cnn_w = d_w;
    c->stall = stall_ratio;
    return IGAMG_OK;
}

int igamg_smoother_fell_back(const igamg_ctx* c) { return c ? c->fell_back : 0; }

int igamg_coarse_tail_level(const igamg_ctx* c) {
    return (c && c->assembled) ? tail_level(c) : 0;
}

static void drop_graphs(igamg_ctx* c) {
    for (int sl = 0; sl < 3; ++sl) {
        if (c->exec[sl]) {
            cudaGraphExecDestroy(c->exec[sl]);
            c->exec[sl] = nullptr;
            c->key[sl] = igamg_ctx::Key{};
        }
        if (c->loop_exec[sl]) {
            cudaGraphExecDestroy(c->loop_exec[sl]);
            c->loop_exec[sl] = nullptr;
            c->loop_key[sl] = igamg_ctx::Key{};
        }
    }
}

igamg_status igamg_set_schedule(igamg_ctx* c, int gs_threads, int tail_levels) {
    if (igamg_status st = check_ctx(c)) return st;
    if (gs_threads != 0 && gs_threads != 128 && gs_threads != 256 && gs_threads != 512)
        return fail(IGAMG_EINVAL, "gs_threads must be 0, 128, 256 or 512");
    if (tail_levels < -1) return fail(IGAMG_EINVAL, "tail_levels must be >= -1");
    c->gs_cap32 = gs_threads;
    if (tail_levels >= 0) select_tail(c, c->tail_ctas, tail_levels);
    drop_graphs(c);
    return IGAMG_OK;
}

igamg_status igamg_set_tail_ctas(igamg_ctx* c, int ctas) {
    if (igamg_status st = check_ctx(c)) return st;
    if (ctas != 1 && ctas != kTailCtas[0] && ctas != kTailCtas[1])
        return fail(IGAMG_EINVAL, "tail CTAs must be 1, 8 or 16");
    // the same tail depth where the other form has it, else its deepest
    const int want = c->tail_on ? tail_level(c) : 0;
    select_tail(c, ctas, want > 0 ? want : tail_most(c, ctas));
    drop_graphs(c);
    return IGAMG_OK;
}

int igamg_get_tail_ctas(const igamg_ctx* c) { return c ? c->tail_ctas : 1; }

int igamg_tail_levels_available(const igamg_ctx* c, int ctas) {
    return (c && c->assembled) ? tail_most(c, ctas) : 0;
}

igamg_status igamg_set_cycle(igamg_ctx* c, int smoother, int mu, double omega) {
    if (igamg_status st = check_ctx(c)) return st;
    if ((smoother != IGAMG_SMOOTH_GS && smoother != IGAMG_SMOOTH_JACOBI) || (mu != 1 && mu != 2))
        return fail(IGAMG_EINVAL, "smoother must be IGAMG_SMOOTH_GS or IGAMG_SMOOTH_JACOBI, mu 1 or 2");
    if (smoother == IGAMG_SMOOTH_JACOBI && !(omega > 0.0 && omega < 2.0))
        return fail(IGAMG_EINVAL, "Jacobi weight must lie in (0, 2)");
    c->smoother = smoother;
    c->mu = mu;
    if (smoother == IGAMG_SMOOTH_JACOBI) c->omega = omega;
    drop_graphs(c);
    return IGAMG_OK;
}

void igamg_get_cycle(const igamg_ctx* c, int* smoother, int* mu, double* omega) {
    if (smoother) *smoother = c ? c->smoother : 0;
    if (mu) *mu = c ? c->mu : 1;
    if (omega) *omega = c ? c->omega : 2.0 / 3.0;
}

void igamg_set_launch_overlap(int enable) { set_launch_overlap(enable != 0); }
int igamg_get_launch_overlap(void) { return launch_overlap() ? 1 : 0; }

void igamg_get_schedule(const igamg_ctx* c, int* gs_threads, int* tail_levels) {
    if (gs_threads) *gs_threads = c ? c->gs_cap32 : 0;
    if (tail_levels) *tail_levels = (c && c->assembled) ? tail_level(c) : 0;
}

igamg_status igamg_autotune(igamg_ctx* c, void* d_ws, size_t ws_bytes, void* stream, int reps) {
    if (igamg_status st = check_ctx(c)) return st;
    if (c && c->general) return fail(IGAMG_EINVAL, "not available for a general-operator context");
    if (reps < 1) return fail(IGAMG_EINVAL, "reps must be >= 1");
    if (igamg_status st = check_ws(c, d_ws, ws_bytes, 1, IGAMG_FP32_IR)) return st;
    Workspace w = carve(c, d_ws, 1, IGAMG_FP32_IR);
    cudaStream_t s = (cudaStream_t)stream;
    const int top = c->L - 1;
    LevelBuf<float>& G = w.f[top];
    const size_t N = finestN(c);
    CUDA_TRY(clear_sync(w, s));
    // a right side with every frequency: b = 1 (x = 0 at the start of every cycle)
    CUDA_TRY(cudaMemsetAsync(G.b, 0x3f, N * sizeof(float), s));       // 0x3f3f3f3f = 0.747
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    // on any error: the schedule found on entry, no leaked events, no graphs
    // captured with a trial schedule
    struct Restore {
        igamg_ctx* c;
        cudaEvent_t *e0, *e1;
        int cap, flow32, flow64;
        bool tail_on;
        TailView<float> tail;
        int tail_ctas;
        ClusterTailView<float> ctail;
        bool armed = true;
        ~Restore() {
            if (*e0) cudaEventDestroy(*e0);
            if (*e1) cudaEventDestroy(*e1);
            if (!armed) return;
            c->gs_cap32 = cap;
            c->flow32 = flow32;
            c->flow64 = flow64;
            c->tail_on = tail_on;
            c->tail32 = tail;
            c->tail_ctas = tail_ctas;
            c->ctail32 = ctail;
            drop_graphs(c);
        }
    } restore{c, &e0, &e1, c->gs_cap32, c->flow32, c->flow64, c->tail_on, c->tail32, c->tail_ctas, c->ctail32};
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    const int caps[3] = {128, 256, 512};
    // one-launch sweep thresholds tried (rows per level; kNever = row phases only)
    const int flows[3] = {igamg_ctx::kNever, 16384, 4096};
    auto time_cycles = [&](auto tag, float* ms) -> igamg_status {
        using T = decltype(tag);
        auto& B = Views<T>::buf(w);
        T* x = B[top].x;
        const T* b = B[top].b;
        if constexpr (std::is_same<T, double>::value)     // FP64 cycles: a constant right side too
            CUDA_TRY(cudaMemsetAsync(B[top].b, 0x3f, lv64_n(c, top) * sizeof(double), s));
        vcycle<T>(c, s, w, top, x, b, true);                               // warm-up
        CUDA_TRY(cudaEventRecord(e0, s));
        for (int r = 0; r < reps; ++r) vcycle<T>(c, s, w, top, x, b, true);
        CUDA_TRY(cudaEventRecord(e1, s));
        CUDA_TRY(cudaEventSynchronize(e1));
        CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
        return IGAMG_OK;
    };
    // coarse tails tried: none, then each depth on one CTA and on each cluster size
    std::vector<std::pair<int, int>> tails_tried{{1, 0}};
    for (int ctas : {1, kTailCtas[0], kTailCtas[1]})
        if (ctas == 1 || c->tune_clusters)
            for (int lc = 1; lc <= tail_most(c, ctas); ++lc) tails_tried.push_back({ctas, lc});
    float best = 1e30f;
    int best_cap = 0, best_flow = c->flow32;
    std::pair<int, int> best_tail{c->tail_ctas, tail_level(c)};
    for (int fi = 0; fi < 3; ++fi)
        for (int ci = 0; ci < (c->dim == 2 ? 3 : 1); ++ci)
            for (const auto& tt : tails_tried) {
                c->flow32 = flows[fi];
                c->gs_cap32 = c->dim == 2 ? caps[ci] : 0;
                select_tail(c, tt.first, tt.second);
                float ms = 0.f;
                if (igamg_status st = time_cycles(0.0f, &ms)) return st;
                if (ms < best) { best = ms; best_cap = c->gs_cap32; best_tail = tt; best_flow = c->flow32; }
            }
    c->gs_cap32 = best_cap;
    select_tail(c, best_tail.first, best_tail.second);
    c->flow32 = best_flow;
    // FP64 cycles: the sweep form only (on the same workspace; b = the FP32 b in FP64)
    float best64 = 1e30f;
    int best_flow64 = c->flow64;
    for (int fi = 0; fi < 3; ++fi) {
        c->flow64 = flows[fi];
        float ms = 0.f;
        if (igamg_status st = time_cycles(0.0, &ms)) return st;
        if (ms < best64) { best64 = ms; best_flow64 = c->flow64; }
    }
    c->flow64 = best_flow64;
    CUDA_TRY(cudaGetLastError());
    restore.armed = false;
    drop_graphs(c);
    return IGAMG_OK;
}

igamg_status igamg_set_coarse_tail(igamg_ctx* c, int enable) {
    if (igamg_status st = check_ctx(c)) return st;
    const bool on = enable != 0;
    if (on == c->tail_on) return IGAMG_OK;
    c->tail_on = on && tail_most(c, c->tail_ctas) > 0;
    drop_graphs(c);                             // recapture with the other form
    return IGAMG_OK;
}

igamg_status igamg_vcycle_probe(igamg_ctx* c, double* d_x, const double* d_b, double* d_x_mid, void* d_ws,
                                size_t ws_bytes, void* stream) {
    if (c && !default_cycle(c)) return fail(IGAMG_EINVAL, "the probe follows the Gauss-Seidel V-cycle");
    if (c && c->general) return fail(IGAMG_EINVAL, "not available for a general-operator context");
    if (igamg_status st = check_ctx(c)) return st;
    if (!d_x || !d_b || !d_x_mid) return fail(IGAMG_EINVAL, "bad probe arguments");
    if (igamg_status st = check_ws(c, d_ws, ws_bytes, 1, IGAMG_FP64)) return st;
    Workspace w = carve(c, d_ws, 1, IGAMG_FP64);
    cudaStream_t s = (cudaStream_t)stream;
    const int top = c->L - 1;
    CUDA_TRY(clear_sync(w, s));
    dev::xpass<double, double>(s, c->lv64[top], d_x, nullptr, nullptr, 0, nullptr, nullptr, 0, w.d[top].TM,
                               w.d[top].TK);
    vcycle<double>(c, s, w, top, d_x, d_b, false, false, d_x_mid);
    CUDA_TRY(cudaGetLastError());
    return IGAMG_OK;
}

size_t igamg_training_workspace_bytes(const igamg_ctx* c, int k) {
    if (!c || k < 1 || k > kMaxQ) return 0;
    return carve(c, nullptr, k, IGAMG_FP64).bytes + 3 * (((finestN(c) * sizeof(double)) + 255) & ~(size_t)255) + 256;
}

igamg_status igamg_training_pairs(igamg_ctx* c, const double* d_b, const double* d_uh, int k, double tol,
                                  int max_restarts, float* d_R, float* d_E, int max_pairs, void* d_ws,
                                  size_t ws_bytes, void* stream, int* h_pairs) {
    if (c && !default_cycle(c)) return fail(IGAMG_EINVAL, "the probe follows the Gauss-Seidel V-cycle");
    if (c && c->general) return fail(IGAMG_EINVAL, "not available for a general-operator context");
    if (igamg_status st = check_ctx(c)) return st;
    if (!d_b || !d_uh || !d_R || !d_E || !h_pairs || k < 1 || k > kMaxQ || max_restarts < 1 || max_pairs < 0 ||
        !(tol >= 0.0))
        return fail(IGAMG_EINVAL, "bad training-pair arguments");
    if (!d_ws || ((uintptr_t)d_ws & 255)) return fail(IGAMG_EINVAL, "bad workspace");
    if (ws_bytes < igamg_training_workspace_bytes(c, k)) return fail(IGAMG_ENOMEM, "training workspace too small");
    Workspace w = carve(c, d_ws, k, IGAMG_FP64);
    const size_t N = finestN(c);
    const size_t vb = ((N * sizeof(double)) + 255) & ~(size_t)255;
    char* extra = (char*)d_ws + ((w.bytes + 255) & ~(size_t)255);
    double* mid = (double*)extra;                   // iterate before the finest post-smoothing
    double* r64 = (double*)(extra + vb);            // b - A mid
    double* e64 = (double*)(extra + 2 * vb);        // u_h - mid
    cudaStream_t s = (cudaStream_t)stream;
    const int top = c->L - 1;
    LevelBuf<double>& F = w.d[top];
    *h_pairs = 0;
    CUDA_TRY(clear_sync(w, s));
    // ||b||, s_0 = 0 and its row sums
    dev::sumsq_partial(s, d_b, N, w.partial, 256);
    dev::norm_final(s, w.partial, 256, nullptr, w.scal, 0);
    dev::fill_zero<double>(s, w.S, N);
    dev::xpass<double, double>(s, c->lv64[top], w.S, w.S, nullptr, 0, nullptr, nullptr, 0, F.TM, F.TK);
    int pairs = 0;
    for (int rs = 0; rs < max_restarts; ++rs) {
        for (int j = 0; j <= k; ++j) {
            double* Sj = w.S + (size_t)j * w.ld;
            double* Sn = w.S + (size_t)(j + 1) * w.ld;
            CUDA_TRY(cudaMemcpyAsync(Sn, Sj, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
            vcycle<double>(c, s, w, top, Sn, d_b, false, false, mid);            // s_{j+1} = G(s_j), probed
            if (pairs < max_pairs) {
                // e = u_h - mid, r = b - A mid (row sums of mid in F.r / F.tmp2), unit RMS of e
                dev::diff_sumsq(s, d_uh, mid, N, e64, w.partial, 256);
                dev::norm_final(s, w.partial, 256, nullptr, w.scal, 2);
                dev::xpass<double, double>(s, c->lv64[top], mid, nullptr, nullptr, 0, nullptr, nullptr, 0, F.r,
                                           F.tmp2);
                dev::residual<double, double>(s, c->dim, c->lv64[top], d_b, F.r, F.tmp2, r64, nullptr);
                dev::scale_pair(s, r64, e64, w.scal + 2, N, d_R + (size_t)pairs * N, d_E + (size_t)pairs * N);
                ++pairs;
            }
        }
        // t = RRE(s_0..s_{k+1}) (Algorithm 3), s_0 := t, ||b - A t|| / ||b||
        const int nb = dev::gram_blocks(N);
        dev::extrap_gammas(s, k, IGAMG_RRE, w.S, w.ld, N, w.partial, nb, w.info, w.gamma, w.qused);
        dev::xpass<double, double>(s, c->lv64[top], nullptr, w.S, nullptr, k + 2, w.gamma, w.S, w.ld, F.TM, F.TK);
        residual_norm(c, s, w, d_b, w.scal);
        CUDA_TRY(cudaMemcpyAsync(c->h_pin, w.scal + 1, 8, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        CUDA_TRY(cudaGetLastError());
        if (!std::isfinite(c->h_pin[0])) return fail(IGAMG_EBREAKDOWN, "non-finite residual");
        if (c->h_pin[0] <= tol) break;
    }
    *h_pairs = pairs;
    return IGAMG_OK;
}

void igamg_destroy(igamg_ctx* c) {
    if (!c) return;
    for (int sl = 0; sl < 3; ++sl)
        if (c->exec[sl]) cudaGraphExecDestroy(c->exec[sl]);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->h_pin) cudaFreeHost(c->h_pin);
    for (int sl = 0; sl < 3; ++sl)
        if (c->loop_exec[sl]) cudaGraphExecDestroy(c->loop_exec[sl]);
    if (c->h_loop) cudaFreeHost(c->h_loop);
    if (c->h_hist) cudaFreeHost(c->h_hist);
    if (c->dmem) cudaFree(c->dmem);
    if (c->gmem) cudaFree(c->gmem);
    free_tail_images(c);
    delete c;
}

}  // extern "C"

// ====================================================================== batches
// Many independent problems of uneven size and degree.  Every problem keeps
// its own hierarchy, workspace slice and restart-cycle CUDA graph; a round
// replays one restart cycle of every problem that has not converged, spread
// over a fixed set of streams so that the latency-bound kernels of different
// problems overlap on the GPU, then reads every residual at once.
struct igamg_batch {
    int count = 0, dim = 2;
    std::vector<igamg_ctx*> ctx;
    std::vector<size_t> voff;               // packed-vector offsets, count + 1
    std::vector<int> lane;                  // stream of each problem
    std::vector<cudaStream_t> streams;
    cudaEvent_t ev = nullptr;
    double* h_pin = nullptr;                // 2 per problem: ||b||, last residual
    unsigned* h_err = nullptr;              // per problem: its workspace's device-wait error word
    // device-side loops: one graph whose independent branches are, per
    // problem, an init kernel and a conditional WHILE node around that
    // problem's restart cycle; d_state / h_state: per-problem loop states
    bool device_loop = true;
    LoopState* d_state = nullptr;
    LoopState* h_state = nullptr;
    cudaGraphExec_t loop_exec[2] = {nullptr, nullptr};
    igamg_ctx::Key loop_key[2];
    std::vector<long long> body_launches[2];
};

namespace {
// Measured on GB300 for 256 problems (n ~ U[32,512], p in {2,3,4}): the
// makespan falls from 836 ms (8 streams) to 470 (16), 370 (32), 338 (64) and
// 331 ms (128), then flattens; assigning problems round-robin beat a
// longest-processing-time assignment at every stream count (the round ends
// when every stream has drained, and round-robin mixes large and small
// problems on every stream).
constexpr int kBatchStreams = 128;

std::vector<size_t> batch_ws_offsets(const igamg_batch* B, int k, int prec) {
    std::vector<size_t> off(B->count + 1, 0);
    for (int i = 0; i < B->count; ++i)
        off[i + 1] = off[i] + ((carve(B->ctx[i], nullptr, k, prec).bytes + 255) & ~(size_t)255);
    return off;
}

// The batch's device-side loops in one graph (see igamg_batch::device_loop):
// problem i contributes a root init kernel (condition = state i running) and
// a WHILE node after it whose body is its restart cycle and loop_step.
igamg_status ensure_batch_loop_graph(igamg_batch* B, std::vector<Workspace>& W, const std::vector<size_t>& wo,
                                     const double* d_b, void* d_ws, int k, int extrap, int prec) {
    igamg_ctx::Key key;
    key.b = d_b; key.ws = d_ws; key.k = k; key.extrap = extrap; key.prec = prec;
    key.abs_tol = 0;
    key.overlap = launch_overlap() ? 1 : 0;
    key.sync = sync_generation();
    if (B->loop_exec[prec] && B->loop_key[prec] == key) return IGAMG_OK;
    if (B->loop_exec[prec]) { cudaGraphExecDestroy(B->loop_exec[prec]); B->loop_exec[prec] = nullptr; }
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaGraphCreate(&g, 0));
    struct GraphGuard { cudaGraph_t g; ~GraphGuard() { if (g) cudaGraphDestroy(g); } } guard{g};
    B->body_launches[prec].assign(B->count, 0);
    cudaStream_t cap = B->ctx[0]->cap;
    for (int i = 0; i < B->count; ++i) {
        igamg_ctx* c = B->ctx[i];
        cudaGraphConditionalHandle h;
        CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
        cudaGraphNode_t init;
        CUDA_TRY(dev::add_loop_init_node(g, h, B->d_state + i, &init));
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        CUDA_TRY(cudaGraphAddNode(&node, g, &init, nullptr, 1, &np));
        cudaGraph_t body = np.conditional.phGraph_out[0];
        const long long before = launch_count();
        CUDA_TRY(cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        restart_body(c, cap, W[i], extrap, k, prec, d_b + B->voff[i], W[i].scal);
        dev::loop_step(cap, h, B->d_state + i, W[i].scal + 1, W[i].err, nullptr);
        cudaGraph_t got = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(cap, &got);
        B->body_launches[prec][i] = launch_count() - before;
        count_launch(-B->body_launches[prec][i]);
        if (ce != cudaSuccess) return fail(IGAMG_ECUDA, std::string("batch loop capture: ") + cudaGetErrorString(ce));
    }
    const cudaError_t ce = cudaGraphInstantiate(&B->loop_exec[prec], g, 0);
    if (ce != cudaSuccess) {
        B->loop_exec[prec] = nullptr;
        return fail(IGAMG_ECUDA, std::string("batch loop instantiate: ") + cudaGetErrorString(ce));
    }
    B->loop_key[prec] = key;
    return IGAMG_OK;
}
}  // namespace

extern "C" {

igamg_status igamg_batch_create(int count, int dim, const int* p, const int* n, igamg_batch** out) {
    if (!out || !p || !n || count < 1) return fail(IGAMG_EINVAL, "bad batch arguments");
    *out = nullptr;
    igamg_batch* B = new (std::nothrow) igamg_batch();
    if (!B) return fail(IGAMG_ENOMEM, "host allocation");
    B->count = count;
    B->dim = dim;
    B->voff.assign(count + 1, 0);
    for (int i = 0; i < count; ++i) {
        const int ne[3] = {n[i], n[i], n[i]};
        igamg_ctx* c = nullptr;
        igamg_status st = igamg_setup(dim, p[i], ne, 0, &c);
        if (st == IGAMG_OK) st = igamg_assemble(c);
        if (st != IGAMG_OK) {
            if (c) igamg_destroy(c);
            igamg_batch_destroy(B);
            return st;
        }
        B->ctx.push_back(c);
        B->voff[i + 1] = B->voff[i] + finestN(c);
    }
    B->streams.resize(std::min(count, kBatchStreams));
    for (auto& s : B->streams) CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    B->lane.assign(count, 0);
    for (int i = 0; i < count; ++i) B->lane[i] = i % (int)B->streams.size();
    CUDA_TRY(cudaEventCreateWithFlags(&B->ev, cudaEventDisableTiming));
    CUDA_TRY(cudaMallocHost(&B->h_pin, sizeof(double) * 2 * count));
    CUDA_TRY(cudaMallocHost(&B->h_err, sizeof(unsigned) * count));
    CUDA_TRY(cudaMallocHost(&B->h_state, sizeof(LoopState) * count));
    CUDA_TRY(cudaMalloc(&B->d_state, sizeof(LoopState) * count));
    *out = B;
    return IGAMG_OK;
}

igamg_status igamg_batch_layout(const igamg_batch* B, long* h_offsets) {
    if (!B || !h_offsets) return fail(IGAMG_EINVAL, "null batch or offsets");
    for (int i = 0; i <= B->count; ++i) h_offsets[i] = (long)B->voff[i];
    return IGAMG_OK;
}

size_t igamg_batch_workspace_bytes(const igamg_batch* B, int k, int prec) {
    if (!B || k < 1 || k > kMaxQ || prec < 0 || prec > 1) return 0;
    return batch_ws_offsets(B, k, prec).back() + 256;
}

igamg_status igamg_batch_rhs_sine(igamg_batch* B, int modes, const double* h_coeffs, double* d_b, void* stream) {
    if (!B || !h_coeffs || !d_b || modes < 1) return fail(IGAMG_EINVAL, "bad batch rhs arguments");
    size_t per = 1;
    for (int d = 0; d < B->dim; ++d) per *= (size_t)modes;
    for (int i = 0; i < B->count; ++i)
        if (igamg_status st = igamg_rhs_sine(B->ctx[i], modes, h_coeffs + per * i, d_b + B->voff[i], stream))
            return st;
    return IGAMG_OK;
}

igamg_status igamg_batch_solve(igamg_batch* B, const double* d_b, double* d_x, double tol, int extrap, int k,
                               int max_cycles, int prec, void* d_ws, size_t ws_bytes, void* stream,
                               int* h_cycles, int* h_status, double* h_res) {
    const NoOverlapScope serial;                // many streams: no launch overlap (see device.hpp)
    if (!B || !d_b || !d_x) return fail(IGAMG_EINVAL, "null batch or vector");
    if (extrap < 1 || extrap > 2 || k < 1 || k > kMaxQ || prec < 0 || prec > 1 || max_cycles < 0 || !(tol >= 0.0))
        return fail(IGAMG_EINVAL, "bad batch solve arguments");
    const std::vector<size_t> wo = batch_ws_offsets(B, k, prec);
    if (!d_ws || ((uintptr_t)d_ws & 255) || ws_bytes < wo.back()) return fail(IGAMG_ENOMEM, "batch workspace too small");
    cudaStream_t caller = (cudaStream_t)stream;
    CUDA_TRY(cudaEventRecord(B->ev, caller));
    for (auto s : B->streams) CUDA_TRY(cudaStreamWaitEvent(s, B->ev, 0));
    std::vector<Workspace> W(B->count);
    std::vector<int> cyc(B->count, 0), stat(B->count, IGAMG_ENOTCONV);
    // initial state of every problem: ||b||, s_0 = 0 with its row sums, ||b - A s_0|| / ||b||
    for (int i = 0; i < B->count; ++i) {
        igamg_ctx* c = B->ctx[i];
        cudaStream_t s = B->streams[B->lane[i]];
        W[i] = carve(c, (char*)d_ws + wo[i], k, prec);
        Workspace& w = W[i];
        const size_t N = finestN(c);
        const double* b = d_b + B->voff[i];
        CUDA_TRY(clear_sync(w, s));
        dev::sumsq_partial(s, b, N, w.partial, 256);
        dev::norm_final(s, w.partial, 256, nullptr, w.scal, 0);
        dev::fill_zero<double>(s, w.S, N);
        dev::xpass<double, double>(s, c->lv64[c->L - 1], w.S, w.S, nullptr, 0, nullptr, nullptr, 0,
                                   w.d[c->L - 1].TM, w.d[c->L - 1].TK);
        residual_norm(c, s, w, b, w.scal);
        CUDA_TRY(cudaMemcpyAsync(B->h_pin + 2 * i, w.scal, 16, cudaMemcpyDeviceToHost, s));
    }
    const bool device_loop = B->device_loop;
    if (device_loop) {
        if (igamg_status st = ensure_batch_loop_graph(B, W, wo, d_b, d_ws, k, extrap, prec)) return st;
    } else {
        for (int i = 0; i < B->count; ++i)
            if (igamg_status st = ensure_graph(B->ctx[i], W[i], d_b + B->voff[i], (char*)d_ws + wo[i], k, extrap,
                                               prec, W[i].scal))
                return st;
    }
    for (auto s : B->streams) CUDA_TRY(cudaStreamSynchronize(s));
    CUDA_TRY(cudaGetLastError());
    for (int i = 0; i < B->count; ++i) {
        const double bn = B->h_pin[2 * i], r = B->h_pin[2 * i + 1];
        if (h_res) h_res[i] = r;
        if (!std::isfinite(bn)) stat[i] = IGAMG_EBREAKDOWN;
        else if (bn == 0.0) { stat[i] = IGAMG_OK; if (h_res) h_res[i] = 0.0; }
        else if (r <= tol) stat[i] = IGAMG_OK;
    }
    if (device_loop && max_cycles > 0) {
        // every problem's restart loop on the GPU: one graph launch
        for (int i = 0; i < B->count; ++i) {
            LoopState& ls = B->h_state[i];
            ls.cyc = 0;
            ls.max_cycles = max_cycles;
            ls.code = stat[i] == IGAMG_ENOTCONV ? kLoopRunning : kLoopConverged;
            ls.pad = 0;
            ls.tol = tol;
            ls.res = B->h_pin[2 * i + 1];
        }
        CUDA_TRY(cudaMemcpyAsync(B->d_state, B->h_state, sizeof(LoopState) * B->count, cudaMemcpyHostToDevice,
                                 caller));
        CUDA_TRY(cudaGraphLaunch(B->loop_exec[prec], caller));
        CUDA_TRY(cudaMemcpyAsync(B->h_state, B->d_state, sizeof(LoopState) * B->count, cudaMemcpyDeviceToHost,
                                 caller));
        CUDA_TRY(cudaStreamSynchronize(caller));
        CUDA_TRY(cudaGetLastError());
        for (int i = 0; i < B->count; ++i) {
            if (stat[i] != IGAMG_ENOTCONV) continue;
            const LoopState& ls = B->h_state[i];
            cyc[i] = ls.cyc;
            count_launch((long long)ls.cyc * B->body_launches[prec][i]);
            if (h_res) h_res[i] = ls.res;
            stat[i] = ls.code == kLoopConverged ? IGAMG_OK
                      : ls.code == kLoopBreakdown ? IGAMG_EBREAKDOWN
                      : ls.code == kLoopTimeout ? IGAMG_ETIMEOUT
                                                : IGAMG_ENOTCONV;
        }
        CUDA_TRY(cudaEventRecord(B->ev, caller));
        for (auto s : B->streams) CUDA_TRY(cudaStreamWaitEvent(s, B->ev, 0));
        max_cycles = 0;                             // the per-round host loop below has nothing left to do
    }
    for (int round = 1; round <= max_cycles; ++round) {
        int active = 0;
        for (int i = 0; i < B->count; ++i) {
            if (stat[i] != IGAMG_ENOTCONV) continue;
            cudaStream_t s = B->streams[B->lane[i]];
            CUDA_TRY(cudaGraphLaunch(B->ctx[i]->exec[prec], s));
            count_launch(B->ctx[i]->exec_launches[prec]);
            CUDA_TRY(cudaMemcpyAsync(B->h_pin + 2 * i + 1, W[i].scal + 1, 8, cudaMemcpyDeviceToHost, s));
            ++active;
        }
        if (!active) break;
        for (auto s : B->streams) CUDA_TRY(cudaStreamSynchronize(s));
        for (int i = 0; i < B->count; ++i) {
            if (stat[i] != IGAMG_ENOTCONV) continue;
            const double r = B->h_pin[2 * i + 1];
            cyc[i] = round;
            if (h_res) h_res[i] = r;
            if (!std::isfinite(r)) stat[i] = IGAMG_EBREAKDOWN;
            else if (r <= tol) stat[i] = IGAMG_OK;
        }
    }
    for (int i = 0; i < B->count; ++i) {
        cudaStream_t s = B->streams[B->lane[i]];
        const size_t N = finestN(B->ctx[i]);
        if (stat[i] == IGAMG_OK && B->h_pin[2 * i] == 0.0) CUDA_TRY(cudaMemsetAsync(d_x + B->voff[i], 0, N * 8, s));
        else CUDA_TRY(cudaMemcpyAsync(d_x + B->voff[i], W[i].S, N * 8, cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(B->h_err + i, W[i].err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    }
    for (auto s : B->streams) CUDA_TRY(cudaStreamSynchronize(s));
    CUDA_TRY(cudaGetLastError());
    for (int i = 0; i < B->count; ++i)
        if (B->h_err[i]) stat[i] = IGAMG_ETIMEOUT;
    igamg_status all = IGAMG_OK;
    for (int i = 0; i < B->count; ++i) {
        if (h_cycles) h_cycles[i] = cyc[i];
        if (h_status) h_status[i] = stat[i];
        if (stat[i] != IGAMG_OK && all == IGAMG_OK) all = (igamg_status)stat[i];
    }
    if (all != IGAMG_OK) fail(all, "some problems did not converge");
    return all;
}

igamg_status igamg_batch_set_device_loop(igamg_batch* B, int enable) {
    if (!B) return fail(IGAMG_EINVAL, "null batch");
    B->device_loop = enable != 0;
    return IGAMG_OK;
}

igamg_status igamg_batch_set_tail_ctas(igamg_batch* B, int ctas) {
    if (!B) return fail(IGAMG_EINVAL, "null batch");
    if (ctas != 1 && ctas != kTailCtas[0] && ctas != kTailCtas[1])
        return fail(IGAMG_EINVAL, "tail CTAs must be 1, 8 or 16");
    for (auto c : B->ctx) {
        if (igamg_status st = check_ctx(c)) return st;
        select_tail(c, ctas, tail_most(c, ctas));
        drop_graphs(c);
    }
    for (int sl = 0; sl < 2; ++sl)              // members' cycles change: recapture the loops
        if (B->loop_exec[sl]) {
            cudaGraphExecDestroy(B->loop_exec[sl]);
            B->loop_exec[sl] = nullptr;
            B->loop_key[sl] = igamg_ctx::Key{};
        }
    return IGAMG_OK;
}

igamg_status igamg_batch_autotune(igamg_batch* B, void* d_ws, size_t ws_bytes, void* stream, int reps) {
    const NoOverlapScope serial;                // time the schedules as batched solves run them
    if (!B || !d_ws) return fail(IGAMG_EINVAL, "bad batch autotune arguments");
    for (int sl = 0; sl < 2; ++sl)              // members' schedules change: recapture the loops
        if (B->loop_exec[sl]) {
            cudaGraphExecDestroy(B->loop_exec[sl]);
            B->loop_exec[sl] = nullptr;
            B->loop_key[sl] = igamg_ctx::Key{};
        }
    const std::vector<size_t> off = batch_ws_offsets(B, 1, IGAMG_FP32_IR);
    if (off.back() > ws_bytes) return fail(IGAMG_ENOMEM, "batch workspace too small (size it for IGAMG_FP32_IR)");
    // one tuning run per degree, on the problem of median size; the others
    // take its row-CTA cap and the tail down to the same level size
    std::vector<int> ps;
    for (int i = 0; i < B->count; ++i)
        if (std::find(ps.begin(), ps.end(), B->ctx[i]->p) == ps.end()) ps.push_back(B->ctx[i]->p);
    for (int p : ps) {
        std::vector<int> ids;
        for (int i = 0; i < B->count; ++i)
            if (B->ctx[i]->p == p) ids.push_back(i);
        std::sort(ids.begin(), ids.end(), [&](int a, int b) { return finestN(B->ctx[a]) < finestN(B->ctx[b]); });
        const int m = ids[ids.size() / 2];
        igamg_ctx* cm = B->ctx[m];
        // members run concurrently: a member's cluster tail holds 16 SMs for a
        // latency-bound stretch that the others could use (measured, 256
        // problems: 254 -> 333 ms), so batches tune the one-CTA tail only
        cm->tune_clusters = false;
        const igamg_status tst = igamg_autotune(cm, (char*)d_ws + off[m], off[m + 1] - off[m], stream, reps);
        cm->tune_clusters = true;
        if (tst) return tst;
        const int cap = cm->gs_cap32, ctas = cm->tail_ctas;
        const size_t nthr = tail_level(cm) > 0 ? cm->hl[tail_level(cm)].N() : 0;
        for (int i : ids) {
            if (i == m) continue;
            igamg_ctx* ci = B->ctx[i];
            int lc = 0;
            for (int l = 1; l <= tail_most(ci, ctas); ++l)
                if (ci->hl[l].N() <= nthr) lc = l;
            ci->tail_ctas = ctas;
            if (igamg_status st = igamg_set_schedule(ci, cap, lc)) return st;
        }
    }
    return IGAMG_OK;
}

void igamg_batch_destroy(igamg_batch* B) {
    if (!B) return;
    for (auto c : B->ctx) igamg_destroy(c);
    for (auto s : B->streams) if (s) cudaStreamDestroy(s);
    if (B->ev) cudaEventDestroy(B->ev);
    if (B->h_pin) cudaFreeHost(B->h_pin);
    if (B->h_err) cudaFreeHost(B->h_err);
    if (B->h_state) cudaFreeHost(B->h_state);
    if (B->d_state) cudaFree(B->d_state);
    for (auto& e : B->loop_exec)
        if (e) cudaGraphExecDestroy(e);
    delete B;
}

}  // extern "C"
