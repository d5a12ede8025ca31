// Device-side views and kernel launch wrappers (internal; not part of the C ABI).
#pragma once
#include <cstddef>
#include <string>
#include <cuda_runtime.h>

#ifdef __CUDACC__
#define IGAMG_HD __host__ __device__
#else
#define IGAMG_HD
#endif

namespace igamg {

constexpr int kMaxP = 7;
constexpr int kMaxQ = 12;                 // largest restart number k

// One grid level as the kernels see it.  Grid vectors are rows of length m[0]
// (x fastest); rows are indexed j + m[1] k.  Bands are stored band-major:
// Mb[d][b * m[d] + i] = M_d(i, i + b - p), zero outside the matrix.
template <typename T>
struct LevelView {
    int m[3];
    int p;
    const T* Mb[3];
    const T* Kb[3];
    const T* invdiag;                     // 1 / A_ii
    // per direction d, rows i in [tlo[d], thi[d]) share one band (the uniform
    // interior of an open knot vector) and have all 2p+1 neighbours inside
    // the grid (p <= i < m - p); kernels read it from these parameters
    // instead of Mb/Kb[d].
    int tlo[3], thi[3];
    T Mc[3][2 * kMaxP + 1], Kc[3][2 * kMaxP + 1];
    IGAMG_HD size_t n() const { return (size_t)m[0] * m[1] * m[2]; }
    IGAMG_HD int rows() const { return m[1] * m[2]; }
};

// 1D transfer between a fine level and the next coarser one, direction d.
// Row form of P (prolongation): fine i -> coarse [plo[i], plo[i] + pw).
// Column form (restriction R = P^T): coarse I -> fine [rlo[I], rlo[I] + rw).
template <typename T>
struct TransferView {
    int mf[3], mc[3];
    int pw[3], rw[3];
    const int* plo[3];
    const T* pv[3];
    const int* rlo[3];
    const T* rv[3];
};

// Coarsest-grid fast diagonalisation: A_0^{-1} = V diag(laminv) V^T with
// V = V_z (x) V_y (x) V_x; V[d] is m x m row-major (column I = eigenvector I).
template <typename T>
struct CoarseView {
    int m[3];
    const T* V[3];
    const T* laminv;                      // 1 / (lam_x + lam_y (+ lam_z)), x fastest
};

// Coarse part of a 2D V-cycle run by one CTA (levels 0..lc): the level views,
// the transfers X[l] between levels l-1 and l, the coarsest solve, and the
// shared-memory element offsets of every level's x, b, inverse diagonal,
// four band arrays (M_x, K_x, M_y, K_y, band-major) and row partial sums, and
// of two scratch vectors.  lc = 0 means the hierarchy has no such tail.
constexpr int kTailLevels = 6;
template <typename T>
struct TailView {
    int lc;
    int off_x[kTailLevels], off_b[kTailLevels], off_inv[kTailLevels], off_band[kTailLevels], off_r, off_t;
    int off_tm[kTailLevels];              // T_M then T_K, (m[1] + 2p) x m[0] each
    int off_tc[kTailLevels];              // Toeplitz interior of M_x then K_x (2p+1 each)
    int off_tr[kTailLevels];              // transfer tables of X[l] (see tail_transfer_elems)
    int off_cv;                           // V_x, V_y, laminv of the coarsest solve
    size_t smem;                          // dynamic shared memory in bytes
    LevelView<T> L[kTailLevels];
    TransferView<T> X[kTailLevels];
    CoarseView<T> C;
};

// Coarse part of a 2D V-cycle run by one thread-block cluster of `ctas` CTAs
// (levels 0..lc).  On level q >= 1, CTA r owns the grid rows
// [r R[q], min((r + 1) R[q], m_y)); the coarsest level (R[0] = m_y) is owned
// by CTA 0.  Every CTA keeps its rows' x (zero-padded by p columns on each
// side), b, 1 / A_ii, T_M, T_K and y-band rows in its shared memory and reads
// a neighbour's rows through distributed shared memory.  Offsets (elements)
// are the same in every CTA: off_x, off_b, off_inv, off_tm (T_M then T_K,
// R x m_x each), off_yb (M_y then K_y of the own rows, band-major, W x R
// each), off_xb (M_x then K_x: the boundary columns i < tlo or i >= thi,
// then the Toeplitz interior, (nbc + 1) x W each), off_tx (x-axis
// transfer tables of X[q]: plo, pv, rlo, rv), off_ty (y-axis tables of X[q]:
// pv of the own fine rows, rv of the own coarse rows of level q - 1, then plo
// of the own fine rows and rlo of the own coarse rows), off_rp
// (generic row pointers, 8-byte aligned: the y-band neighbours' T_M rows of
// the own rows, the t rows the own coarse rows' restriction and the own fine
// rows' prolongation combine), off_cv (coarsest V_x, V_y, laminv), off_r and
// off_t (two scratch arrays), off_z (a zero row).  lc = 0: no cluster tail.
constexpr int kCTailLevels = 7;
template <typename T>
struct ClusterTailView {
    int lc, ctas;
    int R[kCTailLevels], nbc[kCTailLevels];
    int off_x[kCTailLevels], off_b[kCTailLevels], off_inv[kCTailLevels], off_tm[kCTailLevels];
    int off_yb[kCTailLevels], off_xb[kCTailLevels], off_tx[kCTailLevels];
    int off_ty[kCTailLevels], off_rp[kCTailLevels];
    int off_cv, off_r, off_t, off_z;
    size_t smem;
    // The static part of every CTA's shared memory (the pointer tables as
    // (owner CTA, element offset) pairs, then the operator data, transfer
    // tables, coarsest eigenbasis and the zero row: elements [0, 4 img16)),
    // built once per context into img[rank * img16 ..] (uint4 units); npair
    // pointer entries start at element 0.
    const uint4* img;
    int img16, npair;
    LevelView<T> L[kCTailLevels];
    TransferView<T> X[kCTailLevels];
    CoarseView<T> C;
};

// Coarse part of a 3D V-cycle on one thread-block cluster (levels 0..lc).
// Grid rows (j, k) are numbered r = k m_y + j; on level q >= 1, CTA c owns
// the rows [c R[q], min((c + 1) R[q], m_y m_z)), and CTA 0 all rows of the
// coarsest level (R[0] = m_y m_z).  Every CTA keeps its rows' x (zero-padded
// by p columns on each side), b, 1 / A_ii, T_M, T_K (with halo copies of the
// H = p m_y + p rows on each side of its range, written by their owners) and
// the (2p+1)^2 row couplings (weights on T_M and T_K) of each own row in
// shared memory, with the level's whole y- and z-bands and the three axes'
// transfer tables.  Offsets (elements): off_rp (8-byte aligned generic
// pointers: the t rows each own coarse row's y-z restriction combines
// (rw_y rw_z) and each own fine row's y-z prolongation combines (pw_y pw_z)),
// off_x, off_b, off_inv, off_tm (T_M then T_K, (R + 2H) x m_x each), off_cc (own rows x (2p+1)^2 weight pairs), off_yb (M_y
// then K_y, W x m_y), off_zb (M_z then K_z, W x m_z), off_xb (M_x then K_x:
// the boundary columns, then the Toeplitz interior, (nbc + 1) x W each),
// off_tx (for axes x, y, z: plo, pv, rlo, rv), off_cv (V_x, V_y, V_z,
// laminv), off_r, off_t (scratch), off_z (a zero row).  lc = 0: none.
template <typename T>
struct ClusterTail3View {
    int lc, ctas;
    int R[kCTailLevels], nbc[kCTailLevels];
    int off_rp[kCTailLevels], off_x[kCTailLevels], off_b[kCTailLevels], off_inv[kCTailLevels];
    int off_tm[kCTailLevels], off_cc[kCTailLevels], off_yb[kCTailLevels], off_zb[kCTailLevels];
    int off_xb[kCTailLevels], off_tx[kCTailLevels];
    int off_cv, off_r, off_t, off_z;
    size_t smem;
    // The static part of every CTA's shared memory, as in ClusterTailView
    // (pointer pairs, operator data with the row weights cc, transfer tables,
    // coarsest eigenbasis, zero row), built once per context.
    const uint4* img;
    int img16, npair;
    LevelView<T> L[kCTailLevels];
    TransferView<T> X[kCTailLevels];
    CoarseView<T> C;
};

// Shared-memory elements (4-byte) of the staged tables of one 2D transfer:
// plo/pv and rlo/rv of both directions.
template <typename T>
IGAMG_HD inline int tail_transfer_elems(const TransferView<T>& X) {
    return X.mf[0] * (1 + X.pw[0]) + X.mf[1] * (1 + X.pw[1]) + X.mc[0] * (1 + X.rw[0]) + X.mc[1] * (1 + X.rw[1]);
}

// The finest 2D or 3D level's 1D factors with every FP64 entry split into a
// float pair (hi = float(v), lo = float(v - hi); hi + lo = v to about 2^-48
// relative), band-major as in LevelView, and the uniform interior's pairs;
// m[2] = 1 in 2D.
struct DFView {
    int m[3], p;
    int tlo[3], thi[3];
    const float *Mh[3], *Ml[3], *Kh[3], *Kl[3];
    float Mch[3][2 * kMaxP + 1], Mcl[3][2 * kMaxP + 1], Kch[3][2 * kMaxP + 1], Kcl[3][2 * kMaxP + 1];
};

// A 2D level of the general operator (Sec. 4.3) in stencil form:
// S[k N + I] = A(I, I + dx + m[0] dy), k = (dy + p)(2p+1) + (dx + p), and the
// inverse diagonal.
struct StencilView {
    int m[2];
    int p;
    const double* S;
    const double* inv;
    IGAMG_HD size_t n() const { return (size_t)m[0] * m[1]; }
};

// Synchronisation words of a single-launch Gauss-Seidel sweep on one level
// (in the caller's workspace).  They are zero before a sweep and every sweep
// leaves them zero, so they are cleared once when a workspace is taken into
// use.  Every wait on them is bounded: after limit_ns the kernel sets bit 0
// of *err and carries on.
struct SweepSync {
    unsigned* done;          // one flag per row of the level
    unsigned* ctr;           // [0] next row claim, [1] CTAs finished
    unsigned* err;           // bit 0: a bounded wait gave up
    const unsigned* never;   // a word nothing sets (tests of the bounded wait)
    long long limit_ns;      // bound of every wait
    int test_unset;          // 1: every CTA first waits on *never
};

// Process-wide bound of the device-side waits and the test switch that makes
// every single-launch sweep wait on a flag nothing sets (read when a sweep is
// enqueued or a graph captured); sync_generation() changes with either.
void set_wait_limit(long long ns, int test_unset);
long long wait_limit_ns();
int wait_test_unset();
int sync_generation();

// Device-side state of the restart loop of Algorithm 5 when the loop runs on
// the GPU (a conditional WHILE node of a CUDA graph around the restart cycle).
enum LoopCode { kLoopRunning = 0, kLoopConverged = 1, kLoopMaxCycles = 2, kLoopBreakdown = 3, kLoopTimeout = 4 };
struct LoopState {
    int cyc;              // restart cycles run
    int max_cycles;
    int code;             // LoopCode
    int pad;
    double tol;           // the accuracy test: residual <= tol
    double res;           // the last residual
};
constexpr int kLoopHist = 2048;           // residual history capacity of a device-side loop

// Device-side state of one extrapolation (CholeskyQR2 pass-1 results).
struct ExtrapInfo {
    int done, a, dep, pad;
    double D[kMaxQ + 1];
    double R1h[(kMaxQ + 1) * (kMaxQ + 1)];
    double R1p[(kMaxQ + 1) * (kMaxQ + 1)];
    double R1pinv[kMaxQ + 1];
};

// Sets the message returned by igamg_last_error() on this thread.
void set_last_error(const char* msg);
inline void set_last_error(const std::string& msg) { set_last_error(msg.c_str()); }

// Learned post-smoother network (cnn.cu): workspace for an image of `pixels`
// pixels; y (+)= network(r) for a batch x H x W image.
size_t cnn_workspace_bytes(long long pixels);
// raises the network kernels' shared-memory limit on the current device (outside capture)
void cnn_prepare();
void cnn_forward(cudaStream_t st, int B, int H, int W, const float* r, const float* w, float* y, int accumulate,
                 void* ws);

// Launch accounting (kernels enqueued by this thread).
void count_launch(long long n = 1);
long long launch_count();

// Programmatic dependent launch.  The V-cycle is a chain of short dependent
// kernels whose cost is dominated by the gap between one grid's end and the
// next one's start.  With overlap on, each kernel of the chain is launched
// with programmatic stream serialisation: its CTAs may be scheduled while the
// previous kernel on the stream is still running, and pdl_enter() holds them
// until that kernel has completed and its writes are visible, then lets the
// next kernel be scheduled.  Every such kernel calls pdl_enter() before its
// first access to memory that a kernel writes (before it, only operator data
// uploaded at assembly is read).  Kernels that call pdl_enter() behave
// exactly as before when launched normally.
// Process-wide switch, read when a launch is enqueued or a graph captured.
bool launch_overlap();
void set_launch_overlap(bool on);
// Launches enqueued (and graphs captured) by this thread while one of these
// is alive never overlap.  Batched solves use it: with 128 streams in flight,
// CTAs parked at the wait hold SM slots that other problems' kernels could
// run in (measured 260 -> 280 ms on 256 problems with overlap).
struct NoOverlapScope {
    NoOverlapScope();
    ~NoOverlapScope();
    NoOverlapScope(const NoOverlapScope&) = delete;
    NoOverlapScope& operator=(const NoOverlapScope&) = delete;
};

// Per-launch timing for measurement (igamg_profile_start / igamg_profile_stop):
// while a profile is active on this thread, launch_chained brackets each
// launch with CUDA events on its stream (not during stream capture), and the
// stop call reads the durations.  Off by default; adds nothing then.
bool profiling();
cudaEvent_t profile_before(cudaStream_t s);
void profile_after(cudaStream_t s, const void* func, dim3 grid, cudaEvent_t e0);
void profile_start();
long profile_stop(int cap, char* names, int name_len, double* us, int* grid);

#ifdef __CUDACC__
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// kern<<<grid, block, smem, s>>>(args...), with programmatic stream
// serialisation when overlap is on.  kern must call pdl_enter() as described
// above.
template <typename... KArgs, typename... Args>
inline void launch_chained(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                           Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = launch_overlap() ? 1 : 0;
    cudaEvent_t e0 = profiling() ? profile_before(s) : nullptr;
    cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
    if (e0) profile_after(s, (const void*)kern, grid, e0);
}
#endif

namespace dev {

// Raise every kernel's dynamic shared-memory limit on the current device
// (once per device; must run outside stream capture).
void prepare_kernels();
void prepare_tail_kernels(int optin);

// Largest single-CTA shared-memory size for the coarse tail on this device.
size_t tail_smem_limit();

// Levels lc..0 of one 2D V-cycle (pre-smoothing, residual, restriction,
// coarsest solve, prolongation, post-smoothing) in one CTA, starting from
// x = 0 on every level: reads level lc's right side b, writes its x.
// Smoothing is multicolour Gauss-Seidel, or weighted Jacobi with weight omega
// when jacobi != 0.
template <typename T>
void coarse_tail(cudaStream_t s, const TailView<T>& V, const T* b, T* x, int jacobi = 0, T omega = 0);

// The same on one thread-block cluster (ClusterTailView).  Host side:
// cluster_tail_fits tells whether a view's cluster can be resident on this
// device (shared memory and cluster size).
template <typename T>
void cluster_tail(cudaStream_t s, const ClusterTailView<T>& V, const T* b, T* x, int jacobi = 0, T omega = 0);
template <typename T>
bool cluster_tail_fits(const ClusterTailView<T>& V);
// Fills V's image buffer img (ctas x img16 uint4, device memory) with every
// CTA's static shared memory; synchronous, outside stream capture.
template <typename T>
cudaError_t cluster_tail_image(const ClusterTailView<T>& V, uint4* img);

// The 3D form (ClusterTail3View): levels lc..0 of an FP32 3D V-cycle.
template <typename T>
void cluster_tail3(cudaStream_t s, const ClusterTail3View<T>& V, const T* b, T* x, int jacobi = 0, T omega = 0);
template <typename T>
bool cluster_tail3_fits(const ClusterTail3View<T>& V);
template <typename T>
cudaError_t cluster_tail3_image(const ClusterTail3View<T>& V, uint4* img);

// T_M = (I (x) M_x) x, T_K = (I (x) K_x) x row by row.  With add != nullptr the
// row is first replaced by x + add (written to x_out), with nS > 0 by
// sum_j gamma[j] S_j (written to x_out).
template <typename T, typename A>
void xpass(cudaStream_t s, const LevelView<T>& L, const T* x, T* x_out, const A* add,
           int nS, const double* gamma, const T* S, size_t ldS, T* TM, T* TK);

// One multicolour Gauss-Seidel sweep (all (p+1)^dim colours): with sy ==
// nullptr as (p+1)^(dim-1) row-phase launches, else in one launch whose rows
// wait on their earlier-phase neighbours through *sy (same results); cap
// bounds the threads of a row CTA (0: the default).
template <typename T>
void gs_sweep(cudaStream_t s, int dim, const LevelView<T>& L, bool descending, T* x,
              const T* b, T* TM, T* TK, int cap = 0, const SweepSync* sy = nullptr);

// One weighted-Jacobi sweep x += omega D^{-1} (b - A x) (the paper's smoother,
// Sec. 4) from the row partial sums TM, TK of x, then the sums of the new x:
// in 2D written to TMo, TKo (one kernel; must not alias TM, TK), in 3D back
// to TM, TK (a second kernel; TMo, TKo unused).
template <typename T>
void jacobi_sweep(cudaStream_t s, int dim, const LevelView<T>& L, T omega, T* x, const T* b, T* TM, T* TK,
                  T* TMo, T* TKo);

// r = b - A x from the row partial sums; optional per-row partial ||r||^2.
// In 3D with scratch u, v (N each, not aliasing the other arguments) the
// residual is sum-factorised across y and z (two passes), else each row
// couples to its (2p+1)^2 neighbour rows.
template <typename T, typename R>
void residual(cudaStream_t s, int dim, const LevelView<T>& L, const T* b, const T* TM,
              const T* TK, R* r, double* partial, double* r64 = nullptr, T* u = nullptr, T* v = nullptr);

// Double-FP32 refinement update on the finest level (refine.cu; 2D and 3D rows):
// S_out = S_in + e and the row sums of e, (I (x) M_x) e and (I (x) K_x) e,
// each as a float pair (hi + lo) ...
void refine_xpass_df(cudaStream_t s, const DFView& D, const double* S_in, double* S_out, const float* e,
                     float* tm_h, float* tm_l, float* tk_h, float* tk_l);
// ... then r -= A e from those sums in float-pair arithmetic (FP64 r) and
// rf = float(r), the right side of the next FP32 V-cycle.
void refine_residual_df(cudaStream_t s, const DFView& D, const float* tm_h, const float* tm_l,
                        const float* tk_h, const float* tk_l, double* r, float* rf);
// The 3D form of the second step, sum-factorised as the FP64 3D residual:
// the y pass U = (I (x) M_y) T_M, V = (I (x) K_y) T_M + (I (x) M_y) T_K (float
// pairs, u = [Uh | Ul], v = [Vh | Vl], N floats each half), then
// r -= sum_dk K_z U + M_z V and rf = float(r).
void refine_residual_df3(cudaStream_t s, const DFView& D, const float* tm_h, const float* tm_l,
                         const float* tk_h, const float* tk_l, float* u, float* v, double* r, float* rf);

// coarse = P^T fine (tmp holds the intermediate axis passes).
template <typename T>
void restrict_(cudaStream_t s, int dim, const TransferView<T>& P, const T* fine, T* coarse,
               T* tmp1, T* tmp2,
               T* zero = nullptr, size_t nzero = 0);

// coarse = P^T (b - A x) (x given by its row sums T_M, T_K), optionally also
// clearing zero[0, nzero); 2D fuses the residual with the x-axis pass (r is
// not written), 3D goes through r.
template <typename T>
void residual_restrict(cudaStream_t s, int dim, const LevelView<T>& L, const TransferView<T>& X, const T* b,
                       const T* TM, const T* TK, T* r, T* coarse, T* tmp1, T* tmp2, T* zero, size_t nzero);

// x += P e, then refresh the row partial sums of x.
template <typename T>
void prolong_add(cudaStream_t s, int dim, const TransferView<T>& P, const LevelView<T>& Lf,
                 const T* e, T* x, T* TM, T* TK, T* tmp1, T* tmp2);

// e = A_0^{-1} r on the coarsest grid.
template <typename T>
void coarse_solve(cudaStream_t s, int dim, const CoarseView<T>& C, const T* r, T* e);

// End of one restart cycle of a device-side loop: cyc += 1, the residual
// res[0] into hist[cyc] (hist may be null) and st->res, the accuracy test,
// and the WHILE condition (1 = run another cycle).  A set error word ends the
// loop with kLoopTimeout.
void loop_step(cudaStream_t s, cudaGraphConditionalHandle h, LoopState* st, const double* res,
               const unsigned* err, double* hist);
// Sets the WHILE condition from st->code (1 while kLoopRunning).
void loop_init(cudaStream_t s, cudaGraphConditionalHandle h, const LoopState* st);
// The same kernel added to graph g as a root node.
cudaError_t add_loop_init_node(cudaGraph_t g, cudaGraphConditionalHandle h, const LoopState* st,
                               cudaGraphNode_t* node);

// Training pairs of the learned smoother: e = u - v with nblocks partial sums
// of e^2; then R = float(c r), E = float(c e), c = sqrt(n) / *enorm.
void diff_sumsq(cudaStream_t s, const double* u, const double* v, size_t n, double* e, double* partial,
                int nblocks);
void scale_pair(cudaStream_t s, const double* r, const double* e, const double* enorm, size_t n, float* R, float* E);

// ---- general operator (general.cu)
// r = b - A x (b null: r = A x), with gen_blocks(n) per-block
// partial sums of r^2 into partial when non-null (nparts = gen_blocks(n)).
int gen_blocks(size_t n);
void gen_residual(cudaStream_t s, const StencilView& V, const double* x, const double* b, double* r,
                  double* partial);
// One multicolour Gauss-Seidel sweep ((p+1)^2 colours in colour order, each
// colour from the x the previous ones left), descending = reversed order.
void gen_gs_sweep(cudaStream_t s, const StencilView& V, bool descending, double* x, const double* b);
// x += omega D^{-1} r.
void gen_jacobi_update(cudaStream_t s, const StencilView& V, double omega, const double* r, double* x);
// x += P e for a 2D transfer (row form of P).
void gen_prolong_add(cudaStream_t s, const TransferView<double>& X, const double* e, double* x);
// e = Ainv r, dense n x n (the coarsest level).
void gen_dense_apply(cudaStream_t s, const double* Ainv, int n, const double* r, double* e);

// Partial sums of squares of v (deterministic): nblocks partials.
void sumsq_partial(cudaStream_t s, const double* v, size_t n, double* partial, int nblocks);
// out[slot] = sqrt(sum partial) / (*denom), and non-finite flag.
void norm_final(cudaStream_t s, const double* partial, int nparts, const double* denom,
                double* out, int slot);

// RRE / MPE on S_0..S_{q+1} (stride ld): the gammas (q+2 entries) and
// q_used on the device, via two Gram passes (CholeskyQR2).
int gram_blocks(size_t n);
void gram_partial(cudaStream_t s, int q, const double* S, size_t ld, size_t n, double* partial,
                  int nblocks);
void extrap_gammas(cudaStream_t s, int q, int method, const double* S, size_t ld, size_t n,
                   double* partial, int nblocks, ExtrapInfo* info, double* gamma, int* qused);
// t = sum_{j=0}^{q+1} gamma_j S_j (elementwise).
void combine(cudaStream_t s, int q, const double* gamma, const double* S, size_t ld, size_t n,
             double* t);

// b = sum_k H[k](outer directions) ... : load vector from separable sine moments.
void rhs_sine(cudaStream_t s, int dim, const int* m, int modes, const double* gx_H,
              const double* gy, const double* gz, double* b);

template <typename T>
void fill_zero(cudaStream_t s, T* p, size_t n);

}  // namespace dev
}  // namespace igamg
