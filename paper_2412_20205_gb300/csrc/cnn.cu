// Learned post-smoother network: forward, gradient and Adam kernels.
//
// Three 3x3 zero-padded convolutions without biases, 1 -> 16 -> 16 -> 1
// channels, ReLU after the first two.  Images are batch x H x W (x fastest);
// the hidden activations are stored in BF16, channel-last (16 channels = 32
// bytes per pixel), arithmetic accumulates in FP32.  Weights are one FP32
// vector: W1[co][tap] (144), W2[co][ci][tap] (2304), W3[ci][tap] (144), with
// tap = 3 (dy + 1) + (dx + 1) reading pixel (y + dy, x + dx).
//
// Numerics everywhere: the input residual and the weights are rounded to
// BF16, products accumulate in FP32, hidden activations are stored in BF16.
//
// Inference (the solver's post-smoother) runs the whole network in one fused
// kernel per output tile with the activations in shared memory and all three
// layers on the tensor cores (implicit GEMMs, M = pixels: 1 -> 16 with K = 9
// taps, 16 -> 16 with K = 144, 16 -> 1 with K = 144).  Training runs the
// layers as separate kernels that keep both activations for the backward
// pass, every contraction on the tensor cores as well: the layer forwards,
// the input gradients and the weight gradients (implicit GEMMs over pixels).
#include "../../include/igamg.h"
#include "device.hpp"

#include <cuda_bf16.h>

#include <cstdint>
#include <string>

namespace igamg {
namespace cnn {

constexpr int C = 16;
constexpr int NW1 = C * 9, NW2 = C * C * 9, NW3 = C * 9;
constexpr int NW = NW1 + NW2 + NW3;
constexpr int kT = 256;

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

struct Shape {
    int B, H, W;
    __host__ __device__ long long pixels() const { return (long long)B * H * W; }
};

// A pixel with its row/column, decomposed once; nb(t) is its neighbour
// through tap t (-1 outside the image).
struct Pix {
    long long p;
    int y, x;
    __device__ __forceinline__ Pix(const Shape& s, long long q) : p(q) {
        const long long r = q / s.W;
        x = (int)(q - r * s.W);
        y = (int)(r % s.H);
    }
    __device__ __forceinline__ long long nb(const Shape& s, int t) const {
        const int dx = (t % 3) - 1, dy = (t / 3) - 1;
        const int xx = x + dx, yy = y + dy;
        if (xx < 0 || xx >= s.W || yy < 0 || yy >= s.H) return -1;
        return p + (long long)dy * s.W + dx;
    }
};
__device__ __forceinline__ long long neighbour(const Shape& s, long long p, int t) { return Pix(s, p).nb(s, t); }

__device__ __forceinline__ void load16(const __nv_bfloat16* a, long long p, float* v) {
    const uint4* q = reinterpret_cast<const uint4*>(a + p * C);
    const uint4 u0 = q[0], u1 = q[1];
    const __nv_bfloat162* h0 = reinterpret_cast<const __nv_bfloat162*>(&u0);
    const __nv_bfloat162* h1 = reinterpret_cast<const __nv_bfloat162*>(&u1);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 f0 = __bfloat1622float2(h0[i]), f1 = __bfloat1622float2(h1[i]);
        v[2 * i] = f0.x; v[2 * i + 1] = f0.y;
        v[8 + 2 * i] = f1.x; v[8 + 2 * i + 1] = f1.y;
    }
}

__device__ __forceinline__ void store16(__nv_bfloat16* a, long long p, const float* v) {
    uint4 u0, u1;
    __nv_bfloat162* h0 = reinterpret_cast<__nv_bfloat162*>(&u0);
    __nv_bfloat162* h1 = reinterpret_cast<__nv_bfloat162*>(&u1);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        h0[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        h1[i] = __floats2bfloat162_rn(v[8 + 2 * i], v[8 + 2 * i + 1]);
    }
    uint4* q = reinterpret_cast<uint4*>(a + p * C);
    q[0] = u0;
    q[1] = u1;
}

// ------------------------------------------------------------------ forward
// Tensor-core fragments (mma.sync.m16n8k16, BF16 inputs, FP32 accumulators).
// Per warp: a strip of 16 consecutive pixels (M) x 16 output channels (two N
// tiles of 8); K runs over the 9 taps x 16 input channels, one k16 step per
// tap.  A(m, k) = act[neighbour(pixel m, tap)][k], B(k, n) = weight(tap, k, n).
__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
}

// Implicit-GEMM 16 -> 16 convolution of one 16-pixel strip starting at p0:
// acc (C fragments of the two 8-channel N tiles) = sum over taps of
// act[neighbour(pixel, tap)] x Wt[tap].  Wt is the tap-major weight table in
// shared memory, Wt[t][k][n] (k = contracted channel, n = produced channel);
// FLIP reads the taps mirrored, which turns the convolution into its adjoint.
template <bool FLIP>
__device__ void conv16_strip(const Shape& s, long long p0, const __nv_bfloat16* __restrict__ act,
                             const float* Wt, float* acc /*[2][4]*/) {
    const int lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = 0.f;
    const long long P = s.pixels();
    const long long pa = p0 + g, pb = p0 + g + 8;
    const Pix xa(s, pa < P ? pa : 0), xb(s, pb < P ? pb : 0);
#pragma unroll 1
    for (int t = 0; t < 9; ++t) {
        const int tt = FLIP ? 8 - t : t;            // input gradient: flipped taps
        // A fragment: rows g and g+8 of the strip, columns 2tq, 2tq+1, 2tq+8, 2tq+9
        uint32_t a[4];
        {
            const long long qa = pa < P ? xa.nb(s, t) : -1;
            const long long qb = pb < P ? xb.nb(s, t) : -1;
            const __nv_bfloat162 z = __floats2bfloat162_rn(0.f, 0.f);
            const __nv_bfloat162* ra = qa >= 0 ? reinterpret_cast<const __nv_bfloat162*>(act + qa * C) : nullptr;
            const __nv_bfloat162* rb = qb >= 0 ? reinterpret_cast<const __nv_bfloat162*>(act + qb * C) : nullptr;
            __nv_bfloat162 v0 = ra ? ra[tq] : z, v1 = rb ? rb[tq] : z, v2 = ra ? ra[tq + 4] : z, v3 = rb ? rb[tq + 4] : z;
            a[0] = *reinterpret_cast<uint32_t*>(&v0);
            a[1] = *reinterpret_cast<uint32_t*>(&v1);
            a[2] = *reinterpret_cast<uint32_t*>(&v2);
            a[3] = *reinterpret_cast<uint32_t*>(&v3);
        }
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            // B fragment: rows (k) 2tq, 2tq+1 and 2tq+8, 2tq+9; column (n) g of tile nt
            const float* Wk = Wt + tt * C * C;
            const int n = nt * 8 + g;
            uint32_t b[2];
            b[0] = pack_bf16(Wk[(2 * tq) * C + n], Wk[(2 * tq + 1) * C + n]);
            b[1] = pack_bf16(Wk[(2 * tq + 8) * C + n], Wk[(2 * tq + 9) * C + n]);
            mma_bf16(acc + 4 * nt, a, b);
        }
    }
}

// a2 = relu(W2 * a1), tensor cores
__global__ void __launch_bounds__(kT) k_conv2(Shape s, const __nv_bfloat16* __restrict__ a1,
                                              const float* __restrict__ w, __nv_bfloat16* __restrict__ a2) {
    __shared__ float Wt[9 * C * C];                 // [tap][ci][co]
    for (int i = threadIdx.x; i < NW2; i += blockDim.x) {
        const int co = i / (C * 9), ci = (i / 9) % C, t = i % 9;
        Wt[(t * C + ci) * C + co] = w[NW1 + i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
    const long long P = s.pixels();
    const long long strips = (P + 15) / 16;
    for (long long st = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); st < strips;
         st += (long long)gridDim.x * (blockDim.x / 32)) {
        const long long p0 = st * 16;
        float acc[8];
        conv16_strip<false>(s, p0, a1, Wt, acc);
        // C fragment: rows g / g+8, columns nt*8 + 2tq, 2tq+1
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const long long p = p0 + g + 8 * h;
            if (p >= P) continue;
            __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(a2 + p * C);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
                o[nt * 4 + tq] = __floats2bfloat162_rn(fmaxf(acc[4 * nt + 2 * h], 0.f), fmaxf(acc[4 * nt + 2 * h + 1], 0.f));
        }
    }
}


// ------------------------------------------------------------------ fused inference
// One CTA pass computes the network on a TH x TW output tile: the residual is
// staged with a 3-pixel halo, layer-1 activations are computed on a 2-pixel
// halo and layer-2 activations on a 1-pixel halo (the halos are recomputed by
// the neighbouring tiles), all in shared memory; only r is read and y written
// in global memory.  The weight fragments are packed once per CTA of the
// persistent, grid-stride kernel.
namespace fused {
constexpr int TH = 16, TW = 32;
constexpr int RH = TH + 6, RW = TW + 6;
constexpr int A1H = TH + 4, A1W = TW + 4;
constexpr int A2H = TH + 2, A2W = TW + 2;
constexpr int NR = RH * RW, NA1 = A1H * A1W, NA2 = A2H * A2W, NO = TH * TW;
constexpr int S1 = (NA1 + 15) / 16, S2 = (NA2 + 15) / 16, S3 = NO / 16;
constexpr int NB2 = 9 * 2 * 32, NB3 = 9 * 32;     // per-lane B fragments (uint2) of layers 2, 3
constexpr int kSmem = NA1 * 32 + NA2 * 32 + NR * 4 + (NB2 + NB3) * 8;
constexpr int kThreads = 256, kWarps = kThreads / 32;
constexpr int kBlocks = 152 * 3;
static_assert(TW % 16 == 0, "output strips of 16 pixels run along x");
static_assert(kSmem <= 64 * 1024, "three CTAs per SM");
}  // namespace fused

// Byte offset of half h (channels 8h .. 8h+7) of pixel q in a shared-memory
// activation tile: 32 bytes per pixel, the two halves swapped when bit 2 of q
// is set, so that one half of eight consecutive pixels falls in eight distinct
// 16-byte bank groups (conflict-free ldmatrix phases).
__device__ __forceinline__ uint32_t act_off(int q, int h) {
    return (uint32_t)q * 32u + ((uint32_t)(h ^ ((q >> 2) & 1)) << 4);
}

// Four 8x8 BF16 matrices from shared memory; lanes 8i .. 8i+7 give the row
// addresses of matrix i, which lands in register i of every lane in the
// m16n8k16 A-fragment order.
__device__ __forceinline__ void ldsm_x4(uint32_t* a, uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                 : "r"(addr)
                 : "memory");
}

// Stores the two 16-row x 16-channel C fragments of a strip (after ReLU) as
// BF16 activations of pixels q0 + g and q0 + g + 8 of a tile whose pixel
// (0, 0) is image pixel (y0, x0); pixels outside the image store 0 (the zero
// padding of the next layer).
template <int WIDTH, int NPIX>
__device__ __forceinline__ void store_act(unsigned char* act, int q0, const float (*acc)[4], int y0, int x0,
                                          const Shape& s) {
    const int lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
        const int q = q0 + g + 8 * hh;
        if (q >= NPIX) continue;
        const int yy = y0 + q / WIDTH, xx = x0 + q % WIDTH;
        const bool in = yy >= 0 && yy < s.H && xx >= 0 && xx < s.W;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const float v0 = in ? fmaxf(acc[nt][2 * hh], 0.f) : 0.f;
            const float v1 = in ? fmaxf(acc[nt][2 * hh + 1], 0.f) : 0.f;
            *reinterpret_cast<__nv_bfloat162*>(act + act_off(q, nt) + 4 * tq) = __floats2bfloat162_rn(v0, v1);
        }
    }
}

__global__ void __launch_bounds__(fused::kThreads, 3)
k_forward_fused(Shape s, const float* __restrict__ r, const float* __restrict__ w, float* __restrict__ y,
                int accumulate) {
    pdl_enter();
    using namespace fused;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* a1 = smem;
    unsigned char* a2 = smem + NA1 * 32;
    float* sr = reinterpret_cast<float*>(smem + (NA1 + NA2) * 32);
    const uint32_t a1s = (uint32_t)__cvta_generic_to_shared(a1);
    const uint32_t a2s = (uint32_t)__cvta_generic_to_shared(a2);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, tq = lane & 3;

    // B fragments: B(k, n) = weight of input k (tap or channel) for output n.
    // Layer 1's stay in registers; layers 2 and 3 keep one uint2 per (tap,
    // N tile, lane) in shared memory, which leaves registers for three CTAs
    // per SM.
    uint2* Bt2 = reinterpret_cast<uint2*>(smem + (NA1 + NA2) * 32 + NR * 4);
    uint2* Bt3 = Bt2 + NB2;
    uint32_t b1[2][2];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        const int n = nt * 8 + g;
        b1[nt][0] = pack_bf16(w[n * 9 + 2 * tq], w[n * 9 + 2 * tq + 1]);
        b1[nt][1] = pack_bf16(tq == 0 ? w[n * 9 + 8] : 0.f, 0.f);             // taps 9..15 are padding
    }
    for (int idx = threadIdx.x; idx < NB2; idx += kThreads) {
        const int t = idx / 64, nt = (idx / 32) % 2, ln = idx % 32, lg = ln >> 2, lq = ln & 3;
        const float* Wn = w + NW1 + (nt * 8 + lg) * C * 9 + t;                 // W2[n][ci][t], ci stride 9
        Bt2[idx] = make_uint2(pack_bf16(Wn[(2 * lq) * 9], Wn[(2 * lq + 1) * 9]),
                              pack_bf16(Wn[(2 * lq + 8) * 9], Wn[(2 * lq + 9) * 9]));
    }
    for (int idx = threadIdx.x; idx < NB3; idx += kThreads) {
        const int t = idx / 32, ln = idx % 32, lg = ln >> 2, lq = ln & 3;
        const float* W3 = w + NW1 + NW2 + t;                                   // W3[ci][t]; output column 0 only
        Bt3[idx] = lg == 0 ? make_uint2(pack_bf16(W3[(2 * lq) * 9], W3[(2 * lq + 1) * 9]),
                                        pack_bf16(W3[(2 * lq + 8) * 9], W3[(2 * lq + 9) * 9]))
                           : make_uint2(0u, 0u);
    }

    const int tiles_x = (s.W + TW - 1) / TW, tiles_y = (s.H + TH - 1) / TH;
    const long long per_img = (long long)tiles_x * tiles_y;
    const long long ntiles = per_img * s.B;
    const int lm = (lane & 7) + ((lane >> 3) & 1) * 8, lh = lane >> 4;          // this lane's ldmatrix row
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long img = tile / per_img;
        const int rem = (int)(tile - img * per_img);
        const int oy = (rem / tiles_x) * TH, ox = (rem % tiles_x) * TW;
        const long long base = img * s.H * s.W;

        for (int i = threadIdx.x; i < NR; i += kThreads) {                      // residual, 3-pixel halo
            const int yy = oy - 3 + i / RW, xx = ox - 3 + i % RW;
            sr[i] = (yy >= 0 && yy < s.H && xx >= 0 && xx < s.W) ? r[base + (long long)yy * s.W + xx] : 0.f;
        }
        __syncthreads();

        // layer 1: K = 9 taps (padded to 16), on the 2-pixel halo region
        for (int st = warp; st < S1; st += kWarps) {
            uint32_t a[4];
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int q = min(st * 16 + g + 8 * hh, NA1 - 1);
                const float* rp = sr + (q / A1W) * RW + q % A1W;                // tap t reads rp[(t/3) RW + t%3]
                const int t0 = 2 * tq, t1 = 2 * tq + 1;
                a[hh] = pack_bf16(rp[(t0 / 3) * RW + t0 % 3], rp[(t1 / 3) * RW + t1 % 3]);
                a[2 + hh] = pack_bf16(tq == 0 ? rp[2 * RW + 2] : 0.f, 0.f);
            }
            float acc[2][4] = {};
            mma_bf16(acc[0], a, b1[0]);
            mma_bf16(acc[1], a, b1[1]);
            store_act<A1W, NA1>(a1, st * 16, acc, oy - 2, ox - 2, s);
        }
        __syncthreads();

        // layer 2: K = 9 taps x 16 channels, on the 1-pixel halo region
        for (int st = warp; st < S2; st += kWarps) {
            const int qm = min(st * 16 + lm, NA2 - 1);
            const int q1 = (qm / A2W) * A1W + qm % A2W;                         // a1 pixel under tap (0, 0)
            float acc[2][4] = {};
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                uint32_t a[4];
                ldsm_x4(a, a1s + act_off(q1 + (t / 3) * A1W + t % 3, lh));
                const uint2 w0 = Bt2[(t * 2) * 32 + lane], w1 = Bt2[(t * 2 + 1) * 32 + lane];
                const uint32_t bb0[2] = {w0.x, w0.y}, bb1[2] = {w1.x, w1.y};
                mma_bf16(acc[0], a, bb0);
                mma_bf16(acc[1], a, bb1);
            }
            store_act<A2W, NA2>(a2, st * 16, acc, oy - 1, ox - 1, s);
        }
        __syncthreads();

        // layer 3: K = 9 taps x 16 channels, N = 8 with only column 0 in use
        for (int st = warp; st < S3; st += kWarps) {
            const int q0 = st * 16, oyq = q0 / TW, ox0 = q0 % TW;
            const int q2 = oyq * A2W + ox0 + lm;                                // a2 pixel under tap (0, 0)
            float acc[4] = {};
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                uint32_t a[4];
                ldsm_x4(a, a2s + act_off(q2 + (t / 3) * A2W + t % 3, lh));
                const uint2 w3 = Bt3[t * 32 + lane];
                const uint32_t bb3[2] = {w3.x, w3.y};
                mma_bf16(acc, a, bb3);
            }
            if (tq == 0) {
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int yy = oy + oyq, xx = ox + ox0 + g + 8 * hh;
                    if (yy < s.H && xx < s.W) {
                        const long long i = base + (long long)yy * s.W + xx;
                        y[i] = accumulate ? y[i] + acc[2 * hh] : acc[2 * hh];
                    }
                }
            }
        }
        // The next pass rewrites sr (read only by layer 1), then a1 and a2,
        // each after a barrier that every warp reaches only when done here.
    }
}

// ------------------------------------------------------------------ backward
// gy = (y - e) / n, per-block partial sums of (y - e)^2
__global__ void __launch_bounds__(kT) k_loss(Shape s, const float* __restrict__ y, const float* __restrict__ e,
                                             float* __restrict__ gy, double* __restrict__ partial) {
    __shared__ double red[kT / 32];
    const long long P = s.pixels();
    const float inv = 1.0f / (float)P;
    double ss = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const float d = y[p] - e[p];
        gy[p] = d * inv;
        ss += (double)d * d;
    }
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)blockDim.x / 32; ++i) t += red[i];
        partial[blockIdx.x] = t;
    }
}

// g1 = (a1 > 0) . (W2^T g2): tensor cores with flipped taps and transposed
// channel roles (contract over the produced channel)
__global__ void __launch_bounds__(kT) k_conv2_dgrad(Shape s, const __nv_bfloat16* __restrict__ g2,
                                                    const float* __restrict__ w, const __nv_bfloat16* __restrict__ a1,
                                                    __nv_bfloat16* __restrict__ g1) {
    __shared__ float Wt[9 * C * C];                 // [tap][co][ci]: contract over co, produce ci
    for (int i = threadIdx.x; i < NW2; i += blockDim.x) {
        const int co = i / (C * 9), ci = (i / 9) % C, t = i % 9;
        Wt[(t * C + co) * C + ci] = w[NW1 + i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
    const long long P = s.pixels();
    const long long strips = (P + 15) / 16;
    for (long long st = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); st < strips;
         st += (long long)gridDim.x * (blockDim.x / 32)) {
        const long long p0 = st * 16;
        float acc[8];
        conv16_strip<true>(s, p0, g2, Wt, acc);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const long long p = p0 + g + 8 * h;
            if (p >= P) continue;
            const __nv_bfloat162* am = reinterpret_cast<const __nv_bfloat162*>(a1 + p * C);
            __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(g1 + p * C);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const float2 m = __bfloat1622float2(am[nt * 4 + tq]);
                o[nt * 4 + tq] = __floats2bfloat162_rn(m.x > 0.f ? acc[4 * nt + 2 * h] : 0.f,
                                                       m.y > 0.f ? acc[4 * nt + 2 * h + 1] : 0.f);
            }
        }
    }
}

// ------------------------------------------------------------------ training on the tensor cores
// The remaining contractions of the training step as implicit GEMMs on
// mma.sync.m16n8k16 (BF16 operands, FP32 accumulation), one warp per strip
// of 16 consecutive pixels.

// BF16 bits of channel c of pixel q of a channel-last activation (0 outside).
__device__ __forceinline__ uint32_t act_bits(const __nv_bfloat16* a, long long q, int c) {
    return q >= 0 ? (uint32_t)__bfloat16_as_ushort(a[q * C + c]) : 0u;
}
__device__ __forceinline__ uint32_t f_bits(float v) { return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v)); }
__device__ __forceinline__ uint32_t pk(uint32_t lo, uint32_t hi) { return lo | (hi << 16); }

// Nine-tap layers with one input channel: out[p][c] = sum_t w9[c][t] in[q(p, t)],
// M = the strip's pixels, N = 16 channels (two n-tiles), K = 9 taps padded to
// 16.  FLIP reads in[] through the mirrored tap (the adjoint of a 16 -> 1
// layer).  MODE 0 (layer 1 forward): out = relu(.); MODE 1 (layer 3 input
// gradient): out = . where mask[p][c] > 0, else 0.
template <bool FLIP, int MODE>
__global__ void __launch_bounds__(kT) k_tap9_tc(Shape s, const float* __restrict__ in, const float* __restrict__ w9,
                                                const __nv_bfloat16* __restrict__ mask, __nv_bfloat16* __restrict__ out) {
    __shared__ float W[C * 9];
    for (int i = threadIdx.x; i < C * 9; i += blockDim.x) W[i] = w9[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
    // B fragments (k = tap, n = channel), fixed for the kernel
    uint32_t b[2][2];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        const int c = nt * 8 + g;
        b[nt][0] = pk(f_bits(W[c * 9 + 2 * tq]), f_bits(W[c * 9 + 2 * tq + 1]));
        b[nt][1] = tq == 0 ? pk(f_bits(W[c * 9 + 8]), 0u) : 0u;
    }
    const long long P = s.pixels();
    const long long strips = (P + 15) / 16;
    for (long long st = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); st < strips;
         st += (long long)gridDim.x * (blockDim.x / 32)) {
        const long long p0 = st * 16;
        const long long pa = p0 + g, pb = p0 + g + 8;
        const Pix xa(s, pa < P ? pa : 0), xb(s, pb < P ? pb : 0);
        auto v = [&](const Pix& x, long long p, int t) -> uint32_t {
            if (p >= P || t > 8) return 0u;
            const long long q = x.nb(s, FLIP ? 8 - t : t);
            return q >= 0 ? f_bits(in[q]) : 0u;
        };
        uint32_t a[4];
        a[0] = pk(v(xa, pa, 2 * tq), v(xa, pa, 2 * tq + 1));
        a[1] = pk(v(xb, pb, 2 * tq), v(xb, pb, 2 * tq + 1));
        a[2] = pk(v(xa, pa, 2 * tq + 8), 0u);
        a[3] = pk(v(xb, pb, 2 * tq + 8), 0u);
        float acc[2][4] = {};
        mma_bf16(acc[0], a, b[0]);
        mma_bf16(acc[1], a, b[1]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const long long p = p0 + g + 8 * h;
            if (p >= P) continue;
            __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(out + p * C);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                float v0 = acc[nt][2 * h], v1 = acc[nt][2 * h + 1];
                if (MODE == 0) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                } else {
                    const float2 m = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(mask + p * C)[nt * 4 + tq]);
                    v0 = m.x > 0.f ? v0 : 0.f;
                    v1 = m.y > 0.f ? v1 : 0.f;
                }
                o[nt * 4 + tq] = __floats2bfloat162_rn(v0, v1);
            }
        }
    }
}

// y = W3 * a2 (layer 3, 16 -> 1) with the 16 -> 16 strip contraction: the
// weight table holds W3 in output column 0 and zeros elsewhere.
__global__ void __launch_bounds__(kT) k_conv3_tc(Shape s, const __nv_bfloat16* __restrict__ a2, const float* __restrict__ w,
                                                 float* __restrict__ y) {
    __shared__ float Wt[9 * C * C];                 // [tap][ci][n], n = 0 only
    for (int i = threadIdx.x; i < 9 * C * C; i += blockDim.x) {
        const int t = i / (C * C), ci = (i / C) % C, n = i % C;
        Wt[i] = n == 0 ? w[NW1 + NW2 + ci * 9 + t] : 0.f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
    const long long P = s.pixels();
    const long long strips = (P + 15) / 16;
    for (long long st = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); st < strips;
         st += (long long)gridDim.x * (blockDim.x / 32)) {
        const long long p0 = st * 16;
        float acc[8];
        conv16_strip<false>(s, p0, a2, Wt, acc);
        if (tq == 0) {                              // column 0 of n-tile 0: rows g and g + 8
            if (p0 + g < P) y[p0 + g] = acc[0];
            if (p0 + g + 8 < P) y[p0 + g + 8] = acc[2];
        }
    }
}

// Weight gradients on the tensor cores, K = pixels.  Per strip of 16 pixels:
//   dW2[co][ci][t] += sum_p g2[p][co] a1[q(p,t)][ci]   (M = co, N = (t, ci): 18 n-tiles)
//   dW1[co][t]     += sum_p g1[p][co] r[q(p,t)]        (M = co, N = t: 2 n-tiles)
//   dW3[c][t]      += sum_q a2[q][c] gy[q(q,8-t)]      (the same sum as sum_p gy[p] a2[q(p,t)][c],
//                                                        indexed by the pixel a2 is read at)
// The A operands (channel x pixel) are the transposed channel-last tensors.
// Each warp keeps its sums over a fixed sequence of strips and writes them to
// its own row of `partial`; k_reduce adds the rows in fixed order, so the
// gradient is deterministic.
constexpr int kWgradWarpsPerBlock = kT / 32;

__global__ void __launch_bounds__(kT) k_wgrad_tc(Shape s, const float* __restrict__ r, const __nv_bfloat16* __restrict__ a1,
                                                 const __nv_bfloat16* __restrict__ a2, const __nv_bfloat16* __restrict__ g1,
                                                 const __nv_bfloat16* __restrict__ g2, const float* __restrict__ gy,
                                                 float* __restrict__ partial) {
    const int lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
    const int warp = blockIdx.x * kWgradWarpsPerBlock + (threadIdx.x >> 5);
    const int nwarps = gridDim.x * kWgradWarpsPerBlock;
    float acc2[18][4] = {}, acc1[2][4] = {}, acc3[2][4] = {};
    const long long P = s.pixels();
    const long long strips = (P + 15) / 16;
    for (long long st = warp; st < strips; st += nwarps) {
        const long long p0 = st * 16;
        long long pk4[4] = {p0 + 2 * tq, p0 + 2 * tq + 1, p0 + 2 * tq + 8, p0 + 2 * tq + 9};
        Pix px[4] = {Pix(s, 0), Pix(s, 0), Pix(s, 0), Pix(s, 0)};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (pk4[i] < P) px[i] = Pix(s, pk4[i]);
            else pk4[i] = -1;
        }
        // A fragments (m = channel g / g + 8, k = pixels 2tq, 2tq+1 / 2tq+8, 2tq+9)
        auto afrag = [&](const __nv_bfloat16* x, uint32_t* a) {
            a[0] = pk(act_bits(x, pk4[0], g), act_bits(x, pk4[1], g));
            a[1] = pk(act_bits(x, pk4[0], g + 8), act_bits(x, pk4[1], g + 8));
            a[2] = pk(act_bits(x, pk4[2], g), act_bits(x, pk4[3], g));
            a[3] = pk(act_bits(x, pk4[2], g + 8), act_bits(x, pk4[3], g + 8));
        };
        uint32_t A2[4], A1[4], A3[4];
        afrag(g2, A2);
        afrag(g1, A1);
        afrag(a2, A3);
        auto nbq = [&](int i, int t) -> long long { return pk4[i] >= 0 ? px[i].nb(s, t) : -1; };
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            long long q[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) q[i] = nbq(i, t);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t b[2];
                b[0] = pk(act_bits(a1, q[0], 8 * h + g), act_bits(a1, q[1], 8 * h + g));
                b[1] = pk(act_bits(a1, q[2], 8 * h + g), act_bits(a1, q[3], 8 * h + g));
                mma_bf16(acc2[2 * t + h], A2, b);
            }
        }
        // dW1 and dW3: n = tap (g in n-tile 0, tap 8 at column 0 of n-tile 1)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int tap = nt == 0 ? g : (g == 0 ? 8 : -1);
            uint32_t b1[2] = {0u, 0u}, b3[2] = {0u, 0u};
            if (tap >= 0) {
                long long q1[4], q3[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    q1[i] = nbq(i, tap);
                    q3[i] = nbq(i, 8 - tap);
                }
                auto rv = [&](long long q) { return q >= 0 ? f_bits(r[q]) : 0u; };
                auto gv = [&](long long q) { return q >= 0 ? f_bits(gy[q]) : 0u; };
                b1[0] = pk(rv(q1[0]), rv(q1[1]));
                b1[1] = pk(rv(q1[2]), rv(q1[3]));
                b3[0] = pk(gv(q3[0]), gv(q3[1]));
                b3[1] = pk(gv(q3[2]), gv(q3[3]));
            }
            mma_bf16(acc1[nt], A1, b1);
            mma_bf16(acc3[nt], A3, b3);
        }
    }
    // C fragments: rows (co / c) g and g + 8, columns 2tq, 2tq + 1 of each n-tile
    float* row = partial + (size_t)warp * NW;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
        const int co = g + 8 * hh;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
#pragma unroll
            for (int t = 0; t < 9; ++t)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int ci = 8 * h + 2 * tq + j;
                    row[NW1 + (co * C + ci) * 9 + t] = acc2[2 * t + h][2 * hh + j];
                }
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const int tap = nt * 8 + 2 * tq + j;
                if (tap < 9) {
                    row[co * 9 + tap] = acc1[nt][2 * hh + j];
                    row[NW1 + NW2 + co * 9 + tap] = acc3[nt][2 * hh + j];
                }
            }
        }
    }
}

__global__ void k_reduce(const float* __restrict__ partial, int nblocks, const double* __restrict__ lpart,
                         int nl, long long P, float* __restrict__ grad, float* __restrict__ loss) {
    for (int wi = blockIdx.x * blockDim.x + threadIdx.x; wi < NW; wi += gridDim.x * blockDim.x) {
        float a = 0.f;
        for (int b = 0; b < nblocks; ++b) a += partial[(size_t)b * NW + wi];
        grad[wi] = a;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && loss) {
        double t = 0.0;
        for (int i = 0; i < nl; ++i) t += lpart[i];
        *loss = (float)(0.5 * t / (double)P);
    }
}

__global__ void k_adam(int n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// ------------------------------------------------------------------ host side
static int grid(long long n, int per) {
    long long g = (n + per - 1) / per;
    if (g > 152 * 8) g = 152 * 8;
    return (int)(g < 1 ? 1 : g);
}
constexpr int kWgradBlocks = 152;
constexpr int kWgradRows = kWgradBlocks * kWgradWarpsPerBlock;      // partial-sum rows (one per warp)

size_t workspace_bytes(long long P) {
    const size_t act = ((size_t)P * C * 2 + 255) / 256 * 256;      // one BF16 channel-last tensor
    return 4 * act + ((size_t)P * 4 + 255) / 256 * 256 + (size_t)kWgradRows * NW * 4 + 8 * 1024 * 8 + 1024;
}

struct WS {
    __nv_bfloat16 *a1, *a2, *g1, *g2;
    float* gy;
    float* partial;
    double* lpart;
};

static WS carve_ws(void* base, long long P) {
    char* p = (char*)base;
    const size_t act = ((size_t)P * C * 2 + 255) / 256 * 256;
    WS w;
    w.a1 = (__nv_bfloat16*)p; p += act;
    w.a2 = (__nv_bfloat16*)p; p += act;
    w.g1 = (__nv_bfloat16*)p; p += act;
    w.g2 = (__nv_bfloat16*)p; p += act;
    w.gy = (float*)p; p += ((size_t)P * 4 + 255) / 256 * 256;
    w.partial = (float*)p; p += (size_t)kWgradRows * NW * 4;
    w.lpart = (double*)p;
    return w;
}

// Forward pass that keeps both hidden activations in the workspace (training).
void forward_stored(cudaStream_t st, Shape s, const float* r, const float* w, float* y, void* ws) {
    WS W = carve_ws(ws, s.pixels());
    const long long P = s.pixels();
    const int gs = grid((P + 15) / 16, kT / 32);
    k_tap9_tc<false, 0><<<gs, kT, 0, st>>>(s, r, w, nullptr, W.a1);
    k_conv2<<<gs, kT, 0, st>>>(s, W.a1, w, W.a2);
    k_conv3_tc<<<gs, kT, 0, st>>>(s, W.a2, w, y);
    count_launch(3);
}

// Inference: y = net(r), or y += net(r) with accumulate; one fused launch.
// The fused kernel needs more than the default 48 KB of dynamic shared memory;
// the limit is raised once per device, outside any stream capture.
void prepare(int optin) {
    (void)optin;
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || done[dev]) return;
    cudaFuncSetAttribute(k_forward_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, fused::kSmem);
    done[dev] = true;
}

void forward(cudaStream_t st, Shape s, const float* r, const float* w, float* y, int accumulate) {
    const long long tiles = (long long)s.B * ((s.H + fused::TH - 1) / fused::TH) * ((s.W + fused::TW - 1) / fused::TW);
    const int blocks = (int)(tiles < fused::kBlocks ? tiles : fused::kBlocks);
    launch_chained(k_forward_fused, blocks, fused::kThreads, fused::kSmem, st, s, r, w, y, accumulate);
    count_launch();
}

void gradient(cudaStream_t st, Shape s, const float* r, const float* e, const float* w, float* grad, float* loss,
              float* y, void* ws) {
    WS W = carve_ws(ws, s.pixels());
    const long long P = s.pixels();
    forward_stored(st, s, r, w, y, ws);
    const int gl = grid(P, kT) > 1024 ? 1024 : grid(P, kT);
    k_loss<<<gl, kT, 0, st>>>(s, y, e, W.gy, W.lpart);
    const int gs = grid((P + 15) / 16, kT / 32);
    k_tap9_tc<true, 1><<<gs, kT, 0, st>>>(s, W.gy, w + NW1 + NW2, W.a2, W.g2);
    k_conv2_dgrad<<<gs, kT, 0, st>>>(s, W.g2, w, W.a1, W.g1);
    k_wgrad_tc<<<kWgradBlocks, kT, 0, st>>>(s, r, W.a1, W.a2, W.g1, W.g2, W.gy, W.partial);
    k_reduce<<<(NW + 255) / 256, 256, 0, st>>>(W.partial, kWgradRows, W.lpart, gl, P, grad, loss);
    count_launch(5);
}

}  // namespace cnn

size_t cnn_workspace_bytes(long long pixels) { return cnn::workspace_bytes(pixels); }
void cnn_prepare() { cnn::prepare(0); }
void cnn_forward(cudaStream_t st, int B, int H, int W, const float* r, const float* w, float* y, int accumulate,
                 void* ws) {
    (void)ws;
    cnn::forward(st, cnn::Shape{B, H, W}, r, w, y, accumulate);
}

}  // namespace igamg

using namespace igamg;

extern "C" {

int igamg_cnn_num_weights(void) { return cnn::NW; }

size_t igamg_cnn_workspace_bytes(int batch, int H, int W) {
    if (batch < 1 || H < 1 || W < 1) return 0;
    return cnn::workspace_bytes((long long)batch * H * W) + (size_t)batch * H * W * 4 + 256;
}

igamg_status igamg_cnn_forward(int batch, int H, int W, const float* d_r, const float* d_w, float* d_y, void* d_ws,
                               size_t ws_bytes, void* stream) {
    if (batch < 1 || H < 1 || W < 1 || !d_r || !d_w || !d_y || !d_ws) {
        set_last_error("bad network arguments");
        return IGAMG_EINVAL;
    }
    if (ws_bytes < igamg_cnn_workspace_bytes(batch, H, W) || ((uintptr_t)d_ws & 255)) {
        set_last_error("network workspace too small or unaligned");
        return IGAMG_ENOMEM;
    }
    cnn::prepare(0);
    cnn::forward((cudaStream_t)stream, cnn::Shape{batch, H, W}, d_r, d_w, d_y, 0);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_last_error(std::string("network forward: ") + cudaGetErrorString(e)); return IGAMG_ECUDA; }
    return IGAMG_OK;
}

igamg_status igamg_cnn_grad(int batch, int H, int W, const float* d_r, const float* d_e, const float* d_w,
                            float* d_grad, float* d_loss, void* d_ws, size_t ws_bytes, void* stream) {
    if (batch < 1 || H < 1 || W < 1 || !d_r || !d_e || !d_w || !d_grad || !d_ws) {
        set_last_error("bad network arguments");
        return IGAMG_EINVAL;
    }
    if (ws_bytes < igamg_cnn_workspace_bytes(batch, H, W) || ((uintptr_t)d_ws & 255)) {
        set_last_error("network workspace too small or unaligned");
        return IGAMG_ENOMEM;
    }
    const long long P = (long long)batch * H * W;
    float* y = (float*)((char*)d_ws + cnn::workspace_bytes(P));
    cnn::gradient((cudaStream_t)stream, cnn::Shape{batch, H, W}, d_r, d_e, d_w, d_grad, d_loss, y, d_ws);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_last_error(std::string("network gradient: ") + cudaGetErrorString(e)); return IGAMG_ECUDA; }
    return IGAMG_OK;
}

igamg_status igamg_adam_step(int n, float* d_w, const float* d_g, float* d_m, float* d_v, int step, float lr, float b1,
                             float b2, float eps, void* stream) {
    if (n < 1 || step < 1 || !d_w || !d_g || !d_m || !d_v) {
        set_last_error("bad Adam arguments");
        return IGAMG_EINVAL;
    }
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    cnn::k_adam<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(n, d_w, d_g, d_m, d_v, lr, b1, b2, eps, c1, c2);
    count_launch();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_last_error(std::string("Adam: ") + cudaGetErrorString(e)); return IGAMG_ECUDA; }
    return IGAMG_OK;
}

}  // extern "C"
